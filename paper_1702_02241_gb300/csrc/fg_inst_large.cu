// Instantiations of the fused kernel in fg mode for factor rank K = 9..16.
#include "fg_kernel.cuh"
#include "fg_variants.h"

namespace rpca {

template <int K, int R, int J>
static void reg(FgVariant (*tab)[2]) {
  tab[K][0] = FgVariant{(const void*)&fg_kernel<K, K, true, false, R, J>, R, J,
                        (const void*)&fg_group_kernel<K, K, true, false, R, J>};
  tab[K][1] = FgVariant{(const void*)&fg_kernel<K, K, true, true, R, J>, R, J};
}

void fg_register_same_large(FgVariant (*tab)[2]) {
  reg<9, 4, 2>(tab);
  reg<10, 4, 2>(tab);
  reg<11, 4, 2>(tab);
  reg<12, 4, 2>(tab);
  reg<13, 2, 2>(tab);
  reg<14, 2, 2>(tab);
  reg<15, 2, 2>(tab);
  reg<16, 2, 2>(tab);
}

}  // namespace rpca
