// Instantiations of the fused kernel in fg mode for factor rank K = 1..8.
#include "fg_kernel.cuh"
#include "fg_variants.h"

namespace rpca {

template <int K, int R, int J>
static void reg(FgVariant (*tab)[2]) {
  tab[K][0] = FgVariant{(const void*)&fg_kernel<K, K, true, false, R, J>, R, J,
                        (const void*)&fg_group_kernel<K, K, true, false, R, J>};
  tab[K][1] = FgVariant{(const void*)&fg_kernel<K, K, true, true, R, J>, R, J};
}

void fg_register_same_small(FgVariant (*tab)[2]) {
  reg<1, 8, 4>(tab);
  reg<2, 8, 4>(tab);
  reg<3, 8, 4>(tab);
  reg<4, 8, 4>(tab);
  reg<5, 8, 4>(tab);
  reg<6, 8, 2>(tab);
  reg<7, 4, 2>(tab);
  reg<8, 4, 2>(tab);
}

}  // namespace rpca
