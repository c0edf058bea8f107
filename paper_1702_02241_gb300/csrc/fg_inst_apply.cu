// Instantiations of the fused kernel in apply mode: D Bv and D^T Bu for the certificate's
// spectral step (forming rank padded to 8 or 16, block width 8) and the sketch (no forming
// factors, block width 16).
#include "fg_kernel.cuh"
#include "fg_variants.h"

namespace rpca {

template <int K, int B, int R, int J>
static void reg(FgVariant (*tab)[2], int slot) {
  tab[slot][0] = FgVariant{(const void*)&fg_kernel<K, B, false, false, R, J>, R, J};
  tab[slot][1] = FgVariant{(const void*)&fg_kernel<K, B, false, true, R, J>, R, J};
}

// Slots: 0 -> (K=0, B=16), 1 -> (K=8, B=8), 2 -> (K=16, B=8).
void fg_register_apply(FgVariant (*tab)[2]) {
  reg<0, 16, 2, 1>(tab, 0);
  reg<8, 8, 4, 2>(tab, 1);
  reg<16, 8, 2, 2>(tab, 2);
}

}  // namespace rpca
