// Instantiations of the fused kernel in apply mode (products with the clipped residual D
// and other matrices): forming rank 0 (the sketch: D = -A*(X)), 8 or 16 (the certificate's
// spectral step, factors zero-padded), block width 8; both products (rpca_apply), only
// D Bv, or only D^T Bu (each Lanczos half-step and each sketch product needs one).
#include "fg_kernel.cuh"
#include "fg_variants.h"

namespace rpca {

template <int K, int R, int J, int SIDE>
static void reg(FgVariant (*tab)[3][2], int slot) {
  tab[slot][SIDE][0] = FgVariant{(const void*)&fg_kernel<K, 8, false, false, R, J, SIDE>, R, J};
  tab[slot][SIDE][1] = FgVariant{(const void*)&fg_kernel<K, 8, false, true, R, J, SIDE>, R, J};
}

// Slots: 0 -> K = 0, 1 -> K = 8, 2 -> K = 16.
void fg_register_apply(FgVariant (*tab)[3][2]) {
  reg<0, 4, 2, 0>(tab, 0);
  reg<0, 8, 1, 1>(tab, 0);
  reg<0, 8, 2, 2>(tab, 0);
  reg<8, 4, 2, 0>(tab, 1);
  reg<8, 8, 1, 1>(tab, 1);
  reg<8, 8, 1, 2>(tab, 1);
  reg<16, 2, 2, 0>(tab, 2);
  reg<16, 4, 1, 1>(tab, 2);
  reg<16, 4, 1, 2>(tab, 2);
}

// The sketch's products with 16 columns at a time (no forming factors), one pass over X for
// what two 8-column passes would do: tab[side][masked], sides 1 (D Bv) and 2 (D^T Bu).
template <int SIDE>
static void reg16(FgVariant (*tab)[2]) {
  tab[SIDE][0] = FgVariant{(const void*)&fg_kernel<0, 16, false, false, 8, 1, SIDE>, 8, 1};
  tab[SIDE][1] = FgVariant{(const void*)&fg_kernel<0, 16, false, true, 8, 1, SIDE>, 8, 1};
}

void fg_register_apply16(FgVariant (*tab)[2]) {
  reg16<1>(tab);
  reg16<2>(tab);
}

}  // namespace rpca
