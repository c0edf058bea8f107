// Declarations shared by the kernel translation units and the host API.
#pragma once
#include <algorithm>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpca {

// FIN_FG: gradient + penalty at the trial point; FIN_FG_RAW: same objective, but GU/GV get
// the raw products D V and D^T U; FIN_APPLY: plain products D Bv, D^T Bu, no objective.
enum { FIN_FG = 0, FIN_APPLY = 1, FIN_FG_RAW = 2 };

struct FinArgs {
  int m, n, B, mpad, nrb, ncs, nctas;
  int gu;  // blocks [0, gu) handle the m x B side; the rest the n x B side
  const float* PU;
  const float* PV;
  const double* Ppsi;  // per-CTA psi sums of the fused pass, float-float pairs (ff_store)
  int mode;  // FIN_*
  int side;  // 0 both sides, 1 only the m x B side (GU), 2 only the n x B side (GV)
  const float* U;
  const float* V;
  const float* dU;
  const float* dV;
  float alpha;
  const double* alpha_dev;  // when non-null, the step is read from here
  const int* gate;          // when non-null and *gate == 0 the launch does nothing
  double lam_L;
  float lam_f;  // lam_L as float32 (converted on the host)
  float* GU;  // m x B (ld m): G_U (fg) or D Bv (apply)
  float* GV;  // n x B (ld n): G_V (fg) or D^T Bu (apply)
  float* Ut;  // optional copy of the trial point
  float* Vt;
  const float* DU;  // optional direction for g.d
  const float* DV;
  double* blk;              // [3 * gridDim.x] block partials (float-float pairs, ff_store)
  unsigned int* counter;    // zero between launches (reset by the last block)
  double* out;              // [4]: f, g.d, ||g||^2, ||x_t||^2
  // Row shard of a partitioned problem (rpca_fg_rows): the n x B side writes the raw partial
  // D^T U (no lam_L V) and adds nothing to the sums (V is shared by every shard).
  int vpart;
  // The m x B side in float4 (four consecutive elements per thread): set by fin_vec4 when m
  // and mpad are multiples of 4 and every m x B array the assembly touches is 16-byte aligned.
  int vec4;
};

inline bool fin_aligned16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline int fin_vec4(const FinArgs& f) {
  return f.m % 4 == 0 && f.mpad % 4 == 0 && fin_aligned16(f.PU) && fin_aligned16(f.U) && fin_aligned16(f.dU) &&
         fin_aligned16(f.DU) && fin_aligned16(f.Ut) && fin_aligned16(f.GU);
}

// Finalize grid: FIN_EPT elements per thread of the m x B side (256 threads per block), 32
// elements (eight groups of 32 threads splitting the row-block partials, FIN_VB loads in
// flight per thread) per block on the n x B side.
constexpr int FIN_EPT = 4;
constexpr int FIN_VB = 16;
inline int fin_grid_u(int64_t m, int B) {
  return (int)std::max<int64_t>(1, (m * B + 256 * FIN_EPT - 1) / (256 * FIN_EPT));
}
inline int fin_grid_v(int64_t n, int B) { return (int)std::max<int64_t>(1, (n * B + 31) / 32); }

__global__ void finalize_kernel(FinArgs a);
__global__ void finalize_reduce_kernel(FinArgs a, int nblocks);
__global__ void pack_mask_kernel(const uint8_t* mask, int64_t ldmask, int m, int n, int wpad, uint32_t* bits);
__global__ void check_x_kernel(const float* X, int64_t ldx, const uint8_t* mask, int64_t ldmask, int m, int n,
                               unsigned long long* bad, unsigned long long* observed);

}  // namespace rpca
