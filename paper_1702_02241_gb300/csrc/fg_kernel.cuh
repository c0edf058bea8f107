// Fused evaluation of the Split-SPCP objective and gradient (paper Eq. Thm5 / Eq. 7,
// gradient from Sec. 3.2, masked form Sec. 6.2) in one pass over X.
//
// For a tile of X (rows [row0, row0+BM) x columns [col0, col0+BN)) a CTA forms
//   r_ij = (u_i . v_j) - x_ij,  d_ij = clip(r_ij, +-lam_S) (0 off the mask),
//   psi_ij = d_ij (r_ij - d_ij / 2)                       (Huber value, Sec. 1)
// and accumulates  PU = -(D Bv) over its columns,  PV = D^T Bu over its rows,  sum psi.
// In "fg" mode Bu = u and Bv = v (so PU, PV give the gradient terms D V and D^T U); in
// "apply" mode Bu, Bv are other matrices (the certificate's spectral step and the sketch).
// R = U V^T - X is never written to memory.
//
// Layout: X, U, V, Bu, Bv column-major.  One producer warp streams X (and the observation
// bitmap) into a ring of shared-memory stages with 2-D TMA tensor copies; WC consumer warps
// each own 32*R rows of the tile (R rows per lane, as float2 pairs for the packed fp32x2
// FMA pipe) and walk the tile's columns.  Per lane the factor rows live in registers for
// the whole tile; the gradient rows (D Bv) accumulate in registers over all columns; the
// column sums (D^T Bu) are reduced across lanes with a shuffle reduce-scatter into a
// per-warp shared-memory slab, and across warps once at the end of the tile, in a fixed
// order (bitwise deterministic).
#pragma once
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace rpca {

struct FgArgs {
  int m, n;
  int mpad;  // leading dimension of PU (multiple of 4, >= m)
  const float* U;   // m x K (ld m): forming factor, trial point U + alpha dU
  const float* V;   // n x K (ld n)
  const float* dU;  // may be null
  const float* dV;  // may be null
  float alpha;
  const double* alpha_dev;  // when non-null, the step is read from here (CUDA-graph replay)
  const int* gate;          // when non-null and *gate == 0 the launch does nothing
  const float* BU;  // apply mode: m x B (ld m)
  const float* BV;  // apply mode: n x B (ld n)
  float lam_S;
  int nrb, ncs, BN;  // row blocks, column splits, columns per split (multiple of 8)
  int nstage;        // pipeline depth (2 .. FG_NSTAGE)
  float* PU;         // [ncs][B][mpad]  -(D Bv) partial sums over a CTA's columns
  float* PV;         // [nrb][B][n]      D^T Bu partial sums over a CTA's rows
  double* Ppsi;      // [nrb*ncs]        sum of psi over a CTA's tile (float-float pair, ff_store)
  int* err;          // device status word (error bits)
  const float* xscale;  // FP8 storage: per-column scales (x = stored value * scale)
  int npass;         // tensor-core form: row passes of 32 * (consumer warps) rows per CTA
  // Failure injection (rpca_inject_fault): the producer issues no copies, so the consumers'
  // bounded waits run out (after wait_ns, 0 = the default limit) and report a status bit.
  int starve;
  unsigned long long wait_ns;
};

// Storage type of X read by an instantiation: float32, bfloat16, or FP8 E4M3 with a
// per-column scale.
enum { FG_X_F32 = 0, FG_X_BF16 = 1, FG_X_E4M3 = 2 };
__host__ __device__ constexpr int fg_x_bytes(int xt) { return xt == FG_X_F32 ? 4 : (xt == FG_X_BF16 ? 2 : 1); }

constexpr int FG_BJ = 4;      // columns per pipeline stage
constexpr int FG_NSTAGE = 8;  // maximum pipeline depth

struct FgSmem {
  size_t x_off, m_off, v_off, cs_off, tr_off, sc_off, bar_off, scr_off, total;
};

constexpr int FG_TR_LD = 36;  // row stride (floats) of the column-sum transposition buffer

// Observation bitmap of one stage: one TMA box per CTA, {WC * R words, BJ columns}, so the
// box's x coordinate row0 / 32 is a multiple of WC * R >= 4 words (16 bytes).
__host__ __device__ inline size_t fg_mask_stage_bytes(int WC, int R) {
  return ((size_t)FG_BJ * WC * R * 4 + 127) & ~(size_t)127;
}

// Shared-memory carve-up (byte offsets from a 1024-byte aligned base): X stages (xbytes per
// element), bitmap stages, the CTA's factor slice, one slab of column sums per consumer warp,
// one transposition buffer per consumer warp (JB rows of FG_TR_LD floats), the column scales
// of FP8 storage, mbarriers.
__host__ __device__ inline FgSmem fg_smem_layout(int WC, int R, bool masked, int BN, int KV, int B, int nstage,
                                                 int JB, int xbytes = 4) {
  FgSmem L;
  size_t o = 0;
  L.x_off = o;
  o += (size_t)nstage * WC * FG_BJ * 32 * R * xbytes;
  L.m_off = o;
  if (masked) o += (size_t)nstage * fg_mask_stage_bytes(WC, R);
  o = (o + 15) & ~(size_t)15;
  L.v_off = o;
  o += (size_t)BN * KV * 8;
  L.cs_off = o;
  o += (size_t)WC * BN * B * 4;
  o = (o + 15) & ~(size_t)15;
  L.tr_off = o;
  o += (size_t)WC * JB * FG_TR_LD * 4;
  L.sc_off = o;
  if (xbytes == 1) o += (size_t)BN * 4;
  o = (o + 7) & ~(size_t)7;
  L.bar_off = o;
  o += 2 * FG_NSTAGE * 8;
  L.scr_off = o;
  o += 32 * 8;
  L.total = o + 1024;  // slack for aligning the base
  return L;
}

// Shared-memory carve-up of the tensor-core form (fg_mma.cu), byte offsets from a 1024-byte
// aligned base: X stages (one 2 KB box of 32 rows x 16 columns per consumer warp, 128-byte
// swizzle), D^T U slabs per stage (16 columns x 8 per consumer warp), the slice's
// (v, v, v', v') rows (per 16-column group, 8 x K float4), the CTA's column sums [K][BN], psi
// scratch, mbarriers.
struct FgMmaSmem {
  size_t x_off, slab_off, vr_off, col_off, scr_off, bar_off, total;
};
__host__ __device__ inline FgMmaSmem fg_mma_smem_layout(int WC, int BN, int K, int nstage) {
  FgMmaSmem L;
  size_t o = 0;
  const size_t ng = (size_t)(BN + 15) / 16;
  L.x_off = o;
  o += (size_t)nstage * WC * 2048;
  L.slab_off = o;
  o += (size_t)nstage * WC * 16 * 8 * 4;
  L.vr_off = o;
  o += ng * 8 * K * 16;
  L.col_off = o;
  o += (size_t)K * BN * 4;
  o = (o + 15) & ~(size_t)15;
  L.scr_off = o;
  o += 32 * 8;
  L.bar_off = o;
  o += 2 * FG_NSTAGE * 8;
  L.total = o + 1024;  // slack for aligning the base
  return L;
}

// SIDE (apply mode): 0 both products, 1 only D Bv (row side), 2 only D^T Bu (column side).
template <int K, int B, bool SAME, int R, int J, int SIDE = 0>
struct FgTraits {
  static constexpr int NP = R / 2;       // float2 pairs of rows per lane
  static constexpr int ROWS_W = 32 * R;  // rows per warp
  static constexpr int KV = (SAME || SIDE == 2) ? K : K + B;
  static constexpr int CSB = SIDE == 1 ? 0 : B;  // column sums per column kept in the slabs
  static constexpr int JB = J * B;
  static_assert(R == 2 || R == 4 || R == 8, "rows per lane");
  static_assert(FG_BJ % J == 0, "group size");
  static_assert(!SAME || K == B, "fg mode multiplies D by the forming factors");
  static_assert(!SAME || SIDE == 0, "fg mode needs both products");
};

// Row of pair p, element e (0/1) for this lane, relative to the warp's first row.
template <int R>
RPCA_DEV int lane_row(int p, int e, int lane) {
  if constexpr (R == 2) return 2 * lane + e;
  else return (p >> 1) * 128 + 4 * lane + (p & 1) * 2 + e;
}
// Offset of the lane's x values for pair-group `grp` inside one column of the warp's box.
template <int R>
RPCA_DEV int lane_xoff(int grp, int lane) {
  if constexpr (R == 2) return 2 * lane;
  else return grp * 128 + 4 * lane;
}
// Bitmap word (within the warp's R words of one column) and bit for pair p, element e.
template <int R>
RPCA_DEV void lane_bit(int p, int e, int lane, int& word, int& bit) {
  if constexpr (R == 2) {
    word = lane >> 4;
    bit = 2 * (lane & 15) + e;
  } else {
    word = (p >> 1) * 4 + (lane >> 3);
    bit = 4 * (lane & 7) + (p & 1) * 2 + e;
  }
}

// The pass over one tile: block `bid` of a grid of nrb x ncs tiles.  tmX, tmM: the tensor maps
// (kernel parameters, or global memory written by the host before the launch: GMAP).
template <int K, int B, bool SAME, bool MASKED, int R, int J, int SIDE, int XT, bool GMAP>
__device__ __forceinline__ void fg_body(const CUtensorMap* tmX, const CUtensorMap* tmM, const FgArgs& a,
                                        const int bid) {
  using T = FgTraits<K, B, SAME, R, J, SIDE>;
  constexpr int NP = T::NP, ROWS_W = T::ROWS_W, KV = T::KV, JB = T::JB;
  constexpr bool ROWSIDE = SIDE != 2, COLSIDE = SIDE != 1;  // which products are formed
  constexpr int XB = fg_x_bytes(XT);
  static_assert(XT == FG_X_F32 || R >= 4, "narrow storage is read four rows per lane at a time");
  if (a.gate != nullptr && *a.gate == 0) return;  // uniform over the grid
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                       ~static_cast<uintptr_t>(1023));
  const int WC = (int)(blockDim.x >> 5) - 1;  // consumer warps; the last warp produces
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = bid % a.nrb, cs = bid / a.nrb;
  const int row0 = rb * WC * ROWS_W;
  const int col0 = cs * a.BN;
  const int ncols = min(a.BN, a.n - col0);
  const int nchunks = (ncols + FG_BJ - 1) / FG_BJ;
  const int nst = a.nstage;
  const FgSmem L = fg_smem_layout(WC, R, MASKED, a.BN, KV, T::CSB, nst, COLSIDE ? JB : 0, XB);
  unsigned char* xs_all = sm + L.x_off;
  float* xsc = reinterpret_cast<float*>(sm + L.sc_off);  // FP8 storage: column scales of the slice
  uint32_t* ms_all = reinterpret_cast<uint32_t*>(sm + L.m_off);
  float2* vsl = reinterpret_cast<float2*>(sm + L.v_off);
  float* csum = reinterpret_cast<float*>(sm + L.cs_off);  // [WC][BN][B]
  float* trbuf = reinterpret_cast<float*>(sm + L.tr_off);  // [WC][JB][FG_TR_LD]
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar_off);
  uint64_t* empty = full + FG_NSTAGE;
  double* scr = reinterpret_cast<double*>(sm + L.scr_off);
  const size_t xbox = (size_t)FG_BJ * ROWS_W;                // elements per warp box of X
  const size_t mstage = fg_mask_stage_bytes(WC, R) / 4;      // words per bitmap stage
  const int mrow = WC * R;                                   // bitmap words per column of a stage
  const uint32_t stage_bytes = (uint32_t)(WC * xbox * XB + (MASKED ? (size_t)FG_BJ * mrow * 4 : 0));

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], WC);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == WC) {  // ---------------- producer ----------------
    if (lane == 0 && !a.starve) {
      if constexpr (GMAP) {
        fence_tensormap_acquire(tmX);
        if (MASKED) fence_tensormap_acquire(tmM);
      }
      prefetch_tmap(tmX);
      if (MASKED) prefetch_tmap(tmM);
      const uint64_t pol = l2_evict_first_policy();  // X and its bitmap are streamed once per pass
      int issued = 0;
      bool ok = true;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % nst;
        const uint32_t ph = (uint32_t)(c / nst) & 1u;
        if (c >= nst && !mbar_wait_bounded(&empty[s], ph ^ 1u)) {
          atomicOr(a.err, DEV_ERR_TIMEOUT_EMPTY);
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        for (int w = 0; w < WC; ++w)
          tma_load_2d_hint(xs_all + ((size_t)s * WC + w) * xbox * XB, tmX, row0 + w * ROWS_W, col0 + c * FG_BJ,
                           &full[s], pol);
        if constexpr (MASKED)
          tma_load_2d_hint(ms_all + (size_t)s * mstage, tmM, row0 / 32, col0 + c * FG_BJ, &full[s], pol);
        issued = c + 1;
      }
      // Wait (bounded) until every copy this thread issued has landed before leaving.
      for (int c = max(0, issued - nst); c < issued; ++c) {
        if (!mbar_wait_bounded(&full[c % nst], (uint32_t)(c / nst) & 1u)) {
          atomicOr(a.err, DEV_ERR_TIMEOUT_DRAIN);
          break;
        }
      }
      (void)ok;
    }
    return;
  }

  // ---------------- consumers ----------------
  const int nct = WC * 32;
  const int tid = threadIdx.x;
  const int wrow0 = row0 + warp * ROWS_W;
  const float alpha = a.alpha_dev ? (float)*a.alpha_dev : a.alpha;
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;

  // Factor slice for this CTA's columns, as duplicated pairs (v, v) for the fp32x2 FMA.
  for (int idx = tid; idx < a.BN * KV; idx += nct) {
    const int jj = idx / KV, q = idx - jj * KV;
    const int j = col0 + jj;
    float v = 0.f;
    if (jj < ncols) {
      if (q < K) {
        const size_t o = (size_t)q * a.n + j;
        v = a.V[o];
        if (a.dV) v = fmaf(alpha, a.dV[o], v);
      } else {
        v = a.BV[(size_t)(q - K) * a.n + j];
      }
    }
    vsl[idx] = f2(v, v);
  }
  if constexpr (XT == FG_X_E4M3) {
    for (int jj = tid; jj < a.BN; jj += nct) xsc[jj] = jj < ncols ? a.xscale[col0 + jj] : 0.f;
  }

  // This lane's rows of the forming factor (negated, so that r' = x - u.v = -r) and,
  // in apply mode, of Bu (negated too, which makes D^T Bu come out with its own sign).
  float2 un[NP][K > 0 ? K : 1];
  float2 bun[NP][(SAME || !COLSIDE) ? 1 : B];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i0 = wrow0 + lane_row<R>(p, 0, lane), i1 = i0 + 1;
#pragma unroll
    for (int l = 0; l < K; ++l) {
      float u0 = 0.f, u1 = 0.f;
      const size_t o = (size_t)l * a.m;
      if (i0 < a.m) {
        u0 = a.U[o + i0];
        if (a.dU) u0 = fmaf(alpha, a.dU[o + i0], u0);
      }
      if (i1 < a.m) {
        u1 = a.U[o + i1];
        if (a.dU) u1 = fmaf(alpha, a.dU[o + i1], u1);
      }
      un[p][l] = f2(-u0, -u1);
    }
    if constexpr (!SAME && COLSIDE) {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const size_t o = (size_t)b * a.m;
        const float b0 = i0 < a.m ? a.BU[o + i0] : 0.f;
        const float b1 = i1 < a.m ? a.BU[o + i1] : 0.f;
        bun[p][b] = f2(-b0, -b1);
      }
    }
  }
  named_bar(1, nct);

  float2 gu[NP][ROWSIDE ? B : 1];
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int b = 0; b < (ROWSIDE ? B : 1); ++b) gu[p][b] = f2(0.f, 0.f);
  // Sum of psi over the lane's elements: float32 with Kahan compensation (a float64 add per
  // chunk would occupy this GPU's narrow float64 pipe); float64 once per tile.
  float psi_s = 0.f, psi_c = 0.f;
  const float lam = a.lam_S;
  const float2 mhalf = f2(-0.5f, -0.5f);
  bool failed = false;

  for (int c = 0; c < nchunks; ++c) {
    const int s = c % nst;
    if (!failed && !mbar_wait_bounded(&full[s], (uint32_t)(c / nst) & 1u, wait_ns)) {
      failed = true;
      if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT_FULL);
    }
    const unsigned char* xsw = xs_all + ((size_t)s * WC + warp) * xbox * XB;  // this warp's box
    const uint32_t* ms = ms_all + (size_t)s * mstage + warp * R;  // this warp's words of column 0
    float2 psi2 = f2(0.f, 0.f);
#pragma unroll 1
    for (int g = 0; g < FG_BJ / J; ++g) {
      float2 gv[J][COLSIDE ? B : 1];
#pragma unroll
      for (int jj = 0; jj < J; ++jj)
#pragma unroll
        for (int b = 0; b < (COLSIDE ? B : 1); ++b) gv[jj][b] = f2(0.f, 0.f);
#pragma unroll
      for (int jj = 0; jj < J; ++jj) {
        const int cc = g * J + jj;           // column within the stage
        const int jl = c * FG_BJ + cc;       // column within the CTA slice
        const float2* vrow = vsl + (size_t)jl * KV;
        float2 vv[K > 0 ? K : 1];
#pragma unroll
        for (int l = 0; l < K; ++l) vv[l] = vrow[l];
        float2 bvv[(SAME || !ROWSIDE) ? 1 : B];
        if constexpr (!SAME && ROWSIDE) {
#pragma unroll
          for (int b = 0; b < B; ++b) bvv[b] = vrow[K + b];
        }
        float xv[R];
        if constexpr (XT == FG_X_F32) {
          const float* xs = reinterpret_cast<const float*>(xsw);
          if constexpr (R == 2) {
            const float2 t = *reinterpret_cast<const float2*>(xs + (size_t)cc * ROWS_W + lane_xoff<R>(0, lane));
            xv[0] = t.x;
            xv[1] = t.y;
          } else {
#pragma unroll
            for (int grp = 0; grp < R / 4; ++grp) {
              const float4 t = *reinterpret_cast<const float4*>(xs + (size_t)cc * ROWS_W + lane_xoff<R>(grp, lane));
              xv[grp * 4 + 0] = t.x;
              xv[grp * 4 + 1] = t.y;
              xv[grp * 4 + 2] = t.z;
              xv[grp * 4 + 3] = t.w;
            }
          }
        } else if constexpr (XT == FG_X_BF16) {
          // bfloat16 -> float32 is exact: the 16 stored bits are the top half of the float.
          const uint16_t* xs = reinterpret_cast<const uint16_t*>(xsw);
#pragma unroll
          for (int grp = 0; grp < R / 4; ++grp) {
            const uint2 t = *reinterpret_cast<const uint2*>(xs + (size_t)cc * ROWS_W + lane_xoff<R>(grp, lane));
            xv[grp * 4 + 0] = __uint_as_float(t.x << 16);
            xv[grp * 4 + 1] = __uint_as_float(t.x & 0xffff0000u);
            xv[grp * 4 + 2] = __uint_as_float(t.y << 16);
            xv[grp * 4 + 3] = __uint_as_float(t.y & 0xffff0000u);
          }
        } else {
          // E4M3 pairs -> half2 (exact) -> float2 (exact), times the column's scale.
          const uint8_t* xs = reinterpret_cast<const uint8_t*>(xsw);
          const float sc = xsc[jl];
#pragma unroll
          for (int grp = 0; grp < R / 4; ++grp) {
            const uint32_t t = *reinterpret_cast<const uint32_t*>(xs + (size_t)cc * ROWS_W + lane_xoff<R>(grp, lane));
            const float2 lo = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(t & 0xffffu), __NV_E4M3)));
            const float2 hi = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(t >> 16), __NV_E4M3)));
            xv[grp * 4 + 0] = lo.x * sc;
            xv[grp * 4 + 1] = lo.y * sc;
            xv[grp * 4 + 2] = hi.x * sc;
            xv[grp * 4 + 3] = hi.y * sc;
          }
        }
        uint32_t mw[R == 2 ? 1 : R / 4];
        if constexpr (MASKED) {
          if constexpr (R == 2) {
            mw[0] = ms[(size_t)cc * mrow + (lane >> 4)];
          } else {
#pragma unroll
            for (int grp = 0; grp < R / 4; ++grp) mw[grp] = ms[(size_t)cc * mrow + grp * 4 + (lane >> 3)];
          }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          float2 r = f2(xv[2 * p], xv[2 * p + 1]);
#pragma unroll
          for (int l = 0; l < K; ++l) r = ffma2(un[p][l], vv[l], r);
          if constexpr (MASKED) {
            int w0, b0, w1, b1;
            lane_bit<R>(p, 0, lane, w0, b0);
            lane_bit<R>(p, 1, lane, w1, b1);
            const uint32_t word = mw[R == 2 ? 0 : (p >> 1)];
            r.x = ((word >> b0) & 1u) ? r.x : 0.f;
            r.y = ((word >> b1) & 1u) ? r.y : 0.f;
            (void)w0;
            (void)w1;
          }
          const float2 d = f2(fminf(fmaxf(r.x, -lam), lam), fminf(fmaxf(r.y, -lam), lam));
          if constexpr (SAME) {
            psi2 = ffma2(d, ffma2(d, mhalf, r), psi2);
#pragma unroll
            for (int b = 0; b < B; ++b) gu[p][b] = ffma2(d, vv[b], gu[p][b]);
#pragma unroll
            for (int b = 0; b < B; ++b) gv[jj][b] = ffma2(d, un[p][b], gv[jj][b]);
          } else {
            if constexpr (ROWSIDE) {
#pragma unroll
              for (int b = 0; b < B; ++b) gu[p][b] = ffma2(d, bvv[b], gu[p][b]);
            }
            if constexpr (COLSIDE) {
#pragma unroll
              for (int b = 0; b < B; ++b) gv[jj][b] = ffma2(d, bun[p][b], gv[jj][b]);
            }
          }
        }
      }
      // Column sums of this group over the warp's rows: each lane writes its JB partials
      // (value-major, so the 32 lanes fill one row of the buffer), then lane t < JB sums
      // row t with 16-byte loads in four independent chains (fixed order).  The warp's sums
      // for the group's J columns go to its own slab (no barrier across warps here).
      if constexpr (COLSIDE) {
        static_assert(JB <= 32, "one lane per column sum");
        float* tr = trbuf + (size_t)warp * JB * FG_TR_LD;
#pragma unroll
        for (int jj = 0; jj < J; ++jj)
#pragma unroll
          for (int b = 0; b < B; ++b) tr[(jj * B + b) * FG_TR_LD + lane] = gv[jj][b].x + gv[jj][b].y;
        __syncwarp();
        if (lane < JB) {
          const float4* row = reinterpret_cast<const float4*>(tr + lane * FG_TR_LD);
          float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 t4 = row[q];
            s0 += t4.x;
            s1 += t4.y;
            s2 += t4.z;
            s3 += t4.w;
          }
          float* slab = csum + ((size_t)warp * a.BN + (size_t)c * FG_BJ + g * J) * B;
          slab[lane] = (s0 + s1) + (s2 + s3);
        }
        __syncwarp();
      }
    }
    {
      const float y = (psi2.x + psi2.y) - psi_c;
      const float t = psi_s + y;
      psi_c = (t - psi_s) - y;
      psi_s = t;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

  // Row sums -(D Bv) over this CTA's columns.
#pragma unroll
  for (int p = 0; p < (ROWSIDE ? NP : 0); ++p) {
    const int i0 = wrow0 + lane_row<R>(p, 0, lane);
    if (i0 < a.mpad) {
#pragma unroll
      for (int b = 0; b < B; ++b)
        *reinterpret_cast<float2*>(a.PU + ((size_t)cs * B + b) * a.mpad + i0) = gu[p][ROWSIDE ? b : 0];
    }
  }
  // Sum of psi over the tile (float-float: lanes, then the consumer warps in fixed order);
  // column sums over the consumer warps in fixed order.
  const ff2 psi_w = warp_ff_sum(ff_from_kahan(psi_s, psi_c));
  if (lane == 0) ff_store(&scr[warp], psi_w);
  named_bar(1, nct);
  if (tid == 0) {
    ff2 s = ff_load(&scr[0]);
    for (int w = 1; w < WC; ++w) s = ff_add(s, ff_load(&scr[w]));
    ff_store(&a.Ppsi[bid], s);
  }
  for (int idx = tid; idx < (COLSIDE ? ncols * B : 0); idx += nct) {
    const int b = idx / ncols, jl = idx - b * ncols;
    float sum = 0.f;
    for (int w = 0; w < WC; ++w) sum += csum[((size_t)w * a.BN + jl) * B + b];
    a.PV[((size_t)rb * B + b) * a.n + col0 + jl] = sum;
  }
}

template <int K, int B, bool SAME, bool MASKED, int R, int J, int SIDE = 0, int XT = FG_X_F32>
__global__ void __launch_bounds__(288, 1) fg_kernel(const __grid_constant__ CUtensorMap tmX,
                                                 const __grid_constant__ CUtensorMap tmM, FgArgs a) {
  fg_body<K, B, SAME, MASKED, R, J, SIDE, XT, false>(&tmX, &tmM, a, (int)blockIdx.x);
}

// Grouped form: the tiles of many independent problems in one launch.  Entry q of the launch's
// list is instance ids[q], which owns the blocks [off[q], off[q + 1]) of the grid; its tensor
// maps and arguments are the FgInst at the start of record ids[q] (records `stride` bytes
// apart).  Every instance of a launch has the same instantiation and consumer-warp count
// (blockDim), and the dynamic shared memory is the largest any of them needs.
struct alignas(64) FgInst {
  CUtensorMap tmX;
  CUtensorMap tmM;
  FgArgs a;
};

template <int K, int B, bool SAME, bool MASKED, int R, int J, int SIDE = 0, int XT = FG_X_F32>
__global__ void __launch_bounds__(288, 1) fg_group_kernel(const unsigned char* __restrict__ rec, size_t stride,
                                                       const int* __restrict__ ids, const int* __restrict__ off,
                                                       int cnt) {
  __shared__ FgArgs sa;
  const int q = group_find(off, cnt, (int)blockIdx.x);
  const FgInst* p = reinterpret_cast<const FgInst*>(rec + (size_t)__ldg(ids + q) * stride);
  args_to_shared(&sa, &p->a);
  __syncthreads();
  fg_body<K, B, SAME, MASKED, R, J, SIDE, XT, true>(&p->tmX, &p->tmM, sa, (int)blockIdx.x - __ldg(off + q));
}

}  // namespace rpca
