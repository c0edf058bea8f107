// Fused evaluation of the Split-SPCP objective and gradient (paper Eq. Thm5 / Eq. 7, gradient
// from Sec. 3.2) in one pass over float32 X, with the column-side contraction D^T U on the
// tensor pipe.
//
// Per element the CUDA-core form of this pass (fg_kernel.cuh) spends 3k fused multiply-adds
// on r = u.v - x, D V and D^T U, plus a cross-lane reduction of the column sums; at k = 5
// that is ~18 instructions per element of X and the pass is issue-bound at about half of the
// HBM rate.  Here the column side, D^T U and its reduction over rows, is a warp-level MMA
// (m16n8k8, tf32 operands, float32 accumulate): a lane holds the residuals of a 16-column x
// 8-row tile in the MMA's accumulator layout (columns g, g + 8; rows 2q, 2q + 1), which is
// the A layout of D^T (-U) once the k index is permuted (k = q <-> row 2q, k = q + 4 <-> row
// 2q + 1; the permutation is applied to U's rows instead), so the clipped residuals feed the
// tensor pipe straight from registers.  The residual r = x - u.v and D V stay on the packed
// fp32x2 FMA pipe: r in float32 FMAs keeps the objective and D exact to float32 rounding when
// the residual is small against u.v (near a solution), where tf32 products would not.
//
// Float32 accuracy of D^T U from tf32 operands: both operands are split as x = hi + lo with
// hi the tf32 value nearest to x and lo = x - hi (exact), and the product is
// d_lo u_hi + d_hi u_lo + d_hi u_hi (three MMAs, small terms first; the dropped lo lo term and
// the tf32 truncation of lo are ~2^-21 relative and unbiased).
//
// Tile: WC consumer warps, 32 rows each (four 8-row blocks), stream 16-column groups of a
// CTA slice of BN columns, npass row passes of 32 WC rows per CTA.  A producer warp issues
// the TMA copies (boxes of 32 rows x 16 columns, 128-byte swizzle, so that the fragment loads
// are free of bank conflicts) and, once the consumers have released a stage, adds the
// consumer warps' D^T U partials of that stage in a fixed order into the CTA's column sums.
// Outputs are the partial sums fg_kernel writes (PU = -(D V) per column split, PV = D^T U
// per row range, psi per CTA), so the same finalize kernel completes the evaluation.
//
// Measured on GB300 (76800 x 1000, k = 5): 146-191 us per pass against 87 us for the CUDA-core
// form.  With the compute removed the same pipeline still takes 113 us (the 2 KB TMA boxes,
// 128 bytes per column, are not fed above ~2.7 TB/s), and with the copies removed the compute
// takes ~125 us (about 24 issued instructions per element, not the ~12 the count of
// arithmetic suggests).  The planner therefore uses this form only on request.
#include "fg_kernel.cuh"
#include "fg_variants.h"

namespace rpca {

namespace {

constexpr int MG = 16;          // columns per group (the M extent of one MMA)
constexpr int MT = 4;           // 8-row blocks per warp
constexpr int MBOX = 32 * MG * 4;  // bytes of one warp's X box (32 rows x 16 columns)

RPCA_DEV void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                       uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// x = hi + lo: hi = x rounded to tf32 (10 fraction bits; to nearest, ties away from zero, by
// an integer add on the bit pattern, valid for finite x below the float32 maximum), lo the
// exact remainder.
RPCA_DEV uint32_t tf32_round(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }
RPCA_DEV void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round(x);
  lo = __float_as_uint(x - __uint_as_float(hi));
}

// split_tf32 of a float pair, the remainders formed by one fp32x2 FMA.
RPCA_DEV void split_pair(float2 x, uint32_t& h0, uint32_t& h1, uint32_t& l0, uint32_t& l1) {
  h0 = tf32_round(x.x);
  h1 = tf32_round(x.y);
  const float2 r = ffma2(f2(__uint_as_float(h0), __uint_as_float(h1)), f2(-1.f, -1.f), x);
  l0 = __float_as_uint(r.x);
  l1 = __float_as_uint(r.y);
}

// Byte offset, inside a warp's 32 x 16 box written by TMA with the 128-byte swizzle, of the
// float pair (rows 8 t + 2 q, 8 t + 2 q + 1) of column j: the box is 16 lines of 128 bytes
// (one column each); the 16-byte chunk c of line j sits at chunk c ^ (j & 7).
RPCA_DEV uint32_t mbox_off(int t, int q, int j) {
  return (uint32_t)j * 128u + ((uint32_t)((2 * t + (q >> 1)) ^ (j & 7)) << 4) + ((uint32_t)(q & 1) << 3);
}

// Column (of a 16-column group) of the MMA row g of lane (g, q); the lane also holds column
// mcol(g) + 8.  64-bit shared loads are served per half-warp (g = 0..3 or 4..7): with columns
// 0, 2, 4, 6 (and 1, 3, 5, 7) the half-warp's eight (column, row pair) loads fall in eight
// distinct 16-byte chunks of the swizzled box (bank-conflict free); with columns 0..3 two
// loads would share a chunk.
RPCA_DEV int mcol(int g) { return 2 * (g & 3) + (g >> 2); }

}  // namespace

template <int K>
__global__ void __launch_bounds__(288, 1) fg_mma_kernel(const __grid_constant__ CUtensorMap tmX,
                                                     const __grid_constant__ CUtensorMap tmM, FgArgs a) {
  static_assert(K >= 1 && K <= 8, "factor rank 1..8 (one k8 MMA step)");
  (void)tmM;
  if (a.gate != nullptr && *a.gate == 0) return;  // uniform over the grid
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                       ~static_cast<uintptr_t>(1023));
  const int WC = (int)(blockDim.x >> 5) - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int jg = mcol(g);  // this lane's columns of a group: jg, jg + 8
  const int rb = blockIdx.x % a.nrb, cs = blockIdx.x / a.nrb;
  const int rows_pass = 32 * WC;
  const int row0 = rb * rows_pass * a.npass;
  const int col0 = cs * a.BN;
  const int ncols = min(a.BN, a.n - col0);
  const int ngroups = (ncols + MG - 1) / MG;
  const int npass = a.npass;
  const int nchunks = npass * ngroups;
  const int nst = a.nstage;
  const FgMmaSmem L = fg_mma_smem_layout(WC, a.BN, K, nst);
  unsigned char* xs_all = sm + L.x_off;
  float* slab_all = reinterpret_cast<float*>(sm + L.slab_off);   // [nst][WC][16 columns][8]
  float4* vrow = reinterpret_cast<float4*>(sm + L.vr_off);        // [group][g][K]: (v_g, v_g, v_g8, v_g8)
  float* colacc = reinterpret_cast<float*>(sm + L.col_off);       // [K][BN]
  double* scr = reinterpret_cast<double*>(sm + L.scr_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar_off);
  uint64_t* empty = full + FG_NSTAGE;
  const uint32_t stage_bytes = (uint32_t)(WC * MBOX);

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], WC);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == WC) {  // ---------------- producer ----------------
    if (lane == 0) prefetch_tmap(&tmX);
    const uint64_t pol = l2_evict_first_policy();
    // D^T U partials of chunk cc (stage s): consumer warps' slabs summed in warp order, then
    // added to the CTA's column sums in pass order.
    auto fold = [&](int p, int gi, int s) {
      const float* sl = slab_all + (size_t)s * WC * (MG * 8);
      for (int v = lane; v < MG * K; v += 32) {
        const int col = v / K, l = v - col * K;
        float t = 0.f;
        for (int w = 0; w < WC; ++w) t += sl[w * (MG * 8) + col * 8 + l];
        float* dst = colacc + (size_t)l * a.BN + gi * MG + col;
        *dst = p == 0 ? t : *dst + t;
      }
    };
    int issued = 0;
    bool ok = true;
    int s = 0, ip = 0, igi = 0, fp = 0, fgi = 0;  // stage, (pass, group) issued, (pass, group) folded
    uint32_t ph = 0;                                // (c / nst) & 1
    for (int c = 0; c < nchunks && ok; ++c) {
      if (c >= nst) {
        if (!mbar_wait_bounded(&empty[s], ph ^ 1u)) {
          if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT_EMPTY);
          ok = false;
          break;
        }
        fold(fp, fgi, s);
        if (++fgi == ngroups) {
          fgi = 0;
          ++fp;
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        for (int w = 0; w < WC; ++w)
          tma_load_2d_hint(xs_all + ((size_t)s * WC + w) * MBOX, &tmX, row0 + ip * rows_pass + 32 * w,
                           col0 + igi * MG, &full[s], pol);
      }
      if (++igi == ngroups) {
        igi = 0;
        ++ip;
      }
      if (++s == nst) {
        s = 0;
        ph ^= 1u;
      }
      issued = c + 1;
    }
    // The last stages: wait (bounded) for the consumers to release them, fold their partials.
    for (int c = max(0, issued - nst); c < issued && ok; ++c) {
      if (!mbar_wait_bounded(&empty[c % nst], (uint32_t)((c / nst) & 1))) {
        if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT_DRAIN);
        ok = false;
        break;
      }
      fold(fp, fgi, c % nst);
      if (++fgi == ngroups) {
        fgi = 0;
        ++fp;
      }
    }
    if (!ok) {
      // Copies still in flight land before the CTA exits (bounded waits).
      for (int c = max(0, issued - nst); c < issued; ++c)
        if (!mbar_wait_bounded(&full[c % nst], (uint32_t)((c / nst) & 1))) break;
    }
    __syncwarp();
    for (int idx = lane; idx < K * ncols; idx += 32) {
      const int l = idx / ncols, j = idx - l * ncols;
      a.PV[((size_t)rb * K + l) * a.n + col0 + j] = ok ? colacc[(size_t)l * a.BN + j] : 0.f;
    }
    return;
  }

  // ---------------- consumers ----------------
  const int nct = WC * 32;
  const int tid = threadIdx.x;
  const float alpha = a.alpha_dev ? (float)*a.alpha_dev : a.alpha;

  // The slice's factor V at the trial point, per 16-column group: (v_j, v_j, v_j+8, v_j+8) for
  // lane rows g (the pairs the fp32x2 FMAs multiply two rows by).
  for (int idx = tid; idx < ngroups * 8 * K; idx += nct) {
    const int gi = idx / (8 * K), r = idx - gi * 8 * K;
    const int gg = r / K, l = r - gg * K;
    float v2[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int jl = gi * MG + mcol(gg) + 8 * e;
      float v = 0.f;
      if (jl < ncols) {
        const size_t o = (size_t)l * a.n + col0 + jl;
        v = a.V[o];
        if (a.dV) v = fmaf(alpha, a.dV[o], v);
      }
      v2[e] = v;
    }
    vrow[idx] = make_float4(v2[0], v2[0], v2[1], v2[1]);
  }
  named_bar(1, nct);

  const float lam = a.lam_S;
  const float2 mhalf = f2(-0.5f, -0.5f);
  float psi_s = 0.f, psi_c = 0.f;
  bool failed = false;
  // Per pass: this lane's rows of U at the trial point: -(u_i) for rows 8t + 2q, 8t + 2q + 1
  // as fp32x2 pairs (residuals), and -U as the MMA B fragment of D^T (-U) (hi / lo): rows
  // 8t + 2q, 8t + 2q + 1 at k index g.
  float2 un[MT][K];
  uint32_t ug[MT][4];
  float2 gu[MT][K];

  int p = 0, gi = 0, s = 0;  // pass, group and stage of chunk c
  uint32_t ph = 0;            // (c / nst) & 1
  for (int c = 0; c < nchunks; ++c) {
    const int rbase = row0 + p * rows_pass + 32 * warp;
    if (gi == 0) {
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        const int i0 = rbase + 8 * t + 2 * q, i1 = i0 + 1;
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
          un[t][l] = f2(-u0, -u1);
          gu[t][l] = f2(0.f, 0.f);
        }
        // k index g: u_{i, g} (zero for g >= K).
        float ub0 = 0.f, ub1 = 0.f;
#pragma unroll
        for (int l = 0; l < K; ++l) {
          if (g == l) {
            ub0 = un[t][l].x;
            ub1 = un[t][l].y;
          }
        }
        split_tf32(ub0, ug[t][0], ug[t][2]);
        split_tf32(ub1, ug[t][1], ug[t][3]);
      }
    }
    if (!failed && !mbar_wait_bounded(&full[s], ph)) {
      failed = true;
      if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT_FULL);
    }
    const unsigned char* xw = xs_all + ((size_t)s * WC + warp) * MBOX;
    float4 vr[K];
#pragma unroll
    for (int l = 0; l < K; ++l) vr[l] = vrow[((size_t)gi * 8 + g) * K + l];
    float gacc[4] = {0.f, 0.f, 0.f, 0.f};
    float2 psi2 = f2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      // x - u.v for rows 8t + 2q, 8t + 2q + 1 of columns jg (ra) and jg + 8 (rc).
      float2 ra = *reinterpret_cast<const float2*>(xw + mbox_off(t, q, jg));
      float2 rc = *reinterpret_cast<const float2*>(xw + mbox_off(t, q, jg + 8));
#pragma unroll
      for (int l = 0; l < K; ++l) {
        ra = ffma2(un[t][l], f2(vr[l].x, vr[l].y), ra);
        rc = ffma2(un[t][l], f2(vr[l].z, vr[l].w), rc);
      }
      const float2 da = f2(fminf(fmaxf(ra.x, -lam), lam), fminf(fmaxf(ra.y, -lam), lam));
      const float2 dc = f2(fminf(fmaxf(rc.x, -lam), lam), fminf(fmaxf(rc.y, -lam), lam));
      psi2 = ffma2(da, ffma2(da, mhalf, ra), psi2);
      psi2 = ffma2(dc, ffma2(dc, mhalf, rc), psi2);
      // -(D V) rows 8t + 2q, 8t + 2q + 1 over this lane's columns jg, jg + 8.
#pragma unroll
      for (int l = 0; l < K; ++l) {
        gu[t][l] = ffma2(da, f2(vr[l].x, vr[l].y), gu[t][l]);
        gu[t][l] = ffma2(dc, f2(vr[l].z, vr[l].w), gu[t][l]);
      }
      // D^T U: A = the clipped residuals with k permuted (k = q <-> row 2q, k = q + 4 <->
      // row 2q + 1) and MMA row g <-> column jg: a0 = d(2q, jg), a1 = d(2q, jg + 8),
      // a2 = d(2q + 1, jg), a3 = d(2q + 1, jg + 8).
      uint32_t dh[4], dl[4];
      split_pair(da, dh[0], dh[2], dl[0], dl[2]);
      split_pair(dc, dh[1], dh[3], dl[1], dl[3]);
      mma_tf32(gacc, dl[0], dl[1], dl[2], dl[3], ug[t][0], ug[t][1]);
      mma_tf32(gacc, dh[0], dh[1], dh[2], dh[3], ug[t][2], ug[t][3]);
      mma_tf32(gacc, dh[0], dh[1], dh[2], dh[3], ug[t][0], ug[t][1]);
    }
    // This warp's D^T U for the group's 16 columns (c0 = (col jg, l 2q), c1 = (jg, 2q + 1),
    // c2 = (jg + 8, 2q), c3 = (jg + 8, 2q + 1)) to its slab of the stage.
    float* sl = slab_all + ((size_t)s * WC + warp) * (MG * 8);
    *reinterpret_cast<float2*>(sl + jg * 8 + 2 * q) = f2(gacc[0], gacc[1]);
    *reinterpret_cast<float2*>(sl + (jg + 8) * 8 + 2 * q) = f2(gacc[2], gacc[3]);
    {
      const float y = (psi2.x + psi2.y) - psi_c;
      const float tt = psi_s + y;
      psi_c = (tt - psi_s) - y;
      psi_s = tt;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);

    if (gi == ngroups - 1) {
      // End of a pass: -(D V) of the warp's 32 rows summed over the lanes that share rows
      // (same q, g = 0..7) by a reduce-scatter over lane bits 4, 3, 2; lane (g, q) ends with
      // the flat values [g K, g K + K) of (t, l, row parity).
      float v[8 * K];
#pragma unroll
      for (int t = 0; t < MT; ++t)
#pragma unroll
        for (int l = 0; l < K; ++l) {
          v[(t * K + l) * 2 + 0] = gu[t][l].x;
          v[(t * K + l) * 2 + 1] = gu[t][l].y;
        }
      int base = 0;
#pragma unroll
      for (int st = 0; st < 3; ++st) {
        const int o = 16 >> st;
        const int H = (8 * K) >> (st + 1);
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int u = 0; u < (8 * K) / 2; ++u) {
          if (u < H) {
            const float send = up ? v[u] : v[u + H];
            const float keep = up ? v[u + H] : v[u];
            v[u] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
        }
        if (up) base += H;
      }
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int idx = base + u;
        const int e = idx & 1, tl = idx >> 1;
        const int t = tl / K, l = tl - t * K;
        const int i = rbase + 8 * t + 2 * q + e;
        if (i < a.mpad) a.PU[((size_t)cs * K + l) * a.mpad + i] = v[u];
      }
    }
    if (++gi == ngroups) {
      gi = 0;
      ++p;
    }
    if (++s == nst) {
      s = 0;
      ph ^= 1u;
    }
  }

  // Sum of psi over the tile (float-float: lanes, then the consumer warps in fixed order).
  const ff2 psi_w = warp_ff_sum(ff_from_kahan(psi_s, psi_c));
  if (lane == 0) ff_store(&scr[warp], psi_w);
  named_bar(1, nct);
  if (tid == 0) {
    ff2 sacc = ff_load(&scr[0]);
    for (int w = 1; w < WC; ++w) sacc = ff_add(sacc, ff_load(&scr[w]));
    ff_store(&a.Ppsi[blockIdx.x], sacc);
  }
}

template <int K>
static void reg_mma(FgVariant* tab) {
  tab[K] = FgVariant{(const void*)&fg_mma_kernel<K>, 32, MG};
}

void fg_register_mma(FgVariant* tab) {
  reg_mma<1>(tab);
  reg_mma<2>(tab);
  reg_mma<3>(tab);
  reg_mma<4>(tab);
  reg_mma<5>(tab);
  reg_mma<6>(tab);
  reg_mma<7>(tab);
  reg_mma<8>(tab);
}

}  // namespace rpca
