// Fused evaluation of the Split-SPCP objective and gradient (paper Eq. Thm5 / Eq. 7, gradient
// from Sec. 3.2) in one pass over float32 X, with the residual's product U V^T on the 5th-
// generation tensor cores (tcgen05, accumulators in tensor memory).
//
// The CUDA-core form (fg_kernel.cuh) forms r = x - u.v with k packed fp32x2 FMAs per pair of
// elements; here each CTA keeps its rows of U in tensor memory (TMEM) as the A operand and
// its columns of V in shared memory as the B operand, and one elected thread issues, per
// group of 16 columns, the MMAs of U V^T for every row slot of the tile into a TMEM
// accumulator (128 lanes = 128 rows per slot, 16 columns).  The consumer warps read their
// residual products back with tcgen05.ld (lane = row, so a lane's eight rows are eight
// slots), form r' = x - u.v with one packed subtraction per pair, and go on exactly as the
// CUDA-core form: clip, Huber value, D V on the FMA pipe (row sums in registers), D^T U on the
// FMA pipe with the shuffle-free transposition reduction.  D V and D^T U stay on the FMA pipe:
// as tensor-core operands they would need D in shared memory (a 32-bit operand per element,
// written and read on top of X's own stage traffic), where U V^T needs only the two factors.
//
// Float32 accuracy from tf32 operands: u = u_hi + u_lo, v = v_hi + v_lo with hi the tf32 value
// nearest the float and lo the remainder rounded to tf32; the four products u_lo v_lo +
// u_hi v_lo + u_lo v_hi + u_hi v_hi are accumulated in float32 by the tensor core (four MMAs of
// K = 8 per slot), so u.v is exact up to the tf32 rounding of the remainders (2^-22 relative)
// and the tensor core's float32 accumulation.  Measured: that accumulation errs by about an ulp
// of |u.v| with a sign that follows u.v (not the unbiased rounding of the FMA pipe), so where the
// residual is small against u.v (|r| ~ 0.01 |u.v| / 2) the gradient's relative error grows to
// ~1e-4; the planner therefore uses this form only on request.
//
// Roles (192 threads): warps 0..3 consume (warp w reads TMEM lanes 32 w .. 32 w + 31, the lane
// quarter the hardware gives it), warp 4 streams X with 2-D TMA copies into a ring of stages
// (as the CUDA-core form), warp 5 owns the tensor memory (allocates 256 columns, issues the
// MMAs from one lane, frees it at the end).  TMEM columns: [0, 128) A = (U_hi | U_lo) per slot
// (16 columns each), [128, 256) the accumulator per slot (16 columns each); one accumulator
// group is in flight: the consumers release it once they have read its last four columns, so
// the next group's MMAs overlap with their arithmetic on those columns.  Every wait is bounded
// and reports a status bit; TMEM is released on every path.
#include "fg_kernel.cuh"
#include "fg_variants.h"

namespace rpca {

namespace {

constexpr int TC_R = 8;        // rows per lane = accumulator slots per CTA (slot = 128 rows)
constexpr int TC_G = 16;       // columns per MMA group (the N extent)
constexpr int TC_WC = 4;       // consumer warps: one per TMEM lane quarter
constexpr int TC_NCOL = 256;   // TMEM columns allocated per CTA
constexpr int TC_ACC = 128;    // first accumulator column
constexpr int TC_THREADS = (TC_WC + 2) * 32;
constexpr int TC_VB = 32;      // bytes per column of one V operand (K = 8 tf32 values)

// ---- tcgen05 inline PTX -------------------------------------------------------------
RPCA_DEV void tmem_alloc(uint32_t* dst, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
RPCA_DEV void tmem_relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
RPCA_DEV void tmem_dealloc(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
RPCA_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
RPCA_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
RPCA_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Arrives once on `bar` when every tcgen05 operation this thread issued before has completed.
RPCA_DEV void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// D (TMEM) = A (TMEM) x B (shared-memory descriptor) [+ D when acc != 0], kind::tf32.
RPCA_DEV void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// Stores 16 consecutive 32-bit columns of this thread's TMEM lane.
RPCA_DEV void tc_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}
// Loads 2 consecutive columns of this thread's lane for each of the eight slots (slot s at
// column offset s * 16) and waits for them, in one block, so that no use of the registers can
// be scheduled ahead of the wait.
RPCA_DEV void tc_ld8x2(uint32_t taddr, float (&u)[TC_R][2]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [%17];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%18];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6, %7}, [%19];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%20];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%21];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12, %13}, [%22];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%14, %15}, [%23];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr), "r"(taddr + 16), "r"(taddr + 32), "r"(taddr + 48), "r"(taddr + 64), "r"(taddr + 80),
        "r"(taddr + 96), "r"(taddr + 112)
      : "memory");
#pragma unroll
  for (int s = 0; s < TC_R; ++s) {
    u[s][0] = __uint_as_float(r[s * 2]);
    u[s][1] = __uint_as_float(r[s * 2 + 1]);
  }
}

// tf32 value nearest to x (round to nearest, ties away from zero, on the bit pattern; finite x).
RPCA_DEV float tf32_near(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u); }

// Shared-memory matrix descriptor of a K-major operand without swizzle: core matrices of
// 8 rows x 16 bytes stored contiguously, LBO = byte distance between the two core matrices
// of one row group along K, SBO = byte distance between row groups of 8.
RPCA_DEV uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::tf32: float32 accumulator, tf32 A and B, both K-major,
// N = 16, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_G >> 3) << 17) | ((128u >> 4) << 24);

struct TcSmem {
  size_t x_off, v_off, cs_off, tr_off, vb_off, bar_off, scr_off, tm_off, total;
};
// Shared memory of the tcgen05 form: X stages, the (v, v) pairs of the slice for D V, the
// column-sum slabs and transposition buffers (as the CUDA-core form), the V operand of the
// MMAs (hi and lo, BNP x 32 bytes each), mbarriers, scratch, the TMEM base address.  The total
// is kept above a third of the SM's shared memory so that at most two CTAs (2 x 256 TMEM
// columns) share an SM.
__host__ __device__ inline TcSmem tc_smem_layout(int BN, int K, int nstage, int JB) {
  TcSmem L;
  size_t o = 0;
  const int BNP = (BN + TC_G - 1) / TC_G * TC_G;
  L.x_off = o;
  o += (size_t)nstage * TC_WC * FG_BJ * 32 * TC_R * 4;
  L.v_off = o;
  o += (size_t)BN * K * 8;
  L.cs_off = o;
  o += (size_t)TC_WC * BN * K * 4;
  o = (o + 15) & ~(size_t)15;
  L.tr_off = o;
  o += (size_t)TC_WC * JB * FG_TR_LD * 4;
  o = (o + 127) & ~(size_t)127;
  L.vb_off = o;
  o += (size_t)2 * BNP * TC_VB;
  o = (o + 7) & ~(size_t)7;
  L.bar_off = o;
  o += (2 * FG_NSTAGE + 2) * 8;
  L.scr_off = o;
  o += 32 * 8;
  L.tm_off = o;
  o += 16;
  o += 1024;  // slack for aligning the base
  L.total = o < 80 * 1024 ? 80 * 1024 : o;
  return L;
}

}  // namespace

size_t fg_tc_smem_bytes(int BN, int K, int nstage, int J) { return tc_smem_layout(BN, K, nstage, J * K).total; }

template <int K, int J>
__global__ void __launch_bounds__(TC_THREADS, 2) fg_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                                                           const __grid_constant__ CUtensorMap tmM, FgArgs a) {
  static_assert(K >= 1 && K <= 8, "factor rank 1..8 (one K = 8 tf32 MMA step)");
  constexpr int R = TC_R, NP = R / 2, ROWS_W = 32 * R, JB = J * K;
  static_assert(JB <= 32, "one lane per column sum");
  (void)tmM;
  if (a.gate != nullptr && *a.gate == 0) return;  // uniform over the grid
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                       ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.x % a.nrb, cs = blockIdx.x / a.nrb;
  const int row0 = rb * TC_WC * ROWS_W;
  const int col0 = cs * a.BN;
  const int ncols = min(a.BN, a.n - col0);
  const int nchunks = (ncols + FG_BJ - 1) / FG_BJ;
  const int ngroups = (ncols + TC_G - 1) / TC_G;
  const int nst = a.nstage;
  const int BNP = (a.BN + TC_G - 1) / TC_G * TC_G;
  const TcSmem L = tc_smem_layout(a.BN, K, nst, JB);
  float* xs_all = reinterpret_cast<float*>(sm + L.x_off);
  float2* vsl = reinterpret_cast<float2*>(sm + L.v_off);
  float* csum = reinterpret_cast<float*>(sm + L.cs_off);   // [WC][BN][K]
  float* trbuf = reinterpret_cast<float*>(sm + L.tr_off);  // [WC][JB][FG_TR_LD]
  unsigned char* vb = sm + L.vb_off;                       // V operand: hi | lo
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar_off);
  uint64_t* empty = full + FG_NSTAGE;
  uint64_t* acc_full = empty + FG_NSTAGE;
  uint64_t* acc_empty = acc_full + 1;
  double* scr = reinterpret_cast<double*>(sm + L.scr_off);
  uint32_t* tm_slot = reinterpret_cast<uint32_t*>(sm + L.tm_off);
  const size_t xbox = (size_t)FG_BJ * ROWS_W;  // floats per warp box of X
  const uint32_t stage_bytes = (uint32_t)(TC_WC * xbox * 4);
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TC_WC);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, TC_WC);
    fence_barrier_init();
  }
  if (warp == TC_WC + 1) {  // the TMEM owner allocates (whole warp)
    tmem_alloc(tm_slot, TC_NCOL);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tm_slot;

  const int nct = TC_WC * 32;
  const float alpha = a.alpha_dev ? (float)*a.alpha_dev : a.alpha;
  // This lane's rows of U (the trial point U + alpha dU), negated for r' = x - u.v (so that
  // D^T U comes out with its own sign, as in the CUDA-core form).
  float2 un[NP][K];
  if (warp < TC_WC) {
    const int wrow0 = row0 + warp * ROWS_W;
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
    }
    // A operand: slot s = 2 p + e holds this lane's row of pair p, element e; its 16 TMEM
    // columns are (u_hi[0..8) | u_lo[0..8)).
    const uint32_t lane_base = tbase + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      uint32_t w[16];
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        float u = 0.f;
        if (l < K) u = -((s & 1) ? un[s >> 1][l < K ? l : 0].y : un[s >> 1][l < K ? l : 0].x);
        const float hi = tf32_near(u);
        w[l] = __float_as_uint(hi);
        w[8 + l] = __float_as_uint(tf32_near(u - hi));
      }
      tc_st16(lane_base + (uint32_t)(16 * s), w);
    }
    // The slice's columns of V: (v, v) pairs for D V, and the MMA's B operand, K-major
    // (core matrices of 8 columns x 4 k; k chunks 128 bytes apart, column groups 256 apart).
    for (int idx = threadIdx.x; idx < a.BN * K; idx += nct) {
      const int jj = idx / K, q = idx - jj * K;
      float v = 0.f;
      if (jj < ncols) {
        const size_t o = (size_t)q * a.n + col0 + jj;
        v = a.V[o];
        if (a.dV) v = fmaf(alpha, a.dV[o], v);
      }
      vsl[idx] = f2(v, v);
    }
    for (int idx = threadIdx.x; idx < BNP * 8; idx += nct) {
      const int jj = idx >> 3, q = idx & 7;
      float v = 0.f;
      if (jj < ncols && q < K) {
        const size_t o = (size_t)q * a.n + col0 + jj;
        v = a.V[o];
        if (a.dV) v = fmaf(alpha, a.dV[o], v);
      }
      const float hi = tf32_near(v);
      const float lo = tf32_near(v - hi);
      const size_t off = (size_t)(jj >> 3) * 256 + (q >> 2) * 128 + (jj & 7) * 16 + (q & 3) * 4;
      *reinterpret_cast<float*>(vb + off) = hi;
      *reinterpret_cast<float*>(vb + (size_t)BNP * TC_VB + off) = lo;
    }
    fence_async_smem();  // the tensor core reads the B operand through the async proxy
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == TC_WC) {  // ---------------- TMA producer ----------------
    if (lane == 0 && !a.starve) {
      prefetch_tmap(&tmX);
      const uint64_t pol = l2_evict_first_policy();
      int issued = 0;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % nst;
        const uint32_t ph = (uint32_t)(c / nst) & 1u;
        if (c >= nst && !mbar_wait_bounded(&empty[s], ph ^ 1u)) {
          atomicOr(a.err, DEV_ERR_TIMEOUT_EMPTY);
          break;
        }
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        for (int w = 0; w < TC_WC; ++w)
          tma_load_2d_hint(xs_all + ((size_t)s * TC_WC + w) * xbox, &tmX, row0 + w * ROWS_W, col0 + c * FG_BJ,
                           &full[s], pol);
        issued = c + 1;
      }
      for (int c = max(0, issued - nst); c < issued; ++c) {
        if (!mbar_wait_bounded(&full[c % nst], (uint32_t)(c / nst) & 1u)) {
          atomicOr(a.err, DEV_ERR_TIMEOUT_DRAIN);
          break;
        }
      }
    }
    return;
  }

  if (warp == TC_WC + 1) {  // ---------------- MMA issuer / TMEM owner ----------------
    if (lane == 0) {
      const uint32_t vb_hi = smem_u32(vb), vb_lo = vb_hi + (uint32_t)BNP * TC_VB;
      int committed = 0;
      for (int g = 0; g < ngroups; ++g) {
        if (g > 0) {
          if (!mbar_wait_bounded(acc_empty, (uint32_t)(g - 1) & 1u, wait_ns)) {
            atomicOr(a.err, DEV_ERR_TIMEOUT_EMPTY);
            break;
          }
          tc_fence_after();
        }
        const uint64_t bh = smem_desc(vb_hi + (uint32_t)g * 512u, 128u, 256u);
        const uint64_t bl = smem_desc(vb_lo + (uint32_t)g * 512u, 128u, 256u);
#pragma unroll 1
        for (int s = 0; s < R; ++s) {
          const uint32_t d = tbase + TC_ACC + 16u * s, ah = tbase + 16u * s, al = ah + 8u;
          // Smallest terms first: the float32 accumulation then rounds the large u_hi v_hi
          // product once, at the end, instead of once per correction term.
          tc_mma(d, al, bl, TC_IDESC, 0u);
          tc_mma(d, ah, bl, TC_IDESC, 1u);
          tc_mma(d, al, bh, TC_IDESC, 1u);
          tc_mma(d, ah, bh, TC_IDESC, 1u);
        }
        tc_commit(acc_full);
        committed = g + 1;
      }
      // The last committed group must have completed before the tensor memory is freed.
      if (committed > 0 && !mbar_wait_bounded(acc_full, (uint32_t)(committed - 1) & 1u, wait_ns))
        atomicOr(a.err, DEV_ERR_TIMEOUT_DRAIN);
    }
    __syncwarp();
    tc_fence_before();
    named_bar(2, nct + 32);  // the consumers have read their last accumulator columns
    tc_fence_after();
    tmem_dealloc(tbase, TC_NCOL);
    return;
  }

  // ---------------- consumers ----------------
  const int tid = threadIdx.x;
  const uint32_t acc_lane = tbase + ((uint32_t)(32 * warp) << 16) + TC_ACC;
  float2 gu[NP][K];
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int b = 0; b < K; ++b) gu[p][b] = f2(0.f, 0.f);
  float psi_s = 0.f, psi_c = 0.f;
  const float lam = a.lam_S;
  const float2 mhalf = f2(-0.5f, -0.5f);
  bool failed = false;

  for (int c = 0; c < nchunks; ++c) {
    const int s = c % nst;
    const int g = c >> 2, q4 = c & 3;
    if (q4 == 0) {
      if (!failed && !mbar_wait_bounded(acc_full, (uint32_t)g & 1u, wait_ns)) {
        failed = true;
        if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT_FULL);
      }
      tc_fence_after();
    }
    if (!failed && !mbar_wait_bounded(&full[s], (uint32_t)(c / nst) & 1u, wait_ns)) {
      failed = true;
      if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT_FULL);
    }
    const float* xsw = xs_all + ((size_t)s * TC_WC + warp) * xbox;  // this warp's box
    float2 psi2 = f2(0.f, 0.f);
#pragma unroll
    for (int gg = 0; gg < FG_BJ / J; ++gg) {
      float2 gv[J][K];
#pragma unroll
      for (int jj = 0; jj < J; ++jj)
#pragma unroll
        for (int b = 0; b < K; ++b) gv[jj][b] = f2(0.f, 0.f);
      float uv[R][2];
#pragma unroll
      for (int jj = 0; jj < J; ++jj) {
        const int cc = gg * J + jj;      // column within the stage
        const int jl = c * FG_BJ + cc;   // column within the CTA slice
        if ((cc & 1) == 0) {
          // u.v of this column and the next for the lane's eight rows, from the accumulator.
          tc_ld8x2(acc_lane + (uint32_t)(q4 * 4 + cc), uv);
          if (cc == FG_BJ - 2 && (q4 == 3 || c == nchunks - 1)) {  // the group's last columns are read:
            tc_fence_before();                                  // its accumulator is free for the
            __syncwarp();                                       // next group's MMAs
            if (lane == 0) mbar_arrive(acc_empty);
          }
        }
        const float2* vrow = vsl + (size_t)jl * K;
        float2 vv[K];
#pragma unroll
        for (int l = 0; l < K; ++l) vv[l] = vrow[l];
        float xv[R];
#pragma unroll
        for (int grp = 0; grp < R / 4; ++grp) {
          const float4 t = *reinterpret_cast<const float4*>(xsw + (size_t)cc * ROWS_W + lane_xoff<R>(grp, lane));
          xv[grp * 4 + 0] = t.x;
          xv[grp * 4 + 1] = t.y;
          xv[grp * 4 + 2] = t.z;
          xv[grp * 4 + 3] = t.w;
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          // r' = x - u.v for the pair's rows (slots 2p, 2p + 1), one packed subtraction.
          const float2 r = fadd2(f2(xv[2 * p], xv[2 * p + 1]), f2(-uv[2 * p][cc & 1], -uv[2 * p + 1][cc & 1]));
          const float2 d = f2(fminf(fmaxf(r.x, -lam), lam), fminf(fmaxf(r.y, -lam), lam));
          psi2 = ffma2(d, ffma2(d, mhalf, r), psi2);
#pragma unroll
          for (int b = 0; b < K; ++b) gu[p][b] = ffma2(d, vv[b], gu[p][b]);
#pragma unroll
          for (int b = 0; b < K; ++b) gv[jj][b] = ffma2(d, un[p][b], gv[jj][b]);
        }
      }
      // Column sums of this group over the warp's rows (as the CUDA-core form).
      float* tr = trbuf + (size_t)warp * JB * FG_TR_LD;
#pragma unroll
      for (int jj = 0; jj < J; ++jj)
#pragma unroll
        for (int b = 0; b < K; ++b) tr[(jj * K + b) * FG_TR_LD + lane] = gv[jj][b].x + gv[jj][b].y;
      __syncwarp();
      if (lane < JB) {
        const float4* row = reinterpret_cast<const float4*>(tr + lane * FG_TR_LD);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) {
          const float4 t4 = row[qq];
          s0 += t4.x;
          s1 += t4.y;
          s2 += t4.z;
          s3 += t4.w;
        }
        float* slab = csum + ((size_t)warp * a.BN + (size_t)c * FG_BJ + gg * J) * K;
        slab[lane] = (s0 + s1) + (s2 + s3);
      }
      __syncwarp();
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
  tc_fence_before();
  named_bar(2, nct + 32);  // release the tensor memory to its owner

  // Row sums -(D V) over this CTA's columns.
  const int wrow0 = row0 + warp * ROWS_W;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i0 = wrow0 + lane_row<R>(p, 0, lane);
    if (i0 < a.mpad) {
#pragma unroll
      for (int b = 0; b < K; ++b) *reinterpret_cast<float2*>(a.PU + ((size_t)cs * K + b) * a.mpad + i0) = gu[p][b];
    }
  }
  // Sum of psi over the tile (float-float: lanes, then the consumer warps in fixed order);
  // column sums over the consumer warps in fixed order.
  const ff2 psi_w = warp_ff_sum(ff_from_kahan(psi_s, psi_c));
  if (lane == 0) ff_store(&scr[warp], psi_w);
  named_bar(1, nct);
  if (tid == 0) {
    ff2 sacc = ff_load(&scr[0]);
    for (int w = 1; w < TC_WC; ++w) sacc = ff_add(sacc, ff_load(&scr[w]));
    ff_store(&a.Ppsi[blockIdx.x], sacc);
  }
  for (int idx = tid; idx < ncols * K; idx += nct) {
    const int b = idx / ncols, jl = idx - b * ncols;
    float sum = 0.f;
    for (int w = 0; w < TC_WC; ++w) sum += csum[((size_t)w * a.BN + jl) * K + b];
    a.PV[((size_t)rb * K + b) * a.n + col0 + jl] = sum;
  }
}

template <int K, int J>
static void reg_tc(FgVariant* tab) {
  tab[K] = FgVariant{(const void*)&fg_tc_kernel<K, J>, TC_R, J};
}

void fg_register_tc(FgVariant* tab) {
  reg_tc<1, 4>(tab);
  reg_tc<2, 4>(tab);
  reg_tc<3, 4>(tab);
  reg_tc<4, 4>(tab);
  reg_tc<5, 2>(tab);
  reg_tc<6, 2>(tab);
}

}  // namespace rpca
