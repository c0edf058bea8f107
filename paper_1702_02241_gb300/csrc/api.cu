// C ABI: context creation, launch planning, one-pass objective/gradient and D-products.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <unordered_map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>
#include <new>

#include "ctx.h"
#include "fg_kernel.cuh"

namespace rpca {

// Message of the last failure of a call without a context (a fixed buffer: recording it
// never allocates).
static thread_local char g_create_err[512];

rpca_status set_err(rpca_ctx* c, rpca_status s, const std::string& msg) {
  if (c) c->err = msg;
  else snprintf(g_create_err, sizeof g_create_err, "%s", msg.c_str());
  return s;
}

rpca_status set_err_noctx(rpca_status s, const char* msg) {
  snprintf(g_create_err, sizeof g_create_err, "%s", msg);
  return s;
}

rpca_status cuda_err(rpca_ctx* c, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return set_err(c, e == cudaErrorMemoryAllocation ? RPCA_ENOMEM : RPCA_ECUDA, msg);
}



// Reads (and clears) the device status word; call after a synchronise.
rpca_status check_dev_err(rpca_ctx* c) {
  int h = 0;
  RPCA_CUDA(c, cudaMemcpyAsync(&h, c->ws.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h != 0) {
    RPCA_CUDA(c, cudaMemsetAsync(c->ws.err, 0, sizeof(int), c->stream));
    char buf[128];
    snprintf(buf, sizeof buf, "a bounded device wait gave up (status bits 0x%x); results are invalid", h);
    return set_err(c, RPCA_ETIMEOUT, buf);
  }
  return RPCA_OK;
}

// ---- kernel variant table ----------------------------------------------------------------
static FgVariant g_same[17][2];
static FgVariant g_same_x[2][17][2];  // narrow storage of X: bfloat16, FP8 E4M3
static FgVariant g_apply[3][3][2];
static FgVariant g_apply16[3][2];  // K = 0, B = 16, by side (1, 2) and mask
static FgVariant g_mma[17];  // tensor-core form, unmasked, K = 1..8
static FgVariant g_tc[17];   // tcgen05 form, unmasked, K = 1..6
static std::once_flag g_once;

static void init_tables() {
  std::call_once(g_once, [] {
    memset(g_same, 0, sizeof g_same);
    memset(g_same_x, 0, sizeof g_same_x);
    memset(g_apply, 0, sizeof g_apply);
    memset(g_apply16, 0, sizeof g_apply16);
    memset(g_mma, 0, sizeof g_mma);
    memset(g_tc, 0, sizeof g_tc);
    fg_register_mma(g_mma);
    fg_register_tc(g_tc);
    fg_register_same_small(g_same);
    fg_register_same_bf16(g_same_x[0]);
    fg_register_same_e4m3(g_same_x[1]);
    fg_register_same_large(g_same);
    fg_register_apply(g_apply);
    fg_register_apply16(g_apply16);
  });
}

const FgVariant* fg_variant(int K, int B, bool same, bool masked, int side, int xt) {
  init_tables();
  if (xt != 0) {
    if (!same || xt < 1 || xt > 2 || K < 1 || K > 16 || B != K || side != 0) return nullptr;
    const FgVariant* v = &g_same_x[xt - 1][K][masked ? 1 : 0];
    return v->fn ? v : nullptr;
  }
  if (same) {
    if (K < 1 || K > 16 || B != K || side != 0) return nullptr;
    return g_same[K][masked ? 1 : 0].fn ? &g_same[K][masked ? 1 : 0] : nullptr;
  }
  if (B == 16 && K == 0 && (side == 1 || side == 2)) {
    const FgVariant* v16 = &g_apply16[side][masked ? 1 : 0];
    return v16->fn ? v16 : nullptr;
  }
  if (B != 8 || side < 0 || side > 2) return nullptr;
  const int slot = K == 0 ? 0 : (K == 8 ? 1 : (K == 16 ? 2 : -1));
  if (slot < 0) return nullptr;
  const FgVariant* v = &g_apply[slot][side][masked ? 1 : 0];
  return v->fn ? v : nullptr;
}

const FgVariant* fg_mma_variant(int K, bool masked) {
  init_tables();
  if (masked || K < 1 || K > 8) return nullptr;
  return g_mma[K].fn ? &g_mma[K] : nullptr;
}

const FgVariant* fg_tc_variant(int K, bool masked) {
  init_tables();
  if (masked || K < 1 || K > 16) return nullptr;
  return g_tc[K].fn ? &g_tc[K] : nullptr;
}

// ---- TMA descriptors -----------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

static rpca_status make_tmap_swz(rpca_ctx* c, CUtensorMap* map, CUtensorMapDataType dt, const void* base,
                                 int64_t d0, int64_t d1, int64_t stride_bytes, int b0, int b1,
                                 CUtensorMapSwizzle swz);

rpca_status make_tmap(rpca_ctx* c, CUtensorMap* map, CUtensorMapDataType dt, const void* base, int64_t d0,
                      int64_t d1, int64_t stride_bytes, int b0, int b1) {
  return make_tmap_swz(c, map, dt, base, d0, d1, stride_bytes, b0, b1, CU_TENSOR_MAP_SWIZZLE_NONE);
}

// swz = CU_TENSOR_MAP_SWIZZLE_128B needs b0 * element size <= 128 bytes and a 1024-byte
// aligned shared-memory destination.
static rpca_status make_tmap_swz(rpca_ctx* c, CUtensorMap* map, CUtensorMapDataType dt, const void* base,
                                 int64_t d0, int64_t d1, int64_t stride_bytes, int b0, int b1,
                                 CUtensorMapSwizzle swz) {
  auto fn = encode_fn();
  if (!fn) {
    const char* msg = "cuTensorMapEncodeTiled is not available from the driver";
    return c ? set_err(c, RPCA_ECUDA, msg) : set_err_noctx(RPCA_ECUDA, msg);
  }
  cuuint64_t dims[2] = {(cuuint64_t)d0, (cuuint64_t)d1};
  cuuint64_t strides[1] = {(cuuint64_t)stride_bytes};
  cuuint32_t box[2] = {(cuuint32_t)b0, (cuuint32_t)b1};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[160];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) for dims %lld x %lld, box %d x %d", (int)r,
             (long long)d0, (long long)d1, b0, b1);
    return c ? set_err(c, RPCA_ECUDA, buf) : set_err_noctx(RPCA_ECUDA, buf);
  }
  return RPCA_OK;
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes` (once per kernel and size;
// the limit only ever grows, so a configuration planned earlier with more shared memory stays
// launchable).  False when the device cannot give that much.
bool allow_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<const void*, size_t> lim;
  std::lock_guard<std::mutex> lock(mu);
  auto it = lim.find(fn);
  if (it != lim.end() && it->second >= bytes) return true;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  lim[fn] = bytes;
  return true;
}

// ---- autotuner support ----------------------------------------------------------------------
struct PlanKey {
  int dev, m, n;
  int64_t ldx;
  int K, B;
  bool same, masked;
  int xt;
  bool operator<(const PlanKey& o) const {
    return std::tie(dev, m, n, ldx, K, B, same, masked, xt) <
           std::tie(o.dev, o.m, o.n, o.ldx, o.K, o.B, o.same, o.masked, o.xt);
  }
};
static std::mutex g_cache_mu;
static std::map<PlanKey, std::pair<int, int>> g_plan_cache;

static bool plan_cache_get(const PlanKey& k, int* wc, int* ncs) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  auto it = g_plan_cache.find(k);
  if (it == g_plan_cache.end()) return false;
  *wc = it->second.first;
  *ncs = it->second.second;
  return true;
}
static void plan_cache_put(const PlanKey& k, int wc, int ncs) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  g_plan_cache[k] = {wc, ncs};
}
static bool autotune_enabled() {
  const char* e = getenv("RPCA_AUTOTUNE");
  return !(e && e[0] == '0');
}

static rpca_status size_workspace(rpca_ctx* c, const FgPlan& P);
static Workspace& plan_ws(rpca_ctx* c, const FgPlan& P);

// Tensor maps for a chosen configuration.
static rpca_status finish_plan(rpca_ctx* c, FgPlan* q) {
  rpca_status s;
  if (q->mma) {
    s = make_tmap_swz(c, &q->tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->X, c->m, c->n, c->ldx * 4, 32, 16,
                      CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != RPCA_OK) return s;
    q->tmM = q->tmX;
    return RPCA_OK;
  }
  if (q->xt == FG_X_F32) {
    s = make_tmap(c, &q->tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->X, c->m, c->n, c->ldx * 4, 32 * q->R, FG_BJ);
  } else {
    const CUtensorMapDataType dt = q->xt == FG_X_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    s = make_tmap(c, &q->tmX, dt, c->Xq, c->m, c->n, c->ldq * fg_x_bytes(q->xt), 32 * q->R, FG_BJ);
  }
  if (s != RPCA_OK) return s;
  if (q->masked) {
    s = make_tmap(c, &q->tmM, CU_TENSOR_MAP_DATA_TYPE_UINT32, c->bits, c->wpad, c->n, (int64_t)c->wpad * 4,
                  q->WC * q->R, FG_BJ);
    if (s != RPCA_OK) return s;
  } else {
    q->tmM = q->tmX;
  }
  return RPCA_OK;
}

// Average duration of the fused kernel alone for configuration q (zero factors: the pass
// over X and the arithmetic are the same as for any factors), CUDA events on the stream.
static rpca_status time_plan(rpca_ctx* c, const FgPlan& q, double* ms) {
  rpca_status s = size_workspace(c, q);
  if (s != RPCA_OK) return s;
  const int w = std::max(q.K, q.B);
  float* z = nullptr;
  RPCA_CUDA(c, cudaMalloc(&z, sizeof(float) * (size_t)(c->m + c->n) * std::max(w, 1)));
  RPCA_CUDA(c, cudaMemsetAsync(z, 0, sizeof(float) * (size_t)(c->m + c->n) * std::max(w, 1), c->stream));
  FgArgs a;
  memset(&a, 0, sizeof a);
  a.m = c->m;
  a.n = c->n;
  a.mpad = c->mpad;
  a.U = z;
  a.V = z + (size_t)c->m * w;
  a.BU = z;
  a.BV = z + (size_t)c->m * w;
  a.lam_S = std::isinf(c->lam_S) ? INFINITY : (float)c->lam_S;
  a.nrb = q.nrb;
  a.ncs = q.ncs;
  a.BN = q.BN;
  a.nstage = q.nstage;
  a.npass = q.npass;
  Workspace& wsp = plan_ws(c, q);
  a.PU = wsp.PU;
  a.PV = wsp.PV;
  a.Ppsi = wsp.Ppsi;
  a.err = c->ws.err;
  a.xscale = c->xscale;
  void* args[] = {(void*)&q.tmX, (void*)&q.tmM, (void*)&a};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = cudaLaunchKernel(q.var->fn, dim3(q.nrb * q.ncs), dim3(q.threads), args, q.smem, c->stream);
  const int reps = 3;
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  for (int i = 0; i < reps && e == cudaSuccess; ++i)
    e = cudaLaunchKernel(q.var->fn, dim3(q.nrb * q.ncs), dim3(q.threads), args, q.smem, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0;
  if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(z);
  count_launches(c, reps + 1);
  if (e != cudaSuccess) return cuda_err(c, e, "timing a launch configuration");
  *ms = t / reps;
  return check_dev_err(c);
}

// ---- launch planning -----------------------------------------------------------------------
// Chooses consumer warps per CTA (WC) and the column split (ncs, BN).  A time model ranks
// the configurations that fit: an SM streams its tiles at a bounded rate (the kernel is
// limited per SM by issue as much as by HBM), so the time is the larger of the busiest SM's
// bytes (waves of cps tiles) at that rate and all bytes at the HBM rate, plus the write and
// re-read of the partial sums.  The twelve best are then timed on the device and the fastest
// is kept (cached per shape in this process).  RPCA_PLAN="warps,splits[,stages]" forces one
// configuration; RPCA_AUTOTUNE=0 keeps the model's choice without timing.
// Cache code of a plan's kernel configuration (warps, stages).
static int plan_code(const FgPlan& q) {
  return (q.mma ? (1 << 20) + (q.npass << 10) : 0) + (q.tc ? (1 << 24) : 0) + q.WC * 16 + q.nstage;
}

static rpca_status make_plan(rpca_ctx* c, FgPlan* P, int K, int B, bool same, int side, int xt = FG_X_F32) {
  const bool masked = c->bits != nullptr;
  const FgVariant* v = fg_variant(K, B, same, masked, side, xt);
  if (!v) return set_err(c, RPCA_EUNSUPPORTED, "no compiled kernel for this factor rank and storage type");
  const int KV = (same || side == 2) ? K : K + B;
  const int CSB = side == 1 ? 0 : B;
  double best = 1e300;
  std::vector<std::pair<double, FgPlan>> cands;
  int force_wc = 0, force_ncs = 0, force_nst = 0, n_smem = 0, n_attr = 0, n_occ = 0, n_try = 0;
  cudaError_t last_occ = cudaSuccess;
  if (const char* env = getenv("RPCA_PLAN")) sscanf(env, "%d,%d,%d", &force_wc, &force_ncs, &force_nst);
  for (int WC : {8, 4, 2}) for (int nst : {6, 4, 2}) {
    if ((force_wc && WC != force_wc) || (force_nst && nst != force_nst)) continue;
    const int BM = WC * 32 * v->R;
    const int nrb = (c->m + BM - 1) / BM;
    if (WC > 2 && BM / 2 >= c->m) continue;  // a smaller CTA covers the rows
    const int maxsplit = std::max(1, (c->n + FG_BJ - 1) / FG_BJ);
    int last_ncs = -1;
    for (int ncs_req = 1; ncs_req <= std::min(maxsplit, 256); ++ncs_req) {
      int BN = (c->n + ncs_req - 1) / ncs_req;
      BN = (BN + FG_BJ - 1) / FG_BJ * FG_BJ;
      const int ncs = (c->n + BN - 1) / BN;
      if (ncs == last_ncs) continue;
      if (force_ncs && ncs != force_ncs) continue;
      last_ncs = ncs;
      const FgSmem L = fg_smem_layout(WC, v->R, masked, BN, KV, CSB, nst, side == 1 ? 0 : v->J * B, fg_x_bytes(xt));
      ++n_try;
      if (L.total > c->max_smem) {
        ++n_smem;
        continue;
      }
      const int threads = (WC + 1) * 32;
      if (!allow_smem(v->fn, L.total)) {
        ++n_attr;
        continue;
      }
      int cps = 0;
      cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cps, v->fn, threads, L.total);
      if (oe != cudaSuccess || cps < 1) {
        if (oe != cudaSuccess) last_occ = oe;
        cudaGetLastError();
        ++n_occ;
        continue;
      }
      const double tiles = (double)nrb * ncs;
      const double tile_bytes = (double)BM * BN * fg_x_bytes(xt) + (masked ? (double)BM * BN / 8.0 : 0.0);
      // The busiest SM holds kt tiles, cw of them at a time; its rate grows with the consumer
      // warps resident on it up to about eight.
      constexpr double SM_GBS = 30.0, HBM_GBS = 6700.0;  // per-SM streaming rate, whole-GPU rate
      const double kt = std::ceil(tiles / c->nsm);
      const double cw = std::min<double>(cps, kt);
      const double waves = std::ceil(kt / cw);
      const double rate = SM_GBS * std::min(1.0, cw * WC / 8.0);
      const double t_sm = waves * cw * tile_bytes / rate;
      const double t_hbm = tiles * tile_bytes / HBM_GBS;
      double t = std::max(t_sm, t_hbm);
      t += 2.0 * 4.0 * ((double)ncs * c->mpad * B + (double)nrb * c->n * B) / HBM_GBS;
      FgPlan cand;
      cand.valid = true;
      cand.var = v;
      cand.K = K;
      cand.B = B;
      cand.same = same;
      cand.side = side;
      cand.masked = masked;
      cand.R = v->R;
      cand.WC = WC;
      cand.nrb = nrb;
      cand.ncs = ncs;
      cand.BN = BN;
      cand.threads = threads;
      cand.smem = L.total;
      cand.cps = cps;
      cand.nstage = nst;
      cand.xt = xt;
      cands.push_back({t, cand});
      if (t < best) best = t;
    }
  }
  // Tensor-core form (fg_mma.cu; float32 X, fg mode, K <= 8, unmasked): consumer warps x 32
  // rows per pass, npass passes per CTA, BN (a multiple of 16) columns per CTA.  Measured on
  // the 76800 x 1000, k = 5 pass it is slower than the CUDA-core form (152 against 87 us: its
  // 32 x 16 TMA boxes alone cannot be fed above ~2.7 TB/s, and its compute alone takes
  // ~125 us), so it is planned only on request: RPCA_FG_KERNEL=mma (=cuda: the CUDA-core
  // form only, the default).
  const char* kenv = getenv("RPCA_FG_KERNEL");
  const bool only_mma = kenv && strcmp(kenv, "mma") == 0;
  const FgVariant* mv = (same && side == 0 && B == K && xt == FG_X_F32) ? fg_mma_variant(K, masked) : nullptr;
  if (only_mma && mv) cands.clear();
  if (mv && only_mma && !(force_wc || force_ncs)) {
    for (int WC : {8, 4}) for (int nst : {8, 6, 4}) {
      const int rows_pass = 32 * WC;
      if (WC > 4 && rows_pass / 2 >= c->m) continue;
      const int maxsplit = std::max(1, (c->n + 15) / 16);
      int last_ncs = -1;
      for (int ncs_req = 1; ncs_req <= std::min(maxsplit, 32); ++ncs_req) {
        int BN = (c->n + ncs_req - 1) / ncs_req;
        BN = (BN + 15) / 16 * 16;
        const int ncs = (c->n + BN - 1) / BN;
        if (ncs == last_ncs) continue;
        last_ncs = ncs;
        const FgMmaSmem L = fg_mma_smem_layout(WC, BN, K, nst);
        ++n_try;
        if (L.total > c->max_smem) {
          ++n_smem;
          continue;
        }
        const int threads = (WC + 1) * 32;
        if (!allow_smem(mv->fn, L.total)) {
          ++n_attr;
          continue;
        }
        int cps = 0;
        cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cps, mv->fn, threads, L.total);
        if (oe != cudaSuccess || cps < 1) {
          if (oe != cudaSuccess) last_occ = oe;
          cudaGetLastError();
          ++n_occ;
          continue;
        }
        for (int npass = 1; npass <= 256; npass *= 2) {
          const int rows_cta = rows_pass * npass;
          if (npass > 1 && rows_cta / 2 >= c->m) break;
          const int nrb = (c->m + rows_cta - 1) / rows_cta;
          const double tiles = (double)nrb * ncs;
          const double tile_bytes = (double)rows_cta * BN * 4.0;
          constexpr double SM_GBS = 20.0, HBM_GBS = 6700.0;
          const double kt = std::ceil(tiles / c->nsm);
          const double cw = std::min<double>(cps, kt);
          const double waves = std::ceil(kt / cw);
          const double rate = SM_GBS * std::min(1.0, cw * WC / 8.0);
          double t = std::max(waves * cw * tile_bytes / rate, tiles * tile_bytes / HBM_GBS);
          t += 2.0 * 4.0 * ((double)ncs * c->mpad * B + (double)nrb * c->n * B) / HBM_GBS;
          FgPlan cand;
          cand.valid = true;
          cand.var = mv;
          cand.K = K;
          cand.B = B;
          cand.same = same;
          cand.side = side;
          cand.masked = masked;
          cand.R = 1;
          cand.WC = WC;
          cand.nrb = nrb;
          cand.ncs = ncs;
          cand.BN = BN;
          cand.threads = threads;
          cand.smem = L.total;
          cand.cps = cps;
          cand.nstage = nst;
          cand.xt = xt;
          cand.mma = true;
          cand.npass = npass;
          cands.push_back({t, cand});
        }
      }
    }
  }
  // tcgen05 form (fg_tc.cu; float32 X, fg mode, K <= 6, unmasked): four consumer warps of 256
  // rows (1024 rows per CTA), U V^T from tensor memory, the rest as the CUDA-core form.
  // Planned on request (RPCA_FG_KERNEL=tc) or beside the CUDA-core form when the environment
  // variable is unset and RPCA_FG_TC=1.
  const bool only_tc = kenv && strcmp(kenv, "tc") == 0;
  const char* tcenv = getenv("RPCA_FG_TC");
  const bool with_tc = only_tc || (!kenv && tcenv && strcmp(tcenv, "1") == 0);
  const FgVariant* tv = (same && side == 0 && B == K && xt == FG_X_F32) ? fg_tc_variant(K, masked) : nullptr;
  if (only_tc && tv) cands.clear();
  if (tv && with_tc && !(force_wc || force_ncs)) {
    for (int nst : {6, 4, 3, 2}) {
      const int BM = 4 * 32 * tv->R;
      const int nrb = (c->m + BM - 1) / BM;
      const int maxsplit = std::max(1, (c->n + FG_BJ - 1) / FG_BJ);
      int last_ncs = -1;
      for (int ncs_req = 1; ncs_req <= std::min(maxsplit, 256); ++ncs_req) {
        int BN = (c->n + ncs_req - 1) / ncs_req;
        BN = (BN + FG_BJ - 1) / FG_BJ * FG_BJ;
        const int ncs = (c->n + BN - 1) / BN;
        if (ncs == last_ncs) continue;
        last_ncs = ncs;
        const size_t smem = fg_tc_smem_bytes(BN, K, nst, tv->J);
        ++n_try;
        if (smem > c->max_smem) {
          ++n_smem;
          continue;
        }
        const int threads = 6 * 32;
        if (!allow_smem(tv->fn, smem)) {
          ++n_attr;
          continue;
        }
        int cps = 0;
        cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cps, tv->fn, threads, smem);
        if (oe != cudaSuccess || cps < 1) {
          if (oe != cudaSuccess) last_occ = oe;
          cudaGetLastError();
          ++n_occ;
          continue;
        }
        cps = std::min(cps, 2);  // two CTAs of 256 TMEM columns per SM
        const double tiles = (double)nrb * ncs;
        const double tile_bytes = (double)BM * BN * 4.0;
        constexpr double SM_GBS = 36.0, HBM_GBS = 6700.0;
        const double kt = std::ceil(tiles / c->nsm);
        const double cw = std::min<double>(cps, kt);
        const double waves = std::ceil(kt / cw);
        const double rate = SM_GBS * std::min(1.0, cw * 4 / 8.0);
        double t = std::max(waves * cw * tile_bytes / rate, tiles * tile_bytes / HBM_GBS);
        t += 2.0 * 4.0 * ((double)ncs * c->mpad * B + (double)nrb * c->n * B) / HBM_GBS;
        FgPlan cand;
        cand.valid = true;
        cand.var = tv;
        cand.K = K;
        cand.B = B;
        cand.same = same;
        cand.side = side;
        cand.masked = masked;
        cand.R = tv->R;
        cand.WC = 4;
        cand.nrb = nrb;
        cand.ncs = ncs;
        cand.BN = BN;
        cand.threads = threads;
        cand.smem = smem;
        cand.cps = cps;
        cand.nstage = nst;
        cand.xt = xt;
        cand.tc = true;
        cands.push_back({t, cand});
      }
    }
  }
  // A context that shares the GPU (grid_cap > 0) keeps the configurations within its CTA
  // budget, or the smallest grids when none is.
  if (c->grid_cap > 0 && !cands.empty()) {
    int gmin = INT_MAX;
    for (auto& cp : cands) gmin = std::min(gmin, cp.second.nrb * cp.second.ncs);
    const int cap = std::max(c->grid_cap, gmin);
    cands.erase(std::remove_if(cands.begin(), cands.end(),
                               [&](const std::pair<double, FgPlan>& cp) { return cp.second.nrb * cp.second.ncs > cap; }),
                cands.end());
  }
  // A batch instance (plan_wc > 0) keeps its fused-pass configurations at plan_wc consumer
  // warps where it has any: instances of one factor rank then share one instantiation and
  // block size, so that the grouped driver launches one fused pass for all of them.
  if (c->plan_wc > 0 && same && side == 0) {
    auto other = [&](const std::pair<double, FgPlan>& cp) { return cp.second.mma || cp.second.tc || cp.second.WC != c->plan_wc; };
    if (!std::all_of(cands.begin(), cands.end(), other)) cands.erase(std::remove_if(cands.begin(), cands.end(), other), cands.end());
  }
  if (cands.empty()) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "no launch configuration for K=%d B=%d (m=%d n=%d): %d tried, %d over %zu B of shared memory, "
             "%d refused the smem attribute, %d with zero occupancy (%s)",
             K, B, c->m, c->n, n_try, n_smem, c->max_smem, n_attr, n_occ, cudaGetErrorName(last_occ));
    return set_err(c, RPCA_EUNSUPPORTED, buf);
  }
  std::sort(cands.begin(), cands.end(),
            [](const std::pair<double, FgPlan>& a, const std::pair<double, FgPlan>& b) { return a.first < b.first; });
  for (auto& cp : cands) {
    FgPlan& q = cp.second;
    q.fin_gu = fin_grid_u(c->m, B);
    q.fin_gv = fin_grid_v(c->n, B);
    q.fin_grid = q.fin_gu + q.fin_gv;
  }
  // Cached choice for this shape, or measure the best few candidates of the model.
  const PlanKey key{c->device, c->m, c->n, c->ldx, K, B * 4 + side, same, masked, xt};
  int pick = 0;
  int cached_wc = 0, cached_ncs = 0;
  const bool measure = !(force_wc || force_ncs) && autotune_enabled() && c->opt.autotune && cands.size() > 1;
  if (measure && !kenv && plan_cache_get(key, &cached_wc, &cached_ncs)) {
    for (size_t i = 0; i < cands.size(); ++i)
      if (plan_code(cands[i].second) == cached_wc && cands[i].second.ncs == cached_ncs) pick = (int)i;
  } else if (measure) {
    // The best few of each form by the model are timed.
    const int per_form = same ? 8 : 6;
    std::vector<int> tried;
    int n_cuda = 0, n_mma = 0, n_tc = 0;
    for (int i = 0; i < (int)cands.size(); ++i) {
      int& cnt = cands[i].second.mma ? n_mma : (cands[i].second.tc ? n_tc : n_cuda);
      if (cnt < per_form) {
        ++cnt;
        tried.push_back(i);
      }
    }
    double best_ms = 1e300;
    for (int i : tried) {
      FgPlan& q = cands[i].second;
      rpca_status s = finish_plan(c, &q);
      if (s != RPCA_OK) return s;
      double ms = 0;
      s = time_plan(c, q, &ms);
      if (s != RPCA_OK) return s;
      if (ms < best_ms) {
        best_ms = ms;
        pick = i;
      }
    }
    if (!kenv) plan_cache_put(key, plan_code(cands[pick].second), cands[pick].second.ncs);
  }
  FgPlan bp = cands[pick].second;
  rpca_status s = finish_plan(c, &bp);
  if (s != RPCA_OK) return s;
  *P = bp;
  return RPCA_OK;
}

// Grows a workspace buffer.  Work already queued on the context's stream may still use the
// old buffer (the stream may be non-blocking, which cudaFree's implicit synchronisation does
// not cover), so the stream is drained first.
// Device allocations of the context's set-up go through here so that a test can make the
// next ones fail (rpca_inject_fault, RPCA_FAULT_ALLOC) without exhausting the GPU.
static std::atomic<int> g_fault_alloc{0};

// Blocks of destroyed contexts are kept for the next ones: a context's set-up allocates some
// twenty device buffers and two pinned host words, and each cudaMalloc / cudaFree costs tens of
// microseconds (cudaFree also waits for the device), cudaMallocHost / cudaFreeHost more.
// Freed blocks go to a free list keyed by their size class (powers of two up to 1 MiB, then
// multiples of 1 MiB) and serve the next request of that class; at most kCacheMax bytes are
// kept (beyond that a freed block is returned at once), and rpca_release_memory returns them
// all.  A block is freed only after the work that used it has completed (callers synchronise
// the context's stream, rpca_destroy the device).
namespace {
constexpr size_t kCacheMax = (size_t)4 << 30;
size_t size_class(size_t bytes) {
  if (bytes <= ((size_t)1 << 20)) {
    size_t c = 256;
    while (c < bytes) c <<= 1;
    return c;
  }
  return (bytes + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
}
struct BlockCache {
  std::mutex mu;
  std::unordered_map<void*, size_t> live;              // block -> size class
  std::unordered_map<size_t, std::vector<void*>> free;  // size class -> cached blocks
  size_t cached = 0;
};
BlockCache& dev_cache() {
  static BlockCache c;
  return c;
}
BlockCache& host_cache() {
  static BlockCache c;
  return c;
}
void* cache_take(BlockCache& bc, size_t cls) {
  std::lock_guard<std::mutex> lock(bc.mu);
  auto it = bc.free.find(cls);
  if (it == bc.free.end() || it->second.empty()) return nullptr;
  void* p = it->second.back();
  it->second.pop_back();
  bc.cached -= cls;
  bc.live[p] = cls;
  return p;
}
// Keeps p for reuse (or releases it when the cache is full or p is not one of its blocks).
template <typename Release>
void cache_give(BlockCache& bc, void* p, Release release) {
  if (!p) return;
  std::unique_lock<std::mutex> lock(bc.mu);
  auto it = bc.live.find(p);
  if (it == bc.live.end()) {  // not ours (should not happen): release it directly
    lock.unlock();
    release(p);
    return;
  }
  const size_t cls = it->second;
  bc.live.erase(it);
  if (bc.cached + cls <= kCacheMax) {
    bc.free[cls].push_back(p);
    bc.cached += cls;
    return;
  }
  lock.unlock();
  release(p);
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  int left = g_fault_alloc.load();
  while (left > 0) {
    if (g_fault_alloc.compare_exchange_weak(left, left - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  const size_t cls = size_class(std::max<size_t>(bytes, 1));
  if ((*p = cache_take(dev_cache(), cls)) != nullptr) return cudaSuccess;
  const cudaError_t e = cudaMalloc(p, cls);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lock(dev_cache().mu);
  dev_cache().live[*p] = cls;
  return cudaSuccess;
}

void dev_free(void* p) {
  cache_give(dev_cache(), p, [](void* q) { cudaFree(q); });
}

cudaError_t host_pinned_malloc(void** p, size_t bytes) {
  const size_t cls = size_class(std::max<size_t>(bytes, 1));
  if ((*p = cache_take(host_cache(), cls)) != nullptr) return cudaSuccess;
  const cudaError_t e = cudaMallocHost(p, cls);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lock(host_cache().mu);
  host_cache().live[*p] = cls;
  return cudaSuccess;
}

void host_pinned_free(void* p) {
  cache_give(host_cache(), p, [](void* q) { cudaFreeHost(q); });
}

// Releases every cached block; returns the bytes released.
static size_t release_cached() {
  size_t total = 0;
  for (int h = 0; h < 2; ++h) {
    BlockCache& bc = h ? host_cache() : dev_cache();
    std::lock_guard<std::mutex> lock(bc.mu);
    for (auto& kv : bc.free) {
      for (void* q : kv.second) {
        if (h) cudaFreeHost(q);
        else cudaFree(q);
        total += kv.first;
      }
    }
    bc.free.clear();
    bc.cached = 0;
  }
  return total;
}

template <typename T>
static rpca_status ensure(rpca_ctx* c, T** p, size_t* have, size_t need) {
  if (*have >= need) return RPCA_OK;
  if (*p) {
    RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(*p);
  }
  *p = nullptr;
  *have = 0;
  RPCA_CUDA(c, dev_malloc(reinterpret_cast<void**>(p), std::max<size_t>(need, 1) * sizeof(T)));
  *have = need;
  return RPCA_OK;
}

// Partial-sum buffers: the objective/gradient plan (whose buffers CUDA graphs capture) and
// the apply plans (created on first use) have separate ones, so that a new apply plan never
// moves a captured buffer.
static Workspace& plan_ws(rpca_ctx* c, const FgPlan& P) { return P.same ? c->ws : c->ws_ap; }

static rpca_status size_workspace(rpca_ctx* c, const FgPlan& P) {
  rpca_status s;
  Workspace& w = plan_ws(c, P);
  if ((s = ensure(c, &w.PU, &w.PU_n, (size_t)P.ncs * P.B * c->mpad)) != RPCA_OK) return s;
  if ((s = ensure(c, &w.PV, &w.PV_n, (size_t)P.nrb * P.B * c->n)) != RPCA_OK) return s;
  if ((s = ensure(c, &w.Ppsi, &w.Ppsi_n, (size_t)P.nrb * P.ncs)) != RPCA_OK) return s;
  if ((s = ensure(c, &w.blk, &w.blk_n, (size_t)3 * P.fin_grid)) != RPCA_OK) return s;
  return RPCA_OK;
}

const FgPlan* apply_plan(rpca_ctx* c, int K, int side) {
  const int slot = K == 0 ? 0 : (K <= 8 ? 1 : 2);
  FgPlan* P = &c->ap_plan[slot][side];
  if (!P->valid) {
    const int KK = slot == 0 ? 0 : (slot == 1 ? 8 : 16);
    if (make_plan(c, P, KK, 8, false, side) != RPCA_OK) return nullptr;
    if (size_workspace(c, *P) != RPCA_OK) return nullptr;
  }
  return P;
}

// The sketch's 16-column product on side 1 or 2 (no forming factors), or nullptr when it has
// no launch configuration (the sketch then takes 8 columns at a time).
const FgPlan* apply_plan16(rpca_ctx* c, int side) {
  if (side < 1 || side > 2 || c->ap16_none[side]) return nullptr;
  FgPlan* P = &c->ap16_plan[side];
  if (!P->valid) {
    const std::string err = c->err;
    if (make_plan(c, P, 0, 16, false, side) != RPCA_OK || size_workspace(c, *P) != RPCA_OK) {
      P->valid = false;
      c->ap16_none[side] = true;
      c->err = err;  // not an error of the call: the 8-column form serves
      return nullptr;
    }
  }
  return P;
}

// The arguments of one fused pass (a) and of its assembly (f) for launch L on plan P.
void fg_launch_args(rpca_ctx* c, const FgPlan& P, const FgLaunch& L, FgArgs* ap, FinArgs* fp) {
  FgArgs& a = *ap;
  a.starve = 0;
  a.wait_ns = 0;
  a.m = c->m;
  a.n = c->n;
  a.mpad = c->mpad;
  a.U = L.U;
  a.V = L.V;
  a.dU = L.dU;
  a.dV = L.dV;
  a.alpha = L.alpha;
  a.alpha_dev = L.alpha_dev;
  a.gate = L.gate;
  a.BU = L.BU;
  a.BV = L.BV;
  const double lam = L.lam >= 0.0 ? L.lam : c->lam_S;
  a.lam_S = std::isinf(lam) ? INFINITY : (float)lam;
  a.nrb = P.nrb;
  a.ncs = P.ncs;
  a.BN = P.BN;
  a.nstage = P.nstage;
  a.npass = P.npass;
  Workspace& w = plan_ws(c, P);
  a.PU = w.PU;
  a.PV = w.PV;
  a.Ppsi = w.Ppsi;
  a.err = c->ws.err;
  a.xscale = c->xscale;
  FinArgs& f = *fp;
  f = FinArgs{};  // every field not set below is zero (vpart, vec4, ...)
  f.m = c->m;
  f.n = c->n;
  f.B = P.B;
  f.mpad = c->mpad;
  f.nrb = P.nrb;
  f.ncs = P.ncs;
  f.nctas = P.nrb * P.ncs;
  f.gu = P.fin_gu;
  f.PU = w.PU;
  f.PV = w.PV;
  f.Ppsi = w.Ppsi;
  f.mode = L.fin_mode;
  f.side = P.side;
  f.U = L.U;
  f.V = L.V;
  f.dU = L.dU;
  f.dV = L.dV;
  f.alpha = L.alpha;
  f.alpha_dev = L.alpha_dev;
  f.gate = L.gate;
  f.lam_L = c->lam_L;
  f.lam_f = (float)c->lam_L;
  f.GU = L.GU;
  f.GV = L.GV;
  f.Ut = L.Ut;
  f.Vt = L.Vt;
  f.DU = L.DU;
  f.DV = L.DV;
  f.blk = w.blk;
  f.counter = c->ws.counter;
  f.out = L.out ? L.out : c->ws.out;
  f.vpart = L.vpart;
  f.vec4 = fin_vec4(f);
}

rpca_status launch_fg(rpca_ctx* c, const FgPlan& P, const FgLaunch& L, cudaStream_t stream) {
  if (P.large) return launch_fg_large(c, P, L, stream);
  FgArgs a;
  FinArgs f;
  fg_launch_args(c, P, L, &a, &f);
  if (c->fault_fg > 0 && !P.mma && !P.tc) {  // failure injection: this launch's copies are never issued
    --c->fault_fg;
    a.starve = 1;
    a.wait_ns = 1000000ull;  // 1 ms
  }
  void* args[] = {(void*)&P.tmX, (void*)&P.tmM, (void*)&a};
  // Event pairs bracket the two launches while profiling (never inside a graph capture).
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (c->prof) cudaStreamIsCapturing(stream, &cap);
  const bool timed = c->prof && cap == cudaStreamCaptureStatusNone;
  if (timed) {
    while (c->ev_pool.size() < c->ev_used + 4) {
      cudaEvent_t e;
      RPCA_CUDA(c, cudaEventCreate(&e));
      c->ev_pool.push_back(e);
    }
    for (int i = 0; i < 4; ++i) ev[i] = c->ev_pool[c->ev_used + i];
    c->ev_used += 4;
    RPCA_CUDA(c, cudaEventRecord(ev[0], stream));
  }
  RPCA_CUDA(c, cudaLaunchKernel(P.var->fn, dim3(P.nrb * P.ncs), dim3(P.threads), args, P.smem, stream));
  if (timed) RPCA_CUDA(c, cudaEventRecord(ev[1], stream));
  const bool fuse_ls = L.ls_st != nullptr && L.fin_mode == FIN_FG;
  count_launches(c, fuse_ls ? 2 : (L.fin_mode != FIN_APPLY ? 3 : 2));
  if (timed) RPCA_CUDA(c, cudaEventRecord(ev[2], stream));
  if (fuse_ls) {
    RPCA_CUDA(c, launch_finalize_ls(f, P.fin_grid, L, stream));
  } else {
    finalize_kernel<<<P.fin_grid, 256, 0, stream>>>(f);
    if (L.fin_mode != FIN_APPLY) finalize_reduce_kernel<<<1, 256, 0, stream>>>(f, P.fin_grid);
  }
  RPCA_CUDA(c, cudaGetLastError());
  if (timed) {
    RPCA_CUDA(c, cudaEventRecord(ev[3], stream));
    if (c->ev_used >= 4096) {  // fold the recorded pairs into the running sums
      RPCA_CUDA(c, cudaStreamSynchronize(stream));
      for (size_t i = 0; i + 3 < c->ev_used; i += 4) {
        float a0 = 0, a1 = 0;
        cudaEventElapsedTime(&a0, c->ev_pool[i], c->ev_pool[i + 1]);
        cudaEventElapsedTime(&a1, c->ev_pool[i + 2], c->ev_pool[i + 3]);
        c->prof_ms[0] += a0;
        c->prof_ms[1] += a1;
        c->prof_n[0] += 1;
        c->prof_n[1] += 1;
      }
      c->ev_used = 0;
    }
  }
  return RPCA_OK;
}

void free_solver(rpca_ctx* c);  // solver.cu
void free_cert(rpca_ctx* c);    // cert.cu

}  // namespace rpca

using namespace rpca;

extern "C" {

void rpca_default_options(rpca_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->lbfgs_mem = 10;
  o->max_iter = 1000;
  o->cert_tol = 1e-4;
  o->cert_every = 25;
  o->init = RPCA_INIT_SKETCH;
  o->seed = 0;
  o->x_dtype = RPCA_F32;
  o->refine_fp32 = 1;
  o->autotune = 1;
  o->timeout_s = 0.0;
  o->gtol = 0.0;
  o->sketch_oversample = 10;
  o->sketch_power = 2;
  o->ls_noise = 1e-8;
}

const char* rpca_version(void) { return "rpca-gb300 0.2 (sm_103a)"; }

rpca_status rpca_inject_fault(rpca_ctx* c, int kind, int count) {
  if (count < 0) return set_err(c, RPCA_EINVAL, "count must be >= 0");
  if (kind == RPCA_FAULT_FG_STARVE) {
    if (!c) return set_err(nullptr, RPCA_EINVAL, "RPCA_FAULT_FG_STARVE needs a context");
    c->fault_fg = count;
    return RPCA_OK;
  }
  if (kind == RPCA_FAULT_ALLOC) {
    rpca::g_fault_alloc.store(count);
    return RPCA_OK;
  }
  return set_err(c, RPCA_EINVAL, "unknown fault kind");
}

rpca_status rpca_profile(rpca_ctx* c, int enable) {
  if (!c) return RPCA_EINVAL;
  if (enable && !c->prof) {
    c->ev_used = 0;
    c->prof_ms[0] = c->prof_ms[1] = 0;
    c->prof_n[0] = c->prof_n[1] = 0;
    c->launches = 0;
    c->graph_launches = 0;
  }
  c->prof = enable != 0;
  return RPCA_OK;
}

rpca_status rpca_profile_read(rpca_ctx* c, double* out) {
  if (!c || !out) return RPCA_EINVAL;
  RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i + 3 < c->ev_used; i += 4) {
    float a0 = 0, a1 = 0;
    cudaEventElapsedTime(&a0, c->ev_pool[i], c->ev_pool[i + 1]);
    cudaEventElapsedTime(&a1, c->ev_pool[i + 2], c->ev_pool[i + 3]);
    c->prof_ms[0] += a0;
    c->prof_ms[1] += a1;
    c->prof_n[0] += 1;
    c->prof_n[1] += 1;
  }
  c->ev_used = 0;
  out[0] = (double)c->prof_n[0];
  out[1] = c->prof_ms[0];
  out[2] = (double)c->prof_n[1];
  out[3] = c->prof_ms[1];
  out[4] = (double)c->launches;
  out[5] = (double)c->graph_launches;
  return RPCA_OK;
}

rpca_status rpca_plan_info(rpca_ctx* c, int which, int64_t* out) {
  if (!c || !out || which < 0 || which > 2) return RPCA_EINVAL;
  const FgPlan* Pp = which == 0 ? &eval_plan(c) : apply_plan(c, which == 1 ? c->k : 0, 1);
  if (!Pp || !Pp->valid) return RPCA_EINVAL;
  const FgPlan& P = *Pp;
  const int64_t v[9] = {P.R, P.WC, P.nrb, P.ncs, P.BN, P.threads, (int64_t)P.smem, P.cps, P.nstage};
  for (int i = 0; i < 9; ++i) out[i] = v[i];
  return RPCA_OK;
}

rpca_status rpca_plan_kernel(rpca_ctx* c, int which, int64_t* out) {
  if (!c || !out || which < 0 || which > 2) return RPCA_EINVAL;
  const FgPlan* Pp = which == 0 ? &eval_plan(c) : apply_plan(c, which == 1 ? c->k : 0, 1);
  if (!Pp || !Pp->valid) return RPCA_EINVAL;
  out[0] = Pp->large ? 2 : (Pp->mma ? 1 : (Pp->tc ? 3 : 0));
  out[1] = Pp->npass;
  return RPCA_OK;
}

const char* rpca_last_error(const rpca_ctx* c) { return c ? c->err.c_str() : g_create_err; }

rpca_status rpca_create(rpca_ctx** out, int64_t m, int64_t n, const float* X, int64_t ldx, const uint8_t* mask,
                        int64_t ldmask, int k, double lambda_L, double lambda_S, const rpca_options* opt,
                        void* cuda_stream) {
  return rpca::create_ctx(out, m, n, X, ldx, mask, ldmask, k, lambda_L, lambda_S, opt, cuda_stream, 0);
}

}  // extern "C"

namespace rpca {

// rpca_create with a cap on the CTAs of the objective/gradient launch (0: none), for
// contexts that share the GPU with many others (the batched form).
rpca_status create_ctx(rpca_ctx** out, int64_t m, int64_t n, const float* X, int64_t ldx, const uint8_t* mask,
                       int64_t ldmask, int k, double lambda_L, double lambda_S, const rpca_options* opt,
                       void* cuda_stream, int grid_cap, int plan_wc) {
  if (!out) return set_err(nullptr, RPCA_EINVAL, "out is NULL");
  *out = nullptr;
  // m and n up to 2^27: every (row or column) x (block of <= 16 columns) index fits 31 bits.
  if (m < 1 || n < 1 || m > (1LL << 27) || n > (1LL << 27))
    return set_err(nullptr, RPCA_EINVAL, "m and n must be in [1, 2^27]");
  if ((m * n) > (1LL << 40)) return set_err(nullptr, RPCA_EINVAL, "m * n too large");
  if (!X) return set_err(nullptr, RPCA_EINVAL, "X is NULL");
  if (ldx < m) return set_err(nullptr, RPCA_EINVAL, "ldx < m");
  if ((ldx * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0)
    return set_err(nullptr, RPCA_EINVAL, "X must be 16-byte aligned with ldx a multiple of 4");
  if (mask && ldmask < m) return set_err(nullptr, RPCA_EINVAL, "ldmask < m");
  if (k < 1 || k > std::min<int64_t>(m, n)) return set_err(nullptr, RPCA_EINVAL, "k must be in [1, min(m, n)]");
  if (k > 256) return set_err(nullptr, RPCA_EUNSUPPORTED, "k must be at most 256");
  if (!(lambda_L > 0) || !std::isfinite(lambda_L)) return set_err(nullptr, RPCA_EINVAL, "lambda_L must be finite and > 0");
  if (!(lambda_S > 0)) return set_err(nullptr, RPCA_EINVAL, "lambda_S must be > 0 (+inf allowed)");
  rpca_options o;
  rpca_default_options(&o);
  if (opt) o = *opt;
  if (o.lbfgs_mem < 1 || o.lbfgs_mem > 32) return set_err(nullptr, RPCA_EINVAL, "lbfgs_mem must be in [1, 32]");
  if (o.x_dtype != RPCA_F32 && o.x_dtype != RPCA_BF16 && o.x_dtype != RPCA_FP8E4M3)
    return set_err(nullptr, RPCA_EINVAL, "x_dtype must be RPCA_F32, RPCA_BF16 or RPCA_FP8E4M3");
  if (o.x_dtype != RPCA_F32 && k > 8)
    return set_err(nullptr, RPCA_EUNSUPPORTED, "narrow storage of X is compiled for k <= 8");

  rpca_ctx* c = new (std::nothrow) rpca_ctx();
  if (!c) return set_err(nullptr, RPCA_ENOMEM, "host allocation failed");
  c->m = (int)m;
  c->n = (int)n;
  c->k = k;
  c->X = X;
  c->ldx = ldx;
  c->mask = mask;
  c->ldmask = ldmask;
  c->lam_L = lambda_L;
  c->lam_S = lambda_S;
  c->opt = o;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->grid_cap = std::max(0, grid_cap);
  c->plan_wc = std::max(0, plan_wc);
  c->mpad = (int)((m + 3) / 4 * 4);
  auto fail = [&](rpca_status s) {
    snprintf(g_create_err, sizeof g_create_err, "%s", c->err.c_str());
    rpca_destroy(c);
    return s;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess) return fail(cuda_err(c, e, "cudaGetDevice"));
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, c->device);
  c->nsm = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  c->max_smem = (size_t)v;
  int cc_major = 0, cc_minor = 0;
  cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, c->device);
  cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, c->device);
  if (cc_major != 10 || cc_minor != 3)
    return fail(set_err(c, RPCA_EUNSUPPORTED, "this library is built for sm_103a (GB300) only"));

  if ((e = dev_malloc(reinterpret_cast<void**>(&c->ws.counter), 64)) != cudaSuccess) return fail(cuda_err(c, e, "cudaMalloc"));
  if ((e = dev_malloc(reinterpret_cast<void**>(&c->ws.out), 8 * sizeof(double))) != cudaSuccess) return fail(cuda_err(c, e, "cudaMalloc"));
  if ((e = dev_malloc(reinterpret_cast<void**>(&c->ws.err), 64)) != cudaSuccess) return fail(cuda_err(c, e, "cudaMalloc"));
  cudaMemsetAsync(c->ws.counter, 0, 64, c->stream);
  cudaMemsetAsync(c->ws.err, 0, 64, c->stream);

  // Validate X on the observed set.
  unsigned long long* cnt = nullptr;
  if ((e = dev_malloc(reinterpret_cast<void**>(&cnt), 2 * sizeof(unsigned long long))) != cudaSuccess) return fail(cuda_err(c, e, "cudaMalloc"));
  cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), c->stream);
  check_x_kernel<<<4 * c->nsm, 256, 0, c->stream>>>(X, ldx, mask, ldmask, c->m, c->n, cnt, cnt + 1);
  unsigned long long hc[2] = {0, 0};
  cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, c->stream);
  e = cudaStreamSynchronize(c->stream);
  dev_free(cnt);
  if (e != cudaSuccess) return fail(cuda_err(c, e, "validating X"));
  if (hc[0] != 0) return fail(set_err(c, RPCA_EINVAL, "X has non-finite observed entries"));
  c->p_hat = (double)hc[1] / ((double)m * (double)n);

  if (mask) {
    c->wpad = (int)(((m + 31) / 32 + 3) / 4 * 4);
    if ((e = dev_malloc(reinterpret_cast<void**>(&c->bits), (size_t)c->wpad * n * 4)) != cudaSuccess) return fail(cuda_err(c, e, "cudaMalloc"));
    const int64_t warps = (int64_t)c->wpad * n;
    pack_mask_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, c->stream>>>(mask, ldmask, c->m, c->n, c->wpad,
                                                                                c->bits);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_err(c, e, "pack_mask_kernel"));
  }
  rpca_status s;
  if (k > 16) {
    // Above the fused kernel's ranks: GEMMs and an elementwise pass (largek.cu).
    if ((s = lk_setup(c)) != RPCA_OK) return fail(s);
  } else {
    if ((s = make_plan(c, &c->fg_plan, k, k, true, 0)) != RPCA_OK) return fail(s);
    if ((s = size_workspace(c, c->fg_plan)) != RPCA_OK) return fail(s);
  }
  if (o.x_dtype != RPCA_F32) {
    // Both objective/gradient plans share one workspace (captured by the solver's graph):
    // size it for both before any capture.
    if ((s = make_xq(c, (int)o.x_dtype)) != RPCA_OK) return fail(s);
    if ((s = make_plan(c, &c->fg_plan_q, k, k, true, 0, (int)o.x_dtype)) != RPCA_OK) return fail(s);
    if ((s = size_workspace(c, c->fg_plan_q)) != RPCA_OK) return fail(s);
  }
  c->solve_plan = &c->fg_plan;
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return fail(cuda_err(c, e, "rpca_create"));
  c->F_best = INFINITY;
  c->F0 = NAN;
  *out = c;
  return RPCA_OK;
}

}  // namespace rpca

extern "C" {

rpca_status rpca_x_storage(rpca_ctx* c, int* dtype, void* host_out, int64_t ld_out, float* scales_out) {
  if (!c || !dtype) return RPCA_EINVAL;
  *dtype = c->xq_dt;
  if (c->xq_dt == 0) return RPCA_OK;
  const size_t eb = (size_t)fg_x_bytes(c->xq_dt);
  if (host_out) {
    if (ld_out < c->m) return set_err(c, RPCA_EINVAL, "ld_out < m");
    RPCA_CUDA(c, cudaMemcpy2DAsync(host_out, (size_t)ld_out * eb, c->Xq, (size_t)c->ldq * eb, (size_t)c->m * eb, c->n,
                                   cudaMemcpyDeviceToHost, c->stream));
  }
  if (scales_out && c->xscale)
    RPCA_CUDA(c, cudaMemcpyAsync(scales_out, c->xscale, sizeof(float) * c->n, cudaMemcpyDeviceToHost, c->stream));
  RPCA_CUDA(c, cudaStreamSynchronize(c->stream));
  return RPCA_OK;
}

rpca_status rpca_fg(rpca_ctx* c, const float* U, const float* V, double* f, float* gU, float* gV) {
  if (!c) return RPCA_EINVAL;
  if (!U || !V || !gU || !gV) return set_err(c, RPCA_EINVAL, "U, V, gU and gV are required");
  FgLaunch L;
  L.U = U;
  L.V = V;
  L.GU = gU;
  L.GV = gV;
  L.out = c->ws.out;
  rpca_status s = launch_fg(c, eval_plan(c), L, c->stream);
  if (s != RPCA_OK) return s;
  if (f) {
    RPCA_CUDA(c, cudaMemcpyAsync(f, c->ws.out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((s = check_dev_err(c)) != RPCA_OK) return s;
    if (*f < c->F_best) c->F_best = *f;
  }
  return RPCA_OK;
}

rpca_status rpca_apply(rpca_ctx* c, const float* U, const float* V, int b, const float* Bv, const float* Bu,
                       float* DBv, float* DtBu) {
  if (!c) return RPCA_EINVAL;
  if (!U || !V || !Bv || !Bu || !DBv || !DtBu) return set_err(c, RPCA_EINVAL, "null argument");
  if (b < 1 || b > 8) return set_err(c, RPCA_EINVAL, "b must be in [1, 8]");
  const FgPlan* P = apply_plan(c, c->k, 0);
  if (!P) return RPCA_EUNSUPPORTED;
  // The kernel reads P->K columns of U, V and 8 of Bu, Bv: pass zero-padded copies.
  const int Kp = P->K;
  float *Up = nullptr, *Vp = nullptr, *Bup = nullptr, *Bvp = nullptr, *Y1 = nullptr, *Y2 = nullptr;
  const size_t m = c->m, n = c->n;
  cudaError_t e = cudaMalloc(&Up, sizeof(float) * (m * Kp + n * Kp + m * 8 + n * 8 + m * 8 + n * 8));
  if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc");
  Vp = Up + m * Kp;
  Bup = Vp + n * Kp;
  Bvp = Bup + m * 8;
  Y1 = Bvp + n * 8;
  Y2 = Y1 + m * 8;
  cudaMemsetAsync(Up, 0, sizeof(float) * (m * Kp + n * Kp + m * 8 + n * 8), c->stream);
  cudaMemcpyAsync(Up, U, sizeof(float) * m * c->k, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(Vp, V, sizeof(float) * n * c->k, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(Bup, Bu, sizeof(float) * m * b, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(Bvp, Bv, sizeof(float) * n * b, cudaMemcpyDeviceToDevice, c->stream);
  FgLaunch L;
  L.U = Up;
  L.V = Vp;
  L.BU = Bup;
  L.BV = Bvp;
  L.fin_mode = FIN_APPLY;
  L.GU = Y1;
  L.GV = Y2;
  rpca_status s = launch_fg(c, *P, L, c->stream);
  if (s == RPCA_OK) {
    cudaMemcpyAsync(DBv, Y1, sizeof(float) * m * b, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(DtBu, Y2, sizeof(float) * n * b, cudaMemcpyDeviceToDevice, c->stream);
    s = check_dev_err(c);
  }
  cudaStreamSynchronize(c->stream);
  cudaFree(Up);
  return s;
}

size_t rpca_release_memory(void) {
  cudaDeviceSynchronize();
  return release_cached();
}

void rpca_destroy(rpca_ctx* c) {
  if (!c) return;
  for (rpca_ctx* g : c->grown)
    if (g) rpca_destroy(g);
  c->grown.clear();
  lk_free(c);
  // Nothing of this context may still run when its blocks go back to the cache.
  cudaStreamSynchronize(c->stream);
  cudaDeviceSynchronize();
  cvx_free(c);
  free_solver(c);
  free_cert(c);
  sk_free(c);
  dev_free(c->bits);
  dev_free(c->Xq);
  dev_free(c->xscale);
  dev_free(c->sk_sigma);
  dev_free(c->ws_buf);
  dev_free(c->ws.PU);
  dev_free(c->ws.PV);
  dev_free(c->ws.Ppsi);
  dev_free(c->ws.blk);
  dev_free(c->ws_ap.PU);
  dev_free(c->ws_ap.PV);
  dev_free(c->ws_ap.Ppsi);
  dev_free(c->ws_ap.blk);
  dev_free(c->ws.counter);
  dev_free(c->ws.out);
  dev_free(c->ws.err);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"
