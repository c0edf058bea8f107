// rpca_fg_noalloc: one objective/gradient evaluation that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they evaluate the
// objective: applications that own all device memory through their own arena and forbid
// cudaMalloc (and the device-wide synchronisation a cudaFree implies) on their hot path,
// or hosts that load this library as a plugin and hand it only the buffers they own.
// rpca_fg needs a context, and rpca_create allocates (partial-sum buffers, the mask bitmap,
// the autotuner's trial buffers).  This entry point does the same evaluation with the
// scratch it needs taken from one fixed device array declared in this file
// (NOALLOC_SCRATCH_BYTES, reserved on every GPU that loads the library, until exit).
// The caller passes X, the factors and the outputs.  The call waits for its stream before
// it returns (it reads f and the status word back into host variables).
#include <cmath>
#include <cstring>
#include <mutex>

#include "ctx.h"
#include "fg_kernel.cuh"

namespace rpca {

constexpr size_t NOALLOC_SCRATCH_BYTES = 32u << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array, looked up once per device with that device current.
// (In host code the array's name is only a host-side stand-in, never a device address.)
static std::mutex g_na_mu;
static void* g_na_addr[128];

static rpca_status noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 128) return set_err_noctx(RPCA_ECUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      char buf[160];
      snprintf(buf, sizeof buf, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorName(e));
      return set_err_noctx(RPCA_ECUDA, buf);
    }
    g_na_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_na_addr[dev]);
  return RPCA_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_fg_noalloc(int64_t m, int64_t n, const float* X, int64_t ldx, int k, double lambda_L,
                                       double lambda_S, const float* U, const float* V, double* f, float* gU,
                                       float* gV, void* cuda_stream) {
  if (m < 1 || n < 1 || m > (1LL << 27) || n > (1LL << 27)) return set_err_noctx(RPCA_EINVAL, "m and n out of range");
  if (!X || !U || !V || !gU || !gV) return set_err_noctx(RPCA_EINVAL, "X, U, V, gU and gV are required");
  if (ldx < m || (ldx * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0)
    return set_err_noctx(RPCA_EINVAL, "X must be 16-byte aligned with ldx >= m a multiple of 4");
  if (k < 1 || k > 16 || k > std::min<int64_t>(m, n)) return set_err_noctx(RPCA_EINVAL, "k must be in [1, min(16, m, n)]");
  if (!(lambda_L > 0) || !std::isfinite(lambda_L) || !(lambda_S > 0))
    return set_err_noctx(RPCA_EINVAL, "lambda_L must be finite and > 0, lambda_S > 0");
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, nsm = 0, smem_optin = 0, ccmaj = 0, ccmin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_err_noctx(RPCA_ECUDA, "cudaGetDevice failed");
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&ccmaj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&ccmin, cudaDevAttrComputeCapabilityMinor, dev);
  if (ccmaj != 10 || ccmin != 3) return set_err_noctx(RPCA_EUNSUPPORTED, "built for sm_103a (GB300) only");
  const FgVariant* v = fg_variant(k, k, true, false);
  if (!v) return set_err_noctx(RPCA_EUNSUPPORTED, "no compiled kernel for this k");

  // Fixed launch configuration (no timing runs: they would need buffers): the widest CTA
  // that the rows fill, four pipeline stages (the depth rpca_fg's planner settles on for
  // most shapes measured), enough column splits to cover the SMs once.
  int WC = 2;
  for (int w : {8, 4}) {
    if ((int64_t)w * 32 * v->R / 2 < m) {
      WC = w;
      break;
    }
  }
  const int BM = WC * 32 * v->R, nst = 4;
  const int nrb = (int)((m + BM - 1) / BM);
  const int mpad = (int)((m + 3) / 4 * 4);
  int ncs_req = std::max(1, (nsm + nrb - 1) / nrb);
  int BN = 0, ncs = 0;
  size_t smem = 0;
  for (;; ++ncs_req) {
    BN = (int)((n + ncs_req - 1) / ncs_req);
    BN = (BN + FG_BJ - 1) / FG_BJ * FG_BJ;
    ncs = (int)((n + BN - 1) / BN);
    smem = fg_smem_layout(WC, v->R, false, BN, k, k, nst, v->J * k).total;
    if (smem <= (size_t)smem_optin || BN <= FG_BJ) break;
  }
  if (smem > (size_t)smem_optin) return set_err_noctx(RPCA_EUNSUPPORTED, "no launch configuration fits");
  const int fin_gu = fin_grid_u(m, k);
  const int fin_gv = fin_grid_v(n, k);
  const int fin_grid = fin_gu + fin_gv;

  // Scratch carve-up: partial sums, per-CTA psi sums, finalize block partials, counter,
  // outputs, status word.
  size_t o = 0;
  const size_t off_pu = o;
  o = align256(o + sizeof(float) * (size_t)ncs * k * mpad);
  const size_t off_pv = o;
  o = align256(o + sizeof(float) * (size_t)nrb * k * n);
  const size_t off_psi = o;
  o = align256(o + sizeof(double) * (size_t)nrb * ncs);
  const size_t off_blk = o;
  o = align256(o + sizeof(double) * 3 * (size_t)fin_grid);
  const size_t off_ctr = o;
  o = align256(o + 64);
  const size_t off_out = o;
  o = align256(o + 8 * sizeof(double));
  const size_t off_err = o;
  o = align256(o + 64);
  if (o > NOALLOC_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof buf, "this shape needs %zu bytes of scratch; rpca_fg_noalloc has %zu (use rpca_fg)", o,
             NOALLOC_SCRATCH_BYTES);
    return set_err_noctx(RPCA_EINVAL, buf);
  }
  unsigned char* base = nullptr;
  rpca_status st = noalloc_scratch(dev, &base);
  if (st != RPCA_OK) return st;
  if (!allow_smem(v->fn, smem)) return set_err_noctx(RPCA_ECUDA, "could not raise the shared-memory limit");
  CUtensorMap tmX;
  if ((st = make_tmap(nullptr, &tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, m, n, ldx * 4, 32 * v->R, FG_BJ)) != RPCA_OK)
    return st;

  // The counter and the status word must start at zero (the array keeps the last call's
  // contents); everything else is written before it is read.
  if (cudaMemsetAsync(base + off_ctr, 0, 64, stream) != cudaSuccess ||
      cudaMemsetAsync(base + off_err, 0, 64, stream) != cudaSuccess)
    return set_err_noctx(RPCA_ECUDA, "cudaMemsetAsync failed");
  FgArgs a;
  memset(&a, 0, sizeof a);
  a.m = (int)m;
  a.n = (int)n;
  a.mpad = mpad;
  a.U = U;
  a.V = V;
  a.lam_S = std::isinf(lambda_S) ? INFINITY : (float)lambda_S;
  a.nrb = nrb;
  a.ncs = ncs;
  a.BN = BN;
  a.nstage = nst;
  a.PU = reinterpret_cast<float*>(base + off_pu);
  a.PV = reinterpret_cast<float*>(base + off_pv);
  a.Ppsi = reinterpret_cast<double*>(base + off_psi);
  a.err = reinterpret_cast<int*>(base + off_err);
  void* args[] = {(void*)&tmX, (void*)&tmX, (void*)&a};
  cudaError_t e = cudaLaunchKernel(v->fn, dim3(nrb * ncs), dim3((WC + 1) * 32), args, smem, stream);
  if (e != cudaSuccess) return set_err_noctx(RPCA_ECUDA, cudaGetErrorString(e));
  FinArgs fa;
  memset(&fa, 0, sizeof fa);
  fa.m = (int)m;
  fa.n = (int)n;
  fa.B = k;
  fa.mpad = mpad;
  fa.nrb = nrb;
  fa.ncs = ncs;
  fa.nctas = nrb * ncs;
  fa.gu = fin_gu;
  fa.PU = a.PU;
  fa.PV = a.PV;
  fa.Ppsi = a.Ppsi;
  fa.mode = FIN_FG;
  fa.U = U;
  fa.V = V;
  fa.lam_L = lambda_L;
  fa.lam_f = (float)lambda_L;
  fa.GU = gU;
  fa.GV = gV;
  fa.blk = reinterpret_cast<double*>(base + off_blk);
  fa.counter = reinterpret_cast<unsigned int*>(base + off_ctr);
  fa.out = reinterpret_cast<double*>(base + off_out);
  fa.vec4 = fin_vec4(fa);
  finalize_kernel<<<fin_grid, 256, 0, stream>>>(fa);
  finalize_reduce_kernel<<<1, 256, 0, stream>>>(fa, fin_grid);
  if ((e = cudaGetLastError()) != cudaSuccess) return set_err_noctx(RPCA_ECUDA, cudaGetErrorString(e));
  // Synchronise and read f and the status word into host variables (no allocation).
  double fh = 0.0;
  int errh = 0;
  if ((e = cudaMemcpyAsync(&fh, fa.out, sizeof(double), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&errh, a.err, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return set_err_noctx(RPCA_ECUDA, cudaGetErrorString(e));
  if (errh != 0) return set_err_noctx(RPCA_ETIMEOUT, "a bounded device wait gave up; results are invalid");
  if (f) *f = fh;
  return RPCA_OK;
}
