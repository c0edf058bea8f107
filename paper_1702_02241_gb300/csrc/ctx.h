// Private host-side state of an rpca_ctx.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rpca.h"
#include "fg_variants.h"
#include "kernels.h"

namespace rpca {

// One launch configuration of the fused kernel for a (K, B, mode, mask) combination.
struct FgPlan {
  bool valid = false;
  const FgVariant* var = nullptr;
  int K = 0, B = 0;
  bool same = true, masked = false;
  int side = 0;  // apply mode: 0 both products, 1 D Bv only, 2 D^T Bu only
  int R = 0, WC = 0, nrb = 0, ncs = 0, BN = 0;
  int threads = 0;
  size_t smem = 0;
  int fin_grid = 0, fin_gu = 0, fin_gv = 0;
  int cps = 0;  // CTAs per SM at this configuration
  int nstage = 3;
  int xt = 0;       // storage type of X read by this plan (FG_X_*)
  bool large = false;  // k > 16: GEMMs + elementwise pass (largek.cu) instead of the fused kernel
  bool mma = false;    // tensor-core form (fg_mma.cu): WC warps x 32 rows per pass, npass passes
  int npass = 1;
  bool tc = false;     // tcgen05 form (fg_tc.cu): U V^T on the tensor cores, 4 consumer warps x 256 rows
  CUtensorMap tmX;  // box {32 R rows, FG_BJ columns}; tensor-core form: {32, 16}, 128-byte swizzle
  CUtensorMap tmM;  // bitmap box {WC * R words, FG_BJ columns}
};

struct Workspace {
  float* PU = nullptr;
  size_t PU_n = 0;
  float* PV = nullptr;
  size_t PV_n = 0;
  double* Ppsi = nullptr;
  size_t Ppsi_n = 0;
  double* blk = nullptr;
  size_t blk_n = 0;
  unsigned int* counter = nullptr;
  double* out = nullptr;  // [8]
  int* err = nullptr;     // device status word
};

struct SolverBuffers;  // solver.cu
struct SolverState;    // solver.h
struct CertBuffers;    // cert.cu
struct LargeK;         // largek.cu
struct SketchBuffers;  // sketch.cu
struct ConvexBuffers;  // convex.cu

}  // namespace rpca

struct rpca_ctx {
  int m = 0, n = 0, k = 0;
  const float* X = nullptr;
  int64_t ldx = 0;
  const uint8_t* mask = nullptr;
  int64_t ldmask = 0;
  double lam_L = 0, lam_S = 0;
  rpca_options opt;
  cudaStream_t stream = nullptr;
  int grid_cap = 0;  // CTA budget of the objective/gradient and L-BFGS launches (0: the whole GPU)
  int plan_wc = 0;   // preferred consumer warps of the fg-mode fused pass (batch instances; 0: any)
  int device = 0, nsm = 0;
  size_t max_smem = 0;
  int mpad = 0;
  uint32_t* bits = nullptr;  // observation bitmap [n][wpad], owned
  int wpad = 0;
  double p_hat = 1.0;        // observed fraction
  double F0 = 0.0;           // F(0) = phi(0), for the distance bound
  double F_best = 0.0;       // best objective seen on this context
  rpca::FgPlan fg_plan;      // K = k, fg mode, float32 X
  // Precision form: X stored by the library as bfloat16 or FP8 E4M3 (column-major, ld ldq).
  void* Xq = nullptr;        // owned
  int64_t ldq = 0;
  int xq_dt = 0;             // FG_X_* (0: no narrow copy)
  float* xscale = nullptr;   // FP8: per-column scales, owned
  rpca::FgPlan fg_plan_q;    // K = k, fg mode, narrow X
  const rpca::FgPlan* solve_plan = nullptr;  // the plan the solver's iteration uses
  rpca::FgPlan ap_plan[3][3];  // apply modes: forming rank 0 / 8 / 16 x side
  rpca::FgPlan ap16_plan[3];   // the sketch's 16-column products, by side (1, 2)
  bool ap16_none[3] = {false, false, false};  // no configuration for that side
  rpca::Workspace ws;          // partial sums of the objective/gradient plan (graph-captured)
  rpca::Workspace ws_ap;       // partial sums of the apply plans
  rpca::SolverBuffers* sol = nullptr;
  rpca::CertBuffers* cert = nullptr;
  rpca::LargeK* lk = nullptr;  // k > 16 (largek.cu)
  rpca::ConvexBuffers* cvx = nullptr;  // the convex baseline's scratch (convex.cu), made on first use
  // Scratch of the randomized-SVD start (sketch.cu) and of the learned start (ws.cu), made on
  // first use and kept: a cudaFree per solve would wait for every stream of the device.
  rpca::SketchBuffers* sk = nullptr;
  float* ws_buf = nullptr;
  size_t ws_buf_n = 0;
  // Learned warm start: the model (not owned) and the last sketch's singular values.
  const rpca_ws* ws_model = nullptr;
  float* sk_sigma = nullptr;  // 32 floats on the device, owned
  int sk_l = 0;
  // Rank increase: contexts for k + 1, k + 2, ... on the same X (owned), made on demand.
  std::vector<rpca_ctx*> grown;
  bool grow_stop = false;  // a solve returns once t1..t3 meet the tolerance but t4 > 0
  std::string err;
  // Instrumentation (rpca_profile).
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;  // pairs: fused kernel start/stop, finalize start/stop
  size_t ev_used = 0;
  double prof_ms[2] = {0, 0};
  int64_t prof_n[2] = {0, 0};
  int64_t launches = 0;
  int64_t graph_launches = 0;
  // Set by the batched form's grouped iteration: the solver captures no iteration graph of
  // its own for this context (one is captured when a later solve needs it).
  bool no_iter_graph = false;
  // Failure injection (rpca_inject_fault): fused-kernel launches left to starve.
  int fault_fg = 0;
};

namespace rpca {

rpca_status set_err(rpca_ctx* c, rpca_status s, const std::string& msg);
rpca_status set_err_noctx(rpca_status s, const char* msg);  // no allocation
bool allow_smem(const void* fn, size_t bytes);
rpca_status make_tmap(rpca_ctx* c, CUtensorMap* map, CUtensorMapDataType dt, const void* base, int64_t d0,
                      int64_t d1, int64_t stride_bytes, int b0, int b1);
rpca_status cuda_err(rpca_ctx* c, cudaError_t e, const char* what);
rpca_status check_dev_err(rpca_ctx* c);
cudaError_t dev_malloc(void** p, size_t bytes);  // cudaMalloc through the block cache, or an injected failure
void dev_free(void* p);                          // back to the block cache (after the work using it is done)
cudaError_t host_pinned_malloc(void** p, size_t bytes);  // cudaMallocHost through the block cache
void host_pinned_free(void* p);
template <typename T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
template <typename T>
inline cudaError_t host_pinned_alloc(T** p, size_t bytes) {
  return host_pinned_malloc(reinterpret_cast<void**>(p), bytes);
}

// Returns from the calling function with RPCA_ECUDA (and the context's error text) on failure.
#define RPCA_CUDA(c, call)                              \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_err((c), e_, #call); \
  } while (0)

// Launches fused kernel + finalize for plan P.  fin_mode FIN_FG: (GU, GV) <- gradient at
// the trial point, out[0..3] <- f, g.d, ||g||^2, ||x||^2.  FIN_APPLY: GU <- D Bv, GV <- D^T Bu.
struct FgLaunch {
  const float* U = nullptr;
  const float* V = nullptr;
  const float* dU = nullptr;
  const float* dV = nullptr;
  float alpha = 0.f;
  const double* alpha_dev = nullptr;
  const int* gate = nullptr;
  const float* BU = nullptr;
  const float* BV = nullptr;
  int fin_mode = FIN_FG;
  float* GU = nullptr;
  float* GV = nullptr;
  float* Ut = nullptr;
  float* Vt = nullptr;
  const float* DU = nullptr;
  const float* DV = nullptr;
  double* out = nullptr;
  double lam = -1.0;  // clip threshold override (< 0: the context's lam_S; +inf allowed)
  // A line-search trial of the solver (fg mode, fused-kernel plans): the finalize stage, its
  // sums and the line-search step run as one launch (finalize_ls_kernel, solver.cu).
  SolverState* ls_st = nullptr;
  cudaGraphConditionalHandle ls_h = 0;
  int ls_in_graph = 0;
  unsigned int* ls_ticket = nullptr;  // zero between launches (reset by the last block)
  int vpart = 0;  // row shard: GV <- the raw partial D^T U, no V terms in the sums
};
rpca_status launch_fg(rpca_ctx* c, const FgPlan& P, const FgLaunch& L, cudaStream_t stream);
// The arguments launch_fg passes to the fused pass and to its assembly (fused-kernel plans).
void fg_launch_args(rpca_ctx* c, const FgPlan& P, const FgLaunch& L, FgArgs* a, FinArgs* f);
cudaError_t launch_finalize_ls(const FinArgs& f, int grid, const FgLaunch& L, cudaStream_t stream);  // solver.cu
const FgPlan* apply_plan(rpca_ctx* c, int K, int side);  // forming rank >= K (0, 8 or 16), side
const FgPlan* apply_plan16(rpca_ctx* c, int side);       // K = 0, 16 columns (sketch), or nullptr
rpca_status make_xq(rpca_ctx* c, int xt);                // narrow copy of X (xq.cu)
rpca_status ws_learned_init(rpca_ctx* c, float* U, float* V, int* used);  // ws.cu
rpca_status lk_setup(rpca_ctx* c);                                           // largek.cu
void lk_free(rpca_ctx* c);
void cvx_free(rpca_ctx* c);  // convex.cu
void sk_free(rpca_ctx* c);   // sketch.cu
rpca_status launch_fg_large(rpca_ctx* c, const FgPlan& P, const FgLaunch& L, cudaStream_t stream);
rpca_status lk_product(rpca_ctx* c, const float* U, const float* V, const float** Lp, int64_t* ldl);
rpca_status create_ctx(rpca_ctx** out, int64_t m, int64_t n, const float* X, int64_t ldx, const uint8_t* mask,
                       int64_t ldmask, int k, double lambda_L, double lambda_S, const rpca_options* opt,
                       void* cuda_stream, int grid_cap, int plan_wc = 0);  // api.cu
// The objective/gradient plan rpca_fg uses: the narrow copy's when there is one.
inline const FgPlan& eval_plan(const rpca_ctx* c) { return c->xq_dt ? c->fg_plan_q : c->fg_plan; }
inline void count_launches(rpca_ctx* c, int64_t n) { c->launches += n; }

}  // namespace rpca
