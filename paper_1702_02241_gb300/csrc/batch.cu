// Batched form: many independent problems (the C4 workload of varied m, n, k) solved
// concurrently.  Each instance is a full context with its own CUDA stream, planned by the
// time model alone (no per-shape timing: hundreds of shapes).  Three drivers:
//   grouped (the default where every instance is eligible: float32 X, fused-kernel plans,
//     memory cap <= 10): the line-search trials of all instances run in shared launches, one
//     fused-pass launch per group of instances with the same instantiation and one launch each
//     of the assembly, inner products and direction over all of them; the host decides between
//     chunks of rounds and worker threads evaluate certificates on the instances' own streams
//     while the others keep iterating (solve_jobs_grouped);
//   threads (RPCA_BATCH_MODE=threads): host threads (RPCA_BATCH_THREADS) step each instance's
//     own graph-captured iteration on its own stream;
//   rounds (RPCA_BATCH_MODE=rounds): one CUDA graph holds ROUNDS_PER_LAUNCH L-BFGS iterations of
//     every instance (each on a branch of its own) and one launch advances them all.
// Measured on the 256-instance workload, threads and rounds are bound by the dispatch of ~1000
// small kernels per trial of all instances, which a graph does not shorten; the grouped
// driver launches a few tens per trial round.
#include <algorithm>
#include <cstring>
#include <cstdlib>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"

namespace rpca {
struct RoundsGraph;
rpca_status solve_jobs(rpca_ctx* const* ctx, float* const* U, float* const* V, rpca_result* res, int count,
                       rpca_status* status, int threads);  // solve.cu
rpca_status solve_jobs_rounds(rpca_ctx* const* ctx, float* const* U, float* const* V, rpca_result* res, int count,
                              rpca_status* status, int threads, RoundsGraph** cache);  // solve.cu
void rounds_free(RoundsGraph* g);                                                      // solve.cu
struct GroupCache;
bool group_eligible(rpca_ctx* const* ctx, int count);                                   // solve.cu
rpca_status solve_jobs_grouped(rpca_ctx* const* ctx, float* const* U, float* const* V, rpca_result* res, int count,
                               rpca_status* status, int threads, GroupCache** cache);  // solve.cu
void group_free(GroupCache* g);                                                         // solve.cu
}

struct rpca_batch {
  std::vector<rpca_ctx*> ctx;
  std::vector<cudaStream_t> streams;  // owned
  cudaStream_t user = nullptr;
  std::string err;
  rpca::RoundsGraph* rounds = nullptr;  // the batched iteration graph, kept across solves
  rpca::GroupCache* group = nullptr;     // the grouped driver's stream and buffers
  int driver = -1;                       // RPCA_DRIVER_* of the last solve
};

namespace {
thread_local char g_batch_err[512];
}  // namespace

extern "C" {

rpca_status rpca_create_batch(rpca_batch** out, int count, const int64_t* m, const int64_t* n, const float* const* X,
                              const int64_t* ldx, const int* k, const double* lambda_L, const double* lambda_S,
                              const rpca_options* opt, void* cuda_stream) {
  if (!out) return RPCA_EINVAL;
  *out = nullptr;
  if (count < 1 || !m || !n || !X || !k || !lambda_L || !lambda_S) {
    snprintf(g_batch_err, sizeof g_batch_err, "count >= 1 and the m, n, X, k, lambda arrays are required");
    return RPCA_EINVAL;
  }
  rpca_batch* b = new (std::nothrow) rpca_batch();
  if (!b) return RPCA_ENOMEM;
  b->user = static_cast<cudaStream_t>(cuda_stream);
  b->ctx.assign(count, nullptr);
  b->streams.assign(count, nullptr);
  rpca_options o;
  rpca_default_options(&o);
  if (opt) o = *opt;
  o.autotune = 0;  // the time model only: timing every shape would dominate
  for (int i = 0; i < count; ++i) {
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      rpca_destroy_batch(b);
      snprintf(g_batch_err, sizeof g_batch_err, "cudaStreamCreate failed");
      return RPCA_ECUDA;
    }
  }
  int grid_cap = 0;
  if (const char* e = getenv("RPCA_BATCH_GRID")) grid_cap = std::max(0, atoi(e));
  // One block size for every instance's fused pass (four consumer warps), so that the grouped
  // driver's fused-pass launches are one per factor rank.
  const int plan_wc = 4;
  for (int i = 0; i < count; ++i) {
    const int64_t ld = ldx ? ldx[i] : m[i];
    const rpca_status r = rpca::create_ctx(&b->ctx[i], m[i], n[i], X[i], ld, nullptr, 0, k[i], lambda_L[i],
                                           lambda_S[i], &o, b->streams[i], grid_cap, plan_wc);
    if (r != RPCA_OK) {
      snprintf(g_batch_err, sizeof g_batch_err, "instance %d: %s", i, rpca_last_error(nullptr));
      rpca_destroy_batch(b);
      return r;
    }
  }
  *out = b;
  return RPCA_OK;
}

rpca_status rpca_solve_batch(rpca_batch* b, float* const* U, float* const* V, rpca_result* res) {
  if (!b || !U || !V) return RPCA_EINVAL;
  const int count = (int)b->ctx.size();
  // Inputs written on the caller's stream come first.
  cudaEvent_t ready = nullptr;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return RPCA_ECUDA;
  cudaEventRecord(ready, b->user);
  for (int i = 0; i < count; ++i) cudaStreamWaitEvent(b->streams[i], ready, 0);
  cudaEventDestroy(ready);
  std::vector<rpca_result> local(count);
  std::vector<rpca_status> st(count, RPCA_OK);
  // Host threads stepping the solves: they mostly wait on their jobs' streams (a certificate
  // evaluation blocks its thread for milliseconds while that thread's other jobs run dry), so
  // more threads than cores pays: 256 instances took 2.83 s with 16 threads and 2.75 s with 64
  // on a 16-core host.
  int threads = (int)std::min(64u, 4u * std::max(1u, std::thread::hardware_concurrency()));
  if (const char* e = getenv("RPCA_BATCH_THREADS")) threads = std::max(1, atoi(e));
  // The grouped driver where every instance can take part (unless RPCA_BATCH_MODE names
  // another), rounds on request where every instance iterates on the device on float32 X,
  // else host threads stepping each instance's own graph.
  const char* mode = getenv("RPCA_BATCH_MODE");
  bool rounds = mode && strcmp(mode, "rounds") == 0;
  for (rpca_ctx* c : b->ctx) rounds = rounds && c->xq_dt == 0 && c->lk == nullptr && c->device == b->ctx[0]->device;
  const bool grouped = !rounds && !(mode && strcmp(mode, "threads") == 0) &&
                       rpca::group_eligible(b->ctx.data(), count);
  for (rpca_ctx* c : b->ctx) c->no_iter_graph = false;
  b->driver = grouped ? RPCA_DRIVER_GROUPED : (rounds ? RPCA_DRIVER_ROUNDS : RPCA_DRIVER_THREADS);
  if (grouped)
    rpca::solve_jobs_grouped(b->ctx.data(), U, V, local.data(), count, st.data(), threads, &b->group);
  else if (rounds)
    rpca::solve_jobs_rounds(b->ctx.data(), U, V, local.data(), count, st.data(), threads, &b->rounds);
  else
    rpca::solve_jobs(b->ctx.data(), U, V, local.data(), count, st.data(), threads);
  int notconv = 0;
  rpca_status s = RPCA_OK;
  for (int i = 0; i < count; ++i) {
    if (st[i] == RPCA_ENOTCONV) ++notconv;
    else if (st[i] != RPCA_OK && s == RPCA_OK) s = st[i];
  }
  if (res) memcpy(res, local.data(), sizeof(rpca_result) * count);
  // Every solve has synchronised its own stream; order the caller's stream after them too.
  for (int i = 0; i < count; ++i) {
    cudaEvent_t done = nullptr;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(done, b->streams[i]);
      cudaStreamWaitEvent(b->user, done, 0);
      cudaEventDestroy(done);
    }
  }
  if (s != RPCA_OK) {
    for (int i = 0; i < count; ++i)
      if (st[i] != RPCA_OK && st[i] != RPCA_ENOTCONV) {
        b->err = "instance " + std::to_string(i) + ": " + rpca_last_error(b->ctx[i]);
        break;
      }
    return s;
  }
  if (notconv > 0) {
    b->err = std::to_string(notconv) + " instance(s) stopped before the certificate tolerance";
    return RPCA_ENOTCONV;
  }
  return RPCA_OK;
}

rpca_ctx* rpca_batch_context(rpca_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

int rpca_batch_size(const rpca_batch* b) { return b ? (int)b->ctx.size() : 0; }

int rpca_batch_driver(const rpca_batch* b) { return b ? b->driver : -1; }

const char* rpca_batch_last_error(const rpca_batch* b) { return b ? b->err.c_str() : g_batch_err; }

void rpca_destroy_batch(rpca_batch* b) {
  if (!b) return;
  rpca::rounds_free(b->rounds);
  rpca::group_free(b->group);
  for (rpca_ctx* c : b->ctx) rpca_destroy(c);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
}

}  // extern "C"
