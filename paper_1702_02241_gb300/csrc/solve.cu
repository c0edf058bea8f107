// rpca_solve: drives the device L-BFGS graph, checks the certificate every cert_every
// iterations, returns the solution and its certificate.  Random initialisation kernel.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "solver.h"

namespace rpca {

rpca_status solver_prepare(rpca_ctx* c, const float* U, const float* V);
rpca_status solver_iterations(rpca_ctx* c, int count);
rpca_status solver_read_state(rpca_ctx* c, SolverState* out);
rpca_status solver_read_scalars(rpca_ctx* c, SolverState* out);
const float* solver_point(rpca_ctx* c);
rpca_status cert_compute(rpca_ctx* c, const float* U, const float* V, rpca_cert* out, bool full,
                         bool reuse = false, const float* grad = nullptr, const double* f_dev = nullptr,
                         double f_host = 0.0);
const float* solver_gradient(rpca_ctx* c);
const double* solver_f_device(rpca_ctx* c);
rpca_status sketch_init(rpca_ctx* c, const float* Omega, float* U, float* V);

// A point is certified at tol when the Sec. 3.4 certificate meets it and so does the cost of
// the directions the certificate truncated (same relative units).
static inline bool cert_meets(const rpca_cert& q, double tol) { return q.cert_rel <= tol && q.trunc_rel <= tol; }

// Counter-based normal variates: splitmix64 of (seed, index) -> two uniforms -> Box-Muller.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ float normal_at(uint64_t seed, uint64_t i) {
  const uint64_t r = splitmix64(seed * 0x632be59bd9b4e019ull + i);
  const double u1 = ((double)(r >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
  const double u2 = (double)(splitmix64(r) >> 11) * (1.0 / 9007199254740992.0);
  return (float)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
}

__global__ void fill_normal_kernel(float* out, int64_t count, uint64_t seed, float scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = scale * normal_at(seed, (uint64_t)i);
}

// CUDA-event pairs per phase (0 init, 1 iterations, 2 certificate), summed by collect().
struct PhaseTimer {
  cudaStream_t s;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  int cur = -1;
  explicit PhaseTimer(cudaStream_t st) : s(st) {}
  ~PhaseTimer() {
    for (auto& e : ev) {
      cudaEventDestroy(e.second.first);
      cudaEventDestroy(e.second.second);
    }
  }
  void begin(int phase) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    ev.push_back({phase, {a, b}});
    cur = (int)ev.size() - 1;
  }
  void end() {
    if (cur >= 0) cudaEventRecord(ev[cur].second.second, s);
    cur = -1;
  }
  void collect(double* init, double* iter, double* cert) {
    cudaStreamSynchronize(s);
    double t[3] = {0, 0, 0};
    for (auto& e : ev) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, e.second.first, e.second.second) == cudaSuccess) t[e.first] += ms;
    }
    *init = t[0];
    *iter = t[1];
    *cert = t[2];
  }
};

__global__ void scale_kernel(float* x, int64_t count, float t) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= t;
}

void fill_scale(float* x, int64_t count, float t, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(1024, (count + 255) / 256);
  scale_kernel<<<std::max(grid, 1), 256, 0, s>>>(x, count, t);
}

void fill_normal(float* out, int64_t count, uint64_t seed, float scale, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(1024, (count + 255) / 256);
  fill_normal_kernel<<<std::max(grid, 1), 256, 0, s>>>(out, count, seed, scale);
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_solve_log(rpca_ctx* c, double* out, int max_rows, int* rows) {
  if (!c || !out || !rows || max_rows < 0) return RPCA_EINVAL;
  *rows = 0;
  if (!c->sol) return RPCA_OK;
  SolverState st;
  rpca_status s = solver_read_state(c, &st);
  if (s != RPCA_OK) return s;
  const int n = std::min(std::min(st.log_n, SOLVER_LOG), max_rows);
  for (int i = 0; i < n; ++i) {
    const int idx = (st.log_n - n + i) % SOLVER_LOG;
    for (int q = 0; q < 7; ++q) out[7 * i + q] = st.log[idx][q];
  }
  *rows = n;
  return RPCA_OK;
}

extern "C" rpca_status rpca_solve_trials(rpca_ctx* c, double* out, int max_rows, int* rows) {
  if (!c || !out || !rows || max_rows < 0) return RPCA_EINVAL;
  *rows = 0;
  if (!c->sol) return RPCA_OK;
  SolverState st;
  rpca_status s = solver_read_state(c, &st);
  if (s != RPCA_OK) return s;
  const int n = std::min(std::min(st.tlog_n, SOLVER_TLOG), max_rows);
  for (int i = 0; i < n; ++i) {
    const int idx = (st.tlog_n - n + i) % SOLVER_TLOG;
    for (int q = 0; q < 7; ++q) out[7 * i + q] = st.tlog[idx][q];
  }
  *rows = n;
  return RPCA_OK;
}

namespace rpca {

// One solve in progress, resumable: start() runs the initialisation and prepares the
// iteration, step() waits for the iterations launched last (this context's stream only),
// evaluates the certificate when due and launches the next batch of iterations, finish()
// writes the result.  rpca_solve runs them back to back; rpca_solve_batch interleaves the
// steps of many jobs from one host thread so that their iterations overlap on the GPU.
struct SolveJob {
  rpca_ctx* c = nullptr;
  float* U = nullptr;
  float* V = nullptr;
  std::chrono::steady_clock::time_point t0;
  PhaseTimer* timer = nullptr;
  int64_t mk = 0, nk = 0, graph_launches0 = 0;
  SolverState st;
  int every = 0, last_cert_iter = -1, iter_base = 0, evals_base = 0, cert_evals = 0;
  // Certificate scheduling: after the first check, the ratio kappa = cert_rel / ||grad F||
  // of the last check predicts cert_rel from the gradient norm the solver keeps on the device.
  double kappa = 0.0;
  // A predicted check runs once kappa ||grad F|| <= margin * tol: below 1, the iterations run a
  // little longer so that the check more often passes at once (the grouped driver, where an
  // iteration is cheap next to a certificate).
  double margin = 1.0;
  int init_used = 0;
  bool narrow = false, certified = false, done = false;
  double narrow_best = INFINITY;
  rpca_cert cert;
  // Recorded after the last iterations launched: lets a host thread that steps many jobs
  // skip the ones whose work is still running instead of blocking on them.
  cudaEvent_t launched = nullptr;
  ~SolveJob() {
    delete timer;
    if (launched) cudaEventDestroy(launched);
  }
};

// Whether the iterations a job launched last have finished (errors count as finished, so that
// the next step reports them).
static bool job_ready(const SolveJob& j) {
  return j.launched == nullptr || cudaEventQuery(j.launched) != cudaErrorNotReady;
}

static rpca_status job_start(SolveJob& j, rpca_ctx* c, float* U, float* V) {
  j.c = c;
  j.U = U;
  j.V = V;
  j.t0 = std::chrono::steady_clock::now();
  j.mk = (int64_t)c->m * c->k;
  j.nk = (int64_t)c->n * c->k;
  memset(&j.cert, 0, sizeof j.cert);
  j.init_used = c->opt.init;
  rpca_status s;
  // Phase timing: event pairs around each phase on the stream, summed at the end.
  j.timer = new PhaseTimer(c->stream);
  j.timer->begin(0);
  switch (c->opt.init) {
    case RPCA_INIT_USER:
      break;
    case RPCA_INIT_RANDOM:
      fill_normal(U, j.mk, c->opt.seed * 2 + 1, 1e-1f, c->stream);
      fill_normal(V, j.nk, c->opt.seed * 2 + 2, 1e-1f, c->stream);
      count_launches(c, 2);
      break;
    case RPCA_INIT_SKETCH:
      if ((s = sketch_init(c, nullptr, U, V)) != RPCA_OK) return s;
      break;
    case RPCA_INIT_LEARNED: {
      if ((s = sketch_init(c, nullptr, U, V)) != RPCA_OK) return s;
      int used = 0;
      if ((s = ws_learned_init(c, U, V, &used)) != RPCA_OK) return s;
      j.init_used = used ? RPCA_INIT_LEARNED : RPCA_INIT_SKETCH;
      break;
    }
    default:
      return set_err(c, RPCA_EUNSUPPORTED, "this initialisation is not built");
  }
  j.graph_launches0 = c->graph_launches;
  j.timer->end();
  j.timer->begin(1);
  // Precision form: iterate on the narrow copy of X first (its objective differs from the
  // float32 one by the storage rounding), then refine on float32 X.  The certificate is
  // always that of the float32 problem.
  j.narrow = c->xq_dt != 0;
  c->solve_plan = j.narrow ? &c->fg_plan_q : &c->fg_plan;
  if ((s = solver_prepare(c, U, V)) != RPCA_OK) return s;
  j.timer->end();
  j.every = c->opt.cert_every > 0 ? c->opt.cert_every : 0;
  return RPCA_OK;
}

// Leaves the narrow phase: the point so far becomes the start of a float32 solve (fresh
// L-BFGS memory; the float32 objective differs from the narrow one).
static rpca_status job_refine(SolveJob& j) {
  rpca_ctx* c = j.c;
  cudaMemcpyAsync(j.U, solver_point(c), sizeof(float) * j.mk, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(j.V, solver_point(c) + j.mk, sizeof(float) * j.nk, cudaMemcpyDeviceToDevice, c->stream);
  j.iter_base += j.st.iter;
  j.evals_base += j.st.evals;
  j.narrow = false;
  c->solve_plan = &c->fg_plan;
  j.last_cert_iter = -1;
  j.kappa = 0.0;
  j.timer->begin(1);
  const rpca_status s = solver_prepare(c, j.U, j.V);
  j.timer->end();
  return s;
}

// When the certificate is evaluated.  The first check comes after cert_every iterations.
// After a check that did not certify, cert_rel / ||grad F|| at that point (kappa) turns the
// gradient norm, which the solver has on the device after every iteration, into a prediction
// of cert_rel (the cheap terms t1..t3 measure first-order stationarity, so the two fall
// together; on the 76800 x 1000 video solve the ratio stays within 0.7e-3 .. 1.8e-3 from
// iteration 25 to 85).  The state is then read every CERT_POLL iterations and the next check
// runs once the prediction meets the tolerance (at least CERT_MIN_GAP iterations after the
// last), or after 2 cert_every iterations at the latest.  The narrow-storage phase keeps the
// fixed schedule: its switch to float32 compares checks cert_every iterations apart.
constexpr int CERT_POLL = 5, CERT_MIN_GAP = 5;

static bool cert_due(const SolveJob& j, const SolverState& st, double tol) {
  if (j.every <= 0 || j.c->lk || st.iter <= 0 || st.iter == j.last_cert_iter) return false;
  // Fixed schedule: every `every` iterations from the last check (the first after `every`).
  if (j.narrow || !(j.kappa > 0.0)) return st.iter >= std::max(0, j.last_cert_iter) + j.every;
  const int since = st.iter - j.last_cert_iter;
  return (since >= CERT_MIN_GAP && j.kappa * sqrt(fmax(st.gg, 0.0)) <= j.margin * tol) || since >= 2 * j.every;
}

// Decisions between iterations on the state j.st (read by the caller): the certificate when
// due and the stop tests.  Sets j.done when the job is finished; *again when the narrow phase
// ended (the caller reads the state again before launching).
static rpca_status job_decide(SolveJob& j, bool* again) {
  rpca_ctx* c = j.c;
  rpca_status s;
  *again = false;
  const SolverState& st = j.st;
  if (!st.active || st.iter >= c->opt.max_iter - j.iter_base) {
    if (j.narrow && c->opt.refine_fp32 && st.iter < c->opt.max_iter - j.iter_base) {
      if ((s = job_refine(j)) != RPCA_OK) return s;
      *again = true;
      return RPCA_OK;
    }
    j.done = true;
    return RPCA_OK;
  }
  if (cert_due(j, st, c->opt.cert_tol)) {
    j.last_cert_iter = st.iter;
    // Cheap terms first; the spectral term only when they already meet the tolerance.
    j.timer->begin(2);
    // On float32 X the solver's gradient and objective at its iterate give the cheap terms'
    // products without a pass over X.
    const bool from_grad = !j.narrow;
    if ((s = cert_compute(c, solver_point(c), solver_point(c) + j.mk, &j.cert, false, false,
                          from_grad ? solver_gradient(c) : nullptr, from_grad ? solver_f_device(c) : nullptr,
                          st.f)) != RPCA_OK)
      return s;
    ++j.cert_evals;
    bool rank_deficit = false;
    if (cert_meets(j.cert, c->opt.cert_tol)) {
      // Same point as the cheap evaluation just made: only the spectral step is added.
      if ((s = cert_compute(c, solver_point(c), solver_point(c) + j.mk, &j.cert, true, true)) != RPCA_OK) return s;
      if (cert_meets(j.cert, c->opt.cert_tol)) j.certified = true;
      else rank_deficit = j.cert.t4 > 0.0;
    }
    j.timer->end();
    // Stationary in the factors' range (t1..t3 meet the tolerance) with a direction outside
    // it that would lower F (t4 > 0): more iterations at this rank cannot certify; the
    // rank-increasing solve takes over from here (Sec. 4.1).
    if (j.certified || (rank_deficit && c->grow_stop)) {
      j.done = true;
      return RPCA_OK;
    }
    const double gn = sqrt(fmax(st.gg, 0.0));
    if (gn > 0.0 && std::isfinite(j.cert.cert_rel) && std::isfinite(gn)) j.kappa = j.cert.cert_rel / gn;
    // The narrow phase has done its part once the float32 certificate stops halving
    // between checks: what is left is the storage rounding of X.
    if (j.narrow && c->opt.refine_fp32) {
      const bool plateau = j.cert.cert_rel > 0.5 * j.narrow_best;
      j.narrow_best = std::min(j.narrow_best, j.cert.cert_rel);
      if (plateau) {
        if ((s = job_refine(j)) != RPCA_OK) return s;
        *again = true;
        return RPCA_OK;
      }
    }
  }
  if (c->opt.timeout_s > 0) {
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - j.t0).count();
    if (el > c->opt.timeout_s) j.done = true;
  }
  return RPCA_OK;
}

// Advances the job until it has iterations in flight (returns with them launched) or is
// done (j.done).
static rpca_status job_step(SolveJob& j) {
  rpca_ctx* c = j.c;
  rpca_status s;
  while (true) {
    if ((s = solver_read_scalars(c, &j.st)) != RPCA_OK) return s;
    bool again = false;
    if ((s = job_decide(j, &again)) != RPCA_OK) return s;
    if (j.done) return RPCA_OK;
    if (again) continue;
    const SolverState& st = j.st;
    int batch = j.every > 0 ? j.every - (st.iter % j.every) : 25;
    if (j.every > 0 && !j.narrow && j.kappa > 0.0 && !c->lk)
      batch = std::max(1, std::min(CERT_POLL, 2 * j.every - (st.iter - j.last_cert_iter)));
    batch = std::max(1, std::min(batch, c->opt.max_iter - j.iter_base - st.iter));
    j.timer->begin(1);
    if ((s = solver_iterations(c, batch)) != RPCA_OK) return s;
    j.timer->end();
    if (!j.launched && cudaEventCreateWithFlags(&j.launched, cudaEventDisableTiming) != cudaSuccess) {
      j.launched = nullptr;
      return cuda_err(c, cudaGetLastError(), "creating a job event");
    }
    if (cudaEventRecord(j.launched, c->stream) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "job event");
    return RPCA_OK;
  }
}

static rpca_status job_finish(SolveJob& j, rpca_result* res) {
  rpca_ctx* c = j.c;
  rpca_status s;
  if ((s = check_dev_err(c)) != RPCA_OK) return s;
  cudaMemcpyAsync(j.U, solver_point(c), sizeof(float) * j.mk, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(j.V, solver_point(c) + j.mk, sizeof(float) * j.nk, cudaMemcpyDeviceToDevice, c->stream);
  if (!j.certified && !c->lk) {
    j.timer->begin(2);
    if ((s = cert_compute(c, j.U, j.V, &j.cert, true)) != RPCA_OK) return s;
    j.timer->end();
    ++j.cert_evals;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "rpca_solve");
  // Four kernels (fused pass, finalize and line-search step, inner products, direction) per
  // pass of the iteration graph's while body: one pass per trial, and one (early-exit) pass in
  // every graph launch that ran no trial.
  const int64_t gl = c->graph_launches - j.graph_launches0;
  if (gl > 0) count_launches(c, 4LL * std::max<int64_t>(gl, (int64_t)(j.evals_base + j.st.evals) - 1));
  rpca_result r;
  memset(&r, 0, sizeof r);
  j.timer->collect(&r.ms_init, &r.ms_iter, &r.ms_cert);
  r.F = j.narrow ? j.cert.F : j.st.f;  // the float32 objective (the narrow phase's st.f is not)
  r.iters = j.iter_base + j.st.iter;
  r.evals = j.evals_base + j.st.evals;
  r.cert_evals = j.cert_evals;
  r.cert = j.cert;
  r.init_used = j.init_used;
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - j.t0).count();
  // Ranks above 16 have no certificate here: the solver's gradient test decides.
  if (c->lk) r.status = j.st.stop == STOP_GTOL ? RPCA_OK : RPCA_ENOTCONV;
  else r.status = cert_meets(j.cert, c->opt.cert_tol) ? RPCA_OK : RPCA_ENOTCONV;
  if (r.F < c->F_best) c->F_best = r.F;
  if (res) *res = r;
  if (r.status != RPCA_OK) {
    char buf[200];
    if (c->lk)
      snprintf(buf, sizeof buf, "stopped after %d iterations (reason %d) before the gradient test (gtol %.1e)",
               r.iters, j.st.stop, c->opt.gtol);
    else
      snprintf(buf, sizeof buf, "stopped after %d iterations (reason %d) with cert_rel %.3e, trunc_rel %.3e (tol %.1e)",
               r.iters, j.st.stop, j.cert.cert_rel, j.cert.trunc_rel, c->opt.cert_tol);
    set_err(c, RPCA_ENOTCONV, buf);
  }
  return r.status;
}

}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_solve(rpca_ctx* c, float* U, float* V, rpca_result* res) {
  if (!c) return RPCA_EINVAL;
  if (!U || !V) return set_err(c, RPCA_EINVAL, "U and V are required");
  SolveJob j;
  rpca_status s = job_start(j, c, U, V);
  while (s == RPCA_OK && !j.done) s = job_step(j);
  if (s != RPCA_OK) return s;
  return job_finish(j, res);
}

namespace rpca {

// Many solves: the jobs are split over up to `threads` host threads (largest instances first,
// each to the least loaded thread); a thread starts its jobs (initialisation, iteration graph)
// and then steps them round-robin.  A step waits for its own context's stream only, so the
// other jobs' iterations keep the GPU busy meanwhile, and a thread blocked in one job's
// certificate holds up only the jobs of its own share.
rpca_status solver_capture_rounds(rpca_ctx* c, cudaStream_t s, int rounds);  // solver.cu
SolverState* solver_state_dev(rpca_ctx* c);
rpca_status solver_deactivate(rpca_ctx* c, cudaStream_t s);

// Each instance's scalars the host decides on, into out[6 i ..]: active, iteration, ||g||^2,
// F, stop reason, evaluations.
__global__ void gather_scalars_kernel(SolverState* const* sts, int count, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const SolverState* st = sts[i];
    double* o = out + 6 * (size_t)i;
    if (!st) {
      o[0] = 0.0;
      continue;
    }
    o[0] = st->active;
    o[1] = st->iter;
    o[2] = st->gg;
    o[3] = st->f;
    o[4] = st->stop;
    o[5] = st->evals;
  }
}

// The batched form's graph: ROUNDS_PER_LAUNCH L-BFGS iterations of every instance, each
// instance on a branch of its own (the iteration ensure_solver captures, repeated), then the
// gather of every instance's scalars into pinned host memory.  Kept by the batch across solves
// while every instance keeps its solver buffers.
constexpr int ROUNDS_PER_LAUNCH = 5;
struct RoundsGraph {
  int count = 0;
  cudaStream_t M = nullptr;               // the stream the graph runs on
  std::vector<cudaStream_t> fork;         // capture branches
  std::vector<cudaEvent_t> join;
  cudaEvent_t ev = nullptr;
  std::vector<const void*> key;           // each instance's solver state at capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  SolverState** d_states = nullptr;
  double* d_out = nullptr;
  double* h_out = nullptr;                // pinned
};

void rounds_free(RoundsGraph* g) {
  if (!g) return;
  if (g->M) cudaStreamSynchronize(g->M);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (cudaStream_t s : g->fork) cudaStreamDestroy(s);
  for (cudaEvent_t e : g->join) cudaEventDestroy(e);
  if (g->ev) cudaEventDestroy(g->ev);
  if (g->M) cudaStreamDestroy(g->M);
  cudaFree(g->d_states);
  cudaFree(g->d_out);
  cudaFreeHost(g->h_out);
  delete g;
}

// Makes (or reuses) the graph for the instances ctx[0..count) whose flag live[i] is set.
static rpca_status rounds_graph(RoundsGraph* g, rpca_ctx* const* ctx, int count, const std::vector<char>& live) {
  std::vector<const void*> key(count, nullptr);
  for (int i = 0; i < count; ++i) key[i] = live[i] ? solver_state_dev(ctx[i]) : nullptr;
  if (g->exec && g->count == count && g->key == key) return RPCA_OK;
  rpca_ctx* c0 = ctx[0];
  auto fail = [&](cudaError_t e, const char* what) { return cuda_err(c0, e, what); };
  cudaError_t e;
  if (g->count != count) {
    if (g->d_states) return set_err(c0, RPCA_EUNSUPPORTED, "batch size changed");
    g->count = count;
    if ((e = cudaStreamCreateWithFlags(&g->M, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
    if ((e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    g->fork.assign(count, nullptr);
    g->join.assign(count, nullptr);
    for (int i = 0; i < count; ++i) {
      if ((e = cudaStreamCreateWithFlags(&g->fork[i], cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
      if ((e = cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    }
    if ((e = cudaMalloc(&g->d_states, sizeof(SolverState*) * count)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&g->d_out, sizeof(double) * 6 * count)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMallocHost(&g->h_out, sizeof(double) * 6 * count)) != cudaSuccess) return fail(e, "cudaMallocHost");
  }
  if (g->exec) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  if (g->graph) {
    cudaGraphDestroy(g->graph);
    g->graph = nullptr;
  }
  std::vector<SolverState*> sts(count, nullptr);
  for (int i = 0; i < count; ++i) sts[i] = live[i] ? solver_state_dev(ctx[i]) : nullptr;
  if ((e = cudaMemcpyAsync(g->d_states, sts.data(), sizeof(SolverState*) * count, cudaMemcpyHostToDevice, g->M)) !=
      cudaSuccess)
    return fail(e, "state table");
  if ((e = cudaStreamSynchronize(g->M)) != cudaSuccess) return fail(e, "state table");
  if ((e = cudaStreamBeginCapture(g->M, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return fail(e, "capture");
  rpca_status st = RPCA_OK;
  e = cudaEventRecord(g->ev, g->M);
  for (int i = 0; i < count && e == cudaSuccess && st == RPCA_OK; ++i) {
    if (!live[i]) continue;
    if ((e = cudaStreamWaitEvent(g->fork[i], g->ev, 0)) != cudaSuccess) break;
    if ((st = solver_capture_rounds(ctx[i], g->fork[i], ROUNDS_PER_LAUNCH)) != RPCA_OK) break;
    if ((e = cudaEventRecord(g->join[i], g->fork[i])) != cudaSuccess) break;
    e = cudaStreamWaitEvent(g->M, g->join[i], 0);
  }
  if (e == cudaSuccess && st == RPCA_OK) {
    gather_scalars_kernel<<<(count + 127) / 128, 128, 0, g->M>>>(g->d_states, count, g->d_out);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->h_out, g->d_out, sizeof(double) * 6 * count, cudaMemcpyDeviceToHost, g->M);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(g->M, &graph);
  if (st != RPCA_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(e, "capturing the batched graph");
  }
  g->graph = graph;
  if ((e = cudaGraphInstantiate(&g->exec, graph, 0)) != cudaSuccess) return fail(e, "instantiating the batched graph");
  g->key = key;
  return RPCA_OK;
}

rpca_status solve_jobs(rpca_ctx* const* ctx, float* const* U, float* const* V, rpca_result* res, int count,
                       rpca_status* status, int threads) {
  std::vector<SolveJob> jobs(count);
  threads = std::max(1, std::min(threads, count));
  std::vector<std::vector<int>> share(threads);
  {
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    auto work = [&](int i) { return (double)ctx[i]->m * (double)ctx[i]->n * (double)ctx[i]->k; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    std::vector<double> load(threads, 0.0);
    for (int i : order) {
      const int t = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      share[t].push_back(i);
      load[t] += work(i);
    }
  }
  auto run = [&](int t) {
    const std::vector<int>& mine = share[t];
    if (mine.empty()) return;
    cudaSetDevice(ctx[mine[0]]->device);
    std::vector<bool> live(mine.size(), true);
    int remaining = 0;
    for (size_t q = 0; q < mine.size(); ++q) {
      const int i = mine[q];
      status[i] = job_start(jobs[i], ctx[i], U[i], V[i]);
      live[q] = status[i] == RPCA_OK;
      remaining += live[q];
    }
    // Step whichever jobs have finished their queued iterations; a job whose GPU work is still
    // running is passed over rather than waited for, so that no finished job sits idle.
    while (remaining > 0) {
      bool stepped = false;
      for (size_t q = 0; q < mine.size(); ++q) {
        if (!live[q]) continue;
        const int i = mine[q];
        if (!job_ready(jobs[i])) continue;
        stepped = true;
        status[i] = job_step(jobs[i]);
        if (status[i] != RPCA_OK || jobs[i].done) {
          live[q] = false;
          --remaining;
        }
      }
      if (!stepped) std::this_thread::yield();
    }
    for (int i : mine)
      if (status[i] == RPCA_OK) status[i] = job_finish(jobs[i], res ? &res[i] : nullptr);
  };
  if (threads == 1) {
    run(0);
  } else {
    std::vector<std::thread> pool;
    pool.reserve(threads);
    for (int t = 0; t < threads; ++t) pool.emplace_back(run, t);
    for (auto& th : pool) th.join();
  }
  return RPCA_OK;
}


}  // namespace rpca

extern "C" rpca_status rpca_perp_directions(rpca_ctx* c, int qmax, float* U, int64_t ldu, float* V, int64_t ldv,
                                            double* sig, int* q_out);  // cert.cu

// Dynamic rank increase (Sec. 4.1): solve; while the certificate's spectral term shows
// directions the factors cannot represent (singular values of P_U1perp D P_V1perp above lam_L)
// and k < kmax, add one column (sqrt(t_i) u_i, -sqrt(t_i) v_i), t_i = sigma_i - lam_L, per such
// direction (the paper allows growing k aggressively), keep them if F drops, and continue on
// a context with the new rank from the grown point.
extern "C" rpca_status rpca_solve_grow(rpca_ctx* c, float* U, float* V, int kmax, rpca_result* res, int* k_out) {
  if (!c) return RPCA_EINVAL;
  if (!U || !V || !k_out) return set_err(c, RPCA_EINVAL, "U, V and k_out are required");
  if (kmax < c->k || kmax > 16 || kmax > std::min(c->m, c->n))
    return set_err(c, RPCA_EINVAL, "kmax must be in [k, min(16, m, n)]");
  *k_out = c->k;
  rpca_result r, tot;
  memset(&tot, 0, sizeof tot);
  rpca_ctx* cur = c;
  int k = c->k;
  struct GrowFlag {  // set for the duration of the call
    rpca_ctx* c;
    explicit GrowFlag(rpca_ctx* x) : c(x) { c->grow_stop = true; }
    ~GrowFlag() { c->grow_stop = false; }
  } flag(c);
  rpca_status s = rpca_solve(cur, U, V, &r);
  auto add = [&](const rpca_result& x) {
    tot.iters += x.iters;
    tot.evals += x.evals;
    tot.cert_evals += x.cert_evals;
    tot.seconds += x.seconds;
    tot.ms_init += x.ms_init;
    tot.ms_iter += x.ms_iter;
    tot.ms_cert += x.ms_cert;
  };
  add(r);
  if (c->grown.size() < 17) c->grown.resize(17, nullptr);
  while (s == RPCA_ENOTCONV && k < kmax && r.cert.t4 > 0.0 && r.cert.sigma1_perp > c->lam_L) {
    const int64_t m = c->m, n = c->n;
    double sig[16];
    int q = 0;
    // The certificate at the returned point left its Lanczos bases on `cur`.
    rpca_status st = rpca_perp_directions(cur, kmax - k, U + m * k, m, V + n * k, n, sig, &q);
    if (st != RPCA_OK) return st;
    int add_cols = 0;
    while (add_cols < q && sig[add_cols] > c->lam_L) ++add_cols;
    if (add_cols == 0) break;
    for (int t = 0; t < add_cols; ++t) {
      const float sc = (float)std::sqrt(sig[t] - c->lam_L);
      fill_scale(U + m * (k + t), m, sc, cur->stream);
      fill_scale(V + n * (k + t), n, -sc, cur->stream);
    }
    const int k2 = k + add_cols;
    if (!c->grown[k2]) {
      rpca_options o = c->opt;
      o.init = RPCA_INIT_USER;
      rpca_ctx* nx = nullptr;
      st = create_ctx(&nx, m, n, c->X, c->ldx, c->mask, c->ldmask, k2, c->lam_L, c->lam_S, &o, c->stream,
                      c->grid_cap);
      if (st != RPCA_OK) return set_err(c, st, std::string("rank increase: ") + rpca_last_error(nullptr));
      nx->grow_stop = true;  // internal: only ever solved by this function
      c->grown[k2] = nx;
    }
    rpca_ctx* nxt = c->grown[k2];
    // Keep the columns only if the objective drops.
    double f_new = 0.0;
    float* g = nullptr;
    if (cudaMalloc(&g, sizeof(float) * (m + n) * k2) != cudaSuccess) return set_err(c, RPCA_ENOMEM, "cudaMalloc");
    st = rpca_fg(nxt, U, V, &f_new, g, g + m * k2);
    cudaStreamSynchronize(nxt->stream);
    cudaFree(g);
    if (st != RPCA_OK) return st;
    if (!(f_new < r.F)) {
      cudaMemsetAsync(U + m * k, 0, sizeof(float) * m * add_cols, cur->stream);
      cudaMemsetAsync(V + n * k, 0, sizeof(float) * n * add_cols, cur->stream);
      break;
    }
    k = k2;
    cur = nxt;
    s = rpca_solve(cur, U, V, &r);
    add(r);
  }
  *k_out = k;
  if (res) {
    rpca_result o = r;
    o.iters = tot.iters;
    o.evals = tot.evals;
    o.cert_evals = tot.cert_evals;
    o.seconds = tot.seconds;
    o.ms_init = tot.ms_init;
    o.ms_iter = tot.ms_iter;
    o.ms_cert = tot.ms_cert;
    o.init_used = c->opt.init;
    *res = o;
  }
  if (s != RPCA_OK && cur != c) set_err(c, s, rpca_last_error(cur));
  return s;
}

namespace rpca {

// fn(i) for the items in `items`, shared among up to `threads` host threads (each sets the
// device first).
template <typename F>
static void parallel_items(const std::vector<int>& items, int threads, int device, F fn) {
  const int nt = std::max(1, std::min(threads, (int)items.size()));
  if (nt == 1) {
    for (int i : items) fn(i);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&, t] {
      cudaSetDevice(device);
      for (size_t q = t; q < items.size(); q += nt) fn(items[q]);
    });
  for (auto& th : pool) th.join();
}

// The batched form in rounds: every instance is started (its initialisation and first
// direction, host threads in parallel), then one graph launch advances every unfinished
// instance by ROUNDS_PER_LAUNCH L-BFGS iterations at once -- the instances' kernels on
// branches of one graph, no host work between them -- and ends with the gather of every
// instance's scalars; between launches the host takes the same decisions as a single solve
// (certificate when due, stop tests), the certificates of the instances that need one in
// parallel, and a finished instance's iteration is switched off on the device.  Float32
// storage of X and factor ranks up to 16 (the device iteration); otherwise solve_jobs.
rpca_status solve_jobs_rounds(rpca_ctx* const* ctx, float* const* U, float* const* V, rpca_result* res, int count,
                              rpca_status* status, int threads, RoundsGraph** cache) {
  const int device = ctx[0]->device;
  std::vector<SolveJob> jobs(count);
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) all[i] = i;
  // Start every instance.
  parallel_items(all, threads, device, [&](int i) { status[i] = job_start(jobs[i], ctx[i], U[i], V[i]); });
  std::vector<char> live(count, 0);
  for (int i = 0; i < count; ++i) live[i] = status[i] == RPCA_OK;
  if (!*cache) *cache = new RoundsGraph();
  RoundsGraph* g = *cache;
  rpca_status s = rounds_graph(g, ctx, count, live);
  if (s != RPCA_OK) {
    for (int i = 0; i < count; ++i)
      if (status[i] == RPCA_OK) status[i] = s;
    return s;
  }
  // The graph's stream waits for every start.
  for (int i = 0; i < count; ++i) {
    if (!live[i]) continue;
    cudaEventRecord(g->join[i], ctx[i]->stream);
    cudaStreamWaitEvent(g->M, g->join[i], 0);
  }
  int remaining = 0;
  for (int i = 0; i < count; ++i) remaining += live[i];
  while (remaining > 0) {
    cudaError_t e = cudaGraphLaunch(g->exec, g->M);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->M);
    if (e != cudaSuccess) {
      for (int i = 0; i < count; ++i)
        if (live[i]) status[i] = cuda_err(ctx[i], e, "batched graph");
      return status[0];
    }
    ctx[0]->graph_launches += 1;
    std::vector<int> decide;
    for (int i = 0; i < count; ++i) {
      if (!live[i]) continue;
      SolveJob& j = jobs[i];
      const double* o = g->h_out + 6 * (size_t)i;
      j.st.active = (int)o[0];
      j.st.iter = (int)o[1];
      j.st.gg = o[2];
      j.st.f = o[3];
      j.st.stop = (int)o[4];
      j.st.evals = (int)o[5];
      const bool stop = !j.st.active || j.st.iter >= ctx[i]->opt.max_iter - j.iter_base;
      if (stop || cert_due(j, j.st, ctx[i]->opt.cert_tol) || ctx[i]->opt.timeout_s > 0) decide.push_back(i);
    }
    if (decide.empty()) continue;
    parallel_items(decide, threads, device, [&](int i) {
      bool again = false;
      status[i] = job_decide(jobs[i], &again);
      if (status[i] == RPCA_OK && jobs[i].done && jobs[i].st.active) status[i] = solver_deactivate(ctx[i], ctx[i]->stream);
    });
    for (int i : decide) {
      if (status[i] != RPCA_OK || jobs[i].done) {
        live[i] = 0;
        --remaining;
      }
      cudaEventRecord(g->join[i], ctx[i]->stream);
      cudaStreamWaitEvent(g->M, g->join[i], 0);
    }
  }
  // The results, ordered after the last graph launch.
  cudaEventRecord(g->ev, g->M);
  std::vector<int> done;
  for (int i = 0; i < count; ++i)
    if (status[i] == RPCA_OK) done.push_back(i);
  parallel_items(done, threads, device, [&](int i) {
    cudaStreamWaitEvent(ctx[i]->stream, g->ev, 0);
    status[i] = job_finish(jobs[i], res ? &res[i] : nullptr);
  });
  return RPCA_OK;
}

// ---- The grouped form ----------------------------------------------------------------------
// Every instance is started (initialisation and first direction, host threads in parallel);
// then the group stream runs chunks of GROUP_ROUNDS trial rounds, each round one fused-pass
// launch per group of instances with the same instantiation and block size and one launch
// each of the assembly + line-search step, the inner products + scalar part and the direction
// over all listed instances (solver_group_round), and ends with the gather of the listed
// instances' scalars.  Between chunks the host takes each listed instance's decisions as a
// single solve does: an instance whose certificate is due, or that stopped, leaves the list
// and a worker thread evaluates its certificate on the instance's own stream while the
// others keep iterating; it rejoins (or is finished) when the worker is done.  An instance
// that stops inside a chunk idles there (its kernels return at once); it leaves the list at
// the chunk's end.  An instance's trials run the same kernels' arithmetic on the same grids as
// its own iteration graph, so its trajectory does not depend on the others; its decisions
// come after whole chunks of its own trials.
constexpr int GROUP_ROUNDS = 5;
constexpr double GROUP_CERT_MARGIN = 0.5;

struct GroupCache {
  int count = 0;
  cudaStream_t gs = nullptr;
  cudaEvent_t chunk_ev = nullptr;
  std::vector<cudaEvent_t> resume;  // per instance, on its own stream
  unsigned char* d_rec = nullptr;
  unsigned char* h_rec = nullptr;   // pinned
  int* d_idx = nullptr;
  int* h_idx = nullptr;             // pinned
  size_t idx_cap = 0;
  double* d_out = nullptr;
  double* h_out = nullptr;          // pinned
};

void group_free(GroupCache* g) {
  if (!g) return;
  if (g->gs) cudaStreamSynchronize(g->gs);
  for (cudaEvent_t e : g->resume)
    if (e) cudaEventDestroy(e);
  if (g->chunk_ev) cudaEventDestroy(g->chunk_ev);
  if (g->gs) cudaStreamDestroy(g->gs);
  dev_free(g->d_rec);
  dev_free(g->d_idx);
  dev_free(g->d_out);
  host_pinned_free(g->h_rec);
  host_pinned_free(g->h_idx);
  host_pinned_free(g->h_out);
  delete g;
}

static rpca_status group_setup(GroupCache* g, rpca_ctx* c0, int count) {
  if (g->count == count) return RPCA_OK;
  if (g->count != 0) return set_err(c0, RPCA_EUNSUPPORTED, "batch size changed");
  auto fail = [&](cudaError_t e, const char* what) { return cuda_err(c0, e, what); };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&g->gs, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
  if ((e = cudaEventCreateWithFlags(&g->chunk_ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
  g->resume.assign(count, nullptr);
  for (int i = 0; i < count; ++i)
    if ((e = cudaEventCreateWithFlags(&g->resume[i], cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
  const size_t rb = solver_group_stride() * (size_t)count;
  if ((e = dev_alloc(&g->d_rec, rb)) != cudaSuccess) return fail(e, "records");
  if ((e = host_pinned_alloc(&g->h_rec, rb)) != cudaSuccess) return fail(e, "records");
  // Lists: per fused-pass group its ids and offsets (2 c_g + 1 entries), then the ids and three
  // offset arrays of the other launches (4 n + 3): at most 7 count + 3 entries (a group per
  // instance at most).
  g->idx_cap = 7 * (size_t)count + 3;
  if ((e = dev_alloc(&g->d_idx, sizeof(int) * g->idx_cap)) != cudaSuccess) return fail(e, "lists");
  if ((e = host_pinned_alloc(&g->h_idx, sizeof(int) * g->idx_cap)) != cudaSuccess) return fail(e, "lists");
  if ((e = dev_alloc(&g->d_out, sizeof(double) * 6 * count)) != cudaSuccess) return fail(e, "scalars");
  if ((e = host_pinned_alloc(&g->h_out, sizeof(double) * 6 * count)) != cudaSuccess) return fail(e, "scalars");
  g->count = count;
  return RPCA_OK;
}

// Whether the grouped form can run this batch (every instance eligible, one device).
bool group_eligible(rpca_ctx* const* ctx, int count) {
  for (int i = 0; i < count; ++i)
    if (!solver_group_eligible(ctx[i]) || ctx[i]->device != ctx[0]->device) return false;
  return true;
}

rpca_status solve_jobs_grouped(rpca_ctx* const* ctx, float* const* U, float* const* V, rpca_result* res, int count,
                               rpca_status* status, int threads, GroupCache** cache) {
  const int device = ctx[0]->device;
  if (!*cache) *cache = new GroupCache();
  GroupCache* g = *cache;
  rpca_status s = group_setup(g, ctx[0], count);
  if (s != RPCA_OK) {
    for (int i = 0; i < count; ++i) status[i] = s;
    return s;
  }
  std::vector<SolveJob> jobs(count);
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) {
    all[i] = i;
    ctx[i]->no_iter_graph = true;
  }
  parallel_items(all, threads, device, [&](int i) { status[i] = job_start(jobs[i], ctx[i], U[i], V[i]); });
  for (SolveJob& j : jobs) j.margin = GROUP_CERT_MARGIN;
  // Records, and the group stream ordered after every start.
  const size_t stride = solver_group_stride();
  std::vector<GroupMember> mem(count);
  std::vector<char> live(count, 0);  // 1: in the lists; 0: with a worker or finished
  std::vector<char> finished(count, 0);
  for (int i = 0; i < count; ++i) {
    if (status[i] == RPCA_OK) status[i] = solver_group_member(ctx[i], g->h_rec + stride * i, &mem[i]);
    if (status[i] != RPCA_OK) {
      finished[i] = 1;
      continue;
    }
    live[i] = 1;
    cudaEventRecord(g->resume[i], ctx[i]->stream);
    cudaStreamWaitEvent(g->gs, g->resume[i], 0);
  }
  // Fused-pass groups: instances with the same grouped instantiation and block size.
  std::vector<std::pair<const void*, int>> gkey;
  std::vector<size_t> gsmem;
  std::vector<int> gof(count, -1);
  for (int i = 0; i < count; ++i) {
    if (!live[i]) continue;
    const std::pair<const void*, int> key{mem[i].fg_fn, mem[i].fg_threads};
    size_t q = 0;
    while (q < gkey.size() && gkey[q] != key) ++q;
    if (q == gkey.size()) {
      gkey.push_back(key);
      gsmem.push_back(0);
    }
    gof[i] = (int)q;
    gsmem[q] = std::max(gsmem[q], mem[i].fg_smem);
  }
  for (size_t q = 0; q < gkey.size(); ++q)
    if (!allow_smem(gkey[q].first, gsmem[q])) {
      for (int i = 0; i < count; ++i)
        if (live[i]) status[i] = set_err(ctx[i], RPCA_ECUDA, "shared memory of the grouped fused pass");
      return RPCA_ECUDA;
    }
  cudaError_t e = cudaMemcpyAsync(g->d_rec, g->h_rec, stride * count, cudaMemcpyHostToDevice, g->gs);
  if (e != cudaSuccess) {
    for (int i = 0; i < count; ++i)
      if (live[i]) status[i] = cuda_err(ctx[i], e, "records");
    return status[0];
  }

  // Worker threads for the decisions (certificates) of instances that left the lists.
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int> work, done_q;
  bool quit = false;
  const int nworkers = std::max(1, std::min(threads, count));
  std::vector<std::thread> workers;
  workers.reserve(nworkers);
  for (int t = 0; t < nworkers; ++t)
    workers.emplace_back([&] {
      cudaSetDevice(device);
      while (true) {
        int i;
        {
          std::unique_lock<std::mutex> lk(mu);
          cv_work.wait(lk, [&] { return quit || !work.empty(); });
          if (work.empty()) return;
          i = work.front();
          work.pop_front();
        }
        bool again = false;
        status[i] = job_decide(jobs[i], &again);
        if (status[i] == RPCA_OK && jobs[i].done && jobs[i].st.active)
          status[i] = solver_deactivate(ctx[i], ctx[i]->stream);
        cudaEventRecord(g->resume[i], ctx[i]->stream);
        {
          std::lock_guard<std::mutex> lk(mu);
          done_q.push_back(i);
        }
        cv_done.notify_one();
      }
    });

  int64_t launches = 0;
  int pending = 0;
  std::vector<int> list;        // the listed instances of the current chunk
  bool lists_stale = true;
  std::vector<GroupFgList> fgl;
  GroupRound R{};
  rpca_status err = RPCA_OK;
  while (err == RPCA_OK) {
    // Decisions that finished: rejoin or finish.  With no instance left to iterate, wait for
    // one; with none pending either, the batch is done.
    {
      std::unique_lock<std::mutex> lk(mu);
      if (std::none_of(live.begin(), live.end(), [](char v) { return v != 0; })) {
        if (pending == 0) break;
        cv_done.wait(lk, [&] { return !done_q.empty(); });
      }
      while (!done_q.empty()) {
        const int i = done_q.front();
        done_q.pop_front();
        --pending;
        if (status[i] != RPCA_OK || jobs[i].done) {
          finished[i] = 1;
        } else {
          live[i] = 1;
          cudaStreamWaitEvent(g->gs, g->resume[i], 0);
        }
        lists_stale = true;
      }
    }
    if (lists_stale) {
      list.clear();
      for (int i = 0; i < count; ++i)
        if (live[i]) list.push_back(i);
      if (list.empty()) continue;
      // Lay out the lists in h_idx: per group ids, offsets; then ids and the three offsets.
      int* h = g->h_idx;
      size_t pos = 0;
      fgl.assign(gkey.size(), GroupFgList{});
      std::vector<size_t> gpos(gkey.size());
      for (size_t q = 0; q < gkey.size(); ++q) {
        int cnt = 0;
        for (int i : list) cnt += gof[i] == (int)q;
        GroupFgList& F = fgl[q];
        F.fn = gkey[q].first;
        F.threads = gkey[q].second;
        F.smem = gsmem[q];
        F.cnt = cnt;
        F.ids = g->d_idx + pos;
        F.off = g->d_idx + pos + cnt;
        int* ids = h + pos;
        int* off = h + pos + cnt;
        int c = 0, b = 0;
        off[0] = 0;
        for (int i : list)
          if (gof[i] == (int)q) {
            ids[c] = i;
            b += mem[i].fg_blocks;
            off[++c] = b;
          }
        F.blocks = b;
        pos += 2 * (size_t)cnt + 1;
      }
      const int n = (int)list.size();
      int* ids = h + pos;
      int* fo = ids + n;
      int* dof = fo + n + 1;
      int* rof = dof + n + 1;
      fo[0] = dof[0] = rof[0] = 0;
      for (int q = 0; q < n; ++q) {
        const int i = list[q];
        ids[q] = i;
        fo[q + 1] = fo[q] + mem[i].fin_blocks;
        dof[q + 1] = dof[q] + mem[i].dots_blocks;
        rof[q + 1] = rof[q] + mem[i].dir_blocks;
      }
      R.rec = g->d_rec;
      R.stride = stride;
      R.fg = fgl.data();
      R.nfg = (int)fgl.size();
      R.cnt = n;
      R.ids = g->d_idx + pos;
      R.fin_off = R.ids + n;
      R.dots_off = R.fin_off + n + 1;
      R.dir_off = R.dots_off + n + 1;
      R.fin_blocks = fo[n];
      R.dots_blocks = dof[n];
      R.dir_blocks = rof[n];
      R.mcap = mem[list[0]].mcap;
      pos += (size_t)n + 3 * ((size_t)n + 1);
      if ((e = cudaMemcpyAsync(g->d_idx, h, sizeof(int) * pos, cudaMemcpyHostToDevice, g->gs)) != cudaSuccess) {
        err = RPCA_ECUDA;
        break;
      }
      lists_stale = false;
    }
    // One chunk of rounds, then the listed instances' scalars.
    for (int r = 0; r < GROUP_ROUNDS && e == cudaSuccess; ++r) e = solver_group_round(R, g->gs, &launches);
    if (e == cudaSuccess) e = solver_group_gather(g->d_rec, R.ids, R.cnt, g->d_out, g->gs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->h_out, g->d_out, sizeof(double) * 6 * R.cnt, cudaMemcpyDeviceToHost, g->gs);
    if (e == cudaSuccess) e = cudaEventRecord(g->chunk_ev, g->gs);
    if (e == cudaSuccess) e = cudaEventSynchronize(g->chunk_ev);
    if (e != cudaSuccess) {
      err = RPCA_ECUDA;
      break;
    }
    launches += 1;
    for (int q = 0; q < (int)list.size(); ++q) {
      const int i = list[q];
      SolveJob& j = jobs[i];
      const double* o = g->h_out + 6 * (size_t)q;
      j.st.active = (int)o[0];
      j.st.iter = (int)o[1];
      j.st.gg = o[2];
      j.st.f = o[3];
      j.st.stop = (int)o[4];
      j.st.evals = (int)o[5];
      const bool stop = !j.st.active || j.st.iter >= ctx[i]->opt.max_iter - j.iter_base;
      if (stop || cert_due(j, j.st, ctx[i]->opt.cert_tol) || ctx[i]->opt.timeout_s > 0) {
        live[i] = 0;
        lists_stale = true;
        {
          std::lock_guard<std::mutex> lk(mu);
          work.push_back(i);
          ++pending;
        }
        cv_work.notify_one();
      }
    }
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    quit = true;
  }
  cv_work.notify_all();
  for (auto& th : workers) th.join();
  count_launches(ctx[0], launches);
  if (err != RPCA_OK) {
    for (int i = 0; i < count; ++i) ctx[i]->no_iter_graph = false;
    for (int i = 0; i < count; ++i)
      if (status[i] == RPCA_OK) status[i] = cuda_err(ctx[i], e, "grouped iteration");
    return status[0];
  }
  // Later solves of these contexts capture their own iteration graph again.
  for (int i = 0; i < count; ++i) ctx[i]->no_iter_graph = false;
  // The results, ordered after the last chunk.
  cudaEventRecord(g->chunk_ev, g->gs);
  std::vector<int> fin;
  for (int i = 0; i < count; ++i)
    if (status[i] == RPCA_OK) fin.push_back(i);
  parallel_items(fin, threads, device, [&](int i) {
    cudaStreamWaitEvent(ctx[i]->stream, g->chunk_ev, 0);
    status[i] = job_finish(jobs[i], res ? &res[i] : nullptr);
  });
  return RPCA_OK;
}
}  // namespace rpca
