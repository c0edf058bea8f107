// Device-resident state of the L-BFGS solver (read by the host between graph launches).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rpca.h"

namespace rpca {

constexpr int SOLVER_MAX_SLOTS = 33;  // history slots: memory cap (<= 32) + 1 spare
constexpr int SOLVER_LOG = 256;       // per-iteration log ring
constexpr int SOLVER_TLOG = 256;      // per-trial log ring

enum { LS_RUNNING = 0, LS_ACCEPTED = 1, LS_FAILED = 2, LS_NONE = 3 };
enum { STOP_NONE = 0, STOP_GTOL = 1, STOP_MAXITER = 2, STOP_LSFAIL = 3, STOP_CERT = 4, STOP_TIMEOUT = 5,
       STOP_NONFINITE = 6 };

struct LineSearch {
  double f0, g0;                  // phi(0), phi'(0)
  double a;                       // current trial step
  double a_prev, f_prev, g_prev;  // previous trial of the bracketing phase
  double lo, flo, glo;            // zoom bracket, left end: phi'(lo) < 0, phi(lo) <= phi(0) + noise
  double hi, fhi, ghi;            // right end: phi'(hi) >= 0 or phi(hi) too large
  double width_prev;              // bracket width before the last zoom trial
  double f_acc;                   // objective at the accepted step
  double best_a, best_gg;         // trial with the smallest ||g||^2 among those with f <= f(0) + noise
  int force;                      // the current trial is the fallback: accept it
  int phase;                      // 0 bracketing, 1 zoom
  int first;                      // first trial of the bracketing phase
  int evals;                      // trials in this line search
  int state;                      // LS_*
};

struct SolverState {
  double f, gg, g1, best_f;
  double out[4];  // finalize output of the last trial: f, g.d, ||g||^2, ||x||^2
  LineSearch ls;
  int mem, count, spare;
  // Set by the scalar part when a line search has accepted its trial: the direction kernel
  // then moves x, g to the trial point and stores the new pair in slot acc_slot (-1: the
  // pair failed the curvature test and is not kept), and its last block clears acc_flag.
  int acc_flag, acc_slot;
  // Set by the scalar part when it has formed new two-loop coefficients; the direction kernel
  // then forms d and its last block clears it.
  int dir_pending;
  // The iteration graph loops over line-search trials while active and iter < target (set
  // from the host's iteration count before each launch), and at most loop_budget passes: a
  // bound that holds whatever the state, so that a launch always ends.
  int target, loop_budget;
  int ids[SOLVER_MAX_SLOTS];  // history slots in the ring, newest first
  // The Gram table, the two-loop coefficients and the inner products they come from are
  // float32: their inputs are float32 vectors, the direction is formed with float32
  // coefficients, and a float64 operation costs 64 cycles on GB300 (a divide ~570), which
  // made the two-loop recursion the longest step of an iteration.
  float SY[SOLVER_MAX_SLOTS][SOLVER_MAX_SLOTS];  // s_i . y_j by slot
  float YY[SOLVER_MAX_SLOTS][SOLVER_MAX_SLOTS];  // y_i . y_j by slot
  float sg[SOLVER_MAX_SLOTS], yg[SOLVER_MAX_SLOTS];
  float coef_g, coef_s[SOLVER_MAX_SLOTS], coef_y[SOLVER_MAX_SLOTS];
  int iter, evals, active, gate, stop, fails, max_iter;
  double gtol;
  double ls_noise;  // relative noise level of f for the approximate Wolfe test
  // Per-iteration log ring: {iteration, f, ||g||, accepted step, line-search trials,
  // outcome (LS_*), history pairs in use}, newest at (log_n - 1) % SOLVER_LOG.
  int log_n;
  double log[SOLVER_LOG][7];
  // Per-trial log ring: {iteration, trial step a, f(a) - f(0), phi'(a) / |phi'(0)|, ||g(a)||^2,
  // phase (0 bracketing, 1 zoom), trial number}, newest at (tlog_n - 1) % SOLVER_TLOG.
  int tlog_n;
  double tlog[SOLVER_TLOG][7];
};

// ---- Grouped iteration: the line-search trials of many instances in shared launches ----
// A round advances every listed instance by one trial, as one pass of the iteration graph's
// body does for one instance: the fused pass (one launch per group of instances that share
// its instantiation and block size), then one launch each of the assembly with the
// line-search step, the inner products with the scalar part, and the direction, over all
// listed instances.  An instance's kernels read its record (tensor maps, arguments, its own
// solver buffers and tickets), written once per solve.

// Launch sizes of one instance in the grouped form.
struct GroupMember {
  const void* fg_fn = nullptr;  // grouped fused-pass instantiation
  int fg_threads = 0;
  size_t fg_smem = 0;
  int fg_blocks = 0, fin_blocks = 0, dots_blocks = 0, dir_blocks = 0;
  int mcap = 0;
};
// One fused-pass launch: cnt instances ids[] with block offsets off[] (cnt + 1 entries).
struct GroupFgList {
  const void* fn;
  int threads;
  size_t smem;
  int blocks, cnt;
  const int* ids;
  const int* off;
};
struct GroupRound {
  const void* rec;  // device records, `stride` bytes apart
  size_t stride;
  const GroupFgList* fg;
  int nfg;
  int cnt;  // the listed instances of the other three launches and their block offsets
  const int* ids;
  const int* fin_off;
  const int* dots_off;
  const int* dir_off;
  int fin_blocks, dots_blocks, dir_blocks, mcap;
};
size_t solver_group_stride();
// Whether a context's solve can take part (float32 X, unmasked, fused-kernel plan with a
// grouped instantiation, memory cap <= 10); checked before the solve starts.
bool solver_group_eligible(rpca_ctx* c);
// Writes this context's record (host memory, solver_group_stride() bytes, 64-byte aligned)
// and launch sizes; the solver must be prepared (its first direction launched).
rpca_status solver_group_member(rpca_ctx* c, void* rec_host, GroupMember* m);
// Launches one round on s; the kernel launches it made are added to *launches.
cudaError_t solver_group_round(const GroupRound& r, cudaStream_t s, int64_t* launches);
// The host's scalars of the listed instances into out[6 q ..]: active, iteration, ||g||^2, F,
// stop reason, evaluations.
cudaError_t solver_group_gather(const void* rec, const int* ids, int cnt, double* out, cudaStream_t s);

}  // namespace rpca
