// L-BFGS with memory M (Sec. 5.1: memory 10) and a strong-Wolfe line search, run entirely
// on the device.
//
// One iteration is one CUDA-graph launch:
//   WHILE (line search running):  fg_kernel at x + a d, then finalize_ls_kernel (gradient
//                         assembly, the objective's sums and the line-search step)
//   lbfgs_dots1_kernel:   all inner products the two-loop recursion needs, with the new pair
//                         s = x_t - x, y = g_t - g formed on the fly; its last block runs the
//                         scalar part (Gram table update, two-loop recursion, stopping tests,
//                         the next line search's start)
//   lbfgs_direction_kernel:  accept the step (the new pair into the history ring, x <- x_t,
//                         g <- g_t) and d = c_g g + sum_j (c_s[j] s_j + c_y[j] y_j) (g.d comes
//                         from the Gram table).
// The two-loop recursion (Nocedal & Wright Alg. 7.4) is evaluated on inner products only:
// with q = g - sum a_j y_j and r = gamma q + sum c_j s_j, every dot it needs is a
// combination of s_i.g, y_i.g, s_i.y_j and y_i.y_j, which are kept in a Gram table and
// updated with one new row and column per accepted pair.  The line search is the
// bracketing + zoom procedure of Nocedal & Wright Alg. 3.5 / 3.6 with safeguarded cubic
// interpolation (the paper is silent on the line search; its solvers came from minFunc),
// with the approximate Wolfe conditions of Hager & Zhang (2005) for steps whose objective
// change is below the float32 noise level of f.
//
// Products are formed in float32 and summed over a few elements per thread in float32; the
// sums across warps and blocks are float-float (fixed order), the line-search arithmetic is
// float64, the Gram table and the two-loop scalars float32 (a float64 operation takes 64
// cycles on GB300, a float32 one 4, and the scalar part of an iteration is a chain of
// dependent operations).
#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "ctx.h"
#include "fg_kernel.cuh"
#include "fin.cuh"
#include "solver.h"

namespace rpca {

constexpr double LS_C1 = 1e-4, LS_C2 = 0.9, LS_AMAX = 1e10;
constexpr int LS_MAX_TRIALS = 25;

// Elements per thread and step of the inner-product pass, loaded as one vector.
constexpr int DOTS_VEC = 4;

template <int NV>
__device__ __forceinline__ void vec_store(float* p, const float (&v)[NV]) {
  if constexpr (NV == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (NV == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    *p = v[0];
  }
}

// n consecutive floats at p (16-byte aligned for n = 4, 8-byte for n = 2), or zeros when !use.
template <int NV>
__device__ __forceinline__ void vec_load(float (&out)[NV], const float* p, bool use) {
  if constexpr (NV == 4) {
    const float4 t = use ? *reinterpret_cast<const float4*>(p) : make_float4(0.f, 0.f, 0.f, 0.f);
    out[0] = t.x;
    out[1] = t.y;
    out[2] = t.z;
    out[3] = t.w;
  } else if constexpr (NV == 2) {
    const float2 t = use ? *reinterpret_cast<const float2*>(p) : make_float2(0.f, 0.f);
    out[0] = t.x;
    out[1] = t.y;
  } else {
    out[0] = use ? *p : 0.f;
  }
}

constexpr int DOTS_GRP = 16;      // blocks per group of the two-level reduction
constexpr int DOTS_MAX_GRP = 60;  // groups the counter buffer has room for

struct SolverArgs {
  SolverState* st;
  int64_t N;
  float* x;
  float* g;
  float* xt;
  float* gt;
  float* d;
  float* S;  // [(MCAP + 1) * N]
  float* Y;
  double* blk;
  unsigned int* counter;
  cudaGraphConditionalHandle loop_h;  // the iteration graph's while node (in_graph)
  int in_graph;
};

// ---------------------------------------------------------------------------------------------
__device__ double cubic_step(double a, double fa, double ga, double b, double fb, double gb, bool* ok) {
  // Minimiser of the cubic through (a, fa, ga), (b, fb, gb) (Nocedal & Wright Eq. 3.59).
  *ok = false;
  if (a == b) return 0.5 * (a + b);
  const double d1 = ga + gb - 3.0 * (fa - fb) / (a - b);
  const double disc = d1 * d1 - ga * gb;
  if (!isfinite(disc) || disc < 0.0) return 0.5 * (a + b);
  const double d2 = (b > a ? 1.0 : -1.0) * sqrt(disc);
  const double den = gb - ga + 2.0 * d2;
  if (den == 0.0 || !isfinite(den)) return 0.5 * (a + b);
  *ok = true;
  return b - (b - a) * (gb + d2 - d1) / den;
}

// Next trial inside the bracket (lo, hi).  Where the objective values differ by more than
// their noise level, the minimiser of the cubic through both ends (f and phi'); where they
// do not, the secant root of phi' (the objective differences are rounding there, the
// directional derivatives are not).  A bracket that did not shrink to 2/3 of its previous
// width is bisected (Hager & Zhang's safeguard).
__device__ double zoom_trial(const LineSearch& L, double epsf) {
  const double w = L.hi - L.lo;
  const double mid = 0.5 * (L.lo + L.hi);
  if (!isfinite(L.fhi) || !isfinite(L.ghi)) return mid;
  if (L.width_prev > 0.0 && w > 0.66 * L.width_prev) return mid;
  double t;
  if (fabs(L.fhi - L.flo) > 100.0 * epsf) {
    bool ok;
    t = cubic_step(L.lo, L.flo, L.glo, L.hi, L.fhi, L.ghi, &ok);
    if (!ok) return mid;
  } else {
    if (!(L.ghi > L.glo)) return mid;
    t = L.lo - L.glo * w / (L.ghi - L.glo);
  }
  if (!isfinite(t)) return mid;
  return fmin(fmax(t, L.lo + 0.01 * w), L.hi - 0.01 * w);
}

// One step of the line-search state machine after the trial at L.a has been evaluated
// (st->out[0] = phi(a), st->out[1] = phi'(a)), run by one thread.
// in_graph = 0: launched from the host-driven loop (no conditional node to set).
__device__ void ls_step_body(SolverState* st, cudaGraphConditionalHandle h, int in_graph) {
  // One thread runs a chain of dependent decisions: it works on a local copy of the line
  // search and of the scalars it reads (one batch of loads, independent of each other) and
  // writes the copy back once, instead of a round trip to memory per field access.
  const int active = st->active;
  LineSearch L = st->ls;
  if (!active || L.state != LS_RUNNING) {
    st->gate = 0;
    if (in_graph) cudaGraphSetConditional(h, 0);
    return;
  }
  const double a = L.a, fa = st->out[0], ga = st->out[1], gga = st->out[2];
  const double ls_noise = st->ls_noise, gg_cur = st->gg;
  const int evals = st->evals, tlog_n = st->tlog_n, iter = st->iter;
  L.evals += 1;
  st->evals = evals + 1;
  bool accept = false;
  // Sufficient decrease: the Armijo test, or -- once the objective differences are at the
  // noise level of f (|f(a) - f(0)| <= ls_noise |f(0)|) -- the approximate Wolfe test of
  // Hager & Zhang, phi'(a) <= (2 c1 - 1) phi'(0), which uses the (float64-accumulated)
  // directional derivative instead of the noisy function difference.
  const double epsf = ls_noise * fabs(L.f0);
  const bool approx_ok = isfinite(fa) && fa <= L.f0 + epsf && ga <= (2.0 * LS_C1 - 1.0) * L.g0;
  {
    double* rec = st->tlog[tlog_n % SOLVER_TLOG];
    rec[0] = iter;
    rec[1] = a;
    rec[2] = fa - L.f0;
    rec[3] = ga / fabs(L.g0);
    rec[4] = gga;
    rec[5] = L.phase;
    rec[6] = L.evals;
    st->tlog_n = tlog_n + 1;
  }
  if (L.force) {  // the fallback trial (see below) is taken as it is
    L.state = LS_ACCEPTED;
    L.f_acc = fa;
  } else {
    if (isfinite(fa) && fa <= L.f0 + epsf && isfinite(gga) && gga < L.best_gg) {
      L.best_gg = gga;
      L.best_a = a;
    }
    const bool armijo_fail = !isfinite(fa) || (fa > L.f0 + LS_C1 * a * L.g0 && !approx_ok);
    if (L.phase == 0) {  // bracketing (Alg. 3.5)
      if (armijo_fail || (!L.first && fa > L.f_prev + epsf) || (fabs(ga) > -LS_C2 * L.g0 && ga >= 0.0)) {
        // [a_prev, a] holds a point of the strong Wolfe conditions: phi'(a_prev) < 0 and phi
        // there is within the sufficient-decrease band, while at a either phi rose or phi' >= 0.
        L.lo = L.a_prev; L.flo = L.f_prev; L.glo = L.g_prev;
        L.hi = a; L.fhi = fa; L.ghi = ga;
        L.width_prev = 0.0;
        L.phase = 1;
      } else if (fabs(ga) <= -LS_C2 * L.g0) {
        accept = true;
      } else {
        // Extrapolation (Alg. 3.5 leaves the next trial in (a, a_max) open): the secant root of
        // phi' through the last two trials -- the minimiser of the quadratic they define --
        // when phi' rose toward zero, kept within [4 a, 100 a]; 4 a otherwise.
        double t = 4.0 * a;
        if (ga > L.g_prev && L.g_prev < 0.0) {
          const double sec = a - ga * (a - L.a_prev) / (ga - L.g_prev);
          if (isfinite(sec)) t = fmin(fmax(sec, 4.0 * a), 100.0 * a);
        }
        L.a_prev = a; L.f_prev = fa; L.g_prev = ga;
        L.a = fmin(t, LS_AMAX);
        L.first = 0;
      }
    } else {  // zoom (Alg. 3.6), with the bracket kept by the sign of phi' (Hager & Zhang)
      const double w = L.hi - L.lo;
      if (armijo_fail || fa > L.flo + epsf) {
        L.hi = a; L.fhi = fa; L.ghi = ga;
      } else if (fabs(ga) <= -LS_C2 * L.g0) {
        accept = true;
      } else if (ga >= 0.0) {
        L.hi = a; L.fhi = fa; L.ghi = ga;
      } else {
        L.lo = a; L.flo = fa; L.glo = ga;
      }
      L.width_prev = w;
    }
    if (accept) {
      L.state = LS_ACCEPTED;
      L.f_acc = fa;
    } else if (L.evals >= LS_MAX_TRIALS - 1) {
      // Out of trials (at the float32 noise floor the curvature test can stay out of reach):
      // re-evaluate the trial with the smallest gradient among those that did not increase f
      // beyond the noise level, if it improves on the current point, and accept it.
      if (L.best_a > 0.0 && L.best_gg < gg_cur) {
        L.a = L.best_a;
        L.force = 1;
      } else {
        L.state = LS_FAILED;
      }
    } else if (L.phase == 1) {
      L.a = zoom_trial(L, epsf);
    }
  }
  st->ls = L;
  const int running = L.state == LS_RUNNING;
  st->gate = running;
  if (in_graph) cudaGraphSetConditional(h, running ? 1u : 0u);
}

__global__ void ls_step_kernel(SolverState* st, cudaGraphConditionalHandle h, int in_graph) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ls_step_body(st, h, in_graph);
}

// Second stage of a line-search trial in one launch: every block assembles its part of the
// gradient (finalize_body), the last block to finish (ticket) forms the fixed-order sums
// (finalize_reduce_body) and its thread 0 takes the line-search step on them.  The same
// arithmetic in the same order as finalize_kernel + finalize_reduce_kernel + ls_step_kernel,
// two fewer launches per trial.  With the gate closed (no search running) only the step runs,
// which ends the graph's while loop.
// Four CTAs per SM (64 registers): the assembly needs few registers, the single thread that
// takes the line-search step many, and the more of the grid one wave holds the better.
// Block bx of a grid of gx blocks.
__device__ __forceinline__ void finalize_ls_body(const FinArgs& a, SolverState* st, cudaGraphConditionalHandle h,
                                                 int in_graph, unsigned int* ticket, unsigned bx, unsigned gx) {
  __shared__ bool is_last;
  if (a.gate != nullptr && *a.gate == 0) {
    if (bx == 0 && threadIdx.x == 0) ls_step_body(st, h, in_graph);
    return;
  }
  finalize_body(a, bx);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gx - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  finalize_reduce_body(a, (int)gx);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    ls_step_body(st, h, in_graph);
  }
}
__global__ void __launch_bounds__(256, 4) finalize_ls_kernel(FinArgs a, SolverState* st, cudaGraphConditionalHandle h,
                                                          int in_graph, unsigned int* ticket) {
  finalize_ls_body(a, st, h, in_graph, ticket, blockIdx.x, gridDim.x);
}

cudaError_t launch_finalize_ls(const FinArgs& f, int grid, const FgLaunch& L, cudaStream_t stream) {
  finalize_ls_kernel<<<grid, 256, 0, stream>>>(f, L.ls_st, L.ls_h, L.ls_in_graph, L.ls_ticket);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// The scalar part of an iteration, run by one warp on the solver state in shared memory.
// `v` holds the reduced inner products in float64 and `vf` the same rounded to float32 (layout:
// see lbfgs_dots_kernel).  Float64 is kept for f, ||g||^2 and the line search; the Gram table
// and the two-loop scalars are float32 (see SolverState), and no float64 square root or
// division is taken.  Lane q works on history position q (newest first), so the table update
// and the two-loop recursion are a few dependent steps per position instead of loops.
//
// Part 1: the new pair enters the Gram table (or the memory is reset after a failed search),
// the history inner products are refreshed, the log record is written, and the stopping
// tests run.
constexpr float CURV_EPS_F = 1e-10f;
constexpr unsigned FULL_MASK = 0xffffffffu;
template <int NS>
__device__ void iteration_update_warp(SolverState* st, SolverState* logst, const double* v, const float* vf) {
  const int lane = threadIdx.x & 31;
  const int state = st->ls.state;
  const int count0 = st->count, sp = st->spare;
  const int myid = lane < count0 ? st->ids[lane] : -1;  // history position `lane`, before the update
  int added = -1;                                        // slot of the pair added by this step, if any
  __syncwarp();
  if (state == LS_ACCEPTED) {
    const float sy = vf[5 * NS + 2], yy = vf[5 * NS + 3], ss = vf[5 * NS + 4];
    if (sy > CURV_EPS_F * (sqrtf(ss) * sqrtf(yy)) && yy > 0.f) {  // curvature: s.y > eps |s| |y|
      if (lane < count0) {
        st->SY[sp][myid] = vf[5 * myid + 3];  // s_new . y_j
        st->SY[myid][sp] = vf[5 * myid + 2];  // s_j . y_new
        st->YY[sp][myid] = vf[5 * myid + 4];
        st->YY[myid][sp] = vf[5 * myid + 4];
      }
      if (lane == 0) {
        st->SY[sp][sp] = sy;
        st->YY[sp][sp] = yy;
      }
      const bool full = count0 == st->mem;
      const int keep = full ? count0 - 1 : count0;
      const int prev = __shfl_up_sync(FULL_MASK, myid, 1);
      const int newid = lane == 0 ? sp : prev;  // the ring shifts by one, the new pair in front
      const int count = keep + 1;
      int spare;
      if (full) {
        spare = __shfl_sync(FULL_MASK, myid, count0 - 1);  // the dropped oldest pair's slot
      } else {  // the lowest slot not in the ring (count <= mem < NS leaves one free)
        const unsigned lo = __reduce_or_sync(FULL_MASK, lane < count && newid < 32 ? 1u << newid : 0u);
        const unsigned hi = __reduce_or_sync(FULL_MASK, lane < count && newid >= 32 ? 1u << (newid - 32) : 0u);
        spare = lo != 0xffffffffu ? __ffs(~lo) - 1 : 32 + __ffs(~hi) - 1;
      }
      if (lane < count) st->ids[lane] = newid;
      if (lane == 0) {
        st->count = count;
        st->spare = spare;
      }
      added = sp;
    }
  }
  __syncwarp();
  if (lane == 0) {
    if (state == LS_ACCEPTED) {
      st->f = st->ls.f_acc;
      st->iter += 1;
      st->fails = 0;
    } else if (state == LS_FAILED) {
      st->count = 0;  // reset the memory; the next direction is steepest descent
      st->fails += 1;
      if (st->fails >= 2) {
        st->stop = STOP_LSFAIL;
        st->active = 0;
      }
    }
    st->acc_flag = state == LS_ACCEPTED;
    st->acc_slot = added;
  }
  __syncwarp();
  const int count = st->count;
  if (lane < count) {
    const int j = st->ids[lane];
    st->sg[j] = j == added ? vf[5 * NS + 0] : vf[5 * j + 0];
    st->yg[j] = j == added ? vf[5 * NS + 1] : vf[5 * j + 1];
  }
  if (lane == 0) {
    st->gg = v[5 * NS + 5];
    st->g1 = v[5 * NS + 6];
    if (state != LS_NONE) {
      double* rec = logst->log[logst->log_n % SOLVER_LOG];
      rec[0] = st->iter;
      rec[1] = st->f;
      rec[2] = sqrtf(vf[5 * NS + 5]);
      rec[3] = st->ls.a;
      rec[4] = st->ls.evals;
      rec[5] = state;
      rec[6] = count;
      logst->log_n += 1;
    }
    const double glim = st->gtol * fmax(1.0, fabs(st->f));
    if (!isfinite(st->f) || !isfinite(st->gg)) {
      st->stop = STOP_NONFINITE;
      st->active = 0;
    } else if (st->gtol > 0.0 && st->gg <= glim * glim) {  // ||g|| <= gtol max(1, |f|)
      st->stop = STOP_GTOL;
      st->active = 0;
    } else if (st->iter >= st->max_iter) {
      st->stop = STOP_MAXITER;
      st->active = 0;
    }
    if (st->f < st->best_f) st->best_f = st->f;
  }
  __syncwarp();
}

// The rest of the scalar part after the two-loop coefficients, run by one warp: the descent
// check g.d < 0 on the Gram table (a fixed-order warp sum, lane 0's value taken), falling
// back to steepest descent otherwise, and the first trial of the next line search.
// gg: ||g||^2 in float32.
__device__ void iteration_finish_warp(SolverState* st, float gg) {
  const int lane = threadIdx.x & 31;
  const int n = st->count;
  float t = 0.f;
  if (lane < n) {
    const int j = st->ids[lane];
    t = fmaf(st->coef_s[j], st->sg[j], st->coef_y[j] * st->yg[j]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  float gd = __shfl_sync(0xffffffffu, fmaf(st->coef_g, gg, t), 0);
  __syncwarp();
  if (!(gd < 0.f)) {  // not a descent direction: reset the memory, steepest descent
    for (int j = lane; j < SOLVER_MAX_SLOTS; j += 32) {
      st->coef_s[j] = 0.f;
      st->coef_y[j] = 0.f;
    }
    if (lane == 0) {
      st->count = 0;
      st->coef_g = -1.f;
    }
    gd = -gg;
  }
  __syncwarp();
  if (lane != 0) return;
  LineSearch& L = st->ls;
  // phi'(0) = g . d from the same inner products: d is a combination of g and the live
  // pairs, so g . d needs no pass over the vectors.
  L.g0 = gd;
  L.g_prev = gd;
  L.a = st->count == 0 ? (double)fminf(1.f, 1.f / (float)st->g1) : 1.0;
  L.f0 = st->f;
  L.a_prev = 0.0;
  L.f_prev = st->f;
  L.phase = 0;
  L.first = 1;
  L.evals = 0;
  L.width_prev = 0.0;
  L.best_a = 0.0;
  L.best_gg = INFINITY;
  L.force = 0;
  L.state = (gd < 0.f && isfinite(gd)) ? LS_RUNNING : LS_FAILED;  // not a descent direction
  st->gate = (st->active && L.state == LS_RUNNING) ? 1 : 0;
}

// Part 2: the two-loop recursion (Nocedal & Wright Alg. 7.4) on the Gram table.  Both loops
// are triangular solves: at step j the lane that owns pair j finishes its coefficient and
// broadcasts it, and every lane that still needs it adds its product.  Each lane first loads
// its row and column of the table (the entries it will use, in registers), so that a step is
// one broadcast and one FMA.
template <int NS>
__device__ void two_loop_coefs_warp(SolverState* st) {
  constexpr int MAXJ = NS - 1;  // history positions (count <= mem <= NS - 1)
  const int lane = threadIdx.x & 31;
  const int n = st->count;
  for (int j = lane; j < SOLVER_MAX_SLOTS; j += 32) {
    st->coef_s[j] = 0.f;
    st->coef_y[j] = 0.f;
  }
  __syncwarp();
  if (n == 0) {
    if (lane == 0) st->coef_g = -1.f;
    __syncwarp();
    return;
  }
  const bool mine = lane < n;
  const int id = mine ? st->ids[lane] : 0;
  float sy_row[MAXJ], sy_col[MAXJ], yy_row[MAXJ];
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    const int idj = j < n ? st->ids[j] : 0;
    sy_row[j] = mine && j < n ? st->SY[id][idj] : 0.f;  // s_id . y_j
    sy_col[j] = mine && j < n ? st->SY[idj][id] : 0.f;  // s_j . y_id
    yy_row[j] = mine && j < n ? st->YY[id][idj] : 0.f;
  }
  const float rho = mine ? 1.f / st->SY[id][id] : 0.f;
  const float sg = mine ? st->sg[id] : 0.f, yg = mine ? st->yg[id] : 0.f;
  const int i0 = st->ids[0];
  const float gamma = st->SY[i0][i0] / st->YY[i0][i0];
  // Loop 1 (newest -> oldest): a_i = rho_i (sg_i - sum_{j < i} a_j s_i . y_j).
  float acc = 0.f, a_mine = 0.f;
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    if (j < n) {
      if (lane == j) a_mine = (sg - acc) * rho;
      const float aj = __shfl_sync(FULL_MASK, a_mine, j);
      if (mine && lane > j) acc = fmaf(aj, sy_row[j], acc);
    }
  }
  // y_i . (sum_j a_j y_j), independent per lane.
  float ay = 0.f;
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    if (j < n) {
      const float aj = __shfl_sync(FULL_MASK, a_mine, j);
      if (mine) ay = fmaf(aj, yy_row[j], ay);
    }
  }
  // Loop 2 (oldest -> newest): c_i = a_i - rho_i (gamma (yg_i - ay_i) + sum_{j > i} c_j s_j . y_i).
  float acc2 = 0.f, c_mine = 0.f;
#pragma unroll
  for (int j = MAXJ - 1; j >= 0; --j) {
    if (j < n) {
      if (lane == j) c_mine = a_mine - fmaf(yg - ay, gamma, acc2) * rho;
      const float cj = __shfl_sync(FULL_MASK, c_mine, j);
      if (mine && lane < j) acc2 = fmaf(cj, sy_col[j], acc2);
    }
  }
  __syncwarp();
  if (mine) {
    st->coef_y[id] = gamma * a_mine;
    st->coef_s[id] = -c_mine;
  }
  if (lane == 0) st->coef_g = -gamma;
  __syncwarp();
}

// The scalar part of an iteration, run by the last block of the dots reduction: the solver
// state up to the log rings is copied to shared memory by the whole block, updated there by
// one warp (chains of dependent operations, which must not wait on global memory), and
// copied back.
constexpr int SOLVER_CORE_WORDS = (int)(offsetof(SolverState, log_n) / sizeof(double));
static_assert(offsetof(SolverState, log_n) % sizeof(double) == 0, "solver core must be whole words");
// fin: the reduced inner products in float64, finf: the same in float32 (shared memory).
template <int NS>
__device__ void scalar_tail(SolverState* gst, const double* fin, const float* finf) {
  __shared__ double core[SOLVER_CORE_WORDS];
  const double* src = reinterpret_cast<const double*>(gst);
  for (int i = threadIdx.x; i < SOLVER_CORE_WORDS; i += blockDim.x) core[i] = __ldcg(src + i);
  __syncthreads();
  SolverState* s = reinterpret_cast<SolverState*>(core);
  if (threadIdx.x < 32) {
    iteration_update_warp<NS>(s, gst, fin, finf);
    two_loop_coefs_warp<NS>(s);
    iteration_finish_warp(s, finf[5 * NS + 5]);
    if (threadIdx.x == 0) s->dir_pending = 1;
  }
  __syncthreads();
  double* dst = reinterpret_cast<double*>(gst);
  for (int i = threadIdx.x; i < SOLVER_CORE_WORDS; i += blockDim.x) dst[i] = core[i];
}

// Inner products.  Block row blockIdx.y = j < NS handles history slot j:
//   v[5 j + 0..4] = s_j.g, y_j.g, s_j.y_new, s_new.y_j, y_new.y_j
// and row NS the new pair and the gradient:
//   v[5 NS + 0..6] = s_new.g, y_new.g, s_new.y_new, y_new.y_new, s_new.s_new, g.g, |g|_1
// Products in float32, summed in float32 over each thread's elements, float64 beyond.
// The last block to finish runs the scalar part of the iteration.
template <int MCAP>
__global__ void __launch_bounds__(256) lbfgs_dots_kernel(SolverArgs a) {
  constexpr int NS = MCAP + 1;
  constexpr int NV = 5 * NS + 7;
  __shared__ float red[8][7];
  __shared__ double fin[NV];
  __shared__ float finf[NV];
  __shared__ bool is_last;
  SolverState* st = a.st;
  if (!st->active || st->ls.state == LS_RUNNING) return;  // nothing to do while a search runs
  const int j = blockIdx.y;
  const bool accepted = st->ls.state == LS_ACCEPTED;
  bool live = false;
  for (int q = 0; q < st->count; ++q) live |= st->ids[q] == j;
  const int64_t N = a.N;
  float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (j < NS ? live : true) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
      const float go = a.g[e];
      float gc = go, s = 0.f, y = 0.f;
      if (accepted) {  // the new pair, formed on the fly (stored by the direction kernel)
        const float xo = a.x[e], xn = a.xt[e], gn = a.gt[e];
        s = xn - xo;
        y = gn - go;
        gc = gn;
      }
      if (j < NS) {
        const float sj = a.S[(int64_t)j * N + e], yj = a.Y[(int64_t)j * N + e];
        acc[0] = fmaf(sj, gc, acc[0]);
        acc[1] = fmaf(yj, gc, acc[1]);
        acc[2] = fmaf(sj, y, acc[2]);
        acc[3] = fmaf(s, yj, acc[3]);
        acc[4] = fmaf(y, yj, acc[4]);
      } else {
        acc[0] = fmaf(s, gc, acc[0]);
        acc[1] = fmaf(y, gc, acc[1]);
        acc[2] = fmaf(s, y, acc[2]);
        acc[3] = fmaf(y, y, acc[3]);
        acc[4] = fmaf(s, s, acc[4]);
        acc[5] = fmaf(gc, gc, acc[5]);
        acc[6] += fabsf(gc);
      }
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nv = j < NS ? 5 : 7;
#pragma unroll
  for (int v = 0; v < 7; ++v) {
    float t = acc[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[w][v] = t;
  }
  __syncthreads();
  const int64_t bid = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x < nv) {
    ff2 t = ff_make(red[0][threadIdx.x]);
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) t = ff_add(t, ff_make(red[q][threadIdx.x]));
    ff_store(&a.blk[bid * 7 + threadIdx.x], t);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(a.counter, 1u) == gridDim.x * gridDim.y - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // Fixed-order reduction over the x-blocks (float-float): warp w owns values w, w + 8, ...
  for (int v = w; v < NV; v += (int)(blockDim.x >> 5)) {
    const int row = v < 5 * NS ? v / 5 : NS;
    const int col = v < 5 * NS ? v - 5 * (v / 5) : v - 5 * NS;
    ff2 t = ff_make(0.f);
    for (int b = lane; b < (int)gridDim.x; b += 32) t = ff_add(t, ff_load_cg(&a.blk[((int64_t)row * gridDim.x + b) * 7 + col]));
    t = warp_ff_sum(t);
    if (lane == 0) {
      fin[v] = ff_to_d(t);
      finf[v] = t.hi + t.lo;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *a.counter = 0u;
  scalar_tail<NS>(st, fin, finf);
}

// The end of a step and the next direction, elementwise.  When the line search accepted
// (acc_flag), s = x_t - x and y = g_t - g (the same float32 operations as in the inner
// products) go to history slot acc_slot and x, g move to the trial point; then, while the
// solver is active, d = coef_g g + sum over live pairs (coef_s s_j + coef_y y_j), the new pair
// taken from registers.  The line search's phi'(0) = g . d is formed from the Gram table by
// the scalar part of the iteration.  Two elements per thread (one for memory caps above 10)
// with every load in flight; the last block (ticket) clears acc_flag.
// Block bx of a grid of gx blocks.
template <int MCAP>
__device__ __forceinline__ void direction_body(const SolverArgs& a, const int bx, const int gx) {
  constexpr int NS = MCAP + 1;
  __shared__ float cs[NS], cy[NS];
  __shared__ float cg;
  SolverState* st = a.st;
  const int acc = st->acc_flag, active = st->active, pending = st->dir_pending;
  // In the iteration graph this is the last kernel of a trial: its first thread sets the
  // loop condition from the state the scalar part left (final by now).
  if (a.in_graph && bx == 0 && threadIdx.x == 0) {
    const int budget = st->loop_budget - 1;
    st->loop_budget = budget;
    cudaGraphSetConditional(a.loop_h, (active && st->iter < st->target && budget > 0) ? 1u : 0u);
  }
  if (!acc && !(active && pending)) return;
  const int slot = acc ? st->acc_slot : -1;
  uint64_t live = 0;
  if (active)
    for (int q = 0; q < st->count; ++q) live |= 1ull << st->ids[q];
  const uint64_t load = slot >= 0 ? live & ~(1ull << slot) : live;
  if (threadIdx.x < NS) {
    cs[threadIdx.x] = st->coef_s[threadIdx.x];
    cy[threadIdx.x] = st->coef_y[threadIdx.x];
  }
  if (threadIdx.x == 0) cg = st->coef_g;
  __syncthreads();
  // EPT consecutive elements per thread and step, each vector loaded and stored at once (the
  // vectors are padded to a multiple of 4 elements); two for memory caps up to 10.
  constexpr int EPT = NS <= 11 ? 2 : 1;
  const int64_t N = a.N;
  for (int64_t e = ((int64_t)bx * blockDim.x + threadIdx.x) * EPT; e < N;
       e += (int64_t)gx * blockDim.x * EPT) {
    float go[EPT], gn[EPT], xo[EPT], xn[EPT], sn[EPT], yn[EPT], sv[NS][EPT], yv[NS][EPT];
    vec_load<EPT>(go, a.g + e, true);
    vec_load<EPT>(xo, a.x + e, acc);
    vec_load<EPT>(xn, a.xt + e, acc);
    vec_load<EPT>(gn, a.gt + e, acc);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const bool use = (load >> j) & 1ull;
      vec_load<EPT>(sv[j], a.S + (int64_t)j * N + e, use);
      vec_load<EPT>(yv[j], a.Y + (int64_t)j * N + e, use);
    }
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      sn[u] = xn[u] - xo[u];  // zero unless accepted
      yn[u] = acc ? gn[u] - go[u] : 0.f;
      if (!acc) gn[u] = go[u];
    }
    if (acc) {
      if (slot >= 0) {
        vec_store<EPT>(a.S + (int64_t)slot * N + e, sn);
        vec_store<EPT>(a.Y + (int64_t)slot * N + e, yn);
      }
      vec_store<EPT>(a.x + e, xn);
      vec_store<EPT>(a.g + e, gn);
    }
    if (active && pending) {
      float dv[EPT];
#pragma unroll
      for (int u = 0; u < EPT; ++u) {
        dv[u] = cg * gn[u];
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          if ((live >> j) & 1ull) {
            dv[u] = fmaf(cs[j], j == slot ? sn[u] : sv[j][u], dv[u]);
            dv[u] = fmaf(cy[j], j == slot ? yn[u] : yv[j][u], dv[u]);
          }
        }
      }
      vec_store<EPT>(a.d + e, dv);
    }
  }
  // Every block has read the flags by the time the last one arrives.
  __syncthreads();
  if (threadIdx.x == 0 && atomicAdd(a.counter + 2 + DOTS_MAX_GRP, 1u) == (unsigned)gx - 1) {
    a.counter[2 + DOTS_MAX_GRP] = 0u;
    st->acc_flag = 0;
    st->dir_pending = 0;
  }
}

template <int MCAP>
__global__ void __launch_bounds__(256, MCAP <= 10 ? 2 : 1) lbfgs_direction_kernel(SolverArgs a) {
  direction_body<MCAP>(a, blockIdx.x, gridDim.x);
}

// The iteration target of the next graph launch: `count` iterations from the current one, in
// at most as many passes as count searches of LS_MAX_TRIALS trials (plus the restart after a
// failed search) can take.
__global__ void set_chunk_kernel(SolverState* st, int count) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->target = st->iter + count;
    st->loop_budget = (count + 2) * (LS_MAX_TRIALS + 2);
  }
}

__global__ void solver_init_kernel(SolverState* st, int mem, int max_iter, double gtol, double ls_noise) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->f = st->out[0];
  st->best_f = st->out[0];
  st->mem = mem;
  st->count = 0;
  st->spare = 0;
  st->iter = 0;
  st->evals = 1;
  st->fails = 0;
  st->stop = STOP_NONE;
  st->active = 1;
  st->gate = 1;
  st->max_iter = max_iter;
  st->gtol = gtol;
  st->ls_noise = ls_noise;
  st->ls.state = LS_NONE;
  st->acc_flag = 0;
  st->acc_slot = -1;
  st->dir_pending = 0;
  st->target = 0;
  st->loop_budget = 0;
  st->log_n = 0;
  st->tlog_n = 0;
}

// ---------------------------------------------------------------------------------------------
// Host side.

struct SolverBuffers {
  int mcap = 0;
  int64_t N = 0;
  float* x = nullptr;  // [U | V], the current point
  float* g = nullptr;
  float* xt = nullptr;
  float* gt = nullptr;
  float* d = nullptr;
  float* S = nullptr;
  float* Y = nullptr;
  SolverState* st = nullptr;
  SolverState* host = nullptr;  // pinned copy
  double* blk = nullptr;
  unsigned int* counter = nullptr;
  int grid = 0;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const FgPlan* plan = nullptr;  // objective/gradient plan the iteration was built for
};

static int mem_cap(int mem) { return mem <= 4 ? 4 : (mem <= 10 ? 10 : (mem <= 16 ? 16 : 32)); }

// Inner products in one pass over the elements (memory caps whose 5 (MCAP + 1) + 7 sums fit
// in 64), in the layout of lbfgs_dots_kernel.  The history slots are split between the two
// block rows (blockIdx.y; one row when there are few slots): row 0 takes the first half of
// the slots and the seven sums of the new pair and the gradient, row 1 the rest, so that a
// thread holds at most 5 ceil(NS / 2) + 7 sums beside its four elements' loads.  Each element of
// x, g, x_t, g_t is read by both rows, every live history pair once, and nothing is written
// (loads of successive elements can be in flight together); when the line search accepted,
// s = x_t - x and y = g_t - g are formed on the fly (the direction kernel stores them and moves
// x, g to the trial point).  A warp reduce-scatter leaves a few sums per lane, the warps are
// added in a fixed order, the last block of each group of DOTS_GRP columns of blocks adds the
// group and the last group adds the groups (float-float throughout, fixed order); that block
// runs the scalar part of the iteration.
template <int NS>
struct Dots1Shape {
  static constexpr int ROWS = NS > 6 ? 2 : 1;         // block rows
  static constexpr int H = (NS + ROWS - 1) / ROWS;    // slots per row (at most)
  static constexpr int C = ((5 * H + 7) + 7) & ~7;    // sums per thread, padded to a multiple of 8
};
// Block (bx, by) of a grid of gx x gy blocks.
template <int MCAP>
__device__ __forceinline__ void dots1_body(const SolverArgs& a, const int bx, const int by, const int gx, const int gy) {
  constexpr int NS = MCAP + 1;
  constexpr int NV = 5 * NS + 7;
  static_assert(NV <= 64, "too many sums for the one-pass kernel");
  using Sh = Dots1Shape<NS>;
  constexpr int C = Sh::C, H = Sh::H;
  constexpr int RC = rs_count(C);
  __shared__ float red[8][C];
  __shared__ double fin[64];
  __shared__ float finf[64];
  __shared__ bool is_last;
  SolverState* st = a.st;
  if (!st->active || st->ls.state == LS_RUNNING) return;  // nothing to do while a search runs
  const int row = by;
  const int j0 = row * H, nj = min(H, NS - j0);  // this row's slots [j0, j0 + nj)
  const bool own_new = row == 0;                 // row 0 also sums the new pair and g
  const bool accepted = st->ls.state == LS_ACCEPTED;
  unsigned int live = 0;
  for (int q = 0; q < st->count; ++q) live |= 1u << st->ids[q];
  live = (live >> j0) & ((1u << nj) - 1u);
  const int64_t N = a.N;
  const float* S0 = a.S + (int64_t)j0 * N;
  const float* Y0 = a.Y + (int64_t)j0 * N;
  float acc[C];
#pragma unroll
  for (int v = 0; v < C; ++v) acc[v] = 0.f;
  // DOTS_VEC consecutive elements per thread and step, loaded as one vector each (the vectors
  // are padded to a multiple of 4 elements): the pass reads from L2, where the number of
  // requests in flight, not the bytes, sets the rate.
  for (int64_t e = ((int64_t)bx * blockDim.x + threadIdx.x) * DOTS_VEC; e < N;
       e += (int64_t)gx * blockDim.x * DOTS_VEC) {
    float sv[H][DOTS_VEC], yv[H][DOTS_VEC];
#pragma unroll
    for (int jj = 0; jj < H; ++jj) {
      const bool use = (live >> jj) & 1u;
      vec_load<DOTS_VEC>(sv[jj], S0 + (int64_t)jj * N + e, use);
      vec_load<DOTS_VEC>(yv[jj], Y0 + (int64_t)jj * N + e, use);
    }
    float go[DOTS_VEC], xo[DOTS_VEC], xn[DOTS_VEC], gn[DOTS_VEC];
    vec_load<DOTS_VEC>(go, a.g + e, true);
    vec_load<DOTS_VEC>(xo, a.x + e, accepted);
    vec_load<DOTS_VEC>(xn, a.xt + e, accepted);
    vec_load<DOTS_VEC>(gn, a.gt + e, accepted);
#pragma unroll
    for (int u = 0; u < DOTS_VEC; ++u) {
      const float s = xn[u] - xo[u];  // zero unless accepted
      const float y = accepted ? gn[u] - go[u] : 0.f;
      const float gc = accepted ? gn[u] : go[u];
#pragma unroll
      for (int jj = 0; jj < H; ++jj) {
        if ((live >> jj) & 1u) {
          acc[5 * jj + 0] = fmaf(sv[jj][u], gc, acc[5 * jj + 0]);
          acc[5 * jj + 1] = fmaf(yv[jj][u], gc, acc[5 * jj + 1]);
          acc[5 * jj + 2] = fmaf(sv[jj][u], y, acc[5 * jj + 2]);
          acc[5 * jj + 3] = fmaf(s, yv[jj][u], acc[5 * jj + 3]);
          acc[5 * jj + 4] = fmaf(y, yv[jj][u], acc[5 * jj + 4]);
        }
      }
      if (own_new) {
        acc[5 * H + 0] = fmaf(s, gc, acc[5 * H + 0]);
        acc[5 * H + 1] = fmaf(y, gc, acc[5 * H + 1]);
        acc[5 * H + 2] = fmaf(s, y, acc[5 * H + 2]);
        acc[5 * H + 3] = fmaf(y, y, acc[5 * H + 3]);
        acc[5 * H + 4] = fmaf(s, s, acc[5 * H + 4]);
        acc[5 * H + 5] = fmaf(gc, gc, acc[5 * H + 5]);
        acc[5 * H + 6] += fabsf(gc);
      }
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int base = 0;
  ReduceScatter<C, 16>::run(acc, lane, base);
#pragma unroll
  for (int t = 0; t < RC; ++t) red[w][base + t] = acc[t];
  __syncthreads();
  // Local sum index u -> global layout v: slot sums 5 (j0 + jj) + c, the new pair's 5 NS + c.
  const int nloc = 5 * nj + (own_new ? 7 : 0);
  if (threadIdx.x < nloc) {
    const int u = threadIdx.x;
    const int ul = u < 5 * nj ? u : 5 * H + (u - 5 * nj);
    const int v = u < 5 * nj ? 5 * j0 + u : 5 * NS + (u - 5 * nj);
    ff2 t = ff_make(red[0][ul]);
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) t = ff_add(t, ff_make(red[q][ul]));
    ff_store(&a.blk[(int64_t)bx * 64 + v], t);
  }
  // Two-level ticket tree over the columns of blocks (both rows of a column write disjoint
  // sums into its 64 slots): the last of the group's blocks sums the group, the last group
  // sums the groups.
  const int nb = gx, grp = bx / DOTS_GRP, ngrp = (nb + DOTS_GRP - 1) / DOTS_GRP;
  const int gsize = min(DOTS_GRP, nb - grp * DOTS_GRP);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(a.counter + 1 + grp, 1u) == (unsigned)(gsize * gy) - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double* gblk = a.blk + (int64_t)nb * 64;
  if (threadIdx.x < NV) {
    ff2 p[DOTS_GRP];
#pragma unroll
    for (int u = 0; u < DOTS_GRP; ++u)
      p[u] = u < gsize ? ff_load_cg(&a.blk[(int64_t)(grp * DOTS_GRP + u) * 64 + threadIdx.x]) : ff_make(0.f);
    ff2 t = p[0];
#pragma unroll
    for (int u = 1; u < DOTS_GRP; ++u)
      if (u < gsize) t = ff_add(t, p[u]);
    ff_store(&gblk[grp * 64 + threadIdx.x], t);
  }
  if (threadIdx.x == 0) a.counter[1 + grp] = 0u;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(a.counter, 1u) == (unsigned)ngrp - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (threadIdx.x < NV) {
    ff2 t = ff_load_cg(&gblk[threadIdx.x]);
#pragma unroll 8
    for (int q = 1; q < ngrp; ++q) t = ff_add(t, ff_load_cg(&gblk[q * 64 + threadIdx.x]));
    fin[threadIdx.x] = ff_to_d(t);
    finf[threadIdx.x] = t.hi + t.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) *a.counter = 0u;
  scalar_tail<NS>(st, fin, finf);
}

template <int MCAP>
__global__ void __launch_bounds__(256, 2) lbfgs_dots1_kernel(SolverArgs a) {
  dots1_body<MCAP>(a, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

template <int MCAP>
static cudaError_t launch_update(const SolverArgs& a, int grid, cudaStream_t s) {
  if constexpr (5 * (MCAP + 1) + 7 <= 64) {
    // Two CTAs per SM (float4 loads: 126 registers): with two rows, half the solver grid per
    // row, so that both rows fit in one wave.
    constexpr int rows = Dots1Shape<MCAP + 1>::ROWS;
    const int gx = rows == 2 ? std::max(1, grid / 2) : grid;
    lbfgs_dots1_kernel<MCAP><<<dim3(gx, rows), 256, 0, s>>>(a);
  } else {
    const int gx = std::max(1, grid / (MCAP + 2));
    lbfgs_dots_kernel<MCAP><<<dim3(gx, MCAP + 2), 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}
template <int MCAP>
static cudaError_t launch_direction(const SolverArgs& a, int grid, cudaStream_t s) {
  // As many blocks as fit at once (the update grid: two per SM), striding over the elements.
  const int64_t g = std::min<int64_t>(std::min<int64_t>((a.N + 511) / 512, grid), (int64_t)DOTS_GRP * DOTS_MAX_GRP);
  lbfgs_direction_kernel<MCAP><<<(int)std::max<int64_t>(1, g), 256, 0, s>>>(a);
  return cudaGetLastError();
}

// Kernels launched by update_and_direction.
static int update_launches(int) { return 2; }

static cudaError_t update_and_direction(int mcap, const SolverArgs& a, int grid, cudaStream_t s) {
  cudaError_t e;
  switch (mcap) {
    case 4: if ((e = launch_update<4>(a, grid, s)) != cudaSuccess) return e; return launch_direction<4>(a, grid, s);
    case 10: if ((e = launch_update<10>(a, grid, s)) != cudaSuccess) return e; return launch_direction<10>(a, grid, s);
    case 16: if ((e = launch_update<16>(a, grid, s)) != cudaSuccess) return e; return launch_direction<16>(a, grid, s);
    default: if ((e = launch_update<32>(a, grid, s)) != cudaSuccess) return e; return launch_direction<32>(a, grid, s);
  }
}

void free_solver(rpca_ctx* c) {
  SolverBuffers* b = c->sol;
  if (!b) return;
  cudaStreamSynchronize(c->stream);  // no graph launch or kernel of this solver still queued
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
  dev_free(b->x);
  dev_free(b->S);
  dev_free(b->st);
  dev_free(b->blk);
  dev_free(b->counter);
  host_pinned_free(b->host);
  delete b;
  c->sol = nullptr;
}

#define SOL_CUDA(call)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(c, e_, #call); \
  } while (0)

static SolverArgs solver_args(rpca_ctx* c) {
  SolverBuffers* b = c->sol;
  SolverArgs a;
  a.st = b->st;
  a.N = b->N;
  a.x = b->x;
  a.g = b->g;
  a.xt = b->xt;
  a.gt = b->gt;
  a.d = b->d;
  a.S = b->S;
  a.Y = b->Y;
  a.blk = b->blk;
  a.counter = b->counter;
  a.loop_h = 0;
  a.in_graph = 0;
  return a;
}

// A line-search trial at x + a d (a read on the device).  For fused-kernel plans the
// line-search step is part of the finalize launch (in_graph: inside the iteration graph,
// whose while node h it drives); the GEMM plans of ranks above 16 launch it separately.
static FgLaunch trial_launch(rpca_ctx* c, cudaGraphConditionalHandle h = 0, int in_graph = 0) {
  SolverBuffers* b = c->sol;
  const int64_t mk = (int64_t)c->m * c->k;
  FgLaunch L;
  L.U = b->x;
  L.V = b->x + mk;
  L.dU = b->d;
  L.dV = b->d + mk;
  L.alpha_dev = &b->st->ls.a;
  L.gate = &b->st->gate;
  L.GU = b->gt;
  L.GV = b->gt + mk;
  L.Ut = b->xt;
  L.Vt = b->xt + mk;
  L.DU = b->d;
  L.DV = b->d + mk;
  L.out = b->st->out;
  if (!b->plan->large) {
    L.ls_st = b->st;
    L.ls_h = h;
    L.ls_in_graph = in_graph;
    L.ls_ticket = b->counter + 1 + DOTS_MAX_GRP;
  }
  return L;
}

// Records the iteration loop on `cap`, which must be capturing: a WHILE node over line-search
// trials, each trial the fused pass at x + a d, the assembly with the line-search step, the
// inner products with the scalar part (which return at once while the search runs) and the
// accepted step with the next direction (likewise); the direction kernel sets the loop
// condition: active and iter < target.  One launch runs the iterations up to the target that
// set_chunk_kernel recorded, with no return to the host and no graph launch per iteration.
static cudaError_t capture_iteration(rpca_ctx* c, cudaStream_t cap) {
  SolverBuffers* b = c->sol;
  SolverArgs a = solver_args(c);
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cap, &cst, nullptr, &g, &deps, nullptr, &ndeps);
  cudaGraphConditionalHandle h;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, g, deps, nullptr, ndeps, &cp);
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cap, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(b->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rpca_status s = launch_fg(c, *b->plan, trial_launch(c), b->cap2);
      e = s == RPCA_OK ? cudaGetLastError() : cudaErrorUnknown;
      a.loop_h = h;
      a.in_graph = 1;
      if (e == cudaSuccess) e = update_and_direction(b->mcap, a, b->grid, b->cap2);
      cudaGraph_t body_out = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(b->cap2, &body_out);
      if (e == cudaSuccess) e = e2;
    }
  }
  return e;
}

static rpca_status capture_solver_graph(rpca_ctx* c);

static rpca_status ensure_solver(rpca_ctx* c) {
  const int mcap = mem_cap(c->opt.lbfgs_mem);
  const FgPlan* plan = c->solve_plan ? c->solve_plan : &c->fg_plan;
  if (c->sol && c->sol->mcap == mcap && c->sol->plan == plan)
    return c->sol->exec || c->no_iter_graph ? RPCA_OK : capture_solver_graph(c);
  free_solver(c);
  SolverBuffers* b = new SolverBuffers();
  c->sol = b;
  b->mcap = mcap;
  b->plan = plan;
  // [U | V] is (m + n) k floats; the vectors are padded with zeros to a multiple of 4 so
  // that the elementwise kernels load aligned vectors.  The padding stays zero: nothing but
  // the elementwise kernels writes it, and they write combinations of zeros there.
  b->N = ((int64_t)(c->m + c->n) * c->k + 3) & ~(int64_t)3;
  const int64_t N = b->N;
  SOL_CUDA(dev_alloc(&b->x, sizeof(float) * 5 * N));
  SOL_CUDA(cudaMemsetAsync(b->x, 0, sizeof(float) * 5 * N, c->stream));
  b->g = b->x + N;
  b->xt = b->g + N;
  b->gt = b->xt + N;
  b->d = b->gt + N;
  SOL_CUDA(dev_alloc(&b->S, sizeof(float) * 2 * (mcap + 1) * N));
  b->Y = b->S + (int64_t)(mcap + 1) * N;
  SOL_CUDA(cudaMemsetAsync(b->S, 0, sizeof(float) * 2 * (mcap + 1) * N, c->stream));
  SOL_CUDA(dev_alloc(&b->st, sizeof(SolverState)));
  SOL_CUDA(cudaMemsetAsync(b->st, 0, sizeof(SolverState), c->stream));
  SOL_CUDA(host_pinned_alloc(&b->host, sizeof(SolverState)));
  // Two CTAs per SM, or the context's CTA budget when it shares the GPU with others (the
  // batched form): a grid that fills every SM leaves no room for the other contexts' kernels.
  int64_t grid_cap = std::min<int64_t>(2LL * c->nsm, (int64_t)DOTS_GRP * DOTS_MAX_GRP);
  if (c->grid_cap > 0) grid_cap = std::min<int64_t>(grid_cap, c->grid_cap);
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid_cap, (N + 255) / 256));
  SOL_CUDA(dev_alloc(&b->blk, sizeof(double) * std::max<size_t>(7 * ((size_t)b->grid + 64) * (mcap + 2),
                                                                  64 * ((size_t)b->grid + DOTS_MAX_GRP))));
  SOL_CUDA(dev_alloc(&b->counter, sizeof(unsigned int) * (1 + DOTS_MAX_GRP + 3)));
  SOL_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(unsigned int) * (1 + DOTS_MAX_GRP + 3), c->stream));
  SOL_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  SOL_CUDA(cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking));
  // The grouped iteration of the batched form launches this instance's trials itself.
  return c->no_iter_graph ? RPCA_OK : capture_solver_graph(c);
}

static rpca_status capture_solver_graph(rpca_ctx* c) {
  SolverBuffers* b = c->sol;
  // RPCA_SOLVER_GRAPH=0 runs the same kernels from a host loop (one synchronisation per
  // line-search trial), for per-kernel profilers that do not see inside conditional graphs.
  if (const char* e = getenv("RPCA_SOLVER_GRAPH"))
    if (e[0] == '0') return RPCA_OK;
  // Ranks above the fused kernel's call cuBLAS in their objective pass: host loop as well.
  if (c->lk) return RPCA_OK;

  // Capture the iteration loop: WHILE(active, iter < target) { fg, finalize + step, dots, direction }.
  SOL_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = capture_iteration(c, b->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(b->cap, &graph);
  if (e == cudaSuccess) e = e3;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_err(c, e, "capturing the L-BFGS iteration graph");
  }
  b->graph = graph;
  SOL_CUDA(cudaGraphInstantiate(&b->exec, graph, 0));
  return RPCA_OK;
}

// Appends this context's rounds of iterations (one iteration each, as the graph of
// ensure_solver) to the graph that `s` is capturing: the batched form's graph holds the
// iterations of every instance, each instance's on a branch of its own.
rpca_status solver_capture_rounds(rpca_ctx* c, cudaStream_t s, int rounds) {
  if (!c->sol || c->lk) return set_err(c, RPCA_EUNSUPPORTED, "no device iteration to capture");
  set_chunk_kernel<<<1, 1, 0, s>>>(c->sol->st, rounds);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = capture_iteration(c, s);
  if (e != cudaSuccess) return cuda_err(c, e, "capturing the batched iteration graph");
  return RPCA_OK;
}

SolverState* solver_state_dev(rpca_ctx* c) { return c->sol ? c->sol->st : nullptr; }

// Stops the device iteration of this context (its kernels in a captured graph then return at
// once): used by the batched form for instances that are finished.
rpca_status solver_deactivate(rpca_ctx* c, cudaStream_t s) {
  SolverBuffers* b = c->sol;
  if (!b) return RPCA_OK;
  SOL_CUDA(cudaMemsetAsync(&b->st->active, 0, sizeof(int), s));
  SOL_CUDA(cudaMemsetAsync(&b->st->gate, 0, sizeof(int), s));
  return RPCA_OK;
}

// Prepares the solver state at the point stored in sol->x: gradient, objective, first
// direction.  Stream-ordered on c->stream.
static rpca_status solver_start(rpca_ctx* c) {
  SolverBuffers* b = c->sol;
  const int64_t mk = (int64_t)c->m * c->k;
  FgLaunch L;
  L.U = b->x;
  L.V = b->x + mk;
  L.GU = b->g;
  L.GV = b->g + mk;
  L.out = b->st->out;
  rpca_status s = launch_fg(c, *b->plan, L, c->stream);
  if (s != RPCA_OK) return s;
  solver_init_kernel<<<1, 1, 0, c->stream>>>(b->st, c->opt.lbfgs_mem, c->opt.max_iter, c->opt.gtol,
                                              c->opt.ls_noise);
  SOL_CUDA(cudaGetLastError());
  SOL_CUDA(update_and_direction(b->mcap, solver_args(c), b->grid, c->stream));
  count_launches(c, 1 + update_launches(b->mcap));
  return RPCA_OK;
}

rpca_status solver_read_state(rpca_ctx* c, SolverState* out) {
  SolverBuffers* b = c->sol;
  SOL_CUDA(cudaMemcpyAsync(b->host, b->st, sizeof(SolverState), cudaMemcpyDeviceToHost, c->stream));
  SOL_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(out, b->host, sizeof(SolverState));
  return RPCA_OK;
}

// The scalars the host's loop reads between graph launches (everything but the Gram tables
// and the log rings): two small copies instead of the whole state.
rpca_status solver_read_scalars(rpca_ctx* c, SolverState* out) {
  SolverBuffers* b = c->sol;
  const size_t a0 = offsetof(SolverState, SY), a1 = offsetof(SolverState, sg), a2 = offsetof(SolverState, log);
  unsigned char* h = reinterpret_cast<unsigned char*>(b->host);
  const unsigned char* d = reinterpret_cast<const unsigned char*>(b->st);
  SOL_CUDA(cudaMemcpyAsync(h, d, a0, cudaMemcpyDeviceToHost, c->stream));
  SOL_CUDA(cudaMemcpyAsync(h + a1, d + a1, a2 - a1, cudaMemcpyDeviceToHost, c->stream));
  SOL_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(out, h, a0);
  memcpy(reinterpret_cast<unsigned char*>(out) + a1, h + a1, a2 - a1);
  return RPCA_OK;
}

rpca_status solver_prepare(rpca_ctx* c, const float* U, const float* V) {
  rpca_status s = ensure_solver(c);
  if (s != RPCA_OK) return s;
  const int64_t mk = (int64_t)c->m * c->k, nk = (int64_t)c->n * c->k;
  SOL_CUDA(cudaMemcpyAsync(c->sol->x, U, sizeof(float) * mk, cudaMemcpyDeviceToDevice, c->stream));
  SOL_CUDA(cudaMemcpyAsync(c->sol->x + mk, V, sizeof(float) * nk, cudaMemcpyDeviceToDevice, c->stream));
  return solver_start(c);
}

// The host-driven form of one graph launch: trials until the line search ends, then the
// update and the next direction.
static rpca_status host_iteration(rpca_ctx* c) {
  SolverBuffers* b = c->sol;
  for (int trial = 0; trial <= LS_MAX_TRIALS + 1; ++trial) {
    SOL_CUDA(cudaMemcpyAsync(&b->host->active, &b->st->active, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SOL_CUDA(cudaMemcpyAsync(&b->host->ls.state, &b->st->ls.state, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SOL_CUDA(cudaStreamSynchronize(c->stream));
    if (!b->host->active || b->host->ls.state != LS_RUNNING) break;
    rpca_status s = launch_fg(c, *b->plan, trial_launch(c), c->stream);
    if (s != RPCA_OK) return s;
    if (b->plan->large) {
      ls_step_kernel<<<1, 32, 0, c->stream>>>(b->st, 0, 0);
      SOL_CUDA(cudaGetLastError());
    }
  }
  SOL_CUDA(update_and_direction(b->mcap, solver_args(c), b->grid, c->stream));
  return RPCA_OK;
}

rpca_status solver_iterations(rpca_ctx* c, int count) {
  if (!c->sol->exec) {
    for (int i = 0; i < count; ++i) {
      rpca_status s = host_iteration(c);
      if (s != RPCA_OK) return s;
    }
    count_launches(c, (int64_t)update_launches(c->sol->mcap) * count);
  } else {
    set_chunk_kernel<<<1, 1, 0, c->stream>>>(c->sol->st, count);
    SOL_CUDA(cudaGetLastError());
    SOL_CUDA(cudaGraphLaunch(c->sol->exec, c->stream));
    c->graph_launches += 1;
    // The while body's four kernels per pass are added from the trial count when the solve
    // finishes.
    count_launches(c, 1);
  }
  return RPCA_OK;
}

const float* solver_point(rpca_ctx* c) { return c->sol ? c->sol->x : nullptr; }
// The gradient at solver_point and the objective there (device copy in the solver state).
const float* solver_gradient(rpca_ctx* c) { return c->sol ? c->sol->g : nullptr; }
const double* solver_f_device(rpca_ctx* c) { return c->sol ? &c->sol->st->f : nullptr; }

// ---------------------------------------------------------------------------------------------
// Grouped iteration.  Each instance's record holds what its own launches would pass: the
// fused pass's tensor maps and arguments (FgInst, first, so that fg_group_kernel finds it at
// the record's start), the solver's arguments, the assembly's arguments and ticket, and its
// grid sizes (those of its own launches, so that a grouped trial sums in the same order).
struct alignas(64) GroupRec {
  FgInst fg;
  SolverArgs a;
  FinArgs f;
  unsigned int* ticket;
  int fin_grid, dots_gx, dir_grid;
};

// Three CTAs per SM: with the arguments read from memory instead of the constant bank the
// line-search step needs more than 64 registers.
__global__ void __launch_bounds__(256, 3) finalize_ls_group_kernel(const GroupRec* __restrict__ rec,
                                                                const int* __restrict__ ids,
                                                                const int* __restrict__ off, int cnt) {
  __shared__ FinArgs sf;
  const int q = group_find(off, cnt, (int)blockIdx.x);
  const GroupRec* r = rec + __ldg(ids + q);
  args_to_shared(&sf, &r->f);
  __syncthreads();
  finalize_ls_body(sf, r->a.st, 0, 0, r->ticket, blockIdx.x - (unsigned)__ldg(off + q), (unsigned)r->fin_grid);
}

template <int MCAP>
__global__ void __launch_bounds__(256, 2) lbfgs_dots1_group_kernel(const GroupRec* __restrict__ rec,
                                                                 const int* __restrict__ ids,
                                                                 const int* __restrict__ off, int cnt) {
  constexpr int rows = Dots1Shape<MCAP + 1>::ROWS;
  __shared__ SolverArgs sa;
  const int q = group_find(off, cnt, (int)blockIdx.x);
  const GroupRec* r = rec + __ldg(ids + q);
  args_to_shared(&sa, &r->a);
  __syncthreads();
  const int local = (int)blockIdx.x - __ldg(off + q), gx = r->dots_gx;
  dots1_body<MCAP>(sa, local % gx, local / gx, gx, rows);
}

template <int MCAP>
__global__ void __launch_bounds__(256, MCAP <= 10 ? 2 : 1) lbfgs_direction_group_kernel(
    const GroupRec* __restrict__ rec, const int* __restrict__ ids, const int* __restrict__ off, int cnt) {
  const int q = group_find(off, cnt, (int)blockIdx.x);
  const GroupRec* r = rec + __ldg(ids + q);
  direction_body<MCAP>(r->a, (int)blockIdx.x - __ldg(off + q), r->dir_grid);
}

__global__ void gather_group_kernel(const GroupRec* __restrict__ rec, const int* __restrict__ ids, int cnt,
                                    double* out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
    const SolverState* st = rec[ids[q]].a.st;
    double* o = out + 6 * (size_t)q;
    o[0] = st->active;
    o[1] = st->iter;
    o[2] = st->gg;
    o[3] = st->f;
    o[4] = st->stop;
    o[5] = st->evals;
  }
}

size_t solver_group_stride() { return sizeof(GroupRec); }

bool solver_group_eligible(rpca_ctx* c) {
  const FgPlan& P = c->fg_plan;
  return c->lk == nullptr && c->xq_dt == 0 && c->bits == nullptr && P.valid && !P.large && !P.mma && !P.tc &&
         !P.masked && P.xt == FG_X_F32 && P.same && P.var != nullptr && P.var->group != nullptr &&
         mem_cap(c->opt.lbfgs_mem) <= 10 && P.smem + sizeof(FgArgs) + 256 <= c->max_smem;  // + its static shared
}

rpca_status solver_group_member(rpca_ctx* c, void* rec_host, GroupMember* m) {
  SolverBuffers* b = c->sol;
  if (!b || !solver_group_eligible(c) || b->plan != &c->fg_plan)
    return set_err(c, RPCA_EUNSUPPORTED, "this solve cannot join the grouped iteration");
  GroupRec* r = static_cast<GroupRec*>(rec_host);
  memset(static_cast<void*>(r), 0, sizeof *r);
  const FgPlan& P = *b->plan;
  const FgLaunch L = trial_launch(c);
  fg_launch_args(c, P, L, &r->fg.a, &r->f);
  r->fg.tmX = P.tmX;
  r->fg.tmM = P.tmM;
  r->a = solver_args(c);
  r->ticket = L.ls_ticket;
  r->fin_grid = P.fin_grid;
  // The grids of launch_update / launch_direction for this instance.
  const int rows = b->mcap == 4 ? Dots1Shape<5>::ROWS : Dots1Shape<11>::ROWS;
  r->dots_gx = rows == 2 ? std::max(1, b->grid / 2) : b->grid;
  r->dir_grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>((b->N + 511) / 512, b->grid), (int64_t)DOTS_GRP * DOTS_MAX_GRP));
  m->fg_fn = P.var->group;
  m->fg_threads = P.threads;
  m->fg_smem = P.smem;
  m->fg_blocks = P.nrb * P.ncs;
  m->fin_blocks = P.fin_grid;
  m->dots_blocks = r->dots_gx * rows;
  m->dir_blocks = r->dir_grid;
  m->mcap = b->mcap;
  return RPCA_OK;
}

cudaError_t solver_group_round(const GroupRound& R, cudaStream_t s, int64_t* launches) {
  const unsigned char* rec = static_cast<const unsigned char*>(R.rec);
  size_t stride = R.stride;
  for (int g = 0; g < R.nfg; ++g) {
    const GroupFgList& F = R.fg[g];
    if (F.cnt <= 0) continue;
    const int* ids = F.ids;
    const int* off = F.off;
    int cnt = F.cnt;
    void* args[] = {(void*)&rec, (void*)&stride, (void*)&ids, (void*)&off, (void*)&cnt};
    cudaError_t e = cudaLaunchKernel(F.fn, dim3(F.blocks), dim3(F.threads), args, F.smem, s);
    if (e != cudaSuccess) return e;
    ++*launches;
  }
  if (R.cnt <= 0) return cudaSuccess;
  const GroupRec* gr = reinterpret_cast<const GroupRec*>(rec);
  finalize_ls_group_kernel<<<R.fin_blocks, 256, 0, s>>>(gr, R.ids, R.fin_off, R.cnt);
  if (R.mcap == 4) {
    lbfgs_dots1_group_kernel<4><<<R.dots_blocks, 256, 0, s>>>(gr, R.ids, R.dots_off, R.cnt);
    lbfgs_direction_group_kernel<4><<<R.dir_blocks, 256, 0, s>>>(gr, R.ids, R.dir_off, R.cnt);
  } else {
    lbfgs_dots1_group_kernel<10><<<R.dots_blocks, 256, 0, s>>>(gr, R.ids, R.dots_off, R.cnt);
    lbfgs_direction_group_kernel<10><<<R.dir_blocks, 256, 0, s>>>(gr, R.ids, R.dir_off, R.cnt);
  }
  *launches += 3;
  return cudaGetLastError();
}

cudaError_t solver_group_gather(const void* rec, const int* ids, int cnt, double* out, cudaStream_t s) {
  if (cnt <= 0) return cudaSuccess;
  gather_group_kernel<<<(cnt + 127) / 128, 128, 0, s>>>(static_cast<const GroupRec*>(rec), ids, cnt, out);
  return cudaGetLastError();
}

}  // namespace rpca
