// Shared device helpers: packed fp32 math, mbarrier / TMA inline PTX, bounded waits,
// deterministic block reductions.  sm_103a only.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define RPCA_DEV __device__ __forceinline__

namespace rpca {

// Error bits written to the device status word by kernels whose bounded waits give up.
enum : int { DEV_ERR_TIMEOUT_FULL = 1, DEV_ERR_TIMEOUT_EMPTY = 2, DEV_ERR_TIMEOUT_DRAIN = 4 };

// Wait limit for every spin on an mbarrier: 2 s of %globaltimer.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

RPCA_DEV uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

RPCA_DEV float2 f2(float a, float b) { return make_float2(a, b); }
RPCA_DEV float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
RPCA_DEV float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

RPCA_DEV uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ------------------------------------------------------------------------
RPCA_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
RPCA_DEV void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
RPCA_DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
               : "memory");
}
RPCA_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
RPCA_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on phase `parity`; returns false (and the caller must bail out) after the limit.
RPCA_DEV bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > limit_ns) return false;
  }
}

// ---- TMA (tiled tensor copies, no multicast) --------------------------------------------
RPCA_DEV void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// L2 policy that makes the lines it tags the first to be evicted: for streams read once per
// pass that are larger than L2 (X), so that the small vectors the next kernels read stay there.
RPCA_DEV uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// tma_load_2d with an L2 cache policy for the copied lines.
RPCA_DEV void tma_load_2d_hint(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
      "[%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
RPCA_DEV void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
// Grouped launches: entry q of a launch list owns the blocks [off[q], off[q + 1]) (off[0] = 0,
// ascending); the entry that owns block `bid` is the last q with off[q] <= bid.
RPCA_DEV int group_find(const int* __restrict__ off, int cnt, int bid) {
  int lo = 0, hi = cnt - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= bid) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Copies a kernel-argument struct from global to shared memory (8-byte words, one per thread;
// the caller synchronises the block before reading it): grouped launches read their
// instance's arguments there, as a plain launch reads its parameters, instead of holding
// them in registers.
template <class T>
RPCA_DEV void args_to_shared(T* dst, const T* __restrict__ src) {
  static_assert(sizeof(T) % 8 == 0 && sizeof(T) / 8 <= 96, "argument struct of whole words, at most 96");
  if (threadIdx.x < sizeof(T) / 8)
    reinterpret_cast<unsigned long long*>(dst)[threadIdx.x] =
        __ldg(reinterpret_cast<const unsigned long long*>(src) + threadIdx.x);
}

// A tensor map in global memory that the host wrote (a copy before the launch) is made
// visible to the tensor-map proxy before its first use by this thread.
RPCA_DEV void fence_tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
}

// Named barrier over `nthreads` threads (ids 1..15; 0 is __syncthreads).
RPCA_DEV void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---- float-float sums ----------------------------------------------------------------------
// An unevaluated sum hi + lo of two floats (about 44 significant bits), added with float32
// operations only.  The fixed-order sums of partials across warps and blocks use it: on GB300
// a float64 add takes 64 cycles and the float64 instructions of all warps on an SM quadrant
// share one narrow unit, so float64 reduction trees were the longest part of the short
// kernels of a solver iteration; a float-float add is ten float32 operations, four deep.
struct ff2 {
  float hi, lo;
};
RPCA_DEV ff2 ff_make(float x) { return {x, 0.f}; }
// Knuth's two-sum of the high parts, the low parts added to its error, renormalised with
// Dekker's fast two-sum.  (No products: nothing for the compiler to contract into an FMA.)
RPCA_DEV ff2 ff_add(ff2 a, ff2 b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  const float e = ((a.hi - (s - v)) + (b.hi - v)) + (a.lo + b.lo);
  const float hi = s + e;
  return {hi, e - (hi - s)};
}
RPCA_DEV double ff_to_d(ff2 a) { return (double)a.hi + (double)a.lo; }
RPCA_DEV ff2 ff_shfl_xor(ff2 a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
// Butterfly sum over the warp; every lane's association differs, so take one lane's result.
RPCA_DEV ff2 warp_ff_sum(ff2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
  return v;
}
// A float-float value kept in an 8-byte slot of a double buffer (block partials).
RPCA_DEV void ff_store(double* slot, ff2 v) { *reinterpret_cast<float2*>(slot) = make_float2(v.hi, v.lo); }
RPCA_DEV ff2 ff_load(const double* slot) {  // any state space (shared scratch)
  const float2 t = *reinterpret_cast<const float2*>(slot);
  return {t.x, t.y};
}
RPCA_DEV ff2 ff_load_cg(const double* slot) {  // global memory another block may have written
  const float2 t = __ldcg(reinterpret_cast<const float2*>(slot));
  return {t.x, t.y};
}
// A lane's Kahan pair (sum s, compensation c; the value is s - c) as a float-float value.
RPCA_DEV ff2 ff_from_kahan(float s, float c) { return ff_add(ff_make(s), ff_make(-c)); }

// ---- warp reduce-scatter of C floats over 32 lanes -----------------------------------
// After the call every lane holds rs_count(C) fully reduced values v[0..), standing for the
// original indices base + t.  Lanes that differ only in the bits of rs_dup_mask(C) hold the
// same values; exactly the lanes with (lane & rs_dup_mask(C)) == 0 should publish them.
__host__ __device__ constexpr int rs_count(int c, int o = 16) {
  return o == 0 ? c : (c % 2 == 0 ? rs_count(c / 2, o / 2) : rs_count(c, o / 2));
}
__host__ __device__ constexpr int rs_dup_mask(int c, int o = 16) {
  return o == 0 ? 0 : (c % 2 == 0 ? rs_dup_mask(c / 2, o / 2) : (o | rs_dup_mask(c, o / 2)));
}
template <int C, int O>
struct ReduceScatter {
  static RPCA_DEV void run(float* v, int lane, int& base) {
    if constexpr (O == 0) {
      return;
    } else if constexpr (C % 2 == 0) {
      constexpr int H = C / 2;
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int t = 0; t < H; ++t) {
        const float send = up ? v[t] : v[t + H];
        const float keep = up ? v[t + H] : v[t];
        v[t] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      if (up) base += H;
      ReduceScatter<H, O / 2>::run(v, lane, base);
    } else {
#pragma unroll
      for (int t = 0; t < C; ++t) v[t] += __shfl_xor_sync(0xffffffffu, v[t], O);
      ReduceScatter<C, O / 2>::run(v, lane, base);
    }
  }
};

RPCA_DEV double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of one double per thread (blockDim.x <= 1024); result valid in
// thread 0.  `scratch` holds >= 32 doubles.
RPCA_DEV double block_sum_d(double v, double* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += scratch[i];
  }
  return s;
}

}  // namespace rpca
