// Device helpers: complex vector types, L2-coherent loads/stores, the bounded group
// barrier with deterministic FP64 reductions, and the small tridiagonal exponential.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kg_internal.h"
#include "kgrape.h"

namespace kg {

// ---------------------------------------------------------------- worker threads
// A block holds at most kWorkMax worker threads, which share the block's data; the headline
// kernel's blocks carry one more warp (the control warp) that serves the group sums of its
// Lanczos loop and meets the workers only at named barriers.  wsync is the workers' block
// barrier (named barrier 1 where a control warp exists, else the block barrier) and nwork their
// number; every device function below that synchronises or strides by the block uses them.
constexpr int kWorkMax = 512;
__device__ __forceinline__ int nwork() { return blockDim.x > (unsigned)kWorkMax ? kWorkMax : (int)blockDim.x; }
__device__ __forceinline__ void wsync() {
  if (blockDim.x > (unsigned)kWorkMax) asm volatile("barrier.sync 1, 512;" ::: "memory");
  else __syncthreads();
}
__device__ __forceinline__ bool wsync_or(bool pred) {
  if (blockDim.x > (unsigned)kWorkMax) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, 1, 512, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((unsigned)pred)
        : "memory");
    return r != 0u;
  }
  return __syncthreads_or(pred) != 0;
}
// Named barrier `id` of `n` threads: wait for it, or only mark this warp's arrival.
__device__ __forceinline__ void nbar_sync(int id, int n) {
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int n) {
  asm volatile("barrier.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// ---------------------------------------------------------------- vector traits
template <class V> struct VecTraits;
template <> struct VecTraits<float2> { using R = float; };
template <> struct VecTraits<double2> { using R = double; };

template <class V> __device__ __forceinline__ V vmake(typename VecTraits<V>::R a, typename VecTraits<V>::R b);
template <> __device__ __forceinline__ float2 vmake<float2>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ double2 vmake<double2>(double a, double b) { return make_double2(a, b); }

// Vectors that other CTAs write during a launch are read through L2 only (ld.global.cg):
// the per-SM L1 is not coherent across CTAs.
__device__ __forceinline__ float2 ldv(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldv(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ void stv(float2* p, float2 v) { __stcg(p, v); }
__device__ __forceinline__ void stv(double2* p, double2 v) { __stcg(p, v); }

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_relaxed_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------- bulk copies (TMA)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
// Global-memory data that other threads wrote with ordinary stores (and this thread acquired)
// before this thread's bulk copies read it.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// Arrive on the barrier and announce `bytes` of asynchronous transactions for this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from global to shared
// memory, completing as transactions on `bar`.
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                            unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst_smem)),
               "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Asynchronous 16-byte copies global -> shared through L2 only (cp.async.cg), grouped per
// thread: a thread waits for its own groups, so a thread that reads back only what it copied
// needs no barrier.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
// L2 eviction policies for data read or written once and not needed again soon (evict_first)
// and for data that should stay in L2 as long as possible (evict_last).
__device__ __forceinline__ unsigned long long l2_policy_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async16_hint(void* smem_dst, const void* gsrc, unsigned long long pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc),
               "l"(pol)
               : "memory");
}
__device__ __forceinline__ void stv_hint(float2* p, float2 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- tensor memory (TMEM)
// The complex64 resident path keeps thread-private arrays (the tile-leaving part X of H v_k
// and the own W_k) in tensor memory instead of shared memory: a warp may access the 32 TMEM
// lanes of its quarter of the warpgroup (lanes 32 (warp % 4) ...) and, with the 32x32b
// shape, thread t of the warp reads or writes row 32 (warp % 4) + t.  Allocation is done by
// one whole warp, which writes the TMEM address to shared memory; the same warp frees it.
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 8 complex64 values (16 columns) of this thread's TMEM row; load and wait in one statement,
// so the registers are never used before the data has arrived.
__device__ __forceinline__ void tmem_ld8c(uint32_t taddr, float2 (&v)[8]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
}
__device__ __forceinline__ void tmem_st8c(uint32_t taddr, const float2 (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
      "r"(__float_as_uint(v[0].x)), "r"(__float_as_uint(v[0].y)), "r"(__float_as_uint(v[1].x)),
      "r"(__float_as_uint(v[1].y)), "r"(__float_as_uint(v[2].x)), "r"(__float_as_uint(v[2].y)),
      "r"(__float_as_uint(v[3].x)), "r"(__float_as_uint(v[3].y)), "r"(__float_as_uint(v[4].x)),
      "r"(__float_as_uint(v[4].y)), "r"(__float_as_uint(v[5].x)), "r"(__float_as_uint(v[5].y)),
      "r"(__float_as_uint(v[6].x)), "r"(__float_as_uint(v[6].y)), "r"(__float_as_uint(v[7].x)),
      "r"(__float_as_uint(v[7].y))
      : "memory");
}

// 8 FP32 values (8 columns) of this thread's TMEM row, stored and loaded with a wait.
__device__ __forceinline__ void tmem_st8f(uint32_t taddr, const float (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}
__device__ __forceinline__ void tmem_ld8f(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Stores that leave their completion to a later tmem_st_wait (before the columns are read again or
// freed), and loads that wait.
__device__ __forceinline__ void tmem_st8c_nowait(uint32_t taddr, const float2 (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n" ::"r"(taddr),
      "r"(__float_as_uint(v[0].x)), "r"(__float_as_uint(v[0].y)), "r"(__float_as_uint(v[1].x)),
      "r"(__float_as_uint(v[1].y)), "r"(__float_as_uint(v[2].x)), "r"(__float_as_uint(v[2].y)),
      "r"(__float_as_uint(v[3].x)), "r"(__float_as_uint(v[3].y)), "r"(__float_as_uint(v[4].x)),
      "r"(__float_as_uint(v[4].y)), "r"(__float_as_uint(v[5].x)), "r"(__float_as_uint(v[5].y)),
      "r"(__float_as_uint(v[6].x)), "r"(__float_as_uint(v[6].y)), "r"(__float_as_uint(v[7].x)),
      "r"(__float_as_uint(v[7].y))
      : "memory");
}
// Four 4-column loads of this thread's TMEM row (2 complex64 values each) under one wait.
__device__ __forceinline__ void tmem_ld2c_x4(uint32_t ta, uint32_t tb, uint32_t tc, uint32_t td, float2 (&a)[2],
                                             float2 (&b)[2], float2 (&c)[2], float2 (&d)[2]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%16];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%17];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%18];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%19];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta), "r"(tb), "r"(tc), "r"(td)
      : "memory");
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    a[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
    b[i] = make_float2(__uint_as_float(r[4 + 2 * i]), __uint_as_float(r[4 + 2 * i + 1]));
    c[i] = make_float2(__uint_as_float(r[8 + 2 * i]), __uint_as_float(r[8 + 2 * i + 1]));
    d[i] = make_float2(__uint_as_float(r[12 + 2 * i]), __uint_as_float(r[12 + 2 * i + 1]));
  }
}
// Three 4-column stores (2 complex64 values each); completion is left to a later tmem_st_wait.
__device__ __forceinline__ void tmem_st2c_x3_nowait(uint32_t ta, uint32_t tb, uint32_t tc, const float2 (&a)[2],
                                                    const float2 (&b)[2], const float2 (&c)[2]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%3, %4, %5, %6};\n"
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%1], {%7, %8, %9, %10};\n"
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%2], {%11, %12, %13, %14};\n" ::"r"(ta),
      "r"(tb), "r"(tc), "r"(__float_as_uint(a[0].x)), "r"(__float_as_uint(a[0].y)), "r"(__float_as_uint(a[1].x)),
      "r"(__float_as_uint(a[1].y)), "r"(__float_as_uint(b[0].x)), "r"(__float_as_uint(b[0].y)),
      "r"(__float_as_uint(b[1].x)), "r"(__float_as_uint(b[1].y)), "r"(__float_as_uint(c[0].x)),
      "r"(__float_as_uint(c[0].y)), "r"(__float_as_uint(c[1].x)), "r"(__float_as_uint(c[1].y))
      : "memory");
}
// One 8-column store (4 complex64 values); completion is left to a later tmem_st_wait.
__device__ __forceinline__ void tmem_st4c_nowait(uint32_t ta, const float2 (&a)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(ta),
               "r"(__float_as_uint(a[0].x)), "r"(__float_as_uint(a[0].y)), "r"(__float_as_uint(a[1].x)),
               "r"(__float_as_uint(a[1].y)), "r"(__float_as_uint(a[2].x)), "r"(__float_as_uint(a[2].y)),
               "r"(__float_as_uint(a[3].x)), "r"(__float_as_uint(a[3].y))
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// ---------------------------------------------------------------- group context
// A group is the set of CTAs that cooperate on one problem.  All CTAs of a group are
// co-resident (cooperative launch), execute the same sequence of barriers/reductions,
// and therefore agree on every reduced scalar bit for bit.
struct Group {
  int rank, size;
  unsigned long long* bar;   // monotone arrival counter (reset to 0 before each launch)
  double* red;               // [2][stride][kNRed] partial slots, alternating by reduction
  int* ctrl;                 // status word, abort flag
  long long wait_limit_ns;
  int phase;                 // reduction counter (slot parity)
  int skip_arrival;          // fault injection: do not arrive at the next barrier (then cleared)
  unsigned long long epoch;  // barriers passed so far (identical in every CTA of the group)
  int stride;                // reduction slots per parity (>= size)
  unsigned long long* iring; // fixed-point sum ring of the group ([kIRing][4], zeroed at launch), or null
  unsigned iseq;             // fixed-point reductions so far (identical in every CTA of the group)
};

struct SmemRed {
  double warp_part[32 * kNRed];
  float warp_part_f[32 * kNRed];
  double out[kNRed];
  float2 cta_ff[kNRed];  // this CTA's float-float partials (single-CTA groups)
  int flag;
};

// ---------------------------------------------------------------- float-float sums
// Error-free transformation of a float sum (Knuth's TwoSum): hi + lo == a + b exactly.
// A float-float value carries ~48 significant bits, enough to add per-CTA partial sums
// of the complex64 path without FP64 instructions (slow on this GPU) and without losing
// accuracy to the number of CTAs.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = ff_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s.hi, e);
  return {hi, __fsub_rn(e, __fsub_rn(hi, s.hi))};
}
__device__ __forceinline__ FF ff_warp_sum(FF a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    a = ff_add(a, FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)});
  return a;
}

// Product of two float-float values (TwoProduct of the high parts with an FMA, plus the
// cross terms); about 44 significant bits, the accuracy of the operands.
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  const float t = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const float hi = __fadd_rn(p, t);
  return {hi, __fsub_rn(t, __fsub_rn(hi, p))};
}
__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// Barrier with a time limit.  Returns false (for every thread of the CTA) if the group
// aborted or this CTA's wait ran past the limit; in the latter case it records
// KG_ERR_TIMEOUT and raises the abort flag so every other CTA leaves at its next wait.
// Arrival is a release reduction on a monotone counter (no round trip); the k-th barrier
// of the launch completes when the counter reaches k * size.
__device__ __forceinline__ bool group_barrier(Group& g, SmemRed& sm) {
  wsync();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (g.size > 1) {
      // The arrival is a release reduction: it orders this CTA's earlier writes (those of other
      // threads through the bar.sync above) before the count; the acquire load below orders
      // the group's writes before everything this CTA reads after the barrier.
      if (g.skip_arrival) {  // injected fault: this CTA never joins; its own wait runs out too
        g.skip_arrival = 0;
      } else {
        red_release_add_u64(g.bar, 1ull);
      }
      g.epoch++;
      const unsigned long long goal = g.epoch * (unsigned long long)g.size;
      unsigned long long t0 = 0;
      unsigned polls = 0;
      while (ld_acquire_u64(g.bar) < goal) {
        if ((++polls & 31u) == 0u) {
          if (ld_volatile_i32(g.ctrl + kCtrlAbort)) { ok = 0; break; }
          const unsigned long long now = globaltimer_ns();
          if (t0 == 0) {
            t0 = now;
          } else if ((long long)(now - t0) > g.wait_limit_ns) {
            atomicCAS(g.ctrl + kCtrlStatus, 0, (int)KG_ERR_TIMEOUT);
            atomicExch(g.ctrl + kCtrlAbort, 1);
            ok = 0;
            break;
          }
          if (polls > 4096u) __nanosleep(64);
        }
      }
    } else if (ld_volatile_i32(g.ctrl + kCtrlAbort)) {
      ok = 0;
    }
    sm.flag = ok;
  }
  wsync();
  return sm.flag != 0;
}

// Sum NV per-thread values over the whole group.  Order of summation is fixed (warp
// butterfly, then warps in order, then CTA partials in rank order), so the result is
// deterministic and identical in every CTA.  Per-thread values may be float (complex64
// path: partial sums over a handful of amplitudes) or double; everything from the warp
// level up is float64.
template <int NV, class A>
__device__ __forceinline__ bool group_reduce(Group& g, SmemRed& sm, A (&vals)[NV], double (&out)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nwork() >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) vals[v] = warp_sum(vals[v]);
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sm.warp_part[warp * kNRed + v] = (double)vals[v];
  }
  wsync();
  double* slots = g.red + (size_t)(g.phase & 1) * g.stride * kNRed;
  g.phase++;
  if (warp < NV) {
    double s = (lane < nw) ? sm.warp_part[lane * kNRed + warp] : 0.0;
    s = warp_sum(s);
    if (lane == 0) {
      if (g.size > 1) __stcg(slots + (size_t)g.rank * kNRed + warp, s);
      else sm.out[warp] = s;
    }
  }
  if (g.size > 1) {
    if (!group_barrier(g, sm)) return false;
    if (warp < NV) {
      double s = 0.0;
      for (int r = lane; r < g.size; r += 32) s += __ldcg(slots + (size_t)r * kNRed + warp);
      s = warp_sum(s);
      if (lane == 0) sm.out[warp] = s;
    }
  } else if (ld_volatile_i32(g.ctrl + kCtrlAbort)) {
    return false;
  }
  wsync();
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = sm.out[v];
  return true;
}

// Same contract for float per-thread values (complex64 path): warp sums in float, the CTA
// partial and the sum over CTAs in float-float, one conversion to FP64 at the end.
template <int NV>
__device__ __forceinline__ bool group_reduce(Group& g, SmemRed& sm, float (&vals)[NV], double (&out)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nwork() >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) vals[v] = warp_sum(vals[v]);
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sm.warp_part_f[warp * kNRed + v] = vals[v];
  }
  wsync();
  float2* slots = reinterpret_cast<float2*>(g.red + (size_t)(g.phase & 1) * g.stride * kNRed);
  g.phase++;
  if (warp < NV) {
    FF s{(lane < nw) ? sm.warp_part_f[lane * kNRed + warp] : 0.f, 0.f};
    s = ff_warp_sum(s);
    if (lane == 0) {
      if (g.size > 1) __stcg(slots + (size_t)g.rank * kNRed + warp, make_float2(s.hi, s.lo));
      else sm.out[warp] = (double)s.hi + (double)s.lo;
    }
  }
  if (g.size > 1) {
    if (!group_barrier(g, sm)) return false;
    if (warp < NV) {
      FF s{0.f, 0.f};
      for (int r = lane; r < g.size; r += 32) {
        const float2 q = __ldcg(slots + (size_t)r * kNRed + warp);
        s = ff_add(s, FF{q.x, q.y});
      }
      s = ff_warp_sum(s);
      if (lane == 0) sm.out[warp] = (double)s.hi + (double)s.lo;
    }
  } else if (ld_volatile_i32(g.ctrl + kCtrlAbort)) {
    return false;
  }
  wsync();
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = sm.out[v];
  return true;
}

// The same float-float reduction split in two, so that the caller can act between the
// barrier and the sum (complex64 resident path): reduce_ff_arrive forms this CTA's partials
// and passes the group barrier (false: the group aborted); reduce_ff_collect, executed by
// warp 0 alone, sums the partials in rank order and leaves the totals in every lane.
template <int NV>
__device__ __forceinline__ bool reduce_ff_arrive(Group& g, SmemRed& sm, float (&vals)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nwork() >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) vals[v] = warp_sum(vals[v]);
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sm.warp_part_f[warp * kNRed + v] = vals[v];
  }
  wsync();
  float2* slots = reinterpret_cast<float2*>(g.red + (size_t)(g.phase & 1) * g.stride * kNRed);
  g.phase++;  // every thread: reduce_ff_collect reads the slots of parity (phase - 1)
  if (warp < NV) {
    FF s{(lane < nw) ? sm.warp_part_f[lane * kNRed + warp] : 0.f, 0.f};
    s = ff_warp_sum(s);
    if (lane == 0) {
      if (g.size > 1) __stcg(slots + (size_t)g.rank * kNRed + warp, make_float2(s.hi, s.lo));
      else sm.cta_ff[warp] = make_float2(s.hi, s.lo);
    }
  }
  if (g.size > 1) return group_barrier(g, sm);
  wsync();
  return ld_volatile_i32(g.ctrl + kCtrlAbort) == 0;
}
template <int NV>
__device__ __forceinline__ void reduce_ff_collect(Group& g, SmemRed& sm, FF (&out)[NV]) {
  const int lane = threadIdx.x & 31;
  const float2* slots = reinterpret_cast<const float2*>(g.red + (size_t)((g.phase - 1) & 1) * g.stride * kNRed);
  if (g.size == 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = FF{sm.cta_ff[v].x, sm.cta_ff[v].y};
    return;
  }
  FF s[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) s[v] = FF{0.f, 0.f};
  for (int r = lane; r < g.size; r += 32) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float2 q = __ldcg(slots + (size_t)r * kNRed + v);
      s[v] = ff_add(s[v], FF{q.x, q.y});
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = ff_warp_sum(s[v]);
}

// Variants for a Group that lives in shared memory, one copy for the whole CTA (the
// complex64 resident loop keeps it there rather than in every thread's stack frame): only
// thread 0 writes it.  The barrier advances the reduction parity as well.
__device__ __forceinline__ bool group_barrier_shared(Group& g, SmemRed& sm) {
  wsync();  // every thread has read g.phase
  if (threadIdx.x == 0) {
    int ok = 1;
    g.phase++;
    if (g.skip_arrival) {
      g.skip_arrival = 0;
    } else {
      red_release_add_u64(g.bar, 1ull);
    }
    g.epoch++;
    const unsigned long long goal = g.epoch * (unsigned long long)g.size;
    unsigned long long t0 = 0;
    unsigned polls = 0;
    while (ld_acquire_u64(g.bar) < goal) {
      if ((++polls & 31u) == 0u) {
        if (ld_volatile_i32(g.ctrl + kCtrlAbort)) { ok = 0; break; }
        const unsigned long long now = globaltimer_ns();
        if (t0 == 0) {
          t0 = now;
        } else if ((long long)(now - t0) > g.wait_limit_ns) {
          atomicCAS(g.ctrl + kCtrlStatus, 0, (int)KG_ERR_TIMEOUT);
          atomicExch(g.ctrl + kCtrlAbort, 1);
          ok = 0;
          break;
        }
        if (polls > 4096u) __nanosleep(64);
      }
    }
    sm.flag = ok;
  }
  wsync();
  return sm.flag != 0;
}
template <int NV>
__device__ __forceinline__ bool reduce_ff_arrive_shared(Group& g, SmemRed& sm, float (&vals)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nwork() >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) vals[v] = warp_sum(vals[v]);
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sm.warp_part_f[warp * kNRed + v] = vals[v];
  }
  wsync();
  const int size = g.size;
  if (warp < NV) {
    FF s{(lane < nw) ? sm.warp_part_f[lane * kNRed + warp] : 0.f, 0.f};
    s = ff_warp_sum(s);
    if (lane == 0) {
      if (size > 1) {
        float2* slots = reinterpret_cast<float2*>(g.red + (size_t)(g.phase & 1) * g.stride * kNRed);
        __stcg(slots + (size_t)g.rank * kNRed + warp, make_float2(s.hi, s.lo));
      } else {
        sm.cta_ff[warp] = make_float2(s.hi, s.lo);
      }
    }
  }
  if (size > 1) return group_barrier_shared(g, sm);
  wsync();
  return ld_volatile_i32(g.ctrl + kCtrlAbort) == 0;
}

// ---------------------------------------------------------------- fixed-point group sums
// Sums over the CTAs of a group by integer atomics.  Every CTA rounds its float-float partial to
// a 64-bit fixed-point number q = round(x 2^S) (S chosen per slice from a bound of the sums, the
// same in every CTA) and adds it into a ring slot in L2.  Integer addition is associative, so the
// total has the same bits whatever the order in which the CTAs arrive, and reading it back after
// the barrier is one load instead of a sum over every CTA's slot.  Reduction t uses slot
// t % kIRing (three sums and a count of partials out of range); rank 0 clears slot
// (t + 2) % kIRing as it arrives: every CTA read that slot before it arrived at the barrier that
// followed it, and nobody adds into it before the barrier after this one.

// q = round(x 2^S) for the float-float partial s (scale = 2^S, a power of two, so the products
// are exact); `bad` is set, and 0 returned, where |x| 2^S reaches 2^61 (or x is not finite).
__device__ __forceinline__ long long ff_to_fix(FF s, float scale, unsigned& bad) {
  const float a = s.hi * scale, b = s.lo * scale;
  if (!(fabsf(a) < 2.0e18f)) {
    bad = 1u;
    return 0;
  }
  return __float2ll_rn(a) + __float2ll_rn(b);
}
// The fixed-point total q 2^-S as a float-float (about 48 of its bits).
__device__ __forceinline__ FF fix_to_ff(long long q, float inv_scale) {
  const float h = __ll2float_rn(q);
  const float l = __ll2float_rn(q - __float2ll_rn(h));  // exact remainder, rounded once more
  return {h * inv_scale, l * inv_scale};
}

// The control warp's side of a fixed-point group sum (one warp serves the block; the workers have
// left their warp partials in sm.warp_part_f).  ctl_add_partials: the CTA partials in
// float-float over the first nw warps' entries, added as fixed-point numbers into the ring slot
// of reduction g.iseq (lane 0; single-CTA groups keep the float-float values in sm.cta_ff).
template <int NV>
__device__ __forceinline__ void ctl_add_partials(const Group& g, SmemRed& sm, int nw, float scale) {
  const int lane = threadIdx.x & 31;
  FF s[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) s[v] = FF{(lane < nw) ? sm.warp_part_f[lane * kNRed + v] : 0.f, 0.f};
#pragma unroll
  for (int v = 0; v < NV; ++v) s[v] = ff_warp_sum(s[v]);
  if (lane != 0) return;
  if (g.size == 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sm.cta_ff[v] = make_float2(s[v].hi, s[v].lo);
    return;
  }
  const unsigned slot = g.iseq % (unsigned)kIRing;
  unsigned long long* r = g.iring + 4u * slot;
  unsigned bad = 0u;
#pragma unroll
  for (int v = 0; v < NV; ++v) red_relaxed_add_u64(r + v, (unsigned long long)ff_to_fix(s[v], scale, bad));
  if (bad) red_relaxed_add_u64(r + 3, 1ull);
  if (g.rank == 0) {
    unsigned long long* z = g.iring + 4u * ((slot + 2u) % (unsigned)kIRing);
    __stcg(z, 0ull);
    __stcg(z + 1, 0ull);
    __stcg(z + 2, 0ull);
    __stcg(z + 3, 0ull);
  }
}
// Lane 0 of the control warp: the CTA's arrival at the group barrier that closes reduction
// g.iseq.  The release orders every store of the block before it (the workers handed over at a
// named barrier), so it waits for the block's stores to drain; no worker waits with it.
__device__ __forceinline__ void ctl_arrive(Group& g) {
  g.iseq++;
  if (g.size > 1) {
    if (g.skip_arrival) {  // injected fault: this CTA never joins; its own wait runs out too
      g.skip_arrival = 0;
    } else {
      red_release_add_u64(g.bar, 1ull);
    }
    g.epoch++;
  }
}
// Lane 0 of the control warp: wait for every arrival at the last barrier (bounded, as
// group_barrier); false if the group aborted or the wait ran out.
__device__ __forceinline__ bool ctl_wait(const Group& g) {
  if (g.size == 1) return ld_volatile_i32(g.ctrl + kCtrlAbort) == 0;
  const unsigned long long goal = g.epoch * (unsigned long long)g.size;
  unsigned long long t0 = 0;
  unsigned polls = 0;
  while (ld_acquire_u64(g.bar) < goal) {
    if ((++polls & 31u) == 0u) {
      if (ld_volatile_i32(g.ctrl + kCtrlAbort)) return false;
      const unsigned long long now = globaltimer_ns();
      if (t0 == 0) {
        t0 = now;
      } else if ((long long)(now - t0) > g.wait_limit_ns) {
        atomicCAS(g.ctrl + kCtrlStatus, 0, (int)KG_ERR_TIMEOUT);
        atomicExch(g.ctrl + kCtrlAbort, 1);
        return false;
      }
      if (polls > 4096u) __nanosleep(64);
    }
  }
  return true;
}

// Totals of the group's last fixed-point reduction (lane 0 of the control warp, after its
// barrier), in two parts: fix_load reads the slot's four words, fix_totals turns them into
// float-float values (false if a partial was out of range).  Single-CTA groups: the CTA's own
// partials.
struct FixRaw {
  unsigned long long w[4];
};
__device__ __forceinline__ FixRaw fix_load(const Group& g) {
  FixRaw r{{0ull, 0ull, 0ull, 0ull}};
  if (g.size > 1) {
    const unsigned long long* s = g.iring + 4u * ((g.iseq - 1u) % (unsigned)kIRing);
#pragma unroll
    for (int v = 0; v < 4; ++v) r.w[v] = __ldcg(s + v);  // weak: the barrier's acquire ordered it
  }
  return r;
}
template <int NV>
__device__ __forceinline__ bool fix_totals(const Group& g, const SmemRed& sm, const FixRaw& r, float inv_scale,
                                           FF (&out)[NV]) {
  if (g.size == 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = FF{sm.cta_ff[v].x, sm.cta_ff[v].y};
    return true;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = fix_to_ff((long long)r.w[v], inv_scale);
  return r.w[3] == 0ull;
}

// ---------------------------------------------------------------- small exponential
// 1/p! for p = 0..40 (exact rationals rounded once by the compiler).
__device__ __constant__ double kInvFact[41] = {
    1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320, 1.0 / 362880,
    1.0 / 3628800.0, 1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0, 1.0 / 87178291200.0,
    1.0 / 1307674368000.0, 1.0 / 20922789888000.0, 1.0 / 355687428096000.0, 1.0 / 6402373705728000.0,
    1.0 / 121645100408832000.0, 1.0 / 2432902008176640000.0, 1.0 / 51090942171709440000.0,
    1.0 / 1124000727777607680000.0, 1.0 / 25852016738884976640000.0, 1.0 / 620448401733239439360000.0,
    1.0 / 15511210043330985984000000.0, 1.0 / 403291461126605635584000000.0,
    1.0 / 10888869450418352160768000000.0, 1.0 / 304888344611713860501504000000.0,
    1.0 / 8841761993739701954543616000000.0, 1.0 / 265252859812191058636308480000000.0,
    1.0 / 8222838654177922817725562880000000.0, 1.0 / 263130836933693530167218012160000000.0,
    1.0 / 8683317618811886495518194401280000000.0, 1.0 / 295232799039604140847618609643520000000.0,
    1.0 / 10333147966386144929666651337523200000000.0, 1.0 / 371993326789901217467999448150835200000000.0,
    1.0 / 13763753091226345046315979581580902400000000.0, 1.0 / 523022617466601111760007224100074291200000000.0,
    1.0 / 20397882081197443358640281739902897356800000000.0,
    1.0 / 815915283247897734345611269596115894272000000000.0};

// c = exp(-i tau T) e_1 for the real symmetric tridiagonal T of order n <= 32
// (diag alpha[0..n-1], off-diagonal beta[1..n-1]; beta[k] couples k-1 and k),
// executed by one full warp; lane k holds c_k.  Method: split tau into s equal steps with
// ||(tau/s) T||_inf <= 4 (Gershgorin row sums) and, with A = (tau/s) T, sum the Taylor
// series exp(-i A) y = sum_p (-i)^p A^p y / p!  until the remainder bound r^(K+1)/(K+1)!
// drops below `tol` (r <= 4: at most 33 terms for tol = 1e-18).  A is real, so for real y
// every A^p y is real and (-i)^p only picks the real or the imaginary part and a sign; a
// complex y is two real series.  The first step starts from the real e_1, so a single step
// (||tau T|| <= 4, the common case) is one real series.  With ||A|| <= 4 the largest term is
// 4^4/4! < 11 times ||y||, so rounding stays below ~1e-14 ||y||.  FP64 throughout (about four
// FP64 operations per term and part).
__device__ __forceinline__ void tridiag_expv_e1(const double* alpha, const double* beta, const float* alpha_f,
                                                const float* beta_f, int n, double tau, float tau_f, double tol,
                                                double& c_re, double& c_im, float& tnorm) {
  const int lane = threadIdx.x & 31;
  const bool in = lane < n;
  const double a = in ? alpha[lane] : 0.0;
  const double bl = (in && lane >= 1) ? beta[lane] : 0.0;
  const double bh = (lane + 1 < n) ? beta[lane + 1] : 0.0;
  // Gershgorin bound of ||tau T||_inf and the step count in FP32 (a bound needs no more)
  float row = 0.f;
  if (in) row = fabsf(tau_f) * (fabsf(alpha_f[lane]) + (lane >= 1 ? beta_f[lane] : 0.f) +
                                (lane + 1 < n ? beta_f[lane + 1] : 0.f));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) row = fmaxf(row, __shfl_xor_sync(0xffffffffu, row, o));
  tnorm = row;
  int s = (int)ceilf(row * 1.0001f * 0.25f);
  if (s < 1) s = 1;
  const double h = (s == 1) ? tau : tau / (double)s;
  const double ha = h * a, hbl = h * bl, hbh = h * bh;  // rows of A = h T
  const float r = row * 1.0001f / (float)s;             // <= 4 bound of ||A||
  int K = 0;
  {
    float rem = r;  // r^(K+1) / (K+1)!, the first omitted term's bound
    while (K < 40 && rem >= (float)tol) { ++K; rem = rem * r / (float)(K + 1); }
  }
  double yr = (lane == 0) ? 1.0 : 0.0, yi = 0.0;
  for (int st = 0; st < s; ++st) {
    const bool cplx = (st > 0);
    double pr = yr, pi = yi;  // A^p y
    double ar = yr, ai = yi;  // accumulated result
    for (int k = 1; k <= K; ++k) {
      const double prm = __shfl_up_sync(0xffffffffu, pr, 1), prp = __shfl_down_sync(0xffffffffu, pr, 1);
      pr = fma(hbl, prm, fma(ha, pr, hbh * prp));
      if (cplx) {
        const double pim = __shfl_up_sync(0xffffffffu, pi, 1), pip = __shfl_down_sync(0xffffffffu, pi, 1);
        pi = fma(hbl, pim, fma(ha, pi, hbh * pip));
      }
      const double w = kInvFact[k];
      // (-i)^k: k%4 == 1 -> -i, 2 -> -1, 3 -> +i, 0 -> +1, applied to (pr + i pi)
      switch (k & 3) {
        case 0: ar = fma(w, pr, ar); if (cplx) ai = fma(w, pi, ai); break;
        case 1: if (cplx) ar = fma(w, pi, ar); ai = fma(-w, pr, ai); break;
        case 2: ar = fma(-w, pr, ar); if (cplx) ai = fma(-w, pi, ai); break;
        default: if (cplx) ar = fma(-w, pi, ar); ai = fma(w, pr, ai); break;
      }
    }
    yr = ar;
    yi = ai;
  }
  c_re = yr;
  c_im = yi;
}

// 1/p as float-float values (high part, remainder), p = 1..41, formed by the compiler (an FP32
// division is a ~85-cycle subroutine on this GPU; these products replace it).
#define KG_IFF(p) {(float)(1.0 / (p)), (float)(1.0 / (p) - (double)(float)(1.0 / (p)))}
__device__ __constant__ float2 kInvFF[42] = {
    {0.f, 0.f}, KG_IFF(1),  KG_IFF(2),  KG_IFF(3),  KG_IFF(4),  KG_IFF(5),  KG_IFF(6),  KG_IFF(7),  KG_IFF(8),
    KG_IFF(9),  KG_IFF(10), KG_IFF(11), KG_IFF(12), KG_IFF(13), KG_IFF(14), KG_IFF(15), KG_IFF(16), KG_IFF(17),
    KG_IFF(18), KG_IFF(19), KG_IFF(20), KG_IFF(21), KG_IFF(22), KG_IFF(23), KG_IFF(24), KG_IFF(25), KG_IFF(26),
    KG_IFF(27), KG_IFF(28), KG_IFF(29), KG_IFF(30), KG_IFF(31), KG_IFF(32), KG_IFF(33), KG_IFF(34), KG_IFF(35),
    KG_IFF(36), KG_IFF(37), KG_IFF(38), KG_IFF(39), KG_IFF(40), KG_IFF(41)};
#undef KG_IFF

__device__ __forceinline__ FF ff_from_double(double d) {
  const float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ FF ff_shfl_up(FF a) {
  return {__shfl_up_sync(0xffffffffu, a.hi, 1), __shfl_up_sync(0xffffffffu, a.lo, 1)};
}
__device__ __forceinline__ FF ff_shfl_down(FF a) {
  return {__shfl_down_sync(0xffffffffu, a.hi, 1), __shfl_down_sync(0xffffffffu, a.lo, 1)};
}

// The same exponential as tridiag_expv_e1 (same split into s steps, same term count K for `tol`,
// same series) in float-float arithmetic (about 44 significant bits) instead of FP64, for the
// complex64 path, whose coefficients are rounded to FP32 afterwards: FP32 instructions run far
// faster than FP64 ones on this GPU.  The FP64 tridiagonal is split into float-float once; the
// terms are formed as t_p = (A t_{p-1}) / p, which keeps them within the FP32 range.
__device__ __forceinline__ void tridiag_expv_e1_ff(const double* alpha, const double* beta, const float* alpha_f,
                                                   const float* beta_f, int n, double tau, float tau_f, double tol,
                                                   double& c_re, double& c_im, float& tnorm) {
  const int lane = threadIdx.x & 31;
  const bool in = lane < n;
  float row = 0.f;
  if (in) row = fabsf(tau_f) * (fabsf(alpha_f[lane]) + (lane >= 1 ? beta_f[lane] : 0.f) +
                                (lane + 1 < n ? beta_f[lane + 1] : 0.f));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) row = fmaxf(row, __shfl_xor_sync(0xffffffffu, row, o));
  tnorm = row;
  int s = (int)ceilf(row * 1.0001f * 0.25f);
  if (s < 1) s = 1;
  const double h = (s == 1) ? tau : tau / (double)s;
  const FF ha = ff_from_double(in ? h * alpha[lane] : 0.0);  // rows of A = h T
  const FF hbl = ff_from_double((in && lane >= 1) ? h * beta[lane] : 0.0);
  const FF hbh = ff_from_double((lane + 1 < n) ? h * beta[lane + 1] : 0.0);
  const float r = row * 1.0001f / (float)s;
  int K = 0;
  {
    const float tolf = (float)tol;
    float rem = r;
    while (K < 40 && rem >= tolf) { ++K; rem = rem * r * kInvFF[K + 1].x; }
  }
  FF yr{(lane == 0) ? 1.f : 0.f, 0.f}, yi{0.f, 0.f};
  for (int st = 0; st < s; ++st) {
    const bool cplx = (st > 0);
    FF pr = yr, pi = yi;  // t_p = A^p y / p!
    FF ar = yr, ai = yi;  // accumulated result
    for (int k = 1; k <= K; ++k) {
      const float2 wf = kInvFF[k];
      const FF w{wf.x, wf.y};
      {
        const FF m1 = ff_shfl_up(pr), p1 = ff_shfl_down(pr);
        pr = ff_mul(w, ff_add(ff_add(ff_mul(hbl, m1), ff_mul(ha, pr)), ff_mul(hbh, p1)));
      }
      if (cplx) {
        const FF m1 = ff_shfl_up(pi), p1 = ff_shfl_down(pi);
        pi = ff_mul(w, ff_add(ff_add(ff_mul(hbl, m1), ff_mul(ha, pi)), ff_mul(hbh, p1)));
      }
      const FF tr = pr;
      const FF ti = cplx ? pi : FF{0.f, 0.f};
      // (-i)^k: k%4 == 1 -> -i, 2 -> -1, 3 -> +i, 0 -> +1, applied to (pr + i pi)
      switch (k & 3) {
        case 0: ar = ff_add(ar, tr); if (cplx) ai = ff_add(ai, ti); break;
        case 1: if (cplx) ar = ff_add(ar, ti); ai = ff_add(ai, ff_neg(tr)); break;
        case 2: ar = ff_add(ar, ff_neg(tr)); if (cplx) ai = ff_add(ai, ff_neg(ti)); break;
        default: if (cplx) ar = ff_add(ar, ff_neg(ti)); ai = ff_add(ai, tr); break;
      }
    }
    yr = ar;
    yi = ai;
  }
  c_re = ff_to_double(yr);
  c_im = ff_to_double(yi);
}

}  // namespace kg
