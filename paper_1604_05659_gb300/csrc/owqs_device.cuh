// Device helpers shared by the pass kernels (owqs_kernels.cu) and the
// pass-group kernels (owqs_group.cu): bit tricks, the bounds checks of the
// checked build, the deterministic two-stage slot reduction, and the
// mbarrier / bulk-copy primitives (inline PTX) of the shared-memory rings.
#pragma once

#include <cstdint>

#include "owqs_internal.h"

namespace owqs {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using V = float2; };
template <> struct Cplx<double> { using V = double2; };

__device__ __forceinline__ uint32_t par64(uint64_t v) { return (uint32_t)__popcll(v) & 1u; }

__device__ __forceinline__ uint64_t ins0(uint64_t j, int b) {
  return ((j >> b) << (b + 1)) | (j & ((1ull << b) - 1));
}

// Compensated (Kahan) FP32 running sum: per-thread sums of squared norms
// stay in FP32 across tiles and are promoted to FP64 once per kernel (FP64
// issues at a small fraction of the FP32 rate on GB300)
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
  const float y = x - comp;
  const float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// Bounds-checked builds (-DOWQS_BOUNDS_CHECK): a global access of the pass
// kernels is first checked against the extent of the buffer it touches (cap
// elements; 0: not checked); an access outside it is skipped and raises bit
// 1 of the run's error flag, which the host reports.  Release builds compile
// the checks away.
#ifdef OWQS_BOUNDS_CHECK
__device__ __forceinline__ bool in_extent(uint64_t first, uint64_t count, uint64_t cap, unsigned int* flag) {
  if (cap == 0 || (first <= cap && count <= cap - first)) return true;
  atomicOr(flag, 2u);
  return false;
}
#define OWQS_IF_IN_EXTENT(first, count, cap, flag) if (in_extent((first), (count), (cap), (flag)))
#else
__device__ __forceinline__ bool in_extent(uint64_t, uint64_t, uint64_t, unsigned int*) { return true; }
#define OWQS_IF_IN_EXTENT(first, count, cap, flag)
#endif

// ---------------------------------------------------------------------------
// Block reduction of NV FP64 values into norms[slot .. slot+NV).  Each block
// stores its partial; the last block to finish (counted with one atomic)
// adds the partials, one warp per value: lane-strided Neumaier sums in block
// order, then a fixed shuffle tree, so the result does not depend on block
// scheduling.  The counter is reset for the next launch.  No thread ever
// waits on another block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finish_slots(double* partials, unsigned int* counter, double* norms, int slot, int nv);
template <int NV>
__device__ __forceinline__ void reduce_to_slots(const double (&acc)[NV], double* partials,
                                                unsigned int* counter, double* norms, int slot, int nv = NV) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[i][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double v = lane < nwarp ? sh[i][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) partials[(size_t)i * gridDim.x + blockIdx.x] = v;
    }
  }
  finish_slots(partials, counter, norms, slot, nv);
}

// Second half of the slot reduction: every block's partials are stored (and
// fenced by the threads that wrote them); the last block to finish adds them
// into norms[slot ..).
__device__ __forceinline__ void finish_slots(double* partials, unsigned int* counter, double* norms, int slot, int nv) {
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // one warp per slot: lane-strided Neumaier sums over the block partials,
  // then a fixed shuffle tree (the order does not depend on scheduling)
  for (int i = warp; i < nv; i += nwarp) {
    double s = 0.0, c = 0.0;
    for (unsigned blk = lane; blk < gridDim.x; blk += 32) {
      const double x = __ldcg(&partials[(size_t)i * gridDim.x + blk]);
      const double t = s + x;
      c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    s += c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) norms[slot + i] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitLimitCycles) return false;
  return true;
}
// Test path of the bounded waits: thread 0 waits on a barrier that nothing
// arrives at, gives up after `limit` cycles and raises the error flag; every
// thread of the block then returns before any copy is issued.
__device__ __forceinline__ void stall_and_give_up(long long limit, unsigned int* errflag) {
  __shared__ uint64_t never;
  if (threadIdx.x == 0) {
    mbar_init(&never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bool done = mbar_try_wait(&never, 0u);
    const long long t0 = clock64();
    while (!done && clock64() - t0 <= limit) done = mbar_try_wait(&never, 0u);
    if (!done) atomicOr(errflag, 1u);
  }
  __syncthreads();
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace owqs
