// The complex64 pass-group kernel (k_group) and its launcher, shared by
// owqs_group.cu (the slot-dispatching instantiations and the launch entry)
// and owqs_group_seq.cu (the instantiations compiled for the register-slot
// sequences of owqs_group_sequences.inc, split over kGroupSeqSlices
// translation units that compile in parallel).
#pragma once

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>

#include "owqs_device.cuh"

namespace owqs {

// VIRT: the group reads the virtual |+> input (G.in == nullptr); a separate
// instantiation keeps the array-reading kernel free of the test.  SEQ bits
// 24-27 nonzero: the group's register-slot sequence fixed at compile time
// (bits 24-27 the number of passes k, bits 2j and 2j+1 the slot pass j
// measures); zero: the kernel reads the slots from the parameter block and
// dispatches on them per pass.  Bit 31: every probability of the group is
// exactly 1/2 and only the last pass's norm is summed (the slot-dispatching
// kernel of such groups runs its passes in a rolled loop).
template <int M, bool VIRT, uint32_t SEQ = 0>
__global__ void __launch_bounds__(kBlock, M == 4 ? 1 : 2) k_group(const __grid_constant__ GroupParams G);

template <int M, bool VIRT, bool NORM>
__global__ void __launch_bounds__(kBlock, 2) k_group64(const GroupParams G);

// a tile of 2^(TB-M) free indices x 2^M configurations: TB = 9 for complex64
// (4 KB, one per warp; 10 and 8 KB with a 4-qubit register, one block per
// SM), 11 for complex128 (32 KB, one per block); the kernel
// pointer selects the precision and the instantiation (the shared-memory
// opt-in and the resident grid are looked up once per kernel)
template <int M, int TB>
static cudaError_t launch_group_t(void (*kern)(const GroupParams), const GroupParams& G, cudaStream_t s) {
  // complex64 (TB 9 or 10): one tile per warp; complex128 (TB 11): one per block
  constexpr bool kWarpTiles = TB < 11;
  // one block-wide 32 KB stage, or the eight warps' stages of 2^TB amplitudes
  constexpr int STAGE = kWarpTiles ? (kBlock / 32) * (1 << TB) * 8 : 32768;
  // stages, barriers, the sign table and the abort flag
  constexpr int SMEM = kTmaStages * STAGE + 1024;
  static std::map<const void*, int> caps;
  static std::mutex mu;
  int grid_cap = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = caps.find((const void*)kern);
    if (it != caps.end()) {
      grid_cap = it->second;
    } else {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, SMEM);
      if (e != cudaSuccess) return e;
      grid_cap = std::max(1, per_sm) * (max_grid() / 8);
      caps[(const void*)kern] = grid_cap;
    }
  }
  const uint64_t tiles = 1ull << (G.nfree - (TB - M));
  const uint64_t blocks = kWarpTiles ? (tiles + kBlock / 32 - 1) / (kBlock / 32) : tiles;
  kern<<<capped_grid((int)std::min<uint64_t>(blocks, (uint64_t)grid_cap)), kBlock, SMEM, s>>>(G);
  return cudaGetLastError();
}

// Register-slot sequences with a compile-time kernel (complex64, from an
// input array; on 2-qubit registers also from the virtual |+> input).  A
// pass's slot is the register position of the qubit it measures; the
// runtime-dispatched kernel chooses one of M code variants per pass, and the
// register values must then agree at the join of the variants, which costs
// moves on every pass.  A kernel whose slots are constants has one variant
// per pass.  The table holds the sequences that carry the most work
// (measurements x 2^width) in brickwork, QFT-shaped and random J/CZ patterns
// and the recognition set's wide unitaries (gen_group_sequences.py rebuilds
// it); any other sequence runs on the dispatching kernel.
// Code: bit 31 exact-half, bits 28-30 M, bits 24-27 k, bits 2j and 2j+1 the slot of pass j.
constexpr uint32_t kGroupSequences[] = {
#include "owqs_group_sequences.inc"
};
constexpr int kNumGroupSequences = (int)(sizeof(kGroupSequences) / sizeof(kGroupSequences[0]));

// the instantiations of sequence i live in slice i % kGroupSeqSlices
constexpr int kGroupSeqSlices = 8;
// launch G on the kernel of its sequence if this slice holds it (*launched)
template <int SLICE>
cudaError_t launch_group_seq_slice(const GroupParams& G, uint32_t code, cudaStream_t s, bool* launched);

// ---------------------------------------------------------------------------
// Group of up to kGroupMax measure passes in one HBM sweep (complex64): per
// free index the group is arithmetic on an M-qubit register (the contract,
// including how the signs and scales are carried, is in owqs_internal.h).
// Pipelines are warp-private: a warp's tile is 2^(9-M) consecutive free
// indices (2^6 with M = 4), whose 2^M input configurations arrive as nruns
// contiguous runs by bulk copies into the warp's own 3-stage ring of 4 KB
// stages (8 KB with M = 4).  The warp refills a stage as soon as its own
// lanes have read it, so no warp ever waits for another.
// Each lane takes two consecutive elements at a time and holds their 2^M
// amplitudes in registers.  Per pass and element: one sign bit XORed into w;
// per butterfly: one complex product and, per output, two FP32 multiply-adds
// for the amplitude and one packed FP32x2 multiply-add for its squared norm.
// The element's sign, the previous array's 1/sqrt(N) and the carried scales
// and register signs are applied once, at the 16-byte stores.
// Sign bits: bit j of an element's sign word is pass j's rho, bit 31 the
// parity of all the group's Z signs.  The tile's part is evaluated by lanes
// 0..k-1 (one pass each) and lane 31 (the Z parity) and OR-reduced across
// the warp; the element's low-bit parities are fixed per lane (a lane always
// takes the same offsets within a tile), so per tile one XOR gives every
// sign bit of an element.
// Norms (Eq. 13, R21): per pass, a lane adds its squared norms in FP32 over
// kNormTiles tiles (at most 2 x 8 x kNormTiles x 4 products); the warp then
// reduce-scatters its twelve per-pass sums (two halving shuffle steps), so
// that each lane adds three of them, summed over four lanes, into FP64
// accumulators; the block adds those in FP64 and the last block adds the
// blocks' totals (finish_slots).
// Every wait is bounded; a warp that gives up raises the block's abort flag,
// lets its issued copies land and returns.
// ---------------------------------------------------------------------------
constexpr int kNormTiles = 2;  // tiles per FP32 partial of a pass's squared norm
static_assert(kGroupMax == 12, "the norm reduce-scatter splits twelve pass sums 2 x 2 ways");

// Block stage of a complex64 group's slot sums.  dacc: this lane's FP64
// sums of passes 6 b4 + 3 b3 + {0, 1, 2} (b4, b3: lane bits 4 and 3) over
// the lanes {l, l^8, l^16, l^24}.  red: 12 x 64 doubles of shared memory.
// Pass j is added by warp j % 8: two values per lane, then a fixed FP64
// shuffle tree; the block's total, times the carried scales, goes to the
// partials.  Out of line, so that the main loop's code does not change with
// it.
static __device__ __noinline__ void group_slot_sums(const double (&dacc)[3], double* red, int k, double c2,
                                             const double* nscale, double* partials, unsigned int* counter,
                                             double* norms, int slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int p0 = 6 * ((lane >> 4) & 1) + 3 * ((lane >> 3) & 1);
  for (int i = 0; i < 3; ++i) red[(p0 + i) * 64 + warp * 8 + (lane & 7)] = dacc[i];
  __syncthreads();
  for (int j = warp; j < k; j += nwarp) {
    double s = red[j * 64 + lane] + red[j * 64 + 32 + lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      partials[(size_t)j * gridDim.x + blockIdx.x] = c2 * nscale[j] * s;
      __threadfence();
    }
  }
  finish_slots(partials, counter, norms, slot, k);
}

// Reduce-scatter of the twelve per-pass FP32 sums across the warp: after
// the xor-16 and xor-8 steps, lane l holds passes 6 b4 + 3 b3 + {0, 1, 2}
// summed over {l, l^8, l^16, l^24}; they are added into the lane's FP64
// accumulators and the FP32 sums restart at zero.
__device__ __forceinline__ void group_flush_norms(float (&s)[kGroupMax], double (&dacc)[3], int lane) {
  const bool h4 = (lane >> 4) & 1, h3 = (lane >> 3) & 1;
  float a[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float keep = h4 ? s[6 + i] : s[i], send = h4 ? s[i] : s[6 + i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float keep = h3 ? a[3 + i] : a[i], send = h3 ? a[i] : a[3 + i];
    dacc[i] += (double)(keep + __shfl_xor_sync(0xffffffffu, send, 8));
  }
#pragma unroll
  for (int j = 0; j < kGroupMax; ++j) s[j] = 0.f;
}

template <int M, int S, bool NORM>
__device__ __forceinline__ void group_butterfly(float2 (&x)[1 << M], const GroupPass& P, float wr, float wi,
                                                float2& nacc, bool first) {
#pragma unroll
  for (int h = 0; h < (1 << (M - 1)); ++h) {
    const int g0 = ((h >> S) << (S + 1)) | (h & ((1 << S) - 1));
    const int g1 = g0 | (1 << S);
    const float2 x0 = x[g0], x1 = x[g1];
    const float2 v = make_float2(fmaf(wr, x1.x, -wi * x1.y), fmaf(wr, x1.y, wi * x1.x));
    const float2 y0 = make_float2(fmaf(P.ct[g0], v.x, x0.x), fmaf(P.ct[g0], v.y, x0.y));
    const float2 y1 = make_float2(fmaf(P.ct[g1], v.x, x0.x), fmaf(P.ct[g1], v.y, x0.y));
    // the pass's first product starts its accumulator (no zeroing)
    if (NORM) {
      nacc = (first && h == 0) ? __fmul2_rn(y0, y0) : __ffma2_rn(y0, y0, nacc);
      nacc = __ffma2_rn(y1, y1, nacc);
    }
    x[g0] = y0;
    x[g1] = y1;
  }
}

// r0, r1: the two elements' sign bits for this pass, at bit 31 (one XOR
// gives +-w)
template <int M, int S, bool NORM>
__device__ __forceinline__ void group_pass2(float2 (&x)[2][1 << M], const GroupPass& P, uint32_t r0, uint32_t r1,
                                            float2& nacc) {
  const uint32_t ur = __float_as_uint(P.fwr), ui = __float_as_uint(P.fwi);
  group_butterfly<M, S, NORM>(x[0], P, __uint_as_float(ur ^ r0), __uint_as_float(ui ^ r0), nacc, true);
  group_butterfly<M, S, NORM>(x[1], P, __uint_as_float(ur ^ r1), __uint_as_float(ui ^ r1), nacc, false);
}

template <int M, bool VIRT, uint32_t SEQ>
__global__ void __launch_bounds__(kBlock, M == 4 ? 1 : 2) k_group(const __grid_constant__ GroupParams G) {
  if (G.stall_limit > 0) {
    stall_and_give_up(G.stall_limit, G.errflag);
    return;
  }
  constexpr int LT = group_tile_bits(OWQS_C64, M) - M, TE = 1 << LT, NC = 1 << M, NS = kTmaStages;
  constexpr int STAGE = NC * TE * 8;
  constexpr int EPT = TE / 32;  // elements per lane per tile (even)
  constexpr int NWARP = kBlock / 32;
  static_assert(EPT >= 2 && EPT <= 8, "tile shape");
  static_assert(kGroupMax <= 31, "one sign bit per pass below the Z-parity bit");
  static_assert(NS * STAGE * NWARP >= kGroupMax * 64 * 8, "the slot sums reuse the stage memory");
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wsm = smem + warp * NS * STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NWARP * NS * STAGE) + warp * NS;
  uint64_t* af = reinterpret_cast<uint64_t*>(smem + NWARP * NS * STAGE + NWARP * NS * 8);
  uint32_t* zbs = reinterpret_cast<uint32_t*>(af + kGroupMax);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(zbs + kGroupMax);
  const float2* __restrict__ in = reinterpret_cast<const float2*>(G.in);
  float2* __restrict__ out = reinterpret_cast<float2*>(G.out);
  double cprev = 1.0;
  if (G.norm_in >= 0) {
    const double nv = G.norms[G.norm_in];
    cprev = (nv >= G.thresh && nv > 0.0) ? 1.0 / sqrt(nv) : 0.0;
  }
  const float fprev = (float)cprev;
  // no input array: every input amplitude is vconst (the virtual |+> input);
  // the ring then carries no data and only paces the loop.  Sequence kernels
  // on at most 2 register qubits (VIRT = false) also see it at run time, for
  // the first group of a run from |+> inputs (on larger registers the run-
  // time test measured slower for the groups that read an array).
  const bool virt = VIRT || (M <= 2 && ((SEQ >> 24) & 15u) != 0 && G.in == nullptr);
  const float vc = (float)G.vconst;
  const uint64_t tiles = 1ull << (G.nfree - LT);
  const uint64_t gw = (uint64_t)blockIdx.x * NWARP + warp;
  const uint64_t step = (uint64_t)gridDim.x * NWARP;
  const uint64_t mine = gw < tiles ? (tiles - gw + step - 1) / step : 0;
  // bits 24-27 of SEQ nonzero: the pass count and the slots are compile-time
  constexpr bool STATIC = ((SEQ >> 24) & 15u) != 0;
  const int k = STATIC ? (int)((SEQ >> 24) & 15u) : G.k;
  // bit 31 of SEQ: every probability of the group is exactly 1/2
  // (GroupParams::half), so only the last pass's squared norm is summed: the
  // next launch divides by it, so that the rounding in the array's norm does
  // not build up from group to group
  constexpr bool NORM = !((SEQ >> 31) & 1u);
  uint32_t lowbits[EPT], spread[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const uint32_t e = (uint32_t)(lane * 2 + (q >> 1) * 64 + (q & 1));
    uint32_t sp = e;
    for (uint32_t lm = G.lowmask; lm; lm &= lm - 1) {
      const int b = __ffs(lm) - 1;
      sp = ((sp >> b) << (b + 1)) | (sp & ((1u << b) - 1u));
    }
    spread[q] = sp;
    uint32_t w = ((uint32_t)__popc(e & G.zall_lo) & 1u) << 31;
#pragma unroll
    for (int j = 0; j < kGroupMax; ++j) w |= ((uint32_t)__popc(e & G.pass[j].alo) & 1u) << j;
    lowbits[q] = w;
  }
  const bool pair_contig = (G.lowmask & 1u) == 0u;

  // Copies of a tile: its 2^M configurations arrive as nruns contiguous runs.
  // Sequence kernels of 11 or more passes on at most 3 register qubits are
  // bound by instruction issue: lane r < nruns computes the addresses of run
  // r and issues its copy, so that the warp computes every run's addresses
  // at once instead of lane 0 one run after another.  The others (closer to
  // the memory bound, where this measured slower) issue every run from
  // lane 0.
  constexpr bool WARP_ISSUE = M <= 3 && ((SEQ >> 24) & 15u) >= 11;
  int wsorted[M];  // WARP_ISSUE: the register's input bits, ascending
#pragma unroll
  for (int q = 0; q < M; ++q) wsorted[q] = G.B[q];
#pragma unroll
  for (int q = 0; q < M; ++q)
#pragma unroll
    for (int r = q + 1; r < M; ++r)
      if (wsorted[r] < wsorted[q]) {
        const int tmp = wsorted[q];
        wsorted[q] = wsorted[r];
        wsorted[r] = tmp;
      }
  uint64_t my_runoff = 0;  // WARP_ISSUE: this lane's run
#pragma unroll
  for (int r = 0; r < NC; ++r)
    if (lane == r) my_runoff = G.runoff[r];
  const bool my_run = lane < G.nruns;

  auto issue_warp = [&](uint64_t i) {  // WARP_ISSUE: the whole warp, converged
    const int st = (int)(i % NS);
    float2* buf = reinterpret_cast<float2*>(wsm + st * STAGE);
    uint64_t ib = (gw + i * step) << LT;
#pragma unroll
    for (int q = 0; q < M; ++q) ib = ins0(ib, wsorted[q]);
#ifdef OWQS_BOUNDS_CHECK
    const bool ok = !my_run || in_extent(ib + my_runoff, G.runlen, G.in_cap, G.errflag);
    if (!__all_sync(0xffffffffu, ok)) {  // a run outside the input: no copy, the run reports the error
      if (lane == 0) mbar_arrive(&full[st]);
      return;
    }
#endif
    // the stage's byte count is armed before any of its copies is issued
    if (lane == 0) mbar_expect_tx(&full[st], (unsigned)STAGE);
    __syncwarp();
    if (my_run) bulk_g2s(buf + lane * G.runlen, in + ib + my_runoff, G.runlen * (unsigned)sizeof(float2), &full[st]);
  };

  auto issue = [&](uint64_t i) {  // lane 0 of the warp
    const int st = (int)(i % NS);
    if (virt) {  // no input array: the stage only paces the loop
      mbar_arrive(&full[st]);
      return;
    }
    float2* buf = reinterpret_cast<float2*>(wsm + st * STAGE);
    const uint64_t L0 = (gw + i * step) << LT;
    uint64_t ib = L0;
    int sorted[M];
#pragma unroll
    for (int q = 0; q < M; ++q) sorted[q] = G.B[q];
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
      for (int r = q + 1; r < M; ++r)
        if (sorted[r] < sorted[q]) {
          const int tmp = sorted[q];
          sorted[q] = sorted[r];
          sorted[r] = tmp;
        }
#pragma unroll
    for (int q = 0; q < M; ++q) ib = ins0(ib, sorted[q]);
#ifdef OWQS_BOUNDS_CHECK
    bool ok = true;
    for (int r = 0; r < G.nruns && ok; ++r) ok = in_extent(ib + G.runoff[r], G.runlen, G.in_cap, G.errflag);
    if (!ok) {  // a run outside the input: no copy, the run reports the error
      mbar_arrive(&full[st]);
      return;
    }
#endif
    mbar_expect_tx(&full[st], (unsigned)STAGE);
    const unsigned rbytes = G.runlen * (unsigned)sizeof(float2);
    for (int r = 0; r < G.nruns; ++r) bulk_g2s(buf + r * G.runlen, in + ib + G.runoff[r], rbytes, &full[st]);
  };

  if (threadIdx.x < kGroupMax) {
    af[threadIdx.x] = G.pass[threadIdx.x].afree;
    zbs[threadIdx.x] = G.pass[threadIdx.x].zb & 1u;
  }
  if (lane == 0)
    for (int q = 0; q < NS; ++q) mbar_init(&full[q], 1);
  if (threadIdx.x == 0) *abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  if (WARP_ISSUE && !virt) {
    for (uint64_t q = 0; q < mine && q < (uint64_t)NS; ++q) issue_warp(q);
  } else if (lane == 0) {
    for (uint64_t q = 0; q < mine && q < (uint64_t)NS; ++q) issue(q);
  }

  float s[kGroupMax];
#pragma unroll
  for (int j = 0; j < kGroupMax; ++j) s[j] = 0.f;
  double dacc[3] = {0.0, 0.0, 0.0};
  float hs = 0.f;    // half groups: the last pass's squared norm over kNormTiles tiles
  double hd = 0.0;   // and its FP64 sum
  uint64_t issued = mine < (uint64_t)NS ? mine : (uint64_t)NS;
  for (uint64_t i = 0; i < mine; ++i) {
    const int st = (int)(i % NS);
    if (*abort_flag) break;
    if (!mbar_wait_bounded(&full[st], (unsigned)((i / NS) & 1u))) {
      *abort_flag = 1;
      break;
    }
    const float2* buf = reinterpret_cast<const float2*>(wsm + st * STAGE);
    const uint64_t L0 = (gw + i * step) << LT;
    // the tile's sign word: lane j < k evaluates pass j's rho, lane 31 the
    // parity of the group's Z signs
    uint32_t mybits = 0;
    if (lane < k) mybits = (zbs[lane] ^ par64(L0 & af[lane])) << lane;
    if (lane == 31) mybits = (G.c0all ^ par64(L0 & G.zall)) << 31;
    const uint32_t sw = __reduce_or_sync(0xffffffffu, mybits);
#pragma unroll
    for (int it = 0; it < EPT / 2; ++it) {
      const int e = lane * 2 + it * 64;
      float2 x[2][NC];
      if (virt) {
#pragma unroll
        for (int c = 0; c < NC; ++c) x[0][c] = x[1][c] = make_float2(vc, 0.f);
      } else if (pair_contig) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(buf + G.cbase[c] + spread[2 * it]);
          x[0][c] = make_float2(v.x, v.y);
          x[1][c] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          x[0][c] = buf[G.cbase[c] + spread[2 * it]];
          x[1][c] = buf[G.cbase[c] + spread[2 * it + 1]];
        }
      }
      const uint32_t b0 = sw ^ lowbits[2 * it], b1 = sw ^ lowbits[2 * it + 1];
      if constexpr (!STATIC && !NORM) {
        // run-time slots: one rolled loop over the passes, with eight code
        // variants (four slots, with and without the last pass's norm)
        // instead of twelve unrolled copies of them, which overflowed the
        // instruction cache; the pass constants are read from the
        // grid-constant parameter at the pass index
#pragma unroll 1
        for (int j = 0; j < k; ++j) {
          const GroupPass& P = G.pass[j];
          const uint32_t r0 = (b0 << (31 - j)) & 0x80000000u, r1 = (b1 << (31 - j)) & 0x80000000u;
          const int slot = P.slot;
          float2 acc = make_float2(0.f, 0.f);
          if (j == k - 1) {
            if (M == 1 || slot == 0) group_pass2<M, 0, true>(x, P, r0, r1, acc);
            else if (M == 2 || slot == 1) group_pass2<M, (M > 1 ? 1 : 0), true>(x, P, r0, r1, acc);
            else if (M == 3 || slot == 2) group_pass2<M, (M > 2 ? 2 : 0), true>(x, P, r0, r1, acc);
            else group_pass2<M, (M > 3 ? 3 : 0), true>(x, P, r0, r1, acc);
            hs += acc.x + acc.y;
          } else {
            if (M == 1 || slot == 0) group_pass2<M, 0, false>(x, P, r0, r1, acc);
            else if (M == 2 || slot == 1) group_pass2<M, (M > 1 ? 1 : 0), false>(x, P, r0, r1, acc);
            else if (M == 3 || slot == 2) group_pass2<M, (M > 2 ? 2 : 0), false>(x, P, r0, r1, acc);
            else group_pass2<M, (M > 3 ? 3 : 0), false>(x, P, r0, r1, acc);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < kGroupMax; ++j) {
          if (j >= k) break;
          const GroupPass& P = G.pass[j];
          const uint32_t r0 = (b0 << (31 - j)) & 0x80000000u, r1 = (b1 << (31 - j)) & 0x80000000u;
          // a compile-time slot leaves one code variant per pass
          const int slot = STATIC ? (int)((SEQ >> (2 * j)) & 3u) : P.slot;
          float2 acc = make_float2(0.f, 0.f);
          if (NORM || j == k - 1) {
            if (M == 1 || slot == 0) group_pass2<M, 0, true>(x, P, r0, r1, acc);
            else if (M == 2 || slot == 1) group_pass2<M, (M > 1 ? 1 : 0), true>(x, P, r0, r1, acc);
            else if (M == 3 || slot == 2) group_pass2<M, (M > 2 ? 2 : 0), true>(x, P, r0, r1, acc);
            else group_pass2<M, (M > 3 ? 3 : 0), true>(x, P, r0, r1, acc);
          } else {
            if (M == 1 || slot == 0) group_pass2<M, 0, false>(x, P, r0, r1, acc);
            else if (M == 2 || slot == 1) group_pass2<M, (M > 1 ? 1 : 0), false>(x, P, r0, r1, acc);
            else if (M == 3 || slot == 2) group_pass2<M, (M > 2 ? 2 : 0), false>(x, P, r0, r1, acc);
            else group_pass2<M, (M > 3 ? 3 : 0), false>(x, P, r0, r1, acc);
          }
          if (NORM) s[j] += acc.x + acc.y;
          else if (j == k - 1) hs += acc.x + acc.y;
        }
      }
      const float f0 = __uint_as_float(__float_as_uint(fprev) ^ (b0 & 0x80000000u));
      const float f1 = __uint_as_float(__float_as_uint(fprev) ^ (b1 & 0x80000000u));
#pragma unroll
      for (int g = 0; g < NC; ++g) {
        const float s0 = f0 * G.fin[g], s1 = f1 * G.fin[g];
        OWQS_IF_IN_EXTENT(L0 + G.outoff[g] + e, 2, G.out_cap, G.errflag)
        *reinterpret_cast<float4*>(out + L0 + G.outoff[g] + e) =
            make_float4(s0 * x[0][g].x, s0 * x[0][g].y, s1 * x[1][g].x, s1 * x[1][g].y);
      }
    }
    if ((i % kNormTiles) == kNormTiles - 1) {
      if (NORM) {
        group_flush_norms(s, dacc, lane);
      } else {
        hd += (double)hs;
        hs = 0.f;
      }
    }
    // every lane has read the stage: refill it with this warp's tile i + NS
    __syncwarp();
    if (WARP_ISSUE && !virt) {
      if (issued < mine) issue_warp(issued);
    } else if (lane == 0 && issued < mine) {
      issue(issued);
    }
    if (issued < mine) ++issued;
  }
  __syncthreads();
  if (*abort_flag) {
    if (lane == 0) {
      if (threadIdx.x == 0) atomicOr(G.errflag, 1u);
      // let every copy this warp issued land before the block's memory goes away
      for (uint64_t j = issued > (uint64_t)NS ? issued - NS : 0; j < issued; ++j)
        mbar_wait_bounded(&full[j % NS], (unsigned)((j / NS) & 1u));
    }
    __syncthreads();
    return;
  }
  if (!NORM) {
    if (G.norm_out >= 0) {
      // slot j < k - 1: the product of the group's first j + 1 probabilities,
      // 2^-(j+1); slot k - 1: the summed squared norm of the output
      if (blockIdx.x == 0 && threadIdx.x < k - 1)
        G.norms[G.norm_out + threadIdx.x] = ldexp(1.0, -(int)(threadIdx.x + 1));
      const double a1[1] = {cprev * cprev * G.nscale[k - 1] * (hd + (double)hs)};
      reduce_to_slots<1>(a1, G.partials, G.counter, G.norms, G.norm_out + k - 1, 1);
    }
    return;
  }
  if (G.norm_out >= 0) {
    // the sums of a last, unfinished set of kNormTiles tiles
    group_flush_norms(s, dacc, lane);
    // every copy has landed and been read: the stage memory now holds the
    // lanes' FP64 sums
    group_slot_sums(dacc, reinterpret_cast<double*>(smem), k, cprev * cprev, G.nscale, G.partials, G.counter,
                    G.norms, G.norm_out);
  }
}

}  // namespace owqs
