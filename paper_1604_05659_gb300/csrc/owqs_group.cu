// Pass groups (Sections 4.2 and 4.4 applied k times per HBM sweep): up to
// kGroupMax consecutive measure passes on an M-qubit register per free
// index, complex64 (k_group) and complex128 (k_group64).  The contract with
// the host planner (signs, scales, register layout) is in owqs_internal.h.
#include "owqs_group_c64.cuh"

namespace owqs {

static_assert(kGroupSeqSlices == 8, "launch_group dispatches eight slices");

uint32_t group_sequence_code(const GroupParams& G) {
  uint32_t c = ((uint32_t)(G.half ? 1 : 0) << 31) | ((uint32_t)G.m << 28) | ((uint32_t)G.k << 24);
  for (int j = 0; j < G.k; ++j) c |= ((uint32_t)G.pass[j].slot & 3u) << (2 * j);
  return c;
}

bool group_sequence_specialised(const GroupParams& G, int dtype, bool virt_in) {
  // from the virtual |+> input: the sequence kernels of registers of at most 2 qubits
  if (dtype != OWQS_C64 || (virt_in && G.m > 2)) return false;
  const uint32_t c = group_sequence_code(G);
  for (int i = 0; i < kNumGroupSequences; ++i)
    if (kGroupSequences[i] == c) return true;
  return false;
}

cudaError_t launch_group(const GroupParams& G, int dtype, cudaStream_t s) {
  const bool v = G.in == nullptr;
  if (dtype == OWQS_C64) {
    if (!v || G.m <= 2) {
      const uint32_t code = group_sequence_code(G);
      for (int i = 0; i < kNumGroupSequences; ++i) {
        if (kGroupSequences[i] != code) continue;
        bool launched = false;
        cudaError_t e = cudaErrorInvalidValue;
        switch (i % kGroupSeqSlices) {
          case 0: e = launch_group_seq_slice<0>(G, code, s, &launched); break;
          case 1: e = launch_group_seq_slice<1>(G, code, s, &launched); break;
          case 2: e = launch_group_seq_slice<2>(G, code, s, &launched); break;
          case 3: e = launch_group_seq_slice<3>(G, code, s, &launched); break;
          case 4: e = launch_group_seq_slice<4>(G, code, s, &launched); break;
          case 5: e = launch_group_seq_slice<5>(G, code, s, &launched); break;
          case 6: e = launch_group_seq_slice<6>(G, code, s, &launched); break;
          case 7: e = launch_group_seq_slice<7>(G, code, s, &launched); break;
          default: break;
        }
        if (launched) return e;
        break;
      }
    }
    // slots read at run time; exact-half groups sum only the last pass's norm
    constexpr uint32_t H = 1u << 31;
    if (G.half) {
      switch (G.m) {
        case 1: return v ? launch_group_t<1, 9>(k_group<1, true, H>, G, s)
                         : launch_group_t<1, 9>(k_group<1, false, H>, G, s);
        case 2: return v ? launch_group_t<2, 9>(k_group<2, true, H>, G, s)
                         : launch_group_t<2, 9>(k_group<2, false, H>, G, s);
        case 3: return v ? launch_group_t<3, 9>(k_group<3, true, H>, G, s)
                         : launch_group_t<3, 9>(k_group<3, false, H>, G, s);
        case 4: return v ? launch_group_t<4, 10>(k_group<4, true, H>, G, s)
                         : launch_group_t<4, 10>(k_group<4, false, H>, G, s);
        default: return cudaErrorInvalidValue;
      }
    }
    switch (G.m) {
      case 1: return v ? launch_group_t<1, 9>(k_group<1, true>, G, s) : launch_group_t<1, 9>(k_group<1, false>, G, s);
      case 2: return v ? launch_group_t<2, 9>(k_group<2, true>, G, s) : launch_group_t<2, 9>(k_group<2, false>, G, s);
      case 3: return v ? launch_group_t<3, 9>(k_group<3, true>, G, s) : launch_group_t<3, 9>(k_group<3, false>, G, s);
      case 4: return v ? launch_group_t<4, 10>(k_group<4, true>, G, s) : launch_group_t<4, 10>(k_group<4, false>, G, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (G.df) return launch_group_df(G, G.df_in != 0, G.df_out != 0, s);
  // the last pass's squared norm only where every probability is exactly 1/2
  // or none is needed (EOWQS)
  if (G.half || G.norm_out < 0) {
    switch (G.m) {
      case 1: return v ? launch_group_t<1, 11>(k_group64<1, true, false>, G, s)
                       : launch_group_t<1, 11>(k_group64<1, false, false>, G, s);
      case 2: return v ? launch_group_t<2, 11>(k_group64<2, true, false>, G, s)
                       : launch_group_t<2, 11>(k_group64<2, false, false>, G, s);
      case 3: return v ? launch_group_t<3, 11>(k_group64<3, true, false>, G, s)
                       : launch_group_t<3, 11>(k_group64<3, false, false>, G, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (G.m) {
    case 1: return v ? launch_group_t<1, 11>(k_group64<1, true, true>, G, s)
                     : launch_group_t<1, 11>(k_group64<1, false, true>, G, s);
    case 2: return v ? launch_group_t<2, 11>(k_group64<2, true, true>, G, s)
                     : launch_group_t<2, 11>(k_group64<2, false, true>, G, s);
    case 3: return v ? launch_group_t<3, 11>(k_group64<3, true, true>, G, s)
                     : launch_group_t<3, 11>(k_group64<3, false, true>, G, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Pass group in complex128: the same contract as k_group (the signs, scales
// and register layout of owqs_internal.h), 2^(11-M) free indices per 32 KB
// tile, one element per thread at a time (a complex128 amplitude is a
// 16-byte vector), FP64 throughout.  Per butterfly: one complex product and,
// per output, two FMAs for the amplitude and two for its squared norm: six
// FP64 instructions per output and measurement, against eight for a single
// measure pass (k_fast<double>), which is bound by the FP64 pipe on GB300.
// ---------------------------------------------------------------------------
template <int M, int S, bool NORM>
__device__ __forceinline__ void group_butterfly64(double2 (&x)[1 << M], const GroupPass& P, double wr, double wi,
                                                  double& nacc) {
#pragma unroll
  for (int h = 0; h < (1 << (M - 1)); ++h) {
    const int g0 = ((h >> S) << (S + 1)) | (h & ((1 << S) - 1));
    const int g1 = g0 | (1 << S);
    const double2 x0 = x[g0], x1 = x[g1];
    const double vx = fma(wr, x1.x, -wi * x1.y), vy = fma(wr, x1.y, wi * x1.x);
    const double2 y0 = make_double2(fma(P.ctd[g0], vx, x0.x), fma(P.ctd[g0], vy, x0.y));
    const double2 y1 = make_double2(fma(P.ctd[g1], vx, x0.x), fma(P.ctd[g1], vy, x0.y));
    if (NORM) {
      nacc = fma(y0.x, y0.x, fma(y0.y, y0.y, nacc));
      nacc = fma(y1.x, y1.x, fma(y1.y, y1.y, nacc));
    }
    x[g0] = y0;
    x[g1] = y1;
  }
}

// NORM = false: every probability of the group is exactly 1/2
// (GroupParams::half) or the run needs none: only the last pass's squared
// norm is summed (the next launch divides by it); the other slots get the
// exact products 2^-(j+1)
template <int M, bool VIRT, bool NORM>
__global__ void __launch_bounds__(kBlock, 2) k_group64(const GroupParams G) {
  if (G.stall_limit > 0) {
    stall_and_give_up(G.stall_limit, G.errflag);
    return;
  }
  constexpr int LT = 11 - M, TE = 1 << LT, NC = 1 << M, NS = kTmaStages;
  constexpr int STAGE = NC * TE * 16;
  constexpr int EPT = TE / kBlock;  // elements per thread per tile
  constexpr int NWARP = kBlock / 32;
  static_assert(EPT >= 1 && EPT <= 4, "tile shape");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * STAGE);
  uint64_t* empty = full + NS;
  uint32_t* signs = reinterpret_cast<uint32_t*>(smem + NS * STAGE + 2 * NS * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(signs + NS);
  const double2* __restrict__ in = reinterpret_cast<const double2*>(G.in);
  double2* __restrict__ out = reinterpret_cast<double2*>(G.out);
  double cprev = 1.0;
  if (G.norm_in >= 0) {
    const double nv = G.norms[G.norm_in];
    cprev = (nv >= G.thresh && nv > 0.0) ? 1.0 / sqrt(nv) : 0.0;
  }
  constexpr bool virt = VIRT;  // virtual |+> input, as in k_group
  const uint64_t tiles = 1ull << (G.nfree - LT);
  const uint64_t step = gridDim.x;
  const uint64_t mine = blockIdx.x < tiles ? (tiles - blockIdx.x + step - 1) / step : 0;
  constexpr unsigned RUN = TE * sizeof(double2);
  const int k = G.k;
  uint32_t lowbits[EPT], spread[EPT];  // element q at offset threadIdx + q kBlock
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const uint32_t e = (uint32_t)(threadIdx.x + q * kBlock);
    uint32_t sp = e;
    for (uint32_t lm = G.lowmask; lm; lm &= lm - 1) {
      const int b = __ffs(lm) - 1;
      sp = ((sp >> b) << (b + 1)) | (sp & ((1u << b) - 1u));
    }
    spread[q] = sp;
    uint32_t w = 0;
#pragma unroll
    for (int j = 0; j < kGroupMax; ++j) {
      w |= ((uint32_t)__popc(e & G.pass[j].zlo) & 1u) << (2 * j);
      w |= ((uint32_t)__popc(e & G.pass[j].alo) & 1u) << (2 * j + 1);
    }
    lowbits[q] = w;
  }
  const uint32_t evenk = 0x55555555u & ((k >= 16) ? 0xffffffffu : ((1u << (2 * k)) - 1u));

  auto issue = [&](uint64_t i) {  // thread 0 only
    const int st = (int)(i % NS);
    double2* buf = reinterpret_cast<double2*>(smem + st * STAGE);
    const uint64_t L0 = (blockIdx.x + i * step) << LT;
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
    uint32_t w = 0;
    for (int j = 0; j < k; ++j) {
      w |= ((G.pass[j].c0 ^ par64(L0 & G.pass[j].zfree)) & 1u) << (2 * j);
      w |= ((G.pass[j].zb ^ par64(L0 & G.pass[j].afree)) & 1u) << (2 * j + 1);
    }
    signs[st] = w;
    if (virt) {  // as in k_group
      mbar_arrive(&full[st]);
      return;
    }
#ifdef OWQS_BOUNDS_CHECK
    bool ok = true;
    for (int r = 0; r < G.nruns && ok; ++r) ok = in_extent(ib + G.runoff[r], G.runlen, G.in_cap, G.errflag);
    if (!ok) {
      mbar_arrive(&full[st]);
      return;
    }
#endif
    mbar_expect_tx(&full[st], NC * RUN);
    const unsigned rbytes = G.runlen * (unsigned)sizeof(double2);
    for (int r = 0; r < G.nruns; ++r) bulk_g2s(buf + r * G.runlen, in + ib + G.runoff[r], rbytes, &full[st]);
  };

  if (threadIdx.x == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], NWARP);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (uint64_t q = 0; q < mine && q < (uint64_t)NS; ++q) issue(q);

  double acc[kGroupMax];
#pragma unroll
  for (int j = 0; j < kGroupMax; ++j) acc[j] = 0.0;
  uint64_t issued = mine < (uint64_t)NS ? mine : (uint64_t)NS;
  for (uint64_t i = 0; i < mine; ++i) {
    const int st = (int)(i % NS);
    if (*abort_flag) break;
    if (!mbar_wait_bounded(&full[st], (unsigned)((i / NS) & 1u))) {
      *abort_flag = 1;
      break;
    }
    const double2* buf = reinterpret_cast<const double2*>(smem + st * STAGE);
    const uint32_t sw = signs[st];
    const uint64_t L0 = (blockIdx.x + i * step) << LT;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = threadIdx.x + q * kBlock;
      double2 x[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) x[c] = virt ? make_double2(G.vconst, 0.0) : buf[G.cbase[c] + spread[q]];
      const uint32_t b = sw ^ lowbits[q];
      // NORM = false: the passes before the last sum no norm; the last one
      // sums its output's squared norm into acc[0]
      const int kl = NORM ? k : k - 1;
#pragma unroll
      for (int j = 0; j < kGroupMax; ++j) {
        if (j >= kl) break;
        const GroupPass& P = G.pass[j];
        const bool rho = (b >> (2 * j + 1)) & 1u;
        const double wr = rho ? -P.wre : P.wre, wi = rho ? -P.wim : P.wim;
        if (M == 1 || P.slot == 0) group_butterfly64<M, 0, NORM>(x, P, wr, wi, acc[j]);
        else if (M == 2 || P.slot == 1) group_butterfly64<M, (M > 1 ? 1 : 0), NORM>(x, P, wr, wi, acc[j]);
        else group_butterfly64<M, (M > 2 ? 2 : 0), NORM>(x, P, wr, wi, acc[j]);
      }
      if (!NORM) {
        const GroupPass& P = G.pass[k - 1];
        const bool rho = (b >> (2 * (k - 1) + 1)) & 1u;
        const double wr = rho ? -P.wre : P.wre, wi = rho ? -P.wim : P.wim;
        if (M == 1 || P.slot == 0) group_butterfly64<M, 0, true>(x, P, wr, wi, acc[0]);
        else if (M == 2 || P.slot == 1) group_butterfly64<M, (M > 1 ? 1 : 0), true>(x, P, wr, wi, acc[0]);
        else group_butterfly64<M, (M > 2 ? 2 : 0), true>(x, P, wr, wi, acc[0]);
      }
      const double f = (__popc(b & evenk) & 1) ? -cprev : cprev;
#pragma unroll
      for (int g = 0; g < NC; ++g) {
        const double sc = f * G.find[g];
        OWQS_IF_IN_EXTENT(L0 + G.outoff[g] + e, 1, G.out_cap, G.errflag)
        out[L0 + G.outoff[g] + e] = make_double2(sc * x[g].x, sc * x[g].y);
      }
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[st]);
    if (threadIdx.x == 0 && issued < mine) {
      if (!mbar_wait_bounded(&empty[st], (unsigned)((i / NS) & 1u))) {
        *abort_flag = 1;
        break;
      }
      issue(issued++);
    }
  }
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) {
      atomicOr(G.errflag, 1u);
      for (uint64_t j = issued > (uint64_t)NS ? issued - NS : 0; j < issued; ++j)
        mbar_wait_bounded(&full[j % NS], (unsigned)((j / NS) & 1u));
    }
    __syncthreads();
    return;
  }
  if (!NORM) {
    if (G.norm_out >= 0) {
      // slot j < k - 1: 2^-(j+1); slot k - 1: the output's summed squared norm
      if (blockIdx.x == 0 && threadIdx.x < k - 1)
        G.norms[G.norm_out + threadIdx.x] = ldexp(1.0, -(int)(threadIdx.x + 1));
      const double a1[1] = {cprev * cprev * G.nscale[k - 1] * acc[0]};
      reduce_to_slots<1>(a1, G.partials, G.counter, G.norms, G.norm_out + k - 1, 1);
    }
    return;
  }
  if (G.norm_out >= 0) {
    const double c2 = cprev * cprev;
    double a[kGroupMax];
#pragma unroll
    for (int j = 0; j < kGroupMax; ++j) a[j] = c2 * G.nscale[j] * acc[j];
    reduce_to_slots<kGroupMax>(a, G.partials, G.counter, G.norms, G.norm_out, k);
  }
}

}  // namespace owqs
