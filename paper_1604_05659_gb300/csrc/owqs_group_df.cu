// Pass groups in complex128 computed in double-float arithmetic on the FP32
// pipes (k_group_df).  GB300 runs FP64 at 1/64 of its FP32 rate, and the
// plain complex128 group (k_group64) is bound by that pipe.  Here every real
// number is an unevaluated sum hi + lo of two floats (about 48 significant
// bits), and the butterflies, signs and squared norms of the pass-group
// contract (owqs_internal.h) use error-free float transforms: Knuth's
// TwoSum, the fast two-sum when the larger operand is known, and the
// FMA-based exact product (Dekker's product with a fused multiply-add).
// The arrays in device memory stay complex128 at the ends of a run; between
// two such groups they may be kept as double-float pairs (four floats per
// amplitude, the same 16 bytes), so that the FP64 conversions happen only
// where a run's input is read or its output written.
#include <algorithm>
#include <mutex>

#include "owqs_device.cuh"

namespace owqs {

namespace {

struct DF {
  float hi, lo;
};

// double -> double-float (exact to about 2^-48 relative) and back
__device__ __forceinline__ DF df_from(double x) {
  const float h = __double2float_rn(x);
  return DF{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly, |a| >= |b| or a == 0
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = a + b;
  return DF{s, b - (s - a)};
}
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return DF{s, (a - (s - bb)) + (b - bb)};
}
// a + sg * b, sg = +-1, with the error of the low parts folded in: absolute
// error about 2^-48 times the larger operand (enough here: the bounds checked
// are absolute on amplitudes of at most 1).  The sign enters as an FMA by
// +-1, which is exact, so no separate negation is needed.
__device__ __forceinline__ DF df_add_signed(DF a, DF b, float sg) {
  const float s = fmaf(sg, b.hi, a.hi);
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + fmaf(sg, b.hi, -bb);
  return fast_two_sum(s, e + fmaf(sg, b.lo, a.lo));
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
// a * b + c * d (one rounding of the cross terms), for the complex product
__device__ __forceinline__ DF df_dot2(DF a, DF b, DF c, DF d) {
  const float p = a.hi * b.hi, q = c.hi * d.hi;
  const float ep = fmaf(a.hi, b.hi, -p), eq = fmaf(c.hi, d.hi, -q);
  const DF s = two_sum(p, q);
  float e = s.lo + ep + eq;
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  e = fmaf(c.hi, d.lo, e);
  e = fmaf(c.lo, d.hi, e);
  return fast_two_sum(s.hi, e);
}
// a * b (the product of the high parts exact, the cross terms rounded once)
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// acc += x^2 (x's square formed exactly in its high part)
__device__ __forceinline__ void df_acc_sq(DF& acc, DF x) {
  const float p = x.hi * x.hi;
  float e = fmaf(x.hi, x.hi, -p);
  e = fmaf(2.f * x.hi, x.lo, e);
  const DF s = two_sum(acc.hi, p);
  acc = fast_two_sum(s.hi, s.lo + (acc.lo + e));
}

struct CDF {
  DF re, im;
};

// one pass on register slot S: y[g0] = x[g0] + ct[g0] v, y[g1] = x[g0] +
// ct[g1] v, v = w x[g1] (w already carries the element's sign); the squared
// norms of the outputs are added to acc
template <int M, int S, bool NORM>
__device__ __forceinline__ void df_pass(CDF (&x)[1 << M], const float (&ct)[1 << M], DF wr, DF wi, DF& acc) {
#pragma unroll
  for (int h = 0; h < (1 << (M - 1)); ++h) {
    const int g0 = ((h >> S) << (S + 1)) | (h & ((1 << S) - 1));
    const int g1 = g0 | (1 << S);
    const CDF x0 = x[g0], x1 = x[g1];
    const DF vr = df_dot2(wr, x1.re, df_neg(wi), x1.im);
    const DF vi = df_dot2(wr, x1.im, wi, x1.re);
    const CDF y0{df_add_signed(x0.re, vr, ct[g0]), df_add_signed(x0.im, vi, ct[g0])};
    const CDF y1{df_add_signed(x0.re, vr, ct[g1]), df_add_signed(x0.im, vi, ct[g1])};
    if (NORM) {
      df_acc_sq(acc, y0.re);
      df_acc_sq(acc, y0.im);
      df_acc_sq(acc, y1.re);
      df_acc_sq(acc, y1.im);
    }
    x[g0] = y0;
    x[g1] = y1;
  }
}

}  // namespace

// The complex128 pass group in double-float.  Same tiling and pipeline as
// k_group64: 2^(11-M) free indices per 32 KB tile, one element per thread
// at a time, a block-wide ring of kDfStages stages filled by bulk copies
// (thread 0) and released by every warp.  IN_DF / OUT_DF: the input / output
// array holds double-float pairs (re.hi, re.lo, im.hi, im.lo) instead of
// complex128.  The pass loop is not unrolled (the code of one double-float
// pass is about four times that of a complex64 one): the per-pass
// constants (w as double-float, the ct signs, the slot) and the per-pass
// norm accumulators of every thread live in shared memory.
constexpr int kDfStages = 2;

template <int M, bool VIRT, bool IN_DF, bool OUT_DF>
__global__ void __launch_bounds__(kBlock, 2) k_group_df(const GroupParams G) {
  if (G.stall_limit > 0) {
    stall_and_give_up(G.stall_limit, G.errflag);
    return;
  }
  constexpr int LT = 11 - M, TE = 1 << LT, NC = 1 << M, NS = kDfStages;
  constexpr int STAGE = NC * TE * 16;
  constexpr int EPT = TE / kBlock;  // elements per thread per tile
  constexpr int NWARP = kBlock / 32;
  static_assert(EPT >= 1 && EPT <= 4, "tile shape");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * STAGE);
  uint64_t* empty = full + NS;
  uint32_t* signs = reinterpret_cast<uint32_t*>(empty + NS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(signs + NS);
  // per pass: w as double-float (wr.hi, wr.lo, wi.hi, wi.lo) and 2^M ct signs
  float4* pw = reinterpret_cast<float4*>(smem + NS * STAGE + 256);
  float* pct = reinterpret_cast<float*>(pw + kGroupMax);
  float2* accs = reinterpret_cast<float2*>(pct + kGroupMax * 8);  // [pass][thread]: double-float sums
  // the output scales +-cprev * fin[g] as double-float, [sign][g]: converted
  // once per block, so that the stores of a double-float output need no FP64
  // instruction (GB300's FP64 pipe runs at 1/64 of the FP32 rate)
  float2* scs = accs + kGroupMax * kBlock;
  // every pass's squared norm unless every probability is exactly 1/2
  // (GroupParams::half) or the run needs none; then only the last pass's (the
  // next launch divides by it) and the other slots get 2^-(j+1)
  const bool norm = !G.half && G.norm_out >= 0;
  const double cprev = [&] {
    if (G.norm_in < 0) return 1.0;
    const double nv = G.norms[G.norm_in];
    return (nv >= G.thresh && nv > 0.0) ? 1.0 / sqrt(nv) : 0.0;
  }();
  constexpr bool virt = VIRT;
  const uint64_t tiles = 1ull << (G.nfree - LT);
  const uint64_t step = gridDim.x;
  const uint64_t mine = blockIdx.x < tiles ? (tiles - blockIdx.x + step - 1) / step : 0;
  const int k = G.k;
  uint32_t slots = 0;
  for (int j = 0; j < kGroupMax; ++j) slots |= ((uint32_t)G.pass[j].slot & 3u) << (2 * j);
  uint32_t lowbits[EPT], spread[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const uint32_t e = (uint32_t)(threadIdx.x + q * kBlock);
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

  auto issue = [&](uint64_t i) {  // thread 0 only
    const int st = (int)(i % NS);
    unsigned char* buf = smem + st * STAGE;
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
    uint32_t w = (G.c0all ^ par64(L0 & G.zall)) << 31;
    for (int j = 0; j < k; ++j) w |= ((G.pass[j].zb ^ par64(L0 & G.pass[j].afree)) & 1u) << j;
    signs[st] = w;
    if (virt) {
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
    mbar_expect_tx(&full[st], (unsigned)STAGE);
    const unsigned rbytes = G.runlen * 16u;
    const unsigned char* src = reinterpret_cast<const unsigned char*>(G.in);
    for (int r = 0; r < G.nruns; ++r)
      bulk_g2s(buf + (size_t)r * G.runlen * 16u, src + (ib + G.runoff[r]) * 16u, rbytes, &full[st]);
  };

  if (threadIdx.x < kGroupMax) {
    const GroupPass& P = G.pass[threadIdx.x];
    const DF wr = df_from(P.wre), wi = df_from(P.wim);
    pw[threadIdx.x] = make_float4(wr.hi, wr.lo, wi.hi, wi.lo);
  }
  for (int t = threadIdx.x; t < kGroupMax * 8; t += kBlock) pct[t] = G.pass[t / 8].ct[t % 8];
  for (int t = threadIdx.x; t < kGroupMax * kBlock; t += kBlock) accs[t] = make_float2(0.f, 0.f);
  if (threadIdx.x < 2 * NC) {
    const int g = threadIdx.x % NC;
    const DF d = df_from((threadIdx.x >= NC ? -cprev : cprev) * G.find[g]);
    scs[threadIdx.x] = make_float2(d.hi, d.lo);
  }
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

  const DF vc = df_from(G.vconst);
  uint64_t issued = mine < (uint64_t)NS ? mine : (uint64_t)NS;
  for (uint64_t i = 0; i < mine; ++i) {
    const int st = (int)(i % NS);
    if (*abort_flag) break;
    if (!mbar_wait_bounded(&full[st], (unsigned)((i / NS) & 1u))) {
      *abort_flag = 1;
      break;
    }
    const unsigned char* buf = smem + st * STAGE;
    const uint32_t sw = signs[st];
    const uint64_t L0 = (blockIdx.x + i * step) << LT;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = threadIdx.x + q * kBlock;
      CDF x[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (virt) {
          x[c] = CDF{vc, DF{0.f, 0.f}};
        } else if (IN_DF) {
          const float4 v = reinterpret_cast<const float4*>(buf)[G.cbase[c] + spread[q]];
          x[c] = CDF{DF{v.x, v.y}, DF{v.z, v.w}};
        } else {
          const double2 v = reinterpret_cast<const double2*>(buf)[G.cbase[c] + spread[q]];
          x[c] = CDF{df_from(v.x), df_from(v.y)};
        }
      }
      const uint32_t b = sw ^ lowbits[q];
#pragma unroll 1
      for (int j = 0; j < k; ++j) {
        const float4 w4 = pw[j];
        const bool rho = (b >> j) & 1u;
        const DF wr = rho ? DF{-w4.x, -w4.y} : DF{w4.x, w4.y};
        const DF wi = rho ? DF{-w4.z, -w4.w} : DF{w4.z, w4.w};
        float ct[NC];
#pragma unroll
        for (int g = 0; g < NC; ++g) ct[g] = pct[j * 8 + g];
        const int slot = (int)((slots >> (2 * j)) & 3u);
        if (norm || j == k - 1) {  // half groups: the last pass's squared norm only
          const float2 a2 = accs[j * kBlock + threadIdx.x];
          DF acc{a2.x, a2.y};
          if (M == 1 || slot == 0) df_pass<M, 0, true>(x, ct, wr, wi, acc);
          else if (M == 2 || slot == 1) df_pass<M, (M > 1 ? 1 : 0), true>(x, ct, wr, wi, acc);
          else df_pass<M, (M > 2 ? 2 : 0), true>(x, ct, wr, wi, acc);
          accs[j * kBlock + threadIdx.x] = make_float2(acc.hi, acc.lo);
        } else {
          DF acc{0.f, 0.f};
          if (M == 1 || slot == 0) df_pass<M, 0, false>(x, ct, wr, wi, acc);
          else if (M == 2 || slot == 1) df_pass<M, (M > 1 ? 1 : 0), false>(x, ct, wr, wi, acc);
          else df_pass<M, (M > 2 ? 2 : 0), false>(x, ct, wr, wi, acc);
        }
      }
      // the element's sign, the previous array's 1/sqrt(N) and the carried
      // scales: applied in FP64 to a complex128 output, in double-float (the
      // block's converted table) to a double-float one
      const uint32_t neg = (b >> 31) & 1u;
#pragma unroll
      for (int g = 0; g < NC; ++g) {
        OWQS_IF_IN_EXTENT(L0 + G.outoff[g] + e, 1, G.out_cap, G.errflag) {
          if (OUT_DF) {
            const float2 s2 = scs[neg * NC + g];
            const DF s{s2.x, s2.y};
            const DF yr = df_mul(s, x[g].re), yi = df_mul(s, x[g].im);
            reinterpret_cast<float4*>(G.out)[L0 + G.outoff[g] + e] = make_float4(yr.hi, yr.lo, yi.hi, yi.lo);
          } else {
            const double sc = (neg ? -cprev : cprev) * G.find[g];
            reinterpret_cast<double2*>(G.out)[L0 + G.outoff[g] + e] =
                make_double2(sc * df_to(x[g].re), sc * df_to(x[g].im));
          }
        }
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
  if (!norm) {
    if (G.norm_out >= 0) {
      if (blockIdx.x == 0 && threadIdx.x < k - 1)
        G.norms[G.norm_out + threadIdx.x] = ldexp(1.0, -(int)(threadIdx.x + 1));
      const float2 sl = accs[(k - 1) * kBlock + threadIdx.x];
      const double a1[1] = {cprev * cprev * G.nscale[k - 1] * ((double)sl.x + (double)sl.y)};
      reduce_to_slots<1>(a1, G.partials, G.counter, G.norms, G.norm_out + k - 1, 1);
    }
    return;
  }
  if (G.norm_out >= 0) {
    const double c2 = cprev * cprev;
    double a[kGroupMax];
#pragma unroll
    for (int j = 0; j < kGroupMax; ++j) {
      const float2 s = accs[j * kBlock + threadIdx.x];
      a[j] = c2 * G.nscale[j] * ((double)s.x + (double)s.y);
    }
    reduce_to_slots<kGroupMax>(a, G.partials, G.counter, G.norms, G.norm_out, k);
  }
}

template <int M, bool VIRT, bool IN_DF, bool OUT_DF>
static cudaError_t launch_df_t(const GroupParams& G, cudaStream_t s) {
  constexpr int STAGE = 32768;
  constexpr int SMEM =
      kDfStages * STAGE + 256 + kGroupMax * 16 + kGroupMax * 8 * 4 + kGroupMax * kBlock * 8 + 2 * 8 * 8;
  auto kern = k_group_df<M, VIRT, IN_DF, OUT_DF>;
  static int grid_cap = 0;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (grid_cap == 0) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, SMEM);
      if (e != cudaSuccess) return e;
      grid_cap = std::max(1, per_sm) * (max_grid() / 8);
    }
  }
  const uint64_t tiles = 1ull << (G.nfree - (11 - M));
  kern<<<capped_grid((int)std::min<uint64_t>(tiles, (uint64_t)grid_cap)), kBlock, SMEM, s>>>(G);
  return cudaGetLastError();
}

template <int M>
static cudaError_t launch_df_m(const GroupParams& G, bool in_df, bool out_df, cudaStream_t s) {
  if (G.in == nullptr)
    return out_df ? launch_df_t<M, true, false, true>(G, s) : launch_df_t<M, true, false, false>(G, s);
  if (in_df)
    return out_df ? launch_df_t<M, false, true, true>(G, s) : launch_df_t<M, false, true, false>(G, s);
  return out_df ? launch_df_t<M, false, false, true>(G, s) : launch_df_t<M, false, false, false>(G, s);
}

cudaError_t launch_group_df(const GroupParams& G, bool in_df, bool out_df, cudaStream_t s) {
  switch (G.m) {
    case 1: return launch_df_m<1>(G, in_df, out_df, s);
    case 2: return launch_df_m<2>(G, in_df, out_df, s);
    case 3: return launch_df_m<3>(G, in_df, out_df, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace owqs
