// Device passes of the GB300 one-way quantum computer simulator (sm_103a).
//
// One launch per measurement: it reads the live amplitude array once and
// writes the halved (after elimination) array once, with the segment's N, E,
// X and Z commands applied on the fly (Sections 4.2 and 4.4; Figs. 5 and 6 do
// the same work as separate sweeps on the CPU).  The pass is a bandwidth-bound
// pairwise update, so there are no tensor cores: the kernels move aligned
// 16-byte vectors, keep every thread's reads and writes contiguous, and fold
// the probability reduction of Eq. 13 into the same sweep (FP32 partial sums
// per thread tile promoted to FP64, FP64 across threads and blocks).
//
// Contract with the schedule compiler: see PassDesc in owqs_internal.h.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>

#include "owqs_device.cuh"

namespace owqs {

// sign bit of x(k): c0 ^ parity(k & zmask) ^ XOR_e k_{qu[e]} parity(k & qa[e])
__device__ __forceinline__ uint32_t qsign(const PassParams& P, uint64_t k) {
  uint32_t s = P.c0 ^ par64(k & P.zmask);
  for (int e = 0; e < P.nq; ++e) s ^= (uint32_t)((k >> P.qu[e]) & 1ull) & par64(k & P.qa[e]);
  return s & 1u;
}

// 1/sqrt(N) of the previous array, 0 for an impossible branch
__device__ __forceinline__ double prev_scale(const PassParams& P) {
  if (P.norm_in < 0) return 1.0;
  const double nv = P.norms[P.norm_in];
  return (nv >= P.thresh && nv > 0.0) ? 1.0 / sqrt(nv) : 0.0;
}

// Per-thread running sum of squared norms: compensated FP32 for complex64
// passes, plain FP64 for complex128
template <typename T>
struct NormAcc;
template <>
struct NormAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) { kahan_add(s, c, x); }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct NormAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

// (-1)^s e^{-i theta} of the pass: a launch parameter, or, when the outcome
// is drawn on the device, the value k_decide wrote before this launch
__device__ __forceinline__ double2 pass_w1(const PassParams& P) {
  if (P.w1dev) return make_double2(P.w1dev[0], P.w1dev[1]);
  return make_double2(P.w1re, P.w1im);
}

// ---------------------------------------------------------------------------
// generic pass: one output amplitude per thread iteration; any sign function,
// any X mask, any measured bit, virtual input (VIRT 1: |+> on every input,
// VIRT 2: the diagonal sum over c of |c>|c> that carries every basis column
// of a unitary at once).  MODE 0 measure, 1 the two outcome probabilities
// only, 2 final pass (corrections + output order).
// ---------------------------------------------------------------------------
// One sweep of the generic pass over outputs j0, j0 + stride, ... (in and
// out may point to global or shared memory); the squared norms (MODE 1: of
// both outcomes) are added to acc.  c: the previous array's 1/sqrt(N).
template <typename T, int MODE, int VIRT>
__device__ __forceinline__ void generic_sweep(const PassParams& P, const typename Cplx<T>::V* __restrict__ in,
                                              typename Cplx<T>::V* __restrict__ out, uint64_t j0, uint64_t stride,
                                              double c, double (&acc)[2]) {
  using V = typename Cplx<T>::V;
  if (j0 >= (1ull << P.n_out)) return;
  const T sc = (T)(P.scale * c);
  const double2 w1 = pass_w1(P);
  const T wr = (T)(P.scale * c * w1.x), wi = (T)(P.scale * c * w1.y);
  const T er = (T)(P.edev ? P.edev[0] : P.ere), ei = (T)(P.edev ? P.edev[1] : P.eim);
  const uint64_t nout = 1ull << P.n_out;
  const uint64_t inmask = (1ull << P.n_in) - 1ull;
  const uint64_t bb = MODE == 2 ? 0ull : (1ull << P.b);
  const T vc = (T)P.vconst;
  const uint64_t dmask = (1ull << P.vdiag) - 1ull;
  auto load = [&](uint64_t k) -> V {
    V x;
    if (VIRT == 1) {
      x.x = vc;
      x.y = (T)0;
    } else if (VIRT == 2) {
      const uint64_t i = (k ^ P.xmask) & inmask;
      x.x = ((i & dmask) == (i >> P.vdiag)) ? (T)1 : (T)0;
      x.y = (T)0;
    } else {
      const uint64_t i = (k ^ P.xmask) & inmask;
      if (in_extent(i, 1, P.in_cap, P.errflag)) {
        x = in[i];
      } else {
        x.x = (T)0;
        x.y = (T)0;
      }
    }
    if (qsign(P, k)) x.x = -x.x, x.y = -x.y;
    return x;
  };
  T part[2] = {(T)0, (T)0};
  int cnt = 0;
  for (uint64_t j = j0; j < nout; j += stride) {
    if (MODE == 2) {
      uint64_t k = j;
      if (!P.identity_perm) {
        k = 0;
        for (int i = 0; i < P.n_out; ++i) k |= ((j >> i) & 1ull) << P.perm[i];
      }
      const V x = load(k);
      V y;
      y.x = sc * x.x;
      y.y = sc * x.y;
      if (in_extent(j, 1, P.out_cap, P.errflag)) out[j] = y;
      part[0] += y.x * y.x + y.y * y.y;
    } else {
      const uint64_t k0 = ins0(j, P.b), k1 = k0 | bb;
      const V x0 = load(k0), x1 = load(k1);
      if (MODE == 0) {
        V y;
        y.x = sc * x0.x + wr * x1.x - wi * x1.y;
        y.y = sc * x0.y + wr * x1.y + wi * x1.x;
        if (in_extent(j, 1, P.out_cap, P.errflag)) out[j] = y;
        part[0] += y.x * y.x + y.y * y.y;
      } else {
        const T ex = er * x1.x - ei * x1.y, ey = er * x1.y + ei * x1.x;
        const T a0 = x0.x + ex, b0 = x0.y + ey, a1 = x0.x - ex, b1 = x0.y - ey;
        part[0] += sc * sc * (a0 * a0 + b0 * b0);
        part[1] += sc * sc * (a1 * a1 + b1 * b1);
      }
    }
    if (++cnt == 8) {  // FP32 partials over short runs, promoted to FP64
      acc[0] += (double)part[0];
      acc[1] += (double)part[1];
      part[0] = part[1] = (T)0;
      cnt = 0;
    }
  }
  acc[0] += (double)part[0];
  acc[1] += (double)part[1];
}

template <typename T, int MODE, int VIRT>
__global__ void __launch_bounds__(kBlock) k_generic(const PassParams P) {
  using V = typename Cplx<T>::V;
  double acc[2] = {0.0, 0.0};
  generic_sweep<T, MODE, VIRT>(P, reinterpret_cast<const V*>(P.in), reinterpret_cast<V*>(P.out),
                               (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x,
                               prev_scale(P), acc);
  if (P.norm_out >= 0) {
    if (MODE == 1) {
      reduce_to_slots<2>(acc, P.partials, P.counter, P.norms, P.norm_out);
    } else {
      const double a1[1] = {acc[0]};
      reduce_to_slots<1>(a1, P.partials, P.counter, P.norms, P.norm_out);
    }
  }
}

// Final pass (corrections and output order, MODE 2 above) from an input
// array: four outputs per thread and iteration, whose four loads are issued
// before any of them is used.  With one 8-byte load in flight per thread the
// resident grid keeps about 2.5 MB in flight, too little to cover HBM
// latency at full bandwidth; four loads keep about four times that.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_final(const PassParams P) {
  using V = typename Cplx<T>::V;
  constexpr int U = 4;
  const V* __restrict__ in = reinterpret_cast<const V*>(P.in);
  V* __restrict__ out = reinterpret_cast<V*>(P.out);
  const T sc = (T)(P.scale * prev_scale(P));
  const uint64_t nout = 1ull << P.n_out;
  const uint64_t inmask = (1ull << P.n_in) - 1ull;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nout; j += U * stride) {
    V x[U];
    uint32_t neg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t jj = j + u * stride;
      x[u].x = x[u].y = (T)0;
      neg[u] = 0;
      if (jj < nout) {
        uint64_t k = jj;
        if (!P.identity_perm) {
          k = 0;
          for (int i = 0; i < P.n_out; ++i) k |= ((jj >> i) & 1ull) << P.perm[i];
        }
        const uint64_t i = (k ^ P.xmask) & inmask;
        if (in_extent(i, 1, P.in_cap, P.errflag)) x[u] = in[i];
        neg[u] = qsign(P, k);
      }
    }
    T part = (T)0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t jj = j + u * stride;
      if (jj < nout) {
        const T f = neg[u] ? -sc : sc;
        V y;
        y.x = f * x[u].x;
        y.y = f * x[u].y;
        if (in_extent(jj, 1, P.out_cap, P.errflag)) out[jj] = y;
        part += y.x * y.x + y.y * y.y;
      }
    }
    acc += (double)part;
  }
  if (P.norm_out >= 0) {
    const double a1[1] = {acc};
    reduce_to_slots<1>(a1, P.partials, P.counter, P.norms, P.norm_out);
  }
}

// Final pass whose output order moves the low array bits away from the low
// output bits (perm maps {0..4} elsewhere), so that consecutive outputs are
// far apart in the array and the loads of k_final would not coalesce.  A
// tile is every setting of the output bits T (2^10 outputs): {0..4}, the
// preimage of the array bits {0..4}, and the next output bits up to ten;
// the other ("free") output bits are fixed: the block reads the tile in array order (the array's low five
// bits innermost: 256-byte runs), applies the X mask and the sign, and
// writes it, scaled, in output order (the output's low five bits innermost)
// through shared memory.  The shared-memory slot of a tile element is its
// output-order index with the bits above the fifth XORed into the low five
// (swizzle), so that the 32 lanes of either phase hit 32 different slots
// modulo 32.  The sign of an index k = k0 | kt (k0: the free bits, fixed per
// tile; kt: the tile's bits) splits, since c0 + z.k + sum_e k_u(e) (a_e.k)
// is a quadratic form over GF(2), into a per-tile part, a per-element table
// bit and the parity of kt against a per-tile mask.  Requires n_in == n_out
// and perm a permutation of 0..n_out-1 (checked by the launcher).
constexpr int kFinalTileMax = 10;
__device__ __forceinline__ uint32_t par_idx(uint32_t v) { return (uint32_t)__popc(v) & 1u; }
__device__ __forceinline__ uint32_t par_idx(uint64_t v) { return par64(v); }
// I: the index type, uint32_t when the array has at most 2^31 amplitudes
// (half the integer work of 64-bit indices), else uint64_t
template <typename T, typename I>
__global__ void __launch_bounds__(kBlock) k_final_tiled(const PassParams P) {
  using V = typename Cplx<T>::V;
  constexpr int TM = 1 << kFinalTileMax;
  __shared__ V tile[TM];
  __shared__ I kt[TM];             // read element e: its array bits within T
  __shared__ I jw[TM];             // write element f: its output bits within T
  __shared__ uint16_t fidx[TM];    // read element e: its shared-memory slot; bit 15: its sign within T
  __shared__ uint16_t waddr[TM];   // write element f: its shared-memory slot
  __shared__ uint8_t fbit[64], fperm[64];  // the free output bits and their array bits
  __shared__ int rbit[kFinalTileMax], wbit[kFinalTileMax], swz[32];
  __shared__ int tsh, nfsh;
  const V* __restrict__ in = reinterpret_cast<const V*>(P.in);
  V* __restrict__ out = reinterpret_cast<V*>(P.out);
  const int n = P.n_out;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    int pinv[64];
    for (int i = 0; i < n; ++i) pinv[P.perm[i]] = i;
    uint64_t o2 = 0;  // the output bits of the array's low five bits
    for (int a = 0; a < 5; ++a) o2 |= 1ull << pinv[a];
    // T: the output's low five bits, o2, and the next output bits up to
    // kFinalTileMax bits (longer output runs, fewer tiles)
    uint64_t tm = 0x1full | o2;
    for (int i = 5; i < n && __popcll(tm) < kFinalTileMax; ++i) tm |= 1ull << i;
    int t = 0;
    for (int a = 0; a < 5; ++a) rbit[t++] = pinv[a];  // read order: the array's low bits first
    for (int i = 0; i < n; ++i)
      if (((tm >> i) & 1ull) && !((o2 >> i) & 1ull)) rbit[t++] = i;
    int u = 0, used = 0;
    for (int i = 0; i < n; ++i)  // write order: the output's low bits first
      if ((tm >> i) & 1ull) wbit[u++] = i;
    for (int a = 0; a < 5; ++a)
      if (pinv[a] < 5) used |= 1 << pinv[a];
    // the write positions 5 + q that hold an array-low bit are XORed into
    // the low positions that no array-low bit takes, one each
    int map[kFinalTileMax - 5], nxt = 0;
    for (int q = 0; q < t - 5; ++q) {
      map[q] = -1;
      if ((o2 >> wbit[5 + q]) & 1ull) {
        while ((used >> nxt) & 1) ++nxt;
        map[q] = nxt++;
      }
    }
    for (int h = 0; h < 32; ++h) {
      int x = 0;
      for (int q = 0; q < t - 5; ++q)
        if (((h >> q) & 1) && map[q] >= 0) x |= 1 << map[q];
      swz[h] = x;
    }
    int nf = 0;
    for (int i = 0; i < n; ++i)
      if (!((tm >> i) & 1ull)) {
        fbit[nf] = (uint8_t)i;
        fperm[nf] = (uint8_t)P.perm[i];
        ++nf;
      }
    tsh = t;
    nfsh = nf;
  }
  __syncthreads();
  const int t = tsh, nf = nfsh;
  for (int e = threadIdx.x; e < (1 << t); e += blockDim.x) {
    uint64_t jr = 0, k = 0, jf = 0;
    for (int r = 0; r < t; ++r)
      if ((e >> r) & 1) {
        jr |= 1ull << rbit[r];
        k |= 1ull << P.perm[rbit[r]];
        jf |= 1ull << wbit[r];
      }
    uint32_t f = 0;
    for (int r = 0; r < t; ++r) f |= (uint32_t)((jr >> wbit[r]) & 1ull) << r;
    kt[e] = (I)k;
    fidx[e] = (uint16_t)((f ^ (uint32_t)swz[f >> 5]) | ((qsign(P, k) ^ (P.c0 & 1u)) << 15));
    jw[e] = (I)jf;
    waddr[e] = (uint16_t)(e ^ swz[e >> 5]);
  }
  const T sc = (T)(P.scale * prev_scale(P));
  const I inmask = (I)((1ull << P.n_in) - 1ull), xmask = (I)P.xmask;
  const uint64_t ntiles = 1ull << (n - t);
  constexpr int EPT = TM / kBlock;  // elements of a tile per thread and phase (t == kFinalTileMax)
  static_assert(EPT * kBlock == TM, "whole tiles per block");
  // per tile: the free output bits j0 and their array bits k0 (lane q
  // deposits bits q and q + 32 of tau), the fixed part s0 of the sign and
  // the mask mm that couples the tile's bits to it
  struct Fix {
    I j0, k0, mm;
    uint32_t s0;
  };
  auto fix = [&](uint64_t tau) {
    uint32_t jl = 0, jh = 0, kl = 0, kh = 0;
    for (int q = lane; q < nf; q += 32)
      if ((tau >> q) & 1ull) {
        if (fbit[q] < 32) jl |= 1u << fbit[q];
        else jh |= 1u << (fbit[q] - 32);
        if (fperm[q] < 32) kl |= 1u << fperm[q];
        else kh |= 1u << (fperm[q] - 32);
      }
    const uint64_t j0 = (uint64_t)__reduce_or_sync(0xffffffffu, jl) |
                        ((uint64_t)__reduce_or_sync(0xffffffffu, jh) << 32);
    const uint64_t k0 = (uint64_t)__reduce_or_sync(0xffffffffu, kl) |
                        ((uint64_t)__reduce_or_sync(0xffffffffu, kh) << 32);
    uint32_t qb = 0;
    uint64_t mm = 0;
    for (int e = lane; e < P.nq; e += 32) {
      const uint32_t ub = (uint32_t)((k0 >> P.qu[e]) & 1ull), pa = par64(k0 & P.qa[e]);
      qb ^= ub & pa;
      if (ub) mm ^= P.qa[e];
      if (pa) mm ^= 1ull << P.qu[e];
    }
    uint32_t ml = (uint32_t)mm, mh = (uint32_t)(mm >> 32);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ml ^= __shfl_xor_sync(0xffffffffu, ml, o);
      mh ^= __shfl_xor_sync(0xffffffffu, mh, o);
    }
    Fix F;
    F.j0 = (I)j0;
    F.k0 = (I)k0;
    F.mm = (I)(((uint64_t)mh << 32) | ml);
    F.s0 = (P.c0 ^ par64(k0 & P.zmask) ^ (uint32_t)__reduce_add_sync(0xffffffffu, qb)) & 1u;
    return F;
  };
  // the loads of a tile, into registers
  auto load = [&](const Fix& F, V (&r)[EPT]) {
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = (int)threadIdx.x + u * kBlock;
      const I i = ((F.k0 | kt[e]) ^ xmask) & inmask;
      r[u].x = r[u].y = (T)0;
      if (in_extent((uint64_t)i, 1, P.in_cap, P.errflag)) r[u] = in[i];
    }
  };
  double acc = 0.0;
  uint64_t tau = blockIdx.x;
  __syncthreads();  // the tables are written
  if (tau < ntiles) {
    Fix cur = fix(tau);
    V r[EPT];
    load(cur, r);
    for (;;) {
      const uint64_t nxt = tau + gridDim.x;
      __syncthreads();  // the previous tile's slots are read out
#pragma unroll
      for (int u = 0; u < EPT; ++u) {
        const int e = (int)threadIdx.x + u * kBlock;
        const uint32_t fi = fidx[e];
        V x = r[u];
        if ((cur.s0 ^ (fi >> 15) ^ par_idx((I)(kt[e] & cur.mm))) & 1u) x.x = -x.x, x.y = -x.y;
        tile[fi & 0x7fffu] = x;
      }
      // the next tile's loads are in flight while this one is written out
      Fix nx = cur;
      if (nxt < ntiles) {
        nx = fix(nxt);
        load(nx, r);
      }
      __syncthreads();
      T part = (T)0;
#pragma unroll
      for (int u = 0; u < EPT; ++u) {
        const int f = (int)threadIdx.x + u * kBlock;
        const I j = cur.j0 | jw[f];
        V y = tile[waddr[f]];
        y.x = sc * y.x;
        y.y = sc * y.y;
        if (in_extent((uint64_t)j, 1, P.out_cap, P.errflag)) out[j] = y;
        part += y.x * y.x + y.y * y.y;
      }
      acc += (double)part;
      if (nxt >= ntiles) break;
      tau = nxt;
      cur = nx;
    }
  }
  if (P.norm_out >= 0) {
    const double a1[1] = {acc};
    reduce_to_slots<1>(a1, P.partials, P.counter, P.norms, P.norm_out);
  }
}

// whether the final pass takes k_final_tiled: an output order that moves the
// low five array bits away from the low five output bits, on an array of at
// least 2^11 amplitudes whose width the pass keeps
static bool final_needs_tiles(const PassParams& P) {
  if (P.identity_perm || P.n_out < kFinalTileMax + 1 || P.n_in != P.n_out || P.n_out > 62) return false;
  uint64_t seen = 0;
  for (int i = 0; i < P.n_out; ++i) {
    if (P.perm[i] < 0 || P.perm[i] >= P.n_out || ((seen >> P.perm[i]) & 1ull)) return false;
    seen |= 1ull << P.perm[i];
  }
  for (int i = 0; i < 5; ++i)
    if (P.perm[i] >= 5) return true;
  return false;
}

// ---------------------------------------------------------------------------
// A whole run of a small pattern in one warp (every array of the run at most
// 2^kSmallLog amplitudes and at most kSmallMaxPasses passes, where one launch
// per pass would be mostly launch latency).  The passes (planned exactly as
// for the per-pass kernels) are first copied into shared memory; each pass
// reads the previous pass's output from shared memory (the first reads the
// input vector or the virtual input) and writes shared memory (the final
// pass writes the output vector).  After each measurement the warp adds the
// squared norms in FP64 (a shuffle tree: every lane holds the total), lane 0
// stores the slot and every lane keeps the next pass's 1/sqrt(N).  One warp:
// the arrays are at most a few hundred amplitudes, the complex128 arithmetic
// is bound by the SM's FP64 pipe, not by warps, and no block barrier is
// needed.  input_norm: slot 0 first gets the input vector's squared norm.
// ---------------------------------------------------------------------------
constexpr int kSmallBlock = 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kSmallBlock) k_small(const PassParams* __restrict__ passes, int npass,
                                                        int input_norm) {
  using V = typename Cplx<T>::V;
  static_assert(sizeof(PassParams) % 16 == 0, "copied as 16-byte words");
  extern __shared__ __align__(16) unsigned char dsm[];
  PassParams* sp = reinterpret_cast<PassParams*>(dsm);  // npass entries
  __shared__ V buf[2][1 << kSmallLog];
  const int lane = threadIdx.x;
  {
    const uint4* src = reinterpret_cast<const uint4*>(passes);
    uint4* dst = reinterpret_cast<uint4*>(sp);
    const int nw = npass * (int)(sizeof(PassParams) / 16);
    for (int k = lane; k < nw; k += 32) dst[k] = src[k];
  }
  __syncwarp();
  int slast = -1;      // the last stored slot
  double cnext = 1.0;  // and its 1/sqrt(N)
  auto keep = [&](const PassParams& P, int slot, double t) {
    if (lane == 0) P.norms[slot] = t;
    cnext = (t >= P.thresh && t > 0.0) ? 1.0 / sqrt(t) : 0.0;
    slast = slot;
  };
  if (input_norm) {
    const PassParams& P0 = sp[0];
    const V* in = reinterpret_cast<const V*>(P0.in);
    double a = 0.0;
    for (uint64_t i = lane; i < (1ull << P0.n_in); i += 32)
      a += (double)in[i].x * (double)in[i].x + (double)in[i].y * (double)in[i].y;
    keep(P0, 0, warp_sum(a));
  }
  for (int p = 0; p < npass; ++p) {
    const PassParams& P = sp[p];
    const bool last = p == npass - 1;
    const V* in = p == 0 ? reinterpret_cast<const V*>(P.in) : buf[(p - 1) & 1];
    V* out = last ? reinterpret_cast<V*>(P.out) : buf[p & 1];
    const double c = P.norm_in < 0 ? 1.0 : (P.norm_in == slast ? cnext : prev_scale(P));
    double acc[2] = {0.0, 0.0};
    const int virt = (p == 0 && P.in == nullptr) ? (P.vdiag ? 2 : 1) : 0;
    if (last) {
      if (virt == 0) generic_sweep<T, 2, 0>(P, in, out, lane, 32, c, acc);
      else if (virt == 1) generic_sweep<T, 2, 1>(P, in, out, lane, 32, c, acc);
      else generic_sweep<T, 2, 2>(P, in, out, lane, 32, c, acc);
    } else {
      if (virt == 0) generic_sweep<T, 0, 0>(P, in, out, lane, 32, c, acc);
      else if (virt == 1) generic_sweep<T, 0, 1>(P, in, out, lane, 32, c, acc);
      else generic_sweep<T, 0, 2>(P, in, out, lane, 32, c, acc);
    }
    const double t = warp_sum(acc[0]);
    if (P.norm_out >= 0) keep(P, P.norm_out, t);
    __syncwarp();  // this pass's outputs are visible to the next
  }
}

cudaError_t launch_small(const PassParams* passes_dev, int npass, int input_norm, int dtype, cudaStream_t s) {
  constexpr int kMaxDyn = kSmallMaxPasses * (int)sizeof(PassParams);
  static bool ready = false;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!ready) {
      cudaError_t e = cudaFuncSetAttribute(k_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
      if (e != cudaSuccess) return e;
      ready = true;
    }
  }
  if (npass < 1 || npass > kSmallMaxPasses) return cudaErrorInvalidValue;
  const size_t dyn = (size_t)npass * sizeof(PassParams);
  if (dtype == OWQS_C64) k_small<float><<<1, kSmallBlock, dyn, s>>>(passes_dev, npass, input_norm);
  else k_small<double><<<1, kSmallBlock, dyn, s>>>(passes_dev, npass, input_norm);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fast measure pass: sign function in star form at the measured bit b (every
// E of the segment touches the measured qubit, which is what reordering by
// the Proposition of Section 4.3 produces), no X mask.  A thread tile is 2^L
// consecutive outputs of the live part times 2^rt values of the lowest
// broadcast (newly prepared) bits; it reads its input amplitudes once with
// 16-byte loads and writes 2^(L+rt) outputs with 16-byte stores.
//   BM < L   : b = BM, the pair partners sit in one aligned run of 2^(L+1)
//   BM == L  : L <= b < n_in, two aligned runs of 2^L, 2^b apart
//   BM == L+1: b is a new qubit, both partners read the same amplitude
// ---------------------------------------------------------------------------
// 16-byte vector loads and stores of aligned runs; HINT 1 marks them
// evict-first (each amplitude is read and written once per pass)
template <int HINT, typename V>
__device__ __forceinline__ V ld16(const V* p) {
  if constexpr (HINT) return __ldcs(p);
  else return *p;
}
template <int HINT, typename V>
__device__ __forceinline__ void st16(V* p, const V& v) {
  if constexpr (HINT) __stcs(p, v);
  else *p = v;
}
template <int HINT, int N>
__device__ __forceinline__ void ld_run(float2 (&v)[N], const float2* p) {
  static_assert(N % 2 == 0, "float2 runs move in pairs");
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    const float4 t = ld16<HINT>(q + i);
    v[2 * i] = make_float2(t.x, t.y);
    v[2 * i + 1] = make_float2(t.z, t.w);
  }
}
template <int HINT, int N>
__device__ __forceinline__ void ld_run(double2 (&v)[N], const double2* p) {
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = ld16<HINT>(p + i);
}
template <int HINT, int N>
__device__ __forceinline__ void st_run(float2* p, const float2 (&v)[N]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int i = 0; i < N / 2; ++i)
    st16<HINT>(q + i, make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y));
}
template <int HINT, int N>
__device__ __forceinline__ void st_run(double2* p, const double2 (&v)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) st16<HINT>(p + i, v[i]);
}

__host__ __device__ constexpr int ins0c(int l, int b) { return ((l >> b) << (b + 1)) | (l & ((1 << b) - 1)); }

template <typename T, int L, int BM, int HINT>
__global__ void __launch_bounds__(kBlock) k_fast(const PassParams P) {
  using V = typename Cplx<T>::V;
  constexpr int NL = 1 << L;
  const V* __restrict__ in = reinterpret_cast<const V*>(P.in);
  V* __restrict__ out = reinterpret_cast<V*>(P.out);
  const double c = prev_scale(P);
  const T sc = (T)(P.scale * c);
  const double2 w1 = pass_w1(P);
  const T wr = (T)(P.scale * c * w1.x), wi = (T)(P.scale * c * w1.y);
  const int b = P.b, nlo = P.nlo, rt = P.rt;
  const uint64_t tiles = 1ull << (P.n_out - L - rt);
  const uint64_t lomask = (1ull << (nlo - L)) - 1ull;
  const int hishift = nlo + rt;
  const uint64_t inmask = (1ull << P.n_in) - 1ull;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  NormAcc<T> acc;
  for (uint64_t tile = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; tile < tiles; tile += stride) {
    const uint64_t J = ((tile & lomask) << L) | ((tile >> (nlo - L)) << hishift);
    const uint64_t K0 = ins0(J, b);
    const uint32_t pz = P.c0 ^ par64(K0 & P.zmask);
    const uint32_t pa = P.zb ^ par64(K0 & P.amask);
    const uint64_t ib = K0 & inmask;
    V v0[NL], v1[NL];
    if (!in_extent(ib, BM == L ? (1ull << b) + NL : (BM < L ? 2 * NL : NL), P.in_cap, P.errflag) ||
        !in_extent(J, ((uint64_t)((1 << rt) - 1) << nlo) + NL, P.out_cap, P.errflag))
      continue;
    if constexpr (BM < L) {
      V run[2 * NL];
      ld_run<HINT>(run, in + ib);
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        v0[l] = run[ins0c(l, BM)];
        v1[l] = run[ins0c(l, BM) | (1 << BM)];
      }
    } else if constexpr (BM == L) {
      ld_run<HINT>(v0, in + ib);
      ld_run<HINT>(v1, in + ib + (1ull << b));
    } else {
      ld_run<HINT>(v0, in + ib);
#pragma unroll
      for (int l = 0; l < NL; ++l) v1[l] = v0[l];
    }
    T tacc = (T)0;
#pragma unroll
    for (int t = 0; t < (1 << kFastRMax); ++t) {
      if (t >= (1 << rt)) break;
      const uint32_t st0 = pz ^ ((P.tzt >> t) & 1u);
      const uint32_t st1 = st0 ^ pa ^ ((P.tat >> t) & 1u);
      V y[NL];
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const uint32_t s0 = (st0 ^ (P.tzl >> l)) & 1u;
        const uint32_t s1 = (st1 ^ (P.tzl >> l) ^ (P.tal >> l)) & 1u;
        const T a = s0 ? -sc : sc;
        const T br = s1 ? -wr : wr, bi = s1 ? -wi : wi;
        y[l].x = a * v0[l].x + br * v1[l].x - bi * v1[l].y;
        y[l].y = a * v0[l].y + br * v1[l].y + bi * v1[l].x;
        tacc += y[l].x * y[l].x + y[l].y * y[l].y;
      }
      st_run<HINT>(out + J + ((uint64_t)t << nlo), y);
    }
    acc.add(tacc);
  }
  if (P.norm_out >= 0) {
    const double a1[1] = {acc.value()};
    reduce_to_slots<1>(a1, P.partials, P.counter, P.norms, P.norm_out);
  }
}


// ---------------------------------------------------------------------------
// TMA-pipelined measure pass (same contract and eligibility as k_fast, for
// passes whose live part spans at least one tile of TE outputs).
//
// A persistent CTA walks tiles of TE consecutive live outputs.  Thread 0
// stages each tile's input amplitudes into shared memory with bulk async
// copies (cp.async.bulk, completion counted in bytes on an mbarrier), up to
// kTmaStages tiles ahead, so many bytes are in flight per SM while the
// threads only hold a few registers.  The threads then combine the pairs
// (x(k0), x(k1)) from shared memory for every value of the broadcast bits and
// write the outputs with 16-byte coalesced stores.
//   CASE 0: b < log2 TE    one run of 2 TE inputs, partners 2^b apart
//   CASE 1: b >= log2 TE   two runs of TE inputs, 2^b apart in the input
//   CASE 2: b >= n_in      b is a new qubit; one run of TE inputs
// Every mbarrier wait is bounded (kWaitLimitCycles): on expiry the block
// agrees to stop, records an error code and returns.
// ---------------------------------------------------------------------------
template <typename T>
struct TmaShape {
  static constexpr int LTE = kTmaLogTileC64;
  static constexpr int TE = 1 << LTE;
  static constexpr int STAGE_BYTES = 2 * TE * (int)sizeof(T) * 2;
  static constexpr int SMEM = kTmaStages * STAGE_BYTES + kTmaStages * 8;
};

// PROB: instead of the outputs, both outcome probabilities of the
// measurement (sampled outcomes): the squared norms of x0' + e x1' and
// x0' - e x1' (x0', x1' the sign-applied pair, e = e^{-i theta}) into slots
// norm_out and norm_out + 1, as k_generic<T, 1, .> computes them.
template <typename T, int CASE, bool PROB>
__global__ void __launch_bounds__(kBlock, 2) k_tma(const PassParams P) {
  if (P.stall_limit > 0) {
    stall_and_give_up(P.stall_limit, P.errflag);
    return;
  }
  using V = typename Cplx<T>::V;
  using S = TmaShape<T>;
  constexpr int LTE = S::LTE, TE = S::TE, NS = kTmaStages;
  constexpr int VE = sizeof(T) == 4 ? 2 : 1;  // outputs per 16-byte vector
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * S::STAGE_BYTES);
  const V* __restrict__ in = reinterpret_cast<const V*>(P.in);
  V* __restrict__ out = reinterpret_cast<V*>(P.out);
  const double c = prev_scale(P);
  const T sc = (T)(P.scale * c);
  const double2 w1 = pass_w1(P);
  const T wr = (T)(P.scale * c * w1.x), wi = (T)(P.scale * c * w1.y);
  const T er = (T)(P.edev ? P.edev[0] : P.ere), ei = (T)(P.edev ? P.edev[1] : P.eim);
  const int b = P.b, nlo = P.nlo, nbc = P.n_out - P.nlo;
  const uint64_t inmask = (1ull << P.n_in) - 1ull;
  const uint64_t tiles = 1ull << (nlo - LTE);
  const uint64_t step = gridDim.x;
  const uint64_t mine = blockIdx.x < tiles ? (tiles - blockIdx.x + step - 1) / step : 0;
  const uint32_t zlo = (uint32_t)(P.zmask & ((2ull << LTE) - 1ull));
  const uint32_t alo = (uint32_t)(P.amask & ((2ull << LTE) - 1ull));
  constexpr unsigned IN_BYTES = (CASE == 2 ? 1u : 2u) * TE * sizeof(V);

  auto issue = [&](uint64_t i) {  // thread 0: stage tile i of this block
    const int st = (int)(i % NS);
    V* buf = reinterpret_cast<V*>(smem + st * S::STAGE_BYTES);
    const uint64_t tile = blockIdx.x + i * step;
    const uint64_t ib = ins0(tile << LTE, b) & inmask;
    if (!in_extent(ib, CASE == 1 ? (1ull << b) + TE : IN_BYTES / sizeof(V), P.in_cap, P.errflag)) {
      mbar_arrive(&full[st]);  // no copy: the stage keeps stale data, the run reports the error
      return;
    }
    mbar_expect_tx(&full[st], IN_BYTES);
    if constexpr (CASE == 1) {
      bulk_g2s(buf, in + ib, TE * sizeof(V), &full[st]);
      bulk_g2s(buf + TE, in + ib + (1ull << b), TE * sizeof(V), &full[st]);
    } else {
      bulk_g2s(buf, in + ib, IN_BYTES, &full[st]);
    }
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) mbar_init(&full[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (uint64_t i = 0; i < mine && i < (uint64_t)NS; ++i) issue(i);

  NormAcc<T> acc, acc1;  // acc1: outcome 1 (PROB)
  uint64_t issued = mine < (uint64_t)NS ? mine : (uint64_t)NS;
  uint64_t i = 0;
  bool failed = false;
  for (; i < mine; ++i) {
    const int st = (int)(i % NS);
    const bool ok = mbar_wait_bounded(&full[st], (unsigned)((i / NS) & 1u));
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const V* buf = reinterpret_cast<const V*>(smem + st * S::STAGE_BYTES);
    const uint64_t tile = blockIdx.x + i * step;
    const uint64_t J = tile << LTE;
    const uint64_t K0 = ins0(J, b);
    const uint32_t pz = P.c0 ^ par64(K0 & P.zmask);
    const uint32_t pa = P.zb ^ par64(K0 & P.amask);
    T tacc = (T)0, tacc1 = (T)0;
    for (uint64_t t = 0; t < (1ull << nbc); ++t) {
      const uint64_t dt = ins0(t << nlo, b);
      const uint32_t s0t = pz ^ par64(dt & P.zmask);
      const uint32_t s1t = s0t ^ pa ^ par64(dt & P.amask);
      V* o = out + J + (t << nlo);
      if (!PROB && !in_extent(J + (t << nlo), TE, P.out_cap, P.errflag)) continue;
#pragma unroll 2
      for (int e = threadIdx.x * VE; e < TE; e += kBlock * VE) {
        V x0[VE], x1[VE], y[VE];
#pragma unroll
        for (int v = 0; v < VE; ++v) {
          const int jj = e + v;
          const int d0 = CASE == 0 ? (int)ins0((uint64_t)jj, b) : jj;
          x0[v] = buf[d0];
          x1[v] = CASE == 0 ? buf[d0 | (1 << b)] : (CASE == 1 ? buf[TE + jj] : buf[jj]);
          const uint32_t s0 = (s0t ^ __popc((uint32_t)d0 & zlo)) & 1u;
          const uint32_t s1 = (s1t ^ __popc((uint32_t)d0 & zlo) ^ __popc((uint32_t)d0 & alo)) & 1u;
          if constexpr (PROB) {
            const T v0x = s0 ? -x0[v].x : x0[v].x, v0y = s0 ? -x0[v].y : x0[v].y;
            T ux = er * x1[v].x - ei * x1[v].y, uy = er * x1[v].y + ei * x1[v].x;
            if (s1) ux = -ux, uy = -uy;
            const T a0x = v0x + ux, a0y = v0y + uy, a1x = v0x - ux, a1y = v0y - uy;
            tacc += a0x * a0x + a0y * a0y;
            tacc1 += a1x * a1x + a1y * a1y;
          } else {
            const T a = s0 ? -sc : sc;
            const T br = s1 ? -wr : wr, bi = s1 ? -wi : wi;
            y[v].x = a * x0[v].x + br * x1[v].x - bi * x1[v].y;
            y[v].y = a * x0[v].y + br * x1[v].y + bi * x1[v].x;
            tacc += y[v].x * y[v].x + y[v].y * y[v].y;
          }
        }
        if constexpr (!PROB) {
          if constexpr (VE == 2) {
            *reinterpret_cast<float4*>(o + e) = make_float4(y[0].x, y[0].y, y[1].x, y[1].y);
          } else {
            o[e] = y[0];
          }
        }
      }
    }
    acc.add(tacc);
    if (PROB) acc1.add(tacc1);
    __syncthreads();  // every thread is done with stage st
    if (threadIdx.x == 0 && issued < mine) issue(issued++);
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicOr(P.errflag, 1u);
      // let copies already issued land before the block's memory goes away
      for (uint64_t j = i; j < issued; ++j) mbar_wait_bounded(&full[j % NS], (unsigned)((j / NS) & 1u));
    }
    __syncthreads();
    return;  // the block partial is skipped; the host reports the error
  }
  if (P.norm_out >= 0) {
    if constexpr (PROB) {
      const double s2 = (P.scale * c) * (P.scale * c);
      const double a2[2] = {s2 * acc.value(), s2 * acc1.value()};
      reduce_to_slots<2>(a2, P.partials, P.counter, P.norms, P.norm_out);
    } else {
      const double a1[1] = {acc.value()};
      reduce_to_slots<1>(a1, P.partials, P.counter, P.norms, P.norm_out);
    }
  }
}


// squared norm of an input vector (OWQS divides by it).  complex64: 16-byte
// loads of two amplitudes, squared norms summed in FP32 (packed FP32x2) over
// chunks of at most 16 amplitudes and the chunks in FP64 (GB300's FP64 pipe
// runs at 1/64 of the FP32 rate: per-amplitude FP64 products made this
// kernel FP64-bound, 2.5 ms for 2^28 amplitudes); complex128, and a
// complex64 vector that is not 16-byte aligned: FP64 per amplitude.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_norm(const void* vin, uint64_t n, double* norms, int slot,
                                                 double* partials, unsigned int* counter) {
  using V = typename Cplx<T>::V;
  double acc = 0.0;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if (sizeof(T) == 4 && ((uintptr_t)vin & 15u) == 0) {
    constexpr int kChunk = 8;  // float4 loads per FP32 partial
    const float4* __restrict__ in4 = reinterpret_cast<const float4*>(vin);
    const uint64_t npairs = n / 2;
    for (uint64_t i = tid; i < npairs;) {
      float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < kChunk; ++c) {
        if (i < npairs) {
          const float4 v = in4[i];
          s2 = __ffma2_rn(make_float2(v.x, v.y), make_float2(v.x, v.y), s2);
          s2 = __ffma2_rn(make_float2(v.z, v.w), make_float2(v.z, v.w), s2);
          i += stride;
        }
      }
      acc += (double)s2.x + (double)s2.y;
    }
    if ((n & 1u) && tid == 0) {
      const float2 x = reinterpret_cast<const float2*>(vin)[n - 1];
      acc += (double)x.x * (double)x.x + (double)x.y * (double)x.y;
    }
  } else {  // complex128, or a complex64 vector that is not 16-byte aligned
    const V* __restrict__ in = reinterpret_cast<const V*>(vin);
    for (uint64_t i = tid; i < n; i += stride) {
      const V x = in[i];
      acc += (double)x.x * (double)x.x + (double)x.y * (double)x.y;
    }
  }
  const double a1[1] = {acc};
  reduce_to_slots<1>(a1, partials, counter, norms, slot);
}

// ---------------------------------------------------------------------------
// launch wrappers.  Grid-stride kernels get at most as many blocks as can be
// resident at once (occupancy x SMs), so every block runs in one wave.
// ---------------------------------------------------------------------------
template <typename K>
static int resident_grid(K kernel, int want) {
  static std::mutex mu;
  static std::map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find((const void*)kernel);
  int cap;
  if (it != cache.end()) {
    cap = it->second;
  } else {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess || per_sm <= 0)
      per_sm = 1;
    cap = std::min(per_sm * (max_grid() / 8), max_grid());
    cache[(const void*)kernel] = cap;
  }
  return std::max(1, std::min(want, cap));
}

template <typename K>
static void go(K kernel, const PassParams& P, int want, cudaStream_t s) {
  kernel<<<capped_grid(resident_grid(kernel, want)), kBlock, 0, s>>>(P);
}

template <typename T, int L, int HINT>
static cudaError_t launch_fast(const PassParams& P, const LaunchPlan& Lp, cudaStream_t s) {
  static_assert(L >= 1 && L <= 3, "tile width");
  switch (Lp.variant) {
    case 0: go(k_fast<T, L, 0, HINT>, P, Lp.grid, s); break;
    case 1: go(k_fast<T, L, (L > 1 ? 1 : L), HINT>, P, Lp.grid, s); break;
    case 2: go(k_fast<T, L, (L > 2 ? 2 : (L == 2 ? L : L + 1)), HINT>, P, Lp.grid, s); break;
    case 3: go(k_fast<T, L, (L == 3 ? L : L + 1), HINT>, P, Lp.grid, s); break;
    case 4: go(k_fast<T, L, L + 1, HINT>, P, Lp.grid, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

template <typename T, int CASE, bool PROB>
static cudaError_t launch_tma_case(const PassParams& P, cudaStream_t s) {
  using S = TmaShape<T>;
  auto kernel = k_tma<T, CASE, PROB>;
  static int grid_cap = 0;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (grid_cap == 0) {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, S::SMEM);
      if (e != cudaSuccess) return e;
      grid_cap = std::max(1, per_sm) * (max_grid() / 8);
    }
  }
  const uint64_t tiles = 1ull << (P.nlo - S::LTE);
  const int grid = capped_grid((int)std::min<uint64_t>(tiles, (uint64_t)grid_cap));
  kernel<<<grid, kBlock, S::SMEM, s>>>(P);
  return cudaSuccess;
}

template <typename T>
static cudaError_t launch_t(const PassParams& P, const LaunchPlan& L, cudaStream_t s) {
  const bool virt = P.in == nullptr;
  switch (L.kind) {
    case KK_TMA: {  // planned for complex64 only
      cudaError_t e = cudaErrorInvalidValue;
      if constexpr (sizeof(T) == 4)
        e = L.variant == 0 ? launch_tma_case<T, 0, false>(P, s)
                           : (L.variant == 1 ? launch_tma_case<T, 1, false>(P, s)
                                             : launch_tma_case<T, 2, false>(P, s));
      if (e != cudaSuccess) return e;
      break;
    }
    case KK_PROB_TMA: {  // both outcome probabilities, the bulk-copy pass's tiles (complex64)
      cudaError_t e = cudaErrorInvalidValue;
      if constexpr (sizeof(T) == 4)
        e = L.variant == 0 ? launch_tma_case<T, 0, true>(P, s)
                           : (L.variant == 1 ? launch_tma_case<T, 1, true>(P, s)
                                             : launch_tma_case<T, 2, true>(P, s));
      if (e != cudaSuccess) return e;
      break;
    }
    case KK_FAST: {
      cudaError_t e = cudaErrorInvalidValue;
      if constexpr (sizeof(T) == 4) {
        if (L.lg == 2) e = L.hint ? launch_fast<T, 2, 1>(P, L, s) : launch_fast<T, 2, 0>(P, L, s);
        else if (L.lg == 3) e = L.hint ? launch_fast<T, 3, 1>(P, L, s) : launch_fast<T, 3, 0>(P, L, s);
      } else {
        if (L.lg == 1) e = L.hint ? launch_fast<T, 1, 1>(P, L, s) : launch_fast<T, 1, 0>(P, L, s);
        else if (L.lg == 2) e = L.hint ? launch_fast<T, 2, 1>(P, L, s) : launch_fast<T, 2, 0>(P, L, s);
      }
      if (e != cudaSuccess) return e;
      break;
    }
    case KK_GENERIC:
      if (!virt) go(k_generic<T, 0, 0>, P, L.grid, s);
      else if (P.vdiag) go(k_generic<T, 0, 2>, P, L.grid, s);
      else go(k_generic<T, 0, 1>, P, L.grid, s);
      break;
    case KK_PROB:
      if (virt) go(k_generic<T, 1, 1>, P, L.grid, s);
      else go(k_generic<T, 1, 0>, P, L.grid, s);
      break;
    case KK_FINAL:
      if (!virt) {
        if (final_needs_tiles(P)) {
          if (P.n_in <= 31) go(k_final_tiled<T, uint32_t>, P, L.grid, s);
          else go(k_final_tiled<T, uint64_t>, P, L.grid, s);
        }
        else go(k_final<T>, P, L.grid, s);
      }
      else if (P.vdiag) go(k_generic<T, 2, 2>, P, L.grid, s);
      else go(k_generic<T, 2, 1>, P, L.grid, s);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pass(const PassParams& P, const LaunchPlan& L, int dtype, cudaStream_t s) {
  return dtype == OWQS_C64 ? launch_t<float>(P, L, s) : launch_t<double>(P, L, s);
}

// ---------------------------------------------------------------------------
// Outcome of one measurement drawn on the device (sampled policy): u is
// output number `draw` of the splitmix64 stream seeded with *seed (the
// generator is counter based: output k mixes seed + (k+1) * 0x9E3779B97F4A7C15
// with the published splitmix64 finaliser), taken as its top 53 bits over
// 2^53; outcome 0 iff u <= prob_0 (Fig. 6).  The thread then writes
// (-1)^outcome e^{-i theta} for the measure pass that follows, and, since
// every signal of the next measurement is now known (its domains were
// measured first), the next measurement's e^{-i theta}, theta = (-1)^s alpha
// + t pi (Eq. 2), for that measurement's probability pass.  One thread.
// ---------------------------------------------------------------------------
__global__ void k_decide(const DecideParams D) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint64_t z = *D.seed + (D.draw + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  const int o = u <= D.norms[D.pslot] ? 0 : 1;
  D.outcomes[D.meas_k] = (uint8_t)o;
  D.w1[0] = o ? -D.e_this[0] : D.e_this[0];
  D.w1[1] = o ? -D.e_this[1] : D.e_this[1];
  if (!D.has_next) return;
  uint32_t ss = 0, tt = 0;
  for (uint32_t i = 0; i < D.sd_len; ++i) ss ^= D.outcomes[D.dom[D.sd_off + i]];
  for (uint32_t i = 0; i < D.td_len; ++i) tt ^= D.outcomes[D.dom[D.td_off + i]];
  double er = D.ca, ei = (ss & 1u) ? D.sa : -D.sa;
  if (tt & 1u) er = -er, ei = -ei;
  D.e_next[0] = er;
  D.e_next[1] = ei;
}

__global__ void k_put_u64(uint64_t* dst, uint64_t v) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *dst = v;
}

cudaError_t launch_decide(const DecideParams& D, cudaStream_t s) {
  k_decide<<<1, 32, 0, s>>>(D);
  return cudaGetLastError();
}

cudaError_t launch_put_u64(uint64_t* dst, uint64_t v, cudaStream_t s) {
  k_put_u64<<<1, 32, 0, s>>>(dst, v);
  return cudaGetLastError();
}

// Join of an input factor (product input, Section 4.1: a tensor product of
// sub-states): out[j] = s in[j mod 2^n_in] phi[j >> n_in], the factor's
// qubits becoming the top bits; s normalises the factor (and the previous
// array in OWQS mode).  Grid-stride over the outputs.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_kron(const KronParams K) {
  using V = typename Cplx<T>::V;
  const V* __restrict__ in = reinterpret_cast<const V*>(K.in);
  const V* __restrict__ phi = reinterpret_cast<const V*>(K.phi);
  V* __restrict__ out = reinterpret_cast<V*>(K.out);
  double sc = 1.0;
  if (K.fnorm >= 0) {  // -1: the factor is taken as normalised
    const double nf = K.norms[K.fnorm];
    sc = nf > 0.0 ? 1.0 / sqrt(nf) : 0.0;
  }
  if (K.norm_in >= 0) {
    const double nv = K.norms[K.norm_in];
    sc = nv > 0.0 ? sc / sqrt(nv) : 0.0;
  }
  const T s = (T)sc;
  const uint64_t n = 1ull << (K.n_in + K.q), lo = (1ull << K.n_in) - 1ull;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const V f = phi[j >> K.n_in];
    V a;
    if (in) {
      if (!in_extent(j & lo, 1, K.in_cap, K.errflag)) continue;
      a = in[j & lo];
    } else {
      a.x = (T)1;
      a.y = (T)0;
    }
    V y;
    y.x = s * (a.x * f.x - a.y * f.y);
    y.y = s * (a.x * f.y + a.y * f.x);
    if (in_extent(j, 1, K.out_cap, K.errflag)) out[j] = y;
  }
}

cudaError_t launch_kron(const KronParams& K, int dtype, cudaStream_t s) {
  const uint64_t n = 1ull << (K.n_in + K.q);
  const int grid = (int)std::min<uint64_t>((n + kBlock - 1) / kBlock, (uint64_t)max_grid());
  if (dtype == OWQS_C64) k_kron<float><<<capped_grid(grid), kBlock, 0, s>>>(K);
  else k_kron<double><<<capped_grid(grid), kBlock, 0, s>>>(K);
  return cudaGetLastError();
}

cudaError_t launch_norm(const void* in, uint64_t n, int dtype, double* norms, int slot, double* partials,
                        unsigned int* counter, int grid, cudaStream_t s) {
  if (dtype == OWQS_C64) k_norm<float><<<capped_grid(grid), kBlock, 0, s>>>(in, n, norms, slot, partials, counter);
  else k_norm<double><<<capped_grid(grid), kBlock, 0, s>>>(in, n, norms, slot, partials, counter);
  return cudaGetLastError();
}

}  // namespace owqs
