// Batched recognition and determinism checks (Section 1, the recognition
// problem; Section 4.5, every branch of a flow pattern gives the same state):
// many patterns, all their basis columns and many outcome branches in one
// persistent launch.
//
// Every item is compiled on the host into its pass list (the same schedule
// owqs_run uses, with the EOWQS scaling: each measurement of the forced
// branch taken with probability 1/2).  Items whose widest array fits a
// shared-memory column block are run by k_batch: persistent CTAs pull
// (item, column block) tasks from a counter, hold the block's states in two
// shared-memory buffers and run the item's whole pass list on chip, writing
// only the final columns to HBM.  Wider items go through the pass kernels of
// owqs_run / owqs_unitary.  An optional overlap kernel reduces <out_ref|out>
// per item on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "owqs_internal.h"

namespace owqs {

// host threads (each with its own stream) that run the wide items of
// different patterns side by side
constexpr size_t kWideWorkers = 8;
// items up to 2^kBatchGlobalLog amplitudes that do not fit shared memory run
// in the persistent global-memory launch (state buffers of 2 x 2 MiB per CTA
// in complex64)
constexpr int kBatchGlobalLog = 18;

struct BPass {
  int32_t n_in, r, b, n_out;  // b < 0: final pass
  uint64_t xmask, zmask;
  uint32_t c0, nq, q_off, perm_off;
  uint32_t star;              // measure pass in star form at b with no X mask:
  uint32_t amask, zb;         //   sign = c0 ^ par(k & zmask) ^ k_b (zb ^ par(k & amask))
  uint32_t pad_;
  double w1re, w1im, scale;
};
struct BQ {
  uint64_t a;
  int32_t u, pad;
};
struct BItem {
  uint32_t pass_off, npass;
  int32_t nin, nout, wmax;
  uint32_t cols;  // 2^nin (all basis columns) or 1 (a given input vector)
  uint32_t cb;    // columns per task
  uint32_t pad;
  const void* psi_in;
  void* out;
};
struct BTask {
  uint32_t item, col0;
};

template <typename T> struct BCplx;
template <> struct BCplx<float> { using V = float2; };
template <> struct BCplx<double> { using V = double2; };

__device__ __forceinline__ uint64_t b_ins0(uint64_t j, int b) {
  return ((j >> b) << (b + 1)) | (j & ((1ull << b) - 1));
}

__device__ __forceinline__ uint32_t b_sign(const BPass& ps, const BQ* __restrict__ qs, uint64_t k) {
  uint32_t s = ps.c0 ^ ((uint32_t)__popcll(k & ps.zmask) & 1u);
  for (uint32_t e = 0; e < ps.nq; ++e) {
    const BQ q = qs[ps.q_off + e];
    s ^= (uint32_t)((k >> q.u) & 1ull) & ((uint32_t)__popcll(k & q.a) & 1u);
  }
  return s & 1u;
}

// GLOBAL: the two state buffers of a task live in this CTA's slice of a
// global-memory scratch (2 cap amplitudes per CTA) instead of shared memory,
// for items too wide for a shared-memory column block; the pass interpreter
// is the same (the CTA's threads share the buffers through __syncthreads).
template <typename T, bool GLOBAL>
__global__ void __launch_bounds__(kBlock) k_batch(const BItem* __restrict__ items, const BPass* __restrict__ passes,
                                                  const BQ* __restrict__ qs, const int32_t* __restrict__ perms,
                                                  const BTask* __restrict__ tasks, uint32_t ntasks,
                                                  unsigned int* next_task, uint32_t cap, void* gscratch) {
  using V = typename BCplx<T>::V;
  extern __shared__ __align__(16) unsigned char bsm[];
  V* const base = GLOBAL ? reinterpret_cast<V*>(gscratch) + (size_t)blockIdx.x * 2 * cap : reinterpret_cast<V*>(bsm);
  __shared__ uint32_t task_id;
  for (;;) {
    if (threadIdx.x == 0) task_id = atomicAdd(next_task, 1u);
    __syncthreads();
    const uint32_t t = task_id;
    __syncthreads();
    if (t >= ntasks) break;
    const BTask tk = tasks[t];
    const BItem it = items[tk.item];
    const uint32_t B = it.cb;
    const uint32_t stride = 1u << it.wmax;
    V* cur = base;
    V* nxt = base + cap;
    {  // basis columns col0 .. col0+B-1, or the given input vector
      const uint32_t n = (uint32_t)it.nin;
      const V* __restrict__ vin = reinterpret_cast<const V*>(it.psi_in);
      for (uint32_t idx = threadIdx.x; idx < (B << n); idx += blockDim.x) {
        const uint32_t col = idx >> n, i = idx & ((1u << n) - 1u);
        V v;
        if (vin) {
          v = vin[i];
        } else {
          v.x = (i == tk.col0 + col) ? (T)1 : (T)0;
          v.y = (T)0;
        }
        cur[col * stride + i] = v;
      }
    }
    __syncthreads();
    for (uint32_t p = 0; p < it.npass; ++p) {
      const BPass ps = passes[it.pass_off + p];
      const uint64_t inmask = (1ull << ps.n_in) - 1ull;
      const T sc = (T)ps.scale, wr = (T)(ps.scale * ps.w1re), wi = (T)(ps.scale * ps.w1im);
      const uint32_t n_out = (uint32_t)ps.n_out;
      const uint32_t total = B << n_out;
      if (ps.b >= 0 && ps.star) {
        // star form, no X mask, every index below 2^24: 32-bit index math and
        // both signs from two parities
        const uint32_t b = (uint32_t)ps.b, z = (uint32_t)ps.zmask;
        const uint32_t lowm = (1u << b) - 1u, nmask = (1u << n_out) - 1u, inm = (1u << ps.n_in) - 1u;
        const T nsc = -sc, nwr = -wr, nwi = -wi;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
          const uint32_t col = idx >> n_out, j = idx & nmask;
          const uint32_t k0 = ((j >> b) << (b + 1)) | (j & lowm);
          const V* src = cur + col * stride;
          const V x0 = src[k0 & inm], x1 = src[(k0 | (1u << b)) & inm];  // prepared qubits: broadcast
          const uint32_t s0 = (ps.c0 ^ (uint32_t)__popc(k0 & z)) & 1u;
          const uint32_t s1 = (s0 ^ ps.zb ^ (uint32_t)__popc(k0 & ps.amask)) & 1u;
          const T a = s0 ? nsc : sc, br = s1 ? nwr : wr, bi = s1 ? nwi : wi;
          V y;
          y.x = a * x0.x + br * x1.x - bi * x1.y;
          y.y = a * x0.y + br * x1.y + bi * x1.x;
          nxt[col * stride + j] = y;
        }
      } else if (ps.b >= 0) {
        const uint64_t bb = 1ull << ps.b;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
          const uint32_t col = idx >> n_out;
          const uint64_t j = idx & ((1u << n_out) - 1u);
          const uint64_t k0 = b_ins0(j, ps.b), k1 = k0 | bb;
          const V* src = cur + col * stride;
          V x0 = src[(k0 ^ ps.xmask) & inmask], x1 = src[(k1 ^ ps.xmask) & inmask];
          if (b_sign(ps, qs, k0)) x0.x = -x0.x, x0.y = -x0.y;
          if (b_sign(ps, qs, k1)) x1.x = -x1.x, x1.y = -x1.y;
          V y;
          y.x = sc * x0.x + wr * x1.x - wi * x1.y;
          y.y = sc * x0.y + wr * x1.y + wi * x1.x;
          nxt[col * stride + j] = y;
        }
      } else {
        V* __restrict__ out = reinterpret_cast<V*>(it.out);
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
          const uint32_t col = idx >> n_out;
          const uint64_t u = idx & ((1u << n_out) - 1u);
          uint64_t k = 0;
          for (uint32_t i = 0; i < n_out; ++i) k |= ((u >> i) & 1ull) << perms[ps.perm_off + i];
          V x = cur[col * stride + ((k ^ ps.xmask) & inmask)];
          if (b_sign(ps, qs, k)) x.x = -x.x, x.y = -x.y;
          x.x *= sc;
          x.y *= sc;
          out[((uint64_t)(tk.col0 + col) << n_out) + u] = x;
        }
      }
      __syncthreads();
      V* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
}

// <ref|out>, |out|^2, |ref|^2 for one item per block (FP64 accumulation)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_overlap(const void* const* outs, const void* const* refs,
                                                    const uint64_t* lens, double* res) {
  using V = typename BCplx<T>::V;
  const V* __restrict__ a = reinterpret_cast<const V*>(refs[blockIdx.x]);
  const V* __restrict__ x = reinterpret_cast<const V*>(outs[blockIdx.x]);
  const uint64_t n = lens[blockIdx.x];
  double re = 0, im = 0, nx = 0, na = 0;
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double ar = a[i].x, ai = a[i].y, xr = x[i].x, xi = x[i].y;
    re += ar * xr + ai * xi;  // conj(a) x
    im += ar * xi - ai * xr;
    nx += xr * xr + xi * xi;
    na += ar * ar + ai * ai;
  }
  __shared__ double sh[4][kBlock / 32];
  double v[4] = {re, im, nx, na};
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0;
    for (int w = 0; w < kBlock / 32; ++w) s += sh[threadIdx.x][w];
    res[4 * blockIdx.x + threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct BatchCache {
  int device = -1;
  DevBuf items, passes, qs, perms, tasks, counter, ov_ptrs, ov_res;
  // the persistent launch (counter reset + kernel) as a CUDA graph, replayed
  // while the launch shape and the buffers stay the same
  std::string gkey;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap = nullptr;
  std::map<std::string, int> tuned;  // signature -> shared-memory budget (bytes per CTA)
  // items too wide for shared memory: global-memory state buffers and the
  // tasks of their persistent launch, also replayed from a graph
  DevBuf gtasks, gscratch;
  std::string gkey2;
  cudaGraphExec_t gexec2 = nullptr;
};

std::mutex g_batch_mu;
std::map<int, BatchCache> g_batch;

owqs_status bfail(cudaError_t e, const char* what) {
  cudaGetLastError();
  return set_error(e == cudaErrorMemoryAllocation ? OWQS_ERR_OOM : OWQS_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

owqs_status upload(DevBuf& d, const void* src, size_t bytes, cudaStream_t s, const char* what) {
  if (bytes == 0) return OWQS_OK;
  if (d.bytes < bytes) {
    if (d.p) cudaFree(d.p);
    d.p = nullptr;
    d.bytes = 0;
    const size_t want = std::max(bytes, 2 * d.bytes);
    cudaError_t e = cudaMalloc(&d.p, want);
    if (e != cudaSuccess) return bfail(e, what);
    d.bytes = want;
  }
  cudaError_t e = cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? OWQS_OK : bfail(e, what);
}

struct ZeroOrBits : OutcomeSource {
  const Pattern& p;
  const uint8_t* bits;
  ZeroOrBits(const Pattern& pp, const uint8_t* b) : p(pp), bits(b) {}
  bool known_upfront(std::vector<int8_t>& o) override {
    for (size_t k = 0; k < p.meas_qubit.size(); ++k) o[p.meas_qubit[k]] = bits ? (int8_t)(bits[k] & 1u) : 0;
    return true;
  }
  int decide(const PassDesc& d) override { return bits ? (bits[d.meas_k] & 1u) : 0; }
};

}  // namespace

static owqs_status run_batch(const owqs_batch_item* items, uint32_t n, const owqs_batch_opts* o,
                             owqs_batch_info* info) {
  if (!o || (n && !items)) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (o->dtype > OWQS_C128) return set_error(OWQS_ERR_ARG, "bad dtype");
  const auto t_call = std::chrono::steady_clock::now();
  const int dtype = (int)o->dtype;
  const size_t amp = dtype == OWQS_C64 ? 8 : 16;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(o->stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bfail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_batch_mu);
  BatchCache& bc = g_batch[dev];
  bc.device = dev;

  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t smem_limit = (size_t)std::max(0, max_smem - 1024);

  const auto t_compile = std::chrono::steady_clock::now();
  // compile every item: items in contiguous slices on host threads, each
  // into its own tables, then concatenated in item order (offsets shifted)
  std::vector<BItem> bitems(n);
  std::vector<BPass> bpasses;
  std::vector<BQ> bqs;
  std::vector<int32_t> bperms;
  std::vector<char> on_chip(n, 0), in_global(n, 0);
  for (uint32_t i = 0; i < n; ++i) {
    const owqs_batch_item& it = items[i];
    if (!it.pattern || !it.out) return set_error(OWQS_ERR_ARG, "batch item " + std::to_string(i) + ": NULL");
    if (((uintptr_t)it.out % 16) || ((uintptr_t)it.psi_in % 16))
      return set_error(OWQS_ERR_ARG, "batch item " + std::to_string(i) + ": vectors must be 16-byte aligned");
  }
  struct Slice {
    std::vector<BPass> passes;
    std::vector<BQ> qs;
    std::vector<int32_t> perms;
    owqs_status st = OWQS_OK;
    std::string msg;
  };
  auto compile_item = [&](uint32_t i, Slice& sl) -> owqs_status {
    const owqs_batch_item& it = items[i];
    const Pattern& p = it.pattern->p;
    ZeroOrBits src(p, it.outcomes);
    std::vector<PassDesc> pd;
    owqs_status st = compile_schedule(p, OWQS_MODE_EOWQS, src, pd);
    if (st != OWQS_OK) return st;
    BItem& b = bitems[i];
    b.pass_off = (uint32_t)sl.passes.size();
    b.npass = (uint32_t)pd.size();
    b.nin = (int32_t)p.inputs.size();
    b.nout = (int32_t)p.outputs.size();
    b.cols = it.psi_in ? 1u : (1u << b.nin);
    b.psi_in = it.psi_in;
    b.out = it.out;
    int wmax = b.nin;
    for (const PassDesc& d : pd) {
      wmax = std::max({wmax, d.n_in, d.n_out});
      BPass bp;
      std::memset(&bp, 0, sizeof(bp));
      bp.n_in = d.n_in;
      bp.r = d.r;
      bp.b = d.kind == 0 ? d.b : -1;
      bp.n_out = d.n_out;
      bp.xmask = d.xmask;
      bp.zmask = d.zmask;
      bp.c0 = d.c0;
      bp.q_off = (uint32_t)sl.qs.size();
      // quadratic terms: one lower endpoint per edge
      for (auto& ed : d.edges) sl.qs.push_back(BQ{1ull << ed.second, ed.first, 0});
      bp.nq = (uint32_t)(sl.qs.size() - bp.q_off);
      if (d.kind == 0 && d.xmask == 0 && d.n_in + d.r <= 24) {
        uint32_t a = 0;
        bool star = true;
        for (auto& ed : d.edges) {
          if (ed.first == d.b) a |= 1u << ed.second;
          else if (ed.second == d.b) a |= 1u << ed.first;
          else star = false;
        }
        if (star) {
          bp.star = 1;
          bp.amask = a;
          bp.zb = (uint32_t)((d.zmask >> d.b) & 1u);
        }
      }
      bp.perm_off = (uint32_t)sl.perms.size();
      for (int q : d.perm) sl.perms.push_back(q);
      bp.w1re = d.w1re;
      bp.w1im = d.w1im;
      bp.scale = d.scale;
      sl.passes.push_back(bp);
    }
    b.wmax = wmax;
    on_chip[i] = wmax <= 16 && 2 * ((size_t)1 << wmax) * amp <= smem_limit && b.nin <= 20;
    in_global[i] = !on_chip[i] && wmax <= kBatchGlobalLog && b.nin <= 20;
    return OWQS_OK;
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const uint32_t nslices = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>({hw, 32u, (n + 255) / 256}));
  std::vector<Slice> slices(nslices);
  std::vector<uint32_t> first(nslices + 1);
  for (uint32_t t = 0; t <= nslices; ++t) first[t] = (uint32_t)((uint64_t)n * t / nslices);
  auto run_slice = [&](uint32_t t) {
    Slice& sl = slices[t];
    for (uint32_t i = first[t]; i < first[t + 1]; ++i) {
      sl.st = compile_item(i, sl);
      if (sl.st != OWQS_OK) {
        sl.msg = owqs_last_error();
        return;
      }
    }
  };
  if (nslices == 1) {
    run_slice(0);
  } else {
    std::vector<std::thread> pool;
    for (uint32_t t = 0; t < nslices; ++t) pool.emplace_back(run_slice, t);
    for (auto& th : pool) th.join();
  }
  size_t np = 0, nq = 0, nm = 0;
  for (const Slice& sl : slices) {
    if (sl.st != OWQS_OK) return set_error(sl.st, sl.msg);
    np += sl.passes.size();
    nq += sl.qs.size();
    nm += sl.perms.size();
  }
  bpasses.reserve(np);
  bqs.reserve(nq);
  bperms.reserve(nm);
  for (uint32_t t = 0; t < nslices; ++t) {
    Slice& sl = slices[t];
    const uint32_t po = (uint32_t)bpasses.size(), qo = (uint32_t)bqs.size(), mo = (uint32_t)bperms.size();
    for (uint32_t i = first[t]; i < first[t + 1]; ++i) bitems[i].pass_off += po;
    for (BPass& bp : sl.passes) {
      bp.q_off += qo;
      bp.perm_off += mo;
    }
    bpasses.insert(bpasses.end(), sl.passes.begin(), sl.passes.end());
    bqs.insert(bqs.end(), sl.qs.begin(), sl.qs.end());
    bperms.insert(bperms.end(), sl.perms.begin(), sl.perms.end());
    std::vector<BPass>().swap(sl.passes);
  }
  std::string sig = std::to_string(dtype) + ":";
  for (uint32_t i = 0; i < n; ++i)
    sig += std::to_string(bitems[i].wmax) + "/" + std::to_string(bitems[i].nin) + "/" +
           std::to_string(items[i].psi_in ? 1 : 0) + ",";
  const float compile_ms =
      std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t_compile).count();

  // shared-memory budget per CTA: tuned once per batch signature by timing
  // the candidates, unless the caller fixes the column block
  std::vector<size_t> budgets;
  for (size_t kb : {24, 48, 96, 200}) {
    const size_t by = kb << 10;
    if (by <= smem_limit) budgets.push_back(by);
  }
  if (budgets.empty()) budgets.push_back(smem_limit);
  auto make_tasks = [&](size_t budget, std::vector<BTask>& tasks, uint32_t& cap) {
    tasks.clear();
    cap = 0;
    std::vector<std::pair<double, BTask>> tmp;
    for (uint32_t i = 0; i < n; ++i) {
      if (!on_chip[i]) continue;
      BItem& b = bitems[i];
      const size_t col_elems = (size_t)1 << b.wmax;
      size_t cb = o->column_block ? o->column_block : std::max<size_t>(1, budget / (2 * amp * col_elems));
      size_t p2 = 1;
      while (p2 * 2 <= cb) p2 *= 2;
      cb = std::min<size_t>(p2, b.cols);
      while (cb > 1 && 2 * cb * col_elems * amp > smem_limit) cb /= 2;
      b.cb = (uint32_t)cb;
      cap = std::max<uint32_t>(cap, (uint32_t)(cb * col_elems));
      double cost = 0;
      for (uint32_t q = 0; q < b.npass; ++q) cost += std::ldexp((double)cb, bpasses[b.pass_off + q].n_out);
      for (uint32_t c0 = 0; c0 < b.cols; c0 += (uint32_t)cb) tmp.push_back({cost, BTask{i, c0}});
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (auto& t : tmp) tasks.push_back(t.second);
  };

  auto kernel = dtype == OWQS_C64 ? (const void*)k_batch<float, false> : (const void*)k_batch<double, false>;
  auto launch_batch = [&](size_t budget, const std::vector<BTask>& tasks, uint32_t cap,
                          bool graph) -> owqs_status {
    if (tasks.empty()) return OWQS_OK;
    owqs_status st = upload(bc.items, bitems.data(), bitems.size() * sizeof(BItem), s, "batch items");
    if (st == OWQS_OK) st = upload(bc.passes, bpasses.data(), bpasses.size() * sizeof(BPass), s, "batch passes");
    if (st == OWQS_OK && !bqs.empty()) st = upload(bc.qs, bqs.data(), bqs.size() * sizeof(BQ), s, "batch terms");
    if (st == OWQS_OK && !bperms.empty())
      st = upload(bc.perms, bperms.data(), bperms.size() * sizeof(int32_t), s, "batch perms");
    if (st == OWQS_OK) st = upload(bc.tasks, tasks.data(), tasks.size() * sizeof(BTask), s, "batch tasks");
    if (st != OWQS_OK) return st;
    if (!bc.counter.p) {
      cudaError_t e2 = cudaMalloc(&bc.counter.p, 256);
      if (e2 != cudaSuccess) return bfail(e2, "batch counter");
      bc.counter.bytes = 256;
    }
    const size_t smem = 2 * (size_t)cap * amp;
    cudaError_t e2 = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e2 != cudaSuccess) return bfail(e2, "batch kernel smem");
    int per_sm = 0;
    e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem);
    if (e2 != cudaSuccess) return bfail(e2, "batch occupancy");
    const int grid = std::max(1, std::min<int>(std::max(1, per_sm) * (max_grid() / 8), (int)tasks.size()));
    auto* ip = static_cast<const BItem*>(bc.items.p);
    auto* pp = static_cast<const BPass*>(bc.passes.p);
    auto* qp = static_cast<const BQ*>(bc.qs.p);
    auto* mp = static_cast<const int32_t*>(bc.perms.p);
    auto* tp = static_cast<const BTask*>(bc.tasks.p);
    auto* cp = static_cast<unsigned int*>(bc.counter.p);
    const uint32_t nt = (uint32_t)tasks.size();
    auto enqueue = [&](cudaStream_t st) -> cudaError_t {
      cudaError_t e3 = cudaMemsetAsync(cp, 0, sizeof(unsigned int), st);
      if (e3 != cudaSuccess) return e3;
      if (dtype == OWQS_C64)
        k_batch<float, false><<<grid, kBlock, smem, st>>>(ip, pp, qp, mp, tp, nt, cp, cap, nullptr);
      else
        k_batch<double, false><<<grid, kBlock, smem, st>>>(ip, pp, qp, mp, tp, nt, cp, cap, nullptr);
      return cudaGetLastError();
    };
    (void)budget;
    if (!graph) {
      e2 = enqueue(s);
      return e2 == cudaSuccess ? OWQS_OK : bfail(e2, "batch kernel launch");
    }
    // one persistent launch under a captured graph
    std::string key;
    auto add = [&](const void* v, size_t nb) { key.append(reinterpret_cast<const char*>(v), nb); };
    const void* ptrs[6] = {ip, pp, qp, mp, tp, cp};
    add(&dtype, sizeof(dtype));
    add(&grid, sizeof(grid));
    add(&smem, sizeof(smem));
    add(&nt, sizeof(nt));
    add(&cap, sizeof(cap));
    add(ptrs, sizeof(ptrs));
    if (!bc.gexec || key != bc.gkey) {
      if (bc.gexec) {
        cudaGraphExecDestroy(bc.gexec);
        bc.gexec = nullptr;
      }
      if (!bc.cap) {
        e2 = cudaStreamCreateWithFlags(&bc.cap, cudaStreamNonBlocking);
        if (e2 != cudaSuccess) return bfail(e2, "batch capture stream");
      }
      e2 = cudaStreamBeginCapture(bc.cap, cudaStreamCaptureModeThreadLocal);
      if (e2 != cudaSuccess) return bfail(e2, "batch begin capture");
      const cudaError_t el = enqueue(bc.cap);
      cudaGraph_t g = nullptr;
      e2 = cudaStreamEndCapture(bc.cap, &g);
      if (el != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(el != cudaSuccess ? el : e2, "batch capture");
      }
      e2 = cudaGraphInstantiate(&bc.gexec, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) {
        bc.gexec = nullptr;
        return bfail(e2, "batch graph instantiate");
      }
      bc.gkey = key;
    }
    e2 = cudaGraphLaunch(bc.gexec, s);
    return e2 == cudaSuccess ? OWQS_OK : bfail(e2, "batch graph launch");
  };

  std::vector<BTask> tasks;
  uint32_t cap = 0;
  size_t budget = budgets.back();
  uint32_t launches = 0;
  const bool any_chip = std::any_of(on_chip.begin(), on_chip.end(), [](char c) { return c != 0; });
  if (any_chip) {
    if (o->column_block) {
      budget = smem_limit;
    } else {
      auto hit = bc.tuned.find(sig);
      if (hit != bc.tuned.end()) {
        budget = (size_t)hit->second;
      } else {  // autotune: time one launch per candidate budget
        float best_ms = 0;
        bool have = false;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (size_t bud : budgets) {
          make_tasks(bud, tasks, cap);
          cudaEventRecord(e0, s);
          owqs_status st = launch_batch(bud, tasks, cap, false);  // timed without graph capture
          cudaEventRecord(e1, s);
          if (st != OWQS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
          }
          cudaError_t e3 = cudaEventSynchronize(e1);
          if (e3 != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return bfail(e3, "batch autotune");
          }
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (!have || ms < best_ms) have = true, best_ms = ms, budget = bud;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        bc.tuned[sig] = (int)budget;
      }
    }
    make_tasks(budget, tasks, cap);
    owqs_status st = launch_batch(budget, tasks, cap, o->use_graph != 0);
    if (st != OWQS_OK) return st;
    ++launches;
  }

  // items too wide for shared memory (up to 2^kBatchGlobalLog amplitudes):
  // one persistent launch over (item, column) tasks with global-memory
  // state buffers, largest item first
  uint32_t global_items = 0;
  {
    std::vector<std::pair<double, BTask>> tmp;
    uint32_t gcap = 0;
    for (uint32_t i = 0; i < n; ++i) {
      if (!in_global[i]) continue;
      ++global_items;
      BItem& b = bitems[i];
      b.cb = 1;
      gcap = std::max<uint32_t>(gcap, 1u << b.wmax);
      double cost = 0;
      for (uint32_t q = 0; q < b.npass; ++q) cost += std::ldexp(1.0, bpasses[b.pass_off + q].n_out);
      for (uint32_t c0 = 0; c0 < b.cols; ++c0) tmp.push_back({cost, BTask{i, c0}});
    }
    if (!tmp.empty()) {
      std::stable_sort(tmp.begin(), tmp.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
      std::vector<BTask> gt;
      gt.reserve(tmp.size());
      for (auto& t : tmp) gt.push_back(t.second);
      auto gkern = dtype == OWQS_C64 ? (const void*)k_batch<float, true> : (const void*)k_batch<double, true>;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gkern, kBlock, 0);
      if (e != cudaSuccess) return bfail(e, "batch occupancy");
      const int grid = std::max(1, std::min<int>(std::max(1, per_sm) * (max_grid() / 8), (int)gt.size()));
      // items (the column blocks changed), tasks, scratch
      owqs_status st = upload(bc.items, bitems.data(), bitems.size() * sizeof(BItem), s, "batch items");
      if (st == OWQS_OK) st = upload(bc.passes, bpasses.data(), bpasses.size() * sizeof(BPass), s, "batch passes");
      if (st == OWQS_OK && !bqs.empty()) st = upload(bc.qs, bqs.data(), bqs.size() * sizeof(BQ), s, "batch terms");
      if (st == OWQS_OK && !bperms.empty())
        st = upload(bc.perms, bperms.data(), bperms.size() * sizeof(int32_t), s, "batch perms");
      if (st == OWQS_OK) st = upload(bc.gtasks, gt.data(), gt.size() * sizeof(BTask), s, "batch tasks");
      if (st != OWQS_OK) return st;
      const size_t scratch = (size_t)grid * 2 * gcap * amp;
      if (bc.gscratch.bytes < scratch) {
        if (bc.gscratch.p) cudaFree(bc.gscratch.p);
        bc.gscratch.p = nullptr;
        bc.gscratch.bytes = 0;
        e = cudaMalloc(&bc.gscratch.p, scratch);
        if (e != cudaSuccess) return bfail(e, "batch scratch");
        bc.gscratch.bytes = scratch;
      }
      if (!bc.counter.p) {
        e = cudaMalloc(&bc.counter.p, 256);
        if (e != cudaSuccess) return bfail(e, "batch counter");
        bc.counter.bytes = 256;
      }
      auto* ip = static_cast<const BItem*>(bc.items.p);
      auto* pp = static_cast<const BPass*>(bc.passes.p);
      auto* qp = static_cast<const BQ*>(bc.qs.p);
      auto* mp = static_cast<const int32_t*>(bc.perms.p);
      auto* tp = static_cast<const BTask*>(bc.gtasks.p);
      auto* cp = static_cast<unsigned int*>(bc.counter.p) + 1;  // the shared-memory launch uses [0]
      void* sp = bc.gscratch.p;
      const uint32_t nt = (uint32_t)gt.size();
      auto enqueue = [&](cudaStream_t st2) -> cudaError_t {
        cudaError_t e3 = cudaMemsetAsync(cp, 0, sizeof(unsigned int), st2);
        if (e3 != cudaSuccess) return e3;
        if (dtype == OWQS_C64)
          k_batch<float, true><<<grid, kBlock, 0, st2>>>(ip, pp, qp, mp, tp, nt, cp, gcap, sp);
        else
          k_batch<double, true><<<grid, kBlock, 0, st2>>>(ip, pp, qp, mp, tp, nt, cp, gcap, sp);
        return cudaGetLastError();
      };
      if (!o->use_graph) {
        e = enqueue(s);
        if (e != cudaSuccess) return bfail(e, "batch kernel launch");
      } else {
        std::string key;
        auto add = [&](const void* v, size_t nb) { key.append(reinterpret_cast<const char*>(v), nb); };
        const void* ptrs[7] = {ip, pp, qp, mp, tp, cp, sp};
        add(&dtype, sizeof(dtype));
        add(&grid, sizeof(grid));
        add(&nt, sizeof(nt));
        add(&gcap, sizeof(gcap));
        add(ptrs, sizeof(ptrs));
        if (!bc.gexec2 || key != bc.gkey2) {
          if (bc.gexec2) {
            cudaGraphExecDestroy(bc.gexec2);
            bc.gexec2 = nullptr;
          }
          if (!bc.cap) {
            e = cudaStreamCreateWithFlags(&bc.cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return bfail(e, "batch capture stream");
          }
          e = cudaStreamBeginCapture(bc.cap, cudaStreamCaptureModeThreadLocal);
          if (e != cudaSuccess) return bfail(e, "batch begin capture");
          const cudaError_t el = enqueue(bc.cap);
          cudaGraph_t g = nullptr;
          e = cudaStreamEndCapture(bc.cap, &g);
          if (el != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(el != cudaSuccess ? el : e, "batch capture");
          }
          e = cudaGraphInstantiate(&bc.gexec2, g, 0);
          cudaGraphDestroy(g);
          if (e != cudaSuccess) {
            bc.gexec2 = nullptr;
            return bfail(e, "batch graph instantiate");
          }
          bc.gkey2 = key;
        }
        e = cudaGraphLaunch(bc.gexec2, s);
        if (e != cudaSuccess) return bfail(e, "batch graph launch");
      }
      ++launches;
    }
  }

  // wide items: the pass kernels.  Items of different patterns are
  // independent (each pattern has its own workspace), so they run on up to
  // kWideWorkers host threads, each with its own stream: the many small
  // launches of items just too wide for shared memory then overlap on the
  // GPU.  The items of one pattern stay in order on one thread.
  uint32_t hbm = 0;
  std::vector<std::vector<uint32_t>> by_pattern;
  {
    std::map<const owqs_pattern*, size_t> slot;
    for (uint32_t i = 0; i < n; ++i) {
      if (on_chip[i] || in_global[i]) continue;
      ++hbm;
      auto it = slot.find(items[i].pattern);
      if (it == slot.end()) {
        slot[items[i].pattern] = by_pattern.size();
        by_pattern.push_back({i});
      } else {
        by_pattern[it->second].push_back(i);
      }
    }
  }
  auto run_wide = [&](uint32_t i, cudaStream_t ws) -> owqs_status {
    owqs_run_opts ro;
    std::memset(&ro, 0, sizeof(ro));
    ro.dtype = o->dtype;
    ro.mode = OWQS_MODE_EOWQS;
    ro.policy = items[i].outcomes ? OWQS_OUTCOME_FORCED : OWQS_OUTCOME_ZERO;
    ro.io = OWQS_IO_DEVICE;
    ro.stream = ws;
    ro.use_graph = o->use_graph;
    owqs_status st;
    if (items[i].psi_in) {
      st = run_unchecked(items[i].pattern->p, &ro, items[i].psi_in, items[i].out,
                         const_cast<uint8_t*>(items[i].outcomes), nullptr);
      if (st == OWQS_ERR_NOT_DETERMINISTIC) st = OWQS_OK;  // the caller compares the overlaps
    } else {
      st = owqs_unitary(items[i].pattern, &ro, items[i].outcomes, items[i].out, nullptr);
    }
    return st;
  };
  const int nworkers = (int)std::min<size_t>(kWideWorkers, by_pattern.size());
  if (nworkers <= 1) {
    for (const auto& grp : by_pattern)
      for (uint32_t i : grp) {
        owqs_status st = run_wide(i, s);
        if (st != OWQS_OK) return st;
        launches += last_launch_count(items[i].pattern->p, items[i].psi_in == nullptr);
      }
  } else {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaEvent_t start = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(start, s);  // work queued before this call comes first
    if (e != cudaSuccess) {
      if (start) cudaEventDestroy(start);
      return bfail(e, "wide item streams");
    }
    // launch settings that are read lazily, read once here before the workers
    int lg = 0, hint = 0;
    (void)max_grid();
    (void)tma_enabled();
    (void)group_enabled();
    fast_config(OWQS_C64, &lg, &hint);
    fast_config(OWQS_C128, &lg, &hint);
    std::atomic<size_t> next{0};
    std::atomic<uint32_t> wl{0};
    std::vector<owqs_status> wst((size_t)nworkers, OWQS_OK);
    std::vector<std::string> wmsg((size_t)nworkers);
    auto worker = [&](int w) {
      cudaStream_t ws = nullptr;
      cudaError_t we = cudaSetDevice(dev);
      if (we == cudaSuccess) we = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
      if (we == cudaSuccess) we = cudaStreamWaitEvent(ws, start, 0);
      if (we != cudaSuccess) {
        wst[(size_t)w] = we == cudaErrorMemoryAllocation ? OWQS_ERR_OOM : OWQS_ERR_CUDA;
        wmsg[(size_t)w] = std::string("wide item stream: ") + cudaGetErrorString(we);
      }
      for (size_t g; wst[(size_t)w] == OWQS_OK && (g = next.fetch_add(1)) < by_pattern.size();)
        for (uint32_t i : by_pattern[g]) {
          const owqs_status st = run_wide(i, ws);
          if (st != OWQS_OK) {
            wst[(size_t)w] = st;
            wmsg[(size_t)w] = owqs_last_error();
            break;
          }
          wl += last_launch_count(items[i].pattern->p, items[i].psi_in == nullptr);
        }
      if (ws) {
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
      }
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < nworkers; ++w) pool.emplace_back(worker, w);
    for (auto& t : pool) t.join();
    cudaEventDestroy(start);
    for (int w = 0; w < nworkers; ++w)
      if (wst[(size_t)w] != OWQS_OK) return set_error(wst[(size_t)w], wmsg[(size_t)w]);
    launches += wl.load();
  }

  // overlaps with reference items
  if (o->overlaps) {
    std::vector<const void*> ptrs;
    std::vector<uint64_t> lens;
    std::vector<uint32_t> which;
    for (uint32_t i = 0; i < n; ++i) {
      const int32_t r = items[i].ref;
      if (r < 0) continue;
      if ((uint32_t)r >= n || bitems[r].nout != bitems[i].nout || bitems[r].cols != bitems[i].cols)
        return set_error(OWQS_ERR_ARG, "batch item " + std::to_string(i) + ": bad reference item");
      which.push_back(i);
      lens.push_back(((uint64_t)bitems[i].cols) << bitems[i].nout);
    }
    const size_t m = which.size();
    if (m) {
      for (uint32_t i : which) ptrs.push_back(items[i].out);
      for (uint32_t i : which) ptrs.push_back(items[items[i].ref].out);
      std::vector<unsigned char> blob(m * 2 * sizeof(void*) + m * sizeof(uint64_t));
      std::memcpy(blob.data(), ptrs.data(), m * 2 * sizeof(void*));
      std::memcpy(blob.data() + m * 2 * sizeof(void*), lens.data(), m * sizeof(uint64_t));
      owqs_status st = upload(bc.ov_ptrs, blob.data(), blob.size(), s, "overlap pointers");
      if (st != OWQS_OK) return st;
      if (bc.ov_res.bytes < m * 4 * sizeof(double)) {
        if (bc.ov_res.p) cudaFree(bc.ov_res.p);
        bc.ov_res.p = nullptr;
        bc.ov_res.bytes = 0;
        cudaError_t e4 = cudaMalloc(&bc.ov_res.p, m * 4 * sizeof(double));
        if (e4 != cudaSuccess) return bfail(e4, "overlap results");
        bc.ov_res.bytes = m * 4 * sizeof(double);
      }
      auto** pv = static_cast<const void**>(bc.ov_ptrs.p);
      auto* lv = reinterpret_cast<const uint64_t*>(static_cast<unsigned char*>(bc.ov_ptrs.p) + m * 2 * sizeof(void*));
      if (dtype == OWQS_C64)
        k_overlap<float><<<(unsigned)m, kBlock, 0, s>>>(pv, pv + m, lv, static_cast<double*>(bc.ov_res.p));
      else
        k_overlap<double><<<(unsigned)m, kBlock, 0, s>>>(pv, pv + m, lv, static_cast<double*>(bc.ov_res.p));
      cudaError_t e4 = cudaGetLastError();
      if (e4 != cudaSuccess) return bfail(e4, "overlap kernel");
      ++launches;
      std::vector<double> res(m * 4);
      e4 = cudaMemcpyAsync(res.data(), bc.ov_res.p, m * 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e4 == cudaSuccess) e4 = cudaStreamSynchronize(s);
      if (e4 != cudaSuccess) return bfail(e4, "overlap readback");
      for (size_t q = 0; q < m; ++q)
        for (int c = 0; c < 4; ++c) o->overlaps[4 * which[q] + c] = res[4 * q + c];
    }
    for (uint32_t i = 0; i < n; ++i)
      if (items[i].ref < 0)
        for (int c = 0; c < 4; ++c) o->overlaps[4 * i + c] = 0.0;
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bfail(e, "batch run");
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->smem_items = (uint32_t)std::count(on_chip.begin(), on_chip.end(), 1);
    info->hbm_items = hbm;
    info->tasks = (uint32_t)tasks.size();
    info->smem_bytes_per_cta = (uint32_t)(2 * (size_t)cap * amp);
    info->launches = launches;
    info->global_items = global_items;
    info->compile_ms = compile_ms;
    info->call_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t_call).count();
  }
  return OWQS_OK;
}

}  // namespace owqs

extern "C" owqs_status owqs_run_batch(const owqs_batch_item* items, uint32_t n, const owqs_batch_opts* opts,
                                      owqs_batch_info* info) {
  owqs::clear_error();
  return owqs::run_batch(items, n, opts, info);
}
