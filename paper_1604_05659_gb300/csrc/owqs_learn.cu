// Learned reorder proposal: candidate features, a small MLP scorer with its
// training kernels, and the learned reordering, kept only where it is no
// worse than the greedy PROA order of Section 4.3.
//
// The paper picks the next measurement with the hand-set Eq. 18 cost.  Here a
// network scores the same candidates from the Eq. 18 criteria plus quantities
// of the single amplitude array the GPU keeps (its live width now and at the
// measurement); it is trained to imitate the cheapest orders found by the
// greedy sweeps, and its order is kept only if its peak live width and
// amplitude updates are no worse than the greedy order's.
//
// Network: F=12 -> 64 -> 64 -> 1, ReLU.  Matrix products take bfloat16
// inputs (features, weights, activations rounded to nearest even) and
// accumulate in FP32; biases and master weights are FP32; Adam in FP32.  The
// shapes are tiny (batch = candidates), so the kernels use the FP32 pipes
// rather than tensor cores; one warp handles one row (lane l owns hidden
// units l and l+32).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "owqs_internal.h"

namespace owqs {

constexpr int NF = OWQS_MODEL_FEATURES;
constexpr int NH = 64;
constexpr int P_W1 = 0;
constexpr int P_B1 = P_W1 + NH * NF;
constexpr int P_W2 = P_B1 + NH;
constexpr int P_B2 = P_W2 + NH * NH;
constexpr int P_W3 = P_B2 + NH;
constexpr int P_B3 = P_W3 + NH;
constexpr int NPARAM = P_B3 + 1;
static_assert(NPARAM == OWQS_MODEL_PARAMS, "parameter count");

// ---------------------------------------------------------------------------
// candidate features (host)
// ---------------------------------------------------------------------------
class FeatureState {
 public:
  FeatureState(const Pattern& p, const ReorderGraph& g, bool eowqs, bool product_input)
      : g_(g), eowqs_(eowqs) {
    const uint32_t n = p.n;
    parent_.resize(n);
    std::iota(parent_.begin(), parent_.end(), 0u);
    size_.assign(n, 1);
    pending_ = g.pending0;
    selected_.assign(n, 0);
    live_.assign(n, 0);
    nsel_.assign(n, 0);
    measured_.assign(n, 0);
    for (uint32_t q : p.inputs) live_[q] = 1;
    live_count_ = (uint32_t)p.inputs.size();
    if (!product_input)
      for (size_t i = 1; i < p.inputs.size(); ++i) merge(p.inputs[0], p.inputs[i]);
    S_ = std::max<double>(1.0, (double)p.outputs.size());
    K_ = (uint32_t)g.measured.size();
    unresolved_.assign(n, 0);
    for (uint32_t v : g.measured) {
      unresolved_[v] = eowqs ? 0 : (uint32_t)g.deps[v].size();
      if (unresolved_[v] == 0) ready_.insert(v);
    }
  }

  const std::set<uint32_t>& ready() const { return ready_; }
  uint32_t steps_done() const { return step_; }

  void features(uint32_t v, float* f) {
    roots_.clear();
    roots_.push_back(find(v));
    uint32_t newly = live_[v] ? 0u : 1u;
    for (uint32_t u : pending_[v]) {
      roots_.push_back(find(u));
      if (!live_[u]) ++newly;
    }
    std::sort(roots_.begin(), roots_.end());
    roots_.erase(std::unique(roots_.begin(), roots_.end()), roots_.end());
    uint32_t ms = 0;
    for (uint32_t r : roots_) ms += size_[r];
    const double proj = (double)live_count_ + newly;
    f[0] = (float)(ms / S_);
    f[1] = (float)(g_.os[v] / S_);
    f[2] = (float)(g_.ss[v] / S_);
    f[3] = nsel_[v] > 0 ? 1.f : 0.f;
    f[4] = (float)(g_.adj[v].size() / 4.0);
    f[5] = (float)(pending_[v].size() / 4.0);
    f[6] = (float)(live_count_ / S_);
    f[7] = (float)(proj / S_);
    f[8] = (float)newly;
    f[9] = live_[v] ? 1.f : 0.f;
    f[10] = (float)(nsel_[v] / 4.0);
    f[11] = K_ ? (float)((double)(K_ - step_) / K_) : 0.f;
  }

  // measure v: apply its pending E commands, merge sub-states, eliminate v
  void apply(uint32_t v) {
    if (!live_[v]) live_[v] = 1, ++live_count_;
    for (uint32_t u : pending_[v]) {
      merge(v, u);
      if (!live_[u]) live_[u] = 1, ++live_count_;
      auto& pu = pending_[u];
      pu.erase(std::remove(pu.begin(), pu.end(), v), pu.end());
    }
    pending_[v].clear();
    size_[find(v)] -= 1;
    live_[v] = 0;
    --live_count_;
    selected_[v] = 1;
    measured_[v] = 1;
    for (uint32_t u : g_.adj[v]) ++nsel_[u];
    ready_.erase(v);
    for (uint32_t w : g_.rdeps[v])
      if (--unresolved_[w] == 0 && !measured_[w]) ready_.insert(w);
    ++step_;
  }

 private:
  uint32_t find(uint32_t x) {
    while (parent_[x] != x) {
      parent_[x] = parent_[parent_[x]];
      x = parent_[x];
    }
    return x;
  }
  void merge(uint32_t x, uint32_t y) {
    uint32_t rx = find(x), ry = find(y);
    if (rx == ry) return;
    uint32_t root = std::min(rx, ry), other = std::max(rx, ry);
    parent_[other] = root;
    size_[root] += size_[other];
  }

  const ReorderGraph& g_;
  bool eowqs_;
  std::vector<uint32_t> parent_, size_;
  std::vector<std::vector<uint32_t>> pending_;
  std::vector<char> selected_, live_, measured_;
  std::vector<uint32_t> nsel_, unresolved_, roots_;
  std::set<uint32_t> ready_;
  uint32_t live_count_ = 0, K_ = 0, step_ = 0;
  double S_ = 1.0;
};

static inline uint64_t sm64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// network kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

struct SmemWeights {
  float w1[NH * NF], b1[NH], w2[NH * NH], b2[NH], w3[NH], b3;
};

__device__ void load_weights(const float* __restrict__ p, SmemWeights& s) {
  for (int i = threadIdx.x; i < NH * NF; i += blockDim.x) s.w1[i] = bf16r(p[P_W1 + i]);
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) s.w2[i] = bf16r(p[P_W2 + i]);
  for (int i = threadIdx.x; i < NH; i += blockDim.x) {
    s.b1[i] = p[P_B1 + i];
    s.b2[i] = p[P_B2 + i];
    s.w3[i] = bf16r(p[P_W3 + i]);
  }
  if (threadIdx.x == 0) s.b3 = p[P_B3];
  __syncthreads();
}

// one warp per row: lane owns hidden units lane and lane + 32
__device__ __forceinline__ float forward_row(const SmemWeights& s, const float* __restrict__ xrow, float h1[2],
                                             float h2[2]) {
  const int lane = threadIdx.x & 31;
  float x[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) x[f] = bf16r(xrow[f]);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = lane + 32 * q;
    float a = s.b1[j];
#pragma unroll
    for (int f = 0; f < NF; ++f) a = fmaf(s.w1[j * NF + f], x[f], a);
    h1[q] = bf16r(fmaxf(a, 0.f));
  }
  float a2[2] = {s.b2[lane], s.b2[lane + 32]};
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    const float hk = __shfl_sync(0xffffffffu, h1[k >> 5], k & 31);
#pragma unroll
    for (int q = 0; q < 2; ++q) a2[q] = fmaf(s.w2[(lane + 32 * q) * NH + k], hk, a2[q]);
  }
  h2[0] = bf16r(fmaxf(a2[0], 0.f));
  h2[1] = bf16r(fmaxf(a2[1], 0.f));
  float sc = s.w3[lane] * h2[0] + s.w3[lane + 32] * h2[1];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sc += __shfl_xor_sync(0xffffffffu, sc, o);
  return sc + s.b3;
}

__global__ void __launch_bounds__(256) k_mlp_score(const float* __restrict__ params, const float* __restrict__ X,
                                                   uint64_t n, float* __restrict__ score) {
  __shared__ SmemWeights s;
  load_weights(params, s);
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp; r < n; r += nwarps) {
    float h1[2], h2[2];
    const float sc = forward_row(s, X + r * NF, h1, h2);
    if ((threadIdx.x & 31) == 0) score[r] = sc;
  }
}

// forward for training: scores and the (rounded) activations of each row
__global__ void __launch_bounds__(256) k_mlp_fwd_train(const float* __restrict__ params, const float* __restrict__ X,
                                                       uint64_t row0, uint64_t n, float* __restrict__ score,
                                                       float* __restrict__ H1, float* __restrict__ H2) {
  __shared__ SmemWeights s;
  load_weights(params, s);
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp; r < n; r += nwarps) {
    float h1[2], h2[2];
    const float sc = forward_row(s, X + (row0 + r) * NF, h1, h2);
    H1[r * NH + lane] = h1[0];
    H1[r * NH + lane + 32] = h1[1];
    H2[r * NH + lane] = h2[0];
    H2[r * NH + lane + 32] = h2[1];
    if (lane == 0) score[r] = sc;
  }
}

// per step: softmax over -score of its rows; dscore = (1[target] - p) / nsteps
__global__ void k_mlp_softmax(const float* __restrict__ score, const uint32_t* __restrict__ first,
                              const uint32_t* __restrict__ target, uint32_t s0, uint32_t ns, uint64_t row0,
                              float inv_steps, float* __restrict__ dscore, double* __restrict__ loss) {
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= ns) return;
  const uint32_t s = s0 + warp;
  const uint64_t a = first[s] - row0, b = first[s + 1] - row0, t = target[s] - row0;
  float m = -INFINITY;
  for (uint64_t r = a + lane; r < b; r += 32) m = fmaxf(m, -score[r]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  float z = 0.f;
  for (uint64_t r = a + lane; r < b; r += 32) z += expf(-score[r] - m);
  for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
  for (uint64_t r = a + lane; r < b; r += 32) {
    const float pr = expf(-score[r] - m) / z;
    dscore[r] = ((r == t ? 1.f : 0.f) - pr) * inv_steps;
  }
  if (lane == 0) atomicAdd(loss, (double)((m + logf(z)) + score[t]) * inv_steps);
}

// backward through the layers per row: dH2, dH1 and the last layer's grads
__global__ void __launch_bounds__(256) k_mlp_bwd_rows(const float* __restrict__ params, uint64_t n,
                                                      const float* __restrict__ dscore, const float* __restrict__ H1,
                                                      const float* __restrict__ H2, float* __restrict__ D1,
                                                      float* __restrict__ D2, float* __restrict__ grad) {
  __shared__ SmemWeights s;
  __shared__ float gw3[NH];
  __shared__ float gb3;
  load_weights(params, s);
  for (int i = threadIdx.x; i < NH; i += blockDim.x) gw3[i] = 0.f;
  if (threadIdx.x == 0) gb3 = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  float aw3[2] = {0.f, 0.f}, ab3 = 0.f;
  for (uint64_t r = warp; r < n; r += nwarps) {
    const float ds = dscore[r];
    float h2[2] = {H2[r * NH + lane], H2[r * NH + lane + 32]};
    float h1[2] = {H1[r * NH + lane], H1[r * NH + lane + 32]};
    float d2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      aw3[q] = fmaf(ds, h2[q], aw3[q]);
      d2[q] = h2[q] > 0.f ? ds * s.w3[lane + 32 * q] : 0.f;
    }
    ab3 += ds;
    float d1[2] = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NH; ++j) {
      const float dj = __shfl_sync(0xffffffffu, d2[j >> 5], j & 31);
#pragma unroll
      for (int q = 0; q < 2; ++q) d1[q] = fmaf(s.w2[j * NH + lane + 32 * q], dj, d1[q]);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!(h1[q] > 0.f)) d1[q] = 0.f;
      D1[r * NH + lane + 32 * q] = d1[q];
      D2[r * NH + lane + 32 * q] = d2[q];
    }
  }
  atomicAdd(&gw3[lane], aw3[0]);
  atomicAdd(&gw3[lane + 32], aw3[1]);
  if (lane == 0) atomicAdd(&gb3, ab3);
  __syncthreads();
  for (int i = threadIdx.x; i < NH; i += blockDim.x) atomicAdd(&grad[P_W3 + i], gw3[i]);
  if (threadIdx.x == 0) atomicAdd(&grad[P_B3], gb3);
}

// weight gradients of the first two layers: sums over rows of outer products
// (dW2 = D2^T H1, dW1 = D1^T X, db = column sums), each block a chunk of rows
__global__ void __launch_bounds__(256) k_mlp_wgrad(const float* __restrict__ X, uint64_t row0, uint64_t n,
                                                   const float* __restrict__ H1, const float* __restrict__ D1,
                                                   const float* __restrict__ D2, uint32_t chunk,
                                                   float* __restrict__ grad) {
  const uint64_t r0 = (uint64_t)blockIdx.x * chunk;
  const uint64_t r1 = r0 + chunk < n ? r0 + chunk : n;
  const int t = threadIdx.x;
  float acc2[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc2[i] = 0.f;
  // thread t owns dW2 entries t*16 .. t*16+15 (row j = t/4, k = (t%4)*16 ..)
  const int j2 = t >> 2, k2 = (t & 3) * 16;
  // dW1: 768 entries, three per thread
  float acc1[3] = {0.f, 0.f, 0.f};
  float accb2 = 0.f, accb1 = 0.f;
  for (uint64_t r = r0; r < r1; ++r) {
    const float dj = D2[r * NH + j2];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc2[i] = fmaf(dj, H1[r * NH + k2 + i], acc2[i]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int e = t + 256 * q;
      const int j = e / NF, f = e % NF;
      acc1[q] = fmaf(D1[r * NH + j], bf16r(X[(row0 + r) * NF + f]), acc1[q]);
    }
    if (t < NH) {
      accb2 += D2[r * NH + t];
      accb1 += D1[r * NH + t];
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) atomicAdd(&grad[P_W2 + j2 * NH + k2 + i], acc2[i]);
#pragma unroll
  for (int q = 0; q < 3; ++q) atomicAdd(&grad[P_W1 + t + 256 * q], acc1[q]);
  if (t < NH) {
    atomicAdd(&grad[P_B2 + t], accb2);
    atomicAdd(&grad[P_B1 + t], accb1);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1c, float b2c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
}

// ---------------------------------------------------------------------------
// model object (host)
// ---------------------------------------------------------------------------
}  // namespace owqs

struct owqs_model {
  int device = -1;
  float* params = nullptr;  // FP32 master weights
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  double* loss = nullptr;
  float* scratch = nullptr;  // scores, dscore, H1, H2, D1, D2 for one minibatch
  size_t scratch_rows = 0;
  float* cand_feats = nullptr;  // learned reordering: one step's candidates
  float* cand_scores = nullptr;
  size_t cand_cap = 0;
  cudaStream_t stream = nullptr;
  uint64_t adam_t = 0;
  ~owqs_model() {
    for (void* p : {(void*)params, (void*)grad, (void*)adam_m, (void*)adam_v, (void*)loss, (void*)scratch,
                    (void*)cand_feats, (void*)cand_scores})
      if (p) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace owqs {

static owqs_status mfail(cudaError_t e, const char* what) {
  cudaGetLastError();
  return set_error(e == cudaErrorMemoryAllocation ? OWQS_ERR_OOM : OWQS_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

static owqs_status ensure_scratch(owqs_model* m, size_t rows) {
  if (rows <= m->scratch_rows && m->scratch) return OWQS_OK;
  if (m->scratch) cudaFree(m->scratch);
  m->scratch = nullptr;
  m->scratch_rows = 0;
  const size_t want = std::max(rows, (size_t)4096);
  cudaError_t e = cudaMalloc(&m->scratch, want * (2 + 4 * NH) * sizeof(float));
  if (e != cudaSuccess) return mfail(e, "model scratch");
  m->scratch_rows = want;
  return OWQS_OK;
}

// one warp per row, eight rows per 256-thread block, capped at the grid limit
static int rows_grid(uint64_t rows) {
  const uint64_t blocks = (rows * 32 + 255) / 256;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)max_grid()));
}

// loss + gradient of steps [s0, s1) into m->grad (zeroed here) and m->loss
static owqs_status grad_steps(owqs_model* m, const float* X, const uint32_t* first_h, const uint32_t* first_d,
                              const uint32_t* target_d, uint32_t s0, uint32_t s1, uint32_t nsteps_norm,
                              cudaStream_t s) {
  const uint64_t row0 = first_h[s0], row1 = first_h[s1];
  const uint64_t n = row1 - row0;
  owqs_status st = ensure_scratch(m, n);
  if (st != OWQS_OK) return st;
  float* score = m->scratch;
  float* dscore = score + m->scratch_rows;
  float* H1 = dscore + m->scratch_rows;
  float* H2 = H1 + m->scratch_rows * NH;
  float* D1 = H2 + m->scratch_rows * NH;
  float* D2 = D1 + m->scratch_rows * NH;
  cudaError_t e = cudaMemsetAsync(m->grad, 0, NPARAM * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return mfail(e, "gradient reset");
  if (n == 0) return OWQS_OK;
  k_mlp_fwd_train<<<rows_grid(n), 256, 0, s>>>(m->params, X, row0, n, score, H1, H2);
  const uint32_t ns = s1 - s0;
  k_mlp_softmax<<<(ns * 32 + 255) / 256, 256, 0, s>>>(score, first_d, target_d, s0, ns, row0,
                                                       1.f / (float)nsteps_norm, dscore, m->loss);
  k_mlp_bwd_rows<<<rows_grid(n), 256, 0, s>>>(m->params, n, dscore, H1, H2, D1, D2, m->grad);
  const uint32_t chunk = 256;
  k_mlp_wgrad<<<(unsigned)((n + chunk - 1) / chunk), 256, 0, s>>>(X, row0, n, H1, D1, D2, chunk, m->grad);
  e = cudaGetLastError();
  return e == cudaSuccess ? OWQS_OK : mfail(e, "model kernels");
}

// ---------------------------------------------------------------------------
// learned reordering (called by owqs_reorder)
// ---------------------------------------------------------------------------
owqs_status learned_order(const Pattern& p, const owqs_model* mc, bool eowqs, bool product_input,
                          std::vector<uint32_t>& order) {
  owqs_model* m = const_cast<owqs_model*>(mc);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != m->device) return set_error(OWQS_ERR_ARG, "the model lives on another device");
  ReorderGraph g = build_reorder_graph(p, eowqs);
  FeatureState st(p, g, eowqs, product_input);
  const uint32_t K = (uint32_t)g.measured.size();
  std::vector<float> feats;
  std::vector<uint32_t> cands;
  std::vector<float> scores;
  order.clear();
  order.reserve(K);
  for (uint32_t step = 0; step < K; ++step) {
    cands.assign(st.ready().begin(), st.ready().end());
    if (cands.empty()) return set_error(OWQS_ERR_PATTERN, "dependency cycle: no ready qubit");
    feats.resize(cands.size() * NF);
    for (size_t i = 0; i < cands.size(); ++i) st.features(cands[i], &feats[i * NF]);
    if (cands.size() > m->cand_cap) {
      if (m->cand_feats) cudaFree(m->cand_feats);
      if (m->cand_scores) cudaFree(m->cand_scores);
      m->cand_feats = m->cand_scores = nullptr;
      m->cand_cap = 0;
      const size_t cap = std::max<size_t>(cands.size() * 2, 1024);
      cudaError_t e = cudaMalloc(&m->cand_feats, cap * NF * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&m->cand_scores, cap * sizeof(float));
      if (e != cudaSuccess) return mfail(e, "candidate buffers");
      m->cand_cap = cap;
    }
    cudaError_t e = cudaMemcpyAsync(m->cand_feats, feats.data(), feats.size() * sizeof(float),
                                    cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return mfail(e, "candidate features");
    k_mlp_score<<<rows_grid(cands.size()), 256, 0, m->stream>>>(m->params, m->cand_feats, cands.size(),
                                                                 m->cand_scores);
    scores.resize(cands.size());
    e = cudaMemcpyAsync(scores.data(), m->cand_scores, scores.size() * sizeof(float), cudaMemcpyDeviceToHost,
                        m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mfail(e, "scoring candidates");
    size_t best = 0;  // lowest score; ties to the lowest label (cands ascending)
    for (size_t i = 1; i < cands.size(); ++i)
      if (scores[i] < scores[best]) best = i;
    order.push_back(cands[best]);
    st.apply(cands[best]);
  }
  return OWQS_OK;
}

}  // namespace owqs

using namespace owqs;

extern "C" {

owqs_status owqs_reorder_features(const owqs_pattern* h, uint32_t mode, uint32_t product_input,
                                  const uint32_t* order, uint32_t max_cands, uint64_t seed, float* feats,
                                  uint32_t* step_first, uint32_t* target_row, uint64_t cap_rows,
                                  uint64_t* nrows) {
  clear_error();
  if (!h || !order || !nrows || max_cands == 0) return set_error(OWQS_ERR_ARG, "NULL or zero argument");
  if (mode > OWQS_MODE_EOWQS) return set_error(OWQS_ERR_ARG, "bad mode");
  const Pattern& p = h->p;
  const bool eowqs = mode == OWQS_MODE_EOWQS;
  ReorderGraph g = build_reorder_graph(p, eowqs);
  FeatureState st(p, g, eowqs, product_input != 0);
  const uint32_t K = (uint32_t)g.measured.size();
  std::vector<char> seen(p.n, 0);
  for (uint32_t k = 0; k < K; ++k) {
    const uint32_t v = order[k];
    if (v >= p.n || !g.is_meas[v] || seen[v]) return set_error(OWQS_ERR_ARG, "order must list every measured qubit once");
    seen[v] = 1;
  }
  uint64_t rng = seed;
  std::vector<float> f(NF);
  std::vector<uint32_t> others;
  uint64_t rows = 0;
  const bool write = feats && step_first && target_row;
  std::vector<float> buf;
  std::vector<uint32_t> first, tgt;
  first.reserve(K + 1);
  tgt.reserve(K);
  for (uint32_t k = 0; k < K; ++k) {
    const uint32_t v = order[k];
    if (!st.ready().count(v)) return set_error(OWQS_ERR_ARG, "order measures a qubit that is not ready");
    others.clear();
    for (uint32_t u : st.ready())
      if (u != v) others.push_back(u);
    const uint32_t take = std::min<uint32_t>((uint32_t)others.size(), max_cands - 1);
    for (uint32_t i = 0; i < take; ++i) {  // partial Fisher-Yates
      const uint32_t j = i + (uint32_t)(sm64_next(rng) % (others.size() - i));
      std::swap(others[i], others[j]);
    }
    first.push_back((uint32_t)rows);
    tgt.push_back((uint32_t)rows);
    st.features(v, f.data());
    buf.insert(buf.end(), f.begin(), f.end());
    ++rows;
    for (uint32_t i = 0; i < take; ++i) {
      st.features(others[i], f.data());
      buf.insert(buf.end(), f.begin(), f.end());
      ++rows;
    }
    st.apply(v);
  }
  first.push_back((uint32_t)rows);
  *nrows = rows;
  if (!write) return OWQS_OK;
  if (rows > cap_rows) return set_error(OWQS_ERR_ARG, "feature buffer too small");
  std::memcpy(feats, buf.data(), buf.size() * sizeof(float));
  std::memcpy(step_first, first.data(), first.size() * sizeof(uint32_t));
  std::memcpy(target_row, tgt.data(), tgt.size() * sizeof(uint32_t));
  return OWQS_OK;
}

owqs_status owqs_model_create(const float* weights, uint64_t seed, owqs_model** out) {
  clear_error();
  if (!out) return set_error(OWQS_ERR_ARG, "NULL argument");
  *out = nullptr;
  auto* m = new (std::nothrow) owqs_model();
  if (!m) return set_error(OWQS_ERR_OOM, "host allocation");
  cudaGetDevice(&m->device);
  std::vector<float> w(NPARAM);
  if (weights) {
    std::memcpy(w.data(), weights, NPARAM * sizeof(float));
  } else {  // uniform +-1/sqrt(fan_in), biases zero
    uint64_t rng = seed;
    auto uni = [&](float a) { return (float)(((sm64_next(rng) >> 11) * (1.0 / 9007199254740992.0)) * 2 - 1) * a; };
    for (int i = 0; i < NH * NF; ++i) w[P_W1 + i] = uni(1.f / std::sqrt((float)NF));
    for (int i = 0; i < NH * NH; ++i) w[P_W2 + i] = uni(1.f / std::sqrt((float)NH));
    for (int i = 0; i < NH; ++i) w[P_W3 + i] = uni(1.f / std::sqrt((float)NH));
    for (int i = 0; i < NH; ++i) w[P_B1 + i] = w[P_B2 + i] = 0.f;
    w[P_B3] = 0.f;
  }
  cudaError_t e = cudaMalloc(&m->params, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(m->params, w.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete m;
    return mfail(e, "model allocation");
  }
  *out = m;
  return OWQS_OK;
}

void owqs_model_free(owqs_model* m) { delete m; }

owqs_status owqs_model_get_weights(const owqs_model* m, float* w) {
  clear_error();
  if (!m || !w) return set_error(OWQS_ERR_ARG, "NULL argument");
  cudaError_t e = cudaMemcpy(w, m->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? OWQS_OK : mfail(e, "copying weights");
}

owqs_status owqs_model_score(owqs_model* m, const float* feats, uint64_t nrows, float* scores, void* stream) {
  clear_error();
  if (!m || (nrows && (!feats || !scores))) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (!nrows) return OWQS_OK;
  k_mlp_score<<<rows_grid(nrows), 256, 0, (cudaStream_t)stream>>>(m->params, feats, nrows, scores);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OWQS_OK : mfail(e, "scoring");
}

owqs_status owqs_model_gradient(owqs_model* m, const float* feats, const uint32_t* step_first,
                                const uint32_t* target_row, uint32_t nsteps, float* grad, float* loss,
                                void* stream) {
  clear_error();
  if (!m || !feats || !step_first || !target_row || !grad) return set_error(OWQS_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uint32_t> first(nsteps + 1);
  cudaError_t e = cudaMemcpyAsync(first.data(), step_first, (nsteps + 1) * sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mfail(e, "step offsets");
  owqs_status st = grad_steps(m, feats, first.data(), step_first, target_row, 0, nsteps, nsteps, s);
  if (st != OWQS_OK) return st;
  double l = 0;
  e = cudaMemcpyAsync(grad, m->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mfail(e, "gradient readback");
  if (loss) *loss = (float)l;
  return OWQS_OK;
}

owqs_status owqs_model_train(owqs_model* m, const float* feats, const uint32_t* step_first,
                             const uint32_t* target_row, uint32_t nsteps, uint32_t epochs, uint32_t batch_steps,
                             float lr, uint64_t seed, float* losses, void* stream) {
  clear_error();
  if (!m || !feats || !step_first || !target_row || nsteps == 0 || batch_steps == 0)
    return set_error(OWQS_ERR_ARG, "NULL or zero argument");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uint32_t> first(nsteps + 1);
  cudaError_t e = cudaMemcpyAsync(first.data(), step_first, (nsteps + 1) * sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mfail(e, "step offsets");
  const uint32_t nb = (nsteps + batch_steps - 1) / batch_steps;
  std::vector<uint32_t> perm(nb);
  std::iota(perm.begin(), perm.end(), 0u);
  uint64_t rng = seed;
  for (uint32_t ep = 0; ep < epochs; ++ep) {
    for (uint32_t i = nb; i > 1; --i) std::swap(perm[i - 1], perm[sm64_next(rng) % i]);
    double ep_loss = 0;
    for (uint32_t bi = 0; bi < nb; ++bi) {
      const uint32_t s0 = perm[bi] * batch_steps, s1 = std::min(nsteps, s0 + batch_steps);
      owqs_status st = grad_steps(m, feats, first.data(), step_first, target_row, s0, s1, s1 - s0, s);
      if (st != OWQS_OK) return st;
      ++m->adam_t;
      const float b1c = 1.f - std::pow(0.9f, (float)m->adam_t), b2c = 1.f - std::pow(0.999f, (float)m->adam_t);
      k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(m->params, m->grad, m->adam_m, m->adam_v, lr, b1c, b2c);
      double l = 0;
      e = cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return mfail(e, "training step");
      ep_loss += l * (s1 - s0);
    }
    if (losses) losses[ep] = (float)(ep_loss / nsteps);
  }
  return OWQS_OK;
}

}  // extern "C"
