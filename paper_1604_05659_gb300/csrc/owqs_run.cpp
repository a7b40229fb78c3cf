// Run driver: device workspace, launch list, CUDA-graph capture and replay,
// sampled outcomes, per-launch profiling, index maps and pass descriptions.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "owqs_internal.h"

namespace owqs {

struct RunCache {
  int device = -1;
  void* buf[2] = {nullptr, nullptr};
  size_t buf_bytes = 0;
  void* in_stage = nullptr;
  size_t in_bytes = 0;
  void* out_stage = nullptr;
  size_t out_bytes = 0;
  double* norms = nullptr;
  size_t nnorms = 0;
  double* partials = nullptr;
  size_t npartials = 0;
  unsigned int* counter = nullptr;
  // device-drawn outcomes: [seed u64][w1: 2K doubles][domains: u32][outcomes: K bytes]
  void* samp = nullptr;
  size_t samp_bytes = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::string gkey;
  void* small_dev = nullptr;  // the passes of a single-block run, and their host copy
  size_t small_bytes = 0;
  std::vector<unsigned char> small_host;
  std::vector<double> h_norms;
  uint32_t last_launches = 0;
  // asynchronous runs (owqs_run_async / owqs_wait), at most two in flight,
  // completed in order
  struct Pending {
    cudaEvent_t done = nullptr;  // the run's output copy and slot read-back have finished
    double* host = nullptr;      // pinned: the K + 2 norm slots, then the error flag
    double* snap = nullptr;      // device: the same, copied right after the final pass
    size_t cap = 0;              // doubles in host and snap
    owqs_run_opts opts{};
    std::vector<PassDesc> passes;
    std::vector<char> in_group;
    std::vector<int> outcome_of_pass;
    bool has_input = false;
  } pend[2];
  int pend_head = 0, pend_count = 0, last_slot = -1;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t in_free = nullptr;  // the last asynchronous run's launches that read in_stage are done
  cudaEvent_t h2d_done = nullptr, ready = nullptr;
  bool in_free_set = false;
  uint32_t last_sample_path = 0;   // OWQS_SAMPLE_* of the last sampled run
  uint32_t last_guessed = 0;       // a whole-run guess ran first
  uint32_t last_relaunches = 0;    // checked launches: launches run again after a corrected outcome
  uint32_t last_checks = 0;        // checked launches: host checks (one per launch that measures)
  void* arena = nullptr;  // separate sub-states: every component array, at planned offsets
  size_t arena_bytes = 0;
  uint32_t last_components = 0;  // separate sub-states: components of the last run (0: one array)
  uint64_t last_peak_bytes = 0;  // device bytes of the last run's live arrays at their peak

  ~RunCache() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (device >= 0 && cur != device) cudaSetDevice(device);
    for (Pending& q : pend) {
      if (q.done) {
        cudaEventSynchronize(q.done);
        cudaEventDestroy(q.done);
      }
      if (q.host) cudaFreeHost(q.host);
      if (q.snap) cudaFree(q.snap);
    }
    for (cudaEvent_t ev : {in_free, h2d_done, ready})
      if (ev) cudaEventDestroy(ev);
    for (cudaStream_t cs : {copy_in, copy_out})
      if (cs) cudaStreamDestroy(cs);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap) cudaStreamDestroy(cap);
    for (void* p : {buf[0], buf[1], in_stage, out_stage, (void*)norms, (void*)partials, (void*)counter, samp,
                    small_dev, arena})
      if (p) cudaFree(p);
    if (device >= 0 && cur >= 0 && cur != device) cudaSetDevice(cur);
  }
};

static owqs_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error
  return set_error(e == cudaErrorMemoryAllocation ? OWQS_ERR_OOM : OWQS_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

static owqs_status ensure_buf(void*& p, size_t& have, size_t need, const char* what) {
  if (need <= have && p) return OWQS_OK;
  if (p) {
    cudaFree(p);
    p = nullptr;
    have = 0;
  }
  size_t freeb = 0, total = 0;
  if (cudaMemGetInfo(&freeb, &total) == cudaSuccess && need > freeb)
    return set_error(OWQS_ERR_OOM, std::string(what) + ": needs " + std::to_string(need) +
                                       " bytes, device has " + std::to_string(freeb) + " free");
  cudaError_t e = cudaMalloc(&p, need);
  if (e != cudaSuccess) {
    p = nullptr;
    return cuda_fail(e, what);
  }
  have = need;
  return OWQS_OK;
}

static owqs_status get_cache(Pattern& p, RunCache*& rc) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (!p.cache) {
    p.cache = std::make_shared<RunCache>();
    p.cache->device = dev;
  }
  if (p.cache->device != dev) return set_error(OWQS_ERR_ARG, "pattern handle used on another device");
  rc = p.cache.get();
  return OWQS_OK;
}

// ---------------------------------------------------------------------------
// outcome sources
// ---------------------------------------------------------------------------
struct FixedSource : OutcomeSource {
  const Pattern& p;
  const uint8_t* bits;  // nullptr => all zero
  FixedSource(const Pattern& pp, const uint8_t* b) : p(pp), bits(b) {}
  bool known_upfront(std::vector<int8_t>& o) override {
    for (size_t k = 0; k < p.meas_qubit.size(); ++k) o[p.meas_qubit[k]] = bits ? (int8_t)(bits[k] & 1u) : 0;
    return true;
  }
  int decide(const PassDesc& d) override { return bits ? (bits[d.meas_k] & 1u) : 0; }
};

// ---------------------------------------------------------------------------
// launch list
// ---------------------------------------------------------------------------
struct Item {
  int type = 0;  // 0 pass, 1 norm, 3 device-drawn outcome, 4 pass group, 5 factor join
  PassParams P;
  KronParams Kp;
  GroupParams G;
  DecideParams D;
  LaunchPlan L;
  const void* norm_in = nullptr;
  uint64_t norm_n = 0;
  int norm_slot = 0;
};

class Runner {
 public:
  Runner(Pattern& p, RunCache& rc, int dtype, int mode, cudaStream_t s)
      : p_(p), rc_(rc), dtype_(dtype), mode_(mode), stream_(s) {
    K_ = (int)p.meas_qubit.size();
    thresh_ = dtype == OWQS_C128 ? 1e-24 : 1e-12;
  }

  bool immediate = false;
  int vdiag = 0;  // virtual diagonal input over 2 * vdiag bits (recognition)
  std::vector<Item> items;
  std::vector<char> in_group;  // per measurement: not the first of a pass group
  owqs_status err = OWQS_OK;

  // in0: the input array (nullptr: virtual input) of in_elems amplitudes;
  // out_final: the output array of out_elems amplitudes
  void begin(const void* in0, uint64_t in_elems, void* out_final, uint64_t out_elems) {
    cur_in_ = in0;
    out_final_ = out_final;
    in0_ = in0;
    in0_cap_ = in_elems;
    out_cap_ = out_elems;
    buf_cap_ = rc_.buf_bytes / (dtype_ == OWQS_C64 ? 8 : 16);
    pass_i_ = 0;
    sel_ = 0;
    prev_slot_ = -1;
    if (in0) {  // input norm: OWQS divides by it, EOWQS checks against it
      Item it;
      it.type = 1;
      it.norm_in = in0;
      it.norm_n = in_elems;
      it.norm_slot = 0;
      it.L.grid = (int)std::min<uint64_t>((in_elems + kBlock - 1) / kBlock, (uint64_t)max_grid());
      it.L.kind = KK_NORM;
      it.L.bytes = (double)in_elems * (dtype_ == OWQS_C64 ? 8.0 : 16.0);
      issue(it);
      if (mode_ == OWQS_MODE_OWQS) prev_slot_ = 0;
    }
  }

  void measure(const PassDesc& d) {
    Item it;
    plan_pass(d, dtype_, cur_in_ == nullptr, it.P, it.L);
    fill_common(it.P);
    if (!cur_in_) it.P.vdiag = vdiag;
    it.P.in = cur_in_;
    it.P.out = rc_.buf[sel_];
    it.P.in_cap = in_cap();
    it.P.out_cap = buf_cap_;
    sel_ ^= 1;
    it.P.norm_in = prev_slot_;
    it.P.norm_out = mode_ == OWQS_MODE_OWQS ? pass_i_ + 1 : -1;
    it.P.w1dev = w1dev_;
    it.L.meas = 1;
    issue(it);
    cur_in_ = it.P.out;
    prev_slot_ = it.P.norm_out;
    in_group.push_back(0);
    ++pass_i_;
  }

  // measure pass whose (-1)^s e^{-i theta} is read from device memory
  // (written by a decide item just before it)
  void measure_dev(const PassDesc& d, const double* w1) {
    w1dev_ = w1;
    measure(d);
    w1dev_ = nullptr;
  }

  // draw the outcome of the next measurement on the device
  void decide(const DecideParams& D) {
    Item it;
    it.type = 3;
    it.D = D;
    it.L.kind = KK_DECIDE;
    it.L.bytes = 0.0;
    issue(it);
  }

  // a group of k consecutive measure passes as one sweep: slots pass_i+1 ..
  // pass_i+k get the running products of the group's probabilities
  void measure_group(const GroupParams& G, const LaunchPlan& L) {
    Item it;
    it.type = 4;
    it.G = G;
    it.L = L;
    it.L.meas = G.k;
    it.G.norms = rc_.norms;
    it.G.partials = rc_.partials;
    it.G.counter = rc_.counter;
    it.G.errflag = rc_.counter + 1;
    it.G.thresh = thresh_;
    it.G.in = cur_in_;
    it.G.out = rc_.buf[sel_];
    it.G.in_cap = in_cap();
    it.G.out_cap = buf_cap_;
    sel_ ^= 1;
    it.G.norm_in = prev_slot_;
    it.G.norm_out = mode_ == OWQS_MODE_OWQS ? pass_i_ + 1 : -1;
    issue(it);
    cur_in_ = it.G.out;
    prev_slot_ = mode_ == OWQS_MODE_OWQS ? pass_i_ + G.k : -1;
    in_group.push_back(0);
    for (int j = 1; j < G.k; ++j) in_group.push_back(1);
    pass_i_ += G.k;
  }

  // Explicit-array forms (separate sub-states): the caller supplies the
  // arrays, their extents in amplitudes and the norm slots.
  void measure_at(const PassDesc& d, const void* in, uint64_t in_cap, void* out, uint64_t out_cap, int norm_in,
                  int norm_out) {
    Item it;
    plan_pass(d, dtype_, in == nullptr, it.P, it.L);
    fill_common(it.P);
    it.P.in = in;
    it.P.out = out;
    it.P.in_cap = in_cap;
    it.P.out_cap = out_cap;
    it.P.norm_in = norm_in;
    it.P.norm_out = norm_out;
    it.L.meas = 1;
    issue(it);
    in_group.push_back(0);
    ++pass_i_;
  }
  void group_at(const GroupParams& G, const LaunchPlan& L, const void* in, uint64_t in_cap, void* out,
                uint64_t out_cap, int norm_in, int norm_out) {
    Item it;
    it.type = 4;
    it.G = G;
    it.L = L;
    it.L.meas = G.k;
    it.G.norms = rc_.norms;
    it.G.partials = rc_.partials;
    it.G.counter = rc_.counter;
    it.G.errflag = rc_.counter + 1;
    it.G.thresh = thresh_;
    it.G.in = in;
    it.G.out = out;
    it.G.in_cap = in_cap;
    it.G.out_cap = out_cap;
    it.G.norm_in = norm_in;
    it.G.norm_out = norm_out;
    issue(it);
    in_group.push_back(0);
    for (int j = 1; j < G.k; ++j) in_group.push_back(1);
    pass_i_ += G.k;
  }
  // out = a (x) b, a's n_a qubits low: each factor divided by the square root
  // of its norm slot (-1: taken as normalised)
  void join_at(const void* a, int n_a, int norm_a, const void* b, int n_b, int norm_b, void* out, uint64_t out_cap) {
    Item it;
    it.type = 5;
    it.Kp.in = a;
    it.Kp.out = out;
    it.Kp.phi = b;
    it.Kp.norms = rc_.norms;
    it.Kp.n_in = n_a;
    it.Kp.q = n_b;
    it.Kp.norm_in = norm_a;
    it.Kp.fnorm = norm_b;
    it.Kp.in_cap = 1ull << n_a;
    it.Kp.out_cap = out_cap;
    it.Kp.errflag = rc_.counter + 1;
    it.L.kind = KK_KRON;
    it.L.bytes = (std::ldexp(1.0, n_a) + std::ldexp(1.0, n_b) + std::ldexp(1.0, n_a + n_b)) *
                 (dtype_ == OWQS_C64 ? 8.0 : 16.0);
    issue(it);
  }
  void final_at(const PassDesc& d, const void* in, uint64_t in_cap, int norm_in) {
    Item it;
    plan_pass(d, dtype_, in == nullptr, it.P, it.L);
    fill_common(it.P);
    it.P.in = in;
    it.P.out = out_final_;
    it.P.in_cap = in_cap;
    it.P.out_cap = out_cap_;
    it.P.norm_in = norm_in;
    it.P.norm_out = K_ + 1;
    issue(it);
  }
  int pass_index() const { return pass_i_; }

  // join of an input factor (product input): its norm into slot fslot, then
  // the tensor product with the live array (normalised), the factor's qubits
  // becoming the top bits
  void join(const PassDesc& d, const void* phi, int fslot) {
    Item nm;
    nm.type = 1;
    nm.norm_in = phi;
    nm.norm_n = 1ull << d.r;
    nm.norm_slot = fslot;
    nm.L.grid = (int)std::min<uint64_t>((nm.norm_n + kBlock - 1) / kBlock, (uint64_t)max_grid());
    nm.L.kind = KK_NORM;
    nm.L.bytes = std::ldexp(1.0, d.r) * (dtype_ == OWQS_C64 ? 8.0 : 16.0);
    issue(nm);
    Item it;
    it.type = 5;
    it.Kp.in = cur_in_;
    it.Kp.out = rc_.buf[sel_];
    it.Kp.in_cap = in_cap();
    it.Kp.out_cap = buf_cap_;
    it.Kp.errflag = rc_.counter + 1;
    sel_ ^= 1;
    it.Kp.phi = phi;
    it.Kp.norms = rc_.norms;
    it.Kp.n_in = d.n_in;
    it.Kp.q = d.r;
    it.Kp.norm_in = prev_slot_;
    it.Kp.fnorm = fslot;
    it.L.kind = KK_KRON;
    it.L.bytes = ((cur_in_ ? std::ldexp(1.0, d.n_in) : 0.0) + std::ldexp(1.0, d.n_out)) *
                 (dtype_ == OWQS_C64 ? 8.0 : 16.0);
    issue(it);
    cur_in_ = it.Kp.out;
    prev_slot_ = -1;  // the joined array is normalised
  }

  // the array the next launch reads is materialised (not the virtual |+> input)
  bool real_input() const { return cur_in_ != nullptr; }

  // both outcome probabilities of the next measurement into slots
  // prob_slot(i), prob_slot(i)+1 (sampled outcomes)
  int prob(const PassDesc& d) {
    Item it;
    plan_pass(d, dtype_, cur_in_ == nullptr, it.P, it.L);
    fill_common(it.P);
    // passes the bulk-copy kernel takes read their probabilities the same way
    it.L.kind = it.L.kind == KK_TMA ? KK_PROB_TMA : KK_PROB;
    it.L.grid = (int)std::min<uint64_t>(((1ull << d.n_out) + kBlock - 1) / kBlock, (uint64_t)max_grid());
    it.L.bytes = (cur_in_ ? std::ldexp(1.0, d.n_in) : 0.0) * (dtype_ == OWQS_C64 ? 8.0 : 16.0);
    it.P.in = cur_in_;
    it.P.out = nullptr;
    it.P.in_cap = in_cap();
    it.P.norm_in = prev_slot_;
    it.P.norm_out = K_ + 2 + 2 * pass_i_;
    it.P.edev = edev_;
    issue(it);
    return it.P.norm_out;
  }

  // probability pass whose e^{-i theta} is read from device memory
  int prob_dev(const PassDesc& d, const double* e) {
    edev_ = e;
    const int slot = prob(d);
    edev_ = nullptr;
    return slot;
  }

  void final_pass(const PassDesc& d) {
    Item it;
    plan_pass(d, dtype_, cur_in_ == nullptr, it.P, it.L);
    fill_common(it.P);
    if (!cur_in_) it.P.vdiag = vdiag;
    it.P.in = cur_in_;
    it.P.out = out_final_;
    it.P.in_cap = in_cap();
    it.P.out_cap = out_cap_;
    it.P.norm_in = mode_ == OWQS_MODE_OWQS ? prev_slot_ : -1;
    it.P.norm_out = K_ + 1;
    issue(it);
  }

  owqs_status launch(const Item& it, cudaStream_t s) {
    cudaError_t e;
    if (it.type == 5)
      e = launch_kron(it.Kp, dtype_, s);
    else if (it.type == 4)
      e = launch_group(it.G, dtype_, s);
    else if (it.type == 3)
      e = launch_decide(it.D, s);
    else if (it.type == 1)
      e = launch_norm(it.norm_in, it.norm_n, dtype_, rc_.norms, it.norm_slot, rc_.partials, rc_.counter,
                      it.L.grid, s);
    else
      e = launch_pass(it.P, it.L, dtype_, s);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return OWQS_OK;
  }

 private:
  // elements of the array the next launch reads (0: virtual input)
  uint64_t in_cap() const { return cur_in_ == nullptr ? 0 : (cur_in_ == in0_ ? in0_cap_ : buf_cap_); }
  void fill_common(PassParams& P) {
    P.norms = rc_.norms;
    P.partials = rc_.partials;
    P.counter = rc_.counter;
    P.errflag = rc_.counter + 1;
    P.thresh = thresh_;
  }
  void issue(const Item& it) {
    if (immediate) {
      if (err == OWQS_OK) err = launch(it, stream_);
    } else {
      items.push_back(it);
    }
  }

  Pattern& p_;
  RunCache& rc_;
  int dtype_, mode_;
  cudaStream_t stream_;
  int K_ = 0;
  double thresh_;
  const void* cur_in_ = nullptr;
  void* out_final_ = nullptr;
  int pass_i_ = 0;
  int sel_ = 0;  // ping-pong buffer the next launch writes
  const double* w1dev_ = nullptr;
  const double* edev_ = nullptr;
  int prev_slot_ = -1;
  const void* in0_ = nullptr;
  uint64_t in0_cap_ = 0, out_cap_ = 0, buf_cap_ = 0;  // buffer extents (bounds-checked builds)
};

// next uniform in [0, 1) of a splitmix64 stream: the state advances by the
// golden-ratio increment, the finaliser mixes it, the top 53 bits are kept
static double splitmix_uniform(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// sampled outcomes: the previous measure pass is launched, then the two
// probabilities of this measurement are reduced and read back, and the
// outcome is 0 iff u <= prob_0 with u the next splitmix64 uniform
struct SampledSource : OutcomeSource {
  Runner& R;
  RunCache& rc;
  cudaStream_t s;
  uint64_t state;
  bool have_pending = false;
  PassDesc pending;
  SampledSource(Runner& r, RunCache& c, cudaStream_t st, uint64_t seed) : R(r), rc(c), s(st), state(seed) {}
  double uniform() { return splitmix_uniform(state); }
  void flush() {
    if (have_pending) {
      R.measure(pending);
      have_pending = false;
    }
  }
  int decide(const PassDesc& d) override {
    flush();
    const int slot = R.prob(d);
    if (R.err != OWQS_OK) return -1;
    double pp[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(pp, rc.norms + slot, sizeof(pp), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cuda_fail(e, "reading outcome probabilities");
      return -1;
    }
    const int o = uniform() <= pp[0] ? 0 : 1;
    pending = d;
    pending.outcome = o;
    pending.w1re = o ? -d.ere : d.ere;
    pending.w1im = o ? -d.eim : d.eim;
    have_pending = true;
    return o;
  }
};

static std::string graph_key(const Pattern& p, const owqs_run_opts* o, const void* in, const void* out,
                             const uint8_t* outcomes) {
  std::string k;
  k.reserve(64 + p.meas_qubit.size());
  auto add = [&](const void* v, size_t n) { k.append(reinterpret_cast<const char*>(v), n); };
  add(&o->dtype, 4);
  add(&o->mode, 4);
  add(&o->policy, 4);
  add(&in, sizeof(in));
  add(&out, sizeof(out));
  const void* pp = &p;
  add(&pp, sizeof(pp));
  uint64_t h = 1469598103934665603ull;  // active order fingerprint (FNV-1a)
  for (uint32_t i : p.active) h = (h ^ i) * 1099511628211ull;
  add(&h, 8);
  if (o->policy == OWQS_OUTCOME_FORCED && outcomes) add(outcomes, p.meas_qubit.size());
  add(&o->flags, 4);
  const int cap = test_grid_cap();
  add(&cap, sizeof(cap));
  const int m4 = group_m4_min_width();  // the launch plan depends on it
  add(&m4, sizeof(m4));
  return k;
}

// product input: the input qubits grouped into factors and each factor's
// amplitudes (device)
struct ProductInput {
  std::vector<std::vector<uint32_t>> qubits;
  std::vector<const void*> vecs;
};

// A forced or zero-outcome run whose arrays all fit 2^kSmallLog amplitudes,
// with at most kSmallMaxPasses passes, runs in one single-block kernel
// (k_small) instead of one kernel per pass.
static bool small_run_ok(const std::vector<PassDesc>& passes) {
  if (passes.empty() || passes.size() > (size_t)kSmallMaxPasses) return false;
  for (const PassDesc& d : passes)
    if (d.kind == 2 || d.n_in > kSmallLog || d.n_out > kSmallLog) return false;
  return true;
}

// What the launch for passes[i] is: a factor join, the final pass, a group
// of k measure passes (k >= 2; reads a materialised input array or the
// virtual |+> input, not the diagonal input of a unitary) or a single
// measure pass.  The run driver and owqs_describe_launches both use it.
enum { LAUNCH_SINGLE = 0, LAUNCH_GROUP = 1, LAUNCH_FINAL = 2, LAUNCH_JOIN = 3 };
static int decide_launch(const std::vector<PassDesc>& passes, size_t i, int dtype, bool real_input, bool diag_input,
                         GroupParams& G, LaunchPlan& GL, int& k) {
  const PassDesc& d = passes[i];
  k = 1;
  if (d.kind == 2) return LAUNCH_JOIN;
  if (d.kind != 0) return LAUNCH_FINAL;
  if ((real_input || !diag_input) && group_enabled()) {
    const int g = plan_group(passes, i, dtype, G, GL, !real_input);
    if (g >= 2) {
      k = g;
      return LAUNCH_GROUP;
    }
  }
  return LAUNCH_SINGLE;
}

struct Prepared {
  std::vector<PassDesc> passes;
  const void* in_dev = nullptr;
  void* out_dev = nullptr;
  size_t amp = 8;
  uint64_t in_elems = 0, out_elems = 0;
};

static owqs_status prepare(Pattern& p, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                           const uint8_t* outcomes, RunCache*& rc, Prepared& pr, bool sampled,
                           const ProductInput* prod = nullptr) {
  if (!o || !psi_out) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (o->dtype > OWQS_C128 || o->mode > OWQS_MODE_EOWQS || o->policy > OWQS_OUTCOME_ZERO || o->io > OWQS_IO_HOST)
    return set_error(OWQS_ERR_ARG, "bad option value");
  if (o->policy == OWQS_OUTCOME_FORCED && !outcomes && !p.meas_qubit.empty())
    return set_error(OWQS_ERR_ARG, "forced outcomes need the outcomes array");
  pr.amp = o->dtype == OWQS_C64 ? 8 : 16;
  pr.in_elems = 1ull << p.inputs.size();
  pr.out_elems = 1ull << p.outputs.size();
  if (o->io == OWQS_IO_DEVICE) {  // refused before any device work
    if (((uintptr_t)psi_in % 16) || ((uintptr_t)psi_out % 16))
      return set_error(OWQS_ERR_ARG, "device vectors must be 16-byte aligned");
    if (psi_in && byte_ranges_overlap(psi_in, pr.in_elems * pr.amp, psi_out, pr.out_elems * pr.amp))
      return set_error(OWQS_ERR_ARG, "psi_in and psi_out must not overlap");
  }
  owqs_status st = get_cache(p, rc);
  if (st != OWQS_OK) return st;
  if (!sampled) {  // sampled runs compile while they execute
    FixedSource src(p, o->policy == OWQS_OUTCOME_ZERO ? nullptr : outcomes);
    st = compile_schedule(p, o->mode, src, pr.passes, nullptr, prod ? &prod->qubits : nullptr);
    if (st != OWQS_OK) return st;
  }
  const int K = (int)p.meas_qubit.size();
  const size_t nfac = prod ? prod->qubits.size() : 0;
  st = ensure_buf((void*&)rc->norms, rc->nnorms, sizeof(double) * (3 * (size_t)K + 8 + nfac), "norm slots");
  if (st == OWQS_OK)
    st = ensure_buf((void*&)rc->partials, rc->npartials, sizeof(double) * kGroupMax * (size_t)max_grid(), "partials");
  if (st == OWQS_OK && !rc->counter) {  // [0] finished-block counter, [1] error flag
    cudaError_t e = cudaMalloc(&rc->counter, 2 * sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_fail(e, "counter");
    e = cudaMemset(rc->counter, 0, 2 * sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_fail(e, "counter");
  }
  if (st != OWQS_OK) return st;
  if (o->io == OWQS_IO_HOST) {
    if (psi_in) {
      st = ensure_buf(rc->in_stage, rc->in_bytes, pr.in_elems * pr.amp, "input staging");
      if (st != OWQS_OK) return st;
      pr.in_dev = rc->in_stage;
    }
    st = ensure_buf(rc->out_stage, rc->out_bytes, pr.out_elems * pr.amp, "output staging");
    if (st != OWQS_OK) return st;
    pr.out_dev = rc->out_stage;
  } else {
    pr.in_dev = psi_in;
    pr.out_dev = psi_out;
  }
  return OWQS_OK;
}

// ---------------------------------------------------------------------------
// separate sub-states: launch records, arena plan, items
// ---------------------------------------------------------------------------
namespace {
// First-fit plan of byte ranges in one arena (256-byte aligned).
struct ArenaPlan {
  std::vector<std::pair<size_t, size_t>> free_;  // (offset, length), sorted by offset
  size_t end = 0;
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (size_t i = 0; i < free_.size(); ++i)
      if (free_[i].second >= bytes) {
        const size_t off = free_[i].first;
        free_[i].first += bytes;
        free_[i].second -= bytes;
        if (free_[i].second == 0) free_.erase(free_.begin() + i);
        return off;
      }
    const size_t off = end;
    end += bytes;
    return off;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(off, (size_t)0));
    it = free_.insert(it, {off, bytes});
    const size_t i = (size_t)(it - free_.begin());
    if (i + 1 < free_.size() && free_[i].first + free_[i].second == free_[i + 1].first) {
      free_[i].second += free_[i + 1].second;
      free_.erase(free_.begin() + i + 1);
    }
    if (i > 0 && free_[i - 1].first + free_[i - 1].second == free_[i].first) {
      free_[i - 1].second += free_[i].second;
      free_.erase(free_.begin() + i);
    }
  }
};
constexpr long long kUserInput = -2;  // the caller's input vector (not in the arena)
struct CompLaunch {
  int type = 0;  // 0 single measure pass, 1 pass group, 2 join, 3 final pass
  PassDesc d;
  GroupParams G;
  LaunchPlan GL;
  long long in_off = -1, in2_off = -1, out_off = -1;  // -1: no array (virtual |+> input) / the caller's output
  uint64_t in_cap = 0, in2_cap = 0, out_cap = 0;
  int n_a = 0, n_b = 0;
  int comp = -1, comp2 = -1;
};
}  // namespace

// A default run takes separate sub-states when they at least halve the
// amplitudes the passes move and need no more memory than one array.
static bool use_substates(const CompSchedule& cs) {
  return 2.0 * cs.work <= cs.single_work && cs.peak_amps <= cs.single_amps;
}

// Walk a component schedule: measure passes of one component that follow
// each other form pass groups as in a one-array run; every array gets an
// arena range while it is live.  Fills `launches`, the arena size and the
// measure passes in launch order (the order of the norm slots).
static owqs_status plan_components(const CompSchedule& cs, int dtype, size_t amp, bool real_input, uint64_t in_elems,
                                   std::vector<CompLaunch>& launches, size_t& arena_bytes,
                                   std::vector<PassDesc>& order) {
  ArenaPlan ap;
  std::vector<long long> off(cs.ncomp, -1);  // arena offset of each component's array
  std::vector<uint64_t> cap(cs.ncomp, 0);
  if (cs.input_comp >= 0 && real_input) {
    off[cs.input_comp] = kUserInput;
    cap[cs.input_comp] = in_elems;
  }
  auto release = [&](int c) {
    if (off[c] >= 0) ap.release((size_t)off[c], cap[c] * amp);
    off[c] = -1;
    cap[c] = 0;
  };
  order.clear();
  for (size_t i = 0; i < cs.ops.size();) {
    const CompOp& op = cs.ops[i];
    if (op.kind == 0) {
      std::vector<PassDesc> chain;
      size_t j = i;
      for (; j < cs.ops.size() && cs.ops[j].kind == 0 && cs.ops[j].a == op.a; ++j) chain.push_back(cs.ops[j].d);
      for (size_t q = 0; q < chain.size();) {
        CompLaunch L;
        L.comp = op.a;
        int k = 1;
        const bool real = off[op.a] != -1;
        if (real && group_enabled()) {
          const int g = plan_group(chain, q, dtype, L.G, L.GL, false);
          if (g >= 2) k = g;
        } else if (!real && group_enabled()) {
          const int g = plan_group(chain, q, dtype, L.G, L.GL, true);
          if (g >= 2) k = g;
        }
        L.type = k >= 2 ? 1 : 0;
        L.d = chain[q];
        L.in_off = off[op.a];
        L.in_cap = cap[op.a];
        L.out_cap = 1ull << chain[q + k - 1].n_out;
        L.out_off = (long long)ap.alloc(L.out_cap * amp);
        release(op.a);
        off[op.a] = L.out_off;
        cap[op.a] = L.out_cap;
        for (int t = 0; t < k; ++t) order.push_back(chain[q + t]);
        launches.push_back(std::move(L));
        q += (size_t)k;
      }
      i = j;
    } else if (op.kind == 1) {
      CompLaunch L;
      L.type = 2;
      L.comp = op.a;
      L.comp2 = op.b;
      L.n_a = op.n_a;
      L.n_b = op.n_b;
      L.in_off = off[op.a];
      L.in_cap = cap[op.a];
      L.in2_off = off[op.b];
      L.in2_cap = cap[op.b];
      L.out_cap = 1ull << (op.n_a + op.n_b);
      L.out_off = (long long)ap.alloc(L.out_cap * amp);
      release(op.a);
      release(op.b);
      off[op.a] = L.out_off;
      cap[op.a] = L.out_cap;
      launches.push_back(std::move(L));
      ++i;
    } else {
      CompLaunch L;
      L.type = 3;
      L.comp = op.a;
      L.d = op.d;
      L.in_off = off[op.a];
      L.in_cap = cap[op.a];
      order.push_back(op.d);
      launches.push_back(std::move(L));
      ++i;
    }
  }
  arena_bytes = std::max<size_t>(ap.end, 256);
  return OWQS_OK;
}

// Issue the launch records as runner items: arena offsets become pointers,
// every component keeps the norm slot that its next launch divides by.
static void issue_components(const std::vector<CompLaunch>& launches, int ncomp, int input_comp, bool owqs,
                             bool real_input, const void* in_dev, char* arena, Runner& R) {
  std::vector<int> prev(ncomp, -1);
  if (input_comp >= 0 && real_input && owqs) prev[input_comp] = 0;  // the input's norm (slot 0)
  auto ptr = [&](long long off) -> const void* {
    return off == kUserInput ? in_dev : (off >= 0 ? (const void*)(arena + off) : nullptr);
  };
  for (const CompLaunch& L : launches) {
    if (L.type == 0 || L.type == 1) {
      const int slot = owqs ? R.pass_index() + 1 : -1;
      void* out = arena + L.out_off;
      if (L.type == 0) R.measure_at(L.d, ptr(L.in_off), L.in_cap, out, L.out_cap, prev[L.comp], slot);
      else R.group_at(L.G, L.GL, ptr(L.in_off), L.in_cap, out, L.out_cap, prev[L.comp], slot);
      if (owqs) prev[L.comp] = R.pass_index();
    } else if (L.type == 2) {
      R.join_at(ptr(L.in_off), L.n_a, prev[L.comp], ptr(L.in2_off), L.n_b, prev[L.comp2], arena + L.out_off,
                L.out_cap);
      prev[L.comp] = -1;  // the tensor product of normalised factors
    } else {
      R.final_at(L.d, ptr(L.in_off), L.in_cap, owqs ? prev[L.comp] : -1);
    }
  }
}

static owqs_status ensure_pingpong(RunCache* rc, size_t elems, size_t amp) {
  const size_t need = std::max<size_t>(elems, 1) * amp;
  if (rc->buf_bytes >= need && rc->buf[0] && rc->buf[1]) return OWQS_OK;
  size_t have0 = rc->buf_bytes, have1 = rc->buf_bytes;
  if (rc->gexec) {  // graphs hold the old buffer addresses
    cudaGraphExecDestroy(rc->gexec);
    rc->gexec = nullptr;
    rc->gkey.clear();
  }
  owqs_status st = ensure_buf(rc->buf[0], have0, need, "state buffer");
  if (st == OWQS_OK) st = ensure_buf(rc->buf[1], have1, need, "state buffer");
  if (st != OWQS_OK) return st;
  rc->buf_bytes = need;
  return OWQS_OK;
}

// The run's result from its norm slots (h_norms: K + 2 values read back from
// the device) and its error flag: probabilities, outcomes of a sampled run,
// the impossible-branch and EOWQS checks.
static owqs_status interpret_run(Pattern& p, const owqs_run_opts* o, const std::vector<double>& h_norms,
                                 unsigned int flag, const std::vector<PassDesc>& passes, uint8_t* outcomes,
                                 double* probs, const std::vector<int>& outcome_of_pass, bool has_input, int vdiag,
                                 double* frob2, const std::vector<char>& in_group) {
  const int K = (int)p.meas_qubit.size();
  if (flag) {  // a device-side wait gave up (bit 0; blocks skipped the reduction) or a bounds check failed (bit 1)
    if (flag & 2u)
      return set_error(OWQS_ERR_CUDA, "a kernel access fell outside its buffer (bounds-checked build); results are invalid");
    return set_error(OWQS_ERR_TIMEOUT, "a device-side wait in a pass kernel gave up; results are invalid");
  }
  const double thresh = o->dtype == OWQS_C128 ? 1e-24 : 1e-12;
  owqs_status st = OWQS_OK;
  int mi = 0;
  for (const PassDesc& d : passes) {
    if (d.kind != 0) continue;
    double pv = o->mode == OWQS_MODE_OWQS ? h_norms[mi + 1] : 0.5;
    if (o->mode == OWQS_MODE_OWQS && (size_t)mi < in_group.size() && in_group[mi]) {
      // later measurement of a pass group: its slot holds the running product of the group's probabilities
      const double first = h_norms[mi];
      pv = first > 0.0 ? pv / first : 0.0;
    }
    if (probs) probs[d.meas_k] = pv;
    if (outcomes && o->policy != OWQS_OUTCOME_FORCED) outcomes[d.meas_k] = (uint8_t)outcome_of_pass[mi];
    if (o->mode == OWQS_MODE_OWQS && !(pv >= thresh) && st == OWQS_OK)
      st = set_error(OWQS_ERR_IMPOSSIBLE_BRANCH, "outcome of measurement " + std::to_string(d.meas_k) +
                                                      " has probability " + std::to_string(pv));
    ++mi;
  }
  if (vdiag > 0) {  // recognition: |U|_F^2 / 2^|I| is 1 for an isometry; reported, not checked
    if (frob2) *frob2 = h_norms[K + 1] / std::ldexp(1.0, vdiag);
    return st;
  }
  if (o->mode == OWQS_MODE_EOWQS) {
    const double nin = has_input ? h_norms[0] : 1.0;
    const double nout = h_norms[K + 1];
    const double tol = o->dtype == OWQS_C128 ? 1e-10 : 1e-4;
    if (!(std::fabs(nout - nin) <= tol * std::max(nin, 1e-300)))
      st = set_error(OWQS_ERR_NOT_DETERMINISTIC,
                     "EOWQS output norm " + std::to_string(nout) + " differs from the input norm " + std::to_string(nin));
  }
  return st;
}

static owqs_status finish(Pattern& p, const owqs_run_opts* o, RunCache* rc, const Prepared& pr,
                          cudaStream_t s, uint8_t* outcomes, double* probs, const std::vector<int>& outcome_of_pass,
                          bool has_input, int vdiag, double* frob2, const std::vector<char>& in_group) {
  const int K = (int)p.meas_qubit.size();
  rc->h_norms.assign((size_t)K + 2, 0.0);
  unsigned int flag = 0;
  cudaError_t e = cudaMemcpyAsync(rc->h_norms.data(), rc->norms, sizeof(double) * (K + 2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, rc->counter + 1, sizeof(flag), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "run");
  if (flag) {
    cudaMemsetAsync(rc->counter, 0, 2 * sizeof(unsigned int), s);
    cudaStreamSynchronize(s);
  }
  return interpret_run(p, o, rc->h_norms, flag, pr.passes, outcomes, probs, outcome_of_pass, has_input, vdiag, frob2,
                       in_group);
}

// Launch a runner's item list: from a CUDA graph cached under `key` (captured
// on first use) or one launch at a time.
static owqs_status replay(RunCache* rc, Runner& R, const std::string& key, bool use_graph, cudaStream_t s) {
  if (!use_graph) {
    for (const Item& it : R.items) {
      owqs_status st = R.launch(it, s);
      if (st != OWQS_OK) return st;
    }
    return OWQS_OK;
  }
  if (!rc->gexec || key != rc->gkey) {
    if (rc->gexec) {
      cudaGraphExecDestroy(rc->gexec);
      rc->gexec = nullptr;
    }
    if (!rc->cap) {
      cudaError_t e = cudaStreamCreateWithFlags(&rc->cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    }
    cudaError_t e = cudaStreamBeginCapture(rc->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    owqs_status st = OWQS_OK;
    for (const Item& it : R.items) {
      st = R.launch(it, rc->cap);
      if (st != OWQS_OK) break;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(rc->cap, &g);
    if (st != OWQS_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&rc->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      rc->gexec = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
    rc->gkey = key;
  }
  cudaError_t e = cudaGraphLaunch(rc->gexec, s);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return OWQS_OK;
}

// Sampled outcomes without a host round trip per measurement.  Possible when
// no X or Z command with a signal comes before the last measurement (so the
// measure passes' sign forms and X masks do not depend on outcomes; true of
// every standard-form pattern): per measurement a probability pass, k_decide
// (draws the outcome, writes (-1)^s e^{-i theta} and the next measurement's
// e^{-i theta}) and the measure pass reading them, all in one graph.  The
// outcomes are read back once, and the final pass, whose corrections depend
// on them, is compiled and launched afterwards.
static bool masks_outcome_free(const Pattern& p) {
  size_t last_m = 0;
  for (size_t i = 0; i < p.active.size(); ++i)
    if (p.cmds[p.active[i]].kind == OWQS_CMD_M) last_m = i;
  for (size_t i = 0; i < last_m; ++i) {
    const Cmd& c = p.cmds[p.active[i]];
    if ((c.kind == OWQS_CMD_X || c.kind == OWQS_CMD_Z) && !c.sdom.empty()) return false;
  }
  return true;
}

static owqs_status sample_on_device(Pattern& p, const owqs_run_opts* o, RunCache* rc, Prepared& pr,
                                    const std::vector<PassDesc>& zero_passes, cudaStream_t s,
                                    std::vector<int>& outcome_of_pass) {
  const size_t K = p.meas_qubit.size();
  std::vector<const Cmd*> mcmd(K, nullptr);
  for (const Cmd& c : p.cmds)
    if (c.kind == OWQS_CMD_M) mcmd[(size_t)p.k_of_qubit[c.q0]] = &c;
  std::vector<const PassDesc*> meas;
  for (const PassDesc& d : zero_passes)
    if (d.kind == 0) meas.push_back(&d);
  // domains of every measurement after the first, as K-indices
  std::vector<uint32_t> dom;
  std::vector<uint32_t> sd_off(meas.size()), td_off(meas.size());
  for (size_t i = 0; i < meas.size(); ++i) {
    const Cmd& c = *mcmd[meas[i]->meas_k];
    sd_off[i] = (uint32_t)dom.size();
    for (uint32_t q : c.sdom) dom.push_back((uint32_t)p.k_of_qubit[q]);
    td_off[i] = (uint32_t)dom.size();
    for (uint32_t q : c.tdom) dom.push_back((uint32_t)p.k_of_qubit[q]);
  }
  // workspace: [seed][e: 2K][w1: 2K][dom][outcomes]
  const size_t off_e = 8, off_w1 = off_e + 16 * K, off_dom = off_w1 + 16 * K;
  const size_t off_oc = off_dom + 4 * ((dom.size() + 1) & ~(size_t)1);
  const size_t need = off_oc + ((K + 15) & ~(size_t)15) + 16;
  if (need > rc->samp_bytes || !rc->samp) {
    if (rc->gexec) {  // graphs hold the old addresses
      cudaGraphExecDestroy(rc->gexec);
      rc->gexec = nullptr;
      rc->gkey.clear();
    }
    owqs_status st = ensure_buf(rc->samp, rc->samp_bytes, need, "sampling workspace");
    if (st != OWQS_OK) return st;
  }
  char* base = static_cast<char*>(rc->samp);
  uint64_t* seed = reinterpret_cast<uint64_t*>(base);
  double* e = reinterpret_cast<double*>(base + off_e);
  double* w1 = reinterpret_cast<double*>(base + off_w1);
  uint32_t* ddom = reinterpret_cast<uint32_t*>(base + off_dom);
  uint8_t* doc = reinterpret_cast<uint8_t*>(base + off_oc);
  // the first measurement's e^{-i theta}: its domains are empty (measured first)
  double e0[2] = {1.0, 0.0};
  if (!meas.empty()) {
    e0[0] = meas[0]->ere;
    e0[1] = meas[0]->eim;
  }
  cudaError_t ce = cudaMemcpyAsync(e, e0, sizeof(e0), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess && !dom.empty())
    ce = cudaMemcpyAsync(ddom, dom.data(), 4 * dom.size(), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);  // host vectors go out of scope
  if (ce != cudaSuccess) return cuda_fail(ce, "sampling tables");

  Runner R(p, *rc, o->dtype, o->mode, s);
  R.begin(pr.in_dev, pr.in_elems, pr.out_dev, pr.out_elems);
  for (size_t i = 0; i < meas.size(); ++i) {
    const PassDesc& d = *meas[i];
    DecideParams D;
    std::memset(&D, 0, sizeof(D));
    D.norms = rc->norms;
    D.pslot = R.prob_dev(d, e + 2 * i);
    D.seed = seed;
    D.draw = i;
    D.outcomes = doc;
    D.meas_k = d.meas_k;
    D.e_this = e + 2 * i;
    D.w1 = w1 + 2 * i;
    if (i + 1 < meas.size()) {
      const Cmd& c = *mcmd[meas[i + 1]->meas_k];
      D.has_next = 1;
      D.dom = ddom;
      D.sd_off = sd_off[i + 1];
      D.sd_len = (uint32_t)c.sdom.size();
      D.td_off = td_off[i + 1];
      D.td_len = (uint32_t)c.tdom.size();
      D.ca = std::cos(c.angle);
      D.sa = std::sin(c.angle);
      D.e_next = e + 2 * (i + 1);
    }
    R.decide(D);
    R.measure_dev(d, w1 + 2 * i);
  }
  owqs_status st = launch_put_u64(seed, o->seed, s) == cudaSuccess ? OWQS_OK : cuda_fail(cudaGetLastError(), "seed");
  if (st != OWQS_OK) return st;
  st = replay(rc, R, graph_key(p, o, pr.in_dev, pr.out_dev, nullptr), o->use_graph != 0, s);
  if (st != OWQS_OK) return st;
  std::vector<uint8_t> oc(std::max<size_t>(K, 1), 0);
  if (K) ce = cudaMemcpyAsync(oc.data(), doc, K, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_fail(ce, "reading sampled outcomes");
  // the whole schedule under the drawn outcomes: the measure passes launched
  // above are its measure passes (up to their phases, read from the device)
  FixedSource src(p, oc.data());
  pr.passes.clear();
  st = compile_schedule(p, o->mode, src, pr.passes);
  if (st != OWQS_OK) return st;
  R.immediate = true;
  R.final_pass(pr.passes.back());
  if (R.err != OWQS_OK) return R.err;
  for (const PassDesc& d : pr.passes)
    if (d.kind == 0) outcome_of_pass.push_back(d.outcome);
  return OWQS_OK;
}

// Pass groups in double-float (complex128, OWQS_RUN_DOUBLE_FLOAT): between
// two such groups on the same array the array stays in double-float pairs.
static void mark_double_float(std::vector<Item>& items) {
  for (size_t i = 0; i < items.size(); ++i) {
    Item& it = items[i];
    if (it.type != 4) continue;
    it.G.df = 1;
    const Item* prev = i > 0 ? &items[i - 1] : nullptr;
    const Item* next = i + 1 < items.size() ? &items[i + 1] : nullptr;
    it.G.df_in = prev && prev->type == 4 && prev->G.df_out && prev->G.out == it.G.in ? 1 : 0;
    it.G.df_out = next && next->type == 4 && next->G.in == it.G.out ? 1 : 0;
  }
}

static owqs_status run_core(Pattern& p, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                            uint8_t* outcomes, double* probs, float* prof_ms, double* prof_bytes,
                            uint32_t* prof_kind, uint32_t prof_cap, uint32_t* prof_n, int vdiag,
                            double* frob2, const ProductInput* prod, uint32_t* prof_meas) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(o ? o->stream : nullptr);
  RunCache* rc = nullptr;
  Prepared pr;
  const bool sampled = o && o->policy == OWQS_OUTCOME_SAMPLED;
  if (prod && (sampled || (o && o->io != OWQS_IO_DEVICE) || vdiag || psi_in))
    return set_error(OWQS_ERR_UNSUPPORTED, "product inputs take device vectors and forced or zero outcomes");
  // host-decided refusals of a one-at-a-time draw, before any device work
  if (sampled && prof_ms) return set_error(OWQS_ERR_ARG, "profiling needs forced or zero outcomes");
  if (sampled && !p.deps_ok)
    return set_error(OWQS_ERR_ARG, "sampled outcomes need an order that measures every domain first");
  owqs_status st = prepare(p, o, psi_in, psi_out, outcomes, rc, pr, sampled, prod);
  if (st != OWQS_OK) return st;
  const int K = (int)p.meas_qubit.size();
  std::vector<int> outcome_of_pass;
  std::vector<char> in_group;

  if (sampled) {
    // structure pass (outcome-independent widths) to size the buffers
    FixedSource zero(p, nullptr);
    std::vector<PassDesc> tmp;
    st = compile_schedule(p, o->mode, zero, tmp);
    if (st != OWQS_OK) return st;
    size_t wmax = 1;
    for (const PassDesc& d : tmp)
      if (d.kind != 1) wmax = std::max<size_t>(wmax, (size_t)1 << d.n_out);
    st = ensure_pingpong(rc, wmax, pr.amp);
    if (st != OWQS_OK) return st;
    if (o->io == OWQS_IO_HOST && psi_in) {
      cudaError_t e = cudaMemcpyAsync(rc->in_stage, psi_in, pr.in_elems * pr.amp, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "input copy");
    }
    if (!(o->flags & OWQS_RUN_HOST_SAMPLING) && vdiag == 0 && masks_outcome_free(p)) {
      st = sample_on_device(p, o, rc, pr, tmp, s, outcome_of_pass);
      if (st != OWQS_OK) return st;
      if (o->io == OWQS_IO_HOST) {
        cudaError_t e = cudaMemcpyAsync(psi_out, rc->out_stage, pr.out_elems * pr.amp, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "output copy");
      }
      return finish(p, o, rc, pr, s, outcomes, probs, outcome_of_pass, pr.in_dev != nullptr, vdiag, frob2,
                    in_group);
    }
    Runner R(p, *rc, o->dtype, o->mode, s);
    R.immediate = true;
    R.begin(pr.in_dev, pr.in_elems, pr.out_dev, pr.out_elems);
    SampledSource src(R, *rc, s, o->seed);
    st = compile_schedule(p, o->mode, src, pr.passes);
    if (st != OWQS_OK) return st;
    src.flush();
    R.final_pass(pr.passes.back());
    if (R.err != OWQS_OK) return R.err;
    for (const PassDesc& d : pr.passes)
      if (d.kind == 0) outcome_of_pass.push_back(d.outcome);
  } else {
    // separate sub-states (Section 4.1) when the components' arrays need at
    // most half the memory of one array over every live qubit, or when asked
    CompSchedule cs;
    bool comps = false;
    if (!prod && vdiag == 0 && !(o->flags & OWQS_RUN_ONE_ARRAY)) {
      FixedSource csrc(p, o->policy == OWQS_OUTCOME_ZERO ? nullptr : outcomes);
      st = compile_components(p, o->mode, csrc, pr.in_dev != nullptr, cs);
      if (st != OWQS_OK) {
        if (o->flags & OWQS_RUN_SUBSTATES) return st;
        clear_error();
      } else {
        comps = (o->flags & OWQS_RUN_SUBSTATES) || use_substates(cs);
      }
    } else if (o->flags & OWQS_RUN_SUBSTATES) {
      return set_error(OWQS_ERR_UNSUPPORTED, "separate sub-states take one input vector (no product input, no unitary)");
    }
    std::vector<CompLaunch> claunch;
    size_t arena_need = 0;
    if (comps) {
      st = plan_components(cs, o->dtype, pr.amp, pr.in_dev != nullptr, pr.in_elems, claunch, arena_need, pr.passes);
      if (st != OWQS_OK) return st;
      if (rc->arena_bytes < arena_need || !rc->arena) {
        if (rc->gexec) {  // graphs hold the old addresses
          cudaGraphExecDestroy(rc->gexec);
          rc->gexec = nullptr;
          rc->gkey.clear();
        }
        st = ensure_buf(rc->arena, rc->arena_bytes, arena_need, "sub-state arena");
        if (st != OWQS_OK) return st;
      }
      rc->last_components = (uint32_t)cs.ncomp;
      rc->last_peak_bytes = (uint64_t)arena_need;
    } else {
      size_t wmax = 1;
      for (const PassDesc& d : pr.passes)
        if (d.kind != 1) wmax = std::max<size_t>(wmax, (size_t)1 << d.n_out);
      st = ensure_pingpong(rc, wmax, pr.amp);
      if (st != OWQS_OK) return st;
      rc->last_components = 0;
      rc->last_peak_bytes = (uint64_t)rc->buf_bytes * 2;
    }
    for (const PassDesc& d : pr.passes)
      if (d.kind == 0) outcome_of_pass.push_back(d.outcome);
    Runner R(p, *rc, o->dtype, o->mode, s);
    R.vdiag = vdiag;
    R.begin(pr.in_dev, pr.in_elems, pr.out_dev, pr.out_elems);
    const bool small = !comps && !prod && !(o->flags & OWQS_RUN_PER_PASS) && small_run_ok(pr.passes);
    if (comps)
      issue_components(claunch, cs.ncomp, cs.input_comp, o->mode == OWQS_MODE_OWQS, pr.in_dev != nullptr, pr.in_dev,
                       static_cast<char*>(rc->arena), R);
    for (size_t i = 0; !comps && i < pr.passes.size(); ++i) {
      const PassDesc& d = pr.passes[i];
      if (small) {  // planned one pass at a time, run in one kernel below
        if (d.kind == 1) R.final_pass(d);
        else R.measure(d);
        continue;
      }
      GroupParams G;
      LaunchPlan GL;
      int gk = 0;
      switch (decide_launch(pr.passes, i, o->dtype, R.real_input(), vdiag > 0, G, GL, gk)) {
        case LAUNCH_JOIN:
          R.join(d, prod->vecs[d.factor], 3 * K + 8 + d.factor);
          break;
        case LAUNCH_FINAL:
          R.final_pass(d);
          break;
        case LAUNCH_GROUP:
          R.measure_group(G, GL);
          i += (size_t)gk - 1;
          break;
        default:
          R.measure(d);
      }
    }
    in_group = R.in_group;
    if (o->dtype == OWQS_C128 && (o->flags & OWQS_RUN_DOUBLE_FLOAT)) mark_double_float(R.items);
    if (o->io == OWQS_IO_HOST && psi_in) {
      cudaError_t e = cudaMemcpyAsync(rc->in_stage, psi_in, pr.in_elems * pr.amp, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "input copy");
    }
    rc->last_launches = (uint32_t)R.items.size();
    if (small) {
      std::vector<PassParams> ps;
      int input_norm = 0;
      for (const Item& it : R.items) {
        if (it.type == 1) input_norm = 1;
        else ps.push_back(it.P);
      }
      const size_t bytes = ps.size() * sizeof(PassParams);
      if (rc->small_host.size() != bytes || std::memcmp(rc->small_host.data(), ps.data(), bytes) != 0) {
        st = ensure_buf(rc->small_dev, rc->small_bytes, bytes, "small-run passes");
        if (st != OWQS_OK) return st;
        cudaError_t e = cudaMemcpyAsync(rc->small_dev, ps.data(), bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "small-run passes");
        rc->small_host.assign(reinterpret_cast<const unsigned char*>(ps.data()),
                              reinterpret_cast<const unsigned char*>(ps.data()) + bytes);
      }
      rc->last_launches = 1;
      const PassParams* pd = reinterpret_cast<const PassParams*>(rc->small_dev);
      if (prof_ms) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_small(pd, (int)ps.size(), input_norm, o->dtype, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        float ms = 0;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_fail(e, "profiled small run");
        if (prof_cap > 0) {
          prof_ms[0] = ms;
          double by = 0.0;
          for (const Item& it : R.items) by += it.L.bytes;
          if (prof_bytes) prof_bytes[0] = by;
          if (prof_kind) prof_kind[0] = (uint32_t)KK_SMALL;
          if (prof_meas) prof_meas[0] = (uint32_t)K;
        }
        if (prof_n) *prof_n = 1;
      } else {
        cudaError_t e = launch_small(pd, (int)ps.size(), input_norm, o->dtype, s);
        if (e != cudaSuccess) return cuda_fail(e, "small run");
      }
    } else if (prof_ms) {
      std::vector<cudaEvent_t> ev(2 * R.items.size());
      for (auto& x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");
      for (size_t i = 0; i < R.items.size(); ++i) {
        cudaEventRecord(ev[2 * i], s);
        st = R.launch(R.items[i], s);
        cudaEventRecord(ev[2 * i + 1], s);
        if (st != OWQS_OK) break;
      }
      cudaError_t e = cudaStreamSynchronize(s);
      if (st == OWQS_OK && e != cudaSuccess) st = cuda_fail(e, "profiled run");
      const uint32_t n = (uint32_t)std::min<size_t>(R.items.size(), prof_cap);
      for (uint32_t i = 0; i < n && st == OWQS_OK; ++i) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
        prof_ms[i] = ms;
        if (prof_bytes) prof_bytes[i] = R.items[i].L.bytes;
        if (prof_kind) prof_kind[i] = (uint32_t)R.items[i].L.kind;
        if (prof_meas) prof_meas[i] = (uint32_t)R.items[i].L.meas;
      }
      if (prof_n) *prof_n = (uint32_t)R.items.size();
      for (auto& x : ev) cudaEventDestroy(x);
      if (st != OWQS_OK) return st;
    } else {
      // test hook: make the first bulk-copy launch give up on a wait
      Item* stall = nullptr;
      for (Item& it : R.items)
        if ((it.type == 0 && it.L.kind == KK_TMA) || it.type == 4) {
          stall = &it;
          break;
        }
      long long limit = 0;
      uint64_t shrink = 0;
      if (stall && take_test_stall(&limit)) {
        if (stall->type == 4) stall->G.stall_limit = limit;
        else stall->P.stall_limit = limit;
        st = replay(rc, R, std::string(), false, s);  // direct launches, no graph
      } else if (take_test_shrink(&shrink)) {
        // test hook: every buffer extent the launches carry is `shrink`
        // amplitudes short (only bounds-checked builds read the extents)
        auto cut = [shrink](uint64_t& cap) {
          if (cap) cap = cap > shrink ? cap - shrink : 1;
        };
        for (Item& it : R.items) {
          cut(it.P.in_cap);
          cut(it.P.out_cap);
          cut(it.G.in_cap);
          cut(it.G.out_cap);
          cut(it.Kp.in_cap);
          cut(it.Kp.out_cap);
        }
        st = replay(rc, R, std::string(), false, s);
      } else {
        std::string key = graph_key(p, o, pr.in_dev, pr.out_dev, outcomes);
        if (comps) {  // a component run: its arena (the items hold pointers into it)
          key.push_back('C');
          key.append(reinterpret_cast<const char*>(&rc->arena), sizeof(rc->arena));
        }
        if (prod)
          for (const void* v : prod->vecs) key.append(reinterpret_cast<const char*>(&v), sizeof(v));
        st = replay(rc, R, key, o->use_graph != 0, s);
      }
      if (st != OWQS_OK) return st;
    }
  }
  if (o->io == OWQS_IO_HOST) {
    cudaError_t e = cudaMemcpyAsync(psi_out, rc->out_stage, pr.out_elems * pr.amp, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "output copy");
  }
  (void)K;
  return finish(p, o, rc, pr, s, outcomes, probs, outcome_of_pass, pr.in_dev != nullptr, vdiag, frob2,
                in_group);
}

// Sampled OWQS by checked launches (the draw of Fig. 6, one launch at a
// time instead of one measurement at a time).
//
// The outcome vector starts as the guesses u_k > 1/2 and the run is the
// forced run of the current vector, launched one kernel at a time.  After
// each launch that measures, the host reads the probabilities it computed
// and takes its measurements in execution order.  One whose draw u_k <=
// prob_0 reproduces its outcome is decided.  At the first one that does not,
// the draw has decided the other outcome: its prob_0 was computed on the
// branch of the decided outcomes before it, so this is the draw a
// one-measurement-at-a-time run makes.  The outcome vector is corrected,
// the schedule recompiled, and the same launch runs again on its input,
// which no later launch has touched.  A launch thus runs once, plus once per
// corrected outcome among its measurements; where every probability is 1/2
// (a gflow, Section 4.5) the guesses hold and this is the forced run with one
// host check per launch.  A draw within rounding of prob_0 follows this
// run's prob_0.  Requires measure passes whose sign forms and X masks do not
// depend on outcomes (masks_outcome_free), so that every recompiled schedule
// has the same launches on the same buffers; returns OWQS_ERR_UNSUPPORTED
// before any launch otherwise.
static bool same_launches(const std::vector<Item>& a, const std::vector<Item>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i) {
    const Item& x = a[i];
    const Item& y = b[i];
    if (x.type != y.type || x.L.meas != y.L.meas || x.L.kind != y.L.kind) return false;
    if (x.type == 4 && (x.G.in != y.G.in || x.G.out != y.G.out || x.G.k != y.G.k)) return false;
    if (x.type == 0 && (x.P.in != y.P.in || x.P.out != y.P.out)) return false;
  }
  return true;
}

// The launch list of a one-array run of pr.passes, one launch per pass or
// pass group, nothing launched (no factor joins: false if the passes have one).
static bool build_one_array(Runner& R, const Prepared& pr, const owqs_run_opts* o) {
  R.begin(pr.in_dev, pr.in_elems, pr.out_dev, pr.out_elems);
  for (size_t i = 0; i < pr.passes.size(); ++i) {
    GroupParams G;
    LaunchPlan GL;
    int gk = 0;
    switch (decide_launch(pr.passes, i, o->dtype, R.real_input(), false, G, GL, gk)) {
      case LAUNCH_JOIN:
        return false;
      case LAUNCH_FINAL:
        R.final_pass(pr.passes[i]);
        break;
      case LAUNCH_GROUP:
        R.measure_group(G, GL);
        i += (size_t)gk - 1;
        break;
      default:
        R.measure(pr.passes[i]);
    }
  }
  if (o->dtype == OWQS_C128 && (o->flags & OWQS_RUN_DOUBLE_FLOAT)) mark_double_float(R.items);
  return R.err == OWQS_OK;
}

static owqs_status sample_checked(Pattern& p, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                                  uint8_t* outcomes, double* probs, const std::vector<double>& u,
                                  std::vector<uint8_t>& oc) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(o->stream);
  owqs_run_opts fo = *o;
  fo.policy = OWQS_OUTCOME_FORCED;
  RunCache* rc = nullptr;
  Prepared pr;
  owqs_status st = prepare(p, &fo, psi_in, psi_out, oc.data(), rc, pr, false);
  if (st != OWQS_OK) return st;
  size_t wmax = 1;
  for (const PassDesc& d : pr.passes)
    if (d.kind != 1) wmax = std::max<size_t>(wmax, (size_t)1 << d.n_out);
  st = ensure_pingpong(rc, wmax, pr.amp);
  if (st != OWQS_OK) return st;
  auto build = [&](Runner& R) { return build_one_array(R, pr, o); };
  Runner R(p, *rc, o->dtype, o->mode, s);
  if (!build(R)) return set_error(OWQS_ERR_UNSUPPORTED, "checked launches: a run without factor joins");
  if (o->io == OWQS_IO_HOST && psi_in) {
    cudaError_t e = cudaMemcpyAsync(rc->in_stage, psi_in, pr.in_elems * pr.amp, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "input copy");
  }
  const size_t K = p.meas_qubit.size();
  std::vector<uint32_t> kpos;  // execution position -> K-index
  for (const PassDesc& d : pr.passes)
    if (d.kind == 0) kpos.push_back(d.meas_k);
  std::vector<char> decided(std::max<size_t>(K, 1), 0);
  std::vector<double> slot(K + 2, 0.0);
  uint32_t relaunches = 0, checks = 0;
  size_t mi0 = 0;  // execution position of the next launch's first measurement
  for (size_t pos = 0; pos < R.items.size();) {
    st = R.launch(R.items[pos], s);
    if (st != OWQS_OK) return st;
    const size_t cnt = (size_t)R.items[pos].L.meas;
    if (cnt == 0) {
      ++pos;
      continue;
    }
    // slots mi0 (the value before this launch) .. mi0 + cnt
    cudaError_t e = cudaMemcpyAsync(slot.data() + mi0, rc->norms + mi0, sizeof(double) * (cnt + 1),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading probabilities");
    ++checks;
    bool corrected = false;
    for (size_t j = 0; j < cnt; ++j) {
      const size_t mi = mi0 + j;
      const uint32_t k = kpos[mi];
      if (decided[k]) continue;
      // later measurements of a group hold the running product of its probabilities
      double pv = slot[mi + 1];
      if (j > 0) pv = slot[mi] > 0.0 ? pv / slot[mi] : 0.0;
      const double p0 = oc[k] ? 1.0 - pv : pv;
      const uint8_t drawn = u[k] <= p0 ? 0 : 1;
      decided[k] = 1;
      if (drawn != oc[k]) {
        oc[k] = drawn;
        corrected = true;
        break;
      }
    }
    if (!corrected) {
      mi0 += cnt;
      ++pos;
      continue;
    }
    // recompile under the corrected outcomes; the launches are the same, on
    // the same buffers, with other signs and phases
    ++relaunches;
    pr.passes.clear();
    FixedSource src(p, oc.data());
    st = compile_schedule(p, o->mode, src, pr.passes);
    if (st != OWQS_OK) return st;
    Runner R2(p, *rc, o->dtype, o->mode, s);
    if (!build(R2) || !same_launches(R.items, R2.items))
      return set_error(OWQS_ERR_UNSUPPORTED, "checked launches: the recompiled schedule has other launches");
    R.items.swap(R2.items);
    R.in_group.swap(R2.in_group);
  }
  rc->last_launches = (uint32_t)R.items.size();
  rc->last_relaunches = relaunches;
  rc->last_checks = checks;
  if (o->io == OWQS_IO_HOST) {
    cudaError_t e = cudaMemcpyAsync(psi_out, rc->out_stage, pr.out_elems * pr.amp, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "output copy");
  }
  std::vector<int> outcome_of_pass;
  for (const PassDesc& d : pr.passes)
    if (d.kind == 0) outcome_of_pass.push_back(d.outcome);
  return finish(p, o, rc, pr, s, outcomes, probs, outcome_of_pass, pr.in_dev != nullptr, 0, nullptr, R.in_group);
}

// Asynchronous runs: the call compiles the schedule, enqueues the run and
// returns; owqs_wait completes the oldest run in flight.  With host vectors,
// the input copy goes on a copy stream once the previous asynchronous run's
// launches that read the input staging buffer are done, the output copy on a
// second copy stream once the final pass has written the output staging
// buffer; a run's final pass waits for the previous run's output copy.  So a
// run's input copy overlaps the previous run's launches and its output copy
// the next run's.  The norm slots and the error flag are copied on the
// compute stream right after the final pass (the next run's launches follow
// on the same stream), then read back on the copy stream.  One array, one
// launch per pass or pass group, forced or zero outcomes.
static owqs_status ensure_async(RunCache* rc, RunCache::Pending& q, size_t doubles) {
  cudaError_t e = cudaSuccess;
  if (!rc->copy_in) e = cudaStreamCreateWithFlags(&rc->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !rc->copy_out) e = cudaStreamCreateWithFlags(&rc->copy_out, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&rc->in_free, &rc->h2d_done, &rc->ready, &q.done})
    if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e == cudaSuccess && q.cap < doubles) {
    if (q.host) cudaFreeHost(q.host);
    if (q.snap) cudaFree(q.snap);
    q.host = nullptr;
    q.snap = nullptr;
    q.cap = 0;
    e = cudaMallocHost(reinterpret_cast<void**>(&q.host), doubles * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&q.snap), doubles * sizeof(double));
    if (e == cudaSuccess) q.cap = doubles;
  }
  return e == cudaSuccess ? OWQS_OK : cuda_fail(e, "asynchronous run resources");
}

static owqs_status run_async_enqueue(Pattern& p, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                                     const uint8_t* outcomes) {
  if (!o || !psi_out) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (o->policy == OWQS_OUTCOME_SAMPLED)
    return set_error(OWQS_ERR_UNSUPPORTED, "asynchronous runs take forced or zero outcomes");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(o->stream);
  RunCache* rc = nullptr;
  owqs_status st = get_cache(p, rc);
  if (st != OWQS_OK) return st;
  if (rc->pend_count == 2) return set_error(OWQS_ERR_ARG, "two asynchronous runs in flight: call owqs_wait first");
  Prepared pr;
  st = prepare(p, o, psi_in, psi_out, outcomes, rc, pr, false);
  if (st != OWQS_OK) return st;
  size_t wmax = 1;
  for (const PassDesc& d : pr.passes)
    if (d.kind != 1) wmax = std::max<size_t>(wmax, (size_t)1 << d.n_out);
  st = ensure_pingpong(rc, wmax, pr.amp);
  if (st != OWQS_OK) return st;
  Runner R(p, *rc, o->dtype, o->mode, s);
  if (!build_one_array(R, pr, o)) return set_error(OWQS_ERR_UNSUPPORTED, "asynchronous runs take one input vector");
  const int slot = (rc->pend_head + rc->pend_count) % 2;
  RunCache::Pending& q = rc->pend[slot];
  const size_t K = p.meas_qubit.size();
  st = ensure_async(rc, q, K + 3);
  if (st != OWQS_OK) return st;
  const bool host_io = o->io == OWQS_IO_HOST;
  // the last launch that reads the input staging buffer
  size_t last_in = SIZE_MAX;
  for (size_t i = 0; i < R.items.size(); ++i) {
    const Item& it = R.items[i];
    const void* in = it.type == 1 ? it.norm_in : it.type == 4 ? it.G.in : it.type == 0 ? it.P.in : nullptr;
    if (pr.in_dev && in == pr.in_dev) last_in = i;
  }
  cudaError_t e = cudaSuccess;
  if (host_io && psi_in) {
    if (rc->in_free_set) e = cudaStreamWaitEvent(rc->copy_in, rc->in_free, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rc->in_stage, psi_in, pr.in_elems * pr.amp, cudaMemcpyHostToDevice, rc->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(rc->h2d_done, rc->copy_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, rc->h2d_done, 0);
    if (e != cudaSuccess) return cuda_fail(e, "asynchronous input copy");
  }
  for (size_t i = 0; i < R.items.size(); ++i) {
    if (host_io && i + 1 == R.items.size() && rc->last_slot >= 0) {
      // the final pass writes the output staging buffer: the previous run's output copy must be done
      e = cudaStreamWaitEvent(s, rc->pend[rc->last_slot].done, 0);
      if (e != cudaSuccess) return cuda_fail(e, "asynchronous run order");
    }
    st = R.launch(R.items[i], s);
    if (st != OWQS_OK) return st;
    if (host_io && i == last_in) {
      e = cudaEventRecord(rc->in_free, s);
      if (e != cudaSuccess) return cuda_fail(e, "asynchronous run order");
      rc->in_free_set = true;
    }
  }
  e = cudaMemcpyAsync(q.snap, rc->norms, sizeof(double) * (K + 2), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(q.snap + K + 2, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(q.snap + K + 2, rc->counter + 1, sizeof(unsigned int),
                                            cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(rc->counter + 1, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaEventRecord(rc->ready, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(rc->copy_out, rc->ready, 0);
  if (e == cudaSuccess && host_io)
    e = cudaMemcpyAsync(psi_out, rc->out_stage, pr.out_elems * pr.amp, cudaMemcpyDeviceToHost, rc->copy_out);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(q.host, q.snap, sizeof(double) * (K + 3), cudaMemcpyDeviceToHost, rc->copy_out);
  if (e == cudaSuccess) e = cudaEventRecord(q.done, rc->copy_out);
  if (e != cudaSuccess) return cuda_fail(e, "asynchronous run");
  q.opts = *o;
  q.passes = pr.passes;
  q.in_group = R.in_group;
  q.outcome_of_pass.clear();
  for (const PassDesc& d : pr.passes)
    if (d.kind == 0) q.outcome_of_pass.push_back(d.outcome);
  q.has_input = pr.in_dev != nullptr;
  rc->last_slot = slot;
  ++rc->pend_count;
  rc->last_launches = (uint32_t)R.items.size();
  return OWQS_OK;
}

static owqs_status run_async_wait(Pattern& p, uint8_t* outcomes, double* probs) {
  RunCache* rc = p.cache.get();
  if (!rc || rc->pend_count == 0) return set_error(OWQS_ERR_ARG, "no asynchronous run in flight");
  RunCache::Pending& q = rc->pend[rc->pend_head];
  const cudaError_t e = cudaEventSynchronize(q.done);
  rc->pend_head = (rc->pend_head + 1) % 2;
  --rc->pend_count;
  if (e != cudaSuccess) return cuda_fail(e, "asynchronous run");
  const size_t K = p.meas_qubit.size();
  const std::vector<double> h(q.host, q.host + K + 2);
  unsigned int flag = 0;
  std::memcpy(&flag, q.host + K + 2, sizeof(flag));
  return interpret_run(p, &q.opts, h, flag, q.passes, outcomes, probs, q.outcome_of_pass, q.has_input, 0, nullptr,
                       q.in_group);
}

// Sampled outcomes as a forced run.
//
// EOWQS (Section 4.5): a pattern with a gflow is strongly deterministic, so
// every measurement gives either outcome with probability 1/2 whatever came
// before, and no probability is computed.  The outcomes are drawn before the
// run, outcome 0 iff u <= 1/2 with u the k-th splitmix64 uniform for the k-th
// measurement in execution order, and the run is then a forced one (pass
// groups, one graph).
//
// OWQS: the outcomes are guessed the same way, the forced run computes the
// probability of every guessed outcome on the branch of the guesses before
// it, and the guess is kept iff every draw, u_k <= prob_0 of measurement k,
// reproduces it.  Then, by induction over k, the one-at-a-time draw would
// have taken the same branch, so the result is that draw's.  On a pattern
// with a gflow every prob_0 is 1/2 (Section 4.5) and the guess holds unless
// a draw lies within a tie margin of 1/2 (1e-6 for complex64, 1e-12 for
// complex128: the two ways of computing prob_0 differ by rounding).  A
// pattern without a gflow skips this whole-run guess.  Otherwise (and on a
// guessed branch of probability 0) the run takes checked launches
// (sample_checked) where the measure passes allow it, else one measurement
// at a time.
//
// Any other policy or mode, and sampling with OWQS_RUN_HOST_SAMPLING or
// OWQS_RUN_SEQUENTIAL_SAMPLING, goes straight to run_core.
static owqs_status run_impl(Pattern& p, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                            uint8_t* outcomes, double* probs, float* prof_ms, double* prof_bytes,
                            uint32_t* prof_kind, uint32_t prof_cap, uint32_t* prof_n, int vdiag = 0,
                            double* frob2 = nullptr, const ProductInput* prod = nullptr,
                            uint32_t* prof_meas = nullptr) {
  if (p.cache && p.cache->pend_count)
    return set_error(OWQS_ERR_ARG, "asynchronous runs in flight on this pattern: call owqs_wait first");
  const bool eowqs = o && o->mode == OWQS_MODE_EOWQS;
  // the path of a one-at-a-time draw (run_core's sampled branch)
  const uint32_t one_at_a_time = o && !(o->flags & OWQS_RUN_HOST_SAMPLING) && masks_outcome_free(p)
                                     ? OWQS_SAMPLE_ONE_AT_A_TIME
                                     : OWQS_SAMPLE_HOST;
  if (!o || o->policy != OWQS_OUTCOME_SAMPLED || prod || vdiag ||
      (!eowqs && (prof_ms || !p.deps_ok || (o->flags & (OWQS_RUN_HOST_SAMPLING | OWQS_RUN_SEQUENTIAL_SAMPLING))))) {
    RunCache* rc0 = nullptr;
    if (o && o->policy == OWQS_OUTCOME_SAMPLED && !prod && !vdiag && !prof_ms && get_cache(p, rc0) == OWQS_OK) {
      rc0->last_sample_path = one_at_a_time;
      rc0->last_guessed = rc0->last_relaunches = rc0->last_checks = 0;
    }
    return run_core(p, o, psi_in, psi_out, outcomes, probs, prof_ms, prof_bytes, prof_kind, prof_cap, prof_n,
                    vdiag, frob2, prod, prof_meas);
  }
  const size_t K = p.meas_qubit.size();
  std::vector<uint8_t> drawn(std::max<size_t>(K, 1), 0);
  std::vector<double> u(std::max<size_t>(K, 1), 0.0);
  uint64_t state = o->seed;
  for (uint32_t ci : p.active) {
    const Cmd& c = p.cmds[ci];
    if (c.kind != OWQS_CMD_M) continue;
    const size_t k = (size_t)p.k_of_qubit[c.q0];
    u[k] = splitmix_uniform(state);
    drawn[k] = u[k] <= 0.5 ? 0 : 1;
  }
  owqs_run_opts fo = *o;
  fo.policy = OWQS_OUTCOME_FORCED;
  std::vector<double> pk(std::max<size_t>(K, 1), 0.0);
  const bool checkable = !eowqs && masks_outcome_free(p);
  RunCache* rc = nullptr;
  owqs_status st = get_cache(p, rc);
  if (st != OWQS_OK) return st;
  auto checked = [&]() {
    std::vector<uint8_t> oc(std::max<size_t>(K, 1), 0);
    for (size_t k = 0; k < K; ++k) oc[k] = u[k] <= 0.5 ? 0 : 1;
    owqs_status cs = sample_checked(p, o, psi_in, psi_out, outcomes, probs, u, oc);
    if (cs == OWQS_ERR_UNSUPPORTED) {  // one measurement at a time
      clear_error();
      cs = run_core(p, o, psi_in, psi_out, outcomes, probs, prof_ms, prof_bytes, prof_kind, prof_cap, prof_n, vdiag,
                    frob2, prod, prof_meas);
      rc->last_sample_path = one_at_a_time;
    } else {
      rc->last_sample_path = OWQS_SAMPLE_CHECKED_LAUNCHES;
    }
    return cs;
  };
  rc->last_guessed = rc->last_relaunches = rc->last_checks = 0;
  if (checkable && !has_gflow(p)) return checked();
  rc->last_sample_path = eowqs ? OWQS_SAMPLE_DRAWN_FIRST : OWQS_SAMPLE_GUESS_KEPT;
  rc->last_guessed = eowqs ? 0 : 1;
  st = run_core(p, &fo, psi_in, psi_out, drawn.data(), pk.data(), prof_ms, prof_bytes, prof_kind, prof_cap, prof_n,
                vdiag, frob2, prod, prof_meas);
  bool kept = st == OWQS_OK;
  if (!eowqs) {
    // The guessed run computes prob_0 as 1 - prob_1 where it guessed 1, and
    // with other kernels than a one-at-a-time run: the two agree only up to
    // rounding.  A draw within tie_margin of that prob_0 could go either way,
    // so the guess is kept only when every draw clears it by more.
    const double tie_margin = o->dtype == OWQS_C64 ? 1e-6 : 1e-12;
    for (size_t k = 0; kept && k < K; ++k) {
      const double p0 = drawn[k] ? 1.0 - pk[k] : pk[k];
      kept = (u[k] <= p0 ? 0 : 1) == drawn[k] && std::fabs(u[k] - p0) > tie_margin;
    }
    if (!kept && (st == OWQS_OK || st == OWQS_ERR_IMPOSSIBLE_BRANCH)) {
      clear_error();
      if (checkable) return checked();
      rc->last_sample_path = one_at_a_time;
      return run_core(p, o, psi_in, psi_out, outcomes, probs, prof_ms, prof_bytes, prof_kind, prof_cap, prof_n,
                      vdiag, frob2, prod, prof_meas);
    }
  }
  if (kept) {
    if (outcomes) std::memcpy(outcomes, drawn.data(), K);
    if (probs) std::memcpy(probs, pk.data(), K * sizeof(double));
  }
  return st;
}

}  // namespace owqs

using namespace owqs;

namespace owqs {
static std::atomic<int> g_test_stall_runs{0};
static std::atomic<long long> g_test_stall_limit{0};
static std::atomic<int> g_test_shrink_runs{0};
static std::atomic<uint64_t> g_test_shrink_elems{0};

int take_test_shrink(uint64_t* elems) {
  int n = g_test_shrink_runs.load();
  while (n > 0 && !g_test_shrink_runs.compare_exchange_weak(n, n - 1)) {
  }
  if (n <= 0) return 0;
  *elems = g_test_shrink_elems.load();
  return 1;
}

int take_test_stall(long long* limit) {
  int n = g_test_stall_runs.load();
  while (n > 0 && !g_test_stall_runs.compare_exchange_weak(n, n - 1)) {
  }
  if (n <= 0) return 0;
  *limit = g_test_stall_limit.load();
  return 1;
}

owqs_status run_unchecked(Pattern& p, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                          uint8_t* outcomes, double* probs) {
  clear_error();
  return run_impl(p, o, psi_in, psi_out, outcomes, probs, nullptr, nullptr, nullptr, 0, nullptr);
}
}  // namespace owqs

extern "C" {

owqs_status owqs_run_product(owqs_pattern* h, const owqs_run_opts* o, uint32_t nfactors, const uint32_t* sizes,
                             const uint32_t* qubits, const void* const* vecs, void* psi_out, uint8_t* outcomes,
                             double* probs) {
  clear_error();
  if (!h || !o || (nfactors && (!sizes || !qubits || !vecs))) return set_error(OWQS_ERR_ARG, "NULL argument");
  const Pattern& p = h->p;
  ProductInput prod;
  std::vector<char> seen(p.n, 0), is_in(p.n, 0);
  for (uint32_t q : p.inputs) is_in[q] = 1;
  size_t at = 0, covered = 0;
  for (uint32_t f = 0; f < nfactors; ++f) {
    if (sizes[f] == 0 || sizes[f] > 30) return set_error(OWQS_ERR_ARG, "factor sizes must be 1 .. 30 qubits");
    if (!vecs[f] || ((uintptr_t)vecs[f] % 16)) return set_error(OWQS_ERR_ARG, "factor vectors must be 16-byte aligned");
    std::vector<uint32_t> qs(qubits + at, qubits + at + sizes[f]);
    at += sizes[f];
    for (uint32_t q : qs) {
      if (q >= p.n || !is_in[q] || seen[q]) return set_error(OWQS_ERR_ARG, "every input must be in exactly one factor");
      seen[q] = 1;
      ++covered;
    }
    prod.qubits.push_back(std::move(qs));
    prod.vecs.push_back(vecs[f]);
  }
  if (covered != p.inputs.size()) return set_error(OWQS_ERR_ARG, "every input must be in exactly one factor");
  if (o->mode == OWQS_MODE_EOWQS && !has_gflow(h->p))
    return set_error(OWQS_ERR_NOT_DETERMINISTIC, "EOWQS: the open graph has no gflow (Section 4.5)");
  return run_impl(h->p, o, nullptr, psi_out, outcomes, probs, nullptr, nullptr, nullptr, 0, nullptr, 0, nullptr,
                  &prod);
}

owqs_status owqs_last_sample_info(const owqs_pattern* h, owqs_sample_info* info) {
  clear_error();
  if (!h || !info) return set_error(OWQS_ERR_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  const RunCache* rc = h->p.cache.get();
  if (rc) {
    info->path = rc->last_sample_path;
    info->guessed = rc->last_guessed;
    info->checks = rc->last_checks;
    info->relaunches = rc->last_relaunches;
  }
  return OWQS_OK;
}

owqs_status owqs_test_grid_cap(uint32_t blocks) {
  clear_error();
  set_test_grid_cap((int)std::min<uint32_t>(blocks, 1u << 30));
  return OWQS_OK;
}

owqs_status owqs_test_group_m4_width(uint32_t width) {
  clear_error();
  set_test_m4_width((int)std::min<uint32_t>(width, 62u));
  return OWQS_OK;
}

owqs_status owqs_test_shrink_extents(uint32_t runs, uint64_t elems) {
  clear_error();
  if (runs && elems == 0) return set_error(OWQS_ERR_ARG, "elems must be positive");
  g_test_shrink_elems.store(elems);
  g_test_shrink_runs.store((int)runs);
  return OWQS_OK;
}

owqs_status owqs_test_wait_timeout(uint32_t runs, uint64_t limit_cycles) {
  clear_error();
  if (runs && (limit_cycles == 0 || limit_cycles > 4000000000ull))
    return set_error(OWQS_ERR_ARG, "limit_cycles must be in 1 .. 4e9");
  g_test_stall_limit.store((long long)limit_cycles);
  g_test_stall_runs.store((int)runs);
  return OWQS_OK;
}

owqs_status owqs_run(owqs_pattern* h, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                     uint8_t* outcomes, double* probs) {
  clear_error();
  if (!h) return set_error(OWQS_ERR_ARG, "NULL pattern");
  if (o && o->mode == OWQS_MODE_EOWQS && !has_gflow(h->p))
    return set_error(OWQS_ERR_NOT_DETERMINISTIC, "EOWQS: the open graph has no gflow (Section 4.5)");
  return run_impl(h->p, o, psi_in, psi_out, outcomes, probs, nullptr, nullptr, nullptr, 0, nullptr);
}

owqs_status owqs_run_async(owqs_pattern* h, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                           const uint8_t* outcomes) {
  clear_error();
  if (!h) return set_error(OWQS_ERR_ARG, "NULL pattern");
  if (o && o->mode == OWQS_MODE_EOWQS && !has_gflow(h->p))
    return set_error(OWQS_ERR_NOT_DETERMINISTIC, "EOWQS: the open graph has no gflow (Section 4.5)");
  return run_async_enqueue(h->p, o, psi_in, psi_out, outcomes);
}

owqs_status owqs_wait(owqs_pattern* h, uint8_t* outcomes, double* probs) {
  clear_error();
  if (!h) return set_error(OWQS_ERR_ARG, "NULL pattern");
  return run_async_wait(h->p, outcomes, probs);
}

// recognition (Section 1: which unitary a pattern implements): the pattern
// with |I| reference qubits that no command touches, started from the sum over
// c of |c>|c>; the output (O bits low, reference bits high) is U column-major
static owqs::Pattern& augmented(owqs::Pattern& p) {
  if (p.aug && p.aug_version == p.order_version) return *p.aug;
  auto a = std::make_shared<owqs::Pattern>();
  const uint32_t nI = (uint32_t)p.inputs.size();
  a->n = p.n + nI;
  a->inputs = p.inputs;
  a->outputs = p.outputs;
  for (uint32_t k = 0; k < nI; ++k) {
    a->inputs.push_back(p.n + k);
    a->outputs.push_back(p.n + k);
  }
  a->cmds = p.cmds;
  a->k_of_qubit = p.k_of_qubit;
  a->k_of_qubit.resize(a->n, -1);
  a->meas_qubit = p.meas_qubit;
  a->active = p.active;
  a->active_meas = p.active_meas;
  a->standard = p.standard;
  a->deps_ok = p.deps_ok;
  p.aug = a;
  p.aug_version = p.order_version;
  return *a;
}

extern "C++" {
namespace owqs {
uint32_t last_launch_count(Pattern& p, bool unitary) {
  Pattern& q = unitary ? augmented(p) : p;
  return q.cache ? q.cache->last_launches : 0u;
}
}  // namespace owqs
}

owqs_status owqs_unitary(owqs_pattern* h, const owqs_run_opts* o, const uint8_t* outcomes, void* U,
                         double* frob2) {
  clear_error();
  if (!h || !o || !U) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (o->io != OWQS_IO_DEVICE) return set_error(OWQS_ERR_ARG, "owqs_unitary writes a device matrix");
  if (o->policy == OWQS_OUTCOME_SAMPLED) return set_error(OWQS_ERR_ARG, "the recognition branch must be forced or zero");
  if (2 * h->p.inputs.size() + 1 > (size_t)kMaxLive) return set_error(OWQS_ERR_OOM, "too many inputs for a unitary");
  owqs_run_opts oo = *o;
  oo.mode = OWQS_MODE_EOWQS;  // fixed sqrt2 per measurement: the branch as a linear map
  Pattern& a = augmented(h->p);
  return run_impl(a, &oo, nullptr, U, const_cast<uint8_t*>(outcomes), nullptr, nullptr, nullptr, nullptr, 0,
                  nullptr, (int)h->p.inputs.size(), frob2);
}

owqs_status owqs_profile_run(owqs_pattern* h, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                             const uint8_t* outcomes, float* ms, double* bytes, uint32_t* kind, uint32_t* nmeas,
                             uint32_t cap, uint32_t* nlaunch) {
  clear_error();
  if (!h || !o || !ms || !nlaunch) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (o->io != OWQS_IO_DEVICE) return set_error(OWQS_ERR_ARG, "profiling takes device vectors");
  if (o->mode == OWQS_MODE_EOWQS && !has_gflow(h->p))
    return set_error(OWQS_ERR_NOT_DETERMINISTIC, "EOWQS: the open graph has no gflow (Section 4.5)");
  std::vector<uint8_t> oc;
  if (outcomes) oc.assign(outcomes, outcomes + h->p.meas_qubit.size());
  return run_impl(h->p, o, psi_in, psi_out, oc.empty() ? nullptr : oc.data(), nullptr, ms, bytes, kind, cap,
                  nlaunch, 0, nullptr, nullptr, nmeas);
}

owqs_status owqs_plan_memory(const owqs_pattern* h, uint32_t dtype, uint32_t mode, uint32_t real_input,
                            const uint8_t* outcomes, owqs_memory_plan* plan) {
  clear_error();
  if (!h || !plan) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (dtype > OWQS_C128 || mode > OWQS_MODE_EOWQS) return set_error(OWQS_ERR_ARG, "bad option value");
  FixedSource src(h->p, outcomes);
  CompSchedule cs;
  owqs_status st = compile_components(h->p, (int)mode, src, real_input != 0, cs);
  if (st != OWQS_OK) return st;
  const size_t amp = dtype == OWQS_C64 ? 8 : 16;
  std::vector<CompLaunch> launches;
  std::vector<PassDesc> order;
  size_t arena = 0;
  st = plan_components(cs, (int)dtype, amp, real_input != 0, 1ull << h->p.inputs.size(), launches, arena, order);
  if (st != OWQS_OK) return st;
  std::memset(plan, 0, sizeof(*plan));
  plan->peak_m = (uint32_t)cs.peak_m;
  plan->components = (uint32_t)cs.ncomp;
  plan->substate_bytes = (uint64_t)arena;
  plan->one_array_bytes = (uint64_t)cs.single_amps * amp;
  for (const CompLaunch& L : launches) plan->joins += L.type == 2 ? 1u : 0u;
  plan->uses_substates = use_substates(cs) ? 1u : 0u;
  plan->substate_work = cs.work;
  plan->one_array_work = cs.single_work;
  return OWQS_OK;
}

owqs_status owqs_describe_groups(const owqs_pattern* h, uint32_t dtype, uint32_t mode, uint32_t real_input,
                                const uint8_t* outcomes, uint32_t* regs, uint32_t* slots, uint32_t* n_in,
                                uint32_t* specialised, uint32_t cap, uint32_t* ngroups) {
  clear_error();
  if (!h || !ngroups) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (dtype > OWQS_C128 || mode > OWQS_MODE_EOWQS) return set_error(OWQS_ERR_ARG, "bad option value");
  FixedSource src(h->p, outcomes);
  std::vector<PassDesc> passes;
  owqs_status st = compile_schedule(h->p, (int)mode, src, passes);
  if (st != OWQS_OK) return st;
  uint32_t n = 0;
  bool real = real_input != 0;
  if (!small_run_ok(passes)) {
    for (size_t i = 0; i < passes.size(); ++i) {
      GroupParams G;
      LaunchPlan GL;
      int k = 0;
      const int kind = decide_launch(passes, i, (int)dtype, real, false, G, GL, k);
      if (kind == LAUNCH_GROUP) {
        if (n < cap) {
          if (regs) regs[n] = (uint32_t)G.m;
          if (slots) slots[n] = group_sequence_code(G) & 0x8fffffffu;
          if (n_in) n_in[n] = (uint32_t)passes[i].n_in;
          // the launch reads the virtual |+> input only while no array exists
          if (specialised) specialised[n] = group_sequence_specialised(G, (int)dtype, !real) ? 1u : 0u;
        }
        ++n;
      }
      if (kind == LAUNCH_GROUP || kind == LAUNCH_SINGLE) real = true;
      if (kind == LAUNCH_GROUP) i += (size_t)k - 1;
    }
  }
  *ngroups = n;
  return OWQS_OK;
}

owqs_status owqs_describe_launches(const owqs_pattern* h, uint32_t dtype, uint32_t mode, uint32_t real_input,
                                   const uint8_t* outcomes, uint32_t* kind, uint32_t* first_meas, uint32_t* nmeas,
                                   uint32_t cap, uint32_t* nlaunch) {
  clear_error();
  if (!h || !nlaunch) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (dtype > OWQS_C128 || mode > OWQS_MODE_EOWQS) return set_error(OWQS_ERR_ARG, "bad option value");
  FixedSource src(h->p, outcomes);
  std::vector<PassDesc> passes;
  owqs_status st = compile_schedule(h->p, (int)mode, src, passes);
  if (st != OWQS_OK) return st;
  uint32_t n = 0, mi = 0;
  auto put = [&](uint32_t kd, uint32_t first, uint32_t m) {
    if (n < cap) {
      if (kind) kind[n] = kd;
      if (first_meas) first_meas[n] = first;
      if (nmeas) nmeas[n] = m;
    }
    ++n;
  };
  bool real = real_input != 0;
  if (small_run_ok(passes)) {  // one single-block kernel for the whole run
    put(KK_SMALL, 0, (uint32_t)h->p.meas_qubit.size());
    *nlaunch = n;
    return OWQS_OK;
  }
  if (real) put(KK_NORM, 0, 0);  // the input norm (OWQS divides by it, EOWQS checks the output against it)
  for (size_t i = 0; i < passes.size(); ++i) {
    GroupParams G;
    LaunchPlan GL;
    int k = 0;
    switch (decide_launch(passes, i, (int)dtype, real, false, G, GL, k)) {
      case LAUNCH_GROUP:
        put(KK_GROUP, mi, (uint32_t)k);
        mi += (uint32_t)k;
        i += (size_t)k - 1;
        break;
      case LAUNCH_FINAL:
        put(KK_FINAL, mi, 0);
        break;
      case LAUNCH_JOIN:
        put(KK_KRON, mi, 0);
        break;
      default: {
        PassParams P;
        LaunchPlan L;
        plan_pass(passes[i], (int)dtype, !real, P, L);
        put((uint32_t)L.kind, mi, 1);
        ++mi;
      }
    }
    real = true;
  }
  *nlaunch = n;
  return OWQS_OK;
}

owqs_status owqs_get_index_map(const owqs_pattern* h, uint32_t pass, int32_t* bit_of_qubit) {
  clear_error();
  if (!h || !bit_of_qubit) return set_error(OWQS_ERR_ARG, "NULL argument");
  FixedSource zero(h->p, nullptr);
  std::vector<PassDesc> passes;
  std::vector<std::vector<int32_t>> maps;
  owqs_status st = compile_schedule(h->p, OWQS_MODE_EOWQS, zero, passes, &maps);
  if (st != OWQS_OK) return st;
  if (pass >= maps.size()) return set_error(OWQS_ERR_ARG, "pass index out of range");
  std::copy(maps[pass].begin(), maps[pass].end(), bit_of_qubit);
  return OWQS_OK;
}

owqs_status owqs_describe_passes(const owqs_pattern* h, uint32_t mode, const uint8_t* outcomes,
                                 owqs_pass_desc* out, uint32_t cap, uint32_t* npass) {
  clear_error();
  if (!h || !npass || (cap && !out)) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (mode > OWQS_MODE_EOWQS) return set_error(OWQS_ERR_ARG, "bad mode");
  FixedSource src(h->p, outcomes);
  std::vector<PassDesc> passes;
  owqs_status st = compile_schedule(h->p, (int)mode, src, passes);
  if (st != OWQS_OK) return st;
  *npass = (uint32_t)passes.size();
  for (uint32_t i = 0; i < passes.size() && i < cap; ++i) {
    const PassDesc& d = passes[i];
    owqs_pass_desc& o = out[i];
    std::memset(&o, 0, sizeof(o));
    o.kind = d.kind;
    o.n_in = d.n_in;
    o.r = d.r;
    o.b = d.b;
    o.n_out = d.n_out;
    o.outcome = d.outcome;
    o.xmask = d.xmask;
    o.zmask = d.zmask;
    o.c0 = d.c0;
    if (d.edges.size() > 64) return set_error(OWQS_ERR_UNSUPPORTED, "more than 64 sign terms in one pass");
    o.nedges = (uint32_t)d.edges.size();
    for (size_t e = 0; e < d.edges.size(); ++e) {
      o.edges[e][0] = (uint32_t)d.edges[e].first;
      o.edges[e][1] = (uint32_t)d.edges[e].second;
    }
    o.w1re = d.w1re;
    o.w1im = d.w1im;
    o.scale = d.scale;
    for (size_t k = 0; k < d.perm.size() && k < 64; ++k) o.perm[k] = d.perm[k];
  }
  return OWQS_OK;
}

}  // extern "C"
