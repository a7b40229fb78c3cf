// Schedule compiler: turns the active command order into device passes.
//
// Each measurement closes a segment.  The segment's N commands are virtual
// (Section 4.1: a new qubit is a tensor factor |+>; here it becomes a new top
// bit that the pass broadcasts, never materialised), its E, X and Z commands
// are folded into one sign function and one index XOR (Section 4.4.1: CZ
// negates the amplitudes whose two bits are 1, Z negates the bit-1 half, X
// exchanges the halves), and the measurement with elimination (Section 4.2,
// Eqs. 11-13, Fig. 6) combines each amplitude pair that differs in the
// measured bit into one output amplitude.  The surviving qubits keep their
// relative order; bits above the measured one shift down.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "owqs_internal.h"

namespace owqs {

static inline int parity_of(const std::vector<int8_t>& outcome, const std::vector<uint32_t>& dom) {
  int s = 0;
  for (uint32_t d : dom) s ^= outcome[d];
  return s;
}

// 2^(-h/2) with h >= 0, exact up to the final 1/sqrt2 rounding
static inline double pow2_half(int h) {
  return std::ldexp((h & 1) ? M_SQRT1_2 : 1.0, -(h / 2));
}

owqs_status compile_schedule(const Pattern& p, int mode, OutcomeSource& src,
                             std::vector<PassDesc>& passes,
                             std::vector<std::vector<int32_t>>* maps,
                             const std::vector<std::vector<uint32_t>>* factors) {
  passes.clear();
  const uint32_t n = p.n;
  std::vector<int32_t> bit_of(n, -1);
  std::vector<uint32_t> at_bit;
  std::vector<int8_t> outcome(n, 0);
  const bool upfront = src.known_upfront(outcome);
  if (!upfront && !p.deps_ok)
    return set_error(OWQS_ERR_ARG, "sampled outcomes need an order that measures every domain first");
  std::vector<int32_t> factor_of(n, -1);
  std::vector<char> joined;
  if (factors) {
    joined.assign(factors->size(), 0);
    for (size_t f = 0; f < factors->size(); ++f)
      for (uint32_t q : (*factors)[f]) factor_of[q] = (int32_t)f;
  } else {
    for (uint32_t q : p.inputs) {
      bit_of[q] = (int32_t)at_bit.size();
      at_bit.push_back(q);
    }
  }
  if ((int)at_bit.size() > kMaxLive) return set_error(OWQS_ERR_OOM, "more than 62 input qubits");
  int n_in = (int)at_bit.size();
  uint64_t adj[64];
  std::memset(adj, 0, sizeof(adj));
  uint64_t z = 0, x = 0;
  uint32_t c0 = 0;
  if (maps) maps->push_back(bit_of);

  // product input: make factor f live as the top bits (a kind-2 pass)
  auto join = [&](int f) -> bool {
    if (joined[f]) return true;
    joined[f] = 1;
    const std::vector<uint32_t>& qs = (*factors)[f];
    if ((int)(at_bit.size() + qs.size()) > kMaxLive) return false;
    PassDesc d;
    d.kind = 2;
    d.factor = f;
    d.n_in = n_in;
    d.r = (int)qs.size();
    d.n_out = n_in + (int)qs.size();
    for (uint32_t q : qs) {
      bit_of[q] = (int32_t)at_bit.size();
      at_bit.push_back(q);
    }
    n_in = (int)at_bit.size();
    passes.push_back(std::move(d));
    return true;
  };
  // at a segment start: join every factor that the segment touches
  auto join_ahead = [&](size_t from) -> bool {
    for (size_t ai = from; ai < p.active.size(); ++ai) {
      const Cmd& c = p.cmds[p.active[ai]];
      const uint32_t q0 = c.q0, q1 = c.kind == OWQS_CMD_E ? c.q1 : c.q0;
      for (uint32_t q : {q0, q1})
        if (factor_of[q] >= 0 && !join(factor_of[q])) return false;
      if (c.kind == OWQS_CMD_M) break;
    }
    return true;
  };

  bool overflow = false;
  auto touch = [&](uint32_t q) -> int {
    if (bit_of[q] >= 0) return bit_of[q];
    if ((int)at_bit.size() >= kMaxLive) {
      overflow = true;
      return 0;
    }
    bit_of[q] = (int32_t)at_bit.size();
    at_bit.push_back(q);
    return bit_of[q];
  };
  auto edges_of = [&](PassDesc& d, int next) {
    for (int u = 0; u < next; ++u) {
      uint64_t m = adj[u] & ~((2ull << u) - 1);  // partners above u
      while (m) {
        int v = __builtin_ctzll(m);
        m &= m - 1;
        d.edges.emplace_back(u, v);
      }
    }
  };

  bool seg_start = true;
  for (size_t ai = 0; ai < p.active.size(); ++ai) {
    const Cmd& c = p.cmds[p.active[ai]];
    if (factors && seg_start) {
      if (!join_ahead(ai)) return set_error(OWQS_ERR_OOM, "live width above 62 qubits");
      seg_start = false;
    }
    switch (c.kind) {
      case OWQS_CMD_N:
        break;  // prepared at first touch
      case OWQS_CMD_E: {
        int u = touch(c.q0), v = touch(c.q1);
        if (overflow) break;
        adj[u] ^= 1ull << v;
        adj[v] ^= 1ull << u;
        break;
      }
      case OWQS_CMD_Z: {
        int u = touch(c.q0);
        if (overflow) break;
        if (parity_of(outcome, c.sdom)) z ^= 1ull << u;
        break;
      }
      case OWQS_CMD_X: {
        int u = touch(c.q0);
        if (overflow) break;
        // X_u D_q X^m = D_{q(. ^ e_u)} X^{m ^ e_u}: substituting k_u -> k_u ^ 1
        // turns each edge (u,w) into a linear term on w and z_u into a constant
        if (parity_of(outcome, c.sdom)) {
          c0 ^= (uint32_t)((z >> u) & 1u);
          z ^= adj[u];
          x ^= 1ull << u;
        }
        break;
      }
      case OWQS_CMD_M: {
        int b = touch(c.q0);
        if (overflow) break;
        const int next = (int)at_bit.size();
        PassDesc d;
        d.kind = 0;
        d.n_in = n_in;
        d.r = next - n_in;
        d.b = b;
        d.n_out = next - 1;
        d.meas_k = (uint32_t)p.k_of_qubit[c.q0];
        d.xmask = n_in ? (x & ((1ull << n_in) - 1)) : 0;  // X on a |+> qubit is dropped
        d.zmask = z;
        d.c0 = c0;
        edges_of(d, next);
        const int s = parity_of(outcome, c.sdom), t = parity_of(outcome, c.tdom);
        // e^{-i theta}, theta = (-1)^s alpha + t pi (Eq. 2), t pi as an exact sign
        double er = std::cos(c.angle), ei = s ? std::sin(c.angle) : -std::sin(c.angle);
        if (t) er = -er, ei = -ei;
        d.ere = er;
        d.eim = ei;
        d.scale = mode == OWQS_MODE_OWQS ? pow2_half(d.r + 1) : pow2_half(d.r);
        int o = src.decide(d);
        if (o < 0) return OWQS_ERR_CUDA;  // error recorded by the source
        d.outcome = o & 1;
        d.w1re = d.outcome ? -er : er;
        d.w1im = d.outcome ? -ei : ei;
        outcome[c.q0] = (int8_t)d.outcome;
        passes.push_back(std::move(d));
        // eliminate bit b (Section 4.2)
        bit_of[c.q0] = -1;
        at_bit.erase(at_bit.begin() + b);
        for (size_t i = (size_t)b; i < at_bit.size(); ++i) bit_of[at_bit[i]] = (int32_t)i;
        n_in = (int)at_bit.size();
        std::memset(adj, 0, sizeof(adj));
        z = x = 0;
        c0 = 0;
        if (maps) maps->push_back(bit_of);
        seg_start = true;
        break;
      }
      default:
        return set_error(OWQS_ERR_ARG, "unknown command kind");
    }
    if (overflow) return set_error(OWQS_ERR_OOM, "live width above 62 qubits; reorder the pattern");
  }
  if (factors)  // input qubits that no command touches: outputs, joined before the final pass
    for (uint32_t q : p.outputs)
      if (factor_of[q] >= 0 && !join(factor_of[q])) return set_error(OWQS_ERR_OOM, "live width above 62 qubits");
  for (uint32_t q : p.outputs) touch(q);
  if (overflow) return set_error(OWQS_ERR_OOM, "live width above 62 qubits");
  if (at_bit.size() != p.outputs.size())
    return set_error(OWQS_ERR_PATTERN, "live qubits at the end are not the outputs");
  PassDesc f;
  f.kind = 1;
  f.n_in = n_in;
  f.r = (int)at_bit.size() - n_in;
  f.b = -1;
  f.n_out = (int)at_bit.size();
  f.xmask = n_in ? (x & ((1ull << n_in) - 1)) : 0;
  f.zmask = z;
  f.c0 = c0;
  edges_of(f, (int)at_bit.size());
  f.scale = pow2_half(f.r);
  f.perm.resize(p.outputs.size());
  for (size_t k = 0; k < p.outputs.size(); ++k) f.perm[k] = bit_of[p.outputs[k]];
  passes.push_back(std::move(f));
  return OWQS_OK;
}

// ---------------------------------------------------------------------------
// separate sub-states (Section 4.1)
// ---------------------------------------------------------------------------
namespace {
struct Comp {
  std::vector<uint32_t> bits;  // qubit at each bit: [0, nmat) in the array, then prepared (|+>) ones
  int nmat = 0;
  bool arr = false;            // an array exists (nmat qubits; nmat = 0: one amplitude)
  bool alive = true;
  uint64_t adj[64] = {0};      // pending segment, over the bit positions
  uint64_t z = 0, x = 0;
  uint32_t c0 = 0;
  std::vector<CompOp> queue;   // ops not emitted yet
};
}  // namespace

owqs_status compile_components(const Pattern& p, int mode, OutcomeSource& src, bool real_input, CompSchedule& cs) {
  cs = CompSchedule();
  const uint32_t n = p.n;
  std::vector<int8_t> outcome(n, 0);
  if (!src.known_upfront(outcome)) return set_error(OWQS_ERR_UNSUPPORTED, "separate sub-states need outcomes known before the run");
  std::vector<Comp> comps;
  std::vector<int32_t> owner(n, -1);
  auto pos_of = [&](const Comp& c, uint32_t q) -> int {
    for (size_t i = 0; i < c.bits.size(); ++i)
      if (c.bits[i] == q) return (int)i;
    return -1;
  };
  auto new_comp = [&](uint32_t q) -> int {
    comps.emplace_back();
    comps.back().bits.push_back(q);
    owner[q] = (int)comps.size() - 1;
    return owner[q];
  };
  if (real_input) {
    comps.emplace_back();
    Comp& c = comps.back();
    c.bits = p.inputs;
    c.nmat = (int)p.inputs.size();
    c.arr = true;
    for (uint32_t q : p.inputs) owner[q] = 0;
    cs.input_comp = 0;
    if (c.nmat > kMaxLive) return set_error(OWQS_ERR_OOM, "more than 62 input qubits");
  } else {
    for (uint32_t q : p.inputs) new_comp(q);
  }
  // live amplitudes: arrays alive now, and the peak over the run
  uint64_t live = real_input ? (1ull << p.inputs.size()) : 0, peak = live;
  uint64_t single_live_max = 0;  // widest single-array pass (the one-array plan)
  int single_w = (int)p.inputs.size();
  auto flush = [&](int id) {
    for (CompOp& op : comps[id].queue) cs.ops.push_back(std::move(op));
    comps[id].queue.clear();
  };
  auto arr_amps = [&](const Comp& c) -> uint64_t { return c.arr ? (1ull << c.nmat) : 0; };
  // join component b into a; returns the merged id (the one holding an
  // array, so that its array keeps its id)
  auto merge = [&](int a, int b) -> int {
    if (comps[b].arr && !comps[a].arr) std::swap(a, b);
    Comp& A = comps[a];
    Comp& B = comps[b];
    flush(a);
    flush(b);
    std::vector<uint32_t> nb;
    nb.insert(nb.end(), A.bits.begin(), A.bits.begin() + A.nmat);
    nb.insert(nb.end(), B.bits.begin(), B.bits.begin() + B.nmat);
    nb.insert(nb.end(), A.bits.begin() + A.nmat, A.bits.end());
    nb.insert(nb.end(), B.bits.begin() + B.nmat, B.bits.end());
    if ((int)nb.size() > kMaxLive) return -1;
    std::vector<int> posA(A.bits.size()), posB(B.bits.size());
    for (size_t i = 0; i < A.bits.size(); ++i) posA[i] = (int)i < A.nmat ? (int)i : B.nmat + (int)i;
    for (size_t i = 0; i < B.bits.size(); ++i)
      posB[i] = (int)i < B.nmat ? A.nmat + (int)i : (int)A.bits.size() + (int)i;
    uint64_t adj[64] = {0}, z = 0, x = 0;
    auto remap = [&](const Comp& C, const std::vector<int>& pos) {
      for (size_t u = 0; u < C.bits.size(); ++u) {
        for (uint64_t m = C.adj[u]; m; m &= m - 1) adj[pos[u]] |= 1ull << pos[__builtin_ctzll(m)];
        if ((C.z >> u) & 1u) z |= 1ull << pos[u];
        if ((C.x >> u) & 1u) x |= 1ull << pos[u];
      }
    };
    remap(A, posA);
    remap(B, posB);
    if (A.arr && B.arr) {  // tensor product of the two arrays
      CompOp op;
      op.kind = 1;
      op.a = a;
      op.b = b;
      op.n_a = A.nmat;
      op.n_b = B.nmat;
      cs.ops.push_back(op);
      cs.work += std::ldexp(1.0, A.nmat) + std::ldexp(1.0, B.nmat) + std::ldexp(1.0, A.nmat + B.nmat);
      const uint64_t before = live;
      live += 1ull << (A.nmat + B.nmat);
      peak = std::max<uint64_t>(peak, live);
      live = before - arr_amps(A) - arr_amps(B) + (1ull << (A.nmat + B.nmat));
    }
    A.c0 ^= B.c0;
    A.nmat += B.nmat;
    A.arr = A.arr || B.arr;
    A.bits = nb;
    std::memcpy(A.adj, adj, sizeof(adj));
    A.z = z;
    A.x = x;
    for (uint32_t q : B.bits) owner[q] = a;
    B.alive = false;
    B.bits.clear();
    return a;
  };
  auto touch = [&](uint32_t q) -> int {
    if (owner[q] < 0) {
      new_comp(q);
      ++single_w;
    }
    return owner[q];
  };
  for (size_t ai = 0; ai < p.active.size(); ++ai) {
    const Cmd& c = p.cmds[p.active[ai]];
    switch (c.kind) {
      case OWQS_CMD_N:
        break;  // prepared at first touch
      case OWQS_CMD_E: {
        int a = touch(c.q0), b = touch(c.q1);
        if (a != b) {
          a = merge(a, b);
          if (a < 0) return set_error(OWQS_ERR_OOM, "a sub-state wider than 62 qubits; reorder the pattern");
        }
        Comp& C = comps[a];
        const int u = pos_of(C, c.q0), v = pos_of(C, c.q1);
        C.adj[u] ^= 1ull << v;
        C.adj[v] ^= 1ull << u;
        break;
      }
      case OWQS_CMD_Z: {
        Comp& C = comps[touch(c.q0)];
        const int u = pos_of(C, c.q0);
        if (parity_of(outcome, c.sdom)) C.z ^= 1ull << u;
        break;
      }
      case OWQS_CMD_X: {
        Comp& C = comps[touch(c.q0)];
        const int u = pos_of(C, c.q0);
        if (parity_of(outcome, c.sdom)) {  // as in compile_schedule
          C.c0 ^= (uint32_t)((C.z >> u) & 1u);
          C.z ^= C.adj[u];
          C.x ^= 1ull << u;
        }
        break;
      }
      case OWQS_CMD_M: {
        const int id = touch(c.q0);
        Comp& C = comps[id];
        const int b = pos_of(C, c.q0);
        const int width = (int)C.bits.size();
        cs.peak_m = std::max(cs.peak_m, width);
        single_live_max = std::max<uint64_t>(single_live_max, 1ull << std::min(single_w, 62));
        cs.work += (C.arr ? std::ldexp(1.0, C.nmat) : 0.0) + std::ldexp(1.0, width - 1);
        cs.single_work += std::ldexp(1.0, single_w);  // read and write about 2^(w-1) each
        PassDesc d;
        d.kind = 0;
        d.n_in = C.nmat;
        d.r = width - C.nmat;
        d.b = b;
        d.n_out = width - 1;
        d.meas_k = (uint32_t)p.k_of_qubit[c.q0];
        d.xmask = C.nmat ? (C.x & ((1ull << C.nmat) - 1)) : 0;  // X on a |+> qubit is dropped
        d.zmask = C.z;
        d.c0 = C.c0;
        for (int u = 0; u < width; ++u)
          for (uint64_t m = C.adj[u] & ~((2ull << u) - 1); m; m &= m - 1) d.edges.emplace_back(u, __builtin_ctzll(m));
        const int s = parity_of(outcome, c.sdom), t = parity_of(outcome, c.tdom);
        double er = std::cos(c.angle), ei = s ? std::sin(c.angle) : -std::sin(c.angle);
        if (t) er = -er, ei = -ei;
        d.ere = er;
        d.eim = ei;
        d.scale = mode == OWQS_MODE_OWQS ? pow2_half(d.r + 1) : pow2_half(d.r);
        const int o = src.decide(d);
        if (o < 0) return OWQS_ERR_CUDA;
        d.outcome = o & 1;
        d.w1re = d.outcome ? -er : er;
        d.w1im = d.outcome ? -ei : ei;
        outcome[c.q0] = (int8_t)d.outcome;
        CompOp op;
        op.kind = 0;
        op.a = id;
        op.d = std::move(d);
        C.queue.push_back(std::move(op));
        // input and output arrays both live during the pass
        peak = std::max<uint64_t>(peak, live + (1ull << (width - 1)));
        live = live - arr_amps(C) + (1ull << (width - 1));
        C.bits.erase(C.bits.begin() + b);
        C.nmat = (int)C.bits.size();
        C.arr = true;
        std::memset(C.adj, 0, sizeof(C.adj));
        C.z = C.x = 0;
        C.c0 = 0;
        owner[c.q0] = -1;
        --single_w;
        break;
      }
      default:
        return set_error(OWQS_ERR_ARG, "unknown command kind");
    }
  }
  for (uint32_t q : p.outputs) touch(q);
  // join every component (arrays, scalars, |+> outputs) into one
  int last = -1;
  for (int id = 0; id < (int)comps.size(); ++id) {
    if (!comps[id].alive || (!comps[id].arr && comps[id].bits.empty())) continue;
    if (last < 0) {
      last = id;
      continue;
    }
    last = merge(last, id);
    if (last < 0) return set_error(OWQS_ERR_OOM, "live width above 62 qubits at the end");
  }
  if (last < 0) {  // nothing at all: no input, output or measurement
    comps.emplace_back();
    last = (int)comps.size() - 1;
  }
  flush(last);
  Comp& C = comps[last];
  if (C.bits.size() != p.outputs.size())
    return set_error(OWQS_ERR_PATTERN, "live qubits at the end are not the outputs");
  PassDesc f;
  f.kind = 1;
  f.n_in = C.arr ? C.nmat : 0;
  f.r = (int)C.bits.size() - f.n_in;
  f.b = -1;
  f.n_out = (int)C.bits.size();
  f.xmask = f.n_in ? (C.x & ((1ull << f.n_in) - 1)) : 0;
  f.zmask = C.z;
  f.c0 = C.c0;
  for (int u = 0; u < f.n_out; ++u)
    for (uint64_t m = C.adj[u] & ~((2ull << u) - 1); m; m &= m - 1) f.edges.emplace_back(u, __builtin_ctzll(m));
  f.scale = pow2_half(f.r);
  f.perm.resize(p.outputs.size());
  for (size_t k = 0; k < p.outputs.size(); ++k) f.perm[k] = pos_of(C, p.outputs[k]);
  CompOp op;
  op.kind = 2;
  op.a = last;
  op.d = std::move(f);
  cs.ops.push_back(std::move(op));
  peak = std::max<uint64_t>(peak, live + (1ull << p.outputs.size()));
  single_live_max = std::max<uint64_t>(single_live_max, 1ull << std::min<size_t>(p.outputs.size(), 62));
  cs.ncomp = (int)comps.size();
  cs.peak_amps = peak;
  cs.single_amps = 2 * single_live_max;
  return OWQS_OK;
}

// ---------------------------------------------------------------------------
// launch planning
// ---------------------------------------------------------------------------
static int g_max_grid = 0;

int max_grid() {
  if (g_max_grid == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      g_max_grid = sms * 8;  // 8 blocks of 256 threads fill an SM
    else
      g_max_grid = 152 * 8;
  }
  return g_max_grid;
}

static std::atomic<int> g_test_grid_cap{0};
static std::atomic<int> g_test_m4_width{0};

int group_m4_min_width() {
  const int w = g_test_m4_width.load();
  return w > 0 ? w : kGroupM4MinWidth;
}
void set_test_m4_width(int width) { g_test_m4_width.store(width > 0 ? width : 0); }

int test_grid_cap() { return g_test_grid_cap.load(); }
void set_test_grid_cap(int blocks) { g_test_grid_cap.store(blocks > 0 ? blocks : 0); }

int capped_grid(int want) {
  const int cap = g_test_grid_cap.load();
  return (cap > 0 && want > cap) ? cap : want;
}

void fast_config(int dtype, int* lg, int* hint) {
  static int cfg[2][2] = {{-1, -1}, {-1, -1}};
  int d = dtype == OWQS_C64 ? 0 : 1;
  if (cfg[d][0] < 0) {
    // measured on GB300 (brickwork 28x40, 2^28 amplitudes per pass): c64 with
    // 8 outputs (64 bytes) per run 0.730 ms/pass vs 0.769 ms with 4; c128 with
    // 4 outputs 4.44 ms vs 4.65 ms with 2; evict-first hints made no difference
    cfg[0][0] = 3, cfg[0][1] = 0;
    cfg[1][0] = 2, cfg[1][1] = 0;
    if (const char* e = std::getenv(d == 0 ? "OWQS_FAST_C64" : "OWQS_FAST_C128")) {
      int a = -1, b = -1;
      if (std::sscanf(e, "%d,%d", &a, &b) == 2) {
        const bool ok = d == 0 ? (a == 2 || a == 3) : (a == 1 || a == 2);
        if (ok && (b == 0 || b == 1)) cfg[d][0] = a, cfg[d][1] = b;
      }
    }
  }
  *lg = cfg[d][0];
  *hint = cfg[d][1];
}

int tma_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("OWQS_TMA");
    on = (e && e[0] == '0') ? 0 : 1;
  }
  return on;
}


// star adjacency of the measured bit, or false if some E term misses it
static bool star_mask(const PassDesc& d, uint64_t* amask) {
  uint64_t a = 0;
  for (auto& e : d.edges) {
    if (e.first == d.b) a ^= 1ull << e.second;
    else if (e.second == d.b) a ^= 1ull << e.first;
    else return false;
  }
  *amask = a;
  return true;
}

int group_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("OWQS_GROUP");
    on = (e && e[0] == '0') ? 0 : 1;
  }
  return on;
}

// Group planning.  A live entry is a free input bit (code >= 0, its input
// bit while scanning, its free index when planning) or a register slot /
// prepared qubit (code < 0).
int plan_group(const std::vector<PassDesc>& passes, size_t i0, int dtype, GroupParams& G, LaunchPlan& L,
               bool virt_in) {
  if (i0 >= passes.size() || passes[i0].kind != 0) return 0;
  // log2 of a tile in amplitudes: a warp's 4 KB stage (complex64; 8 KB with
  // a 4-qubit register), a block's 32 KB stage (complex128)
  const int tb = group_tile_bits(dtype, 1);
  // a 4-qubit register (one block per SM) only where a launch is long: arrays
  // of at least 2^kGroupM4MinWidth amplitudes (a test hook can lower it)
  const int mmax = dtype != OWQS_C64 ? kGroupRegMaxC128 : (passes[i0].n_in >= group_m4_min_width() ? kGroupRegMax : 3);
  const int n0 = passes[i0].n_in;
  if (n0 < tb || n0 > 62) return 0;
  // scan: the longest valid prefix
  std::vector<int> live(n0);
  for (int x = 0; x < n0; ++x) live[x] = x;
  std::vector<int> regs;
  int best_k = 0;
  for (size_t i = i0; i < passes.size() && (int)(i - i0) < kGroupMax; ++i) {
    const PassDesc& d = passes[i];
    uint64_t a;
    if (d.kind != 0 || d.xmask || d.r != 1 || d.b >= d.n_in || d.n_in != (int)live.size() || !star_mask(d, &a))
      break;
    const int src = live[d.b];
    if (src >= 0) {
      if ((int)regs.size() == mmax) break;
      regs.push_back(src);
    }
    live.erase(live.begin() + d.b);
    live.push_back(-1);
    const int k = (int)(i - i0) + 1, m = (int)regs.size(), lt = group_tile_bits(dtype, m) - m;
    // a 4-qubit register runs one block per SM (8 KB warp stages), where long
    // groups are bound by instruction issue: at most kGroupMaxM4 passes
    if (m == 4 && k > kGroupMaxM4) break;
    if (k >= 2 && n0 - m >= lt) best_k = k;
  }
  if (best_k < 2) return 0;
  // plan the first best_k passes
  regs.clear();
  {
    std::vector<int> lv(n0);
    for (int x = 0; x < n0; ++x) lv[x] = x;
    for (int j = 0; j < best_k; ++j) {
      const PassDesc& d = passes[i0 + j];
      if (lv[d.b] >= 0) regs.push_back(lv[d.b]);
      lv.erase(lv.begin() + d.b);
      lv.push_back(-1);
    }
  }
  const int m = (int)regs.size();
  std::memset(&G, 0, sizeof(G));
  G.k = best_k;
  G.m = m;
  G.lt = group_tile_bits(dtype, m) - m;
  G.nfree = n0 - m;
  std::vector<int> slot_of_input(n0, -1), free_of(n0, -1);
  for (int q = 0; q < m; ++q) slot_of_input[regs[q]] = q, G.B[q] = regs[q];
  {  // low register inputs: inside the tile's contiguous input block
    std::vector<int> sorted(regs);
    std::sort(sorted.begin(), sorted.end());
    int nlow = 0;
    for (int b : sorted)
      if (b < G.lt + nlow) ++nlow;
    std::vector<char> low(m, 0);
    for (int q = 0; q < m; ++q) low[q] = regs[q] < G.lt + nlow;
    G.lowmask = 0;
    for (int q = 0; q < m; ++q)
      if (low[q]) G.lowmask |= 1u << regs[q];
    G.nruns = 1 << (m - nlow);
    G.runlen = 1u << (G.lt + nlow);
    for (int c = 0; c < (1 << m); ++c) {
      uint32_t run = 0, lowoff = 0;
      int rank = 0;
      for (int q = 0; q < m; ++q) {
        const uint32_t bit = (c >> q) & 1u;
        if (low[q]) lowoff |= bit << regs[q];
        else run |= bit << rank++;
      }
      G.cbase[c] = run * G.runlen + lowoff;
    }
    for (int r = 0; r < G.nruns; ++r) {
      uint64_t off = 0;
      int rank = 0;
      for (int q = 0; q < m; ++q)
        if (!low[q]) off |= (uint64_t)((r >> rank++) & 1) << regs[q];
      G.runoff[r] = off;
    }
  }
  for (int x = 0, f = 0; x < n0; ++x)
    if (slot_of_input[x] < 0) free_of[x] = f++;
  std::vector<int> lv(n0);
  for (int x = 0; x < n0; ++x) lv[x] = slot_of_input[x] >= 0 ? -(1 + slot_of_input[x]) : free_of[x];
  const uint32_t lomask = (1u << G.lt) - 1u;
  uint32_t pend = 0;  // register-diagonal sign mask carried by the scaled register
  double prod = 1.0;
  G.half = 1;
  for (int j = 0; j < best_k; ++j) {
    const PassDesc& d = passes[i0 + j];
    uint64_t A = 0;
    star_mask(d, &A);
    // bit n_in of the output index is the qubit this pass prepares
    if (!((A >> d.n_in) & 1u)) G.half = 0;
    GroupPass& P = G.pass[j];
    const int s = -lv[d.b] - 1;
    P.slot = s;
    P.c0 = d.c0 & 1u;
    P.zb = (uint32_t)((d.zmask >> d.b) & 1u);
    for (int l = 0; l <= d.n_in; ++l) {  // l = n_in: the prepared qubit, which takes slot s
      if (l == d.b) continue;
      const uint32_t zbit = (uint32_t)((d.zmask >> l) & 1u), abit = (uint32_t)((A >> l) & 1u);
      if (!zbit && !abit) continue;
      const int code = l < d.n_in ? lv[l] : -(1 + s);
      if (code >= 0) {
        P.zfree |= (uint64_t)zbit << code;
        P.afree |= (uint64_t)abit << code;
      } else {
        const int t = -code - 1;
        P.zr ^= zbit << t;
        P.ar ^= abit << t;
      }
    }
    P.zlo = (uint32_t)(P.zfree & lomask);
    P.alo = (uint32_t)(P.afree & lomask);
    P.scale = d.scale;
    P.wre = d.w1re;
    P.wim = d.w1im;
    const uint32_t ps = (pend >> s) & 1u;
    for (int g = 0; g < (1 << kGroupRegMax); ++g) {
      P.ct[g] = ((__builtin_popcount(P.ar & (uint32_t)g) & 1u) ^ ps) ? -1.0f : 1.0f;
      if (g < (1 << kGroupRegMaxC128)) P.ctd[g] = P.ct[g];
    }
    P.fwr = (float)d.w1re;
    P.fwi = (float)d.w1im;
    G.zall ^= P.zfree;
    G.c0all ^= P.c0;
    pend = P.zr ^ (pend & ~(1u << s));
    prod *= d.scale;
    G.nscale[j] = prod * prod;
    lv.erase(lv.begin() + d.b);
    lv.push_back(-(1 + s));
  }
  G.zall_lo = (uint32_t)(G.zall & lomask);
  // final order: the free bits in order, then the register slots
  for (int f = 0; f < G.nfree; ++f)
    if (lv[f] != f) return 0;  // cannot happen: free bits are never removed and keep their order
  for (int g = 0; g < (1 << m); ++g) {
    uint64_t off = 0;
    for (int l = G.nfree; l < n0; ++l) {
      const int t = -lv[l] - 1;
      if ((g >> t) & 1) off |= 1ull << l;
    }
    G.outoff[g] = off;
    const double f = ((__builtin_popcount(pend & (uint32_t)g) & 1u) ? -1.0 : 1.0) * prod;
    if (g < (1 << kGroupRegMaxC128)) G.find[g] = f;
    G.fin[g] = (float)f;
  }
  G.norm_in = G.norm_out = -1;
  L.kind = KK_GROUP;
  G.vconst = virt_in ? std::ldexp((n0 & 1) ? M_SQRT1_2 : 1.0, -(n0 / 2)) : 0.0;
  L.bytes = ((virt_in ? 0.0 : std::ldexp(1.0, n0)) + std::ldexp(1.0, passes[i0 + best_k - 1].n_out)) *
            (dtype == OWQS_C64 ? 8.0 : 16.0);
  L.grid = 1;
  return best_k;
}

static inline uint64_t ins0(uint64_t j, int b) {  // insert a 0 bit at position b
  return ((j >> b) << (b + 1)) | (j & ((1ull << b) - 1));
}

static inline uint32_t par64(uint64_t v) { return (uint32_t)__builtin_parityll(v); }

void plan_pass(const PassDesc& d, int dtype, bool virt_in, PassParams& P, LaunchPlan& L) {
  std::memset(&P, 0, sizeof(P));
  P.n_in = d.n_in;
  P.r = d.r;
  P.b = d.b;
  P.n_out = d.n_out;
  P.norm_in = -1;
  P.norm_out = -1;
  P.xmask = d.xmask;
  P.zmask = d.zmask;
  P.c0 = d.c0;
  P.scale = d.scale;
  P.w1re = d.w1re;
  P.w1im = d.w1im;
  P.ere = d.ere;
  P.eim = d.eim;
  P.vconst = virt_in ? std::ldexp((d.n_in & 1) ? M_SQRT1_2 : 1.0, -(d.n_in / 2)) : 0.0;
  const double amp = dtype == OWQS_C64 ? 8.0 : 16.0;
  const double in_elems = virt_in ? 0.0 : std::ldexp(1.0, d.n_in);
  L.bytes = (in_elems + std::ldexp(1.0, d.n_out)) * amp;
  L.block = kBlock;

  // star form: every quadratic term contains the measured bit
  bool star = d.kind == 0;
  uint64_t amask = 0;
  for (auto& e : d.edges) {
    if (d.kind == 0 && (e.first == d.b || e.second == d.b)) {
      amask ^= 1ull << (e.first == d.b ? e.second : e.first);
    } else {
      star = false;
    }
  }
  // generic quadratic cover: greedy, highest remaining degree first
  {
    std::vector<std::pair<int, int>> rest = d.edges;
    int nq = 0;
    while (!rest.empty() && nq < kQMax) {
      int deg[64] = {0};
      for (auto& e : rest) deg[e.first]++, deg[e.second]++;
      int best = 0;
      for (int u = 1; u < 64; ++u)
        if (deg[u] > deg[best]) best = u;
      uint64_t m = 0;
      std::vector<std::pair<int, int>> keep;
      for (auto& e : rest) {
        if (e.first == best) m ^= 1ull << e.second;
        else if (e.second == best) m ^= 1ull << e.first;
        else keep.push_back(e);
      }
      P.qu[nq] = best;
      P.qa[nq] = m;
      ++nq;
      rest.swap(keep);
    }
    P.nq = nq;  // a graph on at most 62 bits has a vertex cover below 64
  }

  int Lg = 2, hint = 0;
  fast_config(dtype, &Lg, &hint);
  if (d.kind == 1) {
    L.kind = KK_FINAL;
    bool ident = true;
    for (size_t k = 0; k < d.perm.size(); ++k) {
      P.perm[k] = d.perm[k];
      if (d.perm[k] != (int)k) ident = false;
    }
    P.identity_perm = ident ? 1 : 0;
    uint64_t elems = 1ull << d.n_out;
    L.grid = (int)std::min<uint64_t>((elems + kBlock - 1) / kBlock, (uint64_t)max_grid());
    return;
  }
  const bool b_new = d.b >= d.n_in;
  const int nlo = b_new ? d.n_in : d.n_in - 1;
  const bool fast = !virt_in && d.xmask == 0 && star && nlo >= Lg &&
                    (b_new || d.b >= Lg || d.n_in >= Lg + 1);
  if (!fast) {
    L.kind = KK_GENERIC;
    uint64_t elems = 1ull << d.n_out;
    L.grid = (int)std::min<uint64_t>((elems + kBlock - 1) / kBlock, (uint64_t)max_grid());
    return;
  }
  P.nlo = nlo;
  // complex64 only: the complex128 pass is bound by the FP64 rate, where the
  // register-tiled kernel's larger thread count wins (GB300: 4.43 vs 5.15 ms
  // per 2^28 pass; complex64 0.733 vs 0.751 ms in favour of TMA)
  const int lte = kTmaLogTileC64;
  if (tma_enabled() && dtype == OWQS_C64 && nlo >= lte) {
    // whole tiles of 2^lte live outputs: the TMA-pipelined pass
    L.kind = KK_TMA;
    L.variant = b_new ? 2 : (d.b >= lte ? 1 : 0);
    P.amask = amask;
    P.zb = (uint32_t)((d.zmask >> d.b) & 1u);
    P.rt = 0;
    uint64_t tiles = 1ull << (nlo - lte);
    L.grid = (int)std::min<uint64_t>(tiles, (uint64_t)max_grid());
    return;
  }
  L.kind = KK_FAST;
  L.lg = Lg;
  L.hint = hint;
  L.variant = b_new ? Lg + 1 : (d.b >= Lg ? Lg : d.b);
  const int nbc = d.n_out - nlo;
  P.rt = std::min(nbc, kFastRMax);
  P.amask = amask;
  P.zb = (uint32_t)((d.zmask >> d.b) & 1u);
  for (int l = 0; l < (1 << Lg); ++l) {
    uint64_t dl = ins0((uint64_t)l, d.b);
    P.tzl |= par64(dl & d.zmask) << l;
    P.tal |= par64(dl & amask) << l;
  }
  for (int t = 0; t < (1 << P.rt); ++t) {
    uint64_t dt = ins0((uint64_t)t << nlo, d.b);
    P.tzt |= par64(dt & d.zmask) << t;
    P.tat |= par64(dt & amask) << t;
  }
  uint64_t tiles = 1ull << (d.n_out - Lg - P.rt);
  L.grid = (int)std::min<uint64_t>((tiles + kBlock - 1) / kBlock, (uint64_t)max_grid());
}

}  // namespace owqs
