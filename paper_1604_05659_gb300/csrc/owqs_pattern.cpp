// Pattern model, well-formedness (D0-D3), reordering (PROA) and order
// management of the GB300 one-way quantum computer simulator.
//
// Section 2.2: P = (V, I, O, A), commands N, E, M, X, Z; rules D0-D3;
// standard form CME.  Section 4.3: Proposition (Eqs. 14-17) and the greedy
// reordering with the Eq. 18 cost, swept as in Section 5.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include "owqs_internal.h"

namespace owqs {

static thread_local std::string g_last_error;

owqs_status set_error(owqs_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
void clear_error() { g_last_error.clear(); }

Pattern::~Pattern() = default;

// ---------------------------------------------------------------------------
// D0-D3 (Section 2.2).  Non-input qubits without an explicit N are prepared
// before the first command.
// ---------------------------------------------------------------------------
static owqs_status validate(const Pattern& p) {
  const uint32_t n = p.n;
  std::vector<char> is_in(n, 0), is_out(n, 0), explicit_n(n, 0), prepared(n, 0), measured(n, 0),
      seen_n(n, 0);
  for (uint32_t q : p.inputs) {
    if (q >= n) return set_error(OWQS_ERR_ARG, "input label out of range");
    if (is_in[q]) return set_error(OWQS_ERR_ARG, "duplicate input qubit");
    is_in[q] = 1;
  }
  for (uint32_t q : p.outputs) {
    if (q >= n) return set_error(OWQS_ERR_ARG, "output label out of range");
    if (is_out[q]) return set_error(OWQS_ERR_ARG, "duplicate output qubit");
    is_out[q] = 1;
  }
  for (const Cmd& c : p.cmds)
    if (c.kind == OWQS_CMD_N && c.q0 < n) explicit_n[c.q0] = 1;
  for (uint32_t q = 0; q < n; ++q) prepared[q] = is_in[q] || !explicit_n[q];
  for (size_t i = 0; i < p.cmds.size(); ++i) {
    const Cmd& c = p.cmds[i];
    const std::string at = "command " + std::to_string(i) + ": ";
    if (c.kind > OWQS_CMD_Z) return set_error(OWQS_ERR_ARG, at + "unknown kind");
    const bool two = c.kind == OWQS_CMD_E;
    if (c.q0 >= n || (two && c.q1 >= n)) return set_error(OWQS_ERR_ARG, at + "qubit out of range");
    if (two && c.q0 == c.q1) return set_error(OWQS_ERR_PATTERN, at + "E on a single qubit");
    for (const auto* dom : {&c.sdom, &c.tdom})
      for (uint32_t d : *dom) {
        if (d >= n) return set_error(OWQS_ERR_ARG, at + "domain qubit out of range");
        if (!measured[d]) return set_error(OWQS_ERR_PATTERN, at + "D0: depends on an unmeasured qubit");
      }
    if (measured[c.q0] || (two && measured[c.q1]))
      return set_error(OWQS_ERR_PATTERN, at + "D1: acts on a measured qubit");
    if (c.kind == OWQS_CMD_N) {
      if (is_in[c.q0] || seen_n[c.q0])
        return set_error(OWQS_ERR_PATTERN, at + "N on an input or an already prepared qubit");
      seen_n[c.q0] = 1;
      prepared[c.q0] = 1;
      continue;
    }
    if (!prepared[c.q0] || (two && !prepared[c.q1]))
      return set_error(OWQS_ERR_PATTERN, at + "D2: acts on a qubit before its N");
    if (c.kind == OWQS_CMD_M) measured[c.q0] = 1;
  }
  for (uint32_t q = 0; q < n; ++q)
    if ((bool)measured[q] == (bool)is_out[q])
      return set_error(OWQS_ERR_PATTERN,
                       "D3: qubit " + std::to_string(q) + " is measured iff it is an output");
  return OWQS_OK;
}

static bool is_standard(const Pattern& p) {
  int last = 0;
  for (const Cmd& c : p.cmds) {
    int r = (c.kind == OWQS_CMD_N || c.kind == OWQS_CMD_E) ? 0 : (c.kind == OWQS_CMD_M ? 1 : 2);
    if (r < last) return false;
    last = r;
  }
  return true;
}

static void set_active_loaded(Pattern& p) {
  ++p.order_version;
  p.active.resize(p.cmds.size());
  std::iota(p.active.begin(), p.active.end(), 0u);
  p.active_meas.clear();
  for (const Cmd& c : p.cmds)
    if (c.kind == OWQS_CMD_M) p.active_meas.push_back(c.q0);
}

// total + 2^w, saturating at 2^64 - 1 (orders wider than 63 live qubits
// cannot be simulated anyway; their count only has to compare as huge).
static inline uint64_t add_pow2_sat(uint64_t total, uint32_t w) {
  if (w >= 64) return UINT64_MAX;
  uint64_t add = 1ull << w;
  return total > UINT64_MAX - add ? UINT64_MAX : total + add;
}

// Live width and amplitude updates of the active order.  A qubit joins the
// live array just before the first command that touches it (N commutes with
// commands on other qubits); every command counts 2^(live width), N after the
// qubit is added, M before it is removed.
void order_stats(const Pattern& p, uint32_t* peak_live, uint64_t* amp_updates) {
  std::vector<char> live(p.n, 0);
  uint32_t w = 0;
  for (uint32_t q : p.inputs) live[q] = 1, ++w;
  uint32_t peak = w;
  uint64_t total = 0;
  auto touch = [&](uint32_t q) {
    if (!live[q]) {
      live[q] = 1;
      ++w;
      total = add_pow2_sat(total, w);
    }
  };
  for (uint32_t idx : p.active) {
    const Cmd& c = p.cmds[idx];
    if (c.kind == OWQS_CMD_N) continue;  // prepared at first touch
    touch(c.q0);
    if (c.kind == OWQS_CMD_E) touch(c.q1);
    peak = std::max(peak, w);
    total = add_pow2_sat(total, w);
    if (c.kind == OWQS_CMD_M) live[c.q0] = 0, --w;
  }
  for (uint32_t q : p.outputs) touch(q);
  peak = std::max(peak, w);
  if (peak_live) *peak_live = peak;
  if (amp_updates) *amp_updates = total;
}

// ---------------------------------------------------------------------------
// Order from a measurement sequence (Eq. 17): for each v, the E commands on v
// not yet applied (load order), then M_v; afterwards the remaining E commands
// and the corrections in load order.  N commands are dropped: every qubit is
// prepared just in time.
// ---------------------------------------------------------------------------
owqs_status build_active_order(Pattern& p, const std::vector<uint32_t>& order, bool need_deps) {
  const uint32_t n = p.n;
  std::vector<int32_t> m_idx(n, -1);
  std::vector<std::vector<uint32_t>> e_of(n);
  std::vector<uint32_t> corr, e_all;
  for (uint32_t i = 0; i < p.cmds.size(); ++i) {
    const Cmd& c = p.cmds[i];
    if (c.kind == OWQS_CMD_M) m_idx[c.q0] = (int32_t)i;
    else if (c.kind == OWQS_CMD_E) {
      e_of[c.q0].push_back(i);
      e_of[c.q1].push_back(i);
      e_all.push_back(i);
    } else if (c.kind == OWQS_CMD_X || c.kind == OWQS_CMD_Z) corr.push_back(i);
  }
  if (order.size() != p.meas_qubit.size()) return set_error(OWQS_ERR_ARG, "order must list every measured qubit once");
  std::vector<char> done(n, 0);
  bool deps_ok = true;
  for (uint32_t v : order) {
    if (v >= n || m_idx[v] < 0 || done[v]) return set_error(OWQS_ERR_ARG, "order must list every measured qubit once");
    const Cmd& m = p.cmds[m_idx[v]];
    for (const auto* dom : {&m.sdom, &m.tdom})
      for (uint32_t d : *dom)
        if (!done[d]) deps_ok = false;
    done[v] = 1;
  }
  if (need_deps && !deps_ok) return set_error(OWQS_ERR_ARG, "order measures a qubit before its dependencies");
  std::vector<char> used(p.cmds.size(), 0);
  std::vector<uint32_t> act;
  act.reserve(p.cmds.size());
  for (uint32_t v : order) {
    for (uint32_t i : e_of[v])
      if (!used[i]) used[i] = 1, act.push_back(i);
    act.push_back((uint32_t)m_idx[v]);
  }
  for (uint32_t i : e_all)
    if (!used[i]) act.push_back(i);
  for (uint32_t i : corr) act.push_back(i);
  p.active.swap(act);
  p.active_meas = order;
  p.deps_ok = deps_ok;
  ++p.order_version;
  return OWQS_OK;
}

// ---------------------------------------------------------------------------
// PROA (Section 4.3)
// ---------------------------------------------------------------------------
ReorderGraph build_reorder_graph(const Pattern& p, bool eowqs) {
  ReorderGraph g;
  g.n = p.n;
  const uint32_t n = p.n;
  std::vector<std::set<uint32_t>> adj(n), pend(n), dependents(n);
  for (const Cmd& c : p.cmds) {
    if (c.kind == OWQS_CMD_E) {
      adj[c.q0].insert(c.q1);
      adj[c.q1].insert(c.q0);
      auto tog = [&](uint32_t a, uint32_t b) {
        if (!pend[a].erase(b)) pend[a].insert(b);
      };
      tog(c.q0, c.q1);
      tog(c.q1, c.q0);
    }
    if (c.kind == OWQS_CMD_M || c.kind == OWQS_CMD_X || c.kind == OWQS_CMD_Z) {
      for (uint32_t d : c.sdom) dependents[d].insert(c.q0);
      for (uint32_t d : c.tdom) dependents[d].insert(c.q0);
    }
  }
  std::vector<char> is_out(n, 0);
  for (uint32_t o : p.outputs) is_out[o] = 1;
  g.adj.resize(n);
  g.pending0.resize(n);
  g.os.assign(n, 0);
  g.ss.assign(n, 0);
  g.deps.resize(n);
  g.rdeps.resize(n);
  g.is_meas.assign(n, 0);
  for (uint32_t q = 0; q < n; ++q) {
    g.adj[q].assign(adj[q].begin(), adj[q].end());
    g.pending0[q].assign(pend[q].begin(), pend[q].end());
    for (uint32_t u : adj[q]) g.os[q] += is_out[u];
    g.ss[q] = eowqs ? 0u : (uint32_t)dependents[q].size();
  }
  for (const Cmd& c : p.cmds)
    if (c.kind == OWQS_CMD_M) {
      g.measured.push_back(c.q0);
      g.is_meas[c.q0] = 1;
      if (!eowqs) {
        std::set<uint32_t> d(c.sdom.begin(), c.sdom.end());
        d.insert(c.tdom.begin(), c.tdom.end());
        g.deps[c.q0].assign(d.begin(), d.end());
        for (uint32_t x : d) g.rdeps[x].push_back(c.q0);
      }
    }
  return g;
}

namespace {

struct GreedyResult {
  std::vector<uint32_t> order, ms;
};

GreedyResult greedy(const ReorderGraph& g, const std::vector<uint32_t>& inputs, bool product_input,
                    double a, double b, double gm, double d) {
  const uint32_t n = g.n;
  std::vector<uint32_t> parent(n), size(n, 1);
  std::iota(parent.begin(), parent.end(), 0u);
  auto find = [&](uint32_t x) {
    while (parent[x] != x) {
      parent[x] = parent[parent[x]];
      x = parent[x];
    }
    return x;
  };
  auto merge = [&](uint32_t x, uint32_t y) {
    uint32_t rx = find(x), ry = find(y);
    if (rx == ry) return;
    uint32_t root = std::min(rx, ry), other = std::max(rx, ry);
    parent[other] = root;
    size[root] += size[other];
  };
  if (!product_input)
    for (size_t i = 1; i < inputs.size(); ++i) merge(inputs[0], inputs[i]);
  std::vector<std::vector<uint32_t>> pending = g.pending0;
  std::vector<char> selected(n, 0);
  std::vector<uint32_t> unresolved(n, 0);
  std::set<uint32_t> ready;
  for (uint32_t v : g.measured) {
    unresolved[v] = (uint32_t)g.deps[v].size();
    if (unresolved[v] == 0) ready.insert(v);
  }
  GreedyResult res;
  res.order.reserve(g.measured.size());
  std::vector<uint32_t> roots;
  while (!ready.empty()) {
    uint32_t best_v = 0, best_ms = 0;
    double best_cost = 0;
    bool have = false;
    for (uint32_t v : ready) {
      roots.clear();
      roots.push_back(find(v));
      for (uint32_t u : pending[v]) roots.push_back(find(u));
      std::sort(roots.begin(), roots.end());
      roots.erase(std::unique(roots.begin(), roots.end()), roots.end());
      uint32_t ms = 0;
      for (uint32_t r : roots) ms += size[r];
      bool flag = false;
      for (uint32_t u : g.adj[v])
        if (selected[u]) { flag = true; break; }
      double cost = flag ? a * ms + b * g.os[v] - gm * g.ss[v]
                         : a * ((ms + 1) * d) + b * g.os[v] - gm * g.ss[v];
      if (!have || cost < best_cost) {
        have = true;
        best_cost = cost;
        best_v = v;
        best_ms = ms;
      }
    }
    const uint32_t v = best_v;
    for (uint32_t u : pending[v]) {
      merge(v, u);
      auto& pu = pending[u];
      pu.erase(std::remove(pu.begin(), pu.end(), v), pu.end());
    }
    pending[v].clear();
    size[find(v)] -= 1;  // v is eliminated from its sub-state
    selected[v] = 1;
    res.order.push_back(v);
    res.ms.push_back(best_ms);
    ready.erase(v);
    for (uint32_t w : g.rdeps[v])
      if (--unresolved[w] == 0) ready.insert(w);
  }
  return res;
}

}  // namespace

}  // namespace owqs

using namespace owqs;

extern "C" {

uint32_t owqs_abi_version(void) { return OWQS_ABI_VERSION; }

const char* owqs_last_error(void) { return g_last_error.c_str(); }

owqs_status owqs_load_pattern(uint32_t nqubits, const uint32_t* inputs, uint32_t nin,
                              const uint32_t* outputs, uint32_t nout, const owqs_cmd* cmds,
                              size_t ncmd, const uint32_t* domain, size_t ndomain,
                              owqs_pattern** out) {
  clear_error();
  if (!out) return set_error(OWQS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nqubits == 0 || nqubits > (1u << 24)) return set_error(OWQS_ERR_ARG, "nqubits out of range");
  if ((nin && !inputs) || (nout && !outputs) || (ncmd && !cmds) || (ndomain && !domain))
    return set_error(OWQS_ERR_ARG, "NULL array with nonzero length");
  auto* h = new (std::nothrow) owqs_pattern();
  if (!h) return set_error(OWQS_ERR_OOM, "host allocation failed");
  Pattern& p = h->p;
  p.n = nqubits;
  p.inputs.assign(inputs, inputs + nin);
  p.outputs.assign(outputs, outputs + nout);
  p.cmds.resize(ncmd);
  for (size_t i = 0; i < ncmd; ++i) {
    const owqs_cmd& c = cmds[i];
    Cmd& d = p.cmds[i];
    d.kind = c.kind;
    d.q0 = c.q0;
    d.q1 = c.q1;
    d.angle = c.angle;
    if (!std::isfinite(c.angle)) {
      delete h;
      return set_error(OWQS_ERR_ARG, "command " + std::to_string(i) + ": angle is not finite");
    }
    auto take = [&](uint32_t off, uint32_t len, std::vector<uint32_t>& dst) {
      if ((size_t)off + len > ndomain) return false;
      dst.assign(domain + off, domain + off + len);
      return true;
    };
    bool ok = true;
    if (c.kind == OWQS_CMD_M) ok = take(c.s_off, c.s_len, d.sdom) && take(c.t_off, c.t_len, d.tdom);
    else if (c.kind == OWQS_CMD_X || c.kind == OWQS_CMD_Z) ok = take(c.s_off, c.s_len, d.sdom);
    if (!ok) {
      delete h;
      return set_error(OWQS_ERR_ARG, "command " + std::to_string(i) + ": domain range out of bounds");
    }
  }
  owqs_status st = validate(p);
  if (st != OWQS_OK) {
    delete h;
    return st;
  }
  p.k_of_qubit.assign(nqubits, -1);
  for (const Cmd& c : p.cmds)
    if (c.kind == OWQS_CMD_M) {
      p.k_of_qubit[c.q0] = (int32_t)p.meas_qubit.size();
      p.meas_qubit.push_back(c.q0);
    }
  p.standard = is_standard(p);
  set_active_loaded(p);
  *out = h;
  return OWQS_OK;
}

void owqs_free_pattern(owqs_pattern* h) { delete h; }

owqs_status owqs_get_info(const owqs_pattern* h, owqs_pattern_info* info) {
  clear_error();
  if (!h || !info) return set_error(OWQS_ERR_ARG, "NULL argument");
  const Pattern& p = h->p;
  info->nqubits = p.n;
  info->nin = (uint32_t)p.inputs.size();
  info->nout = (uint32_t)p.outputs.size();
  info->nmeas = (uint32_t)p.meas_qubit.size();
  info->standard = p.standard ? 1u : 0u;
  order_stats(p, &info->peak_live, &info->amp_updates);
  return OWQS_OK;
}

owqs_status owqs_reorder(owqs_pattern* h, const owqs_reorder_opts* o, owqs_reorder_info* info,
                         uint32_t* order_out) {
  clear_error();
  if (!h || !o) return set_error(OWQS_ERR_ARG, "NULL argument");
  Pattern& p = h->p;
  if (!p.standard) return set_error(OWQS_ERR_NOT_STANDARD, "reordering needs the standard form (E, then M, then X/Z)");
  if (o->mode > OWQS_MODE_EOWQS) return set_error(OWQS_ERR_ARG, "bad mode");
  if (o->use_learned && !o->model) return set_error(OWQS_ERR_ARG, "use_learned needs a model");
  const bool eowqs = o->mode == OWQS_MODE_EOWQS;
  ReorderGraph g = build_reorder_graph(p, eowqs);
  std::vector<std::array<double, 4>> runs;
  const double k = std::max<double>(1.0, (double)p.outputs.size());
  if (o->sweep) {
    if (p.outputs.empty()) runs.push_back({1.0, k, 0.5, k});
    for (int a = (int)p.outputs.size(); a >= 1; --a) runs.push_back({(double)a, k, 0.5, k});
  } else {
    if (!(o->alpha > 0 && o->beta > 0 && o->gamma > 0 && o->delta > 0))
      return set_error(OWQS_ERR_ARG, "Eq. 18 weights must be positive");
    runs.push_back({o->alpha, o->beta, o->gamma, o->delta});
  }
  GreedyResult best;
  uint32_t best_peak = 0;
  unsigned __int128 best_sum = 0;
  double best_a = 0;
  bool have = false;
  for (const auto& w : runs) {
    GreedyResult r = greedy(g, p.inputs, o->product_input != 0, w[0], w[1], w[2], w[3]);
    if (r.order.size() != g.measured.size())
      return set_error(OWQS_ERR_PATTERN, "dependency cycle: no ready qubit");
    uint32_t peak = 0;
    unsigned __int128 sum = 0;
    for (uint32_t m : r.ms) {
      peak = std::max(peak, m);
      sum += (unsigned __int128)1 << std::min<uint32_t>(m, 126);
    }
    if (!have || peak < best_peak || (peak == best_peak && sum < best_sum)) {
      have = true;
      best = std::move(r);
      best_peak = peak;
      best_sum = sum;
      best_a = w[0];
    }
  }
  owqs_status st = build_active_order(p, best.order, !eowqs);
  if (st != OWQS_OK) return st;
  uint32_t g_peak = 0, l_peak = 0;
  uint64_t g_upd = 0, l_upd = 0;
  order_stats(p, &g_peak, &g_upd);
  bool accepted = false, best_owqs = false;
  std::vector<uint32_t> lorder;
  if (o->use_learned && eowqs) {
    // with preselected outcomes an order that waits for every domain is
    // valid too: the greedy OWQS sweep order is a candidate too
    ReorderGraph g2 = build_reorder_graph(p, false);
    GreedyResult b2;
    uint32_t b2_peak = 0;
    unsigned __int128 b2_sum = 0;
    bool have2 = false;
    for (int a = std::max<int>(1, (int)p.outputs.size()); a >= 1; --a) {
      GreedyResult r = greedy(g2, p.inputs, o->product_input != 0, (double)a, k, 0.5, k);
      if (r.order.size() != g2.measured.size()) break;  // a dependency cycle: no OWQS order
      uint32_t pk = 0;
      unsigned __int128 sum = 0;
      for (uint32_t m : r.ms) {
        pk = std::max(pk, m);
        sum += (unsigned __int128)1 << std::min<uint32_t>(m, 126);
      }
      if (!have2 || pk < b2_peak || (pk == b2_peak && sum < b2_sum)) {
        have2 = true;
        b2 = std::move(r);
        b2_peak = pk;
        b2_sum = sum;
      }
    }
    if (have2) {
      st = build_active_order(p, b2.order, true);
      if (st != OWQS_OK) return st;
      uint32_t o_peak = 0;
      uint64_t o_upd = 0;
      order_stats(p, &o_peak, &o_upd);
      if (o_peak < g_peak || (o_peak == g_peak && o_upd < g_upd)) {
        best_owqs = true;
        best = std::move(b2);
        best_peak = b2_peak;
        g_peak = o_peak;
        g_upd = o_upd;
      } else {
        st = build_active_order(p, best.order, !eowqs);
        if (st != OWQS_OK) return st;
      }
    }
  }
  if (o->use_learned) {
    // the proposal is checked against the best greedy order: kept only if its peak
    // live width and amplitude updates are no worse
    st = learned_order(p, o->model, eowqs, o->product_input != 0, lorder);
    if (st != OWQS_OK) return st;
    st = build_active_order(p, lorder, !eowqs);
    if (st != OWQS_OK) return st;
    order_stats(p, &l_peak, &l_upd);
    accepted = l_peak < g_peak || (l_peak == g_peak && l_upd <= g_upd);
    if (!accepted) {
      st = build_active_order(p, best.order, !eowqs);
      if (st != OWQS_OK) return st;
    }
  }
  const std::vector<uint32_t>& chosen = accepted ? lorder : best.order;
  if (order_out) std::copy(chosen.begin(), chosen.end(), order_out);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->peak_m = best_peak;  // Table I/III m of the greedy order
    order_stats(p, &info->peak_live, &info->amp_updates);
    info->alpha_used = best_a;
    info->learned_accepted = accepted ? 1u : 0u;
    info->greedy_peak_live = g_peak;
    info->greedy_amp_updates = g_upd;
    info->learned_peak_live = l_peak;
    info->learned_amp_updates = l_upd;
    info->greedy_best_owqs = best_owqs ? 1u : 0u;
  }
  return OWQS_OK;
}

owqs_status owqs_set_order(owqs_pattern* h, const uint32_t* order, uint32_t k) {
  clear_error();
  if (!h || (k && !order)) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (!h->p.standard) return set_error(OWQS_ERR_NOT_STANDARD, "setting an order needs the standard form");
  return build_active_order(h->p, std::vector<uint32_t>(order, order + k), true);
}

owqs_status owqs_reset_order(owqs_pattern* h) {
  clear_error();
  if (!h) return set_error(OWQS_ERR_ARG, "NULL argument");
  set_active_loaded(h->p);
  h->p.deps_ok = true;
  return OWQS_OK;
}

owqs_status owqs_get_order(const owqs_pattern* h, uint32_t* order) {
  clear_error();
  if (!h || !order) return set_error(OWQS_ERR_ARG, "NULL argument");
  std::copy(h->p.active_meas.begin(), h->p.active_meas.end(), order);
  return OWQS_OK;
}

}  // extern "C"
