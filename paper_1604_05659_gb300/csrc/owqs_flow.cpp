// Causal flow and gflow of a pattern's open graph (host).
//
// Section 4.5: EOWQS skips the measurement probabilities, which is exact for
// patterns whose open graph (G, I, O) has a generalized flow (ref. [13]); a
// gflow is sought before the simulation and a pattern without one is
// reported as incorrect.  The finding algorithm of ref. [25] is not given in
// the paper, so both searches here are written from the definitions:
//
//   causal flow: f(i) ~ i, f(i) not an input, i before f(i), and i before
//                every other neighbour of f(i);
//   gflow (XY plane): g(i) a set of non-inputs after i, i not in g(i), i in
//                Odd(g(i)), and every other member of Odd(g(i)) after i.
//
// Both are built backwards from the outputs, one layer at a time: a qubit
// joins layer k as soon as a corrector set among the qubits already placed
// (layers < k, minus the inputs) exists for it.  For the causal flow the
// corrector is a placed qubit with exactly one unplaced neighbour.  For the
// gflow the corrector set K must satisfy Odd(K) restricted to the unplaced
// qubits = {u}: a linear system over GF(2) (rows: unplaced qubits; columns:
// candidate correctors; entries: adjacency), solved for every unplaced u at
// once by one reduction to row echelon form with the row operations
// recorded.  Placing every qubit that can be placed as early as possible
// (i.e. as late in the measurement order as possible) loses nothing: a
// qubit placeable now stays placeable later, so if any flow exists the
// search places every qubit.
#include <algorithm>
#include <cstring>
#include <vector>

#include "owqs_internal.h"

namespace owqs {

namespace {

struct OpenGraph {
  uint32_t n = 0;
  std::vector<std::vector<uint32_t>> adj;  // sorted neighbour lists
  std::vector<char> is_in, is_out;
};

OpenGraph open_graph(const Pattern& p) {
  OpenGraph G;
  G.n = p.n;
  std::vector<std::vector<uint32_t>> raw(p.n);
  for (const Cmd& c : p.cmds)
    if (c.kind == OWQS_CMD_E) {
      raw[c.q0].push_back(c.q1);
      raw[c.q1].push_back(c.q0);
    }
  G.adj.resize(p.n);
  for (uint32_t v = 0; v < p.n; ++v) {  // odd multiplicity: E twice on a pair cancels
    std::sort(raw[v].begin(), raw[v].end());
    for (size_t i = 0; i < raw[v].size();) {
      size_t j = i;
      while (j < raw[v].size() && raw[v][j] == raw[v][i]) ++j;
      if ((j - i) & 1) G.adj[v].push_back(raw[v][i]);
      i = j;
    }
  }
  G.is_in.assign(p.n, 0);
  G.is_out.assign(p.n, 0);
  for (uint32_t q : p.inputs) G.is_in[q] = 1;
  for (uint32_t q : p.outputs) G.is_out[q] = 1;
  return G;
}

struct FlowResult {
  bool found = false;
  std::vector<int32_t> layer;
  std::vector<std::vector<uint32_t>> g;
};

FlowResult causal_flow(const OpenGraph& G) {
  FlowResult R;
  const uint32_t n = G.n;
  R.layer.assign(n, -1);
  R.g.assign(n, {});
  std::vector<char> placed(n, 0);
  std::vector<uint32_t> unplaced_nbrs(n, 0);
  for (uint32_t v = 0; v < n; ++v) unplaced_nbrs[v] = (uint32_t)G.adj[v].size();
  std::vector<uint32_t> correctors;
  uint32_t nplaced = 0;
  auto place = [&](uint32_t v, int32_t k) {
    placed[v] = 1;
    R.layer[v] = k;
    ++nplaced;
    for (uint32_t w : G.adj[v]) --unplaced_nbrs[w];
  };
  for (uint32_t v = 0; v < n; ++v)
    if (G.is_out[v]) place(v, 0);
  for (uint32_t v = 0; v < n; ++v)
    if (G.is_out[v] && !G.is_in[v]) correctors.push_back(v);
  for (int32_t k = 1;; ++k) {
    std::vector<uint32_t> newly, keep;
    std::vector<char> taken(n, 0);
    for (uint32_t v : correctors) {
      bool used = false;
      if (unplaced_nbrs[v] == 1) {
        uint32_t u = 0;
        for (uint32_t w : G.adj[v])
          if (!placed[w]) u = w;
        if (!taken[u]) {
          taken[u] = 1;
          R.g[u] = {v};
          newly.push_back(u);
          used = true;
        }
      }
      if (!used) keep.push_back(v);
    }
    if (newly.empty()) break;
    for (uint32_t u : newly) place(u, k);
    for (uint32_t u : newly)
      if (!G.is_in[u]) keep.push_back(u);
    std::sort(keep.begin(), keep.end());
    correctors.swap(keep);
  }
  R.found = nplaced == n;
  return R;
}

// one GF(2) row: adjacency part over the candidate correctors, then the
// record of row operations over the unplaced qubits
struct Rows {
  size_t wa = 0, wt = 0;
  std::vector<uint64_t> bits;  // rows x (wa + wt) words
  uint64_t* row(size_t r) { return bits.data() + r * (wa + wt); }
};

FlowResult gflow_layered(const OpenGraph& G) {
  FlowResult R;
  const uint32_t n = G.n;
  R.layer.assign(n, -1);
  R.g.assign(n, {});
  std::vector<char> placed(n, 0);
  uint32_t nplaced = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (G.is_out[v]) placed[v] = 1, R.layer[v] = 0, ++nplaced;
  std::vector<int32_t> col_of(n), row_of(n);
  for (int32_t k = 1; nplaced < n; ++k) {
    std::vector<uint32_t> rows_q, cols_q;
    for (uint32_t v = 0; v < n; ++v) {
      if (!placed[v]) rows_q.push_back(v);
      else if (!G.is_in[v]) cols_q.push_back(v);
    }
    std::fill(col_of.begin(), col_of.end(), -1);
    std::fill(row_of.begin(), row_of.end(), -1);
    for (size_t c = 0; c < cols_q.size(); ++c) col_of[cols_q[c]] = (int32_t)c;
    for (size_t r = 0; r < rows_q.size(); ++r) row_of[rows_q[r]] = (int32_t)r;
    const size_t nr = rows_q.size(), nc = cols_q.size();
    Rows M;
    M.wa = (nc + 63) / 64;
    M.wt = (nr + 63) / 64;
    M.bits.assign(nr * (M.wa + M.wt), 0);
    for (size_t r = 0; r < nr; ++r) {
      uint64_t* row = M.row(r);
      for (uint32_t w : G.adj[rows_q[r]])
        if (col_of[w] >= 0) row[col_of[w] >> 6] |= 1ull << (col_of[w] & 63);
      row[M.wa + (r >> 6)] |= 1ull << (r & 63);
    }
    // reduced row echelon form over the adjacency part
    const size_t W = M.wa + M.wt;
    std::vector<int32_t> pivot_col;
    size_t rank = 0;
    for (size_t c = 0; c < nc && rank < nr; ++c) {
      const size_t wi = c >> 6;
      const uint64_t bit = 1ull << (c & 63);
      size_t piv = rank;
      while (piv < nr && !(M.row(piv)[wi] & bit)) ++piv;
      if (piv == nr) continue;
      if (piv != rank) std::swap_ranges(M.row(piv), M.row(piv) + W, M.row(rank));
      const uint64_t* pr = M.row(rank);
      for (size_t r = 0; r < nr; ++r) {
        if (r == rank) continue;
        uint64_t* rr = M.row(r);
        if (rr[wi] & bit)
          for (size_t w = wi; w < W; ++w) rr[w] ^= pr[w];
      }
      pivot_col.push_back((int32_t)c);
      ++rank;
    }
    // u is solvable iff no zero row of the reduced adjacency part records u
    std::vector<uint64_t> blocked(M.wt, 0);
    for (size_t r = rank; r < nr; ++r) {
      const uint64_t* t = M.row(r) + M.wa;
      for (size_t w = 0; w < M.wt; ++w) blocked[w] |= t[w];
    }
    std::vector<uint32_t> newly;
    for (size_t u = 0; u < nr; ++u) {
      if (blocked[u >> 6] >> (u & 63) & 1ull) continue;
      std::vector<uint32_t> gs;
      for (size_t r = 0; r < rank; ++r)
        if (M.row(r)[M.wa + (u >> 6)] >> (u & 63) & 1ull) gs.push_back(cols_q[pivot_col[r]]);
      std::sort(gs.begin(), gs.end());
      R.g[rows_q[u]] = std::move(gs);
      newly.push_back(rows_q[u]);
    }
    if (newly.empty()) break;
    for (uint32_t v : newly) placed[v] = 1, R.layer[v] = k, ++nplaced;
  }
  R.found = nplaced == n;
  return R;
}

}  // namespace

bool has_gflow(Pattern& p) {
  if (p.gflow_state < 0) {
    const OpenGraph G = open_graph(p);
    bool ok = causal_flow(G).found;
    if (!ok) ok = gflow_layered(G).found;
    p.gflow_state = ok ? 1 : 0;
  }
  return p.gflow_state == 1;
}

}  // namespace owqs

using namespace owqs;

extern "C" {

owqs_status owqs_find_flow(const owqs_pattern* h, uint32_t kind, uint32_t* found, int32_t* layer,
                           uint32_t* g_first, uint32_t* g_members, uint32_t g_cap, uint32_t* g_total) {
  clear_error();
  if (!h || !found) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (kind != OWQS_FLOW_CAUSAL && kind != OWQS_FLOW_GFLOW) return set_error(OWQS_ERR_ARG, "bad flow kind");
  const OpenGraph G = open_graph(h->p);
  FlowResult R = causal_flow(G);
  if (kind == OWQS_FLOW_GFLOW && !R.found) R = gflow_layered(G);
  *found = R.found ? 1u : 0u;
  const uint32_t n = h->p.n;
  uint64_t total = 0;
  if (R.found)
    for (uint32_t v = 0; v < n; ++v) total += R.g[v].size();
  if (g_total) *g_total = (uint32_t)total;
  if (layer)
    for (uint32_t v = 0; v < n; ++v) layer[v] = R.found ? R.layer[v] : -1;
  if (g_first) {
    uint32_t at = 0;
    for (uint32_t v = 0; v < n; ++v) {
      g_first[v] = at;
      if (R.found) at += (uint32_t)R.g[v].size();
    }
    g_first[n] = at;
  }
  if (g_members && R.found) {
    if (total > g_cap) return set_error(OWQS_ERR_ARG, "g_members too small");
    uint32_t at = 0;
    for (uint32_t v = 0; v < n; ++v)
      for (uint32_t m : R.g[v]) g_members[at++] = m;
  }
  return OWQS_OK;
}

}  // extern "C"
