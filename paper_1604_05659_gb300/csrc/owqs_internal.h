// Internal declarations of the GB300 one-way quantum computer simulator.
// Host side: pattern model, reordering, schedule compiler, run driver.
// Device side: the pass kernels (owqs_kernels.cu) and their parameter block.
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "owqs.h"

namespace owqs {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
owqs_status set_error(owqs_status st, const std::string& msg);
void clear_error();

// ---------------------------------------------------------------------------
// pattern model (Section 2.2)
// ---------------------------------------------------------------------------
struct Cmd {
  uint32_t kind = 0;
  uint32_t q0 = 0, q1 = 0;
  double angle = 0.0;
  std::vector<uint32_t> sdom, tdom;
};

struct RunCache;  // device workspace and graphs (owqs_run.cpp)

struct Pattern {
  uint32_t n = 0;
  std::vector<uint32_t> inputs, outputs;
  std::vector<Cmd> cmds;              // as loaded (execution order)
  std::vector<int32_t> k_of_qubit;    // K-index (order of M commands as loaded), -1 if not measured
  std::vector<uint32_t> meas_qubit;   // qubit of K-index k
  std::vector<uint32_t> active;       // active execution order: indices into cmds
  std::vector<uint32_t> active_meas;  // measurement order of the active order
  bool standard = false;
  bool deps_ok = true;                // active order measures every domain first (D0)
  uint64_t order_version = 0;         // bumped whenever the active order changes
  int gflow_state = -1;               // open graph has a gflow: -1 not searched yet, 0 no, 1 yes
  std::shared_ptr<RunCache> cache;
  // recognition: the same pattern with |I| untouched reference qubits added as
  // inputs and outputs (all basis columns at once); rebuilt on order changes
  std::shared_ptr<Pattern> aug;
  uint64_t aug_version = ~0ull;
  ~Pattern();
};

// Test hook (owqs_test_wait_timeout): runs left that stall their first
// bulk-copy launch, and the cycle limit of that stall
int take_test_stall(long long* limit);
int take_test_shrink(uint64_t* elems);

// Section 4.5 pre-check: does the open graph have a gflow (searched once,
// kept with the pattern; owqs_flow.cpp)
bool has_gflow(Pattern& p);

// owqs_run without the gflow pre-check (batched determinism checks compare
// the branch overlaps themselves)
owqs_status run_unchecked(Pattern& p, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                          uint8_t* outcomes, double* probs);
// kernels launched by the pattern's last forced-outcome run (unitary: of its
// last owqs_unitary call)
uint32_t last_launch_count(Pattern& p, bool unitary);

// peak live width and amplitude updates of the active order (host)
void order_stats(const Pattern& p, uint32_t* peak_live, uint64_t* amp_updates);

// Make a measurement order the active order (Eq. 17); need_deps rejects
// orders that measure a qubit before its domains.
owqs_status build_active_order(Pattern& p, const std::vector<uint32_t>& order, bool need_deps);

// Entanglement graph and dependency data used by the reordering criteria of
// Section 4.3 (shared by the greedy PROA and the learned proposal).
struct ReorderGraph {
  uint32_t n = 0;
  std::vector<std::vector<uint32_t>> adj;       // all E partners (set)
  std::vector<std::vector<uint32_t>> pending0;  // E partners with odd multiplicity
  std::vector<uint32_t> os, ss;                 // OS(v), SS(v)
  std::vector<std::vector<uint32_t>> deps;      // measurement domains (empty in EOWQS)
  std::vector<std::vector<uint32_t>> rdeps;     // qubits whose M depends on q
  std::vector<uint32_t> measured;               // measured qubits (load order)
  std::vector<char> is_meas;
};
ReorderGraph build_reorder_graph(const Pattern& p, bool eowqs);

// The learned proposal's measurement order (owqs_learn.cu): at every step the
// model scores the candidates and the lowest score is measured next.
owqs_status learned_order(const Pattern& p, const owqs_model* m, bool eowqs, bool product_input,
                          std::vector<uint32_t>& order);

// ---------------------------------------------------------------------------
// compiled pass: the contract between the schedule compiler and the kernels
//
// Extended index k of a pass: bits [0, n_in) are the live qubits read from the
// input array, bits [n_in, n_in + r) the r qubits prepared in |+> during this
// segment.  The segment's X, Z and E commands are normalised to
//     x(k) = (-1)^{q(k)} in[(k ^ xmask) & (2^n_in - 1)],
//     q(k) = c0 ^ parity(k & zmask) ^ XOR over edges (u,v) of k_u k_v,
// (N commutes to the front, an X is pushed through the E and Z commands
// before it, and X on a |+> qubit is dropped).  A measure pass writes
//     out[j] = s_c (x(ins(j, b, 0)) + w1 x(ins(j, b, 1))),  j < 2^(n_in+r-1),
// where ins inserts a bit at position b; a final pass writes
//     out[u] = s_c x(sum_k u_k 2^perm[k]).
// s_c = scale / sqrt(norm of the previous array) in OWQS mode, scale in EOWQS.
// ---------------------------------------------------------------------------
struct PassDesc {
  int kind = 0;  // 0 measure, 1 final, 2 join of an input factor (product input)
  int factor = -1;  // kind 2: the factor whose qubits become the top r bits
  int n_in = 0, r = 0, b = -1, n_out = 0;
  int outcome = 0;
  uint32_t meas_k = 0;  // K-index (load order) of the measured qubit
  uint64_t xmask = 0, zmask = 0;
  uint32_t c0 = 0;
  std::vector<std::pair<int, int>> edges;  // u < v
  double w1re = 0, w1im = 0;               // (-1)^outcome e^{-i theta}
  double ere = 0, eim = 0;                 // e^{-i theta}
  double scale = 1.0;
  std::vector<int> perm;                   // final pass
};

// true if the byte ranges [a, a + na) and [b, b + nb) share a byte (an
// input and an output vector that overlap would let the first pass read
// what the final pass overwrites)
inline bool byte_ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return na && nb && x < y + nb && y < x + na;
}

constexpr int kMaxLive = 62;   // widest extended index the compiler accepts
constexpr int kQMax = 64;      // quadratic lower endpoints (a vertex cover of any graph on 62 bits fits)

// Kernel parameter block, passed by value.
struct PassParams {
  const void* in;        // input array, nullptr => virtual |+> input of value vconst
  void* out;             // output array
  double* norms;         // device norm slots
  double* partials;      // per-block partial sums (2 * grid)
  unsigned int* counter; // finished-block counter, left at 0
  unsigned int* errflag; // bit 0: a device-side wait gave up; bit 1: a bounds check failed
  int n_in, r, b, n_out;
  int norm_in;           // slot whose value N gives s_c = scale / sqrt(N); -1: s_c = scale
  int norm_out;          // slot written with sum |out|^2 (prob pass: norm_out, norm_out+1); -1: none
  double thresh;         // N below thresh => s_c = 0 (impossible branch)
  uint64_t xmask, zmask;
  uint32_t c0;
  int nq;                // quadratic terms: k_{qu[e]} * parity(k & qa[e])
  int qu[kQMax];
  uint64_t qa[kQMax];
  double scale, w1re, w1im, ere, eim, vconst;
  const double* w1dev;   // device (-1)^s e^{-i theta} written by k_decide; nullptr: w1re, w1im
  const double* edev;    // device e^{-i theta} (probability pass); nullptr: ere, eim
  long long stall_limit; // > 0 (tests only): wait this many cycles on a barrier nothing arrives at, then give up
  int vdiag;             // virtual input: 0 = |+> of value vconst; h > 0 = amplitude 1 where the
                         // low h input bits equal the next h (all basis columns, recognition)
  // fast pass (star form at b, no X): uniform sign tables
  uint64_t amask;        // neighbours of b
  uint32_t zb;           // z bit at b
  uint32_t tzl, tal;     // bit l: parity(delta_l & zmask), parity(delta_l & amask)
  uint32_t tzt, tat;     // bit t: same for the in-thread broadcast offsets
  int rt;                // in-thread broadcast bits
  int nlo;               // live (non-broadcast) output bits
  // final pass
  int identity_perm;
  int perm[64];
  // elements in the buffers read and written; checked only in builds with
  // OWQS_BOUNDS_CHECK (0: not checked)
  uint64_t in_cap, out_cap;
};

enum KernelKind {
  KK_FAST = 0, KK_GENERIC = 1, KK_FINAL = 2, KK_NORM = 3, KK_PROB = 4, KK_TMA = 5, KK_DECIDE = 7,
  KK_GROUP = 8, KK_KRON = 9, KK_SMALL = 10, KK_PROB_TMA = 11
};



// TMA-pipelined pass (complex64): log2 of the outputs per tile (16 KB of
// outputs, 32 KB of inputs) and the number of shared-memory stages
constexpr int kTmaLogTileC64 = 11;
constexpr int kTmaStages = 3;
// device-side wait limit (cycles) before a TMA pass gives up with an error
constexpr long long kWaitLimitCycles = 4000000000ll;

struct LaunchPlan {
  int kind = KK_GENERIC;
  int meas = 0;          // measurements the launch performs (1 for a measure pass, k for a group)
  int variant = 0;       // fast: measured-bit case (b < lg: b; lg: middle bit; lg+1: new qubit)
  int lg = 2;            // fast: log2 of consecutive outputs per thread tile
  int hint = 0;          // fast: 1 = streaming (evict-first) loads and stores
  int grid = 1, block = 256;
  double bytes = 0;      // algorithmic bytes (amplitudes read + written)
};

constexpr int kFastRMax = 2;  // broadcast bits handled inside a thread

// Fast-pass configuration for a dtype: tile width (c64: 2 or 3, c128: 1 or 2)
// and cache hint.  OWQS_FAST="lg,hint" overrides the default (tuning runs).
void fast_config(int dtype, int* lg, int* hint);
// 1 if eligible wide passes use the TMA-pipelined kernel (OWQS_TMA=0 turns it off)
int tma_enabled();
constexpr int kBlock = 256;
int max_grid();               // grid cap for grid-stride kernels
// the grid a launch uses: `want`, or the test hook's cap (owqs_test_grid_cap) when smaller
int capped_grid(int want);
int test_grid_cap();          // the test hook's cap, 0 for none
void set_test_grid_cap(int blocks);
// the input width from which a complex64 group may take a 4-qubit register
// (kGroupM4MinWidth, or the test hook's owqs_test_group_m4_width)
int group_m4_min_width();
void set_test_m4_width(int width);

// A group of 2..kGroupMax consecutive measure passes run as one sweep
// (bulk copies into shared memory).  Every pass is in star form with no X mask and prepares
// exactly one qubit, and measures either an input qubit of the group's input
// array or a qubit prepared earlier in the group.  Then a constant set of M
// qubits (M = the input qubits the group measures, 1..kGroupRegMax) varies
// per element of the remaining ("free") input bits: the group is M-qubit
// register arithmetic per free index.  Slot i of the register starts as
// input qubit B[i]; the qubit a pass prepares takes the slot of the qubit it
// measures.  The free bits keep their order and become the low output bits;
// the surviving register qubits become the top M output bits (outoff).
//
// Signs.  Pass j's sign for the element's free index f, output register
// configuration g and measured value m splits into
//   m = 0:  c0 ^ par(f & zfree) ^ par(g & zr)
//   m = 1:  the m = 0 sign ^ zb ^ par(f & afree) ^ par(g & ar)
// The kernel keeps a scaled register x~ with x[g] = E D(g) x~[g], where E is
// the element's accumulated sign times the product of the scales and the
// previous array's 1/sqrt(N), and D(g) = (-1)^par(g & p) a register-diagonal
// sign whose mask p the host tracks from pass to pass.  A pass then computes
//   x~'[g] = x~[g0] + ct[g] (-1)^rho w x~[g1]      (g0, g1: g with the
// measured slot 0 / 1), rho = zb ^ par(f & afree) per element, ct[g] =
// (-1)^(par(g & ar) ^ p_slot), and the element's sign collects
// c0 ^ par(f & zfree); the new mask is zr ^ (p without the measured slot).
// The store multiplies by E and fin[g] = D_final(g) * product of scales.
// A tile is 2^(T-M) consecutive free indices (T = 9 for complex64: 4 KB of
// input per warp, T = 10 for a complex64 register of 4 qubits: 8 KB per warp;
// T = 11 for complex128: 32 KB per block).  Register
// inputs with input bit below T - M + (the number of such bits) are "low":
// they lie inside the tile's contiguous input block of 2^(T-M+nlow)
// amplitudes; the others are "high" and select one of 2^(M-nlow) such
// blocks (runoff).  Configuration c of the register is read at smem offset
// cbase[c] + spread(e), spread inserting zeros at the low register bits
// (lowmask) into the element's offset e within the tile.
// norms[norm_out + j] = squared norm after pass j (no rescaling inside the
// group): the product of the group's first j+1 outcome probabilities;
// nscale[j] = product of the first j+1 squared scales.
constexpr int kGroupMax = 12;
constexpr int kGroupRegMax = 4;      // register qubits of a complex64 group
constexpr int kGroupRegMaxC128 = 3;  // of a complex128 group
constexpr int kGroupMaxM4 = 8;       // passes of a group on a 4-qubit register
constexpr int kGroupM4MinWidth = 26; // input width from which a group may take a 4-qubit register
// log2 of a group's tile (the T above) for M register qubits
constexpr int group_tile_bits(int dtype, int m) { return dtype == OWQS_C64 ? (m == 4 ? 10 : 9) : 11; }
struct GroupPass {
  int slot;                 // register slot measured, then refilled by the new qubit
  uint32_t c0, zb;
  uint32_t zr, ar;          // register parts of the sign masks (bit t = slot t)
  uint32_t zlo, alo;        // zfree, afree within a tile (low T - M bits)
  uint64_t zfree, afree;    // sign masks over the free index
  double scale, wre, wim;   // scale and (-1)^s e^{-i theta}
  float ct[1 << kGroupRegMax];  // +-1 per output configuration
  float fwr, fwi;           // (-1)^s e^{-i theta} in FP32
  double ctd[1 << kGroupRegMaxC128];  // ct in FP64 (complex128 groups)
};
struct GroupParams {
  const void* in;
  void* out;
  double* norms;
  double* partials;
  unsigned int* counter;
  unsigned int* errflag;
  int k, m, lt;             // passes, register qubits, log2 tile (T - m)
  int nfree;                // free bits (input bits minus m)
  int B[kGroupRegMax];      // input bit of each slot's initial qubit
  int nruns;                // 2^(number of high register inputs)
  uint32_t runlen;          // amplitudes per run: 2^(T - M + nlow)
  uint32_t lowmask;         // low register input bits (inside the run)
  uint64_t runoff[1 << kGroupRegMax];  // input offset of run r (high register bits)
  uint32_t cbase[1 << kGroupRegMax];   // smem offset of configuration c: run * runlen + low bits
  uint64_t outoff[1 << kGroupRegMax];
  float fin[1 << kGroupRegMax];
  double find[1 << kGroupRegMaxC128];  // fin in FP64 (complex128 groups)
  double nscale[kGroupMax];
  uint64_t zall;            // XOR of the passes' zfree: the element's accumulated Z sign is
  uint32_t zall_lo, c0all;  // c0all ^ par(f & zall); zall_lo = its low (tile) bits
  int norm_in, norm_out;
  double thresh;
  double vconst;            // in == nullptr: the value of every input amplitude (virtual |+> input)
  long long stall_limit;    // > 0 (tests only): as PassParams::stall_limit
  // complex128 in double-float arithmetic (OWQS_RUN_DOUBLE_FLOAT): df = 1;
  // df_in / df_out: the input / output array holds double-float pairs (the
  // previous / next launch is such a group on the same array), else complex128
  int df, df_in, df_out;
  // every pass measures a qubit joined by an odd number of E to the qubit the
  // pass prepares (a fresh |+>): then each probability is exactly 1/2 on any
  // state (the projection leaves |+>phi0 +- e^{-i a}|->phi1, half of phi's
  // squared norm), so no norm is summed and the slots get the exact products
  int half;
  GroupPass pass[kGroupMax];
  uint64_t in_cap, out_cap;  // as PassParams
};
// longest group starting at passes[i] (0 or 1 if none), planned into G
// virt_in: the group reads the virtual |+> input (no input array)
int plan_group(const std::vector<PassDesc>& passes, size_t i, int dtype, GroupParams& G, LaunchPlan& L,
               bool virt_in = false);
cudaError_t launch_group(const GroupParams& G, int dtype, cudaStream_t s);
// complex128 group in double-float arithmetic (owqs_group_df.cu)
cudaError_t launch_group_df(const GroupParams& G, bool in_df, bool out_df, cudaStream_t s);
// the group's register-slot sequence (bit 31 half, bits 28-30 m, 24-27 k, 2j
// and 2j+1 the slot of pass j), and whether a kernel compiled for it runs it
// (complex64; from the virtual |+> input only on registers of at most 2 qubits)
uint32_t group_sequence_code(const GroupParams& G);
bool group_sequence_specialised(const GroupParams& G, int dtype, bool virt_in);
int group_enabled();  // OWQS_GROUP=0 turns group fusion off


// plan + fill the parameter block of one pass (host)
void plan_pass(const PassDesc& d, int dtype, bool virt_in, PassParams& P, LaunchPlan& L);

// device launches (owqs_kernels.cu)
cudaError_t launch_pass(const PassParams& P, const LaunchPlan& L, int dtype, cudaStream_t s);

// A whole run in one block when every array of the run has at most
// 2^kSmallLog amplitudes and it has at most kSmallMaxPasses passes (k_small): passes_dev holds the run's passes, the
// final pass last, planned as for the per-pass kernels (norm slots, scales,
// the first pass's input, the final pass's output); input_norm: slot 0 first
// gets the input vector's squared norm.
constexpr int kSmallLog = 8;
constexpr int kSmallMaxPasses = 160;  // the passes sit in shared memory
cudaError_t launch_small(const PassParams* passes_dev, int npass, int input_norm, int dtype, cudaStream_t s);

// Device-drawn outcome of one measurement (sampled policy, k_decide)
struct DecideParams {
  const double* norms;   // prob_0 = norms[pslot]
  int pslot;
  const uint64_t* seed;  // device: the seed of the splitmix64 stream
  uint64_t draw;         // which output of the stream (measurements in execution order)
  uint8_t* outcomes;     // device, K bytes in load order
  uint32_t meas_k;
  const double* e_this;  // device: e^{-i theta} of this measurement
  double* w1;            // out: (-1)^outcome e^{-i theta}
  // the next measurement in execution order (has_next = 0 for the last)
  int has_next;
  const uint32_t* dom;   // device: K-indices of its s-domain, then its t-domain
  uint32_t sd_off, sd_len, td_off, td_len;
  double ca, sa;         // cos and sin of its angle alpha
  double* e_next;        // out: its e^{-i theta}
};
cudaError_t launch_decide(const DecideParams& D, cudaStream_t s);
cudaError_t launch_put_u64(uint64_t* dst, uint64_t v, cudaStream_t s);
cudaError_t launch_norm(const void* in, uint64_t n, int dtype, double* norms, int slot,
                        double* partials, unsigned int* counter, int grid, cudaStream_t s);

// ---------------------------------------------------------------------------
// schedule compiler
// ---------------------------------------------------------------------------
struct OutcomeSource {
  virtual ~OutcomeSource() = default;
  // forced and preselected outcomes are known before the run: fill
  // outcome_by_qubit and return true.  Signals are then taken from the full
  // outcome vector, which is exact for any order that applies every E on v
  // before M_v, because measurements on different qubits commute (Eq. 14).
  virtual bool known_upfront(std::vector<int8_t>& /*outcome_by_qubit*/) { return false; }
  // decide the outcome of the measurement described by d (outcome field not
  // yet set); return -1 on failure (error already recorded)
  virtual int decide(const PassDesc& d) = 0;
};

// Walk the active order; emits K measure passes then the final pass.  Returns
// OWQS_OK or an error.  maps (optional) receives bit_of_qubit after each pass.
// factors (optional, product inputs): the input qubits grouped into factors
// (each list in the factor's bit order).  No input qubit is live at the start;
// at the start of each segment, every factor with a qubit that the segment
// (up to and including its measurement) touches joins the live array as new
// top bits (a kind-2 pass), and so does every factor holding an output before
// the final pass.
owqs_status compile_schedule(const Pattern& p, int mode, OutcomeSource& src,
                             std::vector<PassDesc>& passes,
                             std::vector<std::vector<int32_t>>* maps = nullptr,
                             const std::vector<std::vector<uint32_t>>* factors = nullptr);

// Separate sub-states (Section 4.1): the live qubits form components that
// only an E joins; each component with prepared-and-touched qubits keeps its
// own array.  The compiler walks the active order as compile_schedule does,
// per component: a component's pending N/E/X/Z commands fold into its next
// measure pass, which reads only that component's array; an E between two
// components joins their arrays (a tensor product, the second component's
// materialised qubits as the new high bits; a component with no array yet,
// only |+> qubits, joins for free).  A component measured away entirely
// leaves a one-amplitude array, a scalar factor.  At the end every
// component is joined into one array, which the final pass (corrections and
// the gather to output order) reads.  Ops of different components commute;
// a component's ops are emitted together, just before its next join and at
// the end, so that its consecutive measure passes can form pass groups.
struct CompOp {
  int kind = 0;        // 0 measure (d on component a), 1 join (b into a), 2 final (d on component a)
  int a = -1, b = -1;
  int n_a = 0, n_b = 0;  // join: the materialised widths of a and b (0: a one-amplitude array)
  PassDesc d;          // measure and final ops
};
struct CompSchedule {
  std::vector<CompOp> ops;   // in launch order
  int ncomp = 0;             // component ids used by ops are < ncomp
  int input_comp = -1;       // component whose first array is the caller's input vector (-1: none)
  int peak_m = 0;            // widest component at a measurement, prepared qubits included (the paper's m)
  uint64_t peak_amps = 0;    // most amplitudes held in component arrays at once (a pass's input and output both)
  uint64_t single_amps = 0;  // the same for one array holding every live qubit (two ping-pong buffers)
  double work = 0;           // amplitudes read and written by the passes and joins
  double single_work = 0;    // the same for one array over every live qubit
};
// real_input: the caller passes an input vector (one component over the
// inputs); otherwise every input qubit starts as its own |+> component.
owqs_status compile_components(const Pattern& p, int mode, OutcomeSource& src, bool real_input, CompSchedule& cs);

// Join of one input factor (product input) or of two components (separate
// sub-states): out[j] = s * in[j mod 2^n_in] * phi[j >> n_in], s =
// 1/sqrt(norms[fnorm]) if fnorm >= 0 (the factor normalised) times
// 1/sqrt(norms[norm_in]) if norm_in >= 0; in == nullptr means the scalar 1.
struct KronParams {
  const void* in;
  void* out;
  const void* phi;
  const double* norms;
  int n_in, q;
  int norm_in, fnorm;
  unsigned int* errflag;
  uint64_t in_cap, out_cap;  // as PassParams
};
cudaError_t launch_kron(const KronParams& K, int dtype, cudaStream_t s);

}  // namespace owqs

// the opaque handle of the C ABI
struct owqs_pattern {
  owqs::Pattern p;
};
