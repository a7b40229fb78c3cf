/*
 * owqs.h -- C ABI of the GB300 one-way quantum computer simulator.
 *
 * Simulates one-way quantum computation (1WQC) measurement patterns with the
 * array method of Nikahd, Houshmand, Saheb Zamani and Sedighi, "One-Way
 * Quantum Computer Simulation" (arXiv:1604.05659): qubit elimination
 * (Section 4.2), pattern reordering (Section 4.3), implicit simulation of
 * actions (Section 4.4) and the probability-free EOWQS mode for patterns with
 * generalised flow (Section 4.5).
 *
 * Conventions shared by every entry point
 *   - Qubits are the labels 0 .. nqubits-1 (the set V of Section 2.2).
 *   - Commands are listed in EXECUTION order: cmds[0] acts first.  (The paper
 *     writes patterns right to left.)
 *   - A vector over an ordered qubit list q[0..n-1] has 2^n complex entries and
 *     bit k of the index is qubit q[k]; input vectors use the input list I,
 *     output vectors the output list O.
 *   - |+-a> = (|0> +- e^{+ia}|1>)/sqrt2.  Eq. 1 prints e^{-ia}; Eqs. 9-12 and
 *     the derivation of Section 4.2 need e^{+ia}, which is what is used.
 *   - Complex numbers are interleaved (re, im): float pairs for OWQS_C64,
 *     double pairs for OWQS_C128.
 *   - The caller owns every buffer it passes.  The library owns the pattern
 *     handle, its compiled schedule, its device workspace and its CUDA graphs;
 *     all of them are released by owqs_free_pattern.
 *   - Every function returns an owqs_status; no exception crosses the ABI.
 *     On any error other than OWQS_ERR_IMPOSSIBLE_BRANCH and
 *     OWQS_ERR_NOT_DETERMINISTIC the caller's output buffers are left untouched.
 *     owqs_last_error() gives a message for the calling thread.
 *   - A handle may be used by one thread at a time.
 */
#ifndef OWQS_H
#define OWQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OWQS_ABI_VERSION 2

typedef enum {
  OWQS_OK = 0,
  OWQS_ERR_ARG = 1,                /* bad argument (null pointer, size, enum)        */
  OWQS_ERR_PATTERN = 2,            /* pattern breaks D0-D3 (Section 2.2)            */
  OWQS_ERR_NOT_STANDARD = 3,       /* reordering needs the standard form CME         */
  OWQS_ERR_IMPOSSIBLE_BRANCH = 4,  /* a forced outcome has probability below 1e-24
                                      (C128) or 1e-12 (C64); the output is zero     */
  OWQS_ERR_NOT_DETERMINISTIC = 5,  /* EOWQS run whose output norm is not 1          */
  OWQS_ERR_OOM = 6,                /* live width too large for device memory        */
  OWQS_ERR_CUDA = 7,               /* a CUDA call failed (see owqs_last_error)      */
  OWQS_ERR_TIMEOUT = 8,            /* a device-side wait gave up                    */
  OWQS_ERR_UNSUPPORTED = 9         /* feature not available in this build           */
} owqs_status;

/* command kinds (Section 2.2) */
enum { OWQS_CMD_N = 0, OWQS_CMD_E = 1, OWQS_CMD_M = 2, OWQS_CMD_X = 3, OWQS_CMD_Z = 4 };

/* One command.
 *   N  q0        prepare q0 in |+>.  Non-input qubits with no N are prepared
 *                before the first command (N commutes with commands on other
 *                qubits, so the simulator prepares them just in time).
 *   E  q0 q1     CZ on q0 and q1 (q0 != q1).
 *   M  q0 angle  measure q0 at angle (-1)^s angle + t pi (Eq. 2), where s and t
 *                are the parities of the outcomes of the qubits listed in
 *                domain[s_off .. s_off+s_len) and domain[t_off .. t_off+t_len).
 *   X, Z q0      Pauli on q0 when the parity of the outcomes in
 *                domain[s_off .. s_off+s_len) is 1 (t_* ignored).            */
typedef struct {
  uint32_t kind;
  uint32_t q0;
  uint32_t q1;
  uint32_t pad_;
  double angle;
  uint32_t s_off, s_len;
  uint32_t t_off, t_len;
} owqs_cmd;

typedef struct owqs_pattern owqs_pattern;

/* Load and validate a pattern P = (V, I, O, A) (Section 2.2).
 *   nqubits        |V|; labels are 0 .. nqubits-1 (at most 1<<24)
 *   inputs/nin     the input list I (distinct labels; bit k of psi_in is inputs[k])
 *   outputs/nout   the output list O (distinct; bit k of psi_out is outputs[k])
 *   cmds/ncmd      commands in execution order
 *   domain/ndomain qubit labels referenced by the commands' signal domains
 *   out            receives the new handle (owned by the library)
 * Returns OWQS_ERR_PATTERN if the commands break D0 (depend on an outcome not
 * yet measured), D1 (act on a measured qubit), D2 (act on a qubit before its
 * N, unless it is an input) or D3 (a qubit is measured iff it is not an
 * output), or if an E joins a qubit to itself.  Host-only; needs no GPU.   */
owqs_status owqs_load_pattern(uint32_t nqubits, const uint32_t* inputs, uint32_t nin,
                              const uint32_t* outputs, uint32_t nout, const owqs_cmd* cmds,
                              size_t ncmd, const uint32_t* domain, size_t ndomain,
                              owqs_pattern** out);

void owqs_free_pattern(owqs_pattern* p);

typedef struct {
  uint32_t nqubits, nin, nout;
  uint32_t nmeas;        /* K = |V| - |O| (Section 4.3)                     */
  uint32_t standard;     /* 1 if the loaded order is the standard form CME  */
  uint32_t peak_live;    /* widest live array of the ACTIVE command order   */
  uint64_t amp_updates;  /* sum over commands of 2^(live width), active order;
                            saturates at UINT64_MAX (orders of 64+ live qubits) */
} owqs_pattern_info;

/* Facts about the pattern under its active order.  Host-only. */
owqs_status owqs_get_info(const owqs_pattern* p, owqs_pattern_info* info);

/* modes (Section 4.5) */
enum { OWQS_MODE_OWQS = 0, OWQS_MODE_EOWQS = 1 };

/* Learned reorder proposal (not in the paper; it proposes, and the proposal is
 * kept only if no worse than the greedy PROA order).  A 3-layer MLP, OWQS_MODEL_FEATURES -> 64 -> 64 -> 1 with ReLU,
 * scores every candidate qubit at each reordering step; the lowest score is
 * measured next.  Its matrix products take bfloat16 inputs (features,
 * weights and activations rounded to nearest even) and accumulate in FP32;
 * biases and the FP32 master weights are FP32.  Parameters, in order:
 * W1[64][F], b1[64], W2[64][64], b2[64], w3[64], b3 (row-major).          */
#define OWQS_MODEL_FEATURES 12
#define OWQS_MODEL_PARAMS 5057
typedef struct owqs_model owqs_model;

typedef struct {
  uint32_t mode;           /* OWQS: dependent measurements wait for their domains;
                              EOWQS: outcomes preselected, every qubit ready   */
  uint32_t product_input;  /* 1: every input qubit starts as its own sub-state  */
  uint32_t sweep;          /* 1: Section 5 sweep a = |O| .. 1 with b = d = |O|,
                              g = 0.5; 0: one run with the weights below        */
  uint32_t use_learned;    /* 1: also build the learned proposal with `model`;
                              it is kept only if its (peak live width, amplitude
                              updates) is no worse than the best greedy order:
                              the greedy order of `mode` and, in EOWQS mode, the
                              greedy OWQS sweep order too (an order that waits
                              for every domain is valid with preselected
                              outcomes), whichever is better                    */
  double alpha, beta, gamma, delta;  /* Eq. 18 weights when sweep == 0 (> 0)   */
  const owqs_model* model; /* use_learned: the scoring network (runs on the
                              current device)                                   */
} owqs_reorder_opts;

typedef struct {
  uint32_t peak_m;         /* largest measurement state-space MS (Table I/III m) */
  uint32_t peak_live;      /* widest single live array under the new order      */
  uint64_t amp_updates;    /* amplitude updates under the new order (saturating,
                              as in owqs_pattern_info)                          */
  double alpha_used;       /* Eq. 18 a of the chosen run                        */
  uint32_t learned_accepted; /* 1 if the learned proposal was kept              */
  uint32_t greedy_peak_live;   /* the greedy order's figures (use_learned)      */
  uint64_t greedy_amp_updates;
  uint32_t learned_peak_live;  /* the proposal's figures (use_learned)          */
  uint32_t greedy_best_owqs;  /* use_learned in EOWQS mode: 1 if the greedy OWQS
                                  sweep order was the better greedy order       */
  uint64_t learned_amp_updates;
} owqs_reorder_info;

/* PROA (Section 4.3): greedy measurement order with the Eq. 18 cost
 *   Cost(v) = a MS(v) + b OS(v) - g SS(v)            (v next to a selected qubit)
 *           = a (MS(v)+1) d + b OS(v) - g SS(v)      (otherwise)
 * MS: size of the sub-state measuring v creates (v's sub-state joined with
 * those of its neighbours over E commands not yet applied); OS: output
 * neighbours; SS: qubits whose domains contain v (0 in EOWQS); ties go to the
 * lowest label.  The pattern must be in standard form.  On success the new
 * order becomes the active order: for each chosen v, its pending E commands
 * then M_v (Eq. 17); then the remaining E commands and the corrections.
 *   order   optional, K entries: the measurement order (qubit labels)
 *   info    optional
 * Host-only; needs no GPU.                                                  */
owqs_status owqs_reorder(owqs_pattern* p, const owqs_reorder_opts* opts,
                         owqs_reorder_info* info, uint32_t* order);

/* Candidate features along a measurement order (training data for the
 * learned proposal).  At every step of `order` the candidates are the ready
 * qubits (all unmeasured qubits in EOWQS mode); the row of the qubit `order`
 * measures there is written with up to max_cands - 1 other candidates drawn
 * without replacement by a splitmix64 stream seeded with `seed`.  Per row,
 * OWQS_MODEL_FEATURES floats, with S = max(|O|, 1):
 *   0 MS/S  1 OS/S  2 SS/S  3 flag  4 degree/4  5 pending E/4
 *   6 live width/S  7 width at the measurement/S  8 its increase
 *   9 candidate already live  10 selected neighbours/4  11 steps left/K
 * (MS, OS, SS and flag as in Eq. 18; live width = qubits of the single
 * amplitude array).  Rows are grouped by step: step s owns rows
 * step_first[s] .. step_first[s+1]-1 and target_row[s] is the row of the
 * measured qubit.  Sizes: feats cap_rows x F, step_first K+1, target_row K;
 * *nrows receives the row count (if it exceeds cap_rows nothing is written
 * and OWQS_ERR_ARG is returned).  Host-only.                              */
owqs_status owqs_reorder_features(const owqs_pattern* p, uint32_t mode, uint32_t product_input,
                                  const uint32_t* order, uint32_t max_cands, uint64_t seed,
                                  float* feats, uint32_t* step_first, uint32_t* target_row,
                                  uint64_t cap_rows, uint64_t* nrows);

/* Model life cycle.  weights: OWQS_MODEL_PARAMS host floats, or NULL for a
 * seeded initialisation (uniform +-1/sqrt(fan_in)).  The model lives on the
 * device that is current at creation.                                      */
owqs_status owqs_model_create(const float* weights, uint64_t seed, owqs_model** m);
void owqs_model_free(owqs_model* m);
owqs_status owqs_model_get_weights(const owqs_model* m, float* weights);

/* Scores of nrows feature rows (device arrays) on `stream`. */
owqs_status owqs_model_score(owqs_model* m, const float* feats, uint64_t nrows, float* scores,
                             void* stream);

/* Loss and gradient (no update).  The loss is the mean over steps of the
 * softmax cross-entropy of -score over each step's rows, with target_row as
 * the label.  feats, step_first, target_row: device arrays as produced by
 * owqs_reorder_features.  grad: OWQS_MODEL_PARAMS host floats.             */
owqs_status owqs_model_gradient(owqs_model* m, const float* feats, const uint32_t* step_first,
                                const uint32_t* target_row, uint32_t nsteps, float* grad,
                                float* loss, void* stream);

/* Adam training on the GPU: `epochs` sweeps over the steps in minibatches of
 * batch_steps consecutive steps (shuffled per epoch with `seed`); losses
 * (optional, host) receives the mean loss of each epoch.                    */
owqs_status owqs_model_train(owqs_model* m, const float* feats, const uint32_t* step_first,
                             const uint32_t* target_row, uint32_t nsteps, uint32_t epochs,
                             uint32_t batch_steps, float lr, uint64_t seed, float* losses,
                             void* stream);

/* Make `order` (K measured qubits, each once, dependencies first) the active
 * measurement order, built as in owqs_reorder.  Standard form required.    */
owqs_status owqs_set_order(owqs_pattern* p, const uint32_t* order, uint32_t k);

/* Restore the command order given to owqs_load_pattern. */
owqs_status owqs_reset_order(owqs_pattern* p);

/* Active measurement order (K labels). */
owqs_status owqs_get_order(const owqs_pattern* p, uint32_t* order);

enum { OWQS_C64 = 0, OWQS_C128 = 1 };
enum { OWQS_OUTCOME_FORCED = 0, OWQS_OUTCOME_SAMPLED = 1, OWQS_OUTCOME_ZERO = 2 };
enum { OWQS_IO_DEVICE = 0, OWQS_IO_HOST = 1 };

typedef struct {
  uint32_t dtype;     /* OWQS_C64 (complex64 amplitudes, FP64 reductions) or OWQS_C128 */
  uint32_t mode;      /* OWQS_MODE_OWQS or OWQS_MODE_EOWQS                            */
  uint32_t policy;    /* forced outcomes, sampled, or all zero.  Sampled: outcome 0
                         iff u <= prob_0, u the k-th splitmix64(seed) uniform in
                         [0,1) for the k-th measurement in execution order; OWQS
                         computes prob_0 (Eq. 13), EOWQS takes it as 1/2 (Section
                         4.5), so an EOWQS sampled run draws every outcome first
                         and then runs as a forced one                             */
  uint32_t io;        /* OWQS_IO_DEVICE: psi_in/psi_out are device pointers;
                         OWQS_IO_HOST: host pointers, copies done inside the call    */
  uint64_t seed;      /* sampled policy only                                          */
  void* stream;       /* cudaStream_t to run on; NULL = the legacy default stream    */
  uint32_t use_graph; /* 1: replay the pass sequence as a CUDA graph                */
  uint32_t flags;     /* Sampled OWQS runs on a pattern with a gflow first guess
                         every outcome as u > 1/2 (the probability of a gflow
                         pattern, Section 4.5), run the guesses as forced
                         outcomes, and keep that run iff every draw u_k <= prob_0
                         it computed reproduces its guess and lies more than a tie
                         margin (1e-6 for OWQS_C64, 1e-12 for OWQS_C128) from that
                         prob_0 (then the one-at-a-time draw, whose prob_0 differs
                         only by rounding, takes the same branch).  Otherwise, and
                         on patterns without a gflow, they take checked launches
                         when no X or Z with a signal comes before the last
                         measurement: the forced run of the current outcome
                         vector (initially those guesses), one kernel at a time;
                         after each launch that measures, the host checks its
                         measurements' draws against the probabilities it
                         computed, in execution order, and at the first draw that
                         decides the other outcome corrects that outcome and runs
                         the same launch again on its untouched input.  The
                         outcomes are those of a one-at-a-time draw (a draw
                         within rounding of prob_0 follows the launch's own
                         prob_0).  Patterns with such an X or Z draw one
                         measurement at a time.  owqs_last_sample_info says which
                         of these ran.
                         Flags:
                         OWQS_RUN_SEQUENTIAL_SAMPLING: draw one measurement at a
                         time from the start, on the device whenever no X or Z with
                         a signal comes before the last measurement (e.g. standard
                         form), else on the host.
                         OWQS_RUN_HOST_SAMPLING: draw one measurement at a time on
                         the host, one device-to-host read per measurement.
                         OWQS_RUN_PER_PASS: one kernel per pass even when every array
                         of a forced or zero-outcome run fits 2^8 amplitudes (such
                         runs otherwise execute in one single-block kernel).
                         Separate sub-states (Section 4.1): qubits that no E has
                         joined yet live in separate arrays, each measure pass
                         reads only its own component's array, and an E between
                         two components joins their arrays (tensor product).
                         Forced and zero-outcome runs with a single input vector
                         use them when the components' arrays need at most half
                         the memory of one array over all live qubits;
                         OWQS_RUN_SUBSTATES: always (forced or zero outcomes);
                         OWQS_RUN_ONE_ARRAY: never (one live array).
                         OWQS_RUN_DOUBLE_FLOAT (OWQS_C128 only): pass groups
                         compute in double-float arithmetic (a value as the sum
                         of two floats, about 48 significant bits) on the FP32
                         pipes instead of FP64; arrays between two such groups
                         hold double-float pairs, every other array complex128. */
} owqs_run_opts;
enum { OWQS_RUN_HOST_SAMPLING = 1, OWQS_RUN_PER_PASS = 2, OWQS_RUN_SEQUENTIAL_SAMPLING = 4,
       OWQS_RUN_SUBSTATES = 8, OWQS_RUN_ONE_ARRAY = 16, OWQS_RUN_DOUBLE_FLOAT = 32 };

/* How the pattern's last run with sampled outcomes (owqs_run, policy
 * OWQS_OUTCOME_SAMPLED) was carried out. */
enum {
  OWQS_SAMPLE_NONE = 0,              /* no sampled run yet                                */
  OWQS_SAMPLE_DRAWN_FIRST = 1,       /* EOWQS: every outcome drawn, then a forced run     */
  OWQS_SAMPLE_GUESS_KEPT = 2,        /* OWQS: the whole-run guess held                     */
  OWQS_SAMPLE_CHECKED_LAUNCHES = 3,  /* OWQS: checked launches                              */
  OWQS_SAMPLE_ONE_AT_A_TIME = 4,     /* OWQS: one measurement at a time, drawn on the device */
  OWQS_SAMPLE_HOST = 5               /* OWQS: one measurement at a time, drawn on the host   */
};
typedef struct {
  uint32_t path;        /* OWQS_SAMPLE_*                                                   */
  uint32_t guessed;     /* 1: a whole-run guess ran first (kept or not)                     */
  uint32_t checks;      /* checked launches: host checks, one per launch that measures      */
  uint32_t relaunches;  /* checked launches: launches run again after a corrected outcome   */
} owqs_sample_info;
/* Fills *info for the pattern's last sampled run (zeros before the first).
 * OWQS_ERR_ARG on a NULL argument. */
owqs_status owqs_last_sample_info(const owqs_pattern* p, owqs_sample_info* info);

/* Simulate the pattern under its active order and return the output state.
 *   psi_in    2^|I| amplitudes (bit k = inputs[k]); NULL = |+> on every input
 *             (generated on the device, nothing is read).  OWQS mode divides
 *             by the input norm; EOWQS uses the vector as given.
 *   psi_out   2^|O| amplitudes (bit k = outputs[k]), the normalised branch
 *             state M_s ... E N psi_in / sqrt(prob) followed by the corrections
 *             (OWQS); in EOWQS every prob is taken as 1/2 (Section 4.5).
 *   outcomes  host, K bytes in the order of the M commands as loaded; read for
 *             the forced policy, written otherwise.  May be NULL for the zero
 *             policy.
 *   probs     host, K doubles or NULL: the probability of each recorded
 *             outcome given the earlier ones (Eq. 13); 0.5 in EOWQS.
 * Returns after the device work has finished.  In EOWQS mode the pattern's
 * open graph must have a gflow (Section 4.5: a pattern without one is
 * reported as incorrect): the first EOWQS run of a loaded pattern searches
 * for one (owqs_find_flow, result kept with the pattern) and returns
 * OWQS_ERR_NOT_DETERMINISTIC, running nothing, if there is none.  The output
 * norm is then checked against the input's (tolerance 1e-10 C128, 1e-4 C64),
 * which catches correction domains that do not match the flow:
 * OWQS_ERR_NOT_DETERMINISTIC as well. */
owqs_status owqs_run(owqs_pattern* p, const owqs_run_opts* opts, const void* psi_in,
                     void* psi_out, uint8_t* outcomes, double* probs);

/* Asynchronous runs of the same simulation as owqs_run (forced or zero
 * outcomes, one live array, one launch per pass or pass group, no CUDA
 * graph).  owqs_run_async compiles the schedule, enqueues the run on
 * opts->stream and returns; owqs_wait blocks until the oldest run in flight
 * on the pattern has finished and returns its status, its outcomes (zero
 * policy) and probabilities (as owqs_run's).  At most two runs are in
 * flight per pattern handle (a third returns OWQS_ERR_ARG, as does owqs_wait
 * with none).  With OWQS_IO_HOST, the input copy runs on a copy stream as
 * soon as the previous run's launches that read the input staging buffer
 * are done, and the output copy on another copy stream after the final pass:
 * the copies of consecutive runs overlap each other's launches.
 *   psi_in, psi_out  as owqs_run; they must stay valid, and psi_out unread,
 *                    until owqs_wait has returned for this run (host
 *                    vectors: pinned memory)
 *   outcomes         forced policy: read during the call (may be reused after
 *                    it returns)
 * owqs_run and the other synchronous runs of a pattern return OWQS_ERR_ARG
 * while it has asynchronous runs in flight.  Errors of the device work
 * (OWQS_ERR_TIMEOUT, ...) are reported by owqs_wait. */
owqs_status owqs_run_async(owqs_pattern* p, const owqs_run_opts* opts, const void* psi_in, void* psi_out,
                           const uint8_t* outcomes);
owqs_status owqs_wait(owqs_pattern* p, uint8_t* outcomes, double* probs);

/* Product input (Section 4.1 and Fig. 8a: the input as separate sub-states).
 * The inputs are given as nfactors factors: factor f holds sizes[f] input
 * qubits (1 .. 30), listed in qubits[] (all factors concatenated, each in its
 * bit order: bit k of factor f's vector is its k-th qubit), and its
 * 2^sizes[f] amplitudes at the device pointer vecs[f] (the run's dtype,
 * 16-byte aligned).  Every input qubit is in exactly one factor; each factor
 * is normalised by the library.  A factor joins the live array (a tensor
 * product, its qubits becoming the top bits) only at the start of the first
 * segment whose commands touch one of its qubits, or before the final pass
 * for an output no command touches, so inputs that a pattern reaches late
 * stay out of the array until then.
 *   opts      as owqs_run; policy FORCED or ZERO, io DEVICE
 *   psi_out, outcomes, probs: as owqs_run
 * OWQS_ERR_ARG if the factors do not cover the inputs exactly once. */
owqs_status owqs_run_product(owqs_pattern* p, const owqs_run_opts* opts, uint32_t nfactors, const uint32_t* sizes,
                             const uint32_t* qubits, const void* const* vecs, void* psi_out, uint8_t* outcomes,
                             double* probs);

/* Test hook for the device-side wait limits (no real stall is needed to
 * exercise them).  Every wait inside the bulk-copy pass kernels is bounded:
 * on expiry the kernel raises an error flag and returns, and the run reports
 * OWQS_ERR_TIMEOUT with the context still usable.  After this call, the
 * next `runs` calls of owqs_run (forced or zero outcomes) that contain a
 * bulk-copy launch make their first such launch wait on a barrier that
 * nothing arrives at, for `limit_cycles` SM cycles (1 .. 4e9), before any
 * copy is issued; that run is launched without a graph and returns
 * OWQS_ERR_TIMEOUT.  runs = 0 cancels.  Not for production use. */
owqs_status owqs_test_wait_timeout(uint32_t runs, uint64_t limit_cycles);

/* Test hook for the bounds-checked build (libowqs_checked.so, compiled with
 * OWQS_BOUNDS_CHECK, in which every global access of the pass kernels is
 * first checked against the extent of the buffer it touches): the next
 * `runs` owqs_run calls launch without a graph with every buffer extent
 * `elems` amplitudes short.  The checked build then skips the accesses
 * beyond the shortened extents and the run returns OWQS_ERR_CUDA ("outside
 * its buffer"); the release build ignores extents.  runs = 0 cancels.
 * Not for production use. */
owqs_status owqs_test_shrink_extents(uint32_t runs, uint64_t elems);

/* Test hook: every later launch of the pass kernels (single passes, pass
 * groups, norms and joins) uses at most `blocks` thread blocks, so that a
 * small array still makes every warp of a persistent kernel loop over many
 * tiles and wrap its shared-memory ring of stages (the path full-size
 * arrays take).  The cap is part of the CUDA-graph key.  blocks = 0 removes
 * the cap.  Not for production use. */
owqs_status owqs_test_grid_cap(uint32_t blocks);

/* Test hook: complex64 pass groups may take a 4-qubit register from input
 * width `width` on (instead of 26, below which the one-block-per-SM kernel
 * of such groups does not pay), so that small arrays exercise that kernel.
 * Part of the CUDA-graph key and of every launch plan.  width = 0 restores
 * the default.  Not for production use. */
owqs_status owqs_test_group_m4_width(uint32_t width);

/* Flows of the pattern's open graph (G, I, O), Section 4.5 with the
 * definitions of ref. [13]; G has an edge u-v iff the pattern holds an odd
 * number of E commands on {u, v}.
 *   OWQS_FLOW_CAUSAL  f maps each measured qubit i to a non-input f(i)
 *                     adjacent to i, with i before f(i) and i before every
 *                     other neighbour of f(i) (returned as g(i) = {f(i)}).
 *   OWQS_FLOW_GFLOW   every measurement in the XY plane: g maps each measured
 *                     i to a set of non-inputs, all after i, with i not in
 *                     g(i), i in Odd(g(i)) (the qubits with an odd number of
 *                     neighbours in g(i)) and every other member of Odd(g(i))
 *                     after i.  The causal flow is returned when one exists.
 * "Before" is by layer: outputs are at layer 0, measured qubits at layers
 * >= 1, and i is measured before j iff layer[i] > layer[j].  Layers are built
 * from the outputs back, each qubit placed in the first layer where a
 * corrector set exists (so the flow is the most delayed one); the gflow
 * search solves a GF(2) system over the unplaced qubits per layer, O(L |V|^3
 * / 64) word operations for L layers, run only when no causal flow exists.
 *   found      out: 1 if a flow of that kind exists, else 0 (status OK)
 *   layer      optional, nqubits entries: each label's layer; all -1 when
 *              found = 0
 *   g_first    optional, nqubits + 1 entries: g(i) is g_members[g_first[i]
 *              .. g_first[i+1]); empty for outputs and when found = 0
 *   g_members  optional, g_cap entries (sorted labels per qubit); if g_cap is
 *              smaller than *g_total nothing is written and OWQS_ERR_ARG is
 *              returned
 *   g_total    optional out: the number of members g needs
 * Host only: needs no GPU. */
enum { OWQS_FLOW_CAUSAL = 0, OWQS_FLOW_GFLOW = 1 };
owqs_status owqs_find_flow(const owqs_pattern* p, uint32_t kind, uint32_t* found, int32_t* layer,
                           uint32_t* g_first, uint32_t* g_members, uint32_t g_cap, uint32_t* g_total);

/* Recognition (Section 1: which unitary a pattern implements).  Computes
 * every basis column at once: the pattern runs with |I| extra reference
 * qubits that no command touches, starting from the sum over c of |c>|c>, so
 * the final array (output bits low, reference bits high) is the matrix.
 * Every measurement of the forced branch is taken with probability 1/2 (the
 * EOWQS scaling of Section 4.5): the result is the branch as a linear map,
 * which for a pattern with flow is the implemented unitary (up to the
 * branch's global phase).
 *   opts      dtype, stream, use_graph; policy FORCED (outcomes, K bytes in
 *             load order) or ZERO (outcomes may be NULL); io must be DEVICE
 *   U         device, 2^|O| x 2^|I| complex, column-major: U[o + 2^|O| c] is
 *             output amplitude o for basis input c (bit k of c is inputs[k])
 *   frob2     optional host double: ||U||_F^2 / 2^|I| (1 for an isometry)
 * The live array is |I| qubits wider than in owqs_run.                     */
owqs_status owqs_unitary(owqs_pattern* p, const owqs_run_opts* opts, const uint8_t* outcomes, void* U,
                         double* frob2);

/* Batched recognition and determinism checks.  One item is one pattern and
 * one forced branch, with either all basis columns (psi_in NULL: out is the
 * matrix, as for owqs_unitary) or one input vector (out is the output
 * state).  Every measurement is taken with probability 1/2 (EOWQS scaling,
 * Section 4.5), so the outputs are the branches as linear maps; for a pattern
 * with flow every branch gives the same state up to a global phase, which the
 * overlaps below measure.  Items whose widest array fits a shared-memory
 * column block (at most 16 live qubits) run in ONE persistent launch: each
 * block of threads pulls (item, column block) tasks, keeps its states on chip
 * for the whole pass list and writes only the final columns; wider items run
 * through the owqs_run / owqs_unitary pass kernels.  The column block is
 * chosen by timing the candidate shared-memory budgets on the first call for
 * a given batch shape (kept for the process) unless opts->column_block fixes
 * it.  All items must be loaded on the current device; the call returns after
 * the device work has finished.                                           */
typedef struct {
  owqs_pattern* pattern;    /* loaded pattern; its active order is used            */
  const uint8_t* outcomes;  /* K forced outcome bits (load order); NULL = all zero  */
  const void* psi_in;       /* NULL: every basis column; else device vector 2^|I|    */
  void* out;                /* device: 2^|O| x 2^|I| (column-major) or 2^|O|         */
  int32_t ref;              /* index of an item to overlap with, -1 for none        */
  uint32_t pad_;
} owqs_batch_item;

typedef struct {
  uint32_t dtype;           /* OWQS_C64 or OWQS_C128                                 */
  uint32_t column_block;    /* columns per task (power of two); 0 = tuned            */
  void* stream;             /* cudaStream_t; NULL = legacy default stream            */
  uint32_t use_graph;       /* 1: the persistent launch and the items run through the
                               pass kernels are replayed from CUDA graphs            */
  uint32_t pad_;
  double* overlaps;         /* optional host array of 4n doubles: for items with
                               ref >= 0, Re and Im of <out_ref|out>, |out|^2 and
                               |out_ref|^2 (outputs as flat vectors); 0 otherwise     */
} owqs_batch_opts;

typedef struct {
  uint32_t smem_items;      /* items run by the persistent shared-memory launch     */
  uint32_t hbm_items;       /* items run through the pass kernels                   */
  uint32_t tasks;           /* (item, column block) tasks of the persistent launch  */
  uint32_t smem_bytes_per_cta;
  uint32_t launches;        /* kernel launches of this call                         */
  uint32_t global_items;    /* items too wide for shared memory run by the second
                               persistent launch, whose state buffers are in
                               global memory (up to 2^18 amplitudes per array);
                               hbm_items counts the items wider still, which
                               run through the pass kernels of owqs_run         */
  float compile_ms;         /* host time compiling the items' pass lists (on
                               up to 32 host threads) and building the tables   */
  float call_ms;            /* host time of the whole call, device work included */
} owqs_batch_info;

owqs_status owqs_run_batch(const owqs_batch_item* items, uint32_t n, const owqs_batch_opts* opts,
                           owqs_batch_info* info);

/* owqs_run without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * a host program whose device memory is entirely owned by another
 * allocator (a framework's caching pool, an embedding application) or held
 * to a fixed budget, where an allocation inside the library could fail or
 * fragment memory that the caller has planned.  The
 * caller passes the input and output vectors exactly as for owqs_run; the
 * library's scratch (two state buffers, the norm slots, the reduction
 * partials and a counter) lives in one statically sized device array of
 * 8.25 MiB that every GPU loading this library holds until the process
 * exits.
 * Limits: device vectors only (io = OWQS_IO_DEVICE), forced or zero outcomes,
 * no CUDA graph, every pass must fit the 4 MiB state buffers (live width at
 * most 19 qubits for OWQS_C64, 18 for OWQS_C128), and at most 5448
 * measurements.  Larger patterns get OWQS_ERR_ARG with the sizes in
 * owqs_last_error().  Nothing else is allocated on the device; the call
 * does not use cudaMalloc, cudaFree or any allocating library routine.
 * The first call on a device looks up the array's device address once (with
 * that device current); make that first call before any stream capture.
 * Every call uses the same array and leaves its contents behind (the counter
 * that must start at zero is cleared at the start of each call), so calls
 * whose work overlaps on the GPU (other streams, other threads) race: issue
 * them one after another.  Returns after the device work has finished: the
 * call reads the norm slots back to the host and synchronises the stream.  */
owqs_status owqs_run_static(owqs_pattern* p, const owqs_run_opts* opts, const void* psi_in,
                            void* psi_out, uint8_t* outcomes, double* probs);

/* The launches owqs_run would make (host only, no GPU needed): for launch i
 * (i < *nlaunch, at most cap), kind[i] as in owqs_profile_run, first_meas[i]
 * the index (execution order) of its first measurement and nmeas[i] the
 * number of measurements it performs.  real_input: the run reads an input
 * vector (0: the virtual |+> input; the first measurement then runs alone).
 * outcomes: forced outcome bits (load order) or NULL for all zero. */
owqs_status owqs_describe_launches(const owqs_pattern* p, uint32_t dtype, uint32_t mode, uint32_t real_input,
                                   const uint8_t* outcomes, uint32_t* kind, uint32_t* first_meas, uint32_t* nmeas,
                                   uint32_t cap, uint32_t* nlaunch);

/* Memory of the two ways to hold the live qubits (host only, no GPU
 * needed), for the active order: one array over every live qubit, or
 * separate sub-states (Section 4.1: a component per set of qubits that E
 * commands have joined; see OWQS_RUN_SUBSTATES).  Arguments as
 * owqs_describe_launches. */
typedef struct {
  uint32_t peak_m;          /* widest sub-state at a measurement, the measured
                               qubit and prepared ones included (Table I/III's m) */
  uint32_t components;      /* sub-states over the run (inputs, prepared qubits)   */
  uint32_t joins;           /* tensor products of two arrays                        */
  uint32_t uses_substates;  /* 1 if a default owqs_run takes separate sub-states:
                               they at least halve the amplitudes moved and need no
                               more memory than one array                          */
  uint64_t substate_bytes;  /* device arena that holds every live component array   */
  uint64_t one_array_bytes; /* the two buffers of a one-array run                   */
  double substate_work;     /* amplitudes read and written, separate sub-states     */
  double one_array_work;    /* the same with one array (estimate)                   */
} owqs_memory_plan;
owqs_status owqs_plan_memory(const owqs_pattern* p, uint32_t dtype, uint32_t mode, uint32_t real_input,
                            const uint8_t* outcomes, owqs_memory_plan* plan);

/* The pass groups owqs_run would launch (host only, no GPU needed), in
 * launch order; for group i (i < *ngroups, at most cap): regs[i] the
 * register qubits M, slots[i] its register-slot sequence (bits 24-27 the
 * number of passes k, bits 2j and 2j+1 the slot that pass j measures, bit
 * 31 set when every pass measures a qubit joined by E to the qubit that
 * pass prepares, so that each probability is exactly 1/2 and the group sums
 * only its last pass's norm),
 * n_in[i] the live width it reads and specialised[i] 1 when a kernel
 * compiled for exactly that sequence runs it (complex64 groups reading an
 * array, or reading the virtual |+> input on a register of at most 2
 * qubits), 0 when the slot-dispatching kernel does.  Arguments
 * as owqs_describe_launches; any output pointer may be NULL. */
owqs_status owqs_describe_groups(const owqs_pattern* p, uint32_t dtype, uint32_t mode, uint32_t real_input,
                                const uint8_t* outcomes, uint32_t* regs, uint32_t* slots, uint32_t* n_in,
                                uint32_t* specialised, uint32_t cap, uint32_t* ngroups);

/* Per-kernel timing of one run (instrumentation).  Runs the same schedule
 * without a graph, with a CUDA event pair around every launch on opts->stream,
 * and fills, for launch i (i < *nlaunch, at most cap): ms[i] its duration,
 * bytes[i] its algorithmic bytes (amplitudes read + written), kind[i] its
 * kernel (0 register-tiled pass, 1 generic pass, 2 final pass, 3 norm,
 * 4 outcome probabilities, 5 bulk-copy pass, 7 device-drawn outcome, 8 pass
 * group, 9 factor join, 10 a whole small run in one launch, 11 outcome
 * probabilities on bulk-copy tiles) and, when nmeas is not NULL, nmeas[i]
 * the number of measurements it performs (1 for a measure pass, k for a
 * group of k, 0 otherwise).  Device IO only; the forced or zero policy, or
 * sampled in EOWQS mode (drawn first, then run as forced).                 */
owqs_status owqs_profile_run(owqs_pattern* p, const owqs_run_opts* opts, const void* psi_in,
                             void* psi_out, const uint8_t* outcomes, float* ms, double* bytes,
                             uint32_t* kind, uint32_t* nmeas, uint32_t cap, uint32_t* nlaunch);

/* Bit position of every qubit in the live array after pass `pass` of the
 * active order (-1 if the qubit is not live), for pass = 0 .. K (pass K is
 * the state before the final corrections).  The array grows by appending a
 * new qubit as the top bit; eliminating a qubit shifts the higher bits down.
 * Host-only. bit_of_qubit has nqubits entries.                             */
owqs_status owqs_get_index_map(const owqs_pattern* p, uint32_t pass, int32_t* bit_of_qubit);

/* Description of one compiled device pass (for host-logic tests). */
typedef struct {
  int32_t kind;        /* 0 measure pass, 1 final pass                          */
  int32_t n_in, r, b;  /* live width in, new qubits, measured bit (extended)     */
  int32_t n_out;
  int32_t outcome;     /* measure pass: chosen outcome                         */
  uint64_t xmask;      /* X on the input bits                                  */
  uint64_t zmask;      /* linear sign terms                                    */
  uint32_t c0;         /* constant sign                                        */
  uint32_t nedges;
  uint32_t edges[64][2]; /* quadratic sign terms (extended bit pairs)          */
  double w1re, w1im;   /* weight of the bit-b = 1 amplitude: (-1)^s e^{-i theta} */
  double scale;        /* constant factor (2^{-r/2} / sqrt2, EOWQS 2^{-r/2})   */
  int32_t perm[64];    /* final pass: extended bit of outputs[k]               */
} owqs_pass_desc;

/* Compile the active order with the given outcome bits (K, load order) and
 * copy up to cap pass descriptors to out; *npass receives the pass count.
 * Host-only.                                                                */
owqs_status owqs_describe_passes(const owqs_pattern* p, uint32_t mode, const uint8_t* outcomes,
                                 owqs_pass_desc* out, uint32_t cap, uint32_t* npass);

/* Message for the last error on the calling thread ("" if none). */
const char* owqs_last_error(void);

/* OWQS_ABI_VERSION of the loaded library. */
uint32_t owqs_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OWQS_H */
