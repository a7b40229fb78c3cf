/* O-A, the direct sub-state simulator, in plain C with OpenMP (oracle; test
 * infrastructure only: only tests/, the smoke check and bench.py's CPU
 * baseline load it; the product library never does, and it shares no code
 * with the CUDA path).
 *
 * It is the same algorithm as oracle/substate.py, step for step, written as
 * plain loops over the amplitude index so that every host core can take a
 * share of each loop (one "#pragma omp parallel for" per step, nothing
 * blocked, fused or reordered):
 *   - state (Section 4.1): separate sub-states, merged by a tensor product
 *     only when an E joins them; the input qubits form one sub-state; bit k
 *     of a sub-state's index is its k-th qubit in ascending label order
 *     (the order Fig. 8 prints);
 *   - N_v (Section 2.2): a new sub-state (1, 1)/sqrt2, made at the first
 *     command that touches v;
 *   - E_uv (Section 4.4.1, Fig. 5): merge the sub-states if needed, then
 *     negate every amplitude whose u and v bits are both 1;
 *   - X_v^s, Z_v^s (Section 4.4.1): with signal parity 1, exchange the v=0
 *     and v=1 halves, or negate the v=1 half;
 *   - ^t[M_v^a]^s (Eq. 2, Section 4.2, Eqs. 11-13, Fig. 6): with
 *     theta = (-1)^s a + t pi, e = e^{-i theta} applied with t as an exact
 *     sign, the two outcome rows give (a0 + e a1)/sqrt2 and (a0 - e a1)/sqrt2
 *     over every pair of amplitudes differing only in bit v; prob_s is the
 *     squared norm of row s over the squared norm of the sub-state (Eq. 13);
 *     OWQS keeps row s divided by sqrt(prob_s) (Eq. 7), EOWQS (Section 4.5)
 *     keeps row s times sqrt2; qubit v is dropped.  A scalar left when a
 *     whole sub-state is measured away is kept as a global factor.
 * Outcomes are forced (per qubit label) or all zero.  The squared norms of a
 * measurement are compensated (Kahan) FP64 sums per thread, added in thread
 * order, so the probabilities stay exact to a few units in the last place
 * at any array size.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { OA_N = 0, OA_E = 1, OA_M = 2, OA_X = 3, OA_Z = 4 };
enum { OA_OK = 0, OA_ERR_PATTERN = 1, OA_ERR_MEMORY = 2, OA_ERR_IMPOSSIBLE = 3, OA_ERR_WIDTH = 4 };

#define OA_MAXQ 62

typedef struct {
  int n;             /* number of qubits */
  int lab[OA_MAXQ];  /* ascending labels; bit k of an index is qubit lab[k] */
  cplx* t;           /* 2^n amplitudes */
} Sub;

/* compensated (Kahan) running sum */
static void kahan(double* sum, double* comp, double x) {
  const double y = x - *comp;
  const double t = *sum + y;
  *comp = (t - *sum) - y;
  *sum = t;
}

static int omp_threads(void) {
#ifdef _OPENMP
  return omp_get_num_threads();
#else
  return 1;
#endif
}

static int pos_of(const Sub* s, int q) {
  for (int k = 0; k < s->n; ++k)
    if (s->lab[k] == q) return k;
  return -1;
}

static Sub* sub_new(int n) {
  Sub* s = (Sub*)calloc(1, sizeof(Sub));
  if (!s) return NULL;
  s->n = n;
  s->t = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n));
  if (!s->t) {
    free(s);
    return NULL;
  }
  return s;
}

static void sub_free(Sub* s) {
  if (s) {
    free(s->t);
    free(s);
  }
}

/* |+> on qubit v (Section 2.2) */
static Sub* plus_sub(int v) {
  Sub* s = sub_new(1);
  if (!s) return NULL;
  s->lab[0] = v;
  s->t[0] = s->t[1] = 1.0 / sqrt(2.0);
  return s;
}

/* tensor product (Section 4.1): the labels of a and b merged in ascending
 * order; each new amplitude is the product of the a and b amplitudes whose
 * bits it holds */
static Sub* kron(const Sub* a, const Sub* b) {
  const int n = a->n + b->n;
  if (n > OA_MAXQ) return NULL;
  Sub* m = sub_new(n);
  if (!m) return NULL;
  int from_a[OA_MAXQ], bit[OA_MAXQ];
  int ia = 0, ib = 0;
  for (int k = 0; k < n; ++k) {
    if (ib >= b->n || (ia < a->n && a->lab[ia] < b->lab[ib])) {
      m->lab[k] = a->lab[ia];
      from_a[k] = 1;
      bit[k] = ia++;
    } else {
      m->lab[k] = b->lab[ib];
      from_a[k] = 0;
      bit[k] = ib++;
    }
  }
  const int64_t size = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < size; ++i) {
    uint64_t xa = 0, xb = 0;
    for (int k = 0; k < n; ++k) {
      const uint64_t v = ((uint64_t)i >> k) & 1u;
      if (from_a[k]) xa |= v << bit[k];
      else xb |= v << bit[k];
    }
    m->t[i] = a->t[xa] * b->t[xb];
  }
  return m;
}

/* the pattern, as flat arrays (commands in execution order) */
typedef struct {
  int nqubits, nin, nout, ncmd;
  const int32_t *inputs, *outputs, *kind, *q0, *q1, *sdom_off, *sdom_len, *tdom_off, *tdom_len, *dom;
  const double* angle;
} Pat;

static int parity(const Pat* P, const uint8_t* meas, int off, int len) {
  int s = 0;
  for (int i = 0; i < len; ++i) s ^= meas[P->dom[off + i]] & 1;
  return s;
}

/* Simulate the pattern.  psi_in: 2^nin interleaved (re, im) doubles, bit k
 * = inputs[k], or NULL for |+> on every input.  outcome_of_label: forced
 * outcome per qubit label, or NULL for all zero.  mode 0 OWQS, 1 EOWQS.
 * stop_after > 0: return after that many measurements (no output).
 * psi_out: 2^nout interleaved doubles, bit k = outputs[k] (may be NULL).
 * probs: per qubit label, the probability of the kept outcome (may be NULL).
 * nthreads > 0 sets the OpenMP thread count.  Returns an OA_* status;
 * *peak receives the widest sub-state (the paper's m). */
int oa_run(int nqubits, const int32_t* inputs, int nin, const int32_t* outputs, int nout, int ncmd,
           const int32_t* kind, const int32_t* q0, const int32_t* q1, const double* angle,
           const int32_t* sdom_off, const int32_t* sdom_len, const int32_t* tdom_off, const int32_t* tdom_len,
           const int32_t* dom, const double* psi_in, const uint8_t* outcome_of_label, int mode, int stop_after,
           double* psi_out, double* probs, int nthreads, int* peak) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  Pat P = {nqubits, nin, nout, ncmd, inputs, outputs, kind, q0, q1, sdom_off, sdom_len, tdom_off, tdom_len, dom,
           angle};
  int status = OA_OK, done = 0, pk = 0;
  cplx gfactor = 1.0;
  Sub** owner = (Sub**)calloc((size_t)nqubits + 1, sizeof(Sub*));
  uint8_t* meas = (uint8_t*)calloc((size_t)nqubits + 1, 1);
  if (!owner || !meas) {
    free(owner);
    free(meas);
    return OA_ERR_MEMORY;
  }
#define FAIL(code) \
  do {             \
    status = code; \
    goto out;      \
  } while (0)
  /* the input sub-state (Section 4.1), normalised in OWQS (Eq. 4) */
  if (nin > 0) {
    if (nin > OA_MAXQ) FAIL(OA_ERR_WIDTH);
    Sub* s = sub_new(nin);
    if (!s) FAIL(OA_ERR_MEMORY);
    int sorted[OA_MAXQ], src_bit[OA_MAXQ];
    for (int k = 0; k < nin; ++k) sorted[k] = inputs[k];
    for (int k = 1; k < nin; ++k)
      for (int j = k; j > 0 && sorted[j - 1] > sorted[j]; --j) {
        const int tmp = sorted[j];
        sorted[j] = sorted[j - 1];
        sorted[j - 1] = tmp;
      }
    for (int k = 0; k < nin; ++k) {
      s->lab[k] = sorted[k];
      for (int j = 0; j < nin; ++j)
        if (inputs[j] == sorted[k]) src_bit[k] = j;
    }
    const int64_t size = (int64_t)1 << nin;
    double norm2 = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : norm2)
    for (int64_t i = 0; i < size; ++i) {
      uint64_t x = 0;
      for (int k = 0; k < nin; ++k) x |= (((uint64_t)i >> k) & 1u) << src_bit[k];
      const cplx v = psi_in ? psi_in[2 * x] + I * psi_in[2 * x + 1] : pow(2.0, -nin / 2.0);
      s->t[i] = v;
      norm2 += creal(v) * creal(v) + cimag(v) * cimag(v);
    }
    if (psi_in && mode == 0) {
      const double f = 1.0 / sqrt(norm2);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < size; ++i) s->t[i] *= f;
    }
    for (int k = 0; k < nin; ++k) owner[inputs[k]] = s;
  } else if (psi_in) {
    /* no input qubit: the input is one amplitude times |+> on every qubit */
    const cplx c = psi_in[0] + I * psi_in[1];
    gfactor *= mode == 0 ? c / cabs(c) : c;
  }

  for (int ci = 0; ci < ncmd; ++ci) {
    const int k = kind[ci];
    if (k == OA_N) {
      if (owner[q0[ci]]) FAIL(OA_ERR_PATTERN);
      owner[q0[ci]] = plus_sub(q0[ci]);
      if (!owner[q0[ci]]) FAIL(OA_ERR_MEMORY);
      continue;
    }
    const int u = q0[ci];
    if (!owner[u] && !(owner[u] = plus_sub(u))) FAIL(OA_ERR_MEMORY);
    if (k == OA_E) {
      const int v = q1[ci];
      if (!owner[v] && !(owner[v] = plus_sub(v))) FAIL(OA_ERR_MEMORY);
      Sub *a = owner[u], *b = owner[v];
      if (a != b) {
        if (a->n + b->n > OA_MAXQ) FAIL(OA_ERR_WIDTH);
        Sub* m = kron(a, b);
        if (!m) FAIL(OA_ERR_MEMORY);
        for (int q = 0; q < nqubits; ++q)
          if (owner[q] == a || owner[q] == b) owner[q] = m;
        sub_free(a);
        sub_free(b);
        a = m;
      }
      if (a->n > pk) pk = a->n;
      const int pu = pos_of(a, u), pv = pos_of(a, v);
      const int64_t size = (int64_t)1 << a->n;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < size; ++i)
        if ((((uint64_t)i >> pu) & 1u) && (((uint64_t)i >> pv) & 1u)) a->t[i] = -a->t[i];
    } else if (k == OA_X || k == OA_Z) {
      if (!parity(&P, meas, sdom_off[ci], sdom_len[ci])) continue;
      Sub* s = owner[u];
      const int pu = pos_of(s, u);
      const int64_t size = (int64_t)1 << s->n;
      const uint64_t bitu = (uint64_t)1 << pu;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < size; ++i) {
        if (k == OA_X) {
          if (!((uint64_t)i & bitu)) {
            const cplx tmp = s->t[i];
            s->t[i] = s->t[(uint64_t)i | bitu];
            s->t[(uint64_t)i | bitu] = tmp;
          }
        } else if ((uint64_t)i & bitu) {
          s->t[i] = -s->t[i];
        }
      }
    } else if (k == OA_M) {
      Sub* s = owner[u];
      if (s->n > pk) pk = s->n;
      const int pu = pos_of(s, u);
      const int sg = parity(&P, meas, sdom_off[ci], sdom_len[ci]);
      const int tg = parity(&P, meas, tdom_off[ci], tdom_len[ci]);
      /* e^{-i theta}, theta = (-1)^s alpha + t pi (Eq. 2), t pi as a sign */
      cplx e = sg == 0 ? cos(angle[ci]) - I * sin(angle[ci]) : cos(angle[ci]) + I * sin(angle[ci]);
      if (tg) e = -e;
      const int out = outcome_of_label ? (outcome_of_label[u] & 1) : 0;
      const int64_t half = (int64_t)1 << (s->n - 1);
      const uint64_t low = ((uint64_t)1 << pu) - 1u;
      const double r2 = 1.0 / sqrt(2.0);
      double n0 = 0.0, n1 = 0.0, nall = 0.0;
      Sub* nw = sub_new(s->n - 1);
      if (!nw) FAIL(OA_ERR_MEMORY);
      /* squared norms: compensated (Kahan) sums per thread, then the
         threads' sums in order, so that the oracle's probabilities stay
         exact to a few units in the last place at any size */
#pragma omp parallel
      {
        double s0 = 0.0, c0 = 0.0, s1 = 0.0, c1 = 0.0, sa = 0.0, ca = 0.0;
#pragma omp for schedule(static)
        for (int64_t j = 0; j < half; ++j) {
          const uint64_t i0 = (((uint64_t)j & ~low) << 1) | ((uint64_t)j & low), i1 = i0 | (low + 1);
          const cplx a0 = s->t[i0], a1 = s->t[i1];
          const cplx h0 = (a0 + e * a1) * r2, h1 = (a0 - e * a1) * r2; /* rows of M_0 and M_1 */
          kahan(&s0, &c0, creal(h0) * creal(h0) + cimag(h0) * cimag(h0));
          kahan(&s1, &c1, creal(h1) * creal(h1) + cimag(h1) * cimag(h1));
          kahan(&sa, &ca, creal(a0) * creal(a0) + cimag(a0) * cimag(a0) + creal(a1) * creal(a1) +
                              cimag(a1) * cimag(a1));
          nw->t[j] = out ? h1 : h0;
        }
#pragma omp for ordered schedule(static, 1)
        for (int th = 0; th < omp_threads(); ++th) {
#pragma omp ordered
          {
            n0 += s0;
            n1 += s1;
            nall += sa;
          }
        }
      }
      const double p = mode == 0 ? (out ? n1 : n0) / nall : 0.5;
      if (mode == 0 && !(p > 0.0)) {
        sub_free(nw);
        FAIL(OA_ERR_IMPOSSIBLE);
      }
      const double f = mode == 0 ? 1.0 / sqrt(p) : sqrt(2.0);
#pragma omp parallel for schedule(static)
      for (int64_t j = 0; j < half; ++j) nw->t[j] *= f;
      meas[u] = (uint8_t)out;
      if (probs) probs[u] = p;
      for (int q = 0, w = 0; q < s->n; ++q)
        if (q != pu) nw->lab[w++] = s->lab[q];
      for (int q = 0; q < nqubits; ++q)
        if (owner[q] == s) owner[q] = nw;
      owner[u] = NULL;
      sub_free(s);
      if (nw->n == 0) {
        gfactor *= nw->t[0];
        sub_free(nw);
      }
      ++done;
      if (stop_after > 0 && done >= stop_after) goto out;
    } else {
      FAIL(OA_ERR_PATTERN);
    }
  }
  /* the live sub-states at the end: outputs no command touched join as |+>,
     then everything is tensored and permuted to bit k = outputs[k] */
  for (int k = 0; k < nout; ++k)
    if (!owner[outputs[k]] && !(owner[outputs[k]] = plus_sub(outputs[k]))) FAIL(OA_ERR_MEMORY);
  {
    Sub* total = NULL;
    for (int q = 0; q < nqubits; ++q) {
      Sub* s = owner[q];
      if (!s || s == total) continue;
      if (!total) {
        total = s;
        continue;
      }
      if (total->n + s->n > OA_MAXQ) FAIL(OA_ERR_WIDTH);
      Sub* m = kron(total, s);
      if (!m) FAIL(OA_ERR_MEMORY);
      for (int r = 0; r < nqubits; ++r)
        if (owner[r] == total || owner[r] == s) owner[r] = m;
      sub_free(total);
      sub_free(s);
      total = m;
    }
    const int nt = total ? total->n : 0;
    if (nt != nout) FAIL(OA_ERR_PATTERN);
    if (psi_out) {
      if (!total) {
        psi_out[0] = creal(gfactor);
        psi_out[1] = cimag(gfactor);
      } else {
        int pos[OA_MAXQ];
        for (int k = 0; k < nout; ++k) {
          pos[k] = pos_of(total, outputs[k]);
          if (pos[k] < 0) FAIL(OA_ERR_PATTERN);
        }
        const int64_t size = (int64_t)1 << nout;
#pragma omp parallel for schedule(static)
        for (int64_t o = 0; o < size; ++o) {
          uint64_t i = 0;
          for (int k = 0; k < nout; ++k) i |= (((uint64_t)o >> k) & 1u) << pos[k];
          const cplx v = total->t[i] * gfactor;
          psi_out[2 * o] = creal(v);
          psi_out[2 * o + 1] = cimag(v);
        }
      }
    }
  }
out:
  if (peak) *peak = pk;
  for (int q = 0; q < nqubits; ++q) {
    Sub* s = owner[q];
    if (!s) continue;
    for (int r = q; r < nqubits; ++r)
      if (owner[r] == s) owner[r] = NULL;
    sub_free(s);
  }
  free(owner);
  free(meas);
  return status;
#undef FAIL
}

/* threads an OpenMP region gets by default (the host cores) */
int oa_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
