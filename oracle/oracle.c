/*
 * CPU oracle for the p-bit Feynman-path sampler (arXiv 2007.07379).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library.  Everything here is plain, scalar and
 * written for a reader checking it against the paper by eye, in FP64 or exact
 * integer arithmetic.
 *
 * Contents (each function cites the passage it follows):
 *   orc_philox4x32_10   Philox4x32-10 (Salmon et al., SC'11, "Parallel random
 *                       numbers: as easy as 1, 2, 3"), from its published
 *                       definition.
 *   orc_gate_element    the gate matrices U^(k)_{p,q} of Sec. 2 / Sec. 4 /
 *                       Appendix, as exact entries 2^{-a/2} * w^b, w=e^{i pi/4}.
 *   orc_statevector     FP64 state vector: psi = U^(d)...U^(1)|beta>  (Eq. U).
 *   orc_pathsum_exact   brute-force Feynman path sum (Eqs. U and path), exact
 *                       in Z[w]: per output alpha, the number of paths in each
 *                       phase class b (mod 8).  U_{alpha,beta} =
 *                       2^{-h/2} sum_b cnt[alpha][b] w^b.
 *   orc_gf2_rank        h (number of H gates) and the GF(2) rank of the map
 *                       from H outputs to the final layer (closed-form
 *                       variance, Eqs. U26/U30 with uniform valid paths).
 *   orc_reach           the outputs reached by valid paths, N_alpha = 2^{h-rank}
 *                       or 0 (affine image of the H outputs).
 *   orc_thresholds      heat-bath thresholds floor(2^32 sigma(-J v)).
 *   orc_colour          the sweep's colour classes.
 *   orc_gibbs           reference Gibbs sampler of the layered J-penalty
 *                       Boltzmann machine (Appendix, "replace zero elements by
 *                       e^{-J}"), following the Fig. 2 flowchart: propose by
 *                       heat-bath (Glauber) on Re E, accept, add the phase
 *                       exp(-i Im E) to the bin of the end state.
 *   orc_elim            exact i.i.d. path sampler on the eliminated network
 *                       (Appendix: non-H bits as functions of the previous
 *                       layer, H outputs fair coins), recorded like orc_gibbs.
 *   orc_elim_clamped    the same with the end state fixed to one output
 *                       alpha (uniform over the paths to alpha, by GF(2)
 *                       elimination).
 *
 * Parity status: every function is pinned by tests under tests/ (hand-worked
 * values of Sec. 4, Eq. stdT, norm invariants, exact agreement of the path sum
 * with the state vector, published Philox answers, properties of the chain).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t op, layer, q0, q1, q2; /* q2: third qubit of a three-qubit gate, else -1 */
} orc_gate;

enum { ORC_H = 0, ORC_S = 1, ORC_T = 2, ORC_CNOT = 3, ORC_CZ = 4 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), published definition:
 * 10 rounds; each round multiplies counter words 0 and 2 by the constants
 * 0xD2511F53 and 0xCD9E8D57 into 64-bit products and mixes
 *   out = (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
 * the key is bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between
 * rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)prod1;
    uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)prod0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Gate matrices, written as exact entries.  An entry is either zero (-1) or
 * w^b with b in 0..7 (w = e^{i pi/4}); H carries an extra 1/sqrt(2).
 * Index convention for a 2-qubit gate on (q0, q1): basis index
 * x = x_{q0} + 2 x_{q1}, i.e. the first-named qubit is the low bit, the order
 * 00,10,01,11 of Sec. 2 (Eq. ET2).  Rows are output states <s^(k)|, columns are
 * input states |s^(k-1)>, as in the kbordermatrix tables of the paper.
 *   H    = (1/sqrt2) [[1, 1], [1, -1]]                          (Eq. Had)
 *   S    = diag(1, i)          T = diag(1, e^{i pi/4})          (Rz family,
 *                                 Appendix; global phase fixed to 1 on |0>)
 *   CNOT(q0=control, q1=target): x_t -> x_t XOR x_c               (Appendix)
 *   CZ   = diag(1, 1, 1, -1)   (exchange-type diagonal gate, Appendix)     */
static const int H_TAB[2][2] = {{0, 0}, {0, 4}};
static const int S_TAB[2][2] = {{0, -1}, {-1, 2}};
static const int T_TAB[2][2] = {{0, -1}, {-1, 1}};
/* CNOT with x = x_c + 2 x_t: |c,t> -> |c, t^c>.  Inputs 0,1,2,3 go to
 * outputs 0,3,2,1. */
static const int CNOT_TAB[4][4] = {
    {0, -1, -1, -1}, {-1, -1, -1, 0}, {-1, -1, 0, -1}, {-1, 0, -1, -1}};
static const int CZ_TAB[4][4] = {
    {0, -1, -1, -1}, {-1, 0, -1, -1}, {-1, -1, 0, -1}, {-1, -1, -1, 4}};

/* Element <y|G|x> of one gate: returns the phase units b (0..7) or -1 for a
 * zero element; *sqrt2_pow gets the number of 1/sqrt(2) factors. */
static int gate_entry(int op, int y, int x, int* sqrt2_pow) {
  *sqrt2_pow = 0;
  switch (op) {
    case ORC_H:
      *sqrt2_pow = 1;
      return H_TAB[y][x];
    case ORC_S:
      return S_TAB[y][x];
    case ORC_T:
      return T_TAB[y][x];
    case ORC_CNOT:
      return CNOT_TAB[y][x];
    case ORC_CZ:
      return CZ_TAB[y][x];
  }
  return -1;
}

static int gate_arity(int op) { return (op == ORC_CNOT || op == ORC_CZ) ? 2 : 1; }

static int bit(uint32_t w, int q) { return (int)((w >> q) & 1u); }

/* Bits of the gate's qubits, packed in the gate's own index convention. */
static int gate_index(const orc_gate* g, uint32_t word) {
  if (gate_arity(g->op) == 2) return bit(word, g->q0) + 2 * bit(word, g->q1);
  return bit(word, g->q0);
}

/* Validate a gate list: ops known, layers in range, qubits in range and used
 * at most once per layer.  Returns 0 on success. */
static int check_circuit(int n, int d, const orc_gate* g, int ng) {
  if (n < 1 || n > 32 || d < 1 || d > 64 || ng < 0) return -1;
  uint32_t* used = (uint32_t*)calloc((size_t)d, sizeof(uint32_t));
  if (!used) return -1;
  int bad = 0;
  for (int i = 0; i < ng && !bad; ++i) {
    const orc_gate* x = &g[i];
    if (x->op < 0 || x->op > 4 || x->layer < 0 || x->layer >= d) { bad = 1; break; }
    if (x->q0 < 0 || x->q0 >= n) { bad = 1; break; }
    uint32_t m = 1u << x->q0;
    if (gate_arity(x->op) == 2) {
      if (x->q1 < 0 || x->q1 >= n || x->q1 == x->q0) { bad = 1; break; }
      m |= 1u << x->q1;
    }
    if (used[x->layer] & m) bad = 1;
    used[x->layer] |= m;
  }
  free(used);
  return bad ? -1 : 0;
}

/* Exact matrix element of the whole layer L (0-based; it maps s_L to
 * s_{L+1}) between input word x and output word y: the tensor product of the
 * layer's gates and the identity on qubits no gate touches.  Returns phase
 * units or -1 (zero); *sqrt2_pow accumulates 1/sqrt(2) factors. */
static int layer_element(int n, const orc_gate* g, int ng, int L, uint32_t x,
                         uint32_t y, int* sqrt2_pow) {
  uint32_t touched = 0;
  int phase = 0, p2 = 0;
  for (int i = 0; i < ng; ++i) {
    if (g[i].layer != L) continue;
    int a;
    int e = gate_entry(g[i].op, gate_index(&g[i], y), gate_index(&g[i], x), &a);
    touched |= 1u << g[i].q0;
    if (gate_arity(g[i].op) == 2) touched |= 1u << g[i].q1;
    if (e < 0) return -1;
    phase += e;
    p2 += a;
  }
  uint32_t nmask = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  if (((x ^ y) & ~touched & nmask) != 0) return -1; /* identity wires */
  *sqrt2_pow = p2;
  return phase & 7;
}

/* ------------------------------------------------------------------------ */
/* FP64 state vector, psi_alpha = U_{alpha,beta} (Eq. U), applying the gates
 * of each layer in turn (gates of one layer act on disjoint qubits and
 * commute).  re, im: 2^n doubles each. */
int orc_statevector(int n, int d, const orc_gate* g, int ng, uint32_t beta,
                    double* re, double* im) {
  if (check_circuit(n, d, g, ng) != 0 || n > 30) return -1;
  const uint64_t N = 1ull << n;
  memset(re, 0, N * sizeof(double));
  memset(im, 0, N * sizeof(double));
  re[beta & (N - 1)] = 1.0;
  const double r2 = 1.0 / sqrt(2.0);
  const double c8 = cos(M_PI / 4.0), s8 = sin(M_PI / 4.0);
  for (int L = 0; L < d; ++L) {
    for (int i = 0; i < ng; ++i) {
      if (g[i].layer != L) continue;
      const int op = g[i].op;
      const uint64_t m0 = 1ull << g[i].q0;
      const uint64_t m1 = gate_arity(op) == 2 ? (1ull << g[i].q1) : 0;
#pragma omp parallel for schedule(static) if (n >= 16)
      for (int64_t a = 0; a < (int64_t)N; ++a) {
        const uint64_t idx = (uint64_t)a;
        if (op == ORC_H) {
          if (idx & m0) continue;
          const uint64_t j = idx | m0;
          double ar = re[idx], ai = im[idx], br = re[j], bi = im[j];
          re[idx] = (ar + br) * r2;
          im[idx] = (ai + bi) * r2;
          re[j] = (ar - br) * r2;
          im[j] = (ai - bi) * r2;
        } else if (op == ORC_S) {
          if (!(idx & m0)) continue; /* multiply by i */
          double ar = re[idx], ai = im[idx];
          re[idx] = -ai;
          im[idx] = ar;
        } else if (op == ORC_T) {
          if (!(idx & m0)) continue; /* multiply by e^{i pi/4} */
          double ar = re[idx], ai = im[idx];
          re[idx] = ar * c8 - ai * s8;
          im[idx] = ar * s8 + ai * c8;
        } else if (op == ORC_CNOT) {
          /* control q0, target q1: swap |c=1,t=0> and |c=1,t=1> */
          if (!(idx & m0) || (idx & m1)) continue;
          const uint64_t j = idx | m1;
          double tr = re[idx], ti = im[idx];
          re[idx] = re[j];
          im[idx] = im[j];
          re[j] = tr;
          im[j] = ti;
        } else if (op == ORC_CZ) {
          if ((idx & m0) && (idx & m1)) {
            re[idx] = -re[idx];
            im[idx] = -im[idx];
          }
        }
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Brute-force Feynman path sum (Eq. U / Eq. path): every path
 * beta -> s_1 -> ... -> s_{d-1} -> alpha contributes the product of its layer
 * elements.  All nonzero Clifford+T elements are 2^{-a/2} w^b, so the sum is
 * kept exactly as integer counts per phase class: cnt[alpha*8 + b] counts the
 * paths to alpha with total phase b (mod 8).  Every nonzero path carries the
 * same power 2^{-h/2} (h = number of H gates), returned in *h_out.
 * Cost 2^{n d}; for small circuits only. */
int orc_pathsum_exact(int n, int d, const orc_gate* g, int ng, uint32_t beta,
                      int64_t* cnt, int* h_out) {
  if (check_circuit(n, d, g, ng) != 0) return -1;
  if ((int64_t)n * d > 30) return -2;
  const uint64_t N = 1ull << n;
  memset(cnt, 0, N * 8 * sizeof(int64_t));
  int h = 0;
  for (int i = 0; i < ng; ++i) h += (g[i].op == ORC_H);
  *h_out = h;
  uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
  if (!s) return -3;
  const uint64_t total = 1ull << (n * d); /* all choices of s_1..s_d */
  s[0] = beta & (uint32_t)(N - 1);
  for (uint64_t code = 0; code < total; ++code) {
    for (int k = 1; k <= d; ++k)
      s[k] = (uint32_t)((code >> ((uint64_t)(k - 1) * n)) & (N - 1));
    int phase = 0, p2 = 0, zero = 0;
    for (int L = 0; L < d && !zero; ++L) {
      int a = 0;
      int e = layer_element(n, g, ng, L, s[L], s[L + 1], &a);
      if (e < 0) zero = 1;
      phase += e;
      p2 += a;
    }
    if (zero) continue;
    if (p2 != h) { free(s); return -4; } /* cannot happen: each H once */
    cnt[(uint64_t)s[d] * 8 + (phase & 7)] += 1;
  }
  free(s);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* h and the GF(2) rank of the affine map from the H outputs to s_d.
 * Every valid path is fixed by the h H-output bits (each other bit is a copy
 * or an XOR of bits of the previous layer, Appendix), so each wire is an
 * affine GF(2) function of those bits.  The valid paths ending at alpha form a
 * coset of the kernel: N_alpha = 2^{h - rank} or 0. */
#define ORC_MAXW 40 /* 64-bit words per bit vector: h <= 2560 */
int orc_gf2_rank(int n, int d, const orc_gate* g, int ng, int* h_out,
                 int* rank_out) {
  if (check_circuit(n, d, g, ng) != 0) return -1;
  int h = 0;
  for (int i = 0; i < ng; ++i) h += (g[i].op == ORC_H);
  if (h > 64 * ORC_MAXW) return -2;
  /* wire[q]: coefficient vector over the H variables (the constant part is
   * irrelevant for the rank). */
  uint64_t(*wire)[ORC_MAXW] = calloc((size_t)n, sizeof(*wire));
  uint64_t(*next)[ORC_MAXW] = calloc((size_t)n, sizeof(*next));
  if (!wire || !next) { free(wire); free(next); return -3; }
  int var = 0;
  for (int L = 0; L < d; ++L) {
    memcpy(next, wire, (size_t)n * sizeof(*wire));
    for (int i = 0; i < ng; ++i) {
      if (g[i].layer != L) continue;
      if (g[i].op == ORC_H) {
        memset(next[g[i].q0], 0, sizeof(next[0]));
        next[g[i].q0][var >> 6] |= 1ull << (var & 63);
        ++var;
      } else if (g[i].op == ORC_CNOT) {
        for (int w = 0; w < ORC_MAXW; ++w)
          next[g[i].q1][w] = wire[g[i].q1][w] ^ wire[g[i].q0][w];
      }
    }
    memcpy(wire, next, (size_t)n * sizeof(*wire));
  }
  /* Gaussian elimination over the n rows. */
  int rank = 0;
  for (int col = 0; col < h && rank < n; ++col) {
    int piv = -1;
    for (int r = rank; r < n; ++r)
      if ((wire[r][col >> 6] >> (col & 63)) & 1ull) { piv = r; break; }
    if (piv < 0) continue;
    if (piv != rank)
      for (int w = 0; w < ORC_MAXW; ++w) {
        uint64_t t = wire[piv][w];
        wire[piv][w] = wire[rank][w];
        wire[rank][w] = t;
      }
    for (int r = 0; r < n; ++r)
      if (r != rank && ((wire[r][col >> 6] >> (col & 63)) & 1ull))
        for (int w = 0; w < ORC_MAXW; ++w) wire[r][w] ^= wire[rank][w];
    ++rank;
  }
  free(wire);
  free(next);
  *h_out = h;
  *rank_out = rank;
  return 0;
}

/* The outputs reached by valid paths (closed-form variance of the estimator,
 * Eqs. U26/U30 with uniform valid paths: E|X_alpha|^2 = N_alpha).  Each wire
 * bit is affine over GF(2) in the H outputs x: s_d = A x + c, where c carries
 * the input bits through the CNOTs (S, T and CZ leave bits unchanged).  The
 * valid paths to alpha are the solutions of A x = alpha + c: 2^{h - rank} of
 * them when alpha + c lies in the column space of A, none otherwise.  Row
 * reduction of [A | I] leaves, for every row without a pivot in A, an output
 * mask m with m A = 0; alpha is reached iff parity(m & (alpha ^ c)) = 0 for
 * every such m.
 *   c_out: the constant c (bit q = qubit q); masks: n words, the first
 *   n - rank of them the constraint masks.  n <= 32. */
int orc_reach(int n, int d, const orc_gate* g, int ng, uint32_t beta, int* h_out, int* rank_out,
              uint32_t* c_out, uint32_t* masks) {
  if (check_circuit(n, d, g, ng) != 0) return -1;
  int h = 0;
  for (int i = 0; i < ng; ++i) h += (g[i].op == ORC_H);
  if (h > 64 * ORC_MAXW) return -2;
  uint64_t(*wire)[ORC_MAXW] = calloc((size_t)n, sizeof(*wire));
  uint64_t(*next)[ORC_MAXW] = calloc((size_t)n, sizeof(*next));
  if (!wire || !next) { free(wire); free(next); return -3; }
  uint32_t cst = beta, ncst;
  int var = 0;
  for (int L = 0; L < d; ++L) {
    memcpy(next, wire, (size_t)n * sizeof(*wire));
    ncst = cst;
    for (int i = 0; i < ng; ++i) {
      if (g[i].layer != L) continue;
      const int a = g[i].q0, t = g[i].q1;
      if (g[i].op == ORC_H) {
        memset(next[a], 0, sizeof(next[0]));
        next[a][var >> 6] |= 1ull << (var & 63);
        ++var;
        ncst &= ~(1u << a);
      } else if (g[i].op == ORC_CNOT) {
        for (int w = 0; w < ORC_MAXW; ++w) next[t][w] = wire[t][w] ^ wire[a][w];
        ncst ^= ((cst >> a) & 1u) << t;
      }
    }
    memcpy(wire, next, (size_t)n * sizeof(*wire));
    cst = ncst;
  }
  /* row q of [A | I]: wire[q] | comb[q] */
  uint32_t comb[32];
  int pivoted[32];
  for (int q = 0; q < n; ++q) { comb[q] = 1u << q; pivoted[q] = 0; }
  int rank = 0;
  for (int col = 0; col < h; ++col) {
    int piv = -1;
    for (int q = 0; q < n; ++q)
      if (!pivoted[q] && ((wire[q][col >> 6] >> (col & 63)) & 1ull)) { piv = q; break; }
    if (piv < 0) continue;
    pivoted[piv] = 1;
    ++rank;
    for (int q = 0; q < n; ++q)
      if (q != piv && ((wire[q][col >> 6] >> (col & 63)) & 1ull)) {
        for (int w = 0; w < ORC_MAXW; ++w) wire[q][w] ^= wire[piv][w];
        comb[q] ^= comb[piv];
      }
  }
  int k = 0;
  for (int q = 0; q < n; ++q) masks[q] = 0u;
  for (int q = 0; q < n; ++q)
    if (!pivoted[q]) masks[k++] = comb[q];
  free(wire);
  free(next);
  *h_out = h;
  *rank_out = rank;
  *c_out = cst;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Heat-bath (Glauber) thresholds.  With the J-penalty energy, flipping a bit
 * changes Re E by J*v, v in {-3..3}; P(bit = 1) = 1 / (1 + e^{J v})
 * (Fig. 2, Step 2: acceptance from the ratio of |e^{-E}|).  A uniform u in
 * [0, 2^32) accepts when u < thr[|v|]; thr[0] = 2^31 exactly. */
int orc_thresholds(double J, uint32_t thr[4]) {
  if (!(J >= 0.0) || !isfinite(J)) return -1;
  thr[0] = 0x80000000u;
  for (int v = 1; v <= 3; ++v) {
    double p = 1.0 / (1.0 + exp(J * (double)v));
    double t = floor(p * 4294967296.0);
    if (t > 4294967295.0) t = 4294967295.0;
    thr[v] = (uint32_t)t;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Layered p-bit network, J-penalty form (Appendix: zero elements replaced by
 * e^{-J}, applied per output bit).  p-bit (k, q), k = 1..d, is bit q of s_k;
 * s_0 = beta is clamped.  For a non-H gate the column of its matrix for the
 * input bits x has exactly one nonzero row y*(x): the gate is a deterministic
 * map with a phase.  Each output bit of a non-H gate that differs from y*(x)
 * costs J; H outputs are free (no zero elements).  */

/* The unique nonzero output index of a non-H gate's column x. */
static int det_output(int op, int x) {
  for (int y = 0; y < (gate_arity(op) == 2 ? 4 : 2); ++y) {
    int a;
    if (gate_entry(op, y, x, &a) >= 0) return y;
  }
  return -1;
}

typedef struct {
  int n, d, ng;
  const orc_gate* g;
  int32_t* gate_of; /* [d][n]: index of the gate on (layer, qubit) or -1 */
} orc_net;

/* Number of violated output bits of layer L (s_L -> s_{L+1}). */
static int layer_violations(const orc_net* net, int L, uint32_t x, uint32_t y) {
  int v = 0;
  for (int q = 0; q < net->n; ++q) {
    int gi = net->gate_of[L * net->n + q];
    if (gi < 0) { /* identity wire */
      v += bit(x, q) != bit(y, q);
      continue;
    }
    const orc_gate* G = &net->g[gi];
    if (G->op == ORC_H) continue;
    if (q != G->q0) continue; /* count a 2-qubit gate once, at q0 */
    int ystar = det_output(G->op, gate_index(G, x));
    int yy = gate_index(G, y);
    v += __builtin_popcount((unsigned)(ystar ^ yy));
  }
  return v;
}

static int total_violations(const orc_net* net, const uint32_t* s) {
  int v = 0;
  for (int L = 0; L < net->d; ++L) v += layer_violations(net, L, s[L], s[L + 1]);
  return v;
}

/* Phase units of a valid path: sum of the layer elements' phases (Eq. path). */
static int path_phase(const orc_net* net, const uint32_t* s) {
  int ph = 0;
  for (int L = 0; L < net->d; ++L) {
    int a;
    int e = layer_element(net->n, net->g, net->ng, L, s[L], s[L + 1], &a);
    if (e < 0) return -1;
    ph += e;
  }
  return ph & 7;
}

/* Colour classes of one sweep.  Two p-bits interact when they belong to one
 * link (factor): a non-H output bit (k, q) together with the layer-(k-1)
 * bits its deterministic value depends on -- (k-1, q) for an identity wire,
 * S, T and CZ, (k-1, c) for a CNOT control output, (k-1, t) and (k-1, c) for a
 * CNOT target output.  Layer 0 is clamped and interacts with nothing.  A
 * class holds no two interacting p-bits, so its bits may be redrawn in any
 * order (in parallel).
 *
 * Rule (DSATUR, Brelaz 1979, with fixed tie-breaks): repeatedly take the
 * uncoloured p-bit with the most distinct colours among its coloured
 * neighbours, then the most neighbours, then the lowest p = (k-1) n + q, and
 * give it the smallest colour none of its neighbours has.  If that needs
 * more than four colours, use instead the fixed four classes
 *   2 [k even] + [q is a CNOT target in layer k+1]
 * (layer parity separates adjacent layers; the second bit separates the
 * control and target inputs of a CNOT).  Returns the number of classes. */
static int pbit_colours(const orc_net* net, int32_t* colour) {
  const int n = net->n, d = net->d, N = n * d;
  enum { MAXN = 8 };  /* neighbours per p-bit: at most 6 in this network */
  int* nb = (int*)malloc(sizeof(int) * (size_t)N * MAXN);
  int* deg = (int*)calloc((size_t)N, sizeof(int));
  uint32_t* seen = (uint32_t*)calloc((size_t)N, sizeof(uint32_t)); /* colours of neighbours */
  if (!nb || !deg || !seen) { free(nb); free(deg); free(seen); return -1; }
  int over = 0;
  /* join the variables of every link pairwise */
  for (int k = 1; k <= d; ++k) {
    for (int q = 0; q < n; ++q) {
      int vars[3], nv = 0;
      vars[nv++] = (k - 1) * n + q;
      const int gi = net->gate_of[(k - 1) * n + q];
      int in0 = q, in1 = -1;
      if (gi >= 0) {
        const orc_gate* G = &net->g[gi];
        if (G->op == ORC_H) continue; /* no link */
        if (G->op == ORC_CNOT) {
          if (q == G->q1) { in0 = G->q1; in1 = G->q0; } else { in0 = G->q0; }
        }
      }
      if (k >= 2) {
        vars[nv++] = (k - 2) * n + in0;
        if (in1 >= 0) vars[nv++] = (k - 2) * n + in1;
      }
      for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) {
          if (a == b) continue;
          const int u = vars[a], v = vars[b];
          int dup = 0;
          for (int e = 0; e < deg[u]; ++e) dup |= nb[u * MAXN + e] == v;
          if (dup) continue;
          if (deg[u] == MAXN) { over = 1; continue; }
          nb[u * MAXN + deg[u]++] = v;
        }
    }
  }
  int ncol = 0;
  for (int i = 0; i < N; ++i) colour[i] = -1;
  for (int step = 0; step < N && !over; ++step) {
    int best = -1, bsat = -1, bdeg = -1;
    for (int v = 0; v < N; ++v) {
      if (colour[v] >= 0) continue;
      const int sat = __builtin_popcount(seen[v]);
      if (sat > bsat || (sat == bsat && deg[v] > bdeg)) { best = v; bsat = sat; bdeg = deg[v]; }
    }
    int c = 0;
    while (c < 32 && ((seen[best] >> c) & 1u)) ++c;
    colour[best] = c;
    if (c + 1 > ncol) ncol = c + 1;
    for (int e = 0; e < deg[best]; ++e) seen[nb[best * MAXN + e]] |= 1u << c;
  }
  if (over || ncol > 4) {
    ncol = 4;
    for (int k = 1; k <= d; ++k)
      for (int q = 0; q < n; ++q) {
        int tgt = 0;
        if (k < d) {
          const int gi = net->gate_of[k * n + q]; /* layer index k maps s_k -> s_{k+1} */
          if (gi >= 0 && net->g[gi].op == ORC_CNOT && net->g[gi].q1 == q) tgt = 1;
        }
        colour[(k - 1) * n + q] = 2 * ((k % 2) == 0) + tgt;
      }
  }
  free(nb); free(deg); free(seen);
  return ncol;
}

int orc_colour(int n, int d, const orc_gate* g, int ng, int32_t* colour) {
  if (check_circuit(n, d, g, ng) != 0) return -1;
  orc_net net = {n, d, ng, g, (int32_t*)malloc((size_t)n * d * sizeof(int32_t))};
  if (!net.gate_of) return -3;
  memset(net.gate_of, -1, (size_t)n * d * sizeof(int32_t));
  for (int i = 0; i < ng; ++i) {
    net.gate_of[g[i].layer * n + g[i].q0] = i;
    if (gate_arity(g[i].op) == 2) net.gate_of[g[i].layer * n + g[i].q1] = i;
  }
  const int ncol = pbit_colours(&net, colour);
  free(net.gate_of);
  return ncol < 0 ? -3 : ncol;
}

/* Counter-based draws.  Key = seed; counter = (chain >> 5, sweep,
 * p | tag << 16, plane >> 2), p = (k-1)*n + q.  The uniform of chain c is
 * assembled from bit (c mod 32) of successive output words ("planes"), most
 * significant first: u = sum_j bit_{c mod 32}(plane_j) 2^{31-j},
 * plane_j = Philox(ctr with last word j/4)[j mod 4]. */
static uint32_t draw_uniform(uint64_t seed, uint32_t chain, uint32_t sweep,
                             uint32_t p, uint32_t tag) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t u = 0;
  for (uint32_t grp = 0; grp < 8; ++grp) {
    uint32_t ctr[4] = {chain >> 5, sweep, p | (tag << 16), grp}, out[4];
    orc_philox4x32_10(ctr, key, out);
    for (int w = 0; w < 4; ++w) {
      uint32_t j = grp * 4 + (uint32_t)w;
      u |= ((out[w] >> (chain & 31)) & 1u) << (31 - j);
    }
  }
  return u;
}

/* Initial bit of an H output: bit (c mod 32) of word 0 of
 * Philox(chain >> 5, 0, p | 1 << 16, 0). */
static int init_bit(uint64_t seed, uint32_t chain, uint32_t p) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {chain >> 5, 0, p | (1u << 16), 0}, out[4];
  orc_philox4x32_10(ctr, key, out);
  return (int)((out[0] >> (chain & 31)) & 1u);
}

/* Reference Gibbs sampler (Fig. 2 flowchart, heat-bath acceptance).
 *
 *   n, d, g, ng, beta : the circuit and its clamped input.
 *   J                 : penalty of a violated output bit (Appendix).
 *   seed              : Philox key.
 *   chain0, chains    : global ids of the chains simulated here.
 *   sweep0, sweeps    : absolute index of the first sweep, number of sweeps.
 *   burn_in, record_every : a sample is recorded after sweep t (absolute)
 *                       when t >= burn_in and (t - burn_in) % record_every == 0.
 *   init              : 1 = start from a valid path with random H outputs
 *                       (the H bits from the tag-1 stream, all other bits
 *                       their deterministic value); 0 = continue from state.
 *   state             : chains x d words, word k-1 = s_k (n bits), in/out.
 *   alphas, n_alphas  : bins to record (NULL -> all 2^n, bin = alpha).
 *   cnt               : bins x 8 counters, cnt[bin*8 + phase] += 1 per valid
 *                       recorded sample (Fig. 2 Step 3: the phase w^phase is
 *                       added to the bin of the end state).
 *   valid_total, samples_total : counters of valid / all recorded samples.
 *
 * One sweep visits the colour classes (pbit_colours) in order; within a class every
 * p-bit gets  v = viol(bit=1) - viol(bit=0)  (the change of Re E / J) and is
 * redrawn as  [v < 0] XOR [u < thr[|v|]]:  P(1) = 1/(1 + e^{J v}).
 * Invalid samples (any violated bit) carry U_C = 0 and add nothing. */
int orc_gibbs(int n, int d, const orc_gate* g, int ng, uint32_t beta, double J,
              uint64_t seed, uint32_t chain0, uint32_t chains, uint32_t sweep0,
              uint32_t sweeps, uint32_t burn_in, uint32_t record_every, int init,
              uint32_t* state, const uint32_t* alphas, int n_alphas,
              uint64_t* cnt, uint64_t* valid_total, uint64_t* samples_total) {
  if (check_circuit(n, d, g, ng) != 0) return -1;
  if (record_every == 0) return -1;
  if (!alphas && n > 24) return -2;
  uint32_t thr[4];
  if (orc_thresholds(J, thr) != 0) return -1;
  orc_net net = {n, d, ng, g, (int32_t*)malloc((size_t)n * d * sizeof(int32_t))};
  if (!net.gate_of) return -3;
  memset(net.gate_of, -1, (size_t)n * d * sizeof(int32_t));
  for (int i = 0; i < ng; ++i) {
    net.gate_of[g[i].layer * n + g[i].q0] = i;
    if (gate_arity(g[i].op) == 2) net.gate_of[g[i].layer * n + g[i].q1] = i;
  }
  const uint32_t nmask = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const uint64_t bins = alphas ? (uint64_t)n_alphas : (1ull << n);
  int32_t* col = (int32_t*)malloc((size_t)n * d * sizeof(int32_t));
  if (!col) { free(net.gate_of); return -3; }
  const int ncol = pbit_colours(&net, col);
  if (ncol < 0) { free(col); free(net.gate_of); return -3; }
  int err = 0;

#pragma omp parallel reduction(| : err)
  {
    uint64_t* my_cnt = (uint64_t*)calloc(bins * 8, sizeof(uint64_t));
    uint64_t my_valid = 0, my_samples = 0;
    uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
    if (!my_cnt || !s) err = 1;
#pragma omp for schedule(dynamic, 1)
    for (int64_t ci = 0; ci < (int64_t)chains; ++ci) {
      if (err) continue;
      const uint32_t chain = chain0 + (uint32_t)ci;
      uint32_t* st = state + (size_t)ci * d;
      s[0] = beta & nmask;
      if (init) {
        for (int k = 1; k <= d; ++k) {
          uint32_t w = 0;
          for (int q = 0; q < n; ++q) {
            int gi = net.gate_of[(k - 1) * n + q];
            int b;
            if (gi >= 0 && g[gi].op == ORC_H) {
              b = init_bit(seed, chain, (uint32_t)((k - 1) * n + q));
            } else if (gi < 0) {
              b = bit(s[k - 1], q);
            } else {
              const orc_gate* G = &g[gi];
              int ystar = det_output(G->op, gate_index(G, s[k - 1]));
              b = (q == G->q0) ? (ystar & 1) : ((ystar >> 1) & 1);
            }
            w |= (uint32_t)b << q;
          }
          s[k] = w;
        }
      } else {
        for (int k = 1; k <= d; ++k) s[k] = st[k - 1] & nmask;
      }
      for (uint32_t t = 0; t < sweeps; ++t) {
        const uint32_t sweep = sweep0 + t;
        for (int colour = 0; colour < ncol; ++colour) {
          for (int k = 1; k <= d; ++k) {
            for (int q = 0; q < n; ++q) {
              if (col[(k - 1) * n + q] != colour) continue;
              /* change of the violation count when bit (k,q) goes 0 -> 1;
               * only layers k-1 -> k and k -> k+1 involve s_k. */
              uint32_t keep = s[k];
              s[k] = keep | (1u << q);
              int v1 = layer_violations(&net, k - 1, s[k - 1], s[k]) +
                       (k < d ? layer_violations(&net, k, s[k], s[k + 1]) : 0);
              s[k] = keep & ~(1u << q);
              int v0 = layer_violations(&net, k - 1, s[k - 1], s[k]) +
                       (k < d ? layer_violations(&net, k, s[k], s[k + 1]) : 0);
              int v = v1 - v0;
              uint32_t p = (uint32_t)((k - 1) * n + q);
              uint32_t u = draw_uniform(seed, chain, sweep, p, 0);
              int av = v < 0 ? -v : v;
              int b = (v < 0) ^ (u < thr[av]);
              s[k] = (keep & ~(1u << q)) | ((uint32_t)b << q);
            }
          }
        }
        if (sweep >= burn_in && (sweep - burn_in) % record_every == 0) {
          ++my_samples;
          if (total_violations(&net, s) == 0) {
            ++my_valid;
            int ph = path_phase(&net, s);
            if (ph < 0) { err = 1; break; }
            if (alphas) {
              for (int a = 0; a < n_alphas; ++a)
                if (alphas[a] == s[d]) { my_cnt[(uint64_t)a * 8 + ph] += 1; break; }
            } else {
              my_cnt[(uint64_t)s[d] * 8 + ph] += 1;
            }
          }
        }
      }
      for (int k = 1; k <= d; ++k) st[k - 1] = s[k];
    }
#pragma omp critical
    {
      if (my_cnt)
        for (uint64_t i = 0; i < bins * 8; ++i) cnt[i] += my_cnt[i];
      *valid_total += my_valid;
      *samples_total += my_samples;
    }
    free(my_cnt);
    free(s);
  }
  free(col);
  free(net.gate_of);
  return err ? -4 : 0;
}

/* Exact path sampler on the eliminated network (R2; Appendix: with the
 * J-penalty links removed, the non-H bits are functions of the previous
 * layer and each H output is a free fair coin).  A sample is one pass from
 * the clamped input: layer by layer, an H output (k, q) of chain c at
 * sample t is bit (c mod 32) of word 0 of Philox(c >> 5, t, p | 4 << 16, 0),
 * p = (k-1) n + q; every other bit is its gate's deterministic value.  The
 * path is valid by construction, so every recorded sample adds one count to
 * (end state, phase) (Fig. 2 Step 3) and the samples are i.i.d. and uniform
 * over the 2^h valid paths.
 *
 *   sweep0, sweeps, burn_in, record_every: sample indices t = sweep0 ..
 *       sweep0 + sweeps - 1; only recorded ones (t >= burn_in and
 *       (t - burn_in) % record_every == 0) are drawn.
 *   state (optional, chains x d): the last drawn path of each chain.
 *   alphas, cnt, valid_total, samples_total: as for orc_gibbs. */
int orc_elim(int n, int d, const orc_gate* g, int ng, uint32_t beta, uint64_t seed,
             uint32_t chain0, uint32_t chains, uint32_t sweep0, uint32_t sweeps,
             uint32_t burn_in, uint32_t record_every, uint32_t* state,
             const uint32_t* alphas, int n_alphas, uint64_t* cnt, uint64_t* valid_total,
             uint64_t* samples_total) {
  if (check_circuit(n, d, g, ng) != 0) return -1;
  if (record_every == 0) return -1;
  if (!alphas && n > 24) return -2;
  orc_net net = {n, d, ng, g, (int32_t*)malloc((size_t)n * d * sizeof(int32_t))};
  if (!net.gate_of) return -3;
  memset(net.gate_of, -1, (size_t)n * d * sizeof(int32_t));
  for (int i = 0; i < ng; ++i) {
    net.gate_of[g[i].layer * n + g[i].q0] = i;
    if (gate_arity(g[i].op) == 2) net.gate_of[g[i].layer * n + g[i].q1] = i;
  }
  const uint32_t nmask = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const uint64_t bins = alphas ? (uint64_t)n_alphas : (1ull << n);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int err = 0;

#pragma omp parallel reduction(| : err)
  {
    uint64_t* my_cnt = (uint64_t*)calloc(bins * 8, sizeof(uint64_t));
    uint64_t my_valid = 0, my_samples = 0;
    uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
    if (!my_cnt || !s) err = 1;
#pragma omp for schedule(dynamic, 1)
    for (int64_t ci = 0; ci < (int64_t)chains; ++ci) {
      if (err) continue;
      const uint32_t chain = chain0 + (uint32_t)ci;
      int drawn = 0;
      for (uint32_t i = 0; i < sweeps; ++i) {
        const uint32_t t = sweep0 + i;
        if (!(t >= burn_in && (t - burn_in) % record_every == 0)) continue;
        s[0] = beta & nmask;
        for (int k = 1; k <= d; ++k) {
          uint32_t w = 0;
          for (int q = 0; q < n; ++q) {
            const int gi = net.gate_of[(k - 1) * n + q];
            int b;
            if (gi >= 0 && g[gi].op == ORC_H) {
              const uint32_t p = (uint32_t)((k - 1) * n + q);
              uint32_t ctr[4] = {chain >> 5, t, p | (4u << 16), 0}, out[4];
              orc_philox4x32_10(ctr, key, out);
              b = (int)((out[0] >> (chain & 31)) & 1u);
            } else if (gi < 0) {
              b = bit(s[k - 1], q);
            } else {
              const orc_gate* G = &g[gi];
              const int ystar = det_output(G->op, gate_index(G, s[k - 1]));
              b = (q == G->q0) ? (ystar & 1) : ((ystar >> 1) & 1);
            }
            w |= (uint32_t)b << q;
          }
          s[k] = w;
        }
        drawn = 1;
        ++my_samples;
        if (total_violations(&net, s) != 0) { err = 1; break; }  /* cannot happen */
        ++my_valid;
        const int ph = path_phase(&net, s);
        if (ph < 0) { err = 1; break; }
        if (alphas) {
          for (int a = 0; a < n_alphas; ++a)
            if (alphas[a] == s[d]) { my_cnt[(uint64_t)a * 8 + ph] += 1; break; }
        } else {
          my_cnt[(uint64_t)s[d] * 8 + ph] += 1;
        }
      }
      if (state && drawn)
        for (int k = 1; k <= d; ++k) state[(size_t)ci * d + k - 1] = s[k];
    }
#pragma omp critical
    {
      if (my_cnt)
        for (uint64_t i = 0; i < bins * 8; ++i) cnt[i] += my_cnt[i];
      *valid_total += my_valid;
      *samples_total += my_samples;
    }
    free(my_cnt);
    free(s);
  }
  free(net.gate_of);
  return err ? -4 : 0;
}

/* End state s_d of the path whose H outputs (in p order) are x[0..h-1]. */
static uint32_t propagate_with(const orc_net* net, uint32_t beta, const uint8_t* x, uint32_t* s) {
  const int n = net->n, d = net->d;
  const uint32_t nmask = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  int j = 0;
  s[0] = beta & nmask;
  for (int k = 1; k <= d; ++k) {
    uint32_t w = 0;
    for (int q = 0; q < n; ++q) {
      const int gi = net->gate_of[(k - 1) * n + q];
      int b;
      if (gi >= 0 && net->g[gi].op == ORC_H) {
        b = x[j++];
      } else if (gi < 0) {
        b = bit(s[k - 1], q);
      } else {
        const orc_gate* G = &net->g[gi];
        const int ystar = det_output(G->op, gate_index(G, s[k - 1]));
        b = (q == G->q0) ? (ystar & 1) : ((ystar >> 1) & 1);
      }
      w |= (uint32_t)b << q;
    }
    s[k] = w;
  }
  return s[d];
}

/* Output-clamped exact sampler ("for a given input beta and output alpha",
 * Sec. 3, with the eliminated network of the Appendix).  Every wire bit is
 * an affine function over GF(2) of the H outputs x (in p order), so
 * s_d = A x + c, and the valid paths ending at alpha are the solutions of
 * A x = alpha + c: an affine subspace of dimension h - r, or none.  A and c
 * come from h + 1 probe paths (x = 0 and the unit vectors).  With the
 * reduced row echelon form of [A | alpha + c] (unique), the free variables
 * (non-pivot columns, increasing) take the draws z_0, z_1, ..., and each
 * pivot variable is its row's right-hand side XOR the free variables in
 * that row.  Draw z_b of chain c at sample t: bit (c mod 32) of word b mod 4
 * of Philox(c >> 5, t, (b >> 2) | 5 << 16, 0).  Each recorded sample adds one
 * count to cnt[phase]; the estimator of U_{alpha,beta} =
 * 2^{-h/2} sum_{paths to alpha} w^phase is 2^{h/2 - r} sum_phi cnt[phi] w^phi / T.
 *
 *   consistent_out : 1 if alpha is reachable (else no sample is drawn).
 *   nfree_out, rank_out : h - r and r.
 *   state (optional, chains x d): the last drawn path of each chain. */
int orc_elim_clamped(int n, int d, const orc_gate* g, int ng, uint32_t beta, uint32_t alpha,
                     uint64_t seed, uint32_t chain0, uint32_t chains, uint32_t sweep0,
                     uint32_t sweeps, uint32_t burn_in, uint32_t record_every, uint32_t* state,
                     uint64_t* cnt8, uint64_t* samples_total, int* consistent_out,
                     int* nfree_out, int* rank_out) {
  if (check_circuit(n, d, g, ng) != 0) return -1;
  if (record_every == 0) return -1;
  orc_net net = {n, d, ng, g, (int32_t*)malloc((size_t)n * d * sizeof(int32_t))};
  if (!net.gate_of) return -3;
  memset(net.gate_of, -1, (size_t)n * d * sizeof(int32_t));
  for (int i = 0; i < ng; ++i) {
    net.gate_of[g[i].layer * n + g[i].q0] = i;
    if (gate_arity(g[i].op) == 2) net.gate_of[g[i].layer * n + g[i].q1] = i;
  }
  int h = 0;
  for (int i = 0; i < ng; ++i) h += g[i].op == ORC_H;
  /* augmented matrix M[row q][col j], col h = right-hand side */
  uint8_t* M = (uint8_t*)calloc((size_t)n * (h + 1), 1);
  uint8_t* x = (uint8_t*)calloc((size_t)h + 1, 1);
  uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
  int* pivot_col = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  int* free_col = (int*)malloc(sizeof(int) * (size_t)(h + 1));
  if (!M || !x || !s || !pivot_col || !free_col) return -3;
  const uint32_t c0 = propagate_with(&net, beta, x, s);
  for (int j = 0; j < h; ++j) {
    x[j] = 1;
    const uint32_t cj = propagate_with(&net, beta, x, s);
    x[j] = 0;
    for (int q = 0; q < n; ++q) M[(size_t)q * (h + 1) + j] = (uint8_t)bit(cj ^ c0, q);
  }
  for (int q = 0; q < n; ++q) M[(size_t)q * (h + 1) + h] = (uint8_t)bit(alpha ^ c0, q);
  /* Gauss-Jordan elimination over GF(2) */
  int r = 0;
  for (int j = 0; j < h && r < n; ++j) {
    int piv = -1;
    for (int q = r; q < n; ++q)
      if (M[(size_t)q * (h + 1) + j]) { piv = q; break; }
    if (piv < 0) continue;
    if (piv != r)
      for (int c = 0; c <= h; ++c) {
        uint8_t t = M[(size_t)piv * (h + 1) + c];
        M[(size_t)piv * (h + 1) + c] = M[(size_t)r * (h + 1) + c];
        M[(size_t)r * (h + 1) + c] = t;
      }
    for (int q = 0; q < n; ++q)
      if (q != r && M[(size_t)q * (h + 1) + j])
        for (int c = 0; c <= h; ++c) M[(size_t)q * (h + 1) + c] ^= M[(size_t)r * (h + 1) + c];
    pivot_col[r++] = j;
  }
  int consistent = 1;
  for (int q = r; q < n; ++q)
    if (M[(size_t)q * (h + 1) + h]) consistent = 0;
  int nfree = 0;
  for (int j = 0, i = 0; j < h; ++j) {
    if (i < r && pivot_col[i] == j) { ++i; continue; }
    free_col[nfree++] = j;
  }
  *consistent_out = consistent;
  *nfree_out = nfree;
  *rank_out = r;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int err = 0;
  uint64_t my_samples = 0;
  if (consistent) {
    for (uint32_t ci = 0; ci < chains && !err; ++ci) {
      const uint32_t chain = chain0 + ci;
      int drawn = 0;
      for (uint32_t i = 0; i < sweeps; ++i) {
        const uint32_t t = sweep0 + i;
        if (!(t >= burn_in && (t - burn_in) % record_every == 0)) continue;
        /* free variables from the draws, pivots from their rows */
        for (int b = 0; b < nfree; ++b) {
          uint32_t ctr[4] = {chain >> 5, t, ((uint32_t)b >> 2) | (5u << 16), 0}, out[4];
          orc_philox4x32_10(ctr, key, out);
          x[free_col[b]] = (uint8_t)((out[b & 3] >> (chain & 31)) & 1u);
        }
        for (int row = 0; row < r; ++row) {
          uint8_t v = M[(size_t)row * (h + 1) + h];
          for (int b = 0; b < nfree; ++b)
            if (M[(size_t)row * (h + 1) + free_col[b]]) v ^= x[free_col[b]];
          x[pivot_col[row]] = v;
        }
        if (propagate_with(&net, beta, x, s) != alpha) { err = 1; break; }
        if (total_violations(&net, s) != 0) { err = 1; break; }
        const int ph = path_phase(&net, s);
        if (ph < 0) { err = 1; break; }
        cnt8[ph] += 1;
        ++my_samples;
        drawn = 1;
      }
      if (state && drawn)
        for (int k = 1; k <= d; ++k) state[(size_t)ci * d + k - 1] = s[k];
    }
  }
  *samples_total += my_samples;
  free(M); free(x); free(s); free(pivot_col); free(free_col);
  free(net.gate_of);
  return err ? -4 : 0;
}

/* Total violated output bits of each chain state (chains x d words). */
int orc_violations(int n, int d, const orc_gate* g, int ng, uint32_t beta,
                   uint32_t chains, const uint32_t* state, int32_t* viol) {
  if (check_circuit(n, d, g, ng) != 0) return -1;
  orc_net net = {n, d, ng, g, (int32_t*)malloc((size_t)n * d * sizeof(int32_t))};
  if (!net.gate_of) return -3;
  memset(net.gate_of, -1, (size_t)n * d * sizeof(int32_t));
  for (int i = 0; i < ng; ++i) {
    net.gate_of[g[i].layer * n + g[i].q0] = i;
    if (gate_arity(g[i].op) == 2) net.gate_of[g[i].layer * n + g[i].q1] = i;
  }
  uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
  const uint32_t nmask = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  for (uint32_t c = 0; c < chains; ++c) {
    s[0] = beta & nmask;
    for (int k = 1; k <= d; ++k) s[k] = state[(size_t)c * d + k - 1];
    viol[c] = total_violations(&net, s);
  }
  free(s);
  free(net.gate_of);
  return 0;
}

/* Phase units of one path (the layer elements' phases summed, Eq. path), or
 * -1 if some element is zero. */
int orc_path_phase(int n, int d, const orc_gate* g, int ng, uint32_t beta,
                   const uint32_t* s1_to_sd) {
  if (check_circuit(n, d, g, ng) != 0) return -2;
  uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
  int32_t* gate_of = (int32_t*)malloc((size_t)n * d * sizeof(int32_t));
  memset(gate_of, -1, (size_t)n * d);
  orc_net net = {n, d, ng, g, gate_of};
  s[0] = beta;
  for (int k = 1; k <= d; ++k) s[k] = s1_to_sd[k - 1];
  int ph = path_phase(&net, s);
  free(s);
  free(gate_of);
  return ph;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops that follow (at least 1); returns the count in
 * force.  For timing the same code on one core and on all of them. */
int orc_set_num_threads(int t) {
#ifdef _OPENMP
  omp_set_num_threads(t < 1 ? 1 : t);
  return omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}
