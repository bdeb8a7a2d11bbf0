/*
 * CPU oracle, part 2: circuits with general one-qubit gates (arXiv 2007.07379,
 * Sec. 2 Eq. EB; Sec. 4.2 Eq. HadT and Fig. 5).
 *
 * TEST INFRASTRUCTURE ONLY, under the same rules as oracle.c (which it is
 * linked with: it calls that file's exported Philox and colouring).  Plain
 * scalar FP64, written to be checked against the paper by eye.
 *
 * A gate row with op = ORC_U (5) carries a 2x2 complex matrix U, rows =
 * output bit, columns = input bit (U_yx = <y|U|x>, the kbordermatrix of
 * Sec. 2), stored as mats[32 i + 0..7] = Re U00, Im U00, Re U01, Im U01,
 * Re U10, Im U10, Re U11, Im U11 for gate row i.  op = ORC_X (6) is the
 * Pauli X of the Appendix (a deterministic NOT, no phase).  op = ORC_U2 (7)
 * is a two-qubit gate on (q0, q1) with a 4x4 complex matrix,
 * mats[32 i + 2 (4 y + x)] = Re, + 1 = Im of <y|U|x>, basis index
 * x = x_{q0} + 2 x_{q1} (the order 00, 10, 01, 11 of Eq. ET2); it must be
 * unitary within 1e-9 with exactly one nonzero entry per column (a
 * permutation with phases: SWAP, the Appendix's exchange operator J12,
 * controlled phases, ...).  Every permutation of two bits is affine over
 * GF(2), so each output bit is a copy or an XOR of the input bits, possibly
 * complemented; an output bit that is the complement of an XOR of both
 * inputs is rejected (the J-penalty links carry at most two words).  A
 * unitary U2 with a column of more than one nonzero is a "table" gate
 * (Eq. ET2): both outputs are free and carry the real energy
 * E(y, x) = -ln |U(y, x)| (J for a zero entry, the Appendix's e^{-J}); a
 * path through a zero entry is invalid; with unequal column sums of |U|
 * the estimator has no closed-form scale (log2z is NaN) and is read
 * L2-normalised (Fig. 2 Step 4).  Rows
 * with other ops are the Clifford+T gates of oracle.c; their mats entries
 * are ignored.  op = ORC_CCX (8) is the Toffoli gate of the Appendix on
 * (q0, q1, q2), controls q0 and q1, target q2: x_{q2} XOR= x_{q0} x_{q1},
 * a deterministic gate whose target output is J-linked to that value.
 *
 * Paths and weights (Eq. U, Eq. path): the weight of a path is the product
 * of its layer elements, complex FP64 here.  Sampling (Eq. weightedS): a path
 * is drawn with probability proportional to |U_C|.
 *
 * Kinds of ORC_U gates (the J-penalty form of the Appendix):
 *   diagonal       U01 = U10 = 0 exactly: the output copies the input; a
 *                  different output bit costs J.
 *   anti-diagonal  U00 = U11 = 0 exactly: the output is NOT the input; the
 *                  copy costs J.
 *   coupled        all four entries nonzero: the output bit is free and the
 *                  real part of E (Eq. EB) is, up to a constant,
 *                      K [s_out != s_in],   K = ln(a / b),
 *                  a = (|U00| + |U11|) / 2, b = (|U01| + |U10|) / 2: for a
 *                  unitary |U00| = |U11| and |U01| = |U10|, so the one-body
 *                  terms ln|a1/c1| s_d + ln|a1/b1| s_{d-1} and the two-body
 *                  term ln|b1 c1 / (a1 A1)| s_{d-1} s_d of Eq. EB combine into
 *                  K (s_d + s_{d-1} - 2 s_{d-1} s_d) = K [s_d != s_{d-1}].
 *   Anything else (one zero entry, or a matrix more than 1e-9 from unitary)
 *   is rejected.  |z| = hypot(Re z, Im z).
 *
 * Contents:
 *   orc_u_statevector  psi = U^(d)...U^(1)|beta>, FP64 (Eq. U).
 *   orc_u_pathstats    brute-force path sum per output alpha: U_alpha,
 *                      Z_alpha = sum |U_C|, sum |U_C|^2, number of nonzero
 *                      paths (Eqs. U343-U30: the std prefactor of weighted
 *                      and of uniform sampling, Fig. 5).
 *   orc_u_gibbs        reference Gibbs sampler (Fig. 2): heat-bath proposal
 *                      on the J-penalty energy, Metropolis acceptance on the
 *                      coupling energy, FP64 phase sums per output.
 *   orc_u_elim         exact i.i.d. sampler (eliminated network, Appendix):
 *                      coupled outputs drawn with P(s_out != s_in) = b/(a+b).
 *   orc_u_log2z        log2 of the estimator scale 2^{h/2} prod (a + b).
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

enum { G_H = 0, G_S = 1, G_T = 2, G_CNOT = 3, G_CZ = 4, G_U = 5, G_X = 6, G_U2 = 7, G_CCX = 8 };
enum { K_STD = 0, K_DIAG = 1, K_ANTI = 2, K_COUPLED = 3, K_TABLE = 4 };
enum { MAT = 32 }; /* doubles per gate row of mats */

/* from oracle.c */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);
int orc_thresholds(double J, uint32_t thr[4]);

static int arity(int op) {
  return op == G_CCX ? 3 : (op == G_CNOT || op == G_CZ || op == G_U2) ? 2 : 1;
}
static int bitof(uint32_t w, int q) { return (int)((w >> q) & 1u); }

/* ------------------------------------------------------------------------ */
/* Gate entries as complex numbers.  Index of a 2-qubit gate's basis state:
 * x = x_{q0} + 2 x_{q1}. */
static void std_entry(int op, int y, int x, double* re, double* im) {
  const double r2 = 1.0 / sqrt(2.0);
  *re = 0.0;
  *im = 0.0;
  switch (op) {
    case G_H: /* (1/sqrt2) [[1, 1], [1, -1]]  (Eq. Had) */
      *re = (y == 1 && x == 1) ? -r2 : r2;
      break;
    case G_S: /* diag(1, i) */
      if (y == x) { if (x == 0) *re = 1.0; else *im = 1.0; }
      break;
    case G_T: /* diag(1, e^{i pi/4}) */
      if (y == x) {
        if (x == 0) *re = 1.0;
        else { *re = cos(M_PI / 4.0); *im = sin(M_PI / 4.0); }
      }
      break;
    case G_CNOT: { /* control q0, target q1: (c, t) -> (c, t ^ c) */
      const int c = x & 1, t = (x >> 1) & 1;
      if (y == (c | ((t ^ c) << 1))) *re = 1.0;
      break;
    }
    case G_CZ: /* diag(1, 1, 1, -1) */
      if (y == x) *re = (x == 3) ? -1.0 : 1.0;
      break;
    case G_X: /* [[0, 1], [1, 0]] */
      if (y != x) *re = 1.0;
      break;
    case G_CCX: /* controls q0, q1, target q2 (x = x0 + 2 x1 + 4 x2): x2 ^= x0 x1 */
      if (y == (x ^ (((x & 1) && (x & 2)) ? 4 : 0))) *re = 1.0;
      break;
  }
}

static void u2_entry(const double* m32, int y, int x, double* re, double* im) {
  const int k = 2 * (4 * y + x);
  *re = m32[k];
  *im = m32[k + 1];
}

/* A two-qubit gate, unitary within 1e-9.  One nonzero per column: perm[x] =
 * the row of column x's nonzero, dmask[o] (bit u: output bit o depends on
 * input bit u) and cbit[o] of the affine map; returns 0.  A column of more
 * than one nonzero: a table gate, returns 1.  -1 if rejected. */
static int u2_classify(const double* m, int perm[4], int dmask[2], int cbit[2]) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double sr = 0.0, si = 0.0;
      for (int y = 0; y < 4; ++y) {
        double ar, ai, br, bi;
        u2_entry(m, y, i, &ar, &ai);
        u2_entry(m, y, j, &br, &bi);
        sr += ar * br + ai * bi;
        si += ar * bi - ai * br;
      }
      if (fabs(sr - (i == j ? 1.0 : 0.0)) > 1e-9 || fabs(si) > 1e-9) return -1;
    }
  for (int x = 0; x < 4; ++x) {
    int nz = 0;
    for (int y = 0; y < 4; ++y) {
      double r, i;
      u2_entry(m, y, x, &r, &i);
      if (r != 0.0 || i != 0.0) { perm[x] = y; ++nz; }
    }
    if (nz != 1) return 1; /* a table gate */
  }
  for (int o = 0; o < 2; ++o) {
    const int c = (perm[0] >> o) & 1, al = ((perm[1] >> o) & 1) ^ c, be = ((perm[2] >> o) & 1) ^ c;
    if ((((perm[3] >> o) & 1) ^ c) != (al ^ be)) return -1; /* not affine (cannot happen) */
    dmask[o] = al | (be << 1);
    cbit[o] = c;
    if (dmask[o] == 0) return -1;
    if (dmask[o] == 3 && c) return -1; /* complement of x1 XOR x2: not representable */
  }
  return 0;
}

static void u_entry(const double* m8, int y, int x, double* re, double* im) {
  const int k = 2 * (2 * y + x);
  *re = m8[k];
  *im = m8[k + 1];
}

static double u_abs(const double* m8, int y, int x) {
  const int k = 2 * (2 * y + x);
  return hypot(m8[k], m8[k + 1]);
}

/* Kind of an ORC_U gate, its a, b and K; -1 if rejected. */
static int u_kind(const double* m8, double* a, double* b, double* K) {
  /* unitarity: U^dagger U = I within 1e-9 */
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double sr = 0.0, si = 0.0;
      for (int y = 0; y < 2; ++y) {
        double ar, ai, br, bi;
        u_entry(m8, y, i, &ar, &ai);
        u_entry(m8, y, j, &br, &bi);
        sr += ar * br + ai * bi; /* conj(U_yi) U_yj */
        si += ar * bi - ai * br;
      }
      if (fabs(sr - (i == j ? 1.0 : 0.0)) > 1e-9 || fabs(si) > 1e-9) return -1;
    }
  const int z00 = m8[0] == 0.0 && m8[1] == 0.0, z01 = m8[2] == 0.0 && m8[3] == 0.0;
  const int z10 = m8[4] == 0.0 && m8[5] == 0.0, z11 = m8[6] == 0.0 && m8[7] == 0.0;
  *a = 0.5 * (u_abs(m8, 0, 0) + u_abs(m8, 1, 1));
  *b = 0.5 * (u_abs(m8, 0, 1) + u_abs(m8, 1, 0));
  *K = 0.0;
  if (z01 && z10 && !z00 && !z11) return K_DIAG;
  if (z00 && z11 && !z01 && !z10) return K_ANTI;
  if (z00 || z01 || z10 || z11) return -1;
  *K = log(*a / *b);
  return K_COUPLED;
}

/* Complex element <y|G|x> of gate row i (its own index convention). */
static void gate_elem(const orc_gate* G, const double* mats, int i, int y, int x, double* re,
                      double* im) {
  if (G->op == G_U) u_entry(mats + (size_t)MAT * i, y, x, re, im);
  else if (G->op == G_U2) u2_entry(mats + (size_t)MAT * i, y, x, re, im);
  else std_entry(G->op, y, x, re, im);
}

static int gidx(const orc_gate* G, uint32_t w) {
  const int a = arity(G->op);
  if (a == 3) return bitof(w, G->q0) + 2 * bitof(w, G->q1) + 4 * bitof(w, G->q2);
  return a == 2 ? bitof(w, G->q0) + 2 * bitof(w, G->q1) : bitof(w, G->q0);
}

typedef struct {
  int n, d, ng;
  const orc_gate* g;
  const double* mats;
  int32_t* gate_of; /* [d][n] gate row acting on (layer, qubit), or -1 */
  int* kind;        /* per gate row: K_STD or the ORC_U kind */
  double *a, *b, *K;
  int (*perm)[4];   /* per gate row (ORC_U2): the permutation */
  int (*dmask)[2], (*cbit)[2];
} unet;

static void unet_free(unet* u) {
  free(u->gate_of); free(u->kind); free(u->a); free(u->b); free(u->K);
  free(u->perm); free(u->dmask); free(u->cbit);
}

/* Checks the circuit and classifies its gates; 0 on success. */
static int unet_init(unet* u, int n, int d, const orc_gate* g, int ng, const double* mats) {
  memset(u, 0, sizeof *u);
  if (n < 1 || n > 32 || d < 1 || d > 64 || ng < 0) return -1;
  u->n = n; u->d = d; u->ng = ng; u->g = g; u->mats = mats;
  u->gate_of = (int32_t*)malloc((size_t)n * d * sizeof(int32_t));
  u->kind = (int*)calloc((size_t)ng + 1, sizeof(int));
  u->a = (double*)calloc((size_t)ng + 1, sizeof(double));
  u->b = (double*)calloc((size_t)ng + 1, sizeof(double));
  u->K = (double*)calloc((size_t)ng + 1, sizeof(double));
  u->perm = calloc((size_t)ng + 1, sizeof *u->perm);
  u->dmask = calloc((size_t)ng + 1, sizeof *u->dmask);
  u->cbit = calloc((size_t)ng + 1, sizeof *u->cbit);
  if (!u->gate_of || !u->kind || !u->a || !u->b || !u->K || !u->perm || !u->dmask || !u->cbit) {
    unet_free(u);
    return -3;
  }
  for (int i = 0; i < n * d; ++i) u->gate_of[i] = -1;
  for (int i = 0; i < ng; ++i) {
    const orc_gate* G = &g[i];
    if (G->op < 0 || G->op > G_CCX || G->layer < 0 || G->layer >= d || G->q0 < 0 || G->q0 >= n) {
      unet_free(u); return -1;
    }
    if (arity(G->op) >= 2 && (G->q1 < 0 || G->q1 >= n || G->q1 == G->q0)) { unet_free(u); return -1; }
    if (arity(G->op) == 3 && (G->q2 < 0 || G->q2 >= n || G->q2 == G->q0 || G->q2 == G->q1)) {
      unet_free(u); return -1;
    }
    int* s0 = &u->gate_of[G->layer * n + G->q0];
    if (*s0 >= 0) { unet_free(u); return -1; }
    *s0 = i;
    if (arity(G->op) >= 2) {
      int* s1 = &u->gate_of[G->layer * n + G->q1];
      if (*s1 >= 0) { unet_free(u); return -1; }
      *s1 = i;
    }
    if (arity(G->op) == 3) {
      int* s2 = &u->gate_of[G->layer * n + G->q2];
      if (*s2 >= 0) { unet_free(u); return -1; }
      *s2 = i;
    }
    u->kind[i] = K_STD;
    if (G->op == G_U) {
      if (!mats) { unet_free(u); return -1; }
      const int k = u_kind(mats + (size_t)MAT * i, &u->a[i], &u->b[i], &u->K[i]);
      if (k < 0) { unet_free(u); return -1; }
      u->kind[i] = k;
    }
    if (G->op == G_U2) {
      const int k = mats ? u2_classify(mats + (size_t)MAT * i, u->perm[i], u->dmask[i], u->cbit[i]) : -1;
      if (k < 0) { unet_free(u); return -1; }
      if (k == 1) u->kind[i] = K_TABLE;
    }
  }
  return 0;
}

/* Complex element of layer L between input word x and output word y. */
static void layer_elem(const unet* u, int L, uint32_t x, uint32_t y, double* re, double* im) {
  double wr = 1.0, wi = 0.0;
  for (int q = 0; q < u->n; ++q) {
    const int gi = u->gate_of[L * u->n + q];
    if (gi < 0) {
      if (bitof(x, q) != bitof(y, q)) { *re = 0.0; *im = 0.0; return; }
      continue;
    }
    const orc_gate* G = &u->g[gi];
    if (q != G->q0) continue; /* a 2-qubit gate once, at q0 */
    double er, ei;
    gate_elem(G, u->mats, gi, gidx(G, y), gidx(G, x), &er, &ei);
    const double tr = wr * er - wi * ei, ti = wr * ei + wi * er;
    wr = tr;
    wi = ti;
  }
  *re = wr;
  *im = wi;
}

/* ------------------------------------------------------------------------ */
int orc_u_statevector(int n, int d, const orc_gate* g, int ng, const double* mats, uint32_t beta,
                      double* re, double* im) {
  unet u;
  if (n > 24 || unet_init(&u, n, d, g, ng, mats) != 0) return -1;
  const uint64_t N = 1ull << n;
  double* nr = (double*)calloc(N, sizeof(double));
  double* ni = (double*)calloc(N, sizeof(double));
  if (!nr || !ni) { free(nr); free(ni); unet_free(&u); return -3; }
  memset(re, 0, N * sizeof(double));
  memset(im, 0, N * sizeof(double));
  re[beta & (N - 1)] = 1.0;
  /* gates of one layer act on disjoint qubits: apply them one at a time,
   * psi'_y = sum_x <y|G|x> psi_x over the gate's qubits */
  for (int L = 0; L < d; ++L)
    for (int i = 0; i < ng; ++i) {
      const orc_gate* G = &g[i];
      if (G->layer != L) continue;
      const int ar = arity(G->op), dim = 1 << ar;
      const uint64_t m0 = 1ull << G->q0, m1 = ar >= 2 ? (1ull << G->q1) : 0,
                     m2 = ar == 3 ? (1ull << G->q2) : 0;
      memset(nr, 0, N * sizeof(double));
      memset(ni, 0, N * sizeof(double));
      for (uint64_t idx = 0; idx < N; ++idx) {
        const int x = ((idx & m0) ? 1 : 0) + ((idx & m1) ? 2 : 0) + ((idx & m2) ? 4 : 0);
        const uint64_t rest = idx & ~(m0 | m1 | m2);
        for (int y = 0; y < dim; ++y) {
          double er, ei;
          gate_elem(G, mats, i, y, x, &er, &ei);
          if (er == 0.0 && ei == 0.0) continue;
          const uint64_t j = rest | ((y & 1) ? m0 : 0) | ((y & 2) ? m1 : 0) | ((y & 4) ? m2 : 0);
          nr[j] += er * re[idx] - ei * im[idx];
          ni[j] += er * im[idx] + ei * re[idx];
        }
      }
      memcpy(re, nr, N * sizeof(double));
      memcpy(im, ni, N * sizeof(double));
    }
  free(nr); free(ni);
  unet_free(&u);
  return 0;
}

/* Brute-force path sum: every path beta -> s_1 -> ... -> s_d (s_d = alpha)
 * with weight U_C = product of its layer elements.  Per alpha:
 *   ure/uim = U_alpha = sum_C U_C,   zabs = sum_C |U_C|,
 *   s2 = sum_C |U_C|^2,   npath = number of paths with U_C != 0.
 * With p_C = |U_C| / zabs over the paths to alpha, W_C = U_C / p_C and
 * Eq. U30 gives std = sqrt(zabs^2 - |U_alpha|^2); with uniform p_C = 1/npath,
 * std = sqrt(npath s2 - |U_alpha|^2).  Cost 2^{n d}: n d <= 24. */
int orc_u_pathstats(int n, int d, const orc_gate* g, int ng, const double* mats, uint32_t beta,
                    double* ure, double* uim, double* zabs, double* s2, uint64_t* npath) {
  unet u;
  if (n * d > 24 || unet_init(&u, n, d, g, ng, mats) != 0) return -1;
  const uint64_t N = 1ull << n, total = 1ull << (n * d);
  const uint32_t nmask = (uint32_t)(N - 1);
  for (uint64_t a = 0; a < N; ++a) { ure[a] = uim[a] = zabs[a] = s2[a] = 0.0; npath[a] = 0; }
  uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
  if (!s) { unet_free(&u); return -3; }
  for (uint64_t code = 0; code < total; ++code) {
    s[0] = beta & nmask;
    for (int k = 1; k <= d; ++k) s[k] = (uint32_t)((code >> ((k - 1) * n)) & nmask);
    double wr = 1.0, wi = 0.0;
    for (int L = 0; L < d && (wr != 0.0 || wi != 0.0); ++L) {
      double er, ei;
      layer_elem(&u, L, s[L], s[L + 1], &er, &ei);
      const double tr = wr * er - wi * ei, ti = wr * ei + wi * er;
      wr = tr;
      wi = ti;
    }
    if (wr == 0.0 && wi == 0.0) continue;
    const uint32_t al = s[d];
    const double m = hypot(wr, wi);
    ure[al] += wr;
    uim[al] += wi;
    zabs[al] += m;
    s2[al] += m * m;
    npath[al] += 1;
  }
  free(s);
  unet_free(&u);
  return 0;
}

/* log2 of the estimator scale: a valid path has |U_C| =
 * 2^{-h/2} prod_{coupled} (a or b) and sum over all paths of |U_C| =
 * 2^{h/2} prod_{coupled} (a + b) (each coupled gate's column of |U| sums to
 * a + b, every other layer factor's columns to 1 or sqrt2), so with
 * p_C = |U_C| / Z the sample weight W_C = Z e^{i arg U_C}. */
static double log2_scale(const unet* u) {
  double l = 0.0;
  for (int i = 0; i < u->ng; ++i) {
    if (u->g[i].op == G_U2 && u->kind[i] == K_TABLE) return NAN; /* no closed form */
    if (u->g[i].op == G_H) l += 0.5;
    if (u->g[i].op == G_U && u->kind[i] == K_COUPLED) l += log2(u->a[i] + u->b[i]);
  }
  return l;
}

int orc_u_log2z(int n, int d, const orc_gate* g, int ng, const double* mats, double* log2z) {
  unet u;
  if (unet_init(&u, n, d, g, ng, mats) != 0) return -1;
  *log2z = log2_scale(&u);
  unet_free(&u);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* J-penalty violations of layer L (s_L = x -> s_{L+1} = y): per output bit of
 * a deterministic gate that differs from the gate's map of its inputs. */
static int layer_viol(const unet* u, int L, uint32_t x, uint32_t y) {
  int v = 0;
  for (int q = 0; q < u->n; ++q) {
    const int gi = u->gate_of[L * u->n + q];
    if (gi < 0) { v += bitof(x, q) != bitof(y, q); continue; }
    const orc_gate* G = &u->g[gi];
    switch (G->op) {
      case G_H: break;
      case G_S: case G_T: v += bitof(x, q) != bitof(y, q); break;
      case G_CZ: v += bitof(x, q) != bitof(y, q); break;
      case G_CNOT:
        if (q == G->q0) v += bitof(x, q) != bitof(y, q);
        else v += bitof(y, q) != (bitof(x, q) ^ bitof(x, G->q0));
        break;
      case G_U:
        if (u->kind[gi] == K_DIAG) v += bitof(x, q) != bitof(y, q);
        else if (u->kind[gi] == K_ANTI) v += bitof(x, q) == bitof(y, q);
        break;
      case G_X: v += bitof(x, q) == bitof(y, q); break;
      case G_CCX:
        if (q == G->q2) v += bitof(y, q) != (bitof(x, q) ^ (bitof(x, G->q0) & bitof(x, G->q1)));
        else v += bitof(x, q) != bitof(y, q);
        break;
      case G_U2: {
        if (u->kind[gi] == K_TABLE) break; /* free outputs (the table's energy) */
        const int o = (q == G->q0) ? 0 : 1;
        v += ((u->perm[gi][gidx(G, x)] >> o) & 1) != bitof(y, q);
        break;
      }
    }
  }
  return v;
}

/* Does the path take a zero entry of a table gate? */
static int table_zero(const unet* u, const uint32_t* s) {
  for (int i = 0; i < u->ng; ++i) {
    const orc_gate* G = &u->g[i];
    if (G->op != G_U2 || u->kind[i] != K_TABLE) continue;
    double r, im;
    u2_entry(u->mats + (size_t)MAT * i, gidx(G, s[G->layer + 1]), gidx(G, s[G->layer]), &r, &im);
    if (r == 0.0 && im == 0.0) return 1;
  }
  return 0;
}

/* Energy of a table gate's entry: -ln |U(y, x)|, J for a zero entry. */
static double table_energy(const unet* u, int gi, int y, int x, double J) {
  double r, im;
  u2_entry(u->mats + (size_t)MAT * gi, y, x, &r, &im);
  const double m = hypot(r, im);
  return m > 0.0 ? -log(m) : J;
}

static int path_viol(const unet* u, const uint32_t* s) {
  int v = 0;
  for (int L = 0; L < u->d; ++L) v += layer_viol(u, L, s[L], s[L + 1]);
  return v;
}

/* e^{i arg U_C} of a nonzero path, or 0 if U_C = 0. */
static int path_phase_c(const unet* u, const uint32_t* s, double* pr, double* pi) {
  double wr = 1.0, wi = 0.0;
  for (int L = 0; L < u->d; ++L) {
    double er, ei;
    layer_elem(u, L, s[L], s[L + 1], &er, &ei);
    const double tr = wr * er - wi * ei, ti = wr * ei + wi * er;
    wr = tr;
    wi = ti;
  }
  const double m = hypot(wr, wi);
  if (m == 0.0) return 0;
  *pr = wr / m;
  *pi = wi / m;
  return 1;
}

/* The deterministic value of output bit q of layer L given s_L = x, for a
 * non-free gate (identity wire, S, T, CZ, CNOT, diagonal / anti-diagonal U). */
static int det_bit(const unet* u, int L, int q, uint32_t x) {
  const int gi = u->gate_of[L * u->n + q];
  if (gi < 0) return bitof(x, q);
  const orc_gate* G = &u->g[gi];
  if (G->op == G_CNOT && q == G->q1) return bitof(x, q) ^ bitof(x, G->q0);
  if (G->op == G_U && u->kind[gi] == K_ANTI) return bitof(x, q) ^ 1;
  if (G->op == G_X) return bitof(x, q) ^ 1;
  if (G->op == G_CCX && q == G->q2) return bitof(x, q) ^ (bitof(x, G->q0) & bitof(x, G->q1));
  if (G->op == G_U2) return (u->perm[gi][gidx(G, x)] >> ((q == G->q0) ? 0 : 1)) & 1;
  return bitof(x, q);
}

/* Is output bit q of layer L free (H, or a coupled U)? */
static int is_free(const unet* u, int L, int q) {
  const int gi = u->gate_of[L * u->n + q];
  if (gi < 0) return 0;
  return u->g[gi].op == G_H || (u->g[gi].op == G_U && u->kind[gi] == K_COUPLED) ||
         (u->g[gi].op == G_U2 && u->kind[gi] == K_TABLE);
}

/* Colour classes of one sweep: the rule of oracle.c's pbit_colours (DSATUR,
 * Brelaz 1979: the uncoloured p-bit with the most distinct neighbour colours,
 * then the most neighbours, then the lowest p, takes the smallest colour its
 * neighbours lack; more than four colours fall back to the fixed classes
 * 2 [k even] + [the p-bit is the second input of a two-input output bit in
 * layer k]) on the factor graph of these gates: the output bit (L+1, q) of
 * every non-H gate or identity wire is one factor with the input bits it
 * depends on -- (L, q) for an identity wire, S, T, CZ, X and any U (a
 * coupled U's energy joins the same two bits), (L, q) and (L, c) for a CNOT
 * target, the inputs in the affine map of a U2 output.  Layer 0 is clamped.
 * Returns the number of classes. */
static int u_colours(const unet* u, int32_t* colour) {
  const int n = u->n, d = u->d, N = n * d;
  enum { MAXN = 16 };
  int* nb = (int*)malloc(sizeof(int) * (size_t)N * MAXN);
  int* deg = (int*)calloc((size_t)N, sizeof(int));
  uint32_t* seen = (uint32_t*)calloc((size_t)N, sizeof(uint32_t));
  if (!nb || !deg || !seen) { free(nb); free(deg); free(seen); return -1; }
  int over = 0;
  for (int L = 0; L < d; ++L)
    for (int q = 0; q < n; ++q) {
      int vars[5], nv = 0, ins[3], ni = 0;
      vars[nv++] = L * n + q; /* p-bit (L+1, q) */
      const int gi = u->gate_of[L * n + q];
      if (gi < 0) {
        ins[ni++] = q;
      } else {
        const orc_gate* G = &u->g[gi];
        if (G->op == G_H) continue;
        if (G->op == G_CNOT) {
          ins[ni++] = q;
          if (q == G->q1) ins[ni++] = G->q0;
        } else if (G->op == G_U2 && u->kind[gi] == K_TABLE) {
          /* the table's factor: both outputs and both inputs */
          vars[nv++] = L * n + (q == G->q0 ? G->q1 : G->q0);
          ins[ni++] = G->q0;
          ins[ni++] = G->q1;
        } else if (G->op == G_U2) {
          const int dm = u->dmask[gi][(q == G->q0) ? 0 : 1];
          if (dm & 1) ins[ni++] = G->q0;
          if (dm & 2) ins[ni++] = G->q1;
        } else if (G->op == G_CCX && q == G->q2) { /* target: t' = t ^ c0 c1 */
          ins[ni++] = q;
          ins[ni++] = G->q0;
          ins[ni++] = G->q1;
        } else {
          ins[ni++] = q;
        }
      }
      if (L >= 1)
        for (int t = 0; t < ni; ++t) vars[nv++] = (L - 1) * n + ins[t];
      for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) {
          if (a == b) continue;
          const int x = vars[a], y = vars[b];
          int dup = 0;
          for (int e = 0; e < deg[x]; ++e) dup |= nb[x * MAXN + e] == y;
          if (dup) continue;
          if (deg[x] == MAXN) { over = 1; continue; }
          nb[x * MAXN + deg[x]++] = y;
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
    /* the fixed classes separate at most two inputs of one factor: a
     * Toffoli's four-bit factor needs the computed colouring */
    for (int i = 0; i < u->ng; ++i)
      if (u->g[i].op == G_CCX || (u->g[i].op == G_U2 && u->kind[i] == K_TABLE)) {
        free(nb); free(deg); free(seen);
        return -2;
      }
    ncol = 4;
    for (int k = 1; k <= d; ++k)
      for (int q = 0; q < n; ++q) {
        int second = 0;
        if (k < d) {
          const int gi = u->gate_of[k * n + q];
          if (gi >= 0) {
            const orc_gate* G = &u->g[gi];
            if (G->op == G_CNOT && G->q1 == q) second = 1;
            if (G->op == G_U2 && G->q1 == q && (u->dmask[gi][0] == 3 || u->dmask[gi][1] == 3))
              second = 1;
            if (G->op == G_CCX && G->q2 == q) second = 1;
          }
        }
        colour[(k - 1) * n + q] = 2 * ((k % 2) == 0) + second;
      }
  }
  free(nb); free(deg); free(seen);
  return ncol;
}

/* The 32-bit uniform of chain c: bit (c mod 32) of successive Philox output
 * words, most significant first (counter (c >> 5, t, p | tag << 16, j / 4),
 * word j mod 4). */
static uint32_t uniform32(uint64_t seed, uint32_t chain, uint32_t t, uint32_t p, uint32_t tag) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t u = 0;
  for (uint32_t grp = 0; grp < 8; ++grp) {
    uint32_t ctr[4] = {chain >> 5, t, p | (tag << 16), grp}, out[4];
    orc_philox4x32_10(ctr, key, out);
    for (int w = 0; w < 4; ++w) u |= ((out[w] >> (chain & 31)) & 1u) << (31 - (grp * 4 + (uint32_t)w));
  }
  return u;
}

/* The 32-bit uniform of chain c as one Philox word: word (c mod 4) of
 * Philox(c >> 5, t, p | tag << 16, (c mod 32) / 4). */
static uint32_t lane_uniform(uint64_t seed, uint32_t chain, uint32_t t, uint32_t p, uint32_t tag) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {chain >> 5, t, p | (tag << 16), (chain & 31u) >> 2}, out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[chain & 3u];
}

/* Change of the table energy when p-bit (k, q) goes 0 -> 1 (path s, layers
 * 0..d): the gate of layer k-1 on q if it is a table (the bit is one of its
 * outputs), plus the gate of layer k if it is a table (one of its inputs). */
static double table_delta(const unet* u, const uint32_t* s, int k, int q, double J) {
  const int n = u->n, d = u->d;
  double din = 0.0, dout = 0.0;
  const int gin = u->gate_of[(k - 1) * n + q];
  if (gin >= 0 && u->g[gin].op == G_U2 && u->kind[gin] == K_TABLE) {
    const orc_gate* G = &u->g[gin];
    const int o = (q == G->q0) ? 0 : 1;
    const int xi = gidx(G, s[k - 1]);
    const int yo = bitof(s[k], o == 0 ? G->q1 : G->q0);  /* the other output */
    const int y1 = o == 0 ? 1 + 2 * yo : yo + 2, y0 = o == 0 ? 2 * yo : yo;
    din = table_energy(u, gin, y1, xi, J) - table_energy(u, gin, y0, xi, J);
  }
  if (k < d) {
    const int gout = u->gate_of[k * n + q];
    if (gout >= 0 && u->g[gout].op == G_U2 && u->kind[gout] == K_TABLE) {
      const orc_gate* G = &u->g[gout];
      const int iu = (q == G->q0) ? 0 : 1;
      const int yi = gidx(G, s[k + 1]);
      const int xo = bitof(s[k], iu == 0 ? G->q1 : G->q0);  /* the other input */
      const int x1 = iu == 0 ? 1 + 2 * xo : xo + 2, x0 = iu == 0 ? 2 * xo : xo;
      dout = table_energy(u, gout, yi, x1, J) - table_energy(u, gout, yi, x0, J);
    }
  }
  return din + dout;
}

/* Bit (c mod 32) of word 0 of Philox(c >> 5, t, p | tag << 16, 0). */
static int coin(uint64_t seed, uint32_t chain, uint32_t t, uint32_t p, uint32_t tag) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {chain >> 5, t, p | (tag << 16), 0}, out[4];
  orc_philox4x32_10(ctr, key, out);
  return (int)((out[0] >> (chain & 31)) & 1u);
}

/* floor(2^32 x) for 0 <= x, capped at 2^32 - 1. */
static uint32_t to_u32_threshold(double x) {
  const double t = floor(x * 4294967296.0);
  return t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
}

static void add_sample(const unet* u, const uint32_t* s, const uint32_t* alphas, int n_alphas,
                       double* sre, double* sim, uint64_t* cnt, uint64_t* my_valid, int* err) {
  if (path_viol(u, s) != 0 || table_zero(u, s)) return;
  double pr, pi;
  if (!path_phase_c(u, s, &pr, &pi)) { *err = 1; return; }
  ++*my_valid;
  const uint32_t al = s[u->d];
  int bin = -1;
  if (alphas) {
    for (int a = 0; a < n_alphas; ++a)
      if (alphas[a] == al) { bin = a; break; }
  } else {
    bin = (int)al;
  }
  if (bin < 0) return;
  sre[bin] += pr;
  sim[bin] += pi;
  cnt[bin] += 1;
}

/* Reference Gibbs sampler, general one-qubit gates (Fig. 2 Steps 1-3).
 *
 * Arguments as orc_gibbs (oracle.c); outputs per bin: sre + i sim = sum over
 * valid recorded samples ending there of e^{i arg U_C}, cnt = their number.
 * The estimator is psi_alpha = 2^{log2z} (sre + i sim) / valid_total.
 *
 * Sweep: the colour classes of u_colours.  Update of p-bit x = (k, q),
 * p = (k-1) n + q:
 *   Step 1 (proposal, heat-bath on the J-penalty energy): v = change of the
 *     violation count when x goes 0 -> 1, u = uniform32(tag 0),
 *     x' = [v < 0] XOR [u < thr[|v|]].
 *   Step 2 (acceptance, Metropolis on the coupling energy): if x' != x,
 *     e_in = x XOR s_{k-1,q} when the gate of layer k-1 on q is coupled
 *     (K_in its K; else e_in = 0, K_in = 0), e_out = x XOR s_{k+1,q} when
 *     k < d and the gate of layer k on q is coupled (K_out; else 0, 0);
 *     dK = K_in (1 - 2 e_in) + K_out (1 - 2 e_out) is the change of
 *     sum K [s_out != s_in] caused by the flip.  Accept when dK <= 0, else
 *     when u' < floor(2^32 e^{-dK}) (capped at 2^32 - 1), u' = uniform32(tag 6).
 *   Step 2b (table gates, Eq. ET2): a flip that passed is kept when the
 *     change dE of the tables' energy (-ln|U| of the entries taken, J for a
 *     zero entry; table_delta, sign by direction) is <= 0, else when
 *     u'' < floor(2^32 e^{-dE}), u'' = lane_uniform(tag 7).
 *   The pair is Metropolis-Hastings with the J-part heat-bath as proposal:
 *   the chain keeps p proportional to e^{-J viol} e^{-sum K [s_out != s_in]}.
 * Initial paths: free outputs (H, coupled U) from the tag-1 coin, the others
 * deterministic.  A recorded sample with no violation adds its phase. */
int orc_u_gibbs(int n, int d, const orc_gate* g, int ng, const double* mats, uint32_t beta,
                double J, uint64_t seed, uint32_t chain0, uint32_t chains, uint32_t sweep0,
                uint32_t sweeps, uint32_t burn_in, uint32_t record_every, int init,
                uint32_t* state, const uint32_t* alphas, int n_alphas, double* sre, double* sim,
                uint64_t* cnt, uint64_t* valid_total, uint64_t* samples_total, double* log2z) {
  unet u;
  if (record_every == 0) return -1;
  if (!alphas && n > 22) return -2;
  if (unet_init(&u, n, d, g, ng, mats) != 0) return -1;
  uint32_t thr[4];
  if (orc_thresholds(J, thr) != 0) { unet_free(&u); return -1; }
  if (log2z) *log2z = log2_scale(&u);
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * d);
  if (!col) { unet_free(&u); return -3; }
  const int ncol = u_colours(&u, col);
  if (ncol <= 0) { free(col); unet_free(&u); return -3; }
  const uint32_t nmask = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const uint64_t bins = alphas ? (uint64_t)n_alphas : (1ull << n);
  int err = 0;

#pragma omp parallel reduction(| : err)
  {
    double* my_re = (double*)calloc(bins, sizeof(double));
    double* my_im = (double*)calloc(bins, sizeof(double));
    uint64_t* my_cnt = (uint64_t*)calloc(bins, sizeof(uint64_t));
    uint64_t my_valid = 0, my_samples = 0;
    uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
    if (!my_re || !my_im || !my_cnt || !s) err = 1;
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
            const uint32_t p = (uint32_t)((k - 1) * n + q);
            const int b = is_free(&u, k - 1, q) ? coin(seed, chain, 0, p, 1) : det_bit(&u, k - 1, q, s[k - 1]);
            w |= (uint32_t)b << q;
          }
          s[k] = w;
        }
      } else {
        for (int k = 1; k <= d; ++k) s[k] = st[k - 1] & nmask;
      }
      for (uint32_t t = 0; t < sweeps && !err; ++t) {
        const uint32_t sweep = sweep0 + t;
        for (int colour = 0; colour < ncol; ++colour)
          for (int k = 1; k <= d; ++k)
            for (int q = 0; q < n; ++q) {
              if (col[(k - 1) * n + q] != colour) continue;
              const uint32_t p = (uint32_t)((k - 1) * n + q);
              const uint32_t keep = s[k];
              const int x = bitof(keep, q);
              /* Step 1: proposal from the J-penalty energy */
              s[k] = keep | (1u << q);
              const int v1 = layer_viol(&u, k - 1, s[k - 1], s[k]) +
                             (k < d ? layer_viol(&u, k, s[k], s[k + 1]) : 0);
              s[k] = keep & ~(1u << q);
              const int v0 = layer_viol(&u, k - 1, s[k - 1], s[k]) +
                             (k < d ? layer_viol(&u, k, s[k], s[k + 1]) : 0);
              const int v = v1 - v0, av = v < 0 ? -v : v;
              const uint32_t uu = uniform32(seed, chain, sweep, p, 0);
              int xn = (v < 0) ^ (uu < thr[av]);
              /* Step 2: Metropolis acceptance on the coupling energy */
              if (xn != x) {
                double kin = 0.0, kout = 0.0;
                int ein = 0, eout = 0;
                const int gin = u.gate_of[(k - 1) * n + q];
                if (gin >= 0 && u.g[gin].op == G_U && u.kind[gin] == K_COUPLED) {
                  kin = u.K[gin];
                  ein = x ^ bitof(s[k - 1], q);
                }
                if (k < d) {
                  const int gout = u.gate_of[k * n + q];
                  if (gout >= 0 && u.g[gout].op == G_U && u.kind[gout] == K_COUPLED) {
                    kout = u.K[gout];
                    eout = x ^ bitof(s[k + 1], q);
                  }
                }
                const double dk = kin * (double)(1 - 2 * ein) + kout * (double)(1 - 2 * eout);
                if (dk > 0.0) {
                  const uint32_t A = to_u32_threshold(exp(-dk));
                  if (!(uniform32(seed, chain, sweep, p, 6) < A)) xn = x;
                }
                /* Step 2b: Metropolis acceptance on the table energy (a second
                 * factor of the acceptance: min(1, e^{-dK}) min(1, e^{-dE})) */
                if (xn != x) {
                  const double de = table_delta(&u, s, k, q, J);
                  const double dt = x == 0 ? de : -de;
                  if (dt > 0.0) {
                    const uint32_t A = to_u32_threshold(exp(-dt));
                    if (!(lane_uniform(seed, chain, sweep, p, 7) < A)) xn = x;
                  }
                }
              }
              s[k] = (keep & ~(1u << q)) | ((uint32_t)xn << q);
            }
        if (sweep >= burn_in && (sweep - burn_in) % record_every == 0) {
          ++my_samples;
          add_sample(&u, s, alphas, n_alphas, my_re, my_im, my_cnt, &my_valid, &err);
        }
      }
      for (int k = 1; k <= d; ++k) st[k - 1] = s[k];
    }
#pragma omp critical
    {
      if (my_re && my_im && my_cnt)
        for (uint64_t i = 0; i < bins; ++i) { sre[i] += my_re[i]; sim[i] += my_im[i]; cnt[i] += my_cnt[i]; }
      *valid_total += my_valid;
      *samples_total += my_samples;
    }
    free(my_re); free(my_im); free(my_cnt); free(s);
  }
  free(col);
  unet_free(&u);
  return err ? -4 : 0;
}

/* Exact i.i.d. sampler on the eliminated network (Appendix), general gates.
 * Sample t of chain c is drawn layer by layer from the clamped input: an H
 * output is the coin bit of tag 4 (as orc_elim); a coupled output is
 * s_in XOR [u < floor(2^32 b / (a + b))] with u = uniform32(tag 4), so that
 * P(s_out != s_in) = b / (a + b) and the path has probability
 * |U_C| / (2^{h/2} prod (a + b)); every other bit is deterministic.
 * Outputs as orc_u_gibbs (every drawn path is valid). */
int orc_u_elim(int n, int d, const orc_gate* g, int ng, const double* mats, uint32_t beta,
               uint64_t seed, uint32_t chain0, uint32_t chains, uint32_t sweep0, uint32_t sweeps,
               uint32_t burn_in, uint32_t record_every, uint32_t* state, const uint32_t* alphas,
               int n_alphas, double* sre, double* sim, uint64_t* cnt, uint64_t* valid_total,
               uint64_t* samples_total, double* log2z) {
  unet u;
  if (record_every == 0) return -1;
  if (!alphas && n > 22) return -2;
  if (unet_init(&u, n, d, g, ng, mats) != 0) return -1;
  for (int i = 0; i < ng; ++i)
    if (g[i].op == G_U2 && u.kind[i] == K_TABLE) { unet_free(&u); return -1; } /* Gibbs only */
  if (log2z) *log2z = log2_scale(&u);
  const uint32_t nmask = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const uint64_t bins = alphas ? (uint64_t)n_alphas : (1ull << n);
  int err = 0;
#pragma omp parallel reduction(| : err)
  {
    double* my_re = (double*)calloc(bins, sizeof(double));
    double* my_im = (double*)calloc(bins, sizeof(double));
    uint64_t* my_cnt = (uint64_t*)calloc(bins, sizeof(uint64_t));
    uint64_t my_valid = 0, my_samples = 0;
    uint32_t* s = (uint32_t*)calloc((size_t)d + 1, sizeof(uint32_t));
    if (!my_re || !my_im || !my_cnt || !s) err = 1;
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
            const uint32_t p = (uint32_t)((k - 1) * n + q);
            const int gi = u.gate_of[(k - 1) * n + q];
            int b;
            if (gi >= 0 && u.g[gi].op == G_H) {
              b = coin(seed, chain, t, p, 4);
            } else if (gi >= 0 && u.g[gi].op == G_U && u.kind[gi] == K_COUPLED) {
              const uint32_t B = to_u32_threshold(u.b[gi] / (u.a[gi] + u.b[gi]));
              b = bitof(s[k - 1], q) ^ (uniform32(seed, chain, t, p, 4) < B);
            } else {
              b = det_bit(&u, k - 1, q, s[k - 1]);
            }
            w |= (uint32_t)b << q;
          }
          s[k] = w;
        }
        drawn = 1;
        ++my_samples;
        const uint64_t before = my_valid;
        add_sample(&u, s, alphas, n_alphas, my_re, my_im, my_cnt, &my_valid, &err);
        if (my_valid == before) err = 1; /* every drawn path is valid */
      }
      if (state && drawn)
        for (int k = 1; k <= d; ++k) state[(size_t)ci * d + k - 1] = s[k];
    }
#pragma omp critical
    {
      if (my_re && my_im && my_cnt)
        for (uint64_t i = 0; i < bins; ++i) { sre[i] += my_re[i]; sim[i] += my_im[i]; cnt[i] += my_cnt[i]; }
      *valid_total += my_valid;
      *samples_total += my_samples;
    }
    free(my_re); free(my_im); free(my_cnt); free(s);
  }
  unet_free(&u);
  return err ? -4 : 0;
}

/* Colour classes (u_colours) of a general circuit, [d][n]; the number of
 * classes, or <= 0 on error. */
int orc_u_colour(int n, int d, const orc_gate* g, int ng, const double* mats, int32_t* colour) {
  unet u;
  if (unet_init(&u, n, d, g, ng, mats) != 0) return -1;
  const int ncol = u_colours(&u, colour);
  unet_free(&u);
  return ncol;
}
