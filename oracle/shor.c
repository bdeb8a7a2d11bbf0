/*
 * CPU oracle, part 3: column sampling of the period-finding circuit
 * (arXiv 2007.07379, Sec. 5.2 and the column-sampling figure).
 *
 * TEST INFRASTRUCTURE ONLY, under the same rules as oracle.c.  Plain scalar
 * code in exact integer arithmetic and FP64.
 *
 * The circuit: t = n input bits x (here t = n = ceil(log2 N), Sec. 5.2),
 * f(x) = a^x mod N on the second register, then the inverse QFT of the first
 * register.  Column sampling: sample i draws a column x_i; the IQFT column
 * U_IQFT[k, x_i] = 2^{-n/2} e^{2 pi i k x_i / 2^n} (k = 0 .. 2^n - 1) is added
 * to column y_i = a^{x_i} mod N of psi (a 2^n x N-column table), and the
 * output distribution is P[k] = sum_y |psi[k, y]|^2.  With T samples the
 * functions below return prob[k] = P[k] / T, which sums to 1 when the drawn
 * columns are distinct (Parseval over k); drawing every column once gives
 * the exact distribution of the first register.
 *
 *   orc_modexp        a^x mod N by binary exponentiation (128-bit products).
 *   orc_shor_columns  prob[k] for a given list of drawn columns, by the
 *                     definition: the samples grouped by y, per k the sum
 *                     over groups of |sum of the group's IQFT entries|^2.
 *   orc_shor_prob_at  the same for a list of k values only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

uint64_t orc_modexp(uint64_t a, uint64_t x, uint64_t N) {
  if (N == 1) return 0;
  unsigned __int128 result = 1, base = a % N;
  while (x) {
    if (x & 1u) result = (result * base) % N;
    base = (base * base) % N;
    x >>= 1;
  }
  return (uint64_t)result;
}

typedef struct {
  uint64_t y;
  uint32_t x;
} col_sample;

static int by_y_then_x(const void* p, const void* q) {
  const col_sample* a = (const col_sample*)p;
  const col_sample* b = (const col_sample*)q;
  if (a->y != b->y) return a->y < b->y ? -1 : 1;
  if (a->x != b->x) return a->x < b->x ? -1 : 1;
  return 0;
}

/* Groups the samples by y: sorted copy, returns it (caller frees). */
static col_sample* group_samples(uint64_t N, uint64_t a, const uint32_t* x, uint32_t T,
                                 uint64_t* y_out) {
  col_sample* s = (col_sample*)malloc(sizeof(col_sample) * (T ? T : 1));
  if (!s) return NULL;
  for (uint32_t i = 0; i < T; ++i) {
    s[i].x = x[i];
    s[i].y = orc_modexp(a, x[i], N);
    if (y_out) y_out[i] = s[i].y;
  }
  qsort(s, T, sizeof(col_sample), by_y_then_x);
  return s;
}

/* P[k] / T at one k: sum over groups of |sum_{i in group} e^{2 pi i k x_i / 2^n}|^2 / (2^n T),
 * the phase k x_i mod 2^n taken exactly in integers. */
static double prob_one(const col_sample* s, uint32_t T, int n, uint64_t k) {
  const uint64_t mask = (n == 64) ? ~0ull : ((1ull << n) - 1ull);
  const double two_n = ldexp(1.0, n);
  double total = 0.0;
  uint32_t i = 0;
  while (i < T) {
    double re = 0.0, im = 0.0;
    const uint64_t y = s[i].y;
    for (; i < T && s[i].y == y; ++i) {
      const uint64_t ph = (k * (uint64_t)s[i].x) & mask;
      const double ang = 2.0 * M_PI * ((double)ph / two_n);
      re += cos(ang);
      im += sin(ang);
    }
    total += re * re + im * im;
  }
  return total / (two_n * (double)T);
}

/* prob[k], k = 0 .. 2^n - 1 (n <= 24 here); y_out (optional) receives y_i. */
int orc_shor_columns(uint64_t N, uint64_t a, int n, const uint32_t* x, uint32_t T,
                     double* prob, uint64_t* y_out) {
  if (n < 1 || n > 24 || N < 2 || T == 0) return -1;
  for (uint32_t i = 0; i < T; ++i)
    if ((uint64_t)x[i] >> n) return -1;
  col_sample* s = group_samples(N, a, x, T, y_out);
  if (!s) return -3;
  const int64_t K = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < K; ++k) prob[k] = prob_one(s, T, n, (uint64_t)k);
  free(s);
  return 0;
}

/* prob at the listed k values only (any n <= 32). */
int orc_shor_prob_at(uint64_t N, uint64_t a, int n, const uint32_t* x, uint32_t T,
                     const uint64_t* ks, uint32_t nk, double* prob) {
  if (n < 1 || n > 32 || N < 2 || T == 0) return -1;
  for (uint32_t i = 0; i < T; ++i)
    if ((uint64_t)x[i] >> n) return -1;
  col_sample* s = group_samples(N, a, x, T, NULL);
  if (!s) return -3;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < (int64_t)nk; ++j) prob[j] = prob_one(s, T, n, ks[j]);
  free(s);
  return 0;
}
