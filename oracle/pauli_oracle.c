/*
 * pauli_oracle.c -- CPU oracle for the dense Pauli decomposition.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the checker, not the product: only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it. It shares
 * no code, header, table or helper with the CUDA library, and it is deliberately slow.
 *
 * Source: T. Jones, "Decomposing dense matrices into dense Pauli tensors" (arXiv 2401.16378).
 *
 * Conventions fixed by the paper (Sec. 2, first paragraph): matrix elements [M]_{ij} with
 * row i and column j counted from zero; bit t of an integer is its t-th bit counted from the
 * rightmost, and the t-th operator of a Pauli tensor is the rightmost factor for t = 0.
 *
 * The Pauli flag of operator t in the tensor with index n is the t-th pair of bits of n
 * (Sec. 2, last paragraph), with flags 0, 1, 2, 3 naming I, X, Y, Z in the order of Eq. (2)
 * (c_1 multiplies 1 (x) X, c_2 multiplies 1 (x) Y, c_3 multiplies 1 (x) Z, c_4 multiplies X (x) 1).
 *
 * decompose  c_n = 2^-N sum_{i < 2^N} lambda_i^(n) [G]_{i xor m^(n), i}            Eq. (13)
 *            lambda_i^(n) = prod_t [sigma_t^(n)]_{i_[t], i_[t] xor m^(n)_[t]}       Eq. (12)
 *            m^(n)_[t] = 1 exactly when sigma_t^(n) is X or Y                    Eq. (11)
 *            lambda is rebuilt in full for every i (no recurrence), and the sum is a
 *            Neumaier-compensated FP64 sum of the real and the imaginary parts.
 *
 * compose    [G]_{rc} = sum_n c_n [P_n]_{rc}                                      Eq. (1)
 *            [P_n]_{rc} = prod_t [sigma_t^(n)]_{r_[t], c_[t]}                      Eq. (7)
 *            summed over every n < 4^N; a product stops at its first zero factor
 *            (the remaining factors cannot make it nonzero).
 *
 * Complex numbers are interleaved (re, im) doubles. Matrices are row-major, element (r, c)
 * at index r * 2^N + c.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The Pauli matrices of Eq. (3), as [flag][row][col] = (re, im). */
static const double PAULI[4][2][2][2] = {
    /* I */ {{{1.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {1.0, 0.0}}},
    /* X */ {{{0.0, 0.0}, {1.0, 0.0}}, {{1.0, 0.0}, {0.0, 0.0}}},
    /* Y */ {{{0.0, 0.0}, {0.0, -1.0}}, {{0.0, 1.0}, {0.0, 0.0}}},
    /* Z */ {{{1.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {-1.0, 0.0}}},
};

/* Bit t of the integer v (Sec. 2). */
static unsigned bit_of(uint64_t v, int t) { return (unsigned)((v >> t) & 1u); }

/* Flag of operator t of tensor n: bits 2t and 2t+1 of n read as a base-4 digit. */
static unsigned pauli_flag(uint64_t n, int t) { return (bit_of(n, 2 * t + 1) << 1) | bit_of(n, 2 * t); }

/* m^(n): bit t set when operator t is X (flag 1) or Y (flag 2), Eq. (11). */
static uint64_t xy_mask(uint64_t n, int N) {
  uint64_t m = 0;
  for (int t = 0; t < N; ++t) {
    unsigned p = pauli_flag(n, t);
    if (p == 1u || p == 2u) m |= (uint64_t)1 << t;
  }
  return m;
}

/* Neumaier's compensated summation. */
typedef struct {
  double sum, comp;
} nsum_t;

static void nsum_add(nsum_t* a, double x) {
  double t = a->sum + x;
  if (fabs(a->sum) >= fabs(x))
    a->comp += (a->sum - t) + x;
  else
    a->comp += (x - t) + a->sum;
  a->sum = t;
}

static double nsum_value(const nsum_t* a) { return a->sum + a->comp; }

/* lambda_i^(n), Eq. (12): the product over t of the entry of operator t at row i_[t] and
 * column i_[t] xor m_[t]. Every factor is one of +-1, +-i, so the product is exact. */
static void lambda_of(uint64_t n, uint64_t i, uint64_t m, int N, double* re, double* im) {
  double lr = 1.0, li = 0.0;
  for (int t = 0; t < N; ++t) {
    unsigned p = pauli_flag(n, t);
    unsigned a = bit_of(i, t);
    unsigned b = a ^ bit_of(m, t);
    double er = PAULI[p][a][b][0], ei = PAULI[p][a][b][1];
    double nr = lr * er - li * ei;
    double ni = lr * ei + li * er;
    lr = nr;
    li = ni;
  }
  *re = lr;
  *im = li;
}

/* One coefficient c_n by Eq. (13). */
static void coeff_literal(const double* G, int N, uint64_t n, double* out) {
  const uint64_t D = (uint64_t)1 << N;
  const uint64_t m = xy_mask(n, N);
  nsum_t sr = {0.0, 0.0}, si = {0.0, 0.0};
  for (uint64_t i = 0; i < D; ++i) {
    double lr, li;
    lambda_of(n, i, m, N, &lr, &li);
    const double* g = G + 2 * ((i ^ m) * D + i); /* [G]_{i xor m, i} */
    nsum_add(&sr, lr * g[0] - li * g[1]);
    nsum_add(&si, lr * g[1] + li * g[0]);
  }
  const double scale = ldexp(1.0, -N); /* 1 / 2^N, exact */
  out[0] = nsum_value(&sr) * scale;
  out[1] = nsum_value(&si) * scale;
}

/* One matrix element [G]_{rc} by Eqs. (1) and (7). */
static void element_literal(const double* c, int N, uint64_t r, uint64_t col, double* out) {
  const uint64_t nterms = (uint64_t)1 << (2 * N);
  nsum_t sr = {0.0, 0.0}, si = {0.0, 0.0};
  for (uint64_t n = 0; n < nterms; ++n) {
    double pr = 1.0, pi = 0.0;
    int zero = 0;
    for (int t = 0; t < N && !zero; ++t) {
      unsigned p = pauli_flag(n, t);
      double er = PAULI[p][bit_of(r, t)][bit_of(col, t)][0];
      double ei = PAULI[p][bit_of(r, t)][bit_of(col, t)][1];
      double nr = pr * er - pi * ei;
      double ni = pr * ei + pi * er;
      pr = nr;
      pi = ni;
      zero = (pr == 0.0 && pi == 0.0);
    }
    if (zero) continue;
    const double* cn = c + 2 * n;
    nsum_add(&sr, pr * cn[0] - pi * cn[1]);
    nsum_add(&si, pr * cn[1] + pi * cn[0]);
  }
  out[0] = nsum_value(&sr);
  out[1] = nsum_value(&si);
}

static int pick_threads(int threads) {
#ifdef _OPENMP
  return threads > 0 ? threads : omp_get_max_threads();
#else
  (void)threads;
  return 1;
#endif
}

/* Number of threads a call with threads <= 0 uses. */
int oracle_default_threads(void) { return pick_threads(0); }

/* c_n for each n in idx[0..k). G: 2^N x 2^N complex (interleaved doubles). out: k complex.
 * Returns 0, or -1 for an argument error. */
int oracle_decompose_at(const double* G, int N, const uint64_t* idx, int64_t k, double* out, int threads) {
  if (!G || !out || (k > 0 && !idx) || N < 1 || N > 20 || k < 0) return -1;
  const uint64_t nmax = (uint64_t)1 << (2 * N);
  for (int64_t q = 0; q < k; ++q)
    if (idx[q] >= nmax) return -1;
  const int nt = pick_threads(threads);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int64_t q = 0; q < k; ++q) coeff_literal(G, N, idx[q], out + 2 * q);
  return 0;
}

/* [G]_{rows[q], cols[q]} for q < k from the 4^N coefficients c (paper order). */
int oracle_compose_at(const double* c, int N, const uint64_t* rows, const uint64_t* cols, int64_t k, double* out,
                      int threads) {
  if (!c || !out || (k > 0 && (!rows || !cols)) || N < 1 || N > 12 || k < 0) return -1;
  const uint64_t D = (uint64_t)1 << N;
  for (int64_t q = 0; q < k; ++q)
    if (rows[q] >= D || cols[q] >= D) return -1;
  const int nt = pick_threads(threads);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int64_t q = 0; q < k; ++q) element_literal(c, N, rows[q], cols[q], out + 2 * q);
  return 0;
}
