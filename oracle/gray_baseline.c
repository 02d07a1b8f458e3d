/*
 * gray_baseline.c -- the paper's own CPU algorithm, as a faster CPU baseline.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE, not the checker and not the product: the benchmark times
 * it beside the oracle as a second CPU baseline, and the tests hold it to the oracle. It
 * shares no code with the CUDA library or with pauli_oracle.c.
 *
 * Source: T. Jones, "Decomposing dense matrices into dense Pauli tensors" (arXiv 2401.16378),
 * Sec. 3 (Algorithm): evaluate Eq. (13) for each coefficient, visiting the sum index i in
 * Gray-code order so that consecutive i differ in one bit t, and update lambda_i by the
 * recurrence of Eq. (14): only the factor of operator t changes.
 *
 * Every factor [sigma_t]_{a, a xor m_t} of Eq. (12) is one of 1, i, -1, -i, i.e. i^q with
 * q in {0, 1, 2, 3}; lambda_i is then i^e with e the sum of the factors' q mod 4, and the
 * recurrence of Eq. (14) is e += q(new factor) - q(old factor). Per flag (I, X, Y, Z) and
 * row bit a the factor is: I: 1, 1; X: 1, 1; Y: -i (row 0, column 1), i (row 1, column 0);
 * Z: 1, -1 (Eq. (3)).
 *
 * Sums are plain FP64 (as the paper's implementation), one coefficient per OpenMP iteration.
 * Conventions as in pauli_oracle.c: flag of operator t = bits (2t, 2t + 1) of n, m bit t set
 * for X and Y, the element [G]_{i xor m, i}, interleaved complex, row-major.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* q of the factor of flag p at row bit a: the factor is i^q */
static const unsigned char FACTOR_Q[4][2] = {{0, 0}, {0, 0}, {3, 1}, {0, 2}};

static void gray_coefficient(const double* G, int N, uint64_t n, double* out) {
  const uint64_t D = (uint64_t)1 << N;
  uint64_t m = 0;
  unsigned flag[32];
  unsigned e = 0; /* lambda_0 = i^e: every operator at row bit 0 */
  for (int t = 0; t < N; ++t) {
    flag[t] = (unsigned)((n >> (2 * t)) & 3u);
    if (flag[t] == 1u || flag[t] == 2u) m |= (uint64_t)1 << t;
    e += FACTOR_Q[flag[t]][0];
  }
  double sr = 0.0, si = 0.0;
  uint64_t i = 0;
  for (uint64_t k = 0;;) {
    const double* g = G + 2 * ((i ^ m) * D + i);
    switch (e & 3u) { /* i^e g */
      case 0: sr += g[0]; si += g[1]; break;
      case 1: sr -= g[1]; si += g[0]; break;
      case 2: sr -= g[0]; si -= g[1]; break;
      default: sr += g[1]; si -= g[0]; break;
    }
    if (++k == D) break;
    /* the next Gray code k ^ (k >> 1) differs from i in bit t = the lowest set bit of k */
    const int t = __builtin_ctzll(k);
    const unsigned a = (unsigned)((i >> t) & 1u);
    e += FACTOR_Q[flag[t]][a ^ 1u] + 4u - FACTOR_Q[flag[t]][a];
    i ^= (uint64_t)1 << t;
  }
  const double scale = ldexp(1.0, -N);
  out[0] = sr * scale;
  out[1] = si * scale;
}

/* c_n for the k indices idx[] (each < 4^N) into out (k interleaved complex). Returns 0, or -1
 * for an N outside [1, 31] or an index out of range. */
int gray_decompose_at(const double* G, int N, const uint64_t* idx, int64_t k, double* out, int threads) {
  if (N < 1 || N > 31 || k < 0) return -1;
  const uint64_t nterms = (uint64_t)1 << (2 * N);
  for (int64_t j = 0; j < k; ++j)
    if (idx[j] >= nterms) return -1;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < k; ++j) gray_coefficient(G, N, idx[j], out + 2 * j);
  return 0;
}

int gray_default_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
