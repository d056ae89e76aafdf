/*
 * nmfa_oracle.c -- plain, slow, FP64 CPU oracle for noisy mean-field annealing
 * (NMFA, Algorithm 1 of King et al., "Emulating the coherent Ising machine with a
 * mean-field algorithm", arXiv 1806.08422).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the CUDA
 * library under paper_1806_08422_gb300/) never calls it, and this file shares no
 * code, header, table or constant generator with it.
 *
 * Everything is IEEE binary64, evaluated in the order written here; the file must
 * be compiled with -ffp-contract=off so that no multiply-add is fused.
 *
 * Pins (see tests/test_oracle_*.py): Philox known-answer vectors, the step-1
 * closed form, recovered-noise statistics, brute-force ground states, closed-form
 * ground energies of K_N / ring / Moebius ladder, gauge and permutation invariance,
 * the sigma=0 symmetries, and the two textbook special cases (deterministic
 * mean-field annealing at sigma=0, alpha=1; zero-temperature sign dynamics).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy */
/* as 1, 2, 3", SC'11).  One round multiplies words 0 and 2 by the two Philox  */
/* multipliers, swaps the halves and mixes in the round key; the Weyl key       */
/* schedule adds the two golden-ratio constants between rounds.                 */
/* ------------------------------------------------------------------------- */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

ORC_EXPORT void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                  uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_WEYL_A;
      k1 += PHILOX_WEYL_B;
    }
    uint64_t pa = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
    uint64_t pb = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
    uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
    uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
    uint32_t y0 = pb_hi ^ x1 ^ k0;
    uint32_t y1 = pb_lo;
    uint32_t y2 = pa_hi ^ x3 ^ k1;
    uint32_t y3 = pa_lo;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* A 32-bit word -> uniform on the odd multiples of 2^-24 in (0,1): the top 23 */
/* bits k give (2k+1) * 2^-24.  Never 0 or 1, and exact in binary32 as well.   */
ORC_EXPORT double orc_uniform(uint32_t x) {
  uint32_t k = x >> 9;
  return ldexp((double)(2u * k + 1u), -24);
}

/* The N(0,1) draw for (replica r, step t, spin i) of noise stream `stream`.
 * Counter = (r/4, t, i, stream), key = (seed low word, seed high word).  The four
 * output words feed two Box-Muller pairs: words (0,1) give replicas 4p (cosine) and
 * 4p+1 (sine); words (2,3) give replicas 4p+2 and 4p+3.  Step t is 0-based
 * (Algorithm 1's t = 1 is t = 0 here). */
ORC_EXPORT double orc_gauss(uint64_t seed, uint32_t stream, int64_t r, int32_t t,
                            int32_t i) {
  uint32_t ctr[4] = {(uint32_t)(r >> 2), (uint32_t)t, (uint32_t)i, stream};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  int k = (int)(r & 3);
  int pair = k >> 1;
  double ua = orc_uniform(w[2 * pair]);
  double ub = orc_uniform(w[2 * pair + 1]);
  double radius = sqrt(-2.0 * log(ua));
  double angle = 2.0 * M_PI * ub;
  return (k & 1) ? radius * sin(angle) : radius * cos(angle);
}

/* ------------------------------------------------------------------------- */
/* Row normalisation of Algorithm 1's field: d_i = sqrt(h_i^2 + sum_j J_ij^2),  */
/* the root mean square of the Hamiltonian terms acting on spin i (Sec. II).    */
/* Sum over j ascending, then add h_i^2.                                        */
/* ------------------------------------------------------------------------- */
ORC_EXPORT void orc_row_norms(int32_t n, const double* h, const double* J,
                              double* d) {
  for (int32_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int32_t j = 0; j < n; ++j) {
      double v = J[(int64_t)i * n + j];
      acc += v * v;
    }
    double hi = h ? h[i] : 0.0;
    d[i] = sqrt(hi * hi + acc);
  }
}

ORC_EXPORT void orc_row_norms_csr(int32_t n, const double* h, const int64_t* row_ptr,
                                  const int32_t* col, const double* val, double* d) {
  (void)col;
  for (int32_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) acc += val[k] * val[k];
    double hi = h ? h[i] : 0.0;
    d[i] = sqrt(hi * hi + acc);
  }
}

/* ------------------------------------------------------------------------- */
/* Ising energy, Eq. (1), with each unordered pair counted once:                */
/*   H = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i.                                */
/* ------------------------------------------------------------------------- */
ORC_EXPORT double orc_energy(int32_t n, const double* h, const double* J,
                             const int8_t* s) {
  double pairs = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = i + 1; j < n; ++j)
      pairs += J[(int64_t)i * n + j] * (double)s[i] * (double)s[j];
  double field = 0.0;
  if (h)
    for (int32_t i = 0; i < n; ++i) field += h[i] * (double)s[i];
  return pairs + field;
}

/* Exact version for integer-valued h and J (every value must be an integer of  */
/* magnitude < 2^31; the caller checks).                                        */
ORC_EXPORT int64_t orc_energy_i64(int32_t n, const double* h, const double* J,
                                  const int8_t* s) {
  int64_t pairs = 0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = i + 1; j < n; ++j)
      pairs += (int64_t)J[(int64_t)i * n + j] * (int64_t)s[i] * (int64_t)s[j];
  int64_t field = 0;
  if (h)
    for (int32_t i = 0; i < n; ++i) field += (int64_t)h[i] * (int64_t)s[i];
  return pairs + field;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1.  One call runs `replicas` independent replicas r = 0..R-1.       */
/*   s := 0 (or s0 when given)                                                  */
/*   for t in 0..t_f-1:                                                         */
/*     for every i, from the old s:                                             */
/*       P_i   = h_i + sum_{j ascending} J_ij s_j                               */
/*       Phi_i = P_i / d_i + sigma * z(r,t,i)   (0 / 0 read as 0)               */
/*       sh_i  = -tanh(Phi_i / T_t)                                             */
/*     then for every i: s_i := alpha sh_i + (1 - alpha) s_i                    */
/*   readout: +1 if s_i >= 0 else -1                                            */
/* noise_sign in {+1, 0, -1} multiplies every draw (the spin-flip symmetry test */
/* uses -1).  Dense J is row-major n*n; for the CSR form the sum runs over the  */
/* stored entries of row i in the stored (ascending column) order.              */
/* s_out / phi_out receive the final state and the last step's Phi (replica-    */
/* major, r*n + i) when not NULL.  r_first offsets the replica index used for   */
/* the noise stream, so that any slice of replicas can be recomputed alone;     */
/* t_first offsets the step index in the same way (T[t] is this call's step t,  */
/* drawn as step t_first + t), so that a run can be continued from its state.   */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t n;
  const double* h;
  const double* J;          /* dense, or NULL for CSR */
  const int64_t* row_ptr;   /* CSR */
  const int32_t* col;
  const double* val;
} orc_problem;

static double coupling_sum(const orc_problem* p, int32_t i, const double* s) {
  double acc = 0.0;
  if (p->J) {
    const double* row = p->J + (int64_t)i * p->n;
    for (int32_t j = 0; j < p->n; ++j) acc += row[j] * s[j];
  } else {
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k)
      acc += p->val[k] * s[p->col[k]];
  }
  return acc;
}

static int run_common(const orc_problem* p, const double* T, int32_t t_f, double sigma,
                      double alpha, int32_t replicas, int64_t r_first, int32_t t_first,
                      uint64_t seed, uint32_t stream, int32_t noise_sign, const double* s0,
                      double* s_out,
                      double* phi_out, int8_t* signs_out, int32_t nthreads) {
  const int32_t n = p->n;
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!d) return -4;
  if (p->J)
    orc_row_norms(n, p->h, p->J, d);
  else
    orc_row_norms_csr(n, p->h, p->row_ptr, p->col, p->val, d);
  const double ns = (double)noise_sign;
  int failed = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
#endif
  for (int32_t r = 0; r < replicas; ++r) {
    double* s = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* sh = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* phi = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!s || !sh || !phi) {
      free(s); free(sh); free(phi);
      failed |= 1;
      continue;
    }
    for (int32_t i = 0; i < n; ++i) s[i] = s0 ? s0[(int64_t)r * n + i] : 0.0;
    for (int32_t t = 0; t < t_f; ++t) {
      for (int32_t i = 0; i < n; ++i) {
        double P = (p->h ? p->h[i] : 0.0) + coupling_sum(p, i, s);
        double field = (d[i] > 0.0) ? P / d[i] : 0.0;
        double z = orc_gauss(seed, stream, r_first + r, t_first + t, i);
        phi[i] = field + sigma * z * ns;
        sh[i] = -tanh(phi[i] / T[t]);
      }
      for (int32_t i = 0; i < n; ++i) {
        double a = alpha * sh[i];
        double b = (1.0 - alpha) * s[i];
        s[i] = a + b;
      }
    }
    for (int32_t i = 0; i < n; ++i) {
      if (signs_out) signs_out[(int64_t)r * n + i] = (s[i] >= 0.0) ? 1 : -1;
      if (s_out) s_out[(int64_t)r * n + i] = s[i];
      if (phi_out) phi_out[(int64_t)r * n + i] = (t_f > 0) ? phi[i] : 0.0;
    }
    free(s); free(sh); free(phi);
  }
  free(d);
  return failed ? -4 : 0;
}

ORC_EXPORT int orc_run_dense(int32_t n, const double* h, const double* J, const double* T,
                             int32_t t_f, double sigma, double alpha, int32_t replicas,
                             int64_t r_first, int32_t t_first, uint64_t seed,
                             uint32_t stream, int32_t noise_sign, const double* s0,
                             double* s_out, double* phi_out, int8_t* signs_out,
                             int32_t nthreads) {
  orc_problem p = {n, h, J, NULL, NULL, NULL};
  return run_common(&p, T, t_f, sigma, alpha, replicas, r_first, t_first, seed, stream,
                    noise_sign, s0, s_out, phi_out, signs_out, nthreads);
}

ORC_EXPORT int orc_run_csr(int32_t n, const double* h, const int64_t* row_ptr,
                           const int32_t* col, const double* val, const double* T,
                           int32_t t_f, double sigma, double alpha, int32_t replicas,
                           int64_t r_first, int32_t t_first, uint64_t seed,
                           uint32_t stream, int32_t noise_sign, const double* s0,
                           double* s_out, double* phi_out, int8_t* signs_out,
                           int32_t nthreads) {
  orc_problem p = {n, h, NULL, row_ptr, col, val};
  return run_common(&p, T, t_f, sigma, alpha, replicas, r_first, t_first, seed, stream,
                    noise_sign, s0, s_out, phi_out, signs_out, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Exhaustive ground state for small n (n <= 30): visits all 2^n sign vectors  */
/* in Gray-code order, updating the energy by the single-flip difference        */
/*   dH = -2 s_k (sum_j J_kj s_j + h_k).                                        */
/* Returns the minimum energy, one minimiser and how many vectors attain it.    */
/* ------------------------------------------------------------------------- */
ORC_EXPORT double orc_brute_force(int32_t n, const double* h, const double* J,
                                  int8_t* best, int64_t* n_best) {
  int8_t* s = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
  double* f = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) s[i] = 1;
  for (int32_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int32_t j = 0; j < n; ++j) acc += J[(int64_t)i * n + j];
    f[i] = acc;
  }
  double E = orc_energy(n, h, J, s);
  double Emin = E;
  int64_t count = 1;
  if (best) memcpy(best, s, (size_t)n);
  const uint64_t total = (n > 0) ? (1ull << n) : 1ull;
  for (uint64_t g = 1; g < total; ++g) {
    int32_t k = __builtin_ctzll(g);
    double hk = h ? h[k] : 0.0;
    E += -2.0 * (double)s[k] * (f[k] + hk);
    int8_t old = s[k];
    s[k] = (int8_t)(-old);
    for (int32_t i = 0; i < n; ++i) f[i] += 2.0 * J[(int64_t)i * n + k] * (double)s[k];
    if (E < Emin - 1e-9) {
      Emin = E;
      count = 1;
      if (best) memcpy(best, s, (size_t)n);
    } else if (fabs(E - Emin) <= 1e-9) {
      ++count;
    }
  }
  free(s);
  free(f);
  if (n_best) *n_best = count;
  return Emin;
}
