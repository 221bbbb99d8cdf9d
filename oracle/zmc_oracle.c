/*
 * zmc_oracle.c — the FP64 CPU oracle for parameter-grid direct Monte Carlo.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The CUDA product path never
 * links, imports or calls it, and shares no code with it: this file has its
 * own Philox4x32-10, its own uniform map, its own grid decode and its own
 * integrand definitions.
 *
 * What it computes (the method of "ZMCintegral-v5", arXiv:1910.01965):
 *   f(x) = \int dy g(y; x) over a box in N dimensions (Eq. 1, Sec. 2), for
 *   every point x of a Cartesian grid built from M per-parameter value lists
 *   (Sec. 2), by the direct (plain) Monte Carlo method (Sec. 1 and Sec. 2:
 *   no stratification, no adaptive search), repeated over T independent
 *   trials (Sec. 3.2, "independently for 10 times").
 *
 * The paper names no random number generator.  This oracle draws samples
 * from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11).  Call j of grid point p in trial t has counter
 * (j, t, p mod 2^32, p >> 32) and key (seed mod 2^32, seed >> 32); its four
 * output words r0..r3 form the 128-bit block B = r0 + r1 2^32 + r2 2^64 +
 * r3 2^96, which is cut into five 23-bit fields (bits 23m .. 23m+22 for
 * m = 0..4; the top 13 bits are not used).  Field i of the stream is field
 * (i mod 5) of call floor(i/5).  Sample s, dimension k uses field i = s*N + k:
 * its value v maps to u = (2 v + 1) * 2^-24, strictly inside (0, 1), and to
 * y_k = fma(b_k - a_k, u, a_k).
 *
 * The estimator is written out plainly, in FP64, in sequential order:
 *   s1_t = sum_s g(y_s; x),  s2_t = sum_s g(y_s; x)^2,
 *   I_t  = V * s1_t / S,     mean = (sum_t I_t) / T,
 *   err  = sqrt( sum_t (I_t - mean)^2 / (T (T - 1)) )      (NaN when T = 1),
 *   errw = V * sqrt( (sum_t (s2_t - s1_t^2/S)/(S - 1)) / T / (T S) )
 *                                                           (NaN when S = 1),
 * with V = prod_k (b_k - a_k).  Grid points are independent, so the loop over
 * them may run on several threads without changing any result.
 *
 * Built with -O2 -ffp-contract=off and without -ffast-math, so that every
 * operation is the one written here, on x86_64 and aarch64 alike.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, SC'11: two 32x32->64 multiplies per round, the high halves  */
/* XORed with the other counter words and the round key; the key advances by */
/* the Weyl increments between rounds.                                        */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void zmc_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                              uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += ORC_PHILOX_W0;
      k1 += ORC_PHILOX_W1;
    }
    uint64_t prod0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A 23-bit field value v (0 <= v < 2^23) -> u = (2 v + 1) * 2^-24, exactly,
 * in (0, 1). */
double zmc_oracle_uniform(uint32_t v) {
  uint32_t odd = 2u * v + 1u;
  return ldexp((double)odd, -24);
}

/* The four output words of call j for (seed, p, t). */
static void oracle_call(uint64_t seed, int64_t p, int t, uint64_t j, uint32_t out[4]) {
  uint32_t ctr[4], key[2];
  ctr[0] = (uint32_t)j;
  ctr[1] = (uint32_t)t;
  ctr[2] = (uint32_t)((uint64_t)p & 0xffffffffu);
  ctr[3] = (uint32_t)((uint64_t)p >> 32);
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32);
  zmc_oracle_philox4x32_10(ctr, key, out);
}

/* Raw word w of the stream of (seed, p, t): lane w mod 4 of call floor(w/4). */
uint32_t zmc_oracle_word(uint64_t seed, int64_t p, int t, uint64_t w) {
  uint32_t out[4];
  oracle_call(seed, p, t, w >> 2, out);
  return out[w & 3u];
}

/* Field i of the stream of (seed, p, t): bits 23m .. 23m+22 of the 128-bit
 * block of call floor(i/5), m = i mod 5. */
uint32_t zmc_oracle_field(uint64_t seed, int64_t p, int t, uint64_t i) {
  uint32_t out[4];
  uint64_t j = i / 5u;
  int m = (int)(i % 5u);
  oracle_call(seed, p, t, j, out);
  int bit = 23 * m;
  int q = bit / 32, sh = bit % 32;
  uint64_t pair = (uint64_t)out[q] | ((uint64_t)out[q + 1] << 32);  /* q <= 2 */
  return (uint32_t)((pair >> sh) & 0x7fffffu);
}

/* Sample point y (N values) for sample s of (p, t): direct MC over the box. */
void zmc_oracle_sample_y(int N, const double* lo, const double* hi,
                         uint64_t seed, int64_t p, int t, int64_t s,
                         double* y) {
  for (int k = 0; k < N; ++k) {
    uint64_t i = (uint64_t)s * (uint64_t)N + (uint64_t)k;
    double u = zmc_oracle_uniform(zmc_oracle_field(seed, p, t, i));
    y[k] = fma(hi[k] - lo[k], u, lo[k]);
  }
}

/* ------------------------------------------------------------------------ */
/* Grid decode (Sec. 2): each parameter x_i takes values from its own list,  */
/* the grid is their Cartesian product.  Flat index p -> digits in C order   */
/* (the last list varies fastest).                                            */
/* ------------------------------------------------------------------------ */
void zmc_oracle_decode(int M, const int64_t* len, int64_t p, int64_t* digit) {
  for (int i = M - 1; i >= 0; --i) {
    digit[i] = p % len[i];
    p = p / len[i];
  }
}

void zmc_oracle_grid_point(int M, const int64_t* len, const double* vals,
                           int64_t p, double* x) {
  int64_t digit[64];
  zmc_oracle_decode(M, len, p, digit);
  int64_t offset = 0;
  for (int i = 0; i < M; ++i) {
    x[i] = vals[offset + digit[i]];
    offset += len[i];
  }
}

/* ------------------------------------------------------------------------ */
/* Integrands g(y; x).  Ids match the library's registry numbering.          */
/* ------------------------------------------------------------------------ */
enum {
  ORC_G_CONST = 0,   /* 1                                                   */
  ORC_G_COSPROD = 1, /* prod_k cos(x_k y_k),                     M = N       */
  ORC_G_GAUSS03 = 2, /* exp(-sum_k (y_k - x_k)^2 / (2 * 0.3^2)), M = N       */
  ORC_G_POLY = 3,    /* prod_k (1 + x_k y_k^2),                  M = N       */
  ORC_G_OSC01 = 4,   /* cos(sum_k x_k y_k + 0.1 sum_k y_k^2),    M = N       */
  ORC_G_SINSUM = 5,  /* sin(sum_k y_k + sum_l x_l), any M (Eq. 2, Eq. 4)      */
  ORC_G_COUNT = 6
};

/* Returns 1 if (id, N, M) is a valid combination. */
int zmc_oracle_integrand_valid(int id, int N, int M) {
  if (N < 1 || N > 8 || M < 1 || M > 64) return 0;
  switch (id) {
    case ORC_G_CONST:
    case ORC_G_SINSUM:
      return 1;
    case ORC_G_COSPROD:
    case ORC_G_GAUSS03:
    case ORC_G_POLY:
    case ORC_G_OSC01:
      return M == N;
    default:
      return 0;
  }
}

double zmc_oracle_integrand(int id, int N, const double* y, int M,
                            const double* x) {
  switch (id) {
    case ORC_G_CONST:
      return 1.0;
    case ORC_G_COSPROD: {
      double g = 1.0;
      for (int k = 0; k < N; ++k) g *= cos(x[k] * y[k]);
      return g;
    }
    case ORC_G_GAUSS03: {
      double sigma = 0.3, q = 0.0;
      for (int k = 0; k < N; ++k) q += (y[k] - x[k]) * (y[k] - x[k]);
      return exp(-q / (2.0 * sigma * sigma));
    }
    case ORC_G_POLY: {
      double g = 1.0;
      for (int k = 0; k < N; ++k) g *= 1.0 + x[k] * y[k] * y[k];
      return g;
    }
    case ORC_G_OSC01: {
      double lin = 0.0, quad = 0.0;
      for (int k = 0; k < N; ++k) {
        lin += x[k] * y[k];
        quad += y[k] * y[k];
      }
      return cos(lin + 0.1 * quad);
    }
    case ORC_G_SINSUM: {
      double a = 0.0;
      for (int k = 0; k < N; ++k) a += y[k];
      for (int l = 0; l < M; ++l) a += x[l];
      return sin(a);
    }
    default:
      return NAN;
  }
}

/* ------------------------------------------------------------------------ */
/* The estimator for one grid point: T trials of S samples each.             */
/* ------------------------------------------------------------------------ */
static void oracle_point(int id, int N, const double* lo, const double* hi,
                         int M, const int64_t* len, const double* vals,
                         int64_t S, int T, uint64_t seed, int64_t p,
                         double* mean_out, double* err_out, double* errw_out,
                         double* s1_out, double* s2_out) {
  double x[64], y[8];
  zmc_oracle_grid_point(M, len, vals, p, x);

  double V = 1.0;
  for (int k = 0; k < N; ++k) V *= hi[k] - lo[k];

  double* I = (double*)malloc(sizeof(double) * (size_t)T);
  double pooled_var = 0.0;
  for (int t = 0; t < T; ++t) {
    double s1 = 0.0, s2 = 0.0;
    for (int64_t s = 0; s < S; ++s) {
      zmc_oracle_sample_y(N, lo, hi, seed, p, t, s, y);
      double g = zmc_oracle_integrand(id, N, y, M, x);
      s1 += g;
      s2 += g * g;
    }
    I[t] = V * s1 / (double)S;
    if (s1_out) s1_out[t] = s1;
    if (s2_out) s2_out[t] = s2;
    pooled_var += (s2 - s1 * s1 / (double)S) / (double)(S - 1);
  }

  double sum = 0.0;
  for (int t = 0; t < T; ++t) sum += I[t];
  double mean = sum / (double)T;

  double dev2 = 0.0;
  for (int t = 0; t < T; ++t) dev2 += (I[t] - mean) * (I[t] - mean);
  double err = (T > 1) ? sqrt(dev2 / ((double)T * (double)(T - 1))) : NAN;

  double errw = NAN;
  if (S > 1) {
    pooled_var = pooled_var / (double)T;
    errw = V * sqrt(pooled_var / ((double)T * (double)S));
  }
  free(I);

  *mean_out = mean;
  *err_out = err;
  if (errw_out) *errw_out = errw;
}

/*
 * Evaluate the listed grid points.  points[i] is a flat index in [0, P).
 * out_mean, out_err (and out_errw if non-NULL) have npoints entries;
 * out_s1, out_s2 (if non-NULL) have npoints*T entries, trial fastest.
 * Returns 0 on success, 1 on invalid arguments.
 * nthreads <= 0 uses every thread OpenMP offers.
 */
int zmc_oracle_scan_points(int id, int N, const double* lo, const double* hi,
                           int M, const int64_t* len, const double* vals,
                           int64_t S, int T, uint64_t seed,
                           const int64_t* points, int64_t npoints,
                           double* out_mean, double* out_err, double* out_errw,
                           double* out_s1, double* out_s2, int nthreads) {
  if (!zmc_oracle_integrand_valid(id, N, M)) return 1;
  if (S < 1 || T < 1 || npoints < 0) return 1;
  int64_t P = 1;
  for (int i = 0; i < M; ++i) {
    if (len[i] < 1) return 1;
    P *= len[i];
  }
  for (int k = 0; k < N; ++k)
    if (!(hi[k] > lo[k])) return 1;
  for (int64_t i = 0; i < npoints; ++i)
    if (points[i] < 0 || points[i] >= P) return 1;

#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < npoints; ++i) {
    oracle_point(id, N, lo, hi, M, len, vals, S, T, seed, points[i],
                 &out_mean[i], &out_err[i], out_errw ? &out_errw[i] : NULL,
                 out_s1 ? &out_s1[i * T] : NULL,
                 out_s2 ? &out_s2[i * T] : NULL);
  }
  return 0;
}

/* Threads the parallel loop would use (for reporting the core count). */
int zmc_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
