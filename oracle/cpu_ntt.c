/*
 * Plain CPU negacyclic NTT (oracle directory; test infrastructure and the
 * timed CPU baseline only).
 *
 * Sec. 5 ("NTT"): the same transform as oracle/ntt.py -- slot i holds
 * a(psi^(2 brv(i) + 1)) -- by radix-2 Cooley-Tukey (forward) and
 * Gentleman-Sande (inverse, then N^-1) loops with Harvey's lazy butterflies
 * and Shoup twiddle companions, 128-bit integer products, and one OpenMP
 * thread per group of polynomials.  Checked against oracle.ntt in
 * tests/test_oracle_cpu_ntt.py.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
  uint64_t r = 1;
  a %= q;
  while (e) {
    if (e & 1) r = mulmod(r, a, q);
    a = mulmod(a, a, q);
    e >>= 1;
  }
  return r;
}

static unsigned brv(unsigned x, int bits) {
  unsigned r = 0;
  for (int i = 0; i < bits; ++i) {
    r = (r << 1) | (x & 1);
    x >>= 1;
  }
  return r;
}

/* Twiddle tables: w[k] = psi^brv(k), wi[k] = psi^-brv(k), with Shoup companions. */
void cpu_ntt_tables(uint64_t q, uint64_t psi, int log_n, uint64_t* w, uint64_t* ws, uint64_t* wi, uint64_t* wis) {
  const unsigned n = 1u << log_n;
  const uint64_t psi_inv = powmod(psi, q - 2, q);
  for (unsigned k = 0; k < n; ++k) {
    w[k] = powmod(psi, brv(k, log_n), q);
    wi[k] = powmod(psi_inv, brv(k, log_n), q);
    ws[k] = (uint64_t)(((u128)w[k] << 64) / q);
    wis[k] = (uint64_t)(((u128)wi[k] << 64) / q);
  }
}

static inline uint64_t shoup(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
  const uint64_t qt = (uint64_t)(((u128)a * ws) >> 64);
  return a * w - qt * q; /* [0, 2q) */
}

static void fwd_one(uint64_t* a, unsigned n, uint64_t q, const uint64_t* w, const uint64_t* ws) {
  const uint64_t q2 = 2 * q;
  for (unsigned m = 1, t = n >> 1; m < n; m <<= 1, t >>= 1) {
    for (unsigned i = 0; i < m; ++i) {
      const uint64_t wi = w[m + i], wsi = ws[m + i];
      uint64_t* x = a + 2 * i * t;
      uint64_t* y = x + t;
      for (unsigned j = 0; j < t; ++j) {
        uint64_t u = x[j];
        if (u >= q2) u -= q2;
        const uint64_t v = shoup(y[j], wi, wsi, q);
        x[j] = u + v;
        y[j] = u - v + q2;
      }
    }
  }
  for (unsigned j = 0; j < n; ++j) {
    uint64_t u = a[j];
    if (u >= q2) u -= q2;
    if (u >= q) u -= q;
    a[j] = u;
  }
}

static void inv_one(uint64_t* a, unsigned n, uint64_t q, const uint64_t* wi, const uint64_t* wis, uint64_t ninv,
                    uint64_t ninvs) {
  const uint64_t q2 = 2 * q;
  for (unsigned m = n >> 1, t = 1; m >= 1; m >>= 1, t <<= 1) {
    for (unsigned i = 0; i < m; ++i) {
      const uint64_t w = wi[m + i], ws = wis[m + i];
      uint64_t* x = a + 2 * i * t;
      uint64_t* y = x + t;
      for (unsigned j = 0; j < t; ++j) {
        const uint64_t u = x[j], v = y[j];
        uint64_t s = u + v;
        if (s >= q2) s -= q2;
        x[j] = s;
        y[j] = shoup(u - v + q2, w, ws, q);
      }
    }
    if (m == 1) break;
  }
  for (unsigned j = 0; j < n; ++j) {
    uint64_t u = shoup(a[j], ninv, ninvs, q);
    if (u >= q) u -= q;
    a[j] = u;
  }
}

/* count polynomials of n = 2^log_n coefficients (canonical in and out), in place. */
void cpu_ntt_batch(uint64_t* a, long count, int log_n, uint64_t q, const uint64_t* w, const uint64_t* ws,
                   const uint64_t* wi, const uint64_t* wis, int inverse, int threads) {
  const unsigned n = 1u << log_n;
  const uint64_t ninv = powmod(n, q - 2, q);
  const uint64_t ninvs = (uint64_t)(((u128)ninv << 64) / q);
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(static)
#endif
  for (long p = 0; p < count; ++p) {
    if (inverse)
      inv_one(a + (size_t)p * n, n, q, wi, wis, ninv, ninvs);
    else
      fwd_one(a + (size_t)p * n, n, q, w, ws);
  }
}

int cpu_ntt_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
