/*
 * Plain CPU build of the HE linear-layer pipeline (oracle directory; test
 * infrastructure and the timed CPU baseline of bench.py only).
 *
 * What it computes is oracle/protocol.py's, step by step, in C with 64-bit
 * limbs, OpenMP over ciphertexts and the NTT of oracle/cpu_ntt.c:
 *   encode   (App. A pi_W / pi_v packing, centred lift, NTT)           Sec. 5, App. A
 *   encrypt  (pi_v or pi_W packing, c1 = a, c0 = NTT(round(q m / t) + e) - a s;
 *             a uniform mod q_j from one 64-bit word per coefficient, rejection)   Sec. 2.2
 *   Alg. 1   (c0 + NTT(round(q pi_v(x0) / t)), sum over input blocks of the
 *             ct x pt products, minus NTT(round(q s / t)); MO share s + b)
 *   Alg. 2   (sum Enc(x1) pt(gy0) + Enc(gy1) pt(x0), minus NTT(round(q s / t)))
 *   decrypt  (INTT(c0 + c1 s), m = round(sum_j y_j t / q_j) mod t from the
 *             RNS residues, y_j = x_j (q / q_j)^{-1} mod q_j; t / q_j in 0.128
 *             fixed point: the exact rounding whenever the noise is below q / (4 t))
 * Randomness: Philox4x64-10 (Salmon et al., SC'11) with the oracle's stream
 * layout (key (seed, domain); counter (block, index, limb, 0)), the CDT table
 * of the discrete Gaussian passed in by the caller.
 * Layouts: ciphertexts [count][2][L][N], plaintexts [count][L][N] (NTT form);
 * role arrays V [B][Ci][H][W] (padded input of the role), K [Co][Ci][KH][KW].
 * Checked bit-exactly against oracle/protocol.py in tests/test_oracle_cpu_he.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef uint64_t u64;

void cpu_ntt_tables(u64 q, u64 psi, int log_n, u64* w, u64* ws, u64* wi, u64* wis);
void cpu_ntt_batch(u64* a, long count, int log_n, u64 q, const u64* w, const u64* ws, const u64* wi,
                   const u64* wis, int inverse, int threads);

#define MAXL 4
#define CDT_LEN 19

typedef struct {
  int log_n, n, L, t_bits;
  u64 t_mask, q_mod_t;
  u64 q[MAXL], delta[MAXL], qtil[MAXL], th_hi[MAXL], th_lo[MAXL];
  u64 cdt[CDT_LEN];
  u64 *w, *ws, *wi, *wis;   /* [L][N] twiddles and Shoup companions */
  u64* s_hat;               /* [L][N] secret key, NTT form */
} HeCtx;

typedef struct {
  int B, Ci, Co, H, W, KH, KW;
} Geom;
typedef struct {
  int bb, cib, cob, th, tw, kth, ktw;
} Part;

/* ------------------------------------------------------------------ Philox4x64-10 */
static void philox(u64 c0, u64 c1, u64 c2, u64 c3, u64 k0, u64 k1, u64 out[4]) {
  const u64 M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const u64 W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  for (int r = 0; r < 10; ++r) {
    const u128 p0 = (u128)M0 * c0, p1 = (u128)M1 * c2;
    const u64 n0 = (u64)(p1 >> 64) ^ c1 ^ k0, n2 = (u64)(p0 >> 64) ^ c3 ^ k1;
    c0 = n0;
    c1 = (u64)p1;
    c2 = n2;
    c3 = (u64)p0;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

enum { DOM_SECRET = 1, DOM_A = 2, DOM_E = 3, DOM_MASK = 4, DOM_MASK_PAD = 5 };

/* ------------------------------------------------------------------ context */
HeCtx* cpu_he_create(int log_n, int L, const u64* q, const u64* psi, int t_bits, u64 q_mod_t, const u64* delta,
                     const u64* qtil, const u64* th_hi, const u64* th_lo, const u64* cdt) {
  if (L < 1 || L > MAXL) return NULL;
  HeCtx* c = (HeCtx*)calloc(1, sizeof(HeCtx));
  c->log_n = log_n;
  c->n = 1 << log_n;
  c->L = L;
  c->t_bits = t_bits;
  c->t_mask = (1ull << t_bits) - 1;
  c->q_mod_t = q_mod_t;
  memcpy(c->cdt, cdt, sizeof(c->cdt));
  const size_t ln = (size_t)L * c->n;
  c->w = (u64*)malloc(ln * sizeof(u64));
  c->ws = (u64*)malloc(ln * sizeof(u64));
  c->wi = (u64*)malloc(ln * sizeof(u64));
  c->wis = (u64*)malloc(ln * sizeof(u64));
  c->s_hat = (u64*)calloc(ln, sizeof(u64));
  for (int j = 0; j < L; ++j) {
    c->q[j] = q[j];
    c->delta[j] = delta[j];
    c->qtil[j] = qtil[j];
    c->th_hi[j] = th_hi[j];
    c->th_lo[j] = th_lo[j];
    const size_t o = (size_t)j * c->n;
    cpu_ntt_tables(q[j], psi[j], log_n, c->w + o, c->ws + o, c->wi + o, c->wis + o);
  }
  return c;
}

void cpu_he_destroy(HeCtx* c) {
  if (!c) return;
  free(c->w);
  free(c->ws);
  free(c->wi);
  free(c->wis);
  free(c->s_hat);
  free(c);
}

static void ntt_limbs(const HeCtx* c, u64* poly /* [L][N] */, int inverse) {
  for (int j = 0; j < c->L; ++j) {
    const size_t o = (size_t)j * c->n;
    cpu_ntt_batch(poly + o, 1, c->log_n, c->q[j], c->w + o, c->ws + o, c->wi + o, c->wis + o, inverse, 1);
  }
}

/* Secret key s_i = (w_i mod 3) - 1, w from (seed, DOM_SECRET), counter (i/4, 0, 0, 0). */
void cpu_he_keygen(HeCtx* c, u64 seed) {
  const int n = c->n;
  for (int blk = 0; blk < n / 4; ++blk) {
    u64 w[4];
    philox((u64)blk, 0, 0, 0, seed, DOM_SECRET, w);
    for (int r = 0; r < 4; ++r) {
      const int s = (int)(w[r] % 3) - 1;
      for (int j = 0; j < c->L; ++j) c->s_hat[(size_t)j * n + 4 * blk + r] = s < 0 ? c->q[j] - 1 : (u64)s;
    }
  }
  ntt_limbs(c, c->s_hat, 0);
}

/* ------------------------------------------------------------------ arithmetic */
static inline u64 mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
static inline u64 addmod(u64 a, u64 b, u64 q) {
  const u64 s = a + b;
  return s >= q ? s - q : s;
}
static inline u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

/* round(Q m / t) mod q_j for m in [0, t) (t = 2^t_bits): Delta m + floor(((Q mod t) m + t/2) / t). */
static inline u64 scaled(const HeCtx* c, int j, u64 m) {
  const u128 r = (u128)c->q_mod_t * m + ((u128)1 << (c->t_bits - 1));
  const u64 extra = (u64)(r >> c->t_bits);
  return addmod(mulmod(c->delta[j], m, c->q[j]), extra % c->q[j], c->q[j]);
}

/* ------------------------------------------------------------------ App. A packing */
static int cdiv(int a, int b) { return (a + b - 1) / b; }
typedef struct {
  int MB, MTH, MTW, KC, KTH, KTW, NC;
} Counts;
static Counts counts(const Geom* g, const Part* p) {
  Counts c;
  c.MB = cdiv(g->B, p->bb);
  c.MTH = cdiv(g->H - g->KH + 1, p->th);
  c.MTW = cdiv(g->W - g->KW + 1, p->tw);
  c.KC = cdiv(g->Ci, p->cib);
  c.KTH = cdiv(g->KH, p->kth);
  c.KTW = cdiv(g->KW, p->ktw);
  c.NC = cdiv(g->Co, p->cob);
  return c;
}
static long cnt_M(Counts c) { return (long)c.MB * c.MTH * c.MTW; }
static long cnt_K(Counts c) { return (long)c.KC * c.KTH * c.KTW; }

/* Exponent maps of App. A over the partition's window (h, w) = (th + kth - 1, tw + ktw - 1):
 *   input (b, c, i, j)  -> b cob cib h w + c h w + i w + j
 *   kernel (o, c, u, v) -> O + o cib h w - c h w - u w - v,  O = (cib - 1) h w + (kth - 1) w + ktw - 1
 *   output (b, o, i, j) -> b cob cib h w + O + o cib h w + i w + j */
static long win_h(const Part* p) { return p->th + p->kth - 1; }
static long win_w(const Part* p) { return p->tw + p->ktw - 1; }
static long off_O(const Part* p) { return (long)(p->cib - 1) * win_h(p) * win_w(p) + (long)(p->kth - 1) * win_w(p) + p->ktw - 1; }

/* m-th (batch block, output tile) and k-th (input-channel block, kernel tile) input window as Z_t values. */
static void pack_input(const u64* V, const Geom* g, const Part* p, long m, long k, int n, u64* out) {
  const Counts c = counts(g, p);
  const long mw = m % c.MTW, mh = (m / c.MTW) % c.MTH, mb = m / ((long)c.MTW * c.MTH);
  const long kw = k % c.KTW, kh = (k / c.KTW) % c.KTH, kc = k / ((long)c.KTW * c.KTH);
  const long h = win_h(p), w = win_w(p);
  memset(out, 0, (size_t)n * sizeof(u64));
  for (long b = 0; b < p->bb; ++b) {
    const long gb = mb * p->bb + b;
    if (gb >= g->B) continue;
    for (long ch = 0; ch < p->cib; ++ch) {
      const long gc = kc * p->cib + ch;
      if (gc >= g->Ci) continue;
      for (long i = 0; i < h; ++i) {
        const long r = mh * p->th + kh * p->kth + i;
        if (r >= g->H) continue;
        for (long j = 0; j < w; ++j) {
          const long s = mw * p->tw + kw * p->ktw + j;
          if (s >= g->W) continue;
          out[b * p->cob * p->cib * h * w + ch * h * w + i * w + j] =
              V[((gb * g->Ci + gc) * g->H + r) * g->W + s];
        }
      }
    }
  }
}

/* kernel block (k, nn) */
static void pack_weight(const u64* K, const Geom* g, const Part* p, long k, long nn, int n, u64* out) {
  const Counts c = counts(g, p);
  const long kw = k % c.KTW, kh = (k / c.KTW) % c.KTH, kc = k / ((long)c.KTW * c.KTH);
  const long h = win_h(p), w = win_w(p), O = off_O(p);
  memset(out, 0, (size_t)n * sizeof(u64));
  for (long o = 0; o < p->cob; ++o) {
    const long go = nn * p->cob + o;
    if (go >= g->Co) continue;
    for (long ch = 0; ch < p->cib; ++ch) {
      const long gc = kc * p->cib + ch;
      if (gc >= g->Ci) continue;
      for (long u = 0; u < p->kth; ++u) {
        const long gu = kh * p->kth + u;
        if (gu >= g->KH) continue;
        for (long v = 0; v < p->ktw; ++v) {
          const long gv = kw * p->ktw + v;
          if (gv >= g->KW) continue;
          out[O + o * p->cib * h * w - ch * h * w - u * w - v] = K[((go * g->Ci + gc) * g->KH + gu) * g->KW + gv];
        }
      }
    }
  }
}

/* Output element carried at every decode position of ct_out[m, nn]: exponent and the flat index
 * in the user's output layout (order 0: [B][Co][Ho][Wo]; order 1 (weight gradient): [Co][B][Ho][Wo]).
 * Returns the number of positions written. */
static long decode_positions(const Geom* g, const Part* p, long m, long nn, int order, long* exps, long* flats) {
  const Counts c = counts(g, p);
  const long mw = m % c.MTW, mh = (m / c.MTW) % c.MTH, mb = m / ((long)c.MTW * c.MTH);
  const long h = win_h(p), w = win_w(p), O = off_O(p);
  const long Ho = g->H - g->KH + 1, Wo = g->W - g->KW + 1;
  long cnt = 0;
  for (long b = 0; b < p->bb; ++b) {
    const long gb = mb * p->bb + b;
    if (gb >= g->B) continue;
    for (long o = 0; o < p->cob; ++o) {
      const long go = nn * p->cob + o;
      if (go >= g->Co) continue;
      for (long i = 0; i < p->th; ++i) {
        const long gi = mh * p->th + i;
        if (gi >= Ho) continue;
        for (long j = 0; j < p->tw; ++j) {
          const long gj = mw * p->tw + j;
          if (gj >= Wo) continue;
          exps[cnt] = b * p->cob * p->cib * h * w + O + o * p->cib * h * w + i * w + j;
          flats[cnt] = order ? ((go * g->B + gb) * Ho + gi) * Wo + gj : ((gb * g->Co + go) * Ho + gi) * Wo + gj;
          ++cnt;
        }
      }
    }
  }
  return cnt;
}

/* ------------------------------------------------------------------ encode / encrypt */
static u64 cdt_sample(const HeCtx* c, u64 w, int* neg) {
  const u64 u = w & ((1ull << 63) - 1);
  u64 mag = 0;
  for (int j = 0; j < CDT_LEN; ++j) mag += u >= c->cdt[j];
  *neg = (int)(w >> 63);
  return mag;
}

/* One polynomial of Z_t values -> NTT(centred lift) per limb (a plaintext multiplier). */
static void encode_one(const HeCtx* c, const u64* m, u64* pt) {
  const int n = c->n;
  const u64 half = (c->t_mask >> 1) + 1;
  for (int j = 0; j < c->L; ++j) {
    u64* d = pt + (size_t)j * n;
    const u64 q = c->q[j];
    for (int e = 0; e < n; ++e) {
      const u64 v = m[e] & c->t_mask;
      d[e] = v >= half ? q - ((c->t_mask + 1) - v) : v;
    }
  }
  ntt_limbs(c, pt, 0);
}

/* One polynomial of Z_t values -> symmetric BFV ciphertext idx of the stream seed. */
static void encrypt_one(const HeCtx* c, const u64* m, u64 seed, long idx, u64* ct) {
  const int n = c->n, L = c->L;
  u64* c0 = ct;
  u64* c1 = ct + (size_t)L * n;
  for (int blk = 0; blk < n / 4; ++blk) {
    u64 w[4];
    philox((u64)blk, (u64)idx, 0, 0, seed, DOM_E, w);
    for (int r = 0; r < 4; ++r) {
      const int e = 4 * blk + r;
      int neg;
      const u64 mag = cdt_sample(c, w[r], &neg);
      const u64 mm = m[e] & c->t_mask;
      for (int j = 0; j < L; ++j) {
        const u64 q = c->q[j], v = scaled(c, j, mm);
        c0[(size_t)j * n + e] = neg ? submod(v, mag, q) : addmod(v, mag, q);
      }
    }
  }
  ntt_limbs(c, c0, 0);
  for (int j = 0; j < L; ++j) {
    const u64 q = c->q[j];
    const u64 bound = (u64)((((u128)1) << 64) / q * q - 1);   /* largest accepted word */
    for (int blk = 0; blk < n / 4; ++blk) {
      u64 w[4];
      philox((u64)blk, (u64)idx, (u64)j, 0, seed, DOM_A, w);
      for (int r = 0; r < 4; ++r) {
        const int e = 4 * blk + r;
        u64 x = w[r];
        for (u64 attempt = 1; x > bound; ++attempt) {   /* rejected: fallback counter (e, idx, j, attempt) */
          u64 f[4];
          philox((u64)e, (u64)idx, (u64)j, attempt, seed, DOM_A, f);
          x = f[0];
        }
        const u64 a = x % q;
        c1[(size_t)j * n + e] = a;
        c0[(size_t)j * n + e] = submod(c0[(size_t)j * n + e], mulmod(a, c->s_hat[(size_t)j * n + e], q), q);
      }
    }
  }
}

static int set_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
  return omp_get_max_threads();
#else
  (void)threads;
  return 1;
#endif
}

/* Operand kind 0: input positions (count M K, pi_v of V); 1: kernel positions (count K NC, pi_W of K). */
static long operand_count(const Geom* g, const Part* p, int kind) {
  const Counts c = counts(g, p);
  return kind ? cnt_K(c) * c.NC : cnt_M(c) * cnt_K(c);
}
static void pack_operand(const u64* src, const Geom* g, const Part* p, int kind, long idx, int n, u64* out) {
  const Counts c = counts(g, p);
  if (kind)
    pack_weight(src, g, p, idx / c.NC, idx % c.NC, n, out);
  else
    pack_input(src, g, p, idx / cnt_K(c), idx % cnt_K(c), n, out);
}

void cpu_he_encode(const HeCtx* c, const Geom* g, const Part* p, int kind, const u64* src, u64* pt, int threads) {
  set_threads(threads);
  const long count = operand_count(g, p, kind);
  const size_t ln = (size_t)c->L * c->n;
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    u64* m = (u64*)malloc((size_t)c->n * sizeof(u64));
#ifdef _OPENMP
#pragma omp for schedule(dynamic)
#endif
    for (long i = 0; i < count; ++i) {
      pack_operand(src, g, p, kind, i, c->n, m);
      encode_one(c, m, pt + i * ln);
    }
    free(m);
  }
}

void cpu_he_encrypt(const HeCtx* c, const Geom* g, const Part* p, int kind, const u64* src, u64 seed, u64* ct,
                    int threads) {
  set_threads(threads);
  const long count = operand_count(g, p, kind);
  const size_t ln = (size_t)c->L * c->n;
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    u64* m = (u64*)malloc((size_t)c->n * sizeof(u64));
#ifdef _OPENMP
#pragma omp for schedule(dynamic)
#endif
    for (long i = 0; i < count; ++i) {
      pack_operand(src, g, p, kind, i, c->n, m);
      encrypt_one(c, m, seed, i, ct + 2 * i * ln);
    }
    free(m);
  }
}

/* ------------------------------------------------------------------ the MO's evaluation */
/* Mask polynomial of ct_out o (coefficient form, Z_t): the mask element of every output it
 * carries (stream (seed, DOM_MASK), counter (flat/4, 0, 0, 0), word flat%4), else the padding
 * stream (seed, DOM_MASK_PAD), counter (i/4, o, 0, 0), word i%4. */
static void mask_poly(const HeCtx* c, const Geom* g, const Part* p, int order, u64 seed, long o, long* exps,
                      long* flats, u64* out) {
  const int n = c->n;
  const Counts cn = counts(g, p);
  for (int blk = 0; blk < n / 4; ++blk) {
    u64 w[4];
    philox((u64)blk, (u64)o, 0, 0, seed, DOM_MASK_PAD, w);
    for (int r = 0; r < 4; ++r) out[4 * blk + r] = w[r] & c->t_mask;
  }
  const long np = decode_positions(g, p, o / cn.NC, o % cn.NC, order, exps, flats);
  for (long i = 0; i < np; ++i) {
    u64 w[4];
    philox((u64)(flats[i] / 4), 0, 0, 0, seed, DOM_MASK, w);
    out[exps[i]] = w[flats[i] % 4] & c->t_mask;
  }
}

/* x mod q of a 128-bit lazy sum. */
static inline u64 red128(u128 x, u64 q) { return (u64)(x % q); }

/* Alg. 1 (roles forward and input gradient) for every output ciphertext:
 * ct_out[m NC + n] = sum_k (ct_in[m K + k] + NTT(round(q pi_v(V0)_{m,k} / t))) pt[k NC + n]
 *                    - NTT(round(q s / t));  y0[flat] = s[flat] (+ bias[o], order 0).
 * V0 may be NULL (no MO input share); bias may be NULL. */
void cpu_he_alg1(const HeCtx* c, const Geom* g, const Part* p, const u64* ct_in, const u64* pt, const u64* V0,
                 const u64* bias, u64 mask_seed, int order, u64* ct_out, u64* y0, int threads) {
  set_threads(threads);
  const Counts cn = counts(g, p);
  const long M = cnt_M(cn), K = cnt_K(cn), NC = cn.NC;
  const int n = c->n, L = c->L;
  const size_t ln = (size_t)L * n;
  /* NTT(round(q pi_v(V0) / t)) of every input position, added to c0 (Alg. 1 step 2) */
  u64* x0hat = NULL;
  if (V0) {
    x0hat = (u64*)malloc((size_t)M * K * ln * sizeof(u64));
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
      u64* m = (u64*)malloc((size_t)n * sizeof(u64));
#ifdef _OPENMP
#pragma omp for schedule(dynamic)
#endif
      for (long i = 0; i < M * K; ++i) {
        pack_input(V0, g, p, i / K, i % K, n, m);
        u64* d = x0hat + i * ln;
        for (int j = 0; j < L; ++j)
          for (int e = 0; e < n; ++e) d[(size_t)j * n + e] = scaled(c, j, m[e] & c->t_mask);
        ntt_limbs(c, d, 0);
      }
      free(m);
    }
  }
  const long ho = g->H - g->KH + 1, wo = g->W - g->KW + 1;
  const long outs = (long)g->B * g->Co * ho * wo;
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    u64* s = (u64*)malloc((size_t)n * sizeof(u64));
    u64* sh = (u64*)malloc(ln * sizeof(u64));
    long* exps = (long*)malloc((size_t)n * sizeof(long));
    long* flats = (long*)malloc((size_t)n * sizeof(long));
    u128* acc = (u128*)malloc(2 * ln * sizeof(u128));
#ifdef _OPENMP
#pragma omp for schedule(dynamic)
#endif
    for (long o = 0; o < M * NC; ++o) {
      const long m = o / NC, nn = o % NC;
      memset(acc, 0, 2 * ln * sizeof(u128));
      for (long k = 0; k < K; ++k) {
        const u64* a = ct_in + 2 * (m * K + k) * ln;
        const u64* b = pt + (k * NC + nn) * ln;
        const u64* x0 = x0hat ? x0hat + (m * K + k) * ln : NULL;
        for (int j = 0; j < L; ++j) {
          const u64 q = c->q[j];
          for (int e = 0; e < n; ++e) {
            const size_t i = (size_t)j * n + e;
            const u64 a0 = x0 ? addmod(a[i], x0[i], q) : a[i];
            acc[i] += (u128)a0 * b[i];
            acc[ln + i] += (u128)a[ln + i] * b[i];
          }
        }
        if ((k & 127) == 127)
          for (size_t i = 0; i < 2 * ln; ++i) acc[i] = red128(acc[i], c->q[(i % ln) / n]);
      }
      mask_poly(c, g, p, order, mask_seed, o, exps, flats, s);
      for (int j = 0; j < L; ++j)
        for (int e = 0; e < n; ++e) sh[(size_t)j * n + e] = scaled(c, j, s[e]);
      ntt_limbs(c, sh, 0);
      u64* out = ct_out + 2 * o * ln;
      for (size_t i = 0; i < ln; ++i) {
        const u64 q = c->q[i / n];
        out[i] = submod(red128(acc[i], q), sh[i], q);
        out[ln + i] = red128(acc[ln + i], q);
      }
    }
    free(s);
    free(sh);
    free(exps);
    free(flats);
    free(acc);
  }
  free(x0hat);
  /* MO share: s[flat] (+ bias of the output channel, forward role) */
  for (long f = 0; f < outs; ++f) {
    u64 w[4];
    philox((u64)(f / 4), 0, 0, 0, mask_seed, DOM_MASK, w);
    u64 v = w[f % 4] & c->t_mask;
    if (bias && !order) v = (v + bias[(f / (ho * wo)) % g->Co]) & c->t_mask;
    y0[f] = v;
  }
}

/* Alg. 2 (weight gradient): ct_out[m NC + n] = sum_k ct_x1[m K + k] pt_gy0[k NC + n]
 *   + ct_gy1[k NC + n] pt_x0[m K + k] - NTT(round(q s / t));  y0 = s ([Co][B][Ho][Wo] order). */
void cpu_he_alg2(const HeCtx* c, const Geom* g, const Part* p, const u64* ct_x1, const u64* pt_gy0,
                 const u64* ct_gy1, const u64* pt_x0, u64 mask_seed, u64* ct_out, u64* y0, int threads) {
  set_threads(threads);
  const Counts cn = counts(g, p);
  const long M = cnt_M(cn), K = cnt_K(cn), NC = cn.NC;
  const int n = c->n, L = c->L;
  const size_t ln = (size_t)L * n;
  const long ho = g->H - g->KH + 1, wo = g->W - g->KW + 1;
  const long outs = (long)g->B * g->Co * ho * wo;
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    u64* s = (u64*)malloc((size_t)n * sizeof(u64));
    u64* sh = (u64*)malloc(ln * sizeof(u64));
    long* exps = (long*)malloc((size_t)n * sizeof(long));
    long* flats = (long*)malloc((size_t)n * sizeof(long));
    u128* acc = (u128*)malloc(2 * ln * sizeof(u128));
#ifdef _OPENMP
#pragma omp for schedule(dynamic)
#endif
    for (long o = 0; o < M * NC; ++o) {
      const long m = o / NC, nn = o % NC;
      memset(acc, 0, 2 * ln * sizeof(u128));
      for (long k = 0; k < K; ++k) {
        const u64* x1 = ct_x1 + 2 * (m * K + k) * ln;
        const u64* g0 = pt_gy0 + (k * NC + nn) * ln;
        const u64* g1 = ct_gy1 + 2 * (k * NC + nn) * ln;
        const u64* x0 = pt_x0 + (m * K + k) * ln;
        for (size_t i = 0; i < ln; ++i) {
          acc[i] += (u128)x1[i] * g0[i] + (u128)g1[i] * x0[i];
          acc[ln + i] += (u128)x1[ln + i] * g0[i] + (u128)g1[ln + i] * x0[i];
        }
        if ((k & 63) == 63)
          for (size_t i = 0; i < 2 * ln; ++i) acc[i] = red128(acc[i], c->q[(i % ln) / n]);
      }
      mask_poly(c, g, p, 1, mask_seed, o, exps, flats, s);
      for (int j = 0; j < L; ++j)
        for (int e = 0; e < n; ++e) sh[(size_t)j * n + e] = scaled(c, j, s[e]);
      ntt_limbs(c, sh, 0);
      u64* out = ct_out + 2 * o * ln;
      for (size_t i = 0; i < ln; ++i) {
        const u64 q = c->q[i / n];
        out[i] = submod(red128(acc[i], q), sh[i], q);
        out[ln + i] = red128(acc[ln + i], q);
      }
    }
    free(s);
    free(sh);
    free(exps);
    free(flats);
    free(acc);
  }
  for (long f = 0; f < outs; ++f) {
    u64 w[4];
    philox((u64)(f / 4), 0, 0, 0, mask_seed, DOM_MASK, w);
    y0[f] = w[f % 4] & c->t_mask;
  }
}

/* ------------------------------------------------------------------ decryption */
/* y1[flat] = round(t x / q) mod t at every output position of every ct_out. */
void cpu_he_decrypt(const HeCtx* c, const Geom* g, const Part* p, int order, const u64* ct_out, u64* y1,
                    int threads) {
  set_threads(threads);
  const Counts cn = counts(g, p);
  const long count = cnt_M(cn) * cn.NC;
  const int n = c->n, L = c->L;
  const size_t ln = (size_t)L * n;
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    u64* x = (u64*)malloc(ln * sizeof(u64));
    long* exps = (long*)malloc((size_t)n * sizeof(long));
    long* flats = (long*)malloc((size_t)n * sizeof(long));
#ifdef _OPENMP
#pragma omp for schedule(dynamic)
#endif
    for (long o = 0; o < count; ++o) {
      const u64* ct = ct_out + 2 * o * ln;
      for (size_t i = 0; i < ln; ++i) {
        const u64 q = c->q[i / n];
        x[i] = addmod(ct[i], mulmod(ct[ln + i], c->s_hat[i], q), q);
      }
      ntt_limbs(c, x, 1);
      const long np = decode_positions(g, p, o / cn.NC, o % cn.NC, order, exps, flats);
      for (long t = 0; t < np; ++t) {
        /* S = sum_j y_j th_j (192 bits), m = floor((S + 2^127) / 2^128) mod 2^t_bits */
        u64 w0 = 0, w1 = 0, w2 = 0;
        for (int j = 0; j < L; ++j) {
          const u64 y = mulmod(x[(size_t)j * n + exps[t]], c->qtil[j], c->q[j]);
          const u128 pl = (u128)y * c->th_lo[j], ph = (u128)y * c->th_hi[j];
          u128 s0 = (u128)w0 + (u64)pl;
          w0 = (u64)s0;
          u128 s1 = (u128)w1 + (u64)(pl >> 64) + (u64)ph + (u64)(s0 >> 64);
          w1 = (u64)s1;
          w2 += (u64)(ph >> 64) + (u64)(s1 >> 64);
        }
        const u128 r1 = (u128)w1 + (1ull << 63);
        const u64 top = w2 + (u64)(r1 >> 64);
        y1[flats[t]] = top & c->t_mask;
      }
    }
    free(x);
    free(exps);
    free(flats);
  }
}
