// Device-side building blocks of the Pencil HE hot path on sm_103a:
// 64-bit modular arithmetic (Shoup, Barrett, Harvey lazy butterflies),
// Philox4x64-10, and the parameter structs every kernel receives by value.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;

#define PENCIL_MAX_LIMBS 4

// ------------------------------------------------------------------ structs
// Per-limb constants for q_j (all computed on the host at context creation).
struct LimbConst {
  u64 q;
  u64 mu;            // floor(2^64 / q)                           (Barrett)
  u64 r64, r64s;     // 2^64 mod q and its Shoup companion
  u64 ninv, ninvs;   // N^{-1} mod q                              (INTT scaling)
  u64 delta, deltas; // floor(q_total / t) mod q                  (BFV Delta)
  u64 qtil, qtils;   // (q_total / q_j)^{-1} mod q_j              (CRT)
  u64 th_hi, th_lo;  // floor(2^(128 + t_bits) / q_j), 128 bits   (t / q_j in 0.128 fixed point)
  u64 c60, c64;      // 2^60 mod q and 2^64 mod q                 (split multiply-accumulate folds)
  u64 nqtil, nqtils; // N^{-1} qtil mod q_j                       (INTT scaling folded into the CRT factor)
  u64 a_max;         // floor(2^64 / q) q - 1: the largest 64-bit word accepted for a uniform residue
  // Final scaling kappa of an inverse transform merged into its last stage (fold
  // engine): {kappa, kappa 2^32, w1 kappa, w1 kappa 2^32} mod q, w1 = psi^-brv(1)
  // the one twiddle of that stage; kappa = N^{-1} (sc_ninv) or N^{-1} qtil (sc_nqtil).
  u64 sc_ninv[4];
  u64 sc_nqtil[4];
};

struct DevCtx {
  int log_n;
  int ntt_loge;              // log2(coefficients per thread) of the NTT kernels: 4 or 5
  int n;
  int L;
  int t_bits;
  u64 t_mask;
  LimbConst limb[PENCIL_MAX_LIMBS];
  const ulonglong2* tw_fwd;  // [L][N] (psi^brv(k), Shoup companion)
  const ulonglong2* tw_inv;  // [L][N] (psi^-brv(k), Shoup companion)
  int ntt_arith;             // butterflies of the NTT kernels: 0 Shoup / Harvey, 1 pseudo-Mersenne folds
  const ulonglong2* tw_fwd_f;  // [L][N] (psi^brv(k), psi^brv(k) 2^32 mod q)   (null unless every
  const ulonglong2* tw_inv_f;  // [L][N] (psi^-brv(k), psi^-brv(k) 2^32 mod q)  q_j = 2^60 - c, c < 2^24)
  int* status;               // device status word (atomicOr of error bits)
  int mac_split;             // 1: every q_j in (2^59 + 2^33, 2^60) with 2^60, 2^64 mod q_j < 2^28 (30-bit split MAC)
  int mac_nt;                // output columns per thread of the split MAC: 2, 4 or 8
  int mac_staging;           // operand staging of the split MAC: 0 per-thread cp.async ring, 1 bulk copies
  u64 q_mod_t;               // (q_total mod t): messages are scaled as round(q_total m / t)
  int flood_bits;            // 0, or the flooding noise of returned ciphertexts: uniform in [-2^b, 2^b)
};

// A strided view of a user tensor seen as (a, b, r, s) with spatial zero
// padding: element = ptr[base + a*s0 + b*s1 + (r-pr)*s2 + (s-ps)*s3] when
// 0 <= r-pr < hr and 0 <= s-ps < wr, else 0.
struct Accessor {
  const u64* ptr;
  i64 base;
  i64 s0, s1, s2, s3;
  int pr, ps, hr, wr;
};

// Packing of one operand position class (inputs, kernels or outputs):
// tab[e] = local (a, b, r, s) of coefficient e packed as 4 x 16 bits, or
// all-ones when coefficient e carries nothing; org[idx] = the block origin of
// polynomial idx; bound = the geometry extent of (a, b, r, s); support = 1 +
// the highest e with an entry (coefficients from support on are always zero).
struct Packing {
  const u64* tab;
  const int4* org;
  int4 bound;
  int support;
};

#define PENCIL_TAB_NONE 0xFFFFFFFFFFFFFFFFull

// ------------------------------------------------------------------ 64-bit modular arithmetic
__device__ __forceinline__ u64 mulhi64(u64 a, u64 b) { return __umul64hi(a, b); }

// a * w mod q in [0, 2q), w < q, ws = floor(w 2^64 / q), any a < 2^64 (Shoup).
__device__ __forceinline__ u64 mul_shoup_lazy(u64 a, u64 w, u64 ws, u64 q) {
  u64 qt = mulhi64(a, ws);
  return a * w - qt * q;
}

__device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }

__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 ws, u64 q) {
  return csub(mul_shoup_lazy(a, w, ws, q), q);
}

// x mod q for any x < 2^64 with mu = floor(2^64 / q) (Barrett, one correction).
__device__ __forceinline__ u64 reduce64(u64 x, const LimbConst& c) {
  u64 qt = mulhi64(x, c.mu);
  return csub(x - qt * c.q, c.q);
}

// (hi * 2^64 + lo) mod q, canonical.  Shoup's product accepts any hi < 2^64.
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const LimbConst& c) {
  u64 t = mul_shoup_lazy(hi, c.r64, c.r64s, c.q);  // [0, 2q)
  u64 rl = reduce64(lo, c);
  u64 s = t + rl;                                   // [0, 3q)
  s = csub(s, 2 * c.q);
  return csub(s, c.q);
}

// Alternative formulations measured by pencil_mul_probe (variants 4, 5, 7):
// on GB300 32x32 high products and 32x32->64 products run at half the rate of
// 32-bit multiply-adds, and these variants came out no faster than the
// compiler's Shoup product, so the NTT kernels use Harvey's butterflies below.
//
// a * w mod q in [0, 3q) for ANY a < 2^64, with w < q < 2^62, ws = floor(w 2^64 / q)
// and nq = 2^64 - q.  Shoup's quotient hi64(a * ws) is formed from three
// 32x32->64 multiply-adds (the low x low partial product is dropped, so the
// quotient may be one below Shoup's and the remainder one q above his range
// [0, 2q)); the remainder a * w - qt * q is computed as a * w + qt * nq mod 2^64
// from two more 32x32->64 products and four 32-bit multiply-adds.
__host__ __device__ __forceinline__ u64 mul_shoup3(u64 a, u64 w, u64 ws, u64 nq) {
  const u32 a0 = (u32)a, a1 = (u32)(a >> 32);
  const u32 s0 = (u32)ws, s1 = (u32)(ws >> 32);
  const u64 t = (u64)a0 * s1;
  const u64 u = (u64)a1 * s0 + (u32)t;
  const u64 qt = (u64)a1 * s1 + ((t >> 32) + (u >> 32));
  const u32 w0 = (u32)w, w1 = (u32)(w >> 32);
  const u32 n0 = (u32)nq, n1 = (u32)(nq >> 32);
  const u32 q0 = (u32)qt, q1 = (u32)(qt >> 32);
  const u64 r = (u64)a0 * w0 + (u64)q0 * n0;
  const u32 hi = a1 * w0 + a0 * w1 + q1 * n0 + q0 * n1;
  return r + ((u64)hi << 32);
}

// x - c if x >= c else x, for x < 2^63 and c < 2^63 (sign of the difference).
__host__ __device__ __forceinline__ u64 csub_s(u64 x, u64 c) {
  const u64 d = x - c;
  return ((i64)d < 0) ? x : d;
}

// Cooley-Tukey butterfly on the lazy range [0, 8q) (needs q < 2^60):
// x, y in [0, 8q) -> x + w y, x - w y (mod q) in [0, 8q).
__host__ __device__ __forceinline__ void ct_bf8(u64& x, u64& y, u64 w, u64 ws, u64 nq, u64 q3, u64 q4) {
  const u64 a = csub_s(x, q4);                 // [0, 4q)
  const u64 t = mul_shoup3(y, w, ws, nq);      // [0, 3q)
  x = a + t;                                   // [0, 7q)
  y = a + q3 - t;                              // (0, 7q]
}

// Gentleman-Sande butterfly on the lazy range [0, 4q):
// x, y in [0, 4q) -> x + y, (x - y) w (mod q) in [0, 4q).
__host__ __device__ __forceinline__ void gs_bf4(u64& x, u64& y, u64 w, u64 ws, u64 nq, u64 q4) {
  const u64 s = csub_s(x + y, q4);             // [0, 4q)
  const u64 d = x + q4 - y;                    // (0, 8q)
  x = s;
  y = mul_shoup3(d, w, ws, nq);                // [0, 3q)
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return csub(a + b, q); }

// round(q_total m / t) mod q_j for m in [0, t): Delta m + floor(((q_total mod t) m + t / 2) / t),
// the BFV message scaling (t = 2^t_bits, so the division is a shift of the
// 128-bit product; the quotient is below t < q_j).
__device__ __forceinline__ u64 scale_msg(u64 m, const LimbConst& lc, const DevCtx& c) {
  const u64 lo = c.q_mod_t * m, hi = __umul64hi(c.q_mod_t, m);
  const u64 slo = lo + (1ull << (c.t_bits - 1));
  const u64 shi = hi + (slo < lo ? 1ull : 0ull);
  const u64 extra = (shi << (64 - c.t_bits)) | (slo >> c.t_bits);
  return add_mod(mul_shoup(m, lc.delta, lc.deltas, lc.q), extra, lc.q);
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulate: (hi, lo) += a * b.
__device__ __forceinline__ void mac128(u64& lo, u64& hi, u64 a, u64 b) {
  u64 plo = a * b;
  u64 phi = mulhi64(a, b);
  lo += plo;
  hi += phi + (lo < plo ? 1ull : 0ull);
}

// Harvey Cooley-Tukey butterfly: x, y in [0, 4q) -> x + w y, x - w y in [0, 4q).
__device__ __forceinline__ void ct_butterfly(u64& x, u64& y, u64 w, u64 ws, u64 q, u64 q2) {
  u64 a = x >= q2 ? x - q2 : x;
  u64 t = mul_shoup_lazy(y, w, ws, q);
  x = a + t;
  y = a - t + q2;
}

// Harvey Gentleman-Sande butterfly: x, y in [0, 2q) -> x + y, (x - y) w in [0, 2q).
__device__ __forceinline__ void gs_butterfly(u64& x, u64& y, u64 w, u64 ws, u64 q, u64 q2) {
  u64 s = x + y;
  s = s >= q2 ? s - q2 : s;
  u64 d = x - y + q2;
  x = s;
  y = mul_shoup_lazy(d, w, ws, q);
}

// ------------------------------------------------------------------ pseudo-Mersenne twiddle products
// For q = 2^60 - c with c < 2^24 (every prime of the 60-bit parameter sets):
// 2^60 = c60 = c and 2^64 = c64 = 16 c (mod q).  Beside each twiddle w the table
// holds w32 = w 2^32 mod q, so that for y = y1 2^32 + y0 (any y < 2^64)
//   y w = y0 w + y1 w32 (mod q),
// a sum S < 2^93 of four 32x32->64 partial products (no quotient estimate).  With
// S = sh 2^64 + sm 2^60 + sl (sh <= 2^29 + 1, sm < 16, sl < 2^60) the folds
//   S = sl + sm c60 + sh c64 (mod q) < 2^60 + 2^57 + 2^30 < 1.13 q
// leave a lazy residue; the product is six 32x32->64 multiply-adds and seven
// 32-bit ALU operations, against six such products, four 32-bit multiply-adds
// and the correction of a Shoup product (measured with pencil_mul_probe's
// counters: a Shoup product occupies the multiply pipe 34 cycles per warp).
// Written as one PTX block so that every 64-bit addend of a 32x32->64
// multiply-add is a register pair that a previous multiply produced (addends
// assembled from 32-bit halves cost register moves: measured 30.6 -> 25.0
// instructions per warp of butterflies in the N = 8192 forward transform).
//   h = y1 w32h + y0 wh (< 2^61),  l = y0 wl,  m = y1 w32l,
//   S = l + m + 2^32 h = u 2^64 + t 2^32 + s0   (one 32-bit carry chain),
//   sm = t >> 28, sl = (t mod 2^28) 2^32 + s0, sh = u.
__device__ __forceinline__ u64 mul_fold(u64 y, u64 w, u64 w32, u32 c60, u32 c64) {
  u64 r;
  asm("{\n\t"
      ".reg .u64 h, l, m, p;\n\t"
      ".reg .u32 y0, y1, w0, w1, v0, v1, l0, l1, m0, m1, h0, h1, s0, t, u, sm, tl;\n\t"
      "mov.b64 {y0, y1}, %1;\n\t"
      "mov.b64 {w0, w1}, %2;\n\t"
      "mov.b64 {v0, v1}, %3;\n\t"
      "mul.wide.u32 h, y1, v1;\n\t"
      "mad.wide.u32 h, y0, w1, h;\n\t"
      "mul.wide.u32 l, y0, w0;\n\t"
      "mul.wide.u32 m, y1, v0;\n\t"
      "mov.b64 {l0, l1}, l;\n\t"
      "mov.b64 {m0, m1}, m;\n\t"
      "mov.b64 {h0, h1}, h;\n\t"
      "add.cc.u32 s0, l0, m0;\n\t"
      "addc.cc.u32 t, l1, m1;\n\t"
      "addc.u32 u, h1, 0;\n\t"
      "add.cc.u32 t, t, h0;\n\t"
      "addc.u32 u, u, 0;\n\t"
      "shr.u32 sm, t, 28;\n\t"
      "and.b32 tl, t, 0x0FFFFFFF;\n\t"
      "mad.lo.cc.u32 s0, sm, %4, s0;\n\t"
      "addc.u32 tl, tl, 0;\n\t"
      "mov.b64 p, {s0, tl};\n\t"
      "mad.wide.u32 %0, u, %5, p;\n\t"
      "}"
      : "=l"(r)
      : "l"(y), "l"(w), "l"(w32), "r"(c60), "r"(c64));
  return r;
}

// The same product in plain C (the reference form of the PTX above; the
// multiply probe times both).
__device__ __forceinline__ u64 mul_fold_c(u64 y, u64 w, u64 w32, u32 c60, u32 c64) {
  const u32 y0 = (u32)y, y1 = (u32)(y >> 32);
  // S = y0 wl + y1 w32l + 2^32 (y0 wh + y1 w32h)   (l, h: low and high 32-bit halves)
  const u64 p1 = (u64)y1 * (u32)w32;                           // y1 w32l
  const u64 p0 = (u64)y0 * (u32)w + (u32)p1;                   // y0 wl + lo(p1) < 2^64 - 2^32
  u64 m = (u64)y1 * (u32)(w32 >> 32) + (p1 >> 32);             // < 2^60 + 2^32
  m = (u64)y0 * (u32)(w >> 32) + m;                            // < 2^61 + 2^32
  m += p0 >> 32;                                               // S = m 2^32 + lo(p0), m < 2^61 + 2^33
  const u32 ml = (u32)m;
  const u64 t = (u64)(ml >> 28) * c60 + (((u64)(ml & 0x0FFFFFFFu) << 32) | (u32)p0);   // sl + sm c60
  return (u64)(u32)(m >> 32) * c64 + t;                                                 // + sh c64
}

// v mod q, lazily: any v < 2^64 -> (v mod 2^60) + (v >> 60) c60 < 2^60 + 2^32 (< 2 q).
// (v >> 60) c60 < 2^32 (c60 < 2^28): a 32-bit multiply-add with carry, not a
// 32x32->64 one (which holds the multiply pipe twice as long).
__device__ __forceinline__ u64 fold60(u64 v, u32 c60) {
  u64 r;
  asm("{\n\t"
      ".reg .u32 v0, v1, s, h;\n\t"
      "mov.b64 {v0, v1}, %1;\n\t"
      "shr.u32 s, v1, 28;\n\t"
      "and.b32 h, v1, 0x0FFFFFFF;\n\t"
      "mad.lo.cc.u32 v0, s, %2, v0;\n\t"
      "addc.u32 h, h, 0;\n\t"
      "mov.b64 %0, {v0, h};\n\t"
      "}"
      : "=l"(r)
      : "l"(v), "r"(c60));
  return r;
}

// Cooley-Tukey butterfly with a lazy pseudo-Mersenne product: x, y < B q ->
// x + w y < (B + 1.13) q, x - w y + 2 q < (B + 2) q (no correction step).
__device__ __forceinline__ void ct_fold(u64& x, u64& y, const ulonglong2 w, u32 c60, u32 c64, u64 q2) {
  const u64 t = mul_fold(y, w.x, w.y, c60, c64);
  y = x + q2 - t;
  x = x + t;
}

// Gentleman-Sande butterfly: x, y < B q <= cq, cq + B q < 2^64 ->
// x + y < 2 B q, (x - y + cq) w < 1.13 q.
__device__ __forceinline__ void gs_fold(u64& x, u64& y, const ulonglong2 w, u32 c60, u32 c64, u64 cq) {
  const u64 d = x + cq - y;
  x = x + y;
  y = mul_fold(d, w.x, w.y, c60, c64);
}

// [0, 8q) -> [0, q)
__device__ __forceinline__ u64 canon8(u64 x, u64 q) {
  return csub(csub_s(csub_s(x, 4 * q), 2 * q), q);
}

// [0, 4q) -> [0, q)
__device__ __forceinline__ u64 canon4(u64 x, u64 q, u64 q2) {
  x = x >= q2 ? x - q2 : x;
  return x >= q ? x - q : x;
}

// ------------------------------------------------------------------ Philox4x64-10
// Salmon et al., SC'11: two 64x64->128 products per round on counter words 0
// and 2, high halves mixed with words 1, 3 and the round key; Weyl key schedule.
struct Philox4 {
  u64 v[4];
};

__device__ __forceinline__ Philox4 philox4x64(u64 c0, u64 c1, u64 c2, u64 c3, u64 k0, u64 k1) {
  const u64 M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const u64 W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    u64 lo0 = M0 * c0, hi0 = mulhi64(M0, c0);
    u64 lo1 = M1 * c2, hi1 = mulhi64(M1, c2);
    u64 n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  Philox4 o;
  o.v[0] = c0;
  o.v[1] = c1;
  o.v[2] = c2;
  o.v[3] = c3;
  return o;
}

// Stream domains (the second key word).
#define PENCIL_DOM_SECRET 1ull
#define PENCIL_DOM_A 2ull
#define PENCIL_DOM_E 3ull
#define PENCIL_DOM_MASK 4ull
#define PENCIL_DOM_MASK_PAD 5ull
#define PENCIL_DOM_FLOOD 6ull
#define PENCIL_DOM_PK_A 7ull    // public key's a
#define PENCIL_DOM_PK_E 8ull    // public key's error
#define PENCIL_DOM_PK_U 9ull    // public-key encryption's ternary u
#define PENCIL_DOM_PK_E2 10ull  // public-key encryption's e2 (its e1 is PENCIL_DOM_E)

__device__ __forceinline__ u64 philox_word(const Philox4& w, int i) {
  return i == 0 ? w.v[0] : i == 1 ? w.v[1] : i == 2 ? w.v[2] : w.v[3];
}

// Uniform residue mod q_j of coefficient `coef` from its 64-bit Philox word w
// (the encryption mask a, the public key's a): w is accepted when w <= a_max
// (below the largest multiple of q_j under 2^64) and reduced; a rejected word is
// replaced by word 0 of the block at counter (coef, ct, limb, r), r = 1, 2, ...
// (probability below 2^-32 per word for the primes used; the loop stops after 64
// replacements, which for primes above 2^40 never happens in practice).
__device__ __forceinline__ u64 uniform_mod_q(u64 w, int coef, int ct, int limb, u64 seed, u64 dom,
                                             const LimbConst& lc) {
  for (u64 r = 1; w > lc.a_max && r <= 64; ++r) w = philox4x64((u64)coef, (u64)ct, (u64)limb, r, seed, dom).v[0];
  return reduce64(w, lc);
}

// ------------------------------------------------------------------ packing gathers
__device__ __forceinline__ u64 gather(const Packing& pk, const Accessor& ac, int idx, int e) {
  u64 ent = __ldg(pk.tab + e);
  if (ent == PENCIL_TAB_NONE) return 0;
  int4 o = __ldg(pk.org + idx);
  int a = o.x + (int)(ent & 0xffff);
  int b = o.y + (int)((ent >> 16) & 0xffff);
  int r = o.z + (int)((ent >> 32) & 0xffff);
  int s = o.w + (int)(ent >> 48);
  if (a >= pk.bound.x || b >= pk.bound.y || r >= pk.bound.z || s >= pk.bound.w) return 0;
  r -= ac.pr;
  s -= ac.ps;
  if ((unsigned)r >= (unsigned)ac.hr || (unsigned)s >= (unsigned)ac.wr) return 0;
  return __ldg(ac.ptr + ac.base + a * ac.s0 + b * ac.s1 + r * ac.s2 + s * ac.s3);
}

// Decryption's CRT step: with y_j = x_j (q/q_j)^{-1} mod q_j,
//   t x / q = sum_j y_j t / q_j - v t  (v integer),
// so round(t x / q) mod t = round(sum_j y_j th_j / 2^128) mod t with
// th_j = floor(2^(128 + t_bits) / q_j).  The sum is kept as a 128-bit window
// (64 integer bits, 64 fraction bits); truncation error < L * 2^-63.
struct CrtSum {
  u64 lo, hi;
};
__device__ __forceinline__ void crt_add(CrtSum& s, u64 y, const LimbConst& lc) {
  const u64 a_hi = __umul64hi(y, lc.th_lo);
  const u64 b_lo = y * lc.th_hi;
  const u64 b_hi = __umul64hi(y, lc.th_hi);
  const u64 w_lo = b_lo + a_hi;
  const u64 w_hi = b_hi + (w_lo < b_lo ? 1ull : 0ull);
  s.lo += w_lo;
  s.hi += w_hi + (s.lo < w_lo ? 1ull : 0ull);
}
// The rounded value mod t; with `check`, flags (status bit 0) a fraction within
// 1/4 of one half (noise too close to the decryption bound).
__device__ __forceinline__ u64 crt_round(const CrtSum& s, u64 t_mask, int check, int* status) {
  if (check) {
    const i64 frac = (i64)s.lo;   // signed distance to the nearest integer, units of 2^-64
    const u64 mag = frac < 0 ? (u64)(-frac) : (u64)frac;
    if (mag >= (1ull << 62)) atomicOr(status, 1);
  }
  const u64 r_lo = s.lo + (1ull << 63);
  const u64 r_hi = s.hi + (r_lo < s.lo ? 1ull : 0ull);
  return r_hi & t_mask;
}

// Output flat index of coefficient e of output polynomial idx, or -1.
__device__ __forceinline__ i64 out_index(const Packing& pk, const Accessor& ac, int idx, int e) {
  u64 ent = __ldg(pk.tab + e);
  if (ent == PENCIL_TAB_NONE) return -1;
  int4 o = __ldg(pk.org + idx);
  int a = o.x + (int)(ent & 0xffff);
  int b = o.y + (int)((ent >> 16) & 0xffff);
  int r = o.z + (int)((ent >> 32) & 0xffff);
  int s = o.w + (int)(ent >> 48);
  if (a >= pk.bound.x || b >= pk.bound.y || r >= pk.bound.z || s >= pk.bound.w) return -1;
  return ac.base + a * ac.s0 + b * ac.s1 + r * ac.s2 + s * ac.s3;
}
