// C ABI of the Pencil HE hot path (declared in include/pencil_he.h).
//
// Host side: BFV/RNS parameter generation (Sec. 2.2, Sec. 5), the planner
// that partitions a layer into polynomial blocks (Appendix A), the packing
// index tables, argument validation, and the launch sequences of Alg. 1 and
// Alg. 2.  Every launch goes to the caller's stream; nothing here allocates
// on the hot path (contexts, keys and plans own their device tables).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/pencil_he.h"
#include "kernels.h"

using namespace pencil;
typedef unsigned __int128 u128;

// ================================================================== number theory (host)
static u64 mulmod(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

static u64 powmod(u64 a, u64 e, u64 m) {
  u64 r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod(r, a, m);
    a = mulmod(a, a, m);
    e >>= 1;
  }
  return r;
}

// Deterministic Miller-Rabin for 64-bit n (bases = first 12 primes).
static bool is_prime64(u64 n) {
  static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 p : bases) {
    if (n % p == 0) return n == p;
  }
  u64 d = n - 1;
  int r = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++r;
  }
  for (u64 a : bases) {
    u64 x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < r; ++i) {
      x = mulmod(x, x, n);
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

// Largest `count` primes q < 2^bits with q = 1 mod two_n, descending.
static bool find_primes(int bits, int count, u64 two_n, std::vector<u64>& out) {
  u64 top = (bits == 64) ? ~0ull : ((1ull << bits) - 1);
  u64 q = top / two_n * two_n + 1;
  if (q > top) q -= two_n;
  while ((int)out.size() < count) {
    if (q <= two_n) return false;
    if (is_prime64(q)) out.push_back(q);
    q -= two_n;
  }
  return true;
}

// Numerically smallest element of multiplicative order exactly two_n mod q.
static u64 min_root_2n(u64 q, u64 two_n) {
  const u64 half = two_n / 2, ex = (q - 1) / two_n;
  u64 psi0 = 0;
  for (u64 g = 2;; ++g) {
    psi0 = powmod(g, ex, q);
    if (powmod(psi0, half, q) == q - 1) break;
  }
  const u64 sq = mulmod(psi0, psi0, q);
  u64 cur = psi0, best = psi0;
  for (u64 k = 1; k < half; ++k) {
    cur = mulmod(cur, sq, q);
    if (cur < best) best = cur;
  }
  return best;
}

static u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

static unsigned brv(unsigned x, int bits) {
  unsigned r = 0;
  for (int i = 0; i < bits; ++i) {
    r = (r << 1) | (x & 1);
    x >>= 1;
  }
  return r;
}

// floor(2^e / q) as a 128-bit value (requires the result < 2^128).
static u128 floor_pow2_div(int e, u64 q) {
  u128 quo = 0;
  u128 rem = 0;
  for (int bit = e; bit >= 0; --bit) {
    rem = (rem << 1) | (bit == e ? 1 : 0);
    quo <<= 1;
    if (rem >= q) {
      rem -= q;
      quo |= 1;
    }
  }
  return quo;
}

// floor(prod(q) / 2^t_bits) mod p, prod(q) held as little-endian 64-bit words.
static u64 delta_mod(const std::vector<u64>& qs, int t_bits, u64 p) {
  std::vector<u64> w(qs.size() + 1, 0);
  w[0] = 1;
  for (u64 q : qs) {
    u128 carry = 0;
    for (size_t i = 0; i < w.size(); ++i) {
      u128 v = (u128)w[i] * q + carry;
      w[i] = (u64)v;
      carry = v >> 64;
    }
  }
  // shift right by t_bits (< 64)
  for (size_t i = 0; i < w.size(); ++i) {
    u64 hi = (i + 1 < w.size()) ? w[i + 1] : 0;
    w[i] = (t_bits == 0) ? w[i] : ((w[i] >> t_bits) | (hi << (64 - t_bits)));
  }
  u64 r = 0;
  for (size_t i = w.size(); i-- > 0;) r = (u64)((((u128)r << 64) | w[i]) % p);
  return r;
}

// ================================================================== handles
struct ProfRec {
  int kernel;
  cudaEvent_t a, b;
};

struct PencilCtx {
  bool prof_on = false;
  std::vector<ProfRec> prof;      // recorded launches
  std::vector<cudaEvent_t> pool;  // spare events
  PencilParams params;
  int device;
  int n;
  std::vector<u64> primes, psis;
  DevCtx dev;
  ulonglong2* tw_fwd = nullptr;
  ulonglong2* tw_inv = nullptr;
  ulonglong2* tw_fwd_f = nullptr;   // fold tables (w, w 2^32 mod q), when every prime allows them
  ulonglong2* tw_inv_f = nullptr;
  int* status = nullptr;
  void* noalloc_addr = nullptr;     // device address of encrypt_share_noalloc's static scratch (this context's)
};

struct PencilSecretKey {
  PencilCtx* ctx;
  ulonglong2* sk = nullptr;
};

struct PencilPublicKey {
  PencilCtx* ctx;
  ulonglong2* key = nullptr;   // [2][L][N] (value, Shoup companion), then N bytes of scratch
};

struct Geom {
  int B, Ci, Co, H, W, KH, KW;
  int Ho() const { return H - KH + 1; }
  int Wo() const { return W - KW + 1; }
};

struct Counts {
  int MB, MTH, MTW, KC, KTH, KTW, NC;
  long long M() const { return (long long)MB * MTH * MTW; }
  long long K() const { return (long long)KC * KTH * KTW; }
};

struct PencilPlan {
  PencilCtx* ctx;
  PencilLayerDesc layer;
  int role;
  Geom g;
  PencilPartition part;
  Counts c;
  long long ct_in, pt, ct_out, products, out_elems;
  Accessor acc_v, acc_w, acc_y;  // ptr filled per call
  long long hw;                  // output spatial size (bias broadcast)
  int co_out;                    // output channel count seen by the bias
  u64* d_tab = nullptr;          // [3][N]: v, w, y tables
  int4* d_org = nullptr;         // origins: v [ct_in], w [pt], y [ct_out]
  Packing pk_v, pk_w, pk_y;
  long long ws_encrypt, ws_forward, ws_backward, ws_decrypt, ws_encrypt_pk;
  // A slice (pencil_plan_slice) covers output rows m in [m_first, m_first + m_count)
  // of its parent and shares the parent's tables; a full plan covers [0, M).
  long long m_first = 0, m_count = 0;
  const PencilPlan* parent = nullptr;
  // input polynomials [in_first, in_first + in_count), output [out_first, out_first + out_count)
  long long in_first() const { return m_first * c.K(); }
  long long in_count() const { return m_count * c.K(); }
  long long out_first() const { return m_first * c.NC; }
  long long out_count() const { return m_count * c.NC; }
};

static int cdiv(int a, int b) { return (a + b - 1) / b; }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

static cudaEvent_t prof_event(PencilCtx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records CUDA events around the launches made while it lives (when enabled).
struct ProfScope {
  PencilCtx* c;
  int k;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(PencilCtx* ctx, int kernel, cudaStream_t st) : c(ctx), k(kernel), s(st) {
    if (c->prof_on) {
      a = prof_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, s);
      c->prof.push_back(ProfRec{k, a, b});
    }
  }
};
#define PROF(ctx, kernel, stream) ProfScope _prof_##kernel(ctx, kernel, stream)

#define CUDA_TRY(x)                               \
  do {                                            \
    cudaError_t _e = (x);                         \
    if (_e != cudaSuccess) {                      \
      fprintf(stderr, "pencil: %s -> %s\n", #x, cudaGetErrorString(_e)); \
      return PENCIL_E_CUDA;                       \
    }                                             \
  } while (0)

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// ================================================================== context
extern "C" int pencil_ctx_create(const PencilParams* params, int device, PencilCtx** out) {
  if (!params || !out) return PENCIL_E_ARG;
  *out = nullptr;
  const PencilParams& p = *params;
  if (p.log_n < 12 || p.log_n > 14) return PENCIL_E_PARAMS;
  if (p.num_primes < 1 || p.num_primes > PENCIL_MAX_LIMBS) return PENCIL_E_PARAMS;
  if (p.prime_bits < 30 || p.prime_bits > 60) return PENCIL_E_PARAMS;
  if (p.t_bits < 8 || p.t_bits > 60) return PENCIL_E_PARAMS;
  const int n = 1 << p.log_n;
  std::vector<u64> qs;
  if (!find_primes(p.prime_bits, p.num_primes, 2ull * n, qs)) return PENCIL_E_PARAMS;
  // q must leave room for t: Delta >= 1 and t < every q_i
  for (u64 q : qs)
    if (p.t_bits >= 63 || q <= (1ull << p.t_bits)) return PENCIL_E_PARAMS;

  PencilCtx* ctx = new (std::nothrow) PencilCtx();
  if (!ctx) return PENCIL_E_CUDA;
  ctx->params = p;
  ctx->device = device;
  ctx->n = n;
  ctx->primes = qs;
  DeviceGuard guard(device);

  DevCtx& d = ctx->dev;
  memset(&d, 0, sizeof(d));
  d.log_n = p.log_n;
  d.ntt_loge = p.log_n <= 13 ? 4 : 5;   // Shoup engine: radix 2^4 (two CTAs per SM) up to N = 8192
  d.n = n;
  d.L = p.num_primes;
  d.t_bits = p.t_bits;
  d.t_mask = (1ull << p.t_bits) - 1;
  std::vector<ulonglong2> tf((size_t)d.L * n), ti((size_t)d.L * n);
  // pseudo-Mersenne fold butterflies need q_j = 2^60 - c with c < 2^24 for every limb
  bool fold_ok = true;
  for (u64 q : qs) fold_ok = fold_ok && q < (1ull << 60) && q > (1ull << 60) - (1ull << 24);
  std::vector<ulonglong2> tff(fold_ok ? (size_t)d.L * n : 0), tif(fold_ok ? (size_t)d.L * n : 0);
  for (int j = 0; j < d.L; ++j) {
    const u64 q = qs[j];
    const u64 psi = min_root_2n(q, 2ull * n);
    ctx->psis.push_back(psi);
    const u64 psi_inv = powmod(psi, q - 2, q);
    for (int k = 0; k < n; ++k) {
      const unsigned r = brv((unsigned)k, p.log_n);
      const u64 w = powmod(psi, r, q), wi = powmod(psi_inv, r, q);
      tf[(size_t)j * n + k] = make_ulonglong2(w, shoup(w, q));
      ti[(size_t)j * n + k] = make_ulonglong2(wi, shoup(wi, q));
      if (fold_ok) {
        tff[(size_t)j * n + k] = make_ulonglong2(w, (u64)((((u128)w) << 32) % q));
        tif[(size_t)j * n + k] = make_ulonglong2(wi, (u64)((((u128)wi) << 32) % q));
      }
    }
    LimbConst& lc = d.limb[j];
    lc.q = q;
    lc.mu = (u64)((((u128)1) << 64) / q);
    lc.r64 = (u64)((((u128)1) << 64) % q);
    lc.r64s = shoup(lc.r64, q);
    lc.ninv = powmod((u64)n, q - 2, q);
    lc.ninvs = shoup(lc.ninv, q);
    lc.delta = delta_mod(qs, p.t_bits, q);
    lc.deltas = shoup(lc.delta, q);
    u64 qt = 1;
    for (int i = 0; i < d.L; ++i)
      if (i != j) qt = mulmod(qt, qs[i] % q, q);
    lc.qtil = powmod(qt, q - 2, q);
    lc.qtils = shoup(lc.qtil, q);
    const u128 th = floor_pow2_div(128 + p.t_bits, q);
    lc.th_hi = (u64)(th >> 64);
    lc.th_lo = (u64)th;
    lc.c60 = (u64)((((u128)1) << 60) % q);
    lc.c64 = (u64)((((u128)1) << 64) % q);
    lc.nqtil = mulmod(lc.ninv, lc.qtil, q);
    lc.nqtils = shoup(lc.nqtil, q);
    lc.a_max = (u64)((((u128)1) << 64) / q * q - 1);
    {
      const u64 w1 = powmod(psi_inv, brv(1u, p.log_n), q);   // the last inverse stage's twiddle
      const u64 ks[2] = {lc.ninv, lc.nqtil};
      u64* dst[2] = {lc.sc_ninv, lc.sc_nqtil};
      for (int i = 0; i < 2; ++i) {
        const u64 wk = mulmod(w1, ks[i], q);
        dst[i][0] = ks[i];
        dst[i][1] = (u64)((((u128)ks[i]) << 32) % q);
        dst[i][2] = wk;
        dst[i][3] = (u64)((((u128)wk) << 32) % q);
      }
    }
  }
  {   // q_total mod t (t = 2^t_bits divides 2^64: the product of the primes mod 2^64, masked)
    u64 qt = 1;
    for (int j = 0; j < d.L; ++j) qt *= qs[j];
    d.q_mod_t = qt & d.t_mask;
  }
  d.mac_nt = 4;
  d.mac_staging = 1;   // measured: bulk copies by a producer warp, 4 columns per thread
  d.mac_split = 1;
  for (int j = 0; j < d.L; ++j)
    if (qs[j] >= (1ull << 60) || qs[j] <= (1ull << 59) + (1ull << 33) || d.limb[j].c60 >= (1ull << 28) ||
        d.limb[j].c64 >= (1ull << 28))
      d.mac_split = 0;   // (q > 2^59 + 2^33: the accumulator's final value, below 2^60 + 2^33, is below 2 q)
  cudaError_t e1 = cudaMalloc(&ctx->tw_fwd, tf.size() * sizeof(ulonglong2));
  cudaError_t e2 = cudaMalloc(&ctx->tw_inv, ti.size() * sizeof(ulonglong2));
  cudaError_t e3 = cudaMalloc(&ctx->status, sizeof(int));
  cudaError_t e4 = fold_ok ? cudaMalloc(&ctx->tw_fwd_f, tff.size() * sizeof(ulonglong2)) : cudaSuccess;
  cudaError_t e5 = fold_ok ? cudaMalloc(&ctx->tw_inv_f, tif.size() * sizeof(ulonglong2)) : cudaSuccess;
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess || e5 != cudaSuccess) {
    pencil_ctx_destroy(ctx);
    return PENCIL_E_CUDA;
  }
  if (cudaMemcpy(ctx->tw_fwd, tf.data(), tf.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->tw_inv, ti.data(), ti.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice) != cudaSuccess ||
      (fold_ok && cudaMemcpy(ctx->tw_fwd_f, tff.data(), tff.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice) !=
                      cudaSuccess) ||
      (fold_ok && cudaMemcpy(ctx->tw_inv_f, tif.data(), tif.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice) !=
                      cudaSuccess) ||
      cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess || upload_cdt() != cudaSuccess) {
    pencil_ctx_destroy(ctx);
    return PENCIL_E_CUDA;
  }
  d.tw_fwd = ctx->tw_fwd;
  d.tw_inv = ctx->tw_inv;
  d.tw_fwd_f = ctx->tw_fwd_f;
  d.tw_inv_f = ctx->tw_inv_f;
  d.ntt_arith = fold_ok ? 1 : 0;
  if (fold_ok) d.ntt_loge = 4;   // fold engine: radix 2^4 at every N (N = 16384: 1024-thread CTAs, measured faster)
  d.status = ctx->status;
  *out = ctx;
  return PENCIL_OK;
}

extern "C" int pencil_ctx_destroy(PencilCtx* ctx) {
  if (!ctx) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  for (ProfRec& r : ctx->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  cudaFree(ctx->tw_fwd);
  cudaFree(ctx->tw_inv);
  cudaFree(ctx->tw_fwd_f);
  cudaFree(ctx->tw_inv_f);
  cudaFree(ctx->status);
  delete ctx;
  return PENCIL_OK;
}

extern "C" int pencil_ctx_primes(const PencilCtx* ctx, uint64_t* primes, uint64_t* psis) {
  if (!ctx || !primes || !psis) return PENCIL_E_ARG;
  for (size_t j = 0; j < ctx->primes.size(); ++j) {
    primes[j] = ctx->primes[j];
    psis[j] = ctx->psis[j];
  }
  return PENCIL_OK;
}

extern "C" int pencil_ctx_tune(PencilCtx* ctx, int32_t knob, int32_t value) {
  if (!ctx) return PENCIL_E_ARG;
  if (knob == PENCIL_TUNE_NTT_LOG_RADIX) {
    if (value != 4 && value != 5) return PENCIL_E_ARG;
    ctx->dev.ntt_loge = value;
    return PENCIL_OK;
  }
  if (knob == PENCIL_TUNE_MAC_COLUMNS) {
    if (value != 0 && value != 2 && value != 4 && value != 8) return PENCIL_E_ARG;
    ctx->dev.mac_nt = value;
    return PENCIL_OK;
  }
  if (knob == PENCIL_TUNE_MAC_STAGING) {
    if (value != 0 && value != 1) return PENCIL_E_ARG;
    ctx->dev.mac_staging = value;
    return PENCIL_OK;
  }
  if (knob == PENCIL_TUNE_NTT_ARITH) {
    if (value != 0 && value != 1) return PENCIL_E_ARG;
    if (value == 1 && !ctx->tw_fwd_f) return PENCIL_E_PARAMS;   // some prime is not 2^60 - c, c < 2^24
    ctx->dev.ntt_arith = value;
    return PENCIL_OK;
  }
  return PENCIL_E_ARG;
}

extern "C" int pencil_ctx_flooding(PencilCtx* ctx, int32_t bits) {
  if (!ctx) return PENCIL_E_ARG;
  if (bits < 0 || bits > 62) return PENCIL_E_ARG;
  // the flooded noise must stay far below Delta / 2: log2 q_total - t_bits - bits >= 8
  int qbits = 0;
  for (u64 q : ctx->primes) qbits += 64 - __builtin_clzll(q);
  if (bits > 0 && qbits - 1 - ctx->dev.t_bits - bits < 8) return PENCIL_E_PARAMS;
  ctx->dev.flood_bits = bits;
  return PENCIL_OK;
}

extern "C" int pencil_ctx_get_tune(const PencilCtx* ctx, int32_t knob, int32_t* value) {
  if (!ctx || !value) return PENCIL_E_ARG;
  if (knob == PENCIL_TUNE_NTT_LOG_RADIX) {
    *value = ctx->dev.ntt_loge;
    return PENCIL_OK;
  }
  if (knob == PENCIL_TUNE_MAC_COLUMNS) {
    *value = ctx->dev.mac_nt;
    return PENCIL_OK;
  }
  if (knob == PENCIL_TUNE_NTT_ARITH) {
    *value = ctx->dev.ntt_arith;
    return PENCIL_OK;
  }
  if (knob == PENCIL_TUNE_MAC_STAGING) {
    *value = ctx->dev.mac_staging;
    return PENCIL_OK;
  }
  return PENCIL_E_ARG;
}

extern "C" int pencil_sync_status(PencilCtx* ctx, int32_t* status) {
  if (!ctx || !status) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  int v = 0;
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(&v, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(ctx->status, 0, sizeof(int)));
  // a timed-out wait leaves outputs unwritten, which then also fail the noise check
  *status = (v & 2) ? PENCIL_E_TIMEOUT : (v & 1) ? PENCIL_E_NOISE : PENCIL_OK;
  return PENCIL_OK;
}

// ================================================================== keys
extern "C" int pencil_keygen(PencilCtx* ctx, uint64_t seed, PencilSecretKey** out, void* stream) {
  if (!ctx || !out) return PENCIL_E_ARG;
  *out = nullptr;
  DeviceGuard guard(ctx->device);
  PencilSecretKey* sk = new (std::nothrow) PencilSecretKey();
  if (!sk) return PENCIL_E_CUDA;
  sk->ctx = ctx;
  if (cudaMalloc(&sk->sk, (size_t)ctx->dev.L * ctx->n * sizeof(ulonglong2)) != cudaSuccess) {
    delete sk;
    return PENCIL_E_CUDA;
  }
  ModeKeygen::Params P;
  P.seed = seed;
  P.sk = sk->sk;
  if (ntt<ModeKeygen, false>(ctx->dev, P, 1, (cudaStream_t)stream) != cudaSuccess) {
    pencil_sk_destroy(sk);
    return PENCIL_E_CUDA;
  }
  *out = sk;
  return PENCIL_OK;
}

extern "C" int pencil_sk_destroy(PencilSecretKey* sk) {
  if (!sk) return PENCIL_E_ARG;
  DeviceGuard guard(sk->ctx->device);
  cudaFree(sk->sk);
  delete sk;
  return PENCIL_OK;
}

extern "C" int pencil_pk_keygen(PencilCtx* ctx, const PencilSecretKey* sk, uint64_t seed, PencilPublicKey** out,
                                void* stream) {
  if (!ctx || !sk || !out || sk->ctx != ctx) return PENCIL_E_ARG;
  *out = nullptr;
  DeviceGuard guard(ctx->device);
  PencilPublicKey* pk = new (std::nothrow) PencilPublicKey();
  if (!pk) return PENCIL_E_CUDA;
  pk->ctx = ctx;
  const size_t key_bytes = 2ull * ctx->dev.L * ctx->n * sizeof(ulonglong2);
  if (cudaMalloc(&pk->key, key_bytes + ctx->n) != cudaSuccess) {
    delete pk;
    return PENCIL_E_CUDA;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  int8_t* err = reinterpret_cast<int8_t*>(pk->key) + key_bytes;
  ModePkKeygen::Params P;
  P.err = err;
  P.sk = sk->sk;
  P.key = pk->key;
  P.seed = seed;
  if (launch_sample_err(seed, 0, 1, ctx->n, err, s, PENCIL_DOM_PK_E) != cudaSuccess ||
      ntt<ModePkKeygen, false>(ctx->dev, P, 1, s) != cudaSuccess) {
    pencil_pk_destroy(pk);
    return PENCIL_E_CUDA;
  }
  *out = pk;
  return PENCIL_OK;
}

extern "C" int pencil_pk_destroy(PencilPublicKey* pk) {
  if (!pk) return PENCIL_E_ARG;
  DeviceGuard guard(pk->ctx->device);
  cudaFree(pk->key);
  delete pk;
  return PENCIL_OK;
}

// ================================================================== plans
static Accessor make_acc(i64 s0, i64 s1, i64 s2, i64 s3, int pr, int ps, int hr, int wr, i64 base = 0) {
  Accessor a;
  a.ptr = nullptr;
  a.base = base;
  a.s0 = s0;
  a.s1 = s1;
  a.s2 = s2;
  a.s3 = s3;
  a.pr = pr;
  a.ps = ps;
  a.hr = hr;
  a.wr = wr;
  return a;
}

// Maps the user's tensors of `role` onto one correlation
//   y[a, o, i, j] = sum_{c, u, v} Wt[o, c, u, v] * V[a, c, i + u, j + v].
static int role_setup(const PencilLayerDesc& L, int role, PencilPlan& P) {
  const bool fc = L.kind == PENCIL_FC;
  const i64 B = L.batch, ni = L.c_in, no = L.c_out;
  if (fc) {
    P.hw = 1;
    if (role == PENCIL_ROLE_FWD) {
      P.g = Geom{(int)B, (int)ni, (int)no, 1, 1, 1, 1};
      P.acc_v = make_acc(ni, 1, 0, 0, 0, 0, 1, 1);
      P.acc_w = make_acc(ni, 1, 0, 0, 0, 0, 1, 1);
      P.acc_y = make_acc(no, 1, 0, 0, 0, 0, 1, 1);
      P.co_out = (int)no;
    } else if (role == PENCIL_ROLE_DGRAD) {
      P.g = Geom{(int)B, (int)no, (int)ni, 1, 1, 1, 1};
      P.acc_v = make_acc(no, 1, 0, 0, 0, 0, 1, 1);   // gY [B][n_o]
      P.acc_w = make_acc(1, ni, 0, 0, 0, 0, 1, 1);   // Wt[i, o] = W[o, i]
      P.acc_y = make_acc(ni, 1, 0, 0, 0, 0, 1, 1);   // gX [B][n_i]
      P.co_out = (int)ni;
    } else {
      P.g = Geom{(int)ni, (int)B, (int)no, 1, 1, 1, 1};
      P.acc_v = make_acc(1, ni, 0, 0, 0, 0, 1, 1);   // V[i, b] = X[b, i]
      P.acc_w = make_acc(1, no, 0, 0, 0, 0, 1, 1);   // Wt[o, b] = gY[b, o]
      P.acc_y = make_acc(1, ni, 0, 0, 0, 0, 1, 1);   // y[i, o] = gW[o, i]
      P.co_out = (int)no;
    }
    return PENCIL_OK;
  }
  const i64 h = L.height, w = L.width, s = L.kernel, p = L.pad;
  const i64 ho = h + 2 * p - s + 1, wo = w + 2 * p - s + 1;
  const i64 Ci = ni, Co = no;
  if (role == PENCIL_ROLE_FWD) {
    P.g = Geom{(int)B, (int)Ci, (int)Co, (int)(h + 2 * p), (int)(w + 2 * p), (int)s, (int)s};
    P.acc_v = make_acc(Ci * h * w, h * w, w, 1, (int)p, (int)p, (int)h, (int)w);
    P.acc_w = make_acc(Ci * s * s, s * s, s, 1, 0, 0, (int)s, (int)s);
    P.acc_y = make_acc(Co * ho * wo, ho * wo, wo, 1, 0, 0, (int)ho, (int)wo);
    P.hw = ho * wo;
    P.co_out = (int)Co;
  } else if (role == PENCIL_ROLE_DGRAD) {
    const i64 e = s - 1 - p;
    P.g = Geom{(int)B, (int)Co, (int)Ci, (int)(ho + 2 * e), (int)(wo + 2 * e), (int)s, (int)s};
    P.acc_v = make_acc(Co * ho * wo, ho * wo, wo, 1, (int)e, (int)e, (int)ho, (int)wo);
    // Wt[c, o, u, v] = W[o, c, s-1-u, s-1-v]
    P.acc_w = make_acc(s * s, Ci * s * s, -s, -1, 0, 0, (int)s, (int)s, (s - 1) * s + (s - 1));
    P.acc_y = make_acc(Ci * h * w, h * w, w, 1, 0, 0, (int)h, (int)w);
    P.hw = h * w;
    P.co_out = (int)Ci;
  } else {
    P.g = Geom{(int)Ci, (int)B, (int)Co, (int)(h + 2 * p), (int)(w + 2 * p), (int)ho, (int)wo};
    P.acc_v = make_acc(h * w, Ci * h * w, w, 1, (int)p, (int)p, (int)h, (int)w);   // V[c, b] = X[b, c]
    P.acc_w = make_acc(ho * wo, Co * ho * wo, wo, 1, 0, 0, (int)ho, (int)wo);      // Wt[o, b] = gY[b, o]
    P.acc_y = make_acc(s * s, Ci * s * s, s, 1, 0, 0, (int)s, (int)s);             // y[c, o] = gW[o, c]
    P.hw = s * s;
    P.co_out = (int)Co;
  }
  return PENCIL_OK;
}

static Counts counts_of(const Geom& g, const PencilPartition& p) {
  return Counts{cdiv(g.B, p.bb), cdiv(g.Ho(), p.th), cdiv(g.Wo(), p.tw), cdiv(g.Ci, p.cib),
                cdiv(g.KH, p.kth), cdiv(g.KW, p.ktw), cdiv(g.Co, p.cob)};
}

static bool part_valid(const Geom& g, const PencilPartition& p, int n) {
  if (p.bb < 1 || p.cib < 1 || p.cob < 1 || p.th < 1 || p.tw < 1 || p.kth < 1 || p.ktw < 1) return false;
  if (p.bb > g.B || p.cib > g.Ci || p.cob > g.Co || p.th > g.Ho() || p.tw > g.Wo() || p.kth > g.KH ||
      p.ktw > g.KW)
    return false;
  const long long hw = (long long)(p.th + p.kth - 1) * (p.tw + p.ktw - 1);
  return (long long)p.bb * p.cob * p.cib * hw <= n;
}

// Distinct values of ceil(x / d), d = 1..x (descending).
static std::vector<int> ceil_divs(int x) {
  std::vector<int> v;
  for (int d = 1; d <= x; ++d) {
    const int c = cdiv(x, d);
    if (v.empty() || v.back() != c) v.push_back(c);
  }
  return v;
}

// Cost model of one call sequence of the role, in 32-bit multiply units:
// limb-NTTs at 10 * (N/2) log2 N, ct x pt slot products at 8 per 64x64->128
// multiply-add, bytes at 3 per byte (the multiply/HBM balance of the GPU).
static double plan_cost(const Geom& g, const PencilPartition& p, int role, int n, int log_n, int L) {
  const Counts c = counts_of(g, p);
  const double M = (double)c.M(), K = (double)c.K(), NC = c.NC;
  const double ntt_u = 10.0 * (n / 2) * log_n;
  const double ln = (double)L * n;
  double ntts, prods, bytes;
  if (role == PENCIL_ROLE_WGRAD) {
    ntts = L * (2 * M * K + 2 * K * NC + 2 * M * NC);
    prods = 2 * M * K * NC;
    bytes = 8 * ln * (2 * M * K * 2 + 2 * K * NC * 2 + K * NC * 2 + M * K * 2 + 2 * M * NC * 3);
  } else {
    ntts = L * (2 * M * K + K * NC + 2 * M * NC);
    prods = M * K * NC;
    bytes = 8 * ln * (2 * M * K * 2 + M * K * 2 + K * NC * 2 + 2 * M * NC * 3);
  }
  return ntts * ntt_u + prods * 2 * ln * 8 + bytes * 3;
}

// Every valid partition of the candidate grid with its modelled cost.
static void enumerate_partitions(const Geom& g, int role, int n, int log_n, int L,
                                 std::vector<std::pair<double, PencilPartition>>& out) {
  const std::vector<int> ths = ceil_divs(g.Ho()), tws = ceil_divs(g.Wo());
  const std::vector<int> khs = ceil_divs(g.KH), kws = ceil_divs(g.KW);
  const std::vector<int> cis = ceil_divs(g.Ci), cos_ = ceil_divs(g.Co), bs = ceil_divs(g.B);
  for (int th : ths)
    for (int tw : tws)
      for (int kth : khs)
        for (int ktw : kws) {
          const long long hw = (long long)(th + kth - 1) * (tw + ktw - 1);
          if (hw > n) continue;
          const long long cap = n / hw;
          for (int ci : cis) {
            if (ci > cap) continue;
            for (int co : cos_) {
              if ((long long)ci * co > cap) continue;
              const long long bmax = cap / ((long long)ci * co);
              // the largest batch block that fits, as one of the distinct ceil values
              int bb = 1;
              for (int b : bs)
                if (b <= bmax) {
                  bb = b;
                  break;
                }
              PencilPartition p{bb, ci, co, th, tw, kth, ktw};
              if (!part_valid(g, p, n)) continue;
              out.push_back({plan_cost(g, p, role, n, log_n, L), p});
            }
          }
        }
}

static PencilPartition choose_partition(const Geom& g, int role, int n, int log_n, int L) {
  std::vector<std::pair<double, PencilPartition>> all;
  enumerate_partitions(g, role, n, log_n, L, all);
  PencilPartition best{1, 1, 1, 1, 1, 1, 1};
  double best_cost = 1e300;
  for (const auto& c : all)
    if (c.first < best_cost) {
      best_cost = c.first;
      best = c.second;
    }
  return best;
}

static inline u64 pack4(int a, int b, int c, int d) {
  return (u64)(uint16_t)a | ((u64)(uint16_t)b << 16) | ((u64)(uint16_t)c << 32) | ((u64)(uint16_t)d << 48);
}

extern "C" int pencil_plan_linear(PencilCtx* ctx, const PencilLayerDesc* layer, int32_t role,
                                  const PencilPartition* part, PencilPlan** out) {
  if (!ctx || !layer || !out) return PENCIL_E_ARG;
  *out = nullptr;
  if (role < PENCIL_ROLE_FWD || role > PENCIL_ROLE_WGRAD) return PENCIL_E_ARG;
  const PencilLayerDesc& L = *layer;
  if (L.kind != PENCIL_FC && L.kind != PENCIL_CONV) return PENCIL_E_ARG;
  if (L.batch < 1 || L.c_in < 1 || L.c_out < 1) return PENCIL_E_SHAPE;
  if (L.kind == PENCIL_FC && (L.height != 1 || L.width != 1 || L.kernel != 1 || L.pad != 0)) return PENCIL_E_SHAPE;
  if (L.kind == PENCIL_CONV) {
    if (L.height < 1 || L.width < 1 || L.kernel < 1 || L.pad < 0 || L.pad > L.kernel - 1) return PENCIL_E_SHAPE;
    if (L.height + 2 * L.pad < L.kernel || L.width + 2 * L.pad < L.kernel) return PENCIL_E_SHAPE;
  }
  const int n = ctx->n;
  if (L.batch > 65535 || L.c_in > 65535 || L.c_out > 65535 || L.height + 2 * L.pad > 65535 ||
      L.width + 2 * L.pad > 65535)
    return PENCIL_E_SHAPE;

  PencilPlan* P = new (std::nothrow) PencilPlan();
  if (!P) return PENCIL_E_CUDA;
  P->ctx = ctx;
  P->layer = L;
  P->role = role;
  role_setup(L, role, *P);
  const Geom& g = P->g;
  if (part) {
    if (!part_valid(g, *part, n)) {
      delete P;
      return PENCIL_E_CAPACITY;
    }
    P->part = *part;
  } else {
    P->part = choose_partition(g, role, n, ctx->params.log_n, ctx->dev.L);
    if (!part_valid(g, P->part, n)) {
      delete P;
      return PENCIL_E_CAPACITY;
    }
  }
  const PencilPartition& p = P->part;
  P->c = counts_of(g, p);
  const Counts& c = P->c;
  P->ct_in = c.M() * c.K();
  P->pt = c.K() * c.NC;
  P->ct_out = c.M() * c.NC;
  P->products = c.M() * c.K() * c.NC;
  if (P->ct_in > (1 << 30) || P->pt > (1 << 30) || P->ct_out > (1 << 30)) {
    delete P;
    return PENCIL_E_CAPACITY;
  }
  if (role == PENCIL_ROLE_WGRAD)
    P->out_elems = (long long)L.c_out * L.c_in * L.kernel * L.kernel;
  else if (role == PENCIL_ROLE_DGRAD)
    P->out_elems = (long long)L.batch * L.c_in * L.height * L.width;
  else
    P->out_elems = (long long)g.B * g.Co * g.Ho() * g.Wo();

  // --- packing tables (Appendix A index maps)
  const int h = p.th + p.kth - 1, w = p.tw + p.ktw - 1;
  const long long O = (long long)(p.cib - 1) * h * w + (long long)(p.kth - 1) * w + p.ktw - 1;
  const long long blk = (long long)p.cob * p.cib * h * w;
  std::vector<u64> tab(3 * (size_t)n, PENCIL_TAB_NONE);
  for (int b = 0; b < p.bb; ++b)
    for (int ch = 0; ch < p.cib; ++ch)
      for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) tab[b * blk + (long long)ch * h * w + (long long)i * w + j] = pack4(b, ch, i, j);
  for (int co = 0; co < p.cob; ++co)
    for (int ch = 0; ch < p.cib; ++ch)
      for (int u = 0; u < p.kth; ++u)
        for (int v = 0; v < p.ktw; ++v)
          tab[n + O + (long long)co * p.cib * h * w - (long long)ch * h * w - (long long)u * w - v] =
              pack4(co, ch, u, v);
  for (int b = 0; b < p.bb; ++b)
    for (int co = 0; co < p.cob; ++co)
      for (int i = 0; i < p.th; ++i)
        for (int j = 0; j < p.tw; ++j)
          tab[2 * (size_t)n + b * blk + O + (long long)co * p.cib * h * w + (long long)i * w + j] =
              pack4(b, co, i, j);
  std::vector<int4> org((size_t)(P->ct_in + P->pt + P->ct_out));
  size_t o = 0;
  for (long long m = 0; m < c.M(); ++m) {
    const int mw = (int)(m % c.MTW), mh = (int)((m / c.MTW) % c.MTH), mb = (int)(m / ((long long)c.MTW * c.MTH));
    for (long long k = 0; k < c.K(); ++k) {
      const int kw = (int)(k % c.KTW), kh = (int)((k / c.KTW) % c.KTH), kc = (int)(k / ((long long)c.KTW * c.KTH));
      org[o++] = make_int4(mb * p.bb, kc * p.cib, mh * p.th + kh * p.kth, mw * p.tw + kw * p.ktw);
    }
  }
  for (long long k = 0; k < c.K(); ++k) {
    const int kw = (int)(k % c.KTW), kh = (int)((k / c.KTW) % c.KTH), kc = (int)(k / ((long long)c.KTW * c.KTH));
    for (int nn = 0; nn < c.NC; ++nn) org[o++] = make_int4(nn * p.cob, kc * p.cib, kh * p.kth, kw * p.ktw);
  }
  for (long long m = 0; m < c.M(); ++m) {
    const int mw = (int)(m % c.MTW), mh = (int)((m / c.MTW) % c.MTH), mb = (int)(m / ((long long)c.MTW * c.MTH));
    for (int nn = 0; nn < c.NC; ++nn) org[o++] = make_int4(mb * p.bb, nn * p.cob, mh * p.th, mw * p.tw);
  }
  DeviceGuard guard(ctx->device);
  if (cudaMalloc(&P->d_tab, tab.size() * sizeof(u64)) != cudaSuccess ||
      cudaMalloc(&P->d_org, org.size() * sizeof(int4)) != cudaSuccess ||
      cudaMemcpy(P->d_tab, tab.data(), tab.size() * sizeof(u64), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(P->d_org, org.data(), org.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess) {
    pencil_plan_destroy(P);
    return PENCIL_E_CUDA;
  }
  int support[3] = {0, 0, 0};
  for (int sgm = 0; sgm < 3; ++sgm)
    for (int e = n - 1; e >= 0; --e)
      if (tab[(size_t)sgm * n + e] != PENCIL_TAB_NONE) {
        support[sgm] = e + 1;
        break;
      }
  P->pk_v = Packing{P->d_tab, P->d_org, make_int4(g.B, g.Ci, g.H, g.W), support[0]};
  P->pk_w = Packing{P->d_tab + n, P->d_org + P->ct_in, make_int4(g.Co, g.Ci, g.KH, g.KW), support[1]};
  P->pk_y = Packing{P->d_tab + 2 * (size_t)n, P->d_org + P->ct_in + P->pt, make_int4(g.B, g.Co, g.Ho(), g.Wo()),
                    support[2]};

  // --- workspace sizes (bytes, each region 256-byte aligned)
  auto al = [](long long b) { return (b + 255) / 256 * 256; };
  const long long lnb = (long long)ctx->dev.L * n * 8;
  P->ws_encrypt = al(std::max(P->ct_in, P->pt) * (long long)n);
  P->ws_encrypt_pk = al(std::max(P->ct_in, P->pt) * lnb) + 3 * al(std::max(P->ct_in, P->pt) * (long long)n);
  // Alg. 1: NTT(Delta x0) per input ct, NTT(Delta s) per output ct, s per output ct
  P->ws_forward = al(P->ct_in * lnb) + al(P->ct_out * lnb) + al(P->ct_out * (long long)n * 8);
  if (role == PENCIL_ROLE_WGRAD)   // Alg. 2: encoded <gY>_0 and <X>_0, NTT(Delta s), s
    P->ws_backward = al(P->pt * lnb) + al(P->ct_in * lnb) + al(P->ct_out * lnb) + al(P->ct_out * (long long)n * 8);
  else
    P->ws_backward = P->ws_forward;
  P->ws_decrypt = al(P->ct_out * lnb);
  P->m_first = 0;
  P->m_count = P->c.M();
  *out = P;
  return PENCIL_OK;
}

extern "C" int pencil_plan_slice(const PencilPlan* plan, int32_t m_first, int32_t m_count, PencilPlan** out) {
  if (!plan || !out) return PENCIL_E_ARG;
  *out = nullptr;
  if (plan->parent || plan->role == PENCIL_ROLE_WGRAD) return PENCIL_E_ARG;
  if (m_first < 0 || m_count < 1 || (long long)m_first + m_count > plan->c.M()) return PENCIL_E_SHAPE;
  PencilPlan* S = new (std::nothrow) PencilPlan(*plan);
  if (!S) return PENCIL_E_CUDA;
  S->parent = plan;
  S->m_first = m_first;
  S->m_count = m_count;
  *out = S;
  return PENCIL_OK;
}

static int validate_layer(const PencilLayerDesc& L) {
  if (L.kind != PENCIL_FC && L.kind != PENCIL_CONV) return PENCIL_E_ARG;
  if (L.batch < 1 || L.c_in < 1 || L.c_out < 1) return PENCIL_E_SHAPE;
  if (L.kind == PENCIL_FC && (L.height != 1 || L.width != 1 || L.kernel != 1 || L.pad != 0)) return PENCIL_E_SHAPE;
  if (L.kind == PENCIL_CONV) {
    if (L.height < 1 || L.width < 1 || L.kernel < 1 || L.pad < 0 || L.pad > L.kernel - 1) return PENCIL_E_SHAPE;
    if (L.height + 2 * L.pad < L.kernel || L.width + 2 * L.pad < L.kernel) return PENCIL_E_SHAPE;
  }
  if (L.batch > 65535 || L.c_in > 65535 || L.c_out > 65535 || L.height + 2 * L.pad > 65535 ||
      L.width + 2 * L.pad > 65535)
    return PENCIL_E_SHAPE;
  return PENCIL_OK;
}

extern "C" int pencil_plan_candidates(PencilCtx* ctx, const PencilLayerDesc* layer, int32_t role, int32_t max_count,
                                      PencilPartition* out, int32_t* count) {
  if (!ctx || !layer || !count || max_count < 0 || (max_count > 0 && !out)) return PENCIL_E_ARG;
  if (role < PENCIL_ROLE_FWD || role > PENCIL_ROLE_WGRAD) return PENCIL_E_ARG;
  const int rc = validate_layer(*layer);
  if (rc != PENCIL_OK) return rc;
  PencilPlan tmp;
  role_setup(*layer, role, tmp);
  std::vector<std::pair<double, PencilPartition>> all;
  enumerate_partitions(tmp.g, role, ctx->n, ctx->params.log_n, ctx->dev.L, all);
  std::stable_sort(all.begin(), all.end(),
                   [](const std::pair<double, PencilPartition>& a, const std::pair<double, PencilPartition>& b) {
                     return a.first < b.first;
                   });
  int k = 0;
  for (size_t i = 0; i < all.size() && k < max_count; ++i) {
    bool dup = false;
    for (int j = 0; j < k; ++j)
      if (memcmp(&out[j], &all[i].second, sizeof(PencilPartition)) == 0) dup = true;
    if (!dup) out[k++] = all[i].second;
  }
  *count = k;
  return PENCIL_OK;
}

extern "C" int pencil_plan_destroy(PencilPlan* P) {
  if (!P) return PENCIL_E_ARG;
  if (!P->parent) {   // a slice does not own the tables
    DeviceGuard guard(P->ctx->device);
    cudaFree(P->d_tab);
    cudaFree(P->d_org);
  }
  delete P;
  return PENCIL_OK;
}

extern "C" int pencil_plan_sizes(const PencilPlan* P, PencilPlanSizes* s) {
  if (!P || !s) return PENCIL_E_ARG;
  s->part = P->part;
  s->ct_in = P->ct_in;
  s->pt = P->pt;
  s->ct_out = P->ct_out;
  s->products = P->products;
  s->ct_words = 2ll * P->ctx->dev.L * P->ctx->n;
  s->pt_words = (long long)P->ctx->dev.L * P->ctx->n;
  s->out_elems = P->out_elems;
  s->ws_encrypt = P->ws_encrypt;
  s->ws_forward = P->ws_forward;
  s->ws_backward = P->ws_backward;
  s->ws_decrypt = P->ws_decrypt;
  s->ws_encrypt_pk = P->ws_encrypt_pk;
  return PENCIL_OK;
}

// ================================================================== hot path
extern "C" int encode_weights(PencilCtx* ctx, const PencilPlan* P, int32_t operand, const int64_t* values,
                              uint64_t* pt, void* stream) {
  if (!ctx || !P || !values || !pt || P->ctx != ctx) return PENCIL_E_ARG;
  if (operand != PENCIL_OPERAND_INPUT && operand != PENCIL_OPERAND_KERNEL) return PENCIL_E_ARG;
  if (!aligned16(pt)) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  ModeEncode::Params M;
  M.pk = operand == PENCIL_OPERAND_KERNEL ? P->pk_w : P->pk_v;
  M.ac = operand == PENCIL_OPERAND_KERNEL ? P->acc_w : P->acc_v;
  M.ac.ptr = reinterpret_cast<const u64*>(values);
  M.pt = pt;
  const long long first = operand == PENCIL_OPERAND_KERNEL ? 0 : P->in_first();
  const long long count = operand == PENCIL_OPERAND_KERNEL ? P->pt : P->in_count();
  {
    PROF(ctx, PENCIL_K_NTT_ENCODE, (cudaStream_t)stream);
    CUDA_TRY((ntt<ModeEncode, false>(ctx->dev, M, (int)count, (cudaStream_t)stream, (int)first)));
  }
  return PENCIL_OK;
}

extern "C" int encrypt_share(PencilCtx* ctx, const PencilSecretKey* sk, const PencilPlan* P, int32_t operand,
                             const uint64_t* share, uint64_t seed, uint64_t* ct, void* ws, size_t ws_bytes,
                             void* stream) {
  if (!ctx || !sk || !P || !share || !ct || !ws || P->ctx != ctx || sk->ctx != ctx) return PENCIL_E_ARG;
  if (operand != PENCIL_OPERAND_INPUT && operand != PENCIL_OPERAND_KERNEL) return PENCIL_E_ARG;
  if (!aligned16(ct) || !aligned16(ws)) return PENCIL_E_ARG;
  if ((long long)ws_bytes < P->ws_encrypt) return PENCIL_E_CAPACITY;
  DeviceGuard guard(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  if (operand == PENCIL_OPERAND_KERNEL && P->parent) return PENCIL_E_ARG;   // slices cover input / output rows
  const long long first = operand == PENCIL_OPERAND_KERNEL ? 0 : P->in_first();
  const long long count = operand == PENCIL_OPERAND_KERNEL ? P->pt : P->in_count();
  int8_t* err = reinterpret_cast<int8_t*>(ws);
  {
    PROF(ctx, PENCIL_K_SAMPLE_ERR, s);
    CUDA_TRY(launch_sample_err(seed, (int)first, (int)count, ctx->n, err, s));
  }
  ModeEncrypt::Params M;
  M.pk = operand == PENCIL_OPERAND_KERNEL ? P->pk_w : P->pk_v;
  M.ac = operand == PENCIL_OPERAND_KERNEL ? P->acc_w : P->acc_v;
  M.ac.ptr = share;
  M.err = err;
  M.sk = sk->sk;
  M.ct = ct;
  M.seed = seed;
  {
    PROF(ctx, PENCIL_K_NTT_ENCRYPT, s);
    CUDA_TRY((ntt<ModeEncrypt, false>(ctx->dev, M, (int)count, s, (int)first)));
  }
  return PENCIL_OK;
}

extern "C" int encrypt_share_pk(PencilCtx* ctx, const PencilPublicKey* pk, const PencilPlan* P, int32_t operand,
                                const uint64_t* share, uint64_t seed, uint64_t* ct, void* ws, size_t ws_bytes,
                                void* stream) {
  if (!ctx || !pk || !P || !share || !ct || !ws || P->ctx != ctx || pk->ctx != ctx) return PENCIL_E_ARG;
  if (operand != PENCIL_OPERAND_INPUT && operand != PENCIL_OPERAND_KERNEL) return PENCIL_E_ARG;
  if (!aligned16(ct) || !aligned16(ws)) return PENCIL_E_ARG;
  if ((long long)ws_bytes < P->ws_encrypt_pk) return PENCIL_E_CAPACITY;
  if (operand == PENCIL_OPERAND_KERNEL && P->parent) return PENCIL_E_ARG;   // slices cover input / output rows
  DeviceGuard guard(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  const long long first = operand == PENCIL_OPERAND_KERNEL ? 0 : P->in_first();
  const long long count = operand == PENCIL_OPERAND_KERNEL ? P->pt : P->in_count();
  // ws: NTT(u) [n_all][L][N], then e1, e2, u [n_all][N] each (int8), indexed by
  // the absolute ciphertext position like encrypt_share's errors.
  const long long n_all = std::max(P->ct_in, P->pt);
  auto al = [](long long b) { return (b + 255) / 256 * 256; };
  char* w = reinterpret_cast<char*>(ws);
  u64* u_hat = reinterpret_cast<u64*>(w);
  int8_t* e1 = reinterpret_cast<int8_t*>(w + al(n_all * (long long)ctx->dev.L * ctx->n * 8));
  int8_t* e2 = e1 + al(n_all * (long long)ctx->n);
  int8_t* u = e2 + al(n_all * (long long)ctx->n);
  {
    PROF(ctx, PENCIL_K_SAMPLE_PK, s);
    CUDA_TRY(launch_sample_pk(seed, (int)first, (int)count, ctx->n, e1, e2, u, s));
  }
  ModePkU::Params U;
  U.u = u;
  U.u_hat = u_hat;
  {
    PROF(ctx, PENCIL_K_NTT_PK_U, s);
    CUDA_TRY((ntt<ModePkU, false>(ctx->dev, U, (int)count, s, (int)first)));
  }
  ModeEncryptPk::Params M;
  M.pk = operand == PENCIL_OPERAND_KERNEL ? P->pk_w : P->pk_v;
  M.ac = operand == PENCIL_OPERAND_KERNEL ? P->acc_w : P->acc_v;
  M.ac.ptr = share;
  M.e1 = e1;
  M.e2 = e2;
  M.u_hat = u_hat;
  M.key = pk->key;
  M.ct = ct;
  {
    PROF(ctx, PENCIL_K_NTT_ENCRYPT_PK, s);
    CUDA_TRY((ntt<ModeEncryptPk, false>(ctx->dev, M, (int)(2 * count), s, (int)(2 * first))));
  }
  return PENCIL_OK;
}

// Workspace regions of Alg. 1 (FWD or DGRAD plan): NTT(Delta x0) [ct_in][L][N],
// NTT(Delta s) [ct_out][L][N], mask coefficients s [ct_out][N].
struct Alg1Ws {
  u64 *p0, *mnt, *mpoly;
};
static Alg1Ws alg1_ws(const PencilPlan* P, char* ws) {
  auto al = [](long long b) { return (b + 255) / 256 * 256; };
  const long long lnb = (long long)P->ctx->dev.L * P->ctx->n * 8;
  Alg1Ws w;
  w.p0 = reinterpret_cast<u64*>(ws);
  w.mnt = reinterpret_cast<u64*>(ws + al(P->ct_in * lnb));
  w.mpoly = reinterpret_cast<u64*>(ws + al(P->ct_in * lnb) + al(P->ct_out * lnb));
  return w;
}

// MO's ciphertext-independent part of Alg. 1 steps 2-3: the mask s (Z_t
// coefficients), then NTT(Delta pi_v(x0)) and NTT(Delta s) in one launch, and
// the MO's share s + b.
static int alg1_prepare(PencilCtx* ctx, const PencilPlan* P, const u64* x0, const u64* bias, u64 mask_seed, u64* y0,
                        char* ws, cudaStream_t s) {
  const Alg1Ws w = alg1_ws(P, ws);
  {
    PROF(ctx, PENCIL_K_MASK_POLY, s);
    CUDA_TRY(launch_mask_poly(ctx->dev, P->pk_y, P->acc_y, mask_seed, (int)P->ct_out, w.mpoly, s));
  }
  ModeMoPrep::Params R;
  R.pk = P->pk_v;
  R.ac = P->acc_v;
  R.ac.ptr = x0;
  R.mpoly = w.mpoly;
  R.n_in = (int)P->ct_in;
  R.out_in = w.p0;
  R.out_mask = w.mnt;
  R.seed = mask_seed;
  {
    PROF(ctx, PENCIL_K_NTT_MO_PREP, s);
    CUDA_TRY((ntt<ModeMoPrep, false>(ctx->dev, R, (int)(P->ct_in + P->ct_out), s)));
  }
  {
    PROF(ctx, PENCIL_K_MO_SHARE, s);
    CUDA_TRY(launch_mo_share(mask_seed, P->out_elems, ctx->dev.t_mask, bias, P->hw, P->co_out, y0, s));
  }
  return PENCIL_OK;
}

// Alg. 1 steps 2-3 on the received ciphertexts: ct_out[m, n] = sum_k
// (ct_in[m, k] + NTT(Delta x0)[m, k]) pt[k, n] - NTT(Delta s)[m, n], one launch.
static int alg1_apply(PencilCtx* ctx, const PencilPlan* P, const u64* ct_in, const u64* pt, u64* ct_out, char* ws,
                      cudaStream_t s) {
  const Alg1Ws w = alg1_ws(P, ws);
  const long long lnw = (long long)ctx->dev.L * ctx->n;
  MacParams M;
  memset(&M, 0, sizeof(M));
  M.a0 = ct_in;
  M.a0_stride = 2 * lnw;
  M.p0 = w.p0;
  M.p0_stride = lnw;
  M.a1 = ct_in + lnw;
  M.a1_stride = 2 * lnw;
  M.b = pt;
  M.b_stride = lnw;
  M.mask = w.mnt;
  M.out = ct_out;
  M.m_base = (int)P->m_first;   // output rows [m_first, m_first + m_count)
  M.M = (int)(P->m_first + P->m_count);
  M.K = (int)P->c.K();
  M.NC = P->c.NC;
  M.lanes = (int)lnw;
  {
    PROF(ctx, PENCIL_K_MAC, s);
    CUDA_TRY(launch_mac(ctx->dev, M, false, s));
  }
  return PENCIL_OK;
}

static int alg1(PencilCtx* ctx, const PencilPlan* P, const u64* ct_in, const u64* pt, const u64* x0, const u64* bias,
                u64 mask_seed, u64* ct_out, u64* y0, char* ws, cudaStream_t s) {
  int rc = alg1_prepare(ctx, P, x0, bias, mask_seed, y0, ws, s);
  return rc != PENCIL_OK ? rc : alg1_apply(ctx, P, ct_in, pt, ct_out, ws, s);
}

static int check_fwd_plan(PencilCtx* ctx, const PencilPlan* P, const void* bias, void* ws, size_t ws_bytes) {
  if (!ctx || !P || !ws || P->ctx != ctx) return PENCIL_E_ARG;
  if (P->role == PENCIL_ROLE_WGRAD) return PENCIL_E_ARG;
  if (bias && P->role != PENCIL_ROLE_FWD) return PENCIL_E_ARG;
  if (!aligned16(ws)) return PENCIL_E_ARG;
  if ((long long)ws_bytes < P->ws_forward) return PENCIL_E_CAPACITY;
  return PENCIL_OK;
}

extern "C" int he_linear_forward(PencilCtx* ctx, const PencilPlan* P, const uint64_t* ct_in, const uint64_t* pt,
                                 const uint64_t* x0, const uint64_t* bias, uint64_t mask_seed, uint64_t* ct_out,
                                 uint64_t* y0, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_fwd_plan(ctx, P, bias, ws, ws_bytes);
  if (rc != PENCIL_OK) return rc;
  if (!ct_in || !pt || !x0 || !ct_out || !y0) return PENCIL_E_ARG;
  if (!aligned16(ct_in) || !aligned16(pt) || !aligned16(ct_out)) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  return alg1(ctx, P, ct_in, pt, x0, bias, mask_seed, ct_out, y0, reinterpret_cast<char*>(ws), (cudaStream_t)stream);
}

extern "C" int he_linear_forward_prepare(PencilCtx* ctx, const PencilPlan* P, const uint64_t* x0,
                                         const uint64_t* bias, uint64_t mask_seed, uint64_t* y0, void* ws,
                                         size_t ws_bytes, void* stream) {
  int rc = check_fwd_plan(ctx, P, bias, ws, ws_bytes);
  if (rc != PENCIL_OK) return rc;
  if (!x0 || !y0) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  return alg1_prepare(ctx, P, x0, bias, mask_seed, y0, reinterpret_cast<char*>(ws), (cudaStream_t)stream);
}

extern "C" int he_linear_forward_apply(PencilCtx* ctx, const PencilPlan* P, const uint64_t* ct_in, const uint64_t* pt,
                                       uint64_t* ct_out, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_fwd_plan(ctx, P, nullptr, ws, ws_bytes);
  if (rc != PENCIL_OK) return rc;
  if (!ct_in || !pt || !ct_out) return PENCIL_E_ARG;
  if (!aligned16(ct_in) || !aligned16(pt) || !aligned16(ct_out)) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  return alg1_apply(ctx, P, ct_in, pt, ct_out, reinterpret_cast<char*>(ws), (cudaStream_t)stream);
}

extern "C" int he_linear_backward(PencilCtx* ctx, const PencilPlan* Pd, const PencilPlan* Pw,
                                  const uint64_t* ct_gy1_d, const uint64_t* pt_wt, const uint64_t* ct_x1_w,
                                  const uint64_t* ct_gy1_w, const uint64_t* gy0, const uint64_t* x0,
                                  uint64_t mask_seed_x, uint64_t mask_seed_w, uint64_t* ct_gx, uint64_t* gx0,
                                  uint64_t* ct_gw, uint64_t* gw_mask, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || (!Pd && !Pw) || !ws || !aligned16(ws)) return PENCIL_E_ARG;
  if ((Pd && Pd->parent) || (Pw && Pw->parent)) return PENCIL_E_ARG;   // whole plans only
  if (Pd && (Pd->ctx != ctx || Pd->role != PENCIL_ROLE_DGRAD || !ct_gy1_d || !pt_wt || !gy0 || !ct_gx || !gx0 ||
             !aligned16(ct_gy1_d) || !aligned16(pt_wt) || !aligned16(ct_gx)))
    return PENCIL_E_ARG;
  if (Pw && (Pw->ctx != ctx || Pw->role != PENCIL_ROLE_WGRAD || !ct_x1_w || !ct_gy1_w || !gy0 || !x0 || !ct_gw ||
             !gw_mask || !aligned16(ct_x1_w) || !aligned16(ct_gy1_w) || !aligned16(ct_gw)))
    return PENCIL_E_ARG;
  if (Pd && Pw) {
    const PencilLayerDesc &a = Pd->layer, &b = Pw->layer;
    if (memcmp(&a, &b, sizeof(a)) != 0) return PENCIL_E_SHAPE;
  }
  const long long need = (Pd ? Pd->ws_backward : 0) + (Pw ? Pw->ws_backward : 0);
  if ((long long)ws_bytes < need) return PENCIL_E_CAPACITY;
  DeviceGuard guard(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  char* w = reinterpret_cast<char*>(ws);
  if (Pd) {
    int rc = alg1(ctx, Pd, ct_gy1_d, pt_wt, gy0, nullptr, mask_seed_x, ct_gx, gx0, w, s);
    if (rc != PENCIL_OK) return rc;
    w += Pd->ws_backward;
  }
  if (Pw) {
    const long long lnw = (long long)ctx->dev.L * ctx->n;
    auto al = [](long long b) { return (b + 255) / 256 * 256; };
    u64* pt_gy0 = reinterpret_cast<u64*>(w);
    u64* pt_x0 = reinterpret_cast<u64*>(w + al(Pw->pt * lnw * 8));
    u64* mnt = reinterpret_cast<u64*>(w + al(Pw->pt * lnw * 8) + al(Pw->ct_in * lnw * 8));
    u64* mpoly = reinterpret_cast<u64*>(w + al(Pw->pt * lnw * 8) + al(Pw->ct_in * lnw * 8) + al(Pw->ct_out * lnw * 8));
    {
      PROF(ctx, PENCIL_K_MASK_POLY, s);
      CUDA_TRY(launch_mask_poly(ctx->dev, Pw->pk_y, Pw->acc_y, mask_seed_w, (int)Pw->ct_out, mpoly, s));
    }
    ModeMoPrep::Params R;
    memset(&R, 0, sizeof(R));
    R.mpoly = mpoly;
    R.n_in = 0;
    R.out_mask = mnt;
    R.seed = mask_seed_w;
    {
      PROF(ctx, PENCIL_K_NTT_MO_PREP, s);
      CUDA_TRY((ntt<ModeMoPrep, false>(ctx->dev, R, (int)Pw->ct_out, s)));
    }
    ModeEncode::Params E1;
    E1.pk = Pw->pk_w;
    E1.ac = Pw->acc_w;
    E1.ac.ptr = gy0;
    E1.pt = pt_gy0;
    {
      PROF(ctx, PENCIL_K_NTT_ENCODE, s);
      CUDA_TRY((ntt<ModeEncode, false>(ctx->dev, E1, (int)Pw->pt, s)));
    }
    ModeEncode::Params E2;
    E2.pk = Pw->pk_v;
    E2.ac = Pw->acc_v;
    E2.ac.ptr = x0;
    E2.pt = pt_x0;
    {
      PROF(ctx, PENCIL_K_NTT_ENCODE, s);
      CUDA_TRY((ntt<ModeEncode, false>(ctx->dev, E2, (int)Pw->ct_in, s)));
    }
    MacParams M;
    memset(&M, 0, sizeof(M));
    M.a0 = ct_x1_w;
    M.a0_stride = 2 * lnw;
    M.a1 = ct_x1_w + lnw;
    M.a1_stride = 2 * lnw;
    M.b = pt_gy0;
    M.b_stride = lnw;
    M.pa = pt_x0;
    M.pa_stride = lnw;
    M.cb0 = ct_gy1_w;
    M.cb1 = ct_gy1_w + lnw;
    M.cb_stride = 2 * lnw;
    M.mask = mnt;
    M.out = ct_gw;
    M.M = (int)Pw->c.M();
    M.K = (int)Pw->c.K();
    M.NC = Pw->c.NC;
    M.lanes = (int)lnw;
    {
      PROF(ctx, PENCIL_K_MAC_DUAL, s);
      CUDA_TRY(launch_mac(ctx->dev, M, true, s));
    }
    {
      PROF(ctx, PENCIL_K_MO_SHARE, s);
      CUDA_TRY(launch_mo_share(mask_seed_w, Pw->out_elems, ctx->dev.t_mask, nullptr, 1, 1, gw_mask, s));
    }
  }
  return PENCIL_OK;
}

extern "C" int decrypt_to_share(PencilCtx* ctx, const PencilSecretKey* sk, const PencilPlan* P,
                                const uint64_t* ct_out, uint64_t* y1, int32_t check_noise, void* ws, size_t ws_bytes,
                                void* stream) {
  if (!ctx || !sk || !P || !ct_out || !y1 || !ws || P->ctx != ctx || sk->ctx != ctx) return PENCIL_E_ARG;
  if (!aligned16(ct_out) || !aligned16(ws)) return PENCIL_E_ARG;
  if ((long long)ws_bytes < P->ws_decrypt) return PENCIL_E_CAPACITY;
  DeviceGuard guard(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  ModeDecrypt::Params D;
  D.ct = ct_out;
  D.sk = sk->sk;
  D.out = reinterpret_cast<u64*>(ws);
  D.skip_c0 = 0;
  if (ctx->dev.L <= 8) {   // INTT and CRT step in one launch, one cluster of L CTAs per ciphertext
    ModeDecryptFused::Params F;
    F.d = D;
    F.pk = P->pk_y;
    F.ac = P->acc_y;
    F.y1 = y1;
    F.check = check_noise ? 1 : 0;
    PROF(ctx, PENCIL_K_INTT_DECRYPT, s);
    CUDA_TRY((ntt<ModeDecryptFused, true>(ctx->dev, F, (int)P->out_count(), s, (int)P->out_first())));
    return PENCIL_OK;
  }
  {
    PROF(ctx, PENCIL_K_INTT_DECRYPT, s);
    CUDA_TRY((ntt<ModeDecrypt, true>(ctx->dev, D, (int)P->out_count(), s, (int)P->out_first())));
  }
  {
    PROF(ctx, PENCIL_K_DECRYPT_COMBINE, s);
    CUDA_TRY(launch_decrypt_combine(ctx->dev, P->pk_y, P->acc_y, D.out, (int)P->out_first(), (int)P->out_count(),
                                    check_noise ? 1 : 0, y1, s));
  }
  return PENCIL_OK;
}

extern "C" int compact_returned(PencilCtx* ctx, const PencilPlan* P, const uint64_t* ct_out, uint64_t* c0c,
                                void* stream) {
  if (!ctx || !P || !ct_out || !c0c || P->ctx != ctx) return PENCIL_E_ARG;
  if (!aligned16(ct_out)) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  ModeCompact::Params C;
  C.ct = ct_out;
  C.pk = P->pk_y;
  C.ac = P->acc_y;
  C.c0c = c0c;
  C.out_elems = P->out_elems;
  {
    PROF(ctx, PENCIL_K_INTT_COMPACT, s);
    CUDA_TRY((ntt<ModeCompact, true>(ctx->dev, C, (int)P->out_count(), s, (int)P->out_first())));
  }
  return PENCIL_OK;
}

extern "C" int decrypt_compact_to_share(PencilCtx* ctx, const PencilSecretKey* sk, const PencilPlan* P,
                                        const uint64_t* ct_out, const uint64_t* c0c, uint64_t* y1,
                                        int32_t check_noise, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !sk || !P || !ct_out || !c0c || !y1 || !ws || P->ctx != ctx || sk->ctx != ctx) return PENCIL_E_ARG;
  if (!aligned16(ct_out) || !aligned16(ws)) return PENCIL_E_ARG;
  if ((long long)ws_bytes < P->ws_decrypt) return PENCIL_E_CAPACITY;
  DeviceGuard guard(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  ModeDecrypt::Params D;
  D.ct = ct_out;
  D.sk = sk->sk;
  D.out = reinterpret_cast<u64*>(ws);
  D.skip_c0 = 1;
  {
    PROF(ctx, PENCIL_K_INTT_DECRYPT, s);
    CUDA_TRY((ntt<ModeDecrypt, true>(ctx->dev, D, (int)P->out_count(), s, (int)P->out_first())));
  }
  {
    PROF(ctx, PENCIL_K_DECRYPT_COMBINE, s);
    CUDA_TRY(launch_decrypt_combine(ctx->dev, P->pk_y, P->acc_y, D.out, (int)P->out_first(), (int)P->out_count(),
                                    check_noise ? 1 : 0, y1, s, c0c, P->out_elems));
  }
  return PENCIL_OK;
}

extern "C" int pencil_ring_linear(PencilCtx* ctx, const PencilPlan* P, const uint64_t* kernel_operand,
                                  const uint64_t* input_operand, const uint64_t* addend,
                                  const uint64_t* addend2, uint64_t* out, void* stream) {
  if (!ctx || !P || !kernel_operand || !input_operand || !out || P->ctx != ctx) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  RingParams R;
  R.kbound = make_int4(P->g.Co, P->g.Ci, P->g.KH, P->g.KW);
  R.Ho = P->g.Ho();
  R.Wo = P->g.Wo();
  R.v = P->acc_v;
  R.v.ptr = input_operand;
  R.w = P->acc_w;
  R.w.ptr = kernel_operand;
  R.y = P->acc_y;
  R.addend = addend;
  R.addend2 = addend2;
  R.out = out;
  R.outs = (long long)P->g.B * P->g.Co * R.Ho * R.Wo;
  R.t_mask = ctx->dev.t_mask;
  PROF(ctx, PENCIL_K_RING, s);
  CUDA_TRY(launch_ring(R, s));
  return PENCIL_OK;
}

static int lincomb(PencilCtx* ctx, const uint64_t* src, int64_t src_offset, int64_t inner, int64_t outer_stride,
                   int64_t term_stride, int32_t terms, int64_t term_stride2, int32_t terms2, const uint64_t* scalars,
                   const uint64_t* addend, int32_t negate, uint64_t* out, int64_t count, void* stream) {
  if (!ctx || !src || !out || count < 0 || inner < 1 || src_offset < 0 || outer_stride < 0 || term_stride < 0 ||
      term_stride2 < 0)
    return PENCIL_E_ARG;
  if (terms < 0 || terms2 < 1 || (long long)terms * terms2 > PENCIL_LINCOMB_MAX_TERMS || (terms > 0 && !scalars))
    return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  LincombP P;
  memset(&P, 0, sizeof(P));
  P.src = src;
  P.off = src_offset;
  P.inner = inner;
  P.outer = outer_stride;
  P.tstride = term_stride;
  P.tstride2 = term_stride2;
  P.count = count;
  P.addend = addend;
  P.out = out;
  P.terms = terms;
  P.terms2 = terms2;
  P.negate = negate ? 1 : 0;
  for (int i = 0; i < terms * terms2; ++i) P.k[i] = scalars[i];
  {
    PROF(ctx, PENCIL_K_LINCOMB, (cudaStream_t)stream);
    CUDA_TRY(launch_lincomb(P, ctx->dev.t_mask, (cudaStream_t)stream));
  }
  return PENCIL_OK;
}

extern "C" int pencil_lincomb(PencilCtx* ctx, const uint64_t* src, int64_t src_offset, int64_t inner,
                              int64_t outer_stride, int64_t term_stride, const uint64_t* scalars, int32_t terms,
                              const uint64_t* addend, int32_t negate, uint64_t* out, int64_t count, void* stream) {
  return lincomb(ctx, src, src_offset, inner, outer_stride, term_stride, terms, 0, 1, scalars, addend, negate, out,
                 count, stream);
}

extern "C" int pencil_lincomb2(PencilCtx* ctx, const uint64_t* src, int64_t src_offset, int64_t inner,
                               int64_t outer_stride, int64_t term_stride, int32_t terms, int64_t term_stride2,
                               int32_t terms2, const uint64_t* scalars, const uint64_t* addend, int32_t negate,
                               uint64_t* out, int64_t count, void* stream) {
  return lincomb(ctx, src, src_offset, inner, outer_stride, term_stride, terms, term_stride2, terms2, scalars, addend,
                 negate, out, count, stream);
}

extern "C" int pencil_bias_grad(PencilCtx* ctx, const PencilPlan* P, const uint64_t* g, uint64_t* out,
                                void* stream) {
  if (!ctx || !P || !g || !out || P->ctx != ctx) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  const PencilLayerDesc& L = P->layer;
  const long long ho = L.height + 2 * L.pad - L.kernel + 1, wo = L.width + 2 * L.pad - L.kernel + 1;
  const long long hw = L.kind == PENCIL_FC ? 1 : ho * wo;
  PROF(ctx, PENCIL_K_BIAS_GRAD, (cudaStream_t)stream);
  CUDA_TRY(launch_bias_grad(g, L.batch, L.c_out, hw, ctx->dev.t_mask, out, (cudaStream_t)stream));
  return PENCIL_OK;
}

extern "C" int pencil_ntt_batch(PencilCtx* ctx, uint64_t* polys, int64_t count, int32_t inverse, void* stream) {
  if (!ctx || !polys || count < 0 || count > (1ll << 31) - 1) return PENCIL_E_ARG;
  if (!aligned16(polys)) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  ModeRaw::Params R;
  R.polys = polys;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess)
    R.ahead = 2 * sms;   // about one wave of transform CTAs (two per SM up to N = 8192)
  if (inverse) {
    PROF(ctx, PENCIL_K_INTT_RAW, (cudaStream_t)stream);
    CUDA_TRY((ntt<ModeRaw, true>(ctx->dev, R, (int)count, (cudaStream_t)stream)));
  } else {
    PROF(ctx, PENCIL_K_NTT_RAW, (cudaStream_t)stream);
    CUDA_TRY((ntt<ModeRaw, false>(ctx->dev, R, (int)count, (cudaStream_t)stream)));
  }
  return PENCIL_OK;
}

// ================================================================== profiling
extern "C" int pencil_profile(PencilCtx* ctx, int32_t enable) {
  if (!ctx) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  if (enable) {
    for (ProfRec& r : ctx->prof) {
      ctx->pool.push_back(r.a);
      ctx->pool.push_back(r.b);
    }
    ctx->prof.clear();
  }
  ctx->prof_on = enable != 0;
  return PENCIL_OK;
}

extern "C" int pencil_profile_read(PencilCtx* ctx, PencilProfEntry* out, int32_t max_entries, int32_t* n_entries) {
  if (!ctx || !n_entries || (max_entries > 0 && !out)) return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  double ms[PENCIL_K_COUNT] = {0};
  int launches[PENCIL_K_COUNT] = {0};
  for (ProfRec& r : ctx->prof) {
    CUDA_TRY(cudaEventSynchronize(r.b));
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.kernel] += t;
    launches[r.kernel] += 1;
  }
  int n = 0;
  for (int k = 0; k < PENCIL_K_COUNT; ++k) {
    if (!launches[k]) continue;
    if (n < max_entries) out[n] = PencilProfEntry{k, launches[k], ms[k]};
    ++n;
  }
  *n_entries = n;
  return PENCIL_OK;
}

extern "C" int pencil_mul_probe(PencilCtx* ctx, int32_t which, int64_t iters, int32_t blocks, int32_t threads,
                                double* ms, double* steps, void* stream) {
  if (!ctx || !ms || !steps || which < 0 || which > 15 || iters < 1 || blocks < 1 || threads < 32 ||
      threads > 1024)
    return PENCIL_E_ARG;
  DeviceGuard guard(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a, b;
  u64* sink = nullptr;
  CUDA_TRY(cudaMalloc(&sink, sizeof(u64)));
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  CUDA_TRY(cudaEventRecord(a, s));
  cudaError_t e = launch_mul_probe(which, iters, blocks, threads, 0x1234567887654321ull, sink, s);
  CUDA_TRY(cudaEventRecord(b, s));
  CUDA_TRY(cudaEventSynchronize(b));
  float t = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  CUDA_TRY(e);
  *ms = t;
  *steps = (double)blocks * threads * 8.0 * (double)iters;
  return PENCIL_OK;
}

// ================================================================== allocation-free encryption
// Scratch of encrypt_share_noalloc: the sampled encryption errors, one byte per
// coefficient of every ciphertext of the call.  A file-scope device array, so
// the call needs no workspace and allocates nothing; each GPU that loads the
// library holds these 8 MiB until the process exits.
#define PENCIL_NOALLOC_SCRATCH_BYTES (8ull << 20)
static __device__ __align__(256) int8_t g_noalloc_scratch[PENCIL_NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mutex;

// Device address of the scratch array for `ctx` (whose device must be current).
// Host code cannot use the symbol itself: its name stands for a host-side
// shadow, not for device memory.  Looked up on the context's first call and kept
// with the context (a context created after a device reset looks it up again).
static int noalloc_scratch(PencilCtx* ctx, int8_t** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!ctx->noalloc_addr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "pencil: encrypt_share_noalloc: cudaGetSymbolAddress failed on device %d: %s\n", ctx->device,
              cudaGetErrorString(e));
      return PENCIL_E_CUDA;
    }
    ctx->noalloc_addr = p;
  }
  *out = reinterpret_cast<int8_t*>(ctx->noalloc_addr);
  return PENCIL_OK;
}

extern "C" int encrypt_share_noalloc(PencilCtx* ctx, const PencilSecretKey* sk, const PencilPlan* P, int32_t operand,
                                     const uint64_t* share, uint64_t seed, uint64_t* ct, void* stream) {
  if (!ctx || !sk || !P || !share || !ct || P->ctx != ctx || sk->ctx != ctx) return PENCIL_E_ARG;
  if (operand != PENCIL_OPERAND_INPUT && operand != PENCIL_OPERAND_KERNEL) return PENCIL_E_ARG;
  if (!aligned16(ct) || P->parent) return PENCIL_E_ARG;   // whole plans only
  const long long count = operand == PENCIL_OPERAND_KERNEL ? P->pt : P->ct_in;
  const unsigned long long need = (unsigned long long)count * (unsigned long long)ctx->n;
  if (need > PENCIL_NOALLOC_SCRATCH_BYTES) {
    fprintf(stderr,
            "pencil: encrypt_share_noalloc: %lld ciphertexts x N = %d need %llu bytes of scratch, more than the "
            "%llu-byte static buffer; use encrypt_share with a workspace\n",
            count, ctx->n, need, (unsigned long long)PENCIL_NOALLOC_SCRATCH_BYTES);
    return PENCIL_E_CAPACITY;
  }
  DeviceGuard guard(ctx->device);
  int8_t* err = nullptr;
  const int rc = noalloc_scratch(ctx, &err);
  if (rc != PENCIL_OK) return rc;
  const cudaStream_t s = (cudaStream_t)stream;
  {
    PROF(ctx, PENCIL_K_SAMPLE_ERR, s);
    CUDA_TRY(launch_sample_err(seed, 0, (int)count, ctx->n, err, s));
  }
  ModeEncrypt::Params M;
  M.pk = operand == PENCIL_OPERAND_KERNEL ? P->pk_w : P->pk_v;
  M.ac = operand == PENCIL_OPERAND_KERNEL ? P->acc_w : P->acc_v;
  M.ac.ptr = share;
  M.err = err;
  M.sk = sk->sk;
  M.ct = ct;
  M.seed = seed;
  {
    PROF(ctx, PENCIL_K_NTT_ENCRYPT, s);
    CUDA_TRY((ntt<ModeEncrypt, false>(ctx->dev, M, (int)count, s)));
  }
  return PENCIL_OK;
}

// ================================================================== batched layers
struct PencilBatch {
  PencilCtx* ctx = nullptr;
  std::vector<const PencilPlan*> plans;
  // FWD / DGRAD layers: W, x1, x0 (the DO's and MO's shares of the product's
  // input), bias, y0, y1.  WGRAD layers: g0, g1 (shares of grad_Y), x0, x1,
  // y0 = the MO's mask share, y1 = the DO's decrypted share.
  struct User {
    const int64_t* W = nullptr;
    const u64 *x1 = nullptr, *x0 = nullptr, *bias = nullptr, *g0 = nullptr, *g1 = nullptr;
    u64 *y0 = nullptr, *y1 = nullptr;
    bool bound = false;
  };
  // p0: NTT(Delta x0) (Alg. 1) or the encoded <X>_0 (Alg. 2); ct_k, err_k: Alg. 2's
  // Enc(<gY>_1) at kernel positions and its errors.
  struct Off {
    long long pt, ct_in, ct_out, err, p0, mnt, mpoly, yres, ct_k, err_k;
  };
  std::vector<User> user;
  std::vector<Off> off;
  long long ws_bytes = 0;
  char* ws = nullptr;
  void* d_mem = nullptr;
  BatchDev dev;
  int mac_nt = 0;
  bool committed = false;
};

extern "C" int pencil_batch_create(PencilCtx* ctx, const PencilPlan* const* plans, int32_t count, PencilBatch** out) {
  if (!ctx || !plans || !out || count < 1) return PENCIL_E_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!plans[i] || plans[i]->ctx != ctx || plans[i]->parent) return PENCIL_E_ARG;
  PencilBatch* B = new (std::nothrow) PencilBatch();
  if (!B) return PENCIL_E_CUDA;
  B->ctx = ctx;
  B->plans.assign(plans, plans + count);
  B->user.resize(count);
  const long long n = ctx->n, lnb = (long long)ctx->dev.L * n * 8;
  auto al = [](long long b) { return (b + 255) / 256 * 256; };
  long long o = 0;
  for (int i = 0; i < count; ++i) {
    const PencilPlan* P = plans[i];
    PencilBatch::Off f;
    f.pt = o;
    o += al(P->pt * lnb);
    f.ct_in = o;
    o += al(P->ct_in * 2 * lnb);
    f.ct_out = o;
    o += al(P->ct_out * 2 * lnb);
    // Buffers whose lifetimes do not overlap share memory (the launches of a batch
    // run in a fixed order on one stream): the mask polynomials and the sampled
    // errors live inside the output ciphertexts' region until the
    // multiply-accumulate writes it; the decryption residues reuse NTT(Delta x0) /
    // <X>_0 and NTT(Delta s), which the multiply-accumulate has finished reading.
    f.mpoly = f.ct_out;
    if (al(P->ct_out * n * 8) + al(P->ct_in * n) <= al(P->ct_out * 2 * lnb)) {
      f.err = f.ct_out + al(P->ct_out * n * 8);
    } else {
      f.err = o;
      o += al(P->ct_in * n);
    }
    f.p0 = o;
    o += al(P->ct_in * lnb);
    f.mnt = o;
    o += al(P->ct_out * lnb);
    f.yres = f.p0;   // ct_out lnb <= (ct_in + ct_out) lnb, the p0 and mnt regions
    f.ct_k = f.err_k = 0;
    if (P->role == PENCIL_ROLE_WGRAD) {
      f.ct_k = o;
      o += al(P->pt * 2 * lnb);
      f.err_k = o;
      o += al(P->pt * n);
    }
    B->off.push_back(f);
  }
  B->ws_bytes = o;
  memset(&B->dev, 0, sizeof(B->dev));
  B->dev.withhold = -1;
  *out = B;
  return PENCIL_OK;
}

extern "C" int pencil_batch_destroy(PencilBatch* B) {
  if (!B) return PENCIL_E_ARG;
  DeviceGuard guard(B->ctx->device);
  cudaFree(B->d_mem);
  delete B;
  return PENCIL_OK;
}

extern "C" int pencil_batch_workspace(const PencilBatch* B, int64_t* bytes) {
  if (!B || !bytes) return PENCIL_E_ARG;
  *bytes = B->ws_bytes;
  return PENCIL_OK;
}

extern "C" int pencil_batch_bind(PencilBatch* B, int32_t layer, const int64_t* W, const uint64_t* x1,
                                 const uint64_t* x0, const uint64_t* bias, uint64_t* y0, uint64_t* y1) {
  if (!B || layer < 0 || layer >= (int)B->plans.size() || !W || !x1 || !x0 || !y0 || !y1) return PENCIL_E_ARG;
  const int role = B->plans[layer]->role;
  if (role == PENCIL_ROLE_WGRAD || (bias && role != PENCIL_ROLE_FWD)) return PENCIL_E_ARG;
  B->user[layer] = PencilBatch::User{W, x1, x0, bias, nullptr, nullptr, y0, y1, true};
  B->committed = false;
  return PENCIL_OK;
}

extern "C" int pencil_batch_bind_wgrad(PencilBatch* B, int32_t layer, const uint64_t* gy0, const uint64_t* gy1,
                                       const uint64_t* x0, const uint64_t* x1, uint64_t* gw_mask, uint64_t* tilde) {
  if (!B || layer < 0 || layer >= (int)B->plans.size() || !gy0 || !gy1 || !x0 || !x1 || !gw_mask || !tilde)
    return PENCIL_E_ARG;
  if (B->plans[layer]->role != PENCIL_ROLE_WGRAD) return PENCIL_E_ARG;
  B->user[layer] = PencilBatch::User{nullptr, x1, x0, nullptr, gy0, gy1, gw_mask, tilde, true};
  B->committed = false;
  return PENCIL_OK;
}

template <class T>
static void put(std::vector<char>& blob, size_t& at, const std::vector<T>& v, size_t& where) {
  at = (at + 255) / 256 * 256;
  where = at;
  blob.resize(at + v.size() * sizeof(T));
  if (!v.empty()) memcpy(blob.data() + at, v.data(), v.size() * sizeof(T));
  at += v.size() * sizeof(T);
}

extern "C" int pencil_batch_commit(PencilBatch* B, const PencilSecretKey* sk, void* ws, size_t ws_bytes,
                                   uint64_t enc_seed, uint64_t mask_seed) {
  if (!B || !sk || !ws || sk->ctx != B->ctx || !aligned16(ws)) return PENCIL_E_ARG;
  if ((long long)ws_bytes < B->ws_bytes) return PENCIL_E_CAPACITY;
  for (const auto& u : B->user)
    if (!u.bound) return PENCIL_E_ARG;
  PencilCtx* ctx = B->ctx;
  DeviceGuard guard(ctx->device);
  const int L = ctx->dev.L, n = ctx->n;
  const long long lnw = (long long)L * n;
  char* w = reinterpret_cast<char*>(ws);
  const int nl = (int)B->plans.size();
  // the persistent multiply-accumulate tiles 2, 4 or 8 output columns per thread
  const int nt = ctx->dev.mac_nt == 0 ? 4 : ctx->dev.mac_nt;
  // encode and encrypt entries: one each per Alg. 1 layer, two each per Alg. 2 layer
  std::vector<ModeEncode::Params> enc;
  std::vector<ModeEncrypt::Params> encr;
  std::vector<SampleP> samp;
  std::vector<ModeMoPrep::Params> prep(nl);
  std::vector<ModeDecrypt::Params> dec(nl);
  std::vector<MaskPolyP> mpol(nl);
  std::vector<MoShareP> mosh(nl);
  std::vector<CombineP> comb(nl);
  std::vector<MacParams> mac(nl);
  std::vector<int2> it_pt, it_in, it_out, it_sh, it_prep;
  std::vector<int4> it_mac;
  bool has_dual = false;
  auto add_encode = [&](const Packing& pk, const Accessor& ac, const void* src, u64* dst, long long count) {
    ModeEncode::Params e;
    e.pk = pk;
    e.ac = ac;
    e.ac.ptr = reinterpret_cast<const u64*>(src);
    e.pt = dst;
    const int idx = (int)enc.size();
    enc.push_back(e);
    for (long long i = 0; i < count; ++i) it_pt.push_back(make_int2(idx, (int)i));
  };
  auto add_encrypt = [&](const Packing& pk, const Accessor& ac, const u64* src, u64* ct, int8_t* err, u64 seed,
                         long long count) {
    ModeEncrypt::Params e;
    e.pk = pk;
    e.ac = ac;
    e.ac.ptr = src;
    e.err = err;
    e.sk = sk->sk;
    e.ct = ct;
    e.seed = seed;
    const int idx = (int)encr.size();
    encr.push_back(e);
    samp.push_back(SampleP{seed, err});
    for (long long i = 0; i < count; ++i) it_in.push_back(make_int2(idx, (int)i));
  };
  for (int l = 0; l < nl; ++l) {
    const PencilPlan* P = B->plans[l];
    const auto& u = B->user[l];
    const auto& f = B->off[l];
    u64* pt = reinterpret_cast<u64*>(w + f.pt);
    u64* ct_in = reinterpret_cast<u64*>(w + f.ct_in);
    u64* ct_out = reinterpret_cast<u64*>(w + f.ct_out);
    int8_t* err = reinterpret_cast<int8_t*>(w + f.err);
    u64* p0 = reinterpret_cast<u64*>(w + f.p0);
    u64* mnt = reinterpret_cast<u64*>(w + f.mnt);
    u64* mpoly = reinterpret_cast<u64*>(w + f.mpoly);
    u64* yres = reinterpret_cast<u64*>(w + f.yres);
    const bool wg = P->role == PENCIL_ROLE_WGRAD;
    memset(&prep[l], 0, sizeof(ModeMoPrep::Params));
    prep[l].mpoly = mpoly;
    prep[l].out_mask = mnt;
    prep[l].seed = mask_seed + (u64)l;
    memset(&mac[l], 0, sizeof(MacParams));
    mac[l].a0 = ct_in;
    mac[l].a0_stride = 2 * lnw;
    mac[l].a1 = ct_in + lnw;
    mac[l].a1_stride = 2 * lnw;
    mac[l].b = pt;
    mac[l].b_stride = lnw;
    mac[l].mask = mnt;   // - NTT(Delta s) on store (Alg. 1 step 3, Alg. 2 step 2)
    mac[l].out = ct_out;
    mac[l].M = (int)P->c.M();
    mac[l].K = (int)P->c.K();
    mac[l].NC = P->c.NC;
    mac[l].lanes = (int)lnw;
    if (wg) {
      // Alg. 2: <gY>_0 at kernel positions and <X>_0 at input positions encoded;
      // Enc(<X>_1) and Enc(<gY>_1) (seed + 2^31); out = Enc(x1) gy0 + Enc(gy1) x0 - Delta s
      u64* ct_k = reinterpret_cast<u64*>(w + f.ct_k);
      int8_t* err_k = reinterpret_cast<int8_t*>(w + f.err_k);
      add_encode(P->pk_w, P->acc_w, u.g0, pt, P->pt);
      add_encode(P->pk_v, P->acc_v, u.x0, p0, P->ct_in);
      add_encrypt(P->pk_v, P->acc_v, u.x1, ct_in, err, enc_seed + (u64)l, P->ct_in);
      add_encrypt(P->pk_w, P->acc_w, u.g1, ct_k, err_k, enc_seed + (u64)l + (1ull << 31), P->pt);
      prep[l].n_in = 0;
      mac[l].pa = p0;
      mac[l].pa_stride = lnw;
      mac[l].cb0 = ct_k;
      mac[l].cb1 = ct_k + lnw;
      mac[l].cb_stride = 2 * lnw;
      has_dual = true;
    } else {
      // Alg. 1 (forward or input gradient): + NTT(Delta x0) on load
      add_encode(P->pk_w, P->acc_w, u.W, pt, P->pt);
      add_encrypt(P->pk_v, P->acc_v, u.x1, ct_in, err, enc_seed + (u64)l, P->ct_in);
      prep[l].pk = P->pk_v;
      prep[l].ac = P->acc_v;
      prep[l].ac.ptr = u.x0;
      prep[l].n_in = (int)P->ct_in;
      prep[l].out_in = p0;
      mac[l].p0 = p0;
      mac[l].p0_stride = lnw;
    }
    mpol[l] = MaskPolyP{P->pk_y, P->acc_y, mask_seed + (u64)l, mpoly};
    mosh[l] = wg ? MoShareP{mask_seed + (u64)l, P->out_elems, nullptr, 1, 1, u.y0}
                 : MoShareP{mask_seed + (u64)l, P->out_elems, u.bias, P->hw, P->co_out, u.y0};
    dec[l].ct = ct_out;
    dec[l].sk = sk->sk;
    dec[l].out = yres;
    dec[l].skip_c0 = 0;
    comb[l] = CombineP{P->pk_y, P->acc_y, yres, u.y1};
    for (long long i = 0; i < P->ct_out; ++i) it_out.push_back(make_int2(l, (int)i));
    for (long long i = 0; i < prep[l].n_in + P->ct_out; ++i) it_prep.push_back(make_int2(l, (int)i));
    for (long long c = 0; c < (P->out_elems + 1023) / 1024; ++c) it_sh.push_back(make_int2(l, (int)c));
    const int lane_blocks = (int)((lnw + 127) / 128);
    for (long long m = 0; m < P->c.M(); ++m)
      for (int n0 = 0; n0 < P->c.NC; n0 += nt)
        for (int lb = 0; lb < lane_blocks; ++lb) it_mac.push_back(make_int4(l, (int)m, n0, lb));
  }
  if (!ctx->dev.mac_split) return PENCIL_E_UNIMPL;
  std::vector<char> blob;
  size_t at = 0, o_enc, o_encr, o_prep, o_dec, o_samp, o_mpol, o_mosh, o_comb, o_mac, o_pt, o_in, o_out, o_sh,
         o_iprep, o_imac, o_words;
  put(blob, at, enc, o_enc);
  put(blob, at, encr, o_encr);
  put(blob, at, prep, o_prep);
  put(blob, at, dec, o_dec);
  put(blob, at, samp, o_samp);
  put(blob, at, mpol, o_mpol);
  put(blob, at, mosh, o_mosh);
  put(blob, at, comb, o_comb);
  put(blob, at, mac, o_mac);
  put(blob, at, it_pt, o_pt);
  put(blob, at, it_in, o_in);
  put(blob, at, it_out, o_out);
  put(blob, at, it_sh, o_sh);
  put(blob, at, it_prep, o_iprep);
  put(blob, at, it_mac, o_imac);
  std::vector<u64> words(nl + 2, 0);  // ready[nl], step, abort flag
  put(blob, at, words, o_words);
  cudaFree(B->d_mem);
  B->d_mem = nullptr;
  B->committed = false;
  CUDA_TRY(cudaMalloc(&B->d_mem, blob.size()));
  CUDA_TRY(cudaMemcpy(B->d_mem, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  char* d = reinterpret_cast<char*>(B->d_mem);
  BatchDev& D = B->dev;
  const int withhold = D.withhold;
  memset(&D, 0, sizeof(D));
  D.n_layers = nl;
  D.encode = reinterpret_cast<const ModeEncode::Params*>(d + o_enc);
  D.encrypt = reinterpret_cast<const ModeEncrypt::Params*>(d + o_encr);
  D.prep = reinterpret_cast<const ModeMoPrep::Params*>(d + o_prep);
  D.decrypt = reinterpret_cast<const ModeDecrypt::Params*>(d + o_dec);
  D.sample = reinterpret_cast<const SampleP*>(d + o_samp);
  D.maskpoly = reinterpret_cast<const MaskPolyP*>(d + o_mpol);
  D.moshare = reinterpret_cast<const MoShareP*>(d + o_mosh);
  D.combine = reinterpret_cast<const CombineP*>(d + o_comb);
  D.mac = reinterpret_cast<const MacParams*>(d + o_mac);
  D.items_pt = reinterpret_cast<const int2*>(d + o_pt);
  D.n_pt = (long long)it_pt.size();
  D.items_in = reinterpret_cast<const int2*>(d + o_in);
  D.n_in = (long long)it_in.size();
  D.items_out = reinterpret_cast<const int2*>(d + o_out);
  D.n_out = (long long)it_out.size();
  D.items_prep = reinterpret_cast<const int2*>(d + o_iprep);
  D.n_prep = (long long)it_prep.size();
  D.items_share = reinterpret_cast<const int2*>(d + o_sh);
  D.n_share = (long long)it_sh.size();
  D.items_mac = reinterpret_cast<const int4*>(d + o_imac);
  D.n_mac = (long long)it_mac.size();
  D.ready = reinterpret_cast<u64*>(d + o_words);
  D.step = D.ready + nl;
  D.abort_flag = reinterpret_cast<int*>(D.ready + nl + 1);
  D.withhold = withhold;
  D.mac_nt = nt;
  D.has_dual = has_dual ? 1 : 0;
  CUDA_TRY(batch_mac_blocks(ctx->dev, nt, D.has_dual, &D.mac_blocks));
  B->ws = w;
  B->mac_nt = ctx->dev.mac_nt;
  B->committed = true;
  return PENCIL_OK;
}

extern "C" int pencil_batch_forward(PencilCtx* ctx, PencilBatch* B, void* stream) {
  if (!ctx || !B || B->ctx != ctx) return PENCIL_E_ARG;
  if (!B->committed || B->mac_nt != ctx->dev.mac_nt) return PENCIL_E_ARG;   // re-commit after re-tuning
  DeviceGuard guard(ctx->device);
  CUDA_TRY(launch_batch_forward(ctx->dev, B->dev, (cudaStream_t)stream));
  return PENCIL_OK;
}

extern "C" int pencil_batch_set_step(PencilBatch* B, uint64_t step) {
  if (!B || !B->committed) return PENCIL_E_ARG;
  DeviceGuard guard(B->ctx->device);
  const u64 words[2] = {step, 0};
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(B->dev.step, words, sizeof(words), cudaMemcpyHostToDevice));
  return PENCIL_OK;
}

extern "C" int pencil_batch_read(const PencilBatch* B, int32_t layer, int32_t which, uint64_t* dst, void* stream) {
  if (!B || !dst || layer < 0 || layer >= (int)B->plans.size() || !B->committed) return PENCIL_E_ARG;
  const auto& f = B->off[layer];
  const PencilPlan* P = B->plans[layer];
  const long long lnb = (long long)B->ctx->dev.L * B->ctx->n * 8;
  long long o, bytes;
  switch (which) {
    case PENCIL_BATCH_PT:
      o = f.pt;
      bytes = P->pt * lnb;
      break;
    case PENCIL_BATCH_CT_IN:
      o = f.ct_in;
      bytes = P->ct_in * 2 * lnb;
      break;
    case PENCIL_BATCH_CT_OUT:
      o = f.ct_out;
      bytes = P->ct_out * 2 * lnb;
      break;
    case PENCIL_BATCH_CT_KERNEL:
      if (P->role != PENCIL_ROLE_WGRAD) return PENCIL_E_ARG;
      o = f.ct_k;
      bytes = P->pt * 2 * lnb;
      break;
    default:
      return PENCIL_E_ARG;
  }
  DeviceGuard guard(B->ctx->device);
  CUDA_TRY(cudaMemcpyAsync(dst, B->ws + o, (size_t)bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return PENCIL_OK;
}

extern "C" int pencil_batch_withhold(PencilBatch* B, int32_t layer) {
  if (!B || layer < -1 || layer >= (int)B->plans.size()) return PENCIL_E_ARG;
  B->dev.withhold = layer;
  return PENCIL_OK;
}
