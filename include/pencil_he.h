/*
 * pencil_he.h -- C ABI of the GB300 (sm_103a) homomorphic linear-layer hot path
 * of Pencil (NDSS 2024): BFV with RNS limbs, negacyclic NTT, coefficient
 * packings of Appendix A, Algorithm 1 (forward / input gradient) and
 * Algorithm 2 (weight-gradient cross terms) between a data owner (DO) and a
 * model owner (MO).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Return value: PENCIL_OK (0) or a negative PENCIL_E_* code.  Arguments are
 *   validated on the host before anything is enqueued; on error nothing has
 *   been launched.  Work is asynchronous on `stream` (a cudaStream_t passed as
 *   void*; NULL = legacy default stream).  Device-detected conditions (noise
 *   check) are OR-ed into a per-context status word read by pencil_sync_status.
 * - Every `uint64_t*` / `int64_t*` / `void* ws` argument is DEVICE memory owned
 *   by the caller, on the context's device.  The library never frees caller
 *   memory.  Handles (PencilCtx, PencilSecretKey, PencilPlan) are owned by the
 *   library and released with the matching *_destroy call.
 * - Ring layouts.  N = 2^log_n slots, L RNS limbs.
 *     ciphertext  uint64[2][L][N]  (c0, c1), NTT (evaluation) form, canonical in [0, q_i)
 *     plaintext   uint64[L][N]     NTT form, canonical
 *   Arrays of ciphertexts / plaintexts are contiguous: [count][2][L][N] / [count][L][N].
 *   NTT slot i of limb j holds a(psi_j^(2 brv(i) + 1)) mod q_j, brv = bit reversal.
 * - Shares and masks are Z_t values (t = 2^t_bits) stored in uint64, row-major in
 *   the user's layout: FC input [B][n_i], output [B][n_o]; conv input
 *   [B][C_in][H][W], output [B][C_out][H_out][W_out]; weights int64 (signed,
 *   any value is read mod t) [n_o][n_i] or [C_out][C_in][s][s].
 * - `ws` is scratch device memory of at least the size reported for that call
 *   by pencil_plan_sizes; its contents on entry are ignored.
 */
#ifndef PENCIL_HE_H
#define PENCIL_HE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define PENCIL_OK 0
#define PENCIL_E_ARG (-1)      /* null pointer, bad enum, bad seed use        */
#define PENCIL_E_SHAPE (-2)    /* layer shape invalid or inconsistent         */
#define PENCIL_E_PARAMS (-3)   /* unsupported N / limb count / prime size / t */
#define PENCIL_E_CAPACITY (-4) /* partition exceeds N or workspace too small  */
#define PENCIL_E_NOISE (-5)    /* decryption noise above q/(4t) (status word) */
#define PENCIL_E_TIMEOUT (-6)  /* a bounded device wait gave up (status word) */
#define PENCIL_E_CUDA (-7)     /* a CUDA runtime call failed                  */
#define PENCIL_E_UNIMPL (-8)   /* combination not implemented                 */

typedef struct PencilCtx PencilCtx;
typedef struct PencilSecretKey PencilSecretKey;
typedef struct PencilPublicKey PencilPublicKey;
typedef struct PencilPlan PencilPlan;

/* BFV instance {N, t, q} (Sec. 2.2) with q the product of `num_primes` RNS
 * limbs (Sec. 5 "RNS Decomposition"): the largest primes below 2^prime_bits
 * that are 1 mod 2N, in descending order.  Supported: log_n in {12, 13, 14},
 * num_primes in [1, 4], prime_bits in [30, 60], t_bits in [8, 60].  The
 * encryption error is a discrete Gaussian with sigma = 3.2 on [-19, 19].
 * Throughout, "Delta m" for a message m in [0, t) denotes the BFV scaling
 * round(q m / t) = floor(q / t) m + round((q mod t) m / t): a plaintext
 * multiple of such a ciphertext then carries no (q mod t)-sized overflow
 * term, which keeps products of two uniform Z_t values decryptable (Alg. 2's
 * cross terms at t = 2^59, q ~ 2^180). */
typedef struct {
  int32_t log_n;
  int32_t num_primes;
  int32_t prime_bits;
  int32_t t_bits;
} PencilParams;

/* Creates a context on CUDA device `device`: primes, NTT tables (psi_i = the
 * smallest primitive 2N-th root of unity mod q_i), RNS constants.
 * Allocates a few MB of device memory (freed by pencil_ctx_destroy). */
int pencil_ctx_create(const PencilParams* params, int device, PencilCtx** out);
int pencil_ctx_destroy(PencilCtx* ctx);
/* Copies the L primes and roots (host arrays of length num_primes). */
int pencil_ctx_primes(const PencilCtx* ctx, uint64_t* primes, uint64_t* psis);
/* Tuning knobs of a context (chosen by the autotuner; results never depend on them).
 * PENCIL_TUNE_NTT_LOG_RADIX: log2 of the coefficients each thread holds in the
 * NTT kernels, i.e. the radix of one shared-memory round: 4 or 5 (default 4
 * up to N = 8192, where two transforms share an SM; 5 above).
 * PENCIL_TUNE_MAC_COLUMNS: output ciphertexts per thread of the ct x pt
 * multiply-accumulate reading operands straight from L2: 2, 4 or 8; or 0: the
 * shared-memory staged kernel (each CTA stages one input block of 32 slots for
 * a 64-pair output block; each operand word read once per CTA).
 * PENCIL_TUNE_MAC_STAGING (columns 2, 4, 8): 0 = every thread copies its own
 * operand words a few input blocks ahead (cp.async ring); 1 = one producer
 * warp per CTA copies whole 1 KB operand rows with bulk asynchronous copies
 * (cp.async.bulk + mbarrier), the other warps only multiply.
 * PENCIL_TUNE_NTT_ARITH: butterfly arithmetic of the NTT kernels: 0 = Shoup
 * products with Harvey's lazy butterflies (any prime); 1 = pseudo-Mersenne
 * products (y w = y0 w + y1 (2^32 w mod q), folded with 2^60 = c and
 * 2^64 = 16 c mod q) with lazily growing values, for contexts whose primes are
 * all q = 2^60 - c with c < 2^24 (every 60-bit parameter set; the default
 * there), PENCIL_E_PARAMS otherwise. */
enum {
  PENCIL_TUNE_NTT_LOG_RADIX = 0,
  PENCIL_TUNE_MAC_COLUMNS = 1,
  PENCIL_TUNE_MAC_STAGING = 2,
  PENCIL_TUNE_NTT_ARITH = 3
};

/* Noise flooding of the ciphertexts the MO returns (circuit privacy; the paper
 * is silent, no counterpart): with bits > 0, every later he_linear_forward(_prepare)
 * and he_linear_backward (and batch commit) adds NTT(f) to each output
 * ciphertext, f_i uniform in [-2^bits, 2^bits) from Philox (key (mask_seed, 6),
 * counter (i / 4, output ciphertext index, 0, 0), word i % 4; for a batch,
 * mask_seed + layer).  Decrypted shares are unchanged.  bits = 0 turns it off.
 * Errors: PENCIL_E_ARG for bits outside [0, 62], PENCIL_E_PARAMS when
 * log2 q - t_bits - bits < 8 (no noise room). */
int pencil_ctx_flooding(PencilCtx* ctx, int32_t bits);
int pencil_ctx_tune(PencilCtx* ctx, int32_t knob, int32_t value);
int pencil_ctx_get_tune(const PencilCtx* ctx, int32_t knob, int32_t* value);

/* Reads and clears the device status word (synchronises the device):
 * *status = 0, or a PENCIL_E_* code recorded by a kernel (PENCIL_E_TIMEOUT
 * takes precedence over PENCIL_E_NOISE, which it usually causes). */
int pencil_sync_status(PencilCtx* ctx, int32_t* status);

/* DO side: ternary secret key s_i = (w_i mod 3) - 1, w = Philox4x64-10 word
 * (key = (seed, 1), counter = (i/4, 0, 0, 0), word i%4), kept as NTT(s) per
 * limb on the device (owned by the handle). */
int pencil_keygen(PencilCtx* ctx, uint64_t seed, PencilSecretKey** out, void* stream);
int pencil_sk_destroy(PencilSecretKey* sk);

/* DO side: BFV public key (the scheme of Sec. 2.2 [Fan-Vercauteren]; the
 * paper's security simulators hand pk between the parties), for
 * encrypt_share_pk:
 *   p1 = a,  a[i] uniform mod q_j as encrypt_share's a, on Philox key (seed, 7)
 *            with ciphertext index 0: counter (i/4, 0, j, 0), word i%4 (rejected
 *            words replaced from counter (i, 0, j, r)) -- NTT form;
 *   p0 = -(a * NTT(s)) - NTT(e),  e[i] from the CDT (as encrypt_share's errors)
 *            on Philox key (seed, 8), counter (i/4, 0, 0, 0), word i%4.
 * Device memory owned by the handle ([2][L][N] values with Shoup companions,
 * plus N bytes of scratch).  Errors: PENCIL_E_ARG (null or foreign sk),
 * PENCIL_E_CUDA (allocation or launch). */
int pencil_pk_keygen(PencilCtx* ctx, const PencilSecretKey* sk, uint64_t seed, PencilPublicKey** out,
                     void* stream);
int pencil_pk_destroy(PencilPublicKey* pk);

/* ---------------------------------------------------------------- plans */
enum { PENCIL_FC = 0, PENCIL_CONV = 1 };
/* Role of a plan: the forward product (Alg. 1), the input gradient
 * grad_X = W (.)_x grad_Y (Sec. 3.2.2, Alg.-1-like) or the weight gradient
 * cross terms (Alg. 2). */
enum { PENCIL_ROLE_FWD = 0, PENCIL_ROLE_DGRAD = 1, PENCIL_ROLE_WGRAD = 2 };
/* Operand positions of a plan: ciphertext-input positions ct_in[m*K+k]
 * (packing pi_v) or kernel positions pt[k*NC+n] (packing pi_W). */
enum { PENCIL_OPERAND_INPUT = 0, PENCIL_OPERAND_KERNEL = 1 };

/* Layer: FC (c_in = n_i, c_out = n_o, height = width = kernel = 1, pad = 0) or
 * stride-1 2-D convolution with zero padding `pad` on an height x width input. */
typedef struct {
  int32_t kind;
  int32_t batch;
  int32_t c_in;
  int32_t c_out;
  int32_t height;
  int32_t width;
  int32_t kernel;
  int32_t pad;
} PencilLayerDesc;

/* Block partition of the correlation (Appendix A: "larger inputs or weights
 * could be partitioned"): bb batch items, cib input channels and cob output
 * channels per polynomial; th x tw output tile; kth x ktw kernel tile.
 * Valid iff bb*cob*cib*(th+kth-1)*(tw+ktw-1) <= N. */
typedef struct {
  int32_t bb, cib, cob, th, tw, kth, ktw;
} PencilPartition;

typedef struct {
  PencilPartition part;
  int64_t ct_in;         /* ciphertexts at input positions  (M*K)      */
  int64_t pt;            /* plaintexts at kernel positions  (K*NC)     */
  int64_t ct_out;        /* output ciphertexts              (M*NC)     */
  int64_t products;      /* ct x pt products per call       (M*K*NC)   */
  int64_t ct_words;      /* uint64 words per ciphertext = 2*L*N        */
  int64_t pt_words;      /* uint64 words per plaintext  = L*N          */
  int64_t out_elems;     /* elements of the user's output tensor       */
  int64_t ws_encrypt;    /* bytes of ws for encrypt_share (either operand) */
  int64_t ws_forward;    /* bytes of ws for he_linear_forward          */
  int64_t ws_backward;   /* bytes of ws for he_linear_backward (this plan's role) */
  int64_t ws_decrypt;    /* bytes of ws for decrypt_to_share           */
  int64_t ws_encrypt_pk; /* bytes of ws for encrypt_share_pk (either operand) */
} PencilPlanSizes;

/* Plans `role` of `layer`.  `part` = NULL lets the planner choose the
 * partition with its cost model (bytes moved and NTT / multiply counts);
 * otherwise `part` is used as given (PENCIL_E_CAPACITY if it does not fit).
 * Builds the packing index tables on the device (owned by the plan). */
int pencil_plan_linear(PencilCtx* ctx, const PencilLayerDesc* layer, int32_t role,
                       const PencilPartition* part, PencilPlan** out);
int pencil_plan_destroy(PencilPlan* plan);

/* A slice of a FWD or DGRAD plan over the output rows m in [m_first, m_first +
 * m_count) of its partition (m = batch block x spatial tile, the row index of
 * ct_in[m * K + k] and ct_out[m * NC + n]), for streaming a layer through the
 * protocol block by block (no counterpart in the paper, which describes whole
 * layers).  A slice shares its parent's tables (destroy it before the parent)
 * and takes the parent's full-size buffers and workspaces (pencil_plan_sizes
 * reports the parent's sizes); with it, encrypt_share (INPUT) and
 * encode_weights (INPUT) touch only input polynomials [m_first K, (m_first +
 * m_count) K), he_linear_forward_apply only output polynomials [m_first NC,
 * (m_first + m_count) NC), decrypt_to_share only those outputs (and the share
 * elements they carry); he_linear_forward_prepare always prepares the whole
 * layer.  Every polynomial is bit-identical to the whole-plan call's.  Calls on
 * disjoint slices may run concurrently on different streams: concurrent
 * encryptions may share one workspace, concurrent decryptions another, but an
 * encryption and a decryption that may overlap need separate workspaces (both
 * use theirs from offset 0).
 * encrypt_share (KERNEL), encrypt_share_noalloc, he_linear_backward and the
 * batch API take whole plans only (PENCIL_E_ARG).  Errors: PENCIL_E_ARG for a
 * WGRAD plan or a slice of a slice, PENCIL_E_SHAPE for an empty or
 * out-of-range row range. */
int pencil_plan_slice(const PencilPlan* plan, int32_t m_first, int32_t m_count, PencilPlan** out);
/* Up to max_count distinct partitions of `role` of `layer`, cheapest first by
 * the planner's cost model (the first is the planner's own choice); the
 * autotuner times them.  Host only. */
int pencil_plan_candidates(PencilCtx* ctx, const PencilLayerDesc* layer, int32_t role, int32_t max_count,
                           PencilPartition* out, int32_t* count);
int pencil_plan_sizes(const PencilPlan* plan, PencilPlanSizes* sizes);

/* ---------------------------------------------------------------- hot path */

/* MO: plaintext encoding (Appendix A pi_W / pi_v).  `values` are read mod t and
 * lifted through their centred representative in [-t/2, t/2) to every limb,
 * then transformed.  operand = KERNEL: writes pt[K*NC][L][N] from the role's
 * kernel tensor (fwd/dgrad: the weights W; wgrad: the MO share <gY>_0).
 * operand = INPUT: writes [M*K][L][N] from the role's input tensor (wgrad: the
 * MO share <X>_0).  `values` is int64 for W and uint64 Z_t shares otherwise
 * (same bits). */
int encode_weights(PencilCtx* ctx, const PencilPlan* plan, int32_t operand,
                   const int64_t* values, uint64_t* pt, void* stream);

/* DO: symmetric BFV encryption of a packed share (Sec. 2.2, Alg. 1 step 1,
 * Alg. 2 step 1).  For ciphertext index c (0-based within this call):
 *   c1 = a,  a[i] = w mod q_j, w = word i%4 of Philox (key (seed, 2), counter
 *             (i/4, c, j, 0)) if w < floor(2^64 / q_j) q_j, else word 0 of the first
 *             accepted block at counter (i, c, j, r), r = 1, 2, ... -- exactly
 *             uniform, NTT form;
 *   c0 = NTT(Delta m + e) - a * NTT(s)  (Delta m = round(q m / t), above),
 *   e[i] from the CDT on Philox (key (seed, 3), counter (i/4, c, 0, 0), word i%4).
 * operand INPUT packs `share` with pi_v into ct[M*K]; operand KERNEL packs it
 * with pi_W into ct[K*NC] (Alg. 2's Enc(<gY>_1)).  ws >= ws_encrypt bytes. */
int encrypt_share(PencilCtx* ctx, const PencilSecretKey* sk, const PencilPlan* plan,
                  int32_t operand, const uint64_t* share, uint64_t seed, uint64_t* ct,
                  void* ws, size_t ws_bytes, void* stream);

/* Public-key BFV encryption of a packed share: the same packing, operands,
 * slices and output layout as encrypt_share, with the randomness of
 * ciphertext index c (0-based within the plan's operand):
 *   u[i]  = (w mod 3) - 1,  Philox key (seed, 9),  counter (i/4, c, 0, 0), word i%4;
 *   e1[i] = CDT on Philox key (seed, 3),  e2[i] = CDT on Philox key (seed, 10),
 *           counter (i/4, c, 0, 0), word i%4;
 *   c0 = NTT(Delta m + e1) + NTT(u) * p0,   c1 = NTT(e2) + NTT(u) * p1,
 * so c0 + c1 s = Delta m + e1 - u e + e2 s (e the key's error).  Three
 * kernels: the samples (int8), NTT(u) into ws, and one NTT pass over both
 * components of every ciphertext with the products fused into its epilogue.
 * ws >= ws_encrypt_pk bytes, 16-byte aligned.  Errors as encrypt_share;
 * PENCIL_E_ARG for a key of another context. */
int encrypt_share_pk(PencilCtx* ctx, const PencilPublicKey* pk, const PencilPlan* plan, int32_t operand,
                     const uint64_t* share, uint64_t seed, uint64_t* ct, void* ws, size_t ws_bytes, void* stream);

/* encrypt_share without a workspace argument and without any allocation.
 * (The paper has no counterpart: this is a deployment variant of the call
 * above.)  It exists for data-owner code that must not allocate device memory
 * when it encrypts: code running under a caching allocator that has already
 * reserved the device's memory, a serving loop in which cudaMalloc's implicit
 * device-wide synchronisation would stall every other stream, or embedders
 * that have no device allocator of their own.
 * Scratch: the sampled errors (count x N bytes, count = ct_in for INPUT,
 * pt for KERNEL) live in a file-scope static device array of 8 MiB
 * (8388608 bytes) inside the library, which every GPU that loads the
 * library holds until the process exits.  Larger calls (e.g. more than 1024
 * ciphertexts at N = 8192) return PENCIL_E_CAPACITY, print the reason on
 * stderr and launch nothing.
 * The first call with each context looks up the array's device address
 * (cudaGetSymbolAddress, with the context's device current) and keeps it with
 * the context; make that first call before any stream capture.  Every call on
 * a device shares the one array,
 * which keeps the previous call's contents: each call writes every byte it
 * then reads, so nothing needs clearing, but calls that overlap on the GPU
 * (different streams, or threads) race on it -- the caller must serialise
 * them.  Outputs are bit-identical to encrypt_share with the same arguments. */
int encrypt_share_noalloc(PencilCtx* ctx, const PencilSecretKey* sk, const PencilPlan* plan, int32_t operand,
                          const uint64_t* share, uint64_t seed, uint64_t* ct, void* stream);

/* MO: Algorithm 1 steps 2-3 for a FWD or DGRAD plan.
 *   ct_out[m,n] = sum_k (ct_in[m,k] + Delta*pi_v(x0)[m,k]) * pt[k,n] - Delta * s
 * with s one Z_t value per output element from Philox (key (mask_seed, 4),
 * counter (flat/4, 0, 0, 0), word flat%4; flat = row-major index in the output)
 * and, at coefficients carrying no output, (key (mask_seed, 5), counter
 * (i/4, ct_out index, 0, 0)).  Writes the MO share y0[flat] = s + bias[o]
 * (bias: nullable, Z_t values [n_o] / [C_out], FWD only).  ct_in is not
 * modified.  ws >= ws_forward bytes. */
int he_linear_forward(PencilCtx* ctx, const PencilPlan* plan, const uint64_t* ct_in,
                      const uint64_t* pt, const uint64_t* x0, const uint64_t* bias,
                      uint64_t mask_seed, uint64_t* ct_out, uint64_t* y0,
                      void* ws, size_t ws_bytes, void* stream);

/* he_linear_forward in two calls, so that the MO's ciphertext-independent work
 * runs before (or concurrently with) the DO's encryption:
 * he_linear_forward_prepare draws s, writes y0 and leaves NTT(Delta pi_v(x0))
 * and NTT(Delta s) in ws; he_linear_forward_apply (same plan, same ws, ordered
 * after the prepare on the GPU) computes ct_out from ct_in and pt.  ws is read,
 * not modified, by the apply.  The pair's outputs are bit-identical to
 * he_linear_forward with the same arguments.  Same argument rules. */
int he_linear_forward_prepare(PencilCtx* ctx, const PencilPlan* plan, const uint64_t* x0,
                              const uint64_t* bias, uint64_t mask_seed, uint64_t* y0,
                              void* ws, size_t ws_bytes, void* stream);
int he_linear_forward_apply(PencilCtx* ctx, const PencilPlan* plan, const uint64_t* ct_in,
                            const uint64_t* pt, uint64_t* ct_out,
                            void* ws, size_t ws_bytes, void* stream);

/* MO: backward pass of one layer (Sec. 3.2.2).
 * Input gradient (plan_dgrad, nullable to skip): Algorithm 1 on the DGRAD plan,
 *   ct_gx = sum_k (ct_gy1_d + Delta pi_v(gy0)) * pt_wt - Delta s_x, gx0 = s_x
 *   (pt_wt = encode_weights(plan_dgrad, KERNEL, W)).
 * Weight gradient (plan_wgrad, nullable to skip): Algorithm 2 steps 2-3,
 *   ct_gw[m,n] = sum_k Enc(<X>_1)[m,k] * NTT(pi_W(<gY>_0))[k,n]
 *              + Enc(<gY>_1)[k,n] * NTT(pi_v(<X>_0))[m,k]  - Delta s_w,
 *   gw_mask = s_w (the MO keeps it; grad_W = decrypted + s_w + local terms).
 *   ct_x1_w = encrypt_share(plan_wgrad, INPUT, <X>_1), ct_gy1_w =
 *   encrypt_share(plan_wgrad, KERNEL, <gY>_1); gy0 / x0 are the MO's shares.
 * ws >= ws_backward of plan_dgrad + ws_backward of plan_wgrad. */
int he_linear_backward(PencilCtx* ctx, const PencilPlan* plan_dgrad, const PencilPlan* plan_wgrad,
                       const uint64_t* ct_gy1_d, const uint64_t* pt_wt,
                       const uint64_t* ct_x1_w, const uint64_t* ct_gy1_w,
                       const uint64_t* gy0, const uint64_t* x0,
                       uint64_t mask_seed_x, uint64_t mask_seed_w,
                       uint64_t* ct_gx, uint64_t* gx0, uint64_t* ct_gw, uint64_t* gw_mask,
                       void* ws, size_t ws_bytes, void* stream);

/* DO: decryption and unpacking (Alg. 1 step 4): x = INTT(c0 + c1 * NTT(s)) per
 * limb, m = round(t x / q) mod t computed from the RNS residues (no big
 * integers), scattered with pi_y^{-1} into y1 (user output layout).  With
 * check_noise != 0, coefficients whose t x / q lies 1/4 or more away from an
 * integer set PENCIL_E_NOISE in the status word.  ws >= ws_decrypt bytes. */
int decrypt_to_share(PencilCtx* ctx, const PencilSecretKey* sk, const PencilPlan* plan,
                     const uint64_t* ct_out, uint64_t* y1, int32_t check_noise,
                     void* ws, size_t ws_bytes, void* stream);

/* Compact send form of returned ciphertexts (communication reduction: the
 * coefficients that carry no output are dropped before the MO sends them).
 * compact_returned (MO) writes c0c[j][flat] = coefficient of INTT(c0) mod q_j
 * at the coefficient carrying output element flat ([L][out_elems] uint64,
 * out_elems from pencil_plan_sizes, flat = the element's row-major index in
 * the output tensor); c1 stays in ct_out in NTT form.  What travels is then
 * the c1 halves of ct_out (L N words per ciphertext) and c0c (L words per
 * output) instead of 2 L N words per ciphertext.  One INTT per ciphertext.
 * decrypt_compact_to_share (DO) reads only the c1 halves of ct_out and c0c
 * and writes the same y1 as decrypt_to_share would on the whole ciphertexts
 * (same noise check, same ws).  Both take slices (their output rows only; c0c
 * is indexed by absolute flat).  Errors as decrypt_to_share. */
int compact_returned(PencilCtx* ctx, const PencilPlan* plan, const uint64_t* ct_out, uint64_t* c0c, void* stream);
int decrypt_compact_to_share(PencilCtx* ctx, const PencilSecretKey* sk, const PencilPlan* plan,
                             const uint64_t* ct_out, const uint64_t* c0c, uint64_t* y1, int32_t check_noise,
                             void* ws, size_t ws_bytes, void* stream);

/* Plaintext ring operator of the plan's role over Z_t (uint64 wrap-around,
 * exact because t divides 2^64): out = addend + addend2 + op(kernel_operand,
 * input_operand) mod t, with op = W o X (FWD), grad_X = W (.)_x grad_Y (DGRAD),
 * grad_W = grad_Y (.) X (WGRAD).  This is Alg. 2's local term
 * <gY>_j (.) <X>_j (steps 4 and 6) when called on one party's shares, with the
 * decrypted cross term (DO) or the decrypted value plus mask (MO) as addend.
 * Operands in the user's layouts: kernel_operand = W (FWD, DGRAD; int64 bits) or
 * grad_Y (WGRAD); input_operand = X (FWD, WGRAD) or grad_Y (DGRAD).  The
 * addends (output layout) are nullable; out may alias either. */
int pencil_ring_linear(PencilCtx* ctx, const PencilPlan* plan, const uint64_t* kernel_operand,
                       const uint64_t* input_operand, const uint64_t* addend, const uint64_t* addend2,
                       uint64_t* out, void* stream);

/* Bias gradient (Sec. 3.2.2, its footnote): out[o] = sum over the batch and
 * the output positions of g mod t, g in the forward output layout of the plan's
 * layer ([B][n_o] or [B][C_out][H_out][W_out]); each party sums its own share. */
int pencil_bias_grad(PencilCtx* ctx, const PencilPlan* plan, const uint64_t* g, uint64_t* out, void* stream);

/* Linear combination over Z_t (t = 2^t_bits of ctx), the HE-free online phase
 * of the preprocessing protocol (Alg. 3: masked operands u - sum k_i u'_i and
 * shares sum_i k_i <u'_i o v'_j>):
 *   out[e] = addend[e] + s * sum_{i < terms} scalars[i] * src[src_offset
 *            + (e / inner) * outer_stride + (e % inner) + i * term_stride]  mod t,
 * e in [0, count), s = -1 if negate else +1.  src, addend (nullable), out: device
 * arrays of Z_t values (out may alias addend, not src); scalars: host array of
 * terms <= 64 values.  Errors: PENCIL_E_ARG for null pointers, negative sizes,
 * inner < 1 or too many terms. */
int pencil_lincomb(PencilCtx* ctx, const uint64_t* src, int64_t src_offset, int64_t inner, int64_t outer_stride,
                   int64_t term_stride, const uint64_t* scalars, int32_t terms, const uint64_t* addend,
                   int32_t negate, uint64_t* out, int64_t count, void* stream);
/* The same with two term indices (a double sum over m x m blocks in one pass,
 * e.g. the shares sum_{i,j} l_j k_i <u'_i o v'_j> of Alg. 3's online phase):
 *   out[e] = addend[e] + s * sum_{i2 < terms2} sum_{i < terms}
 *            scalars[i2 * terms + i] * src[src_offset + (e / inner) * outer_stride
 *            + (e % inner) + i * term_stride + i2 * term_stride2]  mod t,
 * terms * terms2 <= 64 scalars.  Errors as pencil_lincomb (also terms2 < 1). */
int pencil_lincomb2(PencilCtx* ctx, const uint64_t* src, int64_t src_offset, int64_t inner, int64_t outer_stride,
                    int64_t term_stride, int32_t terms, int64_t term_stride2, int32_t terms2, const uint64_t* scalars,
                    const uint64_t* addend, int32_t negate, uint64_t* out, int64_t count, void* stream);

/* In-place batched negacyclic NTT (inverse = 0) or INTT (inverse = 1) of
 * `count` polynomials laid out [count][L][N], canonical in and out (Sec. 5 "NTT"). */
int pencil_ntt_batch(PencilCtx* ctx, uint64_t* polys, int64_t count, int32_t inverse, void* stream);

/* ---------------------------------------------------------------- batched layers
 * Many FWD plans of one context executed as one fixed launch sequence
 * (workload of many uneven layers, Sec. 3.2.1 applied layer by layer): every
 * stage of every layer in one multi-plan launch, and the ct x pt products of
 * all layers in ONE persistent launch over a (layer, block, output tile, slot
 * block) work list.  pencil_batch_forward launches kernels only (no
 * allocation, no copy), so a sequence of calls can be captured in a CUDA graph.
 * A device step counter, advanced by every call, re-keys the randomness: layer
 * l of call number k uses encryption seed enc_seed + l + (k << 32) and mask
 * seed mask_seed + l + (k << 32), i.e. exactly the per-layer calls
 * encrypt_share / he_linear_forward with those seeds; encode_weights and
 * decrypt_to_share complete the sequence.
 * The persistent multiply-accumulate waits (bounded by clock64, about 2 ms)
 * for each layer's ready word written after its input stages; on expiry it
 * sets PENCIL_E_TIMEOUT in the status word and abandons the remaining work
 * (the outputs of that call are then invalid). */
typedef struct PencilBatch PencilBatch;
enum { PENCIL_BATCH_PT = 0, PENCIL_BATCH_CT_IN = 1, PENCIL_BATCH_CT_OUT = 2, PENCIL_BATCH_CT_KERNEL = 3 };
/* plans: `count` whole plans of ctx, any role: a FWD or DGRAD plan is one Alg. 1
 * product (forward, or the input gradient W (.)_x grad_Y), a WGRAD plan one
 * Alg. 2 weight gradient (both cross terms).  A plan may appear several times.
 * So a training step's forward and backward products of every layer run as one
 * launch sequence. */
int pencil_batch_create(PencilCtx* ctx, const PencilPlan* const* plans, int32_t count, PencilBatch** out);
int pencil_batch_destroy(PencilBatch* batch);
/* Bytes of device workspace holding every layer's plaintexts and ciphertexts
 * (buffers with disjoint lifetimes inside one pencil_batch_forward share
 * memory: the mask polynomials and sampled errors sit in the output
 * ciphertexts' region until the multiply-accumulate writes it, and the
 * decryption residues in that of NTT(Delta x0) and NTT(Delta s)). */
int pencil_batch_workspace(const PencilBatch* batch, int64_t* bytes);
/* Device buffers of an Alg. 1 entry `layer` (FWD or DGRAD plan; user layouts as
 * for the per-layer calls): W, the DO's and MO's shares x1, x0 of the product's
 * input (X, or grad_Y for DGRAD), bias (FWD only, nullable), the output shares
 * y0 (MO), y1 (DO).  PENCIL_E_ARG for a WGRAD plan or a DGRAD bias. */
int pencil_batch_bind(PencilBatch* batch, int32_t layer, const int64_t* W, const uint64_t* x1, const uint64_t* x0,
                      const uint64_t* bias, uint64_t* y0, uint64_t* y1);
/* Device buffers of an Alg. 2 entry `layer` (WGRAD plan): shares gy0, gy1 of
 * grad_Y and x0, x1 of X; outputs gw_mask (the MO's mask s) and tilde (the
 * DO's decryption of the cross terms minus s), as he_linear_backward and
 * decrypt_to_share give them.  Enc(<X>_1) uses enc_seed + layer, Enc(<gY>_1)
 * enc_seed + layer + 2^31, the mask mask_seed + layer (plus step 2^32).
 * PENCIL_E_ARG for another role. */
int pencil_batch_bind_wgrad(PencilBatch* batch, int32_t layer, const uint64_t* gy0, const uint64_t* gy1,
                            const uint64_t* x0, const uint64_t* x1, uint64_t* gw_mask, uint64_t* tilde);
/* Builds the device work lists and parameters (allocates and copies: call it
 * before any capture).  Requires every layer bound, ws >= pencil_batch_workspace
 * bytes, and primes near 2^bits (the split multiply-accumulate; else
 * PENCIL_E_UNIMPL).  Re-commit after changing PENCIL_TUNE_MAC_COLUMNS. */
int pencil_batch_commit(PencilBatch* batch, const PencilSecretKey* sk, void* ws, size_t ws_bytes, uint64_t enc_seed,
                        uint64_t mask_seed);
/* One forward pass of every layer on `stream` (capturable). */
int pencil_batch_forward(PencilCtx* ctx, PencilBatch* batch, void* stream);
/* Sets the step counter (synchronises the device) and clears an earlier abort. */
int pencil_batch_set_step(PencilBatch* batch, uint64_t step);
/* Copies layer `layer`'s plaintexts / input / output ciphertexts (as left by the
 * last call) to `dst` (device memory of the plan's counts, stream-ordered).
 * For a WGRAD entry PT is the encoded <gY>_0 (pt count), CT_IN Enc(<X>_1),
 * CT_KERNEL Enc(<gY>_1) (pt count; WGRAD entries only), CT_OUT the cross terms. */
int pencil_batch_read(const PencilBatch* batch, int32_t layer, int32_t which, uint64_t* dst, void* stream);
/* Failure injection for tests: layer `layer`'s ready word is never written
 * (-1: none), so the multiply-accumulate times out instead of hanging. */
int pencil_batch_withhold(PencilBatch* batch, int32_t layer);

/* ---------------------------------------------------------------- profiling
 * Per-kernel timing with CUDA events recorded on the launch stream around every
 * kernel the context launches (not available inside CUDA-graph capture).
 * pencil_profile(ctx, 1) clears and starts recording, (ctx, 0) stops.
 * pencil_profile_read synchronises the recorded events and returns one entry
 * per kernel kind that launched: launches and summed milliseconds. */
enum {
  PENCIL_K_NTT_RAW = 0, PENCIL_K_INTT_RAW, PENCIL_K_NTT_ENCRYPT, PENCIL_K_NTT_ADDPLAIN, PENCIL_K_NTT_ENCODE,
  PENCIL_K_NTT_MASK, PENCIL_K_INTT_DECRYPT, PENCIL_K_NTT_KEYGEN, PENCIL_K_MAC, PENCIL_K_MAC_DUAL,
  PENCIL_K_SAMPLE_ERR, PENCIL_K_MASK_POLY, PENCIL_K_MO_SHARE, PENCIL_K_DECRYPT_COMBINE, PENCIL_K_RING,
  PENCIL_K_BIAS_GRAD, PENCIL_K_NTT_MO_PREP, PENCIL_K_LINCOMB, PENCIL_K_SAMPLE_PK, PENCIL_K_NTT_PK_U,
  PENCIL_K_NTT_ENCRYPT_PK, PENCIL_K_INTT_COMPACT, PENCIL_K_COUNT
};
typedef struct {
  int32_t kernel;   /* PENCIL_K_* */
  int32_t launches;
  double ms;
} PencilProfEntry;
int pencil_profile(PencilCtx* ctx, int32_t enable);
int pencil_profile_read(PencilCtx* ctx, PencilProfEntry* out, int32_t max_entries, int32_t* n_entries);

/* Multiply-pipe probe used to measure the integer roofline: `blocks` x
 * `threads` threads each run 8 independent register-only chains of `iters`
 * steps; which = 0: 32-bit multiply-add (mad.lo.u32), 1: 64-bit Shoup modular
 * multiply, 2: 32x32->64 multiply-add (mad.wide.u32), 3: 64x64->128
 * multiply-accumulate, 4: split-quotient Shoup multiply (mul_shoup3), 5: forward
 * butterfly on [0, 8q), 6: forward butterfly on [0, 4q) (Harvey), 7: inverse
 * butterfly on [0, 4q), 8: inverse butterfly on [0, 2q) (Harvey), 9: 32x32
 * high half (mul.hi.u32), 10: pseudo-Mersenne product (mul_fold, PTX), 11: the
 * same product written in C (mul_fold_c), 12: forward fold butterfly, 13: inverse
 * fold butterfly, 14: fold60 alone, 15: forward butterfly with mul_fold_c; for
 * 5-8 and 12, 13, 15 a step is one butterfly.  Times the launch with CUDA events on `stream` and returns
 * the elapsed milliseconds and the number of chain steps (threads * 8 * iters).
 * Synchronises `stream`. */
int pencil_mul_probe(PencilCtx* ctx, int32_t which, int64_t iters, int32_t blocks, int32_t threads, double* ms,
                     double* steps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PENCIL_HE_H */
