// Host-side launchers of the hot-path kernels (implemented in kernels.cu and
// ntt12.cu / ntt13.cu / ntt14.cu).
#pragma once
#include "ntt.cuh"

namespace pencil {

// Operands of the NTT-domain multiply-accumulate.  All arrays are indexed
// [poly][...][lanes]; `*_stride` is the distance in words between consecutive
// polynomials of that operand, lanes = L * N.
struct MacParams {
  const u64* a0;     // A[m, k] first component  (ciphertext c0, or c0 + Delta x0)
  i64 a0_stride;
  const u64* a1;     // A[m, k] second component (ciphertext c1)
  i64 a1_stride;
  const u64* b;      // B[k, n] plaintext
  i64 b_stride;
  const u64* pa;     // Alg. 2: A'[m, k] plaintext
  i64 pa_stride;
  const u64* cb0;    // Alg. 2: B'[k, n] ciphertext c0
  const u64* cb1;    //                      and c1
  i64 cb_stride;
  const u64* p0;     // Alg. 1: NTT(Delta x0)[m, k] added to A's first component on load (or null)
  i64 p0_stride;
  const u64* mask;   // Alg. 1 step 3: NTT(Delta s)[m * NC + n] ([lanes] each) subtracted from the
                     // first output component on store (or null)
  u64* out;          // [M * NC][2][lanes]
  int M, K, NC;
  int lanes;
  int m_base;
};

#define PENCIL_LINCOMB_MAX_TERMS 64
struct LincombP {
  const u64* src;
  long long off, inner, outer, tstride, count;
  long long tstride2;  // stride of the second term index (terms2 of them; 1: one-index form)
  const u64* addend;   // nullable
  u64* out;
  int terms, terms2, negate;
  u64 k[PENCIL_LINCOMB_MAX_TERMS];   // k[i2 * terms + i]
};
cudaError_t launch_lincomb(const LincombP& P, u64 t_mask, cudaStream_t s);

cudaError_t upload_cdt();
cudaError_t launch_mac(const DevCtx& ctx, const MacParams& P, bool dual, cudaStream_t s);
cudaError_t launch_sample_err(u64 seed, int first, int count, int n, int8_t* out, cudaStream_t s,
                              u64 dom = PENCIL_DOM_E);
cudaError_t launch_sample_pk(u64 seed, int first, int count, int n, int8_t* e1, int8_t* e2, int8_t* u,
                             cudaStream_t s);
cudaError_t launch_mask_poly(const DevCtx& ctx, const Packing& pk, const Accessor& ac, u64 seed, int count, u64* out,
                             cudaStream_t s);
cudaError_t launch_mo_share(u64 seed, long long count, u64 t_mask, const u64* bias, long long hw, int co, u64* y0,
                            cudaStream_t s);
cudaError_t launch_decrypt_combine(const DevCtx& ctx, const Packing& pk, const Accessor& ac, const u64* yres,
                                   int first, int count, int check, u64* y1, cudaStream_t s,
                                   const u64* c0c = nullptr, long long out_elems = 0);

// Plaintext correlation over Z_t of one plan role (see k_ring_* in kernels.cu).
struct RingParams {
  int4 kbound;        // (Co, Ci, KH, KW) of the role's kernel
  int Ho, Wo;         // output spatial size
  Accessor v, w, y;   // input, kernel and output views of the user's tensors
  const u64* addend;  // nullable, output layout
  const u64* addend2; // nullable, output layout
  u64* out;           // output layout
  long long outs;     // B * Co * Ho * Wo
  u64 t_mask;
};
cudaError_t launch_ring(const RingParams& P, cudaStream_t s);
cudaError_t launch_bias_grad(const u64* g, int B, int Co, long long hw, u64 t_mask, u64* out, cudaStream_t s);

// ---- batched layers: per-layer parameters of the non-NTT stages
struct SampleP {
  u64 seed;
  int8_t* err;        // [ct_in][N]
};
struct MaskPolyP {
  Packing pk;
  Accessor ac;
  u64 seed;
  u64* out;           // [ct_out][N]
};
struct MoShareP {
  u64 seed;
  long long count;
  const u64* bias;
  long long hw;
  int co;
  u64* y0;
};
struct CombineP {
  Packing pk;
  Accessor ac;
  const u64* yres;    // [ct_out][L][N]
  u64* y1;
};
// Device-resident description of one batch (all pointers are device memory).
struct BatchDev {
  int n_layers;
  const ModeEncode::Params* encode;
  const ModeEncrypt::Params* encrypt;
  const ModeMoPrep::Params* prep;    // NTT(Delta x0) and NTT(Delta s) of every layer
  const ModeDecrypt::Params* decrypt;
  const SampleP* sample;
  const MaskPolyP* maskpoly;
  const MoShareP* moshare;
  const CombineP* combine;
  const MacParams* mac;
  const int2* items_pt;
  long long n_pt;
  const int2* items_in;
  long long n_in;
  const int2* items_out;
  long long n_out;
  const int2* items_prep;   // (layer, polynomial): input polynomials, then output polynomials
  long long n_prep;
  const int2* items_share;
  long long n_share;
  const int4* items_mac;
  long long n_mac;
  int mac_blocks;
  int mac_nt;          // output columns per thread of the persistent multiply-accumulate: 2, 4 or 8
  int has_dual;        // some layer is an Alg. 2 weight gradient (two products per input block)
  u64* ready;          // [n_layers]
  u64* step;           // replay counter
  int* abort_flag;
  int withhold;        // layer whose ready word is not written (failure injection), or -1
};
cudaError_t launch_batch_forward(const DevCtx& ctx, const BatchDev& B, cudaStream_t s);
cudaError_t batch_mac_blocks(const DevCtx& ctx, int nt, int has_dual, int* blocks);

cudaError_t launch_mul_probe(int which, long long iters, int blocks, int threads, u64 seed, u64* sink,
                             cudaStream_t s);

PENCIL_NTT_INSTANTIATE(extern, 12, false)
PENCIL_NTT_INSTANTIATE(extern, 13, false)
PENCIL_NTT_INSTANTIATE(extern, 14, false)
PENCIL_NTT_INSTANTIATE(extern, 12, true)
PENCIL_NTT_INSTANTIATE(extern, 13, true)
PENCIL_NTT_INSTANTIATE(extern, 14, true)

// Dispatch on log2(N), the context's radix (log2 of coefficients per thread) and
// its butterfly arithmetic (Shoup / Harvey, or pseudo-Mersenne folds).
template <class Mode, bool INV>
cudaError_t ntt_multi(const DevCtx& ctx, const typename Mode::Params* Ps, const int2* items, long long count,
                      const u64* step, cudaStream_t s) {
#define PENCIL_NTT_MULTI_CASE(LOGN)                                                                          \
  case LOGN:                                                                                                 \
    if (ctx.ntt_arith)                                                                                       \
      return r4 ? launch_ntt_multi<LOGN, 4, Mode, INV, true>(ctx, Ps, items, count, step, s)                 \
                : launch_ntt_multi<LOGN, 5, Mode, INV, true>(ctx, Ps, items, count, step, s);                \
    return r4 ? launch_ntt_multi<LOGN, 4, Mode, INV, false>(ctx, Ps, items, count, step, s)                  \
              : launch_ntt_multi<LOGN, 5, Mode, INV, false>(ctx, Ps, items, count, step, s);
  const bool r4 = ctx.ntt_loge == 4;
  switch (ctx.log_n) {
    PENCIL_NTT_MULTI_CASE(12)
    PENCIL_NTT_MULTI_CASE(13)
    PENCIL_NTT_MULTI_CASE(14)
    default:
      return cudaErrorInvalidValue;
  }
#undef PENCIL_NTT_MULTI_CASE
}

// Transforms polynomials [first, first + count) of the mode's arrays.
template <class Mode, bool INV>
cudaError_t ntt(const DevCtx& ctx, const typename Mode::Params& P, int count, cudaStream_t s, int first = 0) {
#define PENCIL_NTT_CASE(LOGN)                                                                                \
  case LOGN:                                                                                                 \
    if (ctx.ntt_arith)                                                                                       \
      return r4 ? launch_ntt<LOGN, 4, Mode, INV, true>(ctx, P, first, count, s)                              \
                : launch_ntt<LOGN, 5, Mode, INV, true>(ctx, P, first, count, s);                             \
    return r4 ? launch_ntt<LOGN, 4, Mode, INV, false>(ctx, P, first, count, s)                               \
              : launch_ntt<LOGN, 5, Mode, INV, false>(ctx, P, first, count, s);
  const bool r4 = ctx.ntt_loge == 4;
  switch (ctx.log_n) {
    PENCIL_NTT_CASE(12)
    PENCIL_NTT_CASE(13)
    PENCIL_NTT_CASE(14)
    default:
      return cudaErrorInvalidValue;
  }
#undef PENCIL_NTT_CASE
}

}  // namespace pencil
