// Batched negacyclic NTT / INTT for one (polynomial, limb) per CTA.
//
// Sec. 5 ("NTT"): ring products in Z_q[X]/(X^N+1) become slot-wise after the
// transform.  Forward = Cooley-Tukey with twiddles psi^brv(m+i) (natural order
// in, bit-reversed evaluation order out); inverse = Gentleman-Sande with
// psi^-brv(m+i), then N^{-1}.  Harvey's lazy butterflies keep forward values
// in [0, 4q) and inverse values in [0, 2q); q < 2^62 keeps 4q < 2^64.  (The
// wider-range variants ct_bf8 / gs_bf4 of common.cuh measured slower on GB300
// with pencil_mul_probe and are not used here.)
//
// GB300 mapping: T = N / E threads each hold E = 2^LOGE coefficients in
// registers and run LOGE radix-2 stages between two shared-memory exchanges
// (a radix-2^LOGE round).  The first forward round reads its coefficients
// straight from the fused prologue (coalesced: thread t holds t + l*T); the
// result goes through shared memory once more so the fused epilogue sees pairs
// of consecutive slots (16-byte coalesced stores, one Philox block per pair).
#pragma once
#include <type_traits>
#include <utility>

#include <cooperative_groups.h>

#include "common.cuh"

namespace pencil {

// Final scaling of an inverse transform, applied by the engine (the mode's store
// receives the canonical scaled coefficient): N^{-1}, or N^{-1} qtil for
// decryption (the CRT factor folded in).
enum class InvScale { kNinv, kNqtil };

// Inverse modes whose store writes shared memory (the run then synchronises the
// CTA before its stores) and that finish with a step across the L limb CTAs of
// one polynomial, launched as a thread-block cluster (1, L, 1).
template <class M, class = void>
struct ClusterLimbs : std::false_type {};
template <class M>
struct ClusterLimbs<M, std::void_t<decltype(M::kClusterLimbs)>> : std::bool_constant<M::kClusterLimbs> {};

// Shared-memory slot of coefficient x: the low four index bits are XOR-ed with
// (bits 4..7) ^ (bits 5..8).  8-byte accesses are served per half-warp (16
// threads over the 16 bank pairs); with this swizzle every round's strided
// accesses and the epilogue's pair accesses hit 16 distinct bank pairs in each
// half-warp (two wavefronts per warp access, the minimum), for every N and radix.
template <int LOGN>
__device__ __forceinline__ int sidx(int x) {
  return x ^ (((x >> 4) ^ (x >> 5)) & 15);
}

template <int LOGN, int LOGE, int S0>
struct Round {
  static constexpr int K = (LOGN - S0) < LOGE ? (LOGN - S0) : LOGE;
  static constexpr int G = 1 << (LOGE - K);
  static constexpr int LOGD = LOGN - S0 - K;
  static constexpr int T = (1 << LOGN) >> LOGE;
  static constexpr int E = 1 << LOGE;

  static __device__ __forceinline__ int pos(int tau, int gg, int l) {
    int g = gg * T + tau;
    int B = g >> LOGD;
    int p = g & ((1 << LOGD) - 1);
    return (B << (LOGD + K)) + p + (l << LOGD);
  }
  static __device__ __forceinline__ void load(u64 (&v)[E], const u64* sm, int tau) {
#pragma unroll
    for (int gg = 0; gg < G; ++gg)
#pragma unroll
      for (int l = 0; l < (1 << K); ++l) v[gg * (1 << K) + l] = sm[sidx<LOGN>(pos(tau, gg, l))];
  }
  static __device__ __forceinline__ void store(const u64 (&v)[E], u64* sm, int tau) {
#pragma unroll
    for (int gg = 0; gg < G; ++gg)
#pragma unroll
      for (int l = 0; l < (1 << K); ++l) sm[sidx<LOGN>(pos(tau, gg, l))] = v[gg * (1 << K) + l];
  }
  // One radix-2 stage J of this round on every group the thread holds.
  template <int J, bool FWD>
  static __device__ __forceinline__ void stage(u64 (&v)[E], const ulonglong2* __restrict__ tw, int tau, u64 q,
                                               u64 q2) {
    constexpr int half = 1 << (K - 1 - J);
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
      const int B = (gg * T + tau) >> LOGD;
#pragma unroll
      for (int i = 0; i < (1 << J); ++i) {
        const ulonglong2 w = __ldg(tw + (1 << (S0 + J)) + (B << J) + i);
#pragma unroll
        for (int r = 0; r < half; ++r) {
          const int l = gg * (1 << K) + i * 2 * half + r;
          if constexpr (FWD)
            ct_butterfly(v[l], v[l + half], w.x, w.y, q, q2);
          else
            gs_butterfly(v[l], v[l + half], w.x, w.y, q, q2);
        }
      }
    }
  }
  template <int... J>
  static __device__ __forceinline__ void fwd_seq(std::integer_sequence<int, J...>, u64 (&v)[E],
                                                 const ulonglong2* tw, int tau, u64 q, u64 q2) {
    (stage<J, true>(v, tw, tau, q, q2), ...);
  }
  template <int... J>
  static __device__ __forceinline__ void inv_seq(std::integer_sequence<int, J...>, u64 (&v)[E],
                                                 const ulonglong2* tw, int tau, u64 q, u64 q2) {
    (stage<K - 1 - J, false>(v, tw, tau, q, q2), ...);
  }
  static __device__ __forceinline__ void fwd(u64 (&v)[E], const ulonglong2* __restrict__ tw, int tau, u64 q, u64 q2) {
    fwd_seq(std::make_integer_sequence<int, K>{}, v, tw, tau, q, q2);
  }
  static __device__ __forceinline__ void inv(u64 (&v)[E], const ulonglong2* __restrict__ tw, int tau, u64 q, u64 q2) {
    inv_seq(std::make_integer_sequence<int, K>{}, v, tw, tau, q, q2);
  }
};

// Forward rounds S0, S0 + LOGE, ...; on return the last round's values are in smem.
template <int LOGN, int LOGE, int S0>
struct FwdRounds {
  static __device__ __forceinline__ void run(u64 (&v)[1 << LOGE], u64* sm, const ulonglong2* tw, int tau, u64 q,
                                             u64 q2) {
    using R = Round<LOGN, LOGE, S0>;
    R::fwd(v, tw, tau, q, q2);
    if constexpr (S0 > 0) __syncthreads();  // previous round's readers are done
    R::store(v, sm, tau);
    __syncthreads();
    if constexpr (S0 + LOGE < LOGN) {
      Round<LOGN, LOGE, S0 + LOGE>::load(v, sm, tau);
      FwdRounds<LOGN, LOGE, S0 + LOGE>::run(v, sm, tw, tau, q, q2);
    }
  }
};

// Inverse rounds from S0 down to 0; on entry the values are in smem (synced);
// on return v holds the coefficients tau + l*T.
template <int LOGN, int LOGE, int S0>
struct InvRounds {
  static __device__ __forceinline__ void run(u64 (&v)[1 << LOGE], u64* sm, const ulonglong2* tw, int tau, u64 q,
                                             u64 q2) {
    using R = Round<LOGN, LOGE, S0>;
    R::load(v, sm, tau);
    R::inv(v, tw, tau, q, q2);
    if constexpr (S0 > 0) {
      __syncthreads();
      R::store(v, sm, tau);
      __syncthreads();
      InvRounds<LOGN, LOGE, S0 - LOGE>::run(v, sm, tw, tau, q, q2);
    }
  }
};

template <int LOGN, int LOGE_>
struct NttCfg {
  static constexpr int LOGE = LOGE_;
  static constexpr int N = 1 << LOGN;
  static constexpr int E = 1 << LOGE;
  static constexpr int T = N >> LOGE;
  static constexpr int LAST_S0 = ((LOGN - 1) / LOGE) * LOGE;
  static constexpr size_t SMEM = (size_t)N * sizeof(u64);
  // two CTAs (two transforms) per SM when their threads and shared memory fit
  static constexpr int MIN_BLOCKS = (T <= 512 && 2 * SMEM <= 227 * 1024) ? 2 : 1;
};

// Forward transform of (poly, limb) with a fused prologue (Mode::load,
// canonical coefficient e) and epilogue (Mode::store2, canonical slots e, e + 1).
template <int LOGN, int LOGE, class Mode>
__device__ __forceinline__ void ntt_fwd_run(const DevCtx& ctx, const typename Mode::Params& P, int poly, int limb,
                                            u64* sm) {
  using C = NttCfg<LOGN, LOGE>;
  const int tau = threadIdx.x;
  const LimbConst& lc = ctx.limb[limb];
  const u64 q = lc.q, q2 = 2 * q;
  const ulonglong2* tw = ctx.tw_fwd + (size_t)limb * C::N;
  u64 v[C::E];
  if constexpr (Mode::kHeavyLoad) {
    // Long prologue (gathers, multiplies): a loop through shared memory bounds
    // the code size (kLoadUnroll iterations in flight); each thread re-reads
    // only the slots it wrote.
#pragma unroll(Mode::kLoadUnroll)
    for (int l = 0; l < C::E; ++l) {
      const int e = tau + l * C::T;
      sm[sidx<LOGN>(e)] = Mode::template load<C::N>(ctx, P, lc, poly, limb, e);
    }
#pragma unroll
    for (int l = 0; l < C::E; ++l) v[l] = sm[sidx<LOGN>(tau + l * C::T)];
    __syncthreads();
  } else {
#pragma unroll
    for (int l = 0; l < C::E; ++l) v[l] = Mode::template load<C::N>(ctx, P, lc, poly, limb, tau + l * C::T);
  }
  FwdRounds<LOGN, C::LOGE, 0>::run(v, sm, tw, tau, q, q2);
  if constexpr (Mode::kQuad) {
#pragma unroll(Mode::kEpilogueUnroll)
    for (int l = 0; l < C::E / 4; ++l) {
      const int e = 4 * (tau + l * C::T);
      u64 x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = canon4(sm[sidx<LOGN>(e + i)], q, q2);
      Mode::template store4<C::N>(ctx, P, lc, poly, limb, e, x);
    }
  } else {
#pragma unroll(Mode::kEpilogueUnroll)
    for (int l = 0; l < C::E / 2; ++l) {
      const int e = 2 * (tau + l * C::T);
      const u64 x0 = canon4(sm[sidx<LOGN>(e)], q, q2);
      const u64 x1 = canon4(sm[sidx<LOGN>(e + 1)], q, q2);
      Mode::template store2<C::N>(ctx, P, lc, poly, limb, e, x0, x1);
    }
  }
}

// Inverse transform of (poly, limb) with a fused prologue (Mode::load, value in
// [0, 2q)) and epilogue (Mode::store, canonical coefficient e).
template <int LOGN, int LOGE, class Mode>
__device__ __forceinline__ void ntt_inv_run(const DevCtx& ctx, const typename Mode::Params& P, int poly, int limb,
                                            u64* sm) {
  using C = NttCfg<LOGN, LOGE>;
  const int tau = threadIdx.x;
  const LimbConst& lc = ctx.limb[limb];
  const u64 q = lc.q, q2 = 2 * q;
  const ulonglong2* tw = ctx.tw_inv + (size_t)limb * C::N;
  u64 v[C::E];
#pragma unroll(Mode::kLoadUnroll)
  for (int l = 0; l < C::E; ++l) {
    const int e = tau + l * C::T;
    sm[sidx<LOGN>(e)] = Mode::template load<C::N>(ctx, P, lc, poly, limb, e);
  }
  __syncthreads();
  InvRounds<LOGN, C::LOGE, C::LAST_S0>::run(v, sm, tw, tau, q, q2);
  // v in [0, 2q); scaled here by the mode's kappa (N^{-1}, possibly with its own constant folded in)
  if constexpr (ClusterLimbs<Mode>::value) __syncthreads();   // the last round's reads are done
  const bool ninv = Mode::kInvScale == InvScale::kNinv;
  const u64 kap = ninv ? lc.ninv : lc.nqtil, kaps = ninv ? lc.ninvs : lc.nqtils;
#pragma unroll
  for (int l = 0; l < C::E; ++l)
    Mode::template store<C::N>(ctx, P, lc, poly, limb, tau + l * C::T, mul_shoup(v[l], kap, kaps, q));
}

// ------------------------------------------------------------------ pseudo-Mersenne engine
// The same transforms for primes q = 2^60 - c (c < 2^24) with ct_fold / gs_fold
// butterflies (common.cuh): no correction step inside a butterfly; values grow
// lazily and are folded (fold60) only where the bound requires it:
//  * forward: a stage adds less than 2q to the bound, so the registers are
//    folded once per round of at most 5 stages (bound < 11.01 q < 2^64) and
//    brought to [0, q) (fold, one conditional subtraction) before the epilogue;
//  * inverse: a stage doubles the bound of its sums, so the sums of every
//    second stage (counted from the first inverse stage) are folded; inputs
//    stay below 2.26 q and the subtraction constant is 2q or 4q.
// Shared memory holds the N words with two spare words after every 32
// (slot ph(x)): every round's accesses are conflict-free and a thread's words of
// one round sit at compile-time offsets from one base address.  The last
// forward round of at most 2 stages runs inside the epilogue on groups of 2 or 4
// consecutive slots read from shared memory, and the first inverse round of at
// most 2 stages inside the prologue, which saves a shared-memory round trip
// (N = 8192 with radix 2^4: rounds of 4, 4, 4 and 1 stages).

__device__ __forceinline__ constexpr int ph(int x) { return x + 2 * (x >> 5); }

template <int LOGN, int LOGE>
struct FCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int E = 1 << LOGE;
  static constexpr int T = N >> LOGE;
  static constexpr int R = (LOGN + LOGE - 1) / LOGE;    // rounds
  static constexpr int SL = (R - 1) * LOGE;              // first stage of the last round
  static constexpr int KL = LOGN - SL;                   // its stages, 1 .. LOGE
  static constexpr bool FUSE = KL <= 2;
  static constexpr size_t SMEM = (size_t)(N + 2 * (N >> 5)) * sizeof(u64);
  static constexpr int MIN_BLOCKS = (T <= 512 && 2 * SMEM <= 227 * 1024) ? 2 : 1;
};

// Barrier between two shared-memory phases: the warp's own when every slot the
// following phase touches was last touched by the same warp, the CTA's otherwise.
template <bool WARP_LOCAL>
__device__ __forceinline__ void phase_sync() {
  if constexpr (WARP_LOCAL)
    __syncwarp();
  else
    __syncthreads();
}

// Round S0 of the fold engine: K stages on G groups of 2^K words per thread;
// group gg of thread tau is at positions base + l 2^LOGD, slot ph(base) + ph(l 2^LOGD).
// A round is warp-local (kLocal) when warp w reads and writes only the 32 E
// consecutive positions [32 E w, 32 E (w + 1)): full rounds with LOGD <= 5, and
// the last (partial) round, whose G groups per thread are numbered warp by warp
// (group 32 G w + 32 gg + lane) for that purpose.  Between two warp-local phases
// the exchange through shared memory needs only __syncwarp.
template <int LOGN, int LOGE, int S0>
struct FRound {
  static constexpr int K = (LOGN - S0) < LOGE ? (LOGN - S0) : LOGE;
  static constexpr int G = 1 << (LOGE - K);
  static constexpr int LOGD = LOGN - S0 - K;
  static constexpr int T = (1 << LOGN) >> LOGE;
  static constexpr int E = 1 << LOGE;
  static constexpr bool kLocal = (K < LOGE) || (LOGD <= 5);
  static_assert(T % 32 == 0, "whole warps");
  static_assert(K == LOGE || LOGD == 0, "only the last round is partial");

  static __device__ __forceinline__ int grp(int tau, int gg) {
    if constexpr (G == 1)
      return tau;
    else
      return ((tau >> 5) << (5 + LOGE - K)) + (gg << 5) + (tau & 31);
  }
  static __device__ __forceinline__ int base(int tau, int gg) {
    const int g = grp(tau, gg);
    return ph(((g >> LOGD) << (LOGD + K)) + (g & ((1 << LOGD) - 1)));
  }
  static __device__ __forceinline__ void load(u64 (&v)[E], const u64* sm, int tau) {
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
      const u64* b = sm + base(tau, gg);
#pragma unroll
      for (int l = 0; l < (1 << K); ++l) v[gg * (1 << K) + l] = b[ph(l << LOGD)];
    }
  }
  static __device__ __forceinline__ void store(const u64 (&v)[E], u64* sm, int tau) {
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
      u64* b = sm + base(tau, gg);
#pragma unroll
      for (int l = 0; l < (1 << K); ++l) b[ph(l << LOGD)] = v[gg * (1 << K) + l];
    }
  }
  // Stage J of the round (global stage S0 + J), forward.
  template <int J>
  static __device__ __forceinline__ void fwd_stage(u64 (&v)[E], const ulonglong2* __restrict__ tw, int tau, u32 c60,
                                                   u32 c64, u64 q2) {
    constexpr int half = 1 << (K - 1 - J);
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
      const int B = grp(tau, gg) >> LOGD;
#pragma unroll
      for (int i = 0; i < (1 << J); ++i) {
        const ulonglong2 w = __ldg(tw + (1 << (S0 + J)) + (B << J) + i);
#pragma unroll
        for (int r = 0; r < half; ++r) {
          const int l = gg * (1 << K) + i * 2 * half + r;
          ct_fold(v[l], v[l + half], w, c60, c64, q2);
        }
      }
    }
  }
  // Stage J of the round, inverse; `step` = its position in the inverse order
  // (LOGN - 1 - (S0 + J)): even steps subtract against 2q, odd ones against 4q
  // and fold their sums.
  template <int J>
  static __device__ __forceinline__ void inv_stage(u64 (&v)[E], const ulonglong2* __restrict__ tw, int tau, u32 c60,
                                                   u32 c64, u64 q2, u64 q4) {
    constexpr int half = 1 << (K - 1 - J);
    constexpr bool odd = ((LOGN - 1 - (S0 + J)) & 1) != 0;
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
      const int B = grp(tau, gg) >> LOGD;
#pragma unroll
      for (int i = 0; i < (1 << J); ++i) {
        const ulonglong2 w = __ldg(tw + (1 << (S0 + J)) + (B << J) + i);
#pragma unroll
        for (int r = 0; r < half; ++r) {
          const int l = gg * (1 << K) + i * 2 * half + r;
          gs_fold(v[l], v[l + half], w, c60, c64, odd ? q4 : q2);
          if constexpr (odd) v[l] = fold60(v[l], c60);
        }
      }
    }
  }
  template <int... J>
  static __device__ __forceinline__ void fwd_seq(std::integer_sequence<int, J...>, u64 (&v)[E],
                                                 const ulonglong2* tw, int tau, u32 c60, u32 c64, u64 q2) {
    (fwd_stage<J>(v, tw, tau, c60, c64, q2), ...);
  }
  // Round 0 of the inverse with the transform's final scaling kappa merged into
  // its last stage (global stage 0, whose butterflies all use w1 = tw[1]):
  //   x' = (x + y) kappa,  y' = (x - y + cq) (w1 kappa),  both < 1.13 q,
  // N / 2 products instead of the stage's N / 2 and the N of a separate scaling.
  // sc = {kappa, kappa 2^32, w1 kappa, w1 kappa 2^32} mod q.
  static __device__ __forceinline__ void inv_scaled(u64 (&v)[E], const ulonglong2* tw, int tau, u32 c60, u32 c64,
                                                    u64 q2, u64 q4, const u64* sc) {
    static_assert(S0 == 0 && G == 1 && K == LOGE, "the first round, full");
    inv_seq(std::make_integer_sequence<int, K - 1>{}, v, tw, tau, c60, c64, q2, q4, 1);
    constexpr bool odd = ((LOGN - 1) & 1) != 0;   // the subtraction constant of inverse step LOGN - 1
    const u64 cq = odd ? q4 : q2;
    const u64 k = sc[0], k32 = sc[1], wk = sc[2], wk32 = sc[3];
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
      const u64 x = v[r], y = v[r + E / 2];
      v[r] = mul_fold(x + y, k, k32, c60, c64);
      v[r + E / 2] = mul_fold(x + cq - y, wk, wk32, c60, c64);
    }
  }
  // Stages K - 1 .. 0 (inverse order), or K - 1 .. 1 with sizeof...(J) = K - 1.
  template <int... J>
  static __device__ __forceinline__ void inv_seq(std::integer_sequence<int, J...>, u64 (&v)[E],
                                                 const ulonglong2* tw, int tau, u32 c60, u32 c64, u64 q2, u64 q4,
                                                 int = 0) {
    (inv_stage<K - 1 - J>(v, tw, tau, c60, c64, q2, q4), ...);
  }
  static __device__ __forceinline__ void fwd(u64 (&v)[E], const ulonglong2* tw, int tau, u32 c60, u32 c64, u64 q2) {
    fwd_seq(std::make_integer_sequence<int, K>{}, v, tw, tau, c60, c64, q2);
  }
  // Stages j0 .. K - 1 only (j0 uniform across the CTA).
  template <int... J>
  static __device__ __forceinline__ void fwd_from_seq(std::integer_sequence<int, J...>, int j0, u64 (&v)[E],
                                                      const ulonglong2* tw, int tau, u32 c60, u32 c64, u64 q2) {
    ((J >= j0 ? fwd_stage<J>(v, tw, tau, c60, c64, q2) : void()), ...);
  }
  static __device__ __forceinline__ void fwd_from(int j0, u64 (&v)[E], const ulonglong2* tw, int tau, u32 c60,
                                                  u32 c64, u64 q2) {
    fwd_from_seq(std::make_integer_sequence<int, K>{}, j0, v, tw, tau, c60, c64, q2);
  }
  static __device__ __forceinline__ void inv(u64 (&v)[E], const ulonglong2* tw, int tau, u32 c60, u32 c64, u64 q2,
                                             u64 q4) {
    inv_seq(std::make_integer_sequence<int, K>{}, v, tw, tau, c60, c64, q2, q4);
  }
};

// Full forward rounds S0, S0 + LOGE, ... before the last round; round 0 takes its
// words from registers (the prologue's coefficients tau + l T), the others from
// shared memory.  Each round folds its words and leaves them in shared memory.
template <int LOGN, int LOGE, int S0>
struct FFwdRounds {
  static __device__ __forceinline__ void run(u64 (&v)[1 << LOGE], u64* sm, const ulonglong2* tw, int tau, u32 c60,
                                             u32 c64, u64 q2) {
    using Rd = FRound<LOGN, LOGE, S0>;
    if constexpr (S0 > 0) Rd::load(v, sm, tau);
    Rd::fwd(v, tw, tau, c60, c64, q2);
#pragma unroll
    for (int l = 0; l < (1 << LOGE); ++l) v[l] = fold60(v[l], c60);
    if constexpr (S0 > 0) phase_sync<Rd::kLocal>();   // every reader of these slots is done
    Rd::store(v, sm, tau);
    phase_sync<Rd::kLocal>();   // the following rounds are warp-local once this one is
    if constexpr (S0 + LOGE < FCfg<LOGN, LOGE>::SL) FFwdRounds<LOGN, LOGE, S0 + LOGE>::run(v, sm, tw, tau, c60, c64, q2);
  }
};

// Inverse rounds from S0 down to 0 (words in shared memory on entry, synced); on
// return v holds the coefficients tau + l T.
template <int LOGN, int LOGE, int S0>
struct FInvRounds {
  static __device__ __forceinline__ void run(u64 (&v)[1 << LOGE], u64* sm, const ulonglong2* tw, int tau, u32 c60,
                                             u32 c64, u64 q2, u64 q4, const u64* sc) {
    using Rd = FRound<LOGN, LOGE, S0>;
    Rd::load(v, sm, tau);
    if constexpr (S0 == 0)
      Rd::inv_scaled(v, tw, tau, c60, c64, q2, q4, sc);
    else
      Rd::inv(v, tw, tau, c60, c64, q2, q4);
    if constexpr (S0 > 0) {
      phase_sync<Rd::kLocal>();
      Rd::store(v, sm, tau);
      phase_sync<Rd::kLocal && FRound<LOGN, LOGE, S0 - LOGE>::kLocal>();
      FInvRounds<LOGN, LOGE, S0 - LOGE>::run(v, sm, tw, tau, c60, c64, q2, q4, sc);
    }
  }
};

// The last forward round's KL stages on one group of W = 2^KL consecutive slots
// (group index g: positions g W .. g W + W - 1), then canonical values.
template <int LOGN, int LOGE>
__device__ __forceinline__ void fold_last_fwd(u64* u, const ulonglong2* __restrict__ tw, int g, u32 c60, u32 c64,
                                              u64 q, u64 q2) {
  using C = FCfg<LOGN, LOGE>;
  constexpr int W = 1 << C::KL;
#pragma unroll
  for (int J = 0; J < C::KL; ++J) {
    const int half = W >> (J + 1);
#pragma unroll
    for (int i = 0; i < (1 << J); ++i) {
      const ulonglong2 w = __ldg(tw + (1 << (C::SL + J)) + (g << J) + i);
#pragma unroll
      for (int r = 0; r < half; ++r) ct_fold(u[i * 2 * half + r], u[i * 2 * half + r + half], w, c60, c64, q2);
    }
  }
#pragma unroll
  for (int i = 0; i < W; ++i) u[i] = csub(fold60(u[i], c60), q);
}

// The first inverse round's KL stages (inverse steps 0 .. KL - 1) on one group.
template <int LOGN, int LOGE>
__device__ __forceinline__ void fold_first_inv(u64 (&u)[1 << FCfg<LOGN, LOGE>::KL],
                                               const ulonglong2* __restrict__ tw, int g, u32 c60, u32 c64, u64 q2,
                                               u64 q4) {
  using C = FCfg<LOGN, LOGE>;
  constexpr int W = 1 << C::KL;
#pragma unroll
  for (int J = C::KL - 1; J >= 0; --J) {
    const int half = W >> (J + 1);
    const bool odd = ((LOGN - 1 - (C::SL + J)) & 1) != 0;
#pragma unroll
    for (int i = 0; i < (1 << J); ++i) {
      const ulonglong2 w = __ldg(tw + (1 << (C::SL + J)) + (g << J) + i);
#pragma unroll
      for (int r = 0; r < half; ++r) {
        u64& x = u[i * 2 * half + r];
        gs_fold(x, u[i * 2 * half + r + half], w, c60, c64, odd ? q4 : q2);
        if (odd) x = fold60(x, c60);
      }
    }
  }
}

// Modes whose input polynomials may have a short support (Mode::support(P):
// coefficients from there on are zero).
template <class M, class = void>
struct SparseInput : std::false_type {};
template <class M>
struct SparseInput<M, std::void_t<decltype(M::kSparse)>> : std::bool_constant<M::kSparse> {};

// Forward rounds 0 and 1 of a polynomial of degree < sup <= T.  After s
// Cooley-Tukey stages, block b of N / 2^s words holds p mod (X^{N/2^s} - zeta_b),
// which is p itself while deg p < N / 2^s: the first LOGN - ceil(log2 sup)
// stages only copy.  Round 0 (LOGE stages) is therefore skipped whole, and so
// are the first j stages of round 1 where sup <= T / 2^j; round 1 then starts
// from word x = p[x mod (N / 2^(LOGE + j))], read from the T prologue values in
// shared memory (one gather per thread instead of E).  The values and their
// bounds are those the skipped butterflies leave (ct_fold(a, 0) = (a, a + 2q)
// only widens the bound).  Leaves round 1's words, folded, in shared memory.
template <int LOGN, int LOGE, class Mode>
__device__ __forceinline__ void fold_sparse_head(const DevCtx& ctx, const typename Mode::Params& P,
                                                 const LimbConst& lc, int poly, int limb, int sup, u64 (&v)[1 << LOGE],
                                                 u64* sm, const ulonglong2* tw, int tau, u32 c60, u32 c64, u64 q2) {
  using C = FCfg<LOGN, LOGE>;
  using R1 = FRound<LOGN, LOGE, LOGE>;
  static_assert(R1::K == LOGE && R1::G == 1, "round 1 must be a full round");
  sm[ph(tau)] = tau < sup ? Mode::template load<C::N>(ctx, P, lc, poly, limb, tau) : 0ull;
  int j = 0;
  while (j < LOGE && sup <= (C::T >> (j + 1))) ++j;
  __syncthreads();
  constexpr int D1 = 1 << R1::LOGD;   // round 1: thread tau holds words base + l D1
  const int m = (C::E >> j) - 1;
  const u64* b = sm + ph(tau & (D1 - 1));
#pragma unroll
  for (int l = 0; l < C::E; ++l) v[l] = b[ph(D1 * (l & m))];
  R1::fwd_from(j, v, tw, tau, c60, c64, q2);
#pragma unroll
  for (int l = 0; l < C::E; ++l) v[l] = fold60(v[l], c60);
  __syncthreads();   // every thread has read the prologue values
  R1::store(v, sm, tau);
  phase_sync<R1::kLocal>();
  if constexpr (2 * LOGE < C::SL) FFwdRounds<LOGN, LOGE, 2 * LOGE>::run(v, sm, tw, tau, c60, c64, q2);
}

template <int LOGN, int LOGE, class Mode>
__device__ __forceinline__ void ntt_fwd_run_fold(const DevCtx& ctx, const typename Mode::Params& P, int poly,
                                                 int limb, u64* sm) {
  using C = FCfg<LOGN, LOGE>;
  const int tau = threadIdx.x;
  const LimbConst& lc = ctx.limb[limb];
  const u64 q = lc.q, q2 = 2 * q;
  const u32 c60 = (u32)lc.c60, c64 = (u32)lc.c64;
  const ulonglong2* tw = ctx.tw_fwd_f + (size_t)limb * C::N;
  u64 v[C::E];
  bool dense = true;
  if constexpr (SparseInput<Mode>::value && C::R >= 3) {
    const int sup = Mode::support(P);
    if (sup <= C::T) {
      dense = false;
      fold_sparse_head<LOGN, LOGE, Mode>(ctx, P, lc, poly, limb, sup, v, sm, tw, tau, c60, c64, q2);
    }
  }
  if (dense) {
    if constexpr (Mode::kHeavyLoad) {
#pragma unroll(Mode::kLoadUnroll)
      for (int l = 0; l < C::E; ++l) {
        const int e = tau + l * C::T;
        sm[ph(e)] = Mode::template load<C::N>(ctx, P, lc, poly, limb, e);
      }
#pragma unroll
      for (int l = 0; l < C::E; ++l) v[l] = sm[ph(tau + l * C::T)];
    } else {
#pragma unroll
      for (int l = 0; l < C::E; ++l) v[l] = Mode::template load<C::N>(ctx, P, lc, poly, limb, tau + l * C::T);
    }
    // (round 0 stores each thread's words at the slots it read them from: no barrier needed here)
    FFwdRounds<LOGN, LOGE, 0>::run(v, sm, tw, tau, c60, c64, q2);
  }
  if constexpr (C::FUSE) {
    // groups of GW consecutive slots per iteration: the last round's groups of
    // W = 2^KL, gathered in fours for modes that store four coefficients at a time
    constexpr int W = 1 << C::KL;
    constexpr int GW = (Mode::kQuad && W < 4) ? 4 : W;
    // group k = 32 (E / GW) w + 32 j + lane: warp w's own positions [32 E w, 32 E (w + 1))
    const int kbase = (tau >> 5) * (32 * C::E / GW) + (tau & 31);
#pragma unroll(Mode::kEpilogueUnroll)
    for (int j = 0; j < C::E / GW; ++j) {
      const int k = kbase + 32 * j;
      u64 u[GW];
      const ulonglong2* b = reinterpret_cast<const ulonglong2*>(sm + ph(k * GW));
#pragma unroll
      for (int i = 0; i < GW / 2; ++i) {
        const ulonglong2 x = b[i];
        u[2 * i] = x.x;
        u[2 * i + 1] = x.y;
      }
#pragma unroll
      for (int s = 0; s < GW / W; ++s) fold_last_fwd<LOGN, LOGE>(u + s * W, tw, k * (GW / W) + s, c60, c64, q, q2);
      if constexpr (Mode::kQuad) {
#pragma unroll
        for (int i = 0; i < GW / 4; ++i) Mode::template store4<C::N>(ctx, P, lc, poly, limb, k * GW + 4 * i, u + 4 * i);
      } else {
#pragma unroll
        for (int i = 0; i < GW / 2; ++i)
          Mode::template store2<C::N>(ctx, P, lc, poly, limb, k * GW + 2 * i, u[2 * i], u[2 * i + 1]);
      }
    }
  } else {
    using Rd = FRound<LOGN, LOGE, C::SL>;
    Rd::load(v, sm, tau);
    Rd::fwd(v, tw, tau, c60, c64, q2);
#pragma unroll
    for (int l = 0; l < C::E; ++l) v[l] = csub(fold60(v[l], c60), q);
    static_assert(Rd::kLocal, "the last round is warp-local");
    __syncwarp();
    Rd::store(v, sm, tau);
    __syncwarp();
    // the epilogue's groups are warp w's own positions [32 E w, 32 E (w + 1))
    const int wbase = (tau >> 5) * 32 * C::E, lane = tau & 31;
    if constexpr (Mode::kQuad) {
#pragma unroll(Mode::kEpilogueUnroll)
      for (int l = 0; l < C::E / 4; ++l) {
        const int e = wbase + 4 * (lane + 32 * l);
        const ulonglong2* b = reinterpret_cast<const ulonglong2*>(sm + ph(e));
        const ulonglong2 x01 = b[0], x23 = b[1];
        u64 x[4] = {x01.x, x01.y, x23.x, x23.y};
        Mode::template store4<C::N>(ctx, P, lc, poly, limb, e, x);
      }
    } else {
#pragma unroll(Mode::kEpilogueUnroll)
      for (int l = 0; l < C::E / 2; ++l) {
        const int e = wbase + 2 * (lane + 32 * l);
        const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(sm + ph(e));
        Mode::template store2<C::N>(ctx, P, lc, poly, limb, e, x.x, x.y);
      }
    }
  }
}

template <int LOGN, int LOGE, class Mode>
__device__ __forceinline__ void ntt_inv_run_fold(const DevCtx& ctx, const typename Mode::Params& P, int poly,
                                                 int limb, u64* sm) {
  using C = FCfg<LOGN, LOGE>;
  const int tau = threadIdx.x;
  const LimbConst& lc = ctx.limb[limb];
  const u64 q = lc.q, q2 = 2 * q, q4 = 4 * q;
  const u32 c60 = (u32)lc.c60, c64 = (u32)lc.c64;
  const ulonglong2* tw = ctx.tw_inv_f + (size_t)limb * C::N;
  const u64* sc = Mode::kInvScale == InvScale::kNinv ? lc.sc_ninv : lc.sc_nqtil;
  u64 v[C::E];
  if constexpr (C::FUSE) {
    constexpr int W = 1 << C::KL;
    // group g = 32 (E / W) w + 32 j + lane: warp w's own positions [32 E w, 32 E (w + 1))
    const int gbase = (tau >> 5) * (32 * C::E / W) + (tau & 31);
#pragma unroll(Mode::kLoadUnroll)
    for (int j = 0; j < (C::E >> C::KL); ++j) {
      const int g = gbase + 32 * j;
      u64 u[W];
#pragma unroll
      for (int i = 0; i < W; ++i) u[i] = Mode::template load<C::N>(ctx, P, lc, poly, limb, g * W + i);
      fold_first_inv<LOGN, LOGE>(u, tw, g, c60, c64, q2, q4);
      ulonglong2* b = reinterpret_cast<ulonglong2*>(sm + ph(g * W));
#pragma unroll
      for (int i = 0; i < W / 2; ++i) b[i] = make_ulonglong2(u[2 * i], u[2 * i + 1]);
    }
    if constexpr (C::SL > 0) {
      phase_sync<FRound<LOGN, LOGE, C::SL - LOGE>::kLocal>();
      FInvRounds<LOGN, LOGE, C::SL - LOGE>::run(v, sm, tw, tau, c60, c64, q2, q4, sc);
    } else {
      __syncthreads();
    }
  } else {
    // warp w loads its own positions [32 E w, 32 E (w + 1)), which the first
    // (warp-local) inverse round reads
    const int wbase = (tau >> 5) * 32 * C::E + (tau & 31);
#pragma unroll(Mode::kLoadUnroll)
    for (int l = 0; l < C::E; ++l) {
      const int e = wbase + 32 * l;
      sm[ph(e)] = Mode::template load<C::N>(ctx, P, lc, poly, limb, e);
    }
    static_assert(FRound<LOGN, LOGE, C::SL>::kLocal, "the last round is warp-local");
    __syncwarp();
    FInvRounds<LOGN, LOGE, C::SL>::run(v, sm, tw, tau, c60, c64, q2, q4, sc);
  }
  // v < 1.13 q, already scaled by the mode's kappa in the last stage
  if constexpr (ClusterLimbs<Mode>::value) __syncthreads();   // the last round's reads are done
#pragma unroll
  for (int l = 0; l < C::E; ++l) Mode::template store<C::N>(ctx, P, lc, poly, limb, tau + l * C::T, csub(v[l], q));
}

// Launch shape of either engine.
template <int LOGN, int LOGE, bool FOLD>
struct KCfg {
  static constexpr int T = (1 << LOGN) >> LOGE;
  static constexpr size_t SMEM = FOLD ? FCfg<LOGN, LOGE>::SMEM : NttCfg<LOGN, LOGE>::SMEM;
  static constexpr int MIN_BLOCKS = FOLD ? FCfg<LOGN, LOGE>::MIN_BLOCKS : NttCfg<LOGN, LOGE>::MIN_BLOCKS;
};

template <int LOGN, int LOGE, class Mode, bool FOLD>
__device__ __forceinline__ void fwd_any(const DevCtx& ctx, const typename Mode::Params& P, int poly, int limb,
                                        u64* sm) {
  if constexpr (FOLD)
    ntt_fwd_run_fold<LOGN, LOGE, Mode>(ctx, P, poly, limb, sm);
  else
    ntt_fwd_run<LOGN, LOGE, Mode>(ctx, P, poly, limb, sm);
}

template <int LOGN, int LOGE, class Mode, bool FOLD>
__device__ __forceinline__ void inv_any(const DevCtx& ctx, const typename Mode::Params& P, int poly, int limb,
                                        u64* sm) {
  if constexpr (FOLD)
    ntt_inv_run_fold<LOGN, LOGE, Mode>(ctx, P, poly, limb, sm);
  else
    ntt_inv_run<LOGN, LOGE, Mode>(ctx, P, poly, limb, sm);
}

// Modes whose input is one contiguous polynomial per (poly, limb): each CTA asks
// L2 for the input of the CTA P.ahead launch positions later (about a wave on),
// so that CTA's first loads hit L2.
template <class M, class = void>
struct PrefetchAhead : std::false_type {};
template <class M>
struct PrefetchAhead<M, std::void_t<decltype(M::kPrefetchAhead)>> : std::bool_constant<M::kPrefetchAhead> {};

template <int N, class Mode>
__device__ __forceinline__ void prefetch_ahead(const DevCtx& ctx, const typename Mode::Params& P, int first) {
  if constexpr (PrefetchAhead<Mode>::value) {
    if (threadIdx.x == 0 && P.ahead > 0) {
      const long long next = (long long)blockIdx.x + (long long)blockIdx.y * gridDim.x + P.ahead;
      const long long y = next / gridDim.x;
      if (y < (long long)gridDim.y) Mode::template prefetch<N>(ctx, P, first + (int)(next % gridDim.x), (int)y);
    }
  }
}

// CTA (x, limb) transforms polynomial first + x.
template <int LOGN, int LOGE, class Mode, bool FOLD>
__global__ void __launch_bounds__(KCfg<LOGN, LOGE, FOLD>::T, KCfg<LOGN, LOGE, FOLD>::MIN_BLOCKS)
    k_ntt_fwd(DevCtx ctx, typename Mode::Params P, int first) {
  extern __shared__ __align__(16) u64 sm[];
  prefetch_ahead<1 << LOGN, Mode>(ctx, P, first);
  fwd_any<LOGN, LOGE, Mode, FOLD>(ctx, P, first + (int)blockIdx.x, blockIdx.y, sm);
}

template <int LOGN, int LOGE, class Mode, bool FOLD>
__global__ void __launch_bounds__(KCfg<LOGN, LOGE, FOLD>::T, KCfg<LOGN, LOGE, FOLD>::MIN_BLOCKS)
    k_ntt_inv(DevCtx ctx, typename Mode::Params P, int first) {
  extern __shared__ __align__(16) u64 sm[];
  prefetch_ahead<1 << LOGN, Mode>(ctx, P, first);
  inv_any<LOGN, LOGE, Mode, FOLD>(ctx, P, first + (int)blockIdx.x, blockIdx.y, sm);
  if constexpr (ClusterLimbs<Mode>::value) Mode::template finish<1 << LOGN>(ctx, P, first + (int)blockIdx.x, sm);
}

// Multi-plan variants: CTA (blockIdx.x, limb) transforms polynomial items[x].y
// of the plan items[x].x with that plan's parameters; `step` (device word,
// nullable) re-keys the randomness of each replay (Mode::rebase).
template <int LOGN, int LOGE, class Mode, bool FOLD>
__global__ void __launch_bounds__(KCfg<LOGN, LOGE, FOLD>::T, KCfg<LOGN, LOGE, FOLD>::MIN_BLOCKS)
    k_ntt_fwd_multi(DevCtx ctx, const typename Mode::Params* __restrict__ Ps, const int2* __restrict__ items,
                    const u64* step) {
  extern __shared__ __align__(16) u64 sm[];
  const int2 it = items[blockIdx.x];
  typename Mode::Params P = Ps[it.x];
  Mode::rebase(P, step ? *step : 0ull);
  fwd_any<LOGN, LOGE, Mode, FOLD>(ctx, P, it.y, blockIdx.y, sm);
}

template <int LOGN, int LOGE, class Mode, bool FOLD>
__global__ void __launch_bounds__(KCfg<LOGN, LOGE, FOLD>::T, KCfg<LOGN, LOGE, FOLD>::MIN_BLOCKS)
    k_ntt_inv_multi(DevCtx ctx, const typename Mode::Params* __restrict__ Ps, const int2* __restrict__ items,
                    const u64* step) {
  extern __shared__ __align__(16) u64 sm[];
  const int2 it = items[blockIdx.x];
  typename Mode::Params P = Ps[it.x];
  Mode::rebase(P, step ? *step : 0ull);
  inv_any<LOGN, LOGE, Mode, FOLD>(ctx, P, it.y, blockIdx.y, sm);
}

// ------------------------------------------------------------------ fused modes
__device__ __forceinline__ size_t limb_off(int poly, int limb, int L, int n) {
  return ((size_t)poly * L + limb) * n;
}
__device__ __forceinline__ size_t ct_off(int poly, int comp, int limb, int L, int n) {
  return (((size_t)poly * 2 + comp) * L + limb) * n;
}

// In-place transform of [count][L][N] polynomials.
struct ModeRaw {
  static constexpr InvScale kInvScale = InvScale::kNinv;
  static constexpr bool kHeavyLoad = false;
  static constexpr bool kQuad = false;
  static constexpr int kLoadUnroll = 32;
  static constexpr int kEpilogueUnroll = 16;
  static constexpr bool kPrefetchAhead = true;
  struct Params {
    u64* polys;
    int ahead = 0;   // CTAs ahead whose input each CTA asks L2 to fetch (0: none)
  };
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx& c, const Params& P, const LimbConst&, int poly, int limb,
                                             int e) {
    return P.polys[limb_off(poly, limb, c.L, N) + e];
  }
  template <int N>
  static __device__ __forceinline__ void prefetch(const DevCtx& c, const Params& P, int poly, int limb) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(P.polys + limb_off(poly, limb, c.L, N)),
                 "r"((u32)(N * sizeof(u64)))
                 : "memory");
  }
  template <int N>
  static __device__ __forceinline__ void store2(const DevCtx& c, const Params& P, const LimbConst&, int poly,
                                                int limb, int e, u64 x0, u64 x1) {
    *reinterpret_cast<ulonglong2*>(P.polys + limb_off(poly, limb, c.L, N) + e) = make_ulonglong2(x0, x1);
  }
  template <int N>
  static __device__ __forceinline__ void store(const DevCtx& c, const Params& P, const LimbConst& lc, int poly,
                                               int limb, int e, u64 x) {
    P.polys[limb_off(poly, limb, c.L, N) + e] = x;   // x = N^{-1} INTT, canonical
  }
};

// DO encryption: prologue round(q m / t) + e (m gathered by the packing), epilogue
// c0 = slot - a*s_hat, c1 = a with a sampled in the NTT domain, four coefficients
// per Philox block (one 64-bit word each, uniform_mod_q).
struct ModeEncrypt {
  static constexpr bool kHeavyLoad = true;
  static constexpr bool kQuad = true;
  static constexpr int kLoadUnroll = 8;
  static constexpr int kEpilogueUnroll = 1;   // Philox + four products per quad
  struct Params {
    Packing pk;
    Accessor ac;
    const int8_t* err;        // [count][N]
    const ulonglong2* sk;     // [L][N] (s_hat, companion)
    u64* ct;                  // [count][2][L][N]
    u64 seed;
  };
  // seed of replay `step` (batched graphs): seed + step * 2^32
  static __device__ __forceinline__ void rebase(Params& P, u64 step) { P.seed += step << 32; }
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx& c, const Params& P, const LimbConst& lc, int poly, int,
                                             int e) {
    const u64 m = gather(P.pk, P.ac, poly, e) & c.t_mask;
    const u64 r = scale_msg(m, lc, c);
    const int ee = P.err[(size_t)poly * N + e];
    return ee >= 0 ? add_mod(r, (u64)ee, lc.q) : sub_mod(r, (u64)(-ee), lc.q);
  }
  template <int N>
  static __device__ __forceinline__ void store4(const DevCtx& c, const Params& P, const LimbConst& lc, int poly,
                                                int limb, int e, const u64* x) {
    const Philox4 w = philox4x64((u64)(e >> 2), (u64)poly, (u64)limb, 0ull, P.seed, PENCIL_DOM_A);
    u64 a[4], c0[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = uniform_mod_q(w.v[i], e + i, poly, limb, P.seed, PENCIL_DOM_A, lc);
      const ulonglong2 s = __ldg(P.sk + (size_t)limb * N + e + i);
      c0[i] = sub_mod(x[i], mul_shoup(a[i], s.x, s.y, lc.q), lc.q);
    }
    ulonglong2* d0 = reinterpret_cast<ulonglong2*>(P.ct + ct_off(poly, 0, limb, c.L, N) + e);
    ulonglong2* d1 = reinterpret_cast<ulonglong2*>(P.ct + ct_off(poly, 1, limb, c.L, N) + e);
    d0[0] = make_ulonglong2(c0[0], c0[1]);
    d0[1] = make_ulonglong2(c0[2], c0[3]);
    d1[0] = make_ulonglong2(a[0], a[1]);
    d1[1] = make_ulonglong2(a[2], a[3]);
  }
};

// MO plaintext encoding: centred lift of Z_t values, NTT (short supports,
// e.g. one small kernel block per plaintext, skip the copy-only stages).
struct ModeEncode {
  static constexpr bool kHeavyLoad = true;
  static constexpr bool kQuad = false;
  static constexpr bool kSparse = true;
  static constexpr int kLoadUnroll = 16;
  static constexpr int kEpilogueUnroll = 4;
  struct Params {
    Packing pk;
    Accessor ac;
    u64* pt;   // [count][L][N]
  };
  static __device__ __forceinline__ int support(const Params& P) { return P.pk.support; }
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx& c, const Params& P, const LimbConst& lc, int poly, int,
                                             int e) {
    const u64 v = gather(P.pk, P.ac, poly, e) & c.t_mask;
    const u64 half = (c.t_mask >> 1) + 1;
    return v >= half ? lc.q - ((c.t_mask + 1) - v) : v;
  }
  template <int N>
  static __device__ __forceinline__ void store2(const DevCtx& c, const Params& P, const LimbConst&, int poly,
                                                int limb, int e, u64 x0, u64 x1) {
    *reinterpret_cast<ulonglong2*>(P.pt + limb_off(poly, limb, c.L, N) + e) = make_ulonglong2(x0, x1);
  }
};

// MO's ciphertext-independent terms of Alg. 1 steps 2-3, one launch for both:
// polynomials [0, n_in) -> out_in = NTT(round(q pi_v(x0) / t)) (added to c0 by the
// multiply-accumulate), [n_in, count) -> out_mask = NTT(round(q s / t)) of the mask
// polynomials (subtracted by the multiply-accumulate's store).
struct ModeMoPrep {
  static constexpr bool kHeavyLoad = true;
  static constexpr bool kQuad = false;
  static constexpr int kLoadUnroll = 16;
  static constexpr int kEpilogueUnroll = 8;
  struct Params {
    Packing pk;
    Accessor ac;
    const u64* mpoly;   // [count - n_in][N] Z_t mask coefficients
    int n_in;
    u64* out_in;        // [n_in][L][N]
    u64* out_mask;      // [count - n_in][L][N]
    u64 seed;           // mask seed (key of the flooding stream)
  };
  static __device__ __forceinline__ void rebase(Params& P, u64 step) { P.seed += step << 32; }   // as the mask's
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx& c, const Params& P, const LimbConst& lc, int poly, int,
                                             int e) {
    if (poly < P.n_in) return scale_msg(gather(P.pk, P.ac, poly, e) & c.t_mask, lc, c);
    const int idx = poly - P.n_in;
    const u64 r = scale_msg(P.mpoly[(size_t)idx * N + e], lc, c);
    if (!c.flood_bits) return r;
    // flooding noise f (uniform in [-2^b, 2^b)) of returned ciphertext idx: Delta s - f
    const u64 w = philox_word(philox4x64((u64)(e >> 2), (u64)idx, 0ull, 0ull, P.seed, PENCIL_DOM_FLOOD), e & 3) &
                  ((2ull << c.flood_bits) - 1);
    const u64 half = 1ull << c.flood_bits;
    return w >= half ? sub_mod(r, reduce64(w - half, lc), lc.q) : add_mod(r, reduce64(half - w, lc), lc.q);
  }
  template <int N>
  static __device__ __forceinline__ void store2(const DevCtx& c, const Params& P, const LimbConst&, int poly,
                                                int limb, int e, u64 x0, u64 x1) {
    u64* dst = poly < P.n_in ? P.out_in + limb_off(poly, limb, c.L, N)
                             : P.out_mask + limb_off(poly - P.n_in, limb, c.L, N);
    *reinterpret_cast<ulonglong2*>(dst + e) = make_ulonglong2(x0, x1);
  }
};

__device__ __forceinline__ u64 shoup_companion(u64 w, u64 q) {
  return (u64)((((unsigned __int128)w) << 64) / q);
}

// DO key generation: ternary s, NTT, stored with Shoup companions.
struct ModeKeygen {
  static constexpr bool kHeavyLoad = true;
  static constexpr bool kQuad = false;
  static constexpr int kLoadUnroll = 4;
  static constexpr int kEpilogueUnroll = 1;
  struct Params {
    u64 seed;
    ulonglong2* sk;   // [L][N]
  };
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx&, const Params& P, const LimbConst& lc, int, int, int e) {
    const Philox4 w = philox4x64((u64)(e >> 2), 0ull, 0ull, 0ull, P.seed, PENCIL_DOM_SECRET);
    const u64 r = w.v[e & 3] % 3ull;
    return r == 0 ? lc.q - 1 : r - 1;
  }
  template <int N>
  static __device__ __forceinline__ void store2(const DevCtx&, const Params& P, const LimbConst& lc, int, int limb,
                                                int e, u64 x0, u64 x1) {
    P.sk[(size_t)limb * N + e] = make_ulonglong2(x0, shoup_companion(x0, lc.q));
    P.sk[(size_t)limb * N + e + 1] = make_ulonglong2(x1, shoup_companion(x1, lc.q));
  }
};

__device__ __forceinline__ u64 lift_small(int v, u64 q) { return v >= 0 ? (u64)v : q - (u64)(-v); }
__device__ __forceinline__ u64 neg_mod(u64 v, u64 q) { return v ? q - v : 0; }

// DO public key (BFV as in Fan-Vercauteren): x = NTT(e) of the sampled error;
// p1 = a, uniform in the NTT domain from Philox (key (seed, 7), counter
// (i/4, 0, limb, 0), word i%4; uniform_mod_q); p0 = -(a s) - x.  Both stored
// with Shoup companions: key[comp][L][N].
struct ModePkKeygen {
  static constexpr bool kHeavyLoad = true;
  static constexpr bool kQuad = true;
  static constexpr int kLoadUnroll = 8;
  static constexpr int kEpilogueUnroll = 1;
  struct Params {
    const int8_t* err;       // [N]
    const ulonglong2* sk;    // [L][N]
    ulonglong2* key;         // [2][L][N]
    u64 seed;
  };
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx&, const Params& P, const LimbConst& lc, int, int, int e) {
    return lift_small(P.err[e], lc.q);
  }
  template <int N>
  static __device__ __forceinline__ void store4(const DevCtx& c, const Params& P, const LimbConst& lc, int, int limb,
                                                int e, const u64* x) {
    const Philox4 w = philox4x64((u64)(e >> 2), 0ull, (u64)limb, 0ull, P.seed, PENCIL_DOM_PK_A);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const u64 a = uniform_mod_q(w.v[i], e + i, 0, limb, P.seed, PENCIL_DOM_PK_A, lc);
      const ulonglong2 s = __ldg(P.sk + (size_t)limb * N + e + i);
      const u64 p0 = neg_mod(add_mod(mul_shoup(a, s.x, s.y, lc.q), x[i], lc.q), lc.q);
      P.key[(size_t)limb * N + e + i] = make_ulonglong2(p0, shoup_companion(p0, lc.q));
      P.key[(size_t)(c.L + limb) * N + e + i] = make_ulonglong2(a, shoup_companion(a, lc.q));
    }
  }
};

// Public-key encryption, first pass: NTT(u) of each ciphertext's ternary u.
struct ModePkU {
  static constexpr bool kHeavyLoad = false;
  static constexpr bool kQuad = false;
  static constexpr int kLoadUnroll = 16;
  static constexpr int kEpilogueUnroll = 8;
  struct Params {
    const int8_t* u;   // [ct][N]
    u64* u_hat;        // [ct][L][N]
  };
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx&, const Params& P, const LimbConst& lc, int poly, int,
                                             int e) {
    return lift_small(P.u[(size_t)poly * N + e], lc.q);
  }
  template <int N>
  static __device__ __forceinline__ void store2(const DevCtx& c, const Params& P, const LimbConst&, int poly,
                                                int limb, int e, u64 x0, u64 x1) {
    *reinterpret_cast<ulonglong2*>(P.u_hat + limb_off(poly, limb, c.L, N) + e) = make_ulonglong2(x0, x1);
  }
};

// Public-key encryption, second pass, over polynomials 2 ct + comp:
//   comp 0: NTT(Delta m + e1) + NTT(u) p0,   comp 1: NTT(e2) + NTT(u) p1,
// written straight into ciphertext ct (whose [2][L][N] layout makes
// polynomial 2 ct + comp the component's slot).
struct ModeEncryptPk {
  static constexpr bool kHeavyLoad = true;
  static constexpr bool kQuad = false;
  static constexpr int kLoadUnroll = 8;
  static constexpr int kEpilogueUnroll = 4;
  struct Params {
    Packing pk;
    Accessor ac;
    const int8_t* e1;          // [ct][N]
    const int8_t* e2;          // [ct][N]
    const u64* u_hat;          // [ct][L][N]
    const ulonglong2* key;     // [2][L][N]
    u64* ct;                   // [ct][2][L][N]
  };
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx& c, const Params& P, const LimbConst& lc, int poly, int,
                                             int e) {
    const int ct = poly >> 1;
    if (poly & 1) return lift_small(P.e2[(size_t)ct * N + e], lc.q);
    const u64 r = scale_msg(gather(P.pk, P.ac, ct, e) & c.t_mask, lc, c);
    const int ee = P.e1[(size_t)ct * N + e];
    return ee >= 0 ? add_mod(r, (u64)ee, lc.q) : sub_mod(r, (u64)(-ee), lc.q);
  }
  template <int N>
  static __device__ __forceinline__ void store2(const DevCtx& c, const Params& P, const LimbConst& lc, int poly,
                                                int limb, int e, u64 x0, u64 x1) {
    const int ct = poly >> 1, comp = poly & 1;
    const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(P.u_hat + limb_off(ct, limb, c.L, N) + e);
    const ulonglong2 k0 = __ldg(P.key + (size_t)(comp * c.L + limb) * N + e);
    const ulonglong2 k1 = __ldg(P.key + (size_t)(comp * c.L + limb) * N + e + 1);
    const u64 y0 = add_mod(x0, mul_shoup(u.x, k0.x, k0.y, lc.q), lc.q);
    const u64 y1 = add_mod(x1, mul_shoup(u.y, k1.x, k1.y, lc.q), lc.q);
    *reinterpret_cast<ulonglong2*>(P.ct + ct_off(ct, comp, limb, c.L, N) + e) = make_ulonglong2(y0, y1);
  }
};

// DO decryption, first half: x = INTT(c0 + c1 * s_hat); stores y = x * qtilde mod q_j
// (the INTT's N^{-1} and qtilde are one constant).
// With skip_c0 (decryption of the compact send form) only c1 * s is transformed;
// the output coefficients' c0 is added by the combine kernel.
struct ModeDecrypt {
  static constexpr InvScale kInvScale = InvScale::kNqtil;
  static constexpr bool kHeavyLoad = true;
  static constexpr bool kQuad = false;
  static constexpr int kLoadUnroll = 8;
  static constexpr int kEpilogueUnroll = 16;
  struct Params {
    const u64* ct;          // [count][2][L][N]
    const ulonglong2* sk;   // [L][N]
    u64* out;               // [count][L][N]
    int skip_c0;
  };
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx& c, const Params& P, const LimbConst& lc, int poly,
                                             int limb, int e) {
    const u64 c1 = __ldg(P.ct + ct_off(poly, 1, limb, c.L, N) + e);
    const ulonglong2 s = __ldg(P.sk + (size_t)limb * N + e);
    const u64 c1s = mul_shoup(c1, s.x, s.y, lc.q);
    if (P.skip_c0) return c1s;
    return add_mod(__ldg(P.ct + ct_off(poly, 0, limb, c.L, N) + e), c1s, lc.q);
  }
  template <int N>
  static __device__ __forceinline__ void store(const DevCtx& c, const Params& P, const LimbConst& lc, int poly,
                                               int limb, int e, u64 x) {
    P.out[limb_off(poly, limb, c.L, N) + e] = x;   // x = N^{-1} qtil INTT, canonical
  }
};

// DO decryption with the CRT step fused (launched as one cluster of the L limb
// CTAs per ciphertext): each CTA leaves its residues y_j = N^{-1} qtil INTT(c0 +
// c1 s) in its own shared memory (word e at slot e); after a cluster barrier CTA j
// takes coefficient pairs j T + tau + i L T, reads the L residues of each through
// distributed shared memory and writes round(t x / q) mod t to the output
// element the coefficient carries; a second barrier keeps every CTA's shared
// memory alive until the others have read it.  Saves the [count][L][N] residue
// array's write and read and a launch.
struct ModeDecryptFused {
  static constexpr InvScale kInvScale = InvScale::kNqtil;
  static constexpr bool kHeavyLoad = true;
  static constexpr bool kQuad = false;
  static constexpr bool kClusterLimbs = true;
  static constexpr int kLoadUnroll = 8;
  static constexpr int kEpilogueUnroll = 16;
  struct Params {
    ModeDecrypt::Params d;   // d.out unused
    Packing pk;              // output packing
    Accessor ac;             // output layout
    u64* y1;
    int check;
  };
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx& c, const Params& P, const LimbConst& lc, int poly,
                                             int limb, int e) {
    return ModeDecrypt::template load<N>(c, P.d, lc, poly, limb, e);
  }
  template <int N>
  static __device__ __forceinline__ void store(const DevCtx&, const Params&, const LimbConst& lc, int, int, int e,
                                               u64 x) {
    extern __shared__ __align__(16) u64 sm_res[];
    sm_res[e] = x;   // x = N^{-1} qtil INTT, canonical
  }
  template <int N>
  static __device__ __forceinline__ void finish(const DevCtx& c, const Params& P, int poly, u64* sm) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();   // every limb's residues are in its CTA's shared memory
    const int T = (int)blockDim.x;
    const int L = c.L;
    const ulonglong2* res[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      res[j] = reinterpret_cast<const ulonglong2*>(j < L ? cl.map_shared_rank(sm, j) : sm);
    // coefficient pairs (2 p, 2 p + 1): 16-byte remote loads
#pragma unroll 2
    for (int p = (int)blockIdx.y * T + (int)threadIdx.x; p < N / 2; p += L * T) {
      const i64 f0 = out_index(P.pk, P.ac, poly, 2 * p), f1 = out_index(P.pk, P.ac, poly, 2 * p + 1);
      if (f0 < 0 && f1 < 0) continue;
      CrtSum s0{0, 0}, s1{0, 0};
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j < L) {
          const ulonglong2 y = res[j][p];
          crt_add(s0, y.x, c.limb[j]);
          crt_add(s1, y.y, c.limb[j]);
        }
      if (f0 >= 0) P.y1[f0] = crt_round(s0, c.t_mask, P.check, c.status);
      if (f1 >= 0) P.y1[f1] = crt_round(s1, c.t_mask, P.check, c.status);
    }
    cl.sync();   // the other CTAs have finished reading this one's shared memory
  }
};

// MO, compact send form of returned ciphertexts: INTT(c0) and, at the
// coefficients carrying output element flat, c0c[limb][flat] = that coefficient
// (the rest is dropped).
struct ModeCompact {
  static constexpr InvScale kInvScale = InvScale::kNinv;
  static constexpr bool kHeavyLoad = false;
  static constexpr bool kQuad = false;
  static constexpr int kLoadUnroll = 16;
  static constexpr int kEpilogueUnroll = 16;
  struct Params {
    const u64* ct;          // [count][2][L][N]
    Packing pk;             // output packing
    Accessor ac;            // output layout
    u64* c0c;               // [L][out_elems]
    long long out_elems;
  };
  static __device__ __forceinline__ void rebase(Params&, u64) {}
  template <int N>
  static __device__ __forceinline__ u64 load(const DevCtx& c, const Params& P, const LimbConst&, int poly, int limb,
                                             int e) {
    return __ldg(P.ct + ct_off(poly, 0, limb, c.L, N) + e);
  }
  template <int N>
  static __device__ __forceinline__ void store(const DevCtx&, const Params& P, const LimbConst& lc, int poly,
                                               int limb, int e, u64 x) {
    const i64 flat = out_index(P.pk, P.ac, poly, e);
    if (flat >= 0) P.c0c[(size_t)limb * P.out_elems + flat] = x;   // x = N^{-1} INTT, canonical
  }
};

// Host-side launcher; explicitly instantiated per LOGN and engine in ntt12.cu /
// ntt13.cu / ntt14.cu (Shoup) and ntt12f.cu / ntt13f.cu / ntt14f.cu (folds).
template <int LOGN, int LOGE, class Mode, bool INV, bool FOLD>
cudaError_t launch_ntt(const DevCtx& ctx, const typename Mode::Params& P, int first, int count, cudaStream_t s) {
  using C = KCfg<LOGN, LOGE, FOLD>;
  if (count <= 0) return cudaSuccess;
  cudaError_t err;
  dim3 grid((unsigned)count, (unsigned)ctx.L);
  if constexpr (INV) {
    err = cudaFuncSetAttribute(k_ntt_inv<LOGN, LOGE, Mode, FOLD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)C::SMEM);
    if (err != cudaSuccess) return err;
    if constexpr (ClusterLimbs<Mode>::value) {
      // the L limb CTAs of a polynomial form one cluster (portable size <= 8)
      if (ctx.L > 8) return cudaErrorInvalidValue;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = grid;
      cfg.blockDim = dim3((unsigned)C::T);
      cfg.dynamicSmemBytes = C::SMEM;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 1;
      at[0].val.clusterDim.y = (unsigned)ctx.L;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_ntt_inv<LOGN, LOGE, Mode, FOLD>, ctx, P, first);
    } else {
      k_ntt_inv<LOGN, LOGE, Mode, FOLD><<<grid, C::T, C::SMEM, s>>>(ctx, P, first);
    }
  } else {
    err = cudaFuncSetAttribute(k_ntt_fwd<LOGN, LOGE, Mode, FOLD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)C::SMEM);
    if (err != cudaSuccess) return err;
    k_ntt_fwd<LOGN, LOGE, Mode, FOLD><<<grid, C::T, C::SMEM, s>>>(ctx, P, first);
  }
  return cudaGetLastError();
}

template <int LOGN, int LOGE, class Mode, bool INV, bool FOLD>
cudaError_t launch_ntt_multi(const DevCtx& ctx, const typename Mode::Params* Ps, const int2* items, long long count,
                             const u64* step, cudaStream_t s) {
  using C = KCfg<LOGN, LOGE, FOLD>;
  if constexpr (ClusterLimbs<Mode>::value) return cudaErrorNotSupported;   // single-plan launches only
  if (count <= 0) return cudaSuccess;
  if (count > 2147483647ll) return cudaErrorInvalidValue;
  cudaError_t err;
  dim3 grid((unsigned)count, (unsigned)ctx.L);
  if constexpr (INV) {
    err = cudaFuncSetAttribute(k_ntt_inv_multi<LOGN, LOGE, Mode, FOLD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)C::SMEM);
    if (err != cudaSuccess) return err;
    k_ntt_inv_multi<LOGN, LOGE, Mode, FOLD><<<grid, C::T, C::SMEM, s>>>(ctx, Ps, items, step);
  } else {
    err = cudaFuncSetAttribute(k_ntt_fwd_multi<LOGN, LOGE, Mode, FOLD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)C::SMEM);
    if (err != cudaSuccess) return err;
    k_ntt_fwd_multi<LOGN, LOGE, Mode, FOLD><<<grid, C::T, C::SMEM, s>>>(ctx, Ps, items, step);
  }
  return cudaGetLastError();
}

#define PENCIL_NTT_INST1(SPEC, LOGN, LOGE, MODE, INV, FOLD)                                                    \
  SPEC template cudaError_t launch_ntt<LOGN, LOGE, MODE, INV, FOLD>(const DevCtx&, const MODE::Params&, int, int, \
                                                                    cudaStream_t);                             \
  SPEC template cudaError_t launch_ntt_multi<LOGN, LOGE, MODE, INV, FOLD>(const DevCtx&, const MODE::Params*,     \
                                                                          const int2*, long long, const u64*,   \
                                                                          cudaStream_t);
#define PENCIL_NTT_INST_E(SPEC, LOGN, LOGE, FOLD)                \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeRaw, false, FOLD)       \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeRaw, true, FOLD)        \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeEncrypt, false, FOLD)   \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeEncode, false, FOLD)    \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeMoPrep, false, FOLD)    \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeKeygen, false, FOLD)    \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModePkKeygen, false, FOLD)  \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModePkU, false, FOLD)       \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeEncryptPk, false, FOLD) \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeCompact, true, FOLD)    \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeDecrypt, true, FOLD)     \
  PENCIL_NTT_INST1(SPEC, LOGN, LOGE, ModeDecryptFused, true, FOLD)
// Radix 2^4 and 2^5 register blocks for one N and one engine.
#define PENCIL_NTT_INSTANTIATE(SPEC, LOGN, FOLD) \
  PENCIL_NTT_INST_E(SPEC, LOGN, 4, FOLD)         \
  PENCIL_NTT_INST_E(SPEC, LOGN, 5, FOLD)

}  // namespace pencil
