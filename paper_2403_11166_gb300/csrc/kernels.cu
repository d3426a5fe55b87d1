// Element-wise kernels of the hot path: the NTT-domain ct x pt
// multiply-accumulate (Alg. 1 step 2 / Alg. 2 step 2), the samplers for the
// encryption error and the re-mask (Alg. 1 step 3), the MO's output share,
// and the RNS scale-and-round of decryption (Alg. 1 step 4).
#include "cdt_table.h"
#include <algorithm>
#include <cstdio>

#include "kernels.h"

namespace pencil {

__constant__ u64 c_cdt[PENCIL_CDT_LEN];

cudaError_t upload_cdt() {
  return cudaMemcpyToSymbol(c_cdt, kPencilCdt, sizeof(kPencilCdt));
}

// ------------------------------------------------------------------ MAC
// acc[m, n] = sum_k A[m, k] * B[k, n] (+ A'[m, k] * B'[k, n] for Alg. 2),
// slot-wise mod q_j, 128-bit lazy accumulation, one reduction per output.
// Thread = one slot (limb, coefficient) of NT consecutive output columns n.
template <int NT, bool DUAL>
__global__ void __launch_bounds__(256) k_mac(DevCtx ctx, MacParams P) {
  const int lane = blockIdx.x * blockDim.x + threadIdx.x;
  if (lane >= P.lanes) return;
  const int n0 = blockIdx.y * NT;
  const int m = blockIdx.z + P.m_base;
  const int nn = min(NT, P.NC - n0);
  const LimbConst& lc = ctx.limb[lane >> ctx.log_n];
  u64 lo0[NT], hi0[NT], lo1[NT], hi1[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) lo0[j] = hi0[j] = lo1[j] = hi1[j] = 0;
  const int fold = DUAL ? 64 : 128;   // products per accumulator stay below 2^128
  for (int k = 0; k < P.K; ++k) {
    const size_t mk = (size_t)m * P.K + k;
    u64 a0 = __ldg(P.a0 + mk * P.a0_stride + lane);
    if (P.p0) a0 = add_mod(a0, __ldg(P.p0 + mk * P.p0_stride + lane), lc.q);
    const u64 a1 = __ldg(P.a1 + mk * P.a1_stride + lane);
    u64 pa = 0;
    if constexpr (DUAL) pa = __ldg(P.pa + mk * P.pa_stride + lane);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      if (j < nn) {
        const size_t kn = (size_t)k * P.NC + n0 + j;
        const u64 b = __ldg(P.b + kn * P.b_stride + lane);
        mac128(lo0[j], hi0[j], a0, b);
        mac128(lo1[j], hi1[j], a1, b);
        if constexpr (DUAL) {
          const u64 c0 = __ldg(P.cb0 + kn * P.cb_stride + lane);
          const u64 c1 = __ldg(P.cb1 + kn * P.cb_stride + lane);
          mac128(lo0[j], hi0[j], c0, pa);
          mac128(lo1[j], hi1[j], c1, pa);
        }
      }
    }
    if ((k % fold) == fold - 1) {
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        lo0[j] = reduce128(hi0[j], lo0[j], lc);
        lo1[j] = reduce128(hi1[j], lo1[j], lc);
        hi0[j] = hi1[j] = 0;
      }
    }
  }
  const size_t ln = (size_t)P.lanes;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    if (j < nn) {
      const size_t mn = (size_t)m * P.NC + n0 + j, o = mn * 2 * ln + lane;
      u64 v0 = reduce128(hi0[j], lo0[j], lc);
      if (P.mask) v0 = sub_mod(v0, __ldg(P.mask + mn * ln + lane), lc.q);
      P.out[o] = v0;
      P.out[o + ln] = reduce128(hi1[j], lo1[j], lc);
    }
  }
}

// ------------------------------------------------------------------ MAC, 30-bit split
// Same product as k_mac, for q_j < 2^60 with 2^60 and 2^64 mod q_j below 2^28.
// Operands a = aH 2^30 + aL, b = bH 2^30 + bL; each partial product is one
// 32x32->64 multiply-add into one of three 64-bit accumulators of weight 1,
// 2^30, 2^60:  S0 += aL bL,  S1 += aH bL + aL bH,  S2 += aH bH.
// Every FOLD k-steps (at most 12 products per accumulator, so all stay below
// 15 * 2^60 even inside the fold) the accumulators are folded mod q using
// 2^60 = c60 and 2^64 = c64:
//   S0 += lo32(S2) c60;  S1 += hi32(S2) 4 c60;  S2 = 0;
//   S0 += (S1 >> 34) c64;  S1 &= 2^34 - 1;  S1 += S0 >> 30;  S0 &= 2^30 - 1,
// after which S0 < 2^30 and S1 < 2^35.  Thread = one slot, NT output columns.
// Each accumulator is kept as two 32-bit registers (l: low, h: high) and updated
// with a 32-bit carry chain (mad.lo.cc, madc.hi), which the compiler turns into
// one 32x32->64 multiply-add per partial product.  Kept as 64-bit C variables,
// the 24 loop-carried accumulators of a thread compiled to about four more
// instructions per partial product (measured with pipe counters on a
// register-only copy of this loop: 188 against 91 instructions per 32 products).
struct Acc3 {
  u32 l0, h0, l1, h1, l2, h2;   // S0, S1, S2
};

__device__ __forceinline__ void madcc(u32& lo, u32& hi, u32 a, u32 b) {
  asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;" : "+r"(lo), "+r"(hi) : "r"(a), "r"(b));
}

// Four 32x32->64 multiply-adds (S1 gets two; the kernels interleave the
// accumulators of different columns so that the two are far apart).
__device__ __forceinline__ void mac_split(Acc3& a, u32 aL, u32 aH, u32 bL, u32 bH) {
  madcc(a.l0, a.h0, aL, bL);
  madcc(a.l1, a.h1, aH, bL);
  madcc(a.l2, a.h2, aH, bH);
  madcc(a.l1, a.h1, aL, bH);
}

__device__ __forceinline__ void fold3(Acc3& a, u64 c60, u64 c64) {
  madcc(a.l0, a.h0, a.l2, (u32)c60);              // S0 += lo32(S2) c60
  madcc(a.l1, a.h1, a.h2, (u32)(4 * c60));        // S1 += hi32(S2) 4 c60
  a.l2 = 0;
  a.h2 = 0;
  madcc(a.l0, a.h0, a.h1 >> 2, (u32)c64);         // S0 += (S1 >> 34) c64
  a.h1 &= 3u;                                     // S1 &= 2^34 - 1
  const u32 sl = __funnelshift_r(a.l0, a.h0, 30), sh = a.h0 >> 30;   // S0 >> 30
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+r"(a.l1), "+r"(a.h1) : "r"(sl), "r"(sh));
  a.l0 &= (1u << 30) - 1;                         // S0 &= 2^30 - 1
  a.h0 = 0;
}

// canonical value of an accumulator.  After fold3, S0 < 2^30 and S1 < 2^35, and
// S0 + S1 2^30 = S0 + (S1 mod 2^30) 2^30 + (S1 >> 30) 2^60 with 2^60 = c60 mod q
// (c60 < 2^28), a sum below 2^60 + 2^33.  The split form is used only for
// q = 2^60 - c60 with c60 < 2^28, so that sum is below 2 q: one conditional
// subtraction.
__device__ __forceinline__ u64 acc3_value(Acc3 a, const LimbConst& lc) {
  fold3(a, lc.c60, lc.c64);
  const u64 s1 = ((u64)a.h1 << 32) | a.l1;
  const u64 v = (u64)a.l0 + ((s1 & ((1ull << 30) - 1)) << 30) + (u64)(u32)(s1 >> 30) * (u32)lc.c60;
  return csub(v, lc.q);
}

__device__ __forceinline__ void cp_async16(u64* smem, const u64* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}
__device__ __forceinline__ void cp_async8(u64* smem, const u64* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Per-thread operand ring of the split multiply-accumulate: every thread copies
// its own operand words of input blocks k + 1 .. k + MAC_RING - 1 into shared
// memory (8-byte cp.async, no sharing between threads, so no barrier) while it
// multiplies block k; words are stored [stage][word][thread] (consecutive
// threads, consecutive banks).
#define MAC_RING 4
template <int NT, bool DUAL>
struct MacRing {
  // a0, a1, (Alg. 1: NTT(Delta x0) | Alg. 2: A'), B[NT] (Alg. 2: + B'0[NT], B'1[NT])
  static constexpr int W = DUAL ? 3 + 3 * NT : 3 + NT;
  static constexpr size_t bytes(int threads) { return (size_t)MAC_RING * W * threads * sizeof(u64); }
};

// Outputs (m, n0 .. n0 + NT - 1) of one slot `lane`; `ring` = this CTA's ring
// (MacRing::bytes(blockDim.x)), `tid` = this thread's column in it.
template <int NT, bool DUAL>
__device__ __forceinline__ void mac_split_tile(const DevCtx& ctx, const MacParams& P, int m, int n0, int lane,
                                               u64* ring, int tid) {
  constexpr int W = MacRing<NT, DUAL>::W;
  const int T = blockDim.x;
  const int nn = min(NT, P.NC - n0);
  const LimbConst& lc = ctx.limb[lane >> ctx.log_n];
  const u64 c60 = lc.c60, c64 = lc.c64;
  constexpr u32 M30 = (1u << 30) - 1;
  Acc3 acc[NT][2];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int c = 0; c < 2; ++c) acc[j][c] = Acc3{0, 0, 0, 0, 0, 0};
  constexpr int FOLD = DUAL ? 3 : 6;   // at most 12 products of < 2^60 per accumulator between folds
  // operand pointers of the next block to copy (advanced by one block per copy)
  const size_t mk0 = (size_t)m * P.K;
  const u64* pa0 = P.a0 + mk0 * P.a0_stride + lane;
  const u64* pa1 = P.a1 + mk0 * P.a1_stride + lane;
  const u64* pp0 = DUAL ? P.pa + mk0 * P.pa_stride + lane : (P.p0 ? P.p0 + mk0 * P.p0_stride + lane : nullptr);
  const i64 p_step = DUAL ? P.pa_stride : P.p0_stride;
  const u64* pb = P.b + (size_t)n0 * P.b_stride + lane;
  const u64* pc0 = DUAL ? P.cb0 + (size_t)n0 * P.cb_stride + lane : nullptr;
  const u64* pc1 = DUAL ? P.cb1 + (size_t)n0 * P.cb_stride + lane : nullptr;
  const size_t kb = (size_t)P.NC * P.b_stride, kc = (size_t)P.NC * P.cb_stride;
  u64* mine = ring + tid;
  auto word = [&](int stage, int w) -> u64* { return mine + (size_t)(stage * W + w) * T; };
  auto issue = [&](int stage) {
    cp_async8(word(stage, 0), pa0);
    cp_async8(word(stage, 1), pa1);
    if (pp0) cp_async8(word(stage, 2), pp0);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int jj = j < nn ? j : 0;
      cp_async8(word(stage, 3 + j), pb + jj * P.b_stride);
      if constexpr (DUAL) {
        cp_async8(word(stage, 3 + NT + j), pc0 + jj * P.cb_stride);
        cp_async8(word(stage, 3 + 2 * NT + j), pc1 + jj * P.cb_stride);
      }
    }
    pa0 += P.a0_stride;
    pa1 += P.a1_stride;
    if (pp0) pp0 += p_step;
    pb += kb;
    if constexpr (DUAL) {
      pc0 += kc;
      pc1 += kc;
    }
  };
#pragma unroll
  for (int st = 0; st < MAC_RING - 1; ++st) {
    if (st < P.K) issue(st);
    cp_async_commit();
  }
  for (int k = 0; k < P.K; ++k) {
    if (k + MAC_RING - 1 < P.K) issue((k + MAC_RING - 1) % MAC_RING);
    cp_async_commit();
    cp_async_wait<MAC_RING - 1>();   // this thread's copies of block k have landed
    const int st = k % MAC_RING;
    u64 a0 = *word(st, 0);
    if (!DUAL && pp0) a0 = add_mod(a0, *word(st, 2), lc.q);   // Alg. 1 step 2: + NTT(Delta x0)
    const u64 a1 = *word(st, 1);
    const u32 a0L = (u32)a0 & M30, a0H = (u32)(a0 >> 30);
    const u32 a1L = (u32)a1 & M30, a1H = (u32)(a1 >> 30);
    u32 pL = 0, pH = 0;
    if constexpr (DUAL) {
      const u64 pa = *word(st, 2);
      pL = (u32)pa & M30;
      pH = (u32)(pa >> 30);
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const u64 b = *word(st, 3 + j);
      const u32 bL = (u32)b & M30, bH = (u32)(b >> 30);
      mac_split(acc[j][0], a0L, a0H, bL, bH);
      mac_split(acc[j][1], a1L, a1H, bL, bH);
      if constexpr (DUAL) {
        const u64 c0 = *word(st, 3 + NT + j), c1 = *word(st, 3 + 2 * NT + j);
        mac_split(acc[j][0], (u32)c0 & M30, (u32)(c0 >> 30), pL, pH);
        mac_split(acc[j][1], (u32)c1 & M30, (u32)(c1 >> 30), pL, pH);
      }
    }
    if ((k % FOLD) == FOLD - 1) {
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        fold3(acc[j][0], c60, c64);
        fold3(acc[j][1], c60, c64);
      }
    }
  }
  const size_t ln = (size_t)P.lanes;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    if (j < nn) {
      const size_t mn = (size_t)m * P.NC + n0 + j, o = mn * 2 * ln + lane;
      u64 v0 = acc3_value(acc[j][0], lc);
      if (P.mask) v0 = sub_mod(v0, __ldg(P.mask + mn * ln + lane), lc.q);
      P.out[o] = v0;
      P.out[o + ln] = acc3_value(acc[j][1], lc);
    }
  }
}

template <int NT, bool DUAL>
__global__ void __launch_bounds__(128, (NT == 4 && !DUAL) ? 6 : 0) k_mac_ring(DevCtx ctx, MacParams P) {
  extern __shared__ u64 ring[];
  const int ntiles = (P.NC + NT - 1) / NT;
  const int m = blockIdx.x / ntiles + P.m_base;
  const int n0 = (blockIdx.x % ntiles) * NT;
  const int lane = blockIdx.y * blockDim.x + threadIdx.x;
  if (lane >= P.lanes || m >= P.M) return;
  mac_split_tile<NT, DUAL>(ctx, P, m, n0, lane, ring, threadIdx.x);
}

// ------------------------------------------------------------------ MAC, bulk-copy staged
// CTA = MAC_BT consecutive slots of one output tile (m, n0 .. n0 + NT - 1).  For
// every input block k, thread 0 copies the tile's operand rows (a0, a1, then
// NTT(Delta x0) for Alg. 1 or A' for Alg. 2, B[NT], Alg. 2: B'0[NT], B'1[NT];
// MAC_BT words = 1 KB each) from global memory into a ring of MAC_BSTAGES
// shared-memory stages with bulk asynchronous copies (cp.async.bulk, completion
// counted in bytes on one mbarrier per stage), MAC_BSTAGES - 1 blocks ahead of
// the multiply; every thread then reads its own slot's words.  The barrier of
// block k also frees the stage read in block k - 1 for the next copy.  A wait on
// an mbarrier gives up after MAC_WAIT_LIMIT polls: the CTA then sets the timeout
// bit of the status word, lets its issued copies land (bounded the same way) and
// returns.
#define MAC_BT 128
#define MAC_BSTAGES 4
#define MAC_WAIT_LIMIT (1 << 20)
#define MAC_WAIT_HINT_NS 1000

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u32 bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u32 bar, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// One poll; the thread may be suspended for up to MAC_WAIT_HINT_NS while the
// phase is incomplete (instead of spinning on issue slots).
__device__ __forceinline__ bool mbar_try_wait(u32 bar, u32 parity) {
  u32 done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity), "n"(MAC_WAIT_HINT_NS)
      : "memory");
  return done != 0;
}
// At most MAC_WAIT_LIMIT polls (about MAC_WAIT_LIMIT x MAC_WAIT_HINT_NS, ~1 s).
__device__ __forceinline__ bool mbar_wait_bounded(u32 bar, u32 parity) {
  for (int i = 0; i < MAC_WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// 16-byte aligned global source and shared destination, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(u32 dst, const void* src, u32 bytes, u32 bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(u32 bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Warp-specialised: warps 0 .. MAC_BT/32 - 1 multiply (thread = slot), the last
// warp's lane 0 produces.  full[s] completes when stage s holds its block (byte
// count), empty[s] when the MAC_BT/32 consumer warps have finished reading it.
template <int NT, bool DUAL>
__global__ void __launch_bounds__(MAC_BT + 32) k_mac_bulk(DevCtx ctx, MacParams P) {
  constexpr int W = MacRing<NT, DUAL>::W;   // rows per stage
  constexpr u32 ROW = MAC_BT * sizeof(u64);
  constexpr int CONSUMER_WARPS = MAC_BT / 32;
  extern __shared__ __align__(128) u64 ring[];   // [MAC_BSTAGES][W][MAC_BT]
  __shared__ __align__(8) u64 full[MAC_BSTAGES], empty[MAC_BSTAGES];
  const int ntiles = (P.NC + NT - 1) / NT;
  const int m = blockIdx.x / ntiles + P.m_base;
  const int n0 = (blockIdx.x % ntiles) * NT;
  const int lane0 = blockIdx.y * MAC_BT;
  const int tid = threadIdx.x;
  if (m >= P.M) return;   // whole CTA
  const int nn = min(NT, P.NC - n0);
  if (tid == 0) {
#pragma unroll
    for (int st = 0; st < MAC_BSTAGES; ++st) {
      mbar_init(smem_u32(&full[st]), 1);
      mbar_init(smem_u32(&empty[st]), CONSUMER_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid >= MAC_BT) {   // producer warp
    if (tid != MAC_BT) return;
    const bool has_p = DUAL || P.p0 != nullptr;
    const u32 stage_bytes = (u32)(has_p ? W : W - 1) * ROW;
    int k = 0;
    for (; k < P.K; ++k) {
      const int st = k % MAC_BSTAGES;
      if (k >= MAC_BSTAGES && !mbar_wait_bounded(smem_u32(&empty[st]), (u32)(k / MAC_BSTAGES - 1) & 1u)) break;
      const u32 bar = smem_u32(&full[st]);
      const u32 dst = smem_u32(ring + (size_t)st * W * MAC_BT);
      mbar_expect_tx(bar, stage_bytes);
      const size_t mk = (size_t)m * P.K + k;
      bulk_g2s(dst, P.a0 + mk * P.a0_stride + lane0, ROW, bar);
      bulk_g2s(dst + ROW, P.a1 + mk * P.a1_stride + lane0, ROW, bar);
      if (DUAL)
        bulk_g2s(dst + 2 * ROW, P.pa + mk * P.pa_stride + lane0, ROW, bar);
      else if (P.p0)
        bulk_g2s(dst + 2 * ROW, P.p0 + mk * P.p0_stride + lane0, ROW, bar);
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const size_t kn = (size_t)k * P.NC + n0 + (j < nn ? j : 0);
        bulk_g2s(dst + (3 + j) * ROW, P.b + kn * P.b_stride + lane0, ROW, bar);
        if (DUAL) {
          bulk_g2s(dst + (3 + NT + j) * ROW, P.cb0 + kn * P.cb_stride + lane0, ROW, bar);
          bulk_g2s(dst + (3 + 2 * NT + j) * ROW, P.cb1 + kn * P.cb_stride + lane0, ROW, bar);
        }
      }
    }
    if (k < P.K) {   // consumers stopped releasing stages: record it, let the issued copies land
      atomicOr(ctx.status, 2);
      for (int kk = max(0, k - MAC_BSTAGES); kk < k; ++kk)
        mbar_wait_bounded(smem_u32(&full[kk % MAC_BSTAGES]), (u32)(kk / MAC_BSTAGES) & 1u);
    }
    return;
  }
  const int lane = lane0 + tid;
  const LimbConst& lc = ctx.limb[lane >> ctx.log_n];
  const u64 c60 = lc.c60, c64 = lc.c64;
  constexpr u32 M30 = (1u << 30) - 1;
  constexpr int FOLD = DUAL ? 3 : 6;   // at most 12 products of < 2^60 per accumulator between folds
  if (P.mask) {   // the re-mask words the store reads: into L2 now, not from DRAM at the end
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j < nn)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(P.mask + ((size_t)m * P.NC + n0 + j) * (size_t)P.lanes + lane));
  }
  Acc3 acc[NT][2];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = Acc3{0, 0, 0, 0, 0, 0};
  for (int k = 0; k < P.K; ++k) {
    const int st = k % MAC_BSTAGES;
    const bool ok = mbar_wait_bounded(smem_u32(&full[st]), (u32)(k / MAC_BSTAGES) & 1u);
    if (!__all_sync(0xffffffffu, ok)) {   // warp-uniform give-up
      if ((tid & 31) == 0) atomicOr(ctx.status, 2);   // the producer then times out on this warp's stages
      return;
    }
    const u64* cur = ring + (size_t)st * W * MAC_BT + tid;
    u64 a0 = cur[0];
    if (!DUAL && P.p0) a0 = add_mod(a0, cur[2 * MAC_BT], lc.q);   // Alg. 1 step 2: + NTT(Delta x0)
    const u64 a1 = cur[MAC_BT];
    u64 pa = 0, bw[NT], c0w[DUAL ? NT : 1], c1w[DUAL ? NT : 1];
    if constexpr (DUAL) pa = cur[2 * MAC_BT];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      bw[j] = cur[(3 + j) * MAC_BT];
      if constexpr (DUAL) {
        c0w[j] = cur[(3 + NT + j) * MAC_BT];
        c1w[j] = cur[(3 + 2 * NT + j) * MAC_BT];
      }
    }
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(smem_u32(&empty[st]));   // this warp is done with stage st
    const u32 a0L = (u32)a0 & M30, a0H = (u32)(a0 >> 30);
    const u32 a1L = (u32)a1 & M30, a1H = (u32)(a1 >> 30);
    const u32 pL = (u32)pa & M30, pH = (u32)(pa >> 30);
    u32 bL[NT], bH[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      bL[j] = (u32)bw[j] & M30;
      bH[j] = (u32)(bw[j] >> 30);
    }
    // Two passes, each touching every accumulator once, so the two S1 terms of a
    // product are 2 NT multiply-adds apart (no back-to-back dependent pair).
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      madcc(acc[j][0].l0, acc[j][0].h0, a0L, bL[j]);
      madcc(acc[j][0].l1, acc[j][0].h1, a0H, bL[j]);
      madcc(acc[j][1].l0, acc[j][1].h0, a1L, bL[j]);
      madcc(acc[j][1].l1, acc[j][1].h1, a1H, bL[j]);
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      madcc(acc[j][0].l2, acc[j][0].h2, a0H, bH[j]);
      madcc(acc[j][0].l1, acc[j][0].h1, a0L, bH[j]);
      madcc(acc[j][1].l2, acc[j][1].h2, a1H, bH[j]);
      madcc(acc[j][1].l1, acc[j][1].h1, a1L, bH[j]);
    }
    if constexpr (DUAL) {
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        mac_split(acc[j][0], (u32)c0w[j] & M30, (u32)(c0w[j] >> 30), pL, pH);
        mac_split(acc[j][1], (u32)c1w[j] & M30, (u32)(c1w[j] >> 30), pL, pH);
      }
    }
    if ((k % FOLD) == FOLD - 1) {
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        fold3(acc[j][0], c60, c64);
        fold3(acc[j][1], c60, c64);
      }
    }
  }
  const size_t ln = (size_t)P.lanes;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    if (j < nn) {
      const size_t mn = (size_t)m * P.NC + n0 + j, o = mn * 2 * ln + lane;
      u64 v0 = acc3_value(acc[j][0], lc);
      if (P.mask) v0 = sub_mod(v0, __ldg(P.mask + mn * ln + lane), lc.q);
      P.out[o] = v0;
      P.out[o + ln] = acc3_value(acc[j][1], lc);
    }
  }
}

// ------------------------------------------------------------------ MAC, shared-memory staged
// CTA = 32 slots x 8 warps.  The CTA owns an output block of MB x NB (m, n)
// pairs (MB * NB = 64) for its 32 slots; warp w owns pairs 8w .. 8w + 7
// (m = p / NB, n = p % NB).  For every input block k the CTA stages A[m, k]
// (both components), B[k, n] (and, for Alg. 2, A'[m, k], B'[k, n]) of its 32
// slots in shared memory with asynchronous 16-byte copies (cp.async, zero-fill
// outside the layer) into a ring of MAC_STAGES buffers, so the next blocks are
// in flight while block k is multiplied; each operand word is read from L2 / HBM
// once per CTA.
// Every thread multiplies its 8 pairs with the 30-bit split accumulators.
#define MAC_LANES 32
#define MAC_PAIRS 8
#define MAC_STAGES 4


// Global address of row `row` of stage k (or nullptr when outside the layer).
// Rows: [0, 2MB) A components; [2MB, 2MB + NB) B; Alg. 2: [.., + MB) A', [.., + 2NB) B' components.
template <bool DUAL>
__device__ __forceinline__ const u64* mac_row(const MacParams& P, int MB, int NB, int m0, int n0, int k, int row) {
  if (row < 2 * MB) {
    const int m = m0 + (row >> 1);
    if (m >= P.M) return nullptr;
    const size_t mk = (size_t)m * P.K + k;
    return (row & 1) ? P.a1 + mk * P.a1_stride : P.a0 + mk * P.a0_stride;
  }
  row -= 2 * MB;
  if (row < NB) {
    const int n = n0 + row;
    return n < P.NC ? P.b + ((size_t)k * P.NC + n) * P.b_stride : nullptr;
  }
  row -= NB;
  if (row < MB) {   // Alg. 2: A'[m, k]; Alg. 1: NTT(Delta x0)[m, k]
    const int m = m0 + row;
    if (m >= P.M) return nullptr;
    const size_t mk = (size_t)m * P.K + k;
    return DUAL ? P.pa + mk * P.pa_stride : P.p0 + mk * P.p0_stride;
  }
  row -= MB;
  const int n = n0 + (row >> 1);
  if (n >= P.NC) return nullptr;
  const size_t kn = (size_t)k * P.NC + n;
  return ((row & 1) ? P.cb1 : P.cb0) + kn * P.cb_stride;
}

template <bool DUAL>
__device__ __forceinline__ void mac_issue(const MacParams& P, int MB, int NB, int m0, int n0, int k, int lane0, int W,
                                          u64* buf) {
  // W rows x 16 chunks of 16 bytes (two slots each)
  for (int idx = threadIdx.x; idx < W * 16; idx += blockDim.x) {
    const int row = idx >> 4, chunk = idx & 15;
    const u64* g = mac_row<DUAL>(P, MB, NB, m0, n0, k, row);
    cp_async16(buf + row * MAC_LANES + 2 * chunk, g ? g + lane0 + 2 * chunk : P.b, g ? 16 : 0);
  }
}

template <bool DUAL>
__global__ void __launch_bounds__(256, 2) k_mac_smem(DevCtx ctx, MacParams P, int MB, int lnb, int mblocks) {
  const int NB = 1 << lnb;
  extern __shared__ u64 st[];                       // [MAC_STAGES][W][MAC_LANES]
  const int lane0 = blockIdx.x * MAC_LANES;
  const int mb = blockIdx.y % mblocks, nb = blockIdx.y / mblocks;
  const int m0 = mb * MB + P.m_base, n0 = nb * NB;
  const int tid = threadIdx.x, col = tid & (MAC_LANES - 1), warp = tid >> 5;
  const int lane = lane0 + col;
  const bool add_p0 = !DUAL && P.p0 != nullptr;
  const int W = DUAL ? 3 * (MB + NB) : 2 * MB + NB + (add_p0 ? MB : 0);
  constexpr int FOLD = DUAL ? 3 : 6;   // at most 12 products of < 2^60 per accumulator between folds
  constexpr u32 M30 = (1u << 30) - 1;
  const LimbConst& lc = ctx.limb[lane >> ctx.log_n];
  Acc3 acc[MAC_PAIRS][2];
#pragma unroll
  for (int i = 0; i < MAC_PAIRS; ++i) acc[i][0] = acc[i][1] = Acc3{0, 0, 0, 0, 0, 0};
  // ring of MAC_STAGES buffers: blocks k + 1 .. k + MAC_STAGES - 1 in flight while k is multiplied
#pragma unroll
  for (int s = 0; s < MAC_STAGES - 1; ++s) {
    if (s < P.K) mac_issue<DUAL>(P, MB, NB, m0, n0, s, lane0, W, st + (size_t)s * W * MAC_LANES);
    cp_async_commit();
  }
  for (int k = 0; k < P.K; ++k) {
    const u64* cur = st + (size_t)(k % MAC_STAGES) * W * MAC_LANES;
    const int nk = k + MAC_STAGES - 1;
    if (nk < P.K) mac_issue<DUAL>(P, MB, NB, m0, n0, nk, lane0, W, st + (size_t)(nk % MAC_STAGES) * W * MAC_LANES);
    cp_async_commit();
    cp_async_wait<MAC_STAGES - 1>();
    __syncthreads();
    if (add_p0) {  // Alg. 1 step 2: first components += NTT(Delta x0), before any word is split
      u64* w = st + (size_t)(k % MAC_STAGES) * W * MAC_LANES;
      for (int idx = tid; idx < MB * MAC_LANES; idx += blockDim.x) {
        const int r = idx / MAC_LANES, c = idx % MAC_LANES;
        const u64 q = ctx.limb[(lane0 + c) >> ctx.log_n].q;
        w[(2 * r) * MAC_LANES + c] = add_mod(w[(2 * r) * MAC_LANES + c], w[(2 * MB + NB + r) * MAC_LANES + c], q);
      }
      __syncthreads();
    }
    {  // split every staged word once: (low 30 bits) | (high 30 bits) << 32
      u64* w = st + (size_t)(k % MAC_STAGES) * W * MAC_LANES;
      for (int idx = tid; idx < W * MAC_LANES; idx += blockDim.x) {
        const u64 x = w[idx];
        w[idx] = (x & M30) | ((x >> 30) << 32);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAC_PAIRS; ++i) {
      const int p = warp * MAC_PAIRS + i;
      const int mr = p >> lnb, nr = p & (NB - 1);
      const u64 a0 = cur[(2 * mr) * MAC_LANES + col], a1 = cur[(2 * mr + 1) * MAC_LANES + col];
      const u64 b = cur[(2 * MB + nr) * MAC_LANES + col];
      const u32 bL = (u32)b, bH = (u32)(b >> 32);
      mac_split(acc[i][0], (u32)a0, (u32)(a0 >> 32), bL, bH);
      mac_split(acc[i][1], (u32)a1, (u32)(a1 >> 32), bL, bH);
      if constexpr (DUAL) {
        const u64 pa = cur[(2 * MB + NB + mr) * MAC_LANES + col];
        const u64 c0 = cur[(3 * MB + NB + 2 * nr) * MAC_LANES + col];
        const u64 c1 = cur[(3 * MB + NB + 2 * nr + 1) * MAC_LANES + col];
        const u32 pL = (u32)pa, pH = (u32)(pa >> 32);
        mac_split(acc[i][0], (u32)c0, (u32)(c0 >> 32), pL, pH);
        mac_split(acc[i][1], (u32)c1, (u32)(c1 >> 32), pL, pH);
      }
    }
    if ((k % FOLD) == FOLD - 1) {
#pragma unroll
      for (int i = 0; i < MAC_PAIRS; ++i) {
        fold3(acc[i][0], lc.c60, lc.c64);
        fold3(acc[i][1], lc.c60, lc.c64);
      }
    }
    __syncthreads();   // this buffer is refilled by the next iteration's issue
  }
  const size_t ln = (size_t)P.lanes;
#pragma unroll
  for (int i = 0; i < MAC_PAIRS; ++i) {
    const int p = warp * MAC_PAIRS + i;
    const int m = m0 + (p >> lnb), n = n0 + (p & (NB - 1));
    if (m < P.M && n < P.NC) {
      const size_t mn = (size_t)m * P.NC + n, o = mn * 2 * ln + lane;
      u64 v0 = acc3_value(acc[i][0], lc);
      if (P.mask) v0 = sub_mod(v0, __ldg(P.mask + mn * ln + lane), lc.q);
      P.out[o] = v0;
      P.out[o + ln] = acc3_value(acc[i][1], lc);
    }
  }
}

static cudaError_t launch_mac_smem(const DevCtx& ctx, const MacParams& P0, bool dual, cudaStream_t s) {
  // output block: NB = min(64, next power of two >= NC), MB = 64 / NB
  int NB = 1, lnb = 0;
  while (NB < P0.NC && NB < 64) {
    NB <<= 1;
    ++lnb;
  }
  const int MB = 64 / NB;
  const int words = dual ? 3 * (MB + NB) : 2 * MB + NB + (P0.p0 ? MB : 0);
  const size_t smem = (size_t)MAC_STAGES * words * MAC_LANES * sizeof(u64);
  cudaError_t e = dual ? cudaFuncSetAttribute(k_mac_smem<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                       : cudaFuncSetAttribute(k_mac_smem<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nblocks = (P0.NC + NB - 1) / NB;
  MacParams P = P0;
  const unsigned gx = (unsigned)((P.lanes + MAC_LANES - 1) / MAC_LANES);
  const int mchunk_blocks = std::max(1, 65535 / nblocks);
  const int mblocks_total = (P0.M - P0.m_base + MB - 1) / MB;   // output rows m in [m_base, M)
  for (int mbase = 0; mbase < mblocks_total; mbase += mchunk_blocks) {
    const int mblocks = std::min(mchunk_blocks, mblocks_total - mbase);
    P.m_base = P0.m_base + mbase * MB;
    dim3 grid(gx, (unsigned)(mblocks * nblocks));
    if (dual)
      k_mac_smem<true><<<grid, 256, smem, s>>>(ctx, P, MB, lnb, mblocks);
    else
      k_mac_smem<false><<<grid, 256, smem, s>>>(ctx, P, MB, lnb, mblocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int NT>
static cudaError_t launch_mac_ring(const DevCtx& ctx, const MacParams& P0, bool dual, cudaStream_t s) {
  const int threads = 128;
  MacParams P = P0;
  const int ntiles = (P.NC + NT - 1) / NT;
  const unsigned gy = (unsigned)((P.lanes + threads - 1) / threads);
  const int mchunk = max(1, 2147483647 / max(1, ntiles));
  const size_t smem = dual ? MacRing<NT, true>::bytes(threads) : MacRing<NT, false>::bytes(threads);
  cudaError_t e0 = dual ? cudaFuncSetAttribute(k_mac_ring<NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem)
                        : cudaFuncSetAttribute(k_mac_ring<NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
  if (e0 != cudaSuccess) return e0;
  for (long long base = P0.m_base; base < P0.M; base += mchunk) {   // output rows m in [m_base, M)
    P.m_base = (int)base;
    const int mc = (int)std::min<long long>(mchunk, P0.M - base);
    dim3 grid((unsigned)(mc * ntiles), gy);
    if (dual)
      k_mac_ring<NT, true><<<grid, threads, smem, s>>>(ctx, P);
    else
      k_mac_ring<NT, false><<<grid, threads, smem, s>>>(ctx, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int NT>
static cudaError_t launch_mac_bulk(const DevCtx& ctx, const MacParams& P0, bool dual, cudaStream_t s) {
  if (P0.lanes % MAC_BT) return cudaErrorInvalidValue;   // L N is a multiple of 4096
  MacParams P = P0;
  const int ntiles = (P.NC + NT - 1) / NT;
  const unsigned gy = (unsigned)(P.lanes / MAC_BT);
  const int mchunk = max(1, 2147483647 / max(1, ntiles));
  const size_t smem = (size_t)MAC_BSTAGES * (dual ? MacRing<NT, true>::W : MacRing<NT, false>::W) * MAC_BT *
                      sizeof(u64);
  const void* fn = dual ? (const void*)k_mac_bulk<NT, true> : (const void*)k_mac_bulk<NT, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (long long base = P0.m_base; base < P0.M; base += mchunk) {   // output rows m in [m_base, M)
    P.m_base = (int)base;
    const int mc = (int)std::min<long long>(mchunk, P0.M - base);
    dim3 grid((unsigned)(mc * ntiles), gy);
    if (dual)
      k_mac_bulk<NT, true><<<grid, MAC_BT + 32, smem, s>>>(ctx, P);
    else
      k_mac_bulk<NT, false><<<grid, MAC_BT + 32, smem, s>>>(ctx, P);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      fprintf(stderr, "pencil: k_mac_bulk<%d> launch (grid %u x %u, %d threads, %zu B shared, rows [%d, %d)): %s\n", NT,
              grid.x, grid.y, MAC_BT + 32, smem, (int)base, P0.M, cudaGetErrorString(e));
      return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_mac(const DevCtx& ctx, const MacParams& P0, bool dual, cudaStream_t s) {
  if (ctx.mac_split && ctx.mac_nt == 0) return launch_mac_smem(ctx, P0, dual, s);
  if (ctx.mac_split && ctx.mac_staging == 1) {
    switch (ctx.mac_nt) {
      case 2:
        return launch_mac_bulk<2>(ctx, P0, dual, s);
      case 8:
        return launch_mac_bulk<8>(ctx, P0, dual, s);
      default:
        return launch_mac_bulk<4>(ctx, P0, dual, s);
    }
  }
  if (ctx.mac_split) {
    switch (ctx.mac_nt) {
      case 2:
        return launch_mac_ring<2>(ctx, P0, dual, s);
      case 8:
        return launch_mac_ring<8>(ctx, P0, dual, s);
      default:
        return launch_mac_ring<4>(ctx, P0, dual, s);
    }
  }
  constexpr int NT = 8;
  const int threads = 256;
  MacParams P = P0;
  const unsigned gx = (unsigned)((P.lanes + threads - 1) / threads);
  const unsigned gy = (unsigned)((P.NC + NT - 1) / NT);
  for (int base = P0.m_base; base < P0.M; base += 65535) {
    P.m_base = base;
    dim3 grid(gx, gy, (unsigned)min(65535, P0.M - base));
    if (dual)
      k_mac<NT, true><<<grid, threads, 0, s>>>(ctx, P);
    else
      k_mac<NT, false><<<grid, threads, 0, s>>>(ctx, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ samplers
// Encryption error: |e| = #{j : T[j] <= w mod 2^63}, sign = top bit of w,
// w = Philox(key (seed, 3), counter (i/4, ct, 0, 0)) word i%4.
__device__ __forceinline__ int8_t cdt_sample(u64 w) {
  const u64 u = w & 0x7FFFFFFFFFFFFFFFull;
  int mag = 0;
#pragma unroll
  for (int j = 0; j < PENCIL_CDT_LEN; ++j) mag += (u >= c_cdt[j]) ? 1 : 0;
  return (int8_t)((w >> 63) ? -mag : mag);
}

__global__ void k_sample_err(u64 seed, int first, int count, int n, int8_t* out, u64 dom) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int per = n >> 2;
  if (id >= (long long)count * per) return;
  const int ct = first + (int)(id / per);
  const int blk = (int)(id % per);
  const Philox4 w = philox4x64((u64)blk, (u64)ct, 0ull, 0ull, seed, dom);
  reinterpret_cast<char4*>(out + (size_t)ct * n)[blk] =
      make_char4(cdt_sample(w.v[0]), cdt_sample(w.v[1]), cdt_sample(w.v[2]), cdt_sample(w.v[3]));
}

cudaError_t launch_sample_err(u64 seed, int first, int count, int n, int8_t* out, cudaStream_t s, u64 dom) {
  const long long total = (long long)count * (n >> 2);
  if (total == 0) return cudaSuccess;
  k_sample_err<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(seed, first, count, n, out, dom);
  return cudaGetLastError();
}

// Public-key encryption's small polynomials of ciphertexts [first, first + count):
// e1 (PENCIL_DOM_E, the symmetric encryption's stream), e2 (PENCIL_DOM_PK_E2) from
// the CDT and u = (w mod 3) - 1 (PENCIL_DOM_PK_U); counter (i/4, ct, 0, 0), word i%4.
__global__ void k_sample_pk(u64 seed, int first, int count, int n, int8_t* e1, int8_t* e2, int8_t* u) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int per = n >> 2;
  if (id >= (long long)count * per) return;
  const int ct = first + (int)(id / per);
  const int blk = (int)(id % per);
  const size_t o = (size_t)ct * n;
  const Philox4 a = philox4x64((u64)blk, (u64)ct, 0ull, 0ull, seed, PENCIL_DOM_E);
  reinterpret_cast<char4*>(e1 + o)[blk] =
      make_char4(cdt_sample(a.v[0]), cdt_sample(a.v[1]), cdt_sample(a.v[2]), cdt_sample(a.v[3]));
  const Philox4 b = philox4x64((u64)blk, (u64)ct, 0ull, 0ull, seed, PENCIL_DOM_PK_E2);
  reinterpret_cast<char4*>(e2 + o)[blk] =
      make_char4(cdt_sample(b.v[0]), cdt_sample(b.v[1]), cdt_sample(b.v[2]), cdt_sample(b.v[3]));
  const Philox4 c = philox4x64((u64)blk, (u64)ct, 0ull, 0ull, seed, PENCIL_DOM_PK_U);
  reinterpret_cast<char4*>(u + o)[blk] = make_char4((signed char)(c.v[0] % 3ull) - 1, (signed char)(c.v[1] % 3ull) - 1,
                                                    (signed char)(c.v[2] % 3ull) - 1, (signed char)(c.v[3] % 3ull) - 1);
}

cudaError_t launch_sample_pk(u64 seed, int first, int count, int n, int8_t* e1, int8_t* e2, int8_t* u,
                             cudaStream_t s) {
  const long long total = (long long)count * (n >> 2);
  if (total == 0) return cudaSuccess;
  k_sample_pk<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(seed, first, count, n, e1, e2, u);
  return cudaGetLastError();
}

// Mask polynomial of each output ciphertext: at coefficients carrying output
// element `flat`, Philox(key (seed, 4), counter (flat/4, 0, 0, 0)) word flat%4;
// elsewhere Philox(key (seed, 5), counter (i/4, ct, 0, 0)) word i%4; mod t.
// Coefficients 4 blk .. 4 blk + 3 of the mask polynomial of output ciphertext ct.
// Coefficients 4 blk .. 4 blk + 3 of output polynomial ct.  Consecutive
// coefficients usually carry consecutive outputs, so one Philox block of the
// element stream is reused while flat / 4 stays the same; the padding stream
// is drawn only if some coefficient carries no output.
__device__ __forceinline__ void mask_poly_block(const DevCtx& ctx, const Packing& pk, const Accessor& ac, u64 seed,
                                                int ct, int blk, u64* out_ct) {
  i64 flat[4];
  bool any_pad = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    flat[i] = out_index(pk, ac, ct, 4 * blk + i);
    any_pad |= flat[i] < 0;
  }
  Philox4 pad = {{0, 0, 0, 0}};
  if (any_pad) pad = philox4x64((u64)blk, (u64)ct, 0ull, 0ull, seed, PENCIL_DOM_MASK_PAD);
  Philox4 el = {{0, 0, 0, 0}};
  i64 cur = -1;
  u64 r[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    u64 w = philox_word(pad, i);
    if (flat[i] >= 0) {
      if ((flat[i] >> 2) != cur) {
        cur = flat[i] >> 2;
        el = philox4x64((u64)cur, 0ull, 0ull, 0ull, seed, PENCIL_DOM_MASK);
      }
      w = philox_word(el, (int)(flat[i] & 3));
    }
    r[i] = w & ctx.t_mask;
  }
  ulonglong2* o = reinterpret_cast<ulonglong2*>(out_ct + 4 * blk);
  o[0] = make_ulonglong2(r[0], r[1]);
  o[1] = make_ulonglong2(r[2], r[3]);
}

__global__ void k_mask_poly(DevCtx ctx, Packing pk, Accessor ac, u64 seed, int count, u64* out) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = ctx.n;
  const int per = n >> 2;
  if (id >= (long long)count * per) return;
  const int ct = (int)(id / per);
  mask_poly_block(ctx, pk, ac, seed, ct, (int)(id % per), out + (size_t)ct * n);
}

cudaError_t launch_mask_poly(const DevCtx& ctx, const Packing& pk, const Accessor& ac, u64 seed, int count, u64* out,
                             cudaStream_t s) {
  const long long total = (long long)count * (ctx.n >> 2);
  if (total == 0) return cudaSuccess;
  k_mask_poly<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ctx, pk, ac, seed, count, out);
  return cudaGetLastError();
}

// MO share: y0[flat] = s[flat] (+ bias[(flat / hw) % co]) mod t.
// Elements 4 blk .. 4 blk + 3 of the MO share.
__device__ __forceinline__ void mo_share_block(u64 seed, long long count, u64 t_mask, const u64* bias, long long hw,
                                               int co, u64* y0, long long blk) {
  if (blk * 4 >= count) return;
  const Philox4 w = philox4x64((u64)blk, 0ull, 0ull, 0ull, seed, PENCIL_DOM_MASK);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long flat = blk * 4 + i;
    if (flat < count) {
      u64 v = w.v[i] & t_mask;
      if (bias) v = (v + __ldg(bias + (flat / hw) % co)) & t_mask;
      y0[flat] = v;
    }
  }
}

__global__ void k_mo_share(u64 seed, long long count, u64 t_mask, const u64* bias, long long hw, int co, u64* y0) {
  const long long blk = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  mo_share_block(seed, count, t_mask, bias, hw, co, y0, blk);
}

cudaError_t launch_mo_share(u64 seed, long long count, u64 t_mask, const u64* bias, long long hw, int co, u64* y0,
                            cudaStream_t s) {
  const long long blocks = (count + 3) / 4;
  if (blocks == 0) return cudaSuccess;
  k_mo_share<<<(unsigned)((blocks + 255) / 256), 256, 0, s>>>(seed, count, t_mask, bias, hw, co, y0);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ decryption, second half
// y_j = x_j * (q/q_j)^{-1} mod q_j (first half), then crt_add / crt_round.
// c0c (compact send form, else null): c0 at the output coefficients in
// coefficient form, [L][out_elems]; added as c0c * qtil to the INTT(c1 s) residues.
__device__ __forceinline__ void decrypt_combine_one(const DevCtx& ctx, const Packing& pk, const Accessor& ac,
                                                    const u64* yres, int ct, int e, int check, u64* y1,
                                                    const u64* c0c = nullptr, long long out_elems = 0) {
  const int n = ctx.n;
  const i64 flat = out_index(pk, ac, ct, e);
  if (flat < 0) return;
  CrtSum sum{0, 0};
  for (int j = 0; j < ctx.L; ++j) {
    const LimbConst& lc = ctx.limb[j];
    u64 y = __ldg(yres + ((size_t)ct * ctx.L + j) * n + e);
    if (c0c) y = add_mod(y, mul_shoup(__ldg(c0c + (size_t)j * out_elems + flat), lc.qtil, lc.qtils, lc.q), lc.q);
    crt_add(sum, y, lc);
  }
  y1[flat] = crt_round(sum, ctx.t_mask, check, ctx.status);
}

__global__ void k_decrypt_combine(DevCtx ctx, Packing pk, Accessor ac, const u64* yres, int first, int count,
                                  int check, u64* y1, const u64* c0c, long long out_elems) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = ctx.n;
  if (id >= (long long)count * n) return;
  decrypt_combine_one(ctx, pk, ac, yres, first + (int)(id / n), (int)(id % n), check, y1, c0c, out_elems);
}

cudaError_t launch_decrypt_combine(const DevCtx& ctx, const Packing& pk, const Accessor& ac, const u64* yres,
                                   int first, int count, int check, u64* y1, cudaStream_t s, const u64* c0c,
                                   long long out_elems) {
  const long long total = (long long)count * ctx.n;
  if (total == 0) return cudaSuccess;
  k_decrypt_combine<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ctx, pk, ac, yres, first, count, check, y1, c0c,
                                                                    out_elems);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ plaintext ring operators
// Alg. 2's local terms <gY>_j (.) <X>_j and the direct operators over Z_t,
// t = 2^t_bits: u64 wrap-around arithmetic is exact mod t because t | 2^64.
//   out[flat(a, o, i, j)] = addend[flat] + sum_{c, u, v} Wt(o, c, u, v) V(a, c, i + u, j + v)  (mod t)
// Reduction length R = Ci * KH * KW.  Short reductions: one thread per output;
// long ones (grad_W: R = batch x H_out x W_out): one block per output.
__device__ __forceinline__ void ring_store(const RingParams& P, int a, int o, int i, int j, u64 acc) {
  const i64 flat = P.y.base + a * P.y.s0 + o * P.y.s1 + i * P.y.s2 + j * P.y.s3;
  if (P.addend) acc += P.addend[flat];
  if (P.addend2) acc += P.addend2[flat];
  P.out[flat] = acc & P.t_mask;
}

// Short reductions: thread = RING_PT consecutive output positions (a, i, j) x
// RING_OT consecutive output channels o; the reduction runs over (c, u, v) in
// nested loops (no divisions), each kernel value loaded once for the thread's
// RING_PT positions and each input value once for its RING_OT channels (the
// kernel values are the same for every thread of the CTA: one channel tile per
// grid row, broadcast loads).  Channels past Co multiply a zero kernel value.
// RING_OT = 8 channels (measured 11 % faster than 4 on a 16-channel layer) when
// Co >= 8, else 4; 8 positions per thread measured slower; capped at 128
// registers (4 CTAs per SM, measured 6 % faster than 146 registers).
#define RING_PT 4
template <int RING_OT>
__global__ void __launch_bounds__(128, 4) k_ring_tile(RingParams P) {
  const long long npos = P.outs / P.kbound.x;   // B * Ho * Wo
  const long long pos0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * RING_PT;
  if (pos0 >= npos) return;
  const int o0 = blockIdx.y * RING_OT;
  const int Co = P.kbound.x, Ci = P.kbound.y, KH = P.kbound.z, KW = P.kbound.w;
  const long long HWo = (long long)P.Ho * P.Wo;
  const int no = min(RING_OT, Co - o0);
  int pa[RING_PT], pi[RING_PT], pj[RING_PT];
  const u64* vb[RING_PT];
#pragma unroll
  for (int q = 0; q < RING_PT; ++q) {
    const long long pos = pos0 + q < npos ? pos0 + q : pos0;   // a dead slot repeats the first (not stored)
    pa[q] = (int)(pos / HWo);
    const int rem = (int)(pos - (long long)pa[q] * HWo);
    pi[q] = rem / P.Wo;
    pj[q] = rem - pi[q] * P.Wo;
    vb[q] = P.v.ptr + P.v.base + pa[q] * P.v.s0;
  }
  u64 acc[RING_PT][RING_OT];
#pragma unroll
  for (int q = 0; q < RING_PT; ++q)
#pragma unroll
    for (int t = 0; t < RING_OT; ++t) acc[q][t] = 0;
  // Index arithmetic stays out of the innermost loop: row pointers per (c, u),
  // then pointer increments along v (the strides are 64-bit).
  const u64* wb = P.w.ptr + P.w.base + (i64)o0 * P.w.s0;
  i64 woff[RING_OT];
#pragma unroll
  for (int t = 0; t < RING_OT; ++t) woff[t] = t < no ? t * P.w.s0 : 0;
  int col0[RING_PT];
#pragma unroll
  for (int q = 0; q < RING_PT; ++q) col0[q] = pj[q] - P.v.ps;
  for (int c = 0; c < Ci; ++c) {
    const u64* wc = wb + c * P.w.s1;
    for (int u = 0; u < KH; ++u) {
      const u64* xp[RING_PT];
      bool rok[RING_PT];
#pragma unroll
      for (int q = 0; q < RING_PT; ++q) {
        const int rr = pi[q] + u - P.v.pr;
        rok[q] = (unsigned)rr < (unsigned)P.v.hr;
        xp[q] = vb[q] + c * P.v.s1 + (rok[q] ? rr : 0) * P.v.s2 + col0[q] * P.v.s3;
      }
      const u64* wp = wc + u * P.w.s2;
      for (int v = 0; v < KW; ++v) {
        u64 wv[RING_OT];
#pragma unroll
        for (int t = 0; t < RING_OT; ++t) wv[t] = t < no ? __ldg(wp + woff[t]) : 0ull;
#pragma unroll
        for (int q = 0; q < RING_PT; ++q) {
          if (rok[q] && (unsigned)(col0[q] + v) < (unsigned)P.v.wr) {
            const u64 x = __ldg(xp[q]);
#pragma unroll
            for (int t = 0; t < RING_OT; ++t) acc[q][t] += x * wv[t];
          }
          xp[q] += P.v.s3;
        }
        wp += P.w.s3;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < RING_PT; ++q)
    if (pos0 + q < npos)
#pragma unroll
      for (int t = 0; t < RING_OT; ++t)
        if (t < no) ring_store(P, pa[q], o0 + t, pi[q], pj[q], acc[q][t]);
}

// Long reductions (grad_W: over batch x output positions): one CTA per output,
// threads over the (u, v) positions of each c (consecutive threads read
// consecutive elements).
__global__ void __launch_bounds__(256) k_ring_block(RingParams P) {
  const long long id = blockIdx.x;
  const int KH = P.kbound.z, KW = P.kbound.w, Ci = P.kbound.y;
  const int j = (int)(id % P.Wo);
  const int i = (int)((id / P.Wo) % P.Ho);
  const int o = (int)((id / ((long long)P.Wo * P.Ho)) % P.kbound.x);
  const int a = (int)(id / ((long long)P.Wo * P.Ho * P.kbound.x));
  const int UV = KH * KW;
  u64 acc = 0;
  const u64* vb = P.v.ptr + P.v.base + a * P.v.s0;
  const u64* wb = P.w.ptr + P.w.base + o * P.w.s0;
  for (int c = 0; c < Ci; ++c) {
    for (int q = threadIdx.x; q < UV; q += blockDim.x) {
      const int u = q / KW, v = q - (q / KW) * KW;
      const int rr = i + u - P.v.pr, ss = j + v - P.v.ps;
      if ((unsigned)rr >= (unsigned)P.v.hr || (unsigned)ss >= (unsigned)P.v.wr) continue;
      acc += __ldg(vb + c * P.v.s1 + rr * P.v.s2 + ss * P.v.s3) * __ldg(wb + c * P.w.s1 + u * P.w.s2 + v * P.w.s3);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ u64 part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    ring_store(P, a, o, i, j, s);
  }
}

// Long reductions with a short output (grad_W's HO x WO kernel offsets, at
// most 5 x 5): one CTA per (a, o) keeps all HO * WO outputs in registers, so
// each kernel value (grad_Y) is loaded once for all of them and the input rows
// around it come from L1; (u, v) advance by the block size without a division.
template <int HO, int WO>
__global__ void __launch_bounds__(256) k_ring_wgrad(RingParams P) {
  const int Co = P.kbound.x, Ci = P.kbound.y, KH = P.kbound.z, KW = P.kbound.w;
  const int o = (int)(blockIdx.x % (unsigned)Co);
  const int a = (int)(blockIdx.x / (unsigned)Co);
  const int UV = KH * KW;
  u64 acc[HO * WO];
#pragma unroll
  for (int t = 0; t < HO * WO; ++t) acc[t] = 0;
  const u64* vb = P.v.ptr + P.v.base + a * P.v.s0;
  const u64* wb = P.w.ptr + P.w.base + (i64)o * P.w.s0;
  const int su = (int)blockDim.x / KW, sv = (int)blockDim.x - su * KW;
  const int u0 = (int)threadIdx.x / KW, v0 = (int)threadIdx.x - u0 * KW;
  for (int c = 0; c < Ci; ++c) {
    const u64* vc = vb + c * P.v.s1;
    const u64* wc = wb + c * P.w.s1;
    int u = u0, v = v0;
    for (int q = threadIdx.x; q < UV; q += blockDim.x) {
      const u64 g = __ldg(wc + u * P.w.s2 + v * P.w.s3);
#pragma unroll
      for (int i = 0; i < HO; ++i) {
        const int rr = i + u - P.v.pr;
        if ((unsigned)rr >= (unsigned)P.v.hr) continue;
        const u64* row = vc + rr * P.v.s2;
#pragma unroll
        for (int j = 0; j < WO; ++j) {
          const int ss = j + v - P.v.ps;
          if ((unsigned)ss < (unsigned)P.v.wr) acc[i * WO + j] += g * __ldg(row + ss * P.v.s3);
        }
      }
      u += su;
      v += sv;
      if (v >= KW) {
        v -= KW;
        ++u;
      }
    }
  }
  __shared__ u64 part[8][HO * WO];   // 256 threads = 8 warps
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < HO * WO; ++t) {
    u64 x = acc[t];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) part[warp][t] = x;
  }
  __syncthreads();
  if ((int)threadIdx.x < HO * WO) {
    u64 sum = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += part[w][threadIdx.x];
    ring_store(P, a, o, (int)threadIdx.x / WO, (int)threadIdx.x % WO, sum);
  }
}

cudaError_t launch_ring(const RingParams& P, cudaStream_t s) {
  const long long R = (long long)P.kbound.y * P.kbound.z * P.kbound.w;
  if (P.outs == 0) return cudaSuccess;
  if ((long long)P.kbound.z * P.kbound.w >= 256 && P.outs <= (1ll << 31) - 1) {
    const long long pairs = P.outs / ((long long)P.Ho * P.Wo);   // (a, o) pairs
    if (P.Ho == 3 && P.Wo == 3)
      k_ring_wgrad<3, 3><<<(unsigned)pairs, 256, 0, s>>>(P);
    else if (P.Ho == 5 && P.Wo == 5)
      k_ring_wgrad<5, 5><<<(unsigned)pairs, 256, 0, s>>>(P);
    else if (P.Ho == 1 && P.Wo == 1)
      k_ring_wgrad<1, 1><<<(unsigned)pairs, 256, 0, s>>>(P);
    else
      k_ring_block<<<(unsigned)P.outs, 256, 0, s>>>(P);
  } else {
    const long long positions = P.outs / P.kbound.x;
    const unsigned gx = (unsigned)((positions + 128 * RING_PT - 1) / (128 * RING_PT));
    const int ot = P.kbound.x >= 8 ? 8 : 4;
    const unsigned gy = (unsigned)((P.kbound.x + ot - 1) / ot);
    if (gy > 65535) return cudaErrorInvalidValue;
    (void)R;
    if (ot == 8)
      k_ring_tile<8><<<dim3(gx, gy), 128, 0, s>>>(P);
    else
      k_ring_tile<4><<<dim3(gx, gy), 128, 0, s>>>(P);
  }
  return cudaGetLastError();
}

// Bias gradient: out[o] = sum_{b, i, j} g[b, o, i, j] mod t   (g row-major [B][Co][HW]).
__global__ void __launch_bounds__(256) k_bias_grad(const u64* g, int B, int Co, long long hw, u64 t_mask, u64* out) {
  const int o = blockIdx.x;
  const long long R = (long long)B * hw;
  u64 acc = 0;
  for (long long r = threadIdx.x; r < R; r += blockDim.x) {
    const long long b = r / hw, p = r % hw;
    acc += __ldg(g + (b * Co + o) * hw + p);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ u64 part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 s = 0;
    for (int w = 0; w < 8; ++w) s += part[w];
    out[o] = s & t_mask;
  }
}

cudaError_t launch_bias_grad(const u64* g, int B, int Co, long long hw, u64 t_mask, u64* out, cudaStream_t s) {
  if (Co == 0) return cudaSuccess;
  k_bias_grad<<<Co, 256, 0, s>>>(g, B, Co, hw, t_mask, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ linear combinations of shares
// Online phase of the preprocessing protocol (Alg. 3): masked operands and
// shares are linear combinations over Z_t, t = 2^t_bits (u64 wrap-around is
// exact mod t):  out[e] = addend[e] (+ or -) sum_{i2, i} k[i2 terms + i]
// src[off + (e / inner) outer + e % inner + i tstride + i2 tstride2].
__global__ void k_lincomb(LincombP P, u64 t_mask) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < P.count; e += stride) {
    const long long base = P.off + (e / P.inner) * P.outer + e % P.inner;
    u64 acc = 0;
    for (int i2 = 0; i2 < P.terms2; ++i2) {
      const u64* src = P.src + base + i2 * P.tstride2;
      const u64* k = P.k + i2 * P.terms;
      for (int i = 0; i < P.terms; ++i) acc += k[i] * __ldg(src + i * P.tstride);
    }
    u64 v = P.addend ? __ldg(P.addend + e) : 0ull;
    v = P.negate ? v - acc : v + acc;
    P.out[e] = v & t_mask;
  }
}

cudaError_t launch_lincomb(const LincombP& P, u64 t_mask, cudaStream_t s) {
  if (P.count <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((P.count + 255) / 256, 152LL * 16);
  k_lincomb<<<(unsigned)blocks, 256, 0, s>>>(P, t_mask);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ batched layers
// Many linear layers (Alg. 1 forward) with a fixed launch sequence: every stage
// of every layer runs in one multi-plan launch over (layer, polynomial) items,
// and the ct x pt products of all layers run in ONE persistent launch over a
// (layer, m, n-tile, lane-block) work list.  Nothing is allocated or copied at
// run time, so the sequence can be captured in a CUDA graph; a device step
// counter re-keys the randomness of every replay.  The persistent
// multiply-accumulate consumes a layer's inputs only after that layer's ready
// word carries the current step (written by a signal kernel after the input
// stages); waits are bounded by clock64 and, on expiry, set PENCIL_E_TIMEOUT in
// the status word and abort the remaining items instead of reading stale data.
// ------------------------------------------------------------------ small multi-plan kernels
__global__ void k_sample_err_multi(const SampleP* __restrict__ Ps, const int2* __restrict__ items, long long n_items,
                                   int n, const u64* step) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int per = n >> 2;
  if (id >= n_items * per) return;
  const int2 it = items[id / per];
  const int blk = (int)(id % per);
  const SampleP P = Ps[it.x];
  const u64 seed = P.seed + ((step ? *step : 0ull) << 32);
  const Philox4 w = philox4x64((u64)blk, (u64)it.y, 0ull, 0ull, seed, PENCIL_DOM_E);
  int8_t v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = cdt_sample(w.v[i]);
  reinterpret_cast<char4*>(P.err + (size_t)it.y * n)[blk] = make_char4(v[0], v[1], v[2], v[3]);
}

__global__ void k_mask_poly_multi(DevCtx ctx, const MaskPolyP* __restrict__ Ps, const int2* __restrict__ items,
                                  long long n_items, const u64* step) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = ctx.n;
  const int per = n >> 2;
  if (id >= n_items * per) return;
  const int2 it = items[id / per];
  const int blk = (int)(id % per);
  const MaskPolyP P = Ps[it.x];
  const u64 seed = P.seed + ((step ? *step : 0ull) << 32);
  mask_poly_block(ctx, P.pk, P.ac, seed, it.y, blk, P.out + (size_t)it.y * n);
}

__global__ void k_mo_share_multi(const MoShareP* __restrict__ Ps, const int2* __restrict__ items, long long n_items,
                                 u64 t_mask, const u64* step) {
  // item = (layer, chunk of 1024 elements); thread = 4 consecutive elements
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_items * 256) return;
  const int2 it = items[id / 256];
  const MoShareP P = Ps[it.x];
  const long long blk = (long long)it.y * 256 + id % 256;
  const u64 seed = P.seed + ((step ? *step : 0ull) << 32);
  mo_share_block(seed, P.count, t_mask, P.bias, P.hw, P.co, P.y0, blk);
}

__global__ void k_combine_multi(DevCtx ctx, const CombineP* __restrict__ Ps, const int2* __restrict__ items,
                                long long n_items) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = ctx.n;
  if (id >= n_items * n) return;
  const int2 it = items[id / n];
  const CombineP P = Ps[it.x];
  decrypt_combine_one(ctx, P.pk, P.ac, P.yres, it.y, (int)(id % n), 1, P.y1);
}

// ready[l] = step + 1 for every layer except one the host asked to withhold
__global__ void k_signal(u64* ready, int n_layers, int withhold, const u64* step) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n_layers && l != withhold) ready[l] = (step ? *step : 0ull) + 1;
}

__global__ void k_step_advance(u64* step) { *step += 1; }

// ------------------------------------------------------------------ persistent multiply-accumulate
#define PENCIL_GATE_LIMIT_CYCLES (4ll << 20)   // about 2 ms at 2 GHz

// Waits until ready[layer] == want; thread 0 polls, the block shares the verdict.
__device__ __forceinline__ bool wait_ready(const u64* ready, int layer, u64 want, int* status, int* abort_flag) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const volatile u64* r = ready + layer;
    const volatile int* ab = abort_flag;
    int good = 1;
    if (*r != want) {
      const long long t0 = clock64();
      while (*r != want) {
        if (*ab) {
          good = 0;
          break;
        }
        if (clock64() - t0 > PENCIL_GATE_LIMIT_CYCLES) {
          atomicOr(status, 2);
          atomicExch(abort_flag, 1);
          good = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    ok = good;
  }
  __syncthreads();
  const int v = ok;
  __syncthreads();
  return v != 0;
}

// HAS_DUAL: the batch holds Alg. 2 layers (MacParams::pa set), whose tiles take
// two products per input block; the ring is then sized for them.
template <int NT, bool HAS_DUAL>
__global__ void __launch_bounds__(128) k_mac_persistent(DevCtx ctx, const MacParams* __restrict__ Ps,
                                                        const int4* __restrict__ items, long long n_items,
                                                        const u64* ready, const u64* step, int* abort_flag) {
  extern __shared__ u64 ring[];
  const u64 want = (step ? *step : 0ull) + 1;
  for (long long i = blockIdx.x; i < n_items; i += gridDim.x) {
    const int4 it = items[i];   // (layer, m, n0, lane block)
    if (!wait_ready(ready, it.x, want, ctx.status, abort_flag)) return;
    const MacParams& P = Ps[it.x];
    const int lane = it.w * blockDim.x + threadIdx.x;
    if (lane >= P.lanes) continue;
    if constexpr (HAS_DUAL) {
      if (P.pa) {
        mac_split_tile<NT, true>(ctx, P, it.y, it.z, lane, ring, threadIdx.x);
        continue;
      }
    }
    mac_split_tile<NT, false>(ctx, P, it.y, it.z, lane, ring, threadIdx.x);
  }
}

template <int NT, bool HAS_DUAL>
static cudaError_t launch_mac_persistent(const DevCtx& ctx, const BatchDev& B, unsigned grid, cudaStream_t s) {
  constexpr size_t smem = MacRing<NT, HAS_DUAL>::bytes(128);
  const cudaError_t e =
      cudaFuncSetAttribute(k_mac_persistent<NT, HAS_DUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_mac_persistent<NT, HAS_DUAL><<<grid, 128, smem, s>>>(ctx, B.mac, B.items_mac, B.n_mac, B.ready, B.step,
                                                         B.abort_flag);
  return cudaGetLastError();
}

template <int NT, bool HAS_DUAL>
static cudaError_t mac_persistent_occupancy(int* per) {
  constexpr size_t smem = MacRing<NT, HAS_DUAL>::bytes(128);
  const cudaError_t e =
      cudaFuncSetAttribute(k_mac_persistent<NT, HAS_DUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_mac_persistent<NT, HAS_DUAL>, 128, smem);
}

// ------------------------------------------------------------------ launchers
static unsigned blocks_for(long long threads, int per) { return (unsigned)((threads + per - 1) / per); }

cudaError_t launch_batch_forward(const DevCtx& ctx, const BatchDev& B, cudaStream_t s) {
  cudaError_t e;
  const int n = ctx.n;
  if (B.n_pt) {
    e = ntt_multi<ModeEncode, false>(ctx, B.encode, B.items_pt, B.n_pt, B.step, s);
    if (e != cudaSuccess) return e;
  }
  if (B.n_in) {
    k_sample_err_multi<<<blocks_for(B.n_in * (n / 4), 256), 256, 0, s>>>(B.sample, B.items_in, B.n_in, n, B.step);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = ntt_multi<ModeEncrypt, false>(ctx, B.encrypt, B.items_in, B.n_in, B.step, s);
    if (e != cudaSuccess) return e;
  }
  if (B.n_out) {   // the MO's mask s, then NTT(Delta x0) and NTT(Delta s) of every layer in one launch
    k_mask_poly_multi<<<blocks_for(B.n_out * (n / 4), 256), 256, 0, s>>>(ctx, B.maskpoly, B.items_out, B.n_out,
                                                                            B.step);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (B.n_prep) {
    e = ntt_multi<ModeMoPrep, false>(ctx, B.prep, B.items_prep, B.n_prep, B.step, s);
    if (e != cudaSuccess) return e;
  }
  k_signal<<<blocks_for(B.n_layers, 128), 128, 0, s>>>(B.ready, B.n_layers, B.withhold, B.step);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (B.n_mac) {
    const unsigned grid = (unsigned)std::min<long long>(B.n_mac, (long long)B.mac_blocks);
    if (B.has_dual) {
      e = B.mac_nt == 2   ? launch_mac_persistent<2, true>(ctx, B, grid, s)
          : B.mac_nt == 8 ? launch_mac_persistent<8, true>(ctx, B, grid, s)
                          : launch_mac_persistent<4, true>(ctx, B, grid, s);
    } else {
      e = B.mac_nt == 2   ? launch_mac_persistent<2, false>(ctx, B, grid, s)
          : B.mac_nt == 8 ? launch_mac_persistent<8, false>(ctx, B, grid, s)
                          : launch_mac_persistent<4, false>(ctx, B, grid, s);
    }
    if (e != cudaSuccess) return e;
  }
  if (B.n_share) {
    k_mo_share_multi<<<blocks_for(B.n_share * 256, 256), 256, 0, s>>>(B.moshare, B.items_share, B.n_share,
                                                                         ctx.t_mask, B.step);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (B.n_out) {
    e = ntt_multi<ModeDecrypt, true>(ctx, B.decrypt, B.items_out, B.n_out, B.step, s);
    if (e != cudaSuccess) return e;
    k_combine_multi<<<blocks_for(B.n_out * n, 256), 256, 0, s>>>(ctx, B.combine, B.items_out, B.n_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_step_advance<<<1, 1, 0, s>>>(B.step);
  return cudaGetLastError();
}

cudaError_t batch_mac_blocks(const DevCtx& ctx, int nt, int has_dual, int* blocks) {
  (void)ctx;
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (has_dual)
      e = nt == 2 ? mac_persistent_occupancy<2, true>(&per)
          : nt == 8 ? mac_persistent_occupancy<8, true>(&per) : mac_persistent_occupancy<4, true>(&per);
    else
      e = nt == 2 ? mac_persistent_occupancy<2, false>(&per)
          : nt == 8 ? mac_persistent_occupancy<8, false>(&per) : mac_persistent_occupancy<4, false>(&per);
  }
  *blocks = std::max(1, sms * std::max(1, per));
  return e;
}

// ------------------------------------------------------------------ multiply-pipe probe
// Register-only chains measuring the 32-bit integer multiply-add rate (which = 0)
// or the 64-bit Shoup modular-multiply rate (which = 1).  Eight independent
// chains per thread; the result is stored only if it equals a value it cannot
// take, so nothing is optimised away and nothing is written.
__global__ void k_mul_probe(int which, long long iters, u64 seed, u64* sink) {
  const u32 t = threadIdx.x + blockIdx.x * blockDim.x;
  if (which == 0) {
    u32 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (u32)seed + t * 2654435761u + i;
    const u32 a = (u32)(seed >> 32) | 1u, b = (u32)seed ^ 0x9e3779b9u;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(a), "r"(b));
    }
    u32 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    if (acc == 0xFFFFFFFFu && seed == 0) sink[0] = acc;
  } else if (which == 1) {
    const u64 q = 0xfffffffffffc001ull;
    const u64 w = (seed | 1ull) % q;
    const u64 ws = (u64)((((unsigned __int128)w) << 64) / q);
    u64 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (seed + t * 0x9E3779B97F4A7C15ull + i) % q;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = mul_shoup_lazy(x[i], w, ws, q);
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    if (acc == ~0ull && seed == 0) sink[0] = acc;
  } else if (which == 2) {
    // 32 x 32 -> 64 multiply with 64-bit accumulate (mad.wide.u32), 8 chains
    u64 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = seed + t + i;
    const u32 a = (u32)(seed >> 32) | 1u, b = (u32)seed ^ 0x9e3779b9u;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        asm volatile("{\n\t.reg .u32 lo;\n\tcvt.u32.u64 lo, %0;\n\tmad.wide.u32 %0, lo, %1, %0;\n\t}"
                     : "+l"(x[i])
                     : "r"(a ^ (b + i)));
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    if (acc == ~0ull && seed == 0) sink[0] = acc;
  } else if (which == 9) {
    // 32 x 32 -> high 32 bits (mul.hi.u32), 8 dependent chains
    u32 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (u32)seed + t * 2654435761u + i;
    const u32 a = (u32)(seed >> 32) | 0x80000001u;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(x[i]) : "r"(a + i));
    }
    u32 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    if (acc == 0xFFFFFFFFu && seed == 0) sink[0] = acc;
  } else if (which >= 10) {
    // pseudo-Mersenne products and butterflies (q = 2^60 - 16383), 8 independent values:
    // 10 mul_fold (PTX), 11 mul_fold_c (C), 12 ct_fold, 13 gs_fold, 14 fold60, 15 ct butterfly with mul_fold_c
    const u64 q = 0xfffffffffffc001ull, q2 = 2 * q, q4 = 4 * q;
    const u32 c60 = 16383u, c64 = 16u * 16383u;
    const u64 w = (seed | 1ull) % q, w32 = (u64)((((unsigned __int128)w) << 32) % q);
    const ulonglong2 ww = make_ulonglong2(w, w32);
    u64 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (seed + t * 0x9E3779B97F4A7C15ull + i) % q;
    for (long long it = 0; it < iters; ++it) {
      if (which == 10) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = mul_fold(x[i], w, w32, c60, c64);
      } else if (which == 11) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = mul_fold_c(x[i], w, w32, c60, c64);
      } else if (which == 12) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) ct_fold(x[i], x[i + 1], ww, c60, c64, q2);
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fold60(x[i], c60);   // keep the chain bounded
      } else if (which == 13) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) gs_fold(x[i], x[i + 1], ww, c60, c64, q4);
#pragma unroll
        for (int i = 0; i < 8; i += 2) x[i] = fold60(x[i], c60);
      } else if (which == 14) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fold60(x[i] * 3 + 1, c60);
      } else {
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          const u64 tt = mul_fold_c(x[i + 1], ww.x, ww.y, c60, c64);
          x[i + 1] = x[i] + q2 - tt;
          x[i] = x[i] + tt;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fold60(x[i], c60);
      }
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    // (the lazy results are below 2^61, so the test must not be provably false)
    if (acc == (seed ^ 0x5DEECE66Dull) * 3u) sink[0] = acc;
  } else if (which >= 4) {
    // butterfly / modmul formulations of the NTT kernels, 8 independent values
    const u64 q = 0xfffffffffffc001ull, q2 = 2 * q, q3 = 3 * q, q4 = 4 * q, nq = 0ull - q;
    const u64 w = (seed | 1ull) % q;
    const u64 ws = (u64)((((unsigned __int128)w) << 64) / q);
    u64 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (seed + t * 0x9E3779B97F4A7C15ull + i) % q;
    for (long long it = 0; it < iters; ++it) {
      if (which == 4) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = mul_shoup3(x[i], w, ws, nq);
      } else if (which == 5) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) ct_bf8(x[i], x[i + 1], w, ws, nq, q3, q4);
#pragma unroll
        for (int i = 0; i < 8; i += 2) ct_bf8(x[i + 1], x[i], w, ws, nq, q3, q4);
      } else if (which == 6) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) ct_butterfly(x[i], x[i + 1], w, ws, q, q2);
#pragma unroll
        for (int i = 0; i < 8; i += 2) ct_butterfly(x[i + 1], x[i], w, ws, q, q2);
      } else if (which == 7) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) gs_bf4(x[i], x[i + 1], w, ws, nq, q4);
#pragma unroll
        for (int i = 0; i < 8; i += 2) gs_bf4(x[i + 1], x[i], w, ws, nq, q4);
      } else {
#pragma unroll
        for (int i = 0; i < 8; i += 2) gs_butterfly(x[i], x[i + 1], w, ws, q, q2);
#pragma unroll
        for (int i = 0; i < 8; i += 2) gs_butterfly(x[i + 1], x[i], w, ws, q, q2);
      }
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    if (acc == ~0ull && seed == 0) sink[0] = acc;
  } else {
    // 64 x 64 -> 128 multiply-accumulate as written in the MAC kernel
    u64 lo[8], hi[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) lo[i] = hi[i] = seed + t + i;
    const u64 a = seed | 1ull, b = seed ^ 0x0123456789abcdefull;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i) mac128(lo[i], hi[i], a + i, b ^ lo[i]);
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= lo[i] ^ hi[i];
    if (acc == ~0ull && seed == 0) sink[0] = acc;
  }
}

cudaError_t launch_mul_probe(int which, long long iters, int blocks, int threads, u64 seed, u64* sink,
                             cudaStream_t s) {
  k_mul_probe<<<blocks, threads, 0, s>>>(which, iters, seed, sink);
  return cudaGetLastError();
}

}  // namespace pencil
