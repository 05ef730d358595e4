// Fused HEOM right-hand side + RK4 (Horner form) stage kernel for sm_103a.
//
// One launch evaluates, for every ADO u in [u_begin, u_end),
//     out_u = y_u + ch * (L zin)_u          (or ch * (L zin)_u when there is no y)
// where L is the right-hand side of Eq. HEOM (arXiv 1803.03498, section "HEOM formalism") with the
// ADO rescaling, written element-wise (hbar = 1, energies in rad/fs):
//   (L s)_ij = -i sum_k (H_ik s_kj - s_ik H_kj) - (sum_l n_l gamma_l) s_ij
//              - [i != j] (Delta_i + Delta_j) s_ij  + (links)
// where every valid +/- link of u to a neighbour v through a mode of state s adds R v_sj to
// element (s, j != s), conj(R) v_is to element (i != s, s) and 2 Re(R) v_ss to (s, s) (V^x is +1 on
// row s and -1 on column s, V^o is +1 on both; see LinkRec).
//
// Every warp works on its own chunks of A = floor(32 / N) consecutive ADOs, independently of the
// other warps (only __syncwarp), in a software pipeline:
//  - the record offsets of the chunk after next are loaded into registers;
//  - 16-byte cp.async copies bring the next chunk's tiles (each ADO's N x N tile is contiguous) and
//    link records into a second buffer, and the current chunk's y tiles into shared memory;
//  - cp.async gathers row s and column s of every linked neighbour of the current chunk;
//  - while those are in flight, lane (a, i) computes row i of ADO a: the commutator (the lanes of
//    one ADO read the same tile words, a broadcast; H sits in the kernel parameters, addressed by
//    the unrolled loops with compile-time offsets), decay and terminator;
//  - links: in Hermitian runs of the FP32 kernels with N <= 16, every link record goes to the one lane
//    that owns row s of its ADO, which adds R v_{s, .} to its row in registers, and a transpose through
//    shared memory forms Q + Q^dagger at the end; otherwise the lanes add each link to elements (s, i)
//    and (i, s) of their ADO's output tile in shared memory;
//  - y + ch * output leaves with 16-byte coalesced stores.
// A chunk with more links than fit the slice buffer (RC slices of 2N elements, or 2 RC
// row-only slices of N elements for Hermitian runs) handles the rest in further synchronous batches.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "heom_internal.h"

namespace heom {

template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
  using type = float2;
};
template <>
struct Cplx<double> {
  using type = double2;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// Copy `bytes` (a multiple of 16; both 16-byte aligned) with the lanes of one warp.
__device__ __forceinline__ void warp_copy16(void *dst, const void *src, int bytes, int lane) {
  char *d = reinterpret_cast<char *>(dst);
  const char *s = reinterpret_cast<const char *>(src);
  for (int o = lane * 16; o < bytes; o += 32 * 16) cp_async16(d + o, s + o);
}

// L2 eviction priorities.  A stage reads its own tiles once (a stream through L2), while a row it
// gathers from a neighbour is wanted again by the neighbour's other linked ADOs of the launch (every
// state has two modes, K + 1 in general): own tiles go in as evict_first, gathered rows as
// evict_last.  HEOM_L2_HINTS=0 (tuning builds) drops the hints.
#ifndef HEOM_L2_HINTS
#define HEOM_L2_HINTS 1
#endif
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async16_hint(void *smem, const void *gmem, uint64_t pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async8_hint(void *smem, const void *gmem, uint64_t pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "l"(pol)
               : "memory");
}
// own tiles: streamed once (read_again: the same tiles are read a second time right after -- the first
// stage of a step, where y is the input -- and keep the default priority)
__device__ __forceinline__ void warp_copy16_stream(void *dst, const void *src, int bytes, int lane,
                                                   bool read_again = false) {
#if HEOM_L2_HINTS
  if (!read_again) {
    const uint64_t pol = l2_evict_first();
    char *d = reinterpret_cast<char *>(dst);
    const char *s = reinterpret_cast<const char *>(src);
    for (int o = lane * 16; o < bytes; o += 32 * 16) cp_async16_hint(d + o, s + o, pol);
    return;
  }
#endif
  warp_copy16(dst, src, bytes, lane);
}
// gathered neighbour rows: kept for the neighbour's other links
__device__ __forceinline__ void cp_async16_keep(void *smem, const void *gmem) {
#if HEOM_L2_HINTS
  cp_async16_hint(smem, gmem, l2_evict_last());
#else
  cp_async16(smem, gmem);
#endif
}
__device__ __forceinline__ void cp_async8_keep(void *smem, const void *gmem) {
#if HEOM_L2_HINTS
  cp_async8_hint(smem, gmem, l2_evict_last());
#else
  cp_async8(smem, gmem);
#endif
}

// Packed FP32x2 FMA (sm_100 family): two independent fma.rn.f32 in one instruction, so the same
// results as two scalar FMAs with half the issue slots.  HEOM_FFMA2=0 (tuning builds) keeps scalar FMAs.
#ifndef HEOM_FFMA2
#define HEOM_FFMA2 1
#endif
constexpr bool kFfma2 = HEOM_FFMA2 != 0;
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Launch shape and buffer sizes (measured on the LHCII-like and FMO-like hierarchies; the macros
// exist for tuning builds).  Link records per warp and batch: RC of 2N-element slices (2 RC row-only
// slices for Hermitian runs).
#ifndef HEOM_STAGE_WARPS
#define HEOM_STAGE_WARPS 4  // warps per CTA, FP32 kernels
#endif
#ifndef HEOM_STAGE_WARPS_FP64
#define HEOM_STAGE_WARPS_FP64 2
#endif
#ifndef HEOM_REC_CAP
#define HEOM_REC_CAP 16  // FP32, N > 10
#endif
#ifndef HEOM_REC_CAP_SMALL
#define HEOM_REC_CAP_SMALL 32  // FP32, N <= 10 (small tiles leave room for more records)
#endif
#ifndef HEOM_REC_CAP_FP64
#define HEOM_REC_CAP_FP64 32
#endif
#ifndef HEOM_Y_SMEM
#define HEOM_Y_SMEM 1
#endif
constexpr bool kYSmem = HEOM_Y_SMEM != 0;  // stage y tiles through shared memory

// RCO != 0 overrides the link records per batch (the tensor-core kernel sizes its own buffers).
template <int N, typename CT, typename BT, int RCO = 0>
struct StageShape {
  static constexpr int E = N * N;
  static constexpr int WARPS = sizeof(CT) == 8 ? HEOM_STAGE_WARPS_FP64 : HEOM_STAGE_WARPS;
  static constexpr int RC = RCO ? RCO : sizeof(CT) == 8 ? HEOM_REC_CAP_FP64 : (N <= 10 ? HEOM_REC_CAP_SMALL : HEOM_REC_CAP);
  static_assert(2 * RC <= 255, "owner table holds record indices in bytes");
  // ADOs per warp; at most 31 so that lanes 0..A hold the A + 1 record offsets of a chunk
  static constexpr int A = (32 / N < 32) ? 32 / N : 31;
  static constexpr bool kOwnHead = sizeof(CT) == 8 && sizeof(BT) == 4;     // mixed-precision head kernel
  static constexpr int EpBody = (sizeof(BT) == 4 && (E & 1)) ? E + 1 : E;  // 16-byte body tiles
  static constexpr int EpOwn = kOwnHead ? E : EpBody;
  static constexpr bool kRowRegs = N <= 16;                                // H row in registers
  static constexpr bool kPairs = sizeof(CT) == 4 && (N % 2) == 0;          // 16-byte tile row loads
  // FP32 kernels add the links to the row in registers, one lane per (ADO, state); for N > 16 (one ADO
  // per warp) this path also keeps H out of lane-dependent loads: S = s H reads H uniformly
  static constexpr bool kOwnerLinks = sizeof(CT) == 4;
  static_assert(!kOwnerLinks || A * N <= 32, "owner lanes index the 32-entry owner table");
};

// Per-warp shared-memory layout (byte offsets).
template <int N, typename CT, typename BT, int RCO = 0>
struct WarpSmem {
  using S = StageShape<N, CT, BT, RCO>;
  static constexpr int c2 = 2 * (int)sizeof(CT);
  static constexpr int tile_bytes = (S::A * S::EpOwn * c2 + 15) & ~15;
  static constexpr int rec_bytes = 2 * S::RC * (int)sizeof(LinkRec<CT>);  // Hermitian runs take 2 RC
  static constexpr int tile0 = 0;
  static constexpr int tile1 = tile0 + tile_bytes;
  static constexpr int ybuf = tile1 + tile_bytes;
  static constexpr int rec0 = ybuf + (kYSmem ? tile_bytes : 0);
  static constexpr int rec1 = rec0 + rec_bytes;
  static constexpr int gbuf = rec1 + rec_bytes;
  static constexpr int tb = gbuf + ((S::RC * 2 * N * c2 + 15) & ~15);  // owner table, 64 bytes
  static constexpr int total = tb + 64;
};

template <int N, typename CT, typename BT>
__device__ __forceinline__ void issue_tiles(const typename Cplx<CT>::type *src_region, int own0, int u0, int cnt,
                                            void *dst, int lane, bool read_again = false) {
  using S = StageShape<N, CT, BT>;
  using C2 = typename Cplx<CT>::type;
  warp_copy16_stream(dst, src_region + (int64_t)(u0 - own0) * S::EpOwn, cnt * S::EpOwn * (int)sizeof(C2), lane,
                     read_again);
}

// Copies W consecutive elements of neighbour v, from element e of its tile, to dst.  Elements of
// the same precision go by cp.async (W * element size = 8 or 16 bytes); elements of the other
// precision region are converted.
template <int N, typename CT, typename BT, int W>
__device__ __forceinline__ void gather_piece(const StageCommon &c, int v, int e, typename Cplx<CT>::type *dst) {
  using S = StageShape<N, CT, BT>;
  using C2 = typename Cplx<CT>::type;
  using B2 = typename Cplx<BT>::type;
  if (v >= c.u_split) {
    const B2 *p = reinterpret_cast<const B2 *>(c.zin.body) + (int64_t)(v - c.u_split) * S::EpBody + e;
    if constexpr (sizeof(B2) == sizeof(C2)) {
      if constexpr (W * sizeof(C2) == 16) cp_async16_keep(dst, p);
      else cp_async8_keep(dst, p);
    } else {  // FP32 body read by the FP64 head kernel
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const B2 bv = p[w];
        C2 x;
        x.x = (CT)bv.x;
        x.y = (CT)bv.y;
        dst[w] = x;
      }
    }
  } else {
    const double2 *p = c.zin.head + (int64_t)v * S::E + e;
    if constexpr (sizeof(C2) == 16) {
      cp_async16_keep(dst, p);
    } else {  // FP64 head read by the FP32 body kernel
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const double2 d = p[w];
        C2 x;
        x.x = (CT)d.x;
        x.y = (CT)d.y;
        dst[w] = x;
      }
    }
  }
}

// Gathers row s -- and, for non-Hermitian runs, column s -- of the neighbours of nrec link records
// into gbuf: slot sl holds v_{s, 0..N-1} at gbuf[sl * pitch] followed (non-Hermitian) by
// v_{0..N-1, s}; pitch N for Hermitian runs (column s is conj(row s)), 2N otherwise.  Rows move in
// 16-byte pieces (two FP32 elements when N is even).  One cp.async group is committed.
template <int N, typename CT, typename BT>
__device__ __forceinline__ void issue_gathers(const StageCommon &c, const LinkRec<CT> *rec, int nrec,
                                              typename Cplx<CT>::type *gbuf, int lane) {
  constexpr int PW = (sizeof(CT) == 4 && N % 2 == 0) ? 2 : 1;  // elements per row piece
  constexpr int P = N / PW;                                     // row pieces
  if (c.herm) {
    for (int t0 = lane; t0 < nrec * P; t0 += 32) {
      const int sl = t0 / P, pc = t0 - sl * P;
      const int s = rec[sl].s & kRecStateMask;
      if (HEOM_IN_RANGE(c.err, rec[sl].v, 0, c.n_ado) && HEOM_IN_RANGE(c.err, s, 0, N))
        gather_piece<N, CT, BT, PW>(c, rec[sl].v, s * N + pc * PW, gbuf + sl * N + pc * PW);
    }
  } else {
    constexpr int per = P + N;
    for (int t0 = lane; t0 < nrec * per; t0 += 32) {
      const int sl = t0 / per, el = t0 - sl * per;
      const int s = rec[sl].s & kRecStateMask;
      if (!HEOM_IN_RANGE(c.err, rec[sl].v, 0, c.n_ado) || !HEOM_IN_RANGE(c.err, s, 0, N)) continue;
      if (el < P) gather_piece<N, CT, BT, PW>(c, rec[sl].v, s * N + el * PW, gbuf + sl * 2 * N + el * PW);
      else gather_piece<N, CT, BT, 1>(c, rec[sl].v, (el - P) * N + s, gbuf + sl * 2 * N + N + (el - P));
    }
  }
  cp_async_commit();
}

// Link contributions by owner lane, for Hermitian runs of the FP32 kernels that keep row li of the
// result in registers.  Every record of the window rec[0 .. nrec) belongs to lane (a, s): a = its
// ADO's place in the chunk starting at u0, s its state.  That lane adds R v_{s, .} to its row
// accumulator (rr, ri); the column part conj(R) v_{., s} follows from Q + Q^dagger at the end.
// The records of one ADO are ordered by state, so a lane's records are
// contiguous; tb (64 bytes of shared memory) carries each lane's [begin, end) from the lanes that
// read the records, 32 records per round.  nrec <= 2 RC <= 255.
template <int N, typename CT>
__device__ __forceinline__ void owner_links(const LinkRec<CT> *rec, int nrec, int u0, int lane, unsigned char *tb,
                                            const typename Cplx<CT>::type *gbuf, CT (&rr)[N], CT (&ri)[N]) {
  using C2 = typename Cplx<CT>::type;
  auto owner_of = [&](int t) -> int {
    if (t >= nrec) return -1;
    const int sw = rec[t].s;
    return (((sw >> 8) - u0) & 31) * N + (sw & kRecStateMask);
  };
  tb[lane] = 0;
  tb[32 + lane] = 0;
  __syncwarp();
  int own = owner_of(lane);
  int before = -1;  // owner of record 32 r - 1
  for (int r = 0; 32 * r < nrec; ++r) {
    const int t = 32 * r + lane;
    const int nxt_round = owner_of(t + 32);
    int prev = __shfl_up_sync(0xffffffffu, own, 1);
    int next = __shfl_down_sync(0xffffffffu, own, 1);
    const int next_first = __shfl_sync(0xffffffffu, nxt_round, 0);
    if (lane == 0) prev = before;
    if (lane == 31) next = next_first;
    if (t < nrec) {
      if (prev != own) tb[own] = (unsigned char)t;
      if (next != own) tb[32 + own] = (unsigned char)(t + 1);
    }
    before = __shfl_sync(0xffffffffu, own, 31);
    own = nxt_round;
  }
  __syncwarp();
  const int pb = tb[lane], pe = tb[32 + lane];
  for (int p = pb; p < pe; ++p) {
    const CT re = rec[p].re, im = rec[p].im;
    const C2 *g = gbuf + p * N;
    if constexpr (sizeof(CT) == 4 && N % 2 == 0) {
      const float4 *g4 = reinterpret_cast<const float4 *>(g);
#pragma unroll
      for (int jp = 0; jp < N / 2; ++jp) {
        const float4 v = g4[jp];
        rr[2 * jp] = fma(re, v.x, fma(-im, v.y, rr[2 * jp]));
        ri[2 * jp] = fma(re, v.y, fma(im, v.x, ri[2 * jp]));
        rr[2 * jp + 1] = fma(re, v.z, fma(-im, v.w, rr[2 * jp + 1]));
        ri[2 * jp + 1] = fma(re, v.w, fma(im, v.z, ri[2 * jp + 1]));
      }
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const C2 v = g[j];
        rr[j] = fma(re, v.x, fma(-im, v.y, rr[j]));
        ri[j] = fma(re, v.y, fma(im, v.x, ri[j]));
      }
    }
  }
}

// Adds the contributions of the records [blo, blo + nrec) (record i at rec[i - blo]) to the output
// tile ot of this lane's ADO, which owns records [my_lo, my_hi).  For the k-th record of its ADO,
// lane (la, li) updates element (s, li) and (li, s) -- or (s, s) when li = s -- which are disjoint
// within one k; the warp synchronises between k.
template <int N, typename CT, typename BT>
__device__ __forceinline__ void apply_links(const LinkRec<CT> *rec, int64_t blo, int nrec, int64_t my_lo,
                                            int64_t my_hi, bool active, int li, bool herm,
                                            typename Cplx<CT>::type *ot, const typename Cplx<CT>::type *gbuf) {
  using C2 = typename Cplx<CT>::type;
  const int64_t a_lo = max(my_lo, blo), a_hi = min(my_hi, blo + nrec);
  const int my_cnt = active ? (int)max((int64_t)0, a_hi - a_lo) : 0;
  const int maxc = (int)__reduce_max_sync(0xffffffffu, (unsigned)my_cnt);
  for (int k = 0; k < maxc; ++k) {
    if (k < my_cnt) {
      const int sl = (int)(a_lo - blo) + k;
      const LinkRec<CT> r = rec[sl];
      const int s = r.s & kRecStateMask;
      const C2 *gv = gbuf + sl * (herm ? N : 2 * N);
      if (li == s) {
        const C2 v = gv[s];
        C2 o = ot[s * N + s];
        o.x = fma(2 * r.re, v.x, o.x);
        o.y = fma(2 * r.re, v.y, o.y);
        ot[s * N + s] = o;
      } else {
        const C2 vr = gv[li];  // element (s, li) of the neighbour: coefficient R
        C2 vc;                 // element (li, s): coefficient conj(R)
        if (herm) {
          vc.x = vr.x;
          vc.y = -vr.y;
        } else {
          vc = gv[N + li];
        }
        C2 o1 = ot[s * N + li];
        o1.x = fma(r.re, vr.x, fma(-r.im, vr.y, o1.x));
        o1.y = fma(r.re, vr.y, fma(r.im, vr.x, o1.y));
        ot[s * N + li] = o1;
        C2 o2 = ot[li * N + s];
        o2.x = fma(r.re, vc.x, fma(r.im, vc.y, o2.x));
        o2.y = fma(r.re, vc.y, fma(-r.im, vc.x, o2.y));
        ot[li * N + s] = o2;
      }
    }
    __syncwarp();
  }
}

// Owner-path link application for a Hermitian run: the first link batch (records in rec, gathers
// landed), then further batches of at most cap records.  (rr, ri) hold row li of Q.
template <int N, typename CT, typename BT>
__device__ __forceinline__ void owner_apply(const StageCommon &c, const LinkRec<CT> *recs, int64_t rbase,
                                            LinkRec<CT> *rec, typename Cplx<CT>::type *gbuf, unsigned char *tb,
                                            int64_t lo, int64_t hi, int nrec, int cap, int u0, int lane,
                                            CT (&rr)[N], CT (&ri)[N]) {
  using R = LinkRec<CT>;
  owner_links<N, CT>(rec, nrec, u0, lane, tb, gbuf, rr, ri);
  const int64_t rlim = StageShape<N, CT, BT>::kOwnHead ? c.rec_split : c.n_recs;
  for (int64_t blo = lo + nrec; blo < hi; blo += cap) {  // further link batches
    __syncwarp();
    const int nr = heom_rec_batch(c.err, blo, (int)min(hi - blo, (int64_t)cap), rbase, rlim);
    warp_copy16(rec, recs + (blo - rbase), nr * (int)sizeof(R), lane);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    issue_gathers<N, CT, BT>(c, rec, nr, gbuf, lane);
    cp_async_wait<0>();
    __syncwarp();
    owner_links<N, CT>(rec, nr, u0, lane, tb, gbuf, rr, ri);
  }
}

// result_ij = Q_ij + conj(Q_ji) through the output tile zt_all (every lane must be done reading it);
// (rr, ri) hold row li of Q on entry, the result row is left in zt_all.
template <int N, typename CT, typename BT>
__device__ __forceinline__ void owner_combine(bool active, int la, int li, typename Cplx<CT>::type *zt_all,
                                              CT (&rr)[N], CT (&ri)[N]) {
  using C2 = typename Cplx<CT>::type;
  constexpr int EPO = StageShape<N, CT, BT>::EpOwn;
  if (active) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      C2 w;
      w.x = rr[j];
      w.y = ri[j];
      zt_all[la * EPO + li * N + j] = w;
    }
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const C2 t = zt_all[la * EPO + j * N + li];
      rr[j] += t.x;
      ri[j] -= t.y;
    }
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      C2 w;
      w.x = rr[j];
      w.y = ri[j];
      zt_all[la * EPO + li * N + j] = w;
    }
  }
}

// out = y + ch * rhs (or ch * rhs) over the chunk's contiguous tiles [u0, u0 + cnt), 16 bytes per
// access; rhs in the tile buffer ot, y in ybuf (or read from y_own when y is not staged).
template <int N, typename CT, typename BT>
__device__ __forceinline__ void store_chunk(typename Cplx<CT>::type *out_own, const typename Cplx<CT>::type *y_own,
                                            int own0, int u0, int cnt, bool has_y, CT ch,
                                            const typename Cplx<CT>::type *ot, const typename Cplx<CT>::type *ybuf,
                                            int lane) {
  using C2 = typename Cplx<CT>::type;
  constexpr int EPO = StageShape<N, CT, BT>::EpOwn;
  C2 *dst = out_own + (int64_t)(u0 - own0) * EPO;
  if constexpr (sizeof(CT) == 4) {
    const float4 *o4 = reinterpret_cast<const float4 *>(ot);
    const float4 *y4 = kYSmem ? reinterpret_cast<const float4 *>(ybuf)
                              : reinterpret_cast<const float4 *>(y_own + (int64_t)(u0 - own0) * EPO);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    const float chv = (float)ch;
    for (int t = lane; t < cnt * EPO / 2; t += 32) {
      float4 w = o4[t];
      if (has_y) {
        const float4 yv = y4[t];
        w.x = fmaf(chv, w.x, yv.x);
        w.y = fmaf(chv, w.y, yv.y);
        w.z = fmaf(chv, w.z, yv.z);
        w.w = fmaf(chv, w.w, yv.w);
      } else {
        w.x *= chv;
        w.y *= chv;
        w.z *= chv;
        w.w *= chv;
      }
      d4[t] = w;
    }
  } else {
    for (int t = lane; t < cnt * EPO; t += 32) {
      C2 w = ot[t];
      if (has_y) {
        const C2 yv = kYSmem ? ybuf[t] : y_own[(int64_t)(u0 - own0) * EPO + t];
        w.x = fma(ch, w.x, yv.x);
        w.y = fma(ch, w.y, yv.y);
      } else {
        w.x *= ch;
        w.y *= ch;
      }
      dst[t] = w;
    }
  }
}

// The chunks first, first + nwarps, ... below n_chunks of one stage (chunk k = ADOs u_begin + k A ..),
// processed by the calling warp with the per-warp buffers at smem_raw + warp * WarpSmem::total.  Args is
// StageArgs<CT> (the kernel parameters of one launch) or GroupArgs<CT> (one run of a work-list launch,
// staged in shared memory): H, the terminator, the Horner coefficient and the StageCommon of the stage.
template <int N, typename CT, typename BT, bool CPLX, typename Args>
__device__ __forceinline__ void stage_chunks(const Args &a, unsigned char *smem_raw, int first, int nwarps,
                                             int n_chunks) {
  using S = StageShape<N, CT, BT>;
  using W = WarpSmem<N, CT, BT>;
  using C2 = typename Cplx<CT>::type;
  using R = LinkRec<CT>;
  constexpr int EPO = S::EpOwn;
  constexpr int A = S::A;
  constexpr bool kOwn = S::kOwnerLinks && !CPLX;  // complex H keeps the shared-memory link path
  const StageCommon &c = a.c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *wb = smem_raw + warp * W::total;
  C2 *ybuf = reinterpret_cast<C2 *>(wb + W::ybuf);
  C2 *gbuf = reinterpret_cast<C2 *>(wb + W::gbuf);

  const int la = lane / N;
  const int li = lane - la * N;
  const bool lane_ok = la < A;
  const bool has_y = (c.y.head != nullptr) || (c.y.body != nullptr);
  // y is the input (first stage of a step): the input tiles are read again as y right after
  const bool same_y = c.y.head == c.zin.head && c.y.body == c.zin.body;
  const CT term_i = lane_ok ? a.term[li] : (CT)0;
  // terminator Delta_i + Delta_j of row li (0 on the diagonal), precomputed in FP64 where every FP64
  // add costs pipe time; FP32 recomputes it (the registers are worth more there)
  constexpr bool kTsum = sizeof(CT) == 8;
  CT tsum[kTsum ? N : 1];
  if constexpr (kTsum) {
#pragma unroll
    for (int j = 0; j < N; ++j) tsum[j] = (lane_ok && j != li) ? term_i + a.term[j] : (CT)0;
  }
  CT Hrow[S::kRowRegs ? N : 1];
  if constexpr (S::kRowRegs) {
#pragma unroll
    for (int k = 0; k < N; ++k) Hrow[k] = lane_ok ? a.H[li * kMaxStates + k] : (CT)0;
  }
  const C2 *zin_own = S::kOwnHead ? reinterpret_cast<const C2 *>(c.zin.head) : reinterpret_cast<const C2 *>(c.zin.body);
  C2 *out_own = S::kOwnHead ? reinterpret_cast<C2 *>(c.out.head) : reinterpret_cast<C2 *>(c.out.body);
  const C2 *y_own = S::kOwnHead ? reinterpret_cast<const C2 *>(c.y.head) : reinterpret_cast<const C2 *>(c.y.body);
  const R *recs = reinterpret_cast<const R *>(S::kOwnHead ? c.recs_head : c.recs_body);
  const int64_t rbase = S::kOwnHead ? 0 : c.rec_split;
  const int64_t rlim = S::kOwnHead ? c.rec_split : c.n_recs;  // records [rbase, rlim) of this region
  const int own0 = S::kOwnHead ? 0 : c.u_split;

  const int cap = c.herm ? 2 * S::RC : S::RC;  // link records per batch (slice buffer: 2 N RC elements)
  // lane a <= cnt of a chunk holds link_off[u0 + a]
  auto load_offs = [&](int chn) -> int64_t {
    if (chn >= n_chunks) return 0;
    const int u0 = c.u_begin + chn * A;
    const int cnt = min(A, c.u_end - u0);
    return (lane <= cnt) ? c.link_off[u0 + lane] : (int64_t)0;
  };
  int64_t off_cur = load_offs(first);
  int64_t off_nxt = load_offs(first + nwarps);
  if (first < n_chunks) {
    const int u0 = c.u_begin + first * A;
    const int cnt = min(A, c.u_end - u0);
    issue_tiles<N, CT, BT>(zin_own, own0, u0, cnt, wb + W::tile0, lane, same_y);
    const int64_t lo = __shfl_sync(0xffffffffu, off_cur, 0), hi = __shfl_sync(0xffffffffu, off_cur, cnt);
    const int nr = heom_rec_batch(c.err, lo, (int)min(hi - lo, (int64_t)cap), rbase, rlim);
    warp_copy16(wb + W::rec0, recs + (lo - rbase), nr * (int)sizeof(R), lane);
    cp_async_commit();
  }
  int b = 0;
  for (int chn = first; chn < n_chunks; chn += nwarps, b ^= 1) {
    const int u0 = c.u_begin + chn * A;
    const int cnt = min(A, c.u_end - u0);
    const int nx = chn + nwarps;
    const int64_t off_nx2 = load_offs(nx + nwarps);  // consumed two iterations later
    C2 *zt_all = reinterpret_cast<C2 *>(wb + (b ? W::tile1 : W::tile0));
    R *rec = reinterpret_cast<R *>(wb + (b ? W::rec1 : W::rec0));
    // next chunk's tiles and records -> the other buffers
    if (nx < n_chunks) {
      const int v0 = c.u_begin + nx * A;
      const int vcnt = min(A, c.u_end - v0);
      issue_tiles<N, CT, BT>(zin_own, own0, v0, vcnt, wb + (b ? W::tile0 : W::tile1), lane, same_y);
      const int64_t lo = __shfl_sync(0xffffffffu, off_nxt, 0), hi = __shfl_sync(0xffffffffu, off_nxt, vcnt);
      const int nr = heom_rec_batch(c.err, lo, (int)min(hi - lo, (int64_t)cap), rbase, rlim);
      warp_copy16(wb + (b ? W::rec0 : W::rec1), recs + (lo - rbase), nr * (int)sizeof(R), lane);
    }
    cp_async_commit();
    if (kYSmem && has_y) issue_tiles<N, CT, BT>(y_own, own0, u0, cnt, ybuf, lane);
    cp_async_commit();
    cp_async_wait<2>();  // this chunk's tiles and first records have landed
    __syncwarp();

    const int64_t lo = __shfl_sync(0xffffffffu, off_cur, 0), hi = __shfl_sync(0xffffffffu, off_cur, cnt);
    const bool active = lane_ok && la < cnt;
    const int64_t my_lo = __shfl_sync(0xffffffffu, off_cur, min(la, A));
    const int64_t my_hi = __shfl_sync(0xffffffffu, off_cur, min(la + 1, A));
    const int nrec = (int)min(hi - lo, (int64_t)cap);
    issue_gathers<N, CT, BT>(c, rec, nrec, gbuf, lane);

    const bool herm = c.herm != 0;
    // owner-lane links for Hermitian runs; non-Hermitian runs need row and column work per link,
    // which the shared-memory form spreads over the lanes
    const bool own_path = kOwn && herm;
    CT rr[N], ri[N];  // row li of the result: real and imaginary parts
    {  // commutator -i (H s - s H), decay and terminator of row li
      const C2 *zt = zt_all + la * EPO;
      C2 zr[N];         // own row s_{li, .}
      if (active) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          rr[j] = 0;
          ri[j] = 0;
          zr[j] = zt[li * N + j];
        }
        if (!own_path) {
          // -i (H s)
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const CT h = S::kRowRegs ? Hrow[S::kRowRegs ? k : 0] : a.H[li * kMaxStates + k];
            if constexpr (S::kPairs) {
              const float4 *zp = reinterpret_cast<const float4 *>(zt + k * N);
#pragma unroll
              for (int jp = 0; jp < N / 2; ++jp) {
                const float4 z = zp[jp];
                rr[2 * jp] = fma(h, z.y, rr[2 * jp]);
                ri[2 * jp] = fma(-h, z.x, ri[2 * jp]);
                rr[2 * jp + 1] = fma(h, z.w, rr[2 * jp + 1]);
                ri[2 * jp + 1] = fma(-h, z.z, ri[2 * jp + 1]);
              }
            } else {
#pragma unroll
              for (int j = 0; j < N; ++j) {
                const C2 z = zt[k * N + j];
                rr[j] = fma(h, z.y, rr[j]);
                ri[j] = fma(-h, z.x, ri[j]);
              }
            }
          }
          if constexpr (CPLX) {  // imaginary part of H in -i (H s)
#pragma unroll
            for (int k = 0; k < N; ++k) {
              const CT h = a.Hi[li * kMaxStates + k];
#pragma unroll
              for (int j = 0; j < N; ++j) {
                const C2 z = zt[k * N + j];
                rr[j] = fma(h, z.x, rr[j]);
                ri[j] = fma(h, z.y, ri[j]);
              }
            }
          }
        }
        if (!herm || own_path) {  // + i (s H); on the owner path Q = i S with S = s H from the own row
          if constexpr (kFfma2 && sizeof(CT) == 4 && N % 2 == 0) {
            // the same FMAs, two columns per packed FP32x2 instruction (bit-identical results)
            uint64_t pr[N / 2], pi[N / 2];
#pragma unroll
            for (int jp = 0; jp < N / 2; ++jp) {
              pr[jp] = pack2(rr[2 * jp], rr[2 * jp + 1]);
              pi[jp] = pack2(ri[2 * jp], ri[2 * jp + 1]);
            }
#pragma unroll
            for (int k = 0; k < N; ++k) {
              const C2 zk = zr[k];
              const uint64_t sy = pack2(-zk.y, -zk.y), sx = pack2(zk.x, zk.x);
#pragma unroll
              for (int jp = 0; jp < N / 2; ++jp) {
                const uint64_t hp = *reinterpret_cast<const uint64_t *>(&a.H[k * kMaxStates + 2 * jp]);
                pr[jp] = ffma2(sy, hp, pr[jp]);
                pi[jp] = ffma2(sx, hp, pi[jp]);
              }
            }
#pragma unroll
            for (int jp = 0; jp < N / 2; ++jp) {
              unpack2(pr[jp], rr[2 * jp], rr[2 * jp + 1]);
              unpack2(pi[jp], ri[2 * jp], ri[2 * jp + 1]);
            }
          } else {
#pragma unroll
            for (int k = 0; k < N; ++k) {
              const C2 zk = zr[k];
#pragma unroll
              for (int j = 0; j < N; ++j) {
                const CT h = a.H[k * kMaxStates + j];
                rr[j] = fma(-zk.y, h, rr[j]);
                ri[j] = fma(zk.x, h, ri[j]);
              }
            }
          }
          if constexpr (CPLX) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
              const C2 zk = zr[k];
#pragma unroll
              for (int j = 0; j < N; ++j) {
                const CT h2 = a.Hi[k * kMaxStates + j];
                rr[j] = fma(-zk.x, h2, rr[j]);
                ri[j] = fma(-zk.y, h2, ri[j]);
              }
            }
          }
        }
      }
      if (herm && !own_path) {
        // s and H Hermitian: s H = (H s)^dagger, so -i (H s - s H)_ij = -i (P_ij - conj(P_ji)) with
        // P = H s; in the (rr, ri) = -i P form that is (rr_ij + rr_ji, ri_ij - ri_ji).
        __syncwarp();  // every lane is done reading the tile
        if (active) {
#pragma unroll
          for (int j = 0; j < N; ++j) {
            C2 w;
            w.x = rr[j];
            w.y = ri[j];
            zt_all[la * EPO + li * N + j] = w;
          }
        }
        __syncwarp();
        if (active) {
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const C2 t = zt_all[la * EPO + j * N + li];
            rr[j] += t.x;
            ri[j] -= t.y;
          }
        }
      }
      if (active) {  // decay and terminator
        const CT gsv = (CT)c.gsum[u0 + la];
        // the owner path adds Q + Q^dagger at the end: half the rate here
        const CT hf = own_path ? (CT)0.5 : (CT)1;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          CT f;
          if constexpr (kTsum) f = gsv + tsum[kTsum ? j : 0];
          else f = gsv + ((j != li) ? (term_i + a.term[j]) : (CT)0);
          if constexpr (kOwn) f *= hf;
          rr[j] = fma(-f, zr[j].x, rr[j]);
          ri[j] = fma(-f, zr[j].y, ri[j]);
        }
      }
      if (!own_path) {
        __syncwarp();  // every lane is done reading the tile: it becomes the output buffer
        if (active) {
#pragma unroll
          for (int j = 0; j < N; ++j) {
            C2 w;
            w.x = rr[j];
            w.y = ri[j];
            zt_all[la * EPO + li * N + j] = w;
          }
        }
      }
    }
    cp_async_wait<0>();  // gathers, y and the next chunk's copies have landed
    __syncwarp();
    if (own_path) {
      // Row li of Q in (rr, ri): -i H s, half the decay, and R v_{li, .} of the records of state li
      owner_apply<N, CT, BT>(c, recs, rbase, rec, gbuf, wb + W::tb, lo, hi, nrec, cap, u0, lane, rr, ri);
      owner_combine<N, CT, BT>(active, la, li, zt_all, rr, ri);
    } else {
      C2 *ot = zt_all + la * EPO;
      apply_links<N, CT, BT>(rec, lo, nrec, my_lo, my_hi, active, li, herm, ot, gbuf);
      for (int64_t blo = lo + nrec; blo < hi; blo += cap) {  // further link batches
        __syncwarp();
        const int nr = heom_rec_batch(c.err, blo, (int)min(hi - blo, (int64_t)cap), rbase, rlim);
        warp_copy16(rec, recs + (blo - rbase), nr * (int)sizeof(R), lane);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        issue_gathers<N, CT, BT>(c, rec, nr, gbuf, lane);
        cp_async_wait<0>();
        __syncwarp();
        apply_links<N, CT, BT>(rec, blo, nr, my_lo, my_hi, active, li, herm, ot, gbuf);
      }
    }
    __syncwarp();
    store_chunk<N, CT, BT>(out_own, y_own, own0, u0, cnt, has_y, a.ch, zt_all, ybuf, lane);
    __syncwarp();  // this tile buffer, record buffer and ybuf are reused by later chunks
    off_cur = off_nxt;
    off_nxt = off_nx2;
  }
  cp_async_wait<0>();
}

template <int N, typename CT, typename BT, bool CPLX>
__global__ void __launch_bounds__(StageShape<N, CT, BT>::WARPS * 32) stage_kernel(const __grid_constant__ StageArgs<CT> a) {
  using S = StageShape<N, CT, BT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n_chunks = (a.c.u_end - a.c.u_begin + S::A - 1) / S::A;
  stage_chunks<N, CT, BT, CPLX>(a, smem_raw, blockIdx.x * S::WARPS + (int)(threadIdx.x >> 5), gridDim.x * S::WARPS,
                                n_chunks);
}

template <int N, typename CT, typename BT, bool CPLX>
int launch_v(const StageArgs<CT> &a, cudaStream_t st, int sm_count) {
  const StageCommon &c = a.c;
  constexpr int WARPS = StageShape<N, CT, BT>::WARPS;
  const size_t smem = (size_t)WARPS * WarpSmem<N, CT, BT>::total;
  static int per_sm = 0;  // occupancy of this instantiation (its shared memory size is fixed)
  if (per_sm == 0) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(stage_kernel<N, CT, BT, CPLX>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) {
        set_error(std::string("stage kernel: shared memory attribute: ") + cudaGetErrorString(e));
        return -4;
      }
    }
    int ps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, stage_kernel<N, CT, BT, CPLX>,
                                                                  WARPS * 32, smem);
    if (e != cudaSuccess || ps < 1) {
      set_error(std::string("stage kernel: occupancy query failed or zero blocks: ") + cudaGetErrorString(e));
      return -4;
    }
    per_sm = ps;
  }
  constexpr int A = StageShape<N, CT, BT>::A;
  const int n_chunks = (c.u_end - c.u_begin + A - 1) / A;
  const int blocks_needed = (n_chunks + WARPS - 1) / WARPS;
  const int grid = std::max(1, std::min(blocks_needed, sched_ctas(per_sm, c.occ_pct) * sm_count));
  stage_kernel<N, CT, BT, CPLX><<<grid, WARPS * 32, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("stage kernel launch: ") + cudaGetErrorString(e));
    return -4;
  }
  return 0;
}

template <int N, typename CT, typename BT>
int launch_n(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi,
             cudaStream_t st, int sm_count) {
  StageArgs<CT> a;
  a.c = c;
  a.ch = (CT)ch;
  for (int i = 0; i < kMaxStates; ++i) a.term[i] = (i < c.n) ? (CT)term[i] : (CT)0;
  for (int i = 0; i < kMaxStates * kMaxStates; ++i) {
    a.H[i] = 0;
    a.Hi[i] = 0;
  }
  for (int i = 0; i < c.n; ++i)
    for (int j = 0; j < c.n; ++j) {
      a.H[i * kMaxStates + j] = (CT)H[i * c.n + j];
      a.Hi[i * kMaxStates + j] = Hi ? (CT)Hi[i * c.n + j] : (CT)0;
    }
  return c.cplx_h ? launch_v<N, CT, BT, true>(a, st, sm_count) : launch_v<N, CT, BT, false>(a, st, sm_count);
}

}  // namespace heom
