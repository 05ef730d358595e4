// Fused HEOM right-hand side + RK4 (Horner form) stage kernel for sm_103a.
//
// One launch evaluates, for every ADO u in [u_begin, u_end),
//     out_u = y_u + ch * (L zin)_u          (or ch * (L zin)_u when there is no y)
// where L is the right-hand side of Eq. HEOM (arXiv 1803.03498, section "HEOM formalism") with the
// ADO rescaling, written element-wise (hbar = 1, energies in rad/fs):
//   (L s)_ij = -i sum_k (H_ik s_kj - s_ik H_kj) - (sum_l n_l gamma_l) s_ij
//              - [i != j] (Delta_i + Delta_j) s_ij
//              + sum_{l: s_l = i} i s+_l s^{+l}_ij [j != i]  - sum_{l: s_l = j} i s+_l s^{+l}_ij [i != j]
//              + sum_{l: s_l = i} s-_l (i c_l + lamnu_l) s^{-l}_ij + sum_{l: s_l = j} s-_l (-i c_l + lamnu_l) s^{-l}_ij
// i.e. V^x = (delta_is - delta_sj), V^x V^x = (1 - delta_ij)(delta_is + delta_sj) and
// V^o = (delta_is + delta_sj) applied element by element.  A link through a mode of state s touches
// only row s and column s: its row part gets coefficient R, its column part C, element (s, s) gets Dg:
//   up   (factor s+):            R = +i s+,             C = -i s+,             Dg = 0
//   down (factor s-, c, lamnu):  R = s- (lamnu + i c),  C = s- (lamnu - i c),  Dg = 2 s- lamnu.
//
// Every warp works on its own chunks of A = floor(32 / N) consecutive ADOs, independently of the
// other warps (only __syncwarp), and pipelines them:
//  - 16-byte cp.async copies bring the next chunk's tiles (each ADO's N x N tile is contiguous) and
//    link-table rows into a second buffer while the current chunk is computed, and the current
//    chunk's y tiles into shared memory;
//  - a ballot scan numbers the valid links (ADO, mode, up/down) and records each link's neighbour,
//    state and coefficients; cp.async then gathers row s and column s of every linked neighbour;
//  - while the gathers are in flight, lane (a, i) computes row i of ADO a: the commutator (the lanes
//    of one ADO read the same tile word, a broadcast; H sits in the kernel parameters, addressed by
//    the unrolled loops with compile-time offsets), decay and terminator;
//  - every lane adds the link contributions to elements (s, i) and (i, s) of its ADO's output, and
//    y + ch * output leaves with coalesced stores.
// A chunk with more links than slice slots handles the remainder in further synchronous batches.
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

constexpr int kWarpSlots = 24;  // staged neighbour slices per warp and batch

template <int N, typename CT, typename BT>
struct StageShape {
  using C2 = typename Cplx<CT>::type;
  static constexpr int E = N * N;
  static constexpr int A = 32 / N;                          // ADOs per warp
  static constexpr bool kOwnHead = sizeof(CT) == 8 && sizeof(BT) == 4;  // mixed-precision head kernel
  static constexpr int EpBody = (sizeof(BT) == 4 && (E & 1)) ? E + 1 : E;  // 16-byte body tiles
  static constexpr int EpOwn = kOwnHead ? E : EpBody;
  static constexpr int kRowRegs = N <= 16;                  // H row in registers
  static constexpr int JB = N <= 16 ? N : 8;                // output columns per register block
};

// Per-warp shared-memory layout (byte offsets); Mp (padded mode count) is a run-time value.
template <int N, typename CT, typename BT>
struct WarpSmem {
  using S = StageShape<N, CT, BT>;
  int tile0, tile1, ybuf, tp0, tp1, tm0, tm1, tt0, tt1, sv, sst, sco, gbuf, total;
  __host__ __device__ WarpSmem(int Mp) {
    constexpr int c2 = 2 * (int)sizeof(CT);
    auto al = [](int x) { return (x + 15) & ~15; };
    int o = 0;
    tile0 = o; o = al(o + S::A * S::EpOwn * c2);
    tile1 = o; o = al(o + S::A * S::EpOwn * c2);
    ybuf = o; o = al(o + S::A * S::EpOwn * c2);
    tp0 = o; o = al(o + S::A * Mp * 4);
    tp1 = o; o = al(o + S::A * Mp * 4);
    tm0 = o; o = al(o + S::A * Mp * 4);
    tm1 = o; o = al(o + S::A * Mp * 4);
    tt0 = o; o = al(o + S::A * Mp);
    tt1 = o; o = al(o + S::A * Mp);
    sv = o; o = al(o + kWarpSlots * 4);        // neighbour ADO of each slot
    sst = o; o = al(o + kWarpSlots * 4);       // (ADO in chunk) << 8 | state
    sco = o; o = al(o + kWarpSlots * 3 * c2);  // R, C, Dg coefficients
    gbuf = o; o = al(o + kWarpSlots * 2 * N * c2);
    total = o;
  }
};

template <typename CT>
__host__ __device__ inline int stage_const_bytes(int M, int D) {
  return ((2 * M * (D + 1) + 2 * M) * (int)sizeof(CT) + M * 4 + 15) & ~15;
}

// Numbers up to kWarpSlots valid links (entry e = (a * M + q) * 2 + dir) from entry e_pos on, records
// each link's neighbour, state and coefficients, and issues the gathers of row s and column s of
// the linked neighbours ([slot][0..N) row, [slot][N..2N) column) as one cp.async group (elements
// that need a precision conversion are loaded directly).  Returns the number of links; advances
// e_pos.
template <int N, typename CT, typename BT>
__device__ __forceinline__ int plan_and_gather(const StageCommon &c, int lane, int tot, int &e_pos, const int *tp,
                                               const int *tm, const unsigned char *tt, const CT *sp_s,
                                               const CT *sm_s, const CT *cc_s, const CT *ln_s, const int *st_s,
                                               int *sv, int *sst, typename Cplx<CT>::type *sco,
                                               typename Cplx<CT>::type *gbuf) {
  using S = StageShape<N, CT, BT>;
  using C2 = typename Cplx<CT>::type;
  using B2 = typename Cplx<BT>::type;
  const int M = c.M, Mp = c.Mp, D1 = c.D + 1;
  int nb = 0, e_scan = e_pos;
  while (e_scan < tot && nb < kWarpSlots) {
    const int e = e_scan + lane;
    int v = -1, q = 0, aa = 0, dir = 0;
    if (e < tot) {
      aa = e / (2 * M);
      const int r = e - aa * 2 * M;
      q = r >> 1;
      dir = r & 1;
      v = dir ? tm[aa * Mp + q] : tp[aa * Mp + q];
    }
    const unsigned mask = __ballot_sync(0xffffffffu, v >= 0);
    const int room = kWarpSlots - nb;
    int take_upto = 32;  // entries at lanes >= take_upto wait for the next batch
    if (__popc(mask) > room) {
      unsigned m = mask;
      for (int k = 0; k < room; ++k) m &= m - 1;
      take_upto = __ffs(m) - 1;
    }
    if (v >= 0 && lane < take_upto) {
      const int sidx = nb + __popc(mask & ((1u << lane) - 1u));
      const int nl = tt[aa * Mp + q];
      sv[sidx] = v;
      sst[sidx] = (aa << 8) | st_s[q];
      C2 R, Cc, Dg;
      if (dir == 0) {
        const CT f = sp_s[q * D1 + nl];
        R.x = 0; R.y = f;
        Cc.x = 0; Cc.y = -f;
        Dg.x = 0; Dg.y = 0;
      } else {
        const CT f = sm_s[q * D1 + nl];
        const CT fc = f * cc_s[q], fl = f * ln_s[q];
        R.x = fl; R.y = fc;
        Cc.x = fl; Cc.y = -fc;
        Dg.x = 2 * fl; Dg.y = 0;
      }
      sco[3 * sidx] = R;
      sco[3 * sidx + 1] = Cc;
      sco[3 * sidx + 2] = Dg;
    }
    nb += __popc(take_upto >= 32 ? mask : (mask & ((1u << take_upto) - 1u)));
    e_scan += take_upto;
  }
  e_pos = e_scan;
  __syncwarp();
  const B2 *zb = reinterpret_cast<const B2 *>(c.zin.body);
  for (int t = lane; t < nb * 2 * N; t += 32) {
    const int sl = t / (2 * N), el = t - sl * 2 * N;
    const int st = sst[sl] & 255;
    const int e = (el < N) ? (st * N + el) : ((el - N) * N + st);
    const int v = sv[sl];
    if (v >= c.u_split) {
      const B2 *p = zb + (int64_t)(v - c.u_split) * S::EpBody + e;
      if (sizeof(B2) == sizeof(C2)) {
        if (sizeof(C2) == 16) cp_async16(gbuf + t, p);
        else cp_async8(gbuf + t, p);
      } else {  // FP32 body read by the FP64 head kernel
        const B2 bv = *p;
        C2 w;
        w.x = (CT)bv.x;
        w.y = (CT)bv.y;
        gbuf[t] = w;
      }
    } else {  // FP64 head
      const double2 d = c.zin.head[(int64_t)v * S::E + e];
      C2 w;
      w.x = (CT)d.x;
      w.y = (CT)d.y;
      gbuf[t] = w;
    }
  }
  cp_async_commit();
  return nb;
}

// Adds the contributions of nb staged links to the output tiles ot_all (pitch EpOwn).  For the k-th
// link of its ADO, lane (la, li) updates elements (s, li) and (li, s), or (s, s) when li = s: these
// are disjoint within one k, and the warp synchronises between k.  Links of one ADO occupy
// consecutive slots.
template <int N, typename CT, typename BT>
__device__ __forceinline__ void apply_links(int nb, int cnt, int lane, int la, int li, bool active,
                                            typename Cplx<CT>::type *ot_all, const int *sst,
                                            const typename Cplx<CT>::type *sco,
                                            const typename Cplx<CT>::type *gbuf) {
  using S = StageShape<N, CT, BT>;
  using C2 = typename Cplx<CT>::type;
  int my_first = 0, my_cnt = 0, maxc = 0;
  const int owner = (lane < nb) ? (sst[lane] >> 8) : -1;
  for (int aa = 0; aa < cnt; ++aa) {
    const unsigned m = __ballot_sync(0xffffffffu, owner == aa);
    const int k = __popc(m);
    if (aa == la) {
      my_cnt = k;
      my_first = k ? __ffs(m) - 1 : 0;
    }
    maxc = max(maxc, k);
  }
  C2 *ot = ot_all + la * S::EpOwn;
  for (int k = 0; k < maxc; ++k) {
    if (active && k < my_cnt) {
      const int sl = my_first + k;
      const int st = sst[sl] & 255;
      const C2 *gv = gbuf + sl * 2 * N;
      if (li == st) {
        const C2 Dg = sco[3 * sl + 2];
        const C2 v = gv[st];
        C2 o = ot[st * N + st];
        o.x = fma(Dg.x, v.x, fma(-Dg.y, v.y, o.x));
        o.y = fma(Dg.x, v.y, fma(Dg.y, v.x, o.y));
        ot[st * N + st] = o;
      } else {
        const C2 R = sco[3 * sl], Cc = sco[3 * sl + 1];
        const C2 vr = gv[li];      // element (s, li) of the neighbour
        const C2 vc = gv[N + li];  // element (li, s)
        C2 o1 = ot[st * N + li];
        o1.x = fma(R.x, vr.x, fma(-R.y, vr.y, o1.x));
        o1.y = fma(R.x, vr.y, fma(R.y, vr.x, o1.y));
        ot[st * N + li] = o1;
        C2 o2 = ot[li * N + st];
        o2.x = fma(Cc.x, vc.x, fma(-Cc.y, vc.y, o2.x));
        o2.y = fma(Cc.x, vc.y, fma(Cc.y, vc.x, o2.y));
        ot[li * N + st] = o2;
      }
    }
    __syncwarp();
  }
}

// Copies of one chunk's tiles and table rows into one buffer (one cp.async group).
template <int N, typename CT, typename BT>
__device__ __forceinline__ void issue_chunk(const StageCommon &c, int lane, int u0, int cnt,
                                            const typename Cplx<CT>::type *zin_own, int own0, char *tile,
                                            char *tpb, char *tmb, char *ttb) {
  using S = StageShape<N, CT, BT>;
  using C2 = typename Cplx<CT>::type;
  const int Mp = c.Mp;
  const char *src = reinterpret_cast<const char *>(zin_own + (int64_t)(u0 - own0) * S::EpOwn);
  const int bytes = cnt * S::EpOwn * (int)sizeof(C2);
  for (int o = lane * 16; o < bytes; o += 32 * 16) cp_async16(tile + o, src + o);
  const int tb = cnt * Mp * 4;
  const char *ps = reinterpret_cast<const char *>(c.plusA + (int64_t)u0 * Mp);
  const char *ms = reinterpret_cast<const char *>(c.minusA + (int64_t)u0 * Mp);
  for (int o = lane * 16; o < tb; o += 32 * 16) {
    cp_async16(tpb + o, ps + o);
    cp_async16(tmb + o, ms + o);
  }
  const char *ts = reinterpret_cast<const char *>(c.tupA + (int64_t)u0 * Mp);
  for (int o = lane * 16; o < cnt * Mp; o += 32 * 16) cp_async16(ttb + o, ts + o);
  cp_async_commit();
}

template <int N, typename CT, typename BT, bool CPLX>
__global__ void __launch_bounds__(kStageWarps * 32) stage_kernel(const __grid_constant__ StageArgs<CT> a) {
  using S = StageShape<N, CT, BT>;
  using C2 = typename Cplx<CT>::type;
  constexpr int E = S::E, A = S::A, EPO = S::EpOwn;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StageCommon &c = a.c;
  const int M = c.M, D1 = c.D + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // block-wide constants: rescaling tables and per-mode c, lamnu, state
  CT *sp_s = reinterpret_cast<CT *>(smem_raw);
  CT *sm_s = sp_s + M * D1;
  CT *cc_s = sm_s + M * D1;
  CT *ln_s = cc_s + M;
  int *st_s = reinterpret_cast<int *>(ln_s + M);
  for (int t = threadIdx.x; t < M * D1; t += blockDim.x) {
    sp_s[t] = (CT)c.sp_tab[t];
    sm_s[t] = (CT)c.sm_tab[t];
  }
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    cc_s[t] = (CT)c.modes[t].c;
    ln_s[t] = (CT)c.modes[t].lamnu;
    st_s[t] = c.modes[t].state;
  }
  __syncthreads();

  const WarpSmem<N, CT, BT> W(c.Mp);
  unsigned char *wb = smem_raw + stage_const_bytes<CT>(M, c.D) + warp * W.total;
  const int d_tile = W.tile1 - W.tile0, d_tp = W.tp1 - W.tp0, d_tm = W.tm1 - W.tm0, d_tt = W.tt1 - W.tt0;
  C2 *ybuf = reinterpret_cast<C2 *>(wb + W.ybuf);
  int *sv = reinterpret_cast<int *>(wb + W.sv);
  int *sst = reinterpret_cast<int *>(wb + W.sst);
  C2 *sco = reinterpret_cast<C2 *>(wb + W.sco);
  C2 *gbuf = reinterpret_cast<C2 *>(wb + W.gbuf);

  const int la = lane / N;
  const int li = lane - la * N;
  const bool lane_ok = la < A;
  const bool has_y = (c.y.head != nullptr) || (c.y.body != nullptr);
  const CT term_i = lane_ok ? a.term[li] : (CT)0;
  CT Hrow[S::kRowRegs ? N : 1];
  if (S::kRowRegs) {
#pragma unroll
    for (int k = 0; k < (S::kRowRegs ? N : 1); ++k) Hrow[k] = lane_ok ? a.H[li * kMaxStates + k] : (CT)0;
  }
  const C2 *zin_own = S::kOwnHead ? reinterpret_cast<const C2 *>(c.zin.head) : reinterpret_cast<const C2 *>(c.zin.body);
  C2 *out_own = S::kOwnHead ? reinterpret_cast<C2 *>(c.out.head) : reinterpret_cast<C2 *>(c.out.body);
  const C2 *y_own = S::kOwnHead ? reinterpret_cast<const C2 *>(c.y.head) : reinterpret_cast<const C2 *>(c.y.body);
  const int own0 = S::kOwnHead ? 0 : c.u_split;

  const int n_chunks = (c.u_end - c.u_begin + A - 1) / A;
  const int nwarps = gridDim.x * kStageWarps;
  int chunk = blockIdx.x * kStageWarps + warp;
  if (chunk < n_chunks) {
    const int u0 = c.u_begin + chunk * A;
    issue_chunk<N, CT, BT>(c, lane, u0, min(A, c.u_end - u0), zin_own, own0, (char *)(wb + W.tile0),
                           (char *)(wb + W.tp0), (char *)(wb + W.tm0), (char *)(wb + W.tt0));
  }
  for (int b = 0; chunk < n_chunks; chunk += nwarps, b ^= 1) {
    const int u0 = c.u_begin + chunk * A;
    const int cnt = min(A, c.u_end - u0);
    const int nxt = chunk + nwarps;
    const int nb_ = b ^ 1;
    if (nxt < n_chunks) {
      const int v0 = c.u_begin + nxt * A;
      issue_chunk<N, CT, BT>(c, lane, v0, min(A, c.u_end - v0), zin_own, own0, (char *)(wb + W.tile0 + nb_ * d_tile),
                             (char *)(wb + W.tp0 + nb_ * d_tp), (char *)(wb + W.tm0 + nb_ * d_tm),
                             (char *)(wb + W.tt0 + nb_ * d_tt));
    } else {
      cp_async_commit();  // keep the group count uniform
    }
    if (has_y) {  // this chunk's y tiles
      const char *src = reinterpret_cast<const char *>(y_own + (int64_t)(u0 - own0) * EPO);
      const int bytes = cnt * EPO * (int)sizeof(C2);
      for (int o = lane * 16; o < bytes; o += 32 * 16) cp_async16(reinterpret_cast<char *>(ybuf) + o, src + o);
    }
    cp_async_commit();
    cp_async_wait<2>();  // the current chunk's tiles and tables have landed
    __syncwarp();
    C2 *zt_all = reinterpret_cast<C2 *>(wb + W.tile0 + b * d_tile);
    const int *tp = reinterpret_cast<const int *>(wb + W.tp0 + b * d_tp);
    const int *tm = reinterpret_cast<const int *>(wb + W.tm0 + b * d_tm);
    const unsigned char *tt = wb + W.tt0 + b * d_tt;
    const bool active = lane_ok && la < cnt;
    const int tot = cnt * M * 2;
    int e_pos = 0;

    // first link batch: its gathers fly while the commutator is computed
    int nb = plan_and_gather<N, CT, BT>(c, lane, tot, e_pos, tp, tm, tt, sp_s, sm_s, cc_s, ln_s, st_s, sv, sst, sco,
                                        gbuf);
    {
      const C2 *zt = zt_all + la * EPO;
      CT rr[N], ri[N];
      if (active) {
        // commutator -i (H s - s H), decay and terminator
#pragma unroll
        for (int j = 0; j < N; ++j) { rr[j] = 0; ri[j] = 0; }
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const CT h = S::kRowRegs ? Hrow[S::kRowRegs ? k : 0] : a.H[li * kMaxStates + k];
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const C2 z = zt[k * N + j];
            rr[j] = fma(h, z.y, rr[j]);
            ri[j] = fma(-h, z.x, ri[j]);
          }
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const C2 zk = zt[li * N + k];
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const CT h = a.H[k * kMaxStates + j];
            rr[j] = fma(-zk.y, h, rr[j]);
            ri[j] = fma(zk.x, h, ri[j]);
          }
        }
        if constexpr (CPLX) {  // imaginary part of H
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const CT h = a.Hi[li * kMaxStates + k];
            const C2 zk = zt[li * N + k];
#pragma unroll
            for (int j = 0; j < N; ++j) {
              const C2 z = zt[k * N + j];
              rr[j] = fma(h, z.x, rr[j]);
              ri[j] = fma(h, z.y, ri[j]);
              const CT h2 = a.Hi[k * kMaxStates + j];
              rr[j] = fma(-zk.x, h2, rr[j]);
              ri[j] = fma(-zk.y, h2, ri[j]);
            }
          }
        }
        const CT gsv = (CT)c.gsum[u0 + la];
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const C2 zij = zt[li * N + j];
          const CT f = gsv + ((j != li) ? (term_i + a.term[j]) : (CT)0);
          rr[j] = fma(-f, zij.x, rr[j]);
          ri[j] = fma(-f, zij.y, ri[j]);
        }
      }
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
    cp_async_wait<0>();  // gathers (and the next chunk's copies) have landed
    __syncwarp();
    apply_links<N, CT, BT>(nb, cnt, lane, la, li, active, zt_all, sst, sco, gbuf);
    while (e_pos < tot) {  // remaining link batches
      __syncwarp();
      nb = plan_and_gather<N, CT, BT>(c, lane, tot, e_pos, tp, tm, tt, sp_s, sm_s, cc_s, ln_s, st_s, sv, sst, sco,
                                      gbuf);
      cp_async_wait<0>();
      __syncwarp();
      apply_links<N, CT, BT>(nb, cnt, lane, la, li, active, zt_all, sst, sco, gbuf);
    }
    __syncwarp();
    // y + ch * rhs, coalesced over the chunk's contiguous tiles
    {
      C2 *dst = out_own + (int64_t)(u0 - own0) * EPO;
      for (int t = lane; t < cnt * E; t += 32) {
        const int aa = t / E, e = t - aa * E;
        C2 w = zt_all[aa * EPO + e];
        w.x *= a.ch;
        w.y *= a.ch;
        if (has_y) {
          const C2 yv = ybuf[aa * EPO + e];
          w.x += yv.x;
          w.y += yv.y;
        }
        dst[aa * EPO + e] = w;
      }
    }
    __syncwarp();  // this tile buffer and ybuf are reused by later chunks
  }
  cp_async_wait<0>();
}

template <int N, typename CT, typename BT>
size_t stage_smem_total(int M, int Mp, int D) {
  const WarpSmem<N, CT, BT> W(Mp);
  return (size_t)stage_const_bytes<CT>(M, D) + (size_t)kStageWarps * W.total;
}

template <int N, typename CT, typename BT, bool CPLX>
int launch_v(const StageArgs<CT> &a, cudaStream_t st, int sm_count) {
  const StageCommon &c = a.c;
  const size_t smem = stage_smem_total<N, CT, BT>(c.M, c.Mp, c.D);
  // per-instantiation cache of the occupancy for the last shared-memory size
  static size_t cached_smem = 0;
  static int cached_per_sm = 0;
  if (smem != cached_smem) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(stage_kernel<N, CT, BT, CPLX>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) {
        set_error(std::string("stage kernel: shared memory attribute: ") + cudaGetErrorString(e));
        return -4;
      }
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel<N, CT, BT, CPLX>,
                                                                  kStageWarps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) {
      set_error(std::string("stage kernel: occupancy query failed or zero blocks: ") + cudaGetErrorString(e));
      return -4;
    }
    cached_smem = smem;
    cached_per_sm = per_sm;
  }
  constexpr int A = StageShape<N, CT, BT>::A;
  const int n_chunks = (c.u_end - c.u_begin + A - 1) / A;
  const int blocks_needed = (n_chunks + kStageWarps - 1) / kStageWarps;
  const int grid = std::max(1, std::min(blocks_needed, cached_per_sm * sm_count));
  stage_kernel<N, CT, BT, CPLX><<<grid, kStageWarps * 32, smem, st>>>(a);
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
