// Stage kernel for runs in the excited-ground coherence block (linear-absorption runs).
//
// When state 0 carries no bath, H has no element between state 0 and the others, and every ADO
// starts in span{|a><0| : a != 0} (a dipole run: sigma_0(0) = mu^+ |0><0|, all other ADOs zero),
// every term of Eq. HEOM (arXiv 1803.03498, section "HEOM formalism") keeps every ADO in that block:
// the commutator maps |a><0| to sum_b H_ba |b><0| - |a><0| H_00, and V_s = |s><s| with s != 0 acts on
// |a><0| only through its row (V_s |a><0| = delta_sa |s><0|, |a><0| V_s = 0).  Each ADO is then the
// column x_a = sigma[a][0] (x_0 = 0), and its right-hand side is
//     (L x)_a = -i sum_b (H_ab - H_00 delta_ab) x_b - (sum_l n_l gamma_l + Delta_a) x_a
//               + sum over the links of u through a mode of state a of R v_a
// with the link coefficients R of the full form (its column part and diagonal part vanish here).
// out_u = y_u + ch (L zin)_u as in stage_kernel (Horner RK4).  A chunk is A = floor(32 / N)
// consecutive ADOs; lane (a, i) of a warp holds element i of ADO a of a chunk.  A warp works on G
// consecutive chunks at once (G, the chunks per warp, is a
// launch-schedule choice of the autotuner; at most 32 ADOs per warp step): each lane holds one
// element of each, and the link records of all of them load together, G per lane per window of 32 G,
// followed by the neighbour elements they name.  The products go into a per-warp shared-memory list
// in record order; records are sorted by ADO and state, so each owner's products form one segment,
// whose bounds a per-window table gives to the owner lane, which adds them in order.  H x reads the
// chunk's column from shared memory (one broadcast load per term).  Every G sums the same terms
// in the same order for each element, and the serial memory round trips of a warp step (offsets,
// records, neighbour elements) are shared by G chunks.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "heom_internal.h"

namespace heom {

template <typename T>
struct VCplx;
template <>
struct VCplx<float> {
  using type = float2;
};
template <>
struct VCplx<double> {
  using type = double2;
};

constexpr int kVecWarps = 8;  // warps per CTA

// Element s of ADO v's column from the head (FP64) or body (storage type BT) region, as CT.
template <int N, typename CT, typename BT>
__device__ __forceinline__ typename VCplx<CT>::type vec_load(const StateView &s, int u_split, int64_t v, int e) {
  typename VCplx<CT>::type r;
  if (v < u_split) {
    const double2 d = s.head[v * N + e];
    r.x = (CT)d.x;
    r.y = (CT)d.y;
  } else {
    const typename VCplx<BT>::type b = reinterpret_cast<const typename VCplx<BT>::type *>(s.body)[(v - u_split) * N + e];
    r.x = (CT)b.x;
    r.y = (CT)b.y;
  }
  return r;
}

// One warp step: GE = vec_group(N, G) chunks, i.e. the SA = GE A consecutive ADOs starting at
// u0 = c.u_begin + step SA, of the stage out = y + ch L zin.  kOwnHead: CT = double, BT = float -- the
// FP64 head kernel of a mixed-precision run (its own ADOs are in the head region); otherwise the
// own ADOs are in the body region of storage type BT == CT.  hrow: row li of H; h00 = H_00;
// term_i = Delta of state li.
// Shared memory of one warp: the link products of a window in record order, the segment of each
// owner in it, and the columns of the step's chunks.
template <typename CT, int GE>
struct VecWarpSmem {
  typename VCplx<CT>::type del[32 * GE];  // R v of window entry k
  int first[32 * GE], end[32 * GE];       // per owner (g 32 + lane): its entries [first, end)
  typename VCplx<CT>::type xs[32 * GE];
};

template <int N, typename CT, typename BT, int G>
__device__ __forceinline__ void vec_step(const StageCommon &c, const CT (&hrow)[N], CT h00, CT term_i, CT ch,
                                         int step, int lane, VecWarpSmem<CT, vec_group(N, G)> &ws) {
  using C2 = typename VCplx<CT>::type;
  constexpr int A = 32 / N;
  constexpr int GE = vec_group(N, G);
  constexpr int SA = GE * A;
  constexpr bool kOwnHead = sizeof(CT) == 8 && sizeof(BT) == 4;
  const int la = lane / N, li = lane - la * N;
  const bool lane_ok = la < A;
  const bool has_y = (c.y.head != nullptr) || (c.y.body != nullptr);
  const LinkRec<CT> *recs = reinterpret_cast<const LinkRec<CT> *>(kOwnHead ? c.recs_head : c.recs_body);
  const int64_t rbase = kOwnHead ? 0 : c.rec_split;
  const int64_t rlim = kOwnHead ? c.rec_split : c.n_recs;  // records [rbase, rlim) of this region
  const int u0 = c.u_begin + step * SA;
  const int cnt = min(SA, c.u_end - u0);
  C2 x[GE], yv[GE];
  CT rr[GE], ri[GE];
#pragma unroll
  for (int g = 0; g < GE; ++g) {
    const int a = g * A + la;
    x[g].x = 0;
    x[g].y = 0;
    yv[g] = x[g];
    if (lane_ok && a < cnt) {
      x[g] = vec_load<N, CT, BT>(c.zin, c.u_split, u0 + a, li);
      if (has_y) yv[g] = vec_load<N, CT, BT>(c.y, c.u_split, u0 + a, li);
    }
  }
  // -i (H x)_i + i H_00 x_i, then decay and terminator; the columns go through shared memory (every
  // lane of an ADO reads the same word: one broadcast load per term)
  __syncwarp();  // the previous step's readers of ws are done
#pragma unroll
  for (int g = 0; g < GE; ++g) ws.xs[g * 32 + lane] = x[g];
  __syncwarp();
#pragma unroll
  for (int g = 0; g < GE; ++g) {
    rr[g] = -h00 * x[g].y;
    ri[g] = h00 * x[g].x;
    const C2 *col = ws.xs + g * 32 + min(la, A - 1) * N;
#pragma unroll
    for (int b = 0; b < N; ++b) {
      const C2 xb = col[b];
      rr[g] = fma(hrow[b], xb.y, rr[g]);
      ri[g] = fma(-hrow[b], xb.x, ri[g]);
    }
    const int a = g * A + la;
    if (lane_ok && a < cnt) {
      const CT f = (CT)c.gsum[u0 + a] + term_i;
      rr[g] = fma(-f, x[g].x, rr[g]);
      ri[g] = fma(-f, x[g].y, ri[g]);
    }
  }
  // links, 32 GE records of the step at a time: lane l loads records base + 32 q + l (q < GE), then
  // the neighbour element s each names, and forms R v_s; the contributions then go to their owner
  // (chunk g, lane (a, s)), o = g A + a the record's ADO in the step (tag u mod 32): entry k of the
  // window's list holds record base + k, the owner's entries are contiguous (records sorted by ADO
  // and state), and the owner adds its segment in order
  {
    const int64_t lo = c.link_off[u0], hi = c.link_off[u0 + cnt];
    for (int64_t base = lo; base < hi; base += 32 * GE) {
      LinkRec<CT> rq[GE];
#pragma unroll
      for (int q = 0; q < GE; ++q) {
        const int64_t t = base + q * 32 + lane;
        rq[q].v = -1;
        if (t < hi && HEOM_IN_RANGE(c.err, t, rbase, rlim)) rq[q] = recs[t - rbase];
      }
      int owner[GE];
      CT cr[GE], ci[GE];
#pragma unroll
      for (int q = 0; q < GE; ++q) {
        const int64_t t = base + q * 32 + lane;
        owner[q] = -1;
        cr[q] = 0;
        ci[q] = 0;
        if (t < hi && HEOM_IN_RANGE(c.err, rq[q].v, 0, c.n_ado) &&
            HEOM_IN_RANGE(c.err, rq[q].s & kRecStateMask, 0, N)) {
          const int st = rq[q].s & kRecStateMask;
          const int o = ((rq[q].s >> 8) - u0) & 31;
          const int og = o / A;
          owner[q] = og * 32 + (o - og * A) * N + st;
          const C2 v = vec_load<N, CT, BT>(c.zin, c.u_split, rq[q].v, st);
          cr[q] = fma(rq[q].re, v.x, -rq[q].im * v.y);
          ci[q] = fma(rq[q].re, v.y, rq[q].im * v.x);
        }
      }
      __syncwarp();  // the previous window's readers of the list and the table are done
#pragma unroll
      for (int q = 0; q < GE; ++q) {
        C2 d;
        d.x = cr[q];
        d.y = ci[q];
        ws.del[q * 32 + lane] = d;
        ws.first[q * 32 + lane] = 0;
        ws.end[q * 32 + lane] = 0;
      }
      __syncwarp();
      // segment bounds: entry k starts its owner's segment when entry k - 1 has another owner, and
      // ends it when entry k + 1 has another owner (invalid entries have owner -1)
#pragma unroll
      for (int q = 0; q < GE; ++q) {
        const int up = __shfl_up_sync(0xffffffffu, owner[q], 1);
        const int dn = __shfl_down_sync(0xffffffffu, owner[q], 1);
        const int pq = __shfl_sync(0xffffffffu, owner[q > 0 ? q - 1 : 0], 31);
        const int nq = __shfl_sync(0xffffffffu, owner[q + 1 < GE ? q + 1 : q], 0);
        const int prev = lane > 0 ? up : (q > 0 ? pq : -2);
        const int next = lane < 31 ? dn : (q + 1 < GE ? nq : -2);
        const int o = owner[q], k = q * 32 + lane;
        if (o >= 0) {
          if (o != prev) ws.first[o] = k;
          if (o != next) ws.end[o] = k + 1;
        }
      }
      __syncwarp();
#pragma unroll
      for (int g = 0; g < GE; ++g) {
        const int f = ws.first[g * 32 + lane], e = ws.end[g * 32 + lane];
        for (int k = f; k < e; ++k) {
          const C2 d = ws.del[k];
          rr[g] += d.x;
          ri[g] += d.y;
        }
      }
    }
  }
#pragma unroll
  for (int g = 0; g < GE; ++g) {
    const int a = g * A + la;
    if (!(lane_ok && a < cnt)) continue;
    const int64_t u = u0 + a;
    C2 o;
    o.x = has_y ? fma(ch, rr[g], yv[g].x) : ch * rr[g];
    o.y = has_y ? fma(ch, ri[g], yv[g].y) : ch * ri[g];
    if (kOwnHead || u < c.u_split) {
      c.out.head[u * N + li] = make_double2((double)o.x, (double)o.y);
    } else {
      typename VCplx<BT>::type w;
      w.x = (BT)o.x;
      w.y = (BT)o.y;
      reinterpret_cast<typename VCplx<BT>::type *>(c.out.body)[(u - c.u_split) * N + li] = w;
    }
  }
}

template <int N, typename CT, typename BT, int G>
__global__ void __launch_bounds__(kVecWarps * 32) vec_stage_kernel(const __grid_constant__ StageArgs<CT> a) {
  constexpr int A = 32 / N;
  constexpr int SA = vec_group(N, G) * A;
  const StageCommon &c = a.c;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kVecWarps + (threadIdx.x >> 5);
  const int nw = gridDim.x * kVecWarps;
  const int la = lane / N, li = lane - la * N;
  const bool lane_ok = la < A;
  CT hrow[N];
#pragma unroll
  for (int b = 0; b < N; ++b) hrow[b] = lane_ok ? a.H[li * kMaxStates + b] : (CT)0;
  const CT h00 = a.H[0];
  const CT term_i = lane_ok ? a.term[li] : (CT)0;
  const int n_steps = (c.u_end - c.u_begin + SA - 1) / SA;
  __shared__ VecWarpSmem<CT, vec_group(N, G)> wsm[kVecWarps];
  VecWarpSmem<CT, vec_group(N, G)> &ws = wsm[threadIdx.x >> 5];
  for (int sp = gw; sp < n_steps; sp += nw) vec_step<N, CT, BT, G>(c, hrow, h00, term_i, a.ch, sp, lane, ws);
}

// Many runs of the same N in one launch (ragged batches): run k's warp steps (of vec_group(N, G)
// chunks each) are the launch's steps [chunk0[k], chunk0[k+1]); its stage arguments sit in its own
// workspace (d[k]).
template <int N, typename CT, typename BT, int G>
__global__ void __launch_bounds__(kVecWarps * 32) vec_batch_kernel(const __grid_constant__ VecBatchArgs a) {
  constexpr int A = 32 / N;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kVecWarps + (threadIdx.x >> 5);
  const int nw = gridDim.x * kVecWarps;
  const int la = lane / N, li = lane - la * N;
  const bool lane_ok = la < A;
  const int64_t total = a.chunk0[a.nruns];
  __shared__ VecWarpSmem<CT, vec_group(N, G)> wsm[kVecWarps];
  VecWarpSmem<CT, vec_group(N, G)> &ws = wsm[threadIdx.x >> 5];
  int k = 0;
  for (int64_t g = gw; g < total; g += nw) {
    int lo = 0, hi = a.nruns - 1;  // the run holding global chunk g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.chunk0[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    k = lo;
    const VecRunDesc *d = a.d[k];
    const StageCommon c = d->c;  // by value: registers, not reloads after the chunk's stores
    CT hrow[N];
#pragma unroll
    for (int b = 0; b < N; ++b) hrow[b] = lane_ok ? (CT)__ldg(&d->H[li * kMaxStates + b]) : (CT)0;
    const CT h00 = (CT)__ldg(&d->H[0]), term_i = lane_ok ? (CT)__ldg(&d->term[li]) : (CT)0;
    vec_step<N, CT, BT, G>(c, hrow, h00, term_i, (CT)__ldg(&d->ch), (int)(g - a.chunk0[k]), lane, ws);
  }
  (void)k;
}

template <int N, typename CT, typename BT, int G>
int launch_vec_n(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                 int sm_count) {
  StageArgs<CT> a;
  a.c = c;
  a.ch = (CT)ch;
  for (int i = 0; i < kMaxStates; ++i) a.term[i] = (i < c.n) ? (CT)term[i] : (CT)0;
  for (int i = 0; i < kMaxStates * kMaxStates; ++i) {
    a.H[i] = 0;
    a.Hi[i] = 0;
  }
  for (int i = 0; i < c.n; ++i)
    for (int j = 0; j < c.n; ++j) a.H[i * kMaxStates + j] = (CT)H[i * c.n + j];
  static int per_sm = 0;
  if (per_sm == 0) {
    int ps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, vec_stage_kernel<N, CT, BT, G>, kVecWarps * 32, 0);
    if (e != cudaSuccess || ps < 1) {
      set_error(std::string("vector stage kernel: occupancy query failed: ") + cudaGetErrorString(e));
      return -4;
    }
    per_sm = ps;
  }
  constexpr int SA = vec_group(N, G) * (32 / N);
  const int n_steps = (c.u_end - c.u_begin + SA - 1) / SA;
  const int grid = std::max(1, std::min((n_steps + kVecWarps - 1) / kVecWarps, sched_ctas(per_sm, c.occ_pct) * sm_count));
  vec_stage_kernel<N, CT, BT, G><<<grid, kVecWarps * 32, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("vector stage kernel launch: ") + cudaGetErrorString(e));
    return -4;
  }
  return 0;
}

template <int N, typename CT, typename BT, int G>
int launch_vec_batch_n(const VecBatchArgs &a, cudaStream_t st, int sm_count) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int ps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, vec_batch_kernel<N, CT, BT, G>, kVecWarps * 32, 0);
    if (e != cudaSuccess || ps < 1) {
      set_error(std::string("batched vector kernel: occupancy query failed: ") + cudaGetErrorString(e));
      return -4;
    }
    per_sm = ps;
  }
  const int64_t total = a.chunk0[a.nruns];
  if (total <= 0) return 0;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((total + kVecWarps - 1) / kVecWarps, (int64_t)sched_ctas(per_sm, a.occ_pct) * sm_count));
  vec_batch_kernel<N, CT, BT, G><<<grid, kVecWarps * 32, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("batched vector kernel launch: ") + cudaGetErrorString(e));
    return -4;
  }
  return 0;
}

// The launchers of one chunks-per-warp value for n_states 2..kMaxStates: kind 0 FP64 (double,
// double), 1 mixed body (float, float), 2 mixed head (double, float).
template <int G, int N = 2>
int vec_dispatch(int kind, const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                 int sm_count) {
  if constexpr (N > kMaxStates) {
    set_error("vector stage kernel: n_states not compiled");
    return -1;
  } else {
    if (c.n != N) return vec_dispatch<G, N + 1>(kind, c, ch, term, H, st, sm_count);
    return kind == 0 ? launch_vec_n<N, double, double, G>(c, ch, term, H, st, sm_count)
         : kind == 1 ? launch_vec_n<N, float, float, G>(c, ch, term, H, st, sm_count)
                     : launch_vec_n<N, double, float, G>(c, ch, term, H, st, sm_count);
  }
}

template <int G, int N = 2>
int vec_batch_dispatch(int kind, int n, const VecBatchArgs &a, cudaStream_t st, int sm_count) {
  if constexpr (N > kMaxStates) {
    set_error("batched vector kernel: n_states not compiled");
    return -1;
  } else {
    if (n != N) return vec_batch_dispatch<G, N + 1>(kind, n, a, st, sm_count);
    return kind == 0 ? launch_vec_batch_n<N, double, double, G>(a, st, sm_count)
         : kind == 1 ? launch_vec_batch_n<N, float, float, G>(a, st, sm_count)
                     : launch_vec_batch_n<N, double, float, G>(a, st, sm_count);
  }
}

}  // namespace heom
