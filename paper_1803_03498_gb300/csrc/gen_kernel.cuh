// General stage kernel: runs the specialised kernels do not cover -- couplings V_b that are diagonal
// with several 1s (the site-number operators of the two-exciton space, section "Dipole operators and
// rotational averaging"), a time-dependent H(t) (the laser field of Eq. h-field-rwa, evaluated on the
// host at each RK4 stage time and passed with the launch) and up to kGenMaxStates states (29 for
// the FMO two-exciton space).  One launch computes, for every ADO u of its range,
//     k_u = (L(t) zin)_u      (Eq. HEOM, element-wise)
//     out1_u = base1_u + c1 k_u,   and, if out2 is set, out2_u = base2_u + c2 k_u
// which covers Horner RK4 (out2 unset) and the classic four-copy RK4 of a time-dependent L
// (X_{s+1} = y + a_{s+1} h k_s and acc += w_s h k_s in one pass).
//
// Element (i, j) of L sigma_u:
//   -i sum_k (H_ik s_kj - s_ik H_kj) - (sum_l n_l gamma_l + T_ij) s_ij + link terms
// with T_ij = sum_b Delta_b (v_b[i] - v_b[j])^2 the terminator of Eq. HEOM for diagonal V_b (host),
// and per link record (v, s, R): R v_sj added to element (s, j) and conj(R) v_is to element (i, s)
// (both for i = j = s: 2 Re R on the diagonal), as for every other kernel.
//
// A warp works on rows [i0, i1) of one ADO -- all rows, or a share of them when a launch has fewer
// ADOs than SMs (the FP64 head of a mixed run): element (i, j) needs only row i's own terms, so the
// rows of an ADO can go to warps on different SMs (GB300's FP64 pipe, 2 FMA per clock per SM, is
// then shared by fewer warps).  Lane j owns column j (N <= 32).  The input tile is staged in shared memory
// (column reads conflict-free, row reads broadcast); H, Im H and T sit in shared memory once per
// CTA.  The commutator, decay and terminator go to a result tile R that lane j writes in column j;
// the row parts of the links also land in column j of R (lane j loads v_sj, coalesced), the column
// parts in row i of a second tile C (lane i loads v_is; C reuses the input tile's buffer), so no
// element is written by two lanes and no synchronisation is needed between records.  The records of
// an ADO load 32 at a time, one per lane, and reach every lane by shuffles.  out = base + c (R + C).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "heom_internal.h"

namespace heom {

constexpr int kGenWarps = 4;

template <typename T>
struct GCplx;
template <>
struct GCplx<float> {
  using type = float2;
};
template <>
struct GCplx<double> {
  using type = double2;
};

// Element e of ADO v of a state copy (head FP64, body storage BT), as CT.
template <typename CT, typename BT>
__device__ __forceinline__ typename GCplx<CT>::type gen_load(const StateView &s, int E, int Ep, int u_split, int64_t v,
                                                             int e) {
  typename GCplx<CT>::type r;
  if (v < u_split) {
    const double2 d = s.head[v * E + e];
    r.x = (CT)d.x;
    r.y = (CT)d.y;
  } else {
    const typename GCplx<BT>::type b = reinterpret_cast<const typename GCplx<BT>::type *>(s.body)[(v - u_split) * Ep + e];
    r.x = (CT)b.x;
    r.y = (CT)b.y;
  }
  return r;
}

template <typename CT, typename BT>
__device__ __forceinline__ void gen_store(const StateView &s, int E, int Ep, int u_split, int64_t v, int e, CT re,
                                          CT im) {
  if (v < u_split) {
    s.head[v * E + e] = make_double2((double)re, (double)im);
  } else {
    typename GCplx<BT>::type w;
    w.x = (BT)re;
    w.y = (BT)im;
    reinterpret_cast<typename GCplx<BT>::type *>(s.body)[(v - u_split) * Ep + e] = w;
  }
}

// Kind as the other kernels: (double, double) FP64; (float, float) mixed body; (double, float) mixed
// head (own ADOs in the FP64 head region, neighbours in either region).
// kSplit: the launch splits ADO rows over warps (splits > 1); otherwise every warp takes whole ADOs.
template <typename CT, typename BT, bool kSplit>
__global__ void __launch_bounds__(kGenWarps * 32) gen_stage_kernel(const __grid_constant__ GenArgs<CT> a, int splits_arg) {
  using C2 = typename GCplx<CT>::type;
  constexpr bool kOwnHead = sizeof(CT) == 8 && sizeof(BT) == 4;
  const StageCommon &c = a.c;
  const int N = c.n, E = c.E, Ep = c.Ep;
  const int splits = kSplit ? splits_arg : 1;
  const int wpc = blockDim.x >> 5;             // warps per CTA
  const int rows = kSplit ? (N + splits - 1) / splits : N;  // rows per task
  extern __shared__ __align__(16) unsigned char gsm[];
  CT *Hs = reinterpret_cast<CT *>(gsm);  // [N][N] Re H(t), then Im H(t), then T
  CT *His = Hs + E;
  CT *Ts = His + E;
  const size_t off = (((size_t)3 * E * sizeof(CT)) + 15) & ~(size_t)15;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  C2 *Z = reinterpret_cast<C2 *>(gsm + off) + (size_t)warp * 2 * E;  // input tile, then the column parts
  C2 *R = Z + E;                                                      // commutator, decay, row parts
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    const int i = e / N, j = e - (e / N) * N;
    Hs[e] = a.H[i * kGenMaxStates + j];
    His[e] = a.Hi[i * kGenMaxStates + j];
    Ts[e] = a.T[i * kGenMaxStates + j];
  }
  __syncthreads();
  const LinkRec<CT> *recs = reinterpret_cast<const LinkRec<CT> *>(kOwnHead ? c.recs_head : c.recs_body);
  const int64_t rbase = kOwnHead ? 0 : c.rec_split;
  const int64_t rlim = kOwnHead ? c.rec_split : c.n_recs;  // records [rbase, rlim) of this region
  const bool has_b1 = c.y.head != nullptr || c.y.body != nullptr;
  const bool has_o2 = a.out2.head != nullptr || a.out2.body != nullptr;
  const bool has_b2 = a.base2.head != nullptr || a.base2.body != nullptr;
  const int j = lane;
  const bool lj = j < N;
  const int64_t gw = (int64_t)blockIdx.x * wpc + warp, nw = (int64_t)gridDim.x * wpc;
  const int64_t n_tasks = (int64_t)(c.u_end - c.u_begin) * splits;
  for (int64_t task = gw; task < n_tasks; task += nw) {
    const int64_t u = c.u_begin + (kSplit ? task / splits : task);
    const int i0 = kSplit ? (int)(task % splits) * rows : 0, i1 = kSplit ? min(N, i0 + rows) : N;
    for (int e = lane; e < E; e += 32) Z[e] = gen_load<CT, BT>(c.zin, E, Ep, c.u_split, u, e);
    __syncwarp();
    const CT g = (CT)c.gsum[u];
    if (lj) {
      for (int i = i0; i < i1; ++i) {
        // -i (H s - s H)_ij with H = Hr + i Hi
        // (H s - s H)_ij as a chain of FMAs, four per component and k (on GB300 every FP64 warp
        // instruction occupies the SM's FP64 pipe for 16 cycles: no separate multiplies and adds)
        CT pr = 0, pi = 0;
        for (int k = 0; k < N; ++k) {
          const C2 skj = Z[k * N + j], sik = Z[i * N + k];
          const CT hr1 = Hs[i * N + k], hi1 = His[i * N + k], hr2 = Hs[k * N + j], hi2 = His[k * N + j];
          pr = fma(hr1, skj.x, pr);
          pr = fma(-hi1, skj.y, pr);
          pr = fma(-sik.x, hr2, pr);
          pr = fma(sik.y, hi2, pr);
          pi = fma(hr1, skj.y, pi);
          pi = fma(hi1, skj.x, pi);
          pi = fma(-sik.x, hi2, pi);
          pi = fma(-sik.y, hr2, pi);
        }
        const C2 sij = Z[i * N + j];
        const CT f = g + Ts[i * N + j];
        C2 r;
        r.x = pi - f * sij.x;  // -i (pr + i pi) = pi - i pr
        r.y = -pr - f * sij.y;
        R[i * N + j] = r;
      }
    }
    __syncwarp();
    for (int e = lane; e < E; e += 32) Z[e] = C2{0, 0};  // Z becomes the column-part tile
    __syncwarp();
    const int64_t lo = c.link_off[u], hi = c.link_off[u + 1];
    // the records of a window of 32 load together, one per lane, and reach every lane by shuffles;
    // the neighbour loads of 4 records are in flight together (unrolled)
    for (int64_t base = lo; base < hi; base += 32) {
      const int cnt = (int)min((int64_t)32, hi - base);
      LinkRec<CT> mine{};
      mine.v = -1;
      if (lane < cnt && HEOM_IN_RANGE(c.err, base + lane, rbase, rlim)) mine = recs[base + lane - rbase];
#pragma unroll 4
      for (int k = 0; k < cnt; ++k) {
        const int v = __shfl_sync(0xffffffffu, mine.v, k);
        const int s = __shfl_sync(0xffffffffu, mine.s, k) & kRecStateMask;
        const CT rre = __shfl_sync(0xffffffffu, mine.re, k), rim = __shfl_sync(0xffffffffu, mine.im, k);
        if (!HEOM_IN_RANGE(c.err, v, 0, c.n_ado) || !HEOM_IN_RANGE(c.err, s, 0, N)) continue;
        if (lj && s >= i0 && s < i1) {  // row part: element (s, j) += R v_sj (lane j, column j of R)
          const C2 vs = gen_load<CT, BT>(c.zin, E, Ep, c.u_split, v, s * N + j);
          C2 &rs = R[s * N + j];
          rs.x += rre * vs.x - rim * vs.y;
          rs.y += rre * vs.y + rim * vs.x;
        }
        if (j >= i0 && j < i1) {  // column part: element (i = j, s) += conj(R) v_js (lane j, row j of Z)
          const C2 vc = gen_load<CT, BT>(c.zin, E, Ep, c.u_split, v, j * N + s);
          C2 &zc = Z[j * N + s];
          zc.x += rre * vc.x + rim * vc.y;
          zc.y += rre * vc.y - rim * vc.x;
        }
      }
    }
    __syncwarp();
    if (lj) {
      for (int i = i0; i < i1; ++i) {
        const int e = i * N + j;
        const C2 r = R[e], z = Z[e];
        const CT kr = r.x + z.x, ki = r.y + z.y;
        C2 b1 = C2{0, 0};
        if (has_b1) b1 = gen_load<CT, BT>(c.y, E, Ep, c.u_split, u, e);
        CT o2r = 0, o2i = 0;
        if (has_o2) {
          C2 b2 = C2{0, 0};
          if (has_b2) b2 = gen_load<CT, BT>(a.base2, E, Ep, c.u_split, u, e);
          o2r = fma(a.c2, kr, b2.x);
          o2i = fma(a.c2, ki, b2.y);
        }
        // every read of base1 / base2 for this element happens before its writes (out1 may be base2)
        gen_store<CT, BT>(c.out, E, Ep, c.u_split, u, e, fma(a.c1, kr, b1.x), fma(a.c1, ki, b1.y));
        if (has_o2) gen_store<CT, BT>(a.out2, E, Ep, c.u_split, u, e, o2r, o2i);
      }
    }
    __syncwarp();  // Z and R are reused by the next ADO
  }
}

template <typename CT, typename BT>
int launch_gen_kind(const GenArgs<CT> &a, cudaStream_t st, int sm_count) {
  const StageCommon &c = a.c;
  if (c.u_end <= c.u_begin) return 0;
  const int64_t n = c.u_end - c.u_begin;
  // fewer ADOs than SMs: split each ADO's rows over single-warp CTAs on different SMs
  const int splits = n * 2 <= sm_count ? (int)std::min<int64_t>(c.n, (sm_count + n - 1) / n) : 1;
  const int wpc = splits > 1 ? 1 : kGenWarps;
  const size_t head_bytes = (((size_t)3 * c.E * sizeof(CT)) + 15) & ~(size_t)15;
  const size_t smem = head_bytes + (size_t)wpc * 2 * c.E * sizeof(typename GCplx<CT>::type);
  const size_t smem_max = ((((size_t)3 * kGenMaxStates * kGenMaxStates * sizeof(CT)) + 15) & ~(size_t)15) +
                          (size_t)kGenWarps * 2 * kGenMaxStates * kGenMaxStates * sizeof(typename GCplx<CT>::type);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gen_stage_kernel<CT, BT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_max);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gen_stage_kernel<CT, BT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_max);
    if (e != cudaSuccess) {
      set_error(std::string("general stage kernel: shared memory attribute: ") + cudaGetErrorString(e));
      return -4;
    }
    attr = true;
  }
  static int occ[2][kGenMaxStates + 1] = {{0}};  // CTAs per SM by CTA shape and n_states
  int &per_sm = occ[wpc == 1 ? 0 : 1][c.n];
  cudaError_t e;
  if (per_sm == 0) {
    int ps = 0;
    e = splits > 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, gen_stage_kernel<CT, BT, true>, wpc * 32, smem)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, gen_stage_kernel<CT, BT, false>, wpc * 32, smem);
    if (e != cudaSuccess || ps < 1) {
      set_error(std::string("general stage kernel: occupancy query failed: ") + cudaGetErrorString(e));
      return -4;
    }
    per_sm = ps;
  }
  const int64_t tasks = n * splits;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((tasks + wpc - 1) / wpc, (int64_t)sched_ctas(per_sm, c.occ_pct) * sm_count));
  if (splits > 1) gen_stage_kernel<CT, BT, true><<<grid, wpc * 32, smem, st>>>(a, splits);
  else gen_stage_kernel<CT, BT, false><<<grid, wpc * 32, smem, st>>>(a, 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("general stage kernel launch: ") + cudaGetErrorString(e));
    return -4;
  }
  return 0;
}

}  // namespace heom
