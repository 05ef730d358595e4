// FP64 stage kernel for Hermitian runs with a real H, column form (sm_103a).
//
// Same operation as stage_kernel: for every ADO u in [u_begin, u_end),
//     out_u = y_u + ch * (L zin)_u          (or ch * (L zin)_u when there is no y)
// with L the right-hand side of Eq. HEOM (arXiv 1803.03498, section "HEOM formalism", with the ADO
// rescaling; hbar = 1, energies in rad/fs).  For a Hermitian run (Hermitian H and ADOs, real c: every
// ADO stays Hermitian) the result is R = Q + Q^dagger with
//     Q_ij = -i (H s)_ij + coef_ij s_ij + sum over the links of state s = i of R_link v_ij
//     coef_ij = -(g / 2 + Delta_i)  (i != j),   coef_ii = -g / 2,     g = sum_l n_l gamma_l
// because s H = (H s)^dagger, the terminator (Delta_i + Delta_j) s_ij (i != j) splits into a row and
// a column part, and a link adds R v_sj to row s, conj(R) v_is = conj(R v_si) to column s and
// 2 Re(R) v_ss to the diagonal (see LinkRec).
//
// GB300's FP64 pipe retires 2 FMAs per clock per SM, so this kernel is bound by its FP64 instruction
// count, and a warp instruction costs the same whether 28 or 32 lanes do useful work.  The row form
// of stage_kernel maps lane (a, i) to row i of ADO a: at N = 14 two ADOs fill 28 of 32 lanes.  Here a
// lane owns one column of one part: lane (a, p, j) computes column j of Q_re (p = 0, from H Im s) or
// of Q_im (p = 1, from -H Re s) of ADO a -- 2N columns per ADO.  A warp takes chunks of G consecutive
// ADOs, G chosen so that 2 N G is a multiple of 32, and covers their 2 N G columns in P = 2 N G / 32
// passes with every lane busy (N = 14: 8 ADOs in 7 passes).  Per pass a lane
//   - loads column j of its ADO's zin tile from global memory (the 2N lanes of an ADO read whole rows:
//     coalesced), H enters every FMA as a kernel-parameter (constant-bank) operand;
//   - accumulates the N entries of its column of H (Im s) or -H (Re s) and adds coef * (own part);
//   - writes the column into its ADO's slot of a per-warp ring of Q tiles in shared memory.
// An ADO whose last column was computed in this pass is finalised by lanes (p, j) of the warp: the
// row s of every linked neighbour (gathered into shared memory by cp.async while the pass computed)
// is added to row s of Q, records in order; then R_ij = Q_ij + conj(Q_ji) and out = y + ch R leave
// with coalesced loads and stores.  Warps are independent (only __syncwarp).  Every output element
// sums the same terms in the same order under every launch schedule.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "heom_internal.h"

namespace heom {

__host__ __device__ constexpr int col_gcd(int a, int b) { return b == 0 ? a : col_gcd(b, a % b); }

// Most ADOs of C columns that one pass of 32 consecutive columns touches, over the P passes of a chunk.
__host__ __device__ constexpr int col_ring(int C, int P) {
  int m = 1;
  for (int q = 0; q < P; ++q) {
    const int t = (32 * q + 31) / C - (32 * q) / C + 1;
    m = t > m ? t : m;
  }
  return m;
}

template <int N>
struct ColShape {
  static constexpr int C = 2 * N;                  // columns per ADO (both parts)
  static constexpr int G = 32 / col_gcd(C, 32);    // ADOs per warp chunk
  static constexpr int P = C * G / 32;             // passes of 32 columns per chunk
  static constexpr int E = N * N;
  static constexpr int RING = col_ring(C, P);      // Q slots: the ADOs one pass touches (N = 14: 2)
  static constexpr int RB = 12;                    // link records per batch and finalising ADO
  static constexpr int WARPS = 4;                  // 4 CTAs of 4 warps per SM (128 registers, < 57 KB)
  static_assert(C >= 16 && G <= 31, "column kernel covers 8 <= N <= 16");
};

// Per-warp shared memory (byte offsets; every region 16-byte aligned).
template <int N>
struct ColSmem {
  using S = ColShape<N>;
  static constexpr int q = 0;                                    // [RING][2][N][N] double
  static constexpr int coef = q + S::RING * 2 * S::E * 8;        // [G][N] double: -(g/2 + Delta_i)
  static constexpr int gh = coef + S::G * N * 8;                 // [G] double: -g/2
  static constexpr int rec = (gh + S::G * 8 + 15) & ~15;         // [2 RB] LinkRec<double>
  static constexpr int gbuf = rec + 2 * S::RB * 32;              // [2 RB][N] double2: gathered rows
  static constexpr int total = gbuf + 2 * S::RB * N * 16;
};

__device__ __forceinline__ void col_cp16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void col_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void col_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// -x without an FP64 instruction (sign bit of the high word)
__device__ __forceinline__ double col_neg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// Records [lo, lo + nr) into rec (32 bytes each), one cp.async group.
__device__ __forceinline__ void col_load_recs(const LinkRec<double> *recs, int64_t lo, int nr, LinkRec<double> *rec,
                                              int lane) {
  const char *src = reinterpret_cast<const char *>(recs + lo);
  char *dst = reinterpret_cast<char *>(rec);
  for (int o = lane * 16; o < nr * 32; o += 32 * 16) col_cp16(dst + o, src + o);
  col_commit();
}

// Row s of the neighbour of each of the nr records into gbuf[r][0..N), one cp.async group.
template <int N>
__device__ __forceinline__ void col_gather(const StageCommon &c, const double2 *zin, int Ep, const LinkRec<double> *rec,
                                           int nr, double2 *gbuf, int lane) {
  for (int t = lane; t < nr * N; t += 32) {
    const int r = t / N, k = t - r * N;
    const int s = rec[r].s & kRecStateMask;
    if (HEOM_IN_RANGE(c.err, rec[r].v, 0, c.n_ado) && HEOM_IN_RANGE(c.err, s, 0, N))
      col_cp16(gbuf + r * N + k, zin + (int64_t)rec[r].v * Ep + s * N + k);
  }
  col_commit();
}

// Adds the nr records of rec (gathered rows in gbuf) to row s of the Q tile qs ([2][N][N]): lane
// (p, j) owns element (s, j) of part p; records are ordered by s, so each lane keeps its element in a
// register while s stays the same.  R v = (Rr vr - Ri vi) + i (Rr vi + Ri vr).
template <int N>
__device__ __forceinline__ void col_links(const LinkRec<double> *rec, int nr, const double2 *gbuf, double *qs, int lane) {
  if (lane >= 2 * N) return;
  const int p = lane / N, j = lane - p * N;
  double *qp = qs + p * N * N;
  int cur = -1;
  double acc = 0;
  for (int r = 0; r < nr; ++r) {
    const int s = rec[r].s & kRecStateMask;
    if (s != cur) {
      if (cur >= 0) qp[cur * N + j] = acc;
      cur = s;
      acc = qp[s * N + j];
    }
    const double2 v = gbuf[r * N + j];
    const double rr = rec[r].re, ri = rec[r].im;
    const double a1 = p ? v.y : v.x;             // Re part: Rr vr - Ri vi;  Im part: Rr vi + Ri vr
    const double a2 = p ? v.x : v.y;
    const double b2 = p ? ri : col_neg(ri);
    acc = fma(rr, a1, fma(b2, a2, acc));
  }
  if (cur >= 0) qp[cur * N + j] = acc;
}

template <int N>
__global__ void __launch_bounds__(ColShape<N>::WARPS * 32, 4) stage_col_kernel(const __grid_constant__ StageArgs<double> a) {
  using S = ColShape<N>;
  using W = ColSmem<N>;
  constexpr int C = S::C, G = S::G, P = S::P, E = S::E, RB = S::RB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StageCommon &c = a.c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *wb = smem_raw + warp * W::total;
  double *qring = reinterpret_cast<double *>(wb + W::q);
  double *coef = reinterpret_cast<double *>(wb + W::coef);
  double *gh = reinterpret_cast<double *>(wb + W::gh);
  LinkRec<double> *recb = reinterpret_cast<LinkRec<double> *>(wb + W::rec);
  double2 *gbuf = reinterpret_cast<double2 *>(wb + W::gbuf);

  const double2 *zin = reinterpret_cast<const double2 *>(c.zin.body);
  double *out = reinterpret_cast<double *>(c.out.body);
  const double *yv = reinterpret_cast<const double *>(c.y.body);
  const bool has_y = yv != nullptr;
  const LinkRec<double> *recs = reinterpret_cast<const LinkRec<double> *>(c.recs_body);
  const int Ep = c.Ep;
  const double ch = a.ch;

  const int n_chunks = (c.u_end - c.u_begin + G - 1) / G;
  const int nwarps = gridDim.x * S::WARPS;
  for (int chn = blockIdx.x * S::WARPS + warp; chn < n_chunks; chn += nwarps) {
    const int u0 = c.u_begin + chn * G;
    const int cnt = min(G, c.u_end - u0);
    // lane a <= cnt holds link_off[u0 + a]
    const int64_t off = (lane <= cnt) ? c.link_off[u0 + lane] : (int64_t)0;
    // per-ADO coefficients of this chunk
    for (int t = lane; t < cnt * N; t += 32) {
      const int ad = t / N, i = t - ad * N;
      coef[t] = fma(-0.5, c.gsum[u0 + ad], -a.term[i]);
    }
    if (lane < cnt) gh[lane] = -0.5 * c.gsum[u0 + lane];
    __syncwarp();

    for (int q = 0; q < P; ++q) {
      // ADOs whose last column falls in this pass: [fa, fb)
      const int fa = (32 * q) / C, fb = min((32 * q + 32) / C, cnt);
      // first record batch of each finalising ADO (at most 2 per pass for C >= 16) and its gathers
      int nrf0 = 0, nrf1 = 0;
      for (int f = fa, k = 0; f < fb; ++f, ++k) {
        const int64_t lo = __shfl_sync(0xffffffffu, off, f), hi = __shfl_sync(0xffffffffu, off, f + 1);
        const int nr = heom_rec_batch(c.err, lo, (int)min(hi - lo, (int64_t)RB), 0, c.n_recs);
        if (k == 0) nrf0 = nr;
        else nrf1 = nr;
        col_load_recs(recs, lo, nr, recb + k * RB, lane);
      }
      // this pass's column: lane -> (ADO ad, part p, column j)
      const int col = 32 * q + lane;
      const int ad = col / C, rem = col - ad * C;
      const int p = rem / N, j = rem - p * N;
      const bool act = ad < cnt;
      double2 zc[N];
      if (act) {
        const double2 *zt = zin + (int64_t)(u0 + ad) * Ep + j;
#pragma unroll
        for (int k = 0; k < N; ++k) zc[k] = zt[k * N];
      }
      col_wait_all();
      __syncwarp();
      for (int f = fa, k = 0; f < fb; ++f, ++k)
        col_gather<N>(c, zin, Ep, recb + k * RB, k == 0 ? nrf0 : nrf1, gbuf + k * RB * N, lane);
      if (act) {
        // p = 0: Q_re = H Im s + coef Re s;  p = 1: Q_im = -H Re s + coef Im s
        double src[N], own[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
          src[k] = p ? col_neg(zc[k].x) : zc[k].y;
          own[k] = p ? zc[k].y : zc[k].x;
        }
        double acc[N];
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
#pragma unroll
          for (int i = 0; i < N; ++i) acc[i] = fma(a.H[i * kMaxStates + k], src[k], acc[i]);
        }
        double *qs = qring + (ad % S::RING) * 2 * E + p * E;
        const double *cf = coef + ad * N;
        const double gd = gh[ad];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const double ci = (i == j) ? gd : cf[i];
          qs[i * N + j] = fma(ci, own[i], acc[i]);
        }
      }
      col_wait_all();  // gathers
      __syncwarp();
      // finalise every ADO completed in this pass
      for (int f = fa, k = 0; f < fb; ++f, ++k) {
        const int u = u0 + f;
        double *qs = qring + (f % S::RING) * 2 * E;
        const int64_t lo = __shfl_sync(0xffffffffu, off, f), hi = __shfl_sync(0xffffffffu, off, f + 1);
        const int nr0 = k == 0 ? nrf0 : nrf1;
        col_links<N>(recb + k * RB, nr0, gbuf + k * RB * N, qs, lane);
        for (int64_t blo = lo + nr0; blo < hi; blo += RB) {  // further record batches
          __syncwarp();
          const int nr = heom_rec_batch(c.err, blo, (int)min(hi - blo, (int64_t)RB), 0, c.n_recs);
          col_load_recs(recs, blo, nr, recb + k * RB, lane);
          col_wait_all();
          __syncwarp();
          col_gather<N>(c, zin, Ep, recb + k * RB, nr, gbuf + k * RB * N, lane);
          col_wait_all();
          __syncwarp();
          col_links<N>(recb + k * RB, nr, gbuf + k * RB * N, qs, lane);
        }
        __syncwarp();
        if (lane < C) {  // R = Q + Q^dagger, out = y + ch R; lane (pp, jj) writes part pp of column jj
          const int pp = lane / N, jj = lane - pp * N;
          const double *qp = qs + pp * E;
          const int64_t base = 2 * ((int64_t)u * Ep + jj) + pp;  // element (i, jj), part pp: + 2 N i
          double yr[N];
          if (has_y) {
#pragma unroll
            for (int i = 0; i < N; ++i) yr[i] = yv[base + 2 * N * i];
          }
          const double sg = pp ? -1.0 : 1.0;  // Re R symmetric, Im R antisymmetric
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const double r = fma(sg, qp[jj * N + i], qp[i * N + jj]);
            out[base + 2 * N * i] = has_y ? fma(ch, r, yr[i]) : ch * r;
          }
        }
        __syncwarp();
      }
    }
  }
  col_wait_all();
}

template <int N>
int launch_col(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st, int sm_count) {
  StageArgs<double> a;
  a.c = c;
  a.ch = ch;
  for (int i = 0; i < kMaxStates; ++i) a.term[i] = (i < c.n) ? term[i] : 0.0;
  for (int i = 0; i < kMaxStates * kMaxStates; ++i) {
    a.H[i] = 0.0;
    a.Hi[i] = 0.0;
  }
  for (int i = 0; i < c.n; ++i)
    for (int j = 0; j < c.n; ++j) a.H[i * kMaxStates + j] = H[i * c.n + j];
  constexpr int WARPS = ColShape<N>::WARPS;
  const size_t smem = (size_t)WARPS * ColSmem<N>::total;
  static int per_sm = 0;
  if (per_sm == 0) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(stage_col_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) {
        set_error(std::string("column stage kernel: shared memory attribute: ") + cudaGetErrorString(e));
        return -4;
      }
    }
    int ps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, stage_col_kernel<N>, WARPS * 32, smem);
    if (e != cudaSuccess || ps < 1) {
      set_error(std::string("column stage kernel: occupancy query failed or zero blocks: ") + cudaGetErrorString(e));
      return -4;
    }
    per_sm = ps;
  }
  constexpr int G = ColShape<N>::G;
  const int n_chunks = (c.u_end - c.u_begin + G - 1) / G;
  const int blocks_needed = (n_chunks + WARPS - 1) / WARPS;
  const int grid = std::max(1, std::min(blocks_needed, sched_ctas(per_sm, c.occ_pct) * sm_count));
  stage_col_kernel<N><<<grid, WARPS * 32, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("column stage kernel launch: ") + cudaGetErrorString(e));
    return -4;
  }
  return 0;
}

}  // namespace heom
