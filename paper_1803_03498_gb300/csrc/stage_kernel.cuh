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
// V^o = (delta_is + delta_sj) applied element by element (on the diagonal the up terms and the
// c parts cancel, the lamnu parts add).
//
// Mapping: a warp holds floor(32 / n) ADOs and lane (a, i) computes output row i of ADO a, in
// blocks of JB columns.  A CTA stages the tiles of a chunk of consecutive ADOs in shared memory,
// element-major with the ADO index fastest ([e][g]): the lanes of one ADO read the same word
// (broadcast), lanes of different ADOs read consecutive words.  H lives in the kernel parameters
// (constant bank) and the fully unrolled loops address it with compile-time offsets.  Neighbour
// elements are gathered from global memory: with the level-ordered colex numbering the "-"
// neighbours of consecutive ADOs are consecutive, and the element-major store keeps those
// gathers contiguous.  Results go to a second shared buffer and are combined with y and stored
// with coalesced accesses.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

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

template <typename CT, typename BT>
__device__ __forceinline__ typename Cplx<CT>::type load_state(const StateView &s, int64_t hp, int64_t bp,
                                                            int u_split, int e, int v) {
  using C2 = typename Cplx<CT>::type;
  using B2 = typename Cplx<BT>::type;
  C2 r;
  if (v < u_split) {
    const double2 d = s.head[(int64_t)e * hp + v];
    r.x = (CT)d.x;
    r.y = (CT)d.y;
  } else {
    const B2 b = reinterpret_cast<const B2 *>(s.body)[(int64_t)e * bp + (v - u_split)];
    r.x = (CT)b.x;
    r.y = (CT)b.y;
  }
  return r;
}

template <typename CT, typename BT>
__device__ __forceinline__ void store_state(const StateView &s, int64_t hp, int64_t bp, int u_split, int e, int v,
                                            CT re, CT im) {
  using B2 = typename Cplx<BT>::type;
  if (v < u_split) {
    s.head[(int64_t)e * hp + v] = make_double2((double)re, (double)im);
  } else {
    B2 b;
    b.x = (BT)re;
    b.y = (BT)im;
    reinterpret_cast<B2 *>(s.body)[(int64_t)e * bp + (v - u_split)] = b;
  }
}

template <int NM>
struct StageShape {
  static constexpr bool kRowInRegs = NM <= 16;  // keep own row and H row in registers
  static constexpr int JB = NM <= 16 ? NM : 8;  // columns per block
};

template <int NM, typename CT, typename BT>
__global__ void __launch_bounds__(kStageWarps * 32) stage_kernel(const __grid_constant__ StageArgs<CT> a) {
  using C2 = typename Cplx<CT>::type;
  constexpr bool RR = StageShape<NM>::kRowInRegs;
  constexpr int JB = StageShape<NM>::JB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StageCommon &c = a.c;
  const int n = c.n;
  const int A = 32 / n;           // ADOs per warp
  const int G = A * kStageWarps;  // ADOs per chunk
  const int GP = G + 1;           // padded element stride in shared memory
  const int E = n * n;
  const int M = c.M, D1 = c.D + 1;
  C2 *tile = reinterpret_cast<C2 *>(smem_raw);
  C2 *obuf = tile + (size_t)E * GP;
  CT *sp_s = reinterpret_cast<CT *>(obuf + (size_t)E * GP);
  CT *sm_s = sp_s + M * D1;
  CT *cc_s = sm_s + M * D1;
  CT *ln_s = cc_s + M;
  int *smo_s = reinterpret_cast<int *>(ln_s + M);  // [n + 1]

  for (int t = threadIdx.x; t < M * D1; t += blockDim.x) {
    sp_s[t] = (CT)c.sp_tab[t];
    sm_s[t] = (CT)c.sm_tab[t];
  }
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    cc_s[t] = (CT)c.modes[t].c;
    ln_s[t] = (CT)c.modes[t].lamnu;
  }
  for (int t = threadIdx.x; t <= n; t += blockDim.x) smo_s[t] = c.state_mode_off[t];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int la = lane / n;
  const int li = lane - la * n;
  const bool lane_ok = la < A;
  const int g = warp * A + la;
  const bool has_y = (c.y.head != nullptr) || (c.y.body != nullptr);
  const CT term_i = lane_ok ? a.term[li] : (CT)0;

  CT Hrow[RR ? NM : 1];
  if (RR) {
#pragma unroll
    for (int k = 0; k < (RR ? NM : 1); ++k) Hrow[k] = (k < n && lane_ok) ? a.H[li * kMaxStates + k] : (CT)0;
  }
  __syncthreads();

  const int n_chunks = (c.u_end - c.u_begin + G - 1) / G;
  int chunk = blockIdx.x;
  // stage the first chunk's tiles: element-major, coalesced over consecutive ADOs
  if (chunk < n_chunks) {
    const int u0 = c.u_begin + chunk * G;
    const int cnt = min(G, c.u_end - u0);
    for (int t = threadIdx.x; t < E * G; t += blockDim.x) {
      const int e = t / G, gg = t - e * G;
      if (gg < cnt) tile[e * GP + gg] = load_state<CT, BT>(c.zin, c.head_pitch, c.body_pitch, c.u_split, e, u0 + gg);
    }
  }
  __syncthreads();
  for (; chunk < n_chunks; chunk += gridDim.x) {
    const int u0 = c.u_begin + chunk * G;
    const int cnt = min(G, c.u_end - u0);
    if (lane_ok && g < cnt) {
      const int u = u0 + g;
      const CT gs = (CT)c.gsum[u];
      C2 zr[RR ? NM : 1];
      if (RR) {
#pragma unroll
        for (int k = 0; k < (RR ? NM : 1); ++k) {
          if (k < n) zr[k] = tile[(li * n + k) * GP + g];
          else { zr[k].x = 0; zr[k].y = 0; }
        }
      }
#pragma unroll
      for (int jb = 0; jb < NM; jb += JB) {
        CT rr[JB], ri[JB];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) { rr[jj] = 0; ri[jj] = 0; }
        // rhs = -i (H s - s H):  (H s) part
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          if (k < n) {
            const CT h = RR ? Hrow[RR ? k : 0] : a.H[li * kMaxStates + k];
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) {
              const int j = jb + jj;
              if (j < n) {
                const C2 z = tile[(k * n + j) * GP + g];
                rr[jj] = fma(h, z.y, rr[jj]);
                ri[jj] = fma(-h, z.x, ri[jj]);
              }
            }
          }
        }
        // (s H) part, H_kj from the constant bank
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          if (k < n) {
            const C2 zk = RR ? zr[RR ? k : 0] : tile[(li * n + k) * GP + g];
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) {
              const int j = jb + jj;
              if (j < n) {
                const CT h = a.H[k * kMaxStates + j];
                rr[jj] = fma(-zk.y, h, rr[jj]);
                ri[jj] = fma(zk.x, h, ri[jj]);
              }
            }
          }
        }
        if (c.cplx_h) {  // imaginary part of H
#pragma unroll
          for (int k = 0; k < NM; ++k) {
            if (k < n) {
              const CT h = a.Hi[li * kMaxStates + k];
              const C2 zk = tile[(li * n + k) * GP + g];
#pragma unroll
              for (int jj = 0; jj < JB; ++jj) {
                const int j = jb + jj;
                if (j < n) {
                  const C2 z = tile[(k * n + j) * GP + g];
                  rr[jj] = fma(h, z.x, rr[jj]);
                  ri[jj] = fma(h, z.y, ri[jj]);
                  const CT h2 = a.Hi[k * kMaxStates + j];
                  rr[jj] = fma(-zk.x, h2, rr[jj]);
                  ri[jj] = fma(-zk.y, h2, ri[jj]);
                }
              }
            }
          }
        }
        // decay and terminator
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          const int j = jb + jj;
          if (j < n) {
            const C2 zij = RR ? zr[RR ? j : 0] : tile[(li * n + j) * GP + g];
            const CT f = gs + ((j != li) ? (term_i + a.term[j]) : (CT)0);
            rr[jj] = fma(-f, zij.x, rr[jj]);
            ri[jj] = fma(-f, zij.y, ri[jj]);
          }
        }
        // modes of state li: row li of the neighbours
        for (int q = smo_s[li]; q < smo_s[li + 1]; ++q) {
          const int nl = c.tupT[(int64_t)q * c.u_pitch + u];
          const int vp = c.plusT[(int64_t)q * c.u_pitch + u];
          const int vm = c.minusT[(int64_t)q * c.u_pitch + u];
          if (vp >= 0) {
            const CT sp = sp_s[q * D1 + nl];
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) {
              const int j = jb + jj;
              if (j < n && j != li) {  // + i s+ s^+_ij
                const C2 v = load_state<CT, BT>(c.zin, c.head_pitch, c.body_pitch, c.u_split, li * n + j, vp);
                rr[jj] = fma(-sp, v.y, rr[jj]);
                ri[jj] = fma(sp, v.x, ri[jj]);
              }
            }
          }
          if (vm >= 0) {
            const CT sm = sm_s[q * D1 + nl];
            const CT scc = sm * cc_s[q], sln = sm * ln_s[q];
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) {
              const int j = jb + jj;
              if (j < n) {
                const C2 v = load_state<CT, BT>(c.zin, c.head_pitch, c.body_pitch, c.u_split, li * n + j, vm);
                if (j != li) {  // s- (i c + lamnu) s^-_ij
                  rr[jj] = fma(sln, v.x, fma(-scc, v.y, rr[jj]));
                  ri[jj] = fma(sln, v.y, fma(scc, v.x, ri[jj]));
                } else {  // diagonal: 2 s- lamnu s^-_ii
                  rr[jj] = fma(2 * sln, v.x, rr[jj]);
                  ri[jj] = fma(2 * sln, v.y, ri[jj]);
                }
              }
            }
          }
        }
        // modes of the column states j != li: element (li, j) of the neighbours
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          const int j = jb + jj;
          if (j < n && j != li) {
            for (int q = smo_s[j]; q < smo_s[j + 1]; ++q) {
              const int nl = c.tupT[(int64_t)q * c.u_pitch + u];
              const int vp = c.plusT[(int64_t)q * c.u_pitch + u];
              const int vm = c.minusT[(int64_t)q * c.u_pitch + u];
              if (vp >= 0) {  // - i s+ s^+_ij
                const CT sp = sp_s[q * D1 + nl];
                const C2 v = load_state<CT, BT>(c.zin, c.head_pitch, c.body_pitch, c.u_split, li * n + j, vp);
                rr[jj] = fma(sp, v.y, rr[jj]);
                ri[jj] = fma(-sp, v.x, ri[jj]);
              }
              if (vm >= 0) {  // s- (-i c + lamnu) s^-_ij
                const CT sm = sm_s[q * D1 + nl];
                const CT scc = sm * cc_s[q], sln = sm * ln_s[q];
                const C2 v = load_state<CT, BT>(c.zin, c.head_pitch, c.body_pitch, c.u_split, li * n + j, vm);
                rr[jj] = fma(sln, v.x, fma(scc, v.y, rr[jj]));
                ri[jj] = fma(sln, v.y, fma(-scc, v.x, ri[jj]));
              }
            }
          }
        }
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          const int j = jb + jj;
          if (j < n) {
            C2 w;
            w.x = a.ch * rr[jj];
            w.y = a.ch * ri[jj];
            obuf[(li * n + j) * GP + g] = w;
          }
        }
      }
    }
    __syncthreads();  // obuf complete; every lane is done with tile
    // combine with y and store this chunk; stage the next chunk's tiles
    for (int t = threadIdx.x; t < E * G; t += blockDim.x) {
      const int e = t / G, gg = t - e * G;
      if (gg < cnt) {
        C2 w = obuf[e * GP + gg];
        if (has_y) {
          const C2 yv = load_state<CT, BT>(c.y, c.head_pitch, c.body_pitch, c.u_split, e, u0 + gg);
          w.x += yv.x;
          w.y += yv.y;
        }
        store_state<CT, BT>(c.out, c.head_pitch, c.body_pitch, c.u_split, e, u0 + gg, w.x, w.y);
      }
    }
    const int nxt = chunk + gridDim.x;
    if (nxt < n_chunks) {
      const int v0 = c.u_begin + nxt * G;
      const int vcnt = min(G, c.u_end - v0);
      for (int t = threadIdx.x; t < E * G; t += blockDim.x) {
        const int e = t / G, gg = t - e * G;
        if (gg < vcnt) tile[e * GP + gg] = load_state<CT, BT>(c.zin, c.head_pitch, c.body_pitch, c.u_split, e, v0 + gg);
      }
    }
    __syncthreads();
  }
}

inline size_t stage_smem_bytes_t(size_t cs, int n, int M, int D) {
  const int A = 32 / n, G = A * kStageWarps, GP = G + 1;
  size_t b = 2 * (size_t)n * n * GP * 2 * cs;     // tile + obuf
  b += (size_t)(2 * M * (D + 1) + 2 * M) * cs;  // sp, sm, c, lamnu
  b += (size_t)(n + 1) * sizeof(int);
  return (b + 15) & ~(size_t)15;
}

template <int NM, typename CT, typename BT>
int launch_nm(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi,
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
  const size_t smem = stage_smem_bytes_t(sizeof(CT), c.n, c.M, c.D);
  // per-instantiation cache of the occupancy for the last shared-memory size
  static size_t cached_smem = 0;
  static int cached_per_sm = 0;
  if (smem != cached_smem) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(stage_kernel<NM, CT, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) {
        set_error(std::string("stage kernel: shared memory attribute: ") + cudaGetErrorString(e));
        return -4;
      }
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel<NM, CT, BT>,
                                                                  kStageWarps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) {
      set_error(std::string("stage kernel: occupancy query failed or zero blocks: ") + cudaGetErrorString(e));
      return -4;
    }
    cached_smem = smem;
    cached_per_sm = per_sm;
  }
  const int G = (32 / c.n) * kStageWarps;
  const int n_chunks = (c.u_end - c.u_begin + G - 1) / G;
  const int grid = std::max(1, std::min(n_chunks, cached_per_sm * sm_count));
  stage_kernel<NM, CT, BT><<<grid, kStageWarps * 32, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("stage kernel launch: ") + cudaGetErrorString(e));
    return -4;
  }
  return 0;
}

// Register-array sizes compiled; a run uses the smallest one >= n.
constexpr int kNmList[] = {2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 18, 20, 24};

inline int nm_for(int n) {
  for (int v : kNmList)
    if (n <= v) return v;
  return -1;
}

}  // namespace heom
