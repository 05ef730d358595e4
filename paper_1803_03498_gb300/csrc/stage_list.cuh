// Work-list form of the row stage kernel (sm_103a): one launch evaluates the same RK4 stage for many
// runs of equal n_states -- the ragged hierarchies of concurrent requests -- instead of one launch per
// run.  The launch's work list is the concatenation of the runs' chunk ranges: run i owns items
// [item0[i], item0[i+1]), each item cpi chunks of floor(32 / N) consecutive ADOs of that run.  A CTA
// takes items in turn: it finds the item's run by binary search, stages the run's stage arguments
// (H, terminator, Horner coefficient, pointers: GroupArgs, kept in the run's workspace) in shared
// memory, and its warps cover the item's chunks with the same per-chunk code as stage_kernel
// (stage_chunks), so every ADO gets the same arithmetic in the same order as a launch of its own.
// Runs with a real H only (the H of a run enters from shared memory, not the constant bank).
#pragma once
#include "stage_kernel.cuh"

namespace heom {

template <int N, typename CT, typename BT>
__global__ void __launch_bounds__(StageShape<N, CT, BT>::WARPS * 32) stage_list_kernel(const __grid_constant__ ListLaunch L) {
  using S = StageShape<N, CT, BT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ GroupArgs<CT> ga;
  static_assert(sizeof(GroupArgs<CT>) % 16 == 0, "16-byte copies");
  const int items = L.item0[L.nruns];
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    int lo = 0, hi = L.nruns;  // the run i with item0[i] <= it < item0[i + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (L.item0[mid] <= it) lo = mid;
      else hi = mid;
    }
    __syncthreads();  // every warp is done with the previous item's arguments
    {
      const int4 *src = reinterpret_cast<const int4 *>(L.args[lo]);
      int4 *dst = reinterpret_cast<int4 *>(&ga);
      for (int t = threadIdx.x; t < (int)(sizeof(GroupArgs<CT>) / 16); t += blockDim.x) dst[t] = src[t];
    }
    __syncthreads();
    const int n_chunks = (ga.c.u_end - ga.c.u_begin + S::A - 1) / S::A;
    const int c0 = (it - L.item0[lo]) * L.cpi;
    stage_chunks<N, CT, BT, false>(ga, smem_raw, c0 + (int)(threadIdx.x >> 5), S::WARPS, min(n_chunks, c0 + L.cpi));
  }
}

template <int N, typename CT, typename BT>
int launch_list_n(const ListLaunch &L, cudaStream_t st, int sm_count) {
  constexpr int WARPS = StageShape<N, CT, BT>::WARPS;
  const size_t smem = (size_t)WARPS * WarpSmem<N, CT, BT>::total;
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(stage_list_kernel<N, CT, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    int ps = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, stage_list_kernel<N, CT, BT>, WARPS * 32, smem);
    if (e != cudaSuccess || ps < 1) {
      set_error(std::string("work-list stage kernel: attributes / occupancy: ") + cudaGetErrorString(e));
      return -4;
    }
    per_sm = ps;
  }
  const int items = L.item0[L.nruns];
  if (items <= 0) return 0;
  const int grid = std::max(1, std::min(items, per_sm * sm_count));
  stage_list_kernel<N, CT, BT><<<grid, WARPS * 32, smem, st>>>(L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("work-list stage kernel launch: ") + cudaGetErrorString(e));
    return -4;
  }
  return 0;
}

}  // namespace heom
