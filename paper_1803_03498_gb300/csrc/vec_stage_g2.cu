// Instantiations of the coherence-block (column-0) stage kernels, n_states 2..24, with 2 chunk(s)
// per warp step.
#include "vec_kernel.cuh"

namespace heom {

int launch_stage_vec_g2(int kind, const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                        int sm_count) {
  if (c.u_end <= c.u_begin) return 0;
  return vec_dispatch<2>(kind, c, ch, term, H, st, sm_count);
}

int launch_stage_vec_batch_g2(int kind, int n, const VecBatchArgs &a, cudaStream_t st, int sm_count) {
  if (a.nruns <= 0) return 0;
  return vec_batch_dispatch<2>(kind, n, a, st, sm_count);
}

}  // namespace heom
