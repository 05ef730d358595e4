// Instantiations of the stage kernel: compute float, storage float, n_states 13..18.
#include "stage_kernel.cuh"

namespace heom {

int launch_stage_fp32_c(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi,
                       cudaStream_t st, int sm_count) {
  switch (c.n) {
    case 13: return launch_n<13, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 14: return launch_n<14, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 15: return launch_n<15, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 16: return launch_n<16, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 17: return launch_n<17, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 18: return launch_n<18, float, float>(c, ch, term, H, Hi, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
