// Instantiations of the stage kernel: compute double, storage double, n_states 19..24.
#include "stage_kernel.cuh"

namespace heom {

int launch_stage_fp64_d(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi,
                       cudaStream_t st, int sm_count) {
  switch (c.n) {
    case 19: return launch_n<19, double, double>(c, ch, term, H, Hi, st, sm_count);
    case 20: return launch_n<20, double, double>(c, ch, term, H, Hi, st, sm_count);
    case 21: return launch_n<21, double, double>(c, ch, term, H, Hi, st, sm_count);
    case 22: return launch_n<22, double, double>(c, ch, term, H, Hi, st, sm_count);
    case 23: return launch_n<23, double, double>(c, ch, term, H, Hi, st, sm_count);
    case 24: return launch_n<24, double, double>(c, ch, term, H, Hi, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
