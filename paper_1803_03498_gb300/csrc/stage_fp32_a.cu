// Instantiations of the stage kernel: compute float, storage float, n_states 1..6.
#include "stage_kernel.cuh"

namespace heom {

int launch_stage_fp32_a(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi,
                       cudaStream_t st, int sm_count) {
  switch (c.n) {
    case 1: return launch_n<1, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 2: return launch_n<2, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 3: return launch_n<3, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 4: return launch_n<4, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 5: return launch_n<5, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 6: return launch_n<6, float, float>(c, ch, term, H, Hi, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
