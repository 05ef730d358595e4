// Instantiations of the stage kernel: compute double, storage float, n_states 7..12.
#include "stage_kernel.cuh"

namespace heom {

int launch_stage_head_b(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi,
                       cudaStream_t st, int sm_count) {
  switch (c.n) {
    case 7: return launch_n<7, double, float>(c, ch, term, H, Hi, st, sm_count);
    case 8: return launch_n<8, double, float>(c, ch, term, H, Hi, st, sm_count);
    case 9: return launch_n<9, double, float>(c, ch, term, H, Hi, st, sm_count);
    case 10: return launch_n<10, double, float>(c, ch, term, H, Hi, st, sm_count);
    case 11: return launch_n<11, double, float>(c, ch, term, H, Hi, st, sm_count);
    case 12: return launch_n<12, double, float>(c, ch, term, H, Hi, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
