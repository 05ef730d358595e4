// Instantiations of the stage kernel: compute float, storage float, n_states in {13, 14, 15, 16, 18, 20, 24}.
#include "stage_kernel.cuh"

namespace heom {

int launch_stage_fp32_hi(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi,
                        cudaStream_t st, int sm_count) {
  switch (nm_for(c.n)) {
    case 13: return launch_nm<13, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 14: return launch_nm<14, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 15: return launch_nm<15, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 16: return launch_nm<16, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 18: return launch_nm<18, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 20: return launch_nm<20, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 24: return launch_nm<24, float, float>(c, ch, term, H, Hi, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
