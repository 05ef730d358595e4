// Instantiations of the stage kernel: compute float, storage float, n_states in {2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12}.
#include "stage_kernel.cuh"

namespace heom {

int launch_stage_fp32_lo(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi,
                        cudaStream_t st, int sm_count) {
  switch (nm_for(c.n)) {
    case 2: return launch_nm<2, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 3: return launch_nm<3, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 4: return launch_nm<4, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 5: return launch_nm<5, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 6: return launch_nm<6, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 7: return launch_nm<7, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 8: return launch_nm<8, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 9: return launch_nm<9, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 10: return launch_nm<10, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 11: return launch_nm<11, float, float>(c, ch, term, H, Hi, st, sm_count);
    case 12: return launch_nm<12, float, float>(c, ch, term, H, Hi, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
