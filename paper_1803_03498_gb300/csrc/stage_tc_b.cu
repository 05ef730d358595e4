// Instantiations of the split-TF32 tensor-core stage kernel: n_states 9..16.
#include "stage_tc.cuh"

namespace heom {

int launch_stage_tc_b(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                      int sm_count) {
  switch (c.n) {
    case 9: return launch_tc<9>(c, ch, term, H, st, sm_count);
    case 10: return launch_tc<10>(c, ch, term, H, st, sm_count);
    case 11: return launch_tc<11>(c, ch, term, H, st, sm_count);
    case 12: return launch_tc<12>(c, ch, term, H, st, sm_count);
    case 13: return launch_tc<13>(c, ch, term, H, st, sm_count);
    case 14: return launch_tc<14>(c, ch, term, H, st, sm_count);
    case 15: return launch_tc<15>(c, ch, term, H, st, sm_count);
    case 16: return launch_tc<16>(c, ch, term, H, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
