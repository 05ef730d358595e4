// Instantiations of the split-TF32 tensor-core stage kernel: n_states 1..8.
#include "stage_tc.cuh"

namespace heom {

int launch_stage_tc_a(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                      int sm_count) {
  switch (c.n) {
    case 1: return launch_tc<1>(c, ch, term, H, st, sm_count);
    case 2: return launch_tc<2>(c, ch, term, H, st, sm_count);
    case 3: return launch_tc<3>(c, ch, term, H, st, sm_count);
    case 4: return launch_tc<4>(c, ch, term, H, st, sm_count);
    case 5: return launch_tc<5>(c, ch, term, H, st, sm_count);
    case 6: return launch_tc<6>(c, ch, term, H, st, sm_count);
    case 7: return launch_tc<7>(c, ch, term, H, st, sm_count);
    case 8: return launch_tc<8>(c, ch, term, H, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
