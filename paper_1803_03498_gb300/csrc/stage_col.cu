// Instantiations of the column-form FP64 stage kernel (Hermitian runs, real H), n_states 8..16.
#include "stage_col.cuh"

namespace heom {

int launch_stage_col(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                     int sm_count) {
  switch (c.n) {
    case 8: return launch_col<8>(c, ch, term, H, st, sm_count);
    case 9: return launch_col<9>(c, ch, term, H, st, sm_count);
    case 10: return launch_col<10>(c, ch, term, H, st, sm_count);
    case 11: return launch_col<11>(c, ch, term, H, st, sm_count);
    case 12: return launch_col<12>(c, ch, term, H, st, sm_count);
    case 13: return launch_col<13>(c, ch, term, H, st, sm_count);
    case 14: return launch_col<14>(c, ch, term, H, st, sm_count);
    case 15: return launch_col<15>(c, ch, term, H, st, sm_count);
    case 16: return launch_col<16>(c, ch, term, H, st, sm_count);
    default:
      return 1;  // not covered: the row-form stage kernel runs
  }
}

}  // namespace heom
