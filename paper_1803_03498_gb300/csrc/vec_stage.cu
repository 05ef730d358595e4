// Instantiations of the coherence-block (vector) stage kernel, n_states 2..24.
#include "vec_kernel.cuh"

namespace heom {

// kind 0: FP64 (double, double); 1: mixed body (float, float); 2: mixed head (double, float).
int launch_stage_vec(int kind, const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                     int sm_count) {
  if (c.u_end <= c.u_begin) return 0;
  switch (c.n) {
    case 2:
      return kind == 0 ? launch_vec_n<2, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<2, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<2, double, float>(c, ch, term, H, st, sm_count);
    case 3:
      return kind == 0 ? launch_vec_n<3, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<3, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<3, double, float>(c, ch, term, H, st, sm_count);
    case 4:
      return kind == 0 ? launch_vec_n<4, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<4, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<4, double, float>(c, ch, term, H, st, sm_count);
    case 5:
      return kind == 0 ? launch_vec_n<5, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<5, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<5, double, float>(c, ch, term, H, st, sm_count);
    case 6:
      return kind == 0 ? launch_vec_n<6, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<6, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<6, double, float>(c, ch, term, H, st, sm_count);
    case 7:
      return kind == 0 ? launch_vec_n<7, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<7, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<7, double, float>(c, ch, term, H, st, sm_count);
    case 8:
      return kind == 0 ? launch_vec_n<8, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<8, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<8, double, float>(c, ch, term, H, st, sm_count);
    case 9:
      return kind == 0 ? launch_vec_n<9, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<9, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<9, double, float>(c, ch, term, H, st, sm_count);
    case 10:
      return kind == 0 ? launch_vec_n<10, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<10, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<10, double, float>(c, ch, term, H, st, sm_count);
    case 11:
      return kind == 0 ? launch_vec_n<11, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<11, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<11, double, float>(c, ch, term, H, st, sm_count);
    case 12:
      return kind == 0 ? launch_vec_n<12, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<12, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<12, double, float>(c, ch, term, H, st, sm_count);
    case 13:
      return kind == 0 ? launch_vec_n<13, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<13, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<13, double, float>(c, ch, term, H, st, sm_count);
    case 14:
      return kind == 0 ? launch_vec_n<14, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<14, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<14, double, float>(c, ch, term, H, st, sm_count);
    case 15:
      return kind == 0 ? launch_vec_n<15, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<15, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<15, double, float>(c, ch, term, H, st, sm_count);
    case 16:
      return kind == 0 ? launch_vec_n<16, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<16, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<16, double, float>(c, ch, term, H, st, sm_count);
    case 17:
      return kind == 0 ? launch_vec_n<17, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<17, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<17, double, float>(c, ch, term, H, st, sm_count);
    case 18:
      return kind == 0 ? launch_vec_n<18, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<18, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<18, double, float>(c, ch, term, H, st, sm_count);
    case 19:
      return kind == 0 ? launch_vec_n<19, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<19, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<19, double, float>(c, ch, term, H, st, sm_count);
    case 20:
      return kind == 0 ? launch_vec_n<20, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<20, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<20, double, float>(c, ch, term, H, st, sm_count);
    case 21:
      return kind == 0 ? launch_vec_n<21, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<21, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<21, double, float>(c, ch, term, H, st, sm_count);
    case 22:
      return kind == 0 ? launch_vec_n<22, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<22, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<22, double, float>(c, ch, term, H, st, sm_count);
    case 23:
      return kind == 0 ? launch_vec_n<23, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<23, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<23, double, float>(c, ch, term, H, st, sm_count);
    case 24:
      return kind == 0 ? launch_vec_n<24, double, double>(c, ch, term, H, st, sm_count)
           : kind == 1 ? launch_vec_n<24, float, float>(c, ch, term, H, st, sm_count)
                       : launch_vec_n<24, double, float>(c, ch, term, H, st, sm_count);
    default:
      set_error("vector stage kernel: n_states not compiled");
      return -1;
  }
}

int launch_stage_vec_batch(int kind, int n, const VecBatchArgs &a, cudaStream_t st, int sm_count) {
  if (a.nruns <= 0) return 0;
  switch (n) {
    case 2:
      return kind == 0 ? launch_vec_batch_n<2, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<2, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<2, double, float>(a, st, sm_count);
    case 3:
      return kind == 0 ? launch_vec_batch_n<3, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<3, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<3, double, float>(a, st, sm_count);
    case 4:
      return kind == 0 ? launch_vec_batch_n<4, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<4, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<4, double, float>(a, st, sm_count);
    case 5:
      return kind == 0 ? launch_vec_batch_n<5, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<5, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<5, double, float>(a, st, sm_count);
    case 6:
      return kind == 0 ? launch_vec_batch_n<6, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<6, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<6, double, float>(a, st, sm_count);
    case 7:
      return kind == 0 ? launch_vec_batch_n<7, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<7, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<7, double, float>(a, st, sm_count);
    case 8:
      return kind == 0 ? launch_vec_batch_n<8, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<8, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<8, double, float>(a, st, sm_count);
    case 9:
      return kind == 0 ? launch_vec_batch_n<9, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<9, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<9, double, float>(a, st, sm_count);
    case 10:
      return kind == 0 ? launch_vec_batch_n<10, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<10, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<10, double, float>(a, st, sm_count);
    case 11:
      return kind == 0 ? launch_vec_batch_n<11, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<11, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<11, double, float>(a, st, sm_count);
    case 12:
      return kind == 0 ? launch_vec_batch_n<12, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<12, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<12, double, float>(a, st, sm_count);
    case 13:
      return kind == 0 ? launch_vec_batch_n<13, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<13, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<13, double, float>(a, st, sm_count);
    case 14:
      return kind == 0 ? launch_vec_batch_n<14, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<14, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<14, double, float>(a, st, sm_count);
    case 15:
      return kind == 0 ? launch_vec_batch_n<15, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<15, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<15, double, float>(a, st, sm_count);
    case 16:
      return kind == 0 ? launch_vec_batch_n<16, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<16, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<16, double, float>(a, st, sm_count);
    case 17:
      return kind == 0 ? launch_vec_batch_n<17, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<17, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<17, double, float>(a, st, sm_count);
    case 18:
      return kind == 0 ? launch_vec_batch_n<18, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<18, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<18, double, float>(a, st, sm_count);
    case 19:
      return kind == 0 ? launch_vec_batch_n<19, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<19, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<19, double, float>(a, st, sm_count);
    case 20:
      return kind == 0 ? launch_vec_batch_n<20, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<20, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<20, double, float>(a, st, sm_count);
    case 21:
      return kind == 0 ? launch_vec_batch_n<21, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<21, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<21, double, float>(a, st, sm_count);
    case 22:
      return kind == 0 ? launch_vec_batch_n<22, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<22, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<22, double, float>(a, st, sm_count);
    case 23:
      return kind == 0 ? launch_vec_batch_n<23, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<23, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<23, double, float>(a, st, sm_count);
    case 24:
      return kind == 0 ? launch_vec_batch_n<24, double, double>(a, st, sm_count)
           : kind == 1 ? launch_vec_batch_n<24, float, float>(a, st, sm_count)
                       : launch_vec_batch_n<24, double, float>(a, st, sm_count);
    default:
      set_error("batched vector kernel: n_states not compiled");
      return -1;
  }
}

}  // namespace heom
