// Instantiations of the work-list stage kernel (FP32 body and FP64 head of mixed runs), n_states 9..16.
#include "stage_list.cuh"

namespace heom {

int launch_stage_list_b(int kind, int n, const ListLaunch &L, cudaStream_t st, int sm_count) {
  switch (n) {
    case 9: return kind == 2 ? launch_list_n<9, double, float>(L, st, sm_count) : launch_list_n<9, float, float>(L, st, sm_count);
    case 10: return kind == 2 ? launch_list_n<10, double, float>(L, st, sm_count) : launch_list_n<10, float, float>(L, st, sm_count);
    case 11: return kind == 2 ? launch_list_n<11, double, float>(L, st, sm_count) : launch_list_n<11, float, float>(L, st, sm_count);
    case 12: return kind == 2 ? launch_list_n<12, double, float>(L, st, sm_count) : launch_list_n<12, float, float>(L, st, sm_count);
    case 13: return kind == 2 ? launch_list_n<13, double, float>(L, st, sm_count) : launch_list_n<13, float, float>(L, st, sm_count);
    case 14: return kind == 2 ? launch_list_n<14, double, float>(L, st, sm_count) : launch_list_n<14, float, float>(L, st, sm_count);
    case 15: return kind == 2 ? launch_list_n<15, double, float>(L, st, sm_count) : launch_list_n<15, float, float>(L, st, sm_count);
    case 16: return kind == 2 ? launch_list_n<16, double, float>(L, st, sm_count) : launch_list_n<16, float, float>(L, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
