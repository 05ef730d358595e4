// Instantiations of the work-list stage kernel (FP32 body and FP64 head of mixed runs), n_states 17..24.
#include "stage_list.cuh"

namespace heom {

int launch_stage_list_c(int kind, int n, const ListLaunch &L, cudaStream_t st, int sm_count) {
  switch (n) {
    case 17: return kind == 2 ? launch_list_n<17, double, float>(L, st, sm_count) : launch_list_n<17, float, float>(L, st, sm_count);
    case 18: return kind == 2 ? launch_list_n<18, double, float>(L, st, sm_count) : launch_list_n<18, float, float>(L, st, sm_count);
    case 19: return kind == 2 ? launch_list_n<19, double, float>(L, st, sm_count) : launch_list_n<19, float, float>(L, st, sm_count);
    case 20: return kind == 2 ? launch_list_n<20, double, float>(L, st, sm_count) : launch_list_n<20, float, float>(L, st, sm_count);
    case 21: return kind == 2 ? launch_list_n<21, double, float>(L, st, sm_count) : launch_list_n<21, float, float>(L, st, sm_count);
    case 22: return kind == 2 ? launch_list_n<22, double, float>(L, st, sm_count) : launch_list_n<22, float, float>(L, st, sm_count);
    case 23: return kind == 2 ? launch_list_n<23, double, float>(L, st, sm_count) : launch_list_n<23, float, float>(L, st, sm_count);
    case 24: return kind == 2 ? launch_list_n<24, double, float>(L, st, sm_count) : launch_list_n<24, float, float>(L, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
