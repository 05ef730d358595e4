// Instantiations of the work-list stage kernel (FP32 body and FP64 head of mixed runs), n_states 1..8.
#include "stage_list.cuh"

namespace heom {

int launch_stage_list_a(int kind, int n, const ListLaunch &L, cudaStream_t st, int sm_count) {
  switch (n) {
    case 1: return kind == 2 ? launch_list_n<1, double, float>(L, st, sm_count) : launch_list_n<1, float, float>(L, st, sm_count);
    case 2: return kind == 2 ? launch_list_n<2, double, float>(L, st, sm_count) : launch_list_n<2, float, float>(L, st, sm_count);
    case 3: return kind == 2 ? launch_list_n<3, double, float>(L, st, sm_count) : launch_list_n<3, float, float>(L, st, sm_count);
    case 4: return kind == 2 ? launch_list_n<4, double, float>(L, st, sm_count) : launch_list_n<4, float, float>(L, st, sm_count);
    case 5: return kind == 2 ? launch_list_n<5, double, float>(L, st, sm_count) : launch_list_n<5, float, float>(L, st, sm_count);
    case 6: return kind == 2 ? launch_list_n<6, double, float>(L, st, sm_count) : launch_list_n<6, float, float>(L, st, sm_count);
    case 7: return kind == 2 ? launch_list_n<7, double, float>(L, st, sm_count) : launch_list_n<7, float, float>(L, st, sm_count);
    case 8: return kind == 2 ? launch_list_n<8, double, float>(L, st, sm_count) : launch_list_n<8, float, float>(L, st, sm_count);
    default:
      return 1;  // not in this translation unit
  }
}

}  // namespace heom
