// Instantiations of the general stage kernel (FP64, mixed body, mixed head).
#include "gen_kernel.cuh"

namespace heom {

template <typename CT>
static void fill_gen(GenArgs<CT> &a, const StageCommon &c, StateView base2, StateView out2, double c1, double c2,
                     const double *H, const double *Hi, const double *T) {
  a.c = c;
  a.base2 = base2;
  a.out2 = out2;
  a.c1 = (CT)c1;
  a.c2 = (CT)c2;
  for (int i = 0; i < kGenMaxStates * kGenMaxStates; ++i) a.H[i] = a.Hi[i] = a.T[i] = 0;
  for (int i = 0; i < c.n; ++i)
    for (int j = 0; j < c.n; ++j) {
      a.H[i * kGenMaxStates + j] = (CT)H[i * c.n + j];
      a.Hi[i * kGenMaxStates + j] = Hi ? (CT)Hi[i * c.n + j] : (CT)0;
      a.T[i * kGenMaxStates + j] = (CT)T[i * c.n + j];
    }
}

int launch_stage_gen(int kind, const StageCommon &c, StateView base2, StateView out2, double c1, double c2,
                     const double *H, const double *Hi, const double *T, cudaStream_t st, int sm_count) {
  if (c.n < 1 || c.n > kGenMaxStates) {
    set_error("general stage kernel: n_states above 32");
    return -1;
  }
  if (kind == 1) {
    GenArgs<float> a;
    fill_gen(a, c, base2, out2, c1, c2, H, Hi, T);
    return launch_gen_kind<float, float>(a, st, sm_count);
  }
  GenArgs<double> a;
  fill_gen(a, c, base2, out2, c1, c2, H, Hi, T);
  return kind == 0 ? launch_gen_kind<double, double>(a, st, sm_count) : launch_gen_kind<double, float>(a, st, sm_count);
}

}  // namespace heom
