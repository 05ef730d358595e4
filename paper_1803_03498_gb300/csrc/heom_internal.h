// Internal declarations shared by the CUDA translation units of libheom (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hierarchy.h"

namespace heom {

constexpr int kMaxStates = 24;
constexpr int kStageWarps = 4;  // warps per CTA of the stage kernel

void set_error(const std::string &msg);

// Per-mode constants, one record per mode l = b * (K + 1) + k, grouped by state on the device.
struct ModeDev {
  int state;      // s_l, the state coupled to the mode's bath
  int pad;
  double c;       // c(b, k), real
  double lamnu;   // lambda_b nu_b for k = 0, else 0
};

// Hierarchy state storage of one RK4 copy: ADOs u < u_split ("head") as FP64 complex, ADOs
// u >= u_split ("body") as complex of the run's storage type.  Every ADO's N x N tile is contiguous
// and row-major: head[u * E + e], body[(u - u_split) * Ep + e] with E = N^2 and Ep = E rounded up so
// that a body tile is a multiple of 16 bytes.
struct StateView {
  double2 *head;
  void *body;
};

// Everything a stage launch needs besides H, passed by value in the kernel parameters.
struct StageCommon {
  StateView zin;        // state the RHS is evaluated on (own tile and neighbour gathers)
  StateView y;          // Horner base y (head == nullptr && body == nullptr: none)
  StateView out;        // result y + ch * L zin (or ch * L zin)
  const int32_t *plusA; // [n_ado][Mp], modes in state order, -1 = no link
  const int32_t *minusA;
  const uint8_t *tupA;  // [n_ado][Mp] n_l
  const double *gsum;   // [n_ado] sum_l n_l gamma_l
  const ModeDev *modes; // [M], ordered by state
  const int *state_mode_off;  // [n + 1] modes of state s: [off[s], off[s+1])
  const double *sp_tab;       // [M][D + 1] up factor  s+_l(n_l)
  const double *sm_tab;       // [M][D + 1] down factor s-_l(n_l)
  int E, Ep, Mp;        // N^2, body tile pitch, padded mode count (multiple of 16)
  int u_split, n_ado;
  int u_begin, u_end;   // ADO range of this launch
  int n, M, D;
  int cplx_h;           // H has an imaginary part
};

template <typename CT>
struct StageArgs {
  StageCommon c;
  CT ch;                      // Horner coefficient times h (1 for a bare RHS evaluation)
  CT term[kMaxStates];        // terminator Delta per state (0 if none)
  CT H[kMaxStates * kMaxStates];   // Re H - h0 I, row stride kMaxStates, rad/fs
  CT Hi[kMaxStates * kMaxStates];  // Im H
};

// Stage launchers, one per storage combination and range of n (stage_*.cu); each returns 0 on
// success, 1 if n is not compiled in that unit, negative on error.
#define HEOM_DECLARE_LAUNCH(NAME)                                                                      \
  int NAME(const StageCommon &c, double ch, const double *term, const double *H, const double *Hi, \
           cudaStream_t st, int sm_count);
HEOM_DECLARE_LAUNCH(launch_stage_fp64_a)
HEOM_DECLARE_LAUNCH(launch_stage_fp64_b)
HEOM_DECLARE_LAUNCH(launch_stage_fp64_c)
HEOM_DECLARE_LAUNCH(launch_stage_fp64_d)
HEOM_DECLARE_LAUNCH(launch_stage_fp32_a)
HEOM_DECLARE_LAUNCH(launch_stage_fp32_b)
HEOM_DECLARE_LAUNCH(launch_stage_fp32_c)
HEOM_DECLARE_LAUNCH(launch_stage_fp32_d)
HEOM_DECLARE_LAUNCH(launch_stage_head_a)
HEOM_DECLARE_LAUNCH(launch_stage_head_b)
HEOM_DECLARE_LAUNCH(launch_stage_head_c)
HEOM_DECLARE_LAUNCH(launch_stage_head_d)
#undef HEOM_DECLARE_LAUNCH

// precision: 0 = FP64 (compute and storage double), 1 = mixed body (float, float), 2 = mixed head
// (compute double, body storage float).
int launch_stage(int precision, const StageCommon &c, double ch, const double *term, const double *H,
                 const double *Hi, cudaStream_t st, int sm_count);

}  // namespace heom
