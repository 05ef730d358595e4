// Internal declarations shared by the CUDA translation units of libheom (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hierarchy.h"

namespace heom {

constexpr int kMaxStates = 24;

void set_error(const std::string &msg);

// Device error word of a run (StageCommon::err): bit 0 -- a bounded device-side wait gave up (the
// tensor-core kernel); bit 1 -- a bounds check of the debug build failed.  heom_observables reports
// them as HEOM_E_TIMEOUT and HEOM_E_BOUNDS.
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;

// Debug build (compiled with -DHEOM_DEBUG): every neighbour index a link record names, its coupled
// state and every record range a stage kernel reads are checked before use; an index outside its
// range sets kErrBounds in the run's error word and the access is skipped.  Without HEOM_DEBUG the
// check is the constant true and costs nothing.
#ifdef HEOM_DEBUG
__device__ __forceinline__ bool heom_in_range(int *err, int64_t idx, int64_t lo, int64_t hi) {
  if (idx >= lo && idx < hi) return true;
  if (err) atomicOr(err, kErrBounds);
  return false;
}
#define HEOM_IN_RANGE(err, idx, lo, hi) heom_in_range((err), (int64_t)(idx), (int64_t)(lo), (int64_t)(hi))
#else
#define HEOM_IN_RANGE(err, idx, lo, hi) true
#endif

// A batch of nr link records starting at record lo, read from a region that holds records
// [rbase, limit): nr, or 0 (and kErrBounds) when the debug build finds the batch outside the region.
__device__ __forceinline__ int heom_rec_batch(int *err, int64_t lo, int nr, int64_t rbase, int64_t limit) {
#ifdef HEOM_DEBUG
  if (lo < rbase || nr < 0 || lo + nr > limit) {
    if (err) atomicOr(err, kErrBounds);
    return 0;
  }
#endif
  return nr;
}

// One link of an ADO u to a neighbour v = n(u) +- e_l through a mode l of state s.  Only row s and
// column s of v contribute to row s and column s of d sigma_u / dt: element (s, j != s) with
// coefficient R, element (i != s, s) with conj(R), element (s, s) with 2 Re R, where
//   up link (v = n + e_l):    R = i s+_l(n_l)            (s+ = sqrt((n_l + 1) |c_l|), or 1)
//   down link (v = n - e_l):  R = s-_l(n_l) (lamnu_l + i c_l)   (s- = sqrt(n_l / |c_l|), or n_l)
// (V^x contributes +1 on row s and -1 on column s, V^o +1 on both, 2 on the diagonal).
// The records of one ADO are ordered by s.  Field s holds the state in bits 0..7 and the owning
// ADO's index u mod 32 in bits 8..12, so that a warp working on ADOs u0 .. u0 + 31 finds the owner
// of a record as ((s >> 8) - u0) mod 32 without a search.
constexpr int kRecStateMask = 0xff;
template <typename T>
struct LinkRec;
template <>
struct alignas(16) LinkRec<float> {
  int v, s;
  float re, im;
};
template <>
struct alignas(16) LinkRec<double> {
  int v, s, pad0, pad1;
  double re, im;
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
  const int64_t *link_off;  // [n_ado + 1] first link record of each ADO
  const void *recs_head;    // LinkRec<double> of ADOs u < u_split, indexed by link_off[u]
  const void *recs_body;    // LinkRec<body compute type> of ADOs u >= u_split, by link_off[u] - rec_split
  int64_t rec_split;        // link_off[u_split]
  const double *gsum;       // [n_ado] sum_l n_l gamma_l
  int E, Ep;                // N^2 and the body tile pitch (E rounded up to 16-byte tiles)
  int u_split, n_ado;
  int u_begin, u_end;   // ADO range of this launch
  int n;
  int cplx_h;           // H has an imaginary part
  int herm;             // every ADO is Hermitian: gather row s only, and s H = (H s)^dagger
  int *err;             // device error word (kErrTimeout, kErrBounds)
  int64_t n_recs;       // link records in all (link_off[n_ado]); the debug build checks ranges against it
  int occ_pct;          // schedule: grid sized for this percentage of the CTAs that fit on an SM
  int cpw;              // schedule: column-0 kernels' chunks per warp step (1, 2, 4)
};

// Nonzero while heom_propagate_static creates its run: the autotuner stays off there.
extern thread_local int g_tune_suppress;

// Chunks of floor(32 / n) ADOs that a column-0 warp step holds for a schedule's chunks per warp g:
// g, capped so that a step holds at most 32 ADOs (a link record names its ADO by u mod 32).
__host__ __device__ constexpr int vec_group(int n, int g) { return g < 32 / (32 / n) ? g : 32 / (32 / n); }

// CTAs per SM of the grid for a schedule's occupancy percentage (at least 1): up to 100 a persistent
// grid filling that share of each SM's CTA slots; above 100 that many percent of one resident wave,
// so that CTAs retire while the launch runs.
inline int sched_ctas(int per_sm, int occ_pct) {
  const int b = occ_pct <= 0 ? per_sm : per_sm * occ_pct / 100;
  return b < 1 ? 1 : b;
}

// Coherence-block (column-0) stage kernels (vec_stage_g{1,2,4}.cu, one unit per chunks-per-warp
// value): kind 0 FP64, 1 mixed body (FP32), 2 mixed head (FP64 compute, FP32 body neighbours).
// launch_stage_vec picks the unit from c.cpw.
int launch_stage_vec(int kind, const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                     int sm_count);
#define HEOM_DECLARE_VEC(R)                                                                                 \
  int launch_stage_vec_g##R(int kind, const StageCommon &c, double ch, const double *term, const double *H, \
                            cudaStream_t st, int sm_count);
HEOM_DECLARE_VEC(1)
HEOM_DECLARE_VEC(2)
HEOM_DECLARE_VEC(4)
#undef HEOM_DECLARE_VEC

// Stage arguments of one run for the batched column-0 kernel; lives in the run's workspace.
struct VecRunDesc {
  StageCommon c;
  double ch;
  double H[kMaxStates * kMaxStates];  // row-major, stride kMaxStates (shifted H, rad/fs)
  double term[kMaxStates];
};
constexpr int kBatchMaxRuns = 1024;   // runs per batched launch (kernel-parameter space)
struct VecBatchArgs {
  const VecRunDesc *d[kBatchMaxRuns];
  int64_t chunk0[kBatchMaxRuns + 1];  // prefix sums of the runs' warp-step counts (for cpw)
  int nruns;
  int occ_pct, cpw;                   // schedule of the launch (the runs' own schedules do not apply)
};
// One launch of the batched column-0 kernel for runs of n states (kind as launch_stage_vec).
int launch_stage_vec_batch(int kind, int n, const VecBatchArgs &a, cudaStream_t st, int sm_count);
int launch_stage_vec_batch_g1(int kind, int n, const VecBatchArgs &a, cudaStream_t st, int sm_count);
int launch_stage_vec_batch_g2(int kind, int n, const VecBatchArgs &a, cudaStream_t st, int sm_count);
int launch_stage_vec_batch_g4(int kind, int n, const VecBatchArgs &a, cudaStream_t st, int sm_count);

// Tensor-core (split-TF32) form of the FP32 body stage: Hermitian runs with real H and N <= 16.
// Returns 1 when it does not cover n_states.
int launch_stage_tc_a(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                      int sm_count);
int launch_stage_tc_b(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                      int sm_count);

template <typename CT>
struct StageArgs {
  StageCommon c;
  CT ch;                      // Horner coefficient times h (1 for a bare RHS evaluation)
  CT term[kMaxStates];        // terminator Delta per state (0 if none)
  alignas(16) CT H[kMaxStates * kMaxStates];   // Re H - h0 I, row stride kMaxStates, rad/fs (pairs load as 8 bytes)
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

// General stage kernel (gen_kernel.cuh): bath couplings with several states, a time-dependent H and
// up to kGenMaxStates states.  out1 (c.out) = base1 (c.y) + c1 L zin; out2 = base2 + c2 L zin when
// out2 is set.  H, Hi, T: host arrays [n][n] (H(t) - h0 and Im H(t) in rad/fs; T_ij the terminator
// rate of element (i, j)).  kind as launch_stage_vec.
constexpr int kGenMaxStates = 32;
template <typename CT>
struct GenArgs {
  StageCommon c;
  StateView base2, out2;
  CT c1, c2;
  CT H[kGenMaxStates * kGenMaxStates];
  CT Hi[kGenMaxStates * kGenMaxStates];
  CT T[kGenMaxStates * kGenMaxStates];
};
int launch_stage_gen(int kind, const StageCommon &c, StateView base2, StateView out2, double c1, double c2,
                     const double *H, const double *Hi, const double *T, cudaStream_t st, int sm_count);

// Column-form FP64 stage kernel (stage_col.cuh) for Hermitian runs with a real H and 8 <= n <= 16:
// every lane of a warp owns one column of one part of an ADO's result, so all 32 lanes do FP64 work.
// Returns 1 when it does not cover n.
int launch_stage_col(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                     int sm_count);

// Work-list launches (stage_list.cuh): one launch covers the same stage of many runs of equal
// n_states (real H).  A run's stage arguments for such launches live in its workspace.
template <typename CT>
struct alignas(16) GroupArgs {
  StageCommon c;
  CT ch;                           // Horner coefficient times h
  CT term[kMaxStates];             // terminator Delta per state
  alignas(16) CT H[kMaxStates * kMaxStates];   // Re H - h0 I, row stride kMaxStates, rad/fs
};
// Per run: the four Horner stages of the FP32 body and of the FP64 head (mixed precision).
struct GroupRunDesc {
  GroupArgs<float> body[4];
  GroupArgs<double> head[4];
};
constexpr int kListMaxRuns = 64;  // runs per work-list launch (kernel parameters: about 0.8 KB)
struct ListLaunch {
  const void *args[kListMaxRuns];  // GroupArgs of run i for this stage and part (device)
  int item0[kListMaxRuns + 1];     // run i owns items [item0[i], item0[i + 1]) of cpi chunks each
  int nruns;
  int cpi;
};
// One work-list launch of runs of n states: kind 1 = mixed body (FP32), 2 = mixed head (FP64 compute,
// FP32 body neighbours).  Returns 1 when n is not compiled in the unit.
int launch_stage_list(int kind, int n, const ListLaunch &L, cudaStream_t st, int sm_count);
int launch_stage_list_a(int kind, int n, const ListLaunch &L, cudaStream_t st, int sm_count);
int launch_stage_list_b(int kind, int n, const ListLaunch &L, cudaStream_t st, int sm_count);
int launch_stage_list_c(int kind, int n, const ListLaunch &L, cudaStream_t st, int sm_count);

// precision: 0 = FP64 (compute and storage double), 1 = mixed body (float, float), 2 = mixed head
// (compute double, body storage float).
int launch_stage(int precision, const StageCommon &c, double ch, const double *term, const double *H,
                 const double *Hi, cudaStream_t st, int sm_count);

}  // namespace heom
