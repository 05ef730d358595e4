// The run handle and the helpers that the library's host units share (internal, not part of the ABI):
// run set-up and state I/O (heom_abi.cu), the RK4 driver (propagate.cu), the launch-schedule
// autotuner (tuner.cu), ragged batches (batch.cu) and the small kernels (aux_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/heom.h"
#include "heom_internal.h"

namespace heom {

// 2 pi c in rad/fs per cm^-1 (c = 2.99792458e-5 cm/fs) and k_B in cm^-1/K (2019 SI, exact ratio).
constexpr double kCmToRadFs = 2.0 * 3.14159265358979323846 * 2.99792458e-5;
constexpr double kBoltzCm = 0.6950348004;

// Sets the thread's error message from a failed CUDA call; returns HEOM_E_CUDA.
int cuda_fail(const char *what, cudaError_t e);

__global__ void record_kernel(StateView y, int u_split, int body_fp32, int vec, int n, const double *w, double *records,
                              int64_t *rec_count, int64_t max_records);
__global__ void scatter_kernel(StateView dst, int Ep, int u_split, int body_fp32, int vec, int n, int64_t u0, int64_t count,
                               const double *re, const double *im);
__global__ void gather_kernel(StateView src, int Ep, int u_split, int body_fp32, int vec, int n, int64_t u0, int64_t count,
                              double *re, double *im);

}  // namespace heom

struct heom_hier {
  heom::Hierarchy h;
};

struct heom_run {
  int precision = 0;
  int n = 0, M = 0, D = 0, K = 0, B = 0;
  int64_t n_ado = 0;
  int u_split = 0;                   // ADOs stored in FP64 in the head region
  int E = 0, Ep = 0;                 // tile size, body tile pitch
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;       // library stream for the FP64 head launches (they overlap the body)
  cudaEvent_t fork = nullptr, join = nullptr;
  int sm_count = 0;
  // host copies of the per-run constants (rad/fs)
  std::vector<double> H, Hi;         // shifted Re H, Im H
  bool cplx_h = false;
  bool herm = false;                 // every ADO Hermitian (Hermitian H and data; paper gauge)
  bool vec = false;                  // every ADO in the coherence block |a><0|: stored as its column 0
  bool gen = false;                  // general stage kernel (bath masks, laser field, > 24 states)
  std::vector<double> T;             // [n][n] terminator rate of each element (general kernel)
  bool has_field = false;            // laser field set (heom_run_set_field): classic four-copy RK4
  std::vector<double> mup;           // [n][n] M+
  double famp = 0, ftc = 0, fsig = 1, fphase = 0, fdet = 0;  // rad/fs, fs, fs, rad, rad/fs
  std::vector<double> Ht, Hit;       // H(t) of the current stage (general kernel)
  size_t copy_bytes = 0;             // bytes of one state copy (head + body, matrix layout)
  double bytes_full_y = 0, bytes_full_noy = 0, flops_full = 0;  // matrix-layout accounting
  heom::VecRunDesc *desc_dev = nullptr;    // [8] stage arguments for batched column-0 launches, or a
                                           // GroupRunDesc for work-list launches (heom_group_propagate)
  const void *desc_owner = nullptr;  // the batch whose stage arguments desc_dev holds (or the work-list tag)
  double desc_dt = 0;                // time step of the work-list stage arguments in desc_dev
  std::vector<double> term;          // per state
  double max_rate = 0;               // D * max gamma
  // device
  heom::StateView y{}, zA{}, zB{}, zC{};   // zC: RK4 accumulator of time-dependent runs
  int64_t *link_off = nullptr;       // [n_ado + 1]
  void *recs_head = nullptr;         // LinkRec<double>, ADOs u < u_split
  void *recs_body = nullptr;         // LinkRec<float or double>, ADOs u >= u_split
  int64_t rec_split = 0;             // link_off[u_split]
  int64_t n_links = 0;               // link_off[n_ado]: link records in all
  double *gsum = nullptr;
  double *records = nullptr;         // [max_records][n + 5]
  double *w_dev = nullptr;           // [n] dipole weights (zeros if none)
  int64_t *rec_count = nullptr;      // device counter of records written
  int *err_dev = nullptr;            // device flag set by a bounded device-side wait that gave up
  int64_t max_records = 0;
  int64_t records_host = 0;          // records enqueued so far (host view)
  int64_t steps_done = 0;
  double t_fs = 0;
  int64_t launches = 0;
  heom_schedule sched[2] = {{100, 1}, {100, 1}};  // launch schedules: [0] body, [1] FP64 head
  // timing of the dominant kernel
  bool timing = false;
  bool pending = false;              // a begin event was recorded for the current launch
  std::vector<cudaEvent_t> ev;       // pairs
  double timed_bytes = 0, timed_flops = 0;
  double bytes_stage_y = 0, bytes_stage_noy = 0;  // per launch over the body range
  double flops_gen = 0, flops_herm = 0;             // per launch: general and Hermitian forms
  ~heom_run() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
  }
};

namespace heom {

// run set-up and state I/O (heom_abi.cu)
// One observable record of sigma_0 on the run's stream.  host_check = false skips the host-side
// count check (graph capture: heom_batch_launch checks the counts per replay); the kernel keeps
// the run's real max_records as its bound either way.
int enqueue_record(heom_run *r, bool host_check = true);
int io_range(heom_run *r, StateView state, int64_t u0, int64_t count, double *re, double *im, bool to_device);

// the RK4 driver (propagate.cu)
StageCommon common_for(const heom_run *r, StateView zin, StateView y, StateView out);
int launch_head(heom_run *r, StageCommon c, double ch, cudaStream_t s);  // FP64 head launch of a stage
int launch_body(heom_run *r, StageCommon c, double ch, cudaStream_t s);  // body launch of a stage
int run_stage(heom_run *r, StateView zin, StateView y, StateView out, double ch);
void field_H(heom_run *r, double t);  // H(t) of a run with a laser field into r->Ht, r->Hit

// the launch-schedule autotuner (tuner.cu)
extern std::atomic<int> g_autotune;  // timed launches per candidate at creation (0: off)
int ilog2(int64_t x);
std::vector<heom_schedule> candidates(int layout);
bool cache_get(const std::array<int, 7> &k, heom_schedule *out);
void cache_put(const std::array<int, 7> &k, const heom_schedule &s);
heom_schedule default_for(int layout);
int schedule_new_run(heom_run *r);  // cache, else tuner (if on), else default, per part
void reschedule_cached(heom_run *r);

// Times probe(schedule) for every candidate (one warm-up, reps timed launches each, on stream s);
// returns the index of the fastest in *best.
template <typename Probe>
int time_candidates(const std::vector<heom_schedule> &cand, int reps, cudaStream_t s, Probe probe,
                    std::vector<double> &ms, int *best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int rc = HEOM_OK;
  ms.assign(cand.size(), 0.0);
  *best = 0;
  for (size_t i = 0; i < cand.size() && e == cudaSuccess && rc == HEOM_OK; ++i) {
    if ((rc = probe(cand[i]))) break;
    e = cudaEventRecord(e0, s);
    for (int k = 0; k < reps && e == cudaSuccess && rc == HEOM_OK; ++k) rc = probe(cand[i]);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    ms[i] = (double)t / reps;
    if (ms[i] < ms[*best]) *best = (int)i;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != HEOM_OK) return rc;
  return e == cudaSuccess ? HEOM_OK : cuda_fail("autotune timing", e);
}

}  // namespace heom
