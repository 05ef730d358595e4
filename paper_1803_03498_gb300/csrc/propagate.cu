// C ABI of libheom, part 2: the RK4 driver.  Stage launches (head, body, general kernel), the laser
// field's H(t), Horner and classic RK4 steps, kernel timing, observables and one RHS evaluation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/heom.h"
#include "heom_internal.h"
#include "heom_run.h"

using namespace heom;

// ------------------------------------------------------------------------------------------------
// propagation: classic RK4 of a linear, time-independent right-hand side, evaluated in Horner form
//   y_{t+h} = y + h L (y + h/2 L (y + h/3 L (y + h/4 L y)))
// which is the same degree-4 polynomial as the four-stage classic tableau and needs three state
// copies (y, zA, zB) instead of four.

StageCommon heom::common_for(const heom_run *r, StateView zin, StateView y, StateView out) {
  StageCommon c{};
  c.zin = zin;
  c.y = y;
  c.out = out;
  c.link_off = r->link_off;
  c.recs_head = r->recs_head;
  c.recs_body = r->recs_body;
  c.rec_split = r->rec_split;
  c.gsum = r->gsum;
  c.E = r->E;
  c.Ep = r->Ep;
  c.u_split = r->u_split;
  c.n_ado = (int)r->n_ado;
  c.n = r->n;
  c.cplx_h = r->cplx_h ? 1 : 0;
  c.herm = r->herm ? 1 : 0;
  c.err = r->err_dev;
  c.n_recs = r->n_links;
  return c;
}

static int timed_begin(heom_run *r) {
  r->pending = false;
  if (!r->timing || r->ev.size() >= 2 * 65536) return HEOM_OK;
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) return cuda_fail("timing event", e);
  r->ev.push_back(a);
  r->ev.push_back(b);
  e = cudaEventRecord(a, r->stream);
  if (e != cudaSuccess) return cuda_fail("timing event record", e);
  r->pending = true;
  return HEOM_OK;
}

static int timed_end(heom_run *r, double bytes) {
  if (!r->pending) return HEOM_OK;
  r->pending = false;
  cudaError_t e = cudaEventRecord(r->ev.back(), r->stream);
  if (e != cudaSuccess) return cuda_fail("timing event record", e);
  r->timed_bytes += bytes;
  r->timed_flops += r->herm ? r->flops_herm : r->flops_gen;
  return HEOM_OK;
}

// The FP64 head launch of a mixed-precision stage goes to the run's side stream, forked from and
// joined back into the run's stream (capturable), so that it overlaps the body launch: both read zin
// and write disjoint parts of out.
static cudaStream_t fork_head(heom_run *r) {
  if (!r->side) return r->stream;
  if (cudaEventRecord(r->fork, r->stream) != cudaSuccess || cudaStreamWaitEvent(r->side, r->fork, 0) != cudaSuccess)
    return r->stream;
  return r->side;
}
static int join_head(heom_run *r, cudaStream_t hs) {
  if (hs == r->stream) return HEOM_OK;
  cudaError_t e = cudaEventRecord(r->join, hs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(r->stream, r->join, 0);
  return e == cudaSuccess ? HEOM_OK : cuda_fail("head stream join", e);
}

// The FP64 head launch (ADOs u < u_split) of a mixed-precision stage, on stream s.
int heom::launch_head(heom_run *r, StageCommon c, double ch, cudaStream_t s) {
  c.u_begin = 0;
  c.u_end = r->u_split;
  c.occ_pct = r->sched[1].occupancy_pct;
  c.cpw = r->sched[1].chunks_per_warp;
  const double *Hi = r->cplx_h ? r->Hi.data() : nullptr;
  const int rc = r->vec ? launch_stage_vec(2, c, ch, r->term.data(), r->H.data(), s, r->sm_count)
                        : launch_stage(2, c, ch, r->term.data(), r->H.data(), Hi, s, r->sm_count);
  if (rc) return HEOM_E_CUDA;
  ++r->launches;
  return HEOM_OK;
}

// The body launch of a stage (every ADO for FP64, u >= u_split otherwise), on stream s.
int heom::launch_body(heom_run *r, StageCommon c, double ch, cudaStream_t s) {
  c.u_begin = (r->precision == HEOM_FP64) ? 0 : r->u_split;
  c.u_end = (int)r->n_ado;
  if (c.u_end <= c.u_begin) return HEOM_OK;
  c.occ_pct = r->sched[0].occupancy_pct;
  c.cpw = r->sched[0].chunks_per_warp;
  const double *Hi = r->cplx_h ? r->Hi.data() : nullptr;
  const bool fp64 = r->precision == HEOM_FP64;
  int rc = 1;
  if (r->vec) {
    rc = launch_stage_vec(fp64 ? 0 : 1, c, ch, r->term.data(), r->H.data(), s, r->sm_count);
  } else if (fp64) {
    rc = launch_stage(0, c, ch, r->term.data(), r->H.data(), Hi, s, r->sm_count);
  } else {
    if (r->precision == HEOM_SPLIT_TF32 && r->herm && !r->cplx_h) {  // tensor-core commutator
      rc = launch_stage_tc_a(c, ch, r->term.data(), r->H.data(), s, r->sm_count);
      if (rc == 1) rc = launch_stage_tc_b(c, ch, r->term.data(), r->H.data(), s, r->sm_count);
    }
    if (rc == 1) rc = launch_stage(1, c, ch, r->term.data(), r->H.data(), Hi, s, r->sm_count);
  }
  if (rc) return HEOM_E_CUDA;
  ++r->launches;
  return HEOM_OK;
}

// H(t) of a run with a laser field (Eq. h-field-rwa in the rotating frame):
// H - g M+ - conj(g) (M+)^T, g = amp exp(-(t - t_c)^2 / (2 sigma^2)) exp(-i (Delta t + phi)).
void heom::field_H(heom_run *r, double t) {
  const int n = r->n;
  const double x = (t - r->ftc) / r->fsig;
  const double env = r->famp * std::exp(-0.5 * x * x);
  const double ph = r->fdet * t + r->fphase;
  const double gr = env * std::cos(ph), gi = -env * std::sin(ph);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double a = r->mup[(size_t)i * n + j], b = r->mup[(size_t)j * n + i];
      r->Ht[(size_t)i * n + j] = r->H[(size_t)i * n + j] - gr * (a + b);
      r->Hit[(size_t)i * n + j] = r->Hi[(size_t)i * n + j] - gi * a + gi * b;
    }
}

// One stage on the general kernel: out1 = base1 + c1 L zin and, if out2 is set, out2 = base2 + c2 L zin,
// with H(t) from r->Ht (field) or the constant H.
static int run_stage_gen(heom_run *r, StateView zin, StateView b1, StateView o1, double c1, StateView b2, StateView o2,
                         double c2) {
  StageCommon c = common_for(r, zin, b1, o1);
  const double *H = r->has_field ? r->Ht.data() : r->H.data();
  const double *Hi = r->has_field ? r->Hit.data() : r->Hi.data();
  const bool fp64 = r->precision == HEOM_FP64;
  cudaStream_t hs = r->stream;
  int rc;
  if (!fp64) {  // FP64 head (levels 0, 1) on the side stream
    hs = fork_head(r);
    StageCommon ch = c;
    ch.u_begin = 0;
    ch.u_end = r->u_split;
    ch.occ_pct = r->sched[1].occupancy_pct;
    if (launch_stage_gen(2, ch, b2, o2, c1, c2, H, Hi, r->T.data(), hs, r->sm_count)) return HEOM_E_CUDA;
    ++r->launches;
  }
  c.u_begin = fp64 ? 0 : r->u_split;
  c.u_end = (int)r->n_ado;
  c.occ_pct = r->sched[0].occupancy_pct;
  if (c.u_end > c.u_begin) {
    if ((rc = timed_begin(r))) return rc;
    if (launch_stage_gen(fp64 ? 0 : 1, c, b2, o2, c1, c2, H, Hi, r->T.data(), r->stream, r->sm_count))
      return HEOM_E_CUDA;
    ++r->launches;
    if ((rc = timed_end(r, r->bytes_stage_y))) return rc;
  }
  return join_head(r, hs);
}

int heom::run_stage(heom_run *r, StateView zin, StateView y, StateView out, double ch) {
  if (r->gen) return run_stage_gen(r, zin, y, out, ch, StateView{nullptr, nullptr}, StateView{nullptr, nullptr}, 0.0);
  const StageCommon c = common_for(r, zin, y, out);
  const bool same_y = (y.head == zin.head && y.body == zin.body);
  const bool no_y = (y.head == nullptr && y.body == nullptr);
  int rc;
  cudaStream_t hs = r->stream;
  if (r->precision != HEOM_FP64) {  // FP64 head (levels 0, 1) on the side stream
    hs = fork_head(r);
    if ((rc = launch_head(r, c, ch, hs))) return rc;
  }
  if ((int)r->n_ado > ((r->precision == HEOM_FP64) ? 0 : r->u_split)) {
    if ((rc = timed_begin(r))) return rc;
    if ((rc = launch_body(r, c, ch, r->stream))) return rc;
    if ((rc = timed_end(r, (same_y || no_y) ? r->bytes_stage_noy : r->bytes_stage_y))) return rc;
  }
  return join_head(r, hs);
}


extern "C" int heom_run_set_timing(heom_run *r, int enable) {
  if (!r) { set_error("heom_run_set_timing: NULL run"); return HEOM_E_ARG; }
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail("heom_run_set_timing: stream", e);
  for (cudaEvent_t ev : r->ev) cudaEventDestroy(ev);
  r->ev.clear();
  r->timed_bytes = r->timed_flops = 0;
  r->timing = enable != 0;
  return HEOM_OK;
}

extern "C" int heom_run_kernel_time(heom_run *r, double *ms, int64_t *launches, double *alg_bytes, double *alg_flops) {
  if (!r) { set_error("heom_run_kernel_time: NULL run"); return HEOM_E_ARG; }
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail("heom_run_kernel_time: stream", e);
  double tot = 0;
  for (size_t i = 0; i + 1 < r->ev.size(); i += 2) {
    float t = 0;
    e = cudaEventElapsedTime(&t, r->ev[i], r->ev[i + 1]);
    if (e != cudaSuccess) return cuda_fail("heom_run_kernel_time: elapsed", e);
    tot += t;
  }
  if (ms) *ms = tot;
  if (launches) *launches = (int64_t)(r->ev.size() / 2);
  if (alg_bytes) *alg_bytes = r->timed_bytes;
  if (alg_flops) *alg_flops = r->timed_flops;
  return HEOM_OK;
}

extern "C" int heom_propagate(heom_run *r, double dt_fs, int64_t n_steps, int64_t obs_stride) {
  if (!r) { set_error("heom_propagate: NULL run"); return HEOM_E_ARG; }
  if (!(dt_fs > 0) || n_steps < 0 || obs_stride < 0) {
    set_error("heom_propagate: need dt_fs > 0, n_steps >= 0, obs_stride >= 0");
    return HEOM_E_ARG;
  }
  if (dt_fs * r->max_rate > 2.5) {
    set_error("heom_propagate: dt_fs * depth * max gamma > 2.5 (RK4 unstable; the paper asks dt << 1/gamma_k)");
    return HEOM_E_ARG;
  }
  if (obs_stride > 0) {
    const int64_t first = obs_stride - (r->steps_done % obs_stride);
    const int64_t need = (n_steps >= first) ? 1 + (n_steps - first) / obs_stride : 0;
    if (r->records_host + need > r->max_records) {
      set_error("heom_propagate: observable records would exceed max_records");
      return HEOM_E_NOMEM;
    }
  }
  const double h = dt_fs;
  StateView none{nullptr, nullptr};
  if (r->has_field) {
    // classic four-copy RK4 of the time-dependent L(t): k_s = L(t_s) X_s, X_{s+1} = y + a h k_s,
    // acc (zC) = y + h (k1 + 2 k2 + 2 k3) / 6, y = acc + h k4 / 6
    const double t0 = r->t_fs;
    for (int64_t s = 0; s < n_steps; ++s) {
      const double t = t0 + (double)s * h;
      int rc;
      field_H(r, t);
      if ((rc = run_stage_gen(r, r->y, r->y, r->zA, h / 2, r->y, r->zC, h / 6))) return rc;
      field_H(r, t + h / 2);
      if ((rc = run_stage_gen(r, r->zA, r->y, r->zB, h / 2, r->zC, r->zC, h / 3))) return rc;
      if ((rc = run_stage_gen(r, r->zB, r->y, r->zA, h, r->zC, r->zC, h / 3))) return rc;
      field_H(r, t + h);
      if ((rc = run_stage_gen(r, r->zA, r->zC, r->y, h / 6, none, none, 0.0))) return rc;
      ++r->steps_done;
      r->t_fs = t0 + (double)(s + 1) * h;
      if (obs_stride > 0 && r->steps_done % obs_stride == 0)
        if ((rc = enqueue_record(r))) return rc;
    }
    return HEOM_OK;
  }
  for (int64_t s = 0; s < n_steps; ++s) {
    int rc;
    if ((rc = run_stage(r, r->y, r->y, r->zA, h / 4))) return rc;
    if ((rc = run_stage(r, r->zA, r->y, r->zB, h / 3))) return rc;
    if ((rc = run_stage(r, r->zB, r->y, r->zA, h / 2))) return rc;
    if ((rc = run_stage(r, r->zA, r->y, r->y, h))) return rc;
    ++r->steps_done;
    r->t_fs += h;
    if (obs_stride > 0 && r->steps_done % obs_stride == 0)
      if ((rc = enqueue_record(r))) return rc;
  }
  return HEOM_OK;
}

extern "C" int heom_observables(heom_run *r, double *out, int64_t cap_records, int64_t *written) {
  if (!r || !out || cap_records < 0) { set_error("heom_observables: bad arguments"); return HEOM_E_ARG; }
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail("heom_observables: stream", e);
  int64_t cnt_err[2] = {0, 0};
  e = cudaMemcpy(cnt_err, r->rec_count, sizeof(cnt_err), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("heom_observables: counter", e);
  int err_flag = 0;
  std::memcpy(&err_flag, &cnt_err[1], sizeof(int));
  if (err_flag & kErrBounds) {
    set_error("heom_observables: a bounds check of the debug build failed (a link record names an ADO, state or "
              "record range outside the run; its results are invalid)");
    return HEOM_E_BOUNDS;
  }
  if (err_flag) {
    set_error("heom_observables: a device-side wait of the tensor-core stage kernel gave up (its results are invalid)");
    return HEOM_E_TIMEOUT;
  }
  int64_t cnt = cnt_err[0];
  cnt = std::min(cnt, cap_records);
  const int rl = r->n + 5;
  if (cnt > 0) {
    e = cudaMemcpy(out, r->records, (size_t)cnt * rl * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail("heom_observables: copy", e);
  }
  if (written) *written = cnt;
  for (int64_t i = 0; i < cnt * rl; ++i)
    if (!std::isfinite(out[i])) {
      set_error("heom_observables: NaN/Inf in the root ADO");
      return HEOM_E_NUMERIC;
    }
  return HEOM_OK;
}


extern "C" int heom_rhs_eval(heom_run *r, int64_t u0, int64_t count, double *re, double *im) {
  if (!r) { set_error("heom_rhs_eval: NULL run"); return HEOM_E_ARG; }
  StateView none{nullptr, nullptr};
  if (r->has_field) field_H(r, r->t_fs);  // L at the current time
  int rc = run_stage(r, r->y, none, r->zA, 1.0);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail("heom_rhs_eval: stream", e);
  return io_range(r, r->zA, u0, count, re, im, false);
}
