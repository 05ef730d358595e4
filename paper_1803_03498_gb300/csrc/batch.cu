// C ABI of libheom, part 4: ragged batches (heom_batch_*): many runs in one CUDA graph, small
// column-0 runs of equal n_states grouped into one launch per stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/heom.h"
#include "heom_internal.h"
#include "heom_run.h"

using namespace heom;

// ------------------------------------------------------------------------------------------------
// runs with more ADOs than this launch per run inside a batch even in the column-0 layout
static const int64_t kBatchGroupMaxAdos = 50000;

// ragged batches: the stage launches of many runs, each on one of a pool of streams, captured into
// one CUDA graph that advances every run by steps_per_launch RK4 steps per replay.

// A schedule for a batched column-0 launch over runs of n states with the given ADO counts: the
// prefix sums of the runs' warp steps (vec_group(n, cpw) chunks of floor(32 / n) ADOs each).
static void set_batch_schedule(VecBatchArgs &x, const std::vector<int64_t> &ados, int n, const heom_schedule &sc) {
  const int64_t sa = (int64_t)vec_group(n, sc.chunks_per_warp) * (32 / n);
  x.chunk0[0] = 0;
  for (size_t q = 0; q < ados.size(); ++q) x.chunk0[q + 1] = x.chunk0[q] + (ados[q] + sa - 1) / sa;
  x.occ_pct = sc.occupancy_pct;
  x.cpw = sc.chunks_per_warp;
}

struct heom_batch {
  std::vector<heom_run *> runs;
  std::vector<cudaStream_t> pool;
  std::vector<cudaEvent_t> ev;  // fork/join events of the capture, then per-launch join events
  cudaStream_t origin = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double dt = 0;
  int64_t steps_per_launch = 0, obs_stride = 0;
  std::vector<int64_t> launches_per_replay;
  // groups of column-0 runs advanced by batched launches: per group its runs, n_states, FP64 or
  // mixed kernels, stream, and the launch arguments of the 4 stages x {FP64 head, body}
  std::vector<std::vector<int>> gruns;
  std::vector<int> gn;
  std::vector<bool> gfp64;
  std::vector<cudaStream_t> gstream;
  std::vector<std::vector<VecBatchArgs>> gargs;
  std::vector<std::array<heom_schedule, 2>> gsched;  // per group: [0] body, [1] FP64 head
  std::vector<std::array<std::vector<int64_t>, 2>> gados;  // per group and part: each run's ADO count
  ~heom_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaStream_t s : pool) cudaStreamDestroy(s);
    if (origin) cudaStreamDestroy(origin);
  }
};

extern "C" int heom_batch_create(heom_run *const *runs, int n_runs, double dt_fs, int64_t steps_per_launch,
                                 int64_t obs_stride, heom_batch **out) {
  if (!out || !runs || n_runs < 1 || !(dt_fs > 0) || steps_per_launch < 1 || obs_stride < 0 ||
      (obs_stride > 0 && steps_per_launch % obs_stride != 0)) {
    set_error("heom_batch_create: need runs, n_runs >= 1, dt_fs > 0, steps_per_launch >= 1, "
              "obs_stride >= 0 dividing steps_per_launch");
    return HEOM_E_ARG;
  }
  *out = nullptr;
  for (int i = 0; i < n_runs; ++i) {
    if (!runs[i]) { set_error("heom_batch_create: NULL run"); return HEOM_E_ARG; }
    if (dt_fs * runs[i]->max_rate > 2.5) {
      set_error("heom_batch_create: dt_fs * depth * max gamma > 2.5 for a run (RK4 unstable)");
      return HEOM_E_ARG;
    }
    if (runs[i]->timing) { set_error("heom_batch_create: switch timing off on every run first"); return HEOM_E_STATE; }
    if (runs[i]->has_field) {
      set_error("heom_batch_create: a run with a laser field cannot be batched (its graph would replay fixed times)");
      return HEOM_E_ARG;
    }
  }
  heom_batch *b = new (std::nothrow) heom_batch;
  if (!b) { set_error("host allocation failed"); return HEOM_E_NOMEM; }
  b->runs.assign(runs, runs + n_runs);
  b->dt = dt_fs;
  b->steps_per_launch = steps_per_launch;
  b->obs_stride = obs_stride;
  const int P = std::min(n_runs, 32);
  // the graph is captured on (and later launched on) a stream of its own: the runs' streams may be
  // the legacy default stream, which cannot be captured
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete b; return cuda_fail("heom_batch_create: origin stream", e); }
  for (int p = 0; p < P && e == cudaSuccess; ++p) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->pool.push_back(s);
  }
  for (int k = 0; k < P + 1 && e == cudaSuccess; ++k) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev.push_back(ev);
  }
  if (e != cudaSuccess) { delete b; return cuda_fail("heom_batch_create: streams/events", e); }
  const double h = dt_fs;
  // small runs in the column-0 layout: grouped by (n_states, kernel kind); each group advances every stage
  // of all its runs with one batched launch per part (FP64 head, body), stage arguments in the runs'
  // workspaces
  std::vector<std::vector<int>> groups;
  std::vector<bool> grouped(n_runs, false);
  for (int i = 0; i < n_runs; ++i) {
    heom_run *r = b->runs[i];
    // small runs only: their per-run launches are launch-bound; large runs keep their own launches
    // (kernel-bound, concurrent on the stream pool)
    if (!r->vec || r->n_ado > kBatchGroupMaxAdos) continue;
    bool placed = false;
    for (auto &gv : groups) {
      heom_run *q = b->runs[gv[0]];
      if (q->n == r->n && (q->precision == HEOM_FP64) == (r->precision == HEOM_FP64) && gv.size() < (size_t)kBatchMaxRuns) {
        gv.push_back(i);
        placed = true;
        break;
      }
    }
    if (!placed) groups.push_back({i});
    grouped[i] = true;
  }
  int gi = 0;
  for (const auto &gv : groups) {
    cudaStream_t gs = b->pool[gi++ % P];
    const bool fp64 = b->runs[gv[0]]->precision == HEOM_FP64;
    const int n = b->runs[gv[0]]->n;
    std::vector<VecBatchArgs> ba(8);
    std::array<std::vector<int64_t>, 2> ados;
    for (int k = 0; k < 8; ++k) ba[k].nruns = (int)gv.size();
    for (size_t q = 0; q < gv.size(); ++q) {
      heom_run *r = b->runs[gv[q]];
      std::vector<VecRunDesc> hd(8);
      const StateView zins[4] = {r->y, r->zA, r->zB, r->zA}, outs[4] = {r->zA, r->zB, r->zA, r->y};
      const double chs[4] = {h / 4, h / 3, h / 2, h};
      for (int st = 0; st < 4; ++st)
        for (int part = 0; part < 2; ++part) {
          VecRunDesc &d = hd[st * 2 + part];
          std::memset(&d, 0, sizeof(d));
          d.c = common_for(r, zins[st], r->y, outs[st]);
          d.c.u_begin = (part == 0 || fp64) ? 0 : r->u_split;
          d.c.u_end = (part == 0 && !fp64) ? r->u_split : (int)r->n_ado;
          if (part == 0 && fp64) d.c.u_end = 0;  // FP64 runs: one part
          d.ch = chs[st];
          for (int a = 0; a < r->n; ++a)
            for (int c2 = 0; c2 < r->n; ++c2) d.H[a * kMaxStates + c2] = r->H[a * r->n + c2];
          for (int a = 0; a < r->n; ++a) d.term[a] = r->term[a];
          ba[st * 2 + part].d[q] = r->desc_dev + st * 2 + part;
          if (st == 0) ados[part == 0 ? 1 : 0].push_back(std::max(0, d.c.u_end - d.c.u_begin));
        }
      cudaError_t ec = cudaMemcpy(r->desc_dev, hd.data(), 8 * sizeof(VecRunDesc), cudaMemcpyHostToDevice);
      if (ec != cudaSuccess) { delete b; return cuda_fail("heom_batch_create: stage arguments", ec); }
      r->desc_owner = b;
    }
    b->gargs.push_back(std::move(ba));
    b->gados.push_back(std::move(ados));
    b->gstream.push_back(gs);
    b->gfp64.push_back(fp64);
    b->gn.push_back(n);
    b->gruns.push_back(gv);
  }
  // wait for everything already enqueued on the runs' own streams, then capture
  for (heom_run *r : b->runs) {
    e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) { delete b; return cuda_fail("heom_batch_create: run stream", e); }
  }
  // launch schedules of the grouped launches: the cache, else the tuner (if on; probes are stage-1
  // launches, which write only zA), else the default
  const int reps = g_autotune.load();
  for (size_t g = 0; g < b->gruns.size(); ++g) {
    std::array<heom_schedule, 2> gs{default_for(2), default_for(2)};
    for (int part = 0; part < (b->gfp64[g] ? 1 : 2); ++part) {
      int64_t cnt = 0;
      for (int i : b->gruns[g]) {
        const heom_run *r = b->runs[i];
        cnt += part == 1 ? r->u_split : r->n_ado - (b->gfp64[g] ? 0 : r->u_split);
      }
      const std::array<int, 7> key{2, b->gfp64[g] ? 0 : 1, part, b->gn[g], 0, 0, ilog2(cnt)};
      if (cache_get(key, &gs[part]) || reps <= 0) continue;
      const int kind = part == 1 ? 2 : (b->gfp64[g] ? 0 : 1);
      VecBatchArgs &probe = b->gargs[g][part == 1 ? 0 : 1];  // stage 1 (zin = y, out = zA) of that part
      const std::vector<heom_schedule> cand = candidates(2);
      std::vector<double> ms;
      int best = 0;
      const int rc2 = time_candidates(cand, reps, b->gstream[g], [&](const heom_schedule &sc) {
        set_batch_schedule(probe, b->gados[g][part], b->gn[g], sc);
        return launch_stage_vec_batch(kind, b->gn[g], probe, b->gstream[g], b->runs[0]->sm_count) ? HEOM_E_CUDA
                                                                                                 : HEOM_OK;
      }, ms, &best);
      if (rc2 != HEOM_OK) { delete b; return rc2; }
      gs[part] = cand[best];
      cache_put(key, gs[part]);
    }
    for (int k = 0; k < 8; ++k) {  // argument sets st * 2 + {0: head, 1: body}
      const int part = k % 2 == 0 ? 1 : 0;
      set_batch_schedule(b->gargs[g][k], b->gados[g][part], b->gn[g], gs[part]);
    }
    b->gsched.push_back(gs);
  }
  e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { delete b; return cuda_fail("heom_batch_create: begin capture", e); }
  int rc = HEOM_OK;
  e = cudaEventRecord(b->ev[P], b->origin);
  for (int p = 0; p < P && e == cudaSuccess; ++p) e = cudaStreamWaitEvent(b->pool[p], b->ev[P], 0);
  b->launches_per_replay.assign(n_runs, 0);
  // grouped runs: per RK4 step, four stages of batched launches on the group's stream
  for (size_t g = 0; g < b->gruns.size() && e == cudaSuccess && rc == HEOM_OK; ++g) {
    const int kind_body = b->gfp64[g] ? 0 : 1;
    for (int64_t s = 0; s < steps_per_launch && rc == HEOM_OK; ++s) {
      for (int st = 0; st < 4 && rc == HEOM_OK; ++st) {
        if (!b->gfp64[g]) {
          rc = launch_stage_vec_batch(2, b->gn[g], b->gargs[g][st * 2], b->gstream[g], b->runs[0]->sm_count);
          ++b->launches_per_replay[b->gruns[g][0]];
        }
        if (rc == HEOM_OK) {
          rc = launch_stage_vec_batch(kind_body, b->gn[g], b->gargs[g][st * 2 + 1], b->gstream[g],
                                      b->runs[0]->sm_count);
          ++b->launches_per_replay[b->gruns[g][0]];
        }
      }
      if (rc != HEOM_OK) rc = HEOM_E_CUDA;
      if (rc == HEOM_OK && obs_stride > 0 && (s + 1) % obs_stride == 0) {
        for (int i : b->gruns[g]) {
          heom_run *r = b->runs[i];
          cudaStream_t own = r->stream;
          const int64_t l0 = r->launches, rec0 = r->records_host;
          r->stream = b->gstream[g];
          rc = enqueue_record(r, false);  // counts are checked per replay by heom_batch_launch
          b->launches_per_replay[i] += r->launches - l0;
          r->launches = l0;
          r->records_host = rec0;  // advanced by heom_batch_launch
          r->stream = own;
          if (rc != HEOM_OK) break;
        }
      }
    }
  }
  for (int i = 0; i < n_runs && e == cudaSuccess && rc == HEOM_OK; ++i) {
    if (grouped[i]) continue;
    heom_run *r = b->runs[i];
    cudaStream_t own = r->stream;
    const int64_t l0 = r->launches, rec0 = r->records_host;
    r->stream = b->pool[i % P];  // counters are restored below; launches advance them
    for (int64_t s = 0; s < steps_per_launch && rc == HEOM_OK; ++s) {
      if ((rc = run_stage(r, r->y, r->y, r->zA, h / 4))) break;
      if ((rc = run_stage(r, r->zA, r->y, r->zB, h / 3))) break;
      if ((rc = run_stage(r, r->zB, r->y, r->zA, h / 2))) break;
      if ((rc = run_stage(r, r->zA, r->y, r->y, h))) break;
      if (obs_stride > 0 && (s + 1) % obs_stride == 0) rc = enqueue_record(r, false);
    }
    b->launches_per_replay[i] = r->launches - l0;
    r->launches = l0;
    r->records_host = rec0;
    r->stream = own;
  }
  for (int p = 0; p < P && e == cudaSuccess; ++p) {
    e = cudaEventRecord(b->ev[p], b->pool[p]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev[p], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(b->origin, &g);
  if (rc != HEOM_OK) { if (g) cudaGraphDestroy(g); delete b; return rc; }
  if (e == cudaSuccess) e = ee;
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); delete b; return cuda_fail("heom_batch_create: capture", e); }
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) { delete b; return cuda_fail("heom_batch_create: instantiate", e); }
  *out = b;
  return HEOM_OK;
}

extern "C" int heom_batch_launch(heom_batch *b, int64_t n_launches) {
  if (!b || n_launches < 0) { set_error("heom_batch_launch: bad arguments"); return HEOM_E_ARG; }
  const int64_t recs = b->obs_stride > 0 ? b->steps_per_launch / b->obs_stride : 0;
  for (const auto &gv : b->gruns)
    for (int i : gv)
      if (!b->runs[i]->vec || b->runs[i]->desc_owner != b) {
        set_error("heom_batch_launch: a run left the column-0 layout or joined a later batch; create the batch again");
        return HEOM_E_STATE;
      }
  for (heom_run *r : b->runs)
    if (r->records_host + recs * n_launches > r->max_records) {
      set_error("heom_batch_launch: observable records of a run would exceed its max_records");
      return HEOM_E_NOMEM;
    }
  // order after work already enqueued on the runs' own streams (each distinct stream once)
  cudaError_t e = cudaSuccess;
  std::vector<cudaStream_t> seen;
  for (heom_run *r : b->runs) {
    if (std::find(seen.begin(), seen.end(), r->stream) != seen.end()) continue;
    seen.push_back(r->stream);
    e = cudaEventRecord(b->ev[0], r->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev[0], 0);
    if (e != cudaSuccess) return cuda_fail("heom_batch_launch: ordering", e);
  }
  for (int64_t k = 0; k < n_launches; ++k) {
    e = cudaGraphLaunch(b->exec, b->origin);
    if (e != cudaSuccess) return cuda_fail("heom_batch_launch: graph launch", e);
  }
  // later calls on a run's own stream see the batch's work
  e = cudaEventRecord(b->ev[0], b->origin);
  for (size_t k = 0; k < seen.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(seen[k], b->ev[0], 0);
  if (e != cudaSuccess) return cuda_fail("heom_batch_launch: join", e);
  for (size_t i = 0; i < b->runs.size(); ++i) {
    heom_run *r = b->runs[i];
    r->steps_done += n_launches * b->steps_per_launch;
    r->t_fs += (double)(n_launches * b->steps_per_launch) * b->dt;
    r->records_host += recs * n_launches;
    r->launches += n_launches * b->launches_per_replay[i];
  }
  return HEOM_OK;
}

extern "C" int heom_batch_schedule(const heom_batch *b, int g, int part, heom_schedule *out, int *n_groups) {
  if (!b) { set_error("heom_batch_schedule: NULL batch"); return HEOM_E_ARG; }
  if (n_groups) *n_groups = (int)b->gsched.size();
  if (g == -1 && !out) return HEOM_OK;
  if (g < 0 || g >= (int)b->gsched.size() || part < 0 || part > 1 || !out) {
    set_error("heom_batch_schedule: group out of range, part 0 or 1, out needed");
    return HEOM_E_ARG;
  }
  *out = b->gsched[g][part];
  return HEOM_OK;
}

extern "C" int heom_batch_destroy(heom_batch *b) {
  if (b) cudaStreamSynchronize(b->origin);
  delete b;
  return HEOM_OK;
}
