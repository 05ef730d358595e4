// C ABI of libheom, part 5: heom_group_propagate -- many runs advanced together, the RK4 stages of
// small mixed-precision runs of equal n_states sharing work-list launches (stage_list.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/heom.h"
#include "heom_internal.h"
#include "heom_run.h"

using namespace heom;

namespace {

// Runs above this many body ADOs keep launches of their own: the work-list kernel reads H from
// shared memory instead of the constant bank, which costs at the sizes where one run fills the GPU.
constexpr int64_t kListRunMaxAdos = 200000;
// Chunks per work item: one per warp (4-warp FP32 body kernel, 2-warp FP64 head kernel), so that a
// small run spreads over as many CTAs as it has chunks -- at these sizes a launch is latency-bound,
// and the FP64 head of a large n_states (one ADO per chunk) is the longest chain.
constexpr int kListCpiBody = 4;
constexpr int kListCpiHead = 2;
const char kListTag = 0;          // desc_owner of runs whose descriptor area holds work-list arguments

// The Horner stages of one RK4 step: (input, base, output, coefficient of h).
struct HornerStage {
  int zin, y, out;  // 0 = y, 1 = zA, 2 = zB
  double c;
};
constexpr HornerStage kHorner[4] = {{0, 0, 1, 0.25}, {1, 0, 2, 1.0 / 3.0}, {2, 0, 1, 0.5}, {1, 0, 0, 1.0}};

StateView view_of(const heom_run *r, int k) { return k == 0 ? r->y : (k == 1 ? r->zA : r->zB); }

bool list_eligible(const heom_run *r) {
  return r->precision == HEOM_FP32_MIXED && !r->vec && !r->gen && !r->has_field && !r->cplx_h && r->u_split > 0 &&
         r->n_ado - r->u_split <= kListRunMaxAdos;
}

template <typename CT>
void fill_args(GroupArgs<CT> &g, const heom_run *r, int st, double h, bool head) {
  const HornerStage &hs = kHorner[st];
  std::memset(&g, 0, sizeof(g));
  g.c = common_for(r, view_of(r, hs.zin), view_of(r, hs.y), view_of(r, hs.out));
  g.c.u_begin = head ? 0 : r->u_split;
  g.c.u_end = head ? r->u_split : (int)r->n_ado;
  g.c.occ_pct = r->sched[head ? 1 : 0].occupancy_pct;
  g.c.cpw = r->sched[head ? 1 : 0].chunks_per_warp;
  g.ch = (CT)(hs.c * h);
  for (int i = 0; i < kMaxStates; ++i) g.term[i] = (i < r->n) ? (CT)r->term[i] : (CT)0;
  for (int i = 0; i < r->n; ++i)
    for (int j = 0; j < r->n; ++j) g.H[i * kMaxStates + j] = (CT)r->H[(size_t)i * r->n + j];
}

// The run's work-list stage arguments for time step h, written into its descriptor area on stream s
// unless they are there already.
int ensure_args(heom_run *r, double h, cudaStream_t s, std::vector<GroupRunDesc> &host, size_t k) {
  if (r->desc_owner == &kListTag && r->desc_dt == h) return HEOM_OK;
  GroupRunDesc &d = host[k];
  for (int st = 0; st < 4; ++st) {
    fill_args(d.body[st], r, st, h, false);
    fill_args(d.head[st], r, st, h, true);
  }
  cudaError_t e = cudaMemcpyAsync(r->desc_dev, &d, sizeof(GroupRunDesc), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail("heom_group_propagate: stage arguments", e);
  r->desc_owner = &kListTag;
  r->desc_dt = h;
  return HEOM_OK;
}

}  // namespace

extern "C" int heom_group_propagate(heom_run *const *runs, int n_runs, double dt_fs, const int64_t *n_steps,
                                    int64_t obs_stride, void *cuda_stream) {
  if (!runs || n_runs < 0 || (n_runs > 0 && !n_steps) || !(dt_fs > 0) || obs_stride < 0) {
    set_error("heom_group_propagate: need runs, n_runs >= 0, n_steps, dt_fs > 0, obs_stride >= 0");
    return HEOM_E_ARG;
  }
  const double h = dt_fs;
  std::vector<heom_run *> rv(runs, runs + n_runs);
  {
    std::vector<heom_run *> sorted(rv);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
      set_error("heom_group_propagate: a run is listed twice");
      return HEOM_E_ARG;
    }
  }
  int64_t max_steps = 0;
  for (int i = 0; i < n_runs; ++i) {
    heom_run *r = rv[i];
    if (!r || n_steps[i] < 0) {
      set_error("heom_group_propagate: NULL run or negative step count");
      return HEOM_E_ARG;
    }
    if (h * r->max_rate > 2.5) {
      set_error("heom_group_propagate: dt_fs * depth * max gamma > 2.5 for a run (RK4 unstable; the paper asks "
                "dt << 1/gamma_k)");
      return HEOM_E_ARG;
    }
    if (r->has_field) {
      set_error("heom_group_propagate: a run has a laser field (use heom_propagate)");
      return HEOM_E_STATE;
    }
    if (r->timing) {
      set_error("heom_group_propagate: a run has kernel timing on");
      return HEOM_E_STATE;
    }
    if (obs_stride > 0) {
      const int64_t first = obs_stride - (r->steps_done % obs_stride);
      const int64_t need = (n_steps[i] >= first) ? 1 + (n_steps[i] - first) / obs_stride : 0;
      if (r->records_host + need > r->max_records) {
        set_error("heom_group_propagate: observable records of a run would exceed its max_records");
        return HEOM_E_NOMEM;
      }
    }
    max_steps = std::max(max_steps, n_steps[i]);
  }
  if (n_runs == 0 || max_steps == 0) return HEOM_OK;
  cudaStream_t gs = reinterpret_cast<cudaStream_t>(cuda_stream);

  // order after the work already enqueued on every run's stream
  std::vector<cudaStream_t> streams;
  for (heom_run *r : rv)
    if (std::find(streams.begin(), streams.end(), r->stream) == streams.end()) streams.push_back(r->stream);
  std::vector<cudaEvent_t> evs(streams.size() + 1, nullptr);
  auto cleanup = [&]() {
    for (cudaEvent_t e : evs)
      if (e) cudaEventDestroy(e);
  };
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < evs.size() && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&evs[k], cudaEventDisableTiming);
  for (size_t k = 0; k < streams.size() && e == cudaSuccess; ++k) {
    if (streams[k] == gs) continue;
    e = cudaEventRecord(evs[k], streams[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, evs[k], 0);
  }
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail("heom_group_propagate: stream order", e);
  }

  // work-list arguments of the eligible runs
  std::vector<GroupRunDesc> host(n_runs);
  std::vector<bool> listed(n_runs);
  for (int i = 0; i < n_runs; ++i) {
    listed[i] = list_eligible(rv[i]) && n_steps[i] > 0;
    if (listed[i]) {
      const int rc = ensure_args(rv[i], h, gs, host, (size_t)i);
      if (rc != HEOM_OK) {
        cleanup();
        return rc;
      }
    }
  }

  int rc = HEOM_OK;
  // Each size class gets a stream of its own for the whole call (forked from and joined back into the
  // caller's stream): the classes' launch chains run side by side, while the stages of one class
  // follow each other.  A run keeps its class, so its launches stay in order.
  std::vector<cudaStream_t> cls(kMaxStates + 1, nullptr);
  std::vector<cudaEvent_t> cls_ev;
  // one size class and nothing else: its launches go straight to the caller's stream
  bool single = true;
  int n0 = -1;
  for (int i = 0; i < n_runs && single; ++i) {
    if (n_steps[i] == 0) continue;
    if (n0 < 0) n0 = rv[i]->n;
    single = listed[i] && rv[i]->n == n0;
  }
  // the stream of size class n in *out (the caller's stream, which may be the NULL stream, when the call
  // has a single class)
  auto class_stream = [&](int n, cudaStream_t *out) -> int {
    *out = gs;
    if (single) return HEOM_OK;
    if (!cls[n]) {
      // the class streams take the caller's priority, so that a high-priority caller's ticks stay ahead
      // of other streams' launches when SM slots free up
      cudaEvent_t fe = nullptr;
      int prio = 0;
      cudaError_t ce = cudaStreamGetPriority(gs, &prio);
      if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&cls[n], cudaStreamNonBlocking, prio);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&fe, cudaEventDisableTiming);
      if (ce == cudaSuccess) cls_ev.push_back(fe);
      if (ce == cudaSuccess) ce = cudaEventRecord(fe, gs);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cls[n], fe, 0);
      if (ce != cudaSuccess) return cuda_fail("heom_group_propagate: class stream", ce);
    }
    *out = cls[n];
    return HEOM_OK;
  };
  // the work-list launches of one step, rebuilt only when a run's steps end: per class of equal
  // n_states and per batch of at most kListMaxRuns runs, the head and body launch of each stage
  struct Prepared {
    int n, kind, sm_count;
    cudaStream_t stream;
    ListLaunch L[4];
    std::vector<heom_run *> members;
  };
  std::vector<Prepared> prep;
  int64_t rebuilt_at = -1;
  for (int64_t s = 0; s < max_steps && rc == HEOM_OK; ++s) {
    bool change = rebuilt_at < 0;
    for (int i = 0; i < n_runs && !change; ++i) change = listed[i] && n_steps[i] == s;
    if (change) {
      std::map<int, std::vector<int>> classes;  // n_states -> listed runs still stepping
      for (int i = 0; i < n_runs; ++i)
        if (listed[i] && n_steps[i] > s) classes[rv[i]->n].push_back(i);
      prep.clear();
      for (const auto &cl : classes) {
        cudaStream_t cs = gs;
        if ((rc = class_stream(cl.first, &cs)) != HEOM_OK) break;
        for (size_t b0 = 0; b0 < cl.second.size(); b0 += kListMaxRuns) {
          const size_t b1 = std::min(cl.second.size(), b0 + (size_t)kListMaxRuns);
          for (int part = 0; part < 2; ++part) {  // FP64 head, then FP32 body
            Prepared p;
            p.n = cl.first;
            p.kind = part == 0 ? 2 : 1;
            p.sm_count = rv[cl.second[b0]]->sm_count;
            p.stream = cs;
            for (int st = 0; st < 4; ++st) {
              ListLaunch &L = p.L[st];
              L.nruns = (int)(b1 - b0);
              L.cpi = part == 0 ? kListCpiHead : kListCpiBody;
              L.item0[0] = 0;
              for (size_t q = b0; q < b1; ++q) {
                const heom_run *r = rv[cl.second[q]];
                const GroupRunDesc *d = reinterpret_cast<const GroupRunDesc *>(r->desc_dev);
                const int A = 32 / r->n < 32 ? 32 / r->n : 31;
                const int64_t ados = part == 0 ? r->u_split : r->n_ado - r->u_split;
                const int64_t chunks = (ados + A - 1) / A;
                L.args[q - b0] = part == 0 ? (const void *)&d->head[st] : (const void *)&d->body[st];
                L.item0[q - b0 + 1] = L.item0[q - b0] + (int)((chunks + L.cpi - 1) / L.cpi);
              }
            }
            for (size_t q = b0; q < b1; ++q) p.members.push_back(rv[cl.second[q]]);
            prep.push_back(std::move(p));
          }
        }
      }
      rebuilt_at = s;
    }
    for (int st = 0; st < 4 && rc == HEOM_OK; ++st) {
      for (Prepared &p : prep) {
        if (launch_stage_list(p.kind, p.n, p.L[st], p.stream, p.sm_count)) {
          rc = HEOM_E_CUDA;
          break;
        }
        for (heom_run *r : p.members) ++r->launches;  // one work-list launch counts for each of its runs
      }
      // runs outside the work lists: their own launches, on the caller's stream
      for (int i = 0; i < n_runs && rc == HEOM_OK; ++i) {
        if (listed[i] || n_steps[i] <= s) continue;
        heom_run *r = rv[i];
        const HornerStage &hs = kHorner[st];
        cudaStream_t own = r->stream;
        r->stream = gs;
        rc = run_stage(r, view_of(r, hs.zin), view_of(r, hs.y), view_of(r, hs.out), hs.c * h);
        r->stream = own;
      }
    }
    for (int i = 0; i < n_runs && rc == HEOM_OK; ++i) {  // step counters and observable records
      if (n_steps[i] <= s) continue;
      heom_run *r = rv[i];
      ++r->steps_done;
      r->t_fs += h;
      if (obs_stride > 0 && r->steps_done % obs_stride == 0) {
        cudaStream_t own = r->stream;
        r->stream = (listed[i] && !single) ? cls[r->n] : gs;  // after the run's own stage launches
        rc = enqueue_record(r);
        r->stream = own;
      }
    }
  }
  // join the class streams back into the caller's stream
  for (int n = 0; n <= kMaxStates; ++n) {
    if (!cls[n]) continue;
    cudaEvent_t je = nullptr;
    cudaError_t ce = cudaEventCreateWithFlags(&je, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(je, cls[n]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(gs, je, 0);
    if (je) cudaEventDestroy(je);
    cudaStreamDestroy(cls[n]);  // released once its work is done
    if (ce != cudaSuccess && rc == HEOM_OK) rc = cuda_fail("heom_group_propagate: class stream join", ce);
  }
  for (cudaEvent_t fe : cls_ev) cudaEventDestroy(fe);

  // later work on every run's stream is ordered after this call's launches
  e = cudaEventRecord(evs.back(), gs);
  for (size_t k = 0; k < streams.size() && e == cudaSuccess; ++k)
    if (streams[k] != gs) e = cudaStreamWaitEvent(streams[k], evs.back(), 0);
  cleanup();
  if (rc != HEOM_OK) return rc;
  return e == cudaSuccess ? HEOM_OK : cuda_fail("heom_group_propagate: stream order", e);
}
