// C ABI of libheom, part 3: launch schedules and the autotuner (heom_tune and the calls around it).
#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/heom.h"
#include "heom_internal.h"
#include "heom_run.h"

using namespace heom;

// ------------------------------------------------------------------------------------------------
// launch schedules and the autotuner: every candidate is timed on the run's own stage-1 launch
// (zin = y, out = zA; y is not written) and the fastest is kept, per run and in a process-wide
// cache.  All schedules compute the same sums in the same order, so the choice changes only time.

namespace heom {
std::atomic<int> g_autotune{3};  // timed launches per candidate at creation (0: off)
static std::mutex g_tune_mu;  // guards the cache and the defaults
static std::map<std::array<int, 7>, heom_schedule> g_tune_cache;  // (layout, precision, part, n, herm, cplx, log2 ADOs)
static heom_schedule g_default[3] = {{100, 1}, {100, 1}, {100, 1}};  // per layout, without cache entry or tuning

heom_schedule default_for(int layout) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return g_default[layout];
}

int ilog2(int64_t x) {
  int b = 0;
  while (x > 1) {
    x >>= 1;
    ++b;
  }
  return b;
}

std::vector<heom_schedule> candidates(int layout) {
  std::vector<heom_schedule> v;
  if (layout == 0) {
    for (int occ : {100, 75, 50}) v.push_back(heom_schedule{occ, 1});
  } else {
    for (int cpw : {1, 2, 4})
      for (int occ : {100, 50}) v.push_back(heom_schedule{occ, cpw});
  }
  return v;  // the default {100, 1} first: ties keep it
}

static bool valid_schedule(const heom_schedule &s) {
  return s.occupancy_pct >= 1 && s.occupancy_pct <= 1600 &&
         (s.chunks_per_warp == 1 || s.chunks_per_warp == 2 || s.chunks_per_warp == 4);
}

static std::array<int, 7> run_key(const heom_run *r, int part) {
  const int64_t cnt = part == 1 ? r->u_split : r->n_ado - (r->precision == HEOM_FP64 ? 0 : r->u_split);
  return {r->vec ? 1 : 0, r->precision, part, r->n, r->herm ? 1 : 0, r->cplx_h ? 1 : 0, ilog2(cnt)};
}

bool cache_get(const std::array<int, 7> &k, heom_schedule *out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune_cache.find(k);
  if (it == g_tune_cache.end()) return false;
  *out = it->second;
  return true;
}

void cache_put(const std::array<int, 7> &k, const heom_schedule &s) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[k] = s;
}

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}


static int tune_part(heom_run *r, int part, int reps, std::vector<heom_schedule> &tried, std::vector<double> &ms) {
  if (capturing(r->stream)) {
    set_error("heom_tune: the run's stream is being captured");
    return HEOM_E_STATE;
  }
  tried = candidates(r->vec ? 1 : 0);
  const heom_schedule keep = r->sched[part];
  const StageCommon c = common_for(r, r->y, r->y, r->zA);
  int best = 0;
  const int rc = time_candidates(tried, reps, r->stream, [&](const heom_schedule &sc) {
    r->sched[part] = sc;
    return part == 1 ? launch_head(r, c, 0.25, r->stream) : launch_body(r, c, 0.25, r->stream);
  }, ms, &best);
  if (rc != HEOM_OK) {
    r->sched[part] = keep;
    return rc;
  }
  r->sched[part] = tried[best];
  cache_put(run_key(r, part), tried[best]);
  return HEOM_OK;
}

void reschedule_cached(heom_run *r) {
  for (int part = 0; part < 2; ++part) {
    r->sched[part] = default_for(r->vec ? 1 : 0);
    if (part == 0 || r->precision != HEOM_FP64) cache_get(run_key(r, part), &r->sched[part]);
  }
}

// The schedule of each part of a new run: the cache, else the tuner (if on), else the default.
int schedule_new_run(heom_run *r) {
  if (r->gen) return HEOM_OK;  // the general kernel keeps the default schedule
  const int reps = g_autotune.load();
  for (int part = 0; part < (r->precision == HEOM_FP64 ? 1 : 2); ++part) {
    heom_schedule s{100, 1};
    r->sched[part] = default_for(r->vec ? 1 : 0);
    if (cache_get(run_key(r, part), &s)) {
      r->sched[part] = s;
    } else if (reps > 0 && !g_tune_suppress && !capturing(r->stream)) {
      std::vector<heom_schedule> tried;
      std::vector<double> ms;
      const int rc = tune_part(r, part, reps, tried, ms);
      if (rc != HEOM_OK) return rc;
    }
  }
  return HEOM_OK;
}
}  // namespace heom

extern "C" int heom_schedule_candidates(int layout, heom_schedule *out, int cap) {
  if (layout < 0 || layout > 2 || cap < 0 || (cap > 0 && !out)) {
    set_error("heom_schedule_candidates: layout 0..2, cap >= 0, out for cap > 0");
    return HEOM_E_ARG;
  }
  const std::vector<heom_schedule> v = candidates(layout);
  for (int i = 0; i < cap && i < (int)v.size(); ++i) out[i] = v[i];
  return (int)v.size();
}

extern "C" int heom_tune(heom_run *r, int part, int reps, heom_schedule *tried, double *ms, int cap, int *n_tried,
                         heom_schedule *chosen) {
  if (!r || reps < 1 || part < 0 || part > 1 || (part == 1 && r->precision == HEOM_FP64) || cap < 0) {
    set_error("heom_tune: need a run, reps >= 1, part 0 or 1 (1 only with an FP64 head), cap >= 0");
    return HEOM_E_ARG;
  }
  if (r->gen) {
    set_error("heom_tune: runs on the general stage kernel keep the default schedule");
    return HEOM_E_STATE;
  }
  std::vector<heom_schedule> t;
  std::vector<double> m;
  const int rc = tune_part(r, part, reps, t, m);
  if (rc != HEOM_OK) return rc;
  for (int i = 0; i < cap && i < (int)t.size(); ++i) {
    if (tried) tried[i] = t[i];
    if (ms) ms[i] = m[i];
  }
  if (n_tried) *n_tried = (int)t.size();
  if (chosen) *chosen = r->sched[part];
  return HEOM_OK;
}

extern "C" int heom_set_autotune(int reps) {
  if (reps < 0) return g_autotune.load();
  return g_autotune.exchange(reps);
}

extern "C" int heom_get_schedule(const heom_run *r, int part, heom_schedule *out) {
  if (!r || !out || part < 0 || part > 1 || (part == 1 && r->precision == HEOM_FP64)) {
    set_error("heom_get_schedule: need a run, out, part 0 or 1 (1 only with an FP64 head)");
    return HEOM_E_ARG;
  }
  *out = r->sched[part];
  return HEOM_OK;
}

extern "C" int heom_set_schedule(heom_run *r, int part, const heom_schedule *s) {
  if (!r || !s || part < 0 || part > 1 || (part == 1 && r->precision == HEOM_FP64) || !valid_schedule(*s)) {
    set_error("heom_set_schedule: need a run, part 0 or 1 (1 only with an FP64 head), occupancy_pct 1..1600, "
              "chunks_per_warp 1, 2 or 4");
    return HEOM_E_ARG;
  }
  r->sched[part] = *s;
  return HEOM_OK;
}

extern "C" int heom_set_default_schedule(int layout, const heom_schedule *s) {
  if (layout < 0 || layout > 2 || (s && !valid_schedule(*s))) {
    set_error("heom_set_default_schedule: layout 0..2 and a valid schedule (or NULL)");
    return HEOM_E_ARG;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_default[layout] = s ? *s : heom_schedule{100, 1};
  return HEOM_OK;
}

extern "C" int heom_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.clear();
  return HEOM_OK;
}
