// C ABI of libheom (include/heom.h), part 1: hierarchy handles, run set-up (units, Matsubara and Pade
// coefficients, rescaling tables, link records, workspace layout, table upload), state I/O and the
// laser field.  The RK4 driver is in propagate.cu, the autotuner in tuner.cu, batches in batch.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/heom.h"
#include "heom_internal.h"
#include "heom_run.h"

namespace heom {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

int launch_stage(int precision, const StageCommon &c, double ch, const double *term, const double *H,
                 const double *Hi, cudaStream_t st, int sm_count) {
  if (c.u_end <= c.u_begin) return 0;
  static int (*const fns[3][4])(const StageCommon &, double, const double *, const double *, const double *,
                                 cudaStream_t, int) = {
      {launch_stage_fp64_a, launch_stage_fp64_b, launch_stage_fp64_c, launch_stage_fp64_d},
      {launch_stage_fp32_a, launch_stage_fp32_b, launch_stage_fp32_c, launch_stage_fp32_d},
      {launch_stage_head_a, launch_stage_head_b, launch_stage_head_c, launch_stage_head_d}};
  int rc = 1;
  if (precision == 0 && c.herm && !c.cplx_h) rc = launch_stage_col(c, ch, term, H, st, sm_count);
  for (int g = 0; g < 4 && rc == 1; ++g) rc = fns[precision][g](c, ch, term, H, Hi, st, sm_count);
  if (rc == 1) {
    set_error("stage kernel: n_states not compiled");
    return -1;
  }
  return rc;
}

int launch_stage_list(int kind, int n, const ListLaunch &L, cudaStream_t st, int sm_count) {
  int rc = launch_stage_list_a(kind, n, L, st, sm_count);
  if (rc == 1) rc = launch_stage_list_b(kind, n, L, st, sm_count);
  if (rc == 1) rc = launch_stage_list_c(kind, n, L, st, sm_count);
  if (rc == 1) set_error("work-list stage kernel: n_states not compiled");
  return rc;
}

int launch_stage_vec(int kind, const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st,
                     int sm_count) {
  switch (c.cpw) {
    case 2: return launch_stage_vec_g2(kind, c, ch, term, H, st, sm_count);
    case 4: return launch_stage_vec_g4(kind, c, ch, term, H, st, sm_count);
    default: return launch_stage_vec_g1(kind, c, ch, term, H, st, sm_count);
  }
}

int launch_stage_vec_batch(int kind, int n, const VecBatchArgs &a, cudaStream_t st, int sm_count) {
  switch (a.cpw) {
    case 2: return launch_stage_vec_batch_g2(kind, n, a, st, sm_count);
    case 4: return launch_stage_vec_batch_g4(kind, n, a, st, sm_count);
    default: return launch_stage_vec_batch_g1(kind, n, a, st, sm_count);
  }
}

// Set by heom_propagate_static around its run creation: no tuning there.
thread_local int g_tune_suppress = 0;

}  // namespace heom

using namespace heom;


extern "C" const char *heom_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------------------------------------
// hierarchy handles

extern "C" int heom_build_hierarchy(int n_modes, int depth, heom_hier **out) {
  if (!out) { set_error("heom_build_hierarchy: out is NULL"); return HEOM_E_ARG; }
  *out = nullptr;
  heom_hier *h = new (std::nothrow) heom_hier;
  if (!h) { set_error("heom_build_hierarchy: host allocation failed"); return HEOM_E_NOMEM; }
  std::string err;
  int rc = build_hierarchy(n_modes, depth, &h->h, &err);
  if (rc != HEOM_OK) { delete h; set_error(err); return rc; }
  *out = h;
  return HEOM_OK;
}

extern "C" int heom_hier_destroy(heom_hier *h) {
  delete h;
  return HEOM_OK;
}

extern "C" int heom_hier_info(const heom_hier *h, int64_t *n_ado, int64_t *level_offsets) {
  if (!h) { set_error("heom_hier_info: NULL handle"); return HEOM_E_ARG; }
  if (n_ado) *n_ado = h->h.n;
  if (level_offsets)
    for (int L = 0; L <= h->h.D + 1; ++L) level_offsets[L] = h->h.level_off[L];
  return HEOM_OK;
}

extern "C" int heom_hier_export(const heom_hier *h, uint8_t *tuples, int32_t *plus, int32_t *minus) {
  if (!h) { set_error("heom_hier_export: NULL handle"); return HEOM_E_ARG; }
  const size_t cnt = (size_t)h->h.n * h->h.M;
  if (tuples) memcpy(tuples, h->h.tuples.data(), cnt);
  if (plus) memcpy(plus, h->h.plus.data(), cnt * sizeof(int32_t));
  if (minus) memcpy(minus, h->h.minus.data(), cnt * sizeof(int32_t));
  return HEOM_OK;
}

// ------------------------------------------------------------------------------------------------
// run set-up

namespace {

struct Layout {
  size_t off_loff, off_rh, off_rb, off_gsum, off_rec, off_w, off_cnt, off_desc;
  size_t off_state[4];  // y, zA, zB, and (time-dependent runs) the RK4 accumulator
  size_t head_bytes, body_bytes;
  size_t total;
};

inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// The system alone (no hierarchy, no precision).
int check_system_only(const heom_system *s) {
  if (!s) { set_error("NULL system"); return HEOM_E_ARG; }
  if (s->n_states < 1 || s->n_states > kGenMaxStates) {
    set_error("n_states must be in [1, 32]");
    return HEOM_E_ARG;
  }
  if (s->bath_mask)
    for (int64_t e = 0; e < (int64_t)s->n_baths * s->n_states; ++e)
      if (s->bath_mask[e] > 1) {
        set_error("bath_mask entries must be 0 or 1");
        return HEOM_E_ARG;
      }
  if (s->time_dependent != 0 && s->time_dependent != 1) {
    set_error("time_dependent must be 0 or 1");
    return HEOM_E_ARG;
  }
  if (!s->H_re) { set_error("H_re is NULL"); return HEOM_E_ARG; }
  if (s->n_baths < 1 || !s->bath_state || !s->lambda_cm || !s->tau_fs || !s->T_K || s->n_matsubara < 0) {
    set_error("need n_baths >= 1, bath arrays and n_matsubara >= 0");
    return HEOM_E_ARG;
  }
  for (int b = 0; b < s->n_baths; ++b) {
    if (s->bath_state[b] < 0 || s->bath_state[b] >= s->n_states) {
      set_error("bath_state out of range");
      return HEOM_E_ARG;
    }
    if (!(s->tau_fs[b] > 0) || !(s->T_K[b] > 0) || !(s->lambda_cm[b] >= 0)) {
      set_error("need tau_fs > 0, T_K > 0, lambda_cm >= 0");
      return HEOM_E_ARG;
    }
  }
  if (s->decomposition != HEOM_MATSUBARA && s->decomposition != HEOM_PADE) {
    set_error("decomposition must be HEOM_MATSUBARA or HEOM_PADE");
    return HEOM_E_ARG;
  }
  if (s->decomposition == HEOM_PADE && s->n_matsubara > 64) {
    set_error("at most 64 Pade poles per bath");
    return HEOM_E_ARG;
  }
  return HEOM_OK;
}

int check_system(const heom_system *s, const heom_hier *h, int precision) {
  if (!s || !h) { set_error("NULL system or hierarchy"); return HEOM_E_ARG; }
  int rc = check_system_only(s);
  if (rc) return rc;
  if ((int64_t)s->n_baths * (s->n_matsubara + 1) != h->h.M) {
    set_error("hierarchy n_modes != n_baths * (n_matsubara + 1)");
    return HEOM_E_ARG;
  }
  if (precision != HEOM_FP64 && precision != HEOM_FP32_MIXED && precision != HEOM_SPLIT_TF32) {
    set_error("unknown precision");
    return HEOM_E_ARG;
  }
  return HEOM_OK;
}

// Eigenvalues of the symmetric tridiagonal matrix with zero diagonal and off-diagonal e[0..n-2],
// in decreasing order, by bisection on the Sturm count (number of eigenvalues below x from the
// signs of the LDL^T pivots of T - x I).
static std::vector<double> tridiag_eigs_desc(const std::vector<double> &e, int n) {
  double bound = 0;
  for (double v : e) bound = std::max(bound, 2.0 * std::fabs(v));
  bound += 1e-12;
  auto count_below = [&](double x) {
    int cnt = 0;
    double q = -x;
    if (q < 0) ++cnt;
    for (int i = 1; i < n; ++i) {
      if (q == 0) q = 1e-300;
      q = -x - e[i - 1] * e[i - 1] / q;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  std::vector<double> ev(n);
  for (int k = 0; k < n; ++k) {  // k-th largest: n - 1 - k eigenvalues lie below it
    double lo = -bound, hi = bound;
    for (int it = 0; it < 200 && hi - lo > 1e-17 * std::max(1.0, std::fabs(hi)); ++it) {
      const double mid = 0.5 * (lo + hi);
      if (count_below(mid) > n - 1 - k) hi = mid;
      else lo = mid;
    }
    ev[k] = 0.5 * (lo + hi);
  }
  return ev;
}

// [K-1/K] Pade poles xi and weights eta of the Bose function (section "HEOM formalism", method of
// Hu, Xu, Yan 2010): 1/(1 - e^-x) ~ 1/x + 1/2 + sum_i 2 eta_i x / (x^2 + xi_i^2).
static void pade_poles(int K, std::vector<double> &xi, std::vector<double> &eta) {
  xi.assign(K, 0.0);
  eta.assign(K, 0.0);
  if (K < 1) return;
  std::vector<double> e1(2 * K - 1), e2(std::max(0, 2 * K - 2));
  for (int m = 1; m < 2 * K; ++m) e1[m - 1] = 1.0 / std::sqrt((2.0 * m + 1) * (2.0 * m + 3));
  for (int m = 1; m < 2 * K - 1; ++m) e2[m - 1] = 1.0 / std::sqrt((2.0 * m + 3) * (2.0 * m + 5));
  const std::vector<double> l1 = tridiag_eigs_desc(e1, 2 * K);
  const std::vector<double> l2 = K > 1 ? tridiag_eigs_desc(e2, 2 * K - 1) : std::vector<double>();
  std::vector<double> zeta(std::max(0, K - 1));
  for (int i = 0; i < K; ++i) xi[i] = 2.0 / l1[i];
  for (int i = 0; i < K - 1; ++i) zeta[i] = 2.0 / l2[i];
  for (int i = 0; i < K; ++i) {
    double num = 1.0, den = 1.0;
    for (int j = 0; j < K - 1; ++j) num *= zeta[j] * zeta[j] - xi[i] * xi[i];
    for (int j = 0; j < K; ++j)
      if (j != i) den *= xi[j] * xi[j] - xi[i] * xi[i];
    eta[i] = 0.5 * K * (2.0 * K + 3.0) * num / den;
  }
}

// Bath modes of Eq. HEOM (Drude-Lorentz, Omega = 0) in rad/fs: rates, real coefficients, lambda nu
// of the Drude modes, coupled states, per-state terminator; gmax = the largest rate.
// Diagonal of V_b: the bath's row of bath_mask, else 1 at bath_state[b].
static double v_diag(const heom_system *sys, int b, int i) {
  if (sys->bath_mask) return (double)sys->bath_mask[(size_t)b * sys->n_states + i];
  return sys->bath_state[b] == i ? 1.0 : 0.0;
}

// Per mode: gamma, c, lambda nu (k = 0), the bath's labelling state; per state the terminator rate
// sum_b Delta_b V_b,ii; per bath Delta_b (0 without the terminator) in *dbath if given.
static int compute_modes(const heom_system *sys, std::vector<double> &gam, std::vector<double> &cc,
                         std::vector<double> &lnu, std::vector<int> &mstate, std::vector<double> &term,
                         double *gmax, std::vector<double> *dbath = nullptr) {
  const int B = sys->n_baths, K = sys->n_matsubara, M = B * (K + 1);
  gam.assign(M, 0.0);
  cc.assign(M, 0.0);
  lnu.assign(M, 0.0);
  mstate.assign(M, 0);
  term.assign(sys->n_states, 0.0);
  if (dbath) dbath->assign(B, 0.0);
  *gmax = 0;
  std::vector<double> xi, eta;
  if (sys->decomposition == HEOM_PADE) pade_poles(K, xi, eta);
  for (int b = 0; b < B; ++b) {
    const double lam = kCmToRadFs * sys->lambda_cm[b];
    const double nu = 1.0 / sys->tau_fs[b];
    const double beta = 1.0 / (kCmToRadFs * kBoltzCm * sys->T_K[b]);
    double csum = 0;
    for (int k = 0; k <= K; ++k) {
      const int l = b * (K + 1) + k;
      double g = nu, c = 0;
      if (k > 0) {
        g = (sys->decomposition == HEOM_PADE) ? xi[k - 1] / beta : 2.0 * 3.14159265358979323846 * k / beta;
        if (std::fabs(g * g - nu * nu) < 1e-6 * g * g) {
          set_error("bath rate gamma_k equals nu for a bath (c_k diverges)");
          return HEOM_E_ARG;
        }
        c = 4.0 * lam * nu / beta * g / (g * g - nu * nu) * (sys->decomposition == HEOM_PADE ? eta[k - 1] : 1.0);
      }
      gam[l] = g;
      cc[l] = c;
      lnu[l] = (k == 0) ? lam * nu : 0.0;
      mstate[l] = sys->bath_state[b];
    }
    if (sys->decomposition == HEOM_PADE) {  // c(b,0) = (2 lambda / beta) (1 - sum_j 2 eta_j nu^2 / (gamma_j^2 - nu^2))
      double s = 0;
      for (int j = 0; j < K; ++j) {
        const double gj = gam[b * (K + 1) + 1 + j];
        s += 2.0 * eta[j] * nu * nu / (gj * gj - nu * nu);
      }
      cc[b * (K + 1)] = 2.0 * lam / beta * (1.0 - s);
    } else {
      cc[b * (K + 1)] = lam * nu / std::tan(0.5 * beta * nu);
    }
    for (int k = 0; k <= K; ++k) {
      const int l = b * (K + 1) + k;
      csum += cc[l] / gam[l];
      *gmax = std::max(*gmax, gam[l]);
    }
    if (sys->terminator) {
      const double delta = 2.0 * lam / (beta * nu) - csum;
      for (int i = 0; i < sys->n_states; ++i) term[i] += delta * v_diag(sys, b, i);
      if (dbath) (*dbath)[b] = delta;
    }
  }
  return HEOM_OK;
}

// Link records of the ADOs [u_lo, u_hi): one per valid link (up and down) and coupled state; mult[l]
// = states of mode l's V (1 for a projector; nullptr: all 1).
// fn(a, b) over [0, n) split into contiguous ranges, one per host thread (one thread for small n);
// false if any range threw (host allocation).
template <typename F>
bool host_parallel(int64_t n, F fn) {
  constexpr int64_t kMinPerThread = 16384;
  const int T = (int)std::min<int64_t>(host_threads(), std::max<int64_t>(1, n / kMinPerThread));
  std::atomic<bool> failed{false};
  auto guarded = [&](int64_t a, int64_t b) {
    try {
      fn(a, b);
    } catch (...) {
      failed = true;
    }
  };
  if (T <= 1) {
    guarded(0, n);
    return !failed;
  }
  const int64_t per = (n + T - 1) / T;
  std::vector<std::thread> pool;
  int64_t a = 0;
  for (; a < n; a += per) {
    const int64_t b = std::min(n, a + per);
    try {
      pool.emplace_back(guarded, a, b);
    } catch (...) {  // no thread: this range runs here
      guarded(a, b);
    }
  }
  for (auto &th : pool) th.join();
  return !failed;
}

int64_t count_links(const Hierarchy &h, int64_t u_lo, int64_t u_hi, const std::vector<int> *mult = nullptr) {
  int64_t k = 0;
  for (int64_t u = u_lo; u < u_hi; ++u)
    for (int l = 0; l < h.M; ++l)
      k += ((h.plus[(size_t)u * h.M + l] >= 0) + (h.minus[(size_t)u * h.M + l] >= 0)) * (mult ? (*mult)[l] : 1);
  return k;
}

// States coupled by each mode's V (the bath's mask row count, 1 without a mask).
std::vector<int> mode_mult(const heom_system *sys) {
  const int K1 = sys->n_matsubara + 1;
  std::vector<int> m((size_t)sys->n_baths * K1, 1);
  if (sys->bath_mask)
    for (int b = 0; b < sys->n_baths; ++b) {
      int c = 0;
      for (int i = 0; i < sys->n_states; ++i) c += sys->bath_mask[(size_t)b * sys->n_states + i];
      for (int k = 0; k < K1; ++k) m[(size_t)b * K1 + k] = c;
    }
  return m;
}

// Runs the specialised kernels do not cover: several states per bath, a laser field, > 24 states.
bool needs_general(const heom_system *sys) {
  return sys->bath_mask != nullptr || sys->time_dependent || sys->n_states > kMaxStates;
}

int split_of(const Hierarchy &h, int precision) {
  return (precision == HEOM_FP64) ? 0 : (int)std::min<int64_t>(h.n, h.level_off[std::min(2, h.D + 1)]);
}

Layout make_layout(int n, const Hierarchy &h, int u_split, int precision, int64_t max_records, int *Ep,
                   const std::vector<int> *mult = nullptr, int copies = 3) {
  Layout L{};
  const int64_t E = (int64_t)n * n;
  const int64_t n_ado = h.n;
  const size_t be = (precision == HEOM_FP64) ? sizeof(double2) : sizeof(float2);
  const size_t rb = (precision == HEOM_FP64) ? sizeof(LinkRec<double>) : sizeof(LinkRec<float>);
  *Ep = (int)((be == sizeof(float2) && (E & 1)) ? E + 1 : E);
  const int64_t lh = count_links(h, 0, u_split, mult);
  const int64_t lb = (mult ? count_links(h, 0, h.n, mult) : h.n_links) - lh;
  size_t o = 0;
  L.off_loff = o; o = al(o + (size_t)(n_ado + 1) * sizeof(int64_t));
  L.off_rh = o; o = al(o + (size_t)lh * sizeof(LinkRec<double>));
  L.off_rb = o; o = al(o + (size_t)lb * rb);
  L.off_gsum = o; o = al(o + (size_t)n_ado * sizeof(double));
  L.off_rec = o; o = al(o + (size_t)std::max<int64_t>(max_records, 1) * (n + 5) * sizeof(double));
  L.off_w = o; o = al(o + (size_t)n * sizeof(double));
  L.off_cnt = o; o = al(o + 2 * sizeof(int64_t));  // record counter, device error flag
  // stage arguments of grouped launches: batched column-0 (4 stages x 2 VecRunDesc) or work-list (GroupRunDesc)
  L.off_desc = o; o = al(o + std::max(8 * sizeof(VecRunDesc), sizeof(GroupRunDesc)));
  L.head_bytes = al((size_t)u_split * E * sizeof(double2));
  L.body_bytes = al((size_t)(n_ado - u_split) * *Ep * be);
  for (int c = 0; c < copies; ++c) {
    L.off_state[c] = o;
    o = al(o + L.head_bytes + L.body_bytes);
  }
  L.total = o;
  return L;
}

}  // namespace

int heom::cuda_fail(const char *what, cudaError_t e) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return HEOM_E_CUDA;
}

extern "C" int heom_bath_modes(const heom_system *sys, double *gamma, double *c, double *lamnu, int *mode_state,
                               double *term) {
  int rc = check_system_only(sys);
  if (rc) return rc;
  if (!gamma || !c || !lamnu || !mode_state || !term) {
    set_error("heom_bath_modes: NULL output array");
    return HEOM_E_ARG;
  }
  std::vector<double> gam, cc, lnu, tm;
  std::vector<int> ms;
  double gmax = 0;
  if ((rc = compute_modes(sys, gam, cc, lnu, ms, tm, &gmax))) return rc;
  for (size_t l = 0; l < gam.size(); ++l) {
    gamma[l] = gam[l];
    c[l] = cc[l];
    lamnu[l] = lnu[l];
    mode_state[l] = ms[l];
  }
  for (size_t i = 0; i < tm.size(); ++i) term[i] = tm[i];
  return HEOM_OK;
}

extern "C" int heom_run_bytes(const heom_system *sys, const heom_hier *h, int precision, int64_t max_records,
                              size_t *bytes) {
  int rc = check_system(sys, h, precision);
  if (rc) return rc;
  if (!bytes || max_records < 0) { set_error("heom_run_bytes: bad output pointer or max_records"); return HEOM_E_ARG; }
  int Ep;
  const std::vector<int> mult = mode_mult(sys);
  Layout L = make_layout(sys->n_states, h->h, split_of(h->h, precision), precision, max_records, &Ep,
                         sys->bath_mask ? &mult : nullptr, sys->time_dependent ? 4 : 3);
  *bytes = L.total;
  return HEOM_OK;
}


static StateView view_at(char *base, const Layout &L, int c) {
  StateView v;
  v.head = reinterpret_cast<double2 *>(base + L.off_state[c]);
  v.body = base + L.off_state[c] + L.head_bytes;
  return v;
}

int heom::enqueue_record(heom_run *r, bool host_check) {
  if (host_check && r->records_host >= r->max_records) {
    set_error("observable record buffer full (max_records)");
    return HEOM_E_NOMEM;
  }
  record_kernel<<<1, 32, 0, r->stream>>>(r->y, r->u_split, r->precision != HEOM_FP64, r->vec, r->n, r->w_dev, r->records,
                                         r->rec_count, r->max_records);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("record kernel launch", e);
  ++r->records_host;
  ++r->launches;
  return HEOM_OK;
}


extern "C" int heom_run_create(const heom_system *sys, const heom_hier *hh, int precision, int64_t max_records,
                               const double *sigma0_re, const double *sigma0_im, const double *dip_w,
                               void *device_workspace, size_t workspace_bytes, void *cuda_stream, heom_run **out) {
  if (!out) { set_error("heom_run_create: out is NULL"); return HEOM_E_ARG; }
  *out = nullptr;
  int rc = check_system(sys, hh, precision);
  if (rc) return rc;
  if (!sigma0_re || max_records < 1) { set_error("heom_run_create: need sigma0_re and max_records >= 1"); return HEOM_E_ARG; }
  if (!device_workspace || (reinterpret_cast<uintptr_t>(device_workspace) & 255)) {
    set_error("heom_run_create: workspace must be a 256-byte aligned device pointer");
    return HEOM_E_ARG;
  }
  const Hierarchy &h = hh->h;
  const int n = sys->n_states, M = h.M, D = h.D, K = sys->n_matsubara, B = sys->n_baths;
  heom_run *r = new (std::nothrow) heom_run;
  if (!r) { set_error("host allocation failed"); return HEOM_E_NOMEM; }
  r->precision = precision;
  r->n = n; r->M = M; r->D = D; r->K = K; r->B = B;
  r->n_ado = h.n;
  r->u_split = split_of(h, precision);
  r->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  r->max_records = max_records;
  r->gen = needs_general(sys);
  const std::vector<int> mult = mode_mult(sys);
  const std::vector<int> *mp = sys->bath_mask ? &mult : nullptr;  // records per link: 1 without a mask
  Layout L = make_layout(n, h, r->u_split, precision, max_records, &r->Ep, mp, sys->time_dependent ? 4 : 3);
  r->E = n * n;
  if (workspace_bytes < L.total) {
    delete r;
    set_error("workspace too small: need " + std::to_string(L.total) + " bytes");
    return HEOM_E_NOMEM;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&r->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (ce == cudaSuccess && r->u_split > 0) {  // the FP64 head launches run beside the body launches
    ce = cudaStreamCreateWithFlags(&r->side, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&r->join, cudaEventDisableTiming);
  }
  if (ce != cudaSuccess) { delete r; return cuda_fail("device query / head stream", ce); }

  // ---- units and Hamiltonian: H in rad/fs, shifted by h0 = (max + min)/2 of Re diag (exact for
  // the commutator, the only place H enters) to keep the products small in FP32.
  double dmax = -1e300, dmin = 1e300;
  for (int i = 0; i < n; ++i) {
    dmax = std::max(dmax, sys->H_re[i * n + i]);
    dmin = std::min(dmin, sys->H_re[i * n + i]);
  }
  const double h0 = 0.5 * (dmax + dmin);
  r->H.assign((size_t)n * n, 0.0);
  r->Hi.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n * n; ++i) {
    r->H[i] = kCmToRadFs * (sys->H_re[i] - ((i / n == i % n) ? h0 : 0.0));
    r->Hi[i] = sys->H_im ? kCmToRadFs * sys->H_im[i] : 0.0;
    if (r->Hi[i] != 0.0) r->cplx_h = true;
  }
  // With a Hermitian H the real coefficients of the paper's gauge map Hermitian ADOs to Hermitian
  // ADOs; the flag stays on while every uploaded ADO (rho(0) below) is exactly Hermitian.
  r->herm = true;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (sys->H_re[i * n + j] != sys->H_re[j * n + i] ||
          (sys->H_im && sys->H_im[i * n + j] != -sys->H_im[j * n + i]))
        r->herm = false;

  // ---- coherence block (linear-absorption runs): state 0 without a bath, no H element between state
  // 0 and the others, rho(0) supported on column 0 below the diagonal; every ADO then stays of the
  // form sum_a x_a |a><0| and is stored and propagated as that column (vec_kernel.cuh)
  r->vec = n >= 2 && !r->cplx_h && !r->gen;
  for (int b = 0; b < B && r->vec; ++b) r->vec = sys->bath_state[b] != 0;
  for (int a = 1; a < n && r->vec; ++a) r->vec = sys->H_re[a] == 0.0 && sys->H_re[a * n] == 0.0;
  for (int i = 0; i < n && r->vec; ++i)
    for (int j = 0; j < n && r->vec; ++j)
      if (!(j == 0 && i > 0)) r->vec = sigma0_re[i * n + j] == 0.0 && (!sigma0_im || sigma0_im[i * n + j] == 0.0);
  if (r->vec) r->herm = false;

  // ---- bath modes of Eq. HEOM (Drude-Lorentz, Omega = 0), terminator and rescaling
  std::vector<double> gam, cc, lnu, dbath;
  std::vector<int> mstate;
  double gmax = 0;
  if (compute_modes(sys, gam, cc, lnu, mstate, r->term, &gmax, &dbath)) {
    delete r;
    return HEOM_E_ARG;
  }
  r->max_rate = D * gmax;
  if (r->gen) {  // terminator rate of element (i, j): sum_b Delta_b (V_b,ii - V_b,jj)^2
    r->T.assign((size_t)n * n, 0.0);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          const double d = v_diag(sys, b, i) - v_diag(sys, b, j);
          r->T[(size_t)i * n + j] += dbath[b] * d * d;
        }
    r->Ht = r->H;
    r->Hit = r->Hi;
  }

  // ---- rescaling factors s+_l(n), s-_l(n) (section "HEOM formalism", ADO rescaling)
  std::vector<double> sp((size_t)M * (D + 1)), sm((size_t)M * (D + 1));
  for (int l = 0; l < M; ++l) {
    const double ac = std::fabs(cc[l]);
    const bool scaled = sys->rescale && ac >= 1e-300;
    for (int nl = 0; nl <= D; ++nl) {
      sp[(size_t)l * (D + 1) + nl] = scaled ? std::sqrt((nl + 1) * ac) : 1.0;
      sm[(size_t)l * (D + 1) + nl] = scaled ? std::sqrt(nl / ac) : (double)nl;
    }
  }

  // ---- per-ADO link records (CSR), decay sums.  Two passes over ADO ranges on the host threads:
  // the record count of every ADO (then prefix sums: the CSR offsets), then each ADO's records,
  // written at its offset -- the same records in the same order as one pass in u order.
  std::vector<int64_t> loff(h.n + 1, 0);
  std::vector<double> gs(h.n, 0.0);
  std::vector<LinkRec<double>> rh;
  std::vector<LinkRec<double>> rbd;
  std::vector<LinkRec<float>> rbf;
  const bool body_fp64 = precision == HEOM_FP64;
  const int64_t u_split = r->u_split;
  double up_body = 0, dn_body = 0;  // valid up / down links of the body ADOs (flop accounting)
  {
    std::mutex acc_mu;
    const bool ok = host_parallel(h.n, [&](int64_t a, int64_t b) {
      double up = 0, dn = 0;
      for (int64_t u = a; u < b; ++u) {
        int64_t k = 0;
        for (int l = 0; l < M; ++l) {
          const int pv = h.plus[(size_t)u * M + l] >= 0, mv = h.minus[(size_t)u * M + l] >= 0;
          k += (int64_t)(pv + mv) * (mp ? (*mp)[l] : 1);
          if (u >= u_split) {
            up += pv;
            dn += mv;
          }
        }
        loff[u + 1] = k;
      }
      std::lock_guard<std::mutex> lock(acc_mu);
      up_body += up;
      dn_body += dn;
    });
    if (!ok) {
      delete r;
      set_error("host allocation failed (link records)");
      return HEOM_E_NOMEM;
    }
  }
  for (int64_t u = 0; u < h.n; ++u) loff[u + 1] += loff[u];
  const int64_t nlink = loff[h.n];
  r->n_links = nlink;
  r->rec_split = loff[u_split];
  try {
    rh.resize(r->rec_split);
    if (body_fp64) rbd.resize(nlink - r->rec_split);
    else rbf.resize(nlink - r->rec_split);
  } catch (...) {
    delete r;
    set_error("host allocation failed (link records)");
    return HEOM_E_NOMEM;
  }
  struct Pending {
    int v, s;
    double re, im;
  };
  const bool filled = host_parallel(h.n, [&](int64_t a, int64_t b) {
    std::vector<Pending> pend;
    pend.reserve(2 * (size_t)M * (mp ? (size_t)n : 1));
    for (int64_t u = a; u < b; ++u) {
      double g = 0;
      for (int l = 0; l < M; ++l) g += h.tuples[(size_t)u * M + l] * gam[l];
      gs[u] = g;
      pend.clear();
      for (int l = 0; l < M; ++l) {
        const int nl = h.tuples[(size_t)u * M + l];
        for (int dir = 0; dir < 2; ++dir) {
          const int32_t v = dir ? h.minus[(size_t)u * M + l] : h.plus[(size_t)u * M + l];
          if (v < 0) continue;
          double re, im;
          if (dir == 0) {  // up: R = i s+
            re = 0.0;
            im = sp[(size_t)l * (D + 1) + nl];
          } else {  // down: R = s- (lamnu + i c)
            const double f = sm[(size_t)l * (D + 1) + nl];
            re = f * lnu[l];
            im = f * cc[l];
          }
          if (!sys->bath_mask) {
            pend.push_back(Pending{v, mstate[l], re, im});
          } else {  // one record per state of the bath's V (same coefficient)
            const int bb = l / (K + 1);
            for (int st = 0; st < n; ++st)
              if (sys->bath_mask[(size_t)bb * n + st]) pend.push_back(Pending{v, st, re, im});
          }
        }
      }
      // records of one ADO ordered by state (the kernels give all records of a state to one lane);
      // the state field also carries u mod 32 in bits 8..12 (see LinkRec)
      std::stable_sort(pend.begin(), pend.end(), [](const Pending &x, const Pending &y) { return x.s < y.s; });
      const int tag = (int)(u & 31) << 8;
      int64_t k = loff[u];
      for (const Pending &q : pend) {
        if (u < u_split) rh[k] = LinkRec<double>{q.v, q.s | tag, 0, 0, q.re, q.im};
        else if (body_fp64) rbd[k - r->rec_split] = LinkRec<double>{q.v, q.s | tag, 0, 0, q.re, q.im};
        else rbf[k - r->rec_split] = LinkRec<float>{q.v, q.s | tag, (float)q.re, (float)q.im};
        ++k;
      }
    }
  });
  if (!filled) {
    delete r;
    set_error("host allocation failed (link records)");
    return HEOM_E_NOMEM;
  }

  {  // algorithmic bytes and flops of one launch of the dominant kernel (ADOs u >= u_split)
    const double E = (double)n * n;
    const double cs = body_fp64 ? 16.0 : 8.0;
    const double nb = (double)(h.n - r->u_split);
    const double nlb = (double)(nlink - r->rec_split);
    const double tab = nb * 16.0 + nlb * (body_fp64 ? sizeof(LinkRec<double>) : sizeof(LinkRec<float>));
    r->bytes_stage_y = nb * 3.0 * E * cs + tab;
    r->bytes_stage_noy = nb * 2.0 * E * cs + tab;
    const double up = up_body, dn = dn_body;
    // the Hermitian form computes H s only (s H = (H s)^dagger): half the commutator flops
    const double comm = (r->cplx_h ? 16.0 : 8.0) * n * E;
    const double links = up * 8.0 * (n - 1) + dn * 8.0 * (2 * n - 1);
    r->flops_gen = nb * (comm + 8.0 * E) + links;
    r->flops_herm = nb * (0.5 * comm + 8.0 * E) + links;
    r->bytes_full_y = r->bytes_stage_y;
    r->bytes_full_noy = r->bytes_stage_noy;
    r->flops_full = r->flops_gen;
    if (r->vec) {  // column 0 only: N elements per ADO, 8 N^2 flops of H x, one complex FMA per link
      r->bytes_stage_y = nb * 3.0 * n * cs + tab;
      r->bytes_stage_noy = nb * 2.0 * n * cs + tab;
      r->flops_gen = r->flops_herm = nb * (8.0 * n * n + 8.0 * n) + (up + dn) * 8.0;
    }
  }

  char *base = reinterpret_cast<char *>(device_workspace);
  r->link_off = reinterpret_cast<int64_t *>(base + L.off_loff);
  r->recs_head = base + L.off_rh;
  r->recs_body = base + L.off_rb;
  r->gsum = reinterpret_cast<double *>(base + L.off_gsum);
  r->records = reinterpret_cast<double *>(base + L.off_rec);
  r->w_dev = reinterpret_cast<double *>(base + L.off_w);
  r->rec_count = reinterpret_cast<int64_t *>(base + L.off_cnt);
  r->copy_bytes = L.head_bytes + L.body_bytes;
  r->desc_dev = reinterpret_cast<VecRunDesc *>(base + L.off_desc);
  r->err_dev = reinterpret_cast<int *>(base + L.off_cnt + sizeof(int64_t));
  r->y = view_at(base, L, 0);
  r->zA = view_at(base, L, 1);
  r->zB = view_at(base, L, 2);
  if (sys->time_dependent) r->zC = view_at(base, L, 3);

  std::vector<double> w(n, 0.0);
  if (dip_w) for (int i = 0; i < n; ++i) w[i] = dip_w[i];
  cudaStream_t st = r->stream;
  ce = cudaMemcpyAsync(r->link_off, loff.data(), loff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !rh.empty())
    ce = cudaMemcpyAsync(r->recs_head, rh.data(), rh.size() * sizeof(rh[0]), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !rbd.empty())
    ce = cudaMemcpyAsync(r->recs_body, rbd.data(), rbd.size() * sizeof(rbd[0]), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !rbf.empty())
    ce = cudaMemcpyAsync(r->recs_body, rbf.data(), rbf.size() * sizeof(rbf[0]), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(r->gsum, gs.data(), gs.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(r->w_dev, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(r->rec_count, 0, 2 * sizeof(int64_t), st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(base + L.off_state[0], 0, L.head_bytes + L.body_bytes, st);
  // the host vectors are pageable, so each copy has consumed its source when cudaMemcpyAsync returns
  if (ce != cudaSuccess) { delete r; return cuda_fail("workspace upload", ce); }
  // sigma_0 = rho(0): ADO 0 through the host-layout path
  std::vector<double> s0r((size_t)n * n), s0i((size_t)n * n, 0.0);
  for (int i = 0; i < n * n; ++i) { s0r[i] = sigma0_re[i]; if (sigma0_im) s0i[i] = sigma0_im[i]; }
  *out = r;
  rc = heom_set_ados(r, 0, 1, s0r.data(), s0i.data());
  if (rc == HEOM_OK) rc = enqueue_record(r);
  if (rc == HEOM_OK) rc = schedule_new_run(r);
  if (rc != HEOM_OK) { *out = nullptr; delete r; return rc; }
  return HEOM_OK;
}

extern "C" int heom_run_destroy(heom_run *r) {
  delete r;
  return HEOM_OK;
}

extern "C" int heom_record_len(const heom_run *r) { return r ? r->n + 5 : 0; }

// ------------------------------------------------------------------------------------------------
// state I/O through the host layout [count][N][N]; zB is the staging area.

static int64_t staging_ados(const heom_run *r) {
  // zB holds (head + body) bytes; every staged ADO needs 2 * N^2 doubles
  const size_t bytes = (size_t)r->u_split * r->E * sizeof(double2) +
                       (size_t)(r->n_ado - r->u_split) * r->Ep * (r->precision == HEOM_FP64 ? 16 : 8);
  return std::max<int64_t>(1, (int64_t)(bytes / (2 * sizeof(double) * r->n * r->n)));
}

int heom::io_range(heom_run *r, StateView state, int64_t u0, int64_t count, double *re, double *im, bool to_device) {
  if (!r || u0 < 0 || count < 0 || u0 + count > r->n_ado || (count > 0 && (!re || !im))) {
    set_error("ADO range outside the hierarchy or NULL buffer");
    return HEOM_E_ARG;
  }
  const int64_t E = (int64_t)r->n * r->n;
  const int64_t chunk = staging_ados(r);
  double *st_re = reinterpret_cast<double *>(r->zB.head);
  for (int64_t c0 = 0; c0 < count; c0 += chunk) {
    const int64_t cc = std::min(chunk, count - c0);
    double *st_im = st_re + cc * E;
    cudaError_t e;
    if (to_device) {
      e = cudaMemcpyAsync(st_re, re + c0 * E, cc * E * sizeof(double), cudaMemcpyHostToDevice, r->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(st_im, im + c0 * E, cc * E * sizeof(double), cudaMemcpyHostToDevice, r->stream);
      if (e != cudaSuccess) return cuda_fail("state upload", e);
      const int blocks = (int)std::min<int64_t>((cc * E + 255) / 256, 65535);
      scatter_kernel<<<blocks, 256, 0, r->stream>>>(state, r->Ep, r->u_split, r->precision != HEOM_FP64, r->vec, r->n, u0 + c0,
                                                   cc, st_re, st_im);
      ++r->launches;
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail("scatter kernel", e);
      e = cudaStreamSynchronize(r->stream);  // the staging area is reused by the next chunk
      if (e != cudaSuccess) return cuda_fail("state upload sync", e);
    } else {
      const int blocks = (int)std::min<int64_t>((cc * E + 255) / 256, 65535);
      gather_kernel<<<blocks, 256, 0, r->stream>>>(state, r->Ep, r->u_split, r->precision != HEOM_FP64, r->vec, r->n, u0 + c0,
                                                  cc, st_re, st_im);
      ++r->launches;
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail("gather kernel", e);
      e = cudaMemcpyAsync(re + c0 * E, st_re, cc * E * sizeof(double), cudaMemcpyDeviceToHost, r->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(im + c0 * E, st_im, cc * E * sizeof(double), cudaMemcpyDeviceToHost, r->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
      if (e != cudaSuccess) return cuda_fail("state download", e);
    }
  }
  return HEOM_OK;
}

// Leaves the coherence-block layout for good: the current state moves to the matrix layout (through
// zA and host memory, in chunks), then the run uses the matrix kernels.
static int leave_vec(heom_run *r) {
  cudaError_t e = cudaMemcpyAsync(r->zA.head, r->y.head, r->copy_bytes, cudaMemcpyDeviceToDevice, r->stream);
  if (e != cudaSuccess) return cuda_fail("layout change copy", e);
  const int64_t E = (int64_t)r->n * r->n;
  const int64_t chunk = std::max<int64_t>(1, (int64_t)((64u << 20) / (2 * sizeof(double) * E)));
  std::vector<double> hr, hi;
  try {
    hr.resize((size_t)std::min(chunk, r->n_ado) * E);
    hi.resize(hr.size());
  } catch (...) {
    set_error("host allocation failed (layout change)");
    return HEOM_E_NOMEM;
  }
  for (int64_t u0 = 0; u0 < r->n_ado; u0 += chunk) {
    const int64_t cc = std::min(chunk, r->n_ado - u0);
    r->vec = true;
    int rc = io_range(r, r->zA, u0, cc, hr.data(), hi.data(), false);
    r->vec = false;
    if (!rc) rc = io_range(r, r->y, u0, cc, hr.data(), hi.data(), true);
    if (rc) return rc;
  }
  r->bytes_stage_y = r->bytes_full_y;
  r->bytes_stage_noy = r->bytes_full_noy;
  r->flops_gen = r->flops_full;
  r->flops_herm = r->flops_full;
  reschedule_cached(r);  // the matrix-layout kernels: their own cache entries, else the default
  return HEOM_OK;
}

extern "C" int heom_set_ados(heom_run *r, int64_t u0, int64_t count, const double *re, const double *im) {
  if (!r) { set_error("heom_set_ados: NULL run"); return HEOM_E_ARG; }
  if (r->vec && re && im) {  // data outside the coherence block ends the column-0 layout
    const int n = r->n;
    bool in_block = true;
    for (int64_t k = 0; k < count * n * n && in_block; ++k) {
      const int64_t e = k % ((int64_t)n * n), i = e / n, j = e % n;
      if (!(j == 0 && i > 0) && (re[k] != 0.0 || im[k] != 0.0)) in_block = false;
    }
    if (!in_block) {
      int rc = leave_vec(r);
      if (rc) return rc;
    }
  }
  if (r->herm && re && im) {  // a non-Hermitian ADO switches the run to the general kernels for good
    const int n = r->n;
    for (int64_t c = 0; c < count && r->herm; ++c) {
      const double *a = re + c * n * n, *b = im + c * n * n;
      for (int i = 0; i < n && r->herm; ++i)
        for (int j = i; j < n; ++j)
          if (a[i * n + j] != a[j * n + i] || b[i * n + j] != -b[j * n + i]) {
            r->herm = false;
            break;
          }
    }
  }
  return io_range(r, r->y, u0, count, const_cast<double *>(re), const_cast<double *>(im), true);
}

extern "C" int heom_get_ados(heom_run *r, int64_t u0, int64_t count, double *re, double *im) {
  if (!r) { set_error("heom_get_ados: NULL run"); return HEOM_E_ARG; }
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail("heom_get_ados: stream", e);
  return io_range(r, r->y, u0, count, re, im, false);
}

extern "C" int heom_get_sigma0(heom_run *r, double *re, double *im) { return heom_get_ados(r, 0, 1, re, im); }

extern "C" int heom_run_info(const heom_run *r, int64_t *n_ado, int *n_states, int *n_modes, int64_t *steps_done,
                             double *t_fs) {
  if (!r) { set_error("heom_run_info: NULL run"); return HEOM_E_ARG; }
  if (n_ado) *n_ado = r->n_ado;
  if (n_states) *n_states = r->n;
  if (n_modes) *n_modes = r->M;
  if (steps_done) *steps_done = r->steps_done;
  if (t_fs) *t_fs = r->t_fs;
  return HEOM_OK;
}

extern "C" int heom_run_layout(const heom_run *r) { return r ? (r->vec ? 1 : 0) : -1; }

extern "C" int heom_run_set_field(heom_run *r, const heom_field *f) {
  if (!r) { set_error("heom_run_set_field: NULL run"); return HEOM_E_ARG; }
  if (!r->zC.head && !r->zC.body) {
    set_error("heom_run_set_field: the run was created without time_dependent = 1");
    return HEOM_E_STATE;
  }
  if (!f) {
    r->has_field = false;
    return HEOM_OK;
  }
  if (!f->mu_plus || !(f->sigma_fs > 0)) {
    set_error("heom_run_set_field: need mu_plus and sigma_fs > 0");
    return HEOM_E_ARG;
  }
  const int n = r->n;
  r->mup.assign(f->mu_plus, f->mu_plus + (size_t)n * n);
  r->famp = kCmToRadFs * f->amp_cm;
  r->ftc = f->t_center_fs;
  r->fsig = f->sigma_fs;
  r->fphase = f->phase;
  r->fdet = kCmToRadFs * f->detuning_cm;
  r->Ht.assign((size_t)n * n, 0.0);
  r->Hit.assign((size_t)n * n, 0.0);
  r->has_field = true;
  return HEOM_OK;
}

extern "C" int64_t heom_run_launches(const heom_run *r) { return r ? r->launches : -1; }
