// C ABI of libheom (include/heom.h): hierarchy handles, run set-up (units, Matsubara coefficients,
// rescaling tables, workspace layout, table upload), the RK4 driver, observables and state I/O.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/heom.h"
#include "heom_internal.h"

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
  for (int g = 0; g < 4 && rc == 1; ++g) rc = fns[precision][g](c, ch, term, H, Hi, st, sm_count);
  if (rc == 1) {
    set_error("stage kernel: n_states not compiled");
    return -1;
  }
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

// 2 pi c in rad/fs per cm^-1 (c = 2.99792458e-5 cm/fs) and k_B in cm^-1/K (2019 SI, exact ratio).
static const double kCmToRadFs = 2.0 * 3.14159265358979323846 * 2.99792458e-5;
static const double kBoltzCm = 0.6950348004;

}  // namespace heom

using namespace heom;

struct heom_hier {
  Hierarchy h;
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
  VecRunDesc *desc_dev = nullptr;    // [8] stage arguments for batched column-0 launches
  const void *desc_owner = nullptr;  // the batch whose stage arguments desc_dev holds
  std::vector<double> term;          // per state
  double max_rate = 0;               // D * max gamma
  // device
  StateView y{}, zA{}, zB{}, zC{};   // zC: RK4 accumulator of time-dependent runs
  int64_t *link_off = nullptr;       // [n_ado + 1]
  void *recs_head = nullptr;         // LinkRec<double>, ADOs u < u_split
  void *recs_body = nullptr;         // LinkRec<float or double>, ADOs u >= u_split
  int64_t rec_split = 0;             // link_off[u_split]
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
  L.off_desc = o; o = al(o + 8 * sizeof(VecRunDesc));  // batched column-0 stage arguments (4 stages x 2)
  L.head_bytes = al((size_t)u_split * E * sizeof(double2));
  L.body_bytes = al((size_t)(n_ado - u_split) * *Ep * be);
  for (int c = 0; c < copies; ++c) {
    L.off_state[c] = o;
    o = al(o + L.head_bytes + L.body_bytes);
  }
  L.total = o;
  return L;
}

int cuda_fail(const char *what, cudaError_t e) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return HEOM_E_CUDA;
}

}  // namespace

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

namespace heom {
__global__ void record_kernel(StateView y, int u_split, int body_fp32, int vec, int n, const double *w, double *records,
                              int64_t *rec_count, int64_t max_records);
__global__ void scatter_kernel(StateView dst, int Ep, int u_split, int body_fp32, int vec, int n, int64_t u0, int64_t count,
                               const double *re, const double *im);
__global__ void gather_kernel(StateView src, int Ep, int u_split, int body_fp32, int vec, int n, int64_t u0, int64_t count,
                              double *re, double *im);
}  // namespace heom

static StateView view_at(char *base, const Layout &L, int c) {
  StateView v;
  v.head = reinterpret_cast<double2 *>(base + L.off_state[c]);
  v.body = base + L.off_state[c] + L.head_bytes;
  return v;
}

static int enqueue_record(heom_run *r) {
  if (r->records_host >= r->max_records) {
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

namespace {
int schedule_new_run(heom_run *r);  // the autotuner (below)
void reschedule_cached(heom_run *r);
}  // namespace

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

  // ---- per-ADO link records (CSR), decay sums
  std::vector<int64_t> loff(h.n + 1, 0);
  std::vector<double> gs(h.n, 0.0);
  std::vector<LinkRec<double>> rh;
  std::vector<LinkRec<double>> rbd;
  std::vector<LinkRec<float>> rbf;
  const bool body_fp64 = precision == HEOM_FP64;
  try {
    const int64_t lh = count_links(h, 0, r->u_split, mp);
    const int64_t lt = mp ? count_links(h, 0, h.n, mp) : h.n_links;
    rh.reserve(lh);
    if (body_fp64) rbd.reserve(lt - lh);
    else rbf.reserve(lt - lh);
  } catch (...) {
    delete r;
    set_error("host allocation failed (link records)");
    return HEOM_E_NOMEM;
  }
  int64_t nlink = 0;
  struct Pending {
    int v, s;
    double re, im;
  };
  std::vector<Pending> pend;
  pend.reserve(2 * (size_t)M);
  for (int64_t u = 0; u < h.n; ++u) {
    loff[u] = nlink;
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
          const int b = l / (K + 1);
          for (int st = 0; st < n; ++st)
            if (sys->bath_mask[(size_t)b * n + st]) pend.push_back(Pending{v, st, re, im});
        }
      }
    }
    // records of one ADO ordered by state (the kernels give all records of a state to one lane);
    // the state field also carries u mod 32 in bits 8..12 (see LinkRec)
    std::stable_sort(pend.begin(), pend.end(), [](const Pending &x, const Pending &y) { return x.s < y.s; });
    const int tag = (int)(u & 31) << 8;
    for (const Pending &q : pend) {
      if (u < r->u_split) {
        rh.push_back(LinkRec<double>{q.v, q.s | tag, 0, 0, q.re, q.im});
      } else if (body_fp64) {
        rbd.push_back(LinkRec<double>{q.v, q.s | tag, 0, 0, q.re, q.im});
      } else {
        rbf.push_back(LinkRec<float>{q.v, q.s | tag, (float)q.re, (float)q.im});
      }
      ++nlink;
    }
  }
  loff[h.n] = nlink;
  r->rec_split = loff[r->u_split];

  {  // algorithmic bytes and flops of one launch of the dominant kernel (ADOs u >= u_split)
    const double E = (double)n * n;
    const double cs = body_fp64 ? 16.0 : 8.0;
    const double nb = (double)(h.n - r->u_split);
    const double nlb = (double)(nlink - r->rec_split);
    const double tab = nb * 16.0 + nlb * (body_fp64 ? sizeof(LinkRec<double>) : sizeof(LinkRec<float>));
    r->bytes_stage_y = nb * 3.0 * E * cs + tab;
    r->bytes_stage_noy = nb * 2.0 * E * cs + tab;
    double up = 0, dn = 0;
    for (int64_t u = r->u_split; u < h.n; ++u)
      for (int l = 0; l < M; ++l) {
        up += h.plus[(size_t)u * M + l] >= 0;
        dn += h.minus[(size_t)u * M + l] >= 0;
      }
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
// propagation: classic RK4 of a linear, time-independent right-hand side, evaluated in Horner form
//   y_{t+h} = y + h L (y + h/2 L (y + h/3 L (y + h/4 L y)))
// which is the same degree-4 polynomial as the four-stage classic tableau and needs three state
// copies (y, zA, zB) instead of four.

static StageCommon common_for(const heom_run *r, StateView zin, StateView y, StateView out) {
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
static int launch_head(heom_run *r, StageCommon c, double ch, cudaStream_t s) {
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
static int launch_body(heom_run *r, StageCommon c, double ch, cudaStream_t s) {
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
static void field_H(heom_run *r, double t) {
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

static int run_stage(heom_run *r, StateView zin, StateView y, StateView out, double ch) {
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

// ------------------------------------------------------------------------------------------------
// launch schedules and the autotuner: every candidate is timed on the run's own stage-1 launch
// (zin = y, out = zA; y is not written) and the fastest is kept, per run and in a process-wide
// cache.  All schedules compute the same sums in the same order, so the choice changes only time.

namespace {
std::mutex g_tune_mu;                                    // guards the cache
std::map<std::array<int, 7>, heom_schedule> g_tune_cache;  // (layout, precision, part, n, herm, cplx, log2 ADOs)
std::atomic<int> g_autotune{3};                          // timed launches per candidate at creation (0: off)
heom_schedule g_default[3] = {{100, 1}, {100, 1}, {100, 1}};  // per layout, without cache entry or tuning

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

bool valid_schedule(const heom_schedule &s) {
  return s.occupancy_pct >= 1 && s.occupancy_pct <= 100 &&
         (s.chunks_per_warp == 1 || s.chunks_per_warp == 2 || s.chunks_per_warp == 4);
}

std::array<int, 7> run_key(const heom_run *r, int part) {
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

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

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

int tune_part(heom_run *r, int part, int reps, std::vector<heom_schedule> &tried, std::vector<double> &ms) {
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
}  // namespace

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
    set_error("heom_set_schedule: need a run, part 0 or 1 (1 only with an FP64 head), occupancy_pct 1..100, "
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

// ------------------------------------------------------------------------------------------------
// state I/O through the host layout [count][N][N]; zB is the staging area.

static int64_t staging_ados(const heom_run *r) {
  // zB holds (head + body) bytes; every staged ADO needs 2 * N^2 doubles
  const size_t bytes = (size_t)r->u_split * r->E * sizeof(double2) +
                       (size_t)(r->n_ado - r->u_split) * r->Ep * (r->precision == HEOM_FP64 ? 16 : 8);
  return std::max<int64_t>(1, (int64_t)(bytes / (2 * sizeof(double) * r->n * r->n)));
}

static int io_range(heom_run *r, StateView state, int64_t u0, int64_t count, double *re, double *im, bool to_device) {
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

// ------------------------------------------------------------------------------------------------
// small kernels

namespace heom {

__device__ __forceinline__ double2 ld_any(const StateView &s, int E, int Ep, int u_split, int body_fp32, int64_t v,
                                          int64_t e) {
  if (v < u_split) return s.head[v * E + e];
  if (body_fp32) {
    const float2 f = reinterpret_cast<const float2 *>(s.body)[(v - u_split) * Ep + e];
    return make_double2(f.x, f.y);
  }
  return reinterpret_cast<const double2 *>(s.body)[(v - u_split) * Ep + e];
}

// Element e = i n + j of ADO v in the run's layout: matrix tiles, or (vec) column 0 only.
__device__ __forceinline__ double2 ld_elem(const StateView &s, int n, int Ep, int u_split, int body_fp32, int vec,
                                           int64_t v, int64_t e) {
  if (!vec) return ld_any(s, n * n, Ep, u_split, body_fp32, v, e);
  const int64_t i = e / n, j = e - i * n;
  if (j != 0) return make_double2(0.0, 0.0);
  return ld_any(s, n, n, u_split, body_fp32, v, i);
}

// One observable record of sigma_0 (FP64): populations, trace, dipole correlation, Hermiticity.
__global__ void record_kernel(StateView y, int u_split, int body_fp32, int vec, int n, const double *w, double *records,
                              int64_t *rec_count, int64_t max_records) {
  // one warp: lane a handles rows a, a + 32, ...; sums and the maximum are reduced across the warp
  const int lane = threadIdx.x & 31;
  const int64_t idx = *rec_count;
  if (idx >= max_records) return;
  const int E = n * n;
  double *rec = records + idx * (n + 5);
  double tr = 0, ti = 0, cr = 0, ci = 0, herm = 0;
  for (int a = lane; a < n; a += 32) {
    const double2 d = ld_elem(y, n, E, u_split, body_fp32, vec, 0, (int64_t)a * n + a);
    rec[a] = d.x;
    tr += d.x;
    ti += d.y;
    const double2 c0 = ld_elem(y, n, E, u_split, body_fp32, vec, 0, (int64_t)a * n);
    cr += w[a] * c0.x;
    ci += w[a] * c0.y;
    for (int b = 0; b < n; ++b) {
      const double2 x = ld_elem(y, n, E, u_split, body_fp32, vec, 0, (int64_t)a * n + b);
      const double2 z = ld_elem(y, n, E, u_split, body_fp32, vec, 0, (int64_t)b * n + a);
      herm = fmax(herm, hypot(x.x - z.x, x.y + z.y));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_down_sync(0xffffffffu, tr, o);
    ti += __shfl_down_sync(0xffffffffu, ti, o);
    cr += __shfl_down_sync(0xffffffffu, cr, o);
    ci += __shfl_down_sync(0xffffffffu, ci, o);
    herm = fmax(herm, __shfl_down_sync(0xffffffffu, herm, o));
  }
  if (lane == 0) {
    rec[n] = tr;
    rec[n + 1] = ti;
    rec[n + 2] = cr;
    rec[n + 3] = ci;
    rec[n + 4] = herm;
    *rec_count = idx + 1;
  }
}

__global__ void scatter_kernel(StateView dst, int Ep, int u_split, int body_fp32, int vec, int n, int64_t u0, int64_t count,
                               const double *re, const double *im) {
  const int64_t E = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count * E; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / E;
    int64_t e = t - c * E;
    const int64_t v = u0 + c;
    int64_t TE = E, TP = Ep;
    if (vec) {  // column 0 only (the host checked that the rest is zero)
      if (e % n != 0) continue;
      e /= n;
      TE = n;
      TP = n;
    }
    if (v < u_split) {
      dst.head[v * TE + e] = make_double2(re[t], im[t]);
    } else if (body_fp32) {
      reinterpret_cast<float2 *>(dst.body)[(v - u_split) * TP + e] = make_float2((float)re[t], (float)im[t]);
    } else {
      reinterpret_cast<double2 *>(dst.body)[(v - u_split) * TP + e] = make_double2(re[t], im[t]);
    }
  }
}

__global__ void gather_kernel(StateView src, int Ep, int u_split, int body_fp32, int vec, int n, int64_t u0, int64_t count,
                              double *re, double *im) {
  const int64_t E = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count * E; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / E, e = t - c * E;
    const double2 d = ld_elem(src, n, Ep, u_split, body_fp32, vec, u0 + c, e);
    re[t] = d.x;
    im[t] = d.y;
  }
}

}  // namespace heom

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
          const int64_t l0 = r->launches, rec0 = r->records_host, max0 = r->max_records;
          r->stream = b->gstream[g];
          r->max_records = INT64_MAX;
          rc = enqueue_record(r);
          b->launches_per_replay[i] += r->launches - l0;
          r->launches = l0;
          r->records_host = rec0;  // advanced by heom_batch_launch
          r->max_records = max0;
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
    const int64_t l0 = r->launches, rec0 = r->records_host, max0 = r->max_records;
    r->stream = b->pool[i % P];
    r->max_records = INT64_MAX;  // counters are restored below; launches advance them
    for (int64_t s = 0; s < steps_per_launch && rc == HEOM_OK; ++s) {
      if ((rc = run_stage(r, r->y, r->y, r->zA, h / 4))) break;
      if ((rc = run_stage(r, r->zA, r->y, r->zB, h / 3))) break;
      if ((rc = run_stage(r, r->zB, r->y, r->zA, h / 2))) break;
      if ((rc = run_stage(r, r->zA, r->y, r->y, h))) break;
      if (obs_stride > 0 && (s + 1) % obs_stride == 0) rc = enqueue_record(r);
    }
    b->launches_per_replay[i] = r->launches - l0;
    r->launches = l0;
    r->records_host = rec0;
    r->max_records = max0;
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
