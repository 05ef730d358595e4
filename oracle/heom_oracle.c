/*
 * heom_oracle.c -- plain, slow, FP64 CPU statement of the HEOM right-hand side and its classic
 * RK4 integration, written from the paper (Kramer, Noack, Reinefeld, Rodriguez, Zhang,
 * "Efficient calculation of open quantum system dynamics and time-resolved spectroscopy with
 * Distributed Memory HEOM (DM-HEOM)", arXiv 1803.03498).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference
 * arm of bench.py load this library.  It shares no code, header, table or constant with the CUDA
 * library in paper_1803_03498_gb300/; the two are independent statements of the same method.
 *
 * What each part follows:
 *   - hierarchy (tuples, numbering, +/- links): section "HEOM formalism", Eq. (Nmatrices) and the
 *     paragraph on "+" and "-" vertices; mode index l = (b-1)K + k + 1 (0-based here: l = b*K + k).
 *     The paper leaves the order of the consecutive numbering u open; this oracle orders tuples by
 *     level |n| and, inside a level, by colexicographic order of the stars-and-bars bar positions
 *     (a sort with an explicit comparator, not a ranking formula).
 *   - bath coefficients gamma(b,k), c(b,k) and the terminator: Eq. (HEOM) and its definitions
 *     (Matsubara expansion of a Drude-Lorentz density, Omega = 0), or the Pade expansion that
 *     replaces them (same section, the Pade spectrum decomposition; see orc_pade).
 *   - right-hand side: Eq. (HEOM) term by term, with the superoperators V^x, V^x V^x and V^o
 *     written with the Kronecker deltas of their element-wise definitions, and the ADO rescaling
 *     (section "HEOM formalism", last two substitutions).
 *   - integrator: classic four-stage Runge-Kutta with four ADO copies (section "HEOM memory and
 *     compute requirements" and "Distributed memory HEOM implementation"); a time-dependent
 *     Hamiltonian is evaluated at each stage's time t, t + h/2, t + h/2, t + h.
 *   - laser field in the rotating-wave approximation (section "Optical spectra", Eq. h-field-rwa
 *     with Eq. probe_pulse): H(t) = H - g(t) M+ - conj(g(t)) M-, M- = (M+)^T, with the envelope
 *     g(t) = E0 exp(-(t - t_c)^2 / (2 sigma^2)) exp(-i (Delta t + phi)) seen from the frame that
 *     rotates at the reference frequency subtracted from every excitation (Delta = carrier minus
 *     reference, phi the pulse phase); M+ = e . mu^+ is the polarisation-weighted dipole operator.
 *   - two-exciton space (section "Dipole operators and rotational averaging"): the bath of site b
 *     couples through its site-number operator, a diagonal V_b with 1 at every state that has site
 *     b excited (orc_set_bath_mask); V^x, V^x V^x and V^o keep their element-wise definitions for
 *     any diagonal V.
 *   - observables: rho = sigma_0; site populations; trace; the linear-absorption dipole
 *     correlation sum_a w_a sigma_0[a][0] (Eq. lin_abs_mukamel with mu^+ |0><0| as start).
 *
 * Units: energies in cm^-1 are turned into angular frequencies in rad/fs by 2*pi*c with
 * c = 2.99792458e-5 cm/fs; hbar = 1 in these units; times in fs; beta = 1/(k_B T) with
 * k_B = 0.6950348004 cm^-1/K (exact from the 2019 SI constants).  The paper is silent on units.
 *
 * Readings of the paper (each also listed in the project's design notes):
 *   - one bath per coupled state (S(b) = 1): V_b = |s_b><s_b|; several baths may share a state;
 *     in the two-exciton space V_b is the number operator of site b (a 0/1 diagonal).
 *   - K here is the number of Matsubara terms beyond the Drude term, so each bath has K+1 modes.
 *   - hbar = 1 throughout (the paper's hbar placement is not consistent).
 *   - the rescaling uses |c(b,k)| of the real c of the paper; when |c| < 1e-300 the mode is left
 *     unscaled (up factor 1, down factor n).
 *   - The paper prints its dynamics as figures only (no tabulated values); the pins of this oracle
 *     are closed forms, invariants, special cases and independent constructions (tests/).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO_PI_C 1.8836515673088532e-4 /* rad/fs per cm^-1 */
#define ORC_KB_CM 0.6950348004             /* cm^-1 per K */
#define ORC_PI 3.14159265358979323846

typedef double complex cplx;

typedef struct {
  int M, D;
  int64_t n;          /* number of tuples */
  uint8_t *tuples;    /* [n][M] */
  int32_t *plus;      /* [n][M], -1 if invalid */
  int32_t *minus;     /* [n][M], -1 if invalid */
} orc_hier;

typedef struct {
  int N;              /* n_states */
  cplx *H;            /* [N][N] rad/fs, at the current time (orc_set_time) */
  cplx *H0;           /* [N][N] rad/fs, without the field */
  double *vmask;      /* [B][N]: the diagonal of V_b (0 or 1) */
  int has_field;      /* laser field (orc_set_field) */
  double *mup;        /* [N][N] M+ (real) */
  double famp, ftc, fsig, fphase, fdet; /* rad/fs, fs, fs, rad, rad/fs */
  int B, K;           /* baths, Matsubara terms beyond Drude (modes per bath = K+1) */
  int *bath_state;    /* [B] */
  double *lambda, *nu, *beta; /* [B] rad/fs, 1/fs, fs */
  int terminator, rescale;
  /* per mode l = b*(K+1) + k */
  int M;
  double *gamma, *c, *lamnu; /* lamnu = lambda*nu for k = 0, else 0 */
  double *delta_b;           /* [B] terminator coefficient */
  orc_hier h;
} orc_model;

/* ------------------------------------------------------------------------------------------ */
/* Hierarchy: all n in N^M with |n| <= D (Eq. Nmatrices), sorted by (level, colex of bars).    */

static int g_cmp_M; /* comparator context (single-threaded oracle) */

static void bars_of(const uint8_t *n, int M, int *b) {
  /* bar j (j = 1..M-1) sits after the stars of modes 1..j: b_j = (j-1) + sum_{i<=j} n_i */
  int s = 0;
  for (int j = 1; j <= M - 1; ++j) {
    s += n[j - 1];
    b[j - 1] = (j - 1) + s;
  }
}

static int level_of(const uint8_t *n, int M) {
  int s = 0;
  for (int i = 0; i < M; ++i) s += n[i];
  return s;
}

static int tuple_cmp(const void *pa, const void *pb) {
  const uint8_t *a = (const uint8_t *)pa, *b = (const uint8_t *)pb;
  int M = g_cmp_M;
  int la = level_of(a, M), lb = level_of(b, M);
  if (la != lb) return la < lb ? -1 : 1;
  if (M <= 1) return 0;
  int ba[256], bb[256];
  bars_of(a, M, ba);
  bars_of(b, M, bb);
  /* colex: the set whose largest differing element is smaller comes first */
  for (int j = M - 2; j >= 0; --j)
    if (ba[j] != bb[j]) return ba[j] < bb[j] ? -1 : 1;
  return 0;
}

static void enum_rec(int M, int D, int pos, int left, uint8_t *cur, uint8_t *out, int64_t *cnt) {
  if (pos == M) {
    memcpy(out + (*cnt) * M, cur, (size_t)M);
    ++*cnt;
    return;
  }
  for (int v = 0; v <= left; ++v) {
    cur[pos] = (uint8_t)v;
    enum_rec(M, D, pos + 1, left - v, cur, out, cnt);
  }
  cur[pos] = 0;
}

static int64_t count_rec(int M, int pos, int left) {
  if (pos == M) return 1;
  int64_t s = 0;
  for (int v = 0; v <= left; ++v) s += count_rec(M, pos + 1, left - v);
  return s;
}

/* Lookup of a tuple's position: open-addressing hash table over the tuple bytes (FNV-1a). */
typedef struct {
  int64_t cap;
  int64_t *slot; /* position in the sorted tuple list, -1 = empty */
} orc_index;

static uint64_t fnv1a(const uint8_t *k, int M) {
  uint64_t h = 1469598103934665603ULL;
  for (int i = 0; i < M; ++i) { h ^= k[i]; h *= 1099511628211ULL; }
  return h;
}

static int index_build(orc_index *ix, const orc_hier *h) {
  ix->cap = 1;
  while (ix->cap < 2 * h->n + 1) ix->cap <<= 1;
  ix->slot = (int64_t *)malloc(sizeof(int64_t) * ix->cap);
  if (!ix->slot) return -3;
  for (int64_t i = 0; i < ix->cap; ++i) ix->slot[i] = -1;
  for (int64_t u = 0; u < h->n; ++u) {
    uint64_t p = fnv1a(h->tuples + u * h->M, h->M) & (uint64_t)(ix->cap - 1);
    while (ix->slot[p] >= 0) p = (p + 1) & (uint64_t)(ix->cap - 1);
    ix->slot[p] = u;
  }
  return 0;
}

static int64_t find_tuple(const orc_hier *h, const orc_index *ix, const uint8_t *key) {
  uint64_t p = fnv1a(key, h->M) & (uint64_t)(ix->cap - 1);
  while (ix->slot[p] >= 0) {
    if (memcmp(h->tuples + ix->slot[p] * h->M, key, (size_t)h->M) == 0) return ix->slot[p];
    p = (p + 1) & (uint64_t)(ix->cap - 1);
  }
  return -1;
}

static int hier_build(orc_hier *h, int M, int D) {
  if (M < 1 || M > 256 || D < 0 || D > 255) return -1;
  h->M = M;
  h->D = D;
  h->n = count_rec(M, 0, D); /* brute-force count, pinned against C(M+D, D) in the tests */
  if (h->n > INT32_MAX) return -2;
  h->tuples = (uint8_t *)calloc((size_t)h->n * M, 1);
  h->plus = (int32_t *)malloc((size_t)h->n * M * sizeof(int32_t));
  h->minus = (int32_t *)malloc((size_t)h->n * M * sizeof(int32_t));
  if (!h->tuples || !h->plus || !h->minus) return -3;
  uint8_t cur[256] = {0};
  int64_t cnt = 0;
  enum_rec(M, D, 0, D, cur, h->tuples, &cnt);
  g_cmp_M = M;
  qsort(h->tuples, (size_t)h->n, (size_t)M, tuple_cmp);
  orc_index ix;
  if (index_build(&ix, h)) return -3;
  /* "+" link: n + e_l valid iff |n| + 1 <= D.  "-" link: n - e_l valid iff n_l >= 1. */
  uint8_t key[256];
  for (int64_t u = 0; u < h->n; ++u) {
    const uint8_t *nu = h->tuples + u * M;
    int L = level_of(nu, M);
    for (int l = 0; l < M; ++l) {
      memcpy(key, nu, (size_t)M);
      if (L + 1 <= D) {
        key[l] = (uint8_t)(nu[l] + 1);
        h->plus[u * M + l] = (int32_t)find_tuple(h, &ix, key);
      } else {
        h->plus[u * M + l] = -1;
      }
      memcpy(key, nu, (size_t)M);
      if (nu[l] >= 1) {
        key[l] = (uint8_t)(nu[l] - 1);
        h->minus[u * M + l] = (int32_t)find_tuple(h, &ix, key);
      } else {
        h->minus[u * M + l] = -1;
      }
    }
  }
  free(ix.slot);
  return 0;
}

static void hier_free(orc_hier *h) {
  free(h->tuples);
  free(h->plus);
  free(h->minus);
  memset(h, 0, sizeof(*h));
}

int64_t orc_hier_count(int M, int D) {
  if (M < 1 || D < 0) return -1;
  return count_rec(M, 0, D);
}

/* Build the hierarchy and copy it out: tuples [n][M] uint8, plus/minus [n][M] int32. */
int orc_hier_export(int M, int D, int64_t cap, uint8_t *tuples, int32_t *plus, int32_t *minus) {
  orc_hier h;
  memset(&h, 0, sizeof(h));
  int rc = hier_build(&h, M, D);
  if (rc) { hier_free(&h); return rc; }
  if (h.n > cap) { hier_free(&h); return -4; }
  memcpy(tuples, h.tuples, (size_t)h.n * M);
  memcpy(plus, h.plus, (size_t)h.n * M * sizeof(int32_t));
  memcpy(minus, h.minus, (size_t)h.n * M * sizeof(int32_t));
  hier_free(&h);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Model set-up: units and the Matsubara coefficients of Eq. (HEOM).                           */

void orc_destroy(orc_model *m) {
  if (!m) return;
  free(m->H);
  free(m->H0);
  free(m->vmask);
  free(m->mup);
  free(m->bath_state);
  free(m->lambda);
  free(m->nu);
  free(m->beta);
  free(m->gamma);
  free(m->c);
  free(m->lamnu);
  free(m->delta_b);
  hier_free(&m->h);
  free(m);
}

/* Eigenvalues of the symmetric n x n matrix a (row-major, overwritten) by cyclic Jacobi rotations:
 * each rotation in the (p, q) plane zeroes a_pq; sweeps repeat until the off-diagonal part vanishes.
 * ev receives the diagonal, i.e. the eigenvalues, in no particular order. */
static void jacobi_eigenvalues(double *a, int n, double *ev) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a[p * n + q];
        if (apq == 0.0) continue;
        double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) { /* columns p, q */
          double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* rows p, q */
          double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
}

static int desc_cmp(const void *x, const void *y) {
  double a = *(const double *)x, b = *(const double *)y;
  return (a < b) - (a > b);
}

/* Pade spectrum decomposition of the Bose function used by the paper (section "HEOM formalism", the
 * Pade expansion it takes from its reference Hu, Xu, Yan 2010):
 *   1/(1 - exp(-x)) ~ 1/x + 1/2 + sum_{i=1..K} 2 eta_i x / (x^2 + xi_i^2)
 * with xi_i = 2 / (i-th largest eigenvalue of Lambda), Lambda_{m,m+1} = 1/sqrt((2m+1)(2m+3)),
 * m = 1..2K; zeta_j likewise from Lambda' (size 2K-1, entries 1/sqrt((2m+3)(2m+5)));
 * eta_i = K (2K+3)/2 prod_{j<K} (zeta_j^2 - xi_i^2) / prod_{j != i} (xi_j^2 - xi_i^2).
 * (The paper's printed eta pairs zeta_j with xi_j; it is read with xi_i, the form for which the
 * sum above reproduces the Bose function.)  xi, eta: [K].  Returns 0, or -1 for K < 1. */
int orc_pade(int K, double *xi, double *eta) {
  if (K < 1) return -1;
  int n = 2 * K, n2 = 2 * K - 1;
  double *a = (double *)calloc((size_t)n * n, sizeof(double));
  double *ev = (double *)malloc(sizeof(double) * n);
  double *zeta = (double *)malloc(sizeof(double) * (K > 1 ? K - 1 : 1));
  for (int m = 1; m < n; ++m) a[(m - 1) * n + m] = a[m * n + m - 1] = 1.0 / sqrt((2.0 * m + 1) * (2.0 * m + 3));
  jacobi_eigenvalues(a, n, ev);
  qsort(ev, n, sizeof(double), desc_cmp);
  for (int i = 0; i < K; ++i) xi[i] = 2.0 / ev[i];
  if (K > 1) {
    memset(a, 0, sizeof(double) * (size_t)n * n);
    for (int m = 1; m < n2; ++m) a[(m - 1) * n2 + m] = a[m * n2 + m - 1] = 1.0 / sqrt((2.0 * m + 3) * (2.0 * m + 5));
    jacobi_eigenvalues(a, n2, ev);
    qsort(ev, n2, sizeof(double), desc_cmp);
    for (int j = 0; j < K - 1; ++j) zeta[j] = 2.0 / ev[j];
  }
  for (int i = 0; i < K; ++i) {
    double num = 1.0, den = 1.0;
    for (int j = 0; j < K - 1; ++j) num *= zeta[j] * zeta[j] - xi[i] * xi[i];
    for (int j = 0; j < K; ++j)
      if (j != i) den *= xi[j] * xi[j] - xi[i] * xi[i];
    eta[i] = K * (2.0 * K + 3.0) / 2.0 * num / den;
  }
  free(a);
  free(ev);
  free(zeta);
  return 0;
}

/* H_re/H_im: [N][N] row-major in cm^-1 (H_im may be NULL).  decomposition 0: Matsubara expansion,
 * 1: Pade expansion with K poles.  Returns NULL on bad input. */
orc_model *orc_create(int N, const double *H_re, const double *H_im, int B, const int *bath_state,
                      const double *lambda_cm, const double *tau_fs, const double *T_K, int K,
                      int D, int terminator, int rescale, int decomposition) {
  if (N < 1 || B < 1 || K < 0 || D < 0 || decomposition < 0 || decomposition > 1) return NULL;
  double pxi[64], peta[64];
  if (decomposition == 1 && K > 64) return NULL;
  if (decomposition == 1 && K > 0) orc_pade(K, pxi, peta);
  orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
  m->N = N;
  m->B = B;
  m->K = K;
  m->terminator = terminator;
  m->rescale = rescale;
  m->H = (cplx *)malloc(sizeof(cplx) * N * N);
  m->H0 = (cplx *)malloc(sizeof(cplx) * N * N);
  for (int i = 0; i < N * N; ++i) {
    m->H0[i] = ORC_TWO_PI_C * (H_re[i] + I * (H_im ? H_im[i] : 0.0));
    m->H[i] = m->H0[i];
  }
  m->vmask = (double *)calloc((size_t)B * N, sizeof(double));
  m->bath_state = (int *)malloc(sizeof(int) * B);
  m->lambda = (double *)malloc(sizeof(double) * B);
  m->nu = (double *)malloc(sizeof(double) * B);
  m->beta = (double *)malloc(sizeof(double) * B);
  m->delta_b = (double *)malloc(sizeof(double) * B);
  m->M = B * (K + 1);
  m->gamma = (double *)malloc(sizeof(double) * m->M);
  m->c = (double *)malloc(sizeof(double) * m->M);
  m->lamnu = (double *)malloc(sizeof(double) * m->M);
  for (int b = 0; b < B; ++b) {
    if (bath_state[b] < 0 || bath_state[b] >= N) { orc_destroy(m); return NULL; }
    m->bath_state[b] = bath_state[b];
    m->vmask[(size_t)b * N + bath_state[b]] = 1.0;  /* V_b = |s_b><s_b| */
    m->lambda[b] = ORC_TWO_PI_C * lambda_cm[b];
    m->nu[b] = 1.0 / tau_fs[b];
    m->beta[b] = 1.0 / (ORC_TWO_PI_C * ORC_KB_CM * T_K[b]);
    double lam = m->lambda[b], nu = m->nu[b], beta = m->beta[b];
    double sum_c_over_gamma = 0.0;
    for (int k = 0; k <= K; ++k) {
      int l = b * (K + 1) + k;
      double g, c;
      if (k == 0) {
        g = nu;                                      /* gamma(b,0) = nu_b */
        if (decomposition == 0) {
          c = nu * lam / tan(beta * nu / 2.0);       /* c(b,0) = nu lambda cot(beta nu / 2) */
        } else {                                     /* c(b,0) = 2 lambda / beta (1 - sum_j ...) */
          double sum = 0.0;
          for (int j = 0; j < K; ++j) {
            double gj = pxi[j] / beta;
            sum += 2.0 * peta[j] * nu * nu / (gj * gj - nu * nu);
          }
          c = 2.0 * lam / beta * (1.0 - sum);
        }
      } else {
        if (decomposition == 0) {
          g = 2.0 * ORC_PI * k / beta;                 /* gamma(b,k) = 2 pi k / beta */
        } else {
          g = pxi[k - 1] / beta;                       /* gamma(b,k) = xi_k / beta */
        }
        if (fabs(g * g - nu * nu) < 1e-6 * g * g) { orc_destroy(m); return NULL; } /* gamma_k = nu */
        c = 4.0 * lam * nu / beta * g / (g * g - nu * nu);
        if (decomposition == 1) c *= peta[k - 1];    /* c(b,k) = ... eta_k ... */
      }
      m->gamma[l] = g;
      m->c[l] = c;
      m->lamnu[l] = (k == 0) ? lam * nu : 0.0;
      sum_c_over_gamma += c / g;
    }
    /* terminator: 2 lambda / (beta nu) - sum_k c(b,k) / gamma(b,k) */
    m->delta_b[b] = 2.0 * lam / (beta * nu) - sum_c_over_gamma;
  }
  memset(&m->h, 0, sizeof(m->h));
  if (hier_build(&m->h, m->M, D)) { orc_destroy(m); return NULL; }
  return m;
}

/* V_b as a 0/1 diagonal over the states (mask [B][N]), replacing |s_b><s_b|: the number operator
 * of site b in the two-exciton space.  Returns -1 on a value other than 0 or 1. */
int orc_set_bath_mask(orc_model *m, const uint8_t *mask) {
  for (int64_t e = 0; e < (int64_t)m->B * m->N; ++e)
    if (mask[e] > 1) return -1;
  for (int64_t e = 0; e < (int64_t)m->B * m->N; ++e) m->vmask[e] = (double)mask[e];
  return 0;
}

/* H(t) = H0 - g(t) M+ - conj(g(t)) (M+)^T with g(t) = E0 exp(-(t - t_c)^2 / (2 sigma^2))
 * exp(-i (Delta t + phi)); E0 and Delta in cm^-1.  mu_plus == NULL removes the field. */
int orc_set_field(orc_model *m, const double *mu_plus, double amp_cm, double t_center_fs, double sigma_fs,
                  double phase, double detuning_cm) {
  if (!mu_plus) {
    m->has_field = 0;
    return 0;
  }
  if (!(sigma_fs > 0)) return -1;
  const int N = m->N;
  if (!m->mup) m->mup = (double *)malloc(sizeof(double) * N * N);
  memcpy(m->mup, mu_plus, sizeof(double) * N * N);
  m->famp = ORC_TWO_PI_C * amp_cm;
  m->ftc = t_center_fs;
  m->fsig = sigma_fs;
  m->fphase = phase;
  m->fdet = ORC_TWO_PI_C * detuning_cm;
  m->has_field = 1;
  return 0;
}

/* The Hamiltonian that orc_rhs uses from now on: H(t). */
void orc_set_time(orc_model *m, double t_fs) {
  const int N = m->N;
  if (!m->has_field) {
    for (int e = 0; e < N * N; ++e) m->H[e] = m->H0[e];
    return;
  }
  const double x = (t_fs - m->ftc) / m->fsig;
  const cplx g = m->famp * exp(-0.5 * x * x) * cexp(-I * (m->fdet * t_fs + m->fphase));
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      m->H[i * N + j] = m->H0[i * N + j] - g * m->mup[i * N + j] - conj(g) * m->mup[j * N + i];
}

int64_t orc_n_ado(const orc_model *m) { return m->h.n; }
int orc_n_modes(const orc_model *m) { return m->M; }

/* gamma, c, lamnu: [M]; mode_state: [M]; delta_b: [B] */
void orc_export_modes(const orc_model *m, double *gamma, double *c, double *lamnu, int *mode_state,
                      double *delta_b) {
  for (int l = 0; l < m->M; ++l) {
    gamma[l] = m->gamma[l];
    c[l] = m->c[l];
    lamnu[l] = m->lamnu[l];
    mode_state[l] = m->bath_state[l / (m->K + 1)];
  }
  for (int b = 0; b < m->B; ++b) delta_b[b] = m->delta_b[b];
}

void orc_export_hierarchy(const orc_model *m, uint8_t *tuples, int32_t *plus, int32_t *minus) {
  memcpy(tuples, m->h.tuples, (size_t)m->h.n * m->M);
  memcpy(plus, m->h.plus, (size_t)m->h.n * m->M * sizeof(int32_t));
  memcpy(minus, m->h.minus, (size_t)m->h.n * m->M * sizeof(int32_t));
}

/* ------------------------------------------------------------------------------------------ */
/* Superoperators, element-wise from their delta definitions.                                  */

/* For a diagonal V with diagonal v[]: (V^x A)_ij = (v_i - v_j) A_ij, (V^x V^x A)_ij = (v_i - v_j)^2 A_ij,
 * (V^o A)_ij = (v_i + v_j) A_ij.  For V = |s><s| these are (delta_is - delta_sj), (1 - delta_ij)
 * (delta_is + delta_sj) and (delta_is + delta_sj). */
static inline double vx(const double *v, int i, int j) { return v[i] - v[j]; }
static inline double vxvx(const double *v, int i, int j) { return (v[i] - v[j]) * (v[i] - v[j]); }
static inline double vo(const double *v, int i, int j) { return v[i] + v[j]; }

/* scale factors of the ADO rescaling */
static double up_factor(const orc_model *m, int l, int n_l) {
  double ac = fabs(m->c[l]);
  if (!m->rescale || ac < 1e-300) return 1.0;
  return sqrt((n_l + 1) * ac);
}
static double down_factor(const orc_model *m, int l, int n_l) {
  double ac = fabs(m->c[l]);
  if (!m->rescale || ac < 1e-300) return (double)n_l;
  return sqrt(n_l / ac);
}

/* d sigma_u / dt for one ADO u.  in/out: [n][N][N] complex in split re/im arrays. */
static void rhs_one(const orc_model *m, int64_t u, const double *in_re, const double *in_im,
                    cplx *out /* [N][N] */) {
  const int N = m->N, M = m->M, K1 = m->K + 1;
  const int64_t NN = (int64_t)N * N;
  const uint8_t *n = m->h.tuples + u * M;
#define SIG(v, i, j) (in_re[(v) * NN + (i) * N + (j)] + I * in_im[(v) * NN + (i) * N + (j)])
  /* -i [H, sigma_u] */
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      cplx acc = 0.0;
      for (int k = 0; k < N; ++k) acc += m->H[i * N + k] * SIG(u, k, j) - SIG(u, i, k) * m->H[k * N + j];
      out[i * N + j] = -I * acc;
    }
  /* - sigma_u sum_{b,k} n_{u,(b,k)} gamma(b,k) */
  double gsum = 0.0;
  for (int l = 0; l < M; ++l) gsum += n[l] * m->gamma[l];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) out[i * N + j] -= gsum * SIG(u, i, j);
  /* - sum_b [2 lambda/(beta nu) - sum_k c/gamma] V^x V^x sigma_u */
  if (m->terminator)
    for (int b = 0; b < m->B; ++b) {
      const double *v = m->vmask + (size_t)b * N;
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) out[i * N + j] -= m->delta_b[b] * vxvx(v, i, j) * SIG(u, i, j);
    }
  /* + sum i V^x sigma^+  and  + sum n theta sigma^-, with the rescaled factors */
  for (int l = 0; l < M; ++l) {
    int b = l / K1, k = l % K1;
    const double *v = m->vmask + (size_t)b * N;
    int32_t vp = m->h.plus[u * M + l], vm = m->h.minus[u * M + l];
    if (vp >= 0) {
      double f = up_factor(m, l, n[l]);
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) out[i * N + j] += I * f * vx(v, i, j) * SIG(vp, i, j);
    }
    if (vm >= 0) {
      double f = down_factor(m, l, n[l]);
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
          /* theta = i c V^x + delta_{k0} lambda nu V^o */
          cplx theta = I * m->c[l] * vx(v, i, j) + (k == 0 ? m->lamnu[l] : 0.0) * vo(v, i, j);
          out[i * N + j] += f * theta * SIG(vm, i, j);
        }
    }
  }
#undef SIG
}

/* Full RHS over every ADO.  Arrays [n][N][N]. */
void orc_rhs(const orc_model *m, const double *in_re, const double *in_im, double *out_re,
             double *out_im) {
  const int64_t NN = (int64_t)m->N * m->N;
  cplx *tmp = (cplx *)malloc(sizeof(cplx) * NN);
  for (int64_t u = 0; u < m->h.n; ++u) {
    rhs_one(m, u, in_re, in_im, tmp);
    for (int64_t e = 0; e < NN; ++e) {
      out_re[u * NN + e] = creal(tmp[e]);
      out_im[u * NN + e] = cimag(tmp[e]);
    }
  }
  free(tmp);
}

/* RHS of a list of ADOs (sampled checks on large hierarchies).  out: [count][N][N]. */
void orc_rhs_list(const orc_model *m, const int64_t *us, int64_t count, const double *in_re,
                  const double *in_im, double *out_re, double *out_im) {
  const int64_t NN = (int64_t)m->N * m->N;
  cplx *tmp = (cplx *)malloc(sizeof(cplx) * NN);
  for (int64_t t = 0; t < count; ++t) {
    rhs_one(m, us[t], in_re, in_im, tmp);
    for (int64_t e = 0; e < NN; ++e) {
      out_re[t * NN + e] = creal(tmp[e]);
      out_im[t * NN + e] = cimag(tmp[e]);
    }
  }
  free(tmp);
}

/* ------------------------------------------------------------------------------------------ */
/* Observables of rho = sigma_0.  One record: pop[N], tr_re, tr_im, corr_re, corr_im.          */

int orc_record_len(const orc_model *m) { return m->N + 4; }

static void record(const orc_model *m, const double *y_re, const double *y_im, const double *w,
                   double *rec) {
  const int N = m->N;
  double tr_re = 0, tr_im = 0, cr = 0, ci = 0;
  for (int a = 0; a < N; ++a) {
    rec[a] = y_re[a * N + a];
    tr_re += y_re[a * N + a];
    tr_im += y_im[a * N + a];
    if (w) {
      cr += w[a] * y_re[a * N + 0];
      ci += w[a] * y_im[a * N + 0];
    }
  }
  rec[N] = tr_re;
  rec[N + 1] = tr_im;
  rec[N + 2] = cr;
  rec[N + 3] = ci;
}

/* Classic RK4 with four ADO copies from time t0: k1 = f(t, y), k2 = f(t + h/2, y + h/2 k1),
 * k3 = f(t + h/2, y + h/2 k2), k4 = f(t + h, y + h k3), y <- y + h/6 (k1 + 2 k2 + 2 k3 + k4).
 * y: [n][N][N] split re/im, updated in place.  Records every obs_stride steps (after the step),
 * plus one record of the start state; obs must hold (n_steps/obs_stride + 1) records.
 * w: [N] weights of the dipole correlation (may be NULL).  Leaves H at t0 + n_steps h. */
int orc_rk4_t(orc_model *m, double *y_re, double *y_im, double t0_fs, double dt_fs, int64_t n_steps,
              int64_t obs_stride, const double *w, double *obs) {
  const int64_t tot = m->h.n * (int64_t)m->N * m->N;
  double *k_re = (double *)malloc(sizeof(double) * tot), *k_im = (double *)malloc(sizeof(double) * tot);
  double *x_re = (double *)malloc(sizeof(double) * tot), *x_im = (double *)malloc(sizeof(double) * tot);
  double *a_re = (double *)malloc(sizeof(double) * tot), *a_im = (double *)malloc(sizeof(double) * tot);
  if (!k_re || !k_im || !x_re || !x_im || !a_re || !a_im) {
    free(k_re); free(k_im); free(x_re); free(x_im); free(a_re); free(a_im);
    return -3;
  }
  const double h = dt_fs;
  const double wacc[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const double anext[3] = {0.5, 0.5, 1.0};
  const double cstage[4] = {0.0, 0.5, 0.5, 1.0};
  int64_t rec_i = 0;
  const int rl = orc_record_len(m);
  if (obs) record(m, y_re, y_im, w, obs + (rec_i++) * rl);
  for (int64_t step = 0; step < n_steps; ++step) {
    memcpy(a_re, y_re, sizeof(double) * tot);
    memcpy(a_im, y_im, sizeof(double) * tot);
    const double *xin_re = y_re, *xin_im = y_im;
    for (int s = 0; s < 4; ++s) {
      orc_set_time(m, t0_fs + ((double)step + cstage[s]) * h);
      orc_rhs(m, xin_re, xin_im, k_re, k_im);
      for (int64_t e = 0; e < tot; ++e) {
        a_re[e] += wacc[s] * h * k_re[e];
        a_im[e] += wacc[s] * h * k_im[e];
      }
      if (s < 3) {
        for (int64_t e = 0; e < tot; ++e) {
          x_re[e] = y_re[e] + anext[s] * h * k_re[e];
          x_im[e] = y_im[e] + anext[s] * h * k_im[e];
        }
        xin_re = x_re;
        xin_im = x_im;
      }
    }
    memcpy(y_re, a_re, sizeof(double) * tot);
    memcpy(y_im, a_im, sizeof(double) * tot);
    if (obs && obs_stride > 0 && (step + 1) % obs_stride == 0) record(m, y_re, y_im, w, obs + (rec_i++) * rl);
  }
  free(k_re); free(k_im); free(x_re); free(x_im); free(a_re); free(a_im);
  orc_set_time(m, t0_fs + (double)n_steps * h);
  return 0;
}

int orc_rk4(orc_model *m, double *y_re, double *y_im, double dt_fs, int64_t n_steps, int64_t obs_stride,
            const double *w, double *obs) {
  return orc_rk4_t(m, y_re, y_im, 0.0, dt_fs, n_steps, obs_stride, w, obs);
}
