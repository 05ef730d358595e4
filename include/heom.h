/*
 * heom.h -- C ABI of libheom, a single-GPU (GB300, sm_103a) propagator for the hierarchical
 * equations of motion (HEOM) of a Frenkel-exciton system coupled to Drude-Lorentz baths, after
 * arXiv 1803.03498 (DM-HEOM).
 *
 * Conventions for every call:
 *   - Returns an int status: HEOM_OK (0) or a negative HEOM_E_* code.  heom_last_error() returns
 *     a thread-local, human-readable message for the last failing call of the calling thread.
 *     No C++ exception crosses this boundary.
 *   - Energies in cm^-1, times in fs, temperatures in K.  Internally hbar = 1 with energies in
 *     rad/fs (E[rad/fs] = 2 pi c E[cm^-1], c = 2.99792458e-5 cm/fs).
 *   - Host matrices are row-major.  A hierarchy state on the host is ADO-major: [n_ado][N][N],
 *     real and imaginary parts in two separate double arrays.
 *   - The caller owns all device memory the run uses (one workspace block) and the CUDA stream;
 *     the library owns only the small opaque handles.  Calls that launch work enqueue it on the
 *     run's stream and return without waiting, except where stated ("synchronises").
 *   - Asynchronous CUDA errors surface as HEOM_E_CUDA at the next synchronising call.
 */
#ifndef HEOM_H
#define HEOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HEOM_OK 0
#define HEOM_E_ARG (-1)      /* bad shape or parameter, Matsubara resonance, unstable time step */
#define HEOM_E_OVERFLOW (-2) /* hierarchy size or an offset overflows int32 / int64 */
#define HEOM_E_NOMEM (-3)    /* workspace too small, record buffer full, host allocation failed */
#define HEOM_E_CUDA (-4)     /* a CUDA runtime call failed */
#define HEOM_E_TIMEOUT (-5)  /* a bounded device-side wait gave up */
#define HEOM_E_NUMERIC (-6)  /* NaN/Inf detected in the root ADO */
#define HEOM_E_STATE (-7)    /* call not valid for the handle's current state */
#define HEOM_E_BOUNDS (-8)   /* debug build only (compiled with -DHEOM_DEBUG): a stage kernel found a link
                                record naming an ADO, a state or a record range outside the run */

/* Arithmetic of a run. */
#define HEOM_FP64 0       /* every ADO stored and computed in FP64 */
#define HEOM_FP32_MIXED 1 /* levels >= 2 stored and computed in FP32; levels 0 and 1 (the root ADO
                             sigma_0 and its direct neighbours), the RK4 combination of sigma_0 and
                             every observable reduction in FP64 */
#define HEOM_SPLIT_TF32 2 /* storage and arithmetic as HEOM_FP32_MIXED, except that for Hermitian runs
                             with real H and n_states <= 16 the commutator of levels >= 2 runs on the
                             tensor cores: sigma and H are split into TF32 high and low parts and
                             sigma H = hi*hi + lo*hi + hi*lo is accumulated in FP32 (about 21 bits).
                             Other runs at this precision compute exactly as HEOM_FP32_MIXED.  Not in
                             the paper (which computes in FP64). */

typedef struct heom_hier heom_hier;
typedef struct heom_run heom_run;

/*
 * The physical model: H (n_states x n_states, Hermitian, cm^-1) and n_baths Drude-Lorentz baths
 * (Omega = 0), bath b coupled to state bath_state[b] through V_b = |s><s| (Eq. HEOM, with S(b) = 1;
 * several baths may couple to the same state, states without a bath get no bath terms).  Each
 * bath contributes n_matsubara + 1 modes (the Drude term k = 0 and Matsubara terms k = 1..K), so
 * the hierarchy has n_modes = n_baths * (n_matsubara + 1); mode l = b * (n_matsubara + 1) + k
 * (the 0-based form of the paper's l = (b-1)K + k + 1).
 * terminator: 1 adds the Matsubara terminator term of Eq. HEOM, 0 drops it.
 * rescale: 1 applies the ADO rescaling (sqrt((n+1)|c|) up, sqrt(n/|c|) down), 0 uses 1 and n.
 * bath_mask (may be NULL): [n_baths][n_states] of 0/1; bath b then couples through the diagonal
 *   V_b with 1 at every state whose entry is 1 -- in the two-exciton space (section "Dipole
 *   operators and rotational averaging") the number operator of site b: its single-exciton state and
 *   every pair that contains it.  V^x, V^x V^x and V^o keep their element-wise definitions; the
 *   terminator then has the element rate T_ij = sum_b Delta_b (V_b,ii - V_b,jj)^2.  bath_state[b]
 *   must still name a state of the bath (it labels the bath's modes in heom_bath_modes).
 * time_dependent: 1 reserves a fourth state copy so that the run can take a laser field
 *   (heom_run_set_field) and be propagated by classic four-copy RK4 with H(t) at each stage time.
 * Runs with a bath_mask, with time_dependent = 1 or with more than 24 states (up to 32, e.g. the
 * 29 states of a 7-site two-exciton space) use the general stage kernel; all others use the
 * specialised ones.
 * All pointers are read during the call only (copied).
 */
typedef struct {
  int n_states;
  const double *H_re;      /* [n_states * n_states] */
  const double *H_im;      /* [n_states * n_states] or NULL for a real H */
  int n_baths;
  const int *bath_state;   /* [n_baths], each in [0, n_states) */
  const double *lambda_cm; /* [n_baths] reorganisation energy */
  const double *tau_fs;    /* [n_baths] correlation time 1/nu */
  const double *T_K;       /* [n_baths] temperature */
  int n_matsubara;         /* K >= 0: modes per bath beyond the Drude mode (Matsubara terms or Pade poles) */
  int terminator;
  int rescale;
  int decomposition;       /* HEOM_MATSUBARA or HEOM_PADE */
  const unsigned char *bath_mask; /* [n_baths * n_states] 0/1 diagonal of each V_b, or NULL */
  int time_dependent;      /* 1: the run keeps a fourth state copy for a laser field */
} heom_system;

/* Expansion of the Bose function behind the bath modes (section "HEOM formalism"):
 *   HEOM_MATSUBARA  gamma(b,k) = 2 pi k / beta, c(b,0) = lambda nu cot(beta nu / 2);
 *   HEOM_PADE       the [K-1/K] Pade spectrum decomposition the paper uses (the method of its
 *                   reference Hu, Xu, Yan 2010): xi_i = 2 / (i-th largest eigenvalue of the 2K x 2K
 *                   tridiagonal Lambda, entries 1/sqrt((2m+1)(2m+3))), zeta_i likewise from the
 *                   (2K-1) x (2K-1) Lambda' (entries 1/sqrt((2m+3)(2m+5))),
 *                   eta_i = K (2K+3)/2 prod_j (zeta_j^2 - xi_i^2) / prod_{j != i} (xi_j^2 - xi_i^2),
 *                   gamma(b,k) = xi_k / beta, c(b,k) = 4 lambda nu eta_k gamma_k / (beta (gamma_k^2 - nu^2)),
 *                   c(b,0) = (2 lambda / beta) (1 - sum_j 2 eta_j nu^2 / (gamma_j^2 - nu^2)).
 *                   The paper's printed c(b,0) sums over j but indexes eta_k, xi_k, and its eta
 *                   numerator pairs zeta_j with xi_j; both are read as above (the form for which
 *                   the approximant reproduces the Bose function). */
#define HEOM_MATSUBARA 0
#define HEOM_PADE 1

/* Message of the calling thread's last failing call ("" if none).  Valid until that thread's next
 * call into the library. */
const char *heom_last_error(void);

/*
 * heom_build_hierarchy -- enumerate every multi-index n in N^n_modes with |n| <= depth (Eq.
 * Nmatrices: C(n_modes + depth, depth) ADOs) and build the "+"/"-" link tables (u -> n +- e_l,
 * section "HEOM formalism").  Numbering u: by level |n|, then by the colexicographic rank of the
 * stars-and-bars positions b_j = (j - 1) + n_1 + ... + n_j (j = 1..n_modes-1):
 *     u = C(n_modes + L - 1, n_modes) [L > 0] + sum_j C(b_j, j).
 * The root (all zeros) is u = 0.  Host-only; the tables are uploaded into a run's workspace at
 * heom_run_create.  Errors: HEOM_E_ARG (n_modes < 1, n_modes > 255, depth < 0, depth > 255),
 * HEOM_E_OVERFLOW (more than 2^31 - 1 ADOs), HEOM_E_NOMEM.  *out is owned by the caller and
 * freed with heom_hier_destroy.
 */
int heom_build_hierarchy(int n_modes, int depth, heom_hier **out);
int heom_hier_destroy(heom_hier *h);

/* n_ado and, if level_offsets is not NULL, the first u of every level L = 0..depth plus n_ado
 * (depth + 2 entries). */
int heom_hier_info(const heom_hier *h, int64_t *n_ado, int64_t *level_offsets);

/* Copy the tables into caller-owned host arrays of n_ado * n_modes entries, row u = ADO:
 * tuples[u][l] = n_l, plus[u][l] = index of n + e_l or -1 (|n| = depth),
 * minus[u][l] = index of n - e_l or -1 (n_l = 0).  Any pointer may be NULL. */
int heom_hier_export(const heom_hier *h, uint8_t *tuples, int32_t *plus, int32_t *minus);

/*
 * heom_bath_modes -- the bath modes a run of this system uses (host only; no GPU needed).
 *   Section "HEOM formalism": per bath b and k = 0..K, mode l = b (K+1) + k with rate gamma_l
 *   (rad/fs), real coefficient c_l ((rad/fs)^2), lamnu_l = lambda_b nu_b for k = 0 else 0, and
 *   the state s_b it couples to; term[s] = sum over the baths of state s of the terminator
 *   2 lambda / (beta nu) - sum_k c(b,k) / gamma(b,k) (0 for every state when sys->terminator is 0).
 *   Outputs (caller-owned host arrays): gamma, c, lamnu, mode_state [n_baths (K+1)], term [n_states].
 *   Errors: HEOM_E_ARG for an invalid system or a rate gamma_k equal to nu (c_k diverges).
 */
int heom_bath_modes(const heom_system *sys, double *gamma, double *c, double *lamnu, int *mode_state,
                    double *term);

/*
 * heom_run_bytes -- device workspace bytes a run of this system, hierarchy and precision needs,
 * including room for max_records observable records.  The hierarchy's n_modes must equal
 * n_baths * (n_matsubara + 1).  Supported: 1 <= n_states <= 32 (above 24 on the general stage kernel).
 */
int heom_run_bytes(const heom_system *sys, const heom_hier *h, int precision, int64_t max_records,
                   size_t *bytes);

/*
 * heom_run_create -- set up a propagation on the caller's device workspace (at least
 * heom_run_bytes bytes, 256-byte aligned, on the current CUDA device) and stream (a
 * cudaStream_t; NULL = the legacy default stream).  Computes the bath coefficients of Eq. HEOM
 * (Matsubara gamma(b,k), c(b,k), the terminator and the rescaling factors) on the host in FP64,
 * uploads the link tables, zeroes every ADO and writes sigma_0 = rho(0) (n_states x n_states,
 * sigma0_im may be NULL).  dip_w (n_states weights w_a, or NULL) selects the dipole correlation
 * sum_a w_a sigma_0[a][0] recorded with every observable record (Eq. lin_abs_mukamel with
 * sigma_0(0) = mu^+|0><0|, state 0 the ground state).  Errors: HEOM_E_ARG, HEOM_E_NOMEM
 * (workspace too small), HEOM_E_CUDA.  The workspace must stay allocated until
 * heom_run_destroy.  Mixed-precision runs also own one library stream and two events: each stage's
 * small FP64 head launch runs there, forked from and joined back into the caller's stream, so that
 * it overlaps the body launch (work enqueued on the caller's stream stays ordered).  The bath
 * coefficients follow sys->decomposition (Matsubara or Pade).  Runs on the general stage kernel
 * (bath_mask, time_dependent or more than 24 states) always use the matrix layout.
 */
int heom_run_create(const heom_system *sys, const heom_hier *h, int precision, int64_t max_records,
                    const double *sigma0_re, const double *sigma0_im, const double *dip_w,
                    void *device_workspace, size_t workspace_bytes, void *cuda_stream, heom_run **out);
int heom_run_destroy(heom_run *r);

/*
 * heom_propagate -- advance the whole hierarchy by n_steps steps of classic RK4 with step dt_fs
 * (four evaluations of the right-hand side of Eq. HEOM per step).  Every obs_stride steps (0 =
 * never) one observable record of sigma_0 is appended after the step.  Enqueued on the run's
 * stream; does not block.  Errors: HEOM_E_ARG (dt_fs <= 0, n_steps < 0, dt_fs times the fastest
 * decay rate D * max gamma above 2.5, where RK4 is no longer stable), HEOM_E_NOMEM (the records
 * would overflow max_records), HEOM_E_CUDA.
 */
int heom_propagate(heom_run *r, double dt_fs, int64_t n_steps, int64_t obs_stride);

/*
 * heom_run_set_field -- a laser field in the rotating-wave approximation (Eq. h-field-rwa with the
 *   pulse of Eq. probe_pulse), seen from the frame that rotates at the reference frequency already
 *   subtracted from each excitation in H:
 *     H(t) = H - g(t) M+ - conj(g(t)) (M+)^T,
 *     g(t) = amp_cm exp(-(t - t_center_fs)^2 / (2 sigma_fs^2)) exp(-i (detuning t + phase)),
 *   with M+ the real polarisation-weighted dipole raising operator e . mu^+ (for example |a><0| and
 *   |ab><b| with weights e . d_a in the two-exciton space), amp_cm the peak of dipole times field and
 *   detuning_cm the carrier minus the reference frequency, both in cm^-1.  The run must have been
 *   created with time_dependent = 1 (else HEOM_E_STATE).  From then on heom_propagate uses classic
 *   four-copy RK4 with H at each stage time t, t + h/2, t + h/2, t + h (t counted from creation, the
 *   time heom_run_info reports) and heom_rhs_eval uses H at the current time.  f == NULL removes
 *   the field (Horner RK4 again).  A run with a field cannot join a batch (its graph would replay
 *   fixed times).  Errors: HEOM_E_ARG (sigma_fs <= 0, NULL mu_plus), HEOM_E_STATE.
 */
typedef struct {
  const double *mu_plus;   /* [n_states * n_states] M+, row-major, real */
  double amp_cm;           /* peak coupling (dipole times field), cm^-1 */
  double t_center_fs;      /* centre of the Gaussian envelope */
  double sigma_fs;         /* its width: exp(-(t - t_c)^2 / (2 sigma^2)) */
  double phase;            /* pulse phase, rad */
  double detuning_cm;      /* carrier minus reference frequency, cm^-1 */
} heom_field;
int heom_run_set_field(heom_run *r, const heom_field *f);

/* Length in doubles of one observable record of the reduced density matrix rho = sigma_0 (the root
 * ADO, section "HEOM formalism"): n_states populations Re sigma_0[a][a], then Re Tr sigma_0,
 * Im Tr sigma_0, Re C, Im C (C = sum_a w_a sigma_0[a][0], the dipole correlation of Eq.
 * lin_abs_mukamel; 0 without dip_w), then max_ij |sigma_0[i][j] - conj(sigma_0[j][i])|.  That is
 * n_states + 5; 0 for a NULL run. */
int heom_record_len(const heom_run *r);

/*
 * heom_observables -- synchronises the run's stream and copies up to cap_records records (the
 * first record is the state at creation, then one per obs_stride steps) into out
 * ([cap_records][heom_record_len]); *written = records copied.  HEOM_E_NUMERIC if a record
 * holds NaN/Inf; HEOM_E_TIMEOUT if a bounded device-side wait gave up; HEOM_E_BOUNDS if a bounds
 * check of a debug build failed.  The record's content is fixed (see heom_record_len): the dipole
 * weights of the correlation are set once at heom_run_create.
 */
int heom_observables(heom_run *r, double *out, int64_t cap_records, int64_t *written);

/* Synchronises; copies the reduced density matrix rho = sigma_0 (the root ADO, section "HEOM
 * formalism"; FP64 in every precision) into caller host arrays of n_states^2 doubles, row-major. */
int heom_get_sigma0(heom_run *r, double *re, double *im);

/* Synchronises; copies ADOs [u0, u0 + count) of the current state into / out of caller host
 * arrays [count][N][N] (FP32-stored ADOs are rounded on the way in).  HEOM_E_ARG if the range is
 * outside [0, n_ado). */
int heom_get_ados(heom_run *r, int64_t u0, int64_t count, double *re, double *im);
int heom_set_ados(heom_run *r, int64_t u0, int64_t count, const double *re, const double *im);

/*
 * heom_rhs_eval -- evaluate the right-hand side of Eq. HEOM once on the current state with the
 * same kernels heom_propagate uses, and copy ADOs [u0, u0 + count) of d sigma / dt into caller
 * host arrays [count][N][N].  The state is not changed (the result goes through a scratch copy of
 * the workspace).  Synchronises.
 */
int heom_rhs_eval(heom_run *r, int64_t u0, int64_t count, double *re, double *im);

/* Number of ADOs, states and modes of a run; the step count and simulated time so far. */
int heom_run_info(const heom_run *r, int64_t *n_ado, int *n_states, int *n_modes, int64_t *steps_done,
                  double *t_fs);

/*
 * heom_run_layout -- how the run stores its ADOs: 0 = N x N matrices; 1 = the excited-ground
 *   coherence block, each ADO stored as its column 0 (chosen at creation when state 0 has no bath,
 *   H has no element between state 0 and the others, and rho(0) lives on column 0 below the
 *   diagonal: a linear-absorption run; every term of Eq. HEOM keeps every ADO in that block, so the
 *   right-hand side acts on columns, with the same results).  heom_set_ados with data outside the
 *   block moves the run to layout 0 for good.  -1 for a NULL run.
 */
int heom_run_layout(const heom_run *r);

/* Kernel launches the library enqueued for this run since creation (all kinds). */
int64_t heom_run_launches(const heom_run *r);

/*
 * Kernel timing of the dominant kernel (the stage kernel over the bulk of the hierarchy: every
 * ADO for HEOM_FP64, levels >= 2 for HEOM_FP32_MIXED).  heom_run_set_timing(r, 1) starts recording
 * a CUDA event pair around each such launch on the run's stream (and clears earlier records);
 * 0 stops.  heom_run_kernel_time synchronises and returns the summed device time in ms, the number
 * of timed launches, and the algorithmic bytes and flops of those launches:
 *   bytes per ADO and launch = (tile reads + tile writes) * N^2 * complex size + M * 9 + 8
 *     (a stage reads its input tile, reads y unless y is the input, writes one tile; the link
 *      tables are 4 + 4 + 1 bytes per mode, the decay sum 8 bytes)
 *   flops per ADO and launch = 8 N^3 (commutator with real H; 16 N^3 with complex H) + 8 N^2
 *     (decay, terminator, RK4 combination) + 8 (N - 1) per valid up link + 8 (2N - 1) per valid
 *     down link.
 * Neighbour gathers count as algorithmically free.  At most 65536 launches are recorded.
 */
int heom_run_set_timing(heom_run *r, int enable);
int heom_run_kernel_time(heom_run *r, double *ms, int64_t *launches, double *alg_bytes, double *alg_flops);

/*
 * Ragged batches (many independent propagations of different sizes advanced together).
 * heom_batch_create captures steps_per_launch RK4 steps of every run into one CUDA graph (one
 * observable record every obs_stride steps, obs_stride dividing steps_per_launch, 0 = none).  Small
 * runs (up to 50,000 ADOs) in the column-0 layout (heom_run_layout 1) of equal n_states and precision
 * class advance together:
 * one launch per stage and part (FP64 head, body) covers all of them, with each run's stage
 * arguments written into its own workspace; such a run's arguments belong to the last batch created
 * over it, and heom_batch_launch answers HEOM_E_STATE if a run left that layout or joined a later
 * batch.  Other runs launch per run, on one of up to 32 library-created streams, so small runs
 * execute concurrently.  The
 * runs must be on the current device, with timing off; the call synchronises their streams first.
 * heom_batch_launch replays the graph n_launches times on a stream of the batch's own (ordered after
 * work already enqueued on every run's stream; later work on a run's stream is ordered after it) and
 * advances each run's step and record counters; HEOM_E_NOMEM if a run's records would overflow
 * max_records.  Results are those of heom_propagate with the same steps (same arithmetic, same order
 * per run).  heom_batch_destroy synchronises the batch's stream and frees the graph (the runs stay).
 * The paper runs independent propagations (rotational averages, polarisation sequences) side by
 * side (section "Distributed memory HEOM implementation"); this is that, on one GPU.
 */
typedef struct heom_batch heom_batch;
int heom_batch_create(heom_run *const *runs, int n_runs, double dt_fs, int64_t steps_per_launch, int64_t obs_stride,
                      heom_batch **out);
int heom_batch_launch(heom_batch *b, int64_t n_launches);
int heom_batch_destroy(heom_batch *b);

/*
 * heom_group_propagate -- advance several runs together: run i by n_steps[i] RK4 steps of dt_fs (as
 * heom_propagate, one observable record every obs_stride steps of each run's own step count, 0 =
 * none), sharing kernel launches.  Small mixed-precision runs (HEOM_FP32_MIXED, the matrix layout,
 * a real H, no laser field, at most 200,000 ADOs) of equal n_states advance in work-list launches:
 * one launch per RK4 stage and part (FP64 head, FP32 body) covers every such run of that size, each
 * run's stage arguments staged from its own workspace, so many small requests cost a few launches
 * per step instead of eight each.  Other runs launch on their own, on the same stream.  Everything is
 * enqueued on cuda_stream (the launches of different sizes on library-created streams forked from and
 * joined back into it, with its priority), ordered after work already enqueued on each run's stream, and later work
 * on each run's stream is ordered after it; the call does not block, except that writing a run's
 * work-list stage arguments (its first grouped call, or a new dt_fs) waits for cuda_stream.
 * Results equal heom_propagate's bit for bit: every ADO gets the same arithmetic in the same order.
 * A work-list launch counts in heom_run_launches of each run it covers.  The paper runs independent
 * propagations side by side (section "Distributed memory HEOM implementation"); this shares their
 * launches on one GPU.  Errors: HEOM_E_ARG (NULL run, a run listed twice, negative steps, dt_fs
 * beyond a run's stability bound as in heom_propagate), HEOM_E_STATE (a run with a laser field or
 * with kernel timing on), HEOM_E_NOMEM (records would exceed a run's max_records), HEOM_E_CUDA.
 */
int heom_group_propagate(heom_run *const *runs, int n_runs, double dt_fs, const int64_t *n_steps, int64_t obs_stride,
                         void *cuda_stream);

/*
 * Launch schedules and the autotuner (not in the paper, whose kernels are fixed; the choices below
 * map the same arithmetic onto the GPU differently).  A stage launch covers its ADOs in chunks of
 * floor(32 / n_states) consecutive ADOs over a persistent grid of CTAs.  A schedule fixes what the
 * arithmetic leaves open:
 *   occupancy_pct     1..1600: the grid is sized for this percentage of the kernel's CTAs that fit
 *                     on one SM (rounded down, at least 1) times the SM count.  Above 100 the grid
 *                     is several waves of CTAs that retire while the launch runs, so that launches
 *                     on other (higher-priority) streams get SM slots before it ends, at the cost
 *                     of more CTA starts;
 *   chunks_per_warp   1, 2 or 4: column-0 kernels (heom_run_layout 1) let each warp hold this many
 *                     consecutive chunks at once (capped at 32 ADOs per warp: 2 for n_states 2, 3
 *                     for 3), one element of each per lane, and load the link records and
 *                     neighbour elements of all of them together, so that their memory round trips
 *                     overlap (more registers per thread).  Matrix-layout kernels ignore it.
 * Every schedule gives bit-identical results: each output element sums the same terms in the same
 * order.  Only the time differs.  The default is {100, 1}.
 *
 * heom_schedule_candidates -- host only: the candidates the tuner times for a layout (0 matrix,
 *   1 column-0 run, 2 column-0 batch group) into out[cap]; returns their number (or a negative
 *   status).
 * heom_tune -- times every candidate of one part of a run (part 0: the body, the stage kernel over
 *   the bulk of the hierarchy; part 1: the FP64 head launch of a mixed-precision run) on the run's
 *   own stage-1 launch (reads the state, writes an intermediate copy: the state is unchanged),
 *   one warm-up and reps timed launches each, on the run's stream, and keeps the fastest for the
 *   run and in a process-wide cache keyed by (layout, precision, part, n_states, Hermitian,
 *   complex H, floor(log2 of the part's ADO count)).  Outputs (caller-owned, may be NULL):
 *   tried[cap] and ms[cap] (mean ms per launch, in candidate order), *n_tried, *chosen.
 *   Synchronises the stream.  HEOM_E_ARG: reps < 1, part not 0/1, part 1 of a run without a head;
 *   HEOM_E_STATE: the run's stream is being captured.
 * heom_set_autotune -- process-wide.  reps > 0: heom_run_create and heom_batch_create tune every
 *   part whose cache key has no entry yet (reps timed launches per candidate), and take cached
 *   entries otherwise; 0: no tuning at creation (cached entries still apply; other parts take the
 *   layout's default schedule, below).  Returns the previous value; a negative argument only queries.  Default 3.
 *   heom_propagate_static never tunes.
 * heom_get_schedule / heom_set_schedule -- the schedule a part of a run launches with; set checks
 *   the ranges above (HEOM_E_ARG) and does not touch the cache.
 * heom_set_default_schedule -- the schedule that parts of a layout (0, 1, 2 as above) take when the
 *   cache has no entry and no tuning runs; NULL restores {100, 1}.  Applies to later creations.
 * heom_tune_cache_clear -- empties the cache.
 * heom_batch_schedule -- the schedule of part (0 body, 1 FP64 head) of group g of a batch's
 *   grouped column-0 launches (tuned at heom_batch_create under autotuning, layout 2 in the cache
 *   key, with the group's total ADO count); *n_groups gets the number of groups (g may then be
 *   -1 to query only that).
 */
typedef struct {
  int occupancy_pct;
  int chunks_per_warp;
} heom_schedule;
int heom_schedule_candidates(int layout, heom_schedule *out, int cap);
int heom_tune(heom_run *r, int part, int reps, heom_schedule *tried, double *ms, int cap, int *n_tried,
              heom_schedule *chosen);
int heom_set_autotune(int reps);
int heom_get_schedule(const heom_run *r, int part, heom_schedule *out);
int heom_set_schedule(heom_run *r, int part, const heom_schedule *s);
int heom_set_default_schedule(int layout, const heom_schedule *s);
int heom_tune_cache_clear(void);
int heom_batch_schedule(const heom_batch *b, int g, int part, heom_schedule *out, int *n_groups);

/*
 * heom_propagate_static -- one complete propagation that allocates no device memory, for callers
 * that cannot call cudaMalloc (plug-ins whose host application owns every device allocation and
 * hands the library no buffer, latency-critical paths that cannot afford the implicit
 * synchronisation of cudaMalloc/cudaFree).  The paper has no counterpart; it is a deployment
 * convenience around the same kernels as heom_run_create + heom_propagate + heom_observables.
 *   Inputs (host, read during the call): sys, h, precision, sigma0_re/sigma0_im (n_states^2,
 *   sigma0_im may be NULL), dip_w (n_states or NULL), dt_fs, n_steps, obs_stride, as for
 *   heom_run_create and heom_propagate; cuda_stream as there.
 *   Outputs (caller-owned host buffers): records_out [cap_records][n_states + 5] (the state at
 *   the start, then one record every obs_stride steps; cap_records >= 1 + n_steps / obs_stride),
 *   *written; sigma0_out_re/sigma0_out_im (n_states^2, both may be NULL) get the final sigma_0.
 * The device workspace of the run (tables, state, the two intermediate RK4 copies and the records)
 * lives in one library-owned static device array of 32 MiB (33554432 bytes) per GPU, which every GPU
 * that loads the library holds until the process exits.  A run whose heom_run_bytes exceeds it is
 * rejected with HEOM_E_NOMEM before any work.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current.  Every call reuses the same array
 * and zeroes what must start at zero; calls serialise on a lock within one process, and calls whose
 * GPU work overlaps (for example from two processes sharing a context, or work still in flight on
 * another stream) would race on it.  On every return path, errors included, the call has waited
 * for the work it queued (on the stream and on the run's side stream) before it returns.  Errors:
 * those of heom_run_bytes, heom_run_create, heom_propagate and heom_observables, and HEOM_E_NOMEM
 * as above.
 */
int heom_propagate_static(const heom_system *sys, const heom_hier *h, int precision, const double *sigma0_re,
                          const double *sigma0_im, const double *dip_w, double dt_fs, int64_t n_steps,
                          int64_t obs_stride, void *cuda_stream, double *records_out, int64_t cap_records,
                          int64_t *written, double *sigma0_out_re, double *sigma0_out_im);

#ifdef __cplusplus
}
#endif
#endif /* HEOM_H */
