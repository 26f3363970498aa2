/*
 * letkf.h -- C ABI of the single-GPU LBM-LETKF hot path (sm_103a).
 *
 * One handle holds one data-assimilation experiment of the paper's OSSE
 * (Sec. V): an ensemble of k D2Q9 lattice-Boltzmann members on a periodic
 * nx x ny grid (Sec. II-A), a static observation network with diagonal
 * observation-error covariance R, and an R-localized LETKF analysis solved
 * independently at every grid point (Sec. II-B, Algorithm 1).
 *
 * Conventions shared by every entry point
 *   - Return value: LETKF_OK (0) or a negative LETKF_E* code.  No entry
 *     point aborts, throws or exits; letkf_strerror() names a code.
 *   - Kernels run asynchronously on the handle's stream.  Errors found on
 *     the device (non-convergence, non-finite output) are latched in a
 *     status word and returned by the next letkf_sync().
 *   - Host pointers passed in are only read/written during the call;
 *     device pointers must stay valid until the stream passes that point.
 *   - Populations are indexed q = 3 (j + 1) + (i + 1) for the lattice
 *     velocity c_q = (i, j), (i, j) in {-1, 0, 1}^2 (Eq. 1).
 *   - Ensemble states cross the ABI in the paper's LBM layout: FP32,
 *     member-major structure of arrays f[m][q][y][x] (Sec. IV-A, X[m,N_v,N_x]).
 *   - A handle is not thread safe; distinct handles are independent.
 */
#ifndef LETKF_H
#define LETKF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LETKF_OK          0
#define LETKF_EINVAL     (-1)  /* an argument is out of range or NULL          */
#define LETKF_ENOMEM     (-2)  /* workspace too small or device allocation failed */
#define LETKF_ENOTCONV   (-3)  /* the eigensolver hit its iteration cap somewhere */
#define LETKF_ENONFINITE (-4)  /* a non-finite value appeared in the analysis  */
#define LETKF_ETIMEOUT   (-5)  /* a bounded device wait expired                */
#define LETKF_ECUDA      (-6)  /* a CUDA runtime call failed                   */
#define LETKF_ESTATE     (-7)  /* call not valid in the handle's current state */

/* ---- enumerations ------------------------------------------------------- */
#define LETKF_HOST    0        /* pointer argument is host memory             */
#define LETKF_DEVICE  1        /* pointer argument is device memory           */

#define LETKF_OBS_RHO 1        /* observed variable bits, output order rho,u,v */
#define LETKF_OBS_U   2
#define LETKF_OBS_V   4

#define LETKF_LOC_NONE  0      /* G = 1 for every observation ("infinite")    */
#define LETKF_LOC_GAUSS 1      /* G = exp(-d^2/(2 r^2)) for d^2 < cutoff^2    */
#define LETKF_LOC_GC    2      /* G = GC(d / c), Gaspari & Cohn (1999) Eq. 4.10, the paper's
                                  localization (Sec. II-B): the fifth-order piecewise rational
                                  function, half-width c = sqrt(10/3) r, zero from d = 2c on
                                  (the default cutoff of LETKF_LOC_GAUSS); the cutoff is
                                  capped at 2c, so every local observation has G > 0   */

#define LETKF_FP32  0          /* plain FP32 CUDA-core analysis                                */
#define LETKF_MIXED 1          /* split-precision: for 17 <= k <= 128 the localized Gram runs on
                                  the tensor cores (tcgen05, FP16 hi+lo operands, FP32
                                  accumulation; for k <= 32 two grid points share one
                                  operand tile); for k <= 16 it stays on CUDA cores        */

/* Eigensolve schedules (same results up to rounding; see letkf_config.eig_schedule). */
#define LETKF_EIG_AUTO        0  /* the handle picks one: at its first analysis the schedules
                                    (FUSED, SPLIT and, for k <= 64, CHEBYSHEV, which passes its
                                    ill-conditioned points to RATIONAL) are timed on
                                    that analysis' first chunk of Gram matrices
                                    (applied to a scratch copy of the forecast, so the analysis
                                    itself is unaffected; one host synchronisation), and the
                                    faster is kept.  The pick is cached per (device, k, chunk
                                    size) for the process: later handles of that shape take it
                                    at letkf_init.  A letkf_cycle that must still pick runs
                                    without graph capture; the next one captures.          */
#define LETKF_EIG_FUSED       1  /* one warp per grid point runs every phase in one launch    */
#define LETKF_EIG_SPLIT       2  /* tridiagonalization (warp per point), QL (thread per point,
                                    rotations recorded), replay + update (warp per point)    */
#define LETKF_EIG_SPLIT_CHECK 3  /* SPLIT with a record of one sweep per point, so that nearly
                                    every point is handed back to the fused kernel: exercises
                                    the hand-off; for tests and diagnosis, not for speed      */
#define LETKF_EIG_RATIONAL    4  /* EVD-free transform, k <= 64 (the paper's future work,
                                    Sec. III): the same Householder tridiagonalization
                                    Q = H T H^T, then Q^-1 c by one tridiagonal solve and
                                    Q^-1/2 applied to the perturbations through Zolotarev's
                                    best rational approximation of t^-1/2 (shifted L D L^T
                                    solves of T, relative error ~1e-8); no eigenvalues or
                                    eigenvectors are formed.  A point whose condition bound
                                    exceeds 1e6 is solved by the fused schedule instead.  A
                                    probe's eigenvalues come from an extra eigenvalue-only QL. */
#define LETKF_EIG_CHEBYSHEV   5  /* EVD-free transform by polynomials in Q, k <= 64: with
                                    S = Q (rho / (k-1)), whose spectrum lies in [1, kappa],
                                    kappa from the least of the Gershgorin, Frobenius and trace
                                    bounds of A, t^-1/2 and t^-1 are replaced by their Chebyshev
                                    interpolants on [1, kappa_max] (relative error < 2e-8,
                                    degree 4 at kappa_max = 1.1 up to 36 at 16) and applied to
                                    [dX; c^T] by Clenshaw's recurrence, one product with A per
                                    degree.  No factorization or tridiagonalization.  Degrees
                                    up to 9k/16 are used (kappa_max 16 at k = 64, 4 at k = 32),
                                    about where a product costs as much as the RATIONAL
                                    schedule; a point beyond is passed to RATIONAL.
                                    Pays where Q is well conditioned (ensemble spread small
                                    against the observation error).  A probe's eigenvalues come
                                    from a tridiagonalization and an eigenvalue-only QL.      */

/* FP32 Gram tile schedules for k >= 17 (letkf_config.gram_tile; k <= 16 has one schedule and
 * LETKF_MIXED uses the tensor cores for k >= 17, so the choice applies to LETKF_FP32 only). */
#define LETKF_GRAM_AUTO   0  /* the handle times both on its first analysis' first chunk and
                                keeps the faster; cached per problem shape for the process,
                                so handles of the same shape run the same arithmetic        */
#define LETKF_GRAM_PIPE   1  /* one CTA per SM over 7 x 2 points (k <= 64; 8 x 6 for k <= 32,
                                3 x 1 for k <= 128), per-point compacted entries, operands
                                double-buffered by cp.async                                */
#define LETKF_GRAM_TEAM   2  /* two CTAs per SM over 4 x 2 points (k <= 64; 8 x 4, 2 x 1), the
                                weights of a chunk in shared memory, a weight test per
                                candidate in the multiply-add loop                         */
#define LETKF_GRAM_TENSOR 3  /* (reported only) the tensor-core Gram of LETKF_MIXED          */

/* ---- problem statement --------------------------------------------------
 * Follows the paper's statement of the problem (Sec. II-B): the grid, the
 * ensemble size M (= k), the observation operator H (observation points and
 * observed variables), R (diagonal) and the localization (Sec. II-B,
 * R-localization paragraph).  Host arrays are copied during letkf_init.
 */
typedef struct letkf_config {
    int32_t nx, ny;            /* periodic grid, N_x = nx * ny points (>= 1 each)      */
    int32_t k;                 /* ensemble size M, 2 <= k <= 128                        */
    int32_t n_aux;             /* extra members advanced by lbm_forecast but never
                                  analysed (e.g. the nature run), 0 <= n_aux <= 4      */
    float   tau;               /* BGK relaxation time, > 0.5                            */
    const float *force;        /* host [2][ny][nx]: F_x then F_y; NULL = no body force  */
    int32_t n_obs;             /* L observation points, >= 0                            */
    const int32_t *obs_xy;     /* host [L][2] grid coordinates (x, y), 0 <= x < nx      */
    int32_t obs_vars;          /* LETKF_OBS_* bit mask, V = number of bits set (>= 1)   */
    const float *obs_err_var;  /* host [L*V] diagonal of R, index l*V + v, > 0          */
    int32_t loc_kind;          /* LETKF_LOC_*                                           */
    float   loc_radius;        /* radius r in cells (> 0 for LOC_GAUSS and LOC_GC)      */
    float   loc_cutoff2;       /* squared cutoff distance; <= 0 selects (40/3) r^2,
                                  i.e. cutoff 2 sqrt(10/3) r                            */
    float   infl;              /* multiplicative inflation rho: Q = (k-1)/rho I + ...;
                                  1 = none (the paper's Eq. letkf_q)                    */
    int32_t precision;         /* LETKF_FP32 or LETKF_MIXED                             */
    int32_t eig_schedule;      /* LETKF_EIG_*; 0 (AUTO) lets the handle choose          */
    int32_t gram_tile;         /* LETKF_GRAM_*; 0 (AUTO) lets the handle choose         */
    int64_t chunk_bytes;       /* device bytes for the per-point k x k Gram buffer;
                                  0 = default (1 GiB; larger chunks give the
                                  thread-per-matrix QL kernel more matrices per launch) */
    void   *stream;            /* cudaStream_t to run on; NULL = a stream the handle
                                  creates and owns                                       */
} letkf_config;

typedef struct letkf_stats {
    int32_t status;            /* last latched LETKF_* code (0 when clean)              */
    int32_t n_points;          /* N_x                                                    */
    int32_t n_zero_obs;        /* grid points with no local observation                 */
    int32_t max_local_obs;     /* l_max: most observation points local to one point     */
    double  mean_local_obs;    /* average observation points per grid point             */
    int32_t n_chunks;          /* Gram/eigensolve launch pairs per analysis             */
    int32_t eig_schedule;      /* LETKF_EIG_FUSED / SPLIT / SPLIT_CHECK in use; AUTO (0)
                                  until the first analysis resolves it                   */
    int32_t cuda_error;        /* first cudaError_t that made a call of this handle
                                  return LETKF_ECUDA or LETKF_ENOMEM; 0 = none           */
    int32_t cycle_kernels;     /* kernel launches of the most recent letkf_cycle (or group
                                  cycle led by this handle): the kernel nodes of its
                                  captured graph; 0 before the first cycle               */
    int32_t gram_tile;         /* LETKF_GRAM_PIPE / TEAM / TENSOR in use; AUTO (0) until the
                                  first analysis resolves it                             */
} letkf_stats;

/* Device time of the phases of the most recent forecast and analysis (milliseconds, CUDA
 * events on the handle's stream), the breakdown of Fig. 3 of the paper for one GPU. */
typedef struct letkf_timings {
    float   forecast_ms;       /* all D2Q9 steps of the last forecast                   */
    int32_t forecast_steps;    /* steps (= kernel launches) in it                       */
    float   obs_ms;            /* observation operator                                   */
    float   transpose_in_ms;   /* member-major -> grid-point-major                       */
    float   gram_ms;           /* localized Gram + innovation projection, all chunks     */
    float   eigen_ms;          /* eigensolve + transform + update, all chunks            */
    float   transpose_out_ms;  /* grid-point-major -> member-major                       */
    int32_t n_chunks;          /* Gram/eigensolve launch pairs                           */
} letkf_timings;

typedef struct letkf_handle letkf_handle;

/* Per-point intermediates of one analysis, for checking (all host, may be NULL). */
typedef struct letkf_probe {
    int32_t n_points;          /* sampled points                                        */
    const int32_t *points;     /* [n_points] linear grid index y*nx + x                 */
    int32_t *nloc;             /* [n_points] local observation points                   */
    float   *gram;             /* [n_points][k][k] dY^T R_loc^-1 dY (Eq. letkf_q); the
                                  kernels form its upper triangle, the probe mirrors it  */
    float   *cvec;             /* [n_points][k]    dY^T R_loc^-1 (yo - ybar) (Eq. letkf_wa) */
    float   *eigval;           /* [n_points][k]    eigenvalues of Q, ascending          */
    float   *xf;               /* [n_points][9][k] forecast block, grid-point-major     */
} letkf_probe;

/* ---- lifecycle ------------------------------------------------------------ */

/* Device bytes a handle for *cfg needs (state, transposed state, observation
 * buffers, Gram chunk).  Validates cfg; LETKF_EINVAL if it is inconsistent. */
int letkf_workspace_size(const letkf_config *cfg, size_t *bytes);

/* Create a handle on the current CUDA device.  workspace: device memory of at
 * least letkf_workspace_size() bytes, 256-byte aligned, owned by the caller
 * and kept alive until letkf_destroy; NULL makes the handle allocate (and
 * free) its own.  Copies the force field, observation network and R, bins
 * the observation points, counts local observations per grid point, and
 * sets every member to rest (f = w_q).  *out is NULL on failure. */
int letkf_init(const letkf_config *cfg, void *workspace, size_t workspace_bytes,
               letkf_handle **out);

/* Wait for the handle's stream, return and clear the latched device status. */
int letkf_sync(letkf_handle *h);

/* Release the handle (waits for its stream first).  NULL is accepted. */
int letkf_destroy(letkf_handle *h);

/* Static text for a status code. */
const char *letkf_strerror(int code);

/* Grid, observation and local-count figures fixed at init. */
int letkf_get_stats(letkf_handle *h, letkf_stats *st);

/* on != 0: lbm_forecast, letkf_analyze and letkf_cycle record CUDA events between their
 * phases (cached cycle graphs are re-captured with the event records).  letkf_get_timings
 * waits for the last recorded event and fills *t; LETKF_ESTATE if timing is off or nothing
 * was recorded yet. */
int letkf_enable_timing(letkf_handle *h, int32_t on);
int letkf_get_timings(letkf_handle *h, letkf_timings *t);

/* ---- state in / out ------------------------------------------------------- */

/* Copy members [m0, m0+count) in or out, layout f[m][q][y][x] FP32
 * (count*9*nx*ny floats).  Members k..k+n_aux-1 are the auxiliary ones.
 * where = LETKF_HOST or LETKF_DEVICE.  Ordered on the handle's stream;
 * letkf_get_state to host memory returns after the copy has landed. */
int letkf_set_state(letkf_handle *h, const float *f, int32_t m0, int32_t count, int32_t where);
int letkf_get_state(letkf_handle *h, float *f, int32_t m0, int32_t count, int32_t where);

/* The same copies for the deviation from the rest state g_q = f_q - w_q (w_q the exact D2Q9
 * weights 4/9, 1/9, 1/36), which is what the device stores: near rest |g| ~ 1e-3 |f|, and an
 * FP32 f rounds away digits of the ensemble perturbations that g keeps (all of them below
 * ~1e-8 absolute, i.e. about 1e-5 of the rest population's perturbations). */
int letkf_set_deviation(letkf_handle *h, const float *g, int32_t m0, int32_t count, int32_t where);
int letkf_get_deviation(letkf_handle *h, float *g, int32_t m0, int32_t count, int32_t where);

/* Set members [m0, m0+count) to the D2Q9 equilibrium f^eq(rho, u) of the
 * given macroscopic fields, each [count][ny][nx] FP32 (Sec. II-A moments). */
int letkf_set_macro(letkf_handle *h, const float *rho, const float *ux, const float *uy,
                    int32_t m0, int32_t count, int32_t where);

/* ---- the hot path -------------------------------------------------------- */

/* Advance every member (ensemble and auxiliary) by nsteps time steps of the
 * lattice Boltzmann equation (Eq. 1): BGK collision with body force, then
 * periodic streaming (Sec. II-A).  nsteps >= 0. */
int lbm_forecast(letkf_handle *h, int32_t nsteps);

/* Forecast observations Y^f[m][l*V+v] = h(x_m) of the ensemble members
 * (Algorithm 1, first step), copied out as [k][L*V] FP32. */
int letkf_get_obs(letkf_handle *h, float *yf, int32_t where);

/* One LETKF analysis of the ensemble in place (Sec. II-B, Algorithm 1):
 * observation operator and obs-space perturbations (Eqs. enkf_ybar,
 * enkf_deltay), transpose to grid-point-major layout (Sec. IV-A), at every
 * grid point the localized Gram matrix and innovation projection
 * (Eqs. letkf_q, letkf_wa), the symmetric eigensolve of Q, the transform
 * (Eqs. letkf_wa, letkf_dwa) and the update (Eq. letkf_xa), then the
 * transpose back.  yo: [L*V] observations (where = LETKF_HOST/DEVICE). */
int letkf_analyze(letkf_handle *h, const float *yo, int32_t where);

/* letkf_analyze that also returns per-point intermediates in *probe. */
int letkf_analyze_probe(letkf_handle *h, const float *yo, int32_t where, letkf_probe *probe);

/* One data-assimilation cycle (Sec. II-B, cycle steps 2-3): lbm_forecast(nsteps)
 * followed by letkf_analyze(yo).  The device work of a cycle is captured
 * once per nsteps into a CUDA graph and replayed. */
int letkf_cycle(letkf_handle *h, int32_t nsteps, const float *yo, int32_t where);

/* ---- groups of co-resident ensembles ------------------------------------
 * Several experiments (handles) of one device analysed as one batch, e.g. ensembles of
 * different sizes over the same or different grids and observation networks.  Per handle the
 * observation operator, the transposes and the localized Gram matrices run as in
 * letkf_analyze.  For the handles on the LETKF_EIG_FUSED schedule the eigensolve, transform
 * and update of all their grid points run as one persistent launch per column class (k <= 32,
 * <= 64, <= 128) in which every warp takes the next grid point from a global counter, so
 * points with any number of local observations (including none) and matrices of every order
 * balance over the GPU.  Handles on the split schedules run their own split kernels in the
 * same stream.  Each handle's result equals its letkf_analyze on its schedule bit for bit.  A
 * handle on LETKF_EIG_AUTO that has not picked yet picks at its first group analysis (as at
 * its first letkf_analyze); a group cycle that contains such a handle runs without capture.
 *   hs     n distinct handles of one device, 1 <= n <= 16; the work runs on hs[0]'s stream,
 *          ordered after each handle's earlier work and before its later work
 *   yo     n observation vectors (where = LETKF_HOST/DEVICE), yo[i] of handle hs[i]
 * letkf_group_cycle(hs, n, nsteps, yo, where): every handle's lbm_forecast(nsteps) and the
 * group analysis, captured once per (membership, schedules, state buffers, nsteps) into a CUDA graph
 * kept by hs[0] (at most 8 such graphs, the oldest dropped) and replayed.  Phase timing of the
 * handles is not recorded by group calls.  Device errors are reported by each handle's
 * letkf_sync. */
int letkf_group_analyze(letkf_handle *const *hs, const float *const *yo, int32_t n,
                        int32_t where);
int letkf_group_cycle(letkf_handle *const *hs, int32_t n, int32_t nsteps,
                      const float *const *yo, int32_t where);

/* ---- local analysis without any device allocation -------------------------------
 * The paper has no counterpart of this entry point; it serves callers that cannot call
 * cudaMalloc and therefore cannot create a handle (whose workspace must be allocated by
 * someone): plugin code that a host framework hands only its input/output device buffers,
 * processes whose device memory is all reserved by another allocator, or loops in which an
 * allocation, and the device synchronisation it can imply, is not allowed.
 *
 * It solves npts independent local analyses (Gram matrix, eigensolve, transform and update
 * of each point's forecast block) given in a padded per-point layout, and allocates nothing:
 * its only scratch (the k x k Gram matrices, the c vectors, the local counts and a status
 * word) sits in one static device array of LETKF_NOALLOC_SCRATCH_BYTES that every GPU loading
 * this library holds until exit.
 *   npts       number of grid points (local problems), >= 0
 *   k          ensemble size, 2..128
 *   lmaxv      rows per point in the padded layout (the largest number of local observed
 *              scalars over the points), >= 0
 *   dy_loc     device [npts][lmaxv][k] obs-space perturbations of each point's local observed
 *              scalars, one row per scalar, padded to lmaxv rows
 *   d_loc      device [npts][lmaxv]    innovations yo - ybar of those scalars
 *   rinv_loc   device [npts][lmaxv]    localized inverse error variances G / sigma^2; 0 marks a
 *                                      padding row (its dy_loc/d_loc entries are ignored)
 *   infl       multiplicative inflation (1 = none): Q = (k-1)/infl I + dY^T R_loc^-1 dY
 *   x          device [npts][9][k] forecast blocks (grid-point-major, any fixed reference such
 *              as f or f - w), overwritten with the analysis blocks
 *   stream     cudaStream_t (NULL = legacy default stream)
 * The call synchronizes its stream (it reads the status word back before returning), so it
 * must not be called while that stream is being captured into a CUDA graph.  It returns after
 * the work has finished, with LETKF_OK, LETKF_ENOTCONV or LETKF_ENONFINITE from the device
 * status; LETKF_EINVAL, before any launch, when npts * (k*k + k + 1) + 64 floats exceed the
 * scratch (at most 15,872 points for k = 32, 4,032 for k = 64) or an argument is invalid.
 * Every call shares the one scratch array: calls that overlap on the GPU (different streams
 * or threads) race; calls ordered on one stream do not.  Each call clears the status word and
 * overwrites the scratch of the points it processes.  The first call on a device also looks
 * up the array's device address and prepares the kernels. */
#define LETKF_NOALLOC_SCRATCH_BYTES (64u << 20)
int letkf_local_analysis_noalloc(int32_t npts, int32_t k, int32_t lmaxv, const float *dy_loc,
                                 const float *d_loc, const float *rinv_loc, float infl, float *x,
                                 void *stream);

/* ---- batched symmetric eigensolver ----------------------------------------
 * The eigensolve of the analysis (Sec. III: Householder tridiagonalization, implicit-shift QL,
 * back-transform; one warp per matrix) on caller-supplied symmetric matrices, exposed on its
 * own: Q_p = V_p diag(lambda_p) V_p^T for p < npts.
 *   npts    number of matrices, >= 0
 *   k       order, 2..128
 *   q       device [npts][k][k], row-major; only the upper triangle with the diagonal is read.
 *           The strictly lower triangle is overwritten (it receives the Householder vectors);
 *           the upper triangle and the diagonal are left as they were.
 *   eigval  device [npts][k] eigenvalues, in the order of the QL (not sorted)
 *   evec    device [npts][k][k]; row i is the unit eigenvector of eigval[p][i]; NULL = skip
 *   refine  1: one FP64 sweep over clustered eigenpairs (eigenvalues within relative distance
 *           1e-6 of another, closer than the FP32 solve resolves): modified Gram-Schmidt within
 *           the neighbourhood, then the Rayleigh quotient v^T Q v as the eigenvalue; 0: FP32
 *           only
 *   stream  cudaStream_t (NULL = legacy default stream)
 * Allocates nothing.  Returns after the work has finished: LETKF_OK, LETKF_ENOTCONV (some QL
 * iteration cap was hit) or LETKF_ENONFINITE; LETKF_EINVAL for bad arguments.  It
 * synchronizes its stream, so it must not be called while that stream is being captured.  The
 * status word shares the static scratch of letkf_local_analysis_noalloc: the same overlap rule
 * holds. */
int letkf_eigh_batch(int32_t npts, int32_t k, float *q, float *eigval, float *evec,
                     int32_t refine, void *stream);

/* letkf_eigh_batch on the split schedule (the analysis' LETKF_EIG_SPLIT: tridiagonalization one
 * warp per matrix, the QL recurrence one thread per matrix with its rotations recorded, then
 * the rotations replayed onto the eigenvectors and the back-transform one warp per matrix;
 * a matrix whose record would overflow is recomputed by the one-warp schedule).  Same
 * arguments, results and return codes as letkf_eigh_batch (the eigenpairs agree to FP32
 * rounding), with the scratch in a caller-owned device workspace instead of the static array:
 *   workspace        device buffer of at least letkf_eigh_workspace_bytes(npts, k) bytes,
 *                    256-byte aligned; its contents on entry do not matter and are overwritten
 *   workspace_bytes  its size
 * Returns LETKF_ENOMEM when the workspace is too small or misaligned.  Like letkf_eigh_batch it
 * synchronizes its stream (not callable during stream capture).  Calls that share a workspace
 * race unless they are ordered on one stream. */
size_t letkf_eigh_workspace_bytes(int32_t npts, int32_t k);
int letkf_eigh_batch_ws(int32_t npts, int32_t k, float *q, float *eigval, float *evec,
                        int32_t refine, void *workspace, size_t workspace_bytes, void *stream);

/* ---- diagnostics ------------------------------------------------------------
 * FP32 FMA throughput microbenchmark: the measured peak that the ALU-bound kernels (the
 * eigensolve, the plain FP32 Gram) are reported against.  Not part of the method.
 * letkf_fp32_peak_grid: the launch's blocks (every SM filled with resident blocks) and threads.
 * letkf_fp32_peak_run: one launch on stream in which every thread runs 16 independent chains
 *   x <- fma(x, a, b) for iters x 8 rounds; out: device buffer of blocks * threads floats (the
 *   chains' sums); *flops = 2 x the FMAs executed.  The caller times the launch (CUDA events on
 *   the stream).  LETKF_EINVAL for iters < 1 or NULL pointers. */
int letkf_fp32_peak_grid(int32_t *blocks, int32_t *threads);
int letkf_fp32_peak_run(int32_t iters, float *out, int64_t *flops, void *stream);

/* The coefficients of LETKF_EIG_RATIONAL (host computation, FP64): Zolotarev's best n-term
 * rational approximation t^-1/2 ~ sum_l residues[l] / (t + poles[l]) on [1/kappa_max, 1]
 * (poles and residues: caller arrays of n doubles, 1 <= n <= 16, 1 < kappa_max < 1e12).
 * Returns the largest relative error found on a fine logarithmic grid of the interval, or -1
 * for invalid arguments. */
double letkf_rational_coefficients(double kappa_max, int32_t n, double *poles,
                                   double *residues);

/* The coefficients of LETKF_EIG_CHEBYSHEV (host computation, FP64): the degree-n interpolants
 * at the Chebyshev points of the first kind of t^-1/2 (c_rsqrt) and t^-1 (c_inv) on
 * [1, kappa_max], as coefficients of T_0..T_n in s = (2 t - kappa_max - 1) / (kappa_max - 1)
 * (caller arrays of n + 1 doubles, 1 <= n <= 256, 1 < kappa_max < 1e6).  Returns the larger of
 * the two largest relative errors on a fine grid of the interval, or -1 for invalid
 * arguments. */
double letkf_chebyshev_coefficients(double kappa_max, int32_t n, double *c_rsqrt,
                                    double *c_inv);

/* Cumulative counts of the LETKF_EIG_CHEBYSHEV transform on this handle since letkf_init
 * (device counters, also advanced by the AUTO tuner's trial runs): counts[0] grid points
 * transformed, counts[1] products with A formed (the sum of the degrees used), counts[2]
 * points passed on to the RATIONAL schedule.  Waits for the handle's stream; LETKF_EINVAL for
 * NULL arguments. */
int letkf_get_work_counts(letkf_handle *h, int64_t *counts);

#ifdef __cplusplus
}
#endif
#endif /* LETKF_H */
