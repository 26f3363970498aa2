// Host-side launchers of the library's kernels (internal to libletkf).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lk {

// Device status bits latched with atomicOr and turned into LETKF_E* codes by the host.
enum : int {
    ST_NOTCONV = 1,
    ST_NONFINITE = 2,
    ST_TIMEOUT = 4,
    ST_BADINDEX = 8,
};

// Static observation network, binned into cs x cs cells, and the localization.
struct ObsNet {
    const int2 *xy;         // [L] observation points (x, y)
    const int *cell_start;  // [ncx*ncy + 1] CSR offsets into cell_obs
    const int *cell_obs;    // [L] observation indices, grouped by cell, ascending within a cell
    int L, V;               // points and observed variables per point
    int cs, ncx, ncy;       // cell edge and number of cells per axis
    int loc_none;           // 1: every observation is local with weight 1
    int d2max;              // local iff integer squared periodic distance <= d2max
    int cr;                 // largest |dx| with dx^2 <= d2max (search half-width in cells)
    float inv2r2;           // 1 / (2 r^2) of the Gaussian weight
    int loc_gc;             // 1: Gaspari-Cohn weight GC(d / c) instead of the Gaussian
    float inv_c;            // 1 / c, c = sqrt(10/3) r (Gaspari-Cohn half-width)
};

// ---- lbm.cu -------------------------------------------------------------------
cudaError_t launch_lbm_step(const float *gin, float *gout, const float2 *force, int nx, int ny,
                            int nmem, float tau, cudaStream_t s);
// two steps in one launch (temporal blocking through shared memory); lbm_prepare once
cudaError_t lbm_prepare();
// Tensor-memory-access (TMA) descriptors of the two-step launch's staging: an opaque image of
// the driver's 128-byte tensor map, for each of the two state buffers and the force.
struct alignas(64) TmaMap {
    unsigned long long w[16];
};
struct LbmTma {
    TmaMap g[2];
    TmaMap f;
    const float *gptr[2] = {nullptr, nullptr};
    int ok = 0;                   // 1: state maps built, 2: force map built
};
// builds the maps where the grid allows them (nx a multiple of 4, at least one tile plus its
// halo) and the driver offers the encoder; leaves ok = 0 otherwise (the staging then uses
// cp.async throughout); an error if the encoder rejects a map
cudaError_t lbm_tma_build(const float *g0, const float *g1, const float2 *force, int nx, int ny,
                          int nmem, LbmTma *out);
// with tma (nullable) the interior tiles stage through TMA; status receives ST_TIMEOUT if a
// staging wait runs out
cudaError_t launch_lbm_2step(const float *gin, float *gout, const float2 *force, int nx, int ny,
                             int nmem, float tau, cudaStream_t s, const LbmTma *tma = nullptr,
                             int *status = nullptr);
cudaError_t launch_f_to_g(const float *f, float *g, int nmem, size_t npts, cudaStream_t s);
cudaError_t launch_g_to_f(const float *g, float *f, int nmem, size_t npts, cudaStream_t s);
cudaError_t launch_macro_to_g(const float *rho, const float *ux, const float *uy, float *g,
                              int nmem, size_t npts, cudaStream_t s);

// ---- obs.cu -------------------------------------------------------------------
struct ObsOpArgs {
    const float *g;         // state [nmem][9][N] (shifted populations)
    const int2 *xy;         // [L]
    int L, nx, ny, k, kp;
    int nmem;               // members observed (k ensemble members first, then auxiliary)
    int obs_vars;           // LETKF_OBS_* mask
    float *yf;              // [nmem][L*V] h(x_m)
    float *yb;              // [L*V][kp]  h(x_m) - mean, zero in columns k..kp-1
    float *ybar;            // [L*V]      mean minus the variable's reference (1 for rho)
};
cudaError_t launch_obs_operator(const ObsOpArgs &a, cudaStream_t s);
cudaError_t launch_count_local(const ObsNet &net, int nx, int ny, int *nloc, cudaStream_t s);

// ---- transpose.cu -------------------------------------------------------------
// member-major g[m][q][p] <-> grid-point-major x[p][q][m], members 0..k-1, p in [0, npts).
cudaError_t launch_transpose_in(const float *g, float *x, int k, size_t npts, cudaStream_t s);
cudaError_t launch_transpose_out(const float *x, float *g, int k, size_t npts, cudaStream_t s);

// ---- gram.cu ------------------------------------------------------------------
struct GramArgs {
    ObsNet net;
    int nx, ny, k, kp;
    const float *yb;        // [L*V][kp]
    const float *ybar;      // [L*V]
    const float *yo;        // [L*V]
    const float *rinv;      // [L*V] 1 / sigma^2
    float yref[3];          // reference of each observed variable (1 for rho, else 0)
    int y_begin, y_end;     // grid rows of this chunk
    const float4 *orec;     // tensor-core form: observation records in bin order [L*V]
    float *gram;            // [(y_end-y_begin)*nx][k][k]
    float *cvec;            // [(y_end-y_begin)*nx][k]
    int *nloc;              // [(y_end-y_begin)*nx]
    int team = 0;           // FP32, kp >= 32: 1 the team kernel, 0 the pipelined one
};
cudaError_t gram_prepare(int kp);            // once per process and kp
// tensor-core (tcgen05) split-FP16 form for kp = 64 or 128; persistent, <= max_ctas CTAs
cudaError_t gram_tc_prepare(int kp);
cudaError_t launch_gram_tc(const GramArgs &a, int *status, int max_ctas, cudaStream_t s);
// records for launch_gram_tc, rebuilt whenever yo or ybar change
cudaError_t launch_obs_records(const GramArgs &a, float4 *rec, cudaStream_t s);
int gram_tc_tile_width(int kp);
int gram_tc_tile_height(int kp);
cudaError_t launch_gram(const GramArgs &a, cudaStream_t s);
// tile of the FP32 Gram: the team kernel (team = 1, and every kp <= 16) or the pipelined one
int gram_tile_width(int kp, int team);
int gram_tile_height(int kp, int team);
int gram_max_cells();

// ---- eigen.cu -----------------------------------------------------------------
struct EigArgs {
    int k = 0;
    float diag = 0.0f;              // (k - 1) / rho_infl
    float sqrt_infl = 1.0f;         // sqrt(rho_infl): a point without local observations keeps
                                    // its mean and has its perturbations scaled by it
    float *gram = nullptr;          // [npts][k][k]; Q is read from the upper triangle and the
                                    // diagonal, the Householder vectors go to the lower one
    const float *cvec = nullptr;    // [npts][k]
    const int *nloc = nullptr;      // [npts]
    float *x = nullptr;             // grid-point-major ensemble [N][9][k], updated in place
    long long pt0 = 0;              // first grid point of the chunk
    int npts = 0;
    float *eigval = nullptr;        // [npts][k] eigenvalues; optional for the fused schedule
    int *status = nullptr;          // device status word
    int max_blocks = 0;             // resident grid of the fused kernel (eigen_prepare)
    const int *list = nullptr;      // only these points (count in *list_count): the fused
    const int *list_count = nullptr;  // kernel, the tridiagonalizations, the rational transform
    float *evec = nullptr;          // optional [npts][k][k]: row i = eigenvector of eigval[i]
    int refine = 0;                 // FP64 refinement sweep of clustered eigenpairs
    float refine_tau = 0.0f;        // relative eigenvalue distance that makes a cluster
    unsigned long long *work = nullptr;  // optional [3] counters added to by the Chebyshev
                                         // transform: points, products, points handed on
};
// Split schedule: scratch of one chunk and the resident grids of its kernels.
struct EigSplit {
    float2 *de = nullptr;           // [npts][k] tridiagonal (d_t, e_t)
    float *taus = nullptr;          // [npts][k] reflector scalars
    float2 *rot = nullptr;          // [npts][rcap] recorded QL rotations
    int *nrot = nullptr;            // [npts] record length, -1: handed to the fused kernel
    int *list = nullptr;            // [npts] points handed to the fused kernel
    int *list_count = nullptr;      // [1]
    int *pre_list = nullptr;        // [npts] points the Chebyshev transform hands to the
    int *pre_count = nullptr;       // [1]    rational schedule
    int list_offset = 0;            // added to a point's index when it is listed
    int rcap = 0;                   // record capacity per point (entries)
    int grid_tri = 0, grid_vec = 0; // resident grids (eigen_split_prepare)
};
// Grouped schedule: the points of several chunks (segments) of any k, one persistent launch
// per column class (k <= 32, <= 64, <= 128) with dynamic work distribution.
constexpr int kMaxGroupSeg = 16;  // segments per column class and launch
struct EigGroup {
    int n;                       // segments
    int kmax;                    // largest k among them: each warp's shared-memory slice
    int start[kMaxGroupSeg + 1]; // prefix of the segments' point counts
    int *counter;                // zeroed before the launch
    EigArgs seg[kMaxGroupSeg];
};
cudaError_t eigen_group_prepare(int *max_blocks);  // max_blocks[3], once per process
// segs: up to 3 kMaxGroupSeg chunks; counters: 3 device ints; max_blocks from the prepare
cudaError_t launch_eigen_group(const EigArgs *segs, int n, int *counters, const int *max_blocks,
                               cudaStream_t s);
// EVD-free transform (LETKF_EIG_RATIONAL, k <= kRationalMaxK): Zolotarev's rational
// approximations of t^-1/2 on [1/kappa_max, 1], FP32 copies of the FP64 coefficients.
constexpr int kZoloSets = 5;
constexpr int kMaxZoloPoles = 16;
constexpr int kRationalMaxK = 64;
struct ZoloTable {
    float kappa_max[kZoloSets];
    int n[kZoloSets];
    float pole[kZoloSets][kMaxZoloPoles];   // t^-1/2 ~ sum_l res_l / (t + pole_l)
    float res[kZoloSets][kMaxZoloPoles];
};
const ZoloTable &zolo_table();              // computed once per process (zolotarev.cu)
double zolotarev_rsqrt(double kappa, int n, double *poles, double *residues);
cudaError_t eigen_rational_prepare(int k, int *grid);
// the transform kernel alone (after the tridiagonalization); hands points beyond the largest
// approximation's range to the fused kernel through sp.list
cudaError_t launch_eigen_rational_transform(const EigArgs &a, const EigSplit &sp, int grid,
                                            cudaStream_t s);
// the whole schedule: tridiagonalization, eigenvalues if a.eigval (values-only QL), the
// transform, then the fused kernel over the handed-off points; sp needs de, taus, list and
// list_count (no rotation record)
cudaError_t launch_eigen_rational(const EigArgs &a, const EigSplit &sp, int grid,
                                  cudaStream_t s);

// EVD-free transform by Chebyshev expansions of t^-1/2 and t^-1 on [1, kappa_max]
// (LETKF_EIG_CHEBYSHEV, k <= kChebMaxK): coefficients of T_j in s = (2t - kappa_max - 1) /
// (kappa_max - 1), FP32 copies of the FP64 interpolants, the first set that covers a point's
// condition bound is used.
constexpr int kChebSets = 15;
constexpr int kChebMaxDeg = 36;
constexpr int kChebMaxK = 64;
struct ChebTable {
    float kappa_max[kChebSets];
    int n[kChebSets];                        // degree
    float2 c[kChebSets][kChebMaxDeg + 1];    // (t^-1/2, t^-1) coefficients of T_0 .. T_n
};
const ChebTable &cheb_table();              // computed once per process (chebyshev.cu)
int cheb_max_set(int k);                    // the largest set used at ensemble size k
double chebyshev_coefficients(double kappa, int n, double *ca, double *cb);
cudaError_t eigen_cheb_prepare(int k, int *grid);
// the Chebyshev transform alone; points beyond the last set go to sp.pre_list
cudaError_t launch_eigen_cheb_transform(const EigArgs &a, const EigSplit &sp, int grid,
                                        cudaStream_t s);
// the whole schedule: the Chebyshev transform, then the rational schedule over the points it
// handed on (sp needs de, taus, list, list_count, pre_list and pre_count)
cudaError_t launch_eigen_chebyshev(const EigArgs &a, const EigSplit &sp, int cheb_grid,
                                   int rat_grid, cudaStream_t s);

cudaError_t eigen_prepare(int k, int *max_blocks);  // once per process and k
cudaError_t eigen_split_prepare(int k, EigSplit *sp);
cudaError_t launch_eigen_update(const EigArgs &a, cudaStream_t s);
// With a second stream s2 and two events (all non-null) a large chunk (k <= 32) runs as two
// halves whose kernels overlap: the second half's tridiagonalization with the first half's QL,
// the first half's vectors with the second half's QL.  Same results as the one-stream order.
cudaError_t launch_eigen_split(const EigArgs &a, const EigSplit &sp, cudaStream_t s,
                               cudaStream_t s2 = nullptr, cudaEvent_t fork = nullptr,
                               cudaEvent_t join = nullptr);
size_t eigen_smem_per_warp(int k);

}  // namespace lk
