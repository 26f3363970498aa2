// C ABI of libletkf: handle lifecycle, device workspace, and the hot-path entry points.
//
// Host code only; every arithmetic step of the method runs in the kernels of
// lbm.cu, obs.cu, transpose.cu, gram.cu and eigen.cu.  The host builds the
// static observation bins once at init and orders the launches of a cycle:
//   lbm_forecast:   nsteps x D2Q9 step (ping-pong between two state buffers)
//   letkf_analyze:  yo -> device, observation operator, transpose to
//                   grid-point-major, then per chunk of grid rows the Gram
//                   kernel and the eigensolve/transform/update kernel, then the
//                   transpose back.
//   letkf_cycle:    both, captured once per (nsteps, buffer parity) into a
//                   CUDA graph and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <numeric>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "kernels.h"
#include "letkf.h"

namespace {

constexpr size_t kAlign = 256;
constexpr int64_t kDefaultChunkBytes = 1ll << 30;  // 1 GiB: 65,536 points at k = 64

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int kp_of(int k) { return k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : k <= 64 ? 64 : 128; }

int popcount3(int v) { return (v & 1) + ((v >> 1) & 1) + ((v >> 2) & 1); }

// Everything derived from the configuration that fixes sizes.
struct Plan {
    size_t npts = 0;
    int nmem = 0, V = 0, LV = 0, kp = 0;
    int tile_w = 1, tile_h = 1;
    bool tensor_gram = false;  // mixed precision with k in 17..128: tcgen05 split-FP16 Gram
    int eig_schedule = LETKF_EIG_FUSED;  // as configured; AUTO keeps both schedules' scratch
    int rcap = 0;              // split schedule: rotation record entries per point
    int chunk_rows = 0;
    size_t chunk_pts = 0;
    int cs = 8, ncx = 1, ncy = 1;
    int d2max = 0, cr = 0;
    float inv2r2 = 0.0f;
    float inv_c = 0.0f;  // Gaspari-Cohn: 1 / (sqrt(10/3) r)
    // byte offsets inside the workspace
    size_t off_state[2], off_force, off_xg, off_obs_xy, off_cell_start, off_cell_obs, off_rinv,
        off_yf, off_yb, off_ybar, off_yo, off_orec, off_gram, off_cvec, off_nloc, off_nloc_all,
        off_eigval, off_de, off_taus, off_rot, off_nrot, off_list, off_pre_list, off_status,
        total;
};

int validate(const letkf_config *c) {
    if (!c) return LETKF_EINVAL;
    if (c->nx < 1 || c->ny < 1 || (int64_t)c->nx * c->ny > (1ll << 30)) return LETKF_EINVAL;
    if (c->k < 2 || c->k > 128 || c->n_aux < 0 || c->n_aux > 4) return LETKF_EINVAL;
    if (!(c->tau > 0.5f) || !isfinite(c->tau)) return LETKF_EINVAL;
    if (c->n_obs < 0 || (c->n_obs > 0 && (!c->obs_xy || !c->obs_err_var))) return LETKF_EINVAL;
    if (c->obs_vars < 1 || c->obs_vars > 7) return LETKF_EINVAL;
    if (c->loc_kind != LETKF_LOC_NONE && c->loc_kind != LETKF_LOC_GAUSS &&
        c->loc_kind != LETKF_LOC_GC)
        return LETKF_EINVAL;
    if (c->loc_kind != LETKF_LOC_NONE && !(c->loc_radius > 0.0f && isfinite(c->loc_radius)))
        return LETKF_EINVAL;
    if (!(c->infl > 0.0f) || !isfinite(c->infl)) return LETKF_EINVAL;
    if (c->precision != LETKF_FP32 && c->precision != LETKF_MIXED) return LETKF_EINVAL;
    if (c->eig_schedule < LETKF_EIG_AUTO || c->eig_schedule > LETKF_EIG_CHEBYSHEV)
        return LETKF_EINVAL;
    if (c->eig_schedule == LETKF_EIG_RATIONAL && c->k > lk::kRationalMaxK) return LETKF_EINVAL;
    if (c->eig_schedule == LETKF_EIG_CHEBYSHEV && c->k > lk::kChebMaxK) return LETKF_EINVAL;
    if (c->gram_tile < LETKF_GRAM_AUTO || c->gram_tile > LETKF_GRAM_TEAM) return LETKF_EINVAL;
    if (c->chunk_bytes < 0) return LETKF_EINVAL;
    const int V = popcount3(c->obs_vars);
    for (int l = 0; l < c->n_obs; ++l) {
        const int x = c->obs_xy[2 * l], y = c->obs_xy[2 * l + 1];
        if (x < 0 || x >= c->nx || y < 0 || y >= c->ny) return LETKF_EINVAL;
        for (int v = 0; v < V; ++v) {
            const float r = c->obs_err_var[(size_t)l * V + v];
            if (!(r > 0.0f) || !isfinite(r)) return LETKF_EINVAL;
        }
    }
    return LETKF_OK;
}

int make_plan(const letkf_config *c, Plan *p) {
    const int rc = validate(c);
    if (rc != LETKF_OK) return rc;
    p->npts = (size_t)c->nx * c->ny;
    p->nmem = c->k + c->n_aux;
    p->V = popcount3(c->obs_vars);
    p->LV = c->n_obs * p->V;
    p->kp = kp_of(c->k);
    // the bins must hold the patch of either FP32 tile schedule, and a chunk holds whole tiles
    // of both
    p->tile_w = std::max(lk::gram_tile_width(p->kp, 0), lk::gram_tile_width(p->kp, 1));
    p->tile_h = std::lcm(lk::gram_tile_height(p->kp, 0), lk::gram_tile_height(p->kp, 1));
    // (the tensor-core kernel's records pack a point as x | y << 16 and a scalar's row with
    // its variable in bits 28..29)
    p->tensor_gram = c->precision == LETKF_MIXED && p->kp >= 32 && c->nx < 65536 &&
                     c->ny < 65536 && p->LV < (1 << 28);
    if (p->tensor_gram) {  // the bins must fit either kernel's tile patch
        p->tile_w = std::max(p->tile_w, lk::gram_tc_tile_width(p->kp));
        p->tile_h = std::max(p->tile_h, lk::gram_tc_tile_height(p->kp));
    }
    // localization: integer threshold of the strict cutoff d^2 < c^2 (Sec. II-B)
    if (c->loc_kind != LETKF_LOC_NONE) {
        const double r = c->loc_radius;
        const double c2 = c->loc_cutoff2 > 0.0f ? (double)c->loc_cutoff2 : 40.0 * r * r / 3.0;
        // Gaspari-Cohn: the observations inside min(cutoff, its support 2c) count as local
        const double c2e = c->loc_kind == LETKF_LOC_GC ? std::min(c2, 40.0 * r * r / 3.0) : c2;
        const double lim = ceil(c2e) - 1.0;
        p->d2max = lim > 2.0e9 ? 2000000000 : (int)lim;
        if (p->d2max < 0) p->d2max = -1;
        int cr = (int)sqrt((double)std::max(p->d2max, 0));
        while ((long long)(cr + 1) * (cr + 1) <= p->d2max) ++cr;
        while (cr > 0 && (long long)cr * cr > p->d2max) --cr;
        p->cr = p->d2max < 0 ? 0 : cr;
        p->inv2r2 = (float)(1.0 / (2.0 * r * r));
        p->inv_c = (float)(1.0 / (sqrt(10.0 / 3.0) * r));
    }
    // bins: smallest power-of-two edge (>= 8) whose patch of one Gram tile fits the kernel
    const int maxc = lk::gram_max_cells();
    for (p->cs = 8;; p->cs *= 2) {
        p->ncx = (c->nx + p->cs - 1) / p->cs;
        p->ncy = (c->ny + p->cs - 1) / p->cs;
        long long bx, by;
        if (c->loc_kind == LETKF_LOC_NONE) {
            bx = p->ncx;
            by = p->ncy;
        } else {
            bx = std::min<long long>(p->ncx, (p->tile_w + 2 * p->cr + p->cs - 1) / p->cs + 2);
            by = std::min<long long>(p->ncy, (p->tile_h + 2 * p->cr + p->cs - 1) / p->cs + 2);
        }
        if (bx * by <= maxc) break;
    }
    // Gram chunk: whole multiples of the tile height, within chunk_bytes
    const int64_t budget = c->chunk_bytes > 0 ? c->chunk_bytes : kDefaultChunkBytes;
    const size_t row_bytes = (size_t)c->nx * c->k * c->k * sizeof(float);
    int rows = (int)std::max<int64_t>(1, budget / (int64_t)row_bytes);
    rows = std::max(p->tile_h, rows / p->tile_h * p->tile_h);
    if (rows >= c->ny) rows = c->ny;
    p->chunk_rows = rows;
    p->chunk_pts = (size_t)rows * c->nx;

    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = align_up(off, kAlign);
        const size_t o = off;
        off += std::max<size_t>(bytes, 1);
        return o;
    };
    const size_t state_bytes = (size_t)p->nmem * 9 * p->npts * sizeof(float);
    p->off_state[0] = take(state_bytes);
    p->off_state[1] = take(state_bytes);
    p->off_force = take(c->force ? p->npts * sizeof(float2) : 0);
    p->off_xg = take(p->npts * 9 * c->k * sizeof(float));
    p->off_obs_xy = take((size_t)c->n_obs * sizeof(int2));
    p->off_cell_start = take(((size_t)p->ncx * p->ncy + 1) * sizeof(int));
    p->off_cell_obs = take((size_t)c->n_obs * sizeof(int));
    p->off_rinv = take((size_t)p->LV * sizeof(float));
    p->off_yf = take((size_t)p->nmem * p->LV * sizeof(float));
    p->off_yb = take((size_t)p->LV * p->kp * sizeof(float));
    p->off_ybar = take((size_t)p->LV * sizeof(float));
    p->off_yo = take((size_t)p->LV * sizeof(float));
    p->off_orec = take(p->tensor_gram ? (size_t)p->LV * sizeof(float4) : 0);
    p->off_gram = take(p->chunk_pts * c->k * c->k * sizeof(float));
    p->off_cvec = take(p->chunk_pts * c->k * sizeof(float));
    p->off_nloc = take(p->chunk_pts * sizeof(int));
    p->off_nloc_all = take(p->npts * sizeof(int));
    p->off_eigval = take(p->chunk_pts * c->k * sizeof(float));
    // split eigensolve: the schedule, and a record of about twice the rotations that the
    // implicit QL needs on these matrices (~k^2 / 2; overflowing points go to the fused kernel)
    p->eig_schedule = c->eig_schedule;
    // (d, e), reflector scalars and the hand-off list: every schedule but FUSED; the rotation
    // record: the split schedules (and AUTO, which may pick one)
    const bool split = p->eig_schedule != LETKF_EIG_FUSED;
    const bool record = split && p->eig_schedule != LETKF_EIG_RATIONAL &&
                        p->eig_schedule != LETKF_EIG_CHEBYSHEV;
    p->rcap = !record ? 0
              : p->eig_schedule == LETKF_EIG_SPLIT_CHECK ? c->k : c->k * c->k + 4 * c->k;
    p->off_de = take(split ? p->chunk_pts * c->k * sizeof(float2) : 0);
    p->off_taus = take(split ? p->chunk_pts * c->k * sizeof(float) : 0);
    p->off_rot = take(record ? p->chunk_pts * (size_t)p->rcap * sizeof(float2) : 0);
    p->off_nrot = take(record ? p->chunk_pts * sizeof(int) : 0);
    p->off_list = take(split ? (p->chunk_pts + 4) * sizeof(int) : 0);
    // the Chebyshev transform's hand-off list (CHEBYSHEV, and AUTO where it is a candidate)
    const bool cheb = (p->eig_schedule == LETKF_EIG_CHEBYSHEV ||
                       p->eig_schedule == LETKF_EIG_AUTO) && c->k <= lk::kChebMaxK;
    p->off_pre_list = take(cheb ? (p->chunk_pts + 4) * sizeof(int) : 0);
    p->off_status = take(kAlign);
    p->total = align_up(off, kAlign);
    return LETKF_OK;
}

}  // namespace

struct letkf_handle {
    letkf_config cfg;
    Plan plan;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the split eigensolve's second stream and its fork/join events (halves of a chunk overlap)
    cudaStream_t stream2 = nullptr;
    cudaEvent_t split_fork = nullptr, split_join = nullptr;
    // in a group: the stream of this handle's own branch and its fork/join events
    cudaStream_t gstream = nullptr;
    cudaEvent_t gfork = nullptr, gjoin = nullptr;
    unsigned char *ws = nullptr;
    bool own_ws = false;
    float *state[2] = {nullptr, nullptr};
    int cur = 0;
    float2 *force = nullptr;
    lk::LbmTma lbm_tma;           // TMA descriptors of the two-step D2Q9 staging
    float *xg = nullptr, *rinv = nullptr, *yf = nullptr, *yb = nullptr, *ybar = nullptr,
          *yo = nullptr, *gram = nullptr, *cvec = nullptr, *eigval = nullptr;
    float4 *orec = nullptr;
    int2 *obs_xy = nullptr;
    int *cell_start = nullptr, *cell_obs = nullptr, *nloc = nullptr, *nloc_all = nullptr,
        *status = nullptr;
    lk::ObsNet net;
    float yref[3] = {0, 0, 0};
    int eig_blocks = 0;
    lk::EigSplit eig_split;
    int eig_schedule = LETKF_EIG_FUSED;  // resolved: FUSED, SPLIT, SPLIT_CHECK or RATIONAL
    int rat_grid = 0;                    // resident grid of the EVD-free transform kernel
    int cheb_grid = 0;                   // resident grid of the Chebyshev transform kernel
    int gram_tile = LETKF_GRAM_PIPE;     // resolved: PIPE, TEAM or TENSOR; AUTO until tuned
    int tc_ctas = 0;
    letkf_stats stats;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_nsteps[2] = {-1, -1};
    int graph_kernels[2] = {0, 0};  // kernel nodes of each captured cycle
    unsigned long long serial = 0;  // unique per handle of the process (group graph keys)
    struct GroupGraph {             // captured group cycles led by this handle
        std::vector<unsigned long long> members;
        std::vector<int> cur, sched;
        int nsteps = -1;
        int kernels = 0;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<GroupGraph> group_graphs;
    int latched = 0;  // host-side error waiting for letkf_sync
    // phase timing: forecast start/end, then analysis boundaries
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // [0..1] forecast, [2..] analysis (4 + 2 * chunks)
    int fc_steps = -1;            // steps of the last timed forecast
    bool an_done = false;         // an analysis has been timed
};

namespace {

// Kernel nodes of a captured graph (the launches one replay makes).
int graph_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int kernels = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            ++kernels;
    }
    return kernels;
}

int cuda_fail(letkf_handle *h, cudaError_t e) {
    if (e == cudaSuccess) return LETKF_OK;
    if (h && !h->latched) h->latched = LETKF_ECUDA;
    if (h && !h->stats.cuda_error) h->stats.cuda_error = (int32_t)e;
    return e == cudaErrorMemoryAllocation ? LETKF_ENOMEM : LETKF_ECUDA;
}

#define CK(expr)                                            \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) return cuda_fail(h, e__);   \
    } while (0)

int device_check(letkf_handle *h) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LETKF_ECUDA;
    if (dev != h->device) CK(cudaSetDevice(h->device));
    return LETKF_OK;
}

int copy_in(letkf_handle *h, void *dst, const void *src, size_t bytes, int where) {
    if (where != LETKF_HOST && where != LETKF_DEVICE) return LETKF_EINVAL;
    if (bytes == 0) return LETKF_OK;
    CK(cudaMemcpyAsync(dst, src, bytes,
                       where == LETKF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       h->stream));
    return LETKF_OK;
}

int copy_out(letkf_handle *h, void *dst, const void *src, size_t bytes, int where) {
    if (where != LETKF_HOST && where != LETKF_DEVICE) return LETKF_EINVAL;
    if (bytes == 0) return LETKF_OK;
    CK(cudaMemcpyAsync(dst, src, bytes,
                       where == LETKF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       h->stream));
    if (where == LETKF_HOST) CK(cudaStreamSynchronize(h->stream));
    return LETKF_OK;
}

int n_chunks(const letkf_handle *h) {
    return (h->cfg.ny + h->plan.chunk_rows - 1) / h->plan.chunk_rows;
}

// Phase boundary event.  Inside a stream capture the record must be an external event node,
// otherwise the capture only uses it as an internal dependency and never records it.
int mark(letkf_handle *h, int idx) {
    if (!h->timing) return LETKF_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(h->stream, &cs));
    if (cs == cudaStreamCaptureStatusActive)
        CK(cudaEventRecordWithFlags(h->ev[idx], h->stream, cudaEventRecordExternal));
    else
        CK(cudaEventRecord(h->ev[idx], h->stream));
    return LETKF_OK;
}

// Ping-pong buffer flips of a forecast: two steps per launch, a single step for an odd rest.
int forecast_flips(int nsteps) { return nsteps / 2 + (nsteps & 1); }

int enqueue_forecast(letkf_handle *h, int nsteps) {
    const Plan &p = h->plan;
    int rc = mark(h, 0);
    if (rc) return rc;
    for (int s = 0; s + 2 <= nsteps; s += 2) {
        CK(lk::launch_lbm_2step(h->state[h->cur], h->state[h->cur ^ 1], h->force, h->cfg.nx,
                                h->cfg.ny, p.nmem, h->cfg.tau, h->stream, &h->lbm_tma,
                                h->status));
        h->cur ^= 1;
    }
    if (nsteps & 1) {
        CK(lk::launch_lbm_step(h->state[h->cur], h->state[h->cur ^ 1], h->force, h->cfg.nx,
                               h->cfg.ny, p.nmem, h->cfg.tau, h->stream));
        h->cur ^= 1;
    }
    if (h->timing) h->fc_steps = nsteps;
    return mark(h, 1);
}

int enqueue_obs(letkf_handle *h) {
    const Plan &p = h->plan;
    lk::ObsOpArgs o;
    o.g = h->state[h->cur];
    o.xy = h->obs_xy;
    o.L = h->cfg.n_obs;
    o.nx = h->cfg.nx;
    o.ny = h->cfg.ny;
    o.k = h->cfg.k;
    o.kp = p.kp;
    o.nmem = p.nmem;
    o.obs_vars = h->cfg.obs_vars;
    o.yf = h->yf;
    o.yb = h->yb;
    o.ybar = h->ybar;
    CK(lk::launch_obs_operator(o, h->stream));
    return LETKF_OK;
}

// Analysis kernels after yo is on the device.  probe may be NULL.
lk::GramArgs gram_args(letkf_handle *h, int y0, int y1) {
    lk::GramArgs g;
    g.net = h->net;
    g.nx = h->cfg.nx;
    g.ny = h->cfg.ny;
    g.k = h->cfg.k;
    g.kp = h->plan.kp;
    g.yb = h->yb;
    g.ybar = h->ybar;
    g.yo = h->yo;
    g.rinv = h->rinv;
    for (int v = 0; v < 3; ++v) g.yref[v] = h->yref[v];
    g.y_begin = y0;
    g.y_end = y1;
    g.gram = h->gram;
    g.cvec = h->cvec;
    g.nloc = h->nloc;
    g.orec = h->orec;
    g.team = h->gram_tile == LETKF_GRAM_TEAM ? 1 : 0;
    return g;
}

// Gram matrices and c of the chunk of rows [y0, y1) (the chunk index selects the records pass)
int enqueue_gram_chunk(letkf_handle *h, int chunk, int y0, int y1) {
    const lk::GramArgs g = gram_args(h, y0, y1);
    if (h->plan.tensor_gram && chunk == 0) CK(lk::launch_obs_records(g, h->orec, h->stream));
    if (h->plan.tensor_gram)
        CK(lk::launch_gram_tc(g, h->status, h->tc_ctas, h->stream));
    else
        CK(lk::launch_gram(g, h->stream));
    return LETKF_OK;
}

// The handle's status block (kAlign bytes, zeroed at letkf_init): word 0 the latched status
// bits, words 16..18 the grouped launches' work counters, bytes 128..151 the Chebyshev
// transform's cumulative counts (points, products, points handed on).
unsigned long long *work_counters(letkf_handle *h) {
    return reinterpret_cast<unsigned long long *>(h->status + 32);
}

lk::EigArgs eig_args(letkf_handle *h, int y0, int y1) {
    const int k = h->cfg.k;
    lk::EigArgs e;
    e.k = k;
    e.diag = (float)((double)(k - 1) / (double)h->cfg.infl);
    e.sqrt_infl = (float)sqrt((double)h->cfg.infl);
    e.gram = h->gram;
    e.cvec = h->cvec;
    e.nloc = h->nloc;
    e.x = h->xg;
    e.pt0 = (long long)y0 * h->cfg.nx;
    e.npts = (y1 - y0) * h->cfg.nx;
    e.eigval = h->eigval;
    e.status = h->status;
    e.max_blocks = h->eig_blocks;
    e.refine = h->cfg.precision == LETKF_MIXED ? 1 : 0;  // FP64 sweep over clustered eigenpairs
    e.refine_tau = 1e-6f;
    e.work = work_counters(h);
    return e;
}

// The EVD-free schedules serve k <= 64; AUTO considers them there.  The Chebyshev schedule
// hands the points beyond its approximations to the rational one, which it therefore needs.
bool rational_candidate(int schedule, int k) {
    return (schedule == LETKF_EIG_RATIONAL || schedule == LETKF_EIG_CHEBYSHEV ||
            schedule == LETKF_EIG_AUTO) &&
           k <= lk::kRationalMaxK;
}
bool cheb_candidate(int schedule, int k) {
    return (schedule == LETKF_EIG_CHEBYSHEV || schedule == LETKF_EIG_AUTO) &&
           k <= lk::kChebMaxK;
}

// The chunk's eigensolve, transform and update on the handle's resolved schedule.
cudaError_t launch_eig_schedule(letkf_handle *h, int schedule, lk::EigArgs e, cudaStream_t s,
                                bool want_eigval) {
    if (schedule == LETKF_EIG_FUSED) {
        e.eigval = want_eigval ? h->eigval : nullptr;
        return lk::launch_eigen_update(e, s);
    }
    if (schedule == LETKF_EIG_RATIONAL) {
        e.eigval = want_eigval ? h->eigval : nullptr;
        return lk::launch_eigen_rational(e, h->eig_split, h->rat_grid, s);
    }
    if (schedule == LETKF_EIG_CHEBYSHEV) {
        e.eigval = want_eigval ? h->eigval : nullptr;
        return lk::launch_eigen_chebyshev(e, h->eig_split, h->cheb_grid, h->rat_grid, s);
    }
    e.eigval = h->eigval;
    return lk::launch_eigen_split(e, h->eig_split, s, h->stream2, h->split_fork, h->split_join);
}

// ---- AUTO eigensolve schedule ----------------------------------------------------------
// Both schedules are timed on the handle's first analysis, on the Gram matrices of its first
// chunk (at most 16384 points), just before that chunk's eigensolve: each runs the full
// eigensolve, transform and update, applied to a scratch copy of the chunk's forecast
// perturbations in the state buffer the next forecast overwrites.  The Gram matrices' upper
// triangles, c and the local counts are left intact by both, so the analysis proper then runs
// on unchanged inputs with the faster schedule.  The choice is cached per (device, k, batch)
// for the life of the process: later handles of that shape take it at letkf_init, so every
// handle of a process with the same k and chunk size runs the same arithmetic.

struct EigTuneCache {
    std::mutex mu;
    std::map<std::pair<int, std::pair<int, int>>, int> pick;
};

EigTuneCache &eig_tune_cache() {
    static EigTuneCache c;
    return c;
}

std::pair<int, std::pair<int, int>> eig_tune_key(const letkf_handle *h) {
    const int batch = (int)std::min<size_t>(h->plan.chunk_pts, 16384);
    return std::make_pair(h->device, std::make_pair(h->cfg.k, batch));
}

int cached_eig_schedule(const letkf_handle *h) {
    EigTuneCache &c = eig_tune_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    const auto it = c.pick.find(eig_tune_key(h));
    return it == c.pick.end() ? LETKF_EIG_AUTO : it->second;
}

int tune_eig_schedule(letkf_handle *h, int y0, int y1) {
    const int cached = cached_eig_schedule(h);
    if (cached != LETKF_EIG_AUTO) {
        h->eig_schedule = h->stats.eig_schedule = cached;
        return LETKF_OK;
    }
    const int k = h->cfg.k;
    lk::EigArgs e = eig_args(h, y0, y1);
    e.npts = std::min(e.npts, 16384);
    float *scratch = h->state[h->cur ^ 1];  // >= k * 9 * npts floats, free until the forecast
    const size_t xbytes = (size_t)e.npts * 9 * k * sizeof(float);
    CK(cudaMemcpyAsync(scratch, h->xg + (size_t)e.pt0 * 9 * k, xbytes,
                       cudaMemcpyDeviceToDevice, h->stream));
    e.x = scratch;
    e.pt0 = 0;
    int saved = 0;                          // status word: the timed runs must not latch
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(&saved, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    // for k <= 64 the Chebyshev schedule stands for both EVD-free schedules: it passes every
    // point beyond its break-even degree to the rational one, so it is never much slower than
    // that, and timing the two on the first analysis (whose spread may be far from the later
    // ones') would tie the process to a transient
    int cand[3] = {LETKF_EIG_FUSED, LETKF_EIG_SPLIT, 0};
    int ncand = 2;
    if (cheb_candidate(LETKF_EIG_AUTO, k)) cand[ncand++] = LETKF_EIG_CHEBYSHEV;
    float best[3] = {0.0f, 0.0f, 0.0f};
    cudaError_t err = cudaEventCreate(&t0);
    if (err == cudaSuccess) err = cudaEventCreate(&t1);
    for (int sch = 0; sch < ncand && err == cudaSuccess; ++sch) {
        for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
            err = cudaEventRecord(t0, h->stream);
            if (err == cudaSuccess) err = launch_eig_schedule(h, cand[sch], e, h->stream, false);
            if (err == cudaSuccess) err = cudaEventRecord(t1, h->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(t1);
            float ms = 0.0f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, t0, t1);
            if (rep > 0 && (rep == 1 || ms < best[sch])) best[sch] = ms;  // run 0 warms up
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(h->status, &saved, sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    if (err != cudaSuccess) return cuda_fail(h, err);
    int ib = 0;
    for (int sch = 1; sch < ncand; ++sch)
        if (best[sch] < best[ib]) ib = sch;
    const int pick = cand[ib];
    {
        EigTuneCache &c = eig_tune_cache();
        std::lock_guard<std::mutex> lock(c.mu);
        h->eig_schedule = c.pick.emplace(eig_tune_key(h), pick).first->second;  // first wins
    }
    h->stats.eig_schedule = h->eig_schedule;
    return LETKF_OK;
}

// ---- AUTO FP32 Gram tile schedule (k >= 17) ---------------------------------------------
// The first analysis times both tile schedules on its first chunk (each twice after a warm-up
// run, the better of the two) and keeps the faster; the kept schedule runs last, so the chunk's
// Gram matrices, c and local counts are its own.  The pick is cached for the process per
// problem shape (device, kp, grid, chunk, observation network size and localization), so that
// handles of one shape run the same arithmetic.

struct GramTuneCache {
    std::mutex mu;
    std::map<std::vector<long long>, int> pick;
};

GramTuneCache &gram_tune_cache() {
    static GramTuneCache c;
    return c;
}

std::vector<long long> gram_tune_key(const letkf_handle *h) {
    return {h->device,   h->plan.kp,   h->cfg.nx,    h->cfg.ny,      h->plan.chunk_rows,
            h->plan.V,   h->plan.d2max, h->cfg.n_obs, h->cfg.loc_kind};
}

int cached_gram_tile(const letkf_handle *h) {
    GramTuneCache &c = gram_tune_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    const auto it = c.pick.find(gram_tune_key(h));
    return it == c.pick.end() ? LETKF_GRAM_AUTO : it->second;
}

int tune_gram_tile(letkf_handle *h, int chunk, int y0, int y1) {
    const int cached = cached_gram_tile(h);
    if (cached != LETKF_GRAM_AUTO) {
        h->gram_tile = h->stats.gram_tile = cached;
        return enqueue_gram_chunk(h, chunk, y0, y1);
    }
    const int cand[2] = {LETKF_GRAM_TEAM, LETKF_GRAM_PIPE};   // the last one timed runs last
    float best[2] = {0.0f, 0.0f};
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t err = cudaEventCreate(&t0);
    if (err == cudaSuccess) err = cudaEventCreate(&t1);
    int rc = LETKF_OK;
    for (int rep = 0; rep < 3 && err == cudaSuccess && !rc; ++rep)
        for (int i = 0; i < 2 && err == cudaSuccess && !rc; ++i) {
            h->gram_tile = cand[i];
            err = cudaEventRecord(t0, h->stream);
            if (err == cudaSuccess) rc = enqueue_gram_chunk(h, chunk, y0, y1);
            if (err == cudaSuccess && !rc) err = cudaEventRecord(t1, h->stream);
            if (err == cudaSuccess && !rc) err = cudaEventSynchronize(t1);
            float ms = 0.0f;
            if (err == cudaSuccess && !rc) err = cudaEventElapsedTime(&ms, t0, t1);
            if (rep > 0 && (rep == 1 || ms < best[i])) best[i] = ms;   // run 0 warms up
        }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (rc) return rc;
    if (err != cudaSuccess) return cuda_fail(h, err);
    int pick = best[0] < best[1] ? cand[0] : cand[1];
    {
        GramTuneCache &c = gram_tune_cache();
        std::lock_guard<std::mutex> lock(c.mu);
        pick = c.pick.emplace(gram_tune_key(h), pick).first->second;  // the first pick wins
    }
    h->gram_tile = h->stats.gram_tile = pick;
    return pick == cand[1] ? LETKF_OK : enqueue_gram_chunk(h, chunk, y0, y1);
}

int enqueue_analysis(letkf_handle *h, letkf_probe *probe) {
    const Plan &p = h->plan;
    const letkf_config &c = h->cfg;
    const int k = c.k;
    int rc = mark(h, 2);
    if (!rc) rc = enqueue_obs(h);
    if (!rc) rc = mark(h, 3);
    if (rc) return rc;
    CK(lk::launch_transpose_in(h->state[h->cur], h->xg, k, p.npts, h->stream));
    if ((rc = mark(h, 4))) return rc;
    int chunk = 0;
    if (probe && probe->xf)
        for (int i = 0; i < probe->n_points; ++i)
            CK(cudaMemcpyAsync(probe->xf + (size_t)i * 9 * k,
                               h->xg + (size_t)probe->points[i] * 9 * k, 9 * k * sizeof(float),
                               cudaMemcpyDeviceToHost, h->stream));
    for (int y0 = 0; y0 < c.ny; y0 += p.chunk_rows) {
        const int y1 = std::min(c.ny, y0 + p.chunk_rows);
        rc = h->gram_tile == LETKF_GRAM_AUTO ? tune_gram_tile(h, chunk, y0, y1)
                                             : enqueue_gram_chunk(h, chunk, y0, y1);
        if (rc) return rc;
        if ((rc = mark(h, 5 + 2 * chunk))) return rc;
        const long long pt0 = (long long)y0 * c.nx;
        const int npts = (y1 - y0) * c.nx;
        if (probe) {
            for (int i = 0; i < probe->n_points; ++i) {
                const long long lp = probe->points[i] - pt0;
                if (lp < 0 || lp >= npts) continue;
                if (probe->nloc)
                    CK(cudaMemcpyAsync(probe->nloc + i, h->nloc + lp, sizeof(int),
                                       cudaMemcpyDeviceToHost, h->stream));
                if (probe->gram)
                    CK(cudaMemcpyAsync(probe->gram + (size_t)i * k * k, h->gram + lp * k * k,
                                       (size_t)k * k * sizeof(float), cudaMemcpyDeviceToHost,
                                       h->stream));
                if (probe->cvec)
                    CK(cudaMemcpyAsync(probe->cvec + (size_t)i * k, h->cvec + lp * k,
                                       (size_t)k * sizeof(float), cudaMemcpyDeviceToHost,
                                       h->stream));
            }
        }
        if (h->eig_schedule == LETKF_EIG_AUTO && (rc = tune_eig_schedule(h, y0, y1))) return rc;
        CK(launch_eig_schedule(h, h->eig_schedule, eig_args(h, y0, y1), h->stream,
                               probe && probe->eigval));
        if ((rc = mark(h, 6 + 2 * chunk))) return rc;
        ++chunk;
        if (probe && probe->eigval)
            for (int i = 0; i < probe->n_points; ++i) {
                const long long lp = probe->points[i] - pt0;
                if (lp < 0 || lp >= npts) continue;
                CK(cudaMemcpyAsync(probe->eigval + (size_t)i * k, h->eigval + lp * k,
                                   (size_t)k * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
            }
    }
    CK(lk::launch_transpose_out(h->xg, h->state[h->cur], k, p.npts, h->stream));
    if ((rc = mark(h, 5 + 2 * chunk))) return rc;
    if (h->timing) h->an_done = true;
    return LETKF_OK;
}

// ---- groups of handles -----------------------------------------------------------------

constexpr int kMaxGroup = 16;

// Resident grids of the grouped eigen kernels, per device, prepared once per process.
int group_blocks(int device, const int **out) {
    static std::mutex mu;
    static std::map<int, std::vector<int>> grids;
    std::lock_guard<std::mutex> lock(mu);
    auto it = grids.find(device);
    if (it == grids.end()) {
        std::vector<int> g(3, 0);
        if (lk::eigen_group_prepare(g.data()) != cudaSuccess) return LETKF_ECUDA;
        it = grids.emplace(device, g).first;
    }
    *out = it->second.data();
    return LETKF_OK;
}

int check_group(letkf_handle *const *hs, int n) {
    if (!hs || n < 1 || n > kMaxGroup) return LETKF_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || hs[i]->device != hs[0]->device) return LETKF_EINVAL;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return LETKF_EINVAL;
    }
    return LETKF_OK;
}

// While it lives, every handle of the group enqueues on the group stream S (the first
// handle's), with its phase timing switched off.
struct GroupScope {
    letkf_handle *const *hs;
    int n;
    cudaStream_t st[kMaxGroup];
    bool tm[kMaxGroup];
    GroupScope(letkf_handle *const *hs_, int n_) : hs(hs_), n(n_) {
        for (int i = 0; i < n; ++i) {
            st[i] = hs[i]->stream;
            tm[i] = hs[i]->timing;
            hs[i]->stream = hs[0]->stream;
            hs[i]->timing = false;
        }
    }
    ~GroupScope() {
        for (int i = 0; i < n; ++i) {
            hs[i]->stream = st[i];
            hs[i]->timing = tm[i];
        }
    }
};

// Orders the group stream after each handle's own stream (join = false), or each handle's
// stream after the group stream (join = true).
int group_fence(letkf_handle *const *hs, int n, bool join) {
    letkf_handle *h = hs[0];
    for (int i = 1; i < n; ++i) {
        if (hs[i]->stream == h->stream) continue;
        cudaEvent_t ev = nullptr;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        const cudaError_t e1 = cudaEventRecord(ev, join ? h->stream : hs[i]->stream);
        const cudaError_t e2 =
            e1 == cudaSuccess ? cudaStreamWaitEvent(join ? hs[i]->stream : h->stream, ev, 0) : e1;
        cudaEventDestroy(ev);
        CK(e2);
    }
    return LETKF_OK;
}

// The group's work (inside a GroupScope, whose stream S is the first handle's).  Every handle's
// own phases run on its own branch stream, forked from S: the forecast, the observation
// operator and transpose, per chunk round its Gram chunk and (SPLIT and RATIONAL schedules) its
// eigensolve, the transpose back.  The handles on the FUSED schedule join S after each round's
// Gram chunks for one grouped eigen launch per column class over all of them, and fork again
// after it.  All branches join S at the end, so the group's work is ordered on S (and inside a
// capture forms one graph with parallel branches).  A handle still on AUTO picks its schedule
// at its first Gram chunk (eager calls only: the callers do not capture while a handle has yet
// to pick).
int enqueue_group(letkf_handle *const *hs, int n, int nsteps) {
    letkf_handle *h = hs[0];
    const cudaStream_t S = h->stream;
    const int *blocks = nullptr;
    int rc = group_blocks(h->device, &blocks);
    if (rc) return rc;
    auto fork = [&](letkf_handle *g) -> int {   // g's branch after S's current work
        CK(cudaEventRecord(h->gfork, S));
        CK(cudaStreamWaitEvent(g->gstream, h->gfork, 0));
        return LETKF_OK;
    };
    auto join = [&](letkf_handle *g) -> int {   // S after g's branch
        CK(cudaEventRecord(g->gjoin, g->gstream));
        CK(cudaStreamWaitEvent(S, g->gjoin, 0));
        return LETKF_OK;
    };
    struct OnBranch {  // g enqueues on its branch while this lives
        letkf_handle *g;
        cudaStream_t s;
        explicit OnBranch(letkf_handle *g_) : g(g_), s(g_->stream) { g->stream = g->gstream; }
        ~OnBranch() { g->stream = s; }
    };
    for (int i = 0; i < n; ++i)
        if ((rc = fork(hs[i]))) return rc;
    int rounds = 0;
    for (int i = 0; i < n; ++i) {
        letkf_handle *g = hs[i];
        OnBranch b(g);
        if (nsteps >= 0 && (rc = enqueue_forecast(g, nsteps))) return rc;
        if ((rc = enqueue_obs(g))) return rc;
        const cudaError_t e = lk::launch_transpose_in(g->state[g->cur], g->xg, g->cfg.k,
                                                      g->plan.npts, g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e);
        rounds = std::max(rounds, (g->cfg.ny + g->plan.chunk_rows - 1) / g->plan.chunk_rows);
    }
    for (int r = 0; r < rounds; ++r) {
        lk::EigArgs segs[kMaxGroup];
        letkf_handle *fused[kMaxGroup];
        int m = 0;
        for (int i = 0; i < n; ++i) {
            letkf_handle *g = hs[i];
            const int y0 = r * g->plan.chunk_rows;
            if (y0 >= g->cfg.ny) continue;
            const int y1 = std::min(g->cfg.ny, y0 + g->plan.chunk_rows);
            OnBranch b(g);
            rc = g->gram_tile == LETKF_GRAM_AUTO ? tune_gram_tile(g, r, y0, y1)
                                                 : enqueue_gram_chunk(g, r, y0, y1);
            if (rc) return rc;
            if (g->eig_schedule == LETKF_EIG_AUTO && (rc = tune_eig_schedule(g, y0, y1)))
                return rc;
            if (g->eig_schedule == LETKF_EIG_FUSED) {
                segs[m] = eig_args(g, y0, y1);
                fused[m++] = g;
            } else {
                const cudaError_t e =
                    launch_eig_schedule(g, g->eig_schedule, eig_args(g, y0, y1), g->stream, false);
                if (e != cudaSuccess) return cuda_fail(g, e);
            }
        }
        if (m > 0) {
            for (int i = 0; i < m; ++i)
                if ((rc = join(fused[i]))) return rc;
            CK(lk::launch_eigen_group(segs, m, h->status + 16, blocks, S));
            for (int i = 0; i < m; ++i)
                if ((rc = fork(fused[i]))) return rc;
        }
    }
    for (int i = 0; i < n; ++i) {
        letkf_handle *g = hs[i];
        {
            OnBranch b(g);
            const cudaError_t e = lk::launch_transpose_out(g->xg, g->state[g->cur], g->cfg.k,
                                                           g->plan.npts, g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e);
        }
        if ((rc = join(g))) return rc;
    }
    return LETKF_OK;
}

int status_to_code(int bits) {
    if (bits & lk::ST_NONFINITE) return LETKF_ENONFINITE;
    if (bits & lk::ST_NOTCONV) return LETKF_ENOTCONV;
    if (bits & lk::ST_TIMEOUT) return LETKF_ETIMEOUT;
    if (bits & lk::ST_BADINDEX) return LETKF_EINVAL;
    return LETKF_OK;
}

void destroy_graphs(letkf_handle *h) {
    for (int i = 0; i < 2; ++i) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        h->graph[i] = nullptr;
        h->graph_nsteps[i] = -1;
    }
    for (auto &gg : h->group_graphs)
        if (gg.exec) cudaGraphExecDestroy(gg.exec);
    h->group_graphs.clear();
}

void destroy_events(letkf_handle *h) {
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
}

}  // namespace

extern "C" {

const char *letkf_strerror(int code) {
    switch (code) {
        case LETKF_OK: return "success";
        case LETKF_EINVAL: return "invalid argument";
        case LETKF_ENOMEM: return "out of device memory or workspace too small";
        case LETKF_ENOTCONV: return "eigensolver did not converge at some grid point";
        case LETKF_ENONFINITE: return "non-finite value in the analysis";
        case LETKF_ETIMEOUT: return "bounded device wait expired";
        case LETKF_ECUDA: return "CUDA runtime error";
        case LETKF_ESTATE: return "call not valid in the handle's current state";
        default: return "unknown status code";
    }
}

int letkf_workspace_size(const letkf_config *cfg, size_t *bytes) {
    if (!bytes) return LETKF_EINVAL;
    Plan p;
    const int rc = make_plan(cfg, &p);
    if (rc) return rc;
    *bytes = p.total;
    return LETKF_OK;
}

int letkf_init(const letkf_config *cfg, void *workspace, size_t workspace_bytes,
               letkf_handle **out) {
    if (!out) return LETKF_EINVAL;
    *out = nullptr;
    Plan plan;
    int rc = make_plan(cfg, &plan);
    if (rc) return rc;
    if (workspace && (workspace_bytes < plan.total || ((uintptr_t)workspace % kAlign)))
        return LETKF_ENOMEM;
    letkf_handle *h = new (std::nothrow) letkf_handle();
    if (!h) return LETKF_ENOMEM;
    h->cfg = *cfg;
    h->cfg.force = nullptr;
    h->cfg.obs_xy = nullptr;
    h->cfg.obs_err_var = nullptr;
    h->plan = plan;
    memset(&h->stats, 0, sizeof(h->stats));
    static std::atomic<unsigned long long> serials{0};
    h->serial = ++serials;
    auto fail = [&](int code) {
        letkf_destroy(h);
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(LETKF_ECUDA);
    if (cfg->stream) {
        h->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(LETKF_ECUDA);
        h->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&h->stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->split_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->split_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->gfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->gjoin, cudaEventDisableTiming) != cudaSuccess)
        return fail(LETKF_ECUDA);
    if (workspace) {
        h->ws = (unsigned char *)workspace;
    } else {
        void *w = nullptr;
        const cudaError_t e = cudaMalloc(&w, plan.total);
        if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? LETKF_ENOMEM : LETKF_ECUDA);
        h->ws = (unsigned char *)w;
        h->own_ws = true;
    }
    unsigned char *w = h->ws;
    h->state[0] = (float *)(w + plan.off_state[0]);
    h->state[1] = (float *)(w + plan.off_state[1]);
    h->force = cfg->force ? (float2 *)(w + plan.off_force) : nullptr;
    h->xg = (float *)(w + plan.off_xg);
    h->obs_xy = (int2 *)(w + plan.off_obs_xy);
    h->cell_start = (int *)(w + plan.off_cell_start);
    h->cell_obs = (int *)(w + plan.off_cell_obs);
    h->rinv = (float *)(w + plan.off_rinv);
    h->yf = (float *)(w + plan.off_yf);
    h->yb = (float *)(w + plan.off_yb);
    h->ybar = (float *)(w + plan.off_ybar);
    h->yo = (float *)(w + plan.off_yo);
    h->orec = plan.tensor_gram ? (float4 *)(w + plan.off_orec) : nullptr;
    h->gram = (float *)(w + plan.off_gram);
    h->cvec = (float *)(w + plan.off_cvec);
    h->nloc = (int *)(w + plan.off_nloc);
    h->nloc_all = (int *)(w + plan.off_nloc_all);
    h->eigval = (float *)(w + plan.off_eigval);
    if (plan.eig_schedule != LETKF_EIG_FUSED) {
        h->eig_split.de = (float2 *)(w + plan.off_de);
        h->eig_split.taus = (float *)(w + plan.off_taus);
        h->eig_split.rot = plan.rcap > 0 ? (float2 *)(w + plan.off_rot) : nullptr;
        h->eig_split.nrot = plan.rcap > 0 ? (int *)(w + plan.off_nrot) : nullptr;
        h->eig_split.list = (int *)(w + plan.off_list);
        h->eig_split.list_count = h->eig_split.list + plan.chunk_pts;
        if (cheb_candidate(plan.eig_schedule, cfg->k)) {
            h->eig_split.pre_list = (int *)(w + plan.off_pre_list);
            h->eig_split.pre_count = h->eig_split.pre_list + plan.chunk_pts;
        }
        h->eig_split.rcap = plan.rcap;
    }
    h->status = (int *)(w + plan.off_status);

    const size_t npts = plan.npts;
    // body force, interleaved per node
    if (cfg->force) {
        std::vector<float2> f(npts);
        for (size_t i = 0; i < npts; ++i) f[i] = make_float2(cfg->force[i], cfg->force[npts + i]);
        if (cudaMemcpy(h->force, f.data(), npts * sizeof(float2), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return fail(LETKF_ECUDA);
    }
    // observation network, bins (ascending observation index within each bin) and R^-1
    const int L = cfg->n_obs;
    std::vector<int2> xy(L);
    for (int l = 0; l < L; ++l) xy[l] = make_int2(cfg->obs_xy[2 * l], cfg->obs_xy[2 * l + 1]);
    const int ncell = plan.ncx * plan.ncy;
    std::vector<int> cstart(ncell + 1, 0), cobs(L);
    for (int l = 0; l < L; ++l) cstart[(xy[l].y / plan.cs) * plan.ncx + xy[l].x / plan.cs + 1]++;
    for (int c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    {
        std::vector<int> fill(cstart.begin(), cstart.end() - 1);
        for (int l = 0; l < L; ++l) cobs[fill[(xy[l].y / plan.cs) * plan.ncx + xy[l].x / plan.cs]++] = l;
    }
    std::vector<float> rinv(plan.LV);
    for (int s = 0; s < plan.LV; ++s) rinv[s] = (float)(1.0 / (double)cfg->obs_err_var[s]);
    if ((L && cudaMemcpy(h->obs_xy, xy.data(), L * sizeof(int2), cudaMemcpyHostToDevice)) ||
        cudaMemcpy(h->cell_start, cstart.data(), cstart.size() * sizeof(int),
                   cudaMemcpyHostToDevice) ||
        (L && cudaMemcpy(h->cell_obs, cobs.data(), L * sizeof(int), cudaMemcpyHostToDevice)) ||
        (plan.LV && cudaMemcpy(h->rinv, rinv.data(), plan.LV * sizeof(float),
                               cudaMemcpyHostToDevice)))
        return fail(LETKF_ECUDA);
    {
        int col = 0;
        for (int vid = 0; vid < 3; ++vid)
            if (cfg->obs_vars & (1 << vid)) h->yref[col++] = vid == 0 ? 1.0f : 0.0f;
    }
    h->net.xy = h->obs_xy;
    h->net.cell_start = h->cell_start;
    h->net.cell_obs = h->cell_obs;
    h->net.L = L;
    h->net.V = plan.V;
    h->net.cs = plan.cs;
    h->net.ncx = plan.ncx;
    h->net.ncy = plan.ncy;
    h->net.loc_none = cfg->loc_kind == LETKF_LOC_NONE;
    h->net.d2max = plan.d2max;
    h->net.cr = plan.cr;
    h->net.inv2r2 = plan.inv2r2;
    h->net.loc_gc = cfg->loc_kind == LETKF_LOC_GC;
    h->net.inv_c = plan.inv_c;

    if (lk::lbm_prepare() != cudaSuccess ||
        lk::lbm_tma_build(h->state[0], h->state[1], h->force, cfg->nx, cfg->ny, plan.nmem,
                          &h->lbm_tma) != cudaSuccess ||
        lk::gram_prepare(plan.kp) != cudaSuccess ||
        lk::eigen_prepare(cfg->k, &h->eig_blocks) != cudaSuccess ||
        (plan.eig_schedule != LETKF_EIG_FUSED &&
         lk::eigen_split_prepare(cfg->k, &h->eig_split) != cudaSuccess) ||
        (rational_candidate(plan.eig_schedule, cfg->k) &&
         lk::eigen_rational_prepare(cfg->k, &h->rat_grid) != cudaSuccess) ||
        (cheb_candidate(plan.eig_schedule, cfg->k) &&
         lk::eigen_cheb_prepare(cfg->k, &h->cheb_grid) != cudaSuccess))
        return fail(LETKF_ECUDA);
    if (plan.tensor_gram) {
        int sms = 0;
        if (lk::gram_tc_prepare(plan.kp) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
            return fail(LETKF_ECUDA);
        h->tc_ctas = sms;  // one CTA per SM: each holds all 512 tensor-memory columns
    }
    // rest state, clean status, zero Gram buffers
    if (cudaMemsetAsync(h->state[0], 0, (size_t)plan.nmem * 9 * npts * sizeof(float), h->stream) ||
        cudaMemsetAsync(h->status, 0, kAlign, h->stream) ||
        cudaMemsetAsync(h->yb, 0, (size_t)plan.LV * plan.kp * sizeof(float), h->stream))
        return fail(LETKF_ECUDA);
    h->cur = 0;
    // static local-observation counts
    if (lk::launch_count_local(h->net, cfg->nx, cfg->ny, h->nloc_all, h->stream) != cudaSuccess)
        return fail(LETKF_ECUDA);
    std::vector<int> nl(npts);
    if (cudaMemcpyAsync(nl.data(), h->nloc_all, npts * sizeof(int), cudaMemcpyDeviceToHost,
                        h->stream) ||
        cudaStreamSynchronize(h->stream))
        return fail(LETKF_ECUDA);
    long long sum = 0;
    int mx = 0, zeros = 0;
    for (size_t i = 0; i < npts; ++i) {
        sum += nl[i];
        mx = std::max(mx, nl[i]);
        zeros += nl[i] == 0;
    }
    h->stats.n_points = (int32_t)npts;
    h->stats.n_zero_obs = zeros;
    h->stats.max_local_obs = mx;
    h->stats.mean_local_obs = (double)sum / (double)npts;
    h->stats.n_chunks = n_chunks(h);
    // AUTO: the process' earlier pick for this shape, else timed at the first analysis
    h->eig_schedule =
        plan.eig_schedule == LETKF_EIG_AUTO ? cached_eig_schedule(h) : plan.eig_schedule;
    h->stats.eig_schedule = h->eig_schedule;
    // the Gram: tensor cores (mixed), the one team schedule (k <= 16), else as configured
    if (plan.tensor_gram)
        h->gram_tile = LETKF_GRAM_TENSOR;
    else if (plan.kp <= 16)
        h->gram_tile = LETKF_GRAM_TEAM;
    else
        h->gram_tile = cfg->gram_tile == LETKF_GRAM_AUTO ? cached_gram_tile(h) : cfg->gram_tile;
    h->stats.gram_tile = h->gram_tile;
    *out = h;
    return LETKF_OK;
}

int letkf_sync(letkf_handle *h) {
    if (!h) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    int bits = 0;
    CK(cudaMemcpy(&bits, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits) CK(cudaMemset(h->status, 0, sizeof(int)));
    int code = status_to_code(bits);
    if (!code && h->latched) code = h->latched;
    h->latched = 0;
    h->stats.status = code;
    return code;
}

int letkf_destroy(letkf_handle *h) {
    if (!h) return LETKF_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->device) cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->stream2) cudaStreamSynchronize(h->stream2);
    if (h->gstream) cudaStreamSynchronize(h->gstream);
    destroy_graphs(h);
    destroy_events(h);
    if (h->split_fork) cudaEventDestroy(h->split_fork);
    if (h->split_join) cudaEventDestroy(h->split_join);
    if (h->gfork) cudaEventDestroy(h->gfork);
    if (h->gjoin) cudaEventDestroy(h->gjoin);
    if (h->stream2) cudaStreamDestroy(h->stream2);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (dev >= 0 && dev != h->device) cudaSetDevice(dev);
    delete h;
    return LETKF_OK;
}

int letkf_get_work_counts(letkf_handle *h, int64_t *counts) {
    if (!h || !counts) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    unsigned long long c[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(c, work_counters(h), sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < 3; ++i) counts[i] = (int64_t)c[i];
    return LETKF_OK;
}

int letkf_get_stats(letkf_handle *h, letkf_stats *st) {
    if (!h || !st) return LETKF_EINVAL;
    *st = h->stats;
    return LETKF_OK;
}

int letkf_enable_timing(letkf_handle *h, int32_t on) {
    if (!h) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    destroy_graphs(h);  // graphs captured with (or without) event records are stale
    destroy_events(h);
    h->timing = false;
    h->fc_steps = -1;
    h->an_done = false;
    if (!on) return LETKF_OK;
    const int n = 2 + 4 + 2 * n_chunks(h);
    h->ev.resize(n, nullptr);
    for (int i = 0; i < n; ++i) CK(cudaEventCreate(&h->ev[i]));
    h->timing = true;
    return LETKF_OK;
}

int letkf_get_timings(letkf_handle *h, letkf_timings *t) {
    if (!h || !t) return LETKF_EINVAL;
    if (!h->timing || (h->fc_steps < 0 && !h->an_done)) return LETKF_ESTATE;
    int rc = device_check(h);
    if (rc) return rc;
    memset(t, 0, sizeof(*t));
    const int nc = n_chunks(h);
    t->n_chunks = nc;
    auto el = [&](int a, int b, float *out) -> int {
        CK(cudaEventSynchronize(h->ev[b]));
        CK(cudaEventElapsedTime(out, h->ev[a], h->ev[b]));
        return LETKF_OK;
    };
    if (h->fc_steps >= 0) {
        t->forecast_steps = h->fc_steps;
        if ((rc = el(0, 1, &t->forecast_ms))) return rc;
    }
    if (h->an_done) {
        if ((rc = el(2, 3, &t->obs_ms)) || (rc = el(3, 4, &t->transpose_in_ms))) return rc;
        for (int c = 0; c < nc; ++c) {
            float a = 0.0f, b = 0.0f;
            if ((rc = el(4 + 2 * c, 5 + 2 * c, &a)) || (rc = el(5 + 2 * c, 6 + 2 * c, &b))) return rc;
            t->gram_ms += a;
            t->eigen_ms += b;
        }
        if ((rc = el(4 + 2 * nc, 5 + 2 * nc, &t->transpose_out_ms))) return rc;
    }
    return LETKF_OK;
}

int letkf_set_state(letkf_handle *h, const float *f, int32_t m0, int32_t count, int32_t where) {
    if (!h || !f || m0 < 0 || count < 0 || m0 + count > h->plan.nmem) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    const size_t n = (size_t)count * 9 * h->plan.npts;
    float *dst = h->state[h->cur] + (size_t)m0 * 9 * h->plan.npts;
    rc = copy_in(h, dst, f, n * sizeof(float), where);
    if (rc) return rc;
    CK(lk::launch_f_to_g(dst, dst, count, h->plan.npts, h->stream));
    if (where == LETKF_HOST) CK(cudaStreamSynchronize(h->stream));
    return LETKF_OK;
}

int letkf_get_state(letkf_handle *h, float *f, int32_t m0, int32_t count, int32_t where) {
    if (!h || !f || m0 < 0 || count < 0 || m0 + count > h->plan.nmem) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    const size_t n = (size_t)count * 9 * h->plan.npts;
    const size_t off = (size_t)m0 * 9 * h->plan.npts;
    float *scratch = h->state[h->cur ^ 1] + off;  // the idle ping-pong buffer
    CK(lk::launch_g_to_f(h->state[h->cur] + off, scratch, count, h->plan.npts, h->stream));
    return copy_out(h, f, scratch, n * sizeof(float), where);
}

int letkf_set_deviation(letkf_handle *h, const float *g, int32_t m0, int32_t count,
                        int32_t where) {
    if (!h || !g || m0 < 0 || count < 0 || m0 + count > h->plan.nmem) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    const size_t n = (size_t)count * 9 * h->plan.npts;
    rc = copy_in(h, h->state[h->cur] + (size_t)m0 * 9 * h->plan.npts, g, n * sizeof(float), where);
    if (rc) return rc;
    if (where == LETKF_HOST) CK(cudaStreamSynchronize(h->stream));
    return LETKF_OK;
}

int letkf_get_deviation(letkf_handle *h, float *g, int32_t m0, int32_t count, int32_t where) {
    if (!h || !g || m0 < 0 || count < 0 || m0 + count > h->plan.nmem) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    const size_t n = (size_t)count * 9 * h->plan.npts;
    return copy_out(h, g, h->state[h->cur] + (size_t)m0 * 9 * h->plan.npts, n * sizeof(float),
                    where);
}

int letkf_set_macro(letkf_handle *h, const float *rho, const float *ux, const float *uy,
                    int32_t m0, int32_t count, int32_t where) {
    if (!h || !rho || !ux || !uy || m0 < 0 || count < 0 || m0 + count > h->plan.nmem)
        return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    const size_t npts = h->plan.npts;
    const size_t n = (size_t)count * npts;
    const float *dr = rho, *du = ux, *dv = uy;
    if (where == LETKF_HOST) {  // stage through the idle state buffer (9 x larger than needed)
        float *s = h->state[h->cur ^ 1];
        if ((rc = copy_in(h, s, rho, n * sizeof(float), where)) ||
            (rc = copy_in(h, s + n, ux, n * sizeof(float), where)) ||
            (rc = copy_in(h, s + 2 * n, uy, n * sizeof(float), where)))
            return rc;
        dr = s;
        du = s + n;
        dv = s + 2 * n;
    } else if (where != LETKF_DEVICE) {
        return LETKF_EINVAL;
    }
    CK(lk::launch_macro_to_g(dr, du, dv, h->state[h->cur] + (size_t)m0 * 9 * npts, count, npts,
                             h->stream));
    if (where == LETKF_HOST) CK(cudaStreamSynchronize(h->stream));
    return LETKF_OK;
}

int lbm_forecast(letkf_handle *h, int32_t nsteps) {
    if (!h || nsteps < 0) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    return enqueue_forecast(h, nsteps);
}

int letkf_get_obs(letkf_handle *h, float *yf, int32_t where) {
    if (!h || !yf) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    if ((rc = enqueue_obs(h))) return rc;
    return copy_out(h, yf, h->yf, (size_t)h->plan.nmem * h->plan.LV * sizeof(float), where);
}

int letkf_analyze_probe(letkf_handle *h, const float *yo, int32_t where, letkf_probe *probe) {
    if (!h || (h->plan.LV > 0 && !yo)) return LETKF_EINVAL;
    if (probe) {
        if (probe->n_points < 0 || (probe->n_points > 0 && !probe->points)) return LETKF_EINVAL;
        for (int i = 0; i < probe->n_points; ++i)
            if (probe->points[i] < 0 || (size_t)probe->points[i] >= h->plan.npts)
                return LETKF_EINVAL;
    }
    int rc = device_check(h);
    if (rc) return rc;
    if ((rc = copy_in(h, h->yo, yo, (size_t)h->plan.LV * sizeof(float), where))) return rc;
    if ((rc = enqueue_analysis(h, probe))) return rc;
    if (probe) CK(cudaStreamSynchronize(h->stream));
    if (probe && probe->gram) {  // the Gram kernels form the upper triangle: mirror it
        const int k = h->cfg.k;
        for (int i = 0; i < probe->n_points; ++i) {
            float *A = probe->gram + (size_t)i * k * k;
            for (int r = 0; r < k; ++r)
                for (int c = r + 1; c < k; ++c) A[c * k + r] = A[r * k + c];
        }
    }
    if (probe && probe->eigval)  // ascending order per point
        for (int i = 0; i < probe->n_points; ++i)
            std::sort(probe->eigval + (size_t)i * h->cfg.k, probe->eigval + (size_t)(i + 1) * h->cfg.k);
    return LETKF_OK;
}

int letkf_analyze(letkf_handle *h, const float *yo, int32_t where) {
    return letkf_analyze_probe(h, yo, where, nullptr);
}

int letkf_cycle(letkf_handle *h, int32_t nsteps, const float *yo, int32_t where) {
    if (!h || nsteps < 0 || (h->plan.LV > 0 && !yo)) return LETKF_EINVAL;
    int rc = device_check(h);
    if (rc) return rc;
    if ((rc = copy_in(h, h->yo, yo, (size_t)h->plan.LV * sizeof(float), where))) return rc;
    if (h->eig_schedule == LETKF_EIG_AUTO || h->gram_tile == LETKF_GRAM_AUTO) {
        // the first analysis times the schedules: eager
        rc = enqueue_forecast(h, nsteps);
        return rc ? rc : enqueue_analysis(h, nullptr);
    }
    const int slot = h->cur;
    if (h->graph_nsteps[slot] != nsteps) {
        if (h->graph[slot]) {
            cudaGraphExecDestroy(h->graph[slot]);
            h->graph[slot] = nullptr;
        }
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
        const int cur0 = h->cur;
        rc = enqueue_forecast(h, nsteps);
        if (!rc) rc = enqueue_analysis(h, nullptr);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
        h->cur = cur0;
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(h, ec);
        h->graph_kernels[slot] = graph_kernel_nodes(g);
        const cudaError_t ei = cudaGraphInstantiate(&h->graph[slot], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return cuda_fail(h, ei);
        h->graph_nsteps[slot] = nsteps;
    }
    CK(cudaGraphLaunch(h->graph[slot], h->stream));
    h->stats.cycle_kernels = h->graph_kernels[slot];
    h->cur ^= (forecast_flips(nsteps) & 1);
    return LETKF_OK;
}

int letkf_group_analyze(letkf_handle *const *hs, const float *const *yo, int32_t n,
                        int32_t where) {
    int rc = check_group(hs, n);
    if (rc) return rc;
    if (where != LETKF_HOST && where != LETKF_DEVICE) return LETKF_EINVAL;
    for (int i = 0; i < n; ++i)
        if (hs[i]->plan.LV > 0 && (!yo || !yo[i])) return LETKF_EINVAL;
    letkf_handle *h = hs[0];
    if ((rc = device_check(h))) return rc;
    if ((rc = group_fence(hs, n, false))) return rc;
    {
        GroupScope scope(hs, n);
        for (int i = 0; i < n && !rc; ++i)
            rc = copy_in(hs[i], hs[i]->yo, yo[i], (size_t)hs[i]->plan.LV * sizeof(float), where);
        if (!rc) rc = enqueue_group(hs, n, -1);
    }
    if (rc) return rc;
    return group_fence(hs, n, true);
}

int letkf_group_cycle(letkf_handle *const *hs, int32_t n, int32_t nsteps, const float *const *yo,
                      int32_t where) {
    int rc = check_group(hs, n);
    if (rc) return rc;
    if (nsteps < 0 || (where != LETKF_HOST && where != LETKF_DEVICE)) return LETKF_EINVAL;
    for (int i = 0; i < n; ++i)
        if (hs[i]->plan.LV > 0 && (!yo || !yo[i])) return LETKF_EINVAL;
    letkf_handle *h = hs[0];
    if ((rc = device_check(h))) return rc;
    if ((rc = group_fence(hs, n, false))) return rc;
    {
        GroupScope scope(hs, n);
        for (int i = 0; i < n && !rc; ++i)
            rc = copy_in(hs[i], hs[i]->yo, yo[i], (size_t)hs[i]->plan.LV * sizeof(float), where);
        if (rc) return rc;
        bool pending = false;  // a handle still picks a schedule: no capture
        for (int i = 0; i < n; ++i)
            pending |= hs[i]->eig_schedule == LETKF_EIG_AUTO ||
                       hs[i]->gram_tile == LETKF_GRAM_AUTO;
        if (pending) {
            if ((rc = enqueue_group(hs, n, nsteps))) return rc;
            h->stats.cycle_kernels = 0;
            return group_fence(hs, n, true);
        }
        // the captured graph of this membership, schedules, state buffers and step count
        std::vector<unsigned long long> ids(n);
        std::vector<int> cur(n), sched(n);
        for (int i = 0; i < n; ++i) {
            ids[i] = hs[i]->serial;
            cur[i] = hs[i]->cur;
            sched[i] = hs[i]->eig_schedule;
        }
        letkf_handle::GroupGraph *gg = nullptr;
        for (auto &e : h->group_graphs)
            if (e.members == ids && e.cur == cur && e.sched == sched && e.nsteps == nsteps)
                gg = &e;
        if (!gg) {
            if (h->group_graphs.size() >= 8) {  // bounded cache: drop the oldest
                if (h->group_graphs.front().exec) cudaGraphExecDestroy(h->group_graphs.front().exec);
                h->group_graphs.erase(h->group_graphs.begin());
            }
            CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
            rc = enqueue_group(hs, n, nsteps);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
            for (int i = 0; i < n; ++i) hs[i]->cur = cur[i];
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ec != cudaSuccess) return cuda_fail(h, ec);
            letkf_handle::GroupGraph e;
            e.members = ids;
            e.cur = cur;
            e.sched = sched;
            e.nsteps = nsteps;
            e.kernels = graph_kernel_nodes(g);
            const cudaError_t ei = cudaGraphInstantiate(&e.exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) return cuda_fail(h, ei);
            h->group_graphs.push_back(e);
            gg = &h->group_graphs.back();
        }
        CK(cudaGraphLaunch(gg->exec, h->stream));
        h->stats.cycle_kernels = gg->kernels;
        for (int i = 0; i < n; ++i) hs[i]->cur ^= (forecast_flips(nsteps) & 1);
    }
    return group_fence(hs, n, true);
}

}  // extern "C"
