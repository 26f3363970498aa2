// EVD-free transform and update (the LETKF_EIG_RATIONAL schedule, FP32).
//
// The transform of each grid point needs two matrix functions of Q = (k-1)/rho I + A, not its
// eigenvectors (Sec. II-B, Eqs. letkf_wa, letkf_dwa, letkf_xa):
//     mean increment   dX wbar = dX Q^-1 c
//     perturbations    dX dW   = sqrt(k-1) dX Q^-1/2
// With the Householder tridiagonalization Q = H T H^T of the split schedule's first kernel
// (H = H_0 H_1 ... H_{k-3}, T symmetric tridiagonal), and B = [dX; c^T] (10 x k):
//     Y = B H                                   (the reflectors applied from the right)
//     dX Q^-1 c      = Y_{0..8} T^-1 Y_9^T      (one tridiagonal solve)
//     dX Q^-1/2      = (Y_{0..8} T^-1/2) H^T
// and T^-1/2 = b^-1/2 (T/b)^-1/2 ~ b^-1/2 sum_l beta_l b (T + p_l b I)^-1 by Zolotarev's best
// rational approximation of t^-1/2 on [1/kappa, 1] (zolotarev.cu), b >= lambda_max(T) the
// Gershgorin bound and kappa >= b / lambda_min from the exact floor lambda_min >= (k-1)/rho.
// Each shifted matrix T + sigma I is symmetric positive definite and is factored as L D L^T
// without pivoting.  The paper notes the eigensolve as half of the LETKF time and leaves
// EVD-free methods as future work (Sec. III); this schedule computes the same W applied to the
// same forecast, up to rounding and the approximation's relative error (~1e-8).
//
// Layout: one warp serves three grid points; lane 10 g + r holds row r of point g (rows 0..8:
// the populations' perturbations, row 9: c), all k entries in registers, so every reflector
// costs one 16-byte broadcast load and four multiply-adds per 4-row group (an unrolled chain
// entered through a jump table at the reflector's first row).  The factorizations of the
// shifted matrices (l_i, 1/d_i) are computed once per point and pole by one lane each and
// shared through shared memory; every row lane then solves its own right-hand side.  A point
// whose condition bound exceeds the largest approximation's range is handed to the fused
// schedule's kernel over the hand-off list (which recomputes it from A, left intact).
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace lk {
namespace {

constexpr unsigned kAll = 0xffffffffu;
constexpr int kPts = 3;       // grid points per warp
constexpr int kTasks = 10;    // factorizations per batch: one per lane of a point
constexpr int kWarpsR = 4;    // warps per block

template <int KM>
struct RatShape {
    static constexpr int VS = KM + 4;                 // one staged reflector (16-byte multiple)
    static constexpr int US = KM + 4;                 // the mean solve's result of one point
    static constexpr int DS = 2 * KM + 2;             // (d, e) of one point (bank offset 2)
    static constexpr int TS = 2 * kTasks * KM + 2;    // (l, 1/d) of 10 factorizations
    static constexpr int off_v = 0;                   // [2][kPts][VS]
    static constexpr int off_q = off_v + 2 * kPts * VS;   // [KM][32] lane-private
    static constexpr int off_u = off_q + 32 * KM;         // [kPts][US]
    static constexpr int off_tau = off_u + kPts * US;     // [kPts][KM]
    static constexpr int off_de = off_tau + kPts * KM;    // [kPts][DS]
    static constexpr int off_tab = off_de + kPts * DS;    // [kPts][TS]
    static constexpr int floats = (off_tab + kPts * TS + 3) & ~3;
};

__device__ __forceinline__ const float *refl(const float *Ag, int k, int j) {
    return Ag + (size_t)(k - 1 - j) * k;   // reflector j: row k-1-j of the Gram slot
}

// ---- one reflector on a row held in registers: y <- y - tau (y . v) v over rows >= 4 G0
template <int KM, int G>
__device__ __forceinline__ void rdot(const float (&y)[KM], const float4 *v4, float (&s)[4]) {
    if constexpr (4 * G < KM) {
        const float4 v = v4[G];
        s[0] = fmaf(v.x, y[4 * G], s[0]);
        s[1] = fmaf(v.y, y[4 * G + 1], s[1]);
        s[2] = fmaf(v.z, y[4 * G + 2], s[2]);
        s[3] = fmaf(v.w, y[4 * G + 3], s[3]);
    }
}
template <int KM, int G>
__device__ __forceinline__ void raxpy(float (&y)[KM], const float4 *v4, float beta) {
    if constexpr (4 * G < KM) {
        const float4 v = v4[G];
        y[4 * G] = fmaf(-beta, v.x, y[4 * G]);
        y[4 * G + 1] = fmaf(-beta, v.y, y[4 * G + 1]);
        y[4 * G + 2] = fmaf(-beta, v.z, y[4 * G + 2]);
        y[4 * G + 3] = fmaf(-beta, v.w, y[4 * G + 3]);
    }
}

#define LKR_G8(M, b) M(b) M(b + 1) M(b + 2) M(b + 3) M(b + 4) M(b + 5) M(b + 6) M(b + 7)
#define LKR_GROUPS16(M) LKR_G8(M, 0) LKR_G8(M, 8)

template <int KM>
__device__ __forceinline__ void apply_reflector(float (&y)[KM], const float4 *v4, float tau,
                                                int g0) {
    static_assert(KM / 4 <= 16, "the chains cover 64 rows");
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    switch (g0) {
#define LKR_DOT(G) \
    case G: rdot<KM, G>(y, v4, s);
        LKR_GROUPS16(LKR_DOT)
#undef LKR_DOT
        default: break;
    }
    const float beta = tau * ((s[0] + s[1]) + (s[2] + s[3]));
    switch (g0) {
#define LKR_AXPY(G) \
    case G: raxpy<KM, G>(y, v4, beta);
        LKR_GROUPS16(LKR_AXPY)
#undef LKR_AXPY
        default: break;
    }
}

// Lane r of a point stages entries r + 10 u of reflector j (m = k-1-j entries) into rows
// j + 1 + r + 10 u of the staging slot, and lanes r < 3 zero the rows 4 G0 .. j below them
// in the 4-row group G0 of row j + 1 (rows at and beyond k stay zero from the start).
constexpr int kStage = 7;  // ceil(64 / 10) entries per lane

__device__ __forceinline__ void fetch_reflector(const float *Ag, int k, int j, int r, bool act,
                                                float (&pf)[kStage]) {
    const int n = act ? k - 1 - j - r : 0;   // entries r, r + 10, .. below m
    const float *v = refl(Ag, k, j) + r;
#pragma unroll
    for (int u = 0; u < kStage; ++u) pf[u] = 10 * u < n ? __ldcg(v + 10 * u) : 0.0f;
}

__device__ __forceinline__ void stage_reflector(float *vb, int k, int j, int r, bool lane_ok,
                                                const float (&pf)[kStage]) {
    if (!lane_ok) return;
    const int n = k - 1 - j - r;
    float *dst = vb + j + 1 + r;
#pragma unroll
    for (int u = 0; u < kStage; ++u)
        if (10 * u < n) dst[10 * u] = pf[u];
    const int pad = 4 * ((j + 1) >> 2) + r;   // rows of the first group below row j + 1
    if (r < 3 && pad <= j) vb[pad] = 0.0f;
}

// y <- y H (forward: H_0 first) or y <- y H^T (reverse: H_{k-3} first), every row of the warp's
// three points at once; reflectors streamed through a double buffer, the next one's loads in
// flight while the current one is applied.
template <int KM>
__device__ __forceinline__ void apply_h(float (&y)[KM], const float *Ag, const float *tau_s,
                                        float *vbuf, int k, int pg, int r, bool act,
                                        bool reverse) {
    constexpr int VS = RatShape<KM>::VS;
    const bool lane_ok = pg < kPts;
    const int nrefl = k - 2;
    if (nrefl <= 0) return;
    float pf[kStage];
    int j = reverse ? k - 3 : 0;
    fetch_reflector(Ag, k, j, r, act, pf);
    float *vb0 = vbuf + (lane_ok ? pg : 0) * VS;
    for (int it = 0; it < nrefl; ++it) {
        float *vb = vb0 + (it & 1) * kPts * VS;
        stage_reflector(vb, k, j, r, lane_ok, pf);
        const int jn = reverse ? j - 1 : j + 1;
        if (it + 1 < nrefl) fetch_reflector(Ag, k, jn, r, act, pf);
        __syncwarp();
        const float tau = act ? tau_s[j] : 0.0f;
        apply_reflector<KM>(y, reinterpret_cast<const float4 *>(vb), tau, (j + 1) >> 2);
        j = jn;
    }
    __syncwarp();
}

// Row load (k floats, 16-byte loads when k is a multiple of 4) into y[0..KM), zero beyond k.
template <int KM>
__device__ __forceinline__ void load_row(const float *src, int k, float (&y)[KM]) {
    if ((k & 3) == 0) {
#pragma unroll
        for (int g = 0; g < KM / 4; ++g) {
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (4 * g < k) v = __ldcg(reinterpret_cast<const float4 *>(src) + g);
            y[4 * g] = v.x;
            y[4 * g + 1] = v.y;
            y[4 * g + 2] = v.z;
            y[4 * g + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < KM; ++i) y[i] = i < k ? __ldcg(src + i) : 0.0f;
    }
}

template <int KM>
__device__ __forceinline__ void store_row(float *dst, int k, const float (&y)[KM]) {
    if ((k & 3) == 0) {
#pragma unroll
        for (int g = 0; g < KM / 4; ++g)
            if (4 * g < k)
                reinterpret_cast<float4 *>(dst)[g] =
                    make_float4(y[4 * g], y[4 * g + 1], y[4 * g + 2], y[4 * g + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < KM; ++i)
            if (i < k) dst[i] = y[i];
    }
}

// L D L^T factorization of T + sigma I: tab[i] = (l_i, 1/d_i) with d_0 = d_0 + sigma,
// l_i = e_i / d_i, d_{i+1} = d_{i+1} + sigma - l_i e_i.
__device__ __forceinline__ void factor(const float2 *de, int k, float sigma, float2 *tab) {
    float lp = 0.0f, ep = 0.0f;
    for (int i = 0; i < k; ++i) {
        const float2 d = de[i];
        const float dp = fmaf(-lp, ep, d.x + sigma);
        const float dinv = __frcp_rn(dp);
        const float l = d.y * dinv;
        tab[i] = make_float2(l, dinv);
        lp = l;
        ep = d.y;
    }
}

template <int KM>
__global__ void __launch_bounds__(32 * kWarpsR) eig_rational_kernel(EigArgs a, EigSplit sp,
                                                                    ZoloTable zt) {
    using S = RatShape<KM>;
    extern __shared__ float smem_r[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int pg = lane / 10, r = lane - 10 * (lane / 10);   // pg == 3: lanes 30, 31 idle
    float *ws = smem_r + (size_t)wib * S::floats;
    float *vbuf = ws + S::off_v;
    float *qs = ws + S::off_q;
    const int pgc = pg < kPts ? pg : 0;
    float *ub = ws + S::off_u + pgc * S::US;
    float *tau_s = ws + S::off_tau + pgc * KM;
    float2 *de_s = reinterpret_cast<float2 *>(ws + S::off_de + pgc * S::DS);
    float2 *tab = reinterpret_cast<float2 *>(ws + S::off_tab + pgc * S::TS);
    const int k = a.k;
    const float sk1 = sqrtf((float)(k - 1));
    // staging slots: rows at and beyond k (and every row before its first use) hold zeros
    for (int i = lane; i < 2 * kPts * S::VS; i += 32) vbuf[i] = 0.0f;
    __syncwarp();
    const long long npts = a.list ? *a.list_count : a.npts;   // the chunk, or the listed points
    const long long ntask = (npts + kPts - 1) / kPts;
    const long long nw = (long long)gridDim.x * kWarpsR;
    for (long long task = (long long)blockIdx.x * kWarpsR + wib; task < ntask; task += nw) {
        const long long it = task * kPts + pg;
        const bool valid = pg < kPts && it < npts;
        const long long lp = valid ? (a.list ? a.list[it] : it) : 0;
        const bool observed = valid && (!a.nloc || a.nloc[lp] != 0);
        float *X = valid ? a.x + (size_t)(a.pt0 + lp) * NV * k : nullptr;
        // ---- rows: perturbations of the nine populations, and c
        float y[KM], acc[KM];
        float xb = 0.0f;
        if (valid && (r < NV ? true : observed)) {
            load_row<KM>(r < NV ? X + r * k : a.cvec + (size_t)lp * k, k, y);
            if (r < NV) {
                float s = 0.0f;
#pragma unroll
                for (int i = 0; i < KM; ++i) s += y[i];
                xb = s / (float)k;
#pragma unroll
                for (int i = 0; i < KM; ++i) y[i] = i < k ? y[i] - xb : 0.0f;
            }
        } else {
#pragma unroll
            for (int i = 0; i < KM; ++i) y[i] = 0.0f;
        }
        // a point without local observations: Q = (k-1)/rho I, wbar = 0, dW = sqrt(rho) I
        if (valid && !observed && r < NV && a.sqrt_infl != 1.0f) {
#pragma unroll
            for (int i = 0; i < KM; ++i) acc[i] = fmaf(a.sqrt_infl, y[i], xb);
            store_row<KM>(X + r * k, k, acc);
        }
        // ---- T of the point, its scale b and condition bound, the approximation to use
        if (observed) {
            for (int i = r; i < k; i += 10) {
                de_s[i] = sp.de[(size_t)lp * k + i];
                tau_s[i] = sp.taus[(size_t)lp * k + i];
            }
        }
        __syncwarp();
        float gmax = 0.0f;
        if (observed)
            for (int i = r; i < k; i += 10) {
                const float2 d = de_s[i];
                const float el = i > 0 ? fabsf(de_s[i - 1].y) : 0.0f;
                const float er = i < k - 1 ? fabsf(d.y) : 0.0f;
                gmax = fmaxf(gmax, d.x + el + er);
            }
        float b = 0.0f;
#pragma unroll
        for (int t = 0; t < 10; ++t) b = fmaxf(b, __shfl_sync(kAll, gmax, 10 * pgc + t));
        // lambda_min >= (k-1)/rho exactly; allow the FP32 tridiagonalization's rounding
        const float lo = a.diag - 1e-5f * b;
        int set = -1;
        if (observed) {
            const float kap = lo > 0.0f ? b / lo : FLT_MAX;
            for (int s = kZoloSets - 1; s >= 0; --s)
                if (kap <= zt.kappa_max[s]) set = s;
            if (set < 0 && r == 0)   // beyond every approximation: the fused kernel solves it
                sp.list[atomicAdd(sp.list_count, 1)] = (int)lp + sp.list_offset;
        }
        const bool act = observed && set >= 0 && isfinite(b) && b > 0.0f;
        const int wset = __reduce_max_sync(kAll, act ? set : -1);
        if (wset < 0) continue;   // nothing to transform in this warp
        const int npole = zt.n[wset];
        // ---- Y = B H
        apply_h<KM>(y, act ? a.gram + (size_t)lp * k * k : a.gram, tau_s, vbuf, k, pgc, r, act,
                    false);
        // ---- factorizations, mean solve, pole solves (batches of 10 tasks: task 0 is the
        // mean's T^-1, task t >= 1 pole t of the set)
        float incr = 0.0f;
#pragma unroll
        for (int i = 0; i < KM; ++i) acc[i] = 0.0f;
        for (int t0 = 0; t0 <= npole; t0 += kTasks) {
            const int t = t0 + r;
            if (act && pg < kPts && t <= npole) {
                const float sigma = t == 0 ? 0.0f : zt.pole[wset][t - 1] * b;
                factor(de_s, k, sigma, tab + (size_t)r * KM);
            }
            __syncwarp();
            if (t0 == 0) {
                // mean: lane 9 solves T u = Y_9 (its own row), then every row takes Y_r . u
                if (act && r == NV) {
                    float z = 0.0f, lpv = 0.0f;
#pragma unroll
                    for (int i = 0; i < KM; ++i)
                        if (i < k) {
                            const float2 f = tab[i];
                            z = fmaf(-lpv, z, y[i]);
                            acc[i] = z * f.y;
                            lpv = f.x;
                        }
                    float x = 0.0f;
#pragma unroll
                    for (int i = KM - 1; i >= 0; --i)
                        if (i < k) {
                            x = fmaf(-tab[i].x, x, acc[i]);
                            ub[i] = x;
                        }
#pragma unroll
                    for (int i = 0; i < KM; ++i) acc[i] = 0.0f;
                }
                __syncwarp();
                if (act && r < NV) {
                    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                    for (int i = 0; i < KM; i += 2) {
                        if (i < k) s0 = fmaf(y[i], ub[i], s0);
                        if (i + 1 < k) s1 = fmaf(y[i + 1], ub[i + 1], s1);
                    }
                    incr = s0 + s1;
                }
            }
            // poles of this batch, every row lane its own right-hand side
            const int tend = min(t0 + kTasks - 1, npole);
            for (int tp = t0 == 0 ? 1 : t0; tp <= tend; ++tp) {
                if (act && r < NV) {
                    const float2 *tb = tab + (size_t)(tp - t0) * KM;
                    const float w = zt.res[wset][tp - 1] * b;
                    float z = 0.0f, lpv = 0.0f;
#pragma unroll
                    for (int i = 0; i < KM; ++i)
                        if (i < k) {
                            const float2 f = tb[i];
                            z = fmaf(-lpv, z, y[i]);
                            qs[i * 32 + lane] = z * f.y;
                            lpv = f.x;
                        }
                    float x = 0.0f;
#pragma unroll
                    for (int i = KM - 1; i >= 0; --i)
                        if (i < k) {
                            x = fmaf(-tb[i].x, x, qs[i * 32 + lane]);
                            acc[i] = fmaf(w, x, acc[i]);
                        }
                }
            }
            __syncwarp();
        }
        // ---- perturbations P = sqrt(k-1) b^-1/2 acc, then F = P H^T
        const float sc = act ? sk1 * rsqrtf(b) : 0.0f;
#pragma unroll
        for (int i = 0; i < KM; ++i) acc[i] *= sc;
        apply_h<KM>(acc, act ? a.gram + (size_t)lp * k * k : a.gram, tau_s, vbuf, k, pgc, r, act,
                    true);
        // ---- X^a = xbar + increment + perturbation
        bool bad = false;
        if (act && r < NV) {
            const float base = xb + incr;
#pragma unroll
            for (int i = 0; i < KM; ++i) {
                acc[i] = base + acc[i];
                bad |= i < k && !isfinite(acc[i]);
            }
            store_row<KM>(X + r * k, k, acc);
        }
        if (__any_sync(kAll, bad) && lane == 0) atomicOr(a.status, ST_NONFINITE);
        __syncwarp();
    }
}

#undef LKR_GROUPS16
#undef LKR_G8

template <int KM>
cudaError_t prepare_km(int *grid) {
    using S = RatShape<KM>;
    const size_t smem = (size_t)S::floats * sizeof(float) * kWarpsR;
    cudaError_t e = cudaFuncSetAttribute(eig_rational_kernel<KM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eig_rational_kernel<KM>,
                                                      32 * kWarpsR, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = sms * per_sm;
    return cudaSuccess;
}

template <int KM>
cudaError_t launch_km(const EigArgs &a, const EigSplit &sp, int grid, cudaStream_t s) {
    using S = RatShape<KM>;
    const long long tasks = ((long long)a.npts + kPts - 1) / kPts;
    const long long need = (tasks + kWarpsR - 1) / kWarpsR;
    const unsigned blocks = (unsigned)(need < grid ? need : grid);
    eig_rational_kernel<KM><<<blocks, 32 * kWarpsR, (size_t)S::floats * sizeof(float) * kWarpsR,
                              s>>>(a, sp, zolo_table());
    return cudaGetLastError();
}

}  // namespace

cudaError_t eigen_rational_prepare(int k, int *grid) {
    if (k <= 32) return prepare_km<32>(grid);
    if (k <= kRationalMaxK) return prepare_km<64>(grid);
    return cudaErrorInvalidValue;
}

cudaError_t launch_eigen_rational_transform(const EigArgs &a, const EigSplit &sp, int grid,
                                            cudaStream_t s) {
    if (a.npts <= 0) return cudaSuccess;
    if (a.k <= 32) return launch_km<32>(a, sp, grid, s);
    if (a.k <= kRationalMaxK) return launch_km<64>(a, sp, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace lk
