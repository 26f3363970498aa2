// EVD-free transform by Chebyshev polynomials in Q (the LETKF_EIG_CHEBYSHEV schedule, FP32).
//
// The transform of a grid point needs two matrix functions of Q = d I + A, d = (k-1)/rho and A
// the localized Gram matrix (positive semidefinite), applied to the forecast (Sec. II-B, Eqs.
// letkf_wa, letkf_dwa, letkf_xa):
//     mean increment   dX Q^-1 c
//     perturbations    sqrt(k-1) dX Q^-1/2
// S = Q / d has its spectrum in [1, kappa] for every kappa >= 1 + lambda_max(A) / d, and on that
// interval t^-1/2 and t^-1 are approximated by Chebyshev expansions
//     t^-1/2 ~ sum_j a_j T_j(s),   t^-1 ~ sum_j b_j T_j(s),   s = (2 t - kappa - 1) / (kappa - 1),
// the interpolants at the Chebyshev points of the first kind (FP64 on the host, the degree
// chosen per kappa so that the relative error stays below 2e-8).  The ten rows R = [dX; c^T]
// (10 x k) are multiplied by these polynomials in S from the right with Clenshaw's recurrence,
// one product with Z = (2 S - (kappa + 1) I) / (kappa - 1) per degree.  Z = gamma A - I with
// gamma = 2 / (d (kappa - 1)): A enters directly, so nothing cancels when kappa is near 1.
// Rows 0..8 take the coefficients of t^-1/2, row 9 those of t^-1; then
//     dX Q^-1/2 = d^-1/2 dX S^-1/2,   Q^-1 c = d^-1 S^-1 c.
// No factorization, eigenvalue or eigenvector is formed.
//
// kappa comes from the cheapest upper bounds of lambda_max(A): the least of the Gershgorin
// bound, the Frobenius norm and the trace.  The degree grows like sqrt(kappa) (1 for kappa <=
// 1.0002, 2 for 1.005, 3 for 1.035, 4 for 1.1, 10 for 2, 36 for 16); a point beyond the last
// approximation goes to the rational schedule (tridiagonalization and Zolotarev's
// approximation) through a list.
//
// Layout: one warp per grid point.  Lane l holds columns l and l + 32 of A in registers, loaded
// from the upper triangle of the Gram slot (the rows above the diagonal coalesced, the lane's
// own row beyond it) with every load in flight at once.  A product R A reads the rows as
// 16-byte broadcasts from shared memory: for k <= 64 five rows per pass (5 loads for 40
// multiply-adds), for k <= 32 all ten.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "letkf.h"

namespace lk {

// ---- coefficients (host, FP64) ---------------------------------------------------------

namespace {

constexpr double kPiC = 3.14159265358979323846;

// Chebyshev series sum_j c_j T_j(s) at s (Clenshaw, FP64).
double cheb_eval(const double *c, int n, double s) {
    double b1 = 0.0, b2 = 0.0;
    for (int j = n; j >= 1; --j) {
        const double b0 = c[j] + 2.0 * s * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return c[0] + s * b1 - b2;
}

}  // namespace

// Coefficients of the degree-n interpolants of t^-1/2 (ca) and t^-1 (cb) on [1, kappa] at the
// Chebyshev points of the first kind, in the variable s = (2 t - kappa - 1) / (kappa - 1);
// returns the larger of the two largest relative errors on a fine grid of the interval.
double chebyshev_coefficients(double kappa, int n, double *ca, double *cb) {
    const int m = n + 1;
    for (int j = 0; j <= n; ++j) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < m; ++i) {
            const double th = kPiC * (i + 0.5) / m;
            const double t = 1.0 + 0.5 * (cos(th) + 1.0) * (kappa - 1.0);
            const double cj = cos(j * th);
            sa += cj / sqrt(t);
            sb += cj / t;
        }
        ca[j] = (j == 0 ? 1.0 : 2.0) * sa / m;
        cb[j] = (j == 0 ? 1.0 : 2.0) * sb / m;
    }
    const int G = 20000;
    double err = 0.0;
    for (int g = 0; g <= G; ++g) {
        const double t = 1.0 + (kappa - 1.0) * g / G;
        const double s = (2.0 * t - kappa - 1.0) / (kappa - 1.0);
        err = fmax(err, fabs(cheb_eval(ca, n, s) * sqrt(t) - 1.0));
        err = fmax(err, fabs(cheb_eval(cb, n, s) * t - 1.0));
    }
    return err;
}

// The approximations the schedule chooses from: for each kappa_max the smallest degree whose
// error stays below 2e-8 (under FP32 rounding of the result).
const ChebTable &cheb_table() {
    static ChebTable t;
    static std::once_flag once;
    std::call_once(once, [] {
        const double kmax[kChebSets] = {1.0002, 1.005, 1.035, 1.1, 1.2,  1.35, 1.5, 1.75,
                                        2.0,    2.5,   3.0,   4.0, 6.0, 10.0, 16.0};
        for (int s = 0; s < kChebSets; ++s) {
            // the interval the kernel maps onto [-1, 1] is the FP32 kappa_max: the coefficients
            // and the degree are those of that interval
            const float kf = (float)kmax[s];
            const double km = (double)kf;
            double ca[kChebMaxDeg + 1], cb[kChebMaxDeg + 1];
            int n = 1;
            while (n < kChebMaxDeg && chebyshev_coefficients(km, n, ca, cb) > 2e-8) ++n;
            chebyshev_coefficients(km, n, ca, cb);
            t.kappa_max[s] = kf;
            t.n[s] = n;
            for (int j = 0; j <= kChebMaxDeg; ++j)
                t.c[s][j] = j <= n ? make_float2((float)ca[j], (float)cb[j])
                                   : make_float2(0.0f, 0.0f);
        }
    });
    return t;
}

// The largest set the transform uses for ensemble size k: degrees up to 9k/16 (at least 4).
// A product with A costs ~20 k^2 flops, the rational schedule's tridiagonalization and
// transform ~(4/3) k^3 + 40 k^2 at a lower issue efficiency; at k = 64 the two measured equal
// near degree 36, and the break-even degree scales with k.  Points beyond go to the rational
// schedule, so the Chebyshev schedule never costs much more than the rational one.
int cheb_max_set(int k) {
    const ChebTable &t = cheb_table();
    const int nmax = std::max(4, 9 * k / 16);
    int s = 0;
    while (s + 1 < kChebSets && t.n[s + 1] <= nmax) ++s;
    return s;
}

// ---- the transform kernel ---------------------------------------------------------------

namespace {

constexpr unsigned kAllC = 0xffffffffu;
constexpr int kWarpsC = 4;   // warps per block
constexpr int kRowsC = 10;   // rows of R: the nine populations' perturbations, then c

template <int KM>
struct ChebShape {
    static constexpr int NS = KM / 32;             // column slots per lane
    static constexpr int RP = KM == 64 ? 5 : 10;   // rows per product pass
    static constexpr int NP = kRowsC / RP;         // passes per product
    static constexpr int BUF = kRowsC * KM;        // one row buffer [10][KM]
    static constexpr int off_xb = 3 * BUF;         // the rows' means [9]
    static constexpr int floats = off_xb + 16;
    static constexpr int SP = KM + 4;               // row stride of the prefetched Gram slot
    static constexpr int PF = KM * SP;              // its floats (after all warps' buffers)
    static_assert((floats * 4 * kWarpsC) % 16 == 0 && (PF * 4) % 16 == 0, "16-byte rows");
};

constexpr unsigned long long kChebWaitNs = 2000000000ull;   // bound of a prefetch wait (2 s)

__device__ __forceinline__ bool cheb_bar_wait(uint32_t bar, uint32_t parity) {
    unsigned long long t0 = 0;
    for (bool first = true;; first = false) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (first) t0 = t;
        else if (t - t0 > kChebWaitNs) return false;
    }
}

__device__ __forceinline__ float warp_max_c(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kAllC, v, o));
    return v;
}

template <int KM>
__global__ void __launch_bounds__(32 * kWarpsC, KM == 64 ? 2 : 3)
    eig_cheb_kernel(EigArgs a, EigSplit sp, const __grid_constant__ ChebTable ct, int max_set) {
    using S = ChebShape<KM>;
    constexpr int NS = S::NS, RP = S::RP, BUF = S::BUF;
    extern __shared__ float4 smem_c4[];
    __shared__ __align__(8) uint64_t pbar[kWarpsC];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *ws = reinterpret_cast<float *>(smem_c4) + (size_t)wib * S::floats;
    float *R0 = ws, *xbs = ws + S::off_xb;
    const int k = a.k;
    const float d = a.diag, inv_d = 1.0f / a.diag;
    const float sc = sqrtf((float)(k - 1)) / sqrtf(a.diag);   // sqrt(k-1) d^-1/2
    unsigned long long n_pts = 0, n_prod = 0, n_hand = 0;
    const long long nw = (long long)gridDim.x * kWarpsC;
    // Where the Gram slot's rows are 16-byte multiples (k a multiple of 4) the warp prefetches
    // its next point's slot into shared memory (rows of k floats at stride SP, one bulk copy
    // per row, counted in bytes on the warp's mbarrier) while it works on the current point.
    const bool pf = (k & 3) == 0;
    float *PS = reinterpret_cast<float *>(smem_c4) + (size_t)kWarpsC * S::floats +
                (size_t)wib * S::PF;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&pbar[wib]);
    uint32_t phase = 0;
    auto prefetch = [&](long long q) {
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"((uint32_t)(k * k * 4))
                         : "memory");
        __syncwarp();
        const float *src = a.gram + (size_t)q * k * k;
        for (int i = lane; i < k; i += 32)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                "[%3];" ::"r"((uint32_t)__cvta_generic_to_shared(PS + i * S::SP)),
                "l"(src + (size_t)i * k), "r"((uint32_t)(k * 4)), "r"(bar)
                : "memory");
    };
    long long lp = (long long)blockIdx.x * kWarpsC + wib;
    if (pf) {
        if (lane == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
            asm volatile("fence.mbarrier_init.release.cluster;");
        }
        __syncwarp();
        if (lp < a.npts) prefetch(lp);
    }
    for (; lp < a.npts; lp += nw) {
        float *X = a.x + (size_t)(a.pt0 + lp) * NV * k;
        const bool zero = a.nloc && a.nloc[lp] == 0;
        float A[NS][KM];
        float dg = 0.0f;
        if (pf) {
            // this point's slot (bounded wait; a timeout is never expected: report it, give
            // the copies a second bounded wait, leave)
            if (!__all_sync(kAllC, cheb_bar_wait(bar, phase))) {
                if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
                cheb_bar_wait(bar, phase);
                return;
            }
            phase ^= 1;
            if (!zero) {
                // A from the staged slot: lane c takes A[i][c] for i <= c down its column and
                // A[c][i] = A[i][c] for i > c along its own row (16-byte reads; the padded
                // stride keeps a quarter warp's rows in distinct banks)
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int c = lane + 32 * q;
#pragma unroll
                    for (int i = 0; i < KM; ++i)
                        A[q][i] = (i < k && c < k && i <= c) ? PS[i * S::SP + c] : 0.0f;
                }
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int c = lane + 32 * q;
                    if (c >= k) continue;
                    const float4 *row = reinterpret_cast<const float4 *>(PS + c * S::SP);
#pragma unroll
                    for (int g = 0; g < KM / 4; ++g)
                        if (4 * g + 3 > c && 4 * g < k) {
                            const float4 v = row[g];
                            if (4 * g > c) A[q][4 * g] = v.x;
                            if (4 * g + 1 > c) A[q][4 * g + 1] = v.y;
                            if (4 * g + 2 > c) A[q][4 * g + 2] = v.z;
                            A[q][4 * g + 3] = v.w;
                        }
                    dg += PS[c * S::SP + c];
                }
            }
            // the slot's reads are done before the next point's copies overwrite it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lp + nw < a.npts) prefetch(lp + nw);
        }
        if (zero) {
            // Q = (k-1)/rho I: wbar = 0 and dW = sqrt(rho) I (untouched for rho = 1)
            if (a.sqrt_infl != 1.0f)
                for (int r = 0; r < NV; ++r) {
                    float v[NS], s = 0.0f;
#pragma unroll
                    for (int q = 0; q < NS; ++q) {
                        const int c = lane + 32 * q;
                        v[q] = c < k ? __ldcg(X + r * k + c) : 0.0f;
                        s += v[q];
                    }
                    const float xb = warp_sum(s) / (float)k;
#pragma unroll
                    for (int q = 0; q < NS; ++q) {
                        const int c = lane + 32 * q;
                        if (c < k) X[r * k + c] = fmaf(a.sqrt_infl, v[q] - xb, xb);
                    }
                }
            continue;
        }
        // ---- A, symmetric, from the upper triangle of the Gram slot straight into registers
        // (without the prefetch), every load of the point in flight at once: lane c takes
        // A[i][c] for i <= c from the rows i (coalesced across the lanes) and A[c][i] = A[i][c]
        // for i > c from its own row
        const float *Ag = a.gram + (size_t)lp * k * k;
        if (!pf) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int c = lane + 32 * q;
#pragma unroll
            for (int i = 0; i < KM; ++i)
                A[q][i] = (i < k && c < k && i <= c) ? __ldg(Ag + i * k + c) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int c = lane + 32 * q;
            if (c >= k) continue;
            const float *row = Ag + (size_t)c * k;
            if ((k & 3) == 0) {   // 16-byte loads: the row starts on a 16-byte boundary
#pragma unroll
                for (int g = 0; g < KM / 4; ++g)
                    if (4 * g + 3 > c && 4 * g < k) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(row) + g);
                        if (4 * g > c) A[q][4 * g] = v.x;
                        if (4 * g + 1 > c) A[q][4 * g + 1] = v.y;
                        if (4 * g + 2 > c) A[q][4 * g + 2] = v.z;
                        A[q][4 * g + 3] = v.w;
                    }
            } else {
#pragma unroll
                for (int i = 0; i < KM; ++i)
                    if (i > c && i < k) A[q][i] = __ldg(row + i);
            }
        }
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int c = lane + 32 * q;
            if (c < k) dg += __ldg(Ag + (size_t)c * k + c);
        }
        }
        // the forecast rows and c, parked in R0 (each lane its columns)
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int c = lane + 32 * q;
#pragma unroll
            for (int r = 0; r < NV; ++r) R0[r * KM + c] = c < k ? __ldcg(X + r * k + c) : 0.0f;
            R0[NV * KM + c] = c < k ? __ldcg(a.cvec + (size_t)lp * k + c) : 0.0f;
        }
        // ---- kappa >= 1 + lambda_max(A) / d from min(Gershgorin, Frobenius, trace)
        float gm = 0.0f, f2 = 0.0f;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            float g = 0.0f;
#pragma unroll
            for (int i = 0; i < KM; ++i) {
                g += fabsf(A[q][i]);
                f2 = fmaf(A[q][i], A[q][i], f2);
            }
            gm = fmaxf(gm, g);
        }
        gm = warp_max_c(gm);
        f2 = warp_sum(f2);
        dg = warp_sum(dg);
        const float e = fmaxf(fminf(gm, fminf(sqrtf(f2), dg)), 0.0f);
        const float kap = fmaf(e * inv_d, 1.0001f, 1.000001f);   // rounding margin
        int set = -1;
        for (int s = max_set; s >= 0; --s)
            if (kap <= ct.kappa_max[s]) set = s;
        if (set < 0) {   // beyond the sets in use (or not finite): the rational schedule
            if (lane == 0) sp.pre_list[atomicAdd(sp.pre_count, 1)] = (int)lp;
            ++n_hand;
            continue;
        }
        // ---- R = [dX; c^T] in R0: the nine rows less their means
        float *Bc = ws + BUF, *Bp = ws + 2 * BUF;
#pragma unroll
        for (int r = 0; r < NV; ++r) {
            float s = 0.0f;
#pragma unroll
            for (int q = 0; q < NS; ++q) s += R0[r * KM + lane + 32 * q];
            const float xb = warp_sum(s) / (float)k;
            if (lane == 0) xbs[r] = xb;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int c = lane + 32 * q;
                if (c < k) R0[r * KM + c] -= xb;
            }
        }
        // ---- Clenshaw: b_n = c_n R, b_j = c_j R + 2 b_{j+1} Z - b_{j+2}, result
        // c_0 R + b_1 Z - b_2, with b_{j+1} Z = gamma b_{j+1} A - b_{j+1}.  Bc holds b_{j+1},
        // Bp b_{j+2}, overwritten entry by entry (each lane its own columns) with b_j.
        const int n = ct.n[set];
        const float gam = 2.0f / (d * (ct.kappa_max[set] - 1.0f));
        {
            const float2 cn = ct.c[set][n];
#pragma unroll
            for (int r = 0; r < kRowsC; ++r)
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int o = r * KM + lane + 32 * q;
                    Bc[o] = (r < NV ? cn.x : cn.y) * R0[o];
                    Bp[o] = 0.0f;
                }
        }
        __syncwarp();
        for (int j = n - 1; j >= 0; --j) {
            const float2 cj = ct.c[set][j];
#pragma unroll
            for (int p = 0; p < S::NP; ++p) {
                float acc[RP][NS];
#pragma unroll
                for (int rr = 0; rr < RP; ++rr)
#pragma unroll
                    for (int q = 0; q < NS; ++q) acc[rr][q] = 0.0f;
                const float4 *B4 = reinterpret_cast<const float4 *>(Bc + p * RP * KM);
#pragma unroll
                for (int g = 0; g < KM / 4; ++g) {
                    float4 bv[RP];
#pragma unroll
                    for (int rr = 0; rr < RP; ++rr) bv[rr] = B4[rr * (KM / 4) + g];
#pragma unroll
                    for (int rr = 0; rr < RP; ++rr)
#pragma unroll
                        for (int q = 0; q < NS; ++q) {
                            float t = acc[rr][q];
                            t = fmaf(bv[rr].x, A[q][4 * g], t);
                            t = fmaf(bv[rr].y, A[q][4 * g + 1], t);
                            t = fmaf(bv[rr].z, A[q][4 * g + 2], t);
                            t = fmaf(bv[rr].w, A[q][4 * g + 3], t);
                            acc[rr][q] = t;
                        }
                }
#pragma unroll
                for (int rr = 0; rr < RP; ++rr) {
                    const int r = p * RP + rr;
                    const float cr = r < NV ? cj.x : cj.y;
#pragma unroll
                    for (int q = 0; q < NS; ++q) {
                        const int o = r * KM + lane + 32 * q;
                        const float z = fmaf(gam, acc[rr][q], -Bc[o]);
                        Bp[o] = j > 0 ? fmaf(cr, R0[o], fmaf(2.0f, z, -Bp[o]))
                                      : fmaf(cr, R0[o], z - Bp[o]);
                    }
                }
            }
            __syncwarp();
            float *t = Bc;
            Bc = Bp;
            Bp = t;
        }
        // ---- u = Q^-1 c = S^-1 c / d; X^a_r = xbar_r + dX_r . u + sqrt(k-1) d^-1/2 (dX S^-1/2)_r
        float uq[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) uq[q] = Bc[NV * KM + lane + 32 * q] * inv_d;
        bool bad = false;
        for (int r = 0; r < NV; ++r) {
            float s = 0.0f;
#pragma unroll
            for (int q = 0; q < NS; ++q) s = fmaf(R0[r * KM + lane + 32 * q], uq[q], s);
            const float base = xbs[r] + warp_sum(s);
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int c = lane + 32 * q;
                if (c < k) {
                    const float v = fmaf(sc, Bc[r * KM + c], base);
                    bad |= !isfinite(v);
                    X[r * k + c] = v;
                }
            }
        }
        if (__any_sync(kAllC, bad) && lane == 0) atomicOr(a.status, ST_NONFINITE);
        ++n_pts;
        n_prod += (unsigned long long)n;
        __syncwarp();   // the row buffers are free for the next point's staging
    }
    if (a.work && lane == 0 && (n_pts | n_hand)) {
        atomicAdd(a.work, n_pts);
        atomicAdd(a.work + 1, n_prod);
        atomicAdd(a.work + 2, n_hand);
    }
}

template <int KM>
cudaError_t cheb_prepare_km(int *grid) {
    using S = ChebShape<KM>;
    const size_t smem = ((size_t)S::floats + S::PF) * sizeof(float) * kWarpsC;
    cudaError_t e = cudaFuncSetAttribute(eig_cheb_kernel<KM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eig_cheb_kernel<KM>,
                                                      32 * kWarpsC, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = sms * per_sm;
    cheb_table();
    return cudaSuccess;
}

template <int KM>
cudaError_t cheb_launch_km(const EigArgs &a, const EigSplit &sp, int grid, cudaStream_t s) {
    using S = ChebShape<KM>;
    const long long need = ((long long)a.npts + kWarpsC - 1) / kWarpsC;
    const unsigned blocks = (unsigned)(need < grid ? need : grid);
    const ChebTable &t = cheb_table();
    eig_cheb_kernel<KM><<<blocks, 32 * kWarpsC,
                          ((size_t)S::floats + S::PF) * sizeof(float) * kWarpsC, s>>>(
        a, sp, t, cheb_max_set(a.k));
    return cudaGetLastError();
}

}  // namespace

cudaError_t eigen_cheb_prepare(int k, int *grid) {
    if (k <= 32) return cheb_prepare_km<32>(grid);
    if (k <= kChebMaxK) return cheb_prepare_km<64>(grid);
    return cudaErrorInvalidValue;
}

cudaError_t launch_eigen_cheb_transform(const EigArgs &a, const EigSplit &sp, int grid,
                                        cudaStream_t s) {
    if (a.npts <= 0) return cudaSuccess;
    if (!sp.pre_list || !sp.pre_count || grid < 1) return cudaErrorInvalidValue;
    if (a.k <= 32) return cheb_launch_km<32>(a, sp, grid, s);
    if (a.k <= kChebMaxK) return cheb_launch_km<64>(a, sp, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace lk

extern "C" double letkf_chebyshev_coefficients(double kappa_max, int32_t n, double *c_rsqrt,
                                               double *c_inv) {
    if (!(kappa_max > 1.0) || !(kappa_max < 1e6) || n < 1 || n > 256 || !c_rsqrt || !c_inv)
        return -1.0;
    return lk::chebyshev_coefficients(kappa_max, n, c_rsqrt, c_inv);
}
