// Batched symmetric eigensolve, transform and update at every grid point (FP32).
//
// Per grid point (Sec. II-B, Eqs. letkf_xa .. letkf_q):
//   Q   = (k-1)/rho I + A                       A = dY^T R_loc^-1 dY from the Gram kernel
//   Q   = V L V^T                               symmetric eigendecomposition
//   X^a = xbar 1^T + dX (V L^-1 V^T c) 1^T + sqrt(k-1) dX V L^-1/2 V^T
// where dX is the 9 x k block of forecast perturbations of the point (all nine
// populations share one transform, Sec. II-B) and c = dY^T R_loc^-1 (yo - ybar).
//
// The eigensolver follows the batched-EVD route the paper gives (Sec. III):
// Householder tridiagonalization Q = H T H^T, then implicit-shift QL on T = Z L Z^T.
// It runs as one warp per matrix -- the paper's warp-per-batch mapping -- with the
// matrix in shared memory.  Unlike a plain EVD it never forms V = H Z: the
// reflectors and the QL rotations are applied to the 10-row right-hand side
// [dX; c^T] instead (10 k^2 flops instead of 2 k^3 for the back-transform):
//     C = [dX; c^T] H Z          (rows 0..8: dX V, row 9: (V^T c)^T)
//     mean increment = C[0..8] L^-1 C[9]^T
//     perturbations  = (sqrt(k-1) C[0..8] L^-1/2) Z^T H^T
// The tridiagonal (d, e) of the QL phase lives in registers, one element per lane
// and read through warp shuffles, so the sequential bulge chase needs no shared
// memory traffic and no intra-warp synchronisation; only the rotation of the
// lane-owned columns of Z touches shared memory.
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace lk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxIter = 30;   // QL iterations per eigenvalue before ENOTCONV is latched
constexpr int kRows = 10;      // right-hand-side rows: 9 populations + c

__host__ __device__ inline int smem_floats(int k) {
    const int ld = k + 1;
    return 2 * k * ld + kRows * ld + 3 * k;
}

template <int NC>
__device__ __forceinline__ float lane_get(const float (&r)[NC], int idx) {
    float v = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float t = __shfl_sync(kFull, r[c], idx & 31);
        if ((idx >> 5) == c) v = t;
    }
    return v;
}

template <int NC>
__device__ __forceinline__ void lane_set(float (&r)[NC], int idx, float v, int lane) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
        if (lane + 32 * c == idx) r[c] = v;
}

// b <- b H_j for rows 0..nrows-1 of B, H_j = I - tau v v^T acting on indices j+1..k-1.
template <int NC>
__device__ __forceinline__ void apply_reflector(float *B, int ld, int nrows, const float *v,
                                                float tau, int j, int k, int lane) {
    const int m = k - 1 - j;
    float part[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) part[r] = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int t = lane + 32 * c;
        if (t < m) {
            const float vt = v[t];
#pragma unroll
            for (int r = 0; r < kRows; ++r)
                if (r < nrows) part[r] = fmaf(B[r * ld + j + 1 + t], vt, part[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r)
        if (r < nrows) part[r] = warp_sum(part[r]) * tau;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int t = lane + 32 * c;
        if (t < m) {
            const float vt = v[t];
#pragma unroll
            for (int r = 0; r < kRows; ++r)
                if (r < nrows) B[r * ld + j + 1 + t] -= part[r] * vt;
        }
    }
    __syncwarp();
}

template <int NC>
__global__ void __launch_bounds__(128) eigen_update_kernel(EigArgs a) {
    extern __shared__ float smem[];
    const int k = a.k;
    const int ld = k + 1;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float *S = smem + (size_t)wib * smem_floats(k);
    float *Z = S + k * ld;
    float *B = Z + k * ld;
    float *wv = B + kRows * ld;   // w = p - K v of the current reflection
    float *es = wv + k;           // subdiagonal from the reflections
    float *taus = es + k;         // reflector scalars

    const int warps_per_block = blockDim.x >> 5;
    const int nw = gridDim.x * warps_per_block;
    const float eps = FLT_EPSILON;
    const float sk1 = sqrtf((float)(k - 1));

    for (int lp = blockIdx.x * warps_per_block + wib; lp < a.npts; lp += nw) {
        if (a.nloc[lp] == 0) {  // no local observation: Q = (k-1)/rho I, X^a = X^f
            if (a.eigval)
                for (int t = lane; t < k; t += 32) a.eigval[(size_t)lp * k + t] = a.diag;
            continue;
        }
        // ---- Q = diag + A, symmetrised from the upper triangle
        const float *Ag = a.gram + (size_t)lp * k * k;
        for (int i = 0; i < k; ++i)
            for (int j = i + lane; j < k; j += 32) {
                const float v = Ag[i * k + j];
                S[i * ld + j] = v;
                S[j * ld + i] = v;
            }
        __syncwarp();
        for (int i = lane; i < k; i += 32) S[i * ld + i] += a.diag;

        // ---- forecast block: mean and perturbations of the 9 populations, and c
        float *X = a.x + (size_t)(a.pt0 + lp) * NV * k;
        float xbar[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float s = 0.0f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) s += X[q * k + t];
            }
            xbar[q] = warp_sum(s) / (float)k;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) B[q * ld + t] = X[q * k + t] - xbar[q];
            }
        }
        for (int t = lane; t < k; t += 32) B[9 * ld + t] = a.cvec[(size_t)lp * k + t];
        __syncwarp();

        // ---- Householder tridiagonalization, reflector j stored in row j of S
        for (int j = 0; j < k - 2; ++j) {
            const int m = k - 1 - j;
            float *vj = S + j * ld + j + 1;
            float x[NC];
            float tail = 0.0f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                x[c] = t < m ? vj[t] : 0.0f;
                if (t >= 1) tail = fmaf(x[c], x[c], tail);
            }
            tail = warp_sum(tail);
            const float alpha = __shfl_sync(kFull, x[0], 0);
            float tau = 0.0f, beta = alpha, scale = 0.0f;
            if (tail > 0.0f) {
                beta = -copysignf(sqrtf(fmaf(alpha, alpha, tail)), alpha);
                tau = (beta - alpha) / beta;
                scale = 1.0f / (alpha - beta);
            }
            __syncwarp();
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < m) vj[t] = t == 0 ? 1.0f : x[c] * scale;
            }
            if (lane == 0) {
                taus[j] = tau;
                es[j] = beta;
            }
            __syncwarp();
            if (tau != 0.0f) {
                // p = tau S' v, with S' the trailing block (its column t is read by lane t)
                float pv[NC], vt[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    pv[c] = 0.0f;
                    const int t = lane + 32 * c;
                    vt[c] = t < m ? vj[t] : 0.0f;
                }
                for (int s = 0; s < m; ++s) {
                    const float vs = vj[s];
                    const float *rowS = S + (j + 1 + s) * ld + j + 1;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int t = lane + 32 * c;
                        if (t < m) pv[c] = fmaf(rowS[t], vs, pv[c]);
                    }
                }
                float kk = 0.0f;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    pv[c] *= tau;
                    kk = fmaf(pv[c], vt[c], kk);
                }
                const float K = 0.5f * tau * warp_sum(kk);
                float wvl[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int t = lane + 32 * c;
                    wvl[c] = pv[c] - K * vt[c];
                    if (t < m) wv[t] = wvl[c];
                }
                __syncwarp();
                // S' -= v w^T + w v^T
                for (int s = 0; s < m; ++s) {
                    const float vs = vj[s];
                    const float ws = wv[s];
                    float *rowS = S + (j + 1 + s) * ld + j + 1;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int t = lane + 32 * c;
                        if (t < m) rowS[t] -= fmaf(vs, wvl[c], ws * vt[c]);
                    }
                }
                __syncwarp();
            }
        }
        // ---- tridiagonal into lane registers: lane t holds d_t, e_t (e_t couples t, t+1)
        float dr[NC], er[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            dr[c] = t < k ? S[t * ld + t] : 0.0f;
            er[c] = t < k - 2 ? es[t] : (t == k - 2 ? S[t * ld + t + 1] : 0.0f);
        }
        // ---- reflectors applied to the right-hand side [dX; c^T]
        for (int j = 0; j < k - 2; ++j) {
            const float tau = taus[j];
            if (tau != 0.0f) apply_reflector<NC>(B, ld, kRows, S + j * ld + j + 1, tau, j, k, lane);
        }
        // ---- Z = I
        for (int i = 0; i < k; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) Z[i * ld + t] = (i == t) ? 1.0f : 0.0f;
            }
        __syncwarp();

        // ---- implicit-shift QL on (d, e); Z accumulates the rotations (Z[i][:] = column i)
        bool notconv = false;
        for (int l = 0; l < k; ++l) {
            int iter = 0;
            for (;;) {
                // first m >= l whose coupling e_m is negligible against |d_m| + |d_m+1|
                int msplit = k - 1;
#pragma unroll
                for (int c = NC - 1; c >= 0; --c) {
                    const int t = lane + 32 * c;
                    const float dn0 = __shfl_down_sync(kFull, dr[c], 1);
                    const float dn1 = (c + 1 < NC) ? __shfl_sync(kFull, dr[c + 1 < NC ? c + 1 : c], 0) : 0.0f;
                    const float dnext = lane == 31 ? dn1 : dn0;
                    const bool small = t >= l && t < k - 1 &&
                                       fabsf(er[c]) <= eps * (fabsf(dr[c]) + fabsf(dnext));
                    const unsigned bal = __ballot_sync(kFull, small);
                    if (bal) msplit = 32 * c + __ffs(bal) - 1;
                }
                const int m = msplit;
                if (m == l) break;
                if (iter++ >= kMaxIter) {
                    notconv = true;
                    break;
                }
                // shift: eigenvalue of the leading 2 x 2 block nearer to d_l
                const float dl = lane_get<NC>(dr, l);
                const float el = lane_get<NC>(er, l);
                const float dl1 = lane_get<NC>(dr, l + 1);
                const float th = (dl1 - dl) / (2.0f * el);
                const float rt = hypotf(th, 1.0f);
                float g = lane_get<NC>(dr, m) - dl + el / (th + copysignf(rt, th));
                float s = 1.0f, co = 1.0f, pacc = 0.0f;
                float di1 = lane_get<NC>(dr, m);
                bool underflow = false;
                for (int i = m - 1; i >= l; --i) {
                    const float ei = lane_get<NC>(er, i);
                    const float di = lane_get<NC>(dr, i);
                    const float f = s * ei, b = co * ei;
                    float r = hypotf(f, g);
                    lane_set<NC>(er, i + 1, r, lane);
                    if (r == 0.0f) {
                        lane_set<NC>(dr, i + 1, di1 - pacc, lane);
                        lane_set<NC>(er, m, 0.0f, lane);
                        underflow = true;
                        break;
                    }
                    const float rinv = 1.0f / r;
                    s = f * rinv;
                    co = g * rinv;
                    g = di1 - pacc;
                    r = (di - g) * s + 2.0f * co * b;
                    pacc = s * r;
                    lane_set<NC>(dr, i + 1, g + pacc, lane);
                    g = co * r - b;
                    // Z <- Z G_i on columns i, i+1 (rows i, i+1 of the stored transpose)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int t = lane + 32 * c;
                        if (t < k) {
                            float *zi = Z + i * ld + t;
                            const float za = zi[0], zb = zi[ld];
                            zi[ld] = s * za + co * zb;
                            zi[0] = co * za - s * zb;
                        }
                    }
                    di1 = di;
                }
                if (underflow) continue;
                lane_set<NC>(dr, l, di1 - pacc, lane);
                lane_set<NC>(er, l, g, lane);
                lane_set<NC>(er, m, 0.0f, lane);
            }
        }
        if (notconv && lane == 0) atomicOr(a.status, ST_NOTCONV);
        __syncwarp();

        if (a.eigval)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) a.eigval[(size_t)lp * k + t] = dr[c];
            }

        // ---- C = B Z^T-stored (C[r][j] = sum_i B[r][i] Z[j][i]); lane owns columns j
        float C[NC][kRows];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int r = 0; r < kRows; ++r) C[c][r] = 0.0f;
        for (int i = 0; i < k; ++i) {
            float bi[kRows];
#pragma unroll
            for (int r = 0; r < kRows; ++r) bi[r] = B[r * ld + i];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                const float z = t < k ? Z[t * ld + i] : 0.0f;
#pragma unroll
                for (int r = 0; r < kRows; ++r) C[c][r] = fmaf(bi[r], z, C[c][r]);
            }
        }
        // mean increment dX wbar = C[0..8] L^-1 C[9]; perturbation scaling sqrt(k-1) L^-1/2
        float inc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) inc[q] = 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k) {
                const float lam = dr[c];
                const float wl = C[c][9] / lam;
                const float sc = sk1 / sqrtf(lam);
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    inc[q] = fmaf(C[c][q], wl, inc[q]);
                    C[c][q] *= sc;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) inc[q] = warp_sum(inc[q]);
        __syncwarp();
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k)
#pragma unroll
                for (int q = 0; q < NV; ++q) B[q * ld + t] = C[c][q];
        }
        __syncwarp();
        // ---- E = D Z^T: E[q][i] = sum_j D[q][j] Z[j][i]; lane owns columns i
        float E[NC][NV];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int q = 0; q < NV; ++q) E[c][q] = 0.0f;
        for (int j = 0; j < k; ++j) {
            float dj[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) dj[q] = B[q * ld + j];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                const float z = t < k ? Z[j * ld + t] : 0.0f;
#pragma unroll
                for (int q = 0; q < NV; ++q) E[c][q] = fmaf(dj[q], z, E[c][q]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k)
#pragma unroll
                for (int q = 0; q < NV; ++q) B[q * ld + t] = E[c][q];
        }
        __syncwarp();
        // ---- F = E H^T: reflectors in reverse order on the 9 population rows
        for (int j = k - 3; j >= 0; --j) {
            const float tau = taus[j];
            if (tau != 0.0f) apply_reflector<NC>(B, ld, NV, S + j * ld + j + 1, tau, j, k, lane);
        }
        // ---- X^a = xbar + increment + perturbation, in place
        bool bad = false;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const float base = xbar[q] + inc[q];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) {
                    const float v = base + B[q * ld + t];
                    bad |= !isfinite(v);
                    X[q * k + t] = v;
                }
            }
        }
        if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.status, ST_NONFINITE);
        __syncwarp();
    }
}

template <int NC>
int warps_per_block(int k) {
    const size_t per_warp = (size_t)smem_floats(k) * sizeof(float);
    int warps = (int)((200 * 1024) / per_warp);
    return warps < 1 ? 1 : (warps > 4 ? 4 : warps);
}

template <int NC>
cudaError_t prepare_nc(int k, int *max_blocks) {
    const int warps = warps_per_block<NC>(k);
    const size_t smem = (size_t)smem_floats(k) * sizeof(float) * warps;
    cudaError_t e = cudaFuncSetAttribute(eigen_update_kernel<NC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eigen_update_kernel<NC>, 32 * warps,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *max_blocks = sms * per_sm;
    return cudaSuccess;
}

template <int NC>
cudaError_t launch_nc(const EigArgs &a, cudaStream_t s) {
    const int warps = warps_per_block<NC>(a.k);
    const size_t smem = (size_t)smem_floats(a.k) * sizeof(float) * warps;
    long long need = ((long long)a.npts + warps - 1) / warps;
    long long blocks = a.max_blocks > 0 ? a.max_blocks : 1;
    if (blocks > need) blocks = need;
    eigen_update_kernel<NC><<<(unsigned)blocks, 32 * warps, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t eigen_smem_per_warp(int k) { return (size_t)smem_floats(k) * sizeof(float); }

cudaError_t eigen_prepare(int k, int *max_blocks) {
    if (k <= 32) return prepare_nc<1>(k, max_blocks);
    if (k <= 64) return prepare_nc<2>(k, max_blocks);
    if (k <= 128) return prepare_nc<4>(k, max_blocks);
    return cudaErrorInvalidValue;
}

cudaError_t launch_eigen_update(const EigArgs &a, cudaStream_t s) {
    if (a.npts <= 0) return cudaSuccess;
    if (a.k <= 32) return launch_nc<1>(a, s);
    if (a.k <= 64) return launch_nc<2>(a, s);
    if (a.k <= 128) return launch_nc<4>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace lk
