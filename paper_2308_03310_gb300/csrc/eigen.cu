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
// Householder tridiagonalization Q = H T H^T, then implicit-shift QL on T = Z L Z^T,
// then the back-transform V = H Z.  It runs as one warp per matrix -- the paper's
// warp-per-batch mapping -- with the matrix in shared memory.  W is never formed:
//     C = [dX; c^T] V            (rows 0..8: dX V, row 9: (V^T c)^T)
//     mean increment = C[0..8] L^-1 C[9]^T
//     perturbations  = (sqrt(k-1) C[0..8] L^-1/2) V^T
// (two 10 x k x k products instead of the k^3 product that forms W and the 9 k^2 one
// that applies it).
// In the QL phase every lane runs the same scalar recurrence on (d, e) in shared
// memory, and each lane rotates its own columns of Z, carrying one row in registers
// so that a rotation costs one shared load and one store per lane.
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
    const int n = k * ld + kRows * ld + 6 * k;
    return (n + 3) & ~3;  // keep every warp's slice 16-byte aligned
}

// Block shape per NC (columns per lane): warps per block and the resident blocks per SM that
// the register budget targets, chosen with the shared memory per matrix (k x (k+1) + 10 (k+1)
// + 6k floats) so that registers and shared memory allow the same number of matrices in flight.
template <int NC>
struct EigCfg {
    static constexpr int WARPS = NC == 1 ? 4 : (NC == 2 ? 2 : 1);
    static constexpr int MINB = NC == 1 ? 5 : (NC == 2 ? 5 : 3);
};

template <int NC>
__global__ void __launch_bounds__(32 * EigCfg<NC>::WARPS, EigCfg<NC>::MINB)
    eigen_update_kernel(EigArgs a) {
    extern __shared__ float smem[];
    const int k = a.k;
    const int ld = k + 1;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    // S holds Q during the tridiagonalization; its reflectors are then kept in the point's
    // (already consumed) Gram slot in global memory, and Z reuses S's shared memory.
    float *S = smem + (size_t)wib * smem_floats(k);
    float *Z = S;
    float *B = S + k * ld;
    float2 *vw = reinterpret_cast<float2 *>(B + kRows * ld);  // (v_t, w_t) of the reflection
    float2 *de = vw + k;                    // tridiagonal (d_t, e_t), e_t couples t and t+1
    float *taus = reinterpret_cast<float *>(de + k);  // reflector scalars
    float *vtmp = taus + k;                 // one reflector, back in shared memory

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
        // ---- Q = diag + A, symmetrised from the upper triangle.  Rows are fetched eight at a
        // time with every load of a batch issued before its shared stores.
        float *Ag = a.gram + (size_t)lp * k * k;
        for (int i0 = 0; i0 < k; i0 += 8) {
            float v[8][NC];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int i = i0 + u, j = lane + 32 * c;
                    v[u][c] = (i < k && j < k) ? __ldcg(Ag + i * k + j) : 0.0f;
                }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int i = i0 + u, j = lane + 32 * c;
                    if (i < k && j < k && j >= i) {
                        S[i * ld + j] = v[u][c];
                        S[j * ld + i] = v[u][c];
                    }
                }
        }
        __syncwarp();
        for (int i = lane; i < k; i += 32) S[i * ld + i] += a.diag;

        // ---- forecast block: mean and perturbations of the 9 populations, and c
        float *X = a.x + (size_t)(a.pt0 + lp) * NV * k;
        float xv[NV][NC], cv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
#pragma unroll
            for (int q = 0; q < NV; ++q) xv[q][c] = t < k ? X[q * k + t] : 0.0f;
            cv[c] = t < k ? __ldg(a.cvec + (size_t)lp * k + t) : 0.0f;
        }
        float xbar[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float sum = 0.0f;
#pragma unroll
            for (int c = 0; c < NC; ++c) sum += xv[q][c];
            xbar[q] = warp_sum(sum) / (float)k;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k) {
#pragma unroll
                for (int q = 0; q < NV; ++q) B[q * ld + t] = xv[q][c] - xbar[q];
                B[9 * ld + t] = cv[c];
            }
        }
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
            // H x = beta e_0 with beta = -sign(alpha) ||x||, tau = 1 + |alpha| / ||x||,
            // v = x / (alpha - beta), v_0 = 1 (one rsqrt, one reciprocal, no division)
            float tau = 0.0f, beta = alpha, scale = 0.0f;
            if (tail > 0.0f) {
                const float n2 = fmaf(alpha, alpha, tail);
                float rn = rsqrtf(n2);
                rn = rn * fmaf(-0.5f * n2, rn * rn, 1.5f);
                const float nrm = n2 * rn;
                beta = -copysignf(nrm, alpha);
                tau = fmaf(fabsf(alpha), rn, 1.0f);
                scale = copysignf(__frcp_rn(fabsf(alpha) + nrm), alpha);
            }
            float vt[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                vt[c] = t < m ? (t == 0 ? 1.0f : x[c] * scale) : 0.0f;
            }
            __syncwarp();
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < m) {
                    vj[t] = vt[c];
                    Ag[j * k + j + 1 + t] = vt[c];  // reflector j kept in row j of the slot
                }
            }
            if (lane == 0) {
                taus[j] = tau;
                de[j].y = beta;
            }
            __syncwarp();
            if (tau != 0.0f) {
                // p = tau S' v, with S' the trailing block (its column t is read by lane t);
                // two accumulators halve the dependent FMA chain
                float pv[NC], pw[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) pv[c] = pw[c] = 0.0f;
                int s = 0;
                for (; s + 2 <= m; s += 2) {
                    const float vs0 = vj[s], vs1 = vj[s + 1];
                    const float *r0 = S + (j + 1 + s) * ld + j + 1;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int t = lane + 32 * c;
                        if (t < m) {
                            pv[c] = fmaf(r0[t], vs0, pv[c]);
                            pw[c] = fmaf(r0[ld + t], vs1, pw[c]);
                        }
                    }
                }
                if (s < m) {
                    const float vs0 = vj[s];
                    const float *r0 = S + (j + 1 + s) * ld + j + 1;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int t = lane + 32 * c;
                        if (t < m) pv[c] = fmaf(r0[t], vs0, pv[c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) pv[c] += pw[c];
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
                    if (t < m) vw[t] = make_float2(vt[c], wvl[c]);
                }
                __syncwarp();
                // S' -= v w^T + w v^T  (one 8-byte broadcast load of (v_s, w_s) per row)
#pragma unroll 4
                for (int s = 0; s < m; ++s) {
                    const float2 p2 = vw[s];
                    float *rowS = S + (j + 1 + s) * ld + j + 1;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int t = lane + 32 * c;
                        if (t < m) rowS[t] -= fmaf(p2.x, wvl[c], p2.y * vt[c]);
                    }
                }
                __syncwarp();
            }
        }
        // ---- tridiagonal (d, e) into shared memory, e_t couples t and t+1; Z = I over S
        for (int t = lane; t < k; t += 32) {
            de[t].x = S[t * ld + t];
            if (t == k - 2) de[t].y = S[t * ld + t + 1];
            if (t == k - 1) de[t].y = 0.0f;
        }
        __syncwarp();
        for (int i = 0; i < k; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) Z[i * ld + t] = (i == t) ? 1.0f : 0.0f;
            }
        __syncwarp();

        // ---- implicit-shift QL on (d, e); Z accumulates the rotations (Z[i][:] = column i).
        // Every lane runs the same scalar recurrence; d and e are read from shared memory
        // (the next index is fetched one rotation ahead, off the dependency chain) and each
        // rotation's results are written by all lanes with identical values, ordered by one
        // __syncwarp per rotation.  The rotation needs 1/sqrt(f^2 + g^2): MUFU rsqrt refined
        // by one Newton step; there is no branch on the hot path other than the underflow
        // exit of the classical algorithm.
        bool notconv = false;
        for (int l = 0; l < k; ++l) {
            int iter = 0;
            for (;;) {
                // first m >= l whose coupling e_m is negligible against |d_m| + |d_m+1|
                int msplit = k - 1;
#pragma unroll
                for (int c = NC - 1; c >= 0; --c) {
                    const int t = lane + 32 * c;
                    bool small = false;
                    if (t >= l && t < k - 1) {
                        const float2 a0 = de[t];
                        small = fabsf(a0.y) <= eps * (fabsf(a0.x) + fabsf(de[t + 1].x));
                    }
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
                const float2 del = de[l];
                const float dl = del.x, el = del.y, dl1 = de[l + 1].x;
                const float th = (dl1 - dl) / (2.0f * el);
                const float rt = hypotf(th, 1.0f);
                float di1 = de[m].x;
                float g = di1 - dl + el / (th + copysignf(rt, th));
                float s = 1.0f, co = 1.0f, pacc = 0.0f;
                float zc[NC];  // carried column entries of row i+1 of Z
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int t = lane + 32 * c;
                    zc[c] = t < k ? Z[m * ld + t] : 0.0f;
                }
                float ei = de[m - 1].y, di = de[m - 1].x;
                bool underflow = false;
                int i = m - 1;
                float *zp = Z + i * ld + lane;  // row i of Z at this lane's first column
                for (; i >= l; --i) {
                    // next index fetched ahead; at i == l == 0 this reads the pair before de,
                    // which lies inside this warp's slice and is never used
                    const float2 dnext = de[i - 1];
                    const float f = s * ei, b = co * ei;
                    const float ff = fmaf(f, f, g * g);
                    __syncwarp();   // every lane has read index i+1 before it is rewritten
                    if (ff < 1e-30f) {  // f and g vanish: the coupling has underflowed
                        de[i + 1] = make_float2(di1 - pacc, 0.0f);
                        de[m].y = 0.0f;
                        underflow = true;
                        break;
                    }
                    float rinv = rsqrtf(ff);
                    rinv = rinv * fmaf(-0.5f * ff, rinv * rinv, 1.5f);
                    const float enew = ff * rinv;
                    s = f * rinv;
                    co = g * rinv;
                    g = di1 - pacc;
                    const float r = (di - g) * s + 2.0f * co * b;
                    pacc = s * r;
                    de[i + 1] = make_float2(g + pacc, enew);
                    g = co * r - b;
                    // Z <- Z G_i on columns i, i+1: row i+1 is final, row i is carried on
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        if (lane + 32 * c < k) {
                            const float za = zp[32 * c];
                            zp[ld + 32 * c] = s * za + co * zc[c];
                            zc[c] = co * za - s * zc[c];
                        }
                    }
                    zp -= ld;
                    di1 = di;
                    ei = dnext.y;
                    di = dnext.x;
                }
                // the carried row: row i+1 after an underflow break, row l after a full sweep
                const int last = underflow ? i + 1 : l;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int t = lane + 32 * c;
                    if (t < k) Z[last * ld + t] = zc[c];
                }
                __syncwarp();
                if (!underflow) {
                    de[l] = make_float2(di1 - pacc, g);
                    de[m].y = 0.0f;
                }
                __syncwarp();
            }
        }
        if (notconv && lane == 0) atomicOr(a.status, ST_NOTCONV);
        __syncwarp();
        float dr[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            dr[c] = t < k ? de[t].x : 1.0f;
        }

        // ---- V = H Z: the reflectors applied from the left, innermost first.  Lane owns
        // column col of Z (a stored row, odd stride: no bank conflicts); every lane is busy
        // and no cross-lane reduction is needed.  Reflector j comes back from row j of the
        // point's Gram slot (L2), fetched one reflector ahead.
        float vnext[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c, m0 = 2;  // reflector k-3 has m = 2
            vnext[c] = (k >= 3 && t < m0) ? __ldcg(Ag + (k - 3) * k + (k - 2) + t) : 0.0f;
        }
        for (int j = k - 3; j >= 0; --j) {
            const int m = k - 1 - j;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < m) vtmp[t] = vnext[c];
            }
            __syncwarp();
            if (j > 0)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int t = lane + 32 * c;
                    vnext[c] = t < m + 1 ? __ldcg(Ag + (j - 1) * k + j + t) : 0.0f;
                }
            const float tau = taus[j];
            const float *v = vtmp;
            if (tau != 0.0f) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int col = lane + 32 * c;
                    if (col < k) {
                        float *zc_ = Z + col * ld + j + 1;
                        float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, d3 = 0.0f;
                        int t = 0;
                        for (; t + 4 <= m; t += 4) {
                            d0 = fmaf(v[t], zc_[t], d0);
                            d1 = fmaf(v[t + 1], zc_[t + 1], d1);
                            d2 = fmaf(v[t + 2], zc_[t + 2], d2);
                            d3 = fmaf(v[t + 3], zc_[t + 3], d3);
                        }
                        for (; t < m; ++t) d0 = fmaf(v[t], zc_[t], d0);
                        const float beta = ((d0 + d1) + (d2 + d3)) * tau;
#pragma unroll 4
                        for (t = 0; t < m; ++t) zc_[t] = fmaf(-beta, v[t], zc_[t]);
                    }
                }
            }
            __syncwarp();
        }

        if (a.eigval)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) a.eigval[(size_t)lp * k + t] = dr[c];
            }

        // ---- C = B V (C[r][j] = sum_i B[r][i] V[i][j], V[i][j] stored at Z[j][i]); lane owns j
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
        // ---- F = D V^T: F[q][i] = sum_j D[q][j] V[i][j]; lane owns columns i
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
cudaError_t prepare_nc(int k, int *max_blocks) {
    const int warps = EigCfg<NC>::WARPS;
    const size_t smem = (size_t)smem_floats(k) * sizeof(float) * warps;
    auto kern = eigen_update_kernel<NC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *max_blocks = sms * per_sm;
    return cudaSuccess;
}

template <int NC>
cudaError_t launch_nc(const EigArgs &a, cudaStream_t s) {
    const int warps = EigCfg<NC>::WARPS;
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
