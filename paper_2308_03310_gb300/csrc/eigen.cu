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
// then the back-transform V = H Z.  W is never formed:
//     C = [dX; c^T] V            (rows 0..8: dX V, row 9: (V^T c)^T)
//     mean increment = C[0..8] L^-1 C[9]^T
//     perturbations  = (sqrt(k-1) C[0..8] L^-1/2) V^T
// (two 10 x k x k products instead of the k^3 product that forms W and the 9 k^2 one
// that applies it).
//
// Two schedules compute the same thing:
//  * fused: one warp per matrix -- the paper's warp-per-batch mapping -- runs every phase
//    with the matrix in shared memory.  In its QL phase every lane runs the same scalar
//    recurrence on (d, e), and each lane rotates its own columns of Z, carrying one row in
//    registers so that a rotation costs one shared load and one store per lane.
//  * split: three launches.  (1) warp per matrix: tridiagonalization; (2) thread per
//    matrix: the QL recurrence of 32 matrices per warp instruction, each thread recording
//    its matrix's rotations (one header per sweep, then the sweep's (c, s) pairs) in global
//    memory; (3) warp per matrix: Z = I, the recorded rotations replayed onto Z (no serial
//    recurrence left on the warp's critical path), back-transform, transform and update.
//    A matrix whose rotations outgrow its record is recomputed by the fused kernel, which
//    finds A intact: reflectors live in the strictly lower triangle of the Gram slot.
#include <float.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxIter = 30;   // QL iterations per eigenvalue before ENOTCONV is latched
constexpr int kRows = 10;      // right-hand-side rows: 9 populations + c
constexpr int kQlThreads = 64; // split schedule, QL kernel: matrices per block

__host__ __device__ inline int round4(int n) { return (n + 3) & ~3; }  // 16-byte slices
// fused: S/Z (k x ld), B (kRows x ld), vw (k float2), de (k float2), taus (k), vtmp (k)
__host__ __device__ inline int smem_floats(int k) {
    const int ld = k + 1;
    return round4(k * ld + kRows * ld + 6 * k);
}
// split, tridiagonalization: S (k x ld), vw (tri_vw(k) float2: k rounded up to a multiple of
// 32, the rows the register chains of k <= 64 read), de (k float2), taus (k)
__host__ __device__ inline int tri_vw(int k) { return (k + 31) & ~31; }
__host__ __device__ inline int tri_smem_floats(int k) {
    return round4(round4(k * (k + 1)) + 2 * tri_vw(k) + 3 * k);  // vw 16-byte aligned
}
// split, vectors and update: a staging area first (16-byte aligned; 2 tri_vw(k) + 8 floats:
// the replay's (c, s) by row, rows 0..k+1, then one reflector by absolute row for the
// back-transform, zero-padded to a multiple of 32), Z (k x ld), B (kRows x ld), taus (k)
__host__ __device__ inline int vec_stage_floats(int k) { return 2 * tri_vw(k) + 8; }
__host__ __device__ inline int vec_smem_floats(int k) {
    const int ld = k + 1;
    return round4(vec_stage_floats(k) + k * ld + kRows * ld + k);
}

// Reflector j (m = k-1-j entries) is kept in row k-1-j of the point's Gram slot, columns
// 0..m-1: the strictly lower triangle, so the upper triangle and the diagonal, from which
// Q is read, survive the tridiagonalization.
__device__ __forceinline__ float *refl_row(float *Ag, int k, int j) {
    return Ag + (size_t)(k - 1 - j) * k;
}

// Block shape per NC (columns per lane): warps per block and the resident blocks per SM that
// the register budget targets, chosen with the shared memory per matrix so that registers
// and shared memory allow the same number of matrices in flight.
template <int NC>
struct EigCfg {
    static constexpr int WARPS = NC == 1 ? 4 : (NC == 2 ? 2 : 1);
    static constexpr int MINB = NC == 1 ? 5 : (NC == 2 ? 5 : 3);
    // the split schedule's vector kernel at k <= 32: 8 blocks (64 registers) measured 4 %
    // faster than 5
    static constexpr int MINB_VEC = NC == 1 ? 8 : MINB;
};

// ---- phases (one warp, one matrix) --------------------------------------------------------

// Q = diag + A into S, symmetrised from the upper triangle of the Gram slot.
template <int NC>
__device__ __forceinline__ void load_q(const float *Ag, float *S, int k, int ld, int lane,
                                       float diag) {
    // ---- Q = diag + A, symmetrised from the upper triangle.  Rows are fetched eight at a
    // time with every load of a batch issued before its shared stores.
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
    for (int i = lane; i < k; i += 32) S[i * ld + i] += diag;

}

// Forecast block of the point: B rows 0..8 = dX (perturbations), row 9 = c; returns X.
template <int NC>
__device__ __forceinline__ float *load_forecast(const EigArgs &a, size_t lp, float *B, int k,
                                                int ld, int lane, float (&xbar)[NV]) {
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

    return X;
}

// Householder tridiagonalization of S in place: (d, e) into de, scalars into taus, the
// reflectors into shared memory and into the lower triangle of the Gram slot.
template <int NC>
__device__ __forceinline__ void tridiagonalize(float *Ag, float *S, float2 *vw, float2 *de,
                                               float *taus, int k, int ld, int lane) {
    // ---- Householder tridiagonalization, reflector j stored in row j of S (and in global
    // memory, see refl_row)
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
                refl_row(Ag, k, j)[t] = vt[c];  // lower triangle of the slot
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
    // ---- tridiagonal (d, e) into shared memory, e_t couples t and t+1
    for (int t = lane; t < k; t += 32) {
        de[t].x = S[t * ld + t];
        if (t == k - 2) de[t].y = S[t * ld + t + 1];
        if (t == k - 1) de[t].y = 0.0f;
    }
    __syncwarp();
}

// Z = I (Z[i][:] holds column i of the eigenvector matrix).
template <int NC>
__device__ __forceinline__ void set_identity(float *Z, int k, int ld, int lane) {
    for (int i = 0; i < k; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k) Z[i * ld + t] = (i == t) ? 1.0f : 0.0f;
        }
    __syncwarp();
}

// Implicit-shift QL on (d, e) with the rotations accumulated into Z (fused schedule).
// Returns true if some eigenvalue did not converge.
template <int NC>
__device__ __forceinline__ bool ql_warp(float2 *de, float *Z, int k, int ld, int lane) {
    const float eps = FLT_EPSILON;
    // ---- implicit-shift QL on (d, e); Z accumulates the rotations (Z[i][:] = column i).
    // Every lane runs the same scalar recurrence; d and e are read from shared memory
    // (the next index is fetched one rotation ahead, off the dependency chain) and each
    // rotation's results are written by all lanes with identical values, ordered by one
    // __syncwarp per rotation.  The rotation needs 1/sqrt(f^2 + g^2): MUFU rsqrt refined
    // by one Newton step; there is no branch on the hot path other than the underflow
    // exit of the classical algorithm.
    // Deflation: a coupling e_m is negligible once |e_m| <= eps ||T|| (||T|| the largest
    // |d_t| + |e_t| + |e_t-1|).  A test against the local |d_m| + |d_m+1| alone never fires
    // inside a cluster of small eigenvalues next to large ones: every sweep through the large
    // entries leaves rounding of order eps ||T|| on the small couplings.
    float tn = 0.0f;
    for (int t = lane; t < k; t += 32) {
        const float2 a0 = de[t];
        tn = fmaxf(tn, fabsf(a0.x) + fabsf(a0.y) + (t > 0 ? fabsf(de[t - 1].y) : 0.0f));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tn = fmaxf(tn, __shfl_xor_sync(kFull, tn, o));
    const float tol = eps * tn;
    bool notconv = false;
    for (int l = 0; l < k; ++l) {
        int iter = 0;
        for (;;) {
            // first m >= l whose coupling e_m is negligible
            int msplit = k - 1;
#pragma unroll
            for (int c = NC - 1; c >= 0; --c) {
                const int t = lane + 32 * c;
                bool small = false;
                if (t >= l && t < k - 1) {
                    const float2 a0 = de[t];
                    small = fabsf(a0.y) <= tol;
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
    return notconv;
}

// V = H Z in Z (reflectors from the Gram slot, scalars in taus).
template <int NC>
__device__ __forceinline__ void back_transform(float *Ag, float *Z, const float *taus,
                                               float *vtmp, int k, int ld, int lane) {
    // ---- V = H Z: the reflectors applied from the left, innermost first.  Lane owns
    // column col of Z (a stored row, odd stride: no bank conflicts); every lane is busy
    // and no cross-lane reduction is needed.  Reflector j comes back from the point's
    // Gram slot (L2), fetched one reflector ahead.
    float vnext[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int t = lane + 32 * c, m0 = 2;  // reflector k-3 has m = 2
        vnext[c] = (k >= 3 && t < m0) ? __ldcg(refl_row(Ag, k, k - 3) + t) : 0.0f;
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
                vnext[c] = t < m + 1 ? __ldcg(refl_row(Ag, k, j - 1) + t) : 0.0f;
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

}

// ---- V = H Z with the lane's rows of Z in registers (split schedule, k <= 64) --------------
// Lane owns rows col = lane + 32 c of the stored Z (columns of the eigenvector matrix), all
// 32 NC entries, in registers.  Reflector j is staged in vtmp by absolute row (rows j+1..k-1;
// rows above k and the rows of its first 4-row group below j+1 stay zero), so the dot product
// and the update run over whole 4-row groups from the group holding row j + 1: one 16-byte
// broadcast load and 4 NC multiply-adds per group, entered through a jump table on the group.

template <int NC, int G>
__device__ __forceinline__ void bt_dot(const float (&zr)[NC][32 * NC], const float4 *v4,
                                       float (&acc)[NC][4]) {
    if constexpr (4 * G < 32 * NC) {
        const float4 v = v4[G];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            acc[c][0] = fmaf(v.x, zr[c][4 * G], acc[c][0]);
            acc[c][1] = fmaf(v.y, zr[c][4 * G + 1], acc[c][1]);
            acc[c][2] = fmaf(v.z, zr[c][4 * G + 2], acc[c][2]);
            acc[c][3] = fmaf(v.w, zr[c][4 * G + 3], acc[c][3]);
        }
    }
}

template <int NC, int G>
__device__ __forceinline__ void bt_update(float (&zr)[NC][32 * NC], const float4 *v4,
                                          const float (&beta)[NC]) {
    if constexpr (4 * G < 32 * NC) {
        const float4 v = v4[G];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            zr[c][4 * G] = fmaf(-beta[c], v.x, zr[c][4 * G]);
            zr[c][4 * G + 1] = fmaf(-beta[c], v.y, zr[c][4 * G + 1]);
            zr[c][4 * G + 2] = fmaf(-beta[c], v.z, zr[c][4 * G + 2]);
            zr[c][4 * G + 3] = fmaf(-beta[c], v.w, zr[c][4 * G + 3]);
        }
    }
}

#define LK_G8(M, b) M(b) M(b + 1) M(b + 2) M(b + 3) M(b + 4) M(b + 5) M(b + 6) M(b + 7)
#define LK_GROUPS16(M) LK_G8(M, 0) LK_G8(M, 8)

// The same V = H Z as back_transform(); vtmp holds 32 NC floats, 16-byte aligned.
template <int NC>
__device__ __forceinline__ void back_transform_registers(float *Ag, float *Z, const float *taus,
                                                         float *vtmp, int k, int ld, int lane) {
    constexpr int KM = 32 * NC;
    static_assert(KM / 4 <= 16, "group chain covers 64 rows");
    float zr[NC][KM];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int col = lane + 32 * c;
#pragma unroll
        for (int t = 0; t < KM; ++t) zr[c][t] = (col < k && t < k) ? Z[col * ld + t] : 0.0f;
        vtmp[col] = 0.0f;
    }
    float vnext[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int t = lane + 32 * c;  // reflector k-3 has m = 2
        vnext[c] = (k >= 3 && t < 2) ? __ldcg(refl_row(Ag, k, k - 3) + t) : 0.0f;
    }
    __syncwarp();
    const float4 *v4 = reinterpret_cast<const float4 *>(vtmp);
    for (int j = k - 3; j >= 0; --j) {
        const int m = k - 1 - j;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < m) vtmp[j + 1 + t] = vnext[c];
        }
        __syncwarp();
        if (j > 0)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                vnext[c] = t < m + 1 ? __ldcg(refl_row(Ag, k, j - 1) + t) : 0.0f;
            }
        const float tau = taus[j];
        if (tau != 0.0f) {
            float acc[NC][4];
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[c][u] = 0.0f;
            switch ((j + 1) >> 2) {
#define LK_BT_DOT(G) \
    case G: bt_dot<NC, G>(zr, v4, acc);
                LK_GROUPS16(LK_BT_DOT)
#undef LK_BT_DOT
                default: break;
            }
            float beta[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c)
                beta[c] = ((acc[c][0] + acc[c][1]) + (acc[c][2] + acc[c][3])) * tau;
            switch ((j + 1) >> 2) {
#define LK_BT_UPDATE(G) \
    case G: bt_update<NC, G>(zr, v4, beta);
                LK_GROUPS16(LK_BT_UPDATE)
#undef LK_BT_UPDATE
                default: break;
            }
        }
        __syncwarp();  // every group has read vtmp before the next reflector is staged
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int col = lane + 32 * c;
#pragma unroll
        for (int t = 0; t < KM; ++t)
            if (col < k && t < k) Z[col * ld + t] = zr[c][t];
    }
    __syncwarp();
}
#undef LK_GROUPS16
#undef LK_G8

// C = B V, mean increment, scaled perturbations, X^a written in place.
template <int NC>
__device__ __forceinline__ void transform_update(float *X, float *B, const float *Z,
                                                 const float (&dr)[NC], const float (&xbar)[NV],
                                                 int k, int ld, int lane, int *status) {
    const float sk1 = sqrtf((float)(k - 1));
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
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(status, ST_NONFINITE);
    __syncwarp();
}

// ---- FP64 refinement of clustered eigenpairs ---------------------------------------------

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// One refinement sweep in FP64 for the eigenpairs whose eigenvalue has a neighbour within
// relative distance tau: in index order, each such eigenvector is re-orthogonalized (modified
// Gram-Schmidt) against the earlier vectors of its neighbourhood and normalized, then its
// eigenvalue is replaced by the Rayleigh quotient v^T Q v with Q = diag I + A read from the
// upper triangle of the Gram slot.  Z[i][:] holds eigenvector i, dr[c] the eigenvalue of
// index lane + 32 c.  The only FP64 arithmetic of the analysis.
// Eigenvalues at the floor diag (within 1e-4 relative: directions where A is negligible,
// A's near-null space) are left alone: there Q is diag I to within the cluster's width, the
// matrix functions of the transform are flat, and a cluster of tens of such eigenvalues would
// cost O(cluster^2 k + cluster k^2) FP64 operations for nothing.
template <int NC>
__device__ __forceinline__ void refine_clusters(float *Z, int ld, const float *Ag, float diag,
                                                int k, float (&dr)[NC], int lane, float tau) {
    bool clus[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) clus[c] = false;
    for (int j = 0; j < k; ++j) {
        const float lj = __shfl_sync(kFull, dr[0], j & 31);
        float lv = lj;
#pragma unroll
        for (int c = 1; c < NC; ++c)
            if ((j >> 5) == c) lv = __shfl_sync(kFull, dr[c], j & 31);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k && t != j && fabsf(dr[c] - lv) <= tau * fabsf(dr[c])) clus[c] = true;
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
        if (diag > 0.0f && fabsf(dr[c] - diag) <= 1e-4f * diag) clus[c] = false;
    auto value_of = [&](int i) -> float {  // eigenvalue i, broadcast from its lane
        float v = __shfl_sync(kFull, dr[0], i & 31);
#pragma unroll
        for (int c = 1; c < NC; ++c)
            if ((i >> 5) == c) v = __shfl_sync(kFull, dr[c], i & 31);
        return v;
    };
    unsigned any = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) any |= __ballot_sync(kFull, clus[c]);
    if (!any) return;
    for (int i = 0; i < k; ++i) {
        int ci = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if ((i >> 5) == c) ci = __shfl_sync(kFull, clus[c] ? 1 : 0, i & 31);
        if (!ci) continue;
        const float li = value_of(i);
        double v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            v[c] = t < k ? (double)Z[i * ld + t] : 0.0;
        }
        for (int j = 0; j < i; ++j) {
            if (fabsf(li - value_of(j)) > tau * fabsf(li)) continue;
            double d = 0.0;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) d = fma(v[c], (double)Z[j * ld + t], d);
            }
            d = warp_sum_d(d);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) v[c] = fma(-d, (double)Z[j * ld + t], v[c]);
            }
        }
        double n2 = 0.0;
#pragma unroll
        for (int c = 0; c < NC; ++c) n2 = fma(v[c], v[c], n2);
        const double rn = 1.0 / sqrt(warp_sum_d(n2));
        __syncwarp();
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k) Z[i * ld + t] = (float)(v[c] * rn);
        }
        __syncwarp();
    }
    // Rayleigh quotients v^T Q v of the re-orthogonalized vectors, up to four per pass over
    // the upper triangle of Q (row r read coalesced; each off-diagonal entry counted twice)
    constexpr int RB = 4;
    int batch[RB], nb = 0;
    auto flush = [&]() {
        double part[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) part[b] = 0.0;
        for (int r = 0; r < k; ++r) {
            const float *qrow = Ag + (size_t)r * k;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < r || t >= k) continue;
                double q = (double)__ldcg(qrow + t);
                if (t == r) q += (double)diag;
                const double w = t == r ? 1.0 : 2.0;
#pragma unroll
                for (int b = 0; b < RB; ++b)
                    if (b < nb)
                        part[b] = fma(q * w * (double)Z[batch[b] * ld + r],
                                      (double)Z[batch[b] * ld + t], part[b]);
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            if (b >= nb) break;
            const double rq = warp_sum_d(part[b]);
            const int i = batch[b];
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if ((i >> 5) == c && lane == (i & 31)) dr[c] = (float)rq;
        }
        nb = 0;
    };
    for (int i = 0; i < k; ++i) {
        int ci = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if ((i >> 5) == c) ci = __shfl_sync(kFull, clus[c] ? 1 : 0, i & 31);
        if (!ci) continue;
        batch[nb++] = i;
        if (nb == RB) flush();
    }
    if (nb) flush();
}

// Eigenvector i (row i of Z) into out[i][:].
template <int NC>
__device__ __forceinline__ void store_vectors(const float *Z, int ld, float *out, int k, int lane) {
    for (int i = 0; i < k; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k) out[(size_t)i * k + t] = Z[i * ld + t];
        }
}

// A point without local observations: Q = (k-1)/rho I, so wbar = 0 and dW = sqrt(rho) I; the
// members keep their mean and their perturbations are scaled by sqrt(rho).  With rho = 1 the
// point is left exactly as it is.
__device__ __forceinline__ void inflate_point(const EigArgs &a, long long lp, int lane) {
    if (a.sqrt_infl == 1.0f || !a.x) return;
    const int k = a.k;
    float *X = a.x + (size_t)(a.pt0 + lp) * NV * k;
    for (int q = 0; q < NV; ++q) {
        float sum = 0.0f;
        for (int t = lane; t < k; t += 32) sum += X[q * k + t];
        const float xbar = warp_sum(sum) / (float)k;
        for (int t = lane; t < k; t += 32) X[q * k + t] = fmaf(a.sqrt_infl, X[q * k + t] - xbar, xbar);
    }
    __syncwarp();
}

// ---- fused schedule -----------------------------------------------------------------------

// The whole analysis of grid point lp of a (fused schedule) by one warp, in its slice W of
// shared memory (smem_floats(a.k) floats).
template <int NC>
__device__ __forceinline__ void analyze_point(const EigArgs &a, int lp, float *W, int lane) {
    const int k = a.k;
    const int ld = k + 1;
    // S holds Q during the tridiagonalization; its reflectors are then kept in the point's
    // Gram slot in global memory, and Z reuses S's shared memory.
    float *S = W;
    float *Z = S;
    float *B = S + k * ld;
    float2 *vw = reinterpret_cast<float2 *>(B + kRows * ld);  // (v_t, w_t) of the reflection
    float2 *de = vw + k;                    // tridiagonal (d_t, e_t), e_t couples t and t+1
    float *taus = reinterpret_cast<float *>(de + k);  // reflector scalars
    float *vtmp = taus + k;                 // one reflector, back in shared memory
    if (a.nloc && a.nloc[lp] == 0) {  // no local observation: Q = (k-1)/rho I
        if (a.eigval)
            for (int t = lane; t < k; t += 32) a.eigval[(size_t)lp * k + t] = a.diag;
        inflate_point(a, lp, lane);
        return;
    }
    float *Ag = a.gram + (size_t)lp * k * k;
    load_q<NC>(Ag, S, k, ld, lane, a.diag);
    float xbar[NV];
    float *X = a.x ? load_forecast<NC>(a, lp, B, k, ld, lane, xbar) : nullptr;
    tridiagonalize<NC>(Ag, S, vw, de, taus, k, ld, lane);
    set_identity<NC>(Z, k, ld, lane);
    const bool notconv = ql_warp<NC>(de, Z, k, ld, lane);
    if (notconv && lane == 0) atomicOr(a.status, ST_NOTCONV);
    __syncwarp();
    float dr[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int t = lane + 32 * c;
        dr[c] = t < k ? de[t].x : 1.0f;
    }
    back_transform<NC>(Ag, Z, taus, vtmp, k, ld, lane);
    if (a.refine) refine_clusters<NC>(Z, ld, Ag, a.diag, k, dr, lane, a.refine_tau);
    if (a.evec) store_vectors<NC>(Z, ld, a.evec + (size_t)lp * k * k, k, lane);
    if (a.eigval)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t < k) a.eigval[(size_t)lp * k + t] = dr[c];
        }
    if (X) {
        transform_update<NC>(X, B, Z, dr, xbar, k, ld, lane, a.status);
    } else {  // eigenpairs only: report non-finite eigenvalues
        bool bad = false;
#pragma unroll
        for (int c = 0; c < NC; ++c) bad |= lane + 32 * c < k && !isfinite(dr[c]);
        if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.status, ST_NONFINITE);
    }
    __syncwarp();
}

template <int NC>
__global__ void __launch_bounds__(32 * EigCfg<NC>::WARPS, EigCfg<NC>::MINB)
    eigen_update_kernel(EigArgs a) {
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float *W = smem + (size_t)wib * smem_floats(a.k);
    const int warps_per_block = blockDim.x >> 5;
    const int nw = gridDim.x * warps_per_block;
    // the whole chunk, or only the points of a list (matrices the split schedule hands back)
    const int n = a.list ? *a.list_count : a.npts;
    for (int it = blockIdx.x * warps_per_block + wib; it < n; it += nw)
        analyze_point<NC>(a, a.list ? a.list[it] : it, W, lane);
}

// ---- grouped schedule: several ensembles' grid points in one persistent launch -------------

// One launch over the points of up to kMaxGroupSeg segments (chunks of different handles,
// any k of this NC class): every warp takes the next point from a global counter, so grid
// points with many, few or no local observations and matrices of different order spread
// over the warps as they free up.  Segments are ordered by decreasing k (largest jobs first).
template <int NC>
__global__ void __launch_bounds__(32 * EigCfg<NC>::WARPS, EigCfg<NC>::MINB)
    eigen_group_kernel(const __grid_constant__ EigGroup g) {
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float *W = smem + (size_t)wib * smem_floats(g.kmax);
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(g.counter, 1);
        i = __shfl_sync(kFull, i, 0);
        if (i >= g.start[g.n]) break;
        int sg = 0;
        while (i >= g.start[sg + 1]) ++sg;
        analyze_point<NC>(g.seg[sg], i - g.start[sg], W, lane);
    }
}

// ---- split schedule -----------------------------------------------------------------------

// ---- tridiagonalization with Q in registers (split schedule) ------------------------------
// Written for NC <= 2 and used for k <= 32: at 33 <= k <= 64 the 212-register form ran 10 %
// slower than the shared-memory one (occupancy), at k <= 32 it cut the kernel by ~40 %.
// The lane keeps its NC columns of Q, all 32 NC rows, in registers: q[c][i] = Q[i][t] with
// t = lane + 32 c.  Every loop over the rows of the trailing block (the product Q'v and the
// rank-2 update) enters an unrolled chain of row steps at row j + 1 through a jump table on j
// and runs to row 32 NC - 1; rows at and beyond k hold zeros (their v and w are zero, and
// step j writes v and w of rows j + 1..k - 1 before its chains read them).  The broadcast
// operands (v, then w) come from shared memory at compile-time offsets.

// q[c][row] for a row index uniform across the warp (jump table)
template <int NC, int I>
__device__ __forceinline__ void tri_pick(const float (&q)[NC][32 * NC], float (&x)[NC]) {
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c] = q[c][I];
}

// Case labels 0..63 in increasing order: a chain entered at case j falls through the rows
// above j + 1.
// The same two row loops over 4-row groups: (v, w) of rows 4G..4G+3 come as two 16-byte
// broadcast loads, the product keeps one accumulator per row mod 4 (four independent
// multiply-add chains), and the rows of the first group below j + 1 hold v = w = 0.
template <int NC, int G>
__device__ __forceinline__ void tri_mv4(const float (&q)[NC][32 * NC], const float4 *vw4,
                                        float (&p)[NC][4]) {
    if constexpr (4 * G < 32 * NC) {
        const float4 a = vw4[2 * G], b = vw4[2 * G + 1];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            p[c][0] = fmaf(q[c][4 * G], a.x, p[c][0]);
            p[c][1] = fmaf(q[c][4 * G + 1], a.z, p[c][1]);
            p[c][2] = fmaf(q[c][4 * G + 2], b.x, p[c][2]);
            p[c][3] = fmaf(q[c][4 * G + 3], b.z, p[c][3]);
        }
    }
}

template <int NC, int G>
__device__ __forceinline__ void tri_up4(float (&q)[NC][32 * NC], const float4 *vw4,
                                        const float (&vt)[NC], const float (&wt)[NC]) {
    if constexpr (4 * G < 32 * NC) {
        const float4 a = vw4[2 * G], b = vw4[2 * G + 1];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            q[c][4 * G] -= fmaf(a.x, wt[c], a.y * vt[c]);
            q[c][4 * G + 1] -= fmaf(a.z, wt[c], a.w * vt[c]);
            q[c][4 * G + 2] -= fmaf(b.x, wt[c], b.y * vt[c]);
            q[c][4 * G + 3] -= fmaf(b.z, wt[c], b.w * vt[c]);
        }
    }
}

#define LK_CASE8(M, b) M(b) M(b + 1) M(b + 2) M(b + 3) M(b + 4) M(b + 5) M(b + 6) M(b + 7)
#define LK_GROUPS16(M) LK_CASE8(M, 0) LK_CASE8(M, 8)
#define LK_CASES64(M)                                                                      \
    LK_CASE8(M, 0) LK_CASE8(M, 8) LK_CASE8(M, 16) LK_CASE8(M, 24) LK_CASE8(M, 32)         \
    LK_CASE8(M, 40) LK_CASE8(M, 48) LK_CASE8(M, 56)

// Householder tridiagonalization of Q (symmetric, in S) with the same reflectors, scalars and
// outputs as tridiagonalize(): reflector j into the lower triangle of the Gram slot, tau_j into
// taus, (d, e) into de.  S is only read.
template <int NC>
__device__ __forceinline__ void tridiagonalize_registers(float *Ag, const float *S, float2 *vw,
                                                         float2 *de, float *taus, int k,
                                                         int ld, int lane) {
    constexpr int KM = 32 * NC;
    float q[NC][KM];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int t = lane + 32 * c;
#pragma unroll
        for (int i = 0; i < KM; ++i) q[c][i] = (i < k && t < k) ? S[i * ld + t] : 0.0f;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) vw[lane + 32 * c] = make_float2(0.0f, 0.0f);
    __syncwarp();
    for (int j = 0; j < k - 2; ++j) {
        // x_t = Q'[t][j] = Q'[j][t] for t > j: the lane's own entries of row j
        float x[NC];
        switch (j) {
#define LK_PICK(i) \
    case i: tri_pick<NC, (i < KM ? i : 0)>(q, x); break;
            LK_CASES64(LK_PICK)
#undef LK_PICK
            default: break;
        }
        float tail = 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            if (t <= j || t >= k) x[c] = 0.0f;
            if (t > j + 1) tail = fmaf(x[c], x[c], tail);
        }
        tail = warp_sum(tail);
        const int ta = j + 1;
        const float alpha =
            __shfl_sync(kFull, NC == 1 || ta < 32 ? x[0] : x[NC > 1 ? 1 : 0], ta & 31);
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
        float *refl = refl_row(Ag, k, j);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            vt[c] = t > j + 1 ? x[c] * scale : (t == j + 1 ? 1.0f : 0.0f);
            if (t > j && t < k) {
                vw[t].x = vt[c];
                refl[t - j - 1] = vt[c];  // lower triangle of the slot
            }
        }
        const int g0 = (j + 1) >> 2;  // the group of row j + 1
        if (lane < 4 && 4 * g0 + lane <= j) vw[4 * g0 + lane] = make_float2(0.0f, 0.0f);
        if (lane == 0) {
            taus[j] = tau;
            de[j].y = beta;
        }
        __syncwarp();
        if (tau != 0.0f) {
            const float4 *vw4 = reinterpret_cast<const float4 *>(vw);
            float p4[NC][4];
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int u = 0; u < 4; ++u) p4[c][u] = 0.0f;
            switch (g0) {
#define LK_MV4(G) \
    case G: tri_mv4<NC, G>(q, vw4, p4);
                LK_GROUPS16(LK_MV4)
#undef LK_MV4
                default: break;
            }
            float p[NC];
            float kk = 0.0f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                p[c] = ((p4[c][0] + p4[c][1]) + (p4[c][2] + p4[c][3])) * tau;
                kk = fmaf(p[c], vt[c], kk);
            }
            const float K = 0.5f * tau * warp_sum(kk);
            float wt[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                wt[c] = t > j && t < k ? p[c] - K * vt[c] : 0.0f;
                if (t > j && t < k) vw[t].y = wt[c];
            }
            __syncwarp();
            switch (g0) {
#define LK_UP4(G) \
    case G: tri_up4<NC, G>(q, vw4, vt, wt);
                LK_GROUPS16(LK_UP4)
#undef LK_UP4
                default: break;
            }
        }
        __syncwarp();  // every row step has read vw before the next step rewrites it
    }
    // ---- (d, e): d_t = Q'[t][t] (the lane's own diagonal), e_{k-2} = Q'[k-2][k-1]
    float dg[NC], el[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        dg[c] = 0.0f;
        el[c] = 0.0f;
        const int t = lane + 32 * c;
#pragma unroll
        for (int i = 0; i < KM; ++i) {
            if (i == t) dg[c] = q[c][i];
            if (i == k - 2) el[c] = q[c][i];
        }
        if (t < k) de[t].x = dg[c];
        if (t == k - 1 && k >= 2) de[k - 2].y = el[c];
        if (t == k - 1) de[t].y = 0.0f;
    }
    __syncwarp();
}
#undef LK_GROUPS16
#undef LK_CASES64
#undef LK_CASE8

// (1) tridiagonalization, warp per matrix: (d, e) and the reflector scalars to global memory.
template <int NC>
__global__ void __launch_bounds__(32 * EigCfg<NC>::WARPS) eig_tridiag_kernel(EigArgs a,
                                                                             EigSplit sp) {
    extern __shared__ float smem[];
    const int k = a.k, ld = k + 1;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *S = smem + (size_t)wib * tri_smem_floats(k);
    float2 *vw = reinterpret_cast<float2 *>(S + round4(k * ld));
    float2 *de = vw + tri_vw(k);
    float *taus = reinterpret_cast<float *>(de + k);
    const int warps_per_block = blockDim.x >> 5;
    const int nw = gridDim.x * warps_per_block;
    const int npts = a.list ? *a.list_count : a.npts;   // the chunk, or the listed points
    for (int it = blockIdx.x * warps_per_block + wib; it < npts; it += nw) {
        const int lp = a.list ? a.list[it] : it;
        if (a.nloc && a.nloc[lp] == 0) continue;
        float *Ag = a.gram + (size_t)lp * k * k;
        load_q<NC>(Ag, S, k, ld, lane, a.diag);
        if constexpr (NC == 1)  // at k <= 64 (212 registers) the shared-memory form is faster
            tridiagonalize_registers<NC>(Ag, S, vw, de, taus, k, ld, lane);
        else
            tridiagonalize<NC>(Ag, S, vw, de, taus, k, ld, lane);
        for (int t = lane; t < k; t += 32) {
            sp.de[(size_t)lp * k + t] = de[t];
            sp.taus[(size_t)lp * k + t] = taus[t];
        }
        __syncwarp();
    }
}

// ---- tridiagonalization by a pair of warps, Q in registers (33 <= k <= 64) ----------------
// The same reflectors, scalars and outputs as tridiagonalize(), with the matrix split over two
// warps: lane l of warp h holds column t = 32 h + l, all 64 rows, in registers (64 floats per
// lane instead of the 128 a single warp would need).  Per reflector the pair meets four times
// at a named barrier: after the column's norm and alpha, after v, after the dot product v.p,
// after w; (v, w) and the partial sums live in shared memory, double-buffered by reflector
// parity so that the next reflector's writes never meet this one's reads.  The product Q'v and
// the rank-2 update run as unrolled chains over 4-row groups entered at the group of row j + 1
// (a jump table on j), with 16-byte broadcast loads of (v, w) pairs.
constexpr int kPairWarps = 4;   // warps per block: two pairs, one matrix each

__host__ __device__ inline int pair_smem_floats(int k) {
    // load staging k x (k+1) | (v, w) [2][64] float2 | partial sums [2][8] | betas, taus [64]
    return round4(k * (k + 1)) + 2 * 64 * 2 + 16 + 64 + 64;
}

__device__ __forceinline__ void pair_sync(int id) {
    asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

template <int G>
__device__ __forceinline__ void tp_mv4(const float (&q)[64], const float4 *vw4, float (&p)[4]) {
    if constexpr (G < 16) {
        const float4 a = vw4[2 * G], b = vw4[2 * G + 1];
        p[0] = fmaf(q[4 * G], a.x, p[0]);
        p[1] = fmaf(q[4 * G + 1], a.z, p[1]);
        p[2] = fmaf(q[4 * G + 2], b.x, p[2]);
        p[3] = fmaf(q[4 * G + 3], b.z, p[3]);
    }
}

template <int G>
__device__ __forceinline__ void tp_up4(float (&q)[64], const float4 *vw4, float vt, float wt) {
    if constexpr (G < 16) {
        const float4 a = vw4[2 * G], b = vw4[2 * G + 1];
        q[4 * G] = fmaf(-a.x, wt, fmaf(-a.y, vt, q[4 * G]));
        q[4 * G + 1] = fmaf(-a.z, wt, fmaf(-a.w, vt, q[4 * G + 1]));
        q[4 * G + 2] = fmaf(-b.x, wt, fmaf(-b.y, vt, q[4 * G + 2]));
        q[4 * G + 3] = fmaf(-b.z, wt, fmaf(-b.w, vt, q[4 * G + 3]));
    }
}

#define LKP_CASE8(M, b) M(b) M(b + 1) M(b + 2) M(b + 3) M(b + 4) M(b + 5) M(b + 6) M(b + 7)
#define LKP_GROUPS16(M) LKP_CASE8(M, 0) LKP_CASE8(M, 8)
#define LKP_CASES64(M)                                                                      \
    LKP_CASE8(M, 0) LKP_CASE8(M, 8) LKP_CASE8(M, 16) LKP_CASE8(M, 24) LKP_CASE8(M, 32)      \
    LKP_CASE8(M, 40) LKP_CASE8(M, 48) LKP_CASE8(M, 56)

__global__ void __launch_bounds__(32 * kPairWarps, 5) eig_tridiag_pair_kernel(EigArgs a,
                                                                              EigSplit sp) {
    extern __shared__ float smem[];
    const int k = a.k;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int pair = wib >> 1, h = wib & 1, t = 32 * h + lane;
    float *S = smem + (size_t)pair * pair_smem_floats(k);
    float2 *vw = reinterpret_cast<float2 *>(S + round4(k * (k + 1)));  // [2][64], 16-byte aligned
    float *red = reinterpret_cast<float *>(vw + 128);             // [2][8]
    float *betas = red + 16, *taus_s = betas + 64;
    const int bar = 1 + pair;
    const int npairs = gridDim.x * (kPairWarps / 2);
    const int npts = a.list ? *a.list_count : a.npts;   // the chunk, or the listed points
    for (int it = blockIdx.x * (kPairWarps / 2) + pair; it < npts; it += npairs) {
        const int lp = a.list ? a.list[it] : it;
        if (a.nloc && a.nloc[lp] == 0) continue;   // the same decision for both warps
        float *Ag = a.gram + (size_t)lp * k * k;
        // ---- Q = diag + A, symmetrised from the upper triangle: warp h stages the row blocks
        // 8 (2 b + h) .. +7 with coalesced row loads (a measured 10 % faster than each lane
        // gathering its column from global memory), then every lane reads its column
        const int ld = k + 1;
        for (int i0 = 8 * h; i0 < k; i0 += 16) {
            float v[8][2];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = i0 + u, j = lane + 32 * c;
                    v[u][c] = (i < k && j < k) ? __ldcg(Ag + i * k + j) : 0.0f;
                }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = i0 + u, j = lane + 32 * c;
                    if (i < k && j < k && j >= i) {
                        S[i * ld + j] = v[u][c];
                        S[j * ld + i] = v[u][c];
                    }
                }
        }
        vw[t] = make_float2(0.0f, 0.0f);
        vw[64 + t] = make_float2(0.0f, 0.0f);
        pair_sync(bar);
        float q[64];
#pragma unroll
        for (int i = 0; i < 64; ++i)
            q[i] = (i < k && t < k) ? S[i * ld + t] + (i == t ? a.diag : 0.0f) : 0.0f;
        for (int j = 0; j < k - 2; ++j) {
            float2 *vwb = vw + (j & 1) * 64;
            float *rb = red + (j & 1) * 8;
            // x_t = Q'[t][j] = Q'[j][t] for t > j: the lane's own entry of row j
            float x = 0.0f;
            switch (j) {
#define LKP_PICK(i) \
    case i: x = q[i]; break;
                LKP_CASES64(LKP_PICK)
#undef LKP_PICK
                default: break;
            }
            if (t <= j || t >= k) x = 0.0f;
            const float tl = warp_sum(t > j + 1 ? x * x : 0.0f);
            if (lane == 0) rb[h] = tl;
            if (t == j + 1) rb[4] = x;
            pair_sync(bar);
            const float tail = rb[0] + rb[1], alpha = rb[4];
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
            const float vt = t > j + 1 ? x * scale : (t == j + 1 ? 1.0f : 0.0f);
            if (t > j && t < k) {
                vwb[t].x = vt;
                refl_row(Ag, k, j)[t - j - 1] = vt;  // lower triangle of the slot
            }
            const int g0 = (j + 1) >> 2;  // the group of row j + 1
            if (t >= 4 * g0 && t <= j) vwb[t] = make_float2(0.0f, 0.0f);
            if (t == 0) {
                taus_s[j] = tau;
                betas[j] = beta;
            }
            if (tau == 0.0f) continue;  // the same for both warps; x is already reduced
            pair_sync(bar);
            const float4 *vw4 = reinterpret_cast<const float4 *>(vwb);
            float p4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            switch (g0) {
#define LKP_MV4(G) \
    case G: tp_mv4<G>(q, vw4, p4);
                LKP_GROUPS16(LKP_MV4)
#undef LKP_MV4
                default: break;
            }
            const float p = ((p4[0] + p4[1]) + (p4[2] + p4[3])) * tau;
            const float kk = warp_sum(p * vt);
            if (lane == 0) rb[2 + h] = kk;
            pair_sync(bar);
            const float K = 0.5f * tau * (rb[2] + rb[3]);
            const float wt = t > j && t < k ? p - K * vt : 0.0f;
            if (t > j && t < k) vwb[t].y = wt;
            pair_sync(bar);
            switch (g0) {
#define LKP_UP4(G) \
    case G: tp_up4<G>(q, vw4, vt, wt);
                LKP_GROUPS16(LKP_UP4)
#undef LKP_UP4
                default: break;
            }
        }
        // ---- (d, e): d_t = Q'[t][t] (the lane's own diagonal), e_j = beta_j, e_{k-2} =
        // Q'[k-2][k-1]; the reflector scalars
        float dg = 0.0f, el = 0.0f;
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            if (i == t) dg = q[i];
            if (i == k - 2) el = q[i];
        }
        if (t == k - 1) betas[k - 2] = el;   // column k-1 holds Q'[k-2][k-1]
        pair_sync(bar);   // every beta and tau is written
        if (t < k) {
            sp.de[(size_t)lp * k + t] = make_float2(dg, t < k - 1 ? betas[t] : 0.0f);
            sp.taus[(size_t)lp * k + t] = t < k - 2 ? taus_s[t] : 0.0f;
        }
        pair_sync(bar);   // the next matrix's staging may overwrite S, betas and taus
    }
}
#undef LKP_CASES64
#undef LKP_GROUPS16
#undef LKP_CASE8

// (2) implicit-shift QL, thread per matrix: the recurrence of the fused schedule on (d, e)
// kept in shared memory as [index][thread] (the threads of a warp touch consecutive words),
// every rotation recorded.  Record of a point: per sweep a header (m, count) -- bit patterns
// of two ints -- then the sweep's (c, s) for i = m-1 down to m-count.
__global__ void __launch_bounds__(kQlThreads) eig_ql_kernel(EigArgs a, EigSplit sp) {
    extern __shared__ float2 des[];  // [k][kQlThreads]
    const int k = a.k, tid = threadIdx.x;
    const int lp0 = blockIdx.x * kQlThreads;
    const int lp = lp0 + tid;
    // the block's (d, e) arrays are contiguous in global memory: coalesced load
    const int nb = min(kQlThreads, a.npts - lp0);
    for (int e = tid; e < nb * k; e += kQlThreads) {
        const int p = e / k, i = e - p * k;
        des[i * kQlThreads + p] = sp.de[(size_t)lp0 * k + e];
    }
    __syncthreads();
    if (lp >= a.npts) return;
    if (a.nloc && a.nloc[lp] == 0) {
        for (int t = 0; t < k; ++t) a.eigval[(size_t)lp * k + t] = a.diag;
        if (sp.nrot) sp.nrot[lp] = 0;
        return;
    }
    float2 *D = des + tid;  // D[i * kQlThreads] = (d_i, e_i)
    constexpr int L = kQlThreads;
    // without a record buffer the kernel computes eigenvalues only (no record, no hand-off)
    const bool record = sp.rot != nullptr;
    float2 *rec = record ? sp.rot + (size_t)lp * sp.rcap : nullptr;
    const float eps = FLT_EPSILON;
    float tn = 0.0f;  // deflation threshold eps ||T||, as in the fused schedule
    for (int t = 0; t < k; ++t)
        tn = fmaxf(tn, fabsf(D[t * L].x) + fabsf(D[t * L].y) +
                           (t > 0 ? fabsf(D[(t - 1) * L].y) : 0.0f));
    const float tol = eps * tn;
    // QL as nested loops (per eigenvalue l: sweeps on [l, m] until e_l deflates).  The first
    // small coupling at or above l (m) is scanned for only when l advances without a known
    // one: a sweep compares the couplings it writes with the deflation threshold as it forms
    // them, which gives the next m (and, when e_l itself became small, the first small
    // coupling above l).  A flat single-loop form with the between-sweep work batched across
    // the warp measured 5 % slower at k = 32 and 3 % at k = 64.
    int pos = 0;
    bool notconv = false, overflow = false;
    int known = -1;  // first small coupling above l, found by the last sweep
    for (int l = 0; l < k && !overflow; ++l) {
        int iter = 0;
        int m = known >= l ? known : l;
        if (known < l)
            for (; m < k - 1; ++m)
                if (fabsf(D[m * L].y) <= tol) break;
        known = -1;
        while (m != l) {
            if (iter++ >= kMaxIter) {
                notconv = true;
                break;
            }
            if (record && pos + 1 + (m - l) > sp.rcap) {
                overflow = true;
                break;
            }
            // shift: eigenvalue of the leading 2 x 2 block nearer to d_l
            const float2 del = D[l * L];
            const float dl = del.x, el = del.y, dl1 = D[(l + 1) * L].x;
            const float th = (dl1 - dl) / (2.0f * el);
            const float rt = hypotf(th, 1.0f);
            float di1 = D[m * L].x;
            float g = di1 - dl + el / (th + copysignf(rt, th));
            float s = 1.0f, co = 1.0f, pacc = 0.0f;
            const int hdr = pos++;
            float2 dcur = D[(m - 1) * L];
            float ei = dcur.y, di = dcur.x;
            int sm = m;  // first small coupling in [l + 1, m] after this sweep
            int next = -1;
            for (int i = m - 1; i >= l; --i) {
                const float2 dnext = i > 0 ? D[(i - 1) * L] : make_float2(0.0f, 0.0f);
                const float f = s * ei, b = co * ei;
                const float ff = fmaf(f, f, g * g);
                if (ff < 1e-30f) {  // f and g vanish: the coupling has underflowed
                    D[(i + 1) * L] = make_float2(di1 - pacc, 0.0f);
                    D[m * L].y = 0.0f;
                    next = i + 1;  // e_l..e_i are as before the sweep (above the threshold)
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
                D[(i + 1) * L] = make_float2(g + pacc, enew);
                if (i + 1 < m && fabsf(enew) <= tol) sm = i + 1;
                g = co * r - b;
                if (record) rec[pos] = make_float2(co, s);
                ++pos;
                di1 = di;
                ei = dnext.y;
                di = dnext.x;
            }
            if (record) rec[hdr] = make_float2(__int_as_float(m), __int_as_float(pos - hdr - 1));
            if (next >= 0) {
                m = next;
            } else {
                D[l * L] = make_float2(di1 - pacc, g);
                D[m * L].y = 0.0f;
                if (fabsf(g) <= tol) {
                    known = sm;
                    m = l;
                } else {
                    m = sm;
                }
            }
        }
    }
    if (notconv) atomicOr(a.status, ST_NOTCONV);
    if (overflow) {  // handed to the fused kernel, which recomputes the point from A
        sp.nrot[lp] = -1;
        sp.list[atomicAdd(sp.list_count, 1)] = lp + sp.list_offset;
        return;
    }
    if (sp.nrot) sp.nrot[lp] = pos;
    for (int t = 0; t < k; ++t) a.eigval[(size_t)lp * k + t] = D[t * L].x;
}

// One 4-row group of a replay sweep with the lane's entries of Z in registers: the rotations
// of rows 4G+3, 4G+2, 4G+1, 4G in that order, row i turning rows i and i + 1 of Z (columns i,
// i + 1 of the eigenvector matrix) by (c, s) of cs[i]; pa, pb hold the group's four pairs.
// Rows of the group outside the sweep hold (1, 0), which leaves both rows exactly as they are.
template <int NC, int R>
__device__ __forceinline__ void replay_rot(float (&z)[NC][32 * NC], float co, float s) {
    if constexpr (R + 1 < 32 * NC) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float za = z[c][R], zb = z[c][R + 1];
            z[c][R + 1] = fmaf(s, za, co * zb);
            z[c][R] = fmaf(co, za, -(s * zb));
        }
    }
}

template <int NC, int G>
__device__ __forceinline__ void replay_group(float (&z)[NC][32 * NC], const float4 &pa,
                                             const float4 &pb) {
    if constexpr (4 * G < 32 * NC) {
        replay_rot<NC, 4 * G + 3>(z, pb.z, pb.w);
        replay_rot<NC, 4 * G + 2>(z, pb.x, pb.y);
        replay_rot<NC, 4 * G + 1>(z, pa.z, pa.w);
        replay_rot<NC, 4 * G>(z, pa.x, pa.y);
    }
}

// Replay of the recorded QL rotations onto Z = I with Z held in registers (k <= 64): the lane
// keeps its NC columns of the shared-memory image of Z, all 32 NC rows, so a rotation costs
// four multiply-adds per column and no shared-memory traffic for Z.  A sweep's rotations act
// on rows m-1, m-2, ..., m-cnt in that order.  For 33 <= k <= 64 the sweep enters an unrolled
// chain of 4-row groups at the group of row m-1 (a jump table) and leaves it after the group
// of row m-cnt, the rows of those two groups outside the sweep padded with identity
// rotations; the pairs are staged in shared memory by row (cs[row], rows 0..k+1) and read as
// 16-byte broadcast loads, one group ahead.  For k <= 32 (one column per lane) the chain goes
// row by row (GR = 1: no padding, an exit test per row, the pair two rows ahead in flight):
// measured 3 % faster there than groups of 2 or 4, and 4 % slower at k = 64.  Each sweep's record (header and pairs, at most 32 NC
// entries) is read as one window, one entry per lane and column, the next window's loads in
// flight while the current sweep runs.  Z is written to shared memory at the end.
template <int NC>
__device__ __forceinline__ void replay_in_registers(const float2 *__restrict__ rec, int nrec,
                                                    float *Z, float2 *cs, int k, int ld,
                                                    int lane) {
    constexpr int KM = 32 * NC;
    constexpr int GR = NC == 1 ? 1 : 4;   // rows per group
    constexpr int LG = GR == 1 ? 0 : 2;   // log2 GR
    static_assert(GR == 1 ? KM <= 64 : KM / GR <= 16, "the chains have 64 and 16 cases");
    float z[NC][KM];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int i = 0; i < KM; ++i) z[c][i] = i == lane + 32 * c ? 1.0f : 0.0f;
    const float4 *cs4 = reinterpret_cast<const float4 *>(cs);
    float2 win[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int idx = lane + 32 * c;
        win[c] = idx < nrec ? __ldcs(rec + idx) : make_float2(0.0f, 0.0f);
    }
    int pos = 0;
    while (pos < nrec) {
        const int m = __float_as_int(__shfl_sync(kFull, win[0].x, 0));
        const int cnt = __float_as_int(__shfl_sync(kFull, win[0].y, 0));
        const int next = pos + 1 + cnt;
        float2 nwin[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int idx = next + lane + 32 * c;
            nwin[c] = idx < nrec ? __ldcs(rec + idx) : make_float2(0.0f, 0.0f);
        }
        const bool valid = cnt > 0 && cnt <= m && m <= k - 1;  // as the QL kernel writes them
        const int lo = m - cnt;
        const int gt = (m - 1) >> LG, gb = lo >> LG;
        if (valid) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int r = lane + 32 * c - 1;  // window entry 1 + r is pair r
                if (r >= 0 && r < cnt) cs[m - 1 - r] = win[c];
            }
            // identity pads: rows GR gb .. lo-1 and m .. GR gt + GR - 1 (fewer than GR each)
            const int row = lane < GR ? GR * gb + lane : m + lane - GR;
            if ((lane < GR && row < lo) || (lane >= GR && lane < 2 * GR && row < GR * (gt + 1)))
                cs[row] = make_float2(1.0f, 0.0f);
        }
        __syncwarp();
        if (valid) {
            if constexpr (GR == 1) {
                float2 g0 = cs[m - 1], g1 = cs[m > 1 ? m - 2 : 0];
#define LK_REPLAY_ROW(i)                                  \
    case i: {                                             \
        const float2 g2 = cs[i > 1 ? i - 2 : 0];          \
        replay_rot<NC, i>(z, g0.x, g0.y);                 \
        if (i == lo) break;                               \
        g0 = g1;                                          \
        g1 = g2;                                          \
    }
#define LK_REPLAY_ROW8(b)                                                           \
    LK_REPLAY_ROW(b + 7) LK_REPLAY_ROW(b + 6) LK_REPLAY_ROW(b + 5) LK_REPLAY_ROW(b + 4) \
    LK_REPLAY_ROW(b + 3) LK_REPLAY_ROW(b + 2) LK_REPLAY_ROW(b + 1) LK_REPLAY_ROW(b)
                switch (m - 1) {
                    LK_REPLAY_ROW8(56) LK_REPLAY_ROW8(48) LK_REPLAY_ROW8(40) LK_REPLAY_ROW8(32)
                    LK_REPLAY_ROW8(24) LK_REPLAY_ROW8(16) LK_REPLAY_ROW8(8) LK_REPLAY_ROW8(0)
                    default: break;
                }
#undef LK_REPLAY_ROW8
#undef LK_REPLAY_ROW
            } else {
                // group G's four pairs: float4 2 G and 2 G + 1
                float4 pa = cs4[2 * gt], pb = cs4[2 * gt + 1];
#define LK_REPLAY_GROUP(G)                          \
    case G: {                                       \
        const float4 na = cs4[G > 0 ? 2 * G - 2 : 0]; \
        const float4 nb = cs4[G > 0 ? 2 * G - 1 : 1]; \
        replay_group<NC, G>(z, pa, pb);             \
        if (G == gb) break;                         \
        pa = na;                                    \
        pb = nb;                                    \
    }
                switch (gt) {
                    LK_REPLAY_GROUP(15) LK_REPLAY_GROUP(14) LK_REPLAY_GROUP(13) LK_REPLAY_GROUP(12)
                    LK_REPLAY_GROUP(11) LK_REPLAY_GROUP(10) LK_REPLAY_GROUP(9) LK_REPLAY_GROUP(8)
                    LK_REPLAY_GROUP(7) LK_REPLAY_GROUP(6) LK_REPLAY_GROUP(5) LK_REPLAY_GROUP(4)
                    LK_REPLAY_GROUP(3) LK_REPLAY_GROUP(2) LK_REPLAY_GROUP(1) LK_REPLAY_GROUP(0)
                    default: break;
                }
#undef LK_REPLAY_GROUP
            }
        }
        __syncwarp();
        pos = next;
#pragma unroll
        for (int c = 0; c < NC; ++c) win[c] = nwin[c];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int t = lane + 32 * c;
#pragma unroll
        for (int i = 0; i < KM; ++i)
            if (i < k && t < k) Z[i * ld + t] = z[c][i];
    }
    __syncwarp();
}

// (3) vectors, transform and update, warp per matrix: Z = I, the recorded rotations replayed
// onto Z, V = H Z, then the fused schedule's transform and update (kUpdate; without it, the
// eigenpairs only, for letkf_eigh_batch_ws: a separate instantiation, so that the analysis
// path carries no extra registers).
template <int NC, bool kUpdate>
__global__ void __launch_bounds__(32 * EigCfg<NC>::WARPS, EigCfg<NC>::MINB_VEC)
    eig_vec_kernel(EigArgs a, EigSplit sp) {
    extern __shared__ float smem[];
    const int k = a.k, ld = k + 1;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *vtmp = smem + (size_t)wib * vec_smem_floats(k);
    float *Z = vtmp + vec_stage_floats(k);
    float *B = Z + k * ld;
    float *taus = B + kRows * ld;
    const int warps_per_block = blockDim.x >> 5;
    const int nw = gridDim.x * warps_per_block;
    for (int lp = blockIdx.x * warps_per_block + wib; lp < a.npts; lp += nw) {
        const int nrec = sp.nrot[lp];
        if (a.nloc && a.nloc[lp] == 0) {  // no local observation: Q = (k-1)/rho I
            if constexpr (kUpdate) inflate_point(a, lp, lane);
            continue;
        }
        if (nrec < 0) continue;  // recomputed by the fused kernel
        float *Ag = a.gram + (size_t)lp * k * k;
        float xbar[NV];
        float *X = kUpdate ? load_forecast<NC>(a, lp, B, k, ld, lane, xbar) : nullptr;
        for (int t = lane; t < k; t += 32) taus[t] = sp.taus[(size_t)lp * k + t];
        const float2 *rec = sp.rot + (size_t)lp * sp.rcap;
        if constexpr (NC <= 2) {
            replay_in_registers<NC>(rec, nrec, Z, reinterpret_cast<float2 *>(vtmp), k, ld, lane);
        } else {
            set_identity<NC>(Z, k, ld, lane);
            // replay: the record is read 32 entries at a time, one per lane, and each entry is
            // broadcast from its lane
            int wbase = 0;
            float2 win = lane < nrec ? __ldcs(rec + lane) : make_float2(0.0f, 0.0f);
            auto entry = [&](int idx) -> float2 {
                if (idx - wbase >= 32) {
                    wbase = idx;
                    win = idx + lane < nrec ? __ldcs(rec + idx + lane) : make_float2(0.0f, 0.0f);
                }
                const int src = idx - wbase;
                return make_float2(__shfl_sync(kFull, win.x, src), __shfl_sync(kFull, win.y, src));
            };
            int pos = 0;
            while (pos < nrec) {
                const float2 h = entry(pos++);
                const int m = __float_as_int(h.x), cnt = __float_as_int(h.y);
                float zc[NC];  // carried column entries of row i+1 of Z
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int t = lane + 32 * c;
                    zc[c] = t < k ? Z[m * ld + t] : 0.0f;
                }
                float *zp = Z + (m - 1) * ld + lane;
                for (int r = 0; r < cnt; ++r) {
                    const float2 cs = entry(pos++);
                    const float co = cs.x, s = cs.y;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        if (lane + 32 * c < k) {
                            const float za = zp[32 * c];
                            zp[ld + 32 * c] = s * za + co * zc[c];
                            zc[c] = co * za - s * zc[c];
                        }
                    }
                    zp -= ld;
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int t = lane + 32 * c;
                    if (t < k) Z[(m - cnt) * ld + t] = zc[c];
                }
            }
        }
        __syncwarp();
        float dr[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = lane + 32 * c;
            dr[c] = t < k ? a.eigval[(size_t)lp * k + t] : 1.0f;
        }
        if constexpr (NC <= 2)
            back_transform_registers<NC>(Ag, Z, taus, vtmp, k, ld, lane);
        else
            back_transform<NC>(Ag, Z, taus, vtmp, k, ld, lane);
        if (a.refine) {
            refine_clusters<NC>(Z, ld, Ag, a.diag, k, dr, lane, a.refine_tau);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int t = lane + 32 * c;
                if (t < k) a.eigval[(size_t)lp * k + t] = dr[c];
            }
        }
        if (a.evec) store_vectors<NC>(Z, ld, a.evec + (size_t)lp * k * k, k, lane);
        if constexpr (kUpdate) transform_update<NC>(X, B, Z, dr, xbar, k, ld, lane, a.status);
    }
}

// The dynamic shared-memory cap of a kernel is a process-wide attribute shared by every
// handle: it is set for the largest k the kernel's template serves (the shared memory grows
// with k), never for one handle's k, so that no handle can lower it under another's launch.
template <int NC>
cudaError_t occupancy(const void *kern, int warps, size_t smem, size_t smem_cap,
                      int *max_blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_cap)) != cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *max_blocks = sms * per_sm;
    return cudaSuccess;
}

constexpr int kmax_of(int nc) { return 32 * nc; }  // largest k of an NC instantiation

template <int NC>
cudaError_t prepare_nc(int k, int *max_blocks) {
    const int warps = EigCfg<NC>::WARPS;
    return occupancy<NC>((const void *)eigen_update_kernel<NC>, warps,
                         (size_t)smem_floats(k) * sizeof(float) * warps,
                         (size_t)smem_floats(kmax_of(NC)) * sizeof(float) * warps, max_blocks);
}

template <int NC>
cudaError_t prepare_split_nc(int k, EigSplit *sp) {
    const int warps = EigCfg<NC>::WARPS;
    cudaError_t e;
    if constexpr (NC == 2) {  // the pair kernel (two matrices per block)
        e = cudaFuncSetAttribute((const void *)eig_tridiag_pair_kernel,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        e = occupancy<NC>((const void *)eig_tridiag_pair_kernel, kPairWarps,
                          (size_t)pair_smem_floats(k) * sizeof(float) * (kPairWarps / 2),
                          (size_t)pair_smem_floats(64) * sizeof(float) * (kPairWarps / 2),
                          &sp->grid_tri);
    } else
        e = occupancy<NC>((const void *)eig_tridiag_kernel<NC>, warps,
                          (size_t)tri_smem_floats(k) * sizeof(float) * warps,
                          (size_t)tri_smem_floats(kmax_of(NC)) * sizeof(float) * warps,
                          &sp->grid_tri);
    if (e != cudaSuccess) return e;
    e = occupancy<NC>((const void *)eig_vec_kernel<NC, true>, warps,
                      (size_t)vec_smem_floats(k) * sizeof(float) * warps,
                      (size_t)vec_smem_floats(kmax_of(NC)) * sizeof(float) * warps,
                      &sp->grid_vec);
    if (e != cudaSuccess) return e;
    int unused = 0;
    e = occupancy<NC>((const void *)eig_vec_kernel<NC, false>, warps,
                      (size_t)vec_smem_floats(k) * sizeof(float) * warps,
                      (size_t)vec_smem_floats(kmax_of(NC)) * sizeof(float) * warps, &unused);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(eig_ql_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(128 * kQlThreads * sizeof(float2)));
}

unsigned grid_for(int max_blocks, long long npts, int warps) {
    long long need = (npts + warps - 1) / warps;
    long long blocks = max_blocks > 0 ? max_blocks : 1;
    return (unsigned)(blocks > need ? need : blocks);
}

template <int NC>
cudaError_t launch_nc(const EigArgs &a, cudaStream_t s) {
    const int warps = EigCfg<NC>::WARPS;
    const size_t smem = (size_t)smem_floats(a.k) * sizeof(float) * warps;
    eigen_update_kernel<NC><<<grid_for(a.max_blocks, a.npts, warps), 32 * warps, smem, s>>>(a);
    return cudaGetLastError();
}

// The points [p0, p0 + n) of a chunk as a chunk of their own (the same buffers, offset).
void split_part(const EigArgs &a, const EigSplit &sp, int p0, int n, EigArgs *b, EigSplit *c) {
    const size_t k = (size_t)a.k, o = (size_t)p0;
    *b = a;
    *c = sp;
    b->npts = n;
    b->pt0 = a.pt0 + p0;
    b->gram = a.gram + o * k * k;
    b->cvec = a.cvec ? a.cvec + o * k : nullptr;
    b->nloc = a.nloc ? a.nloc + o : nullptr;
    b->eigval = a.eigval + o * k;
    b->evec = a.evec ? a.evec + o * k * k : nullptr;
    c->de = sp.de + o * k;
    c->taus = sp.taus + o * k;
    c->rot = sp.rot + o * (size_t)sp.rcap;
    c->nrot = sp.nrot + o;
    c->list_offset = sp.list_offset + p0;
}

template <int NC>
void launch_tri(const EigArgs &a, const EigSplit &sp, cudaStream_t s) {
    if constexpr (NC == 2) {  // 33 <= k <= 64: a pair of warps per matrix, Q in registers
        constexpr int pairs = kPairWarps / 2;
        eig_tridiag_pair_kernel<<<grid_for(sp.grid_tri, a.npts, pairs), 32 * kPairWarps,
                                  (size_t)pair_smem_floats(a.k) * sizeof(float) * pairs, s>>>(a,
                                                                                          sp);
        return;
    }
    const int warps = EigCfg<NC>::WARPS;
    eig_tridiag_kernel<NC><<<grid_for(sp.grid_tri, a.npts, warps), 32 * warps,
                             (size_t)tri_smem_floats(a.k) * sizeof(float) * warps, s>>>(a, sp);
}

void launch_ql(const EigArgs &a, const EigSplit &sp, cudaStream_t s) {
    eig_ql_kernel<<<(unsigned)((a.npts + kQlThreads - 1) / kQlThreads), kQlThreads,
                    (size_t)a.k * kQlThreads * sizeof(float2), s>>>(a, sp);
}

template <int NC>
void launch_vec(const EigArgs &a, const EigSplit &sp, cudaStream_t s) {
    const int warps = EigCfg<NC>::WARPS;
    if (a.x)
        eig_vec_kernel<NC, true><<<grid_for(sp.grid_vec, a.npts, warps), 32 * warps,
                                   (size_t)vec_smem_floats(a.k) * sizeof(float) * warps, s>>>(a,
                                                                                         sp);
    else
        eig_vec_kernel<NC, false><<<grid_for(sp.grid_vec, a.npts, warps), 32 * warps,
                                    (size_t)vec_smem_floats(a.k) * sizeof(float) * warps, s>>>(a,
                                                                                          sp);
}

// Chunks below this many points run on one stream: their halves would not fill the GPU.  The
// overlap is used for k <= 32, where it measured 11 % faster (256^2); at k = 64 (1024^2) it
// measured 1 % slower: there the vector kernel is limited by shared memory and shares the SMs
// with the QL blocks.
constexpr int kSplitOverlapMin = 16384;

template <int NC>
cudaError_t launch_split_nc(const EigArgs &a, const EigSplit &sp, cudaStream_t s,
                            cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join) {
    const int warps = EigCfg<NC>::WARPS;
    cudaError_t e = cudaMemsetAsync(sp.list_count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (NC == 1 && s2 && fork && join && a.npts >= kSplitOverlapMin) {
        // halves h0, h1: s runs tri(h0), QL(h0), vec(h0); s2 starts after tri(h0) and runs
        // tri(h1), QL(h1), vec(h1); s waits for s2 before the hand-off kernel
        const int n0 = (a.npts / 2 + kQlThreads - 1) / kQlThreads * kQlThreads;
        EigArgs a0, a1;
        EigSplit p0, p1;
        split_part(a, sp, 0, n0, &a0, &p0);
        split_part(a, sp, n0, a.npts - n0, &a1, &p1);
        launch_tri<NC>(a0, p0, s);
        if ((e = cudaEventRecord(fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s2, fork, 0)) != cudaSuccess) return e;
        launch_ql(a0, p0, s);
        launch_tri<NC>(a1, p1, s2);
        launch_ql(a1, p1, s2);
        launch_vec<NC>(a0, p0, s);
        launch_vec<NC>(a1, p1, s2);
        if ((e = cudaEventRecord(join, s2)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, join, 0)) != cudaSuccess) return e;
    } else {
        launch_tri<NC>(a, sp, s);
        launch_ql(a, sp, s);
        launch_vec<NC>(a, sp, s);
    }
    // matrices whose rotation record overflowed: the fused kernel over the list
    EigArgs f = a;
    f.list = sp.list;
    f.list_count = sp.list_count;
    eigen_update_kernel<NC><<<grid_for(a.max_blocks, a.npts, warps), 32 * warps,
                              (size_t)smem_floats(a.k) * sizeof(float) * warps, s>>>(f);
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

cudaError_t eigen_split_prepare(int k, EigSplit *sp) {
    if (k <= 32) return prepare_split_nc<1>(k, sp);
    if (k <= 64) return prepare_split_nc<2>(k, sp);
    if (k <= 128) return prepare_split_nc<4>(k, sp);
    return cudaErrorInvalidValue;
}

cudaError_t launch_eigen_update(const EigArgs &a, cudaStream_t s) {
    if (a.npts <= 0) return cudaSuccess;
    if (a.k <= 32) return launch_nc<1>(a, s);
    if (a.k <= 64) return launch_nc<2>(a, s);
    if (a.k <= 128) return launch_nc<4>(a, s);
    return cudaErrorInvalidValue;
}

template <int NC>
cudaError_t launch_group_nc(EigGroup &g, int max_blocks, cudaStream_t s) {
    const int warps = EigCfg<NC>::WARPS;
    const size_t smem = (size_t)smem_floats(g.kmax) * sizeof(float) * warps;
    cudaError_t e = cudaMemsetAsync(g.counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    eigen_group_kernel<NC><<<grid_for(max_blocks, g.start[g.n], warps), 32 * warps, smem, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_eigen_group(const EigArgs *segs, int n, int *counters, const int *max_blocks,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (n > kMaxGroupSeg * 3) return cudaErrorInvalidValue;
    // one launch per column class, segments by decreasing k
    for (int cls = 0; cls < 3; ++cls) {
        const int lo = cls == 0 ? 2 : (cls == 1 ? 33 : 65), hi = 32 << cls;
        EigGroup g;
        g.n = 0;
        g.kmax = 0;
        g.start[0] = 0;
        g.counter = counters + cls;
        int order[kMaxGroupSeg * 3], m = 0;
        for (int i = 0; i < n; ++i)
            if (segs[i].k >= lo && segs[i].k <= hi && segs[i].npts > 0) order[m++] = i;
        if (m == 0) continue;
        if (m > kMaxGroupSeg) return cudaErrorInvalidValue;
        std::sort(order, order + m, [&](int x, int y) { return segs[x].k > segs[y].k; });
        for (int j = 0; j < m; ++j) {
            g.seg[j] = segs[order[j]];
            g.kmax = std::max(g.kmax, g.seg[j].k);
            g.start[j + 1] = g.start[j] + g.seg[j].npts;
        }
        g.n = m;
        const cudaError_t e = cls == 0 ? launch_group_nc<1>(g, max_blocks[0], s)
                            : cls == 1 ? launch_group_nc<2>(g, max_blocks[1], s)
                                       : launch_group_nc<4>(g, max_blocks[2], s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t eigen_group_prepare(int *max_blocks) {
    cudaError_t e = occupancy<1>((const void *)eigen_group_kernel<1>, EigCfg<1>::WARPS,
                                 (size_t)smem_floats(32) * sizeof(float) * EigCfg<1>::WARPS,
                                 (size_t)smem_floats(32) * sizeof(float) * EigCfg<1>::WARPS,
                                 &max_blocks[0]);
    if (e == cudaSuccess)
        e = occupancy<2>((const void *)eigen_group_kernel<2>, EigCfg<2>::WARPS,
                         (size_t)smem_floats(64) * sizeof(float) * EigCfg<2>::WARPS,
                         (size_t)smem_floats(64) * sizeof(float) * EigCfg<2>::WARPS,
                         &max_blocks[1]);
    if (e == cudaSuccess)
        e = occupancy<4>((const void *)eigen_group_kernel<4>, EigCfg<4>::WARPS,
                         (size_t)smem_floats(128) * sizeof(float) * EigCfg<4>::WARPS,
                         (size_t)smem_floats(128) * sizeof(float) * EigCfg<4>::WARPS,
                         &max_blocks[2]);
    return e;
}

template <int NC>
cudaError_t launch_rational_nc(const EigArgs &a, const EigSplit &sp, int grid, cudaStream_t s) {
    const int warps = EigCfg<NC>::WARPS;
    cudaError_t e = cudaMemsetAsync(sp.list_count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    EigArgs t = a;   // eigenvalues asked for: every point of the chunk is tridiagonalized
    if (a.eigval) {
        t.list = nullptr;
        t.list_count = nullptr;
    }
    launch_tri<NC>(t, sp, s);
    if (a.eigval) {  // eigenvalues for a caller that asked for them: the QL without a record
        EigSplit v = sp;
        v.rot = nullptr;
        v.nrot = nullptr;
        launch_ql(t, v, s);
    }
    if ((e = launch_eigen_rational_transform(a, sp, grid, s)) != cudaSuccess) return e;
    EigArgs f = a;  // points beyond the approximations' range: the fused kernel
    f.list = sp.list;
    f.list_count = sp.list_count;
    eigen_update_kernel<NC><<<grid_for(a.max_blocks, a.npts, warps), 32 * warps,
                              (size_t)smem_floats(a.k) * sizeof(float) * warps, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_eigen_rational(const EigArgs &a, const EigSplit &sp, int grid,
                                  cudaStream_t s) {
    if (a.npts <= 0) return cudaSuccess;
    if (!sp.de || !sp.taus || !sp.list || !sp.list_count || !a.x || !a.cvec)
        return cudaErrorInvalidValue;
    if (a.k <= 32) return launch_rational_nc<1>(a, sp, grid, s);
    if (a.k <= kRationalMaxK) return launch_rational_nc<2>(a, sp, grid, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_eigen_chebyshev(const EigArgs &a, const EigSplit &sp, int cheb_grid,
                                   int rat_grid, cudaStream_t s) {
    if (a.npts <= 0) return cudaSuccess;
    if (!sp.de || !sp.taus || !sp.list || !sp.list_count || !sp.pre_list || !sp.pre_count ||
        !a.x || !a.cvec || a.list)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(sp.pre_count, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_eigen_cheb_transform(a, sp, cheb_grid, s);
    if (e != cudaSuccess) return e;
    EigArgs r = a;   // the points beyond the Chebyshev sets: the rational schedule
    r.list = sp.pre_list;
    r.list_count = sp.pre_count;
    if (a.k <= 32) return launch_rational_nc<1>(r, sp, rat_grid, s);
    if (a.k <= kChebMaxK) return launch_rational_nc<2>(r, sp, rat_grid, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_eigen_split(const EigArgs &a, const EigSplit &sp, cudaStream_t s,
                               cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join) {
    if (a.npts <= 0) return cudaSuccess;
    if (!a.eigval || !sp.de || !sp.taus || !sp.rot || !sp.nrot || !sp.list || !sp.list_count)
        return cudaErrorInvalidValue;
    if (a.k <= 32) return launch_split_nc<1>(a, sp, s, s2, fork, join);
    if (a.k <= 64) return launch_split_nc<2>(a, sp, s, s2, fork, join);
    if (a.k <= 128) return launch_split_nc<4>(a, sp, s, s2, fork, join);
    return cudaErrorInvalidValue;
}

}  // namespace lk
