// Layout change between the LBM and the LETKF (Sec. IV-A).
//
// The LBM keeps member-major structure of arrays g[m][q][p]; the batched local
// problems want the batch (grid point) outermost, x[p][q][m], so that the 9 x k
// block of one grid point is contiguous (the paper's X^f[N_x, M, N_v] ordering,
// with populations before members).  For each population q this is a k x N
// transpose, staged through a 32 x 33 shared-memory tile so that both the
// read (along p) and the write (along m) are coalesced (16-byte accesses where k and
// the point count are multiples of 4).  HBM bound: 2 x 36 k bytes per grid point.
#include "common.cuh"
#include "kernels.h"

namespace lk {
namespace {

__global__ void __launch_bounds__(256) transpose_in_kernel(const float *__restrict__ g,
                                                           float *__restrict__ x, int k,
                                                           size_t npts) {
    __shared__ float tile[32][33];
    const size_t p0 = (size_t)blockIdx.x * 32;
    const int m0 = blockIdx.y * 32;
    const int q = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = ty; i < 32; i += 8) {
        const int m = m0 + i;
        const size_t p = p0 + tx;
        if (m < k && p < npts) tile[i][tx] = __ldcs(g + ((size_t)m * NV + q) * npts + p);
    }
    __syncthreads();
#pragma unroll
    for (int i = ty; i < 32; i += 8) {
        const size_t p = p0 + i;
        const int m = m0 + tx;
        if (m < k && p < npts) __stcs(x + (p * NV + q) * k + m, tile[tx][i]);
    }
}

__global__ void __launch_bounds__(256) transpose_out_kernel(const float *__restrict__ x,
                                                            float *__restrict__ g, int k,
                                                            size_t npts) {
    __shared__ float tile[32][33];
    const size_t p0 = (size_t)blockIdx.x * 32;
    const int m0 = blockIdx.y * 32;
    const int q = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = ty; i < 32; i += 8) {
        const size_t p = p0 + i;
        const int m = m0 + tx;
        if (m < k && p < npts) tile[tx][i] = __ldcs(x + (p * NV + q) * k + m);
    }
    __syncthreads();
#pragma unroll
    for (int i = ty; i < 32; i += 8) {
        const int m = m0 + i;
        const size_t p = p0 + tx;
        if (m < k && p < npts) __stcs(g + ((size_t)m * NV + q) * npts + p, tile[i][tx]);
    }
}

// 16-byte form (k and npts multiples of 4): a 64-point x 32-member tile per block, float4
// loads along the contiguous axis of the source and float4 stores along that of the
// destination, through a [32][65] shared tile.
constexpr int kVP = 64, kVM = 32;

__global__ void __launch_bounds__(256) transpose_in_vec_kernel(const float *__restrict__ g,
                                                               float *__restrict__ x, int k,
                                                               size_t npts) {
    __shared__ float tile[kVM][kVP + 1];
    const size_t p0 = (size_t)blockIdx.x * kVP;
    const int m0 = blockIdx.y * kVM;
    const int q = blockIdx.z;
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 2; ++i) {   // member m, points 4 p4 .. 4 p4 + 3
        const int m = t / 16 + 16 * i, p4 = t % 16;
        const size_t p = p0 + 4 * p4;
        if (m0 + m < k && p < npts) {
            const float4 v = __ldcs(reinterpret_cast<const float4 *>(
                g + ((size_t)(m0 + m) * NV + q) * npts + p));
            tile[m][4 * p4] = v.x;
            tile[m][4 * p4 + 1] = v.y;
            tile[m][4 * p4 + 2] = v.z;
            tile[m][4 * p4 + 3] = v.w;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2; ++i) {   // point p, members 4 m4 .. 4 m4 + 3
        const int pl = t / 8 + 32 * i, m4 = t % 8;
        const size_t p = p0 + pl;
        const int m = m0 + 4 * m4;
        if (m < k && p < npts)
            __stcs(reinterpret_cast<float4 *>(x + (p * NV + q) * k + m),
                   make_float4(tile[4 * m4][pl], tile[4 * m4 + 1][pl], tile[4 * m4 + 2][pl],
                               tile[4 * m4 + 3][pl]));
    }
}

__global__ void __launch_bounds__(256) transpose_out_vec_kernel(const float *__restrict__ x,
                                                                float *__restrict__ g, int k,
                                                                size_t npts) {
    __shared__ float tile[kVM][kVP + 1];
    const size_t p0 = (size_t)blockIdx.x * kVP;
    const int m0 = blockIdx.y * kVM;
    const int q = blockIdx.z;
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 2; ++i) {   // point p, members 4 m4 .. 4 m4 + 3
        const int pl = t / 8 + 32 * i, m4 = t % 8;
        const size_t p = p0 + pl;
        const int m = m0 + 4 * m4;
        if (m < k && p < npts) {
            const float4 v =
                __ldcs(reinterpret_cast<const float4 *>(x + (p * NV + q) * k + m));
            tile[4 * m4][pl] = v.x;
            tile[4 * m4 + 1][pl] = v.y;
            tile[4 * m4 + 2][pl] = v.z;
            tile[4 * m4 + 3][pl] = v.w;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2; ++i) {   // member m, points 4 p4 .. 4 p4 + 3
        const int m = t / 16 + 16 * i, p4 = t % 16;
        const size_t p = p0 + 4 * p4;
        if (m0 + m < k && p < npts)
            __stcs(reinterpret_cast<float4 *>(g + ((size_t)(m0 + m) * NV + q) * npts + p),
                   make_float4(tile[m][4 * p4], tile[m][4 * p4 + 1], tile[m][4 * p4 + 2],
                               tile[m][4 * p4 + 3]));
    }
}

}  // namespace

cudaError_t launch_transpose_in(const float *g, float *x, int k, size_t npts, cudaStream_t s) {
    if (npts == 0 || k <= 0) return cudaSuccess;
    if ((k & 3) == 0 && (npts & 3) == 0) {
        dim3 grid((unsigned)((npts + kVP - 1) / kVP), (k + kVM - 1) / kVM, NV);
        transpose_in_vec_kernel<<<grid, 256, 0, s>>>(g, x, k, npts);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((npts + 31) / 32), (k + 31) / 32, NV);
    transpose_in_kernel<<<grid, dim3(32, 8), 0, s>>>(g, x, k, npts);
    return cudaGetLastError();
}

cudaError_t launch_transpose_out(const float *x, float *g, int k, size_t npts, cudaStream_t s) {
    if (npts == 0 || k <= 0) return cudaSuccess;
    if ((k & 3) == 0 && (npts & 3) == 0) {
        dim3 grid((unsigned)((npts + kVP - 1) / kVP), (k + kVM - 1) / kVM, NV);
        transpose_out_vec_kernel<<<grid, 256, 0, s>>>(x, g, k, npts);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((npts + 31) / 32), (k + 31) / 32, NV);
    transpose_out_kernel<<<grid, dim3(32, 8), 0, s>>>(x, g, k, npts);
    return cudaGetLastError();
}

}  // namespace lk
