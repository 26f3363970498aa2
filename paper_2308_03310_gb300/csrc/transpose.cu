// Layout change between the LBM and the LETKF (Sec. IV-A).
//
// The LBM keeps member-major structure of arrays g[m][q][p]; the batched local
// problems want the batch (grid point) outermost, x[p][q][m], so that the 9 x k
// block of one grid point is contiguous (the paper's X^f[N_x, M, N_v] ordering,
// with populations before members).  For each population q this is a k x N
// transpose, staged through a 32 x 33 shared-memory tile so that both the
// read (along p) and the write (along m) are coalesced.  HBM bound: 2 x 36 k
// bytes per grid point.
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

}  // namespace

cudaError_t launch_transpose_in(const float *g, float *x, int k, size_t npts, cudaStream_t s) {
    if (npts == 0 || k <= 0) return cudaSuccess;
    dim3 grid((unsigned)((npts + 31) / 32), (k + 31) / 32, NV);
    transpose_in_kernel<<<grid, dim3(32, 8), 0, s>>>(g, x, k, npts);
    return cudaGetLastError();
}

cudaError_t launch_transpose_out(const float *x, float *g, int k, size_t npts, cudaStream_t s) {
    if (npts == 0 || k <= 0) return cudaSuccess;
    dim3 grid((unsigned)((npts + 31) / 32), (k + 31) / 32, NV);
    transpose_out_kernel<<<grid, dim3(32, 8), 0, s>>>(x, g, k, npts);
    return cudaGetLastError();
}

}  // namespace lk
