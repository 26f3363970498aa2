// Batched ensemble D2Q9 lattice Boltzmann kernels (Sec. II-A).
//
// One time step of Eq. 1 for every member at once: each thread reads the nine
// populations of one node of one member, forms the moments (Eqs. 2-3), applies
// the BGK relaxation towards the second-order D2Q9 equilibrium plus the body-force
// source F_q = 3 w_q c_q . F, and pushes each post-collision population to the
// neighbour x + c_q (periodic).  The stored state is the post-streaming f.
//
// Layout: member-major structure of arrays g[m][q][y][x] (the paper's LBM layout
// X[m, N_v, N_x], Sec. IV-A), FP32, holding the deviation g_q = f_q - w_q from the
// rest state (exact weights).  Every load and store is a coalesced 4-byte access of a warp along x;
// the kernel moves 72 bytes per lattice update and is HBM bound.
#include "common.cuh"
#include "kernels.h"

namespace lk {
namespace {

template <bool kForce>
__global__ void __launch_bounds__(256) lbm_step_kernel(const float *__restrict__ gin,
                                                       float *__restrict__ gout,
                                                       const float2 *__restrict__ force,
                                                       int nx, int ny, float omega) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const size_t npts = (size_t)nx * ny;
    const size_t mbase = (size_t)blockIdx.z * NV * npts;
    const size_t p = (size_t)y * nx + x;

    float g[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) g[q] = __ldcs(gin + mbase + q * npts + p);

    // density and momentum of the deviation from rest
    float drho = 0.0f, jx = 0.0f, jy = 0.0f;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        drho += g[q];
        if (cx(q) != 0) jx += cx(q) > 0 ? g[q] : -g[q];
        if (cy(q) != 0) jy += cy(q) > 0 ? g[q] : -g[q];
    }
    const float rho = 1.0f + drho;
    const float rinv = 1.0f / rho;
    const float ux = jx * rinv, uy = jy * rinv;
    const float usq = 1.5f * (ux * ux + uy * uy);
    float fx = 0.0f, fy = 0.0f;
    if (kForce) {
        const float2 F = __ldg(force + p);
        fx = F.x;
        fy = F.y;
    }
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    float *dst = gout + mbase;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const float cu = (float)cx(q) * ux + (float)cy(q) * uy;
        const float geq = wq(q) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - usq));
        float gs = g[q] - omega * (g[q] - geq);
        if (kForce) gs += 3.0f * wq(q) * ((float)cx(q) * fx + (float)cy(q) * fy);
        const int xd = cx(q) < 0 ? xm : (cx(q) > 0 ? xp : x);
        const int yd = cy(q) < 0 ? ym : (cy(q) > 0 ? yp : y);
        __stcs(dst + q * npts + (size_t)yd * nx + xd, gs);
    }
}

// f -> g = (f - fl(w_q)) - dw_q and g -> f = fl(w_q) + (g + dw_q).
template <bool kToG>
__global__ void shift_kernel(const float *__restrict__ in, float *__restrict__ out, size_t npts) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    const int q = blockIdx.y % NV;
    const size_t off = (size_t)blockIdx.y * npts + i;
    const int cls = q == 4 ? 4 : ((q & 1) ? 1 : 0);
    const float w = wq(cls), dw = dwq(cls);
    out[off] = kToG ? __fsub_rn(__fsub_rn(in[off], w), dw) : __fadd_rn(w, __fadd_rn(in[off], dw));
}

// g_q = f^eq_q(rho, u) - w_q = w_q ((rho - 1) + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)).
__global__ void macro_kernel(const float *__restrict__ rho, const float *__restrict__ ux,
                             const float *__restrict__ uy, float *__restrict__ g, size_t npts) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    const size_t m = blockIdx.y;
    const float r = rho[m * npts + i], u = ux[m * npts + i], v = uy[m * npts + i];
    const float dr = r - 1.0f;
    const float usq = 1.5f * (u * u + v * v);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const float cu = (float)cx(q) * u + (float)cy(q) * v;
        g[(m * NV + q) * npts + i] = wq(q) * (dr + r * (3.0f * cu + 4.5f * cu * cu - usq));
    }
}

}  // namespace

cudaError_t launch_lbm_step(const float *gin, float *gout, const float2 *force, int nx, int ny,
                            int nmem, float tau, cudaStream_t s) {
    if (nmem <= 0) return cudaSuccess;
    const int bx = nx >= 128 ? 128 : ((nx + 31) / 32) * 32;
    const int by = 256 / bx;
    dim3 block(bx, by);
    dim3 grid((nx + bx - 1) / bx, (ny + by - 1) / by, nmem);
    const float omega = 1.0f / tau;
    if (force)
        lbm_step_kernel<true><<<grid, block, 0, s>>>(gin, gout, force, nx, ny, omega);
    else
        lbm_step_kernel<false><<<grid, block, 0, s>>>(gin, gout, force, nx, ny, omega);
    return cudaGetLastError();
}

cudaError_t launch_f_to_g(const float *f, float *g, int nmem, size_t npts, cudaStream_t s) {
    if (nmem <= 0 || npts == 0) return cudaSuccess;
    dim3 grid((unsigned)((npts + 255) / 256), nmem * NV);
    shift_kernel<true><<<grid, 256, 0, s>>>(f, g, npts);
    return cudaGetLastError();
}

cudaError_t launch_g_to_f(const float *g, float *f, int nmem, size_t npts, cudaStream_t s) {
    if (nmem <= 0 || npts == 0) return cudaSuccess;
    dim3 grid((unsigned)((npts + 255) / 256), nmem * NV);
    shift_kernel<false><<<grid, 256, 0, s>>>(g, f, npts);
    return cudaGetLastError();
}

cudaError_t launch_macro_to_g(const float *rho, const float *ux, const float *uy, float *g,
                              int nmem, size_t npts, cudaStream_t s) {
    if (nmem <= 0 || npts == 0) return cudaSuccess;
    dim3 grid((unsigned)((npts + 255) / 256), nmem);
    macro_kernel<<<grid, 256, 0, s>>>(rho, ux, uy, g, npts);
    return cudaGetLastError();
}

}  // namespace lk
