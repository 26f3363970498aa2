// Observation operator (Algorithm 1, first step) and the static local-observation count.
//
// Y^f[m, :] = h(x_m): for every observation point and member, the moments
// rho, u_x, u_y (Eqs. 2-3) of the forecast state, of which the observed subset
// (bit mask, order rho, u, v) is kept.  The obs-space ensemble mean and the
// perturbations dY (Eqs. enkf_ybar, enkf_deltay) are formed in the same pass.
// One warp per observation point, lanes over members; the perturbations are
// written obs-major dY[o][m] (members contiguous) for the Gram kernel.
#include "common.cuh"
#include "kernels.h"

namespace lk {
namespace {

__global__ void __launch_bounds__(128) obs_operator_kernel(ObsOpArgs a) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const size_t npts = (size_t)a.nx * a.ny;
    const int V = __popc(a.obs_vars & 7);
    const int LV = a.L * V;
    for (int l = warp; l < a.L; l += nwarps) {
        const int2 o = a.xy[l];
        const size_t p = (size_t)o.y * a.nx + o.x;
        float val[5][3];
        float sum[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            const int m = lane + 32 * r;
            val[r][0] = val[r][1] = val[r][2] = 0.0f;
            if (m < a.nmem) {
                const float *src = a.g + (size_t)m * NV * npts + p;
                float gq[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) gq[q] = src[q * npts];
                // rho - 1 summed over opposite directions first: their deviations' parts that
                // are odd in c (the momentum) cancel inside each pair, so the partial sums stay
                // at the size of rho - 1 instead of the flow's u / 3
                const float drho = gq[4] + ((gq[0] + gq[8]) + (gq[2] + gq[6])) +
                                   ((gq[1] + gq[7]) + (gq[3] + gq[5]));
                float jx = 0.0f, jy = 0.0f;
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    if (cx(q) != 0) jx += cx(q) > 0 ? gq[q] : -gq[q];
                    if (cy(q) != 0) jy += cy(q) > 0 ? gq[q] : -gq[q];
                }
                const float rinv = 1.0f / (1.0f + drho);
                // density is carried as rho - 1 so that its perturbations keep their digits
                val[r][0] = drho;
                val[r][1] = jx * rinv;
                val[r][2] = jy * rinv;
                if (m < a.k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) sum[c] += val[r][c];
            }
        }
        float mean[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) mean[c] = warp_sum(sum[c]) / (float)a.k;
        int col = 0;
#pragma unroll
        for (int vid = 0; vid < 3; ++vid) {
            if (!(a.obs_vars & (1 << vid))) continue;
            const int s = l * V + col;
            const float ref = vid == 0 ? 1.0f : 0.0f;
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                const int m = lane + 32 * r;
                if (m < a.nmem) a.yf[(size_t)m * LV + s] = val[r][vid] + ref;
                if (m < a.k) {
                    a.yb[(size_t)s * a.kp + m] = val[r][vid] - mean[vid];
                } else if (m < a.kp) {
                    a.yb[(size_t)s * a.kp + m] = 0.0f;
                }
            }
            if (lane == 0) a.ybar[s] = mean[vid];
            ++col;
        }
    }
}

// Number of observation points within the cutoff of every grid point (thread per point).
__global__ void count_local_kernel(ObsNet net, int nx, int ny, int *nloc) {
    const size_t npts = (size_t)nx * ny;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    if (net.loc_none) {
        nloc[p] = net.L;
        return;
    }
    const int x = (int)(p % nx), y = (int)(p / nx);
    const int cr = net.cr;
    const BinRanges rx = bin_ranges(x - cr, x + cr, nx, net.cs);
    const BinRanges ry = bin_ranges(y - cr, y + cr, ny, net.cs);
    int count = 0;
    for (int iy = 0; iy < ry.n; ++iy)
        for (int by = ry.lo[iy]; by <= ry.hi[iy]; ++by)
            for (int ix = 0; ix < rx.n; ++ix)
                for (int bx = rx.lo[ix]; bx <= rx.hi[ix]; ++bx) {
                    const int cell = by * net.ncx + bx;
                    for (int i = net.cell_start[cell]; i < net.cell_start[cell + 1]; ++i) {
                        const int2 o = net.xy[net.cell_obs[i]];
                        const int dx = min_image(o.x - x, nx), dy = min_image(o.y - y, ny);
                        count += (dx * dx + dy * dy <= net.d2max) ? 1 : 0;
                    }
                }
    nloc[p] = count;
}

}  // namespace

cudaError_t launch_obs_operator(const ObsOpArgs &a, cudaStream_t s) {
    if (a.L <= 0) return cudaSuccess;
    int blocks = (a.L + 3) / 4;
    if (blocks > 8192) blocks = 8192;
    obs_operator_kernel<<<blocks, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_count_local(const ObsNet &net, int nx, int ny, int *nloc, cudaStream_t s) {
    const size_t npts = (size_t)nx * ny;
    count_local_kernel<<<(unsigned)((npts + 255) / 256), 256, 0, s>>>(net, nx, ny, nloc);
    return cudaGetLastError();
}

}  // namespace lk
