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
// one step moves 72 bytes per lattice update and is HBM bound.
//
// Two steps per launch (temporal blocking): a CTA stages a TX x TY tile of one member with a
// periodic halo of two nodes in shared memory, collides every staged node and pushes into a
// second tile (halo one), collides again and pushes the second step's populations of the
// tile's own nodes to HBM.  Per two steps a node is read ~1.3 times (the halos) and written
// once: ~84 bytes instead of 144.  The collision of a node is the same function in both
// kernels, so the arithmetic is the same as two single steps.
#include "common.cuh"
#include "kernels.h"

namespace lk {
namespace {

// c_q . v for a lattice direction known at compile time (no multiplications by 0 or +-1).
template <int CX, int CY>
__device__ __forceinline__ float cdot(float vx, float vy) {
    if constexpr (CX == 0) return CY > 0 ? vy : -vy;
    else if constexpr (CY == 0) return CX > 0 ? vx : -vx;
    else return (CX > 0 ? vx : -vx) + (CY > 0 ? vy : -vy);
}

// Direction Q (0..3) and its opposite 8 - Q: the equilibrium of the pair from its symmetric
// and antisymmetric parts, w (a +- b) with a = base + 4.5 rho (c.u)^2 and b = 3 rho c.u, then
// the BGK relaxation and the force term +- 3 w c.F.
template <bool kForce, int Q>
__device__ __forceinline__ void collide_pair(const float (&g)[NV], float ux, float uy, float base,
                                             float r3, float r45, float f3x, float f3y,
                                             float omega, float (&out)[NV]) {
    constexpr float w = wq(Q);
    const float cu = cdot<cx(Q), cy(Q)>(ux, uy);
    const float a = fmaf(r45 * cu, cu, base);
    const float b = r3 * cu;
    const float gp = w * (a + b), gm = w * (a - b);  // equilibria of Q and 8 - Q
    float sp = fmaf(omega, gp - g[Q], g[Q]);
    float sm = fmaf(omega, gm - g[8 - Q], g[8 - Q]);
    if (kForce) {
        const float fq = w * cdot<cx(Q), cy(Q)>(f3x, f3y);
        sp += fq;
        sm -= fq;
    }
    out[Q] = sp;
    out[8 - Q] = sm;
}

// BGK collision with the body-force source for one node: post-collision populations out[q]
// from the node's deviations g[q] (Eq. 1, Sec. II-A).  f^eq_q = w_q (rho + rho (3 c.u +
// 4.5 (c.u)^2 - 1.5 |u|^2)) written for the deviations: geq_q = w_q (drho - 1.5 rho |u|^2 +
// 4.5 rho (c.u)^2 + 3 rho c.u), evaluated per pair of opposite directions (q, 8 - q), whose
// terms differ only in the sign of c.u.
template <bool kForce>
__device__ __forceinline__ void collide(const float (&g)[NV], float fx, float fy, float omega,
                                        float (&out)[NV]) {
    const float drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const float jx = ((g[2] + g[5]) + g[8]) - ((g[0] + g[3]) + g[6]);
    const float jy = ((g[6] + g[7]) + g[8]) - ((g[0] + g[1]) + g[2]);
    const float rho = 1.0f + drho;
    const float rinv = __frcp_rn(rho);
    const float ux = jx * rinv, uy = jy * rinv;
    const float base = fmaf(-1.5f * rho, fmaf(ux, ux, uy * uy), drho);
    const float r3 = 3.0f * rho, r45 = 4.5f * rho;
    const float f3x = 3.0f * fx, f3y = 3.0f * fy;
    collide_pair<kForce, 0>(g, ux, uy, base, r3, r45, f3x, f3y, omega, out);
    collide_pair<kForce, 1>(g, ux, uy, base, r3, r45, f3x, f3y, omega, out);
    collide_pair<kForce, 2>(g, ux, uy, base, r3, r45, f3x, f3y, omega, out);
    collide_pair<kForce, 3>(g, ux, uy, base, r3, r45, f3x, f3y, omega, out);
    out[4] = fmaf(omega, wq(4) * base - g[4], g[4]);
}

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

    float g[NV], out[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) g[q] = __ldcs(gin + mbase + q * npts + p);
    float fx = 0.0f, fy = 0.0f;
    if (kForce) {
        const float2 F = __ldg(force + p);
        fx = F.x;
        fy = F.y;
    }
    collide<kForce>(g, fx, fy, omega, out);
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    float *dst = gout + mbase;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const int xd = cx(q) < 0 ? xm : (cx(q) > 0 ? xp : x);
        const int yd = cy(q) < 0 ? ym : (cy(q) > 0 ? yp : y);
        __stcs(dst + q * npts + (size_t)yd * nx + xd, out[q]);
    }
}

// Two-step tile: 64 x 12 output nodes, 256 threads, four CTAs (47 KB of shared memory each)
// per SM.  Measured against 64 x 8/16/20, 32 x 16 and 128 x 8 tiles and 128/512-thread CTAs:
// the fastest at 256^2 (k = 32) and 1024^2 (k = 64).
constexpr int kTX = 64;                  // output tile width
constexpr int kTY = 12;                  // output tile height
constexpr int kStep2Threads = 256;
constexpr int kStep2MinBlocks = 4;

template <int TX, int TY>
constexpr size_t step2_smem() {          // staged tile (halo 2) and its force
    return (size_t)(TX + 4) * (TY + 4) * (NV * sizeof(float) + sizeof(float2));
}

// Periodic wrap of a coordinate at most one period outside [0, n).
__device__ __forceinline__ int wrap1(int a, int n) {
    const int r = a < 0 ? a + n : (a >= n ? a - n : a);
    return (unsigned)r < (unsigned)n ? r : posmod(a, n);   // grids narrower than the halo
}

template <bool kForce, int TX, int TY, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) lbm_2step_kernel(const float *__restrict__ gin,
                                                             float *__restrict__ gout,
                                                             const float2 *__restrict__ force,
                                                             int nx, int ny, float omega) {
    constexpr int AX = TX + 4, AY = TY + 4;      // staged step-t tile, origin (x0 - 2, y0 - 2)
    constexpr int BX = TX + 2, BY = TY + 2;      // step-(t+1) nodes, origin (x0 - 1, y0 - 1)
    extern __shared__ float sm[];
    float *A = sm;                                              // [q][AY][AX]
    float2 *Fs = reinterpret_cast<float2 *>(sm + NV * AX * AY); // force over A's nodes
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const size_t npts = (size_t)nx * ny;
    const size_t mbase = (size_t)blockIdx.z * NV * npts;
    const int tid = threadIdx.x;
    // ---- stage the step-t populations of the tile and its halo (periodic) with cp.async:
    // every copy of the thread is in flight before the one wait
    for (int e = tid; e < AX * AY; e += NT) {
        const int ay = e / AX, ax = e - ay * AX;
        const size_t p = (size_t)wrap1(y0 - 2 + ay, ny) * nx + wrap1(x0 - 2 + ax, nx);
#pragma unroll
        for (int q = 0; q < NV; ++q)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)
                             __cvta_generic_to_shared(A + (q * AY + ay) * AX + ax)),
                         "l"(gin + mbase + q * npts + p)
                         : "memory");
        if (kForce)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)
                             __cvta_generic_to_shared(Fs + e)),
                         "l"(force + p)
                         : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // ---- collision t of every staged node, in place (a node owns its nine slots)
    for (int e = tid; e < AX * AY; e += NT) {
        float g[NV], out[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) g[q] = A[q * AY * AX + e];
        float fx = 0.0f, fy = 0.0f;
        if (kForce) {
            const float2 F = Fs[e];
            fx = F.x;
            fy = F.y;
        }
        collide<kForce>(g, fx, fy, omega, out);
#pragma unroll
        for (int q = 0; q < NV; ++q) A[q * AY * AX + e] = out[q];
    }
    __syncthreads();
    // ---- streaming t -> t+1 as a pull from the collided neighbours, collision t+1, and the
    // push of t+1 -> t+2 into the tile's own nodes in HBM
    float *dst = gout + mbase;
    for (int e = tid; e < BX * BY; e += NT) {
        const int by = e / BX, bx = e - by * BX;
        const int ay = by + 1, ax = bx + 1;                     // the node's slot in A
        float g[NV], out[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) g[q] = A[(q * AY + ay - cy(q)) * AX + ax - cx(q)];
        float fx = 0.0f, fy = 0.0f;
        if (kForce) {
            const float2 F = Fs[ay * AX + ax];
            fx = F.x;
            fy = F.y;
        }
        collide<kForce>(g, fx, fy, omega, out);
        // targets (bx - 1 + c_x, by - 1 + c_y): inside the tile and the grid per axis
        const int tx0 = bx - 1, ty0 = by - 1;
        bool vx[3], vy[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            vx[c] = (unsigned)(tx0 + c - 1) < (unsigned)TX && x0 + tx0 + c - 1 < nx;
            vy[c] = (unsigned)(ty0 + c - 1) < (unsigned)TY && y0 + ty0 + c - 1 < ny;
        }
        const long long at = (long long)(y0 + ty0) * nx + (x0 + tx0);
#pragma unroll
        for (int q = 0; q < NV; ++q)
            if (vx[cx(q) + 1] && vy[cy(q) + 1])
                __stcs(dst + at + (long long)q * (long long)npts + cy(q) * nx + cx(q), out[q]);
    }
}

template <int TX, int TY, int NT, int MINB>
cudaError_t set_step2_smem() {
    cudaError_t e = cudaFuncSetAttribute(lbm_2step_kernel<true, TX, TY, NT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step2_smem<TX, TY>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(lbm_2step_kernel<false, TX, TY, NT, MINB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step2_smem<TX, TY>());
}

template <int TX, int TY, int NT, int MINB>
cudaError_t launch_2step(const float *gin, float *gout, const float2 *force, int nx, int ny,
                         int nmem, float tau, cudaStream_t s) {
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, nmem);
    const float omega = 1.0f / tau;
    const size_t smem = step2_smem<TX, TY>();
    if (force)
        lbm_2step_kernel<true, TX, TY, NT, MINB><<<grid, NT, smem, s>>>(gin, gout, force, nx,
                                                                        ny, omega);
    else
        lbm_2step_kernel<false, TX, TY, NT, MINB><<<grid, NT, smem, s>>>(gin, gout, force, nx,
                                                                         ny, omega);
    return cudaGetLastError();
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

cudaError_t lbm_prepare() { return set_step2_smem<kTX, kTY, kStep2Threads, kStep2MinBlocks>(); }

cudaError_t launch_lbm_2step(const float *gin, float *gout, const float2 *force, int nx, int ny,
                             int nmem, float tau, cudaStream_t s) {
    if (nmem <= 0) return cudaSuccess;
    return launch_2step<kTX, kTY, kStep2Threads, kStep2MinBlocks>(gin, gout, force, nx, ny, nmem,
                                                                   tau, s);
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
