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
// periodic halo of two nodes in shared memory (rows copied in 16-byte runs), collides every staged node and pushes into a
// second tile (halo one), collides again and pushes the second step's populations of the
// tile's own nodes to HBM.  Per two steps a node is read ~1.3 times (the halos) and written
// once: ~84 bytes instead of 144.  The collision runs on pairs of neighbouring nodes with
// packed FP32 arithmetic; it is the same function in both kernels, so the arithmetic is the
// same as two single steps.
//
// Staging: where the window lies inside the grid (the tile is not at a periodic edge) and nx is
// a multiple of 4, one thread loads it with two bulk tensor copies (TMA: the nine population
// planes of the member as one 3-D box, the force as one 2-D box of interleaved components),
// their completion counted in bytes on an mbarrier; elsewhere every thread issues 16-byte (or
// 4-byte) cp.async copies with the periodic wrap.  Both put the same values in the same places.
#include <cuda.h>   // CUtensorMap and the tensor-map encoder's types

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace lk {
namespace {

// The collision works on two nodes at once: every quantity is a float2 (node pair) and every
// operation a packed FP32 instruction, which rounds each lane exactly as the scalar operation
// would.  Both kernels use this function (the single-step kernel with a node in both lanes),
// so their arithmetic is the same.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {   // a - b, one rounding
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// 1 / x for x near 1 (the density): the hardware approximation refined by one Newton-Raphson
// step y + y (1 - x y), which squares its relative error.
__device__ __forceinline__ float2 rcp2(float2 x) {
    float2 y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.x) : "f"(x.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.y) : "f"(x.y));
    const float2 e = fma2(neg2(x), y, dup2(1.0f));
    return fma2(y, e, y);
}

// c_q . v for a lattice direction known at compile time (no multiplications by 0 or +-1).
template <int CX, int CY>
__device__ __forceinline__ float2 cdot2(float2 vx, float2 vy) {
    if constexpr (CX == 0) return CY > 0 ? vy : neg2(vy);
    else if constexpr (CY == 0) return CX > 0 ? vx : neg2(vx);
    else return add2(CX > 0 ? vx : neg2(vx), CY > 0 ? vy : neg2(vy));
}

// Direction Q (0..3) and its opposite 8 - Q: the equilibrium of the pair from its symmetric
// and antisymmetric parts, w (a +- b) with a = base + 4.5 rho (c.u)^2 and b = 3 rho c.u, then
// the BGK relaxation and the force term +- 3 w c.F.
template <bool kForce, int Q>
__device__ __forceinline__ void collide_pair(const float2 (&g)[NV], float2 ux, float2 uy,
                                             float2 base, float2 r3, float2 r45, float2 f3x,
                                             float2 f3y, float2 omega, float2 (&out)[NV]) {
    const float2 w = dup2(wq(Q));
    const float2 cu = cdot2<cx(Q), cy(Q)>(ux, uy);
    const float2 a = fma2(mul2(r45, cu), cu, base);
    const float2 b = mul2(r3, cu);
    const float2 gp = mul2(w, add2(a, b)), gm = mul2(w, sub2(a, b));  // equilibria of Q, 8 - Q
    float2 sp = fma2(omega, sub2(gp, g[Q]), g[Q]);
    float2 sm = fma2(omega, sub2(gm, g[8 - Q]), g[8 - Q]);
    if (kForce) {
        const float2 fq = mul2(w, cdot2<cx(Q), cy(Q)>(f3x, f3y));
        sp = add2(sp, fq);
        sm = sub2(sm, fq);
    }
    out[Q] = sp;
    out[8 - Q] = sm;
}

// BGK collision with the body-force source for two nodes: post-collision populations out[q]
// from the nodes' deviations g[q] (Eq. 1, Sec. II-A).  f^eq_q = w_q (rho + rho (3 c.u +
// 4.5 (c.u)^2 - 1.5 |u|^2)) written for the deviations: geq_q = w_q (drho - 1.5 rho |u|^2 +
// 4.5 rho (c.u)^2 + 3 rho c.u), evaluated per pair of opposite directions (q, 8 - q), whose
// terms differ only in the sign of c.u.
template <bool kForce>
__device__ __forceinline__ void collide2(const float2 (&g)[NV], float2 fx, float2 fy,
                                         float2 omega, float2 (&out)[NV]) {
    const float2 g01 = add2(g[0], g[1]);
    const float2 drho = add2(add2(add2(g01, add2(g[2], g[3])), add2(add2(g[4], g[5]),
                                                                  add2(g[6], g[7]))), g[8]);
    const float2 jx = sub2(add2(add2(g[2], g[5]), g[8]), add2(add2(g[0], g[3]), g[6]));
    const float2 jy = sub2(add2(add2(g[6], g[7]), g[8]), add2(g01, g[2]));
    const float2 rho = add2(dup2(1.0f), drho);
    const float2 rinv = rcp2(rho);
    const float2 ux = mul2(jx, rinv), uy = mul2(jy, rinv);
    const float2 base = fma2(mul2(dup2(-1.5f), rho), fma2(ux, ux, mul2(uy, uy)), drho);
    const float2 r3 = mul2(dup2(3.0f), rho), r45 = mul2(dup2(4.5f), rho);
    const float2 f3x = mul2(dup2(3.0f), fx), f3y = mul2(dup2(3.0f), fy);
    collide_pair<kForce, 0>(g, ux, uy, base, r3, r45, f3x, f3y, omega, out);
    collide_pair<kForce, 1>(g, ux, uy, base, r3, r45, f3x, f3y, omega, out);
    collide_pair<kForce, 2>(g, ux, uy, base, r3, r45, f3x, f3y, omega, out);
    collide_pair<kForce, 3>(g, ux, uy, base, r3, r45, f3x, f3y, omega, out);
    out[4] = fma2(omega, sub2(mul2(dup2(wq(4)), base), g[4]), g[4]);
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

    float2 g[NV], out[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) g[q] = dup2(__ldcs(gin + mbase + q * npts + p));
    float2 fx = dup2(0.0f), fy = dup2(0.0f);
    if (kForce) {
        const float2 F = __ldg(force + p);
        fx = dup2(F.x);
        fy = dup2(F.y);
    }
    collide2<kForce>(g, fx, fy, dup2(omega), out);
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    float *dst = gout + mbase;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const int xd = cx(q) < 0 ? xm : (cx(q) > 0 ? xp : x);
        const int yd = cy(q) < 0 ? ym : (cy(q) > 0 ? yp : y);
        __stcs(dst + q * npts + (size_t)yd * nx + xd, out[q].x);
    }
}

// Two-step tile: 64 x 12 output nodes, 256 threads, four CTAs (51 KB of shared memory each)
// per SM.  Measured against 64 x 8/16/20, 32 x 16 and 128 x 8 tiles and 128/512-thread CTAs:
// the fastest at 256^2 (k = 32) and 1024^2 (k = 64).
constexpr int kTX = 64;                  // output tile width
constexpr int kTY = 12;                  // output tile height
constexpr int kStep2Threads = 256;
constexpr int kStep2MinBlocks = 4;

template <int TX, int TY>
constexpr size_t step2_smem() {          // staged tile (halo 2, x window widened to 16 bytes)
    return (size_t)(TX + 8) * (TY + 4) * (NV + 2) * sizeof(float);   // and its force
}

static_assert(sizeof(TmaMap) == sizeof(CUtensorMap) && alignof(TmaMap) >= 64, "tensor map image");

constexpr unsigned long long kTmaWaitNs = 2000000000ull;   // bound of a staging wait (2 s)

__device__ __forceinline__ unsigned long long lbm_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool tma_bar_try(uint32_t bar) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar)
        : "memory");
    return done != 0;
}
// bounded wait for the staging barrier's first phase
__device__ __forceinline__ bool tma_bar_wait(uint32_t bar) {
    if (tma_bar_try(bar)) return true;
    const unsigned long long t0 = lbm_ns();
    for (;;) {
        if (tma_bar_try(bar)) return true;
        if (lbm_ns() - t0 > kTmaWaitNs) return false;
    }
}

// Periodic wrap of a coordinate at most one period outside [0, n).
__device__ __forceinline__ int wrap1(int a, int n) {
    const int r = a < 0 ? a + n : (a >= n ? a - n : a);
    return (unsigned)r < (unsigned)n ? r : posmod(a, n);   // grids narrower than the halo
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)
                     __cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)
                     __cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

template <bool kForce, int TX, int TY, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) lbm_2step_kernel(const float *__restrict__ gin,
                                                             float *__restrict__ gout,
                                                             const float2 *__restrict__ force,
                                                             int nx, int ny, float omega_s,
                                                             const __grid_constant__ TmaMap tg,
                                                             const __grid_constant__ TmaMap tf,
                                                             int use_tma, int *status) {
    // staged step-t window: x in [x0 - 4, x0 + TX + 4), y in [y0 - 2, y0 + TY + 2); the nodes
    // two beyond the tile on each side are the halo, the outer two columns only align the
    // window's rows to 16 bytes
    constexpr int AX = TX + 8, AY = TY + 4;
    constexpr int BX = TX + 2, BY = TY + 2;      // step-(t+1) nodes, origin (x0 - 1, y0 - 1)
    constexpr int HX = TX + 4;                   // collided columns 2 .. AX - 3
    static_assert(TX % 4 == 0 && HX % 2 == 0 && BX % 2 == 0, "16-byte rows, node pairs");
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t tbar;
    float *A = sm;                                               // [q][AY][AX]
    float2 *Fs = reinterpret_cast<float2 *>(sm + NV * AX * AY);  // force over A's nodes
    static_assert((NV * AX * AY * 4) % 128 == 0, "the force box starts 128-byte aligned");
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const size_t npts = (size_t)nx * ny;
    const size_t mbase = (size_t)blockIdx.z * NV * npts;
    const int tid = threadIdx.x;
    const float2 omega = dup2(omega_s);
    // ---- stage the window: a window inside the grid by TMA (the maps exist only where nx is a
    // multiple of 4, so x0 - 4 is a 16-byte boundary); otherwise with cp.async, every copy of
    // the thread in flight before the one wait: runs of four nodes (16 bytes) where nx is a
    // multiple of 4 -- x0 is, so every run starts on a 16-byte boundary, also where it wraps --
    // single nodes otherwise
    const bool by_tma = use_tma && x0 >= 4 && x0 + TX + 4 <= nx && y0 >= 2 && y0 + TY + 2 <= ny;
    if (by_tma) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&tbar);
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
            asm volatile("fence.mbarrier_init.release.cluster;");
        }
        __syncthreads();
        if (tid == 0) {
            constexpr uint32_t bytes = NV * AX * AY * 4 + (kForce ? AX * AY * 8 : 0);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"((uint32_t)__cvta_generic_to_shared(A)),
                "l"(reinterpret_cast<uint64_t>(&tg)), "r"(x0 - 4), "r"(y0 - 2),
                "r"((int)blockIdx.z * NV), "r"(bar)
                : "memory");
            if (kForce)
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::"
                    "bytes [%0], [%1, {%2, %3}], [%4];" ::"r"((uint32_t)__cvta_generic_to_shared(Fs)),
                    "l"(reinterpret_cast<uint64_t>(&tf)), "r"(2 * (x0 - 4)), "r"(y0 - 2), "r"(bar)
                    : "memory");
        }
        // the outcome made uniform over the CTA; a timeout is never expected: report it, give
        // the copies a second bounded wait to land, leave
        if (__syncthreads_and(tma_bar_wait(bar)) == 0) {
            if (tid == 0 && status) atomicOr(status, ST_TIMEOUT);
            tma_bar_wait(bar);
            return;
        }
    } else if ((nx & 3) == 0) {
        constexpr int GX = AX / 4;
        for (int e = tid; e < AY * GX; e += NT) {
            const int ay = e / GX, gx = e - ay * GX;
            const size_t p = (size_t)wrap1(y0 - 2 + ay, ny) * nx + wrap1(x0 - 4 + 4 * gx, nx);
            float *a = A + ay * AX + 4 * gx;
#pragma unroll
            for (int q = 0; q < NV; ++q) cp_async16(a + q * AY * AX, gin + mbase + q * npts + p);
            if (kForce) {
                cp_async16(Fs + ay * AX + 4 * gx, force + p);
                cp_async16(Fs + ay * AX + 4 * gx + 2, force + p + 2);
            }
        }
    } else {
        for (int e = tid; e < AX * AY; e += NT) {
            const int ay = e / AX, ax = e - ay * AX;
            const size_t p = (size_t)wrap1(y0 - 2 + ay, ny) * nx + wrap1(x0 - 4 + ax, nx);
#pragma unroll
            for (int q = 0; q < NV; ++q) cp_async4(A + (q * AY + ay) * AX + ax, gin + mbase + q * npts + p);
            if (kForce) {
                const float *F = reinterpret_cast<const float *>(force + p);
                cp_async4(reinterpret_cast<float *>(Fs + e), F);
                cp_async4(reinterpret_cast<float *>(Fs + e) + 1, F + 1);
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // ---- collision t of the tile and its halo, in place (a node owns its nine slots), two
    // neighbouring nodes (ax, ax + 1), ax even, per thread
    for (int e = tid; e < HX * AY / 2; e += NT) {
        const int ay = (2 * e) / HX, ax = 2 + 2 * e - ay * HX;
        const int i = ay * AX + ax;
        float2 g[NV], out[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) g[q] = *reinterpret_cast<const float2 *>(A + q * AY * AX + i);
        float2 fx = dup2(0.0f), fy = dup2(0.0f);
        if (kForce) {
            const float4 F = *reinterpret_cast<const float4 *>(Fs + i);
            fx = make_float2(F.x, F.z);
            fy = make_float2(F.y, F.w);
        }
        collide2<kForce>(g, fx, fy, omega, out);
#pragma unroll
        for (int q = 0; q < NV; ++q) *reinterpret_cast<float2 *>(A + q * AY * AX + i) = out[q];
    }
    __syncthreads();
    // ---- streaming t -> t+1 as a pull from the collided neighbours, collision t+1, and the
    // push of t+1 -> t+2 into the tile's own nodes in HBM; node pairs (bx, bx + 1), bx even
    float *dst = gout + mbase;
    for (int e = tid; e < BX * BY / 2; e += NT) {
        const int by = (2 * e) / BX, bx = 2 * e - by * BX;
        const int ay = by + 1, ax = bx + 3;                     // the first node's slot in A
        float2 g[NV], out[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const float *src = A + (q * AY + ay - cy(q)) * AX + ax - cx(q);
            // the pair's sources are 8-byte aligned where ax - c_x is even (c_x = +-1)
            g[q] = cx(q) != 0 ? *reinterpret_cast<const float2 *>(src)
                              : make_float2(src[0], src[1]);
        }
        float2 fx = dup2(0.0f), fy = dup2(0.0f);
        if (kForce) {
            const float2 F0 = Fs[ay * AX + ax], F1 = Fs[ay * AX + ax + 1];
            fx = make_float2(F0.x, F1.x);
            fy = make_float2(F0.y, F1.y);
        }
        collide2<kForce>(g, fx, fy, omega, out);
        // targets (bx - 1 + h + c_x, by - 1 + c_y) of node h: inside the tile and the grid
        const int tx0 = bx - 1, ty0 = by - 1;
        bool vx[4], vy[3];
#pragma unroll
        for (int c = 0; c < 4; ++c)
            vx[c] = (unsigned)(tx0 + c - 1) < (unsigned)TX && x0 + tx0 + c - 1 < nx;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            vy[c] = (unsigned)(ty0 + c - 1) < (unsigned)TY && y0 + ty0 + c - 1 < ny;
        const long long at = (long long)(y0 + ty0) * nx + (x0 + tx0);
        // a pair's targets are 8-byte aligned where c_x = +-1 and nx is even (x0 + bx even):
        // one float2 store where both are inside
        const bool pair_ok = (nx & 1) == 0;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float *d = dst + at + (long long)q * (long long)npts + cy(q) * nx + cx(q);
            if (vy[cy(q) + 1]) {
                const bool v0 = vx[cx(q) + 1], v1 = vx[cx(q) + 2];
                if (cx(q) != 0 && pair_ok && v0 && v1) {
                    __stcs(reinterpret_cast<float2 *>(d), out[q]);
                } else {
                    if (v0) __stcs(d, out[q].x);
                    if (v1) __stcs(d + 1, out[q].y);
                }
            }
        }
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
                         int nmem, float tau, cudaStream_t s, const LbmTma *tma, int *status) {
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, nmem);
    const float omega = 1.0f / tau;
    const size_t smem = step2_smem<TX, TY>();
    // the state map of the buffer read, and the force map where the force is staged
    const int b = !tma || !(tma->ok & 1) ? -1 : gin == tma->gptr[0] ? 0 : gin == tma->gptr[1] ? 1 : -1;
    const int use = b >= 0 && (!force || (tma->ok & 2));
    static const TmaMap none = {};
    const TmaMap &tg = use ? tma->g[b] : none;
    const TmaMap &tf = use && force ? tma->f : none;
    if (force)
        lbm_2step_kernel<true, TX, TY, NT, MINB><<<grid, NT, smem, s>>>(gin, gout, force, nx,
                                                                        ny, omega, tg, tf, use,
                                                                        status);
    else
        lbm_2step_kernel<false, TX, TY, NT, MINB><<<grid, NT, smem, s>>>(gin, gout, force, nx,
                                                                         ny, omega, tg, tf, use,
                                                                         status);
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
                             int nmem, float tau, cudaStream_t s, const LbmTma *tma, int *status) {
    if (nmem <= 0) return cudaSuccess;
    return launch_2step<kTX, kTY, kStep2Threads, kStep2MinBlocks>(gin, gout, force, nx, ny, nmem,
                                                                   tau, s, tma, status);
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// the driver's tensor-map encoder, through the runtime (no link against the driver library)
EncodeTiled encode_tiled() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}
}  // namespace

cudaError_t lbm_tma_build(const float *g0, const float *g1, const float2 *force, int nx, int ny,
                          int nmem, LbmTma *out) {
    out->ok = 0;
    constexpr int AX = kTX + 8, AY = kTY + 4;
    static_assert(2 * AX <= 256 && AY <= 256 && NV <= 256, "a TMA box has at most 256 per side");
    if ((nx & 3) != 0 || nx < AX || ny < AY || nmem <= 0) return cudaSuccess;   // cp.async only
    // without the driver's encoder the staging stays on cp.async (the same values); a map the
    // encoder rejects is an error
    const EncodeTiled enc = encode_tiled();
    if (!enc) return cudaSuccess;
    const cuuint32_t es[3] = {1, 1, 1};
    // state [nmem * 9 planes][ny][nx] floats; box: one member's nine planes of the window
    const cuuint64_t gdim[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nmem * NV};
    const cuuint64_t gstr[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    const cuuint32_t gbox[3] = {AX, AY, NV};
    for (int b = 0; b < 2; ++b)
        if (enc(reinterpret_cast<CUtensorMap *>(&out->g[b]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                const_cast<float *>(b ? g1 : g0), gdim, gstr, gbox, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    out->gptr[0] = g0;
    out->gptr[1] = g1;
    out->ok = 1;
    if (force) {   // [ny][2 nx] floats (the components interleaved); box: the window's rows
        const cuuint64_t fdim[2] = {(cuuint64_t)2 * nx, (cuuint64_t)ny};
        const cuuint64_t fstr[1] = {(cuuint64_t)2 * nx * 4};
        const cuuint32_t fbox[2] = {2 * AX, AY};
        if (enc(reinterpret_cast<CUtensorMap *>(&out->f), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                const_cast<float2 *>(force), fdim, fstr, fbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        out->ok |= 2;
    }
    return cudaSuccess;
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
