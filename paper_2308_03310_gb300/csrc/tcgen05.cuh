// tcgen05 / mbarrier helpers shared by the tensor-core Gram kernels (inline PTX, sm_103a).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "patch.cuh"

namespace lk {
namespace tc {

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory descriptor: K-major, no swizzle, LBO = 128 B (next 8-element K block),
// SBO = bytes to the next 8-row block, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of the 16-byte run (row, k8..k8+7) of a K-major tile with KC columns.
template <int KC>
__device__ __forceinline__ uint32_t core_off_b(int row, int k8) {
    return (uint32_t)((((row >> 3) * (KC / 8) + (k8 >> 3)) * 64 + (row & 7) * 8) * 2);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar)));
}

__device__ __forceinline__ void bar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the completion of the phase with the given parity; gives up after kWaitNs
// or once another role has raised the abort flag.  The outcome is made uniform over the warp
// (every lane of the calling warp waits on the same phase).
__device__ inline bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    bool ok = bar_try(bar, parity);
    if (!ok) {
        const unsigned long long t0 = global_ns();
        for (;;) {
#pragma unroll 1
            for (int i = 0; i < 4 && !ok; ++i) ok = bar_try(bar, parity);
            if (ok || *abort_flag || global_ns() - t0 > kWaitNs) break;
        }
    }
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Square root of the localization weight of an observation at (ox, oy) seen from grid point
// (qx, qy): the Gaussian's exp(-d^2 / (4 r^2)) directly, or sqrt(GC(d / c)); 0 beyond the
// cutoff.
__device__ __forceinline__ float weight_sqrt_d2(const ObsNet &net, int d2) {
    return net.loc_gc ? sqrtf(fmaxf(gaspari_cohn(sqrtf((float)d2) * net.inv_c), 0.0f))
                      : __expf(-0.5f * (float)d2 * net.inv2r2);
}
// wtab: the same function tabulated for d2 = 0 .. d2max in shared memory (tab_n = d2max + 1
// entries), or tab_n = 0
__device__ __forceinline__ float loc_weight_sqrt(const ObsNet &net, int ox, int oy, int qx,
                                                 int qy, int nx, int ny, const float *wtab,
                                                 int tab_n) {
    if (net.loc_none) return 1.0f;
    const int dx = min_image(ox - qx, nx), dy = min_image(oy - qy, ny);
    const int d2 = dx * dx + dy * dy;
    if (d2 > net.d2max) return 0.0f;
    return tab_n ? wtab[d2] : weight_sqrt_d2(net, d2);
}

// A_p row `row` (accumulator values v[0..31] for columns c0..c0+31) to global memory.
__device__ __forceinline__ void store_row32(float *dst, const float *v, int c0, int k) {
    if ((k & 3) == 0) {
#pragma unroll
        for (int i = 0; i < 32; i += 4)
            if (c0 + i < k)
                *reinterpret_cast<float4 *>(dst + c0 + i) =
                    make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (c0 + i < k) dst[c0 + i] = v[i];
    }
}

}  // namespace tc
}  // namespace lk
