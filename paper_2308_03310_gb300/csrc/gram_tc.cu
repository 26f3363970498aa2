// Localized Gram matrices on the 5th-generation tensor cores (tcgen05), split FP16, FP32
// accumulation: the mixed-precision form of
//     A_p = sum_o G_po / sigma_o^2  dy_o dy_o^T ,   c_p = sum_o G_po / sigma_o^2  dy_o (yo_o - ybar_o)
// (the k x k term of Eq. letkf_q and the vector of Eq. letkf_wa, R-localization of Sec. II-B).
//
// With y_o = dy_o / sigma_o (O(1) values) a tile of P grid points that share one observation
// patch computes, per point, A_p = Y^T (diag(G_p) Y) with Y the patch's scaled perturbations.
// Both operands are split into FP16 hi + lo parts and all four products are accumulated in
// FP32 in tensor memory, so the result carries ~22 significant bits, like FP32:
//     k = 64:  one M = 128 MMA per K-step stacks [Y_hi; Y_lo] as rows, and the N dimension
//              holds [B_hi | B_lo] of every point (B = diag(G_p) Y), P = 4 points, N = 512;
//     k = 128: two M = 128 MMAs (Y_hi, Y_lo) per point and K-step, P = 2 points, N = 512.
// The tile's accumulators fill all 512 TMEM columns.  CUDA cores build the next 64-scalar
// K-chunk of both operands (scaling, localization weights, hi/lo split, c) into the second
// shared-memory stage while the tensor cores consume the current one; a single thread issues
// the MMAs and commits them to the stage's mbarrier.  The chunk's perturbation rows are staged
// in shared memory by 1-D TMA bulk copies (cp.async.bulk, completion counted in bytes on an
// mbarrier) one chunk ahead of their use.  Operands are K-major without swizzle (8 x 16-byte
// core matrices).  Every wait on an mbarrier is bounded: on expiry the status
// word gets ST_TIMEOUT, the CTA stops issuing work, waits (bounded) for its MMAs and frees
// its tensor memory.  Candidate order is fixed, so results are bitwise reproducible.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "patch.cuh"

namespace lk {
namespace {

constexpr int kTcThreads = 256;      // 8 warps: operand production; warps w, w+4 share a TMEM quadrant
constexpr int kMetaCap = 1024;       // candidate scalars whose metadata one segment keeps
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitSpins = 1ll << 24;

template <int KP>
struct TcShape {
    static constexpr int P = 512 / (2 * KP);                       // points per tile
    static constexpr int TW = 2, TH = P / 2;                       // 2x2 (k=64), 2x1 (k=128)
    static constexpr int KC = KP == 64 ? 64 : 32;                  // scalars per K-chunk
    static constexpr int SBO = (KC / 8) * 128;                     // bytes between row blocks
    static constexpr int AROWS = 2 * KP;                           // Y_hi rows then Y_lo rows
    static constexpr int BROWS = P * 2 * KP;                       // per point B_hi then B_lo
    static constexpr int A_BYTES = AROWS * KC * 2;
    static constexpr int B_BYTES = BROWS * KC * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int YLD = KP + 4;                             // padded FP32 staging row
    static constexpr int Y_BYTES = KC * YLD * 4;
    static constexpr int NM = KP / 64;                             // member slots per thread
    static constexpr int SMEM = 2 * STAGE + 2 * Y_BYTES;
};

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

// Half offset of element (row, kk) of a K-major tile with KC columns (core-matrix layout).
template <int KC>
__device__ __forceinline__ int core_off(int row, int kk) {
    return ((row >> 3) * (KC / 8) + (kk >> 3)) * 64 + (row & 7) * 8 + (kk & 7);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done = 0;
    for (long long it = 0; it < kWaitSpins && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
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

template <int KP>
__global__ void __launch_bounds__(kTcThreads, 1) gram_tc_kernel(GramArgs a, int *status) {
    using S = TcShape<KP>;
    constexpr int P = S::P, TW = S::TW, TH = S::TH, NM = S::NM, KC = S::KC, YLD = S::YLD;
    extern __shared__ __align__(1024) unsigned char dyn[];
    __shared__ int cell_base[kMaxPatchCells];
    __shared__ int cell_pre[kMaxPatchCells + 1];
    __shared__ int warp_tot[kTcThreads / 32];
    __shared__ int gidx[kMetaCap];       // global scalar index of each candidate slot (-1: pad)
    __shared__ float sr[kMetaCap];       // sqrt(R^-1) of the slot
    __shared__ float cm[kMetaCap];       // sqrt(R^-1) (yo - ybar) of the slot
    __shared__ int2 opos[kMetaCap];      // observation point of the slot
    __shared__ float wts[2][P][KC];      // localization weights of the current / next chunk
    __shared__ int nloc_s[P];
    __shared__ __align__(8) uint64_t mbar[2];   // MMAs of an operand stage done
    __shared__ __align__(8) uint64_t ybar[2];   // bulk copies of a staging buffer landed
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const ObsNet &net = a.net;
    const int V = net.V;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rows = a.y_end - a.y_begin;
    const int ntx = (a.nx + TW - 1) / TW, nty = (rows + TH - 1) / TH;
    const int ntiles = ntx * nty;
    float *ystage = reinterpret_cast<float *>(dyn + 2 * S::STAGE);

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ybar[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    // barrier bookkeeping (identical in every thread): each completion is waited exactly once
    bool mpend[2] = {false, false}, ypend[2] = {false, false};
    uint32_t mph[2] = {0u, 0u}, yph[2] = {0u, 0u};
    auto wait_mma = [&](int b) -> bool {
        if (!mpend[b]) return true;
        const bool ok = mbar_wait(&mbar[b], mph[b]);
        mph[b] ^= 1u;
        mpend[b] = false;
        return ok;
    };
    auto wait_y = [&](int b) -> bool {
        if (!ypend[b]) return true;
        const bool ok = mbar_wait(&ybar[b], yph[b]);
        yph[b] ^= 1u;
        ypend[b] = false;
        return ok;
    };
    // warp 1: bulk-copy the dY rows of the KC slots starting at segment slot `first` (n of
    // them real) into staging buffer yb.  Lane 0 announces the byte count on the buffer's
    // mbarrier, then every lane issues the copies of its own slots.  All threads mark the
    // buffer pending.
    auto prefetch = [&](int yb, int first, int n) {
        if (warp == 1) {
            float *dst = ystage + yb * KC * YLD;
            int mine[KC / 32];
            int cnt = 0;
#pragma unroll
            for (int r = 0; r < KC / 32; ++r) {
                const int kk = lane + 32 * r;
                mine[r] = kk < n ? gidx[first + kk] : -1;
                cnt += __popc(__ballot_sync(0xffffffffu, mine[r] >= 0));
            }
            if (lane == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                 smem_u32(&ybar[yb])),
                             "r"((uint32_t)(cnt * KP * 4)));
            __syncwarp();
#pragma unroll
            for (int r = 0; r < KC / 32; ++r) {
                if (mine[r] < 0) continue;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
                    "%2, [%3];" ::"r"(smem_u32(dst + (lane + 32 * r) * YLD)),
                    "l"(a.yb + (size_t)mine[r] * KP), "r"(KP * 4), "r"(smem_u32(&ybar[yb]))
                    : "memory");
            }
        }
        ypend[yb] = true;
    };
    // localization weights of the KC slots starting at `first` for every point of the tile
    auto weights = [&](int wb, int seg, int first, int n, int tx0, int ty0) {
        for (int e = tid; e < P * KC; e += kTcThreads) {
            const int p = e / KC, kk = e % KC;
            const int qx = tx0 + (p % TW), qy = ty0 + (p / TW);
            float w = 0.0f;
            if (kk < n && gidx[first + kk] >= 0 && qx < a.nx && qy < a.y_end) {
                w = loc_weight(net, opos[first + kk], qx, qy, a.nx, a.ny);
                if (w != 0.0f && (seg + first + kk) % V == 0) atomicAdd(&nloc_s[p], 1);
            }
            wts[wb][p][kk] = w;
        }
    };

    int gch = 0;  // chunks issued by this CTA (selects operand stage and staging buffer)
    for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
        const int tx0 = (tile % ntx) * TW;
        const int ty0 = a.y_begin + (tile / ntx) * TH;
        const int nc = build_patch<kTcThreads>(net, a.nx, a.ny, tx0, ty0, TW, TH, cell_base,
                                               cell_pre, warp_tot);
        const int total_slots = cell_pre[nc] * V;
        if (tid < P) nloc_s[tid] = 0;
        float cacc[P][NM];
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int i = 0; i < NM; ++i) cacc[p][i] = 0.0f;
        int tile_chunks = 0;

        for (int seg = 0; seg < total_slots && !abort_flag; seg += kMetaCap) {
            const int nseg = min(kMetaCap, total_slots - seg);
            __syncthreads();  // previous segment's metadata no longer in use
            // ---- segment metadata: every candidate scalar slot at once
            for (int e = tid; e < kMetaCap; e += kTcThreads) {
                int sidx = -1;
                float r = 0.0f, c = 0.0f;
                int2 xy = make_int2(0, 0);
                if (e < nseg) {
                    const int j = seg + e, v = j % V;
                    const int o = patch_obs(net, cell_base, cell_pre, nc, j / V);
                    sidx = o * V + v;
                    xy = net.xy[o];
                    r = sqrtf(a.rinv[sidx]);
                    c = r * ((a.yo[sidx] - a.yref[v]) - a.ybar[sidx]);
                }
                gidx[e] = sidx;
                sr[e] = r;
                cm[e] = c;
                opos[e] = xy;
            }
            __syncthreads();
            const int nchunks = (nseg + KC - 1) / KC;
            prefetch(gch & 1, 0, min(KC, nseg));
            weights(0, seg, 0, min(KC, nseg), tx0, ty0);
            __syncthreads();
            for (int ch = 0; ch < nchunks; ++ch, ++gch) {
                const int b = gch & 1, wb = ch & 1;
                const int first = ch * KC, n = min(KC, nseg - first);
                const bool okm = wait_mma(b);   // operand stage b free again
                const bool oky = wait_y(b);     // this chunk's dY rows landed
                // a wait that gave up is reported through the shared flag; every thread reads
                // it after the chunk's barrier, so all of them leave the loop together
                if (!okm || !oky) abort_flag = 1;
                // next chunk's rows into the other staging buffer (its last reader, the
                // previous chunk's production, finished before the last barrier)
                if (ch + 1 < nchunks) prefetch(b ^ 1, first + KC, min(KC, nseg - first - KC));
                unsigned char *stage = dyn + b * S::STAGE;
                __half *sA = reinterpret_cast<__half *>(stage);
                __half *sB = reinterpret_cast<__half *>(stage + S::A_BYTES);
                const float *ys = ystage + b * KC * YLD;
                // ---- operands: (member, slot pair) items, 8 members x 4 pairs per instruction
#pragma unroll
                for (int im = 0; im < NM; ++im) {
                    const int m = 8 * (warp + 8 * im) + (lane >> 2);
#pragma unroll 2
                    for (int kb = 0; kb < KC / 8; ++kb) {
                        const int kk = 8 * kb + 2 * (lane & 3);
                        const bool v0 = kk < n && gidx[first + kk] >= 0;
                        const bool v1 = kk + 1 < n && gidx[first + kk + 1] >= 0;
                        const float y0 = v0 ? ys[kk * YLD + m] * sr[first + kk] : 0.0f;
                        const float y1 = v1 ? ys[(kk + 1) * YLD + m] * sr[first + kk + 1] : 0.0f;
                        const __half h0 = __float2half_rn(y0), h1 = __float2half_rn(y1);
                        const __half l0 = __float2half_rn(y0 - __half2float(h0));
                        const __half l1 = __float2half_rn(y1 - __half2float(h1));
                        *reinterpret_cast<__half2 *>(sA + core_off<KC>(m, kk)) =
                            __halves2half2(h0, h1);
                        *reinterpret_cast<__half2 *>(sA + core_off<KC>(KP + m, kk)) =
                            __halves2half2(l0, l1);
                        const float c0 = v0 ? cm[first + kk] * y0 : 0.0f;
                        const float c1 = v1 ? cm[first + kk + 1] * y1 : 0.0f;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            const float w0 = wts[wb][p][kk], w1 = wts[wb][p][kk + 1];
                            const float b0 = w0 * y0, b1 = w1 * y1;
                            const __half bh0 = __float2half_rn(b0), bh1 = __float2half_rn(b1);
                            const __half bl0 = __float2half_rn(b0 - __half2float(bh0));
                            const __half bl1 = __float2half_rn(b1 - __half2float(bh1));
                            const int rb = p * 2 * KP + m;
                            *reinterpret_cast<__half2 *>(sB + core_off<KC>(rb, kk)) =
                                __halves2half2(bh0, bh1);
                            *reinterpret_cast<__half2 *>(sB + core_off<KC>(rb + KP, kk)) =
                                __halves2half2(bl0, bl1);
                            cacc[p][im] = fmaf(w0, c0, fmaf(w1, c1, cacc[p][im]));
                        }
                    }
                }
                // the next chunk's weights, for use after the barrier
                if (ch + 1 < nchunks)
                    weights(wb ^ 1, seg, first + KC, min(KC, nseg - first - KC), tx0, ty0);
                asm volatile("fence.proxy.async.shared::cta;");
                __syncthreads();
                if (abort_flag) break;
                // ---- tensor cores: the chunk's K-steps of 16, committed to the stage barrier
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint32_t acc = (tile_chunks > 0 || ks > 0) ? 1u : 0u;
                        if (KP == 64) {
                            const uint64_t da = sdesc(a0 + ks * 256, S::SBO);
#pragma unroll
                            for (int h = 0; h < 2; ++h)
                                mma_f16(tmem + h * 256, da,
                                        sdesc(b0 + h * (256 / 8) * S::SBO + ks * 256, S::SBO),
                                        idesc_f16(128, 256), acc);
                        } else {
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                const uint64_t db =
                                    sdesc(b0 + p * (256 / 8) * S::SBO + ks * 256, S::SBO);
                                mma_f16(tmem + p * 256, sdesc(a0 + ks * 256, S::SBO), db,
                                        idesc_f16(128, 256), acc);
                                mma_f16(tmem + p * 256,
                                        sdesc(a0 + (128 / 8) * S::SBO + ks * 256, S::SBO), db,
                                        idesc_f16(128, 256), 1u);
                            }
                        }
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_u32(&mbar[b])));
                }
                mpend[b] = true;
                ++tile_chunks;
            }
        }
        // ---- all MMAs and copies of the tile done
        const bool ok = wait_mma(0) & wait_mma(1) & wait_y(0) & wait_y(1);
        if (!ok && tid == 0) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;");

        // ---- epilogue: A_p = sum of the hi/lo blocks; warps w and w+4 share TMEM lanes
        const int quad = warp & 3, half = warp >> 2;
        const int trow = 32 * quad + lane;                      // D row of this thread
        const uint32_t tl = tmem + ((uint32_t)(32 * quad) << 16);
        float *red = reinterpret_cast<float *>(dyn);            // [P][64][65] (k = 64)
        if (KP == 64 && tile_chunks > 0 && quad >= 2) {         // rows 64..127: Y_lo part
            const int m = trow - 64, c0 = 32 * half;
#pragma unroll 1
            for (int p = 0; p < P; ++p) {
                float vh[32], vl[32];
                tmem_ld32(tl + p * 128 + c0, vh);
                tmem_ld32(tl + p * 128 + 64 + c0, vl);
#pragma unroll
                for (int i = 0; i < 32; ++i) red[(p * 64 + m) * 65 + c0 + i] = vh[i] + vl[i];
            }
        }
        __syncthreads();
        if (tile_chunks > 0 && (KP == 128 || quad < 2)) {
            const int m = trow;
#pragma unroll 1
            for (int p = 0; p < P; ++p) {
                const int qx = tx0 + (p % TW), qy = ty0 + (p / TW);
                const bool valid = qx < a.nx && qy < a.y_end && m < a.k;
                const size_t lp = valid ? (size_t)(qy - a.y_begin) * a.nx + qx : 0;
#pragma unroll 1
                for (int cc = 0; cc < KP / 64; ++cc) {
                    const int c0 = (KP / 2) * half + 32 * cc;
                    float vh[32], vl[32];
                    tmem_ld32(tl + p * 2 * KP + c0, vh);
                    tmem_ld32(tl + p * 2 * KP + KP + c0, vl);
                    if (!valid) continue;
                    float *dst = a.gram + lp * a.k * a.k + (size_t)m * a.k;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        vh[i] += vl[i];
                        if (KP == 64) vh[i] += red[(p * 64 + m) * 65 + c0 + i];
                    }
                    if ((a.k & 3) == 0) {  // rows start 16-byte aligned: vector stores
#pragma unroll
                        for (int i = 0; i < 32; i += 4)
                            if (c0 + i < a.k)
                                *reinterpret_cast<float4 *>(dst + c0 + i) =
                                    make_float4(vh[i], vh[i + 1], vh[i + 2], vh[i + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (c0 + i < a.k) dst[c0 + i] = vh[i];
                    }
                }
            }
        }
        // ---- c_p: the 4 lanes sharing a member hold partial sums; nloc from the counters
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int im = 0; im < NM; ++im) {
                float v = cacc[p][im];
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                const int m = 8 * (warp + 8 * im) + (lane >> 2);
                const int qx = tx0 + (p % TW), qy = ty0 + (p / TW);
                if ((lane & 3) == 0 && m < a.k && qx < a.nx && qy < a.y_end) {
                    const size_t lp = (size_t)(qy - a.y_begin) * a.nx + qx;
                    a.cvec[lp * a.k + m] = v;
                }
            }
        if (tid < P) {
            const int qx = tx0 + (tid % TW), qy = ty0 + (tid / TW);
            if (qx < a.nx && qy < a.y_end) {
                const size_t lp = (size_t)(qy - a.y_begin) * a.nx + qx;
                a.nloc[lp] = nloc_s[tid];
                if (tile_chunks == 0)  // no candidate at all: the Gram matrix is zero
                    for (int e = 0; e < a.k * a.k; ++e) a.gram[lp * a.k * a.k + e] = 0.0f;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    // ---- stop: outstanding MMAs and copies (bounded), then free the tensor memory
    wait_mma(0);
    wait_mma(1);
    wait_y(0);
    wait_y(1);
    if (abort_flag && tid == 0) atomicOr(status, ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

template <int KP>
size_t tc_smem() {
    return (size_t)TcShape<KP>::SMEM;
}

}  // namespace

int gram_tc_tile_width(int kp) { return kp == 64 ? TcShape<64>::TW : TcShape<128>::TW; }
int gram_tc_tile_height(int kp) { return kp == 64 ? TcShape<64>::TH : TcShape<128>::TH; }

cudaError_t gram_tc_prepare(int kp) {
    if (kp == 64)
        return cudaFuncSetAttribute(gram_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tc_smem<64>());
    if (kp == 128)
        return cudaFuncSetAttribute(gram_tc_kernel<128>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tc_smem<128>());
    return cudaErrorInvalidValue;
}

cudaError_t launch_gram_tc(const GramArgs &a, int *status, int max_ctas, cudaStream_t s) {
    if (a.y_end <= a.y_begin) return cudaSuccess;
    if (a.kp != 64 && a.kp != 128) return cudaErrorInvalidValue;
    const int TW = gram_tc_tile_width(a.kp), TH = gram_tc_tile_height(a.kp);
    const long long tiles =
        (long long)((a.nx + TW - 1) / TW) * ((a.y_end - a.y_begin + TH - 1) / TH);
    const unsigned grid = (unsigned)(tiles < max_ctas ? tiles : max_ctas);
    if (a.kp == 64)
        gram_tc_kernel<64><<<grid, kTcThreads, tc_smem<64>(), s>>>(a, status);
    else
        gram_tc_kernel<128><<<grid, kTcThreads, tc_smem<128>(), s>>>(a, status);
    return cudaGetLastError();
}

}  // namespace lk
