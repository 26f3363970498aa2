// Localized Gram matrices on the 5th-generation tensor cores (tcgen05), split FP16 with FP32
// accumulation: the mixed-precision form of
//     A_p = sum_o G_po / sigma_o^2  dy_o dy_o^T ,   c_p = sum_o G_po / sigma_o^2  dy_o (yo_o - ybar_o)
// (the k x k term of Eq. letkf_q and the vector of Eq. letkf_wa, R-localization of Sec. II-B).
//
// Symmetric form.  With x_po = sqrt(G_po) dy_o / sigma_o the Gram matrix of point p is
// A_p = X_p^T X_p, so one operand tile per point serves as both MMA operands.  X_p is split
// into FP16 parts X = Xh + Xl (Xl carries the rounding residual, ~22 significant bits in all)
// and A_p = Xh Xh^T + Xl Xh^T + (Xl Xh^T)^T; the Xl Xl^T term (relative size 2^-22) is dropped.
// The tile [Xl; Xh] (2 kp rows, K-major) gives with one M = 128 MMA per K-step
//     kp = 64:  D = [Xl; Xh] Xh^T  (128 x 64): rows 0..63 Xl Xh^T, rows 64..127 Xh Xh^T;
//     kp = 128: two MMAs, D_lh = Xl Xh^T and D_hh = Xh Xh^T (128 x 128 each);
//     kp = 32:  two grid points side by side form one 64-member operand X = [X_a | X_b] and
//               the kp = 64 MMA: the diagonal 32 x 32 blocks of X^T X are A_a and A_b (the
//               off-diagonal products X_a^T X_b are formed and discarded: the tensor pipe
//               is far from the kernel's bound).
// The epilogue forms A = D_hh + (D_lh + D_lh^T) through a shared-memory transpose.
// c_p = sum_o x_po (sqrt(G_po) (yo_o - ybar_o) / sigma_o) is accumulated in FP32 on the CUDA
// cores by the threads that build the operands.
//
// Warp roles of one persistent CTA per SM, linked by mbarrier rings (no block-wide barrier in
// the steady state):
//   warps 0, 1  candidates, alternating tiles, each through its own ring: walk the tile's
//               observation patch (bins of the cs x cs cell grid, contiguous runs of the
//               observation records per bin row), compute the square-root localization
//               weights of the tile's points, drop candidates that no point of the tile sees,
//               and publish segments of slots;
//   warp 2      MMA issue: one thread issues the tile's MMAs and commits them to mbarriers;
//   warp 3      loads: the slots' dy rows into a staging ring, 16-byte cp.async per lane;
//   warps 4..7  epilogue: tensor memory (double-buffered across tiles) -> A_p in global memory;
//   warps 8..15 operands: weights x dy rows, hi/lo split, core-matrix layout, and c_p.
// Every wait is bounded in time: on expiry the status word gets ST_TIMEOUT, all roles leave
// their loops, the CTA waits (bounded) for its MMAs and copies and frees its tensor memory.
// Candidate order and every summation order are fixed, so results are bitwise reproducible.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace lk {
namespace {

using namespace tc;

constexpr int kMetaWarps = 2, kWarpMma = 2, kWarpLoad = 3, kWarpEpi = 4, kWarpProd = 8;
constexpr int kEpiWarps = 4, kProdWarps = 8;
constexpr int kTcThreads = 32 * (kWarpProd + kProdWarps);  // 512
constexpr int kProdThreads = 32 * kProdWarps, kEpiThreads = 32 * kEpiWarps;
constexpr uint32_t kTmemCols = 512;
static_assert(kWarpEpi + kEpiWarps == kWarpProd, "warp roles");

template <int KP>
struct TcShape {
    static constexpr bool PAIR = KP == 32;                  // two points per operand tile
    static constexpr int KW = PAIR ? 64 : KP;               // members of one operand tile
    static constexpr int P = KP == 64 ? 4 : KP == 32 ? 8 : 1;   // grid points per tile
    static constexpr int PV = PAIR ? P / 2 : P;             // operand tiles per tile
    static constexpr int TW = KP == 128 ? 1 : (PAIR ? 4 : 2), TH = KP == 128 ? 1 : 2;
    static constexpr int KC = 32;                           // slots per chunk (MMA K)
    static constexpr int NOP = KP == 128 ? 4 : 2;           // operand stages
    static constexpr int NY = KP == 128 ? 4 : 8;            // dy staging stages
    static constexpr int SEG = KP == 128 ? 512 : 256;       // slots per candidate segment
    static constexpr int SBO = (KC / 8) * 128;              // bytes between 8-row core blocks
    static constexpr int OPB = 2 * KW * KC * 2;             // operand bytes per tile and stage
    static constexpr int STAGE = PV * OPB;
    static constexpr int YROW = KP * 4;                     // bytes of one staged dy row
    static constexpr int YSTAGE = KC * YROW;
    static constexpr int MQ = KW / 32;                      // member quarters of the producers
    static constexpr int KQ = kProdWarps / MQ;              // producer warps per member quarter
    static constexpr int NG = KC / 8, GPW = NG / KQ;        // 8-slot groups: per chunk, per warp
    static constexpr int ELD = KW + 1;                      // padded row of the transpose buffer
    static constexpr int OFF_OP = 0;
    static constexpr int OFF_Y = OFF_OP + NOP * STAGE;
    static constexpr int NMB = 2 * kMetaWarps;              // candidate buffers: 2 per ring
    static constexpr int OFF_GIDX = OFF_Y + NY * YSTAGE;    // int   [NMB][SEG]
    static constexpr int OFF_SW = OFF_GIDX + NMB * SEG * 4; // float [NMB][P][SEG]
    static constexpr int OFF_SU = OFF_SW + NMB * P * SEG * 4;  // float [NMB][P][SEG]
    static constexpr int OFF_E = OFF_SU + NMB * P * SEG * 4;   // float [KW][ELD]
    static constexpr int OFF_CRED = OFF_E + KW * ELD * 4;   // float [2][KQ][PV][KW]
    static constexpr int SMEM = OFF_CRED + 2 * KQ * PV * KW * 4;
    static_assert(SEG % KC == 0 && NG % KQ == 0, "chunking");
    static_assert(SMEM <= 227 * 1024 - 1024, "shared memory");
};

template <int KP>
__global__ void __launch_bounds__(kTcThreads, 1) gram_tc_kernel(GramArgs a, int *status,
                                                                 int tab_n) {
    using S = TcShape<KP>;
    constexpr int P = S::P, TW = S::TW, TH = S::TH, KC = S::KC, SEG = S::SEG;
    constexpr int NOP = S::NOP, NY = S::NY;
    extern __shared__ __align__(1024) unsigned char dyn[];
    __shared__ __align__(8) uint64_t meta_full[S::NMB], meta_empty[S::NMB];
    __shared__ __align__(8) uint64_t y_full[NY], y_empty[NY];
    __shared__ __align__(8) uint64_t op_full[NOP], op_empty[NOP];
    __shared__ __align__(8) uint64_t tm_full[2], tm_empty[2];
    __shared__ __align__(8) uint64_t prod_sync, epi_sync, mma_done;
    __shared__ int4 mdesc[S::NMB];  // segment: tile, slots, flags (1: first of tile, 2: last)
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const ObsNet &net = a.net;
    const int V = net.V;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rows = a.y_end - a.y_begin;
    const int ntx = (a.nx + TW - 1) / TW, nty = (rows + TH - 1) / TH;
    const int ntiles = ntx * nty;
    int *gidx_s = reinterpret_cast<int *>(dyn + S::OFF_GIDX);
    float *sw_s = reinterpret_cast<float *>(dyn + S::OFF_SW);
    float *su_s = reinterpret_cast<float *>(dyn + S::OFF_SU);
    float *ystage = reinterpret_cast<float *>(dyn + S::OFF_Y);
    float *E = reinterpret_cast<float *>(dyn + S::OFF_E);
    float *cred = reinterpret_cast<float *>(dyn + S::OFF_CRED);
    float *wtab = reinterpret_cast<float *>(dyn + S::SMEM);   // tab_n localization weights

    // ---- set-up: barriers, tensor memory, finite contents for every staged value
    if (tid == 0) {
        for (int i = 0; i < S::NMB; ++i) {
            bar_init(&meta_full[i], 32);
            bar_init(&meta_empty[i], 32 + 32 + kProdThreads);  // loader, MMA, producers
        }
        for (int i = 0; i < 2; ++i) {
            bar_init(&tm_full[i], 1);
            bar_init(&tm_empty[i], kEpiThreads);
        }
        for (int i = 0; i < NY; ++i) {
            bar_init(&y_full[i], 32);  // one arrival per loader lane, when its copies land
            bar_init(&y_empty[i], kProdThreads);
        }
        for (int i = 0; i < NOP; ++i) {
            bar_init(&op_full[i], kProdThreads);
            bar_init(&op_empty[i], 1);
        }
        bar_init(&prod_sync, kProdThreads);
        bar_init(&epi_sync, kEpiThreads);
        bar_init(&mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    for (int i = tid; i < (S::OFF_E - S::OFF_Y) / 4; i += kTcThreads)
        reinterpret_cast<float *>(dyn + S::OFF_Y)[i] = 0.0f;
    for (int i = tid; i < tab_n; i += kTcThreads) wtab[i] = weight_sqrt_d2(net, i);
    if (warp == kWarpMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    auto fail = [&]() {
        abort_flag = 1;
        if (lane == 0) atomicOr(status, ST_TIMEOUT);
    };
    auto tile_origin = [&](int tile, int &tx0, int &ty0) {
        tx0 = (tile % ntx) * TW;
        ty0 = a.y_begin + (tile / ntx) * TH;
    };

    if (warp < kMetaWarps) {
        // ===================== candidates and weights =====================
        // warp w serves the CTA's tiles w, w + 2, ... through its own ring of two buffers
        int segc = 0;
        const unsigned lt_mask = (1u << lane) - 1u;
        for (int tile = blockIdx.x + warp * gridDim.x; tile < ntiles && !abort_flag;
             tile += kMetaWarps * gridDim.x) {
            int tx0, ty0;
            tile_origin(tile, tx0, ty0);
            BinRanges rx, ry;
            if (net.loc_none) {
                rx.n = ry.n = 1;
                rx.lo[0] = ry.lo[0] = 0;
                rx.hi[0] = net.ncx - 1;
                ry.hi[0] = net.ncy - 1;
            } else {
                rx = bin_ranges(tx0 - net.cr, tx0 + TW - 1 + net.cr, a.nx, net.cs);
                ry = bin_ranges(ty0 - net.cr, ty0 + TH - 1 + net.cr, a.ny, net.cs);
            }
            int cnt_p[P];
#pragma unroll
            for (int p = 0; p < P; ++p) cnt_p[p] = 0;
            int mb = 2 * warp + (segc & 1), nfill = 0, first = 1;
            bool ok = wait_bar(&meta_empty[mb], ((segc >> 1) & 1) ^ 1, &abort_flag);
            // close the current segment (pad its last chunk with zero weights) and publish it
            auto publish = [&](int last) {
                const int pad_end = min(SEG, max(KC, (nfill + KC - 1) / KC * KC));
                for (int e = nfill + lane; e < pad_end; e += 32) {
                    gidx_s[mb * SEG + e] = -1;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        sw_s[(mb * P + p) * SEG + e] = 0.0f;
                        su_s[(mb * P + p) * SEG + e] = 0.0f;
                    }
                }
                if (lane == 0) mdesc[mb] = make_int4(tile, nfill, first | (last ? 2 : 0), 0);
                __syncwarp();
                bar_arrive(&meta_full[mb]);
                ++segc;
                first = 0;
            };
            // Ranges of records: two slots per bin row of the patch (its x ranges, the second
            // empty unless the row's range wraps), in that order.  A bin row's x range spans the
            // bins within the cutoff at the row's distance from the tile (a disk, not the
            // bounding square: the dropped bins hold no local observation).  32 ranges at a
            // time, every lane fetches one
            // range's bounds; the slots of the batch are then walked as one flat list, 32 per
            // step, with the next step's record fetched ahead.
            const int ly0 = ry.hi[0] - ry.lo[0] + 1;
            const int nyb = ly0 + (ry.n > 1 ? ry.hi[1] - ry.lo[1] + 1 : 0);
            const int nr = nyb * 2;
            for (int rb = 0; rb < nr && ok; rb += 32) {
                int j0 = 0, cnt = 0;
                if (rb + lane < nr) {
                    const int yi = (rb + lane) >> 1, xr = (rb + lane) & 1;
                    const int by = yi < ly0 ? ry.lo[0] + yi : ry.lo[1] + (yi - ly0);
                    BinRanges rr = rx;
                    if (!net.loc_none) {
                        const int gy = axis_gap(by * net.cs, min((by + 1) * net.cs, a.ny) - 1,
                                                ty0, ty0 + TH - 1, a.ny);
                        const long long rem = (long long)net.d2max - (long long)gy * gy;
                        if (rem < 0) {
                            rr.n = 0;
                        } else {
                            long long w = (long long)sqrt((double)rem);
                            while ((w + 1) * (w + 1) <= rem) ++w;
                            while (w * w > rem) --w;
                            rr = bin_ranges(tx0 - (int)w, tx0 + TW - 1 + (int)w, a.nx, net.cs);
                        }
                    }
                    if (xr < rr.n) {
                        const int blo = xr ? rr.lo[1] : rr.lo[0], bhi = xr ? rr.hi[1] : rr.hi[0];
                        const int c0 = by * net.ncx + blo;
                        j0 = __ldg(net.cell_start + c0) * V;
                        cnt = __ldg(net.cell_start + c0 + (bhi - blo) + 1) * V - j0;
                    }
                }
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                // record index of flat slot f of this batch (f < tot)
                auto record_of = [&](int f) -> int {
                    int lo = 0;  // first range whose inclusive end exceeds f
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int e = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                        if (e <= f) lo += step;
                    }
                    const int e_lo = __shfl_sync(0xffffffffu, incl, lo);
                    const int c_lo = __shfl_sync(0xffffffffu, cnt, lo);
                    const int b_lo = __shfl_sync(0xffffffffu, j0, lo);
                    return b_lo + (f - (e_lo - c_lo));
                };
                float4 rn = make_float4(0.f, 0.f, 0.f, 0.f);
                {
                    const int jn = record_of(min(lane, max(tot - 1, 0)));
                    if (lane < tot) rn = __ldg(a.orec + jn);
                }
                for (int fb = 0; fb < tot; fb += 32) {
                    const float4 r = rn;
                    const bool in = fb + lane < tot;
                    if (fb + 32 < tot) {
                        const int jn = record_of(min(fb + 32 + lane, tot - 1));
                        if (fb + 32 + lane < tot) rn = __ldg(a.orec + jn);
                    }
                    const int sv = __float_as_int(r.x), pk = __float_as_int(r.y);
                    const int s = sv & 0x0FFFFFFF;
                    const bool first_var = (sv >> 28) == 0;
                    const int ox = pk & 0xffff, oy = (int)((unsigned)pk >> 16);
                    float sw[P];
                    bool keep = false;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const int qx = tx0 + p % TW, qy = ty0 + p / TW;
                        float w = 0.0f;
                        if (in && qx < a.nx && qy < a.y_end)
                            w = loc_weight_sqrt(net, ox, oy, qx, qy, a.nx, a.ny, wtab, tab_n);
                        keep |= w != 0.0f;
                        if (w != 0.0f && first_var) ++cnt_p[p];
                        sw[p] = w * r.z;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    const int n = __popc(bal);
                    if (n == 0) continue;
                    if (nfill + n > SEG) {
                        publish(0);
                        mb = 2 * warp + (segc & 1);
                        nfill = 0;
                        ok = wait_bar(&meta_empty[mb], ((segc >> 1) & 1) ^ 1, &abort_flag);
                        if (!ok) break;
                    }
                    if (keep) {
                        const int e = nfill + __popc(bal & lt_mask);
                        gidx_s[mb * SEG + e] = s;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            sw_s[(mb * P + p) * SEG + e] = sw[p];
                            su_s[(mb * P + p) * SEG + e] = sw[p] * r.w;
                        }
                    }
                    nfill += n;
                }
            }
            if (!ok) {
                fail();
                break;
            }
            publish(1);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                int c = cnt_p[p];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                const int qx = tx0 + p % TW, qy = ty0 + p / TW;
                if (lane == 0 && qx < a.nx && qy < a.y_end)
                    a.nloc[(size_t)(qy - a.y_begin) * a.nx + qx] = c;
            }
        }
    } else if (warp == kWarpLoad) {
        // ===================== dy rows into the staging ring =====================
        // 16-byte cp.async per lane; each lane's arrival on y_full[s] fires once its copies
        // have landed (cp.async.mbarrier.arrive.noinc)
        constexpr int PARTS = S::YROW / 16;  // 16-byte pieces of one row
        int segc[2] = {0, 0}, tcount = 0;
        uint32_t g = 0;
        for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x, ++tcount) {
            const int ring = tcount & 1;
            bool last = false, ok = true;
            while (!last && ok) {
                const int mb = 2 * ring + (segc[ring] & 1);
                if (!(ok = wait_bar(&meta_full[mb], (segc[ring] >> 1) & 1, &abort_flag))) break;
                const int4 d = mdesc[mb];
                last = (d.z & 2) != 0;
                const int nch = max(1, (d.y + KC - 1) / KC);
                for (int ch = 0; ch < nch; ++ch, ++g) {
                    const int s = g % NY;
                    if (!(ok = wait_bar(&y_empty[s], ((g / NY) & 1) ^ 1, &abort_flag))) break;
                    const int cnt = min(KC, d.y - ch * KC);
                    const uint32_t dst = smem_u32(ystage + (size_t)s * (S::YSTAGE / 4));
#pragma unroll 4
                    for (int it = lane; it < KC * PARTS; it += 32) {
                        const int kk = it / PARTS, part = it - kk * PARTS;
                        if (kk < cnt) {
                            const int row = gidx_s[mb * SEG + ch * KC + kk];
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                             dst + (uint32_t)(kk * S::YROW + part * 16)),
                                         "l"(a.yb + (size_t)row * KP + part * 4)
                                         : "memory");
                        }
                    }
                    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                                     smem_u32(&y_full[s]))
                                 : "memory");
                }
                if (!ok) break;
                bar_arrive(&meta_empty[mb]);
                ++segc[ring];
            }
            if (!ok) {
                fail();
                break;
            }
        }
        // every issued copy has landed before the CTA may exit
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == kWarpMma) {
        // ===================== tensor-core issue =====================
        int segc[2] = {0, 0}, tcount = 0;
        uint32_t g = 0;
        const uint32_t op0 = smem_u32(dyn + S::OFF_OP);
        for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x, ++tcount) {
            const int tb = tcount & 1;
            bool last = false, ok = true, firstc = true;
            const int ring = tcount & 1;
            while (!last && ok) {
                const int mb = 2 * ring + (segc[ring] & 1);
                if (!(ok = wait_bar(&meta_full[mb], (segc[ring] >> 1) & 1, &abort_flag))) break;
                const int4 d = mdesc[mb];
                last = (d.z & 2) != 0;
                const int nch = max(1, (d.y + KC - 1) / KC);
                for (int ch = 0; ch < nch; ++ch, ++g) {
                    const int so = g % NOP;
                    if (!(ok = wait_bar(&op_full[so], (g / NOP) & 1, &abort_flag))) break;
                    if (firstc &&
                        !(ok = wait_bar(&tm_empty[tb], ((tcount >> 1) & 1) ^ 1, &abort_flag)))
                        break;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    if (lane == 0) {
                        const uint32_t st = op0 + so * S::STAGE;
#pragma unroll
                        for (int ks = 0; ks < KC / 16; ++ks) {
                            const uint32_t acc = (firstc && ks == 0) ? 0u : 1u;
#pragma unroll
                            for (int p = 0; p < S::PV; ++p) {
                                const uint32_t tp = st + p * S::OPB + ks * 256;
                                const uint64_t dl = sdesc(tp, S::SBO);
                                const uint64_t dh = sdesc(tp + (S::KW / 8) * S::SBO, S::SBO);
                                if (S::KW == 64) {
                                    mma_f16(tmem + tb * 256 + p * 64, dl, dh, idesc_f16(128, 64),
                                            acc);
                                } else {
                                    mma_f16(tmem + tb * 256, dl, dh, idesc_f16(128, 128), acc);
                                    mma_f16(tmem + tb * 256 + 128, dh, dh, idesc_f16(128, 128),
                                            acc);
                                }
                            }
                        }
                        mma_commit(&op_empty[so]);
                        if (last && ch == nch - 1) mma_commit(&tm_full[tb]);
                    }
                    __syncwarp();
                    firstc = false;
                }
                if (!ok) break;
                bar_arrive(&meta_empty[mb]);
                ++segc[ring];
            }
            if (!ok) {
                fail();
                break;
            }
        }
        // all MMAs issued by this CTA complete before its tensor memory is freed (bounded)
        if (lane == 0) mma_commit(&mma_done);
        __syncwarp();
        volatile int no_abort = 0;
        if (!wait_bar(&mma_done, 0, &no_abort)) fail();
    } else if (warp < kWarpEpi + kEpiWarps) {
        // ===================== epilogue: tensor memory -> A_p =====================
        const int eq = warp & 3;           // tensor-memory lane quadrant of this warp
        const int r = 32 * eq + lane;      // accumulator row of this thread
        const uint32_t lane_base = tmem + ((uint32_t)(32 * eq) << 16);
        int tcount = 0;
        uint32_t esync = 0;
        bool ok = true;
        auto epi_barrier = [&]() {
            bar_arrive(&epi_sync);
            ok = wait_bar(&epi_sync, esync & 1, &abort_flag);
            ++esync;
        };
        for (int tile = blockIdx.x; tile < ntiles && !abort_flag && ok;
             tile += gridDim.x, ++tcount) {
            const int tb = tcount & 1;
            if (!(ok = wait_bar(&tm_full[tb], (tcount >> 1) & 1, &abort_flag))) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            int tx0, ty0;
            tile_origin(tile, tx0, ty0);
            for (int p = 0; p < S::PV && ok; ++p) {
                const int qx = tx0 + p % TW, qy = ty0 + p / TW;
                const bool valid = qx < a.nx && qy < a.y_end;
                const size_t lp = valid ? (size_t)(qy - a.y_begin) * a.nx + qx : 0;
                float v[32];
                if (S::PAIR) {
                    // operand tile p holds points 2p (members 0..31) and 2p + 1 (32..63):
                    // row m of the 64 x 64 product belongs to point 2p + m / 32, and only its
                    // diagonal 32 x 32 block is kept
                    const uint32_t col = tb * 256 + p * 64;
                    if (eq < 2) {  // rows of Xl Xh^T
#pragma unroll
                        for (int c0 = 0; c0 < 64; c0 += 32) {
                            tmem_ld32(lane_base + col + c0, v);
#pragma unroll
                            for (int i = 0; i < 32; ++i) E[r * S::ELD + c0 + i] = v[i];
                        }
                    }
                    epi_barrier();
                    if (!ok) break;
                    if (eq >= 2) {  // rows of Xh Xh^T
                        const int m = r - 64, half = m >> 5, mm = m & 31, c0 = 32 * half;
                        const int pr = 2 * p + half;
                        const int rx = tx0 + pr % TW, ry = ty0 + pr / TW;
                        const bool rvalid = rx < a.nx && ry < a.y_end;
                        const size_t rlp = rvalid ? (size_t)(ry - a.y_begin) * a.nx + rx : 0;
                        tmem_ld32(lane_base + col + c0, v);
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            v[i] += E[m * S::ELD + c0 + i] + E[(c0 + i) * S::ELD + m];
                        if (rvalid && mm < a.k)
                            store_row32(a.gram + rlp * a.k * a.k + (size_t)mm * a.k, v, 0, a.k);
                    }
                    epi_barrier();
                } else if (KP == 64) {
                    const uint32_t col = tb * 256 + p * 64;
                    if (eq < 2) {  // rows of Xl Xh^T
#pragma unroll
                        for (int c0 = 0; c0 < 64; c0 += 32) {
                            tmem_ld32(lane_base + col + c0, v);
#pragma unroll
                            for (int i = 0; i < 32; ++i) E[r * S::ELD + c0 + i] = v[i];
                        }
                    }
                    epi_barrier();
                    if (!ok) break;
                    if (eq >= 2) {  // rows of Xh Xh^T
                        const int m = r - 64;
                        float *dst = a.gram + lp * a.k * a.k + (size_t)m * a.k;
#pragma unroll
                        for (int c0 = 0; c0 < 64; c0 += 32) {
                            tmem_ld32(lane_base + col + c0, v);
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                v[i] += E[m * S::ELD + c0 + i] + E[(c0 + i) * S::ELD + m];
                            if (valid && m < a.k) store_row32(dst, v, c0, a.k);
                        }
                    }
                    epi_barrier();
                } else {
                    const uint32_t col = tb * 256;
#pragma unroll 1
                    for (int c0 = 0; c0 < 128; c0 += 32) {  // D_lh row r
                        tmem_ld32(lane_base + col + c0, v);
#pragma unroll
                        for (int i = 0; i < 32; ++i) E[r * S::ELD + c0 + i] = v[i];
                    }
                    epi_barrier();
                    if (!ok) break;
                    float *dst = a.gram + lp * a.k * a.k + (size_t)r * a.k;
#pragma unroll 1
                    for (int c0 = 0; c0 < 128; c0 += 32) {  // D_hh row r
                        tmem_ld32(lane_base + col + 128 + c0, v);
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            v[i] += E[r * S::ELD + c0 + i] + E[(c0 + i) * S::ELD + r];
                        if (valid && r < a.k) store_row32(dst, v, c0, a.k);
                    }
                    epi_barrier();
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            bar_arrive(&tm_empty[tb]);
        }
        if (!ok) fail();
    } else {
        // ===================== operands and c_p =====================
        const int pw = warp - kWarpProd;
        const int mq = pw % S::MQ, kq = pw / S::MQ;
        const int m = 32 * mq + lane;               // member of the operand tile
        const int mr = S::PAIR ? lane : m;          // member of its grid point
        unsigned char *op = dyn + S::OFF_OP;
        int segc[2] = {0, 0}, par = 0, tcount = 0;
        uint32_t g = 0, psync = 0;
        float cacc[S::PV];
#pragma unroll
        for (int p = 0; p < S::PV; ++p) cacc[p] = 0.0f;
        for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x, ++tcount) {
            const int ring = tcount & 1;
            bool last = false, ok = true;
            while (!last && ok) {
                const int mb = 2 * ring + (segc[ring] & 1);
                if (!(ok = wait_bar(&meta_full[mb], (segc[ring] >> 1) & 1, &abort_flag))) break;
                const int4 d = mdesc[mb];
                last = (d.z & 2) != 0;
                if (d.z & 1) {
#pragma unroll
                    for (int p = 0; p < S::PV; ++p) cacc[p] = 0.0f;
                }
                const int nch = max(1, (d.y + KC - 1) / KC);
                for (int ch = 0; ch < nch; ++ch, ++g) {
                    const int s = g % NY, so = g % NOP;
                    if (!(ok = wait_bar(&y_full[s], (g / NY) & 1, &abort_flag))) break;
                    if (!(ok = wait_bar(&op_empty[so], ((g / NOP) & 1) ^ 1, &abort_flag))) break;
                    const int first = ch * KC, cnt = min(KC, d.y - first);
                    const float *ys = ystage + (size_t)s * (S::YSTAGE / 4);
                    unsigned char *st = op + so * S::STAGE;
#pragma unroll
                    for (int gi = 0; gi < S::GPW; ++gi) {
                        const int k8 = 8 * (kq + S::KQ * gi);
                        float yv[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            yv[i] = k8 + i < cnt ? ys[(k8 + i) * KP + mr] : 0.0f;
#pragma unroll
                        for (int p = 0; p < S::PV; ++p) {
                            const int pp = S::PAIR ? 2 * p + mq : p;   // the grid point
                            const float *wp = sw_s + (mb * P + pp) * SEG + first + k8;
                            const float *up = su_s + (mb * P + pp) * SEG + first + k8;
                            const float4 w0 = *reinterpret_cast<const float4 *>(wp);
                            const float4 w1 = *reinterpret_cast<const float4 *>(wp + 4);
                            const float4 u0 = *reinterpret_cast<const float4 *>(up);
                            const float4 u1 = *reinterpret_cast<const float4 *>(up + 4);
                            const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                            const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                            // pairs of slots with packed FP32 instructions (each lane rounds
                            // as the scalar operation); c in two chains (even, odd slots)
                            uint32_t hw[4], lw[4];
                            float2 c2 = make_float2(cacc[p], 0.0f);
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const float2 x = __fmul2_rn(make_float2(yv[2 * i], yv[2 * i + 1]),
                                                            make_float2(w[2 * i], w[2 * i + 1]));
                                const __half2 h = __floats2half2_rn(x.x, x.y);
                                const float2 hf = __half22float2(h);
                                const float2 r = __ffma2_rn(hf, make_float2(-1.0f, -1.0f), x);
                                const __half2 l = __floats2half2_rn(r.x, r.y);
                                hw[i] = *reinterpret_cast<const uint32_t *>(&h);
                                lw[i] = *reinterpret_cast<const uint32_t *>(&l);
                                c2 = __ffma2_rn(x, make_float2(u[2 * i], u[2 * i + 1]), c2);
                            }
                            cacc[p] = c2.x + c2.y;
                            unsigned char *tp = st + p * S::OPB;
                            *reinterpret_cast<uint4 *>(tp + core_off_b<KC>(S::KW + m, k8)) =
                                make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            *reinterpret_cast<uint4 *>(tp + core_off_b<KC>(m, k8)) =
                                make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_arrive(&op_full[so]);
                    bar_arrive(&y_empty[s]);
                }
                if (!ok) break;
                bar_arrive(&meta_empty[mb]);
                ++segc[ring];
            }
            if (!ok) {
                fail();
                break;
            }
            // ---- c_p: partial sums of the KQ warps sharing a member quarter
#pragma unroll
            for (int p = 0; p < S::PV; ++p)
                cred[((par * S::KQ + kq) * S::PV + p) * S::KW + m] = cacc[p];
            bar_arrive(&prod_sync);
            if (!wait_bar(&prod_sync, psync & 1, &abort_flag)) {
                fail();
                break;
            }
            ++psync;
            if (kq == 0) {
                int tx0, ty0;
                tile_origin(tile, tx0, ty0);
#pragma unroll
                for (int p = 0; p < S::PV; ++p) {
                    float c = 0.0f;
#pragma unroll
                    for (int q = 0; q < S::KQ; ++q)
                        c += cred[((par * S::KQ + q) * S::PV + p) * S::KW + m];
                    const int pp = S::PAIR ? 2 * p + mq : p;
                    const int qx = tx0 + pp % TW, qy = ty0 + pp / TW;
                    if (mr < a.k && qx < a.nx && qy < a.y_end)
                        a.cvec[((size_t)(qy - a.y_begin) * a.nx + qx) * a.k + mr] = c;
                }
            }
            par ^= 1;
        }
    }

    // ---- stop: every role has left its loop; free the tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == kWarpMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

// Observation records in bin order: slot j = V * (position in cell_obs) + v holds the row s
// of the scalar in dy with v in bits 28..29, the packed point (x | y << 16), 1 / sigma and
// yo - reference - ybar.
__global__ void obs_records_kernel(ObsNet net, const float *rinv, const float *yo,
                                   const float *ybar, float r0, float r1, float r2,
                                   float4 *rec) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= net.L * net.V) return;
    const int o = net.cell_obs[j / net.V], v = j % net.V, s = o * net.V + v;
    const int2 xy = net.xy[o];
    const float ref = v == 0 ? r0 : (v == 1 ? r1 : r2);
    rec[j] = make_float4(__int_as_float(s | (v << 28)), __int_as_float(xy.x | (xy.y << 16)),
                         sqrtf(rinv[s]), (yo[s] - ref) - ybar[s]);
}

}  // namespace

int gram_tc_tile_width(int kp) {
    return kp == 32 ? TcShape<32>::TW : kp == 64 ? TcShape<64>::TW : TcShape<128>::TW;
}
int gram_tc_tile_height(int kp) {
    return kp == 32 ? TcShape<32>::TH : kp == 64 ? TcShape<64>::TH : TcShape<128>::TH;
}

// dynamic shared memory a CTA may use: the kernel's buffers plus the weight table
constexpr int kTcDynMax = 227 * 1024 - 1024;

// entries of the localization-weight table for the launch (d2max + 1 where it fits beside
// the buffers, else 0: the weights are then evaluated per candidate)
template <int KP>
int wtab_entries(const GramArgs &a) {
    if (a.net.loc_none || a.net.d2max < 0) return 0;
    const long long n = (long long)a.net.d2max + 1;
    return (long long)TcShape<KP>::SMEM + 4 * n <= kTcDynMax ? (int)n : 0;
}

cudaError_t gram_tc_prepare(int kp) {
    if (kp == 32)
        return cudaFuncSetAttribute(gram_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kTcDynMax);
    if (kp == 64)
        return cudaFuncSetAttribute(gram_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kTcDynMax);
    if (kp == 128)
        return cudaFuncSetAttribute(gram_tc_kernel<128>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kTcDynMax);
    return cudaErrorInvalidValue;
}

cudaError_t launch_obs_records(const GramArgs &a, float4 *rec, cudaStream_t s) {
    const int n = a.net.L * a.net.V;
    if (n == 0) return cudaSuccess;
    obs_records_kernel<<<(n + 255) / 256, 256, 0, s>>>(a.net, a.rinv, a.yo, a.ybar, a.yref[0],
                                                        a.yref[1], a.yref[2], rec);
    return cudaGetLastError();
}

cudaError_t launch_gram_tc(const GramArgs &a, int *status, int max_ctas, cudaStream_t s) {
    if (a.y_end <= a.y_begin) return cudaSuccess;
    if (a.kp != 32 && a.kp != 64 && a.kp != 128) return cudaErrorInvalidValue;
    if (a.orec == nullptr) return cudaErrorInvalidValue;
    const int TW = gram_tc_tile_width(a.kp), TH = gram_tc_tile_height(a.kp);
    const long long tiles =
        (long long)((a.nx + TW - 1) / TW) * ((a.y_end - a.y_begin + TH - 1) / TH);
    const unsigned grid = (unsigned)(tiles < max_ctas ? tiles : max_ctas);
    // Each CTA needs an SM to itself (~190 KB of shared memory, all tensor-memory columns).
    // Launched at the device's highest priority, its CTAs are placed ahead of the pending
    // blocks of other streams as SMs drain, instead of waiting behind kernels with small
    // blocks that keep refilling them (several handles sharing the GPU).
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = hi;  // numerically lowest = highest priority
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTcThreads);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a.kp == 32) {
        const int n = wtab_entries<32>(a);
        cfg.dynamicSmemBytes = TcShape<32>::SMEM + 4 * n;
        return cudaLaunchKernelEx(&cfg, gram_tc_kernel<32>, a, status, n);
    }
    if (a.kp == 64) {
        const int n = wtab_entries<64>(a);
        cfg.dynamicSmemBytes = TcShape<64>::SMEM + 4 * n;
        return cudaLaunchKernelEx(&cfg, gram_tc_kernel<64>, a, status, n);
    }
    const int n = wtab_entries<128>(a);
    cfg.dynamicSmemBytes = TcShape<128>::SMEM + 4 * n;
    return cudaLaunchKernelEx(&cfg, gram_tc_kernel<128>, a, status, n);
}

}  // namespace lk
