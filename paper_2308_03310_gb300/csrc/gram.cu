// Localized Gram matrix and innovation projection at every grid point (FP32, CUDA cores).
//
// For grid point p with local observations o (R-localization, Sec. II-B):
//     A_p = sum_o G_po / sigma_o^2  dy_o dy_o^T        (the k x k term of Eq. letkf_q)
//     c_p = sum_o G_po / sigma_o^2  dy_o (yo_o - ybar_o) (the vector of Eq. letkf_wa)
// with G_po = exp(-d^2 / (2 r^2)) for integer periodic d^2 <= d2max, else 0.
//
// Design (GB300): a CTA owns a TW x TH tile of grid points and a team of KB (KB + 1) / 2
// threads per point (KB = KP / 8), each thread accumulating one 8 x 8 block (ti, tj), ti <= tj,
// of A_p in registers: A is symmetric and the eigensolve reads only its upper triangle and
// diagonal, so only the upper blocks are formed (36 of 64 at KP = 64; the diagonal blocks'
// threads also accumulate c).  The CTA gathers the observation patch of its tile once -- the
// observations of every bin (cs x cs cell) that the tile's cutoff disks touch -- and stages it
// through shared memory 64 observation points at a time: their perturbation rows dy_o (k
// floats each, read from L2, where the whole dY lives), innovations and inverse variances.
// The weight of each (point, observation) pair is computed once per chunk into shared memory;
// a team skips observations outside its point's cutoff.  Nothing per-point is materialized in
// HBM except the upper triangle of the k x k result (the paper's padded Y_loc[M, N_x, l_max V]
// array is never formed).  Summation order is fixed by the bin order and the interleaving of
// the chunks, so results are bitwise reproducible.
#include "common.cuh"
#include "kernels.h"
#include "patch.cuh"

namespace lk {
namespace {

constexpr int kChunk = 64;  // observation points per staged chunk

// Staged dy rows are stored with their 16-byte pieces permuted: piece 2 b + h (h = 0, 1: the
// two halves of the 8-float block b) goes to position h KB + b.  A warp's 16-byte loads of the
// first (or second) halves of up to 8 distinct blocks then fall in distinct bank groups
// (position mod 8), where the natural order put blocks b and b + 4 in the same group.
template <int KB>
__device__ __forceinline__ int piece_pos(int c4) {
    return (c4 & 1) * KB + (c4 >> 1);
}

template <int KP>
struct GramShape {
    static constexpr int KB = KP / 8;
    static constexpr int T = KB * (KB + 1) / 2;   // threads per grid point (upper blocks)
    // grid points per CTA: about 256-320 threads, a rectangle of points
    static constexpr int P = KP == 8 ? 256 : KP == 16 ? 64 : KP == 32 ? 32 : KP == 64 ? 8 : 2;
    static constexpr int TW = KP == 8 ? 16 : KP == 16 ? 8 : KP == 32 ? 8 : KP == 64 ? 4 : 2;
    static constexpr int TH = P / TW;
    static constexpr int NT = (P * T + 31) / 32 * 32;   // threads per CTA, whole warps (two
                                                        // CTAs resident per SM)
    static_assert(TW * TH == P, "tile");
};

// (ti, tj) of upper block r, row-major over ti <= tj < KB
template <int KB>
__device__ __forceinline__ void upper_block(int r, int &ti, int &tj) {
    int i = 0, rem = r;
    while (rem >= KB - i) {
        rem -= KB - i;
        ++i;
    }
    ti = i;
    tj = i + rem;
}

// VV: observed variables per point (1..3), a template parameter so the per-scalar loop unrolls
template <int KP, int VV>
__global__ void __launch_bounds__(GramShape<KP>::NT, 2) gram_kernel(GramArgs a) {
    using S = GramShape<KP>;
    constexpr int KB = S::KB, T = S::T, P = S::P, TW = S::TW, TH = S::TH, NT = S::NT;
    constexpr int V = VV;

    __shared__ int cell_base[kMaxPatchCells];
    __shared__ int cell_pre[kMaxPatchCells + 1];
    __shared__ int warp_tot[NT / 32];
    __shared__ int2 opos[kChunk];
    __shared__ int oidx[kChunk];
    __shared__ float dv[kChunk * 3];
    __shared__ float rv[kChunk * 3];
    extern __shared__ float4 dyn4[];
    float *ys = reinterpret_cast<float *>(dyn4);       // [kChunk * V][KP]
    float *wts = ys + kChunk * 3 * KP;                 // [P][kChunk]

    const ObsNet &net = a.net;
    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * TW;
    const int ty0 = a.y_begin + blockIdx.y * TH;

    // ---- the tile's observation patch: bins touched by any cutoff disk of the tile
    const int nc = build_patch<NT>(net, a.nx, a.ny, tx0, ty0, TW, TH, cell_base, cell_pre,
                                   warp_tot);
    const int total = cell_pre[nc];

    // ---- this thread's role: point p of the tile, upper 8 x 8 block (ti, tj) of A_p
    const int p = tid / T, r = tid - (tid / T) * T;
    int ti = 0, tj = 0;
    upper_block<KB>(r, ti, tj);
    const int px = tx0 + p % TW, py = ty0 + p / TW;
    const bool valid = p < P && px < a.nx && py < a.y_end;
    const bool diag_block = ti == tj;

    float2 acc[8][4];    // acc[i][jp] = (A[i][2 jp], A[i][2 jp + 1]) of the block
    float2 cacc[4];      // (c[2 ip], c[2 ip + 1])
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) cacc[i] = make_float2(0.0f, 0.0f);
    int nl = 0;

    // chunk c takes the candidates c, c + nck, c + 2 nck, ... of the patch: a uniform sample
    // of it, so that every point of the tile finds about the same share of its local
    // observations in every chunk (in patch order the share swings with the chunk's place, and
    // the block barrier between chunks waits for the busiest point's team)
    const int nck = (total + kChunk - 1) / kChunk;
    for (int ck = 0; ck < nck; ++ck) {
        const int nch = (total - ck + nck - 1) / nck;
        if (tid < nch) {
            const int o = patch_obs(net, cell_base, cell_pre, nc, ck + tid * nck);
            oidx[tid] = o;
            opos[tid] = net.xy[o];
            for (int v = 0; v < V; ++v) {
                const int s = o * V + v;
                dv[tid * V + v] = (a.yo[s] - a.yref[v]) - a.ybar[s];
                rv[tid * V + v] = a.rinv[s];
            }
        }
        __syncthreads();
        // perturbation rows of the chunk: nch * V rows of KP floats, 16-byte copies
        constexpr int Q4 = KP / 4;
        for (int e = tid; e < nch * V * Q4; e += NT) {
            const int row = e / Q4, c4 = e % Q4;
            const int s = oidx[row / V] * V + row % V;
            reinterpret_cast<float4 *>(ys + row * KP)[piece_pos<KB>(c4)] =
                __ldg(reinterpret_cast<const float4 *>(a.yb + (size_t)s * KP) + c4);
        }
        // localization weights of every (point, observation) pair of the chunk
        for (int e = tid; e < P * nch; e += NT) {
            const int pp = e / nch, t = e % nch;
            const int qx = tx0 + pp % TW, qy = ty0 + pp / TW;
            const float w = (qx < a.nx && qy < a.y_end) ? loc_weight(net, opos[t], qx, qy, a.nx, a.ny)
                                                        : 0.0f;
            wts[pp * kChunk + t] = w;
        }
        __syncthreads();
        if (valid) {
            for (int t = 0; t < nch; ++t) {
                const float w = wts[p * kChunk + t];
                if (w == 0.0f) continue;
                nl += (r == 0);
#pragma unroll 1
                for (int v = 0; v < V; ++v) {
                    // the same multiply-adds as one fmaf per element, two per instruction
                    // (packed FP32: identical roundings)
                    const float sw = w * rv[t * V + v];
                    const float4 *row = reinterpret_cast<const float4 *>(ys + (t * V + v) * KP);
                    const float4 a0 = row[ti], a1 = row[KB + ti];
                    const float4 b0 = row[tj], b1 = row[KB + tj];
                    const float2 sw2 = make_float2(sw, sw);
                    const float2 sa2[4] = {__fmul2_rn(sw2, make_float2(a0.x, a0.y)),
                                           __fmul2_rn(sw2, make_float2(a0.z, a0.w)),
                                           __fmul2_rn(sw2, make_float2(a1.x, a1.y)),
                                           __fmul2_rn(sw2, make_float2(a1.z, a1.w))};
                    const float2 b2[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                                          make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
                    const float dvs = dv[t * V + v];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float sa = (i & 1) ? sa2[i >> 1].y : sa2[i >> 1].x;
                        const float2 s2 = make_float2(sa, sa);
#pragma unroll
                        for (int jp = 0; jp < 4; ++jp) acc[i][jp] = __ffma2_rn(s2, b2[jp], acc[i][jp]);
                    }
                    if (diag_block) {
                        const float2 d2 = make_float2(dvs, dvs);
#pragma unroll
                        for (int ip = 0; ip < 4; ++ip) cacc[ip] = __ffma2_rn(sa2[ip], d2, cacc[ip]);
                    }
                }
            }
        }
        __syncthreads();
    }

    if (!valid) return;
    const size_t lp = (size_t)(py - a.y_begin) * a.nx + px;
    const int k = a.k;
    float *A = a.gram + lp * k * k;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = ti * 8 + i;
        if (row >= k) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = tj * 8 + j;
            if (col < k && col >= row) A[row * k + col] = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
        }
        if (diag_block) a.cvec[lp * k + row] = (i & 1) ? cacc[i >> 1].y : cacc[i >> 1].x;
    }
    if (r == 0) a.nloc[lp] = nl;
}

// ---- the pipelined form (k >= 17: KP = 32, 64, 128) ---------------------------------------
//
// One CTA per SM over a TW x TH tile of points, a team of KB (KB + 1) / 2 threads per point as
// in the team kernel, at most 16 warps: a scheduler's 16,384 registers then hold four warps
// of up to 128 registers, room for the next entry's operands beside the 64 accumulators.  Per
// chunk of CH candidates, one warp per point compacts its local (row, weight) entries in
// candidate order (a ballot over the localization weights), so the multiply-add loop has no
// branch and loads the next entry's operands while it multiplies the current ones.  The
// candidates' indices are copied into shared memory two chunks ahead and their rows and
// metadata one chunk ahead (cp.async, double buffered), so the copies overlap the arithmetic.

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int KP>
struct PipeShape {
    static constexpr int KB = KP / 8;
    static constexpr int T = KB * (KB + 1) / 2;                  // threads per point
    static constexpr int TW = KP == 32 ? 8 : KP == 64 ? 7 : 3;
    static constexpr int TH = KP == 32 ? 6 : KP == 64 ? 2 : 1;
    static constexpr int P = TW * TH;                            // 48 / 14 / 3 points
    static constexpr int NT = (P * T + 31) / 32 * 32;            // 480 / 512 / 416 threads
    static constexpr int CH = KP == 128 ? 32 : 64;               // candidates per chunk
    static_assert(NT <= 512, "at most 16 warps");
    static_assert(CH <= 64, "two ballots per point");
};

template <int KP, int VV>
struct PipeSmem {
    using S = PipeShape<KP>;
    static constexpr int R = S::CH * VV;                  // rows per chunk
    static constexpr int rows = 0;                        // [2][R][KP]
    static constexpr int ent = rows + 2 * R * KP;         // [P][R] float2 (row, sw)
    static constexpr int entd = ent + 2 * S::P * R;       // [P][R] sw * dv
    static constexpr int xy = entd + S::P * R;            // [2][CH] int2
    static constexpr int yo = xy + 4 * S::CH;             // [2][R]
    static constexpr int yb = yo + 2 * R;                 // [2][R]
    static constexpr int ri = yb + 2 * R;                 // [2][R]
    static constexpr int oidx = ri + 2 * R;               // [2][CH]
    static constexpr int floats = oidx + 2 * S::CH;
    static_assert(ent % 4 == 0 && xy % 2 == 0, "alignment");
};

template <int KP, int VV>
__global__ void __launch_bounds__(PipeShape<KP>::NT, 1) gram_pipe_kernel(GramArgs a) {
    using S = PipeShape<KP>;
    using M = PipeSmem<KP, VV>;
    constexpr int KB = S::KB, P = S::P, TW = S::TW, TH = S::TH, NT = S::NT, CH = S::CH;
    constexpr int V = VV, R = M::R, Q4 = KP / 4;

    __shared__ int cell_base[kMaxPatchCells];
    __shared__ int cell_pre[kMaxPatchCells + 1];
    __shared__ int warp_tot[NT / 32];
    __shared__ int cnt[P];
    __shared__ int nls[P];
    extern __shared__ float4 dyn4[];
    float *sm = reinterpret_cast<float *>(dyn4);
    float *rows = sm + M::rows;
    float2 *ent = reinterpret_cast<float2 *>(sm + M::ent);
    float *entd = sm + M::entd;
    int2 *xy = reinterpret_cast<int2 *>(sm + M::xy);
    float *yo_s = sm + M::yo, *yb_s = sm + M::yb, *ri_s = sm + M::ri;
    int *oidx = reinterpret_cast<int *>(sm + M::oidx);

    const ObsNet &net = a.net;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int tx0 = blockIdx.x * TW;
    const int ty0 = a.y_begin + blockIdx.y * TH;

    const int nc = build_patch<NT>(net, a.nx, a.ny, tx0, ty0, TW, TH, cell_base, cell_pre,
                                   warp_tot, VV <= 2);
    const int total = cell_pre[nc];
    // chunk c holds the candidates c, c + nck, c + 2 nck, ... of the patch (a uniform sample)
    const int nck = (total + CH - 1) / CH;
    auto chunk_size = [&](int ck) { return (total - ck + nck - 1) / nck; };
    if (tid < P) nls[tid] = 0;

    // S1: the candidates' observation indices
    auto stage_idx = [&](int ck, int buf) {
        if (tid < chunk_size(ck))
            cp_async4(oidx + buf * CH + tid,
                      net.cell_obs + patch_slot(cell_base, cell_pre, nc, ck + tid * nck));
    };
    // S2: their points, innovations' parts, inverse variances and perturbation rows
    auto stage_rows = [&](int ck, int buf) {
        const int nch = chunk_size(ck);
        const int *oi = oidx + buf * CH;
        if (tid < nch) {
            const int o = oi[tid];
            cp_async8(xy + buf * CH + tid, net.xy + o);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int s = o * V + v, d = buf * R + tid * V + v;
                cp_async4(yo_s + d, a.yo + s);
                cp_async4(yb_s + d, a.ybar + s);
                cp_async4(ri_s + d, a.rinv + s);
            }
        }
        for (int e = tid; e < nch * V * Q4; e += NT) {
            const int row = e / Q4, c4 = e - row * Q4;
            const int s = oi[row / V] * V + row % V;
            cp_async16(rows + (size_t)(buf * R + row) * KP + 4 * piece_pos<KB>(c4),
                       a.yb + (size_t)s * KP + 4 * c4);
        }
    };
    // S3: each point's local entries of the chunk, in candidate order
    auto build_entries = [&](int ck, int buf) {
        const int nch = chunk_size(ck);
        for (int pw = wid; pw < P; pw += NT / 32) {
            const int qx = tx0 + pw % TW, qy = ty0 + pw / TW;
            const bool qok = qx < a.nx && qy < a.y_end;
            int base = 0;
#pragma unroll
            for (int h = 0; h < CH; h += 32) {
                const int t = h + lane;
                const float wt = (qok && t < nch)
                                     ? loc_weight(net, xy[buf * CH + t], qx, qy, a.nx, a.ny)
                                     : 0.0f;
                const unsigned m = __ballot_sync(0xffffffffu, wt != 0.0f);
                if (wt != 0.0f) {
                    const int pos = base + __popc(m & ((1u << lane) - 1u));
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int rr = buf * R + t * V + v;
                        const float sw = wt * ri_s[rr];
                        ent[pw * R + pos * V + v] = make_float2(__int_as_float(rr), sw);
                        entd[pw * R + pos * V + v] = sw * ((yo_s[rr] - a.yref[v]) - yb_s[rr]);
                    }
                }
                base += __popc(m);
            }
            if (lane == 0) {
                cnt[pw] = base * V;
                nls[pw] += base;
            }
        }
    };

    // ---- this thread's role: point p of the tile, upper 8 x 8 block (ti, tj) of A_p
    const int p = tid / S::T;
    int ti = 0, tj = 0;
    upper_block<KB>(tid - p * S::T, ti, tj);
    const bool diag = ti == tj;
    float2 acc[8][4];   // acc[i][jp] = (A[i][2 jp], A[i][2 jp + 1]) of the block
    float2 cacc[4];     // diagonal blocks: (c[2 ip], c[2 ip + 1])
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < 4; ++i) cacc[i] = make_float2(0.0f, 0.0f);

    // ---- the pipeline: indices two chunks ahead, rows and metadata one chunk ahead
    if (nck > 0) stage_idx(0, 0);
    cp_commit();
    if (nck > 1) stage_idx(1, 1);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    if (nck > 0) stage_rows(0, 0);
    cp_commit();
    for (int ck = 0; ck < nck; ++ck) {
        const int buf = ck & 1;
        cp_wait_all();      // chunk ck's rows and metadata, chunk ck + 1's indices
        __syncthreads();    // ... visible to all; chunk ck - 1's arithmetic is done
        build_entries(ck, buf);
        if (ck + 1 < nck) stage_rows(ck + 1, buf ^ 1);
        cp_commit();
        if (ck + 2 < nck) stage_idx(ck + 2, buf);
        cp_commit();
        __syncthreads();    // the entries are visible
        // acc += a (s b)^T over the point's entries (and c += a s dv on the diagonal blocks),
        // the next entry's operands in flight
        const int n = p < P ? cnt[p] : 0;
        if (n > 0) {
            const float2 *E = ent + p * R;
            const float *ED = entd + p * R;
            float2 e = E[0];
            const float4 *rw = reinterpret_cast<const float4 *>(rows + __float_as_int(e.x) * KP);
            float4 A0 = rw[ti], A1 = rw[KB + ti], B0 = rw[tj], B1 = rw[KB + tj];
            float sw = e.y, sd = ED[0];
            // kept rolled: unrolled by two the kernel took 128 registers and 19 % longer
#pragma unroll 1
            for (int i = 0; i < n; ++i) {
                float4 nA0 = A0, nA1 = A1, nB0 = B0, nB1 = B1;
                float nsw = sw, nsd = sd;
                if (i + 1 < n) {
                    const float2 en = E[i + 1];
                    const float4 *rn =
                        reinterpret_cast<const float4 *>(rows + __float_as_int(en.x) * KP);
                    nA0 = rn[ti];
                    nA1 = rn[KB + ti];
                    nB0 = rn[tj];
                    nB1 = rn[KB + tj];
                    nsw = en.y;
                    nsd = ED[i + 1];
                }
                // the same multiply-adds as one fmaf per element, two per instruction
                const float2 s2 = make_float2(sw, sw);
                const float2 b2[4] = {__fmul2_rn(s2, make_float2(B0.x, B0.y)),
                                      __fmul2_rn(s2, make_float2(B0.z, B0.w)),
                                      __fmul2_rn(s2, make_float2(B1.x, B1.y)),
                                      __fmul2_rn(s2, make_float2(B1.z, B1.w))};
                const float av[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
#pragma unroll
                for (int ii = 0; ii < 8; ++ii) {
                    const float2 a2 = make_float2(av[ii], av[ii]);
#pragma unroll
                    for (int jp = 0; jp < 4; ++jp) acc[ii][jp] = __ffma2_rn(a2, b2[jp], acc[ii][jp]);
                }
                if (diag) {
                    const float2 d2 = make_float2(sd, sd);
                    cacc[0] = __ffma2_rn(make_float2(A0.x, A0.y), d2, cacc[0]);
                    cacc[1] = __ffma2_rn(make_float2(A0.z, A0.w), d2, cacc[1]);
                    cacc[2] = __ffma2_rn(make_float2(A1.x, A1.y), d2, cacc[2]);
                    cacc[3] = __ffma2_rn(make_float2(A1.z, A1.w), d2, cacc[3]);
                }
                A0 = nA0;
                A1 = nA1;
                B0 = nB0;
                B1 = nB1;
                sw = nsw;
                sd = nsd;
            }
        }
    }

    // ---- results: the upper triangle of A (off-diagonal blocks whole), c, local counts
    const int px = tx0 + p % TW, py = ty0 + p / TW;
    if (p < P && px < a.nx && py < a.y_end) {
        const size_t lp = (size_t)(py - a.y_begin) * a.nx + px;
        const int k = a.k;
        float *A = a.gram + lp * k * k;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = ti * 8 + i;
            if (row >= k) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = tj * 8 + j;
                if (col < k && col >= row)
                    A[row * k + col] = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
            }
            if (diag) a.cvec[lp * k + row] = (i & 1) ? cacc[i >> 1].y : cacc[i >> 1].x;
        }
    }
    __syncthreads();
    if (tid < P) {
        const int qx = tx0 + tid % TW, qy = ty0 + tid / TW;
        if (qx < a.nx && qy < a.y_end) a.nloc[(size_t)(qy - a.y_begin) * a.nx + qx] = nls[tid];
    }
}

template <int KP>
size_t gram_smem() {
    return (size_t)(kChunk * 3 * KP + GramShape<KP>::P * kChunk) * sizeof(float);
}

template <int KP>
cudaError_t prepare_kp() {
    const int smem = (int)gram_smem<KP>();
    cudaError_t e = cudaFuncSetAttribute(gram_kernel<KP, 1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gram_kernel<KP, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gram_kernel<KP, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
    return e;
}

template <int KP>
cudaError_t launch_kp(const GramArgs &a, cudaStream_t s) {
    using S = GramShape<KP>;
    const size_t smem = gram_smem<KP>();
    const int rows = a.y_end - a.y_begin;
    dim3 grid((a.nx + S::TW - 1) / S::TW, (rows + S::TH - 1) / S::TH);
    switch (a.net.V) {
        case 1: gram_kernel<KP, 1><<<grid, S::NT, smem, s>>>(a); break;
        case 2: gram_kernel<KP, 2><<<grid, S::NT, smem, s>>>(a); break;
        case 3: gram_kernel<KP, 3><<<grid, S::NT, smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int KP, int VV>
constexpr size_t pipe_smem() {
    return (size_t)PipeSmem<KP, VV>::floats * sizeof(float);
}

template <int KP>
cudaError_t prepare_pipe() {
    cudaError_t e = cudaFuncSetAttribute(gram_pipe_kernel<KP, 1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pipe_smem<KP, 1>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gram_pipe_kernel<KP, 2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pipe_smem<KP, 2>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gram_pipe_kernel<KP, 3>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pipe_smem<KP, 3>());
    return e;
}

template <int KP>
cudaError_t launch_pipe(const GramArgs &a, cudaStream_t s) {
    using S = PipeShape<KP>;
    const int rows = a.y_end - a.y_begin;
    dim3 grid((a.nx + S::TW - 1) / S::TW, (rows + S::TH - 1) / S::TH);
    switch (a.net.V) {
        case 1: gram_pipe_kernel<KP, 1><<<grid, S::NT, pipe_smem<KP, 1>(), s>>>(a); break;
        case 2: gram_pipe_kernel<KP, 2><<<grid, S::NT, pipe_smem<KP, 2>(), s>>>(a); break;
        case 3: gram_pipe_kernel<KP, 3><<<grid, S::NT, pipe_smem<KP, 3>(), s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

// k <= 16: the team kernel (KP = 8, 16); k >= 17: the pipelined kernel (KP = 32, 64, 128) or,
// on request (team = 1), the team kernel
int gram_tile_height(int kp, int team) {
    if (kp <= 16 || team) {
        switch (kp) {
            case 8: return GramShape<8>::TH;
            case 16: return GramShape<16>::TH;
            case 32: return GramShape<32>::TH;
            case 64: return GramShape<64>::TH;
            default: return GramShape<128>::TH;
        }
    }
    switch (kp) {
        case 32: return PipeShape<32>::TH;
        case 64: return PipeShape<64>::TH;
        default: return PipeShape<128>::TH;
    }
}
int gram_tile_width(int kp, int team) {
    if (kp <= 16 || team) {
        switch (kp) {
            case 8: return GramShape<8>::TW;
            case 16: return GramShape<16>::TW;
            case 32: return GramShape<32>::TW;
            case 64: return GramShape<64>::TW;
            default: return GramShape<128>::TW;
        }
    }
    switch (kp) {
        case 32: return PipeShape<32>::TW;
        case 64: return PipeShape<64>::TW;
        default: return PipeShape<128>::TW;
    }
}
int gram_max_cells() { return kMaxPatchCells; }

cudaError_t gram_prepare(int kp) {
    cudaError_t e = cudaSuccess;
    switch (kp) {
        case 8: return prepare_kp<8>();
        case 16: return prepare_kp<16>();
        case 32: e = prepare_kp<32>(); return e == cudaSuccess ? prepare_pipe<32>() : e;
        case 64: e = prepare_kp<64>(); return e == cudaSuccess ? prepare_pipe<64>() : e;
        case 128: e = prepare_kp<128>(); return e == cudaSuccess ? prepare_pipe<128>() : e;
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gram(const GramArgs &a, cudaStream_t s) {
    if (a.y_end <= a.y_begin) return cudaSuccess;
    switch (a.kp) {
        case 8: return launch_kp<8>(a, s);
        case 16: return launch_kp<16>(a, s);
        case 32: return a.team ? launch_kp<32>(a, s) : launch_pipe<32>(a, s);
        case 64: return a.team ? launch_kp<64>(a, s) : launch_pipe<64>(a, s);
        case 128: return a.team ? launch_kp<128>(a, s) : launch_pipe<128>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lk
