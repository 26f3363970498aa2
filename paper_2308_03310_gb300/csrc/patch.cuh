// The observation patch of a tile of grid points: every bin (cs x cs cell) that the
// cutoff disk of some point of the tile reaches, laid out as a prefix-summed list of bins so
// that the j-th candidate observation of the patch is found by a binary search.  Shared by
// the FP32 and the tensor-core Gram kernels; the candidate order (bins in patch order,
// observations ascending within a bin) fixes the summation order.
#pragma once

#include "common.cuh"

namespace lk {

constexpr int kMaxPatchCells = 1024;  // bins in one tile's patch (the host sizes bins to fit)

__device__ __forceinline__ int range_len(const BinRanges &r) {
    int n = 0;
    for (int i = 0; i < r.n; ++i) n += r.hi[i] - r.lo[i] + 1;
    return n;
}
__device__ __forceinline__ int range_at(const BinRanges &r, int i) {
    const int l0 = r.hi[0] - r.lo[0] + 1;
    return i < l0 ? r.lo[0] + i : r.lo[1] + (i - l0);
}

// Exclusive prefix sum in place over s[0..n], n <= kMaxPatchCells; s[n] receives the total.
// NT (the block's threads) is a multiple of 32.
template <int NT>
__device__ void block_exclusive_scan(int *s, int n, int *warp_tot) {
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
    constexpr int IT = (kMaxPatchCells + NT - 1) / NT;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int v[IT], local = 0;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int idx = tid * IT + i;
        v[i] = idx < n ? s[idx] : 0;
        local += v[i];
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < NT / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < NT / 32) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    int run = incl - local + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int idx = tid * IT + i;
        if (idx < n) s[idx] = run;
        run += v[i];
    }
    if (tid == NT - 1) s[n] = run;
    __syncthreads();
}

// Least periodic distance (period n) between a point of [a0, a1] and a point of [b0, b1], both
// intervals within [0, n) except that b1 may pass n - 1 at a ragged tile edge (which only
// shortens the distance).
__device__ __forceinline__ int axis_gap(int a0, int a1, int b0, int b1, int n) {
    int g = max(0, max(a0 - b1, b0 - a1));
    g = min(g, max(0, max(a0 + n - b1, b0 - a1 - n)));
    g = min(g, max(0, max(a0 - n - b1, b0 - a1 + n)));
    return g;
}

// Whether bin (bx, by) lies beyond the cutoff from every point of the tile.  Kept out of line:
// inlined into the pipelined FP32 Gram kernel it raised its register allocation to 128 and its
// executed instructions by a quarter (measured), which cost more than the pruning saved.  The
// caller opts in (prune): the pipelined kernel with at most two observed variables, where it
// measured faster; with three the kernel still went to 128 registers, and the team kernel was
// not measured with it.
static __device__ __noinline__ bool bin_beyond(const ObsNet &net, int bx, int by, int tx0,
                                               int ty0, int TW, int TH, int nx, int ny) {
    const int gx = axis_gap(bx * net.cs, min((bx + 1) * net.cs, nx) - 1, tx0, tx0 + TW - 1, nx);
    const int gy = axis_gap(by * net.cs, min((by + 1) * net.cs, ny) - 1, ty0, ty0 + TH - 1, ny);
    return (long long)gx * gx + (long long)gy * gy > (long long)net.d2max;
}

// Bins of the patch of the tile [tx0, tx0+TW) x [ty0, ty0+TH): cell_base[c] is the bin's
// first entry in net.cell_obs, cell_pre the exclusive prefix of the bin sizes.  Returns the
// number of bins; cell_pre[nc] holds the number of candidate observations.
template <int NT>
__device__ int build_patch(const ObsNet &net, int nx, int ny, int tx0, int ty0, int TW, int TH,
                           int *cell_base, int *cell_pre, int *warp_tot, bool prune = false) {
    BinRanges rx, ry;
    if (net.loc_none) {
        rx.n = ry.n = 1;
        rx.lo[0] = ry.lo[0] = 0;
        rx.hi[0] = net.ncx - 1;
        ry.hi[0] = net.ncy - 1;
    } else {
        rx = bin_ranges(tx0 - net.cr, tx0 + TW - 1 + net.cr, nx, net.cs);
        ry = bin_ranges(ty0 - net.cr, ty0 + TH - 1 + net.cr, ny, net.cs);
    }
    const int ncx_p = range_len(rx);
    const int nc = ncx_p * range_len(ry);  // <= kMaxPatchCells by construction of the bin size
    for (int c = threadIdx.x; c < nc; c += NT) {
        const int bx = range_at(rx, c % ncx_p), by = range_at(ry, c / ncx_p);
        const int cell = by * net.ncx + bx;
        const int b0 = net.cell_start[cell];
        // with prune, a bin of the bounding square beyond the cutoff from every point of the
        // tile (its corners) keeps its place with no candidates: it holds no local observation
        const bool beyond =
            prune && !net.loc_none && bin_beyond(net, bx, by, tx0, ty0, TW, TH, nx, ny);
        cell_base[c] = b0;
        cell_pre[c] = beyond ? 0 : net.cell_start[cell + 1] - b0;
    }
    __syncthreads();
    block_exclusive_scan<NT>(cell_pre, nc, warp_tot);
    return nc;
}

// Position in net.cell_obs of the j-th candidate of the patch.
__device__ __forceinline__ int patch_slot(const int *cell_base, const int *cell_pre, int nc,
                                          int j) {
    int lo = 0, hi = nc - 1;  // last bin whose prefix is <= j
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cell_pre[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return cell_base[lo] + (j - cell_pre[lo]);
}

// Observation index of the j-th candidate of the patch.
__device__ __forceinline__ int patch_obs(const ObsNet &net, const int *cell_base,
                                         const int *cell_pre, int nc, int j) {
    return net.cell_obs[patch_slot(cell_base, cell_pre, nc, j)];
}

// Localization weight (Gaussian, or Gaspari-Cohn) of observation point o seen from grid
// point (qx, qy).
__device__ __forceinline__ float loc_weight(const ObsNet &net, int2 o, int qx, int qy, int nx,
                                            int ny) {
    if (net.loc_none) return 1.0f;
    const int dx = min_image(o.x - qx, nx), dy = min_image(o.y - qy, ny);
    const int d2 = dx * dx + dy * dy;
    if (d2 > net.d2max) return 0.0f;
    return net.loc_gc ? gaspari_cohn(sqrtf((float)d2) * net.inv_c)
                      : expf(-(float)d2 * net.inv2r2);
}

}  // namespace lk
