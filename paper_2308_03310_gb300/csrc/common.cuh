// Device-side constants and helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace lk {

// D2Q9 lattice (Sec. II-A, Eq. 1): population q = 3 (j + 1) + (i + 1) moves with c_q = (i, j).
constexpr int NV = 9;
__host__ __device__ constexpr int cx(int q) { return q % 3 - 1; }
__host__ __device__ constexpr int cy(int q) { return q / 3 - 1; }
// Weights 4/9 (rest), 1/9 (axis: odd q), 1/36 (diagonal: even q other than 4).
__host__ __device__ constexpr float wq(int q) {
    return q == 4 ? 4.0f / 9.0f : ((q & 1) ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// The device stores the deviation from the rest state g_q = f_q - w_q with the exact weights
// w_q, so that the moments of the small departures from rest are formed without
// cancellation and g = 0 is the rest state exactly.  The FP32 weights differ from the exact
// ones by dw_q = w_q - fl(w_q); converting an FP32 f to g subtracts fl(w_q) (exact near rest,
// by Sterbenz' lemma) and then dw_q (one rounding at the scale of g).
__host__ __device__ constexpr float dwq(int q) {
    return q == 4 ? (float)(4.0 / 9.0 - (double)(4.0f / 9.0f))
                  : ((q & 1) ? (float)(1.0 / 9.0 - (double)(1.0f / 9.0f))
                             : (float)(1.0 / 36.0 - (double)(1.0f / 36.0f)));
}

// Gaspari-Cohn correlation of the scaled distance z = d / c >= 0 inside its support (Gaspari
// & Cohn 1999, Eq. 4.10): fifth-order piecewise rational, 1 at z = 0, zero at z = 2.  The
// outer piece, z^5/12 - z^4/2 + 5 z^3/8 + 5 z^2/3 - 5 z + 4 - 2/(3 z), is evaluated in its
// factored form (2 - z)^4 (2 z^2 + 4 z - 1) / (24 z): no cancellation near z = 2, and never
// negative.  Callers pass points strictly inside the support; z is held below 2 so that a
// rounding of z up to 2 still leaves a positive weight.
__device__ __forceinline__ float gaspari_cohn(float z) {
    if (z <= 1.0f)
        return fmaf(fmaf(fmaf(fmaf(-0.25f, z, 0.5f), z, 0.625f), z, -5.0f / 3.0f), z * z, 1.0f);
    z = fminf(z, 1.99999988f);  // the float below 2
    const float t = 2.0f - z, t2 = t * t;
    return t2 * t2 * fmaf(fmaf(2.0f, z, 4.0f), z, -1.0f) / (24.0f * z);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int floordiv(int a, int b) {  // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ int posmod(int a, int n) {  // n > 0
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Periodic minimum-image displacement on a ring of n cells, in [-n/2, n - n/2), for
// -n < d < n (a difference of two coordinates on the ring): two compares, no division.
__device__ __forceinline__ int min_image(int d, int n) {
    const int h = n >> 1;
    d -= d >= n - h ? n : 0;
    d += d < -h ? n : 0;
    return d;
}

// The coordinate interval [c0, c1] of a periodic axis of n cells, as at most two ranges of
// bins of size cs that cover it without visiting a bin twice.
struct BinRanges {
    int lo[2], hi[2], n;
};
__device__ __forceinline__ BinRanges bin_ranges(int c0, int c1, int n, int cs) {
    BinRanges r;
    const int nb = (n + cs - 1) / cs;
    if (c1 - c0 + 1 >= n) {
        r.n = 1; r.lo[0] = 0; r.hi[0] = nb - 1;
        return r;
    }
    const int a = posmod(c0, n), b = posmod(c1, n);
    if (a <= b) {
        r.n = 1; r.lo[0] = a / cs; r.hi[0] = b / cs;
    } else if (b / cs >= a / cs) {  // the two pieces would share a bin: take every bin once
        r.n = 1; r.lo[0] = 0; r.hi[0] = nb - 1;
    } else {
        r.n = 2; r.lo[0] = a / cs; r.hi[0] = nb - 1; r.lo[1] = 0; r.hi[1] = b / cs;
    }
    return r;
}

}  // namespace lk
