// Local analysis that allocates nothing: scratch in a file-scope device array.
//
// For callers that cannot call cudaMalloc -- code running inside a host framework that
// hands a plugin only its input/output device buffers, processes whose device memory is
// reserved up front by another allocator, or real-time loops where an allocation (and the
// device synchronisation it can imply) is not allowed.  They cannot create a letkf handle,
// whose workspace must be allocated by someone.  This entry point takes the per-point local
// observation data in the padded layout of Algorithm 1 (Y_loc[N_x, l_max V, M]) plus the
// grid-point-major forecast blocks, and keeps its only scratch -- the k x k Gram matrices,
// the c vectors, the local counts and a status word -- in the static device array below.
//
// The array is a fixed LETKF_NOALLOC_SCRATCH_BYTES; every GPU that loads this code holds it
// until the process exits.  Every call shares it, so calls that overlap on the GPU (two
// streams, two threads) race; calls ordered on one stream do not.  Each call overwrites the
// Gram matrices, c vectors and counts of the points it processes and clears the status word
// before its kernels run.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) and prepares the kernels.  Every call reads the status word back and
// synchronizes its stream, so none may run while that stream is being captured.  Larger
// problems than the scratch holds are rejected with LETKF_EINVAL before any launch.
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "letkf.h"

namespace lk {
namespace {

constexpr size_t kScratchFloats = LETKF_NOALLOC_SCRATCH_BYTES / sizeof(float);
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once per device).
cudaError_t scratch_for_current_device(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

constexpr int kThreads = 256;

template <int KP>
struct Shape {
    static constexpr int KB = KP / 8;
    static constexpr int T = KB * KB;              // threads per grid point
    static constexpr int P = kThreads / T;         // grid points per CTA
    static constexpr int CH = (16384 / (P * KP)) < 32 ? (16384 / (P * KP)) : 32;  // rows staged
};

// A_p = sum_o r_po dy_po dy_po^T and c_p = sum_o r_po dy_po d_po over the padded rows of each
// point (rows with r_po = 0 are padding).  8 x 8 register blocks per thread, as in gram.cu.
template <int KP>
__global__ void __launch_bounds__(kThreads) gram_padded_kernel(const float *__restrict__ dy,
                                                               const float *__restrict__ dl,
                                                               const float *__restrict__ rl,
                                                               int npts, int lmaxv, int k,
                                                               float *gram, float *cvec,
                                                               int *nloc) {
    using S = Shape<KP>;
    constexpr int KB = S::KB, T = S::T, P = S::P, CH = S::CH;
    extern __shared__ float4 dyn4[];
    float *ys = reinterpret_cast<float *>(dyn4);   // [P][CH][KP]
    float *dv = ys + P * CH * KP;                   // [P][CH]
    float *rv = dv + P * CH;                        // [P][CH]
    const int tid = threadIdx.x, p = tid / T, r = tid % T, ti = r / KB, tj = r % KB;
    const long long pt = (long long)blockIdx.x * P + p;
    const bool valid = pt < npts;
    float acc[8][8], cacc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        cacc[i] = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    }
    int nl = 0;
    for (int base = 0; base < lmaxv; base += CH) {
        const int nch = min(CH, lmaxv - base);
        float *my = ys + p * CH * KP;
        for (int e = r; e < nch * KP; e += T) {
            const int row = e / KP, col = e % KP;
            my[row * KP + col] =
                (valid && col < k) ? dy[((size_t)pt * lmaxv + base + row) * k + col] : 0.0f;
        }
        for (int e = r; e < nch; e += T) {
            dv[p * CH + e] = valid ? dl[(size_t)pt * lmaxv + base + e] : 0.0f;
            rv[p * CH + e] = valid ? rl[(size_t)pt * lmaxv + base + e] : 0.0f;
        }
        __syncthreads();
        if (valid) {
            for (int t = 0; t < nch; ++t) {
                const float w = rv[p * CH + t];
                if (w == 0.0f) continue;
                nl += (r == 0);
                const float *row = my + t * KP;
                const float4 a0 = reinterpret_cast<const float4 *>(row + ti * 8)[0];
                const float4 a1 = reinterpret_cast<const float4 *>(row + ti * 8)[1];
                const float4 b0 = reinterpret_cast<const float4 *>(row + tj * 8)[0];
                const float4 b1 = reinterpret_cast<const float4 *>(row + tj * 8)[1];
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                const float dd = dv[p * CH + t];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float sa = w * av[i];
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(sa, bv[j], acc[i][j]);
                    if (tj == 0) cacc[i] = fmaf(sa, dd, cacc[i]);
                }
            }
        }
        __syncthreads();
    }
    if (!valid) return;
    float *A = gram + (size_t)pt * k * k;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = ti * 8 + i;
        if (row >= k) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = tj * 8 + j;
            if (col < k) A[row * k + col] = acc[i][j];
        }
        if (tj == 0) cvec[(size_t)pt * k + row] = cacc[i];
    }
    if (r == 0) nloc[pt] = nl;
}

template <int KP>
cudaError_t launch_gram_padded(const float *dy, const float *dl, const float *rl, int npts,
                               int lmaxv, int k, float *gram, float *cvec, int *nloc,
                               cudaStream_t s) {
    using S = Shape<KP>;
    const size_t smem = (size_t)S::P * S::CH * (KP + 2) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(gram_padded_kernel<KP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((npts + S::P - 1) / S::P);
    gram_padded_kernel<KP><<<blocks, kThreads, smem, s>>>(dy, dl, rl, npts, lmaxv, k, gram, cvec,
                                                          nloc);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lk

extern "C" int letkf_local_analysis_noalloc(int32_t npts, int32_t k, int32_t lmaxv,
                                            const float *dy_loc, const float *d_loc,
                                            const float *rinv_loc, float infl, float *x,
                                            void *stream) {
    if (npts < 0 || k < 2 || k > 128 || lmaxv < 0 || !(infl > 0.0f)) return LETKF_EINVAL;
    if (npts == 0) return LETKF_OK;
    if (!x || (lmaxv > 0 && (!dy_loc || !d_loc || !rinv_loc))) return LETKF_EINVAL;
    // scratch: [npts][k][k] Gram | [npts][k] c | [npts] counts | status word
    const size_t gram_f = (size_t)npts * k * k, cvec_f = (size_t)npts * k;
    const size_t need = gram_f + cvec_f + (size_t)npts + 64;
    if (need > lk::kScratchFloats) return LETKF_EINVAL;
    float *base = nullptr;
    if (lk::scratch_for_current_device(&base) != cudaSuccess) return LETKF_ECUDA;
    float *gram = base, *cvec = base + gram_f;
    int *nloc = reinterpret_cast<int *>(cvec + cvec_f);
    int *status = reinterpret_cast<int *>(base + need - 64);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return LETKF_ECUDA;
    cudaError_t e;
    const int kp = k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : k <= 64 ? 64 : 128;
    switch (kp) {
        case 8: e = lk::launch_gram_padded<8>(dy_loc, d_loc, rinv_loc, npts, lmaxv, k, gram, cvec, nloc, s); break;
        case 16: e = lk::launch_gram_padded<16>(dy_loc, d_loc, rinv_loc, npts, lmaxv, k, gram, cvec, nloc, s); break;
        case 32: e = lk::launch_gram_padded<32>(dy_loc, d_loc, rinv_loc, npts, lmaxv, k, gram, cvec, nloc, s); break;
        case 64: e = lk::launch_gram_padded<64>(dy_loc, d_loc, rinv_loc, npts, lmaxv, k, gram, cvec, nloc, s); break;
        default: e = lk::launch_gram_padded<128>(dy_loc, d_loc, rinv_loc, npts, lmaxv, k, gram, cvec, nloc, s); break;
    }
    if (e != cudaSuccess) return LETKF_ECUDA;
    lk::EigArgs a;
    a.k = k;
    a.diag = (float)((double)(k - 1) / (double)infl);
    a.sqrt_infl = (float)sqrt((double)infl);
    a.gram = gram;
    a.cvec = cvec;
    a.nloc = nloc;
    a.x = x;
    a.pt0 = 0;
    a.npts = npts;
    a.eigval = nullptr;
    a.status = status;
    if (lk::eigen_prepare(k, &a.max_blocks) != cudaSuccess) return LETKF_ECUDA;
    if (lk::launch_eigen_update(a, s) != cudaSuccess) return LETKF_ECUDA;
    int bits = 0;
    if (cudaMemcpyAsync(&bits, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LETKF_ECUDA;
    if (bits & lk::ST_NONFINITE) return LETKF_ENONFINITE;
    if (bits & lk::ST_NOTCONV) return LETKF_ENOTCONV;
    return LETKF_OK;
}

extern "C" int letkf_eigh_batch(int32_t npts, int32_t k, float *q, float *eigval, float *evec,
                                int32_t refine, void *stream) {
    if (npts < 0 || k < 2 || k > 128 || (refine != 0 && refine != 1)) return LETKF_EINVAL;
    if (npts == 0) return LETKF_OK;
    if (!q || !eigval) return LETKF_EINVAL;
    float *base = nullptr;
    if (lk::scratch_for_current_device(&base) != cudaSuccess) return LETKF_ECUDA;
    int *status = reinterpret_cast<int *>(base + lk::kScratchFloats - 64);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return LETKF_ECUDA;
    lk::EigArgs a;
    a.k = k;
    a.diag = 0.0f;           // the matrices are Q themselves
    a.gram = q;
    a.npts = npts;
    a.eigval = eigval;
    a.evec = evec;
    a.refine = refine;
    a.refine_tau = 1e-6f;
    a.status = status;       // no counts, no forecast blocks: eigenpairs only
    if (lk::eigen_prepare(k, &a.max_blocks) != cudaSuccess) return LETKF_ECUDA;
    if (lk::launch_eigen_update(a, s) != cudaSuccess) return LETKF_ECUDA;
    int bits = 0;
    if (cudaMemcpyAsync(&bits, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LETKF_ECUDA;
    if (bits & lk::ST_NONFINITE) return LETKF_ENONFINITE;
    if (bits & lk::ST_NOTCONV) return LETKF_ENOTCONV;
    return LETKF_OK;
}

namespace {

// Split-schedule scratch for npts matrices of order k, each array 256-byte aligned.
struct EighLayout {
    size_t de, taus, rot, nrot, list, count, status, total;
    int rcap;
};

EighLayout eigh_layout(int32_t npts, int32_t k) {
    EighLayout l{};
    l.rcap = k * k + 4 * k;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    };
    const size_t n = (size_t)npts;
    l.de = take(n * k * sizeof(float2));
    l.taus = take(n * k * sizeof(float));
    l.rot = take(n * (size_t)l.rcap * sizeof(float2));
    l.nrot = take(n * sizeof(int));
    l.list = take((n + 4) * sizeof(int));
    l.count = take(sizeof(int));
    l.status = take(sizeof(int));
    l.total = off;
    return l;
}

}  // namespace

extern "C" size_t letkf_eigh_workspace_bytes(int32_t npts, int32_t k) {
    if (npts < 0 || k < 2 || k > 128) return 0;
    return eigh_layout(npts, k).total;
}

extern "C" int letkf_eigh_batch_ws(int32_t npts, int32_t k, float *q, float *eigval, float *evec,
                                   int32_t refine, void *workspace, size_t workspace_bytes,
                                   void *stream) {
    if (npts < 0 || k < 2 || k > 128 || (refine != 0 && refine != 1)) return LETKF_EINVAL;
    if (npts == 0) return LETKF_OK;
    if (!q || !eigval) return LETKF_EINVAL;
    const EighLayout l = eigh_layout(npts, k);
    if (!workspace || workspace_bytes < l.total || ((uintptr_t)workspace & 255))
        return LETKF_ENOMEM;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lk::EigSplit sp;
    sp.de = reinterpret_cast<float2 *>(ws + l.de);
    sp.taus = reinterpret_cast<float *>(ws + l.taus);
    sp.rot = reinterpret_cast<float2 *>(ws + l.rot);
    sp.nrot = reinterpret_cast<int *>(ws + l.nrot);
    sp.list = reinterpret_cast<int *>(ws + l.list);
    sp.list_count = reinterpret_cast<int *>(ws + l.count);
    sp.rcap = l.rcap;
    int *status = reinterpret_cast<int *>(ws + l.status);
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return LETKF_ECUDA;
    lk::EigArgs a;
    a.k = k;
    a.diag = 0.0f;           // the matrices are Q themselves
    a.gram = q;
    a.npts = npts;
    a.eigval = eigval;
    a.evec = evec;
    a.refine = refine;
    a.refine_tau = 1e-6f;
    a.status = status;       // no counts, no forecast blocks: eigenpairs only
    if (lk::eigen_prepare(k, &a.max_blocks) != cudaSuccess ||
        lk::eigen_split_prepare(k, &sp) != cudaSuccess)
        return LETKF_ECUDA;
    if (lk::launch_eigen_split(a, sp, s) != cudaSuccess) return LETKF_ECUDA;
    int bits = 0;
    if (cudaMemcpyAsync(&bits, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LETKF_ECUDA;
    if (bits & lk::ST_NONFINITE) return LETKF_ENONFINITE;
    if (bits & lk::ST_NOTCONV) return LETKF_ENOTCONV;
    return LETKF_OK;
}
