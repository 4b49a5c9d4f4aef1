// nb_order.cu -- spatial ordering and per-tile reference points for
// positions held in FP64 (the leap-frog state).
//
// Rounding an FP64 position to FP32 before forming x_i - x_j loses
// u |x| absolute (u = 2^-24), which is large relative to |x_i - x_j| for close
// pairs far from the origin. The compensated path instead stores, for each
// j-tile J of a spatially ordered copy of the particles, an FP32 reference
// point c_J (the tile's centroid) and the FP32 offsets fl32(x_j - c_J) formed
// in FP64; the pair kernel re-centres its i-particles on c_J once per tile.
// The error in x_i - x_j is then about u (|x_i - c_J| + |x_j - c_J|), i.e. set
// by the tile's extent, not by the distance to the origin.
//
// Ordering: particles are sorted by the 63-bit Morton code (21 bits per axis)
// of their position in the bounding box, carrying their index as a payload.
// The sort is a bitonic network (data-oblivious, so equal codes end in the
// same order on every run): chunks of kChunk keys are merged in shared
// memory and strides of kChunk and more run as global compare-exchange
// passes.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "nb_device.cuh"
#include "nb_ext.h"
#include "nb_internal.h"
#include "nb_order.h"

namespace nbk {

constexpr int kChunk = 2048;          // keys merged per block in shared memory
constexpr int kOrderThreads = 1024;   // threads of the shared-memory sort blocks
constexpr int kBoxThreads = 256;

// Per-block min/max of the positions (fixed tree order), then one block
// combines the block results: box = {min x, min y, min z, max x, max y, max z}.
__global__ void bbox_partial_kernel(const double *__restrict__ x, int64_t n,
                                    double *__restrict__ part) {
    __shared__ double s[6][kBoxThreads];
    const int t = threadIdx.x;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)kBoxThreads + t; i < n;
         i += (int64_t)gridDim.x * kBoxThreads)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], x[3 * i + c]);
            hi[c] = fmax(hi[c], x[3 * i + c]);
        }
    for (int c = 0; c < 3; ++c) {
        s[c][t] = lo[c];
        s[3 + c][t] = hi[c];
    }
    __syncthreads();
    for (int w = kBoxThreads / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int c = 0; c < 3; ++c) {
                s[c][t] = fmin(s[c][t], s[c][t + w]);
                s[3 + c][t] = fmax(s[3 + c][t], s[3 + c][t + w]);
            }
        __syncthreads();
    }
    if (t < 6) part[6 * blockIdx.x + t] = s[t][0];
}

__global__ void bbox_final_kernel(const double *__restrict__ part, int nblocks,
                                  double *__restrict__ box) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < nblocks; ++k)
        for (int c = 0; c < 3; ++c) {
            b[c] = fmin(b[c], part[6 * k + c]);
            b[3 + c] = fmax(b[3 + c], part[6 * k + 3 + c]);
        }
    for (int c = 0; c < 6; ++c) box[c] = b[c];
}

// Spread the low 21 bits of v so that they occupy every third bit of a
// 63-bit word (bit k of v moves to bit 3k).
__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void morton_keys_kernel(const double *__restrict__ x, int64_t n, int64_t npow2,
                                   const double *__restrict__ box,
                                   unsigned long long *__restrict__ keys,
                                   int32_t *__restrict__ idx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    if (i >= n) {
        keys[i] = ~0ull;  // sorts after every real code (< 2^63)
        idx[i] = -1;
        return;
    }
    unsigned long long q[3];
    for (int c = 0; c < 3; ++c) {
        const double ext = box[3 + c] - box[c];
        double f = ext > 0.0 ? (x[3 * i + c] - box[c]) / ext : 0.0;
        f = fmin(fmax(f, 0.0), 1.0);
        q[c] = (unsigned long long)fmin(f * 2097152.0, 2097151.0);
    }
    keys[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    idx[i] = (int32_t)i;
}

// All bitonic stages with stride < kChunk for merge size k (k <= kChunk: the
// whole local sort up to k). Ascending where (index & k) == 0.
__global__ void __launch_bounds__(kOrderThreads) bitonic_local_kernel(unsigned long long *keys,
                                                                      int32_t *idx, int64_t k_from,
                                                                      int64_t k_to) {
    __shared__ unsigned long long s[kChunk];
    __shared__ int32_t si[kChunk];
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    for (int t = threadIdx.x; t < kChunk; t += kOrderThreads) {
        s[t] = keys[base + t];
        si[t] = idx[base + t];
    }
    __syncthreads();
    for (int64_t k = k_from; k <= k_to; k <<= 1) {
        for (int64_t j = (k < kChunk ? k : (int64_t)kChunk) >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < kChunk / 2; t += kOrderThreads) {
                // t-th compare pair: lower index has bit j clear
                const int lo = (int)(2 * t - (t & (j - 1)));
                const int hi = lo + (int)j;
                const bool asc = ((base + lo) & k) == 0;
                const unsigned long long a = s[lo], b = s[hi];
                if (a != b && (a > b) == asc) {
                    s[lo] = b;
                    s[hi] = a;
                    const int32_t ia = si[lo];
                    si[lo] = si[hi];
                    si[hi] = ia;
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < kChunk; t += kOrderThreads) {
        keys[base + t] = s[t];
        idx[base + t] = si[t];
    }
}

// One global compare-exchange pass (stride j >= kChunk) of merge size k.
__global__ void bitonic_global_kernel(unsigned long long *keys, int32_t *idx, int64_t npow2,
                                      int64_t k, int64_t j) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= npow2 / 2) return;
    const int64_t lo = 2 * t - (t & (j - 1));
    const int64_t hi = lo + j;
    const bool asc = (lo & k) == 0;
    const unsigned long long a = keys[lo], b = keys[hi];
    if (a != b && (a > b) == asc) {
        keys[lo] = b;
        keys[hi] = a;
        const int32_t ia = idx[lo];
        idx[lo] = idx[hi];
        idx[hi] = ia;
    }
}

// One block per j-tile of the ordered particles: the tile's centroid (FP64,
// fixed tree order) rounded to FP32 is its reference point; each particle is
// packed as the FP32 offset from it, formed in FP64.
template <int JT>
__global__ void __launch_bounds__(JT) frames_pack_kernel(const double *__restrict__ x,
                                                         const float *__restrict__ m,
                                                         const int32_t *__restrict__ perm, int64_t n,
                                                         JPart *__restrict__ jp,
                                                         float4 *__restrict__ cref) {
    __shared__ double s[3][JT];
    __shared__ int cnt;
    const int t = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * JT + t;
    const bool real = k < n;
    int64_t src = real ? perm[k] : 0;
#ifdef NB_DEBUG
    // perm must be a permutation of [0, n); checked without an error word
    // here: an out-of-range entry is replaced by 0 and the particle made inert.
    const bool ok = src >= 0 && src < n;
    if (real && !ok) src = 0;
#endif
    double p[3] = {0.0, 0.0, 0.0};
    if (real)
        for (int c = 0; c < 3; ++c) p[c] = x[3 * src + c];
    for (int c = 0; c < 3; ++c) s[c][t] = p[c];
    if (t == 0) {
        const int64_t left = n - (int64_t)blockIdx.x * JT;
        cnt = left <= 0 ? 0 : (left >= JT ? JT : (int)left);
    }
    __syncthreads();
    for (int w = JT / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int c = 0; c < 3; ++c) s[c][t] += s[c][t + w];
        __syncthreads();
    }
    float cc[3] = {0.f, 0.f, 0.f};
    if (cnt > 0)
        for (int c = 0; c < 3; ++c) cc[c] = (float)(s[c][0] / cnt);
    if (t == 0) cref[blockIdx.x] = make_float4(cc[0], cc[1], cc[2], 0.f);
    float d[3] = {0.f, 0.f, 0.f};
    float hm = 0.f;
    if (real) {
        for (int c = 0; c < 3; ++c) d[c] = (float)(p[c] - (double)cc[c]);
        hm = -0.5f * m[src];
    }
    float4 *dst = reinterpret_cast<float4 *>(jp + k);
    dst[0] = make_float4(-d[0], -d[0], -d[1], -d[1]);
    dst[1] = make_float4(-d[2], -d[2], hm, hm);
}

template __global__ void frames_pack_kernel<256>(const double *, const float *, const int32_t *,
                                                 int64_t, JPart *, float4 *);

}  // namespace nbk

namespace nbx {

using namespace nbk;

int64_t order_pow2(int64_t n) {
    int64_t p = kChunk;
    while (p < n) p <<= 1;
    return p;
}

size_t order_scratch_bytes(int64_t n) {
    // keys (npow2 x 8 B) + box partials (<= 1024 blocks x 6 doubles) + box;
    // the index payload is sorted in place in the permutation buffer, which
    // the caller sizes for npow2 entries (order_pow2).
    return (size_t)order_pow2(n) * 8 + 1024 * 6 * 8 + 6 * 8;
}

cudaError_t launch_spatial_order(const double *x, int64_t n, void *scratch, int32_t *perm,
                                 cudaStream_t st) {
    const int64_t np2 = order_pow2(n);
    unsigned long long *keys = static_cast<unsigned long long *>(scratch);
    double *part = reinterpret_cast<double *>(keys + np2);
    double *box = part + 1024 * 6;
    const int nblk = (int)std::min<int64_t>(1024, (n + kBoxThreads - 1) / kBoxThreads);
    bbox_partial_kernel<<<nblk, kBoxThreads, 0, st>>>(x, n, part);
    bbox_final_kernel<<<1, 32, 0, st>>>(part, nblk, box);
    morton_keys_kernel<<<(unsigned)((np2 + 255) / 256), 256, 0, st>>>(x, n, np2, box, keys, perm);
    const unsigned chunks = (unsigned)(np2 / kChunk);
    bitonic_local_kernel<<<chunks, kOrderThreads, 0, st>>>(keys, perm, 2, kChunk);
    for (int64_t k = 2 * kChunk; k <= np2; k <<= 1) {
        for (int64_t j = k >> 1; j >= kChunk; j >>= 1)
            bitonic_global_kernel<<<(unsigned)((np2 / 2 + 255) / 256), 256, 0, st>>>(keys, perm, np2,
                                                                                    k, j);
        bitonic_local_kernel<<<chunks, kOrderThreads, 0, st>>>(keys, perm, k, k);
    }
    return cudaGetLastError();
}

cudaError_t launch_frames_pack(const double *x, const float *m, const int32_t *perm, int64_t n,
                               int64_t npad, int jtile, JPart *jp, float4 *cref, cudaStream_t st) {
    if (jtile != 256) return cudaErrorInvalidValue;
    frames_pack_kernel<256><<<(unsigned)(npad / 256), 256, 0, st>>>(x, m, perm, n, jp, cref);
    return cudaGetLastError();
}

}  // namespace nbx
