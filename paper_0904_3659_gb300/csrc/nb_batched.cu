// nb_batched.cu -- Eq. (gravity) (Fujiwara & Nakasato, arXiv:0904.3659,
// Section "Introduction") for many independent clusters in one persistent
// launch, and the leap-frog of Section "Method" over such a batch.
//
// Layout: the clusters, concatenated by the caller, are packed into a padded
// copy in which every cluster starts on a multiple of kClusterPad particles
// and is padded with inert entries (m = 0), so every j-tile and i-block lies
// inside one cluster. Work item = (cluster, i-block); a one-block planning
// kernel lists the items grouped by the cluster's padded size, largest first
// (close to longest-processing-time order), and the pair kernel's CTAs pop
// items from an atomic counter. Each item is summed entirely by one CTA in a
// fixed order, so the results do not depend on which CTA pops what.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include "nb_device.cuh"
#include "nb_ext.h"
#include "nb_internal.h"
#include "nb_tile.cuh"

namespace nbk {
using namespace nbdev;

constexpr int kClusterPad = 128;  // >= every batched i-block and j-tile
// The batched kernels' i-block (32 lanes x 4 i) and j-tile sizes, fixed so
// that the planner and the combine divide by constants (batch_prepare checks
// every compiled shape against them).
constexpr int kBatchIB = 128, kBatchJT = 128;
static_assert(kClusterPad % kBatchIB == 0 && kClusterPad % kBatchJT == 0,
              "i-blocks and j-tiles lie inside one padded cluster");
constexpr int kPlanThreads = 1024;
constexpr int kMaxChunks = 4;      // the j-range of an i-block is split into at most this many items

// Chunks an i-block of a cluster with ntiles j-tiles is split into.
__host__ __device__ __forceinline__ int64_t chunks_of(int64_t ntiles) {
    return ntiles < kMaxChunks ? ntiles : kMaxChunks;
}

struct BatchPlanArgs {
    const int64_t *off;   // [C+1] caller's offsets
    const float *eps;     // [C] caller's softening lengths
    int64_t C;
    int64_t n_total;      // the caller's particle count (offsets[C] must equal it)
    int64_t cap_padded;   // capacity of the padded particle array
    int64_t cap_items;    // capacity of the item list
    int64_t *poff;        // [C+1] padded offsets (out)
    int4 *items;          // [cap_items] (cluster, i-block, chunk, chunks) (out)
    int64_t *ibase;       // [C] index of the cluster's first item (out)
    int *nitems;          // item count (out)
    int *err;             // set if the offsets do not fit the capacities
    int64_t *planned_off; // [C+1] offsets of the plan in poff/items/ibase (in/out)
    uint32_t *planned_eps;// [C] bits of its eps (in/out)
    int replan;           // 1: the scratch holds no plan of this (C, n_total)
};

// Exclusive block-wide scan of one value per thread (kPlanThreads threads):
// a shuffle scan within each warp, then one over the warps' totals. On
// return smem[t] holds thread t's inclusive prefix and *total the block's sum.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *smem, int64_t *total) {
    constexpr int kWarps = kPlanThreads / 32;
    static_assert(kWarps <= 32, "the warps' totals are scanned by one warp");
    __shared__ int64_t wsum[kWarps];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int64_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kWarps ? wsum[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < kWarps) wsum[lane] = w;
    }
    __syncthreads();
    const int64_t incl = x + (warp > 0 ? wsum[warp - 1] : 0);
    smem[t] = incl;
    *total = wsum[kWarps - 1];
    __syncthreads();
    return incl - v;
}

__device__ __forceinline__ int size_class(int64_t psz) {
    return psz > 0 ? 63 - __clzll((unsigned long long)psz) : -1;
}

__global__ void __launch_bounds__(kPlanThreads) batch_plan_kernel(const BatchPlanArgs P) {
    __shared__ int64_t scan[kPlanThreads];
    const int t = threadIdx.x;
    // The same offsets and eps as the plan already in the scratch (it was
    // valid, or planned_off[0] would be -1): that plan stands.
    if (!P.replan) {
        int diff = 0;
        for (int64_t c = t; c <= P.C; c += kPlanThreads) {
            diff |= P.off[c] != P.planned_off[c];
            if (c < P.C) diff |= __float_as_uint(P.eps[c]) != P.planned_eps[c];
        }
        if (!__syncthreads_or(diff)) return;
    }
    // Offsets must start at 0, never decrease and end at n_total, and every
    // non-empty cluster's eps must be > 0 with eps^2 a finite normal FP32
    // number (as for nb_force); otherwise every cluster is given zero size so
    // no later kernel reads anything.
    int bad = 0;
    for (int64_t c = t; c < P.C; c += kPlanThreads) {
        bad |= P.off[c + 1] < P.off[c];
        if (P.off[c + 1] > P.off[c]) {
            const float e = P.eps[c], e2 = e * e;
            bad |= !(e > 0.f && e2 >= FLT_MIN && e2 <= FLT_MAX);  // also false for NaN
        }
    }
    if (t == 0) bad |= (P.off[0] != 0) | (P.off[P.C] != P.n_total);
    const bool valid = !__syncthreads_or(bad);
    if (!valid) {
        for (int64_t c = t; c <= P.C; c += kPlanThreads) P.poff[c] = 0;
        if (t == 0) {
            *P.nitems = 0;
            P.planned_off[0] = -1;  // no valid plan in the scratch
            atomicOr(P.err, kErrBatchPlan);
        }
        return;
    }
    // Padded offsets.
    int64_t carry = 0;
    for (int64_t base = 0; base < P.C; base += kPlanThreads) {
        const int64_t c = base + t;
        int64_t psz = 0;
        if (c < P.C) {
            const int64_t nc = P.off[c + 1] - P.off[c];
            psz = nc > 0 ? (nc + kClusterPad - 1) / kClusterPad * kClusterPad : 0;
        }
        int64_t total;
        const int64_t ex = block_exclusive_scan(psz, scan, &total);
        if (c < P.C) P.poff[c] = carry + ex;
        carry += total;
    }
    if (t == 0) P.poff[P.C] = carry;
    const bool fits = carry <= P.cap_padded;
    // Size classes present (one bit each), so the item pass below visits only those.
    __shared__ unsigned long long present;
    if (t == 0) present = 0ull;
    __syncthreads();
    unsigned long long mine = 0ull;
    for (int64_t c = t; c < P.C; c += kPlanThreads) {
        const int64_t nc = P.off[c + 1] - P.off[c];
        const int64_t psz = nc > 0 ? (nc + kClusterPad - 1) / kClusterPad * kClusterPad : 0;
        if (psz > 0) mine |= 1ull << size_class(psz);
    }
    for (int d = 16; d > 0; d >>= 1) mine |= __shfl_xor_sync(0xffffffffu, mine, d);
    if ((t & 31) == 0 && mine) atomicOr(&present, mine);
    __syncthreads();
    const unsigned long long classes = present;
    // Items, largest size class first; clusters in index order within a class,
    // and (i-block, chunk) in order within a cluster.
    int64_t nit = 0;
    for (int cls = 62; cls >= 0 && fits; --cls) {
        if (!((classes >> cls) & 1ull)) continue;
        for (int64_t base = 0; base < P.C; base += kPlanThreads) {
            const int64_t c = base + t;
            int64_t cnt = 0, nch = 0;
            if (c < P.C) {
                const int64_t nc = P.off[c + 1] - P.off[c];
                const int64_t psz = nc > 0 ? (nc + kClusterPad - 1) / kClusterPad * kClusterPad : 0;
                if (size_class(psz) == cls) {
                    nch = chunks_of(psz / kBatchJT);
                    cnt = psz / kBatchIB * nch;
                }
            }
            int64_t total;
            const int64_t ex = block_exclusive_scan(cnt, scan, &total);
            if (cnt) P.ibase[c] = nit + ex;
            // Each warp writes the items of its threads' clusters, one
            // cluster at a time with all 32 lanes (consecutive items, so the
            // stores coalesce).
            if (nit + total <= P.cap_items) {
                const int lane = t & 31;
                unsigned todo = __ballot_sync(0xffffffffu, cnt > 0);
                while (todo) {
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const int64_t first = nit + __shfl_sync(0xffffffffu, ex, src);
                    const int ccnt = (int)__shfl_sync(0xffffffffu, cnt, src);  // <= 4 x i-blocks
                    const int cn = (int)__shfl_sync(0xffffffffu, nch, src);
                    const int cc = (int)(base + (t - lane) + src);
                    for (int q = lane; q < ccnt; q += 32) {
                        const int bi = q / cn;
                        P.items[first + q] = make_int4(cc, bi, q - bi * cn, cn);
                    }
                }
            }
            nit += total;
        }
    }
    const bool ok = fits && nit <= P.cap_items;
    if (t == 0) {
        *P.nitems = ok ? (int)nit : 0;
        if (!ok) atomicOr(P.err, kErrBatchPlan);
    }
    // Remember what this plan was made for (an unusable plan: nothing).
    for (int64_t c = t; c <= P.C; c += kPlanThreads) {
        P.planned_off[c] = ok ? P.off[c] : -1;
        if (c < P.C) P.planned_eps[c] = __float_as_uint(P.eps[c]);
    }
}

// The cluster holding padded row s (0 <= s < poff[C]): the largest c with
// poff[c] <= s (an empty cluster has poff[c] == poff[c + 1]).
__device__ __forceinline__ int64_t padded_cluster(const int64_t *__restrict__ poff, int64_t C,
                                                  int64_t s) {
    int64_t lo = 0, hi = C - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (poff[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The padded rows are processed in blocks of kClusterPad rows, each inside
// one cluster: one CTA per block, one thread per row, so every row's loads
// are in flight at once however the sizes are distributed. Blocks past
// poff[C] (the capacity bound, or every block when the planner rejected the
// offsets and left poff zero) do nothing.

// Pack the padded rows (FP32 or FP64 source, rounded to FP32); rows past a
// cluster's particles are inert (zero position and mass).
template <typename T>
__global__ void __launch_bounds__(kClusterPad) batch_pack_kernel(const T *__restrict__ x,
                                                                 const float *__restrict__ m,
                                                                 const int64_t *__restrict__ off,
                                                                 const int64_t *__restrict__ poff,
                                                                 int64_t C, JPart *__restrict__ jp) {
    const int64_t s = (int64_t)blockIdx.x * kClusterPad;
    if (s >= poff[C]) return;
    const int64_t c = padded_cluster(poff, C, s);
    const int64_t li = s - poff[c] + threadIdx.x, o = off[c], nc = off[c + 1] - o;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (li < nc) {
        const int64_t i = o + li;
        const float px = (float)x[3 * i], py = (float)x[3 * i + 1], pz = (float)x[3 * i + 2];
        const float hm = -0.5f * m[i];
        lo = make_float4(-px, -px, -py, -py);
        hi = make_float4(-pz, -pz, hm, hm);
    }
    float4 *dst = reinterpret_cast<float4 *>(jp + s + threadIdx.x);
    dst[0] = lo;
    dst[1] = hi;
}

// Order-preserving map of an FP64 value's bits to a signed 64-bit integer
// (its own inverse): the bounding box below is reduced with integer min/max,
// which run at the integer pipe's rate rather than the FP64 pipe's.
__device__ __forceinline__ long long ordered_key(long long bits) {
    return bits >= 0 ? bits : bits ^ 0x7fffffffffffffffll;
}

constexpr int kFrameThreads = 512;

// Compensated mode on FP64 state, first pass: the frame of cluster
// blockIdx.x, the centre of its bounding box and the grid 2^(E-23) set by
// the box's half-width (all pairs lie inside one cluster, so each cluster
// has its own frame): frame[c] = (centre, grid). Positions are finite.
__global__ void __launch_bounds__(kFrameThreads) batch_frame_kernel(const double *__restrict__ x,
                                                                    const int64_t *__restrict__ off,
                                                                    const int64_t *__restrict__ poff,
                                                                    double4 *__restrict__ frame) {
    __shared__ long long s[6][kFrameThreads / 32];
    const int64_t c = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t o = off[c], psz = poff[c + 1] - poff[c];
    const int64_t nc = psz > 0 ? off[c + 1] - o : 0;
    if (psz <= 0) return;
    const long long *xb = reinterpret_cast<const long long *>(x) + 3 * o;
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
#pragma unroll 4
    for (int64_t li = t; li < nc; li += kFrameThreads)
        for (int k = 0; k < 3; ++k) {
            const long long v = ordered_key(xb[3 * li + k]);
            lo[k] = v < lo[k] ? v : lo[k];
            hi[k] = v > hi[k] ? v : hi[k];
        }
    for (int k = 0; k < 3; ++k)
        for (int d = 16; d > 0; d >>= 1) {
            const long long a = __shfl_xor_sync(0xffffffffu, lo[k], d);
            const long long b = __shfl_xor_sync(0xffffffffu, hi[k], d);
            lo[k] = a < lo[k] ? a : lo[k];
            hi[k] = b > hi[k] ? b : hi[k];
        }
    if (lane == 0)
        for (int k = 0; k < 3; ++k) {
            s[k][warp] = lo[k];
            s[3 + k][warp] = hi[k];
        }
    __syncthreads();
    if (t == 0) {
        double cen[3], ext = 0.0;
        for (int k = 0; k < 3; ++k) {
            long long l = s[k][0], h = s[3 + k][0];
            for (int w = 1; w < kFrameThreads / 32; ++w) {
                l = s[k][w] < l ? s[k][w] : l;
                h = s[3 + k][w] > h ? s[3 + k][w] : h;
            }
            const double dl = __longlong_as_double(ordered_key(l)), dh = __longlong_as_double(ordered_key(h));
            cen[k] = 0.5 * (dl + dh);
            ext = fmax(ext, 0.5 * (dh - dl));
        }
        frame[c] = make_double4(cen[0], cen[1], cen[2], ldexp(1.0, hl_grid_exponent(ext) - 23));
    }
}

// Second pass: the padded rows as HL records (two JParts per particle, see
// kHLRecords) in their cluster's frame; padding rows are inert (zero
// position and mass). Each coordinate y = x - centre (|y| <= 2^E) is split
// into h, y rounded to a multiple of the grid G (adding and subtracting
// 1.5 * 2^52 G, whose unit in the last place is G, rounds to the nearest
// multiple exactly), and the FP32 remainder l = fl32(y - h).
__global__ void __launch_bounds__(kClusterPad) batch_pack_hl_kernel(const double *__restrict__ x,
                                                                    const float *__restrict__ m,
                                                                    const int64_t *__restrict__ off,
                                                                    const int64_t *__restrict__ poff,
                                                                    const double4 *__restrict__ frame,
                                                                    int64_t C, JPart *__restrict__ jp) {
    const int64_t s = (int64_t)blockIdx.x * kClusterPad;
    if (s >= poff[C]) return;
    const int64_t c = padded_cluster(poff, C, s);
    const int64_t li = s - poff[c] + threadIdx.x, o = off[c], nc = off[c + 1] - o;
    float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f}, hm = 0.f;
    if (li < nc) {
        const double4 f = frame[c];
        const double cen[3] = {f.x, f.y, f.z};
        const double magic = 6755399441055744.0 * f.w;  // 1.5 * 2^52 * G
        const int64_t i = o + li;
        for (int k = 0; k < 3; ++k) {
            const double y = __dsub_rn(x[3 * i + k], cen[k]);
            const double yh = __dsub_rn(__dadd_rn(y, magic), magic);
            h[k] = (float)yh;
            l[k] = (float)__dsub_rn(y, yh);
        }
        hm = -0.5f * m[i];
    }
    float4 *dst = reinterpret_cast<float4 *>(jp + kHLRecords * (s + threadIdx.x));
    dst[0] = make_float4(-h[0], -h[0], -h[1], -h[1]);
    dst[1] = make_float4(-h[2], -h[2], hm, hm);
    dst[2] = make_float4(-l[0], -l[0], -l[1], -l[1]);
    dst[3] = make_float4(-l[2], -l[2], 0.f, 0.f);
}

struct BatchArgs {
    const JPart *jp;
    const int64_t *off;
    const int64_t *poff;
    const float *eps;
    const int4 *items;
    const int *nitems;
    int *counter;
    float4 *partial;  // [item][words][ib]: one item's sums for its i-block
    int *err;
    uint64_t wait_ns;
    int64_t cap_padded, cap_items, partial_len;  // extents (debug-build bounds checks)
};

struct StageMeta {
    int item, cluster, iblock, jt, end;
    int len;  // particles copied into the stage: JT, or the cluster's last, shorter tile
};

// HL: the particles are HL records (two JParts each, batch_pack_hl_kernel)
// and each pair's x_i - x_j is formed by tile_pass_hl.
// Warp-level persistent kernel: every warp of a CTA is an independent
// worker with its own shared-memory stages, barriers and item stream. Lane 0
// pops (cluster, i-block) items from the device queue, issues the 1-D bulk
// copies of that cluster's j-tiles, and the whole warp consumes them. A work
// item is 32 lanes x IPT i-particles (IPT/2 packed pairs per lane), so the
// item equals the cluster padding and no CTA-wide barrier is needed.
template <int WARPS, int IPT, int JT, int STAGES, bool COMP, bool HL>
__global__ void __launch_bounds__(WARPS * 32) batched_pair_kernel(const BatchArgs A) {
    constexpr int P = IPT / 2;
    constexpr int IB = 32 * IPT;
    constexpr int RS = HL ? kHLRecords : 1;  // JParts per particle
    constexpr uint32_t TILE_BYTES = JT * RS * sizeof(JPart);
    static_assert(kClusterPad % IB == 0 && kClusterPad % JT == 0, "tiles must divide the padding");
    constexpr size_t WARP_BYTES = (size_t)STAGES * TILE_BYTES;

    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    JPart *tiles = reinterpret_cast<JPart *>(smem + warp * WARP_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + WARPS * WARP_BYTES) + warp * STAGES;
    StageMeta *meta =
        reinterpret_cast<StageMeta *>(reinterpret_cast<uint64_t *>(smem + WARPS * WARP_BYTES) +
                                      WARPS * STAGES) + warp * STAGES;
    int *issued_at = reinterpret_cast<int *>(
                         reinterpret_cast<StageMeta *>(reinterpret_cast<uint64_t *>(
                                                           smem + WARPS * WARP_BYTES) +
                                                       WARPS * STAGES) +
                         WARPS * STAGES) + warp * STAGES;

    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            issued_at[s] = -1;
        }
        fence_mbar_init();
    }
    __syncwarp();

    // Producer state (lane 0): walks the (item, j-tile) stream, popping items.
    int p_item = -1, p_cluster = 0, p_b = 0, p_jt = 0, p_ntiles = 0, p_done = 0;
    int64_t p_base = 0, p_nc = 0;
    const int nitems = *A.nitems;
    auto produce = [&](int kk) {
        const int s = kk % STAGES;
        if (!p_done && p_jt >= p_ntiles) {
            const int it = atomicAdd(A.counter, 1);
            if (it >= nitems || !NB_IN(A.err, 10, it < A.cap_items)) {
                p_done = 1;
            } else {
                const int4 w = A.items[it];
                p_item = it;
                p_cluster = w.x;
                p_b = w.y;
                p_base = A.poff[w.x];
                p_nc = A.off[w.x + 1] - A.off[w.x];
                const int ntiles = (int)((A.poff[w.x + 1] - p_base) / JT);
                // chunk w.z of w.w: tiles [w.z*ntiles/w.w, (w.z+1)*ntiles/w.w)
                p_jt = (int)((int64_t)w.z * ntiles / w.w);
                p_ntiles = (int)((int64_t)(w.z + 1) * ntiles / w.w);
            }
        }
        // The cluster's last tile stops at its last particle, rounded up to a
        // multiple of 32: the padding rows beyond add nothing (zero mass).
        const int64_t rem = p_nc - (int64_t)p_jt * JT;
        const int len = rem >= JT ? JT : rem > 0 ? (int)((rem + 31) & ~(int64_t)31) : 32;
        StageMeta mt;
        mt.end = p_done;
        mt.item = p_item;
        mt.cluster = p_cluster;
        mt.iblock = p_b;
        mt.jt = p_jt;
        mt.len = len;
        meta[s] = mt;
        if (!p_done && !NB_IN(A.err, 11, p_base + (int64_t)(p_jt + 1) * JT <= A.cap_padded))
            p_done = 1;
        if (p_done) {
            mt.end = 1;
            meta[s] = mt;
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[s]))
                         : "memory");
        } else {
            issued_at[s] = kk;
            const uint32_t bytes = (uint32_t)len * RS * (uint32_t)sizeof(JPart);
            mbar_arrive_expect_tx(&full[s], bytes);
            bulk_g2s(tiles + (size_t)s * JT * RS, A.jp + (p_base + (int64_t)p_jt * JT) * RS, bytes,
                     &full[s]);
            ++p_jt;
        }
    };
    if (lane == 0)
        for (int kk = 0; kk < STAGES - 1; ++kk) produce(kk);

    float2 xi[P], yi[P], zi[P];
    float2 lxi[P], lyi[P], lzi[P];  // HL: remainders of the i-particles' positions
    float2 sum[P][4], cmp[P][4];
    const float2 zero2 = splat2(0.f);
    int cur_item = -1, cur_cluster = 0, cur_b = 0;
    float2 eps2 = zero2;

    // The item's sums (and Kahan carries) for its i-block.
    auto write_out = [&]() {
        if (!NB_IN(A.err, 13, ((int64_t)cur_item + 1) * (COMP ? 2 : 1) * IB <= A.partial_len)) return;
        float4 *dst = A.partial + (int64_t)cur_item * (COMP ? 2 : 1) * IB;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int i0 = (2 * q) * 32 + lane, i1 = i0 + 32;
            dst[i0] = make_float4(sum[q][0].x, sum[q][1].x, sum[q][2].x, sum[q][3].x);
            dst[i1] = make_float4(sum[q][0].y, sum[q][1].y, sum[q][2].y, sum[q][3].y);
            if (COMP) {
                dst[IB + i0] = make_float4(cmp[q][0].x, cmp[q][1].x, cmp[q][2].x, cmp[q][3].x);
                dst[IB + i1] = make_float4(cmp[q][0].y, cmp[q][1].y, cmp[q][2].y, cmp[q][3].y);
            }
        }
    };

    int bad = 0;
    for (int k = 0;; ++k) {
        // All lanes are done with iteration k-1: its stage may be refilled.
        __syncwarp();
        if (lane == 0) produce(k + STAGES - 1);
        const int s = k % STAGES;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((k / STAGES) & 1), A.wait_ns)) bad = 1;
        if (__any_sync(0xffffffffu, bad)) {
            bad = 1;
            break;
        }
        const StageMeta mt = meta[s];
        if (mt.end) break;
        if (mt.item != cur_item) {
            if (cur_item >= 0) write_out();
            cur_item = mt.item;
            cur_cluster = mt.cluster;
            cur_b = mt.iblock;
            eps2 = splat2(A.eps[cur_cluster] * A.eps[cur_cluster]);
            const int64_t base = A.poff[cur_cluster] + (int64_t)cur_b * IB;
#pragma unroll
            for (int q = 0; q < P; ++q) {
                int64_t i0 = base + (2 * q) * 32 + lane, i1 = i0 + 32;
                if (!NB_IN(A.err, 12, i1 < A.cap_padded)) i0 = i1 = 0;
                const float4 A0 = reinterpret_cast<const float4 *>(A.jp + i0 * RS)[0];
                const float4 B0 = reinterpret_cast<const float4 *>(A.jp + i0 * RS)[1];
                const float4 A1 = reinterpret_cast<const float4 *>(A.jp + i1 * RS)[0];
                const float4 B1 = reinterpret_cast<const float4 *>(A.jp + i1 * RS)[1];
                xi[q] = make_float2(-A0.x, -A1.x);
                yi[q] = make_float2(-A0.z, -A1.z);
                zi[q] = make_float2(-B0.x, -B1.x);
                if (HL) {
                    const float4 C0 = reinterpret_cast<const float4 *>(A.jp + i0 * RS + 1)[0];
                    const float4 D0 = reinterpret_cast<const float4 *>(A.jp + i0 * RS + 1)[1];
                    const float4 C1 = reinterpret_cast<const float4 *>(A.jp + i1 * RS + 1)[0];
                    const float4 D1 = reinterpret_cast<const float4 *>(A.jp + i1 * RS + 1)[1];
                    lxi[q] = make_float2(-C0.x, -C1.x);
                    lyi[q] = make_float2(-C0.z, -C1.z);
                    lzi[q] = make_float2(-D0.x, -D1.x);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    sum[q][r] = zero2;
                    cmp[q][r] = zero2;
                }
            }
        }
        const JPart *T = tiles + (size_t)s * JT * RS;
        float2 acc[P][4];
#pragma unroll
        for (int q = 0; q < P; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[q][r] = zero2;
        const int ibase = cur_b * IB, jbase = mt.jt * JT;
        int self0[P], self1[P];
        if (jbase < ibase + IB && ibase < jbase + JT) {
            if constexpr (JT == IB && JT == 128 && P == 2 && COMP) {
                // The tile is the i-block itself: its 32-particle quarter k
                // holds slot k of every lane (particle 32 k + lane), so each
                // quarter runs the lane-diagonal form for its slot. (The
                // compensated kernels only: with it, the plain kernel compiled
                // to 96 instead of 112 registers and ran 7% slower; the
                // compensated ones gained 2-3%.)
#pragma unroll
                for (int q = 0; q < P; ++q) self0[q] = self1[q] = lane;
                // Quarters past a short last tile hold only padding: skipped.
                if constexpr (HL) {
                    tile_pass_hl<P, 32, 4, true, true, 0>(T, xi, yi, zi, lxi, lyi, lzi, acc, eps2, self0, self1);
                    if (mt.len > 32)
                        tile_pass_hl<P, 32, 4, true, true, 1>(T + 64, xi, yi, zi, lxi, lyi, lzi, acc, eps2,
                                                              self0, self1);
                    if (mt.len > 64)
                        tile_pass_hl<P, 32, 4, true, true, 2>(T + 128, xi, yi, zi, lxi, lyi, lzi, acc, eps2,
                                                              self0, self1);
                    if (mt.len > 96)
                        tile_pass_hl<P, 32, 4, true, true, 3>(T + 192, xi, yi, zi, lxi, lyi, lzi, acc, eps2,
                                                              self0, self1);
                } else {
                    constexpr bool NW = kDefaultRefine != 0;
                    tile_pass<P, 32, 4, true, kMixAll, NW, true, 0>(T, xi, yi, zi, acc, eps2, self0, self1);
                    if (mt.len > 32)
                        tile_pass<P, 32, 4, true, kMixAll, NW, true, 1>(T + 32, xi, yi, zi, acc, eps2, self0,
                                                                        self1);
                    if (mt.len > 64)
                        tile_pass<P, 32, 4, true, kMixAll, NW, true, 2>(T + 64, xi, yi, zi, acc, eps2, self0,
                                                                        self1);
                    if (mt.len > 96)
                        tile_pass<P, 32, 4, true, kMixAll, NW, true, 3>(T + 96, xi, yi, zi, acc, eps2, self0,
                                                                        self1);
                }
            } else {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    self0[q] = ibase + (2 * q) * 32 + lane - jbase;
                    self1[q] = self0[q] + 32;
                }
                if (mt.len == JT) {
                    if constexpr (HL)
                        tile_pass_hl<P, JT, 1, true, true>(T, xi, yi, zi, lxi, lyi, lzi, acc, eps2, self0,
                                                           self1);
                    else
                        tile_pass<P, JT, 1, true, kMixAll, kDefaultRefine != 0>(T, xi, yi, zi, acc, eps2,
                                                                                self0, self1);
                } else {
                    // A short last tile, in 32-particle pieces (self indices
                    // relative to each piece).
                    for (int o = 0; o < mt.len; o += 32) {
                        if constexpr (HL)
                            tile_pass_hl<P, 32, 1, true, true>(T + o * RS, xi, yi, zi, lxi, lyi, lzi, acc, eps2,
                                                               self0, self1);
                        else
                            tile_pass<P, 32, 1, true, kMixAll, kDefaultRefine != 0>(T + o, xi, yi, zi, acc,
                                                                                    eps2, self0, self1);
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            self0[q] -= 32;
                            self1[q] -= 32;
                        }
                    }
                }
            }
        } else if (mt.len == JT) {
            if constexpr (HL)
                tile_pass_hl<P, JT, 4, false, true>(T, xi, yi, zi, lxi, lyi, lzi, acc, eps2, self0,
                                                    self1);
            else
                tile_pass<P, JT, 4, false, kMixAll, kDefaultRefine != 0>(T, xi, yi, zi, acc, eps2,
                                                                         self0, self1);
        } else {
            // A short last tile, in 32-particle pieces.
            for (int o = 0; o < mt.len; o += 32) {
                if constexpr (HL)
                    tile_pass_hl<P, 32, 4, false, true>(T + o * RS, xi, yi, zi, lxi, lyi, lzi, acc, eps2,
                                                        self0, self1);
                else
                    tile_pass<P, 32, 4, false, kMixAll, kDefaultRefine != 0>(T + o, xi, yi, zi, acc, eps2,
                                                                             self0, self1);
            }
        }
#pragma unroll
        for (int q = 0; q < P; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (COMP) {
                    const float2 y = add2(acc[q][r], neg2(cmp[q][r]));
                    const float2 t = add2(sum[q][r], y);
                    cmp[q][r] = add2(add2(t, neg2(sum[q][r])), neg2(y));
                    sum[q][r] = t;
                } else {
                    sum[q][r] = add2(sum[q][r], acc[q][r]);
                }
            }
    }
    if (!bad) {
        if (cur_item >= 0) write_out();
        return;
    }
    if (lane == 0) {
        atomicOr(A.err, kErrTimeout);
        // Let this warp's copies in flight land before the CTA can exit.
        for (int s = 0; s < STAGES; ++s)
            if (issued_at[s] >= 0)
                mbar_wait_bounded(&full[s], (uint32_t)((issued_at[s] / STAGES) & 1), A.wait_ns);
    }
    __syncwarp();
}

// Per particle: add the chunk sums of its (cluster, i-block) in chunk order
// and remove the factors the pair sums carry (accel_scale, pot_scale of the
// batched kernel's refine setting). One CTA per padded i-block of kBatchIB
// rows (which divides kClusterPad, so the block lies inside one cluster), one
// thread per particle.
template <bool COMP>
__global__ void batch_combine_kernel(const float4 *__restrict__ partial,
                                     const int64_t *__restrict__ off, const int64_t *__restrict__ poff,
                                     const int64_t *__restrict__ ibase, int64_t C,
                                     float *__restrict__ a, float *__restrict__ p,
                                     int64_t partial_len, int64_t n_total, int *err) {
    // poff holds the validated padded sizes: all zero when the planner
    // rejected the offsets, so nothing is written for an invalid batch, and
    // a valid cluster's real size never exceeds its padded size.
    constexpr int ib = kBatchIB;
    const int64_t s = (int64_t)blockIdx.x * ib;
    if (s >= poff[C]) return;
    const int64_t c = padded_cluster(poff, C, s);
    const int64_t psz = poff[c + 1] - poff[c];
    const int64_t o = off[c];
    const int64_t nc = off[c + 1] - o < psz ? off[c + 1] - o : psz;
    const int64_t b = (s - poff[c]) / ib, w = threadIdx.x, li = b * ib + w;
    if (li >= nc) return;
    const int64_t nch = chunks_of(psz / kBatchJT);
    const int64_t first = ibase[c] + b * nch;
    float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t k = 0; k < nch; ++k) {
        const int64_t base = (first + k) * (COMP ? 2 : 1) * ib + w;
        if (!NB_IN(err, 14, base + (COMP ? ib : 0) < partial_len)) continue;
        const float4 hi = partial[base];
        const float h[4] = {hi.x, hi.y, hi.z, hi.w};
        if (COMP) {
            const float4 lo = partial[base + ib];
            const float l[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // TwoSum(S, h) then add the chunk's lost low part (h - l is its value)
                const float t = __fadd_rn(S[q], h[q]);
                const float bp = __fsub_rn(t, S[q]);
                const float e = __fadd_rn(__fsub_rn(S[q], __fsub_rn(t, bp)), __fsub_rn(h[q], bp));
                S[q] = t;
                E[q] = __fadd_rn(E[q], __fsub_rn(e, l[q]));
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) S[q] = __fadd_rn(S[q], h[q]);
        }
    }
    const int64_t gi = o + li;
    if (!NB_IN(err, 14, gi >= 0 && gi < n_total)) return;
    constexpr float as = accel_scale(kDefaultRefine), ps = pot_scale(kDefaultRefine);
    a[3 * gi + 0] = as * __fadd_rn(S[0], E[0]);
    a[3 * gi + 1] = as * __fadd_rn(S[1], E[1]);
    a[3 * gi + 2] = as * __fadd_rn(S[2], E[2]);
    p[gi] = ps * __fadd_rn(S[3], E[3]);
}

// Leap-frog pieces that do not pack (the batched pack follows them).
__global__ void batch_kick_drift_kernel(double *__restrict__ x, double *__restrict__ v,
                                        const float *__restrict__ a, int64_t n, double dt,
                                        int kick_back) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const double h = 0.5 * dt, g = -(double)a[k];
    double vc = v[k];
    if (kick_back) vc = vc + h * g;  // Eq. (3) of the previous step
    vc = vc + h * g;                 // Eq. (1)
    v[k] = vc;
    x[k] = x[k] + dt * vc;           // Eq. (2)
}

// Plain mode: the same kick and drift for the particles of one block of
// kClusterPad padded rows, fused with the packing of the moved positions
// (batch_pack_kernel<double>'s records), so the positions are read once.
__global__ void __launch_bounds__(kClusterPad) batch_kick_drift_pack_kernel(
    double *__restrict__ x, double *__restrict__ v, const float *__restrict__ a,
    const float *__restrict__ m, const int64_t *__restrict__ off, const int64_t *__restrict__ poff,
    int64_t C, double dt, int kick_back, JPart *__restrict__ jp) {
    const int64_t s = (int64_t)blockIdx.x * kClusterPad;
    if (s >= poff[C]) return;
    const int64_t c = padded_cluster(poff, C, s);
    const int64_t li = s - poff[c] + threadIdx.x, o = off[c], nc = off[c + 1] - o;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (li < nc) {
        const int64_t i = o + li;
        const double h = 0.5 * dt;
        float q[3];
        for (int k = 0; k < 3; ++k) {
            const int64_t e = 3 * i + k;
            const double g = -(double)a[e];
            double vc = v[e];
            if (kick_back) vc = vc + h * g;  // Eq. (3) of the previous step
            vc = vc + h * g;                 // Eq. (1)
            v[e] = vc;
            const double xn = x[e] + dt * vc;  // Eq. (2)
            x[e] = xn;
            q[k] = (float)xn;
        }
        const float hm = -0.5f * m[i];
        lo = make_float4(-q[0], -q[0], -q[1], -q[1]);
        hi = make_float4(-q[2], -q[2], hm, hm);
    }
    float4 *dst = reinterpret_cast<float4 *>(jp + s + threadIdx.x);
    dst[0] = lo;
    dst[1] = hi;
}

__global__ void batch_kick_kernel(double *__restrict__ v, const float *__restrict__ a, int64_t n,
                                  double dt) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    v[k] = v[k] + (0.5 * dt) * (-(double)a[k]);  // Eq. (3)
}

// Registry of batched shapes.
template <int W, int I, int J, int S, bool C, bool H>
cudaError_t launch_batched(const BatchArgs &a, int grid, size_t smem, cudaStream_t st) {
    batched_pair_kernel<W, I, J, S, C, H><<<grid, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

struct BatchVariant {
    int threads, ipt, jtile, stages;
    bool comp, hl;
    const void *kernel;
    size_t smem;
    cudaError_t (*launch)(const BatchArgs &, int, size_t, cudaStream_t);
};

template <int W, int S, int J, int RS>
constexpr size_t batch_smem() {
    return (size_t)W * S * (J * RS * sizeof(JPart) + sizeof(uint64_t) + sizeof(StageMeta) + sizeof(int));
}

// threads = warps x 32; ipt; jtile; stages; compensated; HL records
#define NB_BVARIANT(W, I, J, S, C, H)                                                           \
    {W * 32, I, J, S, C, H, (const void *)batched_pair_kernel<W, I, J, S, C, H>,                  \
     batch_smem<W, S, J, H ? kHLRecords : 1>(), launch_batched<W, I, J, S, C, H>}

// One warp per CTA (up to 18 resident per SM, bounded by shared memory):
// 0.902 against 0.943 ms per plain evaluation of 1024 clusters with 4 warps
// per CTA (16 resident), the compensated mode unchanged (0.958 ms); 2 stages
// or 4 were slower (GB300, one process, interleaved).
static const BatchVariant kBatch[] = {
    NB_BVARIANT(1, 4, 128, 3, false, false),
    NB_BVARIANT(1, 4, 128, 3, true, false),
    // Compensated on FP64 state (HL records, 64 B per particle): 2 stages keep
    // 13 one-warp CTAs per SM resident (3 stages: 9, bounded by shared memory).
    NB_BVARIANT(1, 4, 128, 2, true, true),
};
#undef NB_BVARIANT

}  // namespace nbk

using namespace nbk;
using namespace nbx;

namespace {

enum BSlot : int {
    B_JP = SLOT_BATCH_JP,
    B_POFF = SLOT_BATCH_POFF,
    B_ITEMS = SLOT_BATCH_ITEMS,
    B_NITEMS = SLOT_BATCH_COUNT,
    B_PART = SLOT_BATCH_PART,
    B_IBASE = SLOT_BATCH_IBASE,
    B_FRAME = SLOT_BATCH_FRAME,
    B_PLANNED = SLOT_BATCH_PLANNED
};

void *bslot(nb_ctx *ctx, int k) { return ctx_ext(ctx).buf[k]; }

nb_status bensure(nb_ctx *ctx, int k, size_t bytes) {
    ExtState &s = ctx_ext(ctx);
    cudaError_t e = ensure_buffer(&s.buf[k], &s.cap[k], bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation (batched)");
    return NB_OK;
}

struct BatchPlanHost {
    const BatchVariant *v;
    int64_t n_total;
    int64_t cap_padded, cap_items;
    int grid;
};

int batch_resident(const BatchVariant &v, int sm_count) {
    if (v.smem > 48 * 1024)
        cudaFuncSetAttribute(v.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.kernel, v.threads, v.smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    cudaGetLastError();
    return per_sm * sm_count;
}

// Scratch for a batch, sized from (n_total, C) alone (offsets stay on the device).
nb_status batch_prepare(nb_ctx *ctx, int64_t C, int64_t n_total, bool comp, bool hl,
                        BatchPlanHost *out) {
    const BatchVariant &v = kBatch[hl ? 2 : comp ? 1 : 0];
    const int ib = 32 * v.ipt;  // one warp per work item
    if (ib != kBatchIB || v.jtile != kBatchJT)
        return fail(ctx, NB_ERR_ARG, "batched shape does not match the planner's block sizes");
    out->v = &v;
    out->n_total = n_total;
    out->cap_padded = n_total + C * (int64_t)kClusterPad;
    out->cap_items = kMaxChunks * (out->cap_padded / ib) + 1;
    if (out->cap_items > 0x7fffffff || C > 0x7fffffff)
        return fail(ctx, NB_ERR_ARG, "batch too large for 32-bit work items");
    out->grid = batch_resident(v, ctx_sm_count(ctx));
    nb_status st;
    if ((st = bensure(ctx, B_JP, (size_t)out->cap_padded * (hl ? kHLRecords : 1) * sizeof(JPart))) !=
        NB_OK)
        return st;
    if ((st = bensure(ctx, B_POFF, (size_t)(C + 1) * sizeof(int64_t))) != NB_OK) return st;
    if ((st = bensure(ctx, B_ITEMS, (size_t)out->cap_items * sizeof(int4))) != NB_OK) return st;
    if ((st = bensure(ctx, B_NITEMS, 2 * sizeof(int))) != NB_OK) return st;  // count, queue head
    if ((st = bensure(ctx, B_IBASE, (size_t)std::max<int64_t>(C, 1) * sizeof(int64_t))) != NB_OK)
        return st;
    if ((st = bensure(ctx, B_PART, (size_t)out->cap_items * ib * sizeof(float4) * (comp ? 2 : 1))) !=
        NB_OK)
        return st;
    return NB_OK;
}

nb_status batch_plan(nb_ctx *ctx, const int64_t *offsets, const float *eps, int64_t C,
                     const BatchPlanHost &h, cudaStream_t st) {
    BatchPlanArgs P{};
    P.off = offsets;
    P.eps = eps;
    P.C = C;
    P.n_total = h.n_total;
    P.cap_padded = h.cap_padded;
    P.cap_items = h.cap_items;
    P.poff = static_cast<int64_t *>(bslot(ctx, B_POFF));
    P.items = static_cast<int4 *>(bslot(ctx, B_ITEMS));
    P.ibase = static_cast<int64_t *>(bslot(ctx, B_IBASE));
    P.nitems = static_cast<int *>(bslot(ctx, B_NITEMS));
    P.err = ctx_err_word(ctx);
    // The previous plan is reused when the offsets and eps are the same
    // values (checked on the device); it can only be in the scratch if the
    // last plan was made for the same (C, n_total), which sized the scratch.
    ExtState &es = ctx_ext(ctx);
    nb_status rs = bensure(ctx, B_PLANNED, (size_t)(C + 1) * sizeof(int64_t) + (size_t)C * sizeof(uint32_t));
    if (rs != NB_OK) return rs;
    P.planned_off = static_cast<int64_t *>(bslot(ctx, B_PLANNED));
    P.planned_eps = reinterpret_cast<uint32_t *>(P.planned_off + C + 1);
    P.replan = !(es.plan_clusters == C && es.plan_total == h.n_total);
    batch_plan_kernel<<<1, kPlanThreads, 0, st>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        es.plan_clusters = es.plan_total = -1;
        return cuda_fail(ctx, e, "batch plan launch");
    }
    es.plan_clusters = C;
    es.plan_total = h.n_total;
    return NB_OK;
}

// pack (already done by the caller of this helper) -> reset queue -> pair kernel
nb_status batch_pair(nb_ctx *ctx, const int64_t *offsets, int64_t C, const float *eps, float *a,
                     float *p, const BatchPlanHost &h, cudaStream_t st) {
    int *nit = static_cast<int *>(bslot(ctx, B_NITEMS));
    cudaError_t e = cudaMemsetAsync(nit + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "queue reset");
    BatchArgs A{};
    A.jp = static_cast<const JPart *>(bslot(ctx, B_JP));
    A.off = offsets;
    A.poff = static_cast<const int64_t *>(bslot(ctx, B_POFF));
    A.eps = eps;
    A.items = static_cast<const int4 *>(bslot(ctx, B_ITEMS));
    A.nitems = nit;
    A.counter = nit + 1;
    A.partial = static_cast<float4 *>(bslot(ctx, B_PART));
    A.err = ctx_err_word(ctx);
    A.wait_ns = ctx_wait_ns(ctx);
    A.cap_padded = h.cap_padded;
    A.cap_items = h.cap_items;
    A.partial_len = h.cap_items * (int64_t)(32 * h.v->ipt) * (h.v->comp ? 2 : 1);
    {
        TimedLaunch t(ctx, 4, st);
        e = h.v->launch(A, h.grid, h.v->smem, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched pair kernel launch");
    const int ib = 32 * h.v->ipt;
    const unsigned nblk = (unsigned)((h.cap_padded + ib - 1) / ib);
    if (h.v->comp)
        batch_combine_kernel<true><<<nblk, ib, 0, st>>>(
            A.partial, offsets, A.poff, static_cast<const int64_t *>(bslot(ctx, B_IBASE)), C, a, p,
            A.partial_len, h.n_total, A.err);
    else
        batch_combine_kernel<false><<<nblk, ib, 0, st>>>(
            A.partial, offsets, A.poff, static_cast<const int64_t *>(bslot(ctx, B_IBASE)), C, a, p,
            A.partial_len, h.n_total, A.err);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "batched combine launch");
    return NB_OK;
}

nb_status check_batch_args(nb_ctx *ctx, int64_t C, int64_t n_total, int mode) {
    if (C < 0 || n_total < 0) return fail(ctx, NB_ERR_ARG, "n_clusters and n_total must be >= 0");
    if (mode != NB_PLAIN && mode != NB_COMPENSATED) return fail(ctx, NB_ERR_ARG, "unknown mode");
    return NB_OK;
}

}  // namespace

extern "C" {

nb_status nb_force_batched(nb_ctx *ctx, const float *x, const float *m, const int64_t *offsets,
                           int64_t n_clusters, int64_t n_total, const float *eps, float *a, float *p,
                           nb_mode mode, void *stream) {
    if (!ctx) return NB_ERR_ARG;
    nb_status st = check_batch_args(ctx, n_clusters, n_total, mode);
    if (st != NB_OK) return st;
    if (n_clusters == 0 || n_total == 0) return NB_OK;
    if (!x || !m || !offsets || !eps || !a || !p) return fail(ctx, NB_ERR_ARG, "NULL array pointer");
    DeviceGuard g(ctx_device(ctx));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchPlanHost h{};
    if ((st = batch_prepare(ctx, n_clusters, n_total, mode == NB_COMPENSATED, false, &h)) != NB_OK)
        return st;
    if ((st = batch_plan(ctx, offsets, eps, n_clusters, h, s)) != NB_OK) return st;
    batch_pack_kernel<float><<<(unsigned)(h.cap_padded / kClusterPad), kClusterPad, 0, s>>>(
        x, m, offsets, static_cast<const int64_t *>(bslot(ctx, B_POFF)), n_clusters,
        static_cast<JPart *>(bslot(ctx, B_JP)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched pack launch");
    return batch_pair(ctx, offsets, n_clusters, eps, a, p, h, s);
}

nb_status nb_leapfrog_batched_step(nb_ctx *ctx, double *x, double *v, const float *m,
                                   const int64_t *offsets, int64_t n_clusters, int64_t n_total,
                                   const float *eps, float *a, float *p, double dt, int nsteps,
                                   int a_valid, nb_mode mode, void *stream) {
    if (!ctx) return NB_ERR_ARG;
    nb_status st = check_batch_args(ctx, n_clusters, n_total, mode);
    if (st != NB_OK) return st;
    if (nsteps < 0) return fail(ctx, NB_ERR_ARG, "nsteps must be >= 0");
    if (!std::isfinite(dt)) return fail(ctx, NB_ERR_ARG, "dt must be finite");
    if (n_clusters == 0 || n_total == 0) return NB_OK;
    if (!x || !v || !m || !offsets || !eps || !a || !p)
        return fail(ctx, NB_ERR_ARG, "NULL array pointer");
    DeviceGuard g(ctx_device(ctx));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool hl = mode == NB_COMPENSATED;
    BatchPlanHost h{};
    if ((st = batch_prepare(ctx, n_clusters, n_total, hl, hl, &h)) != NB_OK) return st;
    if ((st = batch_plan(ctx, offsets, eps, n_clusters, h, s)) != NB_OK) return st;
    const int64_t *poff = static_cast<const int64_t *>(bslot(ctx, B_POFF));
    JPart *jp = static_cast<JPart *>(bslot(ctx, B_JP));
    const unsigned nb3 = (unsigned)((3 * n_total + 255) / 256);
    cudaError_t e;

    double4 *frame = nullptr;
    if (hl) {
        if ((st = bensure(ctx, B_FRAME, (size_t)n_clusters * sizeof(double4))) != NB_OK) return st;
        frame = static_cast<double4 *>(bslot(ctx, B_FRAME));
    }
    const unsigned npack = (unsigned)(h.cap_padded / kClusterPad);
    auto force = [&]() -> nb_status {
        if (hl) {
            batch_frame_kernel<<<(unsigned)n_clusters, kFrameThreads, 0, s>>>(x, offsets, poff, frame);
            batch_pack_hl_kernel<<<npack, kClusterPad, 0, s>>>(x, m, offsets, poff, frame, n_clusters, jp);
        } else {
            batch_pack_kernel<double><<<npack, kClusterPad, 0, s>>>(x, m, offsets, poff, n_clusters, jp);
        }
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return cuda_fail(ctx, le, "batched pack launch");
        return batch_pair(ctx, offsets, n_clusters, eps, a, p, h, s);
    };
    auto step = [&](int kick_back) -> nb_status {
        if (!hl) {  // kick, drift and pack in one pass, then the force
            batch_kick_drift_pack_kernel<<<npack, kClusterPad, 0, s>>>(x, v, a, m, offsets, poff, n_clusters,
                                                                       dt, kick_back, jp);
            cudaError_t le = cudaGetLastError();
            if (le != cudaSuccess) return cuda_fail(ctx, le, "leap-frog update launch");
            return batch_pair(ctx, offsets, n_clusters, eps, a, p, h, s);
        }
        batch_kick_drift_kernel<<<nb3, 256, 0, s>>>(x, v, a, n_total, dt, kick_back);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return cuda_fail(ctx, le, "leap-frog update launch");
        return force();
    };

    if (!a_valid && (st = force()) != NB_OK) return st;
    if (nsteps == 0) return NB_OK;
    if ((st = step(0)) != NB_OK) return st;
    const int rest = nsteps - 1;
    if (rest >= 2 && s != nullptr) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture begin");
        const bool timing = ctx_set_timing(ctx, false);
        nb_status cst = step(1);
        ctx_set_timing(ctx, timing);
        e = cudaStreamEndCapture(s, &graph);
        if (cst != NB_OK) {
            if (graph) cudaGraphDestroy(graph);
            return cst;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture end");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
        for (int k = 0; k < rest && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, s);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    } else {
        for (int k = 0; k < rest; ++k)
            if ((st = step(1)) != NB_OK) return st;
    }
    batch_kick_kernel<<<nb3, 256, 0, s>>>(v, a, n_total, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "kick launch");
    return NB_OK;
}

}  // extern "C"
