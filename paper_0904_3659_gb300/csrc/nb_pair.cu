// nb_pair.cu -- the pair kernel of Eq. (gravity) (Fujiwara & Nakasato,
// arXiv:0904.3659, Section "Introduction") for sm_103a, with its pack and
// combine kernels, the fused single-launch kernel for small n, the registry
// of compiled shapes and the work plan.
//
// Design (GB300-first; the paper's RV770 unrolled loops, Figs. 1-3, are prior
// art whose idea -- reuse one loaded x_j for several i -- is kept):
//  * Each thread holds IPT i-particles in registers, as IPT/2 packed pairs,
//    and every interaction is evaluated with packed FP32x2 instructions
//    (two i against the same j per instruction), which halves the issue
//    slots the FP32 work takes and leaves room for the special-function
//    unit's reciprocal square root and the shared-memory loads.
//  * j-particles stream through shared memory in tiles of JT, copied by the
//    tensor memory accelerator (1-D bulk copies) into STAGES buffers with
//    mbarrier completion; every wait is bounded.
//  * The kernel is persistent: the grid is the number of CTAs that fit on the
//    GPU at once, and the (i-block, j-tile) work units are split into equal
//    contiguous ranges, one per CTA, so every SM gets the same work however
//    N divides. A CTA that covers only part of an i-block's j range writes a
//    partial sum; a second kernel adds the partials of each i-block in CTA
//    order. No float atomics: results are bit-reproducible for a fixed launch.
//  * Per interaction: 13 FP32 lane operations + 1 reciprocal square root,
//    or 16 with the optional Newton step (template knob NEWTON):
//      d  = x_i - x_j                      3 add
//      s  = eps^2 + d.d                    3 fma
//      y  = rsqrt(s)                       1 special-function op
//      NEWTON, folded into the mass:       y2 = y*y, t = s*y2 - 3, u = y*t
//        (the refined value is y1 = -u/2, see tile_pass); else u = y
//      q  = (-m_j/2) * u                   1 mul     p_i += q   1 add
//      w  = q * u*u                        2 mul
//      a_i += w d                           3 fma
//    The sums carry a factor (4 for a and 1 for p with NEWTON, -1/2 for both
//    without) that the combine removes, an exact scaling. On sm_103a the
//    special-function unit's estimate is already within 2^-22.9 of s^{-1/2}
//    and the FP32 Newton step does not improve on it, so the built-in
//    shapes omit it.
#include <algorithm>
#include <cooperative_groups.h>
#include <cstdio>

#include "nb_combine.cuh"
#include "nb_device.cuh"
#include "nb_internal.h"
#include "nb_tile.cuh"

namespace nbk {
using namespace nbdev;

// ---------------------------------------------------------------------------
// Pack: x [n][3], m [n] -> JPart [npad]; rows n..npad-1 are inert (m = 0 at 0).
__global__ void pack_f32_kernel(const float *__restrict__ x, const float *__restrict__ m,
                                int64_t n, int64_t npad, JPart *__restrict__ jp) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 hi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n) {
        const float px = x[3 * i + 0], py = x[3 * i + 1], pz = x[3 * i + 2];
        const float hm = -0.5f * m[i];
        lo = make_float4(-px, -px, -py, -py);
        hi = make_float4(-pz, -pz, hm, hm);
    }
    float4 *dst = reinterpret_cast<float4 *>(jp + i);
    dst[0] = lo;
    dst[1] = hi;
}

// ---------------------------------------------------------------------------
// Persistent pair kernel. See PairArgs for the work split.
//
// Template knobs (all searched by the tuner):
//   THREADS, IPT  CTA size and i-particles per thread (IPT/2 packed pairs)
//   JT, STAGES    j-tile length and number of shared-memory stages
//   UNR           unroll factor of the j loop inside a tile
//   MINB          minimum resident CTAs per SM asked of the register allocator
//   REL           how a consumed stage is handed back to the producer:
//                 0: a CTA-wide barrier per tile, after which thread 0 issues
//                    the copy of the unit STAGES-1 ahead;
//                 1: no barrier: each warp counts itself out of the stage in a
//                    shared counter and the last warp to finish issues the
//                    copy of the unit STAGES ahead into it.
//   ACCS          where the running sums (and Kahan carries) live between
//                 tiles: 0 registers, 1 shared memory (one slot per thread,
//                 touched once per tile; frees 8-16 registers per i-particle)
//   MIX           which op groups of an interaction run packed (see kMix*)
//   NEWTON        one Newton-Raphson step on the reciprocal square root
//   COMP          Kahan-compensated running sums (NB_COMPENSATED)
//   HL            positions are packed as HL records (two JParts per
//                 particle, see kHLRecords): x_i - x_j is formed from the
//                 exact difference of the grid parts plus the difference of
//                 the remainders (tile_pass_hl)
//   NP            no potential: only a_i is summed (12 FP32 operations per
//                 pair); the potential slot of the partial sums stays zero.
template <int THREADS, int IPT, int JT, int STAGES, int UNR, int MINB, int REL, int ACCS, int MIX,
          bool NEWTON, bool COMP, bool HL, bool NP = false>
__global__ void __launch_bounds__(THREADS, MINB) pair_kernel(const PairArgs args) {
    static_assert(IPT % 2 == 0, "i-particles are processed in packed pairs");
    static_assert(!(HL && NEWTON), "the HL pass has no Newton step");
    constexpr int P = IPT / 2;
    constexpr int IB = THREADS * IPT;
    constexpr int NWARPS = THREADS / 32;
    constexpr int RS = HL ? kHLRecords : 1;  // JParts per particle
    constexpr uint32_t TILE_BYTES = JT * RS * sizeof(JPart);
    static_assert(THREADS % 32 == 0, "whole warps");
    static_assert(TILE_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
    // i-blocks and j-tiles must tile the padded particle array exactly, so
    // that every i and j the kernel touches lies inside it.
    static_assert(kPad % IB == 0 && kPad % JT == 0, "tile sizes must divide the padding");

    // Shared memory: [STAGES j-tiles][running sums if ACCS][barriers][counters]
    constexpr int NSUM = ACCS ? (COMP ? 2 : 1) * P * 4 * THREADS : 0;  // float2 slots
    extern __shared__ __align__(128) unsigned char smem[];
    JPart *tiles = reinterpret_cast<JPart *>(smem);
    float2 *ssum = reinterpret_cast<float2 *>(smem + (size_t)STAGES * TILE_BYTES);
    float2 *scmp = ssum + P * 4 * THREADS;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * TILE_BYTES +
                                                  (size_t)NSUM * sizeof(float2));
    int *arrivals = reinterpret_cast<int *>(full + STAGES);  // REL 1: warps done per stage
    int *issued_at = arrivals + STAGES;  // last unit index issued into each stage (-1: none)
    int *abort_flag = issued_at + STAGES;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int64_t c = blockIdx.x;
    const int64_t u0 = c * args.units / args.grid;
    const int64_t u1 = (c + 1) * args.units / args.grid;
    const int count = (int)(u1 - u0);
    const int64_t bfirst = u0 / args.njt;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            arrivals[s] = 0;
            issued_at[s] = -1;
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // Issue the copy of the j-tile of local unit kk into its stage.
    auto issue = [&](int kk) {
        const int s = kk % STAGES;
        const int64_t u = u0 + kk;
        if (u == args.fault_unit) return;  // test hook: this copy never happens
        const int64_t jt = u % args.njt;
        if (!NB_IN(args.err, 2, (jt + 1) * JT <= args.npad)) return;
        issued_at[s] = kk;
        mbar_arrive_expect_tx(&full[s], TILE_BYTES);
        bulk_g2s(tiles + (size_t)s * JT * RS, args.jp + jt * JT * RS, TILE_BYTES, &full[s]);
    };
    if (tid == 0) {
        const int ahead = REL ? STAGES : STAGES - 1;
        for (int kk = 0; kk < count && kk < ahead; ++kk) issue(kk);
    }

    float2 xi[P], yi[P], zi[P];
    float2 lxi[P], lyi[P], lzi[P];  // HL: remainders of the i-particles' positions
    float2 sum[P][4] = {}, cmp[P][4] = {};  // unused when the sums live in shared memory
    const float2 eps2 = splat2(args.eps2);
    const float2 zero2 = splat2(0.f);

    // Running sums: in registers (ACCS 0) or in this thread's shared slots.
    auto get_sum = [&](int q, int r) { return ACCS ? ssum[(q * 4 + r) * THREADS + tid] : sum[q][r]; };
    auto get_cmp = [&](int q, int r) { return ACCS ? scmp[(q * 4 + r) * THREADS + tid] : cmp[q][r]; };
    auto put_sum = [&](int q, int r, float2 v) {
        if (ACCS) ssum[(q * 4 + r) * THREADS + tid] = v; else sum[q][r] = v;
    };
    auto put_cmp = [&](int q, int r, float2 v) {
        if (ACCS) scmp[(q * 4 + r) * THREADS + tid] = v; else cmp[q][r] = v;
    };

    auto flush = [&](int64_t b) {
        const int64_t seg = b - bfirst;
        const int64_t off = (c * args.maxseg + seg) * (COMP ? 2 : 1) * (int64_t)IB;
        if (!NB_IN(args.err, 3, seg >= 0 && seg < args.maxseg &&
                                    off + (COMP ? 2 : 1) * IB <= args.partial_len))
            return;
        float4 *dst = args.partial + off;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int i0 = (2 * q) * THREADS + tid, i1 = i0 + THREADS;
            const float2 s0 = get_sum(q, 0), s1 = get_sum(q, 1), s2 = get_sum(q, 2), s3 = get_sum(q, 3);
            dst[i0] = make_float4(s0.x, s1.x, s2.x, s3.x);
            dst[i1] = make_float4(s0.y, s1.y, s2.y, s3.y);
            if (COMP) {
                const float2 c0 = get_cmp(q, 0), c1 = get_cmp(q, 1), c2 = get_cmp(q, 2),
                             c3 = get_cmp(q, 3);
                dst[IB + i0] = make_float4(c0.x, c1.x, c2.x, c3.x);
                dst[IB + i1] = make_float4(c0.y, c1.y, c2.y, c3.y);
            }
        }
    };

    int64_t b = u0 / args.njt;
    int64_t jt = u0 - b * args.njt;
    int64_t cur_b = -1;
    int bad = 0;
    for (int k = 0; k < count; ++k) {
        if (REL == 0) {
            // Every thread is done with iteration k-1, so its stage may be
            // refilled; a timeout seen by any thread ends the loop for all.
            if (__syncthreads_or(bad)) break;
            if (tid == 0 && k + STAGES - 1 < count) issue(k + STAGES - 1);
        } else if (bad || *reinterpret_cast<volatile int *>(abort_flag)) {
            break;
        }

        if (b != cur_b) {
            if (cur_b >= 0) flush(cur_b);
            cur_b = b;
#pragma unroll
            for (int q = 0; q < P; ++q) {
                int64_t i0 = b * IB + (2 * q) * THREADS + tid, i1 = i0 + THREADS;
                if (!NB_IN(args.err, 1, i1 < args.npad)) i0 = i1 = 0;
                const float4 A0 = reinterpret_cast<const float4 *>(args.jp + i0 * RS)[0];
                const float4 B0 = reinterpret_cast<const float4 *>(args.jp + i0 * RS)[1];
                const float4 A1 = reinterpret_cast<const float4 *>(args.jp + i1 * RS)[0];
                const float4 B1 = reinterpret_cast<const float4 *>(args.jp + i1 * RS)[1];
                xi[q] = make_float2(-A0.x, -A1.x);
                yi[q] = make_float2(-A0.z, -A1.z);
                zi[q] = make_float2(-B0.x, -B1.x);
                if (HL) {
                    const float4 C0 = reinterpret_cast<const float4 *>(args.jp + i0 * RS + 1)[0];
                    const float4 D0 = reinterpret_cast<const float4 *>(args.jp + i0 * RS + 1)[1];
                    const float4 C1 = reinterpret_cast<const float4 *>(args.jp + i1 * RS + 1)[0];
                    const float4 D1 = reinterpret_cast<const float4 *>(args.jp + i1 * RS + 1)[1];
                    lxi[q] = make_float2(-C0.x, -C1.x);
                    lyi[q] = make_float2(-C0.z, -C1.z);
                    lzi[q] = make_float2(-D0.x, -D1.x);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    put_sum(q, r, zero2);
                    if (COMP) put_cmp(q, r, zero2);
                }
            }
        }

        const int s = k % STAGES;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((k / STAGES) & 1), args.wait_ns)) {
            bad = 1;
            if (REL) atomicOr(abort_flag, 1);
            continue;
        }
        const JPart *T = tiles + (size_t)s * JT * RS;

        float2 acc[P][4];
#pragma unroll
        for (int q = 0; q < P; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[q][r] = zero2;

        const int64_t ibase = b * IB, jbase = jt * JT;
        int self0[P], self1[P];
        if (jbase < ibase + IB && ibase < jbase + JT) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                self0[q] = (int)(ibase + (2 * q) * THREADS + tid - jbase);
                self1[q] = self0[q] + THREADS;
            }
            if constexpr (HL)
                tile_pass_hl<P, JT, 1, true, !NP>(T, xi, yi, zi, lxi, lyi, lzi, acc, eps2, self0, self1);
            else
                tile_pass<P, JT, 1, true, MIX, NEWTON, !NP>(T, xi, yi, zi, acc, eps2, self0, self1);
        } else {
            if constexpr (HL)
                tile_pass_hl<P, JT, UNR, false, !NP>(T, xi, yi, zi, lxi, lyi, lzi, acc, eps2, self0,
                                                     self1);
            else
                tile_pass<P, JT, UNR, false, MIX, NEWTON, !NP>(T, xi, yi, zi, acc, eps2, self0, self1);
        }

        if (REL == 1) {
            // Hand the stage back: the last warp out issues its next copy.
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const int target = (k / STAGES + 1) * NWARPS;
                if (atomicAdd(&arrivals[s], 1) == target - 1 && k + STAGES < count) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(k + STAGES);
                }
            }
        }

#pragma unroll
        for (int q = 0; q < P; ++q)
#pragma unroll
            for (int r = 0; r < (NP ? 3 : 4); ++r) {
                if (COMP) {
                    // Kahan: the running sum's lost low part is kept in cmp
                    // (true value = sum - cmp).
                    const float2 s0 = get_sum(q, r);
                    const float2 y = add2(acc[q][r], neg2(get_cmp(q, r)));
                    const float2 t = add2(s0, y);
                    put_cmp(q, r, add2(add2(t, neg2(s0)), neg2(y)));
                    put_sum(q, r, t);
                } else {
                    put_sum(q, r, add2(get_sum(q, r), acc[q][r]));
                }
            }
        if (++jt == args.njt) {
            jt = 0;
            ++b;
        }
    }

    // Every warp leaves the loop (a timed-out wait ends it within the limit).
    bad = __syncthreads_or(bad || *reinterpret_cast<volatile int *>(abort_flag));
    if (!bad) {
        if (cur_b >= 0) flush(cur_b);
        return;
    }
    if (tid == 0) {
        atomicOr(args.err, kErrTimeout);
        // Let every copy still in flight land before this CTA's shared
        // memory is released.
        for (int s = 0; s < STAGES; ++s)
            if (issued_at[s] >= 0)
                mbar_wait_bounded(&full[s], (uint32_t)((issued_at[s] / STAGES) & 1), args.wait_ns);
    }
}

// ---------------------------------------------------------------------------
// Combine: for each i, add the partials of its i-block in CTA order and
// remove the factors the pair kernel's sums carry (r.a_scale, r.p_scale).
// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// Sum, in CTA order, the partials of slot w of i-block b written by CTAs
// clo..chi (layout [cta][maxseg][W][ib] float4, W = 2 with Kahan carries).
// Plain: S += hi. Compensated: TwoSum of the segment values into (S, E).
// The loads of up to 8 segments are issued together (L2 latency, not
// bandwidth, bounds a combine with many segments); the additions keep the
// CTA order, so the result does not depend on the batching. Each CTA's
// segment is located with SegWalk (no 64-bit division per segment).
template <bool COMP>
__device__ __forceinline__ void sum_segments(const float4 *__restrict__ partial, int64_t partial_len,
                                             int *err, int64_t b, int64_t w, int64_t clo, int64_t chi,
                                             int64_t units, int grid, int64_t njt, int maxseg,
                                             int64_t ib, float (&S)[4], float (&E)[4]) {
    constexpr int K = 8;
    constexpr int W = COMP ? 2 : 1;
    SegWalk sw(clo, units, grid, njt);
    for (int64_t c0 = clo; c0 <= chi; c0 += K) {
        float4 hi[K], lo[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t cc = c0 + k;
            hi[k] = lo[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (cc > chi) continue;
            if (cc > clo) sw.next();
            const int64_t bf = sw.bf;
            const int64_t base = (cc * maxseg + (b - bf)) * W * ib + w;
            if (!NB_IN(err, 5, b - bf >= 0 && b - bf < maxseg && base + (W - 1) * ib < partial_len))
                continue;  // (debug build) recorded; the slot adds zero
            hi[k] = __ldcg(partial + base);
            if (COMP) lo[k] = __ldcg(partial + base + ib);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (c0 + k > chi) break;
            const float h[4] = {hi[k].x, hi[k].y, hi[k].z, hi[k].w};
            const float l[4] = {lo[k].x, lo[k].y, lo[k].z, lo[k].w};
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                if (COMP) {
                    float t, e;
                    two_sum(S[qq], h[qq], t, e);
                    S[qq] = t;
                    E[qq] = __fadd_rn(E[qq], __fsub_rn(e, l[qq]));  // segment value = hi - lo
                } else {
                    S[qq] = __fadd_rn(S[qq], h[qq]);
                }
            }
        }
    }
}

template <bool COMP>
__global__ void reduce_kernel(const ReduceArgs r) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= r.n) return;
    const int64_t b = i / r.ib, w = i - b * r.ib;
    const int64_t clo = cta_of_unit(b * r.njt, r.units, r.grid);
    const int64_t chi = cta_of_unit(b * r.njt + r.njt - 1, r.units, r.grid);
    float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
    sum_segments<COMP>(r.partial, r.partial_len, r.err, b, w, clo, chi, r.units, r.grid, r.njt,
                       r.maxseg, r.ib, S, E);
    const int64_t o = i;
    r.a[3 * o + 0] = r.a_scale * __fadd_rn(S[0], E[0]);
    r.a[3 * o + 1] = r.a_scale * __fadd_rn(S[1], E[1]);
    r.a[3 * o + 2] = r.a_scale * __fadd_rn(S[2], E[2]);
    if (r.p) r.p[o] = r.p_scale * __fadd_rn(S[3], E[3]);
}

// ---------------------------------------------------------------------------
// Fused single-launch variant for small n (tile field fused = 1). Work unit:
// (i-block b of IB = 32 IPT particles, j-chunk c of nchunks), one CTA each.
//  * The CTA's WARPS warps all hold the same i-particles (each lane IPT/2
//    packed pairs) and split the chunk's j-range: warp w sums the JT-particle
//    tiles w, w + WARPS, ... of each shared-memory block. The threads load
//    and pack each block of up to JMAX particles from x, m themselves (no
//    pack kernel, no TMA).
//  * The warps' sums are added in warp order through shared memory, giving
//    the CTA's partial for the i-block; the last of the i-block's nchunks
//    CTAs to arrive (a count per i-block, reset by that CTA) adds the chunk
//    partials in chunk order and writes a_i, p_i (no combine kernel).
// Every addition order is fixed by the launch shape, so results are
// bit-reproducible; there are no waits on other CTAs.
constexpr int kFusedJmax = 1024;  // particles per shared-memory block (32 KB)
// Largest cluster of the cluster form: the portable 8 CTAs (clusters of up
// to 16 measured no faster at N = 4096).
constexpr int kMaxClusterChunks = 8;
// Received partials per CTA of a cluster: ceil(IB / nch) slots x nch chunks,
// at most IB + nch - 1, for the largest i-block of the cluster shapes.
constexpr int kClusterSlots = 128 + kMaxClusterChunks;

// Load particles j0 .. j0 + cnt - 1 (cnt <= kFusedJmax) from x, m and pack
// them into blk; rows at or beyond n are inert (m = 0 at the origin). Each
// thread issues the loads of up to 4 particles before any of their stores,
// so the block costs about one L2 round trip instead of four.
template <int THREADS>
__device__ __forceinline__ void pack_block(const float *__restrict__ x, const float *__restrict__ m,
                                           int64_t n, int64_t j0, int cnt, JPart *__restrict__ blk) {
    constexpr int R = 4;
    for (int k0 = 0; k0 < cnt; k0 += R * THREADS) {
        float4 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = k0 + r * THREADS + (int)threadIdx.x;
            const int64_t j = j0 + k;
            v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < cnt && j < n) v[r] = make_float4(x[3 * j], x[3 * j + 1], x[3 * j + 2], m[j]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = k0 + r * THREADS + (int)threadIdx.x;
            if (k >= cnt) continue;
            float4 *dst = reinterpret_cast<float4 *>(blk + k);
            const float hm = -0.5f * v[r].w;
            dst[0] = make_float4(-v[r].x, -v[r].x, -v[r].y, -v[r].y);
            dst[1] = make_float4(-v[r].z, -v[r].z, hm, hm);
        }
    }
}

template <int WARPS, int IPT, int JT, int UNR, int MINB, bool NEWTON, bool COMP>
__global__ void __launch_bounds__(WARPS * 32, MINB) fused_kernel(const FusedArgs args) {
    static_assert(IPT % 2 == 0, "i-particles are processed in packed pairs");
    static_assert(kFusedJmax % JT == 0, "blocks hold whole tiles");
    constexpr int THREADS = WARPS * 32;
    constexpr int P = IPT / 2;
    constexpr int IB = 32 * IPT;
    constexpr int W = COMP ? 2 : 1;  // float4 words per i in a partial
    constexpr int TPB = kFusedJmax / JT;
    static_assert(kPad % IB == 0, "i-blocks must divide the padding");
    static_assert(WARPS * W * IB * sizeof(float4) <= kFusedJmax * sizeof(JPart),
                  "the cross-warp sums reuse the particle block");

    extern __shared__ __align__(128) unsigned char smem[];
    JPart *blk = reinterpret_cast<JPart *>(smem);
    float4 *red = reinterpret_cast<float4 *>(smem);  // [WARPS][W][IB], after the last block
    __shared__ int s_last;
    pdl_wait_then_release();

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = args.n, nch = args.nchunks;
    const int64_t b = blockIdx.x / nch, c = blockIdx.x - b * nch;
    const int64_t t0 = c * args.njt / nch, t1 = (c + 1) * args.njt / nch;  // chunk's tiles

    float2 xi[P], yi[P], zi[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int64_t i0 = b * IB + (2 * q) * 32 + lane, i1 = i0 + 32;
        float3 p0 = make_float3(0.f, 0.f, 0.f), p1 = p0;
        if (i0 < n) p0 = make_float3(args.x[3 * i0], args.x[3 * i0 + 1], args.x[3 * i0 + 2]);
        if (i1 < n) p1 = make_float3(args.x[3 * i1], args.x[3 * i1 + 1], args.x[3 * i1 + 2]);
        xi[q] = make_float2(p0.x, p1.x);
        yi[q] = make_float2(p0.y, p1.y);
        zi[q] = make_float2(p0.z, p1.z);
    }
    const float2 eps2 = splat2(args.eps2);
    const float2 zero2 = splat2(0.f);
    float2 sum[P][4], cmp[P][4];
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) sum[q][r] = cmp[q][r] = zero2;

    for (int64_t bt0 = t0; bt0 < t1; bt0 += TPB) {
        const int64_t bt1 = bt0 + TPB < t1 ? bt0 + TPB : t1;
        const int cnt = (int)(bt1 - bt0) * JT;
        pack_block<THREADS>(args.x, args.m, n, bt0 * JT, cnt, blk);
        __syncthreads();
        for (int64_t t = bt0 + warp; t < bt1; t += WARPS) {
            const JPart *T = blk + (t - bt0) * JT;
            float2 acc[P][4];
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[q][r] = zero2;
            const int64_t ibase = b * IB, jbase = t * JT;
            int self0[P], self1[P];
            if (jbase < ibase + IB && ibase < jbase + JT) {
                // (unrolled like the other tiles: in-process A/B at N = 4096, compensated
                // 15.4 -> 14.5 us, plain unchanged)
                if constexpr (JT == 32) {
                    tile_pass_diag32<P, UNR, NEWTON>((int)((jbase - ibase) / 32), lane, T, xi, yi, zi, acc, eps2);
                } else {
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        self0[q] = (int)(ibase + (2 * q) * 32 + lane - jbase);
                        self1[q] = self0[q] + 32;
                    }
                    tile_pass<P, JT, UNR, true, kMixAll, NEWTON>(T, xi, yi, zi, acc, eps2, self0, self1);
                }
            } else {
                tile_pass<P, JT, UNR, false, kMixAll, NEWTON>(T, xi, yi, zi, acc, eps2, self0, self1);
            }
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (COMP) {
                        // Kahan: true value = sum - cmp.
                        const float2 y = add2(acc[q][r], neg2(cmp[q][r]));
                        const float2 tt = add2(sum[q][r], y);
                        cmp[q][r] = add2(add2(tt, neg2(sum[q][r])), neg2(y));
                        sum[q][r] = tt;
                    } else {
                        sum[q][r] = add2(sum[q][r], acc[q][r]);
                    }
                }
        }
        __syncthreads();  // the block is read by every warp before it is refilled
    }

    // The warps' sums, added in warp order: the CTA's partial for i-block b.
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int i0 = (2 * q) * 32 + lane, i1 = i0 + 32;
        float4 *dst = red + (int64_t)warp * W * IB;
        dst[i0] = make_float4(sum[q][0].x, sum[q][1].x, sum[q][2].x, sum[q][3].x);
        dst[i1] = make_float4(sum[q][0].y, sum[q][1].y, sum[q][2].y, sum[q][3].y);
        if (COMP) {
            dst[IB + i0] = make_float4(cmp[q][0].x, cmp[q][1].x, cmp[q][2].x, cmp[q][3].x);
            dst[IB + i1] = make_float4(cmp[q][0].y, cmp[q][1].y, cmp[q][2].y, cmp[q][3].y);
        }
    }
    __syncthreads();
    const int64_t off = (b * nch + c) * W * (int64_t)IB;
    for (int l = tid; l < IB; l += THREADS) {
        float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
        for (int w = 0; w < WARPS; ++w) {
            const float4 hi = red[(int64_t)w * W * IB + l];
            const float h[4] = {hi.x, hi.y, hi.z, hi.w};
            if (COMP) {
                const float4 lo = red[(int64_t)w * W * IB + IB + l];
                const float lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float t, e;
                    two_sum(S[r], h[r], t, e);
                    S[r] = t;
                    E[r] = __fadd_rn(E[r], __fsub_rn(e, lw[r]));  // warp value = hi - lo
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) S[r] = __fadd_rn(S[r], h[r]);
            }
        }
        if (NB_IN(args.err, 31, off + (W - 1) * IB + l < args.partial_len)) {
            args.partial[off + l] = make_float4(S[0], S[1], S[2], S[3]);
            if (COMP) args.partial[off + IB + l] = make_float4(-E[0], -E[1], -E[2], -E[3]);
        }
    }
    __threadfence();  // this CTA's partial is visible before it counts itself in
    __syncthreads();
    if (tid == 0) {
        int last = 0;
        if (NB_IN(args.err, 32, b >= 0 && b < args.nib)) {
            const int prev = atomicAdd(&args.counters[b], 1);
            last = prev == (int)(nch - 1);
            if (last) atomicExch(&args.counters[b], 0);  // every chunk has arrived
        }
        s_last = last;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int l = tid; l < IB; l += THREADS) {
        const int64_t gi = b * IB + l;
        if (gi >= n) break;
        float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
        // Chunk partials of i-block b are CTAs b*nch .. b*nch + nch - 1, one
        // segment each: the combine's walk over them with units = grid.
        sum_segments<COMP>(args.partial, args.partial_len, args.err, b, l, b * nch, b * nch + nch - 1,
                           args.grid, args.grid, nch, 1, IB, S, E);
        args.a[3 * gi + 0] = args.a_scale * __fadd_rn(S[0], E[0]);
        args.a[3 * gi + 1] = args.a_scale * __fadd_rn(S[1], E[1]);
        args.a[3 * gi + 2] = args.a_scale * __fadd_rn(S[2], E[2]);
        args.p[gi] = args.p_scale * __fadd_rn(S[3], E[3]);
    }
}

// ---------------------------------------------------------------------------
// Stream-K form of the fused kernel (tile field fused = 2), for n up to a few
// 10^4: the (i-block of IB = 32 IPT, JT-particle tile) units are split over
// the resident CTAs in equal contiguous ranges, as in pair_kernel, so every
// SM does the same work; a CTA's range may end in the next i-block (or, when
// there are more i-blocks than CTAs, span several). For each such segment the warps share the segment's tiles as in fused_kernel,
// the warps' sums are added in warp order, the CTA's partial is written in
// pair_kernel's layout and the last contributing CTA of the i-block adds the
// partials in CTA order (the combine kernel's order) and writes a_i, p_i.
template <int WARPS, int IPT, int JT, int UNR, int MINB, bool NEWTON, bool COMP>
__global__ void __launch_bounds__(WARPS * 32, MINB) fused_sk_kernel(const FusedArgs args) {
    static_assert(IPT % 2 == 0, "i-particles are processed in packed pairs");
    static_assert(kFusedJmax % JT == 0, "blocks hold whole tiles");
    constexpr int THREADS = WARPS * 32;
    constexpr int P = IPT / 2;
    constexpr int IB = 32 * IPT;
    constexpr int W = COMP ? 2 : 1;
    constexpr int TPB = kFusedJmax / JT;
    static_assert(kPad % IB == 0, "i-blocks must divide the padding");
    static_assert(WARPS * W * IB * sizeof(float4) <= kFusedJmax * sizeof(JPart),
                  "the cross-warp sums reuse the particle block");

    extern __shared__ __align__(128) unsigned char smem[];
    JPart *blk = reinterpret_cast<JPart *>(smem);
    float4 *red = reinterpret_cast<float4 *>(smem);  // [WARPS][W][IB], after a segment's last block
    __shared__ int s_last;
    pdl_wait_then_release();

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = args.n, njt = args.njt;
    const int64_t c = blockIdx.x;
    const int64_t u0 = c * args.units / args.grid, u1 = (c + 1) * args.units / args.grid;
    const int64_t bfirst = u0 / njt;
    const float2 eps2 = splat2(args.eps2);
    const float2 zero2 = splat2(0.f);

    for (int64_t b = bfirst; b * njt < u1; ++b) {
        const int64_t t0 = (u0 > b * njt ? u0 : b * njt) - b * njt;  // this CTA's tiles of b
        const int64_t t1 = (u1 < (b + 1) * njt ? u1 : (b + 1) * njt) - b * njt;
        float2 xi[P], yi[P], zi[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t i0 = b * IB + (2 * q) * 32 + lane, i1 = i0 + 32;
            float3 p0 = make_float3(0.f, 0.f, 0.f), p1 = p0;
            if (i0 < n) p0 = make_float3(args.x[3 * i0], args.x[3 * i0 + 1], args.x[3 * i0 + 2]);
            if (i1 < n) p1 = make_float3(args.x[3 * i1], args.x[3 * i1 + 1], args.x[3 * i1 + 2]);
            xi[q] = make_float2(p0.x, p1.x);
            yi[q] = make_float2(p0.y, p1.y);
            zi[q] = make_float2(p0.z, p1.z);
        }
        float2 sum[P][4], cmp[P][4];
#pragma unroll
        for (int q = 0; q < P; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) sum[q][r] = cmp[q][r] = zero2;

        for (int64_t bt0 = t0; bt0 < t1; bt0 += TPB) {
            const int64_t bt1 = bt0 + TPB < t1 ? bt0 + TPB : t1;
            const int cnt = (int)(bt1 - bt0) * JT;
            pack_block<THREADS>(args.x, args.m, n, bt0 * JT, cnt, blk);
            __syncthreads();
            for (int64_t t = bt0 + warp; t < bt1; t += WARPS) {
                const JPart *T = blk + (t - bt0) * JT;
                float2 acc[P][4];
#pragma unroll
                for (int q = 0; q < P; ++q)
#pragma unroll
                    for (int r = 0; r < 4; ++r) acc[q][r] = zero2;
                const int64_t ibase = b * IB, jbase = t * JT;
                int self0[P], self1[P];
                if (jbase < ibase + IB && ibase < jbase + JT) {
                    if constexpr (JT == 32) {
                        tile_pass_diag32<P, UNR, NEWTON>((int)((jbase - ibase) / 32), lane, T, xi, yi, zi, acc,
                                                         eps2);
                    } else {
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            self0[q] = (int)(ibase + (2 * q) * 32 + lane - jbase);
                            self1[q] = self0[q] + 32;
                        }
                        tile_pass<P, JT, UNR, true, kMixAll, NEWTON>(T, xi, yi, zi, acc, eps2, self0, self1);
                    }
                } else {
                    tile_pass<P, JT, UNR, false, kMixAll, NEWTON>(T, xi, yi, zi, acc, eps2, self0, self1);
                }
#pragma unroll
                for (int q = 0; q < P; ++q)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (COMP) {
                            // Kahan: true value = sum - cmp.
                            const float2 y = add2(acc[q][r], neg2(cmp[q][r]));
                            const float2 tt = add2(sum[q][r], y);
                            cmp[q][r] = add2(add2(tt, neg2(sum[q][r])), neg2(y));
                            sum[q][r] = tt;
                        } else {
                            sum[q][r] = add2(sum[q][r], acc[q][r]);
                        }
                    }
            }
            __syncthreads();  // the block is read by every warp before it is refilled or reused
        }

        // The warps' sums, added in warp order: the CTA's partial for i-block b.
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int i0 = (2 * q) * 32 + lane, i1 = i0 + 32;
            float4 *dst = red + (int64_t)warp * W * IB;
            dst[i0] = make_float4(sum[q][0].x, sum[q][1].x, sum[q][2].x, sum[q][3].x);
            dst[i1] = make_float4(sum[q][0].y, sum[q][1].y, sum[q][2].y, sum[q][3].y);
            if (COMP) {
                dst[IB + i0] = make_float4(cmp[q][0].x, cmp[q][1].x, cmp[q][2].x, cmp[q][3].x);
                dst[IB + i1] = make_float4(cmp[q][0].y, cmp[q][1].y, cmp[q][2].y, cmp[q][3].y);
            }
        }
        __syncthreads();
        const int64_t seg = b - bfirst;
        const int64_t off = (c * args.maxseg + seg) * W * (int64_t)IB;
        for (int l = tid; l < IB; l += THREADS) {
            float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
            for (int w = 0; w < WARPS; ++w) {
                const float4 hi = red[(int64_t)w * W * IB + l];
                const float h[4] = {hi.x, hi.y, hi.z, hi.w};
                if (COMP) {
                    const float4 lo = red[(int64_t)w * W * IB + IB + l];
                    const float lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        float t, e;
                        two_sum(S[r], h[r], t, e);
                        S[r] = t;
                        E[r] = __fadd_rn(E[r], __fsub_rn(e, lw[r]));  // warp value = hi - lo
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) S[r] = __fadd_rn(S[r], h[r]);
                }
            }
            if (NB_IN(args.err, 33, seg < args.maxseg && off + (W - 1) * IB + l < args.partial_len)) {
                args.partial[off + l] = make_float4(S[0], S[1], S[2], S[3]);
                if (COMP) args.partial[off + IB + l] = make_float4(-E[0], -E[1], -E[2], -E[3]);
            }
        }
        const int64_t clo = cta_of_unit(b * njt, args.units, args.grid);
        const int64_t chi = cta_of_unit(b * njt + njt - 1, args.units, args.grid);
        __threadfence();  // this CTA's partial is visible before it counts itself in
        __syncthreads();  // (also: every thread is done with red before the next block load)
        if (tid == 0) {
            int last = 0;
            if (NB_IN(args.err, 34, b >= 0 && b < args.nib)) {
                const int prev = atomicAdd(&args.counters[b], 1);
                last = prev == (int)(chi - clo);
                if (last) atomicExch(&args.counters[b], 0);  // every contributor has arrived
            }
            s_last = last;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int l = tid; l < IB; l += THREADS) {
                const int64_t gi = b * IB + l;
                if (gi >= n) break;
                float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
                sum_segments<COMP>(args.partial, args.partial_len, args.err, b, l, clo, chi,
                                   args.units, args.grid, njt, (int)args.maxseg, IB, S, E);
                args.a[3 * gi + 0] = args.a_scale * __fadd_rn(S[0], E[0]);
                args.a[3 * gi + 1] = args.a_scale * __fadd_rn(S[1], E[1]);
                args.a[3 * gi + 2] = args.a_scale * __fadd_rn(S[2], E[2]);
                args.p[gi] = args.p_scale * __fadd_rn(S[3], E[3]);
            }
        }
        __syncthreads();  // s_last is read by every thread before the next segment writes it
    }
}

// ---------------------------------------------------------------------------
// Cluster form of the chunked fused kernel (tile field fused = 3). The same
// work split as fused_kernel -- one CTA per (i-block, j-chunk), all warps on
// the same i, the chunk's tiles shared among the warps -- but the nch CTAs of
// an i-block form one thread-block cluster, and the chunks' partial sums meet
// in distributed shared memory: each CTA sends its partial of i-particle l
// to the shared memory of the cluster's CTA l % nch (st.async, counted as
// transaction bytes on that CTA's mbarrier), and CTA r, once its mbarrier
// has counted every byte sent to it (a bounded wait), adds the nch partials
// of its particles l = r, r + nch, ... in chunk order (the chunked form's
// order and arithmetic, so the results are the same bits) and writes a_i,
// p_i. No partials in global memory, no arrival count, no cluster-wide
// barrier after the compute: a CTA waits only for the bytes it receives, and
// every CTA's shared memory outlives the stores into it. Launched with the
// cluster size nch (<= 8) as a launch attribute.
template <int WARPS, int IPT, int JT, int UNR, int MINB, bool NEWTON, bool COMP>
__global__ void __launch_bounds__(WARPS * 32, MINB) fused_cl_kernel(const FusedArgs args) {
    namespace cg = cooperative_groups;
    static_assert(IPT % 2 == 0, "i-particles are processed in packed pairs");
    static_assert(kFusedJmax % JT == 0, "blocks hold whole tiles");
    constexpr int THREADS = WARPS * 32;
    constexpr int P = IPT / 2;
    constexpr int IB = 32 * IPT;
    constexpr int W = COMP ? 2 : 1;  // float4 words per i in a partial
    constexpr int TPB = kFusedJmax / JT;
    static_assert(kPad % IB == 0, "i-blocks must divide the padding");
    static_assert(WARPS * W * IB * sizeof(float4) <= kFusedJmax * sizeof(JPart),
                  "the cross-warp sums reuse the particle block");
    static_assert(IB + kMaxClusterChunks <= kClusterSlots, "room for the received partials");

    extern __shared__ __align__(128) unsigned char smem[];
    JPart *blk = reinterpret_cast<JPart *>(smem);
    float4 *red = reinterpret_cast<float4 *>(smem);  // [WARPS][W][IB], after the last block
    // Received chunk partials of this CTA's particles: [slot][chunk][W].
    float4 *cpart = reinterpret_cast<float4 *>(smem + kFusedJmax * sizeof(JPart));
    __shared__ uint64_t recv_bar;  // counts the bytes the other chunks send here
    pdl_wait_then_release();
    cg::cluster_group cluster = cg::this_cluster();

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = args.n, nch = args.nchunks;
    const int64_t b = blockIdx.x / nch;
    const int c = (int)cluster.block_rank();  // = blockIdx.x % nch
    const int64_t t0 = c * args.njt / nch, t1 = (c + 1) * args.njt / nch;  // chunk's tiles
    if (tid == 0) {
        // This CTA owns l = c, c + nch, ... < IB; each of the other nch - 1
        // chunks sends it W float4 per owned particle.
        const uint32_t owned = (uint32_t)((IB - c + nch - 1) / nch);
        mbar_init(&recv_bar, 1);
        mbar_arrive_expect_tx(&recv_bar, owned * (uint32_t)(nch - 1) * W * (uint32_t)sizeof(float4));
        fence_mbar_init();
    }
    // Distributed shared memory may be touched only once every CTA of the
    // cluster runs and has set up its mbarrier: arrive now, wait just before
    // the first remote store.
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");

    float2 xi[P], yi[P], zi[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int64_t i0 = b * IB + (2 * q) * 32 + lane, i1 = i0 + 32;
        float3 p0 = make_float3(0.f, 0.f, 0.f), p1 = p0;
        if (i0 < n) p0 = make_float3(args.x[3 * i0], args.x[3 * i0 + 1], args.x[3 * i0 + 2]);
        if (i1 < n) p1 = make_float3(args.x[3 * i1], args.x[3 * i1 + 1], args.x[3 * i1 + 2]);
        xi[q] = make_float2(p0.x, p1.x);
        yi[q] = make_float2(p0.y, p1.y);
        zi[q] = make_float2(p0.z, p1.z);
    }
    const float2 eps2 = splat2(args.eps2);
    const float2 zero2 = splat2(0.f);
    float2 sum[P][4], cmp[P][4];
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) sum[q][r] = cmp[q][r] = zero2;

    for (int64_t bt0 = t0; bt0 < t1; bt0 += TPB) {
        const int64_t bt1 = bt0 + TPB < t1 ? bt0 + TPB : t1;
        const int cnt = (int)(bt1 - bt0) * JT;
        pack_block<THREADS>(args.x, args.m, n, bt0 * JT, cnt, blk);
        __syncthreads();
        for (int64_t t = bt0 + warp; t < bt1; t += WARPS) {
            const JPart *T = blk + (t - bt0) * JT;
            float2 acc[P][4];
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[q][r] = zero2;
            const int64_t ibase = b * IB, jbase = t * JT;
            int self0[P], self1[P];
            if (jbase < ibase + IB && ibase < jbase + JT) {
                if constexpr (JT == 32) {
                    tile_pass_diag32<P, UNR, NEWTON>((int)((jbase - ibase) / 32), lane, T, xi, yi, zi, acc, eps2);
                } else {
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        self0[q] = (int)(ibase + (2 * q) * 32 + lane - jbase);
                        self1[q] = self0[q] + 32;
                    }
                    tile_pass<P, JT, UNR, true, kMixAll, NEWTON>(T, xi, yi, zi, acc, eps2, self0, self1);
                }
            } else {
                tile_pass<P, JT, UNR, false, kMixAll, NEWTON>(T, xi, yi, zi, acc, eps2, self0, self1);
            }
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (COMP) {
                        // Kahan: true value = sum - cmp.
                        const float2 y = add2(acc[q][r], neg2(cmp[q][r]));
                        const float2 tt = add2(sum[q][r], y);
                        cmp[q][r] = add2(add2(tt, neg2(sum[q][r])), neg2(y));
                        sum[q][r] = tt;
                    } else {
                        sum[q][r] = add2(sum[q][r], acc[q][r]);
                    }
                }
        }
        __syncthreads();  // the block is read by every warp before it is refilled
    }

    // The warps' sums, added in warp order: this CTA's partial, kept in its
    // own shared memory for the cluster.
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int i0 = (2 * q) * 32 + lane, i1 = i0 + 32;
        float4 *dst = red + (int64_t)warp * W * IB;
        dst[i0] = make_float4(sum[q][0].x, sum[q][1].x, sum[q][2].x, sum[q][3].x);
        dst[i1] = make_float4(sum[q][0].y, sum[q][1].y, sum[q][2].y, sum[q][3].y);
        if (COMP) {
            dst[IB + i0] = make_float4(cmp[q][0].x, cmp[q][1].x, cmp[q][2].x, cmp[q][3].x);
            dst[IB + i1] = make_float4(cmp[q][0].y, cmp[q][1].y, cmp[q][2].y, cmp[q][3].y);
        }
    }
    __syncthreads();
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");  // every CTA of the cluster runs
    // This CTA's partial for i-particle l goes straight into the shared
    // memory of the CTA that owns l (rank l % nch), in the slot of this
    // chunk; its own particles' partials are stored locally. No CTA reads
    // another's shared memory.
    const bool send = (int64_t)blockIdx.x != args.fault_cta;  // test hook
    for (int l = tid; l < IB; l += THREADS) {
        float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
        for (int w = 0; w < WARPS; ++w) {
            const float4 hi = red[(int64_t)w * W * IB + l];
            const float h[4] = {hi.x, hi.y, hi.z, hi.w};
            if (COMP) {
                const float4 lo = red[(int64_t)w * W * IB + IB + l];
                const float lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float t, e;
                    two_sum(S[r], h[r], t, e);
                    S[r] = t;
                    E[r] = __fadd_rn(E[r], __fsub_rn(e, lw[r]));  // warp value = hi - lo
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) S[r] = __fadd_rn(S[r], h[r]);
            }
        }
        // Owner rank l % nch keeps its particles' partials at [slot][chunk][W],
        // slot = l / nch (fewer than IB / nch + 1 slots).
        const int owner = l % (int)nch, slot = l / (int)nch;
        float4 *dst = cpart + ((int64_t)slot * nch + c) * W;
        const float4 hi = make_float4(S[0], S[1], S[2], S[3]);
        const float4 lo = make_float4(-E[0], -E[1], -E[2], -E[3]);
        if (owner == c) {
            dst[0] = hi;
            if (COMP) dst[1] = lo;
        } else if (send) {
            const uint32_t raddr = cluster_map(dst, (uint32_t)owner);
            const uint32_t rbar = cluster_map(&recv_bar, (uint32_t)owner);
            st_async_v4(raddr, hi, rbar);
            if (COMP) st_async_v4(raddr + (uint32_t)sizeof(float4), lo, rbar);
        }
    }
    // Every chunk partial of this CTA's particles has arrived: the other
    // chunks' by the mbarrier's byte count (bounded wait; on a timeout the
    // CTA records it and writes nothing), this CTA's own by the barrier.
    const bool arrived = mbar_wait_bounded(&recv_bar, 0, args.wait_ns);
    __syncthreads();
    if (!arrived) {
        if (tid == 0) atomicOr(args.err, kErrTimeout);
        return;
    }

    // CTA c adds, for its i-particles l = c, c + nch, ..., the nch chunk
    // partials in chunk order (the chunked form's combine) and writes a_i, p_i.
    for (int slot = tid; slot * (int)nch + c < IB; slot += THREADS) {
        const int l = slot * (int)nch + c;
        const int64_t gi = b * IB + l;
        if (gi >= n) break;
        float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < (int)nch; ++k) {
            const float4 *src = cpart + ((int64_t)slot * nch + k) * W;
            const float4 hi = src[0];
            const float h[4] = {hi.x, hi.y, hi.z, hi.w};
            if (COMP) {
                const float4 lo = src[1];
                const float lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float t, e;
                    two_sum(S[r], h[r], t, e);
                    S[r] = t;
                    E[r] = __fadd_rn(E[r], __fsub_rn(e, lw[r]));  // chunk value = hi - lo
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) S[r] = __fadd_rn(S[r], h[r]);
            }
        }
        args.a[3 * gi + 0] = args.a_scale * __fadd_rn(S[0], E[0]);
        args.a[3 * gi + 1] = args.a_scale * __fadd_rn(S[1], E[1]);
        args.a[3 * gi + 2] = args.a_scale * __fadd_rn(S[2], E[2]);
        args.p[gi] = args.p_scale * __fadd_rn(S[3], E[3]);
    }
}

// Synthetic inputs for tuning runs (timing only; values do not matter
// beyond being finite): x uniform in [-1, 1)^3 from a 64-bit mixer, m = 1/n.
__global__ void fill_uniform_kernel(float *x, float *m, int64_t n, uint64_t seed) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 3; ++c) {
        uint64_t z = seed + (uint64_t)(3 * i + c) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[3 * i + c] = (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
    m[i] = 1.0f / (float)n;
}

// ---------------------------------------------------------------------------
// Launchers and the registry of compiled shapes.
template <int T, int I, int J, int S, int U, int M, int R, int A, int X, bool N, bool C, bool F,
          bool NP = false>
static cudaError_t launch_pair(const PairArgs &a, int grid, size_t smem, cudaStream_t st) {
    pair_kernel<T, I, J, S, U, M, R, A, X, N, C, F, NP><<<grid, T, smem, st>>>(a);
    return cudaGetLastError();
}

// The single-launch kernels go out with programmatic stream serialization
// (see pdl_wait_then_release).
template <typename K>
static cudaError_t launch_pdl(K kernel, const FusedArgs &a, int grid, int threads, size_t smem,
                              cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <int WARPS, int I, int J, int U, int M, bool N, bool C>
static cudaError_t launch_fused(const FusedArgs &a, int grid, size_t smem, cudaStream_t st) {
    return launch_pdl(fused_kernel<WARPS, I, J, U, M, N, C>, a, grid, WARPS * 32, smem, st);
}

template <int WARPS, int I, int J, int U, int M, bool N, bool C>
static cudaError_t launch_fused_sk(const FusedArgs &a, int grid, size_t smem, cudaStream_t st) {
    return launch_pdl(fused_sk_kernel<WARPS, I, J, U, M, N, C>, a, grid, WARPS * 32, smem, st);
}

// The cluster form: clusters of a.nchunks CTAs (one i-block each), plus the
// programmatic dependent launch of the other single-launch kernels.
template <int WARPS, int I, int J, int U, int M, bool N, bool C>
static cudaError_t launch_fused_cl(const FusedArgs &a, int grid, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)(WARPS * 32));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = (unsigned)a.nchunks;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, fused_cl_kernel<WARPS, I, J, U, M, N, C>, a);
}


template <int T, int I, int J, int S, int A, bool C, int RS = 1>
constexpr size_t pair_smem() {
    // stages, running sums, their barriers, arrival counters, issue records, abort flag
    return (size_t)S * J * RS * sizeof(JPart) +
           (A ? (C ? 2 : 1) * (I / 2) * 4 * T * sizeof(float2) : 0) + (size_t)S * sizeof(uint64_t) +
           (2 * S + 1) * sizeof(int);
}

// One registry entry: tile fields in nb_tile order (refine last), then the
// compensated flag.
#define NB_VARIANT(T, I, J, S, U, M, R, A, X, N, C)                                             \
    {{T, I, J, S, U, M, R, A, X, N}, C,                                                         \
     (const void *)pair_kernel<T, I, J, S, U, M, R, A, X, (N != 0), C, false>,                  \
     pair_smem<T, I, J, S, A, C>(), launch_pair<T, I, J, S, U, M, R, A, X, (N != 0), C, false>,  \
     nullptr}
// Shapes without the potential (NP), for callers that need only a_i; H: HL records.
#define NB_VARIANT_NP(T, I, J, S, U, M, R, A, X, C, H, NP)                                      \
    {{T, I, J, S, U, M, R, A, X, 0}, C,                                                         \
     (const void *)pair_kernel<T, I, J, S, U, M, R, A, X, false, C, H, NP>,                     \
     pair_smem<T, I, J, S, A, C, H ? kHLRecords : 1>(),                                         \
     launch_pair<T, I, J, S, U, M, R, A, X, false, C, H, NP>, nullptr}
// Fused single-launch shapes: T threads (T / 32 warps sharing one i-block of
// 32 I particles), J-particle warp tiles, one shared-memory block of
// kFusedJmax particles (stages = 1).
#define NB_FUSED(T, I, J, U, M, N, C)                                                        \
    {{T, I, J, 1, U, M, 0, 0, 63, N, 1}, C,                                                     \
     (const void *)fused_kernel<T / 32, I, J, U, M, (N != 0), C>, kFusedJmax * sizeof(JPart), \
     nullptr, launch_fused<T / 32, I, J, U, M, (N != 0), C>}
// The chunked shapes in cluster form (fused = 3): the particle block plus
// the received chunk partials in shared memory. Here minblocks is the CTAs
// per SM: 2 holds the registers to 128 per thread; 1 requests
// kClusterOneSmSmem, so that exactly one CTA runs per SM whatever the
// register count (at N = 4096, 32 clusters of 4 CTAs on 128 SMs: 11.0 us per
// call, against 11.3 us when the 128-register kernel ran two CTAs per SM in
// clusters of 8: 256 CTAs, two on 104 SMs).
constexpr size_t kClusterOneSmSmem = 120 * 1024;
static_assert(kClusterOneSmSmem >= kFusedJmax * sizeof(JPart) + 2 * kClusterSlots * sizeof(float4) &&
                  kClusterOneSmSmem <= 227 * 1024,
              "one CTA's shared memory: room for the cluster form, more than half an SM's");
#define NB_FUSED_CL(T, I, J, U, M, N, C)                                                          \
    {{T, I, J, 1, U, M, 0, 0, 63, N, 3}, C,                                                        \
     (const void *)fused_cl_kernel<T / 32, I, J, U, M, (N != 0), C>,                               \
     (M) == 1 ? kClusterOneSmSmem                                                                   \
              : kFusedJmax * sizeof(JPart) + (size_t)(C ? 2 : 1) * kClusterSlots * sizeof(float4), \
     nullptr, launch_fused_cl<T / 32, I, J, U, M, (N != 0), C>}
// The same shapes in stream-K form (fused = 2).
#define NB_FUSED_SK(T, I, J, U, M, N, C)                                                        \
    {{T, I, J, 1, U, M, 0, 0, 63, N, 2}, C,                                                        \
     (const void *)fused_sk_kernel<T / 32, I, J, U, M, (N != 0), C>, kFusedJmax * sizeof(JPart), \
     nullptr, launch_fused_sk<T / 32, I, J, U, M, (N != 0), C>}

// Plain shapes. The first group evaluates the reciprocal square root without
// the Newton step (refine 0, 13 FP32 ops per pair); the second keeps the
// step (16 ops) for comparison and for callers that ask for it. Measured on
// GB300 with the step: the all-packed mask 63 beats every scalar or mixed
// mask; IPT 6-12 with ~2 warps per scheduler are fastest at large n.
static const PairVariant kPlain[] = {
    NB_VARIANT(128, 8, 256, 3, 8, 1, 1, 0, 63, 0, false),
    NB_VARIANT(128, 6, 256, 3, 8, 1, 1, 1, 63, 0, false),
    NB_VARIANT(128, 12, 256, 3, 4, 1, 0, 1, 63, 0, false),
    NB_VARIANT(128, 8, 512, 3, 8, 1, 0, 0, 63, 0, false),
    NB_VARIANT(128, 8, 256, 3, 8, 1, 1, 1, 63, 0, false),
    NB_VARIANT(256, 4, 256, 3, 4, 1, 0, 0, 63, 0, false),
    NB_VARIANT(256, 2, 128, 4, 4, 1, 0, 0, 63, 0, false),
    NB_VARIANT(128, 2, 128, 4, 4, 1, 0, 0, 63, 0, false),
    NB_VARIANT(64, 2, 64, 4, 4, 1, 0, 0, 63, 0, false),
    NB_VARIANT(64, 4, 128, 4, 4, 1, 0, 0, 63, 0, false),
    NB_VARIANT(256, 4, 512, 3, 4, 1, 0, 0, 63, 0, false),
    NB_VARIANT(384, 4, 1024, 3, 4, 1, 0, 0, 63, 0, false),
    // Kahan-compensated running sum in plain mode (the compensated combine
    // follows): on sm_103a this kernel's compiled schedule runs 2.7% faster
    // than the plain running sum's at the same shape (ncu: 1.3% fewer
    // instructions), so it is the plain path's large-n shape.
    NB_VARIANT(256, 4, 1024, 3, 4, 1, 0, 0, 63, 0, true),
    NB_VARIANT(256, 4, 256, 3, 4, 2, 0, 0, 63, 0, false),
    NB_VARIANT(128, 4, 256, 3, 4, 4, 0, 0, 63, 0, false),
    NB_VARIANT(128, 8, 256, 3, 8, 3, 1, 0, 63, 0, false),
    NB_VARIANT(128, 6, 256, 3, 4, 3, 0, 1, 63, 0, false),
    NB_VARIANT(128, 8, 256, 3, 8, 1, 1, 0, 63, 1, false),
    NB_VARIANT(64, 2, 64, 4, 4, 1, 0, 0, 63, 1, false),
    NB_VARIANT(128, 8, 512, 3, 8, 1, 0, 0, 63, 1, false),
    NB_VARIANT(128, 8, 256, 3, 4, 1, 0, 0, 63, 1, false),
    NB_VARIANT(128, 12, 256, 3, 4, 1, 0, 1, 63, 1, false),
    NB_VARIANT(128, 6, 256, 3, 8, 1, 1, 1, 63, 1, false),
    NB_VARIANT(128, 8, 256, 3, 8, 1, 1, 0, 0, 1, false),
    NB_VARIANT(128, 8, 256, 3, 8, 1, 1, 0, 28, 1, false),
    NB_VARIANT(256, 4, 256, 3, 4, 1, 0, 0, 63, 1, false),
    NB_VARIANT(256, 2, 128, 4, 4, 1, 0, 0, 63, 1, false),
    NB_VARIANT(128, 2, 128, 4, 4, 1, 0, 0, 63, 1, false),
    NB_VARIANT(64, 4, 128, 4, 4, 1, 0, 0, 63, 1, false),
    NB_FUSED(256, 4, 32, 4, 1, 0, false),
    NB_FUSED(256, 2, 32, 4, 1, 0, false),
    NB_FUSED(512, 2, 32, 4, 1, 0, false),
    NB_FUSED_SK(256, 4, 32, 4, 1, 0, false),
    NB_FUSED_SK(128, 4, 32, 4, 1, 0, false),
    NB_FUSED_CL(256, 4, 32, 4, 1, 0, false),
    NB_FUSED_CL(256, 2, 32, 4, 1, 0, false),
    NB_FUSED_CL(256, 4, 32, 4, 2, 0, false),
    NB_FUSED_CL(256, 2, 32, 4, 2, 0, false),
};
static const PairVariant kComp[] = {
    NB_VARIANT(128, 6, 256, 3, 8, 1, 0, 1, 63, 0, true),
    NB_VARIANT(256, 4, 512, 3, 4, 1, 0, 0, 63, 0, true),
    NB_VARIANT(256, 4, 768, 3, 4, 1, 0, 0, 63, 0, true),
    NB_VARIANT(128, 8, 256, 3, 8, 1, 1, 1, 63, 0, true),
    NB_VARIANT(128, 12, 256, 3, 4, 1, 0, 1, 63, 0, true),
    NB_VARIANT(256, 4, 256, 3, 4, 1, 0, 0, 63, 0, true),
    NB_VARIANT(64, 2, 64, 4, 4, 1, 0, 0, 63, 0, true),
    NB_VARIANT(128, 2, 128, 4, 4, 1, 0, 0, 63, 0, true),
    NB_VARIANT(256, 2, 128, 4, 4, 1, 0, 0, 63, 0, true),
    NB_VARIANT(256, 4, 256, 3, 4, 2, 0, 0, 63, 0, true),
    NB_VARIANT(128, 4, 256, 3, 4, 4, 0, 0, 63, 0, true),
    NB_VARIANT(128, 6, 256, 3, 4, 3, 0, 1, 63, 0, true),
    NB_VARIANT(128, 6, 256, 3, 8, 1, 0, 1, 63, 1, true),
    NB_VARIANT(64, 2, 64, 4, 4, 1, 0, 0, 63, 1, true),
    NB_VARIANT(256, 4, 256, 3, 4, 1, 0, 0, 63, 1, true),
    NB_VARIANT(128, 8, 256, 3, 8, 1, 1, 1, 63, 1, true),
    NB_VARIANT(128, 12, 256, 3, 4, 1, 0, 1, 63, 1, true),
    NB_VARIANT(128, 8, 256, 3, 8, 1, 1, 1, 0, 1, true),
    NB_VARIANT(128, 4, 256, 3, 4, 1, 0, 0, 63, 1, true),
    NB_VARIANT(256, 2, 128, 4, 4, 1, 0, 0, 63, 1, true),
    NB_VARIANT(128, 2, 128, 4, 4, 1, 0, 0, 63, 1, true),
    NB_FUSED(256, 4, 32, 4, 1, 0, true),
    NB_FUSED(256, 2, 32, 4, 1, 0, true),
    NB_FUSED(512, 2, 32, 4, 1, 0, true),
    NB_FUSED_SK(256, 4, 32, 4, 1, 0, true),
    NB_FUSED_SK(128, 4, 32, 4, 1, 0, true),
    NB_FUSED_CL(256, 4, 32, 4, 1, 0, true),
    NB_FUSED_CL(256, 2, 32, 4, 1, 0, true),
    NB_FUSED_CL(256, 4, 32, 4, 2, 0, true),
    NB_FUSED_CL(256, 2, 32, 4, 2, 0, true),
};
// HL variants (compensated, positions from FP64 state as HL records), with
// and without the potential, for large and for small n.
static const PairVariant kHL[2][2] = {
    {NB_VARIANT_NP(256, 4, 512, 3, 4, 1, 0, 0, 63, true, true, false),   // large n (the N = 2^16
                                                                         // leap-frog: 1% faster than 256)
     NB_VARIANT_NP(64, 4, 128, 4, 4, 1, 0, 0, 63, true, true, false)},   // small n
    {NB_VARIANT_NP(256, 4, 512, 3, 4, 1, 0, 0, 63, true, true, true),
     NB_VARIANT_NP(64, 4, 128, 4, 4, 1, 0, 0, 63, true, true, true)},
};
// No-potential twins of the built-in packed plain-mode shapes (the
// integrator's force from packed FP64 state, and nb_force with p NULL), and
// of a large-N shape the tuner may pick.
static const PairVariant kNoPot[] = {
    NB_VARIANT_NP(256, 2, 128, 4, 4, 1, 0, 0, 63, false, false, true),
    NB_VARIANT_NP(64, 4, 128, 4, 4, 1, 0, 0, 63, false, false, true),
    NB_VARIANT_NP(256, 4, 256, 3, 4, 1, 0, 0, 63, false, false, true),
    NB_VARIANT_NP(128, 12, 256, 3, 4, 1, 0, 1, 63, false, false, true),
    NB_VARIANT_NP(256, 4, 1024, 3, 4, 1, 0, 0, 63, true, false, true),
    NB_VARIANT_NP(256, 4, 512, 3, 4, 1, 0, 0, 63, false, false, true),
};
static_assert(kDefaultRefine == 0, "the no-potential and HL shapes have no Newton step");
#undef NB_VARIANT
#undef NB_VARIANT_NP
#undef NB_FUSED
#undef NB_FUSED_SK
#undef NB_FUSED_CL

static int pair_variant_index(bool comp, const nb_tile &t);

const PairVariant *hl_variant(int64_t n, bool no_pot) {
    return &kHL[no_pot ? 1 : 0][n >= (int64_t)1 << 15 ? 0 : 1];
}

const PairVariant *chunked_twin(const PairVariant &v) {
    nb_tile t = v.tile;
    t.fused = 1;
    const int k = pair_variant_index(v.comp, t);
    return k >= 0 ? pair_variant(v.comp, k) : nullptr;
}

const PairVariant *no_pot_twin(const PairVariant &v) {
    if (v.tile.fused) return nullptr;
    for (const PairVariant &w : kNoPot)
        if (w.comp == v.comp && same_tile(w.tile, v.tile)) return &w;
    return nullptr;
}

int pair_variant_count(bool comp) {
    return comp ? (int)(sizeof(kComp) / sizeof(kComp[0])) : (int)(sizeof(kPlain) / sizeof(kPlain[0]));
}

const PairVariant *pair_variant(bool comp, int idx) {
    if (idx < 0 || idx >= pair_variant_count(comp)) return nullptr;
    return comp ? &kComp[idx] : &kPlain[idx];
}

static int pair_variant_index(bool comp, const nb_tile &t) {
    for (int k = 0; k < pair_variant_count(comp); ++k)
        if (same_tile(pair_variant(comp, k)->tile, t)) return k;
    return -1;
}

// Built-in packed (not fused) choices per size class, from the measured shape
// sweep (GB300, no Newton step): 2 i per thread and 128-particle tiles while
// the work cannot fill 152 SMs with large i-blocks, then 4 i per thread in
// 256-thread CTAs. From N = 2^17 on, plain mode takes 1024-particle tiles
// with the Kahan running sum (N = 2^20: 2639 against 2572 G-int/s for the
// plain running sum at the same shape); from 2^15, 512-particle tiles, whose
// no-potential twin runs the N = 2^16 leap-frog 0.8% faster than 256-particle
// tiles and 1.4% faster than the Kahan shape's (N = 2^16 with the potential:
// 2511 against 2491 for 256 and 2594 for the Kahan shape, which the tuner
// picks). Compensated mode takes 512-particle tiles from N = 2^15 (N = 2^16:
// 2574 against 2539 for 256 and 2507 for 768) and 768-particle tiles from
// 2^17 (N = 2^20: 2629 against 2618 for 512 and 2582 for 256; every shape
// stays within the mode's 1e-6, the 1536-particle tiles did not).
int pair_default_unfused_index(bool comp, int64_t n) {
    constexpr int R = kDefaultRefine;
    static const nb_tile shapes[2][4] = {
        {{256, 2, 128, 4, 4, 1, 0, 0, 63, R}, {64, 4, 128, 4, 4, 1, 0, 0, 63, R},
         {256, 4, 512, 3, 4, 1, 0, 0, 63, R}, {256, 4, 1024, 3, 4, 1, 0, 0, 63, R}},
        {{256, 2, 128, 4, 4, 1, 0, 0, 63, R}, {256, 4, 256, 3, 4, 1, 0, 0, 63, R},
         {256, 4, 512, 3, 4, 1, 0, 0, 63, R}, {256, 4, 768, 3, 4, 1, 0, 0, 63, R}}};
    static const int idx[2][4] = {
        {pair_variant_index(false, shapes[0][0]), pair_variant_index(false, shapes[0][1]),
         pair_variant_index(false, shapes[0][2]), pair_variant_index(false, shapes[0][3])},
        {pair_variant_index(true, shapes[1][0]), pair_variant_index(true, shapes[1][1]),
         pair_variant_index(true, shapes[1][2]), pair_variant_index(true, shapes[1][3])}};
    const int cls = n >= (int64_t)1 << 17 ? 3 : n >= (int64_t)1 << 15 ? 2 : n >= (int64_t)1 << 13 ? 1 : 0;
    const int k = idx[comp ? 1 : 0][cls];
    return k >= 0 ? k : 0;  // every default above is compiled; 0 guards a stale edit
}

// Single-launch shapes by size (GB300, whole calls, plain / compensated):
// the cluster form up to kClusterMaxN, 2 i per lane below kClusterWideMinN
// (N = 2048: 5.8 / 5.7 us against 7.1 / 7.5 with 4) and 4 from there (N =
// 3072: 8.6 / 9.2 us against 9.2 / 9.9 with 2, whose clusters of 3 do not
// all fit; N = 4096: 11.0 / 11.7 against 12.6 / 13.3 for the chunked form and
// 30.7 for pack + pair + combine; N = 9216: 40.7 / 41.8 against 44.4 / 45.4
// for the stream-K form). kClusterMaxN is 76 i-blocks of 128: the most
// clusters of two that fit at once at one CTA per SM (N = 9728: 42.6 / 43.9
// against 45.9 / 46.7 for stream-K; at N = 10240 the 80 clusters do not fit
// and stream-K wins, 53.5 / 54.6 against 59.2 / 61.0). The stream-K form from
// there to kFusedMaxN (N = 12288: 73.8 / 77.5 us against 92.2 / 94.4 us for
// the best packed shapes; N = 16384: 129.0 / 133.5 against 137.2 / 141.3
// us), the packed shapes above (N = 24576: stream-K 279.0 / 290.5 us against
// 280.5 / 280.7).
constexpr int64_t kClusterMaxN = (int64_t)76 * 128;
constexpr int64_t kClusterWideMinN = (int64_t)3 << 10;
constexpr int64_t kFusedMaxN = (int64_t)3 << 13;

bool fused_candidate(int64_t n) { return n < (int64_t)1 << 16; }

int pair_default_index(bool comp, int64_t n) {
    if (n >= kFusedMaxN) return pair_default_unfused_index(comp, n);
    constexpr int R = kDefaultRefine;
    // Up to kClusterMaxN the cluster form (the chunked split, partials met in
    // distributed shared memory; it runs as the chunked form when its
    // clusters do not fit at once), one CTA per SM: 2 i per lane below
    // kClusterWideMinN, 4 from there.
    static const nb_tile cl2{256, 2, 32, 1, 4, 1, 0, 0, 63, R, 3};
    static const nb_tile cl4{256, 4, 32, 1, 4, 1, 0, 0, 63, R, 3};
    static const nb_tile streamk{256, 4, 32, 1, 4, 1, 0, 0, 63, R, 2};
    static const int idx[3][2] = {{pair_variant_index(false, cl2), pair_variant_index(true, cl2)},
                                  {pair_variant_index(false, cl4), pair_variant_index(true, cl4)},
                                  {pair_variant_index(false, streamk), pair_variant_index(true, streamk)}};
    const int cls = n < kClusterWideMinN ? 0 : n <= kClusterMaxN ? 1 : 2;
    const int k = idx[cls][comp ? 1 : 0];
    return k >= 0 ? k : pair_default_unfused_index(comp, n);
}

PairPlan make_plan(const PairVariant &v, int64_t n, int resident_ctas) {
    PairPlan p{};
    p.n = n;
    p.smem = v.smem;
    if (v.tile.fused == 3) {
        // Cluster form: one CTA per (i-block, j-chunk), the chunks of an
        // i-block one cluster of at most kMaxClusterChunks CTAs, as many as
        // the resident CTAs allow; no global partials.
        p.ib = 32 * v.tile.ipt;
        p.npad = round_up(std::max<int64_t>(n, 1), kPad);
        p.nib = (n + p.ib - 1) / p.ib;
        p.njt = (n + v.tile.jtile - 1) / v.tile.jtile;
        p.nchunks = std::max<int64_t>(
            1, std::min<int64_t>({p.njt, (int64_t)kMaxClusterChunks, resident_ctas / std::max<int64_t>(p.nib, 1)}));
        p.units = p.nib * p.nchunks;
        p.grid = (int)p.units;
        p.maxseg = 1;
        p.words = v.comp ? 2 : 1;
        p.partial_bytes = 0;
        return p;
    }
    if (v.tile.fused == 1) {
        // One CTA per (i-block, j-chunk); as many chunks as fill the GPU once.
        p.ib = 32 * v.tile.ipt;
        p.npad = round_up(std::max<int64_t>(n, 1), kPad);
        p.nib = (n + p.ib - 1) / p.ib;
        p.njt = (n + v.tile.jtile - 1) / v.tile.jtile;
        p.nchunks = std::max<int64_t>(1, std::min<int64_t>(p.njt, resident_ctas / std::max<int64_t>(p.nib, 1)));
        p.units = p.nib * p.nchunks;
        p.grid = (int)p.units;
        p.maxseg = 1;
        p.words = v.comp ? 2 : 1;
        p.partial_bytes = (size_t)p.grid * p.words * p.ib * sizeof(float4);
        return p;
    }
    // Stream-K split of (i-block, j-tile) units over the resident CTAs: the
    // pair kernel, and the fused kernel's stream-K form (whose warps share
    // one i-block of 32 ipt particles).
    p.nchunks = 1;
    p.ib = (v.tile.fused ? 32 : v.tile.threads) * v.tile.ipt;
    p.npad = round_up(std::max<int64_t>(n, 1), kPad);
    p.nib = (n + p.ib - 1) / p.ib;
    p.njt = (n + v.tile.jtile - 1) / v.tile.jtile;
    p.units = p.nib * p.njt;
    p.grid = (int)std::max<int64_t>(1, std::min<int64_t>(p.units, resident_ctas));
    int maxseg = 1;
    for (int64_t c = 0; c < p.grid; ++c) {
        const int64_t u0 = c * p.units / p.grid, u1 = (c + 1) * p.units / p.grid;
        if (u1 <= u0) continue;
        maxseg = std::max<int>(maxseg, (int)((u1 - 1) / p.njt - u0 / p.njt + 1));
    }
    p.maxseg = maxseg;
    p.words = v.comp ? 2 : 1;
    p.partial_bytes = (size_t)p.grid * p.maxseg * p.words * p.ib * sizeof(float4);
    return p;
}

cudaError_t launch_pack_f32(const float *x, const float *m, int64_t n, int64_t npad, JPart *jp,
                            cudaStream_t st) {
    const int threads = 256;
    const int64_t blocks = (npad + threads - 1) / threads;
    pack_f32_kernel<<<(unsigned)blocks, threads, 0, st>>>(x, m, n, npad, jp);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReduceArgs &r, bool comp, cudaStream_t st) {
    const int threads = 64;  // latency-bound: spread small n over many SMs
    const int64_t blocks = (r.n + threads - 1) / threads;
    if (comp)
        reduce_kernel<true><<<(unsigned)blocks, threads, 0, st>>>(r);
    else
        reduce_kernel<false><<<(unsigned)blocks, threads, 0, st>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_fill_uniform(float *x, float *m, int64_t n, uint64_t seed, cudaStream_t st) {
    const int threads = 256;
    const int64_t blocks = (n + threads - 1) / threads;
    fill_uniform_kernel<<<(unsigned)blocks, threads, 0, st>>>(x, m, n, seed);
    return cudaGetLastError();
}

}  // namespace nbk
