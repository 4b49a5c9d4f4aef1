// nb_vjp.cu -- vector-Jacobian product of Eq. (gravity) (Fujiwara & Nakasato,
// arXiv:0904.3659, Section "Introduction"): for upstream gradients ga_i (on
// a_i) and gp_i (on p_i), the gradient of L = sum_i ga_i . a_i + gp_i p_i
// with respect to positions and masses, as one gather pass over all pairs.
//
// For particle i and every l != i, with r = x_i - x_l, s = |r|^2 + eps^2 and
// y = s^{-1/2} (chain rule of the definition):
//   gx_i += m_l [y^3 ga_i - 3 y^5 (r.ga_i) r - gp_i y^3 r]
//         - m_i [y^3 ga_l - 3 y^5 (r.ga_l) r + gp_l y^3 r]
//   gm_i += -(r.ga_l) y^3 + gp_l y
// Regrouped per pair into a coefficient of r and three sums:
//   gx_i = ga_i sum_l m_l y^3 - m_i sum_l y^3 ga_l + sum_l c_il r
//   c_il = 3 y^5 (m_i r.ga_l - m_l r.ga_i) - y^3 (gp_i m_l + m_i gp_l)
// The kernel forms, per pair, with the packed gradient value h_l (below) and
// u the reciprocal square root in the form chosen by kVNewton,
//   C = u^3 (u^2 a + b),  a = m_l (3 ga_i).r + (-3 m_i) ga_l.r,  b = h_i' m_l + (-m_i) h_l
// and accumulates, per i,
//   R = sum C r,  S = sum m_l u^3,  V = sum u^3 ga_l,  G = sum ((r.ga_l) u^3 + h_l u)
// where h_i' = -h_i. With an upstream gradient on p the record carries
// k_l = h_l / 3 instead of h_l, and the kernel regroups u^2 a + b as
//   m_l (u^2 (3 ga_i).r + h_i') + (-3 m_i)(u^2 ga_l.r + k_l)
// (two independent FMAs, then one FMA and one product), and G as
// sum (r.ga_l) u^3 + 3 sum k_l u, the two sums kept apart within a j-tile.
//  * Without the Newton step (the default): u = y, h_l = -gp_l, so C = -c_il,
//    G = -gm_i and gx_i = -R + ga_i S - m_i V, gm_i = -G; 28 FP32 operations
//    per pair.
//  * With it: u = -2 y1 (y1 the refined value, as in the force kernel),
//    h_l = -4 gp_l: y^3 = -u^3/8 and y^5 = -u^5/32 give C = 32 c_il, G = 8 gm_i,
//    so gx_i = R/32 - ga_i S/8 + m_i V/8, gm_i = G/8; 31 operations.
// The scale factors of the combine are exact powers of two; the factor 3 of
// k_l costs one rounding of h_l / 3. One special-function reciprocal square
// root per pair. With no upstream gradient on p (gp NULL) the terms in h
// vanish: C = u^5 a and G = sum (r.ga_l) u^3, 26 operations.
#include <algorithm>
#include <cmath>

#include "nb_combine.cuh"
#include "nb_device.cuh"
#include "nb_ext.h"
#include "nb_internal.h"

namespace nbk {
using namespace nbdev;

// Newton step on the reciprocal square root (see the header comment).
constexpr bool kVNewton = kDefaultRefine != 0;
// Gradient value h = kVGp * gp (the record holds h / 3), and the combine's
// factors for R, S, V, G.
constexpr float kVGp = kVNewton ? -4.f : -1.f;
constexpr float kVScaleR = kVNewton ? 0.03125f : -1.f;
constexpr float kVScaleS = kVNewton ? -0.125f : 1.f;
constexpr float kVScaleV = kVNewton ? 0.125f : -1.f;
constexpr float kVScaleG = kVNewton ? 0.125f : -1.f;

// One j-particle of the VJP pass, 64 bytes, each value duplicated for packed
// FP32x2 use: (-x, -y, -z, m, ga_x, ga_y, ga_z, k = kVGp gp / 3).
struct alignas(64) VPart {
    float2 nx, ny, nz, m, gx, gy, gz, k;
};
static_assert(sizeof(VPart) == 64, "VPart must be 64 bytes");

__global__ void vjp_pack_kernel(const float *__restrict__ x, const float *__restrict__ m,
                                const float *__restrict__ ga, const float *__restrict__ gp,
                                int64_t n, int64_t npad, VPart *__restrict__ vp) {
    pdl_wait_then_release();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < n) {
        v[0] = -x[3 * i];
        v[1] = -x[3 * i + 1];
        v[2] = -x[3 * i + 2];
        v[3] = m[i];
        v[4] = ga[3 * i];
        v[5] = ga[3 * i + 1];
        v[6] = ga[3 * i + 2];
        v[7] = gp ? __fdiv_rn(kVGp * gp[i], 3.f) : 0.f;
    }
    float4 *dst = reinterpret_cast<float4 *>(vp + i);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = make_float4(v[2 * k], v[2 * k], v[2 * k + 1], v[2 * k + 1]);
}

struct VjpArgs {
    const VPart *vp;
    const float *x, *m, *ga, *gp;  // originals (i-side constants)
    float4 *partial;               // [grid][maxseg][2][ib]
    int *err;
    int64_t n, njt, units;
    int grid, maxseg;
    float eps2;
    uint64_t wait_ns;
    int64_t fault_unit;         // test hook: unit whose copy is never issued (-1: none)
    int64_t npad, partial_len;  // extents (debug-build bounds checks)
};

// DIAG with DS >= 0: the lane-diagonal form. Only i-slot DS of the thread
// (pair DS / 2, half DS % 2) meets itself in this tile, at jj == self0[0]
// (a warp-uniform offset plus the lane), so the self term costs one compare
// and one select per j.
template <int P, int JT, int UNR, bool DIAG, bool GP, int DS = -1>
__device__ __forceinline__ void vjp_tile(const VPart *__restrict__ T, const float2 (&xi)[P],
                                         const float2 (&yi)[P], const float2 (&zi)[P],
                                         const float2 (&g3x)[P], const float2 (&g3y)[P],
                                         const float2 (&g3z)[P], const float2 (&nm3)[P],
                                         const float2 (&gp4)[P], float2 (&acc)[P][GP ? 9 : 8],
                                         const float2 eps2, const int (&self0)[P],
                                         const int (&self1)[P]) {
    const float2 m3 = splat2(-3.f);
#pragma unroll UNR
    for (int jj = 0; jj < JT; ++jj) {
        const float4 A = reinterpret_cast<const float4 *>(T + jj)[0];
        const float4 B = reinterpret_cast<const float4 *>(T + jj)[1];
        const float4 C = reinterpret_cast<const float4 *>(T + jj)[2];
        const float4 D = reinterpret_cast<const float4 *>(T + jj)[3];
        const float2 nxj = make_float2(A.x, A.y), nyj = make_float2(A.z, A.w);
        const float2 nzj = make_float2(B.x, B.y), mj = make_float2(B.z, B.w);
        const float2 gxj = make_float2(C.x, C.y), gyj = make_float2(C.z, C.w);
        const float2 gzj = make_float2(D.x, D.y), kj = make_float2(D.z, D.w);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const float2 dx = add2(xi[q], nxj), dy = add2(yi[q], nyj), dz = add2(zi[q], nzj);
            float2 s = fma2(dx, dx, eps2);
            s = fma2(dy, dy, s);
            s = fma2(dz, dz, s);
            const float2 y = make_float2(rsqrt_sfu(s.x), rsqrt_sfu(s.y));
            float2 u = kVNewton ? mul2(y, fma2(s, mul2(y, y), m3)) : y;  // -2 y1, or y
            if constexpr (DIAG && DS >= 0) {
                static_assert(DS < 2 * P, "slot index");
                if (q == DS / 2 && jj == self0[0]) {
                    if (DS % 2 == 0) u.x = 0.f;
                    else u.y = 0.f;
                }
            } else if constexpr (DIAG) {
                if (jj == self0[q]) u.x = 0.f;
                if (jj == self1[q]) u.y = 0.f;
            }
            const float2 u2 = mul2(u, u);
            const float2 u3 = mul2(u, u2);
            const float2 dgi3 = fma2(dz, g3z[q], fma2(dy, g3y[q], mul2(dx, g3x[q])));  // 3 r.ga_i
            const float2 dgj = fma2(dz, gzj, fma2(dy, gyj, mul2(dx, gxj)));           // r.ga_l
            float2 c32;
            if constexpr (GP) {
                const float2 t1 = fma2(u2, dgi3, gp4[q]);  // u^2 (3 r.ga_i) + h_i'
                const float2 t2 = fma2(u2, dgj, kj);        // u^2 r.ga_l + k_l
                c32 = mul2(u3, fma2(mj, t1, mul2(nm3[q], t2)));
            } else {
                c32 = mul2(u3, mul2(u2, fma2(mj, dgi3, mul2(nm3[q], dgj))));  // u^5 a
            }
            acc[q][0] = fma2(c32, dx, acc[q][0]);
            acc[q][1] = fma2(c32, dy, acc[q][1]);
            acc[q][2] = fma2(c32, dz, acc[q][2]);
            acc[q][3] = fma2(mj, u3, acc[q][3]);
            acc[q][4] = fma2(u3, gxj, acc[q][4]);
            acc[q][5] = fma2(u3, gyj, acc[q][5]);
            acc[q][6] = fma2(u3, gzj, acc[q][6]);
            acc[q][7] = fma2(dgj, u3, acc[q][7]);
            if constexpr (GP) acc[q][8] = fma2(kj, u, acc[q][8]);
        }
    }
}

// A tile that holds some of the thread's own i-particles. Slot k of thread
// tid is particle ibase + k * THREADS + tid, and the tile starts at jbase;
// with THREADS and JT multiples of 32 and the tile at most THREADS wide, at
// most one slot of a warp meets the tile, all 32 lanes at once, at
// jj = (that slot's first particle - jbase) + lane. The warp runs the
// lane-diagonal form for that slot, or the plain form when none meets it.
template <int THREADS, int P, int JT, int UNR, bool GP, int K = 0>
__device__ __forceinline__ void vjp_tile_diag(int64_t ibase, int64_t jbase, int tid,
                                              const VPart *__restrict__ T, const float2 (&xi)[P],
                                              const float2 (&yi)[P], const float2 (&zi)[P],
                                              const float2 (&g3x)[P], const float2 (&g3y)[P],
                                              const float2 (&g3z)[P], const float2 (&nm3)[P],
                                              const float2 (&gp4)[P], float2 (&acc)[P][GP ? 9 : 8],
                                              const float2 eps2) {
    static_assert(THREADS % 32 == 0 && JT % 32 == 0 && JT <= THREADS, "warp-aligned slots");
    int self0[P], self1[P];
    if constexpr (K < 2 * P) {
        const int64_t first = ibase + (int64_t)K * THREADS + (tid & ~31);  // the warp's slot-K block
        if (first < jbase + JT && jbase < first + 32) {
            self0[0] = (int)(first - jbase) + (tid & 31);
            vjp_tile<P, JT, UNR, true, GP, K>(T, xi, yi, zi, g3x, g3y, g3z, nm3, gp4, acc, eps2, self0,
                                              self1);
        } else {
            vjp_tile_diag<THREADS, P, JT, UNR, GP, K + 1>(ibase, jbase, tid, T, xi, yi, zi, g3x, g3y,
                                                          g3z, nm3, gp4, acc, eps2);
        }
    } else {
        vjp_tile<P, JT, UNR, false, GP>(T, xi, yi, zi, g3x, g3y, g3z, nm3, gp4, acc, eps2, self0,
                                        self1);
    }
}

// THREADS, IPT (i per thread, in packed pairs), JT (j-tile), STAGES (TMA
// stages), UNR (unroll of the j loop), ACCS (running sums in shared memory,
// one slot per thread, touched once per tile: frees 16 registers per pair).
// GP: the upstream gradient on p is not zero (its terms are summed).
// REL: how a consumed stage goes back to the producer: 0, a CTA-wide barrier
// per tile after which thread 0 issues the copy STAGES-1 tiles ahead; 1, no
// barrier: each warp counts itself out of the stage and the last warp out
// issues the copy STAGES tiles ahead into it.
template <int THREADS, int IPT, int JT, int STAGES, int UNR, int ACCS, bool GP, int MINB = 1,
          int REL = 0>
__global__ void __launch_bounds__(THREADS, MINB) vjp_kernel(const VjpArgs args) {
    constexpr int P = IPT / 2;
    constexpr int IB = THREADS * IPT;
    constexpr int NWARPS = THREADS / 32;
    constexpr uint32_t TILE_BYTES = JT * sizeof(VPart);
    static_assert(kPad % IB == 0 && kPad % JT == 0, "tile sizes must divide the padding");

    // Shared memory: [STAGES j-tiles][running sums if ACCS][barriers][counters]
    extern __shared__ __align__(128) unsigned char smem[];
    VPart *tiles = reinterpret_cast<VPart *>(smem);
    float2 *ssum = reinterpret_cast<float2 *>(smem + (size_t)STAGES * TILE_BYTES);  // ACCS
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * TILE_BYTES +
                                                  (ACCS ? (size_t)P * 8 * THREADS * sizeof(float2) : 0));
    int *arrivals = reinterpret_cast<int *>(full + STAGES);  // REL 1: warps done per stage
    int *issued_at = arrivals + STAGES;  // last tile index issued into each stage (-1: none)
    int *abort_flag = issued_at + STAGES;

    pdl_wait_then_release();
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
        if (u0 + kk == args.fault_unit) return;  // test hook: this copy never happens
        const int64_t jt = (u0 + kk) % args.njt;
        if (!NB_IN(args.err, 21, (jt + 1) * JT <= args.npad)) return;
        issued_at[s] = kk;
        mbar_arrive_expect_tx(&full[s], TILE_BYTES);
        bulk_g2s(tiles + (size_t)s * JT, args.vp + jt * JT, TILE_BYTES, &full[s]);
    };
    if (tid == 0) {
        const int ahead = REL ? STAGES : STAGES - 1;
        for (int kk = 0; kk < count && kk < ahead; ++kk) issue(kk);
    }

    float2 xi[P], yi[P], zi[P], g3x[P], g3y[P], g3z[P], nm3[P], gp4[P];
    float2 sum[P][8] = {};  // unused when the running sums live in shared memory
    const float2 eps2 = splat2(args.eps2);
    const float2 zero2 = splat2(0.f);
    auto get_sum = [&](int q, int r) { return ACCS ? ssum[(q * 8 + r) * THREADS + tid] : sum[q][r]; };
    auto put_sum = [&](int q, int r, float2 v) {
        if (ACCS) ssum[(q * 8 + r) * THREADS + tid] = v; else sum[q][r] = v;
    };

    auto flush = [&](int64_t b) {
        const int64_t off = (c * args.maxseg + (b - bfirst)) * 2 * (int64_t)IB;
        if (!NB_IN(args.err, 22, b - bfirst < args.maxseg && off + 2 * IB <= args.partial_len)) return;
        float4 *dst = args.partial + off;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int i0 = (2 * q) * THREADS + tid, i1 = i0 + THREADS;
            float2 v[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) v[r] = get_sum(q, r);
            dst[i0] = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
            dst[i1] = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
            dst[IB + i0] = make_float4(v[4].x, v[5].x, v[6].x, v[7].x);
            dst[IB + i1] = make_float4(v[4].y, v[5].y, v[6].y, v[7].y);
        }
    };

    int64_t b = u0 / args.njt;
    int64_t jt = u0 - b * args.njt;
    int64_t cur_b = -1;
    int bad = 0, k = 0;
    for (; k < count; ++k) {
        if (REL == 0) {
            // Every thread is done with tile k-1, so its stage may be
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
                float e[2][8];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int64_t i = b * IB + (2 * q + h) * THREADS + tid;
                    if (!NB_IN(args.err, 20, i < args.npad)) i = 0;
                    const VPart &V = args.vp[i];
                    e[h][0] = -V.nx.x;
                    e[h][1] = -V.ny.x;
                    e[h][2] = -V.nz.x;
                    e[h][3] = 3.f * V.gx.x;
                    e[h][4] = 3.f * V.gy.x;
                    e[h][5] = 3.f * V.gz.x;
                    e[h][6] = -3.f * V.m.x;
                    e[h][7] = (GP && i < args.n) ? -kVGp * args.gp[i] : 0.f;  // h_i' = -h_i
                }
                xi[q] = make_float2(e[0][0], e[1][0]);
                yi[q] = make_float2(e[0][1], e[1][1]);
                zi[q] = make_float2(e[0][2], e[1][2]);
                g3x[q] = make_float2(e[0][3], e[1][3]);
                g3y[q] = make_float2(e[0][4], e[1][4]);
                g3z[q] = make_float2(e[0][5], e[1][5]);
                nm3[q] = make_float2(e[0][6], e[1][6]);
                gp4[q] = make_float2(e[0][7], e[1][7]);
#pragma unroll
                for (int r = 0; r < 8; ++r) put_sum(q, r, zero2);
            }
        }
        const int s = k % STAGES;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((k / STAGES) & 1), args.wait_ns)) {
            bad = 1;
            if (REL) atomicOr(abort_flag, 1);
            continue;
        }
        const VPart *T = tiles + (size_t)s * JT;
        constexpr int NACC = GP ? 9 : 8;
        float2 acc[P][NACC];
#pragma unroll
        for (int q = 0; q < P; ++q)
#pragma unroll
            for (int r = 0; r < NACC; ++r) acc[q][r] = zero2;
        const int64_t ibase = b * IB, jbase = jt * JT;
        int self0[P], self1[P];
        if (jbase < ibase + IB && ibase < jbase + JT) {
            if constexpr (JT <= THREADS) {
                vjp_tile_diag<THREADS, P, JT, UNR, GP>(ibase, jbase, tid, T, xi, yi, zi, g3x, g3y, g3z,
                                                       nm3, gp4, acc, eps2);
            } else {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    self0[q] = (int)(ibase + (2 * q) * THREADS + tid - jbase);
                    self1[q] = self0[q] + THREADS;
                }
                vjp_tile<P, JT, 1, true, GP>(T, xi, yi, zi, g3x, g3y, g3z, nm3, gp4, acc, eps2, self0,
                                             self1);
            }
        } else {
            vjp_tile<P, JT, UNR, false, GP>(T, xi, yi, zi, g3x, g3y, g3z, nm3, gp4, acc, eps2, self0,
                                         self1);
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
        for (int q = 0; q < P; ++q) {
            if constexpr (GP) acc[q][7] = fma2(splat2(3.f), acc[q][8], acc[q][7]);  // + 3 sum k_l u
#pragma unroll
            for (int r = 0; r < 8; ++r) put_sum(q, r, add2(get_sum(q, r), acc[q][r]));
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

// Combine the per-segment sums of each i (CTA order) and form gx, gm.
__global__ void vjp_combine_kernel(const VjpArgs A, int ib, float *__restrict__ gx,
                                   float *__restrict__ gm) {
    pdl_wait_then_release();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const int64_t b = i / ib, w = i - b * ib;
    const int64_t clo = cta_of_unit(b * A.njt, A.units, A.grid);
    const int64_t chi = cta_of_unit(b * A.njt + A.njt - 1, A.units, A.grid);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // Loads of up to 8 segments in flight, additions in CTA order.
    constexpr int K = 8;
    SegWalk sw(clo, A.units, A.grid, A.njt);
    for (int64_t c0 = clo; c0 <= chi; c0 += K) {
        float4 p0[K], p1[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t c = c0 + k;
            p0[k] = p1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c > chi) continue;
            if (c > clo) sw.next();
            const int64_t bf = sw.bf;
            const int64_t base = (c * A.maxseg + (b - bf)) * 2 * ib + w;
            if (!NB_IN(A.err, 23, b - bf < A.maxseg && base + ib < A.partial_len)) continue;
            p0[k] = __ldcg(A.partial + base);
            p1[k] = __ldcg(A.partial + base + ib);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (c0 + k > chi) break;
            const float v[8] = {p0[k].x, p0[k].y, p0[k].z, p0[k].w, p1[k].x, p1[k].y, p1[k].z, p1[k].w};
#pragma unroll
            for (int r = 0; r < 8; ++r) s[r] = __fadd_rn(s[r], v[r]);
        }
    }
    const float mi = A.m[i];
    // gx = kVScaleR R + kVScaleS ga_i S + kVScaleV m_i V
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float gai = A.ga[3 * i + c];
        const float t = __fmaf_rn(mi, kVScaleV * s[4 + c], gai * (kVScaleS * s[3]));
        gx[3 * i + c] = __fadd_rn(kVScaleR * s[c], t);
    }
    gm[i] = kVScaleG * s[7];
}

}  // namespace nbk

using namespace nbk;
using namespace nbx;

namespace {

enum VSlot : int { V_VP = SLOT_VJP_VP, V_PART = SLOT_VJP_PART };

// Compiled VJP shapes (nb_tile fields: threads, ipt, jtile, stages, unroll,
// sums_in_smem; the others fixed). Entry kVjpDefault is the built-in choice.
struct VjpVariant {
    nb_tile tile;
    const void *kernel[2];  // [0]: no upstream gradient on p; [1]: with it
    size_t smem;
    void (*launch[2])(const VjpArgs &, int grid, size_t smem, cudaStream_t);
};

template <int T, int I, int J, int S, int U, int A, bool G, int M, int R>
void launch_vjp(const VjpArgs &a, int grid, size_t smem, cudaStream_t st) {
    launch_with_pdl(vjp_kernel<T, I, J, S, U, A, G, M, R>, dim3(grid), dim3(T), smem, st, a);
}

template <int T, int I, int J, int S, int A>
constexpr size_t vjp_smem() {
    return (size_t)S * J * sizeof(VPart) + (A ? (size_t)(I / 2) * 8 * T * sizeof(float2) : 0) +
           (size_t)S * sizeof(uint64_t) + (size_t)(2 * S + 1) * sizeof(int);
}

#define NB_VJP_MR(T, I, J, S, U, A, M, R)                                                    \
    {{T, I, J, S, U, M, R, A, 63, kDefaultRefine, 0},                                        \
     {(const void *)vjp_kernel<T, I, J, S, U, A, false, M, R>,                              \
      (const void *)vjp_kernel<T, I, J, S, U, A, true, M, R>},                              \
     vjp_smem<T, I, J, S, A>(),                                                             \
     {launch_vjp<T, I, J, S, U, A, false, M, R>, launch_vjp<T, I, J, S, U, A, true, M, R>}}
#define NB_VJP_M(T, I, J, S, U, A, M) NB_VJP_MR(T, I, J, S, U, A, M, 0)
#define NB_VJP(T, I, J, S, U, A) NB_VJP_M(T, I, J, S, U, A, 1)
// One packed pair per thread at up to 128 registers: two 256-thread CTAs (or
// four of 128) per SM; the diagonal tiles' lane-diagonal form would
// otherwise take the with-gradient-on-p kernels to 130 and one CTA.
const VjpVariant kVjp[] = {
    NB_VJP_M(256, 2, 128, 3, 2, 0, 2), NB_VJP_M(256, 2, 128, 3, 4, 0, 2), NB_VJP(512, 2, 128, 3, 2, 0),
    NB_VJP_M(128, 2, 128, 3, 2, 0, 4), NB_VJP_M(256, 2, 256, 3, 2, 0, 2), NB_VJP(64, 4, 128, 3, 2, 0),
    NB_VJP(128, 4, 128, 3, 2, 0), NB_VJP(128, 4, 128, 3, 4, 0), NB_VJP_M(256, 2, 64, 4, 2, 0, 2),
    NB_VJP_M(256, 2, 32, 4, 2, 0, 2), NB_VJP(128, 4, 64, 4, 4, 0), NB_VJP(128, 4, 128, 4, 4, 0),
    NB_VJP(128, 4, 64, 4, 2, 0), NB_VJP_M(128, 4, 64, 4, 4, 0, 3), NB_VJP_M(128, 4, 128, 3, 4, 0, 3),
    NB_VJP_MR(128, 4, 64, 4, 4, 0, 1, 1), NB_VJP_MR(128, 4, 64, 4, 4, 0, 3, 1),
    NB_VJP_MR(128, 4, 128, 3, 4, 0, 3, 1), NB_VJP_MR(128, 4, 128, 4, 4, 0, 1, 1),
    NB_VJP(512, 2, 64, 4, 2, 0), NB_VJP(512, 2, 128, 3, 4, 0),
};
#undef NB_VJP
#undef NB_VJP_M
#undef NB_VJP_MR
constexpr int kVjpCount = (int)(sizeof(kVjp) / sizeof(kVjp[0]));
// Built-in shapes (GB300 sweep, G-pairs/s). With an upstream gradient on p:
// two packed pairs per thread in 128-thread CTAs with the barrier-free stage
// release; below 2^15, 128-particle j-tiles at three CTAs per SM (at most 168
// registers; N = 16384: 1010-1016, against 989-999 for 64-particle tiles at
// two CTAs per SM and 955-969 for one pair per thread in 256-thread CTAs);
// from 2^15, 128-particle tiles in 4 stages at two CTAs per SM (N = 65536:
// 1049 against 1042-1044 with a barrier per tile). Without it (26 operations,
// fewer registers): one pair per thread in 512-thread CTAs, with 64-particle
// tiles below 2^15 and 128-particle tiles from there (N = 16384: 1103, N =
// 65536: 1174-1176; the best two-pair shapes 1084-1086 and 1152-1153).
// Measured and not kept: the running sums in
// shared memory at four CTAs per SM (963-978 at 16384), an unroll of 8 (982),
// and u^2 from the special-function unit's reciprocal instead of u * u (one
// FP32 operation fewer, 1-3% slower).
constexpr int kVjpSmall = 17, kVjpLarge = 18, kVjpNoGpSmall = 19, kVjpNoGpLarge = 2;

const VjpVariant &vjp_variant(nb_ctx *ctx, int64_t n, bool with_gp) {
    const int k = ctx_ext(ctx).vjp_idx;
    if (k >= 0 && k < kVjpCount) return kVjp[k];
    const bool small = n < ((int64_t)1 << 15);
    if (!with_gp) return kVjp[small ? kVjpNoGpSmall : kVjpNoGpLarge];
    return kVjp[small ? kVjpSmall : kVjpLarge];
}

}  // namespace

extern "C" nb_status nb_force_vjp(nb_ctx *ctx, const float *x, const float *m, int64_t n, float eps,
                                  const float *ga, const float *gp, float *gx, float *gm,
                                  void *stream) {
    if (!ctx) return NB_ERR_ARG;
    nb_status st = check_common(ctx, n, eps, NB_PLAIN);
    if (st != NB_OK) return st;
    if (n == 0) return NB_OK;
    if (!x || !m || !ga || !gx || !gm) return fail(ctx, NB_ERR_ARG, "NULL array pointer");
    DeviceGuard g(ctx_device(ctx));
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const VjpVariant &vv = vjp_variant(ctx, n, gp != nullptr);
    const int with_gp = gp ? 1 : 0;
    PairVariant shape{};
    shape.tile = vv.tile;
    shape.comp = true;  // two float4 words per i
    shape.kernel = vv.kernel[with_gp];
    shape.smem = vv.smem;
    const PairPlan plan = make_plan(shape, n, resident_ctas(ctx, shape));

    ExtState &es = ctx_ext(ctx);
    cudaError_t e = ensure_buffer(&es.buf[V_VP], &es.cap[V_VP], (size_t)plan.npad * sizeof(VPart));
    if (e == cudaSuccess)
        e = ensure_buffer(&es.buf[V_PART], &es.cap[V_PART], plan.partial_bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation (vjp)");
    VPart *vp = static_cast<VPart *>(es.buf[V_VP]);
    // The three launches go out with programmatic dependent launch: each is
    // scheduled while its predecessor runs and waits for its results.
    e = launch_with_pdl(vjp_pack_kernel, dim3((unsigned)((plan.npad + 255) / 256)), dim3(256), 0, s, x, m, ga,
                        gp, n, plan.npad, vp);
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "vjp pack launch");

    VjpArgs A{};
    A.vp = vp;
    A.x = x;
    A.m = m;
    A.ga = ga;
    A.gp = gp;
    A.partial = static_cast<float4 *>(es.buf[V_PART]);
    A.err = ctx_err_word(ctx);
    A.n = n;
    A.njt = plan.njt;
    A.units = plan.units;
    A.grid = plan.grid;
    A.maxseg = plan.maxseg;
    A.eps2 = eps * eps;
    A.wait_ns = ctx_wait_ns(ctx);
    A.fault_unit = ctx_fault_unit(ctx);
    A.npad = plan.npad;
    A.partial_len = (int64_t)(es.cap[V_PART] / sizeof(float4));
    {
        TimedLaunch t(ctx, 5, s);
        vv.launch[with_gp](A, plan.grid, vv.smem, s);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "vjp kernel launch");
    e = launch_with_pdl(vjp_combine_kernel, dim3((unsigned)((n + 63) / 64)), dim3(64), 0, s, A, plan.ib, gx, gm);
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "vjp combine launch");
    return NB_OK;
}

extern "C" nb_status nb_set_vjp_tile(nb_ctx *ctx, const nb_tile *tile) {
    if (!ctx) return NB_ERR_ARG;
    if (!tile) {
        ctx_ext(ctx).vjp_idx = -1;
        return NB_OK;
    }
    for (int k = 0; k < kVjpCount; ++k)
        if (same_tile(kVjp[k].tile, *tile)) {
            ctx_ext(ctx).vjp_idx = k;
            return NB_OK;
        }
    return fail(ctx, NB_ERR_ARG, "tile shape is not one of the compiled VJP shapes");
}

extern "C" nb_status nb_get_vjp_tile(nb_ctx *ctx, int64_t n, nb_tile *out) {
    if (!ctx || !out) return NB_ERR_ARG;
    *out = vjp_variant(ctx, n, true).tile;
    return NB_OK;
}

extern "C" nb_status nb_list_vjp_tiles(nb_tile *out, int cap, int *count) {
    if (!count) return NB_ERR_ARG;
    *count = kVjpCount;
    if (out)
        for (int k = 0; k < kVjpCount && k < cap; ++k) out[k] = kVjp[k].tile;
    return NB_OK;
}
