// nb_tile.cuh -- the inner loop shared by the pair kernels: one j-tile in
// shared memory against a thread's register-resident i-particles, Eq. (gravity)
// of Fujiwara & Nakasato (arXiv:0904.3659, Section "Introduction").
#pragma once

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nbk {
using namespace nbdev;

// One pass of a j-tile against the thread's P pairs of i-particles, with y
// the special-function unit's estimate of s^{-1/2}.
// NEWTON: acc[q][0..2] += 4 m_j y1^3 (x_i - x_j), acc[q][3] += m_j y1, where
// y1 = y (3 - s y^2) / 2 is one Newton-Raphson step for f(y) = y^-2 - s.
// With t = s y^2 - 3 and u = y t we have y1 = -u/2, so m_j y1 = (-m_j/2) u
// (the packed mass is stored as -m_j/2) and 4 m_j y1^3 = (m_j y1) u^2:
// 16 FP32 operations per pair.
// Without the step: q = (-m_j/2) y, acc[q][3] += q, acc[q][0..2] += q y^2
// (x_i - x_j), i.e. the sums hold -p_i/2 and -a_i/2: 13 FP32 operations.
// In a diagonal tile (DIAG) the j == i term is removed by zeroing the mass
// lane of the thread's own particle; self0/self1 give, per pair, the tile
// position of the thread's own i (outside [0, JT) when it is not here).
// Operation groups of one interaction. Bit g of a MIX mask set: the group
// runs as packed FP32x2 instructions; clear: as two scalar FP32 instructions
// (same IEEE round-to-nearest operations, so every mask gives bit-identical
// results). Mixing trades issue slots (packed: one per two lanes) against
// the lower sustained pipe rate of packed instructions.
// POT = false leaves the potential out (acc[q][3] untouched): 12 FP32
// operations per pair, for callers that need only a_i (the integrator).
enum : int { kMixD = 1, kMixS = 2, kMixN = 4, kMixQ = 8, kMixW = 16, kMixA = 32, kMixAll = 63 };

template <bool PK>
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
    return PK ? add2(a, b) : make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}
template <bool PK>
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
    return PK ? mul2(a, b) : make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
template <bool PK>
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
    return PK ? fma2(a, b, c) : make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}

// DK >= 0 (with DIAG) is the lane-diagonal form of a 32-particle tile whose
// first particle is the thread's i-slot DK (pair DK / 2, half DK % 2) of lane
// 0, with i-slot k of lane l the particle 32 k + l of the i-block: then only
// slot DK of the thread meets itself, at jj == self0[0] (the lane), and the
// mask costs one compare and one select per j instead of two of each per
// pair.
template <int P, int JT, int UNR, bool DIAG, int MIX, bool NEWTON, bool POT = true, int DK = -1>
__device__ __forceinline__ void tile_pass(const JPart *__restrict__ T, const float2 (&xi)[P],
                                          const float2 (&yi)[P], const float2 (&zi)[P],
                                          float2 (&acc)[P][4], const float2 eps2,
                                          const int (&self0)[P], const int (&self1)[P]) {
    const float2 m3 = splat2(-3.f);
#pragma unroll UNR
    for (int jj = 0; jj < JT; ++jj) {
        const float4 A = reinterpret_cast<const float4 *>(T + jj)[0];
        const float4 B = reinterpret_cast<const float4 *>(T + jj)[1];
        const float2 nxj = make_float2(A.x, A.y);
        const float2 nyj = make_float2(A.z, A.w);
        const float2 nzj = make_float2(B.x, B.y);
        const float2 hmj = make_float2(B.z, B.w);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            constexpr bool PD = MIX & kMixD, PS = MIX & kMixS, PN = MIX & kMixN;
            constexpr bool PQ = MIX & kMixQ, PW = MIX & kMixW, PA = MIX & kMixA;
            const float2 dx = vadd<PD>(xi[q], nxj);
            const float2 dy = vadd<PD>(yi[q], nyj);
            const float2 dz = vadd<PD>(zi[q], nzj);
            float2 s = vfma<PS>(dx, dx, eps2);
            s = vfma<PS>(dy, dy, s);
            s = vfma<PS>(dz, dz, s);
            const float2 y = make_float2(rsqrt_sfu(s.x), rsqrt_sfu(s.y));
            float2 u = y;
            if (NEWTON) {
                const float2 y2 = vmul<PN>(y, y);
                const float2 t = vfma<PN>(s, y2, m3);
                u = vmul<PN>(y, t);
            }
            float2 hm = hmj;
            if constexpr (DIAG && DK >= 0) {
                static_assert(JT == 32 && DK < 2 * P, "the lane-diagonal form needs 32-particle tiles");
                if (q == DK / 2 && jj == self0[0]) {
                    if (DK % 2 == 0) hm.x = 0.f;
                    else hm.y = 0.f;
                }
            } else if constexpr (DIAG) {
                if (jj == self0[q]) hm.x = 0.f;
                if (jj == self1[q]) hm.y = 0.f;
            }
            const float2 qv = vmul<PQ>(hm, u);
            if (POT) acc[q][3] = vadd<PQ>(acc[q][3], qv);
            const float2 u2 = vmul<PW>(u, u);
            const float2 w = vmul<PW>(qv, u2);
            acc[q][0] = vfma<PA>(w, dx, acc[q][0]);
            acc[q][1] = vfma<PA>(w, dy, acc[q][1]);
            acc[q][2] = vfma<PA>(w, dz, acc[q][2]);
        }
    }
}

// A diagonal 32-particle tile of the single-launch kernels (i-blocks of
// 32 * 2P particles, slot k of lane l the block's particle 32 k + l, tiles
// starting at multiples of 32): the tile starts at the block's particle
// 32 k, so only slot k of each lane meets itself, at jj == lane. Dispatches
// to the lane-diagonal form for that slot (k is uniform across the warp).
template <int P, int UNR, bool NEWTON, int K = 0>
__device__ __forceinline__ void tile_pass_diag32(int k, int lane, const JPart *__restrict__ T,
                                                 const float2 (&xi)[P], const float2 (&yi)[P],
                                                 const float2 (&zi)[P], float2 (&acc)[P][4],
                                                 const float2 eps2) {
    if constexpr (K < 2 * P) {
        if (k == K) {
            int self0[P], self1[P];
#pragma unroll
            for (int q = 0; q < P; ++q) self0[q] = self1[q] = lane;
            tile_pass<P, 32, UNR, true, kMixAll, NEWTON, true, K>(T, xi, yi, zi, acc, eps2, self0, self1);
        } else {
            tile_pass_diag32<P, UNR, NEWTON, K + 1>(k, lane, T, xi, yi, zi, acc, eps2);
        }
    }
}

// The same pass for positions held as two FP32 words (HL records, see
// JPart): particle k occupies T[2k] = (-h, -h, ..., -m/2, -m/2) and
// T[2k+1] = (-l, -l, ...), with h on a power-of-two grid fine enough that
// h_i - h_j is exact in FP32 and l = x - h the FP32 remainder. Each
// component of x_i - x_j is then (h_i - h_j) + (l_i - l_j): one rounding of
// the exact difference (up to the remainders' own rounding, far below it),
// so close pairs keep their relative accuracy wherever they sit. 6 FP32
// operations per pair more than tile_pass (19, or 18 without the potential).
// DK >= 0: the lane-diagonal form, as for tile_pass.
template <int P, int JT, int UNR, bool DIAG, bool POT, int DK = -1>
__device__ __forceinline__ void tile_pass_hl(const JPart *__restrict__ T, const float2 (&xi)[P],
                                             const float2 (&yi)[P], const float2 (&zi)[P],
                                             const float2 (&lxi)[P], const float2 (&lyi)[P],
                                             const float2 (&lzi)[P], float2 (&acc)[P][4],
                                             const float2 eps2, const int (&self0)[P],
                                             const int (&self1)[P]) {
#pragma unroll UNR
    for (int jj = 0; jj < JT; ++jj) {
        const float4 A = reinterpret_cast<const float4 *>(T + 2 * jj)[0];
        const float4 B = reinterpret_cast<const float4 *>(T + 2 * jj)[1];
        const float4 C = reinterpret_cast<const float4 *>(T + 2 * jj + 1)[0];
        const float4 D = reinterpret_cast<const float4 *>(T + 2 * jj + 1)[1];
        const float2 nxj = make_float2(A.x, A.y), nyj = make_float2(A.z, A.w);
        const float2 nzj = make_float2(B.x, B.y), hmj = make_float2(B.z, B.w);
        const float2 nlxj = make_float2(C.x, C.y), nlyj = make_float2(C.z, C.w);
        const float2 nlzj = make_float2(D.x, D.y);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const float2 dx = add2(add2(xi[q], nxj), add2(lxi[q], nlxj));
            const float2 dy = add2(add2(yi[q], nyj), add2(lyi[q], nlyj));
            const float2 dz = add2(add2(zi[q], nzj), add2(lzi[q], nlzj));
            float2 s = fma2(dx, dx, eps2);
            s = fma2(dy, dy, s);
            s = fma2(dz, dz, s);
            const float2 u = make_float2(rsqrt_sfu(s.x), rsqrt_sfu(s.y));
            float2 hm = hmj;
            if constexpr (DIAG && DK >= 0) {
                static_assert(JT == 32 && DK < 2 * P, "the lane-diagonal form needs 32-particle tiles");
                if (q == DK / 2 && jj == self0[0]) {
                    if (DK % 2 == 0) hm.x = 0.f;
                    else hm.y = 0.f;
                }
            } else if constexpr (DIAG) {
                if (jj == self0[q]) hm.x = 0.f;
                if (jj == self1[q]) hm.y = 0.f;
            }
            const float2 qv = mul2(hm, u);
            if (POT) acc[q][3] = add2(acc[q][3], qv);
            const float2 w = mul2(qv, mul2(u, u));
            acc[q][0] = fma2(w, dx, acc[q][0]);
            acc[q][1] = fma2(w, dy, acc[q][1]);
            acc[q][2] = fma2(w, dz, acc[q][2]);
        }
    }
}

}  // namespace nbk
