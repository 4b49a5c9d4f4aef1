// nb_combine.cuh -- walking the CTAs that contributed partial sums to one
// i-block, for the deterministic cross-CTA combines (pair, fused and VJP
// kernels). CTA c of a persistent launch owns the work units
// [u0(c), u0(c+1)) with u0(c) = floor(c units / grid), and unit u belongs to
// i-block u / njt; its partials of i-block b sit in segment b - bf(c),
// bf(c) = u0(c) / njt.
#pragma once

#include <cstdint>

namespace nbk {

// The CTA that owns unit u.
__device__ __forceinline__ int64_t cta_of_unit(int64_t u, int64_t units, int grid) {
    return ((u + 1) * (int64_t)grid - 1) / units;
}

// u0(c) and bf(c) for c = clo, clo + 1, ..., stepped without 64-bit
// divisions after the first CTA: u0 grows by units / grid, plus one when the
// remainder (c units) mod grid carries, and bf follows u0.
struct SegWalk {
    int64_t q, r, u0, rem, bf, njt;
    int64_t grid;
    __device__ __forceinline__ SegWalk(int64_t clo, int64_t units, int grid_, int64_t njt_)
        : q(units / grid_), r(units % grid_), u0(clo * units / grid_), rem(0), bf(0), njt(njt_),
          grid(grid_) {
        rem = clo * units - u0 * grid;
        bf = u0 / njt;
    }
    __device__ __forceinline__ void next() {
        u0 += q;
        rem += r;
        if (rem >= grid) {
            rem -= grid;
            ++u0;
        }
        while ((bf + 1) * njt <= u0) ++bf;
    }
};

}  // namespace nbk
