// nb_internal.h -- host-side interface between the C ABI (nb_capi.cu) and the
// kernel translation units. Not installed; not part of the public ABI.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nbody.h"

namespace nbk {

// One particle as staged in shared memory for the pair kernel: 32 bytes,
// every value duplicated so that one 64-bit register pair feeds both lanes
// of a packed FP32x2 instruction. Positions are stored negated and the mass
// as -m/2 (both exact): d = x_i + (-x_j); the Newton step folds its factor
// -1/2 into the mass, and without the step the sums carry -1/2, which the
// combine removes (see tile_pass).
struct alignas(32) JPart {
    float2 nx, ny, nz, hm;
};
static_assert(sizeof(JPart) == 32, "JPart must be 32 bytes");

// Positions held in FP64 (the integrator's state) enter the compensated
// kernels as two FP32 words per coordinate (HL records, two JParts per
// particle): relative to a reference point c of the system (or cluster),
// y = x - c is split into h = y rounded to the grid G = 2^(E-23), where
// 2^E bounds every |y|, and l = fl32(y - h). Every h is a multiple of G
// below 2^23 G in magnitude, so h_i - h_j is exact in FP32, and the pair
// kernel forms x_i - x_j as (h_i - h_j) + (l_i - l_j) with a single
// rounding that matters. Record 2k: (-h, -h, ..., -m/2, -m/2); record
// 2k+1: (-l_x, -l_x, -l_y, -l_y, -l_z, -l_z, 0, 0).
constexpr int kHLRecords = 2;

// The grid exponent E for a system whose positions relative to its
// reference point are bounded by `extent` (>= 0): the smallest E with
// |y| <= 2^E (at least -100, so that G stays a normal FP32 number).
__host__ __device__ inline int hl_grid_exponent(double extent) {
    int e = -100;
    if (extent > 0.0) {
        int ex = 0;
        const double f = frexp(extent, &ex);  // extent = f 2^ex, f in [0.5, 1)
        e = f == 0.5 ? ex - 1 : ex;
        if (e < -100) e = -100;
    }
    return e;
}

// Particle arrays are padded to a multiple of this (>= every i-block and
// j-tile size) with inert entries (m = 0 at the origin).
constexpr int64_t kPad = 3072;

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Arguments of the persistent pair kernel (one launch evaluates Eq. (gravity)
// for all i of one system). Work unit u = (i-block u / njt, j-tile u % njt);
// CTA c owns the contiguous units [c*units/grid, (c+1)*units/grid).
struct PairArgs {
    const JPart *jp;       // [npad] packed particles (source of both i and j)
    float4 *partial;       // [grid][maxseg][words][ib] per-segment partial sums
    int *err;              // device error word (bit kErrTimeout)
    int64_t njt;           // j-tiles covering n
    int64_t units;         // nib * njt
    int grid;              // CTAs launched
    int maxseg;            // max i-blocks one CTA touches
    float eps2;            // eps^2 in FP32
    int64_t fault_unit;    // test hook: unit whose copy is never issued (-1: none)
    uint64_t wait_ns;      // limit of one bounded barrier wait
    int64_t npad;          // particles in jp (bounds checks of the debug build)
    int64_t partial_len;   // float4 entries of partial (debug build)
};

// Arguments of the fused single-launch kernel (small n): it reads x, m
// itself and the last CTA to finish an i-block writes its a, p.
struct FusedArgs {
    const float *x;        // [n][3]
    const float *m;        // [n]
    int64_t n;
    float *a;              // [n][3]
    float *p;              // [n]
    float4 *partial;       // per-CTA partial sums: [nib][nchunks][words][ib] (chunked
                           //   form), [grid][maxseg][words][ib] (stream-K form)
    int64_t partial_len;   // float4 entries of partial (debug build)
    int *counters;         // [nib] arrivals per i-block; zero between launches
    int *err;              // device error word (timeouts of the cluster form; debug build)
    int64_t nib;
    int64_t njt;           // j-tiles covering n
    int64_t nchunks;       // chunked form: j-chunks (CTAs) per i-block
    int grid;              // CTAs launched (chunked form: nib * nchunks)
    float eps2;
    float a_scale, p_scale;
    int64_t units;         // stream-K form: (i-block, j-tile) units, nib * njt
    int64_t maxseg;        // stream-K form: most i-blocks one CTA's range touches
    uint64_t wait_ns;      // cluster form: limit of the wait for the other chunks' partials
    int64_t fault_cta;     // cluster form test hook: CTA whose partials are never sent (-1: none)
};

// Arguments of the deterministic cross-CTA combine.
struct ReduceArgs {
    const float4 *partial;
    float *a;              // [n][3]
    float *p;              // [n], or nullptr: the potential is not written
    int64_t n;
    int64_t njt;
    int64_t units;
    int grid;
    int maxseg;
    int ib;
    float a_scale;         // sums -> a_i and p_i: accel_scale / pot_scale of
    float p_scale;         //   the pair variant's refine setting
    int64_t partial_len;   // float4 entries of partial (debug build)
    int *err;              // device error word (debug build)
};

inline bool same_tile(const nb_tile &a, const nb_tile &b) {
    return a.threads == b.threads && a.ipt == b.ipt && a.jtile == b.jtile && a.stages == b.stages &&
           a.unroll == b.unroll && a.minblocks == b.minblocks && a.release == b.release &&
           a.sums_in_smem == b.sums_in_smem && a.packed == b.packed && a.refine == b.refine &&
           a.fused == b.fused;
}

// Factors that turn the pair kernels' sums into a_i and p_i (exact powers of
// two). With the Newton step the sums hold 4 a_i and p_i; without it they
// hold -a_i/2 and -p_i/2, because the packed mass is -m/2 (see tile_pass).
__host__ __device__ constexpr float accel_scale(int refine) { return refine ? 0.25f : -2.0f; }
__host__ __device__ constexpr float pot_scale(int refine) { return refine ? 1.0f : -2.0f; }

// Newton steps of the built-in default shapes and of the fixed-shape kernels
// (batched, HL, allocation-free): none, since on sm_103a the step does
// not improve the FP32 result (see nb_tile.refine).
constexpr int kDefaultRefine = 0;

// A compiled pair-kernel shape.
struct PairVariant {
    nb_tile tile;
    bool comp;                 // Kahan-compensated accumulation
    const void *kernel;        // for occupancy queries
    size_t smem;               // dynamic shared memory bytes
    cudaError_t (*launch)(const PairArgs &, int grid, size_t smem, cudaStream_t);
    cudaError_t (*launch_fused)(const FusedArgs &, int grid, size_t smem, cudaStream_t);
};

// Registry of compiled variants (nb_pair.cu).
// HL variants: compensated kernels on HL records (positions from FP64 state,
// see kHLRecords); no_pot selects the twin that sums a_i only.
const PairVariant *hl_variant(int64_t n, bool no_pot = false);
// The twin of a plain packed shape that sums a_i only (12 FP32 operations
// per pair), or nullptr if that shape has none.
const PairVariant *no_pot_twin(const PairVariant &v);
// The chunked form (fused = 1) of a single-launch shape, or nullptr.
const PairVariant *chunked_twin(const PairVariant &v);
int pair_variant_count(bool comp);
const PairVariant *pair_variant(bool comp, int idx);
int pair_default_index(bool comp, int64_t n);
// The built-in shape for n among those that read packed particles (not
// fused), for callers that pack themselves (leap-frog from FP64 state).
int pair_default_unfused_index(bool comp, int64_t n);
// Whether the tuner times the fused (single-launch, small-n) shapes at n.
bool fused_candidate(int64_t n);

// Launchers (nb_pair.cu).
cudaError_t launch_pack_f32(const float *x, const float *m, int64_t n, int64_t npad, JPart *jp,
                            cudaStream_t st);
cudaError_t launch_reduce(const ReduceArgs &r, bool comp, cudaStream_t st);
cudaError_t launch_fill_uniform(float *x, float *m, int64_t n, uint64_t seed, cudaStream_t st);

// Work decomposition of one nb_force call for a given variant.
struct PairPlan {
    int64_t n, npad, nib, njt, units, nchunks;
    int grid, maxseg, ib, words;
    size_t partial_bytes;
    size_t smem;  // dynamic shared memory of the launch
    int64_t partial_len() const { return (int64_t)(partial_bytes / sizeof(float4)); }
};
PairPlan make_plan(const PairVariant &v, int64_t n, int resident_ctas);

}  // namespace nbk
