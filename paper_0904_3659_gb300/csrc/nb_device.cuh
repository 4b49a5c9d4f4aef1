// nb_device.cuh -- device-side building blocks for the sm_103a kernels:
// mbarrier + bulk-copy (TMA) staging with bounded waits, the special-function
// unit's reciprocal square root, and packed FP32x2 arithmetic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nbdev {

// Error bits a kernel records in the context's device error word.
constexpr int kErrTimeout = 1;
constexpr int kErrBatchPlan = 2;  // batched offsets exceed the capacity sized from n_total
constexpr int kErrBounds = 4;     // a checked access was out of range (debug builds)

// Default limit for one bounded wait on a shared-memory barrier.
constexpr uint64_t kDefaultWaitNs = 1000000000ull;  // one second

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Makes barrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Address of the object at `p` (this CTA's shared memory) in the shared
// memory of CTA `rank` of the cluster, as a shared::cluster address.
__device__ __forceinline__ uint32_t cluster_map(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

// 16-byte store into another CTA's shared memory (shared::cluster address,
// 16-byte aligned) that signals its bytes to that CTA's mbarrier `rbar`
// (also a shared::cluster address, in the same CTA) as transaction bytes.
__device__ __forceinline__ void st_async_v4(uint32_t raddr, float4 v, uint32_t rbar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::
            "r"(raddr),
        "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar)
        : "memory");
}

// One-dimensional bulk copy global -> shared through the tensor memory
// accelerator; completion is signalled on `bar` as transaction bytes.
// Both addresses must be 16-byte aligned and `bytes` a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the phase with parity `parity` of *bar has completed. Gives up
// after limit_ns nanoseconds of wall time (and after 2^26 polls in any case)
// and returns false; the caller then records a timeout and leaves.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Bounds checks of the debug build (-DNB_DEBUG, libnbody_debug.so). NB_IN(err,
// site, cond) is true when the access it guards may go ahead; in a debug
// build a false cond records kErrBounds and the check site (bits 8..15) in
// the error word, and the caller skips the access. Release builds compile
// the check away.
#ifdef NB_DEBUG
__device__ __forceinline__ bool nb_in(int *err, int site, bool cond) {
    if (!cond) atomicOr(err, kErrBounds | (site << 8));
    return cond;
}
#define NB_IN(err, site, cond) ::nbdev::nb_in((err), (site), (cond))
#else
#define NB_IN(err, site, cond) true
#endif

// Reciprocal square root on the special-function unit (within 2^-22.9
// relative on sm_103a; the caller may refine it with a Newton-Raphson step).
__device__ __forceinline__ float rsqrt_sfu(float s) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(s));
    return y;
}

// Packed FP32x2 arithmetic (one instruction for two lanes, round to nearest).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// Programmatic dependent launch: kernels launched with programmatic stream
// serialization (launch_with_pdl) let the next launch on the stream be
// scheduled while they run; such a kernel waits for its predecessor's
// completion (and memory) before it reads anything, and releases its own
// dependents at once (they too wait for its completion before reading).
// Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait_then_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_with_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

}  // namespace nbdev
