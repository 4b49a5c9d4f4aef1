// nb_noalloc.cu -- nb_force_noalloc: Eq. (gravity) without any device
// allocation, for callers that are not allowed to allocate GPU memory.
//
// Who needs this: code that must not call cudaMalloc at the point where it
// wants forces. Examples are a host application whose memory manager owns
// the whole device (every byte is already reserved by a pool or a framework
// allocator, so a raw cudaMalloc would fail or fragment it), a loop with a
// latency budget that cannot absorb the device-wide synchronisation
// cudaMalloc/cudaFree can cause, and plug-in code that is only handed
// input/output buffers and is not trusted with allocation at all. The normal
// entry points need a context whose scratch is allocated on demand; this one
// takes its scratch from a fixed array that is part of the library image.
//
// The scratch lives in a file-scope __device__ array of kScratchBytes
// (16 MiB). Every GPU on which the library is loaded holds that array until
// the process exits, whether or not this entry point is ever called.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <string>

#include "nb_device.cuh"
#include "nb_ext.h"
#include "nb_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int64_t kMaxN = 65536;
constexpr int kMaxDevices = 64;

// Packed particles, then the per-segment partial sums (256-byte aligned).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
// Device error word of this entry point (bounded-wait timeouts).
static __device__ int g_noalloc_err;

// Per-device set-up, done on the first call on each device. In host code the
// names g_scratch / g_noalloc_err denote host-side shadows, not device
// addresses, so the device addresses are looked up with
// cudaGetSymbolAddress while that device is current. They are kept for the
// life of the process: a cudaDeviceReset (which unloads the library's device
// image) leaves them stale, so this entry point is not used after one.
struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;
    int *err = nullptr;
    int resident = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

nb_status noalloc_fail(nb_status st, const std::string &m) {
    nbx::set_global_error("nb_force_noalloc: " + m);
    return st;
}

}  // namespace

extern "C" nb_status nb_force_noalloc(const float *x, const float *m, int64_t n, float eps, float *a,
                                      float *p, void *stream) {
    using namespace nbk;
    if (n < 0) return noalloc_fail(NB_ERR_ARG, "n must be >= 0");
    if (!std::isfinite(eps) || !(eps > 0.f))
        return noalloc_fail(NB_ERR_ARG, "eps must be finite and > 0");
    if (!(eps * eps >= FLT_MIN && eps * eps <= FLT_MAX))
        return noalloc_fail(NB_ERR_ARG, "eps^2 must be a finite normal FP32 number");
    if (n == 0) return NB_OK;
    if (!x || !m || !a || !p) return noalloc_fail(NB_ERR_ARG, "NULL array pointer");
    if (n > kMaxN)
        return noalloc_fail(NB_ERR_ARG, "n = " + std::to_string(n) + " exceeds this entry point's " +
                                            "limit of " + std::to_string(kMaxN) +
                                            " particles (its scratch is a fixed 16 MiB array)");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(NB_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(NB_ERR_ARG, "device index out of range");

    // Every array must live on the current device, where the scratch array
    // and the kernels are taken from (a pointer of another device would be
    // read through peer access, or fault).
    const void *arrays[4] = {x, m, a, p};
    const char *names[4] = {"x", "m", "a", "p"};
    for (int k = 0; k < 4; ++k) {
        cudaPointerAttributes at{};
        e = cudaPointerGetAttributes(&at, arrays[k]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return noalloc_fail(NB_ERR_ARG, std::string(names[k]) + " is not a CUDA pointer");
        }
        const bool ok = at.type == cudaMemoryTypeManaged ||
                        (at.type == cudaMemoryTypeDevice && at.device == dev);
        if (!ok)
            return noalloc_fail(NB_ERR_ARG, std::string(names[k]) +
                                                " is not device memory of the current device " +
                                                std::to_string(dev));
    }

    const PairVariant &v = *pair_variant(false, 0);
    DeviceSetup ds;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        DeviceSetup &s = g_setup[dev];
        if (!s.ready) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(NB_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                                     cudaGetErrorString(e));
            s.scratch = static_cast<unsigned char *>(ptr);
            e = cudaGetSymbolAddress(&ptr, g_noalloc_err);
            if (e != cudaSuccess)
                return noalloc_fail(NB_ERR_CUDA, std::string("cudaGetSymbolAddress(error word): ") +
                                                     cudaGetErrorString(e));
            s.err = static_cast<int *>(ptr);
            int sms = 0, per_sm = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.kernel, v.tile.threads,
                                                                  v.smem);
            if (e != cudaSuccess) return noalloc_fail(NB_ERR_CUDA, cudaGetErrorString(e));
            s.resident = std::max(1, per_sm) * sms;
            s.ready = true;
        }
        ds = s;
    }

    const PairPlan plan = make_plan(v, n, ds.resident);
    const size_t jp_bytes = round_up((int64_t)plan.npad * sizeof(JPart), 256);
    if (jp_bytes + plan.partial_bytes > kScratchBytes)
        return noalloc_fail(NB_ERR_ARG, "the work split for n = " + std::to_string(n) +
                                            " on this device needs more than the 16 MiB scratch array");

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    JPart *jp = reinterpret_cast<JPart *>(ds.scratch);
    float4 *partial = reinterpret_cast<float4 *>(ds.scratch + jp_bytes);

    // The array keeps the previous call's contents: the packed particles and
    // every partial the combine reads are rewritten below; the error word is
    // the one value that must start at zero.
    e = cudaMemsetAsync(ds.err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_pack_f32(x, m, n, plan.npad, jp, st);
    if (e != cudaSuccess) return noalloc_fail(NB_ERR_CUDA, cudaGetErrorString(e));

    PairArgs pa{};
    pa.jp = jp;
    pa.partial = partial;
    pa.err = ds.err;
    pa.njt = plan.njt;
    pa.units = plan.units;
    pa.grid = plan.grid;
    pa.maxseg = plan.maxseg;
    pa.eps2 = eps * eps;
    pa.fault_unit = -1;
    pa.wait_ns = nbdev::kDefaultWaitNs;
    pa.npad = plan.npad;
    pa.partial_len = (int64_t)(plan.partial_bytes / sizeof(float4));
    e = v.launch(pa, plan.grid, v.smem, st);
    if (e != cudaSuccess) return noalloc_fail(NB_ERR_CUDA, cudaGetErrorString(e));

    ReduceArgs ra{};
    ra.partial = partial;
    ra.a = a;
    ra.p = p;
    ra.n = n;
    ra.njt = plan.njt;
    ra.units = plan.units;
    ra.grid = plan.grid;
    ra.maxseg = plan.maxseg;
    ra.ib = plan.ib;
    ra.a_scale = accel_scale(v.tile.refine);
    ra.p_scale = pot_scale(v.tile.refine);
    ra.partial_len = pa.partial_len;
    ra.err = ds.err;
    e = launch_reduce(ra, false, st);
    if (e != cudaSuccess) return noalloc_fail(NB_ERR_CUDA, cudaGetErrorString(e));

    // The error word is read on the caller's stream, so the call waits for
    // that stream alone (not for other streams of the device).
    int word = 0;
    e = cudaMemcpyAsync(&word, ds.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(NB_ERR_CUDA, cudaGetErrorString(e));
    if (word & nbdev::kErrTimeout)
        return noalloc_fail(NB_ERR_TIMEOUT, "a bounded wait for a shared-memory tile ran out");
    return NB_OK;
}
