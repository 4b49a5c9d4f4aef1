// nb_capi.cu -- the C ABI declared in include/nbody.h: contexts, argument
// checks, scratch management, tile selection and tuning, per-kernel timing.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "nb_device.cuh"
#include "nb_internal.h"
#include "nb_ext.h"

using namespace nbk;

namespace {

// Message of the last failed call that has no context (nb_create,
// nb_force_noalloc), per host thread.
thread_local std::string g_create_error;

enum KernelClass { K_PACK = 0, K_PAIR = 1, K_REDUCE = 2, K_LEAPFROG = 3, K_BATCHED = 4, K_VJP = 5,
                   K_COUNT = 8 };

struct PendingTiming {
    int kernel;
    cudaEvent_t start, stop;
};

}  // namespace

struct nb_ctx {
    int device = 0;
    int sm_count = 0;
    std::string msg;
    int *d_err = nullptr;

    // scratch, grow-only
    void *d_jp = nullptr;
    size_t jp_bytes = 0;
    void *d_partial = nullptr;
    size_t partial_bytes = 0;
    int *d_count = nullptr;  // fused shapes: arrivals per i-block, zero between launches
    int64_t count_cap = 0;
    // device staging for nb_force_host
    float *d_hx = nullptr, *d_hm = nullptr, *d_ha = nullptr, *d_hp = nullptr;
    int64_t host_cap = 0;

    // tiles
    bool has_override[2] = {false, false};
    int override_idx[2] = {0, 0};
    std::map<int, int> tuned[2];           // size class -> variant index
    std::map<const void *, int> occupancy;  // kernel -> resident CTAs per SM
    std::map<std::pair<const void *, int>, int> clusters;  // (kernel, size) -> co-resident clusters
    std::map<int64_t, int> cluster_pick[2];  // n -> built-in cluster shape chosen for n, per mode

    // timing
    bool timing = false;
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> spare_events;
    double total_ms[K_COUNT] = {0};
    int64_t launches[K_COUNT] = {0};

    // test hook
    int64_t fault_unit = -1;
    uint64_t wait_ns = nbdev::kDefaultWaitNs;

    // extension state (leap-frog, batched, vjp); see nb_ext.h
    nbx::ExtState ext;
};

namespace {

int size_class(int64_t n) {
    int c = 0;
    while (((int64_t)1 << (c + 1)) <= n) ++c;
    return c;
}

cudaEvent_t take_event(nb_ctx *ctx) {
    if (!ctx->spare_events.empty()) {
        cudaEvent_t e = ctx->spare_events.back();
        ctx->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

nbx::TimedLaunch::TimedLaunch(nb_ctx *ctx, int kernel, cudaStream_t st)
    : ctx_(ctx), kernel_(kernel), st_(st) {
    if (!ctx_->timing) return;
    start_ = take_event(ctx_);
    stop_ = take_event(ctx_);
    if (start_) cudaEventRecord(start_, st_);
}

nbx::TimedLaunch::~TimedLaunch() {
    if (!ctx_->timing || !start_ || !stop_) return;
    cudaEventRecord(stop_, st_);
    ctx_->pending.push_back({kernel_, start_, stop_});
}

namespace nbx {

void set_global_error(const std::string &m) { g_create_error = m; }

nb_status fail(nb_ctx *ctx, nb_status st, const std::string &m) {
    if (ctx) ctx->msg = m;
    return st;
}

nb_status cuda_fail(nb_ctx *ctx, cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a non-sticky launch error where possible
    return fail(ctx, e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

int ctx_device(const nb_ctx *ctx) { return ctx->device; }
int ctx_sm_count(const nb_ctx *ctx) { return ctx->sm_count; }
int *ctx_err_word(nb_ctx *ctx) { return ctx->d_err; }
ExtState &ctx_ext(nb_ctx *ctx) { return ctx->ext; }
bool ctx_set_timing(nb_ctx *ctx, bool on) {
    const bool prev = ctx->timing;
    ctx->timing = on;
    return prev;
}
uint64_t ctx_wait_ns(const nb_ctx *ctx) { return ctx->wait_ns; }
int64_t ctx_fault_unit(const nb_ctx *ctx) { return ctx->fault_unit; }

static_assert(ExtState::kSlots == SLOT_COUNT, "one buffer per slot id");

cudaError_t ensure_buffer(void **ptr, size_t *cap, size_t bytes) {
    if (bytes <= *cap && *ptr) return cudaSuccess;
    if (*ptr) {
        cudaError_t e = cudaFree(*ptr);
        *ptr = nullptr;
        *cap = 0;
        if (e != cudaSuccess) return e;
    }
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(ptr, want);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return e;
    }
    *cap = want;
    return cudaSuccess;
}

// Arrival counters of the fused shapes: zeroed when allocated; every launch
// leaves them zero again (the last CTA of each i-block resets its count).
cudaError_t ensure_counters(nb_ctx *ctx, int64_t nib) {
    if (nib <= ctx->count_cap && ctx->d_count) return cudaSuccess;
    if (ctx->d_count) {
        cudaError_t e = cudaFree(ctx->d_count);
        ctx->d_count = nullptr;
        ctx->count_cap = 0;
        if (e != cudaSuccess) return e;
    }
    const int64_t want = std::max<int64_t>(nib, 1024);
    cudaError_t e = cudaMalloc(&ctx->d_count, (size_t)want * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_count, 0, (size_t)want * sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(ctx->d_count);
        ctx->d_count = nullptr;
        return e;
    }
    ctx->count_cap = want;
    return cudaSuccess;
}

int resident_ctas(nb_ctx *ctx, const PairVariant &v) {
    auto it = ctx->occupancy.find(v.kernel);
    if (it != ctx->occupancy.end()) return it->second * ctx->sm_count;
    if (v.smem > 48 * 1024)
        cudaFuncSetAttribute(v.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.kernel, v.tile.threads, v.smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    cudaGetLastError();
    ctx->occupancy[v.kernel] = per_sm;
    return per_sm * ctx->sm_count;
}

// Clusters of `size` CTAs of v's kernel that the GPU holds at once (the
// cluster form needs all of its clusters resident in one wave to pay off).
int max_active_clusters(nb_ctx *ctx, const PairVariant &v, int size) {
    const auto key = std::make_pair(v.kernel, size);
    auto it = ctx->clusters.find(key);
    if (it != ctx->clusters.end()) return it->second;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(size * ctx->sm_count));
    cfg.blockDim = dim3((unsigned)v.tile.threads);
    cfg.dynamicSmemBytes = v.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, v.kernel, &cfg) != cudaSuccess) num = 0;
    cudaGetLastError();
    ctx->clusters[key] = num;
    return num;
}

// How the cluster form of v would run at n: the pair evaluations on the
// busiest SM, and whether its clusters all fit on the GPU at once (else it
// runs as its chunked twin with the same split; a shape without one is not
// a candidate then).
struct ClusterLoad {
    int64_t load;
    bool fits;
};
ClusterLoad cluster_load(nb_ctx *ctx, const PairVariant &v, int64_t n) {
    const PairPlan p = make_plan(v, n, resident_ctas(ctx, v));
    const bool fits = max_active_clusters(ctx, v, (int)p.nchunks) >= p.nib;
    if (!fits && !chunked_twin(v)) return {INT64_MAX, false};
    const int64_t ctas_per_sm = (p.grid + ctx->sm_count - 1) / ctx->sm_count;
    const int64_t tiles_per_cta = (p.njt + p.nchunks - 1) / p.nchunks;
    return {ctas_per_sm * p.ib * tiles_per_cta * v.tile.jtile, fits};
}

// The built-in shape for n. Where it is a cluster form, the same shape at
// the other residency (minblocks: 1 or 2 CTAs per SM) replaces it when that
// gives the busiest SM less work, or as much work with clusters that fit
// where the built-in one's do not. At N = 7168 two CTAs per SM take clusters
// of 5 where one CTA per SM allows only 2 (29.8 against 32.2 us per call);
// at N = 1024 clusters of 8 CTAs fit only at two per SM (5.7 against 7.5 us).
int default_index(nb_ctx *ctx, int64_t n, bool comp) {
    const int k = pair_default_index(comp, n);
    const PairVariant &v = *pair_variant(comp, k);
    if (v.tile.fused != 3) return k;
    auto &cache = ctx->cluster_pick[comp ? 1 : 0];
    auto it = cache.find(n);
    if (it != cache.end()) return it->second;
    int best = k;
    ClusterLoad best_load = cluster_load(ctx, v, n);
    for (int j = 0; j < pair_variant_count(comp); ++j) {
        const PairVariant &w = *pair_variant(comp, j);
        nb_tile t = w.tile;
        t.minblocks = v.tile.minblocks;
        if (j == k || w.tile.fused != 3 || !same_tile(t, v.tile)) continue;
        const ClusterLoad l = cluster_load(ctx, w, n);
        if (l.load < best_load.load ||
            (l.load == best_load.load && l.fits && !best_load.fits)) {
            best = j;
            best_load = l;
        }
    }
    cache[n] = best;
    return best;
}

const PairVariant &choose_variant(nb_ctx *ctx, int64_t n, bool comp) {
    const int m = comp ? 1 : 0;
    if (ctx->has_override[m]) return *pair_variant(comp, ctx->override_idx[m]);
    auto it = ctx->tuned[m].find(size_class(n));
    if (it != ctx->tuned[m].end()) return *pair_variant(comp, it->second);
    return *pair_variant(comp, default_index(ctx, n, comp));
}

// Enqueue pack -> pair -> combine for one system of n particles already
// packed or to be packed from FP32 x, m. `jp` may be supplied by the caller
// (already packed); else x, m are packed into the context's buffer.
nb_status run_force(nb_ctx *ctx, const float *x, const float *m, const JPart *prepacked,
                    int64_t n, float eps, float *a, float *p, bool comp, cudaStream_t st) {
    const PairVariant *vp = &choose_variant(ctx, n, comp);
    // Packed input (FP64 state packed by the caller), or no potential wanted
    // (p NULL): a shape that reads packed particles.
    if ((prepacked || !p) && vp->tile.fused) vp = pair_variant(comp, pair_default_unfused_index(comp, n));
    // No potential wanted: the same shape without the potential term, if compiled.
    if (!p)
        if (const PairVariant *tw = no_pot_twin(*vp)) vp = tw;
    // The cluster form when its clusters do not all fit at once: the chunked
    // form of the same shape and split (partials through global memory).
    // Smaller clusters that fit would mean longer chunks: at N = 6144 the
    // 4-wide shape's clusters of 3 do not all fit, and clusters of 2 ran
    // 28.2 us against 21.0 for the chunked form.
    if (vp->tile.fused == 3) {
        const PairPlan cp = make_plan(*vp, n, resident_ctas(ctx, *vp));
        if (max_active_clusters(ctx, *vp, (int)cp.nchunks) < cp.nib)
            if (const PairVariant *tw = chunked_twin(*vp)) vp = tw;
    }
    const PairVariant &v = *vp;
    const PairPlan plan = make_plan(v, n, resident_ctas(ctx, v));
    cudaError_t e;
    if (v.tile.fused) {
        e = ensure_buffer(&ctx->d_partial, &ctx->partial_bytes, plan.partial_bytes);
        if (e == cudaSuccess) e = ensure_counters(ctx, plan.nib);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation (partial sums)");
        FusedArgs fa{};
        fa.x = x;
        fa.m = m;
        fa.n = n;
        fa.a = a;
        fa.p = p;
        fa.partial = static_cast<float4 *>(ctx->d_partial);
        fa.partial_len = (int64_t)(ctx->partial_bytes / sizeof(float4));
        fa.counters = ctx->d_count;
        fa.err = ctx->d_err;
        fa.nib = plan.nib;
        fa.njt = plan.njt;
        fa.nchunks = plan.nchunks;
        fa.grid = plan.grid;
        fa.units = plan.units;
        fa.maxseg = plan.maxseg;
        fa.eps2 = eps * eps;
        fa.a_scale = accel_scale(v.tile.refine);
        fa.p_scale = pot_scale(v.tile.refine);
        fa.wait_ns = ctx->wait_ns;
        fa.fault_cta = ctx->fault_unit;
        {
            TimedLaunch t(ctx, K_PAIR, st);
            e = v.launch_fused(fa, plan.grid, plan.smem, st);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "fused pair kernel launch");
        return NB_OK;
    }
    const JPart *jp = prepacked;
    if (!jp) {
        e = ensure_buffer(&ctx->d_jp, &ctx->jp_bytes, (size_t)plan.npad * sizeof(JPart));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation (packed particles)");
        {
            TimedLaunch t(ctx, K_PACK, st);
            e = launch_pack_f32(x, m, n, plan.npad, static_cast<JPart *>(ctx->d_jp), st);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "pack kernel launch");
        jp = static_cast<const JPart *>(ctx->d_jp);
    }
    e = ensure_buffer(&ctx->d_partial, &ctx->partial_bytes, plan.partial_bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation (partial sums)");

    PairArgs pa{};
    pa.jp = jp;
    pa.partial = static_cast<float4 *>(ctx->d_partial);
    pa.err = ctx->d_err;
    pa.njt = plan.njt;
    pa.units = plan.units;
    pa.grid = plan.grid;
    pa.maxseg = plan.maxseg;
    pa.eps2 = eps * eps;
    pa.fault_unit = ctx->fault_unit;
    pa.wait_ns = ctx->wait_ns;
    pa.npad = plan.npad;
    pa.partial_len = (int64_t)(ctx->partial_bytes / sizeof(float4));
    {
        TimedLaunch t(ctx, K_PAIR, st);
        e = v.launch(pa, plan.grid, v.smem, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pair kernel launch");

    ReduceArgs ra{};
    ra.partial = pa.partial;
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
    ra.err = ctx->d_err;
    {
        TimedLaunch t(ctx, K_REDUCE, st);
        e = launch_reduce(ra, v.comp, st);  // the combine matches the kernel's running sums
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "combine kernel launch");
    return NB_OK;
}

nb_status reserve_hl(nb_ctx *ctx, int64_t n) {
    size_t bytes = 0;
    for (bool no_pot : {false, true}) {
        const PairVariant &v = *hl_variant(n, no_pot);
        bytes = std::max(bytes, make_plan(v, n, resident_ctas(ctx, v)).partial_bytes);
    }
    cudaError_t e = ensure_buffer(&ctx->d_partial, &ctx->partial_bytes, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation (partial sums)");
    return NB_OK;
}

nb_status run_force_hl(nb_ctx *ctx, const JPart *jp, int64_t n, float eps, float *a, float *p,
                       cudaStream_t st) {
    const PairVariant &v = *hl_variant(n, p == nullptr);
    const PairPlan plan = make_plan(v, n, resident_ctas(ctx, v));
    nb_status rs = reserve_hl(ctx, n);
    if (rs != NB_OK) return rs;
    PairArgs pa{};
    pa.jp = jp;
    pa.partial = static_cast<float4 *>(ctx->d_partial);
    pa.err = ctx->d_err;
    pa.njt = plan.njt;
    pa.units = plan.units;
    pa.grid = plan.grid;
    pa.maxseg = plan.maxseg;
    pa.eps2 = eps * eps;
    pa.fault_unit = ctx->fault_unit;
    pa.wait_ns = ctx->wait_ns;
    pa.npad = plan.npad;
    pa.partial_len = (int64_t)(ctx->partial_bytes / sizeof(float4));
    cudaError_t e;
    {
        TimedLaunch t(ctx, K_PAIR, st);
        e = v.launch(pa, plan.grid, v.smem, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pair kernel launch (HL)");
    ReduceArgs ra{};
    ra.partial = pa.partial;
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
    ra.err = ctx->d_err;
    {
        TimedLaunch t(ctx, K_REDUCE, st);
        e = launch_reduce(ra, true, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "combine kernel launch (HL)");
    return NB_OK;
}

nb_status check_common(nb_ctx *ctx, int64_t n, float eps, int mode) {
    if (n < 0) return fail(ctx, NB_ERR_ARG, "n must be >= 0");
    if (!std::isfinite(eps) || !(eps > 0.f)) return fail(ctx, NB_ERR_ARG, "eps must be finite and > 0");
    const float e2 = eps * eps;  // the kernels work with eps^2 in FP32
    if (!(e2 >= FLT_MIN && e2 <= FLT_MAX))
        return fail(ctx, NB_ERR_ARG, "eps^2 must be a finite normal FP32 number (about 1.1e-19 <= eps <= 1.8e19)");
    if (mode != NB_PLAIN && mode != NB_COMPENSATED) return fail(ctx, NB_ERR_ARG, "unknown mode");
    return NB_OK;
}

}  // namespace nbx

using namespace nbx;

extern "C" {

const char *nb_status_string(nb_status s) {
    switch (s) {
        case NB_OK: return "NB_OK";
        case NB_ERR_ARG: return "NB_ERR_ARG";
        case NB_ERR_CUDA: return "NB_ERR_CUDA";
        case NB_ERR_OOM: return "NB_ERR_OOM";
        case NB_ERR_TIMEOUT: return "NB_ERR_TIMEOUT";
        case NB_ERR_NOT_IMPLEMENTED: return "NB_ERR_NOT_IMPLEMENTED";
    }
    return "NB_UNKNOWN";
}

nb_status nb_create(nb_ctx **out, int device) {
    if (!out) {
        g_create_error = "out is NULL";
        return NB_ERR_ARG;
    }
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) {
        g_create_error = std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    if (device < 0 || device >= count) {
        g_create_error = "device index out of range";
        return NB_ERR_ARG;
    }
    nb_ctx *ctx = new nb_ctx();
    ctx->device = device;
    DeviceGuard g(device);
    e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        g_create_error = std::string("context set-up: ") + cudaGetErrorString(e);
        cudaFree(ctx->d_err);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;
    }
    *out = ctx;
    return NB_OK;
}

void nb_destroy(nb_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto &pt : ctx->pending) {
        cudaEventDestroy(pt.start);
        cudaEventDestroy(pt.stop);
    }
    for (auto ev : ctx->spare_events) cudaEventDestroy(ev);
    nbx::ext_release(ctx->ext);
    cudaFree(ctx->d_jp);
    cudaFree(ctx->d_partial);
    cudaFree(ctx->d_count);
    cudaFree(ctx->d_hx);
    cudaFree(ctx->d_hm);
    cudaFree(ctx->d_ha);
    cudaFree(ctx->d_hp);
    cudaFree(ctx->d_err);
    delete ctx;
}

const char *nb_last_error(const nb_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->msg.c_str();
}

nb_status nb_force(nb_ctx *ctx, const float *x, const float *m, int64_t n, float eps, float *a,
                   float *p, nb_mode mode, void *stream) {
    if (!ctx) return NB_ERR_ARG;
    nb_status st = check_common(ctx, n, eps, mode);
    if (st != NB_OK) return st;
    if (n == 0) return NB_OK;
    if (!x || !m || !a || !p) return fail(ctx, NB_ERR_ARG, "NULL array pointer");
    DeviceGuard g(ctx->device);
    return run_force(ctx, x, m, nullptr, n, eps, a, p, mode == NB_COMPENSATED,
                     static_cast<cudaStream_t>(stream));
}

nb_status nb_reserve(nb_ctx *ctx, int64_t n, nb_mode mode) {
    if (!ctx) return NB_ERR_ARG;
    if (n < 0) return fail(ctx, NB_ERR_ARG, "n must be >= 0");
    if (mode != NB_PLAIN && mode != NB_COMPENSATED) return fail(ctx, NB_ERR_ARG, "unknown mode");
    if (n == 0) return NB_OK;
    DeviceGuard g(ctx->device);
    const bool comp = mode == NB_COMPENSATED;
    size_t jp = 0, part = 0;
    int64_t nib = 0;
    // Every shape this context might pick for n (and the shapes' twins
    // without the potential): reserve for the largest.
    for (int k = 0; k < pair_variant_count(comp); ++k) {
        const PairVariant *cands[2] = {pair_variant(comp, k), no_pot_twin(*pair_variant(comp, k))};
        for (const PairVariant *vp : cands) {
            if (!vp) continue;
            const PairPlan plan = make_plan(*vp, n, resident_ctas(ctx, *vp));
            jp = std::max(jp, (size_t)plan.npad * sizeof(JPart));
            part = std::max(part, plan.partial_bytes);
            if (vp->tile.fused) nib = std::max(nib, plan.nib);
        }
    }
    cudaError_t e = ensure_buffer(&ctx->d_jp, &ctx->jp_bytes, jp);
    if (e == cudaSuccess) e = ensure_buffer(&ctx->d_partial, &ctx->partial_bytes, part);
    if (e == cudaSuccess && nib > 0) e = ensure_counters(ctx, nib);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "nb_reserve");
    return NB_OK;
}

nb_status nb_force_host(nb_ctx *ctx, const float *x, const float *m, int64_t n, float eps, float *a,
                        float *p, nb_mode mode, void *stream) {
    if (!ctx) return NB_ERR_ARG;
    nb_status st = check_common(ctx, n, eps, mode);
    if (st != NB_OK) return st;
    if (n == 0) return NB_OK;
    if (!x || !m || !a || !p) return fail(ctx, NB_ERR_ARG, "NULL array pointer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (n > ctx->host_cap) {
        cudaStreamSynchronize(s);
        cudaFree(ctx->d_hx);
        cudaFree(ctx->d_hm);
        cudaFree(ctx->d_ha);
        cudaFree(ctx->d_hp);
        ctx->d_hx = ctx->d_hm = ctx->d_ha = ctx->d_hp = nullptr;
        ctx->host_cap = 0;
        e = cudaMalloc(&ctx->d_hx, 3 * n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_hm, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_ha, 3 * n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_hp, n * sizeof(float));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "device staging allocation");
        ctx->host_cap = n;
    }
    e = cudaMemcpyAsync(ctx->d_hx, x, 3 * n * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d_hm, m, n * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "host to device copy");
    st = run_force(ctx, ctx->d_hx, ctx->d_hm, nullptr, n, eps, ctx->d_ha, ctx->d_hp,
                   mode == NB_COMPENSATED, s);
    if (st != NB_OK) return st;
    e = cudaMemcpyAsync(a, ctx->d_ha, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p, ctx->d_hp, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device to host copy");
    return nb_synchronize(ctx, stream);
}

nb_status nb_synchronize(nb_ctx *ctx, void *stream) {
    if (!ctx) return NB_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    int word = 0;
    e = cudaMemcpy(&word, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word read");
    if (word) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        if (word & nbdev::kErrTimeout)
            return fail(ctx, NB_ERR_TIMEOUT,
                        "a bounded wait for a shared-memory tile ran out; results are invalid");
        if (word & nbdev::kErrBounds)
            return fail(ctx, NB_ERR_CUDA,
                        "debug bounds check failed at site " + std::to_string((word >> 8) & 0xff) +
                            "; the access was skipped and results are invalid");
        if (word & nbdev::kErrBatchPlan)
            return fail(ctx, NB_ERR_ARG,
                        "batched offsets or eps are invalid (offsets must start at 0, never "
                        "decrease and end at n_total; each non-empty cluster's eps must be > 0 "
                        "with eps^2 a finite normal FP32 number); nothing was computed");
        return fail(ctx, NB_ERR_CUDA, "device error word set");
    }
    return NB_OK;
}

nb_status nb_get_tile(nb_ctx *ctx, int64_t n, nb_mode mode, nb_tile *out) {
    if (!ctx || !out) return NB_ERR_ARG;
    if (mode != NB_PLAIN && mode != NB_COMPENSATED) return fail(ctx, NB_ERR_ARG, "unknown mode");
    *out = choose_variant(ctx, std::max<int64_t>(n, 1), mode == NB_COMPENSATED).tile;
    return NB_OK;
}

nb_status nb_set_tile(nb_ctx *ctx, nb_mode mode, const nb_tile *tile) {
    if (!ctx) return NB_ERR_ARG;
    if (mode != NB_PLAIN && mode != NB_COMPENSATED) return fail(ctx, NB_ERR_ARG, "unknown mode");
    const int mi = mode == NB_COMPENSATED ? 1 : 0;
    if (!tile) {
        ctx->has_override[mi] = false;
        return NB_OK;
    }
    const bool comp = mode == NB_COMPENSATED;
    for (int k = 0; k < pair_variant_count(comp); ++k) {
        if (same_tile(pair_variant(comp, k)->tile, *tile)) {
            ctx->has_override[mi] = true;
            ctx->override_idx[mi] = k;
            return NB_OK;
        }
    }
    return fail(ctx, NB_ERR_ARG, "tile shape is not one of the compiled shapes");
}

nb_status nb_set_tuned_tile(nb_ctx *ctx, int64_t n, nb_mode mode, const nb_tile *tile) {
    if (!ctx) return NB_ERR_ARG;
    if (n <= 0) return fail(ctx, NB_ERR_ARG, "n must be > 0");
    if (mode != NB_PLAIN && mode != NB_COMPENSATED) return fail(ctx, NB_ERR_ARG, "unknown mode");
    const bool comp = mode == NB_COMPENSATED;
    const int mi = comp ? 1 : 0;
    if (!tile) {
        ctx->tuned[mi].erase(size_class(n));
        return NB_OK;
    }
    for (int k = 0; k < pair_variant_count(comp); ++k)
        if (same_tile(pair_variant(comp, k)->tile, *tile)) {
            ctx->tuned[mi][size_class(n)] = k;
            return NB_OK;
        }
    return fail(ctx, NB_ERR_ARG, "tile shape is not one of the compiled shapes");
}

nb_status nb_list_tiles(nb_mode mode, nb_tile *out, int cap, int *count) {
    if (!count) return NB_ERR_ARG;
    if (mode != NB_PLAIN && mode != NB_COMPENSATED) return NB_ERR_ARG;
    const bool comp = mode == NB_COMPENSATED;
    const int nv = pair_variant_count(comp);
    *count = nv;
    if (out)
        for (int k = 0; k < nv && k < cap; ++k) out[k] = pair_variant(comp, k)->tile;
    return NB_OK;
}

nb_status nb_autotune(nb_ctx *ctx, int64_t n, nb_mode mode, void *stream, nb_tile *best,
                      double *rate) {
    if (!ctx) return NB_ERR_ARG;
    if (n <= 0) return fail(ctx, NB_ERR_ARG, "n must be > 0");
    if (mode != NB_PLAIN && mode != NB_COMPENSATED) return fail(ctx, NB_ERR_ARG, "unknown mode");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool comp = mode == NB_COMPENSATED;
    const int mi = comp ? 1 : 0;
    float *x = nullptr, *m = nullptr, *a = nullptr, *p = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&x, 3 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&a, 3 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&p, n * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch_fill_uniform(x, m, n, 0x5eedull, s);
    const bool saved_override = ctx->has_override[mi];
    const int saved_idx = ctx->override_idx[mi];
    const bool saved_timing = ctx->timing;
    ctx->timing = false;
    nb_status st = NB_OK;
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "autotune set-up");
    // One timed whole call of shape k (after the shape's warm-up call).
    auto time_one = [&](int k, float *ms) -> nb_status {
        ctx->has_override[mi] = true;
        ctx->override_idx[mi] = k;
        cudaEventRecord(e0, s);
        nb_status rs = run_force(ctx, x, m, nullptr, n, 1.0f / 64.f, a, p, comp, s);
        cudaEventRecord(e1, s);
        if (rs != NB_OK) return rs;
        cudaError_t te = cudaEventSynchronize(e1);
        if (te != cudaSuccess) return cuda_fail(ctx, te, "autotune timing");
        cudaEventElapsedTime(ms, e0, e1);
        return NB_OK;
    };
    // Pass 1: every shape, warm-up + best of 2. Pass 2: the three fastest
    // again, 5 times each, interleaved so that a clock change affects them
    // alike; each keeps its best time over both passes.
    const int nv = pair_variant_count(comp);
    std::vector<float> best_ms_of(nv, 0.f);
    std::vector<int> order;  // the shapes timed
    for (int k = 0; st == NB_OK && k < nv; ++k) {
        // Single-launch shapes: small n only.
        if (pair_variant(comp, k)->tile.fused && !fused_candidate(n)) continue;
        order.push_back(k);
        ctx->has_override[mi] = true;
        ctx->override_idx[mi] = k;
        st = run_force(ctx, x, m, nullptr, n, 1.0f / 64.f, a, p, comp, s);  // warm-up
        for (int rep = 0; st == NB_OK && rep < 2; ++rep) {
            float ms = 0.f;
            st = time_one(k, &ms);
            if (st == NB_OK && (rep == 0 || ms < best_ms_of[k])) best_ms_of[k] = ms;
        }
    }
    std::sort(order.begin(), order.end(), [&](int u, int v) { return best_ms_of[u] < best_ms_of[v]; });
    const int finalists = std::min((int)order.size(), 3);
    for (int rep = 0; st == NB_OK && rep < 5; ++rep)
        for (int f = 0; st == NB_OK && f < finalists; ++f) {
            float ms = 0.f;
            st = time_one(order[f], &ms);
            if (st == NB_OK && ms < best_ms_of[order[f]]) best_ms_of[order[f]] = ms;
        }
    int best_idx = -1;
    float best_ms = 0.f;
    for (int f = 0; st == NB_OK && f < finalists; ++f)
        if (best_idx < 0 || best_ms_of[order[f]] < best_ms) {
            best_idx = order[f];
            best_ms = best_ms_of[order[f]];
        }
    ctx->has_override[mi] = saved_override;
    ctx->override_idx[mi] = saved_idx;
    ctx->timing = saved_timing;
    if (st == NB_OK) st = nb_synchronize(ctx, stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(m);
    cudaFree(a);
    cudaFree(p);
    if (st != NB_OK) return st;
    ctx->tuned[mi][size_class(n)] = best_idx;
    if (best) *best = pair_variant(comp, best_idx)->tile;
    if (rate) *rate = (double)n * (double)n / (best_ms * 1e-3);
    return NB_OK;
}

nb_status nb_timing_enable(nb_ctx *ctx, int on) {
    if (!ctx) return NB_ERR_ARG;
    ctx->timing = on != 0;
    return NB_OK;
}

nb_status nb_timing_read(nb_ctx *ctx, int kernel, double *total_ms, int64_t *launches) {
    if (!ctx) return NB_ERR_ARG;
    if (kernel < 0 || kernel >= K_COUNT) return fail(ctx, NB_ERR_ARG, "unknown kernel class");
    DeviceGuard g(ctx->device);
    for (auto &pt : ctx->pending) {
        cudaError_t e = cudaEventSynchronize(pt.stop);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "timing event");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, pt.start, pt.stop);
        ctx->total_ms[pt.kernel] += ms;
        ctx->launches[pt.kernel] += 1;
        ctx->spare_events.push_back(pt.start);
        ctx->spare_events.push_back(pt.stop);
    }
    ctx->pending.clear();
    if (total_ms) *total_ms = ctx->total_ms[kernel];
    if (launches) *launches = ctx->launches[kernel];
    return NB_OK;
}

nb_status nb_timing_reset(nb_ctx *ctx) {
    if (!ctx) return NB_ERR_ARG;
    double dummy;
    nb_status st = nb_timing_read(ctx, 0, &dummy, nullptr);  // drain pending events
    if (st != NB_OK) return st;
    for (int k = 0; k < K_COUNT; ++k) {
        ctx->total_ms[k] = 0;
        ctx->launches[k] = 0;
    }
    return NB_OK;
}

nb_status nb_debug_set_fault(nb_ctx *ctx, int64_t unit, int64_t wait_ns) {
    if (!ctx) return NB_ERR_ARG;
    ctx->fault_unit = unit < 0 ? -1 : unit;
    ctx->wait_ns = wait_ns > 0 ? (uint64_t)wait_ns : nbdev::kDefaultWaitNs;
    return NB_OK;
}

}  // extern "C"
