// nb_ext.h -- services of the context (nb_capi.cu) used by the translation
// units that implement the other entry points (leap-frog, batched, VJP).
#pragma once

#include <cstdint>
#include <string>

#include "nb_internal.h"

namespace nbx {

// Grow-only device buffers owned by the context for the other entry points,
// one per slot id (every translation unit takes its ids from this list).
enum ExtSlot : int {
    SLOT_FP64_JP = 0,   // packed particles from FP64 state (leap-frog, energy)
    SLOT_ENERGY_A,      // accelerations computed by nb_energy
    SLOT_P,             // potentials computed by nb_energy
    SLOT_ENERGY_BLK,    // energy block sums
    SLOT_ENERGY_OUT,    // energy result
    SLOT_BATCH_JP,      // padded packed clusters
    SLOT_BATCH_POFF,    // padded cluster offsets
    SLOT_BATCH_ITEMS,   // batched work items
    SLOT_BATCH_COUNT,   // item count and queue head
    SLOT_BATCH_PART,    // per-item partial sums
    SLOT_BATCH_IBASE,   // first item of each cluster
    SLOT_VJP_VP,        // packed VJP records
    SLOT_VJP_PART,      // VJP partial sums
    SLOT_HL_BOX,        // bounding-box partials of FP64 positions (HL packing)
    SLOT_ADJOINT,       // leap-frog adjoint: replayed state, position history, VJP operands
    SLOT_BATCH_FRAME,   // per-cluster HL frames (centre, grid) of the batched leap-frog
    SLOT_BATCH_PLANNED, // the offsets and eps the current batched plan was made for
    SLOT_COUNT
};

struct ExtState {
    static constexpr int kSlots = SLOT_COUNT;
    void *buf[kSlots] = {};
    size_t cap[kSlots] = {};
    int vjp_idx = -1;  // VJP shape forced by nb_set_vjp_tile (-1: built-in)
    // (n_clusters, n_total) of the batched plan in the scratch (-1: none).
    int64_t plan_clusters = -1, plan_total = -1;
};
void ext_release(ExtState &s);

// Brackets one kernel launch with CUDA events on its stream when the
// context's timing is on (nb_timing_enable).
class TimedLaunch {
  public:
    TimedLaunch(nb_ctx *ctx, int kernel, cudaStream_t st);
    ~TimedLaunch();
    TimedLaunch(const TimedLaunch &) = delete;
    TimedLaunch &operator=(const TimedLaunch &) = delete;

  private:
    nb_ctx *ctx_;
    int kernel_;
    cudaStream_t st_;
    cudaEvent_t start_ = nullptr, stop_ = nullptr;
};

nb_status fail(nb_ctx *ctx, nb_status st, const std::string &m);
// Message returned by nb_last_error(NULL) (calls without a context).
void set_global_error(const std::string &m);
nb_status cuda_fail(nb_ctx *ctx, cudaError_t e, const char *what);
nb_status check_common(nb_ctx *ctx, int64_t n, float eps, int mode);

int ctx_device(const nb_ctx *ctx);
int ctx_sm_count(const nb_ctx *ctx);
int *ctx_err_word(nb_ctx *ctx);
uint64_t ctx_wait_ns(const nb_ctx *ctx);
int64_t ctx_fault_unit(const nb_ctx *ctx);
ExtState &ctx_ext(nb_ctx *ctx);
// Turn per-kernel event timing on or off; returns the previous setting.
bool ctx_set_timing(nb_ctx *ctx, bool on);

cudaError_t ensure_buffer(void **ptr, size_t *cap, size_t bytes);
int resident_ctas(nb_ctx *ctx, const nbk::PairVariant &v);
const nbk::PairVariant &choose_variant(nb_ctx *ctx, int64_t n, bool comp);

// Compensated path on FP64 state: pair kernel on HL records (two JParts per
// particle, nbk::kHLRecords), then the compensated combine; p may be NULL
// (the potential is then not summed).
nb_status run_force_hl(nb_ctx *ctx, const nbk::JPart *jp, int64_t n, float eps, float *a, float *p,
                       cudaStream_t st);
// Allocate the HL path's partial sums for n (before any graph capture).
nb_status reserve_hl(nb_ctx *ctx, int64_t n);

// pack (unless prepacked) -> pair -> combine, enqueued on st.
nb_status run_force(nb_ctx *ctx, const float *x, const float *m, const nbk::JPart *prepacked,
                    int64_t n, float eps, float *a, float *p, bool comp, cudaStream_t st);

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace nbx
