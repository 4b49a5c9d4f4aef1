/*
 * nbody.h -- C ABI of the GB300 (sm_103a) direct-summation gravity library.
 *
 * The library computes the exact softened gravitational acceleration and
 * potential of N particles, Eq. (gravity) of Fujiwara & Nakasato, "Fast
 * Simulations of Gravitational Many-body Problem on RV770 GPU"
 * (arXiv:0904.3659), Section "Introduction":
 *
 *     a_i = sum_{j != i} m_j (x_i - x_j) / (|x_i - x_j|^2 + eps^2)^{3/2}
 *     p_i = sum_{j != i} m_j / (|x_i - x_j|^2 + eps^2)^{1/2}
 *
 * and, around it, the leap-frog integrator of Section "Method", Eqs. (1)-(3).
 * Each compute entry point names the passage that defines its operation;
 * the context, tuning, timing and error entry points are engineering support
 * with no counterpart in the paper.
 *
 * Conventions shared by every entry point:
 *  - Sign: a and p are returned exactly as printed in Eq. (gravity): a_i
 *    points away from the other masses and p_i > 0 (G = 1). The physical
 *    gravitational acceleration is -a_i and the potential energy is
 *    W = -1/2 sum_i m_i p_i. nb_leapfrog_step applies that physical sign.
 *  - The j == i term is left out by index; distinct particles at the same
 *    position are summed (0 to a, m_j/eps to p).
 *  - Layout: positions and accelerations are row-major [n][3] arrays
 *    (x0,y0,z0,x1,...), masses and potentials are [n]. Unless an entry point
 *    says otherwise, every array argument is a DEVICE pointer on the device
 *    the context was created for. The caller owns every data buffer; the
 *    context owns only scratch memory, events and the tuning table.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream). Calls enqueue work on it and return without waiting,
 *    except where stated. Device-side errors (a bounded wait that ran out)
 *    are reported by the next nb_synchronize on that context.
 *  - Errors: every call returns an nb_status. NB_OK on success; on failure
 *    nothing is enqueued, output buffers are untouched, and nb_last_error()
 *    gives a one-line message. n == 0 is a valid no-op. A negative count, a
 *    NULL pointer where data is needed, or eps not finite or not > 0
 *    (the paper's eps exists to prevent division by zero) is NB_ERR_ARG, and
 *    so is an eps whose square is not a normal FP32 number (below about
 *    1.1e-19 it would flush to zero, above about 1.8e19 overflow); batched
 *    calls check each cluster's eps on the device (see nb_force_batched).
 *    Non-finite positions or masses are not checked; they propagate.
 *  - Contexts are not thread-safe: use one per host thread. A context's
 *    scratch (packed particles, partial sums, the fused shapes' per-i-block
 *    arrival counts) is shared by all its calls, so calls on one context must
 *    execute in order on the GPU (one stream, or streams ordered by events);
 *    work that must overlap on the GPU needs one context per stream.
 *  - Graph capture: once nb_reserve has sized the scratch for the (n, mode)
 *    used, nb_force allocates nothing and can be captured into a CUDA graph.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nb_status {
    NB_OK = 0,
    NB_ERR_ARG = 1,              /* invalid argument; nothing was done */
    NB_ERR_CUDA = 2,             /* a CUDA runtime call or launch failed */
    NB_ERR_OOM = 3,              /* scratch allocation failed */
    NB_ERR_TIMEOUT = 4,          /* a bounded device wait ran out (results invalid) */
    NB_ERR_NOT_IMPLEMENTED = 5   /* entry point present but not built */
} nb_status;

/*
 * Arithmetic variants of the pair kernel. Both keep every pair interaction in
 * FP32 (x_i - x_j, s, rsqrt on the special-function unit, optionally refined
 * by one Newton-Raphson step -- see nb_tile.refine -- and products) and add
 * results in FP32.
 *  NB_PLAIN        two-level blocked sum: a register partial per j-tile, then
 *                  a running sum across tiles. Target: max per-particle
 *                  relative error <= 1e-5 against FP64.
 *  NB_COMPENSATED  the tile partials enter the running sum through Kahan
 *                  compensation, the cross-block combine is compensated too,
 *                  and positions held in FP64 (leap-frog state) enter the
 *                  pair arithmetic relative to the centre of their bounding
 *                  box as an exact FP32 grid part plus an FP32 remainder, so
 *                  that x_i - x_j carries one rounding. Target: <= 1e-6.
 */
typedef enum nb_mode { NB_PLAIN = 0, NB_COMPENSATED = 1 } nb_mode;

typedef struct nb_ctx nb_ctx;

/* Tile shape and schedule of the pair kernel: `threads` per CTA, `ipt`
 * i-particles per thread held in registers (even: they are processed in
 * packed FP32 pairs), `jtile` j-particles per shared-memory stage, `stages`
 * stages in flight, `unroll` unroll factor of the j loop, `minblocks` the
 * resident CTAs per SM the register allocation is held to, and `release`
 * how a consumed stage is refilled (0: CTA barrier per tile; 1: the last
 * warp to finish the tile issues the next copy, no barrier), `sums_in_smem`
 * whether the running sums between tiles live in shared memory (1) or in
 * registers (0), and `packed` a bit mask of the interaction's operation
 * groups that run as packed FP32x2 instructions (1 difference, 2 distance,
 * 4 Newton step, 8 potential term, 16 force weight, 32 force accumulation;
 * the others run as scalar FP32; every mask gives bit-identical results),
 * and `refine` the Newton-Raphson steps applied to the special-function
 * unit's reciprocal square root (0 or 1). With refine = 0 a pair costs 13
 * FP32 operations instead of 16 (mask bit 4 then has no effect). On sm_103a
 * the unrefined estimate is within 2^-22.9 relative of 1/sqrt(s) (measured
 * over every FP32 value in [1, 4), i.e. every mantissa and both exponent
 * parities; the PTX ISA gives the same bound for the whole range), and one
 * Newton step evaluated in FP32 does not lower that bound (its own three
 * roundings are of the same size), so both settings meet the same error
 * targets. A tile passed with fewer fields (zero-filled) means refine = 0.
 * `fused` = 1 marks a single-launch shape for small n: each CTA of `threads`
 * threads takes one i-block of 32 * `ipt` particles (every warp holds the
 * same i) and one j-chunk, which its threads load from x and m into shared
 * memory themselves (no pack kernel, no TMA; `stages` = 1); warp w sums the
 * `jtile`-particle tiles w, w + warps, ... and the warps' sums are added in
 * warp order. The last CTA of an i-block to finish adds the chunks' partial
 * sums in chunk order and writes its a, p (no combine kernel). `fused` = 2
 * is the same kernel with the pair kernel's work split: the (i-block,
 * `jtile`-particle tile) units are divided into equal contiguous ranges,
 * one per resident CTA, so a CTA may finish one i-block and start the next;
 * the last contributing CTA adds the partials in CTA order. `fused` = 3 is
 * the chunked split with the chunks of an i-block launched as one
 * thread-block cluster (at most 8 chunks): each CTA sends its partial of
 * every nch-th particle into the shared memory of the cluster's CTA that owns
 * it, which adds them in chunk order once they have arrived (no partials in
 * global memory, no arrival counts); here `minblocks` is the CTAs per SM (1:
 * the CTA takes a full SM's shared memory, so exactly one runs per SM; 2:
 * registers held to 128 per thread); when the GPU cannot hold all of its
 * clusters at once, the call runs the chunked form of the same shape. All
 * single-launch shapes are launched with programmatic stream serialization:
 * the next kernel on the stream may be scheduled while the previous one runs,
 * and each waits for its predecessor's results before reading. Callers that
 * pass packed FP64 state (the leap-frog) use the non-fused shape of the same
 * size class instead. */
typedef struct nb_tile {
    int threads;
    int ipt;
    int jtile;
    int stages;
    int unroll;
    int minblocks;
    int release;
    int sums_in_smem;
    int packed;
    int refine;
    int fused;
} nb_tile;

/* Create a context on CUDA device `device`. *out receives the handle. */
nb_status nb_create(nb_ctx **out, int device);

/* Free the context's scratch, events and streams. NULL is ignored. Waits
 * for the device work the context enqueued to finish. */
void nb_destroy(nb_ctx *ctx);

/* Message describing the last failure on this context ("" if none). The
 * pointer stays valid until the next call on the context. NULL ctx gives the
 * message of the last failed call without a context on this host thread
 * (nb_create, nb_force_noalloc). */
const char *nb_last_error(const nb_ctx *ctx);

/* Static name of a status code. */
const char *nb_status_string(nb_status s);

/*
 * Eq. (gravity) for all n particles.
 *   x    [n][3] FP32 device, positions
 *   m    [n]    FP32 device, masses
 *   eps  softening (> 0, finite)
 *   a    [n][3] FP32 device, output accelerations (literal sign)
 *   p    [n]    FP32 device, output potentials (positive)
 * x/m must not overlap a/p. Asynchronous on `stream`. The first call at a
 * larger n than before (or in a new mode) allocates scratch (cudaMalloc,
 * which synchronises the device); nb_reserve does that ahead of time.
 * Results are bit-for-bit reproducible for a fixed (n, mode, tile, device).
 */
nb_status nb_force(nb_ctx *ctx, const float *x, const float *m, int64_t n, float eps,
                   float *a, float *p, nb_mode mode, void *stream);

/*
 * Eq. (gravity) on HOST buffers: copies x and m to the device, runs nb_force,
 * copies a and p back and waits for the copies to finish. Same argument
 * meaning as nb_force, but all four arrays are host memory (pinned memory
 * gives the fastest copies). Device staging buffers are owned by ctx.
 */
nb_status nb_force_host(nb_ctx *ctx, const float *x, const float *m, int64_t n, float eps,
                        float *a, float *p, nb_mode mode, void *stream);

/* Allocate the scratch nb_force needs for up to n particles in `mode`, so
 * that later calls up to that size allocate nothing. */
nb_status nb_reserve(nb_ctx *ctx, int64_t n, nb_mode mode);

/*
 * Many independent systems in one launch (Eq. (gravity) within each cluster,
 * no interaction between clusters).
 *   x, m, a, p    as in nb_force, clusters concatenated
 *   offsets       [n_clusters + 1] int64 DEVICE array; cluster c is the rows
 *                 offsets[c] .. offsets[c+1]-1; offsets[0] == 0, nondecreasing
 *   eps           [n_clusters] FP32 DEVICE array of per-cluster softening
 *   n_total       offsets[n_clusters] (the total particle count)
 * Asynchronous. Offsets and eps are not read back to the host: offsets that
 * do not start at 0, decrease, or do not end at n_total, and a non-empty
 * cluster whose eps is not > 0 with eps^2 a finite normal FP32 number, are
 * detected on the device; then nothing is read or written and the next
 * nb_synchronize returns NB_ERR_ARG. Work items are (cluster, block of 128 i-particles,
 * chunk of at most a quarter of its j-range), taken from a device queue by
 * the warps of one persistent launch, largest clusters first; each item is
 * summed by one warp in a fixed order and the chunks are added in chunk
 * order (bit-reproducible). The item list is kept in the context and reused
 * by the next call (batched force or batched leap-frog) while n_clusters,
 * n_total and the values of offsets and eps stay the same, which the device
 * checks on every call; any change makes a new list.
 */
nb_status nb_force_batched(nb_ctx *ctx, const float *x, const float *m, const int64_t *offsets,
                           int64_t n_clusters, int64_t n_total, const float *eps,
                           float *a, float *p, nb_mode mode, void *stream);

/*
 * nb_leapfrog_step (Eqs. (1)-(3) of Section "Method") for a batch of
 * independent clusters, each with its own Eq. (gravity) (as nb_force_batched):
 * x, v FP64 device [n_total][3] in/out; m, eps, offsets as in
 * nb_force_batched; a [n_total][3] FP32 device, in (if a_valid) / out;
 * p [n_total] FP32 device, out. One persistent pair launch per step; steps
 * after the first are replayed from a CUDA graph when `stream` is not the
 * legacy default stream. In NB_COMPENSATED mode the FP64 positions enter
 * the pair kernel, at every force evaluation, relative to the centre of
 * their cluster's bounding box, each coordinate as an exact FP32 grid part
 * (a multiple of a power of two fine enough that the difference of two grid
 * parts is exact in FP32) plus an FP32 remainder, so x_i - x_j carries one
 * rounding wherever the cluster sits. Asynchronous.
 */
nb_status nb_leapfrog_batched_step(nb_ctx *ctx, double *x, double *v, const float *m,
                                   const int64_t *offsets, int64_t n_clusters, int64_t n_total,
                                   const float *eps, float *a, float *p, double dt, int nsteps,
                                   int a_valid, nb_mode mode, void *stream);

/*
 * nsteps kick-drift-kick leap-frog steps, Eqs. (1)-(3) of Section "Method",
 * with FP64 state on the device:
 *   v += 1/2 g dt;  x += v dt;  g = -a(x) (Eq. (gravity), FP32 pair kernel);
 *   v += 1/2 g dt
 *   x    [n][3] FP64 device, in/out positions
 *   v    [n][3] FP64 device, in/out velocities
 *   m    [n]    FP32 device masses
 *   a    [n][3] FP32 device: on entry Eq. (gravity) at the entry positions
 *                (literal sign) if a_valid != 0, else it is computed first;
 *                on exit Eq. (gravity) at the exit positions
 *   p    [n]    FP32 device, out: potentials at the exit positions, or NULL:
 *                the integrator needs only a, so the force kernels then leave
 *                the potential out (12 instead of 13 FP32 operations per pair)
 * Asynchronous. In NB_COMPENSATED mode the FP64 positions enter the pair
 * kernel relative to the centre of their bounding box (recomputed at every
 * force evaluation), each coordinate as an exact FP32 grid part plus an FP32
 * remainder, so x_i - x_j carries one rounding.
 */
nb_status nb_leapfrog_step(nb_ctx *ctx, double *x, double *v, const float *m, float *a, float *p,
                           int64_t n, float eps, double dt, int nsteps, int a_valid,
                           nb_mode mode, void *stream);

/*
 * Reverse-mode gradient through nsteps leap-frog steps of nb_leapfrog_step
 * (Eqs. (1)-(3) of Section "Method" with Eq. (gravity)), for one segment of a
 * checkpointed trajectory. The segment is replayed from its entry state with
 * the same kernels nb_leapfrog_step uses (so with the same positions), the
 * positions of every step are kept, and the steps are then swept in reverse:
 * per step, the adjoints of the two kicks and the drift (FP64 kernels) and
 * one nb_force_vjp of the force at the step's end.
 *   x, v  [n][3] FP64 device, in: the state at the segment's start
 *   a     [n][3] FP32 device, in: Eq. (gravity) at x as the forward pass had
 *                it (the a passed to nb_leapfrog_step with a_valid != 0), or
 *                NULL if the forward computed it (a_valid == 0)
 *   m     [n]    FP32 device masses
 *   lx, lv [n][3] FP64 device, in/out: on entry dL/dx, dL/dv at the segment's
 *                end; on exit at its start
 *   la    [n][3] FP64 device, in/out: on entry dL/da for the force at the
 *                segment's end (zero at the trajectory's end); on exit the
 *                same for the force at its start
 *   lm    [n]    FP64 device, in/out: dL/dm is added to it
 *   apply_first  nonzero for the trajectory's first segment: the force at x
 *                is itself a function of x and m, so its adjoint la is
 *                folded into lx and lm by one more VJP and la is cleared
 * mode, eps, dt, nsteps as passed to nb_leapfrog_step for the segment. The
 * caller keeps (x, v, a) of each segment start from the forward pass.
 * Scratch grows with (nsteps + 1) n 24 bytes (the positions kept).
 * Asynchronous on `stream`; the caller's x, v, a are not modified.
 */
nb_status nb_leapfrog_adjoint(nb_ctx *ctx, const double *x, const double *v, const float *a,
                              const float *m, int64_t n, float eps, double dt, int nsteps,
                              double *lx, double *lv, double *la, double *lm, int apply_first,
                              nb_mode mode, void *stream);

/*
 * Total energy of an FP64 state, the conservation check of a leap-frog run
 * (the paper computes no energy): out_kw[0] = K = 1/2 sum m |v|^2 and
 * out_kw[1] = W = -1/2 sum m_i p_i with p from Eq. (gravity), accumulated in
 * FP64 in a fixed order.
 * x, v FP64 device [n][3]; m FP32 device [n]; out_kw HOST double[2].
 * Synchronous (waits for `stream`).
 */
nb_status nb_energy(nb_ctx *ctx, const double *x, const double *v, const float *m, int64_t n,
                    float eps, double *out_kw, nb_mode mode, void *stream);

/*
 * Vector-Jacobian product of Eq. (gravity): for upstream gradients ga [n][3]
 * on a and gp [n] on p, the gradient of L = sum_i ga_i . a_i + gp_i p_i with
 * respect to the positions, gx [n][3], and masses, gm [n]. All FP32 device
 * arrays; gp may be NULL (no upstream gradient on p: a kernel without its
 * terms runs, 26 instead of 28 FP32 operations per pair). Computed as one
 * gather pass over all pairs (no atomics), so the result is reproducible.
 * Asynchronous.
 */
nb_status nb_force_vjp(nb_ctx *ctx, const float *x, const float *m, int64_t n, float eps,
                       const float *ga, const float *gp, float *gx, float *gm, void *stream);

/* Shape of nb_force_vjp's pair kernel (nb_tile fields threads, ipt, jtile,
 * stages, unroll, minblocks, release, sums_in_smem; the others as listed):
 * force one of the compiled shapes listed by nb_list_vjp_tiles (NULL
 * restores the built-in choice, by size and by whether gp is NULL), read the
 * shape nb_force_vjp uses at size n for a call with gp non-NULL, list the
 * compiled shapes (up to `cap` written to out, which may be NULL; the total
 * in *count). */
nb_status nb_set_vjp_tile(nb_ctx *ctx, const nb_tile *tile);
nb_status nb_get_vjp_tile(nb_ctx *ctx, int64_t n, nb_tile *out);
nb_status nb_list_vjp_tiles(nb_tile *out, int cap, int *count);

/*
 * nb_force for callers that may not allocate device memory. (This entry
 * point is an engineering addition; the paper has no counterpart.)
 *
 * Some callers cannot call cudaMalloc where they need forces: their device
 * memory is entirely owned by a pool or framework allocator, they run in a
 * loop that cannot afford the device-wide synchronisation an allocation can
 * trigger, or they are plug-ins that are handed buffers but not allowed to
 * allocate. This call needs no context and allocates nothing: its scratch
 * (packed particles and partial sums, plus an error word) is a fixed 16 MiB
 * array inside the library's device image, which every GPU that loads the
 * library holds until the process exits.
 *
 *   x, m, a, p, eps  as in nb_force (FP32 DEVICE arrays of the current
 *                    device, else NB_ERR_ARG; plain arithmetic, NB_PLAIN
 *                    results)
 *   n                at most 65536; larger n, or a device whose work split
 *                    would not fit the array, is rejected with NB_ERR_ARG
 *                    and a message (nb_last_error(NULL))
 *   stream           cudaStream_t as void* (NULL = legacy default stream)
 * The call waits for `stream` (only that stream) before returning and
 * reports a bounded-wait timeout as NB_ERR_TIMEOUT. Its first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and keeps it for the process; make that first call
 * before any stream capture, and do not use this entry point after a
 * cudaDeviceReset of that device. All calls share the one array, which
 * keeps the previous call's contents (everything that is read is rewritten
 * first): calls that overlap on the GPU, from several host threads or on
 * several streams, race on it and must be serialised by the caller.
 */
nb_status nb_force_noalloc(const float *x, const float *m, int64_t n, float eps, float *a, float *p,
                           void *stream);

/* Wait for `stream` and report device-side errors recorded by this context's
 * kernels since the last check (NB_ERR_TIMEOUT if a bounded wait ran out). */
nb_status nb_synchronize(nb_ctx *ctx, void *stream);

/* Tile shape used for nb_force at size n in `mode` (the override if one is
 * set, else the tuned entry for n's size class, else the built-in default). */
nb_status nb_get_tile(nb_ctx *ctx, int64_t n, nb_mode mode, nb_tile *out);

/* Force a tile shape for `mode` (must be one of the compiled shapes listed by
 * nb_list_tiles); NULL clears the override. */
nb_status nb_set_tile(nb_ctx *ctx, nb_mode mode, const nb_tile *tile);

/* Record `tile` (one of the compiled shapes) as the tuned shape for n's size
 * class (floor(log2 n)) in `mode`, as nb_autotune does after timing; NULL
 * forgets that class's entry. Used to restore saved tuning results. */
nb_status nb_set_tuned_tile(nb_ctx *ctx, int64_t n, nb_mode mode, const nb_tile *tile);

/* The compiled tile shapes of `mode`. Writes up to `cap` entries to out (may
 * be NULL) and the total count to *count. */
nb_status nb_list_tiles(nb_mode mode, nb_tile *out, int cap, int *count);

/*
 * The unroll depth and tile shape the paper leaves to future work (Section
 * "Conclusion"), chosen by measurement: time every compiled tile shape on
 * synthetic data of size n (generated on the device by the library; only
 * the timing is kept). Every shape is timed best of 2 whole calls after a
 * warm-up, then the three fastest 5 more times each, interleaved
 * (single-launch shapes only for n < 2^16). Keep the fastest for n's size class and return
 * it in *best with its rate in interactions per second in *rate (either may
 * be NULL). Synchronous.
 */
nb_status nb_autotune(nb_ctx *ctx, int64_t n, nb_mode mode, void *stream, nb_tile *best,
                      double *rate);

/* Per-kernel timing. With timing on, every kernel launch of this context is
 * bracketed by CUDA events on its stream. nb_timing_read waits for those
 * events and reports, for kernel class `kernel` (0 = pack, 1 = pair,
 * 2 = reduce, 3 = leap-frog update, 4 = batched pair, 5 = vjp pair), the
 * summed duration in ms and the launch count since the last reset. */
nb_status nb_timing_enable(nb_ctx *ctx, int on);
nb_status nb_timing_read(nb_ctx *ctx, int kernel, double *total_ms, int64_t *launches);
nb_status nb_timing_reset(nb_ctx *ctx);

/* Test hook for the bounded-wait path: with unit >= 0 the producer of the
 * pair kernel (and of the adjoint kernel of nb_force_vjp) does not issue the
 * copy of work unit `unit`, so the consumers'
 * bounded wait runs out, the kernel records a timeout and returns, and the
 * next nb_synchronize reports NB_ERR_TIMEOUT. In the cluster form of the
 * single-launch kernel (nb_tile.fused = 3) CTA `unit` does not send its
 * partial sums, and the CTAs that own them time out the same way. wait_ns
 * sets the wait limit (0 keeps the default of one second). -1 disables. */
nb_status nb_debug_set_fault(nb_ctx *ctx, int64_t unit, int64_t wait_ns);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
