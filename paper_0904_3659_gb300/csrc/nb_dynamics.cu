// nb_dynamics.cu -- leap-frog integration (Fujiwara & Nakasato,
// arXiv:0904.3659, Section "Method", Eqs. (1)-(3)) and total energy, with the
// state (x, v) in FP64 on the device and the force from the FP32 pair kernel.
//
// One step (kick-drift-kick, the seven-step algorithm of Section "Method"):
//   v <- v + dt/2 g(x)       Eq. (1)
//   x <- x + dt v            Eq. (2) (x + v dt + g dt^2/2 with the new v)
//   g(x) from Eq. (gravity)  (g = -a: Eq. (gravity) has the sign of a repulsion)
//   v <- v + dt/2 g(x)       Eq. (3)
// The back kick of step k and the front kick of step k+1 use the same g and
// run in one kernel as two separate FP64 additions (identical rounding to
// running them apart), fused with the drift and the FP32 packing of the new
// positions. Steps after the first are replayed from a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "nb_device.cuh"
#include "nb_ext.h"
#include "nb_internal.h"

namespace nbk {

// Pack FP64 positions (rounded to FP32) and FP32 masses into JPart.
__device__ __forceinline__ void pack_one(JPart *jp, int64_t i, double px, double py, double pz,
                                         float mi) {
    const float fx = (float)px, fy = (float)py, fz = (float)pz;
    const float hm = -0.5f * mi;
    float4 *dst = reinterpret_cast<float4 *>(jp + i);
    dst[0] = make_float4(-fx, -fx, -fy, -fy);
    dst[1] = make_float4(-fz, -fz, hm, hm);
}

__global__ void pack_f64_kernel(const double *__restrict__ x, const float *__restrict__ m,
                                int64_t n, int64_t npad, JPart *__restrict__ jp) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i < n)
        pack_one(jp, i, x[3 * i], x[3 * i + 1], x[3 * i + 2], m[i]);
    else
        pack_one(jp, i, 0.0, 0.0, 0.0, 0.f);
}

// v += dt/2 g (back kick, if kick_back), v += dt/2 g (front kick),
// x += dt v, then pack x. g = -a.
__global__ void kick_drift_pack_kernel(double *__restrict__ x, double *__restrict__ v,
                                       const float *__restrict__ a, const float *__restrict__ m,
                                       int64_t n, int64_t npad, double dt, int kick_back,
                                       JPart *__restrict__ jp) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i >= n) {
        pack_one(jp, i, 0.0, 0.0, 0.0, 0.f);
        return;
    }
    const double h = 0.5 * dt;
    double xn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double g = -(double)a[3 * i + c];
        double vc = v[3 * i + c];
        if (kick_back) vc = vc + h * g;  // Eq. (3) of the previous step
        vc = vc + h * g;                 // Eq. (1)
        const double xc = x[3 * i + c] + dt * vc;  // Eq. (2)
        v[3 * i + c] = vc;
        x[3 * i + c] = xc;
        xn[c] = xc;
    }
    pack_one(jp, i, xn[0], xn[1], xn[2], m[i]);
}

// Kicks and drift without packing (the compensated path packs HL records
// in a separate kernel).
__global__ void kick_drift_kernel(double *__restrict__ x, double *__restrict__ v,
                                  const float *__restrict__ a, int64_t n, double dt, int kick_back) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const double h = 0.5 * dt, g = -(double)a[k];
    double vc = v[k];
    if (kick_back) vc = vc + h * g;  // Eq. (3) of the previous step
    vc = vc + h * g;                 // Eq. (1)
    v[k] = vc;
    x[k] = x[k] + dt * vc;           // Eq. (2)
}

__global__ void kick_kernel(double *__restrict__ v, const float *__restrict__ a, int64_t n,
                            double dt) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    v[k] = v[k] + (0.5 * dt) * (-(double)a[k]);  // Eq. (3)
}

// Reverse sweep of one step (the adjoint of the kick-drift-kick step above,
// with a_{t+1} = F(x_{t+1}) from Eq. (gravity) shared by the back kick of
// step t and the front kick of step t+1). lx, lv, la are the adjoints of
// x_{t+1}, v_{t+1} and a_{t+1} (la holding what the front kick of step t+1
// contributed); all in FP64.
// Before the force adjoint: the back kick v_{t+1} = v_h - dt/2 a_{t+1} adds
// -dt/2 lv to la, and the operands of the VJP kernel are formed in FP32.
__global__ void adj_back_kick_kernel(double *__restrict__ la, const double *__restrict__ lv,
                                     const double *__restrict__ x_next, int64_t n, double dt,
                                     float *__restrict__ ga32, float *__restrict__ x32) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const double l = la[k] + (-((0.5 * dt) * lv[k]));
    la[k] = l;
    ga32[k] = (float)l;
    x32[k] = (float)x_next[k];
}

// After the force adjoint (gx, gm = VJP of Eq. (gravity) at x_{t+1} with
// upstream la): lx += gx; the drift x_{t+1} = x_t + dt v_h adds dt lx to the
// adjoint of v_h; the front kick v_h = v_t - dt/2 a_t passes it on to v_t
// and gives a_t the adjoint -dt/2 lv. lm accumulates the mass gradient.
__global__ void adj_drift_kick_kernel(double *__restrict__ lx, double *__restrict__ lv,
                                      double *__restrict__ la, double *__restrict__ lm,
                                      const float *__restrict__ gx, const float *__restrict__ gm,
                                      int64_t n, double dt) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const double x = lx[k] + (double)gx[k];
    const double v = lv[k] + dt * x;
    lx[k] = x;
    lv[k] = v;
    la[k] = -((0.5 * dt) * v);
    if (k < n) lm[k] = lm[k] + (double)gm[k];
}

// The force at the start of a trajectory, a_0 = F(x_0): VJP operands from
// the adjoint of a_0, then its result folded into lx, lm (la cleared).
__global__ void adj_first_operands_kernel(const double *__restrict__ la,
                                          const double *__restrict__ x0, int64_t n,
                                          float *__restrict__ ga32, float *__restrict__ x32) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    ga32[k] = (float)la[k];
    x32[k] = (float)x0[k];
}

__global__ void adj_first_fold_kernel(double *__restrict__ lx, double *__restrict__ la,
                                      double *__restrict__ lm, const float *__restrict__ gx,
                                      const float *__restrict__ gm, int64_t n) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    lx[k] = lx[k] + (double)gx[k];
    la[k] = 0.0;
    if (k < n) lm[k] = lm[k] + (double)gm[k];
}

// HL packing of FP64 positions (compensated mode). Bounding box: per-block
// min/max, then one block combines them (min and max do not depend on the
// order) and forms the frame {centre x, y, z, grid G = 2^(E-23)} with 2^E
// bounding every |x - centre| (hl_grid_exponent).
constexpr int kBoxThreads = 256;

__global__ void __launch_bounds__(kBoxThreads) hl_box_partial_kernel(const double *__restrict__ x,
                                                                    int64_t n,
                                                                    double *__restrict__ part) {
    __shared__ double s[6][kBoxThreads];
    const int t = threadIdx.x;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)kBoxThreads + t; i < n; i += (int64_t)gridDim.x * kBoxThreads)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], x[3 * i + c]);
            hi[c] = fmax(hi[c], x[3 * i + c]);
        }
    for (int c = 0; c < 3; ++c) {
        s[c][t] = lo[c];
        s[3 + c][t] = hi[c];
    }
    __syncthreads();
    for (int w = kBoxThreads / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int c = 0; c < 3; ++c) {
                s[c][t] = fmin(s[c][t], s[c][t + w]);
                s[3 + c][t] = fmax(s[3 + c][t], s[3 + c][t + w]);
            }
        __syncthreads();
    }
    if (t < 6) part[6 * blockIdx.x + t] = s[t][0];
}

__global__ void __launch_bounds__(kBoxThreads) hl_frame_kernel(const double *__restrict__ part,
                                                              int nblocks, double *__restrict__ frame) {
    __shared__ double s[6][kBoxThreads];
    const int t = threadIdx.x;
    double b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int k = t; k < nblocks; k += kBoxThreads)
        for (int c = 0; c < 3; ++c) {
            b[c] = fmin(b[c], part[6 * k + c]);
            b[3 + c] = fmax(b[3 + c], part[6 * k + 3 + c]);
        }
    for (int c = 0; c < 6; ++c) s[c][t] = b[c];
    __syncthreads();
    for (int w = kBoxThreads / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int c = 0; c < 3; ++c) {
                s[c][t] = fmin(s[c][t], s[c][t + w]);
                s[3 + c][t] = fmax(s[3 + c][t], s[3 + c][t + w]);
            }
        __syncthreads();
    }
    if (t == 0) {
        double ext = 0.0;
        for (int c = 0; c < 3; ++c) {
            frame[c] = 0.5 * (s[c][0] + s[3 + c][0]);
            ext = fmax(ext, 0.5 * (s[3 + c][0] - s[c][0]));
        }
        frame[3] = ldexp(1.0, hl_grid_exponent(ext) - 23);
    }
}

// Particle i as HL records relative to the frame: h = y rounded to the grid
// (exact in FP32: |y| <= 2^E), l = fl32(y - h); rows n..npad-1 are inert.
__global__ void hl_pack_kernel(const double *__restrict__ x, const float *__restrict__ m, int64_t n,
                               int64_t npad, const double *__restrict__ frame,
                               JPart *__restrict__ jp) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f}, hm = 0.f;
    if (i < n) {
        const double g = frame[3], ginv = 1.0 / g;  // a power of two: exact
        for (int c = 0; c < 3; ++c) {
            const double y = x[3 * i + c] - frame[c];
            const double yh = rint(y * ginv) * g;
            h[c] = (float)yh;
            l[c] = (float)(y - yh);
        }
        hm = -0.5f * m[i];
    }
    float4 *dst = reinterpret_cast<float4 *>(jp + kHLRecords * i);
    dst[0] = make_float4(-h[0], -h[0], -h[1], -h[1]);
    dst[1] = make_float4(-h[2], -h[2], hm, hm);
    dst[2] = make_float4(-l[0], -l[0], -l[1], -l[1]);
    dst[3] = make_float4(-l[2], -l[2], 0.f, 0.f);
}

// Energy: per-block sums of K = 1/2 m |v|^2 and W = -1/2 m p in a fixed
// tree order, then one block adds the block sums in order.
constexpr int kEnergyThreads = 256;

__global__ void energy_partial_kernel(const double *__restrict__ v, const float *__restrict__ m,
                                      const float *__restrict__ p, int64_t n,
                                      double2 *__restrict__ block_sums) {
    __shared__ double sk[kEnergyThreads], sw[kEnergyThreads];
    const int t = threadIdx.x;
    double k = 0.0, w = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kEnergyThreads + t; i < n;
         i += (int64_t)gridDim.x * kEnergyThreads) {
        const double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
        const double mi = m[i];
        k += 0.5 * mi * (vx * vx + vy * vy + vz * vz);
        w += -0.5 * mi * (double)p[i];
    }
    sk[t] = k;
    sw[t] = w;
    __syncthreads();
    for (int s = kEnergyThreads / 2; s > 0; s >>= 1) {
        if (t < s) {
            sk[t] += sk[t + s];
            sw[t] += sw[t + s];
        }
        __syncthreads();
    }
    if (t == 0) block_sums[blockIdx.x] = make_double2(sk[0], sw[0]);
}

__global__ void energy_final_kernel(const double2 *__restrict__ block_sums, int nblocks,
                                    double2 *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double k = 0.0, w = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        k += block_sums[b].x;
        w += block_sums[b].y;
    }
    *out = make_double2(k, w);
}

}  // namespace nbk

using namespace nbk;
using namespace nbx;

namespace {

enum Slot : int {
    S_JP = SLOT_FP64_JP,
    S_A = SLOT_ENERGY_A,
    S_P = SLOT_P,
    S_EBLK = SLOT_ENERGY_BLK,
    S_EOUT = SLOT_ENERGY_OUT,
    S_BOX = SLOT_HL_BOX,
    S_ADJ = SLOT_ADJOINT
};

void *slot(nb_ctx *ctx, int k) { return ctx_ext(ctx).buf[k]; }

nb_status ensure_slot(nb_ctx *ctx, int k, size_t bytes) {
    ExtState &s = ctx_ext(ctx);
    cudaError_t e = ensure_buffer(&s.buf[k], &s.cap[k], bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation");
    return NB_OK;
}

unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Reserve everything one force evaluation from packed FP64 positions needs
// (HL records, two JParts per particle, in compensated mode).
nb_status reserve_force(nb_ctx *ctx, int64_t n, bool comp) {
    const PairVariant &v = choose_variant(ctx, n, comp);
    const PairPlan plan = make_plan(v, n, resident_ctas(ctx, v));
    return ensure_slot(ctx, S_JP, (size_t)plan.npad * (comp ? kHLRecords : 1) * sizeof(JPart));
}

int64_t padded(int64_t n) { return round_up(std::max<int64_t>(n, 1), kPad); }

// Compensated path for FP64 state: each force evaluation packs HL records
// relative to the centre of the current bounding box (box partials, then one
// block that forms the frame, then the pack), so the grid always covers
// every particle however far the integrator has moved it.
int box_blocks(int64_t n) { return (int)std::min<int64_t>(1024, (n + kBoxThreads - 1) / kBoxThreads); }

nb_status reserve_hl_state(nb_ctx *ctx, int64_t n) {
    nb_status st = ensure_slot(ctx, S_BOX, (size_t)(box_blocks(n) * 6 + 4) * sizeof(double));
    if (st != NB_OK) return st;
    return reserve_hl(ctx, n);
}

// Eq. (gravity) from FP64 positions through HL records (p may be NULL).
nb_status force_hl(nb_ctx *ctx, const double *x, const float *m, int64_t n, float eps, float *a,
                   float *p, cudaStream_t st) {
    JPart *jp = static_cast<JPart *>(slot(ctx, S_JP));
    double *part = static_cast<double *>(slot(ctx, S_BOX));
    double *frame = part + 6 * box_blocks(n);
    const int nblk = box_blocks(n);
    hl_box_partial_kernel<<<nblk, kBoxThreads, 0, st>>>(x, n, part);
    hl_frame_kernel<<<1, kBoxThreads, 0, st>>>(part, nblk, frame);
    hl_pack_kernel<<<blocks_for(padded(n), 256), 256, 0, st>>>(x, m, n, padded(n), frame, jp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "HL pack launch");
    return run_force_hl(ctx, jp, n, eps, a, p, st);
}

// Enqueue the steps 1 .. nsteps-1 body: fused kicks+drift+pack, force.
nb_status steady_step(nb_ctx *ctx, double *x, double *v, const float *m, float *a, float *p,
                      int64_t n, float eps, double dt, bool comp, cudaStream_t st) {
    JPart *jp = static_cast<JPart *>(slot(ctx, S_JP));
    kick_drift_pack_kernel<<<blocks_for(padded(n), 256), 256, 0, st>>>(x, v, a, m, n, padded(n), dt,
                                                                        1, jp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "leap-frog update launch");
    return run_force(ctx, nullptr, nullptr, jp, n, eps, a, p, comp, st);
}

// With x_hist set, copy the positions after step t (t = 0 for the entry
// positions) into x_hist[t] ([nsteps + 1][n][3] FP64): the adjoint's replay.
nb_status record(nb_ctx *ctx, double *x_hist, int t, const double *x, int64_t n, cudaStream_t s) {
    if (!x_hist) return NB_OK;
    const cudaError_t e = cudaMemcpyAsync(x_hist + (size_t)t * 3 * n, x, (size_t)3 * n * sizeof(double),
                                          cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? NB_OK : cuda_fail(ctx, e, "position history copy");
}

// The compensated leap-frog: every force evaluation packs the FP64 positions
// as HL records (force_hl). Steps after the first are replayed from a graph,
// unless the positions of every step are recorded (x_hist).
nb_status leapfrog_hl(nb_ctx *ctx, double *x, double *v, const float *m, float *a, float *p,
                      int64_t n, float eps, double dt, int nsteps, int a_valid, cudaStream_t s,
                      double *x_hist) {
    nb_status st = reserve_hl_state(ctx, n);
    if (st != NB_OK) return st;
    cudaError_t e;
    if (!a_valid && (st = force_hl(ctx, x, m, n, eps, a, p, s)) != NB_OK) return st;
    if ((st = record(ctx, x_hist, 0, x, n, s)) != NB_OK) return st;
    if (nsteps == 0) return NB_OK;
    const unsigned nb3 = blocks_for(3 * n, 256);
    auto step = [&](int kick_back) -> nb_status {
        kick_drift_kernel<<<nb3, 256, 0, s>>>(x, v, a, n, dt, kick_back);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return cuda_fail(ctx, le, "leap-frog update launch");
        return force_hl(ctx, x, m, n, eps, a, p, s);
    };
    if ((st = step(0)) != NB_OK || (st = record(ctx, x_hist, 1, x, n, s)) != NB_OK) return st;
    const int rest = nsteps - 1;
    if (rest >= 2 && s != nullptr && !x_hist) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture begin");
        const bool timing = ctx_set_timing(ctx, false);
        nb_status cst = step(1);
        ctx_set_timing(ctx, timing);
        e = cudaStreamEndCapture(s, &graph);
        if (cst != NB_OK) {
            if (graph) cudaGraphDestroy(graph);
            return cst;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture end");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
        for (int k = 0; k < rest && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, s);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    } else {
        for (int k = 0; k < rest; ++k)
            if ((st = step(1)) != NB_OK || (st = record(ctx, x_hist, k + 2, x, n, s)) != NB_OK)
                return st;
    }
    kick_kernel<<<nb3, 256, 0, s>>>(v, a, n, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "kick launch");
    return NB_OK;
}

// The plain leap-frog (scratch reserved by the caller): fused kicks, drift
// and FP32 packing, then the pair kernel. Steps after the first are replayed
// from a graph unless the positions of every step are recorded (x_hist).
nb_status leapfrog_plain(nb_ctx *ctx, double *x, double *v, const float *m, float *a, float *p,
                         int64_t n, float eps, double dt, int nsteps, int a_valid, cudaStream_t s,
                         double *x_hist) {
    JPart *jp = static_cast<JPart *>(slot(ctx, S_JP));
    cudaError_t e;
    nb_status st;
    if (!a_valid) {
        pack_f64_kernel<<<blocks_for(padded(n), 256), 256, 0, s>>>(x, m, n, padded(n), jp);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "pack launch");
        if ((st = run_force(ctx, nullptr, nullptr, jp, n, eps, a, p, false, s)) != NB_OK) return st;
    }
    if ((st = record(ctx, x_hist, 0, x, n, s)) != NB_OK) return st;
    if (nsteps == 0) return NB_OK;

    // Step 0: front kick + drift + pack, force.
    kick_drift_pack_kernel<<<blocks_for(padded(n), 256), 256, 0, s>>>(x, v, a, m, n, padded(n), dt, 0,
                                                                      jp);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "leap-frog update launch");
    if ((st = run_force(ctx, nullptr, nullptr, jp, n, eps, a, p, false, s)) != NB_OK) return st;
    if ((st = record(ctx, x_hist, 1, x, n, s)) != NB_OK) return st;

    // Steps 1 .. nsteps-1: the same kernels with the same arguments each
    // step, so they are captured once into a graph and replayed (not on the
    // legacy default stream, which cannot be captured).
    const int rest = nsteps - 1;
    if (rest >= 2 && s != nullptr && !x_hist) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture begin");
        const bool timing = ctx_set_timing(ctx, false);  // no event nodes in the graph
        nb_status cst = steady_step(ctx, x, v, m, a, p, n, eps, dt, false, s);
        ctx_set_timing(ctx, timing);
        e = cudaStreamEndCapture(s, &graph);
        if (cst != NB_OK) {
            if (graph) cudaGraphDestroy(graph);
            return cst;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture end");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
        for (int k = 0; k < rest && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, s);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    } else {
        for (int k = 0; k < rest; ++k)
            if ((st = steady_step(ctx, x, v, m, a, p, n, eps, dt, false, s)) != NB_OK ||
                (st = record(ctx, x_hist, k + 2, x, n, s)) != NB_OK)
                return st;
    }
    // Final back kick, Eq. (3).
    kick_kernel<<<blocks_for(3 * n, 256), 256, 0, s>>>(v, a, n, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "kick launch");
    return NB_OK;
}

// Scratch of a leap-frog call (before any graph capture). Without a caller's
// potential array (p NULL) the force kernels sum a_i only.
nb_status reserve_leapfrog(nb_ctx *ctx, int64_t n, nb_mode mode) {
    nb_status st;
    if ((st = reserve_force(ctx, n, mode == NB_COMPENSATED)) != NB_OK) return st;
    return nb_reserve(ctx, n, mode);
}

}  // namespace

extern "C" {

nb_status nb_leapfrog_step(nb_ctx *ctx, double *x, double *v, const float *m, float *a, float *p,
                           int64_t n, float eps, double dt, int nsteps, int a_valid, nb_mode mode,
                           void *stream) {
    if (!ctx) return NB_ERR_ARG;
    nb_status st = check_common(ctx, n, eps, mode);
    if (st != NB_OK) return st;
    if (nsteps < 0) return fail(ctx, NB_ERR_ARG, "nsteps must be >= 0");
    if (!std::isfinite(dt)) return fail(ctx, NB_ERR_ARG, "dt must be finite");
    if (n == 0) return NB_OK;
    if (!x || !v || !m || !a) return fail(ctx, NB_ERR_ARG, "NULL array pointer");
    DeviceGuard g(ctx_device(ctx));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Scratch first (allocation never happens inside the captured graph).
    if ((st = reserve_leapfrog(ctx, n, mode)) != NB_OK) return st;
    if (mode == NB_COMPENSATED)
        return leapfrog_hl(ctx, x, v, m, a, p, n, eps, dt, nsteps, a_valid, s, nullptr);
    return leapfrog_plain(ctx, x, v, m, a, p, n, eps, dt, nsteps, a_valid, s, nullptr);
}

nb_status nb_leapfrog_adjoint(nb_ctx *ctx, const double *x, const double *v, const float *a,
                              const float *m, int64_t n, float eps, double dt, int nsteps,
                              double *lx, double *lv, double *la, double *lm, int apply_first,
                              nb_mode mode, void *stream) {
    if (!ctx) return NB_ERR_ARG;
    nb_status st = check_common(ctx, n, eps, mode);
    if (st != NB_OK) return st;
    if (nsteps < 0) return fail(ctx, NB_ERR_ARG, "nsteps must be >= 0");
    if (!std::isfinite(dt)) return fail(ctx, NB_ERR_ARG, "dt must be finite");
    if (n == 0) return NB_OK;
    if (!x || !v || !m || !lx || !lv || !la || !lm) return fail(ctx, NB_ERR_ARG, "NULL array pointer");
    DeviceGuard g(ctx_device(ctx));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n3 = (size_t)3 * n;

    // One scratch buffer: replayed x, v (FP64), positions of every step
    // (FP64), replayed a, p and the VJP kernel's operands and results (FP32;
    // the trajectory has no upstream gradient on p, so the VJP gets none).
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_xv = al(n3 * sizeof(double)), b_hist = al((size_t)(nsteps + 1) * n3 * sizeof(double));
    const size_t b_v3 = al(n3 * sizeof(float)), b_s = al((size_t)n * sizeof(float));
    const size_t total = 2 * b_xv + b_hist + 4 * b_v3 + b_s;
    if ((st = ensure_slot(ctx, S_ADJ, total)) != NB_OK) return st;
    if ((st = reserve_leapfrog(ctx, n, mode)) != NB_OK) return st;
    unsigned char *base = static_cast<unsigned char *>(slot(ctx, S_ADJ));
    double *xw = reinterpret_cast<double *>(base);
    double *vw = reinterpret_cast<double *>(base + b_xv);
    double *hist = reinterpret_cast<double *>(base + 2 * b_xv);
    float *aw = reinterpret_cast<float *>(base + 2 * b_xv + b_hist);
    float *x32 = aw + b_v3 / sizeof(float);
    float *ga32 = x32 + b_v3 / sizeof(float);
    float *gx32 = ga32 + b_v3 / sizeof(float);
    float *gm32 = gx32 + b_v3 / sizeof(float);

    // Replay the segment on copies with the forward's own kernels (so the
    // same positions), recording x.
    cudaError_t e = cudaMemcpyAsync(xw, x, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vw, v, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && a) e = cudaMemcpyAsync(aw, a, n3 * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint replay copies");
    st = mode == NB_COMPENSATED
             ? leapfrog_hl(ctx, xw, vw, m, aw, nullptr, n, eps, dt, nsteps, a != nullptr, s, hist)
             : leapfrog_plain(ctx, xw, vw, m, aw, nullptr, n, eps, dt, nsteps, a != nullptr, s, hist);
    if (st != NB_OK) return st;

    // Reverse sweep, last step first: one VJP of Eq. (gravity) per step.
    const unsigned nb3 = blocks_for((int64_t)n3, 256);
    for (int t = nsteps - 1; t >= 0; --t) {
        adj_back_kick_kernel<<<nb3, 256, 0, s>>>(la, lv, hist + (size_t)(t + 1) * n3, n, dt, ga32, x32);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "adjoint kick launch");
        if ((st = nb_force_vjp(ctx, x32, m, n, eps, ga32, nullptr, gx32, gm32, stream)) != NB_OK)
            return st;
        adj_drift_kick_kernel<<<nb3, 256, 0, s>>>(lx, lv, la, lm, gx32, gm32, n, dt);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "adjoint drift launch");
    }
    if (apply_first) {
        adj_first_operands_kernel<<<nb3, 256, 0, s>>>(la, hist, n, ga32, x32);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "adjoint launch");
        if ((st = nb_force_vjp(ctx, x32, m, n, eps, ga32, nullptr, gx32, gm32, stream)) != NB_OK)
            return st;
        adj_first_fold_kernel<<<nb3, 256, 0, s>>>(lx, la, lm, gx32, gm32, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "adjoint launch");
    }
    return NB_OK;
}

nb_status nb_energy(nb_ctx *ctx, const double *x, const double *v, const float *m, int64_t n,
                    float eps, double *out_kw, nb_mode mode, void *stream) {
    if (!ctx) return NB_ERR_ARG;
    nb_status st = check_common(ctx, n, eps, mode);
    if (st != NB_OK) return st;
    if (!out_kw) return fail(ctx, NB_ERR_ARG, "out_kw is NULL");
    if (n == 0) {
        out_kw[0] = out_kw[1] = 0.0;
        return NB_OK;
    }
    if (!x || !v || !m) return fail(ctx, NB_ERR_ARG, "NULL array pointer");
    DeviceGuard g(ctx_device(ctx));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool comp = mode == NB_COMPENSATED;
    if ((st = reserve_force(ctx, n, comp)) != NB_OK) return st;
    if ((st = ensure_slot(ctx, S_A, (size_t)3 * n * sizeof(float))) != NB_OK) return st;
    if ((st = ensure_slot(ctx, S_P, (size_t)n * sizeof(float))) != NB_OK) return st;
    const int nblk = (int)std::min<int64_t>(1024, (n + kEnergyThreads - 1) / kEnergyThreads);
    if ((st = ensure_slot(ctx, S_EBLK, (size_t)nblk * sizeof(double2))) != NB_OK) return st;
    if ((st = ensure_slot(ctx, S_EOUT, sizeof(double2))) != NB_OK) return st;
    JPart *jp = static_cast<JPart *>(slot(ctx, S_JP));
    float *abuf = static_cast<float *>(slot(ctx, S_A));
    float *pbuf = static_cast<float *>(slot(ctx, S_P));
    cudaError_t e;
    if (comp) {
        if ((st = reserve_hl_state(ctx, n)) != NB_OK) return st;
        if ((st = force_hl(ctx, x, m, n, eps, abuf, pbuf, s)) != NB_OK) return st;
    } else {
        pack_f64_kernel<<<blocks_for(padded(n), 256), 256, 0, s>>>(x, m, n, padded(n), jp);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "pack launch");
        if ((st = run_force(ctx, nullptr, nullptr, jp, n, eps, abuf, pbuf, comp, s)) != NB_OK) return st;
    }
    double2 *blk = static_cast<double2 *>(slot(ctx, S_EBLK));
    double2 *out = static_cast<double2 *>(slot(ctx, S_EOUT));
    energy_partial_kernel<<<nblk, kEnergyThreads, 0, s>>>(v, m, pbuf, n, blk);
    energy_final_kernel<<<1, 32, 0, s>>>(blk, nblk, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "energy launch");
    double2 host{};
    e = cudaMemcpyAsync(&host, out, sizeof(double2), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "energy read");
    if ((st = nb_synchronize(ctx, stream)) != NB_OK) return st;
    out_kw[0] = host.x;
    out_kw[1] = host.y;
    return NB_OK;
}

}  // extern "C"
