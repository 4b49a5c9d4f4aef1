// Where the time of one N = 4096 force call goes in the cluster form of the
// single-launch kernel, in steady state: 400 launches back to back with
// programmatic dependent launch, as the library issues them. The kernel
// below is fused_cl_kernel<8 warps, 4 i per lane, 32-particle tiles, unroll
// 4, one CTA per SM, plain> of the library (the same building blocks,
// included from its source, in the same order) with %globaltimer stamps
// written per CTA and launch: entry, after the wait for the previous launch,
// after the j-chunk pack, each warp's end of compute, after the cross-warp
// sums, after the cluster barrier, after the partials have arrived, exit.
// Prints one line per phase: name, then the 10th, 50th and 90th percentile
// over launches (of the median CTA where the phase is per CTA), in us; then
// the per-launch time of the back-to-back loop from CUDA events.
#include "../../paper_0904_3659_gb300/csrc/nb_pair.cu"

#include <algorithm>
#include <cstdio>
#include <vector>

using namespace nbk;

namespace {

constexpr int kStamps = 16;  // 0..7 as listed above, 8..15 each warp's end of compute

__device__ __forceinline__ unsigned long long stamp() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(256, 1) traced_cl(const FusedArgs args, unsigned long long *tr, int launch) {
    namespace cg = cooperative_groups;
    constexpr int WARPS = 8, IPT = 4, JT = 32, UNR = 4, THREADS = WARPS * 32;
    constexpr int P = IPT / 2, IB = 32 * IPT, W = 1, TPB = kFusedJmax / JT;
    extern __shared__ __align__(128) unsigned char smem[];
    JPart *blk = reinterpret_cast<JPart *>(smem);
    float4 *red = reinterpret_cast<float4 *>(smem);
    float4 *cpart = reinterpret_cast<float4 *>(smem + kFusedJmax * sizeof(JPart));
    __shared__ uint64_t recv_bar;
    unsigned long long *T = tr + ((size_t)launch * gridDim.x + blockIdx.x) * kStamps;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) T[0] = stamp();
    pdl_wait_then_release();
    if (tid == 0) T[1] = stamp();
    cg::cluster_group cluster = cg::this_cluster();
    const int64_t n = args.n, nch = args.nchunks;
    const int64_t b = blockIdx.x / nch;
    const int c = (int)cluster.block_rank();
    const int64_t t0 = c * args.njt / nch, t1 = (c + 1) * args.njt / nch;
    if (tid == 0) {
        const uint32_t owned = (uint32_t)((IB - c + nch - 1) / nch);
        mbar_init(&recv_bar, 1);
        mbar_arrive_expect_tx(&recv_bar, owned * (uint32_t)(nch - 1) * W * (uint32_t)sizeof(float4));
        fence_mbar_init();
    }
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    float2 xi[P], yi[P], zi[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int64_t i0 = b * IB + (2 * q) * 32 + lane, i1 = i0 + 32;
        float3 p0 = make_float3(0.f, 0.f, 0.f), p1 = p0;
        if (i0 < n) p0 = make_float3(args.x[3 * i0], args.x[3 * i0 + 1], args.x[3 * i0 + 2]);
        if (i1 < n) p1 = make_float3(args.x[3 * i1], args.x[3 * i1 + 1], args.x[3 * i1 + 2]);
        xi[q] = make_float2(p0.x, p1.x);
        yi[q] = make_float2(p0.y, p1.y);
        zi[q] = make_float2(p0.z, p1.z);
    }
    const float2 eps2 = splat2(args.eps2);
    const float2 zero2 = splat2(0.f);
    float2 sum[P][4];
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) sum[q][r] = zero2;
    for (int64_t bt0 = t0; bt0 < t1; bt0 += TPB) {
        const int64_t bt1 = bt0 + TPB < t1 ? bt0 + TPB : t1;
        pack_block<THREADS>(args.x, args.m, n, bt0 * JT, (int)(bt1 - bt0) * JT, blk);
        __syncthreads();
        if (tid == 0) T[2] = stamp();
        for (int64_t t = bt0 + warp; t < bt1; t += WARPS) {
            const JPart *Tl = blk + (t - bt0) * JT;
            float2 acc[P][4];
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[q][r] = zero2;
            const int64_t ibase = b * IB, jbase = t * JT;
            int self0[P], self1[P];
            if (jbase < ibase + IB && ibase < jbase + JT)
                tile_pass_diag32<P, UNR, false>((int)((jbase - ibase) / 32), lane, Tl, xi, yi, zi, acc, eps2);
            else
                tile_pass<P, JT, UNR, false, kMixAll, false>(Tl, xi, yi, zi, acc, eps2, self0, self1);
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
                for (int r = 0; r < 4; ++r) sum[q][r] = add2(sum[q][r], acc[q][r]);
        }
        if (lane == 0) T[8 + warp] = stamp();
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int i0 = (2 * q) * 32 + lane, i1 = i0 + 32;
        float4 *dst = red + (int64_t)warp * W * IB;
        dst[i0] = make_float4(sum[q][0].x, sum[q][1].x, sum[q][2].x, sum[q][3].x);
        dst[i1] = make_float4(sum[q][0].y, sum[q][1].y, sum[q][2].y, sum[q][3].y);
    }
    __syncthreads();
    if (tid == 0) T[4] = stamp();
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    if (tid == 0) T[5] = stamp();
    for (int l = tid; l < IB; l += THREADS) {
        float S[4] = {0.f, 0.f, 0.f, 0.f};
        for (int w = 0; w < WARPS; ++w) {
            const float4 hi = red[(int64_t)w * W * IB + l];
            S[0] = __fadd_rn(S[0], hi.x);
            S[1] = __fadd_rn(S[1], hi.y);
            S[2] = __fadd_rn(S[2], hi.z);
            S[3] = __fadd_rn(S[3], hi.w);
        }
        const int owner = l % (int)nch, slot = l / (int)nch;
        float4 *dst = cpart + ((int64_t)slot * nch + c) * W;
        const float4 hi = make_float4(S[0], S[1], S[2], S[3]);
        if (owner == c)
            dst[0] = hi;
        else
            st_async_v4(cluster_map(dst, (uint32_t)owner), hi, cluster_map(&recv_bar, (uint32_t)owner));
    }
    const bool arrived = mbar_wait_bounded(&recv_bar, 0, kDefaultWaitNs);
    __syncthreads();
    if (tid == 0) T[6] = stamp();
    if (!arrived) {
        if (tid == 0) atomicOr(args.err, kErrTimeout);
        return;
    }
    for (int slot = tid; slot * (int)nch + c < IB; slot += THREADS) {
        const int l = slot * (int)nch + c;
        const int64_t gi = b * IB + l;
        if (gi >= n) break;
        float S[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < (int)nch; ++k) {
            const float4 hi = cpart[((int64_t)slot * nch + k) * W];
            S[0] = __fadd_rn(S[0], hi.x);
            S[1] = __fadd_rn(S[1], hi.y);
            S[2] = __fadd_rn(S[2], hi.z);
            S[3] = __fadd_rn(S[3], hi.w);
        }
        args.a[3 * gi + 0] = args.a_scale * S[0];
        args.a[3 * gi + 1] = args.a_scale * S[1];
        args.a[3 * gi + 2] = args.a_scale * S[2];
        args.p[gi] = args.p_scale * S[3];
    }
    __syncthreads();
    if (tid == 0) T[7] = stamp();
}

double pct(std::vector<double> v, double f) {
    std::sort(v.begin(), v.end());
    return v[(size_t)(f * (v.size() - 1))];
}

}  // namespace

int main() {
    const int n = 4096, IB = 128, nib = n / IB, nch = 4, grid = nib * nch, K = 400, K0 = 100;
    std::vector<float> hx(3 * n), hm(n, 1.0f / n);
    unsigned s = 1;
    for (auto &v : hx) {
        s = s * 1664525u + 1013904223u;
        v = (float)((s >> 8) & 0xffff) / 65536.f - 0.5f;
    }
    float *x, *m, *a, *p;
    int *err;
    unsigned long long *tr;
    const size_t tr_bytes = (size_t)K * grid * kStamps * sizeof(unsigned long long);
    if (cudaMalloc(&x, 3 * n * 4) != cudaSuccess || cudaMalloc(&m, n * 4) != cudaSuccess ||
        cudaMalloc(&a, 3 * n * 4) != cudaSuccess || cudaMalloc(&p, n * 4) != cudaSuccess ||
        cudaMalloc(&err, 4) != cudaSuccess || cudaMalloc(&tr, tr_bytes) != cudaSuccess) {
        printf("status allocation-failed\n");
        return 1;
    }
    cudaMemset(tr, 0, tr_bytes);
    cudaMemset(err, 0, 4);
    cudaMemcpy(x, hx.data(), 3 * n * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m, hm.data(), n * 4, cudaMemcpyHostToDevice);
    FusedArgs fa{};
    fa.x = x;
    fa.m = m;
    fa.n = n;
    fa.a = a;
    fa.p = p;
    fa.err = err;
    fa.nib = nib;
    fa.njt = n / 32;
    fa.nchunks = nch;
    fa.grid = grid;
    fa.eps2 = 1e-4f;
    fa.a_scale = -2.f;
    fa.p_scale = -2.f;
    fa.wait_ns = kDefaultWaitNs;
    fa.fault_cta = -1;
    // One CTA per SM, as the library's minblocks = 1 cluster shape requests.
    const size_t smem = kClusterOneSmSmem;
    cudaFuncSetAttribute(traced_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    auto launch = [&](int k) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = nch;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        return cudaLaunchKernelEx(&cfg, traced_cl, fa, tr, k);
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int k = 0; k < K0; ++k) launch(k);
    cudaEventRecord(e0, st);
    for (int k = K0; k < K; ++k) launch(k);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaStreamSynchronize(st);
    int herr = 0;
    cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
    printf("status %s %d\n", e == cudaSuccess ? "ok" : cudaGetErrorString(e), herr);
    if (e != cudaSuccess || herr != 0) return 1;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    std::vector<unsigned long long> h(tr_bytes / sizeof(unsigned long long));
    cudaMemcpy(h.data(), tr, tr_bytes, cudaMemcpyDeviceToHost);
    std::vector<double> gap, span, pack, comp_diag, comp_other, sums, cwait, arrive, comb;
    for (int k = K0 + 1; k < K; ++k) {
        const unsigned long long *H = &h[(size_t)k * grid * kStamps];
        const unsigned long long *Hp = &h[(size_t)(k - 1) * grid * kStamps];
        unsigned long long first_rel = ~0ull, last_exit = 0, prev_exit = 0;
        std::vector<double> pk, sm, cw, ar, cb;
        for (int c = 0; c < grid; ++c) {
            const unsigned long long *S = H + (size_t)c * kStamps;
            first_rel = std::min(first_rel, S[1]);
            last_exit = std::max(last_exit, S[7]);
            prev_exit = std::max(prev_exit, Hp[(size_t)c * kStamps + 7]);
            unsigned long long wend = 0;
            for (int w = 0; w < 8; ++w) wend = std::max(wend, S[8 + w]);
            const int b = c / nch, ch = c % nch;
            const int t0 = ch * (n / 32) / nch, t1 = (ch + 1) * (n / 32) / nch;
            const bool diag = 4 * b < t1 && t0 < 4 * b + 4;
            (diag ? comp_diag : comp_other).push_back((wend - S[2]) * 1e-3);
            pk.push_back((S[2] - S[1]) * 1e-3);
            sm.push_back((S[4] - wend) * 1e-3);
            cw.push_back((S[5] - S[4]) * 1e-3);
            ar.push_back((S[6] - S[5]) * 1e-3);
            cb.push_back((S[7] - S[6]) * 1e-3);
        }
        gap.push_back(((double)first_rel - (double)prev_exit) * 1e-3);
        span.push_back((last_exit - first_rel) * 1e-3);
        pack.push_back(pct(pk, 0.5));
        sums.push_back(pct(sm, 0.5));
        cwait.push_back(pct(cw, 0.5));
        arrive.push_back(pct(ar, 0.5));
        comb.push_back(pct(cb, 0.5));
    }
    auto row = [](const char *name, const std::vector<double> &v) {
        printf("%s %.3f %.3f %.3f\n", name, pct(v, 0.1), pct(v, 0.5), pct(v, 0.9));
    };
    row("gap_previous_exit_to_release", gap);
    row("span_release_to_last_exit", span);
    row("pack", pack);
    row("compute_cta_with_diagonal", comp_diag);
    row("compute_other_cta", comp_other);
    row("cross_warp_sums", sums);
    row("cluster_barrier_wait", cwait);
    row("send_and_arrival", arrive);
    row("combine_and_write", comb);
    printf("per_launch_us %.3f\n", ms * 1e3 / (K - K0));
    return 0;
}
