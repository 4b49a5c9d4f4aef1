// Sustained FP32 lane operations per SM clock on this GPU, for the two issue
// forms the pair kernels can use: scalar FFMA (one lane-op per lane per
// instruction) and packed FFMA2 (two). One CTA of 1024 threads per SM runs
// 8 independent multiply-add chains per thread (16 lanes' worth for FFMA2);
// each CTA reads its SM's cycle counter (clock64) and the global timer
// around the timed loop, so the rate is in lane-ops per SM cycle and the
// effective SM clock (cycles / ns) comes from the same run: no clock is
// assumed. Prints, per form, the median over CTAs of lane-ops/clk/SM, the
// median SM clock in MHz, and how many distinct SMs the CTAs ran on.
#include <algorithm>
#include <cstdio>
#include <cuda_runtime.h>
#include <vector>

constexpr int kThreads = 1024;
constexpr int kIters = 4096;

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smid() {
    unsigned s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

template <bool PACKED>
__global__ void __launch_bounds__(kThreads, 1) chains(float seed, long long *cyc, long long *ns,
                                                       unsigned *sm, float *sink) {
    __shared__ long long c0, t0;
    float a[8];
    float2 p[8];
    const float b = 1.0f - 1e-7f * (threadIdx.x & 7), c = 1e-8f * seed;
    for (int k = 0; k < 8; ++k) {
        a[k] = seed + k + threadIdx.x;
        p[k] = make_float2(a[k], a[k] + 0.5f);
    }
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    __syncthreads();
    if (threadIdx.x == 0) {
        c0 = clock64();
        t0 = (long long)gtime();
    }
    __syncthreads();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (PACKED)
                p[k] = __ffma2_rn(p[k], b2, c2);
            else
                a[k] = __fmaf_rn(a[k], b, c);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cyc[blockIdx.x] = clock64() - c0;
        ns[blockIdx.x] = (long long)gtime() - t0;
        sm[blockIdx.x] = smid();
    }
    float s = 0.f;
    for (int k = 0; k < 8; ++k) s += PACKED ? p[k].x + p[k].y : a[k];
    if (s == 1234.5f) sink[0] = s;  // keeps the chains alive
}

template <bool PACKED>
int run(int sms) {
    long long *cyc, *ns;
    unsigned *sm;
    float *sink;
    cudaMalloc(&cyc, sms * sizeof(long long));
    cudaMalloc(&ns, sms * sizeof(long long));
    cudaMalloc(&sm, sms * sizeof(unsigned));
    cudaMalloc(&sink, sizeof(float));
    std::vector<double> rate, mhz;
    std::vector<unsigned> ids(sms);
    int distinct = 0;
    for (int rep = 0; rep < 5; ++rep) {
        chains<PACKED><<<sms, kThreads>>>(1.0f + rep, cyc, ns, sm, sink);
        if (cudaDeviceSynchronize() != cudaSuccess) return 1;
        std::vector<long long> hc(sms), hn(sms);
        cudaMemcpy(hc.data(), cyc, sms * sizeof(long long), cudaMemcpyDeviceToHost);
        cudaMemcpy(hn.data(), ns, sms * sizeof(long long), cudaMemcpyDeviceToHost);
        cudaMemcpy(ids.data(), sm, sms * sizeof(unsigned), cudaMemcpyDeviceToHost);
        const double lane_ops = (double)kThreads * kIters * 8 * (PACKED ? 2 : 1);
        if (rep == 0) continue;  // warm-up
        for (int b = 0; b < sms; ++b) {
            rate.push_back(lane_ops / (double)hc[b]);
            mhz.push_back((double)hc[b] / (double)hn[b] * 1e3);
        }
        std::vector<unsigned> u(ids);
        std::sort(u.begin(), u.end());
        distinct = (int)(std::unique(u.begin(), u.end()) - u.begin());
    }
    std::sort(rate.begin(), rate.end());
    std::sort(mhz.begin(), mhz.end());
    printf("%s %.2f %.0f %d\n", PACKED ? "ffma2" : "ffma", rate[rate.size() / 2], mhz[mhz.size() / 2],
           distinct);
    cudaFree(cyc);
    cudaFree(ns);
    cudaFree(sm);
    cudaFree(sink);
    return 0;
}

int main() {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    if (run<false>(sms) || run<true>(sms)) {
        printf("error %s\n", cudaGetErrorString(cudaGetLastError()));
        return 1;
    }
    return 0;
}
