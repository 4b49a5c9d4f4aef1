// Accuracy of the special-function unit's reciprocal square root
// (rsqrt.approx.ftz.f32) and of one Newton-Raphson step evaluated in FP32 the
// way the pair kernels do it (y2 = y*y, t = s*y2 - 3, u = y*t, y1 = -u/2),
// against 1/sqrt(s) in FP64, for every FP32 value s in [1, 4): every mantissa
// with both exponent parities (the estimate of 4^k s is 2^-k times that of s).
// Prints, per quantity (y, y1, y^3, y1^3), the largest relative error and the
// mean relative error.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cuda_runtime.h>

__device__ __forceinline__ float rsqrt_approx(float s) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(s));
    return y;
}

__global__ void probe(unsigned *max_bits, double *sums, unsigned count) {
    __shared__ double part[4][256];
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    double e[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < count) {
        const float s = __uint_as_float(0x3F800000u + i);
        const float y = rsqrt_approx(s);
        const float y2 = __fmul_rn(y, y);
        const float t = __fmaf_rn(s, y2, -3.f);
        const float y1 = -0.5f * __fmul_rn(y, t);
        const double ref = 1.0 / sqrt((double)s), ref3 = ref * ref * ref;
        e[0] = ((double)y - ref) / ref;
        e[1] = ((double)y1 - ref) / ref;
        e[2] = ((double)y * y * y - ref3) / ref3;
        e[3] = ((double)y1 * y1 * y1 - ref3) / ref3;
        for (int k = 0; k < 4; ++k) atomicMax(&max_bits[k], __float_as_uint((float)fabs(e[k])));
    }
    for (int k = 0; k < 4; ++k) part[k][threadIdx.x] = e[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 4; ++k) part[k][threadIdx.x] += part[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) atomicAdd(&sums[k], part[k][0]);
}

int main() {
    const unsigned count = 1u << 24;  // [1, 4): two binades of 2^23 values
    unsigned *max_bits = nullptr;
    double *sums = nullptr;
    if (cudaMalloc(&max_bits, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&sums, 4 * sizeof(double)) != cudaSuccess) {
        printf("error allocation\n");
        return 1;
    }
    cudaMemset(max_bits, 0, 4 * sizeof(unsigned));
    cudaMemset(sums, 0, 4 * sizeof(double));
    probe<<<count / 256, 256>>>(max_bits, sums, count);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        printf("error %s\n", cudaGetErrorString(e));
        return 1;
    }
    unsigned hb[4];
    double hs[4];
    cudaMemcpy(hb, max_bits, sizeof hb, cudaMemcpyDeviceToHost);
    cudaMemcpy(hs, sums, sizeof hs, cudaMemcpyDeviceToHost);
    const char *names[4] = {"y", "y1", "y3", "y13"};
    for (int k = 0; k < 4; ++k) {
        float f;
        memcpy(&f, &hb[k], sizeof f);
        printf("%s %.6e %.6e\n", names[k], (double)f, hs[k] / count);
    }
    cudaFree(max_bits);
    cudaFree(sums);
    return 0;
}
