// nb_order.h -- spatial ordering and per-tile reference points (nb_order.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "nb_internal.h"

namespace nbx {

// Bytes of scratch launch_spatial_order needs for n particles.
size_t order_scratch_bytes(int64_t n);
int64_t order_pow2(int64_t n);

// perm[k] (k < n) = index of the k-th particle in Morton order of x (FP64
// [n][3]); deterministic. perm must hold order_pow2(n) entries (the entries
// from n on are scratch).
cudaError_t launch_spatial_order(const double *x, int64_t n, void *scratch, int32_t *perm,
                                 cudaStream_t st);

// Packs the particles in perm order as FP32 offsets from their j-tile's
// reference point (tile = jtile consecutive ordered particles; only 256 is
// compiled) and writes the reference points cref[npad / jtile].
cudaError_t launch_frames_pack(const double *x, const float *m, const int32_t *perm, int64_t n,
                               int64_t npad, int jtile, nbk::JPart *jp, float4 *cref,
                               cudaStream_t st);

}  // namespace nbx
