// Device-side reduction helpers shared by the kernels of the library.
#pragma once

#include <cuda_runtime.h>

namespace cl {

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
}

// Block-wide sum of NV doubles in a fixed order; thread 0 writes out[0..NV).
// blockDim must be a multiple of 32 and at most 1024 threads.
template <int NV>
__device__ void block_sum_store(double (&v)[NV], double* out) {
    __shared__ double sh[32][NV];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5, nwarps = (nthreads + 31) >> 5;
    warp_sum<NV>(v);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = lane < nwarps ? sh[lane][k] : 0.0;
        warp_sum<NV>(v);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) out[k] = v[k];
    }
}

}  // namespace cl
