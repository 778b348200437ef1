// Shared declarations of the warm-start network kernels (not public ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace cl {

struct ConvGeom {
    int N, D, H, W;           // voxels per batch item
    int ci, co;               // channels
    int in_stride, in_off;    // input channel stride / offset (concat buffers)
    int out_stride, out_off;  // output channel stride / offset
    int periodic_yz;
};

// tcgen05 convolution (conv_tc.cu): shapes it takes, and its launch.  `err`
// is a device word; bit 64 is raised when a bounded wait expired.
bool conv3d_tc_supported(const ConvGeom& g);
cudaError_t launch_conv3d_tc(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, __nv_bfloat16* out,
                             const ConvGeom& g, int relu, int* err, cudaStream_t s);

// tcgen05 weight gradient: per-slice partials [slice][27][co][ci] in
// `partial` (wgrad_tc_workspace_floats of them); *nslices receives their
// count.  lbo_mn selects which descriptor offset field carries the stride
// between core matrices along M / N for the MN-major operands.
bool conv3d_wgrad_tc_supported(const ConvGeom& g);
long long wgrad_tc_workspace_floats(const ConvGeom& g);
cudaError_t launch_conv3d_wgrad_tc(const __nv_bfloat16* in, const __nv_bfloat16* dout, float* partial,
                                   const ConvGeom& g, int lbo_mn, int* err, int* nslices, cudaStream_t s);

// weight gradient from halo tiles (preferred where supported); same
// partial layout and slice sum as the kernel above
bool conv3d_wgrad_halo_supported(const ConvGeom& g);
long long wgrad_halo_workspace_floats(const ConvGeom& g);
cudaError_t launch_conv3d_wgrad_halo(const __nv_bfloat16* in, const __nv_bfloat16* dout, float* partial,
                                     const ConvGeom& g, int* err, int* nslices, cudaStream_t s);

}  // namespace cl
