// Kernels of the warm-start network: a 4-level 3D U-Net that maps the
// structure (phase one-hot, log of the relative diffusivity, the linear ramp)
// to a correction of the linear initial field.  Layout NDHWC, activations
// BF16, accumulation FP32, weights kept as FP32 masters with BF16 copies.
//
// 3x3x3 convolutions are implicit GEMMs on the tensor cores: rows are
// output voxels, columns output channels, the reduction runs over 27 taps x
// input channels.  Channel counts that are multiples of 16 run on tcgen05
// with the accumulator in tensor memory (conv_tc.cu); others on the
// warp-level mma.sync m16n8k16 kernel below (BF16 in, FP32 accumulate).
// x is zero padded, y and z wrap (the catalyst-layer structures are periodic
// in y and z).  The data gradient is the same convolution applied to the
// output gradient with the kernel flipped and its channel axes swapped; the
// weight gradient is a second GEMM reduced over voxels in fixed-size slices
// and summed in a fixed order.
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "internal.cuh"
#include "nn.cuh"

namespace cl {

__device__ __forceinline__ uint32_t ld_bf16x2(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// voxel index of v shifted by tap t, or -1 outside (x zero padded, y/z wrap or zero padded)
__device__ __forceinline__ long long shift_voxel(long long v, int t, const ConvGeom& g) {
    const int x = (int)(v % g.W);
    long long r = v / g.W;
    const int y = (int)(r % g.H);
    r /= g.H;
    const int z = (int)(r % g.D);
    const long long n = r / g.D;
    const int qx = x + t % 3 - 1;
    int qy = y + (t / 3) % 3 - 1;
    int qz = z + t / 9 - 1;
    if (qx < 0 || qx >= g.W) return -1;
    if (g.periodic_yz) {
        qy = qy < 0 ? qy + g.H : (qy >= g.H ? qy - g.H : qy);
        qz = qz < 0 ? qz + g.D : (qz >= g.D ? qz - g.D : qz);
    } else if (qy < 0 || qy >= g.H || qz < 0 || qz >= g.D) {
        return -1;
    }
    return qx + (long long)g.W * (qy + (long long)g.H * (qz + (long long)g.D * n));
}

// ---------------------------------------------------------- forward conv
// Block: 4 warps x 16 output voxels; NT n8-tiles of output channels per block
// (blockIdx.y selects the channel group).  w: [27][co][ci] BF16 (ci
// contiguous), bias FP32 [co].  ci must be a multiple of 16, co of 8*NT.
template <int NT>
__global__ void __launch_bounds__(128) k_conv3d(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ w,
                                                const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                ConvGeom g, int relu) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const long long v0 = ((long long)blockIdx.x * 4 + warp) * 16;
    const int co0 = blockIdx.y * NT * 8;
    const long long va = v0 + gq, vb = v0 + gq + 8;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    if (v0 < M) {
        for (int t = 0; t < 27; ++t) {
            const long long sa = va < M ? shift_voxel(va, t, g) : -1;
            const long long sb = vb < M ? shift_voxel(vb, t, g) : -1;
            const __nv_bfloat16* pa = in + (sa < 0 ? 0 : sa * g.in_stride + g.in_off);
            const __nv_bfloat16* pb = in + (sb < 0 ? 0 : sb * g.in_stride + g.in_off);
            const __nv_bfloat16* wt = w + (long long)t * g.co * g.ci;
            for (int c0 = 0; c0 < g.ci; c0 += 16) {
                const uint32_t a0 = sa < 0 ? 0u : ld_bf16x2(pa + c0 + 2 * tq);
                const uint32_t a1 = sb < 0 ? 0u : ld_bf16x2(pb + c0 + 2 * tq);
                const uint32_t a2 = sa < 0 ? 0u : ld_bf16x2(pa + c0 + 8 + 2 * tq);
                const uint32_t a3 = sb < 0 ? 0u : ld_bf16x2(pb + c0 + 8 + 2 * tq);
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                    const __nv_bfloat16* pw = wt + (long long)(co0 + j * 8 + gq) * g.ci + c0 + 2 * tq;
                    mma_bf16(acc[j], a0, a1, a2, a3, __ldg(reinterpret_cast<const unsigned*>(pw)),
                             __ldg(reinterpret_cast<const unsigned*>(pw + 8)));
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int c = co0 + j * 8 + 2 * tq;
        const float b0 = bias ? bias[c] : 0.f, b1 = bias ? bias[c + 1] : 0.f;
        float r0 = acc[j][0] + b0, r1 = acc[j][1] + b1, r2 = acc[j][2] + b0, r3 = acc[j][3] + b1;
        if (relu) { r0 = fmaxf(r0, 0.f); r1 = fmaxf(r1, 0.f); r2 = fmaxf(r2, 0.f); r3 = fmaxf(r3, 0.f); }
        if (va < M)
            *reinterpret_cast<__nv_bfloat162*>(out + va * g.out_stride + g.out_off + c) = __floats2bfloat162_rn(r0, r1);
        if (vb < M)
            *reinterpret_cast<__nv_bfloat162*>(out + vb * g.out_stride + g.out_off + c) = __floats2bfloat162_rn(r2, r3);
    }
}

// error bits of the network kernels (bit 64: a bounded wait of the tcgen05
// convolution expired), read and cleared by cl_nn_check
__device__ int g_nn_err;

static int* nn_err_ptr() {
    static std::mutex mu;
    static int* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_nn_err) != cudaSuccess) return nullptr;
        addr[dev] = static_cast<int*>(p);
    }
    return addr[dev];
}

cudaError_t launch_conv3d(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, __nv_bfloat16* out,
                          const ConvGeom& g, int relu, cudaStream_t s) {
    if (g.ci % 16 || g.co % 8) return cudaErrorInvalidValue;
    if (conv3d_tc_supported(g)) {
        int* err = nn_err_ptr();
        if (!err) return cudaErrorInvalidValue;
        return launch_conv3d_tc(in, w, bias, out, g, relu, err, s);
    }
    // output channel counts that are not a multiple of 16: warp-level MMA
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const unsigned gx = (unsigned)((M + 63) / 64);
    if (g.co % 64 == 0) k_conv3d<8><<<dim3(gx, g.co / 64), 128, 0, s>>>(in, w, bias, out, g, relu);
    else if (g.co % 32 == 0) k_conv3d<4><<<dim3(gx, g.co / 32), 128, 0, s>>>(in, w, bias, out, g, relu);
    else if (g.co % 16 == 0) k_conv3d<2><<<dim3(gx, g.co / 16), 128, 0, s>>>(in, w, bias, out, g, relu);
    else k_conv3d<1><<<dim3(gx, g.co / 8), 128, 0, s>>>(in, w, bias, out, g, relu);
    return cudaGetLastError();
}

// ------------------------------------------------------------ weight grad
// dW[t][co][ci] = sum_v dO[v][co] * I[shift(v, t)][ci].  Block: one tap, a
// 16 x 16 (co x ci) tile, a slice of voxels split over 4 warps; the warps'
// sums meet in shared memory and the block writes one partial per slice.
__global__ void __launch_bounds__(128) k_conv3d_wgrad(const __nv_bfloat16* __restrict__ in,
                                                      const __nv_bfloat16* __restrict__ dout,
                                                      float* __restrict__ partial, ConvGeom g, long long slice) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int t = blockIdx.y;
    const int ntile_ci = g.ci / 16;
    const int co0 = (blockIdx.z / ntile_ci) * 16, ci0 = (blockIdx.z % ntile_ci) * 16;
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const long long vs = (long long)blockIdx.x * slice;
    const long long ve = vs + slice < M ? vs + slice : M;
    float acc[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    auto dO = [&](long long v, int c) -> unsigned short {
        if (v >= ve) return 0;
        return __bfloat16_as_ushort(dout[v * g.out_stride + g.out_off + c]);
    };
    auto Iv = [&](long long s, int c) -> unsigned short {
        if (s < 0) return 0;
        return __bfloat16_as_ushort(in[s * g.in_stride + g.in_off + c]);
    };
    for (long long v0 = vs + warp * 16; v0 < ve; v0 += 64) {
        const long long k0 = v0 + 2 * tq, k1 = k0 + 1, k8 = k0 + 8, k9 = k0 + 9;
        const uint32_t a0 = dO(k0, co0 + gq) | ((uint32_t)dO(k1, co0 + gq) << 16);
        const uint32_t a1 = dO(k0, co0 + gq + 8) | ((uint32_t)dO(k1, co0 + gq + 8) << 16);
        const uint32_t a2 = dO(k8, co0 + gq) | ((uint32_t)dO(k9, co0 + gq) << 16);
        const uint32_t a3 = dO(k8, co0 + gq + 8) | ((uint32_t)dO(k9, co0 + gq + 8) << 16);
        const long long s0 = k0 < ve ? shift_voxel(k0, t, g) : -1, s1 = k1 < ve ? shift_voxel(k1, t, g) : -1;
        const long long s8 = k8 < ve ? shift_voxel(k8, t, g) : -1, s9 = k9 < ve ? shift_voxel(k9, t, g) : -1;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = ci0 + j * 8 + gq;
            const uint32_t b0 = Iv(s0, c) | ((uint32_t)Iv(s1, c) << 16);
            const uint32_t b1 = Iv(s8, c) | ((uint32_t)Iv(s9, c) << 16);
            mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
        }
    }
    __shared__ float sh[4][16][16];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        sh[warp][gq][j * 8 + 2 * tq] = acc[j][0];
        sh[warp][gq][j * 8 + 2 * tq + 1] = acc[j][1];
        sh[warp][gq + 8][j * 8 + 2 * tq] = acc[j][2];
        sh[warp][gq + 8][j * 8 + 2 * tq + 1] = acc[j][3];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * 16; e += 128) {
        const int r = e / 16, c = e % 16;
        const float sum = (sh[0][r][c] + sh[1][r][c]) + (sh[2][r][c] + sh[3][r][c]);
        partial[(((long long)blockIdx.x * 27 + t) * g.co + co0 + r) * g.ci + ci0 + c] = sum;
    }
}

// dW = sum over slices (fixed order); also accumulates into dW (+= when accumulate)
__global__ void k_sum_slices(const float* __restrict__ partial, int nslices, long long n, float* __restrict__ dw) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < nslices; ++k) s += partial[(long long)k * n + e];
        dw[e] = s;
    }
}

long long wgrad_slice(const ConvGeom& g) {
    const long long M = (long long)g.N * g.D * g.H * g.W;
    long long slice = 16384;
    while ((M + slice - 1) / slice > 64) slice *= 2;
    return slice;
}

// which descriptor field carries the M/N core-matrix stride of the MN-major
// operands of the tcgen05 weight gradient
constexpr int kWgradLboMN = 0;

cudaError_t launch_conv3d_wgrad(const __nv_bfloat16* in, const __nv_bfloat16* dout, float* partial, float* dw,
                                const ConvGeom& g, cudaStream_t s) {
    if (g.ci % 16 || g.co % 16) return cudaErrorInvalidValue;
    if (conv3d_wgrad_halo_supported(g)) {
        int* err = nn_err_ptr();
        if (!err) return cudaErrorInvalidValue;
        int ns = 0;
        cudaError_t e = launch_conv3d_wgrad_halo(in, dout, partial, g, err, &ns, s);
        if (e != cudaSuccess) return e;
        const long long n = 27LL * g.co * g.ci;
        k_sum_slices<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(partial, ns, n, dw);
        return cudaGetLastError();
    }
    if (conv3d_wgrad_tc_supported(g)) {
        int* err = nn_err_ptr();
        if (!err) return cudaErrorInvalidValue;
        int ns = 0;
        cudaError_t e = launch_conv3d_wgrad_tc(in, dout, partial, g, kWgradLboMN, err, &ns, s);
        if (e != cudaSuccess) return e;
        const long long n = 27LL * g.co * g.ci;
        k_sum_slices<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(partial, ns, n, dw);
        return cudaGetLastError();
    }
    // more than 128 output channels: warp-level MMA
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const long long slice = wgrad_slice(g);
    const int ns = (int)((M + slice - 1) / slice);
    k_conv3d_wgrad<<<dim3(ns, 27, (g.co / 16) * (g.ci / 16)), 128, 0, s>>>(in, dout, partial, g, slice);
    const long long n = 27LL * g.co * g.ci;
    k_sum_slices<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(partial, ns, n, dw);
    return cudaGetLastError();
}

// W'[t][ci][co] = W[26 - t][co][ci]: weights of the data-gradient convolution
__global__ void k_wt_dgrad(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wd, int co, int ci) {
    const long long n = 27LL * co * ci;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / ((long long)co * ci));
        const int r = (int)(e % ((long long)co * ci));
        const int o = r / ci, i = r % ci;
        wd[((long long)(26 - t) * ci + i) * co + o] = w[e];
    }
}

cudaError_t launch_wt_dgrad(const __nv_bfloat16* w, __nv_bfloat16* wd, int co, int ci, cudaStream_t s) {
    k_wt_dgrad<<<256, 256, 0, s>>>(w, wd, co, ci);
    return cudaGetLastError();
}

// ------------------------------------------------------------ elementwise
// bias gradient: db[c] = sum_v dO[v][c] (one block per channel, fixed order)
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dout, long long M, int stride, int off, float* db) {
    const int c = blockIdx.x;
    float s = 0.f;
    for (long long v = threadIdx.x; v < M; v += blockDim.x) s += __bfloat162float(dout[v * stride + off + c]);
    __shared__ float sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = sh[0];
}

// dY <- dY * (Y > 0)   (strided channel slice [off, off + C))
__global__ void k_relu_bwd(const __nv_bfloat16* __restrict__ y, __nv_bfloat16* __restrict__ dy, long long M, int C,
                           int stride, int off) {
    const long long n = M * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long v = e / C, c = e % C;
        const long long i = v * stride + off + c;
        if (!(__bfloat162float(y[i]) > 0.f)) dy[i] = __float2bfloat16(0.f);
    }
}

// 2x2x2 average pooling, forward and backward
__global__ void k_pool_fwd(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int N, int D, int H,
                           int W, int C, int xs, int xo) {
    const int d = D / 2, h = H / 2, w = W / 2;
    const long long n = (long long)N * d * h * w * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int ox = (int)(r % w); r /= w;
        const int oy = (int)(r % h); r /= h;
        const int oz = (int)(r % d);
        const long long b = r / d;
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const long long v = (2 * ox + (k & 1)) + (long long)W * ((2 * oy + ((k >> 1) & 1)) + (long long)H * ((2 * oz + (k >> 2)) + (long long)D * b));
            s += __bfloat162float(x[v * xs + xo + c]);
        }
        y[e] = __float2bfloat16(0.125f * s);
    }
}

__global__ void k_pool_bwd(const __nv_bfloat16* __restrict__ dy, __nv_bfloat16* __restrict__ dx, int N, int D, int H,
                           int W, int C, int xs, int xo, int accumulate) {
    const long long n = (long long)N * D * H * W * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int x = (int)(r % W); r /= W;
        const int y = (int)(r % H); r /= H;
        const int z = (int)(r % D);
        const long long b = r / D;
        const long long vo = (x / 2) + (long long)(W / 2) * ((y / 2) + (long long)(H / 2) * ((z / 2) + (long long)(D / 2) * b));
        float g = 0.125f * __bfloat162float(dy[vo * C + c]);
        const long long i = ((long long)x + (long long)W * (y + (long long)H * (z + (long long)D * b))) * xs + xo + c;
        if (accumulate) g += __bfloat162float(dx[i]);
        dx[i] = __float2bfloat16(g);
    }
}

// 2x nearest upsampling into a channel slice, and its backward (sum of 8 children)
__global__ void k_up_fwd(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int N, int D, int H, int W,
                         int C, int ys, int yo) {
    const long long n = (long long)N * D * H * W * C;  // D, H, W: output sizes
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int ox = (int)(r % W); r /= W;
        const int oy = (int)(r % H); r /= H;
        const int oz = (int)(r % D);
        const long long b = r / D;
        const long long vi = (ox / 2) + (long long)(W / 2) * ((oy / 2) + (long long)(H / 2) * ((oz / 2) + (long long)(D / 2) * b));
        const long long vo = ox + (long long)W * (oy + (long long)H * (oz + (long long)D * b));
        y[vo * ys + yo + c] = x[vi * C + c];
    }
}

__global__ void k_up_bwd(const __nv_bfloat16* __restrict__ dy, __nv_bfloat16* __restrict__ dx, int N, int D, int H, int W,
                         int C, int ys, int yo) {
    const int d = D / 2, h = H / 2, w = W / 2;
    const long long n = (long long)N * d * h * w * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int ix = (int)(r % w); r /= w;
        const int iy = (int)(r % h); r /= h;
        const int iz = (int)(r % d);
        const long long b = r / d;
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const long long v = (2 * ix + (k & 1)) + (long long)W * ((2 * iy + ((k >> 1) & 1)) + (long long)H * ((2 * iz + (k >> 2)) + (long long)D * b));
            s += __bfloat162float(dy[v * ys + yo + c]);
        }
        dx[e] = __float2bfloat16(s);
    }
}

// copy a C-channel tensor into / out of a channel slice of a wider buffer
__global__ void k_copy_channels(const __nv_bfloat16* __restrict__ src, int ss, int so, __nv_bfloat16* __restrict__ dst,
                                int ds, int dof, long long M, int C, int accumulate) {
    const long long n = M * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long v = e / C, c = e % C;
        float val = __bfloat162float(src[v * ss + so + c]);
        if (accumulate) val += __bfloat162float(dst[v * ds + dof + c]);
        dst[v * ds + dof + c] = __float2bfloat16(val);
    }
}

// head: y[v] = b + sum_c x[v][c] w[c] (FP32 out), the masked MSE against a
// target, and the gradients dx[v][c] = g[v] w[c], dw[c] = sum_v g[v] x[v][c]
__global__ void k_head_fwd(const __nv_bfloat16* __restrict__ x, const float* __restrict__ w, const float* __restrict__ b,
                           float* __restrict__ y, long long M, int C) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x) {
        float s = b[0];
        for (int c = 0; c < C; ++c) s += __bfloat162float(x[v * C + c]) * w[c];
        y[v] = s;
    }
}

// loss partials: per block sum of mask*(y - t)^2 and count; grad g = 2 mask (y - t) / count_total
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ target, const uint8_t* __restrict__ mask,
                      long long M, double* partial) {
    double s = 0.0, n = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x)
        if (mask[v]) {
            const double d = (double)y[v] - (double)target[v];
            s += d * d;
            n += 1.0;
        }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = n;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) { sh[0][threadIdx.x] += sh[0][threadIdx.x + w]; sh[1][threadIdx.x] += sh[1][threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { partial[2 * blockIdx.x] = sh[0][0]; partial[2 * blockIdx.x + 1] = sh[1][0]; }
}

__global__ void k_loss_finalize(const double* __restrict__ partial, int nb, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0, n = 0;
        for (int i = 0; i < nb; ++i) { s += partial[2 * i]; n += partial[2 * i + 1]; }
        out[0] = n > 0 ? s / n : 0.0;
        out[1] = n;
    }
}

__global__ void k_head_bwd(const __nv_bfloat16* __restrict__ x, const float* __restrict__ w, const float* __restrict__ y,
                           const float* __restrict__ target, const uint8_t* __restrict__ mask, const double* __restrict__ loss,
                           __nv_bfloat16* __restrict__ dx, float* __restrict__ gy, long long M, int C) {
    const double n = loss[1] > 0 ? loss[1] : 1.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x) {
        const float g = mask[v] ? (float)(2.0 * ((double)y[v] - (double)target[v]) / n) : 0.f;
        gy[v] = g;
        for (int c = 0; c < C; ++c) dx[v * C + c] = __float2bfloat16(g * w[c]);
    }
}

// head parameter gradients: one block per (c) plus one for the bias, fixed order
__global__ void k_head_wgrad(const __nv_bfloat16* __restrict__ x, const float* __restrict__ gy, long long M, int C,
                             float* __restrict__ dw, float* __restrict__ db) {
    const int c = blockIdx.x;  // c == C: bias
    float s = 0.f;
    for (long long v = threadIdx.x; v < M; v += blockDim.x) s += gy[v] * (c < C ? __bfloat162float(x[v * C + c]) : 1.f);
    __shared__ float sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (c < C) dw[c] = sh[0];
        else db[0] = sh[0];
    }
}

// Adam on FP32 masters, refreshing the BF16 copies
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ pb, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        const float pn = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        p[e] = pn;
        if (pb) pb[e] = __float2bfloat16(pn);
    }
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = __float2bfloat16(a[e]);
}

// ----------------------------------------------------- warm-start I/O
// D / D_max of an active cell from its relaxation rate (Eq. 24 inverted):
// (1/omega - 1/2) / (tau_ref - 1/2).
__device__ __forceinline__ float rel_diffusivity(float omega, float tau_ref) {
    return (1.f / omega - 0.5f) / (tau_ref - 0.5f);
}

// Cross-section conductances along x, per unit area, in units of D_max:
//   G[2x]     = mean over the ny*nz cells of plane x of D/D_max (0 on
//               inactive cells); the half-cell faces at the two x ends
//               conduct 2 G[0] and 2 G[2(nx-1)];
//   G[2x + 1] = mean over the ny*nz links between planes x and x+1 of the
//               harmonic link conductance 2 D_a D_b / (D_a + D_b) (0 unless
//               both cells are active): the same face conductance as the
//               steady D3Q7 flux between two cells.
// One block per plane, fixed reduction order.
__global__ void k_plane_conductance(const uint16_t* __restrict__ mask, const float* __restrict__ omega, int nx,
                                    long long nyz, float tau_ref, double* __restrict__ G) {
    const int x = blockIdx.x;
    double sp = 0.0, sl = 0.0;
    for (long long r = threadIdx.x; r < nyz; r += blockDim.x) {
        const long long c = x + (long long)nx * r;
        if (!(mask[c] & kActiveBit)) continue;
        const double a = (double)rel_diffusivity(omega[c], tau_ref);
        sp += a;
        if (x + 1 < nx && (mask[c + 1] & kActiveBit)) {
            const double b = (double)rel_diffusivity(omega[c + 1], tau_ref);
            sl += 2.0 * a * b / (a + b);
        }
    }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = sp;
    sh[1][threadIdx.x] = sl;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        G[2 * x] = sh[0][0] / (double)nyz;
        G[2 * x + 1] = sh[1][0] / (double)nyz;
    }
}

// Series-resistor profile between the two Dirichlet faces: the inlet half
// cell (resistance 1/(2 G[0])), the links between planes (1/G[2x+1]) and the
// outlet half cell (1/(2 G[2(nx-1)])) in series; the concentration at the
// centre of plane x is
//   s(x) = c_in - (c_in - c_out) (R_inlet + sum_{x' < x} R_link(x')) / R_total,
// the linear ramp when every plane conducts alike.  One thread.
__global__ void k_series_profile(const double* __restrict__ G, int nx, double c_in, double c_out,
                                 double* __restrict__ s) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double r_in = 1.0 / fmax(2.0 * G[0], 1e-12);
    double tot = r_in + 1.0 / fmax(2.0 * G[2 * (nx - 1)], 1e-12);
    for (int x = 0; x + 1 < nx; ++x) tot += 1.0 / fmax(G[2 * x + 1], 1e-12);
    double acc = r_in;
    for (int x = 0; x < nx; ++x) {
        s[x] = c_in - (c_in - c_out) * acc / tot;
        if (x + 1 < nx) acc += 1.0 / fmax(G[2 * x + 1], 1e-12);
    }
}

// Network input features from a solver's set-up, 16 channels per voxel:
// 0 active, 1 solid, 2 ionomer, 3 micropore, 4 log(D / D_max) mapped to
// max(0, 1 + ln(D/D_max)/6) on active cells (0 elsewhere), 5 the linear ramp,
// 6 the series-resistor profile s(x), 7 (s(x) - ramp(x)) nx / (4 (c_in -
// c_out)), 8..15 zero.  Channels 6 and 7 carry what a field at one place
// cannot see locally: how the resistance of every plane in x shifts the
// mean profile.
__global__ void k_features(const uint8_t* __restrict__ phase, const uint16_t* __restrict__ mask,
                           const float* __restrict__ omega, const double* __restrict__ series, int nx, long long N,
                           float tau_ref, float c_in, float c_out, __nv_bfloat16* __restrict__ feat) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const bool act = (mask[c] & kActiveBit) != 0;
        const uint8_t ph = phase[c];
        float f[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) f[k] = 0.f;
        f[0] = act ? 1.f : 0.f;
        f[1] = ph == 1 ? 1.f : 0.f;
        f[2] = ph == 2 ? 1.f : 0.f;
        f[3] = ph == 3 ? 1.f : 0.f;
        if (act) f[4] = fmaxf(0.f, 1.f + logf(fmaxf(rel_diffusivity(omega[c], tau_ref), 1e-6f)) / 6.f);
        const int x = (int)(c % nx);
        const float ramp = c_in + (c_out - c_in) * (x + 0.5f) / nx;
        f[5] = ramp;
        const float s = (float)series[x];
        f[6] = s;
        f[7] = c_in != c_out ? (s - ramp) * (float)nx / (4.f * (c_in - c_out)) : 0.f;
#pragma unroll
        for (int k = 0; k < 16; k += 2)
            *reinterpret_cast<__nv_bfloat162*>(feat + c * 16 + k) = __floats2bfloat162_rn(f[k], f[k + 1]);
    }
}

// target of the network: (C - ramp) on active cells, 0 elsewhere
// training target (C - ramp) nx / (c_in - c_out): scale-free
__global__ void k_target(const float* __restrict__ C, const uint16_t* __restrict__ mask, int nx, long long N, float c_in,
                         float c_out, float* __restrict__ t) {
    const float scale = (float)nx / (c_in - c_out);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const float ramp = c_in + (c_out - c_in) * (x + 0.5f) / nx;
        t[c] = (mask[c] & kActiveBit) ? (C[c] - ramp) * scale : 0.f;
    }
}

// warm start: C0 = ramp + pred (c_in - c_out) / nx: the prediction is in the units of
// the training target, (C - ramp) nx / (c_in - c_out)
__global__ void k_warm_field(const float* __restrict__ pred, const uint16_t* __restrict__ mask, int nx, long long N,
                             float c_in, float c_out, float* __restrict__ C0) {
    const float scale = (c_in - c_out) / (float)nx;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const float ramp = c_in + (c_out - c_in) * (x + 0.5f) / nx;
        C0[c] = (mask[c] & kActiveBit) ? fmaf(pred[c], scale, ramp) : 0.f;
    }
}

}  // namespace cl

// ================================================================ C ABI
using namespace cl;

static cl_status st_of(cudaError_t e) {
    return e == cudaSuccess ? CL_OK : (e == cudaErrorInvalidValue ? CL_ERR_ARG : CL_ERR_CUDA);
}

static ConvGeom geom(int N, int D, int H, int W, int ci, int co, int in_stride, int in_off, int out_stride, int out_off,
                     int periodic) {
    ConvGeom g;
    g.N = N; g.D = D; g.H = H; g.W = W; g.ci = ci; g.co = co;
    g.in_stride = in_stride; g.in_off = in_off; g.out_stride = out_stride; g.out_off = out_off;
    g.periodic_yz = periodic;
    return g;
}

static const unsigned kEw = 152 * 8;  // grid of the elementwise kernels

extern "C" {

cl_status cl_nn_conv3d(const void* in, const void* w, const float* bias, void* out, int N, int D, int H, int W, int ci,
                       int co, int in_stride, int in_off, int out_stride, int out_off, int relu, int periodic_yz,
                       void* stream) {
    if (!in || !w || !out || N < 1 || D < 1 || H < 1 || W < 1) return CL_ERR_ARG;
    return st_of(launch_conv3d((const __nv_bfloat16*)in, (const __nv_bfloat16*)w, bias, (__nv_bfloat16*)out,
                               geom(N, D, H, W, ci, co, in_stride, in_off, out_stride, out_off, periodic_yz), relu,
                               (cudaStream_t)stream));
}

long long cl_nn_wgrad_workspace(int N, int D, int H, int W, int ci, int co) {
    const ConvGeom g = geom(N, D, H, W, ci, co, ci, 0, co, 0, 1);
    const long long M = (long long)N * D * H * W;
    const long long slice = wgrad_slice(g);
    const long long legacy = ((M + slice - 1) / slice) * 27LL * co * ci;
    const long long tc = wgrad_tc_workspace_floats(g), halo = wgrad_halo_workspace_floats(g);
    long long m = legacy > tc ? legacy : tc;
    m = m > halo ? m : halo;
    return m * (long long)sizeof(float);
}

cl_status cl_nn_conv3d_wgrad(const void* in, const void* dout, float* workspace, float* dw, int N, int D, int H, int W,
                             int ci, int co, int in_stride, int in_off, int out_stride, int out_off, int periodic_yz,
                             void* stream) {
    if (!in || !dout || !workspace || !dw) return CL_ERR_ARG;
    return st_of(launch_conv3d_wgrad((const __nv_bfloat16*)in, (const __nv_bfloat16*)dout, workspace, dw,
                                     geom(N, D, H, W, ci, co, in_stride, in_off, out_stride, out_off, periodic_yz),
                                     (cudaStream_t)stream));
}

cl_status cl_nn_wt_dgrad(const void* w, void* wd, int co, int ci, void* stream) {
    return st_of(launch_wt_dgrad((const __nv_bfloat16*)w, (__nv_bfloat16*)wd, co, ci, (cudaStream_t)stream));
}

cl_status cl_nn_bias_grad(const void* dout, long long M, int C, int stride, int off, float* db, void* stream) {
    k_bias_grad<<<C, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)dout, M, stride, off, db);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_relu_bwd(const void* y, void* dy, long long M, int C, int stride, int off, void* stream) {
    k_relu_bwd<<<kEw, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)y, (__nv_bfloat16*)dy, M, C, stride, off);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_pool(const void* x, void* y, int N, int D, int H, int W, int C, int xs, int xo, void* stream) {
    if ((D | H | W) & 1) return CL_ERR_ARG;
    k_pool_fwd<<<kEw, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)x, (__nv_bfloat16*)y, N, D, H, W, C, xs, xo);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_pool_bwd(const void* dy, void* dx, int N, int D, int H, int W, int C, int xs, int xo, int accumulate,
                         void* stream) {
    k_pool_bwd<<<kEw, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)dy, (__nv_bfloat16*)dx, N, D, H, W, C, xs, xo,
                                                      accumulate);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_upsample(const void* x, void* y, int N, int D, int H, int W, int C, int ys, int yo, void* stream) {
    k_up_fwd<<<kEw, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)x, (__nv_bfloat16*)y, N, D, H, W, C, ys, yo);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_upsample_bwd(const void* dy, void* dx, int N, int D, int H, int W, int C, int ys, int yo, void* stream) {
    k_up_bwd<<<kEw, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)dy, (__nv_bfloat16*)dx, N, D, H, W, C, ys, yo);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_copy_channels(const void* src, int ss, int so, void* dst, int ds, int dof, long long M, int C,
                              int accumulate, void* stream) {
    k_copy_channels<<<kEw, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)src, ss, so, (__nv_bfloat16*)dst, ds, dof,
                                                           M, C, accumulate);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_head(const void* x, const float* w, const float* b, float* y, long long M, int C, void* stream) {
    k_head_fwd<<<kEw, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)x, w, b, y, M, C);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_mse(const float* y, const float* target, const uint8_t* mask, long long M, double* workspace,
                    double* loss, void* stream) {
    const int nb = 256;
    k_mse<<<nb, 256, 0, (cudaStream_t)stream>>>(y, target, mask, M, workspace);
    k_loss_finalize<<<1, 32, 0, (cudaStream_t)stream>>>(workspace, nb, loss);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_head_bwd(const void* x, const float* w, const float* y, const float* target, const uint8_t* mask,
                         const double* loss, void* dx, float* gy, float* dw, float* db, long long M, int C, void* stream) {
    k_head_bwd<<<kEw, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)x, w, y, target, mask, loss,
                                                      (__nv_bfloat16*)dx, gy, M, C);
    k_head_wgrad<<<C + 1, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)x, gy, M, C, dw, db);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_adam(float* p, const float* g, float* m, float* v, void* p_bf16, long long n, float lr, float b1, float b2,
                     float eps, int step, void* stream) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<kEw, 256, 0, (cudaStream_t)stream>>>(p, g, m, v, (__nv_bfloat16*)p_bf16, n, lr, b1, b2, eps, c1, c2);
    return st_of(cudaGetLastError());
}

cl_status cl_nn_check(void* stream) {
    int* err = nn_err_ptr();
    if (!err) return CL_ERR_CUDA;
    int h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
    if (h) {
        const int zero = 0;
        if (cudaMemcpyAsync(err, &zero, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) return CL_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
        return CL_ERR_TIMEOUT;
    }
    return CL_OK;
}

cl_status cl_nn_to_bf16(const float* a, void* b, long long n, void* stream) {
    k_f32_to_bf16<<<kEw, 256, 0, (cudaStream_t)stream>>>(a, (__nv_bfloat16*)b, n);
    return st_of(cudaGetLastError());
}

}  // extern "C"

// Features, targets and warm starts straight from a solver handle
#include "handle.cuh"

extern "C" {

cl_status cl_lbm_features(cl_handle h, void* feat) {
    CKS(h && h->have_structure ? CL_OK : CL_ERR_STATE);
    if (!feat) return CL_ERR_ARG;
    // cross-section conductances and the series profile in the readout scratch (5 nx doubles)
    double* G = h->d_plane;
    double* series = h->d_plane + 2 * h->nx;
    k_plane_conductance<<<h->nx, 256, 0, h->s>>>(h->mask, h->omega, h->nx, h->N / h->nx, (float)h->p.tau_ref, G);
    k_series_profile<<<1, 32, 0, h->s>>>(G, h->nx, h->p.c_in, h->p.c_out, series);
    k_features<<<kEw, 256, 0, h->s>>>(h->phase, h->mask, h->omega, series, h->nx, h->N, (float)h->p.tau_ref,
                                      (float)h->p.c_in, (float)h->p.c_out, (__nv_bfloat16*)feat);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->s));
    return CL_OK;
}

cl_status cl_lbm_target(cl_handle h, float* target) {
    CKS(h && h->have_structure ? CL_OK : CL_ERR_STATE);
    if (!target) return CL_ERR_ARG;
    CKS(cl_lbm_get_field(h, h->fbuf, 1));
    k_target<<<kEw, 256, 0, h->s>>>(h->fbuf, h->mask, h->nx, h->N, (float)h->p.c_in, (float)h->p.c_out, target);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->s));
    return CL_OK;
}

cl_status cl_lbm_init_warm(cl_handle h, const float* pred) {
    CKS(h && h->have_structure ? CL_OK : CL_ERR_STATE);
    if (!pred) return CL_ERR_ARG;
    k_warm_field<<<kEw, 256, 0, h->s>>>(pred, h->mask, h->nx, h->N, (float)h->p.c_in, (float)h->p.c_out, h->fbuf);
    CK(cudaGetLastError());
    return cl_lbm_init(h, h->fbuf, 1);
}

}  // extern "C"
