// Diffusion preconditioner and flexible-GMRES vector kernels of the
// preconditioned Krylov steady solve (D3Q7, plain f32 populations).
//
// The slow modes of the step map S are diffusive: a correction of
// equilibrium shape, w_i eps, changes the cell sums by L eps in one step,
// where L is the graph Laplacian of the active cells with link weight
// w = 1/8 (the one-step exchange of equilibrium populations), 2w on a
// fixed-concentration face (anti-bounce-back returns -w eps), (1 - r) w on
// a catalytic face (the sink keeps 1 - r of what meets it) and nothing on
// a bounce-back face.  The preconditioner P v = v + w_i eps with
// L eps = sum_i v_i puts those modes near 1, so that a Krylov method on
// (I - A) x = b (A: the step with zero boundary values) needs a number of
// step applications that does not grow with the box.  L is symmetric
// positive definite (with a fixed-concentration face or a sink) and is
// solved by conjugate gradients with its diagonal as preconditioner.
//
// Every vector kernel is a grid-stride loop.  The inner CG's dot products
// accumulate per thread in FP32 (a few dozen terms each: ample for a solve
// to 1e-2, and FP64 arithmetic runs at a small fraction of the FP32 rate on
// this GPU), then per block in FP64; the GMRES dot products accumulate in
// FP64.  One block sums the block partials in a fixed order.
// The CG scalars live in device memory, so a batch of iterations runs
// without a host round trip.
#include "internal.cuh"
#include "device_util.cuh"
#include "dsa.cuh"

namespace cl {

namespace {

constexpr int kDT = 256;

// Row of L at cell c: the diagonal, and sum over open links of w * v[neighbour].
__device__ __forceinline__ void lap_row(uint16_t m, int x, int y, int z, long long c, const DsaArgs& a,
                                        const float* __restrict__ v, float* diag, float* off) {
    const long long plane = (long long)a.nx * a.ny;
    float d = 0.f, o = 0.f;
#pragma unroll
    for (int k = 1; k <= 6; ++k) {
        if ((m >> (k - 1)) & 1u) {
            if (k == 2 && x == 0) d += a.bc_in == CL_BC_DIRICHLET ? 2.f * kW1 : 0.f;
            else if (k == 1 && x == a.nx - 1) d += a.bc_out == CL_BC_DIRICHLET ? 2.f * kW1 : 0.f;
            else if ((m >> (kReactShift + k - 1)) & 1u)
                d += (a.kscale ? (float)cell_sink(a.k_lu, a.kscale[c]) : a.rsink) * kW1;
        } else if (v) {
            long long nb;
            if (k == 1) nb = c + 1;
            else if (k == 2) nb = c - 1;
            else if (k == 3) nb = y == a.ny - 1 ? c - (long long)(a.ny - 1) * a.nx : c + a.nx;
            else if (k == 4) nb = y == 0 ? c + (long long)(a.ny - 1) * a.nx : c - a.nx;
            else if (k == 5) nb = z == a.nz - 1 ? c - (long long)(a.nz - 1) * plane : c + plane;
            else nb = z == 0 ? c + (long long)(a.nz - 1) * plane : c - plane;
            d += kW1;
            o += kW1 * v[nb];
        } else {
            d += kW1;
        }
    }
    *diag = d;
    *off = o;
}

// (x, y, z) of cell c: 32-bit division while the box's cell count fits (a
// 64-bit division is a long emulated sequence on the GPU)
__device__ __forceinline__ void cell_xyz(long long c, const DsaArgs& a, int* x, int* y, int* z) {
    if (a.N < (1LL << 31)) {
        const unsigned cc = (unsigned)c, nx = (unsigned)a.nx, ny = (unsigned)a.ny;
        const unsigned r = cc / nx;
        *x = (int)(cc - r * nx);
        *y = (int)(r % ny);
        *z = (int)(r / ny);
        return;
    }
    *x = (int)(c % a.nx);
    const long long r = c / a.nx;
    *y = (int)(r % a.ny);
    *z = (int)(r / a.ny);
}

// 1 / diag(L) on active cells, 0 elsewhere
__global__ void __launch_bounds__(kDT) k_lap_dinv(DsaArgs a, float* __restrict__ dinv) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint16_t m = a.mask[c];
        float out = 0.f;
        if (m & kActiveBit) {
            int x, y, z;
            cell_xyz(c, a, &x, &y, &z);
            float d, o;
            lap_row(m, x, y, z, c, a, nullptr, &d, &o);
            out = d > 0.f ? 1.f / d : 0.f;
        }
        dinv[c] = out;
    }
}

// CG start from eps = 0 on the cell sums of v: r = sum_i v_i, z = dinv r, p = z; partials r.z, r.r
__global__ void __launch_bounds__(kDT) k_cg_start(DsaArgs a, const float* __restrict__ v, const float* __restrict__ dinv,
                                                  float* __restrict__ eps, float* __restrict__ r,
                                                  float* __restrict__ zc, float* __restrict__ p,
                                                  double* __restrict__ part) {
    float af[2] = {0.f, 0.f};  // per-thread FP32 partials (FP64 is a small fraction of the FP32 rate here)
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        float rho = 0.f;
        if (a.mask[c] & kActiveBit) {
#pragma unroll
            for (int i = 0; i < 7; ++i) rho += v[(long long)i * a.N + c];
        }
        const float zz = dinv[c] * rho;
        eps[c] = 0.f;
        r[c] = rho;
        zc[c] = zz;
        p[c] = zz;
        af[0] = fmaf(rho, zz, af[0]);
        af[1] = fmaf(rho, rho, af[1]);
    }
    double acc[2] = {(double)af[0], (double)af[1]};
    block_sum_store<2>(acc, part + 2 * blockIdx.x);
}

// q = L p; partial p.q
__global__ void __launch_bounds__(kDT) k_cg_lap(DsaArgs a, const float* __restrict__ p, float* __restrict__ q,
                                                double* __restrict__ part, const CgScalars* __restrict__ cs) {
    if (cs->bad) return;
    float af = 0.f;  // per-thread FP32 partial
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint16_t m = a.mask[c];
        float out = 0.f;
        if (m & kActiveBit) {
            int x, y, z;
            cell_xyz(c, a, &x, &y, &z);
            float d, o;
            lap_row(m, x, y, z, c, a, p, &d, &o);
            out = d * p[c] - o;
        }
        q[c] = out;
        af = fmaf(p[c], out, af);
    }
    double acc[1] = {(double)af};
    block_sum_store<1>(acc, part + 2 * blockIdx.x);
}

// eps += alpha p; r -= alpha q; z = dinv r; partials r.z, r.r
__global__ void __launch_bounds__(kDT) k_cg_update(long long N, const float* __restrict__ p, const float* __restrict__ q,
                                                   const float* __restrict__ dinv, float* __restrict__ eps,
                                                   float* __restrict__ r, float* __restrict__ zc,
                                                   double* __restrict__ part, const CgScalars* __restrict__ cs) {
    if (cs->bad) return;
    const float al = (float)cs->alpha;
    float af[2] = {0.f, 0.f};  // per-thread FP32 partials
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        eps[c] = fmaf(al, p[c], eps[c]);
        const float rr = fmaf(-al, q[c], r[c]);
        r[c] = rr;
        const float zz = dinv[c] * rr;
        zc[c] = zz;
        af[0] = fmaf(rr, zz, af[0]);
        af[1] = fmaf(rr, rr, af[1]);
    }
    double acc[2] = {(double)af[0], (double)af[1]};
    block_sum_store<2>(acc, part + 2 * blockIdx.x);
}

// p = z + beta p
__global__ void __launch_bounds__(kDT) k_cg_p(long long N, const float* __restrict__ zc, float* __restrict__ p,
                                              const CgScalars* __restrict__ cs) {
    if (cs->bad) return;
    const float be = (float)cs->beta;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        p[c] = fmaf(be, p[c], zc[c]);
}

template <int WHICH>
__global__ void __launch_bounds__(kDT) k_cg_fin(const double* __restrict__ part, int nblk, CgScalars* __restrict__ cs) {
    if (WHICH != CG_START && cs->bad) return;
    double acc[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        acc[0] += part[2 * b];
        if (WHICH != CG_ALPHA) acc[1] += part[2 * b + 1];
    }
    __shared__ double tot[2];
    block_sum_store<2>(acc, tot);
    if (threadIdx.x != 0) return;
    const double t0 = tot[0], t1 = tot[1];
    if (WHICH == CG_START) {
        cs->rz = t0;
        cs->rr = cs->rr0 = t1;
        cs->alpha = cs->beta = 0.0;
        cs->iters = 0;
        cs->bad = isfinite(t0) && isfinite(t1) ? (t1 > 0.0 && t0 > 0.0 ? 0 : 2) : 1;
    } else if (WHICH == CG_ALPHA) {
        const double al = cs->rz / t0;
        if (t0 > 0.0 && isfinite(al)) cs->alpha = al;
        else cs->bad = 1;
    } else {
        cs->rr = t1;
        cs->iters += 1;
        const double be = t0 / cs->rz;
        if (!isfinite(t1) || !isfinite(be)) cs->bad = 1;
        else if (t1 == 0.0 || t0 == 0.0) cs->bad = 2;
        else {
            cs->beta = be;
            cs->rz = t0;
        }
    }
}

// zout_i = v_i + w_i eps
__global__ void __launch_bounds__(kDT) k_prec_out(long long N, const float* __restrict__ v, const float* __restrict__ eps,
                                                  float* __restrict__ zout) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const float e = eps[c];
        zout[c] = fmaf(kW0, e, v[c]);
#pragma unroll
        for (int i = 1; i < 7; ++i) zout[(long long)i * N + c] = fmaf(kW1, e, v[(long long)i * N + c]);
    }
}

// ---- flexible GMRES
// partial a.b
__global__ void __launch_bounds__(kDT) k_dot(const float* __restrict__ x, const float* __restrict__ y, long long L,
                                             double* __restrict__ part) {
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        acc[0] += (double)x[i] * y[i];
    block_sum_store<1>(acc, part + 2 * blockIdx.x);
}

// *out = sum of the partials (take_sqrt: its square root)
__global__ void __launch_bounds__(kDT) k_dot_fin(const double* __restrict__ part, int nblk, double* __restrict__ out,
                                                 int take_sqrt) {
    double acc[1] = {0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc[0] += part[2 * b];
    __shared__ double tot[1];
    block_sum_store<1>(acc, tot);
    if (threadIdx.x == 0) *out = take_sqrt ? sqrt(tot[0]) : tot[0];
}

// y += sign * coef[0] * x
__global__ void __launch_bounds__(kDT) k_axpy_dev(float* __restrict__ y, const float* __restrict__ x,
                                                  const double* __restrict__ coef, float sign, long long L) {
    const float a = sign * (float)coef[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], y[i]);
}

// y = x / nrm[0] (0 if the norm is 0)
__global__ void __launch_bounds__(kDT) k_scale_dev(float* __restrict__ y, const float* __restrict__ x,
                                                   const double* __restrict__ nrm, long long L) {
    const double n = nrm[0];
    const float s = n > 0.0 ? (float)(1.0 / n) : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        y[i] = s * x[i];
}

// out = a - b + c (c nullable)
__global__ void __launch_bounds__(kDT) k_comb(const float* __restrict__ a, const float* __restrict__ b,
                                              const float* __restrict__ c, float* __restrict__ out, long long L) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        out[i] = c ? (a[i] - b[i]) + c[i] : a[i] - b[i];
}

// ---- D3Q19 (Eq. 22-24): link weights 1/18 (axial), 1/36 (diagonal), 1/3 (rest)
// velocities of Eq. 22 in the order of the step kernels: 1-6 axial (+x, -x,
// +y, -y, +z, -z), 7-18 the face diagonals
__device__ __forceinline__ int d19_cx(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__device__ __forceinline__ int d19_cy(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__device__ __forceinline__ int d19_cz(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
__device__ __forceinline__ float d19_w(int i) { return i == 0 ? 1.f / 3.f : (i <= 6 ? 1.f / 18.f : 1.f / 36.f); }

__device__ __forceinline__ void cell_xyz19(long long c, const DsaArgs& a, const Dsa19& b, int* x, int* y, int* z) {
    const long long r = c / b.px;
    *x = (int)(c - r * b.px);
    *y = (int)(r % a.ny);
    *z = (int)(r / a.ny);
}

// Row of L at cell c on D3Q19: for each link toward x + c_i, weight w_i to an
// open neighbour; a closed link is a wall (nothing) or catalytic ((1 - r)
// w_i on the diagonal); a link that leaves the box in x meets the inlet or
// outlet face (2 w_i at a fixed value, nothing at zero flux).  A closed link
// takes precedence over the face, as in the step kernel.
__device__ __forceinline__ void lap_row19(uint32_t m, uint32_t rb, int x, int y, int z, const DsaArgs& a,
                                          const Dsa19& b, const float* __restrict__ v, float* diag, float* off) {
    float d = 0.f, o = 0.f;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const float w = d19_w(i);
        const int cx = d19_cx(i), cy = d19_cy(i), cz = d19_cz(i);
        if ((m >> (i - 1)) & 1u) {
            if ((rb >> (i - 1)) & 1u) d += a.rsink * w;
        } else if ((cx < 0 && x == 0) || (cx > 0 && x == a.nx - 1)) {
            if ((cx < 0 ? a.bc_in : a.bc_out) == CL_BC_DIRICHLET) d += 2.f * w;
        } else {
            d += w;
            if (v) {
                const int yy = y + cy < 0 ? a.ny - 1 : (y + cy >= a.ny ? 0 : y + cy);
                const int zz = z + cz < 0 ? a.nz - 1 : (z + cz >= a.nz ? 0 : z + cz);
                o += w * v[(long long)(x + cx) + (long long)b.px * (yy + (long long)a.ny * zz)];
            }
        }
    }
    *diag = d;
    *off = o;
}

__global__ void __launch_bounds__(kDT) k_lap_dinv19(DsaArgs a, Dsa19 b, float* __restrict__ dinv) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint32_t m = b.mask[c];
        float out = 0.f;
        if (m & kQ19Active) {
            int x, y, z;
            cell_xyz19(c, a, b, &x, &y, &z);
            const uint32_t rb = (m & kQ19HasReact) ? b.react[c] : 0u;
            float d, o;
            lap_row19(m, rb, x, y, z, a, b, nullptr, &d, &o);
            out = d > 0.f ? 1.f / d : 0.f;
        }
        dinv[c] = out;
    }
}

__global__ void __launch_bounds__(kDT) k_cg_start19(DsaArgs a, Dsa19 b, const float* __restrict__ v,
                                                    const float* __restrict__ dinv, float* __restrict__ eps,
                                                    float* __restrict__ r, float* __restrict__ zc,
                                                    float* __restrict__ p, double* __restrict__ part) {
    float af[2] = {0.f, 0.f};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        float rho = 0.f;
        if (b.mask[c] & kQ19Active) {
#pragma unroll
            for (int i = 0; i < 19; ++i) rho += v[(long long)i * a.N + c];
        }
        const float zz = dinv[c] * rho;
        eps[c] = 0.f;
        r[c] = rho;
        zc[c] = zz;
        p[c] = zz;
        af[0] = fmaf(rho, zz, af[0]);
        af[1] = fmaf(rho, rho, af[1]);
    }
    double acc[2] = {(double)af[0], (double)af[1]};
    block_sum_store<2>(acc, part + 2 * blockIdx.x);
}

__global__ void __launch_bounds__(kDT) k_cg_lap19(DsaArgs a, Dsa19 b, const float* __restrict__ p,
                                                  float* __restrict__ q, double* __restrict__ part,
                                                  const CgScalars* __restrict__ cs) {
    if (cs->bad) return;
    float af = 0.f;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint32_t m = b.mask[c];
        float out = 0.f;
        if (m & kQ19Active) {
            int x, y, z;
            cell_xyz19(c, a, b, &x, &y, &z);
            const uint32_t rb = (m & kQ19HasReact) ? b.react[c] : 0u;
            float d, o;
            lap_row19(m, rb, x, y, z, a, b, p, &d, &o);
            out = d * p[c] - o;
        }
        q[c] = out;
        af = fmaf(p[c], out, af);
    }
    double acc[1] = {(double)af};
    block_sum_store<1>(acc, part + 2 * blockIdx.x);
}

// zout_i = v_i + w_i eps over the 19 planes
__global__ void __launch_bounds__(kDT) k_prec_out19(long long N, const float* __restrict__ v,
                                                    const float* __restrict__ eps, float* __restrict__ zout) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const float e = eps[c];
#pragma unroll
        for (int i = 0; i < 19; ++i) zout[(long long)i * N + c] = fmaf(d19_w(i), e, v[(long long)i * N + c]);
    }
}

}  // namespace

cudaError_t launch_lap_dinv(const DsaArgs& a, float* dinv, int nblk, cudaStream_t s) {
    k_lap_dinv<<<nblk, kDT, 0, s>>>(a, dinv);
    return cudaGetLastError();
}

cudaError_t launch_cg_start(const DsaArgs& a, const float* v, const float* dinv, float* eps, float* r, float* zc,
                            float* p, int nblk, double* part, CgScalars* cs, cudaStream_t s) {
    k_cg_start<<<nblk, kDT, 0, s>>>(a, v, dinv, eps, r, zc, p, part);
    k_cg_fin<CG_START><<<1, kDT, 0, s>>>(part, nblk, cs);
    return cudaGetLastError();
}

cudaError_t launch_cg_iter(const DsaArgs& a, const float* dinv, float* eps, float* r, float* zc, float* p, float* q,
                           int nblk, double* part, CgScalars* cs, cudaStream_t s) {
    k_cg_lap<<<nblk, kDT, 0, s>>>(a, p, q, part, cs);
    k_cg_fin<CG_ALPHA><<<1, kDT, 0, s>>>(part, nblk, cs);
    k_cg_update<<<nblk, kDT, 0, s>>>(a.N, p, q, dinv, eps, r, zc, part, cs);
    k_cg_fin<CG_BETA><<<1, kDT, 0, s>>>(part, nblk, cs);
    k_cg_p<<<nblk, kDT, 0, s>>>(a.N, zc, p, cs);
    return cudaGetLastError();
}

cudaError_t launch_prec_out(long long N, const float* v, const float* eps, float* zout, int nblk, cudaStream_t s) {
    k_prec_out<<<nblk, kDT, 0, s>>>(N, v, eps, zout);
    return cudaGetLastError();
}

cudaError_t launch_dot_dev(const float* x, const float* y, long long L, int nblk, double* part, double* out,
                           int take_sqrt, cudaStream_t s) {
    k_dot<<<nblk, kDT, 0, s>>>(x, y, L, part);
    k_dot_fin<<<1, kDT, 0, s>>>(part, nblk, out, take_sqrt);
    return cudaGetLastError();
}

cudaError_t launch_axpy_dev(float* y, const float* x, const double* coef, float sign, long long L, int nblk,
                            cudaStream_t s) {
    k_axpy_dev<<<nblk, kDT, 0, s>>>(y, x, coef, sign, L);
    return cudaGetLastError();
}

cudaError_t launch_scale_dev(float* y, const float* x, const double* nrm, long long L, int nblk, cudaStream_t s) {
    k_scale_dev<<<nblk, kDT, 0, s>>>(y, x, nrm, L);
    return cudaGetLastError();
}

cudaError_t launch_comb(const float* a, const float* b, const float* c, float* out, long long L, int nblk,
                        cudaStream_t s) {
    k_comb<<<nblk, kDT, 0, s>>>(a, b, c, out, L);
    return cudaGetLastError();
}

cudaError_t launch_lap_dinv19(const DsaArgs& a, const Dsa19& b, float* dinv, int nblk, cudaStream_t s) {
    k_lap_dinv19<<<nblk, kDT, 0, s>>>(a, b, dinv);
    return cudaGetLastError();
}

cudaError_t launch_cg_start19(const DsaArgs& a, const Dsa19& b, const float* v, const float* dinv, float* eps,
                              float* r, float* zc, float* p, int nblk, double* part, CgScalars* cs, cudaStream_t s) {
    k_cg_start19<<<nblk, kDT, 0, s>>>(a, b, v, dinv, eps, r, zc, p, part);
    k_cg_fin<CG_START><<<1, kDT, 0, s>>>(part, nblk, cs);
    return cudaGetLastError();
}

cudaError_t launch_cg_iter19(const DsaArgs& a, const Dsa19& b, const float* dinv, float* eps, float* r, float* zc,
                             float* p, float* q, int nblk, double* part, CgScalars* cs, cudaStream_t s) {
    k_cg_lap19<<<nblk, kDT, 0, s>>>(a, b, p, q, part, cs);
    k_cg_fin<CG_ALPHA><<<1, kDT, 0, s>>>(part, nblk, cs);
    k_cg_update<<<nblk, kDT, 0, s>>>(a.N, p, q, dinv, eps, r, zc, part, cs);
    k_cg_fin<CG_BETA><<<1, kDT, 0, s>>>(part, nblk, cs);
    k_cg_p<<<nblk, kDT, 0, s>>>(a.N, zc, p, cs);
    return cudaGetLastError();
}

cudaError_t launch_prec_out19(long long N, const float* v, const float* eps, float* zout, int nblk, cudaStream_t s) {
    k_prec_out19<<<nblk, kDT, 0, s>>>(N, v, eps, zout);
    return cudaGetLastError();
}

}  // namespace cl
