// Vector kernels of the Krylov steady solve (BiCGSTAB on the fixed-point
// equation of the step map).
//
// The steady state the paper's solver marches to (Sec. 3, Eq. 21-24 run
// until the fields stop changing) is the fixed point x = S(x) of one step of
// the scheme on the stored post-collision populations.  S is affine:
// S(x) = A x + b, where A is the step with zero boundary concentrations and
// b carries the Dirichlet terms.  So the steady state solves (I - A) x = b,
// and the residual of an iterate is r = b - (I - A) x = S(x) - x, the change
// one more step would make.  BiCGSTAB (van der Vorst 1992) solves it with
// two applications of A per iteration; A is the step kernel of the lattice
// itself, launched with zero boundary concentrations.
//
// The vectors are flat f32 arrays of the population layout (every entry of
// an inactive cell or a row pad stays 0, because every vector starts at 0
// there and the step writes zeros there).  Dot products accumulate in FP64:
// per-block partial sums in a fixed order, then one block sums the partials
// in a fixed order, so a solve is reproducible run to run.  The scalars of
// the method live in device memory; a flag set on breakdown makes the later
// kernels of the iteration return without touching the vectors, so the host
// reads the scalars only once per batch of iterations.
#include "internal.cuh"
#include "device_util.cuh"

namespace cl {

namespace {

constexpr int kKryThreads = 256;

__device__ __forceinline__ float4 ld4(const float* p, long long i) { return reinterpret_cast<const float4*>(p)[i]; }
__device__ __forceinline__ void st4(float* p, long long i, float4 v) { reinterpret_cast<float4*>(p)[i] = v; }

// r = c + S(x) - x (c nullable); rh = p = r; partial r.r
__global__ void __launch_bounds__(kKryThreads) k_kry_start(const float* __restrict__ x, const float* __restrict__ sx,
                                                            const float* __restrict__ c, float* __restrict__ r,
                                                            float* __restrict__ rh, float* __restrict__ p,
                                                            long long n4, long long L, double* __restrict__ part) {
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 a = ld4(sx, i);
        const float4 b = ld4(x, i);
        if (c) {
            const float4 e = ld4(c, i);
            a = make_float4(a.x + e.x, a.y + e.y, a.z + e.z, a.w + e.w);
        }
        const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        st4(r, i, d);
        st4(rh, i, d);
        st4(p, i, d);
        acc[0] += (double)d.x * d.x + (double)d.y * d.y + (double)d.z * d.z + (double)d.w * d.w;
    }
    if (blockIdx.x == 0 && threadIdx.x < L - 4 * n4) {
        const long long j = 4 * n4 + threadIdx.x;
        const float d = (c ? c[j] + sx[j] : sx[j]) - x[j];
        r[j] = d;
        rh[j] = d;
        p[j] = d;
        acc[0] += (double)d * d;
    }
    block_sum_store<1>(acc, part + 2 * blockIdx.x);
}

// v = p - A p (Ap in ap); partial rh.v
__global__ void __launch_bounds__(kKryThreads) k_kry_v(const float* __restrict__ p, const float* __restrict__ ap,
                                                        const float* __restrict__ rh, float* __restrict__ v,
                                                        long long n4, long long L, double* __restrict__ part,
                                                        const KryScalars* __restrict__ ks) {
    if (ks->bad) return;
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 a = ld4(p, i), b = ld4(ap, i), h = ld4(rh, i);
        const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        st4(v, i, d);
        acc[0] += (double)h.x * d.x + (double)h.y * d.y + (double)h.z * d.z + (double)h.w * d.w;
    }
    if (blockIdx.x == 0 && threadIdx.x < L - 4 * n4) {
        const long long j = 4 * n4 + threadIdx.x;
        const float d = p[j] - ap[j];
        v[j] = d;
        acc[0] += (double)rh[j] * d;
    }
    block_sum_store<1>(acc, part + 2 * blockIdx.x);
}

// s = r - alpha v
__global__ void __launch_bounds__(kKryThreads) k_kry_s(const float* __restrict__ r, const float* __restrict__ v,
                                                        float* __restrict__ s, long long n4, long long L,
                                                        const KryScalars* __restrict__ ks) {
    if (ks->bad) return;
    const float al = (float)ks->alpha;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 a = ld4(r, i), b = ld4(v, i);
        st4(s, i, make_float4(fmaf(-al, b.x, a.x), fmaf(-al, b.y, a.y), fmaf(-al, b.z, a.z), fmaf(-al, b.w, a.w)));
    }
    if (blockIdx.x == 0 && threadIdx.x < L - 4 * n4) {
        const long long j = 4 * n4 + threadIdx.x;
        s[j] = fmaf(-al, v[j], r[j]);
    }
}

// t = s - A s (As in as_); partials t.s, t.t
__global__ void __launch_bounds__(kKryThreads) k_kry_t(const float* __restrict__ s, const float* __restrict__ as_,
                                                        float* __restrict__ t, long long n4, long long L,
                                                        double* __restrict__ part, const KryScalars* __restrict__ ks) {
    if (ks->bad) return;
    double acc[2] = {0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 a = ld4(s, i), b = ld4(as_, i);
        const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        st4(t, i, d);
        acc[0] += (double)d.x * a.x + (double)d.y * a.y + (double)d.z * a.z + (double)d.w * a.w;
        acc[1] += (double)d.x * d.x + (double)d.y * d.y + (double)d.z * d.z + (double)d.w * d.w;
    }
    if (blockIdx.x == 0 && threadIdx.x < L - 4 * n4) {
        const long long j = 4 * n4 + threadIdx.x;
        const float d = s[j] - as_[j];
        t[j] = d;
        acc[0] += (double)d * s[j];
        acc[1] += (double)d * d;
    }
    block_sum_store<2>(acc, part + 2 * blockIdx.x);
}

// x += alpha p + omega s; r = s - omega t; partials rh.r, r.r
__global__ void __launch_bounds__(kKryThreads) k_kry_xr(float* __restrict__ x, const float* __restrict__ p,
                                                         const float* __restrict__ s, const float* __restrict__ t,
                                                         const float* __restrict__ rh, float* __restrict__ r,
                                                         long long n4, long long L, double* __restrict__ part,
                                                         const KryScalars* __restrict__ ks) {
    if (ks->bad) return;
    const float al = (float)ks->alpha, om = (float)ks->omega;
    double acc[2] = {0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 xv = ld4(x, i);
        const float4 pv = ld4(p, i), sv = ld4(s, i), tv = ld4(t, i), h = ld4(rh, i);
        xv.x = fmaf(om, sv.x, fmaf(al, pv.x, xv.x));
        xv.y = fmaf(om, sv.y, fmaf(al, pv.y, xv.y));
        xv.z = fmaf(om, sv.z, fmaf(al, pv.z, xv.z));
        xv.w = fmaf(om, sv.w, fmaf(al, pv.w, xv.w));
        st4(x, i, xv);
        const float4 rv = make_float4(fmaf(-om, tv.x, sv.x), fmaf(-om, tv.y, sv.y), fmaf(-om, tv.z, sv.z),
                                      fmaf(-om, tv.w, sv.w));
        st4(r, i, rv);
        acc[0] += (double)h.x * rv.x + (double)h.y * rv.y + (double)h.z * rv.z + (double)h.w * rv.w;
        acc[1] += (double)rv.x * rv.x + (double)rv.y * rv.y + (double)rv.z * rv.z + (double)rv.w * rv.w;
    }
    if (blockIdx.x == 0 && threadIdx.x < L - 4 * n4) {
        const long long j = 4 * n4 + threadIdx.x;
        x[j] = fmaf(om, s[j], fmaf(al, p[j], x[j]));
        const float rj = fmaf(-om, t[j], s[j]);
        r[j] = rj;
        acc[0] += (double)rh[j] * rj;
        acc[1] += (double)rj * rj;
    }
    block_sum_store<2>(acc, part + 2 * blockIdx.x);
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(kKryThreads) k_kry_p(const float* __restrict__ r, const float* __restrict__ v,
                                                        float* __restrict__ p, long long n4, long long L,
                                                        const KryScalars* __restrict__ ks) {
    if (ks->bad) return;
    const float be = (float)ks->beta, om = (float)ks->omega;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 rv = ld4(r, i), vv = ld4(v, i);
        float4 pv = ld4(p, i);
        pv.x = fmaf(be, fmaf(-om, vv.x, pv.x), rv.x);
        pv.y = fmaf(be, fmaf(-om, vv.y, pv.y), rv.y);
        pv.z = fmaf(be, fmaf(-om, vv.z, pv.z), rv.z);
        pv.w = fmaf(be, fmaf(-om, vv.w, pv.w), rv.w);
        st4(p, i, pv);
    }
    if (blockIdx.x == 0 && threadIdx.x < L - 4 * n4) {
        const long long j = 4 * n4 + threadIdx.x;
        p[j] = fmaf(be, fmaf(-om, v[j], p[j]), r[j]);
    }
}

// One block: sum the per-block partials in a fixed order, then update the
// scalars of the method (thread 0).
template <int WHICH>
__global__ void __launch_bounds__(kKryThreads) k_kry_fin(const double* __restrict__ part, int nblk,
                                                          KryScalars* __restrict__ ks) {
    if (WHICH != KRY_START && ks->bad) return;
    double acc[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        acc[0] += part[2 * b];
        if (WHICH == KRY_OMEGA || WHICH == KRY_BETA) acc[1] += part[2 * b + 1];
    }
    __shared__ double tot[2];
    block_sum_store<2>(acc, tot);
    if (threadIdx.x != 0) return;
    const double t0 = tot[0], t1 = tot[1];
    if (WHICH == KRY_START) {
        // true residual of the current iterate; bad 2: nothing left to solve
        ks->rr = t0;
        ks->rho = t0;
        ks->alpha = ks->omega = ks->beta = 0.0;
        ks->bad = isfinite(t0) ? (t0 > 0.0 ? 0 : 2) : 1;
    } else if (WHICH == KRY_ALPHA) {
        const double al = ks->rho / t0;
        if (t0 != 0.0 && isfinite(al)) ks->alpha = al;
        else ks->bad = 1;
    } else if (WHICH == KRY_OMEGA) {
        // t.t = 0 means s = 0: the half step already solved the system
        const double om = t1 > 0.0 ? t0 / t1 : 0.0;
        if (isfinite(om)) ks->omega = om;
        else ks->bad = 1;
    } else {
        // t0 = rh.r (new rho), t1 = r.r
        ks->rr = t1;
        ks->iters += 1;
        const double be = (t0 / ks->rho) * (ks->alpha / ks->omega);
        if (!isfinite(t1)) ks->bad = 1;
        else if (t1 == 0.0 || ks->omega == 0.0) ks->bad = 2;
        else if (t0 == 0.0 || !isfinite(be)) ks->bad = 1;
        else {
            ks->beta = be;
            ks->rho = t0;
        }
    }
}

// ---- mixed precision: the iterate in FP64, corrections in FP32
__global__ void k_kry_to64(const float* __restrict__ a, double* __restrict__ b, long long L) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void k_kry_to32(const double* __restrict__ a, float* __restrict__ b, long long L) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

__global__ void k_kry_add64(double* __restrict__ x, const float* __restrict__ e, double sign, long long L) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x)
        x[i] += sign * (double)e[i];
}

// c = S(x) - x in FP64 (sx = S(x)), stored as f32; partial |S(x) - x|^2 in FP64
__global__ void __launch_bounds__(kKryThreads) k_kry_res64(const double* __restrict__ x, const double* __restrict__ sx,
                                                            float* __restrict__ c, long long L,
                                                            double* __restrict__ part) {
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x) {
        const double d = sx[i] - x[i];
        c[i] = (float)d;
        acc[0] += d * d;
    }
    block_sum_store<1>(acc, part + 2 * blockIdx.x);
}

}  // namespace

int kry_blocks() {
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return 4 * nsm;
}

cudaError_t launch_kry_start(const float* x, const float* sx, const float* c, float* r, float* rh, float* p,
                             long long L, int nblk, double* part, KryScalars* ks, cudaStream_t s) {
    const long long n4 = L / 4;
    k_kry_start<<<nblk, kKryThreads, 0, s>>>(x, sx, c, r, rh, p, n4, L, part);
    k_kry_fin<KRY_START><<<1, kKryThreads, 0, s>>>(part, nblk, ks);
    return cudaGetLastError();
}

cudaError_t launch_kry_v(const float* p, const float* ap, const float* rh, float* v, long long L, int nblk,
                         double* part, KryScalars* ks, cudaStream_t s) {
    k_kry_v<<<nblk, kKryThreads, 0, s>>>(p, ap, rh, v, L / 4, L, part, ks);
    k_kry_fin<KRY_ALPHA><<<1, kKryThreads, 0, s>>>(part, nblk, ks);
    return cudaGetLastError();
}

cudaError_t launch_kry_s(const float* r, const float* v, float* sv, long long L, int nblk, const KryScalars* ks,
                         cudaStream_t s) {
    k_kry_s<<<nblk, kKryThreads, 0, s>>>(r, v, sv, L / 4, L, ks);
    return cudaGetLastError();
}

cudaError_t launch_kry_t(const float* sv, const float* as_, float* t, long long L, int nblk, double* part,
                         KryScalars* ks, cudaStream_t s) {
    k_kry_t<<<nblk, kKryThreads, 0, s>>>(sv, as_, t, L / 4, L, part, ks);
    k_kry_fin<KRY_OMEGA><<<1, kKryThreads, 0, s>>>(part, nblk, ks);
    return cudaGetLastError();
}

cudaError_t launch_kry_xr(float* x, const float* p, const float* sv, const float* t, const float* rh, float* r,
                          long long L, int nblk, double* part, KryScalars* ks, cudaStream_t s) {
    k_kry_xr<<<nblk, kKryThreads, 0, s>>>(x, p, sv, t, rh, r, L / 4, L, part, ks);
    k_kry_fin<KRY_BETA><<<1, kKryThreads, 0, s>>>(part, nblk, ks);
    return cudaGetLastError();
}

cudaError_t launch_kry_p(const float* r, const float* v, float* p, long long L, int nblk, const KryScalars* ks,
                         cudaStream_t s) {
    k_kry_p<<<nblk, kKryThreads, 0, s>>>(r, v, p, L / 4, L, ks);
    return cudaGetLastError();
}

cudaError_t launch_kry_to64(const float* a, double* b, long long L, int nblk, cudaStream_t s) {
    k_kry_to64<<<nblk, kKryThreads, 0, s>>>(a, b, L);
    return cudaGetLastError();
}

cudaError_t launch_kry_to32(const double* a, float* b, long long L, int nblk, cudaStream_t s) {
    k_kry_to32<<<nblk, kKryThreads, 0, s>>>(a, b, L);
    return cudaGetLastError();
}

cudaError_t launch_kry_add64(double* x, const float* e, double sign, long long L, int nblk, cudaStream_t s) {
    k_kry_add64<<<nblk, kKryThreads, 0, s>>>(x, e, sign, L);
    return cudaGetLastError();
}

cudaError_t launch_kry_res64(const double* x, const double* sx, float* c, long long L, int nblk, double* part,
                             KryScalars* ks, cudaStream_t s) {
    k_kry_res64<<<nblk, kKryThreads, 0, s>>>(x, sx, c, L, part);
    k_kry_fin<KRY_START><<<1, kKryThreads, 0, s>>>(part, nblk, ks);
    return cudaGetLastError();
}

}  // namespace cl
