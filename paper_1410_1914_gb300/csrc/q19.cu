// The paper's own D3Q19 lattice (Eq. 22-24) as a second solver: set-up of
// the link classes, the fused pull-stream + BGK collide step with its fused
// check reduction, and the readouts.  State: 19 f32 post-collision
// populations per cell, structure of arrays with a padded row pitch.
//
// Velocity order (Eq. 22; the public layout of cl_lbm_get_populations):
//   0 rest; 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z;
//   7 (+1,+1,0), 8 (-1,-1,0), 9 (+1,-1,0), 10 (-1,+1,0), 11 (+1,0,+1),
//   12 (-1,0,-1), 13 (+1,0,-1), 14 (-1,0,+1), 15 (0,+1,+1), 16 (0,-1,-1),
//   17 (0,+1,-1), 18 (0,-1,+1).
// Weights (Eq. 23): 1/3 rest, 1/18 axis, 1/36 face diagonal; cs^2 = 1/3.
//
// Link classes of an active cell, per link i toward x + c_i.  The end cell
// of a link that leaves the box through x = 0 or x = L is the mirror image
// (x, y + c_y, z + c_z) of the end plane:
//   wall      end cell inactive: the population comes back (bounce-back),
//             times r = (cs^2 - k) / (cs^2 + k) when the link is reactive;
//   boundary  leaves the box, end cell active: anti-bounce-back
//             -g* + 2 a_i C_bc (Dirichlet) or bounce-back (zero flux);
//   open      otherwise: plain streaming, y and z periodic.
// A link is reactive when its end cell is solid (code 1) and it leaves the
// cell through a catalytic face (one of the faces its non-zero components
// cross that is marked and borders solid).
#include <math.h>

#include "device_util.cuh"
#include "internal.cuh"

namespace cl {

namespace {

__host__ __device__ constexpr int q19_cx(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int q19_cy(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int q19_cz(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
// opposite direction: pairs (1,2), (3,4), ..., (17,18)
__host__ __device__ constexpr int q19_opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float q19_w(int i) {
    return i == 0 ? 1.f / 3.f : (i <= 6 ? 1.f / 18.f : 1.f / 36.f);
}

template <class T>
__host__ __device__ constexpr T q19_wt(int i) {
    return i == 0 ? T(1) / T(3) : (i <= 6 ? T(1) / T(18) : T(1) / T(36));
}

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

}  // namespace

// ----------------------------------------------------------------- set-up
// Link classes into the padded layout: mask bits 0..17 = wall links,
// kQ19HasReact when any link reacts, kQ19Active; react bits 0..17.
__global__ void k_masks19(const uint8_t* __restrict__ phase, const uint8_t* __restrict__ active,
                          const uint8_t* __restrict__ react_in, int rule, int nx, int ny, int nz, int px,
                          uint32_t* __restrict__ mask, uint32_t* __restrict__ react) {
    const long long NP = (long long)px * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < NP;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % px);
        const long long row = p / px;
        const int y = (int)(row % ny), z = (int)(row / ny);
        uint32_t m = 0, rb = 0;
        const long long c = x + (long long)nx * row;
        if (x < nx && active[c]) {
            m = kQ19Active;
            // catalytic faces of this cell (face f toward the axis direction f + 1)
            unsigned cat = 0;
            for (int f = 0; f < 6; ++f) {
                const int fx = x + q19_cx(f + 1);
                if (fx < 0 || fx >= nx) continue;
                const long long n = fx + (long long)nx * (wrap1(y + q19_cy(f + 1), ny) +
                                                          (long long)ny * wrap1(z + q19_cz(f + 1), nz));
                if (phase[n] != 1) continue;
                const bool marked = rule == CL_REACT_ALL_PORE_SOLID ? phase[c] == 0
                                                                    : (react_in && ((react_in[c] >> f) & 1));
                if (marked) cat |= 1u << f;
            }
            for (int i = 1; i < 19; ++i) {
                const int cx = q19_cx(i), cy = q19_cy(i), cz = q19_cz(i);
                int ex = x + cx;
                if (ex < 0 || ex >= nx) ex = x;  // mirror image of the end plane
                const long long e = ex + (long long)nx * (wrap1(y + cy, ny) + (long long)ny * wrap1(z + cz, nz));
                if (active[e]) continue;
                m |= 1u << (i - 1);
                if (phase[e] != 1) continue;
                unsigned crossed = 0;
                if (cx) crossed |= 1u << (cx > 0 ? 0 : 1);
                if (cy) crossed |= 1u << (cy > 0 ? 2 : 3);
                if (cz) crossed |= 1u << (cz > 0 ? 4 : 5);
                if (cat & crossed) rb |= 1u << (i - 1);
            }
            if (rb) m |= kQ19HasReact;
        }
        mask[p] = m;
        react[p] = rb;
    }
}

cudaError_t launch_masks19(const uint8_t* phase, const uint8_t* active, const uint8_t* react_in, int rule,
                           int nx, int ny, int nz, int px, uint32_t* mask, uint32_t* react, cudaStream_t s) {
    k_masks19<<<152 * 8, 256, 0, s>>>(phase, active, react_in, rule, nx, ny, nz, px, mask, react);
    return cudaGetLastError();
}

// omega into the padded layout (0 on padding)
__global__ void k_pad_omega19(const float* __restrict__ omega, int nx, int ny, int nz, int px,
                              float* __restrict__ out) {
    const long long NP = (long long)px * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < NP;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % px);
        out[p] = x < nx ? omega[x + (long long)nx * (p / px)] : 0.f;
    }
}

cudaError_t launch_pad_omega19(const float* omega, int nx, int ny, int nz, int px, float* out, cudaStream_t s) {
    k_pad_omega19<<<152 * 8, 256, 0, s>>>(omega, nx, ny, nz, px, out);
    return cudaGetLastError();
}

// wall and reactive link counts: out[0], out[1]
__global__ void k_linkcount19(const uint32_t* __restrict__ mask, const uint32_t* __restrict__ react,
                              long long NP, double* partials) {
    double v[2] = {0.0, 0.0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < NP;
         p += (long long)gridDim.x * blockDim.x) {
        const uint32_t m = mask[p];
        if (!(m & kQ19Active)) continue;
        v[0] += __popc(m & kQ19LinkBits);
        v[1] += __popc(react[p] & kQ19LinkBits);
    }
    block_sum_store<2>(v, partials + 2LL * blockIdx.x);
}

cudaError_t launch_linkcount19(const uint32_t* mask, const uint32_t* react, long long NP, double* partials,
                               int nblocks, double* out, cudaStream_t s) {
    k_linkcount19<<<nblocks, 256, 0, s>>>(mask, react, NP, partials);
    return launch_finalize(partials, nblocks, 2, out, s);
}

// ------------------------------------------------------------------ state
// Equilibrium a_i C (Eq. 23) from C0 (unpadded, nullable: the linear ramp
// between the half-way faces); Csnap (padded) gets C.
__global__ void k_init19(float* __restrict__ pop, const uint32_t* __restrict__ mask, const float* __restrict__ C0,
                         int nx, int ny, int nz, int px, double c_in, double c_out, float* __restrict__ Csnap) {
    const long long NP = (long long)px * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < NP;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % px);
        const bool act = (mask[p] & kQ19Active) != 0;
        float C = 0.f;
        if (act) C = C0 ? C0[x + (long long)nx * (p / px)] : (float)(c_in + (c_out - c_in) * (x + 0.5) / nx);
#pragma unroll
        for (int i = 0; i < 19; ++i) pop[(long long)i * NP + p] = act ? q19_w(i) * C : 0.f;
        Csnap[p] = C;
    }
}

cudaError_t launch_init19(float* pop, const uint32_t* mask, const float* C0, int nx, int ny, int nz, int px,
                          double c_in, double c_out, float* Csnap, cudaStream_t s) {
    k_init19<<<152 * 8, 256, 0, s>>>(pop, mask, C0, nx, ny, nz, px, c_in, c_out, Csnap);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- step
// One cell per thread, 128 threads along a padded row.  Every population
// arriving at x is pulled from x - c_i (open link), or rebuilt from the
// cell's own post-collision population of the opposite direction (wall or
// boundary link); then C = sum g_i and g*_i = g_i - omega (g_i - a_i C).
// Each link first selects the element to read (the neighbour's population,
// or its own opposite one) and loads it unconditionally, so the 18 loads of
// a cell are independent and all in flight at once; the boundary rules are
// applied to the loaded values afterwards.  Element offsets are 32-bit
// (I = uint32_t) while 19 padded planes fit, 64-bit otherwise.
// Stores: the lanes of a 32-byte sector (8 cells; the pitch is a multiple
// of 32 cells) all store when any of them is active, none otherwise, so
// that no sector is written in part (inactive cells store their zeros).
// T = double is the same step in FP64 arithmetic on FP64 populations (with
// the FP64 weights, boundary values and reactive factor; omega as stored),
// used for the residual of the mixed-precision steady solve.
template <bool REDUCE, class I, class T = float>
__global__ void __launch_bounds__(kQ19Threads) k_step19(const T* __restrict__ src, T* __restrict__ dst,
                                                        Q19Args a) {
    const int x = blockIdx.x * kQ19Threads + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const int nx = a.nx, ny = a.ny, nz = a.nz, px = a.px;
    const I NP = (I)a.NP;
    const I c = (I)x + (I)px * ((I)y + (I)ny * (I)z);
    const bool in_row = x < px;
    const uint32_t m = in_row ? a.mask[c] : 0u;
    const bool act = (m & kQ19Active) != 0;
    constexpr bool kF64 = sizeof(T) == 8;
    T h[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) h[i] = T(0);
    double rv[RED_N];
    if (REDUCE)
#pragma unroll
        for (int k = 0; k < RED_N; ++k) rv[k] = 0.0;
    if (act) {
        const uint32_t rb = (m & kQ19HasReact) ? a.react[c] : 0u;
        // offsets of the rows y -+ 1 and planes z -+ 1 (periodic), relative to c
        const I plane = (I)px * (I)ny;
        const I oym = y == 0 ? (I)(ny - 1) * (I)px : (I)0 - (I)px;  // row y - 1
        const I oyp = y == ny - 1 ? (I)0 - (I)(ny - 1) * (I)px : (I)px;
        const I ozm = z == 0 ? (I)(nz - 1) * plane : (I)0 - plane;
        const I ozp = z == nz - 1 ? (I)0 - (I)(nz - 1) * plane : plane;
        T v[19];
        bool own[19];
        v[0] = src[c];
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int j = q19_opp(i);  // the population arrives through the link toward x + c_j = x - c_i
            const int cx = q19_cx(i), cy = q19_cy(i), cz = q19_cz(i);
            own[i] = ((m >> (j - 1)) & 1u) || (cx > 0 && x == 0) || (cx < 0 && x == nx - 1);
            const I s = c - (I)cx + (cy > 0 ? oym : (cy < 0 ? oyp : (I)0)) + (cz > 0 ? ozm : (cz < 0 ? ozp : (I)0));
            const I e = own[i] ? (I)j * NP + c : (I)i * NP + s;
            v[i] = src[e];
        }
        const T rs = kF64 ? (T)a.rsink_d : (T)a.rsink;  // 1 - r
        const T cin = kF64 ? (T)a.c_in_d : (T)a.c_in, cout = kF64 ? (T)a.c_out_d : (T)a.c_out;
        T g[19];
        g[0] = v[0];
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int j = q19_opp(i);
            const int cx = q19_cx(i);
            const T wi = q19_wt<T>(i);
            T o = v[i];
            if (own[i]) {
                if ((m >> (j - 1)) & 1u) o = ((rb >> (j - 1)) & 1u) ? o - rs * o : o;
                else if (cx > 0) o = a.bc_in == CL_BC_DIRICHLET ? T(2) * wi * cin - o : o;
                else o = a.bc_out == CL_BC_DIRICHLET ? T(2) * wi * cout - o : o;
            }
            g[i] = o;
        }
        // C = sum g_i in a fixed pairwise order
        const T C = (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) +
                        (((g[8] + g[9]) + (g[10] + g[11])) + ((g[12] + g[13]) + (g[14] + g[15]))) +
                        ((g[16] + g[17]) + g[18]);
        const T om = (T)a.omega[c];
#pragma unroll
        for (int i = 0; i < 19; ++i) h[i] = g[i] - om * (g[i] - q19_wt<T>(i) * C);
        if (REDUCE) {
            double jin = 0.0, jout = 0.0, r = 0.0;
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                const bool wall = (m >> (i - 1)) & 1u;
                if (q19_cx(i) < 0 && x == 0 && !wall && a.bc_in == CL_BC_DIRICHLET)
                    jin += 2.0 * ((double)q19_w(i) * a.c_in_d - (double)h[i]);
                if (q19_cx(i) > 0 && x == nx - 1 && !wall && a.bc_out == CL_BC_DIRICHLET)
                    jout += 2.0 * ((double)h[i] - (double)q19_w(i) * a.c_out_d);
                if (rb & (1u << (i - 1))) r += h[i];
            }
            rv[RED_JIN] = jin;
            rv[RED_JOUT] = jout;
            rv[RED_R] = a.rsink_d * r;
            rv[RED_SUMC] = C;
            rv[RED_DC] = fabs((double)C - (double)a.Csnap[c]);
            rv[RED_ABSC] = fabs((double)C);
            rv[RED_NONFINITE] = isfinite(C) ? 0.0 : 1.0;
            a.Csnap[c] = (float)C;
        }
    }
    const unsigned lane = threadIdx.x & 31u;
    const unsigned vote = __ballot_sync(0xffffffffu, act);
    if (in_row && ((vote >> (lane & ~7u)) & 0xFFu)) {
#pragma unroll
        for (int i = 0; i < 19; ++i) dst[(I)i * NP + c] = h[i];
    }
    if (REDUCE) {
        const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        block_sum_store<RED_N>(rv, a.partials + blk * RED_N);
    }
}

dim3 step19_grid(const Q19Args& a) { return dim3((a.px + kQ19Threads - 1) / kQ19Threads, a.ny, a.nz); }

int step19_blocks(const Q19Args& a) {
    const dim3 g = step19_grid(a);
    return (int)(g.x * g.y * g.z);
}

cudaError_t launch_step19(const float* src, float* dst, const Q19Args& a, bool reduce, cudaStream_t s) {
    const dim3 g = step19_grid(a);
    // 32-bit element offsets while every offset into the 19 planes fits
    const bool narrow = !a.wide && 19LL * a.NP < (1LL << 32);
    if (narrow) {
        if (reduce) k_step19<true, uint32_t><<<g, kQ19Threads, 0, s>>>(src, dst, a);
        else k_step19<false, uint32_t><<<g, kQ19Threads, 0, s>>>(src, dst, a);
    } else {
        if (reduce) k_step19<true, unsigned long long><<<g, kQ19Threads, 0, s>>>(src, dst, a);
        else k_step19<false, unsigned long long><<<g, kQ19Threads, 0, s>>>(src, dst, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_step19_f64(const double* src, double* dst, const Q19Args& a, cudaStream_t s) {
    const dim3 g = step19_grid(a);
    if (!a.wide && 19LL * a.NP < (1LL << 32)) k_step19<false, uint32_t, double><<<g, kQ19Threads, 0, s>>>(src, dst, a);
    else k_step19<false, unsigned long long, double><<<g, kQ19Threads, 0, s>>>(src, dst, a);
    return cudaGetLastError();
}

// --------------------------------------------------------------- readouts
// Per x-plane from the stored post-collision populations, one block per
// plane: out[5*x + k] = sum C, active count, R, J_in part, J_out part.
__global__ void k_readout19(const float* __restrict__ pop, Q19Args a, double* out) {
    const int x = blockIdx.x;
    const long long nyz = (long long)a.ny * a.nz;
    double v[5] = {0, 0, 0, 0, 0};
    const double sink = a.rsink_d;
    for (long long j = threadIdx.x; j < nyz; j += blockDim.x) {
        const long long c = x + (long long)a.px * j;
        const uint32_t m = a.mask[c];
        if (!(m & kQ19Active)) continue;
        const uint32_t rb = (m & kQ19HasReact) ? a.react[c] : 0u;
        float h[19];
        double C = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) { h[i] = pop[(long long)i * a.NP + c]; C += (double)h[i]; }
        v[0] += C;
        v[1] += 1.0;
        double r = 0.0;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const bool wall = (m >> (i - 1)) & 1u;
            if (rb & (1u << (i - 1))) r += h[i];
            if (q19_cx(i) < 0 && x == 0 && !wall && a.bc_in == CL_BC_DIRICHLET)
                v[3] += 2.0 * ((double)q19_w(i) * a.c_in_d - (double)h[i]);
            if (q19_cx(i) > 0 && x == a.nx - 1 && !wall && a.bc_out == CL_BC_DIRICHLET)
                v[4] += 2.0 * ((double)h[i] - (double)q19_w(i) * a.c_out_d);
        }
        v[2] += sink * r;
    }
    block_sum_store<5>(v, out + 5LL * x);
}

cudaError_t launch_readout19(const float* pop, const Q19Args& a, double* out, cudaStream_t s) {
    k_readout19<<<a.nx, 256, 0, s>>>(pop, a, out);
    return cudaGetLastError();
}

// C (unpadded, 0 on inactive cells) and/or the populations as [19][nz][ny][nx]
__global__ void k_out19(const float* __restrict__ pop, const uint32_t* __restrict__ mask, int nx, int ny, int nz,
                        int px, float* __restrict__ C, float* __restrict__ g) {
    const long long N = (long long)nx * ny * nz, NP = (long long)px * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const long long p = (c % nx) + (long long)px * (c / nx);
        const bool act = (mask[p] & kQ19Active) != 0;
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float v = act ? pop[(long long)i * NP + p] : 0.f;
            s += v;
            if (g) g[(long long)i * N + c] = v;
        }
        if (C) C[c] = s;
    }
}

cudaError_t launch_out19(const float* pop, const uint32_t* mask, int nx, int ny, int nz, int px, float* C, float* g,
                         cudaStream_t s) {
    k_out19<<<152 * 8, 256, 0, s>>>(pop, mask, nx, ny, nz, px, C, g);
    return cudaGetLastError();
}

// Link classes as public bit sets (unpadded): wall and reactive links,
// bit i-1 for the link toward x + c_i.  q19: from the D3Q19 masks; else
// from the D3Q7 face mask (closed faces minus the x faces of the box,
// which are boundary links on that lattice).
__global__ void k_links_out(const uint32_t* __restrict__ mask19, const uint32_t* __restrict__ react19,
                            const uint16_t* __restrict__ mask7, int nx, int ny, int nz, int px,
                            uint32_t* __restrict__ wall, uint32_t* __restrict__ react) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        uint32_t w = 0, r = 0;
        if (mask19) {
            const long long p = x + (long long)px * (c / nx);
            w = mask19[p] & kQ19LinkBits;
            r = react19[p] & kQ19LinkBits;
        } else {
            const uint16_t m = mask7[c];
            w = (m >> kClosedShift) & 0x3Fu;
            if (x == 0) w &= ~2u;
            if (x == nx - 1) w &= ~1u;
            r = (m >> kReactShift) & 0x3Fu;
        }
        if (wall) wall[c] = w;
        if (react) react[c] = r;
    }
}

cudaError_t launch_links_out(const uint32_t* mask19, const uint32_t* react19, const uint16_t* mask7, int nx, int ny,
                             int nz, int px, uint32_t* wall, uint32_t* react, cudaStream_t s) {
    k_links_out<<<152 * 8, 256, 0, s>>>(mask19, react19, mask7, nx, ny, nz, px, wall, react);
    return cudaGetLastError();
}

}  // namespace cl
