// D3Q19 (Eq. 22-24) on the (C, delta) state: the same pull-stream + BGK step
// as q19.cu, written on small quantities so that FP32 (or FP16) storage
// keeps the steady state to the FP64 answer.
//
// State per active cell after a step (post-collision, Eq. 21 with the
// equilibrium a_i C of Eq. 23):
//     g*_i = a_i C + delta_i,   i = 1..18,   delta_0 = -(delta_1 + ... + delta_18)
// C is an unevaluated sum hi + lo of two floats, stored side by side (one
// 8-byte load per source cell); the deviations are f32 (or f16 scaled by
// s_d).  With e_i
// the arriving population minus a_i C(x):
//     open link:   e_i = a_i (C(x - c_i) - C(x)) + delta_i(x - c_i)
//     wall:        e_i = r delta_opp(x) - (1 - r) a_i C(x)   (r = 1 unless reactive)
//     Dirichlet:   e_i = 2 a_i (C_bc - C(x)) - delta_opp(x)   (anti-bounce-back)
//     zero flux:   e_i = delta_opp(x)
//     dC = sum_i e_i + delta_0(x),  C' = C + dC (double-float),
//     delta'_i = (1 - omega) (e_i - a_i dC)
// which is the BGK step rewritten exactly; delta_0 is implied, so the mass
// of a cell is exact by construction.  Link classes, layout and store
// sectors as in q19.cu; each link loads (hi, lo) and delta of the cell its
// population comes from (its own cell for wall and boundary links)
// unconditionally, so a cell's loads are all in flight together.
#include <cuda_fp16.h>
#include <math.h>

#include "device_util.cuh"
#include "internal.cuh"

namespace cl {

namespace {

__host__ __device__ constexpr int s19_cx(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int s19_cy(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int s19_cz(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int s19_opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float s19_w(int i) {
    return i == 0 ? 1.f / 3.f : (i <= 6 ? 1.f / 18.f : 1.f / 36.f);
}

struct SF32 {
    using T = float;
    static __device__ __forceinline__ float ld(T v) { return v; }
    static __device__ __forceinline__ T st(float v) { return v; }
};
struct SF16 {
    using T = __half;
    static __device__ __forceinline__ float ld(T v) { return __half2float(v); }
    static __device__ __forceinline__ T st(float v) { return __float2half_rn(v); }
};

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum19(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) + d, renormalised
__device__ __forceinline__ void df_add19(float hi, float lo, float d, float& ho, float& lo_out) {
    float s, e;
    two_sum19(hi, d, s, e);
    e += lo;
    ho = s + e;
    lo_out = e - (ho - s);
}

}  // namespace

// ------------------------------------------------------------------- step
// A block is a 32 x 4 tile of cells (x, y) of one plane: a warp is one row,
// and the y-neighbour rows a cell reads are mostly the block's own rows,
// already in L1.  Deviations stay in storage units inside the update
// (scaled by s_d, 1 for FP32), so nothing is rescaled on its way in or out.
constexpr int kS19X = 32, kS19Y = 4;

template <class S, bool REDUCE, class I>
__global__ void __launch_bounds__(kS19X * kS19Y) k_step19s(Q19State src, Q19State dst, Q19Args a) {
    using T = typename S::T;
    constexpr bool HALF = sizeof(T) == 2;
    const int x = blockIdx.x * kS19X + threadIdx.x;
    const int y = blockIdx.y * kS19Y + threadIdx.y, z = blockIdx.z;
    const int nx = a.nx, ny = a.ny, nz = a.nz, px = a.px;
    const I NP = (I)a.NP;
    const I c = (I)x + (I)px * ((I)y + (I)ny * (I)z);
    const bool in_row = x < px && y < ny;
    const uint32_t m = in_row ? a.mask[c] : 0u;
    const bool act = (m & kQ19Active) != 0;
    const float s_d = HALF ? a.s_d : 1.f, inv_d = HALF ? a.inv_d : 1.f;
    const float2* __restrict__ shl = src.hl;
    const T* __restrict__ sd = reinterpret_cast<const T*>(src.d);
    float hnew = 0.f, lnew = 0.f;
    float dn[18];
#pragma unroll
    for (int i = 0; i < 18; ++i) dn[i] = 0.f;
    double rv[RED_N];
    if (REDUCE)
#pragma unroll
        for (int k = 0; k < RED_N; ++k) rv[k] = 0.0;
    if (act) {
        const uint32_t rb = (m & kQ19HasReact) ? a.react[c] : 0u;
        const I plane = (I)px * (I)ny;
        const I oym = y == 0 ? (I)(ny - 1) * (I)px : (I)0 - (I)px;
        const I oyp = y == ny - 1 ? (I)0 - (I)(ny - 1) * (I)px : (I)px;
        const I ozm = z == 0 ? (I)(nz - 1) * plane : (I)0 - plane;
        const I ozp = z == nz - 1 ? (I)0 - (I)(nz - 1) * plane : plane;
        const float2 own_hl = shl[c];
        const float hx = own_hl.x, lx = own_hl.y;
        const float Cx = hx + lx;
        const float rs = a.rsink;  // 1 - r
        // own deviations: their sum is -delta_0
        float sdd = 0.f;
#pragma unroll
        for (int i = 0; i < 18; ++i) sdd += S::ld(sd[(I)i * NP + c]);
        // per link: (hi, lo, delta) of the cell the population comes from, then e_i
        float ev[18];
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int j = s19_opp(i);
            const int cx = s19_cx(i), cy = s19_cy(i), cz = s19_cz(i);
            const bool wall = (m >> (j - 1)) & 1u;
            const bool own = wall || (cx > 0 && x == 0) || (cx < 0 && x == nx - 1);
            const I s = c - (I)cx + (cy > 0 ? oym : (cy < 0 ? oyp : (I)0)) + (cz > 0 ? ozm : (cz < 0 ? ozp : (I)0));
            const I e = own ? c : s;
            const float2 nhl = shl[e];
            const float nd = S::ld(sd[(I)((own ? j : i) - 1) * NP + e]);
            const float ws = s19_w(i) * s_d;
            // open link; for an own link (hi, lo) are the cell's own and nd = delta_opp: the inert wall value
            float ei = ws * ((nhl.x - hx) + (nhl.y - lx)) + nd;
            if (own) {
                if (wall) {
                    if ((rb >> (j - 1)) & 1u) ei = fmaf(-rs, nd + ws * Cx, nd);
                } else if (cx > 0) {
                    if (a.bc_in == CL_BC_DIRICHLET) ei = 2.0f * ws * ((a.c_in - hx) - lx) - nd;
                } else {
                    if (a.bc_out == CL_BC_DIRICHLET) ei = 2.0f * ws * ((a.c_out - hx) - lx) - nd;
                }
            }
            ev[i - 1] = ei;
        }
        float se = 0.f;
#pragma unroll
        for (int i = 0; i < 18; ++i) se += ev[i];
        const float dCs = se - sdd;  // sum e_i + delta_0, storage units
        df_add19(hx, lx, dCs * inv_d, hnew, lnew);
        const float om1 = 1.0f - a.omega[c];
#pragma unroll
        for (int i = 1; i < 19; ++i) dn[i - 1] = om1 * (ev[i - 1] - s19_w(i) * dCs);
        if (REDUCE) {
            const double id = inv_d;
            const double Cn = (double)hnew + (double)lnew;
            double jin = 0.0, jout = 0.0, r = 0.0;
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                const bool wall = (m >> (i - 1)) & 1u;
                const double gs = (double)s19_w(i) * Cn + (double)dn[i - 1] * id;  // g*_i
                if (s19_cx(i) < 0 && x == 0 && !wall && a.bc_in == CL_BC_DIRICHLET)
                    jin += 2.0 * ((double)s19_w(i) * a.c_in_d - gs);
                if (s19_cx(i) > 0 && x == nx - 1 && !wall && a.bc_out == CL_BC_DIRICHLET)
                    jout += 2.0 * (gs - (double)s19_w(i) * a.c_out_d);
                if (rb & (1u << (i - 1))) r += gs;
            }
            rv[RED_JIN] = jin;
            rv[RED_JOUT] = jout;
            rv[RED_R] = a.rsink_d * r;
            const float Cf = hnew + lnew;
            rv[RED_SUMC] = Cf;
            rv[RED_DC] = fabs((double)Cf - (double)a.Csnap[c]);
            rv[RED_ABSC] = fabs((double)Cf);
            rv[RED_NONFINITE] = isfinite(hnew) ? 0.0 : 1.0;
            a.Csnap[c] = Cf;
        }
    }
    const unsigned lane = threadIdx.x;  // blockDim.x = 32: the lane
    const unsigned vote = __ballot_sync(0xffffffffu, act);
    if (in_row && ((vote >> (lane & ~7u)) & 0xFFu)) {
        T* ddv = reinterpret_cast<T*>(dst.d);
        dst.hl[c] = make_float2(hnew, lnew);
#pragma unroll
        for (int i = 0; i < 18; ++i) ddv[(I)i * NP + c] = S::st(dn[i]);
    }
    if (REDUCE) {
        const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        block_sum_store<RED_N>(rv, a.partials + blk * RED_N);
    }
}

// ----------------------------------------------------------- init / readout
// C0 (unpadded, nullable: the linear ramp) into (hi, lo), deviations 0.
template <class S>
__global__ void k_init19s(Q19State st, Q19Args a, const float* __restrict__ C0) {
    using T = typename S::T;
    const long long NP = a.NP;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < NP;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % a.px);
        float hi = 0.f, lo = 0.f;
        if (a.mask[p] & kQ19Active) {
            const double C = C0 ? (double)C0[x + (long long)a.nx * (p / a.px)]
                                : a.c_in_d + (a.c_out_d - a.c_in_d) * (x + 0.5) / a.nx;
            hi = (float)C;
            lo = (float)(C - (double)hi);
        }
        st.hl[p] = make_float2(hi, lo);
        for (int i = 0; i < 18; ++i) reinterpret_cast<T*>(st.d)[i * NP + p] = S::st(0.f);
        a.Csnap[p] = hi + lo;
    }
}

// C = hi + lo and g*_i = a_i C + delta_i of one padded cell
template <class S>
__device__ __forceinline__ double state_cell(const Q19State& st, const Q19Args& a, long long p, float (&g)[19]) {
    using T = typename S::T;
    constexpr bool HALF = sizeof(T) == 2;
    const double C = (double)st.hl[p].x + (double)st.hl[p].y;
    float s = 0.f;
    for (int i = 1; i < 19; ++i) {
        const float d = S::ld(reinterpret_cast<const T*>(st.d)[(i - 1) * a.NP + p]) * (HALF ? a.inv_d : 1.f);
        g[i] = (float)((double)s19_w(i) * C + (double)d);
        s += d;
    }
    g[0] = (float)((double)s19_w(0) * C - (double)s);
    return C;
}

// per x-plane: out[5*x + k] = sum C, active count, R, J_in part, J_out part
template <class S>
__global__ void k_readout19s(Q19State st, Q19Args a, double* out) {
    const int x = blockIdx.x;
    const long long nyz = (long long)a.ny * a.nz;
    double v[5] = {0, 0, 0, 0, 0};
    const double sink = a.rsink_d;
    for (long long j = threadIdx.x; j < nyz; j += blockDim.x) {
        const long long p = x + (long long)a.px * j;
        const uint32_t m = a.mask[p];
        if (!(m & kQ19Active)) continue;
        const uint32_t rb = (m & kQ19HasReact) ? a.react[p] : 0u;
        float g[19];
        const double C = state_cell<S>(st, a, p, g);
        v[0] += C;
        v[1] += 1.0;
        double r = 0.0;
        for (int i = 1; i < 19; ++i) {
            const bool wall = (m >> (i - 1)) & 1u;
            const double gs = (double)s19_w(i) * C +
                              (double)S::ld(reinterpret_cast<const typename S::T*>(st.d)[(i - 1) * a.NP + p]) *
                                  (sizeof(typename S::T) == 2 ? (double)a.inv_d : 1.0);
            if (rb & (1u << (i - 1))) r += gs;
            if (s19_cx(i) < 0 && x == 0 && !wall && a.bc_in == CL_BC_DIRICHLET)
                v[3] += 2.0 * ((double)s19_w(i) * a.c_in_d - gs);
            if (s19_cx(i) > 0 && x == a.nx - 1 && !wall && a.bc_out == CL_BC_DIRICHLET)
                v[4] += 2.0 * (gs - (double)s19_w(i) * a.c_out_d);
        }
        v[2] += sink * r;
    }
    block_sum_store<5>(v, out + 5LL * x);
}

// unpadded C and/or g* as [19][nz][ny][nx]
template <class S>
__global__ void k_out19s(Q19State st, Q19Args a, float* __restrict__ C, float* __restrict__ gout) {
    const long long N = (long long)a.nx * a.ny * a.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const long long p = (c % a.nx) + (long long)a.px * (c / a.nx);
        const bool act = (a.mask[p] & kQ19Active) != 0;
        float g[19];
        double Cv = 0.0;
        if (act) Cv = state_cell<S>(st, a, p, g);
        else
            for (int i = 0; i < 19; ++i) g[i] = 0.f;
        if (C) C[c] = (float)Cv;
        if (gout)
            for (int i = 0; i < 19; ++i) gout[i * N + c] = g[i];
    }
}

// -------------------------------------------------------------- launchers
cudaError_t launch_step19s(int storage, const Q19State& src, const Q19State& dst, const Q19Args& a, bool reduce,
                           cudaStream_t s) {
    const dim3 g((a.px + kS19X - 1) / kS19X, (a.ny + kS19Y - 1) / kS19Y, a.nz);
    const dim3 b(kS19X, kS19Y);
    const bool narrow = !a.wide && 19LL * a.NP < (1LL << 32);
#define CL_Q19S(SS, R, II) k_step19s<SS, R, II><<<g, b, 0, s>>>(src, dst, a)
    if (storage == CL_STORE_FP16DEV) {
        if (narrow) { if (reduce) CL_Q19S(SF16, true, uint32_t); else CL_Q19S(SF16, false, uint32_t); }
        else { if (reduce) CL_Q19S(SF16, true, unsigned long long); else CL_Q19S(SF16, false, unsigned long long); }
    } else {
        if (narrow) { if (reduce) CL_Q19S(SF32, true, uint32_t); else CL_Q19S(SF32, false, uint32_t); }
        else { if (reduce) CL_Q19S(SF32, true, unsigned long long); else CL_Q19S(SF32, false, unsigned long long); }
    }
#undef CL_Q19S
    return cudaGetLastError();
}

int step19s_blocks(int px, int ny, int nz) {
    return ((px + kS19X - 1) / kS19X) * ((ny + kS19Y - 1) / kS19Y) * nz;
}

cudaError_t launch_init19s(int storage, const Q19State& st, const Q19Args& a, const float* C0, cudaStream_t s) {
    if (storage == CL_STORE_FP16DEV) k_init19s<SF16><<<152 * 8, 256, 0, s>>>(st, a, C0);
    else k_init19s<SF32><<<152 * 8, 256, 0, s>>>(st, a, C0);
    return cudaGetLastError();
}

cudaError_t launch_readout19s(int storage, const Q19State& st, const Q19Args& a, double* out, cudaStream_t s) {
    if (storage == CL_STORE_FP16DEV) k_readout19s<SF16><<<a.nx, 256, 0, s>>>(st, a, out);
    else k_readout19s<SF32><<<a.nx, 256, 0, s>>>(st, a, out);
    return cudaGetLastError();
}

cudaError_t launch_out19s(int storage, const Q19State& st, const Q19Args& a, float* C, float* g, cudaStream_t s) {
    if (storage == CL_STORE_FP16DEV) k_out19s<SF16><<<152 * 8, 256, 0, s>>>(st, a, C, g);
    else k_out19s<SF32><<<152 * 8, 256, 0, s>>>(st, a, C, g);
    return cudaGetLastError();
}

}  // namespace cl
