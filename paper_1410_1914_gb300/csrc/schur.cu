// Steady state of the D3Q7 scheme as a fixed point in C alone.
//
// At steady state every population obeys, along the line of its own axis,
//     g_i(x + c_i) = g*_i(x) = (1 - omega_x) g_i(x) + omega_x w C(x) + w S(x)
// (Eq. 21 with the equilibrium w C of Eq. 23 and the a_i S source), and a
// closed face returns the population along the opposite direction (wall:
// times 1 or the catalytic factor r; fixed value: -g* + 2 w C_bc; zero flux:
// g*).  Given C, each run of open faces along an axis is therefore a linear
// two-stream problem with two unknowns (the populations entering its two
// ends), solved exactly by sweeps along the run; a closed loop of y or z
// (no closed face) is a geometric series.  The rest population is
// g_0 = w_0 (C + S / omega).  Summing the incoming populations,
//     C = F(C) = (sum_{i>0} g_i[C] + w_0 S / omega) / (1 - w_0),
// an affine map whose fixed point is exactly the steady state the time
// march approaches; the populations are eliminated without approximation.
//
// (I - M) C = f (M: the linear part of F, f = F(0)) is solved by flexible
// GMRES in FP64, preconditioned by the cell-centred finite-volume operator
// of the same relaxation times: link conductance 2 D_a D_b / (D_a + D_b)
// with D = (1/omega - 1/2) / 4 (the steady one-dimensional flux of the
// scheme, exact in 1D), 2 D on a fixed-value face, 2 k D / (2 D + k) on a
// catalytic face; its systems are solved by diagonal-preconditioned
// conjugate gradients in FP64.  This reaches the steady state where the
// pore / ionomer contrast of dissolved O2 (relaxation times within 1e-5 of
// 1/2 in the ionomer, Eq. 10-15) makes the march and the population-space
// Krylov solves stall: relaxation times near 1/2 leave the non-equilibrium
// populations almost undamped, which the line sweeps resolve exactly.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "device_util.cuh"
#include "handle.cuh"

using namespace cl;

namespace {

constexpr int kSB = 256;          // threads per block
constexpr int kSBlk = 152 * 4;    // blocks of the cell loops
constexpr double kWa = 0.125;     // D3Q7 axis weight
constexpr double kWr = 0.25;      // D3Q7 rest weight

struct SchurArgs {
    int nx, ny, nz;
    long long N;
    const uint16_t* __restrict__ mask;
    const double* __restrict__ D;       // per-cell diffusivity [m^2/s]
    double dt_cs2dx2;                   // dt / (cs^2 dx^2): tau = 1/2 + D dt / (cs^2 dx^2) (Eq. 24)
    double rfac;                        // uniform catalytic factor
    const double* __restrict__ kscale;  // per-cell factor on k_lu (nullable)
    double k_lu;
    const double* __restrict__ src;     // per-cell source per step (nullable)
    double c_in, c_out;
    int bc_in, bc_out;
    // formed once per call (k_schur_setup): omega in FP64, and the finite-volume
    // operator as the conductances of the +x, +y, +z links and the diagonal (4 N)
    const double* __restrict__ om64;
    const double* __restrict__ G;
};

// relaxation rate in FP64 from the cell's D (Eq. 24), as the FP64 oracle forms it
__device__ __forceinline__ double omega_from_D(const SchurArgs& a, long long c) {
    return 1.0 / (0.5 + a.D[c] * a.dt_cs2dx2);
}
__device__ __forceinline__ double cell_omega(const SchurArgs& a, long long c) { return a.om64[c]; }

__device__ __forceinline__ double cat_factor(const SchurArgs& a, long long c) {
    return a.kscale ? cell_rfac(a.k_lu, a.kscale[c]) : a.rfac;
}

// Returning factor and added amount of the closed face `bit` of cell c on axis ax (dir +1/-1).
__device__ __forceinline__ void end_rule(const SchurArgs& a, int ax, int dir, long long c, int xcoord, bool homog,
                                         double& k, double& h) {
    const uint16_t m = a.mask[c];
    const int bit = 2 * ax + (dir > 0 ? 0 : 1);
    h = 0.0;
    if (ax == 0 && dir < 0 && xcoord == 0) {
        if (a.bc_in == CL_BC_DIRICHLET) { k = -1.0; h = homog ? 0.0 : 2.0 * kWa * a.c_in; }
        else k = 1.0;
        return;
    }
    if (ax == 0 && dir > 0 && xcoord == a.nx - 1) {
        if (a.bc_out == CL_BC_DIRICHLET) { k = -1.0; h = homog ? 0.0 : 2.0 * kWa * a.c_out; }
        else k = 1.0;
        return;
    }
    k = ((m >> (kReactShift + bit)) & 1u) ? cat_factor(a, c) : 1.0;
}

// One thread per line of axis ax: the incoming populations of the two
// directions of that axis from C, added to T; with `pop`, the post-collision
// populations of those directions are written too (f32 state layout).
// With `out3` (three cell fields: consumption on catalytic faces, inflow at
// x = 0, outflow at x = L, lattice units per step) the FP64 fluxes of the
// runs' ends are added there as well.
template <int AX>
__global__ void __launch_bounds__(kSB) k_lines(SchurArgs a, const double* __restrict__ C, double* __restrict__ T,
                                               int homog, float* __restrict__ pop, double* __restrict__ out3) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long nlines = AX == 0 ? (long long)ny * nz : (AX == 1 ? (long long)nx * nz : (long long)nx * ny);
    const int L = AX == 0 ? nx : (AX == 1 ? ny : nz);
    const long long stride = AX == 0 ? 1 : (AX == 1 ? (long long)nx : (long long)nx * ny);
    const bool periodic = AX != 0;
    const int bp = 2 * AX, bm = 2 * AX + 1;  // closed-face bits of the + and - faces
    const int ip = 1 + 2 * AX, im = 2 + 2 * AX;  // population indices of the two directions
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < nlines;
         l += (long long)gridDim.x * blockDim.x) {
        long long base;
        if (AX == 0) base = l * nx;
        else if (AX == 1) base = (l % nx) + (l / nx) * (long long)nx * ny;
        else base = l;
        auto cell = [&](int k) { return base + (long long)k * stride; };
        auto act = [&](int k) { return (a.mask[cell(k)] & kActiveBit) != 0; };
        auto coef = [&](int k, double& dec, double& s) {
            const long long c = cell(k);
            const double om = cell_omega(a, c);
            dec = 1.0 - om;
            s = om * kWa * C[c] + (homog || !a.src ? 0.0 : kWa * a.src[c]);
        };
        // a start: a cell whose - face is closed (the x line always has one at x = 0 if active)
        int k0 = -1;
        for (int k = 0; k < L; ++k)
            if (act(k) && ((a.mask[cell(k)] >> bm) & 1u)) { k0 = k; break; }
        if (k0 < 0) {
            // no closed face: either no active cell, or (y, z) a closed loop of active cells
            if (!periodic || !act(0)) continue;
            for (int dir = 0; dir < 2; ++dir) {
                double al = 1.0, be = 0.0;
                for (int j = 0; j < L; ++j) {
                    const int k = dir == 0 ? j : L - 1 - j;
                    double dec, s;
                    coef(k, dec, s);
                    al = dec * al;
                    be = dec * be + s;
                }
                double g = be / (1.0 - al);
                for (int j = 0; j < L; ++j) {
                    const int k = dir == 0 ? j : L - 1 - j;
                    const long long c = cell(k);
                    double dec, s;
                    coef(k, dec, s);
                    T[c] += g;
                    g = dec * g + s;
                    if (pop) pop[(long long)(dir == 0 ? ip : im) * a.N + c] = (float)g;
                }
            }
            continue;
        }
        // walk the line once from k0 (wrapping for y, z), one run of open faces at a time
        int j = 0;
        while (j < L) {
            const int kA = (k0 + j) % L;
            if (!act(kA)) { ++j; continue; }
            // the run kA .. kB: open + faces until one is closed
            int n = 1;
            while (n < L && !((a.mask[cell((kA + n - 1) % L)] >> bp) & 1u)) ++n;
            const int kB = (kA + n - 1) % L;
            // forward: g*_+(B) = alB p + beB; backward: g*_-(A) = alA m + beA
            double alB = 1.0, beB = 0.0, alA = 1.0, beA = 0.0;
            for (int t = 0; t < n; ++t) {
                double dec, s;
                coef((kA + t) % L, dec, s);
                alB = dec * alB;
                beB = dec * beB + s;
                coef((kA + n - 1 - t) % L, dec, s);
                alA = dec * alA;
                beA = dec * beA + s;
            }
            double kL, hL, kR, hR;
            const long long cA = cell(kA), cB = cell(kB);
            end_rule(a, AX, -1, cA, AX == 0 ? kA : -1, homog, kL, hL);
            end_rule(a, AX, +1, cB, AX == 0 ? kB : -1, homog, kR, hR);
            // p = kL g*_-(A) + hL, m = kR g*_+(B) + hR
            const double p = (kL * alA * (kR * beB + hR) + kL * beA + hL) / (1.0 - kL * alA * kR * alB);
            const double m = kR * (alB * p + beB) + hR;
            if (out3) {
                // what leaves through the run's end faces: g*_-(A) through the - face, g*_+(B) through the + face
                const double gA = alA * m + beA, gB = alB * p + beB;
                const bool inlet = AX == 0 && kA == 0, outlet = AX == 0 && kB == a.nx - 1;
                if (inlet) { if (a.bc_in == CL_BC_DIRICHLET) out3[a.N + cA] += 2.0 * kWa * a.c_in - 2.0 * gA; }
                else if ((a.mask[cA] >> (kReactShift + bm)) & 1u) out3[cA] += (1.0 - kL) * gA;
                if (outlet) { if (a.bc_out == CL_BC_DIRICHLET) out3[2 * a.N + cB] += 2.0 * gB - 2.0 * kWa * a.c_out; }
                else if ((a.mask[cB] >> (kReactShift + bp)) & 1u) out3[cB] += (1.0 - kR) * gB;
            }
            double g = p;
            for (int t = 0; t < n; ++t) {
                const long long c = cell((kA + t) % L);
                double dec, s;
                coef((kA + t) % L, dec, s);
                T[c] += g;
                g = dec * g + s;
                if (pop) pop[(long long)ip * a.N + c] = (float)g;
            }
            g = m;
            for (int t = 0; t < n; ++t) {
                const long long c = cell((kA + n - 1 - t) % L);
                double dec, s;
                coef((kA + n - 1 - t) % L, dec, s);
                T[c] += g;
                g = dec * g + s;
                if (pop) pop[(long long)im * a.N + c] = (float)g;
            }
            j += n;
        }
    }
}

// F = (T + w0 S / omega) / (1 - w0) on active cells; with `pop`, the rest population g_0 = w0 (C + S / omega)
__global__ void k_lines_fin(SchurArgs a, const double* __restrict__ C, const double* __restrict__ T, int homog,
                            double* __restrict__ F, float* __restrict__ pop) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        const bool act = (a.mask[c] & kActiveBit) != 0;
        const double S = (act && !homog && a.src) ? a.src[c] / cell_omega(a, c) : 0.0;
        F[c] = act ? (T[c] + kWr * S) / (1.0 - kWr) : 0.0;
        if (pop) pop[c] = act ? (float)(kWr * (C[c] + S)) : 0.f;
    }
}

// lattice diffusivity cs^2 (tau - 1/2) = D dt / dx^2
__device__ __forceinline__ double cell_D(const SchurArgs& a, long long c) {
    return 0.25 * a.D[c] * a.dt_cs2dx2;
}

// neighbour of c across face d (0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z), y and z periodic
__device__ __forceinline__ long long face_nb(const SchurArgs& a, long long c, int d, int y, int z) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long plane = (long long)nx * ny;
    if (d == 0) return c + 1;
    if (d == 1) return c - 1;
    if (d == 2) return y == ny - 1 ? c - (long long)(ny - 1) * nx : c + nx;
    if (d == 3) return y == 0 ? c + (long long)(ny - 1) * nx : c - nx;
    if (d == 4) return z == nz - 1 ? c - (long long)(nz - 1) * plane : c + plane;
    return z == 0 ? c + (long long)(nz - 1) * plane : c - plane;
}

// once per call: omega (FP64) and the finite-volume operator L_D (link conductance
// 2 D_a D_b / (D_a + D_b); 2 D on a fixed-value face; 2 k D / (2 D + k) on a catalytic
// face) as G[0..2] = conductances of the +x, +y, +z links (0 where closed), G[3] = the
// diagonal, and dinv = 1 / diagonal (0 off the active set)
__global__ void k_schur_setup(SchurArgs a, double* __restrict__ om64, double* __restrict__ G,
                              double* __restrict__ dinv) {
    const int nx = a.nx, ny = a.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint16_t m = a.mask[c];
        double g[3] = {0.0, 0.0, 0.0}, diag = 0.0;
        double om = 1.0;
        if (m & kActiveBit) {
            om = omega_from_D(a, c);
            const int x = (int)(c % nx);
            const long long r = c / nx;
            const int y = (int)(r % ny), z = (int)(r / ny);
            const double Dc = cell_D(a, c);
            for (int d = 0; d < 6; ++d) {
                if ((m >> d) & 1u) {
                    if (d == 1 && x == 0) { if (a.bc_in == CL_BC_DIRICHLET) diag += 2.0 * Dc; }
                    else if (d == 0 && x == nx - 1) { if (a.bc_out == CL_BC_DIRICHLET) diag += 2.0 * Dc; }
                    else if ((m >> (kReactShift + d)) & 1u) {
                        const double k = a.k_lu * (a.kscale ? a.kscale[c] : 1.0);
                        diag += 2.0 * k * Dc / (2.0 * Dc + k);
                    }
                    continue;
                }
                const double Dn = cell_D(a, face_nb(a, c, d, y, z));
                const double Gl = 2.0 * Dc * Dn / (Dc + Dn);
                diag += Gl;
                if ((d & 1) == 0) g[d >> 1] = Gl;
            }
        }
        om64[c] = om;
        for (int k = 0; k < 3; ++k) G[(long long)k * a.N + c] = g[k];
        G[3 * a.N + c] = diag;
        dinv[c] = diag > 0.0 ? 1.0 / diag : 0.0;
    }
}

// (L_D p)(c) from the stored conductances
__device__ __forceinline__ double ld_apply(const SchurArgs& a, long long c, const double* __restrict__ p) {
    const int nx = a.nx, ny = a.ny;
    const uint16_t m = a.mask[c];
    const int y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
    const long long N = a.N;
    double q = a.G[3 * N + c] * p[c];
    for (int d = 0; d < 6; ++d) {
        if ((m >> d) & 1u) continue;
        const long long nb = face_nb(a, c, d, y, z);
        const double Gl = (d & 1) == 0 ? a.G[(long long)(d >> 1) * N + c] : a.G[(long long)(d >> 1) * N + nb];
        q -= Gl * p[nb];
    }
    return q;
}

struct Cg64 {
    double rz, alpha, beta, rr, rr0, pq;
    int iters, bad;
};

// CG start from x = 0: r = b, z = dinv r, p = z; partials r.z, r.r
__global__ void k_cg_start64(long long N, const double* __restrict__ b, const double* __restrict__ dinv,
                             double* __restrict__ x, double* __restrict__ r, double* __restrict__ p,
                             double* __restrict__ part) {
    double acc[2] = {0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const double rv = b[c], zv = dinv[c] * rv;
        x[c] = 0.0;
        r[c] = rv;
        p[c] = zv;
        acc[0] += rv * zv;
        acc[1] += rv * rv;
    }
    block_sum_store<2>(acc, part + 2 * blockIdx.x);
}

// q = L_D p, partial p.q
__global__ void k_cg_q64(SchurArgs a, const double* __restrict__ p, double* __restrict__ q, double* __restrict__ part,
                         const Cg64* __restrict__ cs) {
    if (cs->bad) return;
    double acc[1] = {0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        const double out = (a.mask[c] & kActiveBit) ? ld_apply(a, c, p) : 0.0;
        q[c] = out;
        acc[0] += p[c] * out;
    }
    block_sum_store<1>(acc, part + blockIdx.x);
}

// x += alpha p, r -= alpha q; partials r.z (z = dinv r), r.r
__global__ void k_cg_upd64(long long N, const double* __restrict__ dinv, const double* __restrict__ p,
                           const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                           double* __restrict__ part, const Cg64* __restrict__ cs) {
    if (cs->bad) return;
    const double al = cs->alpha;
    double acc[2] = {0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        x[c] += al * p[c];
        const double rv = r[c] - al * q[c];
        r[c] = rv;
        acc[0] += rv * dinv[c] * rv;
        acc[1] += rv * rv;
    }
    block_sum_store<2>(acc, part + 2 * blockIdx.x);
}

// p = dinv r + beta p
__global__ void k_cg_p64(long long N, const double* __restrict__ dinv, const double* __restrict__ r,
                         double* __restrict__ p, const Cg64* __restrict__ cs) {
    if (cs->bad) return;
    const double be = cs->beta;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        p[c] = dinv[c] * r[c] + be * p[c];
}

// one block: the CG scalars from the block partials (fixed order)
// stage 0: start (rz, rr0); 1: alpha = rz / p.q; 2: beta from the new r.z, rr
__global__ void k_cg_fin64(const double* __restrict__ part, int nblk, int stage, Cg64* cs) {
    const int nv = stage == 1 ? 1 : 2;
    double acc[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < nblk; i += blockDim.x)
        for (int k = 0; k < nv; ++k) acc[k] += part[(long long)nv * i + k];
    __shared__ double out[2];
    block_sum_store<2>(acc, out);
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (stage == 0) {
        cs->rz = out[0];
        cs->rr = cs->rr0 = out[1];
        cs->iters = 0;
        cs->bad = (out[1] == 0.0) ? 2 : (isfinite(out[0]) ? 0 : 1);
    } else if (stage == 1) {
        if (cs->bad) return;
        cs->pq = out[0];
        if (!(out[0] > 0.0) || !isfinite(out[0])) {
            // p.q = 0 after the residual has vanished is convergence, not a breakdown
            cs->bad = (isfinite(out[0]) && cs->rr <= 1e-28 * cs->rr0) ? 2 : 1;
            return;
        }
        cs->alpha = cs->rz / out[0];
    } else {
        if (cs->bad) return;
        cs->beta = out[0] / cs->rz;
        cs->rz = out[0];
        cs->rr = out[1];
        cs->iters += 1;
        if (!isfinite(out[0])) cs->bad = 1;
    }
}

// dot products of w with V[0..n) in one pass: part[blk][j]
__global__ void k_mdot(const double* __restrict__ V, long long N, int n, const double* __restrict__ w,
                       double* __restrict__ part) {
    // each block sums its chunk for every j; n <= blockDim.x * kMaxJ handled by the j loop
    __shared__ double sh[kSB];
    const long long chunk = (N + gridDim.x - 1) / gridDim.x;
    const long long c0 = blockIdx.x * chunk, c1 = min(N, c0 + chunk);
    for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        const double* v = V + (long long)j * N;
        for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) acc += v[c] * w[c];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(long long)blockIdx.x * n + j] = sh[0];
        __syncthreads();
    }
}

// h[j] = sum over blocks of part[blk][j] (one thread per j, fixed order)
__global__ void k_mdot_fin(const double* __restrict__ part, int nblk, int n, double* __restrict__ h) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nblk; ++b) acc += part[(long long)b * n + j];
        h[j] = acc;
    }
}

// w -= sum_j h[j] V[j]
__global__ void k_msub(const double* __restrict__ V, long long N, int n, const double* __restrict__ h,
                       double* __restrict__ w) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        double acc = w[c];
        for (int j = 0; j < n; ++j) acc -= h[j] * V[(long long)j * N + c];
        w[c] = acc;
    }
}

// y = alpha x (+ y if add)
__global__ void k_axpy64(long long N, double alpha, const double* __restrict__ x, double* __restrict__ y, int add) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        y[c] = alpha * x[c] + (add ? y[c] : 0.0);
}

// out = a - b (out may alias a)
__global__ void k_sub64(long long N, const double* __restrict__ a, const double* __restrict__ b, double* out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        out[c] = a[c] - b[c];
}

// block partials of the three flux fields (fixed order)
__global__ void k_sum3(long long N, const double* __restrict__ out3, double* __restrict__ part) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        acc[0] += out3[c];
        acc[1] += out3[N + c];
        acc[2] += out3[2 * N + c];
    }
    block_sum_store<3>(acc, part + 3 * blockIdx.x);
}

__global__ void k_sum3_fin(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nblk; i += blockDim.x)
        for (int k = 0; k < 3; ++k) acc[k] += part[3 * i + k];
    block_sum_store<3>(acc, out);
}

__global__ void k_norm2(long long N, const double* __restrict__ v, double* __restrict__ part) {
    double acc[1] = {0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        acc[0] += v[c] * v[c];
    block_sum_store<1>(acc, part + blockIdx.x);
}

__global__ void k_field_to_f64(long long N, const float* __restrict__ pop, const uint16_t* __restrict__ mask,
                               const double* __restrict__ src, double* __restrict__ C) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (mask[c] & kActiveBit) {
            for (int i = 0; i < 7; ++i) v += (double)pop[(long long)i * N + c];
            if (src) v -= src[c];
        }
        C[c] = v;
    }
}

struct Mem {
    cudaStream_t s;
    std::vector<void*> p;
    explicit Mem(cudaStream_t st) : s(st) {}
    cudaError_t get(double** out, long long n) {
        void* v = nullptr;
        cudaError_t e = cudaMallocAsync(&v, sizeof(double) * (size_t)(n > 0 ? n : 1), s);
        if (e == cudaSuccess) p.push_back(v);
        *out = (double*)v;
        return e;
    }
    ~Mem() {
        cudaStreamSynchronize(s);
        for (void* v : p) cudaFreeAsync(v, s);
        cudaStreamSynchronize(s);
    }
};

}  // namespace

extern "C" cl_status cl_lbm_solve_steady_lines(cl_handle h, double tol, int max_iter, int restart, double cg_tol,
                                               cl_steady_info* info) {
    if (!h) { set_msg_txt("NULL handle"); return CL_ERR_ARG; }
    if (!h->have_structure) { set_msg_txt("no structure loaded"); return CL_ERR_STATE; }
    if (h->march || h->q != 7) {
        set_msg_txt("the line-eliminated steady solve needs D3Q7 with the plain f32 population storage");
        return CL_ERR_STATE;
    }
    if (!(tol > 0.0) || max_iter < 1 || restart < 1 || !(cg_tol > 0.0 && cg_tol < 1.0)) {
        set_msg_txt("tol > 0, max_iter >= 1, restart >= 1 and 0 < cg_tol < 1 required");
        return CL_ERR_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = h->s;
    const long long N = h->N;
    const int m = restart < max_iter ? restart : max_iter;
    SchurArgs a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.N = N;
    a.mask = h->mask;
    a.D = h->D;
    a.dt_cs2dx2 = h->dt / (0.25 * h->p.dx_m * h->p.dx_m);
    a.rfac = reactive_factor_d(h);
    a.kscale = h->kscale;
    a.k_lu = h->k_lu;
    a.src = h->src;
    a.c_in = h->p.c_in; a.c_out = h->p.c_out;
    a.bc_in = h->p.bc_in; a.bc_out = h->p.bc_out;
    const int lb = kSB;
    auto nb_lines = [&](long long nl) { return (int)((nl + lb - 1) / lb); };
    cl_steady_info inf;
    memset(&inf, 0, sizeof(inf));
    cl_status result = CL_ERR_NOT_CONVERGED;
    {
        Mem mem(s);
        double *V = nullptr, *Z = nullptr, *x = nullptr, *w = nullptr, *T = nullptr, *part = nullptr, *hv = nullptr;
        double *dinv = nullptr, *cr = nullptr, *cp = nullptr, *cq = nullptr, *cpart = nullptr;
        CK(mem.get(&V, (long long)(m + 1) * N));
        CK(mem.get(&Z, (long long)m * N));
        CK(mem.get(&x, N));
        CK(mem.get(&w, N));
        CK(mem.get(&T, N));
        CK(mem.get(&part, (long long)kSBlk * (m + 1 > 3 ? m + 1 : 3)));
        CK(mem.get(&hv, m + 1 > 3 ? m + 1 : 3));
        CK(mem.get(&dinv, N));
        CK(mem.get(&cr, N));
        CK(mem.get(&cp, N));
        CK(mem.get(&cq, N));
        CK(mem.get(&cpart, 2 * kSBlk));
        double *om64 = nullptr, *G = nullptr;
        CK(mem.get(&om64, N));
        CK(mem.get(&G, 4 * N));
        a.om64 = om64;
        a.G = G;
        Cg64* cs = nullptr;
        {
            void* v = nullptr;
            CK(cudaMallocAsync(&v, sizeof(Cg64), s));
            mem.p.push_back(v);
            cs = (Cg64*)v;
        }
        // F(C) into out (affine: homog = 0; linear part: homog = 1); pop: write the state
        auto apply_F = [&](const double* C, int homog, double* out, float* pop, double* out3 = nullptr) -> cl_status {
            CK(cudaMemsetAsync(T, 0, sizeof(double) * (size_t)N, s));
            k_lines<0><<<nb_lines((long long)a.ny * a.nz), lb, 0, s>>>(a, C, T, homog, pop, out3);
            k_lines<1><<<nb_lines((long long)a.nx * a.nz), lb, 0, s>>>(a, C, T, homog, pop, out3);
            k_lines<2><<<nb_lines((long long)a.nx * a.ny), lb, 0, s>>>(a, C, T, homog, pop, out3);
            k_lines_fin<<<kSBlk, kSB, 0, s>>>(a, C, T, homog, out, pop);
            CK(cudaGetLastError());
            return CL_OK;
        };
        auto norm = [&](const double* v, double* out) -> cl_status {
            k_norm2<<<kSBlk, kSB, 0, s>>>(N, v, part);
            k_mdot_fin<<<1, 32, 0, s>>>(part, kSBlk, 1, hv);
            CK(cudaGetLastError());
            double hs = 0.0;
            CK(cudaMemcpyAsync(&hs, hv, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            *out = sqrt(hs);
            return CL_OK;
        };
        // z = L_D^{-1} v to cg_tol (diagonal-preconditioned CG, FP64)
        // 16 CG iterations on fixed buffers (solution cx), replayed as one CUDA graph
        double* cx = nullptr;
        CK(mem.get(&cx, N));
        constexpr int kCgBatch = 16;
        cudaGraphExec_t cg_graph = nullptr;
        struct GraphGuard {
            cudaGraphExec_t* g;
            ~GraphGuard() { if (*g) cudaGraphExecDestroy(*g); }
        } guard{&cg_graph};
        auto enqueue_cg = [&](cudaStream_t st) {
            for (int k = 0; k < kCgBatch; ++k) {
                k_cg_q64<<<kSBlk, kSB, 0, st>>>(a, cp, cq, cpart, cs);
                k_cg_fin64<<<1, kSB, 0, st>>>(cpart, kSBlk, 1, cs);
                k_cg_upd64<<<kSBlk, kSB, 0, st>>>(N, dinv, cp, cq, cx, cr, cpart, cs);
                k_cg_fin64<<<1, kSB, 0, st>>>(cpart, kSBlk, 2, cs);
                k_cg_p64<<<kSBlk, kSB, 0, st>>>(N, dinv, cr, cp, cs);
            }
        };
        {
            cudaStream_t cap = nullptr;
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
            if (ok) ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                enqueue_cg(cap);
                ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && g;
            }
            if (ok) ok = cudaGraphInstantiate(&cg_graph, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            if (cap) cudaStreamDestroy(cap);
            if (!ok) {
                cg_graph = nullptr;
                cudaGetLastError();  // the same kernels then run as plain launches
            }
        }
        // z = L_D^{-1} v to cg_tol (diagonal-preconditioned CG, FP64)
        auto precondition = [&](const double* v, double* z) -> cl_status {
            k_cg_start64<<<kSBlk, kSB, 0, s>>>(N, v, dinv, cx, cr, cp, cpart);
            k_cg_fin64<<<1, kSB, 0, s>>>(cpart, kSBlk, 0, cs);
            CK(cudaGetLastError());
            Cg64 hc;
            CK(cudaMemcpyAsync(&hc, cs, sizeof(hc), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            while (!hc.bad && hc.rr > cg_tol * cg_tol * hc.rr0 && hc.iters < 100000) {
                if (cg_graph) CK(cudaGraphLaunch(cg_graph, s));
                else enqueue_cg(s);
                CK(cudaGetLastError());
                CK(cudaMemcpyAsync(&hc, cs, sizeof(hc), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
            }
            if (hc.bad == 1) { set_msg_txt("inner conjugate gradients broke down"); return CL_ERR_DIVERGED; }
            CK(cudaMemcpyAsync(z, cx, sizeof(double) * (size_t)N, cudaMemcpyDeviceToDevice, s));
            inf.inner_iterations += hc.iters;
            return CL_OK;
        };
        k_schur_setup<<<kSBlk, kSB, 0, s>>>(a, om64, G, dinv);
        // start from the current state's concentration
        k_field_to_f64<<<kSBlk, kSB, 0, s>>>(N, h->pop[h->cur], h->mask, h->src, x);
        CK(cudaGetLastError());
        // the scale of the residual: |b| = |F(0)|, the right-hand side of (I - M) C = b; a warm
        // start that is already close needs no iteration
        double r0 = 0.0;
        CK(cudaMemsetAsync(w, 0, sizeof(double) * (size_t)N, s));
        CKS(apply_F(w, 0, V, nullptr));
        CKS(norm(V, &r0));
        if (!(r0 > 0.0)) r0 = 1.0;
        std::vector<double> H((size_t)(m + 1) * m), cs_(m), sn_(m), g(m + 1), hcol(m + 1);
        while (inf.iterations < max_iter) {
            // r = F(x) - x  into V[0]
            CKS(apply_F(x, 0, w, nullptr));
            k_sub64<<<kSBlk, kSB, 0, s>>>(N, w, x, V);
            CK(cudaGetLastError());
            double beta;
            CKS(norm(V, &beta));
            inf.residual = beta / r0;
            if (!isfinite(beta)) { set_msg_txt("non-finite residual"); result = CL_ERR_DIVERGED; break; }
            if (beta <= tol * r0 || beta == 0.0) { result = CL_OK; break; }
            k_axpy64<<<kSBlk, kSB, 0, s>>>(N, 1.0 / beta, V, V, 0);
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int j = 0;
            for (; j < m && inf.iterations < max_iter; ++j) {
                double* vj = V + (long long)j * N;
                double* zj = Z + (long long)j * N;
                CKS(precondition(vj, zj));
                // w = (I - M) z = z - F_lin(z)
                CKS(apply_F(zj, 1, w, nullptr));
                k_sub64<<<kSBlk, kSB, 0, s>>>(N, zj, w, w);
                // classical Gram-Schmidt, twice
                for (int k = 0; k <= j; ++k) hcol[k] = 0.0;
                for (int pass = 0; pass < 2; ++pass) {
                    k_mdot<<<kSBlk, kSB, 0, s>>>(V, N, j + 1, w, part);
                    k_mdot_fin<<<(j + 1 + 127) / 128, 128, 0, s>>>(part, kSBlk, j + 1, hv);
                    k_msub<<<kSBlk, kSB, 0, s>>>(V, N, j + 1, hv, w);
                    CK(cudaGetLastError());
                    std::vector<double> hh(j + 1);
                    CK(cudaMemcpyAsync(hh.data(), hv, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
                    CK(cudaStreamSynchronize(s));
                    for (int k = 0; k <= j; ++k) hcol[k] += hh[k];
                }
                double hn;
                CKS(norm(w, &hn));
                hcol[j + 1] = hn;
                ++inf.iterations;
                // Givens rotations of the new column
                for (int k = 0; k < j; ++k) {
                    const double t = cs_[k] * hcol[k] + sn_[k] * hcol[k + 1];
                    hcol[k + 1] = -sn_[k] * hcol[k] + cs_[k] * hcol[k + 1];
                    hcol[k] = t;
                }
                const double den = hypot(hcol[j], hcol[j + 1]);
                cs_[j] = den > 0 ? hcol[j] / den : 1.0;
                sn_[j] = den > 0 ? hcol[j + 1] / den : 0.0;
                hcol[j] = den;
                hcol[j + 1] = 0.0;
                g[j + 1] = -sn_[j] * g[j];
                g[j] = cs_[j] * g[j];
                for (int k = 0; k <= j; ++k) H[(size_t)k * m + j] = hcol[k];
                if (hn > 0 && j + 1 <= m)
                    k_axpy64<<<kSBlk, kSB, 0, s>>>(N, 1.0 / hn, w, V + (long long)(j + 1) * N, 0);
                if (fabs(g[j + 1]) <= 0.5 * tol * r0 || hn == 0.0) { ++j; break; }
            }
            // x += Z y, y from the triangular system H y = g
            std::vector<double> y(j, 0.0);
            for (int k = j - 1; k >= 0; --k) {
                double t = g[k];
                for (int l = k + 1; l < j; ++l) t -= H[(size_t)k * m + l] * y[l];
                y[k] = t / H[(size_t)k * m + k];
            }
            for (int k = 0; k < j; ++k) k_axpy64<<<kSBlk, kSB, 0, s>>>(N, y[k], Z + (long long)k * N, x, 1);
            CK(cudaGetLastError());
            ++inf.cycles;
        }
        if (result == CL_ERR_NOT_CONVERGED) {
            // the residual of the last iterate
            CKS(apply_F(x, 0, w, nullptr));
            k_sub64<<<kSBlk, kSB, 0, s>>>(N, w, x, w);
            double rn;
            CKS(norm(w, &rn));
            inf.residual = r0 > 0 ? rn / r0 : 0.0;
            if (rn <= tol * r0) result = CL_OK;
        }
        // the state: post-collision populations of the steady field, and its fluxes in FP64
        double* out3 = nullptr;
        CK(mem.get(&out3, 3 * N));
        CK(cudaMemsetAsync(out3, 0, sizeof(double) * 3 * (size_t)N, s));
        CKS(apply_F(x, 0, w, h->pop[h->cur], out3));
        k_sum3<<<kSBlk, kSB, 0, s>>>(N, out3, part);
        k_sum3_fin<<<1, kSB, 0, s>>>(part, kSBlk, hv);
        CK(cudaGetLastError());
        double fl[3];
        CK(cudaMemcpyAsync(fl, hv, sizeof(fl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        inf.R = fl[0];
        inf.J_in = fl[1];
        inf.J_out = fl[2];
    }
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return result;
}
