// Set-up kernels and the FP32 fused collide-stream kernel of the D3Q7
// reactive-diffusion LBM (arXiv:1410.1914, Sec. 2.1.3, Eq. 7-9, 19, 21-24).
#include <math.h>
#include <stdlib.h>

#include "device_util.cuh"
#include "internal.cuh"
#include "uf.cuh"

namespace cl {

// --------------------------------------------------------------- helpers
__device__ __forceinline__ bool is_pore(uint8_t p) { return p == 0 || p == 3; }
// `tmask` bit k set: phase code k carries the transported quantity
__device__ __forceinline__ bool is_transport(uint8_t p, int tmask) { return p < 4 && ((tmask >> p) & 1); }
__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// ------------------------------------------------------------ validation
__global__ void k_validate(const uint8_t* __restrict__ phase, long long N, int* err) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        if (phase[c] > 3) atomicOr(err, 1);
}

cudaError_t launch_validate(const uint8_t* phase, long long N, int* d_err, cudaStream_t s) {
    k_validate<<<1024, 256, 0, s>>>(phase, N, d_err);
    return cudaGetLastError();
}

// ------------------------------------------------ percolation (union-find)
// Transport cells 6-connected (y, z periodic) to the inlet plane x = 0.
// Union-find helpers: uf.cuh.

__global__ void k_uf_init(const uint8_t* __restrict__ phase, long long N, int tmask, int* L,
                          uint8_t* touch) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        L[c] = is_transport(phase[c], tmask) ? (int)c : -1;
        touch[c] = 0;
    }
}

__global__ void k_uf_merge(const uint8_t* __restrict__ phase, int nx, int ny, int nz, int tmask, int* L,
                           int* err) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        if (!is_transport(phase[c], tmask)) continue;
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        if (x > 0 && is_transport(phase[c - 1], tmask)) uf_union(L, (int)c, (int)(c - 1), err);
        long long n = x + (long long)nx * (wrapi(y - 1, ny) + (long long)ny * z);
        if (n != c && is_transport(phase[n], tmask)) uf_union(L, (int)c, (int)n, err);
        n = x + (long long)nx * (y + (long long)ny * wrapi(z - 1, nz));
        if (n != c && is_transport(phase[n], tmask)) uf_union(L, (int)c, (int)n, err);
    }
}

__global__ void k_uf_flatten(long long N, int* L, int* err) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        if (L[c] >= 0) L[c] = uf_find(L, (int)c, err);
}

__global__ void k_uf_touch(int nx, long long N, const int* __restrict__ L, uint8_t* touch) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        if (c % nx == 0 && L[c] >= 0) touch[L[c]] = 1;
}

__global__ void k_uf_active(long long N, const int* __restrict__ L, const uint8_t* __restrict__ touch,
                            uint8_t* active) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        active[c] = (L[c] >= 0 && touch[L[c]]) ? 1 : 0;
}

cudaError_t launch_percolation(const uint8_t* phase, int nx, int ny, int nz, int tmask, int* labels,
                               uint8_t* touch, uint8_t* active, int* d_err, cudaStream_t s) {
    const long long N = (long long)nx * ny * nz;
    const int g = 152 * 8, b = 256;
    k_uf_init<<<g, b, 0, s>>>(phase, N, tmask, labels, touch);
    k_uf_merge<<<g, b, 0, s>>>(phase, nx, ny, nz, tmask, labels, d_err);
    k_uf_flatten<<<g, b, 0, s>>>(N, labels, d_err);
    k_uf_touch<<<g, b, 0, s>>>(nx, N, labels, touch);
    k_uf_active<<<g, b, 0, s>>>(N, labels, touch, active);
    return cudaGetLastError();
}

// ------------------------------------- 13-direction pore length + D (Eq. 7-9)
__constant__ int c_dir13[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},  {1, -1, 0},
                                   {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                   {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};

__device__ long long gcd_ll(long long a, long long b) {
    while (b) { long long t = a % b; a = b; b = t; }
    return a;
}

// Run length (cells) of pore cells through (x,y,z) along direction d.  y, z
// periodic; x bounded; a line with no x component is a loop of period P and
// its run is capped at P.  Every loop is bounded by nx or by P.
__device__ int chord_run(const uint8_t* __restrict__ phase, int nx, int ny, int nz, int x, int y, int z,
                         int d) {
    const int ex = c_dir13[d][0], ey = c_dir13[d][1], ez = c_dir13[d][2];
    long long period = -1;
    if (ex == 0) {
        long long py = ey ? ny : 1, pz = ez ? nz : 1;
        period = py / gcd_ll(py, pz) * pz;
    }
    long long run = 1;
    for (int sgn = 1; sgn >= -1; sgn -= 2) {
        int px = x, py = y, pz = z;
        for (;;) {
            if (period > 0 && run >= period) break;
            const int qx = px + sgn * ex;
            if (qx < 0 || qx >= nx) break;
            const int qy = wrapi(py + sgn * ey, ny), qz = wrapi(pz + sgn * ez, nz);
            if (!is_pore(__ldg(phase + qx + (long long)nx * (qy + (long long)ny * qz)))) break;
            px = qx; py = qy; pz = qz;
            ++run;
        }
    }
    return (int)run;
}

__global__ void k_diffusivity(const uint8_t* __restrict__ phase, const uint8_t* __restrict__ active, int nx,
                              int ny, int nz, double dx, double T, double M, double D_b, double D_ion,
                              int knudsen, const double* __restrict__ D_override, double* D, double* dp,
                              int32_t* chord13) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint8_t ph = phase[c];
        const bool act = active[c] != 0;
        double dcell = 0.0, dpc = 0.0;
        const bool need_chords = is_pore(ph) && (chord13 != nullptr || dp != nullptr || (act && knudsen && !D_override));
        if (need_chords) {
            const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
            long long s1 = 0, s2 = 0, s3 = 0;  // axis, face-diagonal, body-diagonal sums
            for (int d = 0; d < 13; ++d) {
                const int r = chord_run(phase, nx, ny, nz, x, y, z, d);
                if (chord13) chord13[c * 13 + d] = r;
                if (d < 3) s1 += r; else if (d < 9) s2 += r; else s3 += r;
            }
            dpc = ((double)s1 + sqrt(2.0) * (double)s2 + sqrt(3.0) * (double)s3) * dx / 13.0;
        } else if (chord13) {
#pragma unroll
            for (int d = 0; d < 13; ++d) chord13[c * 13 + d] = 0;
        }
        if (act) {
            if (D_override) dcell = D_override[c];
            else if (ph == 2) dcell = D_ion;
            else if (knudsen) {
                const double R = 8.314462618;
                const double D_kn = dpc / 3.0 * sqrt(8.0 * R * T / (M_PI * M));  // Eq. 8
                dcell = 1.0 / (1.0 / D_kn + 1.0 / D_b);                           // Eq. 9
            } else dcell = D_b;
        }
        D[c] = dcell;
        if (dp) dp[c] = dpc;
    }
}

// ---- 13-direction lengths line by line ----
// Every cell lies on exactly one line of each direction.  One thread walks
// one line and adds, to each pore cell of a run, the run's length times
// |e_d| dx; the 13 directions run in the order of c_dir13, so that the sum
// (then / 13) is formed in the same order as a cell-by-cell evaluation.
// Lines with an x component start on the plane x = 0 and end at x = L
// (x is bounded); lines without one are closed loops of period P in their
// x-plane, and an all-pore loop gives every cell the length P.

// one step along (e_x, e_y, e_z) with y and z wrapping
__device__ __forceinline__ void chord_step(int ey, int ez, int ny, int nz, int& yy, int& zz) {
    yy += ey;
    yy = yy == ny ? 0 : (yy < 0 ? ny - 1 : yy);
    zz += ez;
    zz = zz == nz ? 0 : (zz < 0 ? nz - 1 : zz);
}

// lines with e_x = 1: one per (y0, z0) of the plane x = 0
__global__ void k_chord_xlines(const uint8_t* __restrict__ phase, int nx, int ny, int nz, int ey, int ez, double len,
                               double dx, double* __restrict__ acc) {
    const long long nlines = (long long)ny * nz;
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < nlines;
         l += (long long)gridDim.x * blockDim.x) {
        int t = 0, yy = (int)(l % ny), zz = (int)(l / ny);
        while (t < nx) {
            if (!is_pore(phase[t + (long long)nx * (yy + (long long)ny * zz)])) {
                ++t;
                chord_step(ey, ez, ny, nz, yy, zz);
                continue;
            }
            const int s = t, ys = yy, zs = zz;
            while (t < nx && is_pore(phase[t + (long long)nx * (yy + (long long)ny * zz)])) {
                ++t;
                chord_step(ey, ez, ny, nz, yy, zz);
            }
            const double add = ((double)(t - s) * len) * dx;
            int uy = ys, uz = zs;
            for (int u = s; u < t; ++u) {
                acc[u + (long long)nx * (uy + (long long)ny * uz)] += add;
                chord_step(ey, ez, ny, nz, uy, uz);
            }
        }
    }
}

// The same for lines with e_x = 1, one warp per line: the lanes read 32
// cells of the line at a time and keep the line's pore bits as 32-bit chunk
// masks in shared memory; each pore cell then finds the ends of its run in
// the masks (leading / trailing ones, continued through whole chunks).
// Lines of up to 32 * kChordChunks cells.
constexpr int kChordWarps = 4, kChordChunks = 64;

__global__ void __launch_bounds__(32 * kChordWarps) k_chord_xlines_warp(const uint8_t* __restrict__ phase, int nx, int ny,
                                                                         int nz, int ey, int ez, double len, double dx,
                                                                         double* __restrict__ acc) {
    __shared__ uint32_t mk[kChordWarps][kChordChunks];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long nlines = (long long)ny * nz;
    const int nch = (nx + 31) >> 5;
    for (long long l = (long long)blockIdx.x * kChordWarps + w; l < nlines; l += (long long)gridDim.x * kChordWarps) {
        const int y0 = (int)(l % ny), z0 = (int)(l / ny);
        auto cell = [&](int t) -> long long {
            int yy = (int)(((long long)y0 + (long long)t * ey) % ny);
            int zz = (int)(((long long)z0 + (long long)t * ez) % nz);
            yy += yy < 0 ? ny : 0;
            zz += zz < 0 ? nz : 0;
            return t + (long long)nx * (yy + (long long)ny * zz);
        };
        for (int k = 0; k < nch; ++k) {
            const int t = (k << 5) + lane;
            const bool p = t < nx && is_pore(phase[cell(t)]);
            const uint32_t b = __ballot_sync(0xffffffffu, p);
            if (lane == 0) mk[w][k] = b;
        }
        __syncwarp();
        for (int k = 0; k < nch; ++k) {
            const int t = (k << 5) + lane;
            const uint32_t m = mk[w][k];
            if (t >= nx || !((m >> lane) & 1u)) continue;
            // run cells at or below this one
            const uint32_t zl = ~m & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u));
            int left;
            if (zl) {
                left = lane - (31 - __clz(zl));
            } else {
                left = lane + 1;
                for (int j = k - 1; j >= 0; --j) {
                    const uint32_t mj = mk[w][j];
                    if (mj == 0xffffffffu) left += 32;
                    else { left += __clz(~mj); break; }
                }
            }
            // run cells at or above this one (bits past the line end are 0)
            const uint32_t zr = ~m & ~((1u << lane) - 1u);
            int right;
            if (zr) {
                right = (__ffs(zr) - 1) - lane;
            } else {
                right = 32 - lane;
                for (int j = k + 1; j < nch; ++j) {
                    const uint32_t mj = mk[w][j];
                    if (mj == 0xffffffffu) right += 32;
                    else { right += __ffs(~mj) - 1; break; }
                }
            }
            acc[cell(t)] += ((double)(left + right - 1) * len) * dx;
        }
        __syncwarp();  // the next line overwrites this warp's masks
    }
}

// Loops without an x component, one warp per loop: the loop is read from
// its first non-pore cell on, so that in that order no run wraps around,
// and then handled as an x-line; an all-pore loop gives every cell the
// period P.  Loops of up to 32 * kChordChunks cells.
__global__ void __launch_bounds__(32 * kChordWarps) k_chord_loops_warp(const uint8_t* __restrict__ phase, int nx, int ny,
                                                                        int nz, int ey, int ez, int P, int nloops,
                                                                        double len, double dx, double* __restrict__ acc) {
    __shared__ uint32_t mk[kChordWarps][kChordChunks];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long total = (long long)nloops * nx;
    const int nch = (P + 31) >> 5;
    for (long long l = (long long)blockIdx.x * kChordWarps + w; l < total; l += (long long)gridDim.x * kChordWarps) {
        const int x = (int)(l % nx), kl = (int)(l / nx);
        const int y0 = ey == 0 ? kl : 0, z0 = ey == 0 ? 0 : kl;
        auto cell = [&](int t) -> long long {  // 0 <= t < P
            const int yy = (int)(((long long)y0 + (long long)t * (ey < 0 ? ny - 1 : ey)) % ny);
            const int zz = (int)(((long long)z0 + (long long)t * (ez < 0 ? nz - 1 : ez)) % nz);
            return x + (long long)nx * (yy + (long long)ny * zz);
        };
        int t0 = -1;
        for (int k = 0; k < nch && t0 < 0; ++k) {
            const int t = (k << 5) + lane;
            const uint32_t b = __ballot_sync(0xffffffffu, t < P && !is_pore(phase[cell(t)]));
            if (b) t0 = (k << 5) + __ffs(b) - 1;
        }
        if (t0 < 0) {
            const double add = ((double)P * len) * dx;
            for (int t = lane; t < P; t += 32) acc[cell(t)] += add;
            continue;
        }
        auto tu = [&](int u) { const int t = t0 + u; return t >= P ? t - P : t; };
        for (int k = 0; k < nch; ++k) {
            const int u = (k << 5) + lane;
            const bool p = u < P && is_pore(phase[cell(tu(u))]);
            const uint32_t b = __ballot_sync(0xffffffffu, p);
            if (lane == 0) mk[w][k] = b;
        }
        __syncwarp();
        for (int k = 0; k < nch; ++k) {
            const int u = (k << 5) + lane;
            const uint32_t m = mk[w][k];
            if (u >= P || !((m >> lane) & 1u)) continue;
            const uint32_t zl = ~m & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u));
            int left;
            if (zl) {
                left = lane - (31 - __clz(zl));
            } else {
                left = lane + 1;
                for (int j = k - 1; j >= 0; --j) {
                    const uint32_t mj = mk[w][j];
                    if (mj == 0xffffffffu) left += 32;
                    else { left += __clz(~mj); break; }
                }
            }
            const uint32_t zr = ~m & ~((1u << lane) - 1u);
            int right;
            if (zr) {
                right = (__ffs(zr) - 1) - lane;
            } else {
                right = 32 - lane;
                for (int j = k + 1; j < nch; ++j) {
                    const uint32_t mj = mk[w][j];
                    if (mj == 0xffffffffu) right += 32;
                    else { right += __ffs(~mj) - 1; break; }
                }
            }
            acc[cell(tu(u))] += ((double)(left + right - 1) * len) * dx;
        }
        __syncwarp();
    }
}

// loops with e_x = 0 in each x-plane: nloops per plane, loop k starting at
// (y, z) = (k, 0) when e_y = 0, else (0, k); period P
__global__ void k_chord_loops(const uint8_t* __restrict__ phase, int nx, int ny, int nz, int ey, int ez, long long P,
                              int nloops, double len, double dx, double* __restrict__ acc) {
    const long long total = (long long)nloops * nx;
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < total;
         l += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(l % nx), k = (int)(l / nx);
        auto at = [&](int yy, int zz) { return x + (long long)nx * (yy + (long long)ny * zz); };
        int yy = ey == 0 ? k : 0, zz = ey == 0 ? 0 : k;
        long long t0 = -1;
        for (long long t = 0; t < P; ++t) {
            if (!is_pore(phase[at(yy, zz)])) { t0 = t; break; }
            chord_step(ey, ez, ny, nz, yy, zz);
        }
        if (t0 < 0) {  // an all-pore loop: every cell gets the period (yy, zz are back at the start)
            const double add = ((double)P * len) * dx;
            for (long long t = 0; t < P; ++t) {
                acc[at(yy, zz)] += add;
                chord_step(ey, ez, ny, nz, yy, zz);
            }
            continue;
        }
        // (yy, zz) is the non-pore cell t0; walk the other P - 1 cells, runs cannot wrap past it
        chord_step(ey, ez, ny, nz, yy, zz);
        long long t = t0 + 1;
        const long long end = t0 + P;
        while (t < end) {
            if (!is_pore(phase[at(yy, zz)])) {
                ++t;
                chord_step(ey, ez, ny, nz, yy, zz);
                continue;
            }
            const long long s = t;
            const int ys = yy, zs = zz;
            while (t < end && is_pore(phase[at(yy, zz)])) {
                ++t;
                chord_step(ey, ez, ny, nz, yy, zz);
            }
            const double add = ((double)(t - s) * len) * dx;
            int uy = ys, uz = zs;
            for (long long u = s; u < t; ++u) {
                acc[at(uy, uz)] += add;
                chord_step(ey, ez, ny, nz, uy, uz);
            }
        }
    }
}

// D from the accumulated lengths: d_p = sum / 13 on pore cells (Sec. 2.1.3), Eq. 7-9
// vkn = sqrt(8 R T / (pi M)) and inv_Db = 1 / D_b come from the host (the
// same correctly rounded values a cell-by-cell evaluation forms)
__global__ void k_diffusivity_dp(const uint8_t* __restrict__ phase, const uint8_t* __restrict__ active, long long N,
                                 double vkn, double inv_Db, double D_b, double D_ion, int knudsen, double* D,
                                 double* dp) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint8_t ph = phase[c];
        const double dpc = is_pore(ph) ? dp[c] / 13.0 : 0.0;
        double dcell = 0.0;
        if (active[c]) {
            if (ph == 2) dcell = D_ion;
            else if (knudsen) {
                const double D_kn = dpc / 3.0 * vkn;   // Eq. 8
                dcell = 1.0 / (1.0 / D_kn + inv_Db);   // Eq. 9
            } else dcell = D_b;
        }
        D[c] = dcell;
        dp[c] = dpc;
    }
}

static long long gcd_host(long long a, long long b) {
    while (b) { const long long t = a % b; a = b; b = t; }
    return a;
}

cudaError_t launch_diffusivity(const uint8_t* phase, const uint8_t* active, int nx, int ny, int nz,
                               double dx, double T, double M, double D_b, double D_ionomer, int knudsen,
                               const double* D_override, double* D, double* dp, int32_t* chord13,
                               cudaStream_t s) {
    if (!dp || D_override || chord13) {
        k_diffusivity<<<152 * 16, 128, 0, s>>>(phase, active, nx, ny, nz, dx, T, M, D_b, D_ionomer, knudsen,
                                               D_override, D, dp, chord13);
        return cudaGetLastError();
    }
    const long long N = (long long)nx * ny * nz;
    cudaError_t e = cudaMemsetAsync(dp, 0, sizeof(double) * (size_t)N, s);
    if (e != cudaSuccess) return e;
    // lines longer than the warp kernels' masks hold take one thread per line;
    // CL_LBM_LINE_THREADS=1 takes that path on any box (it is tested that way)
    static const bool force_threads = [] {
        const char* e = getenv("CL_LBM_LINE_THREADS");
        return e && atoi(e) != 0;
    }();
    const int dirs[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},  {1, -1, 0},
                             {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                             {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
    for (int d = 0; d < 13; ++d) {
        const int ex = dirs[d][0], ey = dirs[d][1], ez = dirs[d][2];
        const double len = sqrt((double)(ex * ex + ey * ey + ez * ez));
        if (ex && nx <= 32 * kChordChunks && !force_threads) {
            const long long nl = (long long)ny * nz;
            const long long blocks = (nl + kChordWarps - 1) / kChordWarps;
            const int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
            k_chord_xlines_warp<<<grid, 32 * kChordWarps, 0, s>>>(phase, nx, ny, nz, ey, ez, len, dx, dp);
        } else if (ex) {
            const long long nl = (long long)ny * nz;
            const int grid = (int)((nl + 127) / 128 < 152 * 16 ? (nl + 127) / 128 : 152 * 16);
            k_chord_xlines<<<grid, 128, 0, s>>>(phase, nx, ny, nz, ey, ez, len, dx, dp);
        } else {
            const long long py = ey ? ny : 1, pz = ez ? nz : 1;
            const long long P = py / gcd_host(py, pz) * pz;
            const int nloops = (int)((long long)ny * nz / P);
            const long long nl = (long long)nloops * nx;
            if (P <= 32 * kChordChunks && !force_threads) {
                const long long blocks = (nl + kChordWarps - 1) / kChordWarps;
                const int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
                k_chord_loops_warp<<<grid, 32 * kChordWarps, 0, s>>>(phase, nx, ny, nz, ey, ez, (int)P, nloops, len,
                                                                      dx, dp);
            } else {
                const int grid = (int)((nl + 127) / 128 < 152 * 16 ? (nl + 127) / 128 : 152 * 16);
                k_chord_loops<<<grid, 128, 0, s>>>(phase, nx, ny, nz, ey, ez, P, nloops, len, dx, dp);
            }
        }
    }
    const double vkn = sqrt(8.0 * 8.314462618 * T / (M_PI * M));
    k_diffusivity_dp<<<152 * 16, 128, 0, s>>>(phase, active, N, vkn, 1.0 / D_b, D_b, D_ionomer, knudsen, D, dp);
    return cudaGetLastError();
}

// 13-direction run lengths only (diagnostic export of the Sec. 2.1.3 lengths)
__global__ void k_chords13(const uint8_t* __restrict__ phase, int nx, int ny, int nz, int32_t* chord13) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        if (!is_pore(phase[c])) {
            for (int d = 0; d < 13; ++d) chord13[c * 13 + d] = 0;
            continue;
        }
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        for (int d = 0; d < 13; ++d) chord13[c * 13 + d] = chord_run(phase, nx, ny, nz, x, y, z, d);
    }
}

cudaError_t launch_chords13(const uint8_t* phase, int nx, int ny, int nz, int32_t* chord13, cudaStream_t s) {
    k_chords13<<<152 * 16, 128, 0, s>>>(phase, nx, ny, nz, chord13);
    return cudaGetLastError();
}

__global__ void k_check_positive(const uint8_t* __restrict__ active, const double* __restrict__ D, long long N,
                                 int* err) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        if (active[c] && !(D[c] > 0.0 && D[c] < INFINITY)) atomicOr(err, 4);
}

cudaError_t launch_check_positive(const uint8_t* active, const double* D, long long N, int* d_err, cudaStream_t s) {
    k_check_positive<<<152 * 4, 256, 0, s>>>(active, D, N, d_err);
    return cudaGetLastError();
}

// ---------------------------------------------------- omega (Eq. 24, D3Q7)
// tau = 1/2 + (tau_ref - 1/2) D / D_max  (dt fixed by tau_ref at D_max)
__global__ void k_omega(const uint8_t* __restrict__ active, const double* __restrict__ D, long long N,
                        double tau_ref, const double* __restrict__ Dmax, float* omega) {
    const double dmax = *Dmax;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        float om = 0.f;
        if (active[c]) {
            const double tau = 0.5 + (tau_ref - 0.5) * D[c] / dmax;
            om = (float)(1.0 / tau);
        }
        omega[c] = om;
    }
}

cudaError_t launch_omega(const uint8_t* active, const double* D, long long N, double tau_ref,
                         const double* d_Dmax, float* omega, cudaStream_t s) {
    k_omega<<<152 * 8, 256, 0, s>>>(active, D, N, tau_ref, d_Dmax, omega);
    return cudaGetLastError();
}

// --------------------------------------------------------------- link masks
__global__ void k_masks(const uint8_t* __restrict__ phase, const uint8_t* __restrict__ active,
                        const uint8_t* __restrict__ react_in, int rule, int nx, int ny, int nz,
                        uint16_t* mask) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        uint16_t m = 0;
        if (active[c]) {
            m = kActiveBit;
            const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
            const int dx[6] = {1, -1, 0, 0, 0, 0}, dy[6] = {0, 0, 1, -1, 0, 0}, dz[6] = {0, 0, 0, 0, 1, -1};
            for (int d = 0; d < 6; ++d) {
                const int qx = x + dx[d];
                if (qx < 0 || qx >= nx) { m |= (uint16_t)(1u << (kClosedShift + d)); continue; }
                const long long n = qx + (long long)nx * (wrapi(y + dy[d], ny) + (long long)ny * wrapi(z + dz[d], nz));
                if (active[n]) continue;
                m |= (uint16_t)(1u << (kClosedShift + d));
                bool react = false;
                if (phase[n] == 1) {
                    if (rule == CL_REACT_ALL_PORE_SOLID) react = phase[c] == 0;
                    else if (rule == CL_REACT_IONOMER_SOLID) react = phase[c] == 2;
                    else if (react_in) react = (react_in[c] >> d) & 1;
                }
                if (react) m |= (uint16_t)(1u << (kReactShift + d));
            }
        }
        mask[c] = m;
    }
}

cudaError_t launch_masks(const uint8_t* phase, const uint8_t* active, const uint8_t* react_in, int rule,
                         int nx, int ny, int nz, uint16_t* mask, cudaStream_t s) {
    k_masks<<<152 * 8, 256, 0, s>>>(phase, active, react_in, rule, nx, ny, nz, mask);
    return cudaGetLastError();
}

// -------------------------------------------------------------------- stats
constexpr int kStatN = 7;
__global__ void k_stats(const uint8_t* __restrict__ phase, const uint16_t* __restrict__ mask,
                        const double* __restrict__ D, const double* __restrict__ dp, long long N, int nx,
                        int tmask, double* partials) {
    double v[kStatN] = {0, 0, 0, 0, 0, 0, 0};
    double dmax = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint8_t ph = phase[c];
        const uint16_t m = mask[c];
        v[0] += is_transport(ph, tmask) ? 1.0 : 0.0;
        if (m & kActiveBit) {
            v[1] += 1.0;
            const int x = (int)(c % nx);
            unsigned closed = m & 0x3fu;
            if (x == 0) closed &= ~2u;       // -x face on the inlet plane
            if (x == nx - 1) closed &= ~1u;  // +x face on the outlet plane
            v[2] += __popc(closed);
            v[3] += __popc((m >> kReactShift) & 0x3fu);
            dmax = fmax(dmax, D[c]);
        }
        if (dp && is_pore(ph)) { v[4] += dp[c]; v[5] += 1.0; }
    }
    // sums for 0..5, max for 6 (max via the same tree with fmax)
    __shared__ double shm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
    if (lane == 0) shm[warp] = dmax;
    __syncthreads();
    if (warp == 0) {
        dmax = lane < nw ? shm[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
    }
    __syncthreads();
    v[6] = 0.0;
    block_sum_store<kStatN>(v, partials + (long long)blockIdx.x * kStatN);
    if (threadIdx.x == 0) partials[(long long)blockIdx.x * kStatN + 6] = dmax;
}

// Fixed-order reduction of partials[nblocks][nslots] -> out[nslots]; slot k
// uses max instead of sum when bit k of max_mask is set.
__global__ void k_finalize(const double* __restrict__ partials, int nblocks, int nslots, unsigned max_mask,
                           double* out) {
    const int slot = blockIdx.x;
    const bool is_max = (max_mask >> slot) & 1u;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double v = partials[(long long)b * nslots + slot];
        acc = is_max ? fmax(acc, v) : acc + v;
    }
    __shared__ double sh[1024];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = is_max ? fmax(sh[threadIdx.x], sh[threadIdx.x + w])
                                                      : sh[threadIdx.x] + sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[slot] = sh[0];
}

cudaError_t launch_stats(const uint8_t* phase, const uint16_t* mask, const double* D, const double* dp,
                            long long N, int nx, int tmask, double* partials, int nblocks, double* out,
                            cudaStream_t s) {
    k_stats<<<nblocks, 256, 0, s>>>(phase, mask, D, dp, N, nx, tmask, partials);
    k_finalize<<<kStatN, 1024, 0, s>>>(partials, nblocks, kStatN, 1u << 6, out);
    return cudaGetLastError();
}

__global__ void k_absmax(const float* __restrict__ v, long long N, double* partials) {
    double m = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs((double)v[c]));
    __shared__ double sh[1024];
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

cudaError_t launch_absmax(const float* v, long long N, double* partials, int nblocks, double* out, cudaStream_t s) {
    k_absmax<<<nblocks, 256, 0, s>>>(v, N, partials);
    k_finalize<<<1, 1024, 0, s>>>(partials, nblocks, 1, 1u, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nblocks, int nslots, double* out, cudaStream_t s) {
    k_finalize<<<nslots, 1024, 0, s>>>(partials, nblocks, nslots, 0u, out);
    return cudaGetLastError();
}

// ====================================================== FP32 solver kernels
// Initial post-collision state: equilibrium w_i C0, plus the w_i S of a
// per-cell source where one is set (the stored state is the post-collision
// populations of the current step, source included).
__global__ void k_init_fp32(float* __restrict__ pop, const uint16_t* __restrict__ mask,
                            const float* __restrict__ C0, int nx, long long N, double c_in, double c_out,
                            float* __restrict__ Csnap, const double* __restrict__ src) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        float C = 0.f;
        const bool act = (mask[c] & kActiveBit) != 0;
        if (act) {
            if (C0) C = C0[c];
            else {
                const int x = (int)(c % nx);
                C = (float)(c_in + (c_out - c_in) * (x + 0.5) / nx);
            }
        }
        const float S = (act && src) ? (float)src[c] : 0.f;
        pop[c] = act ? kW0 * (C + S) : 0.f;
#pragma unroll
        for (int i = 1; i < 7; ++i) pop[(long long)i * N + c] = act ? kW1 * (C + S) : 0.f;
        if (Csnap) Csnap[c] = C;
    }
}

cudaError_t launch_init_fp32(float* pop, const uint16_t* mask, const float* C0, int nx, int ny, int nz,
                             double c_in, double c_out, float* Csnap, const double* src, cudaStream_t s) {
    const long long N = (long long)nx * ny * nz;
    k_init_fp32<<<152 * 8, 256, 0, s>>>(pop, mask, C0, nx, N, c_in, c_out, Csnap, src);
    return cudaGetLastError();
}

// Fused pull-stream + BGK collide (Eq. 21) for one cell per thread.
// Pull: g_i(x) = g*_i(x - c_i) when that face is open; across a closed face
// the cell's own opposite post-collision population comes back:
//   inlet  (x = 0,  i = +x): -g*_{-x} + 2 w C_in  (Dirichlet, anti-bounce-back) or g*_{-x}
//   outlet (x = L,  i = -x): -g*_{+x} + 2 w C_out or g*_{+x}
//   wall:  g*_{opp}(x) times (2w - k)/(2w + k) if catalytic, else 1.
// Collide: C = sum g_i, g*_i = g_i - omega (g_i - w_i C).
// Each population first selects the element it reads (the neighbour's, or
// the cell's own opposite one across a closed face) and loads it
// unconditionally, so the six loads of a cell are in flight together; the
// boundary rules act on the loaded values.  Offsets are 32-bit (I) while
// the seven planes fit.
// T = double is the same step in FP64 arithmetic on FP64 populations (FP64
// boundary values and reactive factor; omega as stored), used for the
// residual of the mixed-precision steady solve.
template <bool REDUCE, class I, class T = float>
__global__ void __launch_bounds__(128) k_step_fp32(const T* __restrict__ src, T* __restrict__ dst,
                                                   StepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const I N = (I)a.N;
    double rv[RED_N];
    if (REDUCE)
#pragma unroll
        for (int k = 0; k < RED_N; ++k) rv[k] = 0.0;
    const bool in_row = x < nx;
    const I plane = (I)nx * (I)ny;
    const I c = (I)x + (I)nx * (I)y + plane * (I)z;
    const uint16_t m = in_row ? a.mask[c] : (uint16_t)0;
    const bool act = (m & kActiveBit) != 0;
    constexpr bool kF64 = sizeof(T) == 8;
    T h[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    {
        if (act) {
            // 1 - r of the catalytic faces; a non-uniform rate constant (Eq. 17b with the local
            // potential) on catalytic cells
            double sink_d = a.rsink_d;
            if (a.kscale && ((m >> kReactShift) & 0x3fu)) sink_d = cell_sink(a.k_lu, a.kscale[c]);
            const T rs = kF64 ? (T)sink_d : (T)(float)sink_d;
            const T abb_in = kF64 ? (T)a.abb_in_d : (T)a.abb_in, abb_out = kF64 ? (T)a.abb_out_d : (T)a.abb_out;
            // source of population i (1..6 = +x, -x, +y, -y, +z, -z): x - c_i, y and z periodic
            const I sy_m = y == 0 ? (I)(ny - 1) * (I)nx : (I)0 - (I)nx;            // row y - 1
            const I sy_p = y == ny - 1 ? (I)0 - (I)(ny - 1) * (I)nx : (I)nx;       // row y + 1
            const I sz_m = z == 0 ? (I)(nz - 1) * plane : (I)0 - plane;
            const I sz_p = z == nz - 1 ? (I)0 - (I)(nz - 1) * plane : plane;
            const I srcoff[7] = {0, (I)0 - (I)1, (I)1, sy_m, sy_p, sz_m, sz_p};
            T v[7];
            v[0] = src[c];
#pragma unroll
            for (int i = 1; i < 7; ++i) {
                const int o = ((i - 1) ^ 1) + 1;          // opposite direction
                const bool closed = (m >> (o - 1)) & 1u;  // the face the population arrives through
                const I e = closed ? (I)o * N + c : (I)i * N + c + srcoff[i];
                v[i] = src[e];
            }
            T g[7];
            g[0] = v[0];
#pragma unroll
            for (int i = 1; i < 7; ++i) {
                const int o = ((i - 1) ^ 1) + 1;
                T gi = v[i];
                if ((m >> (o - 1)) & 1u) {
                    if (i == 1 && x == 0) gi = a.bc_in == CL_BC_DIRICHLET ? abb_in - gi : gi;
                    else if (i == 2 && x == nx - 1) gi = a.bc_out == CL_BC_DIRICHLET ? abb_out - gi : gi;
                    else if (m & (1u << (kReactShift + o - 1))) gi = gi - rs * gi;
                }
                g[i] = gi;
            }
            const T C = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + g[6]);
            const T om = (T)a.omega[c];
            const T e0 = (T)kW0 * C, e1 = (T)kW1 * C;
            h[0] = g[0] - om * (g[0] - e0);
#pragma unroll
            for (int i = 1; i < 7; ++i) h[i] = g[i] - om * (g[i] - e1);
            if (a.src) {  // the a_i S term of Eq. 21, added after collision
                const T S = (T)a.src[c];
                h[0] += (T)kW0 * S;
#pragma unroll
                for (int i = 1; i < 7; ++i) h[i] += (T)kW1 * S;
            }
            if (REDUCE) {
                if (x == 0 && a.bc_in == CL_BC_DIRICHLET) rv[RED_JIN] = 2.0 * ((double)a.w_cin - (double)h[2]);
                if (x == nx - 1 && a.bc_out == CL_BC_DIRICHLET) rv[RED_JOUT] = 2.0 * ((double)h[1] - (double)a.w_cout);
                const unsigned rb = (m >> kReactShift) & 0x3fu;
                if (rb) {
                    const double sink = sink_d;
                    double r = 0.0;
#pragma unroll
                    for (int d = 0; d < 6; ++d)
                        if (rb & (1u << d)) r += h[d + 1];
                    rv[RED_R] = sink * r;
                }
                const double Cd = C;
                rv[RED_SUMC] = Cd;
                rv[RED_DC] = fabs(Cd - (double)a.Csnap[c]);
                rv[RED_ABSC] = fabs(Cd);
                rv[RED_NONFINITE] = isfinite(C) ? 0.0 : 1.0;
                a.Csnap[c] = (float)C;
            }
        }
    }
    // The lanes whose cells share a 32-byte sector (the rows are not padded,
    // so the groups come from matching sector numbers) store together when
    // any of their cells is active, so that no sector is written in part;
    // inactive cells store the zeros they already hold.
    const unsigned long long sector = in_row ? (unsigned long long)(c >> 3) : ~0ULL;
    const unsigned group = __match_any_sync(0xffffffffu, sector);
    const unsigned vote = __ballot_sync(0xffffffffu, act);
    if (in_row && (vote & group)) {
#pragma unroll
        for (int i = 0; i < 7; ++i) dst[(I)i * N + c] = h[i];
    }
    if (REDUCE) {
        const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        block_sum_store<RED_N>(rv, a.partials + blk * RED_N);
    }
}

static dim3 step_grid(const StepArgs& a) { return dim3((a.nx + 127) / 128, a.ny, a.nz); }

int step_fp32_blocks(const StepArgs& a) {
    dim3 g = step_grid(a);
    return (int)(g.x * g.y * g.z);
}

cudaError_t launch_step_fp32(const float* src, float* dst, const StepArgs& a, bool reduce, cudaStream_t s) {
    const dim3 g = step_grid(a);
    if (!a.wide && 7LL * a.N < (1LL << 32)) {
        if (reduce) k_step_fp32<true, uint32_t><<<g, 128, 0, s>>>(src, dst, a);
        else k_step_fp32<false, uint32_t><<<g, 128, 0, s>>>(src, dst, a);
    } else {
        if (reduce) k_step_fp32<true, unsigned long long><<<g, 128, 0, s>>>(src, dst, a);
        else k_step_fp32<false, unsigned long long><<<g, 128, 0, s>>>(src, dst, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_f64(const double* src, double* dst, const StepArgs& a, cudaStream_t s) {
    const dim3 g = step_grid(a);
    if (!a.wide && 7LL * a.N < (1LL << 32)) k_step_fp32<false, uint32_t, double><<<g, 128, 0, s>>>(src, dst, a);
    else k_step_fp32<false, unsigned long long, double><<<g, 128, 0, s>>>(src, dst, a);
    return cudaGetLastError();
}

// C = sum of the stored post-collision populations, less the source the
// last collision added: the concentration before collision, as Eq. 21 sees it.
__global__ void k_field_fp32(const float* __restrict__ pop, const uint16_t* __restrict__ mask, long long N,
                             float* __restrict__ C, const double* __restrict__ src) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (mask[c] & kActiveBit) {
            v = pop[c];
            for (int i = 1; i < 7; ++i) v += pop[(long long)i * N + c];
            if (src) v = (float)((double)v - src[c]);
        }
        C[c] = v;
    }
}

cudaError_t launch_field_fp32(const float* pop, const uint16_t* mask, long long N, float* C, const double* src,
                              cudaStream_t s) {
    k_field_fp32<<<152 * 8, 256, 0, s>>>(pop, mask, N, C, src);
    return cudaGetLastError();
}

// Per-plane readouts from the stored post-collision populations: one block
// per x-plane, fixed-order sums.  out[5*x + k]: sum C, active count, R,
// J_in part, J_out part.
__global__ void k_readout_fp32(const float* __restrict__ pop, StepArgs a, double* out) {
    const int x = blockIdx.x;
    const long long N = a.N;
    const long long nyz = (long long)a.ny * a.nz;
    double v[5] = {0, 0, 0, 0, 0};
    const double sink = a.rsink_d;
    for (long long j = threadIdx.x; j < nyz; j += blockDim.x) {
        const long long c = x + (long long)a.nx * j;
        const uint16_t m = a.mask[c];
        if (!(m & kActiveBit)) continue;
        double C = 0.0;
        float h[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) { h[i] = pop[(long long)i * N + c]; }
        C = (double)(((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + h[6]));
        if (a.src) C -= a.src[c];  // the concentration before the last collision's source
        v[0] += C;
        v[1] += 1.0;
        const unsigned rb = (m >> kReactShift) & 0x3fu;
        double r = 0.0;
        for (int d = 0; d < 6; ++d)
            if (rb & (1u << d)) r += h[d + 1];
        v[2] += (rb && a.kscale ? cell_sink(a.k_lu, a.kscale[c]) : sink) * r;
        if (x == 0 && a.bc_in == CL_BC_DIRICHLET) v[3] += 2.0 * ((double)a.w_cin - (double)h[2]);
        if (x == a.nx - 1 && a.bc_out == CL_BC_DIRICHLET) v[4] += 2.0 * ((double)h[1] - (double)a.w_cout);
    }
    block_sum_store<5>(v, out + 5LL * x);
}

cudaError_t launch_readout_fp32(const float* pop, const StepArgs& a, double* out, cudaStream_t s) {
    k_readout_fp32<<<a.nx, 256, 0, s>>>(pop, a, out);
    return cudaGetLastError();
}

// Per-cell amount consumed per step on the catalytic links, from the stored
// post-collision populations: (1 - r) times the populations that meet a
// catalytic face (lattice units; 0 on cells without one).
__global__ void k_cell_reaction_fp32(const float* __restrict__ pop, StepArgs a, double* __restrict__ out) {
    const long long N = a.N;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint16_t m = a.mask[c];
        const unsigned rb = (m >> kReactShift) & 0x3fu;
        double r = 0.0;
        if ((m & kActiveBit) && rb) {
            for (int d = 0; d < 6; ++d)
                if (rb & (1u << d)) r += (double)pop[(long long)(d + 1) * N + c];
            r *= a.kscale ? cell_sink(a.k_lu, a.kscale[c]) : a.rsink_d;
        }
        out[c] = r;
    }
}

cudaError_t launch_cell_reaction_fp32(const float* pop, const StepArgs& a, double* out, cudaStream_t s) {
    k_cell_reaction_fp32<<<152 * 8, 256, 0, s>>>(pop, a, out);
    return cudaGetLastError();
}

}  // namespace cl
