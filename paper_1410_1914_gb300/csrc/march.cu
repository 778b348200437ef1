// z-marching fused D3Q7 collide-stream kernel on the (C, delta) state.
//
// State per active cell after step t (post-collision, Eq. 21 with the
// equilibrium w_i C of Eq. 23):
//     g*_i = w_i C + delta_i,   i = 1..6,   delta_0 = -(delta_1 + ... + delta_6)
// C is kept as an unevaluated sum hi + lo of two floats (hi f32; lo f32, or
// f16 scaled by s_lo), the deviations as f32 (or f16 scaled by s_d).  Every
// arithmetic step works on small quantities: with a_i the incoming
// population minus w C(x),
//     open face:   a_i = w (C(x - c_i) - C(x)) + delta_i(x - c_i)
//     wall:        a_i = r delta_opp(x) - (1 - r) w C(x)      (r = 1 inert,
//                  (2w - k)/(2w + k) catalytic; the half-way first-order sink)
//     Dirichlet:   a_i = 2 w (C_bc - C(x)) - delta_opp(x)     (anti-bounce-back)
//     zero flux:   a_i = delta_opp(x)
//     dC = sum_i a_i + delta_0(x),  C' = C + dC,
//     delta'_i = (1 - omega) (a_i - w dC)
// which is the BGK step of Eq. 21 rewritten exactly; C' is accumulated in
// double-float so that increments far below ulp(C) are not lost.
//
// Each thread block owns a BX x BY column of cells and marches along z
// through a chunk of planes.  A tile always holds 512 cells, as RW rows of
// 64 / RW cells per consumer warp (RW = 1, 2 or 4: tiles of 64 x 8, 32 x 16 or
// 16 x 32): narrow tiles fit boxes whose rows are not a multiple of 64 cells
// without idle lanes.  Planes are staged into shared memory by TMA
// (cp.async.bulk.tensor.3d) into a ring of S slots guarded by mbarriers;
// the producer thread keeps S - 2 planes in flight.  Arrays carry two ghost
// rows (copies of rows ny-1 and 0 above and below) so the y-halo of a tile
// is one in-bounds box; x-halo columns come from 16-byte boxes just left and
// right of the tile.  Outputs go straight to global memory.
#include <cuda.h>
#include <math.h>

#include "device_util.cuh"
#include "internal.cuh"
#include "march.cuh"

namespace cl {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for one phase of an mbarrier; gives up after `limit` cycles of SM
// clock (0: 2^31, about 1 s) and raises bit 8 of the error word instead of
// spinning forever.
constexpr long long kWaitDefault = 1LL << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long lim = limit > 0 ? limit : kWaitDefault;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > lim) {
            atomicOr(err, 8);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// descriptors that live in global memory are acquired before the TMA unit reads them
__device__ __forceinline__ void tensormap_fence_acquire(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

// ------------------------------------------------------- storage formats
struct StoreF32 {
    using T = float;
    static __device__ __forceinline__ float ld(T v, float inv) { return v; }
    static __device__ __forceinline__ T st(float v, float s) { return v; }
};
struct StoreF16 {
    using T = __half;
    static __device__ __forceinline__ float ld(T v, float inv) { return __half2float(v) * inv; }
    static __device__ __forceinline__ T st(float v, float s) { return __float2half_rn(v * s); }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) + d, renormalised
__device__ __forceinline__ void df_add(float hi, float lo, float d, float& ho, float& lo_out) {
    float s, e;
    two_sum(hi, d, s, e);
    e += lo;
    ho = s + e;
    lo_out = e - (ho - s);
}

// ------------------------------------------------------- shared layout
template <class S, int RW>
struct SlotLayout {
    using T = typename S::T;
    static constexpr int BX = kBX / RW;  // tile width (cells)
    static constexpr int BY = kBY * RW;  // tile height (rows)
    static constexpr int EL = sizeof(T);
    static constexpr int HXL = 16 / EL;  // width of a 16-byte x-halo box in elements of T
    static constexpr int HXF = 4;        // same for f32 arrays
    static constexpr int R2 = BY + 2;
    static constexpr int al(int b) { return (b + 127) & ~127; }
    static constexpr int o_chi = 0;
    static constexpr int o_clo = o_chi + al(R2 * BX * 4);
    static constexpr int o_d3 = o_clo + al(R2 * BX * EL);
    static constexpr int o_d4 = o_d3 + al(R2 * BX * EL);
    static constexpr int o_d1 = o_d4 + al(R2 * BX * EL);
    static constexpr int o_d2 = o_d1 + al(BY * BX * EL);
    static constexpr int o_d5 = o_d2 + al(BY * BX * EL);
    static constexpr int o_d6 = o_d5 + al(BY * BX * EL);
    static constexpr int o_om = o_d6 + al(BY * BX * EL);
    static constexpr int o_mk = o_om + al(BY * BX * 4);
    static constexpr int o_chiL = o_mk + al(BY * BX * 2);
    static constexpr int o_chiR = o_chiL + al(BY * HXF * 4);
    static constexpr int o_cloL = o_chiR + al(BY * HXF * 4);
    static constexpr int o_cloR = o_cloL + al(BY * HXL * EL);
    static constexpr int o_d1L = o_cloR + al(BY * HXL * EL);
    static constexpr int o_d2R = o_d1L + al(BY * HXL * EL);
    static constexpr int bytes = o_d2R + al(BY * HXL * EL);
    // bytes delivered by the TMA loads of one plane (full boxes)
    static constexpr uint32_t tx = R2 * BX * 4 + 3 * R2 * BX * EL + 4 * BY * BX * EL + BY * BX * 4 +
                                   BY * BX * 2 + 2 * BY * HXF * 4 + 4 * BY * HXL * EL;
};

template <class S>
static int slot_bytes_rw(int rw) {
    return rw == 4 ? SlotLayout<S, 4>::bytes : (rw == 2 ? SlotLayout<S, 2>::bytes : SlotLayout<S, 1>::bytes);
}

int march_slot_bytes(int storage, int rw) {
    return storage == CL_STORE_FP16DEV ? slot_bytes_rw<StoreF16>(rw) : slot_bytes_rw<StoreF32>(rw);
}

int march_smem_bytes(int storage, int rw) { return 128 + kStages * march_slot_bytes(storage, rw); }

// the batched kernel marches tiles of every shape
static int batch_smem_bytes(int storage) {
    int m = 0;
    for (int rw = 1; rw <= kRowsMax; rw *= 2) m = m > march_smem_bytes(storage, rw) ? m : march_smem_bytes(storage, rw);
    return m;
}

// Relative cost of a tile shape for a box: the tile slots it steps (the idle
// lanes of a row's last tile count in full; rows past ny count half, their
// warps issue no arithmetic but their planes are still loaded), times the
// per-cell cost of the shape on full tiles.  Per-cell costs measured on one
// GB300 for the 256^3 Pt box (plain steps, all tiles full): FP16 state 1 :
// 1 : 1.027 (1 and 2 rows within 0.5 %) and FP32 state 1 : 1.027 : 1.155
// for 1, 2, 4 rows per warp (narrow tiles issue more TMA rows and x-halo
// boxes per cell).
double march_tile_cost(int nx, int ny, int storage, int rw) {
    static const double f16[3] = {1.0, 1.0, 1.027}, f32[3] = {1.0, 1.027, 1.155};
    const int bx = kBX / rw, by = kBY * rw;
    const double xs = (double)((nx + bx - 1) / bx) * bx;
    const double ys = (double)((ny + by - 1) / by) * by;
    const int k = rw == 4 ? 2 : rw - 1;
    return xs * (ny + 0.5 * (ys - ny)) * (storage == CL_STORE_FP16DEV ? f16[k] : f32[k]);
}

int march_auto_rows(int nx, int ny, int storage) {
    int best = 1;
    double best_cost = 0.0;
    for (int rw = 1; rw <= kRowsMax; rw *= 2) {
        const double c = march_tile_cost(nx, ny, storage, rw);
        if (rw == 1 || c < best_cost * (1.0 - 1e-9)) { best = rw; best_cost = c; }  // ties to the wider tile
    }
    return best;
}

// ------------------------------------------------------------- the kernel
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Per-cell update on the (C, delta) state, in storage units: deviations
// scaled by s_d and low words by s_lo (both 1 for FP32 storage), so that no
// value is rescaled on its way in or out.  nh/nls/nds: neighbour hi, low word
// and the deviation travelling toward this cell, for i = 1..6 (+x, -x, +y,
// -y, +z, -z).  Population i arrives through face opp(i), whose mask bit and
// own opposite deviation index are both i ^ 1.
template <class S, bool REDUCE>
__device__ __forceinline__ void cell_update(const MarchArgs& a, uint32_t m, float om, float hx, float lxs,
                                            const float (&dds)[6], const float (&nh)[6], const float (&nls)[6],
                                            const float (&nds)[6], int x, float& hnew, float& lnew_s,
                                            float (&dns)[6], double (&rv)[RED_N], float (&rs)[4], float csnap,
                                            float& csnap_out) {
    constexpr bool HALF = sizeof(typename S::T) == 2;
    const float inv_lo = HALF ? a.inv_lo : 1.0f, s_lo = HALF ? a.s_lo : 1.0f;
    const float s_d = HALF ? a.s_d : 1.0f, inv_d = HALF ? a.inv_d : 1.0f;
    const float w = kW1;
    const float ws = w * s_d;
    const float sink = a.rsink;  // 1 - r
    const float lx = lxs * inv_lo;
    const float Cx = hx + lx;
    // catalytic face: r dopp - (1 - r) w C = dopp - (1 - r)(dopp + w C) (the half-way first-order sink)
    const float wsC = ws * Cx;
    float av[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int fb = i ^ 1;
        const float dopp = dds[fb];
        const float a_open = ws * ((nh[i] - hx) + (nls[i] - lxs) * inv_lo) + nds[i];
        const float a_closed = (m & (1u << (kReactShift + fb))) ? fmaf(-sink, dopp + wsC, dopp) : dopp;
        av[i] = (m & (1u << fb)) ? a_closed : a_open;
    }
    // the x faces of the box (closed, never catalytic, so the loop gave the wall value dopp):
    // anti-bounce-back at a fixed value, bounce-back at zero flux.  Only the first and last
    // lanes of a row's end tiles take these branches; every other warp passes them uniformly.
    if (x == 0 && a.bc_in == CL_BC_DIRICHLET) av[0] = 2.0f * ws * ((a.c_in - hx) - lx) - dds[1];
    if (x == a.nx - 1 && a.bc_out == CL_BC_DIRICHLET) av[1] = 2.0f * ws * ((a.c_out - hx) - lx) - dds[0];
    const float dCs = ((av[0] + av[1]) + (av[2] + av[3]) + (av[4] + av[5])) -
                      ((dds[0] + dds[1]) + (dds[2] + dds[3]) + (dds[4] + dds[5]));
    float lnew;
    df_add(hx, lx, dCs * inv_d, hnew, lnew);
    lnew_s = lnew * s_lo;
    const float om1 = 1.0f - om;
    const float t = om1 * w * dCs;
#pragma unroll
    for (int i = 0; i < 6; ++i) dns[i] = fmaf(om1, av[i], -t);  // (1 - omega)(a_i - w dC)
    if (REDUCE) {
        // Fluxes and reaction in FP64 (boundary and catalytic cells only:
        // the stopping rule resolves their changes down to 1e-9); the
        // per-cell diagnostics in per-thread FP32 partials that the block
        // sums in FP64 (GB300's FP64 rate is a small fraction of FP32)
        const double id = inv_d;
        if (x == 0 && a.bc_in == CL_BC_DIRICHLET)
            rv[RED_JIN] += 2.0 * (double)w * ((double)a.c_in - ((double)hnew + (double)lnew)) -
                           2.0 * (double)dns[1] * id;
        if (x == a.nx - 1 && a.bc_out == CL_BC_DIRICHLET)
            rv[RED_JOUT] += 2.0 * (double)w * (((double)hnew + (double)lnew) - (double)a.c_out) +
                            2.0 * (double)dns[0] * id;
        const unsigned rb = (m >> kReactShift) & 0x3fu;
        if (rb) {
            const double Cn = (double)hnew + (double)lnew;
            double r = 0.0;
#pragma unroll
            for (int d = 0; d < 6; ++d)
                if (rb & (1u << d)) r += (double)w * Cn + (double)dns[d] * id;
            rv[RED_R] += a.rsink_d * r;
        }
        const float Cf = hnew + lnew;  // the f32 rounding of the double-float C
        rs[0] += Cf;
        rs[1] += fabsf(Cf - csnap);
        rs[2] += fabsf(Cf);
        if (!isfinite(hnew)) rs[3] += 1.0f;
        csnap_out = Cf;
    }
}

// Pair loads/stores of two adjacent cells of one array (f32 or f16)
template <class S>
struct Pair;
template <>
struct Pair<StoreF32> {
    static __device__ __forceinline__ float2 ld(const unsigned char* p, float) {
        return *reinterpret_cast<const float2*>(p);
    }
    static __device__ __forceinline__ void st(void* p, float a, float b, float) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
};
template <>
struct Pair<StoreF16> {
    static __device__ __forceinline__ float2 ld(const unsigned char* p, float) {
        return __half22float2(*reinterpret_cast<const __half2*>(p));
    }
    static __device__ __forceinline__ void st(void* p, float a, float b, float) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
};

// Warp roles: warps 0..kBY-1 each own RW rows of the tile (32 / RW lanes
// per row, two cells per lane) and compute; warp kBY is the producer and
// issues the TMA loads of one plane per slot.  full[s] completes when a plane
// has landed in slot s, empty[s] when every consumer warp has released it.  A
// consumer keeps the z-1 values it needs (its own cells one plane below) in
// registers, so a slot is live only while its plane is the current or the
// next one.
// One work item: the BX x BY column at (x0, y0), planes [zs, ze).  Planes
// zs-1 .. ze stream through the ring; `seq` is the block's running plane
// count before this item (it fixes each plane's slot and mbarrier phase, so
// items can follow each other in one block).  Every plane is released after
// use, including the last one.  Returns false if a bounded wait expired.
template <class S, bool REDUCE, int RW>
__device__ __forceinline__ bool march_item(const MarchMaps* maps, const MarchArgs& a, int x0, int y0, int zs,
                                           int ze, unsigned char* slots, uint64_t* full, uint64_t* empty,
                                           unsigned seq, bool fence_maps, double (&rv)[RED_N]) {
    using T = typename S::T;
    using L = SlotLayout<S, RW>;
    constexpr int BX = L::BX;
    constexpr int LPR = BX / 2;  // lanes per tile row (two cells each)
    using P = Pair<S>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = a.nx, ny = a.ny, nz = a.nz, px = a.px;
    const int nplanes = (ze - zs) + 2;  // zs-1 .. ze
    const long long pstride = (long long)px * (ny + 2);
    bool ok = true;

    if (ty == kBY) {
        // ------------------------------------------------------ producer
        if (tx == 0) {
            if (fence_maps) {  // descriptors written to global memory before the launch
                const CUtensorMap* mp = &maps->chi;
                for (int i = 0; i < 14; ++i) tensormap_fence_acquire(mp + i);
            }
            int k = 0;
            if (a.never_arrive) ok = false;  // test hook: no plane is ever loaded, the consumers' wait runs out
            for (; k < nplanes && ok; ++k) {
                const unsigned g = seq + k;
                const int s = g % kStages;
                const unsigned u = g / kStages;
                if (u > 0) ok = mbar_wait_bounded(&empty[s], (u - 1) & 1, a.err, a.wait_limit);
                if (!ok) break;
                unsigned char* sl = slots + s * L::bytes;
                int z = zs - 1 + k;
                z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
                uint64_t* bar = &full[s];
                fence_proxy_async();
                mbar_expect_tx(bar, L::tx);
                tma_load_3d(sl + L::o_chi, &maps->chi, bar, x0, y0, z);
                tma_load_3d(sl + L::o_clo, &maps->clo, bar, x0, y0, z);
                tma_load_3d(sl + L::o_d3, &maps->d3, bar, x0, y0, z);
                tma_load_3d(sl + L::o_d4, &maps->d4, bar, x0, y0, z);
                tma_load_3d(sl + L::o_d1, &maps->d1, bar, x0, y0 + 1, z);
                tma_load_3d(sl + L::o_d2, &maps->d2, bar, x0, y0 + 1, z);
                tma_load_3d(sl + L::o_d5, &maps->d5, bar, x0, y0 + 1, z);
                tma_load_3d(sl + L::o_d6, &maps->d6, bar, x0, y0 + 1, z);
                tma_load_3d(sl + L::o_om, &maps->om, bar, x0, y0 + 1, z);
                tma_load_3d(sl + L::o_mk, &maps->mk, bar, x0, y0 + 1, z);
                tma_load_3d(sl + L::o_chiL, &maps->chi_h, bar, x0 - L::HXF, y0 + 1, z);
                tma_load_3d(sl + L::o_chiR, &maps->chi_h, bar, x0 + BX, y0 + 1, z);
                tma_load_3d(sl + L::o_cloL, &maps->clo_h, bar, x0 - L::HXL, y0 + 1, z);
                tma_load_3d(sl + L::o_cloR, &maps->clo_h, bar, x0 + BX, y0 + 1, z);
                tma_load_3d(sl + L::o_d1L, &maps->d1_h, bar, x0 - L::HXL, y0 + 1, z);
                tma_load_3d(sl + L::o_d2R, &maps->d2_h, bar, x0 + BX, y0 + 1, z);
                if (a.prefetch > 0 && k + a.prefetch < nplanes) {
                    int zp = zs - 1 + k + a.prefetch;
                    zp = zp >= nz ? zp - nz : zp;
                    tma_prefetch_3d(&maps->chi, x0, y0, zp);
                    tma_prefetch_3d(&maps->clo, x0, y0, zp);
                    tma_prefetch_3d(&maps->d3, x0, y0, zp);
                    tma_prefetch_3d(&maps->d4, x0, y0, zp);
                    tma_prefetch_3d(&maps->d1, x0, y0 + 1, zp);
                    tma_prefetch_3d(&maps->d2, x0, y0 + 1, zp);
                    tma_prefetch_3d(&maps->d5, x0, y0 + 1, zp);
                    tma_prefetch_3d(&maps->d6, x0, y0 + 1, zp);
                    tma_prefetch_3d(&maps->om, x0, y0 + 1, zp);
                    tma_prefetch_3d(&maps->mk, x0, y0 + 1, zp);
                }
            }
            if (!ok) {
                // the loads still in flight land before shared memory is released (they
                // complete on their own, so this waits with the default bound)
                for (int j = k - 1; j >= 0 && j >= k - kStages; --j)
                    mbar_wait_bounded(&full[(seq + j) % kStages], ((seq + j) / kStages) & 1, a.err, 0);
            }
        }
        return ok;
    }
    // ---------------------------------------------------------- consumers
    float rs[4] = {0.f, 0.f, 0.f, 0.f};  // FP32 partials of sum C, sum |dC|, sum |C|, non-finite
    const int xl = tx & (LPR - 1);        // lane within its tile row
    const int row = ty * RW + tx / LPR;   // tile row of this lane
    const int xa = x0 + 2 * xl;  // this lane's cells: xa, xa + 1
    const int y = y0 + row;
    const bool row_ok = y < ny;
    const int c_own = (row + 1) * BX + 2 * xl;  // element index, ghosted arrays
    const int c_pl = row * BX + 2 * xl;         // element index, plain arrays
    // values stay in storage units; cell_update applies the scales
    const float inv_lo = 1.0f, inv_d = 1.0f, s_lo = 1.0f, s_d = 1.0f;
    constexpr int EL = L::EL;
    auto f1 = [&](const unsigned char* sl, int off) { return *reinterpret_cast<const float*>(sl + off); };
    auto t1 = [&](const unsigned char* sl, int off, float inv) {
        return S::ld(*reinterpret_cast<const T*>(sl + off), inv);
    };
    auto slot = [&](int k) { return slots + ((seq + k) % kStages) * L::bytes; };
    auto wait = [&](int k) {
        return mbar_wait_bounded(&full[(seq + k) % kStages], ((seq + k) / kStages) & 1, a.err, a.wait_limit);
    };
    auto release = [&](int k) {
        __syncwarp();
        if (tx == 0) mbar_arrive(&empty[(seq + k) % kStages]);
    };
    // x-halo neighbours: left of xa, right of xa + 1
    const bool lane_l = xl == 0, lane_r = xl == LPR - 1;
    const int xl_f = lane_l ? L::o_chiL + 4 * (row * L::HXF + L::HXF - 1) : L::o_chi + 4 * (c_own - 1);
    const int xr_f = lane_r ? L::o_chiR + 4 * (row * L::HXF) : L::o_chi + 4 * (c_own + 2);
    const int xl_lo = lane_l ? L::o_cloL + EL * (row * L::HXL + L::HXL - 1) : L::o_clo + EL * (c_own - 1);
    const int xr_lo = lane_r ? L::o_cloR + EL * (row * L::HXL) : L::o_clo + EL * (c_own + 2);
    const int xl_d1 = lane_l ? L::o_d1L + EL * (row * L::HXL + L::HXL - 1) : L::o_d1 + EL * (c_pl - 1);
    const int xr_d2 = lane_r ? L::o_d2R + EL * (row * L::HXL) : L::o_d2 + EL * (c_pl + 2);

    // every lane of a warp leaves the plane loop together (warp votes below)
    ok = __all_sync(0xffffffffu, wait(0));  // plane zs-1
    // own cells one plane below
    const unsigned char* s0 = slot(0);
    float2 ph = *reinterpret_cast<const float2*>(s0 + L::o_chi + 4 * c_own);
    float2 pl = P::ld(s0 + L::o_clo + EL * c_own, inv_lo);
    float2 pd5 = P::ld(s0 + L::o_d5 + EL * c_pl, inv_d);
    release(0);
    ok = __all_sync(0xffffffffu, ok && wait(1));  // plane zs

    int k = 1;
    for (int z = zs; z < ze && ok; ++z, ++k) {
        ok = __all_sync(0xffffffffu, ok && wait(k + 1));
        const unsigned char* sc = slot(k);
        const unsigned char* sp = slot(k + 1);
        const uint32_t mm = row_ok ? *reinterpret_cast<const uint32_t*>(sc + L::o_mk + 2 * c_pl) : 0u;
        const uint32_t ma = mm & 0xffffu, mb = mm >> 16;
        // Stores go by whole 32-byte sectors: a lane writes (zeros for an
        // inactive pair, which those cells already hold) whenever any pair
        // in its sector is active, so that no sector is written in part --
        // a partial sector costs a DRAM read to fill it -- and sectors of
        // inactive cells only are not written at all.  Rows start on
        // 16-cell boundaries (px and every tile width are multiples of 16),
        // so 4 lanes of one tile row cover an f32 sector and 8 lanes an f16
        // sector.
        const bool pact = ((ma | mb) & kActiveBit) != 0;
        const unsigned vote = __ballot_sync(0xffffffffu, pact);
        const bool st_f32 = ((vote >> (tx & ~3)) & 0xFu) != 0;
        const bool st_el = EL == 4 ? st_f32 : ((vote >> (tx & ~7)) & 0xFFu) != 0;
        float hA = 0.f, lA = 0.f, hB = 0.f, lB = 0.f, dA[6], dB[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) { dA[i] = 0.f; dB[i] = 0.f; }
        float2 cso = make_float2(0.f, 0.f);
        const long long gi = xa + (long long)px * (y + 1) + pstride * z;
        if (pact) {
            // own pair
            const float2 hx = *reinterpret_cast<const float2*>(sc + L::o_chi + 4 * c_own);
            const float2 lx = P::ld(sc + L::o_clo + EL * c_own, inv_lo);
            float2 dp[6];
            dp[0] = P::ld(sc + L::o_d1 + EL * c_pl, inv_d);
            dp[1] = P::ld(sc + L::o_d2 + EL * c_pl, inv_d);
            dp[2] = P::ld(sc + L::o_d3 + EL * c_own, inv_d);
            dp[3] = P::ld(sc + L::o_d4 + EL * c_own, inv_d);
            dp[4] = P::ld(sc + L::o_d5 + EL * c_pl, inv_d);
            dp[5] = P::ld(sc + L::o_d6 + EL * c_pl, inv_d);
            const float2 om = *reinterpret_cast<const float2*>(sc + L::o_om + 4 * c_pl);
            // y and z neighbours of both cells
            const float2 hym = *reinterpret_cast<const float2*>(sc + L::o_chi + 4 * (c_own - BX));
            const float2 lym = P::ld(sc + L::o_clo + EL * (c_own - BX), inv_lo);
            const float2 dym = P::ld(sc + L::o_d3 + EL * (c_own - BX), inv_d);
            const float2 hyp = *reinterpret_cast<const float2*>(sc + L::o_chi + 4 * (c_own + BX));
            const float2 lyp = P::ld(sc + L::o_clo + EL * (c_own + BX), inv_lo);
            const float2 dyp = P::ld(sc + L::o_d4 + EL * (c_own + BX), inv_d);
            const float2 hzp = *reinterpret_cast<const float2*>(sp + L::o_chi + 4 * c_own);
            const float2 lzp = P::ld(sp + L::o_clo + EL * c_own, inv_lo);
            const float2 dzp = P::ld(sp + L::o_d6 + EL * c_pl, inv_d);
            // outer x neighbours
            const float hxl = f1(sc, xl_f), lxl = t1(sc, xl_lo, inv_lo), dxl = t1(sc, xl_d1, inv_d);
            const float hxr = f1(sc, xr_f), lxr = t1(sc, xr_lo, inv_lo), dxr = t1(sc, xr_d2, inv_d);

            float2 cs = make_float2(0.f, 0.f);
            if (REDUCE) cs = *reinterpret_cast<const float2*>(a.Csnap + gi);

            const bool act_a = (ma & kActiveBit) != 0, act_b = (mb & kActiveBit) != 0;
            const float dda[6] = {dp[0].x, dp[1].x, dp[2].x, dp[3].x, dp[4].x, dp[5].x};
            const float nha[6] = {hxl, hx.y, hym.x, hyp.x, ph.x, hzp.x};
            const float nla[6] = {lxl, lx.y, lym.x, lyp.x, pl.x, lzp.x};
            const float nda[6] = {dxl, dp[1].y, dym.x, dyp.x, pd5.x, dzp.x};
            const float ddb[6] = {dp[0].y, dp[1].y, dp[2].y, dp[3].y, dp[4].y, dp[5].y};
            const float nhb[6] = {hx.x, hxr, hym.y, hyp.y, ph.y, hzp.y};
            const float nlb[6] = {lx.x, lxr, lym.y, lyp.y, pl.y, lzp.y};
            const float ndb[6] = {dp[0].x, dxr, dym.y, dyp.y, pd5.y, dzp.y};
            if (REDUCE) {
                // the reductions must see active cells only
                if (act_a)
                    cell_update<S, true>(a, ma, om.x, hx.x, lx.x, dda, nha, nla, nda, xa, hA, lA, dA, rv, rs, cs.x, cso.x);
                if (act_b)
                    cell_update<S, true>(a, mb, om.y, hx.y, lx.y, ddb, nhb, nlb, ndb, xa + 1, hB, lB, dB, rv, rs, cs.y,
                                         cso.y);
            } else {
                // both cells of the pair without a branch; an inactive cell's
                // result (finite: its neighbours and omega slots hold zeros or
                // state values) is replaced by the zeros it keeps
                cell_update<S, false>(a, ma, om.x, hx.x, lx.x, dda, nha, nla, nda, xa, hA, lA, dA, rv, rs, cs.x, cso.x);
                cell_update<S, false>(a, mb, om.y, hx.y, lx.y, ddb, nhb, nlb, ndb, xa + 1, hB, lB, dB, rv, rs, cs.y,
                                      cso.y);
                if (!act_a) {
                    hA = 0.f; lA = 0.f;
#pragma unroll
                    for (int i = 0; i < 6; ++i) dA[i] = 0.f;
                }
                if (!act_b) {
                    hB = 0.f; lB = 0.f;
#pragma unroll
                    for (int i = 0; i < 6; ++i) dB[i] = 0.f;
                }
            }
            // this plane becomes the z-1 neighbour of the next one
            ph = hx;
            pl = lx;
            pd5 = dp[4];
        }
        if (st_f32) {
            *reinterpret_cast<float2*>(a.chi + gi) = make_float2(hA, hB);
            if (REDUCE) *reinterpret_cast<float2*>(a.Csnap + gi) = cso;
        }
        if (st_el) {
            P::st(reinterpret_cast<T*>(a.clo) + gi, lA, lB, s_lo);
#pragma unroll
            for (int i = 0; i < 6; ++i) P::st(reinterpret_cast<T*>(a.d[i]) + gi, dA[i], dB[i], s_d);
        }
        if (y == ny - 1) {  // ghost row above row 0
            const long long gg = xa + pstride * z;
            if (st_f32) *reinterpret_cast<float2*>(a.chi + gg) = make_float2(hA, hB);
            if (st_el) {
                P::st(reinterpret_cast<T*>(a.clo) + gg, lA, lB, s_lo);
                P::st(reinterpret_cast<T*>(a.d[2]) + gg, dA[2], dB[2], s_d);
            }
        }
        if (y == 0) {  // ghost row below row ny-1
            const long long gg = xa + (long long)px * (ny + 1) + pstride * z;
            if (st_f32) *reinterpret_cast<float2*>(a.chi + gg) = make_float2(hA, hB);
            if (st_el) {
                P::st(reinterpret_cast<T*>(a.clo) + gg, lA, lB, s_lo);
                P::st(reinterpret_cast<T*>(a.d[3]) + gg, dA[3], dB[3], s_d);
            }
        }
        release(k);
    }
    if (ok) release(nplanes - 1);  // plane ze, read only as a z+1 neighbour
    if (REDUCE) {
        rv[RED_SUMC] += (double)rs[0];
        rv[RED_DC] += (double)rs[1];
        rv[RED_ABSC] += (double)rs[2];
        rv[RED_NONFINITE] += (double)rs[3];
    }
    return ok;
}

__device__ __forceinline__ bool smem_ok(const unsigned char* smem, int* err) {
    if (smem_u32(smem) & 127u) {  // TMA destinations need this alignment
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(err, 16);
        return false;
    }
    return true;
}

__device__ __forceinline__ void init_ring(uint64_t* full, uint64_t* empty) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kBY);
        }
        fence_mbar_init();
    }
    __syncthreads();
}

// FP16 plain steps: 72 registers, which still fits three resident blocks per
// SM (3 x 288 x 72 <= 65536) without the recomputation a tighter bound
// forces; FP32 plain steps need fewer than 112; the reducing steps (one per
// check) are capped at 112 so that two blocks fit per SM.
template <class S, bool REDUCE, int RW>
__global__ void __launch_bounds__(kThreads) __maxnreg__((sizeof(typename S::T) == 2 && !REDUCE) ? 72 : 112)
    k_march(const __grid_constant__ MarchMaps maps, const MarchArgs a) {
    // Addressed directly (no integer round trip) so that every slot access
    // compiles to a shared-memory load.
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + kStages;
    unsigned char* slots = smem_raw + 128;
    if (!smem_ok(smem_raw, a.err)) return;
    double rv[RED_N];
#pragma unroll
    for (int k = 0; k < RED_N; ++k) rv[k] = 0.0;
    init_ring(full, empty);
    const int zs = blockIdx.z * a.z_chunk;
    const int ze = min(a.nz, zs + a.z_chunk);
    march_item<S, REDUCE, RW>(&maps, a, blockIdx.x * (kBX / RW), blockIdx.y * (kBY * RW), zs, ze, slots, full, empty,
                              0u, false, rv);
    if (REDUCE) {
        const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        block_sum_store<RED_N>(rv, a.partials + blk * RED_N);
    }
}

// ------------------------------------------------------- batched launch
// The work of a launch is one queue of (step, item) pairs, step-major and,
// within a step, member-major.  A block takes the next pair from a global
// counter; before it marches an item of step t >= 1 it waits until every item
// of the same member at step t - 1 is done (a per-member count of finished
// items), which is all the lattice step needs: a member's step t reads only
// what its own step t - 1 wrote.  Members never wait on one another, so the
// blocks that finish a step early go on with the next step of the members that
// are ready instead of idling at a grid-wide barrier.  A wait only ever
// depends on items taken from the queue before the waiting one, whose blocks
// are running, so it cannot deadlock.
//
// Bounded wait for a member's count of finished items: gives up after `limit`
// cycles (0: 2^32, about 2 s) and raises bit 32 and the abort word, so that no
// block waits forever; another block's abort ends the wait at once.
__device__ bool wait_done(const unsigned long long* done, unsigned long long target, int* abort_flag, int* err,
                          long long limit) {
    const long long lim = limit > 0 ? limit : (1LL << 32);
    const long long t0 = clock64();
    for (;;) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(done) : "memory");
        if (v >= target) return true;
        if (*(volatile int*)abort_flag) return false;
        if (clock64() - t0 > lim) {
            atomicOr(err, 32);
            atomicExch(abort_flag, 1);
            return false;
        }
        __nanosleep(64);
    }
}

constexpr int kFenceBits = 2048;  // (member, parity) pairs whose descriptors a block has fenced

// Plain steps fit three (FP16) or two (FP32) resident blocks per SM, the
// reducing step (one per check interval) two
template <class S, bool REDUCE>
__global__ void __launch_bounds__(kThreads, REDUCE ? 2 : (sizeof(typename S::T) == 2 ? 3 : 2))
    k_march_batch(const BatchInst* __restrict__ insts, const WorkItem* __restrict__ items,
                  const int* __restrict__ n_items_ptr, const int* __restrict__ inst_count, int nsteps, int parity0,
                  unsigned long long* next, unsigned long long* done, int* abort_flag, double* item_partials,
                  int* err, long long wait_limit, int never_arrive) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + kStages;
    unsigned char* slots = smem_raw + 128;
    __shared__ MarchArgs s_args;
    __shared__ WorkItem s_it;
    __shared__ int s_w;      // its index in the work list
    __shared__ int s_step;   // step of the taken item, -1: no more work
    __shared__ int s_fence;  // first use of the item's descriptors by this block
    __shared__ unsigned s_fenced[kFenceBits / 32];
    if (!smem_ok(smem_raw, err)) { atomicExch(abort_flag, 1); return; }
    for (int i = threadIdx.y * 32 + threadIdx.x; i < kFenceBits / 32; i += kThreads) s_fenced[i] = 0u;
    init_ring(full, empty);  // ends with a block barrier
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    const long long n_items = *n_items_ptr;
    const unsigned long long total = (unsigned long long)n_items * (unsigned long long)nsteps;
    unsigned seq = 0;
    for (;;) {
        if (lead) {
            int step = -1;
            const unsigned long long q = atomicAdd(next, 1ull);
            if (q < total && *(volatile int*)abort_flag == 0) {
                step = (int)(q / (unsigned long long)n_items);
                const int w = (int)(q - (unsigned long long)step * n_items);
                const WorkItem it = items[w];
                // test hook: one finished item more than the member has never comes
                if (step > 0 &&
                    !wait_done(done + it.inst,
                               (unsigned long long)step * (unsigned long long)inst_count[it.inst] +
                                   (never_arrive ? 1ull : 0ull),
                               abort_flag, err, wait_limit))
                    step = -1;
                if (step >= 0) {
                    const int par = parity0 ^ (step & 1);
                    s_it = it;
                    s_w = w;
                    s_args = insts[it.inst].args[par];
                    const int fb = 2 * it.inst + par;
                    int fence = 1;
                    if (fb < kFenceBits) {
                        fence = !((s_fenced[fb >> 5] >> (fb & 31)) & 1u);
                        s_fenced[fb >> 5] |= 1u << (fb & 31);
                    }
                    s_fence = fence;
                }
            }
            s_step = step;
        }
        __syncthreads();
        const int step = s_step;
        if (step < 0) break;
        const WorkItem it = s_it;
        const int w = s_w;
        const int par = parity0 ^ (step & 1);
        const MarchArgs& a = s_args;
        // the producer's TMA loads (async proxy) come after the stores of the member's previous
        // step by other blocks (generic proxy), which the lead thread's wait acquired
        if (threadIdx.y == kBY && threadIdx.x == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        double rv[RED_N];
#pragma unroll
        for (int k = 0; k < RED_N; ++k) rv[k] = 0.0;
        const MarchMaps* mp = &insts[it.inst].maps[par];
        const bool fm = s_fence != 0;
        bool ok;
        if (it.rw == 4)
            ok = march_item<S, REDUCE, 4>(mp, a, it.x0, it.y0, it.zs, it.ze, slots, full, empty, seq, fm, rv);
        else if (it.rw == 2)
            ok = march_item<S, REDUCE, 2>(mp, a, it.x0, it.y0, it.zs, it.ze, slots, full, empty, seq, fm, rv);
        else
            ok = march_item<S, REDUCE, 1>(mp, a, it.x0, it.y0, it.zs, it.ze, slots, full, empty, seq, fm, rv);
        if (REDUCE) block_sum_store<RED_N>(rv, item_partials + (long long)w * RED_N);
        seq += (unsigned)(it.ze - it.zs + 2);
        ok = __syncthreads_and(ok);
        if (!ok) {
            if (lead) atomicExch(abort_flag, 1);
            break;
        }
        if (lead) {
            __threadfence();  // this item's stores before its count
            atomicAdd(done + it.inst, 1ull);
        }
    }
}

// per-instance sums of the item partials (items of an instance are contiguous)
__global__ void k_batch_finalize(const double* __restrict__ item_partials, const int* __restrict__ inst_first,
                                 const int* __restrict__ inst_count, double* out) {
    const int inst = blockIdx.x, slot = blockIdx.y;
    const int first = inst_first[inst], cnt = inst_count[inst];
    double acc = 0.0;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) acc += item_partials[(long long)(first + j) * RED_N + slot];
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[inst * RED_N + slot] = sh[0];
}

// ----------------------------------------------------------- host launch
template <class S, bool R, int RW>
static cudaError_t launch_one(const MarchMaps& maps, const MarchArgs& a, dim3 grid, int smem, cudaStream_t s) {
    static bool attr_set = false;  // per template instance
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_march<S, R, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_march<S, R, RW>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_march<S, R, RW><<<grid, dim3(32, kBY + 1, 1), smem, s>>>(maps, a);
    return cudaGetLastError();
}

template <class S, int RW>
static cudaError_t launch_rw(bool reduce, const MarchMaps& maps, const MarchArgs& a, dim3 grid, int smem,
                             cudaStream_t s) {
    return reduce ? launch_one<S, true, RW>(maps, a, grid, smem, s) : launch_one<S, false, RW>(maps, a, grid, smem, s);
}

template <class S>
static cudaError_t launch_s(int rw, bool reduce, const MarchMaps& maps, const MarchArgs& a, dim3 grid, int smem,
                            cudaStream_t s) {
    if (rw == 4) return launch_rw<S, 4>(reduce, maps, a, grid, smem, s);
    if (rw == 2) return launch_rw<S, 2>(reduce, maps, a, grid, smem, s);
    return launch_rw<S, 1>(reduce, maps, a, grid, smem, s);
}

cudaError_t launch_march(int storage, bool reduce, int rw, const MarchMaps& maps, const MarchArgs& a, dim3 grid,
                         cudaStream_t s) {
    if (rw != 1 && rw != 2 && rw != 4) return cudaErrorInvalidValue;
    const int smem = march_smem_bytes(storage, rw);
    if (storage == CL_STORE_FP16DEV) return launch_s<StoreF16>(rw, reduce, maps, a, grid, smem, s);
    return launch_s<StoreF32>(rw, reduce, maps, a, grid, smem, s);
}

template <class S, bool R>
static cudaError_t launch_batch_t(const BatchLaunch& b, int grid, cudaStream_t s) {
    const int smem = batch_smem_bytes(b.storage);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_march_batch<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_march_batch<S, R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(32, kBY + 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every block resident: one persistent block per slot
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_march_batch<S, R>, b.insts, b.items, b.n_items, b.inst_count, b.nsteps,
                              b.parity0, b.next, b.done, b.abort_flag, b.item_partials, b.err, b.wait_limit,
                              b.never_arrive);
}

// queue counter, per-member counts and abort word start from zero in each launch
static cudaError_t reset_queue(const BatchLaunch& b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b.next, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.done, 0, sizeof(unsigned long long) * b.n_inst, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.abort_flag, 0, sizeof(int), s);
    return e;
}

template <class S>
static cudaError_t launch_batch_s(const BatchLaunch& b, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    // plain steps (fewer registers, more resident blocks), then the reducing step
    const int plain = b.reduce_last ? b.nsteps - 1 : b.nsteps;
    BatchLaunch p = b;
    if (plain > 0) {
        p.nsteps = plain;
        e = reset_queue(b, s);
        if (e == cudaSuccess) e = launch_batch_t<S, false>(p, b.grid, s);
        if (e != cudaSuccess) return e;
    }
    if (b.reduce_last) {
        p.nsteps = 1;
        p.parity0 = b.parity0 ^ (plain & 1);
        e = reset_queue(b, s);
        if (e == cudaSuccess) e = launch_batch_t<S, true>(p, b.grid_reduce, s);
    }
    return e;
}

cudaError_t launch_march_batch(const BatchLaunch& b, cudaStream_t s) {
    return b.storage == CL_STORE_FP16DEV ? launch_batch_s<StoreF16>(b, s) : launch_batch_s<StoreF32>(b, s);
}

cudaError_t launch_batch_finalize(const double* item_partials, const int* inst_first, const int* inst_count,
                                  int n_inst, double* out, cudaStream_t s) {
    k_batch_finalize<<<dim3(n_inst, RED_N), 256, 0, s>>>(item_partials, inst_first, inst_count, out);
    return cudaGetLastError();
}

template <class S, bool R>
static int batch_occupancy(int smem) {
    int nb = 0;
    cudaFuncSetAttribute(k_march_batch<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_march_batch<S, R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march_batch<S, R>, kThreads, smem);
    return nb;
}

int march_batch_blocks_per_sm(int storage, bool reduce) {
    const int smem = batch_smem_bytes(storage);
    if (storage == CL_STORE_FP16DEV)
        return reduce ? batch_occupancy<StoreF16, true>(smem) : batch_occupancy<StoreF16, false>(smem);
    return reduce ? batch_occupancy<StoreF32, true>(smem) : batch_occupancy<StoreF32, false>(smem);
}

template <class S, int RW>
static int march_occupancy(int smem) {
    // the plain step variant sets the grid; the reduction variant runs once per check
    int nb = 0;
    cudaFuncSetAttribute(k_march<S, false, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_march<S, false, RW>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march<S, false, RW>, kThreads, smem);
    return nb;
}

template <class S>
static int march_occupancy_s(int rw, int smem) {
    return rw == 4 ? march_occupancy<S, 4>(smem) : (rw == 2 ? march_occupancy<S, 2>(smem) : march_occupancy<S, 1>(smem));
}

int march_blocks_per_sm(int storage, int rw) {
    const int smem = march_smem_bytes(storage, rw);
    const int nb = storage == CL_STORE_FP16DEV ? march_occupancy_s<StoreF16>(rw, smem)
                                               : march_occupancy_s<StoreF32>(rw, smem);
    return nb > 0 ? nb : 1;
}

// ====================================================== state utilities
// Stored row yr in [0, ny+2) -> actual row (ghost rows wrap).
__device__ __forceinline__ int actual_row(int yr, int ny) { return yr == 0 ? ny - 1 : (yr == ny + 1 ? 0 : yr - 1); }

template <class S>
__global__ void k_state_init(MarchArgs a, const uint16_t* __restrict__ mask_p, const float* __restrict__ C0) {
    using T = typename S::T;
    const long long pstride = (long long)a.px * (a.ny + 2);
    const long long total = pstride * a.nz;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(gi % a.px);
        const int yr = (int)((gi / a.px) % (a.ny + 2));
        const int z = (int)(gi / pstride);
        const int y = actual_row(yr, a.ny);
        const long long gm = x + (long long)a.px * (y + 1) + pstride * z;  // owner's slot
        float hi = 0.f, lo = 0.f;
        if (x < a.nx && (mask_p[gm] & kActiveBit)) {
            double C;
            if (C0) C = C0[x + (long long)a.nx * (y + (long long)a.ny * z)];
            else C = (double)a.c_in + ((double)a.c_out - (double)a.c_in) * (x + 0.5) / a.nx;
            hi = (float)C;
            lo = (float)(C - (double)hi);
        }
        a.chi[gi] = hi;
        reinterpret_cast<T*>(a.clo)[gi] = S::st(lo, a.s_lo);
        for (int i = 0; i < 6; ++i) reinterpret_cast<T*>(a.d[i])[gi] = S::st(0.f, a.s_d);
        if (a.Csnap) a.Csnap[gi] = hi + lo;
    }
}

// unpadded outputs: C (N floats) and/or g* (7 x N floats)
template <class S>
__global__ void k_state_out(MarchArgs a, const uint16_t* __restrict__ mask_p, float* __restrict__ C,
                            float* __restrict__ g) {
    using T = typename S::T;
    const long long N = (long long)a.nx * a.ny * a.nz;
    const long long pstride = (long long)a.px * (a.ny + 2);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % a.nx), y = (int)((c / a.nx) % a.ny), z = (int)(c / ((long long)a.nx * a.ny));
        const long long gi = x + (long long)a.px * (y + 1) + pstride * z;
        const bool act = (mask_p[gi] & kActiveBit) != 0;
        float Cv = 0.f, d[6] = {0, 0, 0, 0, 0, 0};
        if (act) {
            Cv = a.chi[gi] + S::ld(reinterpret_cast<const T*>(a.clo)[gi], a.inv_lo);
            for (int i = 0; i < 6; ++i) d[i] = S::ld(reinterpret_cast<const T*>(a.d[i])[gi], a.inv_d);
        }
        if (C) C[c] = Cv;
        if (g) {
            const float d0 = -(((d[0] + d[1]) + (d[2] + d[3])) + (d[4] + d[5]));
            g[c] = act ? kW0 * Cv + d0 : 0.f;
            for (int i = 0; i < 6; ++i) g[(long long)(i + 1) * N + c] = act ? kW1 * Cv + d[i] : 0.f;
        }
    }
}

// per-plane readouts (one block per x-plane): sum C, count, R, J_in part, J_out part
template <class S>
__global__ void k_state_readout(MarchArgs a, const uint16_t* __restrict__ mask_p, double* out) {
    using T = typename S::T;
    const int x = blockIdx.x;
    const long long nyz = (long long)a.ny * a.nz;
    const long long pstride = (long long)a.px * (a.ny + 2);
    const double w = kW1;
    double v[5] = {0, 0, 0, 0, 0};
    for (long long j = threadIdx.x; j < nyz; j += blockDim.x) {
        const int y = (int)(j % a.ny), z = (int)(j / a.ny);
        const long long gi = x + (long long)a.px * (y + 1) + pstride * z;
        const uint16_t m = mask_p[gi];
        if (!(m & kActiveBit)) continue;
        const double C = (double)a.chi[gi] + (double)S::ld(reinterpret_cast<const T*>(a.clo)[gi], a.inv_lo);
        double d[6];
        for (int i = 0; i < 6; ++i) d[i] = S::ld(reinterpret_cast<const T*>(a.d[i])[gi], a.inv_d);
        v[0] += C;
        v[1] += 1.0;
        const unsigned rb = (m >> kReactShift) & 0x3fu;
        double r = 0.0;
        for (int dd = 0; dd < 6; ++dd)
            if (rb & (1u << dd)) r += w * C + d[dd];
        v[2] += a.rsink_d * r;
        if (x == 0 && a.bc_in == CL_BC_DIRICHLET) v[3] += 2.0 * w * ((double)a.c_in - C) - 2.0 * d[1];
        if (x == a.nx - 1 && a.bc_out == CL_BC_DIRICHLET) v[4] += 2.0 * w * (C - (double)a.c_out) + 2.0 * d[0];
    }
    block_sum_store<5>(v, out + 5LL * x);
}

cudaError_t launch_state_init(int storage, const MarchArgs& a, const uint16_t* mask_p, const float* C0,
                              cudaStream_t s) {
    if (storage == CL_STORE_FP16DEV) k_state_init<StoreF16><<<152 * 8, 256, 0, s>>>(a, mask_p, C0);
    else k_state_init<StoreF32><<<152 * 8, 256, 0, s>>>(a, mask_p, C0);
    return cudaGetLastError();
}

cudaError_t launch_state_out(int storage, const MarchArgs& a, const uint16_t* mask_p, float* C, float* g,
                             cudaStream_t s) {
    if (storage == CL_STORE_FP16DEV) k_state_out<StoreF16><<<152 * 8, 256, 0, s>>>(a, mask_p, C, g);
    else k_state_out<StoreF32><<<152 * 8, 256, 0, s>>>(a, mask_p, C, g);
    return cudaGetLastError();
}

cudaError_t launch_state_readout(int storage, const MarchArgs& a, const uint16_t* mask_p, double* out,
                                 cudaStream_t s) {
    if (storage == CL_STORE_FP16DEV) k_state_readout<StoreF16><<<a.nx, 256, 0, s>>>(a, mask_p, out);
    else k_state_readout<StoreF32><<<a.nx, 256, 0, s>>>(a, mask_p, out);
    return cudaGetLastError();
}

// unpadded -> padded (ghosted) copy of the static per-cell arrays
__global__ void k_pad_static(const uint16_t* __restrict__ mask, const float* __restrict__ omega, int nx, int ny,
                             int nz, int px, uint16_t* __restrict__ mask_p, float* __restrict__ omega_p) {
    const long long pstride = (long long)px * (ny + 2);
    const long long total = pstride * nz;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(gi % px);
        const int yr = (int)((gi / px) % (ny + 2));
        const int z = (int)(gi / pstride);
        const int y = actual_row(yr, ny);
        uint16_t m = 0;
        float o = 0.f;
        if (x < nx) {
            const long long c = x + (long long)nx * (y + (long long)ny * z);
            m = mask[c];
            o = omega[c];
        }
        mask_p[gi] = m;
        omega_p[gi] = o;
    }
}

cudaError_t launch_pad_static(const uint16_t* mask, const float* omega, int nx, int ny, int nz, int px,
                              uint16_t* mask_p, float* omega_p, cudaStream_t s) {
    k_pad_static<<<152 * 8, 256, 0, s>>>(mask, omega, nx, ny, nz, px, mask_p, omega_p);
    return cudaGetLastError();
}

}  // namespace cl
