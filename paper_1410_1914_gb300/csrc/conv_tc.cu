// 3x3x3 convolutions of the warm-start network on the 5th-generation tensor
// cores (tcgen05.mma kind::f16, BF16 operands, FP32 accumulators in tensor
// memory).  Implicit GEMMs: out[v][n] = sum over taps t and input channels c
// of in[shift(v, t)][c] * w[t][n][c]; the weight gradient is the GEMM over
// voxels.  Three kernels:
//
//   k_conv3d_halo        forward / data gradient (the main path): one CTA per
//                        8 x 16 block of output voxels; the 10 x 18 x 3 input
//                        halo is staged once per channel chunk and every tap
//                        is a shifted descriptor into it; weights stream.
//   k_conv3d_wgrad_halo  weight gradient of 16-channel inputs: per voxel
//                        block the halo and the output-gradient tile are
//                        staged once, every tap a shifted MN-major
//                        descriptor, accumulation over a slice of blocks in
//                        tensor memory.
//   k_conv3d_wgrad_tc    weight gradient of wider inputs, one gather per tap
//                        and voxel (faster there: see
//                        conv3d_wgrad_halo_supported).
//   k_conv3d_tc          forward with one gather per tap and voxel; used
//                        where a halo tile does not fit.
//
// Roles (160 threads): warps 0-3 stage operands with cp.async (zero fill
// outside the box; y and z wrap by index), make them visible to the tensor
// core (fence.proxy.async) and arrive on the stage's `full` barrier, then
// run the epilogue (tcgen05.ld of their 32 TMEM lanes: warp w owns lanes
// 32w..32w+31); warp 4 allocates and frees the tensor memory and its lane 0
// issues the MMAs of each stage and commits them to the stage's `empty`
// barrier and, after the last stage, to `done`.
//
// Shared-memory operands use the no-swizzle core-matrix layouts: 8 rows of
// 16 bytes, contiguous.  K-major (forward): a row is 8 input channels of one
// voxel; LBO steps to the next 8 channels, SBO to the next 8 rows.  MN-major
// (weight gradient): a row is 8 channels of one voxel read along K = voxels;
// LBO steps to the next 8 voxels, SBO to the next 8 channels.
//
// Every wait is bounded; on expiry the CTA records an error bit, stops
// issuing work, waits (bounded) for the MMAs it issued, frees its tensor
// memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "internal.cuh"
#include "nn.cuh"

namespace cl {

namespace {

constexpr int kTcM = 128;       // output voxels per CTA (TMEM lanes)
constexpr int kTcStages = 4;    // shared-memory stages of the weight gradient
constexpr int kFwStages = 6;    // shared-memory stages of the forward kernel
constexpr int kLag = kFwStages - 2;  // its stages whose copies are in flight per thread
constexpr int kTcThreads = 160; // 4 producer/epilogue warps + 1 MMA warp

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait (~1 s of SM clock); false on expiry
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
    if (bar_try_wait(b, parity)) return true;
    const long long t0 = clock64();
    while (!bar_try_wait(b, parity))
        if (clock64() - t0 > (1LL << 31)) return false;
    return true;
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}

// 16-byte asynchronous copy global -> shared; zero fill when !valid.  The
// .ca form keeps the line in L1: the taps of neighbouring voxels read the
// same activation rows again within the CTA.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async16_ca(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// generic-proxy writes to shared memory become visible to the tensor core
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture
    return d;                // base offset 0, swizzle none
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(b))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcShape {
    int CK;        // channels per k-step (16..64, divides ci)
    int N;         // output channels (co)
    int ncols;     // TMEM columns (power of two >= max(32, N))
    int a_bytes;   // 128 x CK x 2
    int b_bytes;   // N x CK x 2
    int stage;     // a_bytes + b_bytes
    int smem;      // dynamic shared memory
};

}  // namespace

__host__ __device__ inline TcShape tc_shape(int ci, int co) {
    TcShape s;
    // widest channel chunk that divides ci and keeps the stages within ~200 KB
    const int cands[4] = {64, 48, 32, 16};
    s.CK = 16;
    for (int i = 0; i < 4; ++i) {
        const int ck = cands[i];
        if (ck > ci || ci % ck) continue;
        if (1024 + kFwStages * (kTcM + co) * ck * 2 <= 200 * 1024) { s.CK = ck; break; }
    }
    s.N = co;
    int c = 32;
    while (c < co) c <<= 1;
    s.ncols = c;
    s.a_bytes = kTcM * s.CK * 2;
    s.b_bytes = co * s.CK * 2;
    s.stage = s.a_bytes + s.b_bytes;
    s.smem = 1024 + kFwStages * s.stage;
    return s;
}

__global__ void __launch_bounds__(kTcThreads) k_conv3d_tc(const __nv_bfloat16* __restrict__ in,
                                                          const __nv_bfloat16* __restrict__ w,
                                                          const float* __restrict__ bias,
                                                          __nv_bfloat16* __restrict__ out, ConvGeom g, int relu,
                                                          int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcShape sh = tc_shape(g.ci, g.co);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kFwStages;
    uint64_t* done = empty + kFwStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    unsigned char* stages = smem + 1024;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const long long v0 = (long long)blockIdx.x * kTcM;
    const int CK = sh.CK, kgroups = CK / 8;
    const int ksteps = 27 * (g.ci / CK);
    const uint32_t sbo_a = (uint32_t)kgroups * 128u, sbo_b = sbo_a;

    if (tid == 0) {
        for (int s = 0; s < kFwStages; ++s) {
            bar_init(&full[s], 128);
            bar_init(&empty[s], 1);
        }
        bar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(sh.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ------------------------------------------------------ producers
        const int r = tid;  // output row of this thread
        const long long v = v0 + r;
        const bool row_ok = v < M;
        int x = 0, y = 0, z = 0;
        long long nb = 0;
        if (row_ok) {
            x = (int)(v % g.W);
            long long q = v / g.W;
            y = (int)(q % g.H);
            q /= g.H;
            z = (int)(q % g.D);
            nb = q / g.D;
        }
        const uint32_t a_row = (uint32_t)(r >> 3) * sbo_a + (uint32_t)(r & 7) * 16u;
        bool ok = true;
        int issued = 0;  // stages whose copies were issued
        for (int ks = 0; ks < ksteps; ++ks) {
            const int s = ks % kFwStages;
            if (ks >= kFwStages) {
                if (!bar_wait(&empty[s], ((ks / kFwStages) - 1) & 1)) { ok = false; }
            }
            if (!ok || *(volatile int*)abort_flag) { ok = false; break; }
            const int t = ks / (g.ci / CK);
            const int c0 = (ks % (g.ci / CK)) * CK;
            unsigned char* st = stages + s * sh.stage;
            // A: the tap-shifted input row of this voxel
            const int qx = x + t % 3 - 1;
            int qy = y + (t / 3) % 3 - 1, qz = z + t / 9 - 1;
            bool valid = row_ok && qx >= 0 && qx < g.W;
            if (g.periodic_yz) {
                qy = qy < 0 ? qy + g.H : (qy >= g.H ? qy - g.H : qy);
                qz = qz < 0 ? qz + g.D : (qz >= g.D ? qz - g.D : qz);
            } else {
                valid = valid && qy >= 0 && qy < g.H && qz >= 0 && qz < g.D;
            }
            const long long sv = valid ? qx + (long long)g.W * (qy + (long long)g.H * (qz + (long long)g.D * nb)) : 0;
            const __nv_bfloat16* src = in + sv * g.in_stride + g.in_off + c0;
            const uint32_t a_base = smem_addr(st) + a_row;
            for (int h = 0; h < kgroups; ++h) cp_async16_ca(a_base + (uint32_t)h * 128u, src + 8 * h, valid);
            // B: weight rows of this tap and channel chunk, shared by the 128 threads
            const uint32_t b_base = smem_addr(st + sh.a_bytes);
            const __nv_bfloat16* wt = w + (long long)t * g.co * g.ci + c0;
            for (int e = r; e < g.co * kgroups; e += 128) {
                const int n = e / kgroups, h = e % kgroups;
                cp_async16(b_base + (uint32_t)(n >> 3) * sbo_b + (uint32_t)h * 128u + (uint32_t)(n & 7) * 16u,
                           wt + (long long)n * g.ci + 8 * h, true);
            }
            cp_async_commit();
            ++issued;
            // stage ks - kLag has landed: publish it to the tensor core
            if (ks >= kLag) {
                cp_async_wait<kLag>();
                fence_async_shared();
                bar_arrive(&full[(ks - kLag) % kFwStages]);
            }
        }
        // publish the stages still in flight (also after an abort, so that
        // no copy is outstanding when the CTA leaves)
        cp_async_wait<0>();
        fence_async_shared();
        for (int ks = (issued >= kLag ? issued - kLag : 0); ks < issued; ++ks) bar_arrive(&full[ks % kFwStages]);
        if (!ok) {
            atomicOr(err, 64);
            *(volatile int*)abort_flag = 1;
        }
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issuer
        const uint32_t idesc = idesc_bf16(kTcM, g.co);
        int ks = 0;
        for (; ks < ksteps; ++ks) {
            const int s = ks % kFwStages;
            if (!bar_wait(&full[s], (ks / kFwStages) & 1) || *(volatile int*)abort_flag) {
                atomicOr(err, 64);
                *(volatile int*)abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_addr(stages + s * sh.stage), b0 = a0 + (uint32_t)sh.a_bytes;
            for (int kk = 0; kk < CK / 16; ++kk) {
                const uint64_t ad = sdesc(a0 + (uint32_t)kk * 256u, 128u, sbo_a);
                const uint64_t bd = sdesc(b0 + (uint32_t)kk * 256u, 128u, sbo_b);
                mma_bf16_ss(tmem, ad, bd, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        mma_commit(done);  // every MMA issued so far has completed
    }

    // ---------------------------------------------------------- epilogue
    if (warp < 4) {
        const bool ok = bar_wait(done, 0);
        tc_fence_after();
        if (!ok) atomicOr(err, 64);
        const long long v = v0 + tid;
        const bool store = ok && !*(volatile int*)abort_flag && v < M;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < g.co; c += 16) {
            uint32_t acc[16];
            tmem_ld16(lane_base + (uint32_t)c, acc);  // warp-wide: every lane takes part
            if (store) {
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float a = __uint_as_float(acc[2 * j]) + (bias ? bias[c + 2 * j] : 0.f);
                    float b = __uint_as_float(acc[2 * j + 1]) + (bias ? bias[c + 2 * j + 1] : 0.f);
                    if (relu) { a = fmaxf(a, 0.f); b = fmaxf(b, 0.f); }
                    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                    pk[j] = *reinterpret_cast<uint32_t*>(&h);
                }
                uint4* dst = reinterpret_cast<uint4*>(out + v * g.out_stride + g.out_off + c);
                dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(sh.ncols) : "memory");
    }
}

// ------------------------------------------------------------ weight grad
// dW[t][co][ci] = sum_v dO[v][co] * I[shift(v, t)][ci] as, per tap, a GEMM
// D[m = co][n = ci] over K = voxels.  Both operands come straight from the
// NDHWC activations, which hold 8 consecutive channels of one voxel in 16
// bytes: that is the MN-major layout (M, resp. N, contiguous), so A = dO
// and B = the tap-shifted input are staged with 16-byte copies as for the
// forward pass.  A CTA owns a slice of voxels and a group of TG taps, one
// FP32 accumulator of 128 lanes x ci columns per tap in tensor memory
// (TG * ci <= 256 columns, so two CTAs share an SM), and writes one partial
// dW per slice; a second kernel sums the slices in a fixed order.
// Lanes co..127 of the accumulators (M is padded to 128) are never read.
//
// MN-major core matrix: 8 voxels (K) x 8 channels (16 bytes); element
// (m, k) of a stage at (m / 8) * MNS + (k / 8) * 128 + (k % 8) * 16 +
// (m % 8) * 2, MNS = KT / 8 * 128: core matrices adjacent along K are 128
// bytes apart, along M (or N) MNS bytes apart.
constexpr int kWgKT = 32;  // voxels per stage

__host__ __device__ inline int wg_taps_per_group(int ci) {
    int tg = 256 / ci;
    return tg > 27 ? 27 : (tg < 1 ? 1 : tg);
}

__host__ __device__ inline int wg_ncols(int tg, int ci) {
    int c = 32;
    while (c < tg * ci) c <<= 1;
    return c;
}

__host__ __device__ inline int wg_stage_bytes(int tg, int ci) { return kTcM * kWgKT * 2 + tg * ci * kWgKT * 2; }

long long wgrad_tc_slice(const ConvGeom& g) {
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const int groups = (27 + wg_taps_per_group(g.ci) - 1) / wg_taps_per_group(g.ci);
    long long ns = 304 / groups;  // about two CTAs per SM in all
    if (ns < 1) ns = 1;
    long long slice = (M + ns - 1) / ns;
    slice = (slice + kWgKT - 1) / kWgKT * kWgKT;
    return slice < kWgKT ? kWgKT : slice;
}

__global__ void __launch_bounds__(kTcThreads) k_conv3d_wgrad_tc(const __nv_bfloat16* __restrict__ in,
                                                                const __nv_bfloat16* __restrict__ dout,
                                                                float* __restrict__ partial, ConvGeom g,
                                                                long long slice, uint32_t lbo_mn, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int TG = wg_taps_per_group(g.ci);
    const int ncols = wg_ncols(TG, g.ci);
    const int stage_bytes = wg_stage_bytes(TG, g.ci);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kTcStages;
    uint64_t* done = empty + kTcStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    unsigned char* stages = smem + 1024;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const long long vs = (long long)blockIdx.x * slice;
    const long long ve = vs + slice < M ? vs + slice : M;
    const int t0 = blockIdx.y * TG;
    const int ntap = 27 - t0 < TG ? 27 - t0 : TG;
    const int ksteps = vs < ve ? (int)((ve - vs + kWgKT - 1) / kWgKT) : 0;
    const uint32_t mns = (uint32_t)(kWgKT / 8) * 128u;  // stride between core matrices along M / N
    const int a_bytes = kTcM * kWgKT * 2;
    const int b_tap_bytes = g.ci * kWgKT * 2;

    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            bar_init(&full[s], 128);
            bar_init(&empty[s], 1);
        }
        bar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ------------------------------------------------------ producers
        // thread: voxel k = tid % 32 of the stage, chunk lanes tid / 32
        const int k = tid & 31, part = tid >> 5;
        bool ok = true;
        int issued = 0;
        for (int ks = 0; ks < ksteps; ++ks) {
            const int s = ks % kTcStages;
            if (ks >= kTcStages && !bar_wait(&empty[s], ((ks / kTcStages) - 1) & 1)) ok = false;
            if (!ok || *(volatile int*)abort_flag) { ok = false; break; }
            const long long v = vs + (long long)ks * kWgKT + k;
            const bool vok = v < ve;
            int x = 0, y = 0, z = 0;
            long long nb = 0;
            if (vok) {
                x = (int)(v % g.W);
                long long q = v / g.W;
                y = (int)(q % g.H);
                q /= g.H;
                z = (int)(q % g.D);
                nb = q / g.D;
            }
            unsigned char* st = stages + s * stage_bytes;
            const uint32_t kofs = (uint32_t)(k >> 3) * 128u + (uint32_t)(k & 7) * 16u;
            // A: dO[v][0..co), 8 channels per chunk
            const uint32_t a_base = smem_addr(st) + kofs;
            const __nv_bfloat16* srcA = dout + (vok ? v : 0) * g.out_stride + g.out_off;
            for (int mc = part; mc < g.co / 8; mc += 4) cp_async16(a_base + (uint32_t)mc * mns, srcA + 8 * mc, vok);
            // B: for each tap of the group, I[shift(v, t)][0..ci)
            for (int j = 0; j < ntap; ++j) {
                const int t = t0 + j;
                const int qx = x + t % 3 - 1;
                int qy = y + (t / 3) % 3 - 1, qz = z + t / 9 - 1;
                bool valid = vok && qx >= 0 && qx < g.W;
                if (g.periodic_yz) {
                    qy = qy < 0 ? qy + g.H : (qy >= g.H ? qy - g.H : qy);
                    qz = qz < 0 ? qz + g.D : (qz >= g.D ? qz - g.D : qz);
                } else {
                    valid = valid && qy >= 0 && qy < g.H && qz >= 0 && qz < g.D;
                }
                const long long sv =
                    valid ? qx + (long long)g.W * (qy + (long long)g.H * (qz + (long long)g.D * nb)) : 0;
                const __nv_bfloat16* srcB = in + sv * g.in_stride + g.in_off;
                const uint32_t b_base = smem_addr(st + a_bytes + j * b_tap_bytes) + kofs;
                for (int nc = part; nc < g.ci / 8; nc += 4)
                    cp_async16_ca(b_base + (uint32_t)nc * mns, srcB + 8 * nc, valid);
            }
            cp_async_commit();
            ++issued;
            if (ks >= 2) {
                cp_async_wait<2>();
                fence_async_shared();
                bar_arrive(&full[(ks - 2) % kTcStages]);
            }
        }
        cp_async_wait<0>();
        fence_async_shared();
        for (int ks = (issued >= 2 ? issued - 2 : 0); ks < issued; ++ks) bar_arrive(&full[ks % kTcStages]);
        if (!ok) {
            atomicOr(err, 64);
            *(volatile int*)abort_flag = 1;
        }
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issuer
        // A and B MN-major (transpose bits 15 and 16)
        const uint32_t idesc = idesc_bf16(kTcM, g.ci) | (1u << 15) | (1u << 16);
        const uint32_t k_step = 128u;  // stride between core matrices along K
        for (int ks = 0; ks < ksteps; ++ks) {
            const int s = ks % kTcStages;
            if (!bar_wait(&full[s], (ks / kTcStages) & 1) || *(volatile int*)abort_flag) {
                atomicOr(err, 64);
                *(volatile int*)abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_addr(stages + s * stage_bytes);
            for (int kk = 0; kk < kWgKT / 16; ++kk) {
                const uint32_t koff = (uint32_t)kk * 2u * k_step;
                // lbo_mn: which descriptor field carries the M/N stride
                const uint64_t ad = lbo_mn ? sdesc(a0 + koff, mns, k_step) : sdesc(a0 + koff, k_step, mns);
                for (int j = 0; j < ntap; ++j) {
                    const uint32_t b0 = a0 + (uint32_t)a_bytes + (uint32_t)(j * b_tap_bytes) + koff;
                    const uint64_t bd = lbo_mn ? sdesc(b0, mns, k_step) : sdesc(b0, k_step, mns);
                    mma_bf16_ss(tmem + (uint32_t)(j * g.ci), ad, bd, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
                }
            }
            mma_commit(&empty[s]);
        }
        mma_commit(done);
    }

    // ---------------------------------------------------------- epilogue
    if (warp < 4) {
        const bool ok = bar_wait(done, 0);
        tc_fence_after();
        if (!ok) atomicOr(err, 64);
        const int m = tid;  // output channel co of this lane
        const bool store = ok && !*(volatile int*)abort_flag && m < g.co;
        if (warp * 32 < g.co) {  // warps whose lanes are all padding skip the reads
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
            for (int j = 0; j < ntap; ++j) {
                float* dst = partial + (((long long)blockIdx.x * 27 + t0 + j) * g.co + m) * g.ci;
                for (int c = 0; c < g.ci; c += 16) {
                    uint32_t acc[16];
                    tmem_ld16(lane_base + (uint32_t)(j * g.ci + c), acc);
                    if (store) {
                        // an empty slice (no k-step) contributes zeros
                        float4* d4 = reinterpret_cast<float4*>(dst + c);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            d4[q] = ksteps > 0 ? make_float4(__uint_as_float(acc[4 * q]), __uint_as_float(acc[4 * q + 1]),
                                                             __uint_as_float(acc[4 * q + 2]),
                                                             __uint_as_float(acc[4 * q + 3]))
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

bool conv3d_wgrad_tc_supported(const ConvGeom& g) {
    const int tg = wg_taps_per_group(g.ci);
    return g.ci % 16 == 0 && g.co % 16 == 0 && g.co <= 128 && g.ci <= 256 && g.in_stride % 8 == 0 &&
           g.in_off % 8 == 0 && g.out_stride % 8 == 0 && g.out_off % 8 == 0 &&
           1024 + kTcStages * wg_stage_bytes(tg, g.ci) <= 227 * 1024;
}

long long wgrad_tc_workspace_floats(const ConvGeom& g) {
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const long long slice = wgrad_tc_slice(g);
    return ((M + slice - 1) / slice) * 27LL * g.co * g.ci;
}

cudaError_t launch_conv3d_wgrad_tc(const __nv_bfloat16* in, const __nv_bfloat16* dout, float* partial,
                                   const ConvGeom& g, int lbo_mn, int* err, int* nslices, cudaStream_t s) {
    const int tg = wg_taps_per_group(g.ci);
    const int smem = 1024 + kTcStages * wg_stage_bytes(tg, g.ci);
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const long long slice = wgrad_tc_slice(g);
    const int ns = (int)((M + slice - 1) / slice);
    *nslices = ns;
    k_conv3d_wgrad_tc<<<dim3(ns, (27 + tg - 1) / tg), kTcThreads, smem, s>>>(in, dout, partial, g, slice,
                                                                          (uint32_t)lbo_mn, err);
    return cudaGetLastError();
}

// ------------------------------------------------- forward, halo tiles
// The same convolution with the 27 taps read from one gathered neighbourhood
// instead of 27 gathers.  A CTA owns an 8 (x) x 16 (y) block of output
// voxels at one z of one batch item: M row r = 8 yr + xr.  Per chunk of CK
// input channels it stages the 10 x 18 x 3 halo of that block once, laid
// out so that every tap's A operand is the same K-major core-matrix layout
// at a shifted start address:
//   halo voxel (xi, yj, zk), channel group g (8 channels, 16 bytes) at
//   zk PZ + yj PY + g PC + xi 16,   PC = 10 x 16 B, PY = CK/8 PC, PZ = 18 PY;
//   tap (dx, dy, dz): start = (1+dz) PZ + (1+dy) PY + (1+dx) 16,
//   LBO = PC (next 8 channels), SBO = PY (next 8-row group = next y line).
// Only the weights stream, one tap per ring stage.  x is zero padded; y and
// z wrap (or are zero padded); rows outside the box are computed and dropped.
constexpr int kHaloX = 10, kHaloY = 18, kHaloZ = 3;
constexpr int kHaloStages = 4;                 // weight ring
constexpr int kHaloLag = kHaloStages - 2;      // weight stages in flight per thread

struct HaloShape {
    int CK, ncols, halo_bytes, w_bytes, smem;
};

__host__ __device__ inline HaloShape halo_shape(int ci, int co) {
    HaloShape s;
    const int cands[4] = {64, 48, 32, 16};
    s.CK = 16;
    for (int i = 0; i < 4; ++i) {
        const int ck = cands[i];
        if (ck > ci || ci % ck) continue;
        const int hb = kHaloX * kHaloY * kHaloZ * ck * 2, wb = co * ck * 2;
        if (1024 + hb + kHaloStages * wb <= 200 * 1024) { s.CK = ck; break; }
    }
    int c = 32;
    while (c < co) c <<= 1;
    s.ncols = c;
    s.halo_bytes = kHaloX * kHaloY * kHaloZ * s.CK * 2;
    s.w_bytes = co * s.CK * 2;
    s.smem = 1024 + s.halo_bytes + kHaloStages * s.w_bytes;
    return s;
}

__global__ void __launch_bounds__(kTcThreads) k_conv3d_halo(const __nv_bfloat16* __restrict__ in,
                                                            const __nv_bfloat16* __restrict__ w,
                                                            const float* __restrict__ bias,
                                                            __nv_bfloat16* __restrict__ out, ConvGeom g, int relu,
                                                            int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const HaloShape sh = halo_shape(g.ci, g.co);
    uint64_t* wfull = reinterpret_cast<uint64_t*>(smem);
    uint64_t* wempty = wfull + kHaloStages;
    uint64_t* hempty = wempty + kHaloStages;  // the halo may be refilled
    uint64_t* done = hempty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    unsigned char* halo = smem + 1024;
    unsigned char* wring = halo + sh.halo_bytes;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int CK = sh.CK, kg = CK / 8;
    const int nchunks = g.ci / CK;
    const int ksteps = 27 * nchunks;  // one tap of one chunk per step
    const uint32_t PC = 16u * kHaloX, PY = (uint32_t)kg * PC, PZ = (uint32_t)kHaloY * PY;
    // output block
    const int x0 = blockIdx.x * 8, y0 = blockIdx.y * 16;
    const int zb = blockIdx.z % g.D;
    const long long nb = blockIdx.z / g.D;

    if (tid == 0) {
        for (int s = 0; s < kHaloStages; ++s) {
            bar_init(&wfull[s], 128);
            bar_init(&wempty[s], 1);
        }
        bar_init(hempty, 1);
        bar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(sh.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ------------------------------------------------------ producers
        bool ok = true;
        int issued = 0, published = 0;
        const uint32_t halo_s = smem_addr(halo);
        const int nhalo = kHaloX * kHaloY * kHaloZ * kg;  // 16-byte chunks of one halo
        for (int ks = 0; ks < ksteps && ok; ++ks) {
            const int t = ks % 27, chunk = ks / 27;
            if (t == 0) {
                if (chunk > 0) {
                    // publish every step still in flight, then wait until the
                    // previous chunk's MMAs are done with the halo
                    cp_async_wait<0>();
                    fence_async_shared();
                    for (; published < issued; ++published) bar_arrive(&wfull[published % kHaloStages]);
                    if (!bar_wait(hempty, (chunk - 1) & 1)) { ok = false; break; }
                }
                const int c0 = chunk * CK;
                for (int e = tid; e < nhalo; e += 128) {
                    const int grp = e % kg;
                    const int v = e / kg;
                    const int xi = v % kHaloX, yj = (v / kHaloX) % kHaloY, zk = v / (kHaloX * kHaloY);
                    const int qx = x0 - 1 + xi;
                    int qy = y0 - 1 + yj, qz = zb - 1 + zk;
                    bool valid = qx >= 0 && qx < g.W;
                    if (g.periodic_yz) {
                        qy = ((qy % g.H) + g.H) % g.H;
                        qz = ((qz % g.D) + g.D) % g.D;
                    } else {
                        valid = valid && qy >= 0 && qy < g.H && qz >= 0 && qz < g.D;
                    }
                    const long long sv =
                        valid ? qx + (long long)g.W * (qy + (long long)g.H * (qz + (long long)g.D * nb)) : 0;
                    const uint32_t dst = halo_s + (uint32_t)zk * PZ + (uint32_t)yj * PY + (uint32_t)grp * PC +
                                         (uint32_t)xi * 16u;
                    cp_async16(dst, in + sv * g.in_stride + g.in_off + c0 + 8 * grp, valid);
                }
            }
            // the tap's weights into the ring
            const int s = ks % kHaloStages;
            if (ks >= kHaloStages && !bar_wait(&wempty[s], ((ks / kHaloStages) - 1) & 1)) { ok = false; break; }
            if (*(volatile int*)abort_flag) { ok = false; break; }
            const uint32_t wb = smem_addr(wring + s * sh.w_bytes);
            const __nv_bfloat16* wt = w + (long long)t * g.co * g.ci + chunk * CK;
            for (int e = tid; e < g.co * kg; e += 128) {
                const int n = e / kg, h = e % kg;
                cp_async16(wb + (uint32_t)(n >> 3) * (uint32_t)(kg * 128) + (uint32_t)h * 128u + (uint32_t)(n & 7) * 16u,
                           wt + (long long)n * g.ci + 8 * h, true);
            }
            cp_async_commit();
            ++issued;
            if (issued - published > kHaloLag) {
                // every earlier copy of this thread (the halo too) has landed
                cp_async_wait<kHaloLag>();
                fence_async_shared();
                bar_arrive(&wfull[published % kHaloStages]);
                ++published;
            }
        }
        cp_async_wait<0>();
        fence_async_shared();
        for (; published < issued; ++published) bar_arrive(&wfull[published % kHaloStages]);
        if (!ok) {
            atomicOr(err, 64);
            *(volatile int*)abort_flag = 1;
        }
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issuer
        const uint32_t idesc = idesc_bf16(kTcM, g.co);
        const uint32_t halo_s = smem_addr(halo);
        const uint32_t sbo_w = (uint32_t)kg * 128u;
        for (int ks = 0; ks < ksteps; ++ks) {
            const int s = ks % kHaloStages, t = ks % 27;
            if (!bar_wait(&wfull[s], (ks / kHaloStages) & 1) || *(volatile int*)abort_flag) {
                atomicOr(err, 64);
                *(volatile int*)abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;  // tap offset + 1
            const uint32_t a0 = halo_s + (uint32_t)dz * PZ + (uint32_t)dy * PY + (uint32_t)dx * 16u;
            const uint32_t b0 = smem_addr(wring + s * sh.w_bytes);
            for (int kk = 0; kk < CK / 16; ++kk) {
                const uint64_t ad = sdesc(a0 + (uint32_t)kk * 2u * PC, PC, PY);
                const uint64_t bd = sdesc(b0 + (uint32_t)kk * 256u, 128u, sbo_w);
                mma_bf16_ss(tmem, ad, bd, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&wempty[s]);
            if (t == 26) mma_commit(hempty);  // the chunk's halo is no longer read
        }
        mma_commit(done);
    }

    // ---------------------------------------------------------- epilogue
    if (warp < 4) {
        const bool ok = bar_wait(done, 0);
        tc_fence_after();
        if (!ok) atomicOr(err, 64);
        const int r = tid, x = x0 + (r & 7), y = y0 + (r >> 3);
        const bool store = ok && !*(volatile int*)abort_flag && x < g.W && y < g.H;
        const long long v = x + (long long)g.W * (y + (long long)g.H * (zb + (long long)g.D * nb));
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < g.co; c += 16) {
            uint32_t acc[16];
            tmem_ld16(lane_base + (uint32_t)c, acc);
            if (store) {
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float a = __uint_as_float(acc[2 * j]) + (bias ? bias[c + 2 * j] : 0.f);
                    float b = __uint_as_float(acc[2 * j + 1]) + (bias ? bias[c + 2 * j + 1] : 0.f);
                    if (relu) { a = fmaxf(a, 0.f); b = fmaxf(b, 0.f); }
                    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                    pk[j] = *reinterpret_cast<uint32_t*>(&h);
                }
                uint4* dst = reinterpret_cast<uint4*>(out + v * g.out_stride + g.out_off + c);
                dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(sh.ncols) : "memory");
    }
}

// ------------------------------------------ weight gradient, halo tiles
// dW[t][co][ci] over 8 x 16 voxel blocks: per block the input halo (as in
// the forward kernel) and the block's output gradient dO are staged once;
// every tap of the CTA's group is then a shifted descriptor into the halo.
// GEMM per tap: D[m = co][n = ci chunk] += sum over the block's voxels,
// A = dO (MN-major: 8 channels of a voxel in 16 bytes; voxel line yr of
// the block at yr PYo, channel group g at g 128, voxel xr at xr 16),
// B = the halo (MN-major; line stride PY, channel-group stride PC).  M is co
// padded to 128 (rows co.. are never read back).  A CTA accumulates in
// tensor memory over the blocks of its slice for TG taps x CN channels
// (<= 256 columns) and writes one partial per slice; a second kernel sums
// the slices in a fixed order.
constexpr int kWhStages = 2;  // double-buffered block stages

struct WgHaloShape {
    int CN, TG, ngroups, nchunks, ncols, halo_bytes, do_bytes, stage, smem;
};

__host__ __device__ inline WgHaloShape wgh_shape(int ci, int co) {
    WgHaloShape s;
    s.CN = ci <= 64 ? ci : (ci % 64 == 0 ? 64 : (ci % 48 == 0 ? 48 : (ci % 32 == 0 ? 32 : 16)));
    s.TG = 256 / s.CN;
    if (s.TG > 27) s.TG = 27;
    s.ngroups = (27 + s.TG - 1) / s.TG;
    s.nchunks = ci / s.CN;
    int c = 32;
    while (c < s.TG * s.CN) c <<= 1;
    s.ncols = c;
    s.halo_bytes = kHaloX * kHaloY * kHaloZ * s.CN * 2;
    // dO tile of 128 voxels x co, plus slack: the padded M rows of the A
    // descriptor reach up to 15 x 128 bytes past a line
    s.do_bytes = 128 * co * 2 + 2048;
    s.stage = s.halo_bytes + s.do_bytes;
    s.stage = (s.stage + 127) & ~127;
    s.smem = 1024 + kWhStages * s.stage;
    return s;
}

__host__ __device__ inline long long wgrad_halo_blocks(const ConvGeom& g) {
    return (long long)((g.W + 7) / 8) * ((g.H + 15) / 16) * g.D * g.N;
}

int wgrad_halo_slices(const ConvGeom& g) {
    const WgHaloShape s = wgh_shape(g.ci, g.co);
    long long ns = 304 / (s.ngroups * s.nchunks);
    if (ns < 1) ns = 1;
    const long long nb = wgrad_halo_blocks(g);
    return (int)(ns < nb ? ns : nb);
}

__global__ void __launch_bounds__(kTcThreads) k_conv3d_wgrad_halo(const __nv_bfloat16* __restrict__ in,
                                                                  const __nv_bfloat16* __restrict__ dout,
                                                                  float* __restrict__ partial, ConvGeom g,
                                                                  int blocks_per_slice, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const WgHaloShape sh = wgh_shape(g.ci, g.co);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kWhStages;
    uint64_t* done = empty + kWhStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    unsigned char* stages = smem + 1024;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int CN = sh.CN, kg = CN / 8;
    const int t0 = blockIdx.y * sh.TG;
    const int ntap = 27 - t0 < sh.TG ? 27 - t0 : sh.TG;
    const int c0 = blockIdx.z * CN;
    const long long nblocks = wgrad_halo_blocks(g);
    const long long b0 = (long long)blockIdx.x * blocks_per_slice;
    const long long b1 = b0 + blocks_per_slice < nblocks ? b0 + blocks_per_slice : nblocks;
    const int nb = b0 < b1 ? (int)(b1 - b0) : 0;
    const int bxn = (g.W + 7) / 8, byn = (g.H + 15) / 16;
    const uint32_t PC = 16u * kHaloX, PY = (uint32_t)kg * PC, PZ = (uint32_t)kHaloY * PY;
    const uint32_t PYo = (uint32_t)(g.co / 8) * 128u;

    if (tid == 0) {
        for (int s = 0; s < kWhStages; ++s) {
            bar_init(&full[s], 128);
            bar_init(&empty[s], 1);
        }
        bar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(sh.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ------------------------------------------------------ producers
        bool ok = true;
        int issued = 0;
        for (int i = 0; i < nb; ++i) {
            const int s = i % kWhStages;
            if (i >= kWhStages && !bar_wait(&empty[s], ((i / kWhStages) - 1) & 1)) { ok = false; break; }
            if (*(volatile int*)abort_flag) { ok = false; break; }
            long long b = b0 + i;
            const int bx = (int)(b % bxn);
            b /= bxn;
            const int by = (int)(b % byn);
            b /= byn;
            const int zb = (int)(b % g.D);
            const long long nbt = b / g.D;
            const int x0 = bx * 8, y0 = by * 16;
            const uint32_t st = smem_addr(stages + s * sh.stage);
            // halo of the input channels [c0, c0 + CN)
            for (int e = tid; e < kHaloX * kHaloY * kHaloZ * kg; e += 128) {
                const int grp = e % kg, v = e / kg;
                const int xi = v % kHaloX, yj = (v / kHaloX) % kHaloY, zk = v / (kHaloX * kHaloY);
                const int qx = x0 - 1 + xi;
                int qy = y0 - 1 + yj, qz = zb - 1 + zk;
                bool valid = qx >= 0 && qx < g.W;
                if (g.periodic_yz) {
                    qy = ((qy % g.H) + g.H) % g.H;
                    qz = ((qz % g.D) + g.D) % g.D;
                } else {
                    valid = valid && qy >= 0 && qy < g.H && qz >= 0 && qz < g.D;
                }
                const long long sv =
                    valid ? qx + (long long)g.W * (qy + (long long)g.H * (qz + (long long)g.D * nbt)) : 0;
                cp_async16_ca(st + (uint32_t)zk * PZ + (uint32_t)yj * PY + (uint32_t)grp * PC + (uint32_t)xi * 16u,
                              in + sv * g.in_stride + g.in_off + c0 + 8 * grp, valid);
            }
            // dO of the block's 128 voxels (zeros outside the box)
            const uint32_t dst0 = st + (uint32_t)sh.halo_bytes;
            for (int e = tid; e < 128 * (g.co / 8); e += 128) {
                const int grp = e % (g.co / 8), r = e / (g.co / 8);
                const int x = x0 + (r & 7), y = y0 + (r >> 3);
                const bool valid = x < g.W && y < g.H;
                const long long v = valid ? x + (long long)g.W * (y + (long long)g.H * (zb + (long long)g.D * nbt)) : 0;
                cp_async16(dst0 + (uint32_t)(r >> 3) * PYo + (uint32_t)grp * 128u + (uint32_t)(r & 7) * 16u,
                           dout + v * g.out_stride + g.out_off + 8 * grp, valid);
            }
            cp_async_commit();
            ++issued;
            // one block in flight behind this one (two stages)
            cp_async_wait<1>();
            fence_async_shared();
            if (i >= 1) bar_arrive(&full[(i - 1) % kWhStages]);
        }
        cp_async_wait<0>();
        fence_async_shared();
        if (issued >= 1) bar_arrive(&full[(issued - 1) % kWhStages]);
        if (!ok) {
            atomicOr(err, 64);
            *(volatile int*)abort_flag = 1;
        }
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issuer
        const uint32_t idesc = idesc_bf16(kTcM, CN) | (1u << 15) | (1u << 16);  // A, B MN-major
        for (int i = 0; i < nb; ++i) {
            const int s = i % kWhStages;
            if (!bar_wait(&full[s], (i / kWhStages) & 1) || *(volatile int*)abort_flag) {
                atomicOr(err, 64);
                *(volatile int*)abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t st = smem_addr(stages + s * sh.stage);
            const uint32_t a_base = st + (uint32_t)sh.halo_bytes;
            for (int kk = 0; kk < 8; ++kk) {  // two lines of 8 voxels per K = 16
                const uint64_t ad = sdesc(a_base + (uint32_t)(2 * kk) * PYo, PYo, 128u);
                for (int j = 0; j < ntap; ++j) {
                    const int t = t0 + j;
                    const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;
                    const uint32_t b = st + (uint32_t)dz * PZ + (uint32_t)(2 * kk + dy) * PY + (uint32_t)dx * 16u;
                    mma_bf16_ss(tmem + (uint32_t)(j * CN), ad, sdesc(b, PY, PC), idesc, (i > 0 || kk > 0) ? 1u : 0u);
                }
            }
            mma_commit(&empty[s]);
        }
        mma_commit(done);
    }

    // ---------------------------------------------------------- epilogue
    if (warp < 4) {
        const bool ok = bar_wait(done, 0);
        tc_fence_after();
        if (!ok) atomicOr(err, 64);
        const int m = tid;  // output channel of this lane
        const bool store = ok && !*(volatile int*)abort_flag && m < g.co;
        if (warp * 32 < g.co) {
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
            for (int j = 0; j < ntap; ++j) {
                float* dst = partial + (((long long)blockIdx.x * 27 + t0 + j) * g.co + m) * g.ci + c0;
                for (int c = 0; c < CN; c += 16) {
                    uint32_t acc[16];
                    tmem_ld16(lane_base + (uint32_t)(j * CN + c), acc);
                    if (store) {
                        float4* d4 = reinterpret_cast<float4*>(dst + c);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            d4[q] = nb > 0 ? make_float4(__uint_as_float(acc[4 * q]), __uint_as_float(acc[4 * q + 1]),
                                                         __uint_as_float(acc[4 * q + 2]), __uint_as_float(acc[4 * q + 3]))
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(sh.ncols) : "memory");
    }
}

// Taken for 16 input channels only: 16 taps share one staged block there.
// With more channels a CTA covers fewer taps (TG * CN <= 256 columns), the
// block is staged once per tap group, and the per-tap gather kernel measured
// faster (ci = 32: 0.086 vs 0.105 ms; ci = 48: 0.61 vs 1.69 ms at 4 x 48^3).
bool conv3d_wgrad_halo_supported(const ConvGeom& g) {
    const WgHaloShape s = wgh_shape(g.ci, g.co);
    return g.ci == 16 && g.co % 16 == 0 && g.co <= 128 && g.in_stride % 8 == 0 && g.in_off % 8 == 0 &&
           g.out_stride % 8 == 0 && g.out_off % 8 == 0 && s.smem <= 227 * 1024 && (long long)g.D * g.N <= (1LL << 30);
}

long long wgrad_halo_workspace_floats(const ConvGeom& g) {
    return (long long)wgrad_halo_slices(g) * 27LL * g.co * g.ci;
}

cudaError_t launch_conv3d_wgrad_halo(const __nv_bfloat16* in, const __nv_bfloat16* dout, float* partial,
                                     const ConvGeom& g, int* err, int* nslices, cudaStream_t s) {
    const WgHaloShape sh = wgh_shape(g.ci, g.co);
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_wgrad_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem);
    if (e != cudaSuccess) return e;
    const int ns = wgrad_halo_slices(g);
    const long long nb = wgrad_halo_blocks(g);
    const int per = (int)((nb + ns - 1) / ns);
    *nslices = ns;
    k_conv3d_wgrad_halo<<<dim3(ns, sh.ngroups, sh.nchunks), kTcThreads, sh.smem, s>>>(in, dout, partial, g, per, err);
    return cudaGetLastError();
}

bool conv3d_tc_supported(const ConvGeom& g) {
    return g.ci % 16 == 0 && g.co % 16 == 0 && g.co >= 16 && g.co <= 256 && g.in_stride % 8 == 0 &&
           g.in_off % 8 == 0 && g.out_stride % 8 == 0 && g.out_off % 8 == 0 && tc_shape(g.ci, g.co).smem <= 227 * 1024;
}

cudaError_t launch_conv3d_tc(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, __nv_bfloat16* out,
                             const ConvGeom& g, int relu, int* err, cudaStream_t s) {
    const HaloShape hs = halo_shape(g.ci, g.co);
    if (hs.smem <= 227 * 1024 && (long long)g.D * g.N <= 65535) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3d_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, hs.smem);
        if (e != cudaSuccess) return e;
        const dim3 grid((unsigned)((g.W + 7) / 8), (unsigned)((g.H + 15) / 16), (unsigned)(g.D * g.N));
        k_conv3d_halo<<<grid, kTcThreads, hs.smem, s>>>(in, w, bias, out, g, relu, err);
        return cudaGetLastError();
    }
    const TcShape sh = tc_shape(g.ci, g.co);
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem);
    if (e != cudaSuccess) return e;
    const long long M = (long long)g.N * g.D * g.H * g.W;
    const unsigned grid = (unsigned)((M + kTcM - 1) / kTcM);
    k_conv3d_tc<<<grid, kTcThreads, sh.smem, s>>>(in, w, bias, out, g, relu, err);
    return cudaGetLastError();
}

}  // namespace cl
