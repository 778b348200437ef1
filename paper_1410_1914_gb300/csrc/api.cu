// Host implementation of the C ABI declared in include/cl_lbm.h.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "device_util.cuh"
#include "handle.cuh"
#include "dsa.cuh"

using namespace cl;

namespace {

thread_local char g_msg[512] = "";
}  // namespace

namespace cl {
void set_msg(const char* where, cudaError_t e) {
    snprintf(g_msg, sizeof(g_msg), "%s: %s", where, cudaGetErrorString(e));
}
void set_msg_txt(const char* txt) { snprintf(g_msg, sizeof(g_msg), "%s", txt); }
cl_status from_cuda(cudaError_t e) { return e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA; }

// bit k set: phase code k carries the transported quantity
int transport_phases(const cl_params& p) {
    if (p.carrier == CL_CARRIER_PROTON) return 1 << 2;           // ionomer (Eq. 16)
    return (1 << 0) | (1 << 3) | (p.D_ionomer > 0 ? 1 << 2 : 0);  // pore, micropore (+ ionomer, Eq. 15)
}
// Half-way first-order sink (the pair of a link meets the wall value
// C_w = (g* + r g*) / (2 a_i); the link's share of the face's rate k C_w is
// a_i over the weight of all links crossing one face, cs^2 / 2):
// r = (cs^2 - k) / (cs^2 + k); on D3Q7 (cs^2 = 2w = 1/4) that is (2w - k) / (2w + k).
double reactive_factor_d(const cl_lbm* h) {
    const double cs2 = h->q == 19 ? 1.0 / 3.0 : 0.25;
    return (cs2 - h->k_lu) / (cs2 + h->k_lu);
}
float reactive_factor(const cl_lbm* h) { return (float)reactive_factor_d(h); }
// 1 - r = 2k / (cs^2 + k), formed directly: at nm voxels k_lu is ~1e-8..1e-10 of cs^2,
// and 1 - r taken from a rounded r would lose most of its digits (all of them in FP32)
double reactive_sink_d(const cl_lbm* h) {
    const double cs2 = h->q == 19 ? 1.0 / 3.0 : 0.25;
    return 2.0 * h->k_lu / (cs2 + h->k_lu);
}

MarchArgs make_margs(cl_lbm* h, int dst) {
    MarchArgs a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.px = h->px;
    a.z_chunk = h->z_chunk;
    a.prefetch = h->prefetch;
    a.chi = h->st[dst].chi;
    a.clo = h->st[dst].clo;
    for (int i = 0; i < 6; ++i) a.d[i] = h->st[dst].d[i];
    a.rfac = reactive_factor(h);
    a.rsink = (float)reactive_sink_d(h);
    a.rsink_d = reactive_sink_d(h);
    a.c_in = (float)h->p.c_in;
    a.c_out = (float)h->p.c_out;
    a.bc_in = h->p.bc_in;
    a.bc_out = h->p.bc_out;
    a.s_lo = h->s_lo;
    a.inv_lo = 1.0f / h->s_lo;
    a.s_d = h->s_d;
    a.inv_d = 1.0f / h->s_d;
    a.Csnap = h->Csnap_p;
    a.partials = h->partials;
    a.err = h->d_err;
    a.wait_limit = h->wait_limit;
    a.never_arrive = h->never_arrive;
    return a;
}

cl_status check_err_flag(cl_lbm* h) {
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (herr) {
        // reported once: the next call starts from a clean error word
        CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
        CK(cudaStreamSynchronize(h->s));
    }
    if (herr & 1) { set_msg_txt("phase code outside 0..3"); return CL_ERR_ARG; }
    if (herr & 2) { set_msg_txt("connectivity labelling exceeded its iteration bound"); return CL_ERR_TIMEOUT; }
    if (herr & 4) { set_msg_txt("diffusivity override not positive and finite on an active cell"); return CL_ERR_ARG; }
    if (herr & 8) { set_msg_txt("a plane load of the step kernel did not arrive within its wait bound"); return CL_ERR_TIMEOUT; }
    if (herr & 16) { set_msg_txt("dynamic shared memory of the step kernel is not 128-byte aligned"); return CL_ERR_CUDA; }
    return CL_OK;
}
}  // namespace cl

namespace {


// cuTensorMapEncodeTiled, fetched from the driver through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}


}  // namespace


namespace {

cl_status dalloc(cl_lbm* h, void** out, size_t bytes) {
    void* ptr = nullptr;
    if (bytes == 0) bytes = 16;
    if (h->p.alloc) {
        ptr = h->p.alloc(bytes, (void*)h->s, h->p.alloc_ctx);
        if (!ptr) { set_msg_txt("allocator callback returned NULL"); return CL_ERR_OOM; }
    } else {
        cudaError_t e = cudaMallocAsync(&ptr, bytes, h->s);
        if (e != cudaSuccess) { set_msg("cudaMallocAsync", e); return from_cuda(e); }
    }
    h->allocs.emplace_back(ptr, bytes);
    *out = ptr;
    return CL_OK;
}

template <class T>
cl_status dalloc_n(cl_lbm* h, T** out, long long n) {
    return dalloc(h, (void**)out, sizeof(T) * (size_t)n);
}

cudaMemcpyKind kind_in(int dev) { return dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int dev) { return dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }


StepArgs make_args(cl_lbm* h) {
    StepArgs a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.N = h->N;
    a.mask = h->mask;
    a.omega = h->omega;
    const double w = 0.125;
    a.rfac = reactive_factor(h);
    a.rfac_d = reactive_factor_d(h);
    a.rsink = (float)reactive_sink_d(h);
    a.rsink_d = reactive_sink_d(h);
    a.abb_in = (float)(2.0 * w * h->p.c_in);
    a.abb_out = (float)(2.0 * w * h->p.c_out);
    a.abb_in_d = 2.0 * w * h->p.c_in;
    a.abb_out_d = 2.0 * w * h->p.c_out;
    a.w_cin = (float)(w * h->p.c_in);
    a.w_cout = (float)(w * h->p.c_out);
    a.bc_in = h->p.bc_in;
    a.bc_out = h->p.bc_out;
    a.Csnap = h->Csnap;
    a.partials = h->partials;
    a.wide = h->wide;
    a.kscale = h->kscale;
    a.k_lu = h->k_lu;
    a.src = h->src;
    return a;
}


Q19Args make_args19(cl_lbm* h) {
    Q19Args a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.px = h->px19;
    a.NP = h->NP19;
    a.mask = h->mask19;
    a.react = h->react19;
    a.omega = h->omega19;
    a.rfac = reactive_factor(h);
    a.rfac_d = reactive_factor_d(h);
    a.rsink = (float)reactive_sink_d(h);
    a.rsink_d = reactive_sink_d(h);
    a.c_in = (float)h->p.c_in;
    a.c_out = (float)h->p.c_out;
    a.c_in_d = h->p.c_in;
    a.c_out_d = h->p.c_out;
    a.bc_in = h->p.bc_in;
    a.bc_out = h->p.bc_out;
    a.Csnap = h->Csnap;
    a.partials = h->partials;
    a.s_lo = h->s_lo;
    a.inv_lo = 1.0f / h->s_lo;
    a.s_d = h->s_d;
    a.inv_d = 1.0f / h->s_d;
    a.wide = h->wide;
    return a;
}


cl_status make_map(CUtensorMap* m, CUtensorMapDataType dt, int el, void* ptr, int px, int rows, int nz, int bx,
                   int by) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) { set_msg_txt("cuTensorMapEncodeTiled unavailable"); return CL_ERR_CUDA; }
    cuuint64_t dims[3] = {(cuuint64_t)px, (cuuint64_t)rows, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)px * el, (cuuint64_t)px * rows * el};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, dt, 3, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_msg, sizeof(g_msg), "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return CL_ERR_CUDA;
    }
    return CL_OK;
}

// TMA descriptors of both time levels for tiles of rw rows per warp
cl_status build_maps_rw(const cl_lbm* h, int rw, MarchMaps* maps) {
    const CUtensorMapDataType tT = h->el == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUtensorMapDataType tF = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const int R = h->ny + 2, px = h->px, nz = h->nz, el = h->el;
    const int hxl = 16 / el;
    const int bx = kBX / rw, by = kBY * rw;  // the tile of the march
    for (int b = 0; b < 2; ++b) {
        MarchMaps& m = maps[b];
        const MState& s = h->st[b];
        CKS(make_map(&m.chi, tF, 4, s.chi, px, R, nz, bx, by + 2));
        CKS(make_map(&m.clo, tT, el, s.clo, px, R, nz, bx, by + 2));
        CKS(make_map(&m.d3, tT, el, s.d[2], px, R, nz, bx, by + 2));
        CKS(make_map(&m.d4, tT, el, s.d[3], px, R, nz, bx, by + 2));
        CKS(make_map(&m.d1, tT, el, s.d[0], px, R, nz, bx, by));
        CKS(make_map(&m.d2, tT, el, s.d[1], px, R, nz, bx, by));
        CKS(make_map(&m.d5, tT, el, s.d[4], px, R, nz, bx, by));
        CKS(make_map(&m.d6, tT, el, s.d[5], px, R, nz, bx, by));
        CKS(make_map(&m.om, tF, 4, h->omega_p, px, R, nz, bx, by));
        CKS(make_map(&m.mk, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, h->mask_p, px, R, nz, bx, by));
        CKS(make_map(&m.chi_h, tF, 4, s.chi, px, R, nz, 4, by));
        CKS(make_map(&m.clo_h, tT, el, s.clo, px, R, nz, hxl, by));
        CKS(make_map(&m.d1_h, tT, el, s.d[0], px, R, nz, hxl, by));
        CKS(make_map(&m.d2_h, tT, el, s.d[1], px, R, nz, hxl, by));
    }
    return CL_OK;
}

cl_status build_maps(cl_lbm* h) { return build_maps_rw(h, h->tile_rw, h->maps); }

// Tiles of rw rows per warp over the box: (columns along x, rows along y).
// Columns cover the nx cells (the pitch beyond nx holds only inactive cells).
static void march_tiles(const cl_lbm* h, int rw, int& tx, int& ty) {
    const int bx = kBX / rw, by = kBY * rw;
    tx = (h->nx + bx - 1) / bx;
    ty = (h->ny + by - 1) / by;
}

// Blocks per z-column chosen so that the grid fills whole waves of resident
// blocks while keeping at least 8 planes per block.
static dim3 march_grid(cl_lbm* h, int rw, int* z_chunk) {
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int resident = nsm * march_blocks_per_sm(h->p.storage, rw);
    int tx = 1, ty = 1;
    march_tiles(h, rw, tx, ty);
    const int tiles = tx * ty;
    int best_gz = 1;
    double best = 1e30;
    const int gz_max = h->nz < 8 ? 1 : h->nz / 8;
    for (int gz = 1; gz <= gz_max && gz <= 4096; ++gz) {
        const int zc = (h->nz + gz - 1) / gz;
        const int g = (h->nz + zc - 1) / zc;
        const double blocks = (double)tiles * g;
        const double waves = ceil(blocks / resident);
        // time ~ waves * (planes per block + 2 halo planes)
        const double cost = waves * (zc + 2.0);
        if (cost < best - 1e-9) { best = cost; best_gz = g; }
    }
    const int zc = (h->nz + best_gz - 1) / best_gz;
    if (z_chunk) *z_chunk = zc;
    return dim3(tx, ty, (h->nz + zc - 1) / zc);
}

void choose_march_grid(cl_lbm* h) { h->mgrid = march_grid(h, h->tile_rw, &h->z_chunk); }

void drop_graphs(cl_lbm* h) {
    for (auto& g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = Graph();
    }
}

// Enqueue `n` steps (the last one with the fused reduction if `reduce`).
cl_status enqueue_steps(cl_lbm* h, long long n, bool reduce, cudaStream_t s, int* parity) {
    if (h->march) {
        for (long long i = 0; i < n; ++i) {
            const bool red = reduce && i == n - 1;
            MarchArgs a = make_margs(h, *parity ^ 1);
            CK(launch_march(h->p.storage, red, h->tile_rw, h->maps[*parity], a, h->mgrid, s));
            *parity ^= 1;
        }
    } else if (h->q19s) {
        Q19Args a = make_args19(h);
        for (long long i = 0; i < n; ++i) {
            const bool red = reduce && i == n - 1;
            CK(launch_step19s(h->p.storage, h->st19[*parity], h->st19[*parity ^ 1], a, red, s));
            *parity ^= 1;
        }
    } else if (h->q == 19) {
        Q19Args a = make_args19(h);
        for (long long i = 0; i < n; ++i) {
            const bool red = reduce && i == n - 1;
            CK(launch_step19(h->pop[*parity], h->pop[*parity ^ 1], a, red, s));
            *parity ^= 1;
        }
    } else {
        StepArgs a = make_args(h);
        for (long long i = 0; i < n; ++i) {
            const bool red = reduce && i == n - 1;
            CK(launch_step_fp32(h->pop[*parity], h->pop[*parity ^ 1], a, red, s));
            *parity ^= 1;
        }
    }
    if (reduce) CK(launch_finalize(h->partials, h->nblk_step, RED_N, h->d_red, s));
    return CL_OK;
}

// A graph of K steps (K even, so the buffer parity returns) starting at the
// current parity; cached.
cl_status get_graph(cl_lbm* h, long long K, bool reduce, cudaGraphExec_t* out) {
    for (auto& g : h->graphs)
        if (g.exec && g.parity == h->cur && g.K == K && g.reduce == reduce) { *out = g.exec; return CL_OK; }
    Graph* slot = nullptr;
    for (auto& g : h->graphs)
        if (!g.exec) { slot = &g; break; }
    if (!slot) { drop_graphs(h); slot = &h->graphs[0]; }
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int par = h->cur;
    cl_status st = enqueue_steps(h, K, reduce, h->cap, &par);
    if (st == CL_OK && reduce) {
        cudaError_t e = cudaMemcpyAsync(h->h_red, h->d_red, sizeof(double) * RED_N, cudaMemcpyDeviceToHost, h->cap);
        if (e != cudaSuccess) { set_msg("capture memcpy", e); st = from_cuda(e); }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (st != CL_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) { set_msg("cudaStreamEndCapture", e); return from_cuda(e); }
    e = cudaGraphInstantiate(&slot->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { set_msg("cudaGraphInstantiate", e); slot->exec = nullptr; return from_cuda(e); }
    slot->parity = h->cur;
    slot->K = K;
    slot->reduce = reduce;
    *out = slot->exec;
    return CL_OK;
}

cl_status need_structure(cl_lbm* h) {
    if (!h) { set_msg_txt("NULL handle"); return CL_ERR_ARG; }
    if (!h->have_structure) { set_msg_txt("no structure loaded"); return CL_ERR_STATE; }
    return CL_OK;
}


// stats + dt + omega, shared by set_structure and set_diffusivity
cl_status derive_relaxation(cl_lbm* h, bool with_dp) {
    double* stat_out = h->d_red + 8;  // 7 slots
    CK(launch_stats(h->phase, h->mask, h->D, with_dp ? h->dp : nullptr, h->N, h->nx, transport_phases(h->p),
                    h->partials, h->nblk_stats, stat_out, h->s));
    double st[7];
    CK(cudaMemcpyAsync(st, stat_out, sizeof(st), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    h->info.n_cells = h->N;
    h->info.n_transport = (long long)st[0];
    h->info.n_active = (long long)st[1];
    h->info.n_wall_links = (long long)st[2];
    h->info.n_react_links = (long long)st[3];
    if (with_dp) h->info.mean_pore_diameter_m = st[5] > 0 ? st[4] / st[5] : 0.0;
    if (h->info.n_active == 0) { set_msg_txt("no transport cell is connected to the inlet plane"); return CL_ERR_NO_PATH; }
    h->D_max = st[6];
    if (!(h->D_max > 0) || !isfinite(h->D_max)) { set_msg_txt("largest diffusivity is not positive"); return CL_ERR_ARG; }
    // Eq. 24: D = cs^2 (tau - 1/2) dx^2 / dt, cs^2 = 1/4 (D3Q7) or 1/3 (D3Q19); tau_ref at D_max.
    const double cs2 = h->q == 19 ? 1.0 / 3.0 : 0.25;
    h->dt = (h->p.tau_ref - 0.5) * cs2 * h->p.dx_m * h->p.dx_m / h->D_max;
    h->k_lu = h->p.k_ms * h->dt / h->p.dx_m;
    h->info.D_b = h->D_b;
    h->info.D_max = h->D_max;
    h->info.dt_s = h->dt;
    h->info.k_lu = h->k_lu;
    CK(launch_omega(h->active, h->D, h->N, h->p.tau_ref, stat_out + 6, h->omega, h->s));
    if (h->march)
        CK(launch_pad_static(h->mask, h->omega, h->nx, h->ny, h->nz, h->px, h->mask_p, h->omega_p, h->s));
    if (h->q == 19) {
        CK(launch_pad_omega19(h->omega, h->nx, h->ny, h->nz, h->px19, h->omega19, h->s));
        // wall and reactive link counts of the 19-velocity stencil
        double* lc = h->d_red + 8;
        CK(launch_linkcount19(h->mask19, h->react19, h->NP19, h->partials, h->nblk_stats, lc, h->s));
        double cnt[2];
        CK(cudaMemcpyAsync(cnt, lc, sizeof(cnt), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        h->info.n_wall_links = (long long)cnt[0];
        h->info.n_react_links = (long long)cnt[1];
    }
    drop_graphs(h);  // the reactive factor is baked into captured kernel arguments
    return CL_OK;
}

// FP16 scales from the largest concentration magnitude (C < 2^E):
// low word scaled by 2^(38 - E), deviations by 2^(14 - E).
void set_scales(cl_lbm* h, double cmax) {
    if (h->p.storage != CL_STORE_FP16DEV) { h->s_lo = h->s_d = 1.f; return; }
    int E = 0;
    frexp(cmax > 0 ? cmax : 1.0, &E);  // cmax < 2^E
    h->s_lo = ldexpf(1.f, 38 - E);
    h->s_d = ldexpf(1.f, 14 - E);
}

cl_status do_init(cl_lbm* h, const float* C0dev) {
    h->cur = 0;
    double cmax = fmax(fabs(h->p.c_in), fabs(h->p.c_out));
    if (C0dev) {
        double* out = h->d_red + 15;
        CK(launch_absmax(C0dev, h->N, h->partials, h->nblk_stats, out, h->s));
        double m = 0;
        CK(cudaMemcpyAsync(&m, out, sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        cmax = fmax(cmax, m);
    }
    if (h->march) {
        set_scales(h, cmax);
        drop_graphs(h);
        // the other time level must hold zeros on inactive slots: the kernel never writes them
        const MState& o = h->st[1];
        CK(cudaMemsetAsync(o.chi, 0, sizeof(float) * h->NP, h->s));
        CK(cudaMemsetAsync(o.clo, 0, (size_t)h->el * h->NP, h->s));
        for (int i = 0; i < 6; ++i) CK(cudaMemsetAsync(o.d[i], 0, (size_t)h->el * h->NP, h->s));
        MarchArgs a = make_margs(h, 0);
        CK(launch_state_init(h->p.storage, a, h->mask_p, C0dev, h->s));
    } else if (h->q19s) {
        set_scales(h, cmax);
        drop_graphs(h);  // the scales are baked into captured kernel arguments
        // the other time level must hold zeros on inactive cells: sectors without an active cell are never written
        const Q19State& o = h->st19[1];
        CK(cudaMemsetAsync(o.hl, 0, sizeof(float2) * (size_t)h->NP19, h->s));
        CK(cudaMemsetAsync(o.d, 0, (size_t)h->el * 18 * h->NP19, h->s));
        Q19Args a = make_args19(h);
        CK(launch_init19s(h->p.storage, h->st19[0], a, C0dev, h->s));
    } else if (h->q == 19) {
        CK(cudaMemsetAsync(h->pop[1], 0, sizeof(float) * 19 * (size_t)h->NP19, h->s));
        CK(launch_init19(h->pop[0], h->mask19, C0dev, h->nx, h->ny, h->nz, h->px19, h->p.c_in, h->p.c_out, h->Csnap,
                         h->s));
    } else {
        CK(cudaMemsetAsync(h->pop[1], 0, sizeof(float) * 7 * (size_t)h->N, h->s));
        CK(launch_init_fp32(h->pop[0], h->mask, C0dev, h->nx, h->ny, h->nz, h->p.c_in, h->p.c_out, h->Csnap,
                            h->q == 7 ? h->src : nullptr, h->s));
    }
    h->step = 0;
    return CL_OK;
}

cl_status plane_readout(cl_lbm* h, double* tot /* [5] */) {
    if (h->march) {
        MarchArgs a = make_margs(h, h->cur);
        CK(launch_state_readout(h->p.storage, a, h->mask_p, h->d_plane, h->s));
    } else if (h->q19s) {
        Q19Args a = make_args19(h);
        CK(launch_readout19s(h->p.storage, h->st19[h->cur], a, h->d_plane, h->s));
    } else if (h->q == 19) {
        Q19Args a = make_args19(h);
        CK(launch_readout19(h->pop[h->cur], a, h->d_plane, h->s));
    } else {
        StepArgs a = make_args(h);
        CK(launch_readout_fp32(h->pop[h->cur], a, h->d_plane, h->s));
    }
    double* hp = h->h_red + 16;
    CK(cudaMemcpyAsync(hp, h->d_plane, sizeof(double) * 5 * h->nx, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    for (int k = 0; k < 5; ++k) tot[k] = 0.0;
    for (int x = 0; x < h->nx; ++x)
        for (int k = 0; k < 5; ++k) tot[k] += hp[5 * x + k];
    return CL_OK;
}

}  // namespace

namespace cl {
cl_status build_march_maps(const cl_lbm* h, int rw, MarchMaps* maps) { return build_maps_rw(h, rw, maps); }
}  // namespace cl

extern "C" {

void cl_params_default(cl_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->dx_m = 1e-9;
    p->T_K = 353.0;
    p->p_atm = 1.0;
    p->M_kgmol = 0.032;
    p->bc_in = CL_BC_DIRICHLET;
    p->bc_out = CL_BC_DIRICHLET;
    p->c_in = 1.0;
    p->c_out = 0.0;
    p->tau_ref = 1.0;
    p->storage = CL_STORE_FP32;
    p->react_rule = CL_REACT_GIVEN;
    p->check_every = 1000;
    p->tol_flux = 1e-4;
    p->tol_rel = 1e-4;
    p->max_steps = 10000000;
}

const char* cl_status_str(cl_status s) {
    switch (s) {
        case CL_OK: return "CL_OK";
        case CL_ERR_ARG: return "CL_ERR_ARG";
        case CL_ERR_OOM: return "CL_ERR_OOM";
        case CL_ERR_CUDA: return "CL_ERR_CUDA";
        case CL_ERR_STATE: return "CL_ERR_STATE";
        case CL_ERR_DIVERGED: return "CL_ERR_DIVERGED";
        case CL_ERR_NOT_CONVERGED: return "CL_ERR_NOT_CONVERGED";
        case CL_ERR_NO_PATH: return "CL_ERR_NO_PATH";
        case CL_ERR_TIMEOUT: return "CL_ERR_TIMEOUT";
    }
    return "CL_ERR_UNKNOWN";
}

const char* cl_last_error_message(void) { return g_msg; }

double cl_henry_constant(double T_K) { return 1.01325e-1 * exp(-666.0 / T_K + 14.1); }  // Eq. 11

double cl_ionomer_o2_diffusivity(double T_K) { return 1e-10 * (0.1543 * (T_K - 273.0) - 1.65); }  // Eq. 13

double cl_ionomer_effective_diffusivity(double T_K) {
    const double R = 8.314462618;
    return cl_ionomer_o2_diffusivity(T_K) * R * T_K / cl_henry_constant(T_K);  // Eq. 10: C_e = C RT/H
}

double cl_tafel_rate_constant(double i0m, double alpha, double phi_e, double T_K, double c_ref) {
    const double R = 8.314462618, F = 96485.33212;
    return i0m * exp(alpha * F * phi_e / (R * T_K)) * (R * T_K / cl_henry_constant(T_K)) / (4.0 * F * c_ref);
}

const char* cl_version(void) { return "cl_lbm 0.3 (D3Q7 and D3Q19, sm_103a)"; }

cl_status cl_lbm_create(cl_handle* out, const cl_params* p) {
    if (!out || !p) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || N >= (1LL << 31)) { set_msg_txt("box size out of range"); return CL_ERR_ARG; }
    if (p->ny > 65535 || p->nz > 65535) { set_msg_txt("ny and nz must be <= 65535"); return CL_ERR_ARG; }
    if (!(p->dx_m > 0) || !(p->tau_ref > 0.5) || !(p->T_K > 0) || !(p->M_kgmol > 0)) { set_msg_txt("dx_m, T_K, M_kgmol must be > 0 and tau_ref > 0.5"); return CL_ERR_ARG; }
    if (p->D_bulk <= 0 && !(p->p_atm > 0)) { set_msg_txt("p_atm must be > 0 when D_bulk comes from Eq. 7"); return CL_ERR_ARG; }
    if (p->D_ionomer < 0 || p->k_ms < 0) { set_msg_txt("D_ionomer and k_ms must be >= 0"); return CL_ERR_ARG; }
    if ((p->bc_in != 0 && p->bc_in != 1) || (p->bc_out != 0 && p->bc_out != 1)) { set_msg_txt("bad boundary type"); return CL_ERR_ARG; }
    if (p->storage != CL_STORE_FP32 && p->storage != CL_STORE_FP16DEV && p->storage != CL_STORE_FP32POP) { set_msg_txt("bad storage mode"); return CL_ERR_ARG; }
    if (p->react_rule != CL_REACT_GIVEN && p->react_rule != CL_REACT_ALL_PORE_SOLID &&
        p->react_rule != CL_REACT_IONOMER_SOLID) { set_msg_txt("bad react_rule"); return CL_ERR_ARG; }
    if (p->react_rule == CL_REACT_IONOMER_SOLID && p->lattice != CL_LATTICE_D3Q7) {
        set_msg_txt("the ionomer-solid reaction rule is a D3Q7 rule");
        return CL_ERR_ARG;
    }
    if (p->carrier != CL_CARRIER_O2 && p->carrier != CL_CARRIER_PROTON) { set_msg_txt("bad carrier"); return CL_ERR_ARG; }
    if (p->lattice != CL_LATTICE_D3Q7 && p->lattice != CL_LATTICE_D3Q19) { set_msg_txt("bad lattice"); return CL_ERR_ARG; }
    if (p->ionomer_o2 && (p->carrier != CL_CARRIER_O2 || !(cl_ionomer_o2_diffusivity(p->T_K) > 0))) {
        set_msg_txt("ionomer_o2 needs the O2 carrier and T_K > 283.7 K (Eq. 13)");
        return CL_ERR_ARG;
    }
    if (p->carrier == CL_CARRIER_PROTON && !(p->D_ionomer > 0 && p->k_ms == 0)) {
        set_msg_txt("the proton carrier needs D_ionomer > 0 (its conductivity) and k_ms = 0");
        return CL_ERR_ARG;
    }
    if (p->check_every < 2 || (p->check_every & 1)) { set_msg_txt("check_every must be even and >= 2"); return CL_ERR_ARG; }
    if ((p->alloc == nullptr) != (p->free == nullptr)) { set_msg_txt("alloc and free must both be set or both NULL"); return CL_ERR_ARG; }
    if (!(fabs(p->c_in) < 1e30) || !(fabs(p->c_out) < 1e30)) { set_msg_txt("boundary concentrations must be finite"); return CL_ERR_ARG; }

    cl_lbm* h = new cl_lbm();
    h->p = *p;
    if (p->ionomer_o2) h->p.D_ionomer = cl_ionomer_effective_diffusivity(p->T_K);  // Eq. 10-15
    h->nx = p->nx; h->ny = p->ny; h->nz = p->nz; h->N = N;
    h->q = p->lattice == CL_LATTICE_D3Q19 ? 19 : 7;
    h->march = h->q == 7 && p->storage != CL_STORE_FP32POP;
    h->q19s = h->q == 19 && p->storage != CL_STORE_FP32POP;
    // the population kernels switch to 64-bit element offsets once 32 bits
    // no longer hold every offset; this override takes that path on any box
    if (const char* e = getenv("CL_LBM_WIDE_INDEX")) h->wide = atoi(e) != 0;
    h->el = p->storage == CL_STORE_FP16DEV ? 2 : 4;
    h->s = (cudaStream_t)p->cuda_stream;
    memset(&h->info, 0, sizeof(h->info));
    cl_status st = CL_OK;
    auto fail = [&](cl_status s) { cl_lbm_destroy(h); return s; };
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { set_msg("cudaStreamCreate", e); return fail(from_cuda(e)); }

    int nblk_alloc = 0;
    if (h->march) {
        // row pitch: a multiple of 16 cells, so that every row starts on a
        // 32-byte sector of the f16 arrays and the lanes that store a sector
        // never reach past the row; at least one tile.  The last tile may
        // overhang the pitch: TMA zero-fills that part without touching
        // memory, and no lane stores there (a sector with an active cell
        // lies inside the pitch)
        h->px = std::max((h->nx + 15) / 16 * 16, kBX);
        // L2 prefetch pays off for the FP32 state (memory-latency bound), not for FP16 (issue bound)
        h->prefetch = p->storage == CL_STORE_FP32 ? 2 : 0;
        if (const char* e = getenv("CL_LBM_PREFETCH")) h->prefetch = atoi(e);  // tuning override
        h->NP = (long long)h->px * (h->ny + 2) * h->nz;
        h->tile_rw = march_auto_rows(h->nx, h->ny, h->p.storage);
        choose_march_grid(h);
        h->nblk_step = (int)(h->mgrid.x * h->mgrid.y * h->mgrid.z);
        // reduction partials for the largest grid of any tile shape (cl_lbm_set_tile_rows)
        for (int rw = 1; rw <= kRowsMax; rw *= 2) {
            const dim3 g = march_grid(h, rw, nullptr);
            nblk_alloc = std::max(nblk_alloc, (int)(g.x * g.y * g.z));
        }
    } else if (h->q == 19) {
        // row pitch a multiple of 32 cells: every row starts on a 128-byte
        // line, and the 8 lanes of each 32-byte sector hold one row's cells
        h->px19 = (h->nx + 31) / 32 * 32;
        h->NP19 = (long long)h->px19 * h->ny * h->nz;
        Q19Args a;
        a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.px = h->px19;
        h->nblk_step = h->q19s ? step19s_blocks(h->px19, h->ny, h->nz) : step19_blocks(a);
    } else {
        StepArgs a;
        a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
        h->nblk_step = step_fp32_blocks(a);
    }
    h->nblk_stats = 152 * 4;
    nblk_alloc = std::max(nblk_alloc, h->nblk_step);
    const long long npart = (long long)nblk_alloc * RED_N > (long long)h->nblk_stats * 8
                                ? (long long)nblk_alloc * RED_N : (long long)h->nblk_stats * 8;
    if ((st = dalloc_n(h, &h->phase, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->react, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->active, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->touch, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->labels, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->d_err, 4)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->D, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->dp, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->omega, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->mask, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->fbuf, N)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->partials, npart)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->d_red, 16)) != CL_OK) return fail(st);
    if ((st = dalloc_n(h, &h->d_plane, 5LL * h->nx)) != CL_OK) return fail(st);
    if (h->march) {
        for (int b = 0; b < 2; ++b) {
            if ((st = dalloc_n(h, &h->st[b].chi, h->NP)) != CL_OK) return fail(st);
            if ((st = dalloc(h, &h->st[b].clo, (size_t)h->el * h->NP)) != CL_OK) return fail(st);
            for (int i = 0; i < 6; ++i)
                if ((st = dalloc(h, &h->st[b].d[i], (size_t)h->el * h->NP)) != CL_OK) return fail(st);
        }
        if ((st = dalloc_n(h, &h->mask_p, h->NP)) != CL_OK) return fail(st);
        if ((st = dalloc_n(h, &h->omega_p, h->NP)) != CL_OK) return fail(st);
        if ((st = dalloc_n(h, &h->Csnap_p, h->NP)) != CL_OK) return fail(st);
        if ((st = build_maps(h)) != CL_OK) return fail(st);
        e = cudaMemsetAsync(h->mask_p, 0, sizeof(uint16_t) * h->NP, h->s);
        if (e != cudaSuccess) { set_msg("memset", e); return fail(from_cuda(e)); }
    } else if (h->q == 19) {
        const long long NP = h->NP19;
        if (h->q19s) {
            for (int b = 0; b < 2; ++b) {
                if ((st = dalloc_n(h, &h->st19[b].hl, NP)) != CL_OK) return fail(st);
                if ((st = dalloc(h, &h->st19[b].d, (size_t)h->el * 18 * NP)) != CL_OK) return fail(st);
            }
        } else {
            if ((st = dalloc_n(h, &h->pop[0], 19 * NP)) != CL_OK) return fail(st);
            if ((st = dalloc_n(h, &h->pop[1], 19 * NP)) != CL_OK) return fail(st);
        }
        if ((st = dalloc_n(h, &h->Csnap, NP)) != CL_OK) return fail(st);
        if ((st = dalloc_n(h, &h->mask19, NP)) != CL_OK) return fail(st);
        if ((st = dalloc_n(h, &h->react19, NP)) != CL_OK) return fail(st);
        if ((st = dalloc_n(h, &h->omega19, NP)) != CL_OK) return fail(st);
        e = cudaMemsetAsync(h->mask19, 0, sizeof(uint32_t) * (size_t)NP, h->s);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            if (h->q19s) {
                e = cudaMemsetAsync(h->st19[b].hl, 0, sizeof(float2) * (size_t)NP, h->s);
                if (e == cudaSuccess) e = cudaMemsetAsync(h->st19[b].d, 0, (size_t)h->el * 18 * NP, h->s);
            } else {
                e = cudaMemsetAsync(h->pop[b], 0, sizeof(float) * 19 * (size_t)NP, h->s);
            }
        }
        if (e != cudaSuccess) { set_msg("memset", e); return fail(from_cuda(e)); }
    } else {
        if ((st = dalloc_n(h, &h->pop[0], 7 * N)) != CL_OK) return fail(st);
        if ((st = dalloc_n(h, &h->pop[1], 7 * N)) != CL_OK) return fail(st);
        if ((st = dalloc_n(h, &h->Csnap, N)) != CL_OK) return fail(st);
        e = cudaMemsetAsync(h->pop[0], 0, sizeof(float) * 7 * (size_t)N, h->s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->pop[1], 0, sizeof(float) * 7 * (size_t)N, h->s);
        if (e != cudaSuccess) { set_msg("memset", e); return fail(from_cuda(e)); }
    }
    e = cudaMallocHost(&h->h_red, sizeof(double) * (16 + 5 * (size_t)h->nx));
    if (e != cudaSuccess) { set_msg("cudaMallocHost", e); return fail(from_cuda(e)); }
    e = cudaMemsetAsync(h->mask, 0, sizeof(uint16_t) * (size_t)N, h->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) { set_msg("initial memset", e); return fail(from_cuda(e)); }
    *out = h;
    return CL_OK;
}

void cl_lbm_destroy(cl_handle h) {
    if (!h) return;
    drop_graphs(h);
    cudaStreamSynchronize(h->s);
    for (auto& pr : h->allocs) {
        if (h->p.free) h->p.free(pr.first, pr.second, (void*)h->s, h->p.alloc_ctx);
        else cudaFreeAsync(pr.first, h->s);
    }
    cudaStreamSynchronize(h->s);
    if (h->h_red) cudaFreeHost(h->h_red);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}

cl_status cl_lbm_set_structure(cl_handle h, const uint8_t* phase, const uint8_t* reactive_faces, int ptr_is_device) {
    if (!h || !phase) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    const size_t N = (size_t)h->N;
    CK(cudaMemcpyAsync(h->phase, phase, N, kind_in(ptr_is_device), h->s));
    h->have_react = reactive_faces != nullptr;
    if (reactive_faces) CK(cudaMemcpyAsync(h->react, reactive_faces, N, kind_in(ptr_is_device), h->s));
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    CK(launch_validate(h->phase, h->N, h->d_err, h->s));
    CKS(check_err_flag(h));
    h->have_structure = false;
    h->kscale = nullptr;  // per-cell kinetics and sources belong to the previous structure
    h->src = nullptr;
    h->src_sum = 0.0;
    CK(launch_percolation(h->phase, h->nx, h->ny, h->nz, transport_phases(h->p), h->labels, h->touch, h->active,
                          h->d_err, h->s));
    CKS(check_err_flag(h));
    // Eq. 7 unless the bulk value is given
    h->D_b = h->p.D_bulk > 0 ? h->p.D_bulk : 0.22e-4 * pow(h->p.T_K / 293.2, 1.5) / h->p.p_atm;
    CK(launch_diffusivity(h->phase, h->active, h->nx, h->ny, h->nz, h->p.dx_m, h->p.T_K, h->p.M_kgmol, h->D_b,
                          h->p.D_ionomer, h->p.knudsen, nullptr, h->D, h->dp, nullptr, h->s));
    CK(launch_masks(h->phase, h->active, h->have_react ? h->react : nullptr, h->p.react_rule, h->nx, h->ny,
                    h->nz, h->mask, h->s));
    if (h->q == 19)
        CK(launch_masks19(h->phase, h->active, h->have_react ? h->react : nullptr, h->p.react_rule, h->nx, h->ny,
                          h->nz, h->px19, h->mask19, h->react19, h->s));
    CKS(derive_relaxation(h, true));
    CKS(do_init(h, nullptr));
    CK(cudaStreamSynchronize(h->s));
    h->have_structure = true;
    return CL_OK;
}

cl_status cl_lbm_set_diffusivity(cl_handle h, const double* D, int ptr_is_device) {
    CKS(need_structure(h));
    if (!D) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    CK(cudaMemcpyAsync(h->dp, D, sizeof(double) * (size_t)h->N, kind_in(ptr_is_device), h->s));
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    CK(launch_diffusivity(h->phase, h->active, h->nx, h->ny, h->nz, h->p.dx_m, h->p.T_K, h->p.M_kgmol, h->D_b,
                          h->p.D_ionomer, h->p.knudsen, h->dp, h->D, nullptr, nullptr, h->s));
    CK(launch_check_positive(h->active, h->D, h->N, h->d_err, h->s));
    CKS(check_err_flag(h));
    CKS(derive_relaxation(h, false));
    CKS(do_init(h, nullptr));
    CK(cudaStreamSynchronize(h->s));
    return CL_OK;
}

cl_status cl_lbm_init(cl_handle h, const float* C0, int ptr_is_device) {
    CKS(need_structure(h));
    const float* src = nullptr;
    if (C0) {
        if (ptr_is_device) src = C0;
        else {
            CK(cudaMemcpyAsync(h->fbuf, C0, sizeof(float) * (size_t)h->N, cudaMemcpyHostToDevice, h->s));
            src = h->fbuf;
        }
    }
    CKS(do_init(h, src));
    CK(cudaStreamSynchronize(h->s));
    return CL_OK;
}

cl_status cl_lbm_step(cl_handle h, long long nsteps) {
    CKS(need_structure(h));
    if (nsteps < 0) { set_msg_txt("nsteps < 0"); return CL_ERR_ARG; }
    const long long G = 64;  // steps per captured graph (even)
    long long left = nsteps;
    if (left >= G) {
        cudaGraphExec_t g;
        CKS(get_graph(h, G, false, &g));
        while (left >= G) {
            CK(cudaGraphLaunch(g, h->s));
            left -= G;
        }
    }
    int par = h->cur;
    CKS(enqueue_steps(h, left, false, h->s, &par));
    h->cur = par;
    h->step += nsteps;
    CK(cudaGetLastError());
    return CL_OK;
}

cl_status cl_lbm_set_wait_test(cl_handle h, long long wait_limit_clocks, int never_arrive) {
    if (!h) { set_msg_txt("NULL handle"); return CL_ERR_ARG; }
    if (wait_limit_clocks < 0) { set_msg_txt("wait_limit_clocks < 0"); return CL_ERR_ARG; }
    if (never_arrive && wait_limit_clocks == 0) {
        set_msg_txt("never_arrive needs a wait limit (a few hundred clocks)");
        return CL_ERR_ARG;
    }
    h->wait_limit = wait_limit_clocks;
    h->never_arrive = never_arrive ? 1 : 0;
    drop_graphs(h);  // the wait settings are baked into captured kernel arguments
    return CL_OK;
}

cl_status cl_lbm_set_tile_rows(cl_handle h, int rows, int* rows_out) {
    if (!h) { set_msg_txt("NULL handle"); return CL_ERR_ARG; }
    if (!h->march) { set_msg_txt("tile shapes apply to the (C, delta) storage modes"); return CL_ERR_STATE; }
    if (rows != 0 && rows != 1 && rows != 2 && rows != 4) { set_msg_txt("rows must be 0, 1, 2 or 4"); return CL_ERR_ARG; }
    const int rw = rows ? rows : march_auto_rows(h->nx, h->ny, h->p.storage);
    if (rw != h->tile_rw) {
        // queued launches carry their own copies of the descriptors and grid
        h->tile_rw = rw;
        CKS(build_maps(h));
        choose_march_grid(h);
        h->nblk_step = (int)(h->mgrid.x * h->mgrid.y * h->mgrid.z);
        drop_graphs(h);
    }
    if (rows_out) *rows_out = h->tile_rw;
    return CL_OK;
}

cl_status cl_lbm_solve(cl_handle h, cl_solve_info* info) {
    if (!h) { set_msg_txt("NULL handle"); return CL_ERR_ARG; }
    return cl_lbm_solve_budget(h, h->p.max_steps, info);
}

cl_status cl_lbm_solve_budget(cl_handle h, long long max_steps, cl_solve_info* info) {
    CKS(need_structure(h));
    if (max_steps < 0) { set_msg_txt("max_steps < 0"); return CL_ERR_ARG; }
    auto t0 = std::chrono::steady_clock::now();
    const long long K = h->p.check_every;
    cudaGraphExec_t g;
    CKS(get_graph(h, K, true, &g));
    const bool track_deff = h->p.bc_in == CL_BC_DIRICHLET && h->p.bc_out == CL_BC_DIRICHLET && h->p.c_in != h->p.c_out;
    double q_prev = NAN, dq_prev = NAN;
    int nchecks = 0, quiet = 0;
    cl_solve_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.rel_change = INFINITY;
    cl_status result = CL_ERR_NOT_CONVERGED;
    while (inf.steps + K <= max_steps) {
        CK(cudaGraphLaunch(g, h->s));
        CK(cudaStreamSynchronize(h->s));
        inf.steps += K;
        h->step += K;
        const double* r = h->h_red;
        inf.J_in = r[RED_JIN];
        inf.J_out = r[RED_JOUT];
        inf.R = r[RED_R];
        inf.resid = r[RED_ABSC] > 0 ? r[RED_DC] / r[RED_ABSC] : 0.0;
        if (r[RED_NONFINITE] > 0 || !isfinite(inf.J_in) || !isfinite(inf.J_out) || !isfinite(inf.R)) {
            result = CL_ERR_DIVERGED;
            set_msg_txt("non-finite concentration");
            break;
        }
        // per step: sum C changes by J_in - J_out - R plus the sources (zero at steady state)
        inf.flux_balance = fabs(inf.J_in - inf.J_out - inf.R + h->src_sum) / fmax(fabs(inf.J_in), 1e-300);
        const double q = track_deff ? inf.J_out : inf.R;
        const double dq = q - q_prev;
        const double est = nchecks >= 2 ? remaining_change(dq, dq_prev) : INFINITY;
        inf.rel_change = q != 0 ? est / fabs(q) : INFINITY;
        q_prev = q;
        dq_prev = dq;
        ++nchecks;
        // both tests must pass at two checks in a row (one quiet check at a turning point is not enough)
        quiet = (inf.flux_balance < h->p.tol_flux && inf.rel_change < h->p.tol_rel) ? quiet + 1 : 0;
        if (quiet >= 2) {
            result = CL_OK;
            inf.converged = 1;
            break;
        }
    }
    if (h->march) {
        cl_status es = check_err_flag(h);
        if (es != CL_OK) result = es;
    }
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return result;
}

namespace {

// Scratch of one call, freed when the call returns.
struct Scratch {
    cl_lbm* h;
    std::vector<std::pair<void*, size_t>> bufs;
    explicit Scratch(cl_lbm* hh) : h(hh) {}
    cl_status get(void** out, size_t bytes) {
        void* ptr = nullptr;
        if (h->p.alloc) {
            ptr = h->p.alloc(bytes, (void*)h->s, h->p.alloc_ctx);
            if (!ptr) { set_msg_txt("allocator callback returned NULL"); return CL_ERR_OOM; }
        } else {
            cudaError_t e = cudaMallocAsync(&ptr, bytes, h->s);
            if (e != cudaSuccess) { set_msg("cudaMallocAsync", e); return from_cuda(e); }
        }
        bufs.emplace_back(ptr, bytes);
        *out = ptr;
        return CL_OK;
    }
    ~Scratch() {
        cudaStreamSynchronize(h->s);
        for (auto& b : bufs) {
            if (h->p.free) h->p.free(b.first, b.second, (void*)h->s, h->p.alloc_ctx);
            else cudaFreeAsync(b.first, h->s);
        }
    }
};

// One step of the lattice's plain-population kernel from src to dst; with
// `linear` the boundary concentrations are taken as zero, which leaves the
// linear part A of the affine step map S(x) = A x + b.
cudaError_t step_pop(cl_lbm* h, const float* src, float* dst, bool linear) {
    if (h->q == 19) {
        Q19Args a = make_args19(h);
        if (linear) { a.c_in = a.c_out = 0.f; a.c_in_d = a.c_out_d = 0.0; }
        return launch_step19(src, dst, a, false, h->s);
    }
    StepArgs a = make_args(h);
    if (linear) { a.abb_in = a.abb_out = 0.f; a.w_cin = a.w_cout = 0.f; a.src = nullptr; }
    return launch_step_fp32(src, dst, a, false, h->s);
}

// The affine step S in FP64 on FP64 populations.
cudaError_t step_f64(cl_lbm* h, const double* src, double* dst) {
    if (h->q == 19) return launch_step19_f64(src, dst, make_args19(h), h->s);
    return launch_step_f64(src, dst, make_args(h), h->s);
}

// Each f32 BiCGSTAB solve of the refinement reduces the residual to this
// fraction (the f32 vectors reach a few 1e-6 at best).
constexpr double kKryInnerTol = 1e-3;

}  // namespace

cl_status cl_lbm_solve_krylov(cl_handle h, double tol, int max_iter, long long max_steps, cl_solve_info* info,
                              int* iterations) {
    CKS(need_structure(h));
    if (h->march || h->q19s) {
        set_msg_txt("the Krylov solve needs the plain f32 population storage (CL_STORAGE_FP32POP)");
        return CL_ERR_STATE;
    }
    if (!(tol > 0.0) || max_iter < 0 || max_steps < 0) {
        set_msg_txt("tol must be > 0, max_iter and max_steps >= 0");
        return CL_ERR_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    const long long L = h->q == 19 ? 19 * h->NP19 : 7 * h->N;
    const int nblk = kry_blocks();
    int iters = 0;
    {
        Scratch sc(h);
        // f32: r, rh, p, v, s, t of BiCGSTAB, the correction e and its right-hand side c
        float* vec[8];
        for (int k = 0; k < 8; ++k) {
            CKS(sc.get((void**)&vec[k], sizeof(float) * (size_t)L));
            CK(cudaMemsetAsync(vec[k], 0, sizeof(float) * (size_t)L, h->s));
        }
        float *r = vec[0], *rh = vec[1], *pv = vec[2], *v = vec[3], *sv = vec[4], *t = vec[5], *e = vec[6],
              *c = vec[7];
        double *x64 = nullptr, *y64 = nullptr, *part = nullptr;
        KryScalars* ks = nullptr;
        CKS(sc.get((void**)&x64, sizeof(double) * (size_t)L));
        CKS(sc.get((void**)&y64, sizeof(double) * (size_t)L));
        CK(cudaMemsetAsync(y64, 0, sizeof(double) * (size_t)L, h->s));
        CKS(sc.get((void**)&part, sizeof(double) * 2 * (size_t)nblk));
        CKS(sc.get((void**)&ks, sizeof(KryScalars)));
        CK(cudaMemsetAsync(ks, 0, sizeof(KryScalars), h->s));
        float* x = h->pop[h->cur];
        float* u = h->pop[h->cur ^ 1];  // A(.) output; the next step of the march rewrites it
        // the f32 vector kernels move float4s
        uintptr_t bits = (uintptr_t)x | (uintptr_t)u;
        for (int k = 0; k < 8; ++k) bits |= (uintptr_t)vec[k];
        if (bits & 15u) {
            set_msg_txt("population buffers must be 16-byte aligned for the Krylov solve");
            return CL_ERR_STATE;
        }
        KryScalars hs;
        auto read = [&]() -> cl_status {
            CK(cudaMemcpyAsync(&hs, ks, sizeof(hs), cudaMemcpyDeviceToHost, h->s));
            CK(cudaStreamSynchronize(h->s));
            return CL_OK;
        };
        // BiCGSTAB in f32 on (I - A) e = c from e = 0, to tol_in times |c|.  Every pass starts from the
        // true residual c - (I - A) e = c + A e - e; a pass ends on convergence of the recurrence, a breakdown,
        // or growth of the recurrence residual (divergence), and the next pass (at most kMaxPasses) checks
        // the true residual again.  A correction whose true residual is not below |c| is dropped (e = 0).
        auto correct = [&](double tol_in) -> cl_status {
            const double tol2 = tol_in * tol_in;
            const int kBatch = 8;       // iterations between host reads of the scalars
            const int kMaxPasses = 5;
            double rr0 = -1.0;
            CK(cudaMemsetAsync(e, 0, sizeof(float) * (size_t)L, h->s));
            for (int pass = 0;; ++pass) {
                if (pass == 0) CK(launch_kry_start(e, c, nullptr, r, rh, pv, L, nblk, part, ks, h->s));
                else {
                    CK(step_pop(h, e, u, true));
                    CK(launch_kry_start(e, u, c, r, rh, pv, L, nblk, part, ks, h->s));
                }
                CKS(read());
                if (rr0 < 0.0) rr0 = hs.rr;
                if (hs.bad == 1 || (pass > 0 && !(hs.rr < rr0))) {
                    // no better than e = 0
                    CK(cudaMemsetAsync(e, 0, sizeof(float) * (size_t)L, h->s));
                    break;
                }
                if (hs.rr <= tol2 * rr0 || pass + 1 >= kMaxPasses || iters >= max_iter) break;
                double best = hs.rr;
                while (iters < max_iter) {
                    const int n = std::min(kBatch, max_iter - iters);
                    for (int k = 0; k < n; ++k) {
                        CK(step_pop(h, pv, u, true));
                        CK(launch_kry_v(pv, u, rh, v, L, nblk, part, ks, h->s));
                        CK(launch_kry_s(r, v, sv, L, nblk, ks, h->s));
                        CK(step_pop(h, sv, u, true));
                        CK(launch_kry_t(sv, u, t, L, nblk, part, ks, h->s));
                        CK(launch_kry_xr(e, pv, sv, t, rh, r, L, nblk, part, ks, h->s));
                        CK(launch_kry_p(r, v, pv, L, nblk, ks, h->s));
                    }
                    CKS(read());
                    iters = hs.iters;
                    if (hs.bad || !isfinite(hs.rr) || hs.rr <= tol2 * rr0 || hs.rr > 1e4 * best) break;
                    best = std::min(best, hs.rr);
                }
            }
            return CL_OK;
        };
        // Mixed-precision refinement: the iterate x64 and its residual S(x64) - x64 in FP64 (the FP64 step),
        // the correction in f32, so the result is not held to the rounding floor of f32 populations.  A
        // correction that does not reduce the FP64 residual is taken back, and the refinement stops.
        CK(launch_kry_to64(x, x64, L, nblk, h->s));
        const double tol2 = tol * tol;
        const int kMaxRefine = 30;
        double rr0 = -1.0, rr_prev = INFINITY;
        for (int ref = 0; ref < kMaxRefine; ++ref) {
            CK(step_f64(h, x64, y64));
            CK(launch_kry_res64(x64, y64, c, L, nblk, part, ks, h->s));
            CKS(read());
            if (!(hs.rr < rr_prev)) {
                if (ref > 0) CK(launch_kry_add64(x64, e, -1.0, L, nblk, h->s));
                break;
            }
            if (rr0 < 0.0) rr0 = hs.rr;
            // converged, out of iterations, or gaining too little to go on
            if (hs.rr <= tol2 * rr0 || iters >= max_iter || !(hs.rr < 0.25 * rr_prev)) break;
            rr_prev = hs.rr;
            CKS(correct(kKryInnerTol));
            CK(launch_kry_add64(x64, e, 1.0, L, nblk, h->s));
        }
        CK(launch_kry_to32(x64, x, L, nblk, h->s));
    }
    if (iterations) *iterations = iters;
    // certify with the stopping rule of the time march from the Krylov state
    cl_solve_info inf;
    memset(&inf, 0, sizeof(inf));
    cl_status st = cl_lbm_solve_budget(h, max_steps, &inf);
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return st;
}

cl_status cl_lbm_solve_krylov_dsa(cl_handle h, double tol, int max_iter, long long max_steps, cl_solve_info* info,
                                  int* iterations, long long* inner_iterations) {
    CKS(need_structure(h));
    if (h->march || h->q19s) {
        set_msg_txt("the preconditioned Krylov solve needs the plain f32 population storage");
        return CL_ERR_STATE;
    }
    if (!(tol > 0.0) || max_iter < 0 || max_steps < 0) {
        set_msg_txt("tol must be > 0, max_iter and max_steps >= 0");
        return CL_ERR_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    const bool q19 = h->q == 19;  // D3Q19: the padded population layout (pitch px19)
    const long long N = q19 ? h->NP19 : h->N, L = (q19 ? 19 : 7) * N;
    const int nblk = kry_blocks();
    constexpr int kM = 30;           // Krylov vectors per GMRES cycle
    constexpr int kMaxCycles = 10;   // cycles per correction
    constexpr int kCgBatch = 8;      // CG iterations between host reads
    constexpr int kMaxCg = 4000;     // CG iterations per preconditioner application
    const double kCgTol = 1e-2;      // relative residual of the inner CG solve
    int iters = 0;
    long long cg_total = 0;
    {
        Scratch sc(h);
        float* V[kM + 1];
        float* Z[kM];
        for (int k = 0; k <= kM; ++k) CKS(sc.get((void**)&V[k], sizeof(float) * (size_t)L));
        for (int k = 0; k < kM; ++k) CKS(sc.get((void**)&Z[k], sizeof(float) * (size_t)L));
        float *wv = nullptr, *e = nullptr, *c = nullptr;
        CKS(sc.get((void**)&wv, sizeof(float) * (size_t)L));
        CKS(sc.get((void**)&e, sizeof(float) * (size_t)L));
        CKS(sc.get((void**)&c, sizeof(float) * (size_t)L));
        float* cell[6];  // eps, r, z, p, q of the inner CG, and 1/diag(L)
        for (int k = 0; k < 6; ++k) {
            CKS(sc.get((void**)&cell[k], sizeof(float) * (size_t)N));
            CK(cudaMemsetAsync(cell[k], 0, sizeof(float) * (size_t)N, h->s));
        }
        float *eps = cell[0], *rc = cell[1], *zc = cell[2], *pc = cell[3], *qc = cell[4], *dinv = cell[5];
        double *x64 = nullptr, *y64 = nullptr, *part = nullptr, *dH = nullptr, *dnrm = nullptr, *dy = nullptr;
        KryScalars* ks = nullptr;
        CgScalars* cs = nullptr;
        CKS(sc.get((void**)&x64, sizeof(double) * (size_t)L));
        CKS(sc.get((void**)&y64, sizeof(double) * (size_t)L));
        CK(cudaMemsetAsync(y64, 0, sizeof(double) * (size_t)L, h->s));
        CKS(sc.get((void**)&part, sizeof(double) * 2 * (size_t)nblk));
        CKS(sc.get((void**)&dH, sizeof(double) * (kM + 1) * kM));
        CKS(sc.get((void**)&dnrm, sizeof(double)));
        CKS(sc.get((void**)&dy, sizeof(double) * kM));
        CKS(sc.get((void**)&ks, sizeof(KryScalars)));
        CKS(sc.get((void**)&cs, sizeof(CgScalars)));
        CK(cudaMemsetAsync(ks, 0, sizeof(KryScalars), h->s));
        CK(cudaMemsetAsync(cs, 0, sizeof(CgScalars), h->s));
        float* x = h->pop[h->cur];
        float* u = h->pop[h->cur ^ 1];  // A(.) output; the next step of the march rewrites it
        DsaArgs da;
        da.nx = h->nx; da.ny = h->ny; da.nz = h->nz; da.N = N;
        da.mask = h->mask;
        da.rfac = reactive_factor(h);
        da.rsink = (float)reactive_sink_d(h);
        da.bc_in = h->p.bc_in; da.bc_out = h->p.bc_out;
        da.kscale = h->kscale;
        da.k_lu = h->k_lu;
        Dsa19 d19;
        d19.px = h->px19;
        d19.mask = h->mask19;
        d19.react = h->react19;
        CK(q19 ? launch_lap_dinv19(da, d19, dinv, nblk, h->s) : launch_lap_dinv(da, dinv, nblk, h->s));
        auto host_double = [&](const double* dptr, double* out, int n) -> cl_status {
            CK(cudaMemcpyAsync(out, dptr, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
            CK(cudaStreamSynchronize(h->s));
            return CL_OK;
        };
        // kCgBatch CG iterations on the fixed cell buffers, captured once and
        // replayed as one CUDA graph (five launches per iteration otherwise
        // cost more than the iteration's own memory traffic on small boxes)
        auto enqueue_cg = [&](cudaStream_t st) -> cudaError_t {
            for (int k = 0; k < kCgBatch; ++k) {
                const cudaError_t ce = q19 ? launch_cg_iter19(da, d19, dinv, eps, rc, zc, pc, qc, nblk, part, cs, st)
                                           : launch_cg_iter(da, dinv, eps, rc, zc, pc, qc, nblk, part, cs, st);
                if (ce != cudaSuccess) return ce;
            }
            return cudaSuccess;
        };
        cudaGraphExec_t cg_graph = nullptr;
        struct GraphGuard {
            cudaGraphExec_t* g;
            ~GraphGuard() { if (*g) cudaGraphExecDestroy(*g); }
        } guard{&cg_graph};
        {
            cudaStream_t cap = nullptr;
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
            if (ok) ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const cudaError_t ce = enqueue_cg(cap);
                ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && g && ce == cudaSuccess;
            }
            if (ok) ok = cudaGraphInstantiate(&cg_graph, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            if (cap) cudaStreamDestroy(cap);
            if (!ok) {
                cg_graph = nullptr;
                cudaGetLastError();  // the same kernels then run as plain launches
            }
        }
        // P v = v + w_i eps, L eps = sum_i v_i to kCgTol by diagonal-preconditioned CG
        auto precondition = [&](const float* v, float* zout) -> cl_status {
            CK(q19 ? launch_cg_start19(da, d19, v, dinv, eps, rc, zc, pc, nblk, part, cs, h->s)
                   : launch_cg_start(da, v, dinv, eps, rc, zc, pc, nblk, part, cs, h->s));
            CgScalars hc;
            CK(cudaMemcpyAsync(&hc, cs, sizeof(hc), cudaMemcpyDeviceToHost, h->s));
            CK(cudaStreamSynchronize(h->s));
            while (!hc.bad && hc.iters < kMaxCg && hc.rr > kCgTol * kCgTol * hc.rr0) {
                if (cg_graph) CK(cudaGraphLaunch(cg_graph, h->s));
                else CK(enqueue_cg(h->s));
                CK(cudaMemcpyAsync(&hc, cs, sizeof(hc), cudaMemcpyDeviceToHost, h->s));
                CK(cudaStreamSynchronize(h->s));
            }
            cg_total += hc.iters;
            CK(q19 ? launch_prec_out19(N, v, eps, zout, nblk, h->s) : launch_prec_out(N, v, eps, zout, nblk, h->s));
            return CL_OK;
        };
        // flexible GMRES(kM) in f32 on (I - A) e = c from e = 0, to tol_in times |c|
        auto correct = [&](double tol_in) -> cl_status {
            CK(cudaMemsetAsync(e, 0, sizeof(float) * (size_t)L, h->s));
            double beta0 = 0.0;
            CK(launch_dot_dev(c, c, L, nblk, part, dnrm, 1, h->s));
            CKS(host_double(dnrm, &beta0, 1));
            if (!(beta0 > 0.0) || !isfinite(beta0)) return CL_OK;
            double H[kM + 1][kM], cs_[kM], sn_[kM], g[kM + 1], col[kM + 1], y[kM];
            for (int cyc = 0; cyc < kMaxCycles && iters < max_iter; ++cyc) {
                double beta = 0.0;
                if (cyc == 0) {
                    CK(launch_scale_dev(V[0], c, dnrm, L, nblk, h->s));
                    beta = beta0;
                } else {
                    CK(step_pop(h, e, u, true));
                    CK(launch_comb(c, e, u, wv, L, nblk, h->s));  // c - (I - A) e
                    CK(launch_dot_dev(wv, wv, L, nblk, part, dnrm, 1, h->s));
                    CKS(host_double(dnrm, &beta, 1));
                    if (!isfinite(beta)) break;
                    if (beta <= tol_in * beta0) break;
                    CK(launch_scale_dev(V[0], wv, dnrm, L, nblk, h->s));
                }
                for (int k = 0; k <= kM; ++k) g[k] = 0.0;
                g[0] = beta;
                int jend = 0;
                double resid = beta;
                for (int j = 0; j < kM && iters < max_iter; ++j) {
                    CKS(precondition(V[j], Z[j]));
                    CK(step_pop(h, Z[j], u, true));
                    CK(launch_comb(Z[j], u, nullptr, wv, L, nblk, h->s));  // (I - A) Z_j
                    ++iters;
                    // modified Gram-Schmidt, coefficients kept on the device
                    for (int k = 0; k <= j; ++k) {
                        double* hk = dH + k + (kM + 1) * j;
                        CK(launch_dot_dev(V[k], wv, L, nblk, part, hk, 0, h->s));
                        CK(launch_axpy_dev(wv, V[k], hk, -1.f, L, nblk, h->s));
                    }
                    double* hn = dH + (j + 1) + (kM + 1) * j;
                    CK(launch_dot_dev(wv, wv, L, nblk, part, hn, 1, h->s));
                    CK(launch_scale_dev(V[j + 1], wv, hn, L, nblk, h->s));
                    CKS(host_double(dH + (kM + 1) * j, col, j + 2));
                    // Givens rotations: the earlier ones, then a new one that zeroes col[j + 1]
                    for (int k = 0; k < j; ++k) {
                        const double a = cs_[k] * col[k] + sn_[k] * col[k + 1];
                        col[k + 1] = -sn_[k] * col[k] + cs_[k] * col[k + 1];
                        col[k] = a;
                    }
                    const double den = sqrt(col[j] * col[j] + col[j + 1] * col[j + 1]);
                    jend = j + 1;
                    if (!(den > 0.0) || !isfinite(den)) { jend = j; break; }
                    cs_[j] = col[j] / den;
                    sn_[j] = col[j + 1] / den;
                    col[j] = den;
                    col[j + 1] = 0.0;
                    g[j + 1] = -sn_[j] * g[j];
                    g[j] = cs_[j] * g[j];
                    for (int k = 0; k <= j; ++k) H[k][j] = col[k];
                    resid = fabs(g[j + 1]);
                    if (resid <= tol_in * beta0) break;
                }
                if (jend == 0) break;
                // back substitution R y = g, then e += sum_k y_k Z_k
                for (int k = jend - 1; k >= 0; --k) {
                    double t = g[k];
                    for (int l = k + 1; l < jend; ++l) t -= H[k][l] * y[l];
                    y[k] = t / H[k][k];
                }
                CK(cudaMemcpyAsync(dy, y, sizeof(double) * jend, cudaMemcpyHostToDevice, h->s));
                for (int k = 0; k < jend; ++k) CK(launch_axpy_dev(e, Z[k], dy + k, 1.f, L, nblk, h->s));
                CK(cudaStreamSynchronize(h->s));  // y lives on the host stack
                if (resid <= tol_in * beta0) break;
            }
            return CL_OK;
        };
        // mixed-precision refinement, as in cl_lbm_solve_krylov
        CK(launch_kry_to64(x, x64, L, nblk, h->s));
        const double tol2 = tol * tol;
        const int kMaxRefine = 30;
        double rr0 = -1.0, rr_prev = INFINITY;
        KryScalars hs;
        for (int ref = 0; ref < kMaxRefine; ++ref) {
            CK(step_f64(h, x64, y64));
            CK(launch_kry_res64(x64, y64, c, L, nblk, part, ks, h->s));
            CK(cudaMemcpyAsync(&hs, ks, sizeof(hs), cudaMemcpyDeviceToHost, h->s));
            CK(cudaStreamSynchronize(h->s));
            if (!(hs.rr < rr_prev)) {
                if (ref > 0) CK(launch_kry_add64(x64, e, -1.0, L, nblk, h->s));
                break;
            }
            if (rr0 < 0.0) rr0 = hs.rr;
            if (hs.rr <= tol2 * rr0 || iters >= max_iter || !(hs.rr < 0.25 * rr_prev)) break;
            rr_prev = hs.rr;
            CKS(correct(kKryInnerTol));
            CK(launch_kry_add64(x64, e, 1.0, L, nblk, h->s));
        }
        CK(launch_kry_to32(x64, x, L, nblk, h->s));
    }
    if (iterations) *iterations = iters;
    if (inner_iterations) *inner_iterations = cg_total;
    cl_solve_info inf;
    memset(&inf, 0, sizeof(inf));
    cl_status st = cl_lbm_solve_budget(h, max_steps, &inf);
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return st;
}

cl_status cl_lbm_fluxes(cl_handle h, double out[5]) {
    CKS(need_structure(h));
    if (!out) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    double t[5];
    CKS(plane_readout(h, t));
    out[0] = t[3];
    out[1] = t[4];
    out[2] = t[2];
    out[3] = t[0];
    out[4] = t[1];
    return CL_OK;
}

cl_status cl_lbm_effective_diffusivity(cl_handle h, double* d_eff_m2s, double* d_eff_over_db) {
    CKS(need_structure(h));
    if (h->p.bc_in != CL_BC_DIRICHLET || h->p.bc_out != CL_BC_DIRICHLET || h->p.c_in == h->p.c_out) {
        set_msg_txt("D_eff needs fixed, different concentrations at both x faces");
        return CL_ERR_STATE;
    }
    double t[5];
    CKS(plane_readout(h, t));
    // Eq. 19: mean outlet flux density over (C_in - C_out) / L_x, lattice units
    const double jd = t[4] / ((double)h->ny * h->nz);
    const double dlu = jd * h->nx / (h->p.c_in - h->p.c_out);
    const double d = dlu * h->p.dx_m * h->p.dx_m / h->dt;
    if (d_eff_m2s) *d_eff_m2s = d;
    // protons: the effective conductivity over the ionomer's own (Sec. 5.2)
    if (d_eff_over_db) *d_eff_over_db = d / (h->p.carrier == CL_CARRIER_PROTON ? h->p.D_ionomer : h->D_b);
    return CL_OK;
}

cl_status cl_lbm_reaction_rate(cl_handle h, double* total, double* profile_R, double* profile_C) {
    CKS(need_structure(h));
    double t[5];
    CKS(plane_readout(h, t));
    const double scale = h->p.dx_m * h->p.dx_m * h->p.dx_m / h->dt;
    const double* hp = h->h_red + 16;
    if (total) *total = t[2] * scale;
    for (int x = 0; x < h->nx; ++x) {
        if (profile_R) profile_R[x] = hp[5 * x + 2] * scale;
        if (profile_C) profile_C[x] = hp[5 * x + 1] > 0 ? hp[5 * x] / hp[5 * x + 1] : 0.0;
    }
    return CL_OK;
}

cl_status cl_lbm_current_density(cl_handle h, double* i_d) {
    CKS(need_structure(h));
    if (!i_d) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    if (h->p.carrier == CL_CARRIER_PROTON) { set_msg_txt("the proton carrier has no reaction"); return CL_ERR_STATE; }
    double R = 0.0;
    CKS(cl_lbm_reaction_rate(h, &R, nullptr, nullptr));
    const double F = 96485.33212;  // C/mol
    *i_d = 4.0 * F * R / ((double)h->ny * h->nz * h->p.dx_m * h->p.dx_m);  // Eq. 25, A_cross = ny nz dx^2
    return CL_OK;
}

static cl_status state_out(cl_lbm* h, float* C, float* g, int ptr_is_device) {
    const size_t N = (size_t)h->N;
    if (h->march) {
        MarchArgs a = make_margs(h, h->cur);
        if (ptr_is_device) {
            CK(launch_state_out(h->p.storage, a, h->mask_p, C, g, h->s));
        } else if (C) {
            CK(launch_state_out(h->p.storage, a, h->mask_p, h->fbuf, nullptr, h->s));
            CK(cudaMemcpyAsync(C, h->fbuf, sizeof(float) * N, cudaMemcpyDeviceToHost, h->s));
        } else {
            void* tmp = nullptr;
            CK(cudaMallocAsync(&tmp, sizeof(float) * 7 * N, h->s));
            cudaError_t e = launch_state_out(h->p.storage, a, h->mask_p, nullptr, (float*)tmp, h->s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(g, tmp, sizeof(float) * 7 * N, cudaMemcpyDeviceToHost, h->s);
            cudaFreeAsync(tmp, h->s);
            if (e != cudaSuccess) { set_msg("populations", e); return from_cuda(e); }
        }
    } else if (h->q19s) {
        Q19Args a = make_args19(h);
        if (C) {
            float* dstp = ptr_is_device ? C : h->fbuf;
            CK(launch_out19s(h->p.storage, h->st19[h->cur], a, dstp, nullptr, h->s));
            if (!ptr_is_device) CK(cudaMemcpyAsync(C, h->fbuf, sizeof(float) * N, cudaMemcpyDeviceToHost, h->s));
        }
        if (g) {
            float* gd = g;
            void* tmp = nullptr;
            if (!ptr_is_device) {
                CK(cudaMallocAsync(&tmp, sizeof(float) * 19 * N, h->s));
                gd = (float*)tmp;
            }
            cudaError_t e = launch_out19s(h->p.storage, h->st19[h->cur], a, nullptr, gd, h->s);
            if (e == cudaSuccess && !ptr_is_device)
                e = cudaMemcpyAsync(g, gd, sizeof(float) * 19 * N, cudaMemcpyDeviceToHost, h->s);
            if (tmp) cudaFreeAsync(tmp, h->s);
            if (e != cudaSuccess) { set_msg("populations", e); return from_cuda(e); }
        }
    } else if (h->q == 19) {
        if (C) {
            float* dstp = ptr_is_device ? C : h->fbuf;
            CK(launch_out19(h->pop[h->cur], h->mask19, h->nx, h->ny, h->nz, h->px19, dstp, nullptr, h->s));
            if (!ptr_is_device) CK(cudaMemcpyAsync(C, h->fbuf, sizeof(float) * N, cudaMemcpyDeviceToHost, h->s));
        }
        if (g) {
            float* gd = g;
            void* tmp = nullptr;
            if (!ptr_is_device) {
                CK(cudaMallocAsync(&tmp, sizeof(float) * 19 * N, h->s));
                gd = (float*)tmp;
            }
            cudaError_t e = launch_out19(h->pop[h->cur], h->mask19, h->nx, h->ny, h->nz, h->px19, nullptr, gd, h->s);
            if (e == cudaSuccess && !ptr_is_device)
                e = cudaMemcpyAsync(g, gd, sizeof(float) * 19 * N, cudaMemcpyDeviceToHost, h->s);
            if (tmp) cudaFreeAsync(tmp, h->s);
            if (e != cudaSuccess) { set_msg("populations", e); return from_cuda(e); }
        }
    } else {
        if (C) {
            float* dstp = ptr_is_device ? C : h->fbuf;
            CK(launch_field_fp32(h->pop[h->cur], h->mask, h->N, dstp, h->src, h->s));
            if (!ptr_is_device) CK(cudaMemcpyAsync(C, h->fbuf, sizeof(float) * N, cudaMemcpyDeviceToHost, h->s));
        }
        if (g) CK(cudaMemcpyAsync(g, h->pop[h->cur], sizeof(float) * 7 * N, kind_out(ptr_is_device), h->s));
    }
    CK(cudaStreamSynchronize(h->s));
    return CL_OK;
}

namespace {
// the per-cell arrays below act on the plain f32 population kernel of D3Q7
cl_status need_pop7(cl_lbm* h, const char* what) {
    CKS(need_structure(h));
    if (h->march || h->q != 7) {
        set_msg_txt(what);
        return CL_ERR_STATE;
    }
    return CL_OK;
}

__global__ void k_active_sum(const double* __restrict__ v, const uint16_t* __restrict__ mask, long long N,
                             double* partials) {
    double acc[1] = {0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        if (mask[c] & kActiveBit) acc[0] += v[c];
    block_sum_store<1>(acc, partials + blockIdx.x);
}
}  // namespace

cl_status cl_lbm_set_rate_scale(cl_handle h, const double* kscale, int ptr_is_device) {
    CKS(need_pop7(h, "per-cell rate constants need D3Q7 plain f32 populations (CL_STORE_FP32POP)"));
    drop_graphs(h);  // the arrays are baked into captured kernel arguments
    if (!kscale) { h->kscale = nullptr; return CL_OK; }
    if (!h->kscale_buf) CKS(dalloc_n(h, &h->kscale_buf, h->N));
    CK(cudaMemcpyAsync(h->kscale_buf, kscale, sizeof(double) * (size_t)h->N, kind_in(ptr_is_device), h->s));
    CK(cudaStreamSynchronize(h->s));
    h->kscale = h->kscale_buf;
    return CL_OK;
}

cl_status cl_lbm_set_source(cl_handle h, const double* S, int ptr_is_device) {
    CKS(need_pop7(h, "per-cell sources need D3Q7 plain f32 populations (CL_STORE_FP32POP)"));
    drop_graphs(h);
    if (!S) { h->src = nullptr; h->src_sum = 0.0; return CL_OK; }
    if (!h->src_buf) CKS(dalloc_n(h, &h->src_buf, h->N));
    CK(cudaMemcpyAsync(h->src_buf, S, sizeof(double) * (size_t)h->N, kind_in(ptr_is_device), h->s));
    // the sum over active cells enters the flux balance of the stopping rule
    const int nb = 152 * 4;
    CK(cudaMemsetAsync(h->d_red, 0, sizeof(double), h->s));
    k_active_sum<<<nb, 256, 0, h->s>>>(h->src_buf, h->mask, h->N, h->partials);
    CK(cudaGetLastError());
    CK(launch_finalize(h->partials, nb, 1, h->d_red, h->s));
    CK(cudaMemcpyAsync(&h->src_sum, h->d_red, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    h->src = h->src_buf;
    return CL_OK;
}

cl_status cl_lbm_cell_reaction(cl_handle h, double* out, int ptr_is_device) {
    CKS(need_pop7(h, "the per-cell reaction readout needs D3Q7 plain f32 populations (CL_STORE_FP32POP)"));
    if (!out) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    double* d = out;
    void* tmp = nullptr;
    if (!ptr_is_device) {
        CK(cudaMallocAsync(&tmp, sizeof(double) * (size_t)h->N, h->s));
        d = (double*)tmp;
    }
    cudaError_t e = launch_cell_reaction_fp32(h->pop[h->cur], make_args(h), d, h->s);
    if (e == cudaSuccess && !ptr_is_device)
        e = cudaMemcpyAsync(out, d, sizeof(double) * (size_t)h->N, cudaMemcpyDeviceToHost, h->s);
    if (tmp) cudaFreeAsync(tmp, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    CK(e);
    return CL_OK;
}

cl_status cl_lbm_get_field(cl_handle h, float* C, int ptr_is_device) {
    CKS(need_structure(h));
    if (!C) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    return state_out(h, C, nullptr, ptr_is_device);
}

cl_status cl_lbm_get_populations(cl_handle h, float* g, int ptr_is_device) {
    CKS(need_structure(h));
    if (!g) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    return state_out(h, nullptr, g, ptr_is_device);
}

cl_status cl_lbm_get_setup(cl_handle h, uint8_t* active, float* omega, int32_t* chord, uint16_t* link_mask,
                           int ptr_is_device) {
    CKS(need_structure(h));
    const size_t N = (size_t)h->N;
    if (active) CK(cudaMemcpyAsync(active, h->active, N, kind_out(ptr_is_device), h->s));
    if (omega) CK(cudaMemcpyAsync(omega, h->omega, N * sizeof(float), kind_out(ptr_is_device), h->s));
    if (link_mask) CK(cudaMemcpyAsync(link_mask, h->mask, N * sizeof(uint16_t), kind_out(ptr_is_device), h->s));
    if (chord) {
        int32_t* dchord = chord;
        void* tmp = nullptr;
        if (!ptr_is_device) {
            CK(cudaMallocAsync(&tmp, N * 13 * sizeof(int32_t), h->s));
            dchord = (int32_t*)tmp;
        }
        cudaError_t e = launch_chords13(h->phase, h->nx, h->ny, h->nz, dchord, h->s);
        if (e == cudaSuccess && !ptr_is_device)
            e = cudaMemcpyAsync(chord, dchord, N * 13 * sizeof(int32_t), cudaMemcpyDeviceToHost, h->s);
        if (tmp) cudaFreeAsync(tmp, h->s);
        if (e != cudaSuccess) { set_msg("chords", e); return from_cuda(e); }
    }
    CK(cudaStreamSynchronize(h->s));
    return CL_OK;
}

cl_status cl_lbm_get_links(cl_handle h, uint32_t* wall, uint32_t* reactive, int ptr_is_device) {
    CKS(need_structure(h));
    if (!wall && !reactive) return CL_OK;
    const size_t N = (size_t)h->N;
    uint32_t* dw = wall;
    uint32_t* dr = reactive;
    void* tmp = nullptr;
    if (!ptr_is_device) {
        CK(cudaMallocAsync(&tmp, 2 * N * sizeof(uint32_t), h->s));
        dw = wall ? (uint32_t*)tmp : nullptr;
        dr = reactive ? (uint32_t*)tmp + N : nullptr;
    }
    cudaError_t e = h->q == 19
                        ? launch_links_out(h->mask19, h->react19, nullptr, h->nx, h->ny, h->nz, h->px19, dw, dr, h->s)
                        : launch_links_out(nullptr, nullptr, h->mask, h->nx, h->ny, h->nz, 0, dw, dr, h->s);
    if (e == cudaSuccess && !ptr_is_device && wall)
        e = cudaMemcpyAsync(wall, dw, N * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->s);
    if (e == cudaSuccess && !ptr_is_device && reactive)
        e = cudaMemcpyAsync(reactive, dr, N * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->s);
    if (tmp) cudaFreeAsync(tmp, h->s);
    if (e != cudaSuccess) { set_msg("links", e); return from_cuda(e); }
    CK(cudaStreamSynchronize(h->s));
    return CL_OK;
}

cl_status cl_lbm_get_info(cl_handle h, cl_structure_info* info) {
    CKS(need_structure(h));
    if (!info) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    *info = h->info;
    return CL_OK;
}

cl_status cl_lbm_get_step(cl_handle h, long long* step) {
    CKS(need_structure(h));
    if (!step) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    *step = h->step;
    return CL_OK;
}

}  // extern "C"
