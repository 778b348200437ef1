// Connected-phase labelling of Sec. 2.1.3 and its statistics on the GPU.
//
// The paper scans the box with a 13-neighbour label pass (the already
// scanned half of the 26-neighbourhood of Fig. 4a) and repeats scans in
// several directions until labels settle.  Here one pass of a lock-free
// union-find does the same work in parallel: every cell of the phase set
// unites with the set cells among its 13 (or, for 6-connectivity, 3)
// neighbours of the earlier half-space, so each neighbouring pair is united
// once, from one side; then every cell takes its root, the smallest cell
// index of its portion.  Per portion, atomics record whether it reaches the
// end planes x = 0 and x = L and how many cells it has; one more pass sums
// the statistics in FP64 per block (fixed order) and finalises them.
#include "cl_lbm.h"
#include "device_util.cuh"
#include "handle.cuh"
#include "internal.cuh"
#include "uf.cuh"

namespace cl {

namespace {

__device__ __forceinline__ bool in_set(uint8_t p, unsigned set) { return p < 4 && ((set >> p) & 1u); }

// the neighbour (x + dx, y + dy, z + dz), or -1 outside the box (x never wraps)
__device__ __forceinline__ long long cc_neighbor(int x, int y, int z, int dx, int dy, int dz, int nx, int ny, int nz,
                                                 int periodic) {
    const int qx = x + dx;
    if (qx < 0 || qx >= nx) return -1;
    int qy = y + dy, qz = z + dz;
    if (periodic) {
        qy = qy < 0 ? qy + ny : (qy >= ny ? qy - ny : qy);
        qz = qz < 0 ? qz + nz : (qz >= nz ? qz - nz : qz);
    } else if (qy < 0 || qy >= ny || qz < 0 || qz >= nz) {
        return -1;
    }
    return qx + (long long)nx * (qy + (long long)ny * qz);
}

__global__ void k_cc_init(const uint8_t* __restrict__ phase, long long N, unsigned set, int* L, unsigned* ends,
                          int* size, int* err) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint8_t p = phase[c];
        if (p > 3) atomicOr(err, 1);
        L[c] = in_set(p, set) ? (int)c : -1;
        ends[c] = 0;
        size[c] = 0;
    }
}

__global__ void k_cc_merge(const uint8_t* __restrict__ phase, int nx, int ny, int nz, unsigned set, int faces_only,
                           int periodic, int* L, int* err) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        if (!in_set(phase[c], set)) continue;
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        // the earlier half of the neighbourhood: dz < 0, or dz = 0 and dy < 0, or dz = dy = 0 and dx < 0
        for (int dz = -1; dz <= 0; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dz == 0 && (dy > 0 || (dy == 0 && dx >= 0))) continue;
                    if (faces_only && (dx != 0) + (dy != 0) + (dz != 0) != 1) continue;
                    const long long n = cc_neighbor(x, y, z, dx, dy, dz, nx, ny, nz, periodic);
                    if (n >= 0 && n != c && in_set(phase[n], set)) uf_union(L, (int)c, (int)n, err);
                }
    }
}

__global__ void k_cc_flatten(long long N, int* L, int* err) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        if (L[c] >= 0) L[c] = uf_find(L, (int)c, err);
}

__global__ void k_cc_tally(int nx, long long N, const int* __restrict__ L, unsigned* ends, int* size) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int r = L[c];
        if (r < 0) continue;
        const int x = (int)(c % nx);
        const unsigned e = (x == 0 ? 1u : 0u) | (x == nx - 1 ? 2u : 0u);
        if (e) atomicOr(ends + r, e);
        atomicAdd(size + r, 1);
    }
}

// v: cells, portions, transport portions, transport cells, surface faces, transport surface faces
__global__ void k_cc_stats(const uint8_t* __restrict__ phase, int nx, int ny, int nz, unsigned set, int periodic,
                           const int* __restrict__ L, const unsigned* __restrict__ ends,
                           const int* __restrict__ size, double* partials, int* largest) {
    const long long N = (long long)nx * ny * nz;
    double v[6] = {0, 0, 0, 0, 0, 0};
    int big = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int r = L[c];
        if (r < 0) continue;
        const bool tr = ends[r] == 3u;
        v[0] += 1.0;
        if (r == (int)c) {
            v[1] += 1.0;
            if (tr) v[2] += 1.0;
            big = max(big, size[c]);
        }
        if (tr) v[3] += 1.0;
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        int f = 0;
        const int fd[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const long long n = cc_neighbor(x, y, z, fd[k][0], fd[k][1], fd[k][2], nx, ny, nz, periodic);
            if (n >= 0 && !in_set(phase[n], set)) ++f;
        }
        v[4] += f;
        if (tr) v[5] += f;
    }
    if (big > 0) atomicMax(largest, big);
    block_sum_store<6>(v, partials + 6LL * blockIdx.x);
}

}  // namespace

}  // namespace cl

using namespace cl;

extern "C" cl_status cl_phase_connectivity(const uint8_t* phase, int nx, int ny, int nz, unsigned phase_set,
                                           int neighbours, int periodic_yz, int32_t* labels, cl_phase_stats* out,
                                           int ptr_is_device, void* cuda_stream) {
    if (!phase || !out) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    const long long N = (long long)nx * ny * nz;
    if (nx < 1 || ny < 1 || nz < 1 || N >= (1LL << 31)) { set_msg_txt("box size out of range"); return CL_ERR_ARG; }
    if (neighbours != 6 && neighbours != 26) { set_msg_txt("neighbours must be 6 or 26"); return CL_ERR_ARG; }
    if (phase_set == 0 || phase_set > 15) { set_msg_txt("phase_set must name codes 0..3"); return CL_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int grid = 152 * 8, block = 256;
    // scratch: [phase copy] labels, ends, sizes (4 B each per cell), partials, results
    const size_t cells4 = (sizeof(int) * (size_t)N + 255) / 256 * 256;  // keeps every region 256-byte aligned
    const size_t scratch = 3 * cells4 + sizeof(double) * (6 * grid + 8) + 64 + (ptr_is_device ? 0 : (size_t)N);
    unsigned char* base = nullptr;
    CK(cudaMallocAsync((void**)&base, scratch, s));
    int* L = (int*)base;
    unsigned* ends = (unsigned*)(base + cells4);
    int* size = (int*)(base + 2 * cells4);
    double* partials = (double*)(base + 3 * cells4);
    double* dres = partials + 6 * grid;
    int* ints = (int*)(dres + 8);  // [0] largest, [1] error bits
    const uint8_t* ph = phase;
    if (!ptr_is_device) {
        uint8_t* pcopy = (uint8_t*)(ints + 16);
        cudaError_t e = cudaMemcpyAsync(pcopy, phase, (size_t)N, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { cudaFreeAsync(base, s); set_msg("phase upload", e); return from_cuda(e); }
        ph = pcopy;
    }
    cudaError_t e = cudaMemsetAsync(ints, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) {
        k_cc_init<<<grid, block, 0, s>>>(ph, N, phase_set, L, ends, size, ints + 1);
        k_cc_merge<<<grid, block, 0, s>>>(ph, nx, ny, nz, phase_set, neighbours == 6, periodic_yz != 0, L, ints + 1);
        k_cc_flatten<<<grid, block, 0, s>>>(N, L, ints + 1);
        k_cc_tally<<<grid, block, 0, s>>>(nx, N, L, ends, size);
        k_cc_stats<<<grid, block, 0, s>>>(ph, nx, ny, nz, phase_set, periodic_yz != 0, L, ends, size, partials,
                                          ints);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_finalize(partials, grid, 6, dres, s);
    double res[6];
    int hi[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, dres, sizeof(res), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hi, ints, sizeof(hi), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && labels)
        e = cudaMemcpyAsync(labels, L, sizeof(int) * (size_t)N,
                            ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(base, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_msg("cl_phase_connectivity", e); return from_cuda(e); }
    if (hi[1] & 1) { set_msg_txt("phase code outside 0..3"); return CL_ERR_ARG; }
    if (hi[1] & 2) { set_msg_txt("connectivity labelling exceeded its iteration bound"); return CL_ERR_TIMEOUT; }
    out->n_cells = (long long)res[0];
    out->n_portions = (long long)res[1];
    out->n_transport_portions = (long long)res[2];
    out->n_transport_cells = (long long)res[3];
    out->surface_faces = (long long)res[4];
    out->transport_surface_faces = (long long)res[5];
    out->largest_portion = hi[0];
    return CL_OK;
}
