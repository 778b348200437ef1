// Structure generation on the GPU: the quartet structure generation set
// (QSGS) growth of Sec. 2.1.2, the solid-not-touching-ionomer region of the
// micropore step (Sec. 5.3) and the reactive-face sampling of the Pt layer.
// Input generation only (none of the solver's arithmetic); the results are
// bit-identical to the host generator of the inputs module, so that either
// can feed the solver and the oracle.
//
// Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) folded over
// (seed, stream, a, b); a uniform double in [0, 1) is the top 53 bits times
// 2^-53.  Growth (Sec. 2.1.2.1): seeds placed once with probability c_d, then
// synchronous sweeps over the state at the start of the sweep.  A cell that
// may convert and has grown 6-neighbours (x, y and z wrap) is accepted with
// two or more of them (rule 2a), else with probability p_alpha (rule 2b).
// The sweep that would overshoot the target accepts only its `need`
// candidates with the smallest (priority hash, cell index), found here by a
// radix select over the 96-bit composite instead of a sort.
#include "cl_lbm.h"
#include "handle.cuh"
#include "internal.cuh"

namespace cl {

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t hash4(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    uint64_t h = splitmix64(seed);
    h = splitmix64(h ^ stream);
    h = splitmix64(h ^ a);
    return splitmix64(h ^ b);
}

__device__ __forceinline__ double u01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

constexpr uint64_t kKeyStream = 0x5bd1e995ULL;

__global__ void k_count_code(const uint8_t* __restrict__ phase, long long N, int code, unsigned long long* out) {
    unsigned long long n = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        n += phase[c] == code;
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(out, n);
}

// candidates of one sweep, compacted in any order (the selection below does
// not depend on it)
__global__ void k_candidates(const uint8_t* __restrict__ phase, const uint8_t* __restrict__ region, int nx, int ny,
                             int nz, unsigned allowed, unsigned grown, double c_d, double p_alpha, uint64_t seed,
                             uint64_t stream, int sweep, uint64_t* __restrict__ key, uint32_t* __restrict__ cell,
                             unsigned long long* nc) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint8_t pc = phase[c];
        if (pc > 3 || !((allowed >> pc) & 1u) || (region && !region[c])) continue;
        bool accept;
        if (sweep == 0) {
            accept = u01(hash4(seed, stream, 0, (uint64_t)c)) <= c_d;
        } else {
            const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
            const int xs[6] = {x + 1 == nx ? 0 : x + 1, x == 0 ? nx - 1 : x - 1, x, x, x, x};
            const int ys[6] = {y, y, y + 1 == ny ? 0 : y + 1, y == 0 ? ny - 1 : y - 1, y, y};
            const int zs[6] = {z, z, z, z, z + 1 == nz ? 0 : z + 1, z == 0 ? nz - 1 : z - 1};
            int ng = 0, parent = -1;
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                const long long q = xs[d] + (long long)nx * (ys[d] + (long long)ny * zs[d]);
                const uint8_t pq = phase[q];
                if (pq < 4 && ((grown >> pq) & 1u)) { ++ng; parent = d; }
            }
            if (ng == 0) continue;
            accept = ng >= 2 ||
                     u01(hash4(seed, stream, (uint64_t)sweep * 8 + (uint64_t)parent, (uint64_t)c)) <= p_alpha;
        }
        if (!accept) continue;
        const unsigned long long slot = atomicAdd(nc, 1ULL);
        key[slot] = hash4(seed, stream ^ kKeyStream, (uint64_t)sweep, (uint64_t)c);
        cell[slot] = (uint32_t)c;
    }
}

// digit `pass` (0..7: key bytes from the top, 8..11: cell bytes from the top)
// of the candidates whose higher digits equal the fixed prefix
__global__ void k_digit_hist(const uint64_t* __restrict__ key, const uint32_t* __restrict__ cell, long long nc,
                             int pass, uint64_t key_prefix, uint32_t cell_prefix, unsigned* hist) {
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nc;
         j += (long long)gridDim.x * blockDim.x) {
        const uint64_t k = key[j];
        const uint32_t cl = cell[j];
        unsigned digit;
        if (pass < 8) {
            const int hi_bits = 8 * pass;  // bits already fixed, from the top
            if (hi_bits && (k >> (64 - hi_bits)) != (key_prefix >> (64 - hi_bits))) continue;
            digit = (unsigned)(k >> (56 - 8 * pass)) & 0xFFu;
        } else {
            if (k != key_prefix) continue;
            const int hi_bits = 8 * (pass - 8);
            if (hi_bits && (cl >> (32 - hi_bits)) != (cell_prefix >> (32 - hi_bits))) continue;
            digit = (cl >> (24 - 8 * (pass - 8))) & 0xFFu;
        }
        atomicAdd(&h[digit], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

// convert the candidates at or below the composite threshold (t_key, t_cell),
// or all of them
__global__ void k_apply(const uint64_t* __restrict__ key, const uint32_t* __restrict__ cell, long long nc,
                        uint64_t t_key, uint32_t t_cell, int all, uint8_t* phase, int code) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nc;
         j += (long long)gridDim.x * blockDim.x) {
        const uint64_t k = key[j];
        if (all || k < t_key || (k == t_key && cell[j] <= t_cell)) phase[cell[j]] = (uint8_t)code;
    }
}

__global__ void k_region_not_adjacent(const uint8_t* __restrict__ phase, int nx, int ny, int nz, int code, int avoid,
                                      uint8_t* __restrict__ region) {
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        bool ok = phase[c] == code;
        if (ok) {
            const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
            const int xs[6] = {x + 1 == nx ? 0 : x + 1, x == 0 ? nx - 1 : x - 1, x, x, x, x};
            const int ys[6] = {y, y, y + 1 == ny ? 0 : y + 1, y == 0 ? ny - 1 : y - 1, y, y};
            const int zs[6] = {z, z, z, z, z + 1 == nz ? 0 : z + 1, z == 0 ? nz - 1 : z - 1};
#pragma unroll
            for (int d = 0; d < 6; ++d)
                if (phase[xs[d] + (long long)nx * (ys[d] + (long long)ny * zs[d])] == avoid) ok = false;
        }
        region[c] = ok ? 1 : 0;
    }
}

__global__ void k_reactive_faces(const uint8_t* __restrict__ phase, int nx, int ny, int nz, int from_code,
                                 int to_code, double fraction, uint64_t seed, uint8_t* __restrict__ out,
                                 unsigned long long* total) {
    const long long N = (long long)nx * ny * nz;
    unsigned long long n = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        unsigned bits = 0;
        if (phase[c] == from_code) {
            const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
            const int dx[6] = {1, -1, 0, 0, 0, 0}, dy[6] = {0, 0, 1, -1, 0, 0}, dz[6] = {0, 0, 0, 0, 1, -1};
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                const int qx = x + dx[d];
                if (qx < 0 || qx >= nx) continue;
                const int qy = (y + dy[d] + ny) % ny, qz = (z + dz[d] + nz) % nz;
                if (phase[qx + (long long)nx * (qy + (long long)ny * qz)] != to_code) continue;
                if (fraction >= 1.0 || u01(hash4(seed, 0xface, (uint64_t)c, (uint64_t)d)) < fraction) {
                    bits |= 1u << d;
                    ++n;
                }
            }
        }
        out[c] = (uint8_t)bits;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(total, n);
}

constexpr int kGrid = 152 * 8, kBlock = 256;

// scratch: keys (8 B per cell), cells (4 B per cell), then counters and the
// digit histogram from a 256-byte boundary
size_t scratch_tail(long long N) { return (12 * (size_t)N + 255) / 256 * 256; }

cl_status read_u64(unsigned long long* d, unsigned long long* h, cudaStream_t s) {
    CK(cudaMemcpyAsync(h, d, sizeof(*h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return CL_OK;
}

cl_status check_box(int nx, int ny, int nz) {
    const long long N = (long long)nx * ny * nz;
    if (nx < 1 || ny < 1 || nz < 1 || N >= (1LL << 31)) { set_msg_txt("box size out of range"); return CL_ERR_ARG; }
    return CL_OK;
}

cl_status grow_impl(uint8_t* phase, int nx, int ny, int nz, int code, unsigned allowed, unsigned grown,
                    const uint8_t* region, long long target, double c_d, double p_alpha, uint64_t seed,
                    uint64_t stream, int max_sweeps, long long* final_count, cudaStream_t s, unsigned char* scr) {
    const long long N = (long long)nx * ny * nz;
    uint64_t* key = (uint64_t*)scr;
    uint32_t* cell = (uint32_t*)(scr + 8 * (size_t)N);
    unsigned long long* cnt = (unsigned long long*)(scr + scratch_tail(N));  // [0] count, [1] candidates
    unsigned* hist = (unsigned*)(cnt + 4);
    unsigned long long h = 0;
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    k_count_code<<<kGrid, kBlock, 0, s>>>(phase, N, code, cnt);
    CK(cudaGetLastError());
    CKS(read_u64(cnt, &h, s));
    long long count = (long long)h;
    for (int sweep = 0; sweep <= max_sweeps && count < target; ++sweep) {
        if (sweep == 0 && c_d <= 0) continue;
        CK(cudaMemsetAsync(cnt + 1, 0, sizeof(unsigned long long), s));
        k_candidates<<<kGrid, kBlock, 0, s>>>(phase, region, nx, ny, nz, allowed, grown, c_d, p_alpha, seed, stream,
                                              sweep, key, cell, cnt + 1);
        CK(cudaGetLastError());
        CKS(read_u64(cnt + 1, &h, s));
        const long long nc = (long long)h;
        if (nc == 0) continue;
        const long long need = target - count;
        if (nc <= need) {
            k_apply<<<kGrid, kBlock, 0, s>>>(key, cell, nc, 0, 0, 1, phase, code);
            CK(cudaGetLastError());
            count += nc;
            continue;
        }
        // the need-th smallest (key, cell), one byte at a time from the top
        uint64_t t_key = 0;
        uint32_t t_cell = 0;
        long long k = need;
        for (int pass = 0; pass < 12; ++pass) {
            unsigned hh[256];
            CK(cudaMemsetAsync(hist, 0, sizeof(hh), s));
            k_digit_hist<<<kGrid, kBlock, 0, s>>>(key, cell, nc, pass, t_key, t_cell, hist);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            int d = 0;
            while (d < 255 && k > (long long)hh[d]) { k -= hh[d]; ++d; }
            if (pass < 8) t_key |= (uint64_t)d << (56 - 8 * pass);
            else t_cell |= (uint32_t)d << (24 - 8 * (pass - 8));
        }
        k_apply<<<kGrid, kBlock, 0, s>>>(key, cell, nc, t_key, t_cell, 0, phase, code);
        CK(cudaGetLastError());
        count += need;
    }
    if (final_count) *final_count = count;
    return CL_OK;
}

}  // namespace

}  // namespace cl

using namespace cl;

extern "C" {

cl_status cl_qsgs_grow(uint8_t* phase, int nx, int ny, int nz, int code, unsigned allowed_mask, unsigned grown_mask,
                       const uint8_t* region, long long target, double c_d, double p_alpha, uint64_t seed,
                       uint64_t stream, int max_sweeps, long long* final_count, void* cuda_stream) {
    if (!phase) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    CKS(check_box(nx, ny, nz));
    if (code < 0 || code > 3 || !((grown_mask >> code) & 1u)) {
        set_msg_txt("code must be 0..3 and belong to grown_mask");
        return CL_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long N = (long long)nx * ny * nz;
    unsigned char* scr = nullptr;
    CK(cudaMallocAsync((void**)&scr, scratch_tail(N) + 32 + 1024, s));
    cl_status st = grow_impl(phase, nx, ny, nz, code, allowed_mask, grown_mask, region, target, c_d, p_alpha, seed,
                             stream, max_sweeps, final_count, s, scr);
    cudaFreeAsync(scr, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == CL_OK && e != cudaSuccess) { set_msg("cl_qsgs_grow", e); return from_cuda(e); }
    return st;
}

cl_status cl_qsgs_region_not_adjacent(const uint8_t* phase, int nx, int ny, int nz, int code, int avoid,
                                      uint8_t* region, void* cuda_stream) {
    if (!phase || !region) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    CKS(check_box(nx, ny, nz));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_region_not_adjacent<<<kGrid, kBlock, 0, s>>>(phase, nx, ny, nz, code, avoid, region);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return CL_OK;
}

cl_status cl_qsgs_reactive_faces(const uint8_t* phase, int nx, int ny, int nz, int from_code, int to_code,
                                 double fraction, uint64_t seed, uint8_t* out, long long* n_faces, void* cuda_stream) {
    if (!phase || !out) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    CKS(check_box(nx, ny, nz));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned long long* tot = nullptr;
    CK(cudaMallocAsync((void**)&tot, sizeof(*tot), s));
    unsigned long long h = 0;
    cudaError_t e = cudaMemsetAsync(tot, 0, sizeof(*tot), s);
    if (e == cudaSuccess) {
        k_reactive_faces<<<kGrid, kBlock, 0, s>>>(phase, nx, ny, nz, from_code, to_code, fraction, seed, out, tot);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(tot, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_msg("cl_qsgs_reactive_faces", e); return from_cuda(e); }
    if (n_faces) *n_faces = (long long)h;
    return CL_OK;
}

}  // extern "C"
