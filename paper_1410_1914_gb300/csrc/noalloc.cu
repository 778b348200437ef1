// Connectivity mask of the transport phase without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// this answer: a host application that owns every device allocation and
// hands plug-ins only pre-sized buffers, a real-time pipeline that forbids
// allocation after start-up, or a process that has already committed the
// whole device to other work.  For them this file provides a second way to
// compute the set of transport cells connected to the inlet plane: the
// caller passes the phase field and the output mask, and the union-find
// labels, clear flags and error word live in one file-scope static device
// array instead of handle buffers.
//
// The array is sized for kNoAllocMaxCells cells (2^22 = 4,194,304, e.g. a
// 161^3 box): 4 B of labels + 1 B of flags per cell, about 20 MiB, which
// every GPU that loads the library keeps until the process exits.  Every call
// shares it and it keeps the previous call's contents; the kernels rewrite
// labels and flags and this file clears the error word before each use.
// Two calls whose work overlaps on the GPU (different streams, or host
// threads racing) corrupt each other's scratch: serialise them.
//
// Host code must not hand the array's name to a kernel (in host code it is
// only a stand-in symbol); it passes the device address that
// cudaGetSymbolAddress returns.  That address is looked up once per device,
// on the first call made while that device is current; make that first call
// before any stream capture.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr long long kNoAllocMaxCells = 1LL << 22;
constexpr size_t kLabelsBytes = sizeof(int) * (size_t)kNoAllocMaxCells;
constexpr size_t kFlagsBytes = (size_t)kNoAllocMaxCells;
constexpr size_t kScratchBytes = kLabelsBytes + kFlagsBytes + 256;  // + error word

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" cl_status cl_active_mask_noalloc(const uint8_t* phase, int nx, int ny, int nz, int ionomer_transport,
                                            uint8_t* active, void* cuda_stream) {
    if (!phase || !active || nx < 1 || ny < 1 || nz < 1) return CL_ERR_ARG;
    const long long N = (long long)nx * ny * nz;
    if (N > kNoAllocMaxCells) return CL_ERR_ARG;  // larger boxes need the handle API
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CL_ERR_CUDA;
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CL_ERR_CUDA;
            g_scratch_addr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_scratch_addr[dev]);
    }
    int* labels = reinterpret_cast<int*>(base);
    uint8_t* flags = base + kLabelsBytes;
    int* err = reinterpret_cast<int*>(base + kLabelsBytes + kFlagsBytes);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
    if (cl::launch_validate(phase, N, err, s) != cudaSuccess) return CL_ERR_CUDA;
    // transport phases as bits of the phase code: pore and micropore (0x9), plus ionomer (0xD)
    if (cl::launch_percolation(phase, nx, ny, nz, ionomer_transport ? 0xD : 0x9, labels, flags, active, err, s) !=
        cudaSuccess)
        return CL_ERR_CUDA;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
    if (herr & 1) return CL_ERR_ARG;      // a phase code outside 0..3
    if (herr & 2) return CL_ERR_TIMEOUT;  // the labelling hit its iteration bound
    return CL_OK;
}
