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
// cudaGetSymbolAddress returns for the current device.  That lookup is made
// on every call, with the caller's device current: it allocates nothing, and
// an address cached across calls would go stale if the host application reset
// the device's context (cudaDeviceReset), which reloads the module.
//
// Both pointers must be device (or managed) memory of the current device;
// anything else is refused before the first launch.
#include "internal.cuh"

namespace {

constexpr long long kNoAllocMaxCells = 1LL << 22;
constexpr size_t kLabelsBytes = sizeof(int) * (size_t)kNoAllocMaxCells;
constexpr size_t kFlagsBytes = (size_t)kNoAllocMaxCells;
constexpr size_t kScratchBytes = kLabelsBytes + kFlagsBytes + 256;  // + error word

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// true when p is device memory of device dev, or managed memory (a plain or
// pinned host pointer gives false)
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the (non-sticky) error so that later calls do not see it
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == dev;
    return at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" cl_status cl_active_mask_noalloc(const uint8_t* phase, int nx, int ny, int nz, int ionomer_transport,
                                            uint8_t* active, void* cuda_stream) {
    if (!phase || !active || nx < 1 || ny < 1 || nz < 1) return CL_ERR_ARG;
    const long long N = (long long)nx * ny * nz;
    if (N > kNoAllocMaxCells) return CL_ERR_ARG;  // larger boxes need the handle API
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CL_ERR_CUDA;
    if (!on_device(phase, dev) || !on_device(active, dev)) return CL_ERR_ARG;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CL_ERR_CUDA;
    unsigned char* base = static_cast<unsigned char*>(p);
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
