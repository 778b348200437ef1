// z-marching (C, delta) kernel: shared declarations.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cl {

constexpr int kBX = 64;     // widest tile in x (cells; two per lane of a warp)
constexpr int kBY = 8;      // consumer warps per block (tile rows of the widest tile)
constexpr int kRowsMax = 4;  // tile shapes: RW = 1, 2, 4 rows per warp, tiles (kBX / RW) x (kBY * RW)
constexpr int kStages = 4;  // plane slots per block: z, z+1 in use, two in flight
constexpr int kPrefetchDefault = 0;  // planes beyond the TMA load pulled into L2
constexpr int kThreads = 32 * (kBY + 1);  // one warp per row plus one producer warp

// TMA descriptors of one source time level (main boxes and 16-byte x-halo boxes)
struct MarchMaps {
    CUtensorMap chi, clo, d1, d2, d3, d4, d5, d6, om, mk;
    CUtensorMap chi_h, clo_h, d1_h, d2_h;
};

struct MarchArgs {
    int nx, ny, nz, px;  // px: padded row pitch (multiple of 16 cells, >= kBX)
    int z_chunk;         // planes per block
    int prefetch;        // L2 prefetch distance in planes (0: none)
    // destination time level (padded, two ghost rows per plane)
    float* chi;
    void* clo;
    void* d[6];
    float rfac;
    float rsink;     // 1 - rfac = 2 k_lu / (2w + k_lu), without the cancellation of 1 - rfac
    double rsink_d;
    float c_in, c_out;
    int bc_in, bc_out;
    float s_lo, inv_lo, s_d, inv_d;  // FP16 scales (1 for FP32 storage)
    float* Csnap;
    double* partials;
    int* err;
    // bounded waits: clock cycles before a wait gives up (0: the default, about
    // 1 s of SM clock); never_arrive (a test hook) makes the first plane wait
    // of each work item wait for a load the producer never issues
    long long wait_limit;
    int never_arrive;
};

// One structure of a batch: TMA descriptors and arguments for both source
// parities (args[p] reads time level p and writes level p ^ 1).
struct BatchInst {
    MarchMaps maps[2];
    MarchArgs args[2];
};

// A tile column of one instance over planes [zs, ze), tiles of rw rows per warp
struct WorkItem {
    int inst, x0, y0, zs, ze, rw;
};

struct BatchLaunch {
    int storage;
    int grid;         // co-resident blocks of the plain-step launch (cooperative)
    int grid_reduce;  // co-resident blocks of the reducing-step launch
    int n_inst;
    const BatchInst* insts;
    const WorkItem* items;
    const int* n_items;     // device count, so the list can shrink between graph replays
    const int* inst_count;  // items of each member in the list (0 for a member that stopped)
    int nsteps, parity0, reduce_last;
    unsigned long long* next;  // queue position (zeroed before each launch)
    unsigned long long* done;  // [n_inst] finished items per member (zeroed before each launch)
    int* abort_flag;
    double* item_partials;  // [item][RED_N] when reduce_last
    int* err;
    // step-dependency waits: clock cycles before a block gives up (0: the
    // default, about 2 s of SM clock); never_arrive (a test hook) makes every
    // wait ask for one finished item more than the member has
    long long wait_limit;
    int never_arrive;
};

cudaError_t launch_march_batch(const BatchLaunch& b, cudaStream_t s);
cudaError_t launch_batch_finalize(const double* item_partials, const int* inst_first, const int* inst_count,
                                  int n_inst, double* out, cudaStream_t s);
int march_batch_blocks_per_sm(int storage, bool reduce);

int march_slot_bytes(int storage, int rw);
int march_smem_bytes(int storage, int rw);
int march_blocks_per_sm(int storage, int rw);
// relative cost of stepping one nx x ny plane in tiles of rw rows per warp
double march_tile_cost(int nx, int ny, int storage, int rw);
// tile rows per warp of least cost for an nx x ny plane
int march_auto_rows(int nx, int ny, int storage);
cudaError_t launch_march(int storage, bool reduce, int rw, const MarchMaps& maps, const MarchArgs& a, dim3 grid,
                         cudaStream_t s);
cudaError_t launch_state_init(int storage, const MarchArgs& a, const uint16_t* mask_p, const float* C0,
                              cudaStream_t s);
cudaError_t launch_state_out(int storage, const MarchArgs& a, const uint16_t* mask_p, float* C, float* g,
                             cudaStream_t s);
cudaError_t launch_state_readout(int storage, const MarchArgs& a, const uint16_t* mask_p, double* out,
                                 cudaStream_t s);
cudaError_t launch_pad_static(const uint16_t* mask, const float* omega, int nx, int ny, int nz, int px,
                              uint16_t* mask_p, float* omega_p, cudaStream_t s);

}  // namespace cl
