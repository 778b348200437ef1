// The solver handle behind the opaque cl_handle, shared by the host files
// of the library (not part of the public ABI).
#pragma once

#include <math.h>
#include <vector>

#include "internal.cuh"
#include "march.cuh"

namespace cl {

struct Graph {
    cudaGraphExec_t exec = nullptr;
    int parity = -1;
    long long K = 0;
    bool reduce = false;
};

// One time level of the (C, delta) state, padded rows and two ghost rows per plane.
struct MState {
    float* chi = nullptr;
    void* clo = nullptr;
    void* d[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

}  // namespace cl

// Remaining change of the tracked readout after the last check, from the
// last two increments dq (latest) and dq_prev: the geometric tail
// |dq| rho / (1 - rho) when they shrink with the same sign (0 < rho < 1), no
// bound when they do not shrink (rho >= 1), and, when the sign flips (a
// turning point or an oscillation, where the geometric model does not
// hold), the larger of the two increments -- so that a turning point, where
// one increment is near zero, cannot pass for convergence.  Two zero
// increments (a state that no longer changes) give zero.
inline double remaining_change(double dq, double dq_prev) {
    if (dq == 0.0 && dq_prev == 0.0) return 0.0;
    const double rho = dq / dq_prev;
    if (rho >= 1.0) return INFINITY;
    if (rho > 0.0) return fabs(dq) * rho / (1.0 - rho);
    return fmax(fabs(dq), fabs(dq_prev));
}

struct cl_lbm {
    cl_params p;
    int nx, ny, nz;
    long long N;
    bool march = true;  // (C, delta) storage; false: q f32 populations
    int q = 7;          // lattice: 7 (D3Q7) or 19 (D3Q19, Eq. 22)
    int px = 0;         // padded row pitch
    long long NP = 0;   // padded, ghosted cell count
    int el = 4;         // bytes per stored deviation
    cudaStream_t s = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<std::pair<void*, size_t>> allocs;

    uint8_t *phase = nullptr, *react = nullptr, *active = nullptr, *touch = nullptr;
    int* labels = nullptr;
    int* d_err = nullptr;
    double *D = nullptr, *dp = nullptr;
    float* omega = nullptr;
    uint16_t* mask = nullptr;
    // population layout (D3Q19: 19 planes of the padded px19 x ny x nz box)
    float* pop[2] = {nullptr, nullptr};
    float* Csnap = nullptr;
    int px19 = 0;
    long long NP19 = 0;
    uint32_t *mask19 = nullptr, *react19 = nullptr;
    float* omega19 = nullptr;
    bool q19s = false;  // D3Q19 on the (C, delta) state (FP32 or FP16 storage)
    int wide = 0;       // force 64-bit element offsets (test of the large-box path)
    cl::Q19State st19[2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    // (C, delta) layout
    cl::MState st[2];
    uint16_t* mask_p = nullptr;
    float* omega_p = nullptr;
    float* Csnap_p = nullptr;
    cl::MarchMaps maps[2];
    dim3 mgrid;
    int z_chunk = 0;
    int tile_rw = 1;  // tile rows per consumer warp of the plane march (1, 2, 4)
    int prefetch = cl::kPrefetchDefault;
    float s_lo = 1.f, s_d = 1.f;
    double* kscale = nullptr;  // per-cell factor on k (cl_lbm_set_rate_scale), NULL: uniform
    double* src = nullptr;     // per-cell source per step (cl_lbm_set_source), NULL: none
    double src_sum = 0.0;      // sum of the sources over active cells (enters the flux balance)
    double *kscale_buf = nullptr, *src_buf = nullptr;  // their storage, allocated on first use
    long long wait_limit = 0;  // bounded device waits of the step kernel (0: default)
    int never_arrive = 0;      // test hook (cl_lbm_set_wait_test)

    int cur = 0;
    float* fbuf = nullptr;
    double* partials = nullptr;
    int nblk_step = 0, nblk_stats = 0;
    double* d_red = nullptr;    // [16]
    double* d_plane = nullptr;  // [5 * nx]
    double* h_red = nullptr;    // pinned [16 + 5 * nx]
    bool have_react = false;
    bool have_structure = false;
    long long step = 0;
    double D_b = 0, D_max = 0, dt = 0, k_lu = 0;
    cl_structure_info info;
    cl::Graph graphs[4];
};

namespace cl {

// Host helpers defined in api.cu
void set_msg(const char* where, cudaError_t e);
void set_msg_txt(const char* txt);
cl_status from_cuda(cudaError_t e);
int transport_phases(const cl_params& p);
float reactive_factor(const cl_lbm* h);
double reactive_factor_d(const cl_lbm* h);
double reactive_sink_d(const cl_lbm* h);
MarchArgs make_margs(cl_lbm* h, int dst);
// TMA descriptors of both time levels of the (C, delta) state for tiles of rw rows per warp
cl_status build_march_maps(const cl_lbm* h, int rw, MarchMaps* maps);
cl_status check_err_flag(cl_lbm* h);

}  // namespace cl

#define CK(call)                        \
    do {                                \
        cudaError_t e_ = (call);        \
        if (e_ != cudaSuccess) {        \
            cl::set_msg(#call, e_);     \
            return cl::from_cuda(e_);   \
        }                               \
    } while (0)

#define CKS(stmt)                       \
    do {                                \
        cl_status s_ = (stmt);          \
        if (s_ != CL_OK) return s_;     \
    } while (0)
