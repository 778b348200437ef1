// Coupled potential-reaction steady state (Sec. 3.3-3.4, Eq. 16-18).
//
// Two handles on the same voxels: O2 (pore, micropore and ionomer; the
// catalytic faces are the ionomer faces toward solid, the sites of Eq. 18)
// and protons (Eq. 16 in the ionomer, on the box mirrored in x so that its
// inlet plane is the membrane at x = L of the O2 box).  A Picard iteration
// on the ionomer potential phi couples them:
//   1. rate factor per O2 cell (Eq. 17b): s = exp(alpha F (phi - phi_ref) / (R T))
//      on cells with a catalytic face and an ionomer path to the membrane, 0
//      on other catalytic cells (their sites carry no current);
//   2. steady O2 field (Krylov solve of the step map's fixed point);
//   3. proton source per cell (Eq. 18b): S_e = 4 F times the O2 consumed,
//      a sink in Eq. 16, per proton step: -4 F r_cell dt_p / dt_o2 with
//      r_cell the O2 handle's per-cell consumption per step;
//   4. steady potential (Krylov solve on the proton handle);
//   5. phi += relax (phi_new - phi), until max |phi_new - phi| < tol_phi.
// Every per-cell step runs in the kernels below; the host only sequences
// the solves and reads one scalar per outer iteration.
#include <math.h>
#include <string.h>

#include "device_util.cuh"
#include "handle.cuh"

using namespace cl;

namespace {

constexpr double kFaraday = 96485.33212;
constexpr double kRgas = 8.314462618;
constexpr int kCB = 256;
constexpr int kCBlocks = 152 * 4;

__device__ __forceinline__ long long mirror_x(long long c, int nx) {
    const int x = (int)(c % nx);
    return c - x + (nx - 1 - x);
}

// phi = phi_m on proton-conducting cells (in O2 coordinates), 0 elsewhere
__global__ void k_phi_init(const uint8_t* __restrict__ pr_active, int nx, long long N, double phi_m,
                           double* __restrict__ phi) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x)
        phi[c] = pr_active[mirror_x(c, nx)] ? phi_m : 0.0;
}

// step 1: Eq. 17b rate factor on the sites, 0 on catalytic cells without a proton path
__global__ void k_rate_scale(const uint16_t* __restrict__ mask, const uint8_t* __restrict__ pr_active,
                             const double* __restrict__ phi, int nx, long long N, double a_over_rt, double phi_ref,
                             double* __restrict__ kscale) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const uint16_t m = mask[c];
        const bool site = (m & kActiveBit) && ((m >> kReactShift) & 0x3fu) && pr_active[mirror_x(c, nx)];
        kscale[c] = site ? exp(a_over_rt * (phi[c] - phi_ref)) : 0.0;
    }
}

// step 3: proton source (mirrored) from the O2 consumption; block sums of the O2 consumption
__global__ void k_proton_source(const double* __restrict__ r_cell, int nx, long long N, double factor,
                                double* __restrict__ src, double* __restrict__ partials) {
    double acc[1] = {0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const double r = r_cell[c];
        src[mirror_x(c, nx)] = -factor * r;
        acc[0] += r;
    }
    block_sum_store<1>(acc, partials + blockIdx.x);
}

// step 5: relaxed update of phi from the proton field; block maxima of |phi_new - phi|
__global__ void k_phi_update(const float* __restrict__ field_pr, const uint8_t* __restrict__ pr_active, int nx,
                             long long N, double relax, double* __restrict__ phi, double* __restrict__ partials) {
    double m = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const long long cm = mirror_x(c, nx);
        if (!pr_active[cm]) continue;
        const double pn = (double)field_pr[cm];
        const double d = pn - phi[c];
        m = fmax(m, fabs(d));
        phi[c] += relax * d;
    }
    __shared__ double sh[kCB];
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// one block: sum (op 0) or max (op 1) of n partials, in a fixed order
__global__ void k_reduce1(const double* __restrict__ partials, int n, int op, double* out) {
    __shared__ double sh[kCB];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v = op ? fmax(v, partials[i]) : v + partials[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = op ? fmax(sh[threadIdx.x], sh[threadIdx.x + w])
                                                  : sh[threadIdx.x] + sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

struct Buf {
    cudaStream_t s;
    std::vector<void*> p;
    explicit Buf(cudaStream_t st) : s(st) {}
    template <class T>
    cudaError_t get(T** out, long long n) {
        void* v = nullptr;
        cudaError_t e = cudaMallocAsync(&v, sizeof(T) * (size_t)(n > 0 ? n : 1), s);
        if (e == cudaSuccess) p.push_back(v);
        *out = (T*)v;
        return e;
    }
    ~Buf() {
        cudaStreamSynchronize(s);
        for (void* v : p) cudaFreeAsync(v, s);
        cudaStreamSynchronize(s);
    }
};

}  // namespace

extern "C" cl_status cl_coupled_solve(cl_handle o2, cl_handle pr, const cl_coupled_params* cp, double* phi_out,
                                      int phi_out_is_device, cl_coupled_info* info) {
    if (!o2 || !pr || !cp) { set_msg_txt("NULL argument"); return CL_ERR_ARG; }
    for (cl_lbm* h : {o2, pr}) {
        if (!h->have_structure) { set_msg_txt("no structure loaded"); return CL_ERR_STATE; }
        if (h->march || h->q != 7) {
            set_msg_txt("the coupled solve needs D3Q7 handles with plain f32 populations (CL_STORE_FP32POP)");
            return CL_ERR_STATE;
        }
    }
    if (o2->nx != pr->nx || o2->ny != pr->ny || o2->nz != pr->nz) {
        set_msg_txt("the O2 and proton handles must cover the same box");
        return CL_ERR_ARG;
    }
    if (o2->p.carrier != CL_CARRIER_O2 || pr->p.carrier != CL_CARRIER_PROTON) {
        set_msg_txt("first handle: O2 carrier; second: PROTON carrier");
        return CL_ERR_ARG;
    }
    if (!(cp->relax > 0.0 && cp->relax <= 1.0) || !(cp->tol_phi > 0.0) || cp->max_outer < 1 ||
        !(cp->krylov_tol > 0.0) || cp->krylov_max_iter < 1 || (cp->steady_solver != 0 && cp->steady_solver != 1)) {
        set_msg_txt("relax in (0, 1], tol_phi > 0, max_outer >= 1, krylov_tol > 0, krylov_max_iter >= 1 required");
        return CL_ERR_ARG;
    }
    const long long N = o2->N;
    const int nx = o2->nx;
    cudaStream_t s = o2->s;
    CK(cudaStreamSynchronize(pr->s));
    Buf b(s);
    double *phi = nullptr, *ks = nullptr, *rc = nullptr, *src = nullptr, *part = nullptr, *scal = nullptr;
    float* fpr = nullptr;
    CK(b.get(&phi, N));
    CK(b.get(&ks, N));
    CK(b.get(&rc, N));
    CK(b.get(&src, N));
    CK(b.get(&fpr, N));
    CK(b.get(&part, kCBlocks));
    CK(b.get(&scal, 2));
    k_phi_init<<<kCBlocks, kCB, 0, s>>>(pr->active, nx, N, cp->phi_m, phi);
    CK(cudaGetLastError());
    // the steady state of one carrier: the population-space Krylov solve (max_steps 0: no march
    // after it, which reports CL_ERR_NOT_CONVERGED) or the line-eliminated one
    auto steady = [&](cl_lbm* h, int* iters) -> cl_status {
        if (cp->steady_solver == 1) {
            cl_steady_info li;
            const int restart = cp->krylov_max_iter < 1500 ? cp->krylov_max_iter : 1500;
            // the preconditioner's systems to 1e-3: a tighter inner solve does not cut the outer count
            cl_status e = cl_lbm_solve_steady_lines(h, cp->krylov_tol, cp->krylov_max_iter, restart, 1e-3, &li);
            *iters = li.iterations;
            return e;
        }
        cl_solve_info si;
        long long inner = 0;
        return cl_lbm_solve_krylov_dsa(h, cp->krylov_tol, cp->krylov_max_iter, 0, &si, iters, &inner);
    };
    const double a_over_rt = cp->alpha * kFaraday / (kRgas * o2->p.T_K);
    // S_e = 4 F r_cell dx^3 / dt_o2 per cell volume dx^3; a sink of Eq. 16 per proton step
    const double factor = 4.0 * kFaraday * pr->dt / o2->dt;
    cl_coupled_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.dphi = INFINITY;
    cl_status st = CL_ERR_NOT_CONVERGED;
    for (int outer = 1; outer <= cp->max_outer; ++outer) {
        k_rate_scale<<<kCBlocks, kCB, 0, s>>>(o2->mask, pr->active, phi, nx, N, a_over_rt, cp->phi_ref, ks);
        CK(cudaGetLastError());
        CKS(cl_lbm_set_rate_scale(o2, ks, 1));
        int it = 0;
        cl_status e = steady(o2, &it);
        if (e != CL_OK && e != CL_ERR_NOT_CONVERGED) return e;
        inf.o2_iterations += it;
        CKS(cl_lbm_cell_reaction(o2, rc, 1));
        CK(cudaMemsetAsync(src, 0, sizeof(double) * (size_t)N, s));
        k_proton_source<<<kCBlocks, kCB, 0, s>>>(rc, nx, N, factor, src, part);
        CK(cudaGetLastError());
        k_reduce1<<<1, kCB, 0, s>>>(part, kCBlocks, 0, scal);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
        CKS(cl_lbm_set_source(pr, src, 1));
        e = steady(pr, &it);
        if (e != CL_OK && e != CL_ERR_NOT_CONVERGED) return e;
        inf.proton_iterations += it;
        CKS(cl_lbm_get_field(pr, fpr, 1));
        CK(cudaStreamSynchronize(pr->s));
        k_phi_update<<<kCBlocks, kCB, 0, s>>>(fpr, pr->active, nx, N, cp->relax, phi, part);
        CK(cudaGetLastError());
        k_reduce1<<<1, kCB, 0, s>>>(part, kCBlocks, 1, scal + 1);
        CK(cudaGetLastError());
        double hs[2];
        CK(cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        inf.outer = outer;
        inf.dphi = hs[1];
        // current drawn on the O2 side (4 F times the consumption, Eq. 18b), amperes
        inf.current_o2_A = 4.0 * kFaraday * hs[0] * o2->p.dx_m * o2->p.dx_m * o2->p.dx_m / o2->dt;
        if (hs[1] < cp->tol_phi) {
            st = CL_OK;
            inf.converged = 1;
            break;
        }
    }
    // the current through the membrane: the proton inflow at its fixed-potential face
    double f[5];
    CKS(cl_lbm_fluxes(pr, f));
    inf.current_membrane_A = f[0] * pr->p.dx_m * pr->p.dx_m * pr->p.dx_m / pr->dt;
    if (phi_out) {
        CK(cudaMemcpyAsync(phi_out, phi, sizeof(double) * (size_t)N,
                           phi_out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (info) *info = inf;
    return st;
}
