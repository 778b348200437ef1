// Diffusion preconditioner of the Krylov steady solve on the paper's D3Q19
// lattice (Eq. 22-24): the D3Q7 kernels' counterparts that depend on the
// lattice (the Laplacian row, the cell sums of the populations, the
// equilibrium-shaped correction).  The CG update, direction and scalar
// kernels are the lattice-independent ones of dsa.cu.
#pragma once

#include "internal.cuh"

namespace cl {

// The D3Q19 plain-population layout: padded row pitch px (cells x >= nx hold
// no active cell), link word and catalytic links per padded cell.
struct Dsa19 {
    int px;
    const uint32_t* __restrict__ mask;   // bit i-1: link toward x + c_i closed; kQ19Active
    const uint32_t* __restrict__ react;  // bit i-1: that closed link is catalytic
};

// dinv = 1 / diag(L) on active cells (0 elsewhere); a.N = padded cells
cudaError_t launch_lap_dinv19(const DsaArgs& a, const Dsa19& b, float* dinv, int nblk, cudaStream_t s);
// eps = 0, r = sum_i v_i (v: 19 population planes), z = dinv r, p = z; scalars
cudaError_t launch_cg_start19(const DsaArgs& a, const Dsa19& b, const float* v, const float* dinv, float* eps,
                              float* r, float* zc, float* p, int nblk, double* part, CgScalars* cs, cudaStream_t s);
// one CG iteration on L eps = r0
cudaError_t launch_cg_iter19(const DsaArgs& a, const Dsa19& b, const float* dinv, float* eps, float* r, float* zc,
                             float* p, float* q, int nblk, double* part, CgScalars* cs, cudaStream_t s);
// zout_i = v_i + w_i eps (19 planes)
cudaError_t launch_prec_out19(long long N, const float* v, const float* eps, float* zout, int nblk, cudaStream_t s);

}  // namespace cl
