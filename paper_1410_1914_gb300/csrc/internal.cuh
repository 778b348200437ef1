// Internal declarations of the CUDA library (not part of the public ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cl_lbm.h"

namespace cl {

// D3Q7: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z.  w0 = 1/4, w1..6 = 1/8.
constexpr float kW0 = 0.25f;
constexpr float kW1 = 0.125f;

// Link-mask bits per active cell.
constexpr uint16_t kClosedShift = 0;   // bit d-1: face toward x + c_d closed
constexpr uint16_t kReactShift = 6;    // bit 6 + d-1: that face is a catalytic sink
constexpr uint16_t kActiveBit = 1u << 12;

// Reduction slots of the fused check (FP64 per block, then a fixed-order sum).
enum RedSlot { RED_JIN = 0, RED_JOUT, RED_R, RED_SUMC, RED_DC, RED_ABSC, RED_NONFINITE, RED_N };

struct StepArgs {
    int nx, ny, nz;
    long long N;
    const uint16_t* __restrict__ mask;
    const float* __restrict__ omega;
    float rfac;          // (2w - k_lu) / (2w + k_lu), w = 1/8 on every axis link
    float rsink;         // 1 - rfac = 2 k_lu / (2w + k_lu), formed without the cancellation of 1 - rfac
    double rsink_d;      // the same in FP64
    float abb_in;        // 2 w C_in
    float abb_out;       // 2 w C_out
    float w_cin, w_cout; // w C_in, w C_out (reduction)
    double rfac_d, abb_in_d, abb_out_d;  // the same three in FP64 (FP64 step)
    int bc_in, bc_out;   // cl_bc
    float* Csnap;        // C at the previous check (reduction)
    double* partials;    // [blocks][RED_N] (reduction)
    int wide;            // 1: 64-bit element offsets even where 32-bit ones fit
    // non-uniform kinetics and sources (coupled problem, Eq. 16-18); NULL: uniform k, no source
    const double* __restrict__ kscale;  // per-cell factor on k_lu (Eq. 17b with a non-uniform potential)
    double k_lu;                        // k dt / dx
    const double* __restrict__ src;     // per-cell amount added per step, as w_i S after collision (Eq. 21)
};

// reactive factor r = (2w - k) / (2w + k) of a cell whose rate constant is
// k_lu times kscale (w = 1/8, so 2w = 1/4)
__device__ __forceinline__ double cell_rfac(double k_lu, double kscale) {
    const double k = k_lu * kscale;
    return (0.25 - k) / (0.25 + k);
}
// its complement 1 - r = 2k / (2w + k): the fraction a catalytic face keeps.
// Formed directly, because k is often ~1e-8 of 2w at nm-scale voxels, where
// 1 - r taken from a rounded r loses most (FP32: all) of its digits.
__device__ __forceinline__ double cell_sink(double k_lu, double kscale) {
    const double k = k_lu * kscale;
    return 2.0 * k / (0.25 + k);
}

// ---- D3Q19 (q19.cu) ----
constexpr int kQ19Threads = 128;
constexpr uint32_t kQ19LinkBits = (1u << 18) - 1;  // bit i-1: link toward x + c_i
constexpr uint32_t kQ19HasReact = 1u << 18;
constexpr uint32_t kQ19Active = 1u << 19;

struct Q19Args {
    int nx, ny, nz, px;   // px: padded row pitch (multiple of 32 cells)
    long long NP;         // px * ny * nz
    const uint32_t* __restrict__ mask;
    const uint32_t* __restrict__ react;
    const float* __restrict__ omega;
    float rfac;           // (cs^2 - k_lu) / (cs^2 + k_lu), cs^2 = 1/3
    double rfac_d;        // the same in FP64 (FP64 step)
    float rsink;          // 1 - rfac = 2 k_lu / (cs^2 + k_lu), without cancellation
    double rsink_d;
    float c_in, c_out;
    double c_in_d, c_out_d;
    int bc_in, bc_out;
    float* Csnap;         // padded (reduction)
    double* partials;     // [blocks][RED_N] (reduction)
    float s_lo, inv_lo, s_d, inv_d;  // FP16 state scales (1 otherwise)
    int wide;             // 1: 64-bit element offsets even where 32-bit ones fit
};

// One time level of the D3Q19 (C, delta) state in the padded layout:
// (hi, lo) of C side by side as float2, 18 deviation planes (f32 | f16 * s_d).
struct Q19State {
    float2* hl;
    void* d;
};

cudaError_t launch_masks19(const uint8_t* phase, const uint8_t* active, const uint8_t* react_in, int rule,
                           int nx, int ny, int nz, int px, uint32_t* mask, uint32_t* react, cudaStream_t s);
cudaError_t launch_pad_omega19(const float* omega, int nx, int ny, int nz, int px, float* out, cudaStream_t s);
cudaError_t launch_linkcount19(const uint32_t* mask, const uint32_t* react, long long NP, double* partials,
                               int nblocks, double* out, cudaStream_t s);
cudaError_t launch_init19(float* pop, const uint32_t* mask, const float* C0, int nx, int ny, int nz, int px,
                          double c_in, double c_out, float* Csnap, cudaStream_t s);
int step19_blocks(const Q19Args& a);
cudaError_t launch_step19(const float* src, float* dst, const Q19Args& a, bool reduce, cudaStream_t s);
// the same step in FP64 on FP64 populations (no reduction)
cudaError_t launch_step19_f64(const double* src, double* dst, const Q19Args& a, cudaStream_t s);
cudaError_t launch_readout19(const float* pop, const Q19Args& a, double* out, cudaStream_t s);
cudaError_t launch_out19(const float* pop, const uint32_t* mask, int nx, int ny, int nz, int px, float* C, float* g,
                         cudaStream_t s);
int step19s_blocks(int px, int ny, int nz);
cudaError_t launch_step19s(int storage, const Q19State& src, const Q19State& dst, const Q19Args& a, bool reduce,
                           cudaStream_t s);
cudaError_t launch_init19s(int storage, const Q19State& st, const Q19Args& a, const float* C0, cudaStream_t s);
cudaError_t launch_readout19s(int storage, const Q19State& st, const Q19Args& a, double* out, cudaStream_t s);
cudaError_t launch_out19s(int storage, const Q19State& st, const Q19Args& a, float* C, float* g, cudaStream_t s);
cudaError_t launch_links_out(const uint32_t* mask19, const uint32_t* react19, const uint16_t* mask7, int nx, int ny,
                             int nz, int px, uint32_t* wall, uint32_t* react, cudaStream_t s);

// ---- setup (kernels.cu) ----
cudaError_t launch_validate(const uint8_t* phase, long long N, int* d_err, cudaStream_t s);
cudaError_t launch_percolation(const uint8_t* phase, int nx, int ny, int nz, int transport_phase_mask,
                               int* labels, uint8_t* touch, uint8_t* active, int* d_err,
                               cudaStream_t s);
cudaError_t launch_diffusivity(const uint8_t* phase, const uint8_t* active, int nx, int ny, int nz,
                               double dx, double T, double M, double D_b, double D_ionomer,
                               int knudsen, const double* D_override, double* D, double* dp,
                               int32_t* chord13, cudaStream_t s);
cudaError_t launch_chords13(const uint8_t* phase, int nx, int ny, int nz, int32_t* chord13,
                            cudaStream_t s);
cudaError_t launch_check_positive(const uint8_t* active, const double* D, long long N, int* d_err,
                                  cudaStream_t s);
cudaError_t launch_omega(const uint8_t* active, const double* D, long long N, double tau_ref,
                         const double* d_Dmax, float* omega, cudaStream_t s);
cudaError_t launch_masks(const uint8_t* phase, const uint8_t* active, const uint8_t* react_in,
                         int react_rule, int nx, int ny, int nz, uint16_t* mask, cudaStream_t s);
// stats: out[0] n_transport, [1] n_active, [2] wall links, [3] react links,
//        [4] sum d_p over pore cells, [5] pore cells, [6] D_max (max)
cudaError_t launch_stats(const uint8_t* phase, const uint16_t* mask, const double* D,
                         const double* dp, long long N, int nx, int transport_phase_mask,
                         double* partials, int nblocks, double* out, cudaStream_t s);

// ---- FP32 solver (kernels.cu) ----
cudaError_t launch_init_fp32(float* pop, const uint16_t* mask, const float* C0, int nx, int ny,
                             int nz, double c_in, double c_out, float* Csnap, const double* src, cudaStream_t s);
cudaError_t launch_step_fp32(const float* src, float* dst, const StepArgs& a, bool reduce,
                             cudaStream_t s);
// the same step in FP64 on FP64 populations (no reduction)
cudaError_t launch_step_f64(const double* src, double* dst, const StepArgs& a, cudaStream_t s);
int step_fp32_blocks(const StepArgs& a);
cudaError_t launch_absmax(const float* v, long long N, double* partials, int nblocks, double* out,
                          cudaStream_t s);
cudaError_t launch_finalize(const double* partials, int nblocks, int nslots, double* out,
                            cudaStream_t s);
cudaError_t launch_field_fp32(const float* pop, const uint16_t* mask, long long N, float* C,
                              const double* src, cudaStream_t s);
// per-plane readout: out[5*nx]: sumC, count, R, J_in part, J_out part
cudaError_t launch_readout_fp32(const float* pop, const StepArgs& a, double* out, cudaStream_t s);
cudaError_t launch_cell_reaction_fp32(const float* pop, const StepArgs& a, double* out, cudaStream_t s);

// ---- Krylov steady solve (krylov.cu) ----
enum KryFin { KRY_START = 0, KRY_ALPHA, KRY_OMEGA, KRY_BETA };
struct KryScalars {
    double rho, alpha, omega, beta;
    double rr;  // r.r of the latest residual
    int bad;    // 0 running; 1 breakdown or non-finite; 2 nothing left to solve
    int iters;  // BiCGSTAB iterations completed
};
int kry_blocks();
// r = c + sx - x (c nullable), rh = p = r; scalars from r.r
cudaError_t launch_kry_start(const float* x, const float* sx, const float* c, float* r, float* rh, float* p,
                             long long L, int nblk, double* part, KryScalars* ks, cudaStream_t s);
// v = p - Ap; alpha = rho / rh.v
cudaError_t launch_kry_v(const float* p, const float* ap, const float* rh, float* v, long long L, int nblk,
                         double* part, KryScalars* ks, cudaStream_t s);
// s = r - alpha v
cudaError_t launch_kry_s(const float* r, const float* v, float* sv, long long L, int nblk, const KryScalars* ks,
                         cudaStream_t s);
// t = s - As; omega = t.s / t.t
cudaError_t launch_kry_t(const float* sv, const float* as_, float* t, long long L, int nblk, double* part,
                         KryScalars* ks, cudaStream_t s);
// x += alpha p + omega s; r = s - omega t; beta, rho from rh.r; rr = r.r
cudaError_t launch_kry_xr(float* x, const float* p, const float* sv, const float* t, const float* rh, float* r,
                          long long L, int nblk, double* part, KryScalars* ks, cudaStream_t s);
// p = r + beta (p - omega v)
cudaError_t launch_kry_p(const float* r, const float* v, float* p, long long L, int nblk, const KryScalars* ks,
                         cudaStream_t s);
// mixed precision: b = a (f32 -> f64), b = (f32) a, x += sign e, and c = (f32)(sx - x) with ks->rr = |sx - x|^2 (FP64)
cudaError_t launch_kry_to64(const float* a, double* b, long long L, int nblk, cudaStream_t s);
cudaError_t launch_kry_to32(const double* a, float* b, long long L, int nblk, cudaStream_t s);
cudaError_t launch_kry_add64(double* x, const float* e, double sign, long long L, int nblk, cudaStream_t s);
cudaError_t launch_kry_res64(const double* x, const double* sx, float* c, long long L, int nblk, double* part,
                             KryScalars* ks, cudaStream_t s);

// ---- diffusion preconditioner and flexible GMRES (dsa.cu), D3Q7
struct DsaArgs {
    int nx, ny, nz;
    long long N;
    const uint16_t* __restrict__ mask;
    float rfac;          // reactive factor r of a catalytic face
    float rsink;         // 1 - r, without cancellation
    int bc_in, bc_out;   // cl_bc
    const double* __restrict__ kscale;  // per-cell factor on k_lu (NULL: uniform)
    double k_lu;
};
enum CgFin { CG_START = 0, CG_ALPHA, CG_BETA };
struct CgScalars {
    double rz, alpha, beta;
    double rr, rr0;  // r.r now and at the start
    int iters;       // iterations of this solve
    int bad;         // 0 running; 1 breakdown or non-finite; 2 nothing left to solve
};
// dinv = 1 / diag(L) on active cells (0 elsewhere)
cudaError_t launch_lap_dinv(const DsaArgs& a, float* dinv, int nblk, cudaStream_t s);
// eps = 0, r = sum_i v_i (v: 7 population planes), z = dinv r, p = z; scalars
cudaError_t launch_cg_start(const DsaArgs& a, const float* v, const float* dinv, float* eps, float* r, float* zc,
                            float* p, int nblk, double* part, CgScalars* cs, cudaStream_t s);
// one CG iteration on L eps = r0
cudaError_t launch_cg_iter(const DsaArgs& a, const float* dinv, float* eps, float* r, float* zc, float* p, float* q,
                           int nblk, double* part, CgScalars* cs, cudaStream_t s);
// zout_i = v_i + w_i eps
cudaError_t launch_prec_out(long long N, const float* v, const float* eps, float* zout, int nblk, cudaStream_t s);
// *out = x.y (or its square root) in FP64, on the device
cudaError_t launch_dot_dev(const float* x, const float* y, long long L, int nblk, double* part, double* out,
                           int take_sqrt, cudaStream_t s);
// y += sign * coef[0] * x; y = x / nrm[0]; out = a - b (+ c)
cudaError_t launch_axpy_dev(float* y, const float* x, const double* coef, float sign, long long L, int nblk,
                            cudaStream_t s);
cudaError_t launch_scale_dev(float* y, const float* x, const double* nrm, long long L, int nblk, cudaStream_t s);
cudaError_t launch_comb(const float* a, const float* b, const float* c, float* out, long long L, int nblk,
                        cudaStream_t s);

}  // namespace cl
