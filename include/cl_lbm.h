/*
 * cl_lbm.h -- C ABI of the GB300 (sm_103a) reactive-diffusion lattice
 * Boltzmann library for catalyst-layer structures, after Chen et al.,
 * arXiv:1410.1914 ("Nanoscale study of reactive transport in catalyst layer
 * of PEM fuel cells with precious and non-precious catalysts using LBM").
 *
 * The library solves, on one GPU, the steady O2 transport of Eq. 6 / Eq. 15
 * in the transport phase of a voxelised catalyst layer:
 *   - per-voxel diffusivity: Eq. 7 (bulk), Eq. 8 (Knudsen, from the
 *     13-direction local pore length of Sec. 2.1.3), Eq. 9 (Bosanquet);
 *   - relaxation time per voxel from Eq. 24 on one of two lattices: D3Q7
 *     (weights 1/4 rest, 1/8 axis; cs^2 = 1/4; D = (tau - 1/2) dx^2 / (4 dt)),
 *     the default and the fast path, or the paper's D3Q19 (Eq. 22-23:
 *     1/3 rest, 1/18 axis, 1/36 face diagonal; cs^2 = 1/3);
 *   - BGK evolution Eq. 21 with equilibrium w_i C (Eq. 23);
 *   - boundaries of Sec. 3.5: fixed concentration (Eq. 19 setup, Eq. 20b)
 *     or zero flux (Eq. 20a) at the x faces, periodic in y and z,
 *     bounce-back on solid faces, and a first-order surface sink on
 *     catalyst faces (the uniform-potential Tafel rate of Eq. 17b placed as a
 *     flux k*C on the face rather than the volumetric source of Eq. 18a);
 *   - readouts: D_eff of Eq. 19 and the total / per-plane reaction rate
 *     (left side of Eq. 25 divided by 4F).
 *
 * Conventions shared by every call:
 *   - Arrays are x-fastest: index = x + nx*(y + ny*z).
 *   - Phase codes: 0 pore, 1 solid (carbon/Pt/catalyst), 2 ionomer,
 *     3 micropore (transports like pore, never reactive).
 *   - Direction codes d = 1..6 are +x, -x, +y, -y, +z, -z.  D3Q19 adds
 *     7 (+1,+1,0), 8 (-1,-1,0), 9 (+1,-1,0), 10 (-1,+1,0), 11 (+1,0,+1),
 *     12 (-1,0,-1), 13 (+1,0,-1), 14 (-1,0,+1), 15 (0,+1,+1), 16 (0,-1,-1),
 *     17 (0,+1,-1), 18 (0,-1,+1); q = 7 or 19 populations per cell.
 *   - Link classes.  The link of an active cell toward x + c_i ends in the
 *     cell x + c_i, or, when it leaves the box through x = 0 or x = L, in
 *     the mirror image (x, y + c_y, z + c_z) of the end plane.  It is a wall
 *     (bounce-back) when that end cell is not active, a boundary link
 *     (fixed value or zero flux) when it leaves the box and its end cell is
 *     active, and open otherwise.  A wall link reacts when its end cell is
 *     solid (1) and it leaves through a catalytic face: one of the faces
 *     that its non-zero components cross is marked (set_structure) and
 *     borders solid.  On D3Q7 every link crosses exactly its own face.
 *   - A pointer argument documented "host or device" is read or written with
 *     cudaMemcpyAsync on the handle's stream; `ptr_is_device` says which.
 *   - Calls are ordered on the handle's CUDA stream.  Calls that return
 *     values to host memory synchronise that stream before returning.
 *   - Every call returns a cl_status; no call throws or aborts.  On
 *     CL_ERR_ARG nothing was changed.  After CL_ERR_CUDA the handle should
 *     be destroyed.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef CL_LBM_H
#define CL_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cl_lbm* cl_handle;

typedef enum {
    CL_OK = 0,
    CL_ERR_ARG = 1,           /* invalid argument (size, pointer, parameter) */
    CL_ERR_OOM = 2,           /* device allocation failed */
    CL_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    CL_ERR_STATE = 4,         /* call out of order (e.g. solve before set_structure) */
    CL_ERR_DIVERGED = 5,      /* NaN/Inf in the readouts */
    CL_ERR_NOT_CONVERGED = 6, /* max_steps reached before the stopping rule */
    CL_ERR_NO_PATH = 7,       /* no transport cell is connected to the inlet plane */
    CL_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up */
} cl_status;

typedef enum { CL_BC_DIRICHLET = 0, CL_BC_ZERO_FLUX = 1 } cl_bc;

typedef enum {
    /* C as a double-float (two f32) + the q-1 post-collision deviations from
       w_i C as f32 (delta_0 implied); FP32 arithmetic on small quantities only */
    CL_STORE_FP32 = 0,
    /* C as f32 + a scaled f16 low word, deviations as scaled f16; FP32 arithmetic */
    CL_STORE_FP16DEV = 1,
    /* plain q x f32 populations per cell (reference layout; its steady state
       carries an FP32 rounding floor that grows with the box) */
    CL_STORE_FP32POP = 2
} cl_storage;

/* Velocity set (Eq. 22).  Both lattices take every storage mode; D3Q19
   handles cannot join a batch. */
typedef enum { CL_LATTICE_D3Q7 = 0, CL_LATTICE_D3Q19 = 1 } cl_lattice;

/* What the solve transports.  O2: the pore space (pore 0 and micropore 3,
   plus ionomer 2 when D_ionomer > 0), Eq. 6 / Eq. 15.  PROTON: the ionomer
   phase alone with the uniform conductivity D_ionomer and no source --
   Eq. 16 with S_e = 0, whose Eq. 19-type readout is the effective proton
   conductivity of Sec. 5.2 (potential boundary values in c_in / c_out). */
typedef enum { CL_CARRIER_O2 = 0, CL_CARRIER_PROTON = 1 } cl_carrier;

typedef enum {
    CL_REACT_GIVEN = 0,   /* reactive faces from the mask given to set_structure (NULL: none) */
    CL_REACT_ALL_PORE_SOLID = 1, /* every face between a pore (0) and a solid (1) cell */
    /* every face between an ionomer (2) and a solid (1) cell: the reaction
       sites of Eq. 18 (ionomer next to Pt), for O2 carried in the ionomer
       (ionomer_o2 or D_ionomer > 0); D3Q7 only */
    CL_REACT_IONOMER_SOLID = 2
} cl_react_rule;

/* Optional device allocator (e.g. a framework's caching allocator).  Both
   NULL: the library uses cudaMallocAsync / cudaFreeAsync on its stream. */
typedef void* (*cl_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*cl_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct {
    int nx, ny, nz;        /* box in voxels, each >= 1; nx*ny*nz < 2^31 */
    double dx_m;           /* voxel edge [m] */
    double T_K;            /* temperature [K] (Eq. 7, Eq. 8) */
    double p_atm;          /* pressure [atm] (Eq. 7) */
    double M_kgmol;        /* O2 molar mass [kg/mol] (Eq. 8) */
    double D_bulk;         /* bulk diffusivity [m^2/s]; <= 0: Eq. 7 */
    double D_ionomer;      /* > 0: ionomer (phase 2) transports with this D; 0: impermeable */
    double k_ms;           /* first-order surface rate constant [m/s] */
    int knudsen;           /* 1: Eq. 8 + Eq. 9 in pore cells; 0: D = D_b */
    int bc_in, bc_out;     /* cl_bc at x = 0 and x = L */
    double c_in, c_out;    /* boundary concentrations (any unit; readouts carry it) */
    double tau_ref;        /* relaxation time of the most diffusive active cell (> 0.5) */
    int storage;           /* cl_storage */
    int react_rule;        /* cl_react_rule */
    int carrier;           /* cl_carrier; PROTON needs D_ionomer > 0 and k_ms = 0 */
    int lattice;           /* cl_lattice */
    int ionomer_o2;        /* 1: O2 dissolved in the ionomer (Eq. 10-15): the ionomer transports
                              the gas-equivalent C with D = D_e(T) (Eq. 13) times RT/H (Eq. 10-11),
                              replacing D_ionomer; O2 carrier only, T > 283.7 K */
    int check_every;       /* steps between convergence checks in cl_lbm_solve (even, >= 2) */
    double tol_flux;       /* |J_in - J_out - R| / |J_in| below this ... */
    double tol_rel;        /* ... and the extrapolated relative error of the tracked readout
                              (D_eff, or R for zero-flux outlets) below this: converged */
    long long max_steps;   /* step budget of cl_lbm_solve */
    void* cuda_stream;     /* cudaStream_t; NULL = legacy default stream */
    cl_alloc_fn alloc;     /* optional, see above */
    cl_free_fn free;
    void* alloc_ctx;
} cl_params;

/* Fills the defaults: T 353 K, 1 atm, M 0.032, dx 1 nm, Dirichlet both ends,
   c_in 1, c_out 0, tau_ref 1, FP32, check_every 1000, tol_flux 1e-4,
   tol_rel 1e-4, max_steps 10^7; sizes 0. */
void cl_params_default(cl_params* p);

typedef struct {
    long long n_cells;        /* nx*ny*nz */
    long long n_transport;    /* transport-phase cells */
    long long n_active;       /* transport cells 6-connected to the inlet plane */
    long long n_wall_links;   /* wall links of active cells (see "Link classes") */
    long long n_react_links;  /* of those, reactive */
    double D_b;               /* bulk diffusivity used [m^2/s] */
    double D_max;             /* largest active-cell diffusivity [m^2/s] */
    double dt_s;              /* lattice time step [s] (Eq. 24 at tau_ref) */
    double k_lu;              /* k dt / dx */
    double mean_pore_diameter_m; /* mean 13-direction length over pore cells (Sec. 2.1.3) */
} cl_structure_info;

typedef struct {
    long long steps;       /* steps taken by this call */
    int converged;         /* 1 if the stopping rule fired */
    double J_in, J_out, R; /* lattice-unit fluxes at the last check (see cl_lbm_fluxes) */
    double flux_balance;   /* |J_in - J_out - R| / |J_in| at the last check */
    double rel_change;     /* extrapolated relative error of the tracked readout */
    double resid;          /* sum|C(t) - C(t-K)| / sum|C(t)| over the last interval */
    double seconds;        /* wall time of the call */
} cl_solve_info;

/* Create a solver for a box of p->nx * p->ny * p->nz voxels.  Allocates all
   device buffers (through p->alloc if given).  *out is set only on CL_OK.
   Errors: CL_ERR_ARG (bad sizes/parameters, e.g. an unknown lattice or
   storage, ionomer_o2 with the proton carrier), CL_ERR_OOM, CL_ERR_CUDA. */
cl_status cl_lbm_create(cl_handle* out, const cl_params* p);

/* Free every buffer of the handle (NULL is ignored). */
void cl_lbm_destroy(cl_handle h);

/* Load a structure (Sec. 2 reconstruction output) and run the set-up on
   the GPU: transport set, cells reachable from the inlet plane (Sec. 2.1.3
   connectivity), 13-direction pore lengths (Sec. 2.1.3), per-cell D
   (Eq. 7-9), tau/omega (Eq. 24), link masks, then the linear initial field.
     phase:          nx*ny*nz bytes of phase codes (host or device); copied.
     reactive_faces: nx*ny*nz bytes, bit d-1 = face toward x + c_d is
                     catalytic, or NULL (no reaction unless react_rule says
                     otherwise); copied.  A face reacts only if it is marked,
                     belongs to an active cell and its neighbour is solid (1);
                     on D3Q19 the links that cross such a face react (see
                     "Link classes").
   Errors: CL_ERR_ARG (phase code > 3), CL_ERR_NO_PATH, CL_ERR_CUDA. */
cl_status cl_lbm_set_structure(cl_handle h, const uint8_t* phase, const uint8_t* reactive_faces,
                               int ptr_is_device);

/* Replace the Eq. 7-9 diffusivities of the active cells by D [m^2/s]
   (nx*ny*nz doubles, host or device; values of inactive cells ignored; each
   active value must be > 0) and re-derive tau, omega and dt, then re-apply
   the linear initial field.  For layered closed-form cases and for callers
   with their own diffusivity model.  Errors: CL_ERR_STATE, CL_ERR_ARG. */
cl_status cl_lbm_set_diffusivity(cl_handle h, const double* D, int ptr_is_device);

/* Initial field: populations at equilibrium w_i C (Eq. 23).  C0 (nx*ny*nz
   floats, host or device) or NULL for the linear ramp C_in -> C_out between
   the half-way faces x = 0 and x = L.  Resets the step counter. */
cl_status cl_lbm_init(cl_handle h, const float* C0, int ptr_is_device);

/* Advance exactly nsteps time steps (Eq. 21 with the boundaries above). */
cl_status cl_lbm_step(cl_handle h, long long nsteps);

/* Advance until the stopping rule fires or p->max_steps more steps are
   taken: every check_every steps the fused reduction gives J_in, J_out, R
   and sum|dC|; converged when, at two checks in a row, the flux balance is
   below tol_flux and the estimated remaining change of the tracked readout
   (D_eff for a Dirichlet outlet, R otherwise) is below tol_rel of it.  The
   estimate is the geometric-series tail of the last two increments when
   they shrink with one sign, and the larger increment when the sign flips
   (a turning point, as after a warm start that overshoots).
   Returns CL_ERR_NOT_CONVERGED at the budget, CL_ERR_DIVERGED on NaN/Inf.
   info may be NULL. */
cl_status cl_lbm_solve(cl_handle h, cl_solve_info* info);

/* Test hook of the step kernel's bounded waits (no counterpart in the
   paper; D3Q7 (C, delta) storage, the only kernel with device-side waits).
   wait_limit_clocks: SM clock cycles a consumer or producer warp waits on a
   plane's mbarrier before it gives up (0: the default, about 1 s).
   never_arrive (needs a limit > 0): the producer issues no plane load, so
   the consumers' first wait runs out after the limit; the kernel then
   returns without touching the state, and cl_lbm_solve / _solve_budget
   report CL_ERR_TIMEOUT.  The error word is cleared once reported; set
   (0, 0) to restore normal stepping.  Drops the captured step graphs.
   Errors: CL_ERR_ARG. */
cl_status cl_lbm_set_wait_test(cl_handle h, long long wait_limit_clocks, int never_arrive);

/* Tile shape of the plane-marching step kernel ((C, delta) storage; a
   layout choice with no counterpart in the paper).  A thread block steps a
   column of 512 cells, rows x of 64 / rows cells by 8 * rows (rows = 1, 2 or
   4: 64 x 8, 32 x 16, 16 x 32 cells) through its planes; a narrow tile leaves
   fewer lanes idle where nx is not a multiple of 64.  rows = 0 restores the
   default, the shape with the fewest cell slots along x (ties to the wider
   tile).  The arithmetic is the same for every shape (the results are
   bit-identical).  rows_out (may be NULL) receives the shape in use.  Drops
   the captured step graphs.  A batch takes each member's shape when it is
   created.  Errors: CL_ERR_ARG (rows), CL_ERR_STATE (population storage),
   CL_ERR_CUDA. */
cl_status cl_lbm_set_tile_rows(cl_handle h, int rows, int* rows_out);

/* cl_lbm_solve with an explicit step budget instead of p->max_steps (whole
   check intervals only; a budget below check_every runs no step).  Each call
   restarts the stopping rule's history, so a budget of one interval always
   returns CL_ERR_NOT_CONVERGED with that interval's readouts in info. */
cl_status cl_lbm_solve_budget(cl_handle h, long long max_steps, cl_solve_info* info);

/* Steady state by a Krylov method instead of the time march, then the
   stopping rule above as its certificate.  The steady state the march of
   Eq. 21-24 approaches is the fixed point x = S(x) of one step S on the
   stored post-collision populations; S is affine, S(x) = A x + b (A: the
   step with zero boundary concentrations, b: the Dirichlet terms), so the
   fixed point solves (I - A) x = b.  Mixed-precision refinement: the
   iterate is held in FP64 and its residual r = S(x) - x (the change one
   more step would make) is taken with the FP64 step; each correction
   solves (I - A) e = r with BiCGSTAB on f32 vectors and the f32 step
   kernel (two applications per iteration) to 1e-3 of |r|, restarted from
   the true residual on breakdown (at most 4 restarts); x += e.  It stops
   when |r| (2-norm over all populations, FP64) falls to tol times its
   initial value, when max_iter BiCGSTAB iterations are spent, or when a
   correction no longer halves |r|.  The result, rounded to f32, replaces
   the state, and cl_lbm_solve_budget(h, max_steps, info) then runs the
   time march from it: the return value and info are those of the stopping
   rule (max_steps 0: no step, CL_ERR_NOT_CONVERGED with the readouts of
   the Krylov state), except that info->seconds covers the whole call.
     tol:        > 0, relative to the initial residual norm.
     max_iter:   >= 0 BiCGSTAB iterations in all.
     iterations: nullable; the iterations taken.
   Where it pays: with uniform relaxation times (bulk diffusivity, no
   Knudsen term) the 48^3 Pt layer converges in about 330 iterations, far
   fewer step applications than the march needs.  With the Knudsen term the
   relaxation times spread over (1/2, 1], the unpreconditioned iteration
   stalls after the first correction, and the call returns a state of lower
   residual that is not converged: give max_steps for the march to finish.
   Needs storage CL_STORAGE_FP32POP (either lattice), else CL_ERR_STATE.
   Allocates 8 f32 and 2 FP64 population-sized vectors for the call
   (through p->alloc if given) and frees them before returning.
   Errors: CL_ERR_ARG (tol <= 0, max_iter < 0, max_steps < 0), CL_ERR_STATE,
   CL_ERR_OOM, CL_ERR_CUDA, and the codes of cl_lbm_solve_budget. */
cl_status cl_lbm_solve_krylov(cl_handle h, double tol, int max_iter, long long max_steps, cl_solve_info* info,
                              int* iterations);

/* cl_lbm_solve_krylov with each f32 correction found by flexible GMRES(30)
   with a diffusion preconditioner, on either lattice.  The slow modes of the
   step map are diffusive: a correction of equilibrium shape w_i eps changes
   the cell sums by L eps in one step, L being the Laplacian of the active
   cells with the lattice weight w_i on each link (D3Q7: 1/8; D3Q19: 1/18
   axial, 1/36 diagonal; 2 w_i on a fixed-concentration face, (1 - r) w_i
   on a catalytic face, 0 on a bounce-back face).  The preconditioner
   P v = v + w_i eps with L eps = sum_i v_i (diagonal-preconditioned
   conjugate gradients to 1e-2) keeps the number of step applications
   small as the box grows (it levels off near 100) and with a spread of
   relaxation times (Knudsen): 15 for the bulk-D 48^3 Pt layer, about 80
   for Knudsen layers of 24^3 and 32^3, where the unpreconditioned solve
   stalls.
   Each GMRES cycle (at most 10 per correction) restarts from the true
   residual.  Refinement, stopping and certification as in
   cl_lbm_solve_krylov.
     iterations:       nullable; GMRES iterations (step applications).
     inner_iterations: nullable; conjugate-gradient iterations in all.
   Needs CL_STORAGE_FP32POP, else CL_ERR_STATE.  Allocates 64 f32
   and 2 FP64 population-sized vectors plus 6 f32 cell fields for the call
   (through p->alloc if given) and frees them before returning.
   Errors: as cl_lbm_solve_krylov. */
cl_status cl_lbm_solve_krylov_dsa(cl_handle h, double tol, int max_iter, long long max_steps, cl_solve_info* info,
                                  int* iterations, long long* inner_iterations);

/* The steady state with the populations eliminated along lines (no
   counterpart in the paper, which marches Eq. 21 in time).  At steady state
   the populations of each axis obey, along every run of open faces, a
   two-stream recursion driven by C (g_i(x + c_i) = (1 - omega) g_i(x) +
   omega w C(x) + w S(x), with the wall, catalytic, fixed-value and
   zero-flux rules at the run's ends), which one sweep per direction solves
   exactly; summing them gives C = F(C), an affine map of C alone whose fixed
   point is exactly the steady state of the march.  (I - M) C = F(0) (M the
   linear part of F) is solved by flexible GMRES(restart) in FP64,
   preconditioned by the finite-volume operator with the scheme's link
   conductances (2 D_a D_b / (D_a + D_b), D = cs^2 (tau - 1/2); 2 D on a
   fixed-value face; 2 k D / (2 D + k) on a catalytic face), whose systems
   diagonal-preconditioned FP64 conjugate gradients solve to cg_tol.
   Relaxation rates are formed in FP64 from the stored D (Eq. 24).  This
   reaches the steady state of O2 dissolved in the ionomer (Eq. 10-15,
   relaxation times within 1e-5 of 1/2 there), where the march and the
   population-space Krylov solves stall; per-cell rate factors and sources
   (cl_lbm_set_rate_scale / _set_source) are honoured.
     tol:      stop when |F(C) - C| falls to tol times |F(0)| (the right-hand
               side; a warm start close to the answer stops at once).
     max_iter: GMRES iterations (applications of F) in all.
     restart:  Krylov vectors kept; the call allocates 2 * restart + 8
               FP64 cell fields (restart 1000 at 32^3: 0.5 GB), freed
               before returning.
     cg_tol:   relative residual of each preconditioner solve, in (0, 1);
               1e-3 is enough (at 24^3 and 33x33x32 the outer count is the
               same as with 1e-10, the inner work less than half).
   Starts from the current state's C; on return the state holds the
   post-collision populations of the result, so every readout applies.
   Needs D3Q7 and CL_STORE_FP32POP, else CL_ERR_STATE.  Returns
   CL_ERR_NOT_CONVERGED at max_iter, CL_ERR_DIVERGED on a non-finite
   residual or a breakdown of the inner solve, CL_ERR_OOM / CL_ERR_CUDA. */
typedef struct {
    int iterations;              /* GMRES iterations (applications of F) */
    int cycles;                  /* GMRES cycles */
    long long inner_iterations;  /* conjugate-gradient iterations of the preconditioner */
    double residual;             /* |F(C) - C| / |F(0)| at the end */
    double seconds;              /* wall time of the call */
    double J_in, J_out, R;       /* fluxes of the result in FP64, lattice units per step (as
                                    cl_lbm_fluxes, which reads the f32 populations) */
} cl_steady_info;

cl_status cl_lbm_solve_steady_lines(cl_handle h, double tol, int max_iter, int restart, double cg_tol,
                                    cl_steady_info* info);

/* Lattice-unit fluxes of the current state, FP64 sums:
   out[0] J_in  net amount entering through x = 0 per step,
   out[1] J_out net amount leaving through x = L per step,
   out[2] R     amount consumed on reactive faces per step,
   out[3] sum of C over active cells,
   out[4] number of active cells.
   Per step: sum C(t+1) - sum C(t) = J_in - J_out - R. */
cl_status cl_lbm_fluxes(cl_handle h, double out[5]);

/* Eq. 19 from the outlet flux: D_eff [m^2/s] and D_eff / D_b.  For the
   PROTON carrier the same readout is the effective conductivity (in the
   unit of D_ionomer) and the ratio is taken to D_ionomer (Sec. 5.2).  Needs
   Dirichlet at both ends and c_in != c_out (else CL_ERR_STATE).
   Either pointer may be NULL. */
cl_status cl_lbm_effective_diffusivity(cl_handle h, double* d_eff_m2s, double* d_eff_over_db);

/* Reaction rate: total = sum over reactive faces of k C_wall dx^2, in
   (concentration unit) * m^3 / s (mol/s for C in mol/m^3).  profile_R
   (nullable, nx doubles, host): the same per x-plane.  profile_C
   (nullable, nx doubles, host): mean C over the active cells of each plane
   (0 where none). */
cl_status cl_lbm_reaction_rate(cl_handle h, double* total, double* profile_R, double* profile_C);

/* Eq. 25: the discharge current density the reaction carries,
   i_d = 4 F R / A_cross, with R the total rate above (O2 in mol/s when C is
   in mol/m^3), four electrons per O2 (ORR), F = 96485.33212 C/mol and
   A_cross = ny nz dx^2 the cross-section of the layer; A/m^2.
   CL_ERR_STATE for the PROTON carrier (it has no sink). */
cl_status cl_lbm_current_density(cl_handle h, double* i_d);

/* ---------------------------------------------------------------------
 * Non-uniform kinetics and sources: the coupled potential-reaction problem
 * of Sec. 3.3-3.4 (Eq. 16-18).  These act on D3Q7 handles with plain f32
 * populations (CL_STORE_FP32POP; CL_ERR_STATE otherwise), the storage of
 * the Krylov steady solves, and are cleared by cl_lbm_set_structure.
 * --------------------------------------------------------------------- */

/* Per-cell factor s on the rate constant of the catalytic faces (Eq. 17b
   with the local ionomer potential: k = k_ms * s, so r = (2w - k s) /
   (2w + k s) per cell).  kscale: nx*ny*nz doubles (host or device), copied;
   NULL restores the uniform k.  s = 0 makes a face an inert wall. */
cl_status cl_lbm_set_rate_scale(cl_handle h, const double* kscale, int ptr_is_device);

/* Per-cell source S, the amount added to C per step in lattice units
   (Eq. 16's S_e, or Eq. 15's source, times dt): after collision each
   population gains w_i S (the a_i S term of Eq. 21).  S: nx*ny*nz doubles
   (host or device), copied; entries of inactive cells are ignored; NULL
   removes the source.  The stopping rule's flux balance then reads
   J_in - J_out - R + sum S. */
cl_status cl_lbm_set_source(cl_handle h, const double* S, int ptr_is_device);

/* Per-cell amount of the transported quantity consumed per step on the
   catalytic faces (lattice units, C times one cell volume per step; 0 on
   cells without a catalytic face): (1 - r) times the post-collision
   populations that meet those faces.  out: nx*ny*nz doubles, host or
   device.  The O2 consumption of Eq. 18 per cell is out * dx^3 / dt. */
cl_status cl_lbm_cell_reaction(cl_handle h, double* out, int ptr_is_device);

/* The coupled steady state of O2 and protons (Sec. 3.3-3.4): the reading
   of Eq. 16-18 with a non-uniform ionomer potential phi.
   o2: O2 carrier with the ionomer transporting O2 (ionomer_o2 = 1, or
       D_ionomer > 0) and the reaction sites of Eq. 18 as its catalytic faces
       (react_rule CL_REACT_IONOMER_SOLID); its k_ms is the rate constant at
       phi_ref (Eq. 17b).
   pr: PROTON carrier (D_ionomer = the conductivity sigma, k_ms = 0) on the
       same voxels mirrored in x (phase[z][y][nx-1-x]), so that its inlet
       plane is the membrane at x = L of the O2 box: bc_in Dirichlet with
       c_in = phi_m, bc_out zero flux (no protons cross the gas side).
   Both: D3Q7, CL_STORE_FP32POP, structures loaded.
   Picard iteration on phi (O2 coordinates), each step in device kernels:
   rate factor exp(alpha F (phi - phi_ref) / (R T)) on catalytic cells with
   an ionomer path to the membrane (0 on the others, which carry no
   current); the O2 steady state (cl_lbm_solve_krylov_dsa, or
   cl_lbm_solve_steady_lines with steady_solver = 1); the proton
   source -4 F r_cell dt_p / dt_o2 per proton step (Eq. 18b, r_cell the
   per-cell O2 consumption per O2 step); the proton steady state; then
   phi += relax (phi_new - phi) until max |phi_new - phi| < tol_phi.
   phi_out (nullable, nx*ny*nz doubles, host or device): phi on the
   proton-conducting cells, 0 elsewhere.  Leaves both handles at their last
   steady states (their rate scale and source set).  Allocates its scratch
   (5 cell fields) with cudaMallocAsync and frees it before returning.
   Returns CL_ERR_NOT_CONVERGED if max_outer iterations did not bring the
   change of phi below tol_phi.  Errors: CL_ERR_ARG, CL_ERR_STATE and those
   of the Krylov solve. */
typedef struct {
    double alpha;        /* transfer coefficient of Eq. 17b (Table 1: 0.61) */
    double phi_m;        /* membrane potential [V], the proton handle's c_in */
    double phi_ref;      /* potential [V] at which the O2 handle's k_ms holds */
    double relax;        /* Picard relaxation, (0, 1] */
    double tol_phi;      /* stop when max |phi_new - phi| < tol_phi [V] */
    int max_outer;       /* >= 1 */
    double krylov_tol;   /* residual reduction of each steady solve */
    int krylov_max_iter; /* iterations per steady solve */
    int steady_solver;   /* 0: cl_lbm_solve_krylov_dsa; 1: cl_lbm_solve_steady_lines, which
                            also reaches the dissolved-O2 contrast of Eq. 10-15 (ionomer_o2) */
} cl_coupled_params;

typedef struct {
    int outer;                  /* Picard iterations taken */
    int converged;              /* 1 if max |phi_new - phi| fell below tol_phi */
    double dphi;                /* max |phi_new - phi| of the last iteration [V] */
    double current_o2_A;        /* 4 F times the O2 consumed per second [A] */
    double current_membrane_A;  /* proton current through the membrane face [A] */
    long long o2_iterations;    /* step applications of the O2 solves */
    long long proton_iterations;
} cl_coupled_info;

cl_status cl_coupled_solve(cl_handle o2, cl_handle pr, const cl_coupled_params* p, double* phi_out,
                           int phi_out_is_device, cl_coupled_info* info);

/* Current concentration C = sum_i g_i (nx*ny*nz floats, host or device; 0 on
   inactive cells). */
cl_status cl_lbm_get_field(cl_handle h, float* C, int ptr_is_device);

/* Current post-collision populations as f32, layout [q][nz][ny][nx] in the
   direction order above, host or device (decoded from FP16 storage if
   used; 0 on inactive cells). */
cl_status cl_lbm_get_populations(cl_handle h, float* g, int ptr_is_device);

/* Set-up products: active (nx*ny*nz bytes, 0/1), omega (nx*ny*nz floats,
   1/tau; 0 on inactive cells), chord (nx*ny*nz*13 int32: run length in cells
   of pore cells in each of the 13 directions of Sec. 2.1.3, 0 for non-pore
   cells), link mask (nx*ny*nz uint16: bits 0-5 face d closed, 6-11 face d
   reactive, 12 active).  Any pointer may be NULL; all are host or device. */
cl_status cl_lbm_get_setup(cl_handle h, uint8_t* active, float* omega, int32_t* chord,
                           uint16_t* link_mask, int ptr_is_device);

/* Link classes of the loaded structure (nx*ny*nz uint32 each, host or
   device; either may be NULL): wall[c] bit i-1 = the link of cell c toward
   x + c_i is a wall, reactive[c] bit i-1 = that wall link is a catalytic
   sink, for i = 1..q-1 of the handle's lattice (see "Link classes" above);
   0 on inactive cells. */
cl_status cl_lbm_get_links(cl_handle h, uint32_t* wall, uint32_t* reactive, int ptr_is_device);

cl_status cl_lbm_get_info(cl_handle h, cl_structure_info* info);

/* Step counter since the last init. */
cl_status cl_lbm_get_step(cl_handle h, long long* step);

const char* cl_status_str(cl_status s);

/* Text of the last error raised on the calling thread ("" if none). */
const char* cl_last_error_message(void);

/* ---------------------------------------------------------------------
 * Batches: many structures of uneven size advanced by one persistent launch.
 * The paper solves one structure at a time on MPI ranks (Sec. 5.1, 5.3);
 * a batch runs a set of such independent solves on one GPU.  Each member is
 * an ordinary handle with its structure loaded; all members share storage
 * mode (FP32 or FP16DEV, not FP32POP), check_every and step parity.  Batch
 * calls are ordered on member 0's stream; members must not be stepped on
 * their own while they belong to a batch that will step again.  The batch
 * does not own its members: destroy the batch before them.
 * --------------------------------------------------------------------- */
typedef struct cl_batch* cl_batch_handle;

/* Build the batch (work list, per-member TMA descriptors and arguments).
   z_chunk: planes per work item (0: 32).  Errors: CL_ERR_ARG, CL_ERR_STATE
   (member without structure or at another parity), CL_ERR_OOM, CL_ERR_CUDA. */
cl_status cl_batch_create(cl_batch_handle* out, const cl_handle* members, int n, int z_chunk);

/* Free the batch's own buffers (members are untouched; NULL is ignored). */
void cl_batch_destroy(cl_batch_handle b);

/* Advance every member by exactly nsteps steps in one cooperative launch
   (the same arithmetic as cl_lbm_step).  CL_ERR_TIMEOUT if a bounded wait
   for a member's previous step, or a member's own plane wait, gave up (the
   members' states are then partly stepped: re-initialise them).  A member's
   wait settings (cl_lbm_set_wait_test) reach the batch when it is created
   or configured. */
cl_status cl_batch_step(cl_batch_handle b, long long nsteps);

/* Advance all members, check_every steps per launch (a captured CUDA graph
   when the runtime captures cooperative launches), applying each member's
   own stopping rule (as cl_lbm_solve) after every interval; converged
   members leave the work list.  infos (nullable, n entries) receives each
   member's outcome, n_converged (nullable) the count.  Returns
   CL_ERR_NOT_CONVERGED if some member hit max_steps, CL_ERR_DIVERGED on a
   non-finite member. */
cl_status cl_batch_solve(cl_batch_handle b, long long max_steps, cl_solve_info* infos, int* n_converged);

/* Time steps_per_trial (even) steps for each tile shape in {1, 2, 4} rows
   per warp (one shape for every member; cl_lbm_set_tile_rows), z_chunk in
   {8, 16, 32, 64, 128} (up to the deepest member) and L2 prefetch distance in
   {0, 2}, keep the fastest and
   report it (ms per step in best_ms).  The trial steps are real steps of
   every member.  Any out pointer may be NULL. */
cl_status cl_batch_autotune(cl_batch_handle b, int steps_per_trial, int* z_chunk, int* prefetch, int* tile_rows,
                            double* best_ms);

/* Set the work-item z length (>= 8), prefetch distance and tile shape
   directly (e.g. from a cached autotuning result).  tile_rows: 1, 2 or 4
   rows per warp for every member, or 0 for each member's own shape (its
   handle's at batch creation).  A new batch starts with the single shape of
   least modelled cost over its members (idle lanes and rows against each
   shape's per-cell cost); members of different shapes in one launch run
   slower than any single shape.  Errors: CL_ERR_ARG. */
cl_status cl_batch_configure(cl_batch_handle b, int z_chunk, int prefetch, int tile_rows);

/* Test hook of the batch's bounded step-dependency waits (no counterpart in
   the paper).  wait_limit_clocks: SM clock cycles a block waits for a member's
   previous step to finish before it gives up (0: the default, about 2 s).
   never_arrive (needs a limit > 0): every such wait asks for one finished
   item more than the member has, so the first wait of a launch of two or more
   steps runs out; the launch then ends with every block returned and the
   step reports CL_ERR_TIMEOUT.  The members' states are then partly stepped:
   re-initialise them.  Set (0, 0) to restore normal stepping.
   Errors: CL_ERR_ARG. */
cl_status cl_batch_set_wait_test(cl_batch_handle b, long long wait_limit_clocks, int never_arrive);

/* Resident blocks of the persistent launch, current work items, and whether
   the solve runs from a captured graph (1) or plain launches (0). */
cl_status cl_batch_info(cl_batch_handle b, int* grid_blocks, int* n_items, int* uses_graph);

/* Cells of the transport phase 6-connected to the inlet plane x = 0 (y, z
   periodic), computed without allocating any device memory; for callers
   that cannot call cudaMalloc when they need it (a host application that
   owns all device allocations, or a pipeline that forbids allocation after
   start-up).  The paper has no counterpart: it is the same answer as the
   `active` output of cl_lbm_get_setup, obtained without a handle.
     phase:  nx*ny*nz phase codes, DEVICE pointer (read only).
     active: nx*ny*nz bytes, DEVICE pointer, written with 0/1.
     ionomer_transport: nonzero counts ionomer (2) as transport phase.
     cuda_stream: cudaStream_t or NULL; the call synchronises it.
   Limit: nx*ny*nz <= 4,194,304 cells (CL_ERR_ARG beyond).  Scratch space is
   a static device array of about 20 MiB that every GPU loading the library
   keeps until exit; all calls share it and it keeps the last call's
   contents, so calls whose work overlaps on the GPU (two streams, two host
   threads) race: serialise them.  Every call looks up the array's address on
   the current device (no allocation; a cached address would not survive a
   context reset).  The call copies an error word to the host and
   synchronises its stream before it returns, so it cannot be made inside a
   stream capture (CUDA graph).  Allocates nothing.
   Errors: CL_ERR_ARG (NULL pointer, size, a pointer that is not device or
   managed memory of the current device, phase code > 3), CL_ERR_CUDA,
   CL_ERR_TIMEOUT (labelling iteration bound). */
cl_status cl_active_mask_noalloc(const uint8_t* phase, int nx, int ny, int nz, int ionomer_transport,
                                 uint8_t* active, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Structure statistics: the connected-phase labelling of Sec. 2.1.3.
 * The cells whose phase code is in phase_set (bit k = code k, e.g. 0x2 for
 * C/Pt, 0x9 for the void phase of pores and micropores, 0x4 for ionomer)
 * are grouped into portions connected through the 26 neighbours of Fig. 4a
 * (neighbours = 26) or the 6 face neighbours (neighbours = 6); y and z wrap
 * when periodic_yz, x never does.  A portion with cells on both end planes
 * x = 0 and x = L is "transport", the others are "dead".
 * --------------------------------------------------------------------- */
typedef struct {
    long long n_cells;                 /* cells of the phase set */
    long long n_portions;              /* connected portions */
    long long n_transport_portions;    /* portions touching x = 0 and x = L */
    long long n_transport_cells;       /* cells of those portions */
    long long surface_faces;           /* faces between a set cell and an in-box cell of
                                          another phase (surface area in dx^2) */
    long long transport_surface_faces; /* of those, faces of transport cells */
    long long largest_portion;         /* cells of the largest portion */
} cl_phase_stats;

/* Label and count, on the GPU.  phase: nx*ny*nz codes 0..3 (host or
   device); labels (nullable, nx*ny*nz int32, same side as phase): the
   smallest cell index of the cell's portion, -1 outside the set; out: host.
   Allocates its scratch (about 12 B per cell) on the stream with
   cudaMallocAsync and frees it before returning; synchronises the stream.
   Errors: CL_ERR_ARG (NULL, sizes, neighbours not 6 or 26, empty or
   invalid phase_set, a phase code > 3), CL_ERR_OOM, CL_ERR_CUDA,
   CL_ERR_TIMEOUT (labelling iteration bound). */
cl_status cl_phase_connectivity(const uint8_t* phase, int nx, int ny, int nz, unsigned phase_set,
                                int neighbours, int periodic_yz, int32_t* labels, cl_phase_stats* out,
                                int ptr_is_device, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Structure generation on the GPU (input generation, Sec. 2.1.2 and 5.3),
 * bit-identical to the host generator shipped with the inputs module.
 * Random numbers: SplitMix64 folded over (seed, stream, a, b); a uniform
 * draw is the top 53 bits of the hash times 2^-53.  All arrays are device
 * arrays of nx*ny*nz cells; calls synchronise the stream.
 * --------------------------------------------------------------------- */

/* QSGS growth of phase `code` in place until `target` cells carry it
   (Sec. 2.1.2.1): seeds once with probability c_d on cells whose phase is
   in allowed_mask (and region[c] != 0 when region is given), then
   synchronous sweeps: an allowed cell with grown 6-neighbours (phases in
   grown_mask; x, y, z wrap) converts when it has two or more (rule 2a),
   else with probability p_alpha (rule 2b); the sweep that would overshoot
   converts only its candidates with the smallest (priority hash, cell
   index).  At most max_sweeps sweeps; *final_count (nullable) gets the
   resulting count.  Scratch: 12 B per cell, allocated on the stream.
   Errors: CL_ERR_ARG (NULL, sizes, code not in 0..3 or not in grown_mask),
   CL_ERR_OOM, CL_ERR_CUDA. */
cl_status cl_qsgs_grow(uint8_t* phase, int nx, int ny, int nz, int code, unsigned allowed_mask,
                       unsigned grown_mask, const uint8_t* region, long long target, double c_d,
                       double p_alpha, uint64_t seed, uint64_t stream, int max_sweeps,
                       long long* final_count, void* cuda_stream);

/* region[c] = 1 where phase[c] == code and no 6-neighbour (all axes wrap)
   has phase `avoid` (the solid that may hold micropores, Sec. 5.3). */
cl_status cl_qsgs_region_not_adjacent(const uint8_t* phase, int nx, int ny, int nz, int code, int avoid,
                                      uint8_t* region, void* cuda_stream);

/* out[c] bit d-1 (d = 1..6: +x, -x, +y, -y, +z, -z): cell c has phase
   from_code, its neighbour across face d (y, z wrap, x does not) has phase
   to_code, and the face is drawn with probability `fraction` (>= 1: all);
   *n_faces (nullable) = faces set. */
cl_status cl_qsgs_reactive_faces(const uint8_t* phase, int nx, int ny, int nz, int from_code, int to_code,
                                 double fraction, uint64_t seed, uint8_t* out, long long* n_faces,
                                 void* cuda_stream);

/* ---------------------------------------------------------------------
 * Property formulas of Sec. 3 (host arithmetic, SI units).
 * --------------------------------------------------------------------- */

/* Eq. 11: Henry's constant of O2 in the ionomer, H [Pa m^3 / mol]. */
double cl_henry_constant(double T_K);

/* Eq. 13: diffusivity of dissolved O2 in the ionomer, D_e [m^2/s]
   (positive above 283.7 K). */
double cl_ionomer_o2_diffusivity(double T_K);

/* Diffusivity that the ionomer carries in the gas-equivalent variable of
   Eq. 14-15: the dissolved concentration is C_e = C RT/H (Eq. 10), so the
   molar flux D_e grad C_e equals (D_e RT/H) grad C, and with this D the
   flux stays continuous across the pore-ionomer interface. [m^2/s] */
double cl_ionomer_effective_diffusivity(double T_K);

/* First-order surface rate constant k [m/s] of the gas-equivalent C for the
   uniform-potential Tafel rate (Eq. 17b with Eq. 10, four electrons per O2):
   the local current i = i0m (C RT/H / c_ref) exp(alpha F phi_e / (R T))
   consumes O2 at i / (4F) per unit reactive area, i.e. k C with
   k = i0m exp(alpha F phi_e / (R T)) (RT/H) / (4 F c_ref).
   i0m [A/m^2], phi_e [V], c_ref [mol/m^3] (Table 1 gives 0.01, 0.61, 0.6,
   333 K, 40.96). */
double cl_tafel_rate_constant(double i0m, double alpha, double phi_e, double T_K, double c_ref);

/* Library version string. */
const char* cl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CL_LBM_H */
