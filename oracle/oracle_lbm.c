/*
 * FP64 CPU oracle for the D3Q7 reactive-diffusion lattice Boltzmann method of
 * Chen et al., "Nanoscale study of reactive transport in catalyst layer of
 * PEM fuel cells with precious and non-precious catalysts using LBM"
 * (arXiv:1410.1914).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or helper with the CUDA library; neither includes the other.
 *
 * Everything is double precision.  No tiling, no packing, no fusion: every
 * step below follows the paper's order of operations.
 *
 *   Sec. 2.1.3      13-direction pore diameter (orc_chord_counts)
 *   Sec. 2.1.3      connected-phase labelling, adapted to a 6-connected
 *                   "reachable from the inlet plane" set (orc_active_mask)
 *   Eq. 7           bulk O2-N2 diffusivity (orc_bulk_diffusivity)
 *   Eq. 8           Knudsen diffusivity (orc_knudsen_diffusivity)
 *   Eq. 9           Bosanquet combination (orc_bosanquet)
 *   Eq. 21, 23, 24  BGK evolution, equilibrium, C = sum g, D <-> tau, on
 *                   either lattice: D3Q7 (w0 = 1/4, w1..6 = 1/8, cs^2 = 1/4)
 *                   or the paper's D3Q19 (Eq. 22, 23: a0 = 1/3, 1/18 on the
 *                   six axes, 1/36 on the twelve face diagonals, cs^2 = 1/3)
 *   Sec. 3.5.1      Dirichlet inlet/outlet in x, periodic y and z
 *   Sec. 3.5.2      zero-flux outlet (Eq. 20a), Dirichlet inlet (Eq. 20b)
 *   Eq. 17b + 18a   first-order kinetics with uniform ionomer potential,
 *                   placed as a surface (Robin) condition on catalyst faces
 *   Eq. 19          effective diffusivity from the outlet flux
 *   Eq. 16, Sec. 5.2  proton conduction (carrier 1): the same scheme on the
 *                   ionomer phase alone with a uniform conductivity, no
 *                   source; the Eq. 19 readout then is the effective
 *                   conductivity, normalised by the ionomer's own
 *
 * Lattice directions: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z; D3Q19 adds
 * 7 (+1,+1,0), 8 (-1,-1,0), 9 (+1,-1,0), 10 (-1,+1,0), 11 (+1,0,+1),
 * 12 (-1,0,-1), 13 (+1,0,-1), 14 (-1,0,+1), 15 (0,+1,+1), 16 (0,-1,-1),
 * 17 (0,+1,-1), 18 (0,-1,+1).
 * Phase codes: 0 pore, 1 solid (carbon / Pt / catalyst), 2 ionomer,
 *              3 micropore (transports like pore, never reactive).
 * Cell index: x + nx*(y + ny*z)  (x fastest).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 19

typedef struct {
    int q;
    int cx[QMAX], cy[QMAX], cz[QMAX], opp[QMAX];
    double w[QMAX];
    double cs2; /* sum_i w_i c_ia^2 */
} orc_lattice;

/* D3Q7: sum w = 1, sum w c_x^2 = 2/8 = 1/4 */
static const orc_lattice LAT7 = {
    7,
    {0, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0},
    {0, 0, 0, 0, 0, 1, -1},
    {0, 2, 1, 4, 3, 6, 5},
    {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125},
    0.25};

/* D3Q19 (Eq. 22, 23): sum a = 1/3 + 6/18 + 12/36 = 1,
   sum a c_x^2 = 2/18 + 8/36 = 1/3 */
static const orc_lattice LAT19 = {
    19,
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
    {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17},
    {1.0 / 3, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
     1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
     1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36},
    1.0 / 3};

/* the six faces of a voxel, in the order of directions 1..6 above */
static const int FX[6] = {1, -1, 0, 0, 0, 0};
static const int FY[6] = {0, 0, 1, -1, 0, 0};
static const int FZ[6] = {0, 0, 0, 0, 1, -1};

typedef struct {
    int nx, ny, nz;
    double dx_m;        /* voxel edge [m] */
    double T_K;         /* temperature [K] */
    double p_atm;       /* pressure [atm] */
    double M_kgmol;     /* molar mass of O2 [kg/mol] */
    double D_bulk;      /* <= 0: Eq. 7 */
    double D_ionomer;   /* > 0: ionomer transports O2 with this D; 0: impermeable */
    double k_ms;        /* first-order surface rate constant [m/s] */
    int knudsen;        /* 1: Eq. 8-9 in pore cells; 0: D = D_b */
    int bc_in, bc_out;  /* 0 Dirichlet, 1 zero flux */
    double c_in, c_out; /* boundary concentrations */
    double tau_ref;     /* relaxation time of the most diffusive active cell */
    int carrier;        /* 0: O2 in the pore space (Eq. 6); 1: protons in the ionomer
                           (Eq. 16 with S_e = 0 and uniform conductivity D_ionomer) */
    int lattice;        /* 0: D3Q7; 1: D3Q19 (Eq. 22) */
    int ionomer_o2;     /* 1: the ionomer carries the gas-equivalent C of Eq. 14-15 with
                           D = D_e(T) RT / H (Eq. 10, 11, 13), replacing D_ionomer */
} orc_params;

static long idx3(int x, int y, int z, int nx, int ny) { return x + (long)nx * (y + (long)ny * z); }
static int wrap(int a, int n) { return ((a % n) + n) % n; }

/* ----------------------------------------------------------------------
 * Eq. 1-5 (Sec. 2.1.1): volume fractions and Pt loading.
 * out[0] = eps_N, out[1] = eps_C, out[2] = eps_Pt.
 * ---------------------------------------------------------------------- */
void orc_volume_fractions(double eps, double beta_N, double theta_Pt, double rho_N,
                          double rho_C, double rho_Pt, double out[3])
{
    double nafion_term = (1.0 + theta_Pt) * beta_N / (rho_N * (1.0 - beta_N));
    double denom = theta_Pt / rho_Pt + 1.0 / rho_C + nafion_term;
    out[0] = (1.0 - eps) * nafion_term / denom;       /* Eq. 4a */
    out[1] = (1.0 - eps) * (1.0 / rho_C) / denom;     /* Eq. 4b */
    out[2] = (1.0 - eps) * (theta_Pt / rho_Pt) / denom; /* Eq. 4c */
}

/* Eq. 5: gamma_Pt = eps_Pt * rho_Pt * l.  rho in mg/cm^3, l in cm -> mg/cm^2. */
double orc_pt_loading(double eps_Pt, double rho_Pt_mg_cm3, double l_cm)
{
    return eps_Pt * rho_Pt_mg_cm3 * l_cm;
}

/* Eq. 7: D_b = 0.22e-4 (T/293.2)^1.5 / (p / 1 atm)   [m^2/s] */
double orc_bulk_diffusivity(double T_K, double p_atm)
{
    return 0.22e-4 * pow(T_K / 293.2, 1.5) / p_atm;
}

/* Eq. 8: D_Kn = (d_p / 3) sqrt(8 R T / (pi M))   [m^2/s], SI units */
double orc_knudsen_diffusivity(double d_p_m, double T_K, double M_kgmol)
{
    const double R = 8.314462618;
    return d_p_m / 3.0 * sqrt(8.0 * R * T_K / (M_PI * M_kgmol));
}

/* Eq. 11: H = 0.101325 exp(-666/T + 14.1)   [Pa m^3/mol] */
double orc_henry_constant(double T_K)
{
    return 1.01325e-1 * exp(-666.0 / T_K + 14.1);
}

/* Eq. 13: D_e = 1e-10 (0.1543 (T - 273) - 1.65)   [m^2/s] */
double orc_ionomer_o2_diffusivity(double T_K)
{
    return 1e-10 * (0.1543 * (T_K - 273.0) - 1.65);
}

/* Eq. 9: 1/D = 1/D_Kn + 1/D_b */
double orc_bosanquet(double D_kn, double D_b)
{
    return 1.0 / (1.0 / D_kn + 1.0 / D_b);
}

/* ----------------------------------------------------------------------
 * Sec. 2.1.3: 13-direction pore length.
 * For every pore cell (phase 0 or 3) and each of the 13 directions, the
 * length of the line of pore cells through it: walk +e and -e while the
 * next cell is pore, y and z periodic, x bounded by the box.  A line with
 * no x component is a closed loop of period P (the lattice period of that
 * direction in y-z); its run is capped at P cells so that an all-pore loop
 * has length P.  counts[c*13 + d] = number of cells on the run (>= 1);
 * 0 for non-pore cells.  The length is counts * |e_d| * dx.
 * Direction order: 3 axes, 6 face diagonals, 4 body diagonals.
 * ---------------------------------------------------------------------- */
static const int DIR13[13][3] = {
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
    {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1},
    {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};

static long gcd_l(long a, long b) { while (b) { long t = a % b; a = b; b = t; } return a; }

static int is_pore_phase(uint8_t p) { return p == 0 || p == 3; }

void orc_chord_counts(const uint8_t* phase, int nx, int ny, int nz, int32_t* counts)
{
    long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = idx3(x, y, z, nx, ny);
                for (int d = 0; d < 13; ++d) {
                    if (!is_pore_phase(phase[c])) { counts[c * 13 + d] = 0; continue; }
                    int ex = DIR13[d][0], ey = DIR13[d][1], ez = DIR13[d][2];
                    long period = -1; /* only lines without an x component close on themselves */
                    if (ex == 0) {
                        long py = ey ? ny : 1, pz = ez ? nz : 1;
                        period = py / gcd_l(py, pz) * pz;
                    }
                    long run = 1;
                    for (int sgn = 1; sgn >= -1; sgn -= 2) {
                        int px = x, py = y, pz = z;
                        for (;;) {
                            if (period > 0 && run >= period) break;
                            int qx = px + sgn * ex;
                            if (qx < 0 || qx >= nx) break;
                            int qy = wrap(py + sgn * ey, ny), qz = wrap(pz + sgn * ez, nz);
                            if (!is_pore_phase(phase[idx3(qx, qy, qz, nx, ny)])) break;
                            px = qx; py = qy; pz = qz;
                            ++run;
                        }
                    }
                    counts[c * 13 + d] = (int32_t)run;
                }
            }
    (void)N;
}

/* d_p = mean over the 13 directions of counts * |e_d| * dx */
void orc_pore_diameter(const int32_t* counts, long N, double dx_m, double* d_p)
{
    for (long c = 0; c < N; ++c) {
        double s = 0.0;
        for (int d = 0; d < 13; ++d) {
            double len = sqrt((double)(DIR13[d][0] * DIR13[d][0] + DIR13[d][1] * DIR13[d][1] +
                                       DIR13[d][2] * DIR13[d][2]));
            s += counts[c * 13 + d] * len * dx_m;
        }
        d_p[c] = s / 13.0;
    }
}

/* ----------------------------------------------------------------------
 * Transport set and the cells reachable from the inlet plane x = 0
 * (6-connected, y and z periodic): the D3Q7 adaptation of the
 * connected-phase labelling of Sec. 2.1.3.  Plain breadth-first search.
 * Returns the number of active cells.
 * ---------------------------------------------------------------------- */
/* Phases that carry the transported quantity.  mode 0: pore and micropore
 * (O2, Eq. 6); 1: pore, micropore and ionomer (O2 dissolved in ionomer with
 * its own D, Eq. 15); 2: ionomer only (protons, Eq. 16). */
static int is_transport(uint8_t p, int mode)
{
    if (mode == 2) return p == 2;
    return p == 0 || p == 3 || (p == 2 && mode == 1);
}

/* Transport cells 6-connected to the inlet plane x = 0 (y, z periodic),
 * by breadth-first search; `mode` selects the transport phases as in
 * is_transport.  Returns the number of active cells. */
long orc_active_mask(const uint8_t* phase, int nx, int ny, int nz, int mode, uint8_t* active)
{
    long N = (long)nx * ny * nz;
    long* queue = (long*)malloc(sizeof(long) * (N > 0 ? N : 1));
    long head = 0, tail = 0;
    memset(active, 0, (size_t)N);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            long c = idx3(0, y, z, nx, ny);
            if (is_transport(phase[c], mode)) { active[c] = 1; queue[tail++] = c; }
        }
    while (head < tail) {
        long c = queue[head++];
        int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
        for (int d = 0; d < 6; ++d) {
            int qx = x + FX[d];
            if (qx < 0 || qx >= nx) continue;
            long n = idx3(qx, wrap(y + FY[d], ny), wrap(z + FZ[d], nz), nx, ny);
            if (!active[n] && is_transport(phase[n], mode)) {
                active[n] = 1;
                queue[tail++] = n;
            }
        }
    }
    free(queue);
    return tail;
}

/* ----------------------------------------------------------------------
 * Sec. 2.1.3 connected-phase labelling and its statistics.  The cells whose
 * phase code is in `set_mask` (bit k = code k) are grouped into portions:
 * maximal sets connected through the 26 neighbours of Fig. 4a (or the 6
 * face neighbours); y and z wrap when periodic_yz, x never does.  A portion
 * is "transport" when it has cells on both end planes x = 0 and x = nx - 1,
 * "dead" otherwise.  Plain breadth-first search in scan order, so each
 * portion's label is the smallest cell index in it (-1 outside the set).
 * out[0] cells in the set, [1] portions, [2] transport portions,
 * [3] transport cells, [4] faces between a set cell and an in-box cell of
 * another phase (the surface area in dx^2), [5] those faces of transport
 * cells, [6] cells of the largest portion.
 * ---------------------------------------------------------------------- */
void orc_phase_connectivity(const uint8_t* phase, int nx, int ny, int nz, unsigned set_mask, int neighbours,
                            int periodic_yz, int32_t* labels, long long out[7])
{
    long N = (long)nx * ny * nz;
    int off[26][3], noff = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int m = abs(dx) + abs(dy) + abs(dz);
                if (m == 0 || (neighbours == 6 && m != 1)) continue;
                off[noff][0] = dx; off[noff][1] = dy; off[noff][2] = dz; ++noff;
            }
    long* queue = (long*)malloc(sizeof(long) * (N > 0 ? N : 1));
    unsigned char* ends = (unsigned char*)calloc((size_t)(N > 0 ? N : 1), 1);
    long* size = (long*)calloc((size_t)(N > 0 ? N : 1), sizeof(long));
    for (long c = 0; c < N; ++c) labels[c] = -1;
    for (int k = 0; k < 7; ++k) out[k] = 0;
    for (long s = 0; s < N; ++s) {
        if (labels[s] >= 0 || !(set_mask >> phase[s] & 1u)) continue;
        long head = 0, tail = 0;
        labels[s] = (int32_t)s;
        queue[tail++] = s;
        while (head < tail) {
            long c = queue[head++];
            int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
            if (x == 0) ends[s] |= 1;
            if (x == nx - 1) ends[s] |= 2;
            for (int k = 0; k < noff; ++k) {
                int qx = x + off[k][0], qy = y + off[k][1], qz = z + off[k][2];
                if (qx < 0 || qx >= nx) continue;
                if (periodic_yz) { qy = wrap(qy, ny); qz = wrap(qz, nz); }
                else if (qy < 0 || qy >= ny || qz < 0 || qz >= nz) continue;
                long n = idx3(qx, qy, qz, nx, ny);
                if (labels[n] < 0 && (set_mask >> phase[n] & 1u)) { labels[n] = (int32_t)s; queue[tail++] = n; }
            }
        }
        size[s] = tail;
        out[1] += 1;
        if (ends[s] == 3) { out[2] += 1; out[3] += tail; }
        if (tail > out[6]) out[6] = tail;
        out[0] += tail;
    }
    for (long c = 0; c < N; ++c) {
        if (labels[c] < 0) continue;
        int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
        for (int f = 0; f < 6; ++f) {
            int qx = x + FX[f], qy = y + FY[f], qz = z + FZ[f];
            if (qx < 0 || qx >= nx) continue;
            if (periodic_yz) { qy = wrap(qy, ny); qz = wrap(qz, nz); }
            else if (qy < 0 || qy >= ny || qz < 0 || qz >= nz) continue;
            if (set_mask >> phase[idx3(qx, qy, qz, nx, ny)] & 1u) continue;
            out[4] += 1;
            if (ends[labels[c]] == 3) out[5] += 1;
        }
    }
    free(queue); free(ends); free(size);
}

/* ----------------------------------------------------------------------
 * Per-cell diffusivity [m^2/s] of active cells (0 elsewhere):
 *   pore / micropore: Eq. 9 of Eq. 8 (d_p from the 13-direction lengths) and
 *                     D_b (Eq. 7 unless given); D_b alone without Knudsen;
 *   ionomer:          D_ionomer.
 * Returns D_b.
 * ---------------------------------------------------------------------- */
double orc_cell_diffusivity(const orc_params* p, const uint8_t* phase, const uint8_t* active,
                            const double* d_p, double* D)
{
    long N = (long)p->nx * p->ny * p->nz;
    double D_b = p->D_bulk > 0 ? p->D_bulk : orc_bulk_diffusivity(p->T_K, p->p_atm);
    for (long c = 0; c < N; ++c) {
        D[c] = 0.0;
        if (!active[c]) continue;
        if (phase[c] == 2) { D[c] = p->D_ionomer; continue; }
        if (p->knudsen) D[c] = orc_bosanquet(orc_knudsen_diffusivity(d_p[c], p->T_K, p->M_kgmol), D_b);
        else D[c] = D_b;
    }
    return D_b;
}

/* ----------------------------------------------------------------------
 * LBM state.  g holds the pre-collision populations g_i(x, t) of Eq. 21,
 * array of q planes of N doubles.  Inactive cells hold 0 and are never
 * touched.
 * ---------------------------------------------------------------------- */
typedef struct {
    orc_params p;
    const orc_lattice* L;
    long N;
    uint8_t* phase;
    uint8_t* active;
    uint32_t* react;   /* bit (i-1) = link toward x + c_i ends on a catalytic face */
    double* D;         /* m^2/s, 0 for inactive */
    double* tau;       /* per-cell relaxation time, Eq. 24 with the lattice's cs^2 */
    double* g;         /* current pre-collision populations */
    double* gn;        /* scratch for the next step */
    double* kscale;    /* per-cell factor on k (non-uniform potential, Eq. 17b); NULL: 1 */
    double* src;       /* per-cell amount added per step (the source of Eq. 16); NULL: none */
    double D_b, D_max, dt, k_lu;
    long step;
} orc_lbm;

/*
 * End cell of the link of cell c toward x + c_i.  *outside = -1 / +1 when the
 * link leaves the box through x = 0 / x = L.  Beyond those faces the box
 * continues as the mirror image of its first / last plane, so the end cell
 * of a leaving link is then (x, y + c_iy, z + c_iz): the cell itself for the
 * axis link, an in-plane neighbour for a D3Q19 diagonal.  A leaving link
 * whose end cell is active is a boundary link (Dirichlet or zero flux);
 * one whose end cell is not is a wall like any other, so that a wall that
 * meets the inlet or outlet face stays a wall up to the face.
 */
static long orc_neighbor(const orc_lbm* s, long c, int i, int* outside)
{
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    const orc_lattice* L = s->L;
    int qx = x + L->cx[i];
    *outside = (qx < 0) ? -1 : (qx >= nx ? 1 : 0);
    if (*outside) qx = x;
    return idx3(qx, wrap(y + L->cy[i], ny), wrap(z + L->cz[i], nz), nx, ny);
}

/* Face f (0..5, directions 1..6) of cell c is catalytic: marked in the input
 * and its neighbour across the face is solid (code 1). */
static int face_catalytic(const orc_lbm* s, const uint8_t* react_in, long c, int f)
{
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    int qx = x + FX[f];
    if (qx < 0 || qx >= nx || !(react_in[c] >> f & 1)) return 0;
    return s->phase[idx3(qx, wrap(y + FY[f], ny), wrap(z + FZ[f], nz), nx, ny)] == 1;
}

/*
 * Build the solver state.  phase: N codes.  react: N bytes of reactive-face
 * bits or NULL (no reaction).  D_override: N diffusivities [m^2/s] for the
 * transport cells (used instead of Eq. 7-9) or NULL.
 * Returns NULL if no transport cell touches the inlet plane.
 */
orc_lbm* orc_lbm_new(const orc_params* p, const uint8_t* phase, const uint8_t* react,
                     const double* D_override)
{
    orc_lbm* s = (orc_lbm*)calloc(1, sizeof(orc_lbm));
    s->p = *p;
    s->N = (long)p->nx * p->ny * p->nz;
    long N = s->N;
    s->phase = (uint8_t*)malloc((size_t)N);
    memcpy(s->phase, phase, (size_t)N);
    s->active = (uint8_t*)malloc((size_t)N);
    s->L = p->lattice == 1 ? &LAT19 : &LAT7;
    if (p->ionomer_o2) {
        /* Eq. 10: the dissolved concentration is C_e = C RT/H, so the molar
           flux in the ionomer, D_e grad C_e, is (D_e RT/H) grad C: the
           gas-equivalent C of Eq. 14-15 diffuses there with D_e RT/H */
        const double R = 8.314462618;
        s->p.D_ionomer = orc_ionomer_o2_diffusivity(p->T_K) * R * p->T_K / orc_henry_constant(p->T_K);
        p = &s->p;
    }
    s->react = (uint32_t*)calloc((size_t)N, sizeof(uint32_t));
    s->D = (double*)calloc((size_t)N, sizeof(double));
    s->tau = (double*)calloc((size_t)N, sizeof(double));
    s->g = (double*)calloc((size_t)N * s->L->q, sizeof(double));
    s->gn = (double*)calloc((size_t)N * s->L->q, sizeof(double));

    long n_active = orc_active_mask(phase, p->nx, p->ny, p->nz, p->carrier == 1 ? 2 : (p->D_ionomer > 0),
                                    s->active);
    if (n_active == 0) { /* nothing percolates */
        free(s->phase); free(s->active); free(s->react); free(s->D); free(s->tau);
        free(s->g); free(s->gn); free(s->kscale); free(s->src); free(s);
        return NULL;
    }
    if (D_override) {
        s->D_b = p->D_bulk > 0 ? p->D_bulk : orc_bulk_diffusivity(p->T_K, p->p_atm);
        for (long c = 0; c < N; ++c) s->D[c] = s->active[c] ? D_override[c] : 0.0;
    } else {
        int32_t* counts = (int32_t*)malloc(sizeof(int32_t) * 13 * N);
        double* d_p = (double*)malloc(sizeof(double) * N);
        orc_chord_counts(phase, p->nx, p->ny, p->nz, counts);
        orc_pore_diameter(counts, N, p->dx_m, d_p);
        s->D_b = orc_cell_diffusivity(p, phase, s->active, d_p, s->D);
        free(counts);
        free(d_p);
    }
    /* Reactive links.  A link of active cell c toward x + c_i reacts when its
     * end cell is solid (code 1) and it leaves c through a catalytic face:
     * one of the faces that c_i crosses (the axis faces of its non-zero
     * components) is marked in the input and borders solid.  On D3Q7 each
     * link crosses exactly its own face.  On D3Q19 a flat catalytic face is
     * crossed by its axis link and four diagonals; a diagonal that only
     * touches a solid edge between two open faces stays a plain wall. */
    if (react) {
        const orc_lattice* L = s->L;
        for (long c = 0; c < N; ++c) {
            if (!s->active[c]) continue;
            for (int i = 1; i < L->q; ++i) {
                int out;
                long n = orc_neighbor(s, c, i, &out);
                if (phase[n] != 1) continue;
                int hit = 0;
                if (L->cx[i]) hit |= face_catalytic(s, react, c, L->cx[i] > 0 ? 0 : 1);
                if (L->cy[i]) hit |= face_catalytic(s, react, c, L->cy[i] > 0 ? 2 : 3);
                if (L->cz[i]) hit |= face_catalytic(s, react, c, L->cz[i] > 0 ? 4 : 5);
                if (hit) s->react[c] |= 1u << (i - 1);
            }
        }
    }
    /* Eq. 24: D = cs^2 (tau - 1/2) dx^2 / dt.  The most diffusive active cell
       gets tau_ref; that fixes dt. */
    const double cs2 = s->L->cs2;
    s->D_max = 0.0;
    for (long c = 0; c < N; ++c) if (s->active[c] && s->D[c] > s->D_max) s->D_max = s->D[c];
    s->dt = (p->tau_ref - 0.5) * cs2 * p->dx_m * p->dx_m / s->D_max;
    for (long c = 0; c < N; ++c)
        s->tau[c] = s->active[c] ? 0.5 + s->D[c] * s->dt / (cs2 * p->dx_m * p->dx_m) : 0.0;
    s->k_lu = p->k_ms * s->dt / p->dx_m;
    return s;
}

void orc_lbm_free(orc_lbm* s)
{
    if (!s) return;
    free(s->phase); free(s->active); free(s->react); free(s->D); free(s->tau);
    free(s->g); free(s->gn); free(s->kscale); free(s->src); free(s);
}

/* g_i = w_i C  (Eq. 23 equilibrium) for a given field C (active cells only) */
void orc_lbm_init_field(orc_lbm* s, const double* C)
{
    for (long c = 0; c < s->N; ++c)
        for (int i = 0; i < s->L->q; ++i) s->g[i * s->N + c] = s->active[c] ? s->L->w[i] * C[c] : 0.0;
    s->step = 0;
}

/* linear ramp between the boundary values at the half-way faces x = 0, L */
void orc_lbm_init_linear(orc_lbm* s)
{
    double* C = (double*)malloc(sizeof(double) * s->N);
    int nx = s->p.nx;
    for (long c = 0; c < s->N; ++c) {
        int x = (int)(c % nx);
        C[c] = s->p.c_in + (s->p.c_out - s->p.c_in) * (x + 0.5) / nx;
    }
    orc_lbm_init_field(s, C);
    free(C);
}

/* post-collision populations of Eq. 21: g* = g - (g - g_eq) / tau, plus
 * w_i S of a per-cell source S (the a_i S term of Eq. 21) where one is set */
static void collide_cell(const orc_lbm* s, long c, double gs[QMAX])
{
    double C = 0.0;
    for (int i = 0; i < s->L->q; ++i) C += s->g[i * s->N + c];
    const double S = s->src ? s->src[c] : 0.0;
    for (int i = 0; i < s->L->q; ++i) {
        double gi = s->g[i * s->N + c];
        gs[i] = gi - (gi - s->L->w[i] * C) / s->tau[c] + s->L->w[i] * S;
    }
}

/*
 * Half-way first-order sink: a population g* that meets a catalytic face
 * returns as r g*.  The wall value is the mean of the pair,
 * C_w = (g* + r g*) / (2 w_i), and the amount the link delivers, (1 - r) g*,
 * is its share of the face's rate k C_w.  The share is w_i over the weight
 * sum of the links that cross one face (cs^2 / 2 on both lattices: 1/8 on
 * D3Q7, 1/18 + 4/36 on D3Q19), so (1 - r) = k (1 + r) / cs^2 and
 * r = (cs^2 - k) / (cs^2 + k) for every link; on D3Q7 that is
 * (2w - k) / (2w + k).
 */
static double reactive_factor(const orc_lbm* s, long c)
{
    const double k = s->k_lu * (s->kscale ? s->kscale[c] : 1.0);
    return (s->L->cs2 - k) / (s->L->cs2 + k);
}

/*
 * One time step in the order of Eq. 21: collide every active cell, then
 * stream each post-collision population to x + c_i.  Where the link leaves
 * the transport set, the population returns along the opposite direction:
 *   boundary link (leaves through x = 0 or x = L, end cell active, see
 *   orc_neighbor):        anti-bounce-back -g* + 2 w_i C_bc (Dirichlet),
 *                         bounce-back (zero flux);
 *   wall link (end cell solid or inactive): bounce-back, times the reactive
 *                         factor r if the link is reactive (half-way
 *                         first-order sink).
 */
void orc_lbm_step(orc_lbm* s, long nsteps)
{
    long N = s->N;
    for (long t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (long c = 0; c < N; ++c) {
            if (!s->active[c]) continue;
            const orc_lattice* L = s->L;
            double gs[QMAX];
            collide_cell(s, c, gs);
            s->gn[c] = gs[0];
            for (int i = 1; i < L->q; ++i) {
                int out;
                long n = orc_neighbor(s, c, i, &out);
                if (out && s->active[n]) {
                    int bc = out < 0 ? s->p.bc_in : s->p.bc_out;
                    double cb = out < 0 ? s->p.c_in : s->p.c_out;
                    s->gn[L->opp[i] * N + c] = bc == 0 ? -gs[i] + 2.0 * L->w[i] * cb : gs[i];
                } else if (!s->active[n]) {
                    double r = (s->react[c] >> (i - 1) & 1) ? reactive_factor(s, c) : 1.0;
                    s->gn[L->opp[i] * N + c] = r * gs[i];
                } else {
                    s->gn[i * N + n] = gs[i];
                }
            }
        }
        double* tmp = s->g; s->g = s->gn; s->gn = tmp;
        s->step++;
    }
}

void orc_lbm_concentration(const orc_lbm* s, double* C)
{
    for (long c = 0; c < s->N; ++c) {
        double sum = 0.0;
        if (s->active[c])
            for (int i = 0; i < s->L->q; ++i) sum += s->g[i * s->N + c];
        C[c] = sum;
    }
}

/* copy of the pre-collision populations, layout [q][N] */
void orc_lbm_populations(const orc_lbm* s, double* out)
{
    memcpy(out, s->g, sizeof(double) * s->L->q * s->N);
}

/* per-cell factor on the rate constant k (NULL: uniform k); copied */
void orc_lbm_set_kscale(orc_lbm* s, const double* k)
{
    free(s->kscale);
    s->kscale = NULL;
    if (!k) return;
    s->kscale = (double*)malloc(sizeof(double) * s->N);
    memcpy(s->kscale, k, sizeof(double) * s->N);
}

/* per-cell amount added to C per step, lattice units (NULL: none); copied.
 * It enters as w_i S on the post-collision populations (Eq. 21). */
void orc_lbm_set_source(orc_lbm* s, const double* S)
{
    free(s->src);
    s->src = NULL;
    if (!S) return;
    s->src = (double*)malloc(sizeof(double) * s->N);
    for (long c = 0; c < s->N; ++c) s->src[c] = s->active[c] ? S[c] : 0.0;
}

/* amount consumed per step on the reactive links of each cell, lattice units */
void orc_lbm_cell_reaction(const orc_lbm* s, double* out)
{
    for (long c = 0; c < s->N; ++c) {
        out[c] = 0.0;
        if (!s->active[c] || !s->react[c]) continue;
        double gs[QMAX];
        collide_cell(s, c, gs);
        for (int i = 1; i < s->L->q; ++i) {
            int o;
            long n = orc_neighbor(s, c, i, &o);
            if (!s->active[n] && (s->react[c] >> (i - 1) & 1)) out[c] += (1.0 - reactive_factor(s, c)) * gs[i];
        }
    }
}

/* replace the pre-collision populations (layout [q][N]); inactive cells stay 0 */
void orc_lbm_set_populations(orc_lbm* s, const double* g)
{
    for (int i = 0; i < s->L->q; ++i)
        for (long c = 0; c < s->N; ++c) s->g[i * s->N + c] = s->active[c] ? g[i * s->N + c] : 0.0;
}

/*
 * Lattice-unit fluxes of the current state (computed from its post-collision
 * populations, i.e. what the next streaming moves):
 *   out[0] J_in  : net amount entering through the x = 0 face,
 *   out[1] J_out : net amount leaving through the x = L face,
 *   out[2] R     : amount consumed on reactive faces,
 *   out[3] sum C over active cells,
 *   out[4] number of active cells.
 * Per step: sum C(t+1) - sum C(t) = J_in - J_out - R (+ the sum of the
 * per-cell sources, where set).
 */
void orc_lbm_fluxes(const orc_lbm* s, double out[5])
{
    double jin = 0, jout = 0, R = 0, sc = 0, na = 0;
    for (long c = 0; c < s->N; ++c) {
        if (!s->active[c]) continue;
        const orc_lattice* L = s->L;
        double gs[QMAX];
        collide_cell(s, c, gs);
        double C = 0.0;
        for (int i = 0; i < L->q; ++i) C += s->g[i * s->N + c];
        sc += C;
        na += 1;
        for (int i = 1; i < L->q; ++i) {
            int o;
            long n = orc_neighbor(s, c, i, &o);
            if (o < 0 && s->active[n] && s->p.bc_in == 0) jin += 2.0 * L->w[i] * s->p.c_in - 2.0 * gs[i];
            if (o > 0 && s->active[n] && s->p.bc_out == 0) jout += 2.0 * gs[i] - 2.0 * L->w[i] * s->p.c_out;
            if (!s->active[n] && (s->react[c] >> (i - 1) & 1))
                R += (1.0 - reactive_factor(s, c)) * gs[i];
        }
    }
    out[0] = jin; out[1] = jout; out[2] = R; out[3] = sc; out[4] = na;
}

/*
 * Eq. 19: D_eff = (mean outlet flux density) / ((C_in - C_out) / L_x), with
 * the Dirichlet faces half-way outside the first and last cells (L_x = nx dx).
 * out[0] D_eff [m^2/s], out[1] D_eff / D_b, out[2] D_eff in lattice units.
 */
void orc_lbm_effective_diffusivity(const orc_lbm* s, double out[3])
{
    double f[5];
    orc_lbm_fluxes(s, f);
    double jd = f[1] / ((double)s->p.ny * s->p.nz); /* per unit face area, lattice units */
    double dlu = jd * s->p.nx / (s->p.c_in - s->p.c_out);
    out[2] = dlu;
    out[0] = dlu * s->p.dx_m * s->p.dx_m / s->dt;
    /* normalised by the bulk D of O2, or by the ionomer's own conductivity
     * for protons (the effective conductivity of Sec. 5.2) */
    out[1] = out[0] / (s->p.carrier == 1 ? s->p.D_ionomer : s->D_b);
}

/*
 * Total reaction rate [C-units * m^3 / s; mol/s for C in mol/m^3]:
 * sum over reactive links of the consumed amount per step, times dx^3 / dt,
 * which equals sum k C_wall dx^2 (Eq. 25, left side, per 4F).
 * profile_R (nullable, nx): the same per x-plane.  profile_C (nullable, nx):
 * plane mean of C over active cells (0 where a plane has none).
 */
double orc_lbm_reaction_rate(const orc_lbm* s, double* profile_R, double* profile_C)
{
    int nx = s->p.nx;
    double scale = s->p.dx_m * s->p.dx_m * s->p.dx_m / s->dt;
    double total = 0.0;
    double* cnt = (double*)calloc((size_t)nx, sizeof(double));
    if (profile_R) memset(profile_R, 0, sizeof(double) * nx);
    if (profile_C) memset(profile_C, 0, sizeof(double) * nx);
    for (long c = 0; c < s->N; ++c) {
        if (!s->active[c]) continue;
        int x = (int)(c % nx);
        double gs[QMAX];
        collide_cell(s, c, gs);
        double C = 0.0;
        for (int i = 0; i < s->L->q; ++i) C += s->g[i * s->N + c];
        if (profile_C) { profile_C[x] += C; cnt[x] += 1; }
        for (int i = 1; i < s->L->q; ++i) {
            int o;
            long n = orc_neighbor(s, c, i, &o);
            if (!s->active[n] && (s->react[c] >> (i - 1) & 1)) {
                double r = (1.0 - reactive_factor(s, c)) * gs[i] * scale;
                total += r;
                if (profile_R) profile_R[x] += r;
            }
        }
    }
    if (profile_C)
        for (int x = 0; x < nx; ++x) profile_C[x] = cnt[x] > 0 ? profile_C[x] / cnt[x] : 0.0;
    free(cnt);
    return total;
}

/*
 * Eq. 25: the discharge current density carried by the reaction,
 * i_d = (integral of the local current over the reactive surface) / A_cross
 *     = 4 F R / A_cross, four electrons per O2 and A_cross = ny nz dx^2 [A/m^2].
 */
double orc_lbm_current_density(const orc_lbm* s)
{
    const double F = 96485.33212;
    double R = orc_lbm_reaction_rate(s, NULL, NULL);
    return 4.0 * F * R / ((double)s->p.ny * s->p.nz * s->p.dx_m * s->p.dx_m);
}

/*
 * Run until the relative change r = sum|C(t) - C(t-K)| / sum|C(t)| over one
 * check interval K drops below tol, or max_steps.  Returns the steps taken
 * (negative if max_steps was reached first).
 */
long orc_lbm_solve(orc_lbm* s, double tol, long check_every, long max_steps)
{
    double* Cp = (double*)malloc(sizeof(double) * s->N);
    double* Cn = (double*)malloc(sizeof(double) * s->N);
    orc_lbm_concentration(s, Cp);
    long taken = 0;
    int done = 0;
    while (taken < max_steps) {
        orc_lbm_step(s, check_every);
        taken += check_every;
        orc_lbm_concentration(s, Cn);
        double num = 0, den = 0;
        for (long c = 0; c < s->N; ++c) { num += fabs(Cn[c] - Cp[c]); den += fabs(Cn[c]); }
        double* t = Cp; Cp = Cn; Cn = t;
        if (den > 0 && num / den < tol) { done = 1; break; }
    }
    free(Cp); free(Cn);
    return done ? taken : -taken;
}

/* accessors for the Python wrapper */
long orc_lbm_n(const orc_lbm* s) { return s->N; }
long orc_lbm_step_count(const orc_lbm* s) { return s->step; }
double orc_lbm_dt(const orc_lbm* s) { return s->dt; }
double orc_lbm_D_b(const orc_lbm* s) { return s->D_b; }
double orc_lbm_D_max(const orc_lbm* s) { return s->D_max; }
double orc_lbm_k_lu(const orc_lbm* s) { return s->k_lu; }
void orc_lbm_get_tau(const orc_lbm* s, double* out) { memcpy(out, s->tau, sizeof(double) * s->N); }
void orc_lbm_get_D(const orc_lbm* s, double* out) { memcpy(out, s->D, sizeof(double) * s->N); }
void orc_lbm_get_active(const orc_lbm* s, uint8_t* out) { memcpy(out, s->active, (size_t)s->N); }
void orc_lbm_get_react(const orc_lbm* s, uint32_t* out) { memcpy(out, s->react, sizeof(uint32_t) * s->N); }
int orc_lbm_q(const orc_lbm* s) { return s->L->q; }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the later parallel loops of the calling thread (timing on one
   core); returns the new count */
int orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
