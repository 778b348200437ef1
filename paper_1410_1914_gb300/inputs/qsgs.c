/*
 * Seeded synthetic catalyst-layer structures: quartet structure generation
 * set (QSGS) growth of Sec. 2.1.2 of arXiv:1410.1914, plus the reactive-face
 * sampling used for the Pt layer.  This is input generation only: it holds
 * none of the solver's arithmetic and is used identically by the CUDA path's
 * callers and by the CPU oracle's tests.
 *
 * Random numbers come from a counter-based generator, SplitMix64 (Steele,
 * Lea and Flood, OOPSLA 2014) applied to a mix of (seed, stream, a, b), so
 * the result does not depend on the number of threads or the visit order.
 *
 * Growth reading (Sec. 2.1.2.1, steps 1-3): seeds are placed once with
 * probability c_d; then synchronous sweeps over a snapshot of the field.  A
 * candidate cell (allowed to convert, 6-adjacent to the grown set) is
 * accepted when it has at least two grown neighbours (rule 2a: a grown
 * neighbour other than the parent), otherwise with probability P_alpha
 * (rule 2b, isotropic).  Neighbourhoods wrap in x, y and z.  The sweep that
 * would overshoot the target count accepts only the candidates with the
 * smallest priority hash, so every phase ends exactly at its target.
 *
 * Cell index: x + nx*(y + ny*z).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* hash of a 4-tuple; each field is folded through one SplitMix64 round */
uint64_t qsgs_hash4(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b)
{
    uint64_t h = splitmix64(seed);
    h = splitmix64(h ^ stream);
    h = splitmix64(h ^ a);
    h = splitmix64(h ^ b);
    return h;
}

/* uniform double in [0, 1) from the top 53 bits */
static inline double u01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

typedef struct { uint64_t key; long cell; } cand_t;

static int cand_cmp(const void* a, const void* b)
{
    const cand_t* x = (const cand_t*)a;
    const cand_t* y = (const cand_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->cell < y->cell ? -1 : (x->cell > y->cell ? 1 : 0);
}

static inline int in_set(uint32_t setmask, uint8_t code) { return (setmask >> code) & 1u; }

/*
 * Grow phase `code` until `target` cells carry it.
 *   allowed_mask: bit k set -> cells of phase k may convert;
 *   grown_mask:   bit k set -> phase k counts as "grown" for adjacency
 *                 (must include `code`);
 *   region:       optional per-cell 0/1 restriction (NULL = everywhere);
 *   c_d:          seed probability on allowed cells (0: no seeding);
 *   p_alpha:      growth probability for single-neighbour candidates.
 * Returns the final number of `code` cells.
 */
long qsgs_grow(uint8_t* phase, int nx, int ny, int nz, uint8_t code, uint32_t allowed_mask,
               uint32_t grown_mask, const uint8_t* region, long target, double c_d,
               double p_alpha, uint64_t seed, uint64_t stream, int max_sweeps)
{
    long N = (long)nx * ny * nz;
    long count = 0;
    for (long c = 0; c < N; ++c) count += phase[c] == code;
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)(N > 0 ? N : 1));

    for (int sweep = 0; sweep <= max_sweeps && count < target; ++sweep) {
        long nc = 0;
        if (sweep == 0) {
            if (c_d <= 0) continue;
            for (long c = 0; c < N; ++c) {
                if (!in_set(allowed_mask, phase[c]) || (region && !region[c])) continue;
                if (u01(qsgs_hash4(seed, stream, 0, (uint64_t)c)) <= c_d)
                    cand[nc++] = (cand_t){qsgs_hash4(seed, stream ^ 0x5bd1e995ULL, 0, (uint64_t)c), c};
            }
        } else {
#pragma omp parallel
            {
                long cap = 4096, n = 0;
                cand_t* loc = (cand_t*)malloc(sizeof(cand_t) * cap);
#pragma omp for schedule(static)
                for (int z = 0; z < nz; ++z)
                    for (int y = 0; y < ny; ++y)
                        for (int x = 0; x < nx; ++x) {
                            long c = x + (long)nx * (y + (long)ny * z);
                            if (!in_set(allowed_mask, phase[c]) || (region && !region[c])) continue;
                            int xs[6] = {(x + 1) % nx, (x + nx - 1) % nx, x, x, x, x};
                            int ys[6] = {y, y, (y + 1) % ny, (y + ny - 1) % ny, y, y};
                            int zs[6] = {z, z, z, z, (z + 1) % nz, (z + nz - 1) % nz};
                            int ng = 0, parent = -1;
                            for (int d = 0; d < 6; ++d) {
                                long q = xs[d] + (long)nx * (ys[d] + (long)ny * zs[d]);
                                if (in_set(grown_mask, phase[q])) { ++ng; parent = d; }
                            }
                            if (ng == 0) continue;
                            int accept = ng >= 2;
                            if (!accept)
                                accept = u01(qsgs_hash4(seed, stream, (uint64_t)sweep * 8 + (uint64_t)parent,
                                                        (uint64_t)c)) <= p_alpha;
                            if (!accept) continue;
                            if (n == cap) { cap *= 2; loc = (cand_t*)realloc(loc, sizeof(cand_t) * cap); }
                            loc[n++] = (cand_t){qsgs_hash4(seed, stream ^ 0x5bd1e995ULL, (uint64_t)sweep,
                                                           (uint64_t)c), c};
                        }
#pragma omp critical
                {
                    memcpy(cand + nc, loc, sizeof(cand_t) * n);
                    nc += n;
                }
                free(loc);
            }
        }
        if (nc == 0) continue;
        long need = target - count;
        if (nc > need) {
            qsort(cand, (size_t)nc, sizeof(cand_t), cand_cmp);
            nc = need;
        }
        for (long j = 0; j < nc; ++j) phase[cand[j].cell] = code;
        count += nc;
    }
    free(cand);
    return count;
}

/*
 * Reactive faces: for every cell of phase `from_code` and each direction
 * d = 1..6 (+x, -x, +y, -y, +z, -z) whose neighbour (y, z periodic, x not)
 * has phase `to_code`, set bit d-1 with probability `fraction`
 * (fraction >= 1: always).  Returns the number of faces set.
 */
long qsgs_reactive_faces(const uint8_t* phase, int nx, int ny, int nz, uint8_t from_code,
                         uint8_t to_code, double fraction, uint64_t seed, uint8_t* out)
{
    long total = 0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = x + (long)nx * (y + (long)ny * z);
                uint8_t bits = 0;
                if (phase[c] == from_code) {
                    const int dx[6] = {1, -1, 0, 0, 0, 0}, dy[6] = {0, 0, 1, -1, 0, 0},
                              dz[6] = {0, 0, 0, 0, 1, -1};
                    for (int d = 0; d < 6; ++d) {
                        int qx = x + dx[d];
                        if (qx < 0 || qx >= nx) continue;
                        int qy = (y + dy[d] + ny) % ny, qz = (z + dz[d] + nz) % nz;
                        if (phase[qx + (long)nx * (qy + (long)ny * qz)] != to_code) continue;
                        if (fraction >= 1.0 || u01(qsgs_hash4(seed, 0xface, (uint64_t)c, (uint64_t)d)) < fraction) {
                            bits |= (uint8_t)(1u << d);
                            ++total;
                        }
                    }
                }
                out[c] = bits;
            }
    return total;
}

/* cells of phase `code` none of whose 6 neighbours (all periodic) has phase `avoid` */
void qsgs_region_not_adjacent(const uint8_t* phase, int nx, int ny, int nz, uint8_t code,
                              uint8_t avoid, uint8_t* region)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = x + (long)nx * (y + (long)ny * z);
                int ok = phase[c] == code;
                if (ok) {
                    int xs[6] = {(x + 1) % nx, (x + nx - 1) % nx, x, x, x, x};
                    int ys[6] = {y, y, (y + 1) % ny, (y + ny - 1) % ny, y, y};
                    int zs[6] = {z, z, z, z, (z + 1) % nz, (z + nz - 1) % nz};
                    for (int d = 0; d < 6 && ok; ++d)
                        if (phase[xs[d] + (long)nx * (ys[d] + (long)ny * zs[d])] == avoid) ok = 0;
                }
                region[c] = (uint8_t)ok;
            }
}
