// Many structures of uneven size stepped by one persistent launch.
//
// A batch groups existing solver handles (each with its structure loaded).
// One cooperative launch of k_march_batch advances every structure that is
// still running by K steps: the blocks (up to three per SM, all resident) take
// (step, item) pairs from one queue, an item being a (structure, 512-cell
// tile column -- 64 x 8, 32 x 16 or 16 x 32, the member's shape -- z range);
// an item of step t waits only until its own structure's
// step t - 1 is done (a bounded wait on a per-structure count), so structures
// pipeline across steps with no grid-wide barrier.  The last step of a launch also
// reduces each structure's fluxes; the host applies each structure's stopping
// rule and drops converged structures from the work list, whose length is
// read on the device, so the captured graph stays valid as the batch shrinks.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "handle.cuh"

using namespace cl;

struct cl_batch {
    int n = 0;
    std::vector<cl_lbm*> m;
    int storage = 0;
    long long K = 0;
    cudaStream_t s = nullptr;
    cudaStream_t cap = nullptr;
    int grid = 0;
    int grid_reduce = 0;
    int z_chunk = 32;
    int prefetch = 0;
    int parity = 0;
    int max_items = 0;
    int n_items = 0;
    BatchInst* d_insts = nullptr;
    WorkItem* d_items = nullptr;
    int* d_n_items = nullptr;
    int* d_inst_first = nullptr;
    int* d_inst_count = nullptr;
    unsigned long long* d_next = nullptr;  // queue position
    unsigned long long* d_done = nullptr;  // [n] finished items per member
    int* d_abort = nullptr;
    int* d_err = nullptr;
    double* d_item_partials = nullptr;
    double* d_inst_red = nullptr;
    double* h_inst_red = nullptr;  // pinned [n][RED_N]
    std::vector<char> active;
    std::vector<int> own_rw;  // each member's handle's tile shape at creation
    std::vector<int> rw;      // tile rows per warp in use for each member
    int tile_rows = 0;        // 1, 2, 4: one shape for every member; 0: the members' own
    cudaGraphExec_t graph = nullptr;
    bool graph_ok = true;
    long long wait_limit = 0;  // step-dependency wait bound (0: default)
    int never_arrive = 0;      // test hook (cl_batch_set_wait_test)
};

namespace {

int items_of(const cl_lbm* h, int rw, int zc) {
    const int bx = kBX / rw, by = kBY * rw;
    return ((h->nx + bx - 1) / bx) * ((h->ny + by - 1) / by) * ((h->nz + zc - 1) / zc);
}

// One tile shape for every member unless the policy is 0 (the members' own
// shapes): blocks that march different shapes at once on one SM run three
// copies of the march code, which measured slower than any single shape.
void apply_tile_policy(cl_batch* b) {
    for (int i = 0; i < b->n; ++i) b->rw[i] = b->tile_rows ? b->tile_rows : b->own_rw[i];
}

// the uniform shape of least summed cost over the members
int batch_auto_rows(const cl_batch* b) {
    int best = 1;
    double best_cost = 0.0;
    for (int rw = 1; rw <= kRowsMax; rw *= 2) {
        double c = 0.0;
        for (const cl_lbm* h : b->m) c += march_tile_cost(h->nx, h->ny, b->storage, rw) * h->nz;
        if (rw == 1 || c < best_cost * (1.0 - 1e-9)) { best = rw; best_cost = c; }
    }
    return best;
}

// Work list over the running structures: each column's planes split into
// ceil(nz / z_chunk) ranges of nearly equal length (no short remainder range,
// whose two halo planes and pipeline fill would cost as much as its work).
cl_status upload_items(cl_batch* b) {
    std::vector<WorkItem> items;
    std::vector<int> first(b->n, 0), count(b->n, 0);
    for (int i = 0; i < b->n; ++i) {
        first[i] = (int)items.size();
        if (!b->active[i]) continue;
        const cl_lbm* h = b->m[i];
        const int rw = b->rw[i], bx = kBX / rw, by = kBY * rw;
        const int g = (h->nz + b->z_chunk - 1) / b->z_chunk;
        for (int j = 0; j < g; ++j) {
            const int zs = (int)((long long)h->nz * j / g), ze = (int)((long long)h->nz * (j + 1) / g);
            for (int y0 = 0; y0 < h->ny; y0 += by)
                for (int x0 = 0; x0 < h->nx; x0 += bx) items.push_back(WorkItem{i, x0, y0, zs, ze, rw});
        }
        count[i] = (int)items.size() - first[i];
    }
    b->n_items = (int)items.size();
    if (b->n_items > b->max_items) { set_msg_txt("work list larger than allocated"); return CL_ERR_STATE; }
    if (b->n_items) CK(cudaMemcpyAsync(b->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, b->s));
    CK(cudaMemcpyAsync(b->d_n_items, &b->n_items, sizeof(int), cudaMemcpyHostToDevice, b->s));
    CK(cudaMemcpyAsync(b->d_inst_first, first.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->s));
    CK(cudaMemcpyAsync(b->d_inst_count, count.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->s));
    CK(cudaStreamSynchronize(b->s));
    return CL_OK;
}

cl_status upload_insts(cl_batch* b) {
    std::vector<BatchInst> insts(b->n);
    for (int i = 0; i < b->n; ++i) {
        cl_lbm* h = b->m[i];
        CKS(build_march_maps(h, b->rw[i], insts[i].maps));
        for (int par = 0; par < 2; ++par) {
            insts[i].args[par] = make_margs(h, par ^ 1);
            insts[i].args[par].prefetch = b->prefetch;
        }
    }
    CK(cudaMemcpyAsync(b->d_insts, insts.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice, b->s));
    CK(cudaStreamSynchronize(b->s));
    return CL_OK;
}

BatchLaunch launch_desc(cl_batch* b, int nsteps, bool reduce_last) {
    BatchLaunch L;
    L.storage = b->storage;
    L.grid = b->grid;
    L.grid_reduce = b->grid_reduce;
    L.n_inst = b->n;
    L.insts = b->d_insts;
    L.items = b->d_items;
    L.n_items = b->d_n_items;
    L.inst_count = b->d_inst_count;
    L.nsteps = nsteps;
    L.parity0 = b->parity;
    L.reduce_last = reduce_last ? 1 : 0;
    L.next = b->d_next;
    L.done = b->d_done;
    L.abort_flag = b->d_abort;
    L.item_partials = b->d_item_partials;
    L.err = b->d_err;
    L.wait_limit = b->wait_limit;
    L.never_arrive = b->never_arrive;
    return L;
}

cl_status batch_err(cl_batch* b) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->s));
    CK(cudaStreamSynchronize(b->s));
    if (e) {  // reported once: the next call starts from a clean error word
        CK(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->s));
        CK(cudaStreamSynchronize(b->s));
    }
    if (e & 32) {
        set_msg_txt("a step-dependency wait of the batched step did not complete within its bound");
        return CL_ERR_TIMEOUT;
    }
    if (e) { set_msg_txt("batched step kernel raised an error"); return CL_ERR_CUDA; }
    for (auto* h : b->m) CKS(check_err_flag(h));
    return CL_OK;
}

void drop_graph(cl_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// K steps with the per-structure reduction, as one graph when the runtime
// captures cooperative launches, else as plain launches in the same order.
cl_status enqueue_interval(cl_batch* b, cudaStream_t s) {
    CK(launch_march_batch(launch_desc(b, (int)b->K, true), s));
    CK(launch_batch_finalize(b->d_item_partials, b->d_inst_first, b->d_inst_count, b->n, b->d_inst_red, s));
    CK(cudaMemcpyAsync(b->h_inst_red, b->d_inst_red, sizeof(double) * RED_N * b->n, cudaMemcpyDeviceToHost, s));
    return CL_OK;
}

cl_status run_interval(cl_batch* b) {
    if (b->graph_ok && !b->graph) {
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cl_status st = enqueue_interval(b, b->cap);
            ok = cudaStreamEndCapture(b->cap, &g) == cudaSuccess && st == CL_OK && g;
        }
        if (ok) ok = cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            b->graph = nullptr;
            b->graph_ok = false;
            cudaGetLastError();  // clear a capture refusal; run the same work uncaptured
        }
    }
    if (b->graph) CK(cudaGraphLaunch(b->graph, b->s));
    else CKS(enqueue_interval(b, b->s));
    CK(cudaStreamSynchronize(b->s));
    return batch_err(b);
}

}  // namespace

extern "C" {

cl_status cl_batch_create(cl_batch_handle* out, const cl_handle* members, int n, int z_chunk) {
    if (!out || !members || n < 1) { set_msg_txt("NULL argument or empty batch"); return CL_ERR_ARG; }
    const cl_lbm* h0 = members[0];
    for (int i = 0; i < n; ++i) {
        const cl_lbm* h = members[i];
        if (!h) { set_msg_txt("NULL member"); return CL_ERR_ARG; }
        if (!h->have_structure) { set_msg_txt("member without a structure"); return CL_ERR_STATE; }
        if (h->q != 7) { set_msg_txt("batch members must use the D3Q7 lattice"); return CL_ERR_ARG; }
        if (!h->march) { set_msg_txt("batch members need FP32 or FP16 (C, delta) storage"); return CL_ERR_ARG; }
        if (h->p.storage != h0->p.storage || h->p.check_every != h0->p.check_every) {
            set_msg_txt("batch members must share storage mode and check_every");
            return CL_ERR_ARG;
        }
        if (h->cur != h0->cur) { set_msg_txt("batch members must be at the same step parity"); return CL_ERR_STATE; }
    }
    if (z_chunk < 0) { set_msg_txt("z_chunk < 0"); return CL_ERR_ARG; }
    cl_batch* b = new cl_batch();
    b->n = n;
    b->m.assign(members, members + n);
    b->storage = h0->p.storage;
    b->K = h0->p.check_every;
    b->s = h0->s;
    b->parity = h0->cur;
    b->z_chunk = z_chunk > 0 ? z_chunk : 32;
    b->prefetch = h0->prefetch;
    b->active.assign(n, 1);
    for (int i = 0; i < n; ++i) b->own_rw.push_back(members[i]->tile_rw);
    b->rw = b->own_rw;
    b->tile_rows = batch_auto_rows(b);
    apply_tile_policy(b);
    auto fail = [&](cl_status st) { cl_batch_destroy(b); return st; };
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { set_msg("cudaStreamCreate", e); return fail(from_cuda(e)); }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = march_batch_blocks_per_sm(b->storage, false);
    const int per_sm_r = march_batch_blocks_per_sm(b->storage, true);
    if (per_sm < 1 || per_sm_r < 1) { set_msg_txt("batched step kernel does not fit on an SM"); return fail(CL_ERR_CUDA); }
    b->grid = nsm * per_sm;
    b->grid_reduce = nsm * per_sm_r;
    // the work list is largest at the smallest z chunk the autotuner tries, in the member's largest tiling
    for (int i = 0; i < n; ++i) {
        int most = 0;
        for (int rw = 1; rw <= kRowsMax; rw *= 2) most = std::max(most, items_of(b->m[i], rw, std::min(8, b->z_chunk)));
        b->max_items += most;
    }
    e = cudaMallocAsync(&b->d_insts, sizeof(BatchInst) * n, b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_items, sizeof(WorkItem) * b->max_items, b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_n_items, sizeof(int), b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_inst_first, sizeof(int) * n, b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_inst_count, sizeof(int) * n, b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_next, sizeof(unsigned long long), b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_done, sizeof(unsigned long long) * n, b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_abort, sizeof(int), b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_err, sizeof(int), b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_item_partials, sizeof(double) * RED_N * b->max_items, b->s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b->d_inst_red, sizeof(double) * RED_N * n, b->s);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_inst_red, sizeof(double) * RED_N * n);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->s);
    if (e != cudaSuccess) { set_msg("batch allocation", e); return fail(from_cuda(e)); }
    cl_status st = upload_insts(b);
    if (st == CL_OK) st = upload_items(b);
    if (st != CL_OK) return fail(st);
    *out = b;
    return CL_OK;
}

void cl_batch_destroy(cl_batch_handle b) {
    if (!b) return;
    drop_graph(b);
    if (b->s || true) cudaStreamSynchronize(b->s);
    void* ptrs[] = {b->d_insts, b->d_items, b->d_n_items, b->d_inst_first, b->d_inst_count, b->d_next,
                    b->d_done, b->d_abort, b->d_err, b->d_item_partials, b->d_inst_red};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, b->s);
    cudaStreamSynchronize(b->s);
    if (b->h_inst_red) cudaFreeHost(b->h_inst_red);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

cl_status cl_batch_step(cl_batch_handle b, long long nsteps) {
    if (!b || nsteps < 0 || nsteps > (1LL << 30)) { set_msg_txt("bad argument"); return CL_ERR_ARG; }
    for (auto* h : b->m)
        if (h->cur != b->parity) { set_msg_txt("a member was stepped outside the batch"); return CL_ERR_STATE; }
    if (nsteps == 0) return CL_OK;
    CK(launch_march_batch(launch_desc(b, (int)nsteps, false), b->s));
    CK(cudaStreamSynchronize(b->s));
    CKS(batch_err(b));
    b->parity ^= (int)(nsteps & 1);
    for (int i = 0; i < b->n; ++i)
        if (b->active[i]) {
            b->m[i]->cur = b->parity;
            b->m[i]->step += nsteps;
        }
    return CL_OK;
}

cl_status cl_batch_solve(cl_batch_handle b, long long max_steps, cl_solve_info* infos, int* n_converged) {
    if (!b || max_steps < 0) { set_msg_txt("bad argument"); return CL_ERR_ARG; }
    for (auto* h : b->m)
        if (h->cur != b->parity) { set_msg_txt("a member was stepped outside the batch"); return CL_ERR_STATE; }
    if (b->K & 1) { set_msg_txt("check_every must be even"); return CL_ERR_STATE; }
    auto t0 = std::chrono::steady_clock::now();
    const int n = b->n;
    std::vector<cl_solve_info> inf(n);
    std::vector<double> q_prev(n, NAN), dq_prev(n, NAN);
    std::vector<int> nchecks(n, 0), quiet(n, 0);
    for (auto& x : inf) { memset(&x, 0, sizeof(x)); x.rel_change = INFINITY; }
    std::fill(b->active.begin(), b->active.end(), 1);
    CKS(upload_items(b));
    cl_status result = CL_OK;
    long long steps = 0;
    int running = n;
    while (running > 0 && steps + b->K <= max_steps) {
        CKS(run_interval(b));
        steps += b->K;
        bool changed = false;
        for (int i = 0; i < n; ++i) {
            if (!b->active[i]) continue;
            cl_lbm* h = b->m[i];
            h->step += b->K;
            cl_solve_info& x = inf[i];
            x.steps += b->K;
            const double* r = b->h_inst_red + (size_t)RED_N * i;
            x.J_in = r[RED_JIN];
            x.J_out = r[RED_JOUT];
            x.R = r[RED_R];
            x.resid = r[RED_ABSC] > 0 ? r[RED_DC] / r[RED_ABSC] : 0.0;
            bool stop = false;
            if (r[RED_NONFINITE] > 0 || !isfinite(x.J_in) || !isfinite(x.J_out) || !isfinite(x.R)) {
                stop = true;
                result = CL_ERR_DIVERGED;
            } else {
                x.flux_balance = fabs(x.J_in - x.J_out - x.R) / fmax(fabs(x.J_in), 1e-300);
                const bool track_deff = h->p.bc_in == CL_BC_DIRICHLET && h->p.bc_out == CL_BC_DIRICHLET &&
                                        h->p.c_in != h->p.c_out;
                const double q = track_deff ? x.J_out : x.R;
                const double dq = q - q_prev[i];
                const double est = nchecks[i] >= 2 ? remaining_change(dq, dq_prev[i]) : INFINITY;
                x.rel_change = q != 0 ? est / fabs(q) : INFINITY;
                q_prev[i] = q;
                dq_prev[i] = dq;
                ++nchecks[i];
                quiet[i] = (x.flux_balance < h->p.tol_flux && x.rel_change < h->p.tol_rel) ? quiet[i] + 1 : 0;
                if (quiet[i] >= 2) {
                    x.converged = 1;
                    stop = true;
                }
            }
            if (stop) {
                b->active[i] = 0;
                --running;
                changed = true;
            }
        }
        if (changed && running > 0) CKS(upload_items(b));
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int nc = 0;
    for (int i = 0; i < n; ++i) {
        inf[i].seconds = secs;
        nc += inf[i].converged;
        if (infos) infos[i] = inf[i];
    }
    if (n_converged) *n_converged = nc;
    // every member can run again (alone or in the batch)
    std::fill(b->active.begin(), b->active.end(), 1);
    CKS(upload_items(b));
    if (result == CL_OK && nc < n) result = CL_ERR_NOT_CONVERGED;
    return result;
}

cl_status cl_batch_autotune(cl_batch_handle b, int steps_per_trial, int* z_chunk_out, int* prefetch_out,
                            int* tile_rows_out, double* best_ms_out) {
    if (!b || steps_per_trial < 2 || (steps_per_trial & 1)) { set_msg_txt("steps_per_trial must be even, >= 2"); return CL_ERR_ARG; }
    for (auto* h : b->m)
        if (h->cur != b->parity) { set_msg_txt("a member was stepped outside the batch"); return CL_ERR_STATE; }
    int nz_max = 0;
    for (auto* h : b->m) nz_max = std::max(nz_max, h->nz);
    const int zcs[] = {8, 16, 32, 64, 128};
    const int pfs[] = {0, 2};
    const int tiles[] = {1, 2, 4};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = INFINITY;
    int bz = b->z_chunk, bp = b->prefetch, bt = b->tile_rows;
    std::fill(b->active.begin(), b->active.end(), 1);
    for (int tr : tiles) {
        b->tile_rows = tr;
        apply_tile_policy(b);
        for (int zc : zcs) {
            if (zc > std::max(8, nz_max)) continue;
            for (int pf : pfs) {
                b->z_chunk = zc;
                b->prefetch = pf;
                CKS(upload_insts(b));
                CKS(upload_items(b));
                CK(cudaEventRecord(e0, b->s));
                CK(launch_march_batch(launch_desc(b, steps_per_trial, false), b->s));
                CK(cudaEventRecord(e1, b->s));
                CK(cudaEventSynchronize(e1));
                CKS(batch_err(b));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                for (auto* h : b->m) h->step += steps_per_trial;  // the trials are real steps
                if (ms < best) { best = ms; bz = zc; bp = pf; bt = tr; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->z_chunk = bz;
    b->prefetch = bp;
    b->tile_rows = bt;
    apply_tile_policy(b);
    drop_graph(b);
    CKS(upload_insts(b));
    CKS(upload_items(b));
    if (z_chunk_out) *z_chunk_out = bz;
    if (prefetch_out) *prefetch_out = bp;
    if (tile_rows_out) *tile_rows_out = bt;
    if (best_ms_out) *best_ms_out = best / steps_per_trial;
    return CL_OK;
}

cl_status cl_batch_configure(cl_batch_handle b, int z_chunk, int prefetch, int tile_rows) {
    if (!b || z_chunk < 8 || prefetch < 0) { set_msg_txt("z_chunk >= 8 and prefetch >= 0 required"); return CL_ERR_ARG; }
    if (tile_rows != 0 && tile_rows != 1 && tile_rows != 2 && tile_rows != 4) {
        set_msg_txt("tile_rows must be 0, 1, 2 or 4");
        return CL_ERR_ARG;
    }
    b->z_chunk = z_chunk;
    b->prefetch = prefetch;
    b->tile_rows = tile_rows;
    apply_tile_policy(b);
    drop_graph(b);
    CKS(upload_insts(b));
    return upload_items(b);
}

cl_status cl_batch_set_wait_test(cl_batch_handle b, long long wait_limit_clocks, int never_arrive) {
    if (!b) { set_msg_txt("NULL batch"); return CL_ERR_ARG; }
    if (wait_limit_clocks < 0) { set_msg_txt("wait_limit_clocks < 0"); return CL_ERR_ARG; }
    if (never_arrive && wait_limit_clocks == 0) {
        set_msg_txt("never_arrive needs a wait limit (a few hundred clocks)");
        return CL_ERR_ARG;
    }
    b->wait_limit = wait_limit_clocks;
    b->never_arrive = never_arrive ? 1 : 0;
    drop_graph(b);  // the wait settings are baked into the captured launch
    return CL_OK;
}

cl_status cl_batch_info(cl_batch_handle b, int* grid_blocks, int* n_items, int* uses_graph) {
    if (!b) { set_msg_txt("NULL batch"); return CL_ERR_ARG; }
    if (grid_blocks) *grid_blocks = b->grid;
    if (n_items) *n_items = b->n_items;
    if (uses_graph) *uses_graph = b->graph ? 1 : 0;
    return CL_OK;
}

}  // extern "C"
