// batch.cu -- many independent cells with uneven grids in one persistent launch.
//
// Each cell is a full Hartree step (atom preparation with the splat tiles' atom
// lists, the binned splat, five Poisson passes, E_H).  All cells' work is cut into items (stage, cell, tile) and put
// in one global queue in stage-major order: every item of stage s (of every
// cell) precedes every item of stage s + 1.  Persistent CTAs take items with
// one atomic increment; before running an item of stage s of cell c, a CTA
// waits until all items of stage s - 1 of cell c are done (a per-(stage, cell)
// counter).  Those items were taken earlier by running CTAs, so the wait
// always ends; it is nevertheless bounded and sets the batch's error word if
// it gives up.  Loads of data written earlier in the same launch bypass L1.
//
// The launch is asynchronous, allocates nothing and can be captured in a
// CUDA graph (two memsets and one kernel).
#include <algorithm>
#include <vector>

#include "atoms_dev.cuh"
#include "passes_dev.cuh"
#include "tma.cuh"

namespace hartree {

namespace {

enum { ST_PREP, ST_FACT, ST_LEAF, ST_SPLAT, ST_C, ST_B, ST_A, ST_BI, ST_CI, ST_E, NST };

struct BatchCell {
    PoissonArgs<float> pa;
    AtomArgs<float> aa;  // pos / q filled in per launch from the base pointers
    long long grid_off;  // first element of the cell's grid in the caller's vh
    int atom_off;        // first atom of the cell in the caller's pos / q
    int splat_tb, splat_tc;
    int splat_ta;
    int* cursor;         // the cell's splat-tile lists (its plan's): atoms per tile, then the entries
    int4* list;
    double eh_factor;    // 2 pi Omega / N^2
    int cnt[NST];        // items of each stage
};

struct BatchArgs {
    const BatchCell* cells;
    int n_cells;
    const long long* off;  // [NST][n_cells + 1]: first item of (stage, cell); row s ends at the next row's start
    long long total;
    unsigned long long* head;  // next item (zeroed before the launch)
    int* done;                 // [NST][n_cells] finished items (zeroed before the launch)
    int* err;
    // fault injection (tests of the bounded waits; off: skip_stage = -1, spin_limit = kSpinLimit):
    // item 0 of (skip_stage, skip_cell) does its work but is never counted done
    int skip_stage, skip_cell;
    uint32_t spin_limit;  // dependency-wait probes before a wait gives up
};

template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_batched(BatchArgs b, const double* pos, const double* q,
                                                            float* vh, double* eh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kThreads / 32];
    __shared__ int s_stage, s_cell, s_tile, s_ok;
    // Thread 0 takes items, decodes them and waits for their dependencies; the CTA meets once per
    // item before the work and once after it.  It takes the next item while the CTA works on the
    // current one (always a later item in the queue, so the earliest unfinished item never waits
    // on a held one), and it remembers the last (stage, cell) whose previous stage it saw complete:
    // a CTA's consecutive items mostly share it, and then need no look at the counter.
    long long next = 0;
    int seen_s = -1, seen_c = -1;
    if (threadIdx.x == 0) next = (long long)atomicAdd(b.head, 1ULL);
    for (;;) {
        if (threadIdx.x == 0) {
            const long long item = next;
            int s = -1, c = 0, t = 0, ok = 1;
            if (item < b.total) {
                next = (long long)atomicAdd(b.head, 1ULL);
                // decode (stage, cell, tile)
                const int stride = b.n_cells + 1;
                s = 0;
                while (s + 1 < NST && item >= b.off[(s + 1) * stride]) ++s;
                const long long* o = b.off + s * stride;
                int lo = 0, hi = b.n_cells;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (o[mid] <= item)
                        lo = mid;
                    else
                        hi = mid;
                }
                c = lo;
                t = (int)(item - o[c]);
                if (s > 0 && !(s == seen_s && c == seen_c)) {
                    const int need = b.cells[c].cnt[s - 1];
                    volatile int* d = b.done + (s - 1) * b.n_cells + c;
                    uint32_t it = 0;
                    while (*d < need) {
                        if (++it > b.spin_limit) {
                            atomicOr(b.err, kErrTimeout);
                            ok = 0;
                            break;
                        }
                        __nanosleep(64);
                    }
                    __threadfence();
                    if (ok) seen_s = s, seen_c = c;
                }
            }
            s_stage = s;
            s_cell = c;
            s_tile = t;
            s_ok = ok;
        }
        __syncthreads();
        const int s = s_stage, c = s_cell, t = s_tile;
        if (s < 0) break;
        const BatchCell& cell = b.cells[c];
        if (s_ok) {
            const PoissonArgs<float>& pa = cell.pa;
            AtomArgs<float> aa = cell.aa;
            aa.pos = pos + 3LL * cell.atom_off;
            aa.q = q + cell.atom_off;
            float* grid = vh + cell.grid_off;
            switch (s) {
                case ST_PREP:
                    atom_prep_one(aa, t * kThreads + threadIdx.x);
                    if (t == 0)  // empty lists for the leaf stage's appends
                        for (int i = threadIdx.x; i < cell.splat_ta * cell.splat_tb * cell.splat_tc; i += kThreads)
                            cell.cursor[i] = 0;
                    break;
                case ST_FACT: atom_factors_one(aa, (long long)t * kThreads + threadIdx.x); break;
                case ST_LEAF: {
                    const int i = t * kThreads + threadIdx.x;
                    leaf_box_one(aa.prep, aa.n, aa.apl, aa.nleaves, pa.n1, pa.n2, pa.n3, aa.leaf, i);
                    if (i < aa.n)
                        bin_atom(aa, i, cell.splat_ta, cell.splat_tb, cell.splat_tc, cell.cursor, cell.list, 0, 1);
                    break;
                }
                case ST_SPLAT: {
                    SplatWs<float>& w = *reinterpret_cast<SplatWs<float>*>(smem_raw);
                    if (!splat_tile_binned<float, false, true>(aa, grid, cell.splat_tb, cell.splat_tc, t, cell.cursor,
                                                         cell.list, w.ent, w.sorted, w.fa, w.fb, w.fc))
                        splat_tile(aa, grid, cell.splat_tb, cell.splat_tc, t);
                    break;
                }
                case ST_C: c_r2c_tile<float, true>(grid, pa, t, smem_raw); break;
                case ST_B: b_tile<float, false, true>(pa, t, smem_raw); break;
                case ST_A: a_green_tile<float, true>(pa, t, t, smem_raw, red); break;
                case ST_BI: b_tile<float, true, true>(pa, t, smem_raw); break;
                case ST_CI: c_c2r_tile<float, true>(grid, pa, t, smem_raw); break;
                default: {  // ST_E: fixed-order FP64 sum of the a pass's partials
                    double v = 0.0;
                    for (int i = threadIdx.x; i < cell.cnt[ST_A]; i += kThreads) v += __ldcg(pa.eh_partials + i);
                    const double tot = block_sum_double(v, red);
                    if (threadIdx.x == 0) eh[c] = cell.eh_factor * tot;
                    break;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && !(s == b.skip_stage && c == b.skip_cell && t == 0)) {
            __threadfence();
            atomicAdd(b.done + s * b.n_cells + c, 1);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
cudaError_t configure_batched(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_batched<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batched<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

struct BatchHost {
    std::vector<hartree_plan> plans;
    std::vector<long long> grid_off;
    std::vector<int> atom_off;
    BatchCell* cells_d = nullptr;
    long long* off_d = nullptr;
    unsigned long long* head_d = nullptr;
    int* done_d = nullptr;
    int* err_d = nullptr;
    long long total = 0;
    size_t smem = 0;
    int grid = 0;
    int n_cells = 0;
    int minb = 2;                        // the kernel's register budget: 2 or 3 CTAs per SM
    int skip_stage = -1, skip_cell = 0;  // fault injection (hartree_batch_fault_inject)
    uint32_t spin_limit = kSpinLimit;
};

}  // namespace hartree

struct hartree_batch_s {
    hartree::BatchHost h;
};

using namespace hartree;

namespace {

int batch_fail(int status, const char* msg) {
    set_last_error(msg);
    return status;
}

void batch_free(BatchHost& h) {
    for (hartree_plan p : h.plans) hartree_plan_destroy(p);
    h.plans.clear();
    void* ptrs[] = {h.cells_d, h.off_d, h.head_d, h.done_d, h.err_d};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

extern "C" int hartree_batch_create(const hartree_desc* descs, const int* atom_counts, int n_cells,
                                    hartree_batch* out) {
    if (!descs || !atom_counts || !out || n_cells < 1) return batch_fail(HARTREE_ERR_INVALID, "batch_create: bad argument");
    *out = nullptr;
    for (int c = 0; c < n_cells; ++c)  // checked for every cell before any device work
        if (descs[c].precision != HARTREE_FP32 || atom_counts[c] < 0)
            return batch_fail(HARTREE_ERR_INVALID, "batch_create: cells must be FP32 with non-negative atom counts");
    hartree_batch_s* bh = new (std::nothrow) hartree_batch_s();
    if (!bh) return batch_fail(HARTREE_ERR_OOM, "batch_create: host allocation failed");
    BatchHost& h = bh->h;
    h.n_cells = n_cells;
    std::vector<BatchCell> cells(n_cells);
    std::vector<long long> off((size_t)NST * (n_cells + 1));
    h.grid_off.assign(n_cells + 1, 0);
    h.atom_off.assign(n_cells + 1, 0);
    for (int c = 0; c < n_cells; ++c) {
        hartree_desc d = descs[c];
        d.max_atoms = atom_counts[c] > 0 ? atom_counts[c] : 1;
        hartree_plan pl = nullptr;
        const int st = hartree_plan_create(&d, &pl);
        if (st != HARTREE_OK) {
            batch_free(h);
            delete bh;
            return st;  // the plan left its message in hartree_last_error()
        }
        h.plans.push_back(pl);
        const Plan& p = pl->p;
        BatchCell& bc = cells[c];
        bc.pa = make_args<float>(p);
        bc.aa = make_atom_args<float>(p, nullptr, nullptr, atom_counts[c]);
        bc.grid_off = h.grid_off[c];
        bc.atom_off = h.atom_off[c];
        h.grid_off[c + 1] = h.grid_off[c] + (long long)p.n[0] * p.n[1] * p.n[2];
        h.atom_off[c + 1] = h.atom_off[c] + atom_counts[c];
        const int n = atom_counts[c];
        const int runs = (p.box_max + kRun<float>() - 1) / kRun<float>();
        bc.splat_tb = (p.n[1] + TB - 1) / TB;
        bc.splat_tc = (p.n[2] + TC - 1) / TC;
        const int tA = (p.n[0] + TA - 1) / TA;
        bc.splat_ta = tA;
        bc.cursor = p.bin_cursor;
        bc.list = p.bin_list;
        const long long nlines = (long long)p.n[0] * p.n[1];
        bc.cnt[ST_PREP] = std::max(1, (n + kThreads - 1) / kThreads);  // item 0 also empties the tile lists
        bc.cnt[ST_FACT] = (int)((3LL * n * runs + kThreads - 1) / kThreads);
        bc.cnt[ST_LEAF] = (std::max(bc.aa.nleaves, n) + kThreads - 1) / kThreads;  // leaf boxes and tile lists
        bc.cnt[ST_SPLAT] = tA * bc.splat_tb * bc.splat_tc;
        bc.cnt[ST_C] = (int)((nlines + p.c_lines - 1) / p.c_lines);
        bc.cnt[ST_B] = p.n[0] * bc.pa.b_chunks;
        bc.cnt[ST_A] = p.n[1] * bc.pa.a_chunks;
        bc.cnt[ST_BI] = bc.cnt[ST_B];
        bc.cnt[ST_CI] = bc.cnt[ST_C];
        bc.cnt[ST_E] = 1;
        const double ntot = (double)p.n[0] * p.n[1] * p.n[2];
        bc.eh_factor = 2.0 * 3.14159265358979323846 * p.omega / (ntot * ntot);
        size_t sm = p.smem_c;
        if (p.smem_b > sm) sm = p.smem_b;
        if (p.smem_a > sm) sm = p.smem_a;
        if (sm < sizeof(SplatWs<float>)) sm = sizeof(SplatWs<float>);
        if (sm > h.smem) h.smem = sm;
    }
    long long item = 0;
    for (int s = 0; s < NST; ++s) {
        for (int c = 0; c < n_cells; ++c) {
            off[(size_t)s * (n_cells + 1) + c] = item;
            item += cells[c].cnt[s];
        }
        off[(size_t)s * (n_cells + 1) + n_cells] = item;
    }
    h.total = item;
    cudaError_t e = cudaMalloc(&h.cells_d, sizeof(BatchCell) * n_cells);
    if (e == cudaSuccess) e = cudaMalloc(&h.off_d, sizeof(long long) * off.size());
    if (e == cudaSuccess) e = cudaMalloc(&h.head_d, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h.done_d, sizeof(int) * NST * n_cells);
    if (e == cudaSuccess) e = cudaMalloc(&h.err_d, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(h.cells_d, cells.data(), sizeof(BatchCell) * n_cells, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h.off_d, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h.err_d, 0, sizeof(int));
    if (e == cudaSuccess) e = configure_batched(h.smem);
    int per_sm = 0, dev = 0, sms = 0;
    // three CTAs per SM when the tiles' shared memory allows it (the registers are then capped at 80)
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched<3>, kThreads, h.smem);
    if (e == cudaSuccess && per_sm < 3)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched<2>, kThreads, h.smem);
    else
        h.minb = 3;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free(h);
        delete bh;
        return batch_fail(e == cudaErrorMemoryAllocation ? HARTREE_ERR_OOM : HARTREE_ERR_CUDA,
                          "batch_create: device setup failed");
    }
    h.grid = sms * (per_sm > 0 ? per_sm : 1);
    *out = bh;
    return HARTREE_OK;
}

extern "C" void hartree_batch_destroy(hartree_batch batch) {
    if (!batch) return;
    cudaDeviceSynchronize();
    batch_free(batch->h);
    delete batch;
}

extern "C" int hartree_batch_offsets(hartree_batch batch, long long* grid_off, int* atom_off) {
    if (!batch || !grid_off || !atom_off) return batch_fail(HARTREE_ERR_INVALID, "batch_offsets: null argument");
    for (int c = 0; c <= batch->h.n_cells; ++c) {
        grid_off[c] = batch->h.grid_off[c];
        atom_off[c] = batch->h.atom_off[c];
    }
    return HARTREE_OK;
}

extern "C" int hartree_solve_batched(hartree_batch batch, const double* pos, const double* q, void* vh, double* eh,
                                     void* stream) {
    if (!batch || !vh || !eh) return batch_fail(HARTREE_ERR_INVALID, "solve_batched: null argument");
    if (reinterpret_cast<uintptr_t>(vh) % 8 != 0)  // grid lines move as (re, im) float pairs
        return batch_fail(HARTREE_ERR_INVALID, "solve_batched: vh must be aligned to 8 bytes");
    BatchHost& h = batch->h;
    if (h.atom_off[h.n_cells] > 0 && (!pos || !q))
        return batch_fail(HARTREE_ERR_INVALID, "solve_batched: null atom arrays");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(h.head_d, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h.done_d, 0, sizeof(int) * NST * h.n_cells, s);
    if (e == cudaSuccess) {
        BatchArgs a;
        a.cells = h.cells_d;
        a.n_cells = h.n_cells;
        a.off = h.off_d;
        a.total = h.total;
        a.head = h.head_d;
        a.done = h.done_d;
        a.err = h.err_d;
        a.skip_stage = h.skip_stage;
        a.skip_cell = h.skip_cell;
        a.spin_limit = h.spin_limit;
        if (h.minb == 3)
            k_batched<3><<<h.grid, kThreads, h.smem, s>>>(a, pos, q, static_cast<float*>(vh), eh);
        else
            k_batched<2><<<h.grid, kThreads, h.smem, s>>>(a, pos, q, static_cast<float*>(vh), eh);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return batch_fail(HARTREE_ERR_CUDA, cudaGetErrorString(e));
    return HARTREE_OK;
}

extern "C" int hartree_batch_fault_inject(hartree_batch batch, int skip_stage, int skip_cell, unsigned spin_limit) {
    if (!batch) return batch_fail(HARTREE_ERR_INVALID, "batch_fault_inject: null batch");
    BatchHost& h = batch->h;
    if (skip_stage < -1 || skip_stage >= NST - 1 || (skip_stage >= 0 && (skip_cell < 0 || skip_cell >= h.n_cells)))
        return batch_fail(HARTREE_ERR_INVALID, "batch_fault_inject: stage must be in [-1, 8], cell in [0, n_cells)");
    h.skip_stage = skip_stage;
    h.skip_cell = skip_stage >= 0 ? skip_cell : 0;
    h.spin_limit = spin_limit > 0 ? (uint32_t)spin_limit : kSpinLimit;
    return HARTREE_OK;
}

extern "C" int hartree_batch_device_status(hartree_batch batch) {
    if (!batch) return batch_fail(HARTREE_ERR_INVALID, "batch_device_status: null batch");
    int err = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&err, batch->h.err_d, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && err) e = cudaMemset(batch->h.err_d, 0, sizeof(int));
    if (e != cudaSuccess) return batch_fail(HARTREE_ERR_CUDA, cudaGetErrorString(e));
    if (err) return batch_fail(HARTREE_ERR_TIMEOUT, "batched solve: a bounded dependency wait gave up");
    return HARTREE_OK;
}
