/*
 * hartree.h -- C ABI of the GB300 (sm_103a) grid-side Hartree step.
 *
 * The operation is the Hartree part of the Kohn-Sham potential and energy of
 * Duy & Ozaki, arXiv:1209.4506: Sec. 2.1, Eq. Hartree-potential (the
 * potential of the density) and the E_Hartree term of Eq. total-energy, with
 * the potential "found by solving the Poisson equation using FFT" (Sec. 2.1)
 * in the transform order abc -> cab -> cba -> cab -> abc of Sec. 3.2.4.
 *
 * Conventions shared by every entry point
 *   Units       atomic units: Bohr, Hartree, charge in e.  V_H > 0 near a
 *               positive charge (V_H solves lap V = -4 pi rho).
 *   Cell        orthorhombic, sides L = (L1, L2, L3), volume Omega = L1 L2 L3.
 *   Grid        N = (N1, N2, N3) points along a, b, c; point (i, j, k) sits at
 *               (i L1/N1, j L2/N2, k L3/N3); arrays are C order [N1][N2][N3],
 *               c fastest (the paper's structure B "abc" layout).  dV = Omega/N.
 *   Density     atom i is the Gaussian q_i (pi s^2)^(-3/2) exp(-|r - R_i|^2/s^2)
 *               (s = sigma), summed over all periodic images, truncated per
 *               axis at |x| <= cutoff_sigmas * sigma.
 *   Poisson     V~(G) = 4 pi / |G|^2 rho~(G) for G != 0, V~(0) = 0 (uniform
 *               neutralising background; a net charge is allowed).
 *   Energy      E_H = 1/2 dV sum_r rho(r) V_H(r)   (FP64 on the device).
 *   Forces      F_i = -dE_H/dR_i = -dV sum_r V_H(r) d rho_i(r)/dR_i   (FP64).
 *   Precision   the element type of every void* grid buffer follows the plan:
 *               HARTREE_FP64 -> double, HARTREE_FP32 -> float,
 *               HARTREE_FP32_TC_SPLIT -> float.  Positions, charges, energies
 *               and forces are always double.
 *   Alignment   the Poisson passes move grid lines as (re, im) pairs of the
 *               element type, so every grid buffer read or written by a solve
 *               (rho, vh) must start on a multiple of twice the element size:
 *               8 bytes for float, 16 for double.  Calls given a grid that is
 *               not return HARTREE_ERR_INVALID before any device work.  Grids
 *               that are also 16-byte aligned (any cudaMalloc or torch tensor
 *               start) let FP32 plans stream the c passes with bulk copies.
 *   Memory      "device" pointers are CUDA global memory of the current device,
 *               owned by the caller.  The plan owns its workspace, allocated
 *               once in hartree_plan_create; the per-solve calls allocate
 *               nothing and only enqueue work on the given stream.
 *   Streams     `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *               default stream).  Calls return once the work is enqueued; the
 *               *_host entry points also wait for it.
 *   Errors      every call returns a hartree_status; nothing aborts and no
 *               C++ exception crosses the boundary.  hartree_last_error()
 *               returns a thread-local message for the most recent failure.
 *   Threads     a plan may be used from one host thread at a time.
 */
#ifndef HARTREE_H
#define HARTREE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hartree_plan_s* hartree_plan;
typedef struct hartree_batch_s* hartree_batch;

typedef enum {
    HARTREE_FP64 = 0,          /* FP64 transforms and grids                          */
    HARTREE_FP32 = 1,          /* FP32 transforms and grids, FP64 E_H and forces      */
    HARTREE_FP32_TC_SPLIT = 2  /* FP32; the b passes run as two radix-16 stages on the BF16
                                  tensor cores with hi/lo split operands (N2 must be 256)   */
} hartree_precision;

typedef enum {
    HARTREE_OK = 0,
    HARTREE_ERR_INVALID = 1,          /* null pointer, bad count, sigma <= 0, NaN/Inf ... */
    HARTREE_ERR_UNSUPPORTED_SIZE = 2, /* a grid size that is not 2/3/5/7-smooth, odd N3 ... */
    HARTREE_ERR_CUDA = 3,             /* a CUDA runtime call failed                        */
    HARTREE_ERR_OOM = 4,              /* device allocation failed in a *_create call       */
    HARTREE_ERR_TIMEOUT = 5,          /* a bounded device wait gave up (batched form)      */
    HARTREE_ERR_NOT_CAPTURABLE = 6    /* the call cannot run under stream capture          */
} hartree_status;

typedef struct {
    int n[3];             /* grid points N1, N2, N3; 2/3/5/7-smooth, 2 <= N_d <= 4096, N3 even >= 4 */
    double cell[3];       /* L1, L2, L3 in Bohr, > 0                                        */
    double sigma;         /* Gaussian width s in Bohr, > 0                                  */
    double cutoff_sigmas; /* per-axis truncation radius in units of s; 0 = default
                             (8 for FP64, 5 for FP32); must not exceed 16                   */
    int precision;        /* a hartree_precision                                            */
    int atoms_per_leaf;   /* atoms per bisection leaf used by the splat; 0 = default 16     */
    int max_atoms;        /* largest atom count any call on this plan will pass; 0 = 65536 */
    unsigned flags;       /* 0 or a combination of the HARTREE_FLAG_* values below           */
} hartree_desc;

/* HARTREE_FP32_TC_SPLIT operands: FP16 hi/lo pairs with a power-of-two scale per
 * row by default (three products, about 2^-22 relative per product); this flag
 * selects BF16 operands split in three parts instead (the six products of order
 * <= 2, about 2^-24 relative per product, no scaling, twice the tensor work). */
#define HARTREE_FLAG_TC_BF16 1u

/* FP32 plans: calls that need no density grid (hartree_solve and hartree_step with
 * rho = NULL, hartree_step_host, hartree_forces with vh = NULL) compute the density of
 * each tile of c lines inside the first (r2c) pass, so rho never reaches device memory
 * (the calculation flow of Sec. 3.2.4 without the A -> B grid).  Same results to FP32
 * rounding.  Off by default: the separate splat and r2c kernels are faster on GB300
 * (both are bound by instruction issue, not by the density's round trip through HBM).
 * Ignored by FP64 plans and for c lengths N3 / 2 without a fused kernel (it exists for
 * 60, 64, 105, 128, 200, 210 and 256). */
#define HARTREE_FLAG_FUSED_SPLAT 2u

/* ---------------------------------------------------------------- plans */

/*
 * Validate `desc`, allocate the plan's device workspace (half spectrum,
 * one real grid, twiddle and |G|^2 tables, reduction partials, leaf boxes)
 * and upload the FP64-generated twiddle tables.  Uses the current device.
 * desc: host pointer, read only.  out: host pointer receiving the plan.
 * Returns HARTREE_ERR_UNSUPPORTED_SIZE for grids the transforms do not
 * handle, HARTREE_ERR_OOM when the workspace does not fit.
 */
int hartree_plan_create(const hartree_desc* desc, hartree_plan* out);

/* Free the plan and its workspace (synchronises the device first). NULL is a no-op. */
void hartree_plan_destroy(hartree_plan plan);

/* Bytes of device memory the plan holds. */
unsigned long long hartree_plan_workspace_bytes(hartree_plan plan);

/* ---------------------------------------------------------------- atom reorder */

/*
 * Modified recursive bisection with the inertia-tensor principal axis
 * (Sec. 3.1.2-3.1.5; Eqs. center-of-mass, eq-projection-ti, eq-function-F,
 * eq-inertia-tensor).  Host-side and FP64; run once per geometry (Step 1 of
 * Sec. 4), not per solve.
 *   pos        host [n][3] positions in Bohr (used as given, not wrapped)
 *   w          host [n] weights (Eq. eq-weight-def) or NULL for all 1
 *   n_leaves   number of leaves (the paper's process count), >= 1
 *   perm       host [n] out: atom indices in leaf order
 *   leaf_start host [n_leaves + 1] out: leaf l owns perm[leaf_start[l] ..
 *              leaf_start[l + 1])
 * Reading of the paper: the left child takes ceil(p/2) of p processes and the
 * shortest prefix (by projection t) whose weight W_k satisfies
 * p W_k >= ceil(p/2) W; the axis sign makes its largest component positive.
 */
int hartree_atoms_reorder(const double* pos, const double* w, int n, int n_leaves, int* perm, int* leaf_start);

/*
 * The same decomposition on the device (Sec. 3.1.2-3.1.5), for atoms that
 * move between solves: one kernel launch per level of the bisection tree
 * (ceil(log2 n_leaves) + 1 launches), one CTA per node, FP64 reductions for
 * the centre of mass and the moment matrix, the host's 3x3 Jacobi solver for
 * the principal axis, a bitonic sort by (t, atom index) and the same cut.
 * Asynchronous on `stream`; allocates nothing (the plan's workspace holds the
 * scratch); reads nothing back, so it can be captured in a CUDA graph.
 *   plan       supplies the scratch; n and n_leaves must not exceed its max_atoms
 *   pos        device [n][3] positions in Bohr (used as given; must be finite)
 *   w          device [n] weights >= 0, or NULL for all 1
 *   perm       device [n] out: atom indices in leaf order
 *   leaf_start device [n_leaves + 1] out, as hartree_atoms_reorder
 * The result equals hartree_atoms_reorder's wherever the projections t of two
 * atoms of one node are not tied to within the last bits of the sums (the
 * device sums the centre of mass and the moments in a different order).
 * HARTREE_ERR_INVALID for null pointers or counts out of range.
 */
int hartree_atoms_reorder_device(hartree_plan plan, const double* pos, const double* w, int n, int n_leaves,
                                 int* perm, int* leaf_start, void* stream);

/* ---------------------------------------------------------------- single solves */

/*
 * Density splat (Sec. 3.2.2 structure A -> B): rho on the grid from n
 * Gaussian charges.  Leaves are runs of atoms_per_leaf consecutive atoms; pass
 * atoms in hartree_atoms_reorder order so each grid tile touches a few leaves
 * (any order gives the same result up to rounding).
 *   pos  device [n][3] double, Bohr, any values (periodic images are implied)
 *   q    device [n] double
 *   rho  device [N1][N2][N3] element type of the plan, out
 * 0 <= n <= max_atoms.
 */
int hartree_splat(hartree_plan plan, const double* pos, const double* q, int n, void* rho, void* stream);

/*
 * Poisson solve of a density already on the grid: five passes c-r2c, b, a
 * (forward, x 4 pi/|G|^2, E_H reduction, inverse), b^-1, c-c2r.
 *   rho  device [N1][N2][N3], read only (may alias vh: then it is overwritten)
 *   vh   device [N1][N2][N3], out
 *   eh   device double scalar, out (may be NULL)
 */
int hartree_solve_density(hartree_plan plan, const void* rho, void* vh, double* eh, void* stream);

/*
 * Splat + Poisson solve + E_H.
 *   rho  device [N1][N2][N3] out, or NULL (rho then lives in vh until V_H
 *        overwrites it)
 *   vh   device [N1][N2][N3] out;  eh device double out (may be NULL)
 */
int hartree_solve(hartree_plan plan, const double* pos, const double* q, int n, void* rho, void* vh, double* eh,
                  void* stream);

/*
 * Adjoint gather: forces and charge derivatives from V_H.
 *   vh   device [N1][N2][N3] potential of the same atoms, or NULL: then the
 *        plan first solves into its own grid buffer (recompute, no extra memory)
 *   f    device [n][3] double out, Ha/Bohr (F = -dE_H/dR)
 *   phi  device [n] double out (dE_H/dq_i), may be NULL
 */
int hartree_forces(hartree_plan plan, const double* pos, const double* q, int n, const void* vh, double* f,
                   double* phi, void* stream);

/*
 * The whole Hartree step on device buffers: splat, Poisson solve, E_H and the
 * force gather, with the per-atom preparation done once.
 *   pos, q  device [n][3] and [n] double
 *   rho     device grid out, or NULL (rho then lives in vh until V_H overwrites it)
 *   vh      device grid out;  eh device double out (may be NULL)
 *   f       device [n][3] double out;  phi device [n] double out (may be NULL)
 */
int hartree_step(hartree_plan plan, const double* pos, const double* q, int n, void* rho, void* vh, double* eh,
                 double* f, double* phi, void* stream);

/*
 * End-to-end step on host buffers: copies pos and q to the device, runs
 * splat, solve and forces with V_H kept in the plan's grid buffer, copies E_H
 * (and forces when f is not NULL) back, and waits for the work to finish.
 * The work runs on a stream of the plan's own, after the work already queued
 * on `stream`; its device part is captured into a CUDA graph on the first call
 * and replayed while the atom count, the variant picks and the forces request
 * stay the same (one launch instead of about ten).  Not thread-safe per plan.
 *   pos host [n][3], q host [n], eh host double out, f host [n][3] out or NULL.
 * Returns HARTREE_ERR_NOT_CAPTURABLE when `stream` is being captured.
 */
int hartree_step_host(hartree_plan plan, const double* pos, const double* q, int n, double* eh, double* f,
                      void* stream);

/* ---------------------------------------------------------------- introspection */

/*
 * One pass of the Poisson solve alone, for per-kernel timing and profiling.
 * pass 0: c real-to-complex, rho -> the plan's half spectrum
 * pass 1: b forward;  pass 2: a forward, 4 pi/|G|^2, E_H partial sums, a inverse
 * pass 3: b inverse;  pass 4: c complex-to-real, half spectrum -> vh
 * Calling passes 0..4 in order leaves in vh what hartree_solve_density leaves
 * (the E_H reduction is not run).  rho is read by pass 0, vh written by pass 4;
 * the other passes ignore both.  Returns HARTREE_ERR_INVALID for other pass ids.
 */
int hartree_solve_pass(hartree_plan plan, int pass, const void* rho, void* vh, void* stream);

/*
 * The splat fused into pass 0 alone, for per-kernel timing and profiling: the
 * atoms' boxes and factor arrays, then the kernel that computes the density of
 * each tile of c lines and transforms it into the plan's half spectrum (what
 * hartree_splat + pass 0 leave there, to FP32 rounding).  pos, q: device
 * [n][3], [n] (bisection order).  Returns HARTREE_ERR_INVALID for null
 * pointers or n outside [0, max_atoms], HARTREE_ERR_UNSUPPORTED_SIZE when the
 * plan does not use the fused kernel (no HARTREE_FLAG_FUSED_SPLAT, FP64, or a
 * c length N3 / 2 without one).
 */
int hartree_splat_pass(hartree_plan plan, const double* pos, const double* q, int n, void* stream);

/* 1 if calls with no density grid use the splat fused into pass 0, else 0. */
int hartree_plan_fused_splat(hartree_plan plan);

/* Number of CUDA kernels this plan has launched so far (host-side count). */
unsigned long long hartree_plan_launch_count(hartree_plan plan);

/*
 * Device-side status of the plan's kernels: synchronises the device, then
 * returns HARTREE_ERR_TIMEOUT if any bounded wait inside a kernel (an mbarrier
 * of a TMA-streamed pass) gave up since the last call, else HARTREE_OK.  The
 * error word is cleared by the call.  A timed-out kernel leaves its output
 * incomplete but the CUDA context usable.
 */
int hartree_plan_device_status(hartree_plan plan);

/* ---------------------------------------------------------------- autotuning */

/*
 * Kernel variants: each pass kind (0: the two c passes, 1: the two b passes,
 * 2: the a pass) may have several compiled tile shapes (columns or lines per
 * CTA and threads per CTA); for FP32 b and a passes of 256 or 512 points
 * variants 2 and up are persistent kernels that stream tiles with TMA bulk
 * copies, those past the first with radix-32 stages.  The c passes have V
 * variants each (plain tiles, then bulk-copy streams) and V * V picks: a pick
 * v < V runs both c passes on variant v, a pick V + m runs the r2c pass on
 * variant m / (V - 1) and the c2r pass on one of the other V - 1 variants.
 * The b passes pair their forward and inverse variants the same way.
 * hartree_plan_autotune times every variant on the plan's own workspace
 * (overwriting it; waits for the stream; not capturable) and keeps the
 * fastest, each pass of a pair on its own; choice[3] (host, may be NULL)
 * receives the picks.  hartree_plan_set_variants applies picks saved
 * earlier (e.g. from a cache); out-of-range picks return HARTREE_ERR_INVALID.
 * Variants 0..2 apply the same operations to each element, so V_H is
 * identical across them; the radix-32 variants round differently; every
 * variant stays within the precision's tolerance.
 */
int hartree_plan_autotune(hartree_plan plan, void* stream, int* choice);
int hartree_plan_set_variants(hartree_plan plan, const int* choice);

/* ---------------------------------------------------------------- batched cells */

/*
 * Many independent cells (different grids, cells and atom counts), each the
 * operation of hartree_solve (Sec. 2.1 density, Poisson solve and E_H; the
 * five transform passes of Sec. 3.2.4), in ONE persistent kernel launch.  All
 * cells' work items (atom preparation, splat tiles, the tiles of each
 * transform pass, the E_H sum) form one queue ordered stage by stage; resident
 * CTAs take items from it and wait, with a bounded spin, until the previous
 * stage of the same cell is complete.  Small cells no longer leave most SMs
 * idle, and a batch costs one launch instead of about ten per cell.
 *
 * hartree_batch_create
 *   descs        host [n_cells] descriptors; precision must be HARTREE_FP32
 *                (each is validated as by hartree_plan_create; max_atoms is
 *                replaced by atom_counts[c])
 *   atom_counts  host [n_cells] atoms per cell, >= 0
 *   out          host pointer receiving the batch.  Allocates one workspace
 *                per cell plus the queue; HARTREE_ERR_OOM if it does not fit.
 * hartree_batch_offsets
 *   grid_off     host [n_cells + 1] out: first element of cell c in the
 *                concatenated grid buffer (C order [N1][N2][N3] per cell);
 *                grid_off[n_cells] is the total element count
 *   atom_off     host [n_cells + 1] out: first atom of cell c in pos / q
 * hartree_solve_batched
 *   pos, q       device [sum atoms][3] / [sum atoms] doubles, cells concatenated
 *   vh           device float [grid_off[n_cells]]: receives V_H of every cell
 *                (also the density's scratch: the splat writes rho there first)
 *   eh           device double [n_cells]: E_H of every cell
 *   Enqueues two small memsets and one kernel; allocates nothing; can be
 *   captured in a CUDA graph.  Results equal those of a plan solve of each
 *   cell within the FP32 tolerance (the same per-element operations; only
 *   the E_H partial sums are grouped differently).
 * hartree_batch_device_status
 *   Synchronises the device; HARTREE_ERR_TIMEOUT if a dependency wait gave
 *   up since the last call (the results of that launch are incomplete), else
 *   HARTREE_OK.  Clears the error word.
 */
int hartree_batch_create(const hartree_desc* descs, const int* atom_counts, int n_cells, hartree_batch* out);
void hartree_batch_destroy(hartree_batch batch);
int hartree_batch_offsets(hartree_batch batch, long long* grid_off, int* atom_off);
int hartree_solve_batched(hartree_batch batch, const double* pos, const double* q, void* vh, double* eh,
                          void* stream);
int hartree_batch_device_status(hartree_batch batch);

/*
 * Fault injection for the bounded dependency waits of hartree_solve_batched
 * (the paper has no counterpart; it exists so that the timeout path can be
 * exercised on a shared GPU without hanging or faulting it).  Off by default.
 *   skip_stage  -1: off.  0..8: in every later hartree_solve_batched, item 0
 *               of that stage of cell skip_cell does its work but never counts
 *               itself done, so the items of the next stage of that cell wait
 *               for it until their limit runs out, give up, and set the
 *               batch's error word (hartree_batch_device_status then returns
 *               HARTREE_ERR_TIMEOUT and that launch's results are incomplete).
 *               Stages: 0 atom preparation, 1 Gaussian factors, 2 leaf boxes,
 *               3 splat, 4 c pass, 5 b pass, 6 a pass with Green and E_H,
 *               7 b inverse, 8 c inverse (9, the E_H sum, has no successor).
 *   skip_cell   the cell, in [0, n_cells), when skip_stage >= 0
 *   spin_limit  probes (each about 64 ns apart) a dependency wait makes before
 *               it gives up; 0 restores the default (2^26, seconds).  A short
 *               limit keeps an injected timeout to milliseconds.
 * No device work; HARTREE_ERR_INVALID for a stage or cell out of range.
 */
int hartree_batch_fault_inject(hartree_batch batch, int skip_stage, int skip_cell, unsigned spin_limit);

/* ---------------------------------------------------------------- no device allocation */

/*
 * hartree_solve_density without a plan and without allocating device memory.
 * The paper has no counterpart; this exists for callers that cannot call
 * cudaMalloc -- applications that give all device memory to their own
 * allocator or pool up front, and code paths where a device allocation is not
 * allowed or would stall other work.  Creating a plan allocates its
 * workspace; this call instead uses a fixed 8 MiB scratch array that the
 * library declares at file scope, which every GPU that loads the library
 * holds until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   desc  host pointer: grid, cell and precision (HARTREE_FP64 or HARTREE_FP32;
 *         sigma, cutoff, atoms_per_leaf and max_atoms are ignored).  The grid
 *         must fit the scratch: the half spectrum N1 N2 ceil16(N3/2 + 1) x 8
 *         bytes (FP32; ceil8(N3/2 + 1) x 16 bytes in FP64) plus small tables
 *         must stay within 8 MiB, e.g. 120^3 in FP32 or 64^3 in FP64; larger
 *         grids return HARTREE_ERR_UNSUPPORTED_SIZE before any device work.
 *   rho, vh, eh  as in hartree_solve_density (eh may be NULL).
 * The first call on each device looks up the scratch array's address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the array and leaves the
 * last call's contents in it, so calls that overlap on the GPU (two streams,
 * two host threads) race: serialise them.  Results match
 * hartree_solve_density within the precision's tolerance.
 */
int hartree_solve_density_noalloc(const hartree_desc* desc, const void* rho, void* vh, double* eh, void* stream);

/* ---------------------------------------------------------------- errors */

const char* hartree_status_string(int status);
const char* hartree_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HARTREE_H */
