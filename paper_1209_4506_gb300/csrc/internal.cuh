// internal.cuh -- plan layout and launcher declarations shared by the
// library's translation units (not part of the public C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/hartree.h"
#include "fft_engine.cuh"

namespace hartree {

constexpr int kThreads = 256;
constexpr int TA = 16, TB = 8, TC = 32;  // splat tile (a, b, c)
constexpr int kMaxAxis = 4096;       // largest grid size along one axis
constexpr int kMaxBoxPoints = 1024;  // largest per-axis extent of one atom's cutoff box (points)
constexpr int kBinCap = 64;          // atoms listed per splat tile; a fuller tile selects from the leaf boxes

// Arguments of the five Poisson passes (one precision).
template <typename T>
struct PoissonArgs {
    int n1, n2, n3;  // grid
    int M;           // N3 / 2 (length of the packed complex c transform)
    int nh;          // M + 1 half-spectrum columns
    int ldc;         // row stride of the half spectrum (complex elements)
    RadixPlan rpa, rpb, rpc;
    const cpx<T>* twa;  // exp(-2 pi i k / N1), k < N1
    const cpx<T>* twb;  // exp(-2 pi i k / N2)
    const cpx<T>* twc;  // exp(-2 pi i k / N3)   (the M-point transform uses every 2nd entry)
    const cpx<T>* gsqa;  // (2 pi k'/L1)^2 (k' the signed frequency of k) as high + low parts
    const cpx<T>* gsqb;
    const cpx<T>* gsqc;
    cpx<T>* W;          // half spectrum [N1][N2][ldc]
    T green_scale;      // 4 pi / N_tot (inverse-transform normalisation folded in)
    double* eh_partials;
    // tiling
    int c_lines;   // lines per CTA of the c passes
    int b_cols;    // columns per CTA of the b pass
    int a_cols;    // columns per CTA of the a pass
    int b_chunks;  // ceil(nh / b_cols)
    int a_chunks;  // ceil(nh / a_cols)
};

// Twiddle exp(-2 pi i k / N) as a rounded value and its remainder (zero in FP64).
template <typename T>
struct TwPair {
    cpx<T> h, l;
};

// Arguments of the specialised (compile-time radix) passes.
template <typename T>
struct FastArgs {
    int n1, n2, n3, M, nh, ldc;
    const TwPair<T>* twpa;  // N1 entries
    const TwPair<T>* twpb;  // N2 entries
    const TwPair<T>* twpc;  // N3 entries
    const cpx<T>* gsqa;
    const cpx<T>* gsqb;
    const cpx<T>* gsqc;
    cpx<T>* W;
    T green_scale;
    double* eh_partials;
    int a_chunks, b_chunks;
};

// Sum of v over the block in FP64 (fixed order); the result is valid in thread 0.
// `red` holds one double per warp.  Contains __syncthreads().
__device__ __forceinline__ double block_sum_double(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// Sum over the block of values held as (s, e) pairs (value = s + e), reduced
// inside each warp with error-free FP32 TwoSum steps and across warps in FP64.
// FP64 throughput on GB300 is a small fraction of FP32, so per-thread FP64
// shuffles would cost more than the kernel's own arithmetic.  Result valid in
// thread 0; `red` holds one double per warp.  Contains __syncthreads().
__device__ __forceinline__ double block_sum_comp(float s, float e, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, o);
        const float e2 = __shfl_down_sync(0xffffffffu, e, o);
        const float t = s + s2;
        const float bb = t - s;
        const float err = (s - (t - bb)) + (s2 - bb);
        s = t;
        e = e + e2 + err;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = (double)s + (double)e;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    return r;
}
__device__ __forceinline__ double block_sum_comp(double s, double e, double* red) {
    return block_sum_double(s + e, red);
}

// Per-atom data prepared once per call (k_atom_prep): the cutoff box of the
// atom in unwrapped grid indices and the offset of its first point, split in
// a high and a low part so FP32 kernels can form d = (lo + m) h - X to full
// FP32 accuracy without FP64 arithmetic.
template <typename T>
struct AtomPrep {
    int lo[3];   // first unwrapped grid index of the box along a, b, c
    int cnt[3];  // points of the box along a, b, c
    int st[3];   // lo mod N: the wrapped grid index of the box's first point
    T dh[3];     // lo h - X, rounded to T
    T dl[3];     // (lo h - X) - dh (zero for FP64)
    T qn;        // q (pi s^2)^(-3/2), formed in FP64 and rounded once
    T ql;        // its rounding remainder (q norm - qn): one shared rounding of every point of
                 // the atom would otherwise bias E_H by twice its relative size
};

// Arguments of the splat and the force gather.
template <typename T>
struct AtomArgs {
    int n1, n2, n3;
    double h1, h2, h3;
    T hh[3], hl[3];  // grid spacing split into high and low parts
    double L1, L2, L3;
    double rc;      // per-axis truncation radius (Bohr)
    double inv_s2;  // 1 / sigma^2
    double qr[3];   // exp(-2 h^2 / s^2) per axis: the factor by which successive box ratios fall
    T is2h, is2l;   // 1 / sigma^2 split into high and low parts
    double norm;    // (pi sigma^2)^(-3/2)
    double dV;
    const double* pos;
    const double* q;
    int n;          // atoms
    int apl;        // atoms per leaf
    int nleaves;
    AtomPrep<T>* prep;  // [n]
    T* fac;             // [n][3][fb]: exp(-d_m^2/s^2) at box point m of each axis
    T* dfac;            // [n][3][fb]: d_m exp(-d_m^2/s^2)
    int fb;             // row length of fac / dfac (largest box extent)
    int* leaf;          // [nleaves][6]: start a, b, c (unwrapped), length a, b, c (points)
    const int* order = nullptr;  // force gather: CTA -> atom (atoms by the a start of their box), or identity
};

struct Plan {
    hartree_desc desc;
    int prec;         // hartree_precision
    size_t real_size; // sizeof(float) or sizeof(double)
    int n[3];
    int M, nh, ldc;
    double L[3], h[3], rc, sigma, omega, dV;
    int apl, max_atoms, max_leaves;
    RadixPlan rp[3];  // a (N1), b (N2), c (M)
    // device workspace
    void* W = nullptr;        // half spectrum
    void* R = nullptr;        // one real grid (forces recompute, host step)
    void* tw[3] = {nullptr, nullptr, nullptr};
    void* twp[3] = {nullptr, nullptr, nullptr};  // TwPair tables
    void* gsq[3] = {nullptr, nullptr, nullptr};
    double* eh_partials = nullptr;
    int n_eh_partials = 0;
    void* atom_prep = nullptr;  // AtomPrep<T>[max_atoms]
    void* atom_fac = nullptr;   // T[max_atoms][3][box_max]
    void* atom_dfac = nullptr;  // T[max_atoms][3][box_max]
    int* leaf_box = nullptr;    // [max_leaves][6]
    double* force_partials = nullptr;
    int* force_order = nullptr;  // [max_atoms]: the force gather's CTA order (k_slab_order)
    int max_force_slabs = 0;
    int box_max = 0;          // largest per-axis point count of one atom's cutoff box
    double* d_pos = nullptr;  // staging for the host step
    double* d_q = nullptr;
    double* d_f = nullptr;
    double* d_eh = nullptr;
    // hartree_step_host: its device work captured into a CUDA graph on a stream of the plan's own
    // and replayed while the key (atom count, variant picks, forces wanted) stays the same
    cudaStream_t host_stream = nullptr;
    cudaEvent_t host_event = nullptr;
    cudaGraphExec_t host_graph = nullptr;
    int host_key[5] = {-1, -1, -1, -1, -1};
    unsigned long long host_graph_launches = 0;
    size_t bytes = 0;
    // tiling
    int c_lines, b_cols, a_cols;
    mutable unsigned long long launches = 0;  // kernels launched (host-side count)
    int use_fast = 0;
    int var[3] = {0, 0, 0};  // kernel variant of the c, b and a passes (autotuned)
    int sm_count = 0;
    int* d_err = nullptr;     // device error word (bit 0: a bounded wait timed out)
    bool tma_ok = false;      // tensor maps over W are valid
    CUtensorMap tmap_b, tmap_a;    // 16-column boxes of the TMA-streamed b and a passes
    CUtensorMap tmap_b8, tmap_a8;  // 8-column boxes
    CUtensorMap tmap_b4, tmap_a4;  // 4-column boxes
    // use_fast: bit 0: c passes, bit 1: b passes, bit 2: a pass use the specialised kernels
    size_t smem_c, smem_b, smem_a;
    // tile bins of the splat: per 16 x 8 x 32 tile up to kBinCap atoms whose cutoff box reaches it
    int tiles[3] = {0, 0, 0};   // tiles along a, b, c
    int n_tiles = 0;
    int* bin_cursor = nullptr;  // [n_tiles] atoms that reached each tile (may exceed kBinCap)
    int4* bin_list = nullptr;   // [n_tiles][kBinCap]: atom index, then st | cnt << 16 along a, b, c
    void* tc_dft = nullptr;     // HARTREE_FP32_TC_SPLIT: 16-bit split 16-point DFT operands (forward, inverse)
    void* bisect = nullptr;     // scratch of the device atom reorder (bisect_scratch_bytes(max_atoms))
};

// Let kernel `f` use all of the device's opt-in shared memory that its static
// shared memory leaves free (the attribute is per kernel, so plans of any
// size can coexist).
template <typename K>
inline cudaError_t allow_max_dynamic_smem(K* f, int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

inline cudaError_t optin_smem(int* bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return e;
}

// launchers (poisson.cu / atoms.cu); return cudaSuccess or the launch error
cudaError_t launch_poisson(const Plan& p, const void* rho, void* vh, double* eh, cudaStream_t s);
// The passes first .. 4 (the half spectrum W already holds pass first - 1's result) and E_H.
cudaError_t launch_poisson_from(const Plan& p, int first, const void* rho, void* vh, double* eh, cudaStream_t s);
cudaError_t launch_poisson_pass(const Plan& p, int pass, const void* rho, void* vh, cudaStream_t s);
// launch_splat prepares the per-atom boxes and factor arrays in the plan's workspace.
// `prepared` (forces): they already hold these very positions (an earlier launch on the same stream).
cudaError_t launch_splat(const Plan& p, const double* pos, const double* q, int n, void* rho, cudaStream_t s);
// Splat, the five passes and E_H into vh, with no density grid: through the splat fused into the
// r2c pass when the plan has it, else the splat into vh and the solve in place.
cudaError_t launch_splat_solve(const Plan& p, const double* pos, const double* q, int n, void* vh, double* eh,
                               cudaStream_t s);
// The atoms' boxes, factors and leaf boxes, then the fused splat + r2c kernel (splat_fused_available).
cudaError_t launch_splat_r2c(const Plan& p, const double* pos, const double* q, int n, cudaStream_t s);
// The fused splat + r2c kernel (FP32 plans with HARTREE_FLAG_FUSED_SPLAT and a compiled kernel
// for M): the atoms' boxes, factors and leaf boxes must be prepared.
bool splat_fused_available(const Plan& p);
cudaError_t configure_splat_fused(const Plan& p, int optin);
long long launch_r2c_splat(const Plan& p, const AtomArgs<float>& at, cudaStream_t s);
cudaError_t launch_forces(const Plan& p, const double* pos, const double* q, int n, const void* vh, double* f,
                          double* phi, cudaStream_t s, bool prepared = false);
void set_last_error(const char* msg);  // the message hartree_last_error() returns on this thread
// Grid geometry, radix plans and pass tiling of `p` from `d` (sizes already validated):
// HARTREE_OK, or HARTREE_ERR_UNSUPPORTED_SIZE with the thread's message set.
int init_plan_geometry(Plan& p, const hartree_desc& d);
bool smooth_size(int n);  // n is 2/3/5/7-smooth
cudaError_t configure_poisson_kernels(const Plan& p);
cudaError_t configure_fast_kernels(const Plan& p);
int fast_pass_mask(const Plan& p);
int fast_variants(const Plan& p, int kind);  // kind 0: c passes, 1: b passes, 2: a pass
// Pass kinds 0 (c: r2c, c2r) and 1 (b: forward, inverse) pick a variant per pass.  Their
// variant index v: below the single-pass variant count V both passes take v; V + m pairs
// the first pass's variant m / (V - 1) with one of the other V - 1 variants for the second.
int single_variants(const Plan& p, int kind);
void pair_variants(int V, int v, int* first, int* second);
int pair_index(int V, int first, int second);
int pass_variant(const Plan& p, int pass);  // the variant pass 0..4 runs under the plan's picks
void prepare_tma(Plan& p);                   // encode the tensor maps of the TMA-streamed passes
long long launch_fast_pass(const Plan& p, int pass, const void* rho, void* vh, cudaStream_t s);
cudaError_t configure_atom_kernels(const Plan& p);
// device atom reorder (reorder_dev.cu): modified recursive bisection, one launch per tree level
size_t bisect_scratch_bytes(int max_atoms);
cudaError_t configure_bisect();
cudaError_t launch_bisect(const Plan& p, const double* pos, const double* w, int n, int n_leaves, int* perm,
                          int* leaf_start, cudaStream_t s);
// paired-lane TMA column passes (pair_passes.cu), FP32: b (passes 1, 3) and a (pass 2)
int col_pair_variants(int n);
bool col_pair_available(const Plan& p, int axis);
cudaError_t configure_col_pair(const Plan& p, int optin);
long long launch_col_pair(const Plan& p, int pass, int variant, const FastArgs<float>& a, cudaStream_t s);
// tensor-core b passes of HARTREE_FP32_TC_SPLIT plans (tc_split.cu)
bool tc_split_supported(const Plan& p);
size_t tc_table_bytes();
cudaError_t upload_tc_tables(const Plan& p);
cudaError_t configure_tc_kernels(const Plan& p);
long long launch_tc_pass(const Plan& p, int pass, cudaStream_t s);

}  // namespace hartree

// The opaque handle of the C ABI.
struct hartree_plan_s {
    hartree::Plan p;
};
