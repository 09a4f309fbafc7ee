// internal.cuh -- plan layout and launcher declarations shared by the
// library's translation units (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/hartree.h"
#include "fft_engine.cuh"

namespace hartree {

constexpr int kThreads = 256;
constexpr int kMaxAxis = 4096;       // largest grid size along one axis
constexpr int kMaxBoxPoints = 1024;  // largest per-axis extent of one atom's cutoff box (points)

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
    const T* gsqa;      // (2 pi k'/L1)^2, k' the signed frequency of k
    const T* gsqb;
    const T* gsqc;
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

// Arguments of the splat and the force gather.
template <typename T>
struct AtomArgs {
    int n1, n2, n3;
    double h1, h2, h3;
    double L1, L2, L3;
    double rc;      // per-axis truncation radius (Bohr)
    double inv_s2;  // 1 / sigma^2
    double norm;    // (pi sigma^2)^(-3/2)
    double dV;
    const double* pos;
    const double* q;
    int n;          // atoms
    int apl;        // atoms per leaf
    int nleaves;
    double* leaf_box;  // [nleaves][6]: lo xyz, hi xyz (unwrapped)
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
    void* gsq[3] = {nullptr, nullptr, nullptr};
    double* eh_partials = nullptr;
    int n_eh_partials = 0;
    double* leaf_box = nullptr;
    double* force_partials = nullptr;
    int max_force_slabs = 0;
    int box_max = 0;          // largest per-axis point count of one atom's cutoff box
    double* d_pos = nullptr;  // staging for the host step
    double* d_q = nullptr;
    double* d_f = nullptr;
    double* d_eh = nullptr;
    size_t bytes = 0;
    // tiling
    int c_lines, b_cols, a_cols;
    size_t smem_c, smem_b, smem_a;
};

// launchers (poisson.cu / atoms.cu); return cudaSuccess or the launch error
cudaError_t launch_poisson(const Plan& p, const void* rho, void* vh, double* eh, cudaStream_t s);
cudaError_t launch_splat(const Plan& p, const double* pos, const double* q, int n, void* rho, cudaStream_t s);
cudaError_t launch_forces(const Plan& p, const double* pos, const double* q, int n, const void* vh, double* f,
                          double* phi, cudaStream_t s);
cudaError_t configure_poisson_kernels(const Plan& p);
cudaError_t configure_atom_kernels(const Plan& p);

}  // namespace hartree
