// atoms.cu -- density splat (structure A -> B of Sec. 3.2.2) and the adjoint
// force gather.
//
// Atom i is the Gaussian q_i (pi s^2)^-3/2 exp(-|r - R_i|^2/s^2), truncated per
// axis at |d| <= rc.  In an orthorhombic cell the periodic sum over images
// factorises over the axes:
//   sum_T exp(-|r - R - T|^2/s^2) = prod_d sum_m exp(-(x_d - X_d - m L_d)^2/s^2),
// so every atom is described by three one-dimensional arrays over its cutoff
// box (structure A of Sec. 3.2.2): box point m of axis d is the unwrapped grid
// index lo_d + m at offset d_m = (lo_d + m) h_d - X_d, and
//   fac[m] = exp(-d_m^2/s^2),  dfac[m] = d_m exp(-d_m^2/s^2).
// k_atom_prep finds the box; k_atom_factors fills the arrays once per call in
// FP64 (three exponentials per run of 8 box points, then the exact ratio
// recurrence f_{m+1} = f_m r_m, r_{m+1} = r_m exp(-2 h^2/s^2)) and rounds each
// value once, so the FP32 splat and gather carry no exponential rounding bias.
//
// k_leaf_boxes builds, for each leaf of `apl` consecutive atoms, the integer
// box covering its atoms (structure C of Sec. 3.2.2: the parallelepiped
// around the basis spheres of the atoms one process holds).  In the order of
// the modified recursive bisection (Sec. 3.1) a leaf is a compact cluster, so
// a grid tile meets a few leaves, i.e. a few contiguous atom ranges.
//
// k_splat is a gather: each CTA owns a 16 x 8 x 32 grid tile, selects the
// leaves and then the atoms whose boxes reach it (integer tests, ordered
// compaction so the summation order is fixed), stages their factors and adds
// q n fa fb fc with one FMA per grid point and atom.
//
// k_forces walks one atom's box (or a slab of it) per CTA: each thread owns
// fixed (b, c) points with their weights in registers and streams over the a
// slices, so every load is independent of the others; the four sums
//   sum_r V f(x) f(y) f(z) -> phi_i = dE_H/dq_i,   sum_r V f'(x) f(y) f(z) ... -> F_i
// use compensated working-precision accumulators and one FP64 block
// reduction.  Per (atom, slab) partials are reduced in a fixed order.
#include "atoms_dev.cuh"

namespace hartree {

namespace {

template <typename T>
__global__ void k_atom_prep(AtomArgs<T> a) {
    atom_prep_one(a, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void k_atom_factors(AtomArgs<T> a) {
    atom_factors_one(a, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void k_leaf_boxes(const AtomPrep<T>* __restrict__ prep, int n, int apl, int nleaves, int n1, int n2,
                             int n3, int* __restrict__ leaf) {
    leaf_box_one(prep, n, apl, nleaves, n1, n2, n3, leaf, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_splat(AtomArgs<T> a, T* __restrict__ rho, int tiles_b, int tiles_c) {
    splat_tile(a, rho, tiles_b, tiles_c, blockIdx.x);
}

// ---------------------------------------------------------------- forces
template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x) {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

// Dynamic shared memory: fac[3][fb], dfac[3][fb], wrapped grid index[3][fb].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_forces(AtomArgs<T> a, const T* __restrict__ V, int slabs,
                                                     double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int fb = a.fb;
    T* f0 = reinterpret_cast<T*>(smem_raw);
    T* f1 = f0 + 3 * fb;
    int* gix = reinterpret_cast<int*>(f1 + 3 * fb);
    __shared__ double red[4][kThreads / 32];
    const int atom = blockIdx.x / slabs, slab = blockIdx.x - atom * slabs;
    const AtomPrep<T> p = a.prep[atom];
    const int ns[3] = {a.n1, a.n2, a.n3};
    const T* F = a.fac + (long long)atom * 3 * fb;
    const T* DF = a.dfac + (long long)atom * 3 * fb;
    for (int d = 0; d < 3; ++d)
        for (int m = threadIdx.x; m < p.cnt[d]; m += kThreads) {
            f0[d * fb + m] = F[d * fb + m];
            f1[d * fb + m] = DF[d * fb + m];
            gix[d * fb + m] = imod(p.lo[d] + m, ns[d]);
        }
    __syncthreads();
    const int ia0 = (int)((long long)p.cnt[0] * slab / slabs), ia1 = (int)((long long)p.cnt[0] * (slab + 1) / slabs);
    const int cc = p.cnt[2];
    const int P = p.cnt[1] * cc;  // points of one a slice
    const long long slice = (long long)a.n2 * a.n3;
    T s0 = T(0), c0 = T(0), sx = T(0), cx = T(0), sy = T(0), cy = T(0), sz = T(0), cz = T(0);
    if (P <= kThreads * kPT) {
        // (b, c) points of this thread with their weights, reused for every slice
        int off[kPT];  // offset within a slice: b n3 + c < 2^24
        T w[kPT], wy[kPT], wz[kPT];
#pragma unroll
        for (int u = 0; u < kPT; ++u) {
            const int pt = threadIdx.x + kThreads * u;
            const bool ok = pt < P;
            const int j = ok ? pt / cc : 0, k = ok ? pt - j * cc : 0;
            off[u] = gix[fb + j] * a.n3 + gix[2 * fb + k];
            w[u] = ok ? f0[fb + j] * f0[2 * fb + k] : T(0);
            wy[u] = ok ? f1[fb + j] * f0[2 * fb + k] : T(0);
            wz[u] = ok ? f0[fb + j] * f1[2 * fb + k] : T(0);
        }
        for (int i = ia0; i < ia1; ++i) {
            const T* Vs = V + gix[i] * slice;
            T v[kPT];
#pragma unroll
            for (int u = 0; u < kPT; ++u) v[u] = (threadIdx.x + kThreads * u < P) ? __ldg(Vs + off[u]) : T(0);
            T p0 = T(0), py = T(0), pz = T(0);
#pragma unroll
            for (int u = 0; u < kPT; ++u) {
                p0 += v[u] * w[u];
                py += v[u] * wy[u];
                pz += v[u] * wz[u];
            }
            kahan_add(s0, c0, f0[i] * p0);
            kahan_add(sx, cx, f1[i] * p0);
            kahan_add(sy, cy, f0[i] * py);
            kahan_add(sz, cz, f0[i] * pz);
        }
    } else {
        // wide boxes: points revisited per slice with weights from shared memory
        for (int i = ia0; i < ia1; ++i) {
            const T* Vs = V + gix[i] * slice;
            T p0 = T(0), py = T(0), pz = T(0);
            for (int pt = threadIdx.x; pt < P; pt += kThreads) {
                const int j = pt / cc, k = pt - j * cc;
                const T v = __ldg(Vs + (long long)gix[fb + j] * a.n3 + gix[2 * fb + k]);
                p0 += v * f0[fb + j] * f0[2 * fb + k];
                py += v * f1[fb + j] * f0[2 * fb + k];
                pz += v * f0[fb + j] * f1[2 * fb + k];
            }
            kahan_add(s0, c0, f0[i] * p0);
            kahan_add(sx, cx, f1[i] * p0);
            kahan_add(sy, cy, f0[i] * py);
            kahan_add(sz, cz, f0[i] * pz);
        }
    }
    // four block sums: error-free FP32 warp steps, FP64 only across warps
    const T vs[4] = {s0, sx, sy, sz}, ve[4] = {-c0, -cx, -cy, -cz};
    for (int c = 0; c < 4; ++c) {
        const double tot = block_sum_comp(vs[c], ve[c], red[c]);
        if (threadIdx.x == 0) part[(long long)blockIdx.x * 4 + c] = tot;
    }
}

__global__ void k_forces_finalize(const double* __restrict__ part, int n, int slabs, const double* __restrict__ q,
                                  double dV, double norm, double inv_s2, double* __restrict__ f,
                                  double* __restrict__ phi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int sl = 0; sl < slabs; ++sl)
        for (int c = 0; c < 4; ++c) s[c] += part[((long long)i * slabs + sl) * 4 + c];
    // d/dX exp(-(x-X)^2/s^2) = 2 (x - X)/s^2 exp(...);  F = -dE/dX
    const double cf = -dV * q[i] * norm * 2.0 * inv_s2;
    f[3 * i + 0] = cf * s[1];
    f[3 * i + 1] = cf * s[2];
    f[3 * i + 2] = cf * s[3];
    if (phi) phi[i] = dV * norm * s[0];
}


template <typename T>
cudaError_t prep_atoms(const Plan& p, const AtomArgs<T>& a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    p.launches += 2;
    k_atom_prep<T><<<(a.n + 127) / 128, 128, 0, s>>>(a);
    const long long nt = 3LL * a.n * ((a.fb + kRun - 1) / kRun);
    k_atom_factors<T><<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t splat_prepared(const Plan& p, const AtomArgs<T>& a, void* rho, cudaStream_t s) {
    p.launches += (a.nleaves > 0 ? 1 : 0) + 1;
    if (a.nleaves > 0)
        k_leaf_boxes<T><<<(a.nleaves + 127) / 128, 128, 0, s>>>(a.prep, a.n, p.apl, a.nleaves, p.n[0], p.n[1],
                                                                p.n[2], p.leaf_box);
    const int tA = (p.n[0] + TA - 1) / TA, tB = (p.n[1] + TB - 1) / TB, tC = (p.n[2] + TC - 1) / TC;
    k_splat<T><<<(unsigned)tA * tB * tC, kThreads, 0, s>>>(a, static_cast<T*>(rho), tB, tC);
    return cudaGetLastError();
}

template <typename T>
cudaError_t splat_impl(const Plan& p, const double* pos, const double* q, int n, void* rho, bool prepared,
                       cudaStream_t s) {
    AtomArgs<T> a = make_atom_args<T>(p, pos, q, n);
    if (!prepared) {
        cudaError_t e = prep_atoms<T>(p, a, s);
        if (e != cudaSuccess) return e;
    }
    return splat_prepared<T>(p, a, rho, s);
}

size_t forces_smem(const Plan& p, size_t real_size) { return 3 * (size_t)p.box_max * (2 * real_size + sizeof(int)); }

template <typename T>
cudaError_t forces_impl(const Plan& p, const double* pos, const double* q, int n, const void* vh, double* f,
                        double* phi, bool prepared, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    AtomArgs<T> a = make_atom_args<T>(p, pos, q, n);
    if (!prepared) {
        cudaError_t e = prep_atoms<T>(p, a, s);
        if (e != cudaSuccess) return e;
    }
    p.launches += 2;
    int slabs = (4 * 152 * 2 + n - 1) / n;  // enough CTAs to cover the GPU
    if (slabs > p.max_force_slabs) slabs = p.max_force_slabs;
    if (slabs < 1) slabs = 1;
    k_forces<T><<<(unsigned)n * slabs, kThreads, forces_smem(p, sizeof(T)), s>>>(a, static_cast<const T*>(vh), slabs,
                                                                                 p.force_partials);
    k_forces_finalize<<<(n + 127) / 128, 128, 0, s>>>(p.force_partials, n, slabs, q, p.dV, a.norm, a.inv_s2, f, phi);
    return cudaGetLastError();
}

template <typename T>
cudaError_t configure_atoms(int optin) {
    return allow_max_dynamic_smem(k_forces<T>, optin);
}

}  // namespace

cudaError_t configure_atom_kernels(const Plan& p) {
    int optin = 0;
    cudaError_t e = optin_smem(&optin);
    if (e != cudaSuccess) return e;
    if (forces_smem(p, p.real_size) + 1024 > (size_t)optin) return cudaErrorInvalidConfiguration;
    return p.prec == HARTREE_FP64 ? configure_atoms<double>(optin) : configure_atoms<float>(optin);
}

cudaError_t launch_splat(const Plan& p, const double* pos, const double* q, int n, void* rho, cudaStream_t s,
                         bool prepared) {
    return p.prec == HARTREE_FP64 ? splat_impl<double>(p, pos, q, n, rho, prepared, s)
                                  : splat_impl<float>(p, pos, q, n, rho, prepared, s);
}

cudaError_t launch_forces(const Plan& p, const double* pos, const double* q, int n, const void* vh, double* f,
                          double* phi, cudaStream_t s, bool prepared) {
    return p.prec == HARTREE_FP64 ? forces_impl<double>(p, pos, q, n, vh, f, phi, prepared, s)
                                  : forces_impl<float>(p, pos, q, n, vh, f, phi, prepared, s);
}

}  // namespace hartree
