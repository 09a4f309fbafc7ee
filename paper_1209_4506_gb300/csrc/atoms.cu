// atoms.cu -- density splat (structure A -> B of Sec. 3.2.2) and the adjoint
// force gather.
//
// The splat is a gather: each CTA owns one grid tile of 8 x 8 x 32 points and
// pulls the atoms whose cutoff box reaches it.  Atoms are grouped into leaves
// of `apl` consecutive atoms; in the order produced by the modified recursive
// bisection (Sec. 3.1) a leaf is a compact cluster, so a tile meets a few
// leaves, i.e. a few contiguous atom ranges.  Leaf boxes (structure C of
// Sec. 3.2.2, the parallelepiped around a process's atoms) are rebuilt from
// the positions on every call.  The Gaussian of an orthorhombic cell
// factorises over axes, images included:
//   sum_T exp(-|r - R - T|^2/s^2) = prod_d sum_{m_d} exp(-(x_d - X_d - m_d L_d)^2/s^2),
// so each (atom, tile) pair costs 8 + 8 + 32 one-dimensional factors and one
// FMA per grid point.  Atom-to-grid offsets are taken in FP64 and only the
// small offset is rounded to the working precision.
//
// The force gather walks each atom's cutoff box (unwrapped indices, so every
// periodic image is visited once) and accumulates
//   sum_r V(r) f(x) f(y) f(z)            -> phi_i = dE_H/dq_i
//   sum_r V(r) f'(x) f(y) f(z)  (etc.)   -> F_i = -dE_H/dR_i
// with f(d) = exp(-d^2/s^2), f'(d) = d exp(-d^2/s^2).  Partial sums per
// (atom, slab) go to FP64 workspace and are reduced in a fixed order.
#include "internal.cuh"

namespace hartree {

namespace {

constexpr int TA = 8, TB = 8, TC = 32;  // splat tile
constexpr int kBatch = 64;              // atoms whose factors are staged at once

__device__ __forceinline__ long long wrapi(long long i, int n) {
    long long r = i % n;
    return r < 0 ? r + n : r;
}

// Periodic overlap of [lo, hi] (unwrapped, any position) with [t0, t1].
__device__ __forceinline__ bool overlap1(double lo, double hi, double t0, double t1, double L) {
    if (hi - lo >= L) return true;
    const double m = ceil((t0 - hi) / L);
    return lo + m * L <= t1;
}

__global__ void k_leaf_boxes(const double* __restrict__ pos, int n, int apl, int nleaves, double L1, double L2,
                             double L3, double* __restrict__ box) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nleaves) return;
    const int i0 = l * apl, i1 = min(n, i0 + apl);
    const double Ls[3] = {L1, L2, L3};
    double x0[3], lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        x0[d] = pos[3 * i0 + d];
        lo[d] = 0.0;
        hi[d] = 0.0;
    }
    for (int i = i0 + 1; i < i1; ++i)
        for (int d = 0; d < 3; ++d) {
            double dd = pos[3 * i + d] - x0[d];
            dd -= Ls[d] * rint(dd / Ls[d]);  // minimum image relative to the leaf's first atom
            lo[d] = fmin(lo[d], dd);
            hi[d] = fmax(hi[d], dd);
        }
    for (int d = 0; d < 3; ++d) {
        box[6 * l + d] = x0[d] + lo[d];
        box[6 * l + 3 + d] = x0[d] + hi[d];
    }
}

// sum over images m of exp(-(x - X - m L)^2 / s^2), |x - X - m L| <= rc
template <typename T>
__device__ __forceinline__ T image_factor(double x, double X, double L, double rc, T inv_s2) {
    double D = x - X;
    const double mlo = ceil((D - rc) / L), mhi = floor((D + rc) / L);
    T f = T(0);
    for (double m = mlo; m <= mhi; m += 1.0) {
        const T d = (T)(D - m * L);
        f += exp(-d * d * inv_s2);
    }
    return f;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_splat(AtomArgs<T> a, T* __restrict__ rho, int tiles_b, int tiles_c) {
    __shared__ int leaf_list[kThreads];
    __shared__ int cand[kThreads];
    __shared__ int warp_cnt[kThreads / 32];
    __shared__ int n_leaf, n_cand;
    __shared__ T fa[kBatch][TA], fb[kBatch][TB], fc[kBatch][TC];

    const int tile = blockIdx.x;
    const int ta = tile / (tiles_b * tiles_c);
    const int tb = (tile / tiles_c) % tiles_b;
    const int tc = tile % tiles_c;
    const int a0 = ta * TA, b0 = tb * TB, c0 = tc * TC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // tile extent in Bohr (grid points a0 .. a0+TA-1 etc.)
    const double ta0 = a0 * a.h1, ta1 = (min(a0 + TA, a.n1) - 1) * a.h1;
    const double tb0 = b0 * a.h2, tb1 = (min(b0 + TB, a.n2) - 1) * a.h2;
    const double tc0 = c0 * a.h3, tc1 = (min(c0 + TC, a.n3) - 1) * a.h3;
    const T inv_s2 = (T)a.inv_s2;

    T acc[TA];
#pragma unroll
    for (int i = 0; i < TA; ++i) acc[i] = T(0);

    for (int lbase = 0; lbase < a.nleaves; lbase += kThreads) {
        // ---- leaves of this chunk whose inflated box reaches the tile (ordered compaction)
        const int l = lbase + threadIdx.x;
        bool hit = false;
        if (l < a.nleaves) {
            const double* bx = a.leaf_box + 6 * l;
            hit = overlap1(bx[0] - a.rc, bx[3] + a.rc, ta0, ta1, a.L1) &&
                  overlap1(bx[1] - a.rc, bx[4] + a.rc, tb0, tb1, a.L2) &&
                  overlap1(bx[2] - a.rc, bx[5] + a.rc, tc0, tc1, a.L3);
        }
        unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                const int c = warp_cnt[w];
                warp_cnt[w] = s;
                s += c;
            }
            n_leaf = s;
        }
        __syncthreads();
        if (hit) leaf_list[warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u))] = l;
        __syncthreads();
        const int nlf = n_leaf;
        // ---- candidate atoms of those leaves, kThreads at a time
        const int ncand_total = nlf * a.apl;
        for (int cbase = 0; cbase < ncand_total; cbase += kThreads) {
            const int c = cbase + threadIdx.x;
            int atom = -1;
            if (c < ncand_total) {
                const int lf = leaf_list[c / a.apl];
                const int i = lf * a.apl + (c % a.apl);
                if (i < a.n) {
                    const double X = a.pos[3 * i], Y = a.pos[3 * i + 1], Z = a.pos[3 * i + 2];
                    if (overlap1(X - a.rc, X + a.rc, ta0, ta1, a.L1) && overlap1(Y - a.rc, Y + a.rc, tb0, tb1, a.L2) &&
                        overlap1(Z - a.rc, Z + a.rc, tc0, tc1, a.L3))
                        atom = i;
                }
            }
            const bool ok = atom >= 0;
            bal = __ballot_sync(0xffffffffu, ok);
            __syncthreads();  // previous users of warp_cnt / cand are done
            if (lane == 0) warp_cnt[warp] = __popc(bal);
            __syncthreads();
            if (threadIdx.x == 0) {
                int s = 0;
                for (int w = 0; w < kThreads / 32; ++w) {
                    const int cc = warp_cnt[w];
                    warp_cnt[w] = s;
                    s += cc;
                }
                n_cand = s;
            }
            __syncthreads();
            if (ok) cand[warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u))] = atom;
            __syncthreads();
            const int nc = n_cand;
            // ---- factors for batches of kBatch atoms, then accumulate
            for (int bb = 0; bb < nc; bb += kBatch) {
                const int nb = min(kBatch, nc - bb);
                for (int e = threadIdx.x; e < nb * (TA + TB + TC); e += kThreads) {
                    const int t = e / (TA + TB + TC), f = e - t * (TA + TB + TC);
                    const int i = cand[bb + t];
                    if (f < TA) {
                        fa[t][f] = image_factor<T>((a0 + f) * a.h1, a.pos[3 * i], a.L1, a.rc, inv_s2);
                    } else if (f < TA + TB) {
                        fb[t][f - TA] = image_factor<T>((b0 + f - TA) * a.h2, a.pos[3 * i + 1], a.L2, a.rc, inv_s2);
                    } else {
                        const int k = f - TA - TB;
                        const T qn = (T)(a.q[i] * a.norm);
                        fc[t][k] = qn * image_factor<T>((c0 + k) * a.h3, a.pos[3 * i + 2], a.L3, a.rc, inv_s2);
                    }
                }
                __syncthreads();
                for (int t = 0; t < nb; ++t) {
                    const T s = fb[t][warp] * fc[t][lane];
#pragma unroll
                    for (int i = 0; i < TA; ++i) acc[i] += fa[t][i] * s;
                }
                __syncthreads();
            }
        }
    }
    const int b = b0 + warp, c = c0 + lane;
    if (b < a.n2 && c < a.n3) {
#pragma unroll
        for (int i = 0; i < TA; ++i) {
            const int ia = a0 + i;
            if (ia < a.n1) rho[((long long)ia * a.n2 + b) * a.n3 + c] = acc[i];
        }
    }
}

// ---------------------------------------------------------------- forces
// Dynamic shared memory: f0[3][cmax] = exp(-d^2/s^2), f1[3][cmax] = d exp(-d^2/s^2).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_forces(AtomArgs<T> a, const T* __restrict__ V, int slabs, int cmax,
                                                     double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* f0s = reinterpret_cast<T*>(smem_raw);
    T* f1s = f0s + 3 * cmax;
    __shared__ double red[4][kThreads / 32];
    const int atom = blockIdx.x / slabs, slab = blockIdx.x - atom * slabs;
    const double hs[3] = {a.h1, a.h2, a.h3};
    long long lo[3];
    int cnt[3];
    for (int d = 0; d < 3; ++d) {
        const double X = a.pos[3 * atom + d];
        lo[d] = (long long)ceil((X - a.rc) / hs[d]);
        const long long hi = (long long)floor((X + a.rc) / hs[d]);
        cnt[d] = (int)max(0LL, min((long long)cmax, hi - lo[d] + 1));
    }
    const T inv_s2 = (T)a.inv_s2;
    for (int d = 0; d < 3; ++d)
        for (int i = threadIdx.x; i < cnt[d]; i += blockDim.x) {
            const T dd = (T)((double)(lo[d] + i) * hs[d] - a.pos[3 * atom + d]);
            const T g = exp(-dd * dd * inv_s2);
            f0s[d * cmax + i] = g;
            f1s[d * cmax + i] = dd * g;
        }
    __syncthreads();
    const int ia0 = (int)((long long)cnt[0] * slab / slabs), ia1 = (int)((long long)cnt[0] * (slab + 1) / slabs);
    const int nrows = (ia1 - ia0) * cnt[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sp = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    T bp = T(0), bx = T(0), by = T(0), bz = T(0);
    int rows_in_block = 0;
    for (int r = warp; r < nrows; r += kThreads / 32) {
        const int i = ia0 + r / cnt[1], j = r % cnt[1];
        const long long gi = wrapi(lo[0] + i, a.n1), gj = wrapi(lo[1] + j, a.n2);
        const T* row = V + (gi * a.n2 + gj) * a.n3;
        const T w0 = f0s[i] * f0s[cmax + j];
        const T wx = f1s[i] * f0s[cmax + j];
        const T wy = f0s[i] * f1s[cmax + j];
        T rp = T(0), rx = T(0), ry = T(0), rz = T(0);
        for (int k = lane; k < cnt[2]; k += 32) {
            const T v = row[wrapi(lo[2] + k, a.n3)];
            rp += v * f0s[2 * cmax + k];
            rz += v * f1s[2 * cmax + k];
        }
        bp += w0 * rp;
        bx += wx * rp;
        by += wy * rp;
        bz += w0 * rz;
        if (++rows_in_block == 8) {  // flush the short working-precision sums into FP64
            sp += (double)bp;
            sx += (double)bx;
            sy += (double)by;
            sz += (double)bz;
            bp = bx = by = bz = T(0);
            rows_in_block = 0;
        }
    }
    sp += (double)bp;
    sx += (double)bx;
    sy += (double)by;
    sz += (double)bz;
    double v4[4] = {sp, sx, sy, sz};
    for (int c = 0; c < 4; ++c) {
        double v = v4[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
        part[(long long)blockIdx.x * 4 + threadIdx.x] = s;
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
AtomArgs<T> make_atom_args(const Plan& p, const double* pos, const double* q, int n) {
    AtomArgs<T> a;
    a.n1 = p.n[0];
    a.n2 = p.n[1];
    a.n3 = p.n[2];
    a.h1 = p.h[0];
    a.h2 = p.h[1];
    a.h3 = p.h[2];
    a.L1 = p.L[0];
    a.L2 = p.L[1];
    a.L3 = p.L[2];
    a.rc = p.rc;
    a.inv_s2 = 1.0 / (p.sigma * p.sigma);
    a.norm = pow(3.14159265358979323846 * p.sigma * p.sigma, -1.5);
    a.dV = p.dV;
    a.pos = pos;
    a.q = q;
    a.n = n;
    a.apl = p.apl;
    a.nleaves = (n + p.apl - 1) / p.apl;
    a.leaf_box = p.leaf_box;
    return a;
}

template <typename T>
cudaError_t splat_impl(const Plan& p, const double* pos, const double* q, int n, void* rho, cudaStream_t s) {
    AtomArgs<T> a = make_atom_args<T>(p, pos, q, n);
    if (a.nleaves > 0)
        k_leaf_boxes<<<(a.nleaves + 127) / 128, 128, 0, s>>>(pos, n, p.apl, a.nleaves, p.L[0], p.L[1], p.L[2],
                                                             p.leaf_box);
    const int tA = (p.n[0] + TA - 1) / TA, tB = (p.n[1] + TB - 1) / TB, tC = (p.n[2] + TC - 1) / TC;
    k_splat<T><<<(unsigned)tA * tB * tC, kThreads, 0, s>>>(a, static_cast<T*>(rho), tB, tC);
    return cudaGetLastError();
}

template <typename T>
cudaError_t forces_impl(const Plan& p, const double* pos, const double* q, int n, const void* vh, double* f,
                        double* phi, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    AtomArgs<T> a = make_atom_args<T>(p, pos, q, n);
    int slabs = (4 * 152 * 2 + n - 1) / n;  // enough CTAs to cover the GPU
    if (slabs > p.max_force_slabs) slabs = p.max_force_slabs;
    if (slabs < 1) slabs = 1;
    const size_t smem = 2 * 3 * (size_t)p.box_max * sizeof(T);
    k_forces<T><<<(unsigned)n * slabs, kThreads, smem, s>>>(a, static_cast<const T*>(vh), slabs, p.box_max,
                                                             p.force_partials);
    k_forces_finalize<<<(n + 127) / 128, 128, 0, s>>>(p.force_partials, n, slabs, q, p.dV, a.norm, a.inv_s2, f, phi);
    return cudaGetLastError();
}

template <typename T>
cudaError_t configure_atoms(int max_smem) {
    return cudaFuncSetAttribute(k_forces<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

}  // namespace

cudaError_t configure_atom_kernels(const Plan& p) {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (2 * 3 * (size_t)p.box_max * p.real_size > (size_t)max_smem) return cudaErrorInvalidConfiguration;
    return p.prec == HARTREE_FP64 ? configure_atoms<double>(max_smem) : configure_atoms<float>(max_smem);
}

cudaError_t launch_splat(const Plan& p, const double* pos, const double* q, int n, void* rho, cudaStream_t s) {
    return p.prec == HARTREE_FP64 ? splat_impl<double>(p, pos, q, n, rho, s) : splat_impl<float>(p, pos, q, n, rho, s);
}

cudaError_t launch_forces(const Plan& p, const double* pos, const double* q, int n, const void* vh, double* f,
                          double* phi, cudaStream_t s) {
    return p.prec == HARTREE_FP64 ? forces_impl<double>(p, pos, q, n, vh, f, phi, s)
                                  : forces_impl<float>(p, pos, q, n, vh, f, phi, s);
}

}  // namespace hartree
