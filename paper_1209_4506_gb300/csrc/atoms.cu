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
#include "internal.cuh"

namespace hartree {

namespace {

constexpr int TA = 16, TB = 8, TC = 32;  // splat tile (a, b, c)
constexpr int kBatch = 32;               // atoms whose factors are staged at once
constexpr int kPT = 12;                  // force gather: (b, c) points per thread held in registers

__device__ __forceinline__ int imod(int x, int n) {
    int r = x % n;
    return r < 0 ? r + n : r;
}

// Does the index range [s, s + len) taken modulo n meet [t0, t0 + tn)?
__device__ __forceinline__ bool range_hits(int s, int len, int t0, int tn, int n) {
    if (len <= 0) return false;
    if (len >= n) return true;
    const int delta = imod(t0 - s, n);
    return delta < len || delta + tn > n;
}

template <typename T>
__global__ void k_atom_prep(AtomArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double hs[3] = {a.h1, a.h2, a.h3};
    const double Ls[3] = {a.L1, a.L2, a.L3};
    AtomPrep<T> p;
    for (int d = 0; d < 3; ++d) {
        double X = a.pos[3 * i + d];
        X -= Ls[d] * floor(X / Ls[d]);  // any image of the atom gives the same periodic sum
        const double lo = ceil((X - a.rc) / hs[d]);
        const double hi = floor((X + a.rc) / hs[d]);
        p.lo[d] = (int)lo;
        p.cnt[d] = hi >= lo ? min((int)(hi - lo) + 1, a.fb) : 0;
        const double D0 = lo * hs[d] - X;
        p.dh[d] = (T)D0;
        p.dl[d] = (T)(D0 - (double)p.dh[d]);
    }
    p.qn = (T)(a.q[i] * a.norm);
    a.prep[i] = p;
}

// One thread per (atom, axis, run of kRun box points): fac / dfac computed in
// FP64.  FP32 plans start each run with three exponentials and continue with
// the exact ratio recurrence; FP64 plans evaluate every point directly.
constexpr int kRun = 8;

template <typename T>
__global__ void k_atom_factors(AtomArgs<T> a) {
    const int runs = (a.fb + kRun - 1) / kRun;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3LL * a.n * runs) return;
    const int i = (int)(t / (3 * runs));
    const int rem = (int)(t - (long long)i * 3 * runs);
    const int d = rem / runs, m0 = (rem - d * runs) * kRun;
    const AtomPrep<T> p = a.prep[i];
    const int cnt = p.cnt[d];
    if (m0 >= cnt) return;
    const int m1 = min(cnt, m0 + kRun);
    const double h = d == 0 ? a.h1 : (d == 1 ? a.h2 : a.h3);
    const double D0 = (double)p.dh[d] + (double)p.dl[d];  // lo h - X
    T* f = a.fac + ((long long)i * 3 + d) * a.fb;
    T* df = a.dfac + ((long long)i * 3 + d) * a.fb;
    if constexpr (sizeof(T) == 8) {
        for (int m = m0; m < m1; ++m) {
            const double dm = fma((double)m, h, D0);
            const double g = exp(-dm * dm * a.inv_s2);
            f[m] = g;
            df[m] = dm * g;
        }
    } else {
        // exponent(m) = -(D0 + m h)^2 / s^2: successive ratios are exp(-(2 d_m h + h^2) / s^2)
        const double ds = fma((double)m0, h, D0);
        double g = exp(-ds * ds * a.inv_s2);
        double r = exp(-(2.0 * ds * h + h * h) * a.inv_s2);
        const double q = exp(-2.0 * h * h * a.inv_s2);
        for (int m = m0; m < m1; ++m) {
            const double dm = fma((double)m, h, D0);
            f[m] = (T)g;
            df[m] = (T)(dm * g);
            g *= r;
            r *= q;
        }
    }
}

template <typename T>
__global__ void k_leaf_boxes(const AtomPrep<T>* __restrict__ prep, int n, int apl, int nleaves, int n1, int n2,
                             int n3, int* __restrict__ leaf) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nleaves) return;
    const int i0 = l * apl, i1 = min(n, i0 + apl);
    const int ns[3] = {n1, n2, n3};
    for (int d = 0; d < 3; ++d) {
        const int lo0 = prep[i0].lo[d];
        int s = lo0, e = lo0;
        for (int i = i0; i < i1; ++i) {
            int lo = prep[i].lo[d];
            const int c = prep[i].cnt[d];
            // shift by whole periods to the image nearest the leaf's first atom
            const int diff = lo - lo0;
            const int k = (int)floorf(((float)diff + 0.5f * ns[d]) / (float)ns[d]);
            lo -= k * ns[d];
            s = min(s, lo);
            e = max(e, lo + c);
        }
        leaf[6 * l + d] = s;
        leaf[6 * l + 3 + d] = min(e - s, ns[d]);
    }
}

// Sum over the box points of one atom that land on grid index g (all images).
template <typename T>
__device__ __forceinline__ T image_sum(const T* __restrict__ f, int g, int lo, int cnt, int n) {
    T s = T(0);
    for (int m = imod(g - lo, n); m < cnt; m += n) s += f[m];
    return s;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_splat(AtomArgs<T> a, T* __restrict__ rho, int tiles_b, int tiles_c) {
    __shared__ int leaf_list[kThreads];
    __shared__ int cand[kThreads];
    __shared__ int warp_cnt[kThreads / 32];
    __shared__ int n_sel;
    __shared__ __align__(16) T fa[kBatch][TA];
    __shared__ T fb[kBatch][TB], fc[kBatch][TC];

    const int tile = blockIdx.x;
    const int ta = tile / (tiles_b * tiles_c);
    const int tb = (tile / tiles_c) % tiles_b;
    const int tc = tile % tiles_c;
    const int a0 = ta * TA, b0 = tb * TB, c0 = tc * TC;
    const int na = min(TA, a.n1 - a0), nb_ = min(TB, a.n2 - b0), nc_ = min(TC, a.n3 - c0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // ordered compaction of the threads whose flag is set; returns the count
    auto compact = [&](bool flag, int value, int* out) -> int {
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        __syncthreads();  // earlier readers of warp_cnt / n_sel / out are done
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                const int c = warp_cnt[w];
                warp_cnt[w] = s;
                s += c;
            }
            n_sel = s;
        }
        __syncthreads();
        if (flag) out[warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u))] = value;
        __syncthreads();
        return n_sel;
    };

    T acc[TA];
#pragma unroll
    for (int i = 0; i < TA; ++i) acc[i] = T(0);

    for (int lbase = 0; lbase < a.nleaves; lbase += kThreads) {
        const int l = lbase + threadIdx.x;
        bool hit = false;
        if (l < a.nleaves) {
            const int* bx = a.leaf + 6 * l;
            hit = range_hits(bx[0], bx[3], a0, na, a.n1) && range_hits(bx[1], bx[4], b0, nb_, a.n2) &&
                  range_hits(bx[2], bx[5], c0, nc_, a.n3);
        }
        const int nlf = compact(hit, l, leaf_list);
        const int ncand_total = nlf * a.apl;
        for (int cbase = 0; cbase < ncand_total; cbase += kThreads) {
            const int c = cbase + threadIdx.x;
            int atom = -1;
            if (c < ncand_total) {
                const int i = leaf_list[c / a.apl] * a.apl + (c % a.apl);
                if (i < a.n) {
                    const AtomPrep<T>& p = a.prep[i];
                    if (range_hits(p.lo[0], p.cnt[0], a0, na, a.n1) && range_hits(p.lo[1], p.cnt[1], b0, nb_, a.n2) &&
                        range_hits(p.lo[2], p.cnt[2], c0, nc_, a.n3))
                        atom = i;
                }
            }
            const int nc = compact(atom >= 0, atom, cand);
            for (int bb = 0; bb < nc; bb += kBatch) {
                const int nb = min(kBatch, nc - bb);
                for (int e = threadIdx.x; e < nb * (TA + TB + TC); e += kThreads) {
                    const int t = e / (TA + TB + TC), f = e - t * (TA + TB + TC);
                    const int i = cand[bb + t];
                    const AtomPrep<T>& p = a.prep[i];
                    const T* F = a.fac + (long long)i * 3 * a.fb;
                    if (f < TA) {
                        fa[t][f] = image_sum(F, a0 + f, p.lo[0], p.cnt[0], a.n1);
                    } else if (f < TA + TB) {
                        fb[t][f - TA] = image_sum(F + a.fb, b0 + f - TA, p.lo[1], p.cnt[1], a.n2);
                    } else {
                        const int k = f - TA - TB;
                        fc[t][k] = p.qn * image_sum(F + 2 * a.fb, c0 + k, p.lo[2], p.cnt[2], a.n3);
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
AtomArgs<T> make_atom_args(const Plan& p, const double* pos, const double* q, int n) {
    AtomArgs<T> a;
    a.n1 = p.n[0];
    a.n2 = p.n[1];
    a.n3 = p.n[2];
    a.h1 = p.h[0];
    a.h2 = p.h[1];
    a.h3 = p.h[2];
    for (int d = 0; d < 3; ++d) {
        a.hh[d] = (T)p.h[d];
        a.hl[d] = (T)(p.h[d] - (double)a.hh[d]);
    }
    a.L1 = p.L[0];
    a.L2 = p.L[1];
    a.L3 = p.L[2];
    a.rc = p.rc;
    a.inv_s2 = 1.0 / (p.sigma * p.sigma);
    a.is2h = (T)a.inv_s2;
    a.is2l = (T)(a.inv_s2 - (double)a.is2h);
    a.norm = pow(3.14159265358979323846 * p.sigma * p.sigma, -1.5);
    a.dV = p.dV;
    a.pos = pos;
    a.q = q;
    a.n = n;
    a.apl = p.apl;
    a.nleaves = (n + p.apl - 1) / p.apl;
    a.prep = static_cast<AtomPrep<T>*>(p.atom_prep);
    a.fac = static_cast<T*>(p.atom_fac);
    a.dfac = static_cast<T*>(p.atom_dfac);
    a.fb = p.box_max;
    a.leaf = p.leaf_box;
    return a;
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
