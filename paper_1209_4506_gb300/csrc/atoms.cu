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
// k_leaf_setup runs one CTA per leaf of `apl` consecutive atoms: it finds each
// atom's box and fills its factor arrays once per call, each value rounded once
// to the working precision, so the FP32 splat and gather carry no exponential
// rounding bias (FP64 plans: an FP64 exponential per point; FP32 plans: two FP64
// exponentials per run of up to 64 points, then the exact ratio recurrence
// f_{m+1} = f_m r_m, r_{m+1} = r_m exp(-2 h^2/s^2) in float-float).  It then
// builds the leaf's box (structure C of Sec. 3.2.2: the parallelepiped around
// the basis spheres of the atoms one process holds) and lists each atom in every
// splat tile its box reaches.  In the order of the modified recursive bisection
// (Sec. 3.1) a leaf is a compact cluster, so a tile meets a few leaves, i.e. a
// few contiguous atom ranges.
//
// k_splat_binned is a gather: each CTA owns a 16 x 8 x 32 grid tile, takes the
// atoms listed for it in increasing index (or selects them from the leaf boxes
// when the list overflowed), stages their factors and adds q n fa fb fc with
// one FMA per grid point and atom.
//
// k_forces walks one atom's box (or a slab of it) per CTA: each thread owns
// fixed (b, c) points with their weights in registers and streams over the a
// slices, so every load is independent of the others; the four sums
//   sum_r V f(x) f(y) f(z) -> phi_i = dE_H/dq_i,   sum_r V f'(x) f(y) f(z) ... -> F_i
// use compensated working-precision accumulators and one FP64 block
// reduction.  Per (atom, slab) partials are reduced in a fixed order.
#include <algorithm>
#include <climits>

#include "atoms_dev.cuh"
#include "tma.cuh"

namespace hartree {

namespace {

// One CTA per leaf (apl consecutive atoms in bisection order): the atoms' boxes
// and factor arrays; the leaf's box (structure C of Sec. 3.2.2: the box around
// the cutoff boxes of the leaf's atoms, each shifted to the periodic image
// nearest the leaf's first atom; the fused splat selects atoms through these);
// and, with `bins`, each atom appended to the
// list of every splat tile its box reaches.  A list entry carries the atom's
// wrapped box start and length per axis, so the splat reads the factors with no
// further lookup.  Slots are taken with atomics, so a list is unordered (the
// splat sorts it); a tile reached by more than kBinCap atoms keeps counting and
// the splat then selects its atoms from the leaf boxes instead.
// One thread per (atom, axis) finds that axis's box and goes straight on to the
// factors of its first run, so the FP64 divisions and exponentials of the three
// axes run side by side; 128-thread CTAs let several leaves share an SM and
// cover each other's FP64 latency.
constexpr int kSetupThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kSetupThreads) k_leaf_setup(AtomArgs<T> a, int tA, int tB, int tC,
                                                             int* __restrict__ cursor, int4* __restrict__ list,
                                                             bool bins) {
    __shared__ int bmin[3], bmax[3];
    const int l = blockIdx.x;
    const int i0 = l * a.apl, i1 = min(a.n, i0 + a.apl);
    const int na = i1 - i0;
    if (threadIdx.x < 3) {
        bmin[threadIdx.x] = INT_MAX;
        bmax[threadIdx.x] = INT_MIN;
    }
    for (int t = threadIdx.x; t < 3 * na; t += blockDim.x) {
        const int i = i0 + t / 3, d = t - (t / 3) * 3;
        const AxisBox b = atom_axis_box(a, i, d);
        AtomPrep<T>& p = a.prep[i];
        const T dh = (T)b.D0, dl = (T)(b.D0 - (double)dh);
        p.lo[d] = b.lo;
        p.st[d] = b.st;
        p.cnt[d] = b.cnt;
        p.dh[d] = dh;
        p.dl[d] = dl;
        if (d == 0) {
            const double qn = a.q[i] * a.norm;
            p.qn = (T)qn;
            p.ql = (T)(qn - (double)p.qn);
        }
        atom_factors_run(a, i, d, 0, b.cnt, (double)dh + (double)dl);
    }
    __syncthreads();  // the boxes are visible to the whole CTA
    // the later runs of boxes longer than one run
    const int later = (a.fb + kRun<T>() - 1) / kRun<T>() - 1;
    for (int t = threadIdx.x; t < na * 3 * later; t += blockDim.x) {
        const int i = i0 + t / (3 * later), rem = t - (t / (3 * later)) * 3 * later;
        const int d = rem / later, run = 1 + rem - d * later;
        const AtomPrep<T>& p = a.prep[i];
        atom_factors_run(a, i, d, run * kRun<T>(), p.cnt[d], (double)p.dh[d] + (double)p.dl[d]);
    }
    const int ns[3] = {a.n1, a.n2, a.n3};
    for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            int lo = a.prep[i].lo[d];
            const int x = lo - a.prep[i0].lo[d] + ns[d] / 2;
            const int k = x >= 0 ? x / ns[d] : -((-x + ns[d] - 1) / ns[d]);  // floor(x / n)
            lo -= k * ns[d];
            atomicMin(&bmin[d], lo);
            atomicMax(&bmax[d], lo + a.prep[i].cnt[d]);
        }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        a.leaf[6 * l + d] = bmin[d];
        a.leaf[6 * l + 3 + d] = min(bmax[d] - bmin[d], ns[d]);
    }
    if (!bins) return;
    // one warp per atom appends it to its tiles' lists
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int i = i0 + (int)(threadIdx.x >> 5); i < i1; i += nwarps) bin_atom(a, i, tA, tB, tC, cursor, list, lane, 32);
}

// Splat of one tile from its bin: the list is sorted by atom index in shared
// memory (a rank sort; indices in a list are distinct), so the summation order
// is that of the leaf-selecting splat, then factors are staged in batches and
// accumulated as there.  Longer lists take the leaf-selecting path.  The same
// steps as splat_tile_binned (the batched form's), written out here over static
// shared arrays: behind the function's pointers this kernel ran 5% slower.
// Grid (tiles along c, b, a); FULL: every tile lies inside the grid (TA | N1, TB | N2, TC | N3).
template <typename T, bool FULL>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 8 : 4)
    k_splat_binned(AtomArgs<T> a, T* __restrict__ rho, const int* __restrict__ cursor,
                   const int4* __restrict__ list) {
    __shared__ int4 ent[kBinCap];
    __shared__ int4 sorted[kBinCap];
    __shared__ __align__(16) T fa[kBatch][TA];
    __shared__ T fb[kBatch][TB], fc[kBatch][TC];
    const int tiles_c = gridDim.x, tiles_b = gridDim.y;
    const int tc = blockIdx.x, tb = blockIdx.y, ta = blockIdx.z;
    const int tile = (ta * tiles_b + tb) * tiles_c + tc;
    const int L = cursor[tile];
    if (L > kBinCap) {
        splat_tile(a, rho, tiles_b, tiles_c, tile);
        return;
    }
    for (int e = threadIdx.x; e < L; e += kThreads) ent[e] = list[(long long)tile * kBinCap + e];
    __syncthreads();
    for (int e = threadIdx.x; e < L; e += kThreads) {
        const int4 v = ent[e];
        int r = 0;
        for (int f = 0; f < L; ++f) r += ent[f].x < v.x;
        sorted[r] = v;
    }
    const int a0 = ta * TA, b0 = tb * TB, c0 = tc * TC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T acc[TA];
#pragma unroll
    for (int i = 0; i < TA; ++i) acc[i] = T(0);
    for (int bb = 0; bb < L; bb += kBatch) {
        const int nb = min(kBatch, L - bb);
        __syncthreads();  // sorted[] complete / previous batch consumed
        // factors: one global load per staged value (the entry carries the box), plus q n per c value
        for (int e = threadIdx.x; e < nb * TC; e += kThreads) {
            const int t = e / TC, k = e - t * TC;
            const int4 E = sorted[bb + t];
            const T sc = FULL || c0 + k < a.n3 ? image_sum(a.fac + ((long long)E.x * 3 + 2) * a.fb, c0 + k,
                                                           E.w & 0xffff, E.w >> 16, a.n3)
                                               : T(0);
            const AtomPrep<T>& p = a.prep[E.x];
            fc[t][k] = p.qn * sc + p.ql * sc;
        }
        for (int e = threadIdx.x; e < nb * TA; e += kThreads) {
            const int t = e / TA, f = e - t * TA;
            const int4 E = sorted[bb + t];
            fa[t][f] = FULL || a0 + f < a.n1
                           ? image_sum(a.fac + (long long)E.x * 3 * a.fb, a0 + f, E.y & 0xffff, E.y >> 16, a.n1)
                           : T(0);
        }
        for (int e = threadIdx.x; e < nb * TB; e += kThreads) {
            const int t = e / TB, f = e - t * TB;
            const int4 E = sorted[bb + t];
            fb[t][f] = FULL || b0 + f < a.n2 ? image_sum(a.fac + ((long long)E.x * 3 + 1) * a.fb, b0 + f,
                                                         E.z & 0xffff, E.z >> 16, a.n2)
                                             : T(0);
        }
        __syncthreads();
        for (int t = 0; t < nb; ++t) {
            const T s = fb[t][warp] * fc[t][lane];
#pragma unroll
            for (int i = 0; i < TA; ++i) acc[i] += fa[t][i] * s;
        }
    }
    const int b = b0 + warp, c = c0 + lane;
    const long long slice = (long long)a.n2 * a.n3;
    T* out = rho + a0 * slice + (long long)b * a.n3 + c;
    if (FULL) {
#pragma unroll
        for (int i = 0; i < TA; ++i) out[i * slice] = acc[i];
    } else if (b < a.n2 && c < a.n3) {
#pragma unroll
        for (int i = 0; i < TA; ++i)
            if (a0 + i < a.n1) out[i * slice] = acc[i];
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

// Vector of VW consecutive values along c, loaded with one 8- or 16-byte access.
template <typename T, int VW>
struct VecLoad;
// ld: from global memory (read-only path); lds: from shared memory (p aligned to the vector).
template <>
struct VecLoad<float, 4> {
    static __device__ __forceinline__ void ld(const float* p, float* v) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
    }
    static __device__ __forceinline__ void lds(const float* p, float* v) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
    }
};
template <>
struct VecLoad<float, 2> {
    static __device__ __forceinline__ void ld(const float* p, float* v) {
        const float2 x = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = x.x, v[1] = x.y;
    }
    static __device__ __forceinline__ void lds(const float* p, float* v) {
        const float2 x = *reinterpret_cast<const float2*>(p);
        v[0] = x.x, v[1] = x.y;
    }
};
template <typename T>
struct VecLoad<T, 1> {
    static __device__ __forceinline__ void ld(const T* p, T* v) { v[0] = __ldg(p); }
    static __device__ __forceinline__ void lds(const T* p, T* v) { v[0] = *p; }
};
template <>
struct VecLoad<double, 2> {
    static __device__ __forceinline__ void ld(const double* p, double* v) {
        const double2 x = __ldg(reinterpret_cast<const double2*>(p));
        v[0] = x.x, v[1] = x.y;
    }
    static __device__ __forceinline__ void lds(const double* p, double* v) {
        const double2 x = *reinterpret_cast<const double2*>(p);
        v[0] = x.x, v[1] = x.y;
    }
};

constexpr int kDepth = 4;         // slices of V in flight per thread in the force gather
constexpr int kSlicesPerAdd = 4;  // slices summed plainly before one compensated add

__device__ __forceinline__ float fmaf_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaf_t(double a, double b, double c) { return fma(a, b, c); }

// Offset (elements of T) of the cp.async ring after the six weight rows of length ld, 16-byte aligned.
template <typename T>
__host__ __device__ __forceinline__ int ring_offset(int ld) {
    return (int)(((size_t)6 * ld * sizeof(T) + 15) / 16 * 16 / sizeof(T));
}

// Image-summed weights of one atom's box in shared memory: wf[d][slot] = sum over the box
// points m that land on wrapped index t of fac[m] (dfac in wd), for t < nw[d]; the c axis is
// laid out in slots from the VW-aligned index below the box (slot = t + lead), zero outside.
template <typename T>
__device__ __forceinline__ void forces_weights(const AtomArgs<T>& a, const AtomPrep<T>& p, int atom, const int* nw,
                                               int lead, int nslot, T* wf, T* wd, int ld) {
    const int fb = a.fb, n1 = a.n1, n2 = a.n2, n3 = a.n3;
    const T* F = a.fac + (long long)atom * 3 * fb;
    const T* DF = a.dfac + (long long)atom * 3 * fb;
    for (int e = threadIdx.x; e < nw[0] + nw[1] + nslot; e += blockDim.x) {
        int d, t, slot;
        if (e < nw[0]) {
            d = 0, t = e, slot = e;
        } else if (e < nw[0] + nw[1]) {
            d = 1, t = e - nw[0], slot = t;
        } else {
            d = 2, slot = e - nw[0] - nw[1], t = slot - lead;
        }
        const int nd = d == 0 ? n1 : (d == 1 ? n2 : n3);
        const int cd = d == 0 ? p.cnt[0] : (d == 1 ? p.cnt[1] : p.cnt[2]);
        const int wd_ = d == 0 ? nw[0] : (d == 1 ? nw[1] : nw[2]);
        T s = T(0), sd = T(0);
        if (t >= 0 && t < wd_)
            for (int m = t; m < cd; m += nd) {
                s += F[d * fb + m];
                sd += DF[d * fb + m];
            }
        wf[d * ld + slot] = s;
        wd[d * ld + slot] = sd;
    }
}

// The c groups of one atom's box along a grid row.  A group is VW consecutive elements
// starting at a VW-aligned address; a row whose offset in V is r (mod VW) has aligned
// starts at c = -r (mod VW).  The box covers c in [st, end1) and, when it wraps past N3,
// also [0, l2).  Range 1 takes the groups from the aligned start at or below st, range 2
// those from -r; an element counts only inside its own range, so nothing is counted twice
// and the elements a group reads outside its range (the neighbouring rows' ends) get zero
// weight.  With N2 N3 = 0 (mod VW) and V VW-aligned, every such read stays inside V.
template <int VW>
struct CGroups {
    int st, end1, l2, n3;
    __device__ __forceinline__ CGroups(int st_, int nw, int n3_)
        : st(st_), end1(min(n3_, st_ + nw)), l2(max(0, st_ + nw - n3_)), n3(n3_) {}
    __device__ __forceinline__ int cs0(int r) const { return st - (st + r) % VW; }
    __device__ __forceinline__ int n1g(int r) const { return (end1 - cs0(r) + VW - 1) / VW; }
    __device__ __forceinline__ int n2g(int r) const { return l2 > 0 ? (l2 + r + VW - 1) / VW : 0; }
    // groups per row: the most over the residues rows can have
    __device__ __forceinline__ int groups() const {
        int step = n3 % VW == 0 ? VW : (n3 % 2 == 0 ? 2 : 1), g = 0;
        for (int r = 0; r < VW; r += step) g = max(g, n1g(r) + n2g(r));
        return g;
    }
    // first element (row-relative, may be negative) of group g of a row of residue r, and
    // for each element the image-summed weight index t (-1: zero weight)
    __device__ __forceinline__ int group(int r, int g, int* t) const {
        const int m1 = n1g(r);
        const bool second = g >= m1;
        const int cs = second ? -r + VW * (g - m1) : cs0(r) + VW * g;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const int c = cs + e;
            t[e] = second ? (c >= 0 && c < l2 ? c + n3 - st : -1) : (c >= st && c < end1 ? c - st : -1);
        }
        return g < m1 + n2g(r) ? cs : cs0(r);
    }
};

// Force gather of one atom (or a slab of its a range) per CTA.
//
// V is periodic, so sum_m fac[m] V[(lo + m) mod n] = sum_t w[t] V[(lo + t) mod n]
// over the min(cnt, n) distinct wrapped indices t, with the image-summed weight
// w[t] = sum_{m = t (mod n), m < cnt} fac[m] (likewise for dfac).  Shared memory
// holds these weights for the three axes.  Each (b row, c group) pair is one
// aligned vector load (CGroups), its VW c weights gathered into registers once.
// Per a slice a thread contracts its KP pairs: r0 = sum_e V_e wc_e,
// r1 = sum_e V_e dwc_e, then p0 += wb r0, py += dwb r0, pz += wb r1 (FP32: the
// products wb wc_e, dwb wc_e, wb dwc_e are formed once and the three sums run in
// paired lanes over even and odd e); slices are combined with wa / dwa in
// compensated sums.  The gather is bound by loads in
// flight, not by arithmetic: each thread keeps kDepth slices of its pairs in
// flight with cp.async copies into a private ring in shared memory.
template <typename T, int VW, int KP, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 8 ? 2 : NT == 128 ? (KP <= 5 ? 5 : 4) : (KP <= 2 ? 4 : 3))
    k_forces(AtomArgs<T> a, const T* __restrict__ V, int slabs, double* __restrict__ part, double* __restrict__ f,
             double* __restrict__ phi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int fb = a.fb;
    const int ld = fb + 8;
    T* wf = reinterpret_cast<T*>(smem_raw);  // [3][ld] image-summed fac
    T* wd = wf + 3 * ld;                     // [3][ld] image-summed dfac
    __shared__ double red[4][NT / 32];
    const int blk = blockIdx.x / slabs, slab = blockIdx.x - blk * slabs;
    const int atom = a.order ? a.order[blk] : blk;
    const AtomPrep<T> p = a.prep[atom];
    const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
    int nw[3], st[3];
    nw[0] = min(p.cnt[0], n1), nw[1] = min(p.cnt[1], n2), nw[2] = min(p.cnt[2], n3);
    st[0] = imod(p.lo[0], n1), st[1] = imod(p.lo[1], n2), st[2] = imod(p.lo[2], n3);
    const CGroups<VW> cg(st[2], nw[2], n3);
    const int ng = cg.groups();
    forces_weights(a, p, atom, nw, 0, nw[2], wf, wd, ld);
    __syncthreads();
    const int ia0 = (int)((long long)nw[0] * slab / slabs), ia1 = (int)((long long)nw[0] * (slab + 1) / slabs);
    const long long slice = (long long)n2 * n3;
    const int npairs = nw[1] * ng;
    const int rmul = n3 % VW;  // row residue: (b n3) mod VW = (b rmul) mod VW
    const T* wa = wf;
    const T* dwa = wd;
    T s0 = T(0), c0 = T(0), sx = T(0), cx = T(0), sy = T(0), cy = T(0), sz = T(0), cz = T(0);
    if (npairs <= NT * KP) {
        int off[KP];  // b n3 + c of the pair's first point; pairs past the end read row 0's first group with zero weight
        T wb[KP], dwb[KP], wc[KP][VW], dwc[KP][VW];
        // FP32 with even VW and four or more pairs per thread: the b weights folded into the c
        // weights, (even e, odd e) lanes.  With three pairs or fewer (the short boxes of
        // 420 x 420 x 210) the paired form measured 1% slower; with six (512^3) 6% faster.
        constexpr bool kPaired = sizeof(T) == 4 && VW % 2 == 0 && KP >= 4;
        float2 w0[KP][VW / 2 > 0 ? VW / 2 : 1], wy[KP][VW / 2 > 0 ? VW / 2 : 1], wz[KP][VW / 2 > 0 ? VW / 2 : 1];
#pragma unroll
        for (int u = 0; u < KP; ++u) {
            const int pr = threadIdx.x + NT * u;
            const bool ok = pr < npairs;
            const int j = ok ? pr / ng : 0, g = ok ? pr - j * ng : 0;
            int bj = st[1] + j;
            if (bj >= n2) bj -= n2;
            int t[VW];
            const int cs = cg.group(bj * rmul % VW, g, t);
            off[u] = bj * n3 + cs;
            wb[u] = ok ? wf[ld + j] : T(0);
            dwb[u] = ok ? wd[ld + j] : T(0);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                wc[u][e] = t[e] >= 0 ? wf[2 * ld + t[e]] : T(0);
                dwc[u][e] = t[e] >= 0 ? wd[2 * ld + t[e]] : T(0);
            }
            if constexpr (kPaired) {
#pragma unroll
                for (int h = 0; h < VW / 2; ++h) {
                    w0[u][h] = make_float2(wb[u] * wc[u][2 * h], wb[u] * wc[u][2 * h + 1]);
                    wy[u][h] = make_float2(dwb[u] * wc[u][2 * h], dwb[u] * wc[u][2 * h + 1]);
                    wz[u][h] = make_float2(wb[u] * dwc[u][2 * h], wb[u] * dwc[u][2 * h + 1]);
                }
            }
        }
        // ring of kDepth slices of this thread's pairs in shared memory, filled by
        // cp.async: each thread reads back only what it copied itself, so no barrier.
        // Slot s, pair u of this thread sits at ring + ((s KP + u) NT + tid) VW.
        T* ring = wf + ring_offset<T>(ld);
        constexpr uint32_t kPairBytes = NT * VW * sizeof(T), kSlotBytes = KP * kPairBytes;
        const uint32_t ring_s = smem_u32(ring) + threadIdx.x * (uint32_t)(VW * sizeof(T));
        int nbytes[KP];
#pragma unroll
        for (int u = 0; u < KP; ++u) nbytes[u] = threadIdx.x + NT * u < npairs ? (int)(VW * sizeof(T)) : 0;
        T b0 = T(0), bx = T(0), by = T(0), bz = T(0);
        // the next slice to issue: its a index and first element, advanced (with the periodic wrap) per issue
        int ai = st[0] + ia0;
        if (ai >= n1) ai -= n1;
        const T* Vs = V + ai * slice;
        auto issue = [&](uint32_t slot) {
            const uint32_t d = ring_s + slot * kSlotBytes;
#pragma unroll
            for (int u = 0; u < KP; ++u) cp_async_s<VW * sizeof(T)>(d + u * kPairBytes, Vs + off[u], nbytes[u]);
            if (++ai == n1) {
                ai = 0;
                Vs = V;
            } else {
                Vs += slice;
            }
        };
#pragma unroll
        for (int k = 0; k < kDepth - 1; ++k) {
            if (ia0 + k < ia1) issue((uint32_t)k);
            cp_async_commit();
        }
        for (int t = ia0; t < ia1; ++t) {
            const unsigned k = (unsigned)(t - ia0);
            if (t + kDepth - 1 < ia1) issue((k + kDepth - 1) % kDepth);
            cp_async_commit();
            cp_async_wait<kDepth - 1>();  // the group of slice t is complete
            const T* r = ring + ((k % kDepth) * KP * NT + threadIdx.x) * VW;
            T p0 = T(0), py = T(0), pz = T(0);
            if constexpr (kPaired) {
                // sum_e V_e wb wc_e and the like in paired lanes: 3 VW / 2 paired FMAs per pair
                float2 q0 = make_float2(0.f, 0.f), qy = q0, qz = q0;
#pragma unroll
                for (int u = 0; u < KP; ++u) {
                    T v[VW];
                    VecLoad<T, VW>::lds(r + u * NT * VW, v);
#pragma unroll
                    for (int h = 0; h < VW / 2; ++h) {
                        const float2 vv = make_float2(v[2 * h], v[2 * h + 1]);
                        q0 = __ffma2_rn(vv, w0[u][h], q0);
                        qy = __ffma2_rn(vv, wy[u][h], qy);
                        qz = __ffma2_rn(vv, wz[u][h], qz);
                    }
                }
                p0 = q0.x + q0.y;
                py = qy.x + qy.y;
                pz = qz.x + qz.y;
            } else {
#pragma unroll
                for (int u = 0; u < KP; ++u) {
                    T v[VW];
                    VecLoad<T, VW>::lds(r + u * NT * VW, v);
                    T r0 = T(0), r1 = T(0);
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        r0 += v[e] * wc[u][e];
                        r1 += v[e] * dwc[u][e];
                    }
                    p0 += wb[u] * r0;
                    py += dwb[u] * r0;
                    pz += wb[u] * r1;
                }
            }
            // plain sums over groups of kSlicesPerAdd slices, each group added with compensation
            b0 = fmaf_t(wa[t], p0, b0);
            bx = fmaf_t(dwa[t], p0, bx);
            by = fmaf_t(wa[t], py, by);
            bz = fmaf_t(wa[t], pz, bz);
            if ((k + 1) % kSlicesPerAdd == 0 || t + 1 == ia1) {
                kahan_add(s0, c0, b0);
                kahan_add(sx, cx, bx);
                kahan_add(sy, cy, by);
                kahan_add(sz, cz, bz);
                b0 = bx = by = bz = T(0);
            }
        }
        cp_async_wait<0>();
    } else {
        // very wide boxes: pairs revisited per slice, their geometry recomputed
        for (int t = ia0; t < ia1; ++t) {
            int ai = st[0] + t;
            if (ai >= n1) ai -= n1;
            const T* Vs = V + ai * slice;
            T p0 = T(0), py = T(0), pz = T(0);
            for (int pr = threadIdx.x; pr < npairs; pr += NT) {
                const int j = pr / ng, g = pr - j * ng;
                int bj = st[1] + j;
                if (bj >= n2) bj -= n2;
                int tc[VW];
                const int cs = cg.group(bj * rmul % VW, g, tc);
                T v[VW];
                VecLoad<T, VW>::ld(Vs + bj * n3 + cs, v);
                T r0 = T(0), r1 = T(0);
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    r0 += tc[e] >= 0 ? v[e] * wf[2 * ld + tc[e]] : T(0);
                    r1 += tc[e] >= 0 ? v[e] * wd[2 * ld + tc[e]] : T(0);
                }
                p0 += wf[ld + j] * r0;
                py += wd[ld + j] * r0;
                pz += wf[ld + j] * r1;
            }
            kahan_add(s0, c0, wa[t] * p0);
            kahan_add(sx, cx, dwa[t] * p0);
            kahan_add(sy, cy, wa[t] * py);
            kahan_add(sz, cz, wa[t] * pz);
        }
    }
    // four block sums: error-free FP32 warp steps, FP64 only across warps
    const T vs[4] = {s0, sx, sy, sz}, ve[4] = {-c0, -cx, -cy, -cz};
    double tot[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) tot[c] = block_sum_comp(vs[c], ve[c], red[c]);
    if (threadIdx.x != 0) return;
    if (f) {
        // one slab per atom: the forces and phi directly, as k_forces_finalize forms them
        const double cf = -a.dV * a.q[atom] * a.norm * 2.0 * a.inv_s2;
        f[3 * atom + 0] = cf * tot[1];
        f[3 * atom + 1] = cf * tot[2];
        f[3 * atom + 2] = cf * tot[3];
        if (phi) phi[atom] = a.dV * a.norm * tot[0];
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) part[(long long)blockIdx.x * 4 + c] = tot[c];
    }
}

// The force gather's CTA order: atoms by the wrapped a start of their box (a counting sort by a
// index; the order inside one a index is that of the atomics).  The gather streams each box slice
// by slice along a, so CTAs resident together then read the same a slices of V, which stay in L2
// while every atom that overlaps them uses them.  Each CTA computes one atom's sums alone, so the
// results do not depend on this order.  One CTA of kOrderThreads threads; N1 <= kMaxAxis bins.
constexpr int kOrderThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kOrderThreads) k_slab_order(const AtomPrep<T>* __restrict__ prep, int n, int n1,
                                                              int* __restrict__ order) {
    __shared__ int bin[kMaxAxis];
    __shared__ int wsum[kOrderThreads / 32];
    for (int b = threadIdx.x; b < n1; b += kOrderThreads) bin[b] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kOrderThreads) atomicAdd(&bin[prep[i].st[0]], 1);
    __syncthreads();
    // exclusive scan of the bins: each thread a contiguous chunk, warp scans of the chunk sums
    const int chunk = (n1 + kOrderThreads - 1) / kOrderThreads;
    const int b0 = threadIdx.x * chunk, b1 = min(n1, b0 + chunk);
    int local = 0;
    for (int b = b0; b < b1; ++b) local += bin[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kOrderThreads / 32 ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        if (lane < kOrderThreads / 32) wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int run = incl - local + (warp > 0 ? wsum[warp - 1] : 0);  // exclusive start of this thread's chunk
    for (int b = b0; b < b1; ++b) {
        const int c = bin[b];
        bin[b] = run;
        run += c;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kOrderThreads) order[atomicAdd(&bin[prep[i].st[0]], 1)] = i;
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


// Per-atom boxes and factor arrays (one CTA per leaf); with `bins`, also the leaf
// boxes and the atom lists of the splat tiles.
template <typename T>
cudaError_t prep_atoms(const Plan& p, const AtomArgs<T>& a, bool bins, cudaStream_t s) {
    if (bins) {
        cudaError_t e = cudaMemsetAsync(p.bin_cursor, 0, sizeof(int) * (size_t)p.n_tiles, s);
        if (e != cudaSuccess) return e;
    }
    if (a.n == 0) return cudaSuccess;
    p.launches += 1;
    k_leaf_setup<T><<<a.nleaves, kSetupThreads, 0, s>>>(a, p.tiles[0], p.tiles[1], p.tiles[2], p.bin_cursor,
                                                         p.bin_list, bins);
    return cudaGetLastError();
}

template <typename T>
cudaError_t splat_impl(const Plan& p, const double* pos, const double* q, int n, void* rho, cudaStream_t s) {
    AtomArgs<T> a = make_atom_args<T>(p, pos, q, n);
    cudaError_t e = prep_atoms<T>(p, a, true, s);
    if (e != cudaSuccess) return e;
    p.launches += 1;
    const dim3 grid((unsigned)p.tiles[2], (unsigned)p.tiles[1], (unsigned)p.tiles[0]);
    if (p.n[0] % TA == 0 && p.n[1] % TB == 0 && p.n[2] % TC == 0)
        k_splat_binned<T, true><<<grid, kThreads, 0, s>>>(a, static_cast<T*>(rho), p.bin_cursor, p.bin_list);
    else
        k_splat_binned<T, false><<<grid, kThreads, 0, s>>>(a, static_cast<T*>(rho), p.bin_cursor, p.bin_list);
    return cudaGetLastError();
}

// CTA size and pairs per thread of the force gather for the largest box of the plan.
struct ForceShape {
    int nt, kp;
};
ForceShape forces_shape(const Plan& p, int vw);
size_t forces_smem(const Plan& p, size_t real_size, int vw, ForceShape fs);

template <typename T, int VW, int NT>
void launch_k_forces_nt(const Plan& p, const AtomArgs<T>& a, const T* V, unsigned blocks, int slabs, int kp,
                        size_t sm, double* f, double* phi, cudaStream_t s) {
    if constexpr (NT == 128) {
        switch (kp) {
            case 5: k_forces<T, VW, 5, NT><<<blocks, NT, sm, s>>>(a, V, slabs, p.force_partials, f, phi); return;
            case 6: k_forces<T, VW, 6, NT><<<blocks, NT, sm, s>>>(a, V, slabs, p.force_partials, f, phi); return;
            default: break;
        }
    }
    switch (kp) {
        case 1: k_forces<T, VW, 1, NT><<<blocks, NT, sm, s>>>(a, V, slabs, p.force_partials, f, phi); break;
        case 2: k_forces<T, VW, 2, NT><<<blocks, NT, sm, s>>>(a, V, slabs, p.force_partials, f, phi); break;
        case 3: k_forces<T, VW, 3, NT><<<blocks, NT, sm, s>>>(a, V, slabs, p.force_partials, f, phi); break;
        default: k_forces<T, VW, 4, NT><<<blocks, NT, sm, s>>>(a, V, slabs, p.force_partials, f, phi); break;
    }
}

// Pairs per thread: enough for the largest box of the plan (npairs <= box_max x
// (box_max + 2 VW) / VW); boxes beyond that loop over the pairs from shared memory.
template <typename T, int VW>
void launch_k_forces_vw(const Plan& p, const AtomArgs<T>& a, const T* V, unsigned blocks, int slabs, double* f,
                        double* phi, cudaStream_t s) {
    const ForceShape fs = forces_shape(p, VW);
    const size_t sm = forces_smem(p, sizeof(T), VW, fs);
    if constexpr (sizeof(T) == 4 && VW == 4)
        if (fs.nt == 128) return launch_k_forces_nt<T, VW, 128>(p, a, V, blocks, slabs, fs.kp, sm, f, phi, s);
    launch_k_forces_nt<T, VW, kThreads>(p, a, V, blocks, slabs, fs.kp, sm, f, phi, s);
}

// The widest aligned vector along c: V must be VW-element aligned and VW must divide N2 N3
// (every a slice then starts aligned; CGroups handles rows of any residue).  f, phi: written
// directly by a one-slab launch (else null: partials for k_forces_finalize).
template <typename T>
void launch_k_forces(const Plan& p, const AtomArgs<T>& a, const T* V, unsigned blocks, int slabs, double* f,
                     double* phi, cudaStream_t s) {
    const uintptr_t addr = reinterpret_cast<uintptr_t>(V);
    const long long slice = (long long)p.n[1] * p.n[2];
    if constexpr (sizeof(T) == 4) {
        if (slice % 4 == 0 && addr % 16 == 0) {
            launch_k_forces_vw<T, 4>(p, a, V, blocks, slabs, f, phi, s);
            return;
        }
    }
    if (slice % 2 == 0 && addr % (2 * sizeof(T)) == 0)
        launch_k_forces_vw<T, 2>(p, a, V, blocks, slabs, f, phi, s);
    else
        launch_k_forces_vw<T, 1>(p, a, V, blocks, slabs, f, phi, s);
}

size_t forces_smem(const Plan& p, size_t real_size, int vw, ForceShape fs) {
    const int ld = p.box_max + 8;
    const size_t ring = (size_t)kDepth * fs.kp * fs.nt * vw * real_size;
    return (real_size == 4 ? ring_offset<float>(ld) : ring_offset<double>(ld)) * real_size + ring;
}

// FP32 with 16-byte vectors: 128-thread CTAs with up to 6 pairs per thread when that holds
// the box (fewer idle pair slots, the per-slice work spread over more pairs); otherwise 256
// threads with at most 4 (wider boxes loop over the pairs).
ForceShape forces_shape(const Plan& p, int vw) {
    const long long rows = std::min(p.box_max, p.n[1]);
    // CGroups: at most (nw + 2 VW - 2) / VW + 2 groups per row, the wrapped range included
    const long long npairs = rows * ((std::min(p.box_max, p.n[2]) + 2 * vw - 2) / vw + 2);
    if (p.real_size == 4 && vw == 4 && npairs <= 6 * 128) return {128, (int)std::max(1LL, (npairs + 127) / 128)};
    return {kThreads, (int)std::max(1LL, std::min(4LL, (npairs + kThreads - 1) / kThreads))};
}

template <typename T>
cudaError_t forces_impl(const Plan& p, const double* pos, const double* q, int n, const void* vh, double* f,
                        double* phi, bool prepared, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    AtomArgs<T> a = make_atom_args<T>(p, pos, q, n);
    if (!prepared) {
        cudaError_t e = prep_atoms<T>(p, a, false, s);
        if (e != cudaSuccess) return e;
    }
    int slabs = (4 * 152 * 2 + n - 1) / n;  // enough CTAs to cover the GPU
    if (slabs > p.max_force_slabs) slabs = p.max_force_slabs;
    if (slabs < 1) slabs = 1;
    if (slabs == 1) {  // one CTA per atom writes its forces: no partials, no finalize launch
        p.launches += 2;
        k_slab_order<T><<<1, kOrderThreads, 0, s>>>(a.prep, n, p.n[0], p.force_order);
        a.order = p.force_order;
        launch_k_forces<T>(p, a, static_cast<const T*>(vh), (unsigned)n, 1, f, phi, s);
        return cudaGetLastError();
    }
    p.launches += 2;
    launch_k_forces<T>(p, a, static_cast<const T*>(vh), (unsigned)n * slabs, slabs, nullptr, nullptr, s);
    k_forces_finalize<<<(n + 127) / 128, 128, 0, s>>>(p.force_partials, n, slabs, q, p.dV, a.norm, a.inv_s2, f, phi);
    return cudaGetLastError();
}

template <typename T, int VW, int NT>
cudaError_t allow_forces_smem(int optin) {
    cudaError_t e = allow_max_dynamic_smem(k_forces<T, VW, 1, NT>, optin);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_forces<T, VW, 2, NT>, optin);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_forces<T, VW, 3, NT>, optin);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_forces<T, VW, 4, NT>, optin);
    if constexpr (NT == 128) {
        if (e == cudaSuccess) e = allow_max_dynamic_smem(k_forces<T, VW, 5, NT>, optin);
        if (e == cudaSuccess) e = allow_max_dynamic_smem(k_forces<T, VW, 6, NT>, optin);
    }
    return e;
}

template <typename T>
cudaError_t configure_atoms(int optin) {
    cudaError_t e = allow_forces_smem<T, 1, kThreads>(optin);
    if (e == cudaSuccess) e = allow_forces_smem<T, 2, kThreads>(optin);
    if constexpr (sizeof(T) == 4) {
        if (e == cudaSuccess) e = allow_forces_smem<T, 4, kThreads>(optin);
        if (e == cudaSuccess) e = allow_forces_smem<T, 4, 128>(optin);
    }
    return e;
}

}  // namespace

cudaError_t configure_atom_kernels(const Plan& p) {
    int optin = 0;
    cudaError_t e = optin_smem(&optin);
    if (e != cudaSuccess) return e;
    for (int vw : {1, 2, 4})
        if ((vw < 4 || p.real_size == 4) && forces_smem(p, p.real_size, vw, forces_shape(p, vw)) + 1024 > (size_t)optin)
            return cudaErrorInvalidConfiguration;
    return p.prec == HARTREE_FP64 ? configure_atoms<double>(optin) : configure_atoms<float>(optin);
}

cudaError_t launch_splat(const Plan& p, const double* pos, const double* q, int n, void* rho, cudaStream_t s) {
    return p.prec == HARTREE_FP64 ? splat_impl<double>(p, pos, q, n, rho, s) : splat_impl<float>(p, pos, q, n, rho, s);
}

cudaError_t launch_splat_solve(const Plan& p, const double* pos, const double* q, int n, void* vh, double* eh,
                               cudaStream_t s) {
    if (!splat_fused_available(p)) {
        cudaError_t e = launch_splat(p, pos, q, n, vh, s);
        return e == cudaSuccess ? launch_poisson(p, vh, vh, eh, s) : e;
    }
    const cudaError_t e = launch_splat_r2c(p, pos, q, n, s);
    return e == cudaSuccess ? launch_poisson_from(p, 1, nullptr, vh, eh, s) : e;
}

cudaError_t launch_splat_r2c(const Plan& p, const double* pos, const double* q, int n, cudaStream_t s) {
    const AtomArgs<float> a = make_atom_args<float>(p, pos, q, n);
    cudaError_t e = prep_atoms<float>(p, a, false, s);
    if (e != cudaSuccess) return e;
    p.launches += 1;
    launch_r2c_splat(p, a, s);
    return cudaGetLastError();
}

cudaError_t launch_forces(const Plan& p, const double* pos, const double* q, int n, const void* vh, double* f,
                          double* phi, cudaStream_t s, bool prepared) {
    return p.prec == HARTREE_FP64 ? forces_impl<double>(p, pos, q, n, vh, f, phi, prepared, s)
                                  : forces_impl<float>(p, pos, q, n, vh, f, phi, prepared, s);
}

}  // namespace hartree
