// atoms_dev.cuh -- per-atom preparation and the density splat as device
// functions, shared by the kernels of atoms.cu and the batched persistent
// kernel of batch.cu.  See atoms.cu for the method.
#pragma once

#include "internal.cuh"

namespace hartree {

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

// The box of atom i along axis d: the grid points within rc of the atom's position X (wrapped
// into the cell: any image gives the same periodic sum), from the unwrapped index lo, cnt of them
// (at most fb), starting at the wrapped index st, and the offset D0 = lo h - X of the first.
struct AxisBox {
    int lo, cnt, st;
    double D0;
};

template <typename T>
__device__ __forceinline__ AxisBox atom_axis_box(const AtomArgs<T>& a, int i, int d) {
    const double h = d == 0 ? a.h1 : (d == 1 ? a.h2 : a.h3);
    const double L = d == 0 ? a.L1 : (d == 1 ? a.L2 : a.L3);
    double X = a.pos[3 * i + d];
    X -= L * floor(X / L);
    const double lo = ceil((X - a.rc) / h);
    const double hi = floor((X + a.rc) / h);
    AxisBox b;
    b.lo = (int)lo;
    b.st = imod(b.lo, d == 0 ? a.n1 : (d == 1 ? a.n2 : a.n3));
    b.cnt = hi >= lo ? min((int)(hi - lo) + 1, a.fb) : 0;
    b.D0 = lo * h - X;
    return b;
}

template <typename T>
__device__ __forceinline__ void atom_prep_one(const AtomArgs<T>& a, int i) {
    if (i >= a.n) return;
    AtomPrep<T> p;
    for (int d = 0; d < 3; ++d) {
        const AxisBox b = atom_axis_box(a, i, d);
        p.lo[d] = b.lo;
        p.st[d] = b.st;
        p.cnt[d] = b.cnt;
        p.dh[d] = (T)b.D0;
        p.dl[d] = (T)(b.D0 - (double)p.dh[d]);
    }
    const double qn = a.q[i] * a.norm;
    p.qn = (T)qn;
    p.ql = (T)(qn - (double)p.qn);
    a.prep[i] = p;
}

// Float-float numbers: the unevaluated sum hi + lo of two FP32 values with
// |lo| <= ulp(hi) / 2, about 44 significant bits (Dekker's double-length
// arithmetic: an FMA gives the exact error of a product, Knuth's two-sum that
// of a sum).  The _rn intrinsics keep the compiler from contracting the steps.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_of(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

// a * b to float-float (the lo * lo term, 2^-48 relative, is dropped)
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.hi, b.hi, -p)));
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}

// a * b rounded once to FP32 (up to the 2^-44 error of the operands)
__device__ __forceinline__ float ff_mul_round(FF a, FF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    return __fadd_rn(p, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.hi, b.hi, -p))));
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));  // s + e = a.hi + b.hi exactly
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float t = __fadd_rn(s, e);
    return {t, __fsub_rn(e, __fsub_rn(t, s))};
}

// One thread per (atom, axis, run of kRun<T>() box points).  FP64 plans evaluate
// every point directly in FP64.  FP32 plans start each run with two FP64
// exponentials (the ratios' constant decay exp(-2 h^2 / s^2) is formed on the host)
// and continue with the exact ratio recurrence in float-float: FP64
// arithmetic runs at 1/64 of the FP32 rate on GB300, and a recurrence in FP64 made
// the setup FP64-bound.  The recurrence's relative error after m steps is about
// m^2 / 2 float-float roundings (3e-11 at m = 64), far below the single FP32
// rounding of each stored value, so FP32 runs are long and the exponentials few.
template <typename T>
__host__ __device__ constexpr int kRun() {
    return sizeof(T) == 4 ? 64 : 8;
}

// The factors of box points m0 .. min(cnt, m0 + kRun) - 1 of atom i along axis d, whose box
// has cnt points from the offset D0 = lo h - X.
template <typename T>
__device__ __forceinline__ void atom_factors_run(const AtomArgs<T>& a, int i, int d, int m0, int cnt, double D0) {
    constexpr int kRun = hartree::kRun<T>();
    if (m0 >= cnt) return;
    const int m1 = min(cnt, m0 + kRun);
    const double h = d == 0 ? a.h1 : (d == 1 ? a.h2 : a.h3);
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
        // exponent(m) = -(D0 + m h)^2 / s^2: successive ratios are exp(-(2 d_m h + h^2) / s^2),
        // and those ratios fall by the constant factor exp(-2 h^2 / s^2)
        const double ds = fma((double)m0, h, D0);
        FF g = ff_of(exp(-ds * ds * a.inv_s2));
        FF r = ff_of(exp(-(2.0 * ds * h + h * h) * a.inv_s2));
        const FF q = ff_of(d == 0 ? a.qr[0] : (d == 1 ? a.qr[1] : a.qr[2]));  // constant indices: a stays in registers
        FF dm = ff_of(ds);
        const FF hf = ff_of(h);
        for (int m = m0; m < m1; ++m) {
            f[m] = g.hi;  // hi is the FP32 rounding of hi + lo
            df[m] = ff_mul_round(dm, g);
            g = ff_mul(g, r);
            r = ff_mul(r, q);
            dm = ff_add(dm, hf);
        }
    }
}

// One thread per (atom, axis, run of kRun<T>() box points), the box read from prep.
template <typename T>
__device__ __forceinline__ void atom_factors_one(const AtomArgs<T>& a, long long t) {
    constexpr int kRun = hartree::kRun<T>();
    const int runs = (a.fb + kRun - 1) / kRun;
    if (t >= 3LL * a.n * runs) return;
    const int i = (int)(t / (3 * runs));
    const int rem = (int)(t - (long long)i * 3 * runs);
    const int d = rem / runs, m0 = (rem - d * runs) * kRun;
    const AtomPrep<T>& p = a.prep[i];
    atom_factors_run(a, i, d, m0, p.cnt[d], (double)p.dh[d] + (double)p.dl[d]);
}

template <typename T>
__device__ __forceinline__ void leaf_box_one(const AtomPrep<T>* __restrict__ prep, int n, int apl, int nleaves, int n1,
                                             int n2, int n3, int* __restrict__ leaf, int l) {
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

// Sum over the box points of one atom that land on grid index g in [0, n) (all
// images); st = lo mod n is the wrapped index of box point 0.
template <typename T>
__device__ __forceinline__ T image_sum(const T* __restrict__ f, int g, int st, int cnt, int n) {
    int m = g - st;
    if (m < 0) m += n;
    T s = T(0);
    for (; m < cnt; m += n) s += f[m];
    return s;
}

// Stage the separable factors of atoms ids[0..nb) for the tile at (a0, b0, c0):
// fa over TA a-points, fb over TB b-points, fc (times q (pi s^2)^-3/2) over TC
// c-points.  One loop per axis, so the lanes of a warp take the same path.
template <typename T>
__device__ __forceinline__ void stage_factors(const AtomArgs<T>& a, const int* ids, int nb, int a0, int b0, int c0,
                                              T (*fa)[TA], T (*fb)[TB], T (*fc)[TC]) {
    for (int e = threadIdx.x; e < nb * TC; e += kThreads) {
        const int t = e / TC, k = e - t * TC;
        const int i = ids[t];
        const AtomPrep<T>& p = a.prep[i];
        const T sc = c0 + k < a.n3 ? image_sum(a.fac + ((long long)i * 3 + 2) * a.fb, c0 + k, p.st[2], p.cnt[2], a.n3)
                                   : T(0);
        fc[t][k] = p.qn * sc + p.ql * sc;
    }
    for (int e = threadIdx.x; e < nb * TA; e += kThreads) {
        const int t = e / TA, f = e - t * TA;
        const int i = ids[t];
        const AtomPrep<T>& p = a.prep[i];
        fa[t][f] = a0 + f < a.n1 ? image_sum(a.fac + (long long)i * 3 * a.fb, a0 + f, p.st[0], p.cnt[0], a.n1) : T(0);
    }
    for (int e = threadIdx.x; e < nb * TB; e += kThreads) {
        const int t = e / TB, f = e - t * TB;
        const int i = ids[t];
        const AtomPrep<T>& p = a.prep[i];
        fb[t][f] = b0 + f < a.n2
                       ? image_sum(a.fac + ((long long)i * 3 + 1) * a.fb, b0 + f, p.st[1], p.cnt[1], a.n2)
                       : T(0);
    }
}

template <typename T>
__device__ void splat_tile(const AtomArgs<T>& a, T* __restrict__ rho, int tiles_b, int tiles_c, int tile) {
    __shared__ int leaf_list[kThreads];
    __shared__ int cand[kThreads];
    __shared__ int warp_cnt[kThreads / 32];
    __shared__ int n_sel;
    __shared__ __align__(16) T fa[kBatch][TA];
    __shared__ T fb[kBatch][TB], fc[kBatch][TC];

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
                stage_factors(a, cand + bb, nb, a0, b0, c0, fa, fb, fc);
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

template <typename T>
inline AtomArgs<T> make_atom_args(const Plan& p, const double* pos, const double* q, int n) {
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
    for (int d = 0; d < 3; ++d) a.qr[d] = exp(-2.0 * p.h[d] * p.h[d] * a.inv_s2);
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

// ---------------------------------------------------------------- tile binning
// The tiles along one axis that hold at least one wrapped index of the box
// [lo, lo + cnt): count of them, and tile(k) for k < count.
struct AxisTiles {
    int start, c1, count;
    __device__ __forceinline__ int tile(int k) const { return k < c1 ? start + k : k - c1; }
};

__device__ __forceinline__ AxisTiles axis_tiles(int lo, int cnt, int n, int T, int nT) {
    if (cnt <= 0) return {0, 0, 0};
    if (cnt >= n) return {0, nT, nT};
    const int s = imod(lo, n), e = s + cnt;
    const int t0 = s / T;
    if (e <= n) {
        const int c = (e - 1) / T - t0 + 1;
        return {t0, c, c};
    }
    const int t2 = (e - n - 1) / T;  // last tile of the segment wrapped to the start
    if (t2 >= t0) return {0, nT, nT};  // both segments meet: every tile
    return {t0, nT - t0, nT - t0 + t2 + 1};
}


// Append atom i (prepared) to the list of every splat tile (TA x TB x TC) its box reaches, the
// threads lane, lane + lanes, ... of a team sharing its tiles.  Slots are taken with atomics, so a
// list is unordered (the splat sorts it); a tile reached by more than kBinCap atoms keeps counting
// and its splat then selects atoms from the leaf boxes instead.  A list entry carries the atom's
// wrapped box start and length per axis, so the splat reads the factors with no further lookup.
template <typename T>
__device__ __forceinline__ void bin_atom(const AtomArgs<T>& a, int i, int tA, int tB, int tC, int* __restrict__ cursor,
                                         int4* __restrict__ list, int lane, int lanes) {
    const AtomPrep<T> p = a.prep[i];
    const AxisTiles ra = axis_tiles(p.lo[0], p.cnt[0], a.n1, TA, tA);
    const AxisTiles rb = axis_tiles(p.lo[1], p.cnt[1], a.n2, TB, tB);
    const AxisTiles rc = axis_tiles(p.lo[2], p.cnt[2], a.n3, TC, tC);
    const int nbc = rb.count * rc.count;
    const int tot = ra.count * nbc;
    const int4 entry = make_int4(i, p.st[0] | (p.cnt[0] << 16), p.st[1] | (p.cnt[1] << 16), p.st[2] | (p.cnt[2] << 16));
    for (int k = lane; k < tot; k += lanes) {
        const int ka = k / nbc, r = k - ka * nbc, kb = r / rc.count, kc = r - kb * rc.count;
        const int tile = (ra.tile(ka) * tB + rb.tile(kb)) * tC + rc.tile(kc);
        const int slot = atomicAdd(cursor + tile, 1);
        if (slot < kBinCap) list[(long long)tile * kBinCap + slot] = entry;
    }
}

// Splat of one tile from its bin (the batched form's; k_splat_binned takes the
// same steps): the list is sorted by atom index in shared memory (a rank sort;
// indices in a list are distinct), so the summation order is that of the
// leaf-selecting splat, then factors are staged in batches and accumulated as
// there.  Returns false, having done nothing, when more than
// kBinCap atoms reached the tile (the caller then takes the leaf-selecting
// splat_tile).  Shared memory: ent, sorted [kBinCap], fa [kBatch][TA] (16-byte
// aligned), fb [kBatch][TB], fc [kBatch][TC] (SplatWs: the layout of one block).
// FULL: every tile lies inside the grid (TA | N1, TB | N2, TC | N3).  CG: the lists were filled
// earlier in the same launch (the batched form), so they are read through L2.
template <typename T>
struct SplatWs {
    int4 ent[kBinCap], sorted[kBinCap];
    T fa[kBatch][TA], fb[kBatch][TB], fc[kBatch][TC];
};

template <typename T, bool FULL, bool CG = false>
__device__ __forceinline__ bool splat_tile_binned(const AtomArgs<T>& a, T* __restrict__ rho, int tiles_b, int tiles_c,
                                                  int tile,
                                  const int* __restrict__ cursor, const int4* __restrict__ list, int4* ent,
                                  int4* sorted, T (*fa)[TA], T (*fb)[TB], T (*fc)[TC]) {
    const int tc = tile % tiles_c, tb = (tile / tiles_c) % tiles_b, ta = tile / (tiles_c * tiles_b);
    const int L = CG ? __ldcg(cursor + tile) : cursor[tile];
    if (L > kBinCap) return false;
    for (int e = threadIdx.x; e < L; e += kThreads) {
        const int4* src = list + (long long)tile * kBinCap + e;
        ent[e] = CG ? __ldcg(src) : *src;
    }
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
    return true;
}


}  // namespace hartree
