// pair_passes.cu -- the b and a column passes (Sec. 3.2.4 order: b, then a with
// the Green multiply and E_H, then b^-1) on paired FP32 lanes.
//
// sm_100-class GPUs issue add, sub, mul and fma on two FP32 lanes at once
// (the .f32x2 forms).  The column passes are bound by instruction issue, not by
// HBM: every butterfly, twiddle product and Green multiply is plain FP32
// arithmetic.  Here each thread transforms two neighbouring columns together,
// as a pair of lanes: a complex pair c2 holds (re_c, re_c+1) and (im_c, im_c+1),
// so one paired instruction does the work of two scalar ones, and the two
// columns share their twiddles.
//
// Layout of a tile in shared memory (N rows of COLS complex columns):
//   * natural: what the TMA copies in and out, element (n, c) at float
//     2 (n COLS + c), interleaved (re, im);
//   * split: between the first and the last stage, pair p of row n holds
//     (re_2p, re_2p+1, im_2p, im_2p+1) in the 16 bytes of the natural pair, so
//     every load and store of a pair is one 16-byte access.  With 64-byte rows
//     (8 columns) the first stage writes rows R0 apart, which share one half of
//     the banks; the split layout therefore stores row n at n ^ ((n >> SH) & 1),
//     SH = log2 R0, which spreads those rows over both halves and keeps the
//     other stages' consecutive rows in consecutive pairs of rows.
//
// Twiddles: per stage, in the order the stage reads them (output r of butterfly
// k at entry (r - 1) NS + k), each as two 16-byte vectors (hr, hr, hi, hi) and
// (lr, lr, li, li): the value rounded to FP32 and its remainder, both already
// duplicated on the two lanes.  The rounded values of all stages form one array
// and the remainders a second one, so the consecutive entries a warp reads are
// consecutive 16-byte vectors (one shared-memory wavefront per 8 entries).  Forward stages use the remainder (FP32 rounding
// of the twiddles would otherwise shrink |X| and bias E_H); inverse stages,
// which only shape V_H, use the rounded values.
#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "tma.cuh"

namespace hartree {

namespace {

// ------------------------------------------------------------------ two FP32 lanes
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as b (-1) + a: exact product, one rounding, the same result as a subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }

// Two complex values (columns c and c + 1), lane-split.
struct c2 {
    float2 re, im;
};
__device__ __forceinline__ c2 operator+(c2 a, c2 b) { return c2{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ c2 operator-(c2 a, c2 b) { return c2{sub2(a.re, b.re), sub2(a.im, b.im)}; }
// a + rot(b) and a - rot(b), rot(b) = b (-i) forward and b (+i) inverse
template <bool INV>
__device__ __forceinline__ c2 addrot(c2 a, c2 b) {
    return INV ? c2{sub2(a.re, b.im), add2(a.im, b.re)} : c2{add2(a.re, b.im), sub2(a.im, b.re)};
}
template <bool INV>
__device__ __forceinline__ c2 subrot(c2 a, c2 b) {
    return INV ? c2{add2(a.re, b.im), sub2(a.im, b.re)} : c2{sub2(a.re, b.im), add2(a.im, b.re)};
}
// a + (t.re, -t.im) and a - (t.re, -t.im): a product whose imaginary part comes out negated
__device__ __forceinline__ c2 add_cj(c2 a, c2 t) { return c2{add2(a.re, t.re), sub2(a.im, t.im)}; }
__device__ __forceinline__ c2 sub_cj(c2 a, c2 t) { return c2{sub2(a.re, t.re), add2(a.im, t.im)}; }

// x c for a real constant c; COMP: c as a rounded high part plus its remainder
template <bool COMP>
__device__ __forceinline__ float2 kmul2(float2 x, double c) {
    const float hi = (float)c;
    if constexpr (COMP) {
        const float lo = (float)(c - (double)hi);
        return fma2(x, dup(hi), mul2(x, dup(lo)));
    } else {
        return mul2(x, dup(hi));
    }
}
// a (c + i s) for constants c, s
template <bool COMP>
__device__ __forceinline__ c2 kcmul2(c2 a, double c, double s) {
    const float ch = (float)c, sh = (float)s;
    if constexpr (COMP) {
        const float cl = (float)(c - (double)ch), sl = (float)(s - (double)sh);
        return c2{fma2(a.re, dup(ch), fma2(a.im, dup(-sh), fma2(a.re, dup(cl), mul2(a.im, dup(-sl))))),
                  fma2(a.re, dup(sh), fma2(a.im, dup(ch), fma2(a.re, dup(sl), mul2(a.im, dup(cl)))))};
    } else {
        return c2{fma2(a.re, dup(ch), mul2(a.im, dup(-sh))), fma2(a.re, dup(sh), mul2(a.im, dup(ch)))};
    }
}

// ------------------------------------------------------------------ small DFTs on pairs
// v[k] <- sum_m v[m] exp(-+ 2 pi i m k / R)   (minus: forward, plus: INV)
template <bool INV>
__device__ __forceinline__ void pdft2(c2* v) {
    const c2 a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}

template <bool INV>
__device__ __forceinline__ void pdft4(c2* v) {
    const c2 s02 = v[0] + v[2], d02 = v[0] - v[2];
    const c2 s13 = v[1] + v[3], d13 = v[1] - v[3];
    v[0] = s02 + s13;
    v[2] = s02 - s13;
    v[1] = addrot<INV>(d02, d13);
    v[3] = subrot<INV>(d02, d13);
}

// w8^1 o and w8^3 o (the latter with its imaginary part negated), w8 = exp(-+ 2 pi i / 8)
template <bool INV, bool COMP>
__device__ __forceinline__ c2 w8_1(c2 o) {
    constexpr double r = 0.70710678118654752440084436210485;
    return INV ? c2{kmul2<COMP>(sub2(o.re, o.im), r), kmul2<COMP>(add2(o.re, o.im), r)}
               : c2{kmul2<COMP>(add2(o.re, o.im), r), kmul2<COMP>(sub2(o.im, o.re), r)};
}
// forward only: w8^3 o = (A, -B) with A = (o.im - o.re) r, B = (o.re + o.im) r; returns (A, B)
template <bool COMP>
__device__ __forceinline__ c2 w8_3cj(c2 o) {
    constexpr double r = 0.70710678118654752440084436210485;
    return c2{kmul2<COMP>(sub2(o.im, o.re), r), kmul2<COMP>(add2(o.re, o.im), r)};
}

template <bool INV, bool COMP>
__device__ __forceinline__ void pdft8(c2* v) {
    c2 e[4] = {v[0], v[2], v[4], v[6]};
    c2 o[4] = {v[1], v[3], v[5], v[7]};
    pdft4<INV>(e);
    pdft4<INV>(o);
    const c2 o1 = w8_1<INV, COMP>(o[1]);
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = addrot<INV>(e[2], o[2]);
    v[6] = subrot<INV>(e[2], o[2]);
    if constexpr (!INV) {
        const c2 t = w8_3cj<COMP>(o[3]);
        v[3] = add_cj(e[3], t);
        v[7] = sub_cj(e[3], t);
    } else {
        // inverse w8^3 o = (-(o.re + o.im) r, (o.re - o.im) r)
        constexpr double r = 0.70710678118654752440084436210485;
        const c2 t{kmul2<COMP>(add2(o[3].re, o[3].im), r), kmul2<COMP>(sub2(o[3].re, o[3].im), r)};
        v[3] = c2{sub2(e[3].re, t.re), add2(e[3].im, t.im)};
        v[7] = c2{add2(e[3].re, t.re), sub2(e[3].im, t.im)};
    }
}

// Radix 16 from two 8-point halves and the twiddles w16^k, k < 8.
template <bool INV, bool COMP>
__device__ __forceinline__ void pdft16(c2* v) {
    constexpr double c1 = 0.92387953251128675612818318939679, s1 = 0.38268343236508977172845998403040;
    constexpr double sg = INV ? 1.0 : -1.0;
    c2 e[8], o[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        e[m] = v[2 * m];
        o[m] = v[2 * m + 1];
    }
    pdft8<INV, COMP>(e);
    pdft8<INV, COMP>(o);
    c2 t[8];
    t[0] = o[0];
    t[1] = kcmul2<COMP>(o[1], c1, sg * s1);
    t[2] = w8_1<INV, COMP>(o[2]);
    t[3] = kcmul2<COMP>(o[3], s1, sg * c1);
    t[5] = kcmul2<COMP>(o[5], -s1, sg * c1);
    t[7] = kcmul2<COMP>(o[7], -c1, sg * s1);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k == 4) {
            v[4] = addrot<INV>(e[4], o[4]);
            v[12] = subrot<INV>(e[4], o[4]);
        } else if (k == 6) {
            // w16^6 = w8^3
            if constexpr (!INV) {
                const c2 u = w8_3cj<COMP>(o[6]);
                v[6] = add_cj(e[6], u);
                v[14] = sub_cj(e[6], u);
            } else {
                constexpr double r = 0.70710678118654752440084436210485;
                const c2 u{kmul2<COMP>(add2(o[6].re, o[6].im), r), kmul2<COMP>(sub2(o[6].re, o[6].im), r)};
                v[6] = c2{sub2(e[6].re, u.re), add2(e[6].im, u.im)};
                v[14] = c2{add2(e[6].re, u.re), sub2(e[6].im, u.im)};
            }
        } else {
            v[k] = e[k] + t[k];
            v[k + 8] = e[k] - t[k];
        }
    }
}

// The other radices (3, 5, 6, 7, 9, 10, 12) run the engine's butterflies on the paired type f2x.
template <int R, bool INV, bool COMP>
__device__ __forceinline__ void pdft(c2* v) {
    if constexpr (R == 2) {
        pdft2<INV>(v);
    } else if constexpr (R == 4) {
        pdft4<INV>(v);
    } else if constexpr (R == 8) {
        pdft8<INV, COMP>(v);
    } else if constexpr (R == 16) {
        pdft16<INV, COMP>(v);
    } else {
        cpx<f2x> w[R];
#pragma unroll
        for (int r = 0; r < R; ++r) w[r] = mk(f2x(v[r].re), f2x(v[r].im));
        dft<f2x, R, INV, COMP>(w);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = c2{w[r].re.v, w[r].im.v};
    }
}

// a w (forward, with the twiddle's remainder) or a conj(w) (inverse, rounded value only);
// tw points at the entry's rounded value (hr, hr, hi, hi), its remainder (lr, lr, li, li) sits
// `lo` vectors further on
template <bool INV>
__device__ __forceinline__ c2 ptwmul(c2 a, const float4* tw, int lo) {
    const float4 h = tw[0];
    const float2 hr{h.x, h.y}, hi{h.z, h.w};
    if constexpr (INV) {
        const float2 nar = mul2(a.re, make_float2(-1.f, -1.f));
        return c2{fma2(a.re, hr, mul2(a.im, hi)), fma2(a.im, hr, mul2(nar, hi))};
    } else {
        const float4 l = tw[lo];
        const float2 lr{l.x, l.y}, li{l.z, l.w};
        const float2 nai = mul2(a.im, make_float2(-1.f, -1.f));
        return c2{fma2(a.re, hr, fma2(nai, hi, fma2(a.re, lr, mul2(nai, li)))),
                  fma2(a.re, hi, fma2(a.im, hr, fma2(a.re, li, mul2(a.im, lr))))};
    }
}

// ------------------------------------------------------------------ tile accessors
// Pair p of a tile with COLS columns: natural (interleaved, as the TMA moves it) or split.
// A stage touches rows in runs with a compile-time stride: it loads rows j + r NB and stores
// rows o + r NS (r < R).  The accessors turn a run into one or two base rows per thread, so
// every access is a base register plus an immediate offset:
//   lbase<NB>(j)        physical row of j, the run's first load (the others add r NB);
//   sbase<NS, R>(o, j)  physical rows sb[0 .. NC) of the NC classes of the store run,
//                       cls<NS>(r) the class of row o + r NS (which then sits at sb[cls] + r NS).
template <int COLS>
struct NatPair {
    static constexpr int NC = 1;
    float* t;
    int p;
    template <int NB>
    __device__ __forceinline__ int lbase(int j) const {
        return j;
    }
    template <int NS, int R>
    __device__ __forceinline__ void sbase(int o, int, int* sb) const {
        sb[0] = sb[1] = o;
    }
    template <int NS>
    __device__ __forceinline__ static constexpr int cls(int) {
        return 0;
    }
    __device__ __forceinline__ c2 ldp(int n) const {
        const float4 x = *reinterpret_cast<const float4*>(t + (n * COLS + 2 * p) * 2);
        return c2{make_float2(x.x, x.z), make_float2(x.y, x.w)};
    }
    __device__ __forceinline__ void stp(int n, c2 v) const {
        *reinterpret_cast<float4*>(t + (n * COLS + 2 * p) * 2) = make_float4(v.re.x, v.im.x, v.re.y, v.im.y);
    }
};
// Split layout: row n lives at physical row n ^ ((n >> SH) & M) (SH = 0: no swizzle), M + 1 the
// rows of a 128-byte line: 2 for 8-column tiles (64-byte rows), 4 for 4-column tiles.
template <int COLS, int SH>
struct SplitPair {
    static constexpr int M = COLS == 4 ? 3 : 1;
    static constexpr int NC = SH > 0 ? M + 1 : 1;
    static_assert(SH == 0 || (1 << SH) > M, "the swizzle must stay below bit SH");
    float* t;
    int p;
    template <int NB>
    __device__ __forceinline__ int lbase(int j) const {
        if constexpr (SH > 0) {
            // j < NB and NB a multiple of (M + 1) 2^SH: adding r NB leaves the swizzle bits of j alone
            static_assert(NB % ((M + 1) << SH) == 0, "load run stride");
            return j ^ ((j >> SH) & M);
        } else {
            return j;
        }
    }
    template <int NS, int R>
    __device__ __forceinline__ void sbase(int o, int j, int* sb) const {
        if constexpr (SH == 0) {
            sb[0] = o;
        } else if constexpr (NS == 1) {
            // rows j R + r, R = 2^SH: the swizzle j & M flips the low bits of r, so the rows of
            // class c = r & M sit at o + (c ^ (j & M)) + (r - c)
            static_assert(R == (1 << SH), "store run of a first stage");
            const int x = j & M;
#pragma unroll
            for (int c = 0; c <= M; ++c) sb[c] = o + ((c ^ x) - c);
        } else {
            // NS a multiple of 2^SH: the swizzle of o + r NS is ((o >> SH) + r NS / 2^SH) & M, and
            // it only touches bits below SH, which r NS leaves clear
            static_assert(NS % (1 << SH) == 0, "store run stride");
            const int b = (o >> SH) & M;
#pragma unroll
            for (int c = 0; c <= M; ++c) sb[c] = o ^ ((b + c) & M);
        }
    }
    template <int NS>
    __device__ __forceinline__ static constexpr int cls(int r) {
        if constexpr (SH == 0)
            return 0;
        else if constexpr (NS == 1)
            return r & M;
        else
            return (r * (NS >> SH)) & M;
    }
    __device__ __forceinline__ c2 ldp(int n) const {
        const float4 x = *reinterpret_cast<const float4*>(t + (n * COLS + 2 * p) * 2);
        return c2{make_float2(x.x, x.y), make_float2(x.z, x.w)};
    }
    __device__ __forceinline__ void stp(int n, c2 v) const {
        *reinterpret_cast<float4*>(t + (n * COLS + 2 * p) * 2) = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
    }
};

#pragma nv_diag_suppress 177  // the inverse-table offsets are unused by the b passes
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};


__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// Tile buffers of a group of k_col_pair: the ring slots, a work buffer (PP = 1, 2), or three
// rotating buffers (PP = 3).
__host__ __device__ constexpr int pair_bufs(int nbuf, int pp) { return pp == 3 ? 3 : nbuf + (pp > 0 ? 1 : 0); }

// Stage tables of a column transform of radices R0 R1 R2 (R2 = 1: two stages), in entries of
// 32 bytes: stage 2 (R1, NS = R0) at f2, stage 3 (R2, NS = R0 R1) at f3; for MODE 2 the
// inverse transform's stages (radices reversed) follow unless they equal the forward ones.
template <int R0, int R1, int R2, int MODE>
struct PairTwLayout {
    static constexpr int N = R0 * R1 * R2;
    static constexpr int f2 = 0, f3 = (R1 - 1) * R0;
    static constexpr int fend = f3 + (R2 > 1 ? (R2 - 1) * R0 * R1 : 0);
    static constexpr bool share = MODE != 2 || (R2 > 1 ? R0 == R2 : R0 == R1);
    static constexpr int i2 = share ? f2 : fend;  // inverse stage 2: (R1, NS = R2), or (R0, NS = R1) if R2 = 1
    static constexpr int i3 = share ? f3 : fend + (R1 - 1) * R2;  // inverse stage 3: (R0, NS = R2 R1)
    static constexpr int total = share ? fend : (R2 > 1 ? i3 + (R0 - 1) * R2 * R1 : fend + (R0 - 1) * R1);
};

// Fill the table of stage (R, NS) of an N-point transform from the full TwPair table g: rounded
// values at dst, remainders at dst + lo.
template <int N, int R, int NS>
__device__ __forceinline__ void fill_pair_tw(float4* dst, int lo, const TwPair<float>* g, int nthreads) {
    for (int i = threadIdx.x; i < (R - 1) * NS; i += nthreads) {
        const int r = i / NS + 1, k = i - (r - 1) * NS;
        const TwPair<float> w = g[k * r * (N / (NS * R))];
        dst[i] = make_float4(w.h.re, w.h.re, w.h.im, w.h.im);
        dst[lo + i] = make_float4(w.l.re, w.l.re, w.l.im, w.l.im);
    }
}

template <int R0, int R1, int R2, int MODE>
__device__ __forceinline__ void fill_pair_tables(float4* tw, const TwPair<float>* g, int nthreads) {
    using L = PairTwLayout<R0, R1, R2, MODE>;
    constexpr int N = L::N;
    constexpr int lo = L::total;
    fill_pair_tw<N, R1, R0>(tw + L::f2, lo, g, nthreads);
    if constexpr (R2 > 1) fill_pair_tw<N, R2, R0 * R1>(tw + L::f3, lo, g, nthreads);
    if constexpr (!L::share) {
        if constexpr (R2 > 1) {
            fill_pair_tw<N, R1, R2>(tw + L::i2, lo, g, nthreads);
            fill_pair_tw<N, R0, R2 * R1>(tw + L::i3, lo, g, nthreads);
        } else {
            fill_pair_tw<N, R0, R1>(tw + L::i2, lo, g, nthreads);
        }
    }
}

// Barriers of one group of NT threads: the whole block when it is the only group, else the
// group's own named barrier (ids 1 .. G; 0 is the block-wide one).
template <int G, int NT>
struct GroupSync {
    int g;
    __device__ __forceinline__ void sync() const {
        if constexpr (G == 1)
            __syncthreads();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "n"(NT) : "memory");
    }
    // true on every thread of the group iff `pred` holds on every thread of the group
    __device__ __forceinline__ bool sync_and(bool pred) const {
        if constexpr (G == 1) {
            return __syncthreads_and(pred) != 0;
        } else {
            int r;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n"
                " selp.s32 %0, 1, 0, q;\n}"
                : "=r"(r)
                : "r"((int)pred), "r"(g + 1), "n"(NT)
                : "memory");
            return r != 0;
        }
    }
};

// One Stockham stage (radix R, sub-transforms of NS points) on the pair-butterflies
// j = j0 + t JSTEP, in place: every thread reads its inputs, the group waits, then writes.
// tw: the stage's table (unused for NS = 1).
// `hook` runs once every thread has read src (after the barrier); with a hook, each thread first
// orders its reads of src before later async-proxy writes to it (a TMA refill of the buffer).
// INPLACE = false: src and dst are different buffers and nobody writes src before the caller's
// next barrier, so the stage needs no barrier of its own (unless a hook must run after the reads).
template <int N, int R, int NS, int JSTEP, bool INV, bool COMP, bool INPLACE = true, class Src, class Dst,
          class Sync, class Hook = NoHook>
__device__ __forceinline__ void pstage(const Src& src, const Dst& dst, int j0, const float4* tw, int lo,
                                       const Sync& bar, const Hook& hook = Hook{}) {
    constexpr int NB = N / R;
    constexpr int BPT = (NB + JSTEP - 1) / JSTEP;
    constexpr bool GUARD = NB % JSTEP != 0;
    c2 v[BPT][R];
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
        const int j = j0 + t * JSTEP;
        if (GUARD && j >= NB) continue;
        const int lb = src.template lbase<NB>(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[t][r] = src.ldp(lb + r * NB);
    }
    constexpr bool HOOK = !std::is_same<Hook, NoHook>::value;
    if constexpr (HOOK) fence_proxy_async_smem();
    if constexpr (INPLACE || HOOK) bar.sync();
    hook();
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
        const int j = j0 + t * JSTEP;
        if (GUARD && j >= NB) continue;
        const int k = j % NS;
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[t][r] = ptwmul<INV>(v[t][r], tw + ((r - 1) * NS + k), lo);
        }
        pdft<R, INV, COMP>(v[t]);
        const int o = (j - k) * R + k;
        int sb[Dst::NC];
        dst.template sbase<NS, R>(o, j, sb);
#pragma unroll
        for (int r = 0; r < R; ++r) dst.stp(sb[Dst::template cls<NS>(r)] + r * NS, v[t][r]);
    }
}

// The last forward stage (radix R, NS = N / R: butterfly j's outputs sit at j + r NS), the
// Green multiply on each output, and the inverse transform's first stage (radix R, no
// twiddles), whose inputs are exactly the points this thread holds.
template <int N, int R, int JSTEP, bool INPLACE = true, class Sp, class Dp, class Green, class Sync>
__device__ __forceinline__ void pstage_pivot(const Sp& sp, const Dp& dp, int j0, const float4* tw, int lo,
                                             const Green& green, const Sync& bar) {
    constexpr int NS = N / R;
    constexpr int BPT = (NS + JSTEP - 1) / JSTEP;
    constexpr bool GUARD = NS % JSTEP != 0;
    c2 v[BPT][R];
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
        const int j = j0 + t * JSTEP;
        if (GUARD && j >= NS) continue;
        const int lb = sp.template lbase<NS>(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[t][r] = sp.ldp(lb + r * NS);
    }
    if constexpr (INPLACE) bar.sync();
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
        const int j = j0 + t * JSTEP;
        if (GUARD && j >= NS) continue;
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[t][r] = ptwmul<false>(v[t][r], tw + ((r - 1) * NS + j), lo);
        }
        pdft<R, false, true>(v[t]);
#pragma unroll
        for (int r = 0; r < R; ++r) green(j, r, j + r * NS, v[t][r]);
        pdft<R, true, false>(v[t]);
        int sb[Dp::NC];
        dp.template sbase<1, R>(j * R, j, sb);
#pragma unroll
        for (int r = 0; r < R; ++r) dp.stp(sb[Dp::template cls<1>(r)] + r, v[t][r]);
    }
}

// ------------------------------------------------------------------ the kernel
// Persistent CTAs of G groups of NT threads.  Each group is a worker with its own ring of NBUF
// tile buffers, filled and drained by TMA tensor copies (as k_col_tma) and synchronised by its
// own barrier; the groups of a CTA share the twiddle and |G_a|^2 tables, so several rings fit
// in one SM's shared memory beside one copy of the tables.  Worker w = blockIdx.x G + g takes
// the tiles w, w + W, ... (W workers), each an N x COLS block of the half spectrum; thread
// (p, j0) of a group transforms column pair p.
// MODE 0: forward along b, 1: inverse along b, 2: forward along a, Green multiply, E_H
// partial, inverse along a.  Every mbarrier wait is bounded (error word, early exit).
// PP > 0: each group also owns a work buffer, and the stages alternate between the ring slot and
// it (slot -> work -> slot -> ...), so a stage's reads and writes never meet and it needs one
// barrier instead of two.  The last stage writes the work buffer, which the TMA store drains.  The
// slot is refilled with the group's next tile as soon as the last stage has read it (PP = 1, one
// more barrier), or with the store (PP = 2).
// PP = 3: three buffers per group take turns: tile k arrives in buffer k % 3 and is transformed
// through buffer (k + 2) % 3, whose result the TMA store takes at the start of tile k + 1 (the
// barrier that starts a tile also ends the previous one); buffer (k + 1) % 3 is refilled with
// tile k + 1 once that store has read it, during tile k's second stage.  NBUF is unused.
template <int COLS, int NT, int R0, int R1, int R2, int MODE, int NBUF, int MINB, int G, int PP>
__global__ void __launch_bounds__(NT* G, MINB)
    k_col_pair(FastArgs<float> a, const __grid_constant__ CUtensorMap tmap, int ntiles, int chunks, int* err) {
    constexpr int N = R0 * R1 * R2;
    constexpr int P = COLS / 2;
    constexpr int JSTEP = NT / P;
    constexpr int BOXR = box_rows(N);
    constexpr int NBOX = N / BOXR;
    constexpr int TILE = N * COLS * 2;  // floats per tile buffer
    constexpr uint32_t TILE_BYTES = (uint32_t)N * COLS * 8;
    // row swizzle of the split layout (32- or 64-byte rows; power-of-two, mirrored outer radices)
    constexpr bool POW2 = (R0 & (R0 - 1)) == 0;
    constexpr int SH = COLS <= 8 && POW2 && (R2 > 1 ? R0 == R2 : R0 == R1) ? ilog2(R0) : 0;
    static_assert(COLS == 4 || COLS == 8 || COLS == 16, "tiles of 4, 8 or 16 columns");
    static_assert(SH == 0 || (R2 > 1 ? R0 == R2 : R0 == R1), "the row swizzle assumes mirrored radices");
    static_assert(PP == 0 || R2 > 1, "the ping-pong chain is written for three-stage transforms");
    constexpr int NB = pair_bufs(NBUF, PP);  // tile buffers (and mbarriers) per group
    using L = PairTwLayout<R0, R1, R2, MODE>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    float* bufs = reinterpret_cast<float*>(base);  // [G][NB][TILE]: the ring slots, then the work buffer
    float4* TW = reinterpret_cast<float4*>(bufs + G * NB * TILE);
    float4* GA = TW + 2 * L::total;  // MODE 2: |G_a|^2 per a index as (h, h, l, l)
    constexpr int lo = L::total;     // the twiddles' remainders follow their rounded values
    uint64_t* mbar = reinterpret_cast<uint64_t*>(GA + (MODE == 2 ? N : 0));  // [G][NB]
    double* red = reinterpret_cast<double*>(mbar + G * NB);
    fill_pair_tables<R0, R1, R2, MODE>(TW, MODE == 2 ? a.twpa : a.twpb, NT * G);
    if constexpr (MODE == 2)
        for (int k = threadIdx.x; k < N; k += NT * G) {
            const cpx<float> g = a.gsqa[k];
            GA[k] = make_float4(g.re, g.re, g.im, g.im);
        }
    if (threadIdx.x == 0) {
        for (int b = 0; b < G * NB; ++b) mbar_init(&mbar[b], 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int g = threadIdx.x / NT, lt = threadIdx.x - g * NT;
    const GroupSync<G, NT> bar{g};
    float* gbufs = bufs + g * NB * TILE;
    uint64_t* gbar = mbar + g * NB;
    const int worker = blockIdx.x * G + g, nworkers = gridDim.x * G;
    auto issue_load = [&](int t, int b) {
        const int line = t / chunks, c0 = (t - line * chunks) * COLS;
        float* dst = gbufs + b * TILE;
        mbar_arrive_expect_tx(&gbar[b], TILE_BYTES);
        for (int h = 0; h < NBOX; ++h) {
            if (MODE == 2)
                tma_load_3d(dst + h * BOXR * COLS * 2, &tmap, &gbar[b], 2 * c0, line, h * BOXR);
            else
                tma_load_3d(dst + h * BOXR * COLS * 2, &tmap, &gbar[b], 2 * c0, h * BOXR, line);
        }
    };
    auto issue_store = [&](int t, const float* src) {
        const int line = t / chunks, c0 = (t - line * chunks) * COLS;
        for (int h = 0; h < NBOX; ++h) {
            if (MODE == 2)
                tma_store_3d(&tmap, src + h * BOXR * COLS * 2, 2 * c0, line, h * BOXR);
            else
                tma_store_3d(&tmap, src + h * BOXR * COLS * 2, 2 * c0, h * BOXR, line);
        }
        tma_commit();
    };
    if (lt == 0)
        for (int b = 0; b < (PP == 3 ? 1 : NBUF); ++b) {
            const int t = worker + b * nworkers;
            if (t < ntiles) issue_load(t, b);
        }
    const int p = lt % P, j0 = lt / P;
    uint32_t parity = 0;
    float2 sum = make_float2(0.f, 0.f), comp = make_float2(0.f, 0.f);  // E_H, compensated across tiles
    int pend = -1, pend_b = 0;  // PP = 3: the tile whose result waits in buffer pend_b for its store
    for (int k = 0;; ++k) {
        const int t = worker + k * nworkers;
        if (t >= ntiles) break;
        const int b = PP == 3 ? k % 3 : k % NBUF;
        const uint32_t phase = PP == 3 ? (uint32_t)(k / 3) & 1u : (parity >> b) & 1u;
        const bool ok = mbar_wait(&gbar[b], phase, err);
        if constexpr (PP == 1 || PP == 2)
            if (lt == 0) tma_wait_read<0>();  // the work buffer is free once the last store has read it
        const bool all_ok = bar.sync_and(ok);
        if constexpr (PP == 3) {
            // every thread of the group has finished the previous tile (and fenced its writes)
            if (lt == 0 && pend >= 0) issue_store(pend, gbufs + pend_b * TILE);
            pend = -1;
        }
        if (!all_ok) {
            // a load did not arrive: wait (bounded again) for this group's copies still in flight, then leave
            if (lt == 0) {
                if constexpr (PP == 3) {
                    mbar_wait(&gbar[b], phase, err);
                } else {
                    for (int i = 0; i < NBUF; ++i) {
                        const int kk = k + i;
                        if (worker + kk * nworkers < ntiles)
                            mbar_wait(&gbar[kk % NBUF], (uint32_t)(kk / NBUF) & 1u, err);
                    }
                }
            }
            break;
        }
        parity ^= 1u << b;
        float* tile = gbufs + b * TILE;
        float* work = gbufs + (PP == 3 ? (k + 2) % 3 : NBUF) * TILE;  // PP > 0 only
        const NatPair<COLS> nat{tile, p};
        const SplitPair<COLS, SH> spl{tile, p};
        const NatPair<COLS> wnat{work, p};
        const SplitPair<COLS, SH> wsp{work, p};
        // PP = 1, 2: refill the slot with this group's tile k + NBUF once the last stage has read it
        auto refill = [&] {
            if (lt == 0) {
                const int tn = worker + (k + NBUF) * nworkers;
                if (tn < ntiles) issue_load(tn, b);
            }
        };
        // PP = 3, after the first stage: once the previous tile's store has read buffer (k + 1) % 3,
        // load tile k + 1 into it
        auto early = [&] {
            if constexpr (PP == 3)
                if (lt == 0) {
                    const int tn = t + nworkers;
                    if (tn < ntiles) {
                        tma_wait_read<0>();
                        issue_load(tn, (k + 1) % 3);
                    }
                }
        };
        if constexpr (MODE != 2) {
            constexpr bool INV = MODE == 1;
            constexpr bool COMP = !INV;
            if constexpr (PP > 0) {
                pstage<N, R0, 1, JSTEP, INV, COMP, false>(nat, wsp, j0, TW, lo, bar);
                bar.sync();
                early();
                pstage<N, R1, R0, JSTEP, INV, COMP, false>(wsp, spl, j0, TW + L::f2, lo, bar);
                bar.sync();
                if constexpr (PP == 1)
                    pstage<N, R2, R0 * R1, JSTEP, INV, COMP, false>(spl, wnat, j0, TW + L::f3, lo, bar, refill);
                else
                    pstage<N, R2, R0 * R1, JSTEP, INV, COMP, false>(spl, wnat, j0, TW + L::f3, lo, bar);
            } else if constexpr (R2 == 1) {
                pstage<N, R0, 1, JSTEP, INV, COMP>(nat, spl, j0, TW, lo, bar);
                bar.sync();
                pstage<N, R1, R0, JSTEP, INV, COMP>(spl, nat, j0, TW + L::f2, lo, bar);
            } else {
                pstage<N, R0, 1, JSTEP, INV, COMP>(nat, spl, j0, TW, lo, bar);
                bar.sync();
                pstage<N, R1, R0, JSTEP, INV, COMP>(spl, spl, j0, TW + L::f2, lo, bar);
                bar.sync();
                pstage<N, R2, R0 * R1, JSTEP, INV, COMP>(spl, nat, j0, TW + L::f3, lo, bar);
            }
        } else {
            const int line = t / chunks, c0 = (t - line * chunks) * COLS;
            const int ka = c0 + 2 * p, kb = ka + 1;  // the pair's c indices
            const cpx<float> gb = a.gsqb[line];
            const cpx<float> gca = a.gsqc[ka < a.nh ? ka : 0], gcb = a.gsqc[kb < a.nh ? kb : 0];
            // |G|^2 = |G_a|^2 + (|G_b|^2 + |G_c|^2): the b + c part once per tile, high and low apart
            const float2 gbc_h = make_float2(gb.re + gca.re, gb.re + gcb.re);
            const float2 gbc_l = make_float2(gb.im + gca.im, gb.im + gcb.im);
            const float2 gs = dup(a.green_scale);
            const bool zero_g = line == 0 && ka == 0;  // lane x holds G = 0 at a index 0
            float2 tsum = make_float2(0.f, 0.f);
            // output r of butterfly j, at a index k1 = j + r NS
            auto green = [&](int j, int r, int k1, c2& v) {
                const float4 gq = GA[k1];
                const float2 G2 = add2(add2(make_float2(gq.x, gq.y), gbc_h), add2(make_float2(gq.z, gq.w), gbc_l));
                // 1 / G2: hardware estimate r0 and one Newton step r0 + r0 (1 - G2 r0), written as
                // r0 - r0 ne with ne = G2 r0 - 1 exact through the fma
                float2 r0;
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0.x) : "f"(G2.x));
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0.y) : "f"(G2.y));
                const float2 m1 = make_float2(-1.f, -1.f);
                const float2 ne = fma2(G2, r0, m1);
                float2 inv = fma2(mul2(r0, m1), ne, r0);
                if (r == 0 && zero_g && j == 0) inv.x = 0.f;  // the neutralising background: G = 0 dropped
                tsum = fma2(fma2(v.im, v.im, mul2(v.re, v.re)), inv, tsum);
                const float2 sc = mul2(inv, gs);
                v = c2{mul2(v.re, sc), mul2(v.im, sc)};
            };
            if constexpr (PP > 0) {
                pstage<N, R0, 1, JSTEP, false, true, false>(nat, wsp, j0, TW, lo, bar);
                bar.sync();
                early();
                pstage<N, R1, R0, JSTEP, false, true, false>(wsp, spl, j0, TW + L::f2, lo, bar);
                bar.sync();
                pstage_pivot<N, R2, JSTEP, false>(spl, wsp, j0, TW + L::f3, lo, green, bar);
                bar.sync();
                pstage<N, R1, R2, JSTEP, true, false, false>(wsp, spl, j0, TW + L::i2, lo, bar);
                bar.sync();
                if constexpr (PP == 1)
                    pstage<N, R0, R2 * R1, JSTEP, true, false, false>(spl, wnat, j0, TW + L::i3, lo, bar, refill);
                else
                    pstage<N, R0, R2 * R1, JSTEP, true, false, false>(spl, wnat, j0, TW + L::i3, lo, bar);
            } else if constexpr (R2 == 1) {
                pstage<N, R0, 1, JSTEP, false, true>(nat, spl, j0, TW, lo, bar);
                bar.sync();
                pstage_pivot<N, R1, JSTEP>(spl, spl, j0, TW + L::f2, lo, green, bar);
                bar.sync();
                pstage<N, R0, R1, JSTEP, true, false>(spl, nat, j0, TW + L::i2, lo, bar);
            } else {
                pstage<N, R0, 1, JSTEP, false, true>(nat, spl, j0, TW, lo, bar);
                bar.sync();
                pstage<N, R1, R0, JSTEP, false, true>(spl, spl, j0, TW + L::f2, lo, bar);
                bar.sync();
                pstage_pivot<N, R2, JSTEP>(spl, spl, j0, TW + L::f3, lo, green, bar);
                bar.sync();
                pstage<N, R1, R2, JSTEP, true, false>(spl, spl, j0, TW + L::i2, lo, bar);
                bar.sync();
                pstage<N, R0, R2 * R1, JSTEP, true, false>(spl, nat, j0, TW + L::i3, lo, bar);
            }
            // multiplicity of the half spectrum: 1 at c index 0 and M, 2 between; a lane past the
            // spectrum (the row padding, whose contents are arbitrary) contributes nothing
            const float2 term = make_float2(ka < a.nh ? ((ka == 0 || ka == a.M) ? tsum.x : 2.f * tsum.x) : 0.f,
                                            kb < a.nh ? ((kb == 0 || kb == a.M) ? tsum.y : 2.f * tsum.y) : 0.f);
            const float2 y = sub2(term, comp);
            const float2 s2 = add2(sum, y);
            comp = sub2(sub2(s2, sum), y);
            sum = s2;
        }
        fence_proxy_async_smem();
        if constexpr (PP == 3) {
            pend = t;
            pend_b = (k + 2) % 3;
            continue;  // the next tile's first barrier ends this one
        }
        bar.sync();
        if (lt == 0) {
            if constexpr (PP > 0) {
                issue_store(t, work);
            }
            if constexpr (PP == 2) refill();
            if constexpr (PP == 0) {
                issue_store(t, tile);
                const int tn = worker + (k + NBUF) * nworkers;
                if (tn < ntiles) {
                    tma_wait_read<0>();  // the buffer is free once the store has read it
                    issue_load(tn, b);
                }
            }
        }
    }
    if constexpr (PP == 3) {
        bar.sync();
        if (lt == 0 && pend >= 0) issue_store(pend, gbufs + pend_b * TILE);
    }
    if (lt == 0) tma_wait_all();
    if constexpr (MODE == 2) {
        // the two lanes' compensated sums as one (value, error) pair: TwoSum of the values
        const float s = sum.x + sum.y;
        const float bb = s - sum.x;
        const float err2 = (sum.x - (s - bb)) + (sum.y - bb);
        const double bs = block_sum_comp(s, err2 - comp.x - comp.y, red);
        if (threadIdx.x == 0) a.eh_partials[blockIdx.x] = bs;
    }
}

// ------------------------------------------------------------------ configurations
template <int NT, int R0, int R1, int R2, int NBUF, int COLS, int MINB, int G = 1, int PP = 0>
struct ColPairCfg {
    static constexpr int cols = COLS, n = R0 * R1 * R2, groups = G;
    static size_t smem(int mode) {
        const int tw = mode == 2 ? PairTwLayout<R0, R1, R2, 2>::total : PairTwLayout<R0, R1, R2, 0>::total;
        return (size_t)G * pair_bufs(NBUF, PP) * n * COLS * 8 + (size_t)tw * 32 +
               (mode == 2 ? (size_t)n * 16 : 0) + G * pair_bufs(NBUF, PP) * 8 +
               (G * NT / 32) * sizeof(double) + 1024;
    }
    template <int MODE>
    static auto kernel() {
        return k_col_pair<COLS, NT, R0, R1, R2, MODE, NBUF, MINB, G, PP>;
    }
    static int resident(int mode) {
        static int r[3] = {0, 0, 0};
        if (r[mode] == 0) {
            int b = 0;
            cudaError_t e =
                mode == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel<0>(), NT * G, smem(0))
                : mode == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel<1>(), NT * G, smem(1))
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel<2>(), NT * G, smem(2));
            if (e != cudaSuccess) cudaGetLastError();
            r[mode] = e == cudaSuccess && b > 0 ? (b < MINB ? b : MINB) : 1;
        }
        return r[mode];
    }
    static cudaError_t configure(int optin) {
        cudaError_t e;
        if ((e = allow_max_dynamic_smem(kernel<0>(), optin))) return e;
        if ((e = allow_max_dynamic_smem(kernel<1>(), optin))) return e;
        return allow_max_dynamic_smem(kernel<2>(), optin);
    }
    static void launch(int mode, unsigned grid, const FastArgs<float>& a, const CUtensorMap& map, int ntiles,
                       int chunks, int* err, cudaStream_t s) {
        if (mode == 0) kernel<0>()<<<grid, NT * G, smem(0), s>>>(a, map, ntiles, chunks, err);
        if (mode == 1) kernel<1>()<<<grid, NT * G, smem(1), s>>>(a, map, ntiles, chunks, err);
        if (mode == 2) kernel<2>()<<<grid, NT * G, smem(2), s>>>(a, map, ntiles, chunks, err);
    }
};

// Paired variants by line length: one group per CTA (one or two ring slots, several CTAs per
// SM), or one CTA per SM of several groups sharing the tables, with or without work buffers.
// Lengths that are not powers of two take 16-column tiles (128-byte rows: conflict-free without a
// swizzle) or, for 840, unswizzled 8-column tiles, and their butterflies run on the paired type.
template <class F>
bool with_col_pair_cfg(int n, int variant, F&& f) {
    switch (n) {
        case 256:  // 8 x 4 x 8: 32, 64 and 32 butterflies per column, none idle at 32 per pair
            if (variant == 1) f(ColPairCfg<128, 8, 4, 8, 2, 8, 1, 6>{});
            else if (variant == 2) f(ColPairCfg<128, 8, 4, 8, 1, 8, 1, 6, 1>{});
            else if (variant == 3) f(ColPairCfg<128, 8, 4, 8, 2, 8, 1, 4, 2>{});
            else if (variant == 4) f(ColPairCfg<64, 8, 4, 8, 2, 4, 1, 8, 2>{});
            else if (variant == 5) f(ColPairCfg<64, 8, 4, 8, 2, 4, 1, 8, 3>{});
            else f(ColPairCfg<128, 8, 4, 8, 2, 8, 3>{});
            return true;
        case 360:  // 16-column tiles, one group of 480 threads: 60, 36 and 60 (or 36, 60, 60) butterflies
            if (variant == 1) f(ColPairCfg<480, 10, 6, 6, 2, 16, 1, 1, 3>{});
            else f(ColPairCfg<480, 6, 10, 6, 2, 16, 1, 1, 3>{});
            return true;
        case 420:  // 16-column tiles, one group of 576 threads: 42, 60 and 70 butterflies per column and stage
            f(ColPairCfg<576, 10, 7, 6, 2, 16, 1, 1, 3>{});
            return true;
        case 840:  // 8-column tiles, 480 threads: 70, 84 and 120 butterflies per column and stage; one slot
            f(ColPairCfg<480, 12, 10, 7, 1, 8, 1, 1, 1>{});
            return true;
        case 512:
            if (variant == 1) f(ColPairCfg<256, 8, 8, 8, 2, 8, 1, 3>{});
            else if (variant == 2) f(ColPairCfg<256, 8, 8, 8, 3, 8, 1, 2>{});
            else if (variant == 3) f(ColPairCfg<256, 8, 8, 8, 1, 8, 1, 3, 1>{});
            else if (variant == 4) f(ColPairCfg<256, 8, 8, 8, 2, 8, 1, 2, 2>{});
            else if (variant == 5) f(ColPairCfg<256, 8, 8, 8, 2, 8, 1, 2, 3>{});
            else f(ColPairCfg<256, 8, 8, 8, 2, 8, 2>{});
            return true;
        default: return false;
    }
}

}  // namespace

int col_pair_variants(int n) {
    switch (n) {
        case 256: case 512: return 6;
        case 360: return 2;
        case 420: case 840: return 1;
        default: return 0;
    }
}

bool col_pair_available(const Plan& p, int axis) {
    return p.prec != HARTREE_FP64 && p.tma_ok && col_pair_variants(p.n[axis]) > 0;
}

cudaError_t configure_col_pair(const Plan& p, int optin) {
    cudaError_t e = cudaSuccess;
    for (int ax = 0; ax < 2; ++ax) {
        if (!col_pair_available(p, ax)) continue;
        for (int v = 0; v < col_pair_variants(p.n[ax]) && e == cudaSuccess; ++v)
            with_col_pair_cfg(p.n[ax], v, [&](auto c) {
                if (c.smem(2) > (size_t)optin) e = cudaErrorInvalidConfiguration;
                if (e == cudaSuccess) e = c.configure(optin);
            });
    }
    return e;
}

long long launch_col_pair(const Plan& p, int pass, int variant, const FastArgs<float>& a, cudaStream_t s) {
    const int axis = pass == 2 ? 0 : 1;
    long long grid = -1;
    with_col_pair_cfg(p.n[axis], variant, [&](auto c) {
        const int chunks = (p.nh + c.cols - 1) / c.cols;
        const int ntiles = p.n[1 - axis] * chunks;
        const int mode = pass == 1 ? 0 : (pass == 3 ? 1 : 2);
        const int slots = c.resident(mode) * p.sm_count;
        const int need = (ntiles + c.groups - 1) / c.groups;  // CTAs that all have work
        grid = need < slots ? need : slots;
        const CUtensorMap& map = c.cols == 16  ? (axis == 0 ? p.tmap_a : p.tmap_b)
                                 : c.cols == 8 ? (axis == 0 ? p.tmap_a8 : p.tmap_b8)
                                               : (axis == 0 ? p.tmap_a4 : p.tmap_b4);
        c.launch(mode, (unsigned)grid, a, map, ntiles, chunks, p.d_err, s);
    });
    return grid;
}

}  // namespace hartree
