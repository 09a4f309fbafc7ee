// fast_passes.cu -- compile-time specialised Poisson passes for line lengths
// 16 .. 1024 that are powers of two (the cubic 32^3, 256^3 and 512^3 grids) and for
// the mixed lengths of the other workloads (360, 384, 400, 420, 840 and their halves).
//
// Same five-pass schedule as poisson.cu (Sec. 2.1 / Sec. 3.2.4: c, b, a with
// the Green multiply and E_H, b^-1, c^-1), but every radix, stage stride and
// thread->butterfly map is a compile-time constant:
//   * each thread owns BPT butterflies per stage and keeps them in registers;
//     a stage reads all of them, waits once, and writes them back in place,
//     so one shared-memory tile (no ping-pong) holds the lines;
//   * the first stage reads HBM directly and the last stage writes HBM
//     directly (coalesced: columns for the b/a passes, lines for the c passes);
//   * twiddles live in shared memory as FP32 high/low pairs, and forward
//     butterflies use them and split constants, so FP32 rounding carries no
//     systematic magnitude bias into E_H; the inverse transforms only shape
//     V_H and use the plain values.
#include <algorithm>
#include <type_traits>

#include "atoms_dev.cuh"
#include "internal.cuh"
#include "tma.cuh"

namespace hartree {

namespace {

// a w (or a conj(w) when inv).  COMP: FP32 product with the twiddle's low part.
template <bool COMP = true, typename T>
__device__ __forceinline__ cpx<T> twmul(cpx<T> a, const TwPair<T>& w, bool inv) {
    const T hi_im = inv ? -w.h.im : w.h.im;
    const T lo_im = inv ? -w.l.im : w.l.im;
    if constexpr (sizeof(T) == 4 && COMP) {
        const float tr = a.re * w.l.re - a.im * lo_im;
        const float ti = a.re * lo_im + a.im * w.l.re;
        return mk(fmaf(a.re, w.h.re, fmaf(-a.im, hi_im, tr)), fmaf(a.re, hi_im, fmaf(a.im, w.h.re, ti)));
    } else if constexpr (std::is_same<T, f2x>::value && COMP) {
        const T tr = a.re * w.l.re - a.im * lo_im;
        const T ti = a.re * lo_im + a.im * w.l.re;
        return mk(fma_t(a.re, w.h.re, fma_t(-a.im, hi_im, tr)), fma_t(a.re, hi_im, fma_t(a.im, w.h.re, ti)));
    } else {
        return mk(a.re * w.h.re - a.im * hi_im, a.re * hi_im + a.im * w.h.re);
    }
}

// 1 / x rounded to nearest: the reciprocal instruction sequence, not the general division
__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_rn(double x) { return __drcp_rn(x); }

template <int R0, int R1, int R2>
struct RP {
    static constexpr int N = R0 * R1 * R2;
    static constexpr int NST = R2 == 1 ? 2 : 3;
};

// ------------------------------------------------------------------ accessors
template <typename T, int COLS>
struct ColSmem {  // [n][COLS]
    cpx<T>* p;
    __device__ __forceinline__ cpx<T> ld_(int col, int n) const { return p[n * COLS + col]; }
    __device__ __forceinline__ void st_(int col, int n, cpx<T> v) const { p[n * COLS + col] = v; }
};

template <typename T>
struct ColGlobal {  // column `col` of a strided tile; inactive columns read 0 and store nothing
    cpx<T>* p;
    long long sn;
    int nc;
    __device__ __forceinline__ cpx<T> ld_(int col, int n) const {
        return col < nc ? p[(long long)n * sn + col] : mk(T(0), T(0));
    }
    __device__ __forceinline__ void st_(int col, int n, cpx<T> v) const {
        if (col < nc) p[(long long)n * sn + col] = v;
    }
};

__device__ __forceinline__ int pidx(int n) { return n + (n >> 4); }  // one pad slot per 16 elements

template <typename T>
struct LineSmem {  // one line, padded
    cpx<T>* p;
    __device__ __forceinline__ cpx<T> ld_(int, int n) const { return p[pidx(n)]; }
    __device__ __forceinline__ void st_(int, int n, cpx<T> v) const { p[pidx(n)] = v; }
};

template <typename T>
struct LineRealIn {  // z[n] = rho[2n] + i rho[2n+1]
    const cpx<T>* z;
    bool act;
    __device__ __forceinline__ cpx<T> ld_(int, int n) const { return act ? z[n] : mk(T(0), T(0)); }
};

template <typename T>
struct LineRealOut {
    cpx<T>* z;
    bool act;
    __device__ __forceinline__ void st_(int, int n, cpx<T> v) const {
        if (act) z[n] = v;
    }
};

// Z[k] = (X[k] + conj X[M-k]) + i w^-k (X[k] - conj X[M-k]) from the half spectrum (c2r pre-step)
template <typename T, class Tw = const TwPair<T>*>
struct LineC2RIn {
    const cpx<T>* x;
    Tw tw;  // exp(-2 pi i k / N3)
    int M;
    bool act;
    __device__ __forceinline__ cpx<T> ld_(int, int k) const {
        if (!act) return mk(T(0), T(0));
        const cpx<T> x1 = x[k];
        const cpx<T> x2 = conjg(x[M - k]);
        const cpx<T> Ep = x1 + x2;
        const cpx<T> Op = twmul<false>(x1 - x2, tw[k], true);
        return mk(Ep.re - Op.im, Ep.im + Op.re);
    }
};

struct NoPost {
    template <typename T>
    __device__ __forceinline__ void operator()(int, int, cpx<T>&) const {}
};

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Twiddles held as rounded values only (the inverse transforms use no low parts).
template <typename T>
struct TwHi {
    const cpx<T>* p;
    __device__ __forceinline__ TwPair<T> operator[](int i) const { return TwPair<T>{p[i], mk(T(0), T(0))}; }
};

// Twiddles of one Stockham stage in the order the stage reads them.  A stage of radix R on
// sub-transforms of NS points applies w^(k r N / (NS R)) to output r of butterfly k; its
// table holds that factor at entry (r - 1) NS + k, so the lanes of a warp (consecutive k)
// read consecutive entries, which shared memory serves without bank conflicts, instead of
// entries k r apart in the transform's full table.  E: TwPair (compensated) or cpx (rounded).
template <class E, int NS>
struct StageTw {
    const E* p;
};

template <class Tw>
struct is_stage_tw : std::false_type {};
template <class E, int NS>
struct is_stage_tw<StageTw<E, NS>> : std::true_type {};

// The twiddle of output r of butterfly k; idx is its index in a full table.
template <class Tw>
__device__ __forceinline__ decltype(auto) tw_fetch(const Tw& TW, int, int, int idx) {
    return TW[idx];
}
template <typename T, int NS>
__device__ __forceinline__ TwPair<T> tw_fetch(const StageTw<TwPair<T>, NS>& TW, int k, int r, int) {
    return TW.p[(r - 1) * NS + k];
}
template <typename T, int NS>
__device__ __forceinline__ TwPair<T> tw_fetch(const StageTw<cpx<T>, NS>& TW, int k, int r, int) {
    return TwPair<T>{TW.p[(r - 1) * NS + k], mk(T(0), T(0))};
}

// Fill the StageTw table of stage (R, NS) of an N-point transform whose twiddle w^e is get(e TWS).
template <int N, int R, int NS, int TWS, class E, class Get>
__device__ __forceinline__ void fill_stage_tw(E* dst, const Get& get) {
    for (int i = threadIdx.x; i < (R - 1) * NS; i += blockDim.x) {
        const int r = i / NS + 1, k = i - (r - 1) * NS;
        dst[i] = get((k * r * (N / (NS * R))) * TWS);
    }
}

// Shared twiddle tables of the line (c) passes, radices R0 R1 R2 (R2 = 1: two stages): the
// second and third stages' StageTw tables, then the r2c post-processing factors w_2M^k for
// k <= M/2 (r2c) or the c2r pre-processing factors for k < M.
template <int R0, int R1, int R2>
struct LineTwLayout {
    static constexpr int M = R0 * R1 * R2;
    static constexpr int s2 = (R1 - 1) * R0;
    static constexpr int s3 = R2 > 1 ? (R2 - 1) * R0 * R1 : 0;
    static constexpr int fwd = s2 + s3 + M / 2 + 1;  // r2c entries (TwPair)
    static constexpr int inv = s2 + s3 + M;          // c2r entries (cpx, rounded)
};

// Stage twiddle tables and the twiddles of the r2c post-processing (compensated pairs).
template <typename T, int R0, int R1, int R2>
__device__ __forceinline__ void fill_line_tw_fwd(TwPair<T>* tw, const TwPair<T>* g) {
    using L = LineTwLayout<R0, R1, R2>;
    auto get = [&](int e) { return g[e]; };
    fill_stage_tw<L::M, R1, R0, 2>(tw, get);
    if constexpr (R2 > 1) fill_stage_tw<L::M, R2, R0 * R1, 2>(tw + L::s2, get);
    for (int k = threadIdx.x; k <= L::M / 2; k += blockDim.x) tw[L::s2 + L::s3 + k] = g[k];
}
// The same for the c2r pass (rounded values; its pre-processing reads k < M).
template <typename T, int R0, int R1, int R2>
__device__ __forceinline__ void fill_line_tw_inv(cpx<T>* tw, const TwPair<T>* g) {
    using L = LineTwLayout<R0, R1, R2>;
    auto get = [&](int e) { return g[e].h; };
    fill_stage_tw<L::M, R1, R0, 2>(tw, get);
    if constexpr (R2 > 1) fill_stage_tw<L::M, R2, R0 * R1, 2>(tw + L::s2, get);
    for (int k = threadIdx.x; k < L::M; k += blockDim.x) tw[L::s2 + L::s3 + k] = g[k].h;
}

// Shared twiddle tables of the column (b, a) passes, radices R0 R1 R2 (R2 = 1: two stages):
// the StageTw tables of the forward (or MODE 1 inverse) stages 2 and 3, then for MODE 2 those
// of the inverse transform, whose radices run in the reverse order (R2 R1 R0); an inverse
// table equal to a forward one (R0 = R2, or R0 = R1 for two stages) is shared.
template <int R0, int R1, int R2, int MODE>
struct ColTwLayout {
    static constexpr int N = R0 * R1 * R2;
    static constexpr int f2 = 0, f3 = (R1 - 1) * R0;  // T(R1, NS = R0), T(R2, NS = R0 R1)
    static constexpr int fend = f3 + (R2 > 1 ? (R2 - 1) * R0 * R1 : 0);
    static constexpr bool share = MODE != 2 || (R2 > 1 ? R0 == R2 : R0 == R1);
    // MODE 2 inverse: R2 > 1: T(R1, NS = R2) at i2, T(R0, NS = R2 R1) at i3; R2 = 1: T(R0, NS = R1) at i2
    static constexpr int i2 = share ? f2 : fend;
    static constexpr int i3 = share ? f3 : fend + (R1 - 1) * R2;
    static constexpr int total = share ? fend : (R2 > 1 ? i3 + (R0 - 1) * R2 * R1 : fend + (R0 - 1) * R1);
};

template <typename T, int R0, int R1, int R2, int MODE>
__device__ __forceinline__ void fill_col_tw(TwPair<T>* tw, const TwPair<T>* g) {
    using L = ColTwLayout<R0, R1, R2, MODE>;
    auto get = [&](int e) { return g[e]; };
    fill_stage_tw<L::N, R1, R0, 1>(tw + L::f2, get);
    if constexpr (R2 > 1) fill_stage_tw<L::N, R2, R0 * R1, 1>(tw + L::f3, get);
    if constexpr (!L::share) {
        if constexpr (R2 > 1) {
            fill_stage_tw<L::N, R1, R2, 1>(tw + L::i2, get);
            fill_stage_tw<L::N, R0, R2 * R1, 1>(tw + L::i3, get);
        } else {
            fill_stage_tw<L::N, R0, R1, 1>(tw + L::i2, get);
        }
    }
}

// One Stockham stage (radix R, sub-transform NS) for the BPT butterflies
// j = j0 + t JSTEP of this thread; SYNC when src and dst share storage (or when
// `hook` must run once every thread has read src: it runs after that barrier).
template <typename T, int N, int R, int NS, int BPT, int JSTEP, int TWS, bool INV, bool SYNC, class Src, class Dst,
          class Post, class Tw, class Hook = NoHook>
__device__ __forceinline__ void fstage(const Src& src, const Dst& dst, int col, int j0, const Tw& TW,
                                       const Post& post, const Hook& hook = Hook{}) {
    constexpr int NB = N / R;
    constexpr bool GUARD = NB % JSTEP != 0;  // mixed radices: the last round of butterflies is partial
    cpx<T> v[BPT][R];
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
        const int j = j0 + t * JSTEP;
        if (GUARD && j >= NB) continue;
#pragma unroll
        for (int r = 0; r < R; ++r) v[t][r] = src.ld_(col, j + r * NB);
    }
    if constexpr (SYNC) {
        // a hook may hand src to the async proxy (a bulk copy refilling it): order this
        // thread's reads of src before that write
        if constexpr (!std::is_same<Hook, NoHook>::value) fence_proxy_async_smem();
        __syncthreads();
        hook();
    }
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
        const int j = j0 + t * JSTEP;
        if (GUARD && j >= NB) continue;
        const int k = j % NS;
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                if constexpr (is_stage_tw<Tw>::value)
                    v[t][r] = twmul<!INV>(v[t][r], tw_fetch(TW, k, r, 0), INV);
                else
                    v[t][r] = twmul<!INV>(v[t][r], TW[(k * r * (N / (NS * R))) * TWS], INV);
            }
        }
        dft<T, R, INV, !INV>(v[t]);
        const int o = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            post(col, o + r * NS, v[t][r]);
            dst.st_(col, o + r * NS, v[t][r]);
        }
    }
}

// Whole transform of a column tile: stage 0 from src, the rest in place in `sm`, the last
// stage into dst, twiddles w^e at tw[e] (a full table).  Threads: col, j0 in [0, JSTEP).
template <typename T, int R0, int R1, int R2, int JSTEP, bool INV, bool FIRST_SYNC, class Src, class Sm, class Dst>
__device__ __forceinline__ void ftransform(const Src& src, const Sm& sm, const Dst& dst, int col, int j0,
                                           const TwPair<T>* tw) {
    constexpr int N = R0 * R1 * R2;
    constexpr int B0 = (N / R0 + JSTEP - 1) / JSTEP, B1 = (N / R1 + JSTEP - 1) / JSTEP,
                  B2 = (N / R2 + JSTEP - 1) / JSTEP;
    fstage<T, N, R0, 1, B0, JSTEP, 1, INV, FIRST_SYNC>(src, sm, col, j0, tw, NoPost{});
    __syncthreads();
    if constexpr (R2 == 1) {
        fstage<T, N, R1, R0, B1, JSTEP, 1, INV, true>(sm, dst, col, j0, tw, NoPost{});
    } else {
        fstage<T, N, R1, R0, B1, JSTEP, 1, INV, true>(sm, sm, col, j0, tw, NoPost{});
        __syncthreads();
        fstage<T, N, R2, R0 * R1, B2, JSTEP, 1, INV, true>(sm, dst, col, j0, tw, NoPost{});
    }
}

// The twiddles of one stage of a column transform: with STAGE, its StageTw table at tw + off
// (ColTwLayout); else the full table tw.
template <bool STAGE, int NS, class E>
__device__ __forceinline__ auto stage_tw(const E* tw, int off) {
    if constexpr (STAGE)
        return StageTw<E, NS>{tw + off};
    else
        return tw;
}

// ftransform for the line passes: the twiddles of the second and third stages come from
// their StageTw tables at tw (LineTwLayout order); E is TwPair (forward) or cpx (inverse).
template <typename T, int R0, int R1, int R2, int JSTEP, bool INV, bool FIRST_SYNC, class Src, class Sm, class Dst,
          class E, class Hook = NoHook>
__device__ __forceinline__ void line_ftransform(const Src& src, const Sm& sm, const Dst& dst, int j0, const E* tw,
                                                const Hook& hook = Hook{}) {
    constexpr int N = R0 * R1 * R2;
    constexpr int B0 = (N / R0 + JSTEP - 1) / JSTEP, B1 = (N / R1 + JSTEP - 1) / JSTEP,
                  B2 = (N / R2 + JSTEP - 1) / JSTEP;
    const StageTw<E, R0> tw2{tw};
    fstage<T, N, R0, 1, B0, JSTEP, 2, INV, FIRST_SYNC>(src, sm, 0, j0, tw2, NoPost{}, hook);  // no twiddles
    __syncthreads();
    if constexpr (R2 == 1) {
        fstage<T, N, R1, R0, B1, JSTEP, 2, INV, true>(sm, dst, 0, j0, tw2, NoPost{});
    } else {
        fstage<T, N, R1, R0, B1, JSTEP, 2, INV, true>(sm, sm, 0, j0, tw2, NoPost{});
        __syncthreads();
        const StageTw<E, R0 * R1> tw3{tw + LineTwLayout<R0, R1, R2>::s2};
        fstage<T, N, R2, R0 * R1, B2, JSTEP, 2, INV, true>(sm, dst, 0, j0, tw3, NoPost{});
    }
}

// The last forward stage (radix R, so j < N / R, k = j and the outputs sit at
// j + r N / R), the Green multiply `green` on each output, and the first
// stage of the inverse transform.  The inverse takes the radices in the
// reverse order, so its first stage (radix R, no twiddles) reads exactly the
// points the forward stage leaves in this thread's registers: the two stages
// and the multiply run back to back with no shared-memory round trip.
template <typename T, int N, int R, int BPT, int JSTEP, class Sm, class Tw, class Green>
__device__ __forceinline__ void fstage_green_pivot(const Sm& sm, int col, int j0, const Tw& TW, const Green& green) {
    constexpr int NS = N / R;
    constexpr bool GUARD = NS % JSTEP != 0;
    cpx<T> v[BPT][R];
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
        const int j = j0 + t * JSTEP;
        if (GUARD && j >= NS) continue;
#pragma unroll
        for (int r = 0; r < R; ++r) v[t][r] = sm.ld_(col, j + r * NS);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
        const int j = j0 + t * JSTEP;
        if (GUARD && j >= NS) continue;
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[t][r] = twmul<true>(v[t][r], tw_fetch(TW, j, r, j * r), false);
        }
        dft<T, R, false, true>(v[t]);
#pragma unroll
        for (int r = 0; r < R; ++r) green(col, j + r * NS, v[t][r]);
        dft<T, R, true, false>(v[t]);
#pragma unroll
        for (int r = 0; r < R; ++r) sm.st_(col, j * R + r, v[t][r]);
    }
}

// Forward transform of a tile (stage 0 from src), `green` on the spectrum, and
// the inverse transform (radices reversed; last stage into dst), in place in sm.
// STAGE: twiddles from the ColTwLayout<R0, R1, R2, 2> tables at tw, else from the full table tw.
template <typename T, int R0, int R1, int R2, int JSTEP, bool FIRST_SYNC, bool STAGE, class Src, class Sm,
          class Dst, class Green>
__device__ __forceinline__ void ftransform_green(const Src& src, const Sm& sm, const Dst& dst, int col, int j0,
                                                 const TwPair<T>* tw, const Green& green) {
    using L = ColTwLayout<R0, R1, R2, 2>;
    constexpr int N = R0 * R1 * R2;
    constexpr int B0 = (N / R0 + JSTEP - 1) / JSTEP, B1 = (N / R1 + JSTEP - 1) / JSTEP,
                  B2 = (N / R2 + JSTEP - 1) / JSTEP;
    const auto tw2 = stage_tw<STAGE, R0>(tw, L::f2);
    fstage<T, N, R0, 1, B0, JSTEP, 1, false, FIRST_SYNC>(src, sm, col, j0, tw2, NoPost{});  // no twiddles
    __syncthreads();
    if constexpr (R2 == 1) {
        fstage_green_pivot<T, N, R1, B1, JSTEP>(sm, col, j0, tw2, green);
        __syncthreads();
        fstage<T, N, R0, R1, B0, JSTEP, 1, true, true>(sm, dst, col, j0, stage_tw<STAGE, R1>(tw, L::i2), NoPost{});
    } else {
        fstage<T, N, R1, R0, B1, JSTEP, 1, false, true>(sm, sm, col, j0, tw2, NoPost{});
        __syncthreads();
        fstage_green_pivot<T, N, R2, B2, JSTEP>(sm, col, j0, stage_tw<STAGE, R0 * R1>(tw, L::f3), green);
        __syncthreads();
        fstage<T, N, R1, R2, B1, JSTEP, 1, true, true>(sm, sm, col, j0, stage_tw<STAGE, R2>(tw, L::i2), NoPost{});
        __syncthreads();
        fstage<T, N, R0, R2 * R1, B0, JSTEP, 1, true, true>(sm, dst, col, j0, stage_tw<STAGE, R2 * R1>(tw, L::i3),
                                                           NoPost{});
    }
}

// ------------------------------------------------------------------ b and a passes
// MODE 0: forward, 1: inverse (b axis);  2: forward, Green, E_H, inverse (a axis)
// Resident CTAs per SM asked of the register allocator: at least two, so one
// CTA's loads overlap another's butterflies.
template <int NT>
constexpr int min_ctas() {
    return NT >= 512 ? 2 : (NT >= 256 ? 3 : 4);
}

template <typename T, int COLS, int NT, int R0, int R1, int R2, int MODE>
__global__ void __launch_bounds__(NT, MODE == 2 && min_ctas<NT>() > 2 ? min_ctas<NT>() - 1 : min_ctas<NT>())
    k_col_fast(FastArgs<T> a) {
    constexpr int N = R0 * R1 * R2;
    constexpr int JSTEP = NT / COLS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);
    TwPair<T>* TW = reinterpret_cast<TwPair<T>*>(S + N * COLS);
    const TwPair<T>* twg = MODE == 2 ? a.twpa : a.twpb;
    for (int k = threadIdx.x; k < N; k += NT) TW[k] = twg[k];
    const int chunks = MODE == 2 ? a.a_chunks : a.b_chunks;
    const int line = blockIdx.x / chunks;
    const int c0 = (blockIdx.x - line * chunks) * COLS;
    const int nc = min(COLS, a.nh - c0);
    ColGlobal<T> g{MODE == 2 ? a.W + (long long)line * a.ldc + c0 : a.W + (long long)line * a.n2 * a.ldc + c0,
                   MODE == 2 ? (long long)a.n2 * a.ldc : (long long)a.ldc, nc};
    ColSmem<T, COLS> sm{S};
    const int col = threadIdx.x % COLS, j0 = threadIdx.x / COLS;
    __syncthreads();
    if constexpr (MODE != 2) {
        ftransform<T, R0, R1, R2, JSTEP, MODE == 1, false>(g, sm, g, col, j0, static_cast<const TwPair<T>*>(TW));
    } else {
        // forward, then 4 pi / |G|^2 / N and the E_H partial on the last stage's outputs
        const cpx<T> gb = a.gsqb[line];
        const int k3 = c0 + col;
        const cpx<T> gc = a.gsqc[k3 < a.nh ? k3 : 0];
        const T mult = (k3 == 0 || k3 == a.M) ? T(1) : T(2);
        T sum = T(0), comp = T(0);
        auto green = [&](int c, int k1, cpx<T>& v) {
            const cpx<T> ga = a.gsqa[k1];
            const T G2 = ((ga.re + gb.re) + gc.re) + ((ga.im + gb.im) + gc.im);
            const T inv = (G2 > T(0)) ? recip_rn(G2) : T(0);
            if (c < nc) {
                const T term = mult * (v.re * v.re + v.im * v.im) * inv - comp;
                const T t = sum + term;
                comp = (t - sum) - term;
                sum = t;
            }
            v = scale(v, inv * a.green_scale);
        };
        ftransform_green<T, R0, R1, R2, JSTEP, false, false>(g, sm, g, col, j0, static_cast<const TwPair<T>*>(TW),
                                                             green);
        const double bs = block_sum_comp(sum, -comp, red);
        if (threadIdx.x == 0) a.eh_partials[blockIdx.x] = bs;
    }
}

// ------------------------------------------------------------------ TMA-streamed b and a passes (FP32)
// Persistent CTAs walk the tiles blockIdx.x, blockIdx.x + gridDim.x, ... through
// a ring of NBUF shared-memory tile buffers.  Thread 0 keeps NBUF - 1 tile
// loads in flight (cp.async.bulk.tensor, completion counted on one mbarrier
// per buffer) while the CTA transforms the current tile in place, then writes
// it back with a bulk tensor store and refills the buffer once the store has
// read it.  No load or store instruction touches HBM from the threads
// themselves, and memory traffic overlaps the butterflies of the other tiles.
// A wait that does not complete within kSpinLimit probes sets the error word
// and ends the CTA's loop (all threads agree through __syncthreads_and).
template <int COLS, int NT, int R0, int R1, int R2, int MODE, int NBUF, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_col_tma(FastArgs<float> a, const __grid_constant__ CUtensorMap tmap, int ntiles, int chunks, int* err) {
    constexpr int N = R0 * R1 * R2;
    constexpr int JSTEP = NT / COLS;
    constexpr int BOXR = box_rows(N);  // rows per bulk copy (box dimension limit 256)
    constexpr int NBOX = N / BOXR;
    constexpr uint32_t TILE_BYTES = (uint32_t)N * COLS * 8;
    // All shared memory is dynamic (a static array would shift the dynamic base), and the tile
    // buffers start on a 1024-byte boundary (bulk tensor copies need 128-byte aligned buffers).
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    cpx<float>* bufs = reinterpret_cast<cpx<float>*>(base);
    TwPair<float>* TW = reinterpret_cast<TwPair<float>*>(bufs + NBUF * N * COLS);
    // the a pass (MODE 2) reads its twiddles from stage-ordered tables, the b passes from the full table
    uint64_t* mbar = reinterpret_cast<uint64_t*>(TW + (MODE == 2 ? ColTwLayout<R0, R1, R2, 2>::total : N));
    double* red = reinterpret_cast<double*>(mbar + NBUF);  // one double per warp
    if constexpr (MODE == 2)
        fill_col_tw<float, R0, R1, R2, 2>(TW, a.twpa);
    else
        for (int k = threadIdx.x; k < N; k += NT) TW[k] = a.twpb[k];
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&mbar[b], 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int grid = gridDim.x;
    // tile t: line (a index for the b pass, b index for the a pass) and first column
    auto issue_load = [&](int t, int b) {
        const int line = t / chunks, c0 = (t - line * chunks) * COLS;
        cpx<float>* dst = bufs + b * N * COLS;
        mbar_arrive_expect_tx(&mbar[b], TILE_BYTES);
        for (int h = 0; h < NBOX; ++h) {
            if (MODE == 2)
                tma_load_3d(dst + h * BOXR * COLS, &tmap, &mbar[b], 2 * c0, line, h * BOXR);
            else
                tma_load_3d(dst + h * BOXR * COLS, &tmap, &mbar[b], 2 * c0, h * BOXR, line);
        }
    };
    auto issue_store = [&](int t, int b) {
        const int line = t / chunks, c0 = (t - line * chunks) * COLS;
        const cpx<float>* src = bufs + b * N * COLS;
        for (int h = 0; h < NBOX; ++h) {
            if (MODE == 2)
                tma_store_3d(&tmap, src + h * BOXR * COLS, 2 * c0, line, h * BOXR);
            else
                tma_store_3d(&tmap, src + h * BOXR * COLS, 2 * c0, h * BOXR, line);
        }
        tma_commit();
    };
    if (threadIdx.x == 0)
        for (int b = 0; b < NBUF; ++b) {
            const int t = blockIdx.x + b * grid;
            if (t < ntiles) issue_load(t, b);
        }
    const int col = threadIdx.x % COLS, j0 = threadIdx.x / COLS;
    uint32_t parity = 0;
    float sum = 0.f, comp = 0.f;
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * grid;
        if (t >= ntiles) break;
        const int b = k % NBUF;
        const bool ok = mbar_wait(&mbar[b], (parity >> b) & 1u, err);
        if (!__syncthreads_and(ok)) break;
        parity ^= 1u << b;
        ColSmem<float, COLS> sm{bufs + b * N * COLS};
        if constexpr (MODE != 2) {
            ftransform<float, R0, R1, R2, JSTEP, MODE == 1, true>(sm, sm, sm, col, j0,
                                                                  static_cast<const TwPair<float>*>(TW));
        } else {
            const int line = t / chunks, c0 = (t - line * chunks) * COLS;
            const int nc = min(COLS, a.nh - c0);
            const cpx<float> gb = a.gsqb[line];
            const int k3 = c0 + col;
            const cpx<float> gc = a.gsqc[k3 < a.nh ? k3 : 0];
            // |G|^2 = |G_a|^2 + (|G_b|^2 + |G_c|^2): the b + c part once per tile, high and low parts apart
            const float gbc_h = gb.re + gc.re, gbc_l = gb.im + gc.im;
            const float mult = (k3 == 0 || k3 == a.M) ? 1.f : 2.f;
            float tile_sum = 0.f;  // this thread's terms of this tile (its column, BPT R rows)
            auto green = [&](int c, int k1, cpx<float>& v) {
                const float2 ga = __ldg(reinterpret_cast<const float2*>(a.gsqa + k1));
                const float G2 = (ga.x + gbc_h) + (ga.y + gbc_l);
                const float inv = (G2 > 0.f) ? __frcp_rn(G2) : 0.f;  // = 1 / G2, correctly rounded
                tile_sum = fmaf(v.re * v.re + v.im * v.im, inv, tile_sum);
                v = scale(v, inv * a.green_scale);
            };
            ftransform_green<float, R0, R1, R2, JSTEP, true, true>(sm, sm, sm, col, j0,
                                                                   static_cast<const TwPair<float>*>(TW), green);
            if (col < nc) {  // compensated across tiles
                const float term = mult * tile_sum - comp;
                const float tt = sum + term;
                comp = (tt - sum) - term;
                sum = tt;
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            issue_store(t, b);
            const int tn = blockIdx.x + (k + NBUF) * grid;
            if (tn < ntiles) {
                tma_wait_read<0>();  // the buffer is free once the store has read it
                issue_load(tn, b);
            }
        }
    }
    if (threadIdx.x == 0) tma_wait_all();
    if constexpr (MODE == 2) {
        const double bs = block_sum_comp(sum, -comp, red);
        if (threadIdx.x == 0) a.eh_partials[blockIdx.x] = bs;
    }
}

// ------------------------------------------------------------------ c passes
template <typename T, int LINES, int NT, int R0, int R1, int R2>
__global__ void __launch_bounds__(NT, min_ctas<NT>()) k_r2c_fast(const T* __restrict__ rho, FastArgs<T> a) {
    constexpr int M = R0 * R1 * R2;
    constexpr int TPL = NT / LINES;
    constexpr int LDP = M + M / 16 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);
    TwPair<T>* TW = reinterpret_cast<TwPair<T>*>(S + LINES * LDP);
    fill_line_tw_fwd<T, R0, R1, R2>(TW, a.twpc);
    const TwPair<T>* TWP = TW + LineTwLayout<R0, R1, R2>::s2 + LineTwLayout<R0, R1, R2>::s3;  // w_2M^k, k <= M/2
    const int l = threadIdx.x / TPL, j0 = threadIdx.x % TPL;
    const long long gline = (long long)blockIdx.x * LINES + l;
    const bool act = gline < (long long)a.n1 * a.n2;
    LineRealIn<T> src{reinterpret_cast<const cpx<T>*>(rho + (act ? gline : 0) * a.n3), act};
    LineSmem<T> sm{S + l * LDP};
    __syncthreads();
    // M-point transform of z (twiddles exp(-2 pi i e / M) = entry 2e of the 2M-point table)
    line_ftransform<T, R0, R1, R2, TPL, false, false>(src, sm, sm, j0, TW);
    __syncthreads();
    // X[k] = E[k] + w^k O[k], E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / 2i, k = 0..M;
    // the pair k, M - k shares its loads: E[M-k] = conj E[k], O[M-k] = conj O[k], w^(M-k) = -conj w^k,
    // so X[M-k] = conj(E[k] - w^k O[k])
    if (act) {
        cpx<T>* out = a.W + gline * a.ldc;
        const T half = T(0.5);
        for (int k = j0; k <= M / 2; k += TPL) {
            const cpx<T> z1 = sm.ld_(0, k);
            const cpx<T> z2 = conjg(sm.ld_(0, k == 0 ? 0 : M - k));
            const cpx<T> E = scale(z1 + z2, half);
            const cpx<T> d = z1 - z2;
            const cpx<T> O = mk(d.im * half, -d.re * half);
            const cpx<T> t = twmul(O, TWP[k], false);
            out[k] = E + t;
            out[M - k] = conjg(E - t);
        }
    }
}

template <typename T, int LINES, int NT, int R0, int R1, int R2>
__global__ void __launch_bounds__(NT, min_ctas<NT>()) k_c2r_fast(T* __restrict__ vout, FastArgs<T> a) {
    constexpr int M = R0 * R1 * R2;
    constexpr int TPL = NT / LINES;
    constexpr int LDP = M + M / 16 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* TW = S + LINES * LDP;
    fill_line_tw_inv<T, R0, R1, R2>(TW, a.twpc);
    const TwHi<T> TWQ{TW + LineTwLayout<R0, R1, R2>::s2 + LineTwLayout<R0, R1, R2>::s3};  // k < M
    const int l = threadIdx.x / TPL, j0 = threadIdx.x % TPL;
    const long long gline = (long long)blockIdx.x * LINES + l;
    const bool act = gline < (long long)a.n1 * a.n2;
    const long long gl = act ? gline : 0;
    LineSmem<T> sm{S + l * LDP};
    __syncthreads();
    LineC2RIn<T, TwHi<T>> src{a.W + gl * a.ldc, TWQ, M, act};
    LineRealOut<T> dst{reinterpret_cast<cpx<T>*>(vout + gl * a.n3), act};
    line_ftransform<T, R0, R1, R2, TPL, true, false>(src, sm, dst, j0, static_cast<const cpx<T>*>(TW));
}

// ------------------------------------------------------------------ bulk-streamed c passes (FP32)
// Persistent CTAs (two per SM) walk tiles of LINES consecutive lines.  A tile's
// input is one contiguous block (LINES lines of rho, or LINES rows of the half
// spectrum with their padding), brought into a ring slot by one bulk copy that
// completes on the slot's mbarrier; thread 0 keeps NBUF tiles in flight.  The
// first stage reads the slot, and once every thread has read it (the stage's
// barrier) thread 0 refills the slot with the tile NBUF ahead, so the next
// loads overlap this tile's butterflies.  The other stages run in a padded
// work buffer, and results leave from registers with coalesced stores.  Same
// arithmetic, in the same order, as k_r2c_fast / k_c2r_fast.
//
// Every wait is bounded; after a failed wait thread 0 waits (bounded again)
// for the copies this CTA still has in flight before the CTA returns.
template <int NBUF>
__device__ __forceinline__ void drain_ring(uint64_t* mbar, int k, int ntiles, int* err) {
    if (threadIdx.x != 0) return;
    for (int i = 0; i < NBUF; ++i) {
        const int t = blockIdx.x + (k + i) * gridDim.x;
        if (t < ntiles) mbar_wait(&mbar[(k + i) % NBUF], (uint32_t)((k + i) / NBUF) & 1u, err);
    }
}

template <int LINES, int NT, int R0, int R1, int R2, int NBUF, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_r2c_stream(const float* __restrict__ rho, FastArgs<float> a, int ntiles, int* err) {
    constexpr int M = R0 * R1 * R2;
    constexpr int TPL = NT / LINES;
    constexpr int LDP = M + M / 16 + 1;
    constexpr int SLOT = LINES * M;  // complex elements per ring slot
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<float>* ring = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<float>* S = ring + NBUF * SLOT;
    TwPair<float>* TW = reinterpret_cast<TwPair<float>*>(S + LINES * LDP);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(TW + LineTwLayout<R0, R1, R2>::fwd);
    fill_line_tw_fwd<float, R0, R1, R2>(TW, a.twpc);
    const TwPair<float>* TWP = TW + LineTwLayout<R0, R1, R2>::s2 + LineTwLayout<R0, R1, R2>::s3;
    const long long nlines = (long long)a.n1 * a.n2;
    auto issue = [&](int t, int b) {
        const long long l0 = (long long)t * LINES;
        const int nl = (int)min((long long)LINES, nlines - l0);
        const uint32_t bytes = (uint32_t)nl * M * 8u;
        mbar_arrive_expect_tx(&mbar[b], bytes);
        bulk_load(ring + b * SLOT, rho + l0 * 2 * M, bytes, &mbar[b]);
    };
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&mbar[b], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < NBUF; ++b) {
            const int t = blockIdx.x + b * gridDim.x;
            if (t < ntiles) issue(t, b);
        }
    const int l = threadIdx.x / TPL, j0 = threadIdx.x % TPL;
    LineSmem<float> sm{S + l * LDP};
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        const int b = k % NBUF;
        const bool ok = mbar_wait(&mbar[b], (uint32_t)(k / NBUF) & 1u, err);
        if (!__syncthreads_and(ok)) {
            drain_ring<NBUF>(mbar, k, ntiles, err);
            break;
        }
        const long long gline = (long long)t * LINES + l;
        const bool act = gline < nlines;
        LineRealIn<float> src{ring + b * SLOT + l * M, act};
        auto refill = [&] {
            const int tn = t + NBUF * gridDim.x;
            if (threadIdx.x == 0 && tn < ntiles) issue(tn, b);
        };
        // M-point transform of z (twiddles exp(-2 pi i e / M) = entry 2e of the 2M-point table)
        line_ftransform<float, R0, R1, R2, TPL, false, true>(src, sm, sm, j0, static_cast<const TwPair<float>*>(TW),
                                                               refill);
        __syncthreads();
        // X[k] and X[M - k] from one pair of loads, as in k_r2c_fast
        if (act) {
            cpx<float>* out = a.W + gline * a.ldc;
            for (int kk = j0; kk <= M / 2; kk += TPL) {
                const cpx<float> z1 = sm.ld_(0, kk);
                const cpx<float> z2 = conjg(sm.ld_(0, kk == 0 ? 0 : M - kk));
                const cpx<float> E = scale(z1 + z2, 0.5f);
                const cpx<float> d = z1 - z2;
                const cpx<float> O = mk(d.im * 0.5f, -d.re * 0.5f);
                const cpx<float> t = twmul(O, TWP[kk], false);
                out[kk] = E + t;
                out[M - kk] = conjg(E - t);
            }
        }
    }
}

template <int LINES, int NT, int R0, int R1, int R2, int NBUF, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_c2r_stream(float* __restrict__ vout, FastArgs<float> a, int ntiles, int* err) {
    constexpr int M = R0 * R1 * R2;
    constexpr int TPL = NT / LINES;
    constexpr int LDP = M + M / 16 + 1;
    const int slot = LINES * a.ldc;  // complex elements per ring slot: LINES padded rows
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<float>* ring = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<float>* S = ring + NBUF * slot;
    cpx<float>* TWh = S + LINES * LDP;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(TWh + LineTwLayout<R0, R1, R2>::inv);
    fill_line_tw_inv<float, R0, R1, R2>(TWh, a.twpc);
    const TwHi<float> TWQ{TWh + LineTwLayout<R0, R1, R2>::s2 + LineTwLayout<R0, R1, R2>::s3};
    const long long nlines = (long long)a.n1 * a.n2;
    auto issue = [&](int t, int b) {
        const long long l0 = (long long)t * LINES;
        const int nl = (int)min((long long)LINES, nlines - l0);
        const uint32_t bytes = (uint32_t)nl * (uint32_t)a.ldc * 8u;
        mbar_arrive_expect_tx(&mbar[b], bytes);
        bulk_load(ring + b * slot, a.W + l0 * a.ldc, bytes, &mbar[b]);
    };
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&mbar[b], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < NBUF; ++b) {
            const int t = blockIdx.x + b * gridDim.x;
            if (t < ntiles) issue(t, b);
        }
    const int l = threadIdx.x / TPL, j0 = threadIdx.x % TPL;
    LineSmem<float> sm{S + l * LDP};
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        const int b = k % NBUF;
        const bool ok = mbar_wait(&mbar[b], (uint32_t)(k / NBUF) & 1u, err);
        if (!__syncthreads_and(ok)) {
            drain_ring<NBUF>(mbar, k, ntiles, err);
            break;
        }
        const long long gline = (long long)t * LINES + l;
        const bool act = gline < nlines;
        LineC2RIn<float, TwHi<float>> src{ring + b * slot + l * a.ldc, TWQ, M, act};
        LineRealOut<float> dst{reinterpret_cast<cpx<float>*>(vout + (act ? gline : 0) * a.n3), act};
        auto refill = [&] {
            const int tn = t + NBUF * gridDim.x;
            if (threadIdx.x == 0 && tn < ntiles) issue(tn, b);
        };
        line_ftransform<float, R0, R1, R2, TPL, true, true>(src, sm, dst, j0, static_cast<const cpx<float>*>(TWh),
                                                             refill);
    }
}



// ------------------------------------------------------------------ paired-lane streamed c passes (FP32)
// The bulk-streamed c passes with every thread transforming one butterfly of two lines at once, as
// the two lanes of the paired type f2x (radices of any kind): TPL threads per pair of lines, half
// the threads of k_r2c_stream / k_c2r_stream for the same tile.  Same ring, tiles and arithmetic
// (forward twiddles and constants compensated, inverse rounded), so the same results.
__device__ __forceinline__ f2x dup2(float x) { return f2x(make_float2(x, x)); }
__device__ __forceinline__ TwPair<f2x> pair_of(const TwPair<float>& w) {
    return TwPair<f2x>{mk(dup2(w.h.re), dup2(w.h.im)), mk(dup2(w.l.re), dup2(w.l.im))};
}
__device__ __forceinline__ cpx<f2x> pair_of(cpx<float> w) { return mk(dup2(w.re), dup2(w.im)); }
__device__ __forceinline__ cpx<f2x> lanes(cpx<float> x, cpx<float> y) {
    return mk(f2x(make_float2(x.re, y.re)), f2x(make_float2(x.im, y.im)));
}
__device__ __forceinline__ cpx<float> lane0(cpx<f2x> v) { return mk(v.re.v.x, v.im.v.x); }
__device__ __forceinline__ cpx<float> lane1(cpx<f2x> v) { return mk(v.re.v.y, v.im.v.y); }

// Stage and post-processing twiddles of LineTwLayout on both lanes.
template <int R0, int R1, int R2>
__device__ __forceinline__ void fill_line_tw_fwd_pair(TwPair<f2x>* tw, const TwPair<float>* g) {
    using L = LineTwLayout<R0, R1, R2>;
    auto get = [&](int e) { return pair_of(g[e]); };
    fill_stage_tw<L::M, R1, R0, 2>(tw, get);
    if constexpr (R2 > 1) fill_stage_tw<L::M, R2, R0 * R1, 2>(tw + L::s2, get);
    for (int k = threadIdx.x; k <= L::M / 2; k += blockDim.x) tw[L::s2 + L::s3 + k] = pair_of(g[k]);
}
template <int R0, int R1, int R2>
__device__ __forceinline__ void fill_line_tw_inv_pair(cpx<f2x>* tw, const TwPair<float>* g) {
    using L = LineTwLayout<R0, R1, R2>;
    auto get = [&](int e) { return pair_of(g[e].h); };
    fill_stage_tw<L::M, R1, R0, 2>(tw, get);
    if constexpr (R2 > 1) fill_stage_tw<L::M, R2, R0 * R1, 2>(tw + L::s2, get);
    for (int k = threadIdx.x; k < L::M; k += blockDim.x) tw[L::s2 + L::s3 + k] = pair_of(g[k].h);
}

struct LinePairSmem {  // a pair of lines, padded: point n of both at p[pidx(n)]
    cpx<f2x>* p;
    __device__ __forceinline__ cpx<f2x> ld_(int, int n) const { return p[pidx(n)]; }
    __device__ __forceinline__ void st_(int, int n, cpx<f2x> v) const { p[pidx(n)] = v; }
};

struct LinePairRealIn {  // z[n] = rho[2n] + i rho[2n+1] of lines z and z + stride (a ring slot)
    const cpx<float>* z;
    int stride;
    __device__ __forceinline__ cpx<f2x> ld_(int, int n) const { return lanes(z[n], z[stride + n]); }
};

// Z[k] = (X[k] + conj X[M-k]) + i w^-k (X[k] - conj X[M-k]) of rows x and x + stride (c2r pre-step)
struct LinePairC2RIn {
    const cpx<float>* x;
    int stride;
    const cpx<f2x>* tw;  // exp(-2 pi i k / N3), rounded
    int M;
    __device__ __forceinline__ cpx<f2x> ld_(int, int k) const {
        const cpx<f2x> x1 = lanes(x[k], x[stride + k]);
        const cpx<f2x> x2 = conjg(lanes(x[M - k], x[stride + M - k]));
        const cpx<f2x> Ep = x1 + x2;
        const cpx<f2x> Op = twmul<false>(x1 - x2, TwPair<f2x>{tw[k], mk(f2x(0), f2x(0))}, true);
        return mk(Ep.re - Op.im, Ep.im + Op.re);
    }
};

struct LinePairRealOut {  // lines z and z + stride of the real output, each only if it exists
    cpx<float>* z;
    int stride;
    bool act_a, act_b;
    __device__ __forceinline__ void st_(int, int n, cpx<f2x> v) const {
        if (act_a) z[n] = lane0(v);
        if (act_b) z[stride + n] = lane1(v);
    }
};

template <int LINES, int NT, int R0, int R1, int R2, int NBUF, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_r2c_pair(const float* __restrict__ rho, FastArgs<float> a, int ntiles, int* err) {
    constexpr int M = R0 * R1 * R2;
    constexpr int TPL = NT / (LINES / 2);
    constexpr int LDP = M + M / 16 + 1;
    constexpr int SLOT = LINES * M;  // complex elements per ring slot
    static_assert(LINES % 2 == 0 && NT % (LINES / 2) == 0, "pairs of lines");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<float>* ring = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<f2x>* S = reinterpret_cast<cpx<f2x>*>(ring + NBUF * SLOT);
    TwPair<f2x>* TW = reinterpret_cast<TwPair<f2x>*>(S + (LINES / 2) * LDP);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(TW + LineTwLayout<R0, R1, R2>::fwd);
    fill_line_tw_fwd_pair<R0, R1, R2>(TW, a.twpc);
    const TwPair<f2x>* TWP = TW + LineTwLayout<R0, R1, R2>::s2 + LineTwLayout<R0, R1, R2>::s3;
    const long long nlines = (long long)a.n1 * a.n2;
    auto issue = [&](int t, int b) {
        const long long l0 = (long long)t * LINES;
        const int nl = (int)min((long long)LINES, nlines - l0);
        const uint32_t bytes = (uint32_t)nl * M * 8u;
        mbar_arrive_expect_tx(&mbar[b], bytes);
        bulk_load(ring + b * SLOT, rho + l0 * 2 * M, bytes, &mbar[b]);
    };
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&mbar[b], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < NBUF; ++b) {
            const int t = blockIdx.x + b * gridDim.x;
            if (t < ntiles) issue(t, b);
        }
    const int q = threadIdx.x / TPL, j0 = threadIdx.x % TPL;  // pair of lines 2q, 2q + 1
    LinePairSmem sm{S + q * LDP};
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        const int b = k % NBUF;
        const bool ok = mbar_wait(&mbar[b], (uint32_t)(k / NBUF) & 1u, err);
        if (!__syncthreads_and(ok)) {
            drain_ring<NBUF>(mbar, k, ntiles, err);
            break;
        }
        const long long gline = (long long)t * LINES + 2 * q;
        LinePairRealIn src{ring + b * SLOT + 2 * q * M, M};  // lines past the tile hold stale data
        auto refill = [&] {
            const int tn = t + NBUF * gridDim.x;
            if (threadIdx.x == 0 && tn < ntiles) issue(tn, b);
        };
        line_ftransform<f2x, R0, R1, R2, TPL, false, true>(src, sm, sm, j0, static_cast<const TwPair<f2x>*>(TW),
                                                             refill);
        __syncthreads();
        // X[k] and X[M - k] of both lines from one pair of loads, as in k_r2c_fast
        if (gline < nlines) {
            const bool act_b = gline + 1 < nlines;
            cpx<float>* out = a.W + gline * a.ldc;
            const f2x half = dup2(0.5f);
            for (int kk = j0; kk <= M / 2; kk += TPL) {
                const cpx<f2x> z1 = sm.ld_(0, kk);
                const cpx<f2x> z2 = conjg(sm.ld_(0, kk == 0 ? 0 : M - kk));
                const cpx<f2x> E = scale(z1 + z2, half);
                const cpx<f2x> d = z1 - z2;
                const cpx<f2x> O = mk(d.im * half, -(d.re * half));
                const cpx<f2x> tq = twmul(O, TWP[kk], false);
                const cpx<f2x> X1 = E + tq, X2 = conjg(E - tq);
                out[kk] = lane0(X1);
                out[M - kk] = lane0(X2);
                if (act_b) {
                    out[a.ldc + kk] = lane1(X1);
                    out[a.ldc + M - kk] = lane1(X2);
                }
            }
        }
    }
}

template <int LINES, int NT, int R0, int R1, int R2, int NBUF, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_c2r_pair(float* __restrict__ vout, FastArgs<float> a, int ntiles, int* err) {
    constexpr int M = R0 * R1 * R2;
    constexpr int TPL = NT / (LINES / 2);
    constexpr int LDP = M + M / 16 + 1;
    static_assert(LINES % 2 == 0 && NT % (LINES / 2) == 0, "pairs of lines");
    const int slot = LINES * a.ldc;  // complex elements per ring slot: LINES padded rows
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<float>* ring = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<f2x>* S = reinterpret_cast<cpx<f2x>*>(ring + NBUF * slot);
    cpx<f2x>* TWh = S + (LINES / 2) * LDP;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(TWh + LineTwLayout<R0, R1, R2>::inv);
    fill_line_tw_inv_pair<R0, R1, R2>(TWh, a.twpc);
    const cpx<f2x>* TWQ = TWh + LineTwLayout<R0, R1, R2>::s2 + LineTwLayout<R0, R1, R2>::s3;
    const long long nlines = (long long)a.n1 * a.n2;
    auto issue = [&](int t, int b) {
        const long long l0 = (long long)t * LINES;
        const int nl = (int)min((long long)LINES, nlines - l0);
        const uint32_t bytes = (uint32_t)nl * (uint32_t)a.ldc * 8u;
        mbar_arrive_expect_tx(&mbar[b], bytes);
        bulk_load(ring + b * slot, a.W + l0 * a.ldc, bytes, &mbar[b]);
    };
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&mbar[b], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < NBUF; ++b) {
            const int t = blockIdx.x + b * gridDim.x;
            if (t < ntiles) issue(t, b);
        }
    const int q = threadIdx.x / TPL, j0 = threadIdx.x % TPL;
    LinePairSmem sm{S + q * LDP};
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        const int b = k % NBUF;
        const bool ok = mbar_wait(&mbar[b], (uint32_t)(k / NBUF) & 1u, err);
        if (!__syncthreads_and(ok)) {
            drain_ring<NBUF>(mbar, k, ntiles, err);
            break;
        }
        const long long gline = (long long)t * LINES + 2 * q;
        const bool act = gline < nlines;
        LinePairC2RIn src{ring + b * slot + 2 * q * a.ldc, a.ldc, TWQ, M};
        LinePairRealOut dst{reinterpret_cast<cpx<float>*>(vout + (act ? gline : 0) * a.n3), M, act,
                            gline + 1 < nlines};
        auto refill = [&] {
            const int tn = t + NBUF * gridDim.x;
            if (threadIdx.x == 0 && tn < ntiles) issue(tn, b);
        };
        line_ftransform<f2x, R0, R1, R2, TPL, true, true>(src, sm, dst, j0, static_cast<const cpx<f2x>*>(TWh),
                                                            refill);
    }
}

// ------------------------------------------------------------------ splat fused into the r2c pass (FP32)
// The density never reaches HBM: persistent CTAs walk units of up to SEG tiles, a tile being LINES
// consecutive c lines at one a index (b = b0 .. b0 + nl - 1), and compute each tile's density in
// shared memory before the r2c transform of those lines.
//   * Per unit (one a index, SEG tiles along b) the CTA selects, in increasing atom index (the order
//     of the binned splat), the atoms whose cutoff box covers the a index and meets the unit's b
//     range: first the leaf boxes (structure C of Sec. 3.2.2) that do, then each of their atoms.
//     A selected atom becomes a record in shared memory: its index, wrapped b and c box, a factor
//     and q (pi s^2)^-3/2 split in two FP32 parts.
//   * Per tile the records whose b box meets the tile are taken (in order) in batches of kb; a batch
//     stages each atom's a x b factor per line and its image-summed c factors times q, and thread
//     (g, u) adds, for its points 2u and 2u + 1 of the LG lines of group g, one paired FMA per atom
//     and line.  A unit with more atoms than the records hold selects per tile instead, in rounds.
//   * The sums go into the transform's padded work buffer; the lines take the same transform and
//     post-processing as k_r2c_stream.
constexpr int kFuseLines = 16;
constexpr int kFuseSeg = 8;  // tiles per unit

__host__ __device__ constexpr int next_pow2(int n) { return n <= 1 ? 1 : 2 * next_pow2((n + 1) / 2); }

template <int LINES, int NT, int R0, int R1, int R2, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_r2c_splat(AtomArgs<float> at, FastArgs<float> a, int tiles_b, int nunits, int kb, int fsh, int cap, int img) {
    constexpr int M = R0 * R1 * R2;
    constexpr int TPL = NT / LINES;
    constexpr int LDP = M + M / 16 + 1;
    constexpr int PT = next_pow2(M);  // threads per line group of the splat
    constexpr int GL = NT / PT;       // line groups
    constexpr int LG = LINES / GL;    // lines per thread
    static_assert(PT >= 32 && PT <= NT && LINES % GL == 0, "splat thread layout");
    const int fcw = 1 << fsh;  // c factors staged per atom
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<float>* S = reinterpret_cast<cpx<float>*>(smem_raw);
    TwPair<float>* TW = reinterpret_cast<TwPair<float>*>(S + LINES * LDP);
    float2* WL = reinterpret_cast<float2*>(TW + LineTwLayout<R0, R1, R2>::fwd);  // [kb][LINES]: (w, w)
    int4* RI = reinterpret_cast<int4*>(WL + kb * LINES);  // [cap]: atom, b box, c box, a factor
    float2* RQ = reinterpret_cast<float2*>(RI + cap);     // [cap]: q (pi s^2)^-3/2 as two FP32 parts
    float* FC = reinterpret_cast<float*>(RQ + cap);       // [kb][fcw]
    int2* AC = reinterpret_cast<int2*>(FC + kb * fcw);    // [kb]: wrapped c start, points
    int* lst = reinterpret_cast<int*>(AC + kb);           // [NT]: selected leaves
    int* cand = lst + NT;                                 // [NT]: selected records of a tile
    __shared__ int wcnt[NT / 32];
    __shared__ int nsel;
    fill_line_tw_fwd<float, R0, R1, R2>(TW, a.twpc);
    const TwPair<float>* TWP = TW + LineTwLayout<R0, R1, R2>::s2 + LineTwLayout<R0, R1, R2>::s3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // ordered compaction of the threads whose flag is set into out[base + ..]; returns the count
    auto compact = [&](bool flag, int value, int* out, int base, int limit) -> int {
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        __syncthreads();  // earlier readers of wcnt / nsel / out are done
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < NT / 32; ++w) {
                const int c = wcnt[w];
                wcnt[w] = s;
                s += c;
            }
            nsel = s;
        }
        __syncthreads();
        const int pos = base + wcnt[warp] + __popc(bal & ((1u << lane) - 1u));
        if (flag && pos < limit) out[pos] = value;
        __syncthreads();
        return nsel;
    };
    const int g = threadIdx.x / PT, u = threadIdx.x - g * PT;
    const int c0 = 2 * u;           // this thread's points c0, c0 + 1 (u < M)
    const int wc0 = 2 * (u & ~31);  // the first point of this warp's range of 64
    const int l = threadIdx.x / TPL, j0 = threadIdx.x % TPL;
    LineSmem<float> sm{S + l * LDP};
    const long long fstride = at.fb;
    const int upr = (tiles_b + kFuseSeg - 1) / kFuseSeg;  // units per a index
    // does [s, s + len) mod n meet [t0, t0 + tn) (s, t0 in [0, n), len <= n)?  range_hits without a division
    auto meets = [](int s, int len, int t0, int tn, int n) {
        int d = t0 - s;
        if (d < 0) d += n;
        return d < len || d + tn > n;
    };
    // a record for atom i (the caller has checked its boxes)
    auto make_record = [&](int i, int ia, int r) {
        const AtomPrep<float>& p = at.prep[i];
        const float fa = image_sum(at.fac + i * 3 * fstride, ia, p.st[0], p.cnt[0], a.n1);
        RI[r] = make_int4(i, p.st[1] | (p.cnt[1] << 16), p.st[2] | (p.cnt[2] << 16), __float_as_int(fa));
        RQ[r] = make_float2(p.qn, p.ql);
    };
    // the factor of box point g - st (wrapped) of a box starting at st with cnt points: one load when
    // the boxes along this axis fit in the grid (wide: several images, summed)
    auto factor = [](const float* f, int g, int st, int cnt, int n, bool wide) {
        int m = g - st;
        if (m < 0) m += n;
        float v = m < cnt ? __ldg(f + m) : 0.f;
        if (wide)
            for (m += n; m < cnt; m += n) v += __ldg(f + m);
        return v;
    };
    const bool wide_b = img & 2, wide_c = img & 4;
    // stage records cand[bb .. bb + nb) and add them to this thread's points
    auto add_batch = [&](int bb, int nb, int b0, int nl, float2* acc) {
#pragma unroll 4
        for (int e = threadIdx.x; e < nb * LINES; e += NT) {
            const int tt = e / LINES, ll = e - tt * LINES;
            const int4 R = RI[cand[bb + tt]];
            int bg = b0 + ll;
            if (bg >= a.n2) bg -= a.n2;
            const float fb = factor(at.fac + (R.x * 3 + 1) * fstride, bg, R.y & 0xffff, R.y >> 16, a.n2, wide_b);
            const float w = ll < nl ? __int_as_float(R.w) * fb : 0.f;
            WL[e] = make_float2(w, w);
        }
#pragma unroll 4
        for (int e = threadIdx.x; e < (nb << fsh); e += NT) {
            const int tt = e >> fsh, m = e & (fcw - 1);
            const int r = cand[bb + tt];
            const int4 R = RI[r];
            const int st = R.z & 0xffff, cnt = R.z >> 16, nw = min(cnt, a.n3);
            int cc = st + m;
            if (cc >= a.n3) cc -= a.n3;
            const float sc = m < nw ? factor(at.fac + (R.x * 3 + 2) * fstride, cc, st, cnt, a.n3, wide_c) : 0.f;
            const float2 qq = RQ[r];
            FC[e] = qq.x * sc + qq.y * sc;
            if (m == 0) AC[tt] = make_int2(st, nw);
        }
        __syncthreads();
        if (u < M) {
            for (int tt = 0; tt < nb; ++tt) {
                const int2 ac = AC[tt];
                if (!meets(ac.x, ac.y, wc0, 64, a.n3)) continue;  // the same for the whole warp
                int d0 = c0 - ac.x;
                if (d0 < 0) d0 += a.n3;
                const int d1 = d0 + 1 == a.n3 ? 0 : d0 + 1;
                const float* fc = FC + tt * fcw;
                const float2 fp = make_float2(d0 < ac.y ? fc[d0] : 0.f, d1 < ac.y ? fc[d1] : 0.f);
                const float2* wl = WL + tt * LINES + g * LG;
#pragma unroll
                for (int i = 0; i < LG; ++i) acc[i] = __ffma2_rn(wl[i], fp, acc[i]);
            }
        }
        __syncthreads();
    };
    // the atoms whose box covers index ia and meets [b0, b0 + nb_) along b, in increasing index, by
    // rounds of at most NT: each round's atoms become records 0 .. cnt - 1 and go to `round`
    auto select_rounds = [&](int ia, int b0, int nb_, auto&& round) {
        for (int lb = 0; lb < at.nleaves; lb += NT) {
            const int lf = lb + (int)threadIdx.x;
            bool hit = false;
            if (lf < at.nleaves) {
                const int* bx = at.leaf + 6 * lf;
                hit = range_hits(bx[0], bx[3], ia, 1, a.n1) && range_hits(bx[1], bx[4], b0, nb_, a.n2);
            }
            const int nlf = compact(hit, lf, lst, 0, NT);
            const int ncand = nlf * at.apl;
            for (int cb = 0; cb < ncand; cb += NT) {
                const int c = cb + (int)threadIdx.x;
                int atom = -1;
                if (c < ncand) {
                    const int i = lst[c / at.apl] * at.apl + c % at.apl;
                    if (i < at.n) {
                        const AtomPrep<float>& p = at.prep[i];
                        if (range_hits(p.lo[0], p.cnt[0], ia, 1, a.n1) && range_hits(p.lo[1], p.cnt[1], b0, nb_, a.n2))
                            atom = i;
                    }
                }
                round(atom);
            }
        }
    };
    for (int k = 0;; ++k) {
        const int un = blockIdx.x + k * gridDim.x;
        if (un >= nunits) break;
        const int ia = un / upr, tb0 = (un - ia * upr) * kFuseSeg, tb1 = min(tiles_b, tb0 + kFuseSeg);
        const int bu0 = tb0 * LINES, bun = min(tb1 * LINES, a.n2) - bu0;
        // the unit's records (or overflow: more atoms than cap)
        int nrec = 0;
        select_rounds(ia, bu0, bun, [&](int atom) {
            const int cnt = compact(atom >= 0, atom, cand, 0, NT);
            for (int e = threadIdx.x; e < cnt; e += NT)
                if (nrec + e < cap) make_record(cand[e], ia, nrec + e);
            nrec += cnt;
        });
        __syncthreads();  // the records are written
        const bool overflow = nrec > cap;
        for (int tb = tb0; tb < tb1; ++tb) {
            const int b0 = tb * LINES, nl = min(LINES, a.n2 - b0);
            float2 acc[LG];
#pragma unroll
            for (int i = 0; i < LG; ++i) acc[i] = make_float2(0.f, 0.f);
            if (!overflow) {
                for (int rb = 0; rb < nrec; rb += NT) {
                    const int r = rb + (int)threadIdx.x;
                    bool hit = false;
                    if (r < nrec) {
                        const int rb_ = RI[r].y;
                        hit = meets(rb_ & 0xffff, min(rb_ >> 16, a.n2), b0, nl, a.n2);
                    }
                    const int nc = compact(hit, r, cand, 0, NT);
                    for (int bb = 0; bb < nc; bb += kb) add_batch(bb, min(kb, nc - bb), b0, nl, acc);
                }
            } else {
                select_rounds(ia, b0, nl, [&](int atom) {
                    const int cnt = compact(atom >= 0, atom, cand, 0, NT);
                    for (int e = threadIdx.x; e < cnt; e += NT) {
                        make_record(cand[e], ia, e);
                        cand[e] = e;
                    }
                    __syncthreads();
                    for (int bb = 0; bb < cnt; bb += kb) add_batch(bb, min(kb, cnt - bb), b0, nl, acc);
                });
            }
            // the tile's density as z[m] = rho[2m] + i rho[2m + 1], line by line in the work buffer
            if (u < M) {
#pragma unroll
                for (int i = 0; i < LG; ++i) S[(g * LG + i) * LDP + pidx(u)] = mk(acc[i].x, acc[i].y);
            }
            __syncthreads();
            const long long gline = (long long)ia * a.n2 + b0 + l;
            const bool act = l < nl;
            // M-point transform in place (twiddles exp(-2 pi i e / M) = entry 2e of the 2M-point table)
            line_ftransform<float, R0, R1, R2, TPL, false, true>(sm, sm, sm, j0, static_cast<const TwPair<float>*>(TW));
            __syncthreads();
            // X[k] and X[M - k] from one pair of loads, as in k_r2c_fast
            if (act) {
                cpx<float>* out = a.W + gline * a.ldc;
                for (int kk = j0; kk <= M / 2; kk += TPL) {
                    const cpx<float> z1 = sm.ld_(0, kk);
                    const cpx<float> z2 = conjg(sm.ld_(0, kk == 0 ? 0 : M - kk));
                    const cpx<float> E = scale(z1 + z2, 0.5f);
                    const cpx<float> d = z1 - z2;
                    const cpx<float> O = mk(d.im * 0.5f, -d.re * 0.5f);
                    const cpx<float> tq = twmul(O, TWP[kk], false);
                    out[kk] = E + tq;
                    out[M - kk] = conjg(E - tq);
                }
            }
            __syncthreads();  // the work buffer is read before the next tile writes it
        }
        __syncthreads();  // the records are read before the next unit writes them
    }
}

template <int NT, int R0, int R1, int R2, int MINB>
struct SplatLineCfg {
    static constexpr int m = R0 * R1 * R2, lines = kFuseLines;
    static size_t smem(int kb, int fcw, int cap) {
        return (size_t)lines * (m + m / 16 + 1) * sizeof(cpx<float>) +
               (size_t)LineTwLayout<R0, R1, R2>::fwd * sizeof(TwPair<float>) + (size_t)kb * lines * sizeof(float2) +
               (size_t)cap * (sizeof(int4) + sizeof(float2)) + (size_t)kb * fcw * sizeof(float) +
               (size_t)kb * sizeof(int2) + 2 * NT * sizeof(int);
    }
    static auto kernel() { return k_r2c_splat<kFuseLines, NT, R0, R1, R2, MINB>; }
};

template <class F>
bool with_splat_line_cfg(int M, F&& f) {
    switch (M) {
        case 256: f(SplatLineCfg<256, 16, 16, 1, 2>{}); return true;
        case 128: f(SplatLineCfg<256, 16, 8, 1, 2>{}); return true;
        case 210: f(SplatLineCfg<256, 6, 5, 7, 2>{}); return true;
        case 200: f(SplatLineCfg<256, 8, 5, 5, 2>{}); return true;
        case 105: f(SplatLineCfg<256, 3, 5, 7, 2>{}); return true;
        case 64: f(SplatLineCfg<256, 8, 8, 1, 2>{}); return true;
        case 60: f(SplatLineCfg<256, 4, 3, 5, 2>{}); return true;
        default: return false;
    }
}

// ------------------------------------------------------------------ dispatch
template <typename T, int COLS, int NT, int R0, int R1, int R2>
struct ColCfg {
    static constexpr int cols = COLS, n = R0 * R1 * R2;
    static size_t smem(int = 0) { return (size_t)n * COLS * sizeof(cpx<T>) + (size_t)n * sizeof(TwPair<T>); }
    static cudaError_t configure(int optin) {
        cudaError_t e;
        if ((e = allow_max_dynamic_smem(k_col_fast<T, COLS, NT, R0, R1, R2, 0>, optin))) return e;
        if ((e = allow_max_dynamic_smem(k_col_fast<T, COLS, NT, R0, R1, R2, 1>, optin))) return e;
        return allow_max_dynamic_smem(k_col_fast<T, COLS, NT, R0, R1, R2, 2>, optin);
    }
    static void launch(int mode, unsigned grid, const FastArgs<T>& a, cudaStream_t s) {
        if (mode == 0) k_col_fast<T, COLS, NT, R0, R1, R2, 0><<<grid, NT, smem(0), s>>>(a);
        if (mode == 1) k_col_fast<T, COLS, NT, R0, R1, R2, 1><<<grid, NT, smem(1), s>>>(a);
        if (mode == 2) k_col_fast<T, COLS, NT, R0, R1, R2, 2><<<grid, NT, smem(2), s>>>(a);
    }
};

template <typename T, int LINES, int NT, int R0, int R1, int R2>
struct LineCfg {
    static constexpr int lines = LINES, m = R0 * R1 * R2;
    static size_t smem() {
        const size_t tw = std::max((size_t)LineTwLayout<R0, R1, R2>::fwd * sizeof(TwPair<T>),
                                   (size_t)LineTwLayout<R0, R1, R2>::inv * sizeof(cpx<T>));
        return (size_t)LINES * (m + m / 16 + 1) * sizeof(cpx<T>) + tw;
    }
    static cudaError_t configure(int optin) {
        cudaError_t e;
        if ((e = allow_max_dynamic_smem(k_r2c_fast<T, LINES, NT, R0, R1, R2>, optin))) return e;
        return allow_max_dynamic_smem(k_c2r_fast<T, LINES, NT, R0, R1, R2>, optin);
    }
    static void launch(bool inverse, unsigned grid, const void* in, void* out, const FastArgs<T>& a,
                       cudaStream_t s) {
        if (!inverse)
            k_r2c_fast<T, LINES, NT, R0, R1, R2><<<grid, NT, smem(), s>>>(static_cast<const T*>(in), a);
        else
            k_c2r_fast<T, LINES, NT, R0, R1, R2><<<grid, NT, smem(), s>>>(static_cast<T*>(out), a);
    }
};

// Bulk-streamed c-pass configuration (FP32): LINES lines per tile, NBUF ring slots, MINB CTAs per SM
// (fewer where they do not fit).
template <int LINES, int NT, int R0, int R1, int R2, int NBUF, int MINB = 2, bool PAIR = false>
struct LineStreamCfg {
    static constexpr int lines = LINES, m = R0 * R1 * R2;
    using E = std::conditional_t<PAIR, f2x, float>;  // element of the work buffer and the twiddle tables
    static size_t smem_work() { return (size_t)LINES * (m + m / 16 + 1) * sizeof(cpx<float>) + NBUF * 8; }
    static size_t smem_r2c() {
        return (size_t)NBUF * LINES * m * sizeof(cpx<float>) + smem_work() +
               (size_t)LineTwLayout<R0, R1, R2>::fwd * sizeof(TwPair<E>);
    }
    static size_t smem_c2r(int ldc) {
        return (size_t)NBUF * LINES * ldc * sizeof(cpx<float>) + smem_work() +
               (size_t)LineTwLayout<R0, R1, R2>::inv * sizeof(cpx<E>);
    }
    static size_t smem() { return 0; }  // checked per kernel in configure()
    static auto r2c() {
        if constexpr (PAIR)
            return k_r2c_pair<LINES, NT, R0, R1, R2, NBUF, MINB>;
        else
            return k_r2c_stream<LINES, NT, R0, R1, R2, NBUF, MINB>;
    }
    static auto c2r() {
        if constexpr (PAIR)
            return k_c2r_pair<LINES, NT, R0, R1, R2, NBUF, MINB>;
        else
            return k_c2r_stream<LINES, NT, R0, R1, R2, NBUF, MINB>;
    }
    static cudaError_t configure(int optin) {
        cudaError_t e;
        if ((e = allow_max_dynamic_smem(r2c(), optin))) return e;
        return allow_max_dynamic_smem(c2r(), optin);
    }
    // CTAs per SM the persistent grid relies on: MINB, or fewer if they do not fit
    static int resident(bool inverse, size_t need) {
        int b = 0;
        const cudaError_t e = inverse ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, c2r(), NT, need)
                                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, r2c(), NT, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        return b < 1 ? 1 : (b < MINB ? b : MINB);
    }
    static long long launch(bool inverse, int sm_count, const void* in, void* out, const FastArgs<float>& a,
                            int* err, cudaStream_t s) {
        const long long nlines = (long long)a.n1 * a.n2;
        const int ntiles = (int)((nlines + LINES - 1) / LINES);
        const size_t need = inverse ? smem_c2r(a.ldc) : smem_r2c();
        int grid = resident(inverse, need) * sm_count;
        if (grid > ntiles) grid = ntiles;
        if (!inverse)
            r2c()<<<grid, NT, need, s>>>(static_cast<const float*>(in), a, ntiles, err);
        else
            c2r()<<<grid, NT, need, s>>>(static_cast<float*>(out), a, ntiles, err);
        return grid;
    }
};

// Streamed c passes by M = N3 / 2 (tiles of 32 KB of rho).
// Variant 1 (where it exists): one ring slot, three CTAs per SM.
template <class F>
bool with_line_stream_cfg(int m, int variant, F&& f) {
    switch (m) {
        case 128: f(LineStreamCfg<32, 256, 16, 8, 1, 2>{}); return true;
        case 256:
            if (variant == 1) f(LineStreamCfg<16, 256, 16, 16, 1, 1, 3>{});
            else f(LineStreamCfg<16, 256, 16, 16, 1, 2>{});
            return true;
        case 512: f(LineStreamCfg<8, 256, 8, 8, 8, 2>{}); return true;
        // mixed radices, variants 1, 2: each thread takes a butterfly of two lines (paired lanes)
        case 200:
            if (variant == 1) f(LineStreamCfg<16, 128, 8, 5, 5, 2, 3, true>{});
            else if (variant == 2) f(LineStreamCfg<16, 128, 8, 5, 5, 1, 4, true>{});
            else f(LineStreamCfg<16, 256, 8, 5, 5, 2>{});
            return true;
        case 105:
            if (variant == 1) f(LineStreamCfg<16, 128, 3, 5, 7, 2, 3, true>{});
            else if (variant == 2) f(LineStreamCfg<16, 128, 3, 5, 7, 1, 4, true>{});
            else f(LineStreamCfg<16, 256, 3, 5, 7, 2>{});
            return true;
        case 210:
            if (variant == 1) f(LineStreamCfg<16, 128, 6, 5, 7, 2, 3, true>{});
            else if (variant == 2) f(LineStreamCfg<16, 128, 6, 5, 7, 1, 4, true>{});
            else f(LineStreamCfg<16, 256, 6, 5, 7, 2>{});
            return true;
        default: return false;
    }
}
int line_stream_variants(int m) {
    if (m == 200 || m == 105 || m == 210) return 3;
    return m == 256 ? 2 : (with_line_stream_cfg(m, 0, [](auto) {}) ? 1 : 0);
}

// TMA-streamed column pass configuration (FP32): COLS columns (16: 128-byte rows, one CTA per
// SM; 8: 64-byte rows, MINB CTAs per SM, each with its own barriers) per tile.
template <int NT, int R0, int R1, int R2, int NBUF, int COLS = 16, int MINB = 1>
struct ColTmaCfg {
    static constexpr int cols = COLS, n = R0 * R1 * R2, minb = MINB;
    // tile ring, twiddles (MODE 2: the stage tables), mbarriers, reduction slots, alignment slack
    static size_t smem(int mode = 2) {
        const int tw = mode == 2 ? std::max(ColTwLayout<R0, R1, R2, 2>::total, n) : n;
        return (size_t)NBUF * n * COLS * sizeof(cpx<float>) + (size_t)tw * sizeof(TwPair<float>) + NBUF * 8 +
               (NT / 32) * sizeof(double) + 1024;
    }
    // CTAs per SM the launch relies on: MINB, or fewer if they do not fit
    static int resident(int mode) {
        static int r[3] = {0, 0, 0};
        if (r[mode] == 0) {
            int b = 0;
            cudaError_t e = mode == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                              &b, k_col_tma<COLS, NT, R0, R1, R2, 0, NBUF, MINB>, NT, smem(0))
                            : mode == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                              &b, k_col_tma<COLS, NT, R0, R1, R2, 1, NBUF, MINB>, NT, smem(1))
                                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                              &b, k_col_tma<COLS, NT, R0, R1, R2, 2, NBUF, MINB>, NT, smem(2));
            if (e != cudaSuccess) cudaGetLastError();
            r[mode] = e == cudaSuccess && b > 0 ? (b < MINB ? b : MINB) : 1;
        }
        return r[mode];
    }
    static cudaError_t configure(int optin) {
        cudaError_t e;
        if ((e = allow_max_dynamic_smem(k_col_tma<COLS, NT, R0, R1, R2, 0, NBUF, MINB>, optin))) return e;
        if ((e = allow_max_dynamic_smem(k_col_tma<COLS, NT, R0, R1, R2, 1, NBUF, MINB>, optin))) return e;
        return allow_max_dynamic_smem(k_col_tma<COLS, NT, R0, R1, R2, 2, NBUF, MINB>, optin);
    }
    static void launch(int mode, unsigned grid, const FastArgs<float>& a, const CUtensorMap& map, int ntiles,
                       int chunks, int* err, cudaStream_t s) {
        if (mode == 0)
            k_col_tma<COLS, NT, R0, R1, R2, 0, NBUF, MINB><<<grid, NT, smem(0), s>>>(a, map, ntiles, chunks, err);
        if (mode == 1)
            k_col_tma<COLS, NT, R0, R1, R2, 1, NBUF, MINB><<<grid, NT, smem(1), s>>>(a, map, ntiles, chunks, err);
        if (mode == 2)
            k_col_tma<COLS, NT, R0, R1, R2, 2, NBUF, MINB><<<grid, NT, smem(2), s>>>(a, map, ntiles, chunks, err);
    }
};

// TMA variants by line length: thread counts and radix orders (radix 32 stages
// halve the twiddle multiplies and shared-memory round trips of 8 x 8 x 8).
template <class F>
bool with_col_tma_cfg(int n, int variant, F&& f) {
    switch (n) {
        case 256:
            if (variant == 1) f(ColTmaCfg<128, 32, 8, 1, 3>{});
            else if (variant == 2) f(ColTmaCfg<128, 16, 16, 1, 3, 8, 3>{});
            else f(ColTmaCfg<256, 16, 16, 1, 3>{});
            return true;
        case 512:
            if (variant == 1) f(ColTmaCfg<256, 32, 16, 1, 3>{});
            else if (variant == 2) f(ColTmaCfg<256, 16, 32, 1, 3>{});
            else if (variant == 3) f(ColTmaCfg<256, 8, 8, 8, 3, 8, 2>{});
            else if (variant == 4) f(ColTmaCfg<128, 32, 16, 1, 3, 8, 2>{});
            else if (variant == 5) f(ColTmaCfg<256, 8, 8, 8, 2, 8, 3>{});
            else f(ColTmaCfg<512, 8, 8, 8, 3>{});
            return true;
        case 360:
            if (variant == 1) f(ColTmaCfg<256, 9, 5, 8, 3, 8, 2>{});
            else if (variant == 2) f(ColTmaCfg<512, 9, 5, 8, 3>{});
            else f(ColTmaCfg<512, 8, 5, 9, 3>{});
            return true;
        case 384:
            if (variant == 1) f(ColTmaCfg<256, 16, 8, 3, 3, 8, 2>{});
            else f(ColTmaCfg<512, 16, 8, 3, 3>{});
            return true;
        case 420:
            if (variant == 1) f(ColTmaCfg<256, 12, 5, 7, 2, 8, 3>{});
            else f(ColTmaCfg<256, 12, 5, 7, 3, 8, 2>{});
            return true;
        case 840:  // 12 x 7 x 10 or 10 x 7 x 12: 70 / 84, 120 and 84 / 70 butterflies per column
            if (variant == 1) f(ColTmaCfg<512, 10, 7, 12, 2, 8, 1>{});
            else f(ColTmaCfg<512, 12, 7, 10, 2, 8, 1>{});
            return true;
        default: return false;
    }
}

// Column-pass configurations by line length and variant.  Variant 0: rows of
// 128 bytes (16 FP32 / 8 FP64 complex columns per CTA); variant 1: half the
// columns and threads per CTA, so twice as many CTAs share an SM.
template <typename T, class F>
bool with_col_cfg(int n, int variant, F&& f) {
    constexpr bool d = sizeof(T) == 8;
    const bool v1 = variant == 1;
    switch (n) {
        case 16: f(ColCfg<T, d ? 16 : 32, d ? 64 : 128, 4, 4, 1>{}); return true;
        case 32: f(ColCfg<T, d ? 16 : 32, d ? 64 : 128, 8, 4, 1>{}); return true;
        case 64: f(ColCfg<T, d ? 8 : 16, d ? 64 : 128, 8, 8, 1>{}); return true;
        case 128: f(ColCfg<T, d ? 8 : 16, d ? 64 : 128, 16, 8, 1>{}); return true;
        case 256:
            if (v1) f(ColCfg<T, d ? 4 : 8, d ? 64 : 128, 16, 16, 1>{});
            else f(ColCfg<T, d ? 8 : 16, d ? 128 : 256, 16, 16, 1>{});
            return true;
        case 512:
            if (v1) f(ColCfg<T, d ? 4 : 8, d ? 128 : 256, 8, 8, 8>{});
            else f(ColCfg<T, d ? 8 : 16, d ? 256 : 512, 8, 8, 8>{});
            return true;
        case 1024: f(ColCfg<T, 8, 512, 16, 8, 8>{}); return true;
        case 360: f(ColCfg<T, d ? 8 : 16, 256, 8, 5, 9>{}); return true;
        case 420: f(ColCfg<T, 8, 256, 12, 5, 7>{}); return true;
        case 840: f(ColCfg<T, d ? 4 : 8, 512, 12, 7, 10>{}); return true;
        case 384: f(ColCfg<T, d ? 8 : 16, d ? 256 : 512, 16, 8, 3>{}); return true;
        default: return false;
    }
}
int col_variants(int n) { return (n == 256 || n == 512) ? 2 : 1; }
int col_tma_variants(int n) {
    return n == 512 ? 6 : (n == 256 ? 3 : (n == 360 ? 3 : (n == 384 || n == 420 || n == 840 ? 2 : 0)));
}

// Variants col_variants(n) .. of the b / a passes: the TMA-streamed kernels (FP32, plan has the tensor maps).
bool col_tma_available(const Plan& p, int axis) {
    return p.prec != HARTREE_FP64 && p.tma_ok && with_col_tma_cfg(p.n[axis], 0, [](auto) {});
}

// Variants of the b / a passes, in order: the plain kernels (col_variants), the TMA-streamed
// kernels (col_tma_variants, when available) and the paired-lane TMA kernels of pair_passes.cu.
int col_tma_count(const Plan& p, int axis) { return col_tma_available(p, axis) ? col_tma_variants(p.n[axis]) : 0; }
int col_pair_count(const Plan& p, int axis) { return col_pair_available(p, axis) ? col_pair_variants(p.n[axis]) : 0; }

// c-pass configurations by M = N3 / 2 and variant (variant 1: half the lines per CTA).
template <typename T, class F>
bool with_line_cfg(int m, int variant, F&& f) {
    const bool v1 = variant == 1;
    switch (m) {
        case 16: f(LineCfg<T, 32, 128, 4, 4, 1>{}); return true;
        case 32: f(LineCfg<T, 32, 128, 8, 4, 1>{}); return true;
        case 64: f(LineCfg<T, 16, 128, 8, 8, 1>{}); return true;
        case 128:
            if (v1) f(LineCfg<T, 8, 64, 16, 8, 1>{});
            else f(LineCfg<T, 16, 128, 16, 8, 1>{});
            return true;
        case 256:
            if (v1) f(LineCfg<T, 8, 128, 16, 16, 1>{});
            else f(LineCfg<T, 16, 256, 16, 16, 1>{});
            return true;
        case 512:
            if (v1) f(LineCfg<T, 2, 128, 8, 8, 8>{});
            else f(LineCfg<T, 4, 256, 8, 8, 8>{});
            return true;
        case 1024: f(LineCfg<T, 4, 256, 16, 8, 8>{}); return true;
        case 200: f(LineCfg<T, 16, 256, 8, 5, 5>{}); return true;
        case 105: f(LineCfg<T, 16, 256, 3, 5, 7>{}); return true;
        case 210: f(LineCfg<T, 16, 256, 6, 5, 7>{}); return true;
        default: return false;
    }
}
int line_variants(int m) { return (m == 128 || m == 256 || m == 512) ? 2 : 1; }

// Variant line_variants(M) of the c passes: the bulk-streamed kernels (FP32; the plan's
// row stride and the caller's grid pointers must allow 16-byte bulk copies).
bool line_stream_available(const Plan& p) {
    int lines = 0;
    if (p.prec == HARTREE_FP64 || p.d_err == nullptr || p.sm_count <= 0 || (p.ldc * 8) % 16 != 0 ||
        !with_line_stream_cfg(p.M, 0, [&](auto c) { lines = c.lines; }))
        return false;
    // every bulk copy of rho (lines of 8 M bytes) must be a multiple of 16 bytes: M even, or
    // whole tiles only (LINES even)
    return p.M % 2 == 0 || ((long long)p.n[0] * p.n[1]) % lines == 0;
}

// Arguments of pass `pass` (its b-pass tiles follow that pass's own variant).
template <typename T>
FastArgs<T> make_fast_args(const Plan& p, int pass) {
    FastArgs<T> a;
    a.n1 = p.n[0];
    a.n2 = p.n[1];
    a.n3 = p.n[2];
    a.M = p.M;
    a.nh = p.nh;
    a.ldc = p.ldc;
    a.twpa = static_cast<const TwPair<T>*>(p.twp[0]);
    a.twpb = static_cast<const TwPair<T>*>(p.twp[1]);
    a.twpc = static_cast<const TwPair<T>*>(p.twp[2]);
    a.gsqa = static_cast<const cpx<T>*>(p.gsq[0]);
    a.gsqb = static_cast<const cpx<T>*>(p.gsq[1]);
    a.gsqc = static_cast<const cpx<T>*>(p.gsq[2]);
    a.W = static_cast<cpx<T>*>(p.W);
    a.green_scale = T(4.0 * 3.14159265358979323846 / ((double)p.n[0] * p.n[1] * p.n[2]));
    a.eh_partials = p.eh_partials;
    a.a_chunks = 1;
    a.b_chunks = 1;
    with_col_cfg<T>(p.n[0], p.var[2], [&](auto c) { a.a_chunks = (p.nh + c.cols - 1) / c.cols; });
    with_col_cfg<T>(p.n[1], pass_variant(p, pass == 3 ? 3 : 1), [&](auto c) { a.b_chunks = (p.nh + c.cols - 1) / c.cols; });
    return a;
}

}  // namespace

// Which passes have a specialised kernel for this plan (bit 0: c, bit 1: b, bit 2: a).
template <typename T>
int fast_pass_mask_t(const Plan& p) {
    int m = 0;
    if (with_line_cfg<T>(p.M, 0, [](auto) {})) m |= 1;
    if (with_col_cfg<T>(p.n[1], 0, [](auto) {})) m |= 2;
    if (with_col_cfg<T>(p.n[0], 0, [](auto) {})) m |= 4;
    return m;
}

int fast_pass_mask(const Plan& p) {
    return p.prec == HARTREE_FP64 ? fast_pass_mask_t<double>(p) : fast_pass_mask_t<float>(p);
}

template <typename T>
cudaError_t configure_fast_t(const Plan& p, int optin) {
    cudaError_t e = cudaSuccess;
    auto cfg = [&](auto c) {
        if (e == cudaSuccess && c.smem() + 2048 > (size_t)optin) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) e = c.configure(optin);
    };
    for (int v = 0; v < line_variants(p.M); ++v) with_line_cfg<T>(p.M, v, cfg);
    if constexpr (sizeof(T) == 4) {
        if (line_stream_available(p))
            for (int v = 0; v < line_stream_variants(p.M); ++v)
                with_line_stream_cfg(p.M, v, [&](auto c) {
                    const size_t need = std::max(c.smem_r2c(), c.smem_c2r(p.ldc));
                    if (e == cudaSuccess && need + 2048 > (size_t)optin) e = cudaErrorInvalidConfiguration;
                    if (e == cudaSuccess) e = c.configure(optin);
                });
    }
    for (int v = 0; v < col_variants(p.n[1]); ++v) with_col_cfg<T>(p.n[1], v, cfg);
    for (int v = 0; v < col_variants(p.n[0]); ++v) with_col_cfg<T>(p.n[0], v, cfg);
    if constexpr (sizeof(T) == 4) {
        for (int ax = 0; ax < 2; ++ax)
            if (col_tma_available(p, ax))
                for (int v = 0; v < col_tma_variants(p.n[ax]); ++v) with_col_tma_cfg(p.n[ax], v, cfg);
        if (e == cudaSuccess) e = configure_col_pair(p, optin);
    }
    return e;
}

cudaError_t configure_fast_kernels(const Plan& p) {
    int optin = 0;
    cudaError_t e = optin_smem(&optin);
    if (e != cudaSuccess) return e;
    e = p.prec == HARTREE_FP64 ? configure_fast_t<double>(p, optin) : configure_fast_t<float>(p, optin);
    if (e == cudaSuccess && splat_fused_available(p)) e = configure_splat_fused(p, optin);
    return e;
}

// ------------------------------------------------------------------ the splat fused into the r2c pass
bool splat_fused_available(const Plan& p) {
    if (p.prec == HARTREE_FP64 || !(p.desc.flags & HARTREE_FLAG_FUSED_SPLAT) || p.sm_count <= 0) return false;
    return with_splat_line_cfg(p.M, [](auto) {});
}

// Staging of the fused splat: 2^fsh c factors per atom (the box, at most N3 wrapped points, rounded
// up to a power of two), kb atoms per batch (at most 16 KB of c factors) and cap atom records per
// unit (24 KB).
static void splat_fused_shape(const Plan& p, int* kb, int* fsh, int* cap) {
    const int w = std::min(p.box_max, p.n[2]);
    int sh = 1;
    while ((1 << sh) < w) ++sh;
    *fsh = sh;
    *kb = std::max(1, std::min(32, 4096 >> sh));
    *cap = 1024;
}

cudaError_t configure_splat_fused(const Plan& p, int optin) {
    int kb = 0, fsh = 0, cap = 0;
    splat_fused_shape(p, &kb, &fsh, &cap);
    cudaError_t e = cudaSuccess;
    with_splat_line_cfg(p.M, [&](auto c) {
        if (c.smem(kb, 1 << fsh, cap) + 2048 > (size_t)optin) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) e = allow_max_dynamic_smem(c.kernel(), optin);
    });
    return e;
}

long long launch_r2c_splat(const Plan& p, const AtomArgs<float>& at, cudaStream_t s) {
    int kb = 0, fsh = 0, cap = 0;
    splat_fused_shape(p, &kb, &fsh, &cap);
    const FastArgs<float> a = make_fast_args<float>(p, 0);
    long long grid = -1;
    with_splat_line_cfg(p.M, [&](auto c) {
        const int tiles_b = (p.n[1] + c.lines - 1) / c.lines;
        const int nunits = p.n[0] * ((tiles_b + kFuseSeg - 1) / kFuseSeg);
        // axes along which a box can exceed the grid (several images of an atom on one point)
        const int img = (p.box_max > p.n[0] ? 1 : 0) | (p.box_max > p.n[1] ? 2 : 0) | (p.box_max > p.n[2] ? 4 : 0);
        const size_t sm = c.smem(kb, 1 << fsh, cap);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c.kernel(), 256, sm) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        grid = std::min<long long>(nunits, (long long)per_sm * p.sm_count);
        c.kernel()<<<(unsigned)grid, 256, sm, s>>>(at, a, tiles_b, nunits, kb, fsh, cap, img);
    });
    return grid;
}

// pass: 0 = c r2c (rho -> W), 1 = b forward, 2 = a with Green, 3 = b inverse, 4 = c c2r (W -> vh).
// Returns the number of CTAs launched (the a pass's E_H partial count), or -1 if not specialised.
template <typename T>
long long launch_fast_pass_t(const Plan& p, int pass, const void* rho, void* vh, cudaStream_t s) {
    FastArgs<T> a = make_fast_args<T>(p, pass);
    long long grid = -1;
    if (pass == 0 || pass == 4) {
        const int v = pass_variant(p, pass);
        if constexpr (sizeof(T) == 4) {
            const void* grid_ptr = pass == 0 ? rho : vh;
            const int sv = v - line_variants(p.M);
            if (sv >= 0 && line_stream_available(p) && reinterpret_cast<uintptr_t>(grid_ptr) % 16 == 0) {
                with_line_stream_cfg(p.M, sv, [&](auto c) {
                    grid = c.launch(pass == 4, p.sm_count, rho, vh, a, p.d_err, s);
                });
                return grid;
            }
        }
        const int lv = v < line_variants(p.M) ? v : 0;  // misaligned grid: plain kernel
        with_line_cfg<T>(p.M, lv, [&](auto c) {
            grid = ((long long)p.n[0] * p.n[1] + c.lines - 1) / c.lines;
            c.launch(pass == 4, (unsigned)grid, rho, vh, a, s);
        });
        return grid;
    }
    const int axis = (pass == 2) ? 0 : 1;  // transformed axis: a for pass 2, b for passes 1 and 3
    if constexpr (sizeof(T) == 4) {
        const int tv = pass_variant(p, pass) - col_variants(p.n[axis]);
        const int pv = tv - col_tma_count(p, axis);
        if (pv >= 0 && col_pair_available(p, axis)) return launch_col_pair(p, pass, pv, a, s);
        if (tv >= 0 && col_tma_available(p, axis)) {
            // TMA-streamed persistent kernel, one CTA per SM
            with_col_tma_cfg(p.n[axis], tv, [&](auto c) {
                const int chunks = (p.nh + c.cols - 1) / c.cols;
                const int ntiles = p.n[1 - axis] * chunks;
                const int mode = pass == 1 ? 0 : (pass == 3 ? 1 : 2);
                const int slots = c.resident(mode) * p.sm_count;
                grid = ntiles < slots ? ntiles : slots;
                const CUtensorMap& map = c.cols == 16 ? (axis == 0 ? p.tmap_a : p.tmap_b)
                                                      : (axis == 0 ? p.tmap_a8 : p.tmap_b8);
                c.launch(pass == 1 ? 0 : (pass == 3 ? 1 : 2), (unsigned)grid, a, map, ntiles, chunks, p.d_err, s);
            });
            return grid;
        }
    }
    with_col_cfg<T>(p.n[axis], pass_variant(p, pass), [&](auto c) {
        grid = (long long)p.n[1 - axis] * (axis == 0 ? a.a_chunks : a.b_chunks);
        c.launch(pass == 2 ? 2 : (pass == 3 ? 1 : 0), (unsigned)grid, a, s);
    });
    return grid;
}

long long launch_fast_pass(const Plan& p, int pass, const void* rho, void* vh, cudaStream_t s) {
    return p.prec == HARTREE_FP64 ? launch_fast_pass_t<double>(p, pass, rho, vh, s)
                                  : launch_fast_pass_t<float>(p, pass, rho, vh, s);
}

int single_variants(const Plan& p, int kind) {
    if (kind == 0)
        return (p.use_fast & 1) ? line_variants(p.M) + (line_stream_available(p) ? line_stream_variants(p.M) : 0)
                                : 1;
    const int ax = kind == 1 ? 1 : 0;
    if (!(p.use_fast & (kind == 1 ? 2 : 4))) return 1;
    return col_variants(p.n[ax]) + col_tma_count(p, ax) + col_pair_count(p, ax);
}

void pair_variants(int V, int v, int* first, int* second) {
    if (v < V || V < 2) {
        *first = *second = v < V ? v : 0;
        return;
    }
    const int m = v - V, r = m / (V - 1), c = m % (V - 1);
    *first = r;
    *second = c < r ? c : c + 1;
}

int pair_index(int V, int first, int second) {
    if (first == second) return first;
    return V + first * (V - 1) + (second < first ? second : second - 1);
}

int fast_variants(const Plan& p, int kind) {
    const int V = single_variants(p, kind);
    return kind == 2 ? V : V * V;
}

// The variant pass `pass` (0..4) runs under the plan's picks.
int pass_variant(const Plan& p, int pass) {
    if (pass == 2) return p.var[2];
    const int kind = (pass == 0 || pass == 4) ? 0 : 1;
    int first = 0, second = 0;
    pair_variants(single_variants(p, kind), p.var[kind], &first, &second);
    return (pass == 0 || pass == 1) ? first : second;
}

// ------------------------------------------------------------------ host: tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

bool encode_tensor_map_3d(CUtensorMap* map, void* base, const uint64_t dims[3], const uint64_t strides[2],
                          const uint32_t box[3]) {
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t gd[3] = {dims[0], dims[1], dims[2]};
    const cuuint64_t gs[2] = {strides[0], strides[1]};
    const cuuint32_t bd[3] = {box[0], box[1], box[2]};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, gd, gs, bd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps over the half spectrum W (FP32, viewed as floats [N1][N2][2 ldc]) for the b and a
// column passes: boxes of 16, 8 or 4 complex columns by up to 256 rows.
void prepare_tma(Plan& p) {
    p.tma_ok = false;
    if (p.prec == HARTREE_FP64) return;
    const uint64_t dims[3] = {(uint64_t)2 * p.ldc, (uint64_t)p.n[1], (uint64_t)p.n[0]};
    const uint64_t strides[2] = {(uint64_t)2 * p.ldc * 4, (uint64_t)p.n[1] * 2 * p.ldc * 4};
    const uint32_t box_b[3] = {32, (uint32_t)box_rows(p.n[1]), 1};
    const uint32_t box_a[3] = {32, 1, (uint32_t)box_rows(p.n[0])};
    const uint32_t box_b8[3] = {16, (uint32_t)box_rows(p.n[1]), 1};
    const uint32_t box_a8[3] = {16, 1, (uint32_t)box_rows(p.n[0])};
    const uint32_t box_b4[3] = {8, (uint32_t)box_rows(p.n[1]), 1};
    const uint32_t box_a4[3] = {8, 1, (uint32_t)box_rows(p.n[0])};
    const bool ok_b = encode_tensor_map_3d(&p.tmap_b, p.W, dims, strides, box_b) &&
                      encode_tensor_map_3d(&p.tmap_b8, p.W, dims, strides, box_b8) &&
                      encode_tensor_map_3d(&p.tmap_b4, p.W, dims, strides, box_b4);
    const bool ok_a = encode_tensor_map_3d(&p.tmap_a, p.W, dims, strides, box_a) &&
                      encode_tensor_map_3d(&p.tmap_a8, p.W, dims, strides, box_a8) &&
                      encode_tensor_map_3d(&p.tmap_a4, p.W, dims, strides, box_a4);
    p.tma_ok = ok_a && ok_b && p.d_err != nullptr && p.sm_count > 0;
}

}  // namespace hartree
