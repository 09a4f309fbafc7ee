// fft_engine.cuh -- device building blocks of the line transforms of the
// Poisson solve (Sec. 2.1: "the Hartree potential is found by solving the
// Poisson equation using FFT"; pass order of Sec. 3.2.4).
//
// A tile is `ncol` independent lines of length N, all transformed together.
// Stockham autosort stages (radix R, sub-transform size Ns) read butterfly j
// at j + r N/R and write it at (j / Ns) Ns R + (j mod Ns) + r Ns, so every
// stage reads with unit stride across butterflies and the output comes out in
// natural order without a bit-reversal pass.  Threads run column-fastest:
// neighbouring threads handle neighbouring columns, which are contiguous in
// global memory for the b and a passes and in the [n][ld] shared-memory
// layout, so loads, stores and shared-memory accesses are conflict-free.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace hartree {

template <typename T>
struct __align__(2 * sizeof(T)) cpx {
    T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T r, T i) {
    cpx<T> z;
    z.re = r;
    z.im = i;
    return z;
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) {
    return mk(a.re + b.re, a.im + b.im);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) {
    return mk(a.re - b.re, a.im - b.im);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// Two FP32 lanes as one value (the .f32x2 add, mul and fma of sm_100-class GPUs): the butterflies
// below, instantiated with T = f2x, transform two columns at once.  Negation flips the sign bits
// (integer pipe) instead of multiplying by -1.
struct f2x {
    float2 v;
    f2x() = default;
    __device__ __forceinline__ explicit f2x(float2 x) : v(x) {}
    __device__ __forceinline__ explicit f2x(double s) : v(make_float2((float)s, (float)s)) {}
    __device__ __forceinline__ explicit f2x(int s) : v(make_float2((float)s, (float)s)) {}
};
__device__ __forceinline__ f2x operator+(f2x a, f2x b) { return f2x(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2x operator-(f2x a) {
    return f2x(make_float2(__int_as_float(__float_as_int(a.v.x) ^ 0x80000000),
                           __int_as_float(__float_as_int(a.v.y) ^ 0x80000000)));
}
// a - b as b (-1) + a: exact product, one rounding, the same result as a subtraction
__device__ __forceinline__ f2x operator-(f2x a, f2x b) { return f2x(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ f2x operator*(f2x a, f2x b) { return f2x(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2x fma_t(f2x a, f2x b, f2x c) { return f2x(__ffma2_rn(a.v, b.v, c.v)); }

template <typename T>
__host__ __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) {
    return mk(a.re * s, a.im * s);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> conjg(cpx<T> a) {
    return mk(a.re, -a.im);
}
// a * (-i) for the forward sign, a * (+i) for the inverse sign.
template <typename T, bool INV>
__host__ __device__ __forceinline__ cpx<T> rot90(cpx<T> a) {
    return INV ? mk(-a.im, a.re) : mk(a.im, -a.re);
}

// ------------------------------------------------------------------ constants
// Multiplication by a real constant c.  In FP32 the product uses c split into
// a rounded high part and the remainder, so the constant carries no rounding
// bias: a single-rounded sqrt(1/2) shrinks |w| below 1 at every radix-8
// stage, which shows up as a systematic loss of spectral energy (E_H).
template <typename T, bool COMP = true>
__host__ __device__ __forceinline__ T kmul(T x, double c) {
    if constexpr (sizeof(T) == 4 && COMP) {
        const float hi = (float)c;
        const float lo = (float)(c - (double)hi);
        return fmaf(x, hi, x * lo);
    } else if constexpr (std::is_same<T, f2x>::value && COMP) {
        const float hi = (float)c;
        const float lo = (float)(c - (double)hi);
        return fma_t(x, T((double)hi), x * T((double)lo));
    } else {
        return x * (T)c;
    }
}
// (a + ib) (cr + i ci) for a constant twiddle
template <typename T, bool COMP = true>
__host__ __device__ __forceinline__ cpx<T> kcmul(cpx<T> a, double cr, double ci) {
    return mk(kmul<T, COMP>(a.re, cr) - kmul<T, COMP>(a.im, ci), kmul<T, COMP>(a.re, ci) + kmul<T, COMP>(a.im, cr));
}

// ------------------------------------------------------------------ small DFTs
// v[k] <- sum_m v[m] exp(-+ 2 pi i m k / R)   (minus: forward, plus: INV)

template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft2(cpx<T>* v) {
    cpx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}

template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft3(cpx<T>* v) {
    const double s = 0.86602540378443864676372317075294;  // sin(2 pi / 3)
    cpx<T> t = v[1] + v[2];
    cpx<T> d = v[1] - v[2];
    cpx<T> m = v[0] - scale(t, T(0.5));
    cpx<T> r = rot90<T, INV>(mk(kmul<T, COMP>(d.re, s), kmul<T, COMP>(d.im, s)));  // -+ i s (x1 - x2)
    v[0] = v[0] + t;
    v[1] = m + r;
    v[2] = m - r;
}

template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft4(cpx<T>* v) {
    cpx<T> s02 = v[0] + v[2], d02 = v[0] - v[2];
    cpx<T> s13 = v[1] + v[3], d13 = rot90<T, INV>(v[1] - v[3]);
    v[0] = s02 + s13;
    v[2] = s02 - s13;
    v[1] = d02 + d13;
    v[3] = d02 - d13;
}

template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft5(cpx<T>* v) {
    const double c1 = 0.30901699437494742410229341718282;   // cos(2 pi / 5)
    const double c2 = -0.80901699437494742410229341718282;  // cos(4 pi / 5)
    const double s1 = 0.95105651629515357211643933337938;   // sin(2 pi / 5)
    const double s2 = 0.58778525229247312916870595463907;   // sin(4 pi / 5)
    cpx<T> a1 = v[1] + v[4], b1 = v[1] - v[4];
    cpx<T> a2 = v[2] + v[3], b2 = v[2] - v[3];
    cpx<T> x0 = v[0];
    cpx<T> p1 = mk(x0.re + kmul<T, COMP>(a1.re, c1) + kmul<T, COMP>(a2.re, c2), x0.im + kmul<T, COMP>(a1.im, c1) + kmul<T, COMP>(a2.im, c2));
    cpx<T> p2 = mk(x0.re + kmul<T, COMP>(a1.re, c2) + kmul<T, COMP>(a2.re, c1), x0.im + kmul<T, COMP>(a1.im, c2) + kmul<T, COMP>(a2.im, c1));
    cpx<T> q1 = rot90<T, INV>(mk(kmul<T, COMP>(b1.re, s1) + kmul<T, COMP>(b2.re, s2), kmul<T, COMP>(b1.im, s1) + kmul<T, COMP>(b2.im, s2)));
    cpx<T> q2 = rot90<T, INV>(mk(kmul<T, COMP>(b1.re, s2) - kmul<T, COMP>(b2.re, s1), kmul<T, COMP>(b1.im, s2) - kmul<T, COMP>(b2.im, s1)));
    v[0] = x0 + a1 + a2;
    v[1] = p1 + q1;
    v[4] = p1 - q1;
    v[2] = p2 + q2;
    v[3] = p2 - q2;
}

template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft8(cpx<T>* v) {
    const double r = 0.70710678118654752440084436210485;
    cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4<T, INV, COMP>(e);
    dft4<T, INV, COMP>(o);
    // w8^k = exp(-+ 2 pi i k / 8), k = 1, 2, 3
    cpx<T> o1 = INV ? mk(kmul<T, COMP>(o[1].re - o[1].im, r), kmul<T, COMP>(o[1].re + o[1].im, r))
                    : mk(kmul<T, COMP>(o[1].re + o[1].im, r), kmul<T, COMP>(o[1].im - o[1].re, r));
    cpx<T> o2 = rot90<T, INV>(o[2]);
    cpx<T> o3 = INV ? mk(-kmul<T, COMP>(o[3].re + o[3].im, r), kmul<T, COMP>(o[3].re - o[3].im, r))
                    : mk(kmul<T, COMP>(o[3].im - o[3].re, r), -kmul<T, COMP>(o[3].re + o[3].im, r));
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = e[2] + o2;
    v[6] = e[2] - o2;
    v[3] = e[3] + o3;
    v[7] = e[3] - o3;
}

// Radix 7 from the symmetric pairs a_k = x_k + x_(7-k), b_k = x_k - x_(7-k):
// X[m] = p_m -+ i q_m and X[7-m] = p_m +- i q_m with p_m = x_0 + sum_k a_k cos(2 pi k m / 7)
// and q_m = sum_k b_k sin(2 pi k m / 7).
template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft7(cpx<T>* v) {
    const double C[4] = {1.0, 0.623489801858733530525, -0.222520933956314404289, -0.900968867902419126236};
    const double S[4] = {0.0, 0.781831482468029808708, 0.974927912181823607018, 0.433883739117558120475};
    cpx<T> a[4], b[4];
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        a[k] = v[k] + v[7 - k];
        b[k] = v[k] - v[7 - k];
    }
    const cpx<T> x0 = v[0];
    v[0] = ((x0 + a[1]) + a[2]) + a[3];
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        cpx<T> pm = x0, qm = mk(T(0), T(0));
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            const int j = (k * m) % 7;
            const double cj = j <= 3 ? C[j] : C[7 - j];
            const double sj = j <= 3 ? S[j] : -S[7 - j];
            pm = mk(pm.re + kmul<T, COMP>(a[k].re, cj), pm.im + kmul<T, COMP>(a[k].im, cj));
            qm = mk(qm.re + kmul<T, COMP>(b[k].re, sj), qm.im + kmul<T, COMP>(b[k].im, sj));
        }
        const cpx<T> r = rot90<T, INV>(qm);
        v[m] = pm + r;
        v[7 - m] = pm - r;
    }
}

// Radix 12 as 4 x 3: with n = 3 n1 + n2 and k = k1 + 4 k2, three 4-point DFTs over
// n1, the twiddles w12^(n2 k1), then four 3-point DFTs over n2.
template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft12(cpx<T>* v) {
    const double h = 0.866025403784438646764;  // cos(pi / 6) = sin(pi / 3)
    const double sg = INV ? 1.0 : -1.0;
    cpx<T> y[3][4];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
        cpx<T> t[4] = {v[n2], v[n2 + 3], v[n2 + 6], v[n2 + 9]};
        dft4<T, INV, COMP>(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = t[k1];
    }
    y[1][1] = kcmul<T, COMP>(y[1][1], h, sg * 0.5);  // w12^1
    y[1][2] = kcmul<T, COMP>(y[1][2], 0.5, sg * h);  // w12^2
    y[1][3] = rot90<T, INV>(y[1][3]);                // w12^3
    y[2][1] = kcmul<T, COMP>(y[2][1], 0.5, sg * h);  // w12^2
    y[2][2] = kcmul<T, COMP>(y[2][2], -0.5, sg * h);  // w12^4
    y[2][3] = mk(-y[2][3].re, -y[2][3].im);          // w12^6
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        cpx<T> t[3] = {y[0][k1], y[1][k1], y[2][k1]};
        dft3<T, INV, COMP>(t);
        v[k1] = t[0];
        v[k1 + 4] = t[1];
        v[k1 + 8] = t[2];
    }
}

// Radix 6 as 2 x 3: with n = 3 n1 + n2 and k = k1 + 2 k2, three 2-point DFTs over n1, the
// twiddles w6^(n2 k1) (w6 = exp(-+ 2 pi i / 6)), then two 3-point DFTs over n2.
template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft6(cpx<T>* v) {
    const double h = 0.866025403784438646764;  // sin(pi / 3)
    const double sg = INV ? 1.0 : -1.0;
    cpx<T> y[3][2];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
        y[n2][0] = v[n2] + v[n2 + 3];
        y[n2][1] = v[n2] - v[n2 + 3];
    }
    y[1][1] = kcmul<T, COMP>(y[1][1], 0.5, sg * h);   // w6^1
    y[2][1] = kcmul<T, COMP>(y[2][1], -0.5, sg * h);  // w6^2
#pragma unroll
    for (int k1 = 0; k1 < 2; ++k1) {
        cpx<T> t[3] = {y[0][k1], y[1][k1], y[2][k1]};
        dft3<T, INV, COMP>(t);
        v[k1] = t[0];
        v[k1 + 2] = t[1];
        v[k1 + 4] = t[2];
    }
}

// Radix 10 as 2 x 5: with n = 5 n1 + n2 and k = k1 + 2 k2, five 2-point DFTs over n1, the
// twiddles w10^(n2 k1), then two 5-point DFTs over n2.
template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft10(cpx<T>* v) {
    // cos and sin of 2 pi m / 10, m = 1 .. 4
    const double C[5] = {1.0, 0.80901699437494742410229341718282, 0.30901699437494742410229341718282,
                         -0.30901699437494742410229341718282, -0.80901699437494742410229341718282};
    const double S[5] = {0.0, 0.58778525229247312916870595463907, 0.95105651629515357211643933337938,
                         0.95105651629515357211643933337938, 0.58778525229247312916870595463907};
    const double sg = INV ? 1.0 : -1.0;
    cpx<T> y[5][2];
#pragma unroll
    for (int n2 = 0; n2 < 5; ++n2) {
        y[n2][0] = v[n2] + v[n2 + 5];
        y[n2][1] = v[n2] - v[n2 + 5];
    }
#pragma unroll
    for (int n2 = 1; n2 < 5; ++n2) y[n2][1] = kcmul<T, COMP>(y[n2][1], C[n2], sg * S[n2]);  // w10^n2
#pragma unroll
    for (int k1 = 0; k1 < 2; ++k1) {
        cpx<T> t[5] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1], y[4][k1]};
        dft5<T, INV, COMP>(t);
#pragma unroll
        for (int k2 = 0; k2 < 5; ++k2) v[k1 + 2 * k2] = t[k2];
    }
}

// Radix 9 as 3 x 3: with n = 3 n1 + n2 and k = k1 + 3 k2, three 3-point DFTs over
// n1, the twiddles w9^(n2 k1), then three 3-point DFTs over n2.
template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft9(cpx<T>* v) {
    const double c1 = 0.766044443118978035, s1 = 0.642787609686539326;   // cos, sin(2 pi / 9)
    const double c2 = 0.173648177666930349, s2 = 0.984807753012208059;   // cos, sin(4 pi / 9)
    const double c4 = -0.939692620785908384, s4 = 0.342020143325668733;  // cos, sin(8 pi / 9)
    const double sg = INV ? 1.0 : -1.0;
    cpx<T> y[3][3];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
        cpx<T> t[3] = {v[n2], v[n2 + 3], v[n2 + 6]};
        dft3<T, INV, COMP>(t);
        y[n2][0] = t[0];
        y[n2][1] = t[1];
        y[n2][2] = t[2];
    }
    y[1][1] = kcmul<T, COMP>(y[1][1], c1, sg * s1);
    y[1][2] = kcmul<T, COMP>(y[1][2], c2, sg * s2);
    y[2][1] = kcmul<T, COMP>(y[2][1], c2, sg * s2);
    y[2][2] = kcmul<T, COMP>(y[2][2], c4, sg * s4);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        cpx<T> t[3] = {y[0][k1], y[1][k1], y[2][k1]};
        dft3<T, INV, COMP>(t);
        v[k1] = t[0];
        v[k1 + 3] = t[1];
        v[k1 + 6] = t[2];
    }
}

// Radix 16 and 32 from two halves of half the size and the twiddles
// exp(-+ 2 pi i k / R) = cos(2 pi k / R) -+ i sin(2 pi k / R).
template <typename T, int R, bool INV, bool COMP>
__host__ __device__ __forceinline__ void dft_halves(cpx<T>* v);

template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft16(cpx<T>* v) {
    dft_halves<T, 16, INV, COMP>(v);
}
template <typename T, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft32(cpx<T>* v) {
    dft_halves<T, 32, INV, COMP>(v);
}

template <typename T, int R, bool INV, bool COMP>
__host__ __device__ __forceinline__ void dft_halves(cpx<T>* v) {
    // cos(pi k / 16) and sin(pi k / 16), k = 0..16 (radix 32 uses every entry, radix 16 every second)
    const double C[17] = {1.0,
                          0.98078528040323044912618223613424,
                          0.92387953251128675612818318939679,
                          0.83146961230254523707878837761791,
                          0.70710678118654752440084436210485,
                          0.55557023301960222474283081394853,
                          0.38268343236508977172845998403040,
                          0.19509032201612826784828486847702,
                          0.0,
                          -0.19509032201612826784828486847702,
                          -0.38268343236508977172845998403040,
                          -0.55557023301960222474283081394853,
                          -0.70710678118654752440084436210485,
                          -0.83146961230254523707878837761791,
                          -0.92387953251128675612818318939679,
                          -0.98078528040323044912618223613424,
                          -1.0};
    constexpr int H = R / 2;
    constexpr int step = 32 / R;  // index step into the pi/16 tables
    cpx<T> e[H], o[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
        e[m] = v[2 * m];
        o[m] = v[2 * m + 1];
    }
    if constexpr (H == 8) {
        dft8<T, INV, COMP>(e);
        dft8<T, INV, COMP>(o);
    } else {
        dft16<T, INV, COMP>(e);
        dft16<T, INV, COMP>(o);
    }
#pragma unroll
    for (int k = 0; k < H; ++k) {
        cpx<T> t;
        if (k == 0) {
            t = o[0];
        } else if (2 * k == H) {
            t = rot90<T, INV>(o[k]);
        } else {
            // angle 2 pi k / R = pi (k step) / 16; sin(pi m / 16) = cos(pi (8 - m) / 16)
            const int m = k * step;
            const double c = C[m];
            const double sn = m <= 8 ? C[8 - m] : C[m - 8];
            t = kcmul<T, COMP>(o[k], c, INV ? sn : -sn);
        }
        v[k] = e[k] + t;
        v[k + H] = e[k] - t;
    }
}

// COMP (FP32 only): constants carried as high/low pairs.  Forward transforms,
// whose spectrum feeds E_H, use it; inverse transforms, which only shape V_H,
// may use plain constants.
template <typename T, int R, bool INV, bool COMP = true>
__host__ __device__ __forceinline__ void dft(cpx<T>* v) {
    if constexpr (R == 2) dft2<T, INV, COMP>(v);
    if constexpr (R == 3) dft3<T, INV, COMP>(v);
    if constexpr (R == 4) dft4<T, INV, COMP>(v);
    if constexpr (R == 5) dft5<T, INV, COMP>(v);
    if constexpr (R == 6) dft6<T, INV, COMP>(v);
    if constexpr (R == 7) dft7<T, INV, COMP>(v);
    if constexpr (R == 8) dft8<T, INV, COMP>(v);
    if constexpr (R == 9) dft9<T, INV, COMP>(v);
    if constexpr (R == 10) dft10<T, INV, COMP>(v);
    if constexpr (R == 12) dft12<T, INV, COMP>(v);
    if constexpr (R == 16) dft16<T, INV, COMP>(v);
    if constexpr (R == 32) dft32<T, INV, COMP>(v);
}

// ------------------------------------------------------------------ radix plans
constexpr int kMaxStages = 14;

struct RadixPlan {
    int n;                  // line length
    int nst;                // number of stages
    int r[kMaxStages];      // radix of each stage (2, 3, 4, 5, 7, 8 or 16)
};

// ------------------------------------------------------------------ accessors
// Column `col` of a tile, element n of the line.
template <typename T>
struct SmemTile {
    cpx<T>* p;
    int ld;
    __device__ __forceinline__ cpx<T> ld_(int col, int n) const { return p[n * ld + col]; }
    __device__ __forceinline__ void st_(int col, int n, cpx<T> v) const { p[n * ld + col] = v; }
};

// Global load; CG = true bypasses L1 (ld.global.cg), needed when the data was
// written by another CTA of the same launch (L1 is not coherent across SMs).
template <bool CG, typename T>
__device__ __forceinline__ cpx<T> gload(const cpx<T>* p) {
    if constexpr (CG) {
        if constexpr (sizeof(T) == 4) {
            const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
            return mk(v.x, v.y);
        } else {
            const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
            return mk(v.x, v.y);
        }
    } else {
        return *p;
    }
}

template <typename T, bool CG = false>
struct GlobalTile {
    cpx<T>* p;
    long long sn;  // element stride along the line
    __device__ __forceinline__ cpx<T> ld_(int col, int n) const { return gload<CG>(p + (long long)n * sn + col); }
    __device__ __forceinline__ void st_(int col, int n, cpx<T> v) const { p[(long long)n * sn + col] = v; }
};

// x / d by a multiply-high with m = ceil(2^32 / d) (m = 0 marks d = 1).  Exact when
// x (m d - 2^32) < 2^32, which holds for x < 2^20 and d <= 4096.
__device__ __forceinline__ uint32_t fdiv_magic(uint32_t d) { return d <= 1u ? 0u : 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ uint32_t fdiv(uint32_t x, uint32_t m) { return m == 0u ? x : __umulhi(x, m); }

// One Stockham stage over a tile.  tw[e * tws] = exp(-2 pi i e / N) for the
// line length N (tws > 1 when the table belongs to a longer line).  The index
// divisions by the run-time ncol and Ns use precomputed multiply-high constants.
template <typename T, int R, bool INV, class Src, class Dst>
__device__ __forceinline__ void stage(const Src& src, const Dst& dst, int N, int Ns, int ncol,
                                      const cpx<T>* __restrict__ tw, int tws) {
    const int nb = N / R;
    const int total = nb * ncol;
    const int tstep = N / (Ns * R);
    const uint32_t mc = fdiv_magic((uint32_t)ncol), ms = fdiv_magic((uint32_t)Ns);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int j = (int)fdiv((uint32_t)t, mc);
        const int col = t - j * ncol;
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src.ld_(col, j + r * nb);
        const int k = j - (int)fdiv((uint32_t)j, ms) * Ns;
        if (Ns > 1) {
            const int base = k * tstep;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                cpx<T> w = tw[(base * r) * tws];
                if (INV) w = conjg(w);
                v[r] = v[r] * w;
            }
        }
        dft<T, R, INV>(v);
        const int o = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst.st_(col, o + r * Ns, v[r]);
    }
}

template <typename T, bool INV, class Src, class Dst>
__device__ __forceinline__ void stage_any(int R, const Src& src, const Dst& dst, int N, int Ns, int ncol,
                                          const cpx<T>* __restrict__ tw, int tws) {
    switch (R) {
        case 2: stage<T, 2, INV>(src, dst, N, Ns, ncol, tw, tws); break;
        case 3: stage<T, 3, INV>(src, dst, N, Ns, ncol, tw, tws); break;
        case 4: stage<T, 4, INV>(src, dst, N, Ns, ncol, tw, tws); break;
        case 5: stage<T, 5, INV>(src, dst, N, Ns, ncol, tw, tws); break;
        case 7: stage<T, 7, INV>(src, dst, N, Ns, ncol, tw, tws); break;
        case 8: stage<T, 8, INV>(src, dst, N, Ns, ncol, tw, tws); break;
        case 16: stage<T, 16, INV>(src, dst, N, Ns, ncol, tw, tws); break;
        default: break;
    }
}

// Full transform of a tile, src -> dst, through two shared-memory ping-pong
// buffers A and B (each N x ld).  Stage 0 writes A, so a source that lives in
// shared memory must be B (or a third buffer), never A.  With a single stage
// src and dst must not overlap (stage 0 reads and writes in one sweep).
template <typename T, bool INV, class Src, class Dst>
__device__ void run_fft(const RadixPlan& rp, const Src& src, const Dst& dst, cpx<T>* A, cpx<T>* B, int ld, int ncol,
                        const cpx<T>* __restrict__ tw, int tws) {
    const int N = rp.n;
    if (rp.nst == 1) {
        stage_any<T, INV>(rp.r[0], src, dst, N, 1, ncol, tw, tws);
        return;
    }
    SmemTile<T> bufs[2] = {{A, ld}, {B, ld}};
    int Ns = 1;
    stage_any<T, INV>(rp.r[0], src, bufs[0], N, Ns, ncol, tw, tws);
    Ns *= rp.r[0];
    __syncthreads();
    int cur = 0;
    for (int s = 1; s < rp.nst - 1; ++s) {
        stage_any<T, INV>(rp.r[s], bufs[cur], bufs[cur ^ 1], N, Ns, ncol, tw, tws);
        Ns *= rp.r[s];
        cur ^= 1;
        __syncthreads();
    }
    stage_any<T, INV>(rp.r[rp.nst - 1], bufs[cur], dst, N, Ns, ncol, tw, tws);
}

// Transform from `src` into shared memory.  The result lands in A or B; the
// returned pointer says which.  Stage 0 writes A, so a shared-memory source
// must be B.  Ends with __syncthreads().
template <typename T, bool INV, class Src>
__device__ cpx<T>* run_fft_to_smem(const RadixPlan& rp, const Src& src, cpx<T>* A, cpx<T>* B, int ld, int ncol,
                                   const cpx<T>* __restrict__ tw, int tws) {
    const int N = rp.n;
    SmemTile<T> bufs[2] = {{A, ld}, {B, ld}};
    int Ns = 1;
    stage_any<T, INV>(rp.r[0], src, bufs[0], N, Ns, ncol, tw, tws);
    Ns *= rp.r[0];
    __syncthreads();
    int cur = 0;
    for (int s = 1; s < rp.nst; ++s) {
        stage_any<T, INV>(rp.r[s], bufs[cur], bufs[cur ^ 1], N, Ns, ncol, tw, tws);
        Ns *= rp.r[s];
        cur ^= 1;
        __syncthreads();
    }
    return bufs[cur].p;
}

}  // namespace hartree
