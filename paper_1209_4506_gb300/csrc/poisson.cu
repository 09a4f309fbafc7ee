// poisson.cu -- the five HBM sweeps of the periodic Poisson solve.
//
// Sec. 2.1 solves for the Hartree potential with FFT; Sec. 3.2.4 orders the
// transforms abc -> cab -> cba -> cab -> abc.  On one GPU the "structure B"
// redistributions between those orders become the choice of which axis a pass
// transforms, and the passes are:
//   1. c  : real-to-complex along c (packed N3/2-point complex transform +
//           split post-process), rho[N1][N2][N3] -> W[N1][N2][ldc]
//   2. b  : forward along b, in place on W
//   3. a  : forward along a, multiply by 4 pi / |G|^2 (G = 0 -> 0, the
//           neutralising background) with the 1/N normalisation folded in,
//           accumulate the E_H partial sum, inverse along a -- all on one
//           tile resident in shared memory (one HBM round trip)
//   4. b^-1
//   5. c^-1: complex-to-real along c, W -> V_H[N1][N2][N3]
// followed by a one-block FP64 reduction of the E_H partials (fixed order,
// deterministic).
#include "internal.cuh"

namespace hartree {

namespace {

// ---------------------------------------------------------------- pass 1: c r2c
template <typename T>
__global__ void __launch_bounds__(kThreads) k_c_r2c(const T* __restrict__ rho, PoissonArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = a.c_lines, ld = L + 1, M = a.M;
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* B = A + (size_t)(M + 1) * ld;
    const long long nlines = (long long)a.n1 * a.n2;
    const long long line0 = (long long)blockIdx.x * L;
    const int nl = (int)min((long long)L, nlines - line0);
    // z[n] = rho[2n] + i rho[2n+1]: coalesced along the line, transposed into [n][line]
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = e / M, n = e - l * M;
        const cpx<T>* src = reinterpret_cast<const cpx<T>*>(rho + (line0 + l) * a.n3);
        A[n * ld + l] = src[n];
    }
    __syncthreads();
    cpx<T>* Z = run_fft_to_smem<T, false>(a.rpc, SmemTile<T>{A, ld}, B, A, ld, nl, a.twc, 2);
    // X[k] = E[k] + w^k O[k],  E = (Z[k] + conj Z[M-k]) / 2,  O = (Z[k] - conj Z[M-k]) / 2i,  k = 0..M
    const T half = T(0.5);
    for (int e = threadIdx.x; e < nl * (M + 1); e += blockDim.x) {
        const int l = e / (M + 1), k = e - l * (M + 1);
        const cpx<T> z1 = Z[(k == M ? 0 : k) * ld + l];
        const cpx<T> z2 = conjg(Z[(k == 0 ? 0 : M - k) * ld + l]);
        const cpx<T> E = scale(z1 + z2, half);
        const cpx<T> d = z1 - z2;
        const cpx<T> O = mk(d.im * half, -d.re * half);
        a.W[(line0 + l) * a.ldc + k] = E + a.twc[k] * O;
    }
}

// ---------------------------------------------------------------- passes 2 / 4: b
template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads) k_b(PoissonArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int CB = a.b_cols;
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* B = A + (size_t)a.n2 * CB;
    const int ia = blockIdx.x / a.b_chunks;
    const int c0 = (blockIdx.x - ia * a.b_chunks) * CB;
    const int nc = min(CB, a.nh - c0);
    GlobalTile<T> g{a.W + (long long)ia * a.n2 * a.ldc + c0, a.ldc};
    if (a.rpb.nst >= 2) {
        run_fft<T, INV>(a.rpb, g, g, A, B, CB, nc, a.twb, 1);
    } else {
        // one stage reads and writes different rows: go through shared memory
        cpx<T>* F = run_fft_to_smem<T, INV>(a.rpb, g, A, B, CB, nc, a.twb, 1);
        for (int e = threadIdx.x; e < a.n2 * nc; e += blockDim.x) {
            const int col = e % nc, n = e / nc;
            g.st_(col, n, F[n * CB + col]);
        }
    }
}

// ---------------------------------------------------------------- pass 3: a + Green + E_H + a^-1
template <typename T>
__global__ void __launch_bounds__(kThreads) k_a_green(PoissonArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kThreads / 32];
    const int CA = a.a_cols;
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* B = A + (size_t)a.n1 * CA;
    const int ib = blockIdx.x / a.a_chunks;
    const int c0 = (blockIdx.x - ib * a.a_chunks) * CA;
    const int nc = min(CA, a.nh - c0);
    GlobalTile<T> g{a.W + (long long)ib * a.ldc + c0, (long long)a.n2 * a.ldc};
    cpx<T>* F = run_fft_to_smem<T, false>(a.rpa, g, A, B, CA, nc, a.twa, 1);
    // F[k1][col] now holds rho~(k1, ib, c0 + col).
    const cpx<T> gb = a.gsqb[ib];
    T sum = T(0), comp = T(0);  // compensated per-thread partial of sum m |rho~|^2 / G^2
    for (int e = threadIdx.x; e < a.n1 * nc; e += blockDim.x) {
        const int col = e % nc, k1 = e / nc;
        const int k3 = c0 + col;
        const cpx<T> v = F[k1 * CA + col];
        // |G|^2 from the split tables: the high parts sum to within one rounding,
        // the low parts restore the table rounding (no systematic error on 1/|G|^2)
        const cpx<T> ga = a.gsqa[k1], gc = a.gsqc[k3];
        const T G2 = ((ga.re + gb.re) + gc.re) + ((ga.im + gb.im) + gc.im);
        const T inv = (G2 > T(0)) ? T(1) / G2 : T(0);
        const T mult = (k3 == 0 || k3 == a.M) ? T(1) : T(2);
        const T term = mult * (v.re * v.re + v.im * v.im) * inv - comp;
        const T t = sum + term;
        comp = (t - sum) - term;
        sum = t;
        F[k1 * CA + col] = scale(v, inv * a.green_scale);
    }
    const double bs = block_sum_comp(sum, -comp, red);
    if (threadIdx.x == 0) a.eh_partials[blockIdx.x] = bs;
    __syncthreads();
    cpx<T>* other = (F == A) ? B : A;
    run_fft<T, true>(a.rpa, SmemTile<T>{F, CA}, g, other, F, CA, nc, a.twa, 1);
}

// ---------------------------------------------------------------- pass 5: c c2r
template <typename T>
__global__ void __launch_bounds__(kThreads) k_c_c2r(T* __restrict__ out, PoissonArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = a.c_lines, ld = L + 1, M = a.M;
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* B = A + (size_t)(M + 1) * ld;
    const long long nlines = (long long)a.n1 * a.n2;
    const long long line0 = (long long)blockIdx.x * L;
    const int nl = (int)min((long long)L, nlines - line0);
    for (int e = threadIdx.x; e < nl * (M + 1); e += blockDim.x) {
        const int l = e / (M + 1), k = e - l * (M + 1);
        A[k * ld + l] = a.W[(line0 + l) * a.ldc + k];
    }
    __syncthreads();
    // Z[k] = (X[k] + conj X[M-k]) + i w^-k (X[k] - conj X[M-k]),  k < M
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = e / M, k = e - l * M;
        const cpx<T> x1 = A[k * ld + l];
        const cpx<T> x2 = conjg(A[(M - k) * ld + l]);
        const cpx<T> Ep = x1 + x2;
        const cpx<T> Op = (x1 - x2) * conjg(a.twc[k]);
        B[k * ld + l] = mk(Ep.re - Op.im, Ep.im + Op.re);
    }
    __syncthreads();
    cpx<T>* z = run_fft_to_smem<T, true>(a.rpc, SmemTile<T>{B, ld}, A, B, ld, nl, a.twc, 2);
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = e / M, n = e - l * M;
        reinterpret_cast<cpx<T>*>(out + (line0 + l) * a.n3)[n] = z[n * ld + l];
    }
}

// ---------------------------------------------------------------- E_H finalise
__global__ void __launch_bounds__(kThreads) k_eh_finalize(const double* __restrict__ part, int np, double factor,
                                                          double* __restrict__ eh) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
    const double t = block_sum_double(s, red);
    if (threadIdx.x == 0) *eh = factor * t;
}

template <typename T>
PoissonArgs<T> make_args(const Plan& p) {
    PoissonArgs<T> a;
    a.n1 = p.n[0];
    a.n2 = p.n[1];
    a.n3 = p.n[2];
    a.M = p.M;
    a.nh = p.nh;
    a.ldc = p.ldc;
    a.rpa = p.rp[0];
    a.rpb = p.rp[1];
    a.rpc = p.rp[2];
    a.twa = static_cast<const cpx<T>*>(p.tw[0]);
    a.twb = static_cast<const cpx<T>*>(p.tw[1]);
    a.twc = static_cast<const cpx<T>*>(p.tw[2]);
    a.gsqa = static_cast<const cpx<T>*>(p.gsq[0]);
    a.gsqb = static_cast<const cpx<T>*>(p.gsq[1]);
    a.gsqc = static_cast<const cpx<T>*>(p.gsq[2]);
    a.W = static_cast<cpx<T>*>(p.W);
    const double ntot = (double)p.n[0] * p.n[1] * p.n[2];
    a.green_scale = T(4.0 * 3.14159265358979323846 / ntot);
    a.eh_partials = p.eh_partials;
    a.c_lines = p.c_lines;
    a.b_cols = p.b_cols;
    a.a_cols = p.a_cols;
    a.b_chunks = (p.nh + p.b_cols - 1) / p.b_cols;
    a.a_chunks = (p.nh + p.a_cols - 1) / p.a_cols;
    return a;
}

// One pass; returns the number of CTAs of the a pass (its E_H partial count) for pass 2.
template <typename T>
long long pass_impl(const Plan& p, int pass, const void* rho, void* vh, cudaStream_t s) {
    const int bit = (pass == 0 || pass == 4) ? 1 : ((pass == 1 || pass == 3) ? 2 : 4);
    ++p.launches;
    if (p.use_fast & bit) return launch_fast_pass(p, pass, rho, vh, s);
    PoissonArgs<T> a = make_args<T>(p);
    const long long nlines = (long long)p.n[0] * p.n[1];
    const unsigned gc = (unsigned)((nlines + p.c_lines - 1) / p.c_lines);
    const unsigned gb = (unsigned)(p.n[0] * a.b_chunks);
    const unsigned ga = (unsigned)(p.n[1] * a.a_chunks);
    switch (pass) {
        case 0: k_c_r2c<T><<<gc, kThreads, p.smem_c, s>>>(static_cast<const T*>(rho), a); return gc;
        case 1: k_b<T, false><<<gb, kThreads, p.smem_b, s>>>(a); return gb;
        case 2: k_a_green<T><<<ga, kThreads, p.smem_a, s>>>(a); return ga;
        case 3: k_b<T, true><<<gb, kThreads, p.smem_b, s>>>(a); return gb;
        default: k_c_c2r<T><<<gc, kThreads, p.smem_c, s>>>(static_cast<T*>(vh), a); return gc;
    }
}

template <typename T>
cudaError_t poisson_impl(const Plan& p, const void* rho, void* vh, double* eh, cudaStream_t s) {
    long long n_part = 0;
    for (int pass = 0; pass < 5; ++pass) {
        const long long g = pass_impl<T>(p, pass, rho, vh, s);
        if (pass == 2) n_part = g;
    }
    if (eh) {
        const double ntot = (double)p.n[0] * p.n[1] * p.n[2];
        const double factor = 2.0 * 3.14159265358979323846 * p.omega / (ntot * ntot);
        k_eh_finalize<<<1, kThreads, 0, s>>>(p.eh_partials, (int)n_part, factor, eh);
        ++p.launches;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t configure_poisson(int optin) {
    cudaError_t e;
    if ((e = allow_max_dynamic_smem(k_c_r2c<T>, optin))) return e;
    if ((e = allow_max_dynamic_smem(k_c_c2r<T>, optin))) return e;
    if ((e = allow_max_dynamic_smem(k_b<T, false>, optin))) return e;
    if ((e = allow_max_dynamic_smem(k_b<T, true>, optin))) return e;
    return allow_max_dynamic_smem(k_a_green<T>, optin);
}

}  // namespace

cudaError_t launch_poisson(const Plan& p, const void* rho, void* vh, double* eh, cudaStream_t s) {
    return p.prec == HARTREE_FP64 ? poisson_impl<double>(p, rho, vh, eh, s) : poisson_impl<float>(p, rho, vh, eh, s);
}

cudaError_t launch_poisson_pass(const Plan& p, int pass, const void* rho, void* vh, cudaStream_t s) {
    if (p.prec == HARTREE_FP64)
        pass_impl<double>(p, pass, rho, vh, s);
    else
        pass_impl<float>(p, pass, rho, vh, s);
    return cudaGetLastError();
}

cudaError_t configure_poisson_kernels(const Plan& p) {
    int optin = 0;
    cudaError_t e = optin_smem(&optin);
    if (e != cudaSuccess) return e;
    if (p.smem_a + 1024 > (size_t)optin || p.smem_b > (size_t)optin || p.smem_c > (size_t)optin)
        return cudaErrorInvalidConfiguration;
    return p.prec == HARTREE_FP64 ? configure_poisson<double>(optin) : configure_poisson<float>(optin);
}

}  // namespace hartree
