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
#include "passes_dev.cuh"

namespace hartree {

namespace {

template <typename T>
__global__ void __launch_bounds__(kThreads) k_c_r2c(const T* __restrict__ rho, PoissonArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c_r2c_tile<T, false>(rho, a, blockIdx.x, smem_raw);
}

template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads) k_b(PoissonArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    b_tile<T, INV, false>(a, blockIdx.x, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_a_green(PoissonArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kThreads / 32];
    a_green_tile<T, false>(a, blockIdx.x, blockIdx.x, smem_raw, red);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_c_c2r(T* __restrict__ out, PoissonArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c_c2r_tile<T, false>(out, a, blockIdx.x, smem_raw);
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


// One pass; returns the number of CTAs of the a pass (its E_H partial count) for pass 2.
template <typename T>
long long pass_impl(const Plan& p, int pass, const void* rho, void* vh, cudaStream_t s) {
    const int bit = (pass == 0 || pass == 4) ? 1 : ((pass == 1 || pass == 3) ? 2 : 4);
    ++p.launches;
    if (p.prec == HARTREE_FP32_TC_SPLIT && (pass == 1 || pass == 3)) return launch_tc_pass(p, pass, s);
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
cudaError_t poisson_impl(const Plan& p, int first, const void* rho, void* vh, double* eh, cudaStream_t s) {
    long long n_part = 0;
    for (int pass = first; pass < 5; ++pass) {
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
    return launch_poisson_from(p, 0, rho, vh, eh, s);
}

cudaError_t launch_poisson_from(const Plan& p, int first, const void* rho, void* vh, double* eh, cudaStream_t s) {
    return p.prec == HARTREE_FP64 ? poisson_impl<double>(p, first, rho, vh, eh, s)
                                  : poisson_impl<float>(p, first, rho, vh, eh, s);
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
