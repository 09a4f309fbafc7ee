// noalloc.cu -- hartree_solve_density_noalloc: the Poisson solve of a density
// already on the grid, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: applications that hand all device
// memory to their own allocator or pool up front, and code running where a
// cudaMalloc is not allowed or would stall other work.  This entry point
// needs no plan (creating a plan allocates its workspace): its scratch -- the
// half spectrum, the twiddle and |G|^2 tables and the E_H partial sums -- lives
// in one file-scope __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits.  It calls no cudaMalloc,
// cudaFree or other allocating routine.
//
// Host code cannot use the array's name as a device address (it names a
// host-side stand-in), so the first call on each device looks the address up
// with cudaGetSymbolAddress, with that device current, and keeps it.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace hartree {

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

int noalloc_fail(int status, const char* msg) {
    set_last_error(msg);  // reported by hartree_last_error()
    return status;
}

bool smooth_na(int n) {  // 2/3/5/7-smooth
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

bool radix_plan_na(int n, RadixPlan* rp) {
    rp->n = n;
    rp->nst = 0;
    int e2 = 0, m = n, n3 = 0, n5 = 0, n7 = 0;
    while (m % 2 == 0) m /= 2, ++e2;
    while (m % 3 == 0) m /= 3, ++n3;
    while (m % 5 == 0) m /= 5, ++n5;
    while (m % 7 == 0) m /= 7, ++n7;
    if (m != 1) return false;
    if (e2 > 0) {
        const int st = (e2 + 3) / 4;
        for (int s = 0; s < st; ++s) rp->r[rp->nst++] = 1 << (e2 / st + (s < e2 % st ? 1 : 0));
    }
    for (int i = 0; i < n3; ++i) rp->r[rp->nst++] = 3;
    for (int i = 0; i < n5; ++i) rp->r[rp->nst++] = 5;
    for (int i = 0; i < n7; ++i) rp->r[rp->nst++] = 7;
    return rp->nst >= 1 && rp->nst <= kMaxStages;
}

// Twiddle tables (plain and high/low pairs) and |G|^2 pairs of one axis, in FP64 then rounded.
template <typename T>
__global__ void k_noalloc_tables(int n, int len_g, double L, cpx<T>* tw, TwPair<T>* twp, cpx<T>* gsq) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        double s, c;
        sincospi(2.0 * (double)k / (double)n, &s, &c);  // exp(-2 pi i k / n) = c - i s
        const T cr = (T)c, ci = (T)(-s);
        tw[k] = mk(cr, ci);
        TwPair<T> w;
        w.h = mk(cr, ci);
        w.l = mk((T)(c - (double)cr), (T)(-s - (double)ci));
        twp[k] = w;
    }
    if (k < len_g) {
        const int kk = (2 * k <= n) ? k : k - n;
        const double G = 6.283185307179586476925286766559 * kk / L;
        const double g2 = G * G;
        const T hi = (T)g2;
        gsq[k] = mk(hi, (T)(g2 - (double)hi));
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

}  // namespace hartree

using namespace hartree;

extern "C" int hartree_solve_density_noalloc(const hartree_desc* desc, const void* rho, void* vh, double* eh,
                                             void* stream) {
    if (!desc || !rho || !vh) return noalloc_fail(HARTREE_ERR_INVALID, "solve_density_noalloc: null argument");
    const hartree_desc& d = *desc;
    if (d.flags != 0 || (d.precision != HARTREE_FP64 && d.precision != HARTREE_FP32))
        return noalloc_fail(HARTREE_ERR_INVALID, "solve_density_noalloc: precision must be FP64 or FP32, flags 0");
    for (int i = 0; i < 3; ++i) {
        if (d.n[i] < 2 || d.n[i] > kMaxAxis || !smooth_na(d.n[i]))
            return noalloc_fail(HARTREE_ERR_UNSUPPORTED_SIZE, "solve_density_noalloc: a grid size is not 2/3/5/7-smooth");
        if (!(d.cell[i] > 0.0) || !std::isfinite(d.cell[i]))
            return noalloc_fail(HARTREE_ERR_INVALID, "solve_density_noalloc: cell sides must be positive");
    }
    if (d.n[2] % 2 != 0 || d.n[2] < 4)
        return noalloc_fail(HARTREE_ERR_UNSUPPORTED_SIZE, "solve_density_noalloc: N3 must be even and >= 4");
    const uintptr_t pair = d.precision == HARTREE_FP64 ? 16 : 8;  // grid lines move as (re, im) pairs
    if (reinterpret_cast<uintptr_t>(rho) % pair != 0 || reinterpret_cast<uintptr_t>(vh) % pair != 0)
        return noalloc_fail(HARTREE_ERR_INVALID, pair == 16 ? "solve_density_noalloc: grids must be aligned to 16 bytes"
                                                            : "solve_density_noalloc: grids must be aligned to 8 bytes");

    Plan p;
    p.desc = d;
    p.prec = d.precision;
    p.real_size = p.prec == HARTREE_FP64 ? sizeof(double) : sizeof(float);
    const size_t cs = 2 * p.real_size;
    for (int i = 0; i < 3; ++i) {
        p.n[i] = d.n[i];
        p.L[i] = d.cell[i];
        p.h[i] = d.cell[i] / d.n[i];
    }
    p.M = p.n[2] / 2;
    p.nh = p.M + 1;
    const int align = p.prec == HARTREE_FP64 ? 8 : 16;
    p.ldc = (p.nh + align - 1) / align * align;
    p.omega = p.L[0] * p.L[1] * p.L[2];
    p.dV = p.omega / ((double)p.n[0] * p.n[1] * p.n[2]);
    for (int i = 0; i < 3; ++i)
        if (!radix_plan_na(i == 2 ? p.M : p.n[i], &p.rp[i]))
            return noalloc_fail(HARTREE_ERR_UNSUPPORTED_SIZE, "solve_density_noalloc: no radix plan");
    const size_t budget = 64 * 1024;
    p.c_lines = (int)(budget / (2 * (size_t)(p.M + 1) * cs)) - 1;
    p.c_lines = p.c_lines > 32 ? 32 : (p.c_lines < 2 ? 2 : p.c_lines);
    p.c_lines &= ~1;
    p.b_cols = (int)(budget / (2 * (size_t)p.n[1] * cs));
    p.a_cols = (int)(budget / (2 * (size_t)p.n[0] * cs));
    p.b_cols = p.b_cols > 16 ? 16 : (p.b_cols < 1 ? 1 : p.b_cols);
    p.a_cols = p.a_cols > 16 ? 16 : (p.a_cols < 1 ? 1 : p.a_cols);
    p.smem_c = 2 * (size_t)(p.M + 1) * (p.c_lines + 1) * cs;
    p.smem_b = 2 * (size_t)p.n[1] * p.b_cols * cs;
    p.smem_a = 2 * (size_t)p.n[0] * p.a_cols * cs;
    p.n_eh_partials = p.n[1] * p.nh;
    p.use_fast = fast_pass_mask(p);

    // scratch layout: half spectrum, tables, E_H partials (each 256-byte aligned)
    const size_t sz_W = align256((size_t)p.n[0] * p.n[1] * p.ldc * cs);
    size_t sz_tw[3], sz_twp[3], sz_g[3];
    for (int i = 0; i < 3; ++i) {
        sz_tw[i] = align256((size_t)p.n[i] * cs);
        sz_twp[i] = align256((size_t)p.n[i] * 2 * cs);
        sz_g[i] = align256((size_t)(i == 2 ? p.nh : p.n[i]) * cs);
    }
    const size_t sz_e = align256((size_t)p.n_eh_partials * sizeof(double));
    size_t need = sz_W + sz_e;
    for (int i = 0; i < 3; ++i) need += sz_tw[i] + sz_twp[i] + sz_g[i];
    if (need > kNoAllocScratchBytes)
        return noalloc_fail(HARTREE_ERR_UNSUPPORTED_SIZE,
                            "solve_density_noalloc: the grid needs more than the 8 MiB static scratch "
                            "(half spectrum N1*N2*ceil16(N3/2+1)*8 bytes in FP32, *16 in FP64, plus tables)");

    // set-up, once per device: the scratch array's device address
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(HARTREE_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(HARTREE_ERR_CUDA, "solve_density_noalloc: device ordinal");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr)
                return noalloc_fail(HARTREE_ERR_CUDA, "solve_density_noalloc: cudaGetSymbolAddress failed");
            g_noalloc_addr[dev] = ptr;
        }
        base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    }
    size_t off = 0;
    p.W = base + off;
    off += sz_W;
    for (int i = 0; i < 3; ++i) {
        p.tw[i] = base + off;
        off += sz_tw[i];
        p.twp[i] = base + off;
        off += sz_twp[i];
        p.gsq[i] = base + off;
        off += sz_g[i];
    }
    p.eh_partials = reinterpret_cast<double*>(base + off);

    e = configure_poisson_kernels(p);
    if (e == cudaSuccess) e = configure_fast_kernels(p);
    if (e != cudaSuccess) return noalloc_fail(HARTREE_ERR_CUDA, cudaGetErrorString(e));

    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < 3; ++i) {
        const int len_g = i == 2 ? p.nh : p.n[i];
        const int len = p.n[i] > len_g ? p.n[i] : len_g;
        if (p.prec == HARTREE_FP64)
            k_noalloc_tables<double><<<(len + 127) / 128, 128, 0, s>>>(
                p.n[i], len_g, p.L[i], static_cast<cpx<double>*>(p.tw[i]), static_cast<TwPair<double>*>(p.twp[i]),
                static_cast<cpx<double>*>(p.gsq[i]));
        else
            k_noalloc_tables<float><<<(len + 127) / 128, 128, 0, s>>>(
                p.n[i], len_g, p.L[i], static_cast<cpx<float>*>(p.tw[i]), static_cast<TwPair<float>*>(p.twp[i]),
                static_cast<cpx<float>*>(p.gsq[i]));
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_poisson(p, rho, vh, eh, s);
    return e == cudaSuccess ? HARTREE_OK : noalloc_fail(HARTREE_ERR_CUDA, cudaGetErrorString(e));
}
