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
// with cudaGetSymbolAddress, with that device current, and keeps it together
// with the identity of the CUDA context it belongs to.  If that context is
// later torn down and another created (cudaDeviceReset, or the primary context
// released and retained again), the module is loaded anew and the array may
// move: a call that finds a different context looks the address up again.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace hartree {

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Per device: the context the cached set-up belongs to (its process-unique ID), the scratch
// array's address in it, and the precision and grid whose kernels were last configured there
// (the kernels' shared-memory attributes; a new grid may use other kernels).
struct NoAllocDevice {
    unsigned long long ctx_id = 0;  // 0: nothing cached
    void* addr = nullptr;
    int conf[4] = {-1, 0, 0, 0};  // precision, N1, N2, N3 last configured (-1: none)
};
std::mutex g_noalloc_mutex;
NoAllocDevice g_noalloc_dev[kMaxDevices];

int noalloc_fail(int status, const char* msg) {
    set_last_error(msg);  // reported by hartree_last_error()
    return status;
}

// The process-unique ID of the current CUDA context (driver entry points cuCtxGetCurrent and
// cuCtxGetId, looked up through the runtime); false if there is none or the driver lacks them.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {  // called with g_noalloc_mutex held
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS && *id != 0;
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
        if (d.n[i] < 2 || d.n[i] > kMaxAxis || !smooth_size(d.n[i]))
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
    {
        const int st = init_plan_geometry(p, d);
        if (st != HARTREE_OK) return st;
    }
    const size_t cs = 2 * p.real_size;

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

    // set-up, once per device and context: the scratch array's device address and the kernels'
    // shared-memory attributes
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(HARTREE_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(HARTREE_ERR_CUDA, "solve_density_noalloc: device ordinal");
    unsigned char* base = nullptr;
    bool configured = false;
    const int key[4] = {p.prec, p.n[0], p.n[1], p.n[2]};
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        NoAllocDevice& nd = g_noalloc_dev[dev];
        unsigned long long id = 0;
        const bool have_id = current_context_id(&id);
        if (!have_id || nd.ctx_id != id || !nd.addr) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);  // creates the context if there is none yet
            if (e != cudaSuccess || !ptr)
                return noalloc_fail(HARTREE_ERR_CUDA, "solve_density_noalloc: cudaGetSymbolAddress failed");
            unsigned long long id2 = 0;
            nd = NoAllocDevice{};
            nd.addr = ptr;
            nd.ctx_id = current_context_id(&id2) ? id2 : 0;  // 0: look the address up again next call
        }
        base = static_cast<unsigned char*>(nd.addr);
        configured = std::equal(key, key + 4, nd.conf);
    }
    if (!configured) {
        e = configure_poisson_kernels(p);
        if (e == cudaSuccess) e = configure_fast_kernels(p);
        if (e != cudaSuccess) return noalloc_fail(HARTREE_ERR_CUDA, cudaGetErrorString(e));
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        std::copy(key, key + 4, g_noalloc_dev[dev].conf);
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
