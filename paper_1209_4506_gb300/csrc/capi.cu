// capi.cu -- plan creation and the extern "C" entry points of hartree.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace hartree;

namespace {

thread_local std::string g_last_error;

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(HARTREE_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Radices for a line of length n: powers of two in balanced stages of at
// most 16, then the factors 3, 5 and 7 one stage each.
bool make_radix_plan(int n, RadixPlan* rp) {
    rp->n = n;
    rp->nst = 0;
    int e2 = 0, m = n;
    while (m % 2 == 0) {
        m /= 2;
        ++e2;
    }
    int n3 = 0, n5 = 0, n7 = 0;
    while (m % 3 == 0) {
        m /= 3;
        ++n3;
    }
    while (m % 5 == 0) {
        m /= 5;
        ++n5;
    }
    while (m % 7 == 0) {
        m /= 7;
        ++n7;
    }
    if (m != 1) return false;
    if (e2 > 0) {
        const int st = (e2 + 3) / 4;
        for (int s = 0; s < st; ++s) {
            const int bits = e2 / st + (s < e2 % st ? 1 : 0);
            rp->r[rp->nst++] = 1 << bits;
        }
    }
    for (int i = 0; i < n3; ++i) rp->r[rp->nst++] = 3;
    for (int i = 0; i < n5; ++i) rp->r[rp->nst++] = 5;
    for (int i = 0; i < n7; ++i) rp->r[rp->nst++] = 7;
    if (rp->nst == 0) rp->r[rp->nst++] = 2;  // n == 1 never reaches here (n >= 2)
    return rp->nst <= kMaxStages;
}

// exp(-2 pi i k / n), k < n, evaluated in extended precision and rounded once.
void twiddles(int n, std::vector<double>& re, std::vector<double>& im) {
    re.resize(n);
    im.resize(n);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int k = 0; k < n; ++k) {
        const long double a = two_pi * (long double)k / (long double)n;
        re[k] = (double)cosl(a);
        im[k] = (double)(-sinl(a));
    }
}

// (2 pi k' / L)^2 with k' = k for k <= n/2, k - n otherwise.
std::vector<double> gsq_table(int n, int len, double L) {
    std::vector<double> g(len);
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < len; ++k) {
        const int kk = (2 * k <= n) ? k : k - n;
        const double G = two_pi * kk / L;
        g[k] = G * G;
    }
    return g;
}

template <typename T>
int upload_tables(Plan& p) {
    for (int d = 0; d < 3; ++d) {
        std::vector<double> re, im;
        twiddles(p.n[d], re, im);
        std::vector<T> buf(2 * (size_t)p.n[d]);
        for (int k = 0; k < p.n[d]; ++k) {
            buf[2 * k] = (T)re[k];
            buf[2 * k + 1] = (T)im[k];
        }
        cudaError_t e = cudaMemcpy(p.tw[d], buf.data(), buf.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e) return cuda_fail(e, "upload twiddles");
        std::vector<T> pairs(4 * (size_t)p.n[d]);  // (hi.re, hi.im, lo.re, lo.im) per k
        for (int k = 0; k < p.n[d]; ++k) {
            const T hr = (T)re[k], hi = (T)im[k];
            pairs[4 * k] = hr;
            pairs[4 * k + 1] = hi;
            pairs[4 * k + 2] = (T)(re[k] - (double)hr);
            pairs[4 * k + 3] = (T)(im[k] - (double)hi);
        }
        e = cudaMemcpy(p.twp[d], pairs.data(), pairs.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e) return cuda_fail(e, "upload twiddle pairs");
        const int len = d == 2 ? p.nh : p.n[d];
        std::vector<double> g = gsq_table(p.n[d], len, p.L[d]);
        std::vector<T> gb(2 * (size_t)len);  // |G_d|^2 as a high part and the rounding remainder
        for (int k = 0; k < len; ++k) {
            gb[2 * k] = (T)g[k];
            gb[2 * k + 1] = (T)(g[k] - (double)gb[2 * k]);
        }
        e = cudaMemcpy(p.gsq[d], gb.data(), gb.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e) return cuda_fail(e, "upload |G|^2 tables");
    }
    return HARTREE_OK;
}

void free_plan(Plan& p) {
    void* ptrs[] = {p.W,           p.R,        p.tw[0],         p.tw[1], p.tw[2], p.twp[0], p.twp[1], p.twp[2], p.gsq[0],
                    p.gsq[1],      p.gsq[2],   p.eh_partials,   p.leaf_box,
                    p.atom_prep,   p.atom_fac, p.atom_dfac, p.force_partials, p.d_pos,   p.d_q,   p.d_f,   p.d_eh,
                    p.d_err,       p.bin_cursor, p.bin_list, p.tc_dft, p.bisect, p.force_order};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (p.host_graph) cudaGraphExecDestroy(p.host_graph);
    if (p.host_event) cudaEventDestroy(p.host_event);
    if (p.host_stream) cudaStreamDestroy(p.host_stream);
}

bool finite_pos(double x) { return std::isfinite(x); }

}  // namespace

void hartree::set_last_error(const char* msg) { g_last_error = msg; }

bool hartree::smooth_size(int n) {  // 2/3/5/7-smooth
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Grid geometry, radix plans and pass tiling: everything the Poisson passes read from a plan
// besides its device buffers.  hartree_plan_create and the allocation-free solve both build
// their plans with it, so the two run the same passes with the same tiles.
int hartree::init_plan_geometry(Plan& p, const hartree_desc& d) {
    p.desc = d;
    p.prec = d.precision;
    p.real_size = p.prec == HARTREE_FP64 ? sizeof(double) : sizeof(float);
    for (int i = 0; i < 3; ++i) {
        p.n[i] = d.n[i];
        p.L[i] = d.cell[i];
        p.h[i] = d.cell[i] / d.n[i];
    }
    p.M = p.n[2] / 2;
    p.nh = p.M + 1;
    {
        const int align = p.prec == HARTREE_FP64 ? 8 : 16;  // 128-byte rows
        p.ldc = (p.nh + align - 1) / align * align;
    }
    p.omega = p.L[0] * p.L[1] * p.L[2];
    p.dV = p.omega / ((double)p.n[0] * p.n[1] * p.n[2]);
    for (int i = 0; i < 3; ++i) {
        const int len = i == 2 ? p.M : p.n[i];
        if (!make_radix_plan(len, &p.rp[i]))
            return fail(HARTREE_ERR_UNSUPPORTED_SIZE, "plan: no radix plan for length %d", len);
    }
    // tiling of the generic passes: two ping-pong buffers per CTA, about 64 KB of shared memory
    const size_t cs = 2 * p.real_size;  // complex element
    const size_t budget = 64 * 1024;
    p.c_lines = (int)(budget / (2 * (size_t)(p.M + 1) * cs)) - 1;
    if (p.c_lines > 32) p.c_lines = 32;
    if (p.c_lines < 2) p.c_lines = 2;
    p.c_lines &= ~1;  // even, so the padded leading dimension L + 1 is odd
    p.b_cols = (int)(budget / (2 * (size_t)p.n[1] * cs));
    p.a_cols = (int)(budget / (2 * (size_t)p.n[0] * cs));
    p.b_cols = p.b_cols > 16 ? 16 : (p.b_cols < 1 ? 1 : p.b_cols);
    p.a_cols = p.a_cols > 16 ? 16 : (p.a_cols < 1 ? 1 : p.a_cols);
    p.smem_c = 2 * (size_t)(p.M + 1) * (p.c_lines + 1) * cs;
    p.smem_b = 2 * (size_t)p.n[1] * p.b_cols * cs;
    p.smem_a = 2 * (size_t)p.n[0] * p.a_cols * cs;
    p.n_eh_partials = p.n[1] * p.nh;  // enough for one a-pass CTA per (b, column)
    p.use_fast = fast_pass_mask(p);
    return HARTREE_OK;
}

extern "C" {

const char* hartree_status_string(int status) {
    switch (status) {
        case HARTREE_OK: return "ok";
        case HARTREE_ERR_INVALID: return "invalid argument";
        case HARTREE_ERR_UNSUPPORTED_SIZE: return "unsupported size";
        case HARTREE_ERR_CUDA: return "CUDA error";
        case HARTREE_ERR_OOM: return "out of device memory";
        case HARTREE_ERR_TIMEOUT: return "device wait timed out";
        case HARTREE_ERR_NOT_CAPTURABLE: return "not capturable";
        default: return "unknown status";
    }
}

const char* hartree_last_error(void) { return g_last_error.c_str(); }

int hartree_plan_create(const hartree_desc* desc, hartree_plan* out) {
    if (!desc || !out) return fail(HARTREE_ERR_INVALID, "plan_create: null argument");
    *out = nullptr;
    const hartree_desc& d = *desc;
    if (d.flags & ~(HARTREE_FLAG_TC_BF16 | HARTREE_FLAG_FUSED_SPLAT))
        return fail(HARTREE_ERR_INVALID, "plan_create: unknown flags");
    if ((d.flags & HARTREE_FLAG_TC_BF16) && d.precision != HARTREE_FP32_TC_SPLIT)
        return fail(HARTREE_ERR_INVALID, "plan_create: HARTREE_FLAG_TC_BF16 needs HARTREE_FP32_TC_SPLIT");
    if (d.precision != HARTREE_FP64 && d.precision != HARTREE_FP32 && d.precision != HARTREE_FP32_TC_SPLIT)
        return fail(HARTREE_ERR_INVALID, "plan_create: unknown precision %d", d.precision);
    for (int i = 0; i < 3; ++i) {
        if (d.n[i] < 2 || d.n[i] > kMaxAxis || !smooth_size(d.n[i]))
            return fail(HARTREE_ERR_UNSUPPORTED_SIZE, "plan_create: N%d = %d is not a 2/3/5/7-smooth size in [2, %d]",
                        i + 1, d.n[i], kMaxAxis);
        if (!(d.cell[i] > 0.0) || !std::isfinite(d.cell[i]))
            return fail(HARTREE_ERR_INVALID, "plan_create: cell[%d] must be positive and finite", i);
    }
    if (d.n[2] % 2 != 0 || d.n[2] < 4)
        return fail(HARTREE_ERR_UNSUPPORTED_SIZE, "plan_create: N3 = %d must be even and >= 4", d.n[2]);
    if (!(d.sigma > 0.0) || !std::isfinite(d.sigma)) return fail(HARTREE_ERR_INVALID, "plan_create: sigma must be > 0");
    if (d.cutoff_sigmas < 0.0 || d.cutoff_sigmas > 16.0 || !std::isfinite(d.cutoff_sigmas))
        return fail(HARTREE_ERR_INVALID, "plan_create: cutoff_sigmas must be in [0, 16]");
    if (d.atoms_per_leaf < 0 || d.max_atoms < 0) return fail(HARTREE_ERR_INVALID, "plan_create: negative count");

    hartree_plan_s* h = new (std::nothrow) hartree_plan_s();
    if (!h) return fail(HARTREE_ERR_OOM, "plan_create: host allocation failed");
    Plan& p = h->p;
    {
        const int st = init_plan_geometry(p, d);
        if (st != HARTREE_OK) {
            delete h;
            return st;
        }
    }
    if (p.prec == HARTREE_FP32_TC_SPLIT && !tc_split_supported(p)) {
        delete h;
        return fail(HARTREE_ERR_UNSUPPORTED_SIZE, "plan_create: HARTREE_FP32_TC_SPLIT needs N2 = 256 (got %d)", p.n[1]);
    }
    p.sigma = d.sigma;
    p.rc = (d.cutoff_sigmas > 0.0 ? d.cutoff_sigmas : (p.prec == HARTREE_FP64 ? 8.0 : 5.0)) * d.sigma;
    p.apl = d.atoms_per_leaf > 0 ? d.atoms_per_leaf : 16;
    p.max_atoms = d.max_atoms > 0 ? d.max_atoms : 65536;
    p.max_leaves = (p.max_atoms + p.apl - 1) / p.apl;
    p.box_max = 0;
    for (int i = 0; i < 3; ++i) {
        const int c = (int)std::floor(2.0 * p.rc / p.h[i]) + 2;
        if (c > p.box_max) p.box_max = c;
    }
    if (p.box_max > kMaxBoxPoints) {
        delete h;
        return fail(HARTREE_ERR_UNSUPPORTED_SIZE, "plan_create: cutoff box spans %d > %d grid points", p.box_max,
                    kMaxBoxPoints);
    }
    p.max_force_slabs = 1216;

    {
        const int T[3] = {TA, TB, TC};
        for (int i = 0; i < 3; ++i) p.tiles[i] = (p.n[i] + T[i] - 1) / T[i];
        p.n_tiles = p.tiles[0] * p.tiles[1] * p.tiles[2];
    }
    const size_t ntot = (size_t)p.n[0] * p.n[1] * p.n[2];
    const size_t cs = 2 * p.real_size;  // complex element
    struct Alloc {
        void** ptr;
        size_t bytes;
    } allocs[] = {
        {&p.W, (size_t)p.n[0] * p.n[1] * p.ldc * cs},
        {&p.R, ntot * p.real_size},
        {&p.tw[0], (size_t)p.n[0] * cs},
        {&p.tw[1], (size_t)p.n[1] * cs},
        {&p.tw[2], (size_t)p.n[2] * cs},
        {&p.twp[0], (size_t)p.n[0] * 2 * cs},
        {&p.twp[1], (size_t)p.n[1] * 2 * cs},
        {&p.twp[2], (size_t)p.n[2] * 2 * cs},
        {&p.gsq[0], (size_t)p.n[0] * cs},
        {&p.gsq[1], (size_t)p.n[1] * cs},
        {&p.gsq[2], (size_t)p.nh * cs},
        {(void**)&p.eh_partials, (size_t)p.n_eh_partials * sizeof(double)},
        {(void**)&p.leaf_box, (size_t)p.max_leaves * 6 * sizeof(int)},
        {&p.atom_prep, (size_t)p.max_atoms * sizeof(AtomPrep<double>)},
        {&p.atom_fac, (size_t)p.max_atoms * 3 * p.box_max * p.real_size},
        {&p.atom_dfac, (size_t)p.max_atoms * 3 * p.box_max * p.real_size},
        {(void**)&p.force_partials, (size_t)(p.max_atoms + p.max_force_slabs) * 4 * sizeof(double)},
        {(void**)&p.force_order, (size_t)p.max_atoms * sizeof(int)},
        {(void**)&p.d_pos, (size_t)p.max_atoms * 3 * sizeof(double)},
        {(void**)&p.d_q, (size_t)p.max_atoms * sizeof(double)},
        {(void**)&p.d_f, (size_t)p.max_atoms * 3 * sizeof(double)},
        {(void**)&p.d_eh, sizeof(double)},
        {(void**)&p.d_err, sizeof(int)},
        {(void**)&p.bin_cursor, (size_t)p.n_tiles * sizeof(int)},
        {(void**)&p.bin_list, (size_t)p.n_tiles * kBinCap * sizeof(int4)},
        {&p.tc_dft, p.prec == HARTREE_FP32_TC_SPLIT ? tc_table_bytes() : 16},
        {&p.bisect, bisect_scratch_bytes(p.max_atoms)},
    };
    for (auto& a : allocs) {
        cudaError_t e = cudaMalloc(a.ptr, a.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_plan(p);
            delete h;
            return fail(e == cudaErrorMemoryAllocation ? HARTREE_ERR_OOM : HARTREE_ERR_CUDA,
                        "plan_create: cudaMalloc(%zu bytes): %s", a.bytes, cudaGetErrorString(e));
        }
        p.bytes += a.bytes;
    }
    int st = p.prec == HARTREE_FP64 ? upload_tables<double>(p) : upload_tables<float>(p);
    if (st == HARTREE_OK) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaMemset(p.d_err, 0, sizeof(int));
        if (e != cudaSuccess) st = cuda_fail(e, "plan_create: device query");
        else prepare_tma(p);
    }
    if (st == HARTREE_OK) {
        cudaError_t e = configure_poisson_kernels(p);
        if (e == cudaSuccess) e = configure_fast_kernels(p);
        if (e == cudaSuccess) e = configure_atom_kernels(p);
        if (e == cudaSuccess) e = configure_tc_kernels(p);
        if (e == cudaSuccess) e = upload_tc_tables(p);
        if (e == cudaSuccess) e = configure_bisect();
        if (e != cudaSuccess) st = cuda_fail(e, "plan_create: kernel attributes");
    }
    if (st != HARTREE_OK) {
        free_plan(p);
        delete h;
        return st;
    }
    *out = h;
    return HARTREE_OK;
}

void hartree_plan_destroy(hartree_plan plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan(plan->p);
    delete plan;
}

unsigned long long hartree_plan_workspace_bytes(hartree_plan plan) { return plan ? plan->p.bytes : 0ULL; }

// The c passes move grid lines as (re, im) pairs of the plan's real type: a grid that a
// solve reads or writes must start on a multiple of twice the element size.
static bool grid_aligned(const Plan& p, const void* g) {
    return g == nullptr || reinterpret_cast<uintptr_t>(g) % (2 * p.real_size) == 0;
}

int hartree_splat(hartree_plan plan, const double* pos, const double* q, int n, void* rho, void* stream) {
    if (!plan || !rho || (n > 0 && (!pos || !q))) return fail(HARTREE_ERR_INVALID, "splat: null argument");
    if (n < 0 || n > plan->p.max_atoms)
        return fail(HARTREE_ERR_INVALID, "splat: n = %d outside [0, max_atoms = %d]", n, plan->p.max_atoms);
    cudaError_t e = launch_splat(plan->p, pos, q, n, rho, (cudaStream_t)stream);
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "splat");
}

int hartree_solve_density(hartree_plan plan, const void* rho, void* vh, double* eh, void* stream) {
    if (!plan || !rho || !vh) return fail(HARTREE_ERR_INVALID, "solve_density: null argument");
    if (!grid_aligned(plan->p, rho) || !grid_aligned(plan->p, vh))
        return fail(HARTREE_ERR_INVALID, "solve_density: grids must be aligned to %d bytes", (int)(2 * plan->p.real_size));
    cudaError_t e = launch_poisson(plan->p, rho, vh, eh, (cudaStream_t)stream);
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "solve_density");
}

int hartree_solve(hartree_plan plan, const double* pos, const double* q, int n, void* rho, void* vh, double* eh,
                  void* stream) {
    if (!plan || !vh || (n > 0 && (!pos || !q))) return fail(HARTREE_ERR_INVALID, "solve: null argument");
    if (n < 0 || n > plan->p.max_atoms)
        return fail(HARTREE_ERR_INVALID, "solve: n = %d outside [0, max_atoms = %d]", n, plan->p.max_atoms);
    if (!grid_aligned(plan->p, rho) || !grid_aligned(plan->p, vh))
        return fail(HARTREE_ERR_INVALID, "solve: grids must be aligned to %d bytes", (int)(2 * plan->p.real_size));
    cudaError_t e;
    if (rho) {
        e = launch_splat(plan->p, pos, q, n, rho, (cudaStream_t)stream);
        if (e == cudaSuccess) e = launch_poisson(plan->p, rho, vh, eh, (cudaStream_t)stream);
    } else {
        e = launch_splat_solve(plan->p, pos, q, n, vh, eh, (cudaStream_t)stream);
    }
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "solve");
}

int hartree_forces(hartree_plan plan, const double* pos, const double* q, int n, const void* vh, double* f,
                   double* phi, void* stream) {
    if (!plan || (n > 0 && (!pos || !q || !f))) return fail(HARTREE_ERR_INVALID, "forces: null argument");
    if (n < 0 || n > plan->p.max_atoms)
        return fail(HARTREE_ERR_INVALID, "forces: n = %d outside [0, max_atoms = %d]", n, plan->p.max_atoms);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    const bool recompute = vh == nullptr;
    if (recompute) {
        e = launch_splat_solve(plan->p, pos, q, n, plan->p.R, nullptr, s);
        vh = plan->p.R;
    }
    // the splat of a recompute already prepared the atoms' boxes and factors
    if (e == cudaSuccess) e = launch_forces(plan->p, pos, q, n, vh, f, phi, s, recompute);
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "forces");
}

int hartree_step(hartree_plan plan, const double* pos, const double* q, int n, void* rho, void* vh, double* eh,
                 double* f, double* phi, void* stream) {
    if (!plan || !vh || (n > 0 && (!pos || !q || !f))) return fail(HARTREE_ERR_INVALID, "step: null argument");
    if (n < 0 || n > plan->p.max_atoms)
        return fail(HARTREE_ERR_INVALID, "step: n = %d outside [0, max_atoms = %d]", n, plan->p.max_atoms);
    if (!grid_aligned(plan->p, rho) || !grid_aligned(plan->p, vh))
        return fail(HARTREE_ERR_INVALID, "step: grids must be aligned to %d bytes", (int)(2 * plan->p.real_size));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (rho) {
        e = launch_splat(plan->p, pos, q, n, rho, s);
        if (e == cudaSuccess) e = launch_poisson(plan->p, rho, vh, eh, s);
    } else {
        e = launch_splat_solve(plan->p, pos, q, n, vh, eh, s);
    }
    if (e == cudaSuccess && n > 0) e = launch_forces(plan->p, pos, q, n, vh, f, phi, s, true);
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "step");
}

int hartree_solve_pass(hartree_plan plan, int pass, const void* rho, void* vh, void* stream) {
    if (!plan) return fail(HARTREE_ERR_INVALID, "solve_pass: null plan");
    if (pass < 0 || pass > 4) return fail(HARTREE_ERR_INVALID, "solve_pass: pass %d not in 0..4", pass);
    if ((pass == 0 && !rho) || (pass == 4 && !vh)) return fail(HARTREE_ERR_INVALID, "solve_pass: null grid");
    if ((pass == 0 && !grid_aligned(plan->p, rho)) || (pass == 4 && !grid_aligned(plan->p, vh)))
        return fail(HARTREE_ERR_INVALID, "solve_pass: grids must be aligned to %d bytes", (int)(2 * plan->p.real_size));
    cudaError_t e = launch_poisson_pass(plan->p, pass, rho, vh, (cudaStream_t)stream);
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "solve_pass");
}

int hartree_splat_pass(hartree_plan plan, const double* pos, const double* q, int n, void* stream) {
    if (!plan || (n > 0 && (!pos || !q))) return fail(HARTREE_ERR_INVALID, "splat_pass: null argument");
    if (n < 0 || n > plan->p.max_atoms)
        return fail(HARTREE_ERR_INVALID, "splat_pass: n = %d outside [0, max_atoms = %d]", n, plan->p.max_atoms);
    if (!splat_fused_available(plan->p))
        return fail(HARTREE_ERR_UNSUPPORTED_SIZE, "splat_pass: the plan has no splat fused into pass 0");
    cudaError_t e = launch_splat_r2c(plan->p, pos, q, n, (cudaStream_t)stream);
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "splat_pass");
}

int hartree_plan_fused_splat(hartree_plan plan) { return plan && splat_fused_available(plan->p) ? 1 : 0; }

int hartree_atoms_reorder_device(hartree_plan plan, const double* pos, const double* w, int n, int n_leaves,
                                 int* perm, int* leaf_start, void* stream) {
    if (!plan || !leaf_start || (n > 0 && (!pos || !perm)))
        return fail(HARTREE_ERR_INVALID, "atoms_reorder_device: null argument");
    if (n < 0 || n > plan->p.max_atoms || n_leaves < 1 || n_leaves > plan->p.max_atoms)
        return fail(HARTREE_ERR_INVALID, "atoms_reorder_device: n = %d, n_leaves = %d outside [0 / 1, max_atoms = %d]",
                    n, n_leaves, plan->p.max_atoms);
    cudaError_t e = launch_bisect(plan->p, pos, w, n, n_leaves, perm, leaf_start, (cudaStream_t)stream);
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "atoms_reorder_device");
}

unsigned long long hartree_plan_launch_count(hartree_plan plan) { return plan ? plan->p.launches : 0ULL; }

int hartree_plan_device_status(hartree_plan plan) {
    if (!plan) return fail(HARTREE_ERR_INVALID, "device_status: null plan");
    int err = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&err, plan->p.d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && err) e = cudaMemset(plan->p.d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "device_status");
    if (err) return fail(HARTREE_ERR_TIMEOUT, "a bounded device wait gave up (error word %d)", err);
    return HARTREE_OK;
}

int hartree_plan_set_variants(hartree_plan plan, const int* choice) {
    if (!plan || !choice) return fail(HARTREE_ERR_INVALID, "set_variants: null argument");
    for (int k = 0; k < 3; ++k)
        if (choice[k] < 0 || choice[k] >= fast_variants(plan->p, k))
            return fail(HARTREE_ERR_INVALID, "set_variants: pass kind %d has %d variants, got %d", k,
                        fast_variants(plan->p, k), choice[k]);
    for (int k = 0; k < 3; ++k) plan->p.var[k] = choice[k];
    return HARTREE_OK;
}

// Time every kernel variant of each pass kind on the plan's own workspace and keep the fastest.
int hartree_plan_autotune(hartree_plan plan, void* stream, int* choice) {
    if (!plan) return fail(HARTREE_ERR_INVALID, "autotune: null plan");
    Plan& p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(HARTREE_ERR_NOT_CAPTURABLE, "autotune times kernels; it cannot be captured");
    const size_t ntot = (size_t)p.n[0] * p.n[1] * p.n[2];
    e = cudaMemsetAsync(p.R, 0, ntot * p.real_size, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.W, 0, (size_t)p.n[0] * p.n[1] * p.ldc * 2 * p.real_size, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // time `reps` launches of pass `q` (twice: q and q2 when q2 >= 0) under the current variants
    auto time_passes = [&](int q, int q2, float* ms) {
        for (int rep = 0; rep < 3; ++rep) {  // warm-up
            launch_poisson_pass(p, q, p.R, p.R, s);
            if (q2 >= 0) launch_poisson_pass(p, q2, p.R, p.R, s);
        }
        cudaError_t r = cudaEventRecord(e0, s);
        for (int rep = 0; rep < 10; ++rep) {
            launch_poisson_pass(p, q, p.R, p.R, s);
            if (q2 >= 0) launch_poisson_pass(p, q2, p.R, p.R, s);
        }
        if (r == cudaSuccess) r = cudaEventRecord(e1, s);
        if (r == cudaSuccess) r = cudaEventSynchronize(e1);
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
        return r;
    };
    // c and b passes: each of the pair (r2c / c2r, forward / inverse) takes its own fastest variant
    static const int pair_passes[2][2] = {{0, 4}, {1, 3}};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (k == 1 && p.prec == HARTREE_FP32_TC_SPLIT) continue;  // b passes run on the tensor cores
        const int V = single_variants(p, k);
        if (V <= 1) continue;
        int best_v[2] = {0, 0};
        for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
            float best = 1e30f;
            for (int v = 0; v < V && e == cudaSuccess; ++v) {
                p.var[k] = v;
                float ms = 0.f;
                e = time_passes(pair_passes[k][q], -1, &ms);
                if (e == cudaSuccess && ms < best) {
                    best = ms;
                    best_v[q] = v;
                }
            }
        }
        p.var[k] = pair_index(V, best_v[0], best_v[1]);
    }
    // the a pass
    if (e == cudaSuccess && fast_variants(p, 2) > 1) {
        float best = 1e30f;
        int best_v = 0;
        for (int v = 0; v < fast_variants(p, 2) && e == cudaSuccess; ++v) {
            p.var[2] = v;
            float ms = 0.f;
            e = time_passes(2, -1, &ms);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                best_v = v;
            }
        }
        p.var[2] = best_v;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (choice)
        for (int k = 0; k < 3; ++k) choice[k] = p.var[k];
    return HARTREE_OK;
}

// The device work of hartree_step_host on the staged atoms: splat, solve, E_H, forces.
static cudaError_t host_step_work(Plan& p, int n, bool forces, cudaStream_t s) {
    cudaError_t e = launch_splat_solve(p, p.d_pos, p.d_q, n, p.R, p.d_eh, s);
    if (e == cudaSuccess && forces) e = launch_forces(p, p.d_pos, p.d_q, n, p.R, p.d_f, nullptr, s, true);
    return e;
}

// Capture host_step_work into p.host_graph (left null if the capture fails: the caller then
// launches directly).  The plan's launch counter is advanced by the replays, not by the capture.
static void capture_host_step(Plan& p, int n, bool forces, cudaStream_t s, const int* key) {
    const unsigned long long l0 = p.launches;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const cudaError_t e = host_step_work(p, n, forces, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    const unsigned long long l1 = p.launches;
    p.launches = l0;
    if (e == cudaSuccess && ec == cudaSuccess && g && cudaGraphInstantiate(&p.host_graph, g, 0) == cudaSuccess) {
        p.host_graph_launches = l1 - l0;
        for (int i = 0; i < 5; ++i) p.host_key[i] = key[i];
    } else {
        p.host_graph = nullptr;
        cudaGetLastError();
    }
    if (g) cudaGraphDestroy(g);
}

int hartree_step_host(hartree_plan plan, const double* pos, const double* q, int n, double* eh, double* f,
                      void* stream) {
    if (!plan || !eh || (n > 0 && (!pos || !q))) return fail(HARTREE_ERR_INVALID, "step_host: null argument");
    Plan& p = plan->p;
    if (n < 0 || n > p.max_atoms)
        return fail(HARTREE_ERR_INVALID, "step_host: n = %d outside [0, max_atoms = %d]", n, p.max_atoms);
    for (int i = 0; i < 3 * n; ++i)
        if (!finite_pos(pos[i])) return fail(HARTREE_ERR_INVALID, "step_host: position %d is not finite", i / 3);
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "step_host");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(HARTREE_ERR_NOT_CAPTURABLE, "step_host waits for the stream; it cannot be captured");
    // the work runs on the plan's own stream (a capture needs a stream other than the legacy
    // default one), after the caller's earlier work on `stream`; the call waits for it
    if (!p.host_stream) {
        e = cudaStreamCreateWithFlags(&p.host_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.host_event, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "step_host");
    }
    const cudaStream_t hs = p.host_stream;
    e = cudaEventRecord(p.host_event, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, p.host_event, 0);
    if (e == cudaSuccess && n > 0) {
        e = cudaMemcpyAsync(p.d_pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, hs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p.d_q, q, sizeof(double) * n, cudaMemcpyHostToDevice, hs);
    }
    const bool forces = f && n > 0;
    const int key[5] = {n, p.var[0], p.var[1], p.var[2], forces ? 1 : 0};
    if (e == cudaSuccess && (!p.host_graph || !std::equal(key, key + 5, p.host_key))) {
        if (p.host_graph) cudaGraphExecDestroy(p.host_graph);
        p.host_graph = nullptr;
        capture_host_step(p, n, forces, hs, key);
    }
    if (e == cudaSuccess) {
        if (p.host_graph) {
            e = cudaGraphLaunch(p.host_graph, hs);
            p.launches += p.host_graph_launches;
        } else {
            e = host_step_work(p, n, forces, hs);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(eh, p.d_eh, sizeof(double), cudaMemcpyDeviceToHost, hs);
    if (e == cudaSuccess && forces) e = cudaMemcpyAsync(f, p.d_f, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, hs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hs);
    return e == cudaSuccess ? HARTREE_OK : cuda_fail(e, "step_host");
}

}  // extern "C"
