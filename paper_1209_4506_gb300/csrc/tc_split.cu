// tc_split.cu -- the b passes (forward and inverse FFT along b, N2 = 256) of
// HARTREE_FP32_TC_SPLIT plans on the 5th-generation tensor cores.
//
// 256 = 16 x 16 (Cooley-Tukey, Sec. 3.2.4's one-dimensional transforms along
// b): with n = 16 n1 + n2 and k = k1 + 16 k2,
//   Y[n2][k1]     = sum_n1 x[16 n1 + n2] w16^(n1 k1)         stage A (16-point DFTs)
//   Y'[n2][k1]    = Y[n2][k1] w256^(n2 k1)                    twiddle (FP32, CUDA cores)
//   X[k1 + 16 k2] = sum_n2 Y'[n2][k1] w16^(n2 k2)             stage B (16-point DFTs)
// (w_N = exp(-2 pi i / N); the inverse uses conjugates and no scaling).  Each
// 16-point complex DFT of a batch of rows is the real product
//   [Re x | Im x] (rows x 32) . M (32 x 32),
// M holding cos and +-sin of 2 pi n k / 16.  FP32 values are split into
// 16-bit parts and the MMA accumulates, in FP32, the products of the parts
// whose order is low enough for an FP32 result:
//   FP16 (the default, p = 11 significant bits per part): x = x_h + x_l,
//     M = M_h + M_l (the table split in FP64 on the host), and
//     x_h M_h + x_h M_l + x_l M_h as one K = 96 product
//     [x_h | x_h | x_l] . [M_h ; M_l ; M_h]; the dropped x_l M_l term and the
//     split residual are about 2^-22 relative per product.  FP16 needs range:
//     each row of 16 complex inputs is scaled by a power of two that puts its
//     largest magnitude in [2^14, 2^15), which is exact, and the same thread
//     divides its output row by it.
//   BF16 (p = 8, the FP32 exponent range, no scaling): two parts would leave
//     2^-16 per product, and four such stages per solve exceed the 1e-5 bar on
//     V_H, so x = x0 + x1 + x2 and M = M0 + M1 + M2 (24 bits each) and the six
//     products of order <= 2, x0 M0 + x1 M0 + x0 M1 + x2 M0 + x1 M1 + x0 M2, form
//     one K = 192 product [x0 | x1 | x0 | x2 | x1 | x0] . [M0 ; M0 ; M1 ; M0 ; M1 ; M2];
//     the dropped terms are about 2^-24 relative.
//
// One CTA of 128 threads transforms 8 complex columns (128 rows of 16-point
// DFTs per stage, one M = 128 MMA tile of N = 32, accumulator in 32 TMEM
// columns).  Thread r builds row r of the A operand in shared memory; one
// thread issues the six K = 16 MMAs and commits them to an mbarrier; each
// warp reads its 32 TMEM lanes back.  Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace hartree {

namespace {

constexpr int kTcCols = 8;                  // complex columns per CTA
constexpr int kTcThreads = 128;             // one thread per row of the MMA tile
constexpr int kTcKMax = 192;                // the longest contraction (BF16: six segments of 32)
constexpr int kX2Stride = 274;              // c stride of the transposed stage-A output (conflict-free)
constexpr int kX2Row = 17;                  // k1 stride
constexpr uint32_t kTcLbo = 128;            // core matrices along K

// K of the split product: 32 values (Re, Im of 16 inputs) per segment, 3 segments (FP16) or 6 (BF16).
template <bool F16>
__host__ __device__ constexpr int tc_k() {
    return F16 ? 96 : 192;
}

struct TcArgs {
    cpx<float>* W;
    int n1, n2, nh, ldc, chunks;
    const cpx<float>* tw;   // exp(-2 pi i k / 256), k < 256
    const uint16_t* dft;    // [2][32 x 96] operand B (forward, inverse) in the K-major layout
    int* err;
};

// Shared memory of one CTA for a contraction of length K (sized per operand format, so the
// FP16 split keeps its occupancy).
template <int K>
struct TcSmem {
    cpx<float> X[256 * kTcCols];         // input columns: X[n][c]
    cpx<float> X2[kTcCols * kX2Stride];  // stage-A output: X2[c][k1][n2]
    uint16_t A[kTcThreads * K];
    uint16_t B[32 * K];
    uint64_t bar;
    uint32_t tbase;
};

// The 16-bit operand format: FP16 (F16 = true) or BF16, round to nearest.
template <bool F16>
__device__ __forceinline__ uint16_t to16(float x) {
    if constexpr (F16)
        return __half_as_ushort(__float2half_rn(x));
    else
        return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
template <bool F16>
__device__ __forceinline__ float from16(uint16_t x) {
    if constexpr (F16)
        return __half2float(__ushort_as_half(x));
    else
        return __bfloat162float(__ushort_as_bfloat16(x));
}

// Row r of the A operand from 16 complex values, segments of 32 (re(16), im(16)): FP16 [h | h | l],
// BF16 [x0 | x1 | x0 | x2 | x1 | x0].  FP16 rows are scaled by a power of two first; returns the
// factor that undoes it.
template <bool F16>
__device__ __forceinline__ float build_row(uint16_t* A, int r, float* re, float* im) {
    constexpr int K = tc_k<F16>();
    float undo = 1.f;
    if constexpr (F16) {
        float m = 0.f;
#pragma unroll
        for (int n = 0; n < 16; ++n) m = fmaxf(m, fmaxf(fabsf(re[n]), fabsf(im[n])));
        if (m > 0.f && m < 3.0e38f) {
            const int e = ilogbf(m);  // m in [2^e, 2^(e+1))
            const float sc = ldexpf(1.f, 14 - e);
            undo = ldexpf(1.f, e - 14);
#pragma unroll
            for (int n = 0; n < 16; ++n) re[n] *= sc, im[n] *= sc;
        }
    }
    // parts: x = p[0] + p[1] (+ p[2]), each rounded from the remainder of the previous ones
    constexpr int NP = F16 ? 2 : 3;
    uint16_t part[NP][32];
#pragma unroll
    for (int n = 0; n < 32; ++n) {
        float rem = n < 16 ? re[n] : im[n - 16];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            part[q][n] = to16<F16>(rem);
            rem -= from16<F16>(part[q][n]);
        }
    }
    // segment order: FP16 h, h, l; BF16 x0, x1, x0, x2, x1, x0
    constexpr int seg16[3] = {0, 0, 1};
    constexpr int segbf[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
    for (int j = 0; j < K / 8; ++j) {  // 16-byte chunks of 8 K values
        const int sg = F16 ? seg16[j / 4] : segbf[j / 4];
        const uint16_t* src = part[sg] + (j & 3) * 8;
        uint4 v;
        v.x = (uint32_t)src[0] | ((uint32_t)src[1] << 16);
        v.y = (uint32_t)src[2] | ((uint32_t)src[3] << 16);
        v.z = (uint32_t)src[4] | ((uint32_t)src[5] << 16);
        v.w = (uint32_t)src[6] | ((uint32_t)src[7] << 16);
        *reinterpret_cast<uint4*>(A + kmajor_index(r, 8 * j, K)) = v;
    }
    return undo;
}

// The K = 16 MMAs of the 128 x 32 x K product into TMEM (6 for FP16, 12 for BF16), committed to `bar`.
template <bool F16>
__device__ __forceinline__ void issue_dft(TcSmem<tc_k<F16>()>& s, uint32_t tmem) {
    constexpr int K = tc_k<F16>();
    constexpr uint32_t sbo = K / 8 * 128;  // core matrices along rows
    tc_fence_after();
    const uint32_t idesc = F16 ? idesc_f16_f32(128, 32) : idesc_bf16_f32(128, 32);
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks)
        umma_f16(tmem, smem_desc(s.A + kmajor_index(0, 16 * ks, K), kTcLbo, sbo),
                  smem_desc(s.B + kmajor_index(0, 16 * ks, K), kTcLbo, sbo), idesc, ks > 0 ? 1u : 0u);
    umma_commit(&s.bar);
}

template <bool INV, bool F16>
__global__ void __launch_bounds__(kTcThreads) k_col_tc(TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    TcSmem<tc_k<F16>()>& s =
        *reinterpret_cast<TcSmem<tc_k<F16>()>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ia = blockIdx.x / a.chunks;
    const int c0 = (blockIdx.x - ia * a.chunks) * kTcCols;
    const int nc = min(kTcCols, a.nh - c0);
    cpx<float>* col = a.W + (long long)ia * a.n2 * a.ldc + c0;

    if (warp == 0) {
        tmem_alloc(&s.tbase, 32);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&s.bar, 1);
        fence_barrier_init();
    }
    for (int e = tid; e < 256 * kTcCols; e += kTcThreads) {
        const int n = e / kTcCols, c = e - n * kTcCols;
        s.X[e] = c < nc ? col[(long long)n * a.ldc + c] : mk(0.f, 0.f);
    }
    {
        // the host uploads the table of the plan's operand format: [forward, inverse], 32 x K each
        constexpr int K = tc_k<F16>();
        const uint4* src = reinterpret_cast<const uint4*>(a.dft + (INV ? 32 * K : 0));
        uint4* dst = reinterpret_cast<uint4*>(s.B);
        for (int e = tid; e < 32 * K / 8; e += kTcThreads) dst[e] = src[e];
    }
    __syncthreads();

    // stage A: row r = (n2, c) = (r >> 3, r & 7), K over n1
    float undo;
    {
        const int c = tid & 7, n2 = tid >> 3;
        float re[16], im[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            const cpx<float> x = s.X[(16 * n1 + n2) * kTcCols + c];
            re[n1] = x.re;
            im[n1] = x.im;
        }
        undo = build_row<F16>(s.A, tid, re, im);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    const uint32_t tmem = s.tbase;
    const uint32_t tlane = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    if (tid == 0) issue_dft<F16>(s, tmem);
    bool ok = mbar_wait(&s.bar, 0, a.err);
    tc_fence_after();
    if (ok) {
        float v[32];
        tmem_ld32(tlane, v);
        const int r = 32 * warp + lane;
        const int c = r & 7, n2 = r >> 3;
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            cpx<float> t = a.tw[(n2 * k1) & 255];
            if (INV) t.im = -t.im;
            const cpx<float> y = mk(v[k1] * undo, v[16 + k1] * undo);
            s.X2[c * kX2Stride + k1 * kX2Row + n2] = mk(y.re * t.re - y.im * t.im, y.re * t.im + y.im * t.re);
        }
    }
    tc_fence_before();
    __syncthreads();

    // stage B: row r = (k1, c) = (r >> 3, r & 7), K over n2
    if (ok) {
        const int c = tid & 7, k1 = tid >> 3;
        float re[16], im[16];
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) {
            const cpx<float> y = s.X2[c * kX2Stride + k1 * kX2Row + n2];
            re[n2] = y.re;
            im[n2] = y.im;
        }
        undo = build_row<F16>(s.A, tid, re, im);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (ok && tid == 0) issue_dft<F16>(s, tmem);
    if (ok) ok = mbar_wait(&s.bar, 1, a.err);
    tc_fence_after();
    if (ok) {
        float v[32];
        tmem_ld32(tlane, v);
        const int r = 32 * warp + lane;
        const int c = r & 7, k1 = r >> 3;
        if (c < nc) {
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2)
                col[(long long)(k1 + 16 * k2) * a.ldc + c] = mk(v[k2] * undo, v[16 + k2] * undo);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

}  // namespace

bool tc_split_supported(const Plan& p) { return p.n[1] == 256; }

size_t tc_smem(bool f16) {
    return (f16 ? sizeof(TcSmem<tc_k<true>()>) : sizeof(TcSmem<tc_k<false>()>)) + 1024;
}

cudaError_t configure_tc_kernels(const Plan& p) {
    if (p.prec != HARTREE_FP32_TC_SPLIT) return cudaSuccess;
    const int s16 = (int)tc_smem(true), sbf = (int)tc_smem(false);
    cudaError_t e = cudaFuncSetAttribute(k_col_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s16);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s16);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_col_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sbf);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sbf);
    return e;
}

size_t tc_table_bytes() { return 2 * 32 * kTcKMax * sizeof(uint16_t); }

// Operand B of the 16-point DFT for both directions, split into 16-bit parts in
// FP64, laid out K-major: row j < 16 is Re X_j, row 16 + j is Im X_j; within a
// segment of 32 columns, column q < 16 multiplies Re x_q, 16 + q multiplies Im x_q.
// Segments: FP16 M_h, M_l, M_h; BF16 M0, M0, M1, M0, M1, M2 (matching the A rows).
static uint16_t host16(double x, bool f16) {
    return f16 ? __half_as_ushort(__float2half_rn((float)x)) : __bfloat16_as_ushort(__float2bfloat16_rn((float)x));
}
static double host_back(uint16_t x, bool f16) {
    return f16 ? (double)__half2float(__ushort_as_half(x)) : (double)__bfloat162float(__ushort_as_bfloat16(x));
}

static void tc_dft_tables(uint16_t* out /* [2][32 * K] */, bool f16) {
    const double pi = 3.14159265358979323846;
    const int K = f16 ? tc_k<true>() : tc_k<false>();
    static const int seg16[3] = {0, 1, 0}, segbf[6] = {0, 0, 1, 0, 1, 2};
    for (int dir = 0; dir < 2; ++dir) {
        const double sg = dir == 0 ? -1.0 : 1.0;  // exp(sg 2 pi i n k / 16)
        uint16_t* B = out + dir * 32 * K;
        for (int j = 0; j < 32; ++j)
            for (int q = 0; q < 32; ++q) {
                const int k = j & 15, n = q & 15;
                const double th = 2.0 * pi * ((n * k) & 15) / 16.0;
                const double c = std::cos(th), sn = sg * std::sin(th);  // w = c + i sn
                // Re X = sum Re x c - Im x sn;  Im X = sum Re x sn + Im x c
                double m;
                if (j < 16)
                    m = q < 16 ? c : -sn;
                else
                    m = q < 16 ? sn : c;
                uint16_t part[3];
                double rem = m;
                for (int pq = 0; pq < 3; ++pq) {
                    part[pq] = host16(rem, f16);
                    rem -= host_back(part[pq], f16);
                }
                for (int sgi = 0; sgi < K / 32; ++sgi)
                    B[kmajor_index(j, 32 * sgi + q, K)] = part[f16 ? seg16[sgi] : segbf[sgi]];
            }
    }
}

cudaError_t upload_tc_tables(const Plan& p) {
    if (p.prec != HARTREE_FP32_TC_SPLIT) return cudaSuccess;
    std::vector<uint16_t> t(2 * 32 * kTcKMax);
    tc_dft_tables(t.data(), !(p.desc.flags & HARTREE_FLAG_TC_BF16));
    return cudaMemcpy(p.tc_dft, t.data(), tc_table_bytes(), cudaMemcpyHostToDevice);
}

long long launch_tc_pass(const Plan& p, int pass, cudaStream_t s) {
    TcArgs a;
    a.W = static_cast<cpx<float>*>(p.W);
    a.n1 = p.n[0];
    a.n2 = p.n[1];
    a.nh = p.nh;
    a.ldc = p.ldc;
    a.chunks = (p.nh + kTcCols - 1) / kTcCols;
    a.tw = static_cast<const cpx<float>*>(p.tw[1]);
    a.dft = static_cast<const uint16_t*>(p.tc_dft);
    a.err = p.d_err;
    const unsigned grid = (unsigned)(p.n[0] * a.chunks);
    const bool f16 = !(p.desc.flags & HARTREE_FLAG_TC_BF16);
    const size_t sm = tc_smem(f16);
    if (pass == 1) {
        if (f16)
            k_col_tc<false, true><<<grid, kTcThreads, sm, s>>>(a);
        else
            k_col_tc<false, false><<<grid, kTcThreads, sm, s>>>(a);
    } else {
        if (f16)
            k_col_tc<true, true><<<grid, kTcThreads, sm, s>>>(a);
        else
            k_col_tc<true, false><<<grid, kTcThreads, sm, s>>>(a);
    }
    return grid;
}

}  // namespace hartree
