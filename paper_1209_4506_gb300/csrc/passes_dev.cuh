// passes_dev.cuh -- the generic (runtime-radix) Poisson passes as per-tile
// device functions, shared by the one-tile-per-CTA kernels of poisson.cu and
// the batched persistent kernel of batch.cu.  CG = true makes every load of
// data produced in the same launch bypass L1 (not coherent across SMs).
#pragma once

#include "internal.cuh"

namespace hartree {

// ---------------------------------------------------------------- pass 1: c r2c
template <typename T, bool CG>
__device__ void c_r2c_tile(const T* __restrict__ rho, const PoissonArgs<T>& a, int tile, unsigned char* smem_raw) {
    const int L = a.c_lines, ld = L + 1, M = a.M;
    const uint32_t mM = fdiv_magic((uint32_t)M), mM1 = fdiv_magic((uint32_t)(M + 1));
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* B = A + (size_t)(M + 1) * ld;
    const long long nlines = (long long)a.n1 * a.n2;
    const long long line0 = (long long)tile * L;
    const int nl = (int)min((long long)L, nlines - line0);
    // z[n] = rho[2n] + i rho[2n+1]: coalesced along the line, transposed into [n][line]
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = (int)fdiv((uint32_t)e, mM), n = e - l * M;
        const cpx<T>* src = reinterpret_cast<const cpx<T>*>(rho + (line0 + l) * a.n3);
        A[n * ld + l] = gload<CG>(src + n);
    }
    __syncthreads();
    cpx<T>* Z = run_fft_to_smem<T, false>(a.rpc, SmemTile<T>{A, ld}, B, A, ld, nl, a.twc, 2);
    // X[k] = E[k] + w^k O[k],  E = (Z[k] + conj Z[M-k]) / 2,  O = (Z[k] - conj Z[M-k]) / 2i,  k = 0..M
    const T half = T(0.5);
    for (int e = threadIdx.x; e < nl * (M + 1); e += blockDim.x) {
        const int l = (int)fdiv((uint32_t)e, mM1), k = e - l * (M + 1);
        const cpx<T> z1 = Z[(k == M ? 0 : k) * ld + l];
        const cpx<T> z2 = conjg(Z[(k == 0 ? 0 : M - k) * ld + l]);
        const cpx<T> E = scale(z1 + z2, half);
        const cpx<T> d = z1 - z2;
        const cpx<T> O = mk(d.im * half, -d.re * half);
        a.W[(line0 + l) * a.ldc + k] = E + a.twc[k] * O;
    }
}

// ---------------------------------------------------------------- passes 2 / 4: b
template <typename T, bool INV, bool CG>
__device__ void b_tile(const PoissonArgs<T>& a, int tile, unsigned char* smem_raw) {
    const int CB = a.b_cols;
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* B = A + (size_t)a.n2 * CB;
    const int ia = tile / a.b_chunks;
    const int c0 = (tile - ia * a.b_chunks) * CB;
    const int nc = min(CB, a.nh - c0);
    const uint32_t mnc = fdiv_magic((uint32_t)nc);
    GlobalTile<T, CG> g{a.W + (long long)ia * a.n2 * a.ldc + c0, a.ldc};
    if (a.rpb.nst >= 2) {
        run_fft<T, INV>(a.rpb, g, g, A, B, CB, nc, a.twb, 1);
    } else {
        // one stage reads and writes different rows: go through shared memory
        cpx<T>* F = run_fft_to_smem<T, INV>(a.rpb, g, A, B, CB, nc, a.twb, 1);
        for (int e = threadIdx.x; e < a.n2 * nc; e += blockDim.x) {
            const int n = (int)fdiv((uint32_t)e, mnc), col = e - n * nc;
            g.st_(col, n, F[n * CB + col]);
        }
    }
}

// ---------------------------------------------------------------- pass 3: a + Green + E_H + a^-1
// Writes this tile's E_H partial sum to a.eh_partials[part_index].
template <typename T, bool CG>
__device__ void a_green_tile(const PoissonArgs<T>& a, int tile, int part_index, unsigned char* smem_raw,
                             double* red) {
    const int CA = a.a_cols;
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* B = A + (size_t)a.n1 * CA;
    const int ib = tile / a.a_chunks;
    const int c0 = (tile - ib * a.a_chunks) * CA;
    const int nc = min(CA, a.nh - c0);
    const uint32_t mnc = fdiv_magic((uint32_t)nc);
    GlobalTile<T, CG> g{a.W + (long long)ib * a.ldc + c0, (long long)a.n2 * a.ldc};
    cpx<T>* F = run_fft_to_smem<T, false>(a.rpa, g, A, B, CA, nc, a.twa, 1);
    // F[k1][col] now holds rho~(k1, ib, c0 + col).
    const cpx<T> gb = a.gsqb[ib];
    T sum = T(0), comp = T(0);  // compensated per-thread partial of sum m |rho~|^2 / G^2
    for (int e = threadIdx.x; e < a.n1 * nc; e += blockDim.x) {
        const int k1 = (int)fdiv((uint32_t)e, mnc), col = e - k1 * nc;
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
    if (threadIdx.x == 0) a.eh_partials[part_index] = bs;
    __syncthreads();
    cpx<T>* other = (F == A) ? B : A;
    run_fft<T, true>(a.rpa, SmemTile<T>{F, CA}, g, other, F, CA, nc, a.twa, 1);
}

// ---------------------------------------------------------------- pass 5: c c2r
template <typename T, bool CG>
__device__ void c_c2r_tile(T* __restrict__ out, const PoissonArgs<T>& a, int tile, unsigned char* smem_raw) {
    const int L = a.c_lines, ld = L + 1, M = a.M;
    const uint32_t mM = fdiv_magic((uint32_t)M), mM1 = fdiv_magic((uint32_t)(M + 1));
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* B = A + (size_t)(M + 1) * ld;
    const long long nlines = (long long)a.n1 * a.n2;
    const long long line0 = (long long)tile * L;
    const int nl = (int)min((long long)L, nlines - line0);
    for (int e = threadIdx.x; e < nl * (M + 1); e += blockDim.x) {
        const int l = (int)fdiv((uint32_t)e, mM1), k = e - l * (M + 1);
        A[k * ld + l] = gload<CG>(a.W + (line0 + l) * a.ldc + k);
    }
    __syncthreads();
    // Z[k] = (X[k] + conj X[M-k]) + i w^-k (X[k] - conj X[M-k]),  k < M
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = (int)fdiv((uint32_t)e, mM), k = e - l * M;
        const cpx<T> x1 = A[k * ld + l];
        const cpx<T> x2 = conjg(A[(M - k) * ld + l]);
        const cpx<T> Ep = x1 + x2;
        const cpx<T> Op = (x1 - x2) * conjg(a.twc[k]);
        B[k * ld + l] = mk(Ep.re - Op.im, Ep.im + Op.re);
    }
    __syncthreads();
    cpx<T>* z = run_fft_to_smem<T, true>(a.rpc, SmemTile<T>{B, ld}, A, B, ld, nl, a.twc, 2);
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = (int)fdiv((uint32_t)e, mM), n = e - l * M;
        reinterpret_cast<cpx<T>*>(out + (line0 + l) * a.n3)[n] = z[n * ld + l];
    }
}

template <typename T>
inline PoissonArgs<T> make_args(const Plan& p) {
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

}  // namespace hartree
