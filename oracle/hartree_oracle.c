/*
 * hartree_oracle.c -- plain, slow, FP64 CPU oracle for the grid-side Hartree
 * step of Duy & Ozaki, "A three-dimensional domain decomposition method for
 * large-scale DFT electronic structure calculations" (arXiv:1209.4506).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes (all FP64):
 *   splat     rho(r) = sum_i q_i (pi s^2)^(-3/2) sum_T exp(-|r - R_i - T|^2 / s^2),
 *             images T of the periodic cell, truncated at |r - R_i - T| < rc.
 *             (Gaussian atom charges stand in for the density of Eq. charge-density;
 *             the Hartree potential of Eq. Hartree-potential is solved for it.)
 *   fft       naive recursive mixed-radix decimation-in-time DFT (any prime
 *             factor p done as an O(p^2) small DFT), applied along c, then b,
 *             then a -- the transform order of Sec. 3.2.4 (abc -> cab -> cba).
 *   poisson   Sec. 2.1: the Hartree potential is obtained by solving the
 *             Poisson equation with FFT: V~(G) = 4 pi / |G|^2 rho~(G), G = 0
 *             dropped (uniform neutralising background), inverse transform
 *             back along a, b, c (cba -> cab -> abc), scaled by 1/N.
 *   energy    E_H = 1/2 dV sum_r rho_r V_r (the Hartree term of Eq.
 *             total-energy), and the same number from the spectrum,
 *             Omega/(2 N^2) sum_k g_k |rho~_k|^2.
 *   forces    F_i = -dE_H/dR_i = -dV sum_r V_r d rho_i(r)/dR_i  (exact gradient
 *             of the discrete energy), plus phi_i = dE_H/dq_i.
 *   bisect    Sec. 3.1.2-3.1.5: modified recursive bisection of the atoms with
 *             the inertia-tensor principal axis (Eqs. center-of-mass,
 *             eq-projection-ti, eq-function-F, eq-inertia-tensor).
 *   dft_brute O(N^2) 3D DFT straight from its definition, for tiny grids.
 *
 * Grid convention: point (i, j, k) sits at (i h1, j h2, k h3), h_d = L_d / N_d,
 * arrays are C order [N1][N2][N3] with c fastest (structure B "abc").
 *
 * Parity: every routine here is pinned by tests (closed forms, lattice sums,
 * brute force, invariants); see the test-suite.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double re, im;
} cplx;

static const double TWO_PI = 6.283185307179586476925286766559;
static const double PI = 3.141592653589793238462643383279;

/* ------------------------------------------------------------ 1D FFT */

static int smallest_prime_factor(int n) {
    for (int p = 2; (long)p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* roots[e] = exp(sign * 2 pi i e / n), e in [0, n); integer reduction is exact. */
static cplx* make_roots(int n, int sign) {
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    for (int e = 0; e < n; ++e) {
        double a = TWO_PI * (double)e / (double)n;
        w[e].re = cos(a);
        w[e].im = sign * sin(a);
    }
    return w;
}

/*
 * out[k] = sum_{j<n} x[j*stride] w^(j k), w = exp(sign 2 pi i / n), by
 * decimation in time: with p the smallest prime factor of n and m = n/p,
 * the p interleaved subsequences x[r + p j] are transformed (Y_r, length m),
 * then X[k + m s] = sum_r w_n^(r (k + m s)) Y_r[k].
 * roots: table of exp(sign 2 pi i e / n_root) with n_root a multiple of n.
 */
static void fft_rec(int n, const cplx* x, long stride, cplx* out, const cplx* roots, int n_root) {
    if (n == 1) {
        out[0] = x[0];
        return;
    }
    int p = smallest_prime_factor(n);
    int m = n / p;
    for (int r = 0; r < p; ++r) fft_rec(m, x + (long)r * stride, stride * p, out + (long)r * m, roots, n_root);
    int step = n_root / n; /* w_n^e = roots[e * step] */
    cplx tbuf[64];
    cplx* t = p <= 64 ? tbuf : (cplx*)malloc(sizeof(cplx) * (size_t)p);
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) t[r] = out[(long)r * m + k];
        for (int s = 0; s < p; ++s) {
            long idx = k + (long)m * s;
            double are = 0.0, aim = 0.0;
            for (int r = 0; r < p; ++r) {
                long e = ((long)r * idx) % n;
                cplx w = roots[e * step];
                are += t[r].re * w.re - t[r].im * w.im;
                aim += t[r].re * w.im + t[r].im * w.re;
            }
            out[idx].re = are;
            out[idx].im = aim;
        }
    }
    if (t != tbuf) free(t);
}

/* Public 1D transform (unnormalised), for tests. */
void oracle_fft1d(int n, const double* in, double* out, int sign) {
    cplx* w = make_roots(n, sign);
    fft_rec(n, (const cplx*)in, 1, (cplx*)out, w, n);
    free(w);
}

/* ------------------------------------------------------------ 3D FFT */

typedef struct {
    cplx* data;
    int n[3];
    int axis;
    const cplx* roots;
    long line_begin, line_end;
} axis_job;

/* Transform every line along `axis` of the C-order array data[n0][n1][n2]. */
static void* axis_worker(void* arg) {
    axis_job* jb = (axis_job*)arg;
    int len = jb->n[jb->axis];
    long stride = 1;
    for (int d = jb->axis + 1; d < 3; ++d) stride *= jb->n[d];
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)len);
    for (long line = jb->line_begin; line < jb->line_end; ++line) {
        /* line enumerates the other two indices; rebuild the base offset. */
        long base;
        if (jb->axis == 2) {
            base = line * jb->n[2];
        } else if (jb->axis == 1) {
            long a = line / jb->n[2], c = line % jb->n[2];
            base = a * (long)jb->n[1] * jb->n[2] + c;
        } else {
            base = line; /* (b, c) flattened, stride n1*n2 along a */
        }
        fft_rec(len, jb->data + base, stride, buf, jb->roots, len);
        for (int j = 0; j < len; ++j) jb->data[base + (long)j * stride] = buf[j];
    }
    free(buf);
    return NULL;
}

static int g_threads = 1;

void oracle_set_threads(int nthreads) { g_threads = nthreads < 1 ? 1 : nthreads; }
int oracle_get_threads(void) { return g_threads; }

static void fft_axis(cplx* data, const int n[3], int axis, int sign) {
    long lines = (long)n[0] * n[1] * n[2] / n[axis];
    cplx* roots = make_roots(n[axis], sign);
    int nt = g_threads;
    if (nt > lines) nt = (int)lines;
    if (nt < 1) nt = 1;
    axis_job* jobs = (axis_job*)malloc(sizeof(axis_job) * (size_t)nt);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int t = 0; t < nt; ++t) {
        jobs[t].data = data;
        memcpy(jobs[t].n, n, sizeof(int) * 3);
        jobs[t].axis = axis;
        jobs[t].roots = roots;
        jobs[t].line_begin = lines * t / nt;
        jobs[t].line_end = lines * (t + 1) / nt;
    }
    if (nt == 1) {
        axis_worker(&jobs[0]);
    } else {
        for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, axis_worker, &jobs[t]);
        for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    }
    free(th);
    free(jobs);
    free(roots);
}

/*
 * In-place unnormalised 3D DFT of data[n0][n1][n2] (interleaved re, im).
 * sign = -1: forward, axes c, b, a.   sign = +1: inverse, axes a, b, c.
 */
void oracle_fft3d(const int n[3], double* data, int sign) {
    cplx* d = (cplx*)data;
    if (sign < 0) {
        fft_axis(d, n, 2, -1);
        fft_axis(d, n, 1, -1);
        fft_axis(d, n, 0, -1);
    } else {
        fft_axis(d, n, 0, +1);
        fft_axis(d, n, 1, +1);
        fft_axis(d, n, 2, +1);
    }
}

/* out[k] = sum_r in[r] exp(sign 2 pi i (k1 r1/N1 + k2 r2/N2 + k3 r3/N3)), O(N^2). */
void oracle_dft3d_brute(const int n[3], const double* in, double* out, int sign) {
    const cplx* x = (const cplx*)in;
    cplx* X = (cplx*)out;
    long N = (long)n[0] * n[1] * n[2];
    for (int k1 = 0; k1 < n[0]; ++k1)
        for (int k2 = 0; k2 < n[1]; ++k2)
            for (int k3 = 0; k3 < n[2]; ++k3) {
                double are = 0.0, aim = 0.0;
                for (int r1 = 0; r1 < n[0]; ++r1)
                    for (int r2 = 0; r2 < n[1]; ++r2)
                        for (int r3 = 0; r3 < n[2]; ++r3) {
                            /* phase = (k1 r1 N2 N3 + k2 r2 N1 N3 + k3 r3 N1 N2) / N, reduced mod N. */
                            long e = ((long)k1 * r1 % n[0]) * ((long)n[1] * n[2]) +
                                     ((long)k2 * r2 % n[1]) * ((long)n[0] * n[2]) +
                                     ((long)k3 * r3 % n[2]) * ((long)n[0] * n[1]);
                            e %= N;
                            double a = TWO_PI * (double)e / (double)N;
                            double c = cos(a), s = sign * sin(a);
                            cplx v = x[((long)r1 * n[1] + r2) * n[2] + r3];
                            are += v.re * c - v.im * s;
                            aim += v.re * s + v.im * c;
                        }
                X[((long)k1 * n[1] + k2) * n[2] + k3].re = are;
                X[((long)k1 * n[1] + k2) * n[2] + k3].im = aim;
            }
}

/* ------------------------------------------------------------ splat */

/* Signed frequency of index k on an axis of n points: k if k <= n/2, else k - n. */
static int fold(int k, int n) { return (2 * k <= n) ? k : k - n; }

static long wrap_index(long i, int n) {
    long r = i % n;
    return r < 0 ? r + n : r;
}

/*
 * rho[N1][N2][N3] = sum over atoms and periodic images of
 *   q_i (pi s^2)^(-3/2) exp(-|d|^2/s^2),  d = r - R_i - T,  |d| < rc.
 * The unwrapped index range around each atom enumerates every image within rc.
 */
void oracle_splat(const int n[3], const double L[3], double sigma, double rc, int nat, const double* pos,
                  const double* q, double* rho) {
    double h[3] = {L[0] / n[0], L[1] / n[1], L[2] / n[2]};
    double norm = pow(PI * sigma * sigma, -1.5);
    double inv_s2 = 1.0 / (sigma * sigma);
    long N = (long)n[0] * n[1] * n[2];
    memset(rho, 0, sizeof(double) * (size_t)N);
    for (int a = 0; a < nat; ++a) {
        const double* R = pos + 3 * a;
        long lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = (long)ceil((R[d] - rc) / h[d]);
            hi[d] = (long)floor((R[d] + rc) / h[d]);
        }
        for (long i = lo[0]; i <= hi[0]; ++i) {
            double dx = (double)i * h[0] - R[0];
            for (long j = lo[1]; j <= hi[1]; ++j) {
                double dy = (double)j * h[1] - R[1];
                for (long k = lo[2]; k <= hi[2]; ++k) {
                    double dz = (double)k * h[2] - R[2];
                    double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 >= rc * rc) continue;
                    long idx = (wrap_index(i, n[0]) * n[1] + wrap_index(j, n[1])) * n[2] + wrap_index(k, n[2]);
                    rho[idx] += q[a] * norm * exp(-d2 * inv_s2);
                }
            }
        }
    }
}

/* ------------------------------------------------------------ Poisson */

/* g_k = 4 pi / |G_k|^2 with G_k = 2 pi (k1'/L1, k2'/L2, k3'/L3), g_0 = 0. */
static double green(int k1, int k2, int k3, const int n[3], const double L[3]) {
    double g1 = TWO_PI * fold(k1, n[0]) / L[0];
    double g2 = TWO_PI * fold(k2, n[1]) / L[1];
    double g3 = TWO_PI * fold(k3, n[2]) / L[2];
    double G2 = g1 * g1 + g2 * g2 + g3 * g3;
    return G2 == 0.0 ? 0.0 : 4.0 * PI / G2;
}

/*
 * Periodic Poisson solve on the grid.
 * Inputs: rho[N1][N2][N3].  Outputs: vh[N1][N2][N3];
 * out3[0] = E_H from 1/2 dV sum rho V, out3[1] = E_H from the spectrum,
 * out3[2] = max |Im V| / max |Re V| before the real part is taken.
 * Returns 0, or -1 when memory is short.
 */
int oracle_poisson(const int n[3], const double L[3], const double* rho, double* vh, double* out3) {
    long N = (long)n[0] * n[1] * n[2];
    cplx* s = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    if (!s) return -1;
    for (long i = 0; i < N; ++i) {
        s[i].re = rho[i];
        s[i].im = 0.0;
    }
    oracle_fft3d(n, (double*)s, -1);
    double omega = L[0] * L[1] * L[2];
    double espec = 0.0;
    for (int k1 = 0; k1 < n[0]; ++k1)
        for (int k2 = 0; k2 < n[1]; ++k2)
            for (int k3 = 0; k3 < n[2]; ++k3) {
                long idx = ((long)k1 * n[1] + k2) * n[2] + k3;
                double g = green(k1, k2, k3, n, L);
                espec += g * (s[idx].re * s[idx].re + s[idx].im * s[idx].im);
                s[idx].re *= g;
                s[idx].im *= g;
            }
    espec *= omega / (2.0 * (double)N * (double)N);
    oracle_fft3d(n, (double*)s, +1);
    double max_re = 0.0, max_im = 0.0, ereal = 0.0;
    for (long i = 0; i < N; ++i) {
        double re = s[i].re / (double)N, im = s[i].im / (double)N;
        vh[i] = re;
        if (fabs(re) > max_re) max_re = fabs(re);
        if (fabs(im) > max_im) max_im = fabs(im);
        ereal += rho[i] * re;
    }
    ereal *= 0.5 * omega / (double)N;
    out3[0] = ereal;
    out3[1] = espec;
    out3[2] = max_re > 0.0 ? max_im / max_re : max_im;
    free(s);
    return 0;
}

/* ------------------------------------------------------------ forces */

/*
 * F_i = -dV sum_r V_r q_i (pi s^2)^(-3/2) sum_T exp(-|d|^2/s^2) 2 d / s^2,
 * phi_i = dV sum_r V_r (pi s^2)^(-3/2) sum_T exp(-|d|^2/s^2)   (= dE_H/dq_i),
 * d = r - R_i - T, |d| < rc.  f[n][3], phi[n] (phi may be NULL).
 */
void oracle_forces(const int n[3], const double L[3], double sigma, double rc, int nat, const double* pos,
                   const double* q, const double* vh, double* f, double* phi) {
    double h[3] = {L[0] / n[0], L[1] / n[1], L[2] / n[2]};
    double dV = L[0] * L[1] * L[2] / ((double)n[0] * n[1] * n[2]);
    double norm = pow(PI * sigma * sigma, -1.5);
    double inv_s2 = 1.0 / (sigma * sigma);
    for (int a = 0; a < nat; ++a) {
        const double* R = pos + 3 * a;
        long lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = (long)ceil((R[d] - rc) / h[d]);
            hi[d] = (long)floor((R[d] + rc) / h[d]);
        }
        double fx = 0.0, fy = 0.0, fz = 0.0, p = 0.0;
        for (long i = lo[0]; i <= hi[0]; ++i) {
            double dx = (double)i * h[0] - R[0];
            for (long j = lo[1]; j <= hi[1]; ++j) {
                double dy = (double)j * h[1] - R[1];
                for (long k = lo[2]; k <= hi[2]; ++k) {
                    double dz = (double)k * h[2] - R[2];
                    double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 >= rc * rc) continue;
                    long idx = (wrap_index(i, n[0]) * n[1] + wrap_index(j, n[1])) * n[2] + wrap_index(k, n[2]);
                    double gv = vh[idx] * norm * exp(-d2 * inv_s2);
                    p += gv;
                    fx += gv * 2.0 * dx * inv_s2;
                    fy += gv * 2.0 * dy * inv_s2;
                    fz += gv * 2.0 * dz * inv_s2;
                }
            }
        }
        f[3 * a + 0] = -dV * q[a] * fx;
        f[3 * a + 1] = -dV * q[a] * fy;
        f[3 * a + 2] = -dV * q[a] * fz;
        if (phi) phi[a] = dV * p;
    }
}

/* ------------------------------------------------------------ atom decomposition */

/* Cyclic Jacobi rotations on a symmetric 3x3 matrix: A = V diag(lam) V^T, V columns. */
static void jacobi3(const double A_in[9], double lam[3], double V[9]) {
    double A[9];
    memcpy(A, A_in, sizeof(A));
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = fabs(A[1]) + fabs(A[2]) + fabs(A[5]);
        double scale = fabs(A[0]) + fabs(A[4]) + fabs(A[8]);
        if (off <= 1e-300 || off <= 1e-17 * scale) break;
        for (int p = 0; p < 2; ++p)
            for (int r = p + 1; r < 3; ++r) {
                double apr = A[3 * p + r];
                if (apr == 0.0) continue;
                double theta = (A[3 * r + r] - A[3 * p + p]) / (2.0 * apr);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J the (p, r) rotation */
                for (int k = 0; k < 3; ++k) {
                    double akp = A[3 * k + p], akr = A[3 * k + r];
                    A[3 * k + p] = c * akp - s * akr;
                    A[3 * k + r] = s * akp + c * akr;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A[3 * p + k], ark = A[3 * r + k];
                    A[3 * p + k] = c * apk - s * ark;
                    A[3 * r + k] = s * apk + c * ark;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[3 * k + p], vkr = V[3 * k + r];
                    V[3 * k + p] = c * vkp - s * vkr;
                    V[3 * k + r] = s * vkp + c * vkr;
                }
                A[3 * p + r] = 0.0; /* the rotation annihilates this pair */
                A[3 * r + p] = 0.0;
            }
    }
    lam[0] = A[0];
    lam[1] = A[4];
    lam[2] = A[8];
}

typedef struct {
    double t;
    int idx;
} tkey;

static int cmp_tkey(const void* a, const void* b) {
    const tkey* x = (const tkey*)a;
    const tkey* y = (const tkey*)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

typedef struct {
    const double* pos;
    const double* w;
    int* perm;
    int* leaf_start;
    int n_leaf_written;
    tkey* keys;
} bisect_ctx;

/*
 * One node of the modified recursive bisection (Sec. 3.1.5): atoms
 * perm[begin, begin + count), nproc processes.  Leaves are emitted left first.
 */
static void bisect_node(bisect_ctx* cx, int begin, int count, int nproc) {
    if (nproc <= 1 || count == 0) {
        /* leaf node(s): one per process; a node with 0 atoms and several
           processes still owns that many (empty) leaves. */
        for (int p = 0; p < (nproc < 1 ? 1 : nproc); ++p) {
            cx->leaf_start[cx->n_leaf_written++] = (p == 0) ? begin : begin + count;
        }
        return;
    }
    /* Eq. center-of-mass: C = (1/N_a) sum_i w_i x_i */
    double C[3] = {0, 0, 0};
    for (int a = 0; a < count; ++a) {
        int i = cx->perm[begin + a];
        for (int d = 0; d < 3; ++d) C[d] += cx->w[i] * cx->pos[3 * i + d];
    }
    for (int d = 0; d < 3; ++d) C[d] /= (double)count;
    /* Eq. eq-inertia-tensor about C */
    double T[9] = {0};
    for (int a = 0; a < count; ++a) {
        int i = cx->perm[begin + a];
        double X = cx->pos[3 * i] - C[0], Y = cx->pos[3 * i + 1] - C[1], Z = cx->pos[3 * i + 2] - C[2];
        double w = cx->w[i];
        T[0] += w * (Y * Y + Z * Z);
        T[4] += w * (X * X + Z * Z);
        T[8] += w * (X * X + Y * Y);
        T[1] -= w * X * Y;
        T[2] -= w * X * Z;
        T[5] -= w * Y * Z;
    }
    T[3] = T[1];
    T[6] = T[2];
    T[7] = T[5];
    double lam[3], V[9];
    jacobi3(T, lam, V);
    /* Of the three eigenvectors, keep the one maximising F = sum_i w_i t_i^2
       (Eq. eq-function-F with |a| = 1).  Sign: largest |component| positive,
       lowest axis on ties. */
    double best_F = -1.0, axis[3] = {1, 0, 0};
    for (int e = 0; e < 3; ++e) {
        double v[3] = {V[0 * 3 + e], V[1 * 3 + e], V[2 * 3 + e]};
        double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int d = 0; d < 3; ++d) v[d] /= nv;
        int big = 0;
        for (int d = 1; d < 3; ++d)
            if (fabs(v[d]) > fabs(v[big])) big = d;
        if (v[big] < 0)
            for (int d = 0; d < 3; ++d) v[d] = -v[d];
        double F = 0.0;
        for (int a = 0; a < count; ++a) {
            int i = cx->perm[begin + a];
            double t = v[0] * (cx->pos[3 * i] - C[0]) + v[1] * (cx->pos[3 * i + 1] - C[1]) +
                       v[2] * (cx->pos[3 * i + 2] - C[2]);
            F += cx->w[i] * t * t;
        }
        if (F > best_F) {
            best_F = F;
            memcpy(axis, v, sizeof(axis));
        }
    }
    /* Eq. eq-projection-ti, then sort by t (ties by atom index). */
    for (int a = 0; a < count; ++a) {
        int i = cx->perm[begin + a];
        cx->keys[a].t = axis[0] * (cx->pos[3 * i] - C[0]) + axis[1] * (cx->pos[3 * i + 1] - C[1]) +
                        axis[2] * (cx->pos[3 * i + 2] - C[2]);
        cx->keys[a].idx = i;
    }
    qsort(cx->keys, (size_t)count, sizeof(tkey), cmp_tkey);
    for (int a = 0; a < count; ++a) cx->perm[begin + a] = cx->keys[a].idx;
    /* Modified bisection: left child gets ceil(nproc/2) processes and the
       smallest prefix whose weight W_k satisfies nproc * W_k >= n_left * W. */
    int n_left = (nproc + 1) / 2;
    double W = 0.0;
    for (int a = 0; a < count; ++a) W += cx->w[cx->perm[begin + a]];
    double cum = 0.0;
    int k = 0;
    while (k < count && (double)nproc * cum < (double)n_left * W) {
        cum += cx->w[cx->perm[begin + k]];
        ++k;
    }
    bisect_node(cx, begin, k, n_left);
    bisect_node(cx, begin + k, count - k, nproc - n_left);
}

/*
 * Decompose nat atoms over nproc processes (leaves).
 * perm[nat]: atom indices in leaf order; leaf_start[nproc + 1]: leaf l owns
 * perm[leaf_start[l] .. leaf_start[l+1]).  w may be NULL (all weights 1).
 * Returns 0, or -1 on bad arguments.
 */
int oracle_bisect(int nat, const double* pos, const double* w, int nproc, int* perm, int* leaf_start) {
    if (nat < 0 || nproc < 1) return -1;
    double* ww = (double*)malloc(sizeof(double) * (size_t)(nat > 0 ? nat : 1));
    for (int i = 0; i < nat; ++i) ww[i] = w ? w[i] : 1.0;
    for (int i = 0; i < nat; ++i) perm[i] = i;
    bisect_ctx cx;
    cx.pos = pos;
    cx.w = ww;
    cx.perm = perm;
    cx.leaf_start = leaf_start;
    cx.n_leaf_written = 0;
    cx.keys = (tkey*)malloc(sizeof(tkey) * (size_t)(nat > 0 ? nat : 1));
    bisect_node(&cx, 0, nat, nproc);
    leaf_start[nproc] = nat;
    free(cx.keys);
    free(ww);
    return cx.n_leaf_written == nproc ? 0 : -1;
}
