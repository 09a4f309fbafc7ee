// sym3.h -- eigen-decomposition of a symmetric 3x3 matrix by Jacobi rotations, shared by the
// host and the device versions of the atom reorder (the principal axis of the inertia tensor,
// Sec. 3.1.3), so both take the same axis from the same moment matrix.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define SYM3_HD __host__ __device__
#else
#define SYM3_HD
#endif

namespace hartree {

// Eigen-decomposition of a symmetric 3x3 matrix S (row major) by Jacobi
// rotations with the tau-form update; columns of E are the eigenvectors.
SYM3_HD inline void sym3_eigen(double S[3][3], double lam[3], double E[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) E[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        const double off = fabs(S[0][1]) + fabs(S[0][2]) + fabs(S[1][2]);
        if (off == 0.0) break;
        const double diag = fabs(S[0][0]) + fabs(S[1][1]) + fabs(S[2][2]);
        if (off < 1e-18 * diag) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;  // (0, 1), (0, 2), (1, 2)
            const double spq = S[p][q];
            if (spq == 0.0) continue;
            const double h = S[q][q] - S[p][p];
            double t;
            if (fabs(spq) < 1e-300 * fabs(h)) {
                t = spq / h;
            } else {
                const double th = 0.5 * h / spq;
                t = 1.0 / (fabs(th) + sqrt(1.0 + th * th));
                if (th < 0.0) t = -t;
            }
            const double c = 1.0 / sqrt(1.0 + t * t), s = t * c, tau = s / (1.0 + c);
            S[p][p] -= t * spq;
            S[q][q] += t * spq;
            S[p][q] = S[q][p] = 0.0;
            const int r = 3 - p - q;  // the remaining index
            const double srp = S[r][p], srq = S[r][q];
            S[r][p] = S[p][r] = srp - s * (srq + tau * srp);
            S[r][q] = S[q][r] = srq + s * (srp - tau * srq);
            for (int k = 0; k < 3; ++k) {
                const double ekp = E[k][p], ekq = E[k][q];
                E[k][p] = ekp - s * (ekq + tau * ekp);
                E[k][q] = ekq + s * (ekp - tau * ekq);
            }
        }
    }
    for (int i = 0; i < 3; ++i) lam[i] = S[i][i];
}


// The principal axis for the bisection: the eigenvector of the top eigenvalue of M (whose
// eigenvectors are those of the inertia tensor T = tr(M) I - M, and for which F(a) = a^T M a),
// normalised and signed so its largest component is positive (the lowest axis wins ties).
SYM3_HD inline void principal_axis(double M[3][3], double ax[3]) {
    double lam[3], E[3][3];
    sym3_eigen(M, lam, E);
    int top = 0;
    for (int e = 1; e < 3; ++e)
        if (lam[e] > lam[top]) top = e;
    for (int d = 0; d < 3; ++d) ax[d] = E[d][top];
    const double nrm = sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    int big = 0;
    for (int d = 0; d < 3; ++d) {
        ax[d] /= nrm;
        if (fabs(ax[d]) > fabs(ax[big])) big = d;
    }
    if (ax[big] < 0.0)
        for (int d = 0; d < 3; ++d) ax[d] = -ax[d];
}

}  // namespace hartree
