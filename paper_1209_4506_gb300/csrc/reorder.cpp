// reorder.cpp -- atom decomposition by modified recursive bisection with the
// inertia-tensor principal axis (Sec. 3.1.2 - 3.1.5 of the paper).
//
// Each node holds a contiguous range of the permutation and a process count
// p.  A node with p = 1 or no atoms is a leaf.  Otherwise:
//   C   = (1/N_a) sum_i w_i x_i                      (Eq. center-of-mass)
//   T   = inertia tensor about C                     (Eq. eq-inertia-tensor)
//   a   = the eigenvector of T maximising F = sum_i w_i t_i^2 (Eq. eq-function-F)
//   t_i = a . (x_i - C)                              (Eq. eq-projection-ti)
// the atoms are sorted by t and cut so the left child (ceil(p/2) processes)
// receives the shortest prefix whose weight W_k satisfies p W_k >= ceil(p/2) W.
//
// T = tr(M) I - M with M = sum_i w_i X_i X_i^T shares M's eigenvectors, and
// F(a) = a^T M a, so the wanted axis is M's top eigenvector; it is found with
// threshold Jacobi sweeps on M.  Ties: the axis is signed so its largest
// component is positive (lowest axis first), equal t keep atom-index order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/hartree.h"
#include "sym3.h"

namespace {

struct Node {
    int begin, count, procs;
};

}  // namespace

extern "C" int hartree_atoms_reorder(const double* pos, const double* w, int n, int n_leaves, int* perm,
                                     int* leaf_start) {
    if (n < 0 || n_leaves < 1 || !perm || !leaf_start || (n > 0 && !pos)) return HARTREE_ERR_INVALID;
    for (int i = 0; i < 3 * n; ++i)
        if (!std::isfinite(pos[i])) return HARTREE_ERR_INVALID;
    std::vector<double> wt(n > 0 ? n : 1, 1.0);
    if (w)
        for (int i = 0; i < n; ++i) {
            if (!(w[i] >= 0.0) || !std::isfinite(w[i])) return HARTREE_ERR_INVALID;
            wt[i] = w[i];
        }
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::vector<std::pair<double, int>> key;
    std::vector<Node> stack;
    stack.push_back({0, n, n_leaves});
    int leaf = 0;
    while (!stack.empty()) {
        const Node nd = stack.back();
        stack.pop_back();
        if (nd.procs <= 1 || nd.count == 0) {
            for (int p = 0; p < nd.procs; ++p) leaf_start[leaf++] = nd.begin + (p == 0 ? 0 : nd.count);
            continue;
        }
        const int* ids = perm + nd.begin;
        double cm[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < nd.count; ++a)
            for (int d = 0; d < 3; ++d) cm[d] += wt[ids[a]] * pos[3 * ids[a] + d];
        for (int d = 0; d < 3; ++d) cm[d] /= (double)nd.count;
        double Mx[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int a = 0; a < nd.count; ++a) {
            const int i = ids[a];
            const double X[3] = {pos[3 * i] - cm[0], pos[3 * i + 1] - cm[1], pos[3 * i + 2] - cm[2]};
            for (int r = 0; r < 3; ++r)
                for (int c = r; c < 3; ++c) Mx[r][c] += wt[i] * X[r] * X[c];
        }
        Mx[1][0] = Mx[0][1];
        Mx[2][0] = Mx[0][2];
        Mx[2][1] = Mx[1][2];
        double ax[3];
        hartree::principal_axis(Mx, ax);
        key.resize(nd.count);
        for (int a = 0; a < nd.count; ++a) {
            const int i = ids[a];
            key[a].first = ax[0] * (pos[3 * i] - cm[0]) + ax[1] * (pos[3 * i + 1] - cm[1]) +
                           ax[2] * (pos[3 * i + 2] - cm[2]);
            key[a].second = i;
        }
        std::sort(key.begin(), key.end());  // by t, then by atom index
        double W = 0.0;
        for (int a = 0; a < nd.count; ++a) {
            perm[nd.begin + a] = key[a].second;
            W += wt[key[a].second];
        }
        const int left = (nd.procs + 1) / 2;
        int cut = 0;
        double acc = 0.0;
        while (cut < nd.count && (double)nd.procs * acc < (double)left * W) acc += wt[perm[nd.begin + cut++]];
        // right child first on the stack so the left subtree is emitted first
        stack.push_back({nd.begin + cut, nd.count - cut, nd.procs - left});
        stack.push_back({nd.begin, cut, left});
    }
    leaf_start[n_leaves] = n;
    return leaf == n_leaves ? HARTREE_OK : HARTREE_ERR_INVALID;
}
