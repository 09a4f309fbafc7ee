// reorder_dev.cu -- the atom decomposition of Sec. 3.1 (modified recursive bisection with the
// inertia-tensor principal axis, Sec. 3.1.2 - 3.1.5) on the device.
//
// The recursion is taken level by level: one launch per level of the bisection tree, one CTA per
// node of that level.  A node is a contiguous range [begin, begin + count) of the permutation,
// a process (leaf) count p and the index leaf0 of its first leaf.  Its CTA
//   * sums C = (1/N_a) sum_i w_i x_i (Eq. center-of-mass) and M = sum_i w_i X_i X_i^T, X = x - C,
//     in FP64 over the block (fixed order);
//   * takes the principal axis a (the eigenvector of M's top eigenvalue, which maximises
//     F = sum_i w_i t_i^2, Eq. eq-function-F; T = tr(M) I - M of Eq. eq-inertia-tensor has the
//     same eigenvectors) with the same 3x3 Jacobi solver as the host reorder;
//   * projects t_i = a . X_i (Eq. eq-projection-ti), sorts its range by (t, atom index) with a
//     bitonic sort in shared memory (in global scratch for ranges beyond the shared-memory
//     capacity), and cuts it: the left child (ceil(p/2) processes) takes the shortest prefix whose
//     weight W_k satisfies p W_k >= ceil(p/2) W (Sec. 3.1.4 with the 26-atom example's reading).
// Children of node k of a level are nodes 2k and 2k + 1 of the next; the tree's shape depends
// only on the leaf count, so the host launches ceil(log2 n_leaves) + 1 levels without reading
// anything back.  A node with one process, or with no atoms, writes its leaves' starts.
#include <climits>
#include <cmath>

#include "internal.cuh"
#include "sym3.h"

namespace hartree {

namespace {

struct BisectNode {
    int begin, count, procs, leaf0;  // procs = 0: an unused slot of the level
};

constexpr int kBisectThreads = 512;

// Bitonic sort of n2 (a power of two) (key, index) pairs by key, then index; the block's threads
// cooperate, with a barrier between steps.  Padding entries carry key +inf.
__device__ void bitonic_sort(double* key, int* idx, int n2) {
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const double ki = key[i], kl = key[l];
                    const int ii = idx[i], il = idx[l];
                    const bool gt = ki > kl || (ki == kl && ii > il);  // (i) after (l)
                    const bool up = (i & k) == 0;
                    if (gt == up) {
                        key[i] = kl;
                        key[l] = ki;
                        idx[i] = il;
                        idx[l] = ii;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kBisectThreads) k_bisect_level(const double* __restrict__ pos,
                                                                  const double* __restrict__ w, int n, int n_leaves,
                                                                  int level, const BisectNode* in, BisectNode* out,
                                                                  int* perm, int* leaf_start, double* gkey, int* gidx,
                                                                  int cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kBisectThreads / 32];
    __shared__ double axis[3], cm[3];
    const int k = blockIdx.x;
    BisectNode nd;
    if (level == 0)
        nd = BisectNode{0, n, n_leaves, 0};
    else
        nd = in[k];
    if (nd.procs == 0) {  // an unused slot: its children are unused too (the level arrays are reused)
        if (threadIdx.x == 0) out[2 * k] = out[2 * k + 1] = BisectNode{0, 0, 0, 0};
        return;
    }
    if (level == 0) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
        if (threadIdx.x == 0) leaf_start[n_leaves] = n;
        __syncthreads();
    }
    if (nd.procs == 1 || nd.count == 0) {
        // a leaf, or processes without atoms: every leaf of the node starts at begin (the empty
        // ones after the first at begin + count = begin)
        for (int q = threadIdx.x; q < nd.procs; q += blockDim.x) leaf_start[nd.leaf0 + q] = nd.begin + (q == 0 ? 0 : nd.count);
        if (threadIdx.x == 0) out[2 * k] = out[2 * k + 1] = BisectNode{0, 0, 0, 0};
        return;
    }
    const int* ids = perm + nd.begin;
    // centre of mass: sum_i w_i x_i / N_a (Eq. center-of-mass divides by the atom count)
    double s[3] = {0.0, 0.0, 0.0};
    for (int a = threadIdx.x; a < nd.count; a += blockDim.x) {
        const int i = ids[a];
        const double wi = w ? w[i] : 1.0;
        for (int d = 0; d < 3; ++d) s[d] += wi * pos[3 * i + d];
    }
    for (int d = 0; d < 3; ++d) {
        const double t = block_sum_double(s[d], red);
        if (threadIdx.x == 0) cm[d] = t / (double)nd.count;
        __syncthreads();
    }
    // moment matrix M = sum_i w_i X_i X_i^T, upper triangle
    double m[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int a = threadIdx.x; a < nd.count; a += blockDim.x) {
        const int i = ids[a];
        const double wi = w ? w[i] : 1.0;
        const double X[3] = {pos[3 * i] - cm[0], pos[3 * i + 1] - cm[1], pos[3 * i + 2] - cm[2]};
        m[0] += wi * X[0] * X[0];
        m[1] += wi * X[0] * X[1];
        m[2] += wi * X[0] * X[2];
        m[3] += wi * X[1] * X[1];
        m[4] += wi * X[1] * X[2];
        m[5] += wi * X[2] * X[2];
    }
    double M[3][3];
    for (int c = 0; c < 6; ++c) {
        const double t = block_sum_double(m[c], red);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int r = c < 3 ? 0 : (c < 5 ? 1 : 2), col = c < 3 ? c : (c < 5 ? c - 2 : 2);
            M[r][col] = M[col][r] = t;
        }
    }
    if (threadIdx.x == 0) {
        double ax[3];
        principal_axis(M, ax);
        for (int d = 0; d < 3; ++d) axis[d] = ax[d];
    }
    __syncthreads();
    // projections t_i and the sort of the range by (t, atom index)
    int n2 = 1;
    while (n2 < nd.count) n2 <<= 1;
    double* key;
    int* idx;
    if (n2 <= cap) {
        key = reinterpret_cast<double*>(smem_raw);
        idx = reinterpret_cast<int*>(key + cap);
    } else {  // beyond the shared-memory capacity: this node's own range of the global scratch
        key = gkey + 2 * (size_t)nd.begin;
        idx = gidx + 2 * (size_t)nd.begin;
    }
    for (int a = threadIdx.x; a < n2; a += blockDim.x) {
        if (a < nd.count) {
            const int i = ids[a];
            key[a] = axis[0] * (pos[3 * i] - cm[0]) + axis[1] * (pos[3 * i + 1] - cm[1]) +
                     axis[2] * (pos[3 * i + 2] - cm[2]);
            idx[a] = i;
        } else {
            key[a] = INFINITY;
            idx[a] = INT_MAX;
        }
    }
    __syncthreads();
    bitonic_sort(key, idx, n2);
    // the cut: the shortest prefix with p W_k >= ceil(p/2) W
    const int left = (nd.procs + 1) / 2;
    if (threadIdx.x == 0) {
        int cut;
        if (!w) {
            cut = (int)(((long long)left * nd.count + nd.procs - 1) / nd.procs);  // unit weights: exact
        } else {
            double W = 0.0;  // in sorted order, as the host sums it
            for (int a = 0; a < nd.count; ++a) W += w[idx[a]];
            double acc = 0.0;
            cut = 0;
            while (cut < nd.count && (double)nd.procs * acc < (double)left * W) acc += w[idx[cut++]];
        }
        out[2 * k] = BisectNode{nd.begin, cut, left, nd.leaf0};
        out[2 * k + 1] = BisectNode{nd.begin + cut, nd.count - cut, nd.procs - left, nd.leaf0 + left};
    }
    for (int a = threadIdx.x; a < nd.count; a += blockDim.x) perm[nd.begin + a] = idx[a];
}

}  // namespace

// Scratch of the device reorder for up to max_atoms atoms and leaves, span = the next power of two:
// two node levels of 2 span slots (a level of 2^l <= span nodes writes 2^(l+1) children) and the
// global-sort fallback's keys and indices, a node's padded range at twice its offset (2 span each).
size_t bisect_scratch_bytes(int max_atoms) {
    size_t span = 1;
    while (span < (size_t)max_atoms) span <<= 1;
    return 2 * (2 * span) * sizeof(BisectNode) + 2 * span * (sizeof(double) + sizeof(int)) + 256;
}

cudaError_t launch_bisect(const Plan& p, const double* pos, const double* w, int n, int n_leaves, int* perm,
                          int* leaf_start, cudaStream_t s) {
    int span = 1;
    while (span < p.max_atoms) span <<= 1;
    unsigned char* base = static_cast<unsigned char*>(p.bisect);
    BisectNode* lv[2] = {reinterpret_cast<BisectNode*>(base), reinterpret_cast<BisectNode*>(base) + 2 * span};
    double* gkey = reinterpret_cast<double*>(lv[1] + 2 * span);
    int* gidx = reinterpret_cast<int*>(gkey + 2 * span);
    int depth = 0;
    while ((1 << depth) < n_leaves) ++depth;
    // shared-memory sort capacity: the largest range of a level, with room for uneven cuts, at most 2^14
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int level = 0; level <= depth; ++level) {
        int cap = n2 >> level;
        cap = cap < 64 ? 64 : (cap > 16384 ? 16384 : cap);
        if (level > 0 && cap < 16384) cap <<= 1;  // weighted cuts can leave a child above half
        const size_t smem = (size_t)cap * (sizeof(double) + sizeof(int));
        k_bisect_level<<<1u << level, kBisectThreads, smem, s>>>(pos, w, n, n_leaves, level, lv[level & 1],
                                                                 lv[(level + 1) & 1], perm, leaf_start, gkey, gidx,
                                                                 cap);
        ++p.launches;
    }
    return cudaGetLastError();
}

cudaError_t configure_bisect() {
    int optin = 0;
    cudaError_t e = optin_smem(&optin);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_bisect_level, optin);
    return e;
}

}  // namespace hartree
