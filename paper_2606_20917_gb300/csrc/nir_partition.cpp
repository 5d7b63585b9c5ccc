// nir_partition.cpp -- contiguous, cost-balanced element ranges for a solve
// sharded across ranks (host code only).
//
// The elemental operators are local to each element, so the ranks of a
// sharded mesh exchange nothing in an apply; only the load must balance.  An
// element's cost is the sum-factorised Helmholtz flop count of its (shape, P)
// -- the counts the kernels' rooflines are measured against -- so a rank's
// work is the sum over its elements.  Ranges are cut on the concatenation of
// the blocks in block order (the layout of mesh vectors), each cut at the
// element boundary nearest to its share k W / nranks of the total W.
#include <cmath>
#include <vector>

#include "nir_internal.h"

namespace {

// Flops of one Helmholtz apply per element: the BwdTrans contraction stages
// and their transposes (2 flops per multiply-add, in the order of Eq.
// bwdsumfactet for the collapsed shapes), the collocation gradient and its
// transpose, and the per-point metric.
double helm_flops(int shape, int P)
{
    const double N = P + 1, Q = P + 2;
    switch (shape) {
    case NIR_QUAD: return 4 * (N * N * Q + N * Q * Q) + 8 * Q * Q * Q + 10 * Q * Q;
    case NIR_TRI: return 4 * (N * (N + 1) / 2 * Q + N * Q * Q) + 8 * Q * Q * Q + 10 * Q * Q;
    case NIR_HEX: return 4 * (N * N * N * Q + N * N * Q * Q + N * Q * Q * Q) + 12 * Q * Q * Q * Q + 20 * Q * Q * Q;
    case NIR_PRISM:
        return 4 * (N * N * (N + 1) / 2 * Q + N * N * Q * Q + N * Q * Q * Q) + 12 * Q * Q * Q * Q + 20 * Q * Q * Q;
    case NIR_PYR:
        return 4 * (N * (N + 1) * (2 * N + 1) / 6 * Q + N * N * Q * Q + N * Q * Q * Q) + 12 * Q * Q * Q * Q +
               20 * Q * Q * Q;
    case NIR_TET:
        return 4 * (N * (N + 1) * (N + 2) / 6 * Q + N * (N + 1) / 2 * Q * Q + N * Q * Q * Q) + 12 * Q * Q * Q * Q +
               20 * Q * Q * Q;
    default: return -1.0;
    }
}

}  // namespace

extern "C" int nir_partition_elements(int nblocks, const int *shape, const int *P, const int64_t *nelem, int nranks,
                                      int64_t *first_out)
{
    if (nblocks < 1 || !shape || !P || !nelem || nranks < 1 || !first_out) return NIR_ERR_INVALID_ARG;
    std::vector<double> w(nblocks);
    std::vector<int64_t> off(nblocks + 1, 0);
    std::vector<double> cum(nblocks + 1, 0.0);  // weight before block b
    for (int b = 0; b < nblocks; ++b) {
        if (P[b] < 1 || nelem[b] < 0) return NIR_ERR_INVALID_ARG;
        w[b] = helm_flops(shape[b], P[b]);
        if (!(w[b] > 0.0)) return NIR_ERR_INVALID_ARG;
        off[b + 1] = off[b] + nelem[b];
        cum[b + 1] = cum[b] + w[b] * (double)nelem[b];
    }
    const double W = cum[nblocks];
    first_out[0] = 0;
    int b = 0;
    for (int r = 1; r < nranks; ++r) {
        const double target = W * (double)r / (double)nranks;
        while (b + 1 < nblocks && cum[b + 1] < target) ++b;
        // inside block b: k elements of weight w[b] after its start
        double k = (target - cum[b]) / w[b];
        k = std::floor(k + 0.5);
        if (k < 0) k = 0;
        if (k > (double)nelem[b]) k = (double)nelem[b];
        int64_t cut = off[b] + (int64_t)k;
        if (cut < first_out[r - 1]) cut = first_out[r - 1];
        first_out[r] = cut;
    }
    first_out[nranks] = off[nblocks];
    for (int r = 1; r < nranks; ++r)
        if (first_out[r] > first_out[nranks]) first_out[r] = first_out[nranks];
    return NIR_OK;
}
