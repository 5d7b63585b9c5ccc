// Host build of the threading-over-elements stage code (nir_toe.cuh), for the
// CPU test tests/test_toe_stages_cpu.py: the per-element Helmholtz function is
// compiled as plain C++ and run on one element with exactly sized scratch and
// tables (the test builds it with AddressSanitizer, so any index outside them
// fails the run).  Not part of the library.
//
// stdin:  shape P lambda, then NQ*NG metric values (point-major) and M
//         coefficients; stdout: M result values.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <vector>
using std::fma;
#ifndef __launch_bounds__
#define __launch_bounds__(x)
#endif
struct HostDim {
    unsigned x, y, z;
};
static HostDim threadIdx, blockIdx, gridDim;
static inline void __syncthreads() {}
static inline void __syncwarp() {}
#include "nir_basis.h"
#include "nir_toe.cuh"

template <int SH, int N>
static int run(double lam)
{
    constexpr int Q = N + 1, NQ = nirk::npts(SH, Q), M = nirk::nmodes(SH, N), NG = nirk::ngeo(SH);
    constexpr auto L = nirk::layout(SH, N, Q);
    std::vector<double> G((size_t)NQ * NG), u(M);
    for (auto &v : G)
        if (std::scanf("%lf", &v) != 1) return 2;
    for (auto &v : u)
        if (std::scanf("%lf", &v) != 1) return 2;
    double *tab = new double[L.total];
    if (!nirb_build_tables(SH, N - 1, Q, tab, 0)) return 3;
    double *scr = new double[5 * NQ];
    double *geo = new double[(size_t)NQ * NG * 32];  // one element, 32-element interleave
    for (int n = 0; n < NQ; ++n)
        for (int c = 0; c < NG; ++c) geo[((size_t)n * NG + c) * 32] = G[(size_t)n * NG + c];
    nirt::Scr<double, NQ> X{scr, 1u};
    for (int m = 0; m < M; ++m) X(4, m) = u[m];
    nirt::helm_element<SH, N, double, double>(tab, X, geo, 1, 0, lam);
    for (int m = 0; m < M; ++m) std::printf("%.17g\n", X(3, m));
    delete[] tab;
    delete[] scr;
    delete[] geo;
    return 0;
}

template <int SH>
static int by_n(int P, double lam)
{
    switch (P + 1) {
    case 2: return run<SH, 2>(lam);
    case 3: return run<SH, 3>(lam);
    case 4: return run<SH, 4>(lam);
    case 5: return run<SH, 5>(lam);
    case 6: return run<SH, 6>(lam);
    case 7: return run<SH, 7>(lam);
    case 8: return run<SH, 8>(lam);
    case 9: return run<SH, 9>(lam);
    case 10: return run<SH, 10>(lam);
    }
    return 1;
}

int main()
{
    int shape = -1, P = 0;
    double lam = 0;
    if (std::scanf("%d %d %lf", &shape, &P, &lam) != 3) return 2;
    switch (shape) {
    case 0: return by_n<0>(P, lam);
    case 1: return by_n<1>(P, lam);
    case 2: return by_n<2>(P, lam);
    case 3: return by_n<3>(P, lam);
    case 4: return by_n<4>(P, lam);
    }
    return 1;
}
