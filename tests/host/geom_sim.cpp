// Host run of the geometric-factor kernel (k_geometry in nir_geom_kernels.cuh),
// for the CPU test tests/test_geom_sim_cpu.py.  Not part of the library.
//
// The kernel is a grid-stride loop with no shared memory or synchronisation,
// so one host thread runs it over every point (or element) of a small block.
// Its tables are prepared as the library prepares them (per-direction points,
// reference weights, and for quads and hexes the lattice Lagrange tables at
// the points plus the element centre), its outputs are exactly sized (the
// element count rounded up to 64, as the library allocates), and the build
// uses AddressSanitizer.
//
// argv: shape P gorder pp.  stdin: E, then the nodes ([E][nodes per element][d]);
// stdout: the metric per unit ([E][Nq or 1][NG]) then d eta/d x and W
// ([E][Nq or 1][d*d + 1]), read back from the library's layouts; per point,
// then the whole FP32 copy of the metric as k_pack_metric lays it out.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>
using std::fma;
using std::isfinite;

struct HostDim {
    unsigned x, y, z;
};
static HostDim threadIdx, blockIdx, gridDim, blockDim;
static inline int atomicExch(int *p, int v)
{
    const int o = *p;
    *p = v;
    return o;
}
#undef __launch_bounds__
#define __launch_bounds__(...)
#define __double2float_rn(x) ((float)(x))  // round to nearest, as on the host

// the headers nir_geom.cu includes before its device code, then that code
#include "nir_basis.h"
#include "nir_geom.h"
#include "nir_internal.h"
#include "nir_layout.h"
#include "nir_geom_kernels.cuh"

int main(int argc, char **argv)
{
    if (argc != 5) return 1;
    const int shape = std::atoi(argv[1]), P = std::atoi(argv[2]), g = std::atoi(argv[3]), pp = std::atoi(argv[4]);
    const int N = P + 1, Q = P + 2, d = nirk::dim(shape), NQ = nirk::npts(shape, Q);
    const int ng = nirk::ngeo(shape), nl = nirk::nlam(shape);
    const bool tensor = shape == nirk::QUAD || shape == nirk::HEX;
    const int nv = tensor ? (d == 2 ? (g + 1) * (g + 1) : (g + 1) * (g + 1) * (g + 1))
                          : (shape == nirk::TRI ? 3 : shape == nirk::TET ? 4 : shape == nirk::PRISM ? 6 : 5);
    long long E = 0;
    if (std::scanf("%lld", &E) != 1 || E < 1) return 2;
    std::vector<double> nodes((size_t)E * nv * d);
    for (auto &v : nodes)
        if (std::scanf("%lf", &v) != 1) return 2;
    // tables, as the library's geometry set-up builds them
    std::vector<double> z(3 * Q), w(3 * Q), blob(nirb_table_size(shape, P, Q));
    if (!nirb_shape_rules(shape, Q, z.data(), w.data()) || !nirb_build_tables(shape, P, Q, blob.data(), 0)) return 3;
    const nirk::TabLayout L = nirk::layout(shape, N, Q);
    const int g1 = g + 1;
    std::vector<double> host(3 * Q + NQ + 2 * (Q + 1) * g1, 0.0);
    double *hz = host.data(), *hw = hz + 3 * Q, *hL = hw + NQ, *hdL = hL + (Q + 1) * g1;
    std::memcpy(hz, z.data(), sizeof(double) * 3 * Q);
    std::memcpy(hw, blob.data() + L.wq, sizeof(double) * NQ);
    if (tensor) {
        std::vector<double> zz(Q + 1);
        for (int q = 0; q < Q; ++q) zz[q] = z[q];
        zz[Q] = 0.0;  // element centre, for per-element factors
        nirb_lagrange_equi(g, Q + 1, zz.data(), hL, hdL);
    }
    const long long epad = (E + 63) / 64 * 64, units = pp ? epad * NQ : epad;
    std::vector<double> G((size_t)units * ng, 0.0), Lam((size_t)units * nl, 0.0);
    int err = 0;
    nirk::GeoArgs a;
    a.nodes = nodes.data();
    a.z = hz;
    a.wq = hw;
    a.Lg = hL;
    a.dLg = hdL;
    a.G = G.data();
    a.Lam = Lam.data();
    a.err = &err;
    a.nelem = E;
    a.shape = shape;
    a.Q = Q;
    a.g = g;
    a.pp = pp;
    threadIdx = HostDim{0, 0, 0};
    blockIdx = HostDim{0, 0, 0};
    gridDim = HostDim{1, 1, 1};
    blockDim = HostDim{1, 1, 1};
    nirk::k_geometry(a);
    if (err) return 6;
    const int per = pp ? NQ : 1;
    for (long long e = 0; e < E; ++e)
        for (int n = 0; n < per; ++n)
            for (int c = 0; c < ng; ++c)
                std::printf("%.17g\n", pp ? G[(((e >> 5) * NQ + n) * ng + c) * 32 + (e & 31)] : G[e * ng + c]);
    for (long long e = 0; e < E; ++e)
        for (int n = 0; n < per; ++n)
            for (int c = 0; c < nl; ++c)
                std::printf("%.17g\n", pp ? Lam[(((e >> 5) * NQ + n) * nl + c) * 32 + (e & 31)] : Lam[e * nl + c]);
    if (pp) {  // the FP32 copy the fused kernels read: packed by k_pack_metric, printed raw
        std::vector<float> packed((size_t)units * ng, -1.0f);
        nirk::k_pack_metric<float>(G.data(), packed.data(), epad / 32 * NQ, ng);  // one thread: the whole loop
        for (float v : packed) std::printf("%.9g\n", (double)v);
    }
    return 0;
}
