// nir_toe.cuh -- the Helmholtz operator under the "threading over elements"
// strategy of Sec. 3.3: one thread owns one element and runs every
// sum-factorised stage of it alone, with the intermediate tensors, which no
// longer fit in registers or shared memory at one element per thread, held in
// global memory and expanded to the grid size.
//
// The paper contrasts this strategy with threading over the expansion
// coefficients (the library's default kernels: a CTA shares a group of
// elements and its temporaries in shared memory) and measures both (Sec. 4,
// Fig. GPURESULTS).  Here it is built for sm_103a as follows:
//   * scratch: 5 arrays of Q^d values per thread of the grid, laid out
//     [array][index][thread] so the 32 lanes of a warp (32 consecutive
//     elements at the same structural index) touch 32 consecutive words;
//   * the [E][M] coefficient arrays are read and written through a 32 x 33
//     shared-memory tile per warp (row-contiguous global accesses, one
//     transpose), so HBM sees whole lines; the per-point metric is already
//     interleaved by 32 elements, i.e. by warp;
//   * tables live in shared memory; all lanes read the same entry at the same
//     time (broadcast), because every lane runs the same loop nest;
//   * the psiA contractions use the even/odd forms of the symmetric first-
//     direction points (the table block Bs), the collapsed directions the
//     ragged class tables, with the same extra terms for the collapsed vertex
//     and edge modes as the default kernels.
// No thread waits on another except at the warp transposes (__syncwarp).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "nir_layout.h"

namespace nirt {

using nirk::cls_off;
using nirk::layout;
using nirk::prism_m0;
using nirk::sym_ne;
using nirk::sym_no;
using nirk::TabLayout;
using nirk::tet_m0;
using nirk::tet_pair;
using nirk::tri_m0;

constexpr int kThreads = 128;  // threads per CTA (4 warps)
constexpr int kBufs = 5;       // scratch arrays of Q^d values per thread
constexpr int kTile = 33;      // padded row of the warp transpose tile

struct ToeArgs {
    const void *in;   // coefficients [E][M] (storage type)
    void *out;        // coefficients [E][M]
    const void *geo;  // metric: per point, 32-element interleaved; or per element
    const void *tab;  // table blob in the compute type (device)
    void *scr;        // scratch: kBufs * Q^d * (grid threads) compute-type values
    long long nelem;
    double lambda;
    int geo_pp;
};

template <class T> struct CT { using type = float; };
template <> struct CT<double> { using type = double; };

__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ void put(double v, double *p) { *p = v; }
__device__ __forceinline__ void put(float v, float *p) { *p = v; }
__device__ __forceinline__ void put(float v, __nv_bfloat16 *p) { *p = __float2bfloat16_rn(v); }

// A zero the compiler cannot see through.  Table reads indexed with it stay
// inside the loop that calls the line function: otherwise the compiler hoists
// every table value of a ragged class out of the loop into registers (the
// tetrahedron at P = 8 then spills kilobytes per thread).
__device__ __forceinline__ int opaque_zero()
{
#ifdef __CUDA_ARCH__
    int z;
    asm volatile("mov.u32 %0, 0;" : "=r"(z));
    return z;
#else
    return 0;
#endif
}

template <int I, int E, class F>
__device__ __forceinline__ void cfor(F &&f)
{
    if constexpr (I < E) {
        f(std::integral_constant<int, I>{});
        cfor<I + 1, E>(f);
    }
}

// One thread's scratch: array b, index i at p[(b * NQ + i) * n] (32-bit
// offsets: the host keeps the scratch below 2^31 values).  The stride passes
// through an opaque zero at every access, so the compiler recomputes i * n
// next to the load instead of keeping one hoisted offset per unrolled index
// live across the stage loops (which otherwise costs 100+ registers).
template <class A, int NQ>
struct Scr {
    A *p;
    unsigned n;
    __device__ __forceinline__ A &operator()(int b, int i) const
    {
        return p[(unsigned)(b * NQ + i) * (n + (unsigned)opaque_zero())];
    }
};

// psiA line, modes -> points, even/odd form: x[N] -> st(i, u_i), i < Q.
template <class A, int N, int Q, class ST>
__device__ __forceinline__ void line_bwd(const A *Bs0, const A (&x)[N], ST st)
{
    const A *Bs = Bs0 + opaque_zero();
    constexpr int NE = sym_ne(N), NO = sym_no(N), W = NE + NO, QL = Q / 2;
    A xe[NE], xo[NO];
    xe[0] = x[0] + x[1];
    xo[0] = x[0] - x[1];
#pragma unroll
    for (int k = 1; k < NE; ++k) xe[k] = x[2 * k];
#pragma unroll
    for (int k = 1; k < NO; ++k) xo[k] = x[2 * k + 1];
#pragma unroll
    for (int i = 0; i < QL; ++i) {
        A E = A(0), O = A(0);
#pragma unroll
        for (int k = 0; k < NE; ++k) E = fma(Bs[i * W + k], xe[k], E);
#pragma unroll
        for (int k = 0; k < NO; ++k) O = fma(Bs[i * W + NE + k], xo[k], O);
        st(i, E + O);
        st(Q - 1 - i, E - O);
    }
    if constexpr (Q % 2 == 1) {
        A E = A(0);
#pragma unroll
        for (int k = 0; k < NE; ++k) E = fma(Bs[QL * W + k], xe[k], E);
        st(QL, E);
    }
}

// psiA line, points -> modes (the transpose): f[Q] -> st(p, sum_i psiA_p(z_i) f_i).
template <class A, int N, int Q, class ST>
__device__ __forceinline__ void line_iprod(const A *Bs0, const A (&f)[Q], ST st)
{
    const A *Bs = Bs0 + opaque_zero();
    constexpr int NE = sym_ne(N), NO = sym_no(N), W = NE + NO, QL = Q / 2, QH = (Q + 1) / 2;
    A fe[QH], fo[QL > 0 ? QL : 1];
#pragma unroll
    for (int i = 0; i < QL; ++i) {
        fe[i] = f[i] + f[Q - 1 - i];
        fo[i] = f[i] - f[Q - 1 - i];
    }
    if constexpr (Q % 2 == 1) fe[QL] = f[QL];
    A Se = A(0), So = A(0);
#pragma unroll
    for (int i = 0; i < QH; ++i) Se = fma(Bs[i * W], fe[i], Se);
#pragma unroll
    for (int i = 0; i < QL; ++i) So = fma(Bs[i * W + NE], fo[i], So);
    st(0, Se + So);
    st(1, Se - So);
#pragma unroll
    for (int k = 1; k < NE; ++k) {
        A acc = A(0);
#pragma unroll
        for (int i = 0; i < QH; ++i) acc = fma(Bs[i * W + k], fe[i], acc);
        st(2 * k, acc);
    }
#pragma unroll
    for (int k = 1; k < NO; ++k) {
        A acc = A(0);
#pragma unroll
        for (int i = 0; i < QL; ++i) acc = fma(Bs[i * W + NE + k], fo[i], acc);
        st(2 * k + 1, acc);
    }
}

// Ragged class line, modes -> points: out_o = sum_{r<NC} C[o*NC + r] x_r
// (+ C0[o*N + 1] xx for the collapsed extra column when EX).
template <class A, int N, int Q, int NC, bool EX, class ST>
__device__ __forceinline__ void line_cls_bwd(const A *Cc, const A *Cc0, const A (&x)[NC], A xx, ST st)
{
    const int z = opaque_zero();
    const A *C = Cc + z, *C0 = Cc0 + z;
#pragma unroll
    for (int o = 0; o < Q; ++o) {
        A acc = A(0);
#pragma unroll
        for (int r = 0; r < NC; ++r) acc = fma(C[o * NC + r], x[r], acc);
        if constexpr (EX) acc = fma(C0[o * N + 1], xx, acc);
        st(o, acc);
    }
}

// Ragged class line, points -> modes: out_o = sum_i C[i*NC + o] f_i, o < NC
// (+ sum_i C0[i*N + 1] ff_i into output 1 for each of the NEX extra lines
// ff, one line after the other).
template <class A, int N, int Q, int NC, int NEX, class ST>
__device__ __forceinline__ void line_cls_iprod(const A *Cc, const A *Cc0, const A (&f)[Q],
                                               const A (&ff)[NEX > 0 ? NEX : 1][Q], ST st)
{
    const int z = opaque_zero();
    const A *C = Cc + z, *C0 = Cc0 + z;
#pragma unroll
    for (int o = 0; o < NC; ++o) {
        A acc = A(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) acc = fma(C[i * NC + o], f[i], acc);
        if constexpr (NEX > 0) {
            if (o == 1) {
#pragma unroll
                for (int l = 0; l < NEX; ++l)
#pragma unroll
                    for (int i = 0; i < Q; ++i) acc = fma(C0[i * N + 1], ff[l][i], acc);
            }
        }
        st(o, acc);
    }
}

// The Helmholtz operator of one element (thread): modes in scratch array 4,
// result modes in array 3.
//   BwdTrans:  4 -> 1 (-> 2) -> 0 (u at the points)
//   metric:    0 -> 1, 2 (, 3) (v = G grad u), 4 (lambda W)
//   D^T:       1, 2 (, 3), 4, 0 -> 0
//   IProduct:  0 -> 1 (-> 2) -> 3
template <int SH, int N, class T, class A>
__device__ __forceinline__ void helm_element(const A *tab, const Scr<A, nirk::npts(SH, N + 1)> &X, const T *geo,
                                             int geo_pp, long long e, A lam)
{
    constexpr int Q = N + 1, D = nirk::dim(SH), NQ = nirk::npts(SH, Q), QQ = Q * Q, NG = nirk::ngeo(SH);
    constexpr TabLayout L = layout(SH, N, Q);
    const A *Bs = tab + L.Bs, *Bb = tab + L.Bb, *Bc = tab + L.Bc, *wq = tab + L.wq;
    const A *D0 = tab + L.D1, *D1 = tab + L.D2, *D2 = tab + L.D3;

    // ---------------- BwdTrans
    if constexpr (SH == nirk::QUAD) {
#pragma unroll 1
        for (int p = 0; p < N; ++p) {
            A x[N];
#pragma unroll
            for (int q = 0; q < N; ++q) x[q] = X(4, p * N + q);
            line_bwd<A, N, Q>(Bs, x, [&](int o, A v) { X(1, p * Q + o) = v; });
        }
    } else if constexpr (SH == nirk::TRI) {
        cfor<0, N>([&](auto cc) {
            constexpr int p = decltype(cc)::value, NC = N - p;
            A x[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) x[q] = X(4, tri_m0(N, p) + q);
            const A xx = p == 1 ? X(4, 1) : A(0);
            line_cls_bwd<A, N, Q, NC, p == 1>(Bb + cls_off(N, Q, p), Bb, x, xx,
                                               [&](int o, A v) { X(1, p * Q + o) = v; });
        });
    } else if constexpr (SH == nirk::HEX) {
#pragma unroll 1
        for (int s = 0; s < N * N; ++s) {
            A x[N];
#pragma unroll
            for (int r = 0; r < N; ++r) x[r] = X(4, s * N + r);
            line_bwd<A, N, Q>(Bs, x, [&](int o, A v) { X(1, s * Q + o) = v; });
        }
    } else if constexpr (SH == nirk::PRISM) {
        cfor<0, N>([&](auto cc) {
            constexpr int p = decltype(cc)::value, NC = N - p;
#pragma unroll 1
            for (int q = 0; q < N; ++q) {
                A x[NC];
#pragma unroll
                for (int r = 0; r < NC; ++r) x[r] = X(4, prism_m0(N, p, q) + r);
                const A xx = p == 1 ? X(4, prism_m0(N, 0, q) + 1) : A(0);
                line_cls_bwd<A, N, Q, NC, p == 1>(Bb + cls_off(N, Q, p), Bb, x, xx,
                                                   [&](int o, A v) { X(1, (p * N + q) * Q + o) = v; });
            }
        });
    } else {  // TET: pairs (p, q), class c = p + q
        cfor<0, N>([&](auto cc) {
            constexpr int c = decltype(cc)::value, NC = N - c;
#pragma unroll 1
            for (int p = 0; p <= c; ++p) {
                A x[NC];
#pragma unroll
                for (int r = 0; r < NC; ++r) x[r] = X(4, tet_m0(N, p, c - p) + r);
                const A xx = c == 1 ? X(4, 1) : A(0);
                line_cls_bwd<A, N, Q, NC, c == 1>(Bc + cls_off(N, Q, c), Bc, x, xx,
                                                   [&](int o, A v) { X(1, tet_pair(N, p, c - p) * Q + o) = v; });
            }
        });
    }
    if constexpr (D == 3) {  // second direction: 1 -> 2, t2[p][j][k]
        if constexpr (SH == nirk::TET) {
            cfor<0, N>([&](auto cc) {
                constexpr int p = decltype(cc)::value, NC = N - p;
#pragma unroll 1
                for (int k = 0; k < Q; ++k) {
                    A x[NC];
#pragma unroll
                    for (int q = 0; q < NC; ++q) x[q] = X(1, (tet_pair(N, p, 0) + q) * Q + k);
                    const A xx = p == 1 ? X(1, tet_pair(N, 0, 1) * Q + k) : A(0);
                    line_cls_bwd<A, N, Q, NC, p == 1>(Bb + cls_off(N, Q, p), Bb, x, xx,
                                                       [&](int o, A v) { X(2, (p * Q + o) * Q + k) = v; });
                }
            });
        } else {
#pragma unroll 1
            for (int s = 0; s < N * Q; ++s) {
                const int p = s / Q, k = s - p * Q;
                A x[N];
#pragma unroll
                for (int q = 0; q < N; ++q) x[q] = X(1, (p * N + q) * Q + k);
                line_bwd<A, N, Q>(Bs, x, [&](int o, A v) { X(2, (p * Q + o) * Q + k) = v; });
            }
        }
        // first direction: 2 -> 0, u[i + Q j + Q^2 k]
#pragma unroll 1
        for (int s = 0; s < QQ; ++s) {
            const int k = s / Q, j = s - k * Q;
            A x[N];
#pragma unroll
            for (int p = 0; p < N; ++p) x[p] = X(2, (p * Q + j) * Q + k);
            line_bwd<A, N, Q>(Bs, x, [&](int o, A v) { X(0, o + Q * s) = v; });
        }
    } else {
#pragma unroll 1
        for (int j = 0; j < Q; ++j) {
            A x[N];
#pragma unroll
            for (int p = 0; p < N; ++p) x[p] = X(1, p * Q + j);
            line_bwd<A, N, Q>(Bs, x, [&](int o, A v) { X(0, o + Q * j) = v; });
        }
    }

    // ---------------- metric: v_a = sum_b G_ab du/d eta_b; lambda W
    // (the arithmetic, operation for operation, of the default FP64 kernel, so
    // both strategies give the same bits there)
    auto G = [&](int n, int c) -> A {
        if (geo_pp) {  // FP32/BF16 copies use the packed per-point layout
            if constexpr (sizeof(T) < 8) return to_c(geo[nirk::geo_packed_index(e, n, c, NQ, NG)]);
            else return to_c(geo[((((e >> 5) * NQ + n) * NG + c) << 5) + (e & 31)]);
        }
        const A v = to_c(geo[e * NG + c]);
        return c == NG - 1 ? v * wq[n] : v;  // per element: W takes the reference weight
    };
#pragma unroll 1
    for (int n = 0; n < NQ; ++n) {
        const int i = n % Q, j = (n / Q) % Q, k = n / QQ;
        A u0 = A(0), u1 = A(0), u2 = A(0);
#pragma unroll
        for (int r = 0; r < Q; ++r) u0 = fma(D0[i * Q + r], X(0, r + Q * j + QQ * k), u0);
#pragma unroll
        for (int r = 0; r < Q; ++r) u1 = fma(D1[j * Q + r], X(0, i + Q * r + QQ * k), u1);
        if constexpr (D == 3) {
#pragma unroll
            for (int r = 0; r < Q; ++r) u2 = fma(D2[k * Q + r], X(0, i + Q * j + QQ * r), u2);
        }
        if (!geo_pp) {  // per element: the metric components scale the gradient by the reference weight
            u0 *= wq[n];
            u1 *= wq[n];
            if constexpr (D == 3) u2 *= wq[n];
        }
        if constexpr (D == 3) {
            const A g00 = G(n, 0), g01 = G(n, 1), g02 = G(n, 2), g11 = G(n, 3), g12 = G(n, 4), g22 = G(n, 5);
            X(1, n) = fma(g00, u0, fma(g01, u1, g02 * u2));
            X(2, n) = fma(g01, u0, fma(g11, u1, g12 * u2));
            X(3, n) = fma(g02, u0, fma(g12, u1, g22 * u2));
        } else {
            const A g00 = G(n, 0), g01 = G(n, 1), g11 = G(n, 2);
            X(1, n) = fma(g00, u0, g01 * u1);
            X(2, n) = fma(g01, u0, g11 * u1);
        }
        X(4, n) = lam * G(n, NG - 1);
    }
    // ---------------- sum_a D_a^T v_a + lambda W u, in place over u
#pragma unroll 1
    for (int n = 0; n < NQ; ++n) {
        const int i = n % Q, j = (n / Q) % Q, k = n / QQ;
        A acc = A(0);
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fma(D0[r * Q + i], X(1, r + Q * j + QQ * k), acc);
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fma(D1[r * Q + j], X(2, i + Q * r + QQ * k), acc);
        if constexpr (D == 3) {
#pragma unroll
            for (int r = 0; r < Q; ++r) acc = fma(D2[r * Q + k], X(3, i + Q * j + QQ * r), acc);
        }
        X(0, n) = fma(X(4, n), X(0, n), acc);
    }

    // ---------------- IProductWRTBase of the point values in array 0
    if constexpr (D == 3) {
        // first direction: 0 -> 1, t[p][j][k]
#pragma unroll 1
        for (int s = 0; s < QQ; ++s) {
            const int k = s / Q, j = s - k * Q;
            A f[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = X(0, i + Q * s);
            line_iprod<A, N, Q>(Bs, f, [&](int o, A v) { X(1, o * QQ + j * Q + k) = v; });
        }
        // second direction: 1 -> 2
        if constexpr (SH == nirk::TET) {
            cfor<0, N>([&](auto cc) {
                constexpr int p = decltype(cc)::value, NC = N - p;
#pragma unroll 1
                for (int k = 0; k < Q; ++k) {
                    constexpr int NEX = p == 0 ? 1 : 0;
                    A f[Q], ff[NEX > 0 ? NEX : 1][Q];
#pragma unroll
                    for (int j = 0; j < Q; ++j) {
                        f[j] = X(1, p * QQ + j * Q + k);
                        if constexpr (NEX > 0) ff[0][j] = X(1, QQ + j * Q + k);
                    }
                    line_cls_iprod<A, N, Q, NC, NEX>(Bb + cls_off(N, Q, p), Bb, f, ff,
                                                      [&](int o, A v) { X(2, (tet_pair(N, p, 0) + o) * Q + k) = v; });
                }
            });
        } else {
#pragma unroll 1
            for (int s = 0; s < N * Q; ++s) {
                const int p = s / Q, k = s - p * Q;
                A f[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) f[j] = X(1, p * QQ + j * Q + k);
                line_iprod<A, N, Q>(Bs, f, [&](int o, A v) { X(2, (p * N + o) * Q + k) = v; });
            }
        }
        // third direction: 2 -> 3 (modes)
        if constexpr (SH == nirk::HEX) {
#pragma unroll 1
            for (int s = 0; s < N * N; ++s) {
                A f[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k) f[k] = X(2, s * Q + k);
                line_iprod<A, N, Q>(Bs, f, [&](int o, A v) { X(3, s * N + o) = v; });
            }
        } else if constexpr (SH == nirk::PRISM) {
            cfor<0, N>([&](auto cc) {
                constexpr int p = decltype(cc)::value, NC = N - p;
#pragma unroll 1
                for (int q = 0; q < N; ++q) {
                    constexpr int NEX = p == 0 ? 1 : 0;
                    A f[Q], ff[NEX > 0 ? NEX : 1][Q];
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        f[k] = X(2, (p * N + q) * Q + k);
                        if constexpr (NEX > 0) ff[0][k] = X(2, (N + q) * Q + k);
                    }
                    line_cls_iprod<A, N, Q, NC, NEX>(Bb + cls_off(N, Q, p), Bb, f, ff,
                                                      [&](int o, A v) { X(3, prism_m0(N, p, q) + o) = v; });
                }
            });
        } else {  // TET: the top vertex (0,0,1) collects pairs (0,1) and (1,0)
            cfor<0, N>([&](auto cc) {
                constexpr int c = decltype(cc)::value, NC = N - c;
#pragma unroll 1
                for (int p = 0; p <= c; ++p) {
                    constexpr int NEX = c == 0 ? 2 : 0;
                    A f[Q], ff[NEX > 0 ? NEX : 1][Q];
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        f[k] = X(2, tet_pair(N, p, c - p) * Q + k);
                        if constexpr (NEX > 0) {
                            ff[0][k] = X(2, tet_pair(N, 0, 1) * Q + k);
                            ff[1][k] = X(2, tet_pair(N, 1, 0) * Q + k);
                        }
                    }
                    line_cls_iprod<A, N, Q, NC, NEX>(Bc + cls_off(N, Q, c), Bc, f, ff,
                                                      [&](int o, A v) { X(3, tet_m0(N, p, c - p) + o) = v; });
                }
            });
        }
    } else {
        // first direction: 0 -> 1, t[p][j]
#pragma unroll 1
        for (int j = 0; j < Q; ++j) {
            A f[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = X(0, i + Q * j);
            line_iprod<A, N, Q>(Bs, f, [&](int o, A v) { X(1, o * Q + j) = v; });
        }
        if constexpr (SH == nirk::QUAD) {
#pragma unroll 1
            for (int p = 0; p < N; ++p) {
                A f[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) f[j] = X(1, p * Q + j);
                line_iprod<A, N, Q>(Bs, f, [&](int o, A v) { X(3, p * N + o) = v; });
            }
        } else {  // TRI: the collapsed vertex (0,1) also collects the p = 1 line
            cfor<0, N>([&](auto cc) {
                constexpr int p = decltype(cc)::value, NC = N - p;
                constexpr int NEX = p == 0 ? 1 : 0;
                A f[Q], ff[NEX > 0 ? NEX : 1][Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    f[j] = X(1, p * Q + j);
                    if constexpr (NEX > 0) ff[0][j] = X(1, Q + j);
                }
                line_cls_iprod<A, N, Q, NC, NEX>(Bb + cls_off(N, Q, p), Bb, f, ff,
                                                  [&](int o, A v) { X(3, tri_m0(N, p) + o) = v; });
            });
        }
    }
}

// Grid-stride over warps of 32 consecutive elements; lanes past the end take
// part in the tile transposes only.
template <int SH, int N, class T>
__global__ void __launch_bounds__(kThreads) k_helm_toe(ToeArgs a)
{
    using A = typename CT<T>::type;
    constexpr int Q = N + 1, NQ = nirk::npts(SH, Q), M = nirk::nmodes(SH, N);
    constexpr TabLayout L = layout(SH, N, Q);
    constexpr int TABN = (L.total + 1) & ~1;  // keeps the tiles 8-byte aligned
    extern __shared__ __align__(16) unsigned char smraw[];
    A *tab = reinterpret_cast<A *>(smraw);
    const A *tg = reinterpret_cast<const A *>(a.tab);
    for (int i = threadIdx.x; i < L.total; i += kThreads) tab[i] = tg[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    A *tile = tab + TABN + warp * 32 * kTile;
    const size_t nth = (size_t)gridDim.x * kThreads;
    const size_t gtid = (size_t)blockIdx.x * kThreads + threadIdx.x;
    const Scr<A, NQ> X{reinterpret_cast<A *>(a.scr) + gtid, (unsigned)nth};
    const T *in = reinterpret_cast<const T *>(a.in);
    T *out = reinterpret_cast<T *>(a.out);
    const T *geo = reinterpret_cast<const T *>(a.geo);
    const A lam = A(a.lambda);
    for (long long base = (long long)blockIdx.x * kThreads + warp * 32; base < a.nelem; base += (long long)nth) {
        const long long e = base + lane;
        const int nv = (int)(a.nelem - base < 32 ? a.nelem - base : 32);  // valid elements of this warp
        // coefficients: 32 rows of the [E][M] array -> scratch array 4 of each lane
#pragma unroll 1
        for (int c0 = 0; c0 < M; c0 += 32) {
            if (c0 + lane < M)
                for (int r = 0; r < nv; ++r) tile[r * kTile + lane] = to_c(in[(base + r) * M + c0 + lane]);
            __syncwarp();
            const int w = M - c0 < 32 ? M - c0 : 32;
            for (int m = 0; m < w; ++m) X(4, c0 + m) = tile[lane * kTile + m];
            __syncwarp();
        }
        if (lane < nv) helm_element<SH, N, T, A>(tab, X, geo, a.geo_pp, e, lam);
        // result: scratch array 3 -> 32 rows of the output
#pragma unroll 1
        for (int c0 = 0; c0 < M; c0 += 32) {
            const int w = M - c0 < 32 ? M - c0 : 32;
            for (int m = 0; m < w; ++m) tile[lane * kTile + m] = X(3, c0 + m);
            __syncwarp();
            if (c0 + lane < M)
                for (int r = 0; r < nv; ++r) put(tile[r * kTile + lane], &out[(base + r) * M + c0 + lane]);
            __syncwarp();
        }
    }
}

// Dynamic shared memory of one instantiation: the tables plus 4 warp tiles.
template <int SH, int N, class A>
constexpr int toe_smem()
{
    return (((layout(SH, N, N + 1).total + 1) & ~1) + (kThreads / 32) * 32 * kTile) * (int)sizeof(A);
}

}  // namespace nirt
