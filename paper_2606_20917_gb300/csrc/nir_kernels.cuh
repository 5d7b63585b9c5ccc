// nir_kernels.cuh -- sum-factorised spectral/hp elemental operators for sm_103a.
//
// One kernel template covers every (shape, order, precision, operator):
//   BwdTrans             u  = B u_hat                       (Eqs. bwdsumfachex, bwdsumfactet)
//   IProductWRTBase      u_hat = B^T W f                     (Eqs. iprodhex, iprodtet)
//   PhysDeriv            du/dx_l = sum_j (d eta_j/d x_l) D_eta_j u   (Eqs. physderiv, stdderiv)
//   IProductWRTDerivBase sum_l (D_xl B)^T W f_l              (the test_grad operation, Sec. 3.1)
//   mass                 B^T W B u_hat
//   Helmholtz            B^T [ sum_ij D_i^T G_ij D_j + lambda W ] B u_hat   (Eqs. weakmatrixhelm, laplacian)
// where G_ij = W sum_l (d eta_i/d x_l)(d eta_j/d x_l) folds the Jacobian, the
// collapsed-coordinate chain rule (D_xi = Lambda(d eta/d xi) D_eta, Sec. 2.2)
// and the weights into one symmetric per-point tensor.
//
// Execution model.  A CTA owns a group of EPB consecutive elements and keeps
// all of their intermediate tensors in shared memory (Sec. 3.3's "threading
// over coefficients" strategy with the temporaries in shared memory).  Every
// stage maps work items to threads with the element index fastest, so the
// lanes of a warp work on different elements at the same structural index:
//   * shared-memory addresses differ by the per-element stride S, which is odd,
//     so a warp's accesses are bank-conflict free for 32- and 64-bit types;
//   * basis/derivative table reads are warp-uniform (broadcast);
//   * the ragged loops of the collapsed shapes (q < N-p, r < N-p-q) are split
//     into compile-time classes, so no lane runs predicated-off iterations.
// Contractions are written as "pencils": a work item loads one 1-D line of
// NIN values into registers and produces NOUT outputs, so each input is read
// from shared memory once per pencil (Sec. 2.2's sum-factorisation, one
// direction per stage).  Collapsed vertex/edge modes whose eta1 (eta2) factor is
// not a polynomial in xi enter as one extra input column (BwdTrans) or one
// extra input line feeding a single output (the transposed inner products).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "nir_layout.h"

namespace nirk {

enum Op { OP_BWD = 0, OP_IPROD = 1, OP_PHYSDERIV = 2, OP_IPROD_DERIV = 3, OP_MASS = 4, OP_HELM = 5 };

struct KArgs {
    const void *in0, *in1, *in2;  // coefficients [E][M] or physical fields [E][Nq]
    void *out0, *out1, *out2;
    const void *geo;              // G (ngeo) or d eta/d x + W (nlam); storage type
    const void *tab;              // table blob in the compute type
    long long nelem;
    double lambda;
    int geo_pp;                   // 1: per point, 32-element interleaved; 0: per element
    int pad;
};

template <class T> struct CT { using type = float; };
template <> struct CT<double> { using type = double; };

__device__ __forceinline__ double to_a(double v, double) { return v; }
__device__ __forceinline__ float to_a(float v, float) { return v; }
__device__ __forceinline__ float to_a(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ void from_a(double v, double *p) { *p = v; }
__device__ __forceinline__ void from_a(float v, float *p) { *p = v; }
__device__ __forceinline__ void from_a(float v, __nv_bfloat16 *p) { *p = __float2bfloat16_rn(v); }

template <class A> __device__ __forceinline__ A fmaa(A a, A b, A c) { return fma(a, b, c); }

template <int I, int E, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    if constexpr (I < E) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, E>(f);
    }
}

constexpr int odd_stride(int n) { return (n % 2 == 0) ? n + 1 : n; }

// One pencil stage over EPB * per_e work items.  out_o = sum_r T(o,r) x_r
// (+ sum_r TX(r) xx_r when o == OEX).  `rot` rotates the thread->item map so
// consecutive barrier-free stages spread their tails over different threads.
// The table functors receive an offset z that is always 0 but is produced
// inside the loop, so the compiler keeps the (warp-broadcast) table loads in
// the loop instead of hoisting NIN x NOUT values into registers for threads
// that only run one or two iterations.
template <class A, int NIN, int NOUT, int NEX, int OEX, int EPB, int NT, class LD, class TB, class LDX,
          class TBX, class ST>
__device__ __forceinline__ void pencils(int per_e, int &rot, LD ld, TB tb, LDX ldx, TBX tbx, ST st)
{
    // The bound is hidden from the compiler: with few elements per CTA it can
    // otherwise prove the loop runs at most once and straight-lines whole stages
    // into code that needs several times the registers.
    int total = per_e * EPB;
    asm volatile("mov.u32 %0, %0;" : "+r"(total));
    int w = (int)threadIdx.x - (rot % NT);
    if (w < 0) w += NT;
    for (; w < total; w += NT) {
        const int e = w % EPB;
        const int s = w / EPB;
        int z;
        asm volatile("mov.u32 %0, 0;" : "=r"(z));
        A x[NIN];
        ld(e, s, x);
        A xx[NEX > 0 ? NEX : 1];
        if constexpr (NEX > 0) ldx(e, s, xx);
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            A acc = A(0);
#pragma unroll
            for (int r = 0; r < NIN; ++r) acc = fmaa(tb(z, o, r), x[r], acc);
            if constexpr (NEX > 0) {
                if (o == OEX) {
#pragma unroll
                    for (int r = 0; r < NEX; ++r) acc = fmaa(tbx(z, r), xx[r], acc);
                }
            }
            st(e, s, o, acc);
        }
    }
    rot += total;
}

struct NoX {
    template <class A> __device__ void operator()(int, int, A *) const {}
};
struct NoTX {
    __device__ int operator()(int, int) const { return 0; }
};

template <class A, int NIN, int NOUT, int EPB, int NT, class LD, class TB, class ST>
__device__ __forceinline__ void pencils0(int per_e, int &rot, LD ld, TB tb, ST st)
{
    pencils<A, NIN, NOUT, 0, 0, EPB, NT>(per_e, rot, ld, tb, NoX{}, [](int, int) { return A(0); }, st);
}

// ---------------------------------------------------------------------------
// Modal <-> quadrature stages per shape.  Buffers: element e, index i at
// buf[e*S + i].  bwd: p0 (modes) -> p1 -> p2 (-> p3) (points);
// iprod: p0 (points) -> p1 (-> p2) -> last (modes).
// ---------------------------------------------------------------------------
template <int SH, int N, int Q, class A, int EPB, int NT, int S>
struct Modal {
    static constexpr TabLayout L = layout(SH, N, Q);
    static constexpr int QQ = Q * Q;

    static __device__ __forceinline__ void bwd(const A *tab, A *p0, A *p1, A *p2, A *p3)
    {
        const A *Ba = tab + L.Ba;
        int rot = 0;
        auto tBa = [=](int z, int o, int r) { return Ba[z + o * N + r]; };
        if constexpr (SH == QUAD || SH == TRI) {
            if constexpr (SH == QUAD) {
                // t1[p][j] = sum_q u[p][q] psiA_q(z_j)
                pencils0<A, N, Q, EPB, NT>(N, rot,
                    [=](int e, int s, A *x) { const A *b = p0 + e * S + s * N;
#pragma unroll
                        for (int r = 0; r < N; ++r) x[r] = b[r]; },
                    tBa, [=](int e, int s, int o, A v) { p1[e * S + s * Q + o] = v; });
            } else {
                // t1[p][j] = sum_{q<N-p} u[m(p,q)] psiB_pq(z_j) (+ the collapsed vertex (0,1) for p = 1)
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nin = nc + (p == 1 ? 1 : 0);
                    const A *Bp = tab + L.Bb + cls_off(N, Q, p);
                    const A *B0 = tab + L.Bb;
                    pencils0<A, nin, Q, EPB, NT>(1, rot,
                        [=](int e, int, A *x) { const A *b = p0 + e * S + tri_m0(N, p);
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r];
                            if constexpr (p == 1) x[nc] = p0[e * S + 1]; },
                        [=](int z, int o, int r) { return (p == 1 && r == nc) ? B0[z + o * N + 1] : Bp[z + o * nc + r]; },
                        [=](int e, int, int o, A v) { p1[e * S + p * Q + o] = v; });
                });
            }
            __syncthreads();
            // u[i + Q j] = sum_p psiA_p(z_i) t1[p][j]
            pencils0<A, N, Q, EPB, NT>(Q, rot,
                [=](int e, int s, A *x) { const A *b = p1 + e * S + s;
#pragma unroll
                    for (int r = 0; r < N; ++r) x[r] = b[r * Q]; },
                tBa, [=](int e, int s, int o, A v) { p2[e * S + o + Q * s] = v; });
            __syncthreads();
        } else {
            // ---- stage 1: contract the third mode index r -> k
            if constexpr (SH == HEX) {
                pencils0<A, N, Q, EPB, NT>(N * N, rot,
                    [=](int e, int s, A *x) { const A *b = p0 + e * S + s * N;
#pragma unroll
                        for (int r = 0; r < N; ++r) x[r] = b[r]; },
                    tBa, [=](int e, int s, int o, A v) { p1[e * S + s * Q + o] = v; });
            } else if constexpr (SH == PRISM) {
                // t1[p][q][k] = sum_{r<N-p} u[m(p,q,r)] psiB_pr(z3_k) (+ collapsed edge (0,q,1) for p = 1)
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nin = nc + (p == 1 ? 1 : 0);
                    const A *Bp = tab + L.Bb + cls_off(N, Q, p);
                    const A *B0 = tab + L.Bb;
                    pencils0<A, nin, Q, EPB, NT>(N, rot,
                        [=](int e, int q, A *x) { const A *b = p0 + e * S + prism_m0(N, p, q);
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r];
                            if constexpr (p == 1) x[nc] = p0[e * S + prism_m0(N, 0, q) + 1]; },
                        [=](int z, int o, int r) { return (p == 1 && r == nc) ? B0[z + o * N + 1] : Bp[z + o * nc + r]; },
                        [=](int e, int q, int o, A v) { p1[e * S + (p * N + q) * Q + o] = v; });
                });
            } else {  // TET
                // t1[pair(p,q)][k] = sum_{r<N-p-q} u[m(p,q,r)] psiB_(p+q)r(z3_k); the collapsed
                // top vertex (0,0,1) also feeds pairs (0,1) and (1,0) through psiB_01(z3_k).
                sfor<0, N>([&](auto cc) {
                    constexpr int c = decltype(cc)::value;
                    constexpr int nc = N - c;
                    constexpr int nin = nc + (c == 1 ? 1 : 0);
                    const A *Bc = tab + L.Bc + cls_off(N, Q, c);
                    const A *B0 = tab + L.Bc;
                    pencils0<A, nin, Q, EPB, NT>(c + 1, rot,
                        [=](int e, int p, A *x) { const A *b = p0 + e * S + tet_m0(N, p, c - p);
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r];
                            if constexpr (c == 1) x[nc] = p0[e * S + 1]; },
                        [=](int z, int o, int r) { return (c == 1 && r == nc) ? B0[z + o * N + 1] : Bc[z + o * nc + r]; },
                        [=](int e, int p, int o, A v) { p1[e * S + tet_pair(N, p, c - p) * Q + o] = v; });
                });
            }
            __syncthreads();
            // ---- stage 2: contract q -> j
            if constexpr (SH == HEX || SH == PRISM) {
                pencils0<A, N, Q, EPB, NT>(N * Q, rot,
                    [=](int e, int s, A *x) { const int p = s / Q, k = s - p * Q;
                        const A *b = p1 + e * S + p * N * Q + k;
#pragma unroll
                        for (int r = 0; r < N; ++r) x[r] = b[r * Q]; },
                    tBa, [=](int e, int s, int o, A v) { const int p = s / Q, k = s - p * Q;
                        p2[e * S + (p * Q + o) * Q + k] = v; });
            } else {  // TET: t2[p][j][k] = sum_{q<N-p} psiB_pq(z2_j) t1[pair(p,q)][k] (+ edge (0,1,.) for p = 1)
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nin = nc + (p == 1 ? 1 : 0);
                    const A *Bp = tab + L.Bb + cls_off(N, Q, p);
                    const A *B0 = tab + L.Bb;
                    pencils0<A, nin, Q, EPB, NT>(Q, rot,
                        [=](int e, int k, A *x) { const A *b = p1 + e * S + tet_pair(N, p, 0) * Q + k;
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r * Q];
                            if constexpr (p == 1) x[nc] = p1[e * S + tet_pair(N, 0, 1) * Q + k]; },
                        [=](int z, int o, int r) { return (p == 1 && r == nc) ? B0[z + o * N + 1] : Bp[z + o * nc + r]; },
                        [=](int e, int k, int o, A v) { p2[e * S + (p * Q + o) * Q + k] = v; });
                });
            }
            __syncthreads();
            // ---- stage 3: contract p -> i; u[i + Q j + Q^2 k]
            pencils0<A, N, Q, EPB, NT>(QQ, rot,
                [=](int e, int s, A *x) { const int k = s / Q, j = s - k * Q;
                    const A *b = p2 + e * S + j * Q + k;
#pragma unroll
                    for (int r = 0; r < N; ++r) x[r] = b[r * QQ]; },
                tBa, [=](int e, int s, int o, A v) { p3[e * S + o + Q * s] = v; });
            __syncthreads();
        }
    }

    // Transposed stages: p0 (points, weights already applied) -> modes in `last`.
    static __device__ __forceinline__ void iprod(const A *tab, A *p0, A *p1, A *p2, A *last)
    {
        const A *Ba = tab + L.Ba;
        int rot = 0;
        auto tBaT = [=](int z, int o, int r) { return Ba[z + r * N + o]; };
        if constexpr (SH == QUAD || SH == TRI) {
            // t1[p][j] = sum_i psiA_p(z_i) f[i + Q j]
            pencils0<A, Q, N, EPB, NT>(Q, rot,
                [=](int e, int s, A *x) { const A *b = p0 + e * S + Q * s;
#pragma unroll
                    for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                tBaT, [=](int e, int s, int o, A v) { p1[e * S + o * Q + s] = v; });
            __syncthreads();
            if constexpr (SH == QUAD) {
                pencils0<A, Q, N, EPB, NT>(N, rot,
                    [=](int e, int s, A *x) { const A *b = p1 + e * S + s * Q;
#pragma unroll
                        for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                    tBaT, [=](int e, int s, int o, A v) { last[e * S + s * N + o] = v; });
            } else {
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nex = (p == 0 && N > 1) ? Q : 0;
                    const A *Bp = tab + L.Bb + cls_off(N, Q, p);
                    const A *B0 = tab + L.Bb;
                    pencils<A, Q, nc, nex, 1, EPB, NT>(1, rot,
                        [=](int e, int, A *x) { const A *b = p1 + e * S + p * Q;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                        [=](int z, int o, int r) { return Bp[z + r * nc + o]; },
                        [=](int e, int, A *xx) { const A *b = p1 + e * S + 1 * Q;   // the (0,1) vertex: p = 1 line
#pragma unroll
                            for (int r = 0; r < nex; ++r) xx[r] = b[r]; },
                        [=](int z, int r) { return B0[z + r * N + 1]; },
                        [=](int e, int, int o, A v) { last[e * S + tri_m0(N, p) + o] = v; });
                });
            }
            __syncthreads();
        } else {
            // ---- transpose of stage 3: t2[p][j][k] = sum_i psiA_p(z_i) f[i + Q j + Q^2 k]
            pencils0<A, Q, N, EPB, NT>(QQ, rot,
                [=](int e, int s, A *x) { const A *b = p0 + e * S + Q * s;
#pragma unroll
                    for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                tBaT, [=](int e, int s, int o, A v) { const int k = s / Q, j = s - k * Q;
                    p1[e * S + o * QQ + j * Q + k] = v; });
            __syncthreads();
            // ---- transpose of stage 2
            if constexpr (SH == HEX || SH == PRISM) {
                pencils0<A, Q, N, EPB, NT>(N * Q, rot,
                    [=](int e, int s, A *x) { const int p = s / Q, k = s - p * Q;
                        const A *b = p1 + e * S + p * QQ + k;
#pragma unroll
                        for (int r = 0; r < Q; ++r) x[r] = b[r * Q]; },
                    tBaT, [=](int e, int s, int o, A v) { const int p = s / Q, k = s - p * Q;
                        p2[e * S + (p * N + o) * Q + k] = v; });
            } else {  // TET: t1[pair(p,q)][k] = sum_j psiB_pq(z2_j) t2[p][j][k]; edge (0,1,.) also gets p = 1
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nex = (p == 0 && N > 1) ? Q : 0;
                    const A *Bp = tab + L.Bb + cls_off(N, Q, p);
                    const A *B0 = tab + L.Bb;
                    pencils<A, Q, nc, nex, 1, EPB, NT>(Q, rot,
                        [=](int e, int k, A *x) { const A *b = p1 + e * S + p * QQ + k;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r * Q]; },
                        [=](int z, int o, int r) { return Bp[z + r * nc + o]; },
                        [=](int e, int k, A *xx) { const A *b = p1 + e * S + 1 * QQ + k;
#pragma unroll
                            for (int r = 0; r < nex; ++r) xx[r] = b[r * Q]; },
                        [=](int z, int r) { return B0[z + r * N + 1]; },
                        [=](int e, int k, int o, A v) { p2[e * S + (tet_pair(N, p, 0) + o) * Q + k] = v; });
                });
            }
            __syncthreads();
            // ---- transpose of stage 1
            if constexpr (SH == HEX) {
                pencils0<A, Q, N, EPB, NT>(N * N, rot,
                    [=](int e, int s, A *x) { const A *b = p2 + e * S + s * Q;
#pragma unroll
                        for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                    tBaT, [=](int e, int s, int o, A v) { last[e * S + s * N + o] = v; });
            } else if constexpr (SH == PRISM) {
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nex = (p == 0 && N > 1) ? Q : 0;
                    const A *Bp = tab + L.Bb + cls_off(N, Q, p);
                    const A *B0 = tab + L.Bb;
                    pencils<A, Q, nc, nex, 1, EPB, NT>(N, rot,
                        [=](int e, int q, A *x) { const A *b = p2 + e * S + (p * N + q) * Q;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                        [=](int z, int o, int r) { return Bp[z + r * nc + o]; },
                        [=](int e, int q, A *xx) { const A *b = p2 + e * S + (1 * N + q) * Q;
#pragma unroll
                            for (int r = 0; r < nex; ++r) xx[r] = b[r]; },
                        [=](int z, int r) { return B0[z + r * N + 1]; },
                        [=](int e, int q, int o, A v) { last[e * S + prism_m0(N, p, q) + o] = v; });
                });
            } else {  // TET: the top vertex (0,0,1) collects pairs (0,1) and (1,0)
                sfor<0, N>([&](auto cc) {
                    constexpr int c = decltype(cc)::value;
                    constexpr int nc = N - c;
                    constexpr int nex = (c == 0 && N > 1) ? 2 * Q : 0;
                    const A *Bc = tab + L.Bc + cls_off(N, Q, c);
                    const A *B0 = tab + L.Bc;
                    pencils<A, Q, nc, nex, 1, EPB, NT>(c + 1, rot,
                        [=](int e, int p, A *x) { const A *b = p2 + e * S + tet_pair(N, p, c - p) * Q;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                        [=](int z, int o, int r) { return Bc[z + r * nc + o]; },
                        [=](int e, int, A *xx) {
                            const A *b1 = p2 + e * S + tet_pair(N, 0, 1) * Q;
                            const A *b2 = p2 + e * S + tet_pair(N, 1, 0) * Q;
#pragma unroll
                            for (int r = 0; r < nex / 2; ++r) { xx[r] = b1[r]; xx[r + nex / 2] = b2[r]; } },
                        [=](int z, int r) { return B0[z + (r % Q) * N + 1]; },
                        [=](int e, int p, int o, A v) { last[e * S + tet_m0(N, p, c - p) + o] = v; });
                });
            }
            __syncthreads();
        }
    }
};

// ---------------------------------------------------------------------------
// Geometry access.  Per-point arrays are interleaved by 32 elements:
// value c of point n of element e at (((e >> 5) * NQ + n) * NG + c) * 32 + (e & 31).
// Per-element arrays are [E][NG] and exclude the reference weight, which is
// multiplied in here for the W component.
// ---------------------------------------------------------------------------
template <class T, class A, int NQ, int NG>
struct Geo {
    const T *g;
    const A *wq;
    int pp;
    __device__ __forceinline__ A get(long long e, int n, int c) const
    {
        if (pp) return to_a(g[((((e >> 5) * NQ + n) * NG + c) << 5) + (e & 31)], A());
        A v = to_a(g[e * NG + c], A());
        return (c == NG - 1) ? v * wq[n] : v;
    }
    // scale of the metric (non-W) components: 1 per point, wq[n] per element
    __device__ __forceinline__ A gscale(int n) const { return pp ? A(1) : wq[n]; }
};

// Default elements per CTA: fill about 110 KB (FP64) or 56 KB (FP32/BF16) of
// shared memory with the operator's buffers.  EPB_ > 0 overrides it (the
// autotuner picks among compiled alternatives).
template <int SH, int N, int Q, class T, int OP, int EPB_ = 0>
struct Config {
    using A = typename CT<T>::type;
    static constexpr int D = dim(SH);
    static constexpr int NQ = npts(SH, Q);
    static constexpr int M = nmodes(SH, N);
    static constexpr int S = odd_stride(NQ);
    static constexpr int NBUF = (OP == OP_BWD || OP == OP_IPROD || OP == OP_MASS) ? 2 : D + 1;
    static constexpr int TABN = layout(SH, N, Q).total;
    static constexpr int TABB = ((TABN * (int)sizeof(A) + 15) / 16) * 16;
    static constexpr int budget = sizeof(A) == 8 ? 110 * 1024 : 56 * 1024;
    static constexpr int per_elem = NBUF * S * (int)sizeof(A);
    static constexpr int raw = (budget - TABB) / per_elem;
    static constexpr int EPB_DEF = raw >= 64 ? 64 : raw >= 32 ? 32 : raw >= 16 ? 16 : raw >= 8 ? 8 : raw >= 4 ? 4
                                 : raw >= 2 ? 2 : 1;
    static constexpr int EPB = EPB_ > 0 ? EPB_ : EPB_DEF;
    static constexpr int NT = 256;
    static constexpr int BUFB = NBUF * EPB * S * (int)sizeof(A);
    static constexpr int SMEM = TABB + BUFB;
};

template <class T, class A, int LEN, int S, int NT>
__device__ __forceinline__ void gload(const T *__restrict__ g, long long e0, int ne, A *sm)
{
    const T *src = g + e0 * LEN;
    for (int i = threadIdx.x; i < ne * LEN; i += NT) {
        const int e = i / LEN, m = i - e * LEN;
        sm[e * S + m] = to_a(__ldg(src + i), A());
    }
}

template <class T, class A, int LEN, int S, int NT>
__device__ __forceinline__ void gstore(T *__restrict__ g, long long e0, int ne, const A *sm)
{
    T *dst = g + e0 * LEN;
    for (int i = threadIdx.x; i < ne * LEN; i += NT) {
        const int e = i / LEN, m = i - e * LEN;
        from_a(sm[e * S + m], dst + i);
    }
}

// d u / d eta_dir at point (i,j,k) by collocation (Eq. stdderiv).
template <class A, int Q, int D>
__device__ __forceinline__ A dcol(const A *Ue, const A *Dm, int dir, int i, int j, int k)
{
    A acc = A(0);
    if (dir == 0) {
        const A *row = Dm + i * Q;
        const A *u = Ue + Q * (j + Q * k);
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fmaa(row[r], u[r], acc);
    } else if (dir == 1) {
        const A *row = Dm + j * Q;
        const A *u = Ue + i + Q * Q * k;
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fmaa(row[r], u[r * Q], acc);
    } else {
        const A *row = Dm + k * Q;
        const A *u = Ue + i + Q * j;
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fmaa(row[r], u[r * Q * Q], acc);
    }
    return acc;
}

// sum_dir D_dir^T v_dir at point (i,j,k): transposed collocation.
template <class A, int Q, int D>
__device__ __forceinline__ A dcolT(const A *V0, const A *V1, const A *V2, const A *D0, const A *D1,
                                    const A *D2, int i, int j, int k)
{
    A acc = A(0);
    {
        const A *v = V0 + Q * (j + Q * k);
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fmaa(D0[r * Q + i], v[r], acc);
    }
    {
        const A *v = V1 + i + Q * Q * k;
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fmaa(D1[r * Q + j], v[r * Q], acc);
    }
    if constexpr (D == 3) {
        const A *v = V2 + i + Q * j;
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fmaa(D2[r * Q + k], v[r * Q * Q], acc);
    }
    return acc;
}

// Helmholtz metric stage: v_i = sum_j G_ij du_j at every point of the group.
// PP: factors stored per point (true) or per element times the reference
// weight (false), resolved at compile time so no scale is applied per point.
template <bool PP, int D, int Q, int NQ, int NG, int EPB, int NT, class T, class A>
__device__ __forceinline__ void helm_metric(const Geo<T, A, NQ, NG> &geo, long long e0, const A *D0, const A *D1,
                                            const A *D2, int S, A *B0, A *B1, A *B2, A *B3)
{
    for (int w = threadIdx.x; w < EPB * NQ; w += NT) {
        const int e = w % EPB, n = w / EPB;
        const int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
        const A *Ue = B0 + e * S;
        const long long eg = e0 + e;
        A u0 = dcol<A, Q, D>(Ue, D0, 0, i, j, k);
        A u1 = dcol<A, Q, D>(Ue, D1, 1, i, j, k);
        A u2 = A(0);
        if constexpr (D == 3) u2 = dcol<A, Q, D>(Ue, D2, 2, i, j, k);
        if constexpr (!PP) {
            const A sc = geo.wq[n];
            u0 *= sc;
            u1 *= sc;
            if constexpr (D == 3) u2 *= sc;
        }
        if constexpr (D == 2) {
            const A g00 = geo.get(eg, n, 0), g01 = geo.get(eg, n, 1), g11 = geo.get(eg, n, 2);
            B1[e * S + n] = fmaa(g00, u0, g01 * u1);
            B2[e * S + n] = fmaa(g01, u0, g11 * u1);
        } else {
            const A g00 = geo.get(eg, n, 0), g01 = geo.get(eg, n, 1), g02 = geo.get(eg, n, 2);
            const A g11 = geo.get(eg, n, 3), g12 = geo.get(eg, n, 4), g22 = geo.get(eg, n, 5);
            B1[e * S + n] = fmaa(g00, u0, fmaa(g01, u1, g02 * u2));
            B2[e * S + n] = fmaa(g01, u0, fmaa(g11, u1, g12 * u2));
            B3[e * S + n] = fmaa(g02, u0, fmaa(g12, u1, g22 * u2));
        }
    }
}

// One group of ne (<= EPB) elements starting at e0: the whole operator.
// tab: the block's tables in shared memory; buf: NBUF * EPB * S values.
template <int SH, int N, int Q, class T, int OP, int EPB_>
__device__ __forceinline__ void run_group(const KArgs &a, const typename CT<T>::type *tab,
                                          typename CT<T>::type *buf, long long e0, int ne)
{
    using C = Config<SH, N, Q, T, OP, EPB_>;
    using A = typename C::A;
    constexpr int D = C::D, NQ = C::NQ, M = C::M, S = C::S, EPB = C::EPB, NT = C::NT;
    constexpr TabLayout L = layout(SH, N, Q);
    constexpr int NG = (OP == OP_PHYSDERIV || OP == OP_IPROD_DERIV) ? nlam(SH) : ngeo(SH);
    using MD = Modal<SH, N, Q, A, EPB, NT, S>;
    A *B0 = buf, *B1 = buf + EPB * S, *B2 = buf + 2 * EPB * S, *B3 = buf + 3 * EPB * S;
    const A *D0 = tab + L.D1, *D1 = tab + L.D2, *D2 = tab + L.D3;
    const Geo<T, A, NQ, NG> geo{reinterpret_cast<const T *>(a.geo), tab + L.wq, a.geo_pp};

    if constexpr (OP == OP_BWD) {
        gload<T, A, M, S, NT>(reinterpret_cast<const T *>(a.in0), e0, ne, B0);
        __syncthreads();
        if constexpr (D == 2) {
            MD::bwd(tab, B0, B1, B0, nullptr);
            gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, B0);
        } else {
            MD::bwd(tab, B0, B1, B0, B1);
            gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, B1);
        }
    } else if constexpr (OP == OP_IPROD || OP == OP_MASS) {
        A *P = B0;
        if constexpr (OP == OP_IPROD) {
            gload<T, A, NQ, S, NT>(reinterpret_cast<const T *>(a.in0), e0, ne, B0);
            __syncthreads();
        } else {
            gload<T, A, M, S, NT>(reinterpret_cast<const T *>(a.in0), e0, ne, B0);
            __syncthreads();
            if constexpr (D == 2) MD::bwd(tab, B0, B1, B0, nullptr);
            else { MD::bwd(tab, B0, B1, B0, B1); P = B1; }
        }
        for (int w = threadIdx.x; w < EPB * NQ; w += NT) {
            const int e = w % EPB, n = w / EPB;
            P[e * S + n] *= geo.get(e0 + e, n, NG - 1);
        }
        __syncthreads();
        A *O = (P == B0) ? B1 : B0;
        if constexpr (D == 2) {
            MD::iprod(tab, P, O, nullptr, P);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, P);
        } else {
            MD::iprod(tab, P, O, P, O);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, O);
        }
    } else if constexpr (OP == OP_PHYSDERIV) {
        gload<T, A, NQ, S, NT>(reinterpret_cast<const T *>(a.in0), e0, ne, B0);
        __syncthreads();
        A *Vs[3] = {B1, B2, B3};
        for (int w = threadIdx.x; w < EPB * NQ; w += NT) {
            const int e = w % EPB, n = w / EPB;
            const int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
            const A *Ue = B0 + e * S;
            A du[3];
            du[0] = dcol<A, Q, D>(Ue, D0, 0, i, j, k);
            du[1] = dcol<A, Q, D>(Ue, D1, 1, i, j, k);
            if constexpr (D == 3) du[2] = dcol<A, Q, D>(Ue, D2, 2, i, j, k);
#pragma unroll
            for (int l = 0; l < D; ++l) {
                A s = A(0);
#pragma unroll
                for (int jj = 0; jj < D; ++jj) s = fmaa(geo.get(e0 + e, n, jj * D + l), du[jj], s);
                Vs[l][e * S + n] = s;
            }
        }
        __syncthreads();
        gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, B1);
        gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(a.out1), e0, ne, B2);
        if constexpr (D == 3) gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(a.out2), e0, ne, B3);
    } else if constexpr (OP == OP_IPROD_DERIV) {
        gload<T, A, NQ, S, NT>(reinterpret_cast<const T *>(a.in0), e0, ne, B1);
        gload<T, A, NQ, S, NT>(reinterpret_cast<const T *>(a.in1), e0, ne, B2);
        if constexpr (D == 3) gload<T, A, NQ, S, NT>(reinterpret_cast<const T *>(a.in2), e0, ne, B3);
        __syncthreads();
        A *Vs[3] = {B1, B2, B3};
        // g_j = W sum_l (d eta_j / d x_l) f_l, in place
        for (int w = threadIdx.x; w < EPB * NQ; w += NT) {
            const int e = w % EPB, n = w / EPB;
            A f[3];
#pragma unroll
            for (int l = 0; l < D; ++l) f[l] = Vs[l][e * S + n];
            const A Wn = geo.get(e0 + e, n, NG - 1);
#pragma unroll
            for (int jj = 0; jj < D; ++jj) {
                A s = A(0);
#pragma unroll
                for (int l = 0; l < D; ++l) s = fmaa(geo.get(e0 + e, n, jj * D + l), f[l], s);
                Vs[jj][e * S + n] = Wn * s;
            }
        }
        __syncthreads();
        for (int w = threadIdx.x; w < EPB * NQ; w += NT) {
            const int e = w % EPB, n = w / EPB;
            const int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
            B0[e * S + n] = dcolT<A, Q, D>(B1 + e * S, B2 + e * S, B3 + e * S, D0, D1, D2, i, j, k);
        }
        __syncthreads();
        if constexpr (D == 2) {
            MD::iprod(tab, B0, B1, nullptr, B2);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, B2);
        } else {
            MD::iprod(tab, B0, B1, B2, B1);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, B1);
        }
    } else {  // OP_HELM
        gload<T, A, M, S, NT>(reinterpret_cast<const T *>(a.in0), e0, ne, B1);
        __syncthreads();
        if constexpr (D == 2) MD::bwd(tab, B1, B2, B0, nullptr);
        else MD::bwd(tab, B1, B2, B1, B0);
        // v_i = sum_j G_ij du_j  (G includes W and the chain rule)
        if (a.geo_pp) helm_metric<true, D, Q, NQ, NG, EPB, NT>(geo, e0, D0, D1, D2, S, B0, B1, B2, B3);
        else helm_metric<false, D, Q, NQ, NG, EPB, NT>(geo, e0, D0, D1, D2, S, B0, B1, B2, B3);
        __syncthreads();
        // y = sum_i D_i^T v_i + lambda W u, in place over u
        const A lam = A(a.lambda);
        for (int w = threadIdx.x; w < EPB * NQ; w += NT) {
            const int e = w % EPB, n = w / EPB;
            const int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
            const A acc = dcolT<A, Q, D>(B1 + e * S, B2 + e * S, B3 + e * S, D0, D1, D2, i, j, k);
            B0[e * S + n] = fmaa(lam * geo.get(e0 + e, n, NG - 1), B0[e * S + n], acc);
        }
        __syncthreads();
        if constexpr (D == 2) {
            MD::iprod(tab, B0, B1, nullptr, B2);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, B2);
        } else {
            MD::iprod(tab, B0, B1, B2, B1);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(a.out0), e0, ne, B1);
        }
    }
    __syncthreads();
}

// Persistent single-block kernel: CTAs stride over the element groups.
template <int SH, int N, int Q, class T, int OP, int EPB_ = 0>
__global__ void __launch_bounds__(256) k_elem(KArgs a)
{
    using C = Config<SH, N, Q, T, OP, EPB_>;
    using A = typename C::A;
    constexpr int EPB = C::EPB, NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *tab = reinterpret_cast<A *>(smem_raw);
    A *buf = reinterpret_cast<A *>(smem_raw + C::TABB);
    {
        const A *gt = reinterpret_cast<const A *>(a.tab);
        for (int i = threadIdx.x; i < C::TABN; i += NT) tab[i] = gt[i];
    }
    __syncthreads();
    const long long ngroups = (a.nelem + EPB - 1) / EPB;
    for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const long long e0 = g * EPB;
        const int ne = (int)((a.nelem - e0) < EPB ? (a.nelem - e0) : EPB);
        run_group<SH, N, Q, T, OP, EPB_>(a, tab, buf, e0, ne);
    }
}

}  // namespace nirk
