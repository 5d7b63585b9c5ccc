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

// Values the compiler must treat as unknown (a loop bound it could otherwise
// prove small, a zero it could fold).  The stage code also compiles as host
// C++ (a CTA emulation that checks its shared-memory indexing and barriers);
// there both are plain assignments.
#ifdef __CUDA_ARCH__
#define NIR_OPAQUE(v) asm volatile("mov.u32 %0, %0;" : "+r"(v))
#define NIR_ZERO(v) asm volatile("mov.u32 %0, 0;" : "=r"(v))
#else
#define NIR_OPAQUE(v) ((void)(v))
#define NIR_ZERO(v) ((v) = 0)
#endif

// Loads of the metric.  Read once per apply; the paired-element form streams
// them with the evict-first policy (the L2 then keeps prefetched groups rather
// than consumed ones: 3-6 % on P = 4 hexes), while for the one-element form
// that policy costs up to a quarter on high-order and collapsed shapes (tet
// P = 8: 7.1 against 9.2 GDOF/s), so it keeps plain read-only loads.
#define NIR_METRIC_LD __ldg
#define NIR_METRIC_LD_PAIR __ldcs

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
    int pf;                       // FP32/BF16 Helmholtz: 1 = bulk-prefetch the group's metric into L2
    int *err;                     // device error word (bounded waits that gave up set it)
    int nfields;                  // Helmholtz: fields in0..in2 -> out0..out2 sharing the operator (1..3)
    int nodal;                    // quad/hex: coefficients are GLL-Lagrange nodal values
};

// Field f of a multi-field Helmholtz call.
__device__ __forceinline__ const void *field_in(const KArgs &a, int f) { return f == 0 ? a.in0 : f == 1 ? a.in1 : a.in2; }
__device__ __forceinline__ void *field_out(const KArgs &a, int f) { return f == 0 ? a.out0 : f == 1 ? a.out1 : a.out2; }

template <class T> struct CT { using type = float; };
template <> struct CT<double> { using type = double; };

__device__ __forceinline__ double to_a(double v, double) { return v; }
__device__ __forceinline__ float to_a(float v, float) { return v; }
__device__ __forceinline__ float to_a(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ void from_a(double v, double *p) { *p = v; }
__device__ __forceinline__ void from_a(float v, float *p) { *p = v; }
__device__ __forceinline__ void from_a(float v, __nv_bfloat16 *p) { *p = __float2bfloat16_rn(v); }

template <class A> __device__ __forceinline__ A fmaa(A a, A b, A c) { return fma(a, b, c); }

// Two elements' values in one lane (element 2e in x, 2e+1 in y): the value
// type of the paired FP32/BF16 Helmholtz, whose threads each carry one pencil
// of two elements.  The stage code is shared with the one-element form; the
// tables stay scalar, and each table coefficient multiplies both elements
// (one packed FP32x2 multiply-add on sm_100 and later).
struct F2 {
    float x, y;
    F2() = default;
    __device__ __forceinline__ constexpr F2(float v) : x(v), y(v) {}
    __device__ __forceinline__ constexpr F2(float a, float b) : x(a), y(b) {}
};
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ F2 f2_of(float2 v) { return F2(v.x, v.y); }
__device__ __forceinline__ float2 f2_raw(F2 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ F2 fmaa(float a, F2 b, F2 c) { return f2_of(__ffma2_rn(make_float2(a, a), f2_raw(b), f2_raw(c))); }
__device__ __forceinline__ F2 fmaa(F2 a, F2 b, F2 c) { return f2_of(__ffma2_rn(f2_raw(a), f2_raw(b), f2_raw(c))); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2_of(__fadd2_rn(f2_raw(a), f2_raw(b))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return f2_of(__fmul2_rn(f2_raw(a), f2_raw(b))); }
#else
__device__ __forceinline__ F2 fmaa(float a, F2 b, F2 c) { return F2(fmaf(a, b.x, c.x), fmaf(a, b.y, c.y)); }
__device__ __forceinline__ F2 fmaa(F2 a, F2 b, F2 c) { return F2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(a.x * b.x, a.y * b.y); }
#endif
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ F2 operator*(float a, F2 b) { return F2(a) * b; }
__device__ __forceinline__ F2 operator*(F2 a, float b) { return a * F2(b); }
__device__ __forceinline__ F2 &operator*=(F2 &a, F2 b) { return a = a * b; }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = a + b; }
// the compute type of a value type (F2 holds two FP32 values)
template <class A> struct Scalar { using type = A; };
template <> struct Scalar<F2> { using type = float; };

template <int I, int E, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    if constexpr (I < E) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, E>(f);
    }
}

constexpr int odd_stride(int n) { return (n % 2 == 0) ? n + 1 : n; }

// Shared-memory bank degree of one warp's 4-byte accesses when its items are
// units e < epu at kw neighbouring structural indices c apart: the most
// addresses e * S + c * s that fall on one of the 32 banks.
constexpr int bank_ways(int S, int c, int epu, int kw)
{
    int cnt[32] = {};
    int worst = 0;
    for (int e = 0; e < epu; ++e)
        for (int s = 0; s < kw; ++s) {
            const int b = (e * S + c * s) % 32;
            if (++cnt[b] > worst) worst = cnt[b];
        }
    return worst;
}

// The per-unit stride in [s0, s0 + 32) with the least summed bank degree over
// the steps the stages take between neighbouring items: 1, N (modal lines) and
// Q (point lines); the smallest such stride on ties.
constexpr int pick_stride(int s0, int epu, int kw, int n, int q)
{
    int best = s0, bw = 1 << 30;
    for (int d = 0; d < 32; ++d) {
        const int w = bank_ways(s0 + d, 1, epu, kw) + bank_ways(s0 + d, n, epu, kw) + bank_ways(s0 + d, q, epu, kw);
        if (w < bw) {
            bw = w;
            best = s0 + d;
        }
    }
    return best;
}

// One pencil stage over EPB * per_e work items.  out_o = sum_r T(o,r) x_r
// (+ sum_r TX(r) xx_r when o == OEX).  `rot` rotates the thread->item map so
// consecutive barrier-free stages spread their tails over different threads.
// The table functors receive an offset z that is always 0 but is produced
// inside the loop, so the compiler keeps the (warp-broadcast) table loads in
// the loop instead of hoisting NIN x NOUT values into registers for threads
// that only run one or two iterations.
// ROLL keeps the output loop rolled (only the NIN multiply-adds of one output
// are unrolled): the collapsed shapes' class-split stages at high order
// otherwise unroll into more code than the instruction cache holds.
template <class A, int NIN, int NOUT, int NEX, int OEX, int EPB, int NT, bool ROLL = false, class LD, class TB,
          class LDX, class TBX, class ST>
__device__ __forceinline__ void pencils(int per_e, int &rot, LD ld, TB tb, LDX ldx, TBX tbx, ST st)
{
    // The bound is hidden from the compiler: with few elements per CTA it can
    // otherwise prove the loop runs at most once and straight-lines whole stages
    // into code that needs several times the registers.
    int total = per_e * EPB;
    NIR_OPAQUE(total);
    int w = (int)threadIdx.x - (rot % NT);
    if (w < 0) w += NT;
    for (; w < total; w += NT) {
        const int e = w % EPB;
        const int s = w / EPB;
        int z;
        NIR_ZERO(z);
        A x[NIN];
        ld(e, s, x);
        A xx[NEX > 0 ? NEX : 1];
        if constexpr (NEX > 0) ldx(e, s, xx);
        auto one = [&](int o) {
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
        };
        if constexpr (ROLL) {
#pragma unroll 1
            for (int o = 0; o < NOUT; ++o) one(o);
        } else {
#pragma unroll
            for (int o = 0; o < NOUT; ++o) one(o);
        }
    }
    rot += total;
}

// Work-item loop shared by the fused stages: items are (element e, index s)
// with e fastest across lanes; the loop bound is hidden from the compiler and
// z is a loop-local zero for shared-memory table offsets (see pencils()).
template <int EPB, int NT, class F>
__device__ __forceinline__ void for_items(int per_e, int &rot, F f)
{
    int total = per_e * EPB;
    NIR_OPAQUE(total);
    int w = (int)threadIdx.x - (rot % NT);
    if (w < 0) w += NT;
    for (; w < total; w += NT) {
        int z;
        NIR_ZERO(z);
        f(w % EPB, w / EPB, z);
    }
    rot += total;
}

struct NoX {
    template <class A> __device__ void operator()(int, int, A *) const {}
};
struct NoTX {
    __device__ int operator()(int, int) const { return 0; }
};
// A hook with nothing to do (run_group's after-metric callback).
struct NoHook {
    __device__ void operator()() const {}
};

template <class A, int NIN, int NOUT, int EPB, int NT, bool ROLL = false, class LD, class TB, class ST>
__device__ __forceinline__ void pencils0(int per_e, int &rot, LD ld, TB tb, ST st)
{
    pencils<A, NIN, NOUT, 0, 0, EPB, NT, ROLL>(per_e, rot, ld, tb, NoX{}, [](int, int) { return A(0); }, st);
}

// Table accessors.  Tables live either in shared memory (the persistent mesh
// kernel, whose blocks have different tables) or in the kernel-parameter
// constant bank (single-block kernels, passed as a __grid_constant__ struct):
// there, fully unrolled contractions read table entries as constant operands
// with no load instruction.  z is the loop-local zero of pencils() (only the
// shared-memory accessor uses it).
template <class A>
struct STab {
    const A *p;
    __device__ __forceinline__ STab operator+(int o) const { return STab{p + o}; }
    __device__ __forceinline__ A operator()(int z, int i) const { return p[z + i]; }
};

template <class A, int NTAB>
struct TabP {
    A v[NTAB];
};

template <class A, int NTAB>
struct PTab {
    const TabP<A, NTAB> *t;
    int base;
    __device__ __forceinline__ PTab operator+(int o) const { return PTab{t, base + o}; }
    __device__ __forceinline__ A operator()(int, int i) const { return t->v[base + i]; }
};

// Even/odd (symmetric) forms of the psiA contractions.  The first-direction
// points are symmetric (z_{Q-1-i} = -z_i: GLL, or Gauss-Legendre for the
// collapsed shapes' eta1) and psiA_0(-z) = psiA_1(z), psiA_p(-z) = (-1)^p psiA_p(z),
// so with s = x0 + x1, d = x0 - x1:
//   u_i = E_i + O_i, u_{Q-1-i} = E_i - O_i, E_i = Bs_e(i) . (s, x2, x4, ...),
//   O_i = Bs_o(i) . (d, x3, x5, ...),
// and the transpose pairs f_i +- f_{Q-1-i} the same way.  At P = 4 a pencil
// costs 23 instead of 30 multiply-add slots, at P = 6 38 instead of 56.
template <class A, int N, int Q, int EPB, int NT, class TP, class LD, class ST>
__device__ __forceinline__ void sym_bwd(int per_e, int &rot, TP Bs, LD ld, ST st)
{
    constexpr int QL = Q / 2, NE = sym_ne(N), NO = sym_no(N), W = NE + NO;
    for_items<EPB, NT>(per_e, rot, [&](int e, int s, int z) {
        A x[N];
        ld(e, s, x);
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
            for (int k = 0; k < NE; ++k) E = fmaa(Bs(z, i * W + k), xe[k], E);
#pragma unroll
            for (int k = 0; k < NO; ++k) O = fmaa(Bs(z, i * W + NE + k), xo[k], O);
            st(e, s, i, E + O);
            st(e, s, Q - 1 - i, E - O);
        }
        if constexpr (Q % 2 == 1) {
            A E = A(0);
#pragma unroll
            for (int k = 0; k < NE; ++k) E = fmaa(Bs(z, QL * W + k), xe[k], E);
            st(e, s, QL, E);
        }
    });
}

template <class A, int N, int Q, int EPB, int NT, class TP, class LD, class ST>
__device__ __forceinline__ void sym_iprod(int per_e, int &rot, TP Bs, LD ld, ST st)
{
    constexpr int QL = Q / 2, QH = (Q + 1) / 2, NE = sym_ne(N), NO = sym_no(N), W = NE + NO;
    for_items<EPB, NT>(per_e, rot, [&](int e, int s, int z) {
        A f[Q];
        ld(e, s, f);
        A fe[QH], fo[QL > 0 ? QL : 1];
#pragma unroll
        for (int i = 0; i < QL; ++i) {
            fe[i] = f[i] + f[Q - 1 - i];
            fo[i] = f[i] - f[Q - 1 - i];
        }
        if constexpr (Q % 2 == 1) fe[QL] = f[QL];
        {
            A Se = A(0), So = A(0);
#pragma unroll
            for (int i = 0; i < QH; ++i) Se = fmaa(Bs(z, i * W), fe[i], Se);
#pragma unroll
            for (int i = 0; i < QL; ++i) So = fmaa(Bs(z, i * W + NE), fo[i], So);
            st(e, s, 0, Se + So);
            st(e, s, 1, Se - So);
        }
#pragma unroll
        for (int k = 1; k < NE; ++k) {
            A acc = A(0);
#pragma unroll
            for (int i = 0; i < QH; ++i) acc = fmaa(Bs(z, i * W + k), fe[i], acc);
            st(e, s, 2 * k, acc);
        }
#pragma unroll
        for (int k = 1; k < NO; ++k) {
            A acc = A(0);
#pragma unroll
            for (int i = 0; i < QL; ++i) acc = fmaa(Bs(z, i * W + NE + k), fo[i], acc);
            st(e, s, 2 * k + 1, acc);
        }
    });
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
    // class-split stages of the collapsed shapes keep their output loops
    // rolled from P = 6 on in FP32/BF16 (code size; FP64 is bound by its FMA pipe)
    static constexpr bool R = (SH == TRI || SH == TET || SH == PRISM || SH == PYR) && N >= 7 &&
                              sizeof(typename Scalar<A>::type) == 4;

    // All BwdTrans stages but the last: 2-D p0 -> p1; 3-D p0 -> p1 -> p2.
    template <class TP>
    static __device__ __forceinline__ void front(TP tab, A *p0, A *p1, A *p2)
    {
        int rot = 0;
        if constexpr (SH == QUAD || SH == TRI) {
            if constexpr (SH == QUAD) {
                // t1[p][j] = sum_q u[p][q] psiA_q(z_j)
                sym_bwd<A, N, Q, EPB, NT>(N, rot, tab + L.Bs,
                    [=](int e, int s, A *x) { const A *b = p0 + e * S + s * N;
#pragma unroll
                        for (int r = 0; r < N; ++r) x[r] = b[r]; },
                    [=](int e, int s, int o, A v) { p1[e * S + s * Q + o] = v; });
            } else {
                // t1[p][j] = sum_{q<N-p} u[m(p,q)] psiB_pq(z_j) (+ the collapsed vertex (0,1) for p = 1)
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nin = nc + (p == 1 ? 1 : 0);
                    const TP Bp = tab + L.Bb + cls_off(N, Q, p);
                    const TP B0 = tab + L.Bb;
                    pencils0<A, nin, Q, EPB, NT, R>(1, rot,
                        [=](int e, int, A *x) { const A *b = p0 + e * S + tri_m0(N, p);
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r];
                            if constexpr (p == 1) x[nc] = p0[e * S + 1]; },
                        [=](int z, int o, int r) { return (p == 1 && r == nc) ? B0(z, o * N + 1) : Bp(z, o * nc + r); },
                        [=](int e, int, int o, A v) { p1[e * S + p * Q + o] = v; });
                });
            }
            __syncthreads();
        } else {
            // ---- stage 1: contract the third mode index r -> k
            if constexpr (SH == HEX) {
                sym_bwd<A, N, Q, EPB, NT>(N * N, rot, tab + L.Bs,
                    [=](int e, int s, A *x) { const A *b = p0 + e * S + s * N;
#pragma unroll
                        for (int r = 0; r < N; ++r) x[r] = b[r]; },
                    [=](int e, int s, int o, A v) { p1[e * S + s * Q + o] = v; });
            } else if constexpr (SH == PRISM) {
                // t1[p][q][k] = sum_{r<N-p} u[m(p,q,r)] psiB_pr(z3_k) (+ collapsed edge (0,q,1) for p = 1)
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nin = nc + (p == 1 ? 1 : 0);
                    const TP Bp = tab + L.Bb + cls_off(N, Q, p);
                    const TP B0 = tab + L.Bb;
                    pencils0<A, nin, Q, EPB, NT, R>(N, rot,
                        [=](int e, int q, A *x) { const A *b = p0 + e * S + prism_m0(N, p, q);
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r];
                            if constexpr (p == 1) x[nc] = p0[e * S + prism_m0(N, 0, q) + 1]; },
                        [=](int z, int o, int r) { return (p == 1 && r == nc) ? B0(z, o * N + 1) : Bp(z, o * nc + r); },
                        [=](int e, int q, int o, A v) { p1[e * S + (p * N + q) * Q + o] = v; });
                });
            } else if constexpr (SH == PYR) {
                // t1[p][q][k] = sum_{r<N-c} u[m(p,q,r)] psiB_cr(z3_k), c = max(p,q), over the
                // 2c+1 pairs of class c; the apex mode (0,0,1) -- psiA_1(eta3) alone -- also
                // feeds the class-1 pairs (1,0), (1,1), (0,1) through psiB_01(z3_k) = psiA_1(z3_k)
                // (with psiA_0 + psiA_1 = 1 in eta1 and eta2, the four pairs with p, q <= 1
                // then carry psiA_1(eta3) to every point).
                sfor<0, N>([&](auto cc) {
                    constexpr int c = decltype(cc)::value;
                    constexpr int nc = N - c;
                    constexpr int nin = nc + (c == 1 ? 1 : 0);
                    const TP Bc = tab + L.Bb + cls_off(N, Q, c);
                    const TP B0 = tab + L.Bb;
                    pencils0<A, nin, Q, EPB, NT, R>(2 * c + 1, rot,
                        [=](int e, int s, A *x) {
                            const A *b = p0 + e * S + pyr_m0(N, pyr_pair_p(c, s), pyr_pair_q(c, s));
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r];
                            if constexpr (c == 1) x[nc] = p0[e * S + 1]; },
                        [=](int z, int o, int r) { return (c == 1 && r == nc) ? B0(z, o * N + 1) : Bc(z, o * nc + r); },
                        [=](int e, int s, int o, A v) {
                            p1[e * S + (pyr_pair_p(c, s) * N + pyr_pair_q(c, s)) * Q + o] = v; });
                });
            } else {  // TET
                // t1[pair(p,q)][k] = sum_{r<N-p-q} u[m(p,q,r)] psiB_(p+q)r(z3_k); the collapsed
                // top vertex (0,0,1) also feeds pairs (0,1) and (1,0) through psiB_01(z3_k).
                sfor<0, N>([&](auto cc) {
                    constexpr int c = decltype(cc)::value;
                    constexpr int nc = N - c;
                    constexpr int nin = nc + (c == 1 ? 1 : 0);
                    const TP Bc = tab + L.Bc + cls_off(N, Q, c);
                    const TP B0 = tab + L.Bc;
                    pencils0<A, nin, Q, EPB, NT, R>(c + 1, rot,
                        [=](int e, int p, A *x) { const A *b = p0 + e * S + tet_m0(N, p, c - p);
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r];
                            if constexpr (c == 1) x[nc] = p0[e * S + 1]; },
                        [=](int z, int o, int r) { return (c == 1 && r == nc) ? B0(z, o * N + 1) : Bc(z, o * nc + r); },
                        [=](int e, int p, int o, A v) { p1[e * S + tet_pair(N, p, c - p) * Q + o] = v; });
                });
            }
            __syncthreads();
            // ---- stage 2: contract q -> j
            if constexpr (SH == HEX || SH == PRISM || SH == PYR) {
                sym_bwd<A, N, Q, EPB, NT>(N * Q, rot, tab + L.Bs,
                    [=](int e, int s, A *x) { const int p = s / Q, k = s - p * Q;
                        const A *b = p1 + e * S + p * N * Q + k;
#pragma unroll
                        for (int r = 0; r < N; ++r) x[r] = b[r * Q]; },
                    [=](int e, int s, int o, A v) { const int p = s / Q, k = s - p * Q;
                        p2[e * S + (p * Q + o) * Q + k] = v; });
            } else {  // TET: t2[p][j][k] = sum_{q<N-p} psiB_pq(z2_j) t1[pair(p,q)][k] (+ edge (0,1,.) for p = 1)
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nin = nc + (p == 1 ? 1 : 0);
                    const TP Bp = tab + L.Bb + cls_off(N, Q, p);
                    const TP B0 = tab + L.Bb;
                    pencils0<A, nin, Q, EPB, NT, R>(Q, rot,
                        [=](int e, int k, A *x) { const A *b = p1 + e * S + tet_pair(N, p, 0) * Q + k;
#pragma unroll
                            for (int r = 0; r < nc; ++r) x[r] = b[r * Q];
                            if constexpr (p == 1) x[nc] = p1[e * S + tet_pair(N, 0, 1) * Q + k]; },
                        [=](int z, int o, int r) { return (p == 1 && r == nc) ? B0(z, o * N + 1) : Bp(z, o * nc + r); },
                        [=](int e, int k, int o, A v) { p2[e * S + (p * Q + o) * Q + k] = v; });
                });
            }
            __syncthreads();
        }
    }

    // All transposed stages but the first: 2-D p1 -> last; 3-D p1 -> p2 -> last.
    template <class TP>
    static __device__ __forceinline__ void back(TP tab, A *p1, A *p2, A *outm)
    {
        int rot = 0;
        if constexpr (SH == QUAD || SH == TRI) {
            if constexpr (SH == QUAD) {
                sym_iprod<A, N, Q, EPB, NT>(N, rot, tab + L.Bs,
                    [=](int e, int s, A *x) { const A *b = p1 + e * S + s * Q;
#pragma unroll
                        for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                    [=](int e, int s, int o, A v) { outm[e * S + s * N + o] = v; });
            } else {
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nex = (p == 0 && N > 1) ? Q : 0;
                    const TP Bp = tab + L.Bb + cls_off(N, Q, p);
                    const TP B0 = tab + L.Bb;
                    pencils<A, Q, nc, nex, 1, EPB, NT, R>(1, rot,
                        [=](int e, int, A *x) { const A *b = p1 + e * S + p * Q;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                        [=](int z, int o, int r) { return Bp(z, r * nc + o); },
                        [=](int e, int, A *xx) { const A *b = p1 + e * S + 1 * Q;   // the (0,1) vertex: p = 1 line
#pragma unroll
                            for (int r = 0; r < nex; ++r) xx[r] = b[r]; },
                        [=](int z, int r) { return B0(z, r * N + 1); },
                        [=](int e, int, int o, A v) { outm[e * S + tri_m0(N, p) + o] = v; });
                });
            }
            __syncthreads();
        } else {
            // ---- transpose of stage 2
            if constexpr (SH == HEX || SH == PRISM || SH == PYR) {
                sym_iprod<A, N, Q, EPB, NT>(N * Q, rot, tab + L.Bs,
                    [=](int e, int s, A *x) { const int p = s / Q, k = s - p * Q;
                        const A *b = p1 + e * S + p * QQ + k;
#pragma unroll
                        for (int r = 0; r < Q; ++r) x[r] = b[r * Q]; },
                    [=](int e, int s, int o, A v) { const int p = s / Q, k = s - p * Q;
                        p2[e * S + (p * N + o) * Q + k] = v; });
            } else {  // TET: t1[pair(p,q)][k] = sum_j psiB_pq(z2_j) t2[p][j][k]; edge (0,1,.) also gets p = 1
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nex = (p == 0 && N > 1) ? Q : 0;
                    const TP Bp = tab + L.Bb + cls_off(N, Q, p);
                    const TP B0 = tab + L.Bb;
                    pencils<A, Q, nc, nex, 1, EPB, NT, R>(Q, rot,
                        [=](int e, int k, A *x) { const A *b = p1 + e * S + p * QQ + k;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r * Q]; },
                        [=](int z, int o, int r) { return Bp(z, r * nc + o); },
                        [=](int e, int k, A *xx) { const A *b = p1 + e * S + 1 * QQ + k;
#pragma unroll
                            for (int r = 0; r < nex; ++r) xx[r] = b[r * Q]; },
                        [=](int z, int r) { return B0(z, r * N + 1); },
                        [=](int e, int k, int o, A v) { p2[e * S + (tet_pair(N, p, 0) + o) * Q + k] = v; });
                });
            }
            __syncthreads();
            // ---- transpose of stage 1
            if constexpr (SH == HEX) {
                sym_iprod<A, N, Q, EPB, NT>(N * N, rot, tab + L.Bs,
                    [=](int e, int s, A *x) { const A *b = p2 + e * S + s * Q;
#pragma unroll
                        for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                    [=](int e, int s, int o, A v) { outm[e * S + s * N + o] = v; });
            } else if constexpr (SH == PRISM) {
                sfor<0, N>([&](auto cc) {
                    constexpr int p = decltype(cc)::value;
                    constexpr int nc = N - p;
                    constexpr int nex = (p == 0 && N > 1) ? Q : 0;
                    const TP Bp = tab + L.Bb + cls_off(N, Q, p);
                    const TP B0 = tab + L.Bb;
                    pencils<A, Q, nc, nex, 1, EPB, NT, R>(N, rot,
                        [=](int e, int q, A *x) { const A *b = p2 + e * S + (p * N + q) * Q;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                        [=](int z, int o, int r) { return Bp(z, r * nc + o); },
                        [=](int e, int q, A *xx) { const A *b = p2 + e * S + (1 * N + q) * Q;
#pragma unroll
                            for (int r = 0; r < nex; ++r) xx[r] = b[r]; },
                        [=](int z, int r) { return B0(z, r * N + 1); },
                        [=](int e, int q, int o, A v) { outm[e * S + prism_m0(N, p, q) + o] = v; });
                });
            } else if constexpr (SH == PYR) {
                // u[m(p,q,r)] = sum_k psiB_cr(z3_k) t[p][q][k] per pair of class c; the apex
                // mode (0,0,1) also collects the class-1 pairs (0,1), (1,0), (1,1) through
                // psiA_1(z3_k) (the transpose of the extra input of the forward stage)
                sfor<0, N>([&](auto cc) {
                    constexpr int c = decltype(cc)::value;
                    constexpr int nc = N - c;
                    constexpr int nex = (c == 0 && N > 1) ? 3 * Q : 0;
                    const TP Bc = tab + L.Bb + cls_off(N, Q, c);
                    const TP B0 = tab + L.Bb;
                    pencils<A, Q, nc, nex, 1, EPB, NT, R>(2 * c + 1, rot,
                        [=](int e, int s, A *x) {
                            const A *b = p2 + e * S + (pyr_pair_p(c, s) * N + pyr_pair_q(c, s)) * Q;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                        [=](int z, int o, int r) { return Bc(z, r * nc + o); },
                        [=](int e, int, A *xx) {
                            const A *b1 = p2 + e * S + (0 * N + 1) * Q;
                            const A *b2 = p2 + e * S + (1 * N + 0) * Q;
                            const A *b3 = p2 + e * S + (1 * N + 1) * Q;
#pragma unroll
                            for (int r = 0; r < nex / 3; ++r) {
                                xx[r] = b1[r];
                                xx[r + nex / 3] = b2[r];
                                xx[r + 2 * (nex / 3)] = b3[r];
                            } },
                        [=](int z, int r) { return B0(z, (r % Q) * N + 1); },
                        [=](int e, int s, int o, A v) {
                            outm[e * S + pyr_m0(N, pyr_pair_p(c, s), pyr_pair_q(c, s)) + o] = v; });
                });
            } else {  // TET: the top vertex (0,0,1) collects pairs (0,1) and (1,0)
                sfor<0, N>([&](auto cc) {
                    constexpr int c = decltype(cc)::value;
                    constexpr int nc = N - c;
                    constexpr int nex = (c == 0 && N > 1) ? 2 * Q : 0;
                    const TP Bc = tab + L.Bc + cls_off(N, Q, c);
                    const TP B0 = tab + L.Bc;
                    pencils<A, Q, nc, nex, 1, EPB, NT, R>(c + 1, rot,
                        [=](int e, int p, A *x) { const A *b = p2 + e * S + tet_pair(N, p, c - p) * Q;
#pragma unroll
                            for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                        [=](int z, int o, int r) { return Bc(z, r * nc + o); },
                        [=](int e, int, A *xx) {
                            const A *b1 = p2 + e * S + tet_pair(N, 0, 1) * Q;
                            const A *b2 = p2 + e * S + tet_pair(N, 1, 0) * Q;
#pragma unroll
                            for (int r = 0; r < nex / 2; ++r) { xx[r] = b1[r]; xx[r + nex / 2] = b2[r]; } },
                        [=](int z, int r) { return B0(z, (r % Q) * N + 1); },
                        [=](int e, int p, int o, A v) { outm[e * S + tet_m0(N, p, c - p) + o] = v; });
                });
            }
            __syncthreads();
        }
    }
    // Last BwdTrans stage (common to all shapes of a dimension):
    // 2-D u[i + Q j] = sum_p psiA_p(z_i) t1[p][j]; 3-D u[i + Q j + Q^2 k] = sum_p psiA_p(z_i) t2[p][j][k].
    template <class TP>
    static __device__ __forceinline__ void last(TP tab, A *in, A *out)
    {
        int rot = 0;
        if constexpr (SH == QUAD || SH == TRI) {
            sym_bwd<A, N, Q, EPB, NT>(Q, rot, tab + L.Bs,
                [=](int e, int s, A *x) { const A *b = in + e * S + s;
#pragma unroll
                    for (int r = 0; r < N; ++r) x[r] = b[r * Q]; },
                [=](int e, int s, int o, A v) { out[e * S + o + Q * s] = v; });
        } else {
            sym_bwd<A, N, Q, EPB, NT>(QQ, rot, tab + L.Bs,
                [=](int e, int s, A *x) { const int k = s / Q, j = s - k * Q;
                    const A *b = in + e * S + j * Q + k;
#pragma unroll
                    for (int r = 0; r < N; ++r) x[r] = b[r * QQ]; },
                [=](int e, int s, int o, A v) { out[e * S + o + Q * s] = v; });
        }
        __syncthreads();
    }

    // First transposed stage (common): t[p][j](k) = sum_i psiA_p(z_i) f[i + Q j (+ Q^2 k)].
    template <class TP>
    static __device__ __forceinline__ void first(TP tab, A *in, A *out)
    {
        int rot = 0;
        if constexpr (SH == QUAD || SH == TRI) {
            sym_iprod<A, N, Q, EPB, NT>(Q, rot, tab + L.Bs,
                [=](int e, int s, A *x) { const A *b = in + e * S + Q * s;
#pragma unroll
                    for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                [=](int e, int s, int o, A v) { out[e * S + o * Q + s] = v; });
        } else {
            sym_iprod<A, N, Q, EPB, NT>(QQ, rot, tab + L.Bs,
                [=](int e, int s, A *x) { const A *b = in + e * S + Q * s;
#pragma unroll
                    for (int r = 0; r < Q; ++r) x[r] = b[r]; },
                [=](int e, int s, int o, A v) { const int k = s / Q, j = s - k * Q;
                    out[e * S + o * QQ + j * Q + k] = v; });
        }
        __syncthreads();
    }

    // BwdTrans: p0 (modes) -> 2-D: p1 -> p2 (points); 3-D: p1 -> p2 -> p3 (points).
    template <class TP>
    static __device__ __forceinline__ void bwd(TP tab, A *p0, A *p1, A *p2, A *p3)
    {
        front(tab, p0, p1, p2);
        if constexpr (SH == QUAD || SH == TRI) last(tab, p1, p2);
        else last(tab, p2, p3);
    }

    // Transposed: p0 (points, weights applied) -> p1 (-> p2) -> modes in `lastbuf`.
    template <class TP>
    static __device__ __forceinline__ void iprod(TP tab, A *p0, A *p1, A *p2, A *lastbuf)
    {
        first(tab, p0, p1);
        back(tab, p1, p2, lastbuf);
    }
};


// ---------------------------------------------------------------------------
// Geometry access.  Per-point arrays are interleaved by 32 elements:
// value c of point n of element e at (((e >> 5) * NQ + n) * NG + c) * 32 + (e & 31).
// Per-element arrays are [E][NG] and exclude the reference weight, which is
// multiplied in here for the W component.
// ---------------------------------------------------------------------------
// PACK: the FP32/BF16 metric copies (NG = ngeo) use the packed per-point
// layout of geo_packed_index (one element's quad, pair and W adjacent);
// FP64 arrays and the PhysDeriv factors keep the interleaved one.
template <class T, class A, int NQ, int NG, bool PACK = false>
struct Geo {
    const T *g;
    const A *wq;
    int pp;
    __device__ __forceinline__ A get(long long e, int n, int c) const
    {
        if (pp) {
            if constexpr (PACK) return to_a(g[geo_packed_index(e, n, c, NQ, NG)], A());
            else return to_a(g[((((e >> 5) * NQ + n) * NG + c) << 5) + (e & 31)], A());
        }
        A v = to_a(g[e * NG + c], A());
        return (c == NG - 1) ? v * wq[n] : v;
    }
    // All NG values of point n of element e (per-element factors: W scaled by
    // the reference weight).  Packed per-point arrays take one 16-byte (BF16:
    // 8-byte) quad, one pair and one scalar load.
    __device__ __forceinline__ void get_all(long long e, int n, A (&v)[NG]) const
    {
        if constexpr (PACK) {
            if (pp) {
                const long long blk = (((e >> 5) * NQ + n) * NG) << 5;
                const int l = (int)(e & 31);
                load4(g + blk + l * 4, v);
                if constexpr (NG == 7) {
                    load2(g + blk + 128 + l * 2, v[4], v[5]);
                    v[6] = to_a(g[blk + 192 + l], A());
                }
                return;
            }
        }
#pragma unroll
        for (int c = 0; c < NG; ++c) v[c] = get(e, n, c);
    }
    // scale of the metric (non-W) components: 1 per point, wq[n] per element
    __device__ __forceinline__ A gscale(int n) const { return pp ? A(1) : wq[n]; }

  private:
    template <int K>
    static __device__ __forceinline__ void load4(const float *p, A (&v)[K])
    {
        const float4 q = NIR_METRIC_LD(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    template <int K>
    static __device__ __forceinline__ void load4(const __nv_bfloat16 *p, A (&v)[K])
    {
        const uint2 q = NIR_METRIC_LD(reinterpret_cast<const uint2 *>(p));
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void load2(const float *p, A &x, A &y)
    {
        const float2 q = NIR_METRIC_LD(reinterpret_cast<const float2 *>(p));
        x = q.x; y = q.y;
    }
    static __device__ __forceinline__ void load2(const __nv_bfloat16 *p, A &x, A &y)
    {
        const unsigned q = NIR_METRIC_LD(reinterpret_cast<const unsigned *>(p));
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q));
        x = a.x; y = a.y;
    }
    template <int K>
    static __device__ __forceinline__ void load4(const double *, A (&)[K]) {}
    static __device__ __forceinline__ void load2(const double *, A &, A &) {}
};

// The metric of element pairs (2u, 2u+1) for the paired FP32/BF16 Helmholtz.
// In the packed layout the two elements' quads, pairs and W values are
// adjacent: one point takes two 16-byte, one 16-byte and one 8-byte load
// (BF16: 16, 8 and 4 bytes) for both elements.
template <class T, int NQ, int NG, bool PACK>
struct GeoPair {
    Geo<T, float, NQ, NG, PACK> g1;
    const float *wq;
    __device__ __forceinline__ void get_all(long long u, int n, F2 (&v)[NG]) const
    {
        const long long e = 2 * u;
        if constexpr (PACK) {
            if (g1.pp) {
                const long long blk = (((e >> 5) * NQ + n) * NG) << 5;
                const int l = (int)(e & 31);
                float q[8];
                load8(g1.g + blk + l * 4, q);
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c] = F2(q[c], q[4 + c]);
                if constexpr (NG == 7) {
                    float r[4], w[2];
                    load4(g1.g + blk + 128 + l * 2, r);
                    load2(g1.g + blk + 192 + l, w);
                    v[4] = F2(r[0], r[2]);
                    v[5] = F2(r[1], r[3]);
                    v[6] = F2(w[0], w[1]);
                }
                return;
            }
        }
        float a[NG], b[NG];
        g1.get_all(e, n, a);
        g1.get_all(e + 1, n, b);
#pragma unroll
        for (int c = 0; c < NG; ++c) v[c] = F2(a[c], b[c]);
    }

  private:
    static __device__ __forceinline__ void load8(const float *p, float (&v)[8])
    {
        const float4 a = NIR_METRIC_LD_PAIR(reinterpret_cast<const float4 *>(p));
        const float4 b = NIR_METRIC_LD_PAIR(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    static __device__ __forceinline__ void load4(const float *p, float (&v)[4])
    {
        const float4 a = NIR_METRIC_LD_PAIR(reinterpret_cast<const float4 *>(p));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    static __device__ __forceinline__ void load2(const float *p, float (&v)[2])
    {
        const float2 a = NIR_METRIC_LD_PAIR(reinterpret_cast<const float2 *>(p));
        v[0] = a.x; v[1] = a.y;
    }
    static __device__ __forceinline__ void unpack2(unsigned w, float &a, float &b)
    {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
        a = f.x;
        b = f.y;
    }
    static __device__ __forceinline__ void load8(const __nv_bfloat16 *p, float (&v)[8])
    {
        const uint4 a = NIR_METRIC_LD_PAIR(reinterpret_cast<const uint4 *>(p));
        unpack2(a.x, v[0], v[1]); unpack2(a.y, v[2], v[3]); unpack2(a.z, v[4], v[5]); unpack2(a.w, v[6], v[7]);
    }
    static __device__ __forceinline__ void load4(const __nv_bfloat16 *p, float (&v)[4])
    {
        const uint2 a = NIR_METRIC_LD_PAIR(reinterpret_cast<const uint2 *>(p));
        unpack2(a.x, v[0], v[1]); unpack2(a.y, v[2], v[3]);
    }
    static __device__ __forceinline__ void load2(const __nv_bfloat16 *p, float (&v)[2])
    {
        unpack2(NIR_METRIC_LD_PAIR(reinterpret_cast<const unsigned *>(p)), v[0], v[1]);
    }
    template <int K> static __device__ __forceinline__ void load8(const double *, float (&)[K]) {}
    template <int K> static __device__ __forceinline__ void load4(const double *, float (&)[K]) {}
    template <int K> static __device__ __forceinline__ void load2(const double *, float (&)[K]) {}
};

// Default elements per CTA: fill about 110 KB (FP64) or 56 KB (FP32/BF16) of
// shared memory with the operator's buffers.  EPB_ > 0 overrides it (the
// autotuner picks among compiled alternatives).
template <int SH, int N, int Q, class T, int OP, int EPB_ = 0, int NT_ = 0, bool PAIR = false>
struct Config {
    using A = typename CT<T>::type;
    static constexpr int D = dim(SH);
    static constexpr int NQ = npts(SH, Q);
    static constexpr int M = nmodes(SH, N);
    static constexpr int S0 = odd_stride(NQ);
    // the fused FP32/BF16 Helmholtz recomputes du/d eta3 in registers: 3 buffers
    static constexpr bool FUSED = (OP == OP_HELM && sizeof(A) == 4);
    static_assert(!PAIR || FUSED, "paired elements: FP32/BF16 Helmholtz only");
    static constexpr int NBUF = (OP == OP_BWD || OP == OP_IPROD || OP == OP_MASS) ? 2 : FUSED ? 3 : D + 1;
    static constexpr int TABN = layout(SH, N, Q).total;
    static constexpr int TABB = ((TABN * (int)sizeof(A) + 15) / 16) * 16;
    // FP32/BF16 aim at >= 32 elements so a warp covers one structural index of
    // 32 elements (conflict-free with the odd stride); FP64 keeps ~110 KB.
    static constexpr int budget = sizeof(A) == 8 ? 110 * 1024 : 100 * 1024;
    static constexpr int per_elem = NBUF * S0 * (int)sizeof(A);
    static constexpr int raw = (budget - TABB) / per_elem;
    static constexpr int EPB_DEF = raw >= 64 ? 64 : raw >= 32 ? 32 : raw >= 16 ? 16 : raw >= 8 ? 8 : raw >= 4 ? 4
                                 : raw >= 2 ? 2 : 1;
    static constexpr int EPB = EPB_ > 0 ? EPB_ : (PAIR && EPB_DEF < 2 ? 2 : EPB_DEF);
    static_assert(!PAIR || EPB % 2 == 0, "paired elements: an even group");
    // work units per group: elements, or element pairs (a pair's values are
    // adjacent, at the unit's index, so one 8-byte access serves both)
    static constexpr int EPU = PAIR ? EPB / 2 : EPB;
    // Per-unit stride of the group buffers.  Odd, so that one structural index of 32 units
    // spans the 32 banks.  With fewer units per group a warp's items span KW = 32 / EPU
    // structural indices, and no single stride keeps every stage's neighbours on distinct
    // banks: the fused FP32/BF16 stages take the stride with the least summed bank degree
    // over their neighbour steps (pick_stride; P = 6 hexes: 16 elements per group, +13 %).
    // Paired units (8 bytes) and FP64 keep the odd stride.
    static constexpr int KW = EPU < 32 ? 32 / EPU : 1;
    static constexpr int S = (FUSED && !PAIR && KW > 1) ? pick_stride(S0, EPU, KW, N, Q) : S0;
    // Threads: 256 (up to 512 for the fused FP32/BF16 Helmholtz): the fused
    // stages have Q^2 (3-D) or Q (2-D) pencils per element, and the CTA is
    // sized so that its heaviest stages run in whole rounds (two, or more when
    // two would exceed 512 threads) instead of leaving warps idle at every
    // barrier.  NT_ > 0 forces a size (the persistent mesh kernel shares one).
    static constexpr int PENCILS = (D == 3 ? Q * Q : Q) * EPU;
    // at least two rounds, and as many as keep the CTA within 512 threads,
    // every thread running the same number of rounds (1152 pencils: 3 x 384
    // rather than 2.25 x 512)
    static constexpr int ROUNDS = (PENCILS + 511) / 512 > 2 ? (PENCILS + 511) / 512 : 2;
    static constexpr int NT_HALF = ((PENCILS / ROUNDS + (PENCILS % ROUNDS ? 1 : 0) + 31) / 32) * 32;
    static constexpr int NT_AUTO = FUSED ? (NT_HALF >= 512 ? 512 : NT_HALF < 128 ? 128 : NT_HALF) : 256;
    static constexpr int NT = NT_ > 0 ? NT_ : NT_AUTO;
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
// Paired-element forms: unit u holds elements 2u (x) and 2u+1 (y) of the group.
template <class T, int LEN, int S, int NT>
__device__ __forceinline__ void gload_pair(const T *__restrict__ g, long long e0, int ne, F2 *sm)
{
    const T *src = g + e0 * LEN;
    const int nu = (ne + 1) / 2;
    for (int i = threadIdx.x; i < nu * LEN; i += NT) {
        const int u = i / LEN, m = i - u * LEN;
        const float a = to_a(__ldg(src + (2 * u) * LEN + m), float());
        const float b = (2 * u + 1 < ne) ? to_a(__ldg(src + (2 * u + 1) * LEN + m), float()) : 0.0f;
        sm[u * S + m] = F2(a, b);
    }
}

template <class T, int LEN, int S, int NT>
__device__ __forceinline__ void gstore_pair(T *__restrict__ g, long long e0, int ne, const F2 *sm)
{
    T *dst = g + e0 * LEN;
    const int nu = (ne + 1) / 2;
    for (int i = threadIdx.x; i < nu * LEN; i += NT) {
        const int u = i / LEN, m = i - u * LEN;
        const F2 v = sm[u * S + m];
        from_a(v.x, dst + (2 * u) * LEN + m);
        if (2 * u + 1 < ne) from_a(v.y, dst + (2 * u + 1) * LEN + m);
    }
}

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

// ---------------------------------------------------------------------------
// Fused Helmholtz stages (register-blocked pencils).  3-D buffers:
//   in (t2) -> U = u, V1 = du/d eta1      last BwdTrans stage + D1
//   U -> V2 = du/d eta2                  middle gradient direction
//   pencils along k: du/d eta3 = D3 u in registers, per point v = G du and
//   m = lambda W u, then U = m + D3^T v3
//   U += D2^T v2 (pencils along j)
//   y = U + D1^T v1, t2 = B1^T y (pencils along i) -> first IProduct stage
// 2-D drops the middle direction.  Every pencil loads its line once and
// produces a whole output line from registers.
// ---------------------------------------------------------------------------
template <int SH, int N, int Q, class A, int EPB, int NT, int S>
struct HelmStages {
    static constexpr TabLayout L = layout(SH, N, Q);
    static constexpr int D = dim(SH);
    static constexpr int QQ = Q * Q;
    static constexpr int PER = D == 3 ? QQ : Q;  // pencils per direction per element

    template <class TP>
    static __device__ __forceinline__ void last_grad1(TP tab, const A *in, A *U, A *V1)
    {
        const TP Bs = tab + L.Bs, D1 = tab + L.D1;
        int rot = 0;
        for_items<EPB, NT>(PER, rot, [&](int e, int s, int z) {
            A x[N];
            if constexpr (D == 3) {
                const int k = s / Q, j = s - k * Q;
                const A *b = in + e * S + j * Q + k;
#pragma unroll
                for (int r = 0; r < N; ++r) x[r] = b[r * QQ];
            } else {
                const A *b = in + e * S + s;
#pragma unroll
                for (int r = 0; r < N; ++r) x[r] = b[r * Q];
            }
            A u[Q];
            {  // u = psiA x in even/odd form (see sym_bwd)
                constexpr int QL = Q / 2, NE = sym_ne(N), NO = sym_no(N), W = NE + NO;
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
                    for (int k = 0; k < NE; ++k) E = fmaa(Bs(z, i * W + k), xe[k], E);
#pragma unroll
                    for (int k = 0; k < NO; ++k) O = fmaa(Bs(z, i * W + NE + k), xo[k], O);
                    u[i] = E + O;
                    u[Q - 1 - i] = E - O;
                }
                if constexpr (Q % 2 == 1) {
                    A E = A(0);
#pragma unroll
                    for (int k = 0; k < NE; ++k) E = fmaa(Bs(z, QL * W + k), xe[k], E);
                    u[QL] = E;
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) U[e * S + i + Q * s] = u[i];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                A acc = A(0);
#pragma unroll
                for (int r = 0; r < Q; ++r) acc = fmaa(D1(z, i * Q + r), u[r], acc);
                V1[e * S + i + Q * s] = acc;
            }
        });
        __syncthreads();
    }

    // d/d eta2 (3-D: pencils along j; 2-D: pencils along j of the 2-D grid).
    // The 3-D d/d eta3 is formed in registers by metric_tlast.
    template <class TP>
    static __device__ __forceinline__ void grad_rest(TP tab, const A *U, A *V2)
    {
        const TP D2 = tab + L.D2;
        int rot = 0;
        if constexpr (D == 3) {
            for_items<EPB, NT>(QQ, rot, [&](int e, int s, int z) {  // along j: s = i + Q k
                const int k = s / Q, i = s - k * Q;
                const A *b = U + e * S + i + QQ * k;
                A x[Q];
#pragma unroll
                for (int r = 0; r < Q; ++r) x[r] = b[r * Q];
#pragma unroll
                for (int o = 0; o < Q; ++o) {
                    A acc = A(0);
#pragma unroll
                    for (int r = 0; r < Q; ++r) acc = fmaa(D2(z, o * Q + r), x[r], acc);
                    V2[e * S + i + Q * o + QQ * k] = acc;
                }
            });
        } else {
            for_items<EPB, NT>(Q, rot, [&](int e, int s, int z) {  // along j: s = i
                const A *b = U + e * S + s;
                A x[Q];
#pragma unroll
                for (int r = 0; r < Q; ++r) x[r] = b[r * Q];
#pragma unroll
                for (int o = 0; o < Q; ++o) {
                    A acc = A(0);
#pragma unroll
                    for (int r = 0; r < Q; ++r) acc = fmaa(D2(z, o * Q + r), x[r], acc);
                    V2[e * S + s + Q * o] = acc;
                }
            });
        }
        __syncthreads();
    }

    // Per point v = G du (G holds W and the chain rule; per-element factors
    // are scaled by the reference weight) and m = lambda W u; the pencil along
    // the last direction then writes U = m + D_last^T v_last.
    template <bool PP, class TP, class GEO>
    static __device__ __forceinline__ void metric_tlast(TP tab, const GEO &geo, long long e0, A lam, A *U, A *V1,
                                                        A *V2)
    {
        constexpr int ST = D == 3 ? QQ : Q;
        constexpr int NG = D == 3 ? 7 : 4;
        const TP DL = tab + (D == 3 ? L.D3 : L.D2);
        int rot = 0;
        for_items<EPB, NT>(PER, rot, [&](int e, int s, int z) {
            const long long eg = e0 + e;
            A vl[Q], m[Q], d3[Q];
            if constexpr (D == 3) {  // du/d eta3 along this pencil, from u
                A u[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k) u[k] = U[e * S + s + ST * k];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    A acc = A(0);
#pragma unroll
                    for (int r = 0; r < Q; ++r) acc = fmaa(DL(z, k * Q + r), u[r], acc);
                    d3[k] = acc;
                }
            }
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int n = s + ST * k;
                A d0 = V1[e * S + n], d1 = V2[e * S + n], d2 = A(0);
                if constexpr (D == 3) d2 = d3[k];
                if constexpr (!PP) {
                    const A sc = geo.wq[n];
                    d0 *= sc;
                    d1 *= sc;
                    d2 *= sc;
                }
                A g[NG];
                geo.get_all(eg, n, g);
                if constexpr (D == 3) {
                    V1[e * S + n] = fmaa(g[0], d0, fmaa(g[1], d1, g[2] * d2));
                    V2[e * S + n] = fmaa(g[1], d0, fmaa(g[3], d1, g[4] * d2));
                    vl[k] = fmaa(g[2], d0, fmaa(g[4], d1, g[5] * d2));
                } else {
                    V1[e * S + n] = fmaa(g[0], d0, g[1] * d1);
                    vl[k] = fmaa(g[1], d0, g[2] * d1);
                }
                m[k] = lam * g[NG - 1] * U[e * S + n];
            }
#pragma unroll
            for (int o = 0; o < Q; ++o) {
                A acc = m[o];
#pragma unroll
                for (int r = 0; r < Q; ++r) acc = fmaa(DL(z, r * Q + o), vl[r], acc);
                U[e * S + s + ST * o] = acc;
            }
        });
        __syncthreads();
    }

    template <class TP>
    static __device__ __forceinline__ void tmid(TP tab, A *U, const A *V2)
    {
        const TP D2 = tab + L.D2;
        int rot = 0;
        for_items<EPB, NT>(QQ, rot, [&](int e, int s, int z) {  // along j: s = i + Q k
            const int k = s / Q, i = s - k * Q;
            const A *b = V2 + e * S + i + QQ * k;
            A x[Q];
#pragma unroll
            for (int r = 0; r < Q; ++r) x[r] = b[r * Q];
#pragma unroll
            for (int o = 0; o < Q; ++o) {
                A *y = U + e * S + i + Q * o + QQ * k;
                A acc = *y;
#pragma unroll
                for (int r = 0; r < Q; ++r) acc = fmaa(D2(z, r * Q + o), x[r], acc);
                *y = acc;
            }
        });
        __syncthreads();
    }

    template <class TP>
    static __device__ __forceinline__ void t1_first(TP tab, const A *U, const A *V1, A *out)
    {
        const TP Bs = tab + L.Bs, D1 = tab + L.D1;
        int rot = 0;
        for_items<EPB, NT>(PER, rot, [&](int e, int s, int z) {
            const A *bv = V1 + e * S + Q * s;
            const A *bu = U + e * S + Q * s;
            A v[Q], y[Q];
#pragma unroll
            for (int r = 0; r < Q; ++r) v[r] = bv[r];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                A acc = bu[i];
#pragma unroll
                for (int r = 0; r < Q; ++r) acc = fmaa(D1(z, r * Q + i), v[r], acc);
                y[i] = acc;
            }
            // t[p] = sum_i psiA_p(z_i) y_i in even/odd form (see sym_iprod)
            constexpr int QL = Q / 2, QH = (Q + 1) / 2, NE = sym_ne(N), NO = sym_no(N), W = NE + NO;
            A t[N];
            {
                A fe[QH], fo[QL];
#pragma unroll
                for (int i = 0; i < QL; ++i) {
                    fe[i] = y[i] + y[Q - 1 - i];
                    fo[i] = y[i] - y[Q - 1 - i];
                }
                if constexpr (Q % 2 == 1) fe[QL] = y[QL];
                A Se = A(0), So = A(0);
#pragma unroll
                for (int i = 0; i < QH; ++i) Se = fmaa(Bs(z, i * W), fe[i], Se);
#pragma unroll
                for (int i = 0; i < QL; ++i) So = fmaa(Bs(z, i * W + NE), fo[i], So);
                t[0] = Se + So;
                t[1] = Se - So;
#pragma unroll
                for (int k = 1; k < NE; ++k) {
                    A acc = A(0);
#pragma unroll
                    for (int i = 0; i < QH; ++i) acc = fmaa(Bs(z, i * W + k), fe[i], acc);
                    t[2 * k] = acc;
                }
#pragma unroll
                for (int k = 1; k < NO; ++k) {
                    A acc = A(0);
#pragma unroll
                    for (int i = 0; i < QL; ++i) acc = fmaa(Bs(z, i * W + NE + k), fo[i], acc);
                    t[2 * k + 1] = acc;
                }
            }
#pragma unroll
            for (int p = 0; p < N; ++p) {
                if constexpr (D == 3) {
                    const int k = s / Q, j = s - k * Q;
                    out[e * S + p * QQ + j * Q + k] = t[p];
                } else {
                    out[e * S + p * Q + s] = t[p];
                }
            }
        });
        __syncthreads();
    }
};

// Point-wise Helmholtz metric stage (FP64 path): v_i = sum_j G_ij du_j at
// every point of the group, du by collocation gathers.
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

// Nodal (GLL-Lagrange) coefficients of a quad/hex and the reflection-pair
// form the contraction tables are built for (see the table builder): along
// each direction, pair k = 1 .. (N-2)/2 of nodes (k, N-1-k) becomes
// (x_k + x_{N-1-k}, x_k - x_{N-1-k}) in slots (2k, 2k+1), the end nodes go to
// slots 0 and 1 and an odd N's middle node to slot N-1.  to_pairs maps nodal
// input coefficients into that form; otherwise it maps inner products taken
// against the pair functions back to nodal ones (the inverse transpose, which
// for these 2x2 blocks is the sum/difference without the factor 1/2).
// In place on the group's modal block (element stride S), one direction per
// pass.
template <int SH, int N, class A, int EPB, int NT, int S>
__device__ __noinline__ void nodal_pairs(A *buf, bool to_pairs)  // out of line: modified-basis kernels only carry a call
{
    if constexpr ((SH == QUAD || SH == HEX) && N > 2) {
        constexpr int D = dim(SH);
        constexpr int LINES = D == 2 ? N : N * N;
        constexpr int K = (N - 2) / 2;
        for (int dir = 0; dir < D; ++dir) {
            const int stride = D == 2 ? (dir == 0 ? N : 1) : (dir == 0 ? N * N : dir == 1 ? N : 1);
            for (int w = threadIdx.x; w < EPB * LINES; w += NT) {
                const int e = w % EPB, l = w / EPB;
                int base;
                if constexpr (D == 2) base = dir == 0 ? l : l * N;
                else base = dir == 0 ? l : dir == 1 ? (l / N) * N * N + (l % N) : l * N;
                A *v = buf + e * S + base;
                A x[N], y[N];
#pragma unroll
                for (int r = 0; r < N; ++r) x[r] = v[r * stride];
                if (to_pairs) {
                    y[0] = x[0];
                    y[1] = x[N - 1];
#pragma unroll
                    for (int k = 1; k <= K; ++k) {
                        y[2 * k] = x[k] + x[N - 1 - k];
                        y[2 * k + 1] = x[k] - x[N - 1 - k];
                    }
                    if constexpr (N % 2 == 1) y[N - 1] = x[(N - 1) / 2];
                } else {
                    y[0] = x[0];
                    y[N - 1] = x[1];
#pragma unroll
                    for (int k = 1; k <= K; ++k) {
                        y[k] = x[2 * k] + x[2 * k + 1];
                        y[N - 1 - k] = x[2 * k] - x[2 * k + 1];
                    }
                    if constexpr (N % 2 == 1) y[(N - 1) / 2] = x[N - 1];
                }
#pragma unroll
                for (int r = 0; r < N; ++r) v[r * stride] = y[r];
            }
            __syncthreads();
        }
    }
}

// One group of ne (<= EPB) elements starting at e0: the whole operator.
// tab: the block's tables in shared memory; buf: NBUF * EPB * S values.
// TP: table accessor for the contractions (STab or PTab); tab: the same
// tables in shared memory (collocation gathers of PhysDeriv and
// IProductWRTDerivBase, reference weights).
// fin/fout: the group's first input and output arrays (a field of a
// multi-field Helmholtz call; a.in0 / a.out0 otherwise).
// after_metric: called by every thread once the fused FP32/BF16 Helmholtz
// has consumed the group's geometric factors (the staged kernel starts the
// next group's L2 prefetch there).
template <int SH, int N, int Q, class T, int OP, int EPB_, int NT_, bool PAIR = false, class TP, class HOOK = NoHook>
__device__ __forceinline__ void run_group(const KArgs &a, const void *fin, void *fout, TP tp,
                                          const typename CT<T>::type *tab, typename CT<T>::type *buf, long long e0,
                                          int ne, bool staged = false, HOOK after_metric = HOOK{})
{
    using C = Config<SH, N, Q, T, OP, EPB_, NT_, PAIR>;
    using A = typename C::A;
    constexpr int D = C::D, NQ = C::NQ, M = C::M, S = C::S, EPB = C::EPB, NT = C::NT;
    constexpr TabLayout L = layout(SH, N, Q);
    constexpr int NG = (OP == OP_PHYSDERIV || OP == OP_IPROD_DERIV) ? nlam(SH) : ngeo(SH);
    using MD = Modal<SH, N, Q, A, EPB, NT, S>;
    using HS = HelmStages<SH, N, Q, A, EPB, NT, S>;
    A *B0 = buf, *B1 = buf + EPB * S, *B2 = buf + 2 * EPB * S, *B3 = buf + 3 * EPB * S;
    const A *D0 = tab + L.D1, *D1 = tab + L.D2, *D2 = tab + L.D3;
    // the FP32/BF16 metric copies are packed (the PhysDeriv factors are not)
    constexpr bool PACK = sizeof(T) < 8 && NG == ngeo(SH);
    const Geo<T, A, NQ, NG, PACK> geo{reinterpret_cast<const T *>(a.geo), tab + L.wq, a.geo_pp};

    constexpr bool TENSOR = SH == QUAD || SH == HEX;
    auto to_pairs = [&](A *blk) {
        if constexpr (TENSOR) { if (a.nodal) nodal_pairs<SH, N, A, EPB, NT, S>(blk, true); }
    };
    auto from_pairs = [&](A *blk) {
        if constexpr (TENSOR) { if (a.nodal) nodal_pairs<SH, N, A, EPB, NT, S>(blk, false); }
    };
    if constexpr (OP == OP_BWD) {
        gload<T, A, M, S, NT>(reinterpret_cast<const T *>(fin), e0, ne, B0);
        __syncthreads();
        to_pairs(B0);
        if constexpr (D == 2) {
            MD::bwd(tp, B0, B1, B0, nullptr);
            gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(fout), e0, ne, B0);
        } else {
            MD::bwd(tp, B0, B1, B0, B1);
            gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(fout), e0, ne, B1);
        }
    } else if constexpr (OP == OP_IPROD || OP == OP_MASS) {
        A *P = B0;
        if constexpr (OP == OP_IPROD) {
            gload<T, A, NQ, S, NT>(reinterpret_cast<const T *>(fin), e0, ne, B0);
            __syncthreads();
        } else {
            gload<T, A, M, S, NT>(reinterpret_cast<const T *>(fin), e0, ne, B0);
            __syncthreads();
            to_pairs(B0);
            if constexpr (D == 2) MD::bwd(tp, B0, B1, B0, nullptr);
            else { MD::bwd(tp, B0, B1, B0, B1); P = B1; }
        }
        for (int w = threadIdx.x; w < EPB * NQ; w += NT) {
            const int e = w % EPB, n = w / EPB;
            P[e * S + n] *= geo.get(e0 + e, n, NG - 1);
        }
        __syncthreads();
        A *O = (P == B0) ? B1 : B0;
        if constexpr (D == 2) {
            MD::iprod(tp, P, O, nullptr, P);
            from_pairs(P);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(fout), e0, ne, P);
        } else {
            MD::iprod(tp, P, O, P, O);
            from_pairs(O);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(fout), e0, ne, O);
        }
    } else if constexpr (OP == OP_PHYSDERIV) {
        gload<T, A, NQ, S, NT>(reinterpret_cast<const T *>(fin), e0, ne, B0);
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
        gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(fout), e0, ne, B1);
        gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(a.out1), e0, ne, B2);
        if constexpr (D == 3) gstore<T, A, NQ, S, NT>(reinterpret_cast<T *>(a.out2), e0, ne, B3);
    } else if constexpr (OP == OP_IPROD_DERIV) {
        gload<T, A, NQ, S, NT>(reinterpret_cast<const T *>(fin), e0, ne, B1);
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
            MD::iprod(tp, B0, B1, nullptr, B2);
            from_pairs(B2);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(fout), e0, ne, B2);
        } else {
            MD::iprod(tp, B0, B1, B2, B1);
            from_pairs(B1);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(fout), e0, ne, B1);
        }
    } else if constexpr (sizeof(A) == 8) {  // OP_HELM, FP64: point-wise gradient flow
        // (the FP64 pipe is the bound; fine-grained point work items keep it
        // busy across barriers better than whole pencils)
        gload<T, A, M, S, NT>(reinterpret_cast<const T *>(fin), e0, ne, B1);
        __syncthreads();
        to_pairs(B1);
        if constexpr (D == 2) MD::bwd(tp, B1, B2, B0, nullptr);
        else MD::bwd(tp, B1, B2, B1, B0);
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
            MD::iprod(tp, B0, B1, nullptr, B2);
            from_pairs(B2);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(fout), e0, ne, B2);
        } else {
            MD::iprod(tp, B0, B1, B2, B1);
            from_pairs(B1);
            gstore<T, A, M, S, NT>(reinterpret_cast<T *>(fout), e0, ne, B1);
        }
    } else if constexpr (PAIR) {  // OP_HELM, FP32 / BF16, two elements per work unit (see F2)
        using V = F2;
        constexpr int EPU = C::EPU;
        using MV = Modal<SH, N, Q, V, EPU, NT, S>;
        using HV = HelmStages<SH, N, Q, V, EPU, NT, S>;
        V *U0 = reinterpret_cast<V *>(buf), *U1 = U0 + EPU * S, *U2 = U1 + EPU * S;
        const GeoPair<T, NQ, NG, PACK> gp{geo, tab + L.wq};
        const V lam = V(float(a.lambda));
        const long long u0 = e0 / 2;  // groups hold an even number of elements
        if (!staged) {  // otherwise the caller has already put the coefficients in U1
            gload_pair<T, M, S, NT>(reinterpret_cast<const T *>(fin), e0, ne, U1);
            __syncthreads();
        }
        if constexpr (TENSOR) { if (a.nodal) nodal_pairs<SH, N, V, EPU, NT, S>(U1, true); }
        if constexpr (D == 2) {
            MV::front(tp, U1, U2, nullptr);
            HV::last_grad1(tp, U2, U0, U1);
            HV::grad_rest(tp, U0, U2);
            if (a.geo_pp) HV::template metric_tlast<true>(tp, gp, u0, lam, U0, U1, U2);
            else HV::template metric_tlast<false>(tp, gp, u0, lam, U0, U1, U2);
            after_metric();
            HV::t1_first(tp, U0, U1, U2);
            MV::back(tp, U2, nullptr, U0);
        } else {
            MV::front(tp, U1, U2, U1);
            HV::last_grad1(tp, U1, U0, U2);
            HV::grad_rest(tp, U0, U1);
            if (a.geo_pp) HV::template metric_tlast<true>(tp, gp, u0, lam, U0, U2, U1);
            else HV::template metric_tlast<false>(tp, gp, u0, lam, U0, U2, U1);
            after_metric();
            HV::tmid(tp, U0, U1);
            HV::t1_first(tp, U0, U2, U1);
            MV::back(tp, U1, U2, U0);
        }
        if constexpr (TENSOR) { if (a.nodal) nodal_pairs<SH, N, V, EPU, NT, S>(U0, false); }
        gstore_pair<T, M, S, NT>(reinterpret_cast<T *>(fout), e0, ne, U0);
    } else {  // OP_HELM, FP32 / BF16: fused register-blocked pencils
        const A lam = A(a.lambda);
        if (!staged) {  // otherwise the caller has already put the coefficients in B1
            gload<T, A, M, S, NT>(reinterpret_cast<const T *>(fin), e0, ne, B1);
            __syncthreads();
        }
        to_pairs(B1);
        if constexpr (D == 2) {
            // B1 modes -> B2 t1 -> U = B0, V1 = B1, V2 = B2
            MD::front(tp, B1, B2, nullptr);
            HS::last_grad1(tp, B2, B0, B1);
            HS::grad_rest(tp, B0, B2);
            if (a.geo_pp) HS::template metric_tlast<true>(tp, geo, e0, lam, B0, B1, B2);
            else HS::template metric_tlast<false>(tp, geo, e0, lam, B0, B1, B2);
            after_metric();
            HS::t1_first(tp, B0, B1, B2);
            MD::back(tp, B2, nullptr, B0);
        } else {
            // B1 modes -> B2 t1 -> B1 t2 -> U = B0, V1 = B2, V2 = B1
            MD::front(tp, B1, B2, B1);
            HS::last_grad1(tp, B1, B0, B2);
            HS::grad_rest(tp, B0, B1);
            if (a.geo_pp) HS::template metric_tlast<true>(tp, geo, e0, lam, B0, B2, B1);
            else HS::template metric_tlast<false>(tp, geo, e0, lam, B0, B2, B1);
            after_metric();
            HS::tmid(tp, B0, B1);
            HS::t1_first(tp, B0, B2, B1);
            MD::back(tp, B1, B2, B0);
        }
        from_pairs(B0);
        gstore<T, A, M, S, NT>(reinterpret_cast<T *>(fout), e0, ne, B0);
    }
    __syncthreads();
}

#ifdef __CUDACC__  // device-only from here: bulk copies, mbarriers and the kernels
// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, non-tensor form) and mbarriers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global
// to shared memory, completing on `bar`; the caller arrives with expect_tx.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bring `bytes` (multiple of 16, 16-byte aligned) of global memory into L2.
__device__ __forceinline__ void l2_prefetch(const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Wait for phase `parity` of `bar` for at most `limit` clock cycles (by
// default 2^31, about a second).  Returns false on timeout after setting the
// device error word.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int *err,
                                          long long limit = (1LL << 31))
{
    const long long t0 = clock64();
    unsigned done = 0;
    while (true) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) {
            if (err) atomicExch(err, 1);
            return false;
        }
    }
}

// Single-block FP32/BF16 Helmholtz with the next group's coefficients staged
// by a bulk copy while the current group computes (a group's inputs are
// [EPB][M] contiguous values).  With a.pf = 1 the group's per-point metric
// (for EPB a multiple of 32: whole 32-element chunks of the interleaved
// layout) is bulk-prefetched into L2 one group ahead (the first group's at
// the start, each next group's once the current group's metric stage is
// done), so the metric stage finds it there; with a.pf = 2 each group's own
// metric is prefetched when the group starts (half the L2 footprint in
// flight, half the lead time); the autotuner decides which pays.  Groups whose copy would not be 16-byte aligned, and the ragged
// last group, are loaded with plain coalesced loads.
// STAGE = false: no staging buffer (coefficients loaded by the group itself),
// for groups whose buffers alone nearly fill shared memory.
// MULTI: the multi-field form (1..3 fields per group, a.nfields); the
// single-field form is a separate instantiation so its code and register
// allocation do not carry the field loop.
// CTAs of `threads` threads and `smem` bytes of shared memory that fit on one
// SM (228 KB, 1 KB reserved per CTA; 2048 threads), at least 1.  Used as the
// launch bound's minimum blocks per SM: the register budget ptxas may use is
// then what that occupancy leaves, so a kernel whose shared memory already
// limits it to one CTA per SM is not squeezed into 64 registers (and spills).
constexpr int ctas_per_sm(int smem, int threads)
{
    const int by_smem = (228 * 1024) / (smem + 1024);
    const int by_thr = 2048 / threads;
    const int c = by_smem < by_thr ? by_smem : by_thr;
    return c < 1 ? 1 : c;
}
template <int SH, int N, int Q, class T, int EPB_, bool STAGE>
constexpr int helm_tma_smem()
{
    using C = Config<SH, N, Q, T, OP_HELM, EPB_>;
    return C::SMEM + (STAGE ? ((C::EPB * C::M * (int)sizeof(T) + 15) / 16) * 16 : 0);
}

template <int SH, int N, int Q, class T, int EPB_ = 0, bool STAGE = true, bool MULTI = false, bool PAIR = false>
__global__ void __launch_bounds__(Config<SH, N, Q, T, OP_HELM, EPB_, 0, PAIR>::NT,
                                  ctas_per_sm(helm_tma_smem<SH, N, Q, T, EPB_, STAGE>(),
                                              Config<SH, N, Q, T, OP_HELM, EPB_, 0, PAIR>::NT))
    k_helm_tma(KArgs a, const __grid_constant__ TabP<typename CT<T>::type, layout(SH, N, Q).total> tp)
{
    using C = Config<SH, N, Q, T, OP_HELM, EPB_, 0, PAIR>;
    using A = typename C::A;
    static_assert(C::FUSED, "FP32/BF16 Helmholtz only");
    constexpr int EPB = C::EPB, NT = C::NT, M = C::M, S = C::S, NQ = C::NQ, NG = ngeo(SH);
    constexpr int STG = STAGE ? ((EPB * M * (int)sizeof(T) + 15) / 16) * 16 : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *tab = reinterpret_cast<A *>(smem_raw);
    T *stage = reinterpret_cast<T *>(smem_raw + C::TABB);
    A *buf = reinterpret_cast<A *>(smem_raw + C::TABB + STG);
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int s_next, s_fail;
    for (int i = threadIdx.x; i < C::TABN; i += NT) tab[i] = tp.v[i];
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        s_fail = 0;
    }
    __syncthreads();
    const PTab<A, C::TABN> ptab{&tp, 0};
    const long long ngroups = (a.nelem + EPB - 1) / EPB;
    const T *in = reinterpret_cast<const T *>(a.in0);
    const T *G = reinterpret_cast<const T *>(a.geo);
    // issue the copy of group g (thread 0); returns whether it was issued
    // the whole 32-element chunks of the metric covering the group (a group
    // smaller than a chunk prefetches its whole chunk)
    auto prefetch_metric = [&](long long e0) {
        constexpr int span = EPB >= 32 ? EPB : 32;
        if (a.pf && a.geo_pp && ((EPB % 32) == 0 || (32 % EPB) == 0)) {
            const char *gp = reinterpret_cast<const char *>(G + (((e0 >> 5) * NQ * NG) << 5));
            const long long gbytes = (long long)NQ * NG * span * (long long)sizeof(T);
            for (long long off = 0; off < gbytes; off += 32768)
                l2_prefetch(gp + off, (unsigned)((gbytes - off) < 32768 ? (gbytes - off) : 32768));
        }
    };
    // work items: (group g, field f), the fields of a group back to back so
    // the group's metric is read from HBM once and from L2 for later fields
    const int nf = (MULTI && a.nfields > 1) ? (a.nfields < 3 ? a.nfields : 3) : 1;
    auto issue = [&](long long g, int f) -> int {
        if (!STAGE || g >= ngroups) return 0;
        const long long e0 = g * EPB;
        if (e0 + EPB > a.nelem) return 0;
        const T *src = reinterpret_cast<const T *>(field_in(a, f)) + e0 * M;
        const unsigned bytes = (unsigned)(EPB * M * sizeof(T));
        if ((reinterpret_cast<unsigned long long>(src) & 15) || (bytes & 15)) return 0;
        tma_load_1d(stage, src, bytes, &bar);
        return 1;
    };
    (void)in;
    unsigned phase = 0;
    if (threadIdx.x == 0) {
        s_next = issue(blockIdx.x, 0);
        if (blockIdx.x < ngroups) prefetch_metric((long long)blockIdx.x * EPB);  // the first group's factors
    }
    __syncthreads();
    for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const long long e0 = g * EPB;
        const int ne = (int)((a.nelem - e0) < EPB ? (a.nelem - e0) : EPB);
        // once this group's factors are consumed, start bringing the next
        // group's into L2: they then have the rest of this group and the next
        // group's first stages to arrive, and about one group of factors per
        // CTA is resident in L2 at a time
        const long long gn = g + gridDim.x;
        auto prefetch_next = [&]() {
            if (threadIdx.x == 0 && gn < ngroups && a.pf == 1) prefetch_metric(gn * EPB);
        };
        if (a.pf == 2 && threadIdx.x == 0 && g != blockIdx.x) prefetch_metric(e0);  // this group's, now
        for (int f = 0; f < nf; ++f) {
            const bool staged = s_next != 0;
            if (staged) {
                if (!mbar_wait(&bar, phase, a.err)) s_fail = 1;
                phase ^= 1u;
                __syncthreads();
                if (s_fail) return;  // every thread leaves together; the error word is set
                if constexpr (PAIR) {  // element pairs (2u, 2u+1) into one unit each
                    F2 *B1 = reinterpret_cast<F2 *>(buf) + C::EPU * S;
                    for (int i = threadIdx.x; i < C::EPU * M; i += NT) {
                        const int u = i / M, m = i - u * M;
                        B1[u * S + m] = F2(to_a(stage[2 * u * M + m], A()), to_a(stage[(2 * u + 1) * M + m], A()));
                    }
                } else {
                    A *B1 = buf + EPB * S;
                    for (int i = threadIdx.x; i < EPB * M; i += NT) {
                        const int e = i / M, m = i - e * M;
                        B1[e * S + m] = to_a(stage[i], A());
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0)  // stage is free again: the next field, or the next group's first
                s_next = f + 1 < nf ? issue(g, f + 1) : issue(g + gridDim.x, 0);
            run_group<SH, N, Q, T, OP_HELM, EPB_, 0, PAIR>(a, field_in(a, f), field_out(a, f), ptab, tab, buf, e0,
                                                           ne, staged, [&]() {
                                                               if (f == 0) prefetch_next();
                                                           });
        }
    }
}

// Persistent single-block kernel: CTAs stride over the element groups.  The
// tables arrive twice: as a __grid_constant__ parameter (constant bank, used
// by the contractions) and copied once into shared memory (gathers, weights).
template <int SH, int N, int Q, class T, int OP, int EPB_ = 0, bool MULTI = false>
__global__ void __launch_bounds__(256)
    k_elem(KArgs a, const __grid_constant__ TabP<typename CT<T>::type, layout(SH, N, Q).total> tp)
{
    using C = Config<SH, N, Q, T, OP, EPB_>;
    using A = typename C::A;
    constexpr int EPB = C::EPB, NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *tab = reinterpret_cast<A *>(smem_raw);
    A *buf = reinterpret_cast<A *>(smem_raw + C::TABB);
    for (int i = threadIdx.x; i < C::TABN; i += NT) tab[i] = tp.v[i];
    __syncthreads();
    const long long ngroups = (a.nelem + EPB - 1) / EPB;
    // FP32 contractions take table entries as constant-bank operands; DFMA
    // would first load them into register pairs (and the compiler hoists
    // them), so FP64 reads its tables from shared memory instead.
    // Helmholtz fields of a group run back to back (see k_helm_tma)
    const int nf = (MULTI && OP == OP_HELM && a.nfields > 1) ? (a.nfields < 3 ? a.nfields : 3) : 1;
    if constexpr (sizeof(A) == 4) {
        const PTab<A, C::TABN> ptab{&tp, 0};
        for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
            const long long e0 = g * EPB;
            const int ne = (int)((a.nelem - e0) < EPB ? (a.nelem - e0) : EPB);
            for (int f = 0; f < nf; ++f)
                run_group<SH, N, Q, T, OP, EPB_, 0>(a, field_in(a, f), field_out(a, f), ptab, tab, buf, e0, ne);
        }
    } else {
        const STab<A> stab{tab};
        for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
            const long long e0 = g * EPB;
            const int ne = (int)((a.nelem - e0) < EPB ? (a.nelem - e0) : EPB);
            for (int f = 0; f < nf; ++f)
                run_group<SH, N, Q, T, OP, EPB_, 0>(a, field_in(a, f), field_out(a, f), stab, tab, buf, e0, ne);
        }
    }
}

#endif  // __CUDACC__

}  // namespace nirk
