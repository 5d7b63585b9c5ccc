// nir_layout.h -- compile-time sizes and table layout shared by the host table
// builder and the device kernels of the library (not by the oracle).
//
// Notation: N = P+1 modes per direction, Q points per direction, d = 2 or 3.
// Modes are packed p outermost, then q, then r; the collapsed shapes bound
// q < N-p (tri, tet) and r < N-p-q (tet), r < N-p (prism) or
// r < N-max(p,q) (pyramid), as in the sum-factorised loops of Sec. 2.2
// (Eq. bwdsumfactet).  Points are indexed
// i + Q*(j + Q*k) with the first (eta1/xi1) direction fastest.
#pragma once

#ifdef __CUDACC__
#define NIR_HD __host__ __device__
#else
#define NIR_HD
#endif

namespace nirk {

enum Shape { QUAD = 0, TRI = 1, HEX = 2, PRISM = 3, TET = 4, PYR = 5 };

NIR_HD constexpr int dim(int s) { return (s == QUAD || s == TRI) ? 2 : 3; }

NIR_HD constexpr int nmodes(int s, int N)
{
    return s == QUAD ? N * N : s == TRI ? N * (N + 1) / 2 : s == HEX ? N * N * N
         : s == PRISM ? N * N * (N + 1) / 2 : s == PYR ? N * (N + 1) * (2 * N + 1) / 6
         : N * (N + 1) * (N + 2) / 6;
}

NIR_HD constexpr int npts(int s, int Q) { return dim(s) == 2 ? Q * Q : Q * Q * Q; }

// Number of metric values per point: upper triangle of G plus W = w|J|.
NIR_HD constexpr int ngeo(int s) { return dim(s) == 2 ? 4 : 7; }
// Number of PhysDeriv factors per point: d eta_j / d x_l (row j) plus W.
NIR_HD constexpr int nlam(int s) { return dim(s) == 2 ? 5 : 10; }

// Per-point metric (ng = ngeo values) of the FP32/BF16 copies, packed so that
// one element's values are adjacent: per chunk of 32 elements and per point,
// the 32 elements' quads (G00 G01 G02 G11) -- 2-D: (G00 G01 G11 W) -- then
// their pairs (G12 G22), then their W.  A thread reads its point's values
// with three vector loads instead of seven scalar ones; the block of a point
// is the same 32 x ng values as in the interleaved FP64 layout (value c of
// element lane l at c * 32 + l), so chunks stay contiguous.
NIR_HD constexpr long long geo_packed_off(int c, int l, int ng)
{
    return (ng == 4 || c < 4) ? l * 4 + c : c < 6 ? 128 + l * 2 + (c - 4) : 192 + l;
}
NIR_HD constexpr long long geo_packed_index(long long e, int n, int c, int nq, int ng)
{
    return ((((e >> 5) * nq + n) * ng) << 5) + geo_packed_off(c, (int)(e & 31), ng);
}

// Ragged class tables: class c holds Q x (N - c) values.
NIR_HD constexpr int cls_cols(int N, int c) { return N - c; }
NIR_HD constexpr int cls_off(int N, int Q, int c)
{
    int o = 0;
    for (int k = 0; k < c; ++k) o += Q * cls_cols(N, k);
    return o;
}
NIR_HD constexpr int cls_size(int N, int Q) { return cls_off(N, Q, N); }

// Packed-mode helpers for the collapsed shapes.
// tet: first mode of pair (p,q); pairs ordered p outer, q inner, q < N-p.
NIR_HD constexpr int tet_pair(int N, int p, int q)
{
    int o = 0;
    for (int k = 0; k < p; ++k) o += N - k;
    return o + q;
}
NIR_HD constexpr int tet_m0(int N, int p, int q)
{
    int o = 0;
    for (int a = 0; a < p; ++a) o += (N - a) * (N - a + 1) / 2;
    for (int b = 0; b < q; ++b) o += N - p - b;
    return o;
}
NIR_HD constexpr int tri_m0(int N, int p)
{
    int o = 0;
    for (int a = 0; a < p; ++a) o += N - a;
    return o;
}
NIR_HD constexpr int prism_m0(int N, int p, int q)
{
    int o = 0;
    for (int a = 0; a < p; ++a) o += N * (N - a);
    return o + q * (N - p);
}
// pyramid: pair (p,q) holds N - max(p,q) modes r; pairs p outer, q inner.
// Row p holds sum_q (N - max(p,q)) = (N-p)(N+p+1)/2 modes, so the rows before
// p hold p N(N+1)/2 - (p-1)p(p+1)/6; within row p, pair q starts after
// q (N-p) modes when q <= p, else after (p+1)(N-p) + sum_{b=p+1}^{q-1} (N-b).
NIR_HD constexpr int pyr_m0(int N, int p, int q)
{
    const int base = p * N * (N + 1) / 2 - (p - 1) * p * (p + 1) / 6;
    const int in_row = q <= p ? q * (N - p)
                              : (p + 1) * (N - p) + (q - p - 1) * N - (q - 1) * q / 2 + p * (p + 1) / 2;
    return base + in_row;
}
// Pyramid pair s (0 <= s < 2c+1) of class c = max(p,q): s <= c is (c, s),
// s > c is (s - c - 1, c).
NIR_HD constexpr int pyr_pair_p(int c, int s) { return s <= c ? c : s - c - 1; }
NIR_HD constexpr int pyr_pair_q(int c, int s) { return s <= c ? s : c; }

// Table blob layout (units of the compute type).
//  Ba : Q x N, Ba[k*N + r] = psiA_r(z1_k)           (first direction)
//  Bb : ragged classes p = 0..N-1, Q x (N-p): psiB_pq(z2_j)  (tri/tet eta2; prism eta3;
//       pyramid eta3 with the class c = max(p,q))
//  Bc : ragged classes c = 0..N-1, Q x (N-c): psiB_cr(z3_k)  (tet eta3; c = p+q)
//  D1, D2, D3 : Q x Q collocation derivative matrices, D[i*Q + i'] = l'_i'(z_i)
//  wq : reference quadrature weight per point (collapse factors included)
//  Bs : even/odd form of Ba on the symmetric first-direction points, ceil(Q/2)
//       rows of sym_ne(N) + sym_no(N) values: [(Ba_i0 + Ba_i1)/2, Ba_i2, Ba_i4, ...]
//       then [(Ba_i0 - Ba_i1)/2, Ba_i3, Ba_i5, ...]
struct TabLayout {
    int Ba, Bb, Bc, D1, D2, D3, wq, Bs, total;
};

NIR_HD constexpr int sym_ne(int N) { return 1 + (N - 1) / 2; }
NIR_HD constexpr int sym_no(int N) { return 1 + (N - 2) / 2; }

NIR_HD constexpr TabLayout layout(int s, int N, int Q)
{
    TabLayout L{0, 0, 0, 0, 0, 0, 0, 0, 0};
    int o = 0;
    L.Ba = o; o += Q * N;
    L.Bb = o; if (s == TRI || s == TET || s == PRISM || s == PYR) o += cls_size(N, Q);
    L.Bc = o; if (s == TET) o += cls_size(N, Q);
    L.D1 = o; o += Q * Q;
    L.D2 = o; if (s == TRI || s == TET) o += Q * Q;
    L.D3 = o; if (s == TET || s == PRISM || s == PYR) o += Q * Q;
    L.wq = o; o += npts(s, Q);
    L.Bs = o; o += ((Q + 1) / 2) * (sym_ne(N) + sym_no(N));
    L.total = o;
    // directions sharing a rule share a table
    if (s == QUAD || s == HEX) { L.D2 = L.D1; L.D3 = L.D1; }
    if (s == PRISM || s == PYR) L.D2 = L.D1;
    return L;
}

}  // namespace nirk
