// nir_basis.cpp -- host-side FP64 construction of the 1-D quadrature rules,
// modified-basis tables, collocation derivative matrices and geometry
// interpolation tables used by the device kernels.
//
// Quadrature (Sec. 2.2: points avoiding the collapsed endpoints):
//   * Gauss-Jacobi(alpha, beta) nodes and weights by the Golub-Welsch
//     characterisation: the nodes are the eigenvalues of the symmetric
//     tridiagonal Jacobi matrix of the weight (1-x)^alpha (1+x)^beta (found
//     here by Sturm-sequence bisection), the weights the Christoffel numbers
//     mu0 / sum_k p_k(x)^2 of the orthonormal polynomials.
//   * Gauss-Lobatto-Legendre: +-1 plus the Gauss-Jacobi(1,1) nodes, weights
//     2 / (Q (Q-1) P_{Q-1}(x)^2).
// Directions: quad/hex GLL; tri eta1 GJ(0,0), eta2 GJ(1,0); tet eta1 GJ(0,0),
// eta2 GJ(1,0), eta3 GJ(2,0); prism eta1, eta2 GLL, eta3 GJ(1,0); pyramid
// eta1, eta2 GLL, eta3 GJ(2,0).  The collapse Jacobians (1-eta2)/2 and
// ((1-eta3)/2)^2 are absorbed as factors 1/2 and 1/4 of the Gauss-Jacobi
// weights (Eq. iprodtet's tilde weights).
//
// Basis (Sec. 2.2, Eqs. bwdsumfachex/bwdsumfactet, modified C0 expansion):
//   psiA_p(z): (1-z)/2, (1+z)/2, (1-z)(1+z)/4 P^{(1,1)}_{p-2}(z)
//   psiB_pq(z): psiA_q(z) when p = 0; ((1-z)/2)^p when q = 0;
//               ((1-z)/2)^p (1+z)/2 P^{(2p-1,1)}_{q-1}(z) otherwise.
// Collocation derivative (Eq. stdderiv): barycentric form of l_j'(z_i).
#include "nir_basis.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nir_layout.h"

namespace {

// Eigenvalues of the symmetric tridiagonal matrix T (diagonal d[0..n-1],
// off-diagonal e[0..n-2], all e != 0) by bisection on Sturm counts: the
// number of negative pivots of the LDL^T factorisation of T - x I is the
// number of eigenvalues below x (Sylvester's law of inertia).  Each
// eigenvalue is isolated in a Gershgorin interval and halved until the
// interval stops shrinking in floating point.
int sturm_count(int n, const double *d, const double *e, double x)
{
    int neg = 0;
    double q = d[0] - x;
    for (int k = 0;; ++k) {
        if (q == 0.0) q = -1e-300;  // perturb an exact zero pivot (x is then an eigenvalue)
        if (q < 0.0) ++neg;
        if (k + 1 == n) break;
        q = (d[k + 1] - x) - e[k] * e[k] / q;
    }
    return neg;
}

void tridiag_eigenvalues(int n, const double *d, const double *e, double *lam)
{
    double lo = d[0], hi = d[0];
    for (int k = 0; k < n; ++k) {
        const double r = (k > 0 ? std::fabs(e[k - 1]) : 0.0) + (k + 1 < n ? std::fabs(e[k]) : 0.0);
        lo = std::min(lo, d[k] - r);
        hi = std::max(hi, d[k] + r);
    }
    for (int j = 0; j < n; ++j) {  // the (j+1)-th smallest eigenvalue
        double a = lo, b = hi;
        for (int it = 0; it < 200; ++it) {
            const double m = 0.5 * (a + b);
            if (m <= a || m >= b) break;
            if (sturm_count(n, d, e, m) > j) b = m;
            else a = m;
        }
        lam[j] = 0.5 * (a + b);
    }
}

}  // namespace

double nirb_jacobi(int n, double a, double b, double x)
{
    // P_n^{(a,b)} from P_0 = 1, P_1 = ((a+b+2) x + a - b) / 2 and the
    // standard three-term recurrence in n.
    if (n == 0) return 1.0;
    double pm = 1.0, pc = 0.5 * ((a + b + 2.0) * x + (a - b));
    for (int k = 2; k <= n; ++k) {
        double t = 2.0 * k + a + b;
        double A = 2.0 * k * (k + a + b) * (t - 2.0);
        double Bc = (t - 1.0) * (t * (t - 2.0) * x + a * a - b * b);
        double Cc = 2.0 * (k - 1 + a) * (k - 1 + b) * t;
        double pn = (Bc * pc - Cc * pm) / A;
        pm = pc;
        pc = pn;
    }
    return pc;
}

double nirb_jacobi_d(int n, double a, double b, double x)
{
    return n == 0 ? 0.0 : 0.5 * (n + a + b + 1.0) * nirb_jacobi(n - 1, a + 1.0, b + 1.0, x);
}

bool nirb_gauss_jacobi(int Q, double a, double b, double *z, double *w)
{
    std::vector<double> d(Q), e(Q);
    for (int k = 0; k < Q; ++k) {
        double t = 2.0 * k + a + b;
        d[k] = (t == 0.0) ? (b - a) / (a + b + 2.0) : (b * b - a * a) / (t * (t + 2.0));
        if (k + 1 < Q) {
            double n = k + 1.0, s = 2.0 * n + a + b;
            e[k] = std::sqrt(4.0 * n * (n + a) * (n + b) * (n + a + b) / (s * s * (s + 1.0) * (s - 1.0)));
        }
    }
    // nodes: the eigenvalues of the Jacobi matrix (ascending)
    tridiag_eigenvalues(Q, d.data(), e.data(), z);
    // weights (Christoffel numbers): with p_0 .. p_{Q-1} the polynomials
    // orthonormal for the weight, w(x) = mu0 / sum_k p_k(x)^2, where mu0 is the
    // weight's total mass; the p_k follow the Jacobi matrix's recurrence
    // e_k p_{k+1} = (x - d_k) p_k - e_{k-1} p_{k-1}, p_0 = 1.  (The squared
    // first component of the normalised eigenvector, Golub-Welsch's formula,
    // is the same number: the eigenvector of eigenvalue x is (p_k(x))_k.)
    const double mu0 = std::exp((a + b + 1.0) * std::log(2.0) + std::lgamma(a + 1.0) + std::lgamma(b + 1.0)
                                - std::lgamma(a + b + 2.0));
    for (int i = 0; i < Q; ++i) {
        const double x = z[i];
        double pm = 0.0, pc = 1.0, sum = 1.0;
        for (int k = 0; k + 1 < Q; ++k) {
            const double pn = ((x - d[k]) * pc - (k > 0 ? e[k - 1] * pm : 0.0)) / e[k];
            pm = pc;
            pc = pn;
            sum += pc * pc;
        }
        if (!(sum > 0.0) || !std::isfinite(sum)) return false;
        w[i] = mu0 / sum;
    }
    return true;
}

bool nirb_gll(int Q, double *z, double *w)
{
    z[0] = -1.0;
    z[Q - 1] = 1.0;
    if (Q > 2) {
        std::vector<double> wi(Q - 2);
        if (!nirb_gauss_jacobi(Q - 2, 1.0, 1.0, z + 1, wi.data())) return false;
    }
    for (int k = 0; k < Q; ++k) {
        double p = nirb_jacobi(Q - 1, 0.0, 0.0, z[k]);
        w[k] = 2.0 / (double(Q) * (Q - 1) * p * p);
    }
    return true;
}

double nirb_psiA(int p, double z)
{
    if (p == 0) return 0.5 * (1.0 - z);
    if (p == 1) return 0.5 * (1.0 + z);
    return 0.25 * (1.0 - z) * (1.0 + z) * nirb_jacobi(p - 2, 1.0, 1.0, z);
}

double nirb_psiB(int p, int q, double z)
{
    if (p == 0) return nirb_psiA(q, z);
    double h = std::pow(0.5 * (1.0 - z), p);
    if (q == 0) return h;
    return h * 0.5 * (1.0 + z) * nirb_jacobi(q - 1, 2.0 * p - 1.0, 1.0, z);
}

void nirb_colloc(int Q, const double *z, double *D)
{
    std::vector<double> lam(Q);
    for (int j = 0; j < Q; ++j) {
        double p = 1.0;
        for (int k = 0; k < Q; ++k)
            if (k != j) p *= (z[j] - z[k]);
        lam[j] = 1.0 / p;
    }
    for (int i = 0; i < Q; ++i) {
        double diag = 0.0;
        for (int j = 0; j < Q; ++j) {
            if (j == i) continue;
            double v = (lam[j] / lam[i]) / (z[i] - z[j]);
            D[i * Q + j] = v;
            diag -= v;  // rows of a differentiation matrix sum to zero
        }
        D[i * Q + i] = diag;
    }
}

void nirb_lagrange_equi(int g, int Q, const double *z, double *L, double *dL)
{
    const int n = g + 1;
    std::vector<double> t(n), lam(n);
    for (int a = 0; a < n; ++a) t[a] = -1.0 + 2.0 * a / g;
    for (int a = 0; a < n; ++a) {
        double p = 1.0;
        for (int b = 0; b < n; ++b)
            if (b != a) p *= (t[a] - t[b]);
        lam[a] = 1.0 / p;
    }
    for (int q = 0; q < Q; ++q) {
        double x = z[q];
        int hit = -1;
        for (int a = 0; a < n; ++a)
            if (x == t[a]) hit = a;
        if (hit >= 0) {
            for (int a = 0; a < n; ++a) {
                L[q * n + a] = (a == hit) ? 1.0 : 0.0;
                if (a != hit) {
                    dL[q * n + a] = (lam[a] / lam[hit]) / (t[hit] - t[a]);
                } else {
                    double s = 0.0;
                    for (int b = 0; b < n; ++b)
                        if (b != hit) s += 1.0 / (t[hit] - t[b]);
                    dL[q * n + a] = s;
                }
            }
            continue;
        }
        double den = 0.0;
        for (int a = 0; a < n; ++a) den += lam[a] / (x - t[a]);
        for (int a = 0; a < n; ++a) {
            double la = (lam[a] / (x - t[a])) / den;
            double s = 0.0;
            for (int b = 0; b < n; ++b)
                if (b != a) s += 1.0 / (x - t[b]);
            L[q * n + a] = la;
            dL[q * n + a] = la * s;
        }
    }
}

bool nirb_shape_rules(int shape, int Q, double *z /*[3][Q]*/, double *w /*[3][Q]*/)
{
    using namespace nirk;
    // kind: 0 GLL, 1+alpha Gauss-Jacobi(alpha, 0)
    int kind[3] = {0, 0, 0};
    double sc[3] = {1.0, 1.0, 1.0};
    if (shape == TRI) { kind[0] = 1; kind[1] = 2; sc[1] = 0.5; }
    if (shape == TET) { kind[0] = 1; kind[1] = 2; kind[2] = 3; sc[1] = 0.5; sc[2] = 0.25; }
    if (shape == PRISM) { kind[2] = 2; sc[2] = 0.5; }
    if (shape == PYR) { kind[2] = 3; sc[2] = 0.25; }
    for (int dir = 0; dir < 3; ++dir) {
        bool ok = kind[dir] == 0 ? nirb_gll(Q, z + dir * Q, w + dir * Q)
                                 : nirb_gauss_jacobi(Q, kind[dir] - 1.0, 0.0, z + dir * Q, w + dir * Q);
        if (!ok) return false;
        for (int k = 0; k < Q; ++k) w[dir * Q + k] *= sc[dir];
    }
    return true;
}

// Nodal (GLL-Lagrange) basis seen through its reflection pairs: with l_j the
// Lagrange polynomials through the N GLL points, mode 0 is l_0, mode 1 is
// l_{N-1}, modes 2k and 2k+1 (k = 1 .. (N-2)/2) are (l_k + l_{N-1-k})/2 and
// (l_k - l_{N-1-k})/2, and for odd N mode N-1 is the middle l_{(N-1)/2}.  These
// have the modified basis' symmetry (0 <-> 1 under z -> -z, mode p with
// parity (-1)^p), so the even/odd contractions apply unchanged; nodal
// coefficients are mapped to and from this form in the kernels.
double nirb_nodal_pair(int p, int N, double z)
{
    std::vector<double> x(N), w(N);
    nirb_gll(N, x.data(), w.data());
    auto lag = [&](int j) {
        double v = 1.0;
        for (int m = 0; m < N; ++m)
            if (m != j) v *= (z - x[m]) / (x[j] - x[m]);
        return v;
    };
    if (p == 0) return lag(0);
    if (p == 1) return lag(N - 1);
    if (N % 2 == 1 && p == N - 1) return lag((N - 1) / 2);
    const int k = p / 2;
    return (p % 2 == 0) ? 0.5 * (lag(k) + lag(N - 1 - k)) : 0.5 * (lag(k) - lag(N - 1 - k));
}

bool nirb_build_tables(int shape, int P, int Q, double *blob, int basis)
{
    using namespace nirk;
    const int N = P + 1;
    const TabLayout L = layout(shape, N, Q);
    std::vector<double> z(3 * Q), w(3 * Q);
    if (!nirb_shape_rules(shape, Q, z.data(), w.data())) return false;
    if (basis != 0 && shape != QUAD && shape != HEX) return false;
    std::memset(blob, 0, sizeof(double) * L.total);
    const double *z1 = z.data(), *z2 = z.data() + Q, *z3 = z.data() + 2 * Q;
    for (int k = 0; k < Q; ++k)
        for (int r = 0; r < N; ++r) blob[L.Ba + k * N + r] = basis ? nirb_nodal_pair(r, N, z1[k]) : nirb_psiA(r, z1[k]);
    if (shape == TRI || shape == TET || shape == PRISM || shape == PYR) {
        const double *zb = (shape == PRISM || shape == PYR) ? z3 : z2;
        for (int p = 0; p < N; ++p) {
            const int nc = cls_cols(N, p);
            double *T = blob + L.Bb + cls_off(N, Q, p);
            for (int j = 0; j < Q; ++j)
                for (int q = 0; q < nc; ++q) T[j * nc + q] = nirb_psiB(p, q, zb[j]);
        }
    }
    if (shape == TET) {
        for (int c = 0; c < N; ++c) {
            const int nc = cls_cols(N, c);
            double *T = blob + L.Bc + cls_off(N, Q, c);
            for (int k = 0; k < Q; ++k)
                for (int r = 0; r < nc; ++r) T[k * nc + r] = nirb_psiB(c, r, z3[k]);
        }
    }
    nirb_colloc(Q, z1, blob + L.D1);
    if (shape == TRI || shape == TET) nirb_colloc(Q, z2, blob + L.D2);
    if (shape == TET || shape == PRISM || shape == PYR) nirb_colloc(Q, z3, blob + L.D3);
    // even/odd form of Ba (the first-direction points are symmetric for every shape)
    {
        const int ne = sym_ne(N), no = sym_no(N), w = ne + no;
        for (int i = 0; i < (Q + 1) / 2; ++i) {
            const double *B = blob + L.Ba + i * N;
            double *R = blob + L.Bs + i * w;
            R[0] = 0.5 * (B[0] + B[1]);
            for (int k = 1; k < ne; ++k) R[k] = B[2 * k];
            R[ne] = 0.5 * (B[0] - B[1]);
            for (int k = 1; k < no; ++k) R[ne + k] = B[2 * k + 1];
        }
    }
    const int d = dim(shape);
    for (int n = 0; n < npts(shape, Q); ++n) {
        int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
        blob[L.wq + n] = w[i] * w[Q + j] * (d == 3 ? w[2 * Q + k] : 1.0);
    }
    return true;
}

int nirb_table_size(int shape, int P, int Q) { return nirk::layout(shape, P + 1, Q).total; }
