/*
 * oracle.c -- plain, slow, FP64 CPU reference for the spectral/hp elemental
 * operators (BwdTrans, IProductWRTBase, PhysDeriv, IProductWRTDerivBase, mass,
 * Helmholtz) on quadrilaterals, triangles, hexahedra, prisms, tetrahedra and
 * pyramids.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, imports or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA path.
 *
 * Every operator is evaluated through dense elemental matrices built directly
 * from the basis definitions (no sum-factorisation):
 *   B[n][m]      = phi_m(xi_n)                                  (Sec. 2.1, Eq. basis matrix)
 *   dB_i[n][m]   = d phi_m / d xi_i at xi_n, differentiated analytically,
 *                  through the collapsed-coordinate chain rule  (Sec. 2.2, the
 *                  D_xi = Lambda(d eta/d xi) D_eta relation)
 *   W[n]         = w_n |J(xi_n)|                                (Sec. 2.1, weights matrix)
 *   Lambda       = d xi / d x at every point                   (Sec. 2.1, Eq. physderiv)
 *   H            = sum_l (D_xl B)^T W (D_xl B) + lambda B^T W B (Eqs. weakmatrixhelm, laplacian)
 * PhysDeriv of arbitrary point data uses collocation differentiation through
 * the element's own points (Eq. stdderiv) with the same chain rule.
 *
 * Readings of points the paper leaves open:
 *   - H = L + lambda M with lambda > 0 (Eq. weakmatrixhelm; the sign printed
 *     in Eq. weak_helm is not used).
 *   - eta1 = 2(1+xi1)/(-xi2-xi3) - 1 for the tet (Eq. eta-space lacks the -1).
 *   - P is the polynomial degree, N = P+1 modes per direction.
 *   - modes are packed lexicographically, p outermost, then q, then r, with
 *     q < N-p and r < N-p-q for the tet (Eq. bwdsumfactet bounds).
 *   - modified C0 basis; collapsed-vertex/edge modes whose eta factor is not a
 *     polynomial in xi are defined with that factor replaced by 1.
 *   - quadrature: GLL on tensor directions, Gauss-Jacobi(alpha,0) on collapsed
 *     directions with the collapse Jacobian absorbed in the weights.
 *   - pyramid (a shape the paper motivates and leaves to future work): apex at
 *     xi = (-1,-1,1), eta1 = 2(1+xi1)/(1-xi3) - 1, eta2 = 2(1+xi2)/(1-xi3) - 1,
 *     eta3 = xi3; modes p, q < N, r < N - max(p,q), phi_pqr =
 *     psiA_p(eta1) psiA_q(eta2) psiB_(max(p,q)) r(eta3), the apex mode (0,0,1)
 *     being psiA_1(eta3) alone; GLL in eta1, eta2 and Gauss-Jacobi(2,0) in
 *     eta3 with the collapse Jacobian ((1-eta3)/2)^2 in the weights; the
 *     element map is the vertex map of the five vertex functions (rational in
 *     xi; affine for a parallelogram base).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_QUAD = 0, ORC_TRI = 1, ORC_HEX = 2, ORC_PRISM = 3, ORC_TET = 4, ORC_PYR = 5 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ESING = -3 };

#define ORC_MAXQ 16
#define ORC_MAXP 12

static int orc_dim(int shape) { return (shape == ORC_QUAD || shape == ORC_TRI) ? 2 : 3; }

static int shape_ok(int shape) { return shape >= ORC_QUAD && shape <= ORC_PYR; }

int orc_num_modes(int shape, int P)
{
    int N = P + 1;
    if (!shape_ok(shape) || P < 1 || P > ORC_MAXP) return ORC_EINVAL;
    switch (shape) {
    case ORC_QUAD: return N * N;
    case ORC_TRI: return N * (N + 1) / 2;
    case ORC_HEX: return N * N * N;
    case ORC_PRISM: return N * N * (N + 1) / 2;
    case ORC_PYR: return N * (N + 1) * (2 * N + 1) / 6;   /* sum over c = max(p,q) of (2c+1)(N-c) */
    default: return N * (N + 1) * (N + 2) / 6;
    }
}

int orc_num_points(int shape, int Q)
{
    if (!shape_ok(shape) || Q < 2 || Q > ORC_MAXQ) return ORC_EINVAL;
    return orc_dim(shape) == 2 ? Q * Q : Q * Q * Q;
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Jacobi polynomials P_n^{(a,b)} by the three-term recurrence, and quadrature.
 * ------------------------------------------------------------------------- */
double orc_jacobi(int n, double a, double b, double x)
{
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * (a - b + (a + b + 2.0) * x);
    for (int k = 1; k < n; ++k) {
        double s = 2.0 * k + a + b;
        double c1 = 2.0 * (k + 1) * (k + a + b + 1.0) * s;
        double c2 = (s + 1.0) * (a * a - b * b);
        double c3 = s * (s + 1.0) * (s + 2.0);
        double c4 = 2.0 * (k + a) * (k + b) * (s + 2.0);
        double p2 = ((c2 + c3 * x) * p1 - c4 * p0) / c1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/* d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)} */
double orc_jacobi_deriv(int n, double a, double b, double x)
{
    if (n == 0) return 0.0;
    return 0.5 * (n + a + b + 1.0) * orc_jacobi(n - 1, a + 1.0, b + 1.0, x);
}

/* Zeros of P_n^{(a,b)}, ascending: Newton iteration with deflation by the
 * zeros already found, started from the Chebyshev-Gauss points. */
static void jacobi_zeros(int n, double a, double b, double *z)
{
    for (int k = 0; k < n; ++k) {
        double r = -cos((2.0 * k + 1.0) * M_PI / (2.0 * n));
        if (k > 0) r = 0.5 * (r + z[k - 1]);
        for (int it = 0; it < 200; ++it) {
            double s = 0.0;
            for (int i = 0; i < k; ++i) s += 1.0 / (r - z[i]);
            double f = orc_jacobi(n, a, b, r);
            double df = orc_jacobi_deriv(n, a, b, r);
            double delta = -f / (df - s * f);
            r += delta;
            if (fabs(delta) < 1e-16 * (1.0 + fabs(r))) break;
        }
        z[k] = r;
    }
}

/* Gauss-Jacobi rule (interior points) for the weight (1-x)^a (1+x)^b. */
static void gauss_jacobi(int Q, double a, double b, double *z, double *w)
{
    jacobi_zeros(Q, a, b, z);
    double lc = (a + b + 1.0) * log(2.0) + lgamma(a + Q + 1.0) + lgamma(b + Q + 1.0)
              - lgamma(Q + 1.0) - lgamma(a + b + Q + 1.0);
    double C = exp(lc);
    for (int i = 0; i < Q; ++i) {
        double dp = orc_jacobi_deriv(Q, a, b, z[i]);
        w[i] = C / ((1.0 - z[i] * z[i]) * dp * dp);
    }
}

/* Gauss-Lobatto-Legendre rule: +-1 and the zeros of P_{Q-2}^{(1,1)};
 * w_i = 2 / (Q (Q-1) P_{Q-1}(x_i)^2). */
static void gauss_lobatto(int Q, double *z, double *w)
{
    z[0] = -1.0;
    z[Q - 1] = 1.0;
    if (Q > 2) jacobi_zeros(Q - 2, 1.0, 1.0, z + 1);
    for (int i = 0; i < Q; ++i) {
        double p = orc_jacobi(Q - 1, 0.0, 0.0, z[i]);
        w[i] = 2.0 / ((double)Q * (Q - 1) * p * p);
    }
}

/* kind 0: GLL; kind 1 + alpha: Gauss-Jacobi(alpha, 0), alpha = 0, 1, 2. */
int orc_quad_rule(int kind, int Q, double *z, double *w)
{
    if (Q < 2 || Q > ORC_MAXQ || kind < 0 || kind > 3) return ORC_EINVAL;
    if (kind == 0) gauss_lobatto(Q, z, w);
    else gauss_jacobi(Q, (double)(kind - 1), 0.0, z, w);
    return ORC_OK;
}

/* Per-direction rule of each shape and the collapse factor absorbed in w. */
static void shape_rules(int shape, int Q, double z[3][ORC_MAXQ], double w[3][ORC_MAXQ])
{
    int kinds[3] = {0, 0, 0};
    double scale[3] = {1.0, 1.0, 1.0};
    switch (shape) {
    case ORC_TRI: kinds[0] = 1; kinds[1] = 2; scale[1] = 0.5; break;          /* (1-eta2)/2 */
    case ORC_PRISM: kinds[2] = 2; scale[2] = 0.5; break;                      /* (1-eta3)/2 */
    case ORC_TET: kinds[0] = 1; kinds[1] = 2; kinds[2] = 3;                   /* (1-eta2)/2 ((1-eta3)/2)^2 */
        scale[1] = 0.5; scale[2] = 0.25; break;
    case ORC_PYR: kinds[2] = 3; scale[2] = 0.25; break;                       /* ((1-eta3)/2)^2 */
    default: break;
    }
    for (int d = 0; d < 3; ++d) {
        orc_quad_rule(kinds[d], Q, z[d], w[d]);
        for (int i = 0; i < Q; ++i) w[d][i] *= scale[d];
    }
}

/* eta -> xi for the collapsed shapes (identity for quad/hex). */
static void eta_to_xi(int shape, const double *e, double *x)
{
    switch (shape) {
    case ORC_TRI:
        x[0] = 0.5 * (1.0 + e[0]) * (1.0 - e[1]) - 1.0;
        x[1] = e[1];
        break;
    case ORC_PRISM:
        x[0] = 0.5 * (1.0 + e[0]) * (1.0 - e[2]) - 1.0;
        x[1] = e[1];
        x[2] = e[2];
        break;
    case ORC_TET:
        x[0] = 0.25 * (1.0 + e[0]) * (1.0 - e[1]) * (1.0 - e[2]) - 1.0;
        x[1] = 0.5 * (1.0 + e[1]) * (1.0 - e[2]) - 1.0;
        x[2] = e[2];
        break;
    case ORC_PYR:
        x[0] = 0.5 * (1.0 + e[0]) * (1.0 - e[2]) - 1.0;
        x[1] = 0.5 * (1.0 + e[1]) * (1.0 - e[2]) - 1.0;
        x[2] = e[2];
        break;
    default:
        for (int i = 0; i < orc_dim(shape); ++i) x[i] = e[i];
    }
}

/* xi -> eta (defined away from the collapsed vertex/edge). */
static void xi_to_eta(int shape, const double *x, double *e)
{
    switch (shape) {
    case ORC_TRI:
        e[0] = 2.0 * (1.0 + x[0]) / (1.0 - x[1]) - 1.0;
        e[1] = x[1];
        break;
    case ORC_PRISM:
        e[0] = 2.0 * (1.0 + x[0]) / (1.0 - x[2]) - 1.0;
        e[1] = x[1];
        e[2] = x[2];
        break;
    case ORC_TET:
        e[0] = 2.0 * (1.0 + x[0]) / (-x[1] - x[2]) - 1.0;
        e[1] = 2.0 * (1.0 + x[1]) / (1.0 - x[2]) - 1.0;
        e[2] = x[2];
        break;
    case ORC_PYR:
        e[0] = 2.0 * (1.0 + x[0]) / (1.0 - x[2]) - 1.0;
        e[1] = 2.0 * (1.0 + x[1]) / (1.0 - x[2]) - 1.0;
        e[2] = x[2];
        break;
    default:
        for (int i = 0; i < orc_dim(shape); ++i) e[i] = x[i];
    }
}

/* A[j][i] = d eta_j / d xi_i at a point given in eta coordinates. */
static void deta_dxi(int shape, const double *e, double A[3][3])
{
    memset(A, 0, 9 * sizeof(double));
    for (int i = 0; i < 3; ++i) A[i][i] = 1.0;
    switch (shape) {
    case ORC_TRI:
        A[0][0] = 2.0 / (1.0 - e[1]);
        A[0][1] = (1.0 + e[0]) / (1.0 - e[1]);
        break;
    case ORC_PRISM:
        A[0][0] = 2.0 / (1.0 - e[2]);
        A[0][2] = (1.0 + e[0]) / (1.0 - e[2]);
        break;
    case ORC_TET: {
        double s = (1.0 - e[1]) * (1.0 - e[2]); /* = 2(-xi2-xi3) */
        A[0][0] = 4.0 / s;
        A[0][1] = 2.0 * (1.0 + e[0]) / s;
        A[0][2] = 2.0 * (1.0 + e[0]) / s;
        A[1][1] = 2.0 / (1.0 - e[2]);
        A[1][2] = (1.0 + e[1]) / (1.0 - e[2]);
        break;
    }
    case ORC_PYR:
        A[0][0] = 2.0 / (1.0 - e[2]);
        A[0][2] = (1.0 + e[0]) / (1.0 - e[2]);
        A[1][1] = 2.0 / (1.0 - e[2]);
        A[1][2] = (1.0 + e[1]) / (1.0 - e[2]);
        break;
    default: break;
    }
}

/* ---------------------------------------------------------------------------
 * Modified C0 basis (1-D factors with analytic derivatives).
 *   psiA_p: (1-z)/2, (1+z)/2, (1-z)/2 (1+z)/2 P^{(1,1)}_{p-2}(z)
 *   psiB_pq: psiA_q for p = 0; ((1-z)/2)^p for q = 0;
 *            ((1-z)/2)^p (1+z)/2 P^{(2p-1,1)}_{q-1}(z) otherwise.
 * The tet's third factor psiC_pqr is psiB_(p+q) r.
 * ------------------------------------------------------------------------- */
static void psiA(int p, double z, double *f, double *df)
{
    if (p == 0) { *f = 0.5 * (1.0 - z); *df = -0.5; return; }
    if (p == 1) { *f = 0.5 * (1.0 + z); *df = 0.5; return; }
    double g = 0.25 * (1.0 - z) * (1.0 + z), dg = -0.5 * z;
    double J = orc_jacobi(p - 2, 1.0, 1.0, z), dJ = orc_jacobi_deriv(p - 2, 1.0, 1.0, z);
    *f = g * J;
    *df = dg * J + g * dJ;
}

static void psiB(int p, int q, double z, double *f, double *df)
{
    if (p == 0) { psiA(q, z, f, df); return; }
    double h = pow(0.5 * (1.0 - z), p);
    double dh = -0.5 * p * pow(0.5 * (1.0 - z), p - 1);
    if (q == 0) { *f = h; *df = dh; return; }
    double a = 2.0 * p - 1.0;
    double J = orc_jacobi(q - 1, a, 1.0, z), dJ = orc_jacobi_deriv(q - 1, a, 1.0, z);
    double u = 0.5 * (1.0 + z);
    *f = h * u * J;
    *df = dh * u * J + h * 0.5 * J + h * u * dJ;
}

/* Mode list: (p,q,r) in packed order, p outermost. */
static int mode_list(int shape, int P, int (*pqr)[3])
{
    int N = P + 1, m = 0;
    switch (shape) {
    case ORC_QUAD:
        for (int p = 0; p < N; ++p) for (int q = 0; q < N; ++q) { pqr[m][0] = p; pqr[m][1] = q; pqr[m][2] = 0; ++m; }
        break;
    case ORC_TRI:
        for (int p = 0; p < N; ++p) for (int q = 0; q < N - p; ++q) { pqr[m][0] = p; pqr[m][1] = q; pqr[m][2] = 0; ++m; }
        break;
    case ORC_HEX:
        for (int p = 0; p < N; ++p) for (int q = 0; q < N; ++q) for (int r = 0; r < N; ++r) {
            pqr[m][0] = p; pqr[m][1] = q; pqr[m][2] = r; ++m; }
        break;
    case ORC_PRISM:
        for (int p = 0; p < N; ++p) for (int q = 0; q < N; ++q) for (int r = 0; r < N - p; ++r) {
            pqr[m][0] = p; pqr[m][1] = q; pqr[m][2] = r; ++m; }
        break;
    case ORC_TET:
        for (int p = 0; p < N; ++p) for (int q = 0; q < N - p; ++q) for (int r = 0; r < N - p - q; ++r) {
            pqr[m][0] = p; pqr[m][1] = q; pqr[m][2] = r; ++m; }
        break;
    case ORC_PYR:
        for (int p = 0; p < N; ++p) for (int q = 0; q < N; ++q) for (int r = 0; r < N - (p > q ? p : q); ++r) {
            pqr[m][0] = p; pqr[m][1] = q; pqr[m][2] = r; ++m; }
        break;
    }
    return m;
}

/* phi_m and d phi_m / d eta_j at a point in eta coordinates. */
static void mode_eval_eta(int shape, const int *pqr, const double *e, double *f, double *g)
{
    int p = pqr[0], q = pqr[1], r = pqr[2];
    double a, da, b, db, c, dc;
    g[0] = g[1] = g[2] = 0.0;
    switch (shape) {
    case ORC_QUAD:
        psiA(p, e[0], &a, &da); psiA(q, e[1], &b, &db);
        *f = a * b; g[0] = da * b; g[1] = a * db;
        break;
    case ORC_HEX:
        psiA(p, e[0], &a, &da); psiA(q, e[1], &b, &db); psiA(r, e[2], &c, &dc);
        *f = a * b * c; g[0] = da * b * c; g[1] = a * db * c; g[2] = a * b * dc;
        break;
    case ORC_TRI:
        psiB(p, q, e[1], &b, &db);
        if (p == 0 && q == 1) { a = 1.0; da = 0.0; }          /* collapsed vertex */
        else psiA(p, e[0], &a, &da);
        *f = a * b; g[0] = da * b; g[1] = a * db;
        break;
    case ORC_PRISM:
        psiA(q, e[1], &b, &db); psiB(p, r, e[2], &c, &dc);
        if (p == 0 && r == 1) { a = 1.0; da = 0.0; }          /* collapsed edge */
        else psiA(p, e[0], &a, &da);
        *f = a * b * c; g[0] = da * b * c; g[1] = a * db * c; g[2] = a * b * dc;
        break;
    case ORC_TET:
        if (p == 0 && q == 0 && r == 1) {                      /* collapsed top vertex */
            psiA(1, e[2], &c, &dc);
            *f = c; g[2] = dc;
            break;
        }
        psiB(p, q, e[1], &b, &db); psiB(p + q, r, e[2], &c, &dc);
        if (p == 0 && q == 1) { a = 1.0; da = 0.0; }          /* collapsed edge */
        else psiA(p, e[0], &a, &da);
        *f = a * b * c; g[0] = da * b * c; g[1] = a * db * c; g[2] = a * b * dc;
        break;
    case ORC_PYR:
        if (p == 0 && q == 0 && r == 1) {                      /* apex: eta1, eta2 factors dropped */
            psiA(1, e[2], &c, &dc);
            *f = c; g[2] = dc;
            break;
        }
        psiA(p, e[0], &a, &da); psiA(q, e[1], &b, &db); psiB(p > q ? p : q, r, e[2], &c, &dc);
        *f = a * b * c; g[0] = da * b * c; g[1] = a * db * c; g[2] = a * b * dc;
        break;
    }
}

/* phi and grad_xi phi at a point given in eta coordinates (chain rule). */
static void mode_eval(int shape, const int *pqr, const double *e, double *f, double *gx)
{
    double ge[3], A[3][3];
    mode_eval_eta(shape, pqr, e, f, ge);
    deta_dxi(shape, e, A);
    int d = orc_dim(shape);
    for (int i = 0; i < d; ++i) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) s += A[j][i] * ge[j];
        gx[i] = s;
    }
}

/* Reference points: eta, xi coordinates and weights (collapse factor included). */
int orc_ref_points(int shape, int Q, double *eta, double *xi, double *w)
{
    int nq = orc_num_points(shape, Q);
    if (nq < 0) return nq;
    double z[3][ORC_MAXQ], wz[3][ORC_MAXQ];
    shape_rules(shape, Q, z, wz);
    int d = orc_dim(shape);
    for (int n = 0; n < nq; ++n) {
        int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
        double e[3] = {z[0][i], z[1][j], d == 3 ? z[2][k] : 0.0}, x[3];
        eta_to_xi(shape, e, x);
        for (int c = 0; c < d; ++c) {
            if (eta) eta[n * d + c] = e[c];
            if (xi) xi[n * d + c] = x[c];
        }
        if (w) w[n] = wz[0][i] * wz[1][j] * (d == 3 ? wz[2][k] : 1.0);
    }
    return ORC_OK;
}

/* Basis and xi-gradient at npts points given in xi coordinates:
 * B[n][m], dB[i][n][m]. */
int orc_eval_basis(int shape, int P, int npts, const double *xi, double *B, double *dB)
{
    int M = orc_num_modes(shape, P);
    if (M < 0) return M;
    int d = orc_dim(shape);
    int (*pqr)[3] = malloc(sizeof(int[3]) * M);
    if (!pqr) return ORC_ENOMEM;
    mode_list(shape, P, pqr);
    for (int n = 0; n < npts; ++n) {
        double e[3] = {0, 0, 0};
        xi_to_eta(shape, xi + n * d, e);
        for (int m = 0; m < M; ++m) {
            double f, gx[3];
            mode_eval(shape, pqr[m], e, &f, gx);
            if (B) B[(size_t)n * M + m] = f;
            if (dB) for (int i = 0; i < d; ++i) dB[((size_t)i * npts + n) * M + m] = gx[i];
        }
    }
    free(pqr);
    return ORC_OK;
}

/* Basis and xi-gradient at the quadrature points (evaluated in eta, so the
 * collapsed points need no division by zero). */
int orc_ref_basis(int shape, int P, int Q, double *B, double *dB)
{
    int M = orc_num_modes(shape, P), nq = orc_num_points(shape, Q);
    if (M < 0 || nq < 0) return ORC_EINVAL;
    int d = orc_dim(shape);
    double *eta = malloc(sizeof(double) * nq * d);
    int (*pqr)[3] = malloc(sizeof(int[3]) * M);
    if (!eta || !pqr) { free(eta); free(pqr); return ORC_ENOMEM; }
    orc_ref_points(shape, Q, eta, NULL, NULL);
    mode_list(shape, P, pqr);
    for (int n = 0; n < nq; ++n) {
        double e[3] = {0, 0, 0};
        for (int c = 0; c < d; ++c) e[c] = eta[n * d + c];
        for (int m = 0; m < M; ++m) {
            double f, gx[3];
            mode_eval(shape, pqr[m], e, &f, gx);
            if (B) B[(size_t)n * M + m] = f;
            if (dB) for (int i = 0; i < d; ++i) dB[((size_t)i * nq + n) * M + m] = gx[i];
        }
    }
    free(eta);
    free(pqr);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Lagrange interpolation through arbitrary nodes (collocation differentiation
 * and the tensor-lattice element map).
 * ------------------------------------------------------------------------- */
static double lagrange(const double *t, int n, int a, double x)
{
    double v = 1.0;
    for (int b = 0; b < n; ++b) if (b != a) v *= (x - t[b]) / (t[a] - t[b]);
    return v;
}

static double lagrange_deriv(const double *t, int n, int a, double x)
{
    double s = 0.0;
    for (int c = 0; c < n; ++c) {
        if (c == a) continue;
        double v = 1.0 / (t[a] - t[c]);
        for (int b = 0; b < n; ++b) if (b != a && b != c) v *= (x - t[b]) / (t[a] - t[b]);
        s += v;
    }
    return s;
}

/* 1-D collocation derivative matrix D[i][j] = l_j'(z_i). */
int orc_colloc_1d(int Q, const double *z, double *D)
{
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) D[i * Q + j] = lagrange_deriv(z, Q, j, z[i]);
    return ORC_OK;
}

/* Dense xi-collocation derivative operators Dxi[i][n][n'] on the element's
 * points: D_xi_i = sum_j Lambda(d eta_j / d xi_i) D_eta_j. */
static int colloc_dense(int shape, int Q, double *Dxi)
{
    int nq = orc_num_points(shape, Q), d = orc_dim(shape);
    double z[3][ORC_MAXQ], wz[3][ORC_MAXQ], D1[3][ORC_MAXQ * ORC_MAXQ];
    shape_rules(shape, Q, z, wz);
    for (int c = 0; c < d; ++c) orc_colloc_1d(Q, z[c], D1[c]);
    memset(Dxi, 0, sizeof(double) * (size_t)d * nq * nq);
    for (int n = 0; n < nq; ++n) {
        int ii[3] = {n % Q, (n / Q) % Q, n / (Q * Q)};
        double e[3] = {z[0][ii[0]], z[1][ii[1]], d == 3 ? z[2][ii[2]] : 0.0}, A[3][3];
        deta_dxi(shape, e, A);
        for (int j = 0; j < d; ++j) {          /* D_eta_j contribution */
            for (int s = 0; s < Q; ++s) {
                int jj[3] = {ii[0], ii[1], ii[2]};
                jj[j] = s;
                int np = jj[0] + Q * jj[1] + (d == 3 ? Q * Q * jj[2] : 0);
                double dj = D1[j][ii[j] * Q + s];
                for (int i = 0; i < d; ++i)
                    Dxi[((size_t)i * nq + n) * nq + np] += A[j][i] * dj;
            }
        }
    }
    return ORC_OK;
}

int orc_colloc_deriv(int shape, int Q, double *Dxi)
{
    if (orc_num_points(shape, Q) < 0) return ORC_EINVAL;
    return colloc_dense(shape, Q, Dxi);
}

/* ---------------------------------------------------------------------------
 * Geometry: dx/dxi at a reference point from the element's nodes.
 * J[l][i] = d x_l / d xi_i.
 * ------------------------------------------------------------------------- */
static void element_jacobian(int shape, int gorder, const double *nodes, const double *xi,
                             double J[3][3], double *x)
{
    int d = orc_dim(shape);
    memset(J, 0, 9 * sizeof(double));
    if (x) for (int l = 0; l < d; ++l) x[l] = 0.0;
    if (shape == ORC_QUAD || shape == ORC_HEX) {
        int g1 = gorder + 1;
        double t[ORC_MAXQ];
        for (int a = 0; a < g1; ++a) t[a] = -1.0 + 2.0 * a / gorder;
        double L[3][ORC_MAXQ], dL[3][ORC_MAXQ];
        for (int c = 0; c < d; ++c)
            for (int a = 0; a < g1; ++a) {
                L[c][a] = lagrange(t, g1, a, xi[c]);
                dL[c][a] = lagrange_deriv(t, g1, a, xi[c]);
            }
        int nn = d == 2 ? g1 * g1 : g1 * g1 * g1;
        for (int v = 0; v < nn; ++v) {
            int ab[3] = {v % g1, (v / g1) % g1, v / (g1 * g1)};
            double phi = 1.0, gr[3];
            for (int c = 0; c < d; ++c) phi *= L[c][ab[c]];
            for (int i = 0; i < d; ++i) {
                gr[i] = 1.0;
                for (int c = 0; c < d; ++c) gr[i] *= (c == i) ? dL[c][ab[c]] : L[c][ab[c]];
            }
            for (int l = 0; l < d; ++l) {
                double X = nodes[v * d + l];
                if (x) x[l] += X * phi;
                for (int i = 0; i < d; ++i) J[l][i] += X * gr[i];
            }
        }
        return;
    }
    /* vertex maps: value and gradient of each vertex function */
    double N[6], G[6][3];
    int nv = 0;
    memset(G, 0, sizeof(G));
    if (shape == ORC_TRI) {
        nv = 3;
        N[0] = -0.5 * (xi[0] + xi[1]); G[0][0] = -0.5; G[0][1] = -0.5;
        N[1] = 0.5 * (1.0 + xi[0]);    G[1][0] = 0.5;
        N[2] = 0.5 * (1.0 + xi[1]);    G[2][1] = 0.5;
    } else if (shape == ORC_TET) {
        nv = 4;
        N[0] = -0.5 * (1.0 + xi[0] + xi[1] + xi[2]); G[0][0] = G[0][1] = G[0][2] = -0.5;
        N[1] = 0.5 * (1.0 + xi[0]); G[1][0] = 0.5;
        N[2] = 0.5 * (1.0 + xi[1]); G[2][1] = 0.5;
        N[3] = 0.5 * (1.0 + xi[2]); G[3][2] = 0.5;
    } else if (shape == ORC_PYR) {
        /* vertices (-1,-1,-1), (1,-1,-1), (1,1,-1), (-1,1,-1), apex (-1,-1,1):
         * base functions a_i b_j (1-xi3)/2 with a_0 = (-xi1-xi3)/(1-xi3),
         * a_1 = (1+xi1)/(1-xi3) (b likewise in xi2), apex (1+xi3)/2; written
         * as N = u v / (2 s), s = 1 - xi3, and differentiated by the quotient
         * rule. */
        nv = 5;
        double s = 1.0 - xi[2];
        double u[2] = {-xi[0] - xi[2], 1.0 + xi[0]}, du1[2] = {-1.0, 1.0}, du3[2] = {-1.0, 0.0};
        double v[2] = {-xi[1] - xi[2], 1.0 + xi[1]}, dv2[2] = {-1.0, 1.0}, dv3[2] = {-1.0, 0.0};
        int ai[4] = {0, 1, 1, 0}, bj[4] = {0, 0, 1, 1};
        for (int k = 0; k < 4; ++k) {
            double uu = u[ai[k]], vv = v[bj[k]];
            N[k] = uu * vv / (2.0 * s);
            G[k][0] = du1[ai[k]] * vv / (2.0 * s);
            G[k][1] = uu * dv2[bj[k]] / (2.0 * s);
            /* d/dxi3 of uu vv / (2 s) with ds/dxi3 = -1 */
            G[k][2] = (du3[ai[k]] * vv + uu * dv3[bj[k]]) / (2.0 * s) + uu * vv / (2.0 * s * s);
        }
        N[4] = 0.5 * (1.0 + xi[2]);
        G[4][2] = 0.5;
    } else { /* prism: triangle (xi1, xi3) x segment xi2 */
        nv = 6;
        double T[3] = {-0.5 * (xi[0] + xi[2]), 0.5 * (1.0 + xi[0]), 0.5 * (1.0 + xi[2])};
        double dT[3][2] = {{-0.5, -0.5}, {0.5, 0.0}, {0.0, 0.5}}; /* d/dxi1, d/dxi3 */
        double S[2] = {0.5 * (1.0 - xi[1]), 0.5 * (1.0 + xi[1])}, dS[2] = {-0.5, 0.5};
        int tv[6] = {0, 1, 1, 0, 2, 2}, sv[6] = {0, 0, 1, 1, 0, 1};
        for (int v = 0; v < 6; ++v) {
            N[v] = T[tv[v]] * S[sv[v]];
            G[v][0] = dT[tv[v]][0] * S[sv[v]];
            G[v][1] = T[tv[v]] * dS[sv[v]];
            G[v][2] = dT[tv[v]][1] * S[sv[v]];
        }
    }
    for (int v = 0; v < nv; ++v)
        for (int l = 0; l < d; ++l) {
            double X = nodes[v * d + l];
            if (x) x[l] += X * N[v];
            for (int i = 0; i < d; ++i) J[l][i] += X * G[v][i];
        }
}

static double det_inv(int d, double J[3][3], double Ji[3][3])
{
    if (d == 2) {
        double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
        return det;
    }
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    Ji[0][0] = c00 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = c01 / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = c02 / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    return det;
}

static int nodes_per_elem(int shape, int gorder)
{
    int d = orc_dim(shape);
    if (shape == ORC_QUAD || shape == ORC_HEX) {
        if (gorder < 1 || gorder > ORC_MAXQ - 1) return ORC_EINVAL;
        return d == 2 ? (gorder + 1) * (gorder + 1) : (gorder + 1) * (gorder + 1) * (gorder + 1);
    }
    if (gorder != 1) return ORC_EINVAL;
    return shape == ORC_TRI ? 3 : shape == ORC_TET ? 4 : shape == ORC_PYR ? 5 : 6;
}

/* Per-point W = w |J| and Lambda[n][i][l] = d xi_i / d x_l of one element.
 * Returns ORC_ESING on a non-positive Jacobian. */
static int elem_geometry(int shape, int Q, int gorder, const double *nodes, const double *xi,
                         const double *wq, int nq, double *W, double *Lam, double *xp)
{
    int d = orc_dim(shape), bad = 0;
    for (int n = 0; n < nq; ++n) {
        double J[3][3], Ji[3][3], x[3];
        element_jacobian(shape, gorder, nodes, xi + n * d, J, x);
        double det = det_inv(d, J, Ji);
        if (!(det > 0.0)) bad = 1;
        W[n] = wq[n] * det;
        for (int i = 0; i < d; ++i)
            for (int l = 0; l < d; ++l) Lam[(n * d + i) * d + l] = Ji[i][l];
        if (xp) for (int l = 0; l < d; ++l) xp[n * d + l] = x[l];
    }
    (void)Q;
    return bad ? ORC_ESING : ORC_OK;
}

int orc_geom_factors(int shape, int Q, int E, int gorder, const double *nodes,
                     double *W, double *dxi_dx, double *xphys)
{
    int nq = orc_num_points(shape, Q), npe = nodes_per_elem(shape, gorder);
    if (nq < 0 || npe < 0 || E < 0) return ORC_EINVAL;
    int d = orc_dim(shape), err = 0;
    double *xi = malloc(sizeof(double) * nq * d), *wq = malloc(sizeof(double) * nq);
    if (!xi || !wq) { free(xi); free(wq); return ORC_ENOMEM; }
    orc_ref_points(shape, Q, NULL, xi, wq);
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int e = 0; e < E; ++e) {
        int rc = elem_geometry(shape, Q, gorder, nodes + (size_t)e * npe * d, xi, wq, nq,
                               W + (size_t)e * nq, dxi_dx + (size_t)e * nq * d * d,
                               xphys ? xphys + (size_t)e * nq * d : NULL);
        if (rc) err |= 1;
    }
    free(xi);
    free(wq);
    return err ? ORC_ESING : ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Block operators through dense elemental matrices.
 * ------------------------------------------------------------------------- */
typedef struct {
    int shape, P, Q, d, M, nq, npe, gorder;
    double *B, *dB, *xi, *wq, *Dxi;
} refel;

static int refel_init(refel *r, int shape, int P, int Q, int gorder, int need_colloc)
{
    memset(r, 0, sizeof(*r));
    r->shape = shape; r->P = P; r->Q = Q; r->gorder = gorder;
    r->d = orc_dim(shape);
    r->M = P > 0 ? orc_num_modes(shape, P) : 0;
    r->nq = orc_num_points(shape, Q);
    r->npe = gorder > 0 ? nodes_per_elem(shape, gorder) : 0;
    if (r->M < 0 || r->nq < 0 || r->npe < 0) return ORC_EINVAL;
    r->xi = malloc(sizeof(double) * r->nq * r->d);
    r->wq = malloc(sizeof(double) * r->nq);
    if (!r->xi || !r->wq) return ORC_ENOMEM;
    orc_ref_points(shape, Q, NULL, r->xi, r->wq);
    if (r->M > 0) {
        r->B = malloc(sizeof(double) * r->nq * r->M);
        r->dB = malloc(sizeof(double) * r->d * r->nq * r->M);
        if (!r->B || !r->dB) return ORC_ENOMEM;
        orc_ref_basis(shape, P, Q, r->B, r->dB);
    }
    if (need_colloc) {
        r->Dxi = malloc(sizeof(double) * r->d * r->nq * r->nq);
        if (!r->Dxi) return ORC_ENOMEM;
        colloc_dense(shape, Q, r->Dxi);
    }
    return ORC_OK;
}

static void refel_free(refel *r)
{
    free(r->B); free(r->dB); free(r->xi); free(r->wq); free(r->Dxi);
}

int orc_bwd(int shape, int P, int Q, int E, const double *coeff, double *phys)
{
    refel r;
    int rc = refel_init(&r, shape, P, Q, 0, 0);
    if (rc) { refel_free(&r); return rc; }
#pragma omp parallel for schedule(static)
    for (int e = 0; e < E; ++e) {
        const double *u = coeff + (size_t)e * r.M;
        double *out = phys + (size_t)e * r.nq;
        for (int n = 0; n < r.nq; ++n) {
            double s = 0.0;
            for (int m = 0; m < r.M; ++m) s += r.B[(size_t)n * r.M + m] * u[m];
            out[n] = s;
        }
    }
    refel_free(&r);
    return ORC_OK;
}

/* Physical-space derivative matrices of one element: DxB[l][n][m]. */
static void phys_basis_grad(const refel *r, const double *Lam, double *DxB)
{
    int d = r->d;
    for (int l = 0; l < d; ++l)
        for (int n = 0; n < r->nq; ++n)
            for (int m = 0; m < r->M; ++m) {
                double s = 0.0;
                for (int i = 0; i < d; ++i)
                    s += Lam[(n * d + i) * d + l] * r->dB[((size_t)i * r->nq + n) * r->M + m];
                DxB[((size_t)l * r->nq + n) * r->M + m] = s;
            }
}

enum { OP_IPROD, OP_PHYSDERIV, OP_IPROD_DERIV, OP_MASS, OP_HELM, OP_HELM_MATRIX, OP_HELM_SOLVE };

static int cholesky_solve(int M, double *H, const double *b, double *x)
{
    for (int j = 0; j < M; ++j) {
        double s = H[(size_t)j * M + j];
        for (int k = 0; k < j; ++k) s -= H[(size_t)j * M + k] * H[(size_t)j * M + k];
        if (!(s > 0.0)) return ORC_ESING;
        double ljj = sqrt(s);
        H[(size_t)j * M + j] = ljj;
        for (int i = j + 1; i < M; ++i) {
            double t = H[(size_t)i * M + j];
            for (int k = 0; k < j; ++k) t -= H[(size_t)i * M + k] * H[(size_t)j * M + k];
            H[(size_t)i * M + j] = t / ljj;
        }
    }
    for (int i = 0; i < M; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= H[(size_t)i * M + k] * x[k];
        x[i] = t / H[(size_t)i * M + i];
    }
    for (int i = M - 1; i >= 0; --i) {
        double t = x[i];
        for (int k = i + 1; k < M; ++k) t -= H[(size_t)k * M + i] * x[k];
        x[i] = t / H[(size_t)i * M + i];
    }
    return ORC_OK;
}

static int run_op(int op, int shape, int P, int Q, int E, int gorder, const double *nodes,
                  double lambda, const double *in, double *out)
{
    refel r;
    int rc = refel_init(&r, shape, P, Q, gorder, op == OP_PHYSDERIV);
    if (rc) { refel_free(&r); return rc; }
    int d = r.d, M = r.M, nq = r.nq, err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (int e = 0; e < E; ++e) {
        double *W = malloc(sizeof(double) * nq);
        double *Lam = malloc(sizeof(double) * nq * d * d);
        double *DxB = (M > 0) ? malloc(sizeof(double) * d * nq * M) : NULL;
        double *t = malloc(sizeof(double) * (size_t)(d + 1) * nq);
        double *H = (op == OP_HELM_MATRIX || op == OP_HELM_SOLVE) ? malloc(sizeof(double) * M * M) : NULL;
        if (!W || !Lam || !t || (M > 0 && !DxB) ||
            ((op == OP_HELM_MATRIX || op == OP_HELM_SOLVE) && !H)) {
            err |= 2;
        } else if (elem_geometry(shape, Q, gorder, nodes + (size_t)e * r.npe * d, r.xi, r.wq, nq,
                                 W, Lam, NULL)) {
            err |= 1;
        } else {
            if (M > 0) phys_basis_grad(&r, Lam, DxB);
            switch (op) {
            case OP_IPROD: {
                const double *f = in + (size_t)e * nq;
                double *y = out + (size_t)e * M;
                for (int m = 0; m < M; ++m) {
                    double s = 0.0;
                    for (int n = 0; n < nq; ++n) s += r.B[(size_t)n * M + m] * W[n] * f[n];
                    y[m] = s;
                }
                break;
            }
            case OP_PHYSDERIV: {
                const double *u = in + (size_t)e * nq;
                for (int i = 0; i < d; ++i)
                    for (int n = 0; n < nq; ++n) {
                        double s = 0.0;
                        for (int np = 0; np < nq; ++np) s += r.Dxi[((size_t)i * nq + n) * nq + np] * u[np];
                        t[i * nq + n] = s;
                    }
                for (int l = 0; l < d; ++l)
                    for (int n = 0; n < nq; ++n) {
                        double s = 0.0;
                        for (int i = 0; i < d; ++i) s += Lam[(n * d + i) * d + l] * t[i * nq + n];
                        out[((size_t)l * E + e) * nq + n] = s;
                    }
                break;
            }
            case OP_IPROD_DERIV: {
                double *y = out + (size_t)e * M;
                for (int m = 0; m < M; ++m) {
                    double s = 0.0;
                    for (int l = 0; l < d; ++l) {
                        const double *f = in + ((size_t)l * E + e) * nq;
                        for (int n = 0; n < nq; ++n) s += DxB[((size_t)l * nq + n) * M + m] * W[n] * f[n];
                    }
                    y[m] = s;
                }
                break;
            }
            case OP_MASS:
            case OP_HELM: {
                const double *u = in + (size_t)e * M;
                double *y = out + (size_t)e * M;
                /* t[0..nq) = B u ; t[(1+l) nq ..) = DxB_l u */
                for (int n = 0; n < nq; ++n) {
                    double s = 0.0;
                    for (int m = 0; m < M; ++m) s += r.B[(size_t)n * M + m] * u[m];
                    t[n] = s;
                }
                if (op == OP_HELM)
                    for (int l = 0; l < d; ++l)
                        for (int n = 0; n < nq; ++n) {
                            double s = 0.0;
                            for (int m = 0; m < M; ++m) s += DxB[((size_t)l * nq + n) * M + m] * u[m];
                            t[(1 + l) * nq + n] = s;
                        }
                double lam = (op == OP_HELM) ? lambda : 1.0;
                for (int m = 0; m < M; ++m) {
                    double s = 0.0;
                    for (int n = 0; n < nq; ++n) s += lam * r.B[(size_t)n * M + m] * W[n] * t[n];
                    if (op == OP_HELM)
                        for (int l = 0; l < d; ++l)
                            for (int n = 0; n < nq; ++n)
                                s += DxB[((size_t)l * nq + n) * M + m] * W[n] * t[(1 + l) * nq + n];
                    y[m] = s;
                }
                break;
            }
            case OP_HELM_MATRIX:
            case OP_HELM_SOLVE: {
                for (int a = 0; a < M; ++a)
                    for (int b = 0; b < M; ++b) {
                        double s = 0.0;
                        for (int n = 0; n < nq; ++n) {
                            double g = lambda * r.B[(size_t)n * M + a] * r.B[(size_t)n * M + b];
                            for (int l = 0; l < d; ++l)
                                g += DxB[((size_t)l * nq + n) * M + a] * DxB[((size_t)l * nq + n) * M + b];
                            s += W[n] * g;
                        }
                        H[(size_t)a * M + b] = s;
                    }
                if (op == OP_HELM_MATRIX) {
                    memcpy(out + (size_t)e * M * M, H, sizeof(double) * M * M);
                } else if (cholesky_solve(M, H, in + (size_t)e * M, out + (size_t)e * M)) {
                    err |= 4;
                }
                break;
            }
            }
        }
        free(W); free(Lam); free(DxB); free(t); free(H);
    }
    refel_free(&r);
    if (err & 2) return ORC_ENOMEM;
    if (err & 5) return ORC_ESING;
    return ORC_OK;
}

int orc_iprod(int shape, int P, int Q, int E, int gorder, const double *nodes,
              const double *phys, double *coeff)
{ return run_op(OP_IPROD, shape, P, Q, E, gorder, nodes, 0.0, phys, coeff); }

int orc_physderiv(int shape, int Q, int E, int gorder, const double *nodes,
                  const double *phys, double *deriv)
{ return run_op(OP_PHYSDERIV, shape, 0, Q, E, gorder, nodes, 0.0, phys, deriv); }

int orc_iprod_deriv(int shape, int P, int Q, int E, int gorder, const double *nodes,
                    const double *f, double *coeff)
{ return run_op(OP_IPROD_DERIV, shape, P, Q, E, gorder, nodes, 0.0, f, coeff); }

int orc_mass(int shape, int P, int Q, int E, int gorder, const double *nodes,
             const double *in, double *out)
{ return run_op(OP_MASS, shape, P, Q, E, gorder, nodes, 0.0, in, out); }

int orc_helmholtz(int shape, int P, int Q, int E, int gorder, const double *nodes,
                  double lambda, const double *in, double *out)
{ return run_op(OP_HELM, shape, P, Q, E, gorder, nodes, lambda, in, out); }

int orc_helmholtz_matrix(int shape, int P, int Q, int E, int gorder, const double *nodes,
                         double lambda, double *H)
{ return run_op(OP_HELM_MATRIX, shape, P, Q, E, gorder, nodes, lambda, NULL, H); }

int orc_helmholtz_solve(int shape, int P, int Q, int E, int gorder, const double *nodes,
                        double lambda, const double *b, double *x)
{ return run_op(OP_HELM_SOLVE, shape, P, Q, E, gorder, nodes, lambda, b, x); }
