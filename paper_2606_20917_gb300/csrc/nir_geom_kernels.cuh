// nir_geom_kernels.cuh -- the geometry device code: point coordinates, vertex
// gradients, the factor kernels, precision conversion and packing, and the
// FP64 throughput probes.  Included by nir_geom.cu after its headers (and by a
// host emulation of the factor kernel in the tests); not a public header.
namespace nirk {

__device__ void vertex_grads(int shape, const double *xi, const double *eta, double G[6][3], int &nv)
{
    for (int v = 0; v < 6; ++v) G[v][0] = G[v][1] = G[v][2] = 0.0;
    if (shape == PYR) {
        // base vertices a_i(eta1) b_j(eta2) (1-eta3)/2 with a_0 = (1-eta1)/2,
        // a_1 = (1+eta1)/2 (b likewise), apex (1+eta3)/2; the eta-gradient is
        // taken to xi by d eta/d xi (eta1 and eta2 collapse with 1 - eta3)
        nv = 5;
        const double h = 0.5 * (1.0 - eta[2]), r = 1.0 / (1.0 - eta[2]);
        const double a[2] = {0.5 * (1.0 - eta[0]), 0.5 * (1.0 + eta[0])}, da[2] = {-0.5, 0.5};
        const double b[2] = {0.5 * (1.0 - eta[1]), 0.5 * (1.0 + eta[1])}, db[2] = {-0.5, 0.5};
        const int ai[4] = {0, 1, 1, 0}, bj[4] = {0, 0, 1, 1};
        for (int v = 0; v < 4; ++v) {
            const double g1 = da[ai[v]] * b[bj[v]] * h;   // d/d eta1
            const double g2 = a[ai[v]] * db[bj[v]] * h;   // d/d eta2
            const double g3 = -0.5 * a[ai[v]] * b[bj[v]]; // d/d eta3
            G[v][0] = g1 * 2.0 * r;
            G[v][1] = g2 * 2.0 * r;
            G[v][2] = g1 * (1.0 + eta[0]) * r + g2 * (1.0 + eta[1]) * r + g3;
        }
        G[4][2] = 0.5;
        return;
    }
    if (shape == TRI) {
        nv = 3;
        G[0][0] = G[0][1] = -0.5;
        G[1][0] = 0.5;
        G[2][1] = 0.5;
    } else if (shape == TET) {
        nv = 4;
        G[0][0] = G[0][1] = G[0][2] = -0.5;
        G[1][0] = 0.5;
        G[2][1] = 0.5;
        G[3][2] = 0.5;
    } else {  // prism: triangle (xi1, xi3) times segment xi2
        nv = 6;
        const double T[3] = {-0.5 * (xi[0] + xi[2]), 0.5 * (1.0 + xi[0]), 0.5 * (1.0 + xi[2])};
        const double dT1[3] = {-0.5, 0.5, 0.0}, dT3[3] = {-0.5, 0.0, 0.5};
        const double Sg[2] = {0.5 * (1.0 - xi[1]), 0.5 * (1.0 + xi[1])}, dS[2] = {-0.5, 0.5};
        const int tv[6] = {0, 1, 1, 0, 2, 2}, sv[6] = {0, 0, 1, 1, 0, 1};
        for (int v = 0; v < 6; ++v) {
            G[v][0] = dT1[tv[v]] * Sg[sv[v]];
            G[v][1] = T[tv[v]] * dS[sv[v]];
            G[v][2] = dT3[tv[v]] * Sg[sv[v]];
        }
    }
}

// Collapsed (eta) and standard-element (xi) coordinates of point n, and its
// per-direction indices ii.
__device__ void point_coords(const GeoArgs &a, int n, double eta[3], double xi[3], int ii[3])
{
    const int d = dim(a.shape), Q = a.Q;
    ii[0] = n % Q;
    ii[1] = (n / Q) % Q;
    ii[2] = n / (Q * Q);
    eta[0] = eta[1] = eta[2] = 0.0;
    xi[0] = xi[1] = xi[2] = 0.0;
    for (int c = 0; c < d; ++c) eta[c] = a.z[c * Q + ii[c]];
    // collapsed coordinates -> standard element (Eq. eta-space and its inverse)
    if (a.shape == TRI) {
        xi[0] = 0.5 * (1.0 + eta[0]) * (1.0 - eta[1]) - 1.0;
        xi[1] = eta[1];
    } else if (a.shape == PRISM) {
        xi[0] = 0.5 * (1.0 + eta[0]) * (1.0 - eta[2]) - 1.0;
        xi[1] = eta[1];
        xi[2] = eta[2];
    } else if (a.shape == TET) {
        xi[0] = 0.25 * (1.0 + eta[0]) * (1.0 - eta[1]) * (1.0 - eta[2]) - 1.0;
        xi[1] = 0.5 * (1.0 + eta[1]) * (1.0 - eta[2]) - 1.0;
        xi[2] = eta[2];
    } else if (a.shape == PYR) {
        xi[0] = 0.5 * (1.0 + eta[0]) * (1.0 - eta[2]) - 1.0;
        xi[1] = 0.5 * (1.0 + eta[1]) * (1.0 - eta[2]) - 1.0;
        xi[2] = eta[2];
    } else {
        for (int c = 0; c < d; ++c) xi[c] = eta[c];
    }
}

// From Ji[i][l] = d xi_i / d x_l and det = |J| at point n of element e: the
// collapsed factors d eta/d xi, d eta/d x = (d eta/d xi)(d xi/d x), W = w|J|
// (|J| alone for per-element factors) and G = W (d eta/d x)(d eta/d x)^T,
// stored in the library's layouts (per point interleaved by 32 elements, or
// per element).  A det that is not positive and finite raises the error flag.
__device__ void store_factors(const GeoArgs &a, long long e, int n, const double eta[3], const double Ji[3][3],
                              double det)
{
    const int d = dim(a.shape);
    const int NQ = npts(a.shape, a.Q);
    const int ng = ngeo(a.shape), nl = nlam(a.shape);
    if (!(det > 0.0) || !isfinite(det)) atomicExch(a.err, 1);
    // A[j][i] = d eta_j / d xi_i
    double A[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (a.shape == TRI) {
        A[0][0] = 2.0 / (1.0 - eta[1]);
        A[0][1] = (1.0 + eta[0]) / (1.0 - eta[1]);
    } else if (a.shape == PRISM) {
        A[0][0] = 2.0 / (1.0 - eta[2]);
        A[0][2] = (1.0 + eta[0]) / (1.0 - eta[2]);
    } else if (a.shape == TET) {
        const double s = (1.0 - eta[1]) * (1.0 - eta[2]);
        A[0][0] = 4.0 / s;
        A[0][1] = A[0][2] = 2.0 * (1.0 + eta[0]) / s;
        A[1][1] = 2.0 / (1.0 - eta[2]);
        A[1][2] = (1.0 + eta[1]) / (1.0 - eta[2]);
    } else if (a.shape == PYR) {
        A[0][0] = 2.0 / (1.0 - eta[2]);
        A[0][2] = (1.0 + eta[0]) / (1.0 - eta[2]);
        A[1][1] = 2.0 / (1.0 - eta[2]);
        A[1][2] = (1.0 + eta[1]) / (1.0 - eta[2]);
    }
    double Lm[3][3];
    for (int j = 0; j < d; ++j)
        for (int l = 0; l < d; ++l) {
            double s = 0.0;
            for (int i = 0; i < d; ++i) s = fma(A[j][i], Ji[i][l], s);
            Lm[j][l] = s;
        }
    const double W = (a.pp ? a.wq[n] : 1.0) * det;
    double gv[7];
    int c = 0;
    for (int i = 0; i < d; ++i)
        for (int j = i; j < d; ++j) {
            double s = 0.0;
            for (int l = 0; l < d; ++l) s = fma(Lm[i][l], Lm[j][l], s);
            gv[c++] = W * s;
        }
    gv[c] = W;
    if (a.pp) {
        const long long base = (e >> 5) * NQ + n;
        for (int q = 0; q < ng; ++q) a.G[((base * ng + q) << 5) + (e & 31)] = gv[q];
        for (int j = 0; j < d; ++j)
            for (int l = 0; l < d; ++l) a.Lam[((base * nl + j * d + l) << 5) + (e & 31)] = Lm[j][l];
        a.Lam[((base * nl + nl - 1) << 5) + (e & 31)] = W;
    } else {
        for (int q = 0; q < ng; ++q) a.G[e * ng + q] = gv[q];
        for (int j = 0; j < d; ++j)
            for (int l = 0; l < d; ++l) a.Lam[e * nl + j * d + l] = Lm[j][l];
        a.Lam[e * nl + nl - 1] = W;
    }
}

__global__ void k_geometry(GeoArgs a)
{
    const int d = dim(a.shape);
    const int NQ = npts(a.shape, a.Q);
    const long long total = a.pp ? a.nelem * NQ : a.nelem;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long e = a.pp ? t / NQ : t;
        const int n = a.pp ? (int)(t - e * NQ) : 0;
        const int Q = a.Q;
        int ii[3];
        double eta[3], xi[3];
        point_coords(a, n, eta, xi, ii);
        // J[l][i] = d x_l / d xi_i
        double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        if (a.shape == QUAD || a.shape == HEX) {
            const int g1 = a.g + 1;
            const int rows[3] = {a.pp ? ii[0] : Q, a.pp ? ii[1] : Q, a.pp ? ii[2] : Q};
            const int nn = d == 2 ? g1 * g1 : g1 * g1 * g1;
            const double *X = a.nodes + (size_t)e * nn * d;
            for (int v = 0; v < nn; ++v) {
                const int ab[3] = {v % g1, (v / g1) % g1, v / (g1 * g1)};
                double Lv[3], dLv[3];
                for (int c = 0; c < d; ++c) {
                    Lv[c] = a.Lg[rows[c] * g1 + ab[c]];
                    dLv[c] = a.dLg[rows[c] * g1 + ab[c]];
                }
                double gr[3];
                for (int i = 0; i < d; ++i) {
                    double p = 1.0;
                    for (int c = 0; c < d; ++c) p *= (c == i) ? dLv[c] : Lv[c];
                    gr[i] = p;
                }
                for (int l = 0; l < d; ++l) {
                    const double xl = X[v * d + l];
                    for (int i = 0; i < d; ++i) J[l][i] = fma(xl, gr[i], J[l][i]);
                }
            }
        } else {
            double Gv[6][3];
            int nv = 0;
            vertex_grads(a.shape, xi, eta, Gv, nv);
            const double *X = a.nodes + (size_t)e * nv * d;
            for (int v = 0; v < nv; ++v)
                for (int l = 0; l < d; ++l)
                    for (int i = 0; i < d; ++i) J[l][i] = fma(X[v * d + l], Gv[v][i], J[l][i]);
        }
        // determinant and inverse (Ji[i][l] = d xi_i / d x_l)
        double det, Ji[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        if (d == 2) {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
            Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
        } else {
            const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            const double c10 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            const double c20 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            det = J[0][0] * c00 + J[0][1] * c10 + J[0][2] * c20;
            const double r = 1.0 / det;
            Ji[0][0] = c00 * r;
            Ji[1][0] = c10 * r;
            Ji[2][0] = c20 * r;
            Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
            Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
            Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
            Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
            Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
            Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
        }
        store_factors(a, e, n, eta, Ji, det);
    }
}

// Factors given by the caller (Sec. 2.1: Lambda = d xi/d x and |J|), per
// point [E][NQ][d][d] / [E][NQ], or constant over each element [E][d][d] /
// [E] (per_elem).  The block's layout decides the units written: every
// point (a.pp) or every element.
__global__ void k_geometry_from_factors(GeoArgs a)
{
    const int d = dim(a.shape);
    const int NQ = npts(a.shape, a.Q);
    const long long total = a.pp ? a.nelem * NQ : a.nelem;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long e = a.pp ? t / NQ : t;
        const int n = a.pp ? (int)(t - e * NQ) : 0;
        int ii[3];
        double eta[3], xi[3];
        point_coords(a, n, eta, xi, ii);
        const long long u = a.per_elem ? e : e * NQ + n;
        const double *L = a.dxi_dx + u * d * d;
        double Ji[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int i = 0; i < d; ++i)
            for (int l = 0; l < d; ++l) Ji[i][l] = L[i * d + l];
        store_factors(a, e, n, eta, Ji, a.jac[u]);
    }
}

// FP64 interleaved per-point metric -> FP32/BF16 packed layout (the point
// blocks of 32 x ng values keep their place; values move within a block).
template <class T>
__global__ void k_pack_metric(const double *src, T *dst, long long nblocks, int ng)
{
    const long long n = nblocks * ng * 32;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long blk = i / (ng * 32);
        const int r = (int)(i - blk * ng * 32), c = r >> 5, l = r & 31;
        const long long o = blk * ng * 32 + geo_packed_off(c, l, ng);
        if constexpr (sizeof(T) == 4) dst[o] = __double2float_rn(src[i]);
        else dst[o] = __double2bfloat16(src[i]);
    }
}

__global__ void k_to_f32(const double *src, float *dst, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = __double2float_rn(src[i]);
}

__global__ void k_to_bf16(const double *src, __nv_bfloat16 *dst, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = __double2bfloat16(src[i]);
}

#ifdef __CUDACC__  // the throughput probes (inline PTX): device builds only

// Register-resident FP64 FMA chains: 8 independent recurrences per thread.
__global__ void __launch_bounds__(256) k_dfma_probe(double *sink, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == -1.2345) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

// Register-resident FP64 tensor-core (DMMA) chains: mma.sync m8n8k4 with FP64
// operands and accumulators, 8 independent accumulator pairs per thread.  Its
// rate next to the DFMA probe's decides whether FP64 contractions gain
// anything from the tensor pipe on this GPU.
__global__ void __launch_bounds__(256) k_dmma_probe(double *sink, int iters, double a, double b)
{
    double c[8][2];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        c[k][0] = 1e-3 * (threadIdx.x + k);
        c[k][1] = 2e-3 * (threadIdx.x + k);
    }
    const double av = a * (1.0 + 1e-3 * (threadIdx.x & 31)), bv = b;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(av), "d"(bv));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += c[k][0] + c[k][1];
    if (s == -1.2345) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

#endif  // __CUDACC__

}  // namespace nirk
