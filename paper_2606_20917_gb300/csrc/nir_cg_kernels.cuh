// nir_cg_kernels.cuh -- the CG solver's device code: the scalar block, the
// block and grid reductions, and the vector kernels (updates, dot products,
// residual, scaling, probing).  Included by nir_cg.cu after its headers (and
// by a host emulation of these kernels in the tests); not a public header.
namespace {

using nirv::st_v;
using nirv::to_d;

// Device-side CG scalars.  With `defer` set (a solve sharded across ranks)
// the reduction kernels only publish this rank's partial sums (pAp; rzn and
// rr) and the host, after summing them over the ranks, writes alpha and beta
// back; `done` then stays 0 and the host ends the loop.
struct CGScal {
    double rz, pAp, alpha, beta, rr, thresh;
    int done, bad, iters, defer;
    double rzn;
};

constexpr int kThreads = 256;

// Block-wide sum of NV doubles; the result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV])
{
    __shared__ double sh[NV][kThreads / 32];
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][wid] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += sh[k][w];
            v[k] = s;
        }
    __syncthreads();
}

// Publish this CTA's partials; returns true in thread 0 of the last CTA,
// with the totals in tot.  The last CTA sums the partials with all its
// threads (thread t takes CTAs t, t + blockDim, ...) and a block reduction:
// a fixed order for a fixed grid, so results are deterministic.
template <int NV>
__device__ __forceinline__ bool finish_reduce(double (&v)[NV], double *part, unsigned *ticket, double (&tot)[NV])
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        acc[k] = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) acc[k] += __ldcg(part + k * gridDim.x + b);
    }
    block_sum(acc);
    if (threadIdx.x != 0) return false;
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = acc[k];
    *ticket = 0u;
    return true;
}

// The vector kernels are bound by memory latency unless every thread keeps
// several independent loads in flight: each grid-stride step handles kU
// elements i0 + k * stride (coalesced across the warp for every k), loading
// all operands before any arithmetic.
//
// Arithmetic follows the vectors' type.  FP64 vectors (plain CG) compute in
// FP64.  FP32 vectors (the inner solver of the refinement) compute their
// updates in FP32: GB300's FP64 rate is a small fraction of its FP32 rate and
// conversions to and from FP64 run on the same pipe, so FP64 arithmetic per
// element would bound these kernels.  Their dot products keep FP64-level
// accuracy without FP64 operations per element: each thread accumulates
// exact products (TwoProduct by FMA) with compensated summation (TwoSum) in a
// pair of floats -- the Dot2 algorithm of Ogita, Rump and Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 26 (2005) -- and the per-thread
// results are summed in FP64.
constexpr int kU = 4;

struct FF {
    float hi = 0.0f, lo = 0.0f;
};

__device__ __forceinline__ void ff_add_prod(FF &s, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);  // a * b = p + e exactly
    const float t = __fadd_rn(s.hi, p);
    const float bb = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));  // s.hi + p = t + err
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}

__device__ __forceinline__ double ff_value(const FF &s) { return (double)s.hi + (double)s.lo; }

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ void st_f(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_f(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// pAp = p . Ap ; alpha = rz / pAp
template <class V, class T>
__global__ void __launch_bounds__(kThreads) k_alpha(const V *__restrict__ p, const T *__restrict__ Ap, long long n,
                                                    double *part, unsigned *ticket, CGScal *s)
{
    if (s->done) return;
    const long long S = (long long)gridDim.x * kThreads;
    double v[1] = {0.0};
    FF acc;
    for (long long i0 = blockIdx.x * (long long)kThreads + threadIdx.x; i0 < n; i0 += S * kU) {
        V pv[kU];
        T av[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S, j = i < n ? i : i0;  // in-range dummy for the tail
            pv[k] = p[j];
            av[k] = Ap[j];
        }
#pragma unroll
        for (int k = 0; k < kU; ++k)
            if (i0 + k * S < n) {
                if constexpr (std::is_same<V, double>::value) v[0] += to_d(pv[k]) * to_d(av[k]);
                else ff_add_prod(acc, pv[k], to_f(av[k]));
            }
    }
    if constexpr (!std::is_same<V, double>::value) v[0] = ff_value(acc);
    block_sum(v);
    double t[1];
    if (finish_reduce(v, part, ticket, t)) {
        s->pAp = t[0];
        if (s->defer) return;
        if (!isfinite(t[0])) { s->bad = 2; s->done = 1; }
        else if (!(t[0] > 0.0)) { s->bad = 1; s->done = 1; }
        else s->alpha = s->rz / t[0];
    }
}

// x += alpha p; r -= alpha Ap; z = dinv r; rz' = r.z; rr = r.r; beta = rz'/rz
template <class V, class T>
__global__ void __launch_bounds__(kThreads, sizeof(V) == 8 ? 3 : 4) k_update(V *__restrict__ x, V *__restrict__ r,
                                                     V *__restrict__ z,
                                                     const V *__restrict__ p, const T *__restrict__ Ap,
                                                     const V *__restrict__ dinv, long long n, double *part,
                                                     unsigned *ticket, CGScal *s)
{
    if (s->done) return;
    const double a = s->alpha;
    const float af = (float)a;
    const long long S = (long long)gridDim.x * kThreads;
    double v[2] = {0.0, 0.0};
    FF arz, arr;
    for (long long i0 = blockIdx.x * (long long)kThreads + threadIdx.x; i0 < n; i0 += S * kU) {
        V xv[kU], pv[kU], rv[kU], dv[kU];
        T av[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S, j = i < n ? i : i0;  // in-range dummy for the tail
            xv[k] = x[j];
            pv[k] = p[j];
            rv[k] = r[j];
            av[k] = Ap[j];
            if (dinv) dv[k] = dinv[j];
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S;
            if (i >= n) continue;
            if constexpr (std::is_same<V, double>::value) {
                x[i] = xv[k] + a * pv[k];
                const double ri = rv[k] - a * to_d(av[k]);
                r[i] = ri;
                double zi = ri;
                if (dinv) {
                    zi = dv[k] * ri;
                    z[i] = zi;
                }
                v[0] += ri * zi;
                v[1] += ri * ri;
            } else {
                x[i] = fmaf(af, pv[k], xv[k]);
                const float ri = fmaf(-af, to_f(av[k]), rv[k]);
                r[i] = ri;
                float zi = ri;
                if (dinv) {
                    zi = dv[k] * ri;
                    z[i] = zi;
                }
                ff_add_prod(arz, ri, zi);
                ff_add_prod(arr, ri, ri);
            }
        }
    }
    if constexpr (!std::is_same<V, double>::value) {
        v[0] = ff_value(arz);
        v[1] = ff_value(arr);
    }
    block_sum(v);
    double t[2];
    if (finish_reduce(v, part, ticket, t)) {
        if (s->defer) {
            s->rzn = t[0];
            s->rr = t[1];
            return;
        }
        s->beta = t[0] / s->rz;
        s->rz = t[0];
        s->rr = t[1];
        s->iters += 1;
        if (!isfinite(t[0]) || !isfinite(t[1])) { s->bad = 2; s->done = 1; }
        else if (t[1] <= s->thresh) s->done = 1;
    }
}

// p = z + beta p ; pT = p in the operator's storage type
template <class V, class T>
__global__ void __launch_bounds__(kThreads) k_pupdate(V *__restrict__ p, const V *__restrict__ z, T *__restrict__ pT,
                                                      long long n, const CGScal *s)
{
    if (s->done) return;
    const double b = s->beta;
    const float bf = (float)b;
    const long long S = (long long)gridDim.x * kThreads;
    for (long long i0 = blockIdx.x * (long long)kThreads + threadIdx.x; i0 < n; i0 += S * kU) {
        V zv[kU], pv[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S, j = i < n ? i : i0;
            zv[k] = z[j];
            pv[k] = p[j];
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S;
            if (i >= n) continue;
            if constexpr (std::is_same<V, double>::value) {
                const double pi = zv[k] + b * pv[k];
                p[i] = pi;
                if (pT) st_v(pT + i, pi);
            } else {
                const float pi = fmaf(bf, pv[k], zv[k]);
                p[i] = pi;
                if (pT) st_f(pT + i, pi);
            }
        }
    }
}

// start of a CG run: r given; z = dinv r; p = z; rz, rr
template <class V, class T>
__global__ void __launch_bounds__(kThreads) k_start(const V *__restrict__ r, V *__restrict__ z, V *__restrict__ p,
                                                    T *__restrict__ pT, const V *__restrict__ dinv, long long n,
                                                    double *part, unsigned *ticket, CGScal *s, double thresh,
                                                    int defer)
{
    const long long S = (long long)gridDim.x * kThreads;
    double v[2] = {0.0, 0.0};
    FF arz, arr;
    for (long long i0 = blockIdx.x * (long long)kThreads + threadIdx.x; i0 < n; i0 += S * kU) {
        V rv[kU], dv[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S, j = i < n ? i : i0;
            rv[k] = r[j];
            if (dinv) dv[k] = dinv[j];
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S;
            if (i >= n) continue;
            V zi = rv[k];
            if (dinv) {
                zi = dv[k] * rv[k];
                z[i] = zi;
            }
            p[i] = zi;
            if constexpr (std::is_same<V, double>::value) {
                if (pT) st_v(pT + i, zi);
                v[0] += rv[k] * zi;
                v[1] += rv[k] * rv[k];
            } else {
                if (pT) st_f(pT + i, zi);
                ff_add_prod(arz, rv[k], zi);
                ff_add_prod(arr, rv[k], rv[k]);
            }
        }
    }
    if constexpr (!std::is_same<V, double>::value) {
        v[0] = ff_value(arz);
        v[1] = ff_value(arr);
    }
    block_sum(v);
    double t[2];
    if (finish_reduce(v, part, ticket, t)) {
        s->rz = t[0];
        s->rr = t[1];
        s->thresh = thresh;
        s->iters = 0;
        s->defer = defer;
        s->bad = (isfinite(t[0]) && isfinite(t[1])) ? 0 : 2;
        s->done = (!defer && (s->bad || t[1] <= thresh)) ? 1 : 0;
    }
}

// out[0] = a . b (FP64)
template <class V>
__global__ void __launch_bounds__(kThreads) k_dot(const V *__restrict__ a, const V *__restrict__ b, long long n,
                                                  double *part, unsigned *ticket, double *out)
{
    const long long S = (long long)gridDim.x * kThreads;
    double v[1] = {0.0};
    for (long long i0 = blockIdx.x * (long long)kThreads + threadIdx.x; i0 < n; i0 += S * kU) {
        V av[kU], bv[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S, j = i < n ? i : i0;
            av[k] = a[j];
            bv[k] = b[j];
        }
#pragma unroll
        for (int k = 0; k < kU; ++k)
            if (i0 + k * S < n) v[0] += to_d(av[k]) * to_d(bv[k]);
    }
    block_sum(v);
    double t[1];
    if (finish_reduce(v, part, ticket, t)) *out = t[0];
}

// r = b - Ax (FP64)
__global__ void k_residual(double *r, const double *b, const double *Ax, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = b[i] - Ax[i];
}

// out = scale * r in the inner solver's vector type (out may be r for FP64)
template <class V>
__global__ void k_scale_to(V *out, const double *r, double scale, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        st_v(out + i, scale * r[i]);
}

// x += scale * d
template <class V>
__global__ void k_correct(double *x, const V *d, double scale, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += scale * to_d(d[i]);
}

// out[0] = |a - b|^2, out[1] = |a|^2 (FP64)
__global__ void __launch_bounds__(kThreads) k_diff_norms(const double *__restrict__ a, const double *__restrict__ b,
                                                         long long n, double *part, unsigned *ticket, double *out)
{
    const long long S = (long long)gridDim.x * kThreads;
    double v[2] = {0.0, 0.0};
    for (long long i0 = blockIdx.x * (long long)kThreads + threadIdx.x; i0 < n; i0 += S * kU) {
        double av[kU], bv[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S, j = i < n ? i : i0;
            av[k] = a[j];
            bv[k] = b[j];
        }
#pragma unroll
        for (int k = 0; k < kU; ++k)
            if (i0 + k * S < n) {
                const double d = av[k] - bv[k];
                v[0] += d * d;
                v[1] += av[k] * av[k];
            }
    }
    block_sum(v);
    double t[2];
    if (finish_reduce(v, part, ticket, t)) {
        out[0] = t[0];
        out[1] = t[1];
    }
}

template <class V>
__global__ void k_fill(V *x, double v, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        st_v(x + i, v);
}

// Probing: vector with 1 at mode m of every element of every block.
struct ProbeBlk {
    long long off, nelem;
    int M, pad;
};

template <class T>
__global__ void k_probe_fill(T *x, const ProbeBlk *pb, int nb, int m, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int b = 0;
        while (b + 1 < nb && pb[b + 1].off <= i) ++b;
        const long long j = (i - pb[b].off) % pb[b].M;
        st_v(x + i, j == m ? 1.0 : 0.0);
    }
}

template <class T>
__global__ void k_probe_gather(double *diag, const T *y, const ProbeBlk *pb, int nb, int m, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int b = 0;
        while (b + 1 < nb && pb[b + 1].off <= i) ++b;
        const long long j = (i - pb[b].off) % pb[b].M;
        if (j == m) diag[i] = to_d(y[i]);
    }
}

__global__ void k_invert(double *d64, float *d32, long long n, int *bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = d64[i];
        if (!(d > 0.0) || !isfinite(d)) atomicExch(bad, 1);
        const double inv = (d > 0.0) ? 1.0 / d : 1.0;
        d64[i] = inv;
        d32[i] = (float)inv;
    }
}

}  // namespace
