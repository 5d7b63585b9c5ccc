// Host emulation of the CG solver's vector kernels (nir_cg.cu), for the CPU
// test tests/test_cg_sim_cpu.py.  Not part of the library.
//
// The kernels (nir_cg_kernels.cuh) are compiled as plain C++ and launched on a grid of a few CTAs
// of 256 host threads.  No CTA waits on another (each publishes a partial and
// the last one to take the ticket sums them), so the CTAs run one after
// another; within a CTA the threads run one at a time between barriers in a
// per-phase order (forward, reverse or shuffled; see cta_sim.cpp).  A warp
// shuffle is an exchange: every thread deposits its value, a barrier, every
// thread reads its source lane's, a barrier.  The per-CTA shared arrays are
// the kernels' own (static here: the CTAs run in turn).  Vectors, partials
// and scalars are exactly sized heap blocks; the build uses AddressSanitizer
// and no floating-point contraction (the compensated dot products rely on
// exactly rounded separate operations).
//
// argv: test prec grid.  stdin: n, then the vectors the test reads; stdout:
// its results (see tests/test_cg_sim_cpu.py).  Environment: SIM_ORDER.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <pthread.h>
#include <semaphore.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>
using std::fma;
using std::isfinite;
#ifndef __noinline__  // after every standard header (they spell the attribute this way)
#define __noinline__ __attribute__((noinline))
#endif
#undef __launch_bounds__
#define __launch_bounds__(...)
#undef __shared__
#define __shared__ static  // one CTA at a time: a kernel's shared arrays are per-function statics

struct HostDim {
    unsigned x, y, z;
};
static thread_local HostDim threadIdx;
static HostDim blockIdx, gridDim, blockDim;

// One thread at a time between barriers, in a per-phase order (see cta_sim.cpp).
struct Sched {
    int nt = 0, mode = 0, turn = 0;
    unsigned long long seed = 0;
    long phase = 0;
    std::vector<int> perm;
    std::vector<sem_t> sem;
    void order(long ph)
    {
        perm.resize(nt);
        for (int i = 0; i < nt; ++i) perm[i] = mode == 1 ? nt - 1 - i : i;
        if (mode == 2) {  // Fisher-Yates with a 64-bit LCG (Knuth's MMIX constants)
            unsigned long long x = seed ^ (0x9E3779B97F4A7C15ULL * (unsigned long long)(ph + 1));
            for (int i = nt - 1; i > 0; --i) {
                x = x * 6364136223846793005ULL + 1442695040888963407ULL;
                const int j = (int)((x >> 33) % (unsigned long long)(i + 1));
                std::swap(perm[i], perm[j]);
            }
        }
    }
    void pass()
    {
        if (++turn == nt) {
            turn = 0;
            order(++phase);
        }
        sem_post(&sem[perm[turn]]);
    }
};
static Sched g_sched;
static inline void __syncthreads()
{
    g_sched.pass();
    sem_wait(&g_sched.sem[(int)threadIdx.x]);
}
static double g_lanes[1024];
static inline double __shfl_down_sync(unsigned, double v, int o)
{
    const int t = (int)threadIdx.x;
    g_lanes[t] = v;
    __syncthreads();
    const double r = ((t & 31) + o < 32) ? g_lanes[t + o] : v;
    __syncthreads();
    return r;
}
static inline void __threadfence() {}
static inline double __ldcg(const double *p) { return *p; }
static inline unsigned atomicAdd(unsigned *p, unsigned v)
{
    const unsigned o = *p;
    *p += v;
    return o;
}
static inline float sim_fmul_rn(float a, float b) { return a * b; }
static inline float sim_fadd_rn(float a, float b) { return a + b; }
static inline float sim_fsub_rn(float a, float b) { return a - b; }
#define __fmul_rn(a, b) sim_fmul_rn(a, b)
#define __fadd_rn(a, b) sim_fadd_rn(a, b)
#define __fsub_rn(a, b) sim_fsub_rn(a, b)
static inline int atomicExch(int *p, int v)
{
    const int o = *p;
    *p = v;
    return o;
}
template <class T>
static inline T __ldg(const T *p)
{
    return *p;
}
template <class T>
static inline T __ldcs(const T *p)
{
    return *p;
}

// the headers nir_cg.cu includes before its device code, then that code
#include "nir_cg.h"
#include "nir_internal.h"
#include "nir_solve.h"
#include "nir_vec.cuh"
#include "nir_cg_kernels.cuh"

namespace {

void *xalloc(size_t bytes)
{
    void *p = nullptr;
    if (posix_memalign(&p, 64, bytes ? bytes : 1)) return nullptr;
    return p;
}

template <class T>
T *vec(long long n, bool read)
{
    T *v = static_cast<T *>(xalloc((size_t)n * sizeof(T)));
    for (long long i = 0; i < n; ++i) {
        double x = 0;
        if (read && std::scanf("%lf", &x) != 1) std::exit(2);
        v[i] = (T)x;
    }
    return v;
}

// Launch f(thread) on `grid` CTAs of kThreads threads, one CTA after another.
int launch(int grid, const std::function<void()> &kernel)
{
    const int NT = kThreads;
    gridDim = HostDim{(unsigned)grid, 1, 1};
    blockDim = HostDim{(unsigned)NT, 1, 1};
    for (int b = 0; b < grid; ++b) {
        blockIdx = HostDim{(unsigned)b, 0, 0};
        g_sched.nt = NT;
        g_sched.turn = 0;
        g_sched.sem = std::vector<sem_t>(NT);
        for (auto &x : g_sched.sem) sem_init(&x, 0, 0);
        g_sched.order(0);
        struct Arg {
            const std::function<void()> *f;
            int t;
        };
        std::vector<pthread_t> th(NT);
        std::vector<Arg> args(NT);
        for (int t = 0; t < NT; ++t) {
            args[t] = Arg{&kernel, t};
            if (pthread_create(&th[t], nullptr, [](void *p) -> void * {
                    const Arg *a = static_cast<const Arg *>(p);
                    threadIdx = HostDim{(unsigned)a->t, 0, 0};
                    sem_wait(&g_sched.sem[a->t]);
                    (*a->f)();
                    g_sched.pass();
                    return nullptr;
                }, &args[t]))
                return 5;
        }
        sem_post(&g_sched.sem[g_sched.perm[0]]);
        for (int t = 0; t < NT; ++t) pthread_join(th[t], nullptr);
        for (auto &x : g_sched.sem) sem_destroy(&x);
    }
    return 0;
}

// "dot": k_dot of a and b (FP64 accumulation of the stored values); for
// FP32 vectors also k_alpha's compensated p . Ap.
// "cg": one iteration: k_start, k_alpha, k_update, k_pupdate on r, dinv, Ap,
// x; prints rz rr pAp alpha beta, then x, r, z, p, pT.
template <class V>
int run(const char *test, int grid)
{
    long long n = 0;
    if (std::scanf("%lld", &n) != 1 || n < 1) return 2;
    double *part = static_cast<double *>(xalloc(sizeof(double) * 2 * grid));
    unsigned *ticket = static_cast<unsigned *>(xalloc(sizeof(unsigned)));
    *ticket = 0u;
    CGScal *s = static_cast<CGScal *>(xalloc(sizeof(CGScal)));
    std::memset(s, 0, sizeof(CGScal));
    if (!std::strcmp(test, "dot")) {
        V *a = vec<V>(n, true), *b = vec<V>(n, true);
        double *out = static_cast<double *>(xalloc(sizeof(double)));
        if (launch(grid, [&] { k_dot<V>(a, b, n, part, ticket, out); })) return 5;
        std::printf("%.17g\n", *out);
        s->rz = 1.0;
        if (launch(grid, [&] { k_alpha<V, V>(a, b, n, part, ticket, s); })) return 5;
        std::printf("%.17g\n", s->pAp);
        if (*ticket != 0u) return 7;
        std::free(a);
        std::free(b);
        std::free(out);
    } else {  // "cg"
        V *r = vec<V>(n, true), *dinv = vec<V>(n, true), *Ap = vec<V>(n, true), *x = vec<V>(n, true);
        V *z = vec<V>(n, false), *p = vec<V>(n, false), *pT = vec<V>(n, false);
        if (launch(grid, [&] { k_start<V, V>(r, z, p, pT, dinv, n, part, ticket, s, 0.0, 0); })) return 5;
        std::printf("%.17g %.17g\n", s->rz, s->rr);
        if (launch(grid, [&] { k_alpha<V, V>(p, Ap, n, part, ticket, s); })) return 5;
        std::printf("%.17g %.17g\n", s->pAp, s->alpha);
        if (launch(grid, [&] { k_update<V, V>(x, r, z, p, Ap, dinv, n, part, ticket, s); })) return 5;
        std::printf("%.17g %.17g %.17g\n", s->rz, s->rr, s->beta);
        if (launch(grid, [&] { k_pupdate<V, V>(p, z, pT, n, s); })) return 5;
        if (*ticket != 0u || s->bad || s->done) return 7;
        for (V *v : {x, r, z, p, pT})
            for (long long i = 0; i < n; ++i) std::printf("%.17g\n", (double)v[i]);
        for (V *v : {r, dinv, Ap, x, z, p, pT}) std::free(v);
    }
    std::free(part);
    std::free(ticket);
    std::free(s);
    return 0;
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc != 4) return 1;
    if (const char *o = std::getenv("SIM_ORDER")) {
        if (!std::strcmp(o, "rev")) g_sched.mode = 1;
        else if (std::strcmp(o, "fwd")) {
            g_sched.mode = 2;
            g_sched.seed = std::strtoull(o, nullptr, 10);
        }
    }
    const int prec = std::atoi(argv[2]), grid = std::atoi(argv[3]);
    if (grid < 1 || grid > 64) return 1;
    return prec == 0 ? run<double>(argv[1], grid) : prec == 1 ? run<float>(argv[1], grid) : 1;
}
