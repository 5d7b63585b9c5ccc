// Host emulation of one CTA of the threading-over-elements Helmholtz kernel
// (k_helm_toe in nir_toe.cuh), for the CPU test tests/test_toe_sim_cpu.py.
// Not part of the library.
//
// The kernel itself is compiled as plain C++ and run by its 128 threads as host
// threads over every warp of elements of a small case (warps that run out of
// elements leave the loop early, as on the GPU).  Between synchronisation
// points the threads run one at a time in a per-phase order (forward, reverse
// or shuffled; see cta_sim.cpp); __syncwarp is taken as a barrier of the
// threads still running, which is exact here because every warp still in the
// loop makes the same synchronisation calls per iteration.  The kernel's
// dynamic shared memory (tables and warp tiles), its global scratch
// (5 Q^d values per thread), the metric and the coefficient arrays are exactly
// sized heap blocks, and the build uses AddressSanitizer.
//
// argv: P prec (0 FP64, 1 FP32).  stdin: E geo_pp lambda, the metric
// (geo_pp: [E][Nq][NG], else [E][NG]; laid out here as the library stores it,
// FP32 per-point values packed) and the coefficients [E][M]; stdout: the
// result.  Environment: SIM_ORDER = fwd | rev | <shuffle seed>.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <pthread.h>
#include <semaphore.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <type_traits>
#include <utility>
#include <vector>
using std::fma;
#ifndef __noinline__  // after every standard header (they spell the attribute this way)
#define __noinline__ __attribute__((noinline))
#endif
#undef __launch_bounds__
#define __launch_bounds__(...)

struct HostDim {
    unsigned x, y, z;
};
static thread_local HostDim threadIdx;
static HostDim blockIdx, gridDim;

// One thread at a time between synchronisation points, in a per-phase order
// over the threads still running; a thread that returns leaves the rotation.
struct Sched {
    int mode = 0, turn = 0;
    unsigned long long seed = 0;
    long phase = 0;
    std::vector<int> active, perm;
    std::vector<sem_t> sem;
    void order(long ph)
    {
        perm = active;
        if (mode == 1) std::reverse(perm.begin(), perm.end());
        if (mode == 2) {  // Fisher-Yates with a 64-bit LCG (Knuth's MMIX constants)
            unsigned long long x = seed ^ (0x9E3779B97F4A7C15ULL * (unsigned long long)(ph + 1));
            for (int i = (int)perm.size() - 1; i > 0; --i) {
                x = x * 6364136223846793005ULL + 1442695040888963407ULL;
                const int j = (int)((x >> 33) % (unsigned long long)(i + 1));
                std::swap(perm[i], perm[j]);
            }
        }
    }
    void pass(int self, bool leaving)
    {
        if (leaving) active.erase(std::find(active.begin(), active.end(), self));
        if (++turn == (int)perm.size()) {
            turn = 0;
            order(++phase);
        }
        if (!perm.empty()) sem_post(&sem[perm[turn]]);
    }
};
static Sched g_sched;
static inline void sim_sync()
{
    const int t = (int)threadIdx.x;
    g_sched.pass(t, false);
    sem_wait(&g_sched.sem[t]);
}
static inline void __syncthreads() { sim_sync(); }
static inline void __syncwarp() { sim_sync(); }
template <class T>
static inline T __ldg(const T *p)
{
    return *p;
}

// The kernel's dynamic shared memory: an exactly sized heap block.
namespace nirt {
alignas(16) unsigned char (*g_toe_smem)[] = nullptr;
}
#define smraw (*g_toe_smem)
#include "nir_basis.h"
#include "nir_toe.cuh"
#undef smraw

#ifndef SIM_SHAPE
#error "SIM_SHAPE must be defined"
#endif

namespace {

void *xalloc(size_t bytes)
{
    void *p = nullptr;
    if (posix_memalign(&p, 64, bytes ? bytes : 1)) return nullptr;
    return p;
}

template <int SH, int N, class T>
int run()
{
    using A = typename nirt::CT<T>::type;
    constexpr int Q = N + 1, NQ = nirk::npts(SH, Q), M = nirk::nmodes(SH, N), NG = nirk::ngeo(SH);
    constexpr int NT = nirt::kThreads;
    long long E = 0;
    int pp = 1;
    double lam = 0;
    if (std::scanf("%lld %d %lf", &E, &pp, &lam) != 3 || E < 1) return 2;
    const long long epad = (E + 63) / 64 * 64;
    const int total = nirb_table_size(SH, N - 1, Q);
    std::vector<double> t64(total);
    if (!nirb_build_tables(SH, N - 1, Q, t64.data(), 0)) return 3;
    A *tab = static_cast<A *>(xalloc(sizeof(A) * total));
    for (int i = 0; i < total; ++i) tab[i] = (A)t64[i];
    const int per = (pp ? NQ : 1) * NG;
    std::vector<double> g((size_t)E * per);
    for (auto &v : g)
        if (std::scanf("%lf", &v) != 1) return 2;
    const size_t ngeo = (size_t)(pp ? epad * NQ : epad) * NG;
    T *geo = static_cast<T *>(xalloc(ngeo * sizeof(T)));
    for (long long e = 0; e < epad; ++e) {
        const long long es = e < E ? e : 0;
        for (int n = 0; n < (pp ? NQ : 1); ++n)
            for (int c = 0; c < NG; ++c) {
                const long long idx = !pp ? e * NG + c
                                      : sizeof(T) < 8 ? nirk::geo_packed_index(e, n, c, NQ, NG)  // FP32: packed
                                                      : ((((e >> 5) * NQ + n) * NG + c) << 5) + (e & 31);
                geo[idx] = (T)g[(size_t)es * per + (size_t)n * NG + c];
            }
    }
    T *in = static_cast<T *>(xalloc((size_t)E * M * sizeof(T)));
    T *out = static_cast<T *>(xalloc((size_t)E * M * sizeof(T)));
    for (long long i = 0; i < E * M; ++i) {
        double v;
        if (std::scanf("%lf", &v) != 1) return 2;
        in[i] = (T)v;
    }
    A *scr = static_cast<A *>(xalloc((size_t)nirt::kBufs * NQ * NT * sizeof(A)));  // one CTA's threads
    const int smem = nirt::toe_smem<SH, N, A>();
    nirt::g_toe_smem = reinterpret_cast<unsigned char (*)[]>(xalloc((size_t)smem));
    nirt::ToeArgs a{};
    a.in = in;
    a.out = out;
    a.geo = geo;
    a.tab = tab;
    a.scr = scr;
    a.nelem = E;
    a.lambda = lam;
    a.geo_pp = pp;
    blockIdx = HostDim{0, 0, 0};
    gridDim = HostDim{1, 1, 1};
    g_sched.active.clear();
    for (int t = 0; t < NT; ++t) g_sched.active.push_back(t);
    g_sched.sem = std::vector<sem_t>(NT);
    for (auto &x : g_sched.sem) sem_init(&x, 0, 0);
    g_sched.order(0);
    struct Arg {
        const nirt::ToeArgs *a;
        int t;
    };
    std::vector<pthread_t> th(NT);
    std::vector<Arg> args(NT);
    pthread_attr_t at;
    pthread_attr_init(&at);
    pthread_attr_setstacksize(&at, 2u << 20);
    for (int t = 0; t < NT; ++t) {
        args[t] = Arg{&a, t};
        if (pthread_create(&th[t], &at, [](void *p) -> void * {
                const Arg *r = static_cast<const Arg *>(p);
                threadIdx = HostDim{(unsigned)r->t, 0, 0};
                sem_wait(&g_sched.sem[r->t]);
                nirt::k_helm_toe<SH, N, T>(*r->a);
                g_sched.pass(r->t, true);
                return nullptr;
            }, &args[t]))
            return 5;
    }
    sem_post(&g_sched.sem[g_sched.perm[0]]);
    for (int t = 0; t < NT; ++t) pthread_join(th[t], nullptr);
    for (long long i = 0; i < E * M; ++i) std::printf("%.17g\n", (double)out[i]);
    std::free(tab);
    std::free(geo);
    std::free(in);
    std::free(out);
    std::free(scr);
    std::free(nirt::g_toe_smem);
    return 0;
}

template <class T>
int by_p(int P)
{
    switch (P + 1) {
    case 2: return run<SIM_SHAPE, 2, T>();
    case 3: return run<SIM_SHAPE, 3, T>();
    case 5: return run<SIM_SHAPE, 5, T>();
    case 7: return run<SIM_SHAPE, 7, T>();
    case 10: return run<SIM_SHAPE, 10, T>();
    default: return 4;
    }
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc != 3) return 1;
    if (const char *o = std::getenv("SIM_ORDER")) {
        if (!std::strcmp(o, "rev")) g_sched.mode = 1;
        else if (std::strcmp(o, "fwd")) {
            g_sched.mode = 2;
            g_sched.seed = std::strtoull(o, nullptr, 10);
        }
    }
    const int P = std::atoi(argv[1]), prec = std::atoi(argv[2]);
    return prec == 0 ? by_p<double>(P) : prec == 1 ? by_p<float>(P) : 1;
}
