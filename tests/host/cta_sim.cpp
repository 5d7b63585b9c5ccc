// Host emulation of one CTA of the element-group kernels (nir_kernels.cuh),
// for the CPU test tests/test_cta_sim_cpu.py.  Not part of the library.
//
// The stage code of every operator (run_group and everything it calls) is
// compiled as plain C++ and run by NT host threads, one per CUDA thread.  One
// emulated CTA takes every element group in turn (so buffers are reused across
// groups, ragged last group included).  Shared memory is one exactly sized
// heap block, and every global array (inputs, outputs, metric) has exactly the
// size the library allocates or accepts, so built with AddressSanitizer any
// index outside shared memory or outside a global array ends the run with a
// report.  __syncthreads() hands the CTA to the next thread of a per-phase
// order (see Sched): runs in different orders must give the same bits, which
// they do unless two threads touch one shared word between the same two
// barriers (one of them writing).
// The FP32/BF16 Helmholtz runs the staged kernel's group loop (the bulk copy
// of the next group's coefficients into the staging buffer, issued by thread 0
// right after the barrier that frees it, becomes a memcpy at that point).
//
// argv: shape P op prec variant.  stdin: E geo_pp lambda nodal nfields, then
// the metric (geo_pp: [E][Nq][NG], else [E][NG]) and the inputs; stdout: the
// outputs (E = 0: prints the configuration's elements per group, threads per
// CTA, per-unit buffer stride and units per group instead).  Ops 0..5 as nirk::Op; prec 0 FP64, 1 FP32, 2 BF16;
// variant 0 the default group, 1 half, 2 double (Helmholtz only), 3 the
// persistent mesh kernel's form (fixed thread count, tables from shared
// memory), 5 two elements per thread (FP32/BF16 Helmholtz, quad and hex).
// Environment: SIM_ORDER = fwd | rev | <shuffle seed>.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <pthread.h>
#include <semaphore.h>

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

struct HostDim {
    unsigned x, y, z;
};
static thread_local HostDim threadIdx;
static HostDim blockIdx, gridDim;

// The CTA's threads run one at a time: between two barriers each thread runs
// alone, in an order fixed per barrier phase (forward, reverse, or a seeded
// shuffle), and hands over to the next thread of that order at its next
// barrier.  A correctly synchronised CTA gives the same bits in every order;
// a word written by one thread and read or written by another in the same
// phase (a missing barrier) gives results that depend on the order.
struct Sched {
    int nt = 0;
    int mode = 0;  // 0 forward, 1 reverse, 2 shuffled
    unsigned long long seed = 0;
    long phase = 0;
    int turn = 0;
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
                const int t = perm[i];
                perm[i] = perm[j];
                perm[j] = t;
            }
        }
    }
    // the running thread is done with this phase: wake the next one
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
// Planted mistakes that show the checks are live (test-only switches of this
// emulation): SIM_DROP_BARRIER=k makes every thread skip its k-th barrier;
// SIM_SHORT=smem / input allocates shared memory / the first input one
// element short.
static int g_drop = 0;
static thread_local int g_calls = 0;
static inline void __syncthreads()
{
    if (++g_calls == g_drop) return;
    const int t = (int)threadIdx.x;
    g_sched.pass();
    sem_wait(&g_sched.sem[t]);
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

#include "nir_basis.h"
#include "nir_kernels.cuh"

#ifndef SIM_SHAPE
#error "SIM_SHAPE must be defined"
#endif

using namespace nirk;

namespace {

template <class T>
T to_t(double v)
{
    if constexpr (sizeof(T) == 2) return __float2bfloat16_rn((float)v);
    else return (T)v;
}
template <class T>
double from_t(T v)
{
    if constexpr (sizeof(T) == 2) return (double)__bfloat162float(v);
    else return (double)v;
}

void *xalloc(size_t bytes)
{
    void *p = nullptr;
    if (posix_memalign(&p, 64, bytes ? bytes : 1)) return nullptr;
    return p;
}

// Run body(t) on NT threads (one at a time, see Sched).
int run_cta(int NT, const std::function<void(int)> &body)
{
    g_sched.nt = NT;
    g_sched.phase = 0;
    g_sched.turn = 0;
    g_sched.sem = std::vector<sem_t>(NT);
    for (auto &x : g_sched.sem) sem_init(&x, 0, 0);
    g_sched.order(0);
    struct Arg {
        const std::function<void(int)> *f;
        int t;
    };
    std::vector<pthread_t> th(NT);
    std::vector<Arg> args(NT);
    pthread_attr_t at;
    pthread_attr_init(&at);
    pthread_attr_setstacksize(&at, 1u << 20);
    for (int t = 0; t < NT; ++t) {
        args[t] = Arg{&body, t};
        if (pthread_create(&th[t], &at, [](void *p) -> void * {
                const Arg *a = static_cast<const Arg *>(p);
                threadIdx = HostDim{(unsigned)a->t, 0, 0};
                sem_wait(&g_sched.sem[a->t]);
                (*a->f)(a->t);
                g_sched.pass();  // leaving: the next thread of this phase runs
                return nullptr;
            }, &args[t]))
            return 5;
    }
    sem_post(&g_sched.sem[g_sched.perm[0]]);
    for (int t = 0; t < NT; ++t) pthread_join(th[t], nullptr);
    for (auto &x : g_sched.sem) sem_destroy(&x);
    pthread_attr_destroy(&at);
    return 0;
}

struct Input {
    long long E;
    int pp, nodal, nfields;
    double lambda;
};

template <int SH, int N, class T, int OP, int EPB_, int NT_, bool STAGE, bool MESH, bool PAIR = false>
int run(const Input &in)
{
    constexpr int Q = N + 1;
    using C = Config<SH, N, Q, T, OP, EPB_, NT_, PAIR>;
    using A = typename C::A;
    constexpr int D = C::D, NQ = C::NQ, M = C::M, EPB = C::EPB, NT = C::NT, S = C::S;
    constexpr TabLayout L = layout(SH, N, Q);
    constexpr int NG = (OP == OP_PHYSDERIV || OP == OP_IPROD_DERIV) ? nlam(SH) : ngeo(SH);
    constexpr bool PACK = sizeof(T) < 8 && NG == ngeo(SH);
    constexpr bool FUSED = C::FUSED && !MESH;
    if (in.E == 0) {  // query: group size, threads per CTA, unit stride, units per group
        std::printf("%d %d %d %d\n", EPB, NT, S, C::EPU);
        return 0;
    }
    const long long E = in.E;
    const long long epad = (E + 63) / 64 * 64;  // the library pads element arrays to 64
    // tables
    std::vector<double> t64(L.total);
    if (!nirb_build_tables(SH, N - 1, Q, t64.data(), in.nodal)) return 3;
    auto *tp = static_cast<TabP<A, C::TABN> *>(xalloc(sizeof(TabP<A, C::TABN>)));
    for (int i = 0; i < C::TABN; ++i) tp->v[i] = (A)t64[i];
    // metric in the device layout
    const size_t ngeo_vals = (size_t)(in.pp ? epad * NQ : epad) * NG;
    T *geo = static_cast<T *>(xalloc(ngeo_vals * sizeof(T)));
    {
        const size_t per = (size_t)(in.pp ? NQ : 1) * NG;
        std::vector<double> g((size_t)E * per);
        for (auto &v : g)
            if (std::scanf("%lf", &v) != 1) return 2;
        for (long long e = 0; e < epad; ++e) {
            const long long es = e < E ? e : 0;  // padding elements: finite copies of element 0
            for (int n = 0; n < (in.pp ? NQ : 1); ++n)
                for (int c = 0; c < NG; ++c) {
                    const double v = g[(size_t)es * per + (size_t)n * NG + c];
                    long long idx;
                    if (!in.pp) idx = e * NG + c;
                    else if (PACK) idx = geo_packed_index(e, n, c, NQ, NG);
                    else idx = ((((e >> 5) * NQ + n) * NG + c) << 5) + (e & 31);
                    geo[idx] = to_t<T>(v);
                }
        }
    }
    // inputs and outputs, exactly sized
    const bool modal_in = OP == OP_BWD || OP == OP_MASS || OP == OP_HELM;
    const bool modal_out = OP != OP_BWD && OP != OP_PHYSDERIV;
    const int nin = OP == OP_IPROD_DERIV ? D : OP == OP_HELM ? in.nfields : 1;
    const int nout = OP == OP_PHYSDERIV ? D : OP == OP_HELM ? in.nfields : 1;
    const int lin = modal_in ? M : NQ, lout = modal_out ? M : NQ;
    T *ins[3] = {nullptr, nullptr, nullptr}, *outs[3] = {nullptr, nullptr, nullptr};
    const char *shrt = std::getenv("SIM_SHORT");
    const bool short_in = shrt && !std::strcmp(shrt, "input"), short_smem = shrt && !std::strcmp(shrt, "smem");
    for (int f = 0; f < nin; ++f) {
        const long long len = E * lin - (f == 0 && short_in ? 1 : 0);
        ins[f] = static_cast<T *>(xalloc((size_t)len * sizeof(T)));
        for (long long i = 0; i < E * lin; ++i) {
            double v;
            if (std::scanf("%lf", &v) != 1) return 2;
            if (i < len) ins[f][i] = to_t<T>(v);
        }
    }
    for (int f = 0; f < nout; ++f) outs[f] = static_cast<T *>(xalloc((size_t)E * lout * sizeof(T)));
    int err = 0;
    KArgs a{};
    a.in0 = ins[0];
    a.in1 = ins[1];
    a.in2 = ins[2];
    a.out0 = outs[0];
    a.out1 = outs[1];
    a.out2 = outs[2];
    a.geo = geo;
    a.tab = tp->v;
    a.nelem = E;
    a.lambda = in.lambda;
    a.geo_pp = in.pp;
    a.pf = 0;
    a.err = &err;
    a.nfields = OP == OP_HELM ? in.nfields : 1;
    a.nodal = in.nodal;
    // shared memory: tables | staging buffer (staged FP32/BF16 Helmholtz) | group buffers
    constexpr int STG = (FUSED && STAGE) ? ((EPB * M * (int)sizeof(T) + 15) / 16) * 16 : 0;
    const size_t smem_bytes = (size_t)C::TABB + STG + C::BUFB - (short_smem ? S * sizeof(A) : 0);
    unsigned char *smem = static_cast<unsigned char *>(xalloc(smem_bytes));
    A *tab = reinterpret_cast<A *>(smem);
    T *stage = reinterpret_cast<T *>(smem + C::TABB);
    A *buf = reinterpret_cast<A *>(smem + C::TABB + STG);
    const long long ngroups = (E + EPB - 1) / EPB;
    const int nf = OP == OP_HELM ? in.nfields : 1;
    blockIdx = HostDim{0, 0, 0};
    gridDim = HostDim{1, 1, 1};
    int s_next = 0;  // the kernel's shared flag: the staging buffer holds the next item
    auto body = [&](int t) {
        for (int i = t; i < C::TABN; i += NT) tab[i] = tp->v[i];
        __syncthreads();
        if constexpr (FUSED) {
            const PTab<A, C::TABN> ptab{tp, 0};
            auto issue = [&](long long g, int f) -> int {  // the bulk copy, done at issue time
                if (!STAGE || g >= ngroups) return 0;
                const long long e0 = g * EPB;
                if (e0 + EPB > E) return 0;
                std::memcpy(stage, static_cast<const T *>(field_in(a, f)) + e0 * M, (size_t)EPB * M * sizeof(T));
                return 1;
            };
            if (t == 0) s_next = issue(0, 0);
            __syncthreads();
            for (long long g = 0; g < ngroups; ++g) {
                const long long e0 = g * EPB;
                const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
                for (int f = 0; f < nf; ++f) {
                    const bool staged = s_next != 0;
                    if (staged) {
                        __syncthreads();  // the completed copy (the kernel's mbarrier wait)
                        if constexpr (PAIR) {
                            F2 *B1 = reinterpret_cast<F2 *>(buf) + C::EPU * S;
                            for (int i = t; i < C::EPU * M; i += NT) {
                                const int u = i / M, m = i - u * M;
                                B1[u * S + m] = F2(to_a(stage[2 * u * M + m], A()), to_a(stage[(2 * u + 1) * M + m], A()));
                            }
                        } else {
                            A *B1 = buf + EPB * S;
                            for (int i = t; i < EPB * M; i += NT) {
                                const int e = i / M, m = i - e * M;
                                B1[e * S + m] = to_a(stage[i], A());
                            }
                        }
                    }
                    __syncthreads();
                    if (t == 0) s_next = f + 1 < nf ? issue(g, f + 1) : issue(g + 1, 0);
                    run_group<SH, N, Q, T, OP, EPB_, NT_, PAIR>(a, field_in(a, f), field_out(a, f), ptab, tab, buf,
                                                                e0, ne, staged);
                }
            }
        } else {
            for (long long g = 0; g < ngroups; ++g) {
                const long long e0 = g * EPB;
                const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
                for (int f = 0; f < nf; ++f) {
                    if constexpr (sizeof(A) == 4 && !MESH) {
                        const PTab<A, C::TABN> ptab{tp, 0};
                        run_group<SH, N, Q, T, OP, EPB_, NT_>(a, field_in(a, f), field_out(a, f), ptab, tab, buf,
                                                              e0, ne);
                    } else {
                        run_group<SH, N, Q, T, OP, EPB_, NT_>(a, field_in(a, f), field_out(a, f), STab<A>{tab},
                                                              tab, buf, e0, ne);
                    }
                }
            }
        }
    };
    int rc = run_cta(NT, body);
    if (rc) return rc;
    if (err) return 6;
    for (int f = 0; f < nout; ++f)
        for (long long i = 0; i < E * lout; ++i) std::printf("%.17g\n", from_t<T>(outs[f][i]));
    std::fprintf(stderr, "EPB %d NT %d smem %zu\n", EPB, NT, smem_bytes);
    for (int f = 0; f < 3; ++f) {
        std::free(ins[f]);
        std::free(outs[f]);
    }
    std::free(geo);
    std::free(tp);
    std::free(smem);
    return 0;
}

// The Helmholtz variants as the library builds them: default group, half,
// double (staged only while tables, staging buffer and buffers fit in 227 KB),
// and the persistent mesh kernel's form.
template <int SH, int N, class T, int OP>
int by_variant(int variant, const Input &in)
{
    using C0 = Config<SH, N, N + 1, T, OP, 0>;
    constexpr int e0 = C0::EPB;
    constexpr int eh = e0 > 1 ? e0 / 2 : 1;
    constexpr int stg2 = C0::FUSED ? ((2 * e0 * C0::M * (int)sizeof(T) + 15) / 16) * 16 : 0;
    constexpr bool fits = C0::TABB + 2 * C0::BUFB + stg2 <= 227 * 1024 && e0 < 64;
    constexpr bool fits_unstaged = C0::FUSED && !fits && C0::TABB + 2 * C0::BUFB <= 227 * 1024 && e0 < 64;
    constexpr int ed = (fits || fits_unstaged) ? 2 * e0 : e0;
    constexpr int mesh_nt = sizeof(typename CT<T>::type) == 8 ? 256 : 512;
    if (variant == 0) return run<SH, N, T, OP, 0, 0, true, false>(in);
    if constexpr (OP == OP_HELM) {
        if (variant == 1) return run<SH, N, T, OP, eh, 0, true, false>(in);
        if (variant == 2) return run<SH, N, T, OP, ed, 0, !fits_unstaged, false>(in);
        if (variant == 3) return run<SH, N, T, OP, 0, mesh_nt, true, true>(in);
        if constexpr (C0::FUSED && (SH == QUAD || SH == HEX))
            if (variant == 5) return run<SH, N, T, OP, 0, 0, true, false, true>(in);
    }
    return 4;
}

template <int SH, class T, int OP>
int by_n(int P, int variant, const Input &in)
{
    switch (P + 1) {
    case 2: return by_variant<SH, 2, T, OP>(variant, in);
    case 3: return by_variant<SH, 3, T, OP>(variant, in);
    case 4: return by_variant<SH, 4, T, OP>(variant, in);
    case 5: return by_variant<SH, 5, T, OP>(variant, in);
#ifdef SIM_HIGH_P
    // high orders for the Helmholtz only (groups of 4 to 16 elements: the strides
    // chosen for small groups)
    case 7:
        if constexpr (OP == OP_HELM) return by_variant<SH, 7, T, OP>(variant, in);
        else return 4;
    case 10:
        if constexpr (OP == OP_HELM) return by_variant<SH, 10, T, OP>(variant, in);
        else return 4;
#endif
    default: return 4;
    }
}

template <int SH, class T>
int by_op(int op, int P, int variant, const Input &in)
{
    switch (op) {
    case OP_BWD: return by_n<SH, T, OP_BWD>(P, variant, in);
    case OP_IPROD: return by_n<SH, T, OP_IPROD>(P, variant, in);
    case OP_PHYSDERIV: return by_n<SH, T, OP_PHYSDERIV>(P, variant, in);
    case OP_IPROD_DERIV: return by_n<SH, T, OP_IPROD_DERIV>(P, variant, in);
    case OP_MASS: return by_n<SH, T, OP_MASS>(P, variant, in);
    case OP_HELM: return by_n<SH, T, OP_HELM>(P, variant, in);
    default: return 4;
    }
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc != 6) return 1;
    const int shape = std::atoi(argv[1]), P = std::atoi(argv[2]), op = std::atoi(argv[3]),
              prec = std::atoi(argv[4]), variant = std::atoi(argv[5]);
    if (shape != SIM_SHAPE) return 1;
    if (const char *d = std::getenv("SIM_DROP_BARRIER")) g_drop = std::atoi(d);
    if (const char *o = std::getenv("SIM_ORDER")) {  // fwd (default), rev, or a shuffle seed
        if (!std::strcmp(o, "rev")) g_sched.mode = 1;
        else if (std::strcmp(o, "fwd")) {
            g_sched.mode = 2;
            g_sched.seed = std::strtoull(o, nullptr, 10);
        }
    }
    Input in{};
    if (std::scanf("%lld %d %lf %d %d", &in.E, &in.pp, &in.lambda, &in.nodal, &in.nfields) != 5) return 2;
    if (in.E < 0 || in.nfields < 1 || in.nfields > 3) return 1;
    switch (prec) {
    case 0: return by_op<SIM_SHAPE, double>(op, P, variant, in);
    case 1: return by_op<SIM_SHAPE, float>(op, P, variant, in);
    case 2: return by_op<SIM_SHAPE, __nv_bfloat16>(op, P, variant, in);
    default: return 1;
    }
}
