// Host emulation of one CTA of the persistent hybrid-mesh Helmholtz kernel
// (nir_mesh_inst.cu), for the CPU test tests/test_mesh_sim_cpu.py.  Not part
// of the library.
//
// The instantiation unit is compiled as plain C++ (one dimension and precision
// per build, -DNIR_MESH_DIM / -DNIR_PREC) and its per-item code -- dispatch to
// the (shape, P) variant, the table reload when the CTA moves to another block,
// the constant-bank tables of the low-order FP32/BF16 variants, run_group -- is
// run by NT host threads over a work list that alternates between the blocks.
// The item loop is the kernel's (thread 0 takes the next item, two barriers),
// restated here because the kernel's own shared variables are per-CTA.  As in
// cta_sim.cpp, threads run one at a time between barriers in a fixed order per
// phase, shared memory is one exactly sized heap block (the largest variant's),
// every global array is exactly sized, the constant table is the unit's own
// array, and the build uses AddressSanitizer.
//
// stdin: nblocks lambda gran, then per block "shape P E", its metric
// ([E][Nq][NG]) and its coefficients ([E][M]); stdout: each block's result.
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
#include <map>
#include <mutex>
#include <string>
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
                const int t = perm[i];
                perm[i] = perm[j];
                perm[j] = t;
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
static inline int atomicAdd(int *p, int v)  // the kernel's work counter (the kernel itself is not run here)
{
    const int o = *p;
    *p += v;
    return o;
}

#include "nir_basis.h"
namespace nirk {
namespace {
unsigned char smem_raw[16];  // the kernel's dynamic shared memory (the kernel is not run here)
}
}  // namespace nirk
#include "nir_mesh_inst.cu"

#define NIR_KINFO_OF NIR_MCAT(NIR_MESH_DIM, NIR_PREC)

using namespace nirk;

namespace {

using TS = TT;                       // storage type of this build
using AC = typename CT<TS>::type;    // compute type

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

struct Blk {
    int shape, P;
    long long E;
    MeshKInfo k;
    std::vector<AC> tab;  // the block's table blob in the compute type (the reload source)
    TS *geo = nullptr, *in = nullptr, *out = nullptr;
};

int run()
{
    int nb = 0, gran = 1;
    double lam = 0;
    if (std::scanf("%d %lf %d", &nb, &lam, &gran) != 3 || nb < 1 || gran < 1) return 2;
    std::vector<Blk> blocks(nb);
    int smem = 0;
    for (auto &b : blocks) {
        if (std::scanf("%d %d %lld", &b.shape, &b.P, &b.E) != 3 || b.E < 1) return 2;
        b.k = NIR_KINFO_OF(b.shape, b.P);
        if (!b.k.fn) return 4;
        smem = smem > b.k.smem ? smem : b.k.smem;
        const int N = b.P + 1, Q = N + 1;
        const int total = nirb_table_size(b.shape, b.P, Q);
        std::vector<double> t64(total);
        if (!nirb_build_tables(b.shape, b.P, Q, t64.data(), 0)) return 3;
        b.tab.assign(t64.begin(), t64.end());
#if NIR_PREC != 0
        {  // the variant's constant tables, laid out as the library uploads them
            int base = -1, wq = 0, gap = 0, tot = 0;
            bool used = false;
            ctab_range<0>(b.k.vid, base, wq, gap, tot, used);
            if (base < 0 || tot != total) return 3;
            if (used) {
                for (int i = 0; i < wq; ++i) c_tab[base + i] = b.tab[i];
                for (int i = wq + gap; i < total; ++i) c_tab[base + i - gap] = b.tab[i];
            }
        }
#endif
        // metric in the device layout (packed per point for FP32/BF16)
        const int NQ = npts(b.shape, Q), NG = ngeo(b.shape);
        const long long epad = (b.E + 63) / 64 * 64;
        std::vector<double> g((size_t)b.E * NQ * NG);
        for (auto &v : g)
            if (std::scanf("%lf", &v) != 1) return 2;
        b.geo = static_cast<TS *>(xalloc((size_t)epad * NQ * NG * sizeof(TS)));
        for (long long e = 0; e < epad; ++e) {
            const long long es = e < b.E ? e : 0;
            for (int n = 0; n < NQ; ++n)
                for (int c = 0; c < NG; ++c) {
                    const long long idx = sizeof(TS) < 8 ? geo_packed_index(e, n, c, NQ, NG)
                                                         : ((((e >> 5) * NQ + n) * NG + c) << 5) + (e & 31);
                    b.geo[idx] = to_t<TS>(g[((size_t)es * NQ + n) * NG + c]);
                }
        }
        const int M = nmodes(b.shape, N);
        b.in = static_cast<TS *>(xalloc((size_t)b.E * M * sizeof(TS)));
        b.out = static_cast<TS *>(xalloc((size_t)b.E * M * sizeof(TS)));
        for (long long i = 0; i < b.E * M; ++i) {
            double v;
            if (std::scanf("%lf", &v) != 1) return 2;
            b.in[i] = to_t<TS>(v);
        }
    }
    int err = 0;
    std::vector<MeshBlk> mb(nb);
    std::vector<std::vector<MeshItem>> per(nb);
    for (int i = 0; i < nb; ++i) {
        KArgs &a = mb[i].a;
        std::memset(&a, 0, sizeof(a));
        a.nfields = 1;
        a.in0 = blocks[i].in;
        a.out0 = blocks[i].out;
        a.geo = blocks[i].geo;
        a.tab = blocks[i].tab.data();
        a.nelem = blocks[i].E;
        a.lambda = lam;
        a.geo_pp = 1;
        a.err = &err;
        mb[i].vid = blocks[i].k.vid;
        const long long ng = (blocks[i].E + blocks[i].k.epb - 1) / blocks[i].k.epb;
        for (long long g0 = 0; g0 < ng; g0 += gran)
            per[i].push_back(MeshItem{i, (int)g0, (int)(ng - g0 < gran ? ng - g0 : gran), 0});
    }
    // the blocks' items in turn, so the CTA keeps moving between blocks (table reloads)
    std::vector<MeshItem> items;
    for (size_t r = 0;; ++r) {
        bool any = false;
        for (int i = 0; i < nb; ++i)
            if (r < per[i].size()) {
                items.push_back(per[i][r]);
                any = true;
            }
        if (!any) break;
    }
    unsigned char *sm = static_cast<unsigned char *>(xalloc((size_t)smem));
    const int NT = kMeshNT, nitems = (int)items.size();
    int counter = 0, s_item = 0;
    blockIdx = HostDim{0, 0, 0};
    gridDim = HostDim{1, 1, 1};
    std::function<void(int)> body = [&](int t) {
        int cur = -1;
        for (;;) {  // the kernel's item loop
            if (t == 0) s_item = atomicAdd(&counter, 1);
            __syncthreads();
            const int it = s_item;
            __syncthreads();
            if (it >= nitems) break;
            const MeshItem m = items[it];
            const MeshBlk b = mb[m.block];
            dispatch_one<0>(b.vid, b, m, sm, cur);
        }
    };
    g_sched.nt = NT;
    g_sched.sem = std::vector<sem_t>(NT);
    for (auto &x : g_sched.sem) sem_init(&x, 0, 0);
    g_sched.order(0);
    struct Arg {
        std::function<void(int)> *f;
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
                g_sched.pass();
                return nullptr;
            }, &args[t]))
            return 5;
    }
    sem_post(&g_sched.sem[g_sched.perm[0]]);
    for (int t = 0; t < NT; ++t) pthread_join(th[t], nullptr);
    if (err) return 6;
    for (auto &b : blocks) {
        const long long n = b.E * nmodes(b.shape, b.P + 1);
        for (long long i = 0; i < n; ++i) std::printf("%.17g\n", from_t<TS>(b.out[i]));
        std::free(b.geo);
        std::free(b.in);
        std::free(b.out);
    }
    std::free(sm);
    return 0;
}

}  // namespace

int main()
{
    if (const char *o = std::getenv("SIM_ORDER")) {
        if (!std::strcmp(o, "rev")) g_sched.mode = 1;
        else if (std::strcmp(o, "fwd")) {
            g_sched.mode = 2;
            g_sched.seed = std::strtoull(o, nullptr, 10);
        }
    }
    return run();
}
