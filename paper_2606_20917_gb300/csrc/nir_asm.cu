// nir_asm.cu -- conforming C0 assembly of quadrilateral and hexahedral blocks.
//
// The paper applies its operators element by element (Sec. 2.1: the weak
// Helmholtz matrix is built from elemental B, W, Lambda) and leaves the global
// system out; this unit joins the elemental expansions into a continuous one,
// the standard spectral/hp construction of a C0 basis (modified or
// GLL-Lagrange).
//
// Global numbering from vertex connectivity.  Every mode belongs to one mesh
// entity: each direction of the tensor index (p, q, r) plays the role "vertex
// at -1", "vertex at +1" or "bubble".  Modified basis: index 0, 1, and >= 2
// (bubble p - 2); GLL-Lagrange basis: node 0, node N - 1, and the interior
// nodes 1..N-2 (bubble p - 1).  No bubble: a vertex mode; one: an edge mode;
// two (3-D): a face mode; all: an interior mode.  Shared entities are keyed by
// the sorted global ids of their vertices and seen from a canonical frame:
//   - an edge runs from its smaller to its larger vertex id; a local edge
//     running the other way reflects its bubbles: sign (-1)^p for the
//     modified basis (psi_p(-z) = (-1)^p psi_p(z)), node order reversed for
//     the Lagrange basis (l_{N-1-j}(-z) = l_j(z) on the symmetric GLL nodes);
//   - a face's origin is its smallest-id corner, its first axis points to the
//     origin's neighbour with the smaller id.  A local face whose axes are
//     swapped relative to that frame exchanges the two mode indices, and each
//     local axis running against the frame reflects that direction as above.
// Faces (2-D: edges) owned by one element are the boundary.  Free dofs are
// numbered first (element order, entity order vertices, edges, faces, then
// interior), boundary dofs after them, so vectors of the outer solve hold the
// unknowns first and the Dirichlet values last.
//
// Device data: map[i] = +-(g + 1) for local dof i (concatenated blocks,
// element-major [E][M]); rowptr/pos, the transposed map sorted by local index,
// give every global dof its local copies in a fixed order, so the assembly
// y_g = sum_k s_k y_loc[i_k] is a gather (no atomics) and deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "nir_cg.h"
#include "nir_internal.h"
#include "nir_kernels.cuh"
#include "nir_vec.cuh"

namespace {

using nirv::st_v;
using nirv::to_d;

constexpr int kVT = 256;

int vgrid(long long n) { return (int)std::min<long long>((n + kVT - 1) / kVT, 152LL * 16); }

// Gather and assembly are bound by memory latency (an index load, then the
// indexed load): every grid-stride step handles kU entries i0 + k * stride
// with all their loads issued before the arithmetic.
constexpr int kU = 4;

// x_loc[i] = s_i x_g[g_i]; entries g >= n_avail read as zero (held boundary values).
template <class TI>
__global__ void __launch_bounds__(kVT) k_gather(const TI *__restrict__ xg, long long n_avail,
                                                const int *__restrict__ map, long long nloc, TI *__restrict__ xl)
{
    const long long S = (long long)gridDim.x * kVT;
    for (long long i0 = blockIdx.x * (long long)kVT + threadIdx.x; i0 < nloc; i0 += S * kU) {
        int sv[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S;
            sv[k] = map[i < nloc ? i : i0];
        }
        TI v[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long g = (long long)(sv[k] > 0 ? sv[k] : -sv[k]) - 1;
            v[k] = g < n_avail ? xg[g] : TI(0.0f);
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long i = i0 + k * S;
            if (i < nloc) xl[i] = sv[k] > 0 ? v[k] : -v[k];  // a signed copy: exact in every type
        }
    }
}

// Sums run in FP64 for FP64 data and in FP32 for FP32 / bfloat16 data (FP64
// arithmetic and conversions are slow on GB300 and would bound the kernel).
__device__ __forceinline__ double acc_of(double v) { return v; }
__device__ __forceinline__ float acc_of(float v) { return v; }
__device__ __forceinline__ float acc_of(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ void st_acc(double *p, double v) { *p = v; }
__device__ __forceinline__ void st_acc(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_acc(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// y_g[g] = sum over the copies k of g: s_k y_loc[i_k]   (g < nrows), the copies
// summed in their stored order; with absval the signs are dropped (diagonal
// assembly: s_k^2 = 1).
template <class TI, class TO, class Acc = typename std::conditional<sizeof(TI) == 8, double, float>::type>
__global__ void __launch_bounds__(kVT) k_assemble(const TI *__restrict__ yl, const int *__restrict__ rowptr,
                                                  const int *__restrict__ pos, long long nrows, TO *__restrict__ yg,
                                                  int absval)
{
    const long long S = (long long)gridDim.x * kVT;
    for (long long g0 = blockIdx.x * (long long)kVT + threadIdx.x; g0 < nrows; g0 += S * kU) {
        int beg[kU], end[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long g = g0 + k * S;
            beg[k] = g < nrows ? rowptr[g] : 0;
            end[k] = g < nrows ? rowptr[g + 1] : 0;
        }
        Acc acc[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) acc[k] = Acc(0);
        for (int c = 0;; ++c) {
            int sv[kU];
            bool any = false;
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                const int q = beg[k] + c;
                sv[k] = q < end[k] ? pos[q] : 0;
                any |= q < end[k];
            }
            if (!any) break;
            Acc v[kU];
#pragma unroll
            for (int k = 0; k < kU; ++k) v[k] = sv[k] ? acc_of(yl[(sv[k] > 0 ? sv[k] : -sv[k]) - 1]) : Acc(0);
#pragma unroll
            for (int k = 0; k < kU; ++k) acc[k] += (sv[k] > 0 || absval) ? v[k] : -v[k];
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const long long g = g0 + k * S;
            if (g < nrows) st_acc(yg + g, acc[k]);
        }
    }
}

// x_g[g] = s_k x_loc[i_k] of the first copy (the inverse of the gather on a
// continuous local vector).
__global__ void __launch_bounds__(kVT) k_pick(const double *__restrict__ xl, const int *__restrict__ rowptr,
                                              const int *__restrict__ pos, long long n, double *__restrict__ xg)
{
    for (long long g = blockIdx.x * (long long)kVT + threadIdx.x; g < n; g += (long long)gridDim.x * kVT) {
        const int s = pos[rowptr[g]];
        const double v = xl[(s > 0 ? s : -s) - 1];
        xg[g] = s > 0 ? v : -v;
    }
}

// Probing of the elemental diagonal: x = 1 at local mode m of every element.
__global__ void __launch_bounds__(kVT) k_unit_mode(float *x, int M, int m, long long nloc)
{
    for (long long i = blockIdx.x * (long long)kVT + threadIdx.x; i < nloc; i += (long long)gridDim.x * kVT)
        x[i] = (i % M == m) ? 1.0f : 0.0f;
}

__global__ void __launch_bounds__(kVT) k_take_mode(double *d, const float *y, int M, int m, long long nloc)
{
    for (long long i = blockIdx.x * (long long)kVT + threadIdx.x; i < nloc; i += (long long)gridDim.x * kVT)
        if (i % M == m) d[i] = (double)y[i];
}

// ---------------------------------------------------------------------------
// Host numbering.

struct EKey {
    std::array<long long, 4> g;
    int n;
    bool operator==(const EKey &o) const { return n == o.n && g == o.g; }
};

struct EKeyHash {
    size_t operator()(const EKey &k) const
    {
        unsigned long long h = 1469598103934665603ull ^ (unsigned long long)k.n;
        for (int i = 0; i < k.n; ++i) {
            h ^= (unsigned long long)k.g[i] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
            h *= 1099511628211ull;
        }
        return (size_t)h;
    }
};

struct Entity {
    int ndof = 0;
    int count = 0;          // elements holding it (faces in 3-D, edges in 2-D decide the boundary)
    bool boundary = false;
    long long first = -1;   // first global dof
};

EKey make_key(std::initializer_list<long long> ids)
{
    EKey k;
    k.g = {0, 0, 0, 0};
    k.n = 0;
    for (long long v : ids) k.g[k.n++] = v;
    std::sort(k.g.begin(), k.g.begin() + k.n);
    return k;
}

// Local vertex number of the corner with direction bits b[0..d-1].
inline int vnum(const int *b, int d)
{
    int v = 0;
    for (int k = 0; k < d; ++k) v |= b[k] << k;
    return v;
}

}  // namespace

struct AsmOp;

struct nir_asm {
    nir_ctx *ctx = nullptr;
    int dim = 0, shape = 0, P = 0, M = 0;
    std::vector<nir_block *> blocks;
    std::vector<long long> off;          // first local dof of each block
    long long nloc = 0, nglob = 0, nfree = 0;
    std::vector<int> map_h;              // host copy of the map
    int *map = nullptr, *rowptr = nullptr, *pos = nullptr;
    void *xl[3] = {nullptr, nullptr, nullptr}, *yl[3] = {nullptr, nullptr, nullptr};  // local scratch
    double *dloc = nullptr;              // probed elemental diagonal (local)
    cudaStream_t cap_stream = nullptr;
    AsmOp *ops[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [operator][fix_boundary]
    CGWork *cg[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    std::vector<unsigned long long> state_seen;                    // block state at graph capture
};

namespace {

bool valid_prec(int p) { return p == NIR_F64 || p == NIR_F32 || p == NIR_BF16; }

int ensure_local(nir_asm *a, int prec)
{
    if (a->xl[prec]) return NIR_OK;
    const size_t bytes = (size_t)a->nloc * nir_prec_size(prec);
    if (cudaMalloc(&a->xl[prec], bytes) != cudaSuccess) return NIR_ERR_NO_MEMORY;
    if (cudaMalloc(&a->yl[prec], bytes) != cudaSuccess) {
        cudaFree(a->xl[prec]);
        a->xl[prec] = nullptr;
        return NIR_ERR_NO_MEMORY;
    }
    return NIR_OK;
}

// Launch one elemental operator over every block: local x -> local y.
int launch_blocks(nir_asm *a, int op, int prec, double lambda, const void *x, void *y, cudaStream_t st)
{
    const size_t es = nir_prec_size(prec);
    const int kop = op == NIR_ASM_MASS ? nirk::OP_MASS : nirk::OP_HELM;
    for (size_t b = 0; b < a->blocks.size(); ++b) {
        const char *xb = static_cast<const char *>(x) + (size_t)a->off[b] * es;
        char *yb = static_cast<char *>(y) + (size_t)a->off[b] * es;
        int rc = nir_launch_op(a->blocks[b], prec, kop, lambda, xb, nullptr, nullptr, yb, nullptr, nullptr, st, 0);
        if (rc) return rc;
    }
    return NIR_OK;
}

template <class T>
int launch_apply_t(nir_asm *a, int op, int prec, double lambda, const T *x, long long n_avail, T *y,
                   long long nrows, cudaStream_t st)
{
    T *xl = static_cast<T *>(a->xl[prec]), *yl = static_cast<T *>(a->yl[prec]);
    k_gather<T><<<vgrid(a->nloc), kVT, 0, st>>>(x, n_avail, a->map, a->nloc, xl);
    int rc = launch_blocks(a, op, prec, lambda, xl, yl, st);
    if (rc) return rc;
    k_assemble<T, T><<<vgrid(nrows), kVT, 0, st>>>(yl, a->rowptr, a->pos, nrows, y, 0);
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return NIR_ERR_CUDA;
    }
    return nir_debug_after(a->ctx, NIR_OK);
}

// y[0:nrows] = (A^T H A x)[0:nrows] with x[g] = 0 for g >= n_avail.
int launch_apply(nir_asm *a, int op, int prec, double lambda, const void *x, long long n_avail, void *y,
                 long long nrows, cudaStream_t st)
{
    int rc = ensure_local(a, prec);
    if (rc) return rc;
    for (nir_block *b : a->blocks) {
        rc = nir_block_ensure_prec(b, prec);
        if (rc) return rc;
    }
    if (prec == NIR_F64)
        return launch_apply_t<double>(a, op, prec, lambda, static_cast<const double *>(x), n_avail,
                                      static_cast<double *>(y), nrows, st);
    if (prec == NIR_F32)
        return launch_apply_t<float>(a, op, prec, lambda, static_cast<const float *>(x), n_avail,
                                     static_cast<float *>(y), nrows, st);
    return launch_apply_t<__nv_bfloat16>(a, op, prec, lambda, static_cast<const __nv_bfloat16 *>(x), n_avail,
                                         static_cast<__nv_bfloat16 *>(y), nrows, st);
}

// Everything a captured launch depends on besides its pointers.
unsigned long long block_state(const nir_block *b)
{
    unsigned long long h = b->geo_version;
    for (int p = 0; p < 3; ++p) h = h * 1000003ull + (unsigned)(b->helm_variant[p] * 7 + b->helm_pf[p]) +
                                   (unsigned long long)b->helm_grid[p] * 131ull;
    return h;
}

}  // namespace

struct AsmLaunch {
    int prec;
    double lambda;
    const void *x;
    void *y;
};

// A^T H A (or A^T M A) restricted to the unknowns, as seen by the CG solver.
struct AsmOp final : CgOperator {
    nir_asm *a;
    int op;
    bool fix;   // boundary dofs held (Dirichlet) or unknown
    AsmOp(nir_asm *aa, int o, bool f) : a(aa), op(o), fix(f) {}
    nir_ctx *context() override { return a->ctx; }
    long long n() override { return fix ? a->nfree : a->nglob; }
    long long n_full() override { return a->nglob; }
    cudaStream_t capture_stream() override { return a->cap_stream; }
    int prepare(int prec, double lambda, const void *x, void *y, void **handle) override
    {
        // one uncaptured launch sets up everything lazily created (local
        // buffers, low-precision factors, kernel attributes)
        int rc = launch_apply(a, op, prec, lambda, x, n(), y, n(), a->ctx->stream);
        if (rc) return rc;
        AsmLaunch *h = new (std::nothrow) AsmLaunch{prec, lambda, x, y};
        if (!h) return NIR_ERR_NO_MEMORY;
        *handle = h;
        return NIR_OK;
    }
    int launch(void *handle, cudaStream_t st) override
    {
        AsmLaunch *h = static_cast<AsmLaunch *>(handle);
        return launch_apply(a, op, h->prec, h->lambda, h->x, n(), h->y, n(), st);
    }
    void release(void *handle) override { delete static_cast<AsmLaunch *>(handle); }
    int apply64(double lambda, const double *x, double *y, cudaStream_t st) override
    {
        return launch_apply(a, op, NIR_F64, lambda, x, a->nglob, y, n(), st);
    }
    int diagonal(double lambda, double *d, cudaStream_t st) override
    {
        int rc = ensure_local(a, NIR_F32);
        if (rc) return rc;
        if (!a->dloc && cudaMalloc(&a->dloc, sizeof(double) * a->nloc) != cudaSuccess) return NIR_ERR_NO_MEMORY;
        for (nir_block *b : a->blocks) {
            rc = nir_block_ensure_prec(b, NIR_F32);
            if (rc) return rc;
        }
        float *x = static_cast<float *>(a->xl[NIR_F32]), *y = static_cast<float *>(a->yl[NIR_F32]);
        for (int m = 0; m < a->M && !rc; ++m) {
            k_unit_mode<<<vgrid(a->nloc), kVT, 0, st>>>(x, a->M, m, a->nloc);
            rc = launch_blocks(a, op, NIR_F32, lambda, x, y, st);
            if (!rc) k_take_mode<<<vgrid(a->nloc), kVT, 0, st>>>(a->dloc, y, a->M, m, a->nloc);
        }
        if (rc) return rc;
        k_assemble<double, double><<<vgrid(n()), kVT, 0, st>>>(a->dloc, a->rowptr, a->pos, n(), d, 1);
        NIR_CUDA_TRY(cudaStreamSynchronize(st));
        return NIR_OK;
    }
};

namespace {

void asm_free(nir_asm *a)
{
    for (int o = 0; o < 2; ++o)
        for (int f = 0; f < 2; ++f) {
            nir_cg_work_free(a->cg[o][f]);
            delete a->ops[o][f];
        }
    for (int p = 0; p < 3; ++p) {
        if (a->xl[p]) cudaFree(a->xl[p]);
        if (a->yl[p]) cudaFree(a->yl[p]);
    }
    if (a->map) cudaFree(a->map);
    if (a->rowptr) cudaFree(a->rowptr);
    if (a->pos) cudaFree(a->pos);
    if (a->dloc) cudaFree(a->dloc);
    if (a->cap_stream) cudaStreamDestroy(a->cap_stream);
    delete a;
}

// The global numbering (host only): map[i] = s (g + 1) for every local dof of
// the blocks' elements (nelem[b] elements of M modes each, in block order).
int c0_numbering(int d, int P, int basis, const std::vector<long long> &nelem, const int64_t *const *verts,
                 std::vector<int> &map, long long &nglob, long long &nfree)
{
    const int N = P + 1, nv = 1 << d;
    const bool nodal = basis == NIR_BASIS_GLL_LAGRANGE;
    const int M = d == 2 ? N * N : N * N * N;
    const int nb1 = P - 1;  // bubbles per direction
    std::unordered_map<EKey, int, EKeyHash> index;
    std::vector<Entity> ents;
    auto entity = [&](const EKey &k, int ndof) -> int {
        auto it = index.find(k);
        if (it != index.end()) return it->second;
        const int id = (int)ents.size();
        index.emplace(k, id);
        Entity e;
        e.ndof = ndof;
        ents.push_back(e);
        return id;
    };
    long long E = 0;
    for (long long ne : nelem) E += ne;
    const long long nloc = E * M;
    // per element: vertex, edge, face entities (local order), then an interior id
    const int nedge = d * (nv / 2), nface = d == 3 ? 6 : 0;
    const int per = nv + nedge + nface;
    std::vector<int> eent((size_t)E * per);
    std::vector<long long> vid((size_t)E * nv);
    long long e = 0;
    for (size_t bi = 0; bi < nelem.size(); ++bi) {
        for (long long le = 0; le < nelem[bi]; ++le, ++e) {
            const int64_t *vg = verts[bi] + (size_t)le * nv;
            for (int v = 0; v < nv; ++v) vid[(size_t)e * nv + v] = vg[v];
            int *ee = &eent[(size_t)e * per];
            for (int v = 0; v < nv; ++v) ee[v] = entity(make_key({vg[v]}), 1);
            // edges: direction dd, the other bits enumerate the edge
            int k = nv;
            for (int dd = 0; dd < d; ++dd)
                for (int o = 0; o < nv / 2; ++o) {
                    int bits[3] = {0, 0, 0}, t = o;
                    for (int q = 0; q < d; ++q)
                        if (q != dd) { bits[q] = t & 1; t >>= 1; }
                    bits[dd] = 0;
                    const int v0 = vnum(bits, d);
                    bits[dd] = 1;
                    const int v1 = vnum(bits, d);
                    ee[k++] = entity(make_key({vg[v0], vg[v1]}), nb1);
                }
            if (d == 3)
                for (int f = 0; f < 3; ++f)
                    for (int side = 0; side < 2; ++side) {
                        long long c[4];
                        int t = 0;
                        for (int o = 0; o < 4; ++o) {
                            int bits[3] = {0, 0, 0}, u = o;
                            for (int q = 0; q < 3; ++q)
                                if (q != f) { bits[q] = u & 1; u >>= 1; }
                            bits[f] = side;
                            c[t++] = vg[vnum(bits, 3)];
                        }
                        ee[k++] = entity(make_key({c[0], c[1], c[2], c[3]}), nb1 * nb1);
                    }
            // count the elements holding each boundary-deciding entity
            const int lo = d == 3 ? nv + nedge : nv, hi = d == 3 ? per : nv + nedge;
            for (int q = lo; q < hi; ++q) ents[ee[q]].count++;
        }
    }
    // boundary: faces (2-D edges) held once, with their vertices and edges
    e = 0;
    for (long long el = 0; el < E; ++el) {
        const int *ee = &eent[(size_t)el * per];
        if (d == 2) {
            for (int q = 0; q < nedge; ++q) {
                Entity &ed = ents[ee[nv + q]];
                if (ed.count > 2) return NIR_ERR_INVALID_ARG;  // non-manifold
                if (ed.count != 1) continue;
                ed.boundary = true;
                // vertices of edge q: direction q / 2, other bit q % 2
                const int dd = q / 2, ob = q % 2;
                for (int s = 0; s < 2; ++s) {
                    int bits[3] = {0, 0, 0};
                    bits[dd] = s;
                    bits[1 - dd] = ob;
                    ents[ee[vnum(bits, 2)]].boundary = true;
                }
            }
        } else {
            for (int q = 0; q < nface; ++q) {
                Entity &fc = ents[ee[nv + nedge + q]];
                if (fc.count > 2) return NIR_ERR_INVALID_ARG;
                if (fc.count != 1) continue;
                fc.boundary = true;
                const int f = q / 2, side = q % 2;
                for (int o = 0; o < 4; ++o) {  // corners
                    int bits[3] = {0, 0, 0}, u = o;
                    for (int r = 0; r < 3; ++r)
                        if (r != f) { bits[r] = u & 1; u >>= 1; }
                    bits[f] = side;
                    ents[ee[vnum(bits, 3)]].boundary = true;
                }
                // edges in the face: directions other than f, fixed bit of f = side
                for (int dd = 0; dd < 3; ++dd) {
                    if (dd == f) continue;
                    for (int o = 0; o < 4; ++o) {
                        int bits[3] = {0, 0, 0}, u = o;
                        for (int r = 0; r < 3; ++r)
                            if (r != dd) { bits[r] = u & 1; u >>= 1; }
                        if (bits[f] != side) continue;
                        ents[ee[nv + dd * 4 + o]].boundary = true;
                    }
                }
            }
        }
    }
    // numbering: free entities in element order, interiors included; then boundary
    const long long nint = (long long)std::pow(nb1, d);
    std::vector<long long> interior_first((size_t)E, -1);
    long long next = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (long long el = 0; el < E; ++el) {
            const int *ee = &eent[(size_t)el * per];
            for (int q = 0; q < per; ++q) {
                Entity &en = ents[ee[q]];
                if (en.first >= 0 || en.boundary != (pass == 1)) continue;
                en.first = next;
                next += en.ndof;
            }
            if (pass == 0) {
                interior_first[(size_t)el] = next;
                next += nint;
            }
        }
        if (pass == 0) nfree = next;
    }
    nglob = next;
    if (nglob >= (1LL << 31) - 2 || nloc >= (1LL << 31) - 2) return NIR_ERR_TOO_LARGE;
    // local map
    map.assign((size_t)nloc, 0);
    e = 0;
    long long li = 0;
    for (size_t bi = 0; bi < nelem.size(); ++bi) {
        for (long long le = 0; le < nelem[bi]; ++le, ++e) {
            const int *ee = &eent[(size_t)e * per];
            const long long *vg = &vid[(size_t)e * nv];
            for (int m = 0; m < M; ++m, ++li) {
                int idx[3] = {0, 0, 0};
                if (d == 2) { idx[0] = m / N; idx[1] = m % N; }
                else { idx[0] = m / (N * N); idx[1] = (m / N) % N; idx[2] = m % N; }
                // role per direction: vertex bit (vb) or bubble index (bb)
                int nbub = 0, bub[3], fixd[3], nf = 0, vb[3] = {0, 0, 0}, bb[3] = {0, 0, 0};
                for (int k = 0; k < d; ++k) {
                    const bool lo = idx[k] == 0, hi = nodal ? idx[k] == N - 1 : idx[k] == 1;
                    if (lo || hi) {
                        vb[k] = hi;
                        fixd[nf++] = k;
                    } else {
                        bb[k] = idx[k] - (nodal ? 1 : 2);
                        bub[nbub++] = k;
                    }
                }
                long long g = 0;
                int sgn = 1;
                // a bubble seen from the reflected direction
                auto reflect = [&](int b) {
                    if (nodal) return nb1 - 1 - b;
                    if (b & 1) sgn = -sgn;
                    return b;
                };
                if (nbub == 0) {
                    g = ents[ee[vnum(vb, d)]].first;
                } else if (nbub == 1) {
                    const int dd = bub[0];
                    int bits[3] = {vb[0], vb[1], vb[2]};
                    // edge number within direction dd: the other bits in increasing direction order
                    int o = 0, sh = 0;
                    for (int q = 0; q < d; ++q)
                        if (q != dd) { o |= bits[q] << sh; ++sh; }
                    bits[dd] = 0;
                    const long long a0 = vg[vnum(bits, d)];
                    bits[dd] = 1;
                    const long long a1 = vg[vnum(bits, d)];
                    const int b = a0 > a1 ? reflect(bb[dd]) : bb[dd];
                    g = ents[ee[nv + dd * (nv / 2) + o]].first + b;
                } else if (nbub == 2 && d == 3) {
                    const int f = fixd[0], side = vb[f];
                    const int u = bub[0], v = bub[1];
                    long long c[2][2];
                    for (int s = 0; s < 2; ++s)
                        for (int t = 0; t < 2; ++t) {
                            int bits[3] = {0, 0, 0};
                            bits[f] = side;
                            bits[u] = s;
                            bits[v] = t;
                            c[s][t] = vg[vnum(bits, 3)];
                        }
                    int s0 = 0, t0 = 0;
                    for (int s = 0; s < 2; ++s)
                        for (int t = 0; t < 2; ++t)
                            if (c[s][t] < c[s0][t0]) { s0 = s; t0 = t; }
                    const bool transposed = c[1 - s0][t0] > c[s0][1 - t0];
                    const int bu = s0 ? reflect(bb[u]) : bb[u];
                    const int bv = t0 ? reflect(bb[v]) : bb[v];
                    const int fa = transposed ? bv : bu, fb = transposed ? bu : bv;
                    g = ents[ee[nv + nedge + 2 * f + side]].first + (long long)fa * nb1 + fb;
                } else {
                    long long r = 0;
                    for (int k = 0; k < d; ++k) r = r * nb1 + bb[k];
                    g = interior_first[(size_t)e] + r;
                }
                map[(size_t)li] = sgn * (int)(g + 1);
            }
        }
    }
    return NIR_OK;
}

// Numbering, then the device map and its transpose.
int asm_number(nir_asm *a, const int64_t *const *verts)
{
    std::vector<long long> nelem;
    for (nir_block *b : a->blocks) nelem.push_back(b->d.nelem);
    int rc = c0_numbering(a->dim, a->P, a->blocks[0]->d.basis, nelem, verts, a->map_h, a->nglob, a->nfree);
    if (rc) return rc;
    // transpose: copies of every global dof in local order
    std::vector<int> rowptr((size_t)a->nglob + 1, 0), pos((size_t)a->nloc);
    for (long long i = 0; i < a->nloc; ++i) rowptr[(size_t)std::abs(a->map_h[(size_t)i])]++;
    for (long long g = 0; g < a->nglob; ++g) rowptr[(size_t)g + 1] += rowptr[(size_t)g];
    {
        std::vector<int> fill(rowptr.begin(), rowptr.end() - 1);
        for (long long i = 0; i < a->nloc; ++i) {
            const int s = a->map_h[(size_t)i];
            const long long g = std::abs(s) - 1;
            pos[(size_t)fill[(size_t)g]++] = (s > 0 ? 1 : -1) * (int)(i + 1);
        }
    }
    for (long long g = 0; g < a->nglob; ++g)
        if (rowptr[(size_t)g + 1] == rowptr[(size_t)g]) return NIR_ERR_INVALID_ARG;  // unreachable dof
    if (cudaMalloc(&a->map, sizeof(int) * a->nloc) != cudaSuccess ||
        cudaMalloc(&a->rowptr, sizeof(int) * (a->nglob + 1)) != cudaSuccess ||
        cudaMalloc(&a->pos, sizeof(int) * a->nloc) != cudaSuccess)
        return NIR_ERR_NO_MEMORY;
    NIR_CUDA_TRY(cudaMemcpy(a->map, a->map_h.data(), sizeof(int) * a->nloc, cudaMemcpyHostToDevice));
    NIR_CUDA_TRY(cudaMemcpy(a->rowptr, rowptr.data(), sizeof(int) * (a->nglob + 1), cudaMemcpyHostToDevice));
    NIR_CUDA_TRY(cudaMemcpy(a->pos, pos.data(), sizeof(int) * a->nloc, cudaMemcpyHostToDevice));
    return NIR_OK;
}

}  // namespace

extern "C" int nir_asm_create(nir_ctx *ctx, nir_block *const *blocks, const int64_t *const *vertex_ids, int nblocks,
                              nir_asm **out)
{
    if (!ctx || !blocks || !vertex_ids || nblocks < 1 || !out) return NIR_ERR_INVALID_ARG;
    *out = nullptr;
    const int shape = blocks[0] ? blocks[0]->d.shape : -1;
    if (shape != NIR_QUAD && shape != NIR_HEX) return NIR_ERR_UNSUPPORTED;
    for (int i = 0; i < nblocks; ++i) {
        if (!blocks[i] || !vertex_ids[i] || blocks[i]->ctx != ctx) return NIR_ERR_INVALID_ARG;
        if (blocks[i]->d.shape != shape || blocks[i]->d.P != blocks[0]->d.P) return NIR_ERR_UNSUPPORTED;
        if (blocks[i]->d.basis != blocks[0]->d.basis) return NIR_ERR_UNSUPPORTED;
    }
    if (blocks[0]->d.P < 1) return NIR_ERR_UNSUPPORTED;
    NIR_CUDA_TRY(cudaSetDevice(ctx->device));
    nir_asm *a = new (std::nothrow) nir_asm();
    if (!a) return NIR_ERR_NO_MEMORY;
    a->ctx = ctx;
    a->shape = shape;
    a->dim = shape == NIR_HEX ? 3 : 2;
    a->P = blocks[0]->d.P;
    a->M = blocks[0]->M;
    for (int i = 0; i < nblocks; ++i) {
        a->blocks.push_back(blocks[i]);
        a->off.push_back(a->nloc);
        a->nloc += blocks[i]->d.nelem * (long long)blocks[i]->M;
    }
    int rc = asm_number(a, vertex_ids);
    if (!rc && cudaStreamCreateWithFlags(&a->cap_stream, cudaStreamNonBlocking) != cudaSuccess) rc = NIR_ERR_CUDA;
    if (!rc)
        for (int o = 0; o < 2 && !rc; ++o)
            for (int f = 0; f < 2 && !rc; ++f) {
                a->ops[o][f] = new (std::nothrow) AsmOp(a, o, f == 1);
                if (!a->ops[o][f]) rc = NIR_ERR_NO_MEMORY;
            }
    if (rc) {
        asm_free(a);
        return rc;
    }
    *out = a;
    return NIR_OK;
}

extern "C" int nir_c0_numbering(int shape, int P, int basis, int nblocks, const int64_t *nelem,
                                const int64_t *const *vertex_ids, int64_t *map_out, int64_t *n_global, int64_t *n_free)
{
    if ((shape != NIR_QUAD && shape != NIR_HEX)) return NIR_ERR_UNSUPPORTED;
    if (basis != NIR_BASIS_MODIFIED && basis != NIR_BASIS_GLL_LAGRANGE) return NIR_ERR_INVALID_ARG;
    if (P < 1 || P > 9 || nblocks < 1 || !nelem || !vertex_ids) return NIR_ERR_INVALID_ARG;
    std::vector<long long> ne;
    for (int b = 0; b < nblocks; ++b) {
        if (nelem[b] < 1 || !vertex_ids[b]) return NIR_ERR_INVALID_ARG;
        ne.push_back(nelem[b]);
    }
    std::vector<int> map;
    long long ng = 0, nf = 0;
    int rc = c0_numbering(shape == NIR_HEX ? 3 : 2, P, basis, ne, vertex_ids, map, ng, nf);
    if (rc) return rc;
    if (map_out)
        for (size_t i = 0; i < map.size(); ++i) map_out[i] = map[i];
    if (n_global) *n_global = ng;
    if (n_free) *n_free = nf;
    return NIR_OK;
}

extern "C" void nir_asm_destroy(nir_asm *a)
{
    if (!a) return;
    cudaSetDevice(a->ctx->device);
    cudaStreamSynchronize(a->ctx->stream);
    asm_free(a);
}

extern "C" int nir_asm_num_dofs(const nir_asm *a, int64_t *n_global, int64_t *n_free, int64_t *n_local)
{
    if (!a) return NIR_ERR_INVALID_ARG;
    if (n_global) *n_global = a->nglob;
    if (n_free) *n_free = a->nfree;
    if (n_local) *n_local = a->nloc;
    return NIR_OK;
}

extern "C" int nir_asm_local_map(const nir_asm *a, int64_t *map_out)
{
    if (!a || !map_out) return NIR_ERR_INVALID_ARG;
    for (long long i = 0; i < a->nloc; ++i) map_out[i] = a->map_h[(size_t)i];
    return NIR_OK;
}

extern "C" int nir_asm_gather(nir_asm *a, int prec, const void *x_global, void *x_local)
{
    if (!a || !valid_prec(prec) || !x_global || !x_local || x_global == x_local) return NIR_ERR_INVALID_ARG;
    cudaStream_t st = a->ctx->stream;
    if (prec == NIR_F64)
        k_gather<double><<<vgrid(a->nloc), kVT, 0, st>>>(static_cast<const double *>(x_global), a->nglob,
                                                                 a->map, a->nloc, static_cast<double *>(x_local));
    else if (prec == NIR_F32)
        k_gather<float><<<vgrid(a->nloc), kVT, 0, st>>>(static_cast<const float *>(x_global), a->nglob, a->map,
                                                               a->nloc, static_cast<float *>(x_local));
    else
        k_gather<__nv_bfloat16><<<vgrid(a->nloc), kVT, 0, st>>>(
            static_cast<const __nv_bfloat16 *>(x_global), a->nglob, a->map, a->nloc,
            static_cast<__nv_bfloat16 *>(x_local));
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return NIR_ERR_CUDA;
    }
    return nir_debug_after(a->ctx, NIR_OK);
}

extern "C" int nir_asm_assemble(nir_asm *a, int prec, const void *y_local, void *y_global)
{
    if (!a || !valid_prec(prec) || !y_local || !y_global || y_local == y_global) return NIR_ERR_INVALID_ARG;
    cudaStream_t st = a->ctx->stream;
    const long long n = a->nglob;
    if (prec == NIR_F64)
        k_assemble<double, double><<<vgrid(n), kVT, 0, st>>>(static_cast<const double *>(y_local), a->rowptr, a->pos,
                                                             n, static_cast<double *>(y_global), 0);
    else if (prec == NIR_F32)
        k_assemble<float, float><<<vgrid(n), kVT, 0, st>>>(static_cast<const float *>(y_local), a->rowptr, a->pos, n,
                                                           static_cast<float *>(y_global), 0);
    else
        k_assemble<__nv_bfloat16, __nv_bfloat16><<<vgrid(n), kVT, 0, st>>>(
            static_cast<const __nv_bfloat16 *>(y_local), a->rowptr, a->pos, n, static_cast<__nv_bfloat16 *>(y_global),
            0);
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return NIR_ERR_CUDA;
    }
    return nir_debug_after(a->ctx, NIR_OK);
}

extern "C" int nir_asm_pick(nir_asm *a, const double *x_local, double *x_global)
{
    if (!a || !x_local || !x_global || (const void *)x_local == (const void *)x_global) return NIR_ERR_INVALID_ARG;
    k_pick<<<vgrid(a->nglob), kVT, 0, a->ctx->stream>>>(x_local, a->rowptr, a->pos, a->nglob, x_global);
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return NIR_ERR_CUDA;
    }
    return nir_debug_after(a->ctx, NIR_OK);
}

extern "C" int nir_asm_apply(nir_asm *a, int op, double lambda, int prec, const void *x_global, void *y_global)
{
    if (!a || (op != NIR_ASM_HELMHOLTZ && op != NIR_ASM_MASS) || !valid_prec(prec) || !x_global || !y_global ||
        x_global == y_global || !std::isfinite(lambda))
        return NIR_ERR_INVALID_ARG;
    for (nir_block *b : a->blocks)
        if (!b->geo_set) return NIR_ERR_STATE;
    return nir_debug_after(a->ctx,
                           launch_apply(a, op, prec, lambda, x_global, a->nglob, y_global, a->nglob, a->ctx->stream));
}

extern "C" int nir_asm_cg_solve(nir_asm *a, int op, double lambda, int fix_boundary, const double *b, double *x,
                                const nir_cg_opts *o, nir_cg_stats *stats)
{
    if (!a || (op != NIR_ASM_HELMHOLTZ && op != NIR_ASM_MASS) || (fix_boundary != 0 && fix_boundary != 1))
        return NIR_ERR_INVALID_ARG;
    if (op == NIR_ASM_HELMHOLTZ && !(lambda > 0.0) && !fix_boundary) return NIR_ERR_INVALID_ARG;  // singular
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return NIR_ERR_INVALID_ARG;
    for (nir_block *b : a->blocks)
        if (!b->geo_set) return NIR_ERR_STATE;
    // captured graphs and the preconditioner follow the blocks' geometry and tuning
    std::vector<unsigned long long> state;
    for (nir_block *b : a->blocks) state.push_back(block_state(b));
    if (state != a->state_seen) {
        for (int oo = 0; oo < 2; ++oo)
            for (int f = 0; f < 2; ++f) nir_cg_work_invalidate(a->cg[oo][f]);
        a->state_seen = state;
    }
    if (op == NIR_ASM_MASS) lambda = 0.0;
    if (a->ops[op][fix_boundary]->n() == 0) {  // every dof held: nothing to solve
        if (stats) *stats = nir_cg_stats{0, 0, 0.0, 0.0, 0.0};
        return NIR_OK;
    }
    return nir_cg_run(*a->ops[op][fix_boundary], a->cg[op][fix_boundary], lambda, b, x, o, stats);
}
