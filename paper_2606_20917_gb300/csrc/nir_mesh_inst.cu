// nir_mesh_inst.cu -- persistent hybrid-mesh Helmholtz kernel for one spatial
// dimension and one precision (compiled per NIR_MESH_DIM x NIR_PREC).
//
// Blocks of alike elements (Sec. 3.1: same shape, order, quadrature) are
// batched into one launch (Sec. 2.2 last paragraph).  The work list holds
// (block, first group, group count) items sorted by estimated cost, longest
// first; CTAs take items from an atomic counter until it runs past the end, so
// no CTA waits on another.  Each item dispatches to the (shape, P) variant of
// its block; the basis tables are copied into shared memory only when a CTA
// moves to a different block.
#include "nir_internal.h"
#include "nir_kernels.cuh"
#include "nir_mesh.h"

#ifndef NIR_MESH_DIM
#error "NIR_MESH_DIM must be defined"
#endif
#ifndef NIR_PREC
#error "NIR_PREC must be defined"
#endif

namespace nirk {
namespace {

#if NIR_PREC == 0
using TT = double;
#elif NIR_PREC == 1
using TT = float;
#else
using TT = __nv_bfloat16;
#endif

#if NIR_MESH_DIM == 3
constexpr int kShapes[4] = {HEX, PRISM, TET, PYR};
#else
constexpr int kShapes[2] = {QUAD, TRI};
#endif
constexpr int kNumShapes = sizeof(kShapes) / sizeof(int);
// variants per shape: N = P + 1 = 2 .. 10
constexpr int kPerShape = 9;

// every variant of one persistent kernel runs with the same thread count
constexpr int kMeshNT = sizeof(typename CT<TT>::type) == 8 ? 256 : 512;

// FP32/BF16 kernels take the contractions' table values as constant-bank
// operands, as the single-block kernels do with their table parameter: the
// tables of every (shape, P) variant of this kernel live in one __constant__
// array at compile-time offsets (tables depend on shape and P only, so all
// blocks of a variant share them).  The reference weights, read only by the
// per-element-factor path and the gathers, are left out (they stay in the
// shared-memory copy); only the variants that use the constant bank (use_ctab)
// take space in it.
//
// Constant-bank table operands let the compiler keep more values live: the
// high-order variants would need up to 128 registers, and one persistent
// kernel has a single register budget for all variants.  Variants whose
// constant-table form fits in 64 registers use it; the others read their
// tables from shared memory (the kernel is capped at 64 registers, two
// 512-thread CTAs per SM).
NIR_HD constexpr bool use_ctab(int SH, int N)
{
    return SH == HEX ? N <= 4 : SH == PRISM ? N <= 5 : (SH == TET || SH == PYR) ? N <= 3 : true;
}

template <int VID>
NIR_HD constexpr int ctab_size()
{
    constexpr int SH = kShapes[VID / kPerShape], N = VID % kPerShape + 2, Q = N + 1;
    return use_ctab(SH, N) ? layout(SH, N, Q).total - npts(SH, Q) : 0;
}

template <int VID>
NIR_HD constexpr int ctab_base()
{
    if constexpr (VID == 0) return 0;
    else return ctab_base<VID - 1>() + ctab_size<VID - 1>();
}

constexpr int kCTabN = ctab_base<kNumShapes * kPerShape - 1>() + ctab_size<kNumShapes * kPerShape - 1>();

#if NIR_PREC != 0
__constant__ float c_tab[kCTabN];

// VB: the variant's base; WQ, GAP: where the omitted weights started and how many
template <int VB, int WQ, int GAP>
struct CTab {
    int base;
    __device__ __forceinline__ CTab operator+(int o) const { return CTab{base + o}; }
    __device__ __forceinline__ float operator()(int, int i) const
    {
        const int k = base + i;
        return c_tab[VB + (k < WQ ? k : k - GAP)];
    }
};
#endif

template <int SH, int N, int VID>
__device__ __noinline__ void run_item(const MeshBlk &mb, const MeshItem &m, unsigned char *smem, int &cur)
{
    using C = Config<SH, N, N + 1, TT, OP_HELM, 0, kMeshNT>;
    using A = typename C::A;
    A *tab = reinterpret_cast<A *>(smem);
    A *buf = reinterpret_cast<A *>(smem + C::TABB);
    if (cur != m.block) {
        const A *gt = reinterpret_cast<const A *>(mb.a.tab);
        for (int i = threadIdx.x; i < C::TABN; i += C::NT) tab[i] = gt[i];
        __syncthreads();
        cur = m.block;
    }
    for (int g = m.g0; g < m.g0 + m.ng; ++g) {
        const long long e0 = (long long)g * C::EPB;
        const long long left = mb.a.nelem - e0;
        const int ne = (int)(left < C::EPB ? left : C::EPB);
#if NIR_PREC != 0
        // the constant tables hold the modified basis' tables of the variant;
        // a nodal-basis block reads its own tables from shared memory
        if constexpr (use_ctab(SH, N)) {
            if (!mb.a.nodal) {
                constexpr TabLayout L = layout(SH, N, N + 1);
                using CT = CTab<ctab_base<VID>(), L.wq, npts(SH, N + 1)>;
                run_group<SH, N, N + 1, TT, OP_HELM, 0, kMeshNT>(mb.a, mb.a.in0, mb.a.out0, CT{0}, tab, buf, e0, ne);
            } else {
                run_group<SH, N, N + 1, TT, OP_HELM, 0, kMeshNT>(mb.a, mb.a.in0, mb.a.out0, STab<A>{tab}, tab, buf, e0, ne);
            }
        } else {
            run_group<SH, N, N + 1, TT, OP_HELM, 0, kMeshNT>(mb.a, mb.a.in0, mb.a.out0, STab<A>{tab}, tab, buf, e0, ne);
        }
#else
        run_group<SH, N, N + 1, TT, OP_HELM, 0, kMeshNT>(mb.a, mb.a.in0, mb.a.out0, STab<A>{tab}, tab, buf, e0, ne);
#endif
    }
}

template <int VID>
__device__ __forceinline__ void dispatch_one(int vid, const MeshBlk &mb, const MeshItem &m, unsigned char *smem,
                                             int &cur)
{
    if constexpr (VID < kNumShapes * kPerShape) {
        if (vid == VID) {
            run_item<kShapes[VID / kPerShape], VID % kPerShape + 2, VID>(mb, m, smem, cur);
            return;
        }
        dispatch_one<VID + 1>(vid, mb, m, smem, cur);
    }
}


__global__ void __launch_bounds__(kMeshNT, 2) k_mesh(const MeshBlk *__restrict__ blks, const MeshItem *__restrict__ items,
                                              int nitems, int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const MeshItem m = items[it];
        const MeshBlk mb = blks[m.block];
        dispatch_one<0>(mb.vid, mb, m, smem_raw, cur);
    }
}

template <int VID>
int smem_of(int vid)
{
    if constexpr (VID < kNumShapes * kPerShape) {
        if (vid == VID) return Config<kShapes[VID / kPerShape], VID % kPerShape + 2, VID % kPerShape + 3, TT, OP_HELM, 0, kMeshNT>::SMEM;
        return smem_of<VID + 1>(vid);
    }
    return -1;
}

template <int VID>
int epb_of(int vid)
{
    if constexpr (VID < kNumShapes * kPerShape) {
        if (vid == VID) return Config<kShapes[VID / kPerShape], VID % kPerShape + 2, VID % kPerShape + 3, TT, OP_HELM, 0, kMeshNT>::EPB;
        return epb_of<VID + 1>(vid);
    }
    return -1;
}

}  // namespace
}  // namespace nirk

namespace nirk {
namespace {
template <int VID>
void ctab_range(int vid, int &base, int &wq, int &gap, int &total, bool &used)
{
    if constexpr (VID < kNumShapes * kPerShape) {
        if (vid == VID) {
            constexpr int SH = kShapes[VID / kPerShape], N = VID % kPerShape + 2, Q = N + 1;
            used = use_ctab(SH, N);
            base = ctab_base<VID>();
            wq = layout(SH, N, Q).wq;
            gap = npts(SH, Q);
            total = layout(SH, N, Q).total;
            return;
        }
        ctab_range<VID + 1>(vid, base, wq, gap, total, used);
    }
}
}  // namespace
}  // namespace nirk

#define NIR_MCAT2(a, b) nir_mesh_kinfo_d##a##_p##b
#define NIR_MCAT(a, b) NIR_MCAT2(a, b)
#define NIR_TCAT2(a, b) nir_mesh_tables_d##a##_p##b
#define NIR_TCAT(a, b) NIR_TCAT2(a, b)

// Copy variant vid's FP32 table blob (the full layout, n values) into the
// kernel's constant tables, without the reference weights.  FP64 kernels, and
// FP32/BF16 variants that read their tables from shared memory (no space in
// the constant array), need nothing.
int NIR_TCAT(NIR_MESH_DIM, NIR_PREC)(int vid, const float *blob, int n, cudaStream_t st)
{
#if NIR_PREC != 0
    using namespace nirk;
    int base = -1, wq = 0, gap = 0, total = 0;
    bool used = false;
    ctab_range<0>(vid, base, wq, gap, total, used);
    if (base < 0 || n != total || !blob) return NIR_ERR_INVALID_ARG;
    if (!used) return NIR_OK;
    if (base + total - gap > kCTabN) return NIR_ERR_INVALID_ARG;  // never: the layout reserves exactly this
    if (cudaMemcpyToSymbolAsync(c_tab, blob, sizeof(float) * wq, sizeof(float) * base, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_tab, blob + wq + gap, sizeof(float) * (total - wq - gap), sizeof(float) * (base + wq),
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
        return NIR_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? NIR_OK : NIR_ERR_CUDA;
#else
    (void)vid; (void)blob; (void)n; (void)st;
    return NIR_OK;
#endif
}

MeshKInfo NIR_MCAT(NIR_MESH_DIM, NIR_PREC)(int shape, int P)
{
    using namespace nirk;
    MeshKInfo k;
    int si = -1;
    for (int i = 0; i < kNumShapes; ++i)
        if (kShapes[i] == shape) si = i;
    if (si < 0 || P < 1 || P > kPerShape) return k;
    k.vid = si * kPerShape + (P - 1);
    k.fn = reinterpret_cast<const void *>(&k_mesh);
    k.smem = smem_of<0>(k.vid);
    k.epb = epb_of<0>(k.vid);
    k.nt = kMeshNT;
    return k;
}
