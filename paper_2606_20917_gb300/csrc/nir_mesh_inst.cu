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
constexpr int kShapes[3] = {HEX, PRISM, TET};
#else
constexpr int kShapes[2] = {QUAD, TRI};
#endif
constexpr int kNumShapes = sizeof(kShapes) / sizeof(int);

template <int SH, int N>
__device__ __noinline__ void run_item(const MeshBlk &mb, const MeshItem &m, unsigned char *smem, int &cur)
{
    using C = Config<SH, N, N + 1, TT, OP_HELM, 0>;
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
        run_group<SH, N, N + 1, TT, OP_HELM, 0>(mb.a, STab<A>{tab}, tab, buf, e0, ne);
    }
}

template <int VID>
__device__ __forceinline__ void dispatch_one(int vid, const MeshBlk &mb, const MeshItem &m, unsigned char *smem,
                                             int &cur)
{
    if constexpr (VID < kNumShapes * 8) {
        if (vid == VID) {
            run_item<kShapes[VID / 8], VID % 8 + 2>(mb, m, smem, cur);
            return;
        }
        dispatch_one<VID + 1>(vid, mb, m, smem, cur);
    }
}

constexpr int kMeshNT = Config<HEX, 5, 6, TT, OP_HELM, 0>::NT;  // the same for every variant

__global__ void __launch_bounds__(kMeshNT) k_mesh(const MeshBlk *__restrict__ blks, const MeshItem *__restrict__ items,
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
    if constexpr (VID < kNumShapes * 8) {
        if (vid == VID) return Config<kShapes[VID / 8], VID % 8 + 2, VID % 8 + 3, TT, OP_HELM, 0>::SMEM;
        return smem_of<VID + 1>(vid);
    }
    return -1;
}

template <int VID>
int epb_of(int vid)
{
    if constexpr (VID < kNumShapes * 8) {
        if (vid == VID) return Config<kShapes[VID / 8], VID % 8 + 2, VID % 8 + 3, TT, OP_HELM, 0>::EPB;
        return epb_of<VID + 1>(vid);
    }
    return -1;
}

}  // namespace
}  // namespace nirk

#define NIR_MCAT2(a, b) nir_mesh_kinfo_d##a##_p##b
#define NIR_MCAT(a, b) NIR_MCAT2(a, b)

MeshKInfo NIR_MCAT(NIR_MESH_DIM, NIR_PREC)(int shape, int P)
{
    using namespace nirk;
    MeshKInfo k;
    int si = -1;
    for (int i = 0; i < kNumShapes; ++i)
        if (kShapes[i] == shape) si = i;
    if (si < 0 || P < 1 || P > 8) return k;
    k.vid = si * 8 + (P - 1);
    k.fn = reinterpret_cast<const void *>(&k_mesh);
    k.smem = smem_of<0>(k.vid);
    k.epb = epb_of<0>(k.vid);
    k.nt = kMeshNT;
    return k;
}
