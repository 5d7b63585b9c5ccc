// nir_inst.cu -- instantiates the elemental-operator kernels of one shape and
// one precision (compiled once per NIR_SHAPE x NIR_PREC by the build script,
// so the translation units compile in parallel).
#include "nir_internal.h"
#include "nir_kernels.cuh"

#ifndef NIR_SHAPE
#error "NIR_SHAPE must be defined"
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

template <int N, int OP>
KInfo make()
{
    using C = Config<NIR_SHAPE, N, N + 1, TT, OP>;
    KInfo k;
    k.fn = reinterpret_cast<const void *>(&k_elem<NIR_SHAPE, N, N + 1, TT, OP>);
    k.smem = C::SMEM;
    k.epb = C::EPB;
    k.nt = C::NT;
    return k;
}

template <int OP>
KInfo by_n(int N)
{
    switch (N) {
    case 2: return make<2, OP>();
    case 3: return make<3, OP>();
    case 4: return make<4, OP>();
    case 5: return make<5, OP>();
    case 6: return make<6, OP>();
    case 7: return make<7, OP>();
    case 8: return make<8, OP>();
    case 9: return make<9, OP>();
    default: return KInfo{};
    }
}

}  // namespace
}  // namespace nirk

#define NIR_CAT2(a, b, c) nir_kinfo_s##a##_p##b
#define NIR_CAT(a, b) NIR_CAT2(a, b, x)
#define NIR_KINFO_FN NIR_CAT(NIR_SHAPE, NIR_PREC)

KInfo NIR_KINFO_FN(int P, int op)
{
    using namespace nirk;
    const int N = P + 1;
    switch (op) {
    case OP_BWD: return by_n<OP_BWD>(N);
    case OP_IPROD: return by_n<OP_IPROD>(N);
    case OP_PHYSDERIV: return by_n<OP_PHYSDERIV>(N);
    case OP_IPROD_DERIV: return by_n<OP_IPROD_DERIV>(N);
    case OP_MASS: return by_n<OP_MASS>(N);
    case OP_HELM: return by_n<OP_HELM>(N);
    default: return KInfo{};
    }
}
