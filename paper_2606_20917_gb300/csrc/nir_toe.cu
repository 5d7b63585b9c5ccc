// nir_toe.cu -- instantiates the threading-over-elements Helmholtz kernels of
// one shape and one precision (compiled once per NIR_SHAPE x NIR_PREC).
#include "nir_internal.h"
#include "nir_toe.cuh"

#ifndef NIR_SHAPE
#error "NIR_SHAPE must be defined"
#endif
#ifndef NIR_PREC
#error "NIR_PREC must be defined"
#endif

namespace {

#if NIR_PREC == 0
using TT = double;
#elif NIR_PREC == 1
using TT = float;
#else
using TT = __nv_bfloat16;
#endif
using AA = nirt::CT<TT>::type;

template <int N>
KInfo mk()
{
    KInfo k;
    k.fn = reinterpret_cast<const void *>(&nirt::k_helm_toe<NIR_SHAPE, N, TT>);
    k.smem = nirt::toe_smem<NIR_SHAPE, N, AA>();
    k.nt = nirt::kThreads;
    k.epb = nirt::kThreads;  // one element per thread
    return k;
}

}  // namespace

#define NIR_TCAT2(a, b) nir_toe_kinfo_s##a##_p##b
#define NIR_TCAT(a, b) NIR_TCAT2(a, b)

KInfo NIR_TCAT(NIR_SHAPE, NIR_PREC)(int P)
{
    switch (P + 1) {
    case 2: return mk<2>();
    case 3: return mk<3>();
    case 4: return mk<4>();
    case 5: return mk<5>();
    case 6: return mk<6>();
    case 7: return mk<7>();
    case 8: return mk<8>();
    case 9: return mk<9>();
    case 10: return mk<10>();
    default: return KInfo{};
    }
}
