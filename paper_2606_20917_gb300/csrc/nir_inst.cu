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

template <int N, int OP, int EPB, bool STAGE = true, bool PAIR = false>
KInfo make1()
{
    using C = Config<NIR_SHAPE, N, N + 1, TT, OP, EPB, 0, PAIR>;
    KInfo k;
    if constexpr (C::FUSED) {  // FP32/BF16 Helmholtz: bulk-copy staged kernel
        constexpr int stg = STAGE ? ((C::EPB * C::M * (int)sizeof(TT) + 15) / 16) * 16 : 0;
        k.fn = reinterpret_cast<const void *>(&k_helm_tma<NIR_SHAPE, N, N + 1, TT, EPB, STAGE, false, PAIR>);
        if constexpr (EPB == 0 && STAGE && !PAIR)
            k.fn_fields = reinterpret_cast<const void *>(&k_helm_tma<NIR_SHAPE, N, N + 1, TT, 0, true, true>);
        k.smem = C::SMEM + stg;
    } else {
        k.fn = reinterpret_cast<const void *>(&k_elem<NIR_SHAPE, N, N + 1, TT, OP, EPB>);
        if constexpr (EPB == 0 && OP == OP_HELM)
            k.fn_fields = reinterpret_cast<const void *>(&k_elem<NIR_SHAPE, N, N + 1, TT, OP, 0, true>);
        k.smem = C::SMEM;
    }
    k.epb = C::EPB;
    k.nt = C::NT;
    k.tabp_bytes = C::TABN * (int)sizeof(typename C::A);
    return k;
}

// Variant 0: default elements per CTA; 1: half; 2: double (when it fits in
// 227 KB of shared memory; an FP32/BF16 double group that fits only without
// its staging buffer loads its coefficients itself); 3: the default group run
// by the multi-field kernel with one field (the compiler allocates its
// registers differently, which wins at some orders); 5 (FP32/BF16, quad and
// hex): the default group with two elements per thread (F2 values).  Only
// the Helmholtz operator has variants (4 is the threading-over-elements
// kernel, registered separately).
template <int N, int OP>
KInfo make(int variant)
{
    using C0 = Config<NIR_SHAPE, N, N + 1, TT, OP, 0>;
    constexpr int e0 = C0::EPB;
    constexpr int eh = e0 > 1 ? e0 / 2 : 1;
    constexpr int stg2 = C0::FUSED ? ((2 * e0 * C0::M * (int)sizeof(TT) + 15) / 16) * 16 : 0;
    constexpr bool fits = C0::TABB + 2 * C0::BUFB + stg2 <= 227 * 1024 && e0 < 64;
    constexpr bool fits_unstaged = C0::FUSED && !fits && C0::TABB + 2 * C0::BUFB <= 227 * 1024 && e0 < 64;
    constexpr int ed = (fits || fits_unstaged) ? 2 * e0 : e0;
    if constexpr (OP == OP_HELM) {
        if (variant == 1) return make1<N, OP, eh>();
        if (variant == 2) {
            if constexpr (fits_unstaged) return make1<N, OP, ed, false>();
            else return make1<N, OP, ed>();
        }
        if (variant == 3) {  // default group through the multi-field code: another register allocation
            KInfo k = make1<N, OP, 0>();
            if (!k.fn_fields) return KInfo{};
            k.fn = k.fn_fields;
            return k;
        }
        if (variant == 5) {  // two elements per thread
            if constexpr (C0::FUSED && (NIR_SHAPE == QUAD || NIR_SHAPE == HEX))
                return make1<N, OP, 0, true, true>();
            else return KInfo{};
        }
    }
    if (variant != 0) return KInfo{};
    return make1<N, OP, 0>();
}

template <int OP>
KInfo by_n(int N, int v)
{
    switch (N) {
    case 2: return make<2, OP>(v);
    case 3: return make<3, OP>(v);
    case 4: return make<4, OP>(v);
    case 5: return make<5, OP>(v);
    case 6: return make<6, OP>(v);
    case 7: return make<7, OP>(v);
    case 8: return make<8, OP>(v);
    case 9: return make<9, OP>(v);
    case 10: return make<10, OP>(v);
    default: return KInfo{};
    }
}

}  // namespace
}  // namespace nirk

#define NIR_CAT2(a, b, c) nir_kinfo_s##a##_p##b
#define NIR_CAT(a, b) NIR_CAT2(a, b, x)
#define NIR_KINFO_FN NIR_CAT(NIR_SHAPE, NIR_PREC)

KInfo NIR_KINFO_FN(int P, int op, int variant)
{
    using namespace nirk;
    const int N = P + 1;
    switch (op) {
    case OP_BWD: return by_n<OP_BWD>(N, variant);
    case OP_IPROD: return by_n<OP_IPROD>(N, variant);
    case OP_PHYSDERIV: return by_n<OP_PHYSDERIV>(N, variant);
    case OP_IPROD_DERIV: return by_n<OP_IPROD_DERIV>(N, variant);
    case OP_MASS: return by_n<OP_MASS>(N, variant);
    case OP_HELM: return by_n<OP_HELM>(N, variant);
    default: return KInfo{};
    }
}
