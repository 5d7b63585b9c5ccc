// nir_solve.cu -- hybrid mesh, persistent launch, CUDA graph, autotuner and
// the mixed-precision conjugate-gradient solve (filled in below).
#include "nir_internal.h"

struct nir_mesh {
    nir_ctx *ctx = nullptr;
};

extern "C" int nir_mesh_create(nir_ctx *, nir_block *const *, int, nir_mesh **out)
{
    if (out) *out = nullptr;
    return NIR_ERR_UNSUPPORTED;
}
extern "C" void nir_mesh_destroy(nir_mesh *m) { delete m; }
extern "C" int nir_mesh_num_dofs(const nir_mesh *, int64_t *) { return NIR_ERR_UNSUPPORTED; }
extern "C" int nir_mesh_helmholtz(nir_mesh *, int, double, const void *, void *) { return NIR_ERR_UNSUPPORTED; }
extern "C" int nir_tune(nir_mesh *, const char *) { return NIR_ERR_UNSUPPORTED; }
extern "C" int nir_cg_solve(nir_mesh *, double, const double *, double *, const nir_cg_opts *, nir_cg_stats *)
{
    return NIR_ERR_UNSUPPORTED;
}
