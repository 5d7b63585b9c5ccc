// nir_geom.h -- launchers of the geometry, conversion and probe kernels.
#pragma once
#include <cuda_runtime.h>

namespace nirk {
struct GeoArgs {
    const double *nodes;
    const double *z;
    const double *wq;
    const double *Lg;
    const double *dLg;
    double *G;
    double *Lam;
    int *err;
    long long nelem;
    int shape, Q, g, pp;
    // caller-given factors (nir_geom_factors_launch): d xi/d x and |J|
    const double *dxi_dx = nullptr;
    const double *jac = nullptr;
    int per_elem = 0;
};
}  // namespace nirk

int nir_geom_launch(const nirk::GeoArgs &a, cudaStream_t st);
int nir_geom_factors_launch(const nirk::GeoArgs &a, cudaStream_t st);
int nir_convert_launch(const double *src, float *d32, void *d16, long long n, cudaStream_t st);
// Interleaved FP64 per-point metric -> packed FP32 / BF16 (geo_packed_index):
// nblocks = point blocks of 32 elements (chunks x points), ng values each.
int nir_pack_metric_launch(const double *src, float *d32, void *d16, long long nblocks, int ng, cudaStream_t st);
int nir_probe_launch(double *sink, int grid, int iters, cudaStream_t st);
int nir_probe_mma_launch(double *sink, int grid, int iters, cudaStream_t st);
