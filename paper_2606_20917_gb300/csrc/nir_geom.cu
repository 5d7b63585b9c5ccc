// nir_geom.cu -- FP64 geometric factors on the GPU, precision conversion of
// the factors, and the FP64 FMA throughput probe.  The factors come either
// from the element maps (k_geometry) or from the caller's d xi/d x and |J|
// (k_geometry_from_factors); both finish through store_factors.
//
// Per point (or once per element for undeformed quad/hex blocks) the kernel
// forms the Jacobian J = dx/dxi of the element map, W = w |J| (the weights
// matrix of Sec. 2.1), d xi/d x = J^{-1} (Lambda of Eq. physderiv), the
// collapsed-coordinate factors d eta/d xi (Sec. 2.2, D_xi = Lambda(d eta/d xi)
// D_eta) and their product d eta/d x, and the symmetric metric
//   G_ij = W sum_l (d eta_i/d x_l)(d eta_j/d x_l).
#include <cuda_bf16.h>

#include "nir_geom.h"
#include "nir_internal.h"
#include "nir_layout.h"

#include "nir_geom_kernels.cuh"

int nir_probe_mma_launch(double *sink, int grid, int iters, cudaStream_t st)
{
    nirk::k_dmma_probe<<<grid, 256, 0, st>>>(sink, iters, 0.25, 1e-3);
    return cudaPeekAtLastError() == cudaSuccess ? NIR_OK : (cudaGetLastError(), NIR_ERR_CUDA);
}

int nir_geom_launch(const nirk::GeoArgs &a, cudaStream_t st)
{
    const long long total = a.pp ? a.nelem * nirk::npts(a.shape, a.Q) : a.nelem;
    long long blocks = (total + 255) / 256;
    if (blocks > 65535LL * 8) blocks = 65535LL * 8;
    nirk::k_geometry<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? NIR_OK : (cudaGetLastError(), NIR_ERR_CUDA);
}

int nir_geom_factors_launch(const nirk::GeoArgs &a, cudaStream_t st)
{
    const long long total = a.pp ? a.nelem * nirk::npts(a.shape, a.Q) : a.nelem;
    long long blocks = (total + 255) / 256;
    if (blocks > 65535LL * 8) blocks = 65535LL * 8;
    nirk::k_geometry_from_factors<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? NIR_OK : (cudaGetLastError(), NIR_ERR_CUDA);
}

int nir_convert_launch(const double *src, float *d32, void *d16, long long n, cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    if (blocks > 65535LL * 8) blocks = 65535LL * 8;
    if (d32) nirk::k_to_f32<<<(unsigned)blocks, 256, 0, st>>>(src, d32, n);
    if (d16) nirk::k_to_bf16<<<(unsigned)blocks, 256, 0, st>>>(src, reinterpret_cast<__nv_bfloat16 *>(d16), n);
    return cudaPeekAtLastError() == cudaSuccess ? NIR_OK : (cudaGetLastError(), NIR_ERR_CUDA);
}

int nir_pack_metric_launch(const double *src, float *d32, void *d16, long long nblocks, int ng, cudaStream_t st)
{
    long long blocks = (nblocks * ng * 32 + 255) / 256;
    if (blocks > 65535LL * 8) blocks = 65535LL * 8;
    if (d32) nirk::k_pack_metric<float><<<(unsigned)blocks, 256, 0, st>>>(src, d32, nblocks, ng);
    if (d16)
        nirk::k_pack_metric<__nv_bfloat16>
            <<<(unsigned)blocks, 256, 0, st>>>(src, reinterpret_cast<__nv_bfloat16 *>(d16), nblocks, ng);
    return cudaPeekAtLastError() == cudaSuccess ? NIR_OK : (cudaGetLastError(), NIR_ERR_CUDA);
}

int nir_probe_launch(double *sink, int grid, int iters, cudaStream_t st)
{
    nirk::k_dfma_probe<<<grid, 256, 0, st>>>(sink, iters, 0.9999999, 1e-7);
    return cudaPeekAtLastError() == cudaSuccess ? NIR_OK : (cudaGetLastError(), NIR_ERR_CUDA);
}
