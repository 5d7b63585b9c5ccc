// nir_vec.cuh -- element type conversions shared by the vector kernels
// (CG updates, gathers and assembly): FP64 arithmetic on FP64, FP32 and
// bfloat16 storage.
#pragma once

#include <cuda_bf16.h>

namespace nirv {

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
__device__ __forceinline__ void st_v(double *p, double v) { *p = v; }
__device__ __forceinline__ void st_v(float *p, double v) { *p = (float)v; }
__device__ __forceinline__ void st_v(__nv_bfloat16 *p, double v) { *p = __float2bfloat16_rn((float)v); }

}  // namespace nirv
