// nir_noalloc.cu -- host-buffer Helmholtz apply that never allocates device
// memory.
//
// nir_helmholtz_host stages the caller's host arrays through device buffers it
// allocates with cudaMalloc on first use.  Some callers cannot let a library
// do that: applications whose device memory is owned by a pool or caching
// allocator (a stray cudaMalloc/cudaFree fragments the pool, escapes its
// accounting, and implicitly synchronises the whole device), real-time loops
// that must not stall on an allocation, and hosts that forbid allocation once
// set-up is over.  For them this variant stages through one fixed array in
// the library's own device image instead.  The array is a file-scope
// __device__ variable, so every GPU that loads the library holds its
// NIR_NOALLOC_SCRATCH_BYTES until the process exits.
//
// Host code cannot use the array's name as a device address (it names a host
// shadow of the symbol), so the device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, on the first call made
// on that device.
#include <cuda_runtime.h>

#include <mutex>

#include "nir_internal.h"
#include "nir_kernels.cuh"

namespace {

constexpr size_t kHalf = NIR_NOALLOC_MAX_VECTOR_BYTES;  // one staged vector
constexpr size_t kTotal = 2 * kHalf;                     // input half + output half

static __device__ __align__(256) unsigned char g_noalloc_scratch[kTotal];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
int scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) return NIR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_dev_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return NIR_ERR_CUDA;
        g_dev_ptr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[device];
    return NIR_OK;
}

}  // namespace

extern "C" int nir_helmholtz_host_noalloc(nir_block *b, int prec, double lambda, const void *h_in, void *h_out)
{
    if (!b || !h_in || !h_out || h_in == h_out) return NIR_ERR_INVALID_ARG;
    if (prec != NIR_F64 && prec != NIR_F32 && prec != NIR_BF16) return NIR_ERR_INVALID_ARG;
    if (!(lambda == lambda) || lambda > 1e300 || lambda < -1e300) return NIR_ERR_INVALID_ARG;
    if (!b->geo_set) return NIR_ERR_STATE;
    const size_t bytes = (size_t)b->d.nelem * b->M * nir_prec_size(prec);
    if (bytes > kHalf) return NIR_ERR_TOO_LARGE;
    // the FP32/BF16 geometric factors are derived (allocated) by the first
    // allocating call in that precision; this entry point will not create them
    if ((prec == NIR_F32 && !b->G32) || (prec == NIR_BF16 && !b->G16)) return NIR_ERR_STATE;
    if (cudaSetDevice(b->ctx->device) != cudaSuccess) return NIR_ERR_CUDA;
    unsigned char *base = nullptr;
    int rc = scratch_address(b->ctx->device, &base);
    if (rc) return rc;
    void *d_in = base, *d_out = base + kHalf;
    cudaStream_t st = b->ctx->stream;
    NIR_CUDA_TRY(cudaMemcpyAsync(d_in, h_in, bytes, cudaMemcpyHostToDevice, st));
    rc = nir_launch_op(b, prec, nirk::OP_HELM, lambda, d_in, nullptr, nullptr, d_out, nullptr, nullptr, st, 0);
    if (!rc && cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = NIR_ERR_CUDA;
    // once a copy from h_in is queued, return only after the stream has drained
    // (also on failure), so the caller may reuse h_in and h_out at once
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NIR_ERR_CUDA;
    return rc;
}
