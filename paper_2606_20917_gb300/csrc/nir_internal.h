// nir_internal.h -- library-internal objects of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nir.h"

namespace nirk {
struct KArgs;
}

// Chunks of the pipelined host-buffer Helmholtz.
#define NIR_HOST_CHUNKS 8

// Kernel registry entry of one (shape, P, precision, operator) instantiation.
struct KInfo {
    const void *fn = nullptr;  // __global__ function
    int smem = 0;              // dynamic shared memory bytes
    int epb = 0;               // elements per CTA group
    int nt = 0;                // threads per CTA
    int tabp_bytes = 0;        // size of the table parameter (compute type)
    const void *fn_fields = nullptr;  // Helmholtz, default variant: the multi-field form
};

// Debug mode: after a successful operator launch, synchronise the context
// stream (unless it is being captured) and report a launch failure or a set
// device error word at this call.  Returns rc unchanged otherwise.
int nir_debug_after(nir_ctx *ctx, int rc);

// Provided by the instantiation units (one per shape x precision).
KInfo nir_kinfo(int shape, int P, int prec, int op, int variant);
// The threading-over-elements Helmholtz kernel (Helmholtz variant 4).
KInfo nir_toe_kinfo(int shape, int P, int prec);
#define NIR_VARIANT_TOE 4
// The FP32/BF16 Helmholtz with two elements per thread (quad/hex).
#define NIR_VARIANT_PAIR 5
#define NIR_VARIANT_MAX 5

struct nir_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int *derr = nullptr;                    // device error word of bounded in-kernel waits
    bool debug = false;                     // check every operator call synchronously
    std::mutex mu;
    std::map<const void *, int> occupancy;  // CTAs per SM per kernel
    std::map<std::string, int> tuned_grid;  // autotuner overrides (key: shape/P/prec/op)
};

struct nir_block {
    nir_ctx *ctx = nullptr;
    nir_block_desc d{};
    int dim = 0, N = 0, M = 0, NQ = 0, ng = 0, nl = 0;
    long long epad = 0;                       // element count padded to 64
    std::vector<double> tab_h;                // FP64 table blob (host)
    std::vector<float> tab32_h;               // the same tables rounded to FP32 (host)
    double *tab64 = nullptr;                  // table blob, device, FP64
    float *tab32 = nullptr;                   // table blob, device, FP32
    int geo_pp = 1;                           // per-point (1) or per-element (0) factors
    int helm_variant[3] = {0, 0, 0};          // tuned elements-per-CTA variant per precision
    int helm_grid[3] = {0, 0, 0};             // tuned grid size per precision (0: occupancy)
    int helm_pf[3] = {0, 0, 0};               // tuned L2 metric-prefetch policy per precision
    int toe_grid[3] = {0, 0, 0};              // CTAs of the threading-over-elements kernel per precision
    void *toe_scr = nullptr;                  // its per-thread scratch (shared by the precisions)
    size_t toe_bytes = 0;
    bool geo_set = false;
    unsigned geo_version = 0;                 // bumped by every nir_block_set_geometry (and scratch moves)
    double *G64 = nullptr, *L64 = nullptr;    // metric (ng) and d eta/d x + W (nl)
    float *G32 = nullptr, *L32 = nullptr;
    void *G16 = nullptr, *L16 = nullptr;      // bfloat16 copies
    void *stage_in = nullptr, *stage_out = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;   // host-buffer pipeline streams
    cudaEvent_t ev_in[NIR_HOST_CHUNKS] = {}, ev_done[NIR_HOST_CHUNKS] = {};
    // host-buffer pipelines captured as graphs (pinned host buffers only)
    struct HostGraph {
        int prec = 0;
        double lambda = 0.0;
        const void *h_in = nullptr;
        void *h_out = nullptr;
        unsigned long long state = 0;   // geometry version and tuning at capture
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<HostGraph> host_graphs;
    cudaStream_t cap = nullptr;                           // capture origin of those graphs
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

int nir_launch_op(nir_block *blk, int prec, int op, double lambda, const void *in0, const void *in1,
                  const void *in2, void *out0, void *out1, void *out2, cudaStream_t stream, int grid_override);
int nir_launch_op_range(nir_block *b, int prec, int op, double lambda, const void *in0, const void *in1,
                        const void *in2, void *out0, void *out1, void *out2, long long e_begin, long long e_count,
                        cudaStream_t stream, int grid_override);
// Size the threading-over-elements scratch for `grid` CTAs (0: one wave at
// the kernel's occupancy; at most one CTA per 128 elements) and record the
// grid; never called during capture.
int nir_toe_prepare(nir_block *b, int prec, int grid);
// Free that scratch unless a precision of the block is tuned to use it.
void nir_toe_release(nir_block *b);
const void *nir_geo_ptr(nir_block *blk, int prec, bool lam);
const void *nir_tab_ptr(nir_block *blk, int prec);
int nir_occupancy(nir_ctx *ctx, const KInfo &ki);
// Derive the block's FP32/BF16 geometric factors if needed (allocates once).
int nir_block_ensure_prec(nir_block *b, int prec);
size_t nir_prec_size(int prec);

#define NIR_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return NIR_ERR_CUDA;          \
    } while (0)
