// nir_cg.h -- the conjugate-gradient solver's view of a linear operator, so
// one solver serves the broken (element-block-diagonal) mesh operator and the
// assembled C0 operator.
#pragma once

#include <cuda_runtime.h>

#include "nir_internal.h"

struct CGWork;

// A symmetric positive definite operator on n unknowns.  Vectors x of the
// outer FP64 solve hold n_full >= n entries: the n unknowns first, then fixed
// values (Dirichlet data) that enter the FP64 residual only.
struct CgOperator {
    virtual ~CgOperator() {}
    virtual nir_ctx *context() = 0;
    virtual long long n() = 0;
    virtual long long n_full() = 0;
    virtual cudaStream_t capture_stream() = 0;
    // Bind y = H x in precision prec to fixed buffers (n entries of the
    // precision's type) so that launch() can be captured into a CUDA graph.
    virtual int prepare(int prec, double lambda, const void *x, void *y, void **handle) = 0;
    virtual int launch(void *handle, cudaStream_t st) = 0;
    virtual void release(void *handle) = 0;
    // y[0:n] = (H x)[0:n] in FP64, x with n_full entries (not captured).
    virtual int apply64(double lambda, const double *x, double *y, cudaStream_t st) = 0;
    // FP64 diagonal of H, n entries.
    virtual int diagonal(double lambda, double *d, cudaStream_t st) = 0;
};

// Sum of FP64 scalars over the ranks of a sharded solve (nir_cg_solve_dist).
struct CgReducer {
    nir_allreduce_fn fn;
    void *user;
    int sum(double *v, int n) const;   // NIR_OK or NIR_ERR_COMM
};

// Solve H x = b (see nir_cg_solve in nir.h for the options); w is the
// operator's solver workspace, allocated on first use.  red: null for a
// single-rank solve; otherwise every dot product is summed over the ranks.
int nir_cg_run(CgOperator &op, CGWork *&w, double lambda, const double *b, double *x, const nir_cg_opts *o,
               nir_cg_stats *stats, const CgReducer *red = nullptr);
// Drop captured iteration graphs and the preconditioner (operator changed).
void nir_cg_work_invalidate(CGWork *w);
void nir_cg_work_free(CGWork *&w);
