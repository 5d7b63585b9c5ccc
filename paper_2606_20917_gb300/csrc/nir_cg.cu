// nir_cg.cu -- conjugate-gradient solve of an SPD operator (a mesh's broken,
// element-block-diagonal Helmholtz operator, or an assembled C0 operator),
// plain FP64 or mixed precision with FP64 iterative refinement (defect
// correction).
//
// The paper uses the Helmholtz operator inside CG iterations (Sec. 4, first
// paragraph); the solver itself is not described there.  Mixed precision:
//   r = b - H64 x                      (FP64 operator, FP64 vectors)
//   repeat: solve H_lo d = r / |r| by preconditioned CG with the operator in
//           FP32 (or BF16 storage) and FP64 vectors and dot products (or, as
//           an option, FP32 vectors with FP64-accurate dots);
//           x += |r| d;  r = b - H64 x   until |r| / |b| <= tol and, when a
//           forward tolerance is set, |r| |d| <= fwd_tol |x|.
// The last test is the forward-error criterion: the error of x before a sweep
// is what that sweep's correction estimates, and the error after it is a
// fraction of it (the inner solve's accuracy), so a small correction bounds
// the forward error of the result.
// The Jacobi preconditioner's diagonal comes from the operator (for the mesh
// operator by probing: it is block diagonal per element with the same mode
// numbering in every element of a block, so applying it to the vector that is
// 1 at mode m of every element returns column m of every element matrix, whose
// mode-m entries are diagonal entries).
//
// Scalars (alpha, beta, r.z, r.r) live on the device.  Every reduction writes
// one partial per CTA; the last CTA to finish (atomic ticket, no waiting)
// sums the partials in CTA order, so results are deterministic.  Iterations
// run in chunks replayed from a captured CUDA graph; the host reads the
// scalars once per chunk.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>
#include <vector>

#include "nir_cg.h"
#include "nir_internal.h"
#include "nir_solve.h"
#include "nir_vec.cuh"

#include "nir_cg_kernels.cuh"

struct CGWork {
    long long n = 0;              // unknowns
    long long n_full = 0;         // entries of x (unknowns, then fixed values)
    int grid = 0;                 // CTAs of the vector kernels
    // x64: plain CG's solution copy, or the FP64 inner solver's correction d
    double *x64 = nullptr, *r64 = nullptr, *z64 = nullptr, *p64 = nullptr, *Ap64 = nullptr;
    double *xs64 = nullptr;       // plain CG: x before a polishing sweep (allocated on first use)
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *Ap32 = nullptr, *d32 = nullptr;
    __nv_bfloat16 *pb16 = nullptr, *Apb16 = nullptr;
    double *dinv64 = nullptr;
    float *dinv32 = nullptr;
    double *part = nullptr;       // 2 * grid partials
    unsigned *ticket = nullptr;
    CGScal *scal = nullptr;
    double *dots = nullptr;       // scratch scalars: |r|^2, |b|^2, |d|^2 (or |dx|^2), |x|^2
    int *flag = nullptr;
    bool diag_ready = false;
    double diag_lambda = 0.0;
    // chunk graphs per inner solver: 0 plain FP64; operator FP32 / BF16 with
    // FP32 vectors (1 / 2) or with FP64 vectors (3 / 4)
    static constexpr int kModes = 5;
    cudaGraphExec_t chunk[kModes] = {};
    double chunk_lambda[kModes] = {};
    void *chunk_op[kModes] = {};   // operator launch bindings of the graphs
    CgOperator *chunk_owner[kModes] = {};
    int chunk_len = 25;
    const CgReducer *red = nullptr;   // set for the duration of a sharded solve
};

int CgReducer::sum(double *v, int n) const { return fn(v, n, user) == 0 ? NIR_OK : NIR_ERR_COMM; }

void nir_cg_work_invalidate(CGWork *w)
{
    if (!w) return;
    for (int i = 0; i < CGWork::kModes; ++i) {
        if (w->chunk[i]) cudaGraphExecDestroy(w->chunk[i]);
        if (w->chunk_op[i] && w->chunk_owner[i]) w->chunk_owner[i]->release(w->chunk_op[i]);
        w->chunk[i] = nullptr;
        w->chunk_op[i] = nullptr;
        w->chunk_owner[i] = nullptr;
    }
    w->diag_ready = false;
}

void nir_cg_work_free(CGWork *&w)
{
    if (!w) return;
    nir_cg_work_invalidate(w);
    void *ptrs[] = {w->x64, w->xs64, w->r64, w->z64, w->p64, w->Ap64, w->r32, w->z32, w->p32, w->Ap32, w->d32, w->pb16,
                    w->Apb16, w->dinv64, w->dinv32, w->part, w->ticket, w->scal, w->dots, w->flag};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete w;
    w = nullptr;
}

void nir_cg_invalidate(nir_mesh *m) { nir_cg_work_invalidate(m->cg); }
void nir_cg_free(nir_mesh *m) { nir_cg_work_free(m->cg); }

namespace {

int cg_alloc(CgOperator &op, CGWork *&wout)
{
    if (wout) {
        if (wout->n == op.n() && wout->n_full == op.n_full()) return NIR_OK;
        nir_cg_work_free(wout);
    }
    CGWork *w = new (std::nothrow) CGWork();
    if (!w) return NIR_ERR_NO_MEMORY;
    wout = w;
    const long long n = op.n();
    w->n = n;
    w->n_full = op.n_full();
    w->grid = op.context()->num_sms * 8;   // 8 CTAs of 256 threads fill an SM
    const size_t d = sizeof(double) * n, f = sizeof(float) * n, h = sizeof(__nv_bfloat16) * n;
    bool ok = cudaMalloc(&w->x64, sizeof(double) * w->n_full) == cudaSuccess &&
              cudaMalloc(&w->r64, d) == cudaSuccess && cudaMalloc(&w->z64, d) == cudaSuccess &&
              cudaMalloc(&w->p64, d) == cudaSuccess && cudaMalloc(&w->Ap64, d) == cudaSuccess &&
              cudaMalloc(&w->r32, f) == cudaSuccess && cudaMalloc(&w->z32, f) == cudaSuccess &&
              cudaMalloc(&w->p32, f) == cudaSuccess && cudaMalloc(&w->Ap32, f) == cudaSuccess &&
              cudaMalloc(&w->d32, f) == cudaSuccess && cudaMalloc(&w->pb16, h) == cudaSuccess &&
              cudaMalloc(&w->Apb16, h) == cudaSuccess && cudaMalloc(&w->dinv64, d) == cudaSuccess &&
              cudaMalloc(&w->dinv32, f) == cudaSuccess &&
              cudaMalloc(&w->part, sizeof(double) * 2 * w->grid) == cudaSuccess &&
              cudaMalloc(&w->ticket, sizeof(unsigned) * 4) == cudaSuccess &&
              cudaMalloc(&w->scal, sizeof(CGScal)) == cudaSuccess &&
              cudaMalloc(&w->dots, sizeof(double) * 4) == cudaSuccess && cudaMalloc(&w->flag, sizeof(int)) == cudaSuccess;
    if (!ok) {
        nir_cg_work_free(wout);
        return NIR_ERR_NO_MEMORY;
    }
    cudaMemset(w->ticket, 0, sizeof(unsigned) * 4);
    return NIR_OK;
}

int vgrid(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

// Jacobi diagonal from the operator, inverted in FP64 and FP32.
int cg_diagonal(CgOperator &op, CGWork *w, double lambda, cudaStream_t st)
{
    if (w->diag_ready && w->diag_lambda == lambda) return NIR_OK;
    const long long n = w->n;
    int rc = op.diagonal(lambda, w->dinv64, st);
    if (rc) return rc;
    int bad = 0;
    cudaMemsetAsync(w->flag, 0, sizeof(int), st);
    k_invert<<<vgrid(n), 256, 0, st>>>(w->dinv64, w->dinv32, n, w->flag);
    if (cudaMemcpyAsync(&bad, w->flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NIR_ERR_CUDA;
    if (w->red) {  // every rank takes the same branch
        double v = bad ? 1.0 : 0.0;
        rc = w->red->sum(&v, 1);
        if (rc) return rc;
        bad = v > 0.0;
    }
    if (bad) return NIR_ERR_NONFINITE;  // a non-positive diagonal: the operator is not SPD
    w->diag_ready = true;
    w->diag_lambda = lambda;
    return NIR_OK;
}

// Capture `len` CG iterations for the given inner precision into a graph.
template <class V, class T>
int capture_chunk(CgOperator &op, CGWork *w, int mode, int prec, double lambda, V *x, V *r, V *z, V *p, T *pT,
                  T *Ap, const V *dinv)
{
    if (w->chunk[mode] && w->chunk_lambda[mode] == lambda && w->chunk_owner[mode] == &op) return NIR_OK;
    if (w->chunk[mode]) { cudaGraphExecDestroy(w->chunk[mode]); w->chunk[mode] = nullptr; }
    if (w->chunk_op[mode] && w->chunk_owner[mode]) w->chunk_owner[mode]->release(w->chunk_op[mode]);
    w->chunk_op[mode] = nullptr;
    w->chunk_owner[mode] = nullptr;
    const void *apply_in = pT ? (const void *)pT : (const void *)p;
    int rc = op.prepare(prec, lambda, apply_in, Ap, &w->chunk_op[mode]);
    if (rc) return rc;
    w->chunk_owner[mode] = &op;
    cudaStream_t cs = op.capture_stream();
    cudaGraph_t g;
    NIR_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const long long n = w->n;
    for (int it = 0; it < w->chunk_len && !rc; ++it) {
        rc = op.launch(w->chunk_op[mode], cs);
        k_alpha<V, T><<<w->grid, kThreads, 0, cs>>>(p, Ap, n, w->part, w->ticket, w->scal);
        k_update<V, T><<<w->grid, kThreads, 0, cs>>>(x, r, z, p, Ap, dinv, n, w->part, w->ticket + 1, w->scal);
        k_pupdate<V, T><<<w->grid, kThreads, 0, cs>>>(p, dinv ? z : r, (pT == (T *)p) ? nullptr : pT, n, w->scal);
    }
    cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (rc) return rc;
    if (ec != cudaSuccess) return NIR_ERR_CUDA;
    ec = cudaGraphInstantiate(&w->chunk[mode], g, 0);
    cudaGraphDestroy(g);
    if (ec != cudaSuccess) return NIR_ERR_CUDA;
    w->chunk_lambda[mode] = lambda;
    return NIR_OK;
}

// FP64 true residual r64 = b - H x; returns |r|^2 and |b|^2 on the host.
// With `extra`, also returns dots[2] and dots[3], which the caller queued on
// the same stream before this call.
int residual64(CgOperator &op, CGWork *w, double lambda, const double *b, const double *x, double *rr, double *bb,
               cudaStream_t st, double *extra = nullptr)
{
    const long long n = w->n;
    int rc = op.apply64(lambda, x, w->Ap64, st);
    if (rc) return rc;
    k_residual<<<vgrid(n), 256, 0, st>>>(w->r64, b, w->Ap64, n);
    k_dot<double><<<w->grid, kThreads, 0, st>>>(w->r64, w->r64, n, w->part, w->ticket + 2, w->dots);
    if (bb) k_dot<double><<<w->grid, kThreads, 0, st>>>(b, b, n, w->part, w->ticket + 2, w->dots + 1);
    double h[4] = {0, 0, 0, 0};
    const int nd = extra ? 4 : 2;
    NIR_CUDA_TRY(cudaMemcpyAsync(h, w->dots, sizeof(double) * nd, cudaMemcpyDeviceToHost, st));
    NIR_CUDA_TRY(cudaStreamSynchronize(st));
    if (w->red) {  // sharded: sum this rank's partial dot products over the ranks
        rc = w->red->sum(h, nd);
        if (rc) return rc;
    }
    *rr = h[0];
    if (bb) *bb = h[1];
    if (extra) {
        extra[0] = h[2];
        extra[1] = h[3];
    }
    return NIR_OK;
}

// PCG of a solve sharded across ranks: the same kernels with deferred
// scalars.  Each reduction kernel leaves this rank's partial sum in the
// scalar block; the host reads it, sums it over the ranks (the caller's
// reduction), and writes alpha / beta back for the next kernel.  Two host
// round trips per iteration; every rank runs the same iterations because it
// decides on the same reduced scalars.
template <class V, class T>
int run_pcg_dist(CgOperator &op, CGWork *w, int prec, double lambda, V *x, V *r, V *z, V *p, T *pT, T *Ap,
                 const V *dinv, double thresh, int max_iter, int *iters, double *rr_out, int *bad_out, cudaStream_t st)
{
    const long long n = w->n;
    T *pTk = (pT == (T *)p) ? nullptr : pT;
    void *h = nullptr;
    int rc = op.prepare(prec, lambda, pT ? (const void *)pT : (const void *)p, Ap, &h);
    if (rc) return rc;
    CGScal hs;
    auto fetch = [&]() -> int {
        if (cudaMemcpyAsync(&hs, w->scal, sizeof(CGScal), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return NIR_ERR_CUDA;
        return NIR_OK;
    };
    auto put = [&](double *dst, double v) -> int {  // pageable source: copied before the call returns
        return cudaMemcpyAsync(dst, &v, sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess ? NIR_OK
                                                                                                    : NIR_ERR_CUDA;
    };
    k_start<V, T><<<w->grid, kThreads, 0, st>>>(r, z, p, pTk, dinv, n, w->part, w->ticket + 3, w->scal, thresh, 1);
    double v[2] = {0.0, 0.0};
    int it = 0, bad = 0;
    rc = fetch();
    if (!rc) {
        v[0] = hs.rz;
        v[1] = hs.rr;
        rc = w->red->sum(v, 2);
    }
    double rz = v[0], rr = v[1];
    if (!rc && (!std::isfinite(rz) || !std::isfinite(rr))) bad = 2;
    while (!rc && !bad && rr > thresh && it < max_iter) {
        rc = op.launch(h, st);
        if (rc) break;
        k_alpha<V, T><<<w->grid, kThreads, 0, st>>>(p, Ap, n, w->part, w->ticket, w->scal);
        if ((rc = fetch())) break;
        v[0] = hs.pAp;
        if ((rc = w->red->sum(v, 1))) break;
        const double pAp = v[0];
        if (!std::isfinite(pAp)) { bad = 2; break; }
        if (!(pAp > 0.0)) { bad = 1; break; }
        if ((rc = put(&w->scal->alpha, rz / pAp))) break;
        k_update<V, T><<<w->grid, kThreads, 0, st>>>(x, r, z, p, Ap, dinv, n, w->part, w->ticket + 1, w->scal);
        if ((rc = fetch())) break;
        v[0] = hs.rzn;
        v[1] = hs.rr;
        if ((rc = w->red->sum(v, 2))) break;
        ++it;
        if (!std::isfinite(v[0]) || !std::isfinite(v[1])) { bad = 2; break; }
        const double beta = v[0] / rz;
        rz = v[0];
        rr = v[1];
        if (rr <= thresh) break;
        if ((rc = put(&w->scal->beta, beta))) break;
        k_pupdate<V, T><<<w->grid, kThreads, 0, st>>>(p, dinv ? z : r, pTk, n, w->scal);
    }
    op.release(h);
    *iters = it;
    *rr_out = rr;
    *bad_out = bad;
    return rc;
}

// Run PCG chunks until done or max_iter; returns iterations and final rr.
template <class V, class T>
int run_pcg(CgOperator &op, CGWork *w, int mode, int prec, double lambda, V *x, V *r, V *z, V *p, T *pT, T *Ap,
            const V *dinv, double thresh, int max_iter, int *iters, double *rr_out, int *bad_out, cudaStream_t st)
{
    if (w->red) return run_pcg_dist<V, T>(op, w, prec, lambda, x, r, z, p, pT, Ap, dinv, thresh, max_iter, iters,
                                          rr_out, bad_out, st);
    const long long n = w->n;
    k_start<V, T><<<w->grid, kThreads, 0, st>>>(r, z, p, (pT == (T *)p) ? nullptr : pT, dinv, n, w->part,
                                                w->ticket + 3, w->scal, thresh, 0);
    int rc = capture_chunk<V, T>(op, w, mode, prec, lambda, x, r, z, p, pT, Ap, dinv);
    if (rc) return rc;
    CGScal hs;
    NIR_CUDA_TRY(cudaMemcpyAsync(&hs, w->scal, sizeof(CGScal), cudaMemcpyDeviceToHost, st));
    NIR_CUDA_TRY(cudaStreamSynchronize(st));
    while (!hs.done && hs.iters < max_iter) {
        NIR_CUDA_TRY(cudaGraphLaunch(w->chunk[mode], st));
        NIR_CUDA_TRY(cudaMemcpyAsync(&hs, w->scal, sizeof(CGScal), cudaMemcpyDeviceToHost, st));
        NIR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    *iters = hs.iters;
    *rr_out = hs.rr;
    *bad_out = hs.bad;
    return NIR_OK;
}

// The mesh's broken Helmholtz operator: one persistent launch per apply, or
// for a mesh of one block that block's own kernel.
struct MeshLaunch {
    int prec;
    nirk::MeshBlk *blk;   // device block table (persistent launch), or null
    double lambda;
    const void *x;
    void *y;
};

struct MeshOp final : CgOperator {
    nir_mesh *m;
    explicit MeshOp(nir_mesh *mm) : m(mm) {}
    nir_ctx *context() override { return m->ctx; }
    long long n() override { return m->ndof; }
    long long n_full() override { return m->ndof; }
    cudaStream_t capture_stream() override { return m->cap_stream; }
    int prepare(int prec, double lambda, const void *x, void *y, void **handle) override
    {
        nirk::MeshBlk *blk = nullptr;
        if (m->blocks.size() == 1 || m->ps[prec].mode == 1) {
            // one uncaptured launch sets up what is created lazily (factors, attributes)
            int rc = nir_mesh_apply(m, prec, lambda, x, y, m->ctx->stream);
            if (rc) return rc;
        } else {
            int rc = nir_mesh_block_table(m, prec, lambda, x, y, &blk);
            if (rc) return rc;
        }
        MeshLaunch *h = new (std::nothrow) MeshLaunch{prec, blk, lambda, x, y};
        if (!h) {
            cudaFree(blk);
            return NIR_ERR_NO_MEMORY;
        }
        *handle = h;
        return NIR_OK;
    }
    int launch(void *handle, cudaStream_t st) override
    {
        MeshLaunch *h = static_cast<MeshLaunch *>(handle);
        if (!h->blk) return nir_mesh_launch_blocks(m, h->prec, h->lambda, h->x, h->y, st);
        return nir_mesh_launch_raw(m, h->prec, h->blk, st);
    }
    void release(void *handle) override
    {
        MeshLaunch *h = static_cast<MeshLaunch *>(handle);
        if (!h) return;
        if (h->blk) cudaFree(h->blk);
        delete h;
    }
    int apply64(double lambda, const double *x, double *y, cudaStream_t st) override
    {
        return nir_mesh_apply(m, NIR_F64, lambda, x, y, st);
    }
    // Probing with the FP32 operator (block diagonal per element, same mode
    // numbering in every element of a block).
    int diagonal(double lambda, double *d, cudaStream_t st) override
    {
        std::vector<ProbeBlk> hb(m->blocks.size());
        int Mmax = 0;
        for (size_t i = 0; i < m->blocks.size(); ++i) {
            hb[i].off = m->off[i];
            hb[i].nelem = m->blocks[i]->d.nelem;
            hb[i].M = m->blocks[i]->M;
            hb[i].pad = 0;
            Mmax = std::max(Mmax, hb[i].M);
        }
        const long long n = m->ndof;
        ProbeBlk *db = nullptr;
        float *x32 = nullptr, *y32 = nullptr;
        int rc = NIR_OK;
        if (cudaMalloc(&db, sizeof(ProbeBlk) * hb.size()) != cudaSuccess ||
            cudaMalloc(&x32, sizeof(float) * n) != cudaSuccess || cudaMalloc(&y32, sizeof(float) * n) != cudaSuccess)
            rc = NIR_ERR_NO_MEMORY;
        if (!rc && cudaMemcpyAsync(db, hb.data(), sizeof(ProbeBlk) * hb.size(), cudaMemcpyHostToDevice, st) !=
                       cudaSuccess)
            rc = NIR_ERR_CUDA;
        const int nb = (int)hb.size();
        for (int mm = 0; mm < Mmax && !rc; ++mm) {
            k_probe_fill<float><<<vgrid(n), 256, 0, st>>>(x32, db, nb, mm, n);
            rc = nir_mesh_apply(m, NIR_F32, lambda, x32, y32, st);
            if (!rc) k_probe_gather<float><<<vgrid(n), 256, 0, st>>>(d, y32, db, nb, mm, n);
        }
        if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = NIR_ERR_CUDA;
        if (db) cudaFree(db);
        if (x32) cudaFree(x32);
        if (y32) cudaFree(y32);
        return rc;
    }
};

}  // namespace

namespace {

// Inner solve of one refinement sweep, H_lo d = r64 / rn, in the vector type
// V (double or float) with the operator in `prec`; d is left in x64 (FP64
// vectors) or d32 (FP32 vectors).
template <class V>
int inner_sweep(CgOperator &op, CGWork *w, int prec, double lambda, double rn, const nir_cg_opts *o, int *iters,
                int *bad, cudaStream_t st)
{
    const long long n = w->n;
    constexpr bool v64 = std::is_same<V, double>::value;
    V *d, *r, *z, *p;
    const V *dinv;
    if constexpr (v64) {
        d = w->x64; r = w->r64; z = w->z64; p = w->p64; dinv = w->dinv64;
    } else {
        d = w->d32; r = w->r32; z = w->z32; p = w->p32; dinv = w->dinv32;
    }
    if (!o->jacobi) dinv = nullptr;
    k_scale_to<V><<<vgrid(n), 256, 0, st>>>(r, w->r64, 1.0 / rn, n);
    k_fill<V><<<vgrid(n), 256, 0, st>>>(d, 0.0, n);
    const double th = o->inner_tol * o->inner_tol;
    double rr_in = 0.0;
    const int mode = (prec == NIR_F32 ? 1 : 2) + (v64 ? 2 : 0);
    if (prec == NIR_F32) {
        // FP32 vectors: p itself is the operator's input; FP64 vectors: its FP32 copy
        float *pT = v64 ? w->p32 : reinterpret_cast<float *>(p);
        return run_pcg<V, float>(op, w, mode, NIR_F32, lambda, d, r, z, p, pT, w->Ap32, dinv, th, o->max_inner, iters,
                                 &rr_in, bad, st);
    }
    return run_pcg<V, __nv_bfloat16>(op, w, mode, NIR_BF16, lambda, d, r, z, p, w->pb16, w->Apb16, dinv, th,
                                     o->max_inner, iters, &rr_in, bad, st);
}

}  // namespace

namespace {
int cg_run_impl(CgOperator &op, CGWork *&wref, double lambda, const double *b, double *x, const nir_cg_opts *o,
                nir_cg_stats *stats, const CgReducer *red);
}

int nir_cg_run(CgOperator &op, CGWork *&wref, double lambda, const double *b, double *x, const nir_cg_opts *o,
               nir_cg_stats *stats, const CgReducer *red)
{
    if (red && !red->fn) return NIR_ERR_INVALID_ARG;
    // the reducer lives for this call only (it is cleared on every return path)
    struct Guard {
        CGWork *&w;
        ~Guard() { if (w) w->red = nullptr; }
    } guard{wref};
    if (wref) wref->red = red;
    return cg_run_impl(op, wref, lambda, b, x, o, stats, red);
}

namespace {
int cg_run_impl(CgOperator &op, CGWork *&wref, double lambda, const double *b, double *x, const nir_cg_opts *o,
                nir_cg_stats *stats, const CgReducer *red)
{
    if (!b || !x || !o || (const void *)b == (const void *)x) return NIR_ERR_INVALID_ARG;
    if (!(o->tol > 0.0) || o->max_inner < 1 || !std::isfinite(lambda)) return NIR_ERR_INVALID_ARG;
    if (o->inner_prec != NIR_F64 && o->inner_prec != NIR_F32 && o->inner_prec != NIR_BF16) return NIR_ERR_INVALID_ARG;
    if (o->inner_prec != NIR_F64 && (o->max_outer < 1 || !(o->inner_tol > 0.0) || !(o->inner_tol < 1.0)))
        return NIR_ERR_INVALID_ARG;
    if (o->inner_vectors != NIR_F64 && o->inner_vectors != NIR_F32) return NIR_ERR_INVALID_ARG;
    if (!(o->fwd_tol >= 0.0) || !std::isfinite(o->fwd_tol)) return NIR_ERR_INVALID_ARG;
    if (o->inner_prec == NIR_F64 && o->fwd_tol > 0.0 && !(o->inner_tol >= 0.0 && o->inner_tol < 1.0))
        return NIR_ERR_INVALID_ARG;
    NIR_CUDA_TRY(cudaSetDevice(op.context()->device));
    const auto t0 = std::chrono::steady_clock::now();
    int rc = cg_alloc(op, wref);
    if (rc) return rc;
    CGWork *w = wref;
    w->red = red;
    cudaStream_t st = op.context()->stream;
    const long long n = w->n;
    if (o->jacobi) {
        rc = cg_diagonal(op, w, lambda, st);
        if (rc) return rc;
    }
    double rr = 0.0, bb = 0.0;
    rc = residual64(op, w, lambda, b, x, &rr, &bb, st);
    if (rc) return rc;
    if (!std::isfinite(rr) || !std::isfinite(bb)) return NIR_ERR_NONFINITE;
    nir_cg_stats s{0, 0, 0.0, 0.0, 0.0};
    const double bn = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
    const bool fwd = o->fwd_tol > 0.0;
    double corr = fwd ? HUGE_VAL : 0.0;   // last sweep's |dx| / |x|
    auto met = [&] { return std::sqrt(rr) / bn <= o->tol && (!fwd || corr <= o->fwd_tol); };
    int status = NIR_OK;
    if (o->inner_prec == NIR_F64) {
        // plain preconditioned CG, FP64 throughout, on an internal copy of x (the
        // captured iteration graph holds fixed vector addresses).  The recursive
        // residual drifts from the true one, so CG restarts from b - H x until
        // the true residual meets the tolerance or the iteration cap is hit.
        NIR_CUDA_TRY(cudaMemcpyAsync(w->x64, x, sizeof(double) * w->n_full, cudaMemcpyDeviceToDevice, st));
        for (int restart = 0; restart < 50; ++restart) {
            int iters = 0, bad = 0;
            double rr_it = 0.0;
            rc = run_pcg<double, double>(op, w, 0, NIR_F64, lambda, w->x64, w->r64, w->z64, w->p64, w->p64,
                                         w->Ap64, o->jacobi ? w->dinv64 : nullptr, o->tol * o->tol * bb,
                                         o->max_inner - s.inner_total, &iters, &rr_it, &bad, st);
            if (rc) return rc;
            s.inner_total += iters;
            s.outer += 1;
            const double prev = rr;
            rc = residual64(op, w, lambda, b, w->x64, &rr, nullptr, st);  // also refreshes r64 for a restart
            if (rc) return rc;
            if (bad == 2 || !std::isfinite(rr)) { status = NIR_ERR_NONFINITE; break; }
            if (bad == 1) { status = NIR_ERR_NOT_CONVERGED; break; }
            if (std::sqrt(rr) / bn <= o->tol) break;
            if (s.inner_total >= o->max_inner || rr >= prev) { status = NIR_ERR_NOT_CONVERGED; break; }
        }
        // Polishing for the forward tolerance: CG continues from the true
        // residual, cutting it by inner_tol per sweep, and each sweep's update
        // |x_after - x_before| is the correction that fwd_tol bounds.
        if (!status && fwd) {
            if (!w->xs64 && cudaMalloc(&w->xs64, sizeof(double) * n) != cudaSuccess) return NIR_ERR_NO_MEMORY;
            const double red = o->inner_tol > 0.0 ? o->inner_tol : 1e-3;
            double corr_prev = HUGE_VAL;
            for (int sweep = 0; !met(); ++sweep) {
                if (sweep >= 50 || s.inner_total >= o->max_inner) { status = NIR_ERR_NOT_CONVERGED; break; }
                NIR_CUDA_TRY(cudaMemcpyAsync(w->xs64, w->x64, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
                int iters = 0, bad = 0;
                double rr_it = 0.0;
                rc = run_pcg<double, double>(op, w, 0, NIR_F64, lambda, w->x64, w->r64, w->z64, w->p64, w->p64,
                                             w->Ap64, o->jacobi ? w->dinv64 : nullptr, red * red * rr,
                                             o->max_inner - s.inner_total, &iters, &rr_it, &bad, st);
                if (rc) return rc;
                s.inner_total += iters;
                s.outer += 1;
                k_diff_norms<<<w->grid, kThreads, 0, st>>>(w->x64, w->xs64, n, w->part, w->ticket + 2, w->dots + 2);
                const double prev = rr;
                double e[2] = {0, 0};
                rc = residual64(op, w, lambda, b, w->x64, &rr, nullptr, st, e);
                if (rc) return rc;
                if (bad == 2 || !std::isfinite(rr) || !std::isfinite(e[0])) { status = NIR_ERR_NONFINITE; break; }
                corr = e[1] > 0.0 ? std::sqrt(e[0] / e[1]) : 0.0;
                if (bad == 1) { status = NIR_ERR_NOT_CONVERGED; break; }
                if (!met() && rr >= prev && corr >= corr_prev) { status = NIR_ERR_NOT_CONVERGED; break; }
                corr_prev = corr;
            }
        }
        NIR_CUDA_TRY(cudaMemcpyAsync(x, w->x64, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    } else {
        const bool v64 = o->inner_vectors == NIR_F64;
        double corr_prev = HUGE_VAL;
        while (!met() && s.outer < o->max_outer) {
            const double rn = std::sqrt(rr);
            int iters = 0, bad = 0;
            rc = v64 ? inner_sweep<double>(op, w, o->inner_prec, lambda, rn, o, &iters, &bad, st)
                     : inner_sweep<float>(op, w, o->inner_prec, lambda, rn, o, &iters, &bad, st);
            if (rc) return rc;
            s.inner_total += iters;
            s.outer += 1;
            if (bad == 2) { status = NIR_ERR_NONFINITE; break; }
            if (v64) {
                k_correct<double><<<vgrid(n), 256, 0, st>>>(x, w->x64, rn, n);
                k_dot<double><<<w->grid, kThreads, 0, st>>>(w->x64, w->x64, n, w->part, w->ticket + 2, w->dots + 2);
            } else {
                k_correct<float><<<vgrid(n), 256, 0, st>>>(x, w->d32, rn, n);
                k_dot<float><<<w->grid, kThreads, 0, st>>>(w->d32, w->d32, n, w->part, w->ticket + 2, w->dots + 2);
            }
            k_dot<double><<<w->grid, kThreads, 0, st>>>(x, x, n, w->part, w->ticket + 2, w->dots + 3);
            const double prev = rr;
            double e[2] = {0, 0};
            rc = residual64(op, w, lambda, b, x, &rr, nullptr, st, e);
            if (rc) return rc;
            if (!std::isfinite(rr) || !std::isfinite(e[0])) { status = NIR_ERR_NONFINITE; break; }
            corr = e[1] > 0.0 ? rn * std::sqrt(e[0] / e[1]) : 0.0;
            // refinement stalled: neither the residual nor the correction shrinks
            if (!met() && rr >= prev && corr >= corr_prev) { status = NIR_ERR_NOT_CONVERGED; break; }
            corr_prev = corr;
        }
        if (!status && !met()) status = NIR_ERR_NOT_CONVERGED;
    }
    NIR_CUDA_TRY(cudaStreamSynchronize(st));
    s.rel_residual = std::sqrt(rr) / bn;
    s.rel_correction = std::isfinite(corr) ? corr : 0.0;
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = s;
    return status;
}
}  // namespace

extern "C" int nir_cg_solve(nir_mesh *m, double lambda, const double *b, double *x, const nir_cg_opts *o,
                            nir_cg_stats *stats)
{
    if (!m) return NIR_ERR_INVALID_ARG;
    if (!std::isfinite(lambda) || !(lambda > 0.0)) return NIR_ERR_INVALID_ARG;
    if (!m->cg_op) {
        m->cg_op = new (std::nothrow) MeshOp(m);
        if (!m->cg_op) return NIR_ERR_NO_MEMORY;
    }
    int rc = nir_mesh_sync_geometry(m);  // before the preconditioner and graphs are reused
    if (rc) return rc;
    return nir_cg_run(*m->cg_op, m->cg, lambda, b, x, o, stats, nullptr);
}

extern "C" int nir_cg_solve_dist(nir_mesh *m, double lambda, const double *b, double *x, const nir_cg_opts *o,
                                 nir_cg_stats *stats, nir_allreduce_fn allreduce, void *user)
{
    if (!m || !allreduce) return NIR_ERR_INVALID_ARG;
    if (!std::isfinite(lambda) || !(lambda > 0.0)) return NIR_ERR_INVALID_ARG;
    if (!m->cg_op) {
        m->cg_op = new (std::nothrow) MeshOp(m);
        if (!m->cg_op) return NIR_ERR_NO_MEMORY;
    }
    int rc = nir_mesh_sync_geometry(m);
    if (rc) return rc;
    const CgReducer red{allreduce, user};
    return nir_cg_run(*m->cg_op, m->cg, lambda, b, x, o, stats, &red);
}
