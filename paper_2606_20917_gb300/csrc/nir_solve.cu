// nir_solve.cu -- hybrid meshes: the persistent single-launch Helmholtz apply
// over blocks of different shapes and orders, its CUDA-graph cache and the
// autotuner (elements-per-CTA variants, the threading strategy and grid
// sizes, JSON cache file).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "nir_cg.h"
#include "nir_internal.h"
#include "nir_mesh.h"
#include "nir_solve.h"

#define NIR_MDECL(d, p)                                        \
    MeshKInfo nir_mesh_kinfo_d##d##_p##p(int shape, int P);    \
    int nir_mesh_tables_d##d##_p##p(int vid, const float *blob, int n, cudaStream_t st);
NIR_MDECL(2, 0) NIR_MDECL(2, 1) NIR_MDECL(2, 2)
NIR_MDECL(3, 0) NIR_MDECL(3, 1) NIR_MDECL(3, 2)
#undef NIR_MDECL

MeshKInfo nir_mesh_kinfo(int dim, int prec, int shape, int P)
{
    typedef MeshKInfo (*F)(int, int);
    static const F tab[2][3] = {{nir_mesh_kinfo_d2_p0, nir_mesh_kinfo_d2_p1, nir_mesh_kinfo_d2_p2},
                                {nir_mesh_kinfo_d3_p0, nir_mesh_kinfo_d3_p1, nir_mesh_kinfo_d3_p2}};
    if ((dim != 2 && dim != 3) || prec < 0 || prec > 2) return MeshKInfo{};
    return tab[dim - 2][prec](shape, P);
}

// Load a variant's FP32 tables into the mesh kernel's constant tables.
int nir_mesh_tables(int dim, int prec, int vid, const float *blob, int n, cudaStream_t st)
{
    typedef int (*F)(int, const float *, int, cudaStream_t);
    static const F tab[2][3] = {{nir_mesh_tables_d2_p0, nir_mesh_tables_d2_p1, nir_mesh_tables_d2_p2},
                                {nir_mesh_tables_d3_p0, nir_mesh_tables_d3_p1, nir_mesh_tables_d3_p2}};
    if ((dim != 2 && dim != 3) || prec < 0 || prec > 2) return NIR_ERR_INVALID_ARG;
    return tab[dim - 2][prec](vid, blob, n, st);
}

namespace {

// Relative cost of one element's Helmholtz apply (sum-factorised flop count),
// used to order the work list longest first.
double elem_cost(int shape, int P)
{
    const double N = P + 1, Q = P + 2;
    if (shape == NIR_QUAD || shape == NIR_TRI) return 4 * N * (N * Q + Q * Q) + 8 * Q * Q * Q + 10 * Q * Q;
    return 4 * N * (N * N * Q + N * Q * Q + Q * Q * Q) + 12 * Q * Q * Q * Q + 20 * Q * Q * Q;
}

bool valid_prec(int p) { return p == NIR_F64 || p == NIR_F32 || p == NIR_BF16; }

}  // namespace

int nir_mesh_build_items(nir_mesh *m, int prec, int gran)
{
    MeshPrec &ps = m->ps[prec];
    std::vector<std::pair<double, nirk::MeshItem>> items;
    ps.smem = 0;
    ps.fn = nullptr;
    for (size_t bi = 0; bi < m->blocks.size(); ++bi) {
        nir_block *b = m->blocks[bi];
        MeshKInfo k = nir_mesh_kinfo(m->dim, prec, b->d.shape, b->d.P);
        if (!k.fn) return NIR_ERR_UNSUPPORTED;
        ps.fn = k.fn;
        ps.nt = k.nt;
        ps.smem = std::max(ps.smem, k.smem);
        ps.vid[bi] = k.vid;
        if (prec != NIR_F64 && b->d.basis == NIR_BASIS_MODIFIED) {  // constant tables of the FP32/BF16 kernel
            // (the modified basis' tables depend on (shape, P) only: shared by the variant's blocks)
            int rc = nir_mesh_tables(m->dim, prec, k.vid, b->tab32_h.data(), (int)b->tab32_h.size(), m->ctx->stream);
            if (rc) return rc;
        }
        const long long ngroups = (b->d.nelem + k.epb - 1) / k.epb;
        for (long long g = 0; g < ngroups; g += gran) {
            nirk::MeshItem it;
            it.block = (int)bi;
            it.g0 = (int)g;
            it.ng = (int)std::min<long long>(gran, ngroups - g);
            it.pad = 0;
            const long long nel = std::min<long long>((long long)it.ng * k.epb, b->d.nelem - g * k.epb);
            items.push_back({nel * elem_cost(b->d.shape, b->d.P), it});
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, nirk::MeshItem> &a, const std::pair<double, nirk::MeshItem> &b) {
                         return a.first > b.first;
                     });
    std::vector<nirk::MeshItem> h(items.size());
    for (size_t i = 0; i < items.size(); ++i) h[i] = items[i].second;
    if (ps.ditems) cudaFree(ps.ditems);
    ps.ditems = nullptr;
    NIR_CUDA_TRY(cudaMalloc(&ps.ditems, sizeof(nirk::MeshItem) * std::max<size_t>(1, h.size())));
    NIR_CUDA_TRY(cudaMemcpy(ps.ditems, h.data(), sizeof(nirk::MeshItem) * h.size(), cudaMemcpyHostToDevice));
    ps.nitems = (int)h.size();
    ps.gran = gran;
    if (ps.smem > 48 * 1024)
        NIR_CUDA_TRY(cudaFuncSetAttribute(ps.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ps.smem));
    int occ = 0;
    NIR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ps.fn, ps.nt, ps.smem));
    ps.occ = std::max(1, occ);
    if (ps.grid <= 0 || ps.grid > ps.occ * m->ctx->num_sms) ps.grid = ps.occ * m->ctx->num_sms;
    ps.ready = true;
    // captured graphs embed the old work list
    for (auto &g : m->graphs)
        if (g.prec == prec) g.stale = true;
    nir_cg_invalidate(m);
    return NIR_OK;
}

// Launch the persistent kernel for (prec, in, out, lambda) on `st` using a
// device block table `dblk` (already uploaded).
int nir_mesh_launch_raw(nir_mesh *m, int prec, const nirk::MeshBlk *dblk, cudaStream_t st)
{
    MeshPrec &ps = m->ps[prec];
    if (!ps.ready || !ps.fn) return NIR_ERR_STATE;
    NIR_CUDA_TRY(cudaMemsetAsync(m->counter + prec, 0, sizeof(int), st));
    int *ctr = m->counter + prec;
    int nitems = ps.nitems;
    const nirk::MeshItem *items = ps.ditems;
    void *args[] = {(void *)&dblk, (void *)&items, (void *)&nitems, (void *)&ctr};
    if (cudaLaunchKernel(ps.fn, dim3(ps.grid), dim3(ps.nt), args, (size_t)ps.smem, st) != cudaSuccess) {
        (void)cudaGetLastError();  // consume the launch error so it does not surface in a later call
        return NIR_ERR_CUDA;
    }
    return NIR_OK;
}

int nir_mesh_sync_geometry(nir_mesh *m)
{
    // a block whose geometry was set again has new factor arrays: every
    // captured graph and block table of the mesh is out of date
    bool changed = m->geo_seen.size() != m->blocks.size();
    for (size_t i = 0; !changed && i < m->blocks.size(); ++i) changed = m->geo_seen[i] != m->blocks[i]->geo_version;
    if (changed) {
        for (auto &g : m->graphs) g.stale = true;
        nir_cg_invalidate(m);
        m->geo_seen.resize(m->blocks.size());
        for (size_t i = 0; i < m->blocks.size(); ++i) m->geo_seen[i] = m->blocks[i]->geo_version;
        for (size_t i = 0; i < m->blocks.size(); ++i)
            if (!m->blocks[i]->geo_set) return NIR_ERR_STATE;
    }
    return NIR_OK;
}

int nir_mesh_prepare(nir_mesh *m, int prec)
{
    int rc = nir_mesh_sync_geometry(m);
    if (rc) return rc;
    if (m->ps[prec].ready) return NIR_OK;
    return nir_mesh_build_items(m, prec, m->ps[prec].gran > 0 ? m->ps[prec].gran : 1);
}

int nir_mesh_block_table(nir_mesh *m, int prec, double lambda, const void *in, void *out, nirk::MeshBlk **dout)
{
    int rc0 = nir_mesh_prepare(m, prec);
    if (rc0) return rc0;
    const size_t es = nir_prec_size(prec);
    std::vector<nirk::MeshBlk> h(m->blocks.size());
    for (size_t bi = 0; bi < m->blocks.size(); ++bi) {
        nir_block *b = m->blocks[bi];
        int rc = nir_block_ensure_prec(b, prec);
        if (rc) return rc;
        nirk::KArgs &a = h[bi].a;
        std::memset(&a, 0, sizeof(a));
        a.nfields = 1;
        a.nodal = b->d.basis == NIR_BASIS_GLL_LAGRANGE;
        a.in0 = (const char *)in + (size_t)m->off[bi] * es;
        a.out0 = (char *)out + (size_t)m->off[bi] * es;
        a.geo = nir_geo_ptr(b, prec, false);
        a.tab = nir_tab_ptr(b, prec);
        a.nelem = b->d.nelem;
        a.lambda = lambda;
        a.geo_pp = b->geo_pp;
        a.err = m->ctx->derr;
        h[bi].vid = m->ps[prec].vid[bi];
    }
    nirk::MeshBlk *d = nullptr;
    NIR_CUDA_TRY(cudaMalloc(&d, sizeof(nirk::MeshBlk) * h.size()));
    if (cudaMemcpy(d, h.data(), sizeof(nirk::MeshBlk) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return NIR_ERR_CUDA;
    }
    *dout = d;
    return NIR_OK;
}

int nir_mesh_blocks_ready(nir_mesh *m, int prec)
{
    for (nir_block *b : m->blocks) {
        int rc = nir_block_ensure_prec(b, prec);
        if (rc) return rc;
        const int v = b->helm_variant[prec];
        KInfo ki = nir_kinfo(b->d.shape, b->d.P, prec, nirk::OP_HELM, v);
        if (!ki.fn) ki = nir_kinfo(b->d.shape, b->d.P, prec, nirk::OP_HELM, 0);
        if (!ki.fn) return NIR_ERR_UNSUPPORTED;
        if (nir_occupancy(m->ctx, ki) < 0) return NIR_ERR_CUDA;  // sets the kernel's shared-memory attribute
    }
    return NIR_OK;
}

// The blocks' kernels run on kSide concurrent branches (forked from and
// joined back into `st` by events, so a graph captured from `st` holds
// parallel branches): a block too small to fill the GPU overlaps the others.
// Blocks go to branches largest first, each to the least-loaded branch.
int nir_mesh_launch_blocks(nir_mesh *m, int prec, double lambda, const void *in, void *out, cudaStream_t st)
{
    const size_t es = nir_prec_size(prec);
    const int nb = (int)m->blocks.size();
    if (m->side_of.size() != (size_t)nb) {
        std::vector<std::pair<double, int>> cost;
        for (int bi = 0; bi < nb; ++bi)
            cost.push_back({(double)m->blocks[bi]->d.nelem * elem_cost(m->blocks[bi]->d.shape, m->blocks[bi]->d.P), bi});
        std::stable_sort(cost.begin(), cost.end(),
                         [](const std::pair<double, int> &a, const std::pair<double, int> &b) { return a.first > b.first; });
        double load[nir_mesh::kSide] = {};
        m->side_of.assign(nb, 0);
        for (auto &c : cost) {
            int k = 0;
            for (int j = 1; j < nir_mesh::kSide; ++j)
                if (load[j] < load[k]) k = j;
            m->side_of[c.second] = k;
            load[k] += c.first;
        }
    }
    NIR_CUDA_TRY(cudaEventRecord(m->ev_fork, st));
    for (int k = 0; k < nir_mesh::kSide; ++k) NIR_CUDA_TRY(cudaStreamWaitEvent(m->side[k], m->ev_fork, 0));
    int rc = NIR_OK;
    for (int bi = 0; bi < nb && !rc; ++bi) {
        const char *xb = static_cast<const char *>(in) + (size_t)m->off[bi] * es;
        char *yb = static_cast<char *>(out) + (size_t)m->off[bi] * es;
        rc = nir_launch_op(m->blocks[bi], prec, nirk::OP_HELM, lambda, xb, nullptr, nullptr, yb, nullptr, nullptr,
                           m->side[m->side_of[bi]], 0);
    }
    // join every branch back, also after a failed launch (a capture must end joined)
    for (int k = 0; k < nir_mesh::kSide; ++k) {
        if (cudaEventRecord(m->ev_join[k], m->side[k]) != cudaSuccess ||
            cudaStreamWaitEvent(st, m->ev_join[k], 0) != cudaSuccess)
            rc = rc ? rc : NIR_ERR_CUDA;
    }
    return rc;
}

// Apply through a cached CUDA graph (captured on first use per key).
int nir_mesh_apply(nir_mesh *m, int prec, double lambda, const void *in, void *out, cudaStream_t st)
{
    if (m->blocks.size() == 1) {  // one block: its own tuned kernel (a work queue has nothing to balance)
        int rc = nir_mesh_sync_geometry(m);
        if (rc) return rc;
        return nir_launch_op(m->blocks[0], prec, nirk::OP_HELM, lambda, in, nullptr, nullptr, out, nullptr, nullptr,
                             st, 0);
    }
    {
        int rc = nir_mesh_prepare(m, prec);
        if (rc) return rc;
    }
    MeshGraph *hit = nullptr;
    for (auto &g : m->graphs)
        if (g.prec == prec && g.in == in && g.out == out && g.lambda == lambda) hit = &g;
    if (hit && hit->stale) {
        cudaGraphExecDestroy(hit->exec);
        cudaFree(hit->dblk);
        *hit = m->graphs.back();
        m->graphs.pop_back();
        hit = nullptr;
    }
    if (!hit) {
        if (m->graphs.size() >= 32) {  // bounded cache: drop the oldest entry
            cudaGraphExecDestroy(m->graphs.front().exec);
            cudaFree(m->graphs.front().dblk);
            m->graphs.erase(m->graphs.begin());
        }
        MeshGraph g;
        g.prec = prec;
        g.in = in;
        g.out = out;
        g.lambda = lambda;
        const bool blocks = m->ps[prec].mode == 1;
        int rc = blocks ? nir_mesh_blocks_ready(m, prec) : nir_mesh_block_table(m, prec, lambda, in, out, &g.dblk);
        if (rc) return rc;
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaFree(g.dblk);
            return NIR_ERR_CUDA;
        }
        rc = blocks ? nir_mesh_launch_blocks(m, prec, lambda, in, out, m->cap_stream)
                    : nir_mesh_launch_raw(m, prec, g.dblk, m->cap_stream);
        cudaError_t ec = cudaStreamEndCapture(m->cap_stream, &graph);
        if (rc || ec != cudaSuccess) {
            cudaFree(g.dblk);
            return rc ? rc : NIR_ERR_CUDA;
        }
        ec = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ec != cudaSuccess) {
            cudaFree(g.dblk);
            return NIR_ERR_CUDA;
        }
        m->graphs.push_back(g);
        hit = &m->graphs.back();
    }
    NIR_CUDA_TRY(cudaGraphLaunch(hit->exec, st));
    return NIR_OK;
}

// --------------------------------------------------------------------------- C ABI
extern "C" int nir_mesh_create(nir_ctx *ctx, nir_block *const *blocks, int nblocks, nir_mesh **out)
{
    if (!out) return NIR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctx || !blocks || nblocks < 1) return NIR_ERR_INVALID_ARG;
    const int dim = blocks[0] ? blocks[0]->dim : 0;
    for (int i = 0; i < nblocks; ++i) {
        if (!blocks[i] || blocks[i]->ctx != ctx || blocks[i]->dim != dim) return NIR_ERR_INVALID_ARG;
        if (!blocks[i]->geo_set) return NIR_ERR_STATE;
        for (int j = 0; j < i; ++j)
            if (blocks[j] == blocks[i]) return NIR_ERR_INVALID_ARG;
    }
    NIR_CUDA_TRY(cudaSetDevice(ctx->device));
    nir_mesh *m = new (std::nothrow) nir_mesh();
    if (!m) return NIR_ERR_NO_MEMORY;
    m->ctx = ctx;
    m->dim = dim;
    long long o = 0;
    for (int i = 0; i < nblocks; ++i) {
        m->blocks.push_back(blocks[i]);
        m->off.push_back(o);
        o += blocks[i]->d.nelem * blocks[i]->M;
    }
    m->ndof = o;
    for (int p = 0; p < 3; ++p) m->ps[p].vid.assign(nblocks, -1);
    bool ok = cudaMalloc(&m->counter, sizeof(int) * 4) == cudaSuccess &&
              cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < nir_mesh::kSide && ok; ++k)
        ok = cudaStreamCreateWithFlags(&m->side[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&m->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        nir_mesh_destroy(m);
        return NIR_ERR_CUDA;
    }
    *out = m;
    return NIR_OK;
}

extern "C" void nir_mesh_destroy(nir_mesh *m)
{
    if (!m) return;
    for (auto &g : m->graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaFree(g.dblk);
    }
    for (int p = 0; p < 3; ++p)
        if (m->ps[p].ditems) cudaFree(m->ps[p].ditems);
    if (m->counter) cudaFree(m->counter);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    for (int k = 0; k < nir_mesh::kSide; ++k) {
        if (m->side[k]) cudaStreamDestroy(m->side[k]);
        if (m->ev_join[k]) cudaEventDestroy(m->ev_join[k]);
    }
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    nir_cg_free(m);
    delete m->cg_op;
    delete m;
}

extern "C" int nir_mesh_num_dofs(const nir_mesh *m, int64_t *ndof)
{
    if (!m || !ndof) return NIR_ERR_INVALID_ARG;
    *ndof = m->ndof;
    return NIR_OK;
}

extern "C" int nir_mesh_helmholtz(nir_mesh *m, int prec, double lambda, const void *in, void *out)
{
    if (!m || !valid_prec(prec) || !in || !out || in == out || !std::isfinite(lambda)) return NIR_ERR_INVALID_ARG;
    NIR_CUDA_TRY(cudaSetDevice(m->ctx->device));
    return nir_debug_after(m->ctx, nir_mesh_apply(m, prec, lambda, in, out, m->ctx->stream));
}

// --------------------------------------------------------------------------- autotuner
namespace {

std::string gpu_name(int dev)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    std::string s = p.name;
    for (auto &c : s)
        if (c == '"' || c == '|') c = '_';
    return s;
}

std::map<std::string, std::string> read_cache(const char *path)
{
    std::map<std::string, std::string> kv;
    if (!path) return kv;
    std::ifstream f(path);
    if (!f) return kv;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    // flat JSON object of string keys to string values
    size_t i = 0;
    while (true) {
        size_t k0 = s.find('"', i);
        if (k0 == std::string::npos) break;
        size_t k1 = s.find('"', k0 + 1);
        size_t v0 = s.find('"', k1 + 1);
        size_t v1 = v0 == std::string::npos ? v0 : s.find('"', v0 + 1);
        if (k1 == std::string::npos || v1 == std::string::npos) break;
        kv[s.substr(k0 + 1, k1 - k0 - 1)] = s.substr(v0 + 1, v1 - v0 - 1);
        i = v1 + 1;
    }
    return kv;
}

bool write_cache(const char *path, const std::map<std::string, std::string> &kv)
{
    if (!path) return true;
    std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return false;
        f << "{\n";
        size_t n = 0;
        for (auto &e : kv) f << "  \"" << e.first << "\": \"" << e.second << "\"" << (++n < kv.size() ? ",\n" : "\n");
        f << "}\n";
    }
    return std::rename(tmp.c_str(), path) == 0;
}

// Median time (ms) of `reps` launches of f on stream st.
template <class F>
float time_ms(cudaStream_t st, int reps, F f)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<float> t;
    f();
    f();
    // each sample times k back-to-back launches (about 0.5 ms of work), so
    // short kernels are measured in a busy steady state, not one at a time
    float one = 0;
    cudaEventRecord(a, st);
    f();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&one, a, b);
    const int k = one > 0.5f ? 1 : std::min(64, (int)(0.5f / std::max(one, 1e-3f)) + 1);
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, st);
        for (int i = 0; i < k; ++i) f();
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms / k);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

extern "C" int nir_tune(nir_mesh *m, const char *cache_path)
{
    if (!m) return NIR_ERR_INVALID_ARG;
    nir_ctx *ctx = m->ctx;
    NIR_CUDA_TRY(cudaSetDevice(ctx->device));
    const std::string gpu = gpu_name(ctx->device);
    if (!cache_path || !cache_path[0]) {  // the environment may name the cache
        const char *env = std::getenv("NIR_TUNE_CACHE");
        cache_path = env && env[0] ? env : nullptr;
    }
    auto kv = read_cache(cache_path);
    cudaStream_t st = ctx->stream;
    const char *pname[3] = {"f64", "f32", "bf16"};
    // scratch vectors for timing (largest block / whole mesh)
    size_t maxb = 0;
    for (auto *b : m->blocks) maxb = std::max(maxb, (size_t)b->d.nelem * b->M);
    void *x = nullptr, *y = nullptr;
    if (cudaMalloc(&x, std::max(maxb, (size_t)m->ndof) * 8) != cudaSuccess ||
        cudaMalloc(&y, std::max(maxb, (size_t)m->ndof) * 8) != cudaSuccess) {
        if (x) cudaFree(x);
        return NIR_ERR_NO_MEMORY;
    }
    cudaMemsetAsync(x, 0, std::max(maxb, (size_t)m->ndof) * 8, st);
    int rc = NIR_OK;
    for (int prec = 0; prec < 3 && !rc; ++prec) {
        // per-block elements-per-CTA variant and grid size
        for (auto *b : m->blocks) {
            char key[160];
            std::snprintf(key, sizeof key, "%s|block|%d|%d|%d|%lld|%s", gpu.c_str(), b->d.shape, b->d.P, b->d.Q,
                          (long long)b->d.nelem, pname[prec]);
            auto it = kv.find(key);
            if (it != kv.end()) {
                b->helm_pf[prec] = 0;
                std::sscanf(it->second.c_str(), "%d,%d,%d", &b->helm_variant[prec], &b->helm_grid[prec],
                            &b->helm_pf[prec]);
                // a cache entry naming the threading-over-elements kernel gets its
                // scratch here; an unknown variant falls back to 0
                int &v = b->helm_variant[prec];
                if (v == NIR_VARIANT_TOE && nir_toe_prepare(b, prec, b->helm_grid[prec]) != NIR_OK) v = 0;
                if (v < 0 || v > NIR_VARIANT_MAX || (v != NIR_VARIANT_TOE &&
                                                     !nir_kinfo(b->d.shape, b->d.P, prec, 5, v).fn))
                    v = 0;
                if (v != NIR_VARIANT_TOE) nir_toe_release(b);
                continue;
            }
            float best = 1e30f;
            int bv = 0, bg = 0, bp = 0;
            for (int v = 0; v <= NIR_VARIANT_MAX && !rc; ++v) {
                if (v == NIR_VARIANT_TOE) continue;  // timed below
                KInfo ki = nir_kinfo(b->d.shape, b->d.P, prec, 5, v);
                if (!ki.fn || ((v == 1 || v == 2) && ki.epb == nir_kinfo(b->d.shape, b->d.P, prec, 5, 0).epb)) continue;
                int occ = nir_occupancy(ctx, ki);
                const int npf = (prec != NIR_F64 && b->geo_pp && (ki.epb % 32 == 0 || 32 % ki.epb == 0)) ? 3 : 1;
                for (int c = 1; c <= std::max(1, occ) && !rc; ++c)
                    for (int pf = 0; pf < npf && !rc; ++pf) {
                        b->helm_variant[prec] = v;
                        b->helm_grid[prec] = c * ctx->num_sms;
                        b->helm_pf[prec] = pf;
                        float t = time_ms(st, 5, [&] {
                            if (!rc)
                                rc = nir_launch_op(b, prec, 5, 1.0, x, nullptr, nullptr, y, nullptr, nullptr, st, 0);
                        });
                        if (t < best) { best = t; bv = v; bg = c * ctx->num_sms; bp = pf; }
                    }
            }
            // the other threading strategy (one thread per element, Sec. 3.3): it
            // only wins in FP64 on large high-order blocks, so it is timed in FP64
            if (prec == NIR_F64 && !rc && nir_toe_prepare(b, prec, 0) == NIR_OK) {
                b->helm_variant[prec] = NIR_VARIANT_TOE;
                b->helm_grid[prec] = 0;
                b->helm_pf[prec] = 0;
                float t = time_ms(st, 5, [&] {
                    if (!rc) rc = nir_launch_op(b, prec, 5, 1.0, x, nullptr, nullptr, y, nullptr, nullptr, st, 0);
                });
                if (t < best) { best = t; bv = NIR_VARIANT_TOE; bg = 0; bp = 0; }
            }
            b->helm_variant[prec] = bv;
            b->helm_grid[prec] = bg;
            b->helm_pf[prec] = bp;
            if (bv != NIR_VARIANT_TOE) nir_toe_release(b);
            char val[64];
            std::snprintf(val, sizeof val, "%d,%d,%d", bv, bg, bp);
            kv[key] = val;
        }
        if (rc) break;
        // persistent mesh kernel: work-item granularity and grid size
        std::string sig;
        for (auto *b : m->blocks) sig += std::to_string(b->d.shape) + "." + std::to_string(b->d.P) + "." +
                                         std::to_string(b->d.nelem) + ";";
        std::string key = gpu + "|mesh|" + std::to_string(std::hash<std::string>{}(sig)) + "|" + pname[prec];
        auto it = kv.find(key);
        int gran = 1, grid = 0, mode = 0;
        if (it != kv.end()) {
            std::sscanf(it->second.c_str(), "%d,%d,%d", &gran, &grid, &mode);
            m->ps[prec].grid = grid;
            m->ps[prec].mode = (mode == 1 && m->blocks.size() > 1) ? 1 : 0;
            rc = nir_mesh_build_items(m, prec, gran);
            continue;
        }
        float best = 1e30f;
        for (int gr : {1, 2, 4, 8}) {
            m->ps[prec].grid = 0;
            rc = nir_mesh_build_items(m, prec, gr);
            if (rc) break;
            const int occ = m->ps[prec].occ;
            for (int c = 1; c <= occ && !rc; ++c) {
                m->ps[prec].grid = c * ctx->num_sms;
                nirk::MeshBlk *dblk = nullptr;
                rc = nir_mesh_block_table(m, prec, 1.0, x, y, &dblk);
                if (rc) break;
                float t = time_ms(st, 5, [&] {
                    if (!rc) rc = nir_mesh_launch_raw(m, prec, dblk, st);
                });
                cudaStreamSynchronize(st);
                cudaFree(dblk);
                if (t < best) { best = t; gran = gr; grid = c * ctx->num_sms; }
            }
        }
        if (rc) break;
        m->ps[prec].grid = grid;
        rc = nir_mesh_build_items(m, prec, gran);
        if (rc) break;
        // the persistent queue against each block's own (tuned) kernel in sequence
        m->ps[prec].mode = 0;
        if (m->blocks.size() > 1) {
            rc = nir_mesh_blocks_ready(m, prec);
            if (rc) break;
            float tb = time_ms(st, 5, [&] {
                if (!rc) rc = nir_mesh_launch_blocks(m, prec, 1.0, x, y, st);
            });
            if (!rc && tb < best) m->ps[prec].mode = 1;
        }
        char val[64];
        std::snprintf(val, sizeof val, "%d,%d,%d", gran, grid, m->ps[prec].mode);
        kv[key] = val;
    }
    cudaStreamSynchronize(st);
    cudaFree(x);
    cudaFree(y);
    for (auto &g : m->graphs) g.stale = true;  // the launch form or block kernels may have changed
    nir_cg_invalidate(m);
    if (rc) return rc;
    if (!write_cache(cache_path, kv)) return NIR_ERR_INVALID_ARG;
    return NIR_OK;
}

extern "C" int nir_mesh_get_launch(const nir_mesh *m, int prec, int *mode)
{
    if (!m || !valid_prec(prec) || !mode) return NIR_ERR_INVALID_ARG;
    *mode = m->blocks.size() == 1 ? NIR_MESH_BLOCKS : m->ps[prec].mode;
    return NIR_OK;
}

extern "C" int nir_mesh_set_launch(nir_mesh *m, int prec, int mode)
{
    if (!m || !valid_prec(prec) || (mode != NIR_MESH_PERSISTENT && mode != NIR_MESH_BLOCKS)) return NIR_ERR_INVALID_ARG;
    if (m->ps[prec].mode != mode) {
        m->ps[prec].mode = mode;
        for (auto &g : m->graphs)
            if (g.prec == prec) g.stale = true;
        nir_cg_invalidate(m);
    }
    return NIR_OK;
}
