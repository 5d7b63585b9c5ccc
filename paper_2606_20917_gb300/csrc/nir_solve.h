// nir_solve.h -- host-side mesh object shared by the mesh, tuner and CG units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "nir_internal.h"
#include "nir_mesh.h"

struct MeshPrec {
    bool ready = false;
    const void *fn = nullptr;        // persistent kernel of this precision
    int smem = 0;                    // dynamic shared memory (max over the mesh's variants)
    int occ = 1;                     // CTAs per SM at that shared memory
    int nt = 256;                    // threads per CTA of the persistent kernel
    int grid = 0;                    // CTAs launched (tuned; 0: occ * SMs)
    int gran = 1;                    // element groups per work item (tuned)
    int mode = 0;                    // 0: persistent kernel; 1: each block's own kernel in sequence (tuned)
    std::vector<int> vid;            // variant id per block
    nirk::MeshItem *ditems = nullptr;
    int nitems = 0;
};

struct MeshGraph {
    int prec = 0;
    const void *in = nullptr;
    void *out = nullptr;
    double lambda = 0.0;
    bool stale = false;
    nirk::MeshBlk *dblk = nullptr;   // device block table with this call's pointers
    cudaGraphExec_t exec = nullptr;
};

struct CGWork;
struct CgOperator;

struct nir_mesh {
    nir_ctx *ctx = nullptr;
    int dim = 0;
    std::vector<nir_block *> blocks;
    std::vector<long long> off;      // first dof of each block
    long long ndof = 0;
    MeshPrec ps[3];
    int *counter = nullptr;          // work-queue counters, one per precision
    cudaStream_t cap_stream = nullptr;
    std::vector<MeshGraph> graphs;
    std::vector<unsigned> geo_seen;  // blocks' geometry versions the captured graphs use
    CGWork *cg = nullptr;
    CgOperator *cg_op = nullptr;     // the CG solver's view of this mesh
    // concurrent branches of the block-kernel launch form
    static constexpr int kSide = 4;
    cudaStream_t side[kSide] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kSide] = {};
    std::vector<int> side_of;        // branch of each block (cost-balanced)
};

int nir_mesh_build_items(nir_mesh *m, int prec, int gran);
// Drop the mesh's captured graphs and CG state when a block's geometry changed.
int nir_mesh_sync_geometry(nir_mesh *m);
int nir_mesh_prepare(nir_mesh *m, int prec);
int nir_mesh_launch_raw(nir_mesh *m, int prec, const nirk::MeshBlk *dblk, cudaStream_t st);
// Each block's own kernel, one launch per block, on `st` (capturable once the
// blocks' low-precision factors and kernel attributes exist).
int nir_mesh_launch_blocks(nir_mesh *m, int prec, double lambda, const void *in, void *out, cudaStream_t st);
// Create what nir_mesh_launch_blocks needs before it is captured.
int nir_mesh_blocks_ready(nir_mesh *m, int prec);
int nir_mesh_block_table(nir_mesh *m, int prec, double lambda, const void *in, void *out, nirk::MeshBlk **dout);
int nir_mesh_apply(nir_mesh *m, int prec, double lambda, const void *in, void *out, cudaStream_t st);
void nir_cg_free(nir_mesh *m);
// Drop captured CG iteration graphs (after the work list or geometry changed).
void nir_cg_invalidate(nir_mesh *m);
