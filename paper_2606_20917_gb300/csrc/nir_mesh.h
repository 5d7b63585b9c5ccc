// nir_mesh.h -- device-side descriptors of the persistent hybrid-mesh kernel.
#pragma once

#include "nir_kernels.cuh"

namespace nirk {

// One block of the mesh as the persistent kernel sees it.
struct MeshBlk {
    KArgs a;   // in0/out0 point at the block's slice of the mesh vectors
    int vid;   // (shape, P) variant of the kernel for this dimension/precision
    int pad[3];
};

// A work item: element groups [g0, g0 + ng) of one block.
struct MeshItem {
    int block;
    int g0;
    int ng;
    int pad;
};

}  // namespace nirk

struct MeshKInfo {
    const void *fn = nullptr;  // k_mesh of this dimension/precision
    int vid = -1;              // variant id of (shape, P)
    int smem = 0;              // dynamic shared memory the variant needs
    int epb = 0;               // elements per group of the variant
    int nt = 0;
};

// dim in {2, 3}, prec in {0, 1, 2}; fn == nullptr when (shape, P) is not covered
MeshKInfo nir_mesh_kinfo(int dim, int prec, int shape, int P);
