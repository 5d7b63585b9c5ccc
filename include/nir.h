/*
 * nir.h -- C ABI of the GB300 spectral/hp elemental-operator library.
 *
 * The library evaluates the matrix-free, sum-factorised elemental operators
 * of the spectral/hp element method (Sec. 2.1-2.2 of the NektarIR paper,
 * arXiv 2606.20917) on blocks of alike elements (Sec. 3.1, the `block` type):
 * BwdTrans, IProductWRTBase, PhysDeriv, IProductWRTDerivBase, the mass
 * operator and the weak Helmholtz operator H = L + lambda M
 * (Eqs. weakmatrixhelm, laplacian), for quadrilaterals, triangles, hexahedra,
 * prisms and tetrahedra, in FP64, FP32 and BF16 storage with FP32 arithmetic.
 * On top of them it provides a hybrid mixed-shape/mixed-order mesh applied in
 * one persistent launch and a conjugate-gradient Helmholtz solve with FP64
 * iterative refinement around an FP32/BF16 operator.
 *
 * Conventions
 *   - Every call returns NIR_OK (0) or a negative NIR_ERR_* code; nir_strerror
 *     gives a message.  Invalid arguments are rejected before any GPU work.
 *   - Array arguments of the operator calls are DEVICE pointers owned by the
 *     caller (e.g. torch tensors' data_ptr()).  They must not alias each other.
 *     Basis tables, geometric factors and scratch are owned by the library.
 *   - Operator calls are asynchronous on the context's CUDA stream; errors of
 *     the launch itself are returned, device-side errors surface at the next
 *     synchronising call of the caller.
 *   - P is the polynomial degree (N = P+1 modes per direction), Q the number of
 *     quadrature points per direction; supported: 1 <= P <= 9, Q = P + 2.
 *   - Layouts (element-major):
 *       coefficients [E][M], modes packed p outermost, then q, then r, with
 *         quad  q < N;            M = N^2
 *         tri   q < N-p;          M = N(N+1)/2
 *         hex   q, r < N;         M = N^3
 *         prism q < N, r < N-p;   M = N^2(N+1)/2
 *         tet   q < N-p, r < N-p-q; M = N(N+1)(N+2)/6     (Eq. bwdsumfactet bounds)
 *         pyr   q < N, r < N-max(p,q); M = N(N+1)(2N+1)/6
 *       physical values [E][Nq], Nq = Q^d, point index i + Q*(j + Q*k), the
 *         first direction (xi1 / eta1) fastest.
 *   - Basis: modified C0 expansion (psiA, psiB, psiC of Sec. 2.2); collapsed
 *     vertex/edge modes whose eta factor is not a polynomial in xi are defined
 *     with that factor replaced by 1.  Pyramid (the shape the paper motivates
 *     for hybrid meshes and leaves to future work): apex at xi = (-1,-1,1),
 *     eta1 = 2(1+xi1)/(1-xi3) - 1, eta2 = 2(1+xi2)/(1-xi3) - 1, eta3 = xi3,
 *     phi_pqr = psiA_p(eta1) psiA_q(eta2) psiB_{max(p,q) r}(eta3), the apex
 *     mode (0,0,1) being psiA_1(eta3) alone (a rational expansion whose traces
 *     are Q_P on the square base and P_P on the triangular faces).
 *   - Quadrature: Gauss-Lobatto-Legendre on quad/hex directions and the prism's
 *     eta1, eta2; Gauss-Jacobi(alpha,0) on collapsed directions (tri eta1 a=0,
 *     eta2 a=1; tet eta1 a=0, eta2 a=1, eta3 a=2; prism eta3 a=1; pyramid
 *     eta1, eta2 GLL, eta3 a=2), with the collapse Jacobian absorbed in the
 *     weights.
 */
#ifndef NIR_H
#define NIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { NIR_QUAD = 0, NIR_TRI = 1, NIR_HEX = 2, NIR_PRISM = 3, NIR_TET = 4, NIR_PYR = 5 } nir_shape;

/* Storage/arithmetic precision of an operator call.  NIR_BF16 stores
 * coefficients, physical values and geometric factors in bfloat16 and computes
 * in FP32. */
typedef enum { NIR_F64 = 0, NIR_F32 = 1, NIR_BF16 = 2 } nir_prec;

enum {
    NIR_OK = 0,
    NIR_ERR_INVALID_ARG = -1,   /* null/aliased pointer, bad size or enum */
    NIR_ERR_UNSUPPORTED = -2,   /* shape/P/Q combination not compiled */
    NIR_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    NIR_ERR_NOT_CONVERGED = -4, /* CG hit its iteration cap or broke down */
    NIR_ERR_NONFINITE = -5,     /* NaN/Inf met in a CG scalar */
    NIR_ERR_NO_MEMORY = -6,     /* device or host allocation failed */
    NIR_ERR_GEOMETRY = -7,      /* non-positive Jacobian determinant */
    NIR_ERR_STATE = -8,         /* geometry not set / object in wrong state */
    NIR_ERR_TOO_LARGE = -9,     /* request exceeds a fixed capacity of the library */
    NIR_ERR_COMM = -10          /* the caller's cross-rank reduction reported a failure */
};

typedef struct nir_ctx nir_ctx;
typedef struct nir_block nir_block;
typedef struct nir_mesh nir_mesh;

/* A block: alike elements sharing shape, order, quadrature and deformation
 * (Sec. 3.1, the block type's SEShape/Basis/Quadrature/Deformed/Size). */
/* Expansion basis of a block.  NIR_BASIS_MODIFIED: the modified C0 expansion
 * (every shape).  NIR_BASIS_GLL_LAGRANGE: nodal, the tensor products of the
 * Lagrange polynomials through the P+1 Gauss-Lobatto-Legendre points
 * (quadrilaterals and hexahedra; the nodal expansion the paper lists as
 * future work), coefficients = values at those points, packed like the
 * modified modes (p along xi1 outermost). */
typedef enum { NIR_BASIS_MODIFIED = 0, NIR_BASIS_GLL_LAGRANGE = 1 } nir_basis;

typedef struct {
    int shape;       /* nir_shape */
    int64_t nelem;   /* E >= 1 */
    int P;           /* polynomial degree */
    int Q;           /* quadrature points per direction (= P + 2) */
    int deformed;    /* 1: per-point geometric factors; 0: the element maps are
                        affine and quad/hex factors are stored once per element */
    int basis;       /* nir_basis (0, the modified expansion, when zero-initialised) */
} nir_block_desc;

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out owns nothing of
 * the caller.  Errors: INVALID_ARG, CUDA. */
int nir_ctx_create(nir_ctx **out, int device, void *cuda_stream);
/* Re-target subsequent calls of all blocks of this context to another stream. */
int nir_ctx_set_stream(nir_ctx *ctx, void *cuda_stream);
void nir_ctx_destroy(nir_ctx *ctx);
/* Synchronise the context stream and report device-side failures of earlier
 * asynchronous calls: kernels never hang on an asynchronous copy; a bounded
 * wait that runs out sets a device error word and the kernel returns.
 * Returns NIR_ERR_CUDA (and clears the word) if one was set. */
int nir_ctx_check(nir_ctx *ctx);
/* Failure-path self-test of the bounded wait (the paper has no counterpart:
 * this exercises the library's own failure detection).  Launches on the
 * context stream one CTA that waits on an mbarrier nothing arrives on and with
 * no copy in flight, with a wait limit of limit_cycles SM clock cycles
 * (1 .. 2^31; every staged kernel uses 2^31).  The wait runs out, the kernel
 * sets the context's device error word and returns; the next nir_ctx_check
 * reports NIR_ERR_CUDA and clears the word.  Asynchronous.  Errors:
 * INVALID_ARG, CUDA. */
int nir_ctx_selftest_wait(nir_ctx *ctx, int64_t limit_cycles);
/* Debug mode (a library facility; the paper has no counterpart).  When on,
 * every device-buffer operator call (the block operators, nir_mesh_helmholtz,
 * nir_asm_gather / assemble / pick / apply) synchronises the context stream
 * after its launch and reports a failed kernel, or a device error word set by
 * it or by earlier work on the stream, as NIR_ERR_CUDA at that call (clearing
 * the word) instead of at a later nir_ctx_check.  Calls made while the stream
 * is being captured into a CUDA graph are not synchronised.  The initial state
 * comes from the environment variable NIR_DEBUG at nir_ctx_create (set and not
 * "0": on).  Costs one host round trip per call.  Errors: INVALID_ARG (on not
 * 0 or 1). */
int nir_ctx_set_debug(nir_ctx *ctx, int on);
int nir_ctx_get_debug(const nir_ctx *ctx, int *on);

/* Create a block; builds the FP64 basis/quadrature tables (Eqs. basis matrix,
 * bwdsumfachex, bwdsumfactet, stdderiv) and uploads them.  Errors:
 * INVALID_ARG, UNSUPPORTED (also a nodal basis on a collapsed shape),
 * NO_MEMORY, CUDA. */
int nir_block_create(nir_ctx *ctx, const nir_block_desc *desc, nir_block **out);
void nir_block_destroy(nir_block *blk);
/* M (modes per element, Sec. 3.1 storage size) and Nq (points per element). */
int nir_block_num_modes(const nir_block *blk, int64_t *M);
int nir_block_num_points(const nir_block *blk, int64_t *Nq);
/* Reference coordinates of the quadrature points: eta_out [Nq][d] (collapsed
 * coordinates) and xi_out [Nq][d] (standard element, Eq. eta-space); HOST
 * pointers, either may be NULL. */
int nir_block_points(const nir_block *blk, double *eta_out, double *xi_out);

/* Geometry (Sec. 2.1: the weights matrix W and Lambda(d xi/d x)).  `nodes` is
 * a DEVICE FP64 array, read during the call only:
 *   quad/hex: [E][(g+1)^d][d] coordinates of an equispaced lattice of degree
 *             g = gorder per direction (node a + (g+1)(b + (g+1) c) at
 *             xi = -1 + 2(a,b,c)/g); the element map is its Lagrange interpolant.
 *   tri/tet/prism/pyr: gorder = 1, vertices [E][nv][d] in the order
 *             tri (-1,-1),(1,-1),(-1,1); tet (-1,-1,-1),(1,-1,-1),(-1,1,-1),(-1,-1,1);
 *             prism (-1,-1,-1),(1,-1,-1),(1,1,-1),(-1,1,-1),(-1,-1,1),(-1,1,1);
 *             pyr (-1,-1,-1),(1,-1,-1),(1,1,-1),(-1,1,-1),(-1,-1,1), mapped by the
 *             vertex functions a_i(eta1) b_j(eta2) (1-eta3)/2 and (1+eta3)/2
 *             (affine for a parallelogram base).
 * The library computes, in FP64 on the GPU, per point (or per element for an
 * undeformed quad/hex block) the Jacobian, W = w|J|, d eta/d x and the metric
 * G = W (d eta/d x)(d eta/d x)^T, and derives FP32/BF16 copies on first use.
 * Synchronises the context stream.  Errors: INVALID_ARG, GEOMETRY (some
 * det J <= 0 or non-finite), NO_MEMORY, CUDA. */
int nir_block_set_geometry(nir_block *blk, int gorder, const double *nodes);

/* Geometry given as geometric factors, the form of the paper's statement of
 * the problem (Sec. 2.1: the weights matrix W = diag(w |J|) and, in
 * Eq. physderiv, Lambda(d xi/d x)), for callers that already hold them.
 * DEVICE FP64 arrays, caller-owned, read during the call only:
 *   per_element = 0: dxi_dx [E][Nq][d][d], jac [E][Nq] -- at every
 *                    quadrature point (point order as for physical values);
 *   per_element = 1: dxi_dx [E][d][d], jac [E] -- constant over each
 *                    element (an affine element map), any shape.
 * dxi_dx[.][i][l] = d xi_i / d x_l of the standard element (the collapsed
 * coordinates' chain rule d eta/d xi is applied by the library); jac = |J| =
 * det(d x/d xi) > 0.  The library forms W = w |J| (w: quadrature weights with
 * the collapse factors), d eta/d x and G = W (d eta/d x)(d eta/d x)^T in FP64
 * on the GPU, exactly as nir_block_set_geometry does from the element maps,
 * and derives FP32/BF16 copies on first use.  An undeformed quad/hex block
 * stores one set of factors per element and takes only per_element = 1.
 * Synchronises the context stream.  Errors: INVALID_ARG (null or aliased
 * pointers, per_element not 0/1, per-point factors for an undeformed quad/hex
 * block), GEOMETRY (some jac <= 0 or non-finite), NO_MEMORY, CUDA. */
int nir_block_set_geometric_factors(nir_block *blk, int per_element, const double *dxi_dx, const double *jac);

/* BwdTrans u = B u_hat (Eqs. bwdstd, bwdsumfachex, bwdsumfactet).
 * coeff [E][M] -> phys [E][Nq]. */
int nir_bwd_trans(nir_block *blk, int prec, const void *coeff, void *phys);
/* IProductWRTBase u_hat = B^T W u (Eqs. iprodhex, iprodtet).
 * phys [E][Nq] -> coeff [E][M]. */
int nir_iproduct_wrt_base(nir_block *blk, int prec, const void *phys, void *coeff);
/* PhysDeriv du/dx_l = sum_j Lambda(d eta_j/d x_l) D_eta_j u (Eqs. physderiv,
 * stdderiv).  phys [E][Nq] -> d0, d1 (, d2) [E][Nq]; d2 must be NULL in 2-D. */
int nir_phys_deriv(nir_block *blk, int prec, const void *phys, void *d0, void *d1, void *d2);
/* IProductWRTDerivBase: coeff = sum_l (D_xl B)^T W f_l (the test_grad
 * operation, Sec. 3.1).  f0, f1 (, f2) [E][Nq] -> coeff [E][M]. */
int nir_iproduct_wrt_deriv_base(nir_block *blk, int prec, const void *f0, const void *f1,
                                const void *f2, void *coeff);
/* Mass operator M u_hat = B^T W B u_hat (Eq. laplacian). [E][M] -> [E][M]. */
int nir_mass(nir_block *blk, int prec, const void *coeff_in, void *coeff_out);
/* Helmholtz operator (L + lambda M) u_hat (Eqs. weakmatrixhelm, laplacian),
 * one fused launch.  [E][M] -> [E][M]; lambda > 0 for an SPD operator. */
int nir_helmholtz(nir_block *blk, int prec, double lambda, const void *coeff_in, void *coeff_out);
/* The Helmholtz operator applied to 1..3 fields of the same block in one
 * launch (e.g. the velocity components of a velocity-correction step, which
 * share the operator): in[f] -> out[f], each [E][M] in prec, all distinct.
 * Each element group computes its fields back to back, so the group's
 * geometric factors are read from HBM once.  Errors: INVALID_ARG, STATE. */
int nir_helmholtz_fields(nir_block *blk, int prec, double lambda, int nfields, const void *const *in,
                         void *const *out);
/* nir_helmholtz on HOST buffers: copies h_in to the device, applies, copies
 * the result to h_out, and synchronises.  Pinned host memory gives full
 * copy bandwidth.  Device staging buffers are library-owned. */
int nir_helmholtz_host(nir_block *blk, int prec, double lambda, const void *h_in, void *h_out);

/* Largest coefficient vector (bytes) nir_helmholtz_host_noalloc can stage. */
#define NIR_NOALLOC_MAX_VECTOR_BYTES ((size_t)16 << 20)

/* nir_helmholtz_host for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a deployment variant of the host-buffer
 * entry point.  It calls no cudaMalloc/cudaFree or any allocating routine;
 * instead the host arrays are staged through one fixed device array compiled
 * into the library (2 x NIR_NOALLOC_MAX_VECTOR_BYTES = 32 MiB, held on every
 * GPU that loads the library until the process exits).  Meant for programs
 * whose device memory belongs to a pool/caching allocator, loops that must
 * not stall on an allocation, and hosts that forbid allocation after set-up.
 *   - h_in, h_out: HOST arrays [E][M] in the precision's type, as for
 *     nir_helmholtz_host.  Synchronises the context stream before returning.
 *   - Errors: INVALID_ARG; STATE when geometry is not set, or for NIR_F32 /
 *     NIR_BF16 when no allocating call in that precision has yet derived the
 *     block's low-precision factors; TOO_LARGE when E*M*sizeof exceeds
 *     NIR_NOALLOC_MAX_VECTOR_BYTES (nothing is launched); CUDA.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (with that device current) and keeps it for the
 *     life of the process; make that first call before any stream capture,
 *     and do not reset the device (cudaDeviceReset) after it.
 *   - On any error after the input copy was queued the call still waits for
 *     the stream before returning, so h_in and h_out are free on return.
 *   - Every call shares the one array and leaves its last contents there;
 *     calls whose work overlaps on the GPU (other threads or streams) race
 *     on it, so serialise them. */
int nir_helmholtz_host_noalloc(nir_block *blk, int prec, double lambda, const void *h_in, void *h_out);

/* Launch tuning of a block's Helmholtz kernel in one precision (what nir_tune
 * sets): variant 0 = default elements per CTA, 1 = half, 2 = double (where it
 * fits in shared memory; otherwise the default), 3 = the default group run by
 * the multi-field kernel (same results, another register allocation); grid =
 * CTAs launched (0: one wave at the kernel's occupancy); pf = L2 prefetch of
 * the groups' metric (FP32/BF16 with per-point factors; ignored elsewhere):
 * 0 none, 1 each CTA's next group while the current one finishes, 2 each
 * group's own when it starts.
 * Variant 4 selects the other threading strategy of Sec. 3.3, threading over
 * elements: one thread per element runs all stages, its intermediate tensors
 * in library-owned global scratch of 5 Q^d values per thread of the grid
 * (allocated by this call, freed with the block; single-field Helmholtz
 * only, modified basis only; the autotuner times it in FP64, where its
 * results equal the other variants' bit for bit).  grid = CTAs of 128
 * threads (0: one wave at its occupancy), at most one CTA per 128 elements.
 * A block's launches share that scratch: calls on one block must not overlap
 * on the GPU.  Leaving variant 4 in the last precision that used it frees the
 * scratch.  Selecting or leaving variant 4 allocates or frees device memory
 * and synchronises the device, so it must not overlap a stream capture on
 * this device; while the context stream is capturing it returns STATE.
 * Variant 5 (FP32/BF16, quad and hex; UNSUPPORTED elsewhere) runs the default
 * group with two elements per thread: each pencil carries elements 2e and
 * 2e+1 side by side in shared memory (one 8-byte access for both) and each
 * table coefficient multiplies both in one packed FP32x2 operation, halving
 * the per-pencil index and memory instructions.  Same arithmetic per element
 * as variant 0, up to the compiler's contraction of separate multiplies and
 * adds.
 * Errors: INVALID_ARG (also pf outside 0..2), STATE; with variant 4 also
 * UNSUPPORTED (nodal basis), TOO_LARGE (2^31 or more scratch values),
 * NO_MEMORY, CUDA; with variant 5 UNSUPPORTED. */
int nir_block_set_tuning(nir_block *blk, int prec, int variant, int grid, int pf);
int nir_block_get_tuning(const nir_block *blk, int prec, int *variant, int *grid, int *pf);

/* Resources of the kernel a block launches for operator `op` in `prec` (with
 * the block's current tuning): registers per thread, shared memory per CTA
 * (dynamic + static, bytes), threads per CTA and elements per CTA group.  op:
 * 0 BwdTrans, 1 IProductWRTBase, 2 PhysDeriv, 3 IProductWRTDerivBase, 4 mass,
 * 5 Helmholtz.  NULL outputs are skipped.  Errors: INVALID_ARG, UNSUPPORTED,
 * CUDA. */
int nir_block_kernel_info(const nir_block *blk, int prec, int op, int *regs, int *smem_bytes, int *threads,
                          int *elems_per_cta);

/* Hybrid mesh: the concatenation of blocks (each with geometry set), applied
 * by one persistent launch (Sec. 2.2: operators batched over blocks of alike
 * elements).  Vectors are the concatenation of the blocks' coefficient arrays
 * in block order.  The mesh keeps pointers to the blocks, which must outlive it. */
int nir_mesh_create(nir_ctx *ctx, nir_block *const *blocks, int nblocks, nir_mesh **out);
void nir_mesh_destroy(nir_mesh *mesh);
int nir_mesh_num_dofs(const nir_mesh *mesh, int64_t *ndof);
/* Helmholtz apply over all blocks in one persistent kernel launch, replayed
 * from a CUDA graph captured on first use for each (prec, buffers) pair.  A
 * mesh of a single block launches that block's own (tuned) kernel instead: a
 * work queue has nothing to balance there. */
int nir_mesh_helmholtz(nir_mesh *mesh, int prec, double lambda, const void *in, void *out);
/* Autotune elements-per-CTA and grid size of every (shape, P, prec) of the mesh
 * by timing candidates, and per precision the launch form (below); reads/writes
 * a JSON cache at cache_path, or, when cache_path is NULL or empty, at the path
 * the environment variable NIR_TUNE_CACHE names (no cache if that is unset or
 * empty too).  Errors: INVALID_ARG (also an unwritable cache), NO_MEMORY, CUDA. */
int nir_tune(nir_mesh *mesh, const char *cache_path);

/* Launch form of a mesh apply: NIR_MESH_PERSISTENT = one persistent kernel
 * pulling (block, element-group) items from a queue (the default for meshes of
 * several blocks); NIR_MESH_BLOCKS = each block's own tuned kernel, launched in
 * sequence.  Either form is captured in one CUDA graph per (prec, buffers,
 * lambda) and replayed.  nir_tune picks the faster per precision; set/get
 * override and report it (a mesh of one block always reports BLOCKS). */
enum { NIR_MESH_PERSISTENT = 0, NIR_MESH_BLOCKS = 1 };
int nir_mesh_set_launch(nir_mesh *mesh, int prec, int mode);
int nir_mesh_get_launch(const nir_mesh *mesh, int prec, int *mode);

typedef struct {
    int inner_prec;        /* nir_prec of the operator inside CG (F64: plain CG) */
    double tol;            /* target ||b - H x|| / ||b|| (FP64 residual) */
    int max_outer;         /* refinement sweeps (ignored for plain FP64 CG) */
    int max_inner;         /* CG iterations per sweep (total for plain CG) */
    double inner_tol;      /* relative residual reduction per refinement sweep
                              (plain CG: per polishing sweep, see fwd_tol;
                              0 there means 1e-3) */
    int jacobi;            /* 1: diagonal (Jacobi) preconditioner */
    int inner_vectors;     /* storage and arithmetic of the inner solver's
                              vectors (correction, residual, preconditioned
                              residual, search direction) and of its dot
                              products: NIR_F64 (0, the default when the struct
                              is zero-initialised): FP64 vectors, FP64 updates
                              and dots; the operator reads an FP32/BF16 copy of
                              the search direction and returns H p in its own
                              type.  NIR_F32: FP32 vectors and updates, dots of
                              exact FP32 products with compensated summation,
                              per-thread partials summed in FP64 (faster on
                              GB300, whose FP64 rate is a small fraction of
                              FP32).  Ignored for plain FP64 CG. */
    double fwd_tol;        /* > 0: also require the last correction to be
                              small, ||dx|| <= fwd_tol ||x||, which bounds the
                              forward error ||x - H^-1 b|| / ||x|| (the error
                              left after a correction is a fraction of that
                              correction).  Mixed precision: dx is the last
                              refinement sweep's update.  Plain FP64 CG: once
                              the residual meets tol, CG continues in
                              polishing sweeps that each cut the residual by
                              inner_tol, and dx is one sweep's update.
                              0: stop on the residual alone. */
} nir_cg_opts;

typedef struct {
    int outer;             /* refinement (plain CG: restart/polishing) sweeps */
    int inner_total;       /* operator applies in the inner solver */
    double rel_residual;   /* final ||b - H x|| / ||b|| in FP64 */
    double seconds;        /* wall time of the solve */
    double rel_correction; /* ||dx|| / ||x|| of the last sweep's update (the
                              forward-error estimate of fwd_tol; 0 when no
                              sweep measured it) */
} nir_cg_stats;

/* Solve (L + lambda M) x = b on the mesh's broken (element-block-diagonal)
 * operator.  b, x: DEVICE FP64 [ndof]; x holds the initial guess on entry.
 * Plain CG when inner_prec == NIR_F64; otherwise CG in inner_prec on the
 * defect equation inside FP64 iterative refinement: r = b - H x in FP64,
 * solve H_lo d = r / |r| to inner_tol, x += |r| d, until |r| / |b| <= tol (and
 * the correction meets fwd_tol when set).  The refinement residual, the
 * update of x and (with inner_vectors = NIR_F64) the inner CG's residuals,
 * search directions and dot products are FP64 on the GPU.  Synchronous.
 * Errors: INVALID_ARG, NOT_CONVERGED (iteration or sweep cap, stalled
 * refinement, CG breakdown), NONFINITE, CUDA, NO_MEMORY. */
int nir_cg_solve(nir_mesh *mesh, double lambda, const double *b, double *x, const nir_cg_opts *opts,
                 nir_cg_stats *stats);

/* ---------------------------------------------------------------------------
 * Solves sharded across ranks (one process per GPU).
 *
 * The operators are element-local, so a mesh splits into contiguous element
 * ranges, one per rank, with no exchange in the apply (the paper's CPU runs
 * split elements across MPI ranks the same way, Sec. 4).  The broken
 * operator's CG then needs only sums of FP64 scalars over the ranks.
 * --------------------------------------------------------------------------- */

/* Contiguous element ranges of the concatenation of nblocks blocks (block b:
 * shape[b], degree P[b], nelem[b] elements, in block order), one per rank,
 * balanced by the sum-factorised Helmholtz flops per element of each
 * (shape, P) (the costs the kernels' rooflines use).  first_out[nranks + 1]
 * (HOST): rank r owns global elements [first_out[r], first_out[r+1]); first
 * is 0 and last the total.  Host only (no GPU needed).  Errors: INVALID_ARG. */
int nir_partition_elements(int nblocks, const int *shape, const int *P, const int64_t *nelem, int nranks,
                           int64_t *first_out);

/* Sum of n FP64 values over all ranks, in place: `values` is a HOST array of
 * this rank's partial sums on entry and must hold the totals on return, the
 * same on every rank.  Returns 0 on success; anything else aborts the solve
 * with NIR_ERR_COMM. */
typedef int (*nir_allreduce_fn)(double *values, int n, void *user);

/* nir_cg_solve on one rank's part of a sharded mesh: `mesh` holds this rank's
 * elements (e.g. its range from nir_partition_elements), b and x its entries
 * (DEVICE FP64 [ndof of this mesh]).  Every rank calls it collectively with
 * the same options; every dot product (residual norms, CG scalars, the
 * forward-error norms, the preconditioner check) is this rank's partial sum
 * passed through `allreduce`, so all ranks take the same iterations and stop
 * together.  The iterations run without graph capture, with two host round
 * trips per CG iteration (the partial p.Ap, then r.z and r.r).  A rank that
 * fails in its own work returns without further reductions: the caller's
 * reduction must then fail (e.g. a process-group timeout) on the other
 * ranks.  Results equal the single-rank solve up to the rounding of the
 * reduction order.  Errors: as nir_cg_solve, plus COMM. */
int nir_cg_solve_dist(nir_mesh *mesh, double lambda, const double *b, double *x, const nir_cg_opts *opts,
                      nir_cg_stats *stats, nir_allreduce_fn allreduce, void *user);

/* ---------------------------------------------------------------------------
 * Conforming C0 assembly (quadrilateral and hexahedral blocks).
 *
 * The elemental operators above act on broken (element-local) expansions; the
 * paper's solve leaves assembly out (Sec. 2.1).  An assembly object joins the
 * elements of conforming blocks into the continuous spectral/hp space of the
 * modified or the GLL-Lagrange basis: a global vector x_g maps to element
 * coefficients by x_loc = A x_g (every local mode takes +-1 times one global
 * dof; the index and, for the modified basis, the sign account for the
 * orientation of shared edges and faces), and element
 * results are summed back by y_g = A^T y_loc.  The assembled Helmholtz
 * operator is A^T H A (H = L + lambda M elementwise), the assembled mass
 * operator A^T M A.
 *   - Global vectors hold n_global entries: the n_free dofs not on the mesh
 *     boundary first, then the boundary dofs.  Local vectors are the
 *     concatenation of the blocks' [E][M] arrays in block order.
 *   - Boundary = faces (2-D: edges) held by one element, with their vertices
 *     and edges.
 * --------------------------------------------------------------------------- */
typedef struct nir_asm nir_asm;

enum { NIR_ASM_HELMHOLTZ = 0, NIR_ASM_MASS = 1 };

/* Build the global numbering of conforming blocks of one shape (NIR_QUAD or
 * NIR_HEX), one P and one basis (NIR_BASIS_MODIFIED or
 * NIR_BASIS_GLL_LAGRANGE; the Lagrange numbering has all signs +1).
 * vertex_ids[b]: HOST int64 array [nelem_b][2^d] of the global vertex ids of
 * block b's elements, local vertex v = a + 2b (+ 4c) at
 * reference coordinates xi = (-1+2a, -1+2b(, -1+2c)) -- the corners of the
 * geometry lattice of nir_block_set_geometry.  Elements may see shared faces
 * in any orientation.  The object keeps pointers to the blocks, which must
 * outlive it.  Errors: INVALID_ARG (null pointers, a face held by more than
 * two elements), UNSUPPORTED (other shapes, mixed shapes, orders or bases),
 * TOO_LARGE (2^31 or more dofs), NO_MEMORY, CUDA. */
int nir_asm_create(nir_ctx *ctx, nir_block *const *blocks, const int64_t *const *vertex_ids, int nblocks,
                   nir_asm **out);
void nir_asm_destroy(nir_asm *a);
/* The numbering alone, on the host (no GPU needed): nblocks blocks of nelem[b]
 * elements of `shape` (NIR_QUAD / NIR_HEX), degree P and basis (NIR_BASIS_*)
 * with vertex ids as for nir_asm_create.  map_out: HOST int64 [sum_b nelem[b] * M] receiving
 * s (g + 1) per local dof (may be NULL); n_global, n_free as for
 * nir_asm_num_dofs.  nir_asm_create uses exactly this numbering. */
int nir_c0_numbering(int shape, int P, int basis, int nblocks, const int64_t *nelem,
                     const int64_t *const *vertex_ids, int64_t *map_out, int64_t *n_global, int64_t *n_free);
/* Sizes: global dofs, free (non-boundary) dofs, local dofs; NULL outputs skipped. */
int nir_asm_num_dofs(const nir_asm *a, int64_t *n_global, int64_t *n_free, int64_t *n_local);
/* HOST copy of the map: map_out[i] = s (g + 1) for local dof i, s = +-1. */
int nir_asm_local_map(const nir_asm *a, int64_t *map_out);
/* x_local = A x_global; DEVICE arrays in the precision's type. */
int nir_asm_gather(nir_asm *a, int prec, const void *x_global, void *x_local);
/* y_global = A^T y_local (sums in FP64, a fixed order per dof: deterministic). */
int nir_asm_assemble(nir_asm *a, int prec, const void *y_local, void *y_global);
/* x_global from a continuous local vector: each dof takes its first local
 * copy times its sign (the inverse of nir_asm_gather on its range); FP64. */
int nir_asm_pick(nir_asm *a, const double *x_local, double *x_global);
/* y_global = A^T K A x_global with K the elemental Helmholtz (op
 * NIR_ASM_HELMHOLTZ, lambda) or mass (NIR_ASM_MASS) operator: gather, one
 * elemental launch per block, assembly.  DEVICE arrays [n_global] in prec. */
int nir_asm_apply(nir_asm *a, int op, double lambda, int prec, const void *x_global, void *y_global);
/* Solve the assembled system (options as nir_cg_solve).  b, x: DEVICE FP64
 * [n_global].  fix_boundary = 1: the boundary entries of x are Dirichlet
 * data and stay fixed; the free entries solve rows 0..n_free-1 of
 * A^T K A x = b (the boundary values enter through the FP64 residual).
 * fix_boundary = 0: all n_global entries are unknowns (e.g. the L2
 * projection with NIR_ASM_MASS, or natural boundaries with lambda > 0).  x holds
 * the initial guess on entry.  lambda is ignored for NIR_ASM_MASS.
 * Synchronous.  Errors: INVALID_ARG, STATE, NOT_CONVERGED, NONFINITE, CUDA,
 * NO_MEMORY. */
int nir_asm_cg_solve(nir_asm *a, int op, double lambda, int fix_boundary, const double *b, double *x,
                     const nir_cg_opts *opts, nir_cg_stats *stats);

/* Measure the FP64 FMA throughput of the device (TFLOP/s) with a register-
 * resident DFMA loop; used as the FP64 roofline ceiling. Synchronous. */
int nir_probe_fp64_peak(nir_ctx *ctx, double *tflops);
/* Measure the FP64 tensor-core (DMMA, mma.sync m8n8k4 f64) throughput of the
 * device (TFLOP/s) with register-resident accumulator chains; compared with
 * nir_probe_fp64_peak it tells whether FP64 contractions would gain from the
 * tensor pipe.  Synchronous. */
int nir_probe_fp64_mma_peak(nir_ctx *ctx, double *tflops);

const char *nir_strerror(int code);
/* Library version string. */
const char *nir_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NIR_H */
