/*
 * trid.h -- C ABI of the GB300 (sm_103a) batched tridiagonal solver and ADI
 * heat-diffusion step.
 *
 * Method: arXiv 2201.03950, "High Throughput Multidimensional Tridiagonal
 * Systems Solvers on FPGAs".  The problem statement is Section 2, eq.
 * tdma-single / tdma-system:
 *
 *     a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i,   i = 0..N-1,
 *     a_0 = c_{N-1} = 0,
 *
 * with many independent systems laid along one axis of a 2D/3D mesh
 * (Section 2.1).  Meshes are column-major: element (i0, i1, i2) of a mesh with
 * dims (n0, n1, n2) sits at linear index i0 + n0 * (i1 + n1 * i2), so dims[0]
 * is the contiguous (x) axis.
 *
 * Conventions shared by every entry point:
 *   - Pointers named a, b, c, d, u, workspace are DEVICE pointers owned by the
 *     caller; the library never frees or retains them.  Dense, packed arrays
 *     of prod(dims) elements of the given dtype.  Any element-aligned address
 *     is accepted; 16-byte alignment enables vector loads.
 *   - `dims` and `offsets` marked "host" are read on the host during the call.
 *   - Argument errors are detected on the host before any launch: the call
 *     returns a nonzero trid_status and launches nothing.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream).  A launch failure reported by the runtime right
 *     after the launch maps to TRID_ERR_CUDA.
 *   - No exception, abort() or exit() crosses this ABI.
 *   - Every call may be captured into a CUDA graph, EXCEPT the first call on a
 *     device (which queries device attributes) and calls that need to grow
 *     the library's scratch pool (see trid_solve_batch).  trid_init does both
 *     ahead of time, so that every later call can be captured.
 *   - The library caches per-device state (attributes, kernel limits, the
 *     pool, device addresses).  Call trid_finalize before cudaDeviceReset on
 *     a device that the library has used.
 */
#ifndef TRID_H_
#define TRID_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *trid_stream_t; /* identical to cudaStream_t */

typedef enum { TRID_F32 = 0, TRID_F64 = 1 } trid_dtype;

typedef enum {
    TRID_OK = 0,
    TRID_ERR_INVALID_ARG = 1, /* NULL pointer, bad dims/ndim/solve_dim/dtype, aliasing */
    TRID_ERR_UNSUPPORTED = 2, /* valid request this build cannot serve          */
    TRID_ERR_MISALIGNED = 3,  /* pointer not aligned to its element size        */
    TRID_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed           */
    TRID_ERR_ALLOC = 5,       /* scratch allocation failed / workspace too small */
    TRID_ERR_TIMEOUT = 6      /* a bounded device-side wait gave up             */
} trid_status;

/*
 * Library lifecycle on the current device (not a construct of the paper: it
 * owns the scratch that the long-system passes of Section 3.1 need when the
 * caller passes none).
 *
 * trid_init(pool_bytes): queries and caches the current device's attributes,
 *   looks up the device status word and the allocation-free scratch array,
 *   creates the library's auxiliary stream (used by adi2v_backward), and
 *   makes the library's scratch pool at least pool_bytes bytes (0: leave
 *   the pool as it is).  Size the pool with trid_solve_workspace_bytes for the
 *   largest problem to come; trid_solve_batch calls that fit it then never
 *   allocate, so they may be captured into a CUDA graph.  Allocates with
 *   cudaMalloc; not capturable itself.  Calling it again only grows the pool.
 *   Errors: TRID_ERR_CUDA (no usable device), TRID_ERR_UNSUPPORTED (the
 *   driver lacks tensor-map encoding), TRID_ERR_ALLOC (cudaMalloc failed).
 * trid_finalize(): synchronises the current device (every stream), frees its
 *   scratch pool, destroys its auxiliary stream and forgets every cached
 *   state of that device.  Later calls
 *   work as on a fresh device (the first one re-queries the attributes and
 *   grows the pool again when it needs it).  Call it before cudaDeviceReset.
 *   Errors: TRID_ERR_CUDA (no device, or the synchronisation reported an
 *   error, in which case nothing is freed).
 * Neither is required: without trid_init the first call on a device does the
 * same set-up lazily, and the pool lives until the process exits.
 */
trid_status trid_init(size_t pool_bytes);
trid_status trid_finalize(void);

/* Human-readable name of a status code (static storage). */
const char *trid_status_string(trid_status s);

/* Text of the most recent CUDA runtime error that made a call of this library
 * return TRID_ERR_CUDA ("none" if there was none).  Static storage; the
 * record is process-wide and is not cleared by reading it. */
const char *trid_last_cuda_error(void);

/*
 * Batched solve along one mesh axis (Section 2.1; Algorithm "thomas" of
 * Section 2 defines the result, which is the unique x = A^{-1} d).
 *
 *   dims[0..ndim-1]  host int64 mesh extents, ndim in {1, 2, 3}, each >= 0.
 *   solve_dim        axis along which the systems lie, 0 <= solve_dim < ndim.
 *                    There are prod(dims)/dims[solve_dim] systems of length
 *                    dims[solve_dim]; element i of a system is i * stride
 *                    after its first element (stride 1, n0 or n0*n1).
 *   a, b, c          coefficients; a at the first element and c at the last
 *                    element of every system are NOT read (treated as 0).
 *   d                right-hand side.
 *   u == NULL        x overwrites d in place (Algorithm "thomas" updates d).
 *   u != NULL        u += x and d is left unmodified (Algorithm "adi",
 *                    "u = u + d").  u must not alias a, b, c or d.
 *   dtype            TRID_F32 or TRID_F64; all arrays share it.
 *
 * Systems of up to 256 rows are solved in one pass with the tiled hybrid of
 * Section 3.1 held in registers.  Longer FP32 systems of up to 4096 rows
 * are solved in one pass too, without scratch, when their arrays start on
 * 16-byte boundaries and (contiguous systems) the length is a multiple of 4
 * or (strided systems) the contiguous extent times 4 bytes is a multiple of
 * 16: whole systems staged in shared memory, or one thread-block cluster per
 * strip of 16 systems.  All other long systems (longer, FP64, unaligned) go
 * through the hybrid in several passes, which need scratch of
 * trid_solve_workspace_bytes(...) bytes; this entry point takes it from a
 * library-owned pool of the current device, grown (device synchronisation,
 * cudaFree, cudaMalloc) only when the multi-pass path is taken and the pool
 * is too small: such a call must not be inside a stream capture (pre-size
 * the pool with trid_init to avoid it).  The pool is one buffer per device,
 * shared by every stream: multi-pass calls whose work overlaps on the GPU
 * (different streams, no ordering between them) race on it and may return
 * wrong results; order them, or give each stream its own scratch through
 * trid_solve_batch_ws.  trid_finalize frees the pool.
 * No numerical pivoting: the caller guarantees a nonsingular system for
 * which Gaussian elimination without pivoting is stable (e.g. diagonally
 * dominant rows).  An exact zero pivot yields inf/nan, not an error code.
 */
trid_status trid_solve_batch(const void *a, const void *b, const void *c, void *d, void *u,
                             const int64_t *dims, int ndim, int solve_dim, trid_dtype dtype,
                             trid_stream_t stream);

/* Scratch bytes trid_solve_batch_ws needs for this problem: 0 for systems of
 * up to 256 rows, else what the multi-pass path needs (an upper bound: the
 * one-pass long-system kernels need none, but whether they apply depends on
 * the arrays' alignment).  Returns 0 as well for invalid arguments. */
size_t trid_solve_workspace_bytes(const int64_t *dims, int ndim, int solve_dim, trid_dtype dtype);

/* As trid_solve_batch, with caller-owned device scratch `workspace` of
 * `workspace_bytes` bytes (>= trid_solve_workspace_bytes; 256-byte aligned).
 * Never allocates.  Returns TRID_ERR_ALLOC if the workspace is too small. */
trid_status trid_solve_batch_ws(const void *a, const void *b, const void *c, void *d, void *u,
                                const int64_t *dims, int ndim, int solve_dim, trid_dtype dtype,
                                void *workspace, size_t workspace_bytes, trid_stream_t stream);

/*
 * Adjoint of trid_solve_batch, for reverse-mode differentiation of
 * x = A^{-1} d along a mesh axis (the solve is the one Section 2 defines; its
 * adjoint is standard linear algebra, which the paper does not discuss).
 * Given the forward solution x and g_x = dL/dx (device arrays, same layout as
 * the forward call), it writes
 *   g_d = A^{-T} g_x      (A^T: sub-diagonal c_{i-1}, diagonal b_i,
 *                          super-diagonal a_{i+1}),
 *   g_a_i = -g_d_i x_{i-1},  g_b_i = -g_d_i x_i,  g_c_i = -g_d_i x_{i+1},
 * with g_a = 0 on each system's first row and g_c = 0 on its last row (those
 * entries are not part of A).  g_a, g_b, g_c may be NULL (not written); g_d is
 * required.  Outputs must not alias each other or the inputs.  a at each
 * system's first row and c at its last row are not read.
 * Systems longer than 256 need `workspace` of
 * trid_adjoint_workspace_bytes(...) bytes (256-byte aligned); else it may be
 * NULL.  Never allocates.
 */
trid_status trid_solve_batch_adjoint(const void *a, const void *b, const void *c, const void *x,
                                     const void *g_x, void *g_a, void *g_b, void *g_c, void *g_d,
                                     const int64_t *dims, int ndim, int solve_dim,
                                     trid_dtype dtype, void *workspace, size_t workspace_bytes,
                                     trid_stream_t stream);

/* Scratch bytes trid_solve_batch_adjoint needs (0 for systems <= 256). */
size_t trid_adjoint_workspace_bytes(const int64_t *dims, int ndim, int solve_dim,
                                    trid_dtype dtype);

/*
 * Batch of independent systems of different lengths, solved in one
 * persistent launch (the batched solves of Section 4 generalised to uneven
 * lengths; long systems use the tiled Thomas-PCR hybrid of Section 3.1).
 *
 *   offsets    DEVICE int64 array of nsys + 1 entries: system k occupies rows
 *              [offsets[k], offsets[k+1]) of a, b, c, d (and u), which are
 *              dense arrays of `total` elements.  Systems may have length 0;
 *              a system with rows outside [0, total) or longer than max_len
 *              is skipped and TRID_ERR_INVALID_ARG is recorded in the device
 *              status word (trid_get_device_status).
 *   total      host: number of elements of each array.
 *   max_len    host: an upper bound of the system lengths; it sizes the
 *              shared-memory reduced systems (TRID_ERR_UNSUPPORTED when they
 *              do not fit: about 56K rows in FP32, 27K in FP64).
 *   u, dtype, stream  as for trid_solve_batch (u == NULL: in place in d),
 *              except that a, b, c, d and u must start on 16-byte boundaries
 *              (TRID_ERR_MISALIGNED otherwise, nothing launched).
 *   workspace  caller device scratch of trid_solve_varlen_workspace_bytes(nsys)
 *              bytes, 256-byte aligned (work order and queue counters; fully
 *              rewritten by every call, so calls on one workspace must not
 *              overlap on the GPU).
 * Two kernels are enqueued (a planning pass that orders the systems longest
 * first, then the persistent solve); nothing is allocated and the host does
 * not wait.
 */
trid_status trid_solve_batch_varlen(const void *a, const void *b, const void *c, void *d, void *u,
                                    const int64_t *offsets, int64_t nsys, int64_t total,
                                    int64_t max_len, trid_dtype dtype, void *workspace,
                                    size_t workspace_bytes, trid_stream_t stream);

/* Workspace bytes trid_solve_batch_varlen needs for nsys systems. */
size_t trid_solve_varlen_workspace_bytes(int64_t nsys);

/*
 * Allocation-free batched solve.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library call cudaMalloc -- a
 * framework whose own memory pool already holds the device memory, or a
 * latency-critical loop that must not pay the device-wide synchronisation of
 * growing trid_solve_batch's scratch pool.
 *
 * Same arguments and results as trid_solve_batch.  Long systems that the
 * one-pass kernels do not take need scratch (trid_solve_workspace_bytes);
 * here it comes from one fixed device array of TRID_NOALLOC_SCRATCH_BYTES
 * (32 MiB) that the library holds on every GPU that loads it, until the
 * process exits.  The call never allocates or frees device memory.
 *   - Problems needing more scratch than TRID_NOALLOC_SCRATCH_BYTES are
 *     rejected with TRID_ERR_ALLOC before anything is launched (use
 *     trid_solve_batch_ws with your own buffer for those).
 *   - The first call on a device that needs scratch looks up the array's
 *     device address (cudaGetSymbolAddress); make that first call before any
 *     stream capture.
 *   - Every call on a device shares the one array.  Calls whose work overlaps
 *     on the GPU (different streams, no ordering between them) race on it and
 *     may return wrong results; order them, e.g. issue them on one stream.
 *   - The array keeps the last call's contents; the solve overwrites every
 *     scratch value before reading it, so nothing needs clearing.
 *   - The array's device address is cached per device; after a
 *     cudaDeviceReset it would be stale, so call trid_finalize (which forgets
 *     it) before resetting a device.
 */
#define TRID_NOALLOC_SCRATCH_BYTES (32u << 20)
trid_status trid_solve_batch_noalloc(const void *a, const void *b, const void *c, void *d,
                                     void *u, const int64_t *dims, int ndim, int solve_dim,
                                     trid_dtype dtype, trid_stream_t stream);

/*
 * ADI heat-diffusion time steps, Section 4.1, Algorithm "adi": per step,
 * d = lambda * (sum of the 2*ndim axis neighbours of u - 2*ndim*u) on interior
 * nodes (0 on boundary nodes); d <- X^{-1} d; d <- Y^{-1} d; [d <- Z^{-1} d;]
 * u <- u + d.  Each directional operator is tridiag(-lambda, 1 + 2 lambda,
 * -lambda) on interior rows with identity rows at the two Dirichlet-zero
 * boundary nodes; the coefficients are generated inside the kernels and never
 * stored (Section 4.1: coefficient generation fused with the solver).
 *
 *   u          device array of prod(dims) elements, advanced in place by
 *              `nsteps` steps.  Boundary nodes must hold 0 and are left 0.
 *   dims       host int64 extents, ndim in {2, 3}, every extent >= 3.
 *   lambda     diffusion number, > 0.
 *   workspace  caller-owned device scratch of at least
 *              adi_workspace_bytes(dims, ndim, dtype) bytes, 256-byte aligned.
 */
trid_status adi_step(void *u, const int64_t *dims, int ndim, double lambda, int nsteps,
                     trid_dtype dtype, void *workspace, size_t workspace_bytes,
                     trid_stream_t stream);

/* Scratch size adi_step needs: one mesh-sized array (the intermediate d of
 * the two-pass schedule) plus alignment.  0 for invalid arguments. */
size_t adi_workspace_bytes(const int64_t *dims, int ndim, trid_dtype dtype);

/*
 * Device status word: kernels that run a bounded wait, or that meet an
 * invalid entry in a device-side argument (varlen offsets), record the first
 * failure here instead of trapping.  In the debug build (compiled with
 * TRID_DEBUG_BOUNDS) the index checks of the hot kernels (line solves, strided
 * solves, both passes of the windowed ADI step) also record
 * TRID_ERR_INVALID_ARG, having skipped the out-of-range access.  This call
 * synchronises `stream`, returns TRID_OK or the first recorded failure
 * (TRID_ERR_TIMEOUT, TRID_ERR_INVALID_ARG) and clears the word(s).
 */
trid_status trid_get_device_status(trid_stream_t stream);

/*
 * Bounded wait on a device flag (diagnostic; not in the paper): one thread
 * waits on `stream` until the device int *flag equals `expect` or timeout_s
 * seconds (0 < timeout_s <= 1) of device time have passed; on expiry it
 * records TRID_ERR_TIMEOUT in the device status word and returns, the same
 * way the TMA-fed kernels give up on an mbarrier.  Lets a caller check the
 * bounded-wait path without a hang or a fault.  Errors: TRID_ERR_INVALID_ARG
 * (NULL flag, timeout outside (0, 1]), TRID_ERR_MISALIGNED, TRID_ERR_CUDA.
 */
trid_status trid_wait_flag(const int *flag, int expect, double timeout_s, trid_stream_t stream);

/*
 * Length classes, tile height and team size of trid_solve_batch_varlen.  Every thread
 * holds tiles of tile_rows consecutive rows (M = 8, or 16 in FP32; 0 means 8).
 * Systems of up to 32 M - M rows are solved by one warp each, up to team_max
 * rows by a team of 4 warps, up to block_max rows by a whole block (512
 * threads) in one pass, and longer ones by a block in two passes.  With M = 8:
 * team_max is 248 (no team class), 504 or 1016; block_max is team_max (no
 * one-pass block class) or one of 1016, 2040, 4088 not below team_max.  With
 * M = 16 every limit doubles plus 8 (team_max 496, 1008 or 2032; block_max
 * team_max or one of 2032, 4080, 8176).  team_warps is the size of a team:
 * 4 warps (0 means 4; 4 systems in flight per block) or, when team_max is
 * 64 M - M (504 or 1008), 2 warps (8 systems in flight per block).
 * Defaults (trid_solve_batch_varlen): M 8, team_max 1016, block_max 4088,
 * teams of 4 warps.  A caller zero-initialises the struct and sets the fields
 * it uses.  Not a construct of the paper (its FPGA batches are uniform).
 */
typedef struct {
    int32_t team_max;
    int32_t block_max;
    int32_t tile_rows;
    int32_t team_warps;
} trid_varlen_config;

/* trid_solve_batch_varlen with explicit length classes (cfg == NULL: the
 * defaults); TRID_ERR_INVALID_ARG for a configuration outside the list above. */
trid_status trid_solve_batch_varlen_cfg(const void *a, const void *b, const void *c, void *d,
                                        void *u, const int64_t *offsets, int64_t nsys,
                                        int64_t total, int64_t max_len, trid_dtype dtype,
                                        void *workspace, size_t workspace_bytes,
                                        trid_stream_t stream, const trid_varlen_config *cfg);

/* Autotuner: solves the caller's batch once per admissible configuration
 * (every tile height, class split and team size above; tile height 16 in
 * FP32 only) (on
 * a scratch copy of d inside `workspace`; a, b, c, d are not modified), times
 * each with CUDA events on `stream` (best of three after one warm-up run) and
 * writes the fastest to *best (and its time in ms to *best_ms if not NULL).
 * Synchronises `stream`.  workspace: trid_varlen_autotune_workspace_bytes
 * bytes, 256-byte aligned.  Errors as trid_solve_batch_varlen. */
size_t trid_varlen_autotune_workspace_bytes(int64_t nsys, int64_t total, trid_dtype dtype);
trid_status trid_varlen_autotune(const void *a, const void *b, const void *c, const void *d,
                                 const int64_t *offsets, int64_t nsys, int64_t total,
                                 int64_t max_len, trid_dtype dtype, void *workspace,
                                 size_t workspace_bytes, trid_stream_t stream,
                                 trid_varlen_config *best, float *best_ms);

/*
 * ADI steps on a batch of meshes (Section 4.1, Algorithm "adi"; the batched
 * 2D / 3D workloads of Section 4).  u holds nbatch meshes of dims[0] x ...
 * x dims[ndim-1] points (ndim 2 or 3, every extent 3..256), mesh b starting
 * at element b * (product of dims), each column-major (x contiguous); every
 * mesh advances by nsteps steps exactly as with adi_step.  When a mesh and its
 * right-hand side fit one block's shared memory, all nsteps steps run in one
 * kernel with the mesh resident on chip (read and written once per call);
 * otherwise 3D meshes whose extents suit the two-pass 3D schedule (all
 * multiples of 16, z >= 32) run stacked along z through its kernels, and the
 * rest go through adi_step one after another.  `workspace` (256-byte
 * aligned) must hold adi_batched_workspace_bytes(nbatch, dims, ndim, dtype)
 * bytes (0 in the resident case, where workspace may be NULL).  Errors as
 * adi_step; asynchronous on `stream`.
 */
size_t adi_batched_workspace_bytes(int64_t nbatch, const int64_t *dims, int ndim,
                                   trid_dtype dtype);
trid_status adi_step_batched(void *u, int64_t nbatch, const int64_t *dims, int ndim,
                             double lambda, int nsteps, trid_dtype dtype, void *workspace,
                             size_t workspace_bytes, trid_stream_t stream);

/*
 * Differentiable 2D ADI with a diffusivity field (reverse mode of the ADI step
 * of Section 4.1 with checkpointing; the paper has no variable-coefficient
 * form).  Mesh dims[0] x dims[1], column-major (x contiguous), both >= 3.
 * Face diffusivities are node means, kx_p = (kappa_p + kappa_{p+1}) / 2, and
 * on rows 0 < i < nx-1 the x operator is a_p = -lambda kx_{p-1},
 * c_p = -lambda kx_p, b_p = 1 - a_p - c_p (identity rows at the line ends; y
 * alike).  One step: d = explicit part -c_p (u_{p+1} - u_p) + a_p (u_p -
 * u_{p-1}) + (y terms) on the interior, 0 on the boundary; u += Y^{-1} X^{-1} d.
 *
 * adi2v_forward: uT = u0 after nsteps steps (uT may equal u0).  If ckpt is
 *   not NULL it receives u every `every` steps (u0 first), in slots of
 *   adi2v_checkpoint_bytes / ceil(nsteps / every) bytes; keep it for the
 *   backward call.
 * adi2v_backward: from g_uT = dL/du_T, writes g_u0 = dL/du_0 and
 *   g_kappa = dL/dkappa, and, if g_coef is not NULL, the gradients with
 *   respect to the six coefficient arrays (ax, bx, cx, ay, by, cy; 6 packed
 *   mesh arrays) summed over the steps.  Each segment between checkpoints is
 *   recomputed forward, then run in reverse with solves of the transposed
 *   operators (the adjoint solves of trid_solve_batch_adjoint).  With two or
 *   more segments the recomputation runs on the library's auxiliary stream
 *   of the device, ordered against `stream` by events, so that segment s - 1
 *   is recomputed while segment s runs in reverse; every piece of work is
 *   ordered before the call's last operation on `stream`.  The auxiliary
 *   stream is shared: calls from several host threads at once serialise on
 *   it, and two stream captures must not include such calls at the same time.
 * Arrays are device arrays of dims[0] * dims[1] elements of `dtype`; outputs
 * must not alias inputs.  workspace (256-byte aligned) of at least
 * adi2v_workspace_bytes(dims, nsteps, every, dtype) bytes, ckpt 256-byte
 * aligned.  Errors: TRID_ERR_INVALID_ARG (bad dims, nsteps < 0, every < 1,
 * lambda <= 0, NULL arrays), TRID_ERR_ALLOC (workspace or ckpt too small),
 * TRID_ERR_MISALIGNED, TRID_ERR_CUDA.  Asynchronous on `stream`.
 */
size_t adi2v_workspace_bytes(const int64_t *dims, int nsteps, int every, trid_dtype dtype);
size_t adi2v_checkpoint_bytes(const int64_t *dims, int nsteps, int every, trid_dtype dtype);
trid_status adi2v_forward(const void *u0, void *uT, const void *kappa, const int64_t *dims,
                          double lambda, int nsteps, int every, void *ckpt, size_t ckpt_bytes,
                          trid_dtype dtype, void *workspace, size_t workspace_bytes,
                          trid_stream_t stream);
trid_status adi2v_backward(const void *g_uT, void *g_u0, void *g_kappa, void *g_coef,
                           const void *kappa, const int64_t *dims, double lambda, int nsteps,
                           int every, const void *ckpt, size_t ckpt_bytes, trid_dtype dtype,
                           void *workspace, size_t workspace_bytes, trid_stream_t stream);

/*
 * Measured FP64 rates of the current device (diagnostic; not a construct of
 * the paper).  On GB300 the FP64 solves are bound by FP64 arithmetic, not by
 * HBM; their roofline is taken against these rates.  Times, with CUDA events
 * on `stream`, a grid filling every SM with independent chains of fused
 * multiply-adds and one of IEEE divisions, and writes the sustained rates in
 * 10^9 operations per second (an FMA counts as one operation).  Allocates
 * nothing; synchronises `stream`, so not for use inside a stream capture.  Errors: TRID_ERR_INVALID_ARG (NULL outputs),
 * TRID_ERR_CUDA.
 */
trid_status trid_fp64_rates(double *fma_gops, double *div_gops, trid_stream_t stream);

/* Library version string (static storage). */
const char *trid_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TRID_H_ */
