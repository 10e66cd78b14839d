/*
 * hh.h -- C-ABI of the GB300 H_h-matrix library.
 *
 * The library builds a hybrid hierarchical matrix (H_h) of a kernel matrix
 * H_ij = f(|x_i - x_j|) (Khan & Carson, Eq. 5.1) with hybrid admissibility
 * (Eq. 3.1: standard admissibility on levels 1..ell, the remaining
 * off-diagonal pairs compressed at level ell, weak admissibility below, dense
 * blocks only on the leaf diagonal; Algorithm 1), stores every admissible
 * block U_b V_b^T in the precision chosen by the adaptive rule of Algorithm 3
 * (u_b <= eps / (2^{l/2} xi_b), xi_b = ||H~_b||_F / ||H~||_F), and applies it:
 * b = H_hat x (Algorithm 4) and the transpose product, on one GPU.
 *
 * Conventions for every entry point:
 *  - Return value: HH_OK (0) on success, a negative HH_E* code otherwise; the
 *    thread-local message of the last failure is returned by hh_last_error().
 *  - Vectors are column-major (n x nrhs, leading dimension ld >= n) float64
 *    arrays in the caller's point order; device pointers unless stated.
 *    The caller owns them; the library never frees or keeps them.
 *  - Matrix-vector calls are asynchronous on the given cudaStream_t (NULL =
 *    the legacy default stream) and never synchronise, allocate or copy to the
 *    host (except the first tensor-core call of a handle in each direction,
 *    which allocates its workspace and packs its operand panels, and
 *    hh_matvec_host / hh_matvec_timed, which synchronise);
 *    they overwrite the output (no accumulation).  Input and output must
 *    not overlap.
 *  - A handle owns its host metadata and device arenas; it is immutable after
 *    construction.  hh_matvec / hh_matvec_T use a per-handle workspace, so
 *    calls on one handle must be ordered on a single stream; use
 *    hh_matvec_ws with caller-owned workspaces for concurrent streams.
 *  - Device-side anomalies (an invalid descriptor) are recorded in a device
 *    status word and reported by hh_sync_status(); the kernels never trap,
 *    every wait inside a block has a clock limit, and no kernel waits on
 *    other blocks except the batch product's cooperative kernel, whose grid
 *    barriers span one co-resident launch (hh_batch_matvec).
 */
#ifndef HH_H_
#define HH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HH_OK 0
#define HH_EINVAL (-1)   /* invalid argument, size or file content           */
#define HH_ENOMEM (-2)   /* host or device allocation failed                 */
#define HH_ECUDA (-3)    /* a CUDA runtime call failed                        */
#define HH_ETIMEOUT (-4) /* reserved: a bounded device wait gave up           */
#define HH_ENOTSUP (-5)  /* valid but unsupported request (e.g. no device)    */
#define HH_EIO (-6)      /* file could not be read or written                 */
#define HH_EDEVICE (-7)  /* the device status word reports an anomaly         */

/* kernel functions f(r) (Section 5; r = |x_i - x_j|_2, p = kernel_param) */
enum hh_kernel {
  HH_EXP = 0,    /* exp(-r/p)                 (Matern)                        */
  HH_INV_R = 1,  /* 1/r,   f = 0 at r = 0     (3-D single-layer Laplace)      */
  HH_GAUSS = 2,  /* exp(-r^2/p)               (Gaussian)                      */
  HH_LOG = 3,    /* log r, f = 0 at r = 0     (2-D single-layer Laplace)      */
  HH_INV_R2 = 4  /* 1/r^2, f = 0 at r = 0                                     */
};

/* storage formats (Table 1; fp8 e4m3fn stands for the paper's 1-4-3 format) */
enum hh_fmt { HH_FMT_F64 = 0, HH_FMT_F32 = 1, HH_FMT_F16 = 2, HH_FMT_BF16 = 3, HH_FMT_E4M3 = 4 };
/* fmt_mask bits: the set U of available precisions; fp64 is always available */
#define HH_F64 1u
#define HH_F32 2u
#define HH_F16 4u
#define HH_BF16 8u
#define HH_E4M3 16u
/* fmt_mask option: Algorithm 3's rule takes the 8-bit format's unit roundoff
 * as printed in Table 1 (2.5e-1) instead of e4m3's 2^-4, so it picks the
 * 8-bit format only where tau_b >= 1/4; storage, decoding and the error
 * bounds keep 2^-4.  Not a format: combine with HH_E4M3. */
#define HH_RULE_Q43 32u

typedef struct hh_matrix* hh_handle;
typedef struct hh_batch_s* hh_batch;

#define HH_MAX_LEVELS 48

/* Summary of a built matrix (storage in fp64 words as in Section 5.2). */
typedef struct {
  int64_t n;                      /* matrix size N                                   */
  int32_t dim, L, ell, leaf_size; /* point dimension, tree depth, switch level, n_max */
  int32_t kernel, device;         /* hh_kernel; CUDA device or -1 (host only)         */
  double eta, tol, kernel_param;
  int64_t n_lowrank, n_dense;     /* number of admissible / dense blocks             */
  int64_t blocks_per_fmt[5];      /* admissible blocks per hh_fmt                    */
  int64_t factor_bytes_per_fmt[5];/* bytes of U and V per hh_fmt (algorithmic)       */
  int64_t dense_bytes;            /* bytes of the fp64 dense blocks                  */
  int64_t u_bytes, v_bytes;       /* bytes of all U factors / all V factors          */
  int64_t max_rank;
  double storage_amp;             /* sum p(m+n) b/64 + sum m n   (adaptive)          */
  double storage_fp64;            /* the same with every block in fp64               */
  double bytes_per_matvec;        /* algorithmic bytes of one single-RHS product     */
  double flops_per_matvec;        /* 2 (sum p(m+n) + sum m n)                        */
  double norm_ht;                 /* ||H~||_F (Algorithm 5)                          */
  int32_t csp[HH_MAX_LEVELS];     /* measured sparsity constant C_sp(l), l = 0..L    */
  double bound_thm42;             /* (2 sqrt(sum_l C_sp(l)) + 1) eps (Theorem 4.2)   */
  double bound_thm44;             /* 2 * bound_thm42 (Theorem 4.4, backward error)   */
  double bound_rounding;          /* sqrt(sum_b ((2+sqrt(p)u)u||H~_b||)^2)/||H~||    */
  double build_seconds;           /* wall time of hh_build (0 for hh_load)           */
  int64_t tc_blocks;              /* admissible blocks the tensor-core path takes    */
  int64_t tc_factor_bytes;        /* their factor bytes                              */
  int64_t tc_u_elems, tc_v_elems; /* their U and V elements (sum m k, sum n k)        */
  int64_t mr_u_elems, mr_v_elems; /* the same for the 32/16/8-bit blocks that the
                                     many-right-hand-side path runs on CUDA cores  */
  int64_t dense_elems;            /* entries of the dense blocks                     */
  int32_t tuned;                  /* 1 after hh_autotune                             */
  int32_t split_positions;        /* positions of a many-column phase-1 item         */
  int32_t blocks_per_sm[4];       /* streaming CTAs per SM chosen by hh_autotune:
                                     {fwd phase 1, fwd phase 2, T phase 1, T phase 2};
                                     0 = the occupancy maximum                       */
  int64_t tc_panel_bytes[2];      /* device bytes held by the tensor-core operand
                                     panels {forward, transpose} (factor slices and
                                     dense-block digits): 0 until the first
                                     tensor-core product in that direction packs
                                     them                                           */
  int32_t tree_step;              /* binary levels per tree level: 1 for the KD tree,
                                     d for the 2^d-tree (L, ell, csp are binary)   */
  int32_t pad_;
  int32_t build_device;           /* GPU that compressed the blocks (hh_build_dev), -1: the host */
  int32_t pad2_;
  int64_t build_fallback;         /* blocks of a device build that the host compressed        */
  double build_device_seconds;    /* wall time of the device compression                       */
  int32_t stream_depth[4];        /* pipeline depth (stages per CTA) of one-column streaming
                                     launches per [direction][phase] (hh_autotune; default 4)  */
  int64_t item_bytes;             /* factor bytes of a streaming phase-1 item (hh_autotune)     */
  int64_t dense_tc_elems;         /* operand elements of the dense blocks on the tensor cores
                                     in the forward direction: 128 rows x 16 positions per
                                     k-step of every tile entry (padding included)             */
} hh_info_t;

/*
 * hh_build -- construct A_h from points (Algorithms 1, 5 and 3).
 *   points       host, n x dim row-major float64 (user order); read only.
 *   n, dim       n >= 1, 1 <= dim <= 3.
 *   kernel       hh_kernel; kernel_param > 0 is p of exp(-r/p) / exp(-r^2/p).
 *   leaf_size    n_max >= 1: leaves hold at most this many points; the tree is
 *                a binary KD bisection of depth L = ceil(log2(n / n_max)).
 *   eta          admissibility parameter of Eq. 2.2 (> 0).
 *   switch_level ell in [0, L]; -1 selects floor(L/2).  ell = L gives an H_s
 *                matrix, ell = 0 a HODLR matrix.  ell > L -> HH_ENOTSUP.
 *   tol          target accuracy eps of LRcompression (0 < tol < 1).
 *   fmt_mask     HH_F64|HH_F32|... the set U of Algorithm 3; HH_F64 alone
 *                gives uniform fp64 storage; | HH_RULE_Q43 for the rule's
 *                Table 1 reading of the 8-bit format.  Other bits: HH_EINVAL.
 *   seed         recorded in saved files; the build itself is deterministic.
 *   device       CUDA device to upload to, or -1 for a host-only handle
 *                (hh_save / hh_info work; matrix-vector calls return
 *                HH_ENOTSUP).
 *   out          receives the new handle (NULL on failure).
 * Host-synchronous; uses all host cores (HH_BUILD_THREADS overrides).
 */
int hh_build(const double* points, int64_t n, int dim, int kernel, double kernel_param,
             int leaf_size, double eta, int switch_level, double tol, uint32_t fmt_mask,
             uint64_t seed, int device, hh_handle* out);

/* cluster trees (hh_build_ex) */
enum hh_tree {
  HH_TREE_KD = 0,  /* binary KD bisection at the median of the widest axis  */
  HH_TREE_2D = 1   /* balanced 2^d-tree (quad-tree in 2-D, oct-tree in 3-D) */
};

/* hh_build_ex -- hh_build with a choice of cluster tree (Section 2.1).
 *   tree   HH_TREE_KD: as hh_build.  HH_TREE_2D: the geometrically balanced
 *          2^d-tree of the paper: the root is the smallest axis-aligned
 *          hypercube around the points, every cell is split into its 2^d
 *          sub-cubes (a point on a splitting plane goes to the upper cell),
 *          depth the smallest L with ceil(n / 2^{dL}) <= leaf_size; cells
 *          may be empty.  switch_level counts 2^d-tree levels (-1:
 *          floor(L/2)); eta = sqrt(d) is the paper's choice.
 * The 2^d-tree is held as a binary tree whose level b halves its cells along
 * axis b mod d, so hh_info's L and ell and the block levels of hh_save's
 * file are binary levels (d per tree level; the file records d).  Other
 * arguments and errors as hh_build. */
int hh_build_ex(const double* points, int64_t n, int dim, int kernel, double kernel_param,
                int leaf_size, double eta, int switch_level, double tol, uint32_t fmt_mask,
                uint64_t seed, int tree, int device, hh_handle* out);

/* hh_build_dev -- hh_build_ex with Algorithm 1's LRcompression (Eq. 2.1) of
 * every admissible block run on GPU `device` (>= 0), which also receives the
 * matrix.  Per block, in fp64: ACA with partial pivoting to eps / 100 (the
 * entries of Eq. 5.1 generated from the points on the device), CholeskyQR2
 * of both cross factors, the one-sided Jacobi SVD of the k x k core and the
 * truncation of the Frobenius tail at 0.99 eps (U orthonormal, V = Z Sigma,
 * as the host path).  Blocks whose rank would exceed 2,048 columns, or whose
 * factorization fails, are compressed on the host (hh_info.build_fallback).
 * The tree, the partition, Algorithm 5's norms, Algorithm 3's rule and the
 * arena are as in hh_build_ex, so the result differs from it only by the
 * compression's rounding (ranks within a few units, formats alike).
 * Host-synchronous; errors as hh_build_ex, HH_ECUDA for a device failure. */
int hh_build_dev(const double* points, int64_t n, int dim, int kernel, double kernel_param, int leaf_size,
                 double eta, int switch_level, double tol, uint32_t fmt_mask, uint64_t seed, int tree, int device,
                 hh_handle* out);

/* hh_load -- read a file written by hh_save (or by any writer of the same
 * documented layout) and upload it to `device` (-1: host only).  The layout
 * is validated (offsets, alignment, bounds); a bad file gives HH_EINVAL. */
int hh_load(const char* path, int device, hh_handle* out);

/* hh_reencode -- apply Algorithm 3 again to a matrix stored in uniform fp64
 * (every factor fp64, as hh_build with fmt_mask = HH_F64 produces) with the
 * format set fmt_mask, reusing its tree, partition, compression and norms
 * (||H~_b||, ||H~||): the result equals hh_build with that mask.  ell == L
 * gives HH_ENOTSUP (there the dense/low-rank choice of leaf neighbours
 * depends on the format, Section 4.3); a non-uniform source HH_EINVAL.
 * The new handle is independent of src and uploaded to `device` (-1: none). */
int hh_reencode(hh_handle src, uint32_t fmt_mask, int device, hh_handle* out);

/* hh_optimal_switch_level -- Algorithm 2: the switching level ell* whose H_h
 * matrix gains the most storage over the H_s matrix (standard admissibility
 * down to the leaves, ell = L).  The two storages share the far-field blocks
 * of levels 1..ell and the dense diagonal (Section 3.3), so the gain of a
 * level is S_1(ell) - S_2(ell) = S_s - S_h(ell), counted in fp64 words with
 * every low-rank block at its assigned format's bits (Section 5.2's count;
 * with fmt_mask = HH_F64 the uniform-precision gain).  Starting at ell = L
 * (gain 0) the algorithm moves to ell - 1 while the gain grows strictly and
 * stops at the first level whose gain does not.
 *   points ... seed   as for hh_build (switch_level is what is searched).
 *   tree              HH_TREE_KD or HH_TREE_2D (levels are then tree levels).
 *   ell_star          receives ell*.
 *   depth             receives L in tree levels (may be NULL).
 *   gains             NULL or HH_MAX_LEVELS doubles: gains[l] = S_s - S_h(l)
 *                     for each tree level evaluated, NaN for the others.
 * Host-synchronous and host-only: one construction (Algorithm 1, 5, 3) per
 * evaluated level.  A block's compression depends only on its two clusters
 * and tol, so the evaluated levels share them: each block is compressed once,
 * and the search holds every compressed block in fp64 in host memory until it
 * returns (about the fp64 storage of the H_s matrix plus the near-field
 * blocks of the levels evaluated).  HH_EINVAL for bad arguments or a tree
 * deeper than HH_MAX_LEVELS - 1. */
int hh_optimal_switch_level(const double* points, int64_t n, int dim, int kernel, double kernel_param,
                            int leaf_size, double eta, double tol, uint32_t fmt_mask, uint64_t seed, int tree,
                            int* ell_star, int* depth, double* gains);

/* hh_optimal_switch_level_dev -- hh_optimal_switch_level with the
 * compressions of every evaluated level on GPU `device` (as hh_build_dev). */
int hh_optimal_switch_level_dev(const double* points, int64_t n, int dim, int kernel, double kernel_param,
                                int leaf_size, double eta, double tol, uint32_t fmt_mask, uint64_t seed, int tree,
                                int device, int* ell_star, int* depth, double* gains);

/* hh_shard_plan -- ownership of the product's block rows by nranks ranks
 * (one GPU each).  In Algorithm 4 (Section 4.4) every block row
 * b_I = sum_J H_IJ x_J is independent of the others, so the rows split into
 * contiguous ranges of tree positions: bounds[0] = 0 <= bounds[1] <= ... <=
 * bounds[nranks] = n (nranks + 1 int64, caller-owned, host), rank r owning
 * [bounds[r], bounds[r+1]).  The ranges are unions of consecutive clusters of
 * tree level min(L, ceil(log2 nranks) + 3), balanced by the factor and dense
 * bytes their rows stream (a block cut by a boundary counts its U rows to
 * their owner and a row share of its V to each).  Host-only, deterministic;
 * HH_EINVAL for a null handle or bounds, or nranks < 1. */
int hh_shard_plan(hh_handle h, int nranks, int64_t* bounds);

/* hh_shard -- the matrix of block rows [p0, p1) (tree positions, p0 and p1
 * from hh_shard_plan or any cluster boundaries) as a handle of its own on
 * `device` (-1: host only): every low-rank block whose row cluster meets the
 * range, cut to those rows (U's rows, V whole, factors copied into a compact
 * arena, formats and scales unchanged), and the dense blocks inside the
 * range.  Its point order IS the tree order (identity permutation): hh_matvec
 * on it takes all of x in tree order and returns y in tree order, exact in
 * [p0, p1) and zero elsewhere; hh_matvec_T reads only rows [p0, p1) of
 * y_bar and returns this range's contribution to all of x_bar (the sum over
 * the ranks' shards is A_h^T y_bar).  The shard is independent of h.
 * HH_EINVAL if the range lies outside [0, n] or cuts a dense block. */
int hh_shard(hh_handle h, int64_t p0, int64_t p1, int device, hh_handle* out);

/* hh_save -- write the handle's matrix (points, tree, block tables, factor
 * arena in stored formats, dense blocks) to `path`. */
int hh_save(hh_handle h, const char* path);

/* hh_info -- fill *out with sizes, storage, bounds (Theorems 4.2 / 4.4). */
int hh_info(hh_handle h, hh_info_t* out);

/* hh_perm -- copy the tree permutation (perm[p] = user index of tree
 * position p) into the host array perm[n]. */
int hh_perm(hh_handle h, int32_t* perm);

/*
 * hh_matvec -- y = A_h x (Algorithm 4), nrhs right-hand sides.
 *   x  device, n x nrhs, leading dimension ldx >= n;  y device, ldy >= n.
 *   nrhs >= 1 (any number).
 *   stream  cudaStream_t (as void*).
 * Arithmetic: 32-, 16- and 8-bit low-rank blocks are upcast to fp32 and
 * accumulated in fp32 (the input split into fp32 leading and trailing
 * halves); fp64 low-rank blocks and the dense blocks are computed as pairs
 * of fp32 halves (about 2^-48 relative, the fp64 path's 1e-12 parity); the
 * output is accumulated in fp64.  With nrhs <= 4 the columns go through the
 * streaming passes (one launch sequence for 1, 2 or 4 columns).  With
 * nrhs >= 5 (measured crossover: the many-column sequence costs about the
 * same for 5 to 32 columns as the streaming passes for 5; HH_TC_MIN_NRHS in
 * the environment overrides, 0 disables) the columns go in chunks of up to
 * 128 through one pass over the blocks: the fp32, fp16, bf16 and e4m3 blocks
 * whose clusters start at multiples of 16 on the tensor cores (exact bf16
 * slices of the factors and of the fp32 input; products kept down to about
 * 2^-24 for fp32 blocks and below the unit roundoff of the 16- and 8-bit
 * formats; fp32 accumulation drained into round-to-nearest registers every
 * 64 terms for fp32 blocks, every 512 for the others), the other 32/16/8-bit
 * blocks on CUDA-core fp32 kernels, the dense blocks on the tensor cores as
 * six exact 8-bit digits of their fp32-pair entries and of the input (one
 * power of two per row and per right-hand side; digit products summed
 * exactly, about 2^-45 of sum |H||x|), the fp64 low-rank blocks on the
 * streaming passes.  The first such call in each
 * direction allocates the tensor-core workspace and the factor panels packed
 * for the tensor cores (hh_info tc_panel_bytes; an implicit device
 * synchronisation; HH_ENOMEM if they cannot be allocated).  Uses the
 * handle's workspaces.
 */
int hh_matvec(hh_handle h, const double* x, double* y, int nrhs, int64_t ldx, int64_t ldy,
              void* stream);

/* hh_matvec_T -- xbar = A_h^T ybar: every block applied transposed
 * (V_b (U_b^T ybar_I), H_IJ^T ybar_I).  Same argument rules as hh_matvec. */
int hh_matvec_T(hh_handle h, const double* ybar, double* xbar, int nrhs, int64_t ldy,
                int64_t ldx, void* stream);

/* hh_solve_cg -- conjugate gradients (Hestenes-Stiefel) for
 * (A_h + shift I) x = b: the fast iterative solver the product enables
 * (Section 5, end).  Meant for symmetric positive definite kernels (exp(-r),
 * Gaussian), whose A_h is symmetric up to the compression tolerance.
 *   b       device, n (caller's order); not modified.
 *   x       device, n: the initial guess on entry, the solution on return.
 *   shift   added to the diagonal (0 for A_h itself).
 *   rtol    stop when ||r_k|| <= rtol ||b|| (recursively updated residual).
 *   max_iter, iters, relres   iteration cap; iterations done and the final
 *           ||r|| / ||b|| (either pointer may be NULL).
 * Each iteration is one forward product (the streaming passes, on the
 * handle's workspace), two dot products and two vector updates; the scalars
 * (alpha, beta, the convergence and breakdown tests) stay on the device and
 * the host reads them every 8 iterations (iterations past the stop change
 * nothing, so results and counts are those of testing every iteration).
 * The call synchronises `stream`; three n-vectors are allocated for it. 
 * HH_EINVAL if b and x overlap or the iteration breaks down
 * (p^T (A_h + shift I) p <= 0: not positive definite). */
int hh_solve_cg(hh_handle h, const double* b, double* x, double shift, double rtol, int max_iter,
                int* iters, double* relres, void* stream);

/* hh_workspace_bytes -- bytes of device workspace hh_matvec_ws needs. */
int hh_workspace_bytes(hh_handle h, size_t* bytes);

/* hh_matvec_ws -- hh_matvec (transpose != 0: hh_matvec_T) with a
 * caller-owned device workspace of at least hh_workspace_bytes() bytes,
 * 256-byte aligned; concurrent calls with distinct workspaces are safe.
 * Every nrhs goes through the streaming passes (no tensor-core path). */
int hh_matvec_ws(hh_handle h, int transpose, const double* in, double* out, int nrhs,
                 int64_t ld_in, int64_t ld_out, void* workspace, size_t workspace_bytes,
                 void* stream);

/* hh_matvec_host -- end-to-end product from HOST buffers: copies x (n x nrhs,
 * ld = n, pinned or pageable) to the device, applies A_h (or A_h^T when
 * transpose != 0), copies the result to y_host and synchronises `stream`. */
int hh_matvec_host(hh_handle h, int transpose, const double* x_host, double* y_host, int nrhs,
                   void* stream);

/* hh_matvec_timed -- one product (transpose != 0: A_h^T) through the
 * streaming passes with CUDA events recorded on `stream` between its four
 * launches; synchronises the stream and writes the device time in ms of each
 * launch to ms[4] = {prep, phase 1 (t_b = V_b^T x), phase 2 (y += U_b t_b and
 * dense blocks), finish}.  nrhs must be 1, 2 or 4 (one launch sequence).  For
 * measurement; uses the handle's workspace. */
int hh_matvec_timed(hh_handle h, int transpose, const double* in, double* out, int nrhs,
                    int64_t ld_in, int64_t ld_out, void* stream, float* ms);

/* hh_autotune -- choose launch parameters by timing them on the device
 * (CUDA events, a private stream, temporary buffers of 2 n max(4, nrhs_many)
 * doubles): the CTAs per SM of each streaming pass (1 .. occupancy maximum,
 * per direction and phase) and, when nrhs_many > 0, the positions per
 * many-column phase-1 item ({1024, ..., 65536}) for products of nrhs_many
 * columns.  The choices stay in the handle (hh_info reports them); results
 * of products do not depend on them beyond rounding.  Synchronous; not
 * concurrent with products on the same handle. */
int hh_autotune(hh_handle h, int nrhs_many);

/* hh_matvec_stages -- one product of 1 <= nrhs <= 128 right-hand sides
 * through the many-right-hand-side sequence (whatever nrhs), with CUDA events
 * around each launch; synchronises and writes ms[8] = {input images, dense
 * blocks (input digits and the tensor-core kernel), streaming passes over the
 * fp64 low-rank blocks, CUDA-core phase 1, tensor-core phase 1, CUDA-core
 * phase 2, tensor-core phase 2, output permutation}.  For measurement; uses
 * the handle's workspaces. */
int hh_matvec_stages(hh_handle h, int transpose, const double* in, double* out, int nrhs,
                     int64_t ld_in, int64_t ld_out, void* stream, float* ms);

/* hh_matvec_batched -- y_i = A_i x_i for `count` independent matrices (one
 * right-hand side each, ld = n_i) in one launch sequence over the
 * concatenated work lists.  All handles must live on the same device. */
int hh_matvec_batched(const hh_handle* hs, int count, const double* const* xs,
                      double* const* ys, void* stream);

/* Batches of independent matrices (one right-hand side each) in one launch.
 * The product of every matrix is Algorithm 4 as above; the batch only
 * concatenates the work tables, so one product of the whole batch is one
 * persistent cooperative kernel (prep, phase 1, phase 2 and finish separated
 * by grid-wide barriers, one co-resident CTA set) whatever the count.  Where
 * the device has no cooperative launch, or HH_BATCH_LAUNCHES=4 is set when
 * the batch is created, it is four launches (prep, phase 1, phase 2,
 * finish).
 *
 * hh_batch_create -- a batch over `count` >= 1 handles on one device.  The
 *   handles must stay alive (not hh_free'd) while the batch exists.  Allocates
 *   the batch's tables and workspace (about 40 bytes per point plus the t
 *   arenas); HH_ENOTSUP for a handle without device data, HH_EINVAL for
 *   handles on different devices or more than 2^31 positions in total.
 * hh_batch_offsets -- offsets[count + 1]: matrix i's vector occupies
 *   [offsets[i], offsets[i + 1]) of the concatenated input and output (its n
 *   entries in its own point order).
 * hh_batch_matvec -- y = blockdiag(A_i) x (transpose != 0: the transposes)
 *   for concatenated device vectors x and y (no overlap); asynchronous on
 *   `stream`; allocates nothing, so it may be captured in a CUDA graph; calls
 *   on one batch must be ordered on one stream (one workspace).
 * hh_batch_matvec_graph -- the same through a CUDA graph that the batch
 *   captures on first use (and again when x, y or transpose change) and then
 *   replays on `stream` with one graph launch.
 * hh_batch_free -- NULL-safe. */
int hh_batch_create(const hh_handle* hs, int count, hh_batch* out);
int hh_batch_offsets(hh_batch b, int64_t* offsets);
int hh_batch_matvec(hh_batch b, int transpose, const double* x, double* y, void* stream);
int hh_batch_matvec_graph(hh_batch b, int transpose, const double* x, double* y, void* stream);
void hh_batch_free(hh_batch b);

/* hh_matvec_noalloc -- y = A_h x (transpose != 0: A_h^T x) for ONE
 * right-hand side (x, y device, ld = n) that allocates nothing: no
 * cudaMalloc, cudaFree or allocating library call.  It is meant for callers
 * that cannot allocate device memory when they call (a host framework that
 * owns all device memory, or a loop that must not pay cudaMalloc's implicit
 * synchronisation).  The paper has no counterpart: this is a deployment
 * variant of hh_matvec.
 *   Scratch: a fixed 32 MiB file-scope device array inside the library.
 *   A GPU holds it from the first matrix built or loaded on it (hh_build,
 *   hh_build_ex, hh_load or hh_reencode with that device), where its device
 *   address is looked up once (cudaGetSymbolAddress), until the process
 *   exits; so this call itself neither allocates nor loads anything.
 *   Matrices whose scratch (about 40 bytes per point plus 16 to 32 bytes per
 *   unit of rank) exceeds it are rejected with HH_EINVAL and a message.
 *   All calls share the one array: calls that overlap on the GPU (other
 *   streams, other handles) race and give wrong results; order them on one
 *   stream.  Everything the product needs zeroed is cleared by each call.
 *   Asynchronous on `stream`; errors as for hh_matvec. */
int hh_matvec_noalloc(hh_handle h, int transpose, const double* in, double* out, void* stream);

/* hh_sync_status -- synchronise `stream` and report the device status word
 * of the handle (HH_EDEVICE if a kernel recorded an anomaly). */
int hh_sync_status(hh_handle h, void* stream);

/* hh_free -- release a handle (NULL is a no-op).  Pending work that uses the
 * handle must be complete. */
void hh_free(hh_handle h);

/* hh_last_error -- message of the last failing call on this thread. */
const char* hh_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HH_H_ */
