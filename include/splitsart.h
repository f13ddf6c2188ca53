/*
 * splitsart.h: C ABI of the GB300 (sm_103a) symmetric-split SART library.
 *
 * The library follows Alikhanov et al., "About one method of parallelization
 * of calculations during the reconstruction of a tomographic image"
 * (arXiv:1902.10559):
 * - A slice's system A f = p (Eq. 1) whose matrix satisfies
 *   w_{i,j} = w_{M-i+1,N-j+1} (Eq. 2) is folded into two independent systems,
 *   A1 f1 = p1 and A2 f2 = p2 (Eqs. 3, 4). Each has M/2 rows and N/2 columns.
 * - Each system is solved by SART-type iteration.
 * - The image is recombined by Theorem 1 (Eq. 5).
 *
 * Conventions:
 * - Indices are 0-based. The paper's i <-> M-i+1 is i <-> M-1-i here, and
 *   j <-> N-j+1 is j <-> N-1-j. Mh = M/2, Nh = N/2.
 * - Every function returns an int status: 0 on success, a negative
 *   SPLITSART_ERR_* code on failure. splitsart_last_error() gives the
 *   message of the calling thread's last failure.
 * - Handles are opaque and owned by the library. Each is released by its
 *   *_destroy function. Destroying NULL is a no-op.
 * - Arguments ending in _dev are device pointers owned by the caller.
 *   Arguments ending in _host are host pointers owned by the caller. The
 *   library keeps no pointer to caller memory after a call returns.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream). Device work is enqueued on it, and the call returns without
 *   synchronising. Functions named *_result, *_export and *_info synchronise
 *   the system's last stream, because they read device results to the host.
 * - Vector element type ("vec"): double for SPLITSART_F64 systems, float for
 *   all others. The pair layout interleaves the two split systems: element
 *   i of a pair vector is (x1_i, x2_i). Pair vectors are therefore double2 or
 *   float2 arrays.
 */
#ifndef SPLITSART_H
#define SPLITSART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SPLITSART_OK 0
#define SPLITSART_ERR_ARG (-1)        /* bad argument: NULL, size or range */
#define SPLITSART_ERR_ODD_DIM (-2)    /* nx odd or M odd: the split needs N and M even (Section 2) */
#define SPLITSART_ERR_ASYMMETRIC (-3) /* the matrix cannot satisfy Eq. (2) */
#define SPLITSART_ERR_CUDA (-4)       /* a CUDA runtime call failed */
#define SPLITSART_ERR_TIMEOUT (-5)    /* a bounded device-side wait ran out */
#define SPLITSART_ERR_NOMEM (-6)      /* device or host allocation failed */
#define SPLITSART_ERR_STATE (-7)      /* call made in the wrong order */
#define SPLITSART_ERR_NONFINITE (-8)  /* the input holds NaN or Inf */
#define SPLITSART_ERR_NOT_SPD (-9)    /* a normal matrix is not positive definite: the matrix lacks full column rank */

/* ---- value storage of the folded matrices ---- */
#define SPLITSART_F64 0  /* double pairs, double vectors and normalisers */
#define SPLITSART_F32 1  /* float pairs, float vectors and normalisers */
#define SPLITSART_BF16 2 /* bf16 codes + per-row float scales; float vectors; double normalisers */
#define SPLITSART_F16 3  /* fp16 codes + per-row float scales; float vectors; double normalisers */

/* ---- image layouts ---- */
#define SPLITSART_LAYOUT_SNAKE 0 /* f[N] in vertical-snake order (Section 2, Fig. 1) */
#define SPLITSART_LAYOUT_IMAGE 1 /* f[nz][nx], row r from the bottom, column c from the left */

/*
 * Acquisition of one 2D slice (Section 2). Lengths are in mm, angles in
 * degrees.
 * - Object: x in [-W/2, W/2], z in [z0, z0+H], with nx x nz cells.
 * - Sources: K point sources at theta_k = gamma (2k+1-K)/(K-1), at
 *   (R sin theta_k, R cos theta_k). Source K-1-k is the exact mirror (-x, z)
 *   of source k (positions pairwise symmetric about OZ).
 * - Detector: nb bins on z = 0, centred at u_b = D (2b+1-nb)/(2nb).
 * - Rays: ray i = k nb + b runs from source k to the centre of bin b, so
 *   M = K nb. Ray M-1-i is the mirror of ray i.
 * - Voxels: cell (c, r) has vertical-snake index
 *   j = c nz + (c even ? r : nz-1-r). When nx is even, j <-> N-1-j is the
 *   mirror about OZ, which gives Eq. (2).
 */
typedef struct splitsart_geometry_params {
    int32_t nx, nz;
    double W, H, z0;
    int32_t K;
    double gamma_deg, R;
    int32_t nb;
    double D;
} splitsart_geometry_params;

typedef struct splitsart_geometry splitsart_geometry; /* host: first M/2 rows of A */
typedef struct splitsart_system splitsart_system;     /* device: folded A1/A2, CSR + CSC + normalisers */

/*
 * Build the first Mh rows of A on the host, in FP64.
 * - Weights: w_ij is the exact (Siddon) length of ray i inside cell j, in mm.
 * - A ray lying exactly on a vertical cell boundary gives half its length to
 *   each of the two adjacent cells.
 * - Rows i >= Mh are never built. Eq. (2) makes them redundant:
 *   w_{M-1-i, N-1-j} = w_{i,j}.
 * Errors: SPLITSART_ERR_ODD_DIM if nx is odd or K nb is odd;
 * SPLITSART_ERR_ARG for non-positive sizes or K < 2.
 */
int splitsart_make_geometry(const splitsart_geometry_params* params, splitsart_geometry** out);

/*
 * The same rows as splitsart_make_geometry, for n slices at once, traced on
 * the GPU (one thread per ray; Section 2 geometry, Siddon lengths, FP64).
 * - params[n]: one acquisition per slice. out[n] receives n geometries,
 *   each bitwise equal to what splitsart_make_geometry returns for its
 *   params (same rows, columns and FP64 lengths), owned by the caller (free
 *   each with splitsart_geometry_destroy).
 * - The columns and lengths stay in device memory (12 bytes per entry, one
 *   allocation shared by the n geometries and freed with the last of them);
 *   the row pointers are on the host. splitsart_fold_system/_fold_batch copy
 *   the rows on the device; splitsart_geometry_export copies them to the
 *   host.
 * - stream: the CUDA stream of the device work (NULL: the default stream).
 *   The call synchronises that stream before it returns.
 * - Working memory while tracing: about 12 more bytes per entry and 16 per
 *   ray, freed before the call returns.
 * Errors: those of splitsart_make_geometry for any slice (then no geometry
 * is returned); SPLITSART_ERR_CUDA or SPLITSART_ERR_NOMEM.
 */
int splitsart_make_geometries_device(const splitsart_geometry_params* params, int n, void* stream,
                                     splitsart_geometry** out);

/*
 * Wrap caller-supplied first-half rows of any matrix that satisfies Eq. (2).
 * For example, the 4 x 6 system of Example 1.
 * - row_ptr_host[Mh+1] (int64) and col_host/val_host[nnz] hold rows
 *   0..Mh-1 of A in CSR form, with Mh = M/2. Columns are in [0, N) and
 *   strictly increasing within a row.
 * - The data are copied.
 * Errors: SPLITSART_ERR_ODD_DIM if M or N is odd; SPLITSART_ERR_ARG if the
 * CSR is malformed; SPLITSART_ERR_NONFINITE for NaN or Inf values.
 */
int splitsart_make_geometry_from_csr(int64_t M, int64_t N, const int64_t* row_ptr_host,
                                     const int32_t* col_host, const double* val_host,
                                     splitsart_geometry** out);

/* Report M, N and the stored nonzeros of rows 0..Mh-1. Any output may be NULL. */
int splitsart_geometry_info(const splitsart_geometry* g, int64_t* M, int64_t* N, int64_t* nnz_half);

/* Copy the first-half CSR to host buffers sized from splitsart_geometry_info. */
int splitsart_geometry_export(const splitsart_geometry* g, int64_t* row_ptr_host, int32_t* col_host,
                              double* val_host);

void splitsart_geometry_destroy(splitsart_geometry* g);

/*
 * Fold A into A1 and A2 on the device. The formulas are those after Eq. (4):
 *     w1_ij = w_ij - w_{M-1-i,j},   w2_ij = w_ij + w_{M-1-i,j},   i < Mh, j < Nh.
 * Eq. (2) turns the mirror row into a reflection of row i itself:
 * w_{M-1-i,j} = w_{i,N-1-j}. So each folded row i is a merge of row i's left
 * half with its reflected right half. Row M-1-i is never read.
 *
 * The call:
 * - allocates the system, sized from an upper bound;
 * - uploads the half rows;
 * - runs on `stream`: the fold, a deterministic CSC transpose, and the
 *   absolute row/column sums with 1/0 := 0.
 *
 * A1 and A2 share one column-index pattern. It is the union pattern, and it
 * keeps exact zeros made by cancellation. `dtype` selects the value storage
 * (SPLITSART_F64/F32/BF16/F16).
 * - BF16/F16 store codes q_ij = round(a_ij / s_i), with s_i = max_j |a_ij|
 *   per row and per system, as an FP32 scale. The division and the rounding
 *   are done in FP32, round to nearest even.
 * - The normalisers of a BF16/F16 system are taken, in FP64, from the
 *   dequantised values s_i q_ij.
 * Errors: SPLITSART_ERR_ARG, SPLITSART_ERR_NOMEM, SPLITSART_ERR_CUDA.
 */
int splitsart_fold_system(const splitsart_geometry* g, int dtype, void* stream, splitsart_system** out);

/*
 * Fold a batch of independent slices into one system. Each slice is one
 * geometry, with its own sizes, and satisfies Eq. (2) by itself.
 * The slices are concatenated in every index space:
 * - folded rows and columns;
 * - full projections p (slice k at M_off[k]);
 * - full images f (slice k at N_off[k]).
 * The folded matrix is block-diagonal, so the slices stay independent.
 * fold_rhs, fold_image, recombine and project act on all slices at once.
 * splitsart_solve runs every slice in one persistent launch, and each slice
 * has its own stopping test: rho_s of its own residual, its own iteration
 * count and its own returned iterate. Read them with
 * splitsart_solve_result_slices.
 * geoms: array of nslices geometry handles (borrowed; the data are copied).
 */
int splitsart_fold_batch(const splitsart_geometry* const* geoms, int nslices, int dtype, void* stream,
                         splitsart_system** out);

/*
 * Slice offsets. Each array has nslices + 1 entries, or is NULL to skip it.
 * - M_off: full projections;
 * - N_off: full images;
 * - Mh_off: folded rows;
 * - Nh_off: folded columns.
 */
int splitsart_system_slices(const splitsart_system* sys, int64_t* M_off, int64_t* N_off, int64_t* Mh_off,
                            int64_t* Nh_off);

/*
 * Re-run the device fold of an existing system from its uploaded half rows.
 * The fold covers the CSR, the CSC and the normalisers. Nothing is allocated.
 */
int splitsart_refold(splitsart_system* sys, void* stream);

typedef struct splitsart_system_info {
    int64_t M, N, Mh, Nh;   /* totals over all slices */
    int64_t nnz_half;    /* stored entries of rows 0..Mh-1 of A */
    int64_t S;           /* stored entries of the shared folded pattern */
    int64_t empty_rows;  /* folded rows with no entry */
    int64_t exact_zeros; /* entries with w1 = 0 made by cancellation */
    int32_t dtype;
    int32_t nx, nz;      /* 0 when the geometry came from a CSR, or for a batch */
    int64_t device_bytes;
    int32_t nslices;     /* 1, or the slices of a batch */
    int32_t reserved;
} splitsart_system_info;

/* Fill *info. This synchronises with the system's last stream, once, to read S. */
int splitsart_system_info_get(splitsart_system* sys, splitsart_system_info* info);

/*
 * Copy the folded CSR to the host. Buffer sizes:
 * - row_ptr_host: Mh+1 entries (int64);
 * - col_host: S entries (int32);
 * - a1_host, a2_host: S entries (double). These hold the values the
 *   iteration uses: for BF16/F16 systems, the dequantised s_i q_ij.
 * - normalisers (optional, may be NULL): R_host[2 Mh] and C_host[2 Nh],
 *   interleaved (system 1, system 2). They hold the absolute sums, not their
 *   reciprocals.
 * This function is for verification.
 */
int splitsart_system_export(splitsart_system* sys, int64_t* row_ptr_host, int32_t* col_host,
                            double* a1_host, double* a2_host, double* R_host, double* C_host);

/*
 * Copy the folded CSC (the transpose used by the back-projection) to the host.
 * Buffer sizes:
 * - col_ptr_host: Nh+1 entries;
 * - row_host: S entries;
 * - a1_host, a2_host: S entries.
 * Rows within a column are in increasing order.
 */
int splitsart_system_export_csc(splitsart_system* sys, int64_t* col_ptr_host, int32_t* row_host,
                                double* a1_host, double* a2_host);

void splitsart_system_destroy(splitsart_system* sys);

/*
 * Fold a projection vector as after Eq. (4):
 *     p1_i = p_i - p_{M-1-i},   p2_i = p_i + p_{M-1-i},   i < Mh.
 * p_dev: vec[M]. p12_dev: pair[Mh] output.
 */
int splitsart_fold_rhs(const splitsart_system* sys, const void* p_dev, void* p12_dev, void* stream);

/*
 * Fold an image, using the vectors of the proof of Theorem 1:
 *     f1_j = f_j - f_{N-1-j},   f2_j = f_j + f_{N-1-j},   j < Nh.
 * This gives a warm start for splitsart_solve.
 * f_dev: vec[N] in `layout` (SPLITSART_LAYOUT_IMAGE needs a geometry with nx, nz).
 * f12_dev: pair[Nh] output.
 */
int splitsart_fold_image(const splitsart_system* sys, const void* f_dev, int layout, void* f12_dev,
                         void* stream);

/*
 * Recombine by Theorem 1, Eq. (5):
 *     f_j = (f2_j + f1_j)/2,   f_{N-1-j} = (f2_j - f1_j)/2.
 * f12_dev: pair[Nh]. f_dev: vec[N] output, written in `layout`.
 */
int splitsart_recombine(const splitsart_system* sys, const void* f12_dev, void* f_dev, int layout,
                        void* stream);

/*
 * Forward projection p = A f of a full image, through the folded system.
 * Steps: fold f (proof of Theorem 1), apply A1 and A2, then unfold the rays:
 *     p_i = (q2_i + q1_i)/2,   p_{M-1-i} = (q2_i - q1_i)/2.
 * This is exact, because A1 f1 = fold1(A f) and A2 f2 = fold2(A f).
 * f_dev: vec[N] in `layout`. p_dev: vec[M] output.
 * Arithmetic is in the system's precision.
 */
int splitsart_project(splitsart_system* sys, const void* f_dev, int layout, void* p_dev, void* stream);

/*
 * Options of splitsart_solve. Zero-initialise the struct, then set fields.
 */
typedef struct splitsart_solve_opts {
    int32_t max_iters;     /* iteration cap, in [0, 500000] */
    double lambda;         /* relaxation, 0 < lambda < 2 */
    double tol;            /* stop at the first k with rho_k <= tol; 0 = run max_iters (rho is then tested only
                              at k = 0, where p = 0 stops at once, and at k = max_iters) */
    int32_t check_every;   /* test rho every this many iterations (>= 1; 0 means 1); not used when tol = 0 */
    int32_t block_threads; /* threads per CTA, multiple of 32 in [64, 1024]; 0 = the kernel's default.
                              Kernel 1: default 1024. Kernels 2 and 3: at most 512 (default 512;
                              larger values run 512). Kernel 4: at most 384 (default 384) */
    int32_t ctas_per_sm;   /* 0 = as many as fit */
    int32_t lanes_per_col; /* back-projection lanes per column, 0 = default (8); 1,2,4,8,16,32 */
    int32_t kernel;        /* 0 = choose (2 if the system fits on chip, else 3); 0-8. 1 = stream the matrix in
                              CTA-wide tiles; 2 = keep it in shared memory; 3 = stream it row by row
                              through registers; 4 = stream it per warp through shared memory with
                              bulk asynchronous copies (lanes_per_col 4 or 8 only); 5 = stream it row by
                              row in compacted index order, each warp loading its next chunk's row and
                              column data ahead;
                              6 = kernel 5 on the implicit fold (each half-row entry of A stored once,
                              its folded column carrying A1's sign: 8 instead of 12 bytes per entry and
                              pass in FP32; results differ from the explicit fold by rounding where a
                              ray and its mirror cross the same folded cell). 3 to 6 have no CTA
                              barriers inside a pass. 5: every value storage; 6: FP64 and FP32 systems;
                              both lanes_per_col 4 or 8; their first use builds the re-indexed copy of the matrix (4 bytes
                              per entry and pass for 5, 8 or 12 for 6) and keeps it with the system;
                              7 and 8 = kernels 5 and 6 with the matrix fed through a shared-memory ring:
                              per CTA one producer warp copies chunks of rows (columns) with bulk asynchronous
                              copies and the other warps only gather and sum; they return kernel 5's and 6's
                              f bit for bit at equal lanes_per_col. tile_entries is their chunk entry target
                              (0 = 4096 for 12-byte entries, 3072 for 8-byte ones, else about 48 KB of
                              entries); a chunk must fit in the ring (about 225 KB of shared memory; 160 KB
                              for 8-byte entries, leaving the rest to L1), else SPLITSART_ERR_ARG. block_threads and
                              ctas_per_sm are not used (one CTA per SM). Their first use also makes the chunk
                              plans (one synchronisation) and keeps them with the system */
    double timeout_ms;     /* limit of each grid-barrier wait (kernels 4, 7, 8: also of each wait on a bulk copy
                              or a ring release); 0 = default (2000 ms) */
    int32_t inject_barrier_fault; /* test hook: the barrier also waits for a CTA that never comes */
    int32_t tile_entries;  /* kernel 1: entries staged per tile; kernels 7 and 8: chunk entry target. 0 = default;
                              else a multiple of 1024 in [1024, 16384] */
    int32_t row_weight;    /* kernel 2: when rows are dealt to CTAs, each row weighs this many entries more than
                              its length (a row's fixed cost). 0 = default: the heaviest of 240, 160, 80, 40, 0
                              whose plan fits in shared memory; a value that does not fit falls back the same way */
    int32_t lanes_per_row; /* kernels 7 and 8: forward-pass lanes per row, 8, 16 or 32; 0 = default (32). At 32 a
                              row is summed by the whole warp in kernels 5's and 6's order (bitwise their f); fewer
                              lanes put 32 / lanes_per_row rows of a warp in flight at once, with the row's sum
                              lane-strided over its lanes and reduced by their shuffle tree (another fixed order).
                              splitsart_solve_multi: lanes per (row or column, right-hand side), 2, 4 or 8 with
                              rhs_per_cta x lanes_per_row <= 32; 0 = default (2) */
} splitsart_solve_opts;

/*
 * Solve both split systems by the simultaneous SART-type iteration, in one
 * persistent cooperative launch. For system s in {1, 2}:
 *     r^k = p^s - A_s f^k,   u^k_i = r^k_i / R_i,   f^{k+1}_j = f^k_j + lambda (A_s^T u^k)_j / C_j
 * R and C are the absolute row and column sums, with 1/0 := 0.
 * The two systems share each pass over the index pattern.
 *
 * Stopping: with
 *     rho_k = sqrt(||r1^k||^2 + ||r2^k||^2) / sqrt(||p1||^2 + ||p2||^2),
 * which equals ||A f^k - p|| / ||p|| for the recombined image, the solve
 * returns f^k at the first tested k with rho_k <= tol, or at
 * k = max_iters. The update is skipped on the stopping pass. The squares of
 * r are summed in FP32 groups of 16 and the group sums in FP64. With kernels
 * 1 and 2 every sum has a fixed order, so repeated runs of one launch shape
 * are bitwise identical (f^k and rho). Kernels 3 and 4 hand out rows
 * dynamically: their per-row and per-column sums keep a fixed order, but the
 * grouping of the norm sums does not, so rho can differ in its last bits from
 * run to run.
 *
 * Arguments:
 * - p12_dev: pair[Mh] from splitsart_fold_rhs.
 * - f12_dev: pair[Nh], in = f^0, out = f^k.
 *
 * The result (iterations, rho, status) stays on the device until
 * splitsart_solve_result reads it. Errors found before the launch are
 * returned directly. A barrier timeout is reported by splitsart_solve_result.
 */
int splitsart_solve(splitsart_system* sys, const void* p12_dev, void* f12_dev, const splitsart_solve_opts* opts,
                    void* stream);

typedef struct splitsart_solve_info {
    int32_t iters;   /* k of the returned iterate */
    int32_t status;  /* SPLITSART_OK or SPLITSART_ERR_TIMEOUT */
    double rho;      /* rho_k of the returned iterate */
    double rr;       /* ||r1||^2 + ||r2||^2 */
    double pp;       /* ||p1||^2 + ||p2||^2 */
} splitsart_solve_info;

/*
 * Synchronise the system's last stream and read the last solve's result.
 * Returns info->status, or SPLITSART_ERR_CUDA if the device reports an error.
 */
int splitsart_solve_result(splitsart_system* sys, splitsart_solve_info* info);

/*
 * Options of splitsart_solve_os. Zero-initialise, then set fields.
 */
typedef struct splitsart_os_opts {
    int32_t subset_rows; /* folded rows per subset; 0 = one folded view pair (the geometry's nb rows) */
    int32_t cone;        /* 1: keep every voxel of the image non-negative (f2 >= |f1|) */
    int32_t reserved[2]; /* zero */
} splitsart_os_opts;

/*
 * Ordered-subsets SART (OS-SART) on both split systems, with an optional
 * non-negativity constraint, in one persistent cooperative launch.
 *
 * SART as Andersen and Kak state it (Section 1, reference [001]) updates the
 * image once per projection view. Here the folded rows are taken in subsets
 * of subset_rows consecutive rows; by default a subset is one folded view
 * pair (rows t nb .. t nb + nb - 1 carry the rays of sources t and K-1-t).
 * One iteration applies, for t = 0, 1, ..., T-1 in turn and each system s:
 *     u_i = (p^s_i - (A_s f)_i) / R_i                     for rows i of subset t
 *     f_j += lambda (sum_{i in subset t} a_ij u_i) / C_t,j
 * with C_t,j = sum_{i in subset t} |a_ij| and 1/0 := 0. With one subset this
 * is splitsart_solve's simultaneous SART.
 *
 * The cone: f >= 0 for the image holds iff f2_j >= |f1_j| for every voxel
 * pair (Eq. 5). With cone = 1 the start and every subset update are
 * projected onto it: recombine the pair, clip both voxels at zero, fold
 * again.
 *
 * Stopping: rho_k = ||A f^k - p|| / ||p|| of the iterate after k full
 * sweeps, tested when k is a multiple of opts->check_every or k =
 * opts->max_iters, before the sweep. With more than one subset a test costs
 * one extra forward pass. The result is read by splitsart_solve_result.
 *
 * opts: max_iters, lambda, tol, check_every, block_threads (at most 512),
 * lanes_per_col, timeout_ms and inject_barrier_fault are used; the other
 * fields are ignored.
 * The first call for a subset size builds per-subset column tables on the
 * device (about 12 bytes per subset and non-empty column) and keeps them
 * with the system.
 * Errors: SPLITSART_ERR_ARG for a batch system, a BF16/FP16 system, or
 * subset_rows = 0 on a system folded from a CSR (no geometry).
 */
int splitsart_solve_os(splitsart_system* sys, const void* p12_dev, void* f12_dev, const splitsart_solve_opts* opts,
                       const splitsart_os_opts* os, void* stream);

/*
 * CGLS on both split systems in one persistent cooperative launch.
 *
 * The normal matrix of each split system is the fold of the full normal
 * matrix (text after Eq. 18): B_s = A_s^T A_s. CGLS runs conjugate gradients
 * on A_s^T A_s f = A_s^T p_s without forming B_s: one pass over the folded
 * CSR (q = A d) and one over the folded CSC (s = A^T r) per iteration, both
 * systems in the same passes, each with its own step lengths. From f^0 = 0 on
 * a consistent system the iterates tend to the normal pseudo-solution, so the
 * recombined image tends to the full system's (Theorem 2).
 *
 * Stopping is the joint rule of splitsart_solve: rho_k = ||A f^k - p|| / ||p||
 * tested before step k when k is a multiple of opts->check_every or k =
 * opts->max_iters. Reductions are FP64 in a fixed order; repeated runs of one
 * launch shape are bitwise identical.
 * opts: max_iters, tol, check_every, block_threads (at most 512),
 * lanes_per_col, timeout_ms and inject_barrier_fault are used (lambda is not).
 * The first call allocates four work vectors (2 Mh + 2 Nh pairs), kept with
 * the system. The result is read by splitsart_solve_result.
 * Errors: SPLITSART_ERR_ARG for a batch system or a BF16/FP16 system.
 */
int splitsart_solve_cgls(splitsart_system* sys, const void* p12_dev, void* f12_dev, const splitsart_solve_opts* opts,
                         void* stream);

/*
 * ---- The direct method (Example 2, Table 1) ----
 * Least squares A x = b through the normal equations, dense, in FP64 on the
 * device: B = A^T A and c = A^T b from the CSR and CSC of A (row j of B is
 * accumulated in one CTA's shared memory, in a fixed order), a blocked
 * Cholesky factorisation B = L L^T (blocks of 64), then L y = c and
 * L^T x = y. The split form applies it to A1 and A2, whose normal matrices
 * are the folds of A^T A (text after Eq. 18), and recombines by Theorem 1.
 *
 * splitsart_normal_solve_bytes: bytes of the work buffer for n unknowns
 * (8 n^2 + 8 n + 256).
 */
int splitsart_normal_solve_bytes(int64_t n, int64_t* bytes);

/*
 * The normal-equation solve of any m x n matrix with full column rank.
 * - CSR: rp_dev[m+1], col_dev (columns increasing within a row), val_dev;
 *   CSC: cp_dev[n+1], row_dev (rows increasing within a column), valT_dev.
 *   Values are doubles read at stride val_stride: 1 for plain arrays, 2 for
 *   one member of an interleaved pair array (pointer offset by 0 or 1).
 * - b_dev[m] at stride b_stride; x_dev[n] (output) at stride x_stride.
 * - work_dev: caller-owned device buffer of splitsart_normal_solve_bytes(n).
 * - status_dev: device int32, written 0, or SPLITSART_ERR_NOT_SPD when a
 *   pivot of the factorisation is not positive (the later steps are skipped
 *   and x_dev is not written). A column without entries (a voxel no ray
 *   crosses) gives a zero pivot. A matrix that is singular only numerically
 *   may leave a tiny positive pivot instead: full column rank is the
 *   caller's to ensure.
 * n is limited by one CTA's shared memory (8 bytes per unknown; about 29000
 * on this GPU). Errors found before the launch are returned directly.
 */
int splitsart_normal_solve(int64_t m, int64_t n, const int32_t* rp_dev, const int32_t* col_dev, const double* val_dev,
                           const int32_t* cp_dev, const int32_t* row_dev, const double* valT_dev, int32_t val_stride,
                           const double* b_dev, int32_t b_stride, double* x_dev, int32_t x_stride, void* work_dev,
                           int32_t* status_dev, void* stream);

/*
 * The split direct method on a folded FP64 single-slice system: fold p (after
 * Eq. 4), the normal-equation solves of A1 and of A2 one after the other (they
 * share work_dev, splitsart_normal_solve_bytes(N/2) bytes), and the Theorem 1
 * recombination into f_dev[N] (snake order). p_dev[M] FP64. status_dev as for
 * splitsart_normal_solve.
 */
int splitsart_direct_split(splitsart_system* sys, const double* p_dev, double* f_dev, void* work_dev,
                           int32_t* status_dev, void* stream);

/*
 * Allocation-free solve. The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc. Examples are a process that
 * reserves all of its device memory at start-up and forbids allocation
 * afterwards, and a plugin inside a host application that owns the GPU's
 * memory budget. Such a caller cannot use splitsart_fold_system, which
 * allocates. It can place a folded system in buffers of its own and solve it
 * here.
 *
 * The call runs the same persistent SART kernel as splitsart_solve, on a
 * plain folded FP32 system. It allocates nothing. Its working memory is one
 * fixed array inside the library (a static __device__ array of about
 * 0.6 MiB), which every GPU that loads the library holds until the process
 * exits. The array holds:
 * - the launch control block, the result, and the per-CTA norm partials;
 * - u for at most 65536 folded rows.
 * Larger systems (Mh > 65536) are rejected with SPLITSART_ERR_ARG; use
 * splitsart_solve for them.
 *
 * Arguments, all device pointers owned by the caller and never NULL (also
 * not when S = 0; SPLITSART_ERR_ARG otherwise):
 * - rp_dev[Mh+1] int32, col_dev[S] int32, val_dev[S] float2 (a1, a2): the
 *   folded CSR, with columns increasing within a row;
 * - cp_dev[Nh+1] int32, row_dev[S] int32, valT_dev[S] float2: the folded CSC,
 *   with rows increasing within a column;
 * - invR_dev[Mh], invC_dev[Nh] float2: reciprocal absolute row and column
 *   sums, 0 where a sum is 0;
 * - p12_dev[Mh] float2, and f12_dev[Nh] float2 (in: f0, out: the result);
 * - info_dev: device splitsart_solve_info, written when the call's work
 *   completes. status is SPLITSART_ERR_TIMEOUT if a barrier wait ran out.
 * `opts` is read as in splitsart_solve.
 *
 * Every call looks up the array's device address in the current device's
 * context (a host-side lookup; after a context is destroyed and created
 * again the array may move, and the next call finds it). The first call in
 * a context also loads the library's device code there: make that first
 * call before any stream capture.
 * Every call shares the one array and clears its control block on `stream`.
 * Calls that overlap on the GPU (other streams, other host threads) race on
 * the array and must be serialised by the caller.
 */
int splitsart_solve_static(int64_t Mh, int64_t Nh, const int32_t* rp_dev, const int32_t* col_dev, const void* val_dev,
                           const int32_t* cp_dev, const int32_t* row_dev, const void* valT_dev, const void* invR_dev,
                           const void* invC_dev, const void* p12_dev, void* f12_dev, const splitsart_solve_opts* opts,
                           splitsart_solve_info* info_dev, void* stream);

/*
 * Solve one system for many right-hand sides at once, as a sparse matrix
 * times a block of vectors.
 * - Each right-hand side is an independent split-SART solve (the update and
 *   the stopping test of splitsart_solve), with its own iteration count and
 *   rho. The matrix is shared.
 * - The whole folded system is kept in each CTA's shared memory, together
 *   with rhs_per_cta right-hand sides (0 = library default, 4; allowed 1, 2,
 *   4, 8, 16). Every matrix entry read serves all of them.
 * - An iteration touches no global memory, so the launch needs no grid-wide
 *   barrier.
 * - opts->block_threads: a multiple of 32 in [32, 1024] (0 = 512).
 * - opts->lanes_per_row: lanes per (row or column, right-hand side), 2, 4 or
 *   8 (0 = 2); a warp sums 32 / (rhs_per_cta x lanes_per_row) rows at once.
 *   The summation order depends on it (a fixed order for each value).
 * - The system must be a single slice small enough for shared memory.
 *   Otherwise SPLITSART_ERR_ARG: use splitsart_solve per right-hand side.
 * Arguments:
 * - p12_dev: pair[nrhs][Mh], each right-hand side's folded p, contiguous.
 * - f12_dev: pair[nrhs][Nh], in: f0, out: the results.
 * - info_dev: device splitsart_solve_info[nrhs], written as each right-hand
 *   side stops.
 */
int splitsart_solve_multi(splitsart_system* sys, int nrhs, const void* p12_dev, void* f12_dev,
                          const splitsart_solve_opts* opts, int rhs_per_cta, splitsart_solve_info* info_dev,
                          void* stream);

/*
 * splitsart_solve_multi with the order in which the persistent launch takes
 * its right-hand sides: order_dev[nrhs] (device int32) is a permutation of
 * 0..nrhs-1, and queue position q solves right-hand side order_dev[q]
 * (NULL: in index order, as splitsart_solve_multi). The layouts of p12_dev,
 * f12_dev and info_dev stay indexed by right-hand side. With more right-hand
 * sides than resident slots, the launch ends when the last long one does;
 * handing out the longest first shortens that tail.
 */
int splitsart_solve_multi_ordered(splitsart_system* sys, int nrhs, const void* p12_dev, void* f12_dev,
                                  const splitsart_solve_opts* opts, int rhs_per_cta, const int32_t* order_dev,
                                  splitsart_solve_info* info_dev, void* stream);

/*
 * Fallback rule of the warm start, per right-hand side r of a multi solve:
 * if info_warm[r].rho < info_base[r].rho, f12_dev[r] := f12_warm_dev[r];
 * otherwise f12_dev[r] (the base start) is kept. The rho values come from
 * splitsart_solve_multi runs with max_iters = 0 (warm) and the early solve
 * (base). picked_dev[r] (optional) receives 1 where the warm start was kept.
 * f12 arrays are pair[nrhs][Nh] and info arrays device splitsart_solve_info[nrhs].
 */
int splitsart_pick_start(const splitsart_system* sys, int nrhs, const void* f12_warm_dev,
                         const splitsart_solve_info* info_warm_dev, const splitsart_solve_info* info_base_dev,
                         void* f12_dev, int* picked_dev, void* stream);

/*
 * Per-slice results of the last solve of a batch system. info has at least
 * nslices entries. Synchronises like splitsart_solve_result. A single-slice
 * system reports its one result.
 */
int splitsart_solve_result_slices(splitsart_system* sys, splitsart_solve_info* info, int n);

/*
 * ---- Learned warm start ----
 * The paper has no network. This is a small residual CNN that maps an early
 * split-SART image to an initial guess for the solve. The guess is folded
 * into (f1, f2) with splitsart_fold_image, as in the proof of Theorem 1, and
 * the solve continues from it.
 *
 * Network, on images [B][nz][nx] (row r from the bottom, column c from the
 * left, as SPLITSART_LAYOUT_IMAGE):
 *     a1 = relu(conv(x, W1) + b1)     1 -> 32 channels
 *     a2 = relu(conv(a1, W2) + b2)   32 -> 32
 *     a3 = relu(conv(a2, W3) + b3)   32 -> 32
 *     y  = x + conv(a3, W4) + b4     32 -> 1
 * conv is a 3x3 cross-correlation with zero padding 1. Tap (dy, dx) reads
 * pixel (r + dy - 1, c + dx - 1), and weights are [out][in][3][3].
 * Parameters are one float vector of 19105 values, in the order W1, b1, W2,
 * b2, W3, b3, W4, b4.
 * Training minimises mean((y - t)^2) with Adam.
 */
typedef struct splitsart_cnn splitsart_cnn;

/* Create the network for nz x nx images and batches up to max_batch, from
 * initial parameters (host, 19105 floats). Device memory is allocated here.
 * nx <= 256. */
int splitsart_cnn_create(int nz, int nx, int max_batch, const float* params_host, splitsart_cnn** out);
void splitsart_cnn_destroy(splitsart_cnn* cnn);

/* Arithmetic of the two 32 -> 32 layers:
 * - 0: FP32 on the CUDA cores (default);
 * - 1: BF16 tcgen05 tensor-core MMAs with FP32 accumulation in tensor
 *   memory, on tiles of 128 consecutive pixels of the batch (any nz, nx).
 * Layers 1 and 4, the weight gradients and Adam are FP32 in both modes. */
int splitsart_cnn_set_mode(splitsart_cnn* cnn, int mode);

/* Copy the parameters (and, if moments_host is non-NULL, the Adam moments
 * m then v: 2 x 19105 floats) to the host. Synchronising. */
int splitsart_cnn_params(splitsart_cnn* cnn, float* params_host, float* moments_host);

/* Replace the parameters. moments_host may be NULL (then zeroed). step is
 * the Adam step count already taken. Together with splitsart_cnn_params this
 * gives checkpoint and resume. Synchronising. */
int splitsart_cnn_set_params(splitsart_cnn* cnn, const float* params_host, const float* moments_host, int step);

/* Inference: y_dev[B][nz][nx] = net(x_dev[B][nz][nx]). */
int splitsart_cnn_forward(splitsart_cnn* cnn, const float* x_dev, int B, float* y_dev, void* stream);

/* Loss and gradient without an update. loss_dev (1 float) and grad_dev (19105 floats) may each be NULL. */
int splitsart_cnn_loss_grad(splitsart_cnn* cnn, const float* x_dev, const float* t_dev, int B, float* loss_dev,
                            float* grad_dev, void* stream);

/* One Adam step on the batch (x_dev, t_dev). loss_dev (1 float, may be NULL)
 * receives the batch loss before the update. */
int splitsart_cnn_train_step(splitsart_cnn* cnn, const float* x_dev, const float* t_dev, int B, double lr, double beta1,
                             double beta2, double eps, float* loss_dev, void* stream);

/* Copy the thread's last error message into buf (truncated, NUL-terminated). Returns its full length. */
int splitsart_last_error(char* buf, size_t len);

/* Library version string. */
const char* splitsart_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPLITSART_H */
