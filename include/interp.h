/*
 * interp.h -- C ABI of the B300 (sm_103a) lattice convolution-sum evaluator.
 *
 * Operation (Horacsek & Alim, arXiv 2102.08514, Eq. 1 with h = 1, split over Cartesian cosets as
 * in Sec. 4.1):
 *
 *     f(x) = sum_k sum_i c_k[i] * phi(x - (D i + l_k)),      phi(x) = |det L| * M_Xi(x + sum(Xi)/2)
 *
 * where M_Xi is the box spline of Sec. 3 with direction matrix Xi, L Z^s = U_k (D Z^s + l_k) is
 * the lattice, and c_k is the coefficient array of coset k.  phi is centred at the origin and
 * scaled so that it has partition of unity on L Z^s.  Coordinates are in the paper's integer
 * frame: BCC = {all coordinates of equal parity}, FCC = {even coordinate sum}, D4* = {all four
 * coordinates of equal parity}; D = 2 for those three, D = 1 for the Cartesian lattice.
 *
 * Conventions shared by every entry point
 *   - Every function returns an interp_status and never aborts or prints.
 *   - Points are FP32, row-major (npts x s).  Outputs are FP32.
 *   - Point, output and gradient buffers are DEVICE pointers owned by the caller; the library
 *     keeps no pointer to them after the call returns.  Calls are asynchronous on `stream`
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - Coefficients outside the stored arrays are zero ("zero extension"): a query far outside
 *     the data returns 0.  A query with a NaN or infinite coordinate returns NaN.
 *   - A handle may be used from several streams at once for eval calls (read-only).  Calls that
 *     write the handle's coefficients (interp_set_coeffs) or its internal gradient buffer
 *     (interp_backward) must not overlap other calls on the same handle.
 *   - Piece pre-sort: for splines where it measured faster (many large pieces, BCC V_2; the
 *     8-coset D4; interp_info_t.presort says which), eval, eval_grad and interp_backward calls
 *     of 2^16 or more queries first sort the queries on the device by the pieces (Sec. 4.3's
 *     sub-regions) of their first cosets, in chunks of 2^22, so that the piece-binned kernel
 *     runs one piece's code for long stretches; results go back to the callers' positions.
 *     Values, gradients and pullbacks are the same bits as without the sort; the adjoint's
 *     atomic sums have no fixed order either way.  The scratch (at most ~80 bytes per query of
 *     a chunk) comes per call from a stream-ordered memory pool owned by the library (cached up
 *     to 1 GiB per device); under stream capture, or when the pool has no room, the call runs
 *     without the sort.  interp_backward_noalloc never sorts.  The handle's "presort" option
 *     (interp_set_option) forces the sort off / on for any call size: evaluation calls that run
 *     the piece-binned kernels, interp_backward calls of splines with >= 4 pieces.
 *   - Launch options are per handle (interp_set_option).  Their initial values are read from the
 *     environment once, when the handle is created: INTERP_B300_BINNED, INTERP_B300_PRESORT,
 *     INTERP_B300_DENSE, INTERP_B300_ADJOINT_BINS (0 / 1) and INTERP_B300_BINCFG (=small); later changes of the
 *     environment do not affect existing handles.
 */
#ifndef INTERP_B300_H
#define INTERP_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct interp interp_t; /* opaque; owns the halo-padded coefficient arrays */

typedef enum {
    INTERP_OK = 0,
    INTERP_EINVAL = 1,       /* bad argument: null pointer, negative size, singular L, ...      */
    INTERP_EUNSUPPORTED = 2, /* (L, Xi) has no generated tables in this build, or s not in 3..4 */
    INTERP_ENOMEM = 3,       /* device or host allocation failed                                */
    INTERP_ECUDA = 4,        /* a CUDA runtime call or kernel launch failed                     */
    INTERP_ESIZE = 5         /* a size exceeds a documented limit                               */
} interp_status;

typedef enum {
    INTERP_F32 = 0,
    INTERP_F16 = 1,   /* IEEE binary16 storage, FP32 arithmetic */
    INTERP_BF16 = 2,  /* bfloat16 storage, FP32 arithmetic      */
    INTERP_F64 = 3    /* accepted as a SOURCE type by interp_set_coeffs only (rounded to storage) */
} interp_dtype;

/* Human-readable text of a status code (static storage). */
const char *interp_strerror(interp_status st);

/* Built-in splines: the (L, Xi) pairs whose generated tables are compiled into this library.
 * interp_num_splines() returns their count; interp_spline_name(i) their names (NULL if out of
 * range); interp_table_digest() the digest of the generated tables. */
int interp_num_splines(void);
const char *interp_spline_name(int i);
const char *interp_table_digest(void);

/* Number of device allocation calls (cudaMalloc, cudaMallocAsync, cudaMallocFromPoolAsync and
 * cudaMemPoolCreate) the library has made in this process so far, over all handles and devices.
 * For checking that an entry point allocates nothing (interp_backward_noalloc). Not in the paper. */
long long interp_debug_device_allocations(void);

/*
 * interp_create -- build a handle for the lattice L Z^s (L: s x s integer, row-major, full rank)
 * and the box spline with direction matrix Xi (s x n integer, row-major; column order and column
 * signs do not matter, the spline is centred).  dims[a] is the number of samples per axis of
 * EVERY coset array (array k holds the sites D i + l_k, 0 <= i_a < dims[a]).
 *
 * storage selects the device storage type of the coefficients (F32, F16 or BF16).  The handle
 * allocates the coefficient arrays with a zero halo of 2*HALO sites per side (HALO = the largest
 * stencil offset of the spline), so gathers need no bounds checks.  Coefficients start at zero;
 * set them with interp_set_coeffs.
 *
 * Errors: EINVAL (null pointers, dims < 1, singular L, L^{-1} Xi not integer), EUNSUPPORTED (no
 * generated tables for this (L, Xi)), ESIZE (padded arrays above 2^31 - 1 elements), ENOMEM,
 * ECUDA.  On error *out is set to NULL.
 */
interp_status interp_create(int s, const int32_t *L, const int32_t *xi, int n, const int32_t *dims,
                            interp_dtype storage, interp_t **out);

/*
 * interp_create_named -- the same for a built-in spline named by interp_spline_name(i): any
 * built-in box spline, or a Voronoi spline, which has no direction matrix.  The Voronoi
 * splines (Sec. 3: V_0 = chi, 1/|det L| on the Voronoi region of L; V_n = V_0 * V_{n-1}; the
 * basis is phi = |det L| V_n) are built in on their own lattices:
 *   "bcc_voronoi1", "bcc_voronoi2"   BCC, L = L_BCC of Sec. 3 (integer frame, 2 cosets, D = 2)
 *   "fcc_voronoi1", "fcc_voronoi2"   FCC, L = L_FCC of Sec. 3 (4 cosets, D = 2)
 * dims, storage and the coefficient layout are as for interp_create (coset k of the lattice's
 * Cartesian coset decomposition, as reported by interp_info).
 *
 * Errors: EINVAL (null pointers, dims < 1, bad storage), EUNSUPPORTED (no built-in spline of that
 * name, or no FP16/BF16 kernels built for it), ESIZE, ENOMEM, ECUDA.  On error *out is NULL.
 */
interp_status interp_create_named(const char *spline, const int32_t *dims, interp_dtype storage, interp_t **out);

/* Release the handle and its device memory (NULL is a no-op). Synchronises the device. */
void interp_destroy(interp_t *h);

/* Shape queries: spline dimension s, coset count M, coset spacing D, table name. */
typedef struct {
    int s, n_cosets, D, halo, n_pieces, degree, n_monomials;
    int dims[4];
    int32_t cosets[8][4];
    double lookups_per_query;     /* expected coefficient reads per query (all cosets)      */
    double fma_value_per_query;   /* FP32 FMAs of one value evaluation (A c + Horner)       */
    double fma_grad_per_query;    /* FP32 FMAs of one value + gradient evaluation           */
    int64_t coeff_count;          /* n_cosets * prod(dims)                                  */
    const char *name;
    int kind;                     /* 0: box spline; n >= 1: Voronoi spline V_n              */
    int presort;                  /* 1: calls of >= 2^16 queries take the piece pre-sort by  */
                                  /*    default (see the conventions above)                 */
    int binned;                   /* 1: evaluation runs the piece-binned kernels by default  */
                                  /*    (>= 4 pieces with >= 200 nonzeros of A_j in all)     */
    int coop;                     /* 1: evaluation gathers one query's stencil per warp load */
                                  /*    instruction (one piece, 24 to 32 sites per query)    */
} interp_info_t;
interp_status interp_info(const interp_t *h, interp_info_t *info);

/*
 * interp_set_option / interp_get_option -- per-handle launch options (not in the paper; they
 * select among equivalent kernels, results are the same bits except where noted):
 *   "binned"           -1 default (piece-binned kernels where interp_info_t.binned is 1: >= 4
 *                      pieces with >= 200 nonzeros of A_j in all; the rays of value + gradient
 *                      of splines whose pieces have <= 100 nonzeros each stay plain), 0 plain
 *                      kernels, 1 piece-binned kernels for any multi-piece spline
 *   "presort"          -1 default (see the piece pre-sort above), 0 never, 1 every call that
 *                      can take it (adjoint sums change order, see interp_backward)
 *   "dense"            -1 default (dense piece tables for the rays of the splines that have
 *                      them), 0 never, 1 also for the binned evaluation
 *   "bin_small_tiles"  0 default, 1 binned kernels on 256-query tiles of 128-thread CTAs
 *   "adjoint_bins"     -1 default (interp_backward sorts many queries into spatial bins first,
 *                      see there), 0 never, 1 always where the spline allows it
 * Options take effect for calls enqueued after the change; do not change them while another
 * thread enqueues calls on the handle.  Errors: EINVAL (null pointer, unknown name, value out of
 * range).
 */
interp_status interp_set_option(interp_t *h, const char *name, int value);
interp_status interp_get_option(const interp_t *h, const char *name, int *value);

/*
 * interp_set_coeffs -- copy the coefficients into the handle, converting to the storage type.
 * src: n_cosets * prod(dims) values of type src_dtype (F32, F16, BF16 or F64), coset-major, then
 * row-major with the last axis fastest.  src_on_device = 1 for a device pointer, 0 for a host
 * pointer (host data is staged through pageable memcpy; the call then blocks until the copy is
 * done).  Stream-ordered on `stream`.  Errors: EINVAL, ENOMEM, ECUDA.
 */
interp_status interp_set_coeffs(interp_t *h, const void *src, interp_dtype src_dtype, int src_on_device,
                                void *stream);

/*
 * interp_prefilter -- set the coefficients to a discrete filter of samples on the lattice,
 *     c(n) = sum_t w_t f(n + v_t)      for every stored site n = D i + l_k,
 * with f the samples at the stored sites and zero outside them.  Sec. 5.2 prefilters the D4
 * spline's samples this way (7/3 at v = 0, -1/18 at the 24 lattice vectors of length sqrt 2), so
 * that the interpolant of a function's samples converges at the spline's full order; any filter
 * whose taps are lattice vectors is accepted.
 *   samples  device, FP32, n_cosets x prod(dims), coset-major, last axis fastest (the layout of
 *            interp_set_coeffs); read only; must not alias the handle's storage.
 *   taps     host, ntaps x s int32 lattice vectors with |v_a| <= 64; 1 <= ntaps <= 64.
 *   weights  host, ntaps FP32.
 * Sums are FP32 in tap order; the result is rounded once to the storage type.  Stream-ordered,
 * allocates nothing.  Errors: EINVAL (null pointer, ntaps out of range, a tap that is not a
 * lattice vector or too long), ECUDA.
 */
interp_status interp_prefilter(interp_t *h, const float *samples, int ntaps, const int32_t *taps, const float *weights,
                               void *stream);

/*
 * interp_eval -- out[q] = f(pts[q]) for q < npts (Sec. 4, Algorithm 1, per query: coset loop,
 * shift to the region of evaluation, symmetry fold, branch-free piece selection by plane sign
 * bits, coefficient gather, Horner evaluation in FP32 FMA).  npts = 0 is a no-op.  For splines
 * with interp_info_t.coop = 1 a warp gathers the stencil of one query per load instruction
 * (16 KB of static shared memory per 128-thread block); the results are the same bits as with
 * per-query gathers.
 */
interp_status interp_eval(const interp_t *h, const float *pts, int64_t npts, float *out, void *stream);

/*
 * interp_eval_grad -- out[q] = f(pts[q]) and grad[q*s + a] = d f / d x_a at pts[q], from the
 * analytic derivatives of the piece polynomials (not in the paper; same path as interp_eval).
 * out may be NULL when only the gradient is wanted.
 */
interp_status interp_eval_grad(const interp_t *h, const float *pts, int64_t npts, float *out, float *grad,
                               void *stream);

/*
 * interp_eval_host -- interp_eval / interp_eval_grad for HOST buffers (not in the paper): the
 * queries are copied to the device, evaluated and copied back in chunks of 2^20 queries, with the
 * copies of neighbouring chunks overlapping each other and the evaluation (two internal streams,
 * ordered after the work already queued on `stream`; `stream` waits for all of it before later
 * work).  For the copies to overlap, pts / out / grad must be page-locked host memory (cudaHostAlloc or
 * cudaHostRegister); pageable buffers work but serialise.  grad may be NULL (value only).  The
 * handle owns the device staging buffers (allocated on first use); calls on one handle must not
 * overlap.  Returns when the work is queued; synchronise `stream` before reading out / grad.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
interp_status interp_eval_host(interp_t *h, const float *pts, int64_t npts, float *out, float *grad, void *stream);

/*
 * interp_backward -- adjoint of interp_eval (not in the paper).  Given gout[q] = dLoss/df(pts[q]):
 *     dcoeffs[k][i] += sum_q gout[q] * phi(pts[q] - D i - l_k)      (FP32, caller's layout, +=)
 *     dpts[q*s + a]  = gout[q] * d f / d x_a (pts[q])               (if dpts != NULL)
 * dcoeffs has the coefficient layout of interp_set_coeffs (FP32) and is ACCUMULATED into: zero it
 * first for a plain gradient.  The scatter uses FP32 atomics into a handle-owned padded buffer,
 * so the order of additions, and the last bits of dcoeffs, vary between runs.  dcoeffs may be
 * NULL to compute dpts only.
 *   - 3-D splines with fewer than 4 pieces and at least 24 coefficient lookups per query, calls
 *     with many queries (the contributions outnumber the shared-memory boxes' sites at least four
 *     times; option "adjoint_bins" = 0 / 1 forces it off / on): the query indices are first
 *     counting-sorted on the device into spatial bins of 8^3 coset cells; each bin's contributions
 *     are summed in a shared-memory box and added to
 *     the padded buffer once per site.  The scratch (24 bytes per query plus 16 per bin) comes
 *     from the library's stream-ordered pool (see the piece pre-sort); under stream capture, or
 *     when the pool has no room, the call takes the path below.
 *   - Otherwise, 3-D splines: each block of 1024 consecutive queries whose cells fit a small box
 *     (e.g. after interp_sort_points) is summed in shared memory first, with one global atomic per
 *     touched coefficient; other blocks (and 4-D splines) add every contribution with its own
 *     atomic.
 */
interp_status interp_backward(interp_t *h, const float *pts, int64_t npts, const float *gout, float *dcoeffs,
                              float *dpts, void *stream);

/*
 * Batched evaluation (not in the paper): interp_eval over many handles of mixed lattice and spline
 * type in ONE persistent launch per dimension (3-D handles and 4-D handles), replayed from a CUDA
 * graph.  Work items are (handle, tile of queries); resident CTAs claim them from a counter, so
 * cheap and expensive splines balance across the GPU.  Every handle must use FP32 storage.
 *
 *   interp_batch_create    records the items (handles, point / output pointers, counts); the
 *                          pointers must stay valid for the batch's lifetime.  Allocates the
 *                          device descriptor table.  Errors: EINVAL, EUNSUPPORTED (16-bit
 *                          storage), ENOMEM, ECUDA.
 *   interp_batch_autotune  times the candidate tile sizes (256 .. 8192 queries) for each spline
 *                          in the batch on `stream` (running the batch several times: outputs
 *                          are overwritten) and keeps the fastest; blocks until done.
 *   interp_batch_tile /    read / set the tile size of a spline by name (e.g. to re-apply a
 *   interp_batch_set_tile  previous autotune result).  Tile sizes must be multiples of 128.
 *   interp_batch_run       out_i[q] = f_i(pts_i[q]) for every item: launches the batch's CUDA
 *                          graph (captured on the first run after create or a tile change) on
 *                          `stream`.  Runs of one batch must not overlap each other.
 *   interp_batch_destroy   releases it (NULL is a no-op).  Synchronises the device.
 */
typedef struct interp_batch interp_batch_t;
typedef struct {
    const interp_t *vol;   /* handle (FP32 storage)          */
    const float *pts;      /* device, npts x s, row-major    */
    int64_t npts;          /* >= 0                           */
    float *out;            /* device, npts                   */
} interp_batch_item;
interp_status interp_batch_create(const interp_batch_item *items, int n, interp_batch_t **out);
interp_status interp_batch_autotune(interp_batch_t *b, void *stream);
interp_status interp_batch_tile(const interp_batch_t *b, const char *spline, int *tile);
interp_status interp_batch_set_tile(interp_batch_t *b, const char *spline, int tile);
interp_status interp_batch_run(interp_batch_t *b, void *stream);
void interp_batch_destroy(interp_batch_t *b);

/*
 * interp_backward_noalloc -- the same adjoint as interp_backward, for callers that cannot call
 * cudaMalloc when they run it: plug-ins whose host application owns the device allocator, loops
 * with a fixed device-memory budget, and code paths where an allocation's implicit device
 * synchronisation is not acceptable.  The paper has no counterpart; it is a deployment variant.  It allocates nothing: its padded FP32 gradient scratch
 * is a static device array of INTERP_NOALLOC_MAX_GRAD_ELEMS floats (32 MiB) that every GPU which
 * loads this library holds until the process exits.  The caller still passes all inputs and
 * outputs (same arguments and semantics as interp_backward).
 *
 *   - Limit: when dcoeffs is not NULL, n_cosets * (elements of one padded FP32 coset array) must
 *     not exceed INTERP_NOALLOC_MAX_GRAD_ELEMS, else INTERP_ESIZE is returned and nothing runs.
 *     A dpts-only call (dcoeffs == NULL) does not use the array and has no such limit.
 *   - dpts is computed without the piece pre-sort (whose scratch comes from a memory pool), so
 *     no call allocates, whatever the spline and the number of queries.
 *   - The first call on a device (with that device current, which must be the handle's device)
 *     looks up the array's device address once; make that first call before any stream capture.
 *   - All calls share the one array and it keeps the previous call's contents; each call clears
 *     the part it uses first.  Calls that overlap on the GPU (other streams, other threads) race
 *     on it: serialise them.
 * Errors: EINVAL, ESIZE, ECUDA.
 */
#define INTERP_NOALLOC_MAX_GRAD_ELEMS 8388608
interp_status interp_backward_noalloc(interp_t *h, const float *pts, int64_t npts, const float *gout,
                                      float *dcoeffs, float *dpts, void *stream);

/*
 * interp_eval_rays -- ray-coherent queries (not in the paper; the paper's timings come from a
 * volume renderer that marches rays through mostly transparent volumes, Sec. 5.1).  For every
 * pixel (px, py) of a width x height image, the ray starts at
 *     o = origin + (px + 1/2) du + (py + 1/2) dv
 * and runs along dir (any length); its chord with the box [box_lo, box_hi] is split into `steps`
 * equal steps sampled at their midpoints (rays that miss the box give 0).  Output per pixel
 * (row-major, pixel = py * width + px):
 *     with_grad = 0:  out[pixel]         = sum over samples of f
 *     with_grad = 1:  out[4*pixel + 0]   = sum of f,  out[4*pixel + 1 + a] = sum of d f / d x_a
 * pts_out (NULL or width*height*steps*3 floats) receives every sample point (NaN for missed rays).
 * 3-D splines with FP32 storage only (else EUNSUPPORTED).  Errors: EINVAL, EUNSUPPORTED, ECUDA.
 */
typedef struct {
    float origin[3], du[3], dv[3], dir[3], box_lo[3], box_hi[3];
    int32_t width, height, steps;
} interp_rays_t;
interp_status interp_eval_rays(const interp_t *h, const interp_rays_t *rays, int with_grad, float *out,
                               float *pts_out, void *stream);

/*
 * interp_sort_points -- reorder queries so that queries close in space are close in the array (not
 * in the paper).  Bins of 4 x 4 x 4 cells (2 per axis in 4-D) in Morton order; a counting sort.
 * perm[r] (int32, npts) = the original index of the query at sorted position r, and/or
 * pts_sorted[r*s + a] = pts[perm[r]*s + a]; either may be NULL (not both).  The order inside a
 * bin is unspecified.  Evaluating sorted queries reuses coefficients in L1, and interp_backward
 * on sorted queries sums most contributions in shared memory instead of global atomics.  The
 * handle owns the bin counters (allocated on first use); calls on one handle must not overlap.
 * Errors: EINVAL, ESIZE (npts >= 2^31), ENOMEM, ECUDA.
 */
interp_status interp_sort_points(interp_t *h, const float *pts, int64_t npts, int32_t *perm, float *pts_sorted,
                                 void *stream);

/*
 * interp_debug_indices -- for every query q and coset k: cells[(q*M + k)*s + a] = the index i of
 * the nearest coset site (the exact shift rho of Sec. 4.1 to the cube [-D/2, D/2)^s), and
 * piece[q*M + k] = the sub-region index j (Sec. 4.2) of the folded offset.  Either pointer may
 * be NULL.
 */
interp_status interp_debug_indices(const interp_t *h, const float *pts, int64_t npts, int32_t *cells,
                                   int32_t *piece, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* INTERP_B300_H */
