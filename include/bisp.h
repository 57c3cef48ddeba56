/*
 * bisp.h -- C ABI of the GB300 estimator of the redshift-space bispectrum
 * multipoles B_l^m(k1, mu, t) of Gill & Bharadwaj, "Brisk estimator for the
 * angular multipoles of the redshift space bispectrum" (arXiv:2405.14513).
 *
 * The estimator (Sec. II of the paper):
 *   - transforms the gridded field, Delta(k) = (V/N_g^3) sum_x delta(x)
 *     exp(-i k.x), with the line of sight along z (Eq. bs);
 *   - splits k-space into planes n perpendicular to the line of sight and
 *     annular rings r in each plane, ring widths 2^floor((r-1)/10) grid
 *     units, outer radius capped at N_g/3 (Fig. 1, implementation paragraph);
 *   - forms D(r,n,x) = sum_{u in r} Delta(u, n) exp(-i u.x) (Eq. iFT) and, for
 *     every combination of three rings and two planes (n3 = -n1 - n2),
 *     S = sum_x D(r1,n1) D(r2,n2) D(r3,n3) (Eq. fftbs) and the triangle count
 *     N_tri = N_g^-2 sum_x I1 I2 I3 of the unit fields (Eqs. Ntri2, 2FT);
 *   - maps each combination to (p, k1, mu, t) (Eqs. shape, orient) and bins
 *     B_l^m = sqrt((2l+1)/4pi) sum Y* Bhat N_tri / sum |Y|^2 N_tri
 *     (Eq. bs_lm2_1), Bhat = S / (V N_tri N_g^2).
 * The library computes every step on the GPU; it has no CPU fallback.
 *
 * Conventions shared by all entry points:
 *   - the input field delta[x][y][z] is real, z (the line of sight) is the
 *     last and contiguous axis; N_g^3 values of float (precision FP32 or
 *     MIXED) or double (precision FP64);
 *   - the output B[batch][n_k1][n_mu][n_t][n_lm] is double; the moment axis
 *     holds even l only, (l, m) = (0,0), (2,0), (2,1), (2,2), (4,0) ...
 *     (l_max, l_max), so n_lm = (l_max/2 + 1)^2; empty bins hold NaN;
 *   - k1 bins are given by edges (units of k_f = 2 pi / L); mu and t bins
 *     are uniform on [0.5, 1], bin index floor((x - 0.5) 2 n), the top edge
 *     closed;
 *   - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Device pointers must be valid on the current device;
 *   - every function returns a status code (bisp_status) and never throws
 *     across the ABI; estimator_last_error() describes the last failure of
 *     the calling thread.
 */
#ifndef BISP_H
#define BISP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BISP_OK = 0,
    BISP_INVALID_ARG = 1,       /* a parameter is out of range or inconsistent */
    BISP_UNSUPPORTED_SIZE = 2,  /* N_g is not 2^k or 3 x 2^k in [8, 1024]     */
    BISP_OUT_OF_MEMORY = 3,     /* a device or host allocation failed         */
    BISP_CUDA_ERROR = 4,        /* a CUDA call or kernel launch failed        */
    BISP_TIMEOUT = 5,           /* a bounded device wait gave up              */
    BISP_INTERNAL = 6           /* an internal consistency check failed       */
} bisp_status;

typedef enum {
    BISP_PREC_FP32 = 0,     /* FP32 transforms, products and sums ("plain")                */
    BISP_PREC_MIXED = 1,    /* FP32 transforms and products, FP64 sums and binning         */
    BISP_PREC_FP64 = 2,     /* FP64 throughout (verification)                               */
    BISP_PREC_MIXED_TC = 3  /* as MIXED, with the triple sums on the tensor cores: TF32     */
                            /* mma with each FP32 operand split into two TF32 parts        */
} bisp_precision;

/* Opaque plan: ring tables, triangle counts, combination tables, bin
 * denominators and twiddles for one (N_g, L, bins, l_max, precision).  Owned
 * by the library; created by estimator_plan, released by estimator_destroy. */
typedef struct bisp_plan bisp_plan;

typedef struct {
    int n_g;                  /* grid points per side, 2^k or 3 x 2^k, 8..1024    */
    double box_len;           /* L > 0; V = L^3, k_f = 2 pi / L                   */
    int n_k1;                 /* number of k1 bins, >= 1                          */
    const double *k1_edges;   /* HOST pointer, n_k1 + 1 strictly ascending edges, */
                              /* k1_edges[n_k1] <= (N_g/3) k_f                     */
    int n_mu, n_t;            /* uniform mu and t bins on [0.5, 1], each >= 1      */
    int l_max;                /* even, 0..8                                        */
    int precision;            /* bisp_precision                                    */
    int max_batch;            /* largest batch passed to estimator_estimate, 1..65535 */
    const int *n_mu_l;        /* optional HOST pointers, both or neither (NULL): l_max/2 + 1 */
    const int *n_t_l;         /* entries, the (mu, t) bins of the moments of order l = 0, 2, */
                              /* .., l_max (each in [1, 4096]); n_mu and n_t are then      */
                              /* ignored.  Not kept after estimator_plan returns.  The      */
                              /* paper bins l = 0, 2 finer than l = 4, 6 (Sec. III.B,        */
                              /* appendix); see bisp_view_info for the output layout.       */
} bisp_desc;

typedef struct {
    int n_g, n_rings, n_planes;      /* rings per plane; planes 0..N_g/3 stored     */
    int l_max, n_lm, n_k1, n_mu, n_t;
    int n_levels;                    /* number of reduction grids in use             */
    int64_t n_bins;                  /* n_k1 n_mu n_t                                 */
    int64_t n_combos;                /* accepted combinations, one of each +-n pair   */
    int64_t n_pairs;                 /* plane pairs (n1, n2) with a combination       */
    int64_t n_items;                 /* Step-II blocks (pair, grid, x chunk, tiles)   */
    double triple_products;          /* sum over combinations of the points of its    */
                                     /* smallest exact reduction grid                 */
    size_t dstore_bytes;             /* D-field store of one field                    */
    size_t workspace_bytes;          /* estimator_workspace_bytes(plan, 1)            */
    size_t resident_bytes;           /* device memory owned by the plan               */
    int n_views;                     /* binnings (bisp_view_info), >= 1                */
    int64_t out_doubles;             /* doubles of B per field (all views)            */
    double pair_products;            /* distinct pair products D1 D2 on those grids   */
    /* Step-II work on the tensor cores (MIXED_TC; 0 otherwise), in grid points: */
    double tc_row_points;            /* pair products the tiles form (rows x points;   */
                                     /* each (pair, r1, r2) once, on the largest grid  */
                                     /* its r3 need)                                    */
    double tc_lane_points;           /* tensor-memory lanes x points of all tiles      */
    double tc_mma_products;          /* lanes x window columns x points (MMA work)     */
    double tc_staged_bytes;          /* bytes the tiles copy from L2 into shared memory */
} bisp_plan_info;

/* A binning of the output.  Consecutive even l with the same (mu, t) grid
 * share a view; without per-l grids there is one view, l = 0 .. l_max on
 * n_mu x n_t, and B of a field is exactly [n_k1][n_mu][n_t][n_lm].  In
 * general B of a field is the views' blocks one after another, block v
 * [n_k1][n_mu][n_t][n_lm] (its own n_mu, n_t, n_lm) at `offset` doubles;
 * moments in the order (l, m) = (l_lo, 0) .. (l_hi, l_hi), even l. */
typedef struct {
    int l_lo, l_hi;                  /* even orders of the view's moments            */
    int n_mu, n_t;                   /* its (mu, t) grid                             */
    int n_lm;                        /* moments: (l_hi/2 + 1)^2 - (l_lo/2)^2          */
    int64_t n_bins;                  /* n_k1 n_mu n_t                                 */
    int64_t offset;                  /* first double of the block in a field's B      */
} bisp_view_info;

/* Build a plan (Sec. II: ring table, N_tri by Eq. Ntri2 on the GPU in FP64,
 * combination table with its (k1, mu, t) bins and the field-independent
 * denominators of Eq. bs_lm2_1).  Allocates device memory owned by the plan;
 * work is ordered on `stream` and complete on return.  *out is set to NULL
 * on failure. */
int estimator_plan(bisp_plan **out, const bisp_desc *desc, void *stream);

/* Plan summary.  info: host pointer. */
int estimator_plan_info(const bisp_plan *plan, bisp_plan_info *info);

/* Binning `view` (0 <= view < n_views) of the plan's output.  info: host
 * pointer.  BISP_INVALID_ARG for a view out of range. */
int estimator_view_info(const bisp_plan *plan, int view, bisp_view_info *info);

/* Bytes of device workspace estimator_estimate needs for `batch` fields
 * (0 on a bad argument): batch regions of one field's size.  All fields of
 * a batch go through every stage in the same kernel launches (one more
 * grid dimension), each in its own region. */
size_t estimator_workspace_bytes(const bisp_plan *plan, int batch);

/* Estimate B_l^m for `batch` fields (1 <= batch <= max_batch).
 *   delta:     DEVICE pointer, [batch][N_g][N_g][N_g] float or double (see
 *              precision), read only;
 *   workspace: DEVICE pointer to >= estimator_workspace_bytes(plan, batch)
 *              bytes, 256-byte aligned, owned by the caller; contents are
 *              scratch between calls;
 *   B:         DEVICE pointer, [batch][out_doubles] double: per field the
 *              views' blocks (bisp_view_info); with one view
 *              [batch][n_k1][n_mu][n_t][n_lm].
 * Asynchronous: all work is ordered on `stream`.  An estimate only reads
 * the plan's device tables and writes its workspace and B, so estimates of
 * one plan may overlap on the device (on different streams) when each has
 * its own workspace and B and stage timing (estimator_set_timing) is off.
 * Calls that share a workspace must not overlap.  Host calls on one plan
 * are not thread safe: make them from one thread. */
int estimator_estimate(bisp_plan *plan, const void *delta, int batch, void *workspace,
                       double *B, void *stream);

/* Same estimate from and to HOST memory: copies delta in, runs, copies B out,
 * and returns when B is complete (and its wait status is checked).  The plan
 * allocates (once, on first use) its own device workspace and staging
 * buffers for max_batch fields, so calls of this kind on one plan must not
 * overlap. */
int estimator_estimate_host(bisp_plan *plan, const void *delta_host, int batch, double *B_host,
                            void *stream);

/* Streaming estimates from and to HOST memory, for a caller with a sequence
 * of fields in host memory: the copy of each field in overlaps the estimate
 * of the one before.  estimator_host_submit queues the copy of delta_host to
 * the device (on a copy stream the plan owns), the estimate and the copy of
 * its B to B_host (on `stream`) and returns at once; estimator_host_wait
 * returns when the oldest submission's B_host is complete, with its wait
 * status (as estimator_workspace_status).  At most two submissions are in
 * flight (a third submit is BISP_INVALID_ARG; a wait with none is
 * BISP_INVALID_ARG).  delta_host ([batch][N_g]^3 as for estimator_estimate)
 * and B_host ([batch][out_doubles]) must stay valid and unchanged until the
 * submission's wait returns; page-locked host memory makes the copies
 * asynchronous.  Submit on one stream; the plan allocates (once) two input
 * and two output buffers and shares its workspace with
 * estimator_estimate_host, so the two host forms must not overlap.  (The
 * paper has no counterpart: it reads each field from disk.) */
int estimator_host_submit(bisp_plan *plan, const void *delta_host, int batch, double *B_host, void *stream);
int estimator_host_wait(bisp_plan *plan, void *stream);

/* One share of an estimate, for splitting one field over several devices
 * (each holding its own plan).  The numerator of Eq. bs_lm2_1 is a sum over
 * combinations of Re Y_lm S (S of Eq. fftbs), so it splits over any
 * partition of the combinations; this call runs the transforms and Step I
 * whole and the Step-II triple sums of share `part` of `nparts` (the
 * Step-II blocks of each kind split into nparts contiguous runs of about
 * equal cost), and writes
 *   B_part = sqrt((2l+1)/4pi) num_part / (V N_g^2 den),
 * num_part the numerator over the share's combinations, den the whole
 * denominator (plan-resident), NaN where den = 0.  The element-wise sum of
 * B_part over part = 0 .. nparts - 1 is B of estimator_estimate up to FP64
 * rounding (NaN bins stay NaN): one sum-reduction of the output between
 * devices completes the estimate.  Arguments as for estimator_estimate;
 * 0 <= part < nparts, else BISP_INVALID_ARG.  nparts = 1 is the whole
 * estimate.  (The paper has no counterpart: it runs on one CPU node.) */
int estimator_estimate_part(bisp_plan *plan, const void *delta, int batch, void *workspace, double *B_part,
                            int part, int nparts, void *stream);

/* Running statistics of B over many fields (mocks): the spread of the
 * estimates over realisations is what the paper compares deviations with
 * (Sec. III.B).  For i < n, the values B[f][i], f = 0 .. batch - 1, join
 * count[i], mean[i] and m2[i] (sum of squared deviations from the mean) by
 * Welford's update in FP64, in field order; non-finite values (empty bins)
 * are skipped.  The sample variance is m2 / (count - 1).  All DEVICE
 * pointers: B [batch][n] (n = out_doubles for whole outputs), count, mean,
 * m2 [n], zero before the first update, owned by the caller.
 * Stream-ordered.  (The paper has no counterpart: it reports its 50
 * realisations' spread without saying how it was accumulated.) */
int estimator_stats_update(const double *B, int batch, int64_t n, int64_t *count, double *mean, double *m2,
                           void *stream);

/* ---------------- captured estimates (CUDA graphs) ---------------- */

typedef struct bisp_graph bisp_graph;

/* Capture the launches of one estimator_estimate(plan, delta, batch,
 * workspace, B) into a CUDA graph and instantiate it; the arguments keep
 * their meaning and must stay valid while the graph exists.  Capture runs
 * on `stream` (or, when it is NULL, on a stream of the library's); nothing
 * is computed.  Stage timing is off while capturing.  *out is NULL on
 * failure.  (The paper has no counterpart: this removes the per-launch
 * host cost when many fields are estimated with one plan.) */
int estimator_graph_create(bisp_graph **out, bisp_plan *plan, const void *delta, int batch, void *workspace,
                           double *B, void *stream);

/* Run a captured estimate on `stream` (asynchronous, stream-ordered). */
int estimator_graph_launch(bisp_graph *graph, void *stream);

/* Release a captured estimate (NULL is a no-op); no launch of it may still
 * be running. */
void estimator_graph_destroy(bisp_graph *graph);

/* Device-side status of one estimate: synchronises `stream`, then returns
 * BISP_TIMEOUT if a tensor-core Step-II block of the last estimate run in
 * `workspace` gave up a bounded wait for one of its `batch` fields (those
 * combinations then hold NaN, and so do the bins they enter), else BISP_OK.
 * The status lives in the workspace (one word per field, cleared at the start
 * of every estimate and by this call when set), so estimates in different
 * workspaces report separately.  workspace: the DEVICE pointer given to
 * estimator_estimate, or NULL for the array of estimator_estimate_static.
 * estimator_estimate_host checks it after every call.  (The paper has no
 * counterpart: this reports the library's own wait bounds.) */
int estimator_workspace_status(const bisp_plan *plan, const void *workspace, int batch, void *stream);

/* Polls after which the tensor-core Step II's waits on its producer, compute
 * and MMA-issue stages give up (spins >= 1; 0 restores the default, 2^22).
 * The wait for the block's own MMAs before it frees its tensor memory keeps
 * the full bound.  A poll may suspend the waiting thread for a while before
 * it reports; below 64 polls each poll reports at once instead, so a small
 * limit really cuts the waits short.  A host-side knob for exercising the
 * give-up path (a block that gives up writes NaN sums and sets the workspace
 * status); it applies to later estimates of the plan.  (The paper has no
 * counterpart.) */
int estimator_set_wait_limit(bisp_plan *plan, int spins);

/* Release the plan and everything it owns (NULL is a no-op).  The caller
 * makes sure no work that uses the plan is still running. */
void estimator_destroy(bisp_plan *plan);

/* Static description of a status code. */
const char *estimator_status_string(int status);

/* Description of the last failure on the calling thread ("" if none). */
const char *estimator_last_error(void);

/* ---------------- spherical-shell estimator of the m = 0 multipoles ---------------- */

/* A comparison for the m = 0 subset.  The shell-based FFT estimators the
 * paper builds on (Sec. I) bin modes in spherical shells and weight each
 * mode by its own direction, which reaches only the m = 0 moments:
 *   shells  s = {k : e_s <= |k| < e_{s+1}} (3D |k|, the ring edges of Sec. II);
 *   triples s1 >= s2 >= s3 >= 1, binned in (k1, mu, t) from the shells' mean
 *           radii as a ring combination is, kept when N_tri > 0;
 *   num_l = sum Y_l0(k1) Delta(k1) Delta(k2) Delta(k3), den_l = sum Y_l0(k1)^2
 *           over closed triangles with k_i in s_i (on the N_g^3 grid);
 *   B_l^0 = sqrt((2l+1)/4pi) sum num_l / (V sum den_l) per bin (even l), NaN
 *           where the denominator is 0.
 * desc as for estimator_plan except: N_g <= 128, l_max <= 6, precision,
 * max_batch and per-l grids ignored (FP32 fields and products, FP64 sums;
 * FP64 plan-time counts and denominators).  B: DEVICE [n_k1][n_mu][n_t]
 * [l_max/2 + 1].  delta: DEVICE float [N_g][N_g][N_g].  workspace: DEVICE,
 * estimator_shell_info's workspace_bytes, 256-byte aligned.  (The paper
 * has no counterpart in its own method; it cites this family.) */
typedef struct bisp_shell_plan bisp_shell_plan;
int estimator_shell_plan(bisp_shell_plan **out, const bisp_desc *desc, void *stream);
int estimator_shell_info(const bisp_shell_plan *plan, int *n_shells, int64_t *n_triples, size_t *workspace_bytes);
int estimator_shell_estimate(bisp_shell_plan *plan, const float *delta, void *workspace, double *B, void *stream);
/* Accepted triples, HOST pointers (each may be NULL): tri [n][4] = s1, s2,
 * s3, flat (k1, mu, t) bin; ntri [n]; den [n][l_max/2 + 1]. */
int estimator_shell_triples(const bisp_shell_plan *plan, int32_t *tri, double *ntri, double *den);
/* After estimator_shell_estimate on this workspace: num [n][l_max/2 + 1]
 * (HOST), synchronising `stream`. */
int estimator_shell_sums(const bisp_shell_plan *plan, const void *workspace, double *num, void *stream);
void estimator_shell_destroy(bisp_shell_plan *plan);

/* ---------------- estimate without caller-provided workspace ---------------- */

/* estimator_estimate for callers that cannot allocate device memory: code
 * under a memory manager that owns the whole device heap (a framework's
 * caching allocator, a serving runtime with fixed pools) and must not see
 * stray allocations, and plugins handed a device and a stream but no
 * allocator.  (The paper has no counterpart: this is a deployment entry
 * point.)
 *   delta, batch, B, stream: as for estimator_estimate (DEVICE pointers);
 *   the workspace is a file-scope device array of the library,
 *   estimator_static_scratch_bytes() = 64 MiB, held on every GPU where the
 *   library is loaded until the process exits.
 * Allocates nothing.  Returns BISP_INVALID_ARG (see estimator_last_error)
 * when the plan's workspace for `batch` fields is larger than the array.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (on any
 * streams, with any plans) race and give wrong results; serialise them.
 * Stage timing (estimator_set_timing) must be off for the call to allocate
 * nothing (timing creates CUDA events). */
int estimator_estimate_static(bisp_plan *plan, const void *delta, int batch, double *B, void *stream);

/* Bytes of the device array used by estimator_estimate_static. */
size_t estimator_static_scratch_bytes(void);

/* ---------------- stage timing ---------------- */

/* Stages timed by estimator_stage_times. */
typedef enum {
    BISP_STAGE_FORWARD = 0,   /* forward 3D transform (z, y, x passes)          */
    BISP_STAGE_STEP1 = 1,     /* ring-masked 2D transforms on each grid (Eq. iFT) */
    BISP_STAGE_STEP2 = 2,     /* triple-product reduction (Eq. fftbs)            */
    BISP_STAGE_REDUCE = 3,    /* partial sums -> per-combination sums            */
    BISP_STAGE_BIN = 4,       /* Y_lm weighting, binning, ratio (Eq. bs_lm2_1)   */
    BISP_N_STAGES = 5
} bisp_stage;

/* Switch per-stage timing on (1) or off (0) for the following estimates.
 * When on, every estimate records CUDA events on its stream around each
 * stage (one event pair per stage and field).  Switching on clears the
 * totals. */
int estimator_set_timing(bisp_plan *plan, int on);

/* Totals since timing was switched on: ms[BISP_N_STAGES] elapsed time per
 * stage (CUDA events, device clock), launches[BISP_N_STAGES] kernels
 * launched per stage.  HOST pointers; either may be NULL.  Waits for the
 * recorded events. */
int estimator_stage_times(bisp_plan *plan, double *ms, int64_t *launches);

/* Algorithmic floating-point operations of one estimate of one field, per
 * stage (HOST pointer flops[BISP_N_STAGES]): for Step II, 4 per grid point of
 * each combination (Re of a complex product, two FMAs) plus 6 per grid
 * point of each distinct (plane pair, grid, r1, r2) product D1 D2. */
int estimator_stage_flops(const bisp_plan *plan, double *flops);

/* ---------------- introspection, for tests and diagnostics ---------------- */

/* Denominators sum_c |Y_lm(p_c)|^2 N_tri,c of Eq. bs_lm2_1 (counted over both
 * members of each +-n pair).  den: HOST pointer [out_doubles], laid out as
 * a field's B. */
int estimator_denominator(const bisp_plan *plan, double *den);

/* Accepted combinations, one of each pair (n1, n2) / (-n1, -n2), kept with
 * n1 > 0 or (n1 == 0 and n2 >= 0), in the library's internal order.  HOST
 * pointers with room for `cap` rows (any may be NULL):
 *   ints[k][6] = n1, n2, n3, r1, r2, r3 (rings 0-based); ntri[k]; bin[k] =
 *   flat (k1, mu, t) bin; grid[k] = side of the grid its sum runs on.
 * Returns the number of combinations (even when larger than cap), < 0 on error. */
int64_t estimator_combo_table(const bisp_plan *plan, int64_t cap, int32_t *ints, int64_t *ntri,
                              int32_t *bin, int32_t *grid);

/* Shape and orientation of each accepted combination, in estimator_combo_table
 * order (Eqs. shape and orient; Sec. II, the mapping of a combination to
 * (p, k1, mu, t) through its mean ring radii): geo[k][4] = mu, t, p_z and
 * cos phi (the azimuth of the line of sight in the triangle's frame; 1 for a
 * linear triangle).  geo: HOST pointer with room for `cap` rows.  Returns
 * the number of combinations (even when larger than cap), < 0 on error. */
int64_t estimator_combo_geometry(const bisp_plan *plan, int64_t cap, double *geo);

/* After estimator_estimate on this workspace: the real parts of the sums
 * S = sum_x D1 D2 D3 of Eq. fftbs (full N_g^2 grid normalisation) of the last
 * field of the batch, in estimator_combo_table order (the imaginary parts
 * cancel between the members of each +-n pair and are not formed).  S: HOST
 * pointer [n_combos].  Synchronises `stream`. */
int estimator_combo_sums(const bisp_plan *plan, const void *workspace, double *S, void *stream);

/* After estimator_estimate on this workspace: D(r, n, x) of Eq. iFT of the
 * last field at the M x M points x = (N_g/M) y, y integer, i.e.
 * sum_{u in r} Delta(u, n) exp(-2 pi i u.y / M), as stored for the Step-II
 * reduction.  M is one of the plan's reduction grid sides (F x 2^q, F = 1,
 * 3, 5 or 7, a multiple of 4, 8 <= M <= N_g).  out: HOST pointer [M][M][2]
 * (y_x slow, y_y fast), in double.  Returns BISP_INVALID_ARG when (M, n, r) is not stored. */
int estimator_dfield(const bisp_plan *plan, const void *workspace, int M, int n, int r,
                     double *out, void *stream);

/* After estimator_estimate on this workspace: plane n (0 <= n <= N_g/3) of
 * the transformed field Delta(kx, ky, n), FFT index order.  out: HOST pointer
 * [N_g][N_g][2] double. */
int estimator_delta_plane(const bisp_plan *plan, const void *workspace, int n, double *out,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BISP_H */
