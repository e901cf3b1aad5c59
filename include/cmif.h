/*
 * cmif.h -- C ABI of the GB300 CMIF library (libcmif.so).
 *
 * The cross-mutual information function (Eq. cmif) of two label images A
 * and B with region-of-interest masks M_A, M_B (Sec. 3.1):
 *
 *     CMIF(chi; A, B) = I(A, T_chi[B]),   T_chi[B](x) = B(x + chi),
 *
 * the mutual information (Eq. mi / Eq. mientropy) of the label pairs
 * (A(x), B(x + chi)) over the pixels where both masks are 1, for every
 * integer displacement chi of the full linear range
 *
 *     chi = (dy, dx),  dy in [-(H_A-1), H_B-1],  dx in [-(W_A-1), W_B-1].
 *
 * It is computed by the frequency-domain method of Sec. 3.2: the joint
 * counts C_AB^{a,b}(chi) are the cross-correlations (Eq. cc) of the level
 * sets L_a[A] and L_b[B] (Eq. correlationjointhisto), computed with FFTs
 * and rounded to integers, which makes them identical to the direct
 * method's histogram counts (Sec. 3.4).  The marginal counts and N
 * (Eq. correlationmarghisto, Eq. number) are the exact integer sums of the
 * joint counts, and the entropies of Eq. finalentropy are reduced per shift
 * in fixed point.  MI is in bits; 0/0 = 0 and 0 log 0 = 0, so MI = 0 where
 * N = 0.
 *
 * Map layout (all maps): row-major, R = H_A + H_B - 1 rows by
 * C = W_A + W_B - 1 columns; element (r, c) is chi = (r - (H_A-1), c - (W_A-1)).
 *
 * Images: A is int32 H_A x W_A row-major, M_A is uint8 H_A x W_A (nonzero = 1)
 * or NULL for all ones; likewise B, M_B.  Where a mask is 1 the label must
 * lie in [0, K); where it is 0 the label is ignored.
 *
 * Memory: every array argument of cmif_compute / cmif_align_rotations is a
 * DEVICE pointer owned by the caller, on the plan's device.  The plan owns
 * its workspace (allocated by cmif_plan_create*, freed by
 * cmif_plan_destroy); compute calls allocate nothing.  Calls are
 * asynchronous and stream-ordered on the given stream (a cudaStream_t; NULL
 * is the legacy default stream).  A plan must not be used by two calls that
 * may overlap in time (different streams, different threads).
 *
 * Errors: the return value reports argument and launch errors found on the
 * host, synchronously.  Problems found on the device (a label out of range,
 * a rounding residual the chosen precision could not bring under the guard)
 * are recorded in the plan's device status word and read with
 * cmif_get_status(), which synchronises.
 */
#ifndef CMIF_H
#define CMIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cmif_plan_s* cmif_plan;

typedef enum {
    CMIF_OK = 0,
    CMIF_ERR_INVALID_ARG = 1,      /* bad size, K, pointer, gamma, precision or flag          */
    CMIF_ERR_LABEL_RANGE = 2,      /* device: a label under mask 1 lies outside [0, K)        */
    CMIF_ERR_OOM = 3,              /* workspace allocation failed                             */
    CMIF_ERR_CUDA = 4,             /* a CUDA runtime call or launch failed                    */
    CMIF_ERR_PRECISION = 5,        /* device: rounding residual >= 0.25 in the final precision */
    CMIF_ERR_TIMEOUT = 6,          /* device: a bounded wait gave up                          */
    CMIF_ERR_NOT_IMPLEMENTED = 7,  /* precision or mode not built                             */
    CMIF_ERR_UNSUPPORTED = 8       /* size beyond the supported transform lengths             */
} cmif_status;

/* Arithmetic of the FFT correlations.  Counts are exact when every pre-rounding
 * residual |c - round(c)| stays below 0.25 (checked on every call).
 *   CMIF_FP32   : FP32 transforms (fast; exact for balanced labels up to ~1024^2)
 *   CMIF_SPLIT32: two-term FP32 transforms (hi + lo floats, ~48 significant
 *                 bits from FP32 units; exact everywhere in range)
 *   CMIF_FP64   : FP64 transforms (exact everywhere in range; slow on GB300)
 *   CMIF_AUTO   : FP32 transforms with the precision chosen per label pair,
 *                 all on the device (no host round trip).  A predicate sends a
 *                 pair to the second precision up front when the estimated
 *                 FP32 error of its correlation, 0.25 * 2^-24 * log2(P Q) *
 *                 sqrt(|X_a| |Y_b|) (|X_a|, |Y_b|: the two labels' pixel counts
 *                 under the masks), reaches half the guard; the FP32 pass takes
 *                 those pairs' exact counts and records every other pair's
 *                 residual; pairs that still reach the guard are computed in
 *                 the second precision as well and the FP32 row pass runs once
 *                 more.  Only the listed pairs (at most 128 per map) pay for
 *                 the second precision.  The second precision is two-term FP32;
 *                 the environment variable CMIF_AUTO_TIER2=fp64 at plan creation
 *                 makes it FP64, CMIF_AUTO_PREDICATE=0 turns the predicate
 *                 off (the guard alone then picks the pairs) and
 *                 CMIF_AUTO_PREDICATE=all sends every pair (up to the 128-pair
 *                 list) to the second precision (diagnostics). */
typedef enum { CMIF_FP32 = 0, CMIF_SPLIT32 = 1, CMIF_FP64 = 2, CMIF_AUTO = 3 } cmif_precision;

/* Plan flags. */
#define CMIF_FLAG_DEBUG_COUNTS 1u /* allow a non-NULL counts output in cmif_compute */
#define CMIF_FLAG_GRAPH 2u        /* capture each call's launches in a CUDA graph once and replay it while the
                                     call's arguments (pointers, gamma, angles) are unchanged */
#define CMIF_FLAG_WINDOW 4u       /* Alg. 1's padded search window (Sec. 3.6, Alg. 1's ZERO-PAD step: A and M_A zero-padded
                                     by p_i = ceil(|X_B|_i (1 - gamma)) along each axis).  X_S becomes the shifts
                                     that keep B's domain inside padded A's: chi_i in [|X_B|_i - |X_A|_i - p_i, p_i]
                                     (|chi_i| <= p_i for equal sizes), intersected with the full range.  Only the
                                     window's map rows are computed (rows outside it are returned as MI = 0,
                                     N = 0); max N and the peak are taken over the window.  A call whose window
                                     is empty (B cannot fit inside padded A) returns CMIF_ERR_INVALID_ARG. */
#define CMIF_FLAG_NMI 8u          /* the map (mi_map, mi_maps) holds the normalised MI the paper cites next to MI
                                     (Sec. 2.1), NMI = (H_A + H_B) / H_AB, from the same counts and fixed-point
                                     entropy sums; 0 where N = 0 or H_AB = 0 (0/0 = 0, Sec. 3.2).  Alg. 1's
                                     argmax and the peaks then maximise NMI. */
#define CMIF_FLAG_WEIGHTED 16u    /* the plan computes spatially weighted MI with cmif_compute_weighted (needs
                                     CMIF_FP64; not with CMIF_FLAG_NMI or CMIF_FLAG_DEBUG_COUNTS) */
#define CMIF_FLAG_AUTOTUNE 32u    /* run cmif_plan_autotune at creation (cache file: the environment variable
                                     CMIF_TUNE_CACHE, or none) */
#define CMIF_FLAG_BATCH_ANGLES 64u /* FP32 image plans: cmif_align_rotations runs up to 64 angles per launch of
                                     each stage (warp, B's transforms, pair products, row epilogue, peaks), as
                                     many as 40% of the free device memory at creation holds (the environment
                                     variable CMIF_ANGLE_BATCH caps it); the workspace grows accordingly.
                                     Results equal the angle-by-angle ones.  Ignored by other plans. */

/* One argmax record of Alg. 1: the displacement chi = (dy, dx) maximising
 * CMIF among shifts with N(chi) >= gamma * max N, for transform angle_idx
 * (-1: identity / none).  24 bytes, naturally aligned. */
typedef struct {
    int32_t angle_idx;
    int32_t dy;
    int32_t dx;
    int32_t n;
    double mi;
} cmif_peak;

/* Create a plan for equal-sized images H x W with K_A, K_B labels.
 * Same as cmif_plan_create_ex(out, H, W, H, W, K_A, K_B, prec, 0). */
cmif_status cmif_plan_create(cmif_plan* out, int H, int W, int K_A, int K_B, cmif_precision prec);

/* Create a plan (Sec. 3.1: domains X_A, X_B rectangular, any sizes).
 *   H_A, W_A, H_B, W_B >= 1, H*W <= 2^22 per image; 1 <= K_A, K_B <= 64;
 *   the transform sizes P >= H_A+H_B-1 and Q >= W_A+W_B-1 must not exceed
 *   4096 (else CMIF_ERR_UNSUPPORTED).  They are the smallest powers of two
 *   (at least 16) or, for CMIF_FP32 plans, the smallest 3 * 2^k (96 .. 3072)
 *   when that is smaller (CMIF_POW2_ONLY=1 in the environment at creation
 *   keeps powers of two).  Q keeps the power of two 512, 1024 or 2048 when the
 *   Tensor-Memory row kernel runs it (plans without count maps; faster than a
 *   shorter 3 * 2^k width; CMIF_ROWS_POW2=0 keeps the shortest width).  The
 *   counts and MI do not depend on the choice.
 *   prec: see cmif_precision.  flags: CMIF_FLAG_*.
 * Allocates the workspace on the current CUDA device, which becomes the
 * plan's device.  On error *out is NULL.  The environment variable
 * CMIF_DISABLE_TMEM=1 at creation makes FP32 plans use the shared-memory row
 * kernel instead of the Tensor-Memory one, and CMIF_COL_M=16 the 16-lane
 * column-team variant of the FP32 column transforms (P >= 1024; one of the
 * autotuner's candidates); same results, for comparison. */
cmif_status cmif_plan_create_ex(cmif_plan* out, int H_A, int W_A, int H_B, int W_B, int K_A, int K_B,
                                cmif_precision prec, unsigned flags);

/* Create a plan for VOLUMES (Sec. 3.1 with n = 3: the domains are boxes):
 * A is D_A x H_A x W_A, B is D_B x H_B x W_B (slice-major int32; masks uint8
 * of the same shape or NULL).  cmif_compute then returns the CMIF over every
 * displacement chi = (dz, dy, dx), dz in [-(D_A-1), D_B-1] (dy, dx as for
 * images), as maps of (D_A + D_B - 1) * (H_A + H_B - 1) rows by C columns,
 * depth-offset major: map row (D_A - 1 + dz) * (H_A + H_B - 1) + (H_A - 1 + dy).
 * The counts are the 3-D cross-correlations of the level sets: each slice is
 * transformed as an image, and for every depth offset the products of the
 * slice spectra are summed over the overlapping slices before the inverse
 * transform.  The peak record's angle_idx field holds dz.  Limits as
 * cmif_plan_create_ex with D * H * W <= 2^22 per volume and D <= 1024;
 * CMIF_FLAG_WINDOW and CMIF_FLAG_WEIGHTED are not supported (UNSUPPORTED), and
 * cmif_align_rotations / cmif_align_two_stage reject volume plans. */
cmif_status cmif_plan_create_3d(cmif_plan* out, int D_A, int H_A, int W_A, int D_B, int H_B, int W_B, int K_A,
                                int K_B, cmif_precision prec, unsigned flags);

/* Free the plan and its workspace (synchronises the plan's device). NULL is ignored. */
cmif_status cmif_plan_destroy(cmif_plan plan);

/* Bytes of device workspace the plan holds. */
cmif_status cmif_plan_workspace_bytes(cmif_plan plan, size_t* bytes);

/* The CMIF map of (A, M_A) and (B, M_B) over the full linear shift range
 * (Eq. cmif, computed per Sec. 3.2), plus optionally N and the peak.
 *   A, M_A, B, M_B : device images as described above (masks may be NULL)
 *   mi_map  : device double[R*C] (required): MI in bits
 *   n_map   : device int32[R*C] or NULL: N(chi) (Eq. number)
 *   counts  : device int32[(K_A*K_B + K_A + K_B) * R*C] or NULL; only with
 *             CMIF_FLAG_DEBUG_COUNTS.  Maps in order: joint C_AB^{a,b} for
 *             a-major pairs (a*K_B + b), then C_A^a, then C_B^b.
 *   gamma   : overlap fraction in [0, 1] of Alg. 1 for the peak
 *   peak_dev: device cmif_peak* or NULL: the gamma-gated argmax of Alg. 1
 *             (ties: lowest map index), angle_idx = 0
 *   stream  : cudaStream_t.  The call is ordered on it: A's forward transforms
 *             may run on a second stream of the plan, forked from and joined
 *             back into stream (a branch when the call is captured in a graph).
 * Returns CMIF_ERR_INVALID_ARG for NULL A/B/mi_map, a counts pointer
 * without the debug flag, or gamma outside [0, 1]. */
cmif_status cmif_compute(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                         const uint8_t* M_B, double* mi_map, int32_t* n_map, int32_t* counts, double gamma,
                         cmif_peak* peak_dev, void* stream);

/* cmif_compute with HOST buffers: copies the images in, computes, delivers
 * mi_map (and n_map, peak when non-NULL), and synchronises the stream.
 * Host pointers.  Output maps in page-locked (pinned) host memory are written
 * by the kernels directly as their rows are finished; other host memory
 * receives a copy after the map (pinned inputs make the copies in asynchronous
 * DMA).  The device
 * staging buffer belongs to the plan: it is allocated by the first host call
 * (the one exception to "compute calls allocate nothing"; CMIF_ERR_OOM when
 * that fails), reused by later ones and freed by cmif_plan_destroy. */
cmif_status cmif_compute_host(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                              const uint8_t* M_B, double* mi_map, int32_t* n_map, double gamma,
                              cmif_peak* peak_host, void* stream);

/* Nearest-neighbour rotation of the floating image for Alg. 1's rotation grid
 * (Sec. 3.6: NN interpolation, the labels being categorical).  The paper
 * leaves centre, canvas and sign open; here: centre ((H-1)/2, (W-1)/2) in
 * (row, col), canvas = B's own H x W, and output pixel (i, j) takes the source
 *   col = c_col + u cos(theta) - v sin(theta),  row = c_row + u sin(theta) + v cos(theta)
 * with u = j - c_col, v = i - c_row, each rounded half away from zero (the
 * content turns counter-clockwise on screen, rows pointing down).  M_out is 1
 * iff the source lies in B and M_B(source) = 1 (M_B NULL: all ones); elsewhere
 * B_out and M_out are 0.  Device pointers: B, B_out int32 H x W; M_B, M_out
 * uint8 H x W.  Coordinates in FP64. */
cmif_status cmif_rotate_nn(const int32_t* B, const uint8_t* M_B, int H, int W, double theta, int32_t* B_out,
                           uint8_t* M_out, void* stream);

/* Alg. 1 over a set of rotations Omega = {R_theta_i}: for every angle, B and
 * M_B are rotated (cmif_rotate_nn, into the plan's buffers), the CMIF map of
 * A against the rotated B is computed (as cmif_compute; A's transforms are
 * computed once), and its gamma-gated argmax taken (N_cal = gamma * max N,
 * ties to the lowest map index).  The per-angle bests are then ordered by MI,
 * descending, earlier angle first among equals, and the first top_k written to
 * topk_dev; topk_dev[0] is Alg. 1's T-hat (strict > against I = 0) when its MI
 * is > 0.  cmif_peak.angle_idx indexes angles_rad_host.
 *   angles_rad_host: host double[n_angles], radians; 1 <= n_angles <= 4096
 *   top_k          : 1 <= top_k <= n_angles
 *   topk_dev       : device cmif_peak[top_k]
 *   mi_maps        : device double[n_angles * R * C] or NULL (per-angle maps,
 *                    angle-major; NULL keeps only the peaks)
 *   n_maps         : device int32[n_angles * R * C] or NULL: the per-angle
 *                    N maps (Eq. number), same layout
 * The plan's sizes are those of A and of B (the rotation keeps B's canvas). */
cmif_status cmif_align_rotations(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                                 const uint8_t* M_B, const double* angles_rad_host, int n_angles, double gamma,
                                 int top_k, cmif_peak* topk_dev, double* mi_maps, int32_t* n_maps, void* stream);

/* Spatially weighted MI (SWMI, Sec. 3.3 "Generalization to spatially weighted MI"):
 * the level sets carry the weights, L_a^W[A](x) = W_A(x) where A(x) = a, else 0
 * (likewise B with W_B), so every count becomes a weighted sum,
 * C_AB^{a,b}(chi) = sum_x W_A(x) W_B(x + chi) [A(x) = a][B(x + chi) = b], and
 * N(chi) = sum of the joint counts.  MI(chi) follows Eq. finalentropy with
 * these real counts (no rounding: the counts are not integers), computed with
 * FP64 transforms and FP64 sums; c log2 c = 0 for c <= 0; MI = 0 where N = 0.
 *   plan   : created with CMIF_FP64 and CMIF_FLAG_WEIGHTED (else INVALID_ARG)
 *   W_A    : device double[H_A][W_A] weights >= 0, or NULL for all ones; a
 *            weight of 0 acts as mask 0 (the label there is ignored); where the
 *            weight is > 0 the label must lie in [0, K_A) (device status
 *            LABEL_RANGE otherwise).  Likewise W_B.
 *   mi_map : device double[R][C] (as cmif_compute)
 *   nw_map : device double[R][C] weighted N, or NULL
 *   peak_dev: device cmif_peak or NULL: Alg. 1's gamma-gated argmax, with
 *            N >= gamma max N on the weighted N (its n field: N rounded)
 * The window flag and graph replay apply as for cmif_compute. */
cmif_status cmif_compute_weighted(cmif_plan plan, const int32_t* A, const double* W_A, const int32_t* B,
                                  const double* W_B, double* mi_map, double* nw_map, double gamma, cmif_peak* peak_dev,
                                  void* stream);

/* Two-stage rigid alignment (Sec. 3.6, the paragraph after Alg. 1): (i) Alg. 1
 * over the grid theta_t = 2 pi t / n_grid, t < n_grid; (ii) Alg. 1 over
 * n_refine angles theta* + (2 u_i - 1) 2 pi / n_grid around the grid winner
 * theta* (0 when no grid angle has I_T > 0), continuing stage (i)'s I and
 * T-hat (a refinement angle replaces the grid choice only when its I_T is
 * strictly greater).  The paper samples the refinement angles uniformly from
 * that interval; here the caller passes the uniform draws u_i in [0, 1], so
 * that a run is reproducible.
 *   n_grid        : 1..4096;  refine_u_host: host double[n_refine] (NULL if 0)
 *   best_host     : host; angle_idx = t for a grid angle, n_grid + i for
 *                   refinement angle i, -1 for the identity
 *   best_angle_rad: host; the winning rotation angle (0 for the identity)
 * Synchronous: waits for stage (i) to choose the refinement interval and for
 * stage (ii) to finish.  The plan's flags apply to both stages; with
 * CMIF_FLAG_GRAPH the two stages' different angle lists make every call
 * capture its graphs anew, so a plan without graph replay is the better fit. */
cmif_status cmif_align_two_stage(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                                 const uint8_t* M_B, int n_grid, const double* refine_u_host, int n_refine,
                                 double gamma, cmif_peak* best_host, double* best_angle_rad, void* stream);

/* ---- Batches of image pairs (many sizes, label counts and angle sets) ----
 * One batch holds one device workspace sized for its largest pair; the pairs
 * run one after another on the call's stream (each as cmif_align_rotations,
 * or as cmif_compute when it has no angles), so that workspace serves them
 * all.  With CMIF_FLAG_GRAPH the whole batch is captured once into a CUDA
 * graph and replayed.  The paper loops over pairs on the host; the batch is
 * this library's way of running such a loop (Alg. 1 per pair). */
typedef struct cmif_batch_s* cmif_batch;
typedef struct {
    const int32_t* A;           /* device, H_A x W_A */
    const uint8_t* M_A;         /* device or NULL */
    const int32_t* B;           /* device, H_B x W_B */
    const uint8_t* M_B;         /* device or NULL */
    int H_A, W_A, H_B, W_B, K_A, K_B;
    const double* angles_rad;   /* host, n_angles radians (copied at cmif_batch_create) */
    int n_angles;               /* 0: translation only (one map, angle_idx 0) */
    double gamma;               /* Alg. 1 overlap fraction in [0, 1] */
} cmif_pair_desc;

/* Validate the pairs (limits as cmif_plan_create_ex, 0 <= n_angles <= 4096),
 * copy the descriptors and allocate the shared workspace.  The device images
 * the descriptors point to must stay valid and unchanged for the batch's life.
 * prec as for plans; flags: 0 or any of CMIF_FLAG_GRAPH, CMIF_FLAG_WINDOW, CMIF_FLAG_NMI,
 * CMIF_FLAG_AUTOTUNE (each pair's size class timed once) and CMIF_FLAG_BATCH_ANGLES (each
 * pair's angles as units of one launch per stage, as far as memory allows). */
cmif_status cmif_batch_create(cmif_batch* out, int n_pairs, const cmif_pair_desc* descs, cmif_precision prec,
                              unsigned flags);

/* Run the batch on stream.  results_dev: device cmif_peak[n_pairs], pair i's
 * Alg. 1 choice (best over its angles, as topk_dev[0] of cmif_align_rotations).
 * status_dev: device int32[n_pairs] or NULL, pair i's device-side cmif_status. */
cmif_status cmif_compute_batch(cmif_batch batch, cmif_peak* results_dev, int32_t* status_dev, void* stream);

/* Device status over the whole last run (synchronises), as cmif_get_status. */
cmif_status cmif_batch_get_status(cmif_batch batch, cmif_status* device_side, double* max_residual, int* escalations);

/* Free the batch (synchronises its device).  NULL is ignored. */
cmif_status cmif_batch_destroy(cmif_batch batch);

/* Device status of the last call on this plan (synchronises the plan's
 * last stream).  device_side: CMIF_OK, or the first device problem in the
 * order LABEL_RANGE, TIMEOUT (the map is incomplete), PRECISION.  max_residual: the largest
 * pre-rounding residual of the authoritative precision (CMIF_AUTO: over
 * every pair, each in the precision it was computed in).  escalations: label
 * pairs CMIF_AUTO computed in the second precision, summed over the call's
 * maps.  Any output pointer may be NULL. */
cmif_status cmif_get_status(cmif_plan plan, cmif_status* device_side, double* max_residual, int* escalations);

/* Per-pair precision of the last call (synchronises), summed over its maps:
 * pairs_predicted = pairs the CMIF_AUTO predicate sent to the second precision
 * up front, pairs_escalated = pairs sent there after their FP32 residual
 * reached the guard, residual_fp32 = the largest residual of the pairs whose
 * FP32 counts stood, residual_second = the largest residual of the
 * second-precision pairs (FP64 and two-term plans: their one residual; FP32
 * plans: 0).  Any output pointer may be NULL. */
cmif_status cmif_get_precision_report(cmif_plan plan, int* pairs_predicted, int* pairs_escalated,
                                      double* residual_fp32, double* residual_second);

/* Launch timing (instrumentation, off by default).  When enabled, each
 * compute call records a CUDA event pair on its stream around every kernel
 * launch it makes; cmif_plan_stage_times (which synchronises) returns the
 * last call's launches in order: *n = count, ms[i] = duration, names[i] =
 * static kernel name, for i < max_n (ms, names may be NULL). */
cmif_status cmif_plan_set_profiling(cmif_plan plan, int enable);
cmif_status cmif_plan_stage_times(cmif_plan plan, int max_n, int* n, double* ms, const char** names);

/* No-allocation variant of cmif_compute.  The paper has no counterpart: this
 * is for callers that may not allocate device memory at all -- for instance a
 * host framework that owns every device allocation and forbids cudaMalloc in
 * its plug-ins, or a loop that must not synchronise the device (cudaMalloc and
 * cudaFree can synchronise implicitly).  No plan is needed and nothing is
 * allocated: the transform workspace, twiddle tables, status word and peak
 * partials live in one fixed device array of 64 MiB inside the library, which
 * every GPU that loads it holds until the process exits.
 *   Arguments as in cmif_compute, plus the sizes (as in cmif_plan_create_ex)
 *   and status_dev: device int32 or NULL, receives the device-side
 *   cmif_status of this map (CMIF_OK, CMIF_ERR_LABEL_RANGE, CMIF_ERR_PRECISION).
 *   FP32 transforms only; no debug counts.
 * Returns CMIF_ERR_UNSUPPORTED when the workspace would exceed the 64 MiB array
 * (e.g. 64 x 64 with K = 8 needs 6 MB; 128 x 128 with K = 12 about 48 MB) or
 * the B-marginals would not fit in shared memory; CMIF_ERR_INVALID_ARG as
 * cmif_compute.  The first call on a device resolves the array's address and
 * uploads the twiddle tables with a synchronous copy: make that first call
 * before any stream capture (a first call on a stream that is being captured
 * returns CMIF_ERR_INVALID_ARG and does nothing).  All calls share the one array: calls that may
 * overlap on the GPU (different streams, threads) race and must not be issued. */
cmif_status cmif_compute_noalloc(int H_A, int W_A, int H_B, int W_B, int K_A, int K_B, const int32_t* A,
                                 const uint8_t* M_A, const int32_t* B, const uint8_t* M_B, double* mi_map,
                                 int32_t* n_map, double gamma, cmif_peak* peak_dev, int32_t* status_dev,
                                 void* stream);

/* Launch-shape choices of a plan's FP32 transforms, as cmif_plan_autotune made them. */
typedef struct {
    int col_lanes;            /* lanes per group of the column transforms: 32, or 16 (radix-R exchange, more warps) */
    int tmem_rows;            /* 1: the Tensor-Memory row kernel, 0: the generic one */
    int cols_blocks_per_sm;   /* persistent blocks per SM of the pair-column kernel (0: as many as fit) */
    double ms_per_map;        /* the chosen candidate's median time for one map (0 when not timed here) */
    int from_cache;           /* 0: timed now, 1: this process's cache, 2: the cache file */
    int candidates;           /* candidates timed now */
} cmif_tuning;

/* Autotuner (not in the paper: the library's choice of FFT radix split and
 * launch shapes for the frequency-domain method of Sec. 3.2).  Times every
 * candidate launch shape of the plan's FP32 transforms on synthetic labels of
 * the plan's sizes -- the column transforms with 32 lanes per group (radix-2
 * split) or 16 (radix-R split with a register DFT and one exchange), the
 * Tensor-Memory or the generic row kernel, one or as many pair-column blocks
 * per SM as fit -- and keeps the fastest (median of three maps, CUDA events).
 * Choices are cached per process and, when cache_path is non-NULL, appended to
 * that JSON-lines file and read back by later processes, keyed on the
 * transform sizes, label counts, depths, precision, SM count and device name.
 * Results do not depend on the choice (the same counts and MI).  Synchronous;
 * uses a temporary device buffer for the synthetic labels.  FP64 and two-term
 * plans have nothing to choose (out reports zeros).  out may be NULL. */
cmif_status cmif_plan_autotune(cmif_plan plan, const char* cache_path, cmif_tuning* out);

/* Fixed-point scale of the epilogue's per-shift entropy sums (Eq. finalentropy):
 * units of 2^-CMIF_ENTROPY_FIX_BITS. */
#define CMIF_ENTROPY_FIX_BITS 23

/* The per-count entropy term T(c) = c log2 c of Eq. finalentropy, exactly as
 * the row epilogue evaluates it (every precision), for the counts
 * c = c0 .. c0 + n - 1: out_dev[i] = T(c0 + i) in units of
 * 2^-CMIF_ENTROPY_FIX_BITS.  T(c) = c * L(c) with an integer L(c), the
 * fixed-point log2 c; T(0) = T(1) = 0.  The MI of a shift is
 * (sum_joint T - sum_A T - sum_B T + T(N)) / N (Eq. finalentropy rearranged),
 * so its error is at most 4 * max_c |L(c) 2^-23 - log2 c|; this entry point
 * lets a caller measure that maximum over every count a map can hold
 * (c <= 2^22).  out_dev: device int64[n]; 0 <= c0, 0 <= n, c0 + n <= 2^22 + 1
 * (else CMIF_ERR_INVALID_ARG).  Asynchronous on stream. */
cmif_status cmif_entropy_terms(int c0, int n, int64_t* out_dev, void* stream);

/* Diagnostics of the bounded device waits (Sec. 3.2's row transforms run in a
 * kernel whose rows arrive by bulk copies completed on mbarriers; every wait
 * gives up after a poll limit, records CMIF_ERR_TIMEOUT in the status word and
 * ends the kernel's work cleanly).  poll_limit > 0 sets the limit of the
 * plan's later calls (0 restores the default of 2^24 polls); withhold_row >= 0
 * makes the Tensor-Memory row kernel (FP32, transform widths 512, 1024 and 2048)
 * skip the bulk copy of that output row's first label pair, so that the wait
 * for it runs out: the call then reports CMIF_ERR_TIMEOUT from cmif_get_status
 * and that map row is not written.  -1 turns it off.  Used by the tests to
 * exercise the timeout path without any fault; not for production calls. */
cmif_status cmif_plan_set_wait_test(cmif_plan plan, int poll_limit, int withhold_row);

/* Static string for a status code. */
const char* cmif_status_string(cmif_status status);

#ifdef __cplusplus
}
#endif

#endif /* CMIF_H */
