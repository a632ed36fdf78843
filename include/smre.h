/*
 * smre.h -- C ABI of the GB300 (sm_103a) statistical multi-resolution
 * projection library, libsmre.so.
 *
 * What it computes (arXiv 1503.03492):
 *   Given a residual image x0 (H x W, row-major) and a scale set of square
 *   window sides, project x0 onto the intersection of the convex sets
 *       C_s = { v : sum_{i in s} v_i^2 <= cS(|s|) }
 *   one per L x L window s of every side L in the set at every position fully
 *   inside the image (Sec. 2, Eqs. tau_s, tau_G; the projection P_G of
 *   Sec. 2.2).  cS = 1 / c_s(alpha) is the bound of Sec. 2.1.
 *   - smre_dykstra_project runs Dykstra's cyclic projection (Sec. 2.3,
 *     Algorithm 2) to a stopping tolerance or a cycle cap;
 *   - smre_dykstra_project_incomplete runs the incomplete Dykstra variant of
 *     Sec. 3.2 (dyadic squares, passes at shifts 2^i);
 *   - smre_batch_* run the standard projection for many images of different
 *     sizes in shared launches, smre_server_* serve projection requests by
 *     continuous batching (no counterpart in the paper);
 *   - smre_admm_* run the estimator itself: the ADMM loop of Sec. 2.2
 *     (Algorithm 1, Eq. 3) with the projection as its eps-step.
 *
 * Conventions shared by every entry point:
 *   - Errors are returned as smre_status codes; nothing aborts, nothing throws.
 *     smre_last_error gives a one-line message for the last failure.
 *   - Image pointers x0 / x may be host or device pointers (the library asks
 *     the CUDA runtime which).  Host images are staged through device buffers
 *     owned by the handle.  x may equal x0.  Pitch is always `width` floats.
 *   - Work is enqueued on the CUDA stream given to smre_dykstra_create.  When
 *     `res` is non-NULL the call waits for that stream and fills *res; when it
 *     is NULL the call returns once the work is enqueued.
 *   - The handle owns every device allocation (increments q_s, work copies of
 *     x, reduction scratch); none is freed before smre_dykstra_destroy.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef SMRE_H
#define SMRE_H

#include <stddef.h>

#if defined(__GNUC__)
#define SMRE_API __attribute__((visibility("default")))
#else
#define SMRE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smre_dykstra smre_dykstra; /* opaque handle */

typedef enum {
    SMRE_OK = 0,
    SMRE_EINVAL = 1,        /* bad argument; nothing was enqueued                 */
    SMRE_ENOMEM = 2,        /* device or pinned host allocation failed            */
    SMRE_ECUDA = 3,         /* a CUDA runtime call failed (message has the name)  */
    SMRE_ETIMEOUT = 4,      /* a device-side wait ran out of its time limit       */
    SMRE_ENOTCONVERGED = 5  /* cycle cap reached before the tolerance (tol >= 0);
                               the result is still the valid last iterate         */
} smre_status;

/* How the bounds cS are chosen (Sec. 2.1).  With mu_s = (|s| - 1/2)^(1/4) and
 * sigma_s^2 = 1 / (8 sqrt|s|), cS = (q sigma_s + mu_s)^4 where
 *   PERSET   q = Phi^{-1}(alpha): the fourth-root normal approximation of the
 *            per-window chi^2_{|s|} alpha-quantile (default);
 *   MAXSTAT  q = Monte Carlo alpha-quantile of Q_Omega = max_s (t_s^(1/4) - mu_s)
 *            / sigma_s on H x W images of iid N(0,1) noise;
 * and
 *   CHI2     cS = the exact chi^2_{|s|} alpha-quantile;
 *   EXPLICIT cS = c_explicit[j] for sides[j]. */
typedef enum {
    SMRE_C_PERSET = 0,
    SMRE_C_CHI2 = 1,
    SMRE_C_MAXSTAT = 2,
    SMRE_C_EXPLICIT = 3
} smre_cmode;

/* flags */
#define SMRE_F_VIOLATION 1        /* fill smre_result.max_violation (one extra pass)   */
#define SMRE_F_GROUP_LAUNCHES 2   /* run the standard method as one kernel launch per
                                     (side, row offset) group with a host-side stop
                                     check per cycle, instead of the single persistent
                                     cooperative launch (same results, slower)        */
#define SMRE_F_AUTOTUNE 8         /* at create, time three cycles of every schedule that
                                     can run the shape (persistent launch, one-image
                                     batch, group launches) on a seeded test image and
                                     keep the fastest; cached per (device, H, W, sides,
                                     q_dtype) for the process                         */
#define SMRE_F_SELFTEST_TIMEOUT 4 /* testing aid: the persistent launch additionally
                                     waits on a flag nothing sets, with a 50 ms limit,
                                     so smre_dykstra_project must return
                                     SMRE_ETIMEOUT and the handle stay usable        */
#define SMRE_F_BAND_IN_SMEM 16    /* the persistent launch keeps each CTA's band of x
                                     in shared memory and maps warps onto windows per
                                     pass, even where the register-band kernel fits
                                     (row stride <= 1024, sides <= 8, bands of <= 8
                                     rows); same results bit for bit, slower          */

/* increment storage types (smre_params.q_dtype, smre_batch_params.q_dtype) */
#define SMRE_Q_FP32 0
#define SMRE_Q_BF16 1
#define SMRE_Q_FP16 2

typedef struct {
    int height, width;          /* pixels: 1 <= height <= 65535, 1 <= width <= 4096 */
    const int *sides;           /* n_sides window sides, 1 <= L <= min(H, W, 32);
                                   a repeated side is ignored when it repeats its
                                   bound (EXPLICIT), EINVAL otherwise            */
    int n_sides;
    double alpha;               /* confidence, 0 < alpha < 1 (unused for EXPLICIT)  */
    smre_cmode cmode;
    const double *c_explicit;   /* n_sides bounds (EXPLICIT only), aligned with sides */
    int max_cycles;             /* cycle cap of the standard method, >= 1           */
    double tol;                 /* stopping tolerance; < 0: run exactly max_cycles  */
    int tol_relative;           /* 0: |x_r - x_{r-1}|_2 <= tol;
                                   1: |x_r - x_{r-1}|_2 <= tol |x_{r-1}|_2         */
    int q_dtype;                /* increment storage: SMRE_Q_FP32 (0), SMRE_Q_BF16 or
                                   SMRE_Q_FP16 (16-bit values with a per-window scale,
                                   see the batches below; width <= 2048, sides <= 16) */
    int icd_max_sweeps;         /* per-tile sweep cap of the incomplete method (0: 1000) */
    int maxstat_draws;          /* Monte Carlo draws for MAXSTAT (0: 1000)         */
    unsigned long long seed;    /* seed of the MAXSTAT draws                        */
    int flags;                  /* SMRE_F_* */
    int max_ctas;               /* persistent launch: at most this many CTAs (one per
                                   SM; 0 = all SMs), so that several projections can
                                   run side by side on disjoint SMs                  */
} smre_params;

typedef struct {
    int cycles;                 /* standard: cycles run; incomplete: total sweeps of all tiles */
    int status;                 /* smre_status of the run                          */
    double step;                /* standard: |x_r - x_{r-1}|_2 of the last cycle   */
    double rel_step;            /* step / |x_{r-1}|_2                              */
    double max_violation;       /* max_s (|x_s|^2 - cS)/cS over all windows of the
                                   scale set (<= 0: feasible); NaN unless requested */
    long long windows;          /* window projections performed                    */
    int max_tile_sweeps;        /* incomplete: largest per-tile sweep count        */
    double seconds;             /* device time of the run (CUDA events)           */
} smre_result;

/* Bounds cS for p->sides (in that order) under p->cmode, computed on the host
 * in FP64 (Sec. 2.1).  cS_out receives n_sides values.  MAXSTAT needs a CUDA
 * device (the Monte Carlo draws run on it). */
SMRE_API smre_status smre_bounds(const smre_params *p, double *cS_out);

/* Out-of-memory paths of the create calls (smre_dykstra_create,
 * smre_batch_create, smre_server_create, smre_admm_create) can be exercised
 * without exhausting the device: with the environment variable
 * SMRE_TEST_FAIL_ALLOC=N set, the N-th device or pinned host allocation
 * (counting from 0) made during one create call fails as if the memory had
 * run out; the call then returns SMRE_ENOMEM after freeing everything it
 * allocated before.  Unset, it has no effect. */

/* Validate p, compute the bounds, and allocate every device buffer a
 * projection of an H x W image with these sides needs: the increments q_s of
 * all sets (sum over L of L^2 * H * W values, padded rows), two work images and
 * reduction scratch.  With 16-bit increments, and for FP32 images wider than
 * 1024 pixels (width <= 2048, sides <= 16, no SMRE_F_GROUP_LAUNCHES), the
 * handle runs the standard method through a one-image batch (smre_batch_*
 * below), which then holds the increments.  `cuda_stream` is a cudaStream_t (NULL: the
 * legacy default stream).  On success *out owns all of it.
 * Errors: EINVAL (bad parameters), ENOMEM, ECUDA. */
SMRE_API smre_status smre_dykstra_create(const smre_params *p, void *cuda_stream, smre_dykstra **out);

/* Dykstra's cyclic projection (Sec. 2.3, Algorithm 2): starting from q_s = 0,
 * repeat cycles over every set in the fixed order (sides descending; for each
 * side L the tilings (L, a, b), a outer, b inner, a, b in 0..L-1; windows of a
 * tiling in parallel) with, per set, y = x + q_s, x = p_s(y) (the projection of Sec. 2.3),
 * q_s = y - x, until the stopping test of the handle's parameters holds or
 * max_cycles cycles ran.  x0, x: H x W float images (host or device).  The
 * call waits for the projection (its stopping test runs on the device).
 * Returns OK, ENOTCONVERGED (cap hit, x valid), EINVAL (bad arguments, or x0
 * holds a NaN or an infinity: the norm |x_prev| of the first cycle is then not
 * finite and the run stops there; x is not valid), ETIMEOUT or ECUDA. */
SMRE_API smre_status smre_dykstra_project(smre_dykstra *h, const float *x0, float *x, smre_result *res);

/* Incomplete Dykstra (Sec. 3.2): with B = 2^K, passes i = 0..K cover the image
 * with B x B tiles at origins (1 << i) mod B + B * t (tiles fully inside); in
 * each tile, Dykstra's algorithm over the non-overlapping 2^k squares of
 * levels k = K down to i, increments zeroed per tile and pass, repeated until
 * the L1 change of one sweep is <= tol * B^2 (at least one sweep, at most
 * icd_max_sweeps).  Bounds of side 2^k follow the handle's cmode (EXPLICIT
 * and MAXSTAT: 2^k must be one of the handle's sides).  K < 0 means floor(log2 max side);
 * 0 <= K <= 5.  Returns OK, EINVAL, ECUDA. */
SMRE_API smre_status smre_dykstra_project_incomplete(smre_dykstra *h, const float *x0, float *x,
                                            int K, double tol, smre_result *res);

/* Change the stopping rule of the standard method for later calls. */
SMRE_API smre_status smre_dykstra_set_stopping(smre_dykstra *h, int max_cycles, double tol,
                                      int tol_relative);

/* Bounds cS the handle uses for its sides, in ascending side order; n >= n_sides. */
SMRE_API smre_status smre_dykstra_bounds(const smre_dykstra *h, int *sides_out, double *cS_out, int n);

/* Per-cycle history of the last smre_dykstra_project call: out[2r] = step of
 * cycle r+1, out[2r+1] = |x_r|_2 before it.  *n_cycles receives the count;
 * at most n_max cycles are copied. */
SMRE_API smre_status smre_dykstra_history(smre_dykstra *h, double *out, int n_max, int *n_cycles);

/* Per-tile sweep counts of the last smre_dykstra_project_incomplete call,
 * pass by pass (i = 0..K), tiles row-major within a pass.  *n_tiles receives
 * the total; at most n_max values are copied. */
SMRE_API smre_status smre_dykstra_icd_sweeps(smre_dykstra *h, int *out, int n_max, int *n_tiles);

/* How the handle runs the standard method: */
#define SMRE_SCHED_PERSISTENT 1   /* one persistent cooperative launch per projection */
#define SMRE_SCHED_BATCHED 2      /* a one-image batch: one step launch per group     */
#define SMRE_SCHED_GROUPS 3       /* one group-kernel launch per group, host stop check */
SMRE_API int smre_dykstra_schedule(const smre_dykstra *h);

/* Number of kernels the handle has launched since it was created (every
 * launch of every entry point; a monotone counter kept on the host). */
SMRE_API long long smre_dykstra_kernel_launches(const smre_dykstra *h);

/* Standard projection that allocates nothing (the paper has no counterpart:
 * it is a service for callers of this library).  Some callers may not call
 * cudaMalloc while they run -- a real-time acquisition pipeline that reserves
 * all device memory when it starts, or a plugin whose host application's
 * memory pool owns the device -- because the allocation can fail once the pool
 * holds the memory, and it can synchronise the device in the middle of their
 * time budget.  This entry point runs the same computation as
 * smre_dykstra_create + smre_dykstra_project (with SMRE_F_GROUP_LAUNCHES) +
 * smre_dykstra_destroy, but keeps every intermediate buffer (increments, work
 * images, norms, control block, per-cycle history) in one static device array
 * of 16 MiB inside the library.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  The array itself comes into existence when the CUDA
 * runtime loads the library's device code on a device: with the runtime's
 * default lazy loading that happens at the first call of this entry point on
 * that device, which then allocates the 16 MiB (and may synchronise the
 * device).  So make one call on each device at start-up -- any size that
 * fits, even a 1 x 1 image -- before the caller's pool reserves the device's
 * memory and before any stream capture begins; or set CUDA_MODULE_LOADING=EAGER
 * so that the array is created when the library loads.  From then on the
 * device holds the array until the process exits and the calls allocate
 * nothing.
 *   p:    problem and stopping rule as for smre_dykstra_create (cmode PERSET,
 *         CHI2 or EXPLICIT; MAXSTAT is rejected); p->flags is ignored.
 *   cuda_stream: stream the work runs on (NULL: legacy default stream); the
 *         call waits for it before returning.
 *   x0, x: H x W float images (device or host), x may equal x0.
 *   res:  optional host result, as for smre_dykstra_project.
 * Sizes whose buffers exceed the 16 MiB array (roughly sum_L L^2 * H * W * 4
 * bytes plus two images) are rejected with SMRE_EINVAL and a message naming
 * the bytes needed.  The first call on each device also looks up the array's
 * device address (once per device, with that device current).  All calls share the array and it
 * keeps the last call's contents; calls whose work overlaps on the GPU (two
 * streams, two threads) race and corrupt each other.
 * Returns OK, ENOTCONVERGED (cap hit, x valid), EINVAL or ECUDA. */
SMRE_API smre_status smre_dykstra_project_static(const smre_params *p, void *cuda_stream,
                                                 const float *x0, float *x, smre_result *res);

/* ------------------------------------------------------------------------
 * Batches: many images of different sizes projected together.
 *
 * The same standard method as smre_dykstra_project (Sec. 2.3, Algorithm 2,
 * same set order, same per-window arithmetic), run over a batch of images at
 * once: each cycle is one kernel launch per group (L, a) whose work list holds
 * the window-rows of every image in the batch, then one norm and one
 * stopping-test launch.  Every image keeps its own cycle count, stopping test
 * and history, and its result does not depend on the other images in the
 * batch (with FP32 increments it equals smre_dykstra_project's bit for bit).
 *
 * Increments may be stored in 16-bit types: q_s = sw * h with h in BF16 or
 * FP16 and one power-of-two FP32 scale sw per window (x, sums and the test
 * stay FP32; x = y - sw * h keeps x + sum_s q_s = x0 exact for the stored
 * increments).  This halves the bytes the method moves and is an
 * approximation: results differ from the FP32 path by the rounding of the
 * stored increments (unit roundoff 2^-8 for BF16, 2^-11 for FP16).
 *
 * Images live in slots.  A batch owns one device arena (device_bytes) from
 * which each admitted image takes its whole state: two images, the increments
 * of all sum_L L^2 sets, their scales and small tables
 * (smre_batch_image_bytes tells how much).  Work is stream-ordered on the
 * stream given to smre_batch_create; a batch is not thread-safe.
 * ---------------------------------------------------------------------- */
typedef struct smre_batch smre_batch;

typedef struct {
    const int *sides;           /* window sides, 1 <= L <= 16; duplicates ignored   */
    int n_sides;
    double alpha;               /* as smre_params (PERSET and CHI2)                 */
    smre_cmode cmode;           /* PERSET, CHI2 or EXPLICIT (not MAXSTAT: its bound
                                   depends on the image size)                       */
    const double *c_explicit;   /* EXPLICIT: one bound per entry of sides           */
    int max_cycles;             /* per-image cycle cap, >= 1                        */
    double tol;                 /* per-image stopping tolerance; < 0: max_cycles    */
    int tol_relative;           /* as smre_params                                   */
    int q_dtype;                /* SMRE_Q_FP32, SMRE_Q_BF16 or SMRE_Q_FP16          */
    int max_images;             /* slots, 1..65536                                  */
    size_t device_bytes;        /* arena for the images' state                      */
    int flags;                  /* SMRE_BF_* below                                  */
} smre_batch_params;

/* Batch flags.  A step launch's work list holds items of k consecutive
 * window-rows of one image; k is at most the kernel's width over the image's
 * row stride and at most ceil(window-rows of the step / (SMs x spread)), so
 * the items of a step cover every SM `spread` times (more, smaller items
 * balance better; fewer, longer ones refill the shared-memory ring less
 * often).  By default each group (L, a) of the cycle (Sec. 3.1: the tilings
 * of one side and row offset) is one launch, so a group starts when the
 * previous one has ended everywhere.  With SMRE_BF_PER_SIDE the L groups of a
 * side share one cooperative launch: an item starts as soon as the items of
 * the previous group of its image that share its rows have written them back
 * (per-image window-row flags), so the tail of one group overlaps the next.
 * The results depend on neither choice, bit for bit. */
#define SMRE_BF_AUTOTUNE 1        /* the first smre_batch_run of at least 5 cycles on a
                                     set of image shapes times one cycle of each of
                                     spread 1 and 4, one launch per group and per side
                                     (after one untimed cycle), and keeps the fastest;
                                     the choice is cached per (device, shapes, sides,
                                     q_dtype) for the process                       */
#define SMRE_BF_SPREAD2 2         /* spread 2 (default 1)                           */
#define SMRE_BF_SPREAD4 4         /* spread 4                                      */
#define SMRE_BF_PER_SIDE 8        /* one cooperative launch per side               */

/* Arena bytes one height x width image takes under p (0: p invalid or the
 * image unsupported: width above 2048 or a side above min(height, width)). */
SMRE_API size_t smre_batch_image_bytes(const smre_batch_params *p, int height, int width);

/* Validate p, compute the bounds and allocate the arena and the slot tables.
 * Errors: EINVAL, ENOMEM, ECUDA. */
SMRE_API smre_status smre_batch_create(const smre_batch_params *p, void *cuda_stream, smre_batch **out);

/* Admit one image (x0: height x width floats, host or device, read before the
 * call returns or in stream order) into a free slot: *slot receives its
 * index, or -1 when no slot or not enough arena is free right now (status OK:
 * retire finished images and try again).  Its cycles start with the next
 * smre_batch_run, from q_s = 0.  Errors: EINVAL (size), ECUDA. */
SMRE_API smre_status smre_batch_submit(smre_batch *b, int height, int width, const float *x0, int *slot);

/* Enqueue `cycles` cycles for every admitted image that has not stopped
 * (images that stop part-way skip the rest).  Returns once enqueued. */
SMRE_API smre_status smre_batch_run(smre_batch *b, int cycles);

/* Wait for the batch's stream, then report images that stopped since the
 * last poll: up to max_done slot indices into done, the count into *n_done.
 * Returns ETIMEOUT if a device-side wait expired (the batch stays usable). */
SMRE_API smre_status smre_batch_poll(smre_batch *b, int *done, int max_done, int *n_done);

/* Copy a stopped image's result into x (height x width, host or device; NULL
 * to discard), fill *res (seconds = host time from submit to the poll that
 * saw it stop), and free its slot and arena.  Returns the image's status
 * (OK or ENOTCONVERGED; EINVAL when the image held a NaN or an infinity, which
 * its first cycle's norm shows and which stops that image alone), or EINVAL
 * for a slot that is empty or not stopped. */
SMRE_API smre_status smre_batch_retrieve(smre_batch *b, int slot, float *x, smre_result *res);

/* Project n images together and wait: submit all (ENOMEM when they do not
 * fit together), run until each stopped, retrieve all into x[i], res[i]. */
SMRE_API smre_status smre_batch_project(smre_batch *b, int n, const int *heights, const int *widths,
                                        const float *const *x0, float *const *x, smre_result *res);

/* Images admitted and not yet retrieved. */
SMRE_API int smre_batch_active(const smre_batch *b);

/* The spread the batch's step launches use now (1, 2 or 4; see SMRE_BF_*),
 * and in *tuned whether SMRE_BF_AUTOTUNE chose it (1 measured, 2 cached, 0
 * not tuned); tuned may be NULL.  The paper has no counterpart. */
SMRE_API int smre_batch_item_spread(const smre_batch *b, int *tuned);

/* 1 when the batch's step launches run one per side (SMRE_BF_PER_SIDE, or
 * chosen by SMRE_BF_AUTOTUNE), 0 when one per group.  The paper has no
 * counterpart. */
SMRE_API int smre_batch_per_side(const smre_batch *b);

/* Kernels the batch has launched since it was created. */
SMRE_API long long smre_batch_kernel_launches(const smre_batch *b);

/* Device bytes the batch holds (arena and tables). */
SMRE_API size_t smre_batch_device_bytes(const smre_batch *b);

/* Message of the last failure on b (NULL: of the last failed create on this thread). */
SMRE_API const char *smre_batch_last_error(const smre_batch *b);

/* Wait for the stream and free everything (NULL is allowed). */
SMRE_API void smre_batch_destroy(smre_batch *b);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over a batch.
 *
 * Requests (one image each, any size the batch takes) are submitted from any
 * thread and complete asynchronously.  A loop thread owns the batch: each
 * round it admits waiting requests in arrival order while a slot and enough
 * arena bytes are free (admission by increment-storage footprint), runs
 * cycles_per_round cycles for every admitted image (new requests join between
 * cycles, their work shares the launches of the others), and retires the
 * images that stopped, copying each result to the caller's buffer.  A result
 * does not depend on what else was served with it.
 * ---------------------------------------------------------------------- */
typedef struct smre_server smre_server;

typedef struct {
    smre_batch_params batch;    /* the batch the loop serves from (slots, arena,
                                   sides, bounds, stopping rule, q_dtype)         */
    int cycles_per_round;       /* cycles between admission / retirement, >= 1    */
} smre_server_params;

typedef struct {
    long long submitted, completed;
    int waiting;                /* submitted, not yet admitted                    */
    int active;                 /* admitted, on the GPU                           */
    int peak_active;
    long long rounds;
    double p50_s, p99_s, max_s, mean_s;   /* latency submit -> result, completed */
    double images_per_s;        /* completed / (last completion - first submit)   */
} smre_server_counters;

/* Create the batch and start the loop thread (on the calling thread's device). */
SMRE_API smre_status smre_server_create(const smre_server_params *p, void *cuda_stream,
                                        smre_server **out);

/* Queue one request: x0 (height x width floats, host or device) is copied
 * before the call returns; the result goes to x (height x width floats, host
 * or device) before the request completes.  *ticket identifies it.  EINVAL
 * when the size is unsupported or needs more than the whole arena. */
SMRE_API smre_status smre_server_submit(smre_server *s, int height, int width, const float *x0,
                                        float *x, long long *ticket);

/* Wait up to timeout_s seconds (< 0: no limit) for a request; on completion
 * fill *res (seconds = latency from submission) and return its status (OK or
 * ENOTCONVERGED; the ticket is then released).  ETIMEOUT: not finished yet,
 * the ticket stays valid. */
SMRE_API smre_status smre_server_wait(smre_server *s, long long ticket, double timeout_s,
                                      smre_result *res);

/* Counters and latency quantiles so far; returns the status of the last failed
 * round (OK if none). */
SMRE_API smre_status smre_server_stats(smre_server *s, smre_server_counters *st);

/* Finish every submitted request, stop the loop, free everything. */
SMRE_API void smre_server_destroy(smre_server *s);

/* ---- ADMM outer loop: the full estimator (Sec. 2.2, Algorithm 1) ------------
 *
 * Solves the split form (Eq. 3) of the multi-resolution estimator (Eq. 1)
 *     min G(eps) + R(z)  s.t.  I = A x + eps,  z = x,
 * G the indicator of the handle's multi-resolution set (Eq. geq), R the
 * anisotropic total variation (Sec. 2: sum of |forward differences| along both
 * axes, zero across the last row / column), A the convolution with a
 * normalised Gaussian point-spread function (weights exp(-k^2 / (2 sigma^2)),
 * |k| <= radius, per axis; zero outside the image; A is its own adjoint).
 * Multipliers Y1 (I = A x + eps) and Y2 (z = x), penalties rho1, rho2 (Eq. 2).
 * Start x = z = eps = Y1 = Y2 = 0; one iteration:
 *   x   <- x - (1/gamma) [ -A(rho1 (I - A x - eps) + Y1) + rho2 (x - z) + Y2 ]
 *          (the linearised x-step, gamma >= rho1 + rho2)
 *   eps <- P_G(I - A x + Y1 / rho1)      (the projection of this library, from
 *          q = 0, with the cycle cap / tolerance of the smre_params; or, with
 *          eps_incomplete, its incomplete Dykstra approximation of Sec. 3.2,
 *          smre_dykstra_project_incomplete(icd_K, icd_tol), as in the paper's
 *          timings of the estimator)
 *   z   <- prox_{R / rho2}(x + Y2 / rho2) by tv_iters steps of projected
 *          gradient on the dual, p <- clip(p + (rho2/8) D(f - D^T p / rho2), -1, 1),
 *          z = f - D^T p / rho2, p kept from one iteration to the next
 *   Y1  <- Y1 + rho1 (I - A x - eps),  Y2 <- Y2 + rho2 (x - z)
 * until |x_r - x_{r-1}|_2 <= delta and |I - A x_r - eps_r|_2 <= delta (both),
 * or max_iters iterations.  All images are H x W row-major FP32 in device
 * memory; x, z, eps and the multipliers are FP32, the two norms FP64. */
typedef struct {
    double sigma;               /* std of the Gaussian PSF in pixels, > 0          */
    int radius;                 /* PSF radius, 1..16; <= 0: ceil(3 sigma)          */
    double rho1, rho2;          /* penalties, > 0                                  */
    double gamma;               /* x-step 1/gamma; <= 0: 1.01 (rho1 + rho2)        */
    int tv_iters;               /* dual steps of the TV prox per iteration, >= 0   */
    int max_iters;              /* iteration cap, >= 1                             */
    double delta;               /* stopping tolerance; < 0: exactly max_iters      */
    int eps_incomplete;         /* 0: standard projection; 1: incomplete Dykstra   */
    int icd_K;                  /* incomplete eps-step: K (< 0: floor(log2 max side)) */
    double icd_tol;             /* incomplete eps-step: per-tile L1 tolerance       */
} smre_admm_params;

typedef struct {
    int iters;                  /* iterations run                                  */
    int status;                 /* OK, or ENOTCONVERGED (delta >= 0, cap reached)  */
    double dx;                  /* |x_r - x_{r-1}|_2 of the last iteration         */
    double residual;            /* |I - A x_r - eps_r|_2 of the last iteration     */
    long long dykstra_cycles;   /* cycles of all eps-steps together (incomplete:
                                   tile sweeps, summed over the tiles)              */
    double seconds;             /* wall time of the solve (host clock, synchronised) */
    double projection_seconds;  /* device time of the eps-steps alone             */
} smre_admm_result;

typedef struct smre_admm smre_admm;

/* An ADMM solver for H x W images: a projection handle made from `proj`
 * (smre_dykstra_create; its stream is `cuda_stream`) plus the solver's
 * images.  Errors: EINVAL, ENOMEM, ECUDA (message: smre_admm_last_error(NULL)). */
SMRE_API smre_status smre_admm_create(const smre_params *proj, const smre_admm_params *ap,
                                      void *cuda_stream, smre_admm **out);

/* Run the loop on the observed image I (device, H x W).  x (required), z and
 * eps (NULL: not returned) receive the final iterates (device, H x W).  Host
 * pointers are rejected with EINVAL.
 * Returns OK, ENOTCONVERGED, EINVAL, ETIMEOUT or ECUDA. */
SMRE_API smre_status smre_admm_solve(smre_admm *a, const float *I, float *x, float *z, float *eps,
                                     smre_admm_result *res);

/* Kernel launches of the solver's own kernels so far (the eps-steps' launches
 * are counted by the projection handle: smre_dykstra_kernel_launches). */
SMRE_API long long smre_admm_kernel_launches(const smre_admm *a);

/* The projection handle of the eps-step (owned by a). */
SMRE_API smre_dykstra *smre_admm_projector(smre_admm *a);

/* Release everything (NULL is allowed); waits for the stream first. */
SMRE_API void smre_admm_destroy(smre_admm *a);

/* Message of the last failure on a, or of the last failed create on this
 * thread when a is NULL.  Never NULL. */
SMRE_API const char *smre_admm_last_error(const smre_admm *a);

/* Bytes of device memory the handle holds. */
SMRE_API size_t smre_dykstra_device_bytes(const smre_dykstra *h);

/* Release every resource of the handle (NULL is allowed).  Waits for the
 * handle's stream first. */
SMRE_API void smre_dykstra_destroy(smre_dykstra *h);

/* Message of the last failure on h, or of the last failed create / bounds
 * call on this thread when h is NULL.  Never NULL. */
SMRE_API const char *smre_last_error(const smre_dykstra *h);

/* Library version string. */
SMRE_API const char *smre_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SMRE_H */
