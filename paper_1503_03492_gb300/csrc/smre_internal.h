// Internal declarations shared by the translation units of libsmre.so.
// Nothing here is part of the public C ABI (include/smre.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "smre.h"

namespace smre {

constexpr int kMaxSide = 32;      // largest window side the kernels are built for
constexpr int kMaxWidth = 4096;   // widest image (one CTA holds a full window-row)
constexpr int kMaxIcdK = 5;       // incomplete Dykstra: B = 2^K <= 32

// Device-side control block of one projection (lives in device memory).
struct Control {
    int stop;        // 1 once the stopping test held (or the cap was reached)
    int cycles;      // cycles completed
    int status;      // smre_status seen on the device
    int pad;
    double step;     // |x_r - x_{r-1}|_2 of the last completed cycle
    double prev_norm;
};

// One group (L, a): the L tilings (L, a, b), b = 0..L-1, share the same
// window-rows ("units": rows a + L u .. a + L u + L - 1, u < n_units), so one
// CTA can run all L passes of a unit back to back with block-local barriers.
struct Group {
    int L, a, n_units;
    int tiling0;          // index of tiling (L, a, 0) in the cycle order
};

// Tiling (L, a, b): windows with top-left (a + L u, b + L v) fully inside.
// Its increments live in n_u blocks of L rows x qpitch floats; block u starts
// at q_off + u * L * qpitch, column j of a row holds pixel column b + j.
struct Tiling {
    int L, a, b, n_u, n_v;
    long long q_off;      // in floats
};

// Arguments of one launch of the group kernel.
struct GroupArgs {
    float *x;             // work image, H x pitch
    float *q;             // increment store
    long long q_off[kMaxSide];  // q_off of tiling (L, a, b) for b = 0..L-1
    int pitch, H, W;
    int L, a, n_units;
    float cS;             // bound of side L (FP32 copy for the fast test)
    float sqrt_cS;        // sqrt(cS) in FP32: scale = sqrt(cS) * rsqrt(t)
    double cS64;          // the same bound in FP64 for the near-boundary recheck
    int first;            // 1: first cycle, stored increments are taken as 0
};

// ---- persistent standard path (smre_persist.cu)

constexpr int kMaxStages = 16;    // ring stages of the increment stream
constexpr int kPersistThreads = 640;   // most threads per CTA of the persistent kernel
constexpr int kMaxItems = 4;          // (unit, window chunk) items per consumer warp and task
// items a consumer warp may hold in one task of side L (register budget)
__host__ __device__ constexpr int max_items_for_side(int L) { return L <= 4 ? 4 : (L <= 8 ? 2 : 1); }

// Per-CTA schedule, kept in shared memory for the whole launch: one entry per
// side the CTA takes part in (cycle order), then per offset a of that side a
// GrpS, then the q offsets of every pass (a-major, b minor), then flag ids.
struct SideS {
    int L, U;                     // side; units held (the band has U*L rows)
    int r0;                       // first band row at offset a = 0 (L * u0)
    int dep_begin, dep_count;     // side-start flags in the CTA's dependency list
    int grp0;                     // first GrpS entry of the side
    int pass0;                    // first pass q offset of the side
    int flag0;                    // flag of event (side, this CTA, a = 0); a adds a
    unsigned top_final;           // bit a: the top row published after offset a is final
    float cS, sqrt_cS;            // bound of side L (FP32) and its square root
    int pad_;
    unsigned long long end_final; // bit k: band row k published at the side end is final
    double cS64;
};

struct GrpS {
    int U;                        // units present at this offset
    int nb_flag;                  // flag to wait before taking the lower neighbour's
                                  // top row at this offset (a >= 1), or -1
};

struct PersistArgs {
    float *x, *xprev, *q;
    const float *zeros;          // stage_floats zero floats (increments of the first cycle)
    int pitch, H, W;
    int consumer_warps;          // warps 0..consumer_warps-1 consume, the next one produces
    // per-CTA schedule: int hdr[4] = {n_sides, n_grp, n_pass, n_dep} | SideS[] | GrpS[] |
    // long long pass_qoff[] | int deps[]
    const unsigned char *sched;
    const int *cta_off;          // [G]: byte offset of each CTA's segment
    int sched_bytes;             // shared-memory bytes reserved for the largest segment
    unsigned *flags;             // [n_events] cycle + 1 once the event's rows are published
    unsigned *barrier;           // grid barrier counter
    double *partials;            // [2][G][2] per-CTA norms, double-buffered by cycle
    Control *ctl;
    double *hist;
    int hist_cap;
    int max_cycles;
    double tol;
    int tol_relative;
    int stages;
    int stage_floats;            // floats per stage (rows of the shared-memory stride)
    int stage_offset;            // bytes from the start of dynamic shared memory
    unsigned long long timeout_ns;
    int *abort_word;
    int selftest_timeout;
    const unsigned *selftest_flag;
    // register-band kernel only: rows handed to the upper neighbour at offset
    // transitions, one slot of `pitch` 64-bit words (value | tag << 32) per
    // event, and the tag base of this launch (tag = tag_base + cycle + 1)
    unsigned long long *xch;
    unsigned tag_base;
    unsigned *smid_tab;          // [G] SM id of each CTA (the launch orders bands by it)
};

// ---- batched path (smre_batch.cu): many images, one launch per group step

constexpr int kBatchConsumers = 512;   // consumer threads of the step kernel (16 warps, plus
                                       // a producer and a storer warp: at most 5 warps per
                                       // SM sub-partition, 96 registers a thread)
constexpr int kBatchDescs = 8;         // ring descriptors (chunks in flight)
constexpr int kBatchMaxWidth = 2048;   // widest image of the batched path
constexpr int kBatchMaxSide = 16;      // largest window side of the batched path
constexpr int kBatchNormRows = 16;     // rows per norm chunk (fixed: per-image order)

// Per-image state of a batch slot (device memory).
struct BImage {
    float *x;                 // H x pitch work image
    float *xprev;             // previous iterate (cycle norm)
    void *q;                  // increment planes, element type of the batch
    float *qs;                // per-window scales of the planes (BF16/FP16 only)
    const long long *qoff;    // [n_planes] element offset of plane p in q
    const long long *soff;    // [n_planes] float offset of plane p in qs
    Control *ctl;
    double *hist;             // [2 * hist_cap] step and |x_prev| per cycle
    double *part;             // [2 * nchunks] norm partials of the current cycle
    unsigned *uflag;          // [H] per window-row u of the running side: tag of the last
                              // group (L, a) that wrote its rows back (one launch per side)
    int H, W, pitch, nchunks;
    int hist_cap, pad_;
};

// One group (L, a) of a step launch: its items over the active images.
struct BGroup {
    const int *prefix;        // [n_active + 1] first item of each active image
    const int *kpack;         // [n_active] units per item
    int n_items;
    int a, p0;                // row offset, plane of tiling (L, a, 0)
    int seq;                  // place of the group in the cycle (flag tags)
};

// One launch of the step kernel: every item of n_groups consecutive groups
// (L, a) of one side over the batch.  An item is k consecutive units (k L
// rows) of one image, k * pitch <= the kernel's virtual width.  With more
// than one group, an item waits for the items of the previous group of its
// image whose rows it shares (per-image window-row flags; cooperative launch).
struct BStepArgs {
    const BImage *imgs;
    const int *active;        // [n_active] slot of each active image
    const BGroup *groups;     // [n_groups] in cycle order
    int n_active, n_groups;
    int max_items;            // largest n_items of the groups
    int L;                    // side
    float cS, sqrt_cS;
    double cS64;
    int ring_bytes;           // shared-memory ring for x and increment blocks
    int ring_offset;          // its offset in dynamic shared memory
    unsigned long long timeout_ns;
    int *err;                 // SMRE_ETIMEOUT is recorded here
};

struct BNormArgs {
    const BImage *imgs;
    const int *active;
    const int *prefix;        // [n_active + 1] first norm chunk of each active image
    int n_active, n_chunks;
};

struct BDecideArgs {
    const BImage *imgs;
    const int *active;
    int n_active;
    int max_cycles;
    double tol;
    int tol_relative;
};

// q element type of a batch: 0 FP32, 1 BF16, 2 FP16
int batch_lb(int L);                       // kernel variant of side L (L itself up to 12, then 16)
int batch_virtual_width(int L);            // columns one item may span
size_t batch_part_bytes(int L, int qtype);            // shared memory of the window sums
int batch_threads();
cudaError_t batch_prepare(int qtype, size_t smem_max);
cudaError_t launch_batch_step(int qtype, const BStepArgs &A, int grid, size_t smem,
                              cudaStream_t s);
cudaError_t launch_batch_norm(const BNormArgs &A, int grid, cudaStream_t s);
// per increment type (smre_batch_f32.cu, smre_batch_bf16.cu, smre_batch_f16.cu)
cudaError_t launch_batch_step_f32(const BStepArgs &A, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_batch_step_bf16(const BStepArgs &A, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_batch_step_f16(const BStepArgs &A, int grid, size_t smem, cudaStream_t s);
cudaError_t batch_prepare_f32(size_t smem);
cudaError_t batch_prepare_bf16(size_t smem);
cudaError_t batch_prepare_f16(size_t smem);
cudaError_t launch_batch_decide(const BDecideArgs &A, cudaStream_t s);

// A batch serving one image for an smre_dykstra handle (smre_batch_host.cu):
// change the stopping rule (max_cycles up to the history the batch was made
// for), or project one device image and copy its history and control block.
smre_status batch_set_rule(smre_batch *b, int max_cycles, double tol, int tol_relative);
// free a slot whatever its state (after a failed round)
void batch_drop(smre_batch *b, int slot);
smre_status batch_run_one(smre_batch *b, int height, int width, const float *x0, float *x,
                          int ld, double *hist, int hist_cap, Control *ctl_out);
// submit / retrieve with a row stride of ld floats for the caller's image
smre_status batch_submit_ld(smre_batch *b, int height, int width, const float *x0, int ld,
                            int *slot);
smre_status batch_retrieve_ld(smre_batch *b, int slot, float *x, int ld, smre_result *res);

// ---- persistent standard path, band in registers (smre_persist_reg.cu)
constexpr int kRegRows = 8;                 // band rows a lane holds (largest side it takes)
constexpr int kRegMaxWarps = 16;            // consumer warps of 64 columns: pitch <= 1024
constexpr int kRegMaxThreads = (kRegMaxWarps + 2) * 32;   // consumers, producer, storer
constexpr int kRegHeaderBytes = 1024;       // mbarriers and flags before the schedule table
// the shape fits the register-band kernel: pitch <= 1024, sides <= 8, every
// side task's band at most kRegRows rows
bool persist_reg_fits(int pitch, int max_side, int max_band_rows);
// shared memory of its column-sum exchange arrays
size_t persist_reg_exchange_bytes(int pitch);
cudaError_t persist_reg_occupancy(int threads, size_t smem, int *blocks_per_sm);
cudaError_t launch_persist_reg(const PersistArgs &A, int grid, int threads, size_t smem,
                               cudaStream_t s);

bool persist_supported(int max_side);
// shared-memory row stride (power of two >= pitch, 128..1024) or 0 if too wide
int persist_smem_pitch(int pitch);
cudaError_t persist_occupancy(int sp, int pitch, int threads, size_t smem, int *blocks_per_sm);
cudaError_t launch_persist(const PersistArgs &A, int sp, int grid, int threads, size_t smem,
                           cudaStream_t s);

// Launchers (defined next to their kernels).
cudaError_t launch_group(const GroupArgs &args, cudaStream_t s);
cudaError_t launch_cycle_norm(const float *x, float *xprev, int H, int W, int pitch,
                              double *partials, int n_blocks, cudaStream_t s);
cudaError_t launch_decide(const double *partials, int n_blocks, Control *ctl, double *hist,
                          int max_cycles, double tol, int tol_relative, cudaStream_t s);
int norm_blocks();

struct ViolationArgs {
    const float *x;
    int pitch, H, W;
    int n_sides;
    int sides[kMaxSide];
    double cS[kMaxSide];
};
cudaError_t launch_violation(const ViolationArgs &a, double *partials, int n_blocks,
                             double *out, cudaStream_t s);

struct IcdArgs {
    float *x;             // work image, H x pitch
    int pitch, H, W;
    int K, pass, off;     // level count K, pass i, offset (1 << i) mod B
    int n_ti, n_tj;       // tiles of this pass
    float tol_b2;         // tol * B^2
    int max_sweeps;
    float cS[kMaxIcdK + 1];      // bound of side 2^k
    float sqrt_cS[kMaxIcdK + 1]; // its square root (FP32): scale = sqrt(cS) * rsqrt(t)
    double cS64[kMaxIcdK + 1];
    int *sweeps;          // per-tile sweep counts of this pass (n_ti * n_tj)
};
cudaError_t launch_icd_pass(const IcdArgs &a, cudaStream_t s);

// Message returned by smre_last_error(NULL) on this thread (smre_host.cu).
void set_thread_error(const char *msg);

// Device and pinned host allocations (smre_host.cu).  With the environment
// variable SMRE_TEST_FAIL_ALLOC=N set, the N-th allocation (counting from 0)
// made inside the outermost create call of this thread fails with
// cudaErrorMemoryAllocation and allocates nothing: a test aid that drives
// every out-of-memory path of the create calls.  AllocScope marks a create
// call (nested creates share the outer count).
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t host_malloc(void **p, size_t bytes);
template <class T> inline cudaError_t dev_malloc(T **p, size_t bytes) { return dev_malloc((void **)p, bytes); }
template <class T> inline cudaError_t host_malloc(T **p, size_t bytes) { return host_malloc((void **)p, bytes); }
struct AllocScope {
    AllocScope();
    ~AllocScope();
};

// Host FP64 helpers of Sec. 2.1 (smre_weights.cu).
double inv_normal_cdf(double p);
double chi2_quantile(double alpha, int k);
double bound_from_q(double q, int L);

// Monte Carlo of Q_Omega (Sec. 2.1) for the MAXSTAT bounds: per-draw maxima of
// draws draw0 .. draw0 + n_draws - 1 land in maxima[n_draws .. 2 n_draws);
// img holds n_draws * H * pitch floats, maxima 2 * n_draws doubles.
cudaError_t launch_maxstat(int H, int W, int pitch, const int *sides, int n_sides, int draw0,
                           int n_draws, unsigned long long seed, float *img, double *maxima,
                           cudaStream_t s);

}  // namespace smre
