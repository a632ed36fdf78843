// Host side of the batched path: image slots, the device arena that holds
// every image's state, the item tables of the step kernel and the smre_batch_*
// functions of include/smre.h.
//
// A batch owns one device allocation (the arena).  An image admitted into a
// slot gets one contiguous piece of it: work image, previous iterate, the
// increment planes of all Sum_L L^2 sets (FP32, BF16 or FP16) with their
// per-window scales (16-bit types), the plane offset tables, the per-cycle
// history and the norm partials.  Admission fails softly (slot -1) when the
// slots or the arena are full, so a caller can wait for retirements.
//
// Items of a group are at most ceil(units / SMs) window-rows, so a few small
// images still spread over every SM.  The launches of one cycle (every
// group's step kernel, the norm and the decide kernel) are captured once into
// a CUDA graph on a private stream and replayed each cycle; admission,
// retirement or a new stopping rule rebuild the tables and the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "smre_internal.h"

using namespace smre;

namespace {

double now_seconds()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// First-fit allocator over one device allocation, in 256-byte granules; a
// freed range merges with free neighbours.
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t &off)
    {
        n = align256(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            off = it->first;
            const size_t rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = align256(n);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }

private:
    std::map<size_t, size_t> free_;   // offset -> length
};

// Where an H x W image's state sits inside its arena piece.
struct Layout {
    int pitch = 0, nchunks = 0;
    size_t x = 0, xprev = 0, q = 0, qs = 0, qoff = 0, soff = 0, hist = 0, part = 0, uflag = 0, total = 0;
    std::vector<long long> qoff_tab, soff_tab;   // per plane, cycle order
    long long windows_per_cycle = 0;
};

struct Step {
    int L, a, p0;
};

}  // namespace

struct smre_batch {
    // problem shared by every image
    std::vector<int> sides;   // ascending, unique
    double cS_of[kMaxSide + 1] = {};
    int qtype = 0;
    int max_cycles = 1;
    double tol = -1.0;
    int tol_relative = 0;
    int max_images = 0;
    int hist_cap = 0;
    std::vector<Step> steps;   // group steps (L, a) in the cycle order
    int n_planes = 0;
    // device
    cudaStream_t stream = nullptr;
    int sms = 0;
    size_t smem = 0;           // dynamic shared memory of the step kernel
    unsigned char *arena = nullptr;
    size_t arena_bytes = 0;
    Arena heap;
    BImage *d_imgs = nullptr;
    Control *d_ctl = nullptr;
    Control *h_ctl = nullptr;  // pinned mirror
    int *d_err = nullptr;
    int *h_err = nullptr;      // pinned
    int *d_tab = nullptr;      // item tables
    size_t tab_ints = 0;
    BGroup *d_groups = nullptr;   // [steps] group descriptors into d_tab
    bool per_side = false;        // one cooperative launch per side instead of per group
    unsigned long long timeout_ns = 10000000000ull;
    // host state
    struct Slot {
        bool used = false, done = false;
        int H = 0, W = 0;
        size_t off = 0, bytes = 0;
        BImage img{};
        long long windows_per_cycle = 0;
        double t_submit = 0.0, t_done = 0.0;
    };
    std::vector<Slot> slots;
    std::vector<int> active;   // used slots, in admission order
    bool dirty = true;
    std::vector<int> step_items, step_prefix_at, step_kpack_at;
    int norm_chunks = 0, norm_prefix_at = 0;
    // items of a step cover every SM `spread` times (SMRE_BF_*)
    int spread = 1;
    bool autotune = false;
    int tuned = 0;                 // 1 measured, 2 cached, 0 not tuned
    std::string tuned_key;         // the shapes the current spread was tuned for
    cudaEvent_t tev0 = nullptr, tev1 = nullptr;
    long long launches = 0;
    // one cycle's launches captured in a CUDA graph, rebuilt when the item
    // tables or the stopping rule change
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_dirty = true;
    bool graph_ok = true;
    int cycle_kernels = 0;
    std::string err;
};

namespace {

smre_status bfail(smre_batch *b, smre_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    set_thread_error(buf);
    return s;
}

#define BCK(b, call)                                                                      \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA, \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

int scale_row(int W, int L) { return ((W / L) + 3) & ~3; }

// Validation shared by create and image_bytes; sides come back ascending.
smre_status check_batch_params(const smre_batch_params *p, std::vector<int> &sides,
                               std::vector<double> &cS)
{
    if (!p) return bfail(nullptr, SMRE_EINVAL, "params is NULL");
    if (!p->sides || p->n_sides < 1 || p->n_sides > 64)
        return bfail(nullptr, SMRE_EINVAL, "need 1..64 window sides");
    if (p->q_dtype < SMRE_Q_FP32 || p->q_dtype > SMRE_Q_FP16)
        return bfail(nullptr, SMRE_EINVAL, "q_dtype %d unknown", p->q_dtype);
    if (p->flags & ~(SMRE_BF_AUTOTUNE | SMRE_BF_SPREAD2 | SMRE_BF_SPREAD4 | SMRE_BF_PER_SIDE))
        return bfail(nullptr, SMRE_EINVAL, "unknown batch flags 0x%x", p->flags);
    if ((p->flags & SMRE_BF_SPREAD2) && (p->flags & SMRE_BF_SPREAD4))
        return bfail(nullptr, SMRE_EINVAL, "SMRE_BF_SPREAD2 and SMRE_BF_SPREAD4 together");
    if (p->cmode != SMRE_C_PERSET && p->cmode != SMRE_C_CHI2 && p->cmode != SMRE_C_EXPLICIT)
        return bfail(nullptr, SMRE_EINVAL, "batches take cmode PERSET, CHI2 or EXPLICIT");
    if (p->cmode != SMRE_C_EXPLICIT && !(p->alpha > 0.0 && p->alpha < 1.0))
        return bfail(nullptr, SMRE_EINVAL, "alpha %g outside (0, 1)", p->alpha);
    if (p->max_cycles < 1) return bfail(nullptr, SMRE_EINVAL, "max_cycles must be >= 1");
    if (std::isnan(p->tol)) return bfail(nullptr, SMRE_EINVAL, "tol is NaN");
    if (p->max_images < 1 || p->max_images > 65536)
        return bfail(nullptr, SMRE_EINVAL, "max_images %d outside 1..65536", p->max_images);
    std::vector<std::pair<int, double>> sv;
    for (int i = 0; i < p->n_sides; ++i) {
        const int L = p->sides[i];
        if (L < 1 || L > kBatchMaxSide)
            return bfail(nullptr, SMRE_EINVAL, "window side %d outside 1..%d", L, kBatchMaxSide);
        double c;
        if (p->cmode == SMRE_C_EXPLICIT) {
            if (!p->c_explicit) return bfail(nullptr, SMRE_EINVAL, "c_explicit is NULL");
            c = p->c_explicit[i];
            if (!(c > 0.0) || !std::isfinite(c))
                return bfail(nullptr, SMRE_EINVAL, "bound %g of side %d is not a positive number", c, L);
        } else if (p->cmode == SMRE_C_CHI2) {
            c = chi2_quantile(p->alpha, L * L);
        } else {
            c = bound_from_q(inv_normal_cdf(p->alpha), L);
        }
        sv.emplace_back(L, c);
    }
    std::stable_sort(sv.begin(), sv.end(), [](auto &x, auto &y) { return x.first < y.first; });
    sides.clear();
    cS.clear();
    for (auto &pr : sv) {
        if (sides.empty() || sides.back() != pr.first) {
            sides.push_back(pr.first);
            cS.push_back(pr.second);
        } else if (pr.second != cS.back()) {
            // a repeated side is ignored only when it repeats the bound too
            return bfail(nullptr, SMRE_EINVAL, "side %d listed twice with different bounds (%g, %g)",
                         pr.first, cS.back(), pr.second);
        }
    }
    return SMRE_OK;
}

// Footprint of one H x W image (sides ascending).
bool image_layout(const std::vector<int> &sides, int qtype, int hist_cap, int H, int W, Layout &lo)
{
    if (H < 1 || W < 1 || H > 65535 || W > kBatchMaxWidth) return false;
    if (sides.back() > std::min(H, W)) return false;
    lo.pitch = (W + 31) / 32 * 32;
    lo.nchunks = (H + kBatchNormRows - 1) / kBatchNormRows;
    const size_t esz = qtype == SMRE_Q_FP32 ? 4 : 2;
    long long qe = 0, se = 0;
    lo.qoff_tab.clear();
    lo.soff_tab.clear();
    lo.windows_per_cycle = 0;
    for (auto it = sides.rbegin(); it != sides.rend(); ++it) {
        const int L = *it;
        lo.windows_per_cycle += (long long)(H - L + 1) * (W - L + 1);
        for (int a = 0; a < L; ++a) {
            const long long units = (H - a) / L;
            for (int b = 0; b < L; ++b) {
                lo.qoff_tab.push_back(qe);
                lo.soff_tab.push_back(se);
                qe += units * L * lo.pitch;
                if (qtype != SMRE_Q_FP32) se += units * scale_row(W, L);
            }
        }
    }
    const size_t img = sizeof(float) * (size_t)H * lo.pitch;
    const size_t np = lo.qoff_tab.size();
    size_t o = 0;
    lo.x = o;      o += align256(img);
    lo.xprev = o;  o += align256(img);
    lo.q = o;      o += align256(esz * (size_t)qe);
    lo.qs = o;     o += align256(sizeof(float) * (size_t)se);
    lo.qoff = o;   o += align256(sizeof(long long) * np);
    lo.soff = o;   o += align256(sizeof(long long) * np);
    lo.hist = o;   o += align256(sizeof(double) * 2 * (size_t)hist_cap);
    lo.part = o;   o += align256(sizeof(double) * 2 * (size_t)lo.nchunks);
    lo.uflag = o;  o += align256(sizeof(unsigned) * (size_t)H);
    lo.total = o;
    return true;
}

// Spreads chosen by SMRE_BF_AUTOTUNE, per (device, shapes, sides, q_dtype).
std::mutex g_spread_mu;
std::map<std::string, int> g_spread_cache;

std::string spread_key(const smre_batch *b)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<std::pair<int, int>> shapes;
    for (int s : b->active) shapes.emplace_back(b->slots[s].H, b->slots[s].W);
    std::sort(shapes.begin(), shapes.end());
    std::string k = std::to_string(dev) + "|" + std::to_string(b->qtype) + "|";
    for (int L : b->sides) k += std::to_string(L) + ",";
    k += "|";
    for (auto &sh : shapes) k += std::to_string(sh.first) + "x" + std::to_string(sh.second) + ",";
    return k;
}

// Rebuild the item tables of the active images and upload them.
smre_status rebuild_tables(smre_batch *b)
{
    const int n = (int)b->active.size();
    std::vector<int> tab;
    tab.reserve(b->tab_ints);
    tab.insert(tab.end(), b->active.begin(), b->active.end());
    b->step_items.assign(b->steps.size(), 0);
    b->step_prefix_at.assign(b->steps.size(), 0);
    b->step_kpack_at.assign(b->steps.size(), 0);
    for (size_t s = 0; s < b->steps.size(); ++s) {
        const Step &st = b->steps[s];
        const int vw = batch_virtual_width(st.L);
        b->step_prefix_at[s] = (int)tab.size();
        // units per item: as many as fit the kernel's width (a pass's fixed
        // costs are paid per item), but few enough that the step's items
        // cover every SM (few or small images)
        long long total_units = 0;
        for (int i = 0; i < n; ++i) total_units += (b->slots[b->active[i]].H - st.a) / st.L;
        const long long lanes = (long long)b->sms * b->spread;
        const int kcap = (int)std::max(1LL, (total_units + lanes - 1) / lanes);
        int acc = 0;
        std::vector<int> kp(n);
        for (int i = 0; i < n; ++i) {
            const auto &sl = b->slots[b->active[i]];
            tab.push_back(acc);
            const int units = (sl.H - st.a) / st.L;
            const int k = std::max(1, std::min(vw / sl.img.pitch, kcap));
            kp[i] = k;
            acc += (units + k - 1) / k;
        }
        tab.push_back(acc);
        b->step_items[s] = acc;
        b->step_kpack_at[s] = (int)tab.size();
        tab.insert(tab.end(), kp.begin(), kp.end());
    }
    std::vector<BGroup> groups(b->steps.size());
    for (size_t s = 0; s < b->steps.size(); ++s)
        groups[s] = BGroup{b->d_tab + b->step_prefix_at[s], b->d_tab + b->step_kpack_at[s],
                           b->step_items[s], b->steps[s].a, b->steps[s].p0, (int)s};
    b->norm_prefix_at = (int)tab.size();
    int acc = 0;
    for (int i = 0; i < n; ++i) {
        tab.push_back(acc);
        acc += b->slots[b->active[i]].img.nchunks;
    }
    tab.push_back(acc);
    b->norm_chunks = acc;
    if (tab.size() > b->tab_ints) return bfail(b, SMRE_EINVAL, "item table overflow");
    BCK(b, cudaMemcpyAsync(b->d_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice,
                           b->stream));
    BCK(b, cudaMemcpyAsync(b->d_groups, groups.data(), sizeof(BGroup) * groups.size(),
                           cudaMemcpyHostToDevice, b->stream));
    b->dirty = false;
    b->graph_dirty = true;
    return SMRE_OK;
}

// The launches of one cycle: the step kernel once per group with items (or
// once per side, every group of the side in one cooperative launch), then
// the norm and the stopping test.
smre_status enqueue_cycle(smre_batch *b, cudaStream_t stream)
{
    const int n = (int)b->active.size();
    int kernels = 0;
    for (size_t s = 0; s < b->steps.size();) {
        // groups s .. e - 1 go into one launch: one group, or every group of
        // the side (consecutive offsets a = 0 .. L - 1, each waiting for the
        // one before it)
        size_t e = s + 1;
        if (b->per_side)
            while (e < b->steps.size() && b->steps[e].L == b->steps[s].L) ++e;
        int max_items = 0;
        for (size_t k = s; k < e; ++k) max_items = std::max(max_items, b->step_items[k]);
        const Step &st = b->steps[s];
        const size_t first = s;
        s = e;
        if (max_items == 0) continue;
        BStepArgs A{};
        A.imgs = b->d_imgs;
        A.active = b->d_tab;
        A.groups = b->d_groups + first;
        A.n_active = n;
        A.n_groups = (int)(e - first);
        A.max_items = max_items;
        A.L = st.L;
        A.cS = (float)b->cS_of[st.L];
        A.sqrt_cS = (float)std::sqrt(b->cS_of[st.L]);
        A.cS64 = b->cS_of[st.L];
        A.ring_offset = (int)(256 + batch_part_bytes(st.L, b->qtype));
        A.ring_bytes = (int)(b->smem - A.ring_offset);
        A.timeout_ns = b->timeout_ns;
        A.err = b->d_err;
        const int grid = std::min(A.max_items, b->sms);
        BCK(b, launch_batch_step(b->qtype, A, grid, b->smem, stream));
        ++kernels;
    }
    BNormArgs N{b->d_imgs, b->d_tab, b->d_tab + b->norm_prefix_at, n, b->norm_chunks};
    BCK(b, launch_batch_norm(N, std::min(b->norm_chunks, 4 * b->sms), stream));
    BDecideArgs D{b->d_imgs, b->d_tab, n, b->max_cycles, b->tol, b->tol_relative};
    BCK(b, launch_batch_decide(D, stream));
    kernels += 2;
    b->cycle_kernels = kernels;
    b->launches += kernels;
    return SMRE_OK;
}

// Capture one cycle into a graph on the batch's private stream (launched
// later on the caller's stream).  If capture is not possible the batch keeps
// launching the kernels one by one.
void capture_cycle(smre_batch *b)
{
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    b->graph_dirty = false;
    const long long l0 = b->launches;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        b->graph_ok = false;
        return;
    }
    const smre_status st = enqueue_cycle(b, b->cap_stream);
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    b->launches = l0;   // captured, not launched
    if (st != SMRE_OK || e != cudaSuccess || !g ||
        cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        b->gexec = nullptr;
        b->graph_ok = false;
    }
    if (g) cudaGraphDestroy(g);
}

void free_batch(smre_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->tev0) cudaEventDestroy(b->tev0);
    if (b->tev1) cudaEventDestroy(b->tev1);
    cudaFree(b->arena);
    cudaFree(b->d_imgs);
    cudaFree(b->d_ctl);
    cudaFree(b->d_err);
    cudaFree(b->d_tab);
    cudaFree(b->d_groups);
    cudaFreeHost(b->h_ctl);
    cudaFreeHost(b->h_err);
    delete b;
}

}  // namespace

extern "C" {

size_t smre_batch_image_bytes(const smre_batch_params *p, int height, int width)
{
    std::vector<int> sides;
    std::vector<double> cS;
    if (check_batch_params(p, sides, cS) != SMRE_OK) return 0;
    Layout lo;
    if (!image_layout(sides, p->q_dtype, p->max_cycles, height, width, lo)) return 0;
    return lo.total;
}

smre_status smre_batch_create(const smre_batch_params *p, void *cuda_stream, smre_batch **out)
{
    const AllocScope scope;
    if (!out) return bfail(nullptr, SMRE_EINVAL, "out is NULL");
    *out = nullptr;
    std::vector<int> sides;
    std::vector<double> cS;
    smre_status st = check_batch_params(p, sides, cS);
    if (st != SMRE_OK) return st;
    if (p->device_bytes < 4096) return bfail(nullptr, SMRE_EINVAL, "device_bytes too small");
    smre_batch *b = new (std::nothrow) smre_batch;
    if (!b) return bfail(nullptr, SMRE_ENOMEM, "host allocation failed");
    b->sides = sides;
    for (size_t i = 0; i < sides.size(); ++i) b->cS_of[sides[i]] = cS[i];
    b->qtype = p->q_dtype;
    b->spread = (p->flags & SMRE_BF_SPREAD4) ? 4 : (p->flags & SMRE_BF_SPREAD2) ? 2 : 1;
    b->autotune = (p->flags & SMRE_BF_AUTOTUNE) != 0;
    b->per_side = (p->flags & SMRE_BF_PER_SIDE) != 0;
    b->max_cycles = p->max_cycles;
    b->tol = p->tol;
    b->tol_relative = p->tol_relative ? 1 : 0;
    b->max_images = p->max_images;
    b->hist_cap = p->max_cycles;
    b->stream = (cudaStream_t)cuda_stream;
    if (const char *env = getenv("SMRE_WAIT_TIMEOUT_MS")) {
        const double ms = atof(env);
        if (ms > 0) b->timeout_ns = (unsigned long long)(ms * 1e6);
    }
    int p0 = 0;
    for (auto it = sides.rbegin(); it != sides.rend(); ++it)
        for (int a = 0; a < *it; ++a) {
            b->steps.push_back({*it, a, p0});
            p0 += *it;
        }
    b->n_planes = p0;

    auto bail = [&](smre_status s) {
        std::string msg = b->err;
        free_batch(b);
        set_thread_error(msg.c_str());
        return s;
    };
#define CREATE_CK(call)                                                                    \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            bfail(b, e_ == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                          \
            return bail(e_ == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA);       \
        }                                                                                  \
    } while (0)
    int dev = 0, optin = 0;
    CREATE_CK(cudaGetDevice(&dev));
    CREATE_CK(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    CREATE_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    b->smem = (size_t)optin - 1024;   // leave room for the kernel's static shared memory
    // the ring must hold the largest block of any step
    const size_t esz = b->qtype == SMRE_Q_FP32 ? 4 : 2;
    for (int L : sides) {
        const size_t ring = b->smem - 256 - batch_part_bytes(L, b->qtype);
        const size_t vw = batch_virtual_width(L);
        const size_t need = std::max(L * vw * 4, L * vw * esz + (b->qtype == SMRE_Q_FP32 ? 0 : vw * 4));
        if (need > ring) {
            bfail(b, SMRE_EINVAL, "side %d: block of %zu bytes above the %zu-byte ring", L, need, ring);
            return bail(SMRE_EINVAL);
        }
    }
    CREATE_CK(batch_prepare(b->qtype, b->smem));
    b->arena_bytes = align256(p->device_bytes);
    CREATE_CK(dev_malloc(&b->arena, b->arena_bytes));
    b->heap.reset(b->arena_bytes);
    CREATE_CK(dev_malloc(&b->d_imgs, sizeof(BImage) * b->max_images));
    CREATE_CK(dev_malloc(&b->d_ctl, sizeof(Control) * b->max_images));
    CREATE_CK(cudaMemset(b->d_ctl, 0, sizeof(Control) * b->max_images));
    CREATE_CK(dev_malloc(&b->d_err, sizeof(int)));
    CREATE_CK(cudaMemset(b->d_err, 0, sizeof(int)));
    b->tab_ints = (size_t)b->max_images + b->steps.size() * (2 * (size_t)b->max_images + 1) +
                  (size_t)b->max_images + 1;
    CREATE_CK(dev_malloc(&b->d_tab, sizeof(int) * b->tab_ints));
    CREATE_CK(dev_malloc(&b->d_groups, sizeof(BGroup) * b->steps.size()));
    CREATE_CK(host_malloc(&b->h_ctl, sizeof(Control) * b->max_images));
    CREATE_CK(host_malloc(&b->h_err, sizeof(int)));
    CREATE_CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    memset(b->h_ctl, 0, sizeof(Control) * b->max_images);
    *b->h_err = 0;
#undef CREATE_CK
    b->slots.resize(b->max_images);
    *out = b;
    return SMRE_OK;
}

smre_status smre_batch_submit(smre_batch *b, int height, int width, const float *x0, int *slot)
{
    return smre::batch_submit_ld(b, height, width, x0, width, slot);
}

}  // extern "C"

smre_status smre::batch_submit_ld(smre_batch *b, int height, int width, const float *x0, int ld,
                                  int *slot)
{
    if (!b) return bfail(nullptr, SMRE_EINVAL, "batch is NULL");
    if (!slot || !x0) return bfail(b, SMRE_EINVAL, "x0 / slot is NULL");
    *slot = -1;
    Layout lo;
    if (!image_layout(b->sides, b->qtype, b->hist_cap, height, width, lo))
        return bfail(b, SMRE_EINVAL, "image %d x %d not supported (1..65535 x 1..%d, sides <= min(H, W))",
                     height, width, kBatchMaxWidth);
    int s = -1;
    for (int i = 0; i < b->max_images; ++i)
        if (!b->slots[i].used) { s = i; break; }
    if (s < 0) return SMRE_OK;          // no free slot now
    size_t off;
    if (!b->heap.alloc(lo.total, off)) return SMRE_OK;   // no room now
    auto &sl = b->slots[s];
    unsigned char *base = b->arena + off;
    BImage &im = sl.img;
    im.x = reinterpret_cast<float *>(base + lo.x);
    im.xprev = reinterpret_cast<float *>(base + lo.xprev);
    im.q = base + lo.q;
    im.qs = b->qtype != SMRE_Q_FP32 ? reinterpret_cast<float *>(base + lo.qs) : nullptr;
    im.qoff = reinterpret_cast<const long long *>(base + lo.qoff);
    im.soff = reinterpret_cast<const long long *>(base + lo.soff);
    im.ctl = b->d_ctl + s;
    im.hist = reinterpret_cast<double *>(base + lo.hist);
    im.part = reinterpret_cast<double *>(base + lo.part);
    im.uflag = reinterpret_cast<unsigned *>(base + lo.uflag);
    im.H = height;
    im.W = width;
    im.pitch = lo.pitch;
    im.nchunks = lo.nchunks;
    im.hist_cap = b->hist_cap;
    auto release = [&]() { b->heap.release(off, lo.total); };
#define SUB_CK(call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            release();                                                                       \
            return bfail(b, SMRE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));            \
        }                                                                                    \
    } while (0)
    const size_t np = lo.qoff_tab.size();
    SUB_CK(cudaMemcpyAsync(base + lo.qoff, lo.qoff_tab.data(), sizeof(long long) * np,
                           cudaMemcpyHostToDevice, b->stream));
    SUB_CK(cudaMemcpyAsync(base + lo.soff, lo.soff_tab.data(), sizeof(long long) * np,
                           cudaMemcpyHostToDevice, b->stream));
    SUB_CK(cudaMemcpyAsync(b->d_imgs + s, &im, sizeof(BImage), cudaMemcpyHostToDevice, b->stream));
    SUB_CK(cudaMemcpy2DAsync(im.x, sizeof(float) * lo.pitch, x0, sizeof(float) * ld,
                             sizeof(float) * width, height, cudaMemcpyDefault, b->stream));
    SUB_CK(cudaMemcpy2DAsync(im.xprev, sizeof(float) * lo.pitch, im.x, sizeof(float) * lo.pitch,
                             sizeof(float) * width, height, cudaMemcpyDeviceToDevice, b->stream));
    SUB_CK(cudaMemsetAsync(b->d_ctl + s, 0, sizeof(Control), b->stream));
    SUB_CK(cudaMemsetAsync(im.uflag, 0, sizeof(unsigned) * (size_t)height, b->stream));
#undef SUB_CK
    sl.used = true;
    sl.done = false;
    sl.H = height;
    sl.W = width;
    sl.off = off;
    sl.bytes = lo.total;
    sl.windows_per_cycle = lo.windows_per_cycle;
    sl.t_submit = now_seconds();
    memset(&b->h_ctl[s], 0, sizeof(Control));
    b->active.push_back(s);
    b->dirty = true;
    *slot = s;
    return SMRE_OK;
}

extern "C" {

namespace {

// Item tables and the cycle's graph up to date for the active images.
smre_status prepare_cycle(smre_batch *b)
{
    if (b->dirty) {
        smre_status st = rebuild_tables(b);
        if (st != SMRE_OK) return st;
    }
    if (b->graph_ok && b->graph_dirty) capture_cycle(b);
    return SMRE_OK;
}

smre_status launch_cycles(smre_batch *b, int cycles)
{
    for (int c = 0; c < cycles; ++c) {
        if (b->gexec) {
            BCK(b, cudaGraphLaunch(b->gexec, b->stream));
            b->launches += b->cycle_kernels;
        } else {
            smre_status st = enqueue_cycle(b, b->stream);
            if (st != SMRE_OK) return st;
        }
    }
    return SMRE_OK;
}

void set_spread(smre_batch *b, int spread)
{
    if (b->spread != spread) {
        b->spread = spread;
        b->dirty = true;
    }
}

void set_per_side(smre_batch *b, bool per_side)
{
    if (b->per_side != per_side) {
        b->per_side = per_side;
        b->graph_dirty = true;
    }
}

// A schedule as cached: the spread, plus 256 for one launch per side.
void set_schedule(smre_batch *b, int code)
{
    set_spread(b, code & 255);
    set_per_side(b, (code & 256) != 0);
}

// SMRE_BF_AUTOTUNE: pick the schedule (one launch per group or per side) and
// the spread for the active set of shapes, from the process-wide cache or by
// timing one cycle of each candidate (after one untimed cycle: images that
// just joined read no increments in their first cycle).  The cycles it runs
// are counted against `cycles`; the results do not depend on the schedule.
smre_status tune_spread(smre_batch *b, int &cycles)
{
    const std::string key = spread_key(b);
    if (key == b->tuned_key) return SMRE_OK;
    {
        std::lock_guard<std::mutex> lk(g_spread_mu);
        auto it = g_spread_cache.find(key);
        if (it != g_spread_cache.end()) {
            set_schedule(b, it->second);
            b->tuned = 2;
            b->tuned_key = key;
            return SMRE_OK;
        }
    }
    static const int kCand[] = {1, 4, 256 | 1, 256 | 4};
    if (cycles < 1 + (int)(sizeof(kCand) / sizeof(kCand[0]))) return SMRE_OK;   // tune later
    smre_status st = prepare_cycle(b);
    if (st == SMRE_OK) st = launch_cycles(b, 1);
    if (st != SMRE_OK) return st;
    --cycles;
    if (!b->tev0) BCK(b, cudaEventCreate(&b->tev0));
    if (!b->tev1) BCK(b, cudaEventCreate(&b->tev1));
    int best = b->spread | (b->per_side ? 256 : 0);
    float best_ms = 1e30f;
    for (int cand : kCand) {
        set_schedule(b, cand);
        st = prepare_cycle(b);
        if (st != SMRE_OK) return st;
        BCK(b, cudaEventRecord(b->tev0, b->stream));
        st = launch_cycles(b, 1);
        if (st != SMRE_OK) return st;
        BCK(b, cudaEventRecord(b->tev1, b->stream));
        BCK(b, cudaEventSynchronize(b->tev1));
        float ms = 0.f;
        BCK(b, cudaEventElapsedTime(&ms, b->tev0, b->tev1));
        --cycles;
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    set_schedule(b, best);
    b->tuned = 1;
    b->tuned_key = key;
    std::lock_guard<std::mutex> lk(g_spread_mu);
    g_spread_cache[key] = best;
    return SMRE_OK;
}

}  // namespace

smre_status smre_batch_run(smre_batch *b, int cycles)
{
    if (!b) return bfail(nullptr, SMRE_EINVAL, "batch is NULL");
    if (cycles < 0) return bfail(b, SMRE_EINVAL, "cycles is negative");
    if (b->active.empty() || cycles == 0) return SMRE_OK;
    if (b->autotune) {
        smre_status st = tune_spread(b, cycles);
        if (st != SMRE_OK) return st;
    }
    smre_status st = prepare_cycle(b);
    if (st != SMRE_OK) return st;
    return launch_cycles(b, cycles);
}

int smre_batch_item_spread(const smre_batch *b, int *tuned)
{
    if (tuned) *tuned = b ? b->tuned : 0;
    return b ? b->spread : 0;
}

int smre_batch_per_side(const smre_batch *b) { return b && b->per_side ? 1 : 0; }

smre_status smre_batch_poll(smre_batch *b, int *done, int max_done, int *n_done)
{
    if (!b) return bfail(nullptr, SMRE_EINVAL, "batch is NULL");
    if (n_done) *n_done = 0;
    BCK(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(Control) * b->max_images,
                           cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (*b->h_err) {
        BCK(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
        return bfail(b, (smre_status)*b->h_err, "a device-side wait ran out of time");
    }
    const double t = now_seconds();
    int k = 0;
    for (int s : b->active) {
        auto &sl = b->slots[s];
        if (sl.done || !b->h_ctl[s].stop) continue;
        sl.done = true;
        sl.t_done = t;
        if (done && k < max_done) done[k] = s;
        ++k;
    }
    if (n_done) *n_done = std::min(k, max_done);
    return SMRE_OK;
}

smre_status smre_batch_retrieve(smre_batch *b, int slot, float *x, smre_result *res)
{
    const int ld = b && slot >= 0 && slot < b->max_images ? b->slots[slot].W : 0;
    return smre::batch_retrieve_ld(b, slot, x, ld, res);
}

}  // extern "C"

smre_status smre::batch_retrieve_ld(smre_batch *b, int slot, float *x, int ld, smre_result *res)
{
    if (!b) return bfail(nullptr, SMRE_EINVAL, "batch is NULL");
    if (slot < 0 || slot >= b->max_images || !b->slots[slot].used)
        return bfail(b, SMRE_EINVAL, "slot %d holds no image", slot);
    auto &sl = b->slots[slot];
    if (!sl.done) return bfail(b, SMRE_EINVAL, "slot %d has not finished (poll first)", slot);
    if (x)
        BCK(b, cudaMemcpy2DAsync(x, sizeof(float) * ld, sl.img.x, sizeof(float) * sl.img.pitch,
                                 sizeof(float) * sl.W, sl.H, cudaMemcpyDefault, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    const Control &c = b->h_ctl[slot];
    if (res) {
        res->cycles = c.cycles;
        res->status = c.status;
        res->step = c.step;
        res->rel_step = c.prev_norm > 0 ? c.step / c.prev_norm : 0.0;
        res->max_violation = NAN;
        res->windows = (long long)c.cycles * sl.windows_per_cycle;
        res->max_tile_sweeps = 0;
        res->seconds = sl.t_done - sl.t_submit;
    }
    const int status = c.status;
    if (status == SMRE_EINVAL)
        bfail(b, SMRE_EINVAL, "slot %d: the image holds a NaN or an infinity (the first cycle's "
              "norm is not finite)", slot);
    b->heap.release(sl.off, sl.bytes);
    sl.used = false;
    sl.done = false;
    b->active.erase(std::find(b->active.begin(), b->active.end(), slot));
    b->dirty = true;
    return (smre_status)status;
}

extern "C" {

smre_status smre_batch_project(smre_batch *b, int n, const int *heights, const int *widths,
                               const float *const *x0, float *const *x, smre_result *res)
{
    if (!b) return bfail(nullptr, SMRE_EINVAL, "batch is NULL");
    if (n < 1 || !heights || !widths || !x0 || !x)
        return bfail(b, SMRE_EINVAL, "need n >= 1 images with sizes and pointers");
    if (!b->active.empty()) return bfail(b, SMRE_EINVAL, "the batch already holds images");
    std::vector<int> slot(n, -1);
    auto drop = [&]() {
        for (int s : slot)
            if (s >= 0) {
                b->heap.release(b->slots[s].off, b->slots[s].bytes);
                b->slots[s].used = false;
            }
        b->active.clear();
        b->dirty = true;
    };
    for (int i = 0; i < n; ++i) {
        smre_status st = smre_batch_submit(b, heights[i], widths[i], x0[i], &slot[i]);
        if (st != SMRE_OK || slot[i] < 0) {
            drop();
            if (st != SMRE_OK) return st;
            return bfail(b, SMRE_ENOMEM, "image %d (%d x %d) does not fit the batch's slots or arena",
                         i, heights[i], widths[i]);
        }
    }
    int remaining = n;
    std::vector<int> done(n);
    int ran = 0;
    while (remaining > 0) {
        const int k = std::min(8, std::max(1, b->max_cycles - ran));
        smre_status st = smre_batch_run(b, k);
        if (st != SMRE_OK) { drop(); return st; }
        ran += k;
        int nd = 0;
        st = smre_batch_poll(b, done.data(), n, &nd);
        if (st != SMRE_OK) { drop(); return st; }
        remaining -= nd;
    }
    smre_status worst = SMRE_OK;
    for (int i = 0; i < n; ++i) {
        smre_status st = smre_batch_retrieve(b, slot[i], x[i], res ? res + i : nullptr);
        if (st == SMRE_ECUDA || st == SMRE_EINVAL) return st;
        if (st != SMRE_OK && worst == SMRE_OK) worst = st;
    }
    return worst;
}

int smre_batch_active(const smre_batch *b) { return b ? (int)b->active.size() : 0; }

long long smre_batch_kernel_launches(const smre_batch *b) { return b ? b->launches : 0; }

size_t smre_batch_device_bytes(const smre_batch *b)
{
    if (!b) return 0;
    return b->arena_bytes + sizeof(BImage) * b->max_images + sizeof(Control) * b->max_images +
           sizeof(int) * (b->tab_ints + 1);
}

const char *smre_batch_last_error(const smre_batch *b)
{
    if (b) return b->err.c_str();
    return smre_last_error(nullptr);
}

void smre_batch_destroy(smre_batch *b) { free_batch(b); }

}  // extern "C"

namespace smre {

void batch_drop(smre_batch *b, int slot)
{
    if (!b || slot < 0 || slot >= b->max_images || !b->slots[slot].used) return;
    auto &sl = b->slots[slot];
    cudaStreamSynchronize(b->stream);
    b->heap.release(sl.off, sl.bytes);
    sl.used = false;
    sl.done = false;
    b->active.erase(std::find(b->active.begin(), b->active.end(), slot));
    b->dirty = true;
}

smre_status batch_set_rule(smre_batch *b, int max_cycles, double tol, int tol_relative)
{
    if (max_cycles > b->hist_cap)
        return bfail(b, SMRE_EINVAL, "max_cycles %d above the batch's history of %d", max_cycles,
                     b->hist_cap);
    b->max_cycles = max_cycles;
    b->tol = tol;
    b->tol_relative = tol_relative ? 1 : 0;
    b->graph_dirty = true;
    return SMRE_OK;
}

smre_status batch_run_one(smre_batch *b, int height, int width, const float *x0, float *x,
                          int ld, double *hist, int hist_cap, Control *ctl_out)
{
    if (!b->active.empty()) return bfail(b, SMRE_EINVAL, "the batch already holds images");
    int slot = -1;
    smre_status st = batch_submit_ld(b, height, width, x0, ld, &slot);
    if (st != SMRE_OK) return st;
    if (slot < 0) return bfail(b, SMRE_ENOMEM, "image does not fit the batch arena");
    int ran = 0, n_done = 0, done = -1;
    while (n_done == 0) {
        const int k = std::min(8, std::max(1, b->max_cycles - ran));
        st = smre_batch_run(b, k);
        if (st == SMRE_OK) st = smre_batch_poll(b, &done, 1, &n_done);
        if (st != SMRE_OK) {
            b->heap.release(b->slots[slot].off, b->slots[slot].bytes);
            b->slots[slot].used = false;
            b->active.clear();
            b->dirty = true;
            return st;
        }
        ran += k;
    }
    const Control c = b->h_ctl[slot];
    if (ctl_out) *ctl_out = c;
    const int n = std::min(c.cycles, std::min(hist_cap, b->hist_cap));
    if (hist && n > 0)
        BCK(b, cudaMemcpyAsync(hist, b->slots[slot].img.hist, sizeof(double) * 2 * n,
                               cudaMemcpyDeviceToDevice, b->stream));
    st = batch_retrieve_ld(b, slot, x, ld, nullptr);
    return st == SMRE_ENOTCONVERGED ? SMRE_OK : st;
}

}  // namespace smre
