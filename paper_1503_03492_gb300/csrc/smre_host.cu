// Host side of libsmre.so: argument checking, bounds, the cycle schedule
// (Sec. 2.3 set order), device buffers and the C ABI of include/smre.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "smre_internal.h"

using namespace smre;

struct smre_dykstra {
    // problem
    int H = 0, W = 0, pitch = 0;
    std::vector<int> sides;        // ascending, unique
    std::vector<double> cS;        // aligned with sides
    double cS_of[kMaxSide + 1] = {};
    smre_cmode cmode = SMRE_C_PERSET;
    double alpha = 0.9;
    int maxstat_draws = 1000;
    unsigned long long seed = 0;
    int flags = 0;
    int max_ctas = 0;
    int q_dtype = 0;
    // a one-image batch runs the standard method instead of the handle's own
    // kernels (16-bit increments, or FP32 images too wide for the persistent
    // kernel); see use_batch
    smre_batch *bat = nullptr;
    bool persist_ok = false;       // the persistent plan exists (it may not be the one used)
    std::string tuned;             // "", "measured" or "cached"
    // stopping rule
    int max_cycles = 1;
    double tol = -1.0;
    int tol_relative = 0;
    int icd_max_sweeps = 1000;
    // schedule
    std::vector<Group> groups;
    std::vector<Tiling> tilings;
    long long windows_per_cycle = 0;
    // device state
    cudaStream_t stream = nullptr;
    float *q = nullptr;
    size_t q_floats = 0;
    float *xw = nullptr, *xprev = nullptr;
    double *partials = nullptr;
    int n_partials = 0;
    double *hist = nullptr;
    int hist_cap = 0;
    Control *ctl = nullptr;
    Control *ctl_host = nullptr;   // pinned
    int *icd_sweeps = nullptr;
    int icd_sweeps_cap = 0;
    int last_icd_tiles = 0;
    int last_cycles = 0;
    double *viol = nullptr;
    double *viol_host = nullptr;   // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    size_t dev_bytes = 0;
    long long launches = 0;
    // persistent path plan
    bool persist = false;
    int p_grid = 0, p_threads = 0, p_stages = 0, p_ncw = 0, p_maxL = 0;
    size_t p_smem = 0;
    int p_stage_floats = 0, p_stage_offset = 0, p_sp = 0;
    bool p_reg = false;            // the register-band kernel (else the shared-memory band)
    int n_tasks = 0;               // flags: events x (consumer warps of the register kernel)
    unsigned char *d_sched = nullptr;
    int *d_cta_off = nullptr;
    int p_sched_bytes = 0;
    unsigned *d_flags = nullptr, *d_barrier = nullptr, *d_selftest = nullptr;
    double *d_ppartials = nullptr;
    float *d_zeros = nullptr;
    unsigned long long *d_xch = nullptr;   // register kernel: tagged transition rows
    unsigned *d_smid = nullptr;            // register kernel: SM id of each CTA
    unsigned tag_next = 1;                 // tag base of the next persistent launch
    size_t xch_words = 0;
    int *d_abort = nullptr;
    unsigned long long timeout_ns = 10000000000ull;
    std::string err;
};

namespace {

thread_local std::string g_err;

smre_status fail(smre_dykstra *h, smre_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_err = buf;
    return s;
}

#define CK(h, call)                                                                     \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail((h), e_ == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Common validation of the problem description; fills sides (ascending).
smre_status check_params(const smre_params *p, std::vector<int> &sides, std::vector<double> &cexp)
{
    if (!p) return fail(nullptr, SMRE_EINVAL, "params is NULL");
    if (p->height < 1 || p->width < 1 || p->height > 65535)
        return fail(nullptr, SMRE_EINVAL, "image %d x %d out of range", p->height, p->width);
    if (p->width > kMaxWidth)
        return fail(nullptr, SMRE_EINVAL, "width %d above the supported %d", p->width, kMaxWidth);
    if (!p->sides || p->n_sides < 1 || p->n_sides > 64)
        return fail(nullptr, SMRE_EINVAL, "need 1..64 window sides");
    std::vector<std::pair<int, double>> sv;
    for (int i = 0; i < p->n_sides; ++i) {
        const int L = p->sides[i];
        if (L < 1 || L > kMaxSide || L > p->height || L > p->width)
            return fail(nullptr, SMRE_EINVAL, "window side %d outside 1..min(%d, H, W)", L, kMaxSide);
        double c = 0.0;
        if (p->cmode == SMRE_C_EXPLICIT) {
            if (!p->c_explicit) return fail(nullptr, SMRE_EINVAL, "c_explicit is NULL");
            c = p->c_explicit[i];
            if (!(c > 0.0) || !std::isfinite(c))
                return fail(nullptr, SMRE_EINVAL, "bound %g of side %d is not a positive number", c, L);
        }
        sv.emplace_back(L, c);
    }
    std::stable_sort(sv.begin(), sv.end(), [](auto &a, auto &b) { return a.first < b.first; });
    sides.clear();
    cexp.clear();
    for (auto &pr : sv) {
        if (sides.empty() || sides.back() != pr.first) {
            sides.push_back(pr.first);
            cexp.push_back(pr.second);
        } else if (pr.second != cexp.back()) {
            // a repeated side is ignored only when it repeats the bound too
            return fail(nullptr, SMRE_EINVAL, "side %d listed twice with different bounds (%g, %g)",
                        pr.first, cexp.back(), pr.second);
        }
    }
    if (p->cmode != SMRE_C_EXPLICIT && !(p->alpha > 0.0 && p->alpha < 1.0))
        return fail(nullptr, SMRE_EINVAL, "alpha %g outside (0, 1)", p->alpha);
    if ((int)p->cmode < 0 || (int)p->cmode > 3)
        return fail(nullptr, SMRE_EINVAL, "unknown cmode %d", (int)p->cmode);
    if (p->q_dtype < SMRE_Q_FP32 || p->q_dtype > SMRE_Q_FP16)
        return fail(nullptr, SMRE_EINVAL, "q_dtype %d unknown", p->q_dtype);
    if (p->q_dtype != SMRE_Q_FP32 &&
        (p->width > kBatchMaxWidth || sides.back() > kBatchMaxSide))
        return fail(nullptr, SMRE_EINVAL, "16-bit increments need width <= %d and sides <= %d",
                    kBatchMaxWidth, kBatchMaxSide);
    if (p->max_cycles < 1) return fail(nullptr, SMRE_EINVAL, "max_cycles must be >= 1");
    if (std::isnan(p->tol)) return fail(nullptr, SMRE_EINVAL, "tol is NaN");
    if (p->icd_max_sweeps < 0 || p->maxstat_draws < 0)
        return fail(nullptr, SMRE_EINVAL, "negative sweep cap or draw count");
    if (p->max_ctas < 0) return fail(nullptr, SMRE_EINVAL, "max_ctas is negative");
    return SMRE_OK;
}

// Monte Carlo quantile of Q_Omega on the device (MAXSTAT).
smre_status maxstat_q(const smre_params *p, const std::vector<int> &sides, double &q_out)
{
    const int H = p->height, W = p->width, pitch = round_up(W, 32);
    const int draws = p->maxstat_draws ? p->maxstat_draws : 1000;
    const size_t per = (size_t)H * pitch;
    int batch = (int)std::max<size_t>(1, std::min<size_t>(64, (size_t)(256u << 20) / (per * 4)));
    batch = std::min(batch, draws);
    float *img = nullptr;
    double *mx = nullptr;
    cudaStream_t s = nullptr;
    std::vector<double> all(draws), part(batch);
    cudaError_t e = dev_malloc(&img, per * batch * sizeof(float));
    if (e == cudaSuccess) e = dev_malloc(&mx, 2 * batch * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (int d0 = 0; e == cudaSuccess && d0 < draws; d0 += batch) {
        const int n = std::min(batch, draws - d0);
        e = launch_maxstat(H, W, pitch, sides.data(), (int)sides.size(), d0, n, p->seed, img, mx, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), mx + n, n * sizeof(double),
                                                  cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int i = 0; i < n && e == cudaSuccess; ++i) all[d0 + i] = part[i];
    }
    if (s) cudaStreamDestroy(s);
    cudaFree(img);
    cudaFree(mx);
    if (e != cudaSuccess)
        return fail(nullptr, e == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA,
                    "MAXSTAT Monte Carlo: %s", cudaGetErrorString(e));
    std::sort(all.begin(), all.end());
    int idx = (int)std::ceil(p->alpha * draws) - 1;
    idx = std::max(0, std::min(draws - 1, idx));
    q_out = all[idx];
    return SMRE_OK;
}

// Whether the handle projects through a one-image batch: always for 16-bit
// increments (only the batched kernels store them), and for FP32 images
// wider than the persistent kernel takes, where the batched step kernel beats
// one launch per group (unless the caller asked for group launches).
bool use_batch(const smre_params *p, int max_side)
{
    if (p->q_dtype != SMRE_Q_FP32) return true;
    if (p->flags & SMRE_F_GROUP_LAUNCHES) return false;
    return persist_smem_pitch(round_up(p->width, 32)) == 0 && p->width <= kBatchMaxWidth &&
           max_side <= kBatchMaxSide;
}

smre_status make_handle_batch(smre_dykstra *h)
{
    if (h->bat) {
        smre_batch_destroy(h->bat);
        h->bat = nullptr;
    }
    smre_batch_params bp{};
    bp.sides = h->sides.data();
    bp.n_sides = (int)h->sides.size();
    bp.cmode = SMRE_C_EXPLICIT;
    bp.c_explicit = h->cS.data();
    bp.max_cycles = std::max(h->max_cycles, 3);   // room for the tuner's three cycles
    bp.tol = h->tol;
    bp.tol_relative = h->tol_relative;
    bp.q_dtype = h->q_dtype;
    bp.max_images = 1;
    // one cooperative launch per side when a group has more window-rows than
    // there are SMs: the second round of a group's items no longer leaves
    // most SMs idle (2048 x 2048, sides 1..12: 8 % faster per cycle), with
    // the same bits
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        h->H / h->sides.back() > sms)
        bp.flags |= SMRE_BF_PER_SIDE;
    bp.device_bytes = smre_batch_image_bytes(&bp, h->H, h->W) + 4096;
    const smre_status st = smre_batch_create(&bp, h->stream, &h->bat);
    if (st != SMRE_OK) return fail(h, st, "one-image batch: %s", smre_batch_last_error(nullptr));
    batch_set_rule(h->bat, h->max_cycles, h->tol, h->tol_relative);
    return SMRE_OK;
}

// ---- schedule autotuner (SMRE_F_AUTOTUNE)
//
// For one problem shape the standard method can run as the persistent
// cooperative launch, as a one-image batch (one step-kernel launch per group)
// or as one group-kernel launch per group with a host stop check per cycle.
// Which is fastest depends on the size and the sides, so the tuner times
// three cycles of each applicable schedule on a seeded test image (the time of
// a cycle hardly depends on the values) and keeps the fastest.  The choice is
// cached per (device, H, W, sides, q_dtype) for the process.

using TuneKey = std::tuple<int, int, int, std::vector<int>, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune_cache;

smre_status project_core(smre_dykstra *h, const float *x0, float *x, smre_result *res);

int current_schedule(const smre_dykstra *h)
{
    if (h->bat) return SMRE_SCHED_BATCHED;
    return h->persist ? SMRE_SCHED_PERSISTENT : SMRE_SCHED_GROUPS;
}

// Point the handle at schedule s (its state must exist).
void use_schedule(smre_dykstra *h, int s, smre_batch *bat)
{
    h->bat = s == SMRE_SCHED_BATCHED ? bat : nullptr;
    h->persist = s == SMRE_SCHED_PERSISTENT;
}

smre_status autotune(smre_dykstra *h)
{
    int dev = 0;
    CK(h, cudaGetDevice(&dev));
    const TuneKey key{dev, h->H, h->W, h->sides, h->q_dtype};
    int cached = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) cached = it->second;
    }
    smre_batch *bat = h->bat;   // made at create when a batch can run the shape
    std::vector<int> cand;
    if (h->q_dtype == SMRE_Q_FP32) {
        if (h->persist_ok) cand.push_back(SMRE_SCHED_PERSISTENT);
        cand.push_back(SMRE_SCHED_GROUPS);
    }
    if (bat) cand.push_back(SMRE_SCHED_BATCHED);
    int best = cand.empty() ? current_schedule(h) : cand[0];
    if (cached) {
        best = cached;
        h->tuned = "cached";
    } else if (cand.size() > 1) {
        // seeded test image: uniform values in [-3, 3) (many windows violate)
        std::vector<float> img((size_t)h->H * h->W);
        unsigned long long z = 0x9E3779B97F4A7C15ull;
        for (float &v : img) {
            z = z * 6364136223846793005ull + 1442695040888963407ull;
            v = (float)((double)(z >> 11) * (6.0 / 9007199254740992.0) - 3.0);
        }
        float *xt = nullptr;
        CK(h, dev_malloc(&xt, sizeof(float) * img.size()));
        {
            const cudaError_t e = cudaMemcpy(xt, img.data(), sizeof(float) * img.size(),
                                             cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(xt);
                return fail(h, SMRE_ECUDA, "autotune image: %s", cudaGetErrorString(e));
            }
        }
        const int mc = h->max_cycles;
        const double tol = h->tol;
        const int rel = h->tol_relative;
        h->max_cycles = 3;
        h->tol = -1.0;
        if (bat) batch_set_rule(bat, 3, -1.0, 0);
        double best_t = 1e300;
        smre_status st = SMRE_OK;
        for (int c : cand) {
            use_schedule(h, c, bat);
            smre_result r{};
            st = project_core(h, xt, xt, &r);
            if (st != SMRE_OK && st != SMRE_ENOTCONVERGED) break;
            st = SMRE_OK;
            if (r.seconds < best_t) {
                best_t = r.seconds;
                best = c;
            }
        }
        cudaFree(xt);
        h->max_cycles = mc;
        h->tol = tol;
        h->tol_relative = rel;
        if (bat) batch_set_rule(bat, mc, tol, rel);
        if (st != SMRE_OK) return st;
        h->tuned = "measured";
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    use_schedule(h, best, bat);
    if (best != SMRE_SCHED_BATCHED && bat) {
        smre_batch_destroy(bat);
        h->bat = nullptr;
    }
    if (best == SMRE_SCHED_BATCHED && h->q_floats > 0) {
        // the batch holds the increments: drop the handle's own store
        cudaFree(h->q);
        h->q = nullptr;
        CK(h, dev_malloc(&h->q, sizeof(float)));
        h->dev_bytes -= sizeof(float) * (h->q_floats - 1);
        h->q_floats = 0;
    }
    return SMRE_OK;
}

smre_status compute_bounds(const smre_params *p, const std::vector<int> &sides,
                           const std::vector<double> &cexp, std::vector<double> &cS)
{
    cS.assign(sides.size(), 0.0);
    switch (p->cmode) {
        case SMRE_C_EXPLICIT: cS = cexp; return SMRE_OK;
        case SMRE_C_CHI2:
            for (size_t i = 0; i < sides.size(); ++i) cS[i] = chi2_quantile(p->alpha, sides[i] * sides[i]);
            return SMRE_OK;
        case SMRE_C_PERSET: {
            const double q = inv_normal_cdf(p->alpha);
            for (size_t i = 0; i < sides.size(); ++i) cS[i] = bound_from_q(q, sides[i]);
            return SMRE_OK;
        }
        case SMRE_C_MAXSTAT: {
            double q = 0.0;
            smre_status st = maxstat_q(p, sides, q);
            if (st != SMRE_OK) return st;
            for (size_t i = 0; i < sides.size(); ++i) cS[i] = bound_from_q(q, sides[i]);
            return SMRE_OK;
        }
    }
    return fail(nullptr, SMRE_EINVAL, "unknown cmode");
}

// Set order of one cycle (Sec. 2.3): sides descending; per side L the groups
// (L, a), a = 0..L-1, each holding the tilings (L, a, b), b = 0..L-1.
void build_schedule(smre_dykstra *h)
{
    h->groups.clear();
    h->tilings.clear();
    long long off = 0;
    h->windows_per_cycle = 0;
    for (auto it = h->sides.rbegin(); it != h->sides.rend(); ++it) {
        const int L = *it;
        for (int a = 0; a < L; ++a) {
            Group g;
            g.L = L;
            g.a = a;
            g.n_units = (h->H - a) / L;
            g.tiling0 = (int)h->tilings.size();
            h->groups.push_back(g);
            for (int b = 0; b < L; ++b) {
                Tiling t;
                t.L = L;
                t.a = a;
                t.b = b;
                t.n_u = (h->H - a) / L;
                t.n_v = (h->W - b) / L;
                t.q_off = off;
                off += (long long)t.n_u * L * h->pitch;
                h->windows_per_cycle += (long long)t.n_u * t.n_v;
                h->tilings.push_back(t);
            }
        }
    }
    h->q_floats = (size_t)off;
}

smre_status ensure_hist(smre_dykstra *h, int cap)
{
    if (cap <= h->hist_cap) return SMRE_OK;
    if (h->hist) {
        CK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->hist);
        h->dev_bytes -= sizeof(double) * 2 * h->hist_cap;
        h->hist = nullptr;
    }
    CK(h, dev_malloc(&h->hist, sizeof(double) * 2 * cap));
    h->hist_cap = cap;
    h->dev_bytes += sizeof(double) * 2 * cap;
    return SMRE_OK;
}

smre_status stage_in(smre_dykstra *h, const float *x0)
{
    CK(h, cudaMemcpy2DAsync(h->xw, sizeof(float) * h->pitch, x0, sizeof(float) * h->W,
                            sizeof(float) * h->W, h->H, cudaMemcpyDefault, h->stream));
    return SMRE_OK;
}

smre_status stage_out(smre_dykstra *h, float *x)
{
    CK(h, cudaMemcpy2DAsync(x, sizeof(float) * h->W, h->xw, sizeof(float) * h->pitch,
                            sizeof(float) * h->W, h->H, cudaMemcpyDefault, h->stream));
    return SMRE_OK;
}

smre_status violation(smre_dykstra *h, double &out)
{
    ViolationArgs va{};
    va.x = h->xw;
    va.pitch = h->pitch;
    va.H = h->H;
    va.W = h->W;
    va.n_sides = (int)h->sides.size();
    for (int i = 0; i < va.n_sides; ++i) {
        va.sides[i] = h->sides[i];
        va.cS[i] = h->cS[i];
    }
    CK(h, launch_violation(va, h->partials, h->n_partials, h->viol, h->stream));
    h->launches += 2;
    CK(h, cudaMemcpyAsync(h->viol_host, h->viol, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    out = *h->viol_host;
    return SMRE_OK;
}

// Plan of the persistent kernel.  For every side L the window-rows ("units")
// u = 0..n_u(0)-1 of the side are split into contiguous ranges, one per CTA,
// spread over the CTAs; a CTA keeps its range for all offsets a = 0..L-1 of
// the side (the band of U*L rows slides down one row per offset).  Events
// (side L, CTA c, offset a) publish rows: the band's top row after offsets
// a < L-1, the whole band after a = L-1; each event has a flag.  The plan
// gives every side task the flags of the previous sides' last publishers of
// the rows it may read, every offset the flag of the neighbour whose top row
// it takes over, and the rows each event publishes for the last time in a
// cycle (fused norm).  Leaves h->persist false when the shape does not fit.
smre_status plan_persistent(smre_dykstra *h, int flags)
{
    h->persist = false;
    if (flags & SMRE_F_GROUP_LAUNCHES) return SMRE_OK;
    int dev = 0, sms = 0, smem_optin = 0;
    CK(h, cudaGetDevice(&dev));
    CK(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(h, cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int H = h->H, W = h->W, pitch = h->pitch;
    const int sp = persist_smem_pitch(pitch);
    if (sp == 0) return SMRE_OK;
    int G = std::max(1, std::min(sms, H));
    if (h->max_ctas > 0) G = std::min(G, h->max_ctas);

    std::vector<int> sides_desc(h->sides.rbegin(), h->sides.rend());
    struct Side0 {
        int L, c, u0, u1;
        std::vector<int> deps;        // flag ids
        std::vector<int> nb;          // per offset: neighbour flag or -1
        std::vector<int> Ua;          // per offset: units present
        unsigned top_final = 0;
        unsigned long long end_final = 0;
        int flag0 = 0;
    };
    std::vector<Side0> st;            // in cycle order (sides descending), CTA ascending
    std::vector<int> last_pub(H, -1), last_pub_cta(H, -1);
    std::vector<int> ev_of_row(H, -1);   // for the final masks: (side task index, kind)
    struct Pub { int task, a; };          // a = -1: side end
    std::vector<Pub> last_event(H, {-1, 0});
    int nflags = 0;
    int maxL = 0;
    for (int L : sides_desc) {
        maxL = std::max(maxL, L);
        std::vector<int> nu(L);
        for (int a = 0; a < L; ++a) nu[a] = (H - a) / L;
        const int n0 = nu[0];
        if (n0 <= 0) continue;
        // unit ranges: unit u belongs to CTA floor(u G / n0) (spread over all CTAs)
        std::vector<int> owner(n0);
        for (int u = 0; u < n0; ++u) owner[u] = (int)(((long long)u * G) / n0);
        const size_t first_task = st.size();
        for (int u = 0; u < n0;) {
            int v = u + 1;
            while (v < n0 && owner[v] == owner[u]) ++v;
            Side0 t;
            t.L = L;
            t.c = owner[u];
            t.u0 = u;
            t.u1 = v;
            t.flag0 = nflags;
            nflags += L;
            t.Ua.resize(L);
            t.nb.assign(L, -1);
            for (int a = 0; a < L; ++a) t.Ua[a] = std::max(0, std::min(v, nu[a]) - u);
            st.push_back(t);
            u = v;
        }
        // side-start dependencies: last publishers (other CTAs) of every row a
        // task may read during the side: [L u0, L u0 + U L + L - 1)
        for (size_t k = first_task; k < st.size(); ++k) {
            Side0 &t = st[k];
            const int r0 = t.L * t.u0, r1 = std::min(H, r0 + (t.u1 - t.u0) * t.L + t.L - 1);
            for (int r = r0; r < r1; ++r) {
                const int f = last_pub[r];
                if (f >= 0 && last_pub_cta[r] != t.c &&
                    std::find(t.deps.begin(), t.deps.end(), f) == t.deps.end())
                    t.deps.push_back(f);
            }
        }
        // neighbour flags: at offset a >= 1 the task takes row (a-1) + L u1, the top
        // row its lower neighbour (the task owning unit u1) published after offset
        // a-1 -- the neighbour slides and publishes at every offset, with or without
        // units, so it holds that row's latest value; the last task reads it from
        // the image (no task of this side touched it; the side-start flags cover it)
        for (size_t k = first_task; k < st.size(); ++k) {
            Side0 &t = st[k];
            const bool has_nb = k + 1 < st.size() && st[k + 1].L == L;
            for (int a = 1; a < L; ++a)
                if (has_nb) t.nb[a] = st[k + 1].flag0 + (a - 1);
        }
        // events of the side, in order: top rows after a < L-1, bands at a = L-1
        for (int a = 0; a < L; ++a)
            for (size_t k = first_task; k < st.size(); ++k) {
                Side0 &t = st[k];
                const int band = (t.u1 - t.u0) * L;
                const int top = a + L * t.u0;
                const int f = t.flag0 + a;
                if (a < L - 1) {
                    last_pub[top] = f;
                    last_pub_cta[top] = t.c;
                    last_event[top] = {(int)k, a};
                } else {
                    for (int i = 0; i < band && top + i < H; ++i) {
                        last_pub[top + i] = f;
                        last_pub_cta[top + i] = t.c;
                        last_event[top + i] = {(int)k, -1 - i};
                    }
                }
            }
    }
    // rows published for the last time in the cycle: norm there
    for (int r = 0; r < H; ++r) {
        const Pub e = last_event[r];
        if (e.task < 0) return SMRE_OK;   // a row no side touches: keep the group path
        if (e.a >= 0) st[e.task].top_final |= 1u << e.a;
        else st[e.task].end_final |= 1ull << (-1 - e.a);
    }

    // per-CTA schedule segments: header | SideS[] | GrpS[] | pass q offsets | deps
    std::vector<unsigned char> sched;
    std::vector<int> cta_off(G, 0);
    int max_items = 1;
    double items_ratio = 0.0;
    long long stage_floats = 0;
    long long stage_floats_reg = 0;   // U L pitch: the register kernel's stages are packed rows
    int max_band = 0;
    size_t seg_max = 16;
    for (int c = 0; c < G; ++c) {
        std::vector<SideS> ss;
        std::vector<GrpS> gs;
        std::vector<long long> qo;
        std::vector<int> dl;
        // tiling index of (L, a, 0): offset in the cycle order
        for (size_t k = 0; k < st.size(); ++k) {
            const Side0 &t = st[k];
            if (t.c != c) continue;
            const int L = t.L, U = t.u1 - t.u0;
            if (U * L > 64) return SMRE_OK;      // final masks are 64-bit
            SideS x{};
            x.L = L;
            x.U = U;
            x.r0 = L * t.u0;
            x.dep_begin = (int)dl.size();
            for (int f : t.deps) dl.push_back(f);
            x.dep_count = (int)dl.size() - x.dep_begin;
            x.grp0 = (int)gs.size();
            x.pass0 = (int)qo.size();
            x.flag0 = t.flag0;
            x.top_final = t.top_final;
            x.end_final = t.end_final;
            x.cS = (float)h->cS_of[L];
            x.sqrt_cS = (float)std::sqrt(h->cS_of[L]);
            x.cS64 = h->cS_of[L];
            int g_index = -1;
            for (size_t g = 0; g < h->groups.size(); ++g)
                if (h->groups[g].L == L && h->groups[g].a == 0) g_index = (int)g;
            for (int a = 0; a < L; ++a) {
                gs.push_back({t.Ua[a], t.nb[a]});
                const Group &gr = h->groups[g_index + a];
                for (int b = 0; b < L; ++b)
                    qo.push_back(h->tilings[gr.tiling0 + b].q_off + (long long)t.u0 * L * pitch);
            }
            ss.push_back(x);
            const int wpw = 32 / L, nv = W / L;
            const int items = U * ((nv + wpw - 1) / wpw);
            max_items = std::max(max_items, items);
            items_ratio = std::max(items_ratio, (double)items / max_items_for_side(L));
            stage_floats = std::max(stage_floats, (long long)U * L * sp);
            stage_floats_reg = std::max(stage_floats_reg, (long long)U * L * pitch);
            max_band = std::max(max_band, U * L);
        }
        const int hdr[4] = {(int)ss.size(), (int)gs.size(), (int)qo.size(), (int)dl.size()};
        const size_t bytes = sizeof(hdr) + sizeof(SideS) * ss.size() + sizeof(GrpS) * gs.size() +
                             sizeof(long long) * qo.size() + sizeof(int) * dl.size();
        const size_t padded = (bytes + 15) / 16 * 16;
        cta_off[c] = (int)sched.size();
        const size_t at = sched.size();
        sched.resize(at + padded, 0);
        unsigned char *w = sched.data() + at;
        memcpy(w, hdr, sizeof(hdr));
        w += sizeof(hdr);
        memcpy(w, ss.data(), sizeof(SideS) * ss.size());
        w += sizeof(SideS) * ss.size();
        memcpy(w, gs.data(), sizeof(GrpS) * gs.size());
        w += sizeof(GrpS) * gs.size();
        memcpy(w, qo.data(), sizeof(long long) * qo.size());
        w += sizeof(long long) * qo.size();
        memcpy(w, dl.data(), sizeof(int) * dl.size());
        seg_max = std::max(seg_max, padded);
    }

    if (!persist_supported(maxL)) return SMRE_OK;
    const size_t stage_offset = 512 + (seg_max + 127) / 128 * 128;
    const size_t budget = (size_t)smem_optin - 1024;   // static shared memory and slack
    int ncw = 0, threads = 0, S = 0;
    size_t smem = 0, reg_stage_offset = 0;
    bool reg = false;
    if (!(flags & SMRE_F_BAND_IN_SMEM) && persist_reg_fits(pitch, maxL, max_band)) {
        // register-band kernel: warps of 64 columns, stages of packed rows,
        // plus the column-sum exchange arrays
        const int rncw = (pitch + 63) / 64;
        const int rthreads = (rncw + 2) * 32;   // consumers, producer, storer
        const size_t xb = persist_reg_exchange_bytes(pitch);
        const size_t roff = kRegHeaderBytes + (seg_max + 127) / 128 * 128;
        const long long fit = budget > roff + xb
                                  ? (long long)((budget - roff - xb) / (stage_floats_reg * 4))
                                  : 0;
        const int rS = (int)std::min<long long>(kMaxStages, fit);
        const size_t rsmem = roff + (size_t)rS * stage_floats_reg * 4 + xb;
        int occ = 0;
        if (rS >= 3) {
            cudaError_t oe = persist_reg_occupancy(rthreads, rsmem, &occ);
            if (oe != cudaSuccess) {
                cudaGetLastError();
                occ = 0;
            }
        }
        if (occ >= 1) {
            reg = true;
            ncw = rncw;
            threads = rthreads;
            S = rS;
            smem = rsmem;
            stage_floats = stage_floats_reg;
            reg_stage_offset = roff;
        }
    }
    if (!reg) {
        ncw = std::max(4, std::min(kPersistThreads / 32 - 1, max_items));
        if (items_ratio > ncw) return SMRE_OK;   // too many items per warp
        threads = (ncw + 1) * 32;
        const size_t xs_bytes = (size_t)stage_floats * 4;   // the largest band
        if (budget < stage_offset + xs_bytes) return SMRE_OK;
        const long long fit = (long long)((budget - stage_offset - xs_bytes) / (stage_floats * 4));
        S = (int)std::min<long long>(kMaxStages, fit);
        if (S < 3) return SMRE_OK;
        smem = stage_offset + (size_t)S * stage_floats * 4 + xs_bytes;
        int occ = 0;
        cudaError_t oe = persist_occupancy(sp, pitch, threads, smem, &occ);
        if (oe != cudaSuccess || occ < 1) {
            cudaGetLastError();
            return SMRE_OK;
        }
    }
    // the register kernel keeps one flag per (event, consumer warp)
    const int nflag_all = nflags * (reg ? ncw : 1);

    auto up = [&](auto **dptr, const auto &vec) -> cudaError_t {
        using E = typename std::remove_reference<decltype(vec[0])>::type;
        const size_t bytes = sizeof(E) * std::max<size_t>(vec.size(), 1);
        cudaError_t e = dev_malloc((void **)dptr, bytes);
        if (e != cudaSuccess) return e;
        h->dev_bytes += bytes;
        return cudaMemcpy(*dptr, vec.data(), sizeof(E) * vec.size(), cudaMemcpyHostToDevice);
    };
    CK(h, up(&h->d_sched, sched));
    CK(h, up(&h->d_cta_off, cta_off));
    CK(h, dev_malloc(&h->d_flags, sizeof(unsigned) * std::max(nflag_all, 1)));
    CK(h, dev_malloc(&h->d_barrier, 128));   // [0]: per-cycle grid barrier, [16]: launch prologue
    CK(h, dev_malloc(&h->d_selftest, 64));
    CK(h, cudaMemset(h->d_selftest, 0, 64));
    CK(h, dev_malloc(&h->d_abort, 64));
    CK(h, dev_malloc(&h->d_ppartials, sizeof(double) * 4 * G));
    // zero source of the first cycle's copies (one unit-pass of rows at most)
    const size_t zero_floats = reg ? (size_t)stage_floats : (size_t)stage_floats / sp * pitch;
    CK(h, dev_malloc(&h->d_zeros, sizeof(float) * zero_floats));
    CK(h, cudaMemset(h->d_zeros, 0, sizeof(float) * zero_floats));
    h->dev_bytes += sizeof(unsigned) * nflag_all + 192 + sizeof(double) * 4 * G +
                    sizeof(float) * zero_floats;
    h->n_tasks = nflag_all;
    h->p_reg = reg;
    if (reg) {
        // rows handed over at offset transitions: one slot of pitch tagged
        // words per event, zero (no valid tag) until first written
        h->xch_words = (size_t)std::max(nflags, 1) * pitch;
        const size_t xbytes = sizeof(unsigned long long) * h->xch_words;
        CK(h, dev_malloc(&h->d_xch, xbytes));
        CK(h, cudaMemset(h->d_xch, 0, xbytes));
        CK(h, dev_malloc(&h->d_smid, sizeof(unsigned) * G));
        h->dev_bytes += xbytes + sizeof(unsigned) * G;
    }
    h->p_sp = sp;
    h->p_grid = G;
    h->p_threads = threads;
    h->p_stages = S;
    h->p_ncw = ncw;
    h->p_maxL = maxL;
    h->p_smem = smem;
    h->p_stage_floats = (int)stage_floats;
    h->p_stage_offset = (int)(reg ? reg_stage_offset : stage_offset);
    h->p_sched_bytes = (int)seg_max;
    if (const char *env = getenv("SMRE_WAIT_TIMEOUT_MS")) {
        const double ms = atof(env);
        if (ms > 0) h->timeout_ns = (unsigned long long)(ms * 1e6);
    }
    h->persist = true;
    h->persist_ok = true;
    return SMRE_OK;
}

smre_status run_persistent(smre_dykstra *h)
{
    CK(h, cudaMemsetAsync(h->d_flags, 0, sizeof(unsigned) * std::max(h->n_tasks, 1), h->stream));
    CK(h, cudaMemsetAsync(h->d_barrier, 0, 128, h->stream));
    CK(h, cudaMemsetAsync(h->d_abort, 0, 64, h->stream));
    PersistArgs A{};
    A.x = h->xw;
    A.xprev = h->xprev;
    A.q = h->q;
    A.zeros = h->d_zeros;
    A.pitch = h->pitch;
    A.H = h->H;
    A.W = h->W;
    A.consumer_warps = h->p_ncw;
    A.sched = h->d_sched;
    A.cta_off = h->d_cta_off;
    A.sched_bytes = h->p_sched_bytes;
    A.flags = h->d_flags;
    A.barrier = h->d_barrier;
    A.partials = h->d_ppartials;
    A.ctl = h->ctl;
    A.hist = h->hist;
    A.hist_cap = h->hist_cap;
    A.max_cycles = h->max_cycles;
    A.tol = h->tol;
    A.tol_relative = h->tol_relative;
    A.stages = h->p_stages;
    A.stage_floats = h->p_stage_floats;
    A.stage_offset = h->p_stage_offset;
    A.timeout_ns = (h->flags & SMRE_F_SELFTEST_TIMEOUT) ? 50000000ull : h->timeout_ns;
    A.abort_word = h->d_abort;
    A.selftest_timeout = (h->flags & SMRE_F_SELFTEST_TIMEOUT) ? 1 : 0;
    A.selftest_flag = h->d_selftest;
    A.xch = h->d_xch;
    A.smid_tab = h->d_smid;
    // tags of this launch: tag_base + 1 .. tag_base + max_cycles, disjoint
    // from the previous launches' (0 never occurs)
    if ((unsigned long long)h->tag_next + (unsigned)h->max_cycles + 2ull > 0xffffffffull) {
        CK(h, cudaMemsetAsync(h->d_xch, 0, sizeof(unsigned long long) * h->xch_words, h->stream));
        h->tag_next = 1;
    }
    A.tag_base = h->tag_next;
    h->tag_next += (unsigned)h->max_cycles + 1u;
    if (h->p_reg)
        CK(h, launch_persist_reg(A, h->p_grid, h->p_threads, h->p_smem, h->stream));
    else
        CK(h, launch_persist(A, h->p_sp, h->p_grid, h->p_threads, h->p_smem, h->stream));
    h->launches += 1;
    return SMRE_OK;
}


smre_status project_core(smre_dykstra *h, const float *x0, float *x, smre_result *res)
{
    if (!x0 || !x) return fail(h, SMRE_EINVAL, "x0 / x is NULL");
    smre_status st = stage_in(h, x0);
    if (st != SMRE_OK) return st;
    CK(h, cudaMemcpy2DAsync(h->xprev, sizeof(float) * h->pitch, h->xw, sizeof(float) * h->pitch,
                            sizeof(float) * h->W, h->H, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemsetAsync(h->ctl, 0, sizeof(Control), h->stream));
    CK(h, cudaEventRecord(h->ev0, h->stream));

    int cycles = 0;
    if (h->bat) {
        const long long l0 = smre_batch_kernel_launches(h->bat);
        Control c{};
        st = batch_run_one(h->bat, h->H, h->W, h->xw, h->xw, h->pitch, h->hist, h->hist_cap, &c);
        if (st != SMRE_OK) return fail(h, st, "%s", smre_batch_last_error(h->bat));
        h->launches += smre_batch_kernel_launches(h->bat) - l0;
        *h->ctl_host = c;
        cycles = c.cycles;
    } else if (h->persist) {
        st = run_persistent(h);
        if (st != SMRE_OK) return st;
        CK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        cycles = h->ctl_host->cycles;
    }
    for (int cyc = 0; !h->persist && !h->bat && cyc < h->max_cycles; ++cyc) {
        for (const Group &g : h->groups) {
            GroupArgs A{};
            A.x = h->xw;
            A.q = h->q;
            for (int b = 0; b < g.L; ++b) A.q_off[b] = h->tilings[g.tiling0 + b].q_off;
            A.pitch = h->pitch;
            A.H = h->H;
            A.W = h->W;
            A.L = g.L;
            A.a = g.a;
            A.n_units = g.n_units;
            A.cS = (float)h->cS_of[g.L];
            A.sqrt_cS = (float)std::sqrt(h->cS_of[g.L]);
            A.cS64 = h->cS_of[g.L];
            A.first = cyc == 0;
            CK(h, launch_group(A, h->stream));
            h->launches += g.n_units > 0;
        }
        CK(h, launch_cycle_norm(h->xw, h->xprev, h->H, h->W, h->pitch, h->partials,
                                h->n_partials, h->stream));
        CK(h, launch_decide(h->partials, h->n_partials, h->ctl, h->hist, h->hist_cap, h->tol,
                            h->tol_relative, h->stream));
        h->launches += 2;
        CK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        cycles = cyc + 1;
        if (h->ctl_host->stop) break;
    }
    CK(h, cudaEventRecord(h->ev1, h->stream));
    h->last_cycles = cycles;
    double viol = NAN;
    if (h->flags & SMRE_F_VIOLATION) {
        st = violation(h, viol);
        if (st != SMRE_OK) return st;
    }
    st = stage_out(h, x);
    if (st != SMRE_OK) return st;
    // the device's status (every schedule has its control block on the host by now)
    const int dev_status = h->ctl_host->status;
    if (dev_status == SMRE_EINVAL)
        fail(h, SMRE_EINVAL, "x0 holds a NaN or an infinity (the first cycle's norm is not finite)");
    else if (dev_status == SMRE_ETIMEOUT)
        fail(h, SMRE_ETIMEOUT, "a device-side wait ran out of time; the result is not valid");
    if (res) {
        CK(h, cudaStreamSynchronize(h->stream));
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        res->cycles = h->ctl_host->cycles;
        res->status = dev_status;
        res->step = h->ctl_host->step;
        res->rel_step = h->ctl_host->prev_norm > 0 ? h->ctl_host->step / h->ctl_host->prev_norm : 0.0;
        res->max_violation = viol;
        res->windows = (long long)res->cycles * h->windows_per_cycle;
        res->max_tile_sweeps = 0;
        res->seconds = ms * 1e-3;
        return (smre_status)res->status;
    }
    return (smre_status)dev_status;
}

}  // namespace

namespace smre {
void set_thread_error(const char *msg) { g_err = msg; }

namespace {
thread_local int g_alloc_depth = 0;     // create calls in progress on this thread
thread_local long g_alloc_count = 0;    // allocations made since the outermost began
thread_local long g_alloc_fail = -1;    // index of the allocation that fails (-1: none)

bool alloc_should_fail()
{
    if (g_alloc_depth == 0 || g_alloc_fail < 0) return false;
    return g_alloc_count++ == g_alloc_fail;
}
}  // namespace

AllocScope::AllocScope()
{
    if (g_alloc_depth++ == 0) {
        g_alloc_count = 0;
        const char *e = getenv("SMRE_TEST_FAIL_ALLOC");
        g_alloc_fail = (e && *e) ? atol(e) : -1;
    }
}

AllocScope::~AllocScope() { --g_alloc_depth; }

cudaError_t dev_malloc(void **p, size_t bytes)
{
    if (alloc_should_fail()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t host_malloc(void **p, size_t bytes)
{
    if (alloc_should_fail()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}
}  // namespace smre

extern "C" {

const char *smre_version(void) { return "smre-gb300 0.13 (sm_103a)"; }

const char *smre_last_error(const smre_dykstra *h)
{
    if (h) return h->err.c_str();
    return g_err.c_str();
}

smre_status smre_bounds(const smre_params *p, double *cS_out)
{
    std::vector<int> sides;
    std::vector<double> cexp, cS;
    smre_status st = check_params(p, sides, cexp);
    if (st != SMRE_OK) return st;
    if (!cS_out) return fail(nullptr, SMRE_EINVAL, "cS_out is NULL");
    st = compute_bounds(p, sides, cexp, cS);
    if (st != SMRE_OK) return st;
    for (int i = 0; i < p->n_sides; ++i) {
        const int L = p->sides[i];
        const size_t j = std::lower_bound(sides.begin(), sides.end(), L) - sides.begin();
        cS_out[i] = cS[j];
    }
    return SMRE_OK;
}

smre_status smre_dykstra_create(const smre_params *p, void *cuda_stream, smre_dykstra **out)
{
    const AllocScope scope;
    if (!out) return fail(nullptr, SMRE_EINVAL, "out is NULL");
    *out = nullptr;
    std::vector<int> sides;
    std::vector<double> cexp;
    smre_status st = check_params(p, sides, cexp);
    if (st != SMRE_OK) return st;
    smre_dykstra *h = new (std::nothrow) smre_dykstra();
    if (!h) return fail(nullptr, SMRE_ENOMEM, "host allocation failed");
    h->H = p->height;
    h->W = p->width;
    h->pitch = round_up(p->width, 32);
    h->sides = sides;
    h->cmode = p->cmode;
    h->alpha = p->alpha;
    h->maxstat_draws = p->maxstat_draws ? p->maxstat_draws : 1000;
    h->seed = p->seed;
    h->flags = p->flags;
    h->max_ctas = p->max_ctas;
    h->q_dtype = p->q_dtype;
    h->max_cycles = p->max_cycles;
    h->tol = p->tol;
    h->tol_relative = p->tol_relative ? 1 : 0;
    h->icd_max_sweeps = p->icd_max_sweeps ? p->icd_max_sweeps : 1000;
    h->stream = (cudaStream_t)cuda_stream;

    st = compute_bounds(p, sides, cexp, h->cS);
    if (st != SMRE_OK) {
        delete h;
        return st;
    }
    for (size_t i = 0; i < sides.size(); ++i) h->cS_of[sides[i]] = h->cS[i];
    build_schedule(h);
    const bool tune = (p->flags & SMRE_F_AUTOTUNE) != 0;
    const bool batched = use_batch(p, sides.back());
    const bool batch_fits = p->width <= kBatchMaxWidth && sides.back() <= kBatchMaxSide;
    if (batched && !tune) h->q_floats = 0;   // the batch holds the increments
    if (p->q_dtype != SMRE_Q_FP32) h->q_floats = 0;

    auto bail = [&](smre_status s2) {
        g_err = h->err;
        smre_dykstra_destroy(h);
        return s2;
    };
#define CKC(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            fail(h, e_ == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA, "%s: %s", \
                 #call, cudaGetErrorString(e_));                                          \
            return bail(e_ == cudaErrorMemoryAllocation ? SMRE_ENOMEM : SMRE_ECUDA);     \
        }                                                                                 \
    } while (0)

    const size_t img = sizeof(float) * (size_t)h->H * h->pitch;
    CKC(dev_malloc(&h->q, sizeof(float) * std::max<size_t>(h->q_floats, 1)));
    CKC(dev_malloc(&h->xw, img));
    CKC(dev_malloc(&h->xprev, img));
    CKC(cudaMemset(h->xw, 0, img));
    CKC(cudaMemset(h->xprev, 0, img));
    h->n_partials = norm_blocks();
    CKC(dev_malloc(&h->partials, sizeof(double) * 2 * h->n_partials));
    CKC(dev_malloc(&h->ctl, sizeof(Control)));
    CKC(dev_malloc(&h->viol, sizeof(double)));
    CKC(host_malloc(&h->ctl_host, sizeof(Control)));
    CKC(host_malloc(&h->viol_host, sizeof(double)));
    CKC(cudaEventCreate(&h->ev0));
    CKC(cudaEventCreate(&h->ev1));
    h->dev_bytes = sizeof(float) * std::max<size_t>(h->q_floats, 1) + 2 * img +
                   sizeof(double) * 2 * h->n_partials + sizeof(Control) + sizeof(double);
    if (ensure_hist(h, h->max_cycles) != SMRE_OK) return bail(SMRE_ENOMEM);
    if (tune) {
        // every schedule that can run the shape, then time them
        if (p->q_dtype == SMRE_Q_FP32) {
            st = plan_persistent(h, p->flags);
            if (st != SMRE_OK) return bail(st);
        }
        if (batch_fits) {
            st = make_handle_batch(h);
            if (st != SMRE_OK) return bail(st);
        }
        st = autotune(h);
        if (st != SMRE_OK) return bail(st);
    } else if (batched) {
        st = make_handle_batch(h);
        if (st != SMRE_OK) return bail(st);
    } else {
        st = plan_persistent(h, p->flags);
        if (st != SMRE_OK) return bail(st);
    }
#undef CKC
    *out = h;
    return SMRE_OK;
}

smre_status smre_dykstra_set_stopping(smre_dykstra *h, int max_cycles, double tol, int tol_relative)
{
    if (!h) return fail(nullptr, SMRE_EINVAL, "handle is NULL");
    if (max_cycles < 1) return fail(h, SMRE_EINVAL, "max_cycles must be >= 1");
    if (std::isnan(tol)) return fail(h, SMRE_EINVAL, "tol is NaN");
    smre_status st = ensure_hist(h, max_cycles);
    if (st != SMRE_OK) return st;
    h->max_cycles = max_cycles;
    h->tol = tol;
    h->tol_relative = tol_relative ? 1 : 0;
    if (h->bat && batch_set_rule(h->bat, max_cycles, tol, tol_relative) != SMRE_OK)
        return make_handle_batch(h);   // more cycles than its history holds: a new batch
    return SMRE_OK;
}

smre_status smre_dykstra_project(smre_dykstra *h, const float *x0, float *x, smre_result *res)
{
    if (!h) return fail(nullptr, SMRE_EINVAL, "handle is NULL");
    return project_core(h, x0, x, res);
}

int smre_dykstra_schedule(const smre_dykstra *h) { return h ? current_schedule(h) : 0; }

smre_status smre_dykstra_project_incomplete(smre_dykstra *h, const float *x0, float *x, int K,
                                            double tol, smre_result *res)
{
    if (!h) return fail(nullptr, SMRE_EINVAL, "handle is NULL");
    if (!x0 || !x) return fail(h, SMRE_EINVAL, "x0 / x is NULL");
    if (K < 0) K = (int)std::floor(std::log2((double)h->sides.back()) + 1e-12);
    if (K > kMaxIcdK) return fail(h, SMRE_EINVAL, "K = %d above the supported %d", K, kMaxIcdK);
    const int B = 1 << K;
    if (B > h->H || B > h->W) return fail(h, SMRE_EINVAL, "tile side %d larger than the image", B);
    if (std::isnan(tol)) return fail(h, SMRE_EINVAL, "tol is NaN");
    float cS[kMaxIcdK + 1];
    double cS64[kMaxIcdK + 1];
    for (int k = 0; k <= K; ++k) {
        const int L = 1 << k;
        double c = 0.0;
        if (L <= kMaxSide && h->cS_of[L] > 0.0) c = h->cS_of[L];
        else if (h->cmode == SMRE_C_PERSET) c = bound_from_q(inv_normal_cdf(h->alpha), L);
        else if (h->cmode == SMRE_C_CHI2) c = chi2_quantile(h->alpha, L * L);
        else
            return fail(h, SMRE_EINVAL, "no bound for side %d: add it to the sides", L);
        cS[k] = (float)c;
        cS64[k] = c;
    }
    // tile counts of every pass
    std::vector<int> ni(K + 1), nj(K + 1), offs(K + 1);
    int total = 0;
    for (int i = 0; i <= K; ++i) {
        offs[i] = (1 << i) % B;
        ni[i] = h->H - offs[i] >= B ? (h->H - offs[i]) / B : 0;
        nj[i] = h->W - offs[i] >= B ? (h->W - offs[i]) / B : 0;
        total += ni[i] * nj[i];
    }
    if (total > h->icd_sweeps_cap) {
        if (h->icd_sweeps) {
            CK(h, cudaStreamSynchronize(h->stream));
            cudaFree(h->icd_sweeps);
            h->dev_bytes -= sizeof(int) * h->icd_sweeps_cap;
            h->icd_sweeps = nullptr;
        }
        CK(h, dev_malloc(&h->icd_sweeps, sizeof(int) * std::max(total, 1)));
        h->icd_sweeps_cap = std::max(total, 1);
        h->dev_bytes += sizeof(int) * h->icd_sweeps_cap;
    }
    smre_status st = stage_in(h, x0);
    if (st != SMRE_OK) return st;
    CK(h, cudaEventRecord(h->ev0, h->stream));
    int o = 0;
    for (int i = 0; i <= K; ++i) {
        IcdArgs A{};
        A.x = h->xw;
        A.pitch = h->pitch;
        A.H = h->H;
        A.W = h->W;
        A.K = K;
        A.pass = i;
        A.off = offs[i];
        A.n_ti = ni[i];
        A.n_tj = nj[i];
        A.tol_b2 = (float)(tol * (double)B * (double)B);
        A.max_sweeps = h->icd_max_sweeps;
        for (int k = 0; k <= K; ++k) {
            A.cS[k] = cS[k];
            A.sqrt_cS[k] = (float)std::sqrt(cS64[k]);
            A.cS64[k] = cS64[k];
        }
        A.sweeps = h->icd_sweeps + o;
        CK(h, launch_icd_pass(A, h->stream));
        h->launches += ni[i] * nj[i] > 0;
        o += ni[i] * nj[i];
    }
    CK(h, cudaEventRecord(h->ev1, h->stream));
    h->last_icd_tiles = total;
    double viol = NAN;
    if (h->flags & SMRE_F_VIOLATION) {
        st = violation(h, viol);
        if (st != SMRE_OK) return st;
    }
    st = stage_out(h, x);
    if (st != SMRE_OK) return st;
    if (res) {
        std::vector<int> sw(std::max(total, 1));
        CK(h, cudaMemcpyAsync(sw.data(), h->icd_sweeps, sizeof(int) * total,
                              cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        long long windows = 0, sweeps = 0;
        int mx = 0;
        o = 0;
        for (int i = 0; i <= K; ++i) {
            long long per_sweep = 0;
            for (int k = i; k <= K; ++k) per_sweep += (long long)(B >> k) * (B >> k);
            for (int t = 0; t < ni[i] * nj[i]; ++t) {
                windows += per_sweep * sw[o + t];
                sweeps += sw[o + t];
                mx = std::max(mx, sw[o + t]);
            }
            o += ni[i] * nj[i];
        }
        res->cycles = (int)std::min<long long>(sweeps, 2147483647LL);
        res->status = SMRE_OK;
        res->step = NAN;
        res->rel_step = NAN;
        res->max_violation = viol;
        res->windows = windows;
        res->max_tile_sweeps = mx;
        res->seconds = ms * 1e-3;
    }
    return SMRE_OK;
}

smre_status smre_dykstra_bounds(const smre_dykstra *h, int *sides_out, double *cS_out, int n)
{
    if (!h) return fail(nullptr, SMRE_EINVAL, "handle is NULL");
    if (n < (int)h->sides.size() || !sides_out || !cS_out)
        return fail(const_cast<smre_dykstra *>(h), SMRE_EINVAL, "need room for %zu sides",
                    h->sides.size());
    for (size_t i = 0; i < h->sides.size(); ++i) {
        sides_out[i] = h->sides[i];
        cS_out[i] = h->cS[i];
    }
    return SMRE_OK;
}

smre_status smre_dykstra_history(smre_dykstra *h, double *out, int n_max, int *n_cycles)
{
    if (!h) return fail(nullptr, SMRE_EINVAL, "handle is NULL");
    CK(h, cudaStreamSynchronize(h->stream));
    const int n = std::min(h->last_cycles, h->hist_cap);
    if (n_cycles) *n_cycles = n;
    const int m = std::min(n, std::max(n_max, 0));
    if (m > 0 && out)
        CK(h, cudaMemcpy(out, h->hist, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost));
    return SMRE_OK;
}

smre_status smre_dykstra_icd_sweeps(smre_dykstra *h, int *out, int n_max, int *n_tiles)
{
    if (!h) return fail(nullptr, SMRE_EINVAL, "handle is NULL");
    CK(h, cudaStreamSynchronize(h->stream));
    if (n_tiles) *n_tiles = h->last_icd_tiles;
    const int m = std::min(h->last_icd_tiles, std::max(n_max, 0));
    if (m > 0 && out)
        CK(h, cudaMemcpy(out, h->icd_sweeps, sizeof(int) * m, cudaMemcpyDeviceToHost));
    return SMRE_OK;
}

size_t smre_dykstra_device_bytes(const smre_dykstra *h)
{
    return h ? h->dev_bytes + smre_batch_device_bytes(h->bat) : 0;
}

long long smre_dykstra_kernel_launches(const smre_dykstra *h) { return h ? h->launches : 0; }

void smre_dykstra_destroy(smre_dykstra *h)
{
    if (!h) return;
    if (h->stream || h->q) cudaStreamSynchronize(h->stream);
    smre_batch_destroy(h->bat);
    cudaFree(h->q);
    cudaFree(h->xw);
    cudaFree(h->xprev);
    cudaFree(h->partials);
    cudaFree(h->hist);
    cudaFree(h->ctl);
    cudaFree(h->icd_sweeps);
    cudaFree(h->viol);
    cudaFree(h->d_sched);
    cudaFree(h->d_cta_off);
    cudaFree(h->d_flags);
    cudaFree(h->d_barrier);
    cudaFree(h->d_selftest);
    cudaFree(h->d_abort);
    cudaFree(h->d_ppartials);
    cudaFree(h->d_zeros);
    cudaFree(h->d_xch);
    cudaFree(h->d_smid);
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
    if (h->viol_host) cudaFreeHost(h->viol_host);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

}  // extern "C"
