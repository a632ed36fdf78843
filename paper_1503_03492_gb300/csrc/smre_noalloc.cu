// Standard projection for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc while they run: a real-time
// acquisition pipeline that reserves all device memory when it starts, or a
// plugin inside a host application whose own memory pool owns the device.
// For them cudaMalloc can fail (the pool already holds the memory) or stall
// (it may synchronise the device) in the middle of their frame budget.
// smre_dykstra_project_static serves them: every buffer the projection needs
// besides the caller's input and output lives in one file-scope device array
// of kStaticScratchBytes.  The runtime creates that array when it loads this
// library's device code on a device -- with its default lazy loading, at the
// first cudaGetSymbolAddress below, i.e. the first call on that device, which
// therefore allocates (and may synchronise): callers make that first call at
// start-up, or set CUDA_MODULE_LOADING=EAGER.  The device then holds the array
// until the process exits.  The entry point runs the same group kernels as the
// handle-based SMRE_F_GROUP_LAUNCHES schedule, so its results are the same.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include "smre_internal.h"

namespace smre {

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

// The scratch every call shares.  In host code this name is only a stand-in:
// its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Device address of the scratch on the current device, looked up once per device.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

smre_status reject(smre_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_thread_error(buf);
    return st;
}

}  // namespace

}  // namespace smre

using namespace smre;

extern "C" smre_status smre_dykstra_project_static(const smre_params *p, void *cuda_stream,
                                                   const float *x0, float *x, smre_result *res)
{
    const auto t_start = std::chrono::steady_clock::now();
    if (!p) return reject(SMRE_EINVAL, "params is NULL");
    if (!x0 || !x) return reject(SMRE_EINVAL, "x0 / x is NULL");
    if (p->height < 1 || p->width < 1 || p->height > 65535 || p->width > kMaxWidth)
        return reject(SMRE_EINVAL, "image %d x %d out of range", p->height, p->width);
    if (!p->sides || p->n_sides < 1 || p->n_sides > 64)
        return reject(SMRE_EINVAL, "need 1..64 window sides");
    if (p->max_cycles < 1) return reject(SMRE_EINVAL, "max_cycles must be >= 1");
    if (std::isnan(p->tol)) return reject(SMRE_EINVAL, "tol is NaN");
    if (p->q_dtype != 0) return reject(SMRE_EINVAL, "q_dtype %d not supported", p->q_dtype);
    if (p->cmode == SMRE_C_MAXSTAT)
        return reject(SMRE_EINVAL, "MAXSTAT bounds need device allocations; pass EXPLICIT bounds");
    if (p->cmode != SMRE_C_PERSET && p->cmode != SMRE_C_CHI2 && p->cmode != SMRE_C_EXPLICIT)
        return reject(SMRE_EINVAL, "unknown cmode %d", (int)p->cmode);
    if (p->cmode != SMRE_C_EXPLICIT && !(p->alpha > 0.0 && p->alpha < 1.0))
        return reject(SMRE_EINVAL, "alpha %g outside (0, 1)", p->alpha);
    const int H = p->height, W = p->width;

    // bounds of the distinct sides (Sec. 2.1), sides descending (the set order)
    double cS_of[kMaxSide + 1] = {};
    std::vector<int> sides;
    for (int i = 0; i < p->n_sides; ++i) {
        const int L = p->sides[i];
        if (L < 1 || L > kMaxSide || L > H || L > W)
            return reject(SMRE_EINVAL, "window side %d outside 1..min(%d, H, W)", L, kMaxSide);
        double c;
        if (p->cmode == SMRE_C_EXPLICIT) {
            if (!p->c_explicit) return reject(SMRE_EINVAL, "c_explicit is NULL");
            c = p->c_explicit[i];
            if (!(c > 0.0) || !std::isfinite(c))
                return reject(SMRE_EINVAL, "bound %g of side %d is not a positive number", c, L);
        } else if (p->cmode == SMRE_C_CHI2) {
            c = chi2_quantile(p->alpha, L * L);
        } else {
            c = bound_from_q(inv_normal_cdf(p->alpha), L);
        }
        if (std::find(sides.begin(), sides.end(), L) == sides.end()) {
            sides.push_back(L);
            cS_of[L] = c;
        } else if (c != cS_of[L]) {
            // a repeated side is ignored only when it repeats the bound too
            return reject(SMRE_EINVAL, "side %d listed twice with different bounds (%g, %g)", L,
                          cS_of[L], c);
        }
    }
    std::sort(sides.rbegin(), sides.rend());

    // layout of the scratch: increments of every tiling, two work images,
    // norm partials, the control block and the per-cycle history
    const int pitch = (W + 31) / 32 * 32;
    size_t q_floats = 0;
    for (int L : sides)
        for (int a = 0; a < L; ++a) q_floats += (size_t)L * ((H - a) / L) * L * pitch;
    const int nb = norm_blocks();
    const size_t img = sizeof(float) * (size_t)H * pitch;
    const size_t off_x = align256(sizeof(float) * q_floats);
    const size_t off_xp = off_x + align256(img);
    const size_t off_part = off_xp + align256(img);
    const size_t off_ctl = off_part + align256(sizeof(double) * 2 * nb);
    const size_t off_hist = off_ctl + align256(sizeof(Control));
    const size_t need = off_hist + align256(sizeof(double) * 2 * (size_t)p->max_cycles);
    if (need > kStaticScratchBytes)
        return reject(SMRE_EINVAL,
                      "this projection needs %zu bytes of scratch; the static buffer holds %zu "
                      "(use smre_dykstra_create for larger images or more sides)",
                      need, kStaticScratchBytes);

    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess)
        return reject(SMRE_ECUDA, "cudaGetSymbolAddress of the static scratch: %s",
                      cudaGetErrorString(e));
    unsigned char *s = static_cast<unsigned char *>(base);
    float *q = reinterpret_cast<float *>(s);
    float *xw = reinterpret_cast<float *>(s + off_x);
    float *xp = reinterpret_cast<float *>(s + off_xp);
    double *part = reinterpret_cast<double *>(s + off_part);
    Control *ctl = reinterpret_cast<Control *>(s + off_ctl);
    double *hist = reinterpret_cast<double *>(s + off_hist);
    cudaStream_t st = (cudaStream_t)cuda_stream;

#define CKS(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return reject(SMRE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

    // x <- x0, x_prev <- x0, fresh control block; the increments need no
    // clearing: the first cycle treats them as zero and writes all of them
    CKS(cudaMemcpy2DAsync(xw, sizeof(float) * pitch, x0, sizeof(float) * W, sizeof(float) * W, H,
                          cudaMemcpyDefault, st));
    CKS(cudaMemcpy2DAsync(xp, sizeof(float) * pitch, xw, sizeof(float) * pitch,
                          sizeof(float) * W, H, cudaMemcpyDeviceToDevice, st));
    CKS(cudaMemsetAsync(ctl, 0, sizeof(Control), st));

    Control ch{};
    long long windows_per_cycle = 0;
    for (int L : sides) windows_per_cycle += (long long)(H - L + 1) * (W - L + 1);
    for (int cyc = 0; cyc < p->max_cycles; ++cyc) {
        size_t off = 0;
        for (int L : sides)
            for (int a = 0; a < L; ++a) {
                GroupArgs A{};
                A.x = xw;
                A.q = q;
                const int nu = (H - a) / L;
                for (int b = 0; b < L; ++b) {
                    A.q_off[b] = (long long)off;
                    off += (size_t)nu * L * pitch;
                }
                A.pitch = pitch;
                A.H = H;
                A.W = W;
                A.L = L;
                A.a = a;
                A.n_units = nu;
                A.cS = (float)cS_of[L];
                A.sqrt_cS = (float)std::sqrt(cS_of[L]);
                A.cS64 = cS_of[L];
                A.first = cyc == 0;
                CKS(launch_group(A, st));
            }
        CKS(launch_cycle_norm(xw, xp, H, W, pitch, part, nb, st));
        CKS(launch_decide(part, nb, ctl, hist, p->max_cycles, p->tol, p->tol_relative, st));
        CKS(cudaMemcpyAsync(&ch, ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
        CKS(cudaStreamSynchronize(st));
        if (ch.stop) break;
    }
    CKS(cudaMemcpy2DAsync(x, sizeof(float) * W, xw, sizeof(float) * pitch, sizeof(float) * W, H,
                          cudaMemcpyDefault, st));
    CKS(cudaStreamSynchronize(st));
#undef CKS
    if (res) {
        res->cycles = ch.cycles;
        res->status = ch.status;
        res->step = ch.step;
        res->rel_step = ch.prev_norm > 0 ? ch.step / ch.prev_norm : 0.0;
        res->max_violation = NAN;
        res->windows = (long long)ch.cycles * windows_per_cycle;
        res->max_tile_sweeps = 0;
        res->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
    return (smre_status)ch.status;
}
