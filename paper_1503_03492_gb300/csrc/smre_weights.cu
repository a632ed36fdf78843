// Bounds cS = 1 / c_s(alpha) of Sec. 2.1, computed on the host in FP64, plus
// the device Monte Carlo of the extreme-value statistic Q_Omega used by the
// MAXSTAT mode.
//
// With |s| = L^2 pixels, t_s^(1/4) ~ N(mu_s, sigma_s^2), mu_s = (|s| - 1/2)^(1/4),
// sigma_s^2 = 1 / (8 sqrt|s|), and c_s(alpha) = 1 / (q sigma_s + mu_s)^4, so
// the ball radius squared is cS = (q sigma_s + mu_s)^4.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "smre_internal.h"

namespace smre {

// ------------------------------------------------------------------ host math

// Inverse standard normal CDF: the rational approximation of P. J. Acklam
// (2003) as a start, then Newton steps on Phi(x) - p using erfc, which bring
// it to double precision.
double inv_normal_cdf(double p)
{
    if (!(p > 0.0 && p < 1.0)) return NAN;
    static const double a[6] = {-3.969683028665376e+01, 2.209460984245205e+02,
                                -2.759285104469687e+02, 1.383577518672690e+02,
                                -3.066479806614716e+01, 2.506628277459239e+00};
    static const double b[5] = {-5.447609879822406e+01, 1.615858368580409e+02,
                                -1.556989798598866e+02, 6.680131188771972e+01,
                                -1.328068155288572e+01};
    static const double c[6] = {-7.784894002430293e-03, -3.223964580411365e-01,
                                -2.400758277161838e+00, -2.549732539343734e+00,
                                4.374664141464968e+00, 2.938163982698783e+00};
    static const double d[4] = {7.784695709041462e-03, 3.224671290700398e-01,
                                2.445134137142996e+00, 3.754408661907416e+00};
    const double plow = 0.02425;
    double x;
    if (p < plow) {
        double q = std::sqrt(-2.0 * std::log(p));
        x = (((((c[0] * q + c[1]) * q + c[2]) * q + c[3]) * q + c[4]) * q + c[5]) /
            ((((d[0] * q + d[1]) * q + d[2]) * q + d[3]) * q + 1.0);
    } else if (p > 1.0 - plow) {
        double q = std::sqrt(-2.0 * std::log1p(-p));
        x = -(((((c[0] * q + c[1]) * q + c[2]) * q + c[3]) * q + c[4]) * q + c[5]) /
            ((((d[0] * q + d[1]) * q + d[2]) * q + d[3]) * q + 1.0);
    } else {
        double q = p - 0.5, r = q * q;
        x = (((((a[0] * r + a[1]) * r + a[2]) * r + a[3]) * r + a[4]) * r + a[5]) * q /
            (((((b[0] * r + b[1]) * r + b[2]) * r + b[3]) * r + b[4]) * r + 1.0);
    }
    const double inv_sqrt_2pi = 0.39894228040143267794;
    for (int it = 0; it < 4; ++it) {
        const double f = 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
        const double dens = inv_sqrt_2pi * std::exp(-0.5 * x * x);
        if (dens <= 0.0) break;
        x -= f / dens;
    }
    return x;
}

// Regularized lower incomplete gamma P(a, x): power series below a + 1,
// Legendre continued fraction of the upper part (modified Lentz) above.
static double reg_lower_gamma(double a, double x)
{
    if (x <= 0.0) return 0.0;
    const double lead = std::exp(-x + a * std::log(x) - std::lgamma(a));
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term;
        for (int n = 1; n < 10000; ++n) {
            term *= x / (a + n);
            sum += term;
            if (std::fabs(term) < std::fabs(sum) * 1e-17) break;
        }
        return sum * lead;
    }
    const double tiny = 1e-300;
    double bb = x + 1.0 - a, cc = 1.0 / tiny, dd = 1.0 / bb, h = dd;
    for (int i = 1; i < 10000; ++i) {
        const double an = -i * (i - a);
        bb += 2.0;
        dd = an * dd + bb;
        if (std::fabs(dd) < tiny) dd = tiny;
        cc = bb + an / cc;
        if (std::fabs(cc) < tiny) cc = tiny;
        dd = 1.0 / dd;
        const double del = dd * cc;
        h *= del;
        if (std::fabs(del - 1.0) < 1e-16) break;
    }
    return 1.0 - lead * h;
}

// alpha-quantile of chi^2 with k degrees of freedom: CDF(x) = P(k/2, x/2),
// inverted by bisection on a bracket that always holds the root.
double chi2_quantile(double alpha, int k)
{
    double lo = 0.0, hi = 1.0;
    while (reg_lower_gamma(0.5 * k, 0.5 * hi) < alpha) hi *= 2.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (reg_lower_gamma(0.5 * k, 0.5 * mid) < alpha) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

double fourth_root_mu(int n) { return std::pow(n - 0.5, 0.25); }
double fourth_root_sigma(int n) { return 1.0 / std::sqrt(8.0 * std::sqrt((double)n)); }

double bound_from_q(double q, int L)
{
    const int n = L * L;
    const double r = q * fourth_root_sigma(n) + fourth_root_mu(n);
    return r * r * r * r;
}

// ------------------------------------------------- device Monte Carlo (MAXSTAT)

namespace {

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator:
// value(i) = mix(seed + (i + 1) * 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t splitmix_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// N(0,1) number j of stream `seed` (Box-Muller, cosine branch, on the two
// uniforms (top 53 bits + 1) / 2^53 of counters 2j and 2j + 1), in FP32.
__device__ __forceinline__ float normal_at(uint64_t seed, uint64_t j)
{
    const float u1 = (float)(((double)(splitmix_at(seed, 2ull * j) >> 11) + 1.0) *
                             (1.0 / 9007199254740992.0));
    const float u2 = (float)(((double)(splitmix_at(seed, 2ull * j + 1ull) >> 11) + 1.0) *
                             (1.0 / 9007199254740992.0));
    return sqrtf(-2.0f * logf(u1)) * cosf(6.28318530717958647692f * u2);
}

// squared N(0,1) images of draws draw0 .. draw0 + n_draws - 1
__global__ void maxstat_fill_kernel(int H, int W, int pitch, int draw0, int n_draws,
                                    unsigned long long seed, float *img)
{
    const long long hw = (long long)H * W;
    const long long total = hw * n_draws;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long d = idx / hw, p = idx % hw;
        const int r = (int)(p / W), c = (int)(p % W);
        const float v = normal_at(seed, (uint64_t)(draw0 + d) * (uint64_t)hw + (uint64_t)p);
        img[(size_t)d * H * pitch + (size_t)r * pitch + c] = v * v;
    }
}

struct MaxstatSides {
    int n;
    int L[kMaxSide];
    float mu[kMaxSide], inv_sigma[kMaxSide];
};

// order-preserving map of a float onto an unsigned int (for atomicMax)
__device__ __forceinline__ unsigned ord_of(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// one block row of draws: max over windows and sides of (t^(1/4) - mu) / sigma
__global__ void maxstat_window_kernel(int H, int W, int pitch, int n_draws, const float *img,
                                      const MaxstatSides S, unsigned *ordmax)
{
    const int d = blockIdx.y;
    if (d >= n_draws) return;
    const float *im = img + (size_t)d * H * pitch;
    float best = -INFINITY;
    const long long hw = (long long)H * W;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < hw;
         p += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(p / W), c = (int)(p % W);
        for (int si = 0; si < S.n; ++si) {
            const int L = S.L[si];
            if (r + L > H || c + L > W) continue;
            float t = 0.f;
            for (int i = 0; i < L; ++i) {
                const float *row = im + (size_t)(r + i) * pitch + c;
                for (int j = 0; j < L; ++j) t += row[j];
            }
            best = fmaxf(best, (sqrtf(sqrtf(t)) - S.mu[si]) * S.inv_sigma[si]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&ordmax[d], ord_of(best));
}

__global__ void maxstat_decode_kernel(const unsigned *ordmax, int n, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned o = ordmax[i];
    const unsigned u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    out[i] = (double)__uint_as_float(u);
}

}  // namespace

cudaError_t launch_maxstat(int H, int W, int pitch, const int *sides, int n_sides, int draw0,
                           int n_draws, unsigned long long seed, float *img, double *maxima,
                           cudaStream_t s)
{
    MaxstatSides S{};
    S.n = n_sides;
    for (int i = 0; i < n_sides; ++i) {
        const int n = sides[i] * sides[i];
        S.L[i] = sides[i];
        S.mu[i] = (float)fourth_root_mu(n);
        S.inv_sigma[i] = (float)(1.0 / fourth_root_sigma(n));
    }
    unsigned *ordmax = reinterpret_cast<unsigned *>(maxima);  // scratch: first n_draws words
    cudaError_t e = cudaMemsetAsync(ordmax, 0, sizeof(unsigned) * n_draws, s);
    if (e != cudaSuccess) return e;
    maxstat_fill_kernel<<<1024, 256, 0, s>>>(H, W, pitch, draw0, n_draws, seed, img);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid(64, n_draws);
    maxstat_window_kernel<<<grid, 256, 0, s>>>(H, W, pitch, n_draws, img, S, ordmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // decode in place is unsafe (unsigned[] aliases double[]): decode into the
    // upper half of the scratch the caller sized for 2 * n_draws doubles
    maxstat_decode_kernel<<<(n_draws + 255) / 256, 256, 0, s>>>(ordmax, n_draws, maxima + n_draws);
    return cudaGetLastError();
}

}  // namespace smre
