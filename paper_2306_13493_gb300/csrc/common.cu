// Library-wide helpers: error text, stream-ordered allocation, twiddle tables,
// status strings.
#include <cmath>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <utility>

#include "sce_internal.cuh"

static thread_local char g_last_error[512];

void sce_set_last_cuda_error(cudaError_t err, const char *what, const char *file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", what,
             cudaGetErrorString(err), file, line);
    if (getenv("SCE_VERBOSE")) fprintf(stderr, "[sce] %s\n", g_last_error);
}

extern "C" const char *sce_last_error(void) { return g_last_error; }

void sce_set_last_error_text(const char *text) {
    snprintf(g_last_error, sizeof(g_last_error), "%s", text);
    if (getenv("SCE_VERBOSE")) fprintf(stderr, "[sce] %s\n", g_last_error);
}

static std::mutex g_pool_mu;
static bool g_pool_configured[64];

// Test hook: the next g_fail_allocs stream-ordered allocations fail with
// CE_ERR_OOM before reaching the allocator (sce_test_fail_allocs).
static std::atomic<int> g_fail_allocs{0};

extern "C" void sce_test_fail_allocs(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

int sce_alloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) return CE_OK;
    for (int left = g_fail_allocs.load(); left > 0;) {
        if (g_fail_allocs.compare_exchange_weak(left, left - 1)) {
            sce_set_last_error_text("allocation refused by sce_test_fail_allocs");
            return CE_ERR_OOM;
        }
    }
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (dev >= 0 && dev < 64 && !g_pool_configured[dev]) {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = UINT64_MAX;   // keep freed blocks cached in the pool
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
            g_pool_configured[dev] = true;
        }
    }
    SCE_CUDA(cudaMallocAsync(p, bytes, st));
    return CE_OK;
}

int sce_free(void *p, cudaStream_t st) {
    if (p) SCE_CUDA(cudaFreeAsync(p, st));
    return CE_OK;
}

// exp(+2 pi i k / P) for k = 0..P-1, evaluated in FP64 on the host from the
// octant-reduced angle (cos and sin of pi k'/ (P/2) with k' <= P/8 and the
// symmetries of the circle), so every entry is within an ulp or two.
static void host_twiddles(int P, std::vector<double> &re, std::vector<double> &im) {
    re.resize(P);
    im.resize(P);
    const double two_pi_over_P = 2.0 * M_PI / P;
    for (int k = 0; k < P; ++k) {
        // angle = 2 pi k / P = oct * pi/4 + 2 pi kr / P with kr in [0, P/8)
        const int oct = (int)((8LL * k) / P);
        const int kr = k - (int)((long long)oct * P / 8);
        double c, s;
        if (P % 8 == 0) {
            double a;
            if (oct & 1) a = two_pi_over_P * (double)(P / 8 - kr);   // mirrored
            else a = two_pi_over_P * (double)kr;
            double ca = std::cos(a), sa = std::sin(a);
            // angle = oct*pi/4 + kr*2pi/P; express via symmetry
            switch (oct) {
                case 0: c = ca; s = sa; break;           // [0, pi/4)
                case 1: c = sa; s = ca; break;           // [pi/4, pi/2): pi/2 - a
                case 2: c = -sa; s = ca; break;          // pi/2 + a
                case 3: c = -ca; s = sa; break;          // pi - a
                case 4: c = -ca; s = -sa; break;         // pi + a
                case 5: c = -sa; s = -ca; break;         // 3pi/2 - a
                case 6: c = sa; s = -ca; break;          // 3pi/2 + a
                default: c = ca; s = -sa; break;         // 2pi - a
            }
        } else {
            c = std::cos(two_pi_over_P * k);
            s = std::sin(two_pi_over_P * k);
        }
        re[k] = c;
        im[k] = s;
    }
}

struct TwKey {
    int dev, P;
    bool operator<(const TwKey &o) const { return dev != o.dev ? dev < o.dev : P < o.P; }
};
static std::mutex g_smem_mu;
static std::map<std::pair<int, const void *>, size_t> g_smem_limit;

int sce_raise_smem_limit(const void *func, size_t bytes) {
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_smem_mu);
    size_t &cur = g_smem_limit[{dev, func}];
    if (bytes <= cur) return CE_OK;
    SCE_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return CE_OK;
}

static std::mutex g_tw_mu;
static std::map<TwKey, std::pair<double2 *, float2 *>> g_tw;

static int twiddles(int P, double2 **d64, float2 **d32) {
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto it = g_tw.find({dev, P});
    if (it != g_tw.end()) {
        *d64 = it->second.first;
        *d32 = it->second.second;
        return CE_OK;
    }
    std::vector<double> re, im;
    host_twiddles(P, re, im);
    std::vector<double2> h64(P);
    std::vector<float2> h32(P);
    for (int k = 0; k < P; ++k) {
        h64[k] = make_double2(re[k], im[k]);
        h32[k] = make_float2((float)re[k], (float)im[k]);
    }
    double2 *a = nullptr;
    float2 *b = nullptr;
    SCE_CUDA(cudaMalloc(&a, P * sizeof(double2)));
    SCE_CUDA(cudaMalloc(&b, P * sizeof(float2)));
    SCE_CUDA(cudaMemcpy(a, h64.data(), P * sizeof(double2), cudaMemcpyHostToDevice));
    SCE_CUDA(cudaMemcpy(b, h32.data(), P * sizeof(float2), cudaMemcpyHostToDevice));
    g_tw[{dev, P}] = {a, b};
    *d64 = a;
    *d32 = b;
    return CE_OK;
}

// Lookup only: the tables of P on the current device if they were built
// (every embedding set-up builds its P's tables); never allocates.
int sce_twiddles_lookup(int P, const double2 **d64, const float2 **d32) {
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto it = g_tw.find({dev, P});
    if (it == g_tw.end()) return CE_ERR_INVALID_ARG;
    *d64 = it->second.first;
    *d32 = it->second.second;
    return CE_OK;
}

const double2 *sce_twiddles64(int P, int *status) {
    double2 *a = nullptr;
    float2 *b = nullptr;
    *status = twiddles(P, &a, &b);
    return a;
}

const float2 *sce_twiddles32(int P, int *status) {
    double2 *a = nullptr;
    float2 *b = nullptr;
    *status = twiddles(P, &a, &b);
    return b;
}

extern "C" const char *ce_status_string(int status) {
    switch (status) {
        case CE_OK: return "ok";
        case CE_ERR_INVALID_ARG: return "invalid argument";
        case CE_ERR_NOT_PSD: return "embedding not positive semi-definite";
        case CE_ERR_OOM: return "out of memory";
        case CE_ERR_CUDA: return "CUDA runtime error";
        case CE_ERR_NOT_CONVERGED: return "solver did not converge";
        case CE_ERR_TIMEOUT: return "device wait timed out";
        case CE_ERR_NONFINITE: return "non-finite value";
        default: return "unknown status";
    }
}

extern "C" int mlmc_optimal_samples(int L_plus_1, const double *V, const double *C, double eps,
                                    long long *N) {
    if (L_plus_1 <= 0 || !V || !C || !N || !(eps > 0)) return CE_ERR_INVALID_ARG;
    double total = 0.0;
    for (int l = 0; l < L_plus_1; ++l) {
        if (!(C[l] > 0) || !(V[l] >= 0)) return CE_ERR_INVALID_ARG;
        total += std::sqrt(C[l] * V[l]);
    }
    for (int l = 0; l < L_plus_1; ++l)
        N[l] = (long long)std::ceil(2.0 / (eps * eps) * total * std::sqrt(V[l] / C[l]));
    return CE_OK;
}

// §3.6, separable exponential covariance without padding (s = 4 h^-2): the
// smoothing term C_s tau / (s - tau + 1) of the error bound equals the
// discretisation term C_alpha h^alpha.  With h = 2 s^-1/2 that is
// tau / (s - tau + 1) = r, r = 2^alpha s^(-alpha/2) / (C_s / C_alpha), solved
// for tau directly.
extern "C" int mlmc_tau_exponential(double s, double alpha, double cs_over_calpha, double *tau) {
    if (!tau || !(s >= 1.0) || !(alpha > 0.0) || !(cs_over_calpha > 0.0) || !std::isfinite(s))
        return CE_ERR_INVALID_ARG;
    const double r = std::exp(alpha * (std::log(2.0) - 0.5 * std::log(s))) / cs_over_calpha;
    *tau = r * (s + 1.0) / (1.0 + r);
    return CE_OK;
}

// §3.6, Matern covariance under smooth periodisation (s = 4 (1/h + J)^2): the
// tau in [1, s] at which C_s s^-1/2 h^-1 (s - tau + 1)^-(1+nu)/2 tau equals
// C_alpha h^alpha.  In logarithms the condition is g(t) = 0 with
//   g(t) = ln t - (1+nu)/2 ln(s - t + 1) - ln(2 h^(alpha+1) (1/h + J) C_alpha / C_s),
// strictly increasing on [1, s]; Newton's method on g, a step that leaves the
// current bracket replaced by the bracket's midpoint.  A root below 1 or above
// s gives 1 or s.
extern "C" int mlmc_tau_matern(double h, double J, double nu, double alpha, double cs_over_calpha,
                               double *tau) {
    if (!tau || !(h > 0.0) || !(J >= 0.0) || !(nu > 0.0) || !(alpha > 0.0) ||
        !(cs_over_calpha > 0.0) || !std::isfinite(h) || !std::isfinite(J))
        return CE_ERR_INVALID_ARG;
    const double q = 1.0 / h + J, s = 4.0 * q * q, e = 0.5 * (1.0 + nu);
    const double lr = std::log(2.0 / cs_over_calpha) + (alpha + 1.0) * std::log(h) + std::log(q);
    auto g = [&](double t) { return std::log(t) - e * std::log(s - t + 1.0) - lr; };
    double lo = 1.0, hi = s;
    if (g(lo) >= 0.0) { *tau = lo; return CE_OK; }
    if (g(hi) <= 0.0) { *tau = hi; return CE_OK; }
    // first guess for tau << s: ln t = lr + e ln s
    double t = std::exp(lr + e * std::log(s));
    if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        const double gt = g(t);
        if (gt == 0.0) break;
        if (gt > 0.0) hi = t; else lo = t;
        double tn = t - gt / (1.0 / t + e / (s - t + 1.0));
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        const bool done = std::fabs(tn - t) <= 1e-15 * t || hi - lo <= 1e-15 * hi;
        t = tn;
        if (done) break;
    }
    *tau = t;
    return CE_OK;
}

bool sce_smem_pad() {
    const char *e = getenv("SCE_SMEM_PAD");
    return !(e && atoi(e) == 0);
}

bool sce_small_pad() {
    const char *e = getenv("SCE_SMALL_PAD");
    return e && atoi(e) == 1;
}

double sce_inner_rel_f32() {
    const char *e = getenv("SCE_INNER_REL");
    const double v = e ? atof(e) : 0.0;
    return (v >= 1e-8 && v <= 1e-2) ? v : 2e-5;
}
