// C ABI of the LinMin library (see include/linmin.h for the contract).
//
// A call of linmin_unmix queues, on the handle's stream:
//   1. library preparation for this sigma (fp64 Gram, scale, hi/lo splits);
//   2. the double-float projection c~ = B~^T y + rho;
//   3. the interior-point kernel with the float32 residual, every pixel,
//      until mu <= mu_stop (the support is then identified);
//   4. the fp64 active-set crossover to the exact minimiser (abundances,
//      uncertainties); pixels it cannot finish go to a retry list;
//   5. retry list only: interior point from the start, float32 residual to
//      mu <= refine_mu then double-float residual to the stop test, and the
//      crossover again;
//   6. the RMS of the fit.
// Host pointers are staged through handle-owned device buffers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "api_internal.h"
#include "ipm.cuh"
#include "kernels.cuh"
#include "linmin.h"

using namespace lm;

struct linmin_ctx {
    long long fail_at = 0, n_alloc = 0;  // allocation-failure injection (LINMIN_FAIL_ALLOC)
    int L = 0, P = 0;                  // P: spectra of the internal problem
    // slo / pos: the caller's P is P - 1 (the last internal spectrum is the
    // zero slack spectrum), results scaled by M (LINMIN_POS_SCALE for pos)
    int user_P = 0;
    bool slack = false;
    float slack_scale = 1.f;
    float *xa = nullptr, *sxa = nullptr;   // internal x, sx (N x P) of slo / pos
    Bucket bucket{};
    linmin_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;

    float *dS = nullptr;               // P x L library
    Prep prep{};                       // per-sigma buffers
    unsigned long long *dcnt = nullptr;// [0] IPM work counter, [1] retry IPM (float32),
                                       // [2] not converged, [3] unverified after retry,
                                       // [4] retry IPM (double-float), [5] retry list length,
                                       // [6] crossover failures of the first pass
    // per-pixel scratch
    long long capN = 0;
    float *c_hi = nullptr, *c_lo = nullptr, *x = nullptr, *lam = nullptr, *nu = nullptr;
    int *it = nullptr;
    long long *retry = nullptr;
    unsigned long long *mask = nullptr;
    int *rexp = nullptr;               // per-pixel exponents of the TMA projection
    CrossoverScratch xw{};
    // host-pointer staging
    long long capIO = 0;
    float *io_cube = nullptr, *io_sigma = nullptr, *io_x = nullptr, *io_sx = nullptr,
          *io_rms = nullptr;
    int *io_it = nullptr;
    // phase events (profile mode)
    // phase events of the last LINMIN_PHASE_RING calls (ring of event sets),
    // so that a caller can read the phase times of several queued calls
    // after one synchronisation
    cudaEvent_t ev[LINMIN_PHASE_RING][LINMIN_NUM_PHASES + 1] = {};
    long long calls = 0;          // profiled calls so far (ring position)
    int launches = 0;            // kernel launches of the last linmin_unmix
    // full noise covariance (linmin_unmix_cov): C^-1 on the device, the
    // T = C^-1 S^T scratch, and the hash of the C^-1 last checked
    double *cov = nullptr, *covT = nullptr;
    unsigned long long cov_hash = 0;
    // tensor-core projection: slices of B~ and column exponents
    __nv_bfloat16 *bsl = nullptr;
    int *fexp = nullptr;
    cudaMemPool_t pool = nullptr; // device memory of this handle (see pool_acquire)
    // host-buffer pipeline: copy stream and its events
    cudaStream_t cstream = nullptr;
    cudaEvent_t pev_in[8] = {}, pev_out[2] = {};
    // side stream of the tensor-core projection's exponent pass (it needs
    // only the cube, so it runs while the library is prepared)
    cudaStream_t xstream = nullptr;
    cudaEvent_t xev[2] = {};
    // linmin_unmix_batch: the call stops after the projection (defer_ipm)
    // and keeps what the rest of it needs; batch descriptors on the device
    bool defer_ipm = false;
    struct {
        long long N = 0;
        const float *cube = nullptr;
        float *x = nullptr, *sx = nullptr, *rms = nullptr;
        int *it = nullptr;
        int launches = 0;
    } pend;
    unsigned char *bdesc = nullptr;
    size_t bdesc_cap = 0;
};

static void mark(linmin_ctx *h, int i)
{
    if (h->opt.profile) cudaEventRecord(h->ev[h->calls % LINMIN_PHASE_RING][i], h->stream);
}

static std::string g_create_error;
static thread_local std::string g_msg;

static linmin_status fail(linmin_ctx *h, linmin_status st, const std::string &m)
{
    if (h) h->err = m; else g_create_error = m;
    return st;
}

static linmin_status cuda_fail(linmin_ctx *h, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? LINMIN_ERR_OOM : LINMIN_ERR_CUDA, m);
}

#define LM_CUDA(h, call, what)                         \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) return cuda_fail(h, _e, what); \
    } while (0)

// true when p is device (or managed) memory of this process
static bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device memory of handles comes from a library-owned stream-ordered pool
// per device whose freed blocks are kept for reuse while any handle lives:
// creating and destroying handles (a serving loop does both) then neither
// calls cudaMalloc/cudaFree nor synchronises the device.  The pool is
// trimmed when the last handle of its device is destroyed.
struct PoolState {
    cudaMemPool_t pool = nullptr;
    long long live = 0;              // handles of this device
};
static std::mutex g_pool_mu;
static std::map<int, PoolState> g_pools;

static cudaError_t pool_acquire(int dev, cudaMemPool_t *out)
{
    std::lock_guard<std::mutex> g(g_pool_mu);
    PoolState &ps = g_pools[dev];
    if (!ps.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&ps.pool, &props);
        if (e != cudaSuccess) { ps.pool = nullptr; return e; }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(ps.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    ++ps.live;
    *out = ps.pool;
    return cudaSuccess;
}

static void pool_release(int dev)
{
    std::lock_guard<std::mutex> g(g_pool_mu);
    PoolState &ps = g_pools[dev];
    if (--ps.live == 0 && ps.pool) cudaMemPoolTrimTo(ps.pool, 0);
}

// Device allocations the handles hold now (all devices); with
// LINMIN_FAIL_ALLOC the error paths are checked against it for leaks.
static std::atomic<long long> g_live_allocs{0};

// Allocation-failure injection, to exercise the error paths on the host
// (no GPU fault): LINMIN_FAIL_ALLOC = N >= 1, read when a handle is
// created, makes that handle's N-th device allocation fail with
// cudaErrorMemoryAllocation without calling CUDA.  Unset or 0: off.
long long lm::injected_alloc_failure()
{
    const char *e = std::getenv("LINMIN_FAIL_ALLOC");
    if (!e) return 0;
    const long long v = std::atoll(e);
    return v > 0 ? v : 0;
}

template <typename T>
static cudaError_t dalloc(linmin_ctx *h, T **p, size_t n)
{
    if (*p) { cudaFreeAsync(*p, h->stream); *p = nullptr; --g_live_allocs; }
    if (n == 0) n = 1;
    if (h->fail_at > 0 && ++h->n_alloc == h->fail_at) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocFromPoolAsync((void **)p, n * sizeof(T), h->pool, h->stream);
    if (e == cudaSuccess) ++g_live_allocs;
    else *p = nullptr;
    return e;
}

// rank [S^T; 1^T] == P in fp64 (modified Gram-Schmidt with one
// re-orthogonalisation pass on the P columns of length L + 1)
static bool full_rank(const std::vector<float> &S, int L, int P)
{
    const int n = L + 1;
    std::vector<double> Q((size_t)P * n);
    int r = 0;
    for (int j = 0; j < P; ++j) {
        std::vector<double> v(n);
        for (int l = 0; l < L; ++l) v[l] = S[(size_t)j * L + l];
        v[L] = 1.0;
        double n0 = 0.0;
        for (double e : v) n0 += e * e;
        n0 = std::sqrt(n0);
        if (n0 == 0.0) return false;
        for (int pass = 0; pass < 2; ++pass)
            for (int q = 0; q < r; ++q) {
                double d = 0.0;
                for (int l = 0; l < n; ++l) d += Q[(size_t)q * n + l] * v[l];
                for (int l = 0; l < n; ++l) v[l] -= d * Q[(size_t)q * n + l];
            }
        double nv = 0.0;
        for (double e : v) nv += e * e;
        nv = std::sqrt(nv);
        // a float32 library carries its dependencies only to float32
        // rounding (~1e-7 of a column): below 1e-6 a column is dependent
        if (nv <= 1e-6 * n0) return false;
        for (int l = 0; l < n; ++l) Q[(size_t)r * n + l] = v[l] / nv;
        ++r;
    }
    return true;
}

namespace lm {

linmin_status load_library(const float *library, int L, int P, std::vector<float> *host,
                           std::string *why)
{
    host->assign((size_t)P * L, 0.f);
    const bool on_dev = is_device_ptr(library);
    if (on_dev) {
        cudaError_t e = cudaMemcpy(host->data(), library, host->size() * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            *why = std::string("copy library: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? LINMIN_ERR_OOM : LINMIN_ERR_CUDA;
        }
    } else {
        std::memcpy(host->data(), library, host->size() * 4);
    }
    for (float v : *host)
        if (!std::isfinite(v)) { *why = "library has NaN/Inf"; return LINMIN_ERR_INVALID; }
    if (!full_rank(*host, L, P)) {
        *why = "rank [S^T; 1^T] < P: the constrained minimiser is not unique";
        return LINMIN_ERR_RANK;
    }
    return LINMIN_OK;
}

size_t handle_bytes(int L, int P, long long N, bool host_io)
{
    Bucket b{};
    if (!ipm_bucket(P, &b)) return 0;
    const size_t PQ = pq_of(P), n = (size_t)(N > 0 ? N : 1);
    (void)b;
    const size_t PPM = PP_MAX;
    size_t fixed = 4 * (size_t)P * L + 8 * 2 * (size_t)P * P + 8 + 4 * 2 * PPM * PPM + 4 * PPM +
                   4 * (size_t)P + 4 * 2 * (size_t)L * PQ + 4 + 8 * 8 +
                   8 * (MAX_SWAPS + 2) + 8 + 8 * ((size_t)P + 1) + 4 * ((size_t)P + 1);
    // tensor-core projection (the default precision): T, slices, exponents
    fixed += 8 * (size_t)L * P + tc_bslice_bytes(L, P, LINMIN_PROJ_TC) + 4 * (size_t)P;
    size_t per_pixel = 4 * 4 * (size_t)P + 4 + 4 + 8 + 8 + 8 + 8 + 4 + 4;
    if (host_io) per_pixel += 4 * (size_t)L + 2 * 4 * (size_t)P + 4 + 4;
    return fixed + (host_io ? 4 * (size_t)L : 0) + per_pixel * n;
}

}  // namespace lm

extern "C" {

const char *linmin_version(void) { return "linmin-gb300 0.1 (sm_103a)"; }

linmin_status linmin_default_options(linmin_options *opt)
{
    if (!opt) return LINMIN_ERR_INVALID;
    opt->precision = LINMIN_PROJ_TC;
    opt->constraint = LINMIN_STO;
    opt->max_iter = 100;
    opt->tol = 1e-9f;
    opt->refine_mu = 1e-9f;
    opt->cuda_stream = nullptr;
    opt->profile = 0;
    return LINMIN_OK;
}

linmin_status linmin_create(const float *library, int L, int P, const linmin_options *opt,
                            linmin_handle *out)
{
    if (!out) return fail(nullptr, LINMIN_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!library) return fail(nullptr, LINMIN_ERR_INVALID, "library is NULL");
    if (P < 1 || P > LINMIN_MAX_P)
        return fail(nullptr, LINMIN_ERR_UNSUPPORTED, "P must be in [1, LINMIN_MAX_P]");
    if (L < P || L > LINMIN_MAX_L)
        return fail(nullptr, LINMIN_ERR_INVALID, "L must be in [P, 4096]");
    linmin_options o;
    linmin_default_options(&o);
    if (opt) o = *opt;
    if ((o.precision != LINMIN_PROJ_DF && o.precision != LINMIN_PROJ_TC &&
         o.precision != LINMIN_PROJ_BF16) ||
        (o.constraint != LINMIN_STO && o.constraint != LINMIN_SLO && o.constraint != LINMIN_POS))
        return fail(nullptr, LINMIN_ERR_UNSUPPORTED,
                    "precision must be PROJ_DF, PROJ_TC or PROJ_BF16; constraint STO, SLO or POS");
    if (o.constraint != LINMIN_STO && P + 1 > LINMIN_MAX_P)
        return fail(nullptr, LINMIN_ERR_UNSUPPORTED, "SLO and POS need P <= LINMIN_MAX_P - 1");
    if (o.max_iter < 1 || !(o.tol > 0.f) || !(o.refine_mu > 0.f))
        return fail(nullptr, LINMIN_ERR_INVALID, "max_iter >= 1, tol > 0, refine_mu > 0");

    std::vector<float> hS;
    std::string why;
    const linmin_status lst = lm::load_library(library, L, P, &hS, &why);
    if (lst != LINMIN_OK) return fail(nullptr, lst, why);
    if (o.constraint == LINMIN_STO) return lm::create_from_host(hS.data(), L, P, o, out);
    // slo / pos: M S with a zero spectrum appended; rank [M S, 0; 1, 1] =
    // P + 1 exactly when rank S = P
    const float M = o.constraint == LINMIN_POS ? (float)LINMIN_POS_SCALE : 1.f;
    std::vector<float> hA((size_t)(P + 1) * L, 0.f);
    for (size_t e = 0; e < (size_t)P * L; ++e) hA[e] = hS[e];
    if (!full_rank(hA, L, P + 1))          // on S itself: the test is relative to columns
        return fail(nullptr, LINMIN_ERR_RANK,
                    "rank S < P: the SLO / POS minimiser is not unique");
    for (size_t e = 0; e < (size_t)P * L; ++e) hA[e] = M * hS[e];
    const linmin_status cst = lm::create_from_host(hA.data(), L, P + 1, o, out);
    if (cst != LINMIN_OK) return cst;
    (*out)->user_P = P;
    (*out)->slack = true;
    (*out)->slack_scale = M;
    if (o.constraint == LINMIN_POS) {
        // start at abundances 1/P in the caller's units (sum 1 against the
        // bound M): x' = 1/(M P) on the spectra, the rest on the slack
        (*out)->prep.slack_idx = P;
        (*out)->prep.slack_x0 = 1.f - 1.f / M;
    }
    return LINMIN_OK;
}

static linmin_status ensure_scratch(linmin_ctx *h, long long N)
{
    if (N <= h->capN) return LINMIN_OK;
    const size_t np = (size_t)N * h->P;
    cudaError_t a = cudaSuccess;
#define A(call) if (a == cudaSuccess) a = (call)
    A(dalloc(h, &h->c_hi, np));
    A(dalloc(h, &h->c_lo, np));
    A(dalloc(h, &h->x, np));
    A(dalloc(h, &h->lam, np));
    A(dalloc(h, &h->nu, (size_t)N));
    A(dalloc(h, &h->it, (size_t)N));
    A(dalloc(h, &h->retry, (size_t)N));
    A(dalloc(h, &h->mask, (size_t)N));
    A(dalloc(h, &h->xw.list[0], (size_t)N));
    A(dalloc(h, &h->xw.list[1], (size_t)N));
    A(dalloc(h, &h->xw.ksize, (size_t)N));
    A(dalloc(h, &h->rexp, (size_t)N));
    if (h->slack) {
        A(dalloc(h, &h->xa, np));
        A(dalloc(h, &h->sxa, np));
    }
#undef A
    if (a != cudaSuccess) { h->capN = 0; return cuda_fail(h, a, "scratch allocation"); }
    h->capN = N;
    return LINMIN_OK;
}

static IpmArgs ipm_args(linmin_ctx *h, long long N)
{
    IpmArgs ia;
    ia.N = N; ia.P = h->P; ia.max_iter = h->opt.max_iter;
    ia.c_hi = h->c_hi; ia.c_lo = h->c_lo;
    ia.Ghi = h->prep.Ghi; ia.Glo = h->prep.Glo; ia.grs = h->prep.grs;
    ia.slack_idx = h->prep.slack_idx; ia.slack_x0 = h->prep.slack_x0;
    ia.x_state = h->x; ia.lam_state = h->lam; ia.nu_state = h->nu; ia.it_state = h->it;
    ia.n_notconv = h->dcnt + 2;
    // pos works on M S, whose coordinates are M times smaller: the absolute
    // thresholds of the scaled problem shrink with them (mu with M^2)
    const float m = h->slack_scale;
    ia.tol_c = h->opt.tol / (m * m); ia.tol_d = 1e-6f / m; ia.eta = 0.99f;
    ia.list = nullptr; ia.list_len = nullptr;
    ia.mu_ref = MU_STOP / (m * m); ia.counter = h->dcnt + 0;
    return ia;
}

static linmin_status ensure_io(linmin_ctx *h, long long N)
{
    if (N <= h->capIO) return LINMIN_OK;
    const size_t np = (size_t)N * h->P;
    cudaError_t a = cudaSuccess;
#define A(call) if (a == cudaSuccess) a = (call)
    A(dalloc(h, &h->io_cube, (size_t)N * h->L));
    A(dalloc(h, &h->io_sigma, (size_t)h->L));
    A(dalloc(h, &h->io_x, np));
    A(dalloc(h, &h->io_sx, np));
    A(dalloc(h, &h->io_rms, (size_t)N));
    A(dalloc(h, &h->io_it, (size_t)N));
#undef A
    if (a != cudaSuccess) { h->capIO = 0; return cuda_fail(h, a, "staging allocation"); }
    h->capIO = N;
    return LINMIN_OK;
}

// C^-1 of linmin_unmix_cov: copied to the host, checked (finite,
// symmetric, positive definite by an fp64 Cholesky) and uploaded when its
// contents differ from the last checked one.
static linmin_status load_cov(linmin_ctx *h, const double *cov_inv)
{
    const int L = h->L;
    const size_t n = (size_t)L * L;
    std::vector<double> c(n);
    if (is_device_ptr(cov_inv)) {
        LM_CUDA(h, cudaMemcpy(c.data(), cov_inv, n * 8, cudaMemcpyDeviceToHost), "copy cov_inv");
    } else {
        std::memcpy(c.data(), cov_inv, n * 8);
    }
    unsigned long long hsh = 1469598103934665603ULL;
    const unsigned char *b = reinterpret_cast<const unsigned char *>(c.data());
    for (size_t i = 0; i < n * 8; ++i) { hsh ^= b[i]; hsh *= 1099511628211ULL; }
    if (h->cov && hsh == h->cov_hash) return LINMIN_OK;
    double amax = 0.0;
    for (double v : c) {
        if (!std::isfinite(v)) return fail(h, LINMIN_ERR_INVALID, "cov_inv has NaN/Inf");
        amax = std::fmax(amax, std::fabs(v));
    }
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < i; ++j)
            if (std::fabs(c[(size_t)i * L + j] - c[(size_t)j * L + i]) > 1e-9 * amax)
                return fail(h, LINMIN_ERR_INVALID, "cov_inv is not symmetric");
    // symmetric part, then its Cholesky as the positive-definiteness test
    std::vector<double> sym(n), f(n);
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j)
            sym[(size_t)i * L + j] = 0.5 * (c[(size_t)i * L + j] + c[(size_t)j * L + i]);
    f = sym;
    for (int k = 0; k < L; ++k) {
        double d = f[(size_t)k * L + k];
        for (int q = 0; q < k; ++q) d -= f[(size_t)k * L + q] * f[(size_t)k * L + q];
        if (!(d > 0.0)) return fail(h, LINMIN_ERR_INVALID, "cov_inv is not positive definite");
        d = std::sqrt(d);
        f[(size_t)k * L + k] = d;
        for (int i = k + 1; i < L; ++i) {
            double v = f[(size_t)i * L + k];
            for (int q = 0; q < k; ++q) v -= f[(size_t)i * L + q] * f[(size_t)k * L + q];
            f[(size_t)i * L + k] = v / d;
        }
    }
    cudaError_t a = cudaSuccess;
    if (!h->cov) {
        a = dalloc(h, &h->cov, n);
        if (a == cudaSuccess && !h->covT) a = dalloc(h, &h->covT, (size_t)L * h->P);
        if (a != cudaSuccess) return cuda_fail(h, a, "cov allocation");
    }
    LM_CUDA(h, cudaMemcpyAsync(h->cov, sym.data(), n * 8, cudaMemcpyHostToDevice, h->stream),
            "upload cov_inv");
    LM_CUDA(h, cudaStreamSynchronize(h->stream), "upload cov_inv");
    h->cov_hash = hsh;
    return LINMIN_OK;
}

// linmin_unmix (sigma) and linmin_unmix_cov (cov_inv): exactly one is set
static linmin_status unmix_impl(linmin_handle h, const float *cube, long long N, const float *sigma,
                                const double *cov_inv, float *abundances, float *uncertainties,
                                float *residual_rms, int *iterations,
                                const unsigned long long *col_mask = nullptr, int n_minerals = 0);

// Host cube of PIPE_MIN_N pixels or more: copied in PIPE_CHUNKS pieces on a
// copy stream, the projection of each piece starts as soon as it has
// arrived (the copy of the next piece overlaps it); with host outputs, x
// and sigma_x go back on the copy stream while the RMS runs.
constexpr int PIPE_CHUNKS = 8;
constexpr long long PIPE_MIN_N = 65536;

static linmin_status ensure_copy_stream(linmin_ctx *h)
{
    if (h->cstream) return LINMIN_OK;
    LM_CUDA(h, cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking), "copy stream");
    for (int k = 0; k < PIPE_CHUNKS; ++k)
        LM_CUDA(h, cudaEventCreateWithFlags(&h->pev_in[k], cudaEventDisableTiming), "event");
    LM_CUDA(h, cudaEventCreateWithFlags(&h->pev_out[0], cudaEventDisableTiming), "event");
    LM_CUDA(h, cudaEventCreateWithFlags(&h->pev_out[1], cudaEventDisableTiming), "event");
    return LINMIN_OK;
}

static linmin_status ensure_side_stream(linmin_ctx *h)
{
    if (h->xstream) return LINMIN_OK;
    LM_CUDA(h, cudaStreamCreateWithFlags(&h->xstream, cudaStreamNonBlocking), "side stream");
    for (cudaEvent_t &e : h->xev)
        LM_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    return LINMIN_OK;
}

#define LM_TRY(call) do { const cudaError_t e_ = (call); if (e_ != cudaSuccess) return e_; } while (0)
// Steps 4 and 5 of a call, after the interior point over all pixels: the
// crossover of every pixel (failures to the retry list), the retry list
// through the interior point from the start (float32, then double-float
// residual) and the crossover again.  Returns the first CUDA error.
static cudaError_t crossover_and_retry(linmin_ctx *h, long long N, float *d_x, float *d_sx)
{
    cudaStream_t st = h->stream;
    const int P = h->P;
    IpmArgs ia = ipm_args(h, N);
    // 4. crossover; failures appended to the retry list
    CrossArgs ca{};
    ca.N = N; ca.P = P; ca.Gt64 = h->prep.Gt64; ca.Ghi = h->prep.Ghi; ca.Glo = h->prep.Glo;
    ca.PP = h->bucket.PP; ca.scale = h->prep.scale; ca.gdiag = h->prep.gdiag;
    ca.c_hi = h->c_hi; ca.c_lo = h->c_lo; ca.x_in = h->x; ca.lam_in = h->lam;
    ca.x_out = d_x; ca.sx_out = d_sx; ca.mask = h->mask;
    ca.retry_list = h->retry; ca.retry_len = h->dcnt + 5; ca.n_unverified = nullptr;
    ca.tol_x = 1e-9 / h->slack_scale; ca.tol_g = 1e-9 / h->slack_scale;
    LM_TRY(launch_crossover(ca, h->xw, nullptr, nullptr, st));
    mark(h, 4);
    // 5. retry list: the interior point from the start with the accurate
    //    residual phase, then the crossover again
    ia.list = h->retry; ia.list_len = h->dcnt + 5;
    ia.mu_ref = h->opt.refine_mu / (h->slack_scale * h->slack_scale); ia.counter = h->dcnt + 1;
    LM_TRY(launch_ipm(h->bucket, false, ia, st));
    ia.counter = h->dcnt + 4;
    LM_TRY(launch_ipm(h->bucket, true, ia, st));
    // a pixel the retry crossover cannot verify keeps its interior-point
    // iterate and is reported as not converged (negative iteration count)
    ca.retry_list = nullptr; ca.retry_len = nullptr; ca.n_unverified = h->dcnt + 2;
    ca.it_mark = h->it;
    LM_TRY(launch_crossover(ca, h->xw, h->retry, h->dcnt + 5, st));
    mark(h, 5);
    return cudaSuccess;
}

static linmin_status unmix_impl(linmin_handle h, const float *cube, long long N, const float *sigma,
                                const double *cov_inv, float *abundances, float *uncertainties,
                                float *residual_rms, int *iterations,
                                const unsigned long long *col_mask, int n_minerals)
{
    if (!h) return fail(nullptr, LINMIN_ERR_INVALID, "handle is NULL");
    if (N < 0) return fail(h, LINMIN_ERR_INVALID, "N < 0");
    h->launches = 0;
    if (N == 0) return LINMIN_OK;
    if (!cube || (!sigma && !cov_inv))
        return fail(h, LINMIN_ERR_INVALID, sigma || cov_inv ? "cube is NULL" : "sigma is NULL");
    if (N > (1LL << 40)) return fail(h, LINMIN_ERR_INVALID, "N too large");
    const int L = h->L, P = h->P;
    cudaStream_t st = h->stream;
    LM_CUDA(h, cudaSetDevice(h->device), "cudaSetDevice");

    const bool dev_cube = is_device_ptr(cube), dev_sigma = !sigma || is_device_ptr(sigma);
    const bool dev_out[4] = {!abundances || is_device_ptr(abundances),
                             !uncertainties || is_device_ptr(uncertainties),
                             !residual_rms || is_device_ptr(residual_rms),
                             !iterations || is_device_ptr(iterations)};
    const bool host_any = !dev_cube || !dev_sigma || !dev_out[0] || !dev_out[1] || !dev_out[2] ||
                          !dev_out[3];
    if (!dev_sigma) {
        for (int l = 0; l < L; ++l)
            if (!(sigma[l] > 0.f) || !std::isfinite(sigma[l]))
                return fail(h, LINMIN_ERR_INVALID, "sigma must be finite and > 0");
    }
    linmin_status s;
    if (cov_inv && (s = load_cov(h, cov_inv)) != LINMIN_OK) return s;
    if ((s = ensure_scratch(h, N)) != LINMIN_OK) return s;
    if (host_any && (s = ensure_io(h, N)) != LINMIN_OK) return s;

    const size_t np = (size_t)N * h->user_P;    // caller-visible N x P outputs
    const float *d_cube = cube, *d_sigma = sigma;
    const bool piped = !dev_cube && N >= PIPE_MIN_N;
    const long long PC = (N + PIPE_CHUNKS - 1) / PIPE_CHUNKS;
    auto piece = [&](int k, long long &off, long long &nk) {
        off = k * PC;
        nk = off < N ? (N - off < PC ? N - off : PC) : 0;
    };
    if (piped) {
        if ((s = ensure_copy_stream(h)) != LINMIN_OK) return s;
        // after the work already queued on the handle's stream (it may read
        // the staging buffer), the pieces of the cube on the copy stream
        LM_CUDA(h, cudaEventRecord(h->pev_out[0], st), "event");
        LM_CUDA(h, cudaStreamWaitEvent(h->cstream, h->pev_out[0], 0), "event wait");
        for (int k = 0; k < PIPE_CHUNKS; ++k) {
            long long off, nk;
            piece(k, off, nk);
            if (nk > 0)
                LM_CUDA(h, cudaMemcpyAsync(h->io_cube + off * L, cube + off * L, (size_t)nk * L * 4,
                                           cudaMemcpyHostToDevice, h->cstream), "copy cube");
            LM_CUDA(h, cudaEventRecord(h->pev_in[k], h->cstream), "event");
        }
        d_cube = h->io_cube;
    } else if (!dev_cube) {
        LM_CUDA(h, cudaMemcpyAsync(h->io_cube, cube, (size_t)N * L * 4, cudaMemcpyHostToDevice, st),
                "copy cube");
        d_cube = h->io_cube;
    }
    if (!dev_sigma) {
        LM_CUDA(h, cudaMemcpyAsync(h->io_sigma, sigma, (size_t)L * 4, cudaMemcpyHostToDevice, st),
                "copy sigma");
        d_sigma = h->io_sigma;
    }
    float *d_x = abundances ? (dev_out[0] ? abundances : h->io_x) : h->x;
    float *d_sx = uncertainties ? (dev_out[1] ? uncertainties : h->io_sx) : nullptr;
    // slo / pos: the pipeline writes the internal (slack-augmented) results
    float *u_x = d_x, *u_sx = d_sx;
    if (h->slack) {
        d_x = h->xa;
        d_sx = uncertainties ? h->sxa : nullptr;
    }
    float *d_rms = residual_rms ? (dev_out[2] ? residual_rms : h->io_rms) : nullptr;
    int *d_it = iterations ? (dev_out[3] ? iterations : h->io_it) : nullptr;

    LM_CUDA(h, cudaMemsetAsync(h->prep.flags, 0, sizeof(int), st), "memset");
    LM_CUDA(h, cudaMemsetAsync(h->dcnt, 0, 8 * sizeof(unsigned long long), st), "memset");
    // exact tensor-core projection of a resident cube: its exponent pass
    // goes on the side stream, after the work queued so far, concurrent
    // with the library preparation below
    const bool tma_proj = h->opt.precision == LINMIN_PROJ_TC && tma_projection_usable(d_cube, N, L);
    const bool side_exp = tma_proj && !piped;
    if (side_exp) {
        if ((s = ensure_side_stream(h)) != LINMIN_OK) return s;
        LM_CUDA(h, cudaEventRecord(h->xev[0], st), "event");
        LM_CUDA(h, cudaStreamWaitEvent(h->xstream, h->xev[0], 0), "event wait");
        LM_CUDA(h, launch_rowexp(d_cube, N, L, h->rexp, h->xstream), "exponent pass");
        LM_CUDA(h, cudaEventRecord(h->xev[1], h->xstream), "event");
    }
    mark(h, 0);
    if (cov_inv)
        LM_CUDA(h, launch_prep_cov(h->dS, h->cov, L, P, h->bucket.PP, h->prep, h->covT, st),
                "prep kernels");
    else
        LM_CUDA(h, launch_prep(h->dS, d_sigma, L, P, h->bucket.PP, h->prep, st), "prep kernels");
    mark(h, 1);
    int proj_launches = 0;
    if (h->opt.precision != LINMIN_PROJ_DF) {
        LM_CUDA(h, launch_tc_prep(h->dS, d_sigma, cov_inv ? h->covT : nullptr, L, P,
                                  h->prep.scale, h->opt.precision, h->bsl, h->fexp, st),
                "projection prep");
        proj_launches += h->opt.precision == LINMIN_PROJ_TC ? 2 : 1;
    }
    // the projection, piece by piece as the cube arrives when piped
    for (int k = 0; k < (piped ? PIPE_CHUNKS : 1); ++k) {
        long long off = 0, nk = N;
        if (piped) {
            piece(k, off, nk);
            LM_CUDA(h, cudaStreamWaitEvent(st, h->pev_in[k], 0), "event wait");
            if (nk <= 0) continue;
        }
        const float *cin = d_cube + off * L;
        float *chi = h->c_hi + off * P, *clo = h->c_lo + off * P;
        if (h->opt.precision == LINMIN_PROJ_DF) {
            LM_CUDA(h, launch_project(cin, nk, L, P, h->prep.Bhi, h->prep.Blo, chi, clo, st),
                    "projection kernel");
            ++proj_launches;
        } else if (tma_proj) {
            if (side_exp)
                LM_CUDA(h, cudaStreamWaitEvent(st, h->xev[1], 0), "event wait");
            else
                LM_CUDA(h, launch_rowexp(cin, nk, L, h->rexp + off, st), "exponent pass");
            LM_CUDA(h, launch_project_tma(cin, nk, L, P, h->bsl, h->fexp, h->rexp + off, chi, clo,
                                          h->prep.flags, st), "tensor-core projection");
            proj_launches += 2;
        } else {
            LM_CUDA(h, launch_project_tc(cin, nk, L, P, h->opt.precision, h->bsl, h->fexp, chi, clo,
                                         h->prep.flags, st), "tensor-core projection");
            ++proj_launches;
        }
    }
    if (col_mask) {
        LM_CUDA(h, launch_exclude(col_mask, n_minerals, h->c_hi, h->c_lo, N, P, st),
                "column-subset penalty");
        ++proj_launches;
    }
    mark(h, 2);
    if (h->defer_ipm) {
        // batch: the interior point of this cube runs in the batch's launch
        h->pend.N = N; h->pend.cube = d_cube; h->pend.x = d_x; h->pend.sx = d_sx;
        h->pend.rms = d_rms; h->pend.it = d_it;
        h->pend.launches = (cov_inv ? PREP_COV_LAUNCHES : PREP_LAUNCHES) + proj_launches;
        return LINMIN_OK;
    }

    IpmArgs ia = ipm_args(h, N);
    // 3. all pixels: float32 residual until mu <= mu_stop
    ia.counter = h->dcnt + 0;
    LM_CUDA(h, launch_ipm(h->bucket, false, ia, st), "interior-point kernel");
    mark(h, 3);
    LM_CUDA(h, crossover_and_retry(h, N, d_x, d_sx), "crossover");
    // host x and sigma_x: final here without a slack; copied back on the
    // copy stream while the RMS runs
    const bool early_out = piped && !h->slack;
    if (early_out && ((abundances && !dev_out[0]) || (uncertainties && !dev_out[1]))) {
        LM_CUDA(h, cudaEventRecord(h->pev_out[1], st), "event");
        LM_CUDA(h, cudaStreamWaitEvent(h->cstream, h->pev_out[1], 0), "event wait");
        if (abundances && !dev_out[0])
            LM_CUDA(h, cudaMemcpyAsync(abundances, d_x, np * 4, cudaMemcpyDeviceToHost, h->cstream),
                    "copy x");
        if (uncertainties && !dev_out[1])
            LM_CUDA(h, cudaMemcpyAsync(uncertainties, d_sx, np * 4, cudaMemcpyDeviceToHost,
                                       h->cstream), "copy sx");
    }
    if (d_rms) LM_CUDA(h, launch_rms(d_cube, h->dS, d_x, N, L, P, d_rms, st), "rms kernel");
    mark(h, 6);
    if (h->opt.profile) ++h->calls;
    h->launches = (cov_inv ? PREP_COV_LAUNCHES : PREP_LAUNCHES) + proj_launches + 1 +
                  crossover_launches(true, P) +
                  2 + crossover_launches(false, P) + (d_rms ? 1 : 0);
    if (d_it) LM_CUDA(h, cudaMemcpyAsync(d_it, h->it, (size_t)N * 4, cudaMemcpyDeviceToDevice, st),
                      "copy iterations");
    if (h->slack) {
        LM_CUDA(h, launch_strip_slack(h->xa, h->sxa, N, h->user_P, h->slack_scale,
                                      h->opt.constraint == LINMIN_POS,
                                      abundances ? u_x : nullptr, u_sx, d_it, h->dcnt + 2, st),
                "slack outputs");
        ++h->launches;
    }
    d_x = u_x;
    d_sx = u_sx;

    if (!host_any) return LINMIN_OK;
    if (abundances && !dev_out[0] && !early_out)
        LM_CUDA(h, cudaMemcpyAsync(abundances, d_x, np * 4, cudaMemcpyDeviceToHost, st), "copy x");
    if (uncertainties && !dev_out[1] && !early_out)
        LM_CUDA(h, cudaMemcpyAsync(uncertainties, d_sx, np * 4, cudaMemcpyDeviceToHost, st), "copy sx");
    if (residual_rms && !dev_out[2])
        LM_CUDA(h, cudaMemcpyAsync(residual_rms, d_rms, (size_t)N * 4, cudaMemcpyDeviceToHost, st),
                "copy rms");
    if (iterations && !dev_out[3])
        LM_CUDA(h, cudaMemcpyAsync(iterations, d_it, (size_t)N * 4, cudaMemcpyDeviceToHost, st),
                "copy iterations");
    if (piped) LM_CUDA(h, cudaStreamSynchronize(h->cstream), "output copies");
    return linmin_wait(h, nullptr);
}

linmin_status linmin_unmix(linmin_handle h, const float *cube, long long N, const float *sigma,
                           float *abundances, float *uncertainties, float *residual_rms,
                           int *iterations)
{
    if (h && N > 0 && !sigma) return fail(h, LINMIN_ERR_INVALID, "sigma is NULL");
    return unmix_impl(h, cube, N, sigma, nullptr, abundances, uncertainties, residual_rms,
                      iterations);
}

linmin_status linmin_unmix_masked(linmin_handle h, const float *cube, long long N,
                                  const float *sigma, const unsigned long long *mask,
                                  int n_minerals, float *abundances, float *uncertainties,
                                  float *residual_rms, int *iterations)
{
    if (!h) return fail(nullptr, LINMIN_ERR_INVALID, "handle is NULL");
    if (n_minerals < 0 || n_minerals >= h->user_P)
        return fail(h, LINMIN_ERR_INVALID, "0 <= n_minerals < P (columns >= n_minerals are always kept)");
    if (N > 0 && !sigma) return fail(h, LINMIN_ERR_INVALID, "sigma is NULL");
    if (N > 0 && (!mask || !is_device_ptr(mask)))
        return fail(h, LINMIN_ERR_INVALID, "mask must be device memory");
    return unmix_impl(h, cube, N, sigma, nullptr, abundances, uncertainties, residual_rms,
                      iterations, mask, n_minerals);
}

linmin_status linmin_unmix_cov(linmin_handle h, const float *cube, long long N,
                               const double *cov_inv, float *abundances, float *uncertainties,
                               float *residual_rms, int *iterations)
{
    if (h && N > 0 && !cov_inv) return fail(h, LINMIN_ERR_INVALID, "cov_inv is NULL");
    return unmix_impl(h, cube, N, nullptr, cov_inv, abundances, uncertainties, residual_rms,
                      iterations);
}

linmin_status linmin_wait(linmin_handle h, long long *n_not_converged)
{
    if (!h) return fail(nullptr, LINMIN_ERR_INVALID, "handle is NULL");
    unsigned long long c[4] = {0, 0, 0, 0};
    int flags = 0;
    LM_CUDA(h, cudaStreamSynchronize(h->stream), "kernel execution");
    LM_CUDA(h, cudaMemcpy(c, h->dcnt, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
    LM_CUDA(h, cudaMemcpy(&flags, h->prep.flags, sizeof(int), cudaMemcpyDeviceToHost), "read flags");
    if (n_not_converged) *n_not_converged = (long long)c[2];
    if (flags & 1) return fail(h, LINMIN_ERR_INVALID, "sigma must be finite and > 0");
    if (flags & 2) return fail(h, LINMIN_ERR_INVALID, "library has a zero whitened scale");
    if (flags & 4) return fail(h, LINMIN_ERR_TIMEOUT, "tensor-core projection: an MMA did not complete");
    if (c[2]) return fail(h, LINMIN_ERR_NOT_CONVERGED,
                          std::to_string(c[2]) + " pixels hit max_iter");
    return LINMIN_OK;
}

linmin_status linmin_phase_times(linmin_handle h, float *ms_out, int n)
{
    return linmin_phase_times_at(h, 0, ms_out, n);
}

linmin_status linmin_phase_times_at(linmin_handle h, int back, float *ms_out, int n)
{
    if (!h) return fail(nullptr, LINMIN_ERR_INVALID, "handle is NULL");
    if (!h->opt.profile || !ms_out)
        return fail(h, LINMIN_ERR_INVALID, "profiling is off");
    if (back < 0 || back >= LINMIN_PHASE_RING || back >= h->calls)
        return fail(h, LINMIN_ERR_INVALID, "no such profiled call");
    cudaEvent_t *set = h->ev[(h->calls - 1 - back) % LINMIN_PHASE_RING];
    LM_CUDA(h, cudaEventSynchronize(set[LINMIN_NUM_PHASES]), "event sync");
    for (int i = 0; i < n && i < LINMIN_NUM_PHASES; ++i) {
        float ms = 0.f;
        LM_CUDA(h, cudaEventElapsedTime(&ms, set[i], set[i + 1]), "event time");
        ms_out[i] = ms;
    }
    return LINMIN_OK;
}

// The rest of a call stopped by defer_ipm, after the batch's interior
// point: crossover, retry, RMS and the iteration counts (device buffers,
// sum-to-one).
static linmin_status unmix_back(linmin_ctx *h)
{
    const long long N = h->pend.N;
    cudaStream_t st = h->stream;
    mark(h, 3);
    LM_CUDA(h, crossover_and_retry(h, N, h->pend.x, h->pend.sx), "crossover");
    if (h->pend.rms)
        LM_CUDA(h, launch_rms(h->pend.cube, h->dS, h->pend.x, N, h->L, h->P, h->pend.rms, st),
                "rms kernel");
    mark(h, 6);
    if (h->opt.profile) ++h->calls;
    // the batch's interior-point launch is counted with the batch, not here
    h->launches = h->pend.launches + crossover_launches(true, h->P) + 2 +
                  crossover_launches(false, h->P) +
                  (h->pend.rms ? 1 : 0);
    if (h->pend.it)
        LM_CUDA(h, cudaMemcpyAsync(h->pend.it, h->it, (size_t)N * 4, cudaMemcpyDeviceToDevice, st),
                "copy iterations");
    return LINMIN_OK;
}

linmin_status linmin_unmix_batch(int n, const linmin_handle *handles, const float *const *cubes,
                                 const long long *N, const float *const *sigmas,
                                 float *const *abundances, float *const *uncertainties,
                                 float *const *residual_rms, int *const *iterations)
{
    if (n <= 0 || !handles || !handles[0]) return fail(nullptr, LINMIN_ERR_INVALID, "no handles");
    linmin_ctx *h0 = handles[0];
    if (!cubes || !N || !sigmas || !abundances)
        return fail(h0, LINMIN_ERR_INVALID, "cubes, N, sigmas and abundances are required");
    auto dev_or_null = [](const void *q) { return !q || is_device_ptr(q); };
    for (int i = 0; i < n; ++i) {
        linmin_ctx *h = handles[i];
        if (!h) return fail(h0, LINMIN_ERR_INVALID, "a handle is NULL");
        if (h->device != h0->device || h->stream != h0->stream)
            return fail(h0, LINMIN_ERR_INVALID, "batch handles must share the device and the stream");
        if (h->slack) return fail(h0, LINMIN_ERR_INVALID, "batch handles must be sum-to-one");
        if (N[i] < 0 || N[i] > (1LL << 40)) return fail(h0, LINMIN_ERR_INVALID, "N out of range");
        if (N[i] == 0) continue;
        if (!cubes[i] || !sigmas[i] || !abundances[i])
            return fail(h0, LINMIN_ERR_INVALID, "cube, sigma and abundances are required");
        if (!is_device_ptr(cubes[i]) || !is_device_ptr(sigmas[i]) || !is_device_ptr(abundances[i]) ||
            (uncertainties && !dev_or_null(uncertainties[i])) ||
            (residual_rms && !dev_or_null(residual_rms[i])) || (iterations && !dev_or_null(iterations[i])))
            return fail(h0, LINMIN_ERR_INVALID, "batch buffers must be device memory");
        for (int j = 0; j < i; ++j)
            if (handles[j] == h && N[j] > 0)
                return fail(h0, LINMIN_ERR_INVALID, "a handle appears twice in the batch");
    }
    cudaStream_t st = h0->stream;
    LM_CUDA(h0, cudaSetDevice(h0->device), "cudaSetDevice");
    // 1. every cube up to its projection (library preparation, c~)
    for (int i = 0; i < n; ++i) {
        if (N[i] == 0) continue;
        linmin_ctx *h = handles[i];
        h->defer_ipm = true;
        const linmin_status s = unmix_impl(h, cubes[i], N[i], sigmas[i], nullptr, abundances[i],
                                           uncertainties ? uncertainties[i] : nullptr,
                                           residual_rms ? residual_rms[i] : nullptr,
                                           iterations ? iterations[i] : nullptr);
        h->defer_ipm = false;
        if (s != LINMIN_OK) {
            if (h != h0) h0->err = h->err;
            return s;
        }
    }
    // 2. one interior-point launch per group of cubes with the same bucket,
    //    P and stopping options: one work counter over all their pixels
    std::vector<std::vector<int>> groups;
    for (int i = 0; i < n; ++i) {
        if (N[i] == 0) continue;
        const linmin_ctx *h = handles[i];
        bool placed = false;
        for (auto &g : groups) {
            const linmin_ctx *r = handles[g[0]];
            if (r->bucket.NS == h->bucket.NS && r->bucket.G == h->bucket.G && r->P == h->P &&
                r->opt.max_iter == h->opt.max_iter && r->opt.tol == h->opt.tol) {
                g.push_back(i);
                placed = true;
                break;
            }
        }
        if (!placed) groups.push_back({i});
    }
    std::vector<IpmCube> desc;
    std::vector<size_t> first;
    for (auto &g : groups) {
        first.push_back(desc.size());
        long long start = 0;
        for (int i : g) {
            const linmin_ctx *h = handles[i];
            IpmCube c{};
            c.N = N[i]; c.start = start; c.c_hi = h->c_hi; c.Ghi = h->prep.Ghi; c.grs = h->prep.grs;
            c.x_state = h->x; c.lam_state = h->lam; c.nu_state = h->nu; c.it_state = h->it;
            desc.push_back(c);
            start += N[i];
        }
    }
    const size_t counters = sizeof(unsigned long long) * groups.size();
    const size_t need = counters + sizeof(IpmCube) * desc.size();
    if (need > h0->bdesc_cap) {
        h0->bdesc_cap = 0;                 // dalloc frees the old buffer first
        LM_CUDA(h0, dalloc(h0, &h0->bdesc, need), "batch descriptors");
        h0->bdesc_cap = need;
    }
    if (!groups.empty()) {
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(h0->bdesc);
        IpmCube *ddesc = reinterpret_cast<IpmCube *>(h0->bdesc + counters);
        LM_CUDA(h0, cudaMemsetAsync(cnt, 0, counters, st), "memset");
        // pageable source: the copy has taken the data when the call returns
        LM_CUDA(h0, cudaMemcpyAsync(ddesc, desc.data(), sizeof(IpmCube) * desc.size(),
                                    cudaMemcpyHostToDevice, st), "copy batch descriptors");
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            linmin_ctx *r = handles[groups[gi][0]];
            unsigned long long total = 0;
            for (int i : groups[gi]) total += (unsigned long long)N[i];
            IpmArgs ia = ipm_args(r, (long long)total);
            ia.cubes = ddesc + first[gi];
            ia.n_cubes = (int)groups[gi].size();
            ia.total = total;
            ia.counter = cnt + gi;
            LM_CUDA(h0, launch_ipm_batch(r->bucket, ia, st), "batched interior-point kernel");
        }
    }
    // 3. every cube: crossover, retry, RMS
    for (int i = 0; i < n; ++i) {
        if (N[i] == 0) continue;
        const linmin_status s = unmix_back(handles[i]);
        if (s != LINMIN_OK) {
            if (handles[i] != h0) h0->err = handles[i]->err;
            return s;
        }
    }
    return LINMIN_OK;
}

linmin_status linmin_destroy(linmin_handle h)
{
    if (!h) return LINMIN_OK;
    cudaStreamSynchronize(h->stream);
    return lm::destroy_async(h);
}


int linmin_get_lanes(linmin_handle h)
{
    return h ? h->bucket.G : -1;
}

linmin_status linmin_live_allocations(long long *count)
{
    if (!count) return LINMIN_ERR_INVALID;
    *count = g_live_allocs.load();
    return LINMIN_OK;
}

linmin_status linmin_set_lanes(linmin_handle h, int lanes)
{
    if (!h) return fail(nullptr, LINMIN_ERR_INVALID, "handle is NULL");
    Bucket c[16];
    const int n = ipm_candidates(h->P, c, 16);
    for (int i = 0; i < n; ++i)
        if (c[i].G == lanes) { h->bucket = c[i]; return LINMIN_OK; }
    return fail(h, LINMIN_ERR_UNSUPPORTED, "no compiled bucket with that many lanes for this P");
}

linmin_status linmin_autotune(linmin_handle h, const float *cube, long long N, const float *sigma,
                              int *lanes_out, float *ms_out, int n_ms, int *n_candidates)
{
    if (!h) return fail(nullptr, LINMIN_ERR_INVALID, "handle is NULL");
    if (!cube || !sigma || N < 1) return fail(h, LINMIN_ERR_INVALID, "cube, sigma, N >= 1");
    const int L = h->L, P = h->P;
    const long long n = N < 32768 ? N : 32768;
    cudaStream_t st = h->stream;
    const bool dev_cube = is_device_ptr(cube), dev_sigma = !sigma || is_device_ptr(sigma);
    if (!dev_sigma)
        for (int l = 0; l < L; ++l)
            if (!(sigma[l] > 0.f) || !std::isfinite(sigma[l]))
                return fail(h, LINMIN_ERR_INVALID, "sigma must be finite and > 0");
    linmin_status s;
    if ((s = ensure_scratch(h, n)) != LINMIN_OK) return s;
    if ((!dev_cube || !dev_sigma) && (s = ensure_io(h, n)) != LINMIN_OK) return s;
    const float *d_cube = cube, *d_sigma = sigma;
    if (!dev_cube) {
        LM_CUDA(h, cudaMemcpyAsync(h->io_cube, cube, (size_t)n * L * 4, cudaMemcpyHostToDevice, st),
                "copy cube");
        d_cube = h->io_cube;
    }
    if (!dev_sigma) {
        LM_CUDA(h, cudaMemcpyAsync(h->io_sigma, sigma, (size_t)L * 4, cudaMemcpyHostToDevice, st),
                "copy sigma");
        d_sigma = h->io_sigma;
    }
    Bucket cand[16];
    const int nc = ipm_candidates(P, cand, 16);
    if (n_candidates) *n_candidates = nc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LM_CUDA(h, cudaEventCreate(&e0), "event");
    LM_CUDA(h, cudaEventCreate(&e1), "event");
    int best = -1;
    float best_ms = 3.4e38f;
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < nc && err == cudaSuccess; ++i) {
        err = launch_prep(h->dS, d_sigma, L, P, cand[i].PP, h->prep, st);
        if (err == cudaSuccess && i == 0)
            err = launch_project(d_cube, n, L, P, h->prep.Bhi, h->prep.Blo, h->c_hi, h->c_lo, st);
        float t_i = 3.4e38f;
        for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
            err = cudaMemsetAsync(h->dcnt, 0, 8 * sizeof(unsigned long long), st);
            if (err == cudaSuccess) err = cudaEventRecord(e0, st);
            if (err == cudaSuccess) err = launch_ipm(cand[i], false, ipm_args(h, n), st);
            if (err == cudaSuccess) err = cudaEventRecord(e1, st);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && ms < t_i) t_i = ms;
        }
        if (ms_out && i < n_ms) ms_out[i] = t_i;
        if (err == cudaSuccess && t_i < best_ms) { best_ms = t_i; best = i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(h, err, "autotune");
    if (best >= 0) h->bucket = cand[best];
    if (lanes_out) *lanes_out = h->bucket.G;
    return LINMIN_OK;
}

int linmin_last_launches(linmin_handle h)
{
    return h ? h->launches : -1;
}

const char *linmin_last_error(linmin_handle h)
{
    g_msg = h ? h->err : g_create_error;
    return g_msg.c_str();
}

}  // extern "C"

void lm::set_global_error(const std::string &m) { g_create_error = m; }

// outside the C block: a C++ function of namespace lm
linmin_status lm::reserve(linmin_handle h, long long N, bool host_io)
{
    linmin_status st = ensure_scratch(h, N);
    if (st == LINMIN_OK && host_io) st = ensure_io(h, N);
    return st;
}

// A handle for a library already loaded and checked (lm::load_library),
// with validated options.
linmin_status lm::create_from_host(const float *hS, int L, int P, const linmin_options &o,
                                   linmin_handle *out)
{
    *out = nullptr;
    linmin_ctx *h = new linmin_ctx();
    h->L = L; h->P = P; h->user_P = P; h->opt = o;
    h->stream = (cudaStream_t)o.cuda_stream;
    h->fail_at = injected_alloc_failure();
    cudaGetDevice(&h->device);
    if (!ipm_bucket(P, &h->bucket)) { delete h; return fail(nullptr, LINMIN_ERR_UNSUPPORTED, "P"); }
    cudaError_t a = pool_acquire(h->device, &h->pool);
    if (a != cudaSuccess) {
        delete h;
        return cuda_fail(nullptr, a, "memory pool");
    }
    const int PQ = pq_of(P);
#define A(call) if (a == cudaSuccess) a = (call)
    A(dalloc(h, &h->dS, (size_t)P * L));
    A(dalloc(h, &h->prep.G64, (size_t)P * P));
    A(dalloc(h, &h->prep.Gt64, (size_t)P * P));
    A(dalloc(h, &h->prep.scale, 1));
    // sized for the largest bucket: the handle may switch buckets (autotune)
    A(dalloc(h, &h->prep.Ghi, (size_t)PP_MAX * PP_MAX));
    A(dalloc(h, &h->prep.Glo, (size_t)PP_MAX * PP_MAX));
    A(dalloc(h, &h->prep.grs, (size_t)PP_MAX));
    A(dalloc(h, &h->prep.gdiag, (size_t)P));
    A(dalloc(h, &h->prep.Bhi, (size_t)L * PQ));
    A(dalloc(h, &h->prep.Blo, (size_t)L * PQ));
    A(dalloc(h, &h->prep.flags, 1));
    A(dalloc(h, &h->dcnt, 8));
    A(dalloc(h, &h->xw.len, (size_t)MAX_SWAPS + 2));
    A(dalloc(h, &h->xw.len_all, 1));
    A(dalloc(h, &h->xw.cursor, (size_t)P + 1));
    A(dalloc(h, &h->xw.hist, (size_t)P + 1));
    if (o.precision != LINMIN_PROJ_DF) {
        A(dalloc(h, &h->covT, (size_t)L * P));
        A(dalloc(h, &h->bsl, tc_bslice_bytes(L, P, o.precision) / 2));
        A(dalloc(h, &h->fexp, (size_t)P));
    }
    A(cudaMemcpyAsync(h->dS, hS, (size_t)P * L * 4, cudaMemcpyHostToDevice, h->stream));
    // linmin_wait before any call reads no flag and no count
    A(cudaMemsetAsync(h->prep.flags, 0, sizeof(int), h->stream));
    A(cudaMemsetAsync(h->dcnt, 0, 8 * sizeof(unsigned long long), h->stream));
    A(cudaStreamSynchronize(h->stream));       // hS belongs to the caller
    if (o.profile)
        for (auto &set : h->ev)
            for (cudaEvent_t &e : set) A(cudaEventCreate(&e));
#undef A
    if (a != cudaSuccess) {
        linmin_status st = cuda_fail(nullptr, a, "linmin_create allocation");
        linmin_destroy(h);
        return st;
    }
    *out = h;
    return LINMIN_OK;
}

// Free a handle without waiting for its stream: every free is ordered
// after the work already queued there.
linmin_status lm::destroy_async(linmin_handle h)
{
    if (!h) return LINMIN_OK;
    // the side stream may still write rexp if a call failed before joining it
    if (h->xstream) cudaStreamSynchronize(h->xstream);
    for (auto &set : h->ev)
        for (cudaEvent_t e : set)
            if (e) cudaEventDestroy(e);
    void *ptrs[] = {h->dS, h->prep.G64, h->prep.Gt64, h->prep.scale, h->prep.Ghi, h->prep.Glo,
                    h->prep.grs, h->prep.gdiag, h->prep.Bhi, h->prep.Blo, h->prep.flags, h->dcnt,
                    h->c_hi, h->c_lo, h->x, h->lam, h->nu, h->it, h->retry, h->mask, h->rexp,
                    h->xw.list[0], h->xw.list[1], h->xw.ksize, h->xw.len, h->xw.len_all,
                    h->xw.cursor, h->xw.hist, h->io_cube, h->io_sigma,
                    h->io_x, h->io_sx, h->io_rms, h->io_it, h->cov, h->covT, h->bsl,
                    h->fexp, h->xa, h->sxa, h->bdesc};
    for (void *p : ptrs)
        if (p) { cudaFreeAsync(p, h->stream); --g_live_allocs; }
    if (h->cstream) {
        cudaStreamSynchronize(h->cstream);
        cudaStreamDestroy(h->cstream);
    }
    if (h->xstream) cudaStreamDestroy(h->xstream);
    for (cudaEvent_t e : h->xev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->pev_in)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->pev_out)
        if (e) cudaEventDestroy(e);
    if (h->pool) pool_release(h->device);
    delete h;
    return LINMIN_OK;
}
