// linmin_unmix_noalloc: the unmixing path with every scratch buffer carved
// out of one statically sized device array, for callers that cannot
// allocate device memory (see include/linmin.h).
//
// The array is a file-scope __device__ object: each GPU that loads this
// library reserves it for the life of the process.  Host code cannot use
// the symbol as a device address; the address is looked up once per device
// with cudaGetSymbolAddress (first call on that device) and cached.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "ipm.cuh"
#include "kernels.cuh"
#include "linmin.h"

using namespace lm;

namespace {

constexpr size_t NOALLOC_BYTES = (size_t)LINMIN_NOALLOC_SCRATCH_MB << 20;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up on
// the first call per device, with that device current).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Bump allocator over the scratch array (256-byte aligned pieces).  A
// piece that does not fit within cap sets ok = false (and returns the
// base, never an address past the array).
struct Carve {
    unsigned char *base;
    size_t off = 0, cap;
    bool ok = true;
    template <typename T>
    T *take(size_t n)
    {
        if (n == 0) n = 1;
        const size_t start = (off + 255) & ~(size_t)255;
        if (start < off || start > cap || n > (cap - start) / sizeof(T)) {
            ok = false;
            return reinterpret_cast<T *>(base);
        }
        off = start + n * sizeof(T);
        return reinterpret_cast<T *>(base + start);
    }
};

// Every per-pixel piece holds at least 4 (4 P + 11) bytes per pixel, so a
// larger N cannot fit: refused before any size arithmetic can overflow.
long long coarse_max_pixels(int P) { return (long long)(NOALLOC_BYTES / (4 * (4 * (size_t)P + 11))); }

// Bytes the call needs (rounded pieces), or 0 when they exceed the array.
size_t scratch_needed(int L, int P, int PP, long long N)
{
    if (N > coarse_max_pixels(P)) return 0;
    Carve c{nullptr, 0, NOALLOC_BYTES};
    const int PQ = pq_of(P);
    c.take<double>((size_t)P * P);
    c.take<double>((size_t)P * P);
    c.take<double>(1);
    c.take<float>((size_t)PP * PP);
    c.take<float>((size_t)PP * PP);
    c.take<float>(PP);
    c.take<float>(P);
    c.take<float>((size_t)L * PQ);
    c.take<float>((size_t)L * PQ);
    c.take<int>(1);
    c.take<unsigned long long>(8);
    c.take<unsigned long long>(MAX_SWAPS + 2);
    c.take<unsigned long long>(1);
    c.take<unsigned long long>(P + 1);
    c.take<unsigned int>(P + 1);
    for (int k = 0; k < 4; ++k) c.take<float>((size_t)N * P);
    c.take<float>(N);
    c.take<int>(N);
    c.take<long long>(N);
    c.take<unsigned long long>(N);
    c.take<long long>(N);
    c.take<long long>(N);
    c.take<int>(N);
    return c.ok ? c.off : 0;
}

// Device memory of the current device (or managed memory).  Memory of
// another GPU is refused: the kernels run on the current one.
bool is_device(const void *p, int dev)
{
    if (!p) return true;   // NULL outputs are allowed
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// When the preparation flagged sigma (non-finite or <= 0) or the library
// (zero whitened scale), every output of the call is marked: NaN
// abundances, uncertainties and RMS, iteration counts INT_MIN.
__global__ void noalloc_mark_invalid_kernel(const int *flags, long long N, int P, float *x,
                                            float *sx, float *rms, int *it)
{
    if (*flags == 0) return;
    const float nan = __int_as_float(0x7fc00000);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = first; i < N * P; i += stride) {
        if (x) x[i] = nan;
        if (sx) sx[i] = nan;
    }
    for (long long i = first; i < N; i += stride) {
        if (rms) rms[i] = nan;
        if (it) it[i] = INT_MIN;
    }
}

}  // namespace

extern "C" {

linmin_status linmin_unmix_noalloc(const float *library, int L, int P, const float *cube,
                                   long long N, const float *sigma, float *abundances,
                                   float *uncertainties, float *residual_rms, int *iterations,
                                   void *cuda_stream)
{
    if (N < 0 || !library || (N > 0 && (!cube || !sigma))) return LINMIN_ERR_INVALID;
    Bucket b;
    if (P < 1 || P > LINMIN_MAX_P || !ipm_bucket(P, &b)) return LINMIN_ERR_UNSUPPORTED;
    if (L < P || L > LINMIN_MAX_L) return LINMIN_ERR_INVALID;
    if (N == 0) return LINMIN_OK;
    // beyond the static array: refuse (limit stated with LINMIN_NOALLOC_SCRATCH_MB)
    if (scratch_needed(L, P, b.PP, N) == 0) return LINMIN_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LINMIN_ERR_CUDA;
    if (!is_device(library, dev) || !is_device(cube, dev) || !is_device(sigma, dev) ||
        !is_device(abundances, dev) || !is_device(uncertainties, dev) ||
        !is_device(residual_rms, dev) || !is_device(iterations, dev))
        return LINMIN_ERR_INVALID;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return LINMIN_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int PP = b.PP, PQ = pq_of(P);
    Carve c{(unsigned char *)base, 0, NOALLOC_BYTES};
    Prep pr;
    pr.G64 = c.take<double>((size_t)P * P);
    pr.Gt64 = c.take<double>((size_t)P * P);
    pr.scale = c.take<double>(1);
    pr.Ghi = c.take<float>((size_t)PP * PP);
    pr.Glo = c.take<float>((size_t)PP * PP);
    pr.grs = c.take<float>(PP);
    pr.gdiag = c.take<float>(P);
    pr.Bhi = c.take<float>((size_t)L * PQ);
    pr.Blo = c.take<float>((size_t)L * PQ);
    pr.flags = c.take<int>(1);
    unsigned long long *cnt = c.take<unsigned long long>(8);
    CrossoverScratch xw;
    xw.len = c.take<unsigned long long>(MAX_SWAPS + 2);
    xw.len_all = c.take<unsigned long long>(1);
    xw.cursor = c.take<unsigned long long>(P + 1);
    xw.hist = c.take<unsigned int>(P + 1);
    float *c_hi = c.take<float>((size_t)N * P);
    float *c_lo = c.take<float>((size_t)N * P);
    float *xs = c.take<float>((size_t)N * P);
    float *lam = c.take<float>((size_t)N * P);
    float *nu = c.take<float>(N);
    int *its = c.take<int>(N);
    long long *retry = c.take<long long>(N);
    unsigned long long *mask = c.take<unsigned long long>(N);
    xw.list[0] = c.take<long long>(N);
    xw.list[1] = c.take<long long>(N);
    xw.ksize = c.take<int>(N);
    if (!c.ok) return LINMIN_ERR_INVALID;   // cannot happen after scratch_needed

#define NA_CUDA(call)                                  \
    do {                                               \
        if ((call) != cudaSuccess) return LINMIN_ERR_CUDA; \
    } while (0)
    // the array keeps the previous call's contents: zero the counters/flags
    NA_CUDA(cudaMemsetAsync(pr.flags, 0, sizeof(int), st));
    NA_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), st));
    NA_CUDA(launch_prep(library, sigma, L, P, PP, pr, st));
    NA_CUDA(launch_project(cube, N, L, P, pr.Bhi, pr.Blo, c_hi, c_lo, st));
    linmin_options o;
    linmin_default_options(&o);
    IpmArgs ia;
    ia.N = N; ia.P = P; ia.max_iter = o.max_iter;
    ia.c_hi = c_hi; ia.c_lo = c_lo;
    ia.Ghi = pr.Ghi; ia.Glo = pr.Glo; ia.grs = pr.grs;
    ia.x_state = xs; ia.lam_state = lam; ia.nu_state = nu; ia.it_state = its;
    ia.n_notconv = cnt + 2;
    ia.tol_c = o.tol; ia.tol_d = 1e-6f; ia.eta = 0.99f;
    ia.list = nullptr; ia.list_len = nullptr;
    ia.mu_ref = MU_STOP; ia.counter = cnt + 0;
    NA_CUDA(launch_ipm(b, false, ia, st));
    float *x_out = abundances ? abundances : xs;
    CrossArgs ca{};
    ca.N = N; ca.P = P; ca.Gt64 = pr.Gt64; ca.Ghi = pr.Ghi; ca.Glo = pr.Glo; ca.PP = PP;
    ca.scale = pr.scale; ca.gdiag = pr.gdiag; ca.c_hi = c_hi; ca.c_lo = c_lo;
    ca.x_in = xs; ca.lam_in = lam; ca.x_out = x_out; ca.sx_out = uncertainties; ca.mask = mask;
    ca.retry_list = retry; ca.retry_len = cnt + 5; ca.n_unverified = nullptr;
    ca.tol_x = 1e-9; ca.tol_g = 1e-9;
    NA_CUDA(launch_crossover(ca, xw, nullptr, nullptr, st));
    ia.list = retry; ia.list_len = cnt + 5;
    ia.mu_ref = o.refine_mu; ia.counter = cnt + 1;
    NA_CUDA(launch_ipm(b, false, ia, st));
    ia.counter = cnt + 4;
    NA_CUDA(launch_ipm(b, true, ia, st));
    ca.retry_list = nullptr; ca.retry_len = nullptr; ca.n_unverified = cnt + 2;
    ca.it_mark = its;
    NA_CUDA(launch_crossover(ca, xw, retry, cnt + 5, st));
    if (residual_rms) NA_CUDA(launch_rms(cube, library, x_out, N, L, P, residual_rms, st));
    if (iterations)
        NA_CUDA(cudaMemcpyAsync(iterations, its, (size_t)N * sizeof(int),
                                cudaMemcpyDeviceToDevice, st));
    noalloc_mark_invalid_kernel<<<152 * 4, 256, 0, st>>>(pr.flags, N, P, abundances,
                                                         uncertainties, residual_rms, iterations);
    NA_CUDA(cudaGetLastError());
#undef NA_CUDA
    return LINMIN_OK;
}

linmin_status linmin_noalloc_scratch_bytes(int L, int P, long long N, unsigned long long *bytes)
{
    if (bytes) *bytes = 0;
    Bucket b;
    if (P < 1 || P > LINMIN_MAX_P || !ipm_bucket(P, &b)) return LINMIN_ERR_UNSUPPORTED;
    if (N < 0 || L < P || L > LINMIN_MAX_L) return LINMIN_ERR_INVALID;
    const size_t need = scratch_needed(L, P, b.PP, N);
    if (need == 0) return LINMIN_ERR_INVALID;
    if (bytes) *bytes = need;
    return LINMIN_OK;
}

}  // extern "C"
