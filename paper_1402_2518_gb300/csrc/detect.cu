// Detection products: the paper's additional spectra (Sec. 2.5, Appendix),
// the per-pixel detection conditions (Sec. 5), and the statistics of the
// per-mineral threshold (Sec. 3.1, eq. Threshold).
//
// Both device kernels read the N x P abundance array once: a block stages
// a tile of DT pixels (rows padded to P + 1 floats, so that column reads
// are conflict-free) with coalesced loads, evaluates one pixel per thread
// (the detection mask), then one mineral per thread walks the tile's
// pixels and keeps its sums in registers; one atomic per mineral and block
// at the end.  Memory bound: 4P (x) + 4P (sx) + 16 bytes read and 8 bytes
// written per pixel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "api_internal.h"
#include "linmin.h"

namespace {

constexpr int DT = 64;            // pixels per tile = threads per block
constexpr int DMAX_BLOCKS = 152 * 16;

struct DetectArgs {
    const float *x, *sx, *rms;
    const int *it;
    const unsigned long long *truth;
    long long N;
    int P, nm;
    float rms_max;
    unsigned long long *mask;
    linmin_detection *out;
    float xmin[LINMIN_MAX_P];
};

// Stage rows [n0, n0 + rows) of a N x P float array into s (stride P + 1).
__device__ __forceinline__ void stage_rows(float *s, const float *g, long long n0, int rows,
                                           int P)
{
    const long long base = n0 * P;
    const int ne = rows * P;
    for (int e = threadIdx.x; e < ne; e += DT) {
        const int r = e / P, c = e - r * P;
        s[r * (P + 1) + c] = __ldg(g + base + e);
    }
}

// Order key of a detected abundance (x > 0): larger x first, then the
// smaller pixel index.
__device__ __forceinline__ unsigned long long max_key(float x, long long n)
{
    return ((unsigned long long)__float_as_uint(x) << 32) |
           (unsigned long long)(0xffffffffu - (unsigned)n);
}

__global__ void __launch_bounds__(DT) detect_kernel(DetectArgs a)
{
    extern __shared__ float sm[];
    const int P = a.P, ld = P + 1;
    float *xs = sm;
    float *ss = xs + DT * ld;
    unsigned long long *ms = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(ss + DT * ld) + 7) & ~(uintptr_t)7);
    unsigned long long *ts = ms + DT;

    const int i = threadIdx.x;               // mineral of the column pass
    const bool cols = a.out != nullptr && i < a.nm;
    long long cnt = 0, ntr = 0, tp = 0, fp = 0;
    double xsum = 0.0;
    unsigned long long key = 0;

    const long long tiles = (a.N + DT - 1) / DT;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const long long n0 = t * DT;
        const long long rem = a.N - n0;
        const int rows = rem < DT ? (int)rem : DT;
        stage_rows(xs, a.x, n0, rows, P);
        if (a.sx) stage_rows(ss, a.sx, n0, rows, P);
        __syncthreads();
        // one pixel per thread: the detection mask
        if (threadIdx.x < rows) {
            const int r = threadIdx.x;
            const long long n = n0 + r;
            bool ok = true;
            if (a.rms) ok = __ldg(a.rms + n) < a.rms_max;
            if (a.it) ok = ok && __ldg(a.it + n) >= 0;
            unsigned long long m = 0;
            if (ok) {
                for (int j = 0; j < a.nm; ++j) {
                    const float xv = xs[r * ld + j];
                    bool d = xv > a.xmin[j];
                    if (a.sx) d = d && ss[r * ld + j] < xv;
                    m |= (unsigned long long)d << j;
                }
            }
            ms[r] = m;
            ts[r] = a.truth ? __ldg(a.truth + n) : 0ull;
            if (a.mask) a.mask[n] = m;
        }
        __syncthreads();
        // one mineral per thread: counts, sum, arg-max, rates
        if (cols) {
            for (int r = 0; r < rows; ++r) {
                const bool d = (ms[r] >> i) & 1ull;
                const bool tr = (ts[r] >> i) & 1ull;
                ntr += tr;
                tp += d && tr;
                fp += d && !tr;
                if (d) {
                    const float xv = xs[r * ld + i];
                    ++cnt;
                    xsum += (double)xv;
                    const unsigned long long k = max_key(xv, n0 + r);
                    key = k > key ? k : key;
                }
            }
        }
        __syncthreads();
    }
    if (cols) {
        linmin_detection *o = a.out;
        if (cnt) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&o->count[i]), (unsigned long long)cnt);
            atomicAdd(&o->xsum[i], xsum);
            atomicMax(&o->key[i], key);
        }
        if (a.truth) {
            if (ntr) atomicAdd(reinterpret_cast<unsigned long long *>(&o->n_true[i]), (unsigned long long)ntr);
            if (tp) atomicAdd(reinterpret_cast<unsigned long long *>(&o->true_pos[i]), (unsigned long long)tp);
            if (fp) atomicAdd(reinterpret_cast<unsigned long long *>(&o->false_pos[i]), (unsigned long long)fp);
        }
    }
}

__global__ void detect_finish_kernel(linmin_detection *o, int nm)
{
    const int i = threadIdx.x;
    if (i >= LINMIN_MAX_P) return;
    const unsigned long long k = o->key[i];
    if (i < nm && k) {
        o->xmax[i] = __uint_as_float((unsigned)(k >> 32));
        o->argmax[i] = (long long)(0xffffffffu - (unsigned)(k & 0xffffffffull));
    } else {
        o->xmax[i] = 0.f;
        o->argmax[i] = -1;
    }
}

struct StatsArgs {
    const float *x;
    const unsigned long long *truth;
    long long N;
    int P, nm;
    linmin_threshold_sums *out;
};

__global__ void __launch_bounds__(DT) threshold_stats_kernel(StatsArgs a)
{
    extern __shared__ float sm[];
    const int P = a.P, ld = P + 1;
    float *xs = sm;
    unsigned long long *ts = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(xs + DT * ld) + 7) & ~(uintptr_t)7);
    const int i = threadIdx.x;
    long long np = 0, nn = 0;
    double sp = 0.0, qp = 0.0, sn = 0.0, qn = 0.0;
    const long long tiles = (a.N + DT - 1) / DT;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const long long n0 = t * DT;
        const long long rem = a.N - n0;
        const int rows = rem < DT ? (int)rem : DT;
        stage_rows(xs, a.x, n0, rows, P);
        if (threadIdx.x < rows) ts[threadIdx.x] = __ldg(a.truth + n0 + threadIdx.x);
        __syncthreads();
        if (i < a.nm) {
            for (int r = 0; r < rows; ++r) {
                const double v = (double)xs[r * ld + i];
                if ((ts[r] >> i) & 1ull) { ++np; sp += v; qp += v * v; }
                else                     { ++nn; sn += v; qn += v * v; }
            }
        }
        __syncthreads();
    }
    if (i < a.nm) {
        linmin_threshold_sums *o = a.out;
        if (np) atomicAdd(reinterpret_cast<unsigned long long *>(&o->n_pos[i]), (unsigned long long)np);
        if (nn) atomicAdd(reinterpret_cast<unsigned long long *>(&o->n_neg[i]), (unsigned long long)nn);
        atomicAdd(&o->sum_pos[i], sp);
        atomicAdd(&o->sumsq_pos[i], qp);
        atomicAdd(&o->sum_neg[i], sn);
        atomicAdd(&o->sumsq_neg[i], qn);
    }
}

size_t detect_smem(int P) { return (size_t)2 * DT * (P + 1) * sizeof(float) + 8 + 2 * DT * 8; }
size_t stats_smem(int P) { return (size_t)DT * (P + 1) * sizeof(float) + 8 + DT * 8; }

int grid_for(long long N)
{
    const long long tiles = (N + DT - 1) / DT;
    return (int)std::max<long long>(1, std::min<long long>(tiles, DMAX_BLOCKS));
}

linmin_status err(linmin_status st, const std::string &m)
{
    lm::set_global_error(m);
    return st;
}

linmin_status cuda_err(cudaError_t e, const char *what)
{
    return err(LINMIN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool on_device(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

linmin_status check_sizes(long long N, int P, int nm)
{
    if (P < 1 || P > LINMIN_MAX_P) return err(LINMIN_ERR_INVALID, "P must be in 1..64");
    if (nm < 0 || nm > P) return err(LINMIN_ERR_INVALID, "n_minerals must be in 0..P");
    if (N < 0 || N > 0xffffffffll) return err(LINMIN_ERR_INVALID, "N must be in 0..2^32-1");
    return LINMIN_OK;
}

}  // namespace

extern "C" {

linmin_status linmin_extra_spectra(int L, const float *wavelengths, int n_extras, float *out)
{
    if (L < 2 || !out || (n_extras != 4 && n_extras != 12))
        return err(LINMIN_ERR_INVALID, "linmin_extra_spectra: L >= 2, n_extras 4 or 12, out non-NULL");
    double w0 = 0.0, span = (double)(L - 1);
    if (wavelengths) {
        w0 = wavelengths[0];
        span = (double)wavelengths[L - 1] - w0;
        for (int l = 1; l < L; ++l)
            if (!(wavelengths[l] > wavelengths[l - 1]))
                return err(LINMIN_ERR_INVALID, "linmin_extra_spectra: wavelengths must increase");
    }
    const double pi = 3.14159265358979323846;
    for (int l = 0; l < L; ++l) {
        const double u = ((wavelengths ? (double)wavelengths[l] : (double)l) - w0) / span;
        double v[12];
        v[0] = 1.0;
        v[1] = 1e-4;
        v[2] = u;
        v[3] = 1.0 - u;
        for (int f = 0; f < 2; ++f) {      // f = 0: argument pi u / 2, f = 1: pi u
            const double arg = pi * u * (f ? 1.0 : 0.5);
            const double c = std::cos(arg), s = std::sin(arg);
            v[4 + 4 * f] = c;
            v[5 + 4 * f] = s;
            v[6 + 4 * f] = -c;
            v[7 + 4 * f] = -s;
        }
        for (int k = 0; k < n_extras; ++k) out[(size_t)k * L + l] = (float)v[k];
    }
    return LINMIN_OK;
}

linmin_status linmin_detect(const float *x, const float *sx, const float *rms,
                            const int *iterations, const unsigned long long *truth, long long N,
                            int P, int n_minerals, const float *x_min, float rms_max,
                            unsigned long long *mask, linmin_detection *out, void *stream)
{
    linmin_status st = check_sizes(N, P, n_minerals);
    if (st != LINMIN_OK) return st;
    if (N > 0 && !x) return err(LINMIN_ERR_INVALID, "linmin_detect: x is NULL");
    if (n_minerals > 0 && !x_min) return err(LINMIN_ERR_INVALID, "linmin_detect: x_min is NULL");
    for (int i = 0; i < n_minerals; ++i)
        if (!std::isfinite(x_min[i]) || x_min[i] < 0.f)
            return err(LINMIN_ERR_INVALID, "linmin_detect: x_min must be finite and >= 0");
    if (rms && std::isnan(rms_max)) return err(LINMIN_ERR_INVALID, "linmin_detect: rms_max is NaN");
    const void *ptrs[] = {x, sx, rms, iterations, truth, mask, out};
    for (const void *p : ptrs)
        if (!on_device(p)) return err(LINMIN_ERR_INVALID, "linmin_detect: arrays must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (out && (e = cudaMemsetAsync(out, 0, sizeof(linmin_detection), s)) != cudaSuccess)
        return cuda_err(e, "linmin_detect: memset");
    if (N > 0 && (mask || out)) {
        DetectArgs a;
        a.x = x; a.sx = sx; a.rms = rms; a.it = iterations; a.truth = truth;
        a.N = N; a.P = P; a.nm = n_minerals; a.rms_max = rms_max; a.mask = mask;
        a.out = out;
        for (int i = 0; i < LINMIN_MAX_P; ++i) a.xmin[i] = i < n_minerals ? x_min[i] : 0.f;
        const size_t smem = detect_smem(P);
        detect_kernel<<<grid_for(N), DT, smem, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "linmin_detect: launch");
    }
    if (out) {
        detect_finish_kernel<<<1, LINMIN_MAX_P, 0, s>>>(out, n_minerals);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "linmin_detect: finish");
    }
    return LINMIN_OK;
}

linmin_status linmin_threshold_stats(const float *x, const unsigned long long *truth, long long N,
                                     int P, int n_minerals, linmin_threshold_sums *out,
                                     void *stream)
{
    linmin_status st = check_sizes(N, P, n_minerals);
    if (st != LINMIN_OK) return st;
    if (!out || (N > 0 && (!x || !truth)))
        return err(LINMIN_ERR_INVALID, "linmin_threshold_stats: x, truth and out are required");
    const void *ptrs[] = {x, truth, out};
    for (const void *p : ptrs)
        if (!on_device(p))
            return err(LINMIN_ERR_INVALID, "linmin_threshold_stats: arrays must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(linmin_threshold_sums), s);
    if (e != cudaSuccess) return cuda_err(e, "linmin_threshold_stats: memset");
    if (N > 0 && n_minerals > 0) {
        StatsArgs a{x, truth, N, P, n_minerals, out};
        threshold_stats_kernel<<<grid_for(N), DT, stats_smem(P), s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "linmin_threshold_stats: launch");
    }
    return LINMIN_OK;
}

linmin_status linmin_thresholds(const linmin_threshold_sums *st, int n_minerals, float *c_out)
{
    if (!st || !c_out || n_minerals < 0 || n_minerals > LINMIN_MAX_P)
        return err(LINMIN_ERR_INVALID, "linmin_thresholds: stats and c_out required, 0 <= n_minerals <= 64");
    for (int i = 0; i < n_minerals; ++i) {
        const long long np = st->n_pos[i], nn = st->n_neg[i];
        if (np <= 0 || nn <= 0) { c_out[i] = NAN; continue; }
        const double mp = st->sum_pos[i] / (double)np, mn = st->sum_neg[i] / (double)nn;
        const double vp = std::max(0.0, st->sumsq_pos[i] / (double)np - mp * mp);
        const double vn = std::max(0.0, st->sumsq_neg[i] / (double)nn - mn * mn);
        c_out[i] = (float)(0.5 * (mp - 2.0 * std::sqrt(vp) + mn + 6.0 * std::sqrt(vn)));
    }
    return LINMIN_OK;
}

}  // extern "C"
