// Detection products: the paper's additional spectra (Sec. 2.5, Appendix),
// the per-pixel detection conditions (Sec. 4, introduction), and the statistics of the
// per-mineral threshold (Sec. 3.1, eq. Threshold).
//
// Both device kernels stream the N x P abundance array once with the lane
// of a warp as the mineral: a warp walks a contiguous range of pixels,
// lane i reads x[n, i] (and x[n, i + 32]; a pixel's row is one coalesced
// read), decides mineral i, and a warp ballot gives the pixel's detection
// mask; each lane keeps its mineral's counts, sum and arg-max in registers
// over the whole range; the block sums its warps in shared memory and
// issues one atomic per mineral and block.
// Memory bound: 4P (x) + 4P (sx) + 16 bytes read and 8 bytes written per
// pixel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "api_internal.h"
#include "linmin.h"

namespace {

constexpr int DTH = 256;                 // threads per block
constexpr int DBLOCKS = 152 * 4;         // blocks (8 warps each)
constexpr int DU = 8;                    // pixels per warp step (loads in flight)
constexpr unsigned FULLM = 0xffffffffu;

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

// Order key of a detected abundance (x > 0): larger x first, then the
// smaller pixel index.
__device__ __forceinline__ unsigned long long max_key(float x, long long n)
{
    return ((unsigned long long)__float_as_uint(x) << 32) |
           (unsigned long long)(0xffffffffu - (unsigned)n);
}

// Contiguous pixel range of this warp.
__device__ __forceinline__ void warp_range(long long N, long long &n0, long long &n1)
{
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long per = (N + nw - 1) / nw;
    n0 = w * per;
    n1 = n0 + per < N ? n0 + per : N;
}

struct MinAcc {
    int cnt = 0, ntr = 0, tp = 0, fp = 0;    // per warp range: < 2^31 pixels
    double xsum = 0.0;
    unsigned long long key = 0;
};

// TWO: minerals 32..63 exist (n_minerals > 32), the lane owns two.
template <bool TWO>
__global__ void __launch_bounds__(DTH) detect_kernel(DetectArgs a)
{
    const int lane = threadIdx.x & 31;
    const int P = a.P, nm = a.nm;
    const int i0 = lane, i1 = lane + 32;
    const bool has0 = i0 < nm, has1 = TWO && i1 < nm;
    const float xm0 = has0 ? a.xmin[i0] : 0.f, xm1 = has1 ? a.xmin[i1] : 0.f;
    MinAcc m0, m1;
    long long n0, n1;
    warp_range(a.N, n0, n1);
    for (long long nb = n0; nb < n1; nb += DU) {
        float xv0[DU], xv1[TWO ? DU : 1], sv0[DU], sv1[TWO ? DU : 1];
        bool ok[DU];
        unsigned long long tr[DU];
#pragma unroll
        for (int u = 0; u < DU; ++u) {
            const long long n = nb + u;
            const bool in = n < n1;
            const float *xr = a.x + n * P;
            xv0[u] = in && has0 ? __ldg(xr + i0) : 0.f;
            if (TWO) xv1[u] = in && has1 ? __ldg(xr + i1) : 0.f;
            if (a.sx) {
                const float *sr = a.sx + n * P;
                sv0[u] = in && has0 ? __ldg(sr + i0) : 0.f;
                if (TWO) sv1[u] = in && has1 ? __ldg(sr + i1) : 0.f;
            }
            bool o = in;
            if (in && a.rms) o = __ldg(a.rms + n) < a.rms_max;
            if (in && a.it) o = o && __ldg(a.it + n) >= 0;
            ok[u] = o;
            tr[u] = in && a.truth ? __ldg(a.truth + n) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < DU; ++u) {
            const long long n = nb + u;
            bool d0 = ok[u] && has0 && xv0[u] > xm0;
            bool d1 = TWO && ok[u] && has1 && xv1[TWO ? u : 0] > xm1;
            if (a.sx) {
                d0 = d0 && sv0[u] < xv0[u];
                if (TWO) d1 = d1 && sv1[TWO ? u : 0] < xv1[TWO ? u : 0];
            }
            const unsigned b0 = __ballot_sync(FULLM, d0);
            const unsigned b1 = TWO ? __ballot_sync(FULLM, d1) : 0u;
            if (n >= n1) continue;
            if (lane == 0 && a.mask) a.mask[n] = (unsigned long long)b0 | ((unsigned long long)b1 << 32);
            const bool t0 = (tr[u] >> i0) & 1ull, t1 = i1 < 64 && ((tr[u] >> i1) & 1ull);
            if (has0) {
                m0.ntr += t0; m0.tp += d0 && t0; m0.fp += d0 && !t0;
                if (d0) {
                    ++m0.cnt; m0.xsum += (double)xv0[u];
                    const unsigned long long k = max_key(xv0[u], n);
                    m0.key = k > m0.key ? k : m0.key;
                }
            }
            if (TWO && has1) {
                m1.ntr += t1; m1.tp += d1 && t1; m1.fp += d1 && !t1;
                if (d1) {
                    ++m1.cnt; m1.xsum += (double)xv1[TWO ? u : 0];
                    const unsigned long long k = max_key(xv1[TWO ? u : 0], n);
                    m1.key = k > m1.key ? k : m1.key;
                }
            }
        }
    }
    if (!a.out) return;
    // block reduction of the warps' sums (one atomic per mineral and block:
    // same-address atomics from every warp serialise in L2)
    __shared__ int s_cnt[DTH / 32][LINMIN_MAX_P], s_ntr[DTH / 32][LINMIN_MAX_P];
    __shared__ int s_tp[DTH / 32][LINMIN_MAX_P], s_fp[DTH / 32][LINMIN_MAX_P];
    __shared__ double s_sum[DTH / 32][LINMIN_MAX_P];
    __shared__ unsigned long long s_key[DTH / 32][LINMIN_MAX_P];
    const int w = threadIdx.x >> 5;
    for (int h = 0; h < 2; ++h) {
        const MinAcc &m = h ? m1 : m0;
        const int i = lane + 32 * h;
        const bool own = h == 0 || TWO;
        s_cnt[w][i] = own ? m.cnt : 0;
        s_ntr[w][i] = own ? m.ntr : 0;
        s_tp[w][i] = own ? m.tp : 0;
        s_fp[w][i] = own ? m.fp : 0;
        s_sum[w][i] = own ? m.xsum : 0.0;
        s_key[w][i] = own ? m.key : 0ull;
    }
    __syncthreads();
    const int i = threadIdx.x;
    if (i >= nm) return;
    long long cnt = 0, ntr = 0, tp = 0, fp = 0;
    double xsum = 0.0;
    unsigned long long key = 0;
    for (int q = 0; q < DTH / 32; ++q) {
        cnt += s_cnt[q][i]; ntr += s_ntr[q][i]; tp += s_tp[q][i]; fp += s_fp[q][i];
        xsum += s_sum[q][i];
        key = s_key[q][i] > key ? s_key[q][i] : key;
    }
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
    int pass;          // 0: counts and sums; 1: squared deviations from the pass-0 means
};

__global__ void __launch_bounds__(DTH) threshold_stats_kernel(StatsArgs a)
{
    const int lane = threadIdx.x & 31;
    const int P = a.P, nm = a.nm;
    long long np[2] = {0, 0}, nn[2] = {0, 0};
    double sp[2] = {0.0, 0.0}, qp[2] = {0.0, 0.0}, sn[2] = {0.0, 0.0}, qn[2] = {0.0, 0.0};
    // pass 1: the means of pass 0 (complete: same stream), subtracted
    // before squaring, so the variance has no cancellation
    double mp[2] = {0.0, 0.0}, mn[2] = {0.0, 0.0};
    if (a.pass == 1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = lane + 32 * h;
            if (i >= nm) continue;
            const long long cp = a.out->n_pos[i], cn = a.out->n_neg[i];
            mp[h] = cp ? a.out->sum_pos[i] / (double)cp : 0.0;
            mn[h] = cn ? a.out->sum_neg[i] / (double)cn : 0.0;
        }
    }
    long long n0, n1;
    warp_range(a.N, n0, n1);
    for (long long n = n0; n < n1; ++n) {
        const unsigned long long t = __ldg(a.truth + n);
        const float *xr = a.x + n * P;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = lane + 32 * h;
            if (i >= nm) continue;
            const double v = (double)__ldg(xr + i);
            if ((t >> i) & 1ull) {
                ++np[h];
                if (a.pass == 0) sp[h] += v;
                else qp[h] += (v - mp[h]) * (v - mp[h]);
            } else {
                ++nn[h];
                if (a.pass == 0) sn[h] += v;
                else qn[h] += (v - mn[h]) * (v - mn[h]);
            }
        }
    }
    __shared__ long long s_np[DTH / 32][LINMIN_MAX_P], s_nn[DTH / 32][LINMIN_MAX_P];
    __shared__ double s_sp[DTH / 32][LINMIN_MAX_P], s_qp[DTH / 32][LINMIN_MAX_P];
    __shared__ double s_sn[DTH / 32][LINMIN_MAX_P], s_qn[DTH / 32][LINMIN_MAX_P];
    const int w = threadIdx.x >> 5;
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        s_np[w][i] = np[h]; s_nn[w][i] = nn[h];
        s_sp[w][i] = sp[h]; s_qp[w][i] = qp[h]; s_sn[w][i] = sn[h]; s_qn[w][i] = qn[h];
    }
    __syncthreads();
    const int i = threadIdx.x;
    if (i >= nm) return;
    long long tnp = 0, tnn = 0;
    double tsp = 0.0, tqp = 0.0, tsn = 0.0, tqn = 0.0;
    for (int q = 0; q < DTH / 32; ++q) {
        tnp += s_np[q][i]; tnn += s_nn[q][i];
        tsp += s_sp[q][i]; tqp += s_qp[q][i]; tsn += s_sn[q][i]; tqn += s_qn[q][i];
    }
    linmin_threshold_sums *o = a.out;
    if (a.pass == 0) {
        if (tnp) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&o->n_pos[i]), (unsigned long long)tnp);
            atomicAdd(&o->sum_pos[i], tsp);
        }
        if (tnn) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&o->n_neg[i]), (unsigned long long)tnn);
            atomicAdd(&o->sum_neg[i], tsn);
        }
    } else {
        if (tnp) atomicAdd(&o->m2_pos[i], tqp);
        if (tnn) atomicAdd(&o->m2_neg[i], tqn);
    }
}

int grid_for(long long N)
{
    const long long warps = (N + 15) / 16;            // at least 16 pixels per warp
    const long long b = (warps + DTH / 32 - 1) / (DTH / 32);
    return (int)std::max<long long>(1, std::min<long long>(b, DBLOCKS));
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
        if (n_minerals > 32)
            detect_kernel<true><<<grid_for(N), DTH, 0, s>>>(a);
        else
            detect_kernel<false><<<grid_for(N), DTH, 0, s>>>(a);
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
        for (int pass = 0; pass < 2; ++pass) {
            StatsArgs a{x, truth, N, P, n_minerals, out, pass};
            threshold_stats_kernel<<<grid_for(N), DTH, 0, s>>>(a);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return cuda_err(e, "linmin_threshold_stats: launch");
        }
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
        const double vp = std::max(0.0, st->m2_pos[i] / (double)np);
        const double vn = std::max(0.0, st->m2_neg[i] / (double)nn);
        c_out[i] = (float)(0.5 * (mp - 2.0 * std::sqrt(vp) + mn + 6.0 * std::sqrt(vn)));
    }
    return LINMIN_OK;
}

}  // extern "C"
