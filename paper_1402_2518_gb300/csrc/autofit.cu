// Auto-fit of the reference library (Sec. 2.4, "Estimation of
// degeneracies"): every spectrum S_n is fitted by the P - 1 others,
// S_n = A'.S' + E, once without constraints and once with A' >= 0.
//
// One block per left-out spectrum n, all in fp64 (the library is small:
// P <= 64, L <= 4096):
//   1. the Gram G = S S^T of all spectra, one warp per entry;
//   2. unconstrained: classical Gram-Schmidt with a second
//      orthogonalisation pass (CGS2) over the other spectra, columns kept
//      when their norm after both passes is above 1e-13 of the original
//      (exactly dependent spectra add nothing to the span); the residue is
//      S_n minus its projection on the kept columns, projected out twice;
//   3. non-negative: the active-set method of Lawson and Hanson on the
//      normal equations (gradient w = b - G' x with b_j = <S_j, S_n>):
//      move the most positive gradient into the passive set, solve the
//      passive least squares by Cholesky (one warp), step back to the
//      feasible region when a passive coefficient is not positive; a
//      spectrum whose passive Cholesky pivot falls below 1e-14 of its
//      diagonal (numerically dependent on the passive ones) is left out;
//      the residue is S_n - sum_j x_j S_j.
// The basis of step 2 lives in a device scratch of P x P x L doubles.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "api_internal.h"
#include "linmin.h"

namespace {

constexpr int AT = 256, AW = AT / 32;
constexpr unsigned FULL = 0xffffffffu;

struct AfArgs {
    const float *S;
    int L, P;
    double *q;
    float *rls, *rnn, *cnn, *rmsl, *rmsn;
    int *status;
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Sum of v over the block (every thread gets it).
__device__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < AW; ++k) s += red[k];
    return s;
}

// Two passes of v -= Q (Q^T v) over the kept columns (v in shared memory).
__device__ void cgs2(double *v, const double *Q, int kept, int L, double *h)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int pass = 0; pass < 2; ++pass) {
        for (int k = warp; k < kept; k += AW) {
            double s = 0.0;
            for (int l = lane; l < L; l += 32) s += Q[(size_t)k * L + l] * v[l];
            s = warp_sum(s);
            if (lane == 0) h[k] = s;
        }
        __syncthreads();
        for (int l = threadIdx.x; l < L; l += AT) {
            double t = v[l];
            for (int k = 0; k < kept; ++k) t -= h[k] * Q[(size_t)k * L + l];
            v[l] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(AT) autofit_kernel(AfArgs a)
{
    extern __shared__ double sh[];
    __shared__ double red[AW];
    __shared__ int s_status;
    const int P = a.P, L = a.L, n = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *G = sh;                  // P x P
    double *C = G + P * P;           // P x P, Cholesky factor of the passive block
    double *b = C + P * P;           // P
    double *x = b + P;               // P
    double *z = x + P;               // P
    double *h = z + P;               // P
    double *v = h + P;               // L
    int *inP = reinterpret_cast<int *>(v + L);    // P
    int *idx = inP + P;                           // P
    const float *S = a.S;

    // 1. Gram
    const int ne = P * (P + 1) / 2;
    for (int e = warp; e < ne; e += AW) {
        int i = 0, rem = e;
        while (rem >= P - i) { rem -= P - i; ++i; }
        const int j = i + rem;
        double s = 0.0;
        for (int l = lane; l < L; l += 32)
            s += (double)S[(size_t)i * L + l] * (double)S[(size_t)j * L + l];
        s = warp_sum(s);
        if (lane == 0) { G[i * P + j] = s; G[j * P + i] = s; }
    }
    __syncthreads();

    // 2. unconstrained residue
    double *Q = a.q + (size_t)n * P * L;
    int kept = 0;
    for (int j = 0; j < P; ++j) {
        if (j == n) continue;
        for (int l = threadIdx.x; l < L; l += AT) v[l] = (double)S[(size_t)j * L + l];
        __syncthreads();
        cgs2(v, Q, kept, L, h);
        double t = 0.0;
        for (int l = threadIdx.x; l < L; l += AT) t += v[l] * v[l];
        const double nv = sqrt(block_sum(t, red));
        if (nv > 1e-13 * sqrt(G[j * P + j])) {
            const double inv = 1.0 / nv;
            for (int l = threadIdx.x; l < L; l += AT) Q[(size_t)kept * L + l] = v[l] * inv;
            ++kept;
        }
        __syncthreads();
    }
    for (int l = threadIdx.x; l < L; l += AT) v[l] = (double)S[(size_t)n * L + l];
    __syncthreads();
    cgs2(v, Q, kept, L, h);
    {
        double t = 0.0;
        for (int l = threadIdx.x; l < L; l += AT) {
            t += v[l] * v[l];
            if (a.rls) a.rls[(size_t)n * L + l] = (float)v[l];
        }
        const double ss = block_sum(t, red);
        if (a.rmsl && threadIdx.x == 0) a.rmsl[n] = (float)sqrt(ss / L);
    }

    // 3. non-negative least squares (Lawson-Hanson), warp 0
    if (warp == 0) {
        double gmax = 0.0;
        for (int j = lane; j < P; j += 32) {
            x[j] = 0.0;
            inP[j] = 0;
            b[j] = j == n ? 0.0 : G[j * P + n];
            gmax = fmax(gmax, G[j * P + j]);
        }
        for (int o = 16; o; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(FULL, gmax, o));
        const double tol = 1e-12 * gmax;
        int status = 1;                      // iteration cap unless it converges
        unsigned long long barred = 1ull << n;   // never enter the passive set
        __syncwarp();
        for (int outer = 0; outer < 3 * LINMIN_MAX_P; ++outer) {
            // gradient and its largest entry outside the passive set
            double best = -1.0;
            int bj = -1;
            for (int j = lane; j < P; j += 32) {
                double g = b[j];
                for (int k = 0; k < P; ++k) g -= G[j * P + k] * x[k];
                if (!inP[j] && !((barred >> j) & 1ull) && g > best) { best = g; bj = j; }
            }
            for (int o = 16; o; o >>= 1) {
                const double ob = __shfl_xor_sync(FULL, best, o);
                const int oj = __shfl_xor_sync(FULL, bj, o);
                if (ob > best || (ob == best && oj >= 0 && (bj < 0 || oj < bj))) { best = ob; bj = oj; }
            }
            if (bj < 0 || best <= tol) { status = 0; break; }
            if (lane == 0) inP[bj] = 1;
            __syncwarp();
            bool fail = false;
            for (int inner = 0; inner <= P; ++inner) {
                // passive list
                int m = 0;
                for (int j = 0; j < P; ++j)
                    if (inP[j]) { if (lane == 0) idx[m] = j; ++m; }
                __syncwarp();
                for (int e = lane; e < m * m; e += 32) {
                    const int r = e / m, c = e - r * m;
                    C[r * P + c] = G[idx[r] * P + idx[c]];
                }
                __syncwarp();
                // Cholesky (lower), one warp
                for (int k = 0; k < m && !fail; ++k) {
                    const double d = C[k * P + k];
                    const bool ok = d > 1e-14 * G[idx[k] * P + idx[k]];
                    if (!ok) { fail = true; break; }
                    const double dk = sqrt(d);
                    __syncwarp();
                    if (lane == 0) C[k * P + k] = dk;
                    for (int r = k + 1 + lane; r < m; r += 32) C[r * P + k] /= dk;
                    __syncwarp();
                    for (int r = k + 1 + lane; r < m; r += 32) {
                        const double lr = C[r * P + k];
                        for (int c = k + 1; c <= r; ++c) C[r * P + c] -= lr * C[c * P + k];
                    }
                    __syncwarp();
                }
                if (fail) {
                    // the entering spectrum is numerically dependent on the
                    // passive ones (only the first solve can fail: later
                    // passive sets are subsets of a factorable one): bar it
                    __syncwarp();
                    if (lane == 0) inP[bj] = 0;
                    barred |= 1ull << bj;
                    __syncwarp();
                    break;
                }
                if (lane == 0) {
                    for (int r = 0; r < m; ++r) {          // L y = b_P
                        double s = b[idx[r]];
                        for (int c = 0; c < r; ++c) s -= C[r * P + c] * z[c];
                        z[r] = s / C[r * P + r];
                    }
                    for (int r = m - 1; r >= 0; --r) {     // L^T z = y
                        double s = z[r];
                        for (int c = r + 1; c < m; ++c) s -= C[c * P + r] * z[c];
                        z[r] = s / C[r * P + r];
                    }
                }
                __syncwarp();
                // feasible: accept; else step back to the boundary, where
                // the coordinate with the smallest step leaves the passive set
                bool pos = true;
                double alpha = 2.0;
                int rmin = -1;
                for (int r = 0; r < m; ++r) {
                    if (z[r] <= 0.0) {
                        pos = false;
                        const double xj = x[idx[r]], den = xj - z[r];
                        const double t = den > 0.0 ? xj / den : 0.0;
                        if (rmin < 0 || t < alpha) { alpha = t; rmin = r; }
                    }
                }
                if (pos) {
                    __syncwarp();
                    for (int r = lane; r < m; r += 32) x[idx[r]] = z[r];
                    __syncwarp();
                    break;
                }
                if (inner == 0 && idx[rmin] == bj) {
                    // rounding left the entering coordinate non-positive: bar it
                    __syncwarp();
                    if (lane == 0) inP[bj] = 0;
                    barred |= 1ull << bj;
                    __syncwarp();
                    break;
                }
                __syncwarp();
                for (int r = lane; r < m; r += 32) {
                    const int j = idx[r];
                    x[j] += alpha * (z[r] - x[j]);
                }
                __syncwarp();
                if (lane == 0) {
                    const int jm = idx[rmin];
                    x[jm] = 0.0;
                    inP[jm] = 0;
                    for (int r = 0; r < m; ++r)
                        if (x[idx[r]] <= 0.0) { x[idx[r]] = 0.0; inP[idx[r]] = 0; }
                }
                __syncwarp();
            }

        }
        if (lane == 0) s_status = status;
    }
    __syncthreads();
    {
        double t = 0.0;
        for (int l = threadIdx.x; l < L; l += AT) {
            double r = (double)S[(size_t)n * L + l];
            for (int j = 0; j < P; ++j)
                if (x[j] != 0.0) r -= x[j] * (double)S[(size_t)j * L + l];
            t += r * r;
            if (a.rnn) a.rnn[(size_t)n * L + l] = (float)r;
        }
        const double ss = block_sum(t, red);
        if (threadIdx.x == 0) {
            if (a.rmsn) a.rmsn[n] = (float)sqrt(ss / L);
            if (a.status) a.status[n] = s_status;
        }
        if (a.cnn)
            for (int j = threadIdx.x; j < P; j += AT) a.cnn[(size_t)n * P + j] = (float)x[j];
    }
}

size_t af_smem(int P, int L)
{
    return ((size_t)2 * P * P + 5 * P + L) * sizeof(double) + (size_t)2 * P * sizeof(int);
}

bool dev_or_null(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

linmin_status af_err(linmin_status st, const std::string &m)
{
    lm::set_global_error(m);
    return st;
}

}  // namespace

extern "C" linmin_status linmin_autofit(const float *library, int L, int P, float *resid_ls,
                                        float *resid_nn, float *coef_nn, float *rms_ls,
                                        float *rms_nn, int *status, void *stream)
{
    if (P < 2 || P > LINMIN_MAX_P || L < P || L > LINMIN_MAX_L)
        return af_err(LINMIN_ERR_INVALID, "linmin_autofit: 2 <= P <= 64 and P <= L <= 4096");
    if (!library) return af_err(LINMIN_ERR_INVALID, "linmin_autofit: library is NULL");
    const void *ptrs[] = {library, resid_ls, resid_nn, coef_nn, rms_ls, rms_nn, status};
    for (const void *p : ptrs)
        if (!dev_or_null(p))
            return af_err(LINMIN_ERR_INVALID, "linmin_autofit: arrays must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t smem = af_smem(P, L);
    cudaError_t e = cudaFuncSetAttribute(autofit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return af_err(LINMIN_ERR_CUDA, std::string("linmin_autofit: ") + cudaGetErrorString(e));
    double *q = nullptr;
    e = lm::injected_alloc_failure() == 1
            ? cudaErrorMemoryAllocation
            : cudaMallocAsync(&q, (size_t)P * P * L * sizeof(double), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return af_err(e == cudaErrorMemoryAllocation ? LINMIN_ERR_OOM : LINMIN_ERR_CUDA,
                      std::string("linmin_autofit: scratch: ") + cudaGetErrorString(e));
    }
    AfArgs a{library, L, P, q, resid_ls, resid_nn, coef_nn, rms_ls, rms_nn, status};
    autofit_kernel<<<P, AT, smem, s>>>(a);
    e = cudaGetLastError();
    cudaFreeAsync(q, s);
    if (e != cudaSuccess)
        return af_err(LINMIN_ERR_CUDA, std::string("linmin_autofit: launch: ") + cudaGetErrorString(e));
    return LINMIN_OK;
}
