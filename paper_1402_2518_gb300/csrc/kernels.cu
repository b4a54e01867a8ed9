// Library preparation, projection, support refinement and RMS kernels.
//
//   prep     Sec. 2.3: whitening W = diag(1/sigma); G = S W^2 S^T in fp64,
//            its scale s = trace(G)/P, G~ = G/s + rho 1 1^T (fp64 and hi+lo
//            float32), B~ = W^2 S^T / s (hi+lo float32).
//   project  c~ = B~^T y + rho for every pixel, accumulated in double-float
//            (Dot2) so that c~ keeps ~48 bits: the FCLS minimiser moves by
//            up to 1e-2 when c~ is merely rounded to float32 on these
//            libraries (constrained condition numbers up to ~1e6).
//   refine   fp64 active-set crossover from the interior-point iterate:
//            x_S from [[G~_SS, 1],[1^T, 0]] [x_S; nu] = [c~_S; 1] on a
//            support S, with swaps until the KKT conditions hold; the
//            abundance uncertainty (Sec. 2.3, "error from the Hessian") is
//            the square root of the diagonal of the top-left block of the
//            inverse of that bordered matrix, divided by s.
//   rms      sqrt(mean_l (y_l - sum_j x_j S_jl)^2), unwhitened.
#include "common.cuh"
#include "ipm.cuh"
#include "kernels.cuh"

namespace lm {

// ------------------------------------------------------------------ prep
__global__ void prep_gram_kernel(const float *__restrict__ S, const float *__restrict__ sigma,
                                 int L, int P, double *__restrict__ G64, int *flags)
{
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int npairs = P * (P + 1) / 2;
    if (wid >= npairs) return;
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= wid) ++i;
    const int j = wid - i * (i + 1) / 2;
    double acc = 0.0;
    bool bad = false;
    for (int l = lane; l < L; l += 32) {
        const double sg = (double)sigma[l];
        if (!(sg > 0.0) || !isfinite(sg)) bad = true;
        const double w2 = 1.0 / (sg * sg);
        acc += ((double)S[(size_t)i * L + l] * (double)S[(size_t)j * L + l]) * w2;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, 1);
    if (lane == 0) {
        G64[(size_t)i * P + j] = acc;
        G64[(size_t)j * P + i] = acc;
    }
}

__global__ void prep_finish_kernel(int P, int PP, const double *__restrict__ G64,
                                   double *__restrict__ Gt64, double *__restrict__ scale,
                                   float *__restrict__ Ghi, float *__restrict__ Glo,
                                   float *__restrict__ grs, float *__restrict__ gdiag, int *flags,
                                   int slack_idx, float slack_x0)
{
    const double x0o = slack_idx >= 0 ? (1.0 - (double)slack_x0) / (P - 1) : 1.0 / P;
    __shared__ double s_sh;
    if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int i = 0; i < P; ++i) tr += G64[(size_t)i * P + i];
        double s = tr / P;
        if (!(s > 0.0) || !isfinite(s)) { atomicOr(flags, 2); s = 1.0; }
        s_sh = s;
        scale[0] = s;
    }
    __syncthreads();
    const double s = s_sh;
    for (int e = threadIdx.x; e < PP * PP; e += blockDim.x) {
        const int i = e / PP, j = e % PP;
        double v = 0.0;
        if (i < P && j < P) {
            v = G64[(size_t)i * P + j] / s + RHO;
            Gt64[(size_t)i * P + j] = v;
        }
        const df d = split_double(v);
        Ghi[e] = d.hi;
        Glo[e] = d.lo;
    }
    for (int i = threadIdx.x; i < PP; i += blockDim.x) {
        double r = 0.0;
        if (i < P) {
            for (int j = 0; j < P; ++j)
                r += (G64[(size_t)i * P + j] / s + RHO) * (j == slack_idx ? (double)slack_x0 : x0o);
            // curvature of the support test; a zero spectrum (the slack of
            // the sum <= 1 constraint) has none: unit curvature there
            const double gi = G64[(size_t)i * P + i] / s;
            gdiag[i] = gi > 0.0 ? (float)gi : 1.f;
        }
        grs[i] = (float)r;
    }
}

__global__ void prep_b_kernel(const float *__restrict__ S, const float *__restrict__ sigma,
                              int L, int P, int PQ, const double *__restrict__ scale,
                              float *__restrict__ Bhi, float *__restrict__ Blo)
{
    const double s = scale[0];
    const long long total = (long long)L * PQ;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(e / PQ), j = (int)(e % PQ);
        double v = 0.0;
        if (j < P) {
            const double sg = (double)sigma[l];
            v = (double)S[(size_t)j * L + l] / (sg * sg * s);
        }
        const df d = split_double(v);
        Bhi[e] = d.hi;
        Blo[e] = d.lo;
    }
}

cudaError_t launch_prep(const float *S, const float *sigma, int L, int P, int PP,
                        const Prep &o, cudaStream_t st)
{
    const int npairs = P * (P + 1) / 2;
    const int threads = 256, wpb = threads / 32;
    prep_gram_kernel<<<(npairs + wpb - 1) / wpb, threads, 0, st>>>(S, sigma, L, P, o.G64, o.flags);
    prep_finish_kernel<<<1, 256, 0, st>>>(P, PP, o.G64, o.Gt64, o.scale, o.Ghi, o.Glo,
                                          o.grs, o.gdiag, o.flags, o.slack_idx, o.slack_x0);
    const int PQ = pq_of(P);
    const long long total = (long long)L * PQ;
    const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
    prep_b_kernel<<<blocks, 256, 0, st>>>(S, sigma, L, P, PQ, o.scale, o.Bhi, o.Blo);
    return cudaGetLastError();
}

// --------------------------------------------------- prep, full covariance
// Sec. 2.3 with a full noise covariance C: the whitened Gram is
// G = S C^-1 S^T and the projection operator B = C^-1 S^T (fp64).
// T = C^-1 S^T (L x P, row-major [l][j]): thread per entry.
__global__ void prep_t_kernel(const float *__restrict__ S, const double *__restrict__ Cinv,
                              int L, int P, double *__restrict__ T)
{
    const long long total = (long long)L * P;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(e / P), j = (int)(e % P);
        const double *crow = Cinv + (size_t)l * L;
        const float *srow = S + (size_t)j * L;
        double acc = 0.0;
        for (int m = 0; m < L; ++m) acc = fma(crow[m], (double)srow[m], acc);
        T[e] = acc;
    }
}

// G_ij = sum_l S_il T_lj: warp per pair of the lower triangle
__global__ void prep_gram_cov_kernel(const float *__restrict__ S, const double *__restrict__ T,
                                     int L, int P, double *__restrict__ G64)
{
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int npairs = P * (P + 1) / 2;
    if (wid >= npairs) return;
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= wid) ++i;
    const int j = wid - i * (i + 1) / 2;
    double acc = 0.0;
    for (int l = lane; l < L; l += 32) acc = fma((double)S[(size_t)i * L + l], T[(size_t)l * P + j], acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        G64[(size_t)i * P + j] = acc;
        G64[(size_t)j * P + i] = acc;
    }
}

// B~ = T / s as hi + lo float32, [l][j] padded to PQ columns
__global__ void prep_b_cov_kernel(const double *__restrict__ T, int L, int P, int PQ,
                                  const double *__restrict__ scale, float *__restrict__ Bhi,
                                  float *__restrict__ Blo)
{
    const double s = scale[0];
    const long long total = (long long)L * PQ;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(e / PQ), j = (int)(e % PQ);
        const df d = split_double(j < P ? T[(size_t)l * P + j] / s : 0.0);
        Bhi[e] = d.hi;
        Blo[e] = d.lo;
    }
}

// Outputs of the slo / pos constraint sets: the internal problem has the
// slack as coordinate P (last); user x = M x', sx = M sx' for the first P
// coordinates; with bound_check (pos), a pixel whose slack is zero reached
// the bound M: negative iteration count, counted as not converged.
__global__ void strip_slack_kernel(const float *__restrict__ xa, const float *__restrict__ sxa,
                                   long long N, int P, float M, bool bound_check,
                                   float *__restrict__ x, float *__restrict__ sx,
                                   int *__restrict__ it, unsigned long long *__restrict__ nbad)
{
    const long long total = N * (long long)P;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long n = e / P;
        const int j = (int)(e % P);
        const size_t src = (size_t)n * (P + 1) + j;
        if (x) x[e] = M * xa[src];
        if (sx) sx[e] = M * sxa[src];
        if (bound_check && j == 0 && !(xa[(size_t)n * (P + 1) + P] > 0.f)) {
            if (it) it[n] = -abs(it[n]) - 1;
            atomicAdd(nbad, 1ULL);
        }
    }
}

// A warp walks a contiguous range of pixels, lane j holds columns j and
// j + 32 of the pixel's c~ row (coalesced row reads and writes).
__global__ void exclude_kernel(const unsigned long long *__restrict__ mask, int n_minerals,
                               float *c_hi, float *c_lo, long long N, int P)
{
    const unsigned long long keep =
        n_minerals >= 64 ? ~0ull : ((1ull << n_minerals) - 1ull);
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long per = (N + nw - 1) / nw;
    const long long n0 = w * per, n1 = n0 + per < N ? n0 + per : N;
    for (long long n = n0; n < n1; ++n) {
        const unsigned long long drop = keep & ~__ldg(mask + n);
        if (!drop) continue;                            // warp-uniform
        float *hi = c_hi + n * P;
        float *lo = c_lo + n * P;
        const int j0 = lane, j1 = lane + 32;
        const float h0 = j0 < P ? hi[j0] : 0.f, l0 = j0 < P ? lo[j0] : 0.f;
        const float h1 = j1 < P ? hi[j1] : 0.f, l1 = j1 < P ? lo[j1] : 0.f;
        float cmax = fmaxf(fabsf(h0 + l0), fabsf(h1 + l1));
        for (int off = 16; off; off >>= 1) cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
        const float K = 2.f * (cmax + (float)P + (float)RHO) + 1.f;
        if ((drop >> j0) & 1ull) {
            const df r = df_add(df{h0, l0}, df_make(-K));
            hi[j0] = r.hi;
            lo[j0] = r.lo;
        }
        if (j1 < 64 && ((drop >> j1) & 1ull)) {
            const df r = df_add(df{h1, l1}, df_make(-K));
            hi[j1] = r.hi;
            lo[j1] = r.lo;
        }
    }
}

cudaError_t launch_exclude(const unsigned long long *mask, int n_minerals, float *c_hi,
                           float *c_lo, long long N, int P, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    const long long warps = (N + 7) / 8;                // at least 8 pixels per warp
    const long long b = (warps + 7) / 8;
    exclude_kernel<<<(int)(b < 152 * 8 ? b : 152 * 8), 256, 0, st>>>(mask, n_minerals, c_hi, c_lo,
                                                                     N, P);
    return cudaGetLastError();
}

cudaError_t launch_strip_slack(const float *xa, const float *sxa, long long N, int P, float M,
                               bool bound_check, float *x, float *sx, int *it,
                               unsigned long long *nbad, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    const long long total = N * (long long)P;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    strip_slack_kernel<<<blocks, 256, 0, st>>>(xa, sxa, N, P, M, bound_check, x, sx, it, nbad);
    return cudaGetLastError();
}

cudaError_t launch_prep_cov(const float *S, const double *Cinv, int L, int P, int PP,
                            const Prep &o, double *T, cudaStream_t st)
{
    const long long lp = (long long)L * P;
    const int tb = (int)((lp + 255) / 256 < 1024 ? (lp + 255) / 256 : 1024);
    prep_t_kernel<<<tb, 256, 0, st>>>(S, Cinv, L, P, T);
    const int npairs = P * (P + 1) / 2;
    const int threads = 256, wpb = threads / 32;
    prep_gram_cov_kernel<<<(npairs + wpb - 1) / wpb, threads, 0, st>>>(S, T, L, P, o.G64);
    prep_finish_kernel<<<1, 256, 0, st>>>(P, PP, o.G64, o.Gt64, o.scale, o.Ghi, o.Glo,
                                          o.grs, o.gdiag, o.flags, o.slack_idx, o.slack_x0);
    const int PQ = pq_of(P);
    const long long total = (long long)L * PQ;
    const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
    prep_b_cov_kernel<<<blocks, 256, 0, st>>>(T, L, P, PQ, o.scale, o.Bhi, o.Blo);
    return cudaGetLastError();
}

// ------------------------------------------------------------ projection
constexpr int PROJ_THREADS = 128;

// Grid-stride over pixels (a persistent grid: B~ is staged in shared memory
// once per block).  Four bands per step: one 16-byte load of the pixel's
// row when rows are 16-byte aligned (vec), else four scalar loads.
template <int NJ4>
__global__ void __launch_bounds__(PROJ_THREADS)
project_kernel(const float *__restrict__ cube, long long N, int L, int P,
               const float *__restrict__ Bhi, const float *__restrict__ Blo,
               float *__restrict__ c_hi, float *__restrict__ c_lo, bool vec)
{
    constexpr int PQ = 4 * NJ4;
    extern __shared__ __align__(16) float sb[];
    float *sBhi = sb, *sBlo = sb + (size_t)L * PQ;
    for (int e = threadIdx.x; e < L * PQ; e += blockDim.x) {
        sBhi[e] = Bhi[e];
        sBlo[e] = Blo[e];
    }
    __syncthreads();
    const long long stride = (long long)gridDim.x * PROJ_THREADS;
    for (long long n = (long long)blockIdx.x * PROJ_THREADS + threadIdx.x; n < N; n += stride) {
        dot2 acc[PQ];
        const float *y = cube + (size_t)n * L;
        auto band = [&](int l, float yl) {
            const float *bh = sBhi + (size_t)l * PQ, *bl = sBlo + (size_t)l * PQ;
#pragma unroll
            for (int j4 = 0; j4 < NJ4; ++j4) {
                const float4 h = *reinterpret_cast<const float4 *>(bh + 4 * j4);
                const float4 o = *reinterpret_cast<const float4 *>(bl + 4 * j4);
                acc[4 * j4 + 0].add_prod(h.x, yl); acc[4 * j4 + 0].c = fmaf(o.x, yl, acc[4 * j4 + 0].c);
                acc[4 * j4 + 1].add_prod(h.y, yl); acc[4 * j4 + 1].c = fmaf(o.y, yl, acc[4 * j4 + 1].c);
                acc[4 * j4 + 2].add_prod(h.z, yl); acc[4 * j4 + 2].c = fmaf(o.z, yl, acc[4 * j4 + 2].c);
                acc[4 * j4 + 3].add_prod(h.w, yl); acc[4 * j4 + 3].c = fmaf(o.w, yl, acc[4 * j4 + 3].c);
            }
        };
        int l = 0;
        if (vec) {
            for (; l + 4 <= L; l += 4) {
                const float4 yv = __ldg(reinterpret_cast<const float4 *>(y + l));
                band(l, yv.x); band(l + 1, yv.y); band(l + 2, yv.z); band(l + 3, yv.w);
            }
        }
        for (; l < L; ++l) band(l, __ldg(y + l));
#pragma unroll
        for (int j = 0; j < PQ; ++j) {
            if (j < P) {
                acc[j].add_df(df{(float)RHO, 0.f});
                const df r = acc[j].result();
                c_hi[(size_t)n * P + j] = r.hi;
                c_lo[(size_t)n * P + j] = r.lo;
            }
        }
    }
}

// one wave of resident blocks (at most one block per 128 pixels)
template <typename K>
static unsigned persistent_blocks(K kernel, int threads, size_t smem, long long N)
{
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    const long long need = (N + threads - 1) / threads;
    const long long wave = (long long)sms * per_sm;
    return (unsigned)(need < wave ? need : wave);
}

static bool rows_aligned(const float *cube, int L)
{
    return (L % 4) == 0 && (reinterpret_cast<uintptr_t>(cube) % 16) == 0;
}

template <int NJ4>
static cudaError_t launch_project_t(const float *cube, long long N, int L, int P,
                                    const float *Bhi, const float *Blo, float *c_hi,
                                    float *c_lo, cudaStream_t st)
{
    const size_t smem = sizeof(float) * 2 * (size_t)L * 4 * NJ4;
    cudaError_t e = cudaFuncSetAttribute(project_kernel<NJ4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = persistent_blocks(project_kernel<NJ4>, PROJ_THREADS, smem, N);
    project_kernel<NJ4><<<blocks, PROJ_THREADS, smem, st>>>(cube, N, L, P, Bhi, Blo, c_hi, c_lo,
                                                            rows_aligned(cube, L));
    return cudaGetLastError();
}

cudaError_t launch_project(const float *cube, long long N, int L, int P, const float *Bhi,
                           const float *Blo, float *c_hi, float *c_lo, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    switch ((P + 3) / 4) {
#define LM_CASE(n) case n: return launch_project_t<n>(cube, N, L, P, Bhi, Blo, c_hi, c_lo, st);
        LM_CASE(1) LM_CASE(2) LM_CASE(3) LM_CASE(4) LM_CASE(5) LM_CASE(6) LM_CASE(7) LM_CASE(8)
        LM_CASE(9) LM_CASE(10) LM_CASE(11) LM_CASE(12) LM_CASE(13) LM_CASE(14) LM_CASE(15)
        LM_CASE(16)
#undef LM_CASE
    default: return cudaErrorInvalidValue;
    }
}

// Warp-aggregated counting: the active lanes of a warp with the same key
// add their count with one atomic (the leader's), every lane gets its own
// slot: base of the leader's atomic + its rank among those lanes.
__device__ __forceinline__ unsigned long long bucket_slot(unsigned long long *cursor, int key)
{
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(cursor + key, (unsigned long long)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}
__device__ __forceinline__ void bucket_count(unsigned int *hist, int key)
{
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, key);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(hist + key, (unsigned)__popc(peers));
}

// ------------------------------------------------ fp64 crossover/refinement
constexpr int REF_THREADS = 128;

// Support of the interior-point iterate as a bit mask per pixel: lambda_i <
// theta x_i G_ii (theta = SUPPORT_THETA; coordinates whose barrier term is
// far below their curvature), and the histogram of support sizes.
__global__ void support_kernel(long long N, int P, const float *__restrict__ x,
                               const float *__restrict__ lam, const float *__restrict__ gdiag,
                               const long long *list, const unsigned long long *list_len,
                               unsigned long long *__restrict__ mask, int *__restrict__ ksize,
                               unsigned int *__restrict__ hist)
{
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long n_work = list ? *list_len : (unsigned long long)N;
    if (slot >= (long long)n_work) return;
    const long long n = list ? list[slot] : slot;
    const size_t base = (size_t)n * P;
    unsigned long long m = 0;
    int imax = 0;
    float best = -1.f;
    for (int i = 0; i < P; ++i) {
        const float xi = x[base + i], li = lam[base + i];
        if (xi > best) { best = xi; imax = i; }
        if (li < SUPPORT_THETA * xi * gdiag[i]) m |= 1ULL << i;
    }
    if (!m) m = 1ULL << imax;
    mask[n] = m;
    const int kk = __popcll(m);
    ksize[n] = kk;
    if (hist) bucket_count(hist, kk);
}

// Bucket starts of the support sizes in decreasing order (one block): the
// pixels with the largest supports, whose crossover is the longest serial
// computation, are listed first and start first; *total receives the
// number of listed pixels.
__global__ void bucket_scan_kernel(int P, const unsigned int *__restrict__ hist,
                                   unsigned long long *__restrict__ cursor,
                                   unsigned long long *__restrict__ total)
{
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int kk = P; kk >= 0; --kk) { cursor[kk] = s; s += hist[kk]; }
        *total = s;
    }
}

// Pixels listed by support size (counting sort), so that the lanes of a
// warp run the O(k^3) crossover loops to similar k.
__global__ void bucket_scatter_kernel(long long N, const int *__restrict__ ksize,
                                      unsigned long long *__restrict__ cursor,
                                      long long *__restrict__ list)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    list[bucket_slot(cursor, ksize[n])] = n;
}

// The same counting sort for a list of pixels (the supports they have now):
// the lane groups of a warp then start their pixels with similar sizes.
__global__ void list_hist_kernel(const long long *__restrict__ list,
                                 const unsigned long long *__restrict__ len,
                                 const unsigned long long *__restrict__ mask,
                                 int *__restrict__ ksize, unsigned int *__restrict__ hist)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)*len) return;
    const int k = __popcll(mask[list[i]]);
    ksize[i] = k;
    bucket_count(hist, k);
}
__global__ void list_scatter_kernel(const long long *__restrict__ list,
                                    const unsigned long long *__restrict__ len,
                                    const int *__restrict__ ksize,
                                    unsigned long long *__restrict__ cursor,
                                    long long *__restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)*len) return;
    out[bucket_slot(cursor, ksize[i])] = list[i];
}

// One pass of the active-set crossover.  For each listed pixel, solve the
// equality-constrained problem on its support S (mask) in fp64 through the
// Cholesky factor of G~_SS (positive definite since rank [S^T; 1^T] = P),
// then check the KKT conditions of Sec. 2.2's problem: x_S >= -tol_x and
// lambda_i = (G~ x)_i - c~_i + nu >= -tol_g off S.  If they hold, x is the
// minimiser to fp64 accuracy: write it and its uncertainty (square root of
// the diagonal of the top-left block of [[G~_SS, 1],[1^T, 0]]^-1, divided by
// s).  Otherwise drop the most negative coordinate, or add the most
// violated one, and hand the pixel to the next pass; on the last pass (or if
// the factorisation fails) the pixel goes to the retry list.
template <int KMAX>
__global__ void __launch_bounds__(REF_THREADS)
crossover_pass_kernel(const CrossArgs a)
{
    // G~ as hi + lo float32 words in shared memory (P x P)
    extern __shared__ __align__(16) float sgm[];
    const int P = a.P;
    float *sGh = sgm, *sGl = sgm + P * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int i = e / P, j = e % P;
        sGh[e] = a.Ghi[(size_t)i * a.PP + j];
        sGl[e] = a.Glo[(size_t)i * a.PP + j];
    }
    __syncthreads();
    const long long slot = (long long)blockIdx.x * REF_THREADS + threadIdx.x;
    if (slot >= (long long)*a.len_in) return;
    const long long n = a.list_in[slot];
    const size_t base = (size_t)n * P;
    const unsigned long long m = a.mask[n];
    // all arithmetic below is double-float (two float32 words, ~48-bit
    // significand) on the float32 pipes: fp64 is a small fraction of the
    // fp32 rate on this GPU
    int idx[KMAX];
    df M[KMAX * (KMAX + 1) / 2], u[KMAX], v[KMAX], xs[KMAX];
    int k = 0;
    for (int i = 0; i < P; ++i)
        if ((m >> i) & 1ULL) idx[k++] = i;
    auto mat = [&](int r, int c) -> df & { return M[r * (r + 1) / 2 + c]; };
    auto gt = [&](int i, int j) -> df { return df{sGh[i * P + j], sGl[i * P + j]}; };

    // Cholesky of G~_SS (left-looking by columns); the diagonal keeps 1/L_cc.
    // The dot products of a column are independent across rows: four rows
    // run together so that four double-float chains are in flight.
    for (int r = 0; r < k; ++r)
        for (int c = 0; c <= r; ++c) mat(r, c) = gt(idx[r], idx[c]);
    bool fact_ok = true;
    const df zero = df_make(0.f);
    for (int c = 0; c < k; ++c) {
        df d0 = mat(c, c), d1 = zero;
        int q = 0;
        for (; q + 1 < c; q += 2) {
            d0 = df_fms(d0, mat(c, q), mat(c, q));
            d1 = df_fms(d1, mat(c, q + 1), mat(c, q + 1));
        }
        if (q < c) d0 = df_fms(d0, mat(c, q), mat(c, q));
        df d = df_add(d0, d1);
        if (!(d.hi > 0.f)) { fact_ok = false; d = df_make(1e-30f); }
        const df rl = df_rsqrt(d);
        mat(c, c) = rl;
        for (int r = c + 1; r < k; r += 4) {
            const int r1 = min(r + 1, k - 1), r2 = min(r + 2, k - 1), r3 = min(r + 3, k - 1);
            df s0 = mat(r, c), s1 = mat(r1, c), s2 = mat(r2, c), s3 = mat(r3, c);
            for (int p = 0; p < c; ++p) {
                const df mc = mat(c, p);
                s0 = df_fms(s0, mat(r, p), mc);
                s1 = df_fms(s1, mat(r1, p), mc);
                s2 = df_fms(s2, mat(r2, p), mc);
                s3 = df_fms(s3, mat(r3, p), mc);
            }
            mat(r, c) = df_mul(s0, rl);
            if (r + 1 < k) mat(r1, c) = df_mul(s1, rl);
            if (r + 2 < k) mat(r2, c) = df_mul(s2, rl);
            if (r + 3 < k) mat(r3, c) = df_mul(s3, rl);
        }
    }
    // forward: u = L^-1 1, v = L^-1 c~_S (two independent chains, each
    // split in even/odd partial sums)
    for (int r = 0; r < k; ++r) {
        df su0 = df_make(1.f), su1 = zero;
        df sv0 = df{a.c_hi[base + idx[r]], a.c_lo[base + idx[r]]}, sv1 = zero;
        int q = 0;
        for (; q + 1 < r; q += 2) {
            su0 = df_fms(su0, mat(r, q), u[q]); sv0 = df_fms(sv0, mat(r, q), v[q]);
            su1 = df_fms(su1, mat(r, q + 1), u[q + 1]); sv1 = df_fms(sv1, mat(r, q + 1), v[q + 1]);
        }
        if (q < r) { su0 = df_fms(su0, mat(r, q), u[q]); sv0 = df_fms(sv0, mat(r, q), v[q]); }
        u[r] = df_mul(df_add(su0, su1), mat(r, r));
        v[r] = df_mul(df_add(sv0, sv1), mat(r, r));
    }
    df a11 = zero, a1b = zero;
    for (int r = 0; r < k; ++r) { a11 = df_add(a11, df_mul(u[r], u[r])); a1b = df_add(a1b, df_mul(u[r], v[r])); }
    const df nu = df_div(df_sub(a1b, df_make(1.f)), a11);
    // back: xs = L^-T (v - nu u), u <- L^-T u (= G~_SS^-1 1)
    for (int r = k - 1; r >= 0; --r) {
        df sx0 = df_fms(v[r], nu, u[r]), su0 = u[r], sx1 = zero, su1 = zero;
        int q = r + 1;
        for (; q + 1 < k; q += 2) {
            sx0 = df_fms(sx0, mat(q, r), xs[q]); su0 = df_fms(su0, mat(q, r), u[q]);
            sx1 = df_fms(sx1, mat(q + 1, r), xs[q + 1]); su1 = df_fms(su1, mat(q + 1, r), u[q + 1]);
        }
        if (q < k) { sx0 = df_fms(sx0, mat(q, r), xs[q]); su0 = df_fms(su0, mat(q, r), u[q]); }
        xs[r] = df_mul(df_add(sx0, sx1), mat(r, r));
        u[r] = df_mul(df_add(su0, su1), mat(r, r));
    }
    // decision
    int flip = -1;             // coordinate whose membership in S changes
    df xsum = df_make(0.f);
    if (fact_ok) {
        float xmin = (float)-a.tol_x;
        for (int r = 0; r < k; ++r) {
            if (xs[r].hi < xmin) { xmin = xs[r].hi; flip = idx[r]; }
            if (xs[r].hi > 0.f) xsum = df_add(xsum, xs[r]);
        }
        if (flip >= 0 && k == 1) flip = -2;       // cannot drop the last one
        if (flip == -1) {
            // most negative multiplier off S; four coordinates at once
            float lmin = (float)-a.tol_g;
            int off[KMAX];
            int noff = 0;
            for (int i = 0; i < P; ++i)
                if (!((m >> i) & 1ULL)) off[noff++] = i;
            for (int o = 0; o < noff; o += 4) {
                int ii[4];
                dot2 g[4];
#pragma unroll
                for (int w = 0; w < 4; ++w) ii[w] = off[min(o + w, noff - 1)];
                for (int q = 0; q < k; ++q) {
                    const float xh = xs[q].hi, xl = xs[q].lo;
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const float gh = sGh[ii[w] * P + idx[q]], gl = sGl[ii[w] * P + idx[q]];
                        g[w].add_prod(gh, xh);
                        g[w].c = fmaf(gh, xl, fmaf(gl, xh, g[w].c));
                    }
                }
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    if (o + w >= noff) break;
                    g[w].add_df(df{-a.c_hi[base + ii[w]], -a.c_lo[base + ii[w]]});
                    g[w].add_df(nu);
                    const df gv = g[w].result();
                    if (gv.hi < lmin) { lmin = gv.hi; flip = ii[w]; }
                }
            }
        }
    } else {
        flip = -2;
    }
    if (flip == -1 && xsum.hi > 0.f) {
        // KKT holds: abundances and uncertainties
        int r = 0;
        for (int i = 0; i < P; ++i) {
            float xi = 0.f;
            if ((m >> i) & 1ULL) { xi = xs[r].hi > 0.f ? df_div(xs[r], xsum).hi : 0.f; ++r; }
            a.x_out[base + i] = xi;
        }
        if (a.sx_out) {
            const float s = (float)a.scale[0];
            const df inv_a11 = df_div(df_make(1.f), a11);
            // diag of G~_SS^-1 = column norms of L^-1: w = L^-1 e_r by forward
            // substitution from row r; two columns at a time
            df dsq[KMAX];
            for (int r0 = 0; r0 < k; r0 += 2) {
                const int r1 = min(r0 + 1, k - 1);
                df w0[KMAX], w1[KMAX];
                df n0 = zero, n1 = zero;
                for (int q = r0; q < k; ++q) {
                    df s0 = df_make(q == r0 ? 1.f : 0.f), s1 = df_make(q == r1 ? 1.f : 0.f);
                    for (int p = r0; p < q; ++p) {
                        const df lqp = mat(q, p);
                        s0 = df_fms(s0, lqp, w0[p]);
                        s1 = df_fms(s1, lqp, p >= r1 ? w1[p] : zero);
                    }
                    w0[q] = df_mul(s0, mat(q, q));
                    w1[q] = q >= r1 ? df_mul(s1, mat(q, q)) : zero;
                    n0 = df_add(n0, df_mul(w0[q], w0[q]));
                    n1 = df_add(n1, df_mul(w1[q], w1[q]));
                }
                dsq[r0] = n0;
                if (r0 + 1 < k) dsq[r1] = n1;
            }
            int r = 0;
            for (int i = 0; i < P; ++i) {
                float out = 0.f;
                if ((m >> i) & 1ULL) {
                    const df var = df_sub(dsq[r], df_mul(df_mul(u[r], u[r]), inv_a11));
                    out = sqrtf(fmaxf(var.hi, 0.f) / s);
                    ++r;
                }
                a.sx_out[base + i] = out;
            }
        }
        return;
    }
    if (flip >= 0 && a.list_out) {
        a.mask[n] = m ^ (1ULL << flip);
        const unsigned long long pos = atomicAdd(a.len_out, 1ULL);
        a.list_out[pos] = n;
        return;
    }
    // not finished here: retry list, or (retry path) keep the iterate
    if (a.retry_list) {
        const unsigned long long pos = atomicAdd(a.retry_len, 1ULL);
        a.retry_list[pos] = n;
    } else if (a.n_unverified) {
        // the iterate stays as the result: reported as not converged
        if (!a.it_mark || a.it_mark[n] > 0) {
            atomicAdd(a.n_unverified, 1ULL);
            if (a.it_mark) a.it_mark[n] = -a.it_mark[n];
        }
    }
    if (a.x_out != a.x_in)
        for (int i = 0; i < P; ++i) a.x_out[base + i] = a.x_in[base + i];
    if (a.sx_out)
        for (int i = 0; i < P; ++i) a.sx_out[base + i] = 0.f;
}

template <int KMAX>
static cudaError_t launch_pass_t(const CrossArgs &a, cudaStream_t st)
{
    const size_t smem = 2 * sizeof(float) * (size_t)a.P * a.P;
    cudaError_t e = cudaFuncSetAttribute(crossover_pass_kernel<KMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (a.N + REF_THREADS - 1) / REF_THREADS;   // lists hold <= N entries
    crossover_pass_kernel<KMAX><<<(unsigned)blocks, REF_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_pass(const CrossArgs &a, cudaStream_t st)
{
    if (a.P <= 16) return launch_pass_t<16>(a, st);
    if (a.P <= 32) return launch_pass_t<32>(a, st);
    if (a.P <= 48) return launch_pass_t<48>(a, st);
    return launch_pass_t<64>(a, st);
}

// Crossover pass with a group of XG lanes per pixel.  The passes after the
// first see only the pixels whose support changed (a few percent); one
// thread per pixel would leave their time to the longest serial chain
// (~1e5 double-float instructions for a 20-coordinate support).  Here row
// r of L, and entry r of every vector indexed by the support, belong to
// lane r % XG of the group; L (packed lower triangle, double-float) lives
// in the group's shared memory.  Same arithmetic steps as
// crossover_pass_kernel: Cholesky of G~_SS with the forward solves of 1
// and c~_S fused in, nu from the bordered system, the back solve, the
// decision, and on success x / sum(x) and the uncertainties, whose
// diag(G~_SS^-1) comes from L^-1 formed in place (columns right to left).
constexpr int XG = 8;

template <int KMAX>
struct XGCfg {
    static constexpr int KS = (KMAX + XG - 1) / XG;        // row slots per lane
    // 16, 8 or 4 groups per block
    static constexpr int THREADS = KMAX <= XCAP ? 128 : (KMAX > 48 ? 32 : 64);
    static constexpr int MIN_BLOCKS = KMAX <= XCAP ? 4 : 1;
    static constexpr int GROUPS = THREADS / XG;
    // per group, sized by the largest support K = min(P, KMAX) this launch
    // solves: L hi/lo as packed lower triangles, x hi/lo, the support list
    __host__ __device__ static int kdim(int P) { return P < KMAX ? P : KMAX; }
    static int group_words(int P) { return kdim(P) * (kdim(P) + 1) + 3 * kdim(P); }
    static size_t smem(int P) { return sizeof(float) * (2 * (size_t)P * P + (size_t)GROUPS * group_words(P)); }
};

__device__ __forceinline__ int pk(int r, int c) { return r * (r + 1) / 2 + c; }

__device__ __forceinline__ df shfl_df(unsigned mask, df v, int src)
{
    return df{__shfl_sync(mask, v.hi, src, XG), __shfl_sync(mask, v.lo, src, XG)};
}

__device__ __forceinline__ df group_sum_df(unsigned mask, df v)
{
    for (int off = 1; off < XG; off <<= 1)
        v = df_add(v, df{__shfl_xor_sync(mask, v.hi, off, XG), __shfl_xor_sync(mask, v.lo, off, XG)});
    return v;
}

// smallest value, ties to the smallest index (index -1: no candidate)
__device__ __forceinline__ void group_argmin(unsigned mask, float &v, int &i)
{
    for (int off = 1; off < XG; off <<= 1) {
        const float ov = __shfl_xor_sync(mask, v, off, XG);
        const int oi = __shfl_xor_sync(mask, i, off, XG);
        if (oi >= 0 && (i < 0 || ov < v || (ov == v && oi < i))) { v = ov; i = oi; }
    }
}

template <int KMAX>
__global__ void __launch_bounds__(XGCfg<KMAX>::THREADS, XGCfg<KMAX>::MIN_BLOCKS)
crossover_group_kernel(const CrossArgs a)
{
    using C = XGCfg<KMAX>;
    constexpr int KS = C::KS;
    extern __shared__ __align__(16) float sgm[];
    const int P = a.P;
    const unsigned long long n_work = *a.len_in;
    if ((unsigned long long)blockIdx.x * C::GROUPS >= n_work) return;   // no pixel for this block
    float *sGh = sgm, *sGl = sgm + P * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int i = e / P, j = e % P;
        sGh[e] = a.Ghi[(size_t)i * a.PP + j];
        sGl[e] = a.Glo[(size_t)i * a.PP + j];
    }
    const int lane = threadIdx.x & 31, t = lane % XG, grp = threadIdx.x / XG;
    const unsigned gmask = ((1u << XG) - 1u) << ((lane / XG) * XG);
    const int K = C::kdim(P), lsz = K * (K + 1) / 2;
    float *Lh = sgm + 2 * P * P + (size_t)grp * (2 * lsz + 3 * K);
    float *Ll = Lh + lsz, *xh = Ll + lsz, *xl = xh + K;
    int *sidx = reinterpret_cast<int *>(xl + K);
    __syncthreads();
    const df zero = df_make(0.f);
    const long long stride = (long long)gridDim.x * C::GROUPS;
    for (long long slot = (long long)blockIdx.x * C::GROUPS + grp; slot < (long long)n_work;
         slot += stride) {
        // a list entry: the pixel, and above XG_SOLVE_SHIFT the solves it
        // already had (entries handed over from a launch with a smaller K)
        const long long entry = a.list_in[slot];
        const long long n = entry & ((1LL << XG_SOLVE_SHIFT) - 1);
        const size_t base = (size_t)n * P;
        unsigned long long m = a.mask[n];
        // up to max_solves support solves for this pixel: each failed KKT
        // check flips one coordinate and solves again on the new support
        for (int solve = (int)(entry >> XG_SOLVE_SHIFT);; ++solve) {
            const bool can_flip = solve + 1 < a.max_solves;
            const int k = __popcll(m);
            if (k > KMAX) {
                // more coordinates than this launch's factor holds: the pixel,
                // its support already in mask[n], goes to the launch sized by P
                if (t == 0) {
                    const unsigned long long pos = atomicAdd(a.over_len, 1ULL);
                    a.over_list[pos] = n | ((long long)solve << XG_SOLVE_SHIFT);
                }
                break;
            }
            // row slots in use: the slot loops (unrolled to KS) stop there
            const int ks = (k + XG - 1) / XG;
            for (int i = t; i < P; i += XG)
                if ((m >> i) & 1ULL) sidx[__popcll(m & ((1ULL << i) - 1ULL))] = i;
            __syncwarp(gmask);
            // L = G~_SS on the own rows; right-hand sides 1 and c~_S
            df au[KS], av[KS], uu[KS], vv[KS];
#pragma unroll
            for (int s = 0; s < KS && s < ks; ++s) {
                const int r = s * XG + t;
                au[s] = av[s] = uu[s] = vv[s] = zero;
                if (r < k) {
                    const int gr = sidx[r];
                    for (int j = 0; j <= r; ++j) {
                        const int gj = sidx[j];
                        Lh[pk(r, j)] = sGh[gr * P + gj];
                        Ll[pk(r, j)] = sGl[gr * P + gj];
                    }
                    au[s] = df_make(1.f);
                    av[s] = df{a.c_hi[base + gr], a.c_lo[base + gr]};
                }
            }
            __syncwarp(gmask);
            // right-looking Cholesky; the diagonal keeps 1/L_cc
            bool ok = true;
            for (int c = 0; c < k; ++c) {
                df d = df{Lh[pk(c, c)], Ll[pk(c, c)]};
                if (!(d.hi > 0.f)) { ok = false; d = df_make(1e-30f); }
                const df rl = df_rsqrt(d);
                df uc = zero, vc = zero, lrc[KS];
#pragma unroll
                for (int s = 0; s < KS && s < ks; ++s) {
                    const int r = s * XG + t;
                    lrc[s] = zero;
                    if (r > c && r < k) {
                        lrc[s] = df_mul(df{Lh[pk(r, c)], Ll[pk(r, c)]}, rl);
                        Lh[pk(r, c)] = lrc[s].hi;
                        Ll[pk(r, c)] = lrc[s].lo;
                    }
                    if (r == c) {
                        uc = df_mul(au[s], rl);
                        vc = df_mul(av[s], rl);
                        uu[s] = uc;
                        vv[s] = vc;
                        Lh[pk(c, c)] = rl.hi;
                        Ll[pk(c, c)] = rl.lo;
                    }
                }
                uc = shfl_df(gmask, uc, c % XG);
                vc = shfl_df(gmask, vc, c % XG);
                __syncwarp(gmask);                       // column c of L stored
#pragma unroll
                for (int s = 0; s < KS && s < ks; ++s) {
                    const int r = s * XG + t;
                    if (r > c && r < k) {
                        au[s] = df_fms(au[s], lrc[s], uc);
                        av[s] = df_fms(av[s], lrc[s], vc);
                    }
                }
                // trailing update L_rj -= L_rc L_jc (c < j <= r): the lane's rows
                // advance together (independent chains), L_jc read once per j
                for (int j = c + 1; j < k; ++j) {
                    const df ljc = df{Lh[pk(j, c)], Ll[pk(j, c)]};
#pragma unroll
                    for (int s = 0; s < KS && s < ks; ++s) {
                        const int r = s * XG + t;
                        if (r >= j && r < k) {
                            const df v = df_fms(df{Lh[pk(r, j)], Ll[pk(r, j)]}, lrc[s], ljc);
                            Lh[pk(r, j)] = v.hi;
                            Ll[pk(r, j)] = v.lo;
                        }
                    }
                }
                __syncwarp(gmask);                       // trailing block updated
            }
            // nu from the bordered system
            df a11 = zero, a1b = zero;
#pragma unroll
            for (int s = 0; s < KS && s < ks; ++s)
                if (s * XG + t < k) {
                    a11 = df_add(a11, df_mul(uu[s], uu[s]));
                    a1b = df_add(a1b, df_mul(uu[s], vv[s]));
                }
            a11 = group_sum_df(gmask, a11);
            a1b = group_sum_df(gmask, a1b);
            const df nu = df_div(df_sub(a1b, df_make(1.f)), a11);
            // back solve: xs = L^-T (v - nu u), ub = L^-T u (= G~_SS^-1 1)
            df ax[KS], ab[KS], xs[KS], ub[KS];
#pragma unroll
            for (int s = 0; s < KS && s < ks; ++s) {
                ax[s] = df_fms(vv[s], nu, uu[s]);
                ab[s] = uu[s];
                xs[s] = ub[s] = zero;
            }
            for (int r = k - 1; r >= 0; --r) {
                df xr = zero, ur = zero;
#pragma unroll
                for (int s = 0; s < KS && s < ks; ++s)
                    if (s * XG + t == r) {
                        const df rlr = df{Lh[pk(r, r)], Ll[pk(r, r)]};
                        xr = df_mul(ax[s], rlr);
                        ur = df_mul(ab[s], rlr);
                        xs[s] = xr;
                        ub[s] = ur;
                    }
                xr = shfl_df(gmask, xr, r % XG);
                ur = shfl_df(gmask, ur, r % XG);
#pragma unroll
                for (int s = 0; s < KS && s < ks; ++s) {
                    const int q = s * XG + t;
                    if (q < r) {
                        const df lrq = df{Lh[pk(r, q)], Ll[pk(r, q)]};
                        ax[s] = df_fms(ax[s], lrq, xr);
                        ab[s] = df_fms(ab[s], lrq, ur);
                    }
                }
            }
            // decision
            int flip = -1;
            df xsum = zero;
            if (ok) {
                float xmin = (float)-a.tol_x;
                int fr = -1;
#pragma unroll
                for (int s = 0; s < KS && s < ks; ++s) {
                    const int r = s * XG + t;
                    if (r < k) {
                        if (xs[s].hi < xmin) { xmin = xs[s].hi; fr = r; }
                        if (xs[s].hi > 0.f) xsum = df_add(xsum, xs[s]);
                    }
                }
                group_argmin(gmask, xmin, fr);
                xsum = group_sum_df(gmask, xsum);
                if (fr >= 0) flip = (k == 1) ? -2 : sidx[fr];
                if (flip == -1) {
                    // most negative multiplier off S, coordinates spread over the lanes
#pragma unroll
                    for (int s = 0; s < KS && s < ks; ++s) {
                        const int r = s * XG + t;
                        if (r < k) { xh[r] = xs[s].hi; xl[r] = xs[s].lo; }
                    }
                    __syncwarp(gmask);
                    float lmin = (float)-a.tol_g;
                    int fi = -1;
                    for (int i = t; i < P; i += XG) {
                        if ((m >> i) & 1ULL) continue;
                        dot2 g;
                        for (int q = 0; q < k; ++q) {
                            const float gh = sGh[i * P + sidx[q]], gl = sGl[i * P + sidx[q]];
                            g.add_prod(gh, xh[q]);
                            g.c = fmaf(gh, xl[q], fmaf(gl, xh[q], g.c));
                        }
                        g.add_df(df{-a.c_hi[base + i], -a.c_lo[base + i]});
                        g.add_df(nu);
                        const df gv = g.result();
                        if (gv.hi < lmin) { lmin = gv.hi; fi = i; }
                    }
                    group_argmin(gmask, lmin, fi);
                    flip = fi;
                }
            } else {
                flip = -2;
            }
            if (flip == -1 && xsum.hi > 0.f) {
                // KKT holds: abundances and uncertainties
                for (int i = t; i < P; i += XG)
                    if (!((m >> i) & 1ULL)) a.x_out[base + i] = 0.f;
#pragma unroll
                for (int s = 0; s < KS && s < ks; ++s) {
                    const int r = s * XG + t;
                    if (r < k) a.x_out[base + sidx[r]] = xs[s].hi > 0.f ? df_div(xs[s], xsum).hi : 0.f;
                }
                if (a.sx_out) {
                    // L -> L^-1 in place: Linv_ij = -(sum_{j<q<=i} Linv_iq L_qj) / L_jj,
                    // column j from right to left (rows on their lanes)
                    for (int j = k - 2; j >= 0; --j) {
                        const df rlj = df{Lh[pk(j, j)], Ll[pk(j, j)]};
                        df acc[KS];
#pragma unroll
                        for (int s = 0; s < KS && s < ks; ++s) acc[s] = zero;
                        for (int q = j + 1; q < k; ++q) {
                            const df lqj = df{Lh[pk(q, j)], Ll[pk(q, j)]};
#pragma unroll
                            for (int s = 0; s < KS && s < ks; ++s) {
                                const int i = s * XG + t;
                                if (i >= q && i < k)
                                    acc[s] = df_fms(acc[s], df{Lh[pk(i, q)], Ll[pk(i, q)]}, lqj);
                            }
                        }
                        __syncwarp(gmask);               // column j read by every row
#pragma unroll
                        for (int s = 0; s < KS && s < ks; ++s) {
                            const int i = s * XG + t;
                            if (i > j && i < k) {
                                const df v = df_mul(acc[s], rlj);
                                Lh[pk(i, j)] = v.hi;
                                Ll[pk(i, j)] = v.lo;
                            }
                        }
                        __syncwarp(gmask);
                    }
                    const float sc = (float)a.scale[0];
                    const df inv_a11 = df_div(df_make(1.f), a11);
                    for (int i = t; i < P; i += XG)
                        if (!((m >> i) & 1ULL)) a.sx_out[base + i] = 0.f;
                    df nrm[KS];
#pragma unroll
                    for (int s = 0; s < KS && s < ks; ++s) nrm[s] = zero;
                    for (int i = t; i < k; ++i) {
#pragma unroll
                        for (int s = 0; s < KS && s < ks; ++s) {
                            const int j = s * XG + t;
                            if (j <= i) {
                                const df w = df{Lh[pk(i, j)], Ll[pk(i, j)]};
                                nrm[s] = df_add(nrm[s], df_mul(w, w));
                            }
                        }
                    }
#pragma unroll
                    for (int s = 0; s < KS && s < ks; ++s) {
                        const int j = s * XG + t;
                        if (j < k) {
                            const df var = df_sub(nrm[s], df_mul(df_mul(ub[s], ub[s]), inv_a11));
                            a.sx_out[base + sidx[j]] = sqrtf(fmaxf(var.hi, 0.f) / sc);
                        }
                    }
                }
                break;
            } else if (flip >= 0 && can_flip) {
                m ^= 1ULL << flip;
                if (t == 0) a.mask[n] = m;
                __syncwarp(gmask);                       // sidx, xh, xl are rewritten
                continue;
            } else {
                // not finished here: retry list, or (retry path) keep the iterate
                if (t == 0) {
                    if (a.retry_list) {
                        const unsigned long long pos = atomicAdd(a.retry_len, 1ULL);
                        a.retry_list[pos] = n;
                    } else if (a.n_unverified) {
                        // the iterate stays as the result: reported as not converged
                        if (!a.it_mark || a.it_mark[n] > 0) {
                            atomicAdd(a.n_unverified, 1ULL);
                            if (a.it_mark) a.it_mark[n] = -a.it_mark[n];
                        }
                    }
                }
                for (int i = t; i < P; i += XG) {
                    if (a.x_out != a.x_in) a.x_out[base + i] = a.x_in[base + i];
                    if (a.sx_out) a.sx_out[base + i] = 0.f;
                }
                break;
            }
        }
        __syncwarp(gmask);                           // the group's shared memory is reused
    }
}

template <int KMAX>
static cudaError_t launch_group_t(const CrossArgs &a, cudaStream_t st)
{
    using C = XGCfg<KMAX>;
    const size_t smem = C::smem(a.P);
    cudaError_t e = cudaFuncSetAttribute(crossover_group_kernel<KMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crossover_group_kernel<KMAX>, C::THREADS,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    // the list length is on the device: one wave of groups striding over it,
    // at most one group per list entry
    long long blocks = (long long)sms * per_sm;
    const long long need = (a.N + C::GROUPS - 1) / C::GROUPS;
    if (blocks > need) blocks = need;
    crossover_group_kernel<KMAX><<<(unsigned)blocks, C::THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_group_full(const CrossArgs &a, cudaStream_t st)
{
    if (a.P <= 16) return launch_group_t<16>(a, st);
    if (a.P <= 32) return launch_group_t<32>(a, st);
    if (a.P <= 48) return launch_group_t<48>(a, st);
    return launch_group_t<64>(a, st);
}

// Lane groups over a.list_in.  For P > XCAP a first launch factors supports
// of up to XCAP coordinates (a third to a half of the shared memory per group
// at P = 36 to 48, so more groups per SM); the rare pixel whose support
// outgrows that is listed in w.list[1] with its solve count and finished by
// a launch sized by P.  w.list[1] and w.len[2] are free at this point.
static cudaError_t launch_pass_group(const CrossArgs &a, const CrossoverScratch &w, cudaStream_t st)
{
    if (a.P <= XCAP) return launch_group_full(a, st);
    CrossArgs c = a;
    c.over_list = w.list[1];
    c.over_len = w.len + 2;
    cudaError_t e = launch_group_t<XCAP>(c, st);
    if (e != cudaSuccess) return e;
    CrossArgs o = a;
    o.list_in = w.list[1];
    o.len_in = w.len + 2;
    return launch_group_full(o, st);
}

cudaError_t launch_crossover(const CrossArgs &base, const CrossoverScratch &w,
                             const long long *list, const unsigned long long *list_len,
                             cudaStream_t st)
{
    if (base.N <= 0) return cudaSuccess;
    const int T = 256;
    const unsigned gridN = (unsigned)((base.N + T - 1) / T);
    cudaError_t e;
    // counters: w.len[0..MAX_SWAPS+1] list lengths, w.hist support-size counts
    e = cudaMemsetAsync(w.len, 0, sizeof(unsigned long long) * (MAX_SWAPS + 2), st);
    if (e != cudaSuccess) return e;
    const long long *first = list;
    const unsigned long long *first_len = list_len;
    if (!list) {
        // whole cube: counting sort by support size
        e = cudaMemsetAsync(w.hist, 0, sizeof(unsigned int) * (base.P + 1), st);
        if (e != cudaSuccess) return e;
        support_kernel<<<gridN, T, 0, st>>>(base.N, base.P, base.x_in, base.lam_in, base.gdiag,
                                             nullptr, nullptr, base.mask, w.ksize, w.hist);
        bucket_scan_kernel<<<1, 32, 0, st>>>(base.P, w.hist, w.cursor, w.len_all);
        bucket_scatter_kernel<<<gridN, T, 0, st>>>(base.N, w.ksize, w.cursor, w.list[0]);
        first = w.list[0];
        first_len = w.len_all;
    } else {
        support_kernel<<<gridN, T, 0, st>>>(base.N, base.P, base.x_in, base.lam_in, base.gdiag,
                                             list, list_len, base.mask, w.ksize, nullptr);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // whole cube: pass 0 one thread per pixel (throughput bound), the
    // pixels it flips go to list 1; then one launch of lane groups that
    // takes each listed pixel through up to MAX_SWAPS further support
    // changes (latency bound, few pixels).  A given list: the lane groups
    // from its first solve, MAX_SWAPS + 1 solves.
    CrossArgs a = base;
    if (!list) {
        a.list_in = first;
        a.len_in = first_len;
        a.list_out = w.list[1];
        a.len_out = w.len + 1;
        e = launch_pass(a, st);
        if (e != cudaSuccess) return e;
        // the flipped pixels, sorted by their new support size into list 0
        e = cudaMemsetAsync(w.hist, 0, sizeof(unsigned int) * (base.P + 1), st);
        if (e != cudaSuccess) return e;
        list_hist_kernel<<<gridN, T, 0, st>>>(w.list[1], w.len + 1, base.mask, w.ksize, w.hist);
        bucket_scan_kernel<<<1, 32, 0, st>>>(base.P, w.hist, w.cursor, w.len_all);
        list_scatter_kernel<<<gridN, T, 0, st>>>(w.list[1], w.len + 1, w.ksize, w.cursor, w.list[0]);
        a.list_in = w.list[0];
        a.len_in = w.len + 1;
        a.max_solves = MAX_SWAPS;
    } else {
        a.list_in = first;
        a.len_in = first_len;
        a.max_solves = MAX_SWAPS + 1;
    }
    a.list_out = nullptr;
    a.len_out = nullptr;
    return launch_pass_group(a, w, st);
}

// ------------------------------------------------------------------- rms
constexpr int RMS_THREADS = 128;

// Grid-stride over tiles of 2 x RMS_THREADS pixels, a thread takes two
// pixels (t and t + RMS_THREADS of the tile) so that every S^T value read
// from shared memory feeds two fits; S^T staged once per block; four bands
// per step (one 16-byte load of each row when rows are 16-byte aligned).
template <int NJ4>
__global__ void __launch_bounds__(RMS_THREADS)
rms_kernel(const float *__restrict__ cube, const float *__restrict__ S,
           const float *__restrict__ x, long long N, int L, int P, float *__restrict__ rms,
           bool vec)
{
    constexpr int PQ = 4 * NJ4;
    extern __shared__ __align__(16) float st[];   // [l][PQ] = S^T, zero padded
    for (int e = threadIdx.x; e < L * PQ; e += blockDim.x) {
        const int l = e / PQ, j = e % PQ;
        st[e] = j < P ? S[(size_t)j * L + l] : 0.f;
    }
    __syncthreads();
    const long long stride = (long long)gridDim.x * 2 * RMS_THREADS;
    for (long long t0 = (long long)blockIdx.x * 2 * RMS_THREADS; t0 < N; t0 += stride) {
        const long long na = t0 + threadIdx.x, nb = na + RMS_THREADS;
        if (na >= N) continue;                     // nothing left for this thread
        const bool ha = true, hb = nb < N;
        // a missing second pixel repeats the first (its result is dropped)
        const long long ra = na, rb = hb ? nb : ra;
        float xa[PQ], xb[PQ];
#pragma unroll
        for (int j = 0; j < PQ; ++j) {
            xa[j] = j < P ? x[(size_t)ra * P + j] : 0.f;
            xb[j] = j < P ? x[(size_t)rb * P + j] : 0.f;
        }
        const float *ya = cube + (size_t)ra * L, *yb = cube + (size_t)rb * L;
        auto fit2 = [&](int l, float &ma, float &mb) {
            const float *row = st + (size_t)l * PQ;
            ma = 0.f;
            mb = 0.f;
#pragma unroll
            for (int j4 = 0; j4 < NJ4; ++j4) {
                const float4 sv = *reinterpret_cast<const float4 *>(row + 4 * j4);
                ma = fmaf(xa[4 * j4 + 0], sv.x, ma); mb = fmaf(xb[4 * j4 + 0], sv.x, mb);
                ma = fmaf(xa[4 * j4 + 1], sv.y, ma); mb = fmaf(xb[4 * j4 + 1], sv.y, mb);
                ma = fmaf(xa[4 * j4 + 2], sv.z, ma); mb = fmaf(xb[4 * j4 + 2], sv.z, mb);
                ma = fmaf(xa[4 * j4 + 3], sv.w, ma); mb = fmaf(xb[4 * j4 + 3], sv.w, mb);
            }
        };
        float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
        int l = 0;
        if (vec && ha) {
            for (; l + 4 <= L; l += 4) {
                const float4 va = __ldg(reinterpret_cast<const float4 *>(ya + l));
                const float4 vb = __ldg(reinterpret_cast<const float4 *>(yb + l));
                float ma, mb;
                fit2(l, ma, mb);     { const float e = va.x - ma, f = vb.x - mb; a0 = fmaf(e, e, a0); b0 = fmaf(f, f, b0); }
                fit2(l + 1, ma, mb); { const float e = va.y - ma, f = vb.y - mb; a1 = fmaf(e, e, a1); b1 = fmaf(f, f, b1); }
                fit2(l + 2, ma, mb); { const float e = va.z - ma, f = vb.z - mb; a0 = fmaf(e, e, a0); b0 = fmaf(f, f, b0); }
                fit2(l + 3, ma, mb); { const float e = va.w - ma, f = vb.w - mb; a1 = fmaf(e, e, a1); b1 = fmaf(f, f, b1); }
            }
        }
        for (; l < L; ++l) {
            float ma, mb;
            fit2(l, ma, mb);
            const float e = __ldg(ya + l) - ma, f = __ldg(yb + l) - mb;
            a0 = fmaf(e, e, a0);
            b0 = fmaf(f, f, b0);
        }
        if (ha) rms[na] = sqrtf((a0 + a1) / (float)L);
        if (hb) rms[nb] = sqrtf((b0 + b1) / (float)L);
    }
}

template <int NJ4>
static cudaError_t launch_rms_t(const float *cube, const float *S, const float *x, long long N,
                                int L, int P, float *rms, cudaStream_t st)
{
    const size_t smem = sizeof(float) * (size_t)L * 4 * NJ4;
    cudaError_t e = cudaFuncSetAttribute(rms_kernel<NJ4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = persistent_blocks(rms_kernel<NJ4>, RMS_THREADS, smem, (N + 1) / 2);
    rms_kernel<NJ4><<<blocks, RMS_THREADS, smem, st>>>(cube, S, x, N, L, P, rms,
                                                      rows_aligned(cube, L));
    return cudaGetLastError();
}

cudaError_t launch_rms(const float *cube, const float *S, const float *x, long long N, int L,
                       int P, float *rms, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    switch ((P + 3) / 4) {
#define LM_CASE(n) case n: return launch_rms_t<n>(cube, S, x, N, L, P, rms, st);
        LM_CASE(1) LM_CASE(2) LM_CASE(3) LM_CASE(4) LM_CASE(5) LM_CASE(6) LM_CASE(7) LM_CASE(8)
        LM_CASE(9) LM_CASE(10) LM_CASE(11) LM_CASE(12) LM_CASE(13) LM_CASE(14) LM_CASE(15)
        LM_CASE(16)
#undef LM_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lm
