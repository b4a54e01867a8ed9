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
                                   float *__restrict__ grs, float *__restrict__ gdiag, int *flags)
{
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
            for (int j = 0; j < P; ++j) r += G64[(size_t)i * P + j] / s + RHO;
            r /= P;
            gdiag[i] = (float)(G64[(size_t)i * P + i] / s);
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
                                          o.grs, o.gdiag, o.flags);
    const int PQ = pq_of(P);
    const long long total = (long long)L * PQ;
    const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
    prep_b_kernel<<<blocks, 256, 0, st>>>(S, sigma, L, P, PQ, o.scale, o.Bhi, o.Blo);
    return cudaGetLastError();
}

// ------------------------------------------------------------ projection
constexpr int PROJ_THREADS = 128;

template <int NJ4>
__global__ void __launch_bounds__(PROJ_THREADS)
project_kernel(const float *__restrict__ cube, long long N, int L, int P,
               const float *__restrict__ Bhi, const float *__restrict__ Blo,
               float *__restrict__ c_hi, float *__restrict__ c_lo)
{
    constexpr int PQ = 4 * NJ4;
    extern __shared__ __align__(16) float sb[];
    float *sBhi = sb, *sBlo = sb + (size_t)L * PQ;
    for (int e = threadIdx.x; e < L * PQ; e += blockDim.x) {
        sBhi[e] = Bhi[e];
        sBlo[e] = Blo[e];
    }
    __syncthreads();
    const long long n = (long long)blockIdx.x * PROJ_THREADS + threadIdx.x;
    if (n >= N) return;
    dot2 acc[PQ];
    const float *y = cube + (size_t)n * L;
#pragma unroll 2
    for (int l = 0; l < L; ++l) {
        const float yl = __ldg(y + l);
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
    }
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

template <int NJ4>
static cudaError_t launch_project_t(const float *cube, long long N, int L, int P,
                                    const float *Bhi, const float *Blo, float *c_hi,
                                    float *c_lo, cudaStream_t st)
{
    const size_t smem = sizeof(float) * 2 * (size_t)L * 4 * NJ4;
    cudaError_t e = cudaFuncSetAttribute(project_kernel<NJ4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (N + PROJ_THREADS - 1) / PROJ_THREADS;
    project_kernel<NJ4><<<(unsigned)blocks, PROJ_THREADS, smem, st>>>(cube, N, L, P, Bhi, Blo,
                                                                       c_hi, c_lo);
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

// ------------------------------------------------ fp64 crossover/refinement
constexpr int REF_THREADS = 128;

// Exact finish of the interior-point solution by an active-set crossover:
// start from the support S the iterate suggests (lambda_i < x_i G_ii), solve
// the equality-constrained problem on S in fp64 (bordered KKT system through
// the Cholesky factor of G~_SS, positive definite since rank [S^T; 1^T] = P),
// then drop the most negative coordinate, or add the coordinate whose
// multiplier lambda_i = (G~ x)_i - c~_i + nu is the most negative, and
// re-solve, until x_S >= -tol_x and lambda >= -tol_g off S (the KKT
// conditions of Sec. 2.2's problem) or max_swaps is reached.  On success x
// is the minimiser to fp64 accuracy and the uncertainty is read off the same
// factor; otherwise the pixel is appended to the retry list.
template <int KMAX>
__global__ void __launch_bounds__(REF_THREADS)
refine_kernel(const RefineArgs a)
{
    extern __shared__ double sG[];
    const int P = a.P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) sG[e] = a.Gt64[e];
    __syncthreads();
    const long long slot = (long long)blockIdx.x * REF_THREADS + threadIdx.x;
    const unsigned long long n_work = a.list ? *a.list_len : (unsigned long long)a.N;
    if (slot >= (long long)n_work) return;
    const long long n = a.list ? a.list[slot] : slot;
    const size_t base = (size_t)n * P;

    int idx[KMAX];
    double M[KMAX * (KMAX + 1) / 2], u[KMAX], v[KMAX], xs[KMAX];
    int k = 0, imax = 0;
    float best = -1.f;
    for (int i = 0; i < P; ++i) {
        const float xi = a.x_in[base + i], li = a.lam_in[base + i];
        if (xi > best) { best = xi; imax = i; }
        if (li < xi * a.gdiag[i]) idx[k++] = i;
    }
    if (k == 0) idx[k++] = imax;
    auto mat = [&](int r, int c) -> double & { return M[r * (r + 1) / 2 + c]; };

    bool ok = false, fact_ok = true;
    double nu = 0.0, a11 = 1.0, xsum = 1.0;
    for (int sw = 0; sw <= a.max_swaps; ++sw) {
        // Cholesky of G~_SS; the diagonal keeps 1 / L_cc
        for (int r = 0; r < k; ++r)
            for (int c = 0; c <= r; ++c) mat(r, c) = sG[idx[r] * P + idx[c]];
        fact_ok = true;
        for (int c = 0; c < k; ++c) {
            double d = mat(c, c);
            for (int m = 0; m < c; ++m) d -= mat(c, m) * mat(c, m);
            if (!(d > 0.0)) { fact_ok = false; d = 1e-300; }
            const double rl = 1.0 / sqrt(d);
            mat(c, c) = rl;
            for (int r = c + 1; r < k; ++r) {
                double sacc = mat(r, c);
                for (int m = 0; m < c; ++m) sacc -= mat(r, m) * mat(c, m);
                mat(r, c) = sacc * rl;
            }
        }
        // forward: u = L^-1 1, v = L^-1 c~_S
        for (int r = 0; r < k; ++r) {
            double su = 1.0;
            double sv = (double)a.c_hi[base + idx[r]] + (double)a.c_lo[base + idx[r]];
            for (int m = 0; m < r; ++m) { su -= mat(r, m) * u[m]; sv -= mat(r, m) * v[m]; }
            u[r] = su * mat(r, r);
            v[r] = sv * mat(r, r);
        }
        a11 = 0.0;
        double a1b = 0.0;
        for (int r = 0; r < k; ++r) { a11 += u[r] * u[r]; a1b += u[r] * v[r]; }
        nu = (a1b - 1.0) / a11;
        // back: xs = L^-T (v - nu u), u <- L^-T u (= G~_SS^-1 1)
        for (int r = k - 1; r >= 0; --r) {
            double sx = v[r] - nu * u[r], su = u[r];
            for (int m = r + 1; m < k; ++m) { sx -= mat(m, r) * xs[m]; su -= mat(m, r) * u[m]; }
            xs[r] = sx * mat(r, r);
            u[r] = su * mat(r, r);
        }
        if (!fact_ok) break;
        // most negative coordinate on S
        int rneg = -1;
        double xmin = -a.tol_x;
        xsum = 0.0;
        for (int r = 0; r < k; ++r) {
            if (xs[r] < xmin) { xmin = xs[r]; rneg = r; }
            xsum += fmax(xs[r], 0.0);
        }
        if (rneg >= 0) {
            if (sw == a.max_swaps || k == 1) break;
            for (int r = rneg; r + 1 < k; ++r) idx[r] = idx[r + 1];
            --k;
            continue;
        }
        // most negative multiplier off S, in double-float (G~ and x_S as
        // float32 hi + lo pairs) on the float32 pipes
        float xh[KMAX], xl[KMAX];
        for (int r = 0; r < k; ++r) {
            const df d = split_double(xs[r]);
            xh[r] = d.hi; xl[r] = d.lo;
        }
        const df nud = split_double(nu);
        int iadd = -1;
        double lmin = -a.tol_g;
        {
            int r = 0;
            for (int i = 0; i < P; ++i) {
                if (r < k && idx[r] == i) { ++r; continue; }
                dot2 g;
                const float *ghi = a.Ghi + (size_t)i * a.PP, *glo = a.Glo + (size_t)i * a.PP;
                for (int q = 0; q < k; ++q) {
                    const float gh = __ldg(ghi + idx[q]), gl = __ldg(glo + idx[q]);
                    g.add_prod(gh, xh[q]);
                    g.c = fmaf(gh, xl[q], fmaf(gl, xh[q], g.c));
                }
                g.add_df(df{-a.c_hi[base + i], -a.c_lo[base + i]});
                g.add_df(nud);
                const df gv = g.result();
                const double lam_i = (double)gv.hi + (double)gv.lo;
                if (lam_i < lmin) { lmin = lam_i; iadd = i; }
            }
        }
        if (iadd >= 0) {
            if (sw == a.max_swaps || k >= KMAX) break;
            int r = k;
            while (r > 0 && idx[r - 1] > iadd) { idx[r] = idx[r - 1]; --r; }
            idx[r] = iadd;
            ++k;
            continue;
        }
        ok = xsum > 0.0;
        break;
    }
    if (!ok) {
        if (a.retry_list) {
            const unsigned long long pos = atomicAdd(a.retry_len, 1ULL);
            a.retry_list[pos] = n;
        }
        if (a.n_unverified) atomicAdd(a.n_unverified, 1ULL);
    }
    // abundances: the crossover solution, or the interior-point iterate
    if (ok) {
        int r = 0;
        for (int i = 0; i < P; ++i) {
            float xi = 0.f;
            if (r < k && idx[r] == i) { xi = (float)(fmax(xs[r], 0.0) / xsum); ++r; }
            a.x_out[base + i] = xi;
        }
    } else if (a.x_out != a.x_in) {
        for (int i = 0; i < P; ++i) a.x_out[base + i] = a.x_in[base + i];
    }
    // uncertainties on the final support: [K^-1]_rr = (G~_SS^-1)_rr - u_r^2 / (1^T G~_SS^-1 1)
    if (a.sx_out) {
        const double s = a.scale[0];
        double w[KMAX];
        int r = 0;
        for (int i = 0; i < P; ++i) {
            float out = 0.f;
            if (r < k && idx[r] == i) {
                // column r of L^-1: w_r = 1/L_rr, w_m = -(sum_{q=r}^{m-1} L_mq w_q)/L_mm
                double dinv = 0.0;
                for (int m = r; m < k; ++m) {
                    double sacc = (m == r) ? 1.0 : 0.0;
                    for (int q = r; q < m; ++q) sacc -= mat(m, q) * w[q];
                    w[m] = sacc * mat(m, m);
                    dinv += w[m] * w[m];
                }
                const double var = dinv - u[r] * u[r] / a11;
                out = (float)sqrt(fmax(var, 0.0) / s);
                ++r;
            }
            a.sx_out[base + i] = out;
        }
    }
}

template <int KMAX>
static cudaError_t launch_refine_t(const RefineArgs &a, cudaStream_t st)
{
    const size_t smem = sizeof(double) * (size_t)a.P * a.P;
    cudaError_t e = cudaFuncSetAttribute(refine_kernel<KMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (a.N + REF_THREADS - 1) / REF_THREADS;   // list mode: <= N entries
    refine_kernel<KMAX><<<(unsigned)blocks, REF_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_refine(const RefineArgs &a, cudaStream_t st)
{
    if (a.N <= 0) return cudaSuccess;
    if (a.P <= 16) return launch_refine_t<16>(a, st);
    if (a.P <= 32) return launch_refine_t<32>(a, st);
    if (a.P <= 48) return launch_refine_t<48>(a, st);
    return launch_refine_t<64>(a, st);
}

// ------------------------------------------------------------------- rms
constexpr int RMS_THREADS = 128;

template <int NJ4>
__global__ void __launch_bounds__(RMS_THREADS)
rms_kernel(const float *__restrict__ cube, const float *__restrict__ S,
           const float *__restrict__ x, long long N, int L, int P, float *__restrict__ rms)
{
    constexpr int PQ = 4 * NJ4;
    extern __shared__ __align__(16) float st[];   // [l][PQ] = S^T, zero padded
    for (int e = threadIdx.x; e < L * PQ; e += blockDim.x) {
        const int l = e / PQ, j = e % PQ;
        st[e] = j < P ? S[(size_t)j * L + l] : 0.f;
    }
    __syncthreads();
    const long long n = (long long)blockIdx.x * RMS_THREADS + threadIdx.x;
    if (n >= N) return;
    float xv[PQ];
#pragma unroll
    for (int j = 0; j < PQ; ++j) xv[j] = j < P ? x[(size_t)n * P + j] : 0.f;
    const float *y = cube + (size_t)n * L;
    float acc = 0.f;
    for (int l = 0; l < L; ++l) {
        float m = 0.f;
        const float *row = st + (size_t)l * PQ;
#pragma unroll
        for (int j4 = 0; j4 < NJ4; ++j4) {
            const float4 sv = *reinterpret_cast<const float4 *>(row + 4 * j4);
            m = fmaf(xv[4 * j4 + 0], sv.x, m);
            m = fmaf(xv[4 * j4 + 1], sv.y, m);
            m = fmaf(xv[4 * j4 + 2], sv.z, m);
            m = fmaf(xv[4 * j4 + 3], sv.w, m);
        }
        const float e = __ldg(y + l) - m;
        acc = fmaf(e, e, acc);
    }
    rms[n] = sqrtf(acc / (float)L);
}

template <int NJ4>
static cudaError_t launch_rms_t(const float *cube, const float *S, const float *x, long long N,
                                int L, int P, float *rms, cudaStream_t st)
{
    const size_t smem = sizeof(float) * (size_t)L * 4 * NJ4;
    cudaError_t e = cudaFuncSetAttribute(rms_kernel<NJ4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (N + RMS_THREADS - 1) / RMS_THREADS;
    rms_kernel<NJ4><<<(unsigned)blocks, RMS_THREADS, smem, st>>>(cube, S, x, N, L, P, rms);
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
