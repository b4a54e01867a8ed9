// Projection c~ = B~^T y + rho on the 5th-generation tensor cores (tcgen05).
//
// c = S W^2 y / s is a dense contraction (N pixels x L bands x P spectra)
// with one operand shared by every pixel, so it belongs on the tensor
// cores; but the fully constrained solve needs c to ~1e-11 relative (the
// constrained problem is ill-conditioned: rounding c to float32 moves x by
// up to 1e-2), far beyond bf16 or tf32 inputs with float32 accumulation.
//
// Exact mode (LINMIN_PROJ_TC): every pixel row is scaled by a power of two
// so that |y_l| < 1/2 and cut into NS integer slices of 8 bits each,
//     y_l 2^-e = sum_i a_il 2^-8(i+1),   a_i in [-128, 128]
// (round-to-nearest residues, exact in float32), and every column of B~
// likewise (exponent f_j, slices b_qlj).  The integers are exact in bf16;
// the products a b (<= 2^14) are exact in float32 and, summed over at most
// 192 bands and the <= 5 slice pairs of one level l = i + q, stay below
// 2^24, so the tensor core's float32 accumulation is exact too.  The 15 slice pairs with
// i + q <= 4 accumulate into 5 TMEM accumulators (one per level); every 192
// bands each thread adds them, weighted 2^-8(l+2), to double-float sums,
// and c_j = 2^(e + f_j) sum + rho.  Dropped terms (the slice residues and
// the levels above 4) are below 2^-39 of max|y| max|B_j| per band: the
// accuracy the solve needs (~1e-11 relative), as with the double-float
// projection.
//
// BF16 mode (LINMIN_PROJ_BF16): one slice each, the bf16 roundings of y
// and B~ (no scaling): "bf16 in, float32 accumulate" of the CRISM-shaped
// workload's precision study.
//
// Kernels: with 16-byte strided rows, project_ws_kernel (warp-specialised,
// TMA-fed, one CTA per SM; its roles are described at the kernel) after a
// per-pixel exponent pass; otherwise, and for the bf16 mode,
// project_tc_kernel (two CTAs per SM, 64-band chunks loaded by the threads
// themselves, one CTA slicing while the other's MMAs run).  Both read the B~
// slices prepared once per call in the MMA's canonical K-major layout, one
// matrix of 5 NPAD stacked rows per 32 bands; both form the same digits and
// exact level sums and fold them in the same order (their double-float
// additions of the group sums differ).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "linmin.h"

namespace lm {

namespace {

constexpr int TC_M = 128;           // pixels per tile = MMA M = TMEM lanes
constexpr int TC_KC = 64;           // bands per chunk
constexpr int TC_THREADS = 256;     // 8 warps
constexpr int TC_GROUP = 3;         // chunks per exact accumulation group (192 bands)
// TMEM columns a CTA allocates: a power of two >= the NL * NPAD accumulators
__host__ __device__ constexpr int tc_tmem_cols(int need) { return need <= 256 ? 256 : 512; }
constexpr long long WAIT_LIMIT = 1LL << 26;   // bounded mbarrier wait (error flag)

__device__ __forceinline__ uint32_t su32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// canonical K-major layout without swizzle: core matrices of 8 rows x 16 B
// (8 bf16 along K); element (r, k) of an R x K tile at this byte offset
__host__ __device__ __forceinline__ int kmaj(int r, int k, int R)
{
    return ((k >> 3) * (R >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: start, leading (K-adjacent core
// matrices) and stride (8-row groups) byte offsets, version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: bf16 A and B, float32 D, both
// K-major, N and M
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    for (long long i = 0; i < WAIT_LIMIT && !done; ++i)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive floats of row n from band l0 (zeros past L)
__device__ __forceinline__ void load8(const float *cube, long long n, int L, int l0, bool vec,
                                      float (&v)[8])
{
    const float *y = cube + (size_t)n * L + l0;
    if (vec && l0 + 8 <= L) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(y));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(y) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = l0 + q < L ? __ldg(y + q) : 0.f;
    }
}

// eight values rounded to bf16, packed in K order (one core-matrix row)
__device__ __forceinline__ uint4 pack8(const float (&v)[8])
{
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t *>(&b);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// 2^k as a float for -126 <= k <= 127
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }


// exact slice count and levels of a mode
template <int MODE> struct TcMode;
template <> struct TcMode<LINMIN_PROJ_TC> { static constexpr int NS = 5, NL = 5; };
template <> struct TcMode<LINMIN_PROJ_BF16> { static constexpr int NS = 1, NL = 1; };

}  // namespace

// ---------------------------------------------------------------- B~ slices
// B~ = T / s with T = W^2 S^T (T_lj = S_jl / sigma_l^2, formed here from S
// and sigma) or T = C^-1 S^T (given, L x P).
__device__ __forceinline__ double tc_T(const float *__restrict__ S, const float *__restrict__ sigma,
                                       const double *__restrict__ Tin, int L, int P, int l, int j)
{
    if (Tin) return Tin[(size_t)l * P + j];
    const double sg = (double)sigma[l];
    return (double)S[(size_t)j * L + l] / (sg * sg);
}

// Column exponents f_j: max_l |B~_lj| < 2^f_j (exact mode).  Block per
// column, a band per thread (the fp64 divisions of a column in parallel).
constexpr int BEXP_THREADS = 256;

__global__ void __launch_bounds__(BEXP_THREADS)
tc_bexp_kernel(const float *__restrict__ S, const float *__restrict__ sigma,
               const double *__restrict__ Tin, int L, int P, const double *__restrict__ scale,
               int *__restrict__ fexp)
{
    __shared__ double wmax[BEXP_THREADS / 32];
    const int j = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double s = scale[0];
    double m = 0.0;
    for (int l = threadIdx.x; l < L; l += BEXP_THREADS)
        m = fmax(m, fabs(tc_T(S, sigma, Tin, L, P, l, j) / s));
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) wmax[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < BEXP_THREADS / 32; ++w) m = fmax(m, wmax[w]);
        int e = 0;
        if (m > 0.0) { frexp(m, &e); ++e; }          // |B~_lj| 2^-f_j < 1/2
        fexp[j] = e;
    }
}

// Slices per 32-band block: one K-major matrix of NS * NPAD rows (slice q,
// column j at row q NPAD + j) and 32 bands, in the MMA's canonical layout:
// an MMA with B = rows [0, (NS - i) NPAD) pairs A slice i with every B slice
// q <= NS - 1 - i at once, and a 64-band chunk is two consecutive blocks.
// Rows j >= P and bands l >= L are zero.
template <int MODE>
__global__ void tc_bslice_kernel(const float *__restrict__ S, const float *__restrict__ sigma,
                                 const double *__restrict__ Tin, int L, int P, int NPAD,
                                 const double *__restrict__ scale, const int *__restrict__ fexp,
                                 __nv_bfloat16 *__restrict__ out, int nblocks)
{
    constexpr int NS = TcMode<MODE>::NS;
    constexpr int KB = TC_KC / 2;                    // bands per block
    const long long total = (long long)nblocks * NPAD * KB;
    const double s = scale[0];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / (NPAD * KB));
        const int rem = (int)(e % (NPAD * KB));
        const int j = rem / KB, k = rem % KB;
        const int l = c * KB + k;
        const double v = (j < P && l < L) ? tc_T(S, sigma, Tin, L, P, l, j) / s : 0.0;
        char *blk = reinterpret_cast<char *>(out) + (size_t)c * NS * NPAD * KB * 2;
        if (MODE == LINMIN_PROJ_BF16) {
            *reinterpret_cast<__nv_bfloat16 *>(blk + kmaj(j, k, NPAD)) = __double2bfloat16(v);
        } else {
            double r = j < P ? ldexp(v, -fexp[j]) : 0.0;     // |r| < 1/2, exact scaling
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const double t = r * 256.0;
                const double a = rint(t);
                r = t - a;
                *reinterpret_cast<__nv_bfloat16 *>(blk + kmaj(q * NPAD + j, k, NS * NPAD)) =
                    __double2bfloat16(a);
            }
        }
    }
}

// ---------------------------------------------------------------- the GEMM
template <int NPAD, int MODE>
__global__ void __launch_bounds__(TC_THREADS, TcMode<MODE>::NL * NPAD <= 256 ? 2 : 1)
project_tc_kernel(const float *__restrict__ cube, long long N, int L, int P,
                  const __nv_bfloat16 *__restrict__ bsl, const int *__restrict__ fexp,
                  float *__restrict__ c_hi, float *__restrict__ c_lo, int *__restrict__ err)
{
    constexpr int NS = TcMode<MODE>::NS, NL = TcMode<MODE>::NL;
    constexpr int A_SLICE = TC_M * TC_KC * 2;        // bytes of one pixel slice
    constexpr int B_SLICE = NPAD * TC_KC * 2;        // bytes of one B~ slice
    constexpr int HALF = NPAD / 2;                   // columns per epilogue warp
    constexpr int TMEM_COLS = tc_tmem_cols(NL * NPAD);
    static_assert(NL * NPAD <= TMEM_COLS, "TMEM columns");
    static_assert(HALF % 8 == 0, "epilogue loads 8 columns at a time");
    static_assert(TC_M * (TC_KC / 8) % TC_THREADS == 0, "slicing items per thread");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                        // NS pixel slices
    unsigned char *sB = smem + NS * A_SLICE;         // NS B~ slices
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ int pexp[TC_M];                       // per-pixel exponents

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunks = (L + TC_KC - 1) / TC_KC;
    const bool vec = (L % 4) == 0 && (reinterpret_cast<uintptr_t>(cube) % 16) == 0;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&tbase)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tbase;
    uint32_t phase = 0;
    bool ok = true;

    // epilogue role: TMEM lanes of warp (warp & 3), columns of half (warp >> 2)
    const int ep_pix = 32 * (warp & 3) + lane;
    const int ep_col0 = HALF * (warp >> 2);

    const long long ntiles = (N + TC_M - 1) / TC_M;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long p0 = tile * TC_M;
        // per-pixel exponent (max |y| over the row < 2^e): items of 8
        // consecutive bands, consecutive pixels on consecutive lanes
        for (int i = tid; i < TC_M; i += TC_THREADS) pexp[i] = 0;   // float bits of +0
        __syncthreads();
        if (MODE == LINMIN_PROJ_TC) {
            const int noct = (L + 7) / 8;
#pragma unroll 4
            for (int it = tid; it < TC_M * noct; it += TC_THREADS) {
                const int pix = it % TC_M, oct = it / TC_M;
                const long long n = p0 + pix;
                float yv[8];
                if (n < N) load8(cube, n, L, 8 * oct, vec, yv);
                else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) yv[q] = 0.f;
                }
                float m = 0.f;
#pragma unroll
                for (int q = 0; q < 8; ++q) m = fmaxf(m, fabsf(yv[q]));
                atomicMax(pexp + pix, __float_as_int(m));     // m >= 0: int order = float order
            }
            __syncthreads();
            for (int i = tid; i < TC_M; i += TC_THREADS) {
                const float m = __int_as_float(pexp[i]);
                int e = 0;
                if (m > 0.f) { frexpf(m, &e); ++e; }     // |y_l| 2^-e < 1/2
                pexp[i] = e;
            }
        }
        df acc[HALF];
#pragma unroll
        for (int j = 0; j < HALF; ++j) acc[j] = df_make(0.f);

        for (int c = 0; c < nchunks && ok; ++c) {
            // B~ slices of the chunk (16-byte copies of the prepared layout)
            {
                const uint4 *src = reinterpret_cast<const uint4 *>(
                    reinterpret_cast<const char *>(bsl) + (size_t)c * NS * B_SLICE);
                uint4 *dst = reinterpret_cast<uint4 *>(sB);
#pragma unroll 8
                for (int e = tid; e < NS * B_SLICE / 16; e += TC_THREADS) dst[e] = __ldg(src + e);
            }
            // pixel slices: items of 8 consecutive bands of one pixel, one
            // 16-byte shared store per slice (a row of a core matrix); the
            // thread's loads are all issued before any slicing
            constexpr int ITEMS = TC_M * (TC_KC / 8) / TC_THREADS;
            float yv[ITEMS][8];
#pragma unroll
            for (int u = 0; u < ITEMS; ++u) {
                const int it = tid + u * TC_THREADS;
                const long long n = p0 + (it % TC_M);
                if (n < N) load8(cube, n, L, c * TC_KC + 8 * (it / TC_M), vec, yv[u]);
                else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) yv[u][q] = 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < ITEMS; ++u) {
                const int it = tid + u * TC_THREADS;
                const int pix = it % TC_M, oct = it / TC_M;
                const int off = kmaj(pix, 8 * oct, TC_M);
                if (MODE == LINMIN_PROJ_BF16) {
                    *reinterpret_cast<uint4 *>(sA + off) = pack8(yv[u]);
                } else {
                    const int e = pexp[pix];
                    float r[8];
                    const int h = e / 2;
                    const float f1 = pow2f(-h), f2 = pow2f(h - e);
#pragma unroll
                    for (int q = 0; q < 8; ++q) r[q] = yv[u][q] * f1 * f2;       // exact
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        float a[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float t = r[q] * 256.f;
                            a[q] = rintf(t);
                            r[q] = t - a[q];
                        }
                        *reinterpret_cast<uint4 *>(sA + i * A_SLICE + off) = pack8(a);
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            const bool first = (c % TC_GROUP) == 0;
            if (tid == 0) {
                constexpr uint32_t ID = idesc_bf16(TC_M, NPAD);
                // A: K-adjacent core matrices 16 x 128 B apart, 8-row groups
                // 128 B; B: two 32-band blocks of NS NPAD stacked rows
                constexpr uint32_t LBO_A = (TC_M / 8) * 128, LBO_B = (NS * NPAD / 8) * 128;
                constexpr uint32_t BLK_B = NS * NPAD * (TC_KC / 2) * 2;
#pragma unroll
                for (int lv = 0; lv < NL; ++lv) {
                    bool fresh = first;
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        const int q = lv - i;
                        if (q < 0 || q >= NS) continue;
#pragma unroll
                        for (int kk = 0; kk < TC_KC / 16; ++kk) {
                            const uint64_t ad = sdesc(su32(sA + i * A_SLICE) + kk * 2 * LBO_A, LBO_A, 128);
                            const uint64_t bd = sdesc(su32(sB) + (kk >> 1) * BLK_B + q * NPAD * 16 +
                                                          (kk & 1) * 2 * LBO_B, LBO_B, 128);
                            mma_bf16(tmem + (uint32_t)(lv * NPAD), ad, bd, ID, fresh ? 0u : 1u);
                            fresh = false;
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(su32(&mbar)));
            }
            ok = __syncthreads_and(mbar_wait(su32(&mbar), phase));
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!ok) {
                // flag the error, give the MMAs in flight a second bounded
                // wait, then leave (TMEM is freed below)
                if (tid == 0) atomicOr(err, 4);
                mbar_wait(su32(&mbar), phase ^ 1u);
                break;
            }
            // end of an exact group (or of the row): fold the levels in
            if ((c % TC_GROUP) == TC_GROUP - 1 || c == nchunks - 1) {
                // per column: sum_l acc_l 2^-8(l+2) from the smallest level up
                // with TwoSum (every term is exact), then into the df total
#pragma unroll
                for (int j8 = 0; j8 < HALF / 8; ++j8) {
                    float sh[8], sl[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) { sh[q] = 0.f; sl[q] = 0.f; }
#pragma unroll
                    for (int lv = NL - 1; lv >= 0; --lv) {
                        const float w = MODE == LINMIN_PROJ_BF16 ? 1.f : ldexpf(1.f, -8 * (lv + 2));
                        float v[8];
                        tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) +
                                     (uint32_t)(lv * NPAD + ep_col0 + 8 * j8), v);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            float t, e;
                            two_sum(sh[q], v[q] * w, t, e);
                            sh[q] = t;
                            sl[q] += e;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        acc[8 * j8 + q] = df_add(acc[8 * j8 + q], df{sh[q], sl[q]});
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();            // shared slices and TMEM free for the next chunk
        }
        // c~_j = 2^(e + f_j) acc + rho
        const long long n = p0 + ep_pix;
        if (ok && n < N) {
            const int e = pexp[ep_pix];
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                const int col = ep_col0 + j;
                if (col < P) {
                    const int sh = MODE == LINMIN_PROJ_BF16 ? 0 : e + fexp[col];
                    df v = df{ldexpf(acc[j].hi, sh), ldexpf(acc[j].lo, sh)};
                    v = df_add(v, df_make((float)RHO));
                    c_hi[(size_t)n * P + col] = v.hi;
                    c_lo[(size_t)n * P + col] = MODE == LINMIN_PROJ_BF16 ? 0.f : v.lo;
                }
            }
        }
        __syncthreads();                // pexp reused by the next tile
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(TMEM_COLS));
}

// --------------------------------------------------- TMA-fed exact GEMM
// Per-pixel exponents (max_l |y_l| < 2^e) in one coalesced pass: a
// half-warp per row (16-byte loads; this path requires 16-byte strided
// rows), a warp takes 8 consecutive rows per step, every load of a step
// issued before the reductions; grid-stride over the cube.
constexpr int ROWEXP_ROWS = 8;

__global__ void tc_rowexp_kernel(const float *__restrict__ cube, long long N, int L,
                                 int *__restrict__ rexp)
{
    const int lane = threadIdx.x & 31, hw = lane >> 4, hl = lane & 15;
    const int L4 = L / 4;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long n0 = w0 * ROWEXP_ROWS; n0 < N; n0 += nw * ROWEXP_ROWS) {
        float m[ROWEXP_ROWS / 2];
#pragma unroll
        for (int r = 0; r < ROWEXP_ROWS / 2; ++r) m[r] = 0.f;
        for (int l = hl; l < L4; l += 16) {
            float4 v[ROWEXP_ROWS / 2];
#pragma unroll
            for (int r = 0; r < ROWEXP_ROWS / 2; ++r) {
                const long long n = n0 + 2 * r + hw;
                v[r] = n < N ? __ldg(reinterpret_cast<const float4 *>(cube + (size_t)n * L) + l)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < ROWEXP_ROWS / 2; ++r)
                m[r] = fmaxf(fmaxf(m[r], fmaxf(fabsf(v[r].x), fabsf(v[r].y))),
                             fmaxf(fabsf(v[r].z), fabsf(v[r].w)));
        }
#pragma unroll
        for (int r = 0; r < ROWEXP_ROWS / 2; ++r)
            for (int off = 8; off > 0; off >>= 1)
                m[r] = fmaxf(m[r], __shfl_xor_sync(0xffffffffu, m[r], off));
        if (hl < ROWEXP_ROWS / 2) {
            float mm = m[0];
#pragma unroll
            for (int r = 1; r < ROWEXP_ROWS / 2; ++r) mm = hl == r ? m[r] : mm;
            const long long n = n0 + 2 * hl + hw;
            int e = 0;
            if (mm > 0.f) { frexpf(mm, &e); ++e; }   // |y_l| 2^-e < 1/2
            if (n < N) rexp[n] = e;
        }
    }
}

cudaError_t launch_rowexp(const float *cube, long long N, int L, int *rexp, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long warps = (N + ROWEXP_ROWS - 1) / ROWEXP_ROWS;
    const long long blocks = (warps * 32 + 255) / 256;
    tc_rowexp_kernel<<<(unsigned)(blocks < 8LL * sms ? blocks : 8LL * sms), 256, 0, st>>>(cube, N, L,
                                                                                         rexp);
    return cudaGetLastError();
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

// Wait for a phase (try_wait suspends the thread in the barrier for a
// while between tests), give up when another role of the CTA has (abort
// flag), and set the flag after WS_WAIT_NS of global time.
constexpr unsigned long long WS_WAIT_NS = 2000000000ull;

__device__ __forceinline__ bool ws_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    unsigned long long t0 = 0;
    for (;;) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if (*abort_flag) return false;
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > WS_WAIT_NS) {
            *abort_flag = 1;
            return false;
        }
    }
}

// packed double-float pieces (two columns per instruction); a - b as
// fma(b, -1, a): one rounding, the value of a float subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    const float2 aa = sub2(s, bb);
    e = __fadd2_rn(sub2(a, aa), sub2(b, bb));
}
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    e = sub2(b, sub2(s, a));
}

// 8 TMEM columns of the warp's 32 lanes; valid after tmem_wait_ld
__device__ __forceinline__ void tmem_ld8_async(uint32_t addr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
}

// wait for the loads in flight; the registers pass through an empty asm
// after the wait so that no use is scheduled before it
template <int NL>
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[NL][8])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int lv = 0; lv < NL; ++lv)
        asm volatile("" : "+r"(r[lv][0]), "+r"(r[lv][1]), "+r"(r[lv][2]), "+r"(r[lv][3]),
                          "+r"(r[lv][4]), "+r"(r[lv][5]), "+r"(r[lv][6]), "+r"(r[lv][7]));
}

namespace {

// Warp-specialised exact projection: 32-band chunks (one 128-byte row per
// pixel, so the tile is read with the 128-byte swizzle and without bank
// conflicts), groups of 6 chunks (192 bands) per exact accumulation.
constexpr int WS_KC = 32;
constexpr int WS_GROUP = TC_GROUP * TC_KC / WS_KC;
constexpr int WS_SLICE_WARPS = 8;
constexpr int WS_EPI_WARPS = 8;
constexpr int WS_FIRST_SLICER = 3;          // warps 0-2: two producers and the MMA issuer
constexpr int WS_THREADS = 32 * (WS_FIRST_SLICER + WS_SLICE_WARPS + WS_EPI_WARPS);
constexpr float WS_MAGIC = 12582912.f;       // 1.5 2^23: fl(t + WS_MAGIC) - WS_MAGIC = rint(t), |t| < 2^22

template <int NPAD> struct Ws {
    static constexpr int NS = TcMode<LINMIN_PROJ_TC>::NS, NL = TcMode<LINMIN_PROJ_TC>::NL;
    static constexpr int SY = NPAD <= 32 ? 4 : NPAD <= 48 ? 3 : 2;   // pixel-tile stages
    static constexpr int SB = NPAD <= 48 ? 3 : 2;                     // B~ stages
    static constexpr int NSETS = 2 * NL * NPAD <= 512 ? 2 : 1;       // TMEM accumulator sets
    static constexpr int COLS = NSETS * NL * NPAD;
    static constexpr int TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128
                                     : COLS <= 256 ? 256 : 512;
    static constexpr int Y_BYTES = TC_M * WS_KC * 4;              // fp32 pixel tile of a chunk
    static constexpr int B_BYTES = NS * NPAD * WS_KC * 2;         // the chunk's stacked B~ slices
    static constexpr int A_SLICE = TC_M * WS_KC * 2;              // one pixel slice of a chunk
    static constexpr int A_BYTES = NS * A_SLICE;
    // staging tile of c~ (hi and lo words of 128 rows of P floats) last
    static constexpr int FIXED = SY * Y_BYTES + SB * B_BYTES + 2 * A_BYTES + 1024;
    static constexpr int smem(int P) { return FIXED + 2 * TC_M * P * 4; }
    static_assert(COLS <= 512, "TMEM columns");
    static_assert((NPAD / 8) % 2 == 0, "the two epilogue halves take whole 8-column batches");
    static_assert(FIXED + 2 * TC_M * NPAD * 4 + 1024 <= 232448, "shared memory");
};

// Position of a role in the CTA's chunk sequence, advanced one chunk at a
// time (no divisions in the loops): pixel-tile stage, B~ stage and A slot
// with their phases, chunk of the tile, tile, accumulator set and phase.
template <int SY, int SB, int NSETS> struct WsPos {
    int sy = 0, py = 0, sb = 0, pb = 0, k = 0, pk = 0, c = 0, aset = 0, pa = 0;
    long long tile;
    __device__ explicit WsPos(long long t0) : tile(t0) {}
    __device__ bool group_first() const { return c % WS_GROUP == 0; }
    __device__ bool group_last(int nch) const { return c % WS_GROUP == WS_GROUP - 1 || c == nch - 1; }
    __device__ void next(int nch, long long tile_step)
    {
        if (group_last(nch) && ++aset == NSETS) { aset = 0; pa ^= 1; }
        if (++sy == SY) { sy = 0; py ^= 1; }
        if (++sb == SB) { sb = 0; pb ^= 1; }
        if ((k ^= 1) == 0) pk ^= 1;
        if (++c == nch) { c = 0; tile += tile_step; }
    }
};

}  // namespace

// Roles (one CTA per SM, persistent over 128-pixel tiles; chunk g of the CTA
// is chunk g % nch of its tile g / nch):
//   warp 0      pixel-tile producer: the tile of the chunk (tensor map,
//               128-byte swizzle, zero fill past N and L) into stage g % SY;
//   warp 2      B~ producer: the chunk's stacked B~ slices into stage g % SB
//               (two producers, so that neither ring throttles the other);
//   warp 1      MMA issuer: per K-step one MMA per A slice i against the
//               B~ rows of slices 0 .. 4 - i, into accumulator set (group
//               index) % NSETS; commits free the B~ stage and the A slot,
//               and at a group end fill the set;
//   warps 3-10  slicers: pixel tile -> five 8-bit slices of every band
//               (stored negated, see below) into A slot g % 2; they free
//               the pixel-tile stage as soon as it is read;
//   warps 11-18 epilogue: the five level accumulators of a group folded into
//               double-float, scaled by 2^(e + f_j), + rho, into a staging
//               tile (which also holds the partial sums between groups),
//               then copied to c~ with coalesced stores.
// The slicers compute each digit as fl(t + 1.5 2^23) - 1.5 2^23 with
// packed fp32 FMAs: round-to-nearest-even, the digits rintf gives.  They
// store -a (its bf16 is the top half of the fp32 word, the digit having at
// most 8 significant bits); the sign comes back, exactly, in the epilogue.
template <int NPAD>
__global__ void __launch_bounds__(WS_THREADS, 1)
project_ws_kernel(const __grid_constant__ CUtensorMap ymap, long long N, int L, int P,
                  const __nv_bfloat16 *__restrict__ bsl, const int *__restrict__ fexp,
                  const int *__restrict__ rexp, float *__restrict__ c_hi,
                  float *__restrict__ c_lo, int *__restrict__ err)
{
    using C = Ws<NPAD>;
    constexpr int NS = C::NS, NL = C::NL, SY = C::SY, SB = C::SB, NSETS = C::NSETS;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t y_full[SY], y_empty[SY], b_full[SB], b_empty[SB];
    __shared__ __align__(8) uint64_t a_full[2], a_empty[2], acc_full[NSETS], acc_empty[NSETS];
    __shared__ __align__(8) uint64_t drain, epi_full, epi_free;
    __shared__ uint32_t tbase;
    __shared__ int abort_flag;
    __shared__ int sfexp[NPAD];
    __shared__ __align__(16) uint32_t sfbits[NPAD];  // bits of -2^f_j (exponent field + sign)
    __shared__ int sfrange[2];                        // min, max of f_j over j < P

    const uint32_t raw = su32(smem_raw);
    unsigned char *sY = smem_raw + (((raw + 1023u) & ~1023u) - raw);   // 1024-byte aligned
    unsigned char *sB = sY + SY * C::Y_BYTES;
    unsigned char *sA = sB + SB * C::B_BYTES;
    float *sOh = reinterpret_cast<float *>(sA + 2 * C::A_BYTES);        // staging tile [128][P]
    float *sOl = sOh + TC_M * P;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = (L + WS_KC - 1) / WS_KC;
    const int ngroups = (nch + WS_GROUP - 1) / WS_GROUP;
    const long long ntiles = (N + TC_M - 1) / TC_M;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long nwork = my_tiles * nch;
    volatile int *abrt = &abort_flag;

    if (tid == 0) {
        for (int s = 0; s < SY; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&y_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                         :: "r"(su32(&y_empty[s])), "r"(32 * WS_SLICE_WARPS));
        }
        for (int s = 0; s < SB; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&b_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&b_empty[s])));
        }
        for (int k = 0; k < 2; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                         :: "r"(su32(&a_full[k])), "r"(32 * WS_SLICE_WARPS));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&a_empty[k])));
        }
        for (int a = 0; a < NSETS; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&acc_full[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                         :: "r"(su32(&acc_empty[a])), "r"(32 * WS_EPI_WARPS));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&drain)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                     :: "r"(su32(&epi_full)), "r"(32 * WS_EPI_WARPS));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                     :: "r"(su32(&epi_free)), "r"(32 * WS_EPI_WARPS));
        abort_flag = 0;
        int lo = fexp[0], hi = fexp[0];
        for (int j = 1; j < P; ++j) { lo = min(lo, fexp[j]); hi = max(hi, fexp[j]); }
        sfrange[0] = lo;
        sfrange[1] = hi;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int j = tid; j < NPAD; j += WS_THREADS) {
        const int f = j < P ? fexp[j] : 0;
        sfexp[j] = f;
        sfbits[j] = 0x80000000u | ((uint32_t)(127 + f) << 23);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&tbase)), "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tbase;

    if (warp == 0) {
        // ------------------------------------------------------ pixel tiles
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&ymap)) : "memory");
            long long gy = 0;                           // copies issued
            WsPos<SY, SB, NSETS> at(blockIdx.x);
            for (; gy < nwork; at.next(nch, gridDim.x)) {
                if (!ws_wait(su32(&y_empty[at.sy]), (uint32_t)(at.py ^ 1), abrt)) break;
                const uint32_t yb = su32(&y_full[at.sy]);
                mbar_expect_tx(yb, (uint32_t)C::Y_BYTES);
                tma_load_2d(su32(sY + at.sy * C::Y_BYTES), &ymap, at.c * WS_KC,
                            (int)(at.tile * TC_M), yb);
                ++gy;
            }
            // every copy issued has landed before the CTA leaves
            for (int s = 0; s < SY; ++s)
                if (gy > s) mbar_wait(su32(&y_full[s]), (uint32_t)(((gy - 1 - s) / SY) & 1));
        }
        __syncwarp();
    } else if (warp == 2) {
        // ------------------------------------------------------ B~ slices
        if (lane == 0) {
            long long gb = 0;
            WsPos<SY, SB, NSETS> at(blockIdx.x);
            for (; gb < nwork; at.next(nch, gridDim.x)) {
                if (!ws_wait(su32(&b_empty[at.sb]), (uint32_t)(at.pb ^ 1), abrt)) break;
                const uint32_t bb = su32(&b_full[at.sb]);
                mbar_expect_tx(bb, (uint32_t)C::B_BYTES);
                bulk_load(su32(sB + at.sb * C::B_BYTES),
                          reinterpret_cast<const char *>(bsl) + (size_t)at.c * C::B_BYTES,
                          (uint32_t)C::B_BYTES, bb);
                ++gb;
            }
            for (int s = 0; s < SB; ++s)
                if (gb > s) mbar_wait(su32(&b_full[s]), (uint32_t)(((gb - 1 - s) / SB) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t LBO_A = (TC_M / 8) * 128, LBO_B = (NS * NPAD / 8) * 128;
            WsPos<SY, SB, NSETS> at(blockIdx.x);
            for (long long g = 0; g < nwork; ++g, at.next(nch, gridDim.x)) {
                const int k = at.k, aset = at.aset, sb = at.sb;
                const bool first = at.group_first(), last = at.group_last(nch);
                if (first && !ws_wait(su32(&acc_empty[aset]), (uint32_t)(at.pa ^ 1), abrt)) break;
                if (!ws_wait(su32(&a_full[k]), (uint32_t)at.pk, abrt)) break;
                if (!ws_wait(su32(&b_full[sb]), (uint32_t)at.pb, abrt)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint64_t a0 = sdesc(su32(sA + k * C::A_BYTES), LBO_A, 128);
                const uint64_t b0 = sdesc(su32(sB + sb * C::B_BYTES), LBO_B, 128);
                const uint32_t d0 = tmem + (uint32_t)(aset * NL * NPAD);
                // A slice i against B rows [q0 NPAD, q1 NPAD), i.e. the slices
                // q0 <= q < q1 <= NS - i, into the adjacent level columns
                // i + q0 ..: every level accumulator sees each of its slice
                // pairs once; a level is zeroed by the first (i = 0) MMA of
                // a group, which spans all levels (N at most 256 per MMA)
#pragma unroll
                for (int kk = 0; kk < WS_KC / 16; ++kk) {
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        constexpr int QMAX = 256 / NPAD;          // B slices per MMA
#pragma unroll
                        for (int q0 = 0; q0 < NS - i; q0 += QMAX) {
                            const int q1 = q0 + QMAX < NS - i ? q0 + QMAX : NS - i;
                            const uint64_t ad = a0 + (uint64_t)((i * C::A_SLICE + kk * 2 * LBO_A) >> 4);
                            const uint64_t bd = b0 + (uint64_t)((q0 * NPAD * 16 + kk * 2 * LBO_B) >> 4);
                            const bool zero = first && kk == 0 && i == 0;
                            mma_bf16(d0 + (uint32_t)((i + q0) * NPAD), ad, bd,
                                     idesc_bf16(TC_M, (q1 - q0) * NPAD), zero ? 0u : 1u);
                        }
                    }
                }
                mma_commit(su32(&b_empty[sb]));
                mma_commit(su32(&a_empty[k]));
                if (last) mma_commit(su32(&acc_full[aset]));
            }
            // every MMA issued has completed before the CTA leaves
            mma_commit(su32(&drain));
            mbar_wait(su32(&drain), 0);
        }
        __syncwarp();
    } else if (warp < WS_FIRST_SLICER + WS_SLICE_WARPS) {
        // ------------------------------------------------------ slicers
        // thread: one pixel of the tile, octets ob and ob + 2 of each chunk;
        // a warp covers 32 consecutive pixels of one octet, so both its
        // swizzled reads and its core-matrix stores are conflict free
        const int sidx = tid - 32 * WS_FIRST_SLICER;
        const int pix = sidx & (TC_M - 1), ob = sidx >> 7, sw = pix & 7;
        float first_scale = 256.f, f1 = 1.f, f2 = 1.f;
        bool fast = true;
        // exponent of this thread's pixel in tile t (0 past N)
        auto tile_exp = [&](long long t) {
            const long long n = t * TC_M + pix;
            return t < ntiles && n < N ? __ldg(rexp + n) : 0;
        };
        int e_next = tile_exp(blockIdx.x);
        WsPos<SY, SB, NSETS> at(blockIdx.x);
        const float2 k256 = make_float2(256.f, 256.f), kmag = make_float2(WS_MAGIC, WS_MAGIC);
        const float2 kneg = make_float2(-1.f, -1.f);
        for (long long g = 0; g < nwork; ++g, at.next(nch, gridDim.x)) {
            const int k = at.k;
            if (at.c == 0) {
                // the next tile's exponent is loaded a whole tile ahead
                const int e = e_next;
                e_next = tile_exp(at.tile + gridDim.x);
                // y 2^(8-e) in one exact product when 2^(8-e) is a normal
                // float; otherwise the two-factor scaling first
                fast = e >= -119;
                const int h = e / 2;
                f1 = pow2f(-h);
                f2 = pow2f(h - e);
                first_scale = fast ? pow2f(8 - e) : 256.f;
            }
            if (!ws_wait(su32(&y_full[at.sy]), (uint32_t)at.py, abrt)) break;
            if (!ws_wait(su32(&a_empty[k]), (uint32_t)(at.pk ^ 1), abrt)) break;
            const unsigned char *yrow = sY + at.sy * C::Y_BYTES + pix * (WS_KC * 4);
            float4 yv[2][2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int oct = ob + 2 * u;
                yv[u][0] = *reinterpret_cast<const float4 *>(yrow + (((2 * oct) ^ sw) << 4));
                yv[u][1] = *reinterpret_cast<const float4 *>(yrow + (((2 * oct + 1) ^ sw) << 4));
            }
            mbar_arrive(su32(&y_empty[at.sy]));            // the pixel tile is read
            unsigned char *adst = sA + k * C::A_BYTES;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int oct = ob + 2 * u;
                const float4 v0 = yv[u][0], v1 = yv[u][1];
                float2 r[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w),
                               make_float2(v1.x, v1.y), make_float2(v1.z, v1.w)};
                if (!fast) {
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        r[p] = __fmul2_rn(__fmul2_rn(r[p], make_float2(f1, f1)), make_float2(f2, f2));
                }
                float2 sc = make_float2(first_scale, first_scale);
                const int off = kmaj(pix, 8 * oct, TC_M);
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    uint32_t w[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const float2 t = __ffma2_rn(r[p], sc, kmag);      // M + rint(r sc)
                        const float2 na = __ffma2_rn(t, kneg, kmag);     // -rint(r sc), exact
                        if (i + 1 < NS) r[p] = __ffma2_rn(r[p], sc, na); // residue, exact
                        w[p] = __byte_perm(__float_as_uint(na.x), __float_as_uint(na.y), 0x7632);
                    }
                    sc = k256;
                    *reinterpret_cast<uint4 *>(adst + i * C::A_SLICE + off) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(su32(&a_full[k]));
        }
    } else {
        // ------------------------------------------------------ epilogue
        // thread: TMEM lane (pixel) 32 (warp & 3) + lane, column half ew >> 2
        const int ew = warp - WS_FIRST_SLICER - WS_SLICE_WARPS;
        const int q4 = warp & 3, half = ew >> 2;
        const int pix = 32 * q4 + lane, etid = tid - 32 * (WS_FIRST_SLICER + WS_SLICE_WARPS);
        constexpr int NBH = NPAD / 16;                  // 8-column batches per half
        const bool vrow = (P & 3) == 0;                 // staging rows 16-byte aligned
        const bool vout = vrow && (reinterpret_cast<uintptr_t>(c_hi) & 15) == 0 &&
                          (reinterpret_cast<uintptr_t>(c_lo) & 15) == 0;
        float *oh_row = sOh + pix * P, *ol_row = sOl + pix * P;
        int aset = 0, pa = 0;
        bool ok = true;
        for (long long ti = 0; ti < my_tiles && ok; ++ti) {
            const long long t = blockIdx.x + ti * gridDim.x;
            const long long n = t * TC_M + pix;
            const bool valid = n < N;
            const int e = valid ? __ldg(rexp + n) : 0;
            const int rows = (int)(N - t * TC_M < TC_M ? N - t * TC_M : TC_M);
            const uint32_t pe = (uint32_t)(ti & 1);
            // the previous tile's copy has read the staging tile
            ok = __all_sync(0xffffffffu, ws_wait(su32(&epi_free), pe ^ 1u, abrt));
            if (!ok) break;
            for (int grp = 0; grp < ngroups; ++grp, aset = aset + 1 == NSETS ? (pa ^= 1, 0) : aset + 1) {
                ok = __all_sync(0xffffffffu, ws_wait(su32(&acc_full[aset]), (uint32_t)pa, abrt));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const bool lastg = grp == ngroups - 1;
#pragma unroll 1
                for (int bb = 0; bb < NBH; ++bb) {
                    const int col0 = 8 * (half * NBH + bb);
                    uint32_t r[NL][8];
#pragma unroll
                    for (int lv = 0; lv < NL; ++lv)
                        tmem_ld8_async(tmem + ((uint32_t)(32 * q4) << 16) +
                                           (uint32_t)((aset * NL + lv) * NPAD + col0), r[lv]);
                    tmem_wait_ld<NL>(r);
                    if (bb == NBH - 1) {
                        asm volatile("tcgen05.fence::before_thread_sync;");
                        mbar_arrive(su32(&acc_empty[aset]));
                    }
                    if (!valid || col0 >= P) continue;
                    const bool full8 = vrow && col0 + 8 <= P;
                    float ph[8], pl[8];                       // partial of the earlier groups
                    if (grp > 0) {
                        if (full8) {
                            const float4 a = *reinterpret_cast<const float4 *>(oh_row + col0);
                            const float4 b = *reinterpret_cast<const float4 *>(oh_row + col0 + 4);
                            const float4 cc = *reinterpret_cast<const float4 *>(ol_row + col0);
                            const float4 d = *reinterpret_cast<const float4 *>(ol_row + col0 + 4);
                            ph[0] = a.x; ph[1] = a.y; ph[2] = a.z; ph[3] = a.w;
                            ph[4] = b.x; ph[5] = b.y; ph[6] = b.z; ph[7] = b.w;
                            pl[0] = cc.x; pl[1] = cc.y; pl[2] = cc.z; pl[3] = cc.w;
                            pl[4] = d.x; pl[5] = d.y; pl[6] = d.z; pl[7] = d.w;
                        } else {
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                ph[q] = col0 + q < P ? oh_row[col0 + q] : 0.f;
                                pl[q] = col0 + q < P ? ol_row[col0 + q] : 0.f;
                            }
                        }
                    }
                    // per column pair: sum_l acc_l 2^-8(l+2), smallest level
                    // first (TwoSum; every product by the weight is exact),
                    // then into the earlier groups' partial (negated sums)
                    float2 ah[4], al[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const float w4 = pow2f(-8 * (NL + 1));
                        float2 sh = __fmul2_rn(make_float2(__uint_as_float(r[NL - 1][2 * p]),
                                                           __uint_as_float(r[NL - 1][2 * p + 1])),
                                               make_float2(w4, w4));
                        float2 sl = make_float2(0.f, 0.f);
#pragma unroll
                        for (int lv = NL - 2; lv >= 0; --lv) {
                            const float w = pow2f(-8 * (lv + 2));
                            const float2 v = __fmul2_rn(make_float2(__uint_as_float(r[lv][2 * p]),
                                                                    __uint_as_float(r[lv][2 * p + 1])),
                                                        make_float2(w, w));
                            float2 tt, e2;
                            two_sum2(sh, v, tt, e2);
                            sh = tt;
                            sl = __fadd2_rn(sl, e2);
                        }
                        if (grp == 0) {
                            fast_two_sum2(sh, sl, ah[p], al[p]);
                        } else {
                            float2 tt, e2;
                            two_sum2(make_float2(ph[2 * p], ph[2 * p + 1]), sh, tt, e2);
                            e2 = __fadd2_rn(e2, __fadd2_rn(make_float2(pl[2 * p], pl[2 * p + 1]), sl));
                            fast_two_sum2(tt, e2, ah[p], al[p]);
                        }
                    }
                    float oh[8], ol[8];
                    if (lastg) {
                        // c~_j = 2^(e + f_j) acc + rho: the scale is one exact
                        // product (bits of -2^f_j plus e in the exponent field)
                        // when e + f_j is a normal exponent for every j
                        const bool inrange = e + sfrange[0] >= -126 && e + sfrange[1] <= 127;
                        float2 mh[4];
                        if (inrange) {
                            const uint4 b0 = *reinterpret_cast<const uint4 *>(sfbits + col0);
                            const uint4 b1 = *reinterpret_cast<const uint4 *>(sfbits + col0 + 4);
                            const uint32_t e23 = (uint32_t)e << 23;
                            mh[0] = make_float2(__uint_as_float(b0.x + e23), __uint_as_float(b0.y + e23));
                            mh[1] = make_float2(__uint_as_float(b0.z + e23), __uint_as_float(b0.w + e23));
                            mh[2] = make_float2(__uint_as_float(b1.x + e23), __uint_as_float(b1.y + e23));
                            mh[3] = make_float2(__uint_as_float(b1.z + e23), __uint_as_float(b1.w + e23));
                        }
                        const float2 rho = make_float2((float)RHO, (float)RHO);
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            float2 vh, vl;
                            if (inrange) {
                                vh = __fmul2_rn(ah[p], mh[p]);
                                vl = __fmul2_rn(al[p], mh[p]);
                            } else {
                                const int s0 = e + sfexp[col0 + 2 * p], s1 = e + sfexp[col0 + 2 * p + 1];
                                vh = make_float2(-ldexpf(ah[p].x, s0), -ldexpf(ah[p].y, s1));
                                vl = make_float2(-ldexpf(al[p].x, s0), -ldexpf(al[p].y, s1));
                            }
                            // (vh, vl) + rho: TwoSum of the high words, the low
                            // word into the error, renormalised
                            float2 tt, e2, rh, rl;
                            two_sum2(vh, rho, tt, e2);
                            e2 = __fadd2_rn(e2, vl);
                            fast_two_sum2(tt, e2, rh, rl);
                            oh[2 * p] = rh.x; oh[2 * p + 1] = rh.y;
                            ol[2 * p] = rl.x; ol[2 * p + 1] = rl.y;
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            oh[2 * p] = ah[p].x; oh[2 * p + 1] = ah[p].y;
                            ol[2 * p] = al[p].x; ol[2 * p + 1] = al[p].y;
                        }
                    }
                    // into the staging tile (row pix, the layout of c~)
                    if (full8) {
                        *reinterpret_cast<float4 *>(oh_row + col0) = make_float4(oh[0], oh[1], oh[2], oh[3]);
                        *reinterpret_cast<float4 *>(oh_row + col0 + 4) = make_float4(oh[4], oh[5], oh[6], oh[7]);
                        *reinterpret_cast<float4 *>(ol_row + col0) = make_float4(ol[0], ol[1], ol[2], ol[3]);
                        *reinterpret_cast<float4 *>(ol_row + col0 + 4) = make_float4(ol[4], ol[5], ol[6], ol[7]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (col0 + q < P) {
                                oh_row[col0 + q] = oh[q];
                                ol_row[col0 + q] = ol[q];
                            }
                    }
                }
                if (lastg) {
                    // the tile's rows of c~ are contiguous: coalesced copy
                    // once every epilogue thread has staged its values
                    mbar_arrive(su32(&epi_full));
                    ok = ws_wait(su32(&epi_full), pe, abrt);
                    if (!ok) break;
                    const size_t base = (size_t)t * TC_M * P;
                    const int total = rows * P;
                    if (vout) {
                        const float4 *sh4 = reinterpret_cast<const float4 *>(sOh);
                        const float4 *sl4 = reinterpret_cast<const float4 *>(sOl);
                        float4 *gh = reinterpret_cast<float4 *>(c_hi + base);
                        float4 *gl = reinterpret_cast<float4 *>(c_lo + base);
                        for (int i = etid; i < total / 4; i += 32 * WS_EPI_WARPS) {
                            gh[i] = sh4[i];
                            gl[i] = sl4[i];
                        }
                    } else {
                        for (int i = etid; i < total; i += 32 * WS_EPI_WARPS) {
                            c_hi[base + i] = sOh[i];
                            c_lo[base + i] = sOl[i];
                        }
                    }
                    mbar_arrive(su32(&epi_free));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0 && abort_flag) atomicOr(err, 4);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(C::TMEM_COLS));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// the TMA path applies when rows are 16-byte strided and aligned
bool tma_projection_usable(const float *cube, long long N, int L)
{
    return (L % 4) == 0 && (reinterpret_cast<uintptr_t>(cube) % 16) == 0 && N < (1LL << 31) &&
           encode_tiled() != nullptr;
}

template <int NPAD>
static cudaError_t launch_ws_t(const float *cube, long long N, int L, int P,
                               const __nv_bfloat16 *bsl, const int *fexp, const int *rexp,
                               float *c_hi, float *c_lo, int *err, cudaStream_t st)
{
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)L, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)L * 4};
    const cuuint32_t box[2] = {(cuuint32_t)WS_KC, (cuuint32_t)TC_M};
    const cuuint32_t estr[2] = {1, 1};
    if (encode_tiled()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(cube), dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int smem = Ws<NPAD>::smem(P);
    cudaError_t e = cudaFuncSetAttribute(project_ws_kernel<NPAD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ntiles = (N + TC_M - 1) / TC_M;
    const unsigned blocks = (unsigned)(ntiles < sms ? ntiles : sms);
    project_ws_kernel<NPAD><<<blocks, WS_THREADS, smem, st>>>(map, N, L, P, bsl, fexp, rexp,
                                                              c_hi, c_lo, err);
    return cudaGetLastError();
}

cudaError_t launch_project_tma(const float *cube, long long N, int L, int P,
                               const __nv_bfloat16 *bsl, const int *fexp, const int *rexp, float *c_hi,
                               float *c_lo, int *err, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    switch (((P + 15) / 16) * 16) {
    case 16: return launch_ws_t<16>(cube, N, L, P, bsl, fexp, rexp, c_hi, c_lo, err, st);
    case 32: return launch_ws_t<32>(cube, N, L, P, bsl, fexp, rexp, c_hi, c_lo, err, st);
    case 48: return launch_ws_t<48>(cube, N, L, P, bsl, fexp, rexp, c_hi, c_lo, err, st);
    case 64: return launch_ws_t<64>(cube, N, L, P, bsl, fexp, rexp, c_hi, c_lo, err, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ launch
size_t tc_bslice_bytes(int L, int P, int mode)
{
    const int NPAD = ((P + 15) / 16) * 16;
    const int nchunks = (L + TC_KC - 1) / TC_KC;
    const int NS = mode == LINMIN_PROJ_TC ? TcMode<LINMIN_PROJ_TC>::NS : 1;
    return (size_t)nchunks * NS * NPAD * TC_KC * 2;
}

cudaError_t launch_tc_prep(const float *S, const float *sigma, const double *T, int L, int P,
                           const double *scale, int mode, __nv_bfloat16 *bsl, int *fexp,
                           cudaStream_t st)
{
    const int NPAD = ((P + 15) / 16) * 16;
    const int nblocks = 2 * ((L + TC_KC - 1) / TC_KC);
    if (mode == LINMIN_PROJ_TC)
        tc_bexp_kernel<<<P, BEXP_THREADS, 0, st>>>(S, sigma, T, L, P, scale, fexp);
    const long long total = (long long)nblocks * NPAD * (TC_KC / 2);
    const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
    if (mode == LINMIN_PROJ_TC)
        tc_bslice_kernel<LINMIN_PROJ_TC><<<blocks, 256, 0, st>>>(S, sigma, T, L, P, NPAD, scale,
                                                                 fexp, bsl, nblocks);
    else
        tc_bslice_kernel<LINMIN_PROJ_BF16><<<blocks, 256, 0, st>>>(S, sigma, T, L, P, NPAD, scale,
                                                                   fexp, bsl, nblocks);
    return cudaGetLastError();
}

template <int NPAD, int MODE>
static cudaError_t launch_tc_t(const float *cube, long long N, int L, int P,
                               const __nv_bfloat16 *bsl, const int *fexp, float *c_hi,
                               float *c_lo, int *err, cudaStream_t st)
{
    constexpr int NS = TcMode<MODE>::NS;
    const size_t smem = (size_t)NS * (TC_M * TC_KC * 2 + NPAD * TC_KC * 2);
    cudaError_t e = cudaFuncSetAttribute(project_tc_kernel<NPAD, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ntiles = (N + TC_M - 1) / TC_M;
    const long long wave = (long long)sms * (TcMode<MODE>::NL * NPAD <= 256 ? 2 : 1);
    const unsigned blocks = (unsigned)(ntiles < wave ? ntiles : wave);
    project_tc_kernel<NPAD, MODE><<<blocks, TC_THREADS, smem, st>>>(cube, N, L, P, bsl, fexp,
                                                                     c_hi, c_lo, err);
    return cudaGetLastError();
}

cudaError_t launch_project_tc(const float *cube, long long N, int L, int P, int mode,
                              const __nv_bfloat16 *bsl, const int *fexp, float *c_hi,
                              float *c_lo, int *err, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    const int NPAD = ((P + 15) / 16) * 16;
#define LM_TC(NP)                                                                         \
    case NP:                                                                              \
        return mode == LINMIN_PROJ_TC                                                     \
                   ? launch_tc_t<NP, LINMIN_PROJ_TC>(cube, N, L, P, bsl, fexp, c_hi, c_lo, err, st) \
                   : launch_tc_t<NP, LINMIN_PROJ_BF16>(cube, N, L, P, bsl, fexp, c_hi, c_lo, err, st);
    switch (NPAD) {
        LM_TC(16) LM_TC(32) LM_TC(48) LM_TC(64)
    default: return cudaErrorInvalidValue;
    }
#undef LM_TC
}

}  // namespace lm
