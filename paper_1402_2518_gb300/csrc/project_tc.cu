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
// Layout: two CTAs per SM (256 TMEM columns each; one for P > 48), so that
// one CTA slices while the other's MMAs run, persistent over tiles of 128
// pixels; per 64-band chunk the threads write the pixel slices and copy
// the B~ slices (prepared once per call in the MMA's canonical K-major
// layout) to shared memory, one thread issues the MMAs (M = 128, N = P
// padded to 16, K = 16), tcgen05.commit signals an mbarrier, and the
// epilogue reads the accumulators with tcgen05.ld.
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

// x 2^-e exactly (two power-of-two factors keep both in the normal range)
__device__ __forceinline__ float scale_pow2(float x, int e)
{
    const int h = e / 2;
    return x * pow2f(-h) * pow2f(h - e);
}

// df accumulate of a value whose magnitude is close to the total's
__device__ __forceinline__ df df_add_near(df a, float bh, float bl)
{
    float s, e;
    two_sum(a.hi, bh, s, e);
    e += a.lo + bl;
    df r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

// exact slice count and levels of a mode
template <int MODE> struct TcMode;
template <> struct TcMode<LINMIN_PROJ_TC> { static constexpr int NS = 5, NL = 5; };
template <> struct TcMode<LINMIN_PROJ_BF16> { static constexpr int NS = 1, NL = 1; };

}  // namespace

// ---------------------------------------------------------------- B~ slices
// Column exponents f_j: max_l |B~_lj| < 2^f_j (exact mode).  Warp per column.
__global__ void tc_bexp_kernel(const double *__restrict__ T, int L, int P,
                               const double *__restrict__ scale, int *__restrict__ fexp)
{
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= P) return;
    const double s = scale[0];
    double m = 0.0;
    for (int l = lane; l < L; l += 32) m = fmax(m, fabs(T[(size_t)l * P + j] / s));
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
        int e = 0;
        if (m > 0.0) { frexp(m, &e); ++e; }          // |B~_lj| 2^-f_j < 1/2
        fexp[j] = e;
    }
}

// Slices of B~ = T / s in the canonical layout of each 64-band chunk:
// [chunk][slice][NPAD x 64 bf16]; rows j >= P and bands l >= L are zero.
template <int MODE>
__global__ void tc_bslice_kernel(const double *__restrict__ T, int L, int P, int NPAD,
                                 const double *__restrict__ scale, const int *__restrict__ fexp,
                                 __nv_bfloat16 *__restrict__ out, int nchunks)
{
    constexpr int NS = TcMode<MODE>::NS;
    const long long total = (long long)nchunks * NPAD * TC_KC;
    const double s = scale[0];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / (NPAD * TC_KC));
        const int rem = (int)(e % (NPAD * TC_KC));
        const int j = rem / TC_KC, k = rem % TC_KC;
        const int l = c * TC_KC + k;
        const double v = (j < P && l < L) ? T[(size_t)l * P + j] / s : 0.0;
        char *blk = reinterpret_cast<char *>(out) + (size_t)c * NS * NPAD * TC_KC * 2;
        if (MODE == LINMIN_PROJ_BF16) {
            *reinterpret_cast<__nv_bfloat16 *>(blk + kmaj(j, k, NPAD)) = __double2bfloat16(v);
        } else {
            double r = j < P ? ldexp(v, -fexp[j]) : 0.0;     // |r| < 1/2, exact scaling
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const double t = r * 256.0;
                const double a = rint(t);
                r = t - a;
                *reinterpret_cast<__nv_bfloat16 *>(blk + (size_t)q * NPAD * TC_KC * 2 +
                                                   kmaj(j, k, NPAD)) = __double2bfloat16(a);
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
                // A: K-adjacent core matrices 16 x 128 B apart, 8-row groups 128 B
                constexpr uint32_t LBO_A = (TC_M / 8) * 128, LBO_B = (NPAD / 8) * 128;
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
                            const uint64_t bd = sdesc(su32(sB + q * B_SLICE) + kk * 2 * LBO_B, LBO_B, 128);
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
// Per-pixel exponents (max_l |y_l| < 2^e) in one coalesced pass: warp per row.
__global__ void tc_rowexp_kernel(const float *__restrict__ cube, long long N, int L,
                                 int *__restrict__ rexp)
{
    const long long n = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (n >= N) return;
    const float *y = cube + (size_t)n * L;
    float m = 0.f;
    for (int l = lane; l < L; l += 32) m = fmaxf(m, fabsf(__ldg(y + l)));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
        int e = 0;
        if (m > 0.f) { frexpf(m, &e); ++e; }         // |y_l| 2^-e < 1/2
        rexp[n] = e;
    }
}

constexpr int TC2_THREADS = 512;    // 16 warps, one CTA per SM

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes)
                 : "memory");
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

__device__ __forceinline__ void tmem_ld4(uint32_t addr, float (&v)[4])
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// Exact projection with the chunks of every tile double-buffered: while
// chunk g is sliced and multiplied, the tensor map copies the pixel tile of
// chunk g + 1 (128 pixels x 64 bands, zero past N and L) and a bulk copy
// brings its B~ slices, both completing on that buffer's mbarrier.
template <int NPAD>
__global__ void __launch_bounds__(TC2_THREADS, 1)
project_tc2_kernel(const __grid_constant__ CUtensorMap ymap, long long N, int L, int P,
                   const __nv_bfloat16 *__restrict__ bsl, const int *__restrict__ fexp,
                   const int *__restrict__ rexp, float *__restrict__ c_hi,
                   float *__restrict__ c_lo, int *__restrict__ err)
{
    constexpr int NS = TcMode<LINMIN_PROJ_TC>::NS, NL = TcMode<LINMIN_PROJ_TC>::NL;
    constexpr int Y_TILE = TC_M * TC_KC * 4;          // fp32 pixel tile of a chunk
    constexpr int A_SLICE = TC_M * TC_KC * 2;
    constexpr int B_SLICE = NPAD * TC_KC * 2;
    constexpr int QCOL = NPAD / 4;                    // columns per epilogue warp
    constexpr int TMEM_COLS = tc_tmem_cols(NL * NPAD);
    static_assert(QCOL % 4 == 0, "epilogue loads 4 columns at a time");
    static_assert(TC_M * (TC_KC / 8) % TC2_THREADS == 0, "slicing items per thread");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sY = smem;                          // 2 pixel tiles
    unsigned char *sA = smem + 2 * Y_TILE;             // NS pixel slices
    unsigned char *sB = sA + NS * A_SLICE;             // 2 x NS B~ slices
    __shared__ __align__(8) uint64_t bar_load[2];
    __shared__ __align__(8) uint64_t bar_mma;
    __shared__ uint32_t tbase;
    __shared__ int pexp[2][TC_M];                      // exponents of the tile (by parity)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunks = (L + TC_KC - 1) / TC_KC;
    const long long ntiles = (N + TC_M - 1) / TC_M;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long nwork = my_tiles * nchunks;        // chunks this CTA runs

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&bar_load[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&bar_load[1])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(&bar_mma)));
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

    // chunk g of this CTA: tile blockIdx.x + (g / nchunks) * gridDim.x, chunk g % nchunks
    auto issue = [&](long long g) {
        const long long t = blockIdx.x + (g / nchunks) * gridDim.x;
        const int c = (int)(g % nchunks), b = (int)(g & 1);
        const uint32_t bar = su32(&bar_load[b]);
        mbar_expect_tx(bar, (uint32_t)(Y_TILE + NS * B_SLICE));
        tma_load_2d(su32(sY + b * Y_TILE), &ymap, c * TC_KC, (int)(t * TC_M), bar);
        bulk_load(su32(sB + b * NS * B_SLICE),
                  reinterpret_cast<const char *>(bsl) + (size_t)c * NS * B_SLICE,
                  (uint32_t)(NS * B_SLICE), bar);
    };

    // epilogue role: TMEM lanes of warp (warp & 3), columns of quarter (warp >> 2)
    const int ep_pix = 32 * (warp & 3) + lane;
    const int ep_col0 = QCOL * (warp >> 2);
    df acc[QCOL];
#pragma unroll
    for (int j = 0; j < QCOL; ++j) acc[j] = df_make(0.f);

    bool ok = true;
    uint32_t mma_phase = 0;
    if (tid == 0 && nwork > 0) issue(0);
    for (long long g = 0; g <= nwork && ok; ++g) {
        // 1. the MMAs of chunk g - 1 are complete: fold at a group end, write
        //    at a tile end
        if (g > 0) {
            ok = __syncthreads_and(mbar_wait(su32(&bar_mma), mma_phase));
            mma_phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!ok) break;
            const int cp = (int)((g - 1) % nchunks);
            const long long tp = blockIdx.x + ((g - 1) / nchunks) * gridDim.x;
            if ((cp % TC_GROUP) == TC_GROUP - 1 || cp == nchunks - 1) {
#pragma unroll
                for (int j4 = 0; j4 < QCOL / 4; ++j4) {
                    float sh[4], sl[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) { sh[q] = 0.f; sl[q] = 0.f; }
#pragma unroll
                    for (int lv = NL - 1; lv >= 0; --lv) {
                        float v[4];
                        tmem_ld4(tmem + ((uint32_t)(32 * (warp & 3)) << 16) +
                                     (uint32_t)(lv * NPAD + ep_col0 + 4 * j4), v);
                        const float w = pow2f(-8 * (lv + 2));
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float t, e;
                            two_sum(sh[q], v[q] * w, t, e);
                            sh[q] = t;
                            sl[q] += e;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        acc[4 * j4 + q] = df_add_near(acc[4 * j4 + q], sh[q], sl[q]);
                }
                if (cp == nchunks - 1) {
                    const long long n = tp * TC_M + ep_pix;
                    if (n < N) {
                        const int e = pexp[(int)(((g - 1) / nchunks) & 1)][ep_pix];
#pragma unroll
                        for (int j = 0; j < QCOL; ++j) {
                            const int col = ep_col0 + j;
                            if (col < P) {
                                const int sh2 = e + fexp[col];
                                df v = df{ldexpf(acc[j].hi, sh2), ldexpf(acc[j].lo, sh2)};
                                v = df_add(v, df_make((float)RHO));
                                c_hi[(size_t)n * P + col] = v.hi;
                                c_lo[(size_t)n * P + col] = v.lo;
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < QCOL; ++j) acc[j] = df_make(0.f);
                }
            }
        }
        if (g == nwork) break;
        const int c = (int)(g % nchunks), b = (int)(g & 1);
        const long long t = blockIdx.x + (g / nchunks) * gridDim.x;
        if (c == 0)
            for (int i = tid; i < TC_M; i += TC_THREADS) {
                const long long n = t * TC_M + i;
                pexp[(int)((g / nchunks) & 1)][i] = n < N ? rexp[n] : 0;
            }
        // 2. TMEM read and buffer (g + 1) & 1 (last used by chunk g - 1) free
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == 0 && g + 1 < nwork) issue(g + 1);
        // 3. chunk g's pixel tile and B~ slices have landed
        ok = __syncthreads_and(mbar_wait(su32(&bar_load[b]), (uint32_t)((g >> 1) & 1)));
        if (!ok) break;
        // 4. pixel slices from the tile (row-major, 64 bands of 4 bytes)
        const int* pe = pexp[(int)((g / nchunks) & 1)];
#pragma unroll
        for (int u = 0; u < TC_M * (TC_KC / 8) / TC2_THREADS; ++u) {
            const int it = tid + u * TC2_THREADS;
            const int pix = it % TC_M, oct = it / TC_M;
            const float4 *row = reinterpret_cast<const float4 *>(sY + b * Y_TILE + pix * TC_KC * 4 +
                                                                 oct * 32);
            const float4 v0 = row[0], v1 = row[1];
            const int e = pe[pix];
            float r[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            const int h = e / 2;
            const float f1 = pow2f(-h), f2 = pow2f(h - e);
#pragma unroll
            for (int q = 0; q < 8; ++q) r[q] = r[q] * f1 * f2;          // exact
            const int off = kmaj(pix, 8 * oct, TC_M);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                float a[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float tt = r[q] * 256.f;
                    a[q] = rintf(tt);
                    r[q] = tt - a[q];
                }
                *reinterpret_cast<uint4 *>(sA + i * A_SLICE + off) = pack8(a);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // 5. the MMAs of chunk g
        if (tid == 0) {
            constexpr uint32_t ID = idesc_bf16(TC_M, NPAD);
            constexpr uint32_t LBO_A = (TC_M / 8) * 128, LBO_B = (NPAD / 8) * 128;
            const bool first = (c % TC_GROUP) == 0;
            // descriptors are affine in the start address (its 16-byte units
            // are the low bits): bases once, compile-time offsets per MMA
            const uint64_t a0 = sdesc(su32(sA), LBO_A, 128);
            const uint64_t b0 = sdesc(su32(sB + b * NS * B_SLICE), LBO_B, 128);
#pragma unroll
            for (int lv = 0; lv < NL; ++lv) {
                bool fresh = first;
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    const int q = lv - i;
                    if (q < 0 || q >= NS) continue;
#pragma unroll
                    for (int kk = 0; kk < TC_KC / 16; ++kk) {
                        const uint64_t ad = a0 + (uint64_t)((i * A_SLICE + kk * 2 * LBO_A) >> 4);
                        const uint64_t bd = b0 + (uint64_t)((q * B_SLICE + kk * 2 * LBO_B) >> 4);
                        mma_bf16(tmem + (uint32_t)(lv * NPAD), ad, bd, ID, fresh ? 0u : 1u);
                        fresh = false;
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(su32(&bar_mma)));
        }
    }
    if (!ok) {
        // flag, then give copies and MMAs in flight a second bounded wait
        if (tid == 0) atomicOr(err, 4);
        mbar_wait(su32(&bar_mma), mma_phase);
        mbar_wait(su32(&bar_load[0]), 0);
        mbar_wait(su32(&bar_load[1]), 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(TMEM_COLS));
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
bool tc2_usable(const float *cube, long long N, int L)
{
    return (L % 4) == 0 && (reinterpret_cast<uintptr_t>(cube) % 16) == 0 && N < (1LL << 31) &&
           encode_tiled() != nullptr;
}

template <int NPAD>
static cudaError_t launch_tc2_t(const float *cube, long long N, int L, int P,
                                const __nv_bfloat16 *bsl, const int *fexp, const int *rexp,
                                float *c_hi, float *c_lo, int *err, cudaStream_t st)
{
    constexpr int NS = TcMode<LINMIN_PROJ_TC>::NS;
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)L, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)L * 4};
    const cuuint32_t box[2] = {(cuuint32_t)TC_KC, (cuuint32_t)TC_M};
    const cuuint32_t estr[2] = {1, 1};
    if (encode_tiled()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(cube), dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = 2 * (size_t)TC_M * TC_KC * 4 + (size_t)NS * TC_M * TC_KC * 2 +
                        2 * (size_t)NS * NPAD * TC_KC * 2;
    cudaError_t e = cudaFuncSetAttribute(project_tc2_kernel<NPAD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_rowexp_kernel<<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(cube, N, L,
                                                                      const_cast<int *>(rexp));
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ntiles = (N + TC_M - 1) / TC_M;
    const unsigned blocks = (unsigned)(ntiles < sms ? ntiles : sms);
    project_tc2_kernel<NPAD><<<blocks, TC2_THREADS, smem, st>>>(map, N, L, P, bsl, fexp, rexp,
                                                                c_hi, c_lo, err);
    return cudaGetLastError();
}

cudaError_t launch_project_tc2(const float *cube, long long N, int L, int P,
                               const __nv_bfloat16 *bsl, const int *fexp, int *rexp, float *c_hi,
                               float *c_lo, int *err, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    switch (((P + 15) / 16) * 16) {
    case 16: return launch_tc2_t<16>(cube, N, L, P, bsl, fexp, rexp, c_hi, c_lo, err, st);
    case 32: return launch_tc2_t<32>(cube, N, L, P, bsl, fexp, rexp, c_hi, c_lo, err, st);
    case 48: return launch_tc2_t<48>(cube, N, L, P, bsl, fexp, rexp, c_hi, c_lo, err, st);
    case 64: return launch_tc2_t<64>(cube, N, L, P, bsl, fexp, rexp, c_hi, c_lo, err, st);
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

cudaError_t launch_tc_prep(const double *T, int L, int P, const double *scale, int mode,
                           __nv_bfloat16 *bsl, int *fexp, cudaStream_t st)
{
    const int NPAD = ((P + 15) / 16) * 16;
    const int nchunks = (L + TC_KC - 1) / TC_KC;
    if (mode == LINMIN_PROJ_TC)
        tc_bexp_kernel<<<(P * 32 + 255) / 256, 256, 0, st>>>(T, L, P, scale, fexp);
    const long long total = (long long)nchunks * NPAD * TC_KC;
    const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
    if (mode == LINMIN_PROJ_TC)
        tc_bslice_kernel<LINMIN_PROJ_TC><<<blocks, 256, 0, st>>>(T, L, P, NPAD, scale, fexp, bsl,
                                                                 nchunks);
    else
        tc_bslice_kernel<LINMIN_PROJ_BF16><<<blocks, 256, 0, st>>>(T, L, P, NPAD, scale, fexp,
                                                                   bsl, nchunks);
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
