// Launch interfaces between the C ABI (api.cu) and the kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lm {

constexpr double RHO = 1.0;   // rho of G~ = G / s + rho 1 1^T (see ipm.cuh)
// The first interior-point pass stops once mu / s <= MU_STOP: the support is
// then identified on almost every pixel and the crossover finishes it with
// at most MAX_SWAPS support changes (measured on the synthetic workloads:
// ~0.5 changes per pixel on average, at most a few).
constexpr float MU_STOP = 1e-11f;
constexpr int MAX_SWAPS = 8;
// Initial support of the crossover: lambda_i < SUPPORT_THETA x_i G_ii.  A
// threshold below 1 leaves the near-degenerate coordinates out (at mu/s =
// 1e-11 they are the ones the crossover would drop again): ~10% of pixels
// then need a support change instead of ~40% with 1.
constexpr float SUPPORT_THETA = 0.01f;

// Bucket of the interior-point kernel for a library size P.
struct Bucket { int NS, G, PP; };
bool ipm_bucket(int P, Bucket *b);
// Compiled buckets that fit P (P <= PP < P + 16), at most max of them.
int ipm_candidates(int P, Bucket *out, int max);
constexpr int PP_MAX = 64;   // largest padded size of any bucket
inline int pq_of(int P) { return ((P + 3) / 4) * 4; }

// Device buffers produced by the library preparation (per sigma).
struct Prep {
    double *G64;     // P x P   whitened Gram S W^2 S^T (fp64, unscaled)
    double *Gt64;    // P x P   G~ = G / s + rho (fp64)
    double *scale;   // 1       s = trace(G) / P
    float *Ghi, *Glo;// PP x PP G~ as hi + lo float32, zero padded
    float *grs;      // PP      G~ x0 (the gradient term at the start point)
    float *gdiag;    // P       diag(G) / s
    float *Bhi, *Blo;// L x PQ  W^2 S^T / s as hi + lo float32, [l][j]
    int *flags;      // 1       bit 0: invalid sigma, bit 1: bad scale
    // interior-point start x0: 1/P everywhere, or (slack_idx >= 0) slack_x0
    // on that coordinate and (1 - slack_x0) / (P - 1) on the others
    int slack_idx = -1;
    float slack_x0 = 0.f;
};

// kernel launches issued by launch_prep and launch_crossover (kept next to
// them so that the launch count the C ABI reports stays exact)
constexpr int PREP_LAUNCHES = 3;
constexpr int PREP_COV_LAUNCHES = 4;
// The lane-group launch of the crossover factors supports of at most XCAP
// coordinates in its shared memory when P > XCAP (more groups per SM); a
// pixel whose support outgrows that goes on to a second launch sized by P.
constexpr int XCAP = 24;
// list entries of that handoff: pixel | (solves done << XG_SOLVE_SHIFT);
// pixel indices stay below 2^40
constexpr int XG_SOLVE_SHIFT = 56;
constexpr int crossover_launches(bool whole_cube, int P)
{
    return (whole_cube ? 3 + 3 + 2 : 1 + 1) + (P > XCAP ? 1 : 0);
}

cudaError_t launch_prep(const float *S, const float *sigma, int L, int P, int PP,
                        const Prep &o, cudaStream_t st);
// Full noise covariance: C^-1 (L x L fp64, device), T scratch (L x P fp64).
cudaError_t launch_prep_cov(const float *S, const double *Cinv, int L, int P, int PP,
                            const Prep &o, double *T, cudaStream_t st);
// Tensor-core projection (project_tc.cu): mode LINMIN_PROJ_TC or
// LINMIN_PROJ_BF16; err: bit 2 set when an MMA did not complete within the
// wait limit.
size_t tc_bslice_bytes(int L, int P, int mode);
// B~ column exponents (exact mode) and slices: from T (C^-1 S^T) when T is
// given, else from S and sigma (T = W^2 S^T formed on the fly); two
// launches in the exact mode, one in the bf16 mode
cudaError_t launch_tc_prep(const float *S, const float *sigma, const double *T, int L, int P,
                           const double *scale, int mode, __nv_bfloat16 *bsl, int *fexp,
                           cudaStream_t st);
cudaError_t launch_project_tc(const float *cube, long long N, int L, int P, int mode,
                              const __nv_bfloat16 *bsl, const int *fexp, float *c_hi,
                              float *c_lo, int *err, cudaStream_t st);
// TMA-fed exact projection: launch_rowexp writes the per-pixel exponents
// (rexp, N ints), then launch_project_tma runs the warp-specialised GEMM
// that reads them; usable when rows are 16-byte strided and aligned,
// otherwise launch_project_tc.
bool tma_projection_usable(const float *cube, long long N, int L);
cudaError_t launch_rowexp(const float *cube, long long N, int L, int *rexp, cudaStream_t st);
cudaError_t launch_project_tma(const float *cube, long long N, int L, int P,
                               const __nv_bfloat16 *bsl, const int *fexp, const int *rexp, float *c_hi,
                               float *c_lo, int *err, cudaStream_t st);
// slo / pos outputs from the slack-augmented internal problem
// Per-pixel column subsets (the second pass of Sec. 5): for pixel n and
// each column j < n_minerals whose bit is clear in mask[n], c~_j -= K_n
// with K_n = 2 (max_k |c~_k| + P + rho) + 1, an exact linear penalty: the
// multiplier of x_j = 0 in the problem without column j is bounded by
// 2 (max |c~| + max |G~|) and |G~_ij| <= P + rho, so the penalised
// problem has the sub-problem's minimiser with x_j = 0 and lambda_j >= 1.
cudaError_t launch_exclude(const unsigned long long *mask, int n_minerals, float *c_hi,
                           float *c_lo, long long N, int P, cudaStream_t st);

cudaError_t launch_strip_slack(const float *xa, const float *sxa, long long N, int P, float M,
                               bool bound_check, float *x, float *sx, int *it,
                               unsigned long long *nbad, cudaStream_t st);
cudaError_t launch_project(const float *cube, long long N, int L, int P,
                           const float *Bhi, const float *Blo, float *c_hi,
                           float *c_lo, cudaStream_t st);

struct IpmArgs;
cudaError_t launch_ipm(const Bucket &b, bool accurate, const IpmArgs &a,
                       cudaStream_t st);
// One float32 interior-point launch over the pixels of several cubes
// (a.cubes, a.n_cubes, a.total; a.counter zeroed), all of bucket b.
cudaError_t launch_ipm_batch(const Bucket &b, const IpmArgs &a, cudaStream_t st);

struct CrossArgs {
    long long N;
    int P;
    const double *Gt64;            // P x P   G~ (fp64)
    const float *Ghi, *Glo;        // PP x PP G~ as hi + lo float32
    int PP;
    const double *scale;           // s
    const float *gdiag;            // P       diag(G) / s
    const float *c_hi, *c_lo;      // N x P
    const float *x_in, *lam_in;    // N x P   interior-point iterate
    float *x_out;                  // N x P   (may alias x_in)
    float *sx_out;                 // N x P or NULL
    unsigned long long *mask;      // N       support bit masks (in/out)
    const long long *list_in;      // pixels of this pass
    const unsigned long long *len_in;
    long long *list_out;           // pixels handed to the next pass
    unsigned long long *len_out;
    long long *over_list = nullptr;          // lane groups with K < P: pixels whose
    unsigned long long *over_len = nullptr;  // support outgrew K (set by launch_crossover)
    long long *retry_list;         // pixels the crossover could not finish (or NULL)
    unsigned long long *retry_len;
    unsigned long long *n_unverified;   // counted when retry_list is NULL
    int *it_mark;                  // with n_unverified: iteration counts, negated
                                   // (not converged) for a pixel left unverified
    int max_solves;                // lane-group kernel: support solves per pixel
    double tol_x, tol_g;
};

// Device scratch of the crossover: two ping-pong pixel lists, per-pass
// list lengths, the support-size histogram and bucket cursors.
struct CrossoverScratch {
    long long *list[2];            // N each
    unsigned long long *len;       // MAX_SWAPS + 2
    unsigned long long *len_all;   // 1
    unsigned long long *cursor;    // P + 1
    unsigned int *hist;            // P + 1
    int *ksize;                    // N
};

// Crossover of the pixels in list (or of all N pixels, sorted by support
// size, when list is NULL): up to MAX_SWAPS + 1 support solves per pixel
// (all N: a pass of one thread per pixel, then one lane-group launch for
// the pixels it flipped; a list: one lane-group launch).
cudaError_t launch_crossover(const CrossArgs &base, const CrossoverScratch &w,
                             const long long *list, const unsigned long long *list_len,
                             cudaStream_t st);

cudaError_t launch_rms(const float *cube, const float *S, const float *x,
                       long long N, int L, int P, float *rms, cudaStream_t st);

}  // namespace lm
