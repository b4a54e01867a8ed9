// Launch interfaces between the C ABI (api.cu) and the kernels.
#pragma once
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

// Bucket of the interior-point kernel for a library size P.
struct Bucket { int NS, G, PP; };
bool ipm_bucket(int P, Bucket *b);
inline int pq_of(int P) { return ((P + 3) / 4) * 4; }

// Device buffers produced by the library preparation (per sigma).
struct Prep {
    double *G64;     // P x P   whitened Gram S W^2 S^T (fp64, unscaled)
    double *Gt64;    // P x P   G~ = G / s + rho (fp64)
    double *scale;   // 1       s = trace(G) / P
    float *Ghi, *Glo;// PP x PP G~ as hi + lo float32, zero padded
    float *grs;      // PP      G~ 1 / P
    float *gdiag;    // P       diag(G) / s
    float *Bhi, *Blo;// L x PQ  W^2 S^T / s as hi + lo float32, [l][j]
    int *flags;      // 1       bit 0: invalid sigma, bit 1: bad scale
};

cudaError_t launch_prep(const float *S, const float *sigma, int L, int P, int PP,
                        const Prep &o, cudaStream_t st);
cudaError_t launch_project(const float *cube, long long N, int L, int P,
                           const float *Bhi, const float *Blo, float *c_hi,
                           float *c_lo, cudaStream_t st);

struct IpmArgs;
cudaError_t launch_ipm(const Bucket &b, bool accurate, const IpmArgs &a,
                       cudaStream_t st);

struct RefineArgs {
    long long N;
    int P;
    const double *Gt64;            // P x P
    const float *Ghi, *Glo;        // PP x PP, G~ as hi + lo float32
    int PP;
    const double *scale;
    const float *gdiag;            // P
    const float *c_hi, *c_lo;      // N x P
    const float *x_in, *lam_in;    // N x P (interior-point result)
    float *x_out;                  // N x P (may alias x_in)
    float *sx_out;                 // N x P or NULL
    unsigned long long *n_unverified;   // pixels whose crossover did not reach KKT
    double tol_x, tol_g;
    int max_swaps;                 // support changes allowed before giving up
    const long long *list;         // optional: pixels to process (else 0..N-1)
    const unsigned long long *list_len;
    long long *retry_list;         // optional: pixels that failed, appended
    unsigned long long *retry_len;
};
cudaError_t launch_refine(const RefineArgs &a, cudaStream_t st);

cudaError_t launch_rms(const float *cube, const float *S, const float *x,
                       long long N, int L, int P, float *rms, cudaStream_t st);

}  // namespace lm
