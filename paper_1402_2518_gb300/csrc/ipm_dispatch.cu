// Size-bucket selection of the interior-point kernel.
#include "ipm_launch.cuh"
#include "kernels.cuh"

namespace lm {

// Every compiled bucket (NS slots of G lanes per pixel, PP = NS * G rows).
static const Bucket kCompiled[] = {{2, 4, 8},  {2, 8, 16}, {4, 4, 16}, {8, 4, 32},
                                   {4, 8, 32}, {9, 4, 36}, {5, 8, 40}, {6, 8, 48},
                                   {3, 16, 48}, {4, 16, 64}};

// Default bucket per size: the fastest compiled bucket measured on GB300
// (65,536 pixels, L = 184, 4 extra spectra; interior-point phase, ms):
//   P = 16: 4x4 0.43, 2x8 0.79;  P = 32: 8x4 1.94, 4x8 3.09;
//   P = 48: 6x8 5.65, 3x16 7.02; P = 64: 4x16 15.4 (2x32: 25.1).
// Four lanes per pixel wins wherever the registers of H allow it.
bool ipm_bucket(int P, Bucket *b)
{
    static const Bucket table[] = {{2, 4, 8}, {4, 4, 16}, {8, 4, 32},
                                   {9, 4, 36}, {5, 8, 40}, {6, 8, 48},
                                   {4, 16, 64}};
    for (const Bucket &c : table)
        if (P >= 1 && P <= c.PP) { *b = c; return true; }
    return false;
}

int ipm_candidates(int P, Bucket *out, int max)
{
    int n = 0;
    for (const Bucket &c : kCompiled)
        if (P >= 1 && P <= c.PP && c.PP < P + 16 && n < max) out[n++] = c;
    return n;
}

cudaError_t launch_ipm(const Bucket &b, bool accurate, const IpmArgs &a, cudaStream_t st)
{
#define LM_CASE(NS, G)                                                                   \
    case NS * 100 + G:                                                                   \
        return accurate ? launch_ipm_mode<NS, G, true>(a, st) : launch_ipm_mode<NS, G, false>(a, st);
    switch (b.NS * 100 + b.G) {
        LM_CASE(2, 4) LM_CASE(2, 8) LM_CASE(4, 4) LM_CASE(8, 4) LM_CASE(4, 8) LM_CASE(9, 4)
        LM_CASE(5, 8) LM_CASE(6, 8) LM_CASE(3, 16) LM_CASE(4, 16)
    default: return cudaErrorInvalidValue;
    }
#undef LM_CASE
}

cudaError_t launch_ipm_batch(const Bucket &b, const IpmArgs &a, cudaStream_t st)
{
#define LM_CASE(NS, G) \
    case NS * 100 + G: return launch_ipm_mode<NS, G, false, true>(a, st);
    switch (b.NS * 100 + b.G) {
        LM_CASE(2, 4) LM_CASE(2, 8) LM_CASE(4, 4) LM_CASE(8, 4) LM_CASE(4, 8) LM_CASE(9, 4)
        LM_CASE(5, 8) LM_CASE(6, 8) LM_CASE(3, 16) LM_CASE(4, 16)
    default: return cudaErrorInvalidValue;
    }
#undef LM_CASE
}

}  // namespace lm
