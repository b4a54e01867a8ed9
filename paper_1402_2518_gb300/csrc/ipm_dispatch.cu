// Size-bucket selection of the interior-point kernel.
#include "ipm_launch.cuh"
#include "kernels.cuh"

namespace lm {

bool ipm_bucket(int P, Bucket *b)
{
    static const Bucket table[] = {{2, 4, 8}, {4, 4, 16}, {4, 8, 32},
                                   {9, 4, 36}, {5, 8, 40}, {3, 16, 48},
                                   {4, 16, 64}};
    for (const Bucket &c : table)
        if (P >= 1 && P <= c.PP) { *b = c; return true; }
    return false;
}

cudaError_t launch_ipm(const Bucket &b, bool accurate, const IpmArgs &a, cudaStream_t st)
{
#define LM_CASE(NS, G)                                                                   \
    case NS * 100 + G:                                                                   \
        return accurate ? launch_ipm_mode<NS, G, true>(a, st) : launch_ipm_mode<NS, G, false>(a, st);
    switch (b.NS * 100 + b.G) {
        LM_CASE(2, 4) LM_CASE(4, 4) LM_CASE(4, 8) LM_CASE(9, 4) LM_CASE(5, 8) LM_CASE(3, 16)
        LM_CASE(4, 16)
    default: return cudaErrorInvalidValue;
    }
#undef LM_CASE
}

}  // namespace lm
