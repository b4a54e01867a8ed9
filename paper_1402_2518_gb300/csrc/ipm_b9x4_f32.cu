// Interior-point kernel for P <= 36 (NS = 9 slots, G = 4 lanes per pixel),
// float32 residual phase (single cube and batched).
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<9, 4, false>(const IpmArgs &, cudaStream_t);
template cudaError_t launch_ipm_mode<9, 4, false, true>(const IpmArgs &, cudaStream_t);
}
