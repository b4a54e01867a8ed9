// Interior-point kernel, NS = 2 slots of G = 8 lanes per pixel (P <= 16),
// double-float residual phase.
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<2, 8, true>(const IpmArgs &, cudaStream_t);
}
