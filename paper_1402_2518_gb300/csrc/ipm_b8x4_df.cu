// Interior-point kernel, NS = 8 slots of G = 4 lanes per pixel (P <= 32),
// double-float residual phase.
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<8, 4, true>(const IpmArgs &, cudaStream_t);
}
