// Interior-point kernel for P <= 64 (NS = 4 slots, G = 16 lanes per pixel),
// double-float residual phase.
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<4, 16, true>(const IpmArgs &, cudaStream_t);
}
