// Interior-point kernel for P <= 48 (NS = 3 slots, G = 16 lanes per pixel),
// double-float residual phase.
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<3, 16, true>(const IpmArgs &, cudaStream_t);
}
