// Interior-point kernel for P <= 40 (NS = 5 slots, G = 8 lanes per pixel),
// double-float residual phase.
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<5, 8, true>(const IpmArgs &, cudaStream_t);
}
