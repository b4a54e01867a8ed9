// Interior-point kernel for P <= 36 (NS = 9 slots, G = 4 lanes per pixel),
// double-float residual phase.
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<9, 4, true>(const IpmArgs &, cudaStream_t);
}
