// wb_sweep_f32.cu -- float instantiation of the WENO5 sweep kernels.
#include "wb_sweep.cuh"

namespace wb {
template cudaError_t prepare_sweep_kernels<float>();
template cudaError_t launch_sweep<float>(int, const SweepArgs<float>&, int, cudaStream_t);
}  // namespace wb
