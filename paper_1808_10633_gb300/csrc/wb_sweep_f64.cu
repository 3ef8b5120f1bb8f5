// wb_sweep_f64.cu -- double instantiation of the WENO5 sweep kernels, and
// the tile shapes the host uses to build the tile tables.
#include "wb_sweep.cuh"

namespace wb {

void sweep_shape(int axis, int s, int* ta, int* tp) {
    *ta = shape_ta(axis, s);
    *tp = kSweepNT / *ta;
}

template cudaError_t prepare_sweep_kernels<double>();
template cudaError_t launch_sweep<double>(int, const SweepArgs<double>&, int, cudaStream_t);
template cudaError_t launch_harvest<double>(const double*, long long, const PatchDev&, int,
                                            const long long*, long long, const double*,
                                            const double*, double, double, double, float*,
                                            cudaStream_t);
template cudaError_t launch_cell_state_flux<double>(const double*, long long, const PatchDev&, int,
                                                    double, double*, double*, cudaStream_t);

}  // namespace wb
