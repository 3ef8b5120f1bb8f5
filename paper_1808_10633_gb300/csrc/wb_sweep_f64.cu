// wb_sweep_f64.cu -- double instantiation of the WENO5 sweep kernels, and
// the tile shapes the host uses to build the tile tables.
#include "wb_sweep.cuh"

namespace wb {

void sweep_tile_shape(int axis, int* ta, int* tp) {
    if (axis == 0) { *ta = Shape<0>::TA; *tp = Shape<0>::TP; }
    else if (axis == 1) { *ta = Shape<1>::TA; *tp = Shape<1>::TP; }
    else { *ta = Shape<2>::TA; *tp = Shape<2>::TP; }
}

template cudaError_t prepare_sweep_kernels<double>();
template cudaError_t launch_sweep<double>(int, const SweepArgs<double>&, int, cudaStream_t);
template cudaError_t launch_harvest<double>(const double*, long long, const PatchDev&, int,
                                            const long long*, long long, const double*,
                                            const double*, double, double, double, float*,
                                            cudaStream_t);

}  // namespace wb
