// Double-precision instantiations of the MHD bunch kernels.
#include "kernels_impl.cuh"

namespace mhd {

static const StepLaunch kStepF64[] = {
    StepInst<double, 3, 8, 8, 128>::entry(),
    StepInst<double, 2, 16, 16, 256>::entry(),
    StepInst<double, 2, 8, 8, 128>::entry(),
    StepInst<double, 1, 64, 1, 64>::entry(),
};

const PrecisionKernels& kernels_f64() {
    static const PrecisionKernels k{kStepF64, (int)(sizeof(kStepF64) / sizeof(kStepF64[0])), &launch_fill<double>,
                                    &launch_cfl<double>, &launch_adjoint<double>, AF_N,
                                    &launch_fill_interp<double>, &launch_cfl_patch<double>, &launch_fill_cfl<double>,
                                    &prepare_fill_cfl<double>};
    return k;
}

}  // namespace mhd
