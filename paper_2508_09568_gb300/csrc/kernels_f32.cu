// Single-precision instantiations of the MHD bunch kernels.
#include "kernels_impl.cuh"

namespace mhd {

static const StepLaunch kStepF32[] = {
    StepInst<float, 3, 32, 8, 512, 1, true>::entry(),
    StepInst<float, 3, 16, 16, 512, 1, true>::entry(),
    StepInst<float, 3, 16, 16, 512>::entry(),
    StepInst<float, 3, 16, 8, 256, 2>::entry(),
    StepInst<float, 3, 8, 8, 128, 3>::entry(),
    StepInst<float, 3, 16, 16, 384>::entry(),
    StepInst<float, 3, 24, 8, 512, 1, true>::entry(),
    StepInst<float, 2, 16, 16, 256>::entry(),
    StepInst<float, 2, 32, 8, 256>::entry(),
    StepInst<float, 1, 64, 1, 64>::entry(),
};

const PrecisionKernels& kernels_f32() {
    static const PrecisionKernels k{kStepF32, (int)(sizeof(kStepF32) / sizeof(kStepF32[0])), &launch_fill<float>,
                                    &launch_cfl<float>, &launch_adjoint<float>, AF_N,
                                    &launch_fill_interp<float>, &launch_cfl_patch<float>, &launch_fill_cfl<float>,
                                    &prepare_fill_cfl<float>};
    return k;
}

}  // namespace mhd
