// Mixed-precision instantiation: FP32 geometry, splines and bond order;
// positions, displacements and all accumulation stay FP64.
#include "kernels.cuh"

namespace airebo {
template <> void launch_compute<float>(const StepArgs<float>& a, cudaStream_t s, int num_sms, cudaEvent_t* ev) {
    launch_compute_impl<float>(a, s, num_sms, ev);
}
}  // namespace airebo
