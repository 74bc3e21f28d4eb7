// FP64 instantiation of the compute kernels.
#include "kernels.cuh"

namespace airebo {
template <> void launch_compute<double>(const StepArgs<double>& a, cudaStream_t s, int num_sms, cudaEvent_t* ev) {
    launch_compute_impl<double>(a, s, num_sms, ev);
}
void launch_bstar_bound_check(const StepArgs<double>& a, double* out, cudaStream_t s, int num_sms) {
    k_bstar_bound_check<<<num_sms * 8, 128, 0, s>>>(a, out);
}
}  // namespace airebo
