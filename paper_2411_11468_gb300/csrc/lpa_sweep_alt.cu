// The probe-scheme comparison kernels (Section 4.2: linear probing, quadratic probing and
// double hashing beside Algorithm 2's quadratic-double hybrid): the table-dependent sweep
// kernels instantiated once with the scheme read at run time, in their own translation unit
// so that the default kernels keep the scheme fixed at compile time.
#include "sweep_kernels.cuh"

namespace lpa {

cudaError_t sweep_init_constants_alt() { return init_magic(); }

cudaError_t launch_vertex_phase_alt(const SweepPlan &p, cudaStream_t s, LaunchHook *hook, int *launches)
{
    return launch_vertex_phase<kProbeRuntime>(p, s, hook, launches);
}

cudaError_t launch_hub_acc_phase_alt(const SweepPlan &p, const HArgs &h, cudaStream_t s, LaunchHook *hook,
                                     int *launches)
{
    return launch_hub_acc_phase<kProbeRuntime>(p, h, s, hook, launches);
}

}  // namespace lpa
