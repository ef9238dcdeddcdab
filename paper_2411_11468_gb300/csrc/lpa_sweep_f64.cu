// Float64 table values (lpa_tuning.float_values = 2): the table-dependent sweep kernels with
// double label sums, for the value-type comparison of Section 4.4 (32-bit against 64-bit
// floating-point hashtable values).  In their own translation
// unit so that the default kernels and their build are unchanged; both the compile-time
// Algorithm 2 probe and the run-time probe scheme are instantiated.
#include "sweep_kernels.cuh"

namespace lpa {

cudaError_t sweep_init_constants_f64() { return init_magic(); }

cudaError_t launch_vertex_phase_f64(const SweepPlan &p, cudaStream_t s, LaunchHook *hook, int *launches)
{
    return p.probe == kProbeQuadDoublePow2 ? launch_vertex_phase<kProbeQuadDoublePow2, true>(p, s, hook, launches)
                                           : launch_vertex_phase<kProbeRuntime, true>(p, s, hook, launches);
}

cudaError_t launch_hub_acc_phase_f64(const SweepPlan &p, const HArgs &h, cudaStream_t s, LaunchHook *hook,
                                     int *launches)
{
    return p.probe == kProbeQuadDoublePow2 ? launch_hub_acc_phase<kProbeQuadDoublePow2, true>(p, h, s, hook, launches)
                                           : launch_hub_acc_phase<kProbeRuntime, true>(p, h, s, hook, launches);
}

}  // namespace lpa
