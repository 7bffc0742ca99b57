// Sweep kernel instantiations for independent bit and phase flips (Sec.
// IV.B), compiled apart from the depolarizing ones to build in parallel.
#include "sweep_kernel.cuh"

namespace surfmcmc {

cudaError_t prepare_sweep_flips(const SweepParams& p, int lam) { return prepare_noise<true>(p, lam); }

cudaError_t launch_sweep_flips(const SweepParams& p, int lam, cudaStream_t s) {
    return launch_noise<true>(p, lam, s);
}

}  // namespace surfmcmc
