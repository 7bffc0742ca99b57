// Sweep kernel instantiations for depolarizing noise, the shared-memory and
// work-unit sizes, and the launch entry points (independent bit and phase
// flips are instantiated in sweep_flips.cu).
#include "sweep_kernel.cuh"

namespace surfmcmc {

size_t sweep_smem_bytes(int nq, int nc, int lam) {
    const int B = 32 / lam;
    return (size_t)8 * nc * 4 +
           (size_t)kWarps * ((size_t)B * (kHeadFixedWords + bundle_stride(nq, lam)) + warp_aux_words(B)) * 4;
}

long long sweep_units(long long n_bundles, int lam) { return (n_bundles + (long long)kWarps * (32 / lam) - 1) /
                                                               ((long long)kWarps * (32 / lam)); }

// Sets the kernel's shared-memory limit ahead of a stream capture.
cudaError_t prepare_sweep(const SweepParams& p, int lam) {
    return p.noise == 1 ? prepare_sweep_flips(p, lam) : prepare_noise<false>(p, lam);
}

cudaError_t launch_sweep(const SweepParams& p, int lam, cudaStream_t s) {
    // kernels with the launch's digit-plane modes compiled in, where they exist
    const cudaError_t e = launch_sweep_modes(p, lam, s);
    if (e != cudaErrorNotSupported) return e;
    // the general channel (noise 2) runs only in random scan, which reads the
    // energy table and not the template's noise model
    return p.noise == 1 ? launch_sweep_flips(p, lam, s) : launch_noise<false>(p, lam, s);
}

}  // namespace surfmcmc
