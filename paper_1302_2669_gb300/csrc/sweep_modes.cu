// Sweep kernels with the digit-plane modes known at compile time (the three
// head patterns of depolarizing noise, see head_pattern), for plane widths
// of 16 and 32 chains and 8, 16 or 32 lanes per bundle: the shapes that
// decodes with 9 or more chains per syndrome take.  The 32-chain kernels
// take every chain of a bundle as valid, so they serve launches whose chain
// count per syndrome is a multiple of 32.  Other launches use the kernels
// of sweep.cu, which read the modes from their parameters.
#include "sweep_kernel.cuh"

namespace surfmcmc {

template <int G, int HM>
static cudaError_t launch_hm(const SweepParams& p, int lam, cudaStream_t s) {
    switch (lam) {
        case 8: return launch_t<G, 8, false, false, false, HM>(p, s);
        case 16: return launch_t<G, 16, false, false, false, HM>(p, s);
        case 32: return launch_t<G, 32, false, false, false, HM>(p, s);
        default: return cudaErrorNotSupported;
    }
}

template <int G>
static cudaError_t launch_g_hm(const SweepParams& p, int lam, int hm, cudaStream_t s) {
    switch (hm) {
        case 1: return launch_hm<G, 1>(p, lam, s);
        case 2: return launch_hm<G, 2>(p, lam, s);
        case 3: return launch_hm<G, 3>(p, lam, s);
        default: return cudaErrorNotSupported;
    }
}

// cudaErrorNotSupported (nothing launched) when the launch has no
// specialised kernel.
cudaError_t launch_sweep_modes(const SweepParams& p, int lam, cudaStream_t s) {
    if (p.noise != 0 || p.scan || p.accepts) return cudaErrorNotSupported;
    const int hm = head_pattern(p.qmodes);
    if (hm == 0) return cudaErrorNotSupported;
    switch (p.G) {
        case 16: return launch_g_hm<16>(p, lam, hm, s);
        // whole bundles only: the kernels take every chain of a bundle as valid
        case 32: return p.C % 32 == 0 ? launch_g_hm<32>(p, lam, hm, s) : cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}

}  // namespace surfmcmc
