// surfmcmc_decode_noalloc: the decoder for callers that cannot allocate
// device memory.  Its scratch (pure errors, their class codes and the
// per-chain sums) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "plan.cuh"
#include "surfmcmc.h"

using namespace surfmcmc;

namespace {

constexpr size_t kScratchBytes = (size_t)SURFMCMC_NOALLOC_SCRATCH_BYTES;

// The scratch of every call of surfmcmc_decode_noalloc on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Set-up, once per device, with that device current: the host-side name of
// a __device__ array is only a stand-in, so its device address is looked up.
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return SURFMCMC_ENODEV;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return SURFMCMC_ECUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return SURFMCMC_OK;
}

// Device memory of device `dev` (or managed memory): a buffer on another GPU
// is refused, since the kernels run on `dev`.
bool on_device(const void* ptr, int dev) {
    cudaPointerAttributes a;
    if (!ptr || cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" size_t surfmcmc_noalloc_scratch_needed(int64_t n, int32_t L, int32_t chains_per_class) {
    if (n < 0 || L < 2 || L > SURFMCMC_MAX_L || chains_per_class < 1) return 0;
    const size_t Cn = 4 * (size_t)chains_per_class;
    return round256((size_t)n * 2 * n_words(L) * 4) + round256((size_t)n * 4) + round256((size_t)n * Cn * 8) +
           round256(sizeof(unsigned int));
}

extern "C" int surfmcmc_decode_noalloc(const uint8_t* syndromes, int64_t n, int32_t L, double p,
                                       const surfmcmc_opts* opts_in, uint64_t seed, uint32_t id0,
                                       int32_t* out_class, uint64_t* out_class_sum, double* out_log_ratio,
                                       void* stream) {
    surfmcmc_opts o;
    surfmcmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (L < 2 || L > SURFMCMC_MAX_L || n < 0 || (uint64_t)id0 + (uint64_t)n > 4294967296ull)
        return SURFMCMC_EINVAL;
    if (!(p > 0.0 && p <= 0.75) || o.n_classes != 4 || o.chains_per_class < 1 || 4 * o.chains_per_class > 1024 ||
        o.burn_in > o.n_sweeps || !(o.beta_scale >= 0.0) || (std::isinf(o.beta_scale) && p == 0.75) ||
        o.anneal_stages != 0 || o.lanes_per_bundle != 0 || o.scan != 0 || o.noise != 0)
        return SURFMCMC_EINVAL;
    if (n == 0) return SURFMCMC_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SURFMCMC_ECUDA;
    // Device buffers of the current device only: staging host buffers would
    // need memory of its own.
    if (!on_device(syndromes, dev) || !on_device(out_class, dev) ||
        (out_class_sum && !on_device(out_class_sum, dev)) || (out_log_ratio && !on_device(out_log_ratio, dev)))
        return SURFMCMC_EINVAL;
    if (surfmcmc_noalloc_scratch_needed(n, L, o.chains_per_class) > kScratchBytes) return SURFMCMC_EINVAL;

    void* base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;

    const int K = 4, R = o.chains_per_class, Cn = K * R;
    const int W = n_words(L);
    char* sp0 = (char*)base;
    uint32_t* e0 = (uint32_t*)sp0;
    int32_t* code = (int32_t*)(sp0 + round256((size_t)n * 2 * W * 4));
    uint64_t* chain_sum = (uint64_t*)(sp0 + round256((size_t)n * 2 * W * 4) + round256((size_t)n * 4));
    unsigned int* unit_counter =
        (unsigned int*)(sp0 + round256((size_t)n * 2 * W * 4) + round256((size_t)n * 4) + round256((size_t)n * Cn * 8));

    // The launch is planned by the same host rules as surfmcmc_decode's:
    // chain layout, lanes per bundle (widened for small batches on this
    // device's multiprocessors) and the Eq. 2 acceptance table.
    SweepParams sp;
    init_chains(sp, Cn, R, id0);
    sp.noise = 0;
    energy_table(o, sp.energy);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SURFMCMC_ECUDA;
    const int lam = widen_lanes_for(sms, L, heuristic_lanes(L, 0), bundles_of(sp, n), sp.G, 0);
    add_group(sp, L, n, 0, 0, 0, 0, lam);
    GroupDesc& gd = sp.grp[0];
    gd.t_begin = 0;
    gd.t_end = o.n_sweeps;
    gd.burn_in = o.burn_in;
    sp.unit_counter = unit_counter;
    set_temperature(sp, p, o.beta_scale);
    make_round_keys((uint32_t)seed, (uint32_t)(seed >> 32), &sp.rk);
    sp.e0 = e0;
    sp.e0code = code;
    sp.chain_sum = chain_sum;

    cudaStream_t s = (cudaStream_t)stream;
    if (launch_start_frames(syndromes, n, L, e0, code, s) != cudaSuccess) return SURFMCMC_ECUDA;
    if (launch_sweep(sp, lam, s) != cudaSuccess) return SURFMCMC_ECUDA;
    DecideParams dp;
    memset(&dp, 0, sizeof dp);
    dp.n = n;
    dp.K = K;
    dp.R = R;
    dp.samples = o.n_sweeps > o.burn_in ? (uint64_t)4 * R * (o.n_sweeps - o.burn_in) : 0;
    dp.beta_bar = -log(noise_rate(p, 0, sp.energy));
    dp.chain_sum = chain_sum;
    dp.out_class = out_class;
    dp.out_class_sum = out_class_sum;
    dp.out_log_ratio = out_log_ratio;
    if (launch_decide(dp, s) != cudaSuccess) return SURFMCMC_ECUDA;
    if (!stream && cudaStreamSynchronize(s) != cudaSuccess) return SURFMCMC_ECUDA;
    return SURFMCMC_OK;
}
