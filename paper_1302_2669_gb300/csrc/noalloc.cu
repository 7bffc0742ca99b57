// surfmcmc_decode_noalloc: the decoder for callers that cannot allocate
// device memory.  Its scratch (pure errors, their class codes and the
// per-chain sums) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"
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

bool on_device(const void* ptr) {
    cudaPointerAttributes a;
    if (!ptr || cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
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
    // Device buffers only: staging host buffers would need memory of its own.
    if (!on_device(syndromes) || !on_device(out_class) || (out_class_sum && !on_device(out_class_sum)) ||
        (out_log_ratio && !on_device(out_log_ratio)))
        return SURFMCMC_EINVAL;
    if (surfmcmc_noalloc_scratch_needed(n, L, o.chains_per_class) > kScratchBytes) return SURFMCMC_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SURFMCMC_ECUDA;
    void* base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;

    const int K = 4, R = o.chains_per_class, Cn = K * R;
    const int nq = n_qubits(L), W = n_words(L), nc = L * (L - 1) / 2;
    char* sp0 = (char*)base;
    uint32_t* e0 = (uint32_t*)sp0;
    int32_t* code = (int32_t*)(sp0 + round256((size_t)n * 2 * W * 4));
    uint64_t* chain_sum = (uint64_t*)(sp0 + round256((size_t)n * 2 * W * 4) + round256((size_t)n * 4));
    unsigned int* unit_counter =
        (unsigned int*)(sp0 + round256((size_t)n * 2 * W * 4) + round256((size_t)n * 4) + round256((size_t)n * Cn * 8));

    // Lanes per bundle: the smallest power of two >= 2 whose lanes the
    // colour's generators fill to >= 90%, within the shared-memory limit.
    int lam = 32;
    for (int cand = 32; cand >= 2; cand /= 2) {
        if (sweep_smem_bytes(nq, nc, cand) > 200 * 1024) continue;
        const double eff = (double)nc / (double)(cand * ((nc + cand - 1) / cand));
        lam = cand;
        if (eff >= 0.9) break;
    }

    SweepParams sp;
    memset(&sp, 0, sizeof sp);
    int G = 1;
    while (G < Cn && G < 32) G *= 2;
    sp.C = Cn;
    sp.R = R;
    sp.G = G;
    sp.bps = G == 32 ? (Cn + 31) / 32 : 1;
    sp.spb = G == 32 ? 1 : 32 / G;
    sp.id0 = id0;
    sp.n_groups = 1;
    GroupDesc& gd = sp.grp[0];
    gd.L = L;
    gd.nq = nq;
    gd.W = W;
    gd.nc = nc;
    gd.n = n;
    gd.n_bundles = G == 32 ? n * sp.bps : (n + sp.spb - 1) / sp.spb;
    gd.t_begin = 0;
    gd.t_end = o.n_sweeps;
    gd.burn_in = o.burn_in;
    sp.grp_nq_max = nq;
    sp.grp_nc_max = nc;
    sp.total_units = sweep_units(gd.n_bundles, lam);
    sp.unit_counter = unit_counter;
    // Eq. 2 acceptance table, as in surfmcmc_decode.
    const double r = (p / 3.0) / (1.0 - p);
    const double rs = o.beta_scale == 1.0 ? r : exp(-o.beta_scale * -log(r));
    uint64_t T[5] = {0, 0, 0, 0, 0};
    double rd = rs;
    for (int d = 1; d <= 4; ++d) {
        T[d] = (uint64_t)floor(rd * 4294967296.0);
        rd = rd * rs;
    }
    sp.accept_all = T[1] >= 4294967296ull;
    sp.reject_all = T[1] == 0;
    sp.qmodes = 0;
    for (int q = 0; q < 8 && !sp.accept_all; ++q) {
        uint32_t any1 = 0, any234 = 0;
        for (int k = 4 * q; k < 4 * q + 4; ++k) {
            any1 |= (uint32_t)(T[1] >> (31 - k)) & 1u;
            for (int d = 2; d <= 4; ++d) any234 |= (uint32_t)(T[d] >> (31 - k)) & 1u;
        }
        sp.qmodes |= (any234 ? 2u : any1 ? 1u : 0u) << (2 * q);
    }
    for (int k = 0; k < 32 && !sp.accept_all; ++k) {
        uint32_t t[5];
        for (int d = 1; d <= 4; ++d) t[d] = (uint32_t)((T[d] >> (31 - k)) & 1u);
        sp.pc[0][k] = t[1] ? ~0u : 0u;
        sp.pc[1][k] = (t[1] ^ t[2]) ? ~0u : 0u;
        sp.pc[2][k] = (t[1] ^ t[3]) ? ~0u : 0u;
        sp.pc[3][k] = (t[1] ^ t[2] ^ t[3] ^ t[4]) ? ~0u : 0u;
    }
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
    dp.beta_bar = -log(r);
    dp.chain_sum = chain_sum;
    dp.out_class = out_class;
    dp.out_class_sum = out_class_sum;
    dp.out_log_ratio = out_log_ratio;
    if (launch_decide(dp, s) != cudaSuccess) return SURFMCMC_ECUDA;
    if (!stream && cudaStreamSynchronize(s) != cudaSuccess) return SURFMCMC_ECUDA;
    return SURFMCMC_OK;
}
