// C ABI of libsurfmcmc (see include/surfmcmc.h): argument checks, the
// acceptance table of Eq. 2, device scratch, host<->device staging and the
// kernel launches.  All arithmetic of the decoder runs in the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "surfmcmc.h"
#include "common.cuh"

using namespace surfmcmc;

struct surfmcmc_ctx {
    int device = 0;
    void* arena = nullptr;     // grow-only device scratch
    size_t arena_bytes = 0;
    std::string last_error;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;  // recorded around sweep launches
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spare;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(surfmcmc_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->last_error = buf;
    return code;
}

#define CK(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SURFMCMC_ENOMEM : SURFMCMC_ECUDA,         \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);            \
    } while (0)

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Carves aligned sub-buffers out of the context's arena; sizes are computed
// first (reserve), then the arena is grown once and pointers handed out.
struct Carver {
    size_t off = 0;
    size_t reserve(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};

int ensure_arena(surfmcmc_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->arena_bytes) return SURFMCMC_OK;
    if (ctx->arena) {
        CK(cudaDeviceSynchronize());
        CK(cudaFree(ctx->arena));
        ctx->arena = nullptr;
        ctx->arena_bytes = 0;
    }
    size_t want = bytes + bytes / 4;
    CK(cudaMalloc(&ctx->arena, want));
    ctx->arena_bytes = want;
    return SURFMCMC_OK;
}

// A caller buffer as seen by the kernels: the pointer itself if it is device
// memory, else a region of the arena (copied in for inputs).
struct Buf {
    void* user = nullptr;
    size_t bytes = 0;
    bool staged = false;
    size_t off = 0;
    void* dev = nullptr;
};

void plan(Buf& b, void* user, size_t bytes, Carver& cv) {
    b.user = user;
    b.bytes = bytes;
    b.staged = user && bytes && !is_device_ptr(user);
    if (b.staged) b.off = cv.reserve(bytes);
}

void bind(Buf& b, surfmcmc_ctx* ctx) {
    b.dev = b.staged ? (void*)((char*)ctx->arena + b.off) : b.user;
}

int copy_in(surfmcmc_ctx* ctx, Buf& b, cudaStream_t s) {
    if (b.staged) CK(cudaMemcpyAsync(b.dev, b.user, b.bytes, cudaMemcpyHostToDevice, s));
    return SURFMCMC_OK;
}

int copy_out(surfmcmc_ctx* ctx, Buf& b, cudaStream_t s) {
    if (b.staged) CK(cudaMemcpyAsync(b.user, b.dev, b.bytes, cudaMemcpyDeviceToHost, s));
    return SURFMCMC_OK;
}

int check_common(surfmcmc_ctx* ctx, int64_t n, int32_t L, uint32_t id0) {
    if (!ctx) return SURFMCMC_EINVAL;
    if (L < 2 || L > SURFMCMC_MAX_L) return fail(ctx, SURFMCMC_EINVAL, "L=%d outside 2..%d", L, SURFMCMC_MAX_L);
    if (n < 0) return fail(ctx, SURFMCMC_EINVAL, "n=%lld < 0", (long long)n);
    if ((uint64_t)id0 + (uint64_t)n > 4294967296ull)
        return fail(ctx, SURFMCMC_EINVAL, "syndrome ids id0+n exceed 2^32");
    return SURFMCMC_OK;
}

// Eq. 2: r = (p/3)/(1-p) = e^{-beta_bar}; r* = e^{-beta_scale beta_bar};
// T[d] = floor(r*^d 2^32), r*^d by repeated multiplication.
void acceptance_table(double p, double beta_scale, uint64_t T[5], double* beta_bar) {
    const double r = (p / 3.0) / (1.0 - p);
    const double rs = beta_scale == 1.0 ? r : exp(-beta_scale * -log(r));
    double rd = rs;
    T[0] = 0;
    for (int d = 1; d <= 4; ++d) {
        T[d] = (uint64_t)floor(rd * 4294967296.0);
        rd = rd * rs;
    }
    *beta_bar = -log(r);
}

// Burn-in stage j of S runs at beta* (a0 + (1 - a0) j / S).
double anneal_scale(double beta_scale, double a0, int j, int S) {
    return beta_scale * (a0 + (1.0 - a0) * (double)j / (double)S);
}

// Acceptance thresholds of one launch as kernel parameters: flags, the
// number of leading all-zero digit planes, and per plane k the algebraic
// normal form of d-1 -> bit (31-k) of T[d].
void set_temperature(SweepParams& sp, double p, double beta_scale) {
    uint64_t T[5];
    double beta_bar;
    acceptance_table(p, beta_scale, T, &beta_bar);
    sp.accept_all = T[1] >= 4294967296ull;
    sp.reject_all = T[1] == 0;
    sp.lz = sp.accept_all ? 0 : (T[1] == 0 ? 32 : __builtin_clz((uint32_t)T[1]));
    for (int k = 0; k < 32; ++k) {
        uint32_t t[5] = {0, 0, 0, 0, 0};
        if (!sp.accept_all)
            for (int d = 1; d <= 4; ++d) t[d] = (uint32_t)((T[d] >> (31 - k)) & 1u);
        sp.pc[0][k] = t[1] ? ~0u : 0u;
        sp.pc[1][k] = (t[1] ^ t[2]) ? ~0u : 0u;
        sp.pc[2][k] = (t[1] ^ t[3]) ? ~0u : 0u;
        sp.pc[3][k] = (t[1] ^ t[2] ^ t[3] ^ t[4]) ? ~0u : 0u;
    }
}

int pick_lanes(int L, int requested, int* lam_out) {
    const int nq = n_qubits(L), nc = L * (L - 1) / 2;
    auto smem_ok = [&](int lam) { return sweep_smem_bytes(nq, nc, lam) <= 200 * 1024; };
    if (requested) {
        if (requested != 2 && requested != 4 && requested != 8 && requested != 16 && requested != 32)
            return SURFMCMC_EINVAL;
        if (!smem_ok(requested)) return SURFMCMC_EINVAL;
        *lam_out = requested;
        return SURFMCMC_OK;
    }
    int best = 32;
    double best_eff = -1;
    for (int lam = 32; lam >= 2; lam /= 2) {
        if (!smem_ok(lam)) continue;
        const double eff = (double)nc / (double)(lam * ((nc + lam - 1) / lam));
        if (eff >= 0.9) { best = lam; break; }
        if (eff > best_eff + 1e-12) { best_eff = eff; best = lam; }
    }
    *lam_out = best;
    return SURFMCMC_OK;
}


int check_opts(surfmcmc_ctx* ctx, const surfmcmc_opts& o, double p) {
    if (!(p > 0.0 && p <= 0.75)) return fail(ctx, SURFMCMC_EINVAL, "p=%g outside (0, 0.75]", p);
    if (o.n_classes != 4) return fail(ctx, SURFMCMC_EINVAL, "n_classes must be 4 (planar code)");
    if (o.chains_per_class < 1 || 4 * o.chains_per_class > 1024)
        return fail(ctx, SURFMCMC_EINVAL, "chains_per_class=%d outside 1..256", o.chains_per_class);
    if (o.burn_in > o.n_sweeps) return fail(ctx, SURFMCMC_EINVAL, "burn_in > n_sweeps");
    if (!(o.beta_scale >= 0.0)) return fail(ctx, SURFMCMC_EINVAL, "beta_scale must be >= 0");
    if (std::isinf(o.beta_scale) && p == 0.75)
        return fail(ctx, SURFMCMC_EINVAL, "infinite beta_scale needs p < 0.75 (beta_bar = 0)");
    if (o.anneal_stages < 0 || o.anneal_stages > 64)
        return fail(ctx, SURFMCMC_EINVAL, "anneal_stages=%d outside 0..64", o.anneal_stages);
    if (o.anneal_stages > 0 && ((uint32_t)o.anneal_stages > o.burn_in || !(o.anneal_beta0 > 0.0 && o.anneal_beta0 <= 1.0)))
        return fail(ctx, SURFMCMC_EINVAL, "annealing needs anneal_stages <= burn_in and 0 < anneal_beta0 <= 1");
    return SURFMCMC_OK;
}

// Geometry and bundle layout of a run: C chains per syndrome, plane width G,
// bundles of 32 chains (G = 32: C/32 bundles per syndrome; G < 32: 32/G
// syndromes per bundle).
void init_geometry(SweepParams& sp, int L, int Cn, int R, int64_t n, uint32_t id0) {
    memset(&sp, 0, sizeof sp);
    int G = 1;
    while (G < Cn && G < 32) G *= 2;
    sp.L = L;
    sp.nq = n_qubits(L);
    sp.W = n_words(L);
    sp.nc = L * (L - 1) / 2;
    sp.C = Cn;
    sp.R = R;
    sp.G = G;
    sp.bps = G == 32 ? (Cn + 31) / 32 : 1;
    sp.spb = G == 32 ? 1 : 32 / G;
    sp.n = n;
    sp.n_bundles = G == 32 ? n * sp.bps : (n + sp.spb - 1) / sp.spb;
    sp.id0 = id0;
    sp.ids = nullptr;
}

// Launch segments of one run: the annealing stages of the burn-in (no
// sampling), then the rest of the run at beta*.  Sweep indices are absolute.
struct Segment {
    uint32_t t0, t1;
    double scale;
    bool anneal;
};

std::vector<Segment> plan_segments(const surfmcmc_opts& o, double beta_scale, uint32_t sweep_begin) {
    std::vector<Segment> segs;
    const uint32_t B = o.burn_in;
    const int S = o.anneal_stages;
    for (int j = 0; j < S; ++j) {
        const uint32_t lo = (uint32_t)((uint64_t)j * B / (uint64_t)S);
        const uint32_t hi = (uint32_t)((uint64_t)(j + 1) * B / (uint64_t)S);
        const uint32_t a = lo > sweep_begin ? lo : sweep_begin;
        if (a < hi) segs.push_back({a, hi, anneal_scale(beta_scale, o.anneal_beta0, j, S), true});
    }
    const uint32_t main0 = S > 0 && B > sweep_begin ? B : sweep_begin;
    segs.push_back({main0, o.n_sweeps, beta_scale, false});
    return segs;
}

// Where one run reads its start and writes its results.
struct SweepIO {
    uint32_t* e0 = nullptr;
    int32_t* e0code = nullptr;
    const uint32_t* init_frames = nullptr;
    const uint64_t* init_sum = nullptr;
    uint64_t* chain_sum = nullptr;
    int32_t* chain_n = nullptr;
    uint32_t* chain_frames = nullptr;
    uint32_t* state = nullptr;  // bundle state between segments
};

int record_start(surfmcmc_ctx* ctx, std::pair<cudaEvent_t, cudaEvent_t>* ev, cudaStream_t s) {
    if (!ctx->timing) return SURFMCMC_OK;
    if (!ctx->spare.empty()) {
        *ev = ctx->spare.back();
        ctx->spare.pop_back();
    } else {
        CK(cudaEventCreate(&ev->first));
        CK(cudaEventCreate(&ev->second));
    }
    CK(cudaEventRecord(ev->first, s));
    return SURFMCMC_OK;
}

int record_end(surfmcmc_ctx* ctx, std::pair<cudaEvent_t, cudaEvent_t> ev, cudaStream_t s) {
    if (!ctx->timing) return SURFMCMC_OK;
    CK(cudaEventRecord(ev.second, s));
    ctx->pending.push_back(ev);
    return SURFMCMC_OK;
}

int run_segments(surfmcmc_ctx* ctx, SweepParams sp, const std::vector<Segment>& segs, uint32_t burn_in, double p,
                 int lam, const SweepIO& io, cudaStream_t s) {
    int rc;
    for (size_t i = 0; i < segs.size(); ++i) {
        const bool first = i == 0, last = i + 1 == segs.size();
        set_temperature(sp, p, segs[i].scale);
        sp.t_begin = segs[i].t0;
        sp.t_end = segs[i].t1;
        sp.burn_in = segs[i].anneal ? segs[i].t1 : burn_in;
        sp.e0 = first ? io.e0 : nullptr;
        sp.e0code = first ? io.e0code : nullptr;
        sp.init_frames = first ? io.init_frames : nullptr;
        sp.state_in = first ? nullptr : io.state;
        sp.state_out = last ? nullptr : io.state;
        sp.init_sum = last ? io.init_sum : nullptr;
        sp.chain_sum = last ? io.chain_sum : nullptr;
        sp.chain_n = last ? io.chain_n : nullptr;
        sp.chain_frames = last ? io.chain_frames : nullptr;
        std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
        if ((rc = record_start(ctx, &ev, s))) return rc;
        CK(launch_sweep(sp, lam, s));
        if ((rc = record_end(ctx, ev, s))) return rc;
    }
    return SURFMCMC_OK;
}

}  // namespace

extern "C" {

void surfmcmc_default_opts(surfmcmc_opts* o) {
    if (!o) return;
    o->n_classes = 4;
    o->chains_per_class = 4;
    o->n_sweeps = 2000;
    o->burn_in = 0;
    o->beta_scale = 1.0;
    o->lanes_per_bundle = 0;
    o->anneal_stages = 0;
    o->anneal_beta0 = 1.0;
}

const char* surfmcmc_strerror(int code) {
    switch (code) {
        case SURFMCMC_OK: return "success";
        case SURFMCMC_EINVAL: return "invalid argument";
        case SURFMCMC_ENOMEM: return "out of device memory";
        case SURFMCMC_ECUDA: return "CUDA error";
        case SURFMCMC_ENODEV: return "no usable sm_103 device";
        default: return "unknown error";
    }
}

const char* surfmcmc_last_error(const surfmcmc_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int surfmcmc_create(surfmcmc_ctx** out, int device) {
    if (!out) return SURFMCMC_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return SURFMCMC_ENODEV;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SURFMCMC_ENODEV;
    if (prop.major != 10 || prop.minor != 3) return SURFMCMC_ENODEV;
    surfmcmc_ctx* ctx = new surfmcmc_ctx;
    ctx->device = device;
    *out = ctx;
    return SURFMCMC_OK;
}

void surfmcmc_destroy(surfmcmc_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (ctx->arena) {
        cudaDeviceSynchronize();
        cudaFree(ctx->arena);
    }
    for (auto* v : {&ctx->pending, &ctx->spare})
        for (auto& e : *v) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    delete ctx;
}

int surfmcmc_set_timing(surfmcmc_ctx* ctx, int enable) {
    if (!ctx) return SURFMCMC_EINVAL;
    ctx->timing = enable != 0;
    return SURFMCMC_OK;
}

int surfmcmc_sweep_time(surfmcmc_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx) return SURFMCMC_EINVAL;
    DeviceGuard g(ctx->device);
    double total = 0.0;
    int64_t count = 0;
    for (auto& e : ctx->pending) {
        float t = 0.f;
        CK(cudaEventSynchronize(e.second));
        CK(cudaEventElapsedTime(&t, e.first, e.second));
        total += t;
        ++count;
        ctx->spare.push_back(e);
    }
    ctx->pending.clear();
    if (ms) *ms = total;
    if (launches) *launches = count;
    return SURFMCMC_OK;
}

int surfmcmc_gen_syndromes(surfmcmc_ctx* ctx, uint64_t seed, uint32_t id0, int64_t n, int32_t L, double p,
                           uint8_t* syndromes, int32_t* true_class, void* stream) {
    int rc = check_common(ctx, n, L, id0);
    if (rc) return rc;
    if (!(p >= 0.0 && p <= 0.75)) return fail(ctx, SURFMCMC_EINVAL, "p=%g outside [0, 0.75]", p);
    if (n > 0 && !syndromes) return fail(ctx, SURFMCMC_EINVAL, "syndromes is NULL");
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Carver cv;
    Buf bs, bt;
    plan(bs, syndromes, (size_t)n * n_stabs(L), cv);
    plan(bt, true_class, true_class ? (size_t)n * 4 : 0, cv);
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    bind(bs, ctx);
    bind(bt, ctx);
    CK(launch_gen_syndromes(seed, id0, n, L, p, (uint8_t*)bs.dev, (int32_t*)bt.dev, s));
    if ((rc = copy_out(ctx, bs, s)) || (rc = copy_out(ctx, bt, s))) return rc;
    if (!stream || bs.staged || bt.staged) CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}

int surfmcmc_start_frames(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L, uint32_t* frames,
                          int32_t* e0_class, void* stream) {
    int rc = check_common(ctx, n, L, 0);
    if (rc) return rc;
    if (n > 0 && (!syndromes || !frames)) return fail(ctx, SURFMCMC_EINVAL, "NULL syndromes or frames");
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Carver cv;
    Buf bs, bf, bc;
    plan(bs, (void*)syndromes, (size_t)n * n_stabs(L), cv);
    plan(bf, frames, (size_t)n * 2 * n_words(L) * 4, cv);
    plan(bc, e0_class, e0_class ? (size_t)n * 4 : 0, cv);
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    bind(bs, ctx);
    bind(bf, ctx);
    bind(bc, ctx);
    if ((rc = copy_in(ctx, bs, s))) return rc;
    CK(launch_start_frames((const uint8_t*)bs.dev, n, L, (uint32_t*)bf.dev, (int32_t*)bc.dev, s));
    if ((rc = copy_out(ctx, bf, s)) || (rc = copy_out(ctx, bc, s))) return rc;
    if (!stream || bf.staged || bc.staged) CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}

int surfmcmc_decode_ex(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L, double p,
                       const surfmcmc_opts* opts_in, uint64_t seed, uint32_t id0, uint32_t sweep_begin,
                       const uint32_t* init_frames, const uint64_t* init_chain_sum, int32_t* out_class,
                       uint64_t* out_class_sum, double* out_log_ratio, uint64_t* out_chain_sum,
                       int32_t* out_chain_n, uint32_t* out_chain_frames, void* stream) {
    int rc = check_common(ctx, n, L, id0);
    if (rc) return rc;
    surfmcmc_opts o;
    surfmcmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    if ((rc = check_opts(ctx, o, p))) return rc;
    if (sweep_begin > o.n_sweeps) return fail(ctx, SURFMCMC_EINVAL, "sweep_begin > n_sweeps");
    if (!init_frames && sweep_begin != 0)
        return fail(ctx, SURFMCMC_EINVAL, "sweep_begin > 0 needs init_frames");
    if (n > 0 && (!syndromes || !out_class)) return fail(ctx, SURFMCMC_EINVAL, "NULL syndromes or out_class");
    int lam = 0;
    if (pick_lanes(L, o.lanes_per_bundle, &lam))
        return fail(ctx, SURFMCMC_EINVAL, "lanes_per_bundle=%d unsupported for L=%d", o.lanes_per_bundle, L);
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;

    const int K = 4, R = o.chains_per_class, Cn = K * R;
    const int nq = n_qubits(L), W = n_words(L), ns = n_stabs(L);
    int G = 1;
    while (G < Cn && G < 32) G *= 2;

    SweepParams sp;
    init_geometry(sp, L, Cn, R, n, id0);
    make_round_keys((uint32_t)seed, (uint32_t)(seed >> 32), &sp.rk);

    Carver cv;
    Buf b_syn, b_if, b_is, b_cls, b_csum, b_lr, b_chn, b_chf;
    plan(b_syn, (void*)syndromes, (size_t)n * ns, cv);
    plan(b_if, (void*)init_frames, init_frames ? (size_t)n * Cn * 2 * W * 4 : 0, cv);
    plan(b_is, (void*)init_chain_sum, init_chain_sum ? (size_t)n * Cn * 8 : 0, cv);
    plan(b_cls, out_class, (size_t)n * 4, cv);
    plan(b_csum, out_class_sum, out_class_sum ? (size_t)n * K * 8 : 0, cv);
    plan(b_lr, out_log_ratio, out_log_ratio ? (size_t)n * K * 8 : 0, cv);
    plan(b_chn, out_chain_n, out_chain_n ? (size_t)n * Cn * 4 : 0, cv);
    plan(b_chf, out_chain_frames, out_chain_frames ? (size_t)n * Cn * 2 * W * 4 : 0, cv);
    // per-chain sums: the caller's device buffer, else scratch
    const bool chs_scratch = !out_chain_sum || !is_device_ptr(out_chain_sum);
    const size_t off_chs = chs_scratch ? cv.reserve((size_t)n * Cn * 8) : 0;
    const size_t off_e0 = init_frames ? 0 : cv.reserve((size_t)n * 2 * W * 4);
    const size_t off_code = init_frames ? 0 : cv.reserve((size_t)n * 4);
    const std::vector<Segment> segs = plan_segments(o, o.beta_scale, sweep_begin);
    const size_t off_state = segs.size() > 1 ? cv.reserve((size_t)sp.n_bundles * 2 * nq * 4) : 0;
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    Buf* all[] = {&b_syn, &b_if, &b_is, &b_cls, &b_csum, &b_lr, &b_chn, &b_chf};
    for (Buf* b : all) bind(*b, ctx);
    char* base = (char*)ctx->arena;
    uint64_t* chain_sum = chs_scratch ? (uint64_t*)(base + off_chs) : out_chain_sum;
    uint32_t* e0 = init_frames ? nullptr : (uint32_t*)(base + off_e0);
    int32_t* code = init_frames ? nullptr : (int32_t*)(base + off_code);
    uint32_t* state = segs.size() > 1 ? (uint32_t*)(base + off_state) : nullptr;

    if ((rc = copy_in(ctx, b_syn, s)) || (rc = copy_in(ctx, b_if, s)) || (rc = copy_in(ctx, b_is, s))) return rc;
    if (!init_frames) CK(launch_start_frames((const uint8_t*)b_syn.dev, n, L, e0, code, s));

    SweepIO io;
    io.e0 = e0;
    io.e0code = code;
    io.init_frames = (const uint32_t*)b_if.dev;
    io.init_sum = (const uint64_t*)b_is.dev;
    io.chain_sum = chain_sum;
    io.chain_n = (int32_t*)b_chn.dev;
    io.chain_frames = (uint32_t*)b_chf.dev;
    io.state = state;
    if ((rc = run_segments(ctx, sp, segs, o.burn_in, p, lam, io, s))) return rc;

    uint64_t T[5];
    double beta_bar;
    acceptance_table(p, 1.0, T, &beta_bar);
    DecideParams dp;
    dp.n = n;
    dp.K = K;
    dp.R = R;
    dp.samples = o.n_sweeps > o.burn_in ? (uint64_t)4 * R * (o.n_sweeps - o.burn_in) : 0;
    dp.beta_bar = beta_bar;
    dp.chain_sum = chain_sum;
    dp.out_class = (int32_t*)b_cls.dev;
    dp.out_class_sum = (uint64_t*)b_csum.dev;
    dp.out_log_ratio = (double*)b_lr.dev;
    CK(launch_decide(dp, s));

    bool any_host = false;
    for (Buf* b : {&b_cls, &b_csum, &b_lr, &b_chn, &b_chf}) {
        if ((rc = copy_out(ctx, *b, s))) return rc;
        any_host |= b->staged;
    }
    if (out_chain_sum && chs_scratch) {
        CK(cudaMemcpyAsync(out_chain_sum, chain_sum, (size_t)n * Cn * 8, cudaMemcpyDeviceToHost, s));
        any_host = true;
    }
    if (!stream || any_host) CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}


int surfmcmc_decode_ti(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L, double p,
                       const surfmcmc_opts* opts_in, int32_t n_beta, uint64_t seed, uint32_t id0, int32_t* out_class,
                       double* out_log_z, double* out_mean, void* stream) {
    int rc = check_common(ctx, n, L, id0);
    if (rc) return rc;
    surfmcmc_opts o;
    surfmcmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    if ((rc = check_opts(ctx, o, p))) return rc;
    if (!(o.beta_scale < INFINITY)) return fail(ctx, SURFMCMC_EINVAL, "thermodynamic integration needs finite beta*");
    if (n_beta < 3 || n_beta > 129 || n_beta % 2 == 0)
        return fail(ctx, SURFMCMC_EINVAL, "n_beta=%d must be odd in 3..129", n_beta);
    if (o.n_sweeps <= o.burn_in) return fail(ctx, SURFMCMC_EINVAL, "no sampled sweeps");
    if (n > 0 && (!syndromes || !out_class)) return fail(ctx, SURFMCMC_EINVAL, "NULL syndromes or out_class");
    int lam = 0;
    if (pick_lanes(L, o.lanes_per_bundle, &lam))
        return fail(ctx, SURFMCMC_EINVAL, "lanes_per_bundle=%d unsupported for L=%d", o.lanes_per_bundle, L);
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int K = 4, R = o.chains_per_class, Cn = K * R, N = n_beta;
    SweepParams sp;
    init_geometry(sp, L, Cn, R, n, id0);
    const std::vector<Segment> segs0 = plan_segments(o, o.beta_scale, 0);

    Carver cv;
    Buf b_syn, b_cls, b_lz;
    plan(b_syn, (void*)syndromes, (size_t)n * n_stabs(L), cv);
    plan(b_cls, out_class, (size_t)n * 4, cv);
    plan(b_lz, out_log_z, out_log_z ? (size_t)n * K * 8 : 0, cv);
    const bool mean_scratch = !out_mean || !is_device_ptr(out_mean);
    const size_t off_mean = mean_scratch ? cv.reserve((size_t)n * K * N * 8) : 0;
    const size_t off_chs = cv.reserve((size_t)n * Cn * 8);
    const size_t off_e0 = cv.reserve((size_t)n * 2 * sp.W * 4);
    const size_t off_code = cv.reserve((size_t)n * 4);
    const size_t off_state = segs0.size() > 1 ? cv.reserve((size_t)sp.n_bundles * 2 * sp.nq * 4) : 0;
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    for (Buf* b : {&b_syn, &b_cls, &b_lz}) bind(*b, ctx);
    char* base = (char*)ctx->arena;
    double* mean = mean_scratch ? (double*)(base + off_mean) : out_mean;
    uint64_t* chain_sum = (uint64_t*)(base + off_chs);
    uint32_t* e0 = (uint32_t*)(base + off_e0);
    int32_t* code = (int32_t*)(base + off_code);
    uint32_t* state = segs0.size() > 1 ? (uint32_t*)(base + off_state) : nullptr;

    if ((rc = copy_in(ctx, b_syn, s))) return rc;
    CK(launch_start_frames((const uint8_t*)b_syn.dev, n, L, e0, code, s));
    const uint64_t samples = (uint64_t)4 * R * (o.n_sweeps - o.burn_in);
    for (int j = 1; j < N; ++j) {
        // grid point j: beta_j = beta* j/(N-1), randomness keyed by seed + j
        const double bs = o.beta_scale * (double)j / (double)(N - 1);
        const uint64_t sj = seed + (uint64_t)j;
        make_round_keys((uint32_t)sj, (uint32_t)(sj >> 32), &sp.rk);
        SweepIO io;
        io.e0 = e0;
        io.e0code = code;
        io.chain_sum = chain_sum;
        io.state = state;
        if ((rc = run_segments(ctx, sp, plan_segments(o, bs, 0), o.burn_in, p, lam, io, s))) return rc;
        CK(launch_class_means(n, K, R, N, j, samples, chain_sum, mean, s));
    }
    uint64_t T[5];
    double beta_bar;
    acceptance_table(p, 1.0, T, &beta_bar);
    const double h = (o.beta_scale * beta_bar) / (double)(N - 1);
    CK(launch_ti_decide(n, K, N, 0.75 * (double)sp.nq, h / 3.0, mean, (int32_t*)b_cls.dev, (double*)b_lz.dev, s));

    bool any_host = false;
    for (Buf* b : {&b_cls, &b_lz}) {
        if ((rc = copy_out(ctx, *b, s))) return rc;
        any_host |= b->staged;
    }
    if (out_mean && mean_scratch) {
        CK(cudaMemcpyAsync(out_mean, mean, (size_t)n * K * N * 8, cudaMemcpyDeviceToHost, s));
        any_host = true;
    }
    if (!stream || any_host) CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}

int surfmcmc_decode(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L, double p,
                    const surfmcmc_opts* opts, uint64_t seed, uint32_t id0, int32_t* out_class,
                    uint64_t* out_class_sum, double* out_log_ratio, void* stream) {
    return surfmcmc_decode_ex(ctx, syndromes, n, L, p, opts, seed, id0, 0, nullptr, nullptr, out_class,
                              out_class_sum, out_log_ratio, nullptr, nullptr, nullptr, stream);
}

}  // extern "C"
