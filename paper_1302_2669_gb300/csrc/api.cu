// C ABI of libsurfmcmc (see include/surfmcmc.h): argument checks, the
// acceptance table of Eq. 2, device scratch, host<->device staging and the
// kernel launches.  All arithmetic of the decoder runs in the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "surfmcmc.h"
#include "common.cuh"
#include "plan.cuh"

using namespace surfmcmc;

// Launch shape of the sweep kernel chosen by surfmcmc_autotune.
struct Tuned {
    int lam = 0;             // lanes per bundle
    int blocks_per_sm = 0;   // persistent blocks per multiprocessor (0: as many as fit)
};

struct surfmcmc_ctx {
    int device = 0;
    int sms = 0;               // multiprocessors of the device
    void* arena = nullptr;     // grow-only device scratch
    size_t arena_bytes = 0;
    std::string last_error;
    bool timing = false;
    std::map<std::pair<int, int>, Tuned> tuned;  // (L, chains per class) -> launch shape
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

// Lanes per bundle of a run: the caller's choice, else the autotuned value
// for (L, chains per class), else the rule of heuristic_lanes.
int pick_lanes(int L, int requested, int* lam_out, const surfmcmc_ctx* ctx = nullptr, int R = 0, int code = 0) {
    const int nq = geo_nq(code, L), nc = geo_nc(code, L);
    if (requested) {
        if (requested != 2 && requested != 4 && requested != 8 && requested != 16 && requested != 32)
            return SURFMCMC_EINVAL;
        if (sweep_smem_bytes(nq, nc, requested) > kSweepSmemLimit) return SURFMCMC_EINVAL;
        *lam_out = requested;
        return SURFMCMC_OK;
    }
    if (ctx) {
        auto it = ctx->tuned.find({L, R});
        if (it != ctx->tuned.end()) {
            *lam_out = it->second.lam;
            return SURFMCMC_OK;
        }
    }
    *lam_out = heuristic_lanes(L, code);
    return SURFMCMC_OK;
}

// Resident blocks per multiprocessor of a run: the autotuned value for (L,
// chains per class) unless the caller fixed the lanes, else all that fit.
int tuned_blocks(const surfmcmc_ctx* ctx, int L, int R, int requested_lanes) {
    if (requested_lanes || !ctx) return 0;
    auto it = ctx->tuned.find({L, R});
    return it == ctx->tuned.end() ? 0 : it->second.blocks_per_sm;
}

// Widens the lanes of a small batch (widen_lanes_for) unless the caller
// fixed them.
int widen_lanes(const surfmcmc_ctx* ctx, int L, int requested, int lam, long long n_bundles, int G, int code = 0) {
    if (requested || !ctx) return lam;
    return widen_lanes_for(ctx->sms, L, lam, n_bundles, G, code);
}

int check_opts(surfmcmc_ctx* ctx, const surfmcmc_opts& o, double p) {
    if (o.noise < 0 || o.noise > 2) return fail(ctx, SURFMCMC_EINVAL, "noise=%d must be 0, 1 or 2", o.noise);
    if (o.noise != 1 && !(p > 0.0 && p <= 0.75)) return fail(ctx, SURFMCMC_EINVAL, "p=%g outside (0, 0.75]", p);
    if (o.noise == 2) {
        for (int i = 0; i < 3; ++i)
            if (o.pauli_energy[i] < 1 || o.pauli_energy[i] > 8)
                return fail(ctx, SURFMCMC_EINVAL, "pauli_energy[%d]=%d outside 1..8", i, o.pauli_energy[i]);
        if (o.scan != 1) return fail(ctx, SURFMCMC_EINVAL, "the general Pauli channel runs in random scan (scan=1)");
    }
    if (o.noise == 1 && !(p > 0.0 && p <= 0.5)) return fail(ctx, SURFMCMC_EINVAL, "flip p=%g outside (0, 0.5]", p);
    if (o.n_classes != 4 && o.n_classes != 16)
        return fail(ctx, SURFMCMC_EINVAL, "n_classes must be 4 (planar code) or 16 (toric code)");
    if (o.chains_per_class < 1 || o.n_classes * o.chains_per_class > 1024)
        return fail(ctx, SURFMCMC_EINVAL, "n_classes * chains_per_class must be in 1..1024");
    if (o.burn_in > o.n_sweeps) return fail(ctx, SURFMCMC_EINVAL, "burn_in > n_sweeps");
    if (!(o.beta_scale >= 0.0)) return fail(ctx, SURFMCMC_EINVAL, "beta_scale must be >= 0");
    if (std::isinf(o.beta_scale) && p == (o.noise == 1 ? 0.5 : 0.75))
        return fail(ctx, SURFMCMC_EINVAL, "infinite beta_scale needs beta_bar > 0");
    if (o.anneal_stages < 0 || o.anneal_stages > 64)
        return fail(ctx, SURFMCMC_EINVAL, "anneal_stages=%d outside 0..64", o.anneal_stages);
    if (o.anneal_stages > 0 && ((uint32_t)o.anneal_stages > o.burn_in || !(o.anneal_beta0 > 0.0 && o.anneal_beta0 <= 1.0)))
        return fail(ctx, SURFMCMC_EINVAL, "annealing needs anneal_stages <= burn_in and 0 < anneal_beta0 <= 1");
    if (o.scan != 0 && o.scan != 1) return fail(ctx, SURFMCMC_EINVAL, "scan=%d must be 0 or 1", o.scan);
    if (o.scan == 1 && o.lanes_per_bundle != 0 && o.lanes_per_bundle != 32)
        return fail(ctx, SURFMCMC_EINVAL, "random scan runs 32 lanes per bundle");
    return SURFMCMC_OK;
}

// Samples of n per chain and sweep: one per colour phase (sweeps), one per
// step (random scan: n_stab steps per sweep).
uint64_t samples_per_sweep(const surfmcmc_opts& o, int L) {
    return o.scan ? (uint64_t)geo_nstab(o.n_classes == 16, L) : 4u;
}

// The toric code (16 classes) needs an even L in 2..30 (its colouring) and
// runs through decode, decode_ex and decode_ti only.
int check_toric(surfmcmc_ctx* ctx, const surfmcmc_opts& o, int L) {
    if (o.n_classes != 16) return SURFMCMC_OK;
    if (L < 2 || L > 30 || (L & 1)) return fail(ctx, SURFMCMC_EINVAL, "toric code needs an even L in 2..30");
    return SURFMCMC_OK;
}

int reject_toric(surfmcmc_ctx* ctx, const surfmcmc_opts& o, const char* what) {
    if (o.n_classes == 16) return fail(ctx, SURFMCMC_EINVAL, "%s supports the planar code (4 classes) only", what);
    return SURFMCMC_OK;
}

// Launch segments of one run: the S annealing stages of the burn-in (no
// sampling), then the rest of the run at beta*.  Sweep indices are absolute;
// with S > 0 there are always S + 1 segments (some may be empty when a run
// resumes at sweep_begin), so that groups with different sweep counts line up.
struct Segment {
    uint32_t t0, t1;
    double scale;
    bool anneal;
};

std::vector<Segment> plan_segments(uint32_t n_sweeps, uint32_t B, int S, double a0, double beta_scale,
                                   uint32_t sweep_begin) {
    std::vector<Segment> segs;
    for (int j = 0; j < S; ++j) {
        const uint32_t lo = (uint32_t)((uint64_t)j * B / (uint64_t)S);
        const uint32_t hi = (uint32_t)((uint64_t)(j + 1) * B / (uint64_t)S);
        uint32_t a = lo > sweep_begin ? lo : sweep_begin;
        if (a > hi) a = hi;
        segs.push_back({a, hi, anneal_scale(beta_scale, a0, j, S), true});
    }
    uint32_t main0 = S > 0 && B > sweep_begin ? B : sweep_begin;
    if (main0 > n_sweeps) main0 = n_sweeps;
    segs.push_back({main0, n_sweeps, beta_scale, false});
    return segs;
}

std::vector<Segment> plan_segments(const surfmcmc_opts& o, double beta_scale, uint32_t sweep_begin) {
    return plan_segments(o.n_sweeps, o.burn_in, o.anneal_stages, o.anneal_beta0, beta_scale, sweep_begin);
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
    uint32_t* state = nullptr;           // bundle state between segments
    unsigned int* unit_counter = nullptr;  // work queue of the persistent kernel
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

// Runs the segments of every group: plans[g] holds group g's segments (all of
// the same count); burn[g] its burn-in.  Segment i of every group runs in one
// launch at the temperature of plans[0][i].
int run_segments(surfmcmc_ctx* ctx, SweepParams sp, const std::vector<std::vector<Segment>>& plans,
                 const std::vector<uint32_t>& burn, double p, int lam, const SweepIO& io, cudaStream_t s) {
    int rc;
    const size_t ns = plans[0].size();
    for (size_t i = 0; i < ns; ++i) {
        const bool first = i == 0, last = i + 1 == ns;
        set_temperature(sp, p, plans[0][i].scale);
        for (int g = 0; g < sp.n_groups; ++g) {
            sp.grp[g].t_begin = plans[g][i].t0;
            sp.grp[g].t_end = plans[g][i].t1;
            sp.grp[g].burn_in = plans[g][i].anneal ? plans[g][i].t1 : burn[g];
        }
        sp.e0 = first ? io.e0 : nullptr;
        sp.e0code = first ? io.e0code : nullptr;
        sp.init_frames = first ? io.init_frames : nullptr;
        sp.state_in = first ? nullptr : io.state;
        sp.state_out = last ? nullptr : io.state;
        sp.init_sum = last ? io.init_sum : nullptr;
        sp.chain_sum = last ? io.chain_sum : nullptr;
        sp.chain_n = last ? io.chain_n : nullptr;
        sp.chain_frames = last ? io.chain_frames : nullptr;
        sp.unit_counter = io.unit_counter;
        std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
        if ((rc = record_start(ctx, &ev, s))) return rc;
        CK(launch_sweep(sp, lam, s));
        if ((rc = record_end(ctx, ev, s))) return rc;
    }
    return SURFMCMC_OK;
}

int run_segments(surfmcmc_ctx* ctx, const SweepParams& sp, const std::vector<Segment>& segs, uint32_t burn_in,
                 double p, int lam, const SweepIO& io, cudaStream_t s) {
    return run_segments(ctx, sp, std::vector<std::vector<Segment>>{segs}, std::vector<uint32_t>{burn_in}, p, lam,
                        io, s);
}


// ---------------------------------------------------------------------------
// Ragged batches: items of several code sizes and sweep counts in one call.
// ---------------------------------------------------------------------------
struct RaggedGroup {
    int L;
    uint32_t sweeps, burn;
    std::vector<long long> items;  // caller's indices
    double work;
};

struct RaggedLayout {
    std::vector<RaggedGroup> groups;       // in launch order (largest work first)
    std::vector<long long> perm;           // internal index -> caller's index
    std::vector<long long> src_off, dst_off;
    std::vector<int32_t> len;
    std::vector<uint64_t> samples;         // per internal item
    long long syn_bytes = 0, e0_words = 0, state_words = 0;
    int lam = 0;
    SweepParams sp;
};

int ragged_layout(surfmcmc_ctx* ctx, const int32_t* Ls, const uint32_t* sweeps, int64_t n, const surfmcmc_opts& o,
                  RaggedLayout& lay) {
    std::map<std::pair<int, uint32_t>, int> key;
    lay.src_off.resize(n);
    long long off = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int L = Ls[i];
        if (L < 2 || L > SURFMCMC_MAX_L) return fail(ctx, SURFMCMC_EINVAL, "item %lld: L=%d out of range", (long long)i, L);
        const uint32_t sw = sweeps ? sweeps[i] : o.n_sweeps;
        lay.src_off[i] = off;
        off += n_stabs(L);
        auto it = key.find({L, sw});
        if (it == key.end()) {
            if (key.size() == (size_t)kMaxGroups)
                return fail(ctx, SURFMCMC_EINVAL, "more than %d distinct (L, n_sweeps) pairs", kMaxGroups);
            const uint32_t burn = o.n_sweeps ? (uint32_t)((uint64_t)sw * o.burn_in / o.n_sweeps) : 0;
            if (o.anneal_stages > 0 && burn < (uint32_t)o.anneal_stages)
                return fail(ctx, SURFMCMC_EINVAL, "item %lld: burn-in %u shorter than the annealing stages", (long long)i,
                            burn);
            it = key.emplace(std::make_pair(L, sw), (int)lay.groups.size()).first;
            lay.groups.push_back({L, sw, burn, {}, 0.0});
        }
        lay.groups[it->second].items.push_back(i);
    }
    lay.syn_bytes = off;
    for (auto& g : lay.groups) g.work = (double)g.items.size() * g.sweeps * (double)n_stabs(g.L);
    std::stable_sort(lay.groups.begin(), lay.groups.end(),
                     [](const RaggedGroup& a, const RaggedGroup& b) { return a.work > b.work; });
    // lanes per bundle for the heaviest group, widened until the largest size fits
    int lmax = 0;
    for (auto& g : lay.groups) lmax = std::max(lmax, g.L);
    if (pick_lanes(lay.groups.empty() ? 2 : lay.groups[0].L, o.lanes_per_bundle, &lay.lam, ctx, o.chains_per_class))
        return fail(ctx, SURFMCMC_EINVAL, "lanes_per_bundle=%d unsupported", o.lanes_per_bundle);
    if (o.scan) lay.lam = 32;
    while (sweep_smem_bytes(n_qubits(lmax), lmax * (lmax - 1) / 2, lay.lam) > 200 * 1024 && lay.lam < 32) lay.lam *= 2;
    const int Cn = 4 * o.chains_per_class;
    init_chains(lay.sp, Cn, o.chains_per_class, 0);
    if (!lay.groups.empty()) lay.sp.max_blocks_per_sm = tuned_blocks(ctx, lay.groups[0].L, o.chains_per_class, o.lanes_per_bundle);
    lay.sp.scan = o.scan;
    lay.sp.noise = o.noise;
    energy_table(o, lay.sp.energy);
    long long dst = 0, item = 0, e0w = 0, stw = 0;
    for (auto& g : lay.groups) {
        add_group(lay.sp, g.L, (long long)g.items.size(), item, e0w, 0, stw, lay.lam);
        for (long long i : g.items) {
            lay.perm.push_back(i);
            lay.dst_off.push_back(dst);
            lay.len.push_back(n_stabs(g.L));
            lay.samples.push_back(g.sweeps > g.burn ? samples_per_sweep(o, g.L) * o.chains_per_class * (g.sweeps - g.burn)
                                                    : 0);
            dst += n_stabs(g.L);
        }
        item += (long long)g.items.size();
        e0w += (long long)g.items.size() * 2 * n_words(g.L);
        stw += lay.sp.grp[lay.sp.n_groups - 1].n_bundles * 2 * n_qubits(g.L);
    }
    lay.e0_words = e0w;
    lay.state_words = stw;
    return SURFMCMC_OK;
}

// Device scratch of a ragged run, carved from one base pointer.
struct RaggedScratch {
    uint8_t* syn;
    uint32_t* ids;
    long long *src_off, *dst_off, *perm;
    int32_t* len;
    uint64_t* samples;
    uint32_t* e0;
    int32_t* code;
    uint64_t* chain_sum;
    uint32_t* state;
    unsigned int* ctr;
};

size_t ragged_scratch(const RaggedLayout& lay, long long n, int Cn, char* base, RaggedScratch* rs) {
    Carver cv;
    const size_t o_syn = cv.reserve(lay.syn_bytes), o_ids = cv.reserve(n * 4), o_src = cv.reserve(n * 8),
                 o_dst = cv.reserve(n * 8), o_perm = cv.reserve(n * 8), o_len = cv.reserve(n * 4),
                 o_smp = cv.reserve(n * 8), o_e0 = cv.reserve(lay.e0_words * 4), o_code = cv.reserve(n * 4),
                 o_cs = cv.reserve((size_t)n * Cn * 8), o_st = cv.reserve(lay.state_words * 4),
                 o_ctr = cv.reserve(sizeof(unsigned int));
    if (base && rs) {
        rs->syn = (uint8_t*)(base + o_syn);
        rs->ids = (uint32_t*)(base + o_ids);
        rs->src_off = (long long*)(base + o_src);
        rs->dst_off = (long long*)(base + o_dst);
        rs->perm = (long long*)(base + o_perm);
        rs->len = (int32_t*)(base + o_len);
        rs->samples = (uint64_t*)(base + o_smp);
        rs->e0 = (uint32_t*)(base + o_e0);
        rs->code = (int32_t*)(base + o_code);
        rs->chain_sum = (uint64_t*)(base + o_cs);
        rs->state = (uint32_t*)(base + o_st);
        rs->ctr = (unsigned int*)(base + o_ctr);
    }
    return cv.off;
}

// Copies the host-side tables of the layout to the scratch (synchronously).
int ragged_upload(surfmcmc_ctx* ctx, const RaggedLayout& lay, long long n, const RaggedScratch& rs, cudaStream_t s) {
    if (n == 0) return SURFMCMC_OK;
    // src_off is indexed by the caller's index in the gather kernel
    CK(cudaMemcpyAsync(rs.src_off, lay.src_off.data(), n * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(rs.dst_off, lay.dst_off.data(), n * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(rs.perm, lay.perm.data(), n * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(rs.len, lay.len.data(), n * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(rs.samples, lay.samples.data(), n * 8, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}

// All device work of a ragged run (kernels and memsets only, so that it can
// be captured into a graph): gather, start frames per group, the sweep
// segments of every group, decision scattered to the caller's order.
int ragged_enqueue(surfmcmc_ctx* ctx, const RaggedLayout& lay, long long n, const surfmcmc_opts& o, double p,
                   uint64_t seed, const uint8_t* syn, const uint32_t* ids, uint32_t id0, const RaggedScratch& rs,
                   int32_t* out_class, uint64_t* out_class_sum, double* out_log_ratio, cudaStream_t s) {
    int rc;
    if (n == 0) return SURFMCMC_OK;
    CK(launch_gather_rows(n, syn, rs.src_off, rs.dst_off, rs.len, rs.perm, ids, id0, rs.syn, rs.ids, s));
    SweepParams sp = lay.sp;
    sp.ids = rs.ids;
    make_round_keys((uint32_t)seed, (uint32_t)(seed >> 32), &sp.rk);
    std::vector<std::vector<Segment>> plans;
    std::vector<uint32_t> burn;
    long long syn_off = 0;
    for (size_t g = 0; g < lay.groups.size(); ++g) {
        const GroupDesc& gd = sp.grp[g];
        CK(launch_start_frames(rs.syn + syn_off, gd.n, gd.L, rs.e0 + gd.e0_off, rs.code + gd.item_base, s));
        syn_off += gd.n * n_stabs(gd.L);
        plans.push_back(plan_segments(lay.groups[g].sweeps, lay.groups[g].burn, o.anneal_stages, o.anneal_beta0,
                                      o.beta_scale, 0));
        burn.push_back(lay.groups[g].burn);
    }
    SweepIO io;
    io.e0 = rs.e0;
    io.e0code = rs.code;
    io.chain_sum = rs.chain_sum;
    io.state = rs.state;
    io.unit_counter = rs.ctr;
    if ((rc = run_segments(ctx, sp, plans, burn, p, lay.lam, io, s))) return rc;
    uint64_t T[33];
    double beta_bar;
    int Eo[4];
    energy_table(o, Eo);
    acceptance_table(noise_rate(p, o.noise, Eo), 1.0, T, &beta_bar);
    DecideParams dp;
    memset(&dp, 0, sizeof dp);
    dp.n = n;
    dp.K = 4;
    dp.R = o.chains_per_class;
    dp.samples_per_item = rs.samples;
    dp.perm = rs.perm;
    dp.beta_bar = beta_bar;
    dp.chain_sum = rs.chain_sum;
    dp.out_class = out_class;
    dp.out_class_sum = out_class_sum;
    dp.out_log_ratio = out_log_ratio;
    CK(launch_decide(dp, s));
    return SURFMCMC_OK;
}

int ragged_check(surfmcmc_ctx* ctx, const int32_t* Ls, int64_t n, const surfmcmc_opts& o, double p, const uint32_t* ids,
                 uint32_t id0) {
    int rc;
    if (!ctx) return SURFMCMC_EINVAL;
    if (n < 0) return fail(ctx, SURFMCMC_EINVAL, "n=%lld < 0", (long long)n);
    if (n > 0 && !Ls) return fail(ctx, SURFMCMC_EINVAL, "NULL Ls");
    if (!ids && (uint64_t)id0 + (uint64_t)n > 4294967296ull)
        return fail(ctx, SURFMCMC_EINVAL, "syndrome ids id0+n exceed 2^32");
    if ((rc = check_opts(ctx, o, p))) return rc;
    if ((rc = reject_toric(ctx, o, "ragged decoding"))) return rc;
    return SURFMCMC_OK;
}

// Host copies of per-item arrays that may live on the device.
template <typename T>
int host_copy(surfmcmc_ctx* ctx, const T* ptr, int64_t n, std::vector<T>& out) {
    out.resize(n);
    if (n == 0 || !ptr) return SURFMCMC_OK;
    if (is_device_ptr(ptr)) CK(cudaMemcpy(out.data(), ptr, n * sizeof(T), cudaMemcpyDeviceToHost));
    else memcpy(out.data(), ptr, n * sizeof(T));
    return SURFMCMC_OK;
}

}  // namespace

struct surfmcmc_plan {
    surfmcmc_ctx* ctx = nullptr;
    void* scratch = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace surfmcmc {

void ctx_set_error(surfmcmc_ctx* ctx, const char* msg) {
    if (ctx) ctx->last_error = msg;
}

int ctx_device(const surfmcmc_ctx* ctx) { return ctx->device; }

bool device_ptr(const void* p) { return is_device_ptr(p); }

}  // namespace surfmcmc

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
    o->scan = 0;
    o->noise = 0;
    o->pauli_energy[0] = o->pauli_energy[1] = o->pauli_energy[2] = 1;
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
    ctx->sms = prop.multiProcessorCount;
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
    return surfmcmc_gen_syndromes_noise(ctx, seed, id0, n, L, p, 0, syndromes, true_class, stream);
}

int surfmcmc_gen_syndromes_toric(surfmcmc_ctx* ctx, uint64_t seed, uint32_t id0, int64_t n, int32_t L, double p,
                                 uint8_t* syndromes, int32_t* true_class, void* stream) {
    int rc = check_common(ctx, n, L, id0);
    if (rc) return rc;
    if (L < 2 || L > 30 || (L & 1)) return fail(ctx, SURFMCMC_EINVAL, "toric code needs an even L in 2..30");
    if (!(p >= 0.0 && p <= 0.75)) return fail(ctx, SURFMCMC_EINVAL, "p=%g outside [0, 0.75]", p);
    if (n > 0 && !syndromes) return fail(ctx, SURFMCMC_EINVAL, "syndromes is NULL");
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Carver cv;
    Buf bs, bt;
    plan(bs, syndromes, (size_t)n * geo_nstab(1, L), cv);
    plan(bt, true_class, true_class ? (size_t)n * 4 : 0, cv);
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    bind(bs, ctx);
    bind(bt, ctx);
    CK(launch_gen_syndromes_toric(seed, id0, n, L, p, (uint8_t*)bs.dev, (int32_t*)bt.dev, s));
    if ((rc = copy_out(ctx, bs, s)) || (rc = copy_out(ctx, bt, s))) return rc;
    if (!stream || bs.staged || bt.staged) CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}

int surfmcmc_gen_syndromes_pauli(surfmcmc_ctx* ctx, uint64_t seed, uint32_t id0, int64_t n, int32_t L, double px,
                                 double py, double pz, uint8_t* syndromes, int32_t* true_class, void* stream) {
    int rc = check_common(ctx, n, L, id0);
    if (rc) return rc;
    if (!(px >= 0.0 && py >= 0.0 && pz >= 0.0 && px + py + pz <= 0.75))
        return fail(ctx, SURFMCMC_EINVAL, "pX, pY, pZ must be >= 0 with pX + pY + pZ <= 0.75");
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
    CK(launch_gen_syndromes_pauli(seed, id0, n, L, px, py, pz, (uint8_t*)bs.dev, (int32_t*)bt.dev, s));
    if ((rc = copy_out(ctx, bs, s)) || (rc = copy_out(ctx, bt, s))) return rc;
    if (!stream || bs.staged || bt.staged) CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}

int surfmcmc_gen_syndromes_noise(surfmcmc_ctx* ctx, uint64_t seed, uint32_t id0, int64_t n, int32_t L, double p,
                                 int32_t noise, uint8_t* syndromes, int32_t* true_class, void* stream) {
    int rc = check_common(ctx, n, L, id0);
    if (rc) return rc;
    if (noise != 0 && noise != 1) return fail(ctx, SURFMCMC_EINVAL, "noise=%d must be 0 or 1", noise);
    if (!(p >= 0.0 && p <= (noise ? 1.0 : 0.75)))
        return fail(ctx, SURFMCMC_EINVAL, "p=%g outside [0, %g]", p, noise ? 1.0 : 0.75);
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
    CK(launch_gen_syndromes(seed, id0, n, L, p, (uint8_t*)bs.dev, (int32_t*)bt.dev, s, noise));
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
                       int32_t* out_chain_n, uint32_t* out_chain_frames, uint64_t* out_chain_accepts,
                       void* stream) {
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
    if ((rc = check_toric(ctx, o, L))) return rc;
    const int toric = o.n_classes == 16 ? 1 : 0;
    int lam = 0;
    if (pick_lanes(L, o.lanes_per_bundle, &lam, ctx, o.chains_per_class, toric))
        return fail(ctx, SURFMCMC_EINVAL, "lanes_per_bundle=%d unsupported for L=%d", o.lanes_per_bundle, L);
    if (o.scan || out_chain_accepts) lam = 32;   // counting accepts: the LAM = 32 kernels (same results)
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;

    const int K = o.n_classes, R = o.chains_per_class, Cn = K * R;
    const int nq = geo_nq(toric, L), W = geo_words(toric, L), ns = geo_nstab(toric, L);
    int G = 1;
    while (G < Cn && G < 32) G *= 2;

    SweepParams sp;
    init_chains(sp, Cn, R, id0);
    sp.code = toric;
    sp.scan = o.scan;
    sp.noise = o.noise;
    sp.max_blocks_per_sm = tuned_blocks(ctx, L, R, o.lanes_per_bundle);
    energy_table(o, sp.energy);
    lam = widen_lanes(ctx, L, o.lanes_per_bundle, lam, bundles_of(sp, n), sp.G, toric);
    add_group(sp, L, n, 0, 0, 0, 0, lam);
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
    // accept counts: the caller's device buffer, else scratch (when asked for)
    const bool acc_scratch = out_chain_accepts && !is_device_ptr(out_chain_accepts);
    const size_t off_acc = acc_scratch ? cv.reserve((size_t)n * Cn * 8) : 0;
    const size_t off_e0 = init_frames ? 0 : cv.reserve((size_t)n * 2 * W * 4);
    const size_t off_code = init_frames ? 0 : cv.reserve((size_t)n * 4);
    const std::vector<Segment> segs = plan_segments(o, o.beta_scale, sweep_begin);
    const size_t off_state = segs.size() > 1 ? cv.reserve((size_t)sp.grp[0].n_bundles * 2 * nq * 4) : 0;
    const size_t off_ctr = cv.reserve(sizeof(unsigned int));
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    Buf* all[] = {&b_syn, &b_if, &b_is, &b_cls, &b_csum, &b_lr, &b_chn, &b_chf};
    for (Buf* b : all) bind(*b, ctx);
    char* base = (char*)ctx->arena;
    uint64_t* chain_sum = chs_scratch ? (uint64_t*)(base + off_chs) : out_chain_sum;
    uint64_t* accepts = acc_scratch ? (uint64_t*)(base + off_acc) : out_chain_accepts;
    uint32_t* e0 = init_frames ? nullptr : (uint32_t*)(base + off_e0);
    int32_t* code = init_frames ? nullptr : (int32_t*)(base + off_code);
    uint32_t* state = segs.size() > 1 ? (uint32_t*)(base + off_state) : nullptr;
    unsigned int* ctr = (unsigned int*)(base + off_ctr);

    if ((rc = copy_in(ctx, b_syn, s)) || (rc = copy_in(ctx, b_if, s)) || (rc = copy_in(ctx, b_is, s))) return rc;
    if (!init_frames) CK(launch_start_frames((const uint8_t*)b_syn.dev, n, L, e0, code, s, toric));
    if (accepts) CK(cudaMemsetAsync(accepts, 0, (size_t)n * Cn * 8, s));
    sp.accepts = accepts;   // every launch adds to the counts

    SweepIO io;
    io.e0 = e0;
    io.e0code = code;
    io.init_frames = (const uint32_t*)b_if.dev;
    io.init_sum = (const uint64_t*)b_is.dev;
    io.chain_sum = chain_sum;
    io.chain_n = (int32_t*)b_chn.dev;
    io.chain_frames = (uint32_t*)b_chf.dev;
    io.state = state;
    io.unit_counter = ctr;
    if ((rc = run_segments(ctx, sp, segs, o.burn_in, p, lam, io, s))) return rc;

    uint64_t T[33];
    double beta_bar;
    int Eo[4];
    energy_table(o, Eo);
    acceptance_table(noise_rate(p, o.noise, Eo), 1.0, T, &beta_bar);
    DecideParams dp;
    memset(&dp, 0, sizeof dp);
    dp.n = n;
    dp.K = K;
    dp.R = R;
    dp.samples = o.n_sweeps > o.burn_in ? samples_per_sweep(o, L) * R * (o.n_sweeps - o.burn_in) : 0;
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
    if (acc_scratch) {
        CK(cudaMemcpyAsync(out_chain_accepts, accepts, (size_t)n * Cn * 8, cudaMemcpyDeviceToHost, s));
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
    if ((rc = check_toric(ctx, o, L))) return rc;
    const int toric = o.n_classes == 16 ? 1 : 0;
    int lam = 0;
    if (pick_lanes(L, o.lanes_per_bundle, &lam, nullptr, 0, toric))
        return fail(ctx, SURFMCMC_EINVAL, "lanes_per_bundle=%d unsupported for L=%d", o.lanes_per_bundle, L);
    if (o.scan) lam = 32;
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int K = o.n_classes, R = o.chains_per_class, Cn = K * R, N = n_beta;
    SweepParams sp;
    init_chains(sp, Cn, R, id0);
    sp.code = toric;
    sp.scan = o.scan;
    sp.noise = o.noise;
    energy_table(o, sp.energy);
    // a batch too small to fill the device gets more lanes per bundle (the
    // results do not depend on the lane split)
    lam = widen_lanes(ctx, L, o.lanes_per_bundle, lam, bundles_of(sp, n), sp.G, toric);
    add_group(sp, L, n, 0, 0, 0, 0, lam);
    const std::vector<Segment> segs0 = plan_segments(o, o.beta_scale, 0);
    const int W = geo_words(toric, L), nq = geo_nq(toric, L);

    Carver cv;
    Buf b_syn, b_cls, b_lz;
    plan(b_syn, (void*)syndromes, (size_t)n * geo_nstab(toric, L), cv);
    plan(b_cls, out_class, (size_t)n * 4, cv);
    plan(b_lz, out_log_z, out_log_z ? (size_t)n * K * 8 : 0, cv);
    const bool mean_scratch = !out_mean || !is_device_ptr(out_mean);
    const size_t off_mean = mean_scratch ? cv.reserve((size_t)n * K * N * 8) : 0;
    const size_t off_chs = cv.reserve((size_t)n * Cn * 8);
    const size_t off_e0 = cv.reserve((size_t)n * 2 * W * 4);
    const size_t off_code = cv.reserve((size_t)n * 4);
    const size_t off_state = segs0.size() > 1 ? cv.reserve((size_t)sp.grp[0].n_bundles * 2 * nq * 4) : 0;
    const size_t off_ctr = cv.reserve(sizeof(unsigned int));
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    for (Buf* b : {&b_syn, &b_cls, &b_lz}) bind(*b, ctx);
    char* base = (char*)ctx->arena;
    double* mean = mean_scratch ? (double*)(base + off_mean) : out_mean;
    uint64_t* chain_sum = (uint64_t*)(base + off_chs);
    uint32_t* e0 = (uint32_t*)(base + off_e0);
    int32_t* code = (int32_t*)(base + off_code);
    uint32_t* state = segs0.size() > 1 ? (uint32_t*)(base + off_state) : nullptr;
    unsigned int* ctr = (unsigned int*)(base + off_ctr);

    if ((rc = copy_in(ctx, b_syn, s))) return rc;
    CK(launch_start_frames((const uint8_t*)b_syn.dev, n, L, e0, code, s, toric));
    const uint64_t samples = samples_per_sweep(o, L) * R * (o.n_sweeps - o.burn_in);
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
        io.unit_counter = ctr;
        if ((rc = run_segments(ctx, sp, plan_segments(o, bs, 0), o.burn_in, p, lam, io, s))) return rc;
        CK(launch_class_means(n, K, R, N, j, samples, chain_sum, mean, s));
    }
    uint64_t T[33];
    double beta_bar;
    int Eo[4];
    energy_table(o, Eo);
    acceptance_table(noise_rate(p, o.noise, Eo), 1.0, T, &beta_bar);
    const double h = (o.beta_scale * beta_bar) / (double)(N - 1);
    // <n> at beta = 0: every Pauli equally likely on each qubit, so n_q times
    // the mean of the four energies (3/4 n_q depolarizing, n_q flips)
    const double mean0 = (double)nq * (double)(Eo[1] + Eo[2] + Eo[3]) / 4.0;
    CK(launch_ti_decide(n, K, N, mean0, h / 3.0, mean, (int32_t*)b_cls.dev, (double*)b_lz.dev, s));

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


int surfmcmc_decode_ragged(surfmcmc_ctx* ctx, const uint8_t* syndromes, const int32_t* Ls, const uint32_t* n_sweeps,
                           int64_t n, double p, const surfmcmc_opts* opts_in, uint64_t seed, const uint32_t* ids,
                           uint32_t id0, int32_t* out_class, uint64_t* out_class_sum, double* out_log_ratio,
                           void* stream) {
    surfmcmc_opts o;
    surfmcmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    int rc = ragged_check(ctx, Ls, n, o, p, ids, id0);
    if (rc) return rc;
    if (n > 0 && (!syndromes || !out_class)) return fail(ctx, SURFMCMC_EINVAL, "NULL syndromes or out_class");
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> hL;
    std::vector<uint32_t> hS;
    if ((rc = host_copy(ctx, Ls, n, hL))) return rc;
    if (n_sweeps && (rc = host_copy(ctx, n_sweeps, n, hS))) return rc;
    RaggedLayout lay;
    if ((rc = ragged_layout(ctx, hL.data(), n_sweeps ? hS.data() : nullptr, n, o, lay))) return rc;
    const int Cn = 4 * o.chains_per_class;
    Carver cv;
    cv.off = ragged_scratch(lay, n, Cn, nullptr, nullptr);
    Buf b_syn, b_ids, b_cls, b_csum, b_lr;
    plan(b_syn, (void*)syndromes, lay.syn_bytes, cv);
    plan(b_ids, (void*)ids, ids ? (size_t)n * 4 : 0, cv);
    plan(b_cls, out_class, (size_t)n * 4, cv);
    plan(b_csum, out_class_sum, out_class_sum ? (size_t)n * 32 : 0, cv);
    plan(b_lr, out_log_ratio, out_log_ratio ? (size_t)n * 32 : 0, cv);
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    for (Buf* b : {&b_syn, &b_ids, &b_cls, &b_csum, &b_lr}) bind(*b, ctx);
    RaggedScratch rs;
    ragged_scratch(lay, n, Cn, (char*)ctx->arena, &rs);
    if ((rc = ragged_upload(ctx, lay, n, rs, s))) return rc;
    if ((rc = copy_in(ctx, b_syn, s)) || (rc = copy_in(ctx, b_ids, s))) return rc;
    if ((rc = ragged_enqueue(ctx, lay, n, o, p, seed, (const uint8_t*)b_syn.dev, (const uint32_t*)b_ids.dev, id0, rs,
                             (int32_t*)b_cls.dev, (uint64_t*)b_csum.dev, (double*)b_lr.dev, s)))
        return rc;
    bool any_host = false;
    for (Buf* b : {&b_cls, &b_csum, &b_lr}) {
        if ((rc = copy_out(ctx, *b, s))) return rc;
        any_host |= b->staged;
    }
    if (!stream || any_host) CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}

int surfmcmc_ragged_plan_create(surfmcmc_ctx* ctx, const int32_t* Ls, const uint32_t* n_sweeps, int64_t n, double p,
                                const surfmcmc_opts* opts_in, uint64_t seed, const uint8_t* syndromes,
                                const uint32_t* ids, uint32_t id0, int32_t* out_class, uint64_t* out_class_sum,
                                double* out_log_ratio, surfmcmc_plan** out_plan) {
    if (!out_plan) return ctx ? fail(ctx, SURFMCMC_EINVAL, "NULL plan") : SURFMCMC_EINVAL;
    *out_plan = nullptr;
    surfmcmc_opts o;
    surfmcmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    int rc = ragged_check(ctx, Ls, n, o, p, ids, id0);
    if (rc) return rc;
    if (n <= 0) return fail(ctx, SURFMCMC_EINVAL, "a plan needs n > 0");
    if (!is_device_ptr(syndromes) || !is_device_ptr(out_class) || (ids && !is_device_ptr(ids)) ||
        (out_class_sum && !is_device_ptr(out_class_sum)) || (out_log_ratio && !is_device_ptr(out_log_ratio)))
        return fail(ctx, SURFMCMC_EINVAL, "a plan works on device buffers only");
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    std::vector<int32_t> hL;
    std::vector<uint32_t> hS;
    if ((rc = host_copy(ctx, Ls, n, hL))) return rc;
    if (n_sweeps && (rc = host_copy(ctx, n_sweeps, n, hS))) return rc;
    RaggedLayout lay;
    if ((rc = ragged_layout(ctx, hL.data(), n_sweeps ? hS.data() : nullptr, n, o, lay))) return rc;
    const int Cn = 4 * o.chains_per_class;
    surfmcmc_plan* pl = new surfmcmc_plan;
    pl->ctx = ctx;
    auto cleanup = [&](int code) {
        if (pl->exec) cudaGraphExecDestroy(pl->exec);
        if (pl->graph) cudaGraphDestroy(pl->graph);
        if (pl->scratch) cudaFree(pl->scratch);
        delete pl;
        return code;
    };
    const size_t bytes = ragged_scratch(lay, n, Cn, nullptr, nullptr);
    cudaError_t e = cudaMalloc(&pl->scratch, bytes);
    if (e != cudaSuccess) return cleanup(fail(ctx, SURFMCMC_ENOMEM, "plan scratch: %s", cudaGetErrorString(e)));
    RaggedScratch rs;
    ragged_scratch(lay, n, Cn, (char*)pl->scratch, &rs);
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess)
        return cleanup(fail(ctx, SURFMCMC_ECUDA, "stream: %s", cudaGetErrorString(e)));
    if ((rc = ragged_upload(ctx, lay, n, rs, cap)) ||
        (e = prepare_sweep(lay.sp, lay.lam)) != cudaSuccess) {
        cudaStreamDestroy(cap);
        return cleanup(rc ? rc : fail(ctx, SURFMCMC_ECUDA, "prepare: %s", cudaGetErrorString(e)));
    }
    const bool timing = ctx->timing;
    ctx->timing = false;  // no event nodes in the graph
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = ragged_enqueue(ctx, lay, n, o, p, seed, syndromes, ids, id0, rs, out_class, out_class_sum, out_log_ratio,
                            cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &pl->graph);
        if (!rc && e2 != cudaSuccess) e = e2;
    }
    ctx->timing = timing;
    cudaStreamDestroy(cap);
    if (rc) return cleanup(rc);
    if (e != cudaSuccess) return cleanup(fail(ctx, SURFMCMC_ECUDA, "capture: %s", cudaGetErrorString(e)));
    if ((e = cudaGraphInstantiate(&pl->exec, pl->graph, 0)) != cudaSuccess)
        return cleanup(fail(ctx, SURFMCMC_ECUDA, "instantiate: %s", cudaGetErrorString(e)));
    *out_plan = pl;
    return SURFMCMC_OK;
}

int surfmcmc_plan_launch(surfmcmc_plan* plan, void* stream) {
    if (!plan) return SURFMCMC_EINVAL;
    surfmcmc_ctx* ctx = plan->ctx;
    DeviceGuard g(ctx->device);
    CK(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
    if (!stream) CK(cudaStreamSynchronize((cudaStream_t)stream));
    return SURFMCMC_OK;
}

void surfmcmc_plan_destroy(surfmcmc_plan* plan) {
    if (!plan) return;
    DeviceGuard g(plan->ctx->device);
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->scratch) cudaFree(plan->scratch);
    delete plan;
}


int surfmcmc_autotune(surfmcmc_ctx* ctx, int32_t L, int32_t chains_per_class, double p, int64_t n_probe,
                      uint32_t sweeps, int32_t* best_lanes, int32_t* best_blocks_per_sm, double* ms_out) {
    int rc = check_common(ctx, n_probe, L, 0);
    if (rc) return rc;
    if (n_probe < 1 || sweeps < 1 || chains_per_class < 1 || 4 * chains_per_class > 1024 || !(p > 0.0 && p <= 0.75))
        return fail(ctx, SURFMCMC_EINVAL, "autotune needs n_probe, sweeps >= 1, valid R and p");
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    const int R = chains_per_class, Cn = 4 * R, nq = n_qubits(L), W = n_words(L);
    const int cand[SURFMCMC_TUNE_LANES] = {2, 4, 8, 16, 32};
    const int bcand[SURFMCMC_TUNE_BLOCKS] = {6, 5, 4, 3};
    SweepParams base;
    init_chains(base, Cn, R, 0);
    Carver cv;
    const size_t o_syn = cv.reserve((size_t)n_probe * n_stabs(L)), o_e0 = cv.reserve((size_t)n_probe * 2 * W * 4),
                 o_code = cv.reserve((size_t)n_probe * 4), o_cs = cv.reserve((size_t)n_probe * Cn * 8),
                 o_ctr = cv.reserve(sizeof(unsigned int));
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    char* b = (char*)ctx->arena;
    uint8_t* syn = (uint8_t*)(b + o_syn);
    uint32_t* e0 = (uint32_t*)(b + o_e0);
    int32_t* code = (int32_t*)(b + o_code);
    cudaStream_t s;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e_a, e_b;
    CK(cudaEventCreate(&e_a));
    CK(cudaEventCreate(&e_b));
    CK(launch_gen_syndromes(0x7475ull, 0, n_probe, L, p, syn, nullptr, s));
    CK(launch_start_frames(syn, n_probe, L, e0, code, s));
    int best = 0, best_b = 0;
    float best_ms = 0.f;
    for (int i = 0; i < SURFMCMC_TUNE_LANES; ++i) {
        for (int j = 0; j < SURFMCMC_TUNE_BLOCKS; ++j) {
            double* slot = ms_out ? ms_out + i * SURFMCMC_TUNE_BLOCKS + j : nullptr;
            if (slot) *slot = NAN;
            const int lam = cand[i];
            if (sweep_smem_bytes(nq, L * (L - 1) / 2, lam) > kSweepSmemLimit) continue;
            SweepParams sp = base;
            sp.max_blocks_per_sm = bcand[j];
            add_group(sp, L, n_probe, 0, 0, 0, 0, lam);
            set_temperature(sp, p, 1.0);
            make_round_keys(0x7475u, 0u, &sp.rk);
            sp.grp[0].t_begin = 0;
            sp.grp[0].t_end = sweeps;
            sp.grp[0].burn_in = 0;
            sp.e0 = e0;
            sp.e0code = code;
            sp.chain_sum = (uint64_t*)(b + o_cs);
            sp.unit_counter = (unsigned int*)(b + o_ctr);
            CK(launch_sweep(sp, lam, s));  // warm-up
            CK(cudaEventRecord(e_a, s));
            CK(launch_sweep(sp, lam, s));
            CK(cudaEventRecord(e_b, s));
            CK(cudaEventSynchronize(e_b));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e_a, e_b));
            if (slot) *slot = ms;
            if (!best || ms < best_ms) {
                best = lam;
                best_b = bcand[j];
                best_ms = ms;
            }
        }
    }
    cudaEventDestroy(e_a);
    cudaEventDestroy(e_b);
    cudaStreamDestroy(s);
    if (!best) return fail(ctx, SURFMCMC_EINVAL, "no lanes_per_bundle fits L=%d", L);
    ctx->tuned[{L, R}] = Tuned{best, best_b};
    if (best_lanes) *best_lanes = best;
    if (best_blocks_per_sm) *best_blocks_per_sm = best_b;
    return SURFMCMC_OK;
}

int surfmcmc_decode_early(surfmcmc_ctx* ctx, surfmcmc_cnn* net, const uint8_t* syndromes, int64_t n, int32_t L,
                          double p, const surfmcmc_opts* opts_in, uint32_t chunk_sweeps, float tau, int32_t reorder,
                          uint64_t seed, uint32_t id0, int32_t* out_class, uint64_t* out_class_sum,
                          uint32_t* out_sweeps, void* stream) {
    int rc = check_common(ctx, n, L, id0);
    if (rc) return rc;
    surfmcmc_opts o;
    surfmcmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    if ((rc = check_opts(ctx, o, p))) return rc;
    if ((rc = reject_toric(ctx, o, "early stop"))) return rc;
    if (!net || cnn_code_size(net) != L) return fail(ctx, SURFMCMC_EINVAL, "network missing or built for another L");
    if (chunk_sweeps == 0) return fail(ctx, SURFMCMC_EINVAL, "chunk_sweeps must be > 0");
    if (tau != tau) return fail(ctx, SURFMCMC_EINVAL, "tau is NaN");
    if (reorder != 0 && reorder != 1) return fail(ctx, SURFMCMC_EINVAL, "reorder must be 0 or 1");
    if (n > 0 && (!syndromes || !out_class)) return fail(ctx, SURFMCMC_EINVAL, "NULL syndromes or out_class");
    int lam = 0;
    if (pick_lanes(L, o.lanes_per_bundle, &lam, ctx, o.chains_per_class))
        return fail(ctx, SURFMCMC_EINVAL, "lanes_per_bundle=%d unsupported for L=%d", o.lanes_per_bundle, L);
    if (o.scan) lam = 32;
    if (n == 0) return SURFMCMC_OK;
    ctx->last_error.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;

    const int K = 4, R = o.chains_per_class, Cn = K * R;
    const int nq = n_qubits(L), W = n_words(L), ns = n_stabs(L);
    const int fw = Cn * 2 * W;  // frame words per item

    // checkpoints: burn_in + k chunk_sweeps (k >= 1) below n_sweeps, then n_sweeps
    std::vector<uint32_t> marks;
    for (uint64_t t = (uint64_t)o.burn_in + chunk_sweeps; t < o.n_sweeps; t += chunk_sweeps)
        marks.push_back((uint32_t)t);
    marks.push_back(o.n_sweeps);

    SweepParams sp0;
    init_chains(sp0, Cn, R, id0);
    sp0.max_blocks_per_sm = tuned_blocks(ctx, L, R, o.lanes_per_bundle);
    add_group(sp0, L, n, 0, 0, 0, 0, lam);
    const long long nb_max = sp0.grp[0].n_bundles;

    Carver cv;
    Buf b_syn, b_cls, b_csum, b_sw;
    plan(b_syn, (void*)syndromes, (size_t)n * ns, cv);
    plan(b_cls, out_class, (size_t)n * 4, cv);
    plan(b_csum, out_class_sum, out_class_sum ? (size_t)n * K * 8 : 0, cv);
    plan(b_sw, out_sweeps, out_sweeps ? (size_t)n * 4 : 0, cv);
    const size_t off_lp = cv.reserve((size_t)n * 16);
    const size_t off_perm[2] = {cv.reserve((size_t)n * 8), cv.reserve((size_t)n * 8)};
    const size_t off_ids[2] = {cv.reserve((size_t)n * 4), cv.reserve((size_t)n * 4)};
    const size_t off_fin = cv.reserve((size_t)n * fw * 4), off_fout = cv.reserve((size_t)n * fw * 4);
    const size_t off_sin = cv.reserve((size_t)n * Cn * 8), off_sout = cv.reserve((size_t)n * Cn * 8);
    const size_t off_keep = cv.reserve((size_t)n * 4);
    const size_t off_pos = cv.reserve((size_t)n * 8);
    const size_t off_cnt = cv.reserve(8);
    const size_t off_tcls = cv.reserve((size_t)n * 4);
    const size_t off_tsum = cv.reserve((size_t)n * K * 8);
    const size_t off_e0 = cv.reserve((size_t)n * 2 * W * 4);
    const size_t off_code = cv.reserve((size_t)n * 4);
    const size_t off_state = cv.reserve((size_t)nb_max * 2 * nq * 4);
    const size_t off_ctr = cv.reserve(sizeof(unsigned int));
    const size_t off_rank = reorder ? cv.reserve((size_t)n) : 0;
    const size_t off_frozen = reorder ? cv.reserve((size_t)n * 16) : 0;
    if ((rc = ensure_arena(ctx, cv.off))) return rc;
    Buf* all[] = {&b_syn, &b_cls, &b_csum, &b_sw};
    for (Buf* b : all) bind(*b, ctx);
    char* base = (char*)ctx->arena;
    auto at = [&](size_t off) { return (void*)(base + off); };
    float* logprob = (float*)at(off_lp);
    uint32_t* f_in = (uint32_t*)at(off_fin);
    uint32_t* f_out = (uint32_t*)at(off_fout);
    uint64_t* s_in = (uint64_t*)at(off_sin);
    uint64_t* s_out = (uint64_t*)at(off_sout);
    int32_t* keep = (int32_t*)at(off_keep);
    long long* cnt = (long long*)at(off_cnt);
    int32_t* tcls = (int32_t*)at(off_tcls);
    uint64_t* tsum = (uint64_t*)at(off_tsum);

    if ((rc = copy_in(ctx, b_syn, s))) return rc;
    CK(cnn_logprob(net, (const uint8_t*)b_syn.dev, n, logprob, s));
    CK(launch_start_frames((const uint8_t*)b_syn.dev, n, L, (uint32_t*)at(off_e0), (int32_t*)at(off_code), s));
    CK(launch_iota(n, (long long*)at(off_perm[0]), s));

    uint64_t T[33];
    double beta_bar;
    int Eo[4];
    energy_table(o, Eo);
    acceptance_table(noise_rate(p, o.noise, Eo), 1.0, T, &beta_bar);
    long long n_act = n;
    uint32_t t = 0;
    int cur = 0;  // pair holding the active items' caller indices and ids
    uint32_t t_reorder = 0;   // the checkpoint at which the budget was reordered (0: not yet)
    const uint64_t spp_r = (uint64_t)samples_per_sweep(o, L) * R;   // samples of one class per sweep
    for (size_t k = 0; k < marks.size() && n_act > 0; ++k) {
        const uint32_t tk = marks[k];
        const bool final_chunk = k + 1 == marks.size();
        // sweeps [t, tk) of the active items, resumed from their state at t
        SweepParams sp;
        init_chains(sp, Cn, R, id0);
        sp.scan = o.scan;
        sp.noise = o.noise;
        energy_table(o, sp.energy);
        sp.ids = t == 0 ? nullptr : (const uint32_t*)at(off_ids[cur]);
        const int lam_k = widen_lanes(ctx, L, o.lanes_per_bundle, lam, bundles_of(sp, n_act), sp.G);
        add_group(sp, L, n_act, 0, 0, 0, 0, lam_k);
        make_round_keys((uint32_t)seed, (uint32_t)(seed >> 32), &sp.rk);
        // the chunk's non-empty segments (annealing stages already passed are skipped)
        std::vector<Segment> segs;
        for (const Segment& sg : plan_segments(tk, o.burn_in, o.anneal_stages, o.anneal_beta0, o.beta_scale, t))
            if (sg.t1 > sg.t0) segs.push_back(sg);
        if (segs.empty()) segs.push_back({t, tk, o.beta_scale, false});
        SweepIO io;
        if (t == 0) {
            io.e0 = (uint32_t*)at(off_e0);
            io.e0code = (int32_t*)at(off_code);
        } else {
            io.init_frames = f_in;
            io.init_sum = s_in;
        }
        io.chain_sum = s_out;
        io.chain_frames = final_chunk ? nullptr : f_out;
        io.state = segs.size() > 1 ? (uint32_t*)at(off_state) : nullptr;
        io.unit_counter = (unsigned int*)at(off_ctr);
        if ((rc = run_segments(ctx, sp, segs, o.burn_in, p, lam_k, io, s))) return rc;

        // decision so far, then retire the items that may stop here
        if (t_reorder) {
            // reordered items: the top classes have their own chains (sampled
            // since the burn-in) and further replicas (since t_reorder)
            const uint64_t n_top = spp_r * ((uint64_t)(tk - o.burn_in) + (uint64_t)(tk - t_reorder));
            const uint64_t n_low = spp_r * (uint64_t)(t_reorder - o.burn_in);
            CK(launch_decide_reorder(n_act, (const long long*)at(off_perm[cur]), (const uint8_t*)at(off_rank),
                                     (const uint64_t*)at(off_frozen), R, s_out, n_top, n_low, tcls, tsum, s));
        } else {
            DecideParams dp;
            memset(&dp, 0, sizeof dp);
            dp.n = n_act;
            dp.K = K;
            dp.R = R;
            dp.samples = tk > o.burn_in ? samples_per_sweep(o, L) * R * (tk - o.burn_in) : 0;
            dp.beta_bar = beta_bar;
            dp.chain_sum = s_out;
            dp.out_class = tcls;
            dp.out_class_sum = tsum;
            CK(launch_decide(dp, s));
        }
        CK(launch_retire(n_act, (const long long*)at(off_perm[cur]), logprob, tcls, tsum, tau, tk,
                         final_chunk ? 1 : 0, (int32_t*)b_cls.dev, (uint64_t*)b_csum.dev, (uint32_t*)b_sw.dev, keep,
                         s));
        t = tk;
        if (final_chunk) break;
        // survivors, in order: caller indices and ids to the other pair, frames and sums to the inputs
        CK(launch_compact(n_act, keep, (long long*)at(off_pos), cnt, (const long long*)at(off_perm[cur]), id0, fw,
                          Cn, f_out, s_out, (long long*)at(off_perm[cur ^ 1]), (uint32_t*)at(off_ids[cur ^ 1]),
                          f_in, s_in, s));
        long long h_cnt = 0;
        CK(cudaMemcpyAsync(&h_cnt, cnt, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        n_act = h_cnt;
        cur ^= 1;
        if (reorder && !t_reorder) {
            // the chains of the survivors' two least likely classes continue
            // as replicas of the two most likely ones
            CK(launch_reorder(n_act, (const long long*)at(off_perm[cur]), logprob, R, 2 * W, f_in, s_in,
                              (uint8_t*)at(off_rank), (uint64_t*)at(off_frozen), s));
            t_reorder = tk;
        }
    }
    bool any_host = false;
    for (Buf* b : {&b_cls, &b_csum, &b_sw}) {
        if ((rc = copy_out(ctx, *b, s))) return rc;
        any_host |= b->staged;
    }
    if (!stream || any_host) CK(cudaStreamSynchronize(s));
    return SURFMCMC_OK;
}

int surfmcmc_decode(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L, double p,
                    const surfmcmc_opts* opts, uint64_t seed, uint32_t id0, int32_t* out_class,
                    uint64_t* out_class_sum, double* out_log_ratio, void* stream) {
    return surfmcmc_decode_ex(ctx, syndromes, n, L, p, opts, seed, id0, 0, nullptr, nullptr, out_class,
                              out_class_sum, out_log_ratio, nullptr, nullptr, nullptr, nullptr, stream);
}

}  // extern "C"
