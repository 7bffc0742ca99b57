// Internal declarations shared by the translation units of libsurfmcmc.
// Device helpers: Philox4x32-10, code geometry, and the parameter blocks of
// the kernels.  Nothing here is visible through the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

struct surfmcmc_ctx;
struct surfmcmc_cnn;

namespace surfmcmc {

constexpr int kMaxL = 31;
constexpr int kMaxWords = (2 * kMaxL * kMaxL - 2 * kMaxL + 1 + 31) / 32;  // 59
constexpr int kCountBits = 12;  // n <= 2 n_q(31) = 3722 < 2^12 (independent flips)

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  The ten round keys are
// precomputed on the host (key + i * Weyl constants), so a round is two
// 32x32->64 multiplications (written as their high and low halves, which
// measured 2 % faster in the sweep kernel than a 64-bit product) and two
// three-input XORs.
// ---------------------------------------------------------------------------
struct RoundKeys {
    uint32_t k[20];  // k[2i], k[2i+1]: key words used in round i
};

constexpr uint32_t kPhiloxMa = 0xD2511F53u, kPhiloxMb = 0xCD9E8D57u;

// Rounds FIRST .. 9 of Philox4x32-10 on the state c after round FIRST - 1.
template <int FIRST = 0>
__device__ __forceinline__ uint4 philox_rounds(uint4 c, const RoundKeys& rk) {
#pragma unroll
    for (int i = FIRST; i < 10; ++i) {
        const uint32_t h0 = __umulhi(kPhiloxMa, c.x), l0 = kPhiloxMa * c.x;
        const uint32_t h1 = __umulhi(kPhiloxMb, c.z), l1 = kPhiloxMb * c.z;
        c = make_uint4(h1 ^ c.y ^ rk.k[2 * i], l1, h0 ^ c.w ^ rk.k[2 * i + 1], l0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox10(uint4 c, const RoundKeys& rk) { return philox_rounds<0>(c, rk); }

// The same generator split for counters (x0, y0, z0, w0) whose words x0 and
// w0 stay fixed over many blocks.  Round 0 gives z1 = hi(Ma x0) ^ w0 ^ k[1]
// and w1 = lo(Ma x0) from x0 and w0 alone, so round 1's products of z1 and
// w1 ^ k[3] are fixed as well: PhiloxFixed holds M = hi(Mb z1) ^ k[2],
// N = lo(Mb z1) and A = w1 ^ k[3].  The varying words give x1 = hi(Mb z0) ^
// y0 ^ k[0], y1 = lo(Mb z0), and the state after round 1 is
// (M ^ y1, N, hi(Ma x1) ^ A, lo(Ma x1)); rounds 2 .. 9 follow as usual.
struct PhiloxFixed {
    uint32_t M, N, A;
};

__device__ __forceinline__ PhiloxFixed philox_fixed(uint32_t x0, uint32_t w0, const RoundKeys& rk) {
    const uint32_t z1 = __umulhi(kPhiloxMa, x0) ^ w0 ^ rk.k[1];
    return {__umulhi(kPhiloxMb, z1) ^ rk.k[2], kPhiloxMb * z1, (kPhiloxMa * x0) ^ rk.k[3]};
}

// Round 0 and the products of round 1 that depend on the varying words only.
struct PhiloxVarying {
    uint32_t y1, hx1, lx1;
};

__device__ __forceinline__ PhiloxVarying philox_varying(uint32_t y0, uint32_t z0, const RoundKeys& rk) {
    const uint32_t x1 = __umulhi(kPhiloxMb, z0) ^ y0 ^ rk.k[0];
    return {kPhiloxMb * z0, __umulhi(kPhiloxMa, x1), kPhiloxMa * x1};
}

__device__ __forceinline__ uint4 philox10_split(uint32_t M, uint32_t N, uint32_t A, const PhiloxVarying& v,
                                                const RoundKeys& rk) {
    return philox_rounds<2>(make_uint4(M ^ v.y1, N, v.hx1 ^ A, v.lx1), rk);
}

inline void make_round_keys(uint32_t k0, uint32_t k1, RoundKeys* rk) {
    for (int i = 0; i < 10; ++i) {
        rk->k[2 * i] = k0;
        rk->k[2 * i + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// ---------------------------------------------------------------------------
// Geometry of the unrotated planar code on the (2L-1)x(2L-1) grid.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int n_qubits(int L) { return 2 * L * L - 2 * L + 1; }
__host__ __device__ __forceinline__ int n_stabs(int L) { return 2 * L * (L - 1); }
__host__ __device__ __forceinline__ int n_words(int L) { return (n_qubits(L) + 31) / 32; }

// Grid point of the m-th generator of colour col.  Colours 0/1 are the
// sigma_x generators ((L-1) x L cells at (2i+1, 2j)) with i+j even/odd,
// colours 2/3 the sigma_z generators (L x (L-1) cells at (2i, 2j+1)).  Within
// a colour the cells are taken row-major.  With an odd number of columns the
// row-major cell index g has the parity of i+j, so the colour's cells are
// g = 2m + parity; with an even number every row holds half of them.
__host__ __device__ __forceinline__ void colour_cell(int L, int col, int m, int* r, int* c) {
    const int par = col & 1;
    const int wdt = col < 2 ? L : L - 1;
    int i, j;
    if (wdt & 1) {
        const int g = 2 * m + par;
        i = g / wdt;
        j = g - i * wdt;
    } else {
        const int half = wdt / 2;
        i = m / half;
        j = 2 * (m - i * half) + ((i + par) & 1);
    }
    if (col < 2) { *r = 2 * i + 1; *c = 2 * j; }
    else { *r = 2 * i; *c = 2 * j + 1; }
}

// Support of the m-th generator of colour col: up, down, left, right
// neighbours of its grid point.  A neighbour outside the grid (boundary
// generators have weight 3) is replaced by a dummy slot: nq for sigma_x
// generators, nq+1 for sigma_z generators.  The dummy's "other" plane is
// all ones, so it never changes n.
__host__ __device__ __forceinline__ void colour_support(int L, int col, int m, int q[4]) {
    int r, c;
    colour_cell(L, col, m, &r, &c);
    const int n = 2 * L - 1, nq = n_qubits(L);
    const int dummy = col < 2 ? nq : nq + 1;
    const int base = r * n + c;  // odd
    q[0] = r > 0 ? (base - n) / 2 : dummy;
    q[1] = r < n - 1 ? (base + n) / 2 : dummy;
    q[2] = c > 0 ? (base - 1) / 2 : dummy;
    q[3] = c < n - 1 ? (base + 1) / 2 : dummy;
}

// ---------------------------------------------------------------------------
// Geometry of the toric code (16 classes): an L x L torus, L even, on the
// periodic 2L x 2L grid; 2L^2 qubits at r+c odd with index r L + (c div 2);
// stars (sigma_x generators) at (even r, even c), plaquettes (sigma_z) at
// (odd r, odd c), all of weight 4; syndrome layout stars row-major over
// (r/2, c/2), then plaquettes.  Colours 0/1: stars with (i+j) even/odd,
// 2/3: plaquettes; within a colour row-major (each row holds L/2).
// Logicals: X1 on row 1, X2 on column 1 (even rows), Z1 on column 0 (odd
// rows), Z2 on row 0; class code a1 + 2 a2 + 4 b1 + 8 b2 (a: x parity on
// Z1 / Z2's qubits, b: z parity on X1 / X2's qubits).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int t_qidx(int L, int r, int c) {
    const int m = 2 * L;
    r = ((r % m) + m) % m;
    c = ((c % m) + m) % m;
    return r * L + c / 2;
}

__host__ __device__ __forceinline__ void toric_support(int L, int r, int c, int q[4]) {
    q[0] = t_qidx(L, r - 1, c);
    q[1] = t_qidx(L, r + 1, c);
    q[2] = t_qidx(L, r, c - 1);
    q[3] = t_qidx(L, r, c + 1);
}

__host__ __device__ __forceinline__ void toric_colour_support(int L, int col, int m, int q[4]) {
    const int type = col >> 1, par = col & 1, half = L / 2;
    const int i = m / half, t = m - i * half;
    const int j = ((par + i) & 1) + 2 * t;
    toric_support(L, 2 * i + type, 2 * j + type, q);
}

// Generator g in the syndrome layout: support and type (0 star, 1 plaquette).
__host__ __device__ __forceinline__ int toric_generator_support(int L, int g, int q[4]) {
    const int type = g >= L * L ? 1 : 0;
    const int h = g - type * L * L, i = h / L, j = h - i * L;
    toric_support(L, 2 * i + type, 2 * j + type, q);
    return type;
}

// Code-dependent counts: code 0 planar, 1 toric.
__host__ __device__ __forceinline__ int geo_nq(int code, int L) { return code ? 2 * L * L : n_qubits(L); }
__host__ __device__ __forceinline__ int geo_nstab(int code, int L) { return code ? 2 * L * L : n_stabs(L); }
__host__ __device__ __forceinline__ int geo_words(int code, int L) { return (geo_nq(code, L) + 31) / 32; }
__host__ __device__ __forceinline__ int geo_nc(int code, int L) { return code ? L * L / 2 : L * (L - 1) / 2; }

// Shared-memory words of one bundle split over `lam` lanes: X then Z, each
// of the qubits padded with zero words to a multiple of 4 lam (so that the
// lanes' occupancy counts, in batches of 8 or 4 words per lane, need no
// bounds test) and followed by two dummy slots.  The stride is odd so that the bundles of a warp fall on banks of
// opposite parity: same-colour generators in a row are two qubits apart.
__host__ __device__ __forceinline__ int padded_nq(int nq, int lam) { return (nq + 4 * lam - 1) / (4 * lam) * (4 * lam); }
__host__ __device__ __forceinline__ int bundle_stride(int nq, int lam) { return 2 * (padded_nq(nq, lam) + 2) + 1; }

// Blocks per SM the sweep kernel is compiled for (its register bound): 5
// with plane widths of 32 chains (96 registers, no spills: 0.8 % faster at
// L = 13 than 6 blocks at 80 registers), 6 with 16 (6 blocks measured 3.7 %
// faster than 5 there), 3 with narrower planes.
__host__ __device__ constexpr int sweep_blocks_per_sm(int G) { return G == 32 ? 5 : G == 16 ? 6 : 3; }

// ---------------------------------------------------------------------------
// Sweep kernel parameters.  One launch runs the chains of up to kMaxGroups
// groups of syndromes; a group has one code size and one sweep range.  Items
// (syndromes) are numbered globally across the groups; per-item arrays with a
// size-dependent row (pure errors, frames, bundle state) are laid out group
// after group at the given word offsets.
// ---------------------------------------------------------------------------
constexpr int kMaxGroups = 8;

struct GroupDesc {
    int L, nq, W, nc;            // size, qubits, words per plane, generators per colour
    long long n;                 // syndromes of the group
    long long n_bundles;         // 32-chain bundles of the group
    long long item_base;         // global index of the group's first syndrome
    long long e0_off;            // word offset of its pure errors ([n][2][W])
    long long frames_off;        // word offset of its per-chain frames ([n][C][2][W])
    long long state_off;         // word offset of its bundle state ([n_bundles][2][nq])
    long long unit_base;         // first work unit of the group
    uint32_t t_begin, t_end, burn_in;  // sweeps of this launch; sampling from burn_in on
};

struct SweepParams {
    int C, R, G;               // chains per syndrome, per class, plane width
    int bps, spb;              // bundles per syndrome (G == 32), syndromes per bundle (G < 32)
    uint32_t id0;
    const uint32_t* ids;       // per-syndrome ids (NULL: id0 + global index)
    int code;                  // 0: planar code (4 classes); 1: toric code (16 classes)
    int scan;                  // 0: colour sweeps; 1: random scan (one random generator per step)
    int noise;                 // 0: depolarizing; 1: independent bit and phase flips
    uint64_t T[33];            // acceptance thresholds T[d] = floor(r*^d 2^32), d <= 32 (random scan)
    int energy[4];             // energy of a qubit's Pauli, index x + 2z (I, X, Z, Y) (random scan)
    int accept_all;            // r* == 1: every proposal accepted
    int reject_all;            // T[1] == 0: no uphill proposal accepted
    uint32_t qmodes;           // per quad of planes 4q..4q+3, 2 bits: 0 every threshold digit is 0,
                               // 1 only T[1] has nonzero digits, 2 general
    RoundKeys rk;
    // Threshold bits of plane k as the algebraic normal form of the map
    // d-1 = e0 + 2 e1 -> bit (31-k) of T[d]: f = c0 ^ e0 c1 ^ e1 c2 ^ e0 e1 c3.
    uint32_t pc[4][32];
    const uint32_t* e0;        // pure errors
    const int32_t* e0code;     // [items]
    const uint32_t* init_frames;  // per-chain start frames, or NULL
    const uint32_t* state_in;     // bit-sliced state from an earlier launch, or NULL
    uint32_t* state_out;          // state at t_end for a later launch, or NULL
    const uint64_t* init_sum;     // [items][C] or NULL
    uint64_t* chain_sum;       // [items][C] out, or NULL
    int32_t* chain_n;          // [items][C] out or NULL
    uint32_t* chain_frames;    // per-chain final frames or NULL
    uint64_t* accepts;         // [items][C] accepted proposals, added to by every launch, or NULL
    int n_groups;
    int grp_nq_max, grp_nc_max;   // largest group (shared-memory layout)
    long long total_units;
    unsigned int* unit_counter;   // work queue of the persistent blocks (reset by the launcher)
    int max_blocks_per_sm;        // persistent blocks per multiprocessor, at most (0: as many as fit)
    GroupDesc grp[kMaxGroups];
};

struct DecideParams {
    long long n;
    int K, R;
    uint64_t samples;          // 4 R (n_sweeps - burn_in)
    const uint64_t* samples_per_item;  // per internal item, or NULL (then samples)
    const long long* perm;     // caller's index of internal item i, or NULL (identity)
    double beta_bar;
    const uint64_t* chain_sum; // [n][K R]
    int32_t* out_class;        // [n]
    uint64_t* out_class_sum;   // [n][K] or NULL
    double* out_log_ratio;     // [n][K] or NULL
};

// Launchers (return cudaGetLastError() after the launch).
cudaError_t launch_sweep(const SweepParams& p, int lanes_per_bundle, cudaStream_t s);
cudaError_t launch_sweep_flips(const SweepParams& p, int lanes_per_bundle, cudaStream_t s);
// The launch on a kernel with its digit-plane modes compiled in;
// cudaErrorNotSupported (nothing launched) where there is none.
cudaError_t launch_sweep_modes(const SweepParams& p, int lanes_per_bundle, cudaStream_t s);
cudaError_t prepare_sweep_flips(const SweepParams& p, int lanes_per_bundle);
cudaError_t prepare_sweep(const SweepParams& p, int lanes_per_bundle);
size_t sweep_smem_bytes(int nq, int nc, int lanes_per_bundle);  // dynamic shared memory of a block
long long sweep_units(long long n_bundles, int lanes_per_bundle);  // work units of a group
cudaError_t launch_gen_syndromes(uint64_t seed, uint32_t id0, long long n, int L, double p,
                                 uint8_t* syn, int32_t* true_class, cudaStream_t s, int noise = 0);
cudaError_t launch_gen_syndromes_pauli(uint64_t seed, uint32_t id0, long long n, int L, double px, double py,
                                       double pz, uint8_t* syn, int32_t* true_class, cudaStream_t s);
cudaError_t launch_start_frames(const uint8_t* syn, long long n, int L, uint32_t* frames, int32_t* code,
                                cudaStream_t s, int toric = 0);
cudaError_t launch_gen_syndromes_toric(uint64_t seed, uint32_t id0, long long n, int L, double p, uint8_t* syn,
                                       int32_t* true_class, cudaStream_t s);
cudaError_t launch_decide(const DecideParams& p, cudaStream_t s);
cudaError_t launch_gather_rows(long long n, const uint8_t* src, const long long* src_off, const long long* dst_off,
                               const int32_t* len, const long long* perm, const uint32_t* ids, uint32_t id0,
                               uint8_t* dst, uint32_t* ids_out, cudaStream_t s);
cudaError_t launch_class_means(long long n, int K, int R, int N, int j, uint64_t samples, const uint64_t* chain_sum,
                               double* mean, cudaStream_t s);
cudaError_t launch_ti_decide(long long n, int K, int N, double mean0, double h3, double* mean, int32_t* out_class,
                             double* out_log_z, cudaStream_t s);

cudaError_t launch_retire(long long n, const long long* perm, const float* logprob, const int32_t* cls,
                          const uint64_t* class_sum, float tau, uint32_t sweeps, int final_chunk, int32_t* out_class,
                          uint64_t* out_class_sum, uint32_t* out_sweeps, int32_t* keep, cudaStream_t s);
cudaError_t launch_compact(long long n, const int32_t* keep, long long* pos, long long* count, const long long* perm,
                           uint32_t id0, int frame_words, int chains, const uint32_t* frames, const uint64_t* sums,
                           long long* perm_out, uint32_t* ids_out, uint32_t* frames_out, uint64_t* sums_out,
                           cudaStream_t s);
cudaError_t launch_reorder(long long n, const long long* perm, const float* logprob, int R, int chain_words,
                           uint32_t* frames, uint64_t* sums, uint8_t* rank, uint64_t* frozen, cudaStream_t s);
cudaError_t launch_decide_reorder(long long n, const long long* perm, const uint8_t* rank, const uint64_t* frozen,
                                  int R, const uint64_t* chain_sum, uint64_t n_top, uint64_t n_low, int32_t* out_class,
                                  uint64_t* out_class_sum, cudaStream_t s);
cudaError_t launch_iota(long long n, long long* perm, cudaStream_t s);

// Context services shared with the network code (api.cu).
void ctx_set_error(surfmcmc_ctx* ctx, const char* msg);
int ctx_device(const surfmcmc_ctx* ctx);
bool device_ptr(const void* p);

// Network log-probabilities [n][4] of n device syndromes into device memory,
// stream-ordered, batched by the network's max_batch (cnn.cu).
cudaError_t cnn_logprob(surfmcmc_cnn* net, const uint8_t* syn, long long n, float* logprob, cudaStream_t s);
int cnn_code_size(const surfmcmc_cnn* net);

}  // namespace surfmcmc
