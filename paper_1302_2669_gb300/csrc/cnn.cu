// The early-stop network on the GPU: five 3x3 convolutions over the two
// syndrome maps of a size-L code (2 -> 64 -> 64 -> 64 -> 64 -> 2, ReLU after
// the first four) and a parity readout giving the log-probabilities of the 4
// classes; training by the cross entropy with soft targets and Adam.
//
// Readout: class bit a (b) is the parity of an error's sigma_x (sigma_z)
// part on qubit column (row) 0.  With e0 the decoder's pure error of class
// code c0 = a0 + 2 b0, E + e0 has a trivial syndrome, so its parities are
// the same on the middle qubit column / row 2m, m = (L-1) div 2.  The last
// layer gives at map position (i, m) (channel 0) and (m, j) (channel 1) the
// logit s of a flip of (E + e0) on qubit (2i, 2m) / (2m, 2j); with
// independent flips P(odd) = (1 - M)/2, M = prod(-tanh(s/2)) clipped to
// +-(1 - 1e-6), and log p_{a + 2b} = log P_x(a xor a0) + log P_z(b xor b0).
//
// Layouts: activations are NHWC bfloat16, [M][C] with M = n P^2 positions of
// the maps zero-padded to P = L + 2 (syndrome-major, then row, then column):
// every 3x3 tap is then a shift of the position index by dy P + dx, and the
// epilogues keep the one-position border at zero.  Weights live as float32 master
// copies in the flat order W[co][kh][kw][ci] then b[co], layer after layer;
// every step packs them into bfloat16 GEMM operands.
//
// Tensor-core work (tcgen05, BF16 in, FP32 accumulate in tensor memory):
//   forward conv and input-gradient conv (64 input channels): an implicit
//     GEMM, M = positions in tiles of 128, N = output channels, K = 9 x 64.
//     One TMA tiled copy (128-byte swizzle) per tile brings the tile's rows
//     with a halo of P + 1 rows on each side; the operand of tap t is the
//     128 rows starting at row P + 1 + shift(t) of that halo tile, so each
//     input row crosses from L2 once per tile instead of once per tap.  The
//     weight operand stays in shared memory for the whole persistent block;
//     two threads issue the MMAs (alternate tiles), four warps drain the
//     four tensor-memory accumulators (bias + ReLU, or the ReLU gate of the
//     layer below) and store each tile with a TMA copy.  The 64-channel
//     conv is bound by shared-memory bandwidth: an N = 64 MMA reads 6 KB of
//     operands.  The first layer (2 input channels, K = 18 padded to 32)
//     builds its operand from a TMA-loaded strip of input positions, adds
//     the bias through constant-one operand columns and drains alternate
//     tiles with two groups of warps;
//   weight gradient of the 64-channel layers: D[(tap, ci)][co] =
//     sum_p X[p + tap][ci] dZ[p][co], a GEMM over positions whose operands
//     are read MN-major by TMA straight from the [position][channel]
//     tensors (tap windows are row offsets of a halo tile, two taps make
//     M = 128, a constant ones tile gives the bias row); one block per SM
//     over a contiguous range of positions, partial sums added in a fixed
//     order.  The first layer's (2 input channels, 19 rows) is the same
//     GEMM with its operand rows built from an input strip, M padded to
//     128 by the dZ tile.
// The last layer (2 outputs, read and differentiated on the middle lines
// only: forward fused into the readout, backward), the readout, loss and
// Adam steps run on the CUDA cores.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "surfmcmc.h"
#include "common.cuh"

namespace surfmcmc {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kHid = 64;          // hidden channels
constexpr int kOut = 2;           // flip logits per position (last layer)
constexpr float kClip = 1e-6f;    // |M| <= 1 - kClip
constexpr int kEpiWarps = 4;      // accumulator-draining warps
constexpr int kOutTile = 128 * 128;   // one 128 x 64 bf16 output tile
constexpr int kConvAcc = 4;       // tensor-memory accumulators of the conv kernels
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kWaitTimeout = 1;   // error codes written to the device flag
constexpr int kMaxSplits = 64;    // position slices of the weight-gradient GEMM
constexpr int kTmaStages = 4;     // halo tiles in flight in the TMA conv kernel
constexpr int kTmaThreads = 7 * 32;  // TMA warp, MMA warps 1 and 6, 4 accumulator warps

// Channels of the five layers and the offsets of their weights and biases in
// the flat parameter vector.
__host__ __device__ constexpr int layer_cin(int l) { return l == 0 ? 2 : kHid; }
__host__ __device__ constexpr int layer_cout(int l) { return l == 4 ? kOut : kHid; }
__host__ __device__ constexpr long long layer_woff(int l) {
    long long o = 0;
    for (int i = 0; i < l; ++i) o += (long long)layer_cout(i) * 9 * layer_cin(i) + layer_cout(i);
    return o;
}
__host__ __device__ constexpr long long layer_boff(int l) {
    return layer_woff(l) + (long long)layer_cout(l) * 9 * layer_cin(l);
}
constexpr long long kParams = layer_woff(5);
static_assert(kParams == 113154, "parameter count");

// GEMM operand shapes of the forward conv of each layer: N rows (output
// channels, padded to a multiple of 16) by K columns (9 C_in, padded to a
// multiple of 16).
__host__ __device__ constexpr int fwd_np(int l) { return l == 4 ? 16 : kHid; }
__host__ __device__ constexpr int fwd_kp(int l) { return l == 0 ? 32 : 9 * kHid; }

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle, K-major: core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between groups of 8 rows.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B, f32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element group (row r, 16-byte group g) in a K-major
// no-swizzle tile whose rows hold kg groups.
__device__ __forceinline__ uint32_t core_off(int r, int g, int kg) {
    return (uint32_t)(((r >> 3) * kg + g) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Non-blocking test of the same (mbarrier.test_wait never suspends the thread).
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the completion of the phase of the given parity.  Gives up
// when another role of the block has given up, or after `limit` polls (the
// kernel's spin_limit, kSpinLimit unless set smaller to exercise this path;
// then it records the time-out in the device error flag and raises the
// block's abort flag so that every other wait of the block returns too).
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, uint32_t limit) {
    // the first poll does not suspend, so that a bound of one poll gives up
    // whenever the phase is not complete yet
    for (uint32_t it = 0; it < limit; ++it) {
        if (it == 0 ? mbar_test(bar, parity) : mbar_try(bar, parity)) return true;
        if ((it & 31) == 31 && *abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(err, kWaitTimeout);
    return false;
}

// Bounded wait used before tensor memory is released: ignores the abort flag,
// so that MMAs still in flight complete first.
__device__ void mbar_drain(uint64_t* bar, uint32_t parity, int* err) {
    for (uint32_t it = 0; it < kSpinLimit; ++it)
        if (mbar_try(bar, parity)) return;
    atomicExch(err, kWaitTimeout);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// The same with each descriptor given as its 32-bit halves (the low half
// holds the start address field, so moving an operand inside shared memory
// is one 32-bit add).
__device__ __forceinline__ void mma_bf16_lh(uint32_t d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                            uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\tmov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
        "setp.ne.b32 p, %6, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}" ::"r"(d),
        "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrives on the barrier once every tcgen05 operation issued so far by this
// thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Shared-memory descriptor of a K-major tile written by TMA with the 128-byte
// swizzle: rows of 128 bytes (64 bf16 of K), atoms of 8 rows (1024 bytes, the
// stride between 8-row groups); the K step of an MMA (16 elements) advances
// the start address by 32 bytes inside the atom.  The tile must start on a
// 1024-byte boundary.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // leading offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// The transaction count the barrier's current phase waits for, then this
// thread's arrival.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// TMA tiled load of box (c0, c1) of a 2-D tensor map into shared memory,
// completing on the barrier (rows outside the tensor read as zero).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// TMA tiled store of box (c0, c1) of a 2-D tensor map from shared memory
// (rows outside the tensor are not written), in this thread's bulk group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int c0, int c1) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until at most N of this thread's bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Named barrier id (1 by default) over 128 accumulator-draining threads;
// the second form returns whether the predicate held in all of them.
__device__ __forceinline__ void epi_sync(uint32_t id = 1) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
__device__ __forceinline__ bool epi_all(bool v, uint32_t id = 1) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id)
                 : "memory");
    return r != 0;
}

// Padded maps: P = L + 2; interior positions are the L x L map, the rest is
// the zero border.  Whether position rem = m mod P^2 inside its map is
// interior:
__device__ __forceinline__ bool interior_rem(int rem, int L) {
    const int P = L + 2, y = rem / P, x = rem - y * P;
    return y >= 1 && y <= L && x >= 1 && x <= L;
}

// Position shift of tap t = 3 kh + kw: (kh - 1) P + (kw - 1).
__device__ __forceinline__ int tap_shift(int t, int L) { return (t / 3 - 1) * (L + 2) + (t % 3 - 1); }

// 64 consecutive f32 columns of this warp's 32 tensor-memory lanes, one
// load and one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float v[64]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive f32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half)
    return *reinterpret_cast<const uint32_t*>(&h);
}

// The same after max(x, 0), in one conversion (round to nearest even).
__device__ __forceinline__ uint32_t pack_bf16_relu(float a, float b) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));   // b: high half
    return d;
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// ---------------------------------------------------------------------------
// Implicit-GEMM 3x3 conv of the first layer on tcgen05.
// ---------------------------------------------------------------------------
struct Conv1Args {
    CUtensorMap in_map;   // input [M][2] bf16 viewed as [ceil(M/4)][8], box 8 x c1_strip_rows(L), no swizzle
    CUtensorMap out_map;  // output [M_alloc][64] bf16, box 64 x 128, 128-byte swizzle
    const bf16* wmat;     // [64][32] operand B (k = tap * 2 + ci; k = 18..20: the bias in three parts)
    long long M;          // positions n P^2
    int L;
    int* err;
    uint32_t spin_limit;   // polls before a pipeline wait gives up
};

constexpr int kC1KP = 32;                       // K of the first layer: 9 taps x 2 channels, padded
constexpr int kC1Stage = 128 * kC1KP * 2;       // one tile's A operand
constexpr int kC1S = 4;                         // pipeline depth
constexpr int kC1StripStage = 1024;             // one tile's input strip
constexpr int kC1Threads = 14 * 32;             // TMA warp, MMA warp, 2 x 4 accumulator warps, 4 operand warps

// 16-byte rows (4 positions) of the input strip of a 128-position tile: the
// taps reach P + 1 = L + 3 positions either way and the strip starts up to 3
// positions before the first one it needs (row-aligned).
__host__ __device__ constexpr int c1_strip_rows(int L) { return (128 + 2 * (L + 3) + 3 + 3) / 4; }
static_assert(c1_strip_rows(SURFMCMC_MAX_L) * 16 <= kC1StripStage, "input strip");
constexpr size_t kC1Smem = 4 * (size_t)kOutTile + kC1S * kC1Stage + 64 * kC1KP * 2 + kC1S * kC1StripStage + 1024;

// floor(v / 4) for any sign
__device__ __forceinline__ long long floor_div4(long long v) { return v >= 0 ? v / 4 : -((-v + 3) / 4); }

// First layer (2 input channels, K = 18 padded to 32).  Warp 0 (one thread)
// loads by TMA the strip of input positions a tile's taps read (4 B per
// position); warps 10-13 build the tile's operand rows from it in shared
// memory (row r, group g = taps 4g .. 4g+3, then three constant-one columns
// k = 18..20 that multiply the bias's three bf16 parts in the weight operand;
// rows of border positions are all zero, so their outputs are zero; group 3
// stays zero); warp 1 (one thread) issues the two K = 16 MMAs into one of
// four accumulators; two groups of four warps (2-5 and 6-9) drain alternate
// tiles (ReLU and rounding in one conversion) into 128-byte-swizzled staging
// buffers that one thread of the group stores with a TMA copy.  With K this
// small the MMAs are short and the drain is the longest step of a tile, so
// two tiles drain at once.
__global__ void __launch_bounds__(kC1Threads, 1) conv1_kernel(const __grid_constant__ Conv1Args a) {
    constexpr int S = kC1S, KGS = kC1KP / 8, NP = 64, NACC = kConvAcc;
    constexpr uint32_t NCOLS = NACC * NP;
    constexpr uint32_t IDESC = idesc_bf16(128, NP);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sOut = smem;                         // 2 output tiles per drain group, 1024-byte aligned
    uint8_t* sA = sOut + 4 * kOutTile;            // S operand tiles
    uint8_t* sB = sA + S * kC1Stage;              // weights
    uint8_t* sStrip = sB + NP * kC1KP * 2;        // S input strips, 1024-byte aligned
    __shared__ __align__(8) uint64_t full[S], sfree[S], afull[S], aempty[S], accf[NACC], acce[NACC], fin;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = a.M;
    const int L = a.L, P1 = L + 3;
    const long long n_tiles = (M + 127) / 128;

    for (int idx = tid; idx < NP * KGS; idx += kC1Threads) {
        const int r = idx / KGS, g = idx - r * KGS;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.wmat + (size_t)r * kC1KP) + g);
        *reinterpret_cast<uint4*>(sB + core_off(r, g, KGS)) = v;
    }
    // operand group 3 (k = 24 .. 31) is never written again
    for (int idx = tid; idx < S * kC1Stage / 16; idx += kC1Threads)
        reinterpret_cast<uint4*>(sA)[idx] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&sfree[s], 128);
            mbar_init(&afull[s], 128);
            mbar_init(&aempty[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kEpiWarps * 32);
        }
        mbar_init(&fin, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    if (warp == 1) tmem_alloc(&tmem_slot, NCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)c1_strip_rows(L) * 16;
            uint32_t q = 0;
            for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++q) {
                const uint32_t stage = q % S, use = q / S;
                if (use > 0 && !mbar_wait(&sfree[stage], (use - 1) & 1, &abort_flag, a.err, a.spin_limit)) break;
                mbar_expect_tx(&full[stage], bytes);
                tma_load_2d(sStrip + stage * kC1StripStage, &a.in_map, 0, (int)floor_div4(tile * 128 - P1),
                            &full[stage]);
            }
            for (uint32_t k = q > (uint32_t)S ? q - S : 0; k < q; ++k) mbar_drain(&full[k % S], (k / S) & 1, a.err);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0;
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
                const uint32_t b = it % NACC, u = it / NACC;
                const uint32_t stage = it % S, use = it / S;
                if (u > 0 && !mbar_wait(&acce[b], (u - 1) & 1, &abort_flag, a.err, a.spin_limit)) break;
                if (!mbar_wait(&afull[stage], use & 1, &abort_flag, a.err, a.spin_limit)) break;
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < kC1KP / 16; ++ks) {
                    const uint64_t ad = smem_desc(a0 + stage * kC1Stage + ks * 256, 128, KGS * 128);
                    const uint64_t bd = smem_desc(b0 + ks * 256, 128, KGS * 128);
                    mma_bf16(tmem + b * NP, ad, bd, IDESC, ks > 0 ? 1u : 0u);
                }
                mma_commit(&aempty[stage]);
                mma_commit(&accf[b]);
            }
            mma_commit(&fin);
            mbar_drain(&fin, 0, a.err);
        }
    } else if (warp >= 10) {
        // operand rows: thread r builds row r of every tile
        const int r = 32 * (warp - 10) + lane;
        const int PP = (L + 2) * (L + 2);
        int sh[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) sh[t] = tap_shift(t, L);
        uint32_t q = 0;
        for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++q) {
            const uint32_t stage = q % S, use = q / S;
            if (!mbar_wait(&full[stage], use & 1, &abort_flag, a.err, a.spin_limit)) break;
            const long long s0 = tile * 128 - P1;
            const int base = r + P1 + (int)(s0 - 4 * floor_div4(s0));   // strip index of position tile*128 + r
            const uint32_t* strip = reinterpret_cast<const uint32_t*>(sStrip + stage * kC1StripStage);
            const int rem = (int)((tile * 128) % PP + r) % PP;
            const bool keep = tile * 128 + r < M && interior_rem(rem, L);
            uint32_t w[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) w[t] = keep ? strip[base + sh[t]] : 0u;
            const uint32_t one2 = keep ? 0x3F803F80u : 0u;   // bf16 1.0 at k = 18, 19 (and k = 20)
            mbar_arrive(&sfree[stage]);
            if (use > 0 && !mbar_wait(&aempty[stage], (use - 1) & 1, &abort_flag, a.err, a.spin_limit)) break;
            uint8_t* st = sA + stage * kC1Stage;
            *reinterpret_cast<uint4*>(st + core_off(r, 0, KGS)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(st + core_off(r, 1, KGS)) = make_uint4(w[4], w[5], w[6], w[7]);
            *reinterpret_cast<uint4*>(st + core_off(r, 2, KGS)) = make_uint4(w[8], one2, one2 & 0xFFFFu, 0u);
            fence_async_smem();
            mbar_arrive(&afull[stage]);
        }
    } else {
        // drain group grp takes tiles it = grp, grp + 2, ... (accumulators
        // grp, grp + 2), its own named barrier and staging buffers
        const uint32_t grp = warp < 6 ? 0u : 1u, bar_id = 1 + grp;
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        const bool elected = (warp == 2 || warp == 6) && lane == 0;
        uint32_t it = grp, k = 0;
        for (long long tile = blockIdx.x + (long long)grp * gridDim.x; tile < n_tiles;
             tile += 2LL * gridDim.x, it += 2, ++k) {
            const uint32_t b = it % NACC, u = it / NACC;
            uint8_t* out = sOut + (2 * grp + (k & 1)) * kOutTile;
            if (elected) bulk_wait_read<1>();   // the group's store of two tiles back has left this buffer
            const bool ok = mbar_wait(&accf[b], u & 1, &abort_flag, a.err, a.spin_limit);
            if (!epi_all(ok, bar_id)) break;
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + b * NP;
            float v[NP];
            tmem_ld64(taddr, v);
            tc_fence_before();
            mbar_arrive(&acce[b]);
            uint8_t* orow = out + row * 128;
            const int sw = row & 7;
#pragma unroll
            for (int j = 0; j < NP / 8; ++j) {
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) w[h] = pack_bf16_relu(v[8 * j + 2 * h], v[8 * j + 2 * h + 1]);
                *reinterpret_cast<uint4*>(orow + ((j ^ sw) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
            fence_async_smem();
            epi_sync(bar_id);
            if (elected) {
                tma_store_2d(&a.out_map, out, 0, (int)(tile * 128));
                bulk_commit();
            }
        }
        if (elected) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, NCOLS);
}

// ---------------------------------------------------------------------------
// Convolutions with 64 input channels: tap operands by TMA.
// ---------------------------------------------------------------------------
enum Epi { kEpiRelu = 0, kEpiMask = 1 };

struct ConvTmaArgs {
    CUtensorMap map;     // input [M_alloc][64] bf16, box 64 x halo_rows, 128-byte swizzle
    CUtensorMap out_map;   // output [M_alloc][64] bf16, box 64 x 128 (kEpiRelu, kEpiMask)
    CUtensorMap mask_map;  // ReLU gate [M_alloc][64] bf16, box 64 x 128 (kEpiMask)
    const bf16* wmat;    // [NP][576] operand B (k = tap * 64 + ci)
    const float* bias;   // [NP] (kEpiRelu) or NULL
    long long M;         // positions n P^2
    int L;
    int halo_rows;       // rows of one halo tile, halo_tile_rows(L)
    int* err;
    uint32_t spin_limit;   // polls before a pipeline wait gives up
};

// Rows of the halo tile of 128 output positions: the taps shift by up to
// P + 1 = L + 3 rows either way; rounded up to whole 8-row swizzle atoms so
// that every stage starts on a 1024-byte boundary.  At most 200 (L = 31),
// inside the 256-row limit of a TMA box.
__host__ __device__ constexpr int halo_tile_rows(int L) { return (128 + 2 * (L + 3) + 7) / 8 * 8; }
constexpr int kHaloRowsMax = halo_tile_rows(SURFMCMC_MAX_L);
constexpr int kTmaStage = kHaloRowsMax * 128;   // stage stride in bytes
static_assert(kHaloRowsMax <= 256 && kTmaStage % 1024 == 0, "halo tile");


// Staging buffers of the epilogue: two output tiles, or three for the
// ReLU-gate epilogue, whose gate tile is loaded two tiles ahead into the
// buffer that then receives the output in place.
__host__ __device__ constexpr int conv_out_bufs(int epi) { return epi == kEpiMask ? 3 : 2; }

template <int NP, int EPI>
constexpr size_t conv_tma_smem_bytes() {
    return (size_t)kTmaStages * kTmaStage + (size_t)NP * 576 * 2 + conv_out_bufs(EPI) * kOutTile + 1024;
}

// Warp 0 (one thread) loads the halo tile of each position tile by TMA into
// a ring of stages; warps 1 and 6 (one thread each) issue 4 MMAs per tap
// (K = 16 each), 36 per tile, into one of four accumulators, taking the
// block's tiles alternately (one thread cannot issue 128 x 64 x 16 MMAs as
// fast as the tensor pipe runs them; every accumulator still gets its MMAs
// from one thread in order); warps 2-5 drain the accumulators.  A tap's operand starts at a 128-byte row inside the
// 1024-byte-aligned halo tile: the 128-byte swizzle is a function of the
// shared-memory address bits, so the descriptor keeps a zero base offset.
// The bf16 epilogues write their tile into one of two output buffers in the
// 128-byte-swizzled layout (16-byte chunk j of row r at chunk j ^ (r & 7)),
// which one thread then stores with a single TMA copy; the ReLU gate of the
// backward pass arrives by TMA in the buffer of its tile two tiles ahead
// (three buffers) and the gated output overwrites it in place.
template <int NP, int EPI>
__global__ void __launch_bounds__(kTmaThreads, 1) conv_tma_kernel(const __grid_constant__ ConvTmaArgs a) {
    constexpr int S = kTmaStages, KG = 576 / 8, NACC = kConvAcc;
    constexpr uint32_t NCOLS = NACC * NP < 32 ? 32 : NACC * NP;
    constexpr uint32_t IDESC = idesc_bf16(128, NP);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                      // S halo tiles, 1024-byte aligned
    uint8_t* sB = smem + S * kTmaStage;
    uint8_t* sOut = sB + NP * 576 * 2;       // output tiles (bf16 epilogues), 1024-byte aligned
    constexpr int NOB = conv_out_bufs(EPI);
    __shared__ __align__(8) uint64_t full[S], empty[S], accf[NACC], acce[NACC], maskf[3], fin[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    static_assert(NACC % 2 == 0 && S % 2 == 0, "alternating issuers need even rings");
    static_assert(NP == 64, "the epilogue drains 64 accumulator columns");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = a.M;
    const int L = a.L, P1 = L + 3;
    const long long n_tiles = (M + 127) / 128;

    for (int idx = tid; idx < NP * KG; idx += kTmaThreads) {
        const int r = idx / KG, g = idx - r * KG;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.wmat + (size_t)r * 576) + g);
        *reinterpret_cast<uint4*>(sB + core_off(r, g, KG)) = v;
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kEpiWarps * 32);
        }
        for (int k = 0; k < 3; ++k) mbar_init(&maskf[k], 1);
        mbar_init(&fin[0], 1);
        mbar_init(&fin[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    if (warp == 1) tmem_alloc(&tmem_slot, NCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)a.halo_rows * 128;
            uint32_t q = 0;
            for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++q) {
                const uint32_t stage = q % S, use = q / S;
                if (use > 0 && !mbar_wait(&empty[stage], (use - 1) & 1, &abort_flag, a.err, a.spin_limit)) break;
                mbar_expect_tx(&full[stage], bytes);
                tma_load_2d(sA + stage * kTmaStage, &a.map, 0, (int)(tile * 128 - P1), &full[stage]);
            }
            // the last S loads have landed before the block can exit (they
            // are unconsumed only after an abort)
            for (uint32_t k = q > (uint32_t)S ? q - S : 0; k < q; ++k) mbar_drain(&full[k % S], (k / S) & 1, a.err);
        }
    } else if (warp == 1 || warp == 6) {
        if (lane == 0) {
            const uint32_t who = warp == 1 ? 0u : 1u;   // tiles it = who, who + 2, ...
            uint32_t it = who;
            // descriptors as 32-bit halves: the high halves are fixed, the
            // low halves are the start address / 16 plus the operand's offset
            const uint64_t a_desc = smem_desc_sw128(smem_u32(sA) + P1 * 128);
            const uint64_t b_desc = smem_desc(smem_u32(sB), 128, KG * 128);
            const uint32_t a_hi = (uint32_t)(a_desc >> 32), b_hi = (uint32_t)(b_desc >> 32);
            const uint32_t a_lo0 = (uint32_t)a_desc, b_lo0 = (uint32_t)b_desc;
            uint32_t tap_lo[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) tap_lo[c] = (uint32_t)(tap_shift(c, L) * 8);   // 128 B rows / 16
            for (long long tile = blockIdx.x + (long long)who * gridDim.x; tile < n_tiles;
                 tile += 2LL * gridDim.x, it += 2) {
                const uint32_t b = it % NACC, u = it / NACC;
                const uint32_t stage = it % S, use = it / S;
                if (u > 0 && !mbar_wait(&acce[b], (u - 1) & 1, &abort_flag, a.err, a.spin_limit)) break;
                if (!mbar_wait(&full[stage], use & 1, &abort_flag, a.err, a.spin_limit)) break;
                tc_fence_after();
                const uint32_t d = tmem + b * NP;
                const uint32_t a_st = a_lo0 + stage * (kTmaStage / 16);
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    const uint32_t a_tap = a_st + tap_lo[c];
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        mma_bf16_lh(d, a_tap + ks * 2, a_hi, b_lo0 + (c * 8 + ks * 2) * 8, b_hi, IDESC,
                                    (c > 0 || ks > 0) ? 1u : 0u);
                }
                mma_commit(&empty[stage]);
                mma_commit(&accf[b]);
            }
            mma_commit(&fin[who]);
            mbar_drain(&fin[who], 0, a.err);
        }
    } else {
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        const bool elected = warp == 2 && lane == 0;
        const int PP = (L + 2) * (L + 2);
        float bias[EPI == kEpiRelu ? NP : 1];
#pragma unroll
        for (int j = 0; j < (EPI == kEpiRelu ? NP : 1); ++j) bias[j] = EPI == kEpiRelu ? __ldg(a.bias + j) : 0.0f;
        // the block's k-th tile is blockIdx.x + k gridDim.x; its gate tile
        // (ReLU-gate epilogue) goes to buffer k mod 3, two tiles ahead
        const uint32_t n_mine = (uint32_t)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1);
        uint32_t issued = 0, gated = 0;   // gate loads issued / seen complete (elected thread)
        auto issue_gate = [&](uint32_t k) {
            mbar_expect_tx(&maskf[k % NOB], kOutTile);
            tma_load_2d(sOut + (k % NOB) * kOutTile, &a.mask_map, 0,
                        (int)((blockIdx.x + (long long)k * gridDim.x) * 128), &maskf[k % NOB]);
        };
        if (EPI == kEpiMask && elected)
            for (; issued < 2 && issued < n_mine; ++issued) issue_gate(issued);
        uint32_t it = 0;
        for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
            const uint32_t b = it % NACC, u = it / NACC, ob = it % NOB;
            uint8_t* out = sOut + ob * kOutTile;
            if (EPI == kEpiRelu && elected) bulk_wait_read<1>();   // the store of two tiles back has left this buffer
            const bool ok = mbar_wait(&accf[b], u & 1, &abort_flag, a.err, a.spin_limit);
            if (!epi_all(ok)) break;
            tc_fence_after();
            const long long m = tile * 128 + row;
            const int rem = (int)((tile * 128) % PP + row) % PP;
            const bool keep = m < M && interior_rem(rem, L);
            const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + b * NP;
            float v[NP];
            tmem_ld64(taddr, v);
            tc_fence_before();
            mbar_arrive(&acce[b]);
            uint8_t* orow = out + row * 128;
            const int sw = row & 7;
            if (EPI == kEpiMask && mbar_wait(&maskf[ob], (it / NOB) & 1, &abort_flag, a.err, a.spin_limit) && elected) ++gated;
#pragma unroll
            for (int j = 0; j < NP / 8; ++j) {
                uint4* chunk = reinterpret_cast<uint4*>(orow + ((j ^ sw) << 4));
                uint32_t w[4];
                if (EPI == kEpiRelu) {
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int c = 8 * j + 2 * h;
                        w[h] = keep ? pack_bf16(fmaxf(v[c] + bias[c], 0.0f), fmaxf(v[c + 1] + bias[c + 1], 0.0f)) : 0u;
                    }
                } else {
                    const uint4 g = *chunk;
                    const uint32_t mw[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int c = 8 * j + 2 * h;
                        const float x0 = keep && bf16_lo(mw[h]) > 0.0f ? v[c] : 0.0f;
                        const float x1 = keep && bf16_hi(mw[h]) > 0.0f ? v[c + 1] : 0.0f;
                        w[h] = pack_bf16(x0, x1);
                    }
                }
                *chunk = make_uint4(w[0], w[1], w[2], w[3]);
            }
            fence_async_smem();
            epi_sync();
            if (elected) {
                tma_store_2d(&a.out_map, out, 0, (int)(tile * 128));
                bulk_commit();
                if (EPI == kEpiMask && issued < n_mine) {
                    bulk_wait_read<1>();   // the previous tile's store has left buffer (it + 2) mod 3
                    issue_gate(issued++);
                }
            }
        }
        if (elected) {
            // after an abort gate loads may still be in flight
            if (EPI == kEpiMask)
                for (uint32_t k = gated; k < issued; ++k) mbar_drain(&maskf[k % NOB], (k / NOB) & 1, a.err);
            bulk_wait_all();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, NCOLS);
}

// ---------------------------------------------------------------------------
// Weight gradient of the 64-channel layers on tcgen05: D[(tap, ci)][co] =
// sum_p X[p + shift(tap)][ci] dZ[p][co], and the bias gradient sum_p dZ[p][co].
// A GEMM with K = positions whose operands are taken MN-major straight from
// the [position][channel] tensors: per chunk of 64 positions one TMA copy
// brings X's rows with a halo of P + 1 on each side, another dZ's 64 rows
// (128-byte swizzle).  Tap t's operand is the 64 rows starting at halo row
// P + 1 + shift(t): for every position (K) its 64 channels (M) are one
// 128-byte row.  Two taps side by side along M make M = 128 (the step between
// the two 64-channel atoms is the descriptor's leading byte offset), so five
// MMA groups cover taps (0,1) .. (6,7), (8, ones); the ones atom is a constant
// tile whose channel 0 is 1.0, giving the bias gradient in row 576.  D of
// pair j is accumulated in tensor-memory columns 64 j .. 64 j + 63 over the
// block's chunks; row 128 j + r of the block's partial sums is R = 64 tap + ci.
// Each block takes a contiguous range of chunks; the partial sums are added
// over the blocks in order.
// ---------------------------------------------------------------------------
struct WgradArgs {
    CUtensorMap xmap;   // X [M_alloc][64] bf16, box 64 x wg_halo_rows(L), 128-byte swizzle
    CUtensorMap dzmap;  // dZ [M_alloc][64] bf16, box 64 x 64, 128-byte swizzle
    float* partial;     // [slices][640][64]
    long long M;
    int L;
    int halo_rows;
    int* err;
    uint32_t spin_limit;   // polls before a pipeline wait gives up
};

constexpr int kWgS = 4;                          // pipeline depth
__host__ __device__ constexpr int wg_halo_rows(int L) { return (64 + 2 * (L + 3) + 7) / 8 * 8; }
constexpr int kWgXStage = wg_halo_rows(SURFMCMC_MAX_L) * 128;   // 17 KB at L = 31
constexpr int kWgDStage = 64 * 128;
constexpr int kWgStage = kWgXStage + kWgDStage;
static_assert(kWgXStage % 1024 == 0 && wg_halo_rows(SURFMCMC_MAX_L) <= 256, "halo tile");
// stages + the ones tile; requested as 120 KB so that one block holds an SM
// (its 512 tensor-memory columns would stall a second block's allocation)
constexpr size_t kWgSmemNeed = (size_t)kWgS * kWgStage + kWgDStage + 1024;
constexpr size_t kWgSmem = 120 * 1024;
static_assert(kWgSmemNeed <= kWgSmem, "weight-gradient shared memory");
constexpr int kWgPairs = 5;
constexpr int kWgTmaThreads = 6 * 32;            // TMA warp, MMA warp, 4 accumulator warps
constexpr int kWgRows = 128 * kWgPairs;          // 640 rows of partial sums per block

__global__ void __launch_bounds__(kWgTmaThreads, 1) wgrad_kernel(const __grid_constant__ WgradArgs a) {
    constexpr uint32_t IDESC = idesc_bf16(128, 64) | (1u << 15) | (1u << 16);   // A, B MN-major
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sOnes = smem + kWgS * kWgStage;     // 64 rows: channel 0 = 1.0
    __shared__ __align__(8) uint64_t full[kWgS], empty[kWgS], accf;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = a.M;
    const int L = a.L, P1 = L + 3;
    const long long n_chunks = (M + 63) / 64;
    const long long c_begin = n_chunks * blockIdx.x / gridDim.x, c_end = n_chunks * (blockIdx.x + 1) / gridDim.x;

    for (int i = tid; i < kWgDStage / 16; i += blockDim.x) {
        // row r, 16-byte chunk c (stored at chunk c ^ (r & 7)): channel 0 is chunk 0
        const int r = i >> 3, c = i & 7;
        reinterpret_cast<uint4*>(sOnes)[i] = make_uint4((c ^ (r & 7)) == 0 ? 0x3F80u : 0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int s = 0; s < kWgS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accf, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    if (warp == 1) tmem_alloc(&tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)a.halo_rows * 128 + kWgDStage;
            uint32_t q = 0;
            for (long long ch = c_begin; ch < c_end; ++ch, ++q) {
                const uint32_t stage = q % kWgS, use = q / kWgS;
                if (use > 0 && !mbar_wait(&empty[stage], (use - 1) & 1, &abort_flag, a.err, a.spin_limit)) break;
                uint8_t* st = smem + stage * kWgStage;
                mbar_expect_tx(&full[stage], bytes);
                tma_load_2d(st, &a.xmap, 0, (int)(ch * 64 - P1), &full[stage]);
                tma_load_2d(st + kWgXStage, &a.dzmap, 0, (int)(ch * 64), &full[stage]);
            }
            for (uint32_t k = q > (uint32_t)kWgS ? q - kWgS : 0; k < q; ++k)
                mbar_drain(&full[k % kWgS], (k / kWgS) & 1, a.err);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // descriptors as 32-bit halves: start / 16 in bits 0-13, the leading
            // byte offset / 16 (the second M atom) in bits 16-29 of the low half
            const uint32_t base = smem_u32(smem), ones = smem_u32(sOnes);
            const uint64_t d0 = smem_desc_sw128(base);
            const uint32_t a_hi = (uint32_t)(d0 >> 32);
            const uint32_t lo0 = (uint32_t)d0 & 0xFFFFu;   // start field of the smem base, no offset
            uint32_t a_off[kWgPairs];   // start of tap 2j's window relative to its stage / 16, with the pair's offset
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t1 = 2 * j, t2 = 2 * j + 1;
                a_off[j] = (uint32_t)((P1 + tap_shift(t1, L)) * 8) |
                           ((uint32_t)((tap_shift(t2, L) - tap_shift(t1, L)) * 8) << 16);
            }
            a_off[4] = (uint32_t)((P1 + tap_shift(8, L)) * 8);
            uint32_t q = 0;
            for (long long ch = c_begin; ch < c_end; ++ch, ++q) {
                const uint32_t stage = q % kWgS, use = q / kWgS;
                if (!mbar_wait(&full[stage], use & 1, &abort_flag, a.err, a.spin_limit)) break;
                tc_fence_after();
                const uint32_t st = lo0 + stage * (kWgStage / 16);
                // pair 4: the ones atom lies ones - window bytes after tap 8's window
                const uint32_t w8 = base + stage * kWgStage + (P1 + tap_shift(8, L)) * 128;
                const uint32_t off4 = a_off[4] | (((ones - w8) >> 4) << 16);
                const uint32_t b_lo = st + (uint32_t)(kWgXStage / 16) | ((uint32_t)(kWgDStage >> 4) << 16);
#pragma unroll
                for (int j = 0; j < kWgPairs; ++j) {
                    const uint32_t a_lo = st + (j < 4 ? a_off[j] : off4);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        mma_bf16_lh(tmem + 64 * j, a_lo + ks * 128, a_hi, b_lo + ks * 128, a_hi, IDESC,
                                    (ch > c_begin || ks > 0) ? 1u : 0u);
                }
                mma_commit(&empty[stage]);
            }
            // completes after every MMA of the block (also on the abort path);
            // waited out here, so that no MMA outlives the tensor memory even
            // when the accumulator warps gave up first
            mma_commit(&accf);
            mbar_drain(&accf, 0, a.err);
        }
    } else {
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        float* out = a.partial + ((long long)blockIdx.x * kWgRows + row) * 64;
        bool ok = c_end > c_begin;
        if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&accf, 0, &abort_flag, a.err, a.spin_limit));
        if (ok) tc_fence_after();
#pragma unroll 1
        for (int j = 0; j < kWgPairs; ++j) {
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                float v[16];
                if (ok) {
                    tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + 64 * j + cc * 16, v);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0.0f;
                }
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(out + (long long)j * 128 * 64 + cc * 16 + i) =
                        make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// The first layer's weight and bias gradients on tcgen05: D[R][co] = sum_p
// A0[p][R] dZ[p][co] with A0[p][2 tap + ci] = X[p + shift(tap)][ci] and
// A0[p][18] = 1 (the bias row), a GEMM over positions (K) whose operands are
// both MN-major under the 128-byte swizzle.  Per chunk of 128 positions one
// TMA copy brings the strip of input positions its taps read (as for the
// first layer's conv) and another the chunk's 128 dZ rows; four warps write
// the chunk's A0 rows (128 bytes each: values 0..18, then zeros) into a
// swizzled tile; one thread issues eight K = 16 MMAs of M = 128 whose first
// 64-row atom is A0 and whose second is the chunk's dZ tile (the leading
// byte offset is the step from one tile to the other; rows 64..127 of D are
// never read).  D accumulates over the block's contiguous range of chunks in
// 64 tensor-memory columns, and rows 0..18 become the block's partial sums.
// dZ is zero on the map borders and past the batch (the caller zeroes the
// tail of the last chunk), so every position can enter the sums.
// ---------------------------------------------------------------------------
constexpr int kWg0Rows = 19;
struct Wgrad0Args {
    CUtensorMap in_map;   // X: [M][2] bf16 as [ceil(M/4)][8], box 8 x c1_strip_rows(L)
    CUtensorMap dzmap;    // dZ [M_alloc][64] bf16, box 64 x 128, 128-byte swizzle
    float* partial;       // [slices][19][64]
    long long M;
    int L;
    int* err;
    uint32_t spin_limit;   // polls before a pipeline wait gives up
};

constexpr int kW0S = 4;                              // pipeline depth
constexpr int kW0Tile = 128 * 128;                   // one A0 or dZ tile of 128 rows
constexpr int kW0Stage = 2 * kW0Tile;                // A0 tile, then the dZ tile
constexpr int kW0Threads = 6 * 32;                   // TMA warp, MMA warp, 4 operand warps
constexpr size_t kW0Smem = (size_t)kW0S * kW0Stage + kW0S * kC1StripStage + 1024;

__global__ void __launch_bounds__(kW0Threads, 1) wgrad0_kernel(const __grid_constant__ Wgrad0Args a) {
    constexpr uint32_t IDESC = idesc_bf16(128, 64) | (1u << 15) | (1u << 16);   // A, B MN-major
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sStrip = smem + kW0S * kW0Stage;
    __shared__ __align__(8) uint64_t full[kW0S], afull[kW0S], empty[kW0S], accf;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = a.M;
    const int L = a.L, P1 = L + 3;
    const long long n_chunks = (M + 127) / 128;
    const long long c_begin = n_chunks * blockIdx.x / gridDim.x, c_end = n_chunks * (blockIdx.x + 1) / gridDim.x;

    // A0 tiles start zero: 16-byte chunks 3..7 of every row are never written
    for (int i = tid; i < kW0S * (kW0Tile / 16); i += kW0Threads) {
        const int st = i / (kW0Tile / 16), j = i - st * (kW0Tile / 16);
        reinterpret_cast<uint4*>(smem + st * kW0Stage)[j] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int s = 0; s < kW0S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&afull[s], 128);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accf, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    if (warp == 1) tmem_alloc(&tmem_slot, 64);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)c1_strip_rows(L) * 16 + kW0Tile;
            uint32_t q = 0;
            for (long long ch = c_begin; ch < c_end; ++ch, ++q) {
                const uint32_t stage = q % kW0S, use = q / kW0S;
                if (use > 0 && !mbar_wait(&empty[stage], (use - 1) & 1, &abort_flag, a.err, a.spin_limit)) break;
                mbar_expect_tx(&full[stage], bytes);
                tma_load_2d(sStrip + stage * kC1StripStage, &a.in_map, 0, (int)floor_div4(ch * 128 - P1),
                            &full[stage]);
                tma_load_2d(smem + stage * kW0Stage + kW0Tile, &a.dzmap, 0, (int)(ch * 128), &full[stage]);
            }
            for (uint32_t k = q > (uint32_t)kW0S ? q - kW0S : 0; k < q; ++k)
                mbar_drain(&full[k % kW0S], (k / kW0S) & 1, a.err);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // descriptors as 32-bit halves: start / 16 in bits 0-13 and the
            // leading byte offset / 16 (A's second atom: the dZ tile) in bits
            // 16-29 of the low half
            const uint64_t d0 = smem_desc_sw128(smem_u32(smem));
            const uint32_t hi = (uint32_t)(d0 >> 32);
            const uint32_t lo0 = (uint32_t)d0 & 0xFFFFu;
            const uint32_t lbo = (uint32_t)(kW0Tile >> 4) << 16;
            uint32_t q = 0;
            for (long long ch = c_begin; ch < c_end; ++ch, ++q) {
                const uint32_t stage = q % kW0S, use = q / kW0S;
                if (!mbar_wait(&afull[stage], use & 1, &abort_flag, a.err, a.spin_limit)) break;
                tc_fence_after();
                const uint32_t a_lo = (lo0 + stage * (kW0Stage / 16)) | lbo;
                const uint32_t b_lo = (lo0 + stage * (kW0Stage / 16) + kW0Tile / 16) | lbo;
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)   // 16 positions (2048 bytes) per MMA
                    mma_bf16_lh(tmem, a_lo + ks * 128, hi, b_lo + ks * 128, hi, IDESC,
                                (ch > c_begin || ks > 0) ? 1u : 0u);
                mma_commit(&empty[stage]);
            }
            // completes after every MMA of the block (also on the abort path);
            // waited out here, so that no MMA outlives the tensor memory even
            // when the accumulator warps gave up first
            mma_commit(&accf);
            mbar_drain(&accf, 0, a.err);
        }
    } else {
        // operand rows: thread r writes row r (position ch * 128 + r) of every chunk
        const int r = 32 * (warp - 2) + lane, sw = r & 7;
        int sh[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) sh[t] = tap_shift(t, L);
        uint32_t q = 0;
        for (long long ch = c_begin; ch < c_end; ++ch, ++q) {
            const uint32_t stage = q % kW0S, use = q / kW0S;
            if (!mbar_wait(&full[stage], use & 1, &abort_flag, a.err, a.spin_limit)) break;
            const long long s0 = ch * 128 - P1;
            const int base = r + P1 + (int)(s0 - 4 * floor_div4(s0));   // strip index of position ch*128 + r
            const uint32_t* strip = reinterpret_cast<const uint32_t*>(sStrip + stage * kC1StripStage);
            uint32_t w[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) w[t] = strip[base + sh[t]];
            uint8_t* row = smem + stage * kW0Stage + r * 128;
            *reinterpret_cast<uint4*>(row + ((0 ^ sw) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(row + ((1 ^ sw) << 4)) = make_uint4(w[4], w[5], w[6], w[7]);
            *reinterpret_cast<uint4*>(row + ((2 ^ sw) << 4)) = make_uint4(w[8], 0x3F80u, 0u, 0u);   // R = 18: 1.0
            fence_async_smem();
            mbar_arrive(&afull[stage]);
        }
        if (warp == 4) {
            // tensor-memory lanes 0..31 (this warp's quarter): rows R = 0..18
            bool ok = c_end > c_begin;
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&accf, 0, &abort_flag, a.err, a.spin_limit));
            float v[64];
            if (ok) {
                tc_fence_after();
                tmem_ld64(tmem, v);
            } else {
#pragma unroll
                for (int i = 0; i < 64; ++i) v[i] = 0.0f;
            }
            if (lane < kWg0Rows) {
                float* out = a.partial + ((long long)blockIdx.x * kWg0Rows + lane) * 64;
#pragma unroll
                for (int i = 0; i < 64; i += 4)
                    *reinterpret_cast<float4*>(out + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 64);
}

// partial[s][R][co] summed over s -> flat gradient of layer l.  A block of 8
// warps takes 32 consecutive outputs (R, co); warp w adds the slices w, w + 8,
// .. in order and the 8 warp sums are added in order.
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(const float* partial, int n_slices, int rows_pad, int cin,
                                                           float* grad_w, float* grad_b) {
    __shared__ float part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;  // R * 64 + co
    const int R = i >> 6, co = i & 63;
    const bool valid = R <= 9 * cin;
    float s = 0.0f;
    if (valid) {
#pragma unroll 4
        for (int k = w; k < n_slices; k += 8) s += partial[((long long)k * rows_pad + R) * 64 + co];
    }
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && valid) {
        float t = part[0][lane];
#pragma unroll
        for (int j = 1; j < 8; ++j) t += part[j][lane];
        if (R < 9 * cin) grad_w[(long long)co * 9 * cin + R] = t;
        else grad_b[co] = t;
    }
}

// ---------------------------------------------------------------------------
// CUDA-core kernels
// ---------------------------------------------------------------------------

// Syndromes [n][2L(L-1)] -> padded input maps [n P^2][2]: channel 0 the
// sigma_x generators ((L-1) x L, last row zero), channel 1 the sigma_z
// generators (L x (L-1), last column zero); map (y, x) at padded (y+1, x+1).
__global__ void input_maps_kernel(const uint8_t* syn, long long n, int L, bf16* x0) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int P = L + 2;
    const long long PP = (long long)P * P;
    if (m >= n * PP) return;
    const long long item = m / PP;
    const int rem = (int)(m - item * PP), y = rem / P - 1, x = rem - (rem / P) * P - 1;
    float c0 = 0.0f, c1 = 0.0f;
    if (y >= 0 && y < L && x >= 0 && x < L) {
        const uint8_t* s = syn + item * 2 * L * (L - 1);
        c0 = y < L - 1 ? (float)(s[y * L + x] & 1) : 0.0f;
        c1 = x < L - 1 ? (float)(s[L * (L - 1) + y * (L - 1) + x] & 1) : 0.0f;
    }
    reinterpret_cast<uint32_t*>(x0)[m] = pack_bf16(c0, c1);
}

// Master weights -> bf16 GEMM operands.  Forward operand of layer l:
// [np][kp], row co, column tap * cin + ci, zero padded.  Input-gradient
// operand of layers 1..3: [64][576], row ci, column tap' * 64 + co holding
// W[co][8 - tap'][ci] (the kernel flipped in both directions).
struct PackArgs {
    const float* theta;
    bf16* fwd[5];
    bf16* bwd[3];
    long long fwd_begin[6];
    long long total;
};

__global__ void pack_kernel(PackArgs a) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.total) return;
    if (i < a.fwd_begin[5]) {
        int l = 0;
        while (i >= a.fwd_begin[l + 1]) ++l;
        const long long j = i - a.fwd_begin[l];
        const int kp = fwd_kp(l), cin = layer_cin(l);
        const int co = (int)(j / kp), k = (int)(j - (long long)co * kp);
        float v = 0.0f;
        if (co < layer_cout(l) && k < 9 * cin) v = a.theta[layer_woff(l) + (long long)co * 9 * cin + k];
        if (l == 0 && k >= 18 && k < 21) {
            // the bias as the exact sum of three bf16 parts (8 significant
            // bits each), multiplied by constant-one operand columns
            const float b = a.theta[layer_boff(0) + co];
            const float b1 = __bfloat162float(__float2bfloat16_rn(b));
            const float b2 = __bfloat162float(__float2bfloat16_rn(b - b1));
            v = k == 18 ? b1 : k == 19 ? b2 : b - b1 - b2;
        }
        a.fwd[l][j] = __float2bfloat16_rn(v);
    } else {
        const long long j = i - a.fwd_begin[5];
        const int l = (int)(j / (64 * 576)) + 1;
        const int jj = (int)(j - (long long)(l - 1) * 64 * 576);
        const int ci = jj / 576, k = jj - ci * 576, tapf = k / 64, co = k - tapf * 64;
        const float v = a.theta[layer_woff(l) + (long long)co * 576 + (8 - tapf) * 64 + ci];
        a.bwd[l - 1][jj] = __float2bfloat16_rn(v);
    }
}

// One warp per syndrome: the last layer on the middle lines and the parity
// readout.  The readout needs the last layer's channel 0 only on the middle
// column (map positions (i, m)) and channel 1 only on the middle row ((m, j)),
// so it computes just those 2L outputs: lane l holds the bf16 weights of
// input channels 2l, 2l + 1 for both outputs and the 9 taps, every output is
// a warp-wide sum (xor butterfly, fp32) plus the bias, and lane i < L keeps
// the logits of row i / column i.  The products are taken in lane order
// 0..31 by every lane.  With targets, also the loss and d loss / d z5 at the
// middle-line positions (dz5 must be zero elsewhere).
__device__ __forceinline__ float warp_prod_except(float t, int skip) {
    float r = 1.0f;
    for (int j = 0; j < 32; ++j) {
        const float v = __shfl_sync(0xffffffffu, t, j);
        if (j != skip) r *= v;
    }
    return r;
}

// Positions of a middle line evaluated per pass of the readout: their taps
// share rows, so K positions take (K + 2) x 3 loads per line instead of 9 K.
constexpr int kReadK = 4;

__global__ void __launch_bounds__(256, 4) readout_kernel(const bf16* w5, const float* b5, const bf16* a4,
                                                      const uint8_t* syn, long long n, int L, const float* targets,
                                                      float* logprob, float* dz5, float* loss_item) {
    // last-layer weights of channels 2 lane, 2 lane + 1 for (output, tap)
    __shared__ float2 sw[2][9][32];
    for (int idx = threadIdx.x; idx < 2 * 9 * 32; idx += blockDim.x) {
        const int co = idx / 288, t = (idx / 32) % 9, ln = idx % 32;
        const uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(w5 + co * 576 + t * 64) + ln);
        sw[co][t][ln] = make_float2(bf16_lo(v), bf16_hi(v));
    }
    __syncthreads();
    const long long item = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= n) return;
    const int m = (L - 1) / 2, P = L + 2;
    const long long base = item * P * P + P + 1;   // map (0, 0)
    const uint32_t* a = reinterpret_cast<const uint32_t*>(a4) + lane;   // 32 words per position
    float sa = 0.0f, sb = 0.0f;
    for (int i = 0; i < L; i += kReadK) {
        // line a: positions (i + k, m), rows i - 1 .. i + K, columns m - 1 .. m + 1;
        // line b: positions (m, i + k), columns i - 1 .. i + K, rows m - 1 .. m + 1
        uint32_t la[kReadK + 2][3], lb[kReadK + 2][3];
#pragma unroll
        for (int r = 0; r < kReadK + 2; ++r) {
            const int y = i - 1 + r;             // <= L: the bottom (right) border at most
            const bool ok = y <= L;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                la[r][c] = ok ? __ldg(a + (base + (long long)y * P + (m - 1 + c)) * 32) : 0u;
                lb[r][c] = ok ? __ldg(a + (base + (long long)(m - 1 + c) * P + y) * 32) : 0u;
            }
        }
        float acc[2][kReadK];
#pragma unroll
        for (int k = 0; k < kReadK; ++k) acc[0][k] = acc[1][k] = 0.0f;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const float2 wa = sw[0][t][lane], wb = sw[1][t][lane];
            const int dy = t / 3, dx = t % 3;
#pragma unroll
            for (int k = 0; k < kReadK; ++k) {
                const uint32_t xa = la[k + dy][dx], xb = lb[k + dx][dy];
                acc[0][k] = fmaf(bf16_lo(xa), wa.x, acc[0][k]);
                acc[0][k] = fmaf(bf16_hi(xa), wa.y, acc[0][k]);
                acc[1][k] = fmaf(bf16_lo(xb), wb.x, acc[1][k]);
                acc[1][k] = fmaf(bf16_hi(xb), wb.y, acc[1][k]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < kReadK; ++k) {
                acc[0][k] += __shfl_xor_sync(0xffffffffu, acc[0][k], o);
                acc[1][k] += __shfl_xor_sync(0xffffffffu, acc[1][k], o);
            }
#pragma unroll
        for (int k = 0; k < kReadK; ++k)
            if (lane == i + k && i + k < L) {
                sa = acc[0][k] + __ldg(b5 + 0);
                sb = acc[1][k] + __ldg(b5 + 1);
            }
    }
    float ta = 1.0f, tb = 1.0f;
    if (lane < L) {
        ta = -tanhf(0.5f * sa);
        tb = -tanhf(0.5f * sb);
    }
    const float Ma = warp_prod_except(ta, -1), Mb = warp_prod_except(tb, -1);
    // class code of the pure error: sigma_x strings of the sigma_z defects
    // that go left cross column 0, sigma_z strings of the sigma_x defects
    // that go up cross row 0
    const uint8_t* s = syn + item * 2 * L * (L - 1);
    int pa = 0, pb = 0;
    for (int g = lane; g < 2 * L * (L - 1); g += 32) {
        if (!(s[g] & 1)) continue;
        if (g < L * (L - 1)) {
            const int i = g / L;                       // sigma_x generator row (2i+1, 2j)
            pb ^= 2 * (i + 1) <= L;
        } else {
            const int j = (g - L * (L - 1)) % (L - 1);  // sigma_z generator (2i, 2j+1)
            pa ^= 2 * (j + 1) <= L;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        pa ^= __shfl_xor_sync(0xffffffffu, pa, o);
        pb ^= __shfl_xor_sync(0xffffffffu, pb, o);
    }
    const float Mac = fminf(fmaxf(Ma, -1.0f + kClip), 1.0f - kClip);
    const float Mbc = fminf(fmaxf(Mb, -1.0f + kClip), 1.0f - kClip);
    const float ln2 = 0.69314718f;
    const float la[2] = {log1pf(Mac) - ln2, log1pf(-Mac) - ln2};
    const float lb[2] = {log1pf(Mbc) - ln2, log1pf(-Mbc) - ln2};
    float lp[4];
    for (int k = 0; k < 4; ++k) lp[k] = la[(k & 1) ^ pa] + lb[(k >> 1) ^ pb];
    if (lane == 0 && logprob)
        for (int k = 0; k < 4; ++k) logprob[item * 4 + k] = lp[k];
    if (!targets) return;
    float q[4], ga[2] = {0.f, 0.f}, gb[2] = {0.f, 0.f}, loss = 0.0f;
    for (int k = 0; k < 4; ++k) {
        q[k] = targets[item * 4 + k];
        loss -= q[k] * lp[k];
        ga[(k & 1) ^ pa] -= q[k] / (float)n;
        gb[(k >> 1) ^ pb] -= q[k] / (float)n;
    }
    if (lane == 0) loss_item[item] = loss;
    const bool ina = Ma > -1.0f + kClip && Ma < 1.0f - kClip;
    const bool inb = Mb > -1.0f + kClip && Mb < 1.0f - kClip;
    const float dMa = ina ? ga[0] / (1.0f + Ma) - ga[1] / (1.0f - Ma) : 0.0f;
    const float dMb = inb ? gb[0] / (1.0f + Mb) - gb[1] / (1.0f - Mb) : 0.0f;
    const float oa = warp_prod_except(ta, lane), ob = warp_prod_except(tb, lane);
    if (lane < L) {
        dz5[(base + (long long)lane * P + m) * 2 + 0] = dMa * oa * (-0.5f * (1.0f - ta * ta));
        dz5[(base + (long long)m * P + lane) * 2 + 1] = dMb * ob * (-0.5f * (1.0f - tb * tb));
    }
}

// Sum of the per-item losses in a fixed order, divided by n.
__global__ void loss_sum_kernel(const float* loss_item, long long n, float* loss) {
    __shared__ float part[256];
    float s = 0.0f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += loss_item[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)n;
}

// Input gradient of the last layer, gated by the ReLU of layer 4 (padded
// maps; the border of dz5 is zero): dZ4[q][ci] = [a4[q][ci] > 0] sum over
// taps t of sum_co W5[co][t][ci] dz5[q - shift(t)][co] for interior q, and 0
// on the border.  dz5 is nonzero only on channel 0 of the middle column x = m
// and channel 1 of the middle row y = m, so dZ4 can be nonzero only in the
// bands y in [m-1, m+1] (3L positions) and x in [m-1, m+1] outside them
// (3(L-3) at most): the caller zeroes dZ4 and this kernel computes those
// bands, thread = (item, band slot of 6L, 8-channel group).
__global__ void conv5_dgrad_kernel(const bf16* w5, const float* dz5, const bf16* a4, long long n, int L,
                                   bf16* dz4) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int NB = 6 * L;
    if (i >= n * NB * 8) return;
    const long long item = i / (NB * 8);
    const int j = (int)(i / 8 - item * NB), cg = (int)(i & 7) * 8;
    const int m = (L - 1) / 2, P = L + 2;
    int y, x;
    if (j < 3 * L) {
        y = m - 1 + j / L;
        x = j % L;
    } else {
        y = (j - 3 * L) / 3;
        x = m - 1 + (j - 3 * L) % 3;
        if (y >= m - 1 && y <= m + 1) return;   // in the row band
    }
    if (y < 0 || y >= L || x < 0 || x >= L) return;
    const long long q = item * P * P + (long long)(y + 1) * P + (x + 1);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool any = false;
    for (int t = 0; t < 9; ++t) {
        const float2 d = *reinterpret_cast<const float2*>(dz5 + (q - tap_shift(t, L)) * 2);
        if (d.x == 0.0f && d.y == 0.0f) continue;
        any = true;
        const float g[2] = {d.x, d.y};
        for (int co = 0; co < kOut; ++co) {
            const uint4 wv = *reinterpret_cast<const uint4*>(w5 + (long long)co * 576 + t * 64 + cg);
            const uint32_t ww[4] = {wv.x, wv.y, wv.z, wv.w};
            for (int k = 0; k < 4; ++k) {
                acc[2 * k] += bf16_lo(ww[k]) * g[co];
                acc[2 * k + 1] += bf16_hi(ww[k]) * g[co];
            }
        }
    }
    if (!any) return;   // stays zero
    const uint4 av = *reinterpret_cast<const uint4*>(a4 + q * 64 + cg);
    const uint32_t aw[4] = {av.x, av.y, av.z, av.w};
    uint32_t o[4];
    for (int k = 0; k < 4; ++k)
        o[k] = pack_bf16(bf16_lo(aw[k]) > 0.0f ? acc[2 * k] : 0.0f, bf16_hi(aw[k]) > 0.0f ? acc[2 * k + 1] : 0.0f);
    *reinterpret_cast<uint4*>(dz4 + q * 64 + cg) = make_uint4(o[0], o[1], o[2], o[3]);
}

// Last-layer weight and bias gradients of one syndrome (block per item, 576
// threads = (tap, ci)): S[item][co][tap * 64 + ci] = sum_p dz5[p][co]
// a4[p + shift(tap)][ci] over the item's positions p, Sb[item][co] = sum_p
// dz5[p][co].  dz5 is nonzero only on channel 0 of the middle column and
// channel 1 of the middle row, so the sums run over those lines, row by row
// (column by column).  The neighbours of a map position lie in the item's
// padded frame.
__global__ void conv5_wgrad_item_kernel(const float* dz5, const bf16* a4, int L, float* S, float* Sb) {
    const long long item = blockIdx.x;
    const int t = threadIdx.x >> 6, ci = threadIdx.x & 63;
    const int P = L + 2, PP = P * P, sh = tap_shift(t, L), m = (L - 1) / 2;
    const float* d = dz5 + item * PP * 2;
    const bf16* a = a4 + item * (long long)PP * 64;
    float acc0 = 0.0f, acc1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
    for (int i = 0; i < L; ++i) {
        const int pa = (i + 1) * P + m + 1, pb = (m + 1) * P + i + 1;
        const float d0 = d[2 * pa], d1 = d[2 * pb + 1];
        b0 += d0;
        b1 += d1;
        acc0 += d0 * __bfloat162float(a[(pa + sh) * 64 + ci]);
        acc1 += d1 * __bfloat162float(a[(pb + sh) * 64 + ci]);
    }
    S[(item * 2 + 0) * 576 + threadIdx.x] = acc0;
    S[(item * 2 + 1) * 576 + threadIdx.x] = acc1;
    if (threadIdx.x == 0) {
        Sb[item * 2 + 0] = b0;
        Sb[item * 2 + 1] = b1;
    }
}

// Sum over the items: dW5[co][j] = sum_item S[item][co][j], db5[co] =
// sum_item Sb[item][co].  A block of 32 warps takes 32 consecutive outputs;
// warp w adds the items w, w + 32, .. in order and the 32 warp sums are
// added in order.
constexpr int kC5Warps = 32;
__global__ void __launch_bounds__(kC5Warps * 32) conv5_wgrad_kernel(const float* S, const float* Sb, long long n,
                                                                    float* grad_w, float* grad_b) {
    __shared__ float part[kC5Warps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const bool is_w = i < kOut * 576, valid = i < kOut * 576 + kOut;
    float s = 0.0f;
    if (is_w) {
        const int co = i / 576, jj = i - co * 576;
#pragma unroll 4
        for (long long k = w; k < n; k += kC5Warps) s += S[(k * 2 + co) * 576 + jj];
    } else if (valid) {
        const int co = i - kOut * 576;
#pragma unroll 4
        for (long long k = w; k < n; k += kC5Warps) s += Sb[k * 2 + co];
    }
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && valid) {
        float t = part[0][lane];
#pragma unroll
        for (int k = 1; k < kC5Warps; ++k) t += part[k][lane];
        if (is_w) grad_w[i] = t;
        else grad_b[i - kOut * 576] = t;
    }
}

__global__ void adam_kernel(float* theta, float* m1, float* m2, const float* grad, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float a = b1 * m1[i] + (1.0f - b1) * g;
    const float b = b2 * m2[i] + (1.0f - b2) * g * g;
    m1[i] = a;
    m2[i] = b;
    theta[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

__global__ void soft_targets_kernel(const double* lr, long long n, float* q) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = lr[i * 4];
    for (int k = 1; k < 4; ++k) m = fmax(m, lr[i * 4 + k]);
    double e[4], s = 0.0;
    for (int k = 0; k < 4; ++k) {
        e[k] = exp(lr[i * 4 + k] - m);
        s += e[k];
    }
    for (int k = 0; k < 4; ++k) q[i * 4 + k] = (float)(e[k] / s);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ---------------------------------------------------------------------------
// Network state and its launches
// ---------------------------------------------------------------------------
struct CnnNet {
    surfmcmc_ctx* ctx = nullptr;
    int device = 0, L = 0, P = 0, sms = 0;
    long long max_batch = 0;
    long long step = 0;
    // parameters (float32) and Adam moments, gradient
    float *theta = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr;
    // packed operands
    bf16* fwd[5] = {};
    bf16* bwd[3] = {};
    // activations and gradients for max_batch syndromes
    uint8_t* syn = nullptr;
    float* targets = nullptr;
    bf16* x0 = nullptr;
    bf16* act[4] = {};
    bf16* dz[2] = {};
    float *logprob = nullptr, *dz5 = nullptr, *loss_item = nullptr, *loss = nullptr, *S5 = nullptr, *Sb5 = nullptr;
    float* partial = nullptr;
    int* err = nullptr;
    uint32_t spin_limit = kSpinLimit;   // polls of a pipeline wait (smaller only to test the time-out path)
    // TMA map of the first layer's input x0 (16-byte rows of 4 positions)
    CUtensorMap map_x0;
    // TMA maps of the 64-channel tensors that convs read: act[0..3], dz[0..1]
    CUtensorMap map_act[4], map_dz[2];
    // the same tensors in boxes of 128 rows (output tiles, ReLU gates)
    CUtensorMap tile_act[4], tile_dz[2];
    // weight gradient: layer inputs act[0..2] with its halo, dz in 64-row boxes
    CUtensorMap wg_act[3], wg_dz[2];
    std::vector<void*> allocs;
};

namespace {

cudaError_t net_alloc(CnnNet* net, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) net->allocs.push_back(*p);
    return e;
}

// Shared-memory limits of the network kernels, set once per device (the
// attribute belongs to the current device's context), under a lock.
cudaError_t prepare_kernels() {
    constexpr int kMaxDevices = 64;
    static std::mutex m;
    static bool done[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(m);
    if (done[dev]) return cudaSuccess;
    if ((e = set_smem(conv1_kernel, kC1Smem))) return e;
    if ((e = set_smem(conv_tma_kernel<64, kEpiRelu>, conv_tma_smem_bytes<64, kEpiRelu>()))) return e;
    if ((e = set_smem(conv_tma_kernel<64, kEpiMask>, conv_tma_smem_bytes<64, kEpiMask>()))) return e;
    if ((e = set_smem(wgrad_kernel, kWgSmem))) return e;
    if ((e = set_smem(wgrad0_kernel, kW0Smem))) return e;
    done[dev] = true;
    return cudaSuccess;
}

cudaError_t launch_conv1(const CnnNet* net, const Conv1Args& a, cudaStream_t s) {
    const long long tiles = (a.M + 127) / 128;
    if (tiles == 0) return cudaSuccess;
    const int grid = (int)(tiles < net->sms ? tiles : net->sms);
    conv1_kernel<<<grid, kC1Threads, kC1Smem, s>>>(a);
    return cudaGetLastError();
}

template <int NP, int EPI>
cudaError_t launch_conv_tma(const CnnNet* net, const ConvTmaArgs& a, cudaStream_t s) {
    const long long tiles = (a.M + 127) / 128;
    if (tiles == 0) return cudaSuccess;
    const int grid = (int)(tiles < net->sms ? tiles : net->sms);
    conv_tma_kernel<NP, EPI><<<grid, kTmaThreads, conv_tma_smem_bytes<NP, EPI>(), s>>>(a);
    return cudaGetLastError();
}

// TMA map of a [rows][width] bf16 tensor in boxes of box_rows rows x width
// (width 64: 128-byte rows with the 128-byte swizzle; width 8: 16-byte rows,
// no swizzle); rows outside the tensor read as zero.
cudaError_t make_map_w(CUtensorMap* map, void* base, long long rows, int box_rows, int width) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult qr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
        if (e != cudaSuccess) return e;
        if (qr != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)width * 2};
    const cuuint32_t box[2] = {(cuuint32_t)width, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                              CU_TENSOR_MAP_INTERLEAVE_NONE,
                              width == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_map(CUtensorMap* map, void* base, long long rows, int box_rows) {
    return make_map_w(map, base, rows, box_rows, 64);
}

// First layer: rows of dZ past the batch in the last 128-position chunk are
// zeroed first, then the in-order sum over the slices.
cudaError_t launch_wgrad0(const CnnNet* net, int dzi, long long M, cudaStream_t s) {
    const long long chunks = (M + 127) / 128;
    if (chunks == 0) return cudaSuccess;
    const long long m_alloc = net->max_batch * net->P * net->P;
    const long long tail_end = chunks * 128 < m_alloc ? chunks * 128 : m_alloc;
    cudaError_t e;
    if (tail_end > M && (e = cudaMemsetAsync(net->dz[dzi] + M * 64, 0, (size_t)(tail_end - M) * 128, s))) return e;
    const int slices = (int)(chunks < net->sms ? chunks : net->sms);
    Wgrad0Args a;
    memset(&a, 0, sizeof a);
    a.in_map = net->map_x0;
    a.dzmap = net->tile_dz[dzi];
    a.partial = net->partial;
    a.M = M;
    a.L = net->L;
    a.err = net->err;
    a.spin_limit = net->spin_limit;
    wgrad0_kernel<<<slices, kW0Threads, kW0Smem, s>>>(a);
    if ((e = cudaGetLastError())) return e;
    wgrad_reduce_kernel<<<(kWg0Rows * 64 + 31) / 32, 256, 0, s>>>(net->partial, (int)slices, kWg0Rows, 2,
                                                                     net->grad + layer_woff(0),
                                                                     net->grad + layer_boff(0));
    return cudaGetLastError();
}

// Weight gradient of layer l (1..3): X = its input, dZ = the gradient of its
// pre-activation; rows of dZ past the batch in the last 64-position chunk
// are zeroed first (the tensor map spans the whole buffer).
cudaError_t launch_wgrad(const CnnNet* net, int xi, int dzi, long long M, int layer, cudaStream_t s) {
    const long long chunks = (M + 63) / 64;
    if (chunks == 0) return cudaSuccess;
    const long long m_alloc = net->max_batch * net->P * net->P;
    const long long tail_end = chunks * 64 < m_alloc ? chunks * 64 : m_alloc;
    cudaError_t e;
    if (tail_end > M && (e = cudaMemsetAsync(net->dz[dzi] + M * 64, 0, (size_t)(tail_end - M) * 128, s))) return e;
    const int slices = (int)(chunks < net->sms ? chunks : net->sms);
    WgradArgs a;
    memset(&a, 0, sizeof a);
    a.xmap = net->wg_act[xi];
    a.dzmap = net->wg_dz[dzi];
    a.partial = net->partial;
    a.M = M;
    a.L = net->L;
    a.halo_rows = wg_halo_rows(net->L);
    a.err = net->err;
    a.spin_limit = net->spin_limit;
    wgrad_kernel<<<slices, kWgTmaThreads, kWgSmem, s>>>(a);
    if ((e = cudaGetLastError())) return e;
    wgrad_reduce_kernel<<<(577 * 64 + 31) / 32, 256, 0, s>>>(net->partial, slices, kWgRows, 64,
                                                               net->grad + layer_woff(layer),
                                                               net->grad + layer_boff(layer));
    return cudaGetLastError();
}

}  // namespace

cudaError_t cnn_pack(CnnNet* net, cudaStream_t s) {
    PackArgs a;
    a.theta = net->theta;
    long long off = 0;
    for (int l = 0; l < 5; ++l) {
        a.fwd[l] = net->fwd[l];
        a.fwd_begin[l] = off;
        off += (long long)fwd_np(l) * fwd_kp(l);
    }
    a.fwd_begin[5] = off;
    for (int l = 0; l < 3; ++l) a.bwd[l] = net->bwd[l];
    a.total = off + 3LL * 64 * 576;
    pack_kernel<<<(unsigned)((a.total + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Forward pass of n <= max_batch syndromes already in net->syn (or syn):
// activations kept for a backward pass; log-probabilities to logprob.
cudaError_t cnn_forward_dev(CnnNet* net, const uint8_t* syn, long long n, const float* targets, float* logprob,
                            cudaStream_t s) {
    cudaError_t e;
    const int L = net->L;
    const long long M = n * net->P * net->P;
    if (n == 0) return cudaSuccess;
    if ((e = prepare_kernels())) return e;
    input_maps_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(syn, n, L, net->x0);
    if ((e = cudaGetLastError())) return e;
    Conv1Args c1;
    memset(&c1, 0, sizeof c1);
    c1.in_map = net->map_x0;
    c1.out_map = net->tile_act[0];
    c1.wmat = net->fwd[0];
    c1.M = M;
    c1.L = L;
    c1.err = net->err;
    c1.spin_limit = net->spin_limit;
    if ((e = launch_conv1(net, c1, s))) return e;
    ConvTmaArgs a;
    memset(&a, 0, sizeof a);
    a.M = M;
    a.L = L;
    a.halo_rows = halo_tile_rows(L);
    a.err = net->err;
    a.spin_limit = net->spin_limit;
    for (int l = 1; l < 4; ++l) {
        a.map = net->map_act[l - 1];
        a.out_map = net->tile_act[l];
        a.wmat = net->fwd[l];
        a.bias = net->theta + layer_boff(l);
        if ((e = launch_conv_tma<64, kEpiRelu>(net, a, s))) return e;
    }
    if (targets && (e = cudaMemsetAsync(net->dz5, 0, (size_t)M * 8, s))) return e;
    readout_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(net->fwd[4], net->theta + layer_boff(4), net->act[3], syn,
                                                           n, L, targets, logprob, net->dz5, net->loss_item);
    return cudaGetLastError();
}

// Loss and flat gradient of n syndromes with soft targets.
cudaError_t cnn_backward_dev(CnnNet* net, const uint8_t* syn, long long n, const float* targets, cudaStream_t s) {
    cudaError_t e;
    const int L = net->L;
    const long long M = n * net->P * net->P;
    if ((e = cnn_forward_dev(net, syn, n, targets, net->logprob, s))) return e;
    loss_sum_kernel<<<1, 256, 0, s>>>(net->loss_item, n, net->loss);
    if ((e = cudaGetLastError())) return e;
    // last layer (CUDA cores)
    conv5_wgrad_item_kernel<<<(unsigned)n, 576, 0, s>>>(net->dz5, net->act[3], L, net->S5, net->Sb5);
    if ((e = cudaGetLastError())) return e;
    conv5_wgrad_kernel<<<(kOut * 576 + kOut + 31) / 32, kC5Warps * 32, 0, s>>>(net->S5, net->Sb5, n,
                                                                        net->grad + layer_woff(4),
                                                                        net->grad + layer_boff(4));
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaMemsetAsync(net->dz[0], 0, (size_t)M * 128, s))) return e;
    conv5_dgrad_kernel<<<(unsigned)((n * 6 * L * 8 + 255) / 256), 256, 0, s>>>(net->fwd[4], net->dz5, net->act[3], n, L,
                                                                             net->dz[0]);
    if ((e = cudaGetLastError())) return e;
    // layers 4, 3, 2: weight gradient, then input gradient gated by the layer below
    ConvTmaArgs a;
    memset(&a, 0, sizeof a);
    a.M = M;
    a.L = L;
    a.halo_rows = halo_tile_rows(L);
    a.err = net->err;
    a.spin_limit = net->spin_limit;
    int cur = 0;
    for (int l = 3; l >= 1; --l) {
        if ((e = launch_wgrad(net, l - 1, cur, M, l, s))) return e;
        a.map = net->map_dz[cur];
        a.out_map = net->tile_dz[cur ^ 1];
        a.mask_map = net->tile_act[l - 1];
        a.wmat = net->bwd[l - 1];
        if ((e = launch_conv_tma<64, kEpiMask>(net, a, s))) return e;
        cur ^= 1;
    }
    return launch_wgrad0(net, cur, M, s);
}

cudaError_t cnn_adam_dev(CnnNet* net, float lr, cudaStream_t s) {
    net->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - pow(b1, (double)net->step));
    const float c2 = (float)(1.0 - pow(b2, (double)net->step));
    adam_kernel<<<(unsigned)((kParams + 255) / 256), 256, 0, s>>>(net->theta, net->m1, net->m2, net->grad, kParams,
                                                                   lr, (float)b1, (float)b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    return cnn_pack(net, s);
}

}  // namespace surfmcmc

using namespace surfmcmc;

struct surfmcmc_cnn : public CnnNet {};

namespace {

int cfail(surfmcmc_cnn* net, int code, const char* msg) {
    if (net && net->ctx) ctx_set_error(net->ctx, msg);
    return code;
}

int cuda_fail(surfmcmc_cnn* net, cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return cfail(net, e == cudaErrorMemoryAllocation ? SURFMCMC_ENOMEM : SURFMCMC_ECUDA, buf);
}

// Reads the device error flag of the tensor-core kernels (synchronises s).
int check_err(surfmcmc_cnn* net, cudaStream_t s) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, net->err, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(net, e, "network kernels");
    if (h) {
        cudaMemsetAsync(net->err, 0, sizeof(int), s);
        return cfail(net, SURFMCMC_ECUDA, h == kWaitTimeout ? "network kernel: a pipeline wait timed out (device flag 1)"
                                                          : "network kernel: unknown device error flag");
    }
    return SURFMCMC_OK;
}

struct NetGuard {
    int prev = -1;
    explicit NetGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~NetGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

namespace surfmcmc {

cudaError_t cnn_logprob(surfmcmc_cnn* net, const uint8_t* syn, long long n, float* logprob, cudaStream_t s) {
    const long long ns = 2LL * net->L * (net->L - 1);
    for (long long b0 = 0; b0 < n; b0 += net->max_batch) {
        const long long b = n - b0 < net->max_batch ? n - b0 : net->max_batch;
        const cudaError_t e = cnn_forward_dev(net, syn + b0 * ns, b, nullptr, logprob + b0 * 4, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int cnn_code_size(const surfmcmc_cnn* net) { return net->L; }

}  // namespace surfmcmc

extern "C" {

int64_t surfmcmc_cnn_n_params(void) { return kParams; }

int surfmcmc_cnn_create(surfmcmc_ctx* ctx, int32_t L, int64_t max_batch, surfmcmc_cnn** out) {
    if (!ctx || !out) return SURFMCMC_EINVAL;
    *out = nullptr;
    if (L < 3 || L > SURFMCMC_MAX_L) {
        ctx_set_error(ctx, "network: L outside 3..31");
        return SURFMCMC_EINVAL;
    }
    if (max_batch < 1 || max_batch > (1LL << 20)) {
        ctx_set_error(ctx, "network: max_batch outside 1..2^20");
        return SURFMCMC_EINVAL;
    }
    surfmcmc_cnn* net = new surfmcmc_cnn();
    net->ctx = ctx;
    net->device = ctx_device(ctx);
    net->L = L;
    net->P = L + 2;
    net->max_batch = max_batch;
    NetGuard g(net->device);
    cudaError_t e = cudaDeviceGetAttribute(&net->sms, cudaDevAttrMultiProcessorCount, net->device);
    const long long M = max_batch * net->P * net->P;   // padded positions
    const size_t P = (size_t)kParams * 4;
    auto na = [&](auto** field, size_t bytes) {
        void* p = nullptr;
        if (e == cudaSuccess) e = net_alloc(net, &p, bytes);
        *field = (std::remove_pointer_t<decltype(field)>)p;
    };
    na(&net->theta, P);
    na(&net->m1, P);
    na(&net->m2, P);
    na(&net->grad, P);
    for (int l = 0; l < 5; ++l) na(&net->fwd[l], (size_t)fwd_np(l) * fwd_kp(l) * 2);
    for (int l = 0; l < 3; ++l) na(&net->bwd[l], (size_t)64 * 576 * 2);
    na(&net->syn, (size_t)max_batch * 2 * L * (L - 1));
    na(&net->targets, (size_t)max_batch * 16);
    na(&net->x0, (size_t)(M + 3) / 4 * 16);   // whole 16-byte rows for the first layer's TMA map
    for (int l = 0; l < 4; ++l) na(&net->act[l], (size_t)M * 128);
    na(&net->dz5, (size_t)M * 8);
    na(&net->dz[0], (size_t)M * 128);
    na(&net->dz[1], (size_t)M * 128);
    na(&net->logprob, (size_t)max_batch * 16);
    na(&net->loss_item, (size_t)max_batch * 4);
    na(&net->loss, 4);
    na(&net->S5, (size_t)max_batch * 2 * 576 * 4);
    na(&net->Sb5, (size_t)max_batch * 2 * 4);
    na(&net->partial, (size_t)(net->sms > kMaxSplits ? net->sms : kMaxSplits) * kWgRows * 64 * 4);
    na(&net->err, 4);
    const int halo = halo_tile_rows(L);
    if (e == cudaSuccess) e = make_map_w(&net->map_x0, net->x0, (M + 3) / 4, c1_strip_rows(L), 8);
    if (e == cudaSuccess) e = cudaMemset(net->x0, 0, (size_t)(M + 3) / 4 * 16);
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) e = make_map(&net->map_act[l], net->act[l], M, halo);
    for (int l = 0; l < 2 && e == cudaSuccess; ++l) e = make_map(&net->map_dz[l], net->dz[l], M, halo);
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) e = make_map(&net->tile_act[l], net->act[l], M, 128);
    for (int l = 0; l < 2 && e == cudaSuccess; ++l) e = make_map(&net->tile_dz[l], net->dz[l], M, 128);
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) e = make_map(&net->wg_act[l], net->act[l], M, wg_halo_rows(L));
    for (int l = 0; l < 2 && e == cudaSuccess; ++l) e = make_map(&net->wg_dz[l], net->dz[l], M, 64);
    if (e == cudaSuccess) e = cudaMemset(net->err, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(net->theta, 0, P);
    if (e == cudaSuccess) e = cudaMemset(net->m1, 0, P);
    if (e == cudaSuccess) e = cudaMemset(net->m2, 0, P);
    if (e == cudaSuccess) e = prepare_kernels();
    if (e == cudaSuccess) e = cnn_pack(net, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        const int rc = cuda_fail(net, e, "network create");
        surfmcmc_cnn_destroy(net);
        return rc;
    }
    *out = net;
    return SURFMCMC_OK;
}

void surfmcmc_cnn_destroy(surfmcmc_cnn* net) {
    if (!net) return;
    NetGuard g(net->device);
    cudaDeviceSynchronize();
    for (void* p : net->allocs) cudaFree(p);
    delete net;
}

int surfmcmc_cnn_set_params(surfmcmc_cnn* net, const float* params) {
    if (!net || !params) return cfail(net, SURFMCMC_EINVAL, "network: NULL params");
    NetGuard g(net->device);
    const size_t P = (size_t)kParams * 4;
    cudaError_t e = cudaMemcpy(net->theta, params, P, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemset(net->m1, 0, P);
    if (e == cudaSuccess) e = cudaMemset(net->m2, 0, P);
    if (e == cudaSuccess) e = cnn_pack(net, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(net, e, "network set_params");
    net->step = 0;
    return SURFMCMC_OK;
}

int surfmcmc_cnn_get_params(surfmcmc_cnn* net, float* params) {
    if (!net || !params) return cfail(net, SURFMCMC_EINVAL, "network: NULL params");
    NetGuard g(net->device);
    cudaError_t e = cudaMemcpy(params, net->theta, (size_t)kParams * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(net, e, "network get_params");
    return SURFMCMC_OK;
}

int surfmcmc_cnn_forward(surfmcmc_cnn* net, const uint8_t* syndromes, int64_t n, float* out_logprob,
                         void* stream) {
    if (!net) return SURFMCMC_EINVAL;
    if (n < 0 || (n > 0 && (!syndromes || !out_logprob))) return cfail(net, SURFMCMC_EINVAL, "network forward: bad args");
    if (n == 0) return SURFMCMC_OK;
    NetGuard g(net->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ns = (size_t)2 * net->L * (net->L - 1);
    const bool syn_dev = device_ptr(syndromes), out_dev = device_ptr(out_logprob);
    for (int64_t b0 = 0; b0 < n; b0 += net->max_batch) {
        const int64_t b = n - b0 < net->max_batch ? n - b0 : net->max_batch;
        const uint8_t* sp = syndromes + b0 * ns;
        cudaError_t e = cudaSuccess;
        if (!syn_dev) {
            e = cudaMemcpyAsync(net->syn, sp, b * ns, cudaMemcpyHostToDevice, s);
            sp = net->syn;
        }
        float* lp = out_dev ? out_logprob + b0 * 4 : net->logprob;
        if (e == cudaSuccess) e = cnn_forward_dev(net, sp, b, nullptr, lp, s);
        if (e == cudaSuccess && !out_dev)
            e = cudaMemcpyAsync(out_logprob + b0 * 4, net->logprob, b * 16, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(net, e, "network forward");
        if (!out_dev || !syn_dev) {
            const int rc = check_err(net, s);
            if (rc) return rc;
        }
    }
    if (syn_dev && out_dev) return check_err(net, s);
    return SURFMCMC_OK;
}

int surfmcmc_cnn_gradient(surfmcmc_cnn* net, const uint8_t* syndromes, const float* targets, int64_t n,
                          float* out_loss, float* out_grad, void* stream) {
    if (!net) return SURFMCMC_EINVAL;
    if (n < 1 || n > net->max_batch || !syndromes || !targets)
        return cfail(net, SURFMCMC_EINVAL, "network gradient: need 1 <= n <= max_batch and inputs");
    NetGuard g(net->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ns = (size_t)2 * net->L * (net->L - 1);
    cudaError_t e = cudaMemcpyAsync(net->syn, syndromes, n * ns, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->targets, targets, n * 16, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cnn_backward_dev(net, net->syn, n, net->targets, s);
    if (e == cudaSuccess && out_loss) e = cudaMemcpyAsync(out_loss, net->loss, 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess && out_grad) e = cudaMemcpyAsync(out_grad, net->grad, (size_t)kParams * 4, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(net, e, "network gradient");
    return check_err(net, s);
}

int surfmcmc_cnn_train_step(surfmcmc_cnn* net, const uint8_t* syndromes, const float* targets, int64_t n,
                            float lr, float* out_loss, void* stream) {
    if (!net) return SURFMCMC_EINVAL;
    if (n < 1 || n > net->max_batch || !syndromes || !targets || !(lr > 0.0f))
        return cfail(net, SURFMCMC_EINVAL, "network train_step: need 1 <= n <= max_batch, inputs, lr > 0");
    NetGuard g(net->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ns = (size_t)2 * net->L * (net->L - 1);
    const uint8_t* sp = syndromes;
    const float* tp = targets;
    cudaError_t e = cudaSuccess;
    if (!device_ptr(syndromes)) {
        e = cudaMemcpyAsync(net->syn, syndromes, n * ns, cudaMemcpyHostToDevice, s);
        sp = net->syn;
    }
    if (e == cudaSuccess && !device_ptr(targets)) {
        e = cudaMemcpyAsync(net->targets, targets, n * 16, cudaMemcpyHostToDevice, s);
        tp = net->targets;
    }
    if (e == cudaSuccess) e = cnn_backward_dev(net, sp, n, tp, s);
    if (e == cudaSuccess) e = cnn_adam_dev(net, lr, s);
    if (e == cudaSuccess && out_loss) e = cudaMemcpyAsync(out_loss, net->loss, 4, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(net, e, "network train_step");
    if (out_loss && !device_ptr(out_loss)) return check_err(net, s);
    return SURFMCMC_OK;
}

int surfmcmc_cnn_soft_targets(const double* log_ratio, int64_t n, float* targets, void* stream) {
    if (n < 0) return SURFMCMC_EINVAL;
    if (n == 0) return SURFMCMC_OK;
    if (!device_ptr(log_ratio) || !device_ptr(targets)) return SURFMCMC_EINVAL;
    soft_targets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(log_ratio, n, targets);
    return cudaGetLastError() == cudaSuccess ? SURFMCMC_OK : SURFMCMC_ECUDA;
}

int surfmcmc_cnn_set_wait_limit(surfmcmc_cnn* net, uint32_t polls) {
    if (!net) return SURFMCMC_EINVAL;
    net->spin_limit = polls ? polls : kSpinLimit;
    return SURFMCMC_OK;
}

int surfmcmc_cnn_status(surfmcmc_cnn* net, void* stream) {
    if (!net) return SURFMCMC_EINVAL;
    NetGuard g(net->device);
    return check_err(net, (cudaStream_t)stream);
}

}  // extern "C"
