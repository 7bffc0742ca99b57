// The Metropolis sweep kernel (Sec. IV / IV.A, parallelised as in Sec. V),
// templated on the chain layout, the lanes per bundle, the scan mode and the
// noise model; sweep.cu and sweep_flips.cu instantiate it for depolarizing
// noise and for independent bit and phase flips.
//
// Data layout.  Chains are bit-sliced: a "bundle" holds 32 chains, and each
// data qubit of a bundle is two 32-bit words in shared memory, X[q] and Z[q],
// whose bit b is the x (z) part of the Pauli frame of the bundle's chain b.
// One proposal of generator g is therefore evaluated for 32 chains at once
// with bitwise logic on the 3-4 words of its support.
//
// Work split.  A warp holds 32/LAM bundles; LAM lanes share a bundle and
// split the generators of the current colour (Sec. V: the four groups have
// no qubit in common, so their proposals are independent and any order
// within a colour gives the sequential result).  After each colour phase
// every lane adds the occupancy of its slice of the qubits into a running
// carry-save counter; the LAM lanes' counters are added together and credited
// to the chains' sums only when a counter could overflow and at the end.
//
// Acceptance.  Delta n <= 0 is accepted; Delta n = d > 0 is accepted iff the
// chain's uniform u < T[d].  u is compared digit by digit, most significant
// first: plane k of Philox output supplies digit 31-k of u for the 32 chains,
// and a chain is decided at its first digit that differs from T[d]'s.  The
// warp stops drawing planes once every chain of its proposals is decided.
#pragma once
#include <mutex>

#include "common.cuh"

namespace surfmcmc {

__device__ __forceinline__ void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// Occupancy words of the qubits base + i LAM, i < 8 (N = 8) or i < 4 (N =
// 4): for depolarizing noise (IND false) a qubit counts once if it carries
// any error (X | Z); for independent flips (IND true) its bit flip and its
// phase flip count separately, four qubits per batch of 8 words.  The planes
// are zero-padded to a multiple of 4 LAM words, so a depolarizing pass takes
// batches of 8 and at most one batch of 4, every index in range.
template <int LAM, bool IND, int N = 8>
__device__ __forceinline__ void occupancy(const uint32_t* X, const uint32_t* Z, int base, uint32_t x[N]) {
    static_assert(N == 8 || (N == 4 && !IND), "independent flips count in batches of 8 words");
#pragma unroll
    for (int i = 0; i < (IND ? 4 : N); ++i) {
        const int q = base + i * LAM;
        if (IND) {
            x[2 * i] = X[q];
            x[2 * i + 1] = Z[q];
        } else {
            x[i] = X[q] | Z[q];
        }
    }
}

// Adds a batch of occupancy words to a carry-save count (ones, twos, fours)
// and returns the carry of weight 8.
template <int N>
__device__ __forceinline__ uint32_t add_batch(uint32_t& ones, uint32_t& twos, uint32_t& fours, const uint32_t x[N]) {
    uint32_t ta, tb, e;
    if constexpr (N == 8) {
        uint32_t fa, fb;
        csa(ta, ones, ones, x[0], x[1]);
        csa(tb, ones, ones, x[2], x[3]);
        csa(fa, twos, twos, ta, tb);
        csa(ta, ones, ones, x[4], x[5]);
        csa(tb, ones, ones, x[6], x[7]);
        csa(fb, twos, twos, ta, tb);
        csa(e, fours, fours, fa, fb);
    } else {
        uint32_t f;
        csa(ta, ones, ones, x[0], x[1]);
        csa(tb, ones, ones, x[2], x[3]);
        csa(f, twos, twos, ta, tb);
        e = fours & f;
        fours ^= f;
    }
    return e;
}

// n of the 32 chains of a bundle as kCountBits bit planes, identical in all
// LAM lanes of the bundle (nqp: the padded plane length).
template <int LAM, bool IND>
__device__ __forceinline__ void recount(const uint32_t* X, const uint32_t* Z, int nqp, int sub,
                                        uint32_t cnt[kCountBits]) {
    uint32_t ones = 0, twos = 0, fours = 0;
    uint32_t hi[kCountBits - 3];
#pragma unroll
    for (int k = 0; k < kCountBits - 3; ++k) hi[k] = 0;
    auto ripple = [&](uint32_t e) {
#pragma unroll
        for (int k = 0; k < kCountBits - 3; ++k) {
            const uint32_t c = hi[k] & e;
            hi[k] ^= e;
            e = c;
        }
    };
    constexpr int STEP = (IND ? 4 : 8) * LAM;
    const int end8 = nqp - nqp % STEP;
    int base = sub;
    for (; base < end8; base += STEP) {
        uint32_t x[8];
        occupancy<LAM, IND>(X, Z, base, x);
        ripple(add_batch<8>(ones, twos, fours, x));
    }
    if constexpr (!IND) {
        if (end8 < nqp) {   // the last 4 LAM qubits
            uint32_t x[4];
            occupancy<LAM, IND, 4>(X, Z, base, x);
            ripple(add_batch<4>(ones, twos, fours, x));
        }
    }
    cnt[0] = ones;
    cnt[1] = twos;
    cnt[2] = fours;
#pragma unroll
    for (int k = 0; k < kCountBits - 3; ++k) cnt[3 + k] = hi[k];
#pragma unroll
    for (int off = 1; off < LAM; off <<= 1) {
        uint32_t carry = 0;
#pragma unroll
        for (int k = 0; k < kCountBits; ++k) {
            const uint32_t o = __shfl_xor_sync(0xffffffffu, cnt[k], off);
            const uint32_t a = cnt[k];
            cnt[k] = a ^ o ^ carry;
            carry = (a & o) | (carry & (a ^ o));
        }
    }
}

__device__ __forceinline__ uint32_t bit_of(const uint32_t cnt[kCountBits], int b) {
    uint32_t n = 0;
#pragma unroll
    for (int k = 0; k < kCountBits; ++k) n |= ((cnt[k] >> b) & 1u) << k;
    return n;
}

// Running per-lane count of occupied qubits, summed over colour phases, in
// carry-save form: value = ones + 2 twos + 4 fours + 8 hi (hi a bit-sliced
// counter of kAccHi planes).  Each lane accumulates only its own slice of the
// qubits; the slices of a bundle's LAM lanes are added together only when the
// accumulator is flushed into the chains' 64-bit sums.
constexpr int kAccHi = 8;
constexpr uint32_t kAccCapacity = 8u * (1u << kAccHi) - 1u;
constexpr int kFlushPlanes = 3 + kAccHi + 5;  // + butterfly growth over <= 32 lanes

struct OccAcc {
    uint32_t ones, twos, fours, hi[kAccHi];
    __device__ __forceinline__ void clear() {
        ones = twos = fours = 0;
#pragma unroll
        for (int k = 0; k < kAccHi; ++k) hi[k] = 0;
    }
};

template <int LAM, bool IND>
__device__ __forceinline__ void accumulate_phase(OccAcc& a, const uint32_t* X, const uint32_t* Z, int nqp, int sub) {
    // ripple the eights into the high planes: the first levels carry for
    // some of the 32 chains nearly every time, so they run untested
    auto ripple = [&](uint32_t e) {
#pragma unroll
        for (int k = 0; k < kAccHi; ++k) {
            if (k >= 3 && !e) break;
            const uint32_t c = a.hi[k] & e;
            a.hi[k] ^= e;
            e = c;
        }
    };
    constexpr int STEP = (IND ? 4 : 8) * LAM;
    const int end8 = nqp - nqp % STEP;
    int base = sub;
    for (; base < end8; base += STEP) {
        uint32_t x[8];
        occupancy<LAM, IND>(X, Z, base, x);
        ripple(add_batch<8>(a.ones, a.twos, a.fours, x));
    }
    if constexpr (!IND) {
        if (end8 < nqp) {   // the last 4 LAM qubits
            uint32_t x[4];
            occupancy<LAM, IND, 4>(X, Z, base, x);
            ripple(add_batch<4>(a.ones, a.twos, a.fours, x));
        }
    }
}

// Adds the accumulated counts of the bundle's LAM lanes (butterfly) and
// credits every owned chain's sum; clears the accumulator.
template <int LAM, typename ChainIndex>
__device__ __forceinline__ void flush_acc(OccAcc& a, int sub, uint32_t valid, uint64_t* sums, ChainIndex ci_of) {
    uint32_t v[kFlushPlanes];
    v[0] = a.ones;
    v[1] = a.twos;
    v[2] = a.fours;
#pragma unroll
    for (int k = 0; k < kAccHi; ++k) v[3 + k] = a.hi[k];
#pragma unroll
    for (int k = 3 + kAccHi; k < kFlushPlanes; ++k) v[k] = 0;
#pragma unroll
    for (int off = 1; off < LAM; off <<= 1) {
        uint32_t carry = 0;
#pragma unroll
        for (int k = 0; k < kFlushPlanes; ++k) {
            const uint32_t o = __shfl_xor_sync(0xffffffffu, v[k], off);
            const uint32_t x = v[k];
            v[k] = x ^ o ^ carry;
            carry = (x & o) | (carry & (x ^ o));
        }
    }
#pragma unroll
    for (int j = 0; j < 32 / LAM; ++j) {
        const int b = sub + j * LAM;
        if (!((valid >> b) & 1u)) continue;
        uint64_t n = 0;
#pragma unroll
        for (int k = 0; k < kFlushPlanes; ++k) n |= (uint64_t)((v[k] >> b) & 1u) << k;
        if (sums) sums[ci_of(b)] += n;
    }
    a.clear();
}

// Planes of one batch.  G = 32: one block per syndrome group, 4 planes per
// block (word i = plane i).  G < 32: 32/G syndromes share a bundle, each
// block holds 128/G planes of G bits; the bundle's plane word takes bits
// [kG, kG+G) of every slot's block and puts slot s at bits [sG, sG+G).
template <int G>
struct PlaneBatch {
    static constexpr int SLOTS = G == 32 ? 1 : 32 / G;
    static constexpr int PPB = G == 32 ? 4 : 128 / G;
    uint32_t pl[PPB];

    __device__ __forceinline__ void make(const SweepParams& p, const uint32_t* sid, uint32_t w, uint32_t t,
                                         uint32_t colm, uint32_t bt) {
        if constexpr (G == 32) {
            const uint4 b = philox10(make_uint4(sid[0], t, colm, (w << 8) | bt), p.rk);
            pl[0] = b.x; pl[1] = b.y; pl[2] = b.z; pl[3] = b.w;
        } else if constexpr (G == 16) {
            merge16(philox10(make_uint4(sid[0], t, colm, bt), p.rk), philox10(make_uint4(sid[1], t, colm, bt), p.rk));
        } else if constexpr (G == 8) {
            uint32_t bw[4][4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint4 b = philox10(make_uint4(sid[s], t, colm, bt), p.rk);
                bw[s][0] = b.x; bw[s][1] = b.y; bw[s][2] = b.z; bw[s][3] = b.w;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int wi = k / 4, by = k % 4;
                const uint32_t sel = (uint32_t)(by | ((4 + by) << 4));
                const uint32_t lo = __byte_perm(bw[0][wi], bw[1][wi], sel);
                const uint32_t hi = __byte_perm(bw[2][wi], bw[3][wi], sel);
                pl[k] = __byte_perm(lo, hi, 0x5410);
            }
        } else {  // G == 4
            uint32_t bw[8][4];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const uint4 b = philox10(make_uint4(sid[s], t, colm, bt), p.rk);
                bw[s][0] = b.x; bw[s][1] = b.y; bw[s][2] = b.z; bw[s][3] = b.w;
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int wi = k / 8, sh = 4 * (k % 8);
                uint32_t v = 0;
#pragma unroll
                for (int s = 0; s < 8; ++s) v |= ((bw[s][wi] >> sh) & 0xFu) << (4 * s);
                pl[k] = v;
            }
        }
    }

    // The same planes for block bt of the head from the bundle's fixed
    // Philox parts (G = 32 and 16; see head_fixed_words: mn = words 0-3,
    // a2 = words 4-5) and the proposal's varying part.
    __device__ __forceinline__ void make_head(const SweepParams& p, const uint4& mn, const uint2& a2,
                                              const PhiloxVarying& v, int bt) {
        static_assert(G >= 16, "fixed Philox parts are kept for plane widths 16 and 32");
        if constexpr (G == 32) {
            const uint4 b = bt == 0 ? philox10_split(mn.x, mn.y, a2.x, v, p.rk)
                                    : philox10_split(mn.z, mn.w, a2.x, v, p.rk);
            pl[0] = b.x; pl[1] = b.y; pl[2] = b.z; pl[3] = b.w;
        } else {
            merge16(philox10_split(mn.x, mn.y, a2.x, v, p.rk), philox10_split(mn.z, mn.w, a2.y, v, p.rk));
        }
    }

    // G = 16: the blocks a and c of the bundle's two syndromes; plane 2i
    // takes the low halves of word i of each (a's in bits 0-15), plane 2i + 1
    // the high halves.
    __device__ __forceinline__ void merge16(const uint4& a, const uint4& c) {
        const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, cw[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            pl[2 * i] = __byte_perm(aw[i], cw[i], 0x5410);
            pl[2 * i + 1] = __byte_perm(aw[i], cw[i], 0x7632);
        }
    }
};

// Fixed Philox parts of a bundle's head blocks (counter words 0 and 3: the
// syndrome id and (w << 8) | bt), kept per bundle in shared memory for plane
// widths 32 and 16: G = 32, one syndrome and head blocks 0 and 1: (M, N) of
// block bt at 2 bt, A at 4; G = 16, two syndromes and head block 0: (M, N)
// of syndrome s at 2 s, A at 4 + s.  Computing them once per bundle instead
// of once per proposal measured 3.6 % faster at G = 32 and 2.5 % at G = 16;
// keeping them for the straggler blocks too ran 7 % slower at G = 32 than
// keeping them for the head only.
constexpr int kHeadFixedWords = 8;

template <int G>
__device__ __forceinline__ void head_fixed_words(const SweepParams& p, const uint32_t* sid, uint32_t w,
                                                 uint32_t* fx) {
    if constexpr (G == 32) {
#pragma unroll
        for (int bt = 0; bt < 2; ++bt) {
            const PhiloxFixed f = philox_fixed(sid[0], (w << 8) | (uint32_t)bt, p.rk);
            fx[2 * bt] = f.M;
            fx[2 * bt + 1] = f.N;
            fx[4] = f.A;
        }
    } else if constexpr (G == 16) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const PhiloxFixed f = philox_fixed(sid[s], 0u, p.rk);
            fx[2 * s] = f.M;
            fx[2 * s + 1] = f.N;
            fx[4 + s] = f.A;
        }
    }
}

// Digit-plane modes of a launch (per quad of planes: 0 every threshold digit
// is 0, 1 only T[1] has nonzero digits, 2 general).  At every temperature the
// decoder meets, the quads after the first two are general, and the first
// two are (0, 1), (1, 2) or (2, 2); those three patterns have kernels of
// their own (HM = 1, 2, 3) with the modes known at compile time, which saves
// the per-quad dispatch in every proposal.  HM = 0 reads the modes from the
// launch parameters.
// Modes of quads 0 and 1 as in SweepParams::qmodes (quad q in bits 2q, 2q+1).
__host__ __device__ constexpr uint32_t head_modes(int hm) {
    return hm == 1 ? 0x4u /* 0, 1 */ : hm == 2 ? 0x9u /* 1, 2 */ : hm == 3 ? 0xAu /* 2, 2 */ : 0u;
}

template <int HM>
__device__ __forceinline__ uint32_t quad_mode(const SweepParams& p, int q) {
    if constexpr (HM == 0) return (p.qmodes >> (2 * q)) & 3u;
    else return q >= 2 ? 2u : (head_modes(HM) >> (2 * q)) & 3u;
}

// The specialised head pattern of a launch's modes (0: none).
__host__ __device__ inline int head_pattern(uint32_t qmodes) {
    if ((qmodes >> 4) != 0xAAAu) return 0;   // quads 2 .. 7 general (mode 2 each)
    for (int hm = 1; hm <= 3; ++hm)
        if ((qmodes & 0xFu) == head_modes(hm)) return hm;
    return 0;
}

// Accept mask of the undecided uphill chains U (all have Delta n = d > 0,
// d - 1 = E0 + 2 E1 bitwise): chains whose u < T[d], deciding with the digit
// planes of batches BT0 .. BT1-1.  U keeps the chains still undecided.  The
// head batches (BT0 = 0) always run in full: some lane of the warp nearly
// always needs them, so an early exit would only add divergence.
template <int G, int BT0, int BT1, int HM = 0>
__device__ __forceinline__ uint32_t bernoulli_range(const SweepParams& p, uint32_t& U, uint32_t E0, uint32_t E1,
                                                    const uint32_t* sid, uint32_t w, uint32_t t, uint32_t colm,
                                                    const uint32_t* fx = nullptr) {
    using PB = PlaneBatch<G>;
    constexpr int PPB = PB::PPB;
    // the head blocks of plane widths 32 and 16 start from the bundle's fixed
    // Philox parts (fx); the counter's varying words are (t, colm)
    constexpr bool kFixed = BT0 == 0 && G >= 16;
    PhiloxVarying pv{};
    uint4 fmn{};
    uint2 fa{};
    if constexpr (kFixed) {
        pv = philox_varying(t, colm, p.rk);
        fmn = *reinterpret_cast<const uint4*>(fx);      // 32-byte aligned
        fa = *reinterpret_cast<const uint2*>(fx + 4);
    }
    const uint32_t E01 = E0 & E1;
    const uint32_t M1 = ~(E0 | E1);  // chains with Delta n = 1
    uint32_t acc = 0;
#pragma unroll
    for (int bt = BT0; bt < BT1; ++bt) {
        PB pb;
        if constexpr (kFixed) pb.make_head(p, fmn, fa, pv, bt);
        else pb.make(p, sid, w, t, colm, (uint32_t)bt);
#pragma unroll
        for (int qd = 0; qd < PPB / 4; ++qd) {
            const int k0 = bt * PPB + 4 * qd;
            const uint32_t mode = quad_mode<HM>(p, k0 / 4);
            if (mode == 0) {
                // every threshold digit is 0 here: a 1 digit rejects
#pragma unroll
                for (int i = 0; i < 4; ++i) U &= ~pb.pl[4 * qd + i];
            } else if (mode == 1) {
                // only T[1] has nonzero digits here
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t r = pb.pl[4 * qd + i];
                    const uint32_t f = p.pc[0][k0 + i] & M1;
                    acc |= U & f & ~r;
                    U &= ~(f ^ r);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = k0 + i;
                    const uint32_t r = pb.pl[4 * qd + i];
                    const uint32_t f = p.pc[0][k] ^ (E0 & p.pc[1][k]) ^ (E1 & p.pc[2][k]) ^ (E01 & p.pc[3][k]);
                    acc |= U & f & ~r;
                    U &= ~(f ^ r);
                }
            }
        }
        if constexpr (BT0 > 0) {
            if (!U) break;
        }
    }
    return acc;
}

// Proposals whose chains are not all decided after the first kHeadPlanes
// digit planes are queued per warp and finished after the colour's inline
// pass by all lanes together, so that one slow proposal does not hold the
// warp's other lanes.
constexpr int kHeadPlanes = 8;
constexpr int kQueueCap = 64;
constexpr int kQueueItem = 5;  // (m | slot << 16), U, E0, E1, accepted so far
constexpr int kMaxSlots = 8;

// Per warp after the frames: queue counter and items, and the bundles' ids.
__host__ __device__ __forceinline__ int warp_aux_words(int bundles) {
    return 1 + kQueueCap * kQueueItem + bundles * (kMaxSlots + 1);
}

// Support of generator g in the syndrome order (sigma_x block row-major over
// (i, j) at grid point (2i+1, 2j), then the sigma_z block at (2i, 2j+1)):
// up, down, left, right neighbours, a missing one replaced by the dummy slot
// (nq for sigma_x generators, nq + 1 for sigma_z).  Returns 0 for sigma_x
// (flips the X plane), 1 for sigma_z.
__device__ __forceinline__ int generator_support(int L, int g, int q[4]) {
    const int nx = L * (L - 1), n = 2 * L - 1, nq = n_qubits(L);
    int r, c, type;
    if (g < nx) {
        const int i = g / L;
        r = 2 * i + 1;
        c = 2 * (g - i * L);
        type = 0;
    } else {
        const int h = g - nx, i = h / (L - 1);
        r = 2 * i;
        c = 2 * (h - i * (L - 1)) + 1;
        type = 1;
    }
    const int dummy = nq + type, base = r * n + c;
    q[0] = r > 0 ? (base - n) / 2 : dummy;
    q[1] = r < n - 1 ? (base + n) / 2 : dummy;
    q[2] = c > 0 ? (base - 1) / 2 : dummy;
    q[3] = c < n - 1 ? (base + 1) / 2 : dummy;
    return type;
}

// One unit: the bundles of group g handled by this block (warps x 32/LAM
// bundles); every warp runs its bundles' chains from gd.t_begin to gd.t_end.
// SCAN (with LAM = 32, one chain per lane): random-scan steps instead of
// colour sweeps, on the same bit-sliced frames.  IND: independent bit and
// phase flips (n = |x| + |z|, every real qubit movable) instead of
// depolarizing noise (n = |x or z|, a qubit movable when its other part is 0).
// Per-lane count of the accepted proposals of its bundle's chains (bit b =
// chain b), bit-sliced over kAcptPlanes planes, kept in shared memory after
// the block's other data; only the instantiations with ACPT = true (one lane
// split, LAM = 32) count, so the common path carries none of it: word k of lane l of warp w at
// base + (w (kAcptPlanes + 1) + k) 32 + l, the lane's increment count at
// k = kAcptPlanes.  Added into the chains' 64-bit counts (atomically: the
// bundle's LAM lanes share them) before it could overflow and at the end.
constexpr int kAcptPlanes = 8;
constexpr uint32_t kAcptCapacity = (1u << kAcptPlanes) - 1u;
constexpr int kAcptWordsPerWarp = (kAcptPlanes + 1) * 32;

__device__ __forceinline__ uint32_t* acpt_words(uint32_t* smem, const SweepParams& p, int lam) {
    const int B = 32 / lam;
    const int warps = blockDim.x >> 5;
    uint32_t* base = smem + 8 * p.grp_nc_max + warps * (B * (kHeadFixedWords + bundle_stride(p.grp_nq_max, lam)) +
                                                        warp_aux_words(B));
    return base + (threadIdx.x >> 5) * kAcptWordsPerWarp + (threadIdx.x & 31);
}

__device__ __forceinline__ void acpt_clear(uint32_t* a) {
#pragma unroll
    for (int k = 0; k <= kAcptPlanes; ++k) a[32 * k] = 0;
}

template <typename ChainIndex>
__device__ __forceinline__ void acpt_flush(uint32_t* a, uint32_t valid, uint64_t* accepts, ChainIndex ci_of) {
    uint32_t pl[kAcptPlanes];
#pragma unroll
    for (int k = 0; k < kAcptPlanes; ++k) pl[k] = a[32 * k];
    for (int b = 0; b < 32; ++b) {
        if (!((valid >> b) & 1u)) continue;
        unsigned long long v = 0;
#pragma unroll
        for (int k = 0; k < kAcptPlanes; ++k) v |= (unsigned long long)((pl[k] >> b) & 1u) << k;
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(accepts + ci_of(b)), v);
    }
    acpt_clear(a);
}

template <typename ChainIndex>
__device__ __forceinline__ void acpt_add(uint32_t* a, uint32_t acc, uint32_t valid, uint64_t* accepts,
                                         ChainIndex ci_of) {
#pragma unroll
    for (int k = 0; k < kAcptPlanes; ++k) {
        if (!acc) break;
        const uint32_t c = a[32 * k] & acc;
        a[32 * k] ^= acc;
        acc = c;
    }
    if (++a[32 * kAcptPlanes] == kAcptCapacity) acpt_flush(a, valid, accepts, ci_of);
}

template <int G, int LAM, bool SCAN, bool IND, bool ACPT, int HM>
__device__ __forceinline__ void run_unit(const SweepParams& p, const GroupDesc& gd, long long unit,
                                         uint32_t* smem, const ushort4* tab) {
    constexpr int B = 32 / LAM;                       // bundles per warp
    constexpr int NJ = 32 / LAM;                      // chains owned per lane
    constexpr int SLOTS = PlaneBatch<G>::SLOTS;
    const int nc = gd.nc, nq = gd.nq, L = gd.L;
    const int nqp = padded_nq(nq, LAM);    // padded plane length; the dummies follow
    const int stride = bundle_stride(nq, LAM);
    uint32_t* fixed = smem + 8 * p.grp_nc_max;   // per bundle: kHeadFixedWords (a multiple of 32 words in all)
    uint32_t* frames = fixed + (blockDim.x >> 5) * B * kHeadFixedWords;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = lane / LAM, sub = lane % LAM;
    const long long bid = (unit * (blockDim.x >> 5) + warp) * B + slot;   // bundle within the group
    const bool active = bid < gd.n_bundles;
    uint32_t* X = frames + (warp * B + slot) * stride;
    uint32_t* Z = X + nqp + 2;
    uint32_t* q_cnt = frames + (blockDim.x >> 5) * B * bundle_stride(p.grp_nq_max, LAM) + warp * warp_aux_words(B);
    uint32_t* q_items = q_cnt + 1;
    uint32_t* binfo = q_items + kQueueCap * kQueueItem;  // per slot: w, sid[SLOTS]

    // Syndromes and chains of the bundle.
    long long syn[SLOTS];
    uint32_t sid[SLOTS];
    uint32_t w = 0, valid = 0;
    // syn[]: the bundle's syndromes as global item indices
    if constexpr (G == 32) {
        syn[0] = gd.item_base + (active ? bid / p.bps : 0);
        w = active ? (uint32_t)(bid % p.bps) : 0;
        sid[0] = p.ids ? p.ids[syn[0]] : p.id0 + (uint32_t)syn[0];
        const int left = p.C - 32 * (int)w;
        valid = !active ? 0u : left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    } else {
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            long long li = bid * SLOTS + s;
            const bool ok = active && li < gd.n;
            if (!ok) li = bid * SLOTS;  // any in-range syndrome; its bits are masked
            if (!active) li = 0;
            syn[s] = gd.item_base + li;
            sid[s] = p.ids ? p.ids[syn[s]] : p.id0 + (uint32_t)syn[s];
            if (ok) valid |= ((1u << p.C) - 1u) << (s * G);
        }
    }
    uint32_t* fx = fixed + (warp * B + slot) * kHeadFixedWords;
    if (sub == 0) {
        binfo[slot * (kMaxSlots + 1)] = w;
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) binfo[slot * (kMaxSlots + 1) + 1 + s] = sid[s];
        head_fixed_words<G>(p, sid, w, fx);
    }
    // chain index and syndrome of bundle bit b
    auto chain_of = [&](int b) -> int { return G == 32 ? 32 * (int)w + b : b % G; };
    auto syn_of = [&](int b) -> long long { return G == 32 ? syn[0] : syn[G == 32 ? 0 : b / G]; };

    // Start state: pure error times the logical that gives chain c the class
    // code c / R (bit 0: X-bar on row 0, bit 1: Z-bar on column 0).
    // (toric code: 4 logical bits X1, X2, Z1, Z2)
    uint32_t lx = 0, lzm = 0, lx2 = 0, lz2 = 0;
    for (int b = 0; b < 32 && !p.init_frames && !p.state_in; ++b) {
        if (!((valid >> b) & 1u)) continue;
        const int k = chain_of(b) / p.R;
        const int l = k ^ p.e0code[syn_of(b)];
        lx |= (uint32_t)(l & 1) << b;
        if (p.code) {
            lx2 |= (uint32_t)((l >> 1) & 1) << b;
            lzm |= (uint32_t)((l >> 2) & 1) << b;
            lz2 |= (uint32_t)((l >> 3) & 1) << b;
        } else {
            lzm |= (uint32_t)((l >> 1) & 1) << b;
        }
    }
    const int W = gd.W;
    // per-item arrays of the group: pure errors and frames are laid out per group
    const uint32_t* e0g = p.e0 ? p.e0 + gd.e0_off - (size_t)gd.item_base * 2 * W : nullptr;
    const uint32_t* ifg = p.init_frames ? p.init_frames + gd.frames_off - (size_t)gd.item_base * p.C * 2 * W
                                        : nullptr;
    uint32_t* cfg = p.chain_frames ? p.chain_frames + gd.frames_off - (size_t)gd.item_base * p.C * 2 * W : nullptr;
    const uint32_t* st_in = p.state_in ? p.state_in + gd.state_off + (size_t)(active ? bid : 0) * 2 * nq : nullptr;
    for (int q = sub; q < nqp; q += LAM) {
        uint32_t xw = 0, zw = 0;
        if (q >= nq) {
            // zero padding
        } else if (st_in) {
            if (active) {
                xw = st_in[q];
                zw = st_in[nq + q];
            }
        } else if (ifg) {
            for (int b = 0; b < 32; ++b) {
                if (!((valid >> b) & 1u)) continue;
                const uint32_t* f = ifg + ((size_t)syn_of(b) * p.C + chain_of(b)) * 2 * W;
                xw |= ((f[q >> 5] >> (q & 31)) & 1u) << b;
                zw |= ((f[W + (q >> 5)] >> (q & 31)) & 1u) << b;
            }
        } else {
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
                const uint32_t vm = G == 32 ? valid : (valid & (((1u << (G & 31)) - 1u) << (s * G)));
                if (!vm) continue;
                const uint32_t* e = e0g + (size_t)syn[s] * 2 * W;
                if ((e[q >> 5] >> (q & 31)) & 1u) xw |= vm;
                if ((e[W + (q >> 5)] >> (q & 31)) & 1u) zw |= vm;
            }
            if (!p.code) {
                if (q < L) xw ^= lx;                  // row-0 qubits: X-bar
                if (q % (2 * L - 1) == 0) zw ^= lzm;  // column-0 qubits: Z-bar
            } else {
                const int r = q / L;
                if (r == 1) xw ^= lx;                       // X1: row 1
                if (q % L == 0 && !(r & 1)) xw ^= lx2;      // X2: column 1, even rows
                if (q % L == 0 && (r & 1)) zw ^= lzm;       // Z1: column 0, odd rows
                if (r == 0) zw ^= lz2;                      // Z2: row 0
            }
        }
        X[q] = xw;
        Z[q] = zw;
    }
    if (sub == 0) {
        X[nqp] = 0u; Z[nqp] = 0xFFFFFFFFu;          // dummy of sigma_x generators
        X[nqp + 1] = 0xFFFFFFFFu; Z[nqp + 1] = 0u;  // dummy of sigma_z generators
    }
    // Owned chains' sums live in the output array; flushes add to them.
    auto ci_of = [&](int b) -> size_t { return (size_t)syn_of(b) * p.C + chain_of(b); };
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int b = sub + j * LAM;
        if (!((valid >> b) & 1u)) continue;
        const size_t ci = ci_of(b);
        if (p.chain_sum) p.chain_sum[ci] = p.init_sum ? p.init_sum[ci] : 0ull;
    }
    OccAcc occ;
    occ.clear();
    if constexpr (ACPT) acpt_clear(acpt_words(smem, p, LAM));
    const uint32_t qpl = (IND ? 2u : 1u) * (uint32_t)((nq + LAM - 1) / LAM);  // counts per lane and phase
    const uint32_t flush_every = kAccCapacity / qpl;       // phases before the accumulator could overflow
    uint32_t since_flush = 0;
    __syncwarp();

    int scan_n = 0;  // random scan: the lane's chain's n at the end
    if constexpr (SCAN) {
        static_assert(LAM == 32, "random scan runs one chain per lane");
        // Sec. IV as written: each step draws one generator g = floor(w0
        // n_stab / 2^32) and applies it when Delta n <= 0 or w1 < T[Delta n]
        // (Philox counter (id, chain, t, step)); n is summed after every
        // step.  Lane b owns bit b of the bundle's words and flips only it.
        const int b = lane;
        const bool mine = (valid >> b) & 1u;
        const uint32_t bit = 1u << b;
        const uint32_t my_sid = sid[G == 32 ? 0 : b / G];
        const uint32_t chain = (uint32_t)chain_of(b);
        const int ns = geo_nstab(p.code, L);
        // energy of a qubit's Pauli, index x + 2z (I, X, Z, Y): the noise
        // model's table (depolarizing 0 1 1 1, flips 0 1 1 2, general)
        const int E0 = p.energy[0], E1 = p.energy[1], E2 = p.energy[2], E3 = p.energy[3];
        auto energy = [&](uint32_t x, uint32_t z) { return x ? (z ? E3 : E1) : (z ? E2 : E0); };
        int n = 0;
        for (int q = 0; q < nq; ++q) n += energy((X[q] >> b) & 1u, (Z[q] >> b) & 1u);
        uint64_t sum = 0, n_acc = 0;
        const int n_x = p.code ? L * L : L * (L - 1);   // sigma_x generators come first
        for (uint32_t t = gd.t_begin; t < gd.t_end; ++t) {
            const bool sample = t >= gd.burn_in;
            for (int step = 0; step < ns; ++step) {
                const uint4 r = philox10(make_uint4(my_sid, chain, t, (uint32_t)step), p.rk);
                const int g = (int)__umulhi(r.x, (uint32_t)ns);
                const ushort4 sp = tab[g];
                const int q[4] = {sp.x, sp.y, sp.z, sp.w};
                const int type = g >= n_x;
                uint32_t* own = type == 0 ? X : Z;
                const uint32_t* oth = type == 0 ? Z : X;
                int dn = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (q[k] >= nq) continue;  // dummy slot of a weight-3 generator
                    const uint32_t o = (own[q[k]] >> b) & 1u, t2 = (oth[q[k]] >> b) & 1u;
                    dn += type == 0 ? energy(o ^ 1u, t2) - energy(o, t2) : energy(t2, o ^ 1u) - energy(t2, o);
                }
                if (mine && (dn <= 0 || (uint64_t)r.y < p.T[dn])) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) atomicXor(&own[q[k]], bit);
                    n += dn;
                    ++n_acc;
                }
                if (sample) sum += (uint64_t)n;
            }
        }
        if (mine && p.chain_sum) p.chain_sum[ci_of(b)] += sum;
        if (mine && p.accepts) p.accepts[ci_of(b)] += n_acc;   // one lane per chain
        scan_n = n;
        __syncwarp();
    } else
    for (uint32_t t = gd.t_begin; t < gd.t_end; ++t) {
#pragma unroll 1
        for (int col = 0; col < 4; ++col) {
            uint32_t* own = col < 2 ? X : Z;          // plane the generator flips
            const uint32_t* oth = col < 2 ? Z : X;    // plane it only reads
            const uint32_t colm = (uint32_t)col << 24;
            const ushort4* tc = tab + col * nc;
            constexpr int PPB = PlaneBatch<G>::PPB;
            constexpr int NBATCH = 32 / PPB;
            constexpr int HEAD = kHeadPlanes / PPB > 0 ? kHeadPlanes / PPB : 1;
            if (lane == 0) *q_cnt = 0u;
            __syncwarp();
            if (active) {
                for (int m = sub; m < nc; m += LAM) {
                    const ushort4 sp = tc[m];
                    const uint32_t o0 = own[sp.x], o1 = own[sp.y], o2 = own[sp.z], o3 = own[sp.w];
                    // movable qubits (the flip changes their weight): other part 0
                    // (independent flips: every real qubit; the dummy slot never)
                    const uint32_t m0 = IND ? (sp.x < nq ? ~0u : 0u) : ~oth[sp.x];
                    const uint32_t m1 = IND ? (sp.y < nq ? ~0u : 0u) : ~oth[sp.y];
                    const uint32_t m2 = IND ? (sp.z < nq ? ~0u : 0u) : ~oth[sp.z];
                    const uint32_t m3 = IND ? (sp.w < nq ? ~0u : 0u) : ~oth[sp.w];
                    // W = number of movable qubits, bits w2 w1 w0
                    const uint32_t s3 = m0 ^ m1 ^ m2, c3 = (m0 & m1) | (m2 & (m0 ^ m1));
                    const uint32_t w0 = s3 ^ m3, cc = s3 & m3, w1 = c3 ^ cc, w2 = c3 & cc;
                    // D = number of movable qubits whose error the flip removes
                    const uint32_t d0 = m0 & o0, d1 = m1 & o1, d2 = m2 & o2, d3 = m3 & o3;
                    const uint32_t ds = d0 ^ d1 ^ d2, dc = (d0 & d1) | (d2 & (d0 ^ d1));
                    const uint32_t Z0 = ~(ds | dc | d3), D1 = ~dc & (ds ^ d3);
                    // Delta n = W - 2D > 0  iff  (D = 0, W >= 1) or (D = 1, W >= 3)
                    const uint32_t Wge1 = w0 | w1 | w2, Wge3 = w2 | (w1 & w0);
                    const uint32_t P = (Z0 & Wge1) | (D1 & Wge3);
                    // the kernels with a head pattern on 32-chain planes run only
                    // whole bundles (their launches have a multiple of 32 chains)
                    const uint32_t vmask = (HM != 0 && G == 32) ? 0xFFFFFFFFu : valid;
                    uint32_t acc = ~P & vmask;
                    // (a launch with a head pattern has 0 < T[1] < 2^32: neither flag)
                    if (HM == 0 && p.accept_all) {
                        acc = valid;
                    } else {
                        uint32_t U = P & vmask;
                        if (U && (HM != 0 || !p.reject_all)) {
                            // Delta n - 1 = E0 + 2 E1 on the uphill chains
                            const uint32_t E0 = ~w0, E1 = Z0 & Wge3;
                            const uint32_t cm = colm | (uint32_t)m;
                            acc |= bernoulli_range<G, 0, HEAD, HM>(p, U, E0, E1, sid, w, t, cm, fx);
                            if constexpr (HEAD < NBATCH) {
                                if (U) {
                                    const uint32_t qi = atomicAdd(q_cnt, 1u);
                                    if (qi < (uint32_t)kQueueCap) {
                                        uint32_t* it = q_items + kQueueItem * qi;
                                        it[0] = (uint32_t)m | ((uint32_t)slot << 16);
                                        it[1] = U;
                                        it[2] = E0;
                                        it[3] = E1;
                                        it[4] = acc;
                                        continue;  // flipped after the queue is resolved
                                    }
                                    acc |= bernoulli_range<G, HEAD, NBATCH, HM>(p, U, E0, E1, sid, w, t, cm);
                                }
                            }
                        }
                    }
                    if constexpr (ACPT) acpt_add(acpt_words(smem, p, LAM), acc, valid, p.accepts, ci_of);
                    own[sp.x] = o0 ^ acc;
                    own[sp.y] = o1 ^ acc;
                    own[sp.z] = o2 ^ acc;
                    own[sp.w] = o3 ^ acc;
                }
            }
            __syncwarp();
            if constexpr (HEAD < NBATCH) {
                // Finish the queued proposals, one per lane.
                const uint32_t n_items = min(*q_cnt, (uint32_t)kQueueCap);
                for (uint32_t i = lane; i < n_items; i += 32) {
                    uint32_t* it = q_items + kQueueItem * i;
                    const int qm = (int)(it[0] & 0xFFFFu), qs = (int)(it[0] >> 16);
                    uint32_t U = it[1];
                    uint32_t acc = it[4];
                    const uint32_t* info = binfo + qs * (kMaxSlots + 1);
                    uint32_t qsid[SLOTS];
#pragma unroll
                    for (int s = 0; s < SLOTS; ++s) qsid[s] = info[1 + s];
                    acc |= bernoulli_range<G, HEAD, NBATCH, HM>(p, U, it[2], it[3], qsid, info[0], t,
                                                            colm | (uint32_t)qm);
                    if constexpr (ACPT) it[4] = acc;
                    if (acc) {
                        uint32_t* qx = frames + (warp * B + qs) * stride;
                        uint32_t* qown = col < 2 ? qx : qx + nqp + 2;
                        const ushort4 sp = tc[qm];
                        qown[sp.x] ^= acc;
                        qown[sp.y] ^= acc;
                        qown[sp.z] ^= acc;
                        qown[sp.w] ^= acc;
                    }
                }
                __syncwarp();
                if constexpr (ACPT) {
                    // queued proposals of this bundle: counted by its first lane
                    if (sub == 0 && active)
                        for (uint32_t i = 0; i < n_items; ++i) {
                            const uint32_t* it = q_items + kQueueItem * i;
                            if ((int)(it[0] >> 16) == slot)
                                acpt_add(acpt_words(smem, p, LAM), it[4], valid, p.accepts, ci_of);
                        }
                    __syncwarp();
                }
            }
            if (t >= gd.burn_in) {
                accumulate_phase<LAM, IND>(occ, X, Z, nqp, sub);
                if (++since_flush == flush_every) {
                    flush_acc<LAM>(occ, sub, valid, p.chain_sum, ci_of);
                    since_flush = 0;
                }
                __syncwarp();
            }
        }
    }

    flush_acc<LAM>(occ, sub, valid, p.chain_sum, ci_of);
    if constexpr (ACPT) {
        if (active) acpt_flush(acpt_words(smem, p, LAM), valid, p.accepts, ci_of);
    }
    if (p.state_out && active) {
        uint32_t* st = p.state_out + gd.state_off + (size_t)bid * 2 * nq;
        for (int q = sub; q < nq; q += LAM) {
            st[q] = X[q];
            st[nq + q] = Z[q];
        }
    }
    uint32_t cnt[kCountBits] = {};
    if constexpr (!SCAN) recount<LAM, IND>(X, Z, nqp, sub, cnt);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int b = sub + j * LAM;
        if (!((valid >> b) & 1u)) continue;
        const size_t ci = (size_t)syn_of(b) * p.C + chain_of(b);
        if (p.chain_n) p.chain_n[ci] = SCAN ? scan_n : (int32_t)bit_of(cnt, b);
        if (cfg) {
            uint32_t* f = cfg + ci * 2 * W;
            for (int wi = 0; wi < W; ++wi) {
                uint32_t xw = 0, zw = 0;
                for (int i = 0; i < 32; ++i) {
                    const int q = 32 * wi + i;
                    if (q >= nq) break;
                    xw |= ((X[q] >> b) & 1u) << i;
                    zw |= ((Z[q] >> b) & 1u) << i;
                }
                f[wi] = xw;
                f[W + wi] = zw;
            }
        }
    }
}


// Persistent sweep kernel: a block takes units (the bundles of one group that
// fill its warps) first by its index, then from a queue counter, in the order
// the host arranged (largest work first), and rebuilds the support table in
// shared memory when the group's code size changes.
template <int G, int LAM, bool SCAN, bool IND, bool ACPT, int HM = 0>
__global__ void __launch_bounds__(128, sweep_blocks_per_sm(G)) sweep_kernel(const __grid_constant__ SweepParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ long long s_unit;
    ushort4* tab = reinterpret_cast<ushort4*>(smem);
    int cur = -1;
    for (long long it = 0;; ++it) {
        if (threadIdx.x == 0)
            s_unit = it == 0 ? (long long)blockIdx.x
                             : (long long)gridDim.x + (long long)atomicAdd(p.unit_counter, 1u);
        __syncthreads();
        const long long u = s_unit;
        if (u >= p.total_units) break;
        int g = 0;
        while (g + 1 < p.n_groups && u >= p.grp[g + 1].unit_base) ++g;
        const GroupDesc& gd = p.grp[g];
        if (g != cur) {
            // support table: colour-major for sweeps, syndrome order for
            // random scan (4 nc = n_stab entries either way)
            for (int idx = threadIdx.x; idx < 4 * gd.nc; idx += blockDim.x) {
                int q[4];
                if constexpr (SCAN) {
                    if (p.code) toric_generator_support(gd.L, idx, q);
                    else generator_support(gd.L, idx, q);
                } else {
                    const int col = idx / gd.nc, m = idx - col * gd.nc;
                    if (p.code) toric_colour_support(gd.L, col, m, q);
                    else colour_support(gd.L, col, m, q);
                }
                // dummy slots (nq, nq + 1) sit after the zero-padded planes
                const int nq = gd.nq, shift = padded_nq(nq, LAM) - nq;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (q[k] >= nq) q[k] += shift;
                tab[idx] = make_ushort4((unsigned short)q[0], (unsigned short)q[1], (unsigned short)q[2],
                                        (unsigned short)q[3]);
            }
            cur = g;
            __syncthreads();
        }
        run_unit<G, LAM, SCAN, IND, ACPT, HM>(p, gd, u - gd.unit_base, smem, tab);
        __syncthreads();
        if (!p.unit_counter) break;
    }
}

constexpr int kWarps = 4;

// The dynamic shared-memory limit of one kernel instantiation, raised on
// demand.  The attribute belongs to the current device's context, so the
// limit already set is kept per device, under a lock (contexts on several
// host threads may launch at once).
struct SmemLimit {
    static constexpr int kMaxDevices = 64;
    std::mutex m;
    size_t bytes[kMaxDevices] = {};

    template <typename Kernel>
    cudaError_t ensure(Kernel* k, int dev, size_t smem) {
        if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lock(m);
        if (smem <= bytes[dev]) return cudaSuccess;
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) bytes[dev] = smem;
        return e;
    }
};

template <int G, int LAM, bool SCAN, bool IND, bool ACPT = false, int HM = 0>
static cudaError_t launch_t(const SweepParams& p, cudaStream_t s) {
    const size_t smem = sweep_smem_bytes(p.grp_nq_max, p.grp_nc_max, LAM) +
                        (ACPT ? (size_t)kWarps * kAcptWordsPerWarp * 4 : 0);
    static SmemLimit limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = limit.ensure(sweep_kernel<G, LAM, SCAN, IND, ACPT, HM>, dev, smem);
    if (e != cudaSuccess) return e;
    if (p.total_units == 0) return cudaSuccess;
    long long blocks = p.total_units;
    if (p.unit_counter) {
        // persistent: as many blocks as fit on the device at once
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<G, LAM, SCAN, IND, ACPT, HM>, 32 * kWarps,
                                                              smem);
        if (e != cudaSuccess) return e;
        int bps = per_sm > 0 ? per_sm : 1;
        if (p.max_blocks_per_sm > 0 && p.max_blocks_per_sm < bps) bps = p.max_blocks_per_sm;
        const long long resident = (long long)sms * bps;
        if (blocks > resident) blocks = resident;
        e = cudaMemsetAsync(p.unit_counter, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
    }
    sweep_kernel<G, LAM, SCAN, IND, ACPT, HM><<<(unsigned)blocks, 32 * kWarps, smem, s>>>(p);
    return cudaGetLastError();
}

template <int G, int LAM, bool SCAN, bool IND>
static cudaError_t prepare_t(const SweepParams& p) {
    const size_t smem = sweep_smem_bytes(p.grp_nq_max, p.grp_nc_max, LAM);
    return cudaFuncSetAttribute(sweep_kernel<G, LAM, SCAN, IND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <int G, bool IND>
static cudaError_t prepare_g(const SweepParams& p, int lam) {
    if (p.scan) return lam == 32 ? prepare_t<G, 32, true, IND>(p) : cudaErrorInvalidValue;
    switch (lam) {
        case 2: return prepare_t<G, 2, false, IND>(p);
        case 4: return prepare_t<G, 4, false, IND>(p);
        case 8: return prepare_t<G, 8, false, IND>(p);
        case 16: return prepare_t<G, 16, false, IND>(p);
        case 32: return prepare_t<G, 32, false, IND>(p);
        default: return cudaErrorInvalidValue;
    }
}

template <bool IND>
static cudaError_t prepare_noise(const SweepParams& p, int lam) {
    switch (p.G) {
        case 4: return prepare_g<4, IND>(p, lam);
        case 8: return prepare_g<8, IND>(p, lam);
        case 16: return prepare_g<16, IND>(p, lam);
        case 32: return prepare_g<32, IND>(p, lam);
        default: return cudaErrorInvalidValue;
    }
}

template <int G, bool IND>
static cudaError_t launch_g(const SweepParams& p, int lam, cudaStream_t s) {
    if (p.scan) return lam == 32 ? launch_t<G, 32, true, IND>(p, s) : cudaErrorInvalidValue;
    // colour sweeps that count accepted proposals: one lane split only
    if (p.accepts) return lam == 32 ? launch_t<G, 32, false, IND, true>(p, s) : cudaErrorInvalidValue;
    switch (lam) {
        case 2: return launch_t<G, 2, false, IND>(p, s);
        case 4: return launch_t<G, 4, false, IND>(p, s);
        case 8: return launch_t<G, 8, false, IND>(p, s);
        case 16: return launch_t<G, 16, false, IND>(p, s);
        case 32: return launch_t<G, 32, false, IND>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <bool IND>
static cudaError_t launch_noise(const SweepParams& p, int lam, cudaStream_t s) {
    switch (p.G) {
        case 4: return launch_g<4, IND>(p, lam, s);
        case 8: return launch_g<8, IND>(p, lam, s);
        case 16: return launch_g<16, IND>(p, lam, s);
        case 32: return launch_g<32, IND>(p, lam, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace surfmcmc
