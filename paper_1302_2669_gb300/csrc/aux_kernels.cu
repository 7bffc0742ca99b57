// Syndrome generation, start frames and the per-syndrome decision: the small
// kernels around the sweep kernel.  One thread per syndrome; frames are kept
// as packed bit planes in registers/local memory.
#include "common.cuh"

namespace surfmcmc {

__device__ __forceinline__ int getb(const uint32_t* w, int q) { return (w[q >> 5] >> (q & 31)) & 1; }
__device__ __forceinline__ void flipb(uint32_t* w, int q) { w[q >> 5] ^= 1u << (q & 31); }

// Anticommutation parities of every generator, in syndrome order (sigma_x
// generators first, row-major; then sigma_z generators): a sigma_x generator
// sees the z plane, a sigma_z generator the x plane (Sec. II).
__device__ void write_syndrome(int L, const uint32_t* ex, const uint32_t* ez, uint8_t* out) {
    const int n = 2 * L - 1;
    int g = 0;
    for (int i = 0; i < L - 1; ++i)
        for (int j = 0; j < L; ++j, ++g) {
            const int r = 2 * i + 1, c = 2 * j, base = r * n + c;
            int par = getb(ez, (base - n) / 2) ^ getb(ez, (base + n) / 2);
            if (c > 0) par ^= getb(ez, (base - 1) / 2);
            if (c < n - 1) par ^= getb(ez, (base + 1) / 2);
            out[g] = (uint8_t)par;
        }
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L - 1; ++j, ++g) {
            const int r = 2 * i, c = 2 * j + 1, base = r * n + c;
            int par = getb(ex, (base - 1) / 2) ^ getb(ex, (base + 1) / 2);
            if (r > 0) par ^= getb(ex, (base - n) / 2);
            if (r < n - 1) par ^= getb(ex, (base + n) / 2);
            out[g] = (uint8_t)par;
        }
}

// Class code a + 2b: a = x parity on column 0 (qubits i(2L-1)), b = z parity
// on row 0 (qubits 0..L-1).
__device__ int class_code(int L, const uint32_t* ex, const uint32_t* ez) {
    int a = 0, b = 0;
    for (int i = 0; i < L; ++i) a ^= getb(ex, i * (2 * L - 1));
    for (int j = 0; j < L; ++j) b ^= getb(ez, j);
    return a + 2 * b;
}

__global__ void gen_syndromes_kernel(RoundKeys rk, uint32_t id0, long long n, int L, int noise, uint32_t tau1,
                                     uint32_t tau2, uint32_t tau3, uint8_t* syn, int32_t* true_class) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nq = n_qubits(L), W = n_words(L);
    uint32_t ex[kMaxWords], ez[kMaxWords];
    for (int w = 0; w < W; ++w) ex[w] = ez[w] = 0;
    const uint32_t id = id0 + (uint32_t)i;
    if (noise == 1) {
        // independent flips: qubit q uses words 2 (q mod 2) (bit flip) and
        // 2 (q mod 2) + 1 (phase flip) of block (id, q div 2, 1, 0); tau1 =
        // floor(p 2^32)
        for (int q0 = 0; q0 < nq; q0 += 2) {
            const uint4 b = philox10(make_uint4(id, (uint32_t)(q0 / 2), 1u, 0u), rk);
            if (b.x < tau1) flipb(ex, q0);
            if (b.y < tau1) flipb(ez, q0);
            if (q0 + 1 < nq && b.z < tau1) flipb(ex, q0 + 1);
            if (q0 + 1 < nq && b.w < tau1) flipb(ez, q0 + 1);
        }
        write_syndrome(L, ex, ez, syn + i * n_stabs(L));
        if (true_class) true_class[i] = class_code(L, ex, ez);
        return;
    }
    // depolarizing: domain 0, thresholds tau, 2 tau, 3 tau; general channel:
    // domain 2, thresholds pX, pX + pY, pX + pY + pZ (times 2^32)
    const uint32_t domain = noise == 2 ? 2u : 0u;
    for (int q0 = 0; q0 < nq; q0 += 4) {
        const uint4 b = philox10(make_uint4(id, (uint32_t)(q0 / 4), domain, 0u), rk);
        const uint32_t u[4] = {b.x, b.y, b.z, b.w};
        for (int k = 0; k < 4 && q0 + k < nq; ++k) {
            // X for u < tau, Y for tau <= u < 2 tau, Z for 2 tau <= u < 3 tau
            if (u[k] < tau2) flipb(ex, q0 + k);
            if (u[k] >= tau1 && u[k] < tau3) flipb(ez, q0 + k);
        }
    }
    write_syndrome(L, ex, ez, syn + i * n_stabs(L));
    if (true_class) true_class[i] = class_code(L, ex, ez);
}

// Pure error: a straight string from every anyon to its nearer absorbing
// boundary (Sec. III), s-anyons vertically (z string), p-anyons horizontally
// (x string); ties go up/left.
// Toric code: syndrome of a frame, its 4-bit class code, and the pure error
// (defects of each type paired in syndrome order, first with second, ...;
// a pair joined from the first towards increasing c to the second's
// column, then towards increasing r to its row; sigma_z strings between
// stars, sigma_x strings between plaquettes).
__device__ void write_syndrome_toric(int L, const uint32_t* ex, const uint32_t* ez, uint8_t* out) {
    for (int g = 0; g < 2 * L * L; ++g) {
        int q[4];
        const int type = toric_generator_support(L, g, q);
        const uint32_t* f = type == 0 ? ez : ex;
        out[g] = (uint8_t)(getb(f, q[0]) ^ getb(f, q[1]) ^ getb(f, q[2]) ^ getb(f, q[3]));
    }
}

__device__ int class_code_toric(int L, const uint32_t* ex, const uint32_t* ez) {
    int a1 = 0, a2 = 0, b1 = 0, b2 = 0;
    for (int i = 0; i < L; ++i) {
        a1 ^= getb(ex, t_qidx(L, 2 * i + 1, 0));
        a2 ^= getb(ex, t_qidx(L, 0, 2 * i + 1));
        b1 ^= getb(ez, t_qidx(L, 1, 2 * i));
        b2 ^= getb(ez, t_qidx(L, 2 * i, 1));
    }
    return a1 + 2 * a2 + 4 * b1 + 8 * b2;
}

__device__ void pure_error_toric(int L, const uint8_t* s, uint32_t* ex, uint32_t* ez) {
    const int m = 2 * L;
    for (int type = 0; type < 2; ++type) {
        uint32_t* f = type == 0 ? ez : ex;
        int r0 = -1, c0 = -1;
        for (int h = 0; h < L * L; ++h) {
            if (!s[h + type * L * L]) continue;
            const int r = 2 * (h / L) + type, c = 2 * (h % L) + type;
            if (r0 < 0) {
                r0 = r;
                c0 = c;
                continue;
            }
            for (int cc = c0; cc != c; cc = (cc + 2) % m) flipb(f, t_qidx(L, r0, cc + 1));
            for (int rr = r0; rr != r; rr = (rr + 2) % m) flipb(f, t_qidx(L, rr + 1, c));
            r0 = -1;
        }
    }
}

__global__ void start_frames_toric_kernel(const uint8_t* syn, long long n, int L, uint32_t* frames, int32_t* code) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int W = geo_words(1, L);
    uint32_t ex[kMaxWords], ez[kMaxWords];
    for (int w = 0; w < W; ++w) ex[w] = ez[w] = 0;
    pure_error_toric(L, syn + i * 2 * L * L, ex, ez);
    uint32_t* f = frames + i * 2 * W;
    for (int w = 0; w < W; ++w) {
        f[w] = ex[w];
        f[W + w] = ez[w];
    }
    if (code) code[i] = class_code_toric(L, ex, ez);
}

// Depolarizing errors on the torus: the planar generator's draws per qubit.
__global__ void gen_syndromes_toric_kernel(RoundKeys rk, uint32_t id0, long long n, int L, uint32_t tau1,
                                           uint32_t tau2, uint32_t tau3, uint8_t* syn, int32_t* true_class) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nq = 2 * L * L, W = geo_words(1, L);
    uint32_t ex[kMaxWords], ez[kMaxWords];
    for (int w = 0; w < W; ++w) ex[w] = ez[w] = 0;
    const uint32_t id = id0 + (uint32_t)i;
    for (int q0 = 0; q0 < nq; q0 += 4) {
        const uint4 b = philox10(make_uint4(id, (uint32_t)(q0 / 4), 0u, 0u), rk);
        const uint32_t u[4] = {b.x, b.y, b.z, b.w};
        for (int k = 0; k < 4 && q0 + k < nq; ++k) {
            if (u[k] < tau2) flipb(ex, q0 + k);
            if (u[k] >= tau1 && u[k] < tau3) flipb(ez, q0 + k);
        }
    }
    write_syndrome_toric(L, ex, ez, syn + i * 2 * L * L);
    if (true_class) true_class[i] = class_code_toric(L, ex, ez);
}

cudaError_t launch_gen_syndromes_toric(uint64_t seed, uint32_t id0, long long n, int L, double p, uint8_t* syn,
                                       int32_t* true_class, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    RoundKeys rk;
    make_round_keys((uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x53594E44u, &rk);
    const uint64_t tau = (uint64_t)floor((p / 3.0) * 4294967296.0);
    gen_syndromes_toric_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(rk, id0, n, L, (uint32_t)tau,
                                                                           (uint32_t)(2 * tau), (uint32_t)(3 * tau),
                                                                           syn, true_class);
    return cudaGetLastError();
}

__global__ void start_frames_kernel(const uint8_t* syn, long long n, int L, uint32_t* frames, int32_t* code) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int W = n_words(L), n2 = 2 * L - 1;
    uint32_t ex[kMaxWords], ez[kMaxWords];
    for (int w = 0; w < W; ++w) ex[w] = ez[w] = 0;
    const uint8_t* s = syn + i * n_stabs(L);
    int g = 0;
    for (int a = 0; a < L - 1; ++a)
        for (int b = 0; b < L; ++b, ++g) {
            if (!s[g]) continue;
            const int r = 2 * a + 1, c = 2 * b;
            if ((r + 1) / 2 <= L - (r + 1) / 2)
                for (int rr = r - 1; rr >= 0; rr -= 2) flipb(ez, (rr * n2 + c) / 2);
            else
                for (int rr = r + 1; rr < n2; rr += 2) flipb(ez, (rr * n2 + c) / 2);
        }
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < L - 1; ++b, ++g) {
            if (!s[g]) continue;
            const int r = 2 * a, c = 2 * b + 1;
            if ((c + 1) / 2 <= L - (c + 1) / 2)
                for (int cc = c - 1; cc >= 0; cc -= 2) flipb(ex, (r * n2 + cc) / 2);
            else
                for (int cc = c + 1; cc < n2; cc += 2) flipb(ex, (r * n2 + cc) / 2);
        }
    uint32_t* f = frames + i * 2 * W;
    for (int w = 0; w < W; ++w) {
        f[w] = ex[w];
        f[W + w] = ez[w];
    }
    if (code) code[i] = class_code(L, ex, ez);
}

// Sec. IV.A decision: S_k = sum over the R chains of class k; the class with
// the smallest S_k (lowest k on ties); log-ratio proxy -beta_bar (<n>_k -
// <n>_best) in double precision.
__global__ void decide_kernel(DecideParams p) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const uint64_t* cs = p.chain_sum + i * p.K * p.R;
    uint64_t S[16];
    int best = 0;
    for (int k = 0; k < p.K; ++k) {
        uint64_t s = 0;
        for (int r = 0; r < p.R; ++r) s += cs[k * p.R + r];
        S[k] = s;
        if (s < S[best]) best = k;
    }
    const long long o = p.perm ? p.perm[i] : i;  // caller's index of internal item i
    const uint64_t samples = p.samples_per_item ? p.samples_per_item[i] : p.samples;
    p.out_class[o] = best;
    if (p.out_class_sum)
        for (int k = 0; k < p.K; ++k) p.out_class_sum[o * p.K + k] = S[k];
    if (p.out_log_ratio)
        for (int k = 0; k < p.K; ++k) {
            double v = 0.0;
            if (samples) {
                const double mk = (double)S[k] / (double)samples;
                const double mb = (double)S[best] / (double)samples;
                v = -p.beta_bar * (mk - mb);
            }
            p.out_log_ratio[o * p.K + k] = v;
        }
}

// <n>_{beta_j,k} of every syndrome from the chain sums of the run at grid
// point j: mean[i][k][j] = S_k / samples.
__global__ void class_means_kernel(long long n, int K, int R, int N, int j, uint64_t samples,
                                   const uint64_t* chain_sum, double* mean) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < K; ++k) {
        uint64_t S = 0;
        for (int r = 0; r < R; ++r) S += chain_sum[(i * K + k) * R + r];
        mean[(i * K + k) * N + j] = (double)S / (double)samples;
    }
}

// Eq. 6 by the composite Simpson rule over the N grid points (<n> at beta = 0
// is 3/4 n_q, Sec. IV.A): I_k = h/3 sum_j w_j <n>_{beta_j,k}, w = 1 4 2 .. 4 1;
// the class with the smallest I_k (largest Z_k) wins, lowest k on ties;
// log_z[k] = -(I_k - I_best).  Explicit round-to-nearest operations keep the
// summation order and rounding of the plain definition.
__global__ void ti_decide_kernel(long long n, int K, int N, double mean0, double h3, double* mean,
                                 int32_t* out_class, double* out_log_z) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double I[16];
    int best = 0;
    for (int k = 0; k < K; ++k) {
        double* m = mean + (i * K + k) * N;
        m[0] = mean0;
        double acc = 0.0;
        for (int j = 0; j < N; ++j) {
            const double w = (j == 0 || j == N - 1) ? 1.0 : ((j & 1) ? 4.0 : 2.0);
            acc = __dadd_rn(acc, __dmul_rn(w, m[j]));
        }
        I[k] = __dmul_rn(acc, h3);
        if (I[k] < I[best]) best = k;
    }
    out_class[i] = best;
    if (out_log_z)
        for (int k = 0; k < K; ++k) out_log_z[i * K + k] = -__dsub_rn(I[k], I[best]);
}

// Ragged batches: copies the caller's syndrome rows (item perm[i] of the
// input) into group order and sets the internal ids.
__global__ void gather_rows_kernel(long long n, const uint8_t* src, const long long* src_off, const long long* dst_off,
                                   const int32_t* len, const long long* perm, const uint32_t* ids, uint32_t id0,
                                   uint8_t* dst, uint32_t* ids_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint8_t* a = src + src_off[perm[i]];
    uint8_t* b = dst + dst_off[i];
    for (int k = 0; k < len[i]; ++k) b[k] = a[k];
    ids_out[i] = ids ? ids[perm[i]] : id0 + (uint32_t)perm[i];
}

// Early stop, after a chunk of sweeps: item i of the active set (caller's
// index perm[i]) retires when this is the last checkpoint, or when the
// network is confident (log p of its argmax exceeds every other class's by
// more than tau) and its argmax equals the chains' current decision.  A
// retiring item writes its decision, class sums and sweep count.
__global__ void retire_kernel(long long n, const long long* perm, const float* logprob, const int32_t* cls,
                              const uint64_t* class_sum, float tau, uint32_t sweeps, int final_chunk,
                              int32_t* out_class, uint64_t* out_class_sum, uint32_t* out_sweeps, int32_t* keep) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long o = perm[i];
    int am = 0;
    float lp[4];
    for (int k = 0; k < 4; ++k) {
        lp[k] = logprob[o * 4 + k];
        if (lp[k] > lp[am]) am = k;
    }
    float second = -INFINITY;
    for (int k = 0; k < 4; ++k)
        if (k != am && lp[k] > second) second = lp[k];
    const bool retire = final_chunk || (lp[am] - second > tau && am == cls[i]);
    keep[i] = retire ? 0 : 1;
    if (!retire) return;
    out_class[o] = cls[i];
    if (out_class_sum)
        for (int k = 0; k < 4; ++k) out_class_sum[o * 4 + k] = class_sum[i * 4 + k];
    if (out_sweeps) out_sweeps[o] = sweeps;
}

// Exclusive prefix sum of keep[0..n) into pos, total into *count (one block
// of 1024 threads: each thread scans a contiguous run, then the run totals
// are scanned in shared memory).
__global__ void scan_keep_kernel(long long n, const int32_t* keep, long long* pos, long long* count) {
    __shared__ long long tot[1024];
    const int t = threadIdx.x;
    const long long per = (n + 1023) / 1024;
    const long long a = t * per, b = a + per < n ? a + per : n;
    long long s = 0;
    for (long long i = a; i < b; ++i) s += keep[i];
    tot[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const long long v = t >= off ? tot[t - off] : 0;
        __syncthreads();
        tot[t] += v;
        __syncthreads();
    }
    long long run = tot[t] - s;  // exclusive start of this thread's run
    for (long long i = a; i < b; ++i) {
        pos[i] = run;
        run += keep[i];
    }
    if (t == 1023) *count = tot[1023];
}

// Moves the kept items' per-item rows to their compacted positions: the
// caller's index, the chain ids, the per-chain frames and sums.
__global__ void compact_kernel(long long n, const int32_t* keep, const long long* pos, const long long* perm,
                               uint32_t id0, int frame_words, int chains, const uint32_t* frames,
                               const uint64_t* sums, long long* perm_out, uint32_t* ids_out, uint32_t* frames_out,
                               uint64_t* sums_out) {
    const long long i = blockIdx.x;
    if (i >= n || !keep[i]) return;
    const long long j = pos[i];
    if (threadIdx.x == 0) {
        perm_out[j] = perm[i];
        ids_out[j] = id0 + (uint32_t)perm[i];
    }
    for (int w = threadIdx.x; w < frame_words; w += blockDim.x)
        frames_out[j * frame_words + w] = frames[i * frame_words + w];
    for (int c = threadIdx.x; c < chains; c += blockDim.x) sums_out[j * chains + c] = sums[i * chains + c];
}

// Budget reordering of an early-stopped decode (at its first checkpoint):
// for active item i (caller's index perm[i]) the network's classes ranked by
// log-probability, highest first, ties to the lower class: a, b, c, d.  The
// chains of c and d continue as further replicas of a and b: slot c R + r
// takes the frame of slot a R + r and slot d R + r that of b R + r, their
// sums restart from 0, and the class sums of c and d so far are frozen.
// rank[o] = a | b << 2 | c << 4 | d << 6, frozen[o] = (S_c, S_d).  One warp
// per item.
__global__ void reorder_kernel(long long n, const long long* perm, const float* logprob, int R, int chain_words,
                               uint32_t* frames, uint64_t* sums, uint8_t* rank, uint64_t* frozen) {
    const long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const long long o = perm[i];
    int ord[4] = {0, 1, 2, 3};
    float lp[4];
    for (int k = 0; k < 4; ++k) lp[k] = logprob[o * 4 + k];
    for (int x = 1; x < 4; ++x)          // insertion sort, stable: ties keep the lower class first
        for (int y = x; y > 0 && lp[ord[y]] > lp[ord[y - 1]]; --y) {
            const int t = ord[y];
            ord[y] = ord[y - 1];
            ord[y - 1] = t;
        }
    const int C = 4 * R;
    uint64_t* cs = sums + i * C;
    uint32_t* fr = frames + i * (long long)C * chain_words;
    if (lane == 0) {
        uint64_t sc = 0, sd = 0;
        for (int r = 0; r < R; ++r) {
            sc += cs[ord[2] * R + r];
            sd += cs[ord[3] * R + r];
        }
        frozen[o * 2 + 0] = sc;
        frozen[o * 2 + 1] = sd;
        rank[o] = (uint8_t)(ord[0] | ord[1] << 2 | ord[2] << 4 | ord[3] << 6);
    }
    __syncwarp();
    for (int r = 0; r < R; ++r)
        for (int h = 0; h < 2; ++h) {
            const uint32_t* src = fr + (long long)(ord[h] * R + r) * chain_words;
            uint32_t* dst = fr + (long long)(ord[h + 2] * R + r) * chain_words;
            for (int w = lane; w < chain_words; w += 32) dst[w] = src[w];
        }
    __syncwarp();
    for (int j = lane; j < 2 * R; j += 32) cs[ord[2 + j / R] * R + j % R] = 0;
}

// a * b < c * d for 64-bit unsigned operands (128-bit products).
__device__ __forceinline__ bool prod_less(uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    const uint64_t h1 = __umul64hi(a, b), h2 = __umul64hi(c, d);
    return h1 < h2 || (h1 == h2 && a * b < c * d);
}

// Decision of a reordered item: class sums S_a, S_b over the class's own and
// its further replicas' chains (n_top samples each), S_c, S_d the frozen sums
// (n_low samples each); the class with the smallest mean S_k / N_k wins,
// compared exactly (S_k N_j < S_j N_k), lowest class on ties.
__global__ void decide_reorder_kernel(long long n, const long long* perm, const uint8_t* rank, const uint64_t* frozen,
                                      int R, const uint64_t* chain_sum, uint64_t n_top, uint64_t n_low,
                                      int32_t* out_class, uint64_t* out_class_sum) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long o = perm[i];
    const int rk = rank[o];
    const int a = rk & 3, b = (rk >> 2) & 3, c = (rk >> 4) & 3, d = (rk >> 6) & 3;
    const uint64_t* cs = chain_sum + i * 4 * R;
    uint64_t S[4], N[4];
    S[a] = 0;
    S[b] = 0;
    for (int r = 0; r < R; ++r) {
        S[a] += cs[a * R + r] + cs[c * R + r];
        S[b] += cs[b * R + r] + cs[d * R + r];
    }
    S[c] = frozen[o * 2 + 0];
    S[d] = frozen[o * 2 + 1];
    N[a] = N[b] = n_top;
    N[c] = N[d] = n_low;
    int best = 0;
    for (int k = 1; k < 4; ++k)
        if (prod_less(S[k], N[best], S[best], N[k])) best = k;
    out_class[i] = best;
    for (int k = 0; k < 4; ++k) out_class_sum[i * 4 + k] = S[k];
}

__global__ void iota_kernel(long long n, long long* perm) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = i;
}

cudaError_t launch_iota(long long n, long long* perm, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    iota_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, perm);
    return cudaGetLastError();
}

cudaError_t launch_gen_syndromes_pauli(uint64_t seed, uint32_t id0, long long n, int L, double px, double py,
                                       double pz, uint8_t* syn, int32_t* true_class, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    RoundKeys rk;
    make_round_keys((uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x53594E44u, &rk);
    const uint64_t t1 = (uint64_t)floor(px * 4294967296.0);
    const uint64_t t2 = (uint64_t)floor((px + py) * 4294967296.0);
    const uint64_t t3 = (uint64_t)floor((px + py + pz) * 4294967296.0);
    const int bs = 128;
    gen_syndromes_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(rk, id0, n, L, 2, (uint32_t)t1, (uint32_t)t2,
                                                                      (uint32_t)t3, syn, true_class);
    return cudaGetLastError();
}

cudaError_t launch_retire(long long n, const long long* perm, const float* logprob, const int32_t* cls,
                          const uint64_t* class_sum, float tau, uint32_t sweeps, int final_chunk, int32_t* out_class,
                          uint64_t* out_class_sum, uint32_t* out_sweeps, int32_t* keep, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    retire_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, perm, logprob, cls, class_sum, tau, sweeps,
                                                              final_chunk, out_class, out_class_sum, out_sweeps, keep);
    return cudaGetLastError();
}

cudaError_t launch_compact(long long n, const int32_t* keep, long long* pos, long long* count, const long long* perm,
                           uint32_t id0, int frame_words, int chains, const uint32_t* frames, const uint64_t* sums,
                           long long* perm_out, uint32_t* ids_out, uint32_t* frames_out, uint64_t* sums_out,
                           cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    scan_keep_kernel<<<1, 1024, 0, s>>>(n, keep, pos, count);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    compact_kernel<<<(unsigned)n, 128, 0, s>>>(n, keep, pos, perm, id0, frame_words, chains, frames, sums, perm_out,
                                               ids_out, frames_out, sums_out);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(long long n, const uint8_t* src, const long long* src_off, const long long* dst_off,
                               const int32_t* len, const long long* perm, const uint32_t* ids, uint32_t id0,
                               uint8_t* dst, uint32_t* ids_out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    gather_rows_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, src, src_off, dst_off, len, perm, ids, id0, dst,
                                                                   ids_out);
    return cudaGetLastError();
}

cudaError_t launch_class_means(long long n, int K, int R, int N, int j, uint64_t samples, const uint64_t* chain_sum,
                               double* mean, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    class_means_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, K, R, N, j, samples, chain_sum, mean);
    return cudaGetLastError();
}

cudaError_t launch_ti_decide(long long n, int K, int N, double mean0, double h3, double* mean, int32_t* out_class,
                             double* out_log_z, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    ti_decide_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, K, N, mean0, h3, mean, out_class, out_log_z);
    return cudaGetLastError();
}

cudaError_t launch_gen_syndromes(uint64_t seed, uint32_t id0, long long n, int L, double p, uint8_t* syn,
                                 int32_t* true_class, cudaStream_t s, int noise) {
    if (n == 0) return cudaSuccess;
    RoundKeys rk;
    make_round_keys((uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x53594E44u, &rk);
    const uint64_t tau = noise ? (uint64_t)floor(p * 4294967296.0) : (uint64_t)floor((p / 3.0) * 4294967296.0);
    const int bs = 128;
    gen_syndromes_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(rk, id0, n, L, noise, (uint32_t)tau,
                                                                      (uint32_t)(2 * tau), (uint32_t)(3 * tau),
                                                                      syn, true_class);
    return cudaGetLastError();
}

cudaError_t launch_start_frames(const uint8_t* syn, long long n, int L, uint32_t* frames, int32_t* code,
                                cudaStream_t s, int toric) {
    if (n == 0) return cudaSuccess;
    const int bs = 128;
    if (toric)
        start_frames_toric_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(syn, n, L, frames, code);
    else
        start_frames_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(syn, n, L, frames, code);
    return cudaGetLastError();
}

cudaError_t launch_reorder(long long n, const long long* perm, const float* logprob, int R, int chain_words,
                           uint32_t* frames, uint64_t* sums, uint8_t* rank, uint64_t* frozen, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    reorder_kernel<<<(unsigned)((n + 3) / 4), 128, 0, s>>>(n, perm, logprob, R, chain_words, frames, sums, rank,
                                                           frozen);
    return cudaGetLastError();
}

cudaError_t launch_decide_reorder(long long n, const long long* perm, const uint8_t* rank, const uint64_t* frozen,
                                  int R, const uint64_t* chain_sum, uint64_t n_top, uint64_t n_low, int32_t* out_class,
                                  uint64_t* out_class_sum, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    decide_reorder_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, perm, rank, frozen, R, chain_sum, n_top,
                                                                      n_low, out_class, out_class_sum);
    return cudaGetLastError();
}

cudaError_t launch_decide(const DecideParams& p, cudaStream_t s) {
    if (p.n == 0) return cudaSuccess;
    const int bs = 128;
    decide_kernel<<<(unsigned)((p.n + bs - 1) / bs), bs, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace surfmcmc
