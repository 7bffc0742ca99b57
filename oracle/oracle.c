/*
 * CPU ORACLE for the single-temperature Markov chain Monte Carlo decoder of the
 * planar surface code (Hutter, Wootton, Loss, "An efficient Markov chain Monte
 * Carlo algorithm for the surface code", arXiv:1302.2669).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct
 * restatement of what the decoder computes, used only by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg.  It shares no code,
 * header, table or helper with the CUDA library and must never be linked into
 * the product path.
 *
 * Representation: one byte per data qubit for the x part and one for the z
 * part of a Pauli frame (Y = x and z), plain loops everywhere, integers for
 * every decision.  Each function cites the passage of the paper it restates.
 *
 * Readings taken where the paper is silent (each is listed with its reason in
 * the design notes of the repository):
 *   - Geometry of the missing Fig. 1: unrotated planar layout on a
 *     (2L-1)x(2L-1) grid; data qubits at r+c even, sigma_x ("star",
 *     s-anyon) generators at (odd r, even c), sigma_z ("plaquette",
 *     p-anyon) generators at (even r, odd c).  This gives the counts of
 *     Sec. II: n_stab = 2L(L-1) generators of weight 3 or 4 and
 *     n_qubits = n_stab + 1.
 *   - Start state: instead of enhanced MWPM (Sec. III, needs Blossom V) each
 *     anyon is joined by a straight string to its nearer absorbing boundary
 *     (s-anyons: top/bottom, p-anyons: left/right, Sec. III), and class k
 *     multiplies that pure error by a logical operator.  Optionally the
 *     burn-in anneals these starts from a higher temperature down to beta*
 *     (see orc_anneal_scale), standing in for the low-energy starts of
 *     Sec. IV.
 *   - Sweep: the four non-overlapping groups of Sec. V become four colours of
 *     generators; a sweep proposes every generator once, colour by colour.
 *   - n is sampled after every colour phase (one "group step" of Sec. V).
 *   - Randomness: Philox4x32-10 (Salmon et al., SC'11), counter indexed; a
 *     uniform 32-bit u per chain and proposal, assembled from "bit planes"
 *     (see chain_uniform_less below).  Acceptance of Delta n > 0 iff
 *     u < T[Delta n], T[d] = floor(r^d 2^32), r = e^{-beta*} (Eq. 2).
 *   - Decision: argmin over classes of the integer sum of sampled n
 *     (Sec. IV.A, "performing error correction in accordance with the
 *     equivalence class E for which this value is smallest"), lowest class
 *     on ties.
 *   - Class index k is the absolute class code a + 2b of a frame, where a is
 *     the parity of x on the column-0 qubits (the support of the logical
 *     Z-bar) and b the parity of z on the row-0 qubits (support of X-bar);
 *     Sec. II identifies classes by such parities.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_L 64

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. II, Fig. 1 as read above)                                  */
/* ------------------------------------------------------------------------ */

int orc_nq(int L) { return 2 * L * L - 2 * L + 1; }     /* n_stab + 1, Sec. IV.A */
int orc_nstab(int L) { return 2 * L * (L - 1); }         /* Sec. II */

static int qidx(int L, int r, int c) { return (r * (2 * L - 1) + c) / 2; }
static int in_grid(int L, int r, int c) { return r >= 0 && c >= 0 && r <= 2 * L - 2 && c <= 2 * L - 2; }

/* Grid position of stabilizer generator number g in the syndrome layout:
 * first the sigma_x generators row-major over (i, j), i < L-1, j < L, at grid
 * point (2i+1, 2j); then the sigma_z generators row-major over (i, j), i < L,
 * j < L-1, at grid point (2i, 2j+1).  Returns 0 for sigma_x, 1 for sigma_z. */
int orc_stab_pos(int L, int g, int* r, int* c)
{
    int nx = (L - 1) * L;
    if (g < nx) {
        *r = 2 * (g / L) + 1;
        *c = 2 * (g % L);
        return 0;
    }
    g -= nx;
    *r = 2 * (g / (L - 1));
    *c = 2 * (g % (L - 1)) + 1;
    return 1;
}

/* Support of generator g: the data qubits among the four grid neighbours
 * (3 on a boundary, 4 inside, Sec. II).  Returns the weight. */
int orc_stab_support(int L, int g, int32_t* q)
{
    int r, c, w = 0;
    orc_stab_pos(L, g, &r, &c);
    const int dr[4] = {-1, 1, 0, 0};
    const int dc[4] = {0, 0, -1, 1};
    for (int k = 0; k < 4; ++k)
        if (in_grid(L, r + dr[k], c + dc[k])) q[w++] = qidx(L, r + dr[k], c + dc[k]);
    return w;
}

/* Colour of generator g (the four groups of Sec. V): sigma_x generators with
 * (i+j) even -> 0, odd -> 1; sigma_z generators with (i+j) even -> 2, odd -> 3. */
int orc_stab_colour(int L, int g)
{
    int r, c;
    int type = orc_stab_pos(L, g, &r, &c);
    int i, j;
    if (type == 0) { i = (r - 1) / 2; j = c / 2; }
    else { i = r / 2; j = (c - 1) / 2; }
    return 2 * type + ((i + j) & 1);
}

/* Number of generators of a colour, and the m-th generator of a colour in
 * syndrome-layout order (row-major within each type).  Plain enumeration. */
int orc_colour_count(int L, int col)
{
    int n = 0;
    for (int g = 0; g < orc_nstab(L); ++g) n += orc_stab_colour(L, g) == col;
    return n;
}
int orc_colour_member(int L, int col, int m)
{
    for (int g = 0; g < orc_nstab(L); ++g)
        if (orc_stab_colour(L, g) == col && m-- == 0) return g;
    return -1;
}

/* Syndrome of a frame: a sigma_x generator is violated (s-anyon) when it
 * anticommutes with the error, i.e. odd overlap with the z part; a sigma_z
 * generator (p-anyon) when the overlap with the x part is odd (Sec. II). */
void orc_syndrome(int L, const uint8_t* ex, const uint8_t* ez, uint8_t* syn)
{
    int32_t q[4];
    for (int g = 0; g < orc_nstab(L); ++g) {
        int r, c;
        int type = orc_stab_pos(L, g, &r, &c);
        int w = orc_stab_support(L, g, q);
        int par = 0;
        for (int k = 0; k < w; ++k) par ^= type == 0 ? ez[q[k]] : ex[q[k]];
        syn[g] = (uint8_t)par;
    }
}

/* Class code of a frame: a = parity of x on column 0 (support of Z-bar),
 * b = parity of z on row 0 (support of X-bar); code = a + 2b.  Applying a
 * stabilizer generator never changes it (Sec. II: the classes are told apart
 * by the error parity along a line joining two opposite boundaries). */
int orc_class_code(int L, const uint8_t* ex, const uint8_t* ez)
{
    int a = 0, b = 0;
    for (int i = 0; i < L; ++i) a ^= ex[qidx(L, 2 * i, 0)];
    for (int j = 0; j < L; ++j) b ^= ez[qidx(L, 0, 2 * j)];
    return a + 2 * b;
}

/* Multiply a frame by the logical L_k: bit 0 of k applies X-bar = sigma_x on
 * row 0, bit 1 applies Z-bar = sigma_z on column 0. */
void orc_apply_logical(int L, int k, uint8_t* ex, uint8_t* ez)
{
    if (k & 1)
        for (int j = 0; j < L; ++j) ex[qidx(L, 0, 2 * j)] ^= 1;
    if (k & 2)
        for (int i = 0; i < L; ++i) ez[qidx(L, 2 * i, 0)] ^= 1;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two      */
/* 32x32->64 multiplications with the published multipliers and Weyl key     */
/* increments.                                                               */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t* ctr_in, const uint32_t* key_in, uint32_t* out)
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* ------------------------------------------------------------------------ */
/* Synthetic syndromes: i.i.d. depolarizing noise (Eq. 1 with p_x = p_y =    */
/* p_z = p/3, Sec. II).                                                      */
/* ------------------------------------------------------------------------ */

/* Error of syndrome number `id`: qubit q draws word (q mod 4) of the Philox
 * block with counter (id, q div 4, 0, 0) and key (seed_lo, seed_hi ^
 * 0x53594E44); with tau = floor((p/3) 2^32): u < tau -> X, u < 2 tau -> Y,
 * u < 3 tau -> Z, otherwise no error. */
void orc_gen_error(uint64_t seed, uint32_t id, int L, double p, uint8_t* ex, uint8_t* ez)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x53594E44u};
    uint64_t tau = (uint64_t)floor((p / 3.0) * 4294967296.0);
    uint32_t blk[4];
    for (int q = 0; q < orc_nq(L); ++q) {
        uint32_t ctr[4] = {id, (uint32_t)(q / 4), 0, 0};
        orc_philox4x32_10(ctr, key, blk);
        uint64_t u = blk[q % 4];
        int x = 0, z = 0;
        if (u < tau) x = 1;
        else if (u < 2 * tau) { x = 1; z = 1; }
        else if (u < 3 * tau) z = 1;
        ex[q] = (uint8_t)x;
        ez[q] = (uint8_t)z;
    }
}

/* Independent bit and phase flips (Sec. IV.B): sigma_x on each qubit with
 * probability p and, independently, sigma_z with probability p.  tau =
 * floor(p 2^32); qubit q uses words 2 (q mod 2) (bit flip) and 2 (q mod 2) + 1
 * (phase flip) of the block with counter (id, q div 2, 1, 0). */
void orc_gen_error_flips(uint64_t seed, uint32_t id, int L, double p, uint8_t* ex, uint8_t* ez)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x53594E44u};
    uint64_t tau = (uint64_t)floor(p * 4294967296.0);
    uint32_t blk[4];
    for (int q = 0; q < orc_nq(L); ++q) {
        uint32_t ctr[4] = {id, (uint32_t)(q / 2), 1, 0};
        orc_philox4x32_10(ctr, key, blk);
        ex[q] = (uint8_t)((uint64_t)blk[2 * (q % 2)] < tau);
        ez[q] = (uint8_t)((uint64_t)blk[2 * (q % 2) + 1] < tau);
    }
}

/* n syndromes with ids id0 .. id0+n-1; true_class gets the class code of the
 * sampled error (the class a perfect decoder must return).  noise 0:
 * depolarizing, 1: independent bit and phase flips. */
void orc_gen_syndromes_noise(uint64_t seed, uint32_t id0, int64_t n, int L, double p, int noise,
                             uint8_t* syn, int32_t* true_class)
{
    int nq = orc_nq(L), ns = orc_nstab(L);
    uint8_t* ex = malloc(nq);
    uint8_t* ez = malloc(nq);
    for (int64_t i = 0; i < n; ++i) {
        if (noise) orc_gen_error_flips(seed, id0 + (uint32_t)i, L, p, ex, ez);
        else orc_gen_error(seed, id0 + (uint32_t)i, L, p, ex, ez);
        orc_syndrome(L, ex, ez, syn + i * ns);
        if (true_class) true_class[i] = orc_class_code(L, ex, ez);
    }
    free(ex);
    free(ez);
}

void orc_gen_syndromes(uint64_t seed, uint32_t id0, int64_t n, int L, double p,
                       uint8_t* syn, int32_t* true_class)
{
    orc_gen_syndromes_noise(seed, id0, n, L, p, 0, syn, true_class);
}

/* ------------------------------------------------------------------------ */
/* Start state (reading of Sec. III / Sec. IV start "from each equivalence  */
/* class"): every anyon is joined by a straight string to its nearer         */
/* absorbing boundary; ties go left (p-anyons) or up (s-anyons).             */
/* ------------------------------------------------------------------------ */
void orc_pure_error(int L, const uint8_t* syn, uint8_t* ex, uint8_t* ez)
{
    int nq = orc_nq(L);
    memset(ex, 0, nq);
    memset(ez, 0, nq);
    for (int g = 0; g < orc_nstab(L); ++g) {
        if (!syn[g]) continue;
        int r, c;
        int type = orc_stab_pos(L, g, &r, &c);
        if (type == 1) {
            /* p-anyon at (r, c odd): sigma_x string along row r to the left
             * or right boundary, which absorb p-anyons. */
            int left = (c + 1) / 2, right = L - (c + 1) / 2;
            if (left <= right)
                for (int cc = c - 1; cc >= 0; cc -= 2) ex[qidx(L, r, cc)] ^= 1;
            else
                for (int cc = c + 1; cc <= 2 * L - 2; cc += 2) ex[qidx(L, r, cc)] ^= 1;
        } else {
            /* s-anyon at (r odd, c): sigma_z string along column c to the
             * top or bottom boundary, which absorb s-anyons. */
            int up = (r + 1) / 2, down = L - (r + 1) / 2;
            if (up <= down)
                for (int rr = r - 1; rr >= 0; rr -= 2) ez[qidx(L, rr, c)] ^= 1;
            else
                for (int rr = r + 1; rr <= 2 * L - 2; rr += 2) ez[qidx(L, rr, c)] ^= 1;
        }
    }
}

/* Start frame of class k: pure error times the logical that moves its class
 * code to k.  Returns the class code of the pure error. */
int orc_start_frame(int L, const uint8_t* syn, int k, uint8_t* ex, uint8_t* ez)
{
    orc_pure_error(L, syn, ex, ez);
    int code0 = orc_class_code(L, ex, ez);
    orc_apply_logical(L, k ^ code0, ex, ez);
    return code0;
}

/* ------------------------------------------------------------------------ */
/* Toric code (the 16-class variant): an L x L torus, L even, on the periodic */
/* 2L x 2L grid.  Data qubits at r+c odd, index r L + (c div 2) (2L^2 of     */
/* them); sigma_x generators (stars) at (even r, even c), sigma_z generators */
/* (plaquettes) at (odd r, odd c), all of weight 4; syndrome layout: stars   */
/* row-major over (i, j) = (r/2, c/2), then plaquettes over ((r-1)/2,        */
/* (c-1)/2).  Two encoded qubits, so 4 logical operators and 16 classes:     */
/* X1 = sigma_x on row 1, X2 = sigma_x on column 1, Z1 = sigma_z on column   */
/* 0, Z2 = sigma_z on row 0 (X1, Z1 and X2, Z2 anticommute, other pairs     */
/* commute).  Class code a1 + 2 a2 + 4 b1 + 8 b2 with a1 (a2) the parity of */
/* x on the support of Z1 (Z2) and b1 (b2) the parity of z on the support  */
/* of X1 (X2).                                                               */
/* ------------------------------------------------------------------------ */
int orc_t_nq(int L) { return 2 * L * L; }
int orc_t_nstab(int L) { return 2 * L * L; }

static int t_mod(int L, int v) { int m = 2 * L; return ((v % m) + m) % m; }
static int t_qidx(int L, int r, int c) { r = t_mod(L, r); c = t_mod(L, c); return r * L + c / 2; }

int orc_t_stab_pos(int L, int g, int* r, int* c)
{
    int type = g >= L * L;
    if (type) g -= L * L;
    *r = 2 * (g / L) + type;
    *c = 2 * (g % L) + type;
    return type;
}

int orc_t_stab_support(int L, int g, int32_t* q)
{
    int r, c;
    orc_t_stab_pos(L, g, &r, &c);
    q[0] = t_qidx(L, r - 1, c);
    q[1] = t_qidx(L, r + 1, c);
    q[2] = t_qidx(L, r, c - 1);
    q[3] = t_qidx(L, r, c + 1);
    return 4;
}

/* Colours: stars with (i+j) even -> 0, odd -> 1; plaquettes -> 2, 3 (with L
 * even, generators of one colour share no qubit across the periodic edges). */
int orc_t_stab_colour(int L, int g)
{
    int type = g >= L * L;
    int h = type ? g - L * L : g;
    return 2 * type + ((h / L + h % L) & 1);
}

int orc_t_colour_member(int L, int col, int m)
{
    for (int g = 0; g < orc_t_nstab(L); ++g)
        if (orc_t_stab_colour(L, g) == col && m-- == 0) return g;
    return -1;
}

void orc_t_syndrome(int L, const uint8_t* ex, const uint8_t* ez, uint8_t* syn)
{
    int32_t q[4];
    for (int g = 0; g < orc_t_nstab(L); ++g) {
        int r, c;
        int type = orc_t_stab_pos(L, g, &r, &c);
        orc_t_stab_support(L, g, q);
        int par = 0;
        for (int k = 0; k < 4; ++k) par ^= type == 0 ? ez[q[k]] : ex[q[k]];
        syn[g] = (uint8_t)par;
    }
}

int orc_t_class_code(int L, const uint8_t* ex, const uint8_t* ez)
{
    int a1 = 0, a2 = 0, b1 = 0, b2 = 0;
    for (int i = 0; i < L; ++i) {
        a1 ^= ex[t_qidx(L, 2 * i + 1, 0)];   /* Z1: column 0, odd rows */
        a2 ^= ex[t_qidx(L, 0, 2 * i + 1)];   /* Z2: row 0, odd columns */
        b1 ^= ez[t_qidx(L, 1, 2 * i)];       /* X1: row 1, even columns */
        b2 ^= ez[t_qidx(L, 2 * i, 1)];       /* X2: column 1, even rows */
    }
    return a1 + 2 * a2 + 4 * b1 + 8 * b2;
}

void orc_t_apply_logical(int L, int k, uint8_t* ex, uint8_t* ez)
{
    for (int i = 0; i < L; ++i) {
        if (k & 1) ex[t_qidx(L, 1, 2 * i)] ^= 1;       /* X1 */
        if (k & 2) ex[t_qidx(L, 2 * i, 1)] ^= 1;       /* X2 */
        if (k & 4) ez[t_qidx(L, 2 * i + 1, 0)] ^= 1;   /* Z1 */
        if (k & 8) ez[t_qidx(L, 0, 2 * i + 1)] ^= 1;   /* Z2 */
    }
}

/* Pure error on the torus: the violated generators of each type (an even
 * number) are paired in syndrome order, first with second, third with
 * fourth, ...; a pair is joined by a string that runs from the first to the
 * column of the second in the direction of increasing c (mod 2L), then down
 * to its row in the direction of increasing r; sigma_z strings through the
 * qubits between consecutive stars, sigma_x strings between consecutive
 * plaquettes. */
void orc_t_pure_error(int L, const uint8_t* syn, uint8_t* ex, uint8_t* ez)
{
    int nq = orc_t_nq(L);
    memset(ex, 0, nq);
    memset(ez, 0, nq);
    for (int type = 0; type < 2; ++type) {
        int first = -1;
        for (int h = 0; h < L * L; ++h) {
            int g = h + type * L * L;
            if (!syn[g]) continue;
            if (first < 0) { first = g; continue; }
            int r0, c0, r1, c1;
            orc_t_stab_pos(L, first, &r0, &c0);
            orc_t_stab_pos(L, g, &r1, &c1);
            uint8_t* f = type == 0 ? ez : ex;
            for (int c = c0; c != c1; c = t_mod(L, c + 2)) f[t_qidx(L, r0, c + 1)] ^= 1;
            for (int r = r0; r != r1; r = t_mod(L, r + 2)) f[t_qidx(L, r + 1, c1)] ^= 1;
            first = -1;
        }
    }
}

int orc_t_start_frame(int L, const uint8_t* syn, int k, uint8_t* ex, uint8_t* ez)
{
    orc_t_pure_error(L, syn, ex, ez);
    int code0 = orc_t_class_code(L, ex, ez);
    orc_t_apply_logical(L, k ^ code0, ex, ez);
    return code0;
}

/* Depolarizing errors on the torus (same draws per qubit as the planar
 * generator: counter (id, q div 4, 0, 0), word q mod 4). */
void orc_t_gen_syndromes(uint64_t seed, uint32_t id0, int64_t n, int L, double p, uint8_t* syn,
                         int32_t* true_class)
{
    int nq = orc_t_nq(L), ns = orc_t_nstab(L);
    uint8_t* ex = malloc(nq);
    uint8_t* ez = malloc(nq);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x53594E44u};
    uint64_t tau = (uint64_t)floor((p / 3.0) * 4294967296.0);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t blk[4];
        for (int q = 0; q < nq; ++q) {
            uint32_t ctr[4] = {id0 + (uint32_t)i, (uint32_t)(q / 4), 0, 0};
            orc_philox4x32_10(ctr, key, blk);
            uint64_t u = blk[q % 4];
            ex[q] = (uint8_t)(u < 2 * tau);
            ez[q] = (uint8_t)(u >= tau && u < 3 * tau);
        }
        orc_t_syndrome(L, ex, ez, syn + i * ns);
        if (true_class) true_class[i] = orc_t_class_code(L, ex, ez);
    }
    free(ex);
    free(ez);
}

/* Exact weight histogram of the 16 classes on the torus (as for the planar
 * code): all 2^{n_stab} products of generators times each class's start
 * frame, Gray-code order; every frame of a class appears 4 times (the star
 * product and the plaquette product are both the identity).  n_stab <= 30. */
int orc_t_exact_histogram(int L, const uint8_t* syn, uint64_t* hist /* [16][nq+1] */)
{
    int nq = orc_t_nq(L), ns = orc_t_nstab(L);
    if (ns > 30) return -1;
    int32_t sup[4 * 64];
    int type[64];
    for (int g = 0; g < ns; ++g) {
        int r, c;
        type[g] = orc_t_stab_pos(L, g, &r, &c);
        orc_t_stab_support(L, g, sup + 4 * g);
    }
    uint8_t ex[64], ez[64];
    for (int k = 0; k < 16; ++k) {
        uint64_t* h = hist + (size_t)k * (nq + 1);
        memset(h, 0, sizeof(uint64_t) * (nq + 1));
        orc_t_start_frame(L, syn, k, ex, ez);
        int n = 0;
        for (int q = 0; q < nq; ++q) n += ex[q] | ez[q];
        h[n] += 1;
        for (uint64_t i = 1; i < ((uint64_t)1 << ns); ++i) {
            int g = __builtin_ctzll(i);
            for (int e = 0; e < 4; ++e) {
                if (type[g] == 0) ex[sup[4 * g + e]] ^= 1; else ez[sup[4 * g + e]] ^= 1;
            }
            n = 0;
            for (int q = 0; q < nq; ++q) n += ex[q] | ez[q];
            h[n] += 1;
        }
    }
    return 0;
}

/* Geometry of a run: the planar code for 4 classes, the torus for 16. */
static int geo_nq(int K, int L) { return K == 16 ? orc_t_nq(L) : orc_nq(L); }
static int geo_nstab(int K, int L) { return K == 16 ? orc_t_nstab(L) : orc_nstab(L); }
static int geo_stab_pos(int K, int L, int g, int* r, int* c)
{
    return K == 16 ? orc_t_stab_pos(L, g, r, c) : orc_stab_pos(L, g, r, c);
}
static int geo_stab_support(int K, int L, int g, int32_t* q)
{
    return K == 16 ? orc_t_stab_support(L, g, q) : orc_stab_support(L, g, q);
}
static int geo_colour_count(int K, int L, int col)
{
    return K == 16 ? orc_t_nstab(L) / 4 : orc_colour_count(L, col);
}
static int geo_colour_member(int K, int L, int col, int m)
{
    return K == 16 ? orc_t_colour_member(L, col, m) : orc_colour_member(L, col, m);
}
static int geo_start_frame(int K, int L, const uint8_t* syn, int k, uint8_t* ex, uint8_t* ez)
{
    return K == 16 ? orc_t_start_frame(L, syn, k, ex, ez) : orc_start_frame(L, syn, k, ex, ez);
}

/* ------------------------------------------------------------------------ */
/* Acceptance table (Eq. 2): r = (p/3)/(1-p) = e^{-beta_bar}; with a        */
/* scaled temperature beta* = s beta_bar, r* = e^{-beta*}.                   */
/* T[d] = floor(r*^d 2^32) for d = 1..4, r*^d by repeated multiplication.   */
/* ------------------------------------------------------------------------ */
void orc_thresholds_noise(double p, int noise, double beta_scale, uint64_t* T, double* beta_bar)
{
    /* depolarizing: r = (p/3)/(1-p) (Eq. 2); independent flips: each flip
     * costs p/(1-p) (Sec. IV.B) */
    double r = noise ? p / (1.0 - p) : (p / 3.0) / (1.0 - p);
    double rs = beta_scale == 1.0 ? r : exp(-beta_scale * -log(r));
    double rd = rs;
    T[0] = 0;
    for (int d = 1; d <= 4; ++d) {
        T[d] = (uint64_t)floor(rd * 4294967296.0);
        rd = rd * rs;
    }
    if (beta_bar) *beta_bar = -log(r);
}

void orc_thresholds(double p, double beta_scale, uint64_t* T, double* beta_bar)
{
    orc_thresholds_noise(p, 0, beta_scale, T, beta_bar);
}

/* General Pauli channel (Eq. 1 with integer energies, Sec. IV: the method
 * "generalizes straightforwardly to arbitrary error models" of that form):
 * p_X : p_Y : p_Z : p_I = r^eX : r^eY : r^eZ : 1 with e_P in 1..8 and total
 * error probability p = p_X + p_Y + p_Z in (0, 3/4].  r in (0, 1] solves
 * (1 - p)(r^eX + r^eY + r^eZ) = p; found by 100 halvings of [0, 1] (the
 * left end moves when the value at the midpoint is below p), powers by
 * repeated multiplication. */
static double powi(double r, int e)
{
    double v = 1.0;
    for (int i = 0; i < e; ++i) v *= r;
    return v;
}

double orc_rate_general(double p, int eX, int eY, int eZ)
{
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 100; ++it) {
        double mid = 0.5 * (lo + hi);
        double f = (1.0 - p) * (powi(mid, eX) + powi(mid, eY) + powi(mid, eZ));
        if (f < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* T[d] = floor(r*^d 2^32), d = 1..dmax, r* = r or exp(-beta_scale * -log r). */
void orc_thresholds_r(double r, double beta_scale, int dmax, uint64_t* T, double* beta_bar)
{
    double rs = beta_scale == 1.0 ? r : exp(-beta_scale * -log(r));
    double rd = rs;
    T[0] = 0;
    for (int d = 1; d <= dmax; ++d) {
        T[d] = (uint64_t)floor(rd * 4294967296.0);
        rd = rd * rs;
    }
    if (beta_bar) *beta_bar = -log(r);
}

/* Sampled errors of the general channel: u of qubit q is word q mod 4 of the
 * block with counter (id, q div 4, 2, 0) (key as for the other models); X if
 * u < floor(pX 2^32), Y if u < floor((pX + pY) 2^32), Z if u < floor((pX +
 * pY + pZ) 2^32), else I. */
void orc_gen_syndromes_pauli(uint64_t seed, uint32_t id0, int64_t n, int L, double px, double py, double pz,
                             uint8_t* syn, int32_t* true_class)
{
    int nq = orc_nq(L), ns = orc_nstab(L);
    uint8_t* ex = malloc(nq);
    uint8_t* ez = malloc(nq);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x53594E44u};
    uint64_t t1 = (uint64_t)floor(px * 4294967296.0);
    uint64_t t2 = (uint64_t)floor((px + py) * 4294967296.0);
    uint64_t t3 = (uint64_t)floor((px + py + pz) * 4294967296.0);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t blk[4];
        for (int q = 0; q < nq; ++q) {
            uint32_t ctr[4] = {id0 + (uint32_t)i, (uint32_t)(q / 4), 2, 0};
            orc_philox4x32_10(ctr, key, blk);
            uint64_t u = blk[q % 4];
            ex[q] = (uint8_t)(u < t2);
            ez[q] = (uint8_t)(u >= t1 && u < t3);
        }
        orc_syndrome(L, ex, ez, syn + i * ns);
        if (true_class) true_class[i] = orc_class_code(L, ex, ez);
    }
    free(ex);
    free(ez);
}

/* ------------------------------------------------------------------------ */
/* The uniform u of one chain for one proposal.                             */
/*                                                                          */
/* C = chains per syndrome; G = min(32, smallest power of two >= C) is the  */
/* plane width; chain c has group w = c div G and lane b = c mod G.  For    */
/* proposal (syndrome id s, sweep t, colour col, index m within the colour) */
/* and group w, Philox blocks j = 0, 1, ... with counter                    */
/*    (s, t, (col << 24) | m, (w << 8) | j)                                 */
/* and key (seed_lo, seed_hi) are concatenated into one bit stream (block j */
/* supplies stream bits 128j .. 128j+127; word i of a block supplies bits   */
/* 32i .. 32i+31, least significant first).  Plane k (k = 0..31) is stream  */
/* bits kG .. kG+G-1; chain c's bit of plane k is stream bit kG + b, and    */
/*    u_c = sum_k bit_k(c) 2^(31-k)                                         */
/* (plane 0 is the most significant bit).                                   */
/* ------------------------------------------------------------------------ */
int orc_plane_width(int C)
{
    int G = 1;
    while (G < C && G < 32) G *= 2;
    return G;
}

typedef struct {
    uint32_t key[2];
    uint32_t s, t, col, m, w;
    int cached_j;
    uint32_t blk[4];
} stream_t;

static int stream_bit(stream_t* st, uint32_t idx)
{
    int j = (int)(idx / 128);
    if (j != st->cached_j) {
        uint32_t ctr[4] = {st->s, st->t, (st->col << 24) | st->m, (st->w << 8) | (uint32_t)j};
        orc_philox4x32_10(ctr, st->key, st->blk);
        st->cached_j = j;
    }
    return (st->blk[(idx / 32) % 4] >> (idx % 32)) & 1u;
}

/* Full 32-bit u of chain c (assembles all 32 planes). */
uint32_t orc_chain_uniform(uint64_t seed, uint32_t s, uint32_t t, int col, int m, int c, int C)
{
    int G = orc_plane_width(C);
    stream_t st = {{(uint32_t)seed, (uint32_t)(seed >> 32)}, s, t, (uint32_t)col, (uint32_t)m,
                   (uint32_t)(c / G), -1, {0, 0, 0, 0}};
    uint32_t u = 0;
    for (int k = 0; k < 32; ++k) u |= (uint32_t)stream_bit(&st, (uint32_t)(k * G + c % G)) << (31 - k);
    return u;
}

/* u_c < T, evaluated by comparing the binary digits most significant first
 * and stopping at the first digit where they differ (the ordinary
 * lexicographic comparison of two 32-digit binary numbers; it reads only as
 * many planes as the comparison needs).  T may equal 2^32. */
int orc_chain_uniform_less(uint64_t seed, uint32_t s, uint32_t t, int col, int m, int c, int C, uint64_t T)
{
    if (T >= 4294967296ull) return 1;
    int G = orc_plane_width(C);
    stream_t st = {{(uint32_t)seed, (uint32_t)(seed >> 32)}, s, t, (uint32_t)col, (uint32_t)m,
                   (uint32_t)(c / G), -1, {0, 0, 0, 0}};
    for (int k = 0; k < 32; ++k) {
        int ub = stream_bit(&st, (uint32_t)(k * G + c % G));
        int tb = (int)((T >> (31 - k)) & 1u);
        if (ub != tb) return ub < tb;
    }
    return 0; /* equal: u == T is not less */
}

/* ------------------------------------------------------------------------ */
/* The single-temperature algorithm (Sec. IV.A) for one syndrome.           */
/* ------------------------------------------------------------------------ */

/* Energy of a qubit's Pauli, E[x + 2z] for I, X, Z, Y: depolarizing {0, 1,
 * 1, 1} (n = qubits in error, Sec. IV), independent flips {0, 1, 1, 2}
 * (n = bit flips + phase flips, Sec. IV.B), general {0, eX, eZ, eY}. */
static void energy_table(int noise, const int32_t* e, int E[4])
{
    E[0] = 0;
    if (noise == 2) {
        E[1] = e[0];
        E[2] = e[2];
        E[3] = e[1];
    } else {
        E[1] = 1;
        E[2] = 1;
        E[3] = noise ? 2 : 1;
    }
}

static int weight(int nq, const uint8_t* ex, const uint8_t* ez, const int E[4])
{
    int n = 0;
    for (int q = 0; q < nq; ++q) n += E[ex[q] + 2 * ez[q]];
    return n;
}

/* Delta n of applying generator g (Sec. IV: "the number Delta n by which the
 * total number of errors n in the code would change if that stabilizer were
 * applied"); a sigma_x generator flips x on its support, a sigma_z generator
 * flips z.  Plain before/after count over the support. */
static int delta_n(int type, int w, const int32_t* q, const uint8_t* ex, const uint8_t* ez, const int E[4])
{
    int before = 0, after = 0;
    for (int k = 0; k < w; ++k) {
        int x = ex[q[k]], z = ez[q[k]];
        before += E[x + 2 * z];
        if (type == 0) x ^= 1; else z ^= 1;
        after += E[x + 2 * z];
    }
    return after - before;
}

typedef struct {
    int32_t L, K, R;
    uint32_t t_begin, t_end, burn_in;
    double p, beta_scale;
    uint64_t seed;
    uint32_t id;
    int32_t anneal_stages;
    double anneal_beta0;
    int32_t scan;          /* 0: colour sweeps (Sec. V); 1: one random generator per step (Sec. IV) */
    int32_t noise;         /* 0: depolarizing; 1: independent bit and phase flips; 2: general */
    int32_t energy[3];     /* eX, eY, eZ of the general channel (noise 2) */
} orc_run_t;

/* r = e^{-beta_bar} of a run's noise model. */
static double run_rate(const orc_run_t* a)
{
    if (a->noise == 2) return orc_rate_general(a->p, a->energy[0], a->energy[1], a->energy[2]);
    return a->noise ? a->p / (1.0 - a->p) : (a->p / 3.0) / (1.0 - a->p);
}

/* Start preparation (reading of Sec. IV: the chains should start near the
 * low-energy configurations of their class, because heating up from them is
 * fast while cooling down from a high-energy start is slow).  The burn-in
 * sweeps 0 .. B-1 are split into S stages; stage j covers sweeps
 * floor(jB/S) .. floor((j+1)B/S)-1 and runs at beta = beta* times
 * a0 + (1 - a0) j / S.  Nothing is sampled during the burn-in. */
double orc_anneal_scale(double beta_scale, double a0, int j, int S)
{
    return beta_scale * (a0 + (1.0 - a0) * (double)j / (double)S);
}

int orc_anneal_stage(uint32_t t, uint32_t B, int S)
{
    for (int j = 0; j < S; ++j) {
        uint64_t lo = (uint64_t)j * B / (uint64_t)S, hi = (uint64_t)(j + 1) * B / (uint64_t)S;
        if (t >= lo && t < hi) return j;
    }
    return -1;
}

/* Run all K*R chains of one syndrome over sweeps t_begin .. t_end-1.
 *   frames_x/z [C][nq]: in: state at t_begin (if start_from_syndrome the
 *     start frames are built here), out: final state.
 *   chain_sum [C]: in/out running sum of sampled n (after every colour phase
 *     of a sweep t >= burn_in); chain_n [C]: out final n;
 *   accepts [C]: in/out number of accepted proposals (may be NULL);
 *   trace (may be NULL): receives n after every colour phase of chain 0,
 *     4 (t_end - t_begin) entries. */
void orc_run_chains(const orc_run_t* a, const uint8_t* syn, int start_from_syndrome,
                    uint8_t* frames_x, uint8_t* frames_z, uint64_t* chain_sum,
                    int32_t* chain_n, uint64_t* accepts, int32_t* trace)
{
    int L = a->L, nq = geo_nq(a->K, L), C = a->K * a->R;
    uint64_t Tmain[33], Tst[64][33];
    int E[4];
    energy_table(a->noise, a->energy, E);
    double rate = run_rate(a);
    orc_thresholds_r(rate, a->beta_scale, 32, Tmain, NULL);
    for (int j = 0; j < a->anneal_stages && j < 64; ++j)
        orc_thresholds_r(rate, orc_anneal_scale(a->beta_scale, a->anneal_beta0, j, a->anneal_stages), 32, Tst[j],
                         NULL);
    int ncol[4], members[4][ORC_MAX_L * ORC_MAX_L];
    for (int col = 0; col < 4; ++col) {
        ncol[col] = geo_colour_count(a->K, L, col);
        for (int m = 0; m < ncol[col]; ++m) members[col][m] = geo_colour_member(a->K, L, col, m);
    }
    for (int c = 0; c < C; ++c) {
        uint8_t* ex = frames_x + (size_t)c * nq;
        uint8_t* ez = frames_z + (size_t)c * nq;
        if (start_from_syndrome) geo_start_frame(a->K, L, syn, c / a->R, ex, ez);
        int n = weight(nq, ex, ez, E);
        for (uint32_t t = a->t_begin; t < a->t_end; ++t) {
            int stage = a->anneal_stages > 0 ? orc_anneal_stage(t, a->burn_in, a->anneal_stages) : -1;
            const uint64_t* T = stage >= 0 ? Tst[stage] : Tmain;
            if (a->scan) {
                /* Sec. IV as written: each step picks one generator at
                 * random, g = floor(w0 n_stab / 2^32), and applies it when
                 * Delta n <= 0 or w1 < T[Delta n]; f(n) = n is summed after
                 * every step.  A sweep is n_stab steps; Philox counter
                 * (id, chain, t, step), words w0, w1. */
                int ns = geo_nstab(a->K, L);
                for (int step = 0; step < ns; ++step) {
                    uint32_t ctr[4] = {a->id, (uint32_t)c, t, (uint32_t)step}, key[2], blk[4];
                    key[0] = (uint32_t)a->seed;
                    key[1] = (uint32_t)(a->seed >> 32);
                    orc_philox4x32_10(ctr, key, blk);
                    int g = (int)(((uint64_t)blk[0] * (uint64_t)ns) >> 32);
                    int r, cc;
                    int type = geo_stab_pos(a->K, L, g, &r, &cc);
                    int32_t q[4];
                    int w = geo_stab_support(a->K, L, g, q);
                    int dn = delta_n(type, w, q, ex, ez, E);
                    if (dn <= 0 || (uint64_t)blk[1] < T[dn]) {
                        for (int k = 0; k < w; ++k) {
                            if (type == 0) ex[q[k]] ^= 1; else ez[q[k]] ^= 1;
                        }
                        n += dn;
                        if (accepts) accepts[c] += 1;
                    }
                    if (t >= a->burn_in) chain_sum[c] += (uint64_t)n;
                }
                if (trace && c == 0) trace[t - a->t_begin] = n;
                continue;
            }
            for (int col = 0; col < 4; ++col) {
                int type = col / 2;
                for (int m = 0; m < ncol[col]; ++m) {
                    int32_t q[4];
                    int w = geo_stab_support(a->K, L, members[col][m], q);
                    int dn = delta_n(type, w, q, ex, ez, E);
                    /* Metropolis (Sec. IV): apply if Delta n <= 0, otherwise
                     * with probability e^{-beta* Delta n} = T[Delta n] / 2^32. */
                    int accept = dn <= 0 ||
                                 orc_chain_uniform_less(a->seed, a->id, t, col, m, c, C, T[dn]);
                    if (accept) {
                        for (int k = 0; k < w; ++k) {
                            if (type == 0) ex[q[k]] ^= 1; else ez[q[k]] ^= 1;
                        }
                        n += dn;
                        if (accepts) accepts[c] += 1;
                    }
                }
                /* Sec. V: n is added up after every group step. */
                if (t >= a->burn_in) chain_sum[c] += (uint64_t)n;
                if (trace && c == 0) trace[4 * (t - a->t_begin) + col] = n;
            }
        }
        if (chain_n) chain_n[c] = n;
    }
}

/* Decision (Sec. IV.A): S_k = sum over the R chains of class k; choose the
 * class with the smallest S_k (the smallest <n>, all classes having the same
 * number of samples), lowest k on ties.  Also reports the log-ratio proxy
 * -beta_bar (<n>_k - min_k <n>_k). */
int orc_decide(int K, int R, uint32_t n_sweeps, uint32_t burn_in, uint32_t samples_per_sweep, double beta_bar,
               const uint64_t* chain_sum, uint64_t* class_sum, double* log_ratio)
{
    uint64_t S[64];
    int best = 0;
    for (int k = 0; k < K; ++k) {
        S[k] = 0;
        for (int r = 0; r < R; ++r) S[k] += chain_sum[k * R + r];
        if (S[k] < S[best]) best = k;
        if (class_sum) class_sum[k] = S[k];
    }
    if (log_ratio) {
        uint64_t samples =
            n_sweeps > burn_in ? (uint64_t)samples_per_sweep * (uint64_t)R * (n_sweeps - burn_in) : 0;
        for (int k = 0; k < K; ++k) {
            if (samples == 0) { log_ratio[k] = 0.0; continue; }
            double mean_k = (double)S[k] / (double)samples;
            double mean_b = (double)S[best] / (double)samples;
            log_ratio[k] = -beta_bar * (mean_k - mean_b);
        }
    }
    return best;
}

/* Full decode of one syndrome from its start frames. */
int orc_decode_one(int L, double p, int K, int R, uint32_t n_sweeps, uint32_t burn_in,
                   double beta_scale, int anneal_stages, double anneal_beta0, uint64_t seed, uint32_t id,
                   const uint8_t* syn, uint64_t* class_sum, double* log_ratio, uint64_t* chain_sum,
                   int32_t* chain_n, uint8_t* frames_x, uint8_t* frames_z, uint64_t* accepts, int scan,
                   int noise, const int32_t* energy)
{
    int nq = geo_nq(K, L), C = K * R;
    orc_run_t a = {L, K, R, 0, n_sweeps, burn_in, p, beta_scale, seed, id, anneal_stages, anneal_beta0, scan, noise,
                   {1, 1, 1}};
    if (noise == 2)
        for (int i = 0; i < 3; ++i) a.energy[i] = energy[i];
    uint8_t* fx = frames_x ? frames_x : malloc((size_t)C * nq);
    uint8_t* fz = frames_z ? frames_z : malloc((size_t)C * nq);
    uint64_t* cs = chain_sum ? chain_sum : malloc(sizeof(uint64_t) * C);
    memset(cs, 0, sizeof(uint64_t) * C);
    if (accepts) memset(accepts, 0, sizeof(uint64_t) * C);
    orc_run_chains(&a, syn, 1, fx, fz, cs, chain_n, accepts, NULL);
    double beta_bar;
    uint64_t T[5];
    orc_thresholds_r(run_rate(&a), 1.0, 4, T, &beta_bar);
    int k = orc_decide(K, R, n_sweeps, burn_in, scan ? (uint32_t)geo_nstab(K, L) : 4u, beta_bar, cs, class_sum,
                       log_ratio);
    if (!frames_x) free(fx);
    if (!frames_z) free(fz);
    if (!chain_sum) free(cs);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Exact class statistics by enumeration (Eq. 3): the histogram of n over    */
/* all 2^{n_stab} frames of each class (start frame times every product of  */
/* generators).  hist[k][n] counts frames of class k with weight n, so that */
/* Z_k(beta) = sum_n hist[k][n] e^{-beta n} and <n>_{beta,k} follows         */
/* (Eq. 4).  Gray-code order: one generator is toggled per step.  L <= 4.   */
/* ------------------------------------------------------------------------ */
int orc_exact_histogram_energy(int L, const uint8_t* syn, int noise, const int32_t* energy, int width,
                               uint64_t* hist /* [4][width] */)
{
    int E[4];
    energy_table(noise, energy, E);
    int nq = orc_nq(L), ns = orc_nstab(L);
    if (ns > 30) return -1;
    int32_t sup[4 * 64];
    int wt[64], type[64];
    for (int g = 0; g < ns; ++g) {
        int r, c;
        type[g] = orc_stab_pos(L, g, &r, &c);
        wt[g] = orc_stab_support(L, g, sup + 4 * g);
    }
    uint8_t ex[64], ez[64];
    for (int k = 0; k < 4; ++k) {
        uint64_t* h = hist + (size_t)k * width;
        memset(h, 0, sizeof(uint64_t) * width);
        orc_start_frame(L, syn, k, ex, ez);
        h[weight(nq, ex, ez, E)] += 1;
        for (uint64_t i = 1; i < ((uint64_t)1 << ns); ++i) {
            int g = __builtin_ctzll(i); /* generator toggled between Gray codes i-1 and i */
            for (int e = 0; e < wt[g]; ++e) {
                if (type[g] == 0) ex[sup[4 * g + e]] ^= 1; else ez[sup[4 * g + e]] ^= 1;
            }
            h[weight(nq, ex, ez, E)] += 1;
        }
    }
    return 0;
}

int orc_exact_histogram_noise(int L, const uint8_t* syn, int noise, uint64_t* hist /* [4][2 nq + 1] */)
{
    return orc_exact_histogram_energy(L, syn, noise, NULL, noise ? 2 * orc_nq(L) + 1 : orc_nq(L) + 1, hist);
}

int orc_exact_histogram(int L, const uint8_t* syn, uint64_t* hist /* [4][nq+1] */)
{
    return orc_exact_histogram_noise(L, syn, 0, hist);
}

/* ------------------------------------------------------------------------ */
/* Thermodynamic integration (Eq. 6): log Z_E(beta_bar) = -int_0^beta_bar    */
/* <n>_{beta,E} d beta + n_stab log 2.  The integral is taken with the       */
/* composite Simpson rule (Sec. IV) on the equidistant grid                  */
/* beta_j = j beta_bar / (N-1), j = 0..N-1 (N odd; Sec. IV.A uses N = 21),   */
/* with <n> at beta = 0 equal to 3/4 n_qubits (Sec. IV.A).  mean[k*N + j] is */
/* <n>_{beta_j, k}; I[k] receives the integral of class k.                   */
/* ------------------------------------------------------------------------ */
int orc_simpson_integral(int K, int N, const double* mean, double beta_bar, double* I)
{
    if (N < 3 || N % 2 == 0) return -1;
    double h = beta_bar / (double)(N - 1);
    for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (int j = 0; j < N; ++j) {
            double w = (j == 0 || j == N - 1) ? 1.0 : (j % 2 == 1 ? 4.0 : 2.0);
            double term = w * mean[k * N + j];
            acc = acc + term;
        }
        I[k] = acc * (h / 3.0);
    }
    return 0;
}

/* TI decode of one syndrome: chains at beta_j = beta* j/(N-1), j = 1..N-1
 * (seed + j for the randomness of grid point j, the same options otherwise,
 * the burn-in annealing scaled with beta_j), <n> at j = 0 set to 3/4 n_q;
 * class = argmin_k I_k (argmax log Z_k, lowest k on ties);
 * log_z[k] = -(I_k - min_k I_k).  mean_out[k*N + j] receives the means. */
int orc_decode_ti(int L, double p, int K, int R, uint32_t n_sweeps, uint32_t burn_in, double beta_scale,
                  int anneal_stages, double anneal_beta0, int N, uint64_t seed, uint32_t id,
                  const uint8_t* syn, double* mean_out, double* log_z, int scan, int noise,
                  const int32_t* energy)
{
    int nq = geo_nq(K, L), C = K * R;
    if (N < 3 || N % 2 == 0 || N > 129 || K > 64) return -1;
    uint64_t per_sweep = scan ? (uint64_t)geo_nstab(K, L) : 4u;
    uint64_t samples = n_sweeps > burn_in ? per_sweep * (uint64_t)R * (n_sweeps - burn_in) : 0;
    if (samples == 0) return -1;
    uint8_t* fx = malloc((size_t)C * nq);
    uint8_t* fz = malloc((size_t)C * nq);
    uint64_t* cs = malloc(sizeof(uint64_t) * C);
    double* mean = malloc(sizeof(double) * K * N);
    /* beta = 0: every frame of the class equally likely, so each qubit's x
     * and z are uniform: <n> = 3/4 n_q (depolarizing), n_q (flips) */
    int E[4];
    energy_table(noise, energy, E);
    for (int k = 0; k < K; ++k) mean[k * N] = (double)nq * (double)(E[1] + E[2] + E[3]) / 4.0;
    for (int j = 1; j < N; ++j) {
        double bs = beta_scale * (double)j / (double)(N - 1);
        orc_run_t a = {L, K, R, 0, n_sweeps, burn_in, p, bs, seed + (uint64_t)j, id, anneal_stages, anneal_beta0,
                       scan, noise, {1, 1, 1}};
        if (noise == 2)
            for (int i = 0; i < 3; ++i) a.energy[i] = energy[i];
        memset(cs, 0, sizeof(uint64_t) * C);
        orc_run_chains(&a, syn, 1, fx, fz, cs, NULL, NULL, NULL);
        for (int k = 0; k < K; ++k) {
            uint64_t S = 0;
            for (int r = 0; r < R; ++r) S += cs[k * R + r];
            mean[k * N + j] = (double)S / (double)samples;
        }
    }
    double beta_bar;
    uint64_t T[5];
    orc_run_t a0 = {L, K, R, 0, 0, 0, p, 1.0, 0, 0, 0, 1.0, scan, noise, {1, 1, 1}};
    if (noise == 2)
        for (int i = 0; i < 3; ++i) a0.energy[i] = energy[i];
    orc_thresholds_r(run_rate(&a0), 1.0, 4, T, &beta_bar);
    double I[64];
    orc_simpson_integral(K, N, mean, beta_scale * beta_bar, I);
    int best = 0;
    for (int k = 1; k < K; ++k)
        if (I[k] < I[best]) best = k;
    for (int k = 0; k < K; ++k) log_z[k] = -(I[k] - I[best]);
    if (mean_out) memcpy(mean_out, mean, sizeof(double) * K * N);
    free(fx);
    free(fz);
    free(cs);
    free(mean);
    return best;
}
