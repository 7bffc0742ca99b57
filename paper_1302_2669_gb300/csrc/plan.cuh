// Host-side planning of a sweep launch, shared by every entry point that
// launches the sweep kernel (api.cu and noalloc.cu): the noise model's
// energies and rate, the Eq. 2 acceptance table and its digit-plane form,
// the lane split, and the chain layout of a run.  Pure host arithmetic: no
// allocation, no context, no device call.
#pragma once
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "surfmcmc.h"

namespace surfmcmc {

// Energy of a qubit's Pauli, index x + 2z (I, X, Z, Y), of a noise model:
// depolarizing {0, 1, 1, 1} (n = qubits in error, Sec. IV), independent
// flips {0, 1, 1, 2} (Sec. IV.B), general channel {0, eX, eZ, eY}.
inline void energy_table(const surfmcmc_opts& o, int E[4]) {
    E[0] = 0;
    if (o.noise == 2) {
        E[1] = o.pauli_energy[0];
        E[2] = o.pauli_energy[2];
        E[3] = o.pauli_energy[1];
    } else {
        E[1] = 1;
        E[2] = 1;
        E[3] = o.noise ? 2 : 1;
    }
}

inline double powi(double r, int e) {
    double v = 1.0;
    for (int i = 0; i < e; ++i) v *= r;
    return v;
}

// r = e^{-beta_bar}: (p/3)/(1-p) (Eq. 2, depolarizing), p/(1-p)
// (independent flips), or for the general channel the root r in (0, 1] of
// (1 - p)(r^eX + r^eY + r^eZ) = p after 100 halvings of [0, 1] (the left end
// moves when the value at the midpoint is below p).
inline double noise_rate(double p, int noise, const int E[4]) {
    if (noise == 0) return (p / 3.0) / (1.0 - p);
    if (noise == 1) return p / (1.0 - p);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 100; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double f = (1.0 - p) * (powi(mid, E[1]) + powi(mid, E[3]) + powi(mid, E[2]));
        if (f < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// r* = e^{-beta_scale beta_bar}; T[d] = floor(r*^d 2^32), d = 1..32, r*^d by
// repeated multiplication.
inline void acceptance_table(double r, double beta_scale, uint64_t T[33], double* beta_bar) {
    const double rs = beta_scale == 1.0 ? r : exp(-beta_scale * -log(r));
    double rd = rs;
    T[0] = 0;
    for (int d = 1; d <= 32; ++d) {
        T[d] = (uint64_t)floor(rd * 4294967296.0);
        rd = rd * rs;
    }
    *beta_bar = -log(r);
}

// Burn-in stage j of S runs at beta* (a0 + (1 - a0) j / S).
inline double anneal_scale(double beta_scale, double a0, int j, int S) {
    return beta_scale * (a0 + (1.0 - a0) * (double)j / (double)S);
}

// Acceptance thresholds of one launch as kernel parameters: flags, the
// per-quad digit modes, and per plane k the algebraic normal form of
// d-1 -> bit (31-k) of T[d].  Reads sp.noise and sp.energy.
inline void set_temperature(SweepParams& sp, double p, double beta_scale) {
    uint64_t T[33];
    double beta_bar;
    acceptance_table(noise_rate(p, sp.noise, sp.energy), beta_scale, T, &beta_bar);
    for (int d = 0; d < 33; ++d) sp.T[d] = T[d];
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

// Shared memory a block may use for the sweep (the kernel's own limit).
constexpr size_t kSweepSmemLimit = 200 * 1024;

// Lanes per bundle by rule: the most lanes that the colour's generators fill
// to >= 90%, else the best fill, within the shared-memory limit.
inline int heuristic_lanes(int L, int code) {
    const int nq = geo_nq(code, L), nc = geo_nc(code, L);
    int best = 32;
    double best_eff = -1;
    for (int lam = 32; lam >= 2; lam /= 2) {
        if (sweep_smem_bytes(nq, nc, lam) > kSweepSmemLimit) continue;
        const double eff = (double)nc / (double)(lam * ((nc + lam - 1) / lam));
        if (eff >= 0.9) return lam;
        if (eff > best_eff + 1e-12) {
            best_eff = eff;
            best = lam;
        }
    }
    return best;
}

// Small batches: a persistent block takes work units of 4 warps x 32/lam
// bundles, so a batch of few bundles leaves most blocks idle and the run
// time is the latency of one unit.  Widen (more lanes share a bundle's
// generators, shorter units) until the units fill the resident blocks of a
// device with `sms` multiprocessors once.  The results do not depend on the
// lanes.
inline int widen_lanes_for(int sms, int L, int lam, long long n_bundles, int G, int code) {
    if (sms <= 0) return lam;
    const int nq = geo_nq(code, L), nc = geo_nc(code, L);
    const long long capacity = (long long)sms * sweep_blocks_per_sm(G);
    while (lam < 32 && sweep_units(n_bundles, lam) < capacity && sweep_smem_bytes(nq, nc, 2 * lam) <= kSweepSmemLimit)
        lam *= 2;
    return lam;
}

// Chain layout of a run: C chains per syndrome, plane width G, bundles of 32
// chains (G = 32: C/32 bundles per syndrome; G < 32: 32/G syndromes per
// bundle).
inline void init_chains(SweepParams& sp, int Cn, int R, uint32_t id0) {
    memset(&sp, 0, sizeof sp);
    int G = 1;
    while (G < Cn && G < 32) G *= 2;
    sp.C = Cn;
    sp.R = R;
    sp.G = G;
    sp.bps = G == 32 ? (Cn + 31) / 32 : 1;
    sp.spb = G == 32 ? 1 : 32 / G;
    sp.id0 = id0;
    sp.ids = nullptr;
}

inline long long bundles_of(const SweepParams& sp, long long n) {
    return sp.G == 32 ? n * sp.bps : (n + sp.spb - 1) / sp.spb;
}

// Appends a group of n syndromes of size L (items item_base ..) whose
// per-item rows start at the given word offsets.
inline void add_group(SweepParams& sp, int L, long long n, long long item_base, long long e0_off,
                      long long frames_off, long long state_off, int lam) {
    GroupDesc& g = sp.grp[sp.n_groups++];
    g.L = L;
    g.nq = geo_nq(sp.code, L);
    g.W = geo_words(sp.code, L);
    g.nc = geo_nc(sp.code, L);
    g.n = n;
    g.n_bundles = bundles_of(sp, n);
    g.item_base = item_base;
    g.e0_off = e0_off;
    g.frames_off = frames_off;
    g.state_off = state_off;
    g.unit_base = sp.total_units;
    sp.total_units += sweep_units(g.n_bundles, lam);
    if (g.nq > sp.grp_nq_max) sp.grp_nq_max = g.nq;
    if (g.nc > sp.grp_nc_max) sp.grp_nc_max = g.nc;
}

}  // namespace surfmcmc
