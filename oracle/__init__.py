"""CPU oracle of the single-temperature MCMC surface-code decoder (arXiv:1302.2669).

TEST INFRASTRUCTURE ONLY.  This package wraps ``oracle.c`` (plain C, one byte
per qubit, plain loops) through ctypes.  Only the tests, the smoke check and
the benchmark's CPU-baseline leg may import it; the product library never
does, and the two share no code.

Every function here is a thin marshalling wrapper; the arithmetic lives in
``oracle.c`` and cites the paper's sections and equations there.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with plain gcc -O2."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        L.orc_nq.argtypes = [C.c_int]
        L.orc_nstab.argtypes = [C.c_int]
        L.orc_stab_pos.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_stab_support.argtypes = [C.c_int, C.c_int, i32p]
        L.orc_stab_colour.argtypes = [C.c_int, C.c_int]
        L.orc_colour_count.argtypes = [C.c_int, C.c_int]
        L.orc_colour_member.argtypes = [C.c_int, C.c_int, C.c_int]
        L.orc_syndrome.argtypes = [C.c_int, u8p, u8p, u8p]
        L.orc_class_code.argtypes = [C.c_int, u8p, u8p]
        L.orc_apply_logical.argtypes = [C.c_int, C.c_int, u8p, u8p]
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_gen_error.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_double, u8p, u8p]
        L.orc_gen_syndromes.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int, C.c_double, u8p, i32p]
        L.orc_gen_syndromes_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int, C.c_double, C.c_int, u8p,
                                              i32p]
        L.orc_gen_error_flips.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_double, u8p, u8p]
        L.orc_thresholds_noise.argtypes = [C.c_double, C.c_int, C.c_double, u64p, C.POINTER(C.c_double)]
        L.orc_exact_histogram_noise.argtypes = [C.c_int, u8p, C.c_int, u64p]
        L.orc_exact_histogram_energy.argtypes = [C.c_int, u8p, C.c_int, C.c_void_p, C.c_int, u64p]
        L.orc_t_stab_pos.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_t_stab_support.argtypes = [C.c_int, C.c_int, i32p]
        L.orc_t_stab_colour.argtypes = [C.c_int, C.c_int]
        L.orc_t_syndrome.argtypes = [C.c_int, u8p, u8p, u8p]
        L.orc_t_class_code.argtypes = [C.c_int, u8p, u8p]
        L.orc_t_apply_logical.argtypes = [C.c_int, C.c_int, u8p, u8p]
        L.orc_t_pure_error.argtypes = [C.c_int, u8p, u8p, u8p]
        L.orc_t_start_frame.argtypes = [C.c_int, u8p, C.c_int, u8p, u8p]
        L.orc_t_gen_syndromes.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int, C.c_double, u8p, i32p]
        L.orc_t_exact_histogram.argtypes = [C.c_int, u8p, u64p]
        L.orc_rate_general.argtypes = [C.c_double, C.c_int, C.c_int, C.c_int]
        L.orc_rate_general.restype = C.c_double
        L.orc_thresholds_r.argtypes = [C.c_double, C.c_double, C.c_int, u64p, C.POINTER(C.c_double)]
        L.orc_gen_syndromes_pauli.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int, C.c_double, C.c_double,
                                              C.c_double, u8p, i32p]
        L.orc_pure_error.argtypes = [C.c_int, u8p, u8p, u8p]
        L.orc_start_frame.argtypes = [C.c_int, u8p, C.c_int, u8p, u8p]
        L.orc_thresholds.argtypes = [C.c_double, C.c_double, u64p, C.POINTER(C.c_double)]
        L.orc_plane_width.argtypes = [C.c_int]
        L.orc_chain_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_chain_uniform.restype = C.c_uint32
        L.orc_chain_uniform_less.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, C.c_int,
                                             C.c_int, C.c_uint64]
        L.orc_run_chains.argtypes = [C.c_void_p, u8p, C.c_int, u8p, u8p, u64p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_decide.argtypes = [C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_uint32, C.c_double, u64p, u64p, f64p]
        L.orc_decode_one.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_double,
                                     C.c_int, C.c_double, C.c_uint64, C.c_uint32, u8p, u64p, f64p, u64p, i32p, u8p,
                                     u8p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.orc_anneal_scale.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int]
        L.orc_anneal_scale.restype = C.c_double
        L.orc_anneal_stage.argtypes = [C.c_uint32, C.c_uint32, C.c_int]
        L.orc_exact_histogram.argtypes = [C.c_int, u8p, u64p]
        L.orc_simpson_integral.argtypes = [C.c_int, C.c_int, f64p, C.c_double, f64p]
        L.orc_decode_ti.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_double,
                                    C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_uint32, u8p, f64p, f64p, C.c_int,
                                    C.c_int, C.c_void_p]
        _lib = L
    return _lib


class _Run(C.Structure):
    _fields_ = [("L", C.c_int32), ("K", C.c_int32), ("R", C.c_int32), ("t_begin", C.c_uint32),
                ("t_end", C.c_uint32), ("burn_in", C.c_uint32), ("p", C.c_double), ("beta_scale", C.c_double),
                ("seed", C.c_uint64), ("id", C.c_uint32), ("anneal_stages", C.c_int32),
                ("anneal_beta0", C.c_double), ("scan", C.c_int32), ("noise", C.c_int32),
                ("energy", C.c_int32 * 3)]


def _energy(noise, energy):
    """int32[3] array (eX, eY, eZ) for the general channel, else None."""
    if noise != 2:
        return None
    return np.ascontiguousarray(energy if energy is not None else (1, 1, 1), np.int32)


def nq(L: int) -> int:
    return lib().orc_nq(L)


def nstab(L: int) -> int:
    return lib().orc_nstab(L)


def words(L: int) -> int:
    return (nq(L) + 31) // 32


def stab_pos(L: int, g: int):
    r, c = C.c_int(), C.c_int()
    t = lib().orc_stab_pos(L, g, C.byref(r), C.byref(c))
    return t, r.value, c.value


def stab_support(L: int, g: int) -> np.ndarray:
    q = np.zeros(4, np.int32)
    w = lib().orc_stab_support(L, g, q)
    return q[:w].copy()


def stab_colour(L: int, g: int) -> int:
    return lib().orc_stab_colour(L, g)


def colour_count(L: int, col: int) -> int:
    return lib().orc_colour_count(L, col)


def colour_member(L: int, col: int, m: int) -> int:
    return lib().orc_colour_member(L, col, m)


def syndrome(L: int, ex: np.ndarray, ez: np.ndarray) -> np.ndarray:
    s = np.zeros(nstab(L), np.uint8)
    lib().orc_syndrome(L, np.ascontiguousarray(ex, np.uint8), np.ascontiguousarray(ez, np.uint8), s)
    return s


def class_code(L: int, ex: np.ndarray, ez: np.ndarray) -> int:
    return lib().orc_class_code(L, np.ascontiguousarray(ex, np.uint8), np.ascontiguousarray(ez, np.uint8))


def apply_logical(L: int, k: int, ex: np.ndarray, ez: np.ndarray):
    ex = np.array(ex, np.uint8)
    ez = np.array(ez, np.uint8)
    lib().orc_apply_logical(L, k, ex, ez)
    return ex, ez


def philox(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32), np.ascontiguousarray(key, np.uint32), out)
    return out


def gen_error(seed: int, ident: int, L: int, p: float):
    ex = np.zeros(nq(L), np.uint8)
    ez = np.zeros(nq(L), np.uint8)
    lib().orc_gen_error(seed, ident, L, p, ex, ez)
    return ex, ez


def gen_syndromes(seed: int, id0: int, n: int, L: int, p: float, noise: int = 0):
    syn = np.zeros((n, nstab(L)), np.uint8)
    tc = np.zeros(n, np.int32)
    if n:
        lib().orc_gen_syndromes_noise(seed, id0, n, L, p, noise, syn, tc)
    return syn, tc


def gen_error_flips(seed: int, ident: int, L: int, p: float):
    ex = np.zeros(nq(L), np.uint8)
    ez = np.zeros(nq(L), np.uint8)
    lib().orc_gen_error_flips(seed, ident, L, p, ex, ez)
    return ex, ez


def pure_error(L: int, syn: np.ndarray):
    ex = np.zeros(nq(L), np.uint8)
    ez = np.zeros(nq(L), np.uint8)
    lib().orc_pure_error(L, np.ascontiguousarray(syn, np.uint8), ex, ez)
    return ex, ez


def start_frame(L: int, syn: np.ndarray, k: int):
    ex = np.zeros(nq(L), np.uint8)
    ez = np.zeros(nq(L), np.uint8)
    code0 = lib().orc_start_frame(L, np.ascontiguousarray(syn, np.uint8), k, ex, ez)
    return ex, ez, code0


# --- toric code (16 classes) -------------------------------------------------
def t_nq(L: int) -> int:
    return 2 * L * L


def t_nstab(L: int) -> int:
    return 2 * L * L


def t_stab_pos(L: int, g: int):
    r, c = C.c_int(), C.c_int()
    t = lib().orc_t_stab_pos(L, g, C.byref(r), C.byref(c))
    return t, r.value, c.value


def t_stab_support(L: int, g: int) -> np.ndarray:
    q = np.zeros(4, np.int32)
    lib().orc_t_stab_support(L, g, q)
    return q


def t_stab_colour(L: int, g: int) -> int:
    return lib().orc_t_stab_colour(L, g)


def t_syndrome(L: int, ex, ez) -> np.ndarray:
    s = np.zeros(t_nstab(L), np.uint8)
    lib().orc_t_syndrome(L, np.ascontiguousarray(ex, np.uint8), np.ascontiguousarray(ez, np.uint8), s)
    return s


def t_class_code(L: int, ex, ez) -> int:
    return lib().orc_t_class_code(L, np.ascontiguousarray(ex, np.uint8), np.ascontiguousarray(ez, np.uint8))


def t_apply_logical(L: int, k: int, ex, ez):
    ex = np.array(ex, np.uint8)
    ez = np.array(ez, np.uint8)
    lib().orc_t_apply_logical(L, k, ex, ez)
    return ex, ez


def t_pure_error(L: int, syn):
    ex = np.zeros(t_nq(L), np.uint8)
    ez = np.zeros(t_nq(L), np.uint8)
    lib().orc_t_pure_error(L, np.ascontiguousarray(syn, np.uint8), ex, ez)
    return ex, ez


def t_start_frame(L: int, syn, k: int):
    ex = np.zeros(t_nq(L), np.uint8)
    ez = np.zeros(t_nq(L), np.uint8)
    code0 = lib().orc_t_start_frame(L, np.ascontiguousarray(syn, np.uint8), k, ex, ez)
    return ex, ez, code0


def t_gen_syndromes(seed: int, id0: int, n: int, L: int, p: float):
    syn = np.zeros((n, t_nstab(L)), np.uint8)
    tc = np.zeros(n, np.int32)
    if n:
        lib().orc_t_gen_syndromes(seed, id0, n, L, p, syn, tc)
    return syn, tc


def t_exact_histogram(L: int, syn) -> np.ndarray:
    h = np.zeros((16, t_nq(L) + 1), np.uint64)
    if lib().orc_t_exact_histogram(L, np.ascontiguousarray(syn, np.uint8), h) != 0:
        raise ValueError("exact enumeration needs n_stab <= 30")
    return h


def rate_general(p: float, energy) -> float:
    """r = e^{-beta_bar} of the general channel with energies (eX, eY, eZ)."""
    return lib().orc_rate_general(p, int(energy[0]), int(energy[1]), int(energy[2]))


def thresholds_r(r: float, beta_scale: float = 1.0, dmax: int = 32):
    T = np.zeros(dmax + 1, np.uint64)
    bb = C.c_double()
    lib().orc_thresholds_r(r, beta_scale, dmax, T, C.byref(bb))
    return T, bb.value


def gen_syndromes_pauli(seed: int, id0: int, n: int, L: int, px: float, py: float, pz: float):
    syn = np.zeros((n, nstab(L)), np.uint8)
    tc = np.zeros(n, np.int32)
    if n:
        lib().orc_gen_syndromes_pauli(seed, id0, n, L, px, py, pz, syn, tc)
    return syn, tc


def pauli_probs(p: float, energy):
    """(pX, pY, pZ) of the general channel of total error probability p."""
    r = rate_general(p, energy)
    return tuple((1.0 - p) * r ** int(e) for e in energy)


def thresholds(p: float, beta_scale: float = 1.0, noise: int = 0):
    T = np.zeros(5, np.uint64)
    bb = C.c_double()
    lib().orc_thresholds_noise(p, noise, beta_scale, T, C.byref(bb))
    return T, bb.value


def plane_width(Cn: int) -> int:
    return lib().orc_plane_width(Cn)


def chain_uniform(seed, s, t, col, m, c, Cn) -> int:
    return lib().orc_chain_uniform(seed, s, t, col, m, c, Cn)


def chain_uniform_less(seed, s, t, col, m, c, Cn, T) -> bool:
    return bool(lib().orc_chain_uniform_less(seed, s, t, col, m, c, Cn, int(T)))


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """Pack a [..., nq] 0/1 array into [..., ceil(nq/32)] uint32 words, qubit q
    at bit q % 32 of word q // 32 (the library's frame layout)."""
    bits = np.asarray(bits, np.uint8)
    n = bits.shape[-1]
    W = (n + 31) // 32
    pad = np.zeros(bits.shape[:-1] + (W * 32,), np.uint8)
    pad[..., :n] = bits
    pad = pad.reshape(bits.shape[:-1] + (W, 32)).astype(np.uint32)
    return (pad << np.arange(32, dtype=np.uint32)).sum(axis=-1, dtype=np.uint64).astype(np.uint32)


def run_chains(L, K, R, p, seed, ident, syn, t_begin, t_end, burn_in=0, beta_scale=1.0,
               frames=None, chain_sum=None, trace=False, accepts=False, anneal_stages=0, anneal_beta0=1.0, scan=0,
               noise=0, energy=None):
    """Run all K*R chains of one syndrome from sweep t_begin to t_end.  With
    frames=None the chains start from the start frames of `syn`; otherwise
    frames = (fx, fz) [C][nq] uint8 is the state at t_begin.  Returns a dict
    with frames_x/z, chain_sum, chain_n and optionally the colour-phase trace
    of chain 0 and accept counts."""
    Cn = K * R
    n = t_nq(L) if K == 16 else nq(L)
    fx = np.zeros((Cn, n), np.uint8) if frames is None else np.array(frames[0], np.uint8)
    fz = np.zeros((Cn, n), np.uint8) if frames is None else np.array(frames[1], np.uint8)
    cs = np.zeros(Cn, np.uint64) if chain_sum is None else np.array(chain_sum, np.uint64)
    cn = np.zeros(Cn, np.int32)
    acc = np.zeros(Cn, np.uint64) if accepts else None
    tr = np.zeros(4 * (t_end - t_begin), np.int32) if trace else None
    a = _Run(L, K, R, t_begin, t_end, burn_in, p, beta_scale, seed, ident, anneal_stages, anneal_beta0, scan, noise,
             (C.c_int32 * 3)(*(energy if energy is not None else (1, 1, 1))))
    lib().orc_run_chains(C.addressof(a), np.ascontiguousarray(syn, np.uint8), 1 if frames is None else 0,
                         fx, fz, cs, cn.ctypes.data, None if acc is None else acc.ctypes.data,
                         None if tr is None else tr.ctypes.data)
    out = {"frames_x": fx, "frames_z": fz, "chain_sum": cs, "chain_n": cn}
    if trace:
        out["trace"] = tr
    if accepts:
        out["accepts"] = acc
    return out


def decide(K, R, n_sweeps, burn_in, beta_bar, chain_sum, samples_per_sweep=4):
    cs = np.ascontiguousarray(chain_sum, np.uint64)
    S = np.zeros(K, np.uint64)
    lr = np.zeros(K, np.float64)
    k = lib().orc_decide(K, R, n_sweeps, burn_in, samples_per_sweep, beta_bar, cs, S, lr)
    return k, S, lr


def decode_one(L, p, K, R, n_sweeps, seed, ident, syn, burn_in=0, beta_scale=1.0, accepts=False,
               anneal_stages=0, anneal_beta0=1.0, scan=0, noise=0, energy=None):
    """Decode one syndrome; returns a dict with the chosen class, per-class
    sums and log-ratios, per-chain sums, final n and final frames."""
    Cn = K * R
    n = t_nq(L) if K == 16 else nq(L)
    S = np.zeros(K, np.uint64)
    lr = np.zeros(K, np.float64)
    cs = np.zeros(Cn, np.uint64)
    cn = np.zeros(Cn, np.int32)
    fx = np.zeros((Cn, n), np.uint8)
    fz = np.zeros((Cn, n), np.uint8)
    acc = np.zeros(Cn, np.uint64) if accepts else None
    k = lib().orc_decode_one(L, p, K, R, n_sweeps, burn_in, beta_scale, anneal_stages, anneal_beta0, seed, ident,
                             np.ascontiguousarray(syn, np.uint8), S, lr, cs, cn, fx, fz,
                             None if acc is None else acc.ctypes.data, scan, noise,
                             None if noise != 2 else _energy(noise, energy).ctypes.data)
    out = {"cls": k, "class_sum": S, "log_ratio": lr, "chain_sum": cs, "chain_n": cn,
           "frames_x": fx, "frames_z": fz}
    if accepts:
        out["accepts"] = acc
    return out


def exact_histogram(L: int, syn: np.ndarray, noise: int = 0, energy=None) -> np.ndarray:
    """[4][nmax+1] counts of frames with n = w in each class (L <= 4); n is
    the number of qubits in error (noise 0), of bit plus phase flips (noise
    1, nmax = 2 nq) or the summed Pauli energies (noise 2, nmax = max(e) nq)."""
    emax = max(energy) if noise == 2 else (2 if noise else 1)
    h = np.zeros((4, emax * nq(L) + 1), np.uint64)
    e = _energy(noise, energy)
    rc = lib().orc_exact_histogram_energy(L, np.ascontiguousarray(syn, np.uint8), noise,
                                          None if e is None else e.ctypes.data, h.shape[1], h)
    if rc != 0:
        raise ValueError("exact enumeration needs n_stab <= 30")
    return h


def exact_class_stats(L: int, syn: np.ndarray, beta: float, noise: int = 0, energy=None):
    """log Z_k(beta) (Eq. 3, up to the common factor) and <n>_{beta,k} (Eq. 4)
    from the exact histogram."""
    h = exact_histogram(L, syn, noise, energy).astype(np.float64)
    n = np.arange(h.shape[1], dtype=np.float64)
    logw = -beta * n
    m = logw.max()
    Z = (h * np.exp(logw - m)).sum(axis=1)
    mean = (h * n * np.exp(logw - m)).sum(axis=1) / Z
    return np.log(Z) + m, mean


def _decode_worker(args):
    (L, p, K, R, n_sweeps, seed, ident, syn, burn_in, beta_scale, anneal_stages, anneal_beta0, scan, noise,
     energy) = args
    d = decode_one(L, p, K, R, n_sweeps, seed, ident, syn, burn_in=burn_in, beta_scale=beta_scale,
                   anneal_stages=anneal_stages, anneal_beta0=anneal_beta0, scan=scan, noise=noise, energy=energy)
    return d


def anneal_scale(beta_scale, a0, j, S):
    return lib().orc_anneal_scale(beta_scale, a0, j, S)


def anneal_stage(t, B, S):
    return lib().orc_anneal_stage(t, B, S)


def decode_batch(L, p, K, R, n_sweeps, seed, ids, syns, burn_in=0, beta_scale=1.0, processes=None,
                 anneal_stages=0, anneal_beta0=1.0, scan=0, noise=0, energy=None):
    """decode_one over many syndromes, one process per syndrome block
    (multiprocessing with the spawn start method, safe after CUDA use).
    Returns the list of per-syndrome result dicts in input order."""
    import multiprocessing as mp
    jobs = [(L, p, K, R, n_sweeps, seed, int(i), np.ascontiguousarray(s, np.uint8), burn_in, beta_scale,
             anneal_stages, anneal_beta0, scan, noise, energy) for i, s in zip(ids, syns)]
    if processes == 1 or len(jobs) <= 1:
        return [_decode_worker(j) for j in jobs]
    with mp.get_context("spawn").Pool(processes or os.cpu_count()) as pool:
        return pool.map(_decode_worker, jobs, chunksize=1)


def simpson_integral(mean, beta_bar):
    """Composite Simpson integral over the grid beta_j = j beta_bar/(N-1) of
    mean[k][j] (Eq. 6); returns I[k]."""
    mean = np.ascontiguousarray(mean, np.float64)
    K, N = mean.shape
    I = np.zeros(K, np.float64)
    if lib().orc_simpson_integral(K, N, mean, beta_bar, I) != 0:
        raise ValueError("Simpson needs an odd number >= 3 of grid points")
    return I


def decode_ti(L, p, K, R, n_sweeps, seed, ident, syn, n_beta=21, burn_in=0, beta_scale=1.0, anneal_stages=0,
              anneal_beta0=1.0, scan=0, noise=0, energy=None):
    """Thermodynamic-integration decode (Eq. 6, Simpson over n_beta points):
    returns (class, log Z_k - max log Z, means [K][n_beta])."""
    mean = np.zeros((K, n_beta), np.float64)
    lz = np.zeros(K, np.float64)
    k = lib().orc_decode_ti(L, p, K, R, n_sweeps, burn_in, beta_scale, anneal_stages, anneal_beta0, n_beta, seed,
                            ident, np.ascontiguousarray(syn, np.uint8), mean, lz, scan, noise,
                            None if noise != 2 else _energy(noise, energy).ctypes.data)
    if k < 0:
        raise ValueError("bad TI arguments")
    return k, lz, mean
