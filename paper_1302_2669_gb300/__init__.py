"""GB300 (sm_103a) single-temperature MCMC decoder for the planar surface code.

Thin Python binding over the C ABI of ``libsurfmcmc.so`` (declared in
``include/surfmcmc.h``): the names follow the C entry points, and every
function only marshals arguments.  Tensors may be torch tensors (CUDA or CPU)
or numpy arrays; CUDA tensors are passed as device pointers on the current
torch stream, everything else as host pointers.  There is no CPU fallback: if
the compiled library is missing, every call raises.

Reference: Hutter, Wootton, Loss, "An efficient Markov chain Monte Carlo
algorithm for the surface code", arXiv:1302.2669 (Sec. IV.A, algorithm C).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsurfmcmc.so")
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ENODEV = 0, -1, -2, -3, -4
MAX_L = 31


class SurfmcmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"surfmcmc error {code}: {msg}")
        self.code = code


class _Opts(C.Structure):
    _fields_ = [("n_classes", C.c_int32), ("chains_per_class", C.c_int32), ("n_sweeps", C.c_uint32),
                ("burn_in", C.c_uint32), ("beta_scale", C.c_double), ("lanes_per_bundle", C.c_int32),
                ("anneal_stages", C.c_int32), ("anneal_beta0", C.c_double), ("scan", C.c_int32),
                ("noise", C.c_int32), ("pauli_energy", C.c_int32 * 3)]


class _ServerOpts(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("slots", C.c_int32), ("max_L", C.c_int32), ("memory_budget", C.c_int64),
                ("max_wait_us", C.c_double)]


@dataclasses.dataclass
class Opts:
    """Mirror of ``surfmcmc_opts``."""
    n_classes: int = 4
    chains_per_class: int = 4
    n_sweeps: int = 2000
    burn_in: int = 0
    beta_scale: float = 1.0
    lanes_per_bundle: int = 0
    anneal_stages: int = 0
    anneal_beta0: float = 1.0
    scan: int = 0
    noise: int = 0
    pauli_energy: tuple = (1, 1, 1)

    def c(self) -> _Opts:
        return _Opts(self.n_classes, self.chains_per_class, self.n_sweeps, self.burn_in, self.beta_scale,
                     self.lanes_per_bundle, self.anneal_stages, self.anneal_beta0, self.scan, self.noise,
                     (C.c_int32 * 3)(*self.pauli_energy))


EXPORTS = ("surfmcmc_default_opts", "surfmcmc_create", "surfmcmc_destroy", "surfmcmc_strerror",
           "surfmcmc_last_error", "surfmcmc_gen_syndromes", "surfmcmc_gen_syndromes_noise",
           "surfmcmc_gen_syndromes_pauli", "surfmcmc_gen_syndromes_toric", "surfmcmc_start_frames", "surfmcmc_decode",
           "surfmcmc_decode_ex", "surfmcmc_set_timing", "surfmcmc_sweep_time", "surfmcmc_noalloc_scratch_needed",
           "surfmcmc_decode_noalloc", "surfmcmc_decode_ti", "surfmcmc_decode_ragged", "surfmcmc_ragged_plan_create",
           "surfmcmc_plan_launch", "surfmcmc_plan_destroy", "surfmcmc_autotune", "surfmcmc_server_default_opts",
           "surfmcmc_server_create", "surfmcmc_server_submit", "surfmcmc_server_poll", "surfmcmc_server_stats",
           "surfmcmc_server_destroy", "surfmcmc_cnn_n_params", "surfmcmc_cnn_create", "surfmcmc_cnn_destroy",
           "surfmcmc_cnn_set_params", "surfmcmc_cnn_get_params", "surfmcmc_cnn_forward", "surfmcmc_cnn_gradient",
           "surfmcmc_cnn_train_step", "surfmcmc_cnn_status", "surfmcmc_cnn_set_wait_limit", "surfmcmc_cnn_soft_targets",
           "surfmcmc_decode_early")
NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024
TUNE_LANES = (2, 4, 8, 16, 32)              # candidates of surfmcmc_autotune
TUNE_LANES_N = len(TUNE_LANES)
TUNE_BLOCKS = (6, 5, 4, 3)


def lib():
    """Loads libsurfmcmc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1302_2669_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, u32, u64, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
        L.surfmcmc_default_opts.argtypes = [C.POINTER(_Opts)]
        L.surfmcmc_default_opts.restype = None
        L.surfmcmc_create.argtypes = [C.POINTER(vp), C.c_int]
        L.surfmcmc_destroy.argtypes = [vp]
        L.surfmcmc_destroy.restype = None
        L.surfmcmc_strerror.argtypes = [C.c_int]
        L.surfmcmc_strerror.restype = C.c_char_p
        L.surfmcmc_last_error.argtypes = [vp]
        L.surfmcmc_last_error.restype = C.c_char_p
        L.surfmcmc_gen_syndromes.argtypes = [vp, u64, u32, i64, i32, dbl, vp, vp, vp]
        L.surfmcmc_gen_syndromes_noise.argtypes = [vp, u64, u32, i64, i32, dbl, i32, vp, vp, vp]
        L.surfmcmc_gen_syndromes_pauli.argtypes = [vp, u64, u32, i64, i32, dbl, dbl, dbl, vp, vp, vp]
        L.surfmcmc_gen_syndromes_toric.argtypes = [vp, u64, u32, i64, i32, dbl, vp, vp, vp]
        L.surfmcmc_start_frames.argtypes = [vp, vp, i64, i32, vp, vp, vp]
        L.surfmcmc_decode.argtypes = [vp, vp, i64, i32, dbl, C.POINTER(_Opts), u64, u32, vp, vp, vp, vp]
        L.surfmcmc_decode_ex.argtypes = [vp, vp, i64, i32, dbl, C.POINTER(_Opts), u64, u32, u32, vp, vp, vp, vp,
                                         vp, vp, vp, vp, vp, vp]
        L.surfmcmc_noalloc_scratch_needed.argtypes = [i64, i32, i32]
        L.surfmcmc_noalloc_scratch_needed.restype = C.c_size_t
        L.surfmcmc_decode_noalloc.argtypes = [vp, i64, i32, dbl, C.POINTER(_Opts), u64, u32, vp, vp, vp, vp]
        L.surfmcmc_decode_ti.argtypes = [vp, vp, i64, i32, dbl, C.POINTER(_Opts), i32, u64, u32, vp, vp, vp, vp]
        L.surfmcmc_decode_ragged.argtypes = [vp, vp, vp, vp, i64, dbl, C.POINTER(_Opts), u64, vp, u32, vp, vp, vp, vp]
        L.surfmcmc_ragged_plan_create.argtypes = [vp, vp, vp, i64, dbl, C.POINTER(_Opts), u64, vp, vp, u32, vp, vp, vp,
                                                  C.POINTER(vp)]
        L.surfmcmc_plan_launch.argtypes = [vp, vp]
        L.surfmcmc_server_default_opts.argtypes = [C.POINTER(_ServerOpts)]
        L.surfmcmc_server_default_opts.restype = None
        L.surfmcmc_server_create.argtypes = [C.c_int, dbl, C.POINTER(_Opts), u64, C.POINTER(_ServerOpts), C.POINTER(vp)]
        L.surfmcmc_server_submit.argtypes = [vp, u32, i32, u32, vp]
        L.surfmcmc_server_poll.argtypes = [vp, i64, vp, vp, vp, vp, C.POINTER(i64), i32]
        L.surfmcmc_server_stats.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        L.surfmcmc_server_destroy.argtypes = [vp]
        L.surfmcmc_server_destroy.restype = None
        L.surfmcmc_autotune.argtypes = [vp, i32, i32, dbl, i64, u32, C.POINTER(i32), C.POINTER(i32), C.POINTER(dbl)]
        L.surfmcmc_plan_destroy.argtypes = [vp]
        L.surfmcmc_plan_destroy.restype = None
        L.surfmcmc_cnn_n_params.argtypes = []
        L.surfmcmc_cnn_n_params.restype = i64
        L.surfmcmc_cnn_create.argtypes = [vp, i32, i64, C.POINTER(vp)]
        L.surfmcmc_cnn_destroy.argtypes = [vp]
        L.surfmcmc_cnn_destroy.restype = None
        L.surfmcmc_cnn_set_params.argtypes = [vp, vp]
        L.surfmcmc_cnn_get_params.argtypes = [vp, vp]
        L.surfmcmc_cnn_forward.argtypes = [vp, vp, i64, vp, vp]
        L.surfmcmc_cnn_gradient.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        L.surfmcmc_cnn_train_step.argtypes = [vp, vp, vp, i64, C.c_float, vp, vp]
        L.surfmcmc_cnn_status.argtypes = [vp, vp]
        L.surfmcmc_cnn_set_wait_limit.argtypes = [vp, u32]
        L.surfmcmc_cnn_soft_targets.argtypes = [vp, i64, vp, vp]
        L.surfmcmc_decode_early.argtypes = [vp, vp, vp, i64, i32, dbl, C.POINTER(_Opts), u32, C.c_float, i32, u64, u32,
                                            vp, vp, vp, vp]
        L.surfmcmc_set_timing.argtypes = [vp, C.c_int]
        L.surfmcmc_sweep_time.argtypes = [vp, C.POINTER(dbl), C.POINTER(i64)]
        _lib = L
    return _lib


def n_qubits(L: int) -> int:
    return 2 * L * L - 2 * L + 1


def n_stabs(L: int) -> int:
    return 2 * L * (L - 1)


def n_words(L: int) -> int:
    return (n_qubits(L) + 31) // 32


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _empty(like, shape, np_dtype):
    """Output buffer on the same side (torch CUDA / torch CPU / numpy) as `like`."""
    if like is not None and _is_torch(like):
        import torch
        tdt = {np.uint8: torch.uint8, np.int32: torch.int32, np.uint32: torch.uint32, np.uint64: torch.uint64,
               np.float64: torch.float64, np.float32: torch.float32}[np_dtype]
        return torch.empty(shape, dtype=tdt, device=like.device)
    return np.empty(shape, dtype=np_dtype)


def _stream_of(*xs):
    for x in xs:
        if x is not None and _is_torch(x) and x.is_cuda:
            import torch
            return torch.cuda.current_stream(x.device).cuda_stream
    return None


class Context:
    """One surfmcmc_ctx bound to a CUDA device."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        rc = lib().surfmcmc_create(C.byref(self._h), device)
        if rc != OK:
            raise SurfmcmcError(rc, lib().surfmcmc_strerror(rc).decode())
        self.device = device

    def close(self):
        if self._h:
            lib().surfmcmc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise SurfmcmcError(rc, lib().surfmcmc_last_error(self._h).decode() or
                                lib().surfmcmc_strerror(rc).decode())

    def gen_syndromes(self, seed, id0, n, L, p, like=None, syndromes=None, true_class=None, stream=None, noise=0):
        """surfmcmc_gen_syndromes(_noise); outputs are allocated beside `like` if not given."""
        if syndromes is None:
            syndromes = _empty(like, (n, n_stabs(L)), np.uint8)
        if true_class is None:
            true_class = _empty(like, (n,), np.int32)
        st = stream if stream is not None else _stream_of(syndromes)
        self._check(lib().surfmcmc_gen_syndromes_noise(self._h, seed, id0, n, L, p, noise, _ptr(syndromes),
                                                       _ptr(true_class), st))
        return syndromes, true_class

    def gen_syndromes_pauli(self, seed, id0, n, L, px, py, pz, like=None, syndromes=None, true_class=None,
                            stream=None):
        """surfmcmc_gen_syndromes_pauli: errors of a general Pauli channel."""
        if syndromes is None:
            syndromes = _empty(like, (n, n_stabs(L)), np.uint8)
        if true_class is None:
            true_class = _empty(like, (n,), np.int32)
        st = stream if stream is not None else _stream_of(syndromes)
        self._check(lib().surfmcmc_gen_syndromes_pauli(self._h, seed, id0, n, L, px, py, pz, _ptr(syndromes),
                                                       _ptr(true_class), st))
        return syndromes, true_class

    def gen_syndromes_toric(self, seed, id0, n, L, p, like=None, syndromes=None, true_class=None, stream=None):
        """surfmcmc_gen_syndromes_toric: depolarizing errors on the L x L torus."""
        if syndromes is None:
            syndromes = _empty(like, (n, 2 * L * L), np.uint8)
        if true_class is None:
            true_class = _empty(like, (n,), np.int32)
        st = stream if stream is not None else _stream_of(syndromes)
        self._check(lib().surfmcmc_gen_syndromes_toric(self._h, seed, id0, n, L, p, _ptr(syndromes),
                                                       _ptr(true_class), st))
        return syndromes, true_class

    def start_frames(self, syndromes, L, frames=None, e0_class=None, stream=None):
        """surfmcmc_start_frames; returns (frames [n][2][W] uint32, e0_class [n])."""
        n = syndromes.shape[0]
        if frames is None:
            frames = _empty(syndromes, (n, 2, n_words(L)), np.uint32)
        if e0_class is None:
            e0_class = _empty(syndromes, (n,), np.int32)
        st = stream if stream is not None else _stream_of(syndromes, frames)
        self._check(lib().surfmcmc_start_frames(self._h, _ptr(syndromes), n, L, _ptr(frames), _ptr(e0_class), st))
        return frames, e0_class

    def decode(self, syndromes, L, p, opts: Opts | None = None, seed=0, id0=0, out_class=None,
               out_class_sum=None, out_log_ratio=None, want_sums=True, stream=None):
        """surfmcmc_decode; returns (class, class_sum or None, log_ratio or None)."""
        opts = opts or Opts()
        n = syndromes.shape[0]
        K = opts.n_classes
        if out_class is None:
            out_class = _empty(syndromes, (n,), np.int32)
        if want_sums and out_class_sum is None:
            out_class_sum = _empty(syndromes, (n, K), np.uint64)
        if want_sums and out_log_ratio is None:
            out_log_ratio = _empty(syndromes, (n, K), np.float64)
        st = stream if stream is not None else _stream_of(syndromes, out_class)
        o = opts.c()
        self._check(lib().surfmcmc_decode(self._h, _ptr(syndromes), n, L, p, C.byref(o), seed, id0,
                                          _ptr(out_class), _ptr(out_class_sum), _ptr(out_log_ratio), st))
        return out_class, out_class_sum, out_log_ratio

    def decode_ex(self, syndromes, L, p, opts: Opts | None = None, seed=0, id0=0, sweep_begin=0,
                  init_frames=None, init_chain_sum=None, chain_sum=True, chain_n=True, chain_frames=True,
                  accepts=False, stream=None):
        """surfmcmc_decode_ex; returns a dict of the outputs (per-chain ones on request)."""
        opts = opts or Opts()
        n = syndromes.shape[0]
        K = opts.n_classes
        Cn = K * opts.chains_per_class
        out = {"cls": _empty(syndromes, (n,), np.int32), "class_sum": _empty(syndromes, (n, K), np.uint64),
               "log_ratio": _empty(syndromes, (n, K), np.float64)}
        out["chain_sum"] = _empty(syndromes, (n, Cn), np.uint64) if chain_sum else None
        out["chain_n"] = _empty(syndromes, (n, Cn), np.int32) if chain_n else None
        W = (2 * L * L + 31) // 32 if K == 16 else n_words(L)    # toric code: 2 L^2 qubits
        out["chain_frames"] = _empty(syndromes, (n, Cn, 2, W), np.uint32) if chain_frames else None
        out["accepts"] = _empty(syndromes, (n, Cn), np.uint64) if accepts else None
        st = stream if stream is not None else _stream_of(syndromes, out["cls"])
        o = opts.c()
        self._check(lib().surfmcmc_decode_ex(
            self._h, _ptr(syndromes), n, L, p, C.byref(o), seed, id0, sweep_begin, _ptr(init_frames),
            _ptr(init_chain_sum), _ptr(out["cls"]), _ptr(out["class_sum"]), _ptr(out["log_ratio"]),
            _ptr(out["chain_sum"]), _ptr(out["chain_n"]), _ptr(out["chain_frames"]), _ptr(out["accepts"]), st))
        return out

    def decode_ti(self, syndromes, L, p, opts: Opts | None = None, n_beta=21, seed=0, id0=0, stream=None):
        """surfmcmc_decode_ti; returns (class [n], log_z [n][4], mean [n][4][n_beta])."""
        opts = opts or Opts()
        n = syndromes.shape[0]
        K = opts.n_classes
        cls = _empty(syndromes, (n,), np.int32)
        lz = _empty(syndromes, (n, K), np.float64)
        mean = _empty(syndromes, (n, K, n_beta), np.float64)
        st = stream if stream is not None else _stream_of(syndromes, cls)
        o = opts.c()
        self._check(lib().surfmcmc_decode_ti(self._h, _ptr(syndromes), n, L, p, C.byref(o), n_beta, seed, id0,
                                             _ptr(cls), _ptr(lz), _ptr(mean), st))
        return cls, lz, mean

    def decode_ragged(self, syndromes, Ls, p, opts: Opts | None = None, n_sweeps=None, seed=0, ids=None, id0=0,
                      stream=None):
        """surfmcmc_decode_ragged; syndromes = concatenated rows; returns (class, class_sum, log_ratio)."""
        opts = opts or Opts()
        n = len(Ls)
        cls = _empty(syndromes, (n,), np.int32)
        csum = _empty(syndromes, (n, 4), np.uint64)
        lr = _empty(syndromes, (n, 4), np.float64)
        st = stream if stream is not None else _stream_of(syndromes, cls)
        o = opts.c()
        self._check(lib().surfmcmc_decode_ragged(self._h, _ptr(syndromes), _ptr(Ls), _ptr(n_sweeps), n, p, C.byref(o),
                                                 seed, _ptr(ids), id0, _ptr(cls), _ptr(csum), _ptr(lr), st))
        return cls, csum, lr

    def decode_early(self, net, syndromes, L, p, opts: Opts | None = None, chunk_sweeps=64, tau=float("inf"), seed=0,
                     id0=0, reorder=False, stream=None):
        """surfmcmc_decode_early; returns (class [n], class_sum [n][4], sweeps [n])."""
        opts = opts or Opts()
        n = syndromes.shape[0]
        cls = _empty(syndromes, (n,), np.int32)
        csum = _empty(syndromes, (n, 4), np.uint64)
        sw = _empty(syndromes, (n,), np.uint32)
        st = stream if stream is not None else _stream_of(syndromes, cls)
        o = opts.c()
        self._check(lib().surfmcmc_decode_early(self._h, net._h, _ptr(syndromes), n, L, p, C.byref(o), chunk_sweeps,
                                                tau, 1 if reorder else 0, seed, id0, _ptr(cls), _ptr(csum), _ptr(sw),
                                                st))
        return cls, csum, sw

    def autotune(self, L, chains_per_class, p, n_probe=4096, sweeps=20):
        """surfmcmc_autotune: returns (best lanes per bundle, best cap of resident
        blocks per multiprocessor, {(lanes, blocks): ms})."""
        best, best_b = C.c_int32(), C.c_int32()
        ms = (C.c_double * (TUNE_LANES_N * len(TUNE_BLOCKS)))()
        self._check(lib().surfmcmc_autotune(self._h, L, chains_per_class, p, n_probe, sweeps, C.byref(best),
                                            C.byref(best_b), ms))
        return best.value, best_b.value, {(lam, bb): ms[i * len(TUNE_BLOCKS) + j]
                                          for i, lam in enumerate(TUNE_LANES) for j, bb in enumerate(TUNE_BLOCKS)}

    def set_timing(self, enable: bool):
        """surfmcmc_set_timing: record CUDA events around every sweep kernel."""
        self._check(lib().surfmcmc_set_timing(self._h, 1 if enable else 0))

    def sweep_time(self):
        """surfmcmc_sweep_time: (summed sweep-kernel ms, launches) since the last query."""
        ms, n = C.c_double(), C.c_int64()
        self._check(lib().surfmcmc_sweep_time(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value


class RaggedPlan:
    """surfmcmc_ragged_plan_*: a ragged batch captured as a CUDA graph over
    fixed device buffers; launch() replays it on their current contents."""

    def __init__(self, ctx: Context, Ls, p, syndromes, out_class, out_class_sum=None, out_log_ratio=None,
                 opts: Opts | None = None, n_sweeps=None, seed=0, ids=None, id0=0):
        self._ctx = ctx
        self._h = C.c_void_p()
        self._keep = (Ls, n_sweeps, syndromes, ids, out_class, out_class_sum, out_log_ratio)
        o = (opts or Opts()).c()
        ctx._check(lib().surfmcmc_ragged_plan_create(ctx._h, _ptr(Ls), _ptr(n_sweeps), len(Ls), p, C.byref(o), seed,
                                                     _ptr(syndromes), _ptr(ids), id0, _ptr(out_class),
                                                     _ptr(out_class_sum), _ptr(out_log_ratio), C.byref(self._h)))

    def launch(self, stream=None):
        st = stream if stream is not None else _stream_of(self._keep[2])
        self._ctx._check(lib().surfmcmc_plan_launch(self._h, st))

    def close(self):
        if self._h:
            lib().surfmcmc_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """surfmcmc_server_*: continuous batching of single-syndrome requests."""

    def __init__(self, device=0, p=0.12, opts: Opts | None = None, seed=0, max_batch=256, slots=4, max_L=MAX_L,
                 memory_budget=0, max_wait_us=200.0):
        self._h = C.c_void_p()
        so = _ServerOpts(max_batch, slots, max_L, memory_budget, max_wait_us)
        o = (opts or Opts()).c()
        rc = lib().surfmcmc_server_create(device, p, C.byref(o), seed, C.byref(so), C.byref(self._h))
        if rc != OK:
            raise SurfmcmcError(rc, lib().surfmcmc_strerror(rc).decode())

    def submit(self, request_id: int, L: int, n_sweeps: int, syndrome: np.ndarray):
        syn = np.ascontiguousarray(syndrome, np.uint8)
        rc = lib().surfmcmc_server_submit(self._h, request_id, L, n_sweeps, syn.ctypes.data)
        if rc != OK:
            raise SurfmcmcError(rc, lib().surfmcmc_strerror(rc).decode())

    def poll(self, max_results=4096, wait_us=0):
        """Returns (ids, classes, class_sums [k][4], latency_us) of finished requests."""
        ids = np.empty(max_results, np.uint32)
        cls = np.empty(max_results, np.int32)
        sums = np.empty((max_results, 4), np.uint64)
        lat = np.empty(max_results, np.float64)
        n = C.c_int64()
        rc = lib().surfmcmc_server_poll(self._h, max_results, ids.ctypes.data, cls.ctypes.data, sums.ctypes.data,
                                        lat.ctypes.data, C.byref(n), wait_us)
        if rc != OK:
            raise SurfmcmcError(rc, lib().surfmcmc_strerror(rc).decode())
        k = n.value
        return ids[:k], cls[:k], sums[:k], lat[:k]

    def stats(self):
        a, b, m, q = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        lib().surfmcmc_server_stats(self._h, C.byref(a), C.byref(b), C.byref(m), C.byref(q))
        return {"admitted": a.value, "batches": b.value, "memory_stalls": m.value, "pending": q.value}

    def close(self):
        if self._h:
            lib().surfmcmc_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Network:
    """surfmcmc_cnn_*: the early-stop network (five 3x3 convolutions on the
    two syndrome maps, tensor-core forward and backward, Adam)."""

    def __init__(self, ctx: Context, L: int, max_batch: int = 4096):
        self._ctx = ctx
        self._h = C.c_void_p()
        self.L = L
        self.max_batch = max_batch
        ctx._check(lib().surfmcmc_cnn_create(ctx._h, L, max_batch, C.byref(self._h)))

    @staticmethod
    def n_params() -> int:
        return int(lib().surfmcmc_cnn_n_params())

    def set_params(self, params):
        """Float32 parameters (numpy or torch, host or device)."""
        if not _is_torch(params):
            params = np.ascontiguousarray(params, np.float32)
        self._ctx._check(lib().surfmcmc_cnn_set_params(self._h, _ptr(params)))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params(), np.float32)
        self._ctx._check(lib().surfmcmc_cnn_get_params(self._h, _ptr(out)))
        return out

    def forward(self, syndromes, out=None, stream=None):
        """Log-probabilities [n][4] (float32), beside `syndromes`."""
        n = syndromes.shape[0]
        if out is None:
            out = _empty(syndromes, (n, 4), np.float32)
        st = stream if stream is not None else _stream_of(syndromes, out)
        self._ctx._check(lib().surfmcmc_cnn_forward(self._h, _ptr(syndromes), n, _ptr(out), st))
        return out

    def gradient(self, syndromes, targets, stream=None):
        """(loss, flat gradient float32 numpy) of the batch."""
        n = syndromes.shape[0]
        loss = np.zeros(1, np.float32)
        grad = np.empty(self.n_params(), np.float32)
        st = stream if stream is not None else _stream_of(syndromes, targets)
        self._ctx._check(lib().surfmcmc_cnn_gradient(self._h, _ptr(syndromes), _ptr(targets), n, _ptr(loss),
                                                     _ptr(grad), st))
        return float(loss[0]), grad

    def train_step(self, syndromes, targets, lr, loss_out=None, stream=None):
        """One Adam step; returns the loss (float) unless `loss_out` (a device
        tensor of 1 float) receives it without a host wait."""
        n = syndromes.shape[0]
        st = stream if stream is not None else _stream_of(syndromes, targets)
        host = loss_out is None
        if host:
            loss_out = np.zeros(1, np.float32)
        self._ctx._check(lib().surfmcmc_cnn_train_step(self._h, _ptr(syndromes), _ptr(targets), n, lr,
                                                       _ptr(loss_out), st))
        return float(loss_out[0]) if host else None

    def status(self, stream=None):
        self._ctx._check(lib().surfmcmc_cnn_status(self._h, stream))

    def set_wait_limit(self, polls: int = 0):
        """surfmcmc_cnn_set_wait_limit: bound on each pipeline wait of the
        network kernels in polls (0: the default)."""
        self._ctx._check(lib().surfmcmc_cnn_set_wait_limit(self._h, int(polls)))

    @staticmethod
    def soft_targets(log_ratio, out=None, stream=None):
        """softmax of [n][4] float64 log-ratios (CUDA tensors) -> float32 targets."""
        n = log_ratio.shape[0]
        if out is None:
            out = _empty(log_ratio, (n, 4), np.float32)
        st = stream if stream is not None else _stream_of(log_ratio, out)
        rc = lib().surfmcmc_cnn_soft_targets(_ptr(log_ratio), n, _ptr(out), st)
        if rc != OK:
            raise SurfmcmcError(rc, lib().surfmcmc_strerror(rc).decode())
        return out

    def close(self):
        if self._h:
            lib().surfmcmc_cnn_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
