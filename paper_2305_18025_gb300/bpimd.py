"""Thin ctypes binding of the bpimd C ABI (``include/bpimd.h``).

Argument marshalling only: every step of the exchange computation runs in the
CUDA kernels of ``libbpimd.so``.  The functions keep the C names; tensors are
passed as ``torch.Tensor`` (their ``data_ptr()`` is handed to the library) and
streams as ``torch.cuda.Stream`` or raw handles.  There is no CPU fallback:
if the library cannot be loaded, every call raises.
"""
import ctypes
import os

from . import build as _build

BPIMD_OK = 0
BPIMD_ERR_ARG = -1
BPIMD_ERR_NONFINITE = -2
BPIMD_ERR_CUDA = -3
BPIMD_ERR_TIMEOUT = -4
BPIMD_ERR_NOMEM = -5
BPIMD_ERR_STATE = -6
BPIMD_ERR_SIZE = -7
BPIMD_NOALLOC_MAX_N = 256

BPIMD_FP64 = 0
BPIMD_MIXED = 1
BPIMD_MIXED32 = 2
PRECISIONS = {"fp64": BPIMD_FP64, "mixed": BPIMD_MIXED, "mixed32": BPIMD_MIXED32}
BPIMD_MAX_N = 16384
BPIMD_STORE_MAX_N = 8192
BPIMD_FLAG_RECOMPUTE = 1
BPIMD_FLAG_TEST_TIMEOUT = 2

BPIMD_PAIR_NONE = 0
BPIMD_PAIR_GAUSSIAN = 1
BPIMD_PAIR_LJ = 2

EXPORTED = [
    "bpimd_create", "bpimd_destroy", "bpimd_exchange_energy_forces",
    "bpimd_exchange_energy_forces_host", "bpimd_sync", "bpimd_get_potentials",
    "bpimd_connection_probabilities", "bpimd_step", "bpimd_status_string", "bpimd_version",
    "bpimd_profile_begin", "bpimd_profile_end", "bpimd_exchange_energy_forces_noalloc",
    "bpimd_create_batched", "bpimd_exchange_energy_forces_batched", "bpimd_batch_info",
    "bpimd_batch_set_tuning", "bpimd_batch_set_pair_tile", "bpimd_peak_probe", "bpimd_pow2_selftest",
]
BATCH_MAX_N = 4096
BPIMD_NUM_STAGES = 3
STAGE_NAMES = ["prep", "recursions", "prob_forces"]


class bpimd_config(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("P", ctypes.c_int32),
        ("m", ctypes.c_double), ("omega_P", ctypes.c_double), ("beta", ctypes.c_double),
        ("precision", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("dt", ctypes.c_double), ("gamma", ctypes.c_double), ("kT_bead", ctypes.c_double),
        ("omega0", ctypes.c_double),
        ("pair_type", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("pair_a", ctypes.c_double), ("pair_b", ctypes.c_double), ("pair_rc", ctypes.c_double),
        ("box_L", ctypes.c_double), ("seed", ctypes.c_uint64),
    ]


class BpimdError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {bpimd_status_string(status)} ({status})")


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libbpimd.so (building it first if asked); raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise ImportError(f"bpimd CUDA library missing: {_build.LIB}")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.bpimd_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(bpimd_config), vp]
    lib.bpimd_destroy.argtypes = [vp]
    lib.bpimd_exchange_energy_forces.argtypes = [vp, vp, vp, vp]
    lib.bpimd_exchange_energy_forces_host.argtypes = [vp, vp, vp, vp]
    lib.bpimd_sync.argtypes = [vp]
    lib.bpimd_get_potentials.argtypes = [vp, vp, vp, vp]
    lib.bpimd_connection_probabilities.argtypes = [vp, vp]
    lib.bpimd_step.argtypes = [vp, vp, vp, ctypes.c_int32, vp]
    lib.bpimd_status_string.argtypes = [ip]
    lib.bpimd_status_string.restype = ctypes.c_char_p
    lib.bpimd_version.restype = ctypes.c_char_p
    lib.bpimd_profile_begin.argtypes = [vp, ip]
    lib.bpimd_profile_end.argtypes = [vp, vp, vp]
    lib.bpimd_exchange_energy_forces_noalloc.argtypes = [ctypes.POINTER(bpimd_config), vp, vp, vp, vp]
    lib.bpimd_create_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(bpimd_config), ctypes.c_int32,
                                         vp, vp, vp, vp, vp]
    lib.bpimd_exchange_energy_forces_batched.argtypes = [vp, vp, vp, vp]
    lib.bpimd_batch_info.argtypes = [vp, vp, vp, vp]
    lib.bpimd_batch_set_tuning.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    lib.bpimd_batch_set_pair_tile.argtypes = [vp, ctypes.c_int32]
    lib.bpimd_peak_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, vp]
    lib.bpimd_pow2_selftest.argtypes = [ctypes.c_int32, vp, vp, ctypes.c_int32, vp]
    for name in EXPORTED:
        if name not in ("bpimd_status_string", "bpimd_version"):
            getattr(lib, name).restype = ip
    _lib = lib
    return lib


def _ptr(x):
    """Device/host address of a tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status, where):
    if status != BPIMD_OK:
        raise BpimdError(status, where)


def bpimd_status_string(status):
    return load().bpimd_status_string(int(status)).decode()


def bpimd_version():
    return load().bpimd_version().decode()


def bpimd_create(cfg, stream=None):
    """Create a context; returns its opaque handle (int)."""
    h = ctypes.c_void_p()
    _check(load().bpimd_create(ctypes.byref(h), ctypes.byref(cfg), _stream_handle(stream)), "bpimd_create")
    return h.value


def bpimd_destroy(ctx):
    _check(load().bpimd_destroy(ctx), "bpimd_destroy")


def bpimd_exchange_energy_forces(ctx, positions, V_B, forces):
    _check(load().bpimd_exchange_energy_forces(ctx, _ptr(positions), _ptr(V_B), _ptr(forces)),
           "bpimd_exchange_energy_forces")


def bpimd_exchange_energy_forces_host(ctx, positions, V_B, forces):
    _check(load().bpimd_exchange_energy_forces_host(ctx, _ptr(positions), _ptr(V_B), _ptr(forces)),
           "bpimd_exchange_energy_forces_host")


def bpimd_sync(ctx):
    _check(load().bpimd_sync(ctx), "bpimd_sync")


def bpimd_get_potentials(ctx, V_fwd, V_bwd, Eint):
    _check(load().bpimd_get_potentials(ctx, _ptr(V_fwd), _ptr(V_bwd), _ptr(Eint)), "bpimd_get_potentials")


def bpimd_connection_probabilities(ctx, M):
    _check(load().bpimd_connection_probabilities(ctx, _ptr(M)), "bpimd_connection_probabilities")


def bpimd_step(ctx, positions, velocities, nsteps, energies=None):
    _check(load().bpimd_step(ctx, _ptr(positions), _ptr(velocities), int(nsteps), _ptr(energies)),
           "bpimd_step")


def bpimd_profile_begin(ctx, max_evals):
    _check(load().bpimd_profile_begin(ctx, int(max_evals)), "bpimd_profile_begin")


def bpimd_profile_end(ctx):
    """Returns (per-stage summed milliseconds, number of evaluations)."""
    import numpy as np
    ms = np.zeros(BPIMD_NUM_STAGES)
    n = ctypes.c_int()
    _check(load().bpimd_profile_end(ctx, ms.ctypes.data, ctypes.byref(n)), "bpimd_profile_end")
    return ms, n.value


def bpimd_exchange_energy_forces_noalloc(cfg, positions, V_B, forces, stream=None):
    """Allocation-free evaluation (no context; fixed 1 MiB device scratch, N <= 256).

    For callers that cannot allocate device memory when they evaluate (their
    memory manager owns all device memory, or cudaMalloc's device-wide
    synchronisation is not allowed in their loop).  The first call on a device
    sets up the scratch address and should precede any stream capture; calls
    that overlap on the GPU race on the shared scratch."""
    _check(load().bpimd_exchange_energy_forces_noalloc(ctypes.byref(cfg), _ptr(positions), _ptr(V_B),
                                                       _ptr(forces), _stream_handle(stream)),
           "bpimd_exchange_energy_forces_noalloc")


def bpimd_create_batched(cfg, N, P, omega_P, beta, stream=None):
    """Batch context for replicas with per-replica N, P, omega_P, beta (host sequences)."""
    import numpy as np
    N = np.ascontiguousarray(N, dtype=np.int32)
    P = np.ascontiguousarray(P, dtype=np.int32)
    omega_P = np.ascontiguousarray(omega_P, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    R = len(N)
    if not (len(P) == len(omega_P) == len(beta) == R):
        raise ValueError("N, P, omega_P, beta must have the same length")
    h = ctypes.c_void_p()
    _check(load().bpimd_create_batched(ctypes.byref(h), ctypes.byref(cfg), R, N.ctypes.data, P.ctypes.data,
                                       omega_P.ctypes.data, beta.ctypes.data, _stream_handle(stream)),
           "bpimd_create_batched")
    return h.value


def bpimd_exchange_energy_forces_batched(ctx, positions, V_B, forces):
    _check(load().bpimd_exchange_energy_forces_batched(ctx, _ptr(positions), _ptr(V_B), _ptr(forces)),
           "bpimd_exchange_energy_forces_batched")


def bpimd_batch_info(ctx):
    """(R, total elements, element offsets of the replicas)."""
    import numpy as np
    R = ctypes.c_int32()
    n = ctypes.c_int64()
    _check(load().bpimd_batch_info(ctx, ctypes.byref(R), ctypes.byref(n), None), "bpimd_batch_info")
    off = np.zeros(R.value, dtype=np.int64)
    _check(load().bpimd_batch_info(ctx, None, None, off.ctypes.data), "bpimd_batch_info")
    return R.value, n.value, off


def bpimd_batch_set_pair_tile(ctx, lanes_per_particle):
    _check(load().bpimd_batch_set_pair_tile(ctx, int(lanes_per_particle)), "bpimd_batch_set_pair_tile")


def bpimd_batch_set_tuning(ctx, pair_blocks_per_sm, prob_blocks_per_sm):
    _check(load().bpimd_batch_set_tuning(ctx, int(pair_blocks_per_sm), int(prob_blocks_per_sm)),
           "bpimd_batch_set_tuning")


def make_config(N, P, m, omega_P, beta, precision=BPIMD_FP64, **md):
    cfg = bpimd_config()
    cfg.N, cfg.P, cfg.m, cfg.omega_P, cfg.beta = N, P, m, omega_P, beta
    cfg.precision = precision
    for k, v in md.items():
        setattr(cfg, k, v)
    return cfg


def bpimd_peak_probe(kind, iters, sink, stream=None):
    """Enqueue the throughput probe (kind 0: float64 FMA, 1: integer 32x32->64
    multiply-add); returns the number of multiply-adds it performs."""
    ops = ctypes.c_int64(0)
    _check(load().bpimd_peak_probe(int(kind), int(iters), _ptr(sink), _stream_handle(stream), ctypes.byref(ops)),
           "bpimd_peak_probe")
    return ops.value


def bpimd_pow2_selftest(method, x, out, stream=None):
    """out = 2^x (method 0, float64 table method) or 2^-x (method 1, integer
    fixed-point method), elementwise on device tensors."""
    _check(load().bpimd_pow2_selftest(int(method), _ptr(x), _ptr(out), int(x.numel()), _stream_handle(stream)),
           "bpimd_pow2_selftest")
