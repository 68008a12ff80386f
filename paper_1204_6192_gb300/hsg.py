"""Python binding of libhsg (include/hsg.h): argument marshalling only.

Every step of the Monte Carlo path runs inside the CUDA library; this module
converts numpy arrays to plain pointers and C status codes to exceptions.
There is no fallback: if libhsg.so is missing or cannot be loaded, every call
raises.  Method names follow the C entry points (``hsg_sweep_or`` ->
``Context.sweep_or`` and so on); the module-level ``hsg_*`` functions are the
C names themselves.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsg.so")

PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2, "angle16": 3, "oct16": 4, "yx4": 5}
STATUS = {0: "HSG_OK", 1: "HSG_EINVAL", 2: "HSG_ENOMEM", 3: "HSG_ECUDA", 4: "HSG_ETIMEOUT",
          5: "HSG_ESTATE"}
VARIANT_AUTO, VARIANT_TWO_PASS, VARIANT_PERSISTENT = 0, 1, 2
SWEEP_AUTO, SWEEP_HALF, SWEEP_FUSED, SWEEP_WAVE, SWEEP_STAGED = 0, 1, 2, 3, 4


class HsgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("j_fp16", ctypes.c_int), ("fast_math", ctypes.c_int),
                ("n_hb_per_step", ctypes.c_int), ("n_or_per_step", ctypes.c_int),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("variant", ctypes.c_int),
                ("barrier_timeout_ms", ctypes.c_int), ("inject_barrier_fault", ctypes.c_int),
                ("pass_bytes", ctypes.c_longlong), ("chunks_per_thread", ctypes.c_int),
                ("sweep_kernel", ctypes.c_int), ("wave_lag", ctypes.c_int),
                ("inject_alloc_fault", ctypes.c_int)]


class Obs(ctypes.Structure):
    _fields_ = [("E", ctypes.POINTER(ctypes.c_double)), ("q", ctypes.POINTER(ctypes.c_double)),
                ("qk", ctypes.POINTER(ctypes.c_double)), ("perm", ctypes.POINTER(ctypes.c_int32))]


class Info(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int), ("n_temps", ctypes.c_int), ("n_replicas", ctypes.c_int),
                ("W", ctypes.c_int), ("Wp", ctypes.c_int), ("precision", ctypes.c_int),
                ("j_fp16", ctypes.c_int), ("variant", ctypes.c_int),
                ("total_sites", ctypes.c_longlong), ("total_spins", ctypes.c_longlong),
                ("spin_bytes", ctypes.c_longlong), ("rec_bytes", ctypes.c_longlong),
                ("sweep_count", ctypes.c_uint64), ("pt_count", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("chunks_per_thread", ctypes.c_int),
                ("n_passes", ctypes.c_int), ("pass_bytes", ctypes.c_longlong),
                ("n_overlap_pairs", ctypes.c_int), ("sweep_kernel", ctypes.c_int),
                ("fused_band_rows", ctypes.c_int), ("fused_items", ctypes.c_int),
                ("wave_lag", ctypes.c_int), ("staged", ctypes.c_int)]


_lib = None


def use_library(path: str):
    """Load this build of the library instead of libhsg.so (e.g. libhsg_check.so,
    the build with device bounds checks); call before anything else of this module."""
    global LIB_PATH
    if _lib is not None:
        raise RuntimeError("the library is already loaded")
    LIB_PATH = path


def lib() -> ctypes.CDLL:
    """Load libhsg.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhsg.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    ctxpp = ctypes.POINTER(ctypes.c_void_p)
    fpp = ctypes.POINTER(fp)
    sigs = {
        "hsg_default_options": (None, [ctypes.POINTER(Options)]),
        "hsg_create": (ip, [ctxpp, ip, dp, ip, ip, fp, fp, ctypes.c_uint64, ctypes.POINTER(Options)]),
        "hsg_create_batch": (ip, [ctxpp, ip, ctypes.POINTER(ctypes.c_int), dp, ip, ip, fpp, fpp,
                                  ctypes.c_uint64, ctypes.POINTER(Options)]),
        "hsg_sweep_or": (ip, [vp, ip]),
        "hsg_sweep_hb": (ip, [vp, ip]),
        "hsg_pt_exchange": (ip, [vp]),
        "hsg_pt_exchange_energies": (ip, [vp, dp]),
        "hsg_step": (ip, [vp, ip]),
        "hsg_step_multihit": (ip, [vp, ip, ip, ip, ip, ip]),
        "hsg_energies": (ip, [vp, dp]),
        "hsg_last_energies": (ip, [vp, dp]),
        "hsg_measure": (ip, [vp, ctypes.POINTER(Obs)]),
        "hsg_measure_overlaps": (ip, [vp, dp, dp]),
        "hsg_get_spins": (ip, [vp, fp]),
        "hsg_set_spins": (ip, [vp, fp]),
        "hsg_get_spins_dev": (ip, [vp, vp]),
        "hsg_set_spins_dev": (ip, [vp, vp]),
        "hsg_get_perm": (ip, [vp, ctypes.POINTER(ctypes.c_int32)]),
        "hsg_get_pt_stats": (ip, [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
        "hsg_get_info": (ip, [vp, ctypes.POINTER(Info)]),
        "hsg_get_pt_diagnostics": (ip, [vp, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)]),
        "hsg_set_active": (ip, [vp, ctypes.POINTER(ctypes.c_uint8)]),
        "hsg_get_counters": (ip, [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
        "hsg_checkpoint_size": (ip, [vp, ctypes.POINTER(ctypes.c_size_t)]),
        "hsg_checkpoint_save": (ip, [vp, vp, ctypes.c_size_t]),
        "hsg_checkpoint_load": (ip, [vp, vp, ctypes.c_size_t]),
        "hsg_sync": (ip, [vp]),
        "hsg_last_error": (ctypes.c_char_p, [vp]),
        "hsg_status_string": (ctypes.c_char_p, [ip]),
        "hsg_destroy": (None, [vp]),
        "hsg_energies_xyz_noalloc": (ip, [vp, vp, vp, ip, ip, vp, vp]),
        "hsg_philox": (ip, [ctypes.POINTER(ctypes.c_uint32), ctypes.c_longlong, ctypes.c_uint64,
                            ctypes.POINTER(ctypes.c_uint32)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def default_options() -> Options:
    o = Options()
    lib().hsg_default_options(ctypes.byref(o))
    return o


class Context:
    """One hsg_ctx: a batch of disorder samples updated together on one GPU.

    ``samples``: objects with L, J [N,3], H [N,3] or None, temps [n_temps].
    """

    def __init__(self, samples: Sequence, n_replicas: int, seed: int, precision: str = "fp32",
                 j_fp16: bool = False, fast_math: bool = False, n_hb: int = 1, n_or: int = 5,
                 device: int = 0, stream: Optional[int] = None, variant: int = VARIANT_AUTO,
                 barrier_timeout_ms: int = 2000, inject_barrier_fault: bool = False,
                 pass_bytes: int = 0, chunks_per_thread: int = 0, sweep_kernel: int = SWEEP_AUTO,
                 wave_lag: int = 0, inject_alloc_fault: int = 0):
        L = lib()
        self._ctx = ctypes.c_void_p()
        opt = default_options()
        opt.precision = PRECISIONS[precision]
        opt.j_fp16 = int(bool(j_fp16))
        opt.fast_math = int(bool(fast_math))
        opt.n_hb_per_step = n_hb
        opt.n_or_per_step = n_or
        opt.device = device
        opt.stream = stream
        opt.variant = variant
        opt.barrier_timeout_ms = barrier_timeout_ms
        opt.inject_barrier_fault = int(bool(inject_barrier_fault))
        opt.pass_bytes = int(pass_bytes)
        opt.chunks_per_thread = int(chunks_per_thread)
        opt.sweep_kernel = int(sweep_kernel)
        opt.wave_lag = int(wave_lag)
        opt.inject_alloc_fault = int(inject_alloc_fault)
        self.samples = list(samples)
        self.n_samples = len(self.samples)
        self.n_temps = len(self.samples[0].temps)
        self.n_replicas = n_replicas
        self.W = self.n_temps * n_replicas
        self.Ls = [int(s.L) for s in self.samples]
        self.Ns = [l ** 3 for l in self.Ls]
        self.precision = precision
        # keep the float32 copies alive for the call
        Js = [np.ascontiguousarray(s.J, dtype=np.float32) for s in self.samples]
        Hs = [None if s.H is None else np.ascontiguousarray(s.H, dtype=np.float32) for s in self.samples]
        temps = np.ascontiguousarray(np.concatenate([np.asarray(s.temps, dtype=np.float64)
                                                     for s in self.samples]))
        fptr = ctypes.POINTER(ctypes.c_float)
        Jp = (fptr * self.n_samples)(*[_ptr(j, ctypes.c_float) for j in Js])
        Hp = (fptr * self.n_samples)(*[(_ptr(h, ctypes.c_float) if h is not None else fptr())
                                       for h in Hs])
        Ls = (ctypes.c_int * self.n_samples)(*self.Ls)
        st = L.hsg_create_batch(ctypes.byref(self._ctx), self.n_samples, Ls, _ptr(temps, ctypes.c_double),
                                self.n_temps, n_replicas, Jp, Hp, ctypes.c_uint64(seed),
                                ctypes.byref(opt))
        if st != 0:
            raise HsgError(st, (L.hsg_last_error(None) or b"").decode())

    # -- helpers ----------------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            raise HsgError(st, (lib().hsg_last_error(self._ctx) or b"").decode())

    @property
    def handle(self):
        return self._ctx

    def close(self):
        if self._ctx:
            lib().hsg_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the C entry points -----------------------------------------------------
    def sweep_or(self, n: int = 1):
        self._check(lib().hsg_sweep_or(self._ctx, n))

    def sweep_hb(self, n: int = 1):
        self._check(lib().hsg_sweep_hb(self._ctx, n))

    def pt_exchange(self):
        self._check(lib().hsg_pt_exchange(self._ctx))

    def pt_exchange_energies(self, E_sys: np.ndarray):
        E = np.ascontiguousarray(E_sys, dtype=np.float64).reshape(self.n_samples, self.W)
        self._check(lib().hsg_pt_exchange_energies(self._ctx, _ptr(E, ctypes.c_double)))

    def step_multihit(self, n: int = 1, tile: int = 8, n_rounds: int = 10, n_or: int = 10,
                      n_hb: int = 1):
        """n steps of the multi-hit tile schedule (hsg_step_multihit)."""
        self._check(lib().hsg_step_multihit(self._ctx, n, tile, n_rounds, n_or, n_hb))

    def step(self, n: int = 1):
        self._check(lib().hsg_step(self._ctx, n))

    def energies(self) -> np.ndarray:
        E = np.zeros((self.n_samples, self.W))
        self._check(lib().hsg_energies(self._ctx, _ptr(E, ctypes.c_double)))
        return E

    def last_energies(self) -> np.ndarray:
        E = np.zeros((self.n_samples, self.W))
        self._check(lib().hsg_last_energies(self._ctx, _ptr(E, ctypes.c_double)))
        return E

    def measure(self, q: bool = True):
        ns, R_O, R_T = self.n_samples, self.n_replicas, self.n_temps
        E = np.zeros((ns, R_O, R_T))
        perm = np.zeros((ns, R_O, R_T), dtype=np.int32)
        qa = np.zeros((ns, R_T, 3, 3))
        qk = np.zeros((ns, R_T, 3, 3, 3, 2))
        o = Obs()
        o.E = _ptr(E, ctypes.c_double)
        o.perm = _ptr(perm, ctypes.c_int32)
        if q:
            o.q = _ptr(qa, ctypes.c_double)
            o.qk = _ptr(qk, ctypes.c_double)
        self._check(lib().hsg_measure(self._ctx, ctypes.byref(o)))
        return {"E": E, "perm": perm, "q": qa, "qk": qk}

    def measure_overlaps(self, spin: bool = True, chiral: bool = True):
        """Replica-pair overlaps D [ns, R_T, P, 4, 2] and chiral overlaps
        C [ns, R_T, P, 3, 4, 2] (modes k = 0, kx, ky, kz; re, im) for the P pairs
        (0,1) (0,2) (1,2) (0,3) (1,3) (2,3) of the first min(R_O, 4) replicas."""
        P = self.info().n_overlap_pairs
        ns, R_T = self.n_samples, self.n_temps
        D = np.zeros((ns, R_T, P, 4, 2)) if spin else None
        C = np.zeros((ns, R_T, P, 3, 4, 2)) if chiral else None
        dpp = ctypes.POINTER(ctypes.c_double)
        self._check(lib().hsg_measure_overlaps(
            self._ctx, _ptr(D, ctypes.c_double) if spin else dpp(),
            _ptr(C, ctypes.c_double) if chiral else dpp()))
        return {"D": D, "C": C}

    def spin_shapes(self):
        return [(self.W, n, 3) for n in self.Ns]

    def _split(self, flat: np.ndarray):
        out, o = [], 0
        for n in self.Ns:
            k = self.W * n * 3
            out.append(flat[o:o + k].reshape(self.W, n, 3))
            o += k
        return out

    def get_spins(self, out: Optional[np.ndarray] = None):
        """Per-sample float32 arrays [W, N, 3] (memory-slot order)."""
        total = sum(self.W * n * 3 for n in self.Ns)
        flat = out if out is not None else np.empty(total, dtype=np.float32)
        self._check(lib().hsg_get_spins(self._ctx, _ptr(flat, ctypes.c_float)))
        return self._split(flat)

    def set_spins(self, spins):
        if isinstance(spins, np.ndarray) and spins.ndim == 1:
            flat = np.ascontiguousarray(spins, dtype=np.float32)
        else:
            flat = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.float32).ravel()
                                                        for s in spins]))
        self._check(lib().hsg_set_spins(self._ctx, _ptr(flat, ctypes.c_float)))

    def get_spins_dev(self, dev_ptr: int):
        self._check(lib().hsg_get_spins_dev(self._ctx, ctypes.c_void_p(dev_ptr)))

    def set_spins_dev(self, dev_ptr: int):
        self._check(lib().hsg_set_spins_dev(self._ctx, ctypes.c_void_p(dev_ptr)))

    def get_perm(self) -> np.ndarray:
        perm = np.zeros((self.n_samples, self.n_replicas, self.n_temps), dtype=np.int32)
        self._check(lib().hsg_get_perm(self._ctx, _ptr(perm, ctypes.c_int32)))
        return perm

    def pt_stats(self):
        acc = np.zeros((self.n_samples, self.n_replicas, max(self.n_temps - 1, 1)), dtype=np.uint64)
        n = ctypes.c_uint64()
        self._check(lib().hsg_get_pt_stats(self._ctx, _ptr(acc, ctypes.c_uint64), ctypes.byref(n)))
        return acc, int(n.value)

    def set_active(self, active=None):
        """Freeze (0) or run (nonzero) each sample in later steps and sweeps; None: all run."""
        if active is None:
            self._check(lib().hsg_set_active(self._ctx, ctypes.POINTER(ctypes.c_uint8)()))
            return
        a = np.ascontiguousarray(np.asarray(active).astype(np.uint8))
        assert a.size == self.n_samples
        self._check(lib().hsg_set_active(self._ctx, _ptr(a, ctypes.c_uint8)))

    def counters(self):
        """(sweeps [n_samples], pt_passes [n_samples]) each sample has done."""
        sw = np.zeros(self.n_samples, dtype=np.uint64)
        pt = np.zeros(self.n_samples, dtype=np.uint64)
        self._check(lib().hsg_get_counters(self._ctx, _ptr(sw, ctypes.c_uint64), _ptr(pt, ctypes.c_uint64)))
        return sw, pt

    def pt_diagnostics(self):
        """(moved [ns, R_O, R_T] uint64, tunnel [ns, R_O, R_T] uint32 by memory slot, passes)."""
        shape = (self.n_samples, self.n_replicas, self.n_temps)
        moved = np.zeros(shape, dtype=np.uint64)
        tunnel = np.zeros(shape, dtype=np.uint32)
        n = ctypes.c_uint64()
        self._check(lib().hsg_get_pt_diagnostics(self._ctx, _ptr(moved, ctypes.c_uint64),
                                                 _ptr(tunnel, ctypes.c_uint32), ctypes.byref(n)))
        return moved, tunnel, int(n.value)

    def checkpoint_size(self) -> int:
        """Bytes of a checkpoint blob of this context (hsg_checkpoint_size)."""
        n = ctypes.c_size_t()
        self._check(lib().hsg_checkpoint_size(self._ctx, ctypes.byref(n)))
        return int(n.value)

    def checkpoint(self, out: Optional[np.ndarray] = None):
        """The chain's state (hsg_checkpoint_save): a bytes blob, or written into
        `out` (a uint8 array of at least checkpoint_size() bytes, e.g. pinned
        host memory), which is returned."""
        n = self.checkpoint_size()
        if out is not None:
            if out.dtype != np.uint8 or not out.flags.c_contiguous or out.size < n:
                raise ValueError("out must be a contiguous uint8 array of checkpoint_size() bytes")
            self._check(lib().hsg_checkpoint_save(self._ctx, ctypes.c_void_p(out.ctypes.data), out.size))
            return out
        buf = ctypes.create_string_buffer(n)
        self._check(lib().hsg_checkpoint_save(self._ctx, buf, n))
        return buf.raw

    def restore(self, blob):
        """Load a blob from checkpoint() (hsg_checkpoint_load): bytes or a uint8 array."""
        if isinstance(blob, np.ndarray):
            if blob.dtype != np.uint8 or not blob.flags.c_contiguous:
                raise ValueError("blob must be a contiguous uint8 array")
            self._check(lib().hsg_checkpoint_load(self._ctx, ctypes.c_void_p(blob.ctypes.data), blob.size))
            return
        self._check(lib().hsg_checkpoint_load(self._ctx, blob, len(blob)))

    def info(self) -> Info:
        i = Info()
        self._check(lib().hsg_get_info(self._ctx, ctypes.byref(i)))
        return i

    def sync(self):
        self._check(lib().hsg_sync(self._ctx))


def hsg_philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    """The device Philox4x32-10 on counters ctr[n, 4] (uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(c)
    st = lib().hsg_philox(_ptr(c, ctypes.c_uint32), c.shape[0], ctypes.c_uint64(seed),
                          _ptr(out, ctypes.c_uint32))
    if st != 0:
        raise HsgError(st, (lib().hsg_last_error(None) or b"").decode())
    return out


def hsg_energies_xyz_noalloc(spins_dev: int, J_dev: int, H_dev: int, L: int, W: int, E_dev: int,
                             stream: int = 0) -> int:
    """FP64 energies of W systems held in caller-owned device buffers (raw
    device addresses), with no device allocation (scratch is a static array
    inside the library).  Returns the C status code; 0 on success."""
    return lib().hsg_energies_xyz_noalloc(ctypes.c_void_p(spins_dev), ctypes.c_void_p(J_dev),
                                          ctypes.c_void_p(H_dev or None), L, W,
                                          ctypes.c_void_p(E_dev), ctypes.c_void_p(stream or None))


# C names -----------------------------------------------------------------------
def hsg_create(L: int, temps, n_replicas: int, J, H, seed: int, **kw) -> Context:
    from types import SimpleNamespace
    return Context([SimpleNamespace(L=L, J=J, H=H, temps=np.asarray(temps))], n_replicas, seed, **kw)


def hsg_create_batch(samples, n_replicas: int, seed: int, **kw) -> Context:
    return Context(samples, n_replicas, seed, **kw)


hsg_sweep_or = Context.sweep_or
hsg_sweep_hb = Context.sweep_hb
hsg_pt_exchange = Context.pt_exchange
hsg_pt_exchange_energies = Context.pt_exchange_energies
hsg_step = Context.step
hsg_step_multihit = Context.step_multihit
hsg_energies = Context.energies
hsg_last_energies = Context.last_energies
hsg_measure = Context.measure
hsg_measure_overlaps = Context.measure_overlaps
hsg_get_spins = Context.get_spins
hsg_set_spins = Context.set_spins
hsg_get_spins_dev = Context.get_spins_dev
hsg_set_spins_dev = Context.set_spins_dev
hsg_get_perm = Context.get_perm
hsg_get_pt_stats = Context.pt_stats
hsg_get_info = Context.info
hsg_get_pt_diagnostics = Context.pt_diagnostics
hsg_set_active = Context.set_active
hsg_get_counters = Context.counters
hsg_checkpoint_save = Context.checkpoint
hsg_checkpoint_load = Context.restore
hsg_sync = Context.sync
hsg_destroy = Context.close
