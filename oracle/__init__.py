"""FP64 CPU oracle for the Heisenberg spin-glass Monte Carlo (test infrastructure).

Only tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It wraps ``hsg_oracle.c`` (plain C, binary64, built with
``-ffp-contract=off``) through ctypes and drives it in the order the method
prescribes: a step is n_hb heat-bath sweeps, n_or over-relaxation sweeps, an
energy evaluation and one parallel-tempering pass (Sec. 3.2).  Each sweep is an
even half-sweep followed by an odd half-sweep (Sec. 3.1).

Nothing here is shared with the CUDA library; the two agree only on the
conventions written in ``hsg_oracle.h``.
"""

from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsg_oracle.c")
_LIB = os.path.join(_HERE, "libhsg_oracle.so")

CODECS = {"none": 0, "fp16": 1, "bf16": 2, "angle16": 3, "oct16": 4, "fp32": 5, "yx4": 6}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (gcc, -O2, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hsg_oracle.h"))):
        return _LIB
    cc = os.environ.get("CC", "gcc")
    if shutil.which(cc) is None:
        raise RuntimeError("no C compiler for the oracle")
    base = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:6] + ["-fopenmp"] + base[6:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        c_int, c_long, u64, u32 = ctypes.c_int, ctypes.c_long, ctypes.c_uint64, ctypes.c_uint32
        sig = {
            "orc_philox4x32_10": (None, [u32p, u32p, u32p]),
            "orc_philox_many": (None, [u32p, c_long, u64, u32p]),
            "orc_uniform": (ctypes.c_double, [u32]),
            "orc_codec_roundtrip_many": (None, [dp, c_long, c_int]),
            "orc_round_fp16": (ctypes.c_double, [ctypes.c_double]),
            "orc_round_bf16": (ctypes.c_double, [ctypes.c_double]),
            "orc_init_spins": (None, [dp, c_int, c_int, u64, u64, c_int]),
            "orc_local_field": (None, [dp, dp, dp, c_int, c_long, dp]),
            "orc_hb_many": (None, [dp, dp, dp, dp, dp, c_long]),
            "orc_or_half": (None, [dp, dp, dp, c_int, c_int, c_int, c_int]),
            "orc_hb_half": (None, [dp, dp, dp, c_int, c_int, c_int, dp, u64, u64, u32, c_int]),
            "orc_multihit": (None, [dp, dp, dp, c_int, c_int, c_int, c_int, c_int, c_int, c_int,
                                     dp, u64, u64, u32, c_int]),
            "orc_energy": (None, [dp, dp, dp, c_int, c_int, dp]),
            "orc_pt": (None, [dp, dp, i32p, c_int, c_int, u64, u64, u32, i32p]),
            "orc_measure": (None, [dp, c_int, c_int, i32p, dp, dp]),
            "orc_chirality": (None, [dp, c_int, dp]),
            "orc_overlaps": (None, [dp, c_int, c_int, c_int, i32p, dp, dp]),
            "orc_num_threads": (c_int, []),
            "orc_set_num_threads": (None, [c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _dp(a):
    return None if a is None else _p(a, ctypes.c_double)


# --- thin functional wrappers -------------------------------------------------

def philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    lib().orc_philox_many(_p(ctr, ctypes.c_uint32), ctr.shape[0], seed, _p(out, ctypes.c_uint32))
    return out


def uniform(x: np.ndarray) -> np.ndarray:
    f = lib().orc_uniform
    return np.array([f(int(v)) for v in np.asarray(x, dtype=np.uint32).ravel()])


def codec_roundtrip(v: np.ndarray, codec: str) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    lib().orc_codec_roundtrip_many(_dp(v), v.size // 3, CODECS[codec])
    return v


def local_field(s_sys: np.ndarray, J: np.ndarray, H: Optional[np.ndarray], L: int, i: int):
    h = np.zeros(3)
    lib().orc_local_field(_dp(np.ascontiguousarray(s_sys)), _dp(np.ascontiguousarray(J)),
                          _dp(None if H is None else np.ascontiguousarray(H)), L, i, _dp(h))
    return h


def chirality(s: np.ndarray, L: int) -> np.ndarray:
    """Local chirality kappa[N, 3] (a = x, y, z) of one system s[N, 3]."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    k = np.zeros((L ** 3, 3))
    lib().orc_chirality(_dp(s), L, _dp(k))
    return k


def overlaps(s: np.ndarray, L: int, R_O: int, R_T: int, perm: np.ndarray):
    """Replica-pair overlaps of one sample, s[W, N, 3] (memory-slot order) and
    perm[R_O, R_T]: D[R_T, P, 4, 2] and C[R_T, P, 3, 4, 2] (modes 0, kx, ky, kz),
    pairs (0,1) (0,2) (1,2) (0,3) (1,3) (2,3) of the first min(R_O, 4) replicas."""
    r = min(R_O, 4)
    P = r * (r - 1) // 2
    s = np.ascontiguousarray(s, dtype=np.float64)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    D = np.zeros((R_T, P, 4, 2))
    C = np.zeros((R_T, P, 3, 4, 2))
    lib().orc_overlaps(_dp(s), L, R_O, R_T, _p(perm, ctypes.c_int32), _dp(D), _dp(C))
    return D, C


def hb_moves(s, h, beta, u1, u2) -> np.ndarray:
    """Heat-bath draws for independent spins in fixed fields h (arrays [n,3], [n])."""
    s = np.ascontiguousarray(s, dtype=np.float64).copy()
    h = np.ascontiguousarray(h, dtype=np.float64)
    n = s.shape[0]
    b = np.ascontiguousarray(np.broadcast_to(beta, (n,)), dtype=np.float64)
    u1 = np.ascontiguousarray(u1, dtype=np.float64)
    u2 = np.ascontiguousarray(u2, dtype=np.float64)
    lib().orc_hb_many(_dp(s), _dp(h), _dp(b), _dp(u1), _dp(u2), n)
    return s


def energy(s: np.ndarray, J: np.ndarray, H: Optional[np.ndarray], L: int) -> np.ndarray:
    W = s.shape[0]
    E = np.zeros(W)
    lib().orc_energy(_dp(np.ascontiguousarray(s)), _dp(np.ascontiguousarray(J)),
                     _dp(None if H is None else np.ascontiguousarray(H)), L, W, _dp(E))
    return E


def pt(E, temps, perm, R_O, R_T, chain_base, seed, pt_step):
    E = np.ascontiguousarray(E, dtype=np.float64)
    temps = np.ascontiguousarray(temps, dtype=np.float64)
    perm = np.ascontiguousarray(perm, dtype=np.int32).copy()
    acc = np.zeros((R_O, max(R_T - 1, 1)), dtype=np.int32)
    lib().orc_pt(_dp(E), _dp(temps), _p(perm, ctypes.c_int32), R_O, R_T, chain_base, seed,
                 pt_step, _p(acc, ctypes.c_int32))
    return perm, acc


class OracleSample:
    """State of one disorder sample: W = n_replicas * n_temps systems."""

    def __init__(self, L, J, H, temps, n_replicas, sys_base, chain_base, seed, codec):
        self.L = int(L)
        self.N = self.L ** 3
        self.J = np.ascontiguousarray(J, dtype=np.float64).reshape(self.N, 3)
        self.H = None if H is None else np.ascontiguousarray(H, dtype=np.float64).reshape(self.N, 3)
        self.temps = np.ascontiguousarray(temps, dtype=np.float64)
        self.R_T = len(self.temps)
        self.R_O = int(n_replicas)
        self.W = self.R_T * self.R_O
        self.sys_base = int(sys_base)
        self.chain_base = int(chain_base)
        self.seed = int(seed)
        self.codec = codec
        self.s = np.zeros((self.W, self.N, 3))
        lib().orc_init_spins(_dp(self.s), self.L, self.W, self.sys_base, self.seed, codec)
        self.perm = np.tile(np.arange(self.R_T, dtype=np.int32), (self.R_O, 1))
        # temperature random-walk diagnostics (Sec. 4)
        self.moved = np.zeros((self.R_O, self.R_T), dtype=np.int64)
        self.tunnel = np.zeros((self.R_O, self.R_T), dtype=np.int64)
        self._seen_bottom = self.perm == 0          # by memory slot: visited T_1
        self._seen_top = np.zeros((self.R_O, self.R_T), dtype=bool)   # then T_R

    def _diagnose(self, before: np.ndarray):
        """After a PT pass: a slot counts as moved when the configuration it held
        before the pass is elsewhere; a configuration that is back at T_1 after
        visiting T_R after T_1 has completed one tunnelling loop."""
        if self.R_T < 2:
            return
        self.moved += (self.perm != before)
        for r in range(self.R_O):
            for t in range(self.R_T):
                m = self.perm[r, t]
                if t == 0:
                    if self._seen_top[r, m]:
                        self.tunnel[r, m] += 1
                    self._seen_bottom[r, m] = True
                    self._seen_top[r, m] = False
                elif t == self.R_T - 1 and self._seen_bottom[r, m]:
                    self._seen_top[r, m] = True

    def beta_sys(self) -> np.ndarray:
        b = np.zeros(self.W)
        for r in range(self.R_O):
            for t in range(self.R_T):
                b[r * self.R_T + self.perm[r, t]] = 1.0 / self.temps[t]
        return b

    def or_half(self, parity):
        lib().orc_or_half(_dp(self.s), _dp(self.J), _dp(self.H), self.L, self.W, parity, self.codec)

    def hb_half(self, parity, sweep):
        beta = self.beta_sys()
        lib().orc_hb_half(_dp(self.s), _dp(self.J), _dp(self.H), self.L, self.W, parity, _dp(beta),
                          self.sys_base, self.seed, sweep, self.codec)

    def multihit(self, tile, n_rounds, n_or, n_hb, sweep0, colors=3):
        """Tile-local updates of the double checkerboard (Sec. 3.2): see orc_multihit."""
        beta = self.beta_sys()
        lib().orc_multihit(_dp(self.s), _dp(self.J), _dp(self.H), self.L, self.W, tile, colors,
                           n_rounds, n_or, n_hb, _dp(beta), self.sys_base, self.seed, sweep0,
                           self.codec)

    def energies(self) -> np.ndarray:
        E = np.zeros(self.W)
        lib().orc_energy(_dp(self.s), _dp(self.J), _dp(self.H), self.L, self.W, _dp(E))
        return E

    def pt(self, E, pt_step):
        before = self.perm.copy()
        self.perm, acc = pt(E, self.temps, self.perm, self.R_O, self.R_T, self.chain_base,
                            self.seed, pt_step)
        self._diagnose(before)
        return acc

    def measure(self):
        q = np.zeros((self.R_T, 3, 3))
        qk = np.zeros((self.R_T, 3, 3, 3, 2))
        if self.R_O >= 2:
            lib().orc_measure(_dp(self.s), self.L, self.R_T, _p(self.perm, ctypes.c_int32),
                              _dp(q), _dp(qk))
        E = self.energies()
        E_slot = np.array([[E[r * self.R_T + self.perm[r, t]] for t in range(self.R_T)]
                           for r in range(self.R_O)])
        return {"E": E_slot, "q": q, "qk": qk, "perm": self.perm.copy()}


class OracleSim:
    """The Markov chain of the library, on the CPU in FP64, for a batch of samples.

    ``samples`` is a list of objects with attributes L, J, H, temps.  System and
    chain ids are numbered across the batch in sample order, as in the library.
    """

    def __init__(self, samples: Sequence, n_replicas: int, seed: int, codec: str = "none"):
        self.seed = int(seed)
        self.codec = CODECS[codec]
        self.samples: List[OracleSample] = []
        # global system ids: sample s owns s * Wp ... s * Wp + W - 1, Wp = W rounded up to 8;
        # global chain ids: s * n_replicas + r (the library's numbering)
        W = n_replicas * len(samples[0].temps)
        Wp = (W + 7) // 8 * 8
        for k, smp in enumerate(samples):
            o = OracleSample(smp.L, smp.J, smp.H, smp.temps, n_replicas, k * Wp, k * n_replicas,
                             seed, self.codec)
            o.sweep = 0         # the sample's own sweep counter (keys its heat-bath numbers)
            o.pt_step = 0       # and PT pass counter
            self.samples.append(o)
        self.active = [True] * len(self.samples)

    def set_active(self, active=None):
        """Samples with a False entry are frozen in later sweeps, steps and PT passes."""
        self.active = [True] * len(self.samples) if active is None else [bool(a) for a in active]

    def _running(self):
        return [o for o, a in zip(self.samples, self.active) if a]

    def sweep_or(self, n: int = 1):
        for _ in range(n):
            for o in self._running():
                o.or_half(0)
                o.or_half(1)
                o.sweep += 1

    def sweep_hb(self, n: int = 1):
        for _ in range(n):
            for o in self._running():
                o.hb_half(0, o.sweep)
                o.hb_half(1, o.sweep)
                o.sweep += 1

    def energies(self) -> List[np.ndarray]:
        return [o.energies() for o in self.samples]

    def pt_exchange(self, energies: Optional[List[np.ndarray]] = None):
        if energies is None:
            energies = self.energies()
        acc = []
        for o, E, a in zip(self.samples, energies, self.active):
            if a:
                acc.append(o.pt(E, o.pt_step))
                o.pt_step += 1
            else:
                acc.append(np.zeros((o.R_O, max(o.R_T - 1, 1)), dtype=np.int32))
        return acc

    def step(self, n: int = 1, n_hb: int = 1, n_or: int = 5):
        for _ in range(n):
            self.sweep_hb(n_hb)
            self.sweep_or(n_or)
            self.pt_exchange()

    def step_multihit(self, n: int = 1, tile: int = 8, n_rounds: int = 10, n_or: int = 10,
                      n_hb: int = 1):
        """n steps of the multi-hit schedule: per step both tile colours with
        n_rounds x (n_or OR + n_hb HB) tile sweeps each, then the energies and
        one PT pass; every sample's sweep counter advances by n_rounds (n_or + n_hb)."""
        for _ in range(n):
            for o in self._running():
                o.multihit(tile, n_rounds, n_or, n_hb, o.sweep)
                o.sweep += n_rounds * (n_or + n_hb)
            self.pt_exchange()

    def measure(self):
        return [o.measure() for o in self.samples]

    def spins(self) -> List[np.ndarray]:
        return [o.s for o in self.samples]
