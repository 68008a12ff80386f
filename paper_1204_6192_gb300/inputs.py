"""Seeded synthetic inputs for the Heisenberg spin-glass workloads.

This module is shared by the CUDA path's callers and by the FP64 oracle.  It
holds no step of the Monte Carlo method: it only draws the quenched disorder
(couplings J and random fields H) with numpy's PCG64 generator and lays out the
temperature sets.  The random numbers the Markov chain itself consumes come
from counter-based Philox streams that each side implements on its own.

Disorder follows Sec. 2 of Yavors'kii & Weigel: nearest-neighbour couplings
J_ij ~ N(0, 1), precomputed off the GPU.  The random field is either an
i.i.d. Gaussian per component with standard deviation H_r (the production
form used by the workloads below) or the paper's own form, a uniformly random
direction on a sphere of fixed radius |H| (Sec. 2).

Lattice convention (shared by the C ABI): L^3 periodic cubic lattice, site
index i = x + L*(y + L*z), and J[i, a] is the coupling of the bond between
site i and its neighbour i + e_a for a = x, y, z (each bond stored once).
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np


def geometric_temperatures(t_min: float, t_max: float, n: int) -> np.ndarray:
    """Geometric temperature ladder T_i = T_1 f^(i-1), f = (T_n/T_1)^(1/(n-1)) (Sec. 4)."""
    if n < 1:
        raise ValueError("need at least one temperature")
    if n == 1:
        return np.array([float(t_min)])
    f = (t_max / t_min) ** (1.0 / (n - 1))
    t = t_min * f ** np.arange(n, dtype=np.float64)
    t[-1] = t_max
    return t


def gaussian_couplings(L: int, rng: np.random.Generator, std: float = 1.0) -> np.ndarray:
    """J[N, 3] with J ~ N(0, std^2), one value per bond (+x, +y, +z) of each site."""
    return rng.standard_normal((L ** 3, 3)) * std


def gaussian_field(L: int, h_r: float, rng: np.random.Generator) -> np.ndarray:
    """H[N, 3], each component i.i.d. N(0, h_r^2)."""
    if h_r == 0.0:
        return np.zeros((L ** 3, 3))
    return rng.standard_normal((L ** 3, 3)) * h_r


def sphere_field(L: int, h_abs: float, rng: np.random.Generator) -> np.ndarray:
    """H[N, 3] with fixed length |H| and a uniformly random direction (Sec. 2)."""
    v = rng.standard_normal((L ** 3, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * h_abs


@dataclasses.dataclass
class Sample:
    """One disorder sample: lattice size, couplings, field and temperatures."""

    L: int
    J: np.ndarray          # [N, 3] float64
    H: np.ndarray          # [N, 3] float64
    temps: np.ndarray      # [n_temps] float64, strictly increasing


@dataclasses.dataclass
class Workload:
    """A named synthetic workload: samples plus the step schedule."""

    name: str
    samples: List[Sample]
    n_replicas: int
    seed: int
    precision: str = "fp32"        # spin storage: fp32, fp16, bf16, angle16, oct16
    j_fp16: bool = False           # store J and H as FP16
    n_hb: int = 1                  # heat-bath sweeps per step
    n_or: int = 5                  # over-relaxation sweeps per step
    steps: int = 1
    measure_every: int = 0

    @property
    def n_temps(self) -> int:
        return len(self.samples[0].temps)

    @property
    def systems(self) -> int:
        return len(self.samples) * self.n_replicas * self.n_temps

    @property
    def spins(self) -> int:
        return sum(s.L ** 3 for s in self.samples) * self.n_replicas * self.n_temps


def make_sample(L: int, temps: np.ndarray, h_r: float, disorder_seed: int,
                field: str = "gaussian") -> Sample:
    rng = np.random.default_rng(disorder_seed)
    J = gaussian_couplings(L, rng)
    if field == "gaussian":
        H = gaussian_field(L, h_r, rng)
    elif field == "sphere":
        H = sphere_field(L, h_r, rng)
    else:
        raise ValueError(field)
    return Sample(L=L, J=J, H=H, temps=np.asarray(temps, dtype=np.float64))


def round_fp16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest binary16 value (ties to even) and widen back to float64.

    Used so that a caller storing J and H in FP16 hands the oracle exactly the
    values the device holds."""
    return np.asarray(a, dtype=np.float64).astype(np.float16).astype(np.float64)


# ---------------------------------------------------------------------------
# Named workloads.  Sizes follow the production shapes of the method: small
# lattices for checks, L = 32 / 64 / 128 single-disorder production runs and a
# batch of many small samples of mixed size.
# ---------------------------------------------------------------------------

def workload(name: str, steps: Optional[int] = None) -> Workload:
    if name == "L8_plain":
        # L=8, Gaussian J, H = 0, 2 replicas x 8 temperatures in [0.15, 0.6].
        t = geometric_temperatures(0.15, 0.6, 8)
        s = make_sample(8, t, 0.0, disorder_seed=1)
        w = Workload(name, [s], n_replicas=2, seed=1, steps=200)
    elif name.startswith("table1_"):
        # the paper's benchmark of Table 1: R = 256 systems of L = 32 at T = 100
        # (where the result does not depend on the disorder), FP32 spins; the
        # suffix names the step: table1_hb100or = 1 HB + 100 OR, table1_hb10or =
        # 1 HB + 10 OR, table1_hb = 1 HB, table1_or = 1 OR.
        n_hb, n_or = {"table1_hb100or": (1, 100), "table1_hb10or": (1, 10), "table1_hb": (1, 0),
                      "table1_or": (0, 1)}[name]
        s = make_sample(32, np.array([100.0]), 0.0, disorder_seed=6)
        w = Workload(name, [s], n_replicas=256, seed=1, n_hb=n_hb, n_or=n_or, steps=20)
    elif name == "L32_fp32":
        t = geometric_temperatures(0.1, 0.4, 32)
        s = make_sample(32, t, 0.05, disorder_seed=2)
        w = Workload(name, [s], n_replicas=2, seed=1, steps=10_000, measure_every=10)
    elif name in ("L64_fp16", "L64_angle16", "L64_oct16", "L64_bf16"):
        t = geometric_temperatures(0.1, 0.4, 32)
        s = make_sample(64, t, 0.1, disorder_seed=3)
        prec = name.split("_")[1]
        w = Workload(name, [s], n_replicas=2, seed=1, precision=prec, j_fp16=True,
                     steps=5_000)
    elif name == "L128_fp16_w16":
        # the bench lattice with 2 replicas x 8 temperatures (201 MB of FP16 spins, more
        # than L2): the small case for multi-pass profiler captures of the sweep kernels
        t = geometric_temperatures(0.08, 0.3, 8)
        s = make_sample(128, t, 0.1, disorder_seed=5)
        w = Workload(name, [s], n_replicas=2, seed=1, precision="fp16", j_fp16=True, steps=2_000)
    elif name in ("L128_fp16", "L128_fp32", "L128_oct16", "L128_bf16", "L128_yx4"):
        t = geometric_temperatures(0.08, 0.3, 24)
        s = make_sample(128, t, 0.1, disorder_seed=5)
        prec = name.split("_")[1]
        w = Workload(name, [s], n_replicas=2, seed=1, precision=prec,
                     j_fp16=(prec != "fp32"), steps=2_000)
    elif name == "batch512_mixedL":
        t = geometric_temperatures(0.1, 0.5, 16)
        rng = np.random.default_rng(4)
        samples = []
        for k, L in enumerate([8] * 128 + [12] * 128 + [16] * 128 + [24] * 128):
            h_r = float(rng.choice([0.0, 0.05, 0.1]))
            samples.append(make_sample(L, t, h_r, disorder_seed=1000 + k))
        w = Workload(name, samples, n_replicas=2, seed=1, steps=10_000)
    else:
        raise KeyError(name)
    if steps is not None:
        w.steps = steps
    return w


def small_sample(L: int, n_temps: int = 4, h_r: float = 0.1, disorder_seed: int = 0,
                 t_min: float = 0.2, t_max: float = 1.0) -> Sample:
    """A small test sample (for parity tests)."""
    return make_sample(L, geometric_temperatures(t_min, t_max, n_temps), h_r, disorder_seed)


def ferromagnet(L: int, temps: Sequence[float]) -> Sample:
    """Uniform J = 1 couplings, zero field (special case with a closed-form ground state)."""
    N = L ** 3
    return Sample(L=L, J=np.ones((N, 3)), H=np.zeros((N, 3)),
                  temps=np.asarray(temps, dtype=np.float64))
