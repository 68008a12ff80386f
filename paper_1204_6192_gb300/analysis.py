"""Host-side analysis of measurement series (Sec. 2 of the paper).

Inputs are the per-measurement outputs of ``hsg_measure`` (q, qk, E) and
``hsg_measure_overlaps`` (D, C), stacked along a leading time axis.  Thermal
averages <.> run over the time axis (callers pass the equilibrated part of the
series), disorder averages [.] over samples; errors are jackknife over samples
(one sample: over 10 time bins).

Definitions:
* zero-field spin-glass susceptibility  chi_SG(k) = N sum_{mu nu} [<|q^{mu nu}(k)|^2>]
* four-replica form in a field          chi_SG(k) = (1/N) [chi_1 - 2 chi_2 + chi_3]
  with chi_1 = N^2 |D_12|^2, chi_2 = N^2 Re D_13 conj(D_14), chi_3 = N^2 Re D_13 conj(D_24)
  (replicas numbered from 1; D the scalar pair overlaps, whose component sums
  the paper's four-replica expressions contract within each site)
* chiral susceptibility                 chi_CG^a(k) = N [<|q_c^a(k)|^2>], q_c = C_12
  (four-replica chiral form: the same combination of C as of D above)
* second-moment correlation length      xi = (chi(0)/chi(k_min) - 1)^{1/2} / (2 sin(k_min/2)),
  k_min = 2 pi / L
* internal energy and specific heat per spin, u = [<E>]/N and c = [<E^2> - <E>^2]/(T^2 N)
* integrated autocorrelation time of a series, which turns a time per update
  into a time per independent sample (the comparison of schedules Sec. 4 asks
  for): tau_int = 1/2 + sum_{t=1}^{W} rho(t), with the window W the first
  t >= c tau_int(t) (Sokal's self-consistent window, c = 6)
"""
from __future__ import annotations

import numpy as np

# positions of the replica pairs in the overlap outputs: (0,1) (0,2) (1,2) (0,3) (1,3) (2,3)
PAIR_INDEX = {(0, 1): 0, (0, 2): 1, (1, 2): 2, (0, 3): 3, (1, 3): 4, (2, 3): 5}


def _c(v: np.ndarray) -> np.ndarray:
    """[..., 2] (re, im) -> complex."""
    return v[..., 0] + 1j * v[..., 1]


def chi_sg_tensor(q: np.ndarray, qk: np.ndarray, N: int) -> np.ndarray:
    """Instantaneous N sum_{mu nu} |q^{mu nu}(k)|^2 at k = 0, kx, ky, kz.
    q [..., 3, 3], qk [..., 3(axis), 3, 3, 2] -> [..., 4]."""
    c0 = (q ** 2).sum(axis=(-2, -1))
    ck = (np.abs(_c(qk)) ** 2).sum(axis=(-2, -1))
    return N * np.concatenate([c0[..., None], ck], axis=-1)


def four_replica_combination(X: np.ndarray, N: int) -> np.ndarray:
    """Instantaneous (1/N)(chi_1 - 2 chi_2 + chi_3) from pair overlaps X [..., P>=5, M, 2]
    (D: M = 4 modes; C: pass X[..., a, :, :] per axis).  Needs four replicas."""
    x = _c(X)
    d12, d13, d14, d24 = (x[..., PAIR_INDEX[p], :] for p in ((0, 1), (0, 2), (0, 3), (1, 3)))
    return N * (np.abs(d12) ** 2 - 2.0 * (d13 * np.conj(d14)).real + (d13 * np.conj(d24)).real)


def chi_two_replica(X: np.ndarray, N: int) -> np.ndarray:
    """Instantaneous N |X_12(k)|^2 of the first pair: X [..., P, M, 2] -> [..., M]."""
    return N * np.abs(_c(X[..., 0, :, :])) ** 2


def xi_second_moment(chi0, chik, L: int):
    """Second-moment correlation length; nan where chi(0) < chi(k_min)."""
    chi0 = np.asarray(chi0, dtype=np.float64)
    chik = np.asarray(chik, dtype=np.float64)
    r = chi0 / chik - 1.0
    with np.errstate(invalid="ignore"):
        return np.where(r >= 0, np.sqrt(np.maximum(r, 0.0)), np.nan) / (2.0 * np.sin(np.pi / L))


def jackknife(per_sample: np.ndarray, fn=lambda m: m):
    """Estimate fn(mean over axis 0) and its jackknife error over axis 0."""
    x = np.asarray(per_sample, dtype=np.float64)
    n = x.shape[0]
    full = fn(x.mean(axis=0))
    if n < 2:
        return full, np.full(np.shape(full), np.nan)
    loo = np.array([fn((x.sum(axis=0) - x[i]) / (n - 1)) for i in range(n)])
    err = np.sqrt((n - 1) / n * ((loo - loo.mean(axis=0)) ** 2).sum(axis=0))
    return full, err


def _units(thermal: np.ndarray) -> np.ndarray:
    """[T, S, ...] series -> jackknife units [S, ...] of thermal means; one sample:
    10 time bins of it."""
    if thermal.shape[1] > 1:
        return thermal.mean(axis=0)
    bins = np.array_split(thermal[:, 0], 10)
    return np.array([b.mean(axis=0) for b in bins])


def correlation_length(chi_series: np.ndarray, L: int):
    """chi_series [T, S, slots, 4] (k = 0, kx, ky, kz): xi per slot from chi(0)
    and the mean of the three k_min modes.  Returns (xi, err)."""
    u = _units(chi_series)
    fn = lambda m: xi_second_moment(m[..., 0], m[..., 1:].mean(axis=-1), L)
    return jackknife(u, fn)


def energy_and_specific_heat(E: np.ndarray, temps: np.ndarray, N: int):
    """E [T, S, R_O, slots] energies by temperature slot -> (u, du), (c, dc) per
    slot.  Each replica is an independent chain: <E> and <E^2> - <E>^2 are taken
    per chain and averaged over the replicas; the jackknife runs over samples
    (one sample: over 10 time bins)."""
    E = np.asarray(E, dtype=np.float64)
    if E.shape[1] > 1:
        u_units = E.mean(axis=(0, 2))                                  # [S, slots]
        c_units = ((E ** 2).mean(axis=0) - E.mean(axis=0) ** 2).mean(axis=1)
    else:
        bins = np.array_split(np.arange(E.shape[0]), 10)
        u_units = np.array([E[b, 0].mean(axis=(0, 1)) for b in bins])
        c_units = np.array([((E[b, 0] ** 2).mean(axis=0) - E[b, 0].mean(axis=0) ** 2).mean(axis=0)
                            for b in bins])
    u = jackknife(u_units / N)
    c = jackknife(c_units / (np.asarray(temps, dtype=np.float64) ** 2 * N))
    return u, c


def integrated_autocorrelation_time(x: np.ndarray, c: float = 6.0):
    """tau_int of the series x [T] (or of each column of x [T, k]) in units of
    its sampling interval, with Sokal's self-consistent window; returns
    (tau, window).  tau = 1/2 for uncorrelated samples."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    n = x.shape[0]
    d = x - x.mean(axis=0)
    var = (d ** 2).mean(axis=0)
    taus, wins = [], []
    for k in range(x.shape[1]):
        if var[k] == 0.0:
            taus.append(0.5)
            wins.append(0)
            continue
        # autocorrelation by FFT (zero-padded, so not circular)
        f = np.fft.rfft(d[:, k], 2 * n)
        acf = np.fft.irfft(f * np.conj(f))[:n] / (n * var[k])
        tau, w = 0.5, 0
        for t in range(1, n):
            tau += acf[t]
            if t >= c * tau:
                w = t
                break
        else:
            w = n - 1
        taus.append(tau)
        wins.append(w)
    if len(taus) == 1:
        return taus[0], wins[0]
    return np.array(taus), np.array(wins)
