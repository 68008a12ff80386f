"""Host analysis (susceptibilities, correlation lengths, specific heat) against
brute-force evaluation of the paper's double sums (Sec. 2) on tiny lattices and
closed forms."""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import analysis

L = 2
N = L ** 3


def coords():
    i = np.arange(N)
    return np.stack([i % L, (i // L) % L, i // (L * L)], axis=1)


def kvec(m):
    k = np.zeros(3)
    if m > 0:
        k[m - 1] = 2 * np.pi / L
    return k


def random_replicas(seed, R=4, T=3):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(R * T, N, 3))
    s = v / np.linalg.norm(v, axis=2, keepdims=True)
    perm = np.array([rng.permutation(T) for _ in range(R)], dtype=np.int32)
    return s, perm


def brute_four(sys, k):
    """chi_1, chi_2, chi_3 by the double sums over i, j and mu, nu (Sec. 2), for
    one set of four configurations sys[4][N][3] (replicas 1..4)."""
    R = coords()
    ph = np.exp(1j * (R @ k))
    s1, s2, s3, s4 = sys
    chi = []
    for (a, b, c, d) in ((s1, s1, s2, s2), (s1, s1, s3, s4), (s1, s2, s3, s4)):
        # sum_{ij} sum_{mu nu} a_i^mu b_j^nu c_i^mu d_j^nu e^{ik(Ri - Rj)}
        tot = 0.0
        for i in range(N):
            for j in range(N):
                tot += sum(a[i, mu] * b[j, nu] * c[i, mu] * d[j, nu]
                           for mu in range(3) for nu in range(3)) * ph[i] * np.conj(ph[j])
        chi.append(tot)
    return chi


@pytest.mark.parametrize("seed", [1, 2])
def test_four_replica_combination_equals_double_sums(seed):
    s, perm = random_replicas(seed)
    T = perm.shape[1]
    D, C = oracle.overlaps(s, L, 4, T, perm)
    comb = analysis.four_replica_combination(D, N)          # [T, 4 modes]
    for t in range(T):
        sys = [s[r * T + perm[r, t]] for r in range(4)]
        for m in range(4):
            c1, c2, c3 = brute_four(sys, kvec(m))
            np.testing.assert_allclose(comb[t, m], ((c1 - 2 * c2 + c3) / N).real, atol=1e-12)


def test_four_replica_combination_vanishes_for_identical_replicas():
    s, perm = random_replicas(3)
    T = perm.shape[1]
    s[T:] = np.tile(s[:T], (3, 1, 1))
    perm[:] = perm[0]
    D, _ = oracle.overlaps(s, L, 4, T, perm)
    np.testing.assert_allclose(analysis.four_replica_combination(D, N), 0.0, atol=1e-12)


def test_tensor_chi_sg_equals_double_sum():
    """N sum_{mu nu} |q^{mu nu}(k)|^2 = (1/N) sum_{ij} sum_{mu nu}
    s_i^mu(1) s_i^nu(2) s_j^mu(1) s_j^nu(2) e^{ik(Ri - Rj)}."""
    s, perm = random_replicas(4, R=2, T=2)
    T = 2
    q = np.zeros((T, 3, 3))
    qk = np.zeros((T, 3, 3, 3, 2))
    oracle.lib().orc_measure(oracle._dp(s), L, T, oracle._p(perm, oracle.ctypes.c_int32),
                             oracle._dp(q), oracle._dp(qk))
    chi = analysis.chi_sg_tensor(q, qk, N)
    R = coords()
    for t in range(T):
        a, b = s[perm[0, t]], s[T + perm[1, t]]
        for m in range(4):
            ph = np.exp(1j * (R @ kvec(m)))
            tot = 0.0
            for i in range(N):
                for j in range(N):
                    tot += (np.outer(a[i], b[i]) * np.outer(a[j], b[j])).sum() * ph[i] * np.conj(ph[j])
            np.testing.assert_allclose(chi[t, m], (tot / N).real, atol=1e-12)


def test_chiral_two_replica_chi_equals_double_sum():
    s, perm = random_replicas(5, R=2, T=1)
    Lc = 4
    rng = np.random.default_rng(8)
    v = rng.normal(size=(2, Lc ** 3, 3))
    s = v / np.linalg.norm(v, axis=2, keepdims=True)
    perm = np.zeros((2, 1), dtype=np.int32)
    _, C = oracle.overlaps(s, Lc, 2, 1, perm)
    chi = analysis.chi_two_replica(C[:, :, 0], Lc ** 3)     # axis x
    ka, kb = oracle.chirality(s[0], Lc), oracle.chirality(s[1], Lc)
    i = np.arange(Lc ** 3)
    R = np.stack([i % Lc, (i // Lc) % Lc, i // (Lc * Lc)], axis=1)
    for m in range(4):
        k = np.zeros(3)
        if m:
            k[m - 1] = 2 * np.pi / Lc
        f = (ka[:, 0] * kb[:, 0]) * np.exp(1j * (R @ k))
        np.testing.assert_allclose(chi[0, m], np.abs(f.sum()) ** 2 / Lc ** 3, rtol=1e-12)


@pytest.mark.parametrize("xi,Lx", [(0.5, 8), (2.0, 16), (5.0, 32)])
def test_xi_of_ornstein_zernike_form(xi, Lx):
    """chi(k) = A / (1 + xi^2 (2 sin(k/2))^2) gives back xi exactly."""
    kmin = 2 * np.pi / Lx
    chi0, chik = 3.0, 3.0 / (1 + (xi * 2 * np.sin(kmin / 2)) ** 2)
    np.testing.assert_allclose(analysis.xi_second_moment(chi0, chik, Lx), xi, rtol=1e-12)
    assert analysis.xi_second_moment(1.0, 1.0, Lx) == 0.0
    assert np.isnan(analysis.xi_second_moment(1.0, 2.0, Lx))


def test_jackknife_of_mean_is_standard_error():
    x = np.random.default_rng(0).normal(size=37)
    m, e = analysis.jackknife(x)
    assert np.isclose(m, x.mean())
    assert np.isclose(e, x.std(ddof=1) / np.sqrt(len(x)))


def test_specific_heat_of_two_level_series():
    """A chain alternating between energies a and b: <E^2> - <E>^2 = (a - b)^2 / 4."""
    a, b, Nn, T = -10.0, -6.0, 4, 0.5
    E = np.array([a, b] * 50)[:, None, None, None] * np.ones((1, 3, 2, 1))
    (u, du), (c, dc) = analysis.energy_and_specific_heat(E, np.array([T]), Nn)
    np.testing.assert_allclose(u, (a + b) / 2 / Nn)
    np.testing.assert_allclose(c, (a - b) ** 2 / 4 / (T ** 2 * Nn))
    np.testing.assert_allclose(dc, 0.0, atol=1e-12)


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.9, 0.98])
def test_tau_int_of_ar1_process(phi):
    """x_t = phi x_{t-1} + e_t has rho(t) = phi^t, so tau_int = 1/2 + phi/(1 - phi)
    = (1 + phi) / (2 (1 - phi)); the estimate's relative error is about
    sqrt(2 (2W + 1) / n) (Sokal), here a few percent."""
    rng = np.random.default_rng(int(phi * 100))
    n = 400_000
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - phi ** 2)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    tau, w = analysis.integrated_autocorrelation_time(x)
    exact = (1 + phi) / (2 * (1 - phi))
    rel = np.sqrt(2 * (2 * w + 1) / n)
    assert abs(tau - exact) < 4 * rel * exact + 0.01, (tau, exact, w)


def test_tau_int_columns_and_constant_series():
    x = np.random.default_rng(1).normal(size=(5000, 3))
    tau, w = analysis.integrated_autocorrelation_time(x)
    assert tau.shape == (3,) and np.all(np.abs(tau - 0.5) < 0.1)
    assert analysis.integrated_autocorrelation_time(np.ones(100)) == (0.5, 0)
