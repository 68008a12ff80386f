"""Pins of the oracle's lattice functions: energy (Eq. 1), local field (Eq. 2),
checkerboard over-relaxation sweeps (Eq. 3, Sec. 3.1), overlaps (Eq. 5 and its
k-dependent form), against brute force, closed forms and invariants."""
import ctypes
import itertools

import numpy as np
import pytest

from paper_1204_6192_gb300 import inputs


def coords(L):
    i = np.arange(L ** 3)
    return np.stack([i % L, (i // L) % L, i // (L * L)], axis=1)


def random_state(rng, W, L):
    s = rng.standard_normal((W, L ** 3, 3))
    return s / np.linalg.norm(s, axis=2, keepdims=True)


def brute_energy(s, J, H, L):
    """Every ordered pair of sites found adjacent from coordinates alone."""
    R = coords(L)
    N = L ** 3
    E = -np.einsum("ic,ic->", H, s)
    for i in range(N):
        for j in range(N):
            d = (R[j] - R[i]) % L
            for a in range(3):
                e = np.zeros(3, dtype=int)
                e[a] = 1
                if np.array_equal(d, e):        # j = i + e_a (periodic)
                    E -= J[i, a] * (s[i] @ s[j])
    return E


def test_energy_brute_force(orc):
    rng = np.random.default_rng(10)
    L = 4
    J = rng.standard_normal((L ** 3, 3))
    H = rng.standard_normal((L ** 3, 3)) * 0.3
    s = random_state(rng, 2, L)
    E = orc.energy(s, J, H, L)
    for w in range(2):
        assert abs(E[w] - brute_energy(s[w], J, H, L)) < 1e-11


def test_energy_ferromagnet_ground_state(orc):
    for L in (4, 6):
        fm = inputs.ferromagnet(L, [1.0])
        s = np.tile([[0.0, 0.6, 0.8]], (1, L ** 3, 1))
        E = orc.energy(s, fm.J, fm.H, L)
        assert abs(E[0] - (-3.0 * L ** 3)) < 1e-12


def test_local_field_is_energy_gradient(orc):
    """sum_i s_i.(h_i - H_i) counts every bond twice: E = -1/2 sum s.(h-H) - sum H.s."""
    rng = np.random.default_rng(11)
    L = 6
    J = rng.standard_normal((L ** 3, 3))
    H = rng.standard_normal((L ** 3, 3)) * 0.2
    s = random_state(rng, 1, L)[0]
    tot = 0.0
    for i in range(L ** 3):
        h = orc.local_field(s, J, H, L, i)
        tot += s[i] @ (h - H[i])
    E = orc.energy(s[None], J, H, L)[0]
    assert abs(E - (-0.5 * tot - np.einsum("ic,ic->", H, s))) < 1e-11
    # and the field of one site from coordinates: neighbour i + e_a has bond J[i, a],
    # neighbour i - e_a has bond J[i - e_a, a]
    R = coords(L)
    idx = {tuple(r): k for k, r in enumerate(R)}
    i = idx[(L - 1, 0, L - 1)]
    h = H[i].copy()
    for a in range(3):
        e = np.zeros(3, dtype=int)
        e[a] = 1
        jp = idx[tuple((R[i] + e) % L)]
        jm = idx[tuple((R[i] - e) % L)]
        h += J[i, a] * s[jp] + J[jm, a] * s[jm]
    np.testing.assert_allclose(orc.local_field(s, J, H, L, i), h, atol=1e-14)


def _sim(orc, L, W_temps=2, n_rep=1, h_r=0.3, seed=3, codec="none"):
    smp = inputs.small_sample(L, n_temps=W_temps, h_r=h_r, disorder_seed=seed)
    return orc.OracleSim([smp], n_replicas=n_rep, seed=seed, codec=codec), smp


def test_or_sweeps_conserve_energy(orc):
    sim, smp = _sim(orc, 6, W_temps=2, n_rep=2)
    E0 = sim.energies()[0]
    sim.sweep_or(1000)
    E1 = sim.energies()[0]
    np.testing.assert_allclose(E1, E0, rtol=1e-12)
    # unit length kept
    np.testing.assert_allclose(np.linalg.norm(sim.spins()[0], axis=2), 1.0, atol=1e-14)


def test_or_even_odd_odd_even_is_identity(orc):
    sim, smp = _sim(orc, 4, W_temps=2, n_rep=1)
    o = sim.samples[0]
    s0 = o.s.copy()
    o.or_half(0)
    o.or_half(1)
    assert np.max(np.abs(o.s - s0)) > 1e-3      # the spins did move
    o.or_half(1)
    o.or_half(0)
    np.testing.assert_allclose(o.s, s0, atol=1e-12)


def test_checkerboard_order_independence(orc):
    """A half-sweep equals sequential site-by-site updates in any order (no bond
    joins two sites of one parity)."""
    sim, smp = _sim(orc, 4, W_temps=1, n_rep=1)
    o = sim.samples[0]
    s_ref = o.s[0].copy()
    lib = orc.lib()
    dp = ctypes.POINTER(ctypes.c_double)
    rng = np.random.default_rng(4)
    R = coords(4)
    sites = [i for i in rng.permutation(64) if R[i].sum() % 2 == 1]
    for i in sites:
        h = orc.local_field(s_ref, smp.J, smp.H, 4, int(i))
        v = s_ref[i].copy()
        lib.orc_or_move(v.ctypes.data_as(dp), h.ctypes.data_as(dp))
        s_ref[i] = v
    o.or_half(1)
    np.testing.assert_allclose(o.s[0], s_ref, atol=1e-15)


def test_measure_matches_fft(orc):
    rng = np.random.default_rng(12)
    L, R_T = 4, 3
    s = random_state(rng, 2 * R_T, L)
    perm = np.array([[2, 0, 1], [1, 2, 0]], dtype=np.int32)
    q = np.zeros((R_T, 3, 3))
    qk = np.zeros((R_T, 3, 3, 3, 2))
    dp = ctypes.POINTER(ctypes.c_double)
    orc.lib().orc_measure(np.ascontiguousarray(s).ctypes.data_as(dp), L, R_T,
                          perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          q.ctypes.data_as(dp), qk.ctypes.data_as(dp))
    for t in range(R_T):
        a, b = s[perm[0, t]], s[R_T + perm[1, t]]
        for mu, nu in itertools.product(range(3), range(3)):
            p = (a[:, mu] * b[:, nu]).reshape(L, L, L)       # [z, y, x]
            f = np.fft.ifftn(p)                               # (1/N) sum p e^{+i k.r}
            assert abs(q[t, mu, nu] - f[0, 0, 0].real) < 1e-14
            for ax, idx in enumerate([(0, 0, 1), (0, 1, 0), (1, 0, 0)]):
                assert abs(qk[t, ax, mu, nu, 0] - f[idx].real) < 1e-14
                assert abs(qk[t, ax, mu, nu, 1] - f[idx].imag) < 1e-14
    # self overlap has unit trace
    s2 = np.concatenate([s[:R_T], s[:R_T]])
    ident = np.tile(np.arange(R_T, dtype=np.int32), (2, 1))
    orc.lib().orc_measure(np.ascontiguousarray(s2).ctypes.data_as(dp), L, R_T,
                          ident.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          q.ctypes.data_as(dp), qk.ctypes.data_as(dp))
    np.testing.assert_allclose(np.trace(q, axis1=1, axis2=2), 1.0, atol=1e-14)


def test_init_uniform_on_sphere(orc):
    from scipy import stats
    sim, _ = _sim(orc, 16, W_temps=4, n_rep=2)
    s = sim.spins()[0].reshape(-1, 3)
    np.testing.assert_allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    assert np.all(np.abs(s.mean(axis=0)) < 5 * np.sqrt(1 / 3 / len(s)))
    assert stats.kstest(s[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-4
    phi = np.arctan2(s[:, 1], s[:, 0])
    assert stats.kstest(phi, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-4


def test_paper_field_has_fixed_length_and_uniform_direction():
    """The paper's random field (Sec. 2): fixed |H| and a uniformly random
    direction (inputs.make_sample(field="sphere")): |H_i| = H_r at every site,
    cos(theta) uniform on [-1, 1] (Kolmogorov-Smirnov) and no preferred axis."""
    from scipy import stats
    from paper_1204_6192_gb300 import inputs
    smp = inputs.make_sample(16, np.array([0.5, 1.0]), 0.3, disorder_seed=4, field="sphere")
    n = np.linalg.norm(smp.H, axis=1)
    np.testing.assert_allclose(n, 0.3, rtol=1e-12)
    c = smp.H[:, 2] / n
    assert stats.kstest(c, stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3
    assert np.abs(smp.H.mean(axis=0)).max() < 5 * 0.3 / np.sqrt(3 * len(n))


def test_results_do_not_depend_on_the_thread_count():
    """The parallel loops run over independent systems or sites, so one thread
    and all threads give the same bits (the timed CPU baseline uses both)."""
    import oracle
    L = oracle.lib()
    n0 = int(L.orc_num_threads())
    out = []
    try:
        for n in (1, max(2, n0)):
            L.orc_set_num_threads(n)
            smp = inputs.small_sample(8, n_temps=4, h_r=0.1, disorder_seed=11)
            sim = oracle.OracleSim([smp], 2, 5)
            sim.sweep_hb(2)
            sim.sweep_or(3)
            sim.pt_exchange()
            out.append((np.array(sim.spins()[0]), np.array(sim.energies()[0])))
    finally:
        L.orc_set_num_threads(n0)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
