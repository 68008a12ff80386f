"""Pins of the oracle's multi-hit tile schedule (Sec. 3.2, the double
checkerboard; Table 1's "10 x (1 HB + 10 OR)") against what fixes it
independently of its own loops:

* brute force: the same chain written as an explicit visiting list in Python
  (tiles of a colour in reversed order, sites of a parity in reversed order,
  since neither order may matter), with the moves taken from the separately
  pinned single-site routines;
* locality: a colour's pass leaves every spin of the other colour untouched;
* over-relaxation conserves each system's energy exactly (Eq. 3 keeps s.h);
* with J = 0 every spin is independent and the heat-bath draw is exact, so
  the mean energy is -sum_i |H_i| L(beta |H_i|) (Langevin function).
"""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import inputs


def coords(L):
    i = np.arange(L ** 3)
    return np.stack([i % L, (i // L) % L, i // (L * L)], axis=1)


def field(s, J, H, L, i):
    """h_i = sum over the 6 neighbours of J_ij s_j, + H_i (bond (i, i + e_a) is J[i, a])."""
    x, y, z = i % L, (i // L) % L, i // (L * L)
    h = H[i].copy() if H is not None else np.zeros(3)
    for a in range(3):
        c = [x, y, z]
        c[a] = (c[a] + 1) % L
        ip = c[0] + L * (c[1] + L * c[2])
        c = [x, y, z]
        c[a] = (c[a] - 1) % L
        im = c[0] + L * (c[1] + L * c[2])
        h += J[i, a] * s[ip] + J[im, a] * s[im]
    return h


def brute_multihit(s, J, H, L, T, n_rounds, n_or, n_hb, beta, sys_base, seed, sweep0):
    s = s.copy()
    W = s.shape[0]
    B = L // T
    R = coords(L)
    tiles = [(X, Y, Z) for Z in range(B) for Y in range(B) for X in range(B)]
    for w in range(W):
        for color in (0, 1):
            for (X, Y, Z) in reversed(tiles):
                if (X + Y + Z) % 2 != color:
                    continue
                inside = ((R[:, 0] // T == X) & (R[:, 1] // T == Y) & (R[:, 2] // T == Z))
                for r in range(n_rounds):
                    for k in range(n_or + n_hb):
                        sweep = sweep0 + r * (n_or + n_hb) + k
                        for parity in (0, 1):
                            sites = np.nonzero(inside & (R.sum(axis=1) % 2 == parity))[0][::-1]
                            for i in sites:
                                h = field(s[w], J, H, L, i)
                                if k < n_or:
                                    hh = h @ h
                                    v = 2.0 * (s[w, i] @ h) / hh * h - s[w, i] if hh > 0 else s[w, i]
                                    s[w, i] = v / np.linalg.norm(v)
                                else:
                                    g = sys_base + w
                                    out = oracle.philox(np.array([i, g >> 1, sweep, 1]), seed)[0]
                                    u1, u2 = oracle.uniform(out[2 * (g & 1): 2 * (g & 1) + 2])
                                    s[w, i] = oracle.hb_moves(s[w, i][None], h[None], [beta[w]],
                                                              [u1], [u2])[0]
    return s


def sample(L, seed, h_r=0.3, W=2):
    smp = inputs.small_sample(L, n_temps=W, h_r=h_r, disorder_seed=seed)
    o = oracle.OracleSample(L, smp.J, smp.H, smp.temps, 1, 6, 0, 17, 0)
    return smp, o


@pytest.mark.parametrize("T,n_rounds,n_or,n_hb", [(2, 2, 2, 1), (2, 1, 0, 2), (4, 1, 1, 1)])
def test_multihit_equals_explicit_visiting_list(T, n_rounds, n_or, n_hb):
    L = 8 if T == 4 else 4
    smp, o = sample(L, 3)
    s0 = o.s.copy()
    beta = o.beta_sys()
    o.multihit(T, n_rounds, n_or, n_hb, sweep0=5)
    ref = brute_multihit(s0, o.J, o.H, L, T, n_rounds, n_or, n_hb, beta, o.sys_base, o.seed, 5)
    np.testing.assert_allclose(o.s, ref, rtol=0, atol=1e-12)
    assert np.abs(o.s - s0).max() > 0.1


@pytest.mark.parametrize("color", [0, 1])
def test_one_colour_leaves_the_other_untouched(color):
    L, T = 8, 2
    _, o = sample(L, 4)
    s0 = o.s.copy()
    o.multihit(T, 2, 3, 1, sweep0=0, colors=1 << color)
    R = coords(L)
    tile_color = ((R // T).sum(axis=1)) % 2
    same = tile_color == color
    assert np.array_equal(o.s[:, ~same], s0[:, ~same])
    assert np.abs(o.s[:, same] - s0[:, same]).max() > 0.1


def test_over_relaxation_tiles_conserve_energy():
    L, T = 8, 4
    _, o = sample(L, 5, W=3)
    E0 = o.energies()
    o.multihit(T, 3, 5, 0, sweep0=0)
    np.testing.assert_allclose(o.energies(), E0, rtol=1e-12)


def test_independent_spins_follow_langevin():
    """J = 0, random fields: after one tile heat-bath sweep every spin is an
    exact draw, E = -sum_i H_i.s_i has mean -sum_i |H_i| (coth a - 1/a), a = beta |H_i|."""
    L, T, W = 8, 2, 64
    rng = np.random.default_rng(11)
    H = rng.normal(0.0, 0.7, size=(L ** 3, 3))
    temps = np.linspace(0.5, 2.0, W)
    o = oracle.OracleSample(L, np.zeros((L ** 3, 3)), H, temps, 1, 0, 0, 23, 0)
    o.multihit(T, 1, 0, 1, sweep0=0)
    E = o.energies()
    hn = np.linalg.norm(H, axis=1)
    for w, Tw in enumerate(temps):
        a = hn / Tw
        mean = -np.sum(hn * (1.0 / np.tanh(a) - 1.0 / a))
        # variance of -|H| cos t is |H|^2 (1 - L^2 - 2L/a) per spin
        Lg = 1.0 / np.tanh(a) - 1.0 / a
        sd = np.sqrt(np.sum(hn ** 2 * (1.0 - Lg ** 2 - 2.0 * Lg / a)))
        assert abs(E[w] - mean) < 4.5 * sd, (w, E[w], mean, sd)
