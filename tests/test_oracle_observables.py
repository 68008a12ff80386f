"""Pins of the oracle's chirality and replica-pair overlaps (Sec. 2: local
chirality kappa_i^a = s_{i+a} . (s_i x s_{i-a}), the chiral overlap, and the
scalar pair overlaps the four-replica sums chi_1, chi_2, chi_3 are built from).

Each check compares with something fixed outside the oracle's own formulas:
a closed form for a conical spiral, the transformation laws of dot and triple
products under proper and improper rotations, numpy's FFT for the k-modes,
and the phase a lattice translation multiplies them by.
"""
import numpy as np
import pytest

import oracle


def coords(L):
    i = np.arange(L ** 3)
    return np.stack([i % L, (i // L) % L, i // (L * L)], axis=1)


def cone_spiral(L, axis, m, phi):
    """s_j = (sin phi cos(j theta), sin phi sin(j theta), cos phi), j the coordinate
    along `axis`, theta = 2 pi m / L (periodic)."""
    th = 2 * np.pi * m / L
    j = coords(L)[:, axis]
    return np.stack([np.sin(phi) * np.cos(j * th), np.sin(phi) * np.sin(j * th),
                     np.full(j.shape, np.cos(phi))], axis=1)


def random_spins(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("m,phi", [(1, 0.7), (3, 1.2), (2, 2.5)])
def test_chirality_of_conical_spiral(axis, m, phi):
    """Three consecutive spins of a cone of half-angle phi, azimuth step theta:
    s_{+1} . (s_0 x s_{-1}) = cos(phi) sin(phi)^2 (sin 2 theta - 2 sin theta)
    (the determinant of the three rows, worked out by hand); zero along the two
    other axes, where the three spins coincide."""
    L = 8
    th = 2 * np.pi * m / L
    k = oracle.chirality(cone_spiral(L, axis, m, phi), L)
    expect = np.cos(phi) * np.sin(phi) ** 2 * (np.sin(2 * th) - 2 * np.sin(th))
    np.testing.assert_allclose(k[:, axis], expect, atol=1e-13)
    for other in {0, 1, 2} - {axis}:
        np.testing.assert_allclose(k[:, other], 0.0, atol=1e-14)


def test_chirality_is_odd_and_rotation_invariant():
    rng = np.random.default_rng(3)
    L = 6
    s = random_spins(rng, L ** 3)
    k = oracle.chirality(s, L)
    R = random_rotation(rng)
    np.testing.assert_allclose(oracle.chirality(s @ R.T, L), k, atol=1e-13)
    np.testing.assert_allclose(oracle.chirality(-s, L), -k, atol=1e-15)
    # a reflection (det -1) flips every triple product
    M = R @ np.diag([1.0, 1.0, -1.0])
    np.testing.assert_allclose(oracle.chirality(s @ M.T, L), -k, atol=1e-13)


def make_state(rng, L, R_O, R_T):
    W = R_O * R_T
    s = random_spins(rng, W * L ** 3).reshape(W, L ** 3, 3)
    perm = np.array([rng.permutation(R_T) for _ in range(R_O)], dtype=np.int32)
    return s, perm


def pairs(R_O):
    P = [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]
    r = min(R_O, 4)
    return [p for p in P if p[1] < r]


@pytest.mark.parametrize("R_O", [2, 3, 4, 5])
def test_overlap_modes_equal_numpy_fft(R_O):
    """D_ab(k) and C_ab^a(k) at k = 0, (2 pi/L) e_x,y,z equal the numpy FFT of the
    site fields s^A.s^B and kappa^A kappa^B (sign e^{+ik.R}: N * ifftn)."""
    rng = np.random.default_rng(R_O)
    L, R_T = 6, 3
    s, perm = make_state(rng, L, R_O, R_T)
    D, C = oracle.overlaps(s, L, R_O, R_T, perm)
    assert D.shape == (R_T, len(pairs(R_O)), 4, 2)
    N = L ** 3
    modes = [(0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]   # ifftn index order (z, y, x)
    for t in range(R_T):
        for p, (a, b) in enumerate(pairs(R_O)):
            A = s[a * R_T + perm[a, t]]
            B = s[b * R_T + perm[b, t]]
            d = np.fft.ifftn((A * B).sum(axis=1).reshape(L, L, L))
            kA, kB = oracle.chirality(A, L), oracle.chirality(B, L)
            for m, idx in enumerate(modes):
                np.testing.assert_allclose(D[t, p, m], [d[idx].real, d[idx].imag], atol=1e-13)
                for al in range(3):
                    c = np.fft.ifftn((kA[:, al] * kB[:, al]).reshape(L, L, L))
                    np.testing.assert_allclose(C[t, p, al, m], [c[idx].real, c[idx].imag],
                                               atol=1e-13)
    assert N == L ** 3


def test_overlaps_under_rotations_and_reflections():
    """Rotating one replica changes D but not C (kappa is rotation invariant);
    s -> -s of one replica flips the sign of both; the same rotation of both
    leaves both unchanged."""
    rng = np.random.default_rng(11)
    L, R_O, R_T = 4, 2, 2
    s, perm = make_state(rng, L, R_O, R_T)
    D, C = oracle.overlaps(s, L, R_O, R_T, perm)
    R = random_rotation(rng)
    s1 = s.copy()
    s1[R_T:] = s[R_T:] @ R.T                 # replica 1 rotated
    D1, C1 = oracle.overlaps(s1, L, R_O, R_T, perm)
    np.testing.assert_allclose(C1, C, atol=1e-13)
    assert np.abs(D1 - D).max() > 1e-3
    s2 = s.copy()
    s2[R_T:] = -s[R_T:]                      # replica 1 inverted
    D2, C2 = oracle.overlaps(s2, L, R_O, R_T, perm)
    np.testing.assert_allclose(D2, -D, atol=1e-14)
    np.testing.assert_allclose(C2, -C, atol=1e-14)
    D3, C3 = oracle.overlaps(s @ R.T, L, R_O, R_T, perm)
    np.testing.assert_allclose(D3, D, atol=1e-13)
    np.testing.assert_allclose(C3, C, atol=1e-13)


def test_translation_multiplies_modes_by_phase():
    """Shifting both configurations by one site along axis a multiplies the
    mode along a by e^{+i 2 pi / L} and leaves the others unchanged."""
    rng = np.random.default_rng(5)
    L, R_O, R_T = 6, 2, 1
    s, perm = make_state(rng, L, R_O, R_T)
    D, C = oracle.overlaps(s, L, R_O, R_T, perm)
    z = lambda v: v[..., 0] + 1j * v[..., 1]
    for a, shape_axis in ((0, 2), (1, 1), (2, 0)):   # x is the last axis of [z, y, x]
        sh = np.roll(s.reshape(-1, L, L, L, 3), 1, axis=1 + shape_axis).reshape(s.shape)
        Ds, Cs = oracle.overlaps(sh, L, R_O, R_T, perm)
        ph = np.exp(2j * np.pi / L)
        for m in range(4):
            f = ph if m == a + 1 else 1.0
            np.testing.assert_allclose(z(Ds[:, :, m]), f * z(D[:, :, m]), atol=1e-13)
            np.testing.assert_allclose(z(Cs[:, :, :, m]), f * z(C[:, :, :, m]), atol=1e-13)


def test_self_overlap_is_one():
    """D of a configuration with itself is (1/N) sum |s|^2 = 1 at k = 0."""
    rng = np.random.default_rng(2)
    L, R_T = 4, 2
    s, _ = make_state(rng, L, 2, R_T)
    s[R_T:] = s[:R_T]
    perm = np.tile(np.arange(R_T, dtype=np.int32), (2, 1))
    D, _ = oracle.overlaps(s, L, 2, R_T, perm)
    np.testing.assert_allclose(D[:, 0, 0, 0], 1.0, atol=1e-14)
