"""Pins of the oracle's single-spin moves and storage codecs.

Over-relaxation (Eq. 3): algebraic invariants.  Heat bath (Eq. 2): the exact
inverse CDF of cos(t) ~ exp(a cos t), the Langevin mean coth(a) - 1/a, the
beta -> 0 limit (uniform on the sphere) and the orthonormal frame around the
field.  Codecs: FP16 / BF16 rounding against numpy / torch, angle and
octahedral grids against their quantisation bounds.
"""
import numpy as np
import pytest
from scipy import stats


def unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def langevin(a):
    return 1.0 / np.tanh(a) - 1.0 / a


def cdf_cos(c, a):
    # P(cos t <= c) for density ~ exp(a c) on [-1, 1], in an overflow-safe form
    return (np.exp(a * (c - 1.0)) - np.exp(-2.0 * a)) / (1.0 - np.exp(-2.0 * a))


def test_or_invariants(orc):
    rng = np.random.default_rng(1)
    lib = orc.lib()
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    for _ in range(200):
        s = unit(rng, 1)[0].copy()
        h = rng.standard_normal(3) * rng.uniform(0.1, 5)
        s0 = s.copy()
        lib.orc_or_move(s.ctypes.data_as(dp), h.ctypes.data_as(dp))
        assert abs(np.linalg.norm(s) - 1) < 1e-14
        assert abs(s @ h - s0 @ h) < 1e-13 * np.linalg.norm(h)
        # the reflection flips the component perpendicular to h
        hp = h / np.linalg.norm(h)
        np.testing.assert_allclose(s - (s @ hp) * hp, -(s0 - (s0 @ hp) * hp), atol=1e-14)
        lib.orc_or_move(s.ctypes.data_as(dp), h.ctypes.data_as(dp))
        np.testing.assert_allclose(s, s0, atol=1e-14)
    # zero field leaves the spin unchanged
    s = np.array([0.6, 0.0, 0.8])
    lib.orc_or_move(s.ctypes.data_as(dp), np.zeros(3).ctypes.data_as(dp))
    np.testing.assert_allclose(s, [0.6, 0.0, 0.8], atol=0)


def test_hb_inverse_cdf_exact(orc):
    """cos(t) = F^{-1}(u1) exactly, F the CDF of exp(a cos t) on [-1, 1]."""
    rng = np.random.default_rng(2)
    n = 5000
    h = rng.standard_normal((n, 3)) * rng.uniform(0.01, 3, (n, 1))
    beta = rng.uniform(0.01, 20, n)
    u1 = rng.uniform(0, 1, n)
    u2 = rng.uniform(0, 1, n)
    s = orc.hb_moves(unit(rng, n), h, beta, u1, u2)
    hn = np.linalg.norm(h, axis=1)
    a = beta * hn
    c = np.einsum("ij,ij->i", s, h) / hn
    np.testing.assert_allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    ok = a < 30   # beyond this F is flat to machine precision near u1 ~ 1
    np.testing.assert_allclose(cdf_cos(c[ok], a[ok]), u1[ok], atol=1e-9)


def test_hb_azimuth_frame(orc):
    """cos t = 0 (a -> 0, u1 = 1/2) and phi = 0, pi/2, pi give e1, e2, -e1: orthonormal to n."""
    rng = np.random.default_rng(3)
    for n_ in list(unit(rng, 50)) + [np.array([0, 0, 1.0]), np.array([0, 0, -1.0]),
                                     np.array([1.0, 0, 0])]:
        h = n_ * 1e-14            # a = beta |h| below the small-a threshold
        outs = []
        for u2 in (0.0, 0.25, 0.5):
            outs.append(orc.hb_moves(np.zeros((1, 3)), h[None], 1.0, [0.5], [u2])[0])
        e1, e2, me1 = outs
        assert abs(e1 @ n_) < 1e-12 and abs(e2 @ n_) < 1e-12 and abs(e1 @ e2) < 1e-12
        np.testing.assert_allclose(me1, -e1, atol=1e-12)
        # right-handed: e1 x e2 = n
        np.testing.assert_allclose(np.cross(e1, e2), n_, atol=1e-12)


@pytest.mark.parametrize("a", [0.3, 1.0, 4.0, 25.0])
def test_hb_langevin_and_ks(orc, a):
    rng = np.random.default_rng(int(a * 100))
    n = 200_000
    hdir = unit(rng, 1)[0]
    h = np.tile(hdir * 2.0, (n, 1))
    beta = a / 2.0
    s = orc.hb_moves(np.zeros((n, 3)), h, beta, rng.uniform(0, 1, n), rng.uniform(0, 1, n))
    c = s @ hdir
    m = langevin(a)
    var = 1 - 2 * m / a - m * m      # Var(cos t) = 1 - 2L/a - L^2
    assert abs(c.mean() - m) < 5 * np.sqrt(var / n)
    ks = stats.kstest(c, lambda x: cdf_cos(np.clip(x, -1, 1), a))
    assert ks.pvalue > 1e-4
    # azimuth isotropic: perpendicular part has zero mean
    perp = s - np.outer(c, hdir)
    assert np.all(np.abs(perp.mean(axis=0)) < 5 * np.sqrt(1.0 / n))


def test_hb_beta_zero_uniform_sphere(orc):
    rng = np.random.default_rng(5)
    n = 200_000
    h = rng.standard_normal((n, 3))
    s = orc.hb_moves(np.zeros((n, 3)), h, 0.0, rng.uniform(0, 1, n), rng.uniform(0, 1, n))
    assert np.all(np.abs(s.mean(axis=0)) < 5 * np.sqrt(1 / 3 / n))
    np.testing.assert_allclose(s.T @ s / n, np.eye(3) / 3, atol=5e-3)
    assert stats.kstest(s[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-4


def test_round_fp16_matches_numpy(orc):
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.uniform(-1, 1, 20000), rng.uniform(-1e-4, 1e-4, 5000),
                        np.ldexp(rng.integers(-2047, 2048, 2000).astype(np.float64), -11),
                        np.ldexp(rng.integers(-4095, 4096, 2000).astype(np.float64), -12),
                        np.ldexp(rng.integers(-100, 100, 500).astype(np.float64), -25),
                        [0.0, 1.0, -1.0, 6.1e-5, 5.96e-8, 2.98e-8]])
    f = orc.lib().orc_round_fp16
    mine = np.array([f(float(v)) for v in x])
    np.testing.assert_array_equal(mine, x.astype(np.float16).astype(np.float64))


def test_round_bf16_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x32 = np.concatenate([rng.uniform(-1, 1, 20000).astype(np.float32),
                          (np.ldexp(rng.integers(-511, 512, 2000).astype(np.float64), -9)
                           ).astype(np.float32)])
    f = orc.lib().orc_round_bf16
    mine = np.array([f(float(v)) for v in x32.astype(np.float64)])
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mine, ref)


@pytest.mark.parametrize("codec,bound", [("angle16", 1.0e-4), ("oct16", 1.2e-4)])
def test_angle_codecs(orc, codec, bound):
    rng = np.random.default_rng(8)
    v = np.concatenate([unit(rng, 50000), np.eye(3), -np.eye(3),
                        unit(rng, 10) * [1, 1, 0] / np.linalg.norm(unit(rng, 10) * [1, 1, 0],
                                                                     axis=1, keepdims=True)])
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    r = orc.codec_roundtrip(v, codec)
    np.testing.assert_allclose(np.linalg.norm(r, axis=1), 1.0, atol=1e-14)
    err = np.linalg.norm(r - v, axis=1)
    assert err.max() < bound
    # decoding is a projection: re-encoding a decoded vector is the identity
    np.testing.assert_allclose(orc.codec_roundtrip(r, codec), r, atol=1e-12)


def test_fp32_storage_matches_numpy(orc):
    rng = np.random.default_rng(10)
    v = np.concatenate([unit(rng, 5000), rng.uniform(-1, 1, (100, 3))])
    np.testing.assert_array_equal(orc.codec_roundtrip(v, "fp32"),
                                  v.astype(np.float32).astype(np.float64))


def test_component_codecs_bound(orc):
    rng = np.random.default_rng(9)
    v = unit(rng, 20000)
    for codec, eps in (("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)):
        r = orc.codec_roundtrip(v, codec)
        assert np.all(np.abs(r - v) <= eps * np.maximum(np.abs(v), 2.0 ** -14) + 1e-300)


def test_yx4_codec_exact_on_grid(orc):
    """The paper's packing (Sec. 3.3), binary32 s_y and s_x + 4 sign(s_z): for s_x,
    s_y on a 2^-12 grid both stored numbers are exact, so the round trip gives
    s_x, s_y back unchanged, keeps the sign of s_z and restores a unit vector."""
    rng = np.random.default_rng(12)
    x = rng.integers(-2896, 2897, 4000) / 4096.0
    y = rng.integers(-2896, 2897, 4000) / 4096.0
    keep = x * x + y * y < 1.0
    x, y = x[keep], y[keep]
    z = np.sqrt(1.0 - x * x - y * y) * rng.choice([-1.0, 1.0], x.size)
    v = np.stack([x, y, z], axis=1)
    r = orc.codec_roundtrip(v, "yx4")
    np.testing.assert_array_equal(r[:, :2], v[:, :2])
    np.testing.assert_array_equal(np.sign(r[:, 2]), np.sign(z))
    np.testing.assert_allclose(np.linalg.norm(r, axis=1), 1.0, atol=1e-15)


def test_yx4_codec_bounds(orc):
    """Unit spins: s_x is stored as s_x + 4 in binary32 (half an ulp of [2, 8) is
    at most 2^-22), s_y in binary32 (at most 2^-25 for |s_y| < 1); the sign of s_z
    survives; decoding then re-encoding is the identity away from s_z = 0."""
    rng = np.random.default_rng(13)
    v = unit(rng, 40000)
    r = orc.codec_roundtrip(v, "yx4")
    assert np.abs(r[:, 0] - v[:, 0]).max() <= 2.0 ** -22
    assert np.abs(r[:, 1] - v[:, 1]).max() <= 2.0 ** -25
    nz = r[:, 2] != 0.0
    np.testing.assert_array_equal(np.sign(r[nz, 2]), np.sign(v[nz, 2]))
    assert np.abs(np.linalg.norm(r, axis=1) - 1.0).max() < 1e-6
    np.testing.assert_array_equal(orc.codec_roundtrip(r[nz], "yx4"), r[nz])
