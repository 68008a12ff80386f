"""GPU multi-hit tile schedule (hsg_step_multihit; Sec. 3.2's double
checkerboard, Table 1's "10 x (1 HB + 10 OR)") against the oracle's
orc_multihit on the same states and random numbers.

The chains are chaotic, so the GPU's FP32 arithmetic is measured against the
spread that binary32 storage alone produces in the FP64 oracle (as for the
lattice sweeps), with the median held at FP32 rounding.
"""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu

CHAOS_FACTOR = {0.5: 10.0, 0.9: 20.0, 0.99: 20.0, 1.0: 30.0}


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def f32(smp):
    r = lambda a: None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)
    return inputs.Sample(L=smp.L, J=r(smp.J), H=r(smp.H), temps=smp.temps)


def seeded_state(rng, W, N):
    s = rng.standard_normal((W, N, 3))
    return (s / np.linalg.norm(s, axis=2, keepdims=True)).astype(np.float32)


def from_seeded_state(samples, n_rep, seed, mh, precision="fp32", codec="none", j16=False):
    """Both sides start from the same seeded state and run one multi-hit step."""
    rng = np.random.default_rng(seed)
    states = [seeded_state(rng, n_rep * len(s.temps), s.L ** 3) for s in samples]
    ctx = hsg.Context(samples, n_rep, seed, precision=precision, j_fp16=j16)
    orc = oracle.OracleSim(samples, n_rep, seed, codec=codec)
    ctx.set_spins(states)
    for o, st in zip(orc.samples, states):
        o.s = st.astype(np.float64)
        if codec != "none":
            o.s = oracle.codec_roundtrip(o.s.reshape(-1, 3), codec).reshape(o.s.shape)
    ctx.step_multihit(1, **mh)
    orc.step_multihit(1, **mh)
    out = (ctx.get_spins(), orc.spins(), ctx.get_perm(), [o.perm for o in orc.samples],
           ctx.counters())
    ctx.close()
    return out


def fp32_storage_reference(samples, n_rep, seed, mh):
    """|FP64 oracle - FP64 oracle with binary32 storage| after one multi-hit
    step from the seeded state of from_seeded_state: the spread binary32
    storage alone produces, the scale GPU differences are measured against."""
    rng = np.random.default_rng(seed)
    states = [seeded_state(rng, n_rep * len(s.temps), s.L ** 3) for s in samples]
    a = oracle.OracleSim(samples, n_rep, seed)
    b = oracle.OracleSim(samples, n_rep, seed, codec="fp32")
    for sim in (a, b):
        for o, st in zip(sim.samples, states):
            o.s = st.astype(np.float64)
        sim.step_multihit(1, **mh)
    return np.concatenate([np.abs(x - y).ravel() for x, y in zip(a.spins(), b.spins())])


def assert_within_fp32_spread(d, ref):
    for q, k in CHAOS_FACTOR.items():
        lim = k * np.quantile(ref, q) + 1e-6
        assert np.quantile(d, q) <= lim, (q, np.quantile(d, q), lim)


@pytest.mark.parametrize("L,tile", [(8, 4), (16, 4), (16, 8)])
@pytest.mark.parametrize("n_or,n_hb", [(1, 0), (0, 1)])
def test_one_tile_sweep(L, tile, n_or, n_hb):
    """One tile sweep per tile (both colours) from an identical state.  A tile
    sweep chains four dependent stages (colour 0 even, odd, colour 1 even, odd)
    where a lattice sweep chains two, so a site with a small field can carry
    FP32 rounding slightly past 1e-5: the median must stay at FP32 rounding,
    the distribution within the binary32 spread of the FP64 chain."""
    smp = f32(inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L, t_min=0.15, t_max=0.6))
    mh = dict(tile=tile, n_rounds=1, n_or=n_or, n_hb=n_hb)
    g, o, _, _, cnt = from_seeded_state([smp], 2, 7, mh)
    d = np.abs(g[0] - o[0]).ravel()
    assert np.median(d) < 1e-7 and d.max() < 1e-4, (np.median(d), d.max())
    assert_within_fp32_spread(d, fp32_storage_reference([smp], 2, 7, mh))
    sweeps, passes = cnt
    assert int(sweeps[0]) == n_or + n_hb and int(passes[0]) == 1


@pytest.mark.parametrize("Ls,tile", [((8, 8), 4), ((16, 16), 8), ((8, 16), 4)])
def test_multihit_step_within_fp32_spread(Ls, tile):
    """Two rounds of (3 OR + 1 HB) per tile, then energies and PT, for a batch
    of two samples (of equal or different size): spins within the binary32
    spread of the FP64 chain, identical permutations and counters."""
    mh = dict(tile=tile, n_rounds=2, n_or=3, n_hb=1)
    samples = [f32(inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L + k, t_min=0.3,
                                       t_max=0.8)) for k, L in enumerate(Ls)]
    g, o, pg, po, cnt = from_seeded_state(samples, 2, 9, mh)
    d = np.concatenate([np.abs(a - b).ravel() for a, b in zip(g, o)])
    assert_within_fp32_spread(d, fp32_storage_reference(samples, 2, 9, mh))
    for a, b in zip(pg, po):
        np.testing.assert_array_equal(a, b)
    assert [int(x) for x in cnt[0]] == [8, 8] and [int(x) for x in cnt[1]] == [1, 1]


@pytest.mark.parametrize("precision", ["fp16", "bf16", "angle16", "oct16", "yx4"])
def test_multihit_compressed_one_tile_sweep(precision):
    """FP16 couplings, compressed spins, one OR and one HB tile sweep: equal up
    to one storage quantum (a site with a small field amplifies it).  For the
    paper's packing the scale is the format's own sensitivity: one unit in the
    last place of s_x + 4 sign s_z moves a decoded s_z near the equator by
    ~1e-4 after a sweep."""
    quant = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8, "angle16": 1.1e-4, "oct16": 1.3e-4,
             "yx4": 1e-4}[precision]
    smp = inputs.small_sample(8, n_temps=4, h_r=0.2)
    smp16 = inputs.Sample(L=8, J=inputs.round_fp16(smp.J), H=inputs.round_fp16(smp.H),
                          temps=smp.temps)
    g, o, _, _, _ = from_seeded_state([smp16], 2, 3, dict(tile=4, n_rounds=1, n_or=1, n_hb=1),
                                      precision=precision, codec=precision, j16=True)
    d = np.abs(g[0] - o[0]).ravel()
    assert np.quantile(d, 0.99) < 3 * quant, np.quantile(d, 0.99)
    assert np.median(d) < quant and d.max() < 0.05, d.max()


def test_multihit_over_relaxation_conserves_energy():
    """Tiles of over-relaxation sweeps only (10 rounds x 10 OR): every system's
    energy is unchanged up to FP32 rounding."""
    samples = [inputs.small_sample(16, n_temps=4, h_r=0.1, disorder_seed=3)]
    ctx = hsg.Context(samples, 2, 1)
    ctx.sweep_hb(2)
    E0 = ctx.energies()[0]
    ctx.step_multihit(1, tile=8, n_rounds=10, n_or=10, n_hb=0)
    E1 = ctx.last_energies()[0]
    np.testing.assert_allclose(E1, E0, rtol=2e-5)
    ctx.close()


def test_multihit_frozen_sample_is_untouched():
    samples = [inputs.small_sample(8, n_temps=3, disorder_seed=k) for k in (1, 2)]
    ctx = hsg.Context(samples, 2, 4)
    before = [s.copy() for s in ctx.get_spins()]
    ctx.set_active([1, 0])
    ctx.step_multihit(2, tile=4, n_rounds=2, n_or=2, n_hb=1)
    after = ctx.get_spins()
    assert np.abs(after[0] - before[0]).max() > 0.1
    np.testing.assert_array_equal(after[1], before[1])
    sweeps, passes = ctx.counters()
    assert [int(x) for x in sweeps] == [2 * 2 * 3, 0] and [int(x) for x in passes] == [2, 0]
    ctx.close()


def test_multihit_invalid_arguments():
    ctx = hsg.Context([inputs.small_sample(12, n_temps=2)], 2, 1)
    for kw in (dict(tile=4), dict(tile=6), dict(tile=2)):
        with pytest.raises(hsg.HsgError):          # 12 is not a multiple of 8; 6, 2 unsupported
            ctx.step_multihit(1, **kw)
    ctx.close()
    ctx = hsg.Context([inputs.small_sample(8, n_temps=2)], 2, 1)
    for kw in (dict(n_rounds=0), dict(n_or=0, n_hb=0), dict(n_or=-1)):
        with pytest.raises(hsg.HsgError):
            ctx.step_multihit(1, tile=4, **kw)
    ctx.step_multihit(1, tile=4, n_rounds=1, n_or=1, n_hb=1)   # not sticky
    ctx.close()


def test_multihit_independent_spins_follow_langevin():
    """J = 0, random fields: after one heat-bath tile sweep every spin is an
    exact draw; the mean energy per system is -sum_i |H_i| (coth a - 1/a)."""
    L, R_T = 16, 32
    rng = np.random.default_rng(5)
    H = rng.normal(0.0, 0.7, size=(L ** 3, 3))
    temps = np.geomspace(0.5, 2.0, R_T)
    smp = inputs.Sample(L=L, J=np.zeros((L ** 3, 3)), H=H.astype(np.float32).astype(np.float64),
                        temps=temps)
    ctx = hsg.Context([smp], 1, 13)
    ctx.step_multihit(1, tile=8, n_rounds=1, n_or=0, n_hb=1)
    # the tiles were updated before the step's PT pass, at the initial
    # assignment: memory slot t at temperature t
    E = ctx.last_energies()[0]
    hn = np.linalg.norm(smp.H, axis=1)
    for t, T in enumerate(temps):
        a = hn / T
        Lg = 1.0 / np.tanh(a) - 1.0 / a
        mean = -np.sum(hn * Lg)
        sd = np.sqrt(np.sum(hn ** 2 * (1.0 - Lg ** 2 - 2.0 * Lg / a)))
        assert abs(E[t] - mean) < 4.5 * sd, (t, E[t], mean, sd)
    ctx.close()


def test_multihit_fast_math_heat_bath():
    """The fast-math heat bath (hardware exp/log/sincos) in tiles: one tile
    sweep from an identical state stays within the intrinsics' error of the
    FP64 oracle (median 1e-6, max 1e-3)."""
    smp = f32(inputs.small_sample(8, n_temps=4, h_r=0.2, disorder_seed=8, t_min=0.15, t_max=0.6))
    rng = np.random.default_rng(4)
    st = seeded_state(rng, 8, 512)
    ctx = hsg.Context([smp], 2, 4, fast_math=True)
    orc = oracle.OracleSim([smp], 2, 4)
    ctx.set_spins([st])
    orc.samples[0].s = st.astype(np.float64)
    ctx.step_multihit(1, tile=4, n_rounds=1, n_or=0, n_hb=1)
    orc.step_multihit(1, tile=4, n_rounds=1, n_or=0, n_hb=1)
    d = np.abs(ctx.get_spins()[0] - orc.spins()[0]).ravel()
    assert np.median(d) < 1e-6 and d.max() < 1e-3, (np.median(d), d.max())
    ctx.close()


def test_multihit_checkpoint_round_trip_and_persistent_context():
    """A checkpoint taken between multi-hit steps restores the chain exactly
    (spins, permutations, counters); a context on the persistent schedule runs
    the same tile kernels with the same result."""
    samples = [inputs.small_sample(8, n_temps=4, h_r=0.1, disorder_seed=5)]
    mh = dict(tile=4, n_rounds=2, n_or=2, n_hb=1)
    out = []
    for variant in (hsg.VARIANT_TWO_PASS, hsg.VARIANT_PERSISTENT):
        ctx = hsg.Context(samples, 2, 6, variant=variant)
        ctx.step_multihit(1, **mh)
        blob = ctx.checkpoint()
        ctx.step_multihit(2, **mh)
        ref = (ctx.get_spins()[0].copy(), ctx.get_perm()[0].copy(), ctx.counters())
        ctx.restore(blob)
        ctx.step_multihit(2, **mh)
        np.testing.assert_array_equal(ctx.get_spins()[0], ref[0])
        np.testing.assert_array_equal(ctx.get_perm()[0], ref[1])
        assert [int(x) for x in ctx.counters()[0]] == [int(x) for x in ref[2][0]] == [18]
        out.append(ref[0])
        ctx.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_multihit_samples_the_same_equilibrium():
    """Tiles with a fixed halo are a different Markov chain with the same
    stationary distribution: e(T) per temperature slot from the tile schedule
    (one round of 5 OR + 1 HB per 4^3 tile, then PT) agrees with the lattice
    step (1 HB + 5 OR + PT) within the statistical errors (second half of 2000
    steps, 10 bins, L = 8, 2 replicas x 8 temperatures in [0.15, 0.6])."""
    t = inputs.geometric_temperatures(0.15, 0.6, 8)
    smp = inputs.make_sample(8, t, 0.0, disorder_seed=1)
    steps, nb = 2000, 10

    def e_of_T(multihit):
        ctx = hsg.Context([smp], 2, 5)
        E = []
        for _ in range(steps):
            if multihit:
                ctx.step_multihit(1, tile=4, n_rounds=1, n_or=5, n_hb=1)
            else:
                ctx.step(1)
            E.append(ctx.measure(q=False)["E"][0].mean(axis=0) / 512)   # per slot, replica mean
        ctx.close()
        x = np.array(E)[steps // 2:]
        bins = np.array([b.mean(axis=0) for b in np.array_split(x, nb)])
        return x.mean(axis=0), bins.std(axis=0, ddof=1) / np.sqrt(nb)

    (m1, s1), (m2, s2) = e_of_T(False), e_of_T(True)
    z = (m1 - m2) / np.sqrt(s1 ** 2 + s2 ** 2)
    print("e(T) lattice", np.round(m1, 4), "tiles", np.round(m2, 4), "z", np.round(z, 2))
    assert np.all(np.abs(z) < 4.5) and np.sum(np.abs(z) > 2.5) <= 2, z
