"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP32 storage: sweep-by-sweep trajectories agree to 1e-5 per component (FP32
rounding, ~1e-7 per update, grows slowly over the first sweeps).
Compressed storage: one sweep from the same seeded state agrees within the
codec's quantum (the oracle applies the same storage rounding in FP64).
Integer work (parallel-tempering permutations) is compared exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
# storage quantum of one component (max over unit vectors): fp16 2^-11, bf16 2^-8,
# angle16 ~5e-5, oct16 ~6e-5
QUANT = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8, "angle16": 1.1e-4, "oct16": 1.3e-4, "yx4": 2.0 ** -22}


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def seeded_state(rng, W, N):
    s = rng.standard_normal((W, N, 3))
    return (s / np.linalg.norm(s, axis=2, keepdims=True)).astype(np.float32)


def f32(smp):
    """The sample as the library stores it: J and H rounded to binary32."""
    r = lambda a: None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)
    return inputs.Sample(L=smp.L, J=r(smp.J), H=r(smp.H), temps=smp.temps)


def run_pair(samples, n_rep, seed, schedule, precision="fp32", codec="none", j16=False):
    samples = [f32(s) for s in samples]
    ctx = hsg.Context(samples, n_rep, seed, precision=precision, j_fp16=j16)
    orc = oracle.OracleSim(samples, n_rep, seed, codec=codec)
    errs = []
    for g, o in zip(ctx.get_spins(), orc.spins()):
        errs.append(np.abs(g - o).max())
    for op, n in schedule:
        getattr(ctx, op)(n)
        getattr(orc, op)(n)
        e = max(np.abs(g - o).max() for g, o in zip(ctx.get_spins(), orc.spins()))
        errs.append(e)
    ctx.close()
    return np.array(errs)


def test_device_philox_bit_exact_against_oracle():
    """The device generator and the oracle's, both written from Salmon et al.,
    agree bit for bit on 10^6 counters (several seeds, every counter word)."""
    rng = np.random.default_rng(21)
    for seed in (1, 0xFFFFFFFF, 2 ** 40 + 17):
        ctr = rng.integers(0, 2 ** 32, size=(250_000, 4), dtype=np.uint64).astype(np.uint32)
        np.testing.assert_array_equal(hsg.hsg_philox(ctr, seed), oracle.philox(ctr, seed))


def test_initial_state_matches_oracle():
    smp = inputs.small_sample(8, n_temps=4)
    errs = run_pair([smp], 2, 5, [])
    assert errs[0] < 1e-7


def one_sweep_from_seeded_state(samples, n_rep, seed, op, precision="fp32", codec="none",
                                j16=False, pre_sweeps=0):
    """Both sides start from the same seeded float32 state (after `pre_sweeps`
    OR sweeps on both, so the sweep counter is not zero) and do one sweep."""
    samples = [f32(s) for s in samples]
    rng = np.random.default_rng(seed)
    states = [seeded_state(rng, n_rep * len(s.temps), s.L ** 3) for s in samples]
    ctx = hsg.Context(samples, n_rep, seed, precision=precision, j_fp16=j16)
    orc = oracle.OracleSim(samples, n_rep, seed, codec=codec)
    if pre_sweeps:
        ctx.sweep_or(pre_sweeps)
        orc.sweep_or(pre_sweeps)
    ctx.set_spins(states)
    for o, st in zip(orc.samples, states):
        o.s = st.astype(np.float64)
        if codec != "none":
            o.s = oracle.codec_roundtrip(o.s.reshape(-1, 3), codec).reshape(o.s.shape)
    getattr(ctx, op)(1)
    getattr(orc, op)(1)
    d = [np.abs(g - o) for g, o in zip(ctx.get_spins(), orc.spins())]
    ctx.close()
    return np.concatenate([x.ravel() for x in d])


@pytest.mark.parametrize("L", [4, 6, 8, 16])
@pytest.mark.parametrize("op", ["sweep_or", "sweep_hb"])
def test_one_sweep_fp32_strict(L, op):
    """One full sweep (even then odd half) from an identical state: every
    component within 1e-5 of the FP64 oracle."""
    smp = inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L, t_min=0.15, t_max=0.6)
    d = one_sweep_from_seeded_state([smp], 2, 7, op, pre_sweeps=3)
    assert d.max() < TOL_FP32, d.max()


def fp32_storage_reference(samples, n_rep, seed, schedule):
    """|FP64 oracle - FP64 oracle with binary32 spin storage| after the schedule.

    The dynamics amplify small differences (the FP64 oracle moved by 3e-8
    deviates by ~1e-3 after 9 sweeps at L = 8), so no FP32 implementation can
    follow the FP64 trajectory to a fixed max-norm over many sweeps; this is the
    spread that FP32 storage alone produces, the scale GPU differences are
    measured against."""
    a = oracle.OracleSim(samples, n_rep, seed)
    b = oracle.OracleSim(samples, n_rep, seed, codec="fp32")
    for op, n in schedule:
        getattr(a, op)(n)
        getattr(b, op)(n)
    return np.concatenate([np.abs(x - y).ravel() for x, y in zip(a.spins(), b.spins())])


# FP32 arithmetic adds a few ulp per update on top of the half-ulp storage
# rounding.  Measured over ten free-running sweeps of five shapes (L = 4, 8, 16;
# H_r 0 to 2; T from 0.1 to 5), the GPU's deviation from the FP64 oracle is
# 2.7-3.8x the FP32-storage spread at the median, 3.0-4.6x at the 90th and
# 3.1-6.0x at the 99th percentile, and 2.0-15.6x at the maximum (one site).
# At L = 4 (1536 components) the 99th percentile rests on ~15 values and was
# measured at 10.9x in test_or_hb_trajectory_fp32, so it gets 20x; the median
# and the 90th percentile 10x, the maximum 30x.  A wrong index, sign or random
# number gives O(1) deviations and fails all four.
CHAOS_FACTOR = {0.5: 10.0, 0.9: 10.0, 0.99: 20.0, 1.0: 30.0}


def assert_within_fp32_spread(d, ref):
    for q, k in CHAOS_FACTOR.items():
        lim = k * np.quantile(ref, q) + 1e-6
        assert np.quantile(d, q) <= lim, (q, np.quantile(d, q), lim)


def trajectory_check(samples, n_rep, seed, sched):
    samples = [f32(s) for s in samples]
    ctx = hsg.Context(samples, n_rep, seed)
    orc = oracle.OracleSim(samples, n_rep, seed)
    for op, n in sched:
        getattr(ctx, op)(n)
        getattr(orc, op)(n)
    d = np.concatenate([np.abs(g - o).ravel() for g, o in zip(ctx.get_spins(), orc.spins())])
    ctx.close()
    assert_within_fp32_spread(d, fp32_storage_reference(samples, n_rep, seed, sched))
    return d


@pytest.mark.parametrize("L", [4, 6, 8])
def test_or_hb_trajectory_fp32(L):
    smp = inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L, t_min=0.15, t_max=0.6)
    sched = [("sweep_hb", 1), ("sweep_or", 1)] * 2 + [("sweep_or", 3), ("sweep_hb", 1), ("sweep_or", 2)]
    trajectory_check([smp], 2, 7, sched)


def test_trajectory_config1_shape():
    """L = 8, Gaussian J, H = 0, 2 replicas x 8 temperatures in [0.15, 0.6], 10 sweeps."""
    w = inputs.workload("L8_plain")
    sched = [("sweep_hb", 1), ("sweep_or", 5), ("sweep_hb", 1), ("sweep_or", 3)]
    trajectory_check(w.samples, w.n_replicas, w.seed, sched)


# a step's sweeps and the first four of the next: 1 HB + 5 OR, then 1 HB + 3 OR
STEP_SWEEPS = ["sweep_hb"] + ["sweep_or"] * 5 + ["sweep_hb"] + ["sweep_or"] * 3


def parity_mask(L):
    x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return ((x + y + z) % 2).transpose(2, 1, 0).ravel()      # site = x + L (y + L z)


U32 = 2.0 ** -24          # unit roundoff of binary32


def field_conditioning(s, J, H, L):
    """kappa_i = (sum_j |J_ij| + |H_i|) / |h_i| per system and site, with h the
    local field of the state s [W, N, 3] in FP64 (for the error bound only)."""
    W = s.shape[0]
    a = s.reshape(W, L, L, L, 3)                     # [w, z, y, x, c]
    Jg = J.reshape(L, L, L, 3)                       # bonds +x, +y, +z of each site
    h = np.zeros_like(a)
    S = np.zeros((L, L, L))
    for c, ax in ((0, 3), (1, 2), (2, 1)):           # bond direction c along array axis ax
        jp = Jg[..., c]                              # bond to the + neighbour
        jm = np.roll(jp, 1, axis=ax - 1)             # bond to the - neighbour
        h += jp[None, ..., None] * np.roll(a, -1, axis=ax)
        h += jm[None, ..., None] * np.roll(a, 1, axis=ax)
        S += np.abs(jp) + np.abs(jm)
    if H is not None:
        Hg = H.reshape(L, L, L, 3)
        h += Hg[None]
        S = S + np.linalg.norm(Hg, axis=-1)
    hn = np.linalg.norm(h, axis=-1)
    return (S[None] / np.maximum(hn, 1e-300)).reshape(W, -1)


def move_bound(kappa):
    """Largest deviation of one move evaluated in binary32 from the exact one,
    to first order: the field's 7 rounded products and sums err by at most
    8 u sum |J s| (Higham's summation bound), which turns its direction by at
    most 16 u kappa and the moved spin by at most 4x that (the reflection of
    Eq. 3 doubles it twice; the heat bath's frame, Eq. 2, turns with it by less).
    1e-5 wherever that is smaller."""
    return np.maximum(TOL_FP32, 64.0 * U32 * kappa)


def half_sweep_deviations(samples, n_rep, seed, sweeps=STEP_SWEEPS):
    """Consecutive sweeps in a step's order, each half-sweep compared from
    identical inputs.  Before a sweep the oracle takes the GPU's binary32
    state S0 and does the even half-sweep; the GPU does the whole sweep (S1).
    The GPU's even sites in S1 are its even half-sweep's output (the odd half
    does not touch them), so the oracle's odd half-sweep then starts from the
    even sites of S1 and the odd sites of S0 -- the GPU's own intermediate state.
    Returns, per half-sweep, the largest component deviation, the largest
    deviation relative to move_bound, and the largest deviation at sites whose
    field is well conditioned (kappa <= 100) with the number of other sites."""
    samples = [f32(s) for s in samples]
    ctx = hsg.Context(samples, n_rep, seed)
    orc = oracle.OracleSim(samples, n_rep, seed)
    odd = [parity_mask(s.L).astype(bool) for s in samples]
    out = []
    for op in sweeps:
        s0 = ctx.get_spins()
        getattr(ctx, op)(1)
        s1 = ctx.get_spins()
        rec = [[0.0, 0.0, 0.0, 0] for _ in range(2)]
        for o, a, b, m, smp in zip(orc.samples, s0, s1, odd, samples):
            for parity in (0, 1):
                if parity == 0:
                    o.s = a.astype(np.float64)
                else:
                    mid = a.astype(np.float64)
                    mid[:, ~m] = b[:, ~m]
                    o.s = mid
                kap = field_conditioning(o.s, smp.J, smp.H, smp.L)
                if op == "sweep_hb":
                    o.hb_half(parity, o.sweep)
                else:
                    o.or_half(parity)
                sel = m if parity else ~m
                d = np.abs(o.s[:, sel] - b[:, sel]).max(axis=-1)          # [W, sites]
                k = kap[:, sel]
                r = rec[parity]
                r[0] = max(r[0], float(d.max()))
                r[1] = max(r[1], float((d / move_bound(k)).max()))
                good = k <= 100.0
                r[2] = max(r[2], float(d[good].max()))
                r[3] += int((~good).sum())
            o.sweep += 1
        out.append(rec)
    ctx.close()
    return np.array(out)          # [sweep, parity, (max dev, max dev / bound, max dev kappa<=100, n kappa>100)]


@pytest.mark.parametrize("shape", ["L8_plain", "L16_field"])
def test_ten_sweeps_each_half_from_the_gpu_state_within_1e5(shape):
    """Ten consecutive sweeps (HB, 5 OR, HB, 3 OR; sweep counters 0-9); every
    half-sweep is compared with the FP64 oracle from identical inputs, the
    GPU's own state.  Every component of every system is within 1e-5 at every
    site whose local field is not nearly cancelled (kappa <= 100, i.e. |h|
    above ~1/100 of the sum of its terms), and within the binary32 error bound
    of the move (move_bound) at the few sites where it is.  L8_plain: L = 8,
    H = 0, 2 x 8 temperatures in [0.15, 0.6]; L16_field: L = 16, H_r = 0.05,
    2 x 8 temperatures in [0.1, 0.4]."""
    if shape == "L8_plain":
        w = inputs.workload("L8_plain")
        samples, n_rep, seed = w.samples, w.n_replicas, w.seed
    else:
        samples = [inputs.small_sample(16, n_temps=8, h_r=0.05, disorder_seed=16, t_min=0.1,
                                       t_max=0.4)]
        n_rep, seed = 2, 3
    r = half_sweep_deviations(samples, n_rep, seed)
    print(f"\n[{shape}] per half-sweep (even | odd): max |GPU - oracle|, max ratio to the move's "
          f"binary32 bound, max at kappa <= 100, sites with kappa > 100")
    for k in range(r.shape[0]):
        print(f"  {STEP_SWEEPS[k]:9s} " + " | ".join(
            f"{x[0]:.2e} {x[1]:.3f} {x[2]:.2e} {int(x[3])}" for x in r[k]))
    assert np.all(r[..., 2] < TOL_FP32), r[..., 2]
    assert np.all(r[..., 1] <= 1.0), r[..., 1]


def test_field_dominated_trajectory_ten_sweeps_within_1e5():
    """Where the random field dominates the couplings (H_r = 10 against |J| ~ 1)
    a spin's move depends on its neighbours through J/|h| << 1, so rounding
    differences shrink from sweep to sweep instead of growing: the free-running
    FP32 trajectory stays within 1e-5 per component of the FP64 oracle through
    ten sweeps of a step's order (HB, 5 OR, HB, 3 OR), at L = 8, 2 x 4
    temperatures in [0.15, 0.6]."""
    smp = f32(inputs.small_sample(8, n_temps=4, h_r=10.0, disorder_seed=8, t_min=0.15, t_max=0.6))
    ctx = hsg.Context([smp], 2, 7)
    orc = oracle.OracleSim([smp], 2, 7)
    dev = []
    for op in STEP_SWEEPS:
        getattr(ctx, op)(1)
        getattr(orc, op)(1)
        dev.append(max(np.abs(g - o).max() for g, o in zip(ctx.get_spins(), orc.spins())))
    ctx.close()
    print(f"\n[field-dominated] max |GPU - oracle| per sweep: {np.array2string(np.array(dev), precision=2)}")
    assert max(dev) < TOL_FP32, dev


def test_heat_bath_in_a_strong_field_near_the_equator():
    """Heat-bath draws at a = beta |h| = 8 ... 11 (no couplings, a unit field of
    random direction, T = 1/11 ... 1/8), where exp(-2a) is below half an ulp of
    1: draws near the equator (u1 ~ exp(-a)) need the (1 - u1) exp(-2a) term of
    the inverse CDF, which a binary32 1 + (1 - u1)(exp(-2a) - 1) loses (up to
    1.4e-5 in cos t at a = 9).  Without couplings every site is independent, so
    three sweeps of 16^3 sites x 8 systems (~10^5 draws, dozens near the equator
    at each a) compare move by move: every component within 2e-6."""
    L = 16
    rng = np.random.default_rng(23)
    H = inputs.sphere_field(L, 1.0, rng)
    smp = f32(inputs.Sample(L=L, J=np.zeros((L ** 3, 3)), H=H, temps=1.0 / np.array([11.0, 10.0, 9.0, 8.0])))
    ctx = hsg.Context([smp], 2, 31)
    orc = oracle.OracleSim([smp], 2, 31)
    dev = []
    for _ in range(3):
        for o, st in zip(orc.samples, ctx.get_spins()):
            o.s = st.astype(np.float64)
        ctx.sweep_hb(1)
        orc.sweep_hb(1)
        dev.append(max(np.abs(g - o).max() for g, o in zip(ctx.get_spins(), orc.spins())))
    ctx.close()
    print(f"\n[strong field] max |GPU - oracle| per heat-bath sweep: {np.array2string(np.array(dev), precision=2)}")
    assert max(dev) < 2e-6, dev


def test_ragged_system_count_and_batch():
    """W = 3 (padded to 8 lanes) and a batch of three lattice sizes in one context."""
    samples = [inputs.small_sample(L, n_temps=3, h_r=0.1, disorder_seed=10 + L) for L in (4, 6, 8)]
    for op in ("sweep_hb", "sweep_or"):
        d = one_sweep_from_seeded_state(samples, 1, 3, op, pre_sweeps=1)
        assert d.max() < TOL_FP32, (op, d.max())
    trajectory_check(samples, 1, 3, [("sweep_hb", 2), ("sweep_or", 2)])


def test_energies_match_oracle_on_seeded_state():
    rng = np.random.default_rng(1)
    smp = inputs.small_sample(8, n_temps=4, h_r=0.3)
    ctx = hsg.Context([smp], 2, 1)
    s = seeded_state(rng, 8, 512)
    ctx.set_spins([s])
    E = ctx.energies()[0]
    E_ref = oracle.energy(s.astype(np.float64), smp.J.astype(np.float32).astype(np.float64),
                          smp.H.astype(np.float32).astype(np.float64), 8)
    np.testing.assert_allclose(E, E_ref, rtol=2e-6, atol=1e-4)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16", "oct16"])
def test_step_energies_equal_recomputed(precision):
    """The energies the step's PT pass used (summed from the partials of the
    last OR sweep) equal a fresh FP64 energy evaluation of the same state."""
    samples = [inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L) for L in (6, 8)]
    ctx = hsg.Context(samples, 2, 4, precision=precision, j_fp16=precision != "fp32")
    for _ in range(3):
        ctx.step(1)
        E_step = ctx.last_energies()
        E_new = ctx.energies()
        np.testing.assert_allclose(E_step, E_new, rtol=1e-6, atol=1e-6)
    ctx.close()


def test_pt_with_injected_energies_bit_exact():
    rng = np.random.default_rng(2)
    samples = [inputs.small_sample(4, n_temps=8, disorder_seed=k) for k in range(3)]
    ctx = hsg.Context(samples, 2, 9)
    orc = oracle.OracleSim(samples, 2, 9)
    for call in range(20):
        E = [rng.normal(0, 3, 16) for _ in samples]
        ctx.pt_exchange_energies(np.stack(E))
        orc.pt_exchange(E)
        perm = ctx.get_perm()
        for s, o in enumerate(orc.samples):
            np.testing.assert_array_equal(perm[s], o.perm)
    acc, n = ctx.pt_stats()
    assert n == 20 and acc.sum() > 0
    moved, tunnel, passes = ctx.pt_diagnostics()
    assert passes == 20
    for s, o in enumerate(orc.samples):
        np.testing.assert_array_equal(moved[s], o.moved)
        np.testing.assert_array_equal(tunnel[s], o.tunnel)
    ctx.close()


def test_pt_diagnostics_hand_worked_gpu():
    """tests/golden/pt_tunnelling.txt on the device: four forced passes with the
    energies injected; permutations, moved counts and the tunnelling loop agree
    with the hand-worked values."""
    import os
    g = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "pt_tunnelling.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                g[k] = np.array([float(x) for x in v])
    smp = inputs.Sample(L=4, J=np.zeros((64, 3)), H=None, temps=g["temps"])
    ctx = hsg.Context([smp], 1, 5)
    for k in range(4):
        ctx.pt_exchange_energies(g[f"energies_{k}"][None, :])
        np.testing.assert_array_equal(ctx.get_perm()[0, 0], g[f"perm_{k}"])
    moved, tunnel, passes = ctx.pt_diagnostics()
    assert passes == 4
    np.testing.assert_array_equal(moved[0, 0], g["moved"])
    np.testing.assert_array_equal(tunnel[0, 0], g["tunnel"])
    ctx.close()


@pytest.mark.parametrize("variant", [hsg.VARIANT_TWO_PASS, hsg.VARIANT_PERSISTENT])
def test_checkpoint_resume_is_bit_identical(variant):
    """Steps, checkpoint, more steps; a fresh context restored from the
    checkpoint (with the other schedule) and run for the same steps ends in the
    identical state: spins, energies, permutations, counters, PT statistics and
    diagnostics."""
    samples = [inputs.small_sample(L, n_temps=6, h_r=0.2, disorder_seed=L) for L in (4, 8)]
    other = hsg.VARIANT_PERSISTENT if variant == hsg.VARIANT_TWO_PASS else hsg.VARIANT_TWO_PASS

    def state(c):
        return ([x.copy() for x in c.get_spins()], c.last_energies(), c.get_perm(), c.pt_stats()[0],
                c.pt_diagnostics(), c.info().sweep_count, c.info().pt_count)

    a = hsg.Context(samples, 2, 4, precision="fp16", j_fp16=True, variant=variant)
    a.step(3)
    blob = a.checkpoint()
    a.step(2)
    ref = state(a)
    a.close()
    b = hsg.Context(samples, 2, 4, precision="fp16", j_fp16=True, variant=other)
    b.step(1)                       # a different state, overwritten by the restore
    b.restore(blob)
    b.step(2)
    got = state(b)
    b.close()
    for x, y in zip(ref[0], got[0]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(ref[1], got[1])
    np.testing.assert_array_equal(ref[2], got[2])
    np.testing.assert_array_equal(ref[3], got[3])
    for x, y in zip(ref[4], got[4]):
        np.testing.assert_array_equal(x, y)
    assert ref[5:] == got[5:] == (30, 5)


def test_checkpoint_into_caller_buffer_equals_bytes_blob():
    """checkpoint(out=uint8 array) writes the same blob as checkpoint() (the
    bench's end-to-end leg uploads it from pinned memory), and restore() of the
    array continues the chain exactly as restore() of the bytes."""
    smp = inputs.small_sample(8, n_temps=4, h_r=0.1, disorder_seed=9)
    a = hsg.Context([smp], 2, 6, precision="fp16", j_fp16=True)
    a.step(2)
    blob = a.checkpoint()
    arr = np.zeros(a.checkpoint_size() + 16, dtype=np.uint8)
    assert a.checkpoint(out=arr) is arr
    assert bytes(arr[:len(blob)]) == blob
    a.step(2)
    ref = [x.copy() for x in a.get_spins()]
    a.restore(arr)
    a.step(2)
    for x, y in zip(ref, a.get_spins()):
        np.testing.assert_array_equal(x, y)
    a.close()


def test_checkpoint_rejects_other_contexts():
    smp = inputs.small_sample(6, n_temps=4, disorder_seed=1)
    a = hsg.Context([smp], 2, 3)
    a.step(1)
    blob = a.checkpoint()
    perm = a.get_perm()
    for make in (lambda: hsg.Context([smp], 2, 4),                                   # seed
                 lambda: hsg.Context([inputs.small_sample(6, n_temps=4, disorder_seed=2)], 2, 3),
                 lambda: hsg.Context([smp], 2, 3, precision="fp16")):
        c = make()
        with pytest.raises(hsg.HsgError) as ei:
            c.restore(blob)
        assert ei.value.status == 1
        c.close()
    for bad in (blob[:100], b"x" * len(blob), blob[:-8]):
        with pytest.raises(hsg.HsgError):
            a.restore(bad)
    np.testing.assert_array_equal(a.get_perm(), perm)     # untouched by the failed loads
    a.restore(blob)
    a.close()


def test_step_with_pt_matches_oracle():
    """hsg_step (graph: HB, 5 OR, energies, PT) against the oracle's step: the
    permutations agree exactly for three steps; the spins after the first step
    (6 sweeps, before the dynamics have amplified rounding to O(1)) lie within
    the FP32 spread."""
    w = inputs.workload("L8_plain")
    samples = [f32(x) for x in w.samples]
    ctx = hsg.Context(samples, 2, 1)
    orc = oracle.OracleSim(samples, 2, 1)
    for k in range(3):
        ctx.step(1)
        orc.step(1)
        np.testing.assert_array_equal(ctx.get_perm()[0], orc.samples[0].perm)
        if k == 0:
            d = np.abs(ctx.get_spins()[0] - orc.spins()[0]).ravel()
            assert_within_fp32_spread(d, fp32_storage_reference(samples, 2, 1, [("step", 1)]))
    info = ctx.info()
    assert info.sweep_count == 18 and info.pt_count == 3
    ctx.close()


def test_measure_matches_oracle_on_seeded_state():
    rng = np.random.default_rng(3)
    smp = inputs.small_sample(8, n_temps=5)
    ctx = hsg.Context([smp], 2, 1)
    s = seeded_state(rng, 10, 512)
    ctx.set_spins([s])
    perm = np.array([[3, 1, 4, 0, 2], [2, 0, 1, 4, 3]], dtype=np.int32)
    # drive the GPU to this permutation with injected energies is awkward; measure at identity
    m = ctx.measure()
    ident = np.tile(np.arange(5, dtype=np.int32), (2, 1))
    o = oracle.OracleSample(8, smp.J, smp.H, smp.temps, 2, 0, 0, 1, 0)
    o.s = s.astype(np.float64)
    o.perm = ident
    mo = o.measure()
    np.testing.assert_allclose(m["q"][0], mo["q"], atol=1e-6)
    np.testing.assert_allclose(m["qk"][0], mo["qk"], atol=1e-6)
    assert perm.shape == (2, 5)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp16", "bf16", "angle16", "oct16", "yx4"])
def test_codec_roundtrip_matches_oracle(precision):
    rng = np.random.default_rng(4)
    smp = inputs.small_sample(6, n_temps=4)
    ctx = hsg.Context([smp], 2, 1, precision=precision)
    s = seeded_state(rng, 8, 216)
    ctx.set_spins([s])
    g = ctx.get_spins()[0]
    o = oracle.codec_roundtrip(s.astype(np.float64).reshape(-1, 3), precision).reshape(s.shape)
    # one quantum where FP32 and FP64 rounding sit on different sides of a boundary
    assert np.abs(g - o).max() <= QUANT[precision] * 1.01
    assert np.mean(np.abs(g - o) > 1e-6) < 0.02
    ctx.close()


@pytest.mark.parametrize("precision", ["fp16", "bf16", "angle16", "oct16"])
@pytest.mark.parametrize("op", ["sweep_or", "sweep_hb"])
def test_codec_one_sweep_matches_oracle(precision, op):
    """One sweep from the same seeded state with compressed spins and FP16
    couplings; the oracle applies the same storage rounding in FP64."""
    smp = inputs.small_sample(8, n_temps=4, h_r=0.2)
    smp16 = inputs.Sample(L=8, J=inputs.round_fp16(smp.J), H=inputs.round_fp16(smp.H),
                          temps=smp.temps)
    d = one_sweep_from_seeded_state([smp16], 2, 2, op, precision=precision, codec=precision,
                                    j16=True, pre_sweeps=1)
    # equal up to one storage quantum; a site whose field is small amplifies it
    assert np.quantile(d, 0.99) < 3 * QUANT[precision], (op, np.quantile(d, 0.99))
    assert np.median(d) < QUANT[precision] and d.max() < 0.05, (op, d.max())


def yx4_ulp_spread(o, base, parity_of_site, op, rng):
    """The format's own sensitivity: the oracle's even half-sweep, then the odd
    half-sweep once as is and once with every even site's stored s_x + 4 moved by
    one unit in the last place; returns the odd sites' differences (x, y)."""
    out = []
    for perturb in (False, True):
        o.s = base.copy()
        o.or_half(0) if op == "sweep_or" else o.hb_half(0, 1)
        if perturb:
            ev = parity_of_site == 0
            for w in range(o.W):
                sx, sy, sz = o.s[w, ev, 0], o.s[w, ev, 1], o.s[w, ev, 2]
                sg = np.where(sz >= 0, 1.0, -1.0)
                p = (sx + 4 * sg).astype(np.float32)
                up = rng.random(p.size) < 0.5
                p2 = np.nextafter(p, np.where(up, np.float32(10), np.float32(-10))).astype(np.float64)
                x2 = p2 - 4 * sg
                o.s[w, ev, 0] = x2
                o.s[w, ev, 2] = sg * np.sqrt(np.maximum(0.0, 1 - x2 * x2 - sy * sy))
        o.or_half(1) if op == "sweep_or" else o.hb_half(1, 1)
        out.append(o.s.copy())
    return np.abs(out[0] - out[1])[:, parity_of_site == 1, :2].ravel()


@pytest.mark.parametrize("op", ["sweep_or", "sweep_hb"])
def test_yx4_one_sweep_matches_oracle(op):
    """One sweep with the paper's packing (binary32 s_y and s_x + 4 sign s_z) from
    the same seeded state, the oracle applying the same storage in FP64.  The
    format stores s_x, s_y and the sign of s_z; s_z is derived, and one unit in
    the last place of the stored s_x + 4 moves s_z by up to 2^-21 |s_x| / |s_z|.
    Even sites come out of the even half-sweep from identical inputs: s_x and s_y
    within 1e-5, s_z^2 within 2e-5, the sign of s_z wherever |s_z| > 1e-3.  Odd
    sites see their even neighbours through that amplification: their
    differences stay within 4x the spread the oracle itself shows when the even
    sites' stored words move by one unit in the last place."""
    smp = inputs.small_sample(8, n_temps=4, h_r=0.2, disorder_seed=3)
    samples = [f32(smp)]
    rng = np.random.default_rng(21)
    states = [seeded_state(rng, 8, 512)]
    ctx = hsg.Context(samples, 2, 21, precision="yx4")
    orc = oracle.OracleSim(samples, 2, 21, codec="yx4")
    ctx.sweep_or(1)
    orc.sweep_or(1)
    ctx.set_spins(states)
    base = oracle.codec_roundtrip(states[0].astype(np.float64).reshape(-1, 3),
                                  "yx4").reshape(states[0].shape)
    orc.samples[0].s = base.copy()
    getattr(ctx, op)(1)
    getattr(orc, op)(1)
    g = ctx.get_spins()[0].astype(np.float64)
    o = orc.spins()[0]
    ctx.close()
    i = np.arange(512)
    par = (i % 8 + (i // 8) % 8 + i // 64) & 1
    ev, od = par == 0, par == 1
    assert np.abs(g[:, ev, :2] - o[:, ev, :2]).max() < 1e-5
    assert np.abs(g[:, ev, 2] ** 2 - o[:, ev, 2] ** 2).max() < 2e-5
    far = np.abs(o[:, ev, 2]) > 1e-3
    np.testing.assert_array_equal(np.sign(g[:, ev, 2][far]), np.sign(o[:, ev, 2][far]))
    d = np.abs(g[:, od, :2] - o[:, od, :2]).ravel()
    ref = yx4_ulp_spread(orc.samples[0], base, par, op, np.random.default_rng(5))
    for q in (0.5, 0.9, 0.99, 1.0):
        assert np.quantile(d, q) <= 4 * np.quantile(ref, q) + 1e-6, (q, np.quantile(d, q),
                                                                    np.quantile(ref, q))


def test_or_conserves_energy_gpu():
    smp = inputs.small_sample(16, n_temps=4, h_r=0.3)
    ctx = hsg.Context([smp], 2, 4)
    ctx.sweep_hb(2)
    E0 = ctx.energies()[0]
    ctx.sweep_or(200)
    E1 = ctx.energies()[0]
    # FP32 rounding only: a random walk of ~1e-7 relative per update
    assert np.max(np.abs(E1 - E0) / np.abs(E0)) < 1e-4
    s = ctx.get_spins()[0]
    assert np.abs(np.linalg.norm(s, axis=2) - 1).max() < 1e-6
    ctx.close()


def test_runs_are_bit_reproducible():
    w = inputs.workload("L8_plain")
    out = []
    for _ in range(2):
        ctx = hsg.Context(w.samples, 2, 1)
        ctx.step(5)
        out.append((ctx.get_spins()[0].copy(), ctx.energies()[0].copy(), ctx.get_perm().copy()))
        ctx.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_invalid_arguments_rejected():
    smp = inputs.small_sample(8, n_temps=4)
    bad = inputs.Sample(L=8, J=smp.J.copy(), H=smp.H, temps=smp.temps[::-1].copy())
    with pytest.raises(hsg.HsgError):
        hsg.Context([bad], 2, 1)
    J = smp.J.copy()
    J[3, 1] = np.nan
    with pytest.raises(hsg.HsgError):
        hsg.Context([inputs.Sample(L=8, J=J, H=smp.H, temps=smp.temps)], 2, 1)
    for kw in ({"pass_bytes": -1}, {"chunks_per_thread": -2}, {"variant": 3}, {"variant": -1}):
        with pytest.raises(hsg.HsgError) as ei:
            hsg.Context([smp], 2, 1, **kw)
        assert ei.value.status == 1
    # more samples than a grid dimension holds: rejected before any argument is read
    import ctypes
    out = ctypes.c_void_p()
    for n in (0, 65536):
        assert hsg.lib().hsg_create_batch(ctypes.byref(out), n, None, None, 4, 2, None, None,
                                          ctypes.c_uint64(1), None) == 1
        assert out.value is None
    ctx = hsg.Context([smp], 2, 1)
    with pytest.raises(hsg.HsgError):
        ctx.sweep_or(-1)
    ctx.sweep_or(1)       # an argument error is not sticky
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16", "angle16", "oct16", "yx4"])
def test_persistent_schedule_bit_identical(precision):
    """The persistent step kernel (one cooperative launch, grid barriers) runs
    the same arithmetic as the per-phase graph: identical spins, energies and
    permutations, here for a batch of three lattice sizes.  For the packed
    formats the graph decodes each neighbour parity once into binary32 before
    a half-sweep while the persistent kernel decodes at every use, so this also
    checks that the two give the same values."""
    samples = [inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L) for L in (4, 8, 12)]
    out = {}
    for variant in (hsg.VARIANT_TWO_PASS, hsg.VARIANT_PERSISTENT):
        ctx = hsg.Context(samples, 2, 6, precision=precision, j_fp16=precision != "fp32",
                          variant=variant)
        assert ctx.info().variant == variant
        ctx.step(2)
        ctx.step(3)
        out[variant] = ([s.copy() for s in ctx.get_spins()], ctx.last_energies(), ctx.get_perm(),
                        ctx.info().sweep_count, ctx.info().pt_count)
        ctx.close()
    a, b = out[hsg.VARIANT_TWO_PASS], out[hsg.VARIANT_PERSISTENT]
    for x, y in zip(a[0], b[0]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    assert a[3] == b[3] == 30 and a[4] == b[4] == 5


@pytest.mark.parametrize("variant,precision", [(hsg.VARIANT_TWO_PASS, "fp16"), (hsg.VARIANT_PERSISTENT, "fp16"),
                                               (hsg.VARIANT_TWO_PASS, "oct16")])
@pytest.mark.parametrize("pass_bytes", [1, 40000])
def test_system_blocked_passes_bit_identical(variant, precision, pass_bytes):
    """Sweeping the systems pass by pass (each pass a range of 4-system chunks
    swept through the whole step before the next) computes the same step as one
    pass: systems are independent and the random numbers are keyed by site,
    system and sweep.  pass_bytes = 1 makes every chunk its own pass; 40000
    groups chunks, and samples, up to that footprint."""
    samples = [inputs.small_sample(L, n_temps=8, h_r=0.2, disorder_seed=L) for L in (4, 8, 12)]
    out = []
    for pb in (0, pass_bytes):
        ctx = hsg.Context(samples, 2, 6, precision=precision, j_fp16=True, variant=variant,
                          pass_bytes=pb)
        info = ctx.info()
        assert info.pass_bytes == pb
        if pb == 0:
            assert info.n_passes == 1
        elif pb == 1:
            assert info.n_passes == 3 * (info.Wp // 4) // info.chunks_per_thread
        else:
            assert 1 < info.n_passes < 3 * (info.Wp // 4)
        ctx.step(2)
        ctx.step(1)
        out.append(([s.copy() for s in ctx.get_spins()], ctx.last_energies(), ctx.get_perm(),
                    ctx.info().sweep_count))
        ctx.close()
    for x, y in zip(out[0][0], out[1][0]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])
    assert out[0][3] == out[1][3] == 18


def test_persistent_barrier_timeout_is_reported():
    """A block that never arrives at a grid barrier: the other blocks' bounded
    waits run out, the launch ends, and the host gets HSG_ETIMEOUT; the device
    stays usable for a new context."""
    smp = inputs.small_sample(8, n_temps=4)
    ctx = hsg.Context([smp], 2, 1, variant=hsg.VARIANT_PERSISTENT, barrier_timeout_ms=200,
                      inject_barrier_fault=True)
    ctx.step(1)
    with pytest.raises(hsg.HsgError) as ei:
        ctx.sync()
    assert ei.value.status == 4
    with pytest.raises(hsg.HsgError):          # sticky
        ctx.step(1)
    ctx.close()
    ctx = hsg.Context([smp], 2, 1, variant=hsg.VARIANT_PERSISTENT)
    ctx.step(2)
    ctx.sync()
    assert ctx.info().pt_count == 2
    ctx.close()


def test_autotuned_schedule_matches_fixed_schedule():
    """The automatic schedule times the candidates on the live context at the
    first step and restores the state: the trajectory equals the one of a
    fixed two-pass context bit for bit."""
    samples = [inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L) for L in (6, 10)]
    runs = []
    for variant in (hsg.VARIANT_AUTO, hsg.VARIANT_TWO_PASS):
        ctx = hsg.Context(samples, 2, 8, precision="fp16", j_fp16=True, variant=variant)
        ctx.sweep_hb(1)
        ctx.step(3)
        info = ctx.info()
        assert info.variant in (hsg.VARIANT_TWO_PASS, hsg.VARIANT_PERSISTENT)
        assert 1 <= info.chunks_per_thread <= info.Wp // 4
        assert info.sweep_count == 19 and info.pt_count == 3
        runs.append(([s.copy() for s in ctx.get_spins()], ctx.get_perm(), ctx.last_energies()))
        ctx.close()
    for x, y in zip(runs[0][0], runs[1][0]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


@pytest.mark.parametrize("variant", [hsg.VARIANT_TWO_PASS, hsg.VARIANT_PERSISTENT])
def test_per_sample_run_lengths(variant):
    """Samples frozen in turn: after sample 0 runs 1 + 2 steps and sample 1 runs
    3 steps (interleaved), the batch is bit-identical to one where both ran 3
    steps together (each sample's counters key its random numbers)."""
    samples = [inputs.small_sample(L, n_temps=6, h_r=0.1, disorder_seed=L) for L in (6, 8)]

    def state(c):
        sw, pt = c.counters()
        return ([x.copy() for x in c.get_spins()], c.last_energies(), c.get_perm(), c.pt_stats()[0],
                c.pt_diagnostics()[:2], list(sw), list(pt))

    a = hsg.Context(samples, 2, 5, variant=variant)
    a.step(3)
    ref = state(a)
    a.close()
    b = hsg.Context(samples, 2, 5, variant=variant)
    b.set_active([1, 0])
    b.step(1)
    b.set_active([0, 1])
    b.step(3)
    b.set_active([1, 0])
    b.step(2)
    got = state(b)
    b.close()
    for x, y in zip(ref[0], got[0]):
        np.testing.assert_array_equal(x, y)
    for k in (1, 2, 3):
        np.testing.assert_array_equal(ref[k], got[k])
    for x, y in zip(ref[4], got[4]):
        np.testing.assert_array_equal(x, y)
    assert ref[5] == got[5] == [18, 18] and ref[6] == got[6] == [3, 3]


def test_frozen_samples_follow_the_oracle():
    """Masks applied to sweeps, PT passes and steps on the device and in the
    oracle: permutations equal at every step, frozen samples untouched."""
    samples = [f32(inputs.small_sample(L, n_temps=5, disorder_seed=L + 1)) for L in (4, 6, 4)]
    ctx = hsg.Context(samples, 2, 3)
    orc = oracle.OracleSim(samples, 2, 3)
    for mask in ([1, 0, 1], [0, 1, 1], [1, 1, 0], [0, 0, 1]):
        before = [x.copy() for x in ctx.get_spins()]
        ctx.set_active(mask)
        orc.set_active(mask)
        ctx.step(1)
        orc.step(1)
        perm = ctx.get_perm()
        spins = ctx.get_spins()
        for s, o in enumerate(orc.samples):
            np.testing.assert_array_equal(perm[s], o.perm)
            if not mask[s]:
                np.testing.assert_array_equal(spins[s], before[s])
    sw, pt = ctx.counters()
    assert list(pt) == [o.pt_step for o in orc.samples] == [2, 2, 3]
    assert list(sw) == [o.sweep for o in orc.samples]
    ctx.set_active(None)
    ctx.sweep_or(1)
    assert list(ctx.counters()[0]) == [x + 1 for x in sw]
    ctx.close()


@pytest.mark.parametrize("n_hb,n_or", [(1, 10), (1, 100), (2, 0), (0, 3)])
def test_step_ratios_of_table1_match_oracle(n_hb, n_or):
    """Steps with other heat-bath / over-relaxation ratios (Table 1 uses 1 HB +
    10 OR and 1 HB + 100 OR; with no OR sweep the step takes its energies from
    the standalone energy kernel): the PT permutations follow the oracle's step
    exactly and the step's energies equal a fresh FP64 evaluation."""
    smp = f32(inputs.small_sample(6, n_temps=5, h_r=0.1, disorder_seed=9))
    ctx = hsg.Context([smp], 2, 13, n_hb=n_hb, n_or=n_or)
    orc = oracle.OracleSim([smp], 2, 13)
    for _ in range(2):
        ctx.step(1)
        orc.step(1, n_hb=n_hb, n_or=n_or)
        np.testing.assert_array_equal(ctx.get_perm()[0], orc.samples[0].perm)
    np.testing.assert_allclose(ctx.last_energies(), ctx.energies(), rtol=1e-9)
    sw, pt = ctx.counters()
    assert list(sw) == [2 * (n_hb + n_or)] and list(pt) == [2]
    ctx.close()
