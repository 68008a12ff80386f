"""The fused over-relaxation sweep (both half-sweeps in one launch, a z
wavefront through shared memory) against the per-half-sweep kernel and the
FP64 oracle.

Both kernels apply the same arithmetic in the same order to the same inputs
(an even site sees only old odd spins, an odd site only new even spins), so
the fused sweep must reproduce the per-half-sweep sweep bit for bit, in every
storage format, whether a block holds whole planes (small L) or bands of rows
with recomputed halo rows (large L), and whatever the z segments of its work
items.  Against the oracle the FP32 form holds 1e-5 per component per sweep.
"""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu

FORMATS = [("fp32", False), ("fp16", True), ("fp16", False), ("bf16", True), ("angle16", True),
           ("oct16", True)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def seeded_state(rng, W, N):
    s = rng.standard_normal((W, N, 3))
    return (s / np.linalg.norm(s, axis=2, keepdims=True)).astype(np.float32)


def pair(samples, n_rep, seed, precision, j16, n_sweeps=2, states=None, active=None):
    """The spins after n_sweeps OR sweeps with each kernel, from the same state."""
    out = []
    for kernel in (hsg.SWEEP_HALF, hsg.SWEEP_FUSED):
        ctx = hsg.Context(samples, n_rep, seed, precision=precision, j_fp16=j16,
                          variant=hsg.VARIANT_TWO_PASS, sweep_kernel=kernel)
        info = ctx.info()
        assert info.sweep_kernel == kernel, (kernel, info.sweep_kernel)
        if states is not None:
            ctx.set_spins(states)
        if active is not None:
            ctx.set_active(active)
        ctx.sweep_or(n_sweeps)
        out.append(ctx.get_spins())
        if kernel == hsg.SWEEP_FUSED:
            out.append((info.fused_band_rows, info.fused_items))
        ctx.close()
    return out


@pytest.mark.parametrize("precision,j16", FORMATS)
@pytest.mark.parametrize("L", [8, 16, 32])
def test_fused_equals_half_sweeps_bit_for_bit(L, precision, j16):
    smp = inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L, t_min=0.15, t_max=0.6)
    rng = np.random.default_rng(L)
    st = [seeded_state(rng, 8, L ** 3)]
    a, b, (ny, items) = pair([smp], 2, 5, precision, j16, n_sweeps=4, states=st)
    assert ny > 0 and items > 0
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision,j16", [("fp16", True), ("angle16", True), ("fp32", False)])
def test_fused_band_mode_l64(precision, j16):
    """L = 64: blocks hold bands of rows (not whole planes) with halo rows."""
    smp = inputs.small_sample(64, n_temps=4, h_r=0.1, disorder_seed=64, t_min=0.1, t_max=0.4)
    a, b, (ny, items) = pair([smp], 2, 9, precision, j16, n_sweeps=2)
    assert 0 < ny < 64, ny
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_fused_ragged_systems_and_mixed_batch():
    """W = 3 (padded to 8 systems) and a batch of L = 8, 12, 16, 24 in one context."""
    samples = [inputs.small_sample(L, n_temps=3, h_r=0.1, disorder_seed=20 + L) for L in (8, 12, 16, 24)]
    for precision, j16 in (("fp32", False), ("fp16", True)):
        a, b, _ = pair(samples, 1, 3, precision, j16, n_sweeps=2)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_fused_frozen_sample_unchanged():
    samples = [inputs.small_sample(L, n_temps=2, h_r=0.1, disorder_seed=30 + L) for L in (8, 16)]
    ref = hsg.Context(samples, 2, 4, sweep_kernel=hsg.SWEEP_FUSED, variant=hsg.VARIANT_TWO_PASS)
    before = ref.get_spins()
    ref.close()
    a, b, _ = pair(samples, 2, 4, "fp32", False, n_sweeps=2, active=[1, 0])
    np.testing.assert_array_equal(b[1], before[1])
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_fused_odd_sweep_counts_and_steps_match():
    """hsg_sweep_or(3) (one fused pair + one half-sweep sweep) and hsg_step with
    the fused pairs inside its graph: spins, energies and permutations identical."""
    smp = inputs.small_sample(16, n_temps=4, h_r=0.1, disorder_seed=3, t_min=0.15, t_max=0.6)
    res = []
    for kernel in (hsg.SWEEP_HALF, hsg.SWEEP_FUSED):
        ctx = hsg.Context([smp], 2, 11, variant=hsg.VARIANT_TWO_PASS, sweep_kernel=kernel)
        ctx.sweep_or(3)
        ctx.step(4)
        m = ctx.measure()
        res.append((ctx.get_spins(), m["E"], m["perm"]))
        ctx.close()
    (s0, e0, p0), (s1, e1, p1) = res
    for x, y in zip(s0, s1):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(e0, e1)
    np.testing.assert_array_equal(p0, p1)


def test_fused_sweeps_against_oracle_trajectory():
    """Five pairs of fused sweeps from the same state as the FP64 oracle: the
    deviation stays within the spread that binary32 storage alone gives the
    oracle (the trajectory criterion of the per-half-sweep kernel; the fused
    sweep equals that kernel bit for bit, which the tests above check)."""
    from test_gpu_parity import assert_within_fp32_spread, f32, fp32_storage_reference
    w = inputs.workload("L8_plain")
    smp = [f32(s) for s in w.samples]
    ctx = hsg.Context(smp, 2, 1, variant=hsg.VARIANT_TWO_PASS, sweep_kernel=hsg.SWEEP_FUSED)
    orc = oracle.OracleSim(smp, 2, 1)
    sched = [("sweep_or", 2)] * 5
    for op, n in sched:
        getattr(ctx, op)(n)
        getattr(orc, op)(n)
    d = np.concatenate([np.abs(g - o).ravel() for g, o in zip(ctx.get_spins(), orc.spins())])
    ctx.close()
    assert_within_fp32_spread(d, fp32_storage_reference(smp, 2, 1, sched))


def test_fused_fullsize_bench_configuration():
    """L = 128, 2 x 24 temperatures, FP16 spins and couplings (100.7M spins), in
    the launch configuration the benchmark times (band rows, items, grid chosen
    by the library): two OR sweeps and one hsg_step, fused against half-sweeps,
    spins, energies and permutations identical."""
    w = inputs.workload("L128_fp16")
    res = []
    for kernel in (hsg.SWEEP_HALF, hsg.SWEEP_FUSED):
        ctx = hsg.Context(w.samples, w.n_replicas, w.seed, precision="fp16", j_fp16=True,
                          variant=hsg.VARIANT_TWO_PASS, sweep_kernel=kernel)
        assert ctx.info().sweep_kernel == kernel
        ctx.sweep_or(2)
        s2 = ctx.get_spins()[0]
        ctx.step(1)
        m = ctx.measure()
        res.append((s2, ctx.get_spins()[0], m["E"], m["perm"]))
        ctx.close()
    for x, y in zip(res[0], res[1]):
        np.testing.assert_array_equal(x, y)
