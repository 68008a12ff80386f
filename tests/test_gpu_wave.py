"""The wave over-relaxation sweep (both half-sweeps in one launch, odd blocks
trailing the even blocks of their planes) and the staged block body (neighbour
rows through a shared-memory ring) against the per-half-sweep kernel and the
FP64 oracle.

The wave launch runs the per-half-sweep kernel's device body on the same
blocks; an odd block starts only after every even block of the planes it reads
has finished.  So it must reproduce two per-half-sweep launches bit for bit, in
every format it serves, for every lag (1: odd blocks right behind their even
blocks, so nearly every odd block waits; a lag beyond the table: all even
blocks first), for blocks that span several planes (small L) or a part of one
(large L), for several chunk groups per sample, for passes, mixed batches and
frozen samples, and inside hsg_step with its energy sums and PT pass.
"""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu

FORMATS = [("fp32", False), ("fp16", True), ("fp16", False), ("bf16", True)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def seeded_state(rng, W, N):
    s = rng.standard_normal((W, N, 3))
    return (s / np.linalg.norm(s, axis=2, keepdims=True)).astype(np.float32)


def run(samples, n_rep, seed, kernel, precision="fp32", j16=False, states=None, active=None,
        n_sweeps=3, steps=0, **kw):
    ctx = hsg.Context(samples, n_rep, seed, precision=precision, j_fp16=j16,
                      variant=hsg.VARIANT_TWO_PASS, sweep_kernel=kernel, **kw)
    info = ctx.info()
    assert info.sweep_kernel == kernel, (kernel, info.sweep_kernel)
    if states is not None:
        ctx.set_spins(states)
    if active is not None:
        ctx.set_active(active)
    ctx.sweep_or(n_sweeps)
    out = {"spins": ctx.get_spins(), "lag": info.wave_lag, "staged": info.staged,
           "passes": info.n_passes}
    if steps:
        ctx.step(steps)
        m = ctx.measure()
        out.update(after=ctx.get_spins(), E=m["E"], perm=m["perm"])
    ctx.close()
    return out


def assert_same(a, b):
    for x, y in zip(a["spins"], b["spins"]):
        np.testing.assert_array_equal(x, y)
    if "after" in a:
        for x, y in zip(a["after"], b["after"]):
            np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(a["E"], b["E"])
        np.testing.assert_array_equal(a["perm"], b["perm"])


@pytest.mark.parametrize("precision,j16", FORMATS)
@pytest.mark.parametrize("L", [4, 6, 8, 16, 32])
def test_wave_equals_half_sweeps_bit_for_bit(L, precision, j16):
    smp = inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L, t_min=0.15, t_max=0.6)
    st = [seeded_state(np.random.default_rng(L), 8, L ** 3)]
    a = run([smp], 2, 5, hsg.SWEEP_HALF, precision, j16, states=st)
    b = run([smp], 2, 5, hsg.SWEEP_WAVE, precision, j16, states=st)
    assert b["lag"] > 0
    assert_same(a, b)


@pytest.mark.parametrize("lag", [1, 7, 1 << 20])
@pytest.mark.parametrize("gpt", [1, 3])
def test_wave_lags_and_chunk_groups_l48(lag, gpt):
    """L = 48, W = 48 (12 chunk groups): a block covers 256 of a plane's 1152
    sites of one parity, so planes span several blocks and blocks straddle
    planes; gpt 1 and 3 give 12 and 4 chunk-group columns per sample."""
    smp = inputs.small_sample(48, n_temps=24, h_r=0.1, disorder_seed=48, t_min=0.08, t_max=0.3)
    a = run([smp], 2, 7, hsg.SWEEP_HALF, "fp16", True, chunks_per_thread=gpt)
    b = run([smp], 2, 7, hsg.SWEEP_WAVE, "fp16", True, chunks_per_thread=gpt, wave_lag=lag)
    assert b["lag"] == lag
    assert_same(a, b)


@pytest.mark.parametrize("precision,j16", FORMATS)
@pytest.mark.parametrize("kernel", [hsg.SWEEP_STAGED, hsg.SWEEP_WAVE])
def test_staged_equals_half_sweeps_l64(kernel, precision, j16):
    """L = 64 (8 rows per block): the staged block body, in two half-sweep
    launches and in the wave launch, against the per-half-sweep kernel."""
    smp = inputs.small_sample(64, n_temps=6, h_r=0.1, disorder_seed=64, t_min=0.1, t_max=0.4)
    st = [seeded_state(np.random.default_rng(64), 12, 64 ** 3)]
    a = run([smp], 2, 9, hsg.SWEEP_HALF, precision, j16, states=st, n_sweeps=2)
    b = run([smp], 2, 9, kernel, precision, j16, states=st, n_sweeps=2)
    assert b["staged"] == 1
    assert_same(a, b)


@pytest.mark.parametrize("kernel", [hsg.SWEEP_STAGED, hsg.SWEEP_WAVE])
def test_staged_ragged_chunk_groups(kernel):
    """L = 64, 48 systems (12 chunk groups) at 5 chunk groups per thread: blocks
    of 5, 5 and 2 groups, the last shorter than the two-stage ring's depth."""
    smp = inputs.small_sample(64, n_temps=24, h_r=0.1, disorder_seed=65, t_min=0.08, t_max=0.3)
    a = run([smp], 2, 3, hsg.SWEEP_HALF, "fp16", True, n_sweeps=2, steps=1, chunks_per_thread=5)
    b = run([smp], 2, 3, kernel, "fp16", True, n_sweeps=2, steps=1, chunks_per_thread=5)
    assert b["staged"] == 1
    assert_same(a, b)


@pytest.mark.parametrize("kernel", [hsg.SWEEP_STAGED, hsg.SWEEP_WAVE])
def test_staged_l256_two_rows_per_block(kernel):
    """L = 256 (16.8M sites, 2 rows of 128 sites per block), 2 x 4 systems,
    FP16 spins and couplings: two OR sweeps and a step against the per-half-sweep
    kernel, bit for bit."""
    smp = inputs.small_sample(256, n_temps=4, h_r=0.1, disorder_seed=256, t_min=0.1, t_max=0.4)
    a = run([smp], 2, 5, hsg.SWEEP_HALF, "fp16", True, n_sweeps=2, steps=1)
    b = run([smp], 2, 5, kernel, "fp16", True, n_sweeps=2, steps=1)
    assert b["staged"] == 1
    assert_same(a, b)


@pytest.mark.parametrize("lag", [1, 100, 1 << 20])
def test_staged_wave_lags_and_mixed_batch(lag):
    """A batch of L = 32, 64, 32 (16 and 8 rows per block, stage size of the
    largest) with 2 chunk groups per thread, cut into passes; one sample frozen."""
    samples = [inputs.small_sample(L, n_temps=8, h_r=0.1, disorder_seed=40 + k)
               for k, L in enumerate((32, 64, 32))]
    kw = dict(chunks_per_thread=2, pass_bytes=8 << 20)
    a = run(samples, 2, 13, hsg.SWEEP_HALF, "fp16", True, active=[1, 1, 0], steps=2, **kw)
    b = run(samples, 2, 13, hsg.SWEEP_WAVE, "fp16", True, active=[1, 1, 0], steps=2, wave_lag=lag,
            **kw)
    c = run(samples, 2, 13, hsg.SWEEP_STAGED, "fp16", True, active=[1, 1, 0], steps=2, **kw)
    assert b["staged"] == 1 and b["lag"] == lag and b["passes"] > 1
    assert_same(a, b)
    assert_same(a, c)


def test_wave_passes_mixed_batch_and_frozen_sample():
    """A batch of L = 8, 12, 16, 24 cut into passes of a few chunk groups each,
    with one sample frozen: the frozen sample keeps its spins, the others match."""
    samples = [inputs.small_sample(L, n_temps=5, h_r=0.1, disorder_seed=20 + L) for L in (8, 12, 16, 24)]
    kw = dict(pass_bytes=1 << 20, chunks_per_thread=1)
    ref = hsg.Context(samples, 2, 3, variant=hsg.VARIANT_TWO_PASS, **kw)
    before = ref.get_spins()
    assert ref.info().n_passes > 1
    ref.close()
    a = run(samples, 2, 3, hsg.SWEEP_HALF, active=[1, 0, 1, 1], **kw)
    b = run(samples, 2, 3, hsg.SWEEP_WAVE, active=[1, 0, 1, 1], **kw)
    np.testing.assert_array_equal(b["spins"][1], before[1])
    assert_same(a, b)


@pytest.mark.parametrize("precision,j16", [("fp32", False), ("fp16", True)])
def test_wave_in_steps_energies_and_pt(precision, j16):
    """hsg_step with the wave sweeps in its graph (the last one also leaves the
    energy partials): spins, FP64 energies and permutations identical."""
    smp = inputs.small_sample(16, n_temps=6, h_r=0.1, disorder_seed=3, t_min=0.15, t_max=0.6)
    a = run([smp], 2, 11, hsg.SWEEP_HALF, precision, j16, steps=5)
    b = run([smp], 2, 11, hsg.SWEEP_WAVE, precision, j16, steps=5)
    assert_same(a, b)


@pytest.mark.parametrize("L", [8, 16])
def test_wave_sweep_against_oracle(L):
    """One wave sweep from a seeded binary32 state (after three sweeps on both
    sides, so the state is not the initial one) against the FP64 oracle from
    the same state: every component within 1e-5."""
    from test_gpu_parity import TOL_FP32, f32
    smp = f32(inputs.small_sample(L, n_temps=4, h_r=0.2, disorder_seed=L, t_min=0.15, t_max=0.6))
    st = [seeded_state(np.random.default_rng(L + 1), 8, L ** 3)]
    ctx = hsg.Context([smp], 2, 7, variant=hsg.VARIANT_TWO_PASS, sweep_kernel=hsg.SWEEP_WAVE)
    orc = oracle.OracleSim([smp], 2, 7)
    ctx.sweep_or(3)
    orc.sweep_or(3)
    ctx.set_spins(st)
    orc.samples[0].s = st[0].astype(np.float64)
    ctx.sweep_or(1)
    orc.sweep_or(1)
    d = np.abs(ctx.get_spins()[0] - orc.spins()[0]).max()
    ctx.close()
    assert d < TOL_FP32, d


def test_wave_fullsize_bench_configuration():
    """L = 128, 2 x 24 temperatures, FP16 spins and couplings (100.7M spins),
    the lag the library picks: two OR sweeps and one hsg_step, the staged wave
    and the staged half-sweeps against the per-half-sweep kernel, spins,
    energies and permutations identical."""
    w = inputs.workload("L128_fp16")
    a = run(w.samples, w.n_replicas, w.seed, hsg.SWEEP_HALF, "fp16", True, n_sweeps=2, steps=1)
    for kernel in (hsg.SWEEP_WAVE, hsg.SWEEP_STAGED):
        b = run(w.samples, w.n_replicas, w.seed, kernel, "fp16", True, n_sweeps=2, steps=1)
        assert b["staged"] == 1
        assert_same(a, b)


def test_wave_wait_timeout_is_reported():
    """One odd block of a wave launch waits (host-requested fault) for a
    completion flag that no block sets: its bounded wait runs out, the launch
    ends, the host gets HSG_ETIMEOUT (sticky), and the device stays usable for
    a new context."""
    smp = inputs.small_sample(16, n_temps=4, h_r=0.1, disorder_seed=16)
    ctx = hsg.Context([smp], 2, 1, variant=hsg.VARIANT_TWO_PASS, sweep_kernel=hsg.SWEEP_WAVE,
                      barrier_timeout_ms=200, inject_barrier_fault=True)
    ctx.sweep_or(1)
    with pytest.raises(hsg.HsgError) as ei:
        ctx.sync()
    assert ei.value.status == 4
    with pytest.raises(hsg.HsgError):          # sticky
        ctx.sweep_or(1)
    ctx.close()
    a = run([smp], 2, 1, hsg.SWEEP_HALF, n_sweeps=2)
    b = run([smp], 2, 1, hsg.SWEEP_WAVE, n_sweeps=2)
    assert_same(a, b)
