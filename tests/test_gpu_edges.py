"""Edge cases of the GPU path against the oracle and the mathematics:
the largest system count a context takes, a vanishing local field, and a
single temperature (no PT pair)."""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_largest_system_count(precision):
    """W = n_replicas x n_temps = 4 x 256 = 1024 systems at L = 4: a step, the
    overlap tensor, the pair / chiral overlaps and the energies against the
    oracle on the same spins and couplings.  With FP16 spins the tensor runs on
    the staged kernel with 8 sites per stage; everything else here exceeds the
    staged kernels' shared memory and runs on the direct kernels."""
    raw = inputs.small_sample(4, n_temps=256, h_r=0.1, disorder_seed=21, t_min=0.2, t_max=3.0)
    rnd = inputs.round_fp16 if precision == "fp16" else (lambda a: np.asarray(a, np.float32).astype(np.float64))
    smp = inputs.Sample(L=4, J=rnd(raw.J), H=rnd(raw.H), temps=raw.temps)
    ctx = hsg.Context([smp], 4, 3, precision=precision, j_fp16=precision != "fp32")
    assert ctx.info().W == 1024
    ctx.step(2)
    spins = ctx.get_spins()[0].astype(np.float64)
    perm = ctx.get_perm()[0]
    for r in range(4):
        assert sorted(perm[r]) == list(range(256))
    m = ctx.measure()
    o = oracle.OracleSample(4, smp.J, smp.H, smp.temps, 4, 0, 0, 3, 0)
    o.s, o.perm = spins, perm.copy()
    mo = o.measure()
    np.testing.assert_allclose(m["q"][0], mo["q"], rtol=0, atol=2e-6)
    np.testing.assert_allclose(m["qk"][0], mo["qk"], rtol=0, atol=2e-6)
    ov = ctx.measure_overlaps()
    D, C = oracle.overlaps(spins, 4, 4, 256, perm)
    np.testing.assert_allclose(ov["D"][0], D, rtol=0, atol=2e-6)
    np.testing.assert_allclose(ov["C"][0], C, rtol=0, atol=2e-6)
    E = ctx.energies()[0]
    np.testing.assert_allclose(E, o.energies(), rtol=1e-6, atol=1e-6)
    ctx.close()


def test_vanishing_field():
    """J = 0 and H = 0: every local field is zero, so over-relaxation leaves
    every spin as it is (up to the renormalisation's rounding) and the heat
    bath draws uniform directions (mean ~0, second moments 1/3, at any
    temperature)."""
    L = 16
    smp = inputs.Sample(L=L, J=np.zeros((L ** 3, 3)), H=None, temps=np.array([0.1, 1.0]))
    ctx = hsg.Context([smp], 4, 5)
    before = ctx.get_spins()[0].copy()
    ctx.sweep_or(3)
    np.testing.assert_allclose(ctx.get_spins()[0], before, rtol=0, atol=4e-7)
    ctx.sweep_hb(1)
    s = ctx.get_spins()[0].reshape(-1, 3).astype(np.float64)
    n = s.shape[0]
    assert np.abs(s.mean(axis=0)).max() < 5 / np.sqrt(3 * n)
    np.testing.assert_allclose((s ** 2).mean(axis=0), 1 / 3, atol=5 * np.sqrt(4 / 45 / n))
    np.testing.assert_allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-6)
    np.testing.assert_array_equal(ctx.energies()[0], 0.0)
    ctx.close()


def test_single_temperature_has_no_exchange():
    """One temperature: the PT pass has no pair, the permutation stays the
    identity and the acceptance statistics stay empty; steps still advance
    both counters."""
    smp = inputs.small_sample(8, n_temps=1, disorder_seed=2)
    ctx = hsg.Context([smp], 3, 1)
    ctx.step(4)
    np.testing.assert_array_equal(ctx.get_perm()[0], np.zeros((3, 1), dtype=np.int32))
    sweeps, passes = ctx.counters()
    assert int(sweeps[0]) == 24 and int(passes[0]) == 4
    ctx.close()


def test_allocation_failure_releases_the_partial_context():
    """Each device allocation of hsg_create made to fail in turn (host-requested,
    as an out-of-memory would): the call returns HSG_ENOMEM naming the failed
    allocation and releases what it had allocated (device memory back where it
    was), and a context created with one more allocation allowed runs a step."""
    import torch
    smp = inputs.small_sample(16, n_temps=4, h_r=0.1, disorder_seed=5)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n = 1
    while True:
        try:
            ctx = hsg.Context([smp], 2, 1, variant=hsg.VARIANT_TWO_PASS,
                              sweep_kernel=hsg.SWEEP_HALF, inject_alloc_fault=n)
        except hsg.HsgError as e:
            assert e.status == 2 and "injected allocation failure" in str(e), str(e)
            n += 1
            assert n < 200
            continue
        break
    ctx.step(1)
    ctx.sync()
    assert ctx.info().pt_count == 1
    ctx.close()
    assert n > 10                       # the create path has that many allocations
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
