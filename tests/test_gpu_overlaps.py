"""GPU replica-pair and chiral overlaps (hsg_measure_overlaps) against the FP64
oracle on the same spins, through every path: D from the staged kernel over
the spins, C from the chirality buffer and the staged kernel over it, and the
direct kernel (D with C) where the staged systems exceed shared memory.

The GPU reads the stored spins; hsg_get_spins returns exactly the decoded
values, so the oracle sees the same configurations.  Per-thread sums run in FP32
on the GPU (a few hundred terms of magnitude <= 1 at most), everything else in
FP64, so after the 1/N normalisation the difference stays below 2e-6.
"""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def compare_with_oracle(ctx, samples, R_O, tol=TOL, chiral=True):
    """chiral=False measures D alone, which the staged kernel serves; with the
    chiral overlaps both come from the direct kernel."""
    out = ctx.measure_overlaps(chiral=chiral)
    spins = ctx.get_spins()
    perm = ctx.get_perm()
    R_T = len(samples[0].temps)
    P = ctx.info().n_overlap_pairs
    assert P == min(R_O, 4) * (min(R_O, 4) - 1) // 2
    for k, smp in enumerate(samples):
        D, C = oracle.overlaps(spins[k].astype(np.float64), smp.L, R_O, R_T, perm[k])
        np.testing.assert_allclose(out["D"][k], D, rtol=0, atol=tol)
        if chiral:
            np.testing.assert_allclose(out["C"][k], C, rtol=0, atol=tol)
    return out


@pytest.mark.parametrize("chiral", [True, False])
@pytest.mark.parametrize("R_O", [2, 3, 4, 5])
def test_overlaps_match_oracle_batch(R_O, chiral):
    """Mixed lattice sizes (4, 6, 10; row tiles ragged for 5 slots), after steps
    with PT so that the slots map to scattered memory slots."""
    samples = [inputs.small_sample(L, n_temps=5, h_r=0.1, disorder_seed=L) for L in (4, 6, 10)]
    ctx = hsg.Context(samples, R_O, 3, precision="fp32")
    ctx.step(3)
    compare_with_oracle(ctx, samples, R_O, chiral=chiral)
    ctx.close()


@pytest.mark.parametrize("n_temps", [16, 40])
def test_scalar_overlaps_many_slots(n_temps):
    """D alone for 16 slots (two sites per warp step) and 40 (two rounds of 32
    slots), four replicas."""
    samples = [inputs.small_sample(L, n_temps=n_temps, h_r=0.1, disorder_seed=L, t_min=0.3,
                                   t_max=0.6) for L in (6, 8)]
    ctx = hsg.Context(samples, 4, 11, precision="fp32")
    ctx.step(2)
    compare_with_oracle(ctx, samples, 4, chiral=False)
    ctx.close()


@pytest.mark.parametrize("chiral", [True, False])
@pytest.mark.parametrize("precision", ["fp16", "bf16", "angle16", "oct16", "yx4"])
def test_overlaps_match_oracle_compressed(precision, chiral):
    samples = [inputs.small_sample(8, n_temps=6, h_r=0.1, disorder_seed=2)]
    ctx = hsg.Context(samples, 4, 5, precision=precision, j_fp16=True)
    ctx.step(2)
    compare_with_oracle(ctx, samples, 4, chiral=chiral)
    ctx.close()


def test_overlaps_single_slot_many_rows():
    """One temperature slot: 256 rows per tile, a tile larger than the plane."""
    samples = [inputs.small_sample(12, n_temps=1, disorder_seed=4)]
    ctx = hsg.Context(samples, 2, 1)
    ctx.sweep_hb(2)
    compare_with_oracle(ctx, samples, 2)
    ctx.close()


def test_overlaps_of_identical_replicas():
    """Replica 1 set equal to replica 0 (no PT yet, so slot t is memory slot t
    in both): D_01 = 1 at k = 0 and C_01^a(0) is the mean squared chirality."""
    smp = inputs.small_sample(6, n_temps=3, disorder_seed=1)
    ctx = hsg.Context([smp], 2, 2)
    ctx.sweep_hb(1)
    s = ctx.get_spins()[0].copy()
    s[3:] = s[:3]
    ctx.set_spins([s])
    assert (ctx.get_perm()[0] == np.arange(3)).all()
    out = ctx.measure_overlaps()
    for t in range(3):
        np.testing.assert_allclose(out["D"][0, t, 0, 0], [1.0, 0.0], atol=1e-6)
        k = oracle.chirality(s[t].astype(np.float64), 6)
        np.testing.assert_allclose(out["C"][0, t, 0, :, 0, 0], (k ** 2).mean(axis=0), atol=1e-6)
        np.testing.assert_allclose(out["C"][0, t, 0, :, 0, 1], 0.0, atol=0)
    ctx.close()


def test_overlaps_invalid_arguments():
    smp = inputs.small_sample(4, n_temps=2)
    ctx = hsg.Context([smp], 1, 1)
    assert ctx.info().n_overlap_pairs == 0
    with pytest.raises(hsg.HsgError):
        ctx.measure_overlaps()
    ctx.close()


def test_overlaps_direct_kernel_for_many_slots():
    """Four replicas x 100 slots: the staged rows exceed the shared-memory
    budget, so the direct kernel measures D and C; same results."""
    samples = [inputs.small_sample(4, n_temps=100, h_r=0.1, disorder_seed=12, t_min=0.2, t_max=2.0)]
    ctx = hsg.Context(samples, 4, 9, precision="fp32")
    ctx.step(1)
    compare_with_oracle(ctx, samples, 4, chiral=True)
    compare_with_oracle(ctx, samples, 4, chiral=False)
    ctx.close()
