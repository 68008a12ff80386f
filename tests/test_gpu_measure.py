"""GPU overlap tensor q^{mu nu}(k) (hsg_measure, Eqs. 5 and 6 with the modes
k = 0, k_min e_x, e_y, e_z) against the FP64 oracle on the same spins.

The GPU reads the stored spins and hsg_get_spins returns exactly the decoded
values, so the oracle sees the same configurations and the same temperature
assignment (hsg_get_perm).  On the GPU a lane sums its share of a block's
storage sites in FP32 (at most a few hundred products of magnitude <= 1) and
everything after that in FP64, so after the 1/N normalisation the difference
stays below 2e-6.

Covered: both kernels (staged copies into shared memory, and the direct
kernel for contexts whose staged systems exceed shared memory), slot counts
that leave lanes idle (5), fill a warp (24) and need two rounds of 32 (40),
mixed lattice sizes with ragged blocks, scattered permutations after PT, every
storage format, and the benchmark's full size on sampled slots.
"""
import ctypes

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


def oracle_tensor(spins, L, R_T, perm):
    """q [R_T, 3, 3] and qk [R_T, 3(axis), 3, 3, 2] of replicas 0 and 1."""
    q = np.zeros((R_T, 3, 3))
    qk = np.zeros((R_T, 3, 3, 3, 2))
    dp = ctypes.POINTER(ctypes.c_double)
    s = np.ascontiguousarray(spins, dtype=np.float64)
    pm = np.ascontiguousarray(perm, dtype=np.int32)
    oracle.lib().orc_measure(s.ctypes.data_as(dp), L, R_T,
                             pm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             q.ctypes.data_as(dp), qk.ctypes.data_as(dp))
    return q, qk


def compare(ctx, samples, tol=TOL):
    m = ctx.measure()
    spins = ctx.get_spins()
    perm = ctx.get_perm()
    for k, smp in enumerate(samples):
        np.testing.assert_array_equal(m["perm"][k], perm[k])
        q, qk = oracle_tensor(spins[k], smp.L, len(smp.temps), perm[k])
        np.testing.assert_allclose(m["q"][k], q, rtol=0, atol=tol)
        np.testing.assert_allclose(m["qk"][k], qk, rtol=0, atol=tol)
    return m


@pytest.mark.parametrize("n_temps", [5, 24, 40])
@pytest.mark.parametrize("R_O", [2, 3])
def test_tensor_matches_oracle_batch(n_temps, R_O):
    """Lattices of 4, 6 and 10 (blocks that end inside a parity half and
    samples smaller than one block), after steps with PT."""
    samples = [inputs.small_sample(L, n_temps=n_temps, h_r=0.1, disorder_seed=L, t_min=0.3,
                                   t_max=0.6) for L in (4, 6, 10)]
    ctx = hsg.Context(samples, R_O, 7, precision="fp32")
    ctx.step(3)
    assert any((p != np.arange(n_temps)).any() for pk in ctx.get_perm() for p in pk)
    compare(ctx, samples)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp16", "bf16", "angle16", "oct16", "yx4"])
def test_tensor_matches_oracle_compressed(precision):
    samples = [inputs.small_sample(8, n_temps=6, h_r=0.1, disorder_seed=2),
               inputs.small_sample(12, n_temps=6, h_r=0.1, disorder_seed=3)]
    ctx = hsg.Context(samples, 2, 5, precision=precision, j_fp16=True)
    ctx.step(2)
    compare(ctx, samples)
    ctx.close()


def test_tensor_direct_kernel_for_many_slots():
    """160 slots of FP32 spins: the staged rows of replicas 0 and 1 exceed the
    shared-memory budget, so the direct kernel measures; same result."""
    samples = [inputs.small_sample(4, n_temps=160, disorder_seed=9, t_min=0.2, t_max=2.0)]
    ctx = hsg.Context(samples, 2, 3, precision="fp32")
    ctx.step(1)
    compare(ctx, samples)
    ctx.close()


def test_tensor_of_identical_replicas_is_self_overlap():
    """Replica 1 set equal to replica 0 at identity permutation: the trace of
    q(k = 0) is 1 for every slot, and q is symmetric."""
    smp = inputs.small_sample(6, n_temps=3, disorder_seed=1)
    ctx = hsg.Context([smp], 2, 2)
    ctx.sweep_hb(1)
    s = ctx.get_spins()[0].copy()
    s[3:] = s[:3]
    ctx.set_spins([s])
    m = ctx.measure()
    for t in range(3):
        np.testing.assert_allclose(np.trace(m["q"][0, t]), 1.0, atol=1e-6)
        np.testing.assert_allclose(m["q"][0, t], m["q"][0, t].T, atol=1e-6)
    ctx.close()


def test_tensor_fullsize_on_sampled_slots():
    """The benchmark's workload (L = 128, 2 x 24 slots, FP16 spins) after one
    step: q and q(k) of two slots against the oracle's double loop over the two
    configurations alone."""
    w = inputs.workload("L128_fp16")
    smp = w.samples[0]
    smp16 = inputs.Sample(L=smp.L, J=inputs.round_fp16(smp.J), H=inputs.round_fp16(smp.H),
                          temps=smp.temps)
    ctx = hsg.Context([smp16], w.n_replicas, w.seed, precision="fp16", j_fp16=True)
    ctx.step(1)
    m = ctx.measure()
    spins = ctx.get_spins()[0]
    perm = ctx.get_perm()[0]
    R_T = len(smp16.temps)
    for t in (0, R_T - 1):
        sub = np.stack([spins[perm[0, t]], spins[R_T + perm[1, t]]])
        q, qk = oracle_tensor(sub, smp16.L, 1, np.zeros((2, 1), dtype=np.int32))
        np.testing.assert_allclose(m["q"][0, t], q[0], rtol=0, atol=TOL)
        np.testing.assert_allclose(m["qk"][0, t], qk[0], rtol=0, atol=TOL)
    ctx.close()
