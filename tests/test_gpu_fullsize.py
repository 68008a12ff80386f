"""Parity at the benchmark's full size and launch configuration.

L = 128, 2 replicas x 24 temperatures in [0.08, 0.3], FP16 spins and FP16
couplings, H_r = 0.1 (100.7M spins), advanced with hsg_step exactly as
bench.py times it.  The oracle computes complete systems on its own: the
initial state from its own Philox stream, then one step (1 HB + 5 OR sweeps)
for a sample of systems.  Parallel tempering couples all 24 temperatures of a
chain, so after the step it is checked through properties that hold at any
size (valid permutations; the step's energies equal a fresh FP64 evaluation).
"""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu

FP16_QUANTUM = 2.0 ** -11
SAMPLED = (5, 30)          # memory slots compared with the oracle (one per replica)


@pytest.fixture(scope="module")
def full():
    import __graft_entry__
    __graft_entry__.build()
    w = inputs.workload("L128_fp16")
    smp = w.samples[0]
    smp16 = inputs.Sample(L=smp.L, J=inputs.round_fp16(smp.J), H=inputs.round_fp16(smp.H),
                          temps=smp.temps)
    ctx = hsg.Context([smp16], w.n_replicas, w.seed, precision="fp16", j_fp16=True)
    yield w, smp16, ctx
    ctx.close()


def oracle_systems(smp16, w, slots):
    """Initial states of the given memory slots, computed by the oracle."""
    N = smp16.L ** 3
    W = w.n_replicas * len(smp16.temps)
    Wp = (W + 7) // 8 * 8
    out = {}
    lib = oracle.lib()
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    for j in slots:
        s = np.zeros((1, N, 3))
        # one system: global id j (sample 0), fp16 storage
        lib.orc_init_spins(s.ctypes.data_as(dp), smp16.L, 1, j, w.seed, oracle.CODECS["fp16"])
        out[j] = s
    assert W == 48 and Wp == 48
    return out


def test_fullsize_initial_state_and_energy(full):
    w, smp16, ctx = full
    spins = ctx.get_spins()[0]
    ref = oracle_systems(smp16, w, SAMPLED)
    E = ctx.energies()[0]
    for j, s in ref.items():
        d = np.abs(spins[j] - s[0])
        # FP32 and FP64 rounding of the same value to binary16 differ in rare ties
        assert np.median(d) == 0.0 and d.max() <= FP16_QUANTUM
        E_ref = oracle.energy(s, smp16.J, smp16.H, smp16.L)[0]
        assert abs(E[j] - E_ref) < 1e-5 * abs(E_ref)


def test_fullsize_step_matches_oracle_on_sampled_systems(full):
    w, smp16, ctx = full
    ref = oracle_systems(smp16, w, SAMPLED)
    ctx.step(1)                      # the graph bench.py replays: HB, 5 OR, energies, PT
    spins = ctx.get_spins()[0]
    N = smp16.L ** 3
    for j, s0 in ref.items():
        r, t = divmod(j, len(smp16.temps))
        beta = np.array([1.0 / smp16.temps[t]])
        s = s0.copy()
        lib = oracle.lib()
        import ctypes
        dp = ctypes.POINTER(ctypes.c_double)
        args = (smp16.J.ctypes.data_as(dp), smp16.H.ctypes.data_as(dp))
        # the step's heat-bath sweep (sweep counter 0), then five OR sweeps
        for parity in (0, 1):
            lib.orc_hb_half(s.ctypes.data_as(dp), *args, smp16.L, 1, parity,
                            beta.ctypes.data_as(dp), j, w.seed, 0, oracle.CODECS["fp16"])
        for _ in range(5):
            for parity in (0, 1):
                lib.orc_or_half(s.ctypes.data_as(dp), *args, smp16.L, 1, parity,
                                oracle.CODECS["fp16"])
        d = np.abs(spins[j] - s[0]).ravel()
        # equal up to binary16 rounding, amplified by six sweeps of chaotic dynamics
        assert np.median(d) <= FP16_QUANTUM, np.median(d)
        assert np.quantile(d, 0.99) <= 16 * FP16_QUANTUM, np.quantile(d, 0.99)
    perm = ctx.get_perm()[0]
    for r in range(w.n_replicas):
        assert sorted(perm[r]) == list(range(len(smp16.temps)))
    E_step = ctx.last_energies()[0]
    E_new = ctx.energies()[0]
    np.testing.assert_allclose(E_step, E_new, rtol=1e-7)
    assert np.all(np.isfinite(ctx.measure()["q"]))


def test_fullsize_overlaps_on_sampled_slots(full):
    """hsg_measure_overlaps at full size: the spin and chiral pair overlaps of
    two temperature slots, recomputed by the oracle from the two configurations
    alone (FP32 partial sums of at most a few hundred terms)."""
    w, smp16, ctx = full
    out = ctx.measure_overlaps()
    out_d = ctx.measure_overlaps(chiral=False)      # D alone: the staged kernel
    spins = ctx.get_spins()[0]
    perm = ctx.get_perm()[0]
    R_T = len(smp16.temps)
    for t in (0, R_T - 1):
        sub = np.stack([spins[perm[0, t]], spins[R_T + perm[1, t]]]).astype(np.float64)
        D, C = oracle.overlaps(sub, smp16.L, 2, 1, np.zeros((2, 1), dtype=np.int32))
        np.testing.assert_allclose(out["D"][0, t], D[0], rtol=0, atol=2e-6)
        np.testing.assert_allclose(out["C"][0, t], C[0], rtol=0, atol=2e-6)
        np.testing.assert_allclose(out_d["D"][0, t], D[0], rtol=0, atol=2e-6)
