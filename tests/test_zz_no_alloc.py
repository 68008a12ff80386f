"""The allocation-free energy entry point (hsg_energies_xyz_noalloc) agrees with
the FP64 oracle and with the context's hsg_energies.

That entry point serves callers that cannot let a library allocate device
memory (a CUDA graph being captured, a program whose memory belongs to its own
pool allocator, a loop that must not synchronise on cudaMalloc): they hand in
their own device arrays and the library uses a fixed static scratch array.
This file is collected last so that a failure here does not hide the others.
"""
import numpy as np
import pytest

import oracle
from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu

# FP32 products summed in FP64 per thread: a few ulp of binary32 per site term
RTOL = 2e-6


def seeded_state(rng, W, N):
    s = rng.standard_normal((W, N, 3))
    return (s / np.linalg.norm(s, axis=2, keepdims=True)).astype(np.float32)


def noalloc_energies(torch, s, J, H, L, W):
    """One call of the entry point on device copies of s, J and H (H may be None:
    the entry point then gets a NULL field pointer)."""
    s_d = torch.from_numpy(s).cuda()
    J_d = torch.from_numpy(np.ascontiguousarray(J, dtype=np.float32)).cuda()
    H_d = None if H is None else torch.from_numpy(np.ascontiguousarray(H, dtype=np.float32)).cuda()
    E_d = torch.full((W,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    st = hsg.hsg_energies_xyz_noalloc(s_d.data_ptr(), J_d.data_ptr(),
                                      0 if H_d is None else H_d.data_ptr(), L, W,
                                      E_d.data_ptr(), stream.cuda_stream)
    assert st == 0, hsg.lib().hsg_last_error(None)
    torch.cuda.synchronize()
    return E_d.cpu().numpy()


def test_noalloc_energies_match_oracle_and_context_twice():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(17)
    # two calls in a row with different sizes share the static scratch
    cases = [(16, 4, 0.3), (6, 3, 0.0)]
    for L, n_temps, h_r in cases:
        smp = inputs.small_sample(L, n_temps=n_temps, h_r=h_r, disorder_seed=L)
        W = 2 * n_temps
        s = seeded_state(rng, W, L ** 3)
        J32 = np.asarray(smp.J, dtype=np.float32)
        H32 = np.asarray(smp.H, dtype=np.float32)
        # the oracle on exactly the binary32 values the device sees
        E_orc = oracle.energy(s.astype(np.float64), J32.astype(np.float64),
                              H32.astype(np.float64), L)
        ctx = hsg.Context([smp], 2, 3)
        ctx.set_spins([s])
        E_ctx = ctx.energies()[0]
        ctx.close()
        E = noalloc_energies(torch, s, J32, H32, L, W)
        np.testing.assert_allclose(E, E_orc, rtol=RTOL, atol=1e-4)
        np.testing.assert_allclose(E, E_ctx, rtol=RTOL, atol=1e-4)


def test_noalloc_null_field_matches_zero_field():
    """H = NULL means no field: equal to the oracle without a field and to a
    context built with h_r = 0."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(29)
    L, n_temps = 8, 3
    smp = inputs.small_sample(L, n_temps=n_temps, h_r=0.0, disorder_seed=5)
    W = 2 * n_temps
    s = seeded_state(rng, W, L ** 3)
    J32 = np.asarray(smp.J, dtype=np.float32)
    E_orc = oracle.energy(s.astype(np.float64), J32.astype(np.float64), None, L)
    ctx = hsg.Context([smp], 2, 3)
    ctx.set_spins([s])
    E_ctx = ctx.energies()[0]
    ctx.close()
    for _ in range(2):
        E = noalloc_energies(torch, s, J32, None, L, W)
        np.testing.assert_allclose(E, E_orc, rtol=RTOL, atol=1e-4)
        np.testing.assert_allclose(E, E_ctx, rtol=RTOL, atol=1e-4)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    torch = pytest.importorskip("torch")
    L, W = 128, 513          # 513 * 1024 partial sums > 524288
    dummy = torch.zeros(4, device="cuda")
    st = hsg.hsg_energies_xyz_noalloc(dummy.data_ptr(), dummy.data_ptr(), 0, L, W,
                                      dummy.data_ptr(), 0)
    assert st == 1
    assert b"static scratch" in hsg.lib().hsg_last_error(None)
