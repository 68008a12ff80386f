"""Closed-form pins of the oracle's whole Markov chain (heat-bath sweeps on the
lattice, Eq. 2; parallel tempering, Eq. 4).

* Couplings along one axis only: the lattice falls apart into L^2 periodic
  Heisenberg rings, whose partition function is exact,
  Z = sum_l (2l+1) prod_b i_l(beta J_b) (i_l: modified spherical Bessel
  functions, scipy), so <E> = -d ln Z / d beta.  Run for each axis, this pins
  the bond indexing, the periodic wrap and the heat-bath sampler together.
* No couplings, a field: independent spins, <E> = -sum_i |H_i| L(beta |H_i|),
  L(a) = coth a - 1/a.
* All axes and a field at small beta: the high-temperature series
  <E> = -beta k2 + beta^2 k3 / 2 + O(beta^3).
* Parallel tempering: acceptance frequency min(1, exp(dbeta dE)) for injected
  energies; the upward carry of one pass; and per-temperature Boltzmann
  averages of independent spins kept under heat bath + exchange.
"""
import numpy as np
import pytest
from scipy import special

from paper_1204_6192_gb300 import inputs


def langevin(a):
    a = np.asarray(a, dtype=np.float64)
    return 1.0 / np.tanh(a) - 1.0 / a


def i_l(l, x):
    # parity of the modified spherical Bessel function: i_l(-x) = (-1)^l i_l(x)
    return special.spherical_in(l, np.abs(x)) * np.where(x < 0, (-1.0) ** l, 1.0)


def di_l(l, x):
    return special.spherical_in(l, np.abs(x), derivative=True) * np.where(x < 0, (-1.0) ** (l + 1), 1.0)


def ring_energy(J_ring, beta, lmax=60):
    """<E> of a periodic Heisenberg ring with bonds J_ring at inverse temperature beta."""
    K = beta * np.asarray(J_ring)
    Z = 0.0
    dZ = 0.0
    for l in range(lmax):
        v = i_l(l, K)
        d = di_l(l, K) * np.asarray(J_ring)
        prod = np.prod(v)
        Z += (2 * l + 1) * prod
        dZ += (2 * l + 1) * sum(d[b] * np.prod(np.delete(v, b)) for b in range(len(v)))
    return -dZ / Z


def run_energy_series(orc, smp, n_rep, sweeps, burn=50, n_or=1, seed=7):
    sim = orc.OracleSim([smp], n_replicas=n_rep, seed=seed)
    series = []
    for k in range(burn + sweeps):
        sim.sweep_hb(1)
        sim.sweep_or(n_or)
        if k >= burn:
            series.append(sim.energies()[0])
    return np.array(series)          # [sweeps, W]


def binned_error(x, nbins=20):
    b = np.array_split(x, nbins)
    m = np.array([bb.mean(axis=0) for bb in b])
    return m.std(axis=0, ddof=1) / np.sqrt(nbins)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_rings_along_one_axis_exact(orc, axis):
    L = 4
    rng = np.random.default_rng(20 + axis)
    J = np.zeros((L ** 3, 3))
    J[:, axis] = rng.standard_normal(L ** 3) * 1.3
    temps = np.array([0.4, 0.8, 1.6])
    smp = inputs.Sample(L=L, J=J, H=np.zeros((L ** 3, 3)), temps=temps)
    E = run_energy_series(orc, smp, n_rep=2, sweeps=3000)
    mean = E.mean(axis=0)
    err = binned_error(E)
    # exact: sum over the L^2 rings along `axis`
    idx = np.arange(L ** 3).reshape(L, L, L)      # [z, y, x]
    rings = np.moveaxis(idx, 2 - axis, -1).reshape(-1, L)
    for r in range(2):
        for t, T in enumerate(temps):
            w = r * len(temps) + t
            exact = sum(ring_energy(J[ring, axis], 1.0 / T) for ring in rings)
            assert abs(mean[w] - exact) < 5 * err[w] + 1e-3, (axis, T, mean[w], exact, err[w])


def test_rings_differ_from_open_chains(orc):
    """The closed form above is sensitive to the periodic wrap at this size."""
    rng = np.random.default_rng(3)
    Jr = np.abs(rng.standard_normal(4)) + 1.0
    open_chain = -sum(j * langevin(j / 0.4) for j in Jr)
    assert abs(ring_energy(Jr, 1 / 0.4) - open_chain) > 0.05


def test_independent_spins_in_field(orc):
    L = 4
    rng = np.random.default_rng(30)
    H = rng.standard_normal((L ** 3, 3)) * 0.7
    temps = np.array([0.25, 0.5, 1.0, 3.0])
    smp = inputs.Sample(L=L, J=np.zeros((L ** 3, 3)), H=H, temps=temps)
    E = run_energy_series(orc, smp, n_rep=1, sweeps=1500, burn=2, n_or=0)
    hn = np.linalg.norm(H, axis=1)
    for t, T in enumerate(temps):
        a = hn / T
        m = langevin(a)
        exact = -np.sum(hn * m)
        sigma = np.sqrt(np.sum(hn ** 2 * (1 - 2 * m / a - m * m)) / E.shape[0])
        assert abs(E[:, t].mean() - exact) < 5 * sigma


def test_high_temperature_series(orc):
    L = 4
    rng = np.random.default_rng(40)
    J = rng.standard_normal((L ** 3, 3))
    H = rng.standard_normal((L ** 3, 3)) * 0.3
    beta = 0.1
    W = 32
    smp = inputs.Sample(L=L, J=J, H=H, temps=np.full(W, 1.0 / beta))
    E = run_energy_series(orc, smp, n_rep=1, sweeps=2500, burn=10, n_or=1)
    k2 = (J ** 2).sum() / 3 + (H ** 2).sum() / 3
    # k3 = -(2/3) sum_bonds J_b H_i.H_j
    k3 = 0.0
    R = np.stack(np.unravel_index(np.arange(L ** 3), (L, L, L))[::-1], axis=1)  # x, y, z
    idx = np.arange(L ** 3).reshape(L, L, L)
    for i in range(L ** 3):
        x, y, z = R[i]
        nbr = [idx[z, y, (x + 1) % L], idx[z, (y + 1) % L, x], idx[(z + 1) % L, y, x]]
        for a in range(3):
            k3 += -(2.0 / 3.0) * J[i, a] * (H[i] @ H[nbr[a]])
    exact = -beta * k2 + beta ** 2 * k3 / 2
    mean = E.mean()
    err = binned_error(E.mean(axis=1))
    assert abs(mean - exact) < 5 * err + 0.02 * abs(exact) * beta ** 2, (mean, exact, err)


def test_pt_acceptance_frequency(orc):
    n_chains = 4000
    temps = np.array([0.5, 0.7])
    for dE in (-0.8, -0.2, 0.0, 0.3, 1.5):
        # configuration at slot 0 has energy 0, at slot 1 energy dE
        E = np.tile([0.0, dE], n_chains)
        perm0 = np.tile([0, 1], (n_chains, 1)).astype(np.int32)
        acc_total = 0
        steps = 5
        for step in range(steps):
            _, acc = orc.pt(E, temps, perm0, n_chains, 2, 0, 99, step)
            acc_total += acc.sum()
        x = (1 / temps[1] - 1 / temps[0]) * dE
        p = min(1.0, np.exp(x))
        n = n_chains * steps
        freq = acc_total / n
        if p == 1.0:
            assert freq == 1.0
        else:
            assert abs(freq - p) < 5 * np.sqrt(p * (1 - p) / n), (dE, freq, p)


def read_golden(name):
    import os
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                key, *vals = line.split()
                out[key] = np.array([float(v) for v in vals])
    return out


def test_pt_upward_carry(orc):
    """Hand-worked pass of Eq. (4) with R_T = 4 (tests/golden/pt_upward_carry.txt):
    energies fall with slot, every attempt is accepted, so the configuration
    that starts at the lowest temperature is carried to the top in one pass;
    with the energies scaled by -100 nothing is accepted."""
    g = read_golden("pt_upward_carry.txt")
    p0 = g["perm_in"].astype(np.int32)[None, :]
    perm, acc = orc.pt(g["energies"], g["temps"], p0.copy(), 1, 4, 0, 5, 0)
    np.testing.assert_array_equal(perm[0], g["perm_out"])
    np.testing.assert_array_equal(acc[0], g["accepted"])
    perm, acc = orc.pt(g["scaled_energies"], g["temps"], p0.copy(), 1, 4, 0, 5, 0)
    np.testing.assert_array_equal(perm[0], g["scaled_perm_out"])
    np.testing.assert_array_equal(acc[0], g["scaled_accepted"])


def test_pt_keeps_boltzmann_per_temperature(orc):
    """Independent spins in a uniform field under heat bath + exchange: measured
    right after each exchange, slot t must still show <E>/N = -|H| L(|H|/T_t);
    a wrong sign of dbeta or dE, or swapping spins twice, breaks it."""
    L = 4
    N = L ** 3
    H0 = np.array([0.0, 0.0, 1.0])
    temps = np.array([0.3, 0.45, 0.7, 1.1])
    smp = inputs.Sample(L=L, J=np.zeros((N, 3)), H=np.tile(H0, (N, 1)), temps=temps)
    sim = orc.OracleSim([smp], n_replicas=2, seed=11)
    per_slot = []
    acc_sum = 0
    for k in range(2500):
        sim.sweep_hb(1)
        acc = sim.pt_exchange()
        acc_sum += acc[0].sum()
        m = sim.measure()[0]
        per_slot.append(m["E"])           # [R_O, R_T] by temperature slot
    per_slot = np.array(per_slot)
    assert acc_sum > 0
    for t, T in enumerate(temps):
        a = 1.0 / T
        mL = langevin(a)
        exact = -N * mL
        sigma = np.sqrt(N * (1 - 2 * mL / a - mL * mL) / per_slot.shape[0])
        for r in range(2):
            assert abs(per_slot[:, r, t].mean() - exact) < 5 * sigma, (t, r)


def test_oracle_matches_its_recorded_run():
    """The oracle reproduces the run recorded by tests/golden/make_oracle_fixture.py
    (energies, permutation, overlap after two steps of a seeded L = 4 sample)."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "make_oracle_fixture", os.path.join(os.path.dirname(__file__), "golden", "make_oracle_fixture.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    g = read_golden("oracle_L4_two_steps.txt")
    now = mod.run()
    np.testing.assert_array_equal(now["perm"], g["perm"])
    np.testing.assert_allclose(now["E"], g["E"], rtol=1e-10)
    np.testing.assert_allclose(now["q"], g["q"], rtol=0, atol=1e-10)


def test_pt_diagnostics_hand_worked(orc):
    """tests/golden/pt_tunnelling.txt: four forced passes; the oracle's moved
    counts (by comparing the permutation before and after each pass) and its
    tunnelling count match the hand-worked values."""
    g = read_golden("pt_tunnelling.txt")
    o = orc.OracleSample(4, np.zeros((64, 3)), None, g["temps"], 1, 0, 0, 5, 0)
    for k in range(4):
        o.pt(g[f"energies_{k}"], k)
        np.testing.assert_array_equal(o.perm[0], g[f"perm_{k}"])
    np.testing.assert_array_equal(o.moved[0], g["moved"])
    np.testing.assert_array_equal(o.tunnel[0], g["tunnel"])


def test_pt_diagnostics_consistent_with_acceptances(orc):
    """Random passes: with the pairs visited upward, the configuration at slot t
    moves iff pair (t-1, t) or pair (t, t+1) accepts, so the oracle's moved
    counts (taken from the permutations) equal the sums of a_{t-1} | a_t over
    the passes (taken from the acceptances)."""
    rng = np.random.default_rng(3)
    temps = np.array([0.4, 0.5, 0.62, 0.77, 0.95])
    o = orc.OracleSample(4, np.zeros((64, 3)), None, temps, 2, 0, 0, 9, 0)
    expect = np.zeros((2, 5), dtype=np.int64)
    for k in range(300):
        E = rng.normal(scale=3.0, size=10)
        acc = o.pt(E, k)
        a = np.pad(acc.astype(bool), ((0, 0), (1, 1)))
        expect += a[:, :-1] | a[:, 1:]
    np.testing.assert_array_equal(o.moved, expect)
