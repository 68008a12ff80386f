"""The library built with device bounds checks (-DHSG_CHECK, libhsg_check.so):
the sweep kernels check every storage index they form (own site in its parity
half, neighbours in the other half, staged rows within their half and stage)
and a failed check sets an error word that the host reports as HSG_ESTATE.  Run
in a child process (the binding loads one build per process) on small and
ragged lattices with every over-relaxation kernel and both schedules, it must
report no error and give the same spins, bit for bit, as the normal build."""
import hashlib
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1204_6192_gb300 import hsg, inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (L, precision, j_fp16, variant, sweep kernel)
CASES = []
for L in (4, 6, 8, 16, 32, 64):
    for prec, j16 in (("fp32", False), ("fp16", True)):
        kernels = [hsg.SWEEP_HALF, hsg.SWEEP_WAVE]
        if L >= 32:
            kernels.append(hsg.SWEEP_STAGED)
        if L % 4 == 0 and L >= 8:
            kernels.append(hsg.SWEEP_FUSED)
        for k in kernels:
            CASES.append((L, prec, j16, hsg.VARIANT_TWO_PASS, k))
        CASES.append((L, prec, j16, hsg.VARIANT_PERSISTENT, hsg.SWEEP_HALF))

CHILD = r"""
import hashlib, sys
sys.path.insert(0, ROOT)
from paper_1204_6192_gb300 import hsg, inputs
hsg.use_library(LIB)
for (L, prec, j16, variant, kernel) in CASES:
    smp = inputs.small_sample(L, n_temps=3, h_r=0.1, disorder_seed=L)
    ctx = hsg.Context([smp], 2, 7, precision=prec, j_fp16=j16, variant=variant, sweep_kernel=kernel)
    ctx.sweep_or(3)
    ctx.step(2)
    m = ctx.measure()
    h = hashlib.sha256(b"".join(x.tobytes() for x in ctx.get_spins()) + m["E"].tobytes()).hexdigest()
    ctx.close()
    print(L, prec, variant, kernel, h, flush=True)
print("ok")
"""


def digest(L, prec, j16, variant, kernel):
    smp = inputs.small_sample(L, n_temps=3, h_r=0.1, disorder_seed=L)
    ctx = hsg.Context([smp], 2, 7, precision=prec, j_fp16=j16, variant=variant, sweep_kernel=kernel)
    ctx.sweep_or(3)
    ctx.step(2)
    m = ctx.measure()
    h = hashlib.sha256(b"".join(x.tobytes() for x in ctx.get_spins()) + m["E"].tobytes()).hexdigest()
    ctx.close()
    return h


def test_bounds_checked_build_reports_nothing_and_matches():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1204_6192_gb300 import build
    lib = build.build(check=True)
    code = f"ROOT = {ROOT!r}\nLIB = {lib!r}\nCASES = {CASES!r}\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-2000:]
    got = [line.split()[-1] for line in r.stdout.strip().splitlines()[:-1]]
    assert len(got) == len(CASES)
    for case, h in zip(CASES, got):
        assert digest(*case) == h, case
