"""The README's quick-start example runs as written."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_quick_start_runs():
    import __graft_entry__
    __graft_entry__.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "no python example in README.md"
    ns = {}
    exec(compile(blocks[0], "README.md", "exec"), ns)
    assert ns["chi"].shape == (1, 16, 4)
    assert ns["ov"]["C"].shape == (1, 16, 1, 3, 4, 2)
