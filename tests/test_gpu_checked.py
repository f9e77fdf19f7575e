"""The bounds-checked build runs the parity cases without an index out of
range (it stands in for a memory sanitizer: every index read from an index
table is tested against its array before it is used)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_runs_the_parity_cases():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "all cases passed" in r.stdout
