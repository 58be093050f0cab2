"""The checked build (DGC_CHECKED: device bounds checks of every gather index,
the stand-in for a memory checker, which this pool does not offer) on small
cases with full oracle parity, run in a process of its own so that the checked
library is the one loaded."""
import os
import subprocess
import sys

import pytest

from paper_1508_04245_gb300 import build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_checked_build_small_cases_and_caught_gather():
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, DGC_LIBRARY="checked")
    env.pop("DGC_FAULT", None)
    r = subprocess.run([sys.executable, os.path.join(here, "checked_cases.py")], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "all cases OK" in r.stdout
