"""The bounds-checked build (-DMEVP_CHECKED, the substitute for a memory
sanitizer on this platform): every kernel family runs small cases in it with
no out-of-bounds access reported, and its results equal the normal build's
bitwise (the checks do not touch the arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_00466_gb300 import build as B  # noqa: E402
from tests import checked_cases  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_checked_build_reports_nothing_and_matches_bitwise(tmp_path):
    lib = B.build(checked=True)
    out = tmp_path / "checked.npz"
    env = dict(os.environ, MEVP_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases", str(out)],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    checked = dict(np.load(out))
    normal = checked_cases.run_all()
    assert set(checked) == set(normal)
    for k in normal:
        assert np.array_equal(checked[k], normal[k]), k
