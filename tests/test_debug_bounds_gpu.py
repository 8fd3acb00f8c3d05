"""The bounds-checked build (MERF_DEBUG_BOUNDS: every data-dependent index checked, violations
recorded in a device status word, never trapped) gives the release build's results on valid
scenes, records nothing, and reports its status word's self-test bit through merf_check_device."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests import debug_cases

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_matches_release_and_reports(tmp_path):
    for name, fn in debug_cases.CASES.items():
        np.save(tmp_path / (name + ".npy"), fn())
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_child.py"), str(tmp_path)],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug build ok" in r.stdout
