"""Child process of tests/test_debug_bounds_gpu.py: renders with the bounds-checked library
(which must be chosen before the library is first loaded, hence a process of its own) and
compares with the release library's outputs saved by the parent."""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2302_12249_b300 import merf  # noqa: E402
from tests import debug_cases  # noqa: E402


def main(outdir: str) -> int:
    merf.use_debug_build()
    assert "bounds-checked" in merf.version(), merf.version()
    for name, fn in debug_cases.CASES.items():
        got = fn()
        want = np.load(os.path.join(outdir, name + ".npy"))
        err = float(np.abs(got - want).max())
        assert err <= 1e-6, (name, err)
        merf.check_device()                     # nothing out of range on valid scenes
    try:
        merf.check_device(self_test=True)
        raise AssertionError("the self-test bit was not reported")
    except merf.MerfError as e:
        assert e.status == merf.ERR_DEVICE_BOUNDS and "self-test" in str(e), str(e)
    merf.check_device()                         # cleared by the previous read
    torch.cuda.synchronize()
    print("debug build ok:", ", ".join(debug_cases.CASES))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1]))
