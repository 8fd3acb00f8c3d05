"""A scene uploaded from its file (merf_scene_load) renders bit for bit as the same scene uploaded
from its arrays, for every storage kind and the paper-scale scene."""
import numpy as np
import pytest
import torch

from paper_2302_12249_b300 import merf, scene_file, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,W,H,step", [("tiny", 48, 40, 1 / 64), ("tiny_grid", 48, 40, 1 / 64),
                                           ("dense128", 40, 32, 1 / 128)])
def test_file_upload_renders_identically(tmp_path, name, W, H, step):
    sc = synth.make_scene(name)
    p = str(tmp_path / f"{name}.merf")
    scene_file.save(sc, p)
    a, b = merf.Scene(sc), merf.Scene.load(p)
    assert a.device_bytes == b.device_bytes
    cams = synth.sphere_cameras(2, W, H, radius=2.3, seed=61)
    ra = merf.render(a, cams, W, H, step)
    rb = merf.render(b, cams, W, H, step)
    torch.cuda.synchronize()
    assert torch.equal(ra, rb)


def test_paper_scene_file(tmp_path, paper_scene):
    p = str(tmp_path / "paper.merf")
    scene_file.save(paper_scene, p)
    a, b = merf.Scene(paper_scene), merf.Scene.load(p)
    cams = synth.config_cameras("paper", W=320, H=180, n=2)
    ra = merf.render(a, cams, 320, 180, 1 / 256)
    rb = merf.render(b, cams, 320, 180, 1 / 256, precision=merf.PREC_FP32)
    torch.cuda.synchronize()
    assert torch.equal(ra, rb) and np.isfinite(rb.cpu().numpy()).all()
