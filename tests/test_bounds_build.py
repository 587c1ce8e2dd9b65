"""The bounds-checking build (FR_DEBUG_BOUNDS): element offsets and partner indices are checked on
the device, and a failed check sets a status bit (FR_EBOUNDS) and skips the access instead of
touching memory out of bounds. On valid meshes of every element type and form -- hexahedra p = 3
and 4, FP64, low-Mach FP32, the mixed hex/prism grid with the FP16 tensor-core form, tetrahedra,
pyramids, curved hexahedra, an ensemble over graph-replayed RK4 steps, a partitioned mesh -- no
check may fire and every result must equal the release build's bit for bit (the checks do not
change the arithmetic). Each library runs in a fresh process (tests/bounds_case.py)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_build_matches_release_and_reports_nothing(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_06132_gb300 import build as B
    B.build()
    B.build(variant="bounds")
    out = {}
    for lib in ("release", "bounds"):
        env = dict(os.environ)
        env.pop("FR_LIBRARY", None)
        if lib == "bounds":
            env["FR_LIBRARY"] = "bounds"
        path = str(tmp_path / f"{lib}.npz")
        r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_case.py"), path], env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stderr[-3000:]
        out[lib] = dict(np.load(path))
    assert out["release"].keys() == out["bounds"].keys()
    for k in out["release"]:
        assert np.array_equal(out["release"][k], out["bounds"][k]), k
