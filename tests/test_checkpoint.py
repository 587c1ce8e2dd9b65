"""Checkpoint / resume: the FP64 master state plus a JSON header (RK4 carries nothing else between
steps). CPU: round trip, header checks. GPU: 10 RK4 steps equal 5 steps, a checkpoint, a fresh
handle resumed from it and 5 more steps, bit for bit."""
import json

import numpy as np
import pytest

from paper_2401_06132_gb300 import checkpoint, workloads as W


def test_round_trip_and_header(tmp_path):
    U = np.random.default_rng(3).standard_normal(5 * 64 * 8)
    p = str(tmp_path / "ck")
    checkpoint.save(p, U, step=7, time=7e-3, instances=[{"values": U.size, "p": 3}], meta={"mesh": "box 2^3"})
    V, head = checkpoint.load(p, expect_values=U.size)
    assert np.array_equal(U, V) and V.dtype == np.float64
    assert head["step"] == 7 and head["time"] == 7e-3 and head["meta"]["mesh"] == "box 2^3"
    with pytest.raises(ValueError):
        checkpoint.load(p, expect_values=U.size + 1)
    with pytest.raises(ValueError):
        checkpoint.save(p, U, 0, 0.0, instances=[{"values": 3}])


def test_truncated_or_foreign_files_are_refused(tmp_path):
    p = str(tmp_path / "ck")
    checkpoint.save(p, np.ones(10), 1, 0.1)
    np.ones(9).tofile(p + ".bin")
    with pytest.raises(ValueError):
        checkpoint.load(p)
    with open(p + ".json", "w") as f:
        json.dump({"format": "other"}, f)
    with pytest.raises(ValueError):
        checkpoint.load(p)


@pytest.mark.gpu
def test_resume_equals_uninterrupted_run(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_06132_gb300 import build as B, fr
    B.build()
    mesh = W.box_hex_mesh(4)
    prm = fr.make_params(p=3, p_ref=W.tgv_p0())
    m = fr.FRMesh(mesh, prm)
    U0 = W.tgv_state(m.sol_coords(), [(64, 64)], perturb=1e-2)
    Ua = torch.from_numpy(U0).cuda()
    m.rk4_step(Ua, 1e-3, 10)
    m.sync_status()
    Ub = torch.from_numpy(U0).cuda()
    m.rk4_step(Ub, 1e-3, 5)
    m.sync_status()
    p = str(tmp_path / "ck")
    checkpoint.save(p, Ub, step=5, time=5e-3, instances=checkpoint.describe(m))
    m.close()
    m2 = fr.FRMesh(mesh, prm)
    V, head = checkpoint.load(p, expect_values=m2.num_values)
    Uc = torch.from_numpy(V).cuda()
    m2.rk4_step(Uc, 1e-3, 10 - head["step"])
    m2.sync_status()
    assert torch.equal(Ua, Uc)
