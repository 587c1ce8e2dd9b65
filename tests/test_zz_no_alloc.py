"""fr_diagnostics_noalloc against fr_diagnostics (GPU).

fr_diagnostics allocates its device accumulators with cudaMalloc the first time it runs. Some callers
cannot allow that: a framework that owns the whole device memory budget, a real-time loop that cannot
take the device-wide synchronisation a cudaMalloc may cause, or a thread capturing work into a CUDA
graph in global mode, where cudaMalloc is illegal. For them the library offers
fr_diagnostics_noalloc, whose accumulators are a fixed array compiled into the library. These tests
call it through the C ABI twice in a row and compare with the allocating entry point, with the same
tolerances as the other diagnostics test. This file is collected last on purpose, so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_06132_gb300 import fr, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_06132_gb300 import build as B
    B.build()


def _same(d, ref):
    assert abs(d["volume"] - ref["volume"]) <= 1e-12 * abs(ref["volume"])
    assert abs(d["Ek"] - ref["Ek"]) <= 1e-13 * max(1.0, abs(ref["Ek"]))
    assert abs(d["eps"] - ref["eps"]) <= 1e-9 * max(abs(ref["eps"]), 1e-12)
    assert np.all(np.abs(d["sums"] - ref["sums"]) <= 1e-11 * np.maximum(1.0, np.abs(ref["sums"])))


def test_noalloc_diagnostics_match_allocating_entry_point_twice():
    mesh = W.box_hex_mesh(8)
    o = O.Oracle(mesh, 3, 5)
    U = W.tgv_state(o.sol_coords(), [(512, 64)])
    m = fr.FRMesh(mesh, fr.make_params(p=3))
    Ud = torch.from_numpy(U).cuda()
    Rd = torch.empty_like(Ud)
    m.rhs(Ud, Rd)
    ref = m.diagnostics(Ud, Rd)[0]
    first = m.diagnostics_noalloc(Ud, Rd)[0]
    second = m.diagnostics_noalloc(Ud, Rd)[0]   # the scratch keeps the first call's sums until cleared
    _same(first, ref)
    _same(second, ref)
    assert abs(ref["eps"] / (0.75 / 1600) - 1.0) < 1e-3   # the unperturbed TGV: eps(0) near 3 mu / 4


def test_noalloc_diagnostics_per_instance_slots():
    """Three instances of different order: each instance has its own accumulator slots; a call with
    no RHS (kinetic energy only) followed by one with the RHS gives the allocating entry point's
    results both times."""
    meshes = [W.box_hex_mesh(2), W.box_hex_mesh(3), W.sheared_box_mesh(2)]
    orders = [3, 4, 3]
    params = [fr.make_params(p=p) for p in orders]
    states = []
    for mesh, p in zip(meshes, orders):
        o = O.Oracle(mesh, p, p + 2)
        states.append(W.tgv_state(o.sol_coords(), [(mesh["hex_v"].shape[0], (p + 1) ** 3)], perturb=1e-2))
    m = fr.FRMesh(meshes, params)
    Ud = torch.from_numpy(np.concatenate(states)).cuda()
    Rd = torch.empty_like(Ud)
    m.rhs(Ud, Rd)
    ref_u = m.diagnostics(Ud)
    ref_r = m.diagnostics(Ud, Rd)
    got_u = m.diagnostics_noalloc(Ud)
    got_r = m.diagnostics_noalloc(Ud, Rd)
    for a, b in zip(got_u, ref_u):
        assert abs(a["Ek"] - b["Ek"]) <= 1e-13 and abs(a["volume"] - b["volume"]) <= 1e-12 * b["volume"]
    for a, b in zip(got_r, ref_r):
        _same(a, b)


def test_noalloc_allocates_nothing_on_a_fresh_handle():
    """A handle that has never run the allocating entry point: its first fr_diagnostics_noalloc call
    changes neither the device bytes the handle owns (fr_mesh_info) nor the device's free memory
    (cudaMemGetInfo); the allocating entry point, run afterwards, gives the same sums. A first handle
    loads the diagnostics kernel (lazy module loading may place code in device memory) and evaluates
    the RHS, so that the fresh handle does nothing before the call under test."""
    mesh = W.box_hex_mesh(4)
    o = O.Oracle(mesh, 3, 5)
    U = W.tgv_state(o.sol_coords(), [(64, 64)], perturb=1e-2)
    warm = fr.FRMesh(mesh, fr.make_params(p=3))
    Ud = torch.from_numpy(U).cuda()
    Rd = torch.empty_like(Ud)
    warm.rhs(Ud, Rd)
    warm.diagnostics_noalloc(Ud, Rd)
    m = fr.FRMesh(mesh, fr.make_params(p=3))
    torch.cuda.synchronize()
    owned0, free0 = m.info()["device_bytes"], torch.cuda.mem_get_info()[0]
    got = m.diagnostics_noalloc(Ud, Rd)[0]
    torch.cuda.synchronize()
    owned1, free1 = m.info()["device_bytes"], torch.cuda.mem_get_info()[0]
    assert owned1 == owned0, (owned0, owned1)
    assert free1 == free0, (free0, free1)
    ref = m.diagnostics(Ud, Rd)[0]
    _same(got, ref)
    _same(m.diagnostics_noalloc(Ud, Rd)[0], ref)


def test_noalloc_rejects_more_instances_than_its_scratch_holds():
    meshes = [W.box_hex_mesh(1)] * 1025
    m = fr.FRMesh(meshes, fr.make_params(p=3))
    Ud = torch.ones(m.num_values, dtype=torch.float64, device="cuda")
    with pytest.raises(fr.FRError) as e:
        m.diagnostics_noalloc(Ud)
    assert e.value.status == fr.FR_EINVAL and "1024" in str(e.value)
