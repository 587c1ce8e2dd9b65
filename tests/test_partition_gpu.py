"""Partitioned single-mesh RHS on one GPU: the parts of a mesh as separate handles in one process,
the two halo exchanges per RHS done by device-to-device copies (partition.local_exchange), phases run
one part after another (no kernel waits on another). The parts' R concatenated must equal the single
handle's R bit for bit (each side evaluates its own points with the pair's global L/R roles), and
the FP64 oracle to 1e-12.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_06132_gb300 import fr, partition, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_06132_gb300 import build as B
    B.build()


def _partitioned_rhs(mesh, prm, nparts, U):
    """R of the partitioned mesh, parts in one process; U is the whole mesh's state (host)."""
    parts = [fr.FRMesh.part(mesh, prm, nparts, r) for r in range(nparts)]
    rhs = [partition.PartRHS(m) for m in parts]
    Us, Rs, off = [], [], 0
    for m in parts:
        n = m.num_values
        Us.append(torch.from_numpy(np.ascontiguousarray(U[off:off + n])).cuda())
        Rs.append(torch.empty_like(Us[-1]))
        off += n
    assert off == U.size
    counts = [x.counts for x in rhs]
    # phase by phase over all parts, exchanging in between
    for ph in range(3):
        for m, u, r in zip(parts, Us, Rs):
            m.rhs_phase(ph, u, r)
        if ph < 2:
            for x in rhs:
                x.m.halo_pack(ph, x.send[ph])
            partition.local_exchange([x.send[ph] for x in rhs], [x.recv[ph] for x in rhs], counts, rhs[0].nvar[ph])
            for x in rhs:
                x.m.halo_unpack(ph, x.recv[ph])
    for m in parts:
        m.sync_status()
    return np.concatenate([r.cpu().numpy() for r in Rs]), parts


def _single_rhs(mesh, prm, U):
    m = fr.FRMesh(mesh, prm)
    Ud = torch.from_numpy(U).cuda()
    Rd = torch.empty_like(Ud)
    m.rhs(Ud, Rd)
    m.sync_status()
    return Rd.cpu().numpy()


@pytest.mark.parametrize("name,nparts", [("hex8", 2), ("hex8", 3), ("hex4p4", 2), ("mixed4", 2), ("mixed4", 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_partitioned_rhs_equals_single_handle(name, nparts, prec):
    if name == "hex8":
        mesh, p, blocks = W.box_hex_mesh(8), 3, [(512, 64)]
    elif name == "hex4p4":
        mesh, p, blocks = W.box_hex_mesh(4), 4, [(64, 125)]
    else:
        mesh, p = W.mixed_box_mesh(4), 3
        blocks = [(mesh["hex_v"].shape[0], 64), (mesh["pri_v"].shape[0], 40)]
    p0 = W.tgv_p0()
    o = O.Oracle(mesh, p, p + 2, p_ref=p0)
    U = W.tgv_state(o.sol_coords(), blocks, perturb=1e-2)
    # reduced precision in the low-Mach form (exchange 1 then carries the float-float mass flux)
    prm = fr.make_params(p=p, prec=prec, p_ref=p0, rho_ref=1.0)
    if prec == "fp32":
        U = U.astype(np.float32)
    Rp, parts = _partitioned_rhs(mesh, prm, nparts, U)
    Rs = _single_rhs(mesh, prm, U)
    assert np.array_equal(Rp, Rs), np.abs(Rp - Rs).max()
    info = parts[0].halo_info()
    assert info["nparts"] == nparts and info["nhalo"] > 0 and info["nvar"] == (5, 4 if prec == "fp64" else 6)
    if prec == "fp64":
        Ro = o.rhs(U)
        err = max((np.abs(Rp[a:b] - Ro[a:b]).max() / np.abs(Ro[a:b]).max())
                  for a, b in [(0, blocks[0][0] * 5 * blocks[0][1])])
        assert err <= 1e-12, err


def test_partitioned_handle_refuses_whole_rhs_and_rk4():
    mesh = W.box_hex_mesh(4)
    m = fr.FRMesh.part(mesh, fr.make_params(p=3), 2, 0)
    U = torch.zeros(m.num_values, dtype=torch.float64, device="cuda")
    R = torch.empty_like(U)
    with pytest.raises(fr.FRError) as e:
        m.rhs(U, R)
    assert e.value.status == fr.FR_EUNSUPPORTED
    with pytest.raises(fr.FRError) as e:
        m.rk4_step(U, 1e-3, 1)        # parts step through fr_rk4_stage with exchanges
    assert e.value.status == fr.FR_EUNSUPPORTED
    # a one-part "partition" is the whole mesh: fr_rhs_phase 0, 1, 2 equal fr_rhs
    o = O.Oracle(mesh, 3, 5)
    Uh = W.tgv_state(o.sol_coords(), [(64, 64)], perturb=1e-2)
    m1 = fr.FRMesh.part(mesh, fr.make_params(p=3), 1, 0)
    Ud = torch.from_numpy(Uh).cuda()
    R1 = torch.empty_like(Ud)
    for ph in range(3):
        m1.rhs_phase(ph, Ud, R1)
    m1.sync_status()
    assert np.array_equal(R1.cpu().numpy(), _single_rhs(mesh, fr.make_params(p=3), Uh))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_partitioned_rk4_equals_single_handle(prec):
    """Three RK4 steps of a 3-part mesh (fr_rk4_stage, halo exchanges between the phases of every
    stage) equal three fr_rk4_step steps of the single handle bit for bit, FP64 and the low-Mach FP32
    form (FP64 master state either way)."""
    mesh = W.mixed_box_mesh(4)
    p0 = W.tgv_p0()
    prm = fr.make_params(p=3, prec=prec, p_ref=p0, rho_ref=1.0)
    single = fr.FRMesh(mesh, prm)
    blocks = [(mesh["hex_v"].shape[0], 64), (mesh["pri_v"].shape[0], 40)]
    U0 = W.tgv_state(single.sol_coords(), blocks, perturb=1e-2)
    Us = torch.from_numpy(U0).cuda()
    single.rk4_step(Us, 1e-3, 3)
    single.sync_status()
    parts = [fr.FRMesh.part(mesh, prm, 3, r) for r in range(3)]
    rhs = [partition.PartRHS(m) for m in parts]
    Up, off = [], 0
    for m in parts:
        Up.append(torch.from_numpy(np.ascontiguousarray(U0[off:off + m.num_values])).cuda())
        off += m.num_values
    counts = [x.counts for x in rhs]
    for _ in range(3):
        for st in range(4):
            for ph in range(3):
                for m, u in zip(parts, Up):
                    m.rk4_stage(st, ph, u, 1e-3)
                if ph < 2:
                    for x in rhs:
                        x.m.halo_pack(ph, x.send[ph])
                    partition.local_exchange([x.send[ph] for x in rhs], [x.recv[ph] for x in rhs], counts,
                                             rhs[0].nvar[ph])
                    for x in rhs:
                        x.m.halo_unpack(ph, x.recv[ph])
    for m in parts:
        m.sync_status()
    assert torch.equal(torch.cat(Up), Us)
