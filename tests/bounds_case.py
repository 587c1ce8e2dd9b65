"""Runs a fixed set of RHS and RK4 evaluations through the library that FR_LIBRARY selects and saves
the results (used by test_bounds_build.py, which runs it once per library in a fresh process)."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2401_06132_gb300 import fr, partition, workloads as W  # noqa: E402


def _rhs(mesh, prm, blocks, dtype=np.float64, perturb=1e-2):
    m = fr.FRMesh(mesh, prm)
    U = W.tgv_state(m.sol_coords(), blocks, perturb=perturb).astype(dtype)
    Ud = torch.from_numpy(U).cuda()
    Rd = torch.empty_like(Ud)
    m.rhs(Ud, Rd)
    m.sync_status()
    return Rd.cpu().numpy()


def main(out):
    p0 = W.tgv_p0()
    res = {}
    res["hex3_fp64"] = _rhs(W.box_hex_mesh(4), fr.make_params(p=3, p_ref=p0), [(64, 64)])
    res["hex4_fp64"] = _rhs(W.sheared_box_mesh(3), fr.make_params(p=4, p_ref=p0), [(27, 125)])
    res["hex3_fp32"] = _rhs(W.box_hex_mesh(4), fr.make_params(p=3, prec="fp32", p_ref=p0, rho_ref=1.0), [(64, 64)],
                            np.float32)
    mm = W.mixed_box_mesh(2)
    mb = [(mm["hex_v"].shape[0], 64), (mm["pri_v"].shape[0], 40)]
    res["mixed_fp64"] = _rhs(mm, fr.make_params(p=3, p_ref=p0), mb)
    res["mixed_fp16"] = _rhs(mm, fr.make_params(p=3, prec="mixed_fp16", p_ref=p0, rho_ref=1.0), mb, np.float32)
    tm = W.box_tet_mesh(2)
    res["tet_fp64"] = _rhs(tm, fr.make_params(p=3, p_ref=p0), [(tm["tet_v"].shape[0], 20)])
    ym = W.box_pyr_mesh(2)
    res["pyr_fp32"] = _rhs(ym, fr.make_params(p=3, prec="fp32", p_ref=p0, rho_ref=1.0), [(ym["pyr_v"].shape[0], 30)],
                           np.float32)
    res["curved_fp64"] = _rhs(W.curved_box_mesh(3), fr.make_params(p=3, p_ref=p0), [(27, 64)])
    # an ensemble (per-element offsets) over RK4 steps (graph replay, stage updates folded in)
    meshes = [W.box_hex_mesh(2), W.box_hex_mesh(3)]
    prms = [fr.make_params(p=3, p_ref=p0), fr.make_params(p=4, p_ref=p0)]
    m = fr.FRMesh(meshes, prms)
    off = m.instance_offsets()
    xyz = m.sol_coords()
    U = np.concatenate([W.tgv_state(xyz[off[i] // 5:off[i + 1] // 5], [(mh["hex_v"].shape[0], (p + 1) ** 3)],
                                    perturb=1e-2) for i, (mh, p) in enumerate(zip(meshes, (3, 4)))])
    Ud = torch.from_numpy(U).cuda()
    m.rk4_step(Ud, 1e-3, 3)
    m.sync_status()
    res["ensemble_rk4"] = Ud.cpu().numpy()
    # a partitioned mesh (halo slots, per-phase launches)
    mesh = W.box_hex_mesh(4)
    prm = fr.make_params(p=3, p_ref=p0)
    parts = [fr.FRMesh.part(mesh, prm, 2, r) for r in range(2)]
    pr = [partition.PartRHS(x) for x in parts]
    Us, Rs = [], []
    for x in parts:
        u = W.tgv_state(x.sol_coords(), [(x.info()["elements"], 64)], perturb=1e-2)
        Us.append(torch.from_numpy(u).cuda())
        Rs.append(torch.empty_like(Us[-1]))
    for ph in range(3):
        for x, u, r in zip(parts, Us, Rs):
            x.rhs_phase(ph, u, r)
        if ph < 2:
            for y in pr:
                y.m.halo_pack(ph, y.send[ph])
            partition.local_exchange([y.send[ph] for y in pr], [y.recv[ph] for y in pr], [y.counts for y in pr],
                                     pr[0].nvar[ph])
            for y in pr:
                y.m.halo_unpack(ph, y.recv[ph])
    for x in parts:
        x.sync_status()
    res["partitioned"] = np.concatenate([r.cpu().numpy() for r in Rs])
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
