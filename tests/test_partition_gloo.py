"""The partitioned single-mesh exchange on CPU: gloo ranks, no GPU.

Each rank asks the library for its exchange plan (fr_partition_plan, host only), packs the face
data of its own flux points that its peers need into the library's buffer layout, exchanges the
buffers with partition.dist_exchange (the same function the NCCL path uses), and checks what it
received against the single-rank oracle: the halo slots must hold, bit for bit, the face solution
and face gradient of exactly the remote partners of its boundary flux points -- the neighbour data
the paper's kernel groups need at their two boundaries (U^(f) before con_u, face data before
comm_flux). The device path with the same plan is checked against the single handle on the GPU.
"""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_06132_gb300 import fr, partition, workloads as W

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

NVAR = 20   # 5 face-solution values + 15 face-gradient values per flux point


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _mesh(name):
    return W.box_hex_mesh(4) if name == "hex4" else W.mixed_box_mesh(4)


def _face_table(mesh, o, U):
    """[global flux point][20] oracle face solution and gradient; the oracle's stage arrays are
    element by element [elem][comp][local flux point], hexahedra (96 points) before prisms (68)."""
    st = o.rhs_stages(U)
    rows = []
    ou, oq = 0, 0
    for ne, nf in ((mesh["hex_v"].shape[0], 96), (mesh["pri_v"].shape[0], 68)):
        uf = st["uf"][ou:ou + ne * 5 * nf].reshape(ne, 5, nf).transpose(0, 2, 1)
        qf = st["qf"][oq:oq + ne * 15 * nf].reshape(ne, 15, nf).transpose(0, 2, 1)
        rows.append(np.concatenate([uf, qf], axis=2).reshape(ne * nf, NVAR))
        ou += ne * 5 * nf
        oq += ne * 15 * nf
    return np.concatenate(rows)


def _worker(rank, world, port, name, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh = _mesh(name)
        prm = fr.make_params(p=3)
        plan = fr.partition_plan(mesh, prm, world, rank)
        o = O.Oracle(mesh, 3, 5)
        blocks = [(mesh["hex_v"].shape[0], 64), (mesh["pri_v"].shape[0], 40)]
        U = W.tgv_state(o.sol_coords(), [b for b in blocks if b[0]], perturb=1e-2)
        V = _face_table(mesh, o, U)
        counts = plan["counts"]
        segs = partition.segments(counts, NVAR, rank)
        send = torch.zeros(max(1, NVAR * plan["nhalo"]), dtype=torch.float64)
        recv = torch.full_like(send, float("nan"))
        off = np.concatenate([[0], np.cumsum(counts)])
        for qq, s, n in segs:
            pts = plan["send"][off[qq]:off[qq + 1]]
            send[s:s + n] = torch.from_numpy(np.ascontiguousarray(V[pts].T).reshape(-1))
        partition.dist_exchange(send, recv, counts, NVAR, rank)
        ok_vals = True
        for qq, s, n in segs:
            pts = plan["recv"][off[qq]:off[qq + 1]]
            got = recv[s:s + n].numpy().reshape(NVAR, -1).T
            ok_vals &= np.array_equal(got, V[pts])
        # the halo is exactly the set of remote partners of the own flux points
        L, R = o.pairs()
        partner = np.empty(V.shape[0], dtype=np.int64)
        partner[L], partner[R] = R, L
        e0, e1 = plan["elements"]
        nh = mesh["hex_v"].shape[0]
        own = np.concatenate([np.arange(96 * e, 96 * (e + 1)) if e < nh else
                              np.arange(96 * nh + 68 * (e - nh), 96 * nh + 68 * (e - nh + 1)) for e in range(e0, e1)])
        own_set = set(own.tolist())
        remote = {int(g) for g in own if int(partner[g]) not in own_set}
        ok_sets = (set(plan["send"].tolist()) == remote and
                   set(plan["recv"].tolist()) == {int(partner[g]) for g in remote} and
                   len(plan["send"]) == len(remote) == plan["nhalo"] and plan["nfpt_own"] == len(own))
        ranges = [None] * world
        dist.all_gather_object(ranges, (e0, e1))
        q.put((rank, bool(ok_vals), bool(ok_sets), ranges, plan["ne_total"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("hex4", 2), ("hex4", 3), ("mixed4", 2)])
def test_partition_exchange_delivers_the_partners_face_data(name, world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok_vals, ok_sets, ranges, ne in res:
        assert ok_vals, f"rank {rank}: received face data differ from the partners' oracle values"
        assert ok_sets, f"rank {rank}: halo is not the set of remote partners"
        assert ranges[0][0] == 0 and ranges[-1][1] == ne
        assert all(ranges[i][1] == ranges[i + 1][0] and ranges[i][1] > ranges[i][0] for i in range(world - 1))


def test_partition_plan_counts_are_symmetric():
    """Every pair of parts exchanges the same number of points in both directions, and a single
    part has no halo."""
    mesh = W.mixed_box_mesh(4)
    prm = fr.make_params(p=3)
    for nparts in (1, 2, 3, 5):
        plans = [fr.partition_plan(mesh, prm, nparts, r) for r in range(nparts)]
        for r in range(nparts):
            assert plans[r]["counts"][r] == 0
            for q2 in range(nparts):
                assert plans[r]["counts"][q2] == plans[q2]["counts"][r]
        if nparts == 1:
            assert plans[0]["nhalo"] == 0


def test_partition_plan_rejects_bad_arguments():
    mesh = W.box_hex_mesh(2)
    with pytest.raises(fr.FRError):
        fr.partition_plan(mesh, fr.make_params(p=3), 2, 2)
    with pytest.raises(fr.FRError):
        fr.partition_plan(mesh, fr.make_params(p=3), 9, 0)      # 8 elements cannot fill 9 parts
    with pytest.raises(fr.FRError):
        fr.partition_plan(mesh, fr.make_params(p=3, surface_aa=True), 2, 0)
