"""Run one Taylor-Green configuration through the library and report timings.

    python -m paper_2401_06132_gb300.run_case --n 48 --p 3 --prec fp32 --form fused --rhs 4 --rk4 2

Used as the command under Nsight Compute captures of single kernels, and as a quick check of a
configuration. Every evaluation goes through the C ABI (libfrgb300.so).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=16, help="elements per box edge")
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--nq", type=int, default=0, help="1D quadrature points (0: p + 2; p + 1: no anti-aliasing)")
    ap.add_argument("--mesh", default="hex", choices=["hex", "sheared", "mixed", "tet", "tetshear", "pyr", "hexpyr"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "mixed_fp16", "mixed_bf16"])
    ap.add_argument("--lowmach", type=int, default=1, help="FP32 low-Mach form (rho_ref = 1)")
    ap.add_argument("--form", default="fused", choices=["fused", "unfused"])
    ap.add_argument("--rhs", type=int, default=3, help="RHS evaluations")
    ap.add_argument("--rk4", type=int, default=0, help="RK4 steps after the RHS evaluations")
    ap.add_argument("--mach", type=float, default=0.1)
    ap.add_argument("--autotune", type=int, default=0, help="run the launch-shape autotuner first")
    ap.add_argument("--hex-tc", type=int, default=0, help="mixed forms: hexahedral plane contractions on the tensor cores")
    ap.add_argument("--dense-tc", type=int, default=0, help="mixed forms: tetrahedral / pyramidal interpolation on the tensor cores")
    ap.add_argument("--surf", type=int, default=0, help="surface-flux anti-aliasing as well (full anti-aliasing)")
    ap.add_argument("--timing", type=int, default=0, help="per-kernel times (CUDA events) of one more RHS")
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    from paper_2401_06132_gb300 import fr, workloads as W

    mesh = {"hex": W.box_hex_mesh, "sheared": W.sheared_box_mesh, "mixed": W.mixed_box_mesh, "tet": W.box_tet_mesh,
            "tetshear": lambda n: W.box_tet_mesh(n, shear=True), "pyr": W.box_pyr_mesh,
            "hexpyr": lambda n: W.box_pyr_mesh(n, hex_below=n // 2)}[args.mesh](args.n)
    p0 = W.tgv_p0(mach=args.mach)
    m = fr.FRMesh(mesh, fr.make_params(p=args.p, nq1d=args.nq, prec=args.prec, p_ref=p0,
                                       rho_ref=1.0 if args.lowmach else 0.0, surface_aa=bool(args.surf)))
    m.set_form(args.form)
    m.set_hex_tensor_cores(bool(args.hex_tc))
    m.set_dense_tensor_cores(bool(args.dense_tc))
    blocks = []
    if mesh["hex_v"].shape[0]:
        blocks.append((mesh["hex_v"].shape[0], (args.p + 1) ** 3))
    if mesh["pri_v"].shape[0]:
        blocks.append((mesh["pri_v"].shape[0], 40))
    if mesh.get("tet_v") is not None and mesh["tet_v"].shape[0]:
        blocks.append((mesh["tet_v"].shape[0], 20))
    if mesh.get("pyr_v") is not None and mesh["pyr_v"].shape[0]:
        blocks.append((mesh["pyr_v"].shape[0], 30))
    U0 = W.tgv_state(m.sol_coords(), blocks, mach=args.mach, perturb=1e-3)
    U = torch.from_numpy(U0.astype(np.float64 if args.prec == "fp64" else np.float32)).cuda()
    R = torch.empty_like(U)
    tuned = m.autotune(U, R) if args.autotune else None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(args.rhs):
        m.rhs(U, R)
    ev[1].record()
    torch.cuda.synchronize()
    m.sync_status()
    out = {"dof": int(U0.size), "rhs_ms": ev[0].elapsed_time(ev[1]) / max(1, args.rhs), "volume_threads": tuned}
    if args.timing:
        m.set_timing(True)
        m.rhs(U, R)
        torch.cuda.synchronize()
        out["kernel_ms"] = {str(k): round(v[0] / max(1, v[1]), 4) for k, v in m.kernel_times().items()}
        m.set_timing(False)
    if args.rk4:
        Um = torch.from_numpy(U0).cuda()
        m.rk4_step(Um, 2e-4, 1)   # warm-up (and graph capture)
        ev[0].record()
        m.rk4_step(Um, 2e-4, args.rk4)
        ev[1].record()
        torch.cuda.synchronize()
        m.sync_status()
        out["rk4_ms"] = ev[0].elapsed_time(ev[1]) / args.rk4
        out["gdof_rhs_per_s_rk4"] = U0.size * 4 / (out["rk4_ms"] * 1e-3) / 1e9
        if args.timing:
            m.set_timing(True)
            m.rk4_step(Um, 2e-4, 1)
            torch.cuda.synchronize()
            out["rk4_kernel_ms"] = {str(k): round(v[0] / max(1, v[1]), 4) for k, v in m.kernel_times().items()}
            m.set_timing(False)
    out["gdof_rhs_per_s"] = out["dof"] / (out["rhs_ms"] * 1e-3) / 1e9
    print(json.dumps(out))


if __name__ == "__main__":
    main()
