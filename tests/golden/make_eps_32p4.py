"""Writes tests/golden/eps_tgv32_p4.txt: the FP64 oracle's kinetic-energy dissipation rate of the
32^3 hexahedral Taylor-Green vortex at p = 4 (6^3 Gauss-Legendre flux anti-aliasing, p_ref = p0),
at the perturbed initial state and after 100 classical RK4 steps of dt = 2e-4.

This script calls only the oracle (oracle/) and the seeded input generators
(paper_2401_06132_gb300/workloads.py, which hold no arithmetic of the method). The dissipation rate is
eps = -(1/|Omega|) sum W detJ [v . R_rho v - |v|^2/2 R_rho], evaluated by the oracle's diagnostics from
its own RHS at the state (kinetic energy E_k = <rho |v|^2 / 2>; RK4 of Sec. 3 advances du/dt = R(u)
of Sec. 2.1 with the flux anti-aliasing of Sec. 2.1.1). The run is a one-off: about an hour of FP64
dense-operator work on 8 host cores.

    python tests/golden/make_eps_32p4.py [threads]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2401_06132_gb300 import workloads as W  # noqa: E402

N, P, M, DT, STEPS, PERTURB = 32, 4, 6, 2e-4, 100, 1e-3
OUT = os.path.join(HERE, "eps_tgv32_p4.txt")


def main() -> None:
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    mesh = W.box_hex_mesh(N)
    p0 = W.tgv_p0()
    o = O.Oracle(mesh, P, M, threads=threads, p_ref=p0)
    U = W.tgv_state(o.sol_coords(), [(N ** 3, (P + 1) ** 3)], perturb=PERTURB)
    t0 = time.time()
    d0 = o.diagnostics(U, o.rhs(U))
    print(f"initial: Ek {d0['Ek']:.17e} eps {d0['eps']:.17e} ({time.time() - t0:.1f} s per RHS)", flush=True)
    chunk = 5
    for s in range(0, STEPS, chunk):
        U = o.rk4(U, DT, chunk)
        print(f"step {s + chunk}/{STEPS} at {time.time() - t0:.0f} s", flush=True)
    d1 = o.diagnostics(U, o.rhs(U))
    with open(OUT, "w") as f:
        f.write("# FP64 oracle, Taylor-Green vortex on the 32^3 periodic hexahedral box [-pi, pi]^3, p = 4\n")
        f.write("# (5^3 Gauss-Legendre solution points), 6^3 Gauss-Legendre flux anti-aliasing, M = 0.1, Re = 1600,\n")
        f.write("# Pr = 0.71, gamma = 1.4, LDG beta = 0.5, tau = 0.1, p_ref = p0; initial state = the analytic TGV at\n")
        f.write("# the oracle's solution points times (1 + 1e-3 xi), xi ~ U(-1, 1) from SplitMix64(20240111) by DOF id.\n")
        f.write("# Classical RK4 (Sec. 3), dt = 2e-4. Written by tests/golden/make_eps_32p4.py (oracle only).\n")
        f.write("# Format: steps E_k eps\n")
        f.write(f"0 {d0['Ek']:.17e} {d0['eps']:.17e}\n")
        f.write(f"{STEPS} {d1['Ek']:.17e} {d1['eps']:.17e}\n")
    print(f"final: Ek {d1['Ek']:.17e} eps {d1['eps']:.17e}; wrote {OUT} after {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
