"""Benchmark: anti-aliased Navier-Stokes FR right-hand-side throughput on the Taylor-Green vortex.

Workload (default): 48^3 periodic hex box, p = 3 (4^3 Gauss-Legendre solution points), flux
anti-aliasing on 5^3 Gauss-Legendre quadrature points, FP64, Re = 1600, M = 0.1, Pr = 0.71,
Rusanov + LDG (beta = 0.5, tau = 0.1) interface fluxes, synthetic TGV state with a 1e-3 SplitMix64
perturbation. One step = one classical RK4 step = 4 RHS evaluations + 4 stage updates (every step
of the hot path). Metric: GDOF.RHS/s = DOF x RHS evaluations / s, DOF = elements x points x 5.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NS-FR RHS GDOF/s (anti-aliased TGV), % HBM roofline, fused vs unfused"
UNIT = "GDOF*RHS/s"
N_EDGE, P, MQ = 48, 3, 5
DT = 2e-4
RHS_PER_STEP = 4
FR_NV_DOF_PER_ELEMENT = 5 * (P + 1) ** 3


def workload_name(n=N_EDGE, p=P, m=MQ):
    return f"TGV {n}^3 hex p={p} ({p + 1}^3 GL solution pts), {m}^3 GL flux anti-aliasing, RK4 step = 4 RHS"


# FP64 peak of the chip from its unit counts and clock: 152 SMs x 2 FP64 FMA/clock x 2 FLOP x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + written) per element of one FP64 volume-kernel launch, from one Nsight Compute
# capture of that kernel on the 40^3 p = 3 box (859.1 MB / 64,000 elements; the 164 MB state is
# larger than L2); the kernel touches each element's inputs and outputs once, so a launch's traffic
# scales with its element count
VOLUME_FP64_DRAM_BYTES_PER_ELEMENT = 859.063808e6 / 64000

# ---------------------------------------------------------------------------------------------
# FLOP model of the fused volume kernel (phase B), FMA = 2 FLOP; counted from its arithmetic
# ---------------------------------------------------------------------------------------------
VISC_NORMAL_FLOPS = 130   # viscous normal flux at one face point (velocity gradients, stress, heat, n.)
POINT_FLUX_FLOPS = 150    # total flux f^e - f^v at one quadrature point
TRANSFORM_FLOPS = 15      # detJ J^-1 f with a diagonal metric: 15 products (90 with a full 3 x 3)


def phase_b_flops_per_element(p=P, m=MQ, one_sided=True, diagonal_metric=True, divergence_in_projection=True):
    """FLOPs of the volume kernel per element. With beta = +-1/2 the LDG viscous flux needs only the
    weighted side, i.e. half of the flux points on average (one_sided); axis-aligned elements apply
    the metric as 3 products instead of 3 x 3 (diagonal_metric); the corrected divergence rides on
    the projection's sweeps (Dh Pj in place of Pj along each flux component's own direction), so it
    costs no separate sweep (divergence_in_projection)."""
    n = p + 1
    nu, nf, nq = n ** 3, 6 * n * n, m ** 3
    con_u = 5 * nf * 3
    grad = 15 * n * n * n * (2 * n + 3)
    jt = 5 * nu * (3 if diagonal_metric else 15)
    face = (nf // 2 if one_sided else nf) * (20 * 2 * n + VISC_NORMAL_FLOPS)
    interp = 20 * 2 * (n ** 3 * m + n * n * m * m + n * m ** 3)
    tdisf = nq * (POINT_FLUX_FLOPS + TRANSFORM_FLOPS)
    proj = 15 * 2 * (m ** 3 * n + m * m * n * n + m * n ** 3)
    div = 0 if divergence_in_projection else 5 * nu * 3 * n * 2
    return con_u + grad + jt + face + interp + tdisf + proj + div


def tet_phase_b_flops_per_element(nu=20, nf=40, nfaces=4):
    """FLOPs of the dense-element volume kernel per element (p = 3; tetrahedron: 20 solution points,
    40 flux points, 4 faces; pyramid: 30, 56, 5; 125 quadrature points; dense operators, full
    metric, one-sided viscous flux, the divergence folded into the projection as one nu x 375
    operator per variable)."""
    nq = 125
    con_u = 5 * nf * 3
    grad = 3 * nu * nu * 5 * 2 + nf * nu * 5 * 2 + nfaces * 3 * 5 * nu * 2   # Dh u, face lifts, normals
    jt = 5 * nu * 15
    face = (nf // 2) * (20 * nu * 2 + VISC_NORMAL_FLOPS)
    interp = 20 * nq * nu * 2
    tdisf = nq * (POINT_FLUX_FLOPS + 90)
    proj = 5 * nu * 3 * nq * 2
    return con_u + grad + jt + face + interp + tdisf + proj


# ---------------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------------------------
def oracle_sample(seconds=12.0, n_edge=16, threads=None):
    """Oracle RHS evaluations on an n_edge^3 box with the same order, quadrature and physics as the
    workload (same per-element work), repeated for about `seconds`."""
    import numpy as np

    from oracle import oracle as O
    from paper_2401_06132_gb300 import workloads as W
    threads = threads or os.cpu_count() or 1
    mesh = W.box_hex_mesh(n_edge)
    o = O.Oracle(mesh, P, MQ, threads=threads, p_ref=W.tgv_p0())
    U = W.tgv_state(o.sol_coords(), [(n_edge ** 3, (P + 1) ** 3)], perturb=1e-3)
    o.rhs(U)
    t0 = time.perf_counter()
    reps = 0
    while True:
        o.rhs(U)
        reps += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return dict(value=U.size * reps / dt / 1e9, unit=UNIT, cores=threads, kind="oracle",
                sample=f"{reps} oracle RHS evaluations on the {n_edge}^3 box (same p, quadrature, physics; "
                       f"{np.prod(U.shape)} DOF each), {dt:.1f} s, OpenMP over elements"), U.size


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2401_06132_gb300 import workloads as W
    threads = os.cpu_count() or 1
    n_edge = 12
    mesh = W.box_hex_mesh(n_edge)
    o = O.Oracle(mesh, P, MQ, threads=threads, p_ref=W.tgv_p0())
    U = W.tgv_state(o.sol_coords(), [(n_edge ** 3, (P + 1) ** 3)], perturb=1e-3)
    for _ in range(args.warmup):
        U = o.rk4(U, DT, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = o.rk4(U, DT, 1)
    dt = time.perf_counter() - t0
    value = U.size * RHS_PER_STEP * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(), "sample": f"oracle on the {n_edge}^3 box, same per-element work"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} oracle RK4 steps on the {n_edge}^3 box ({U.size} DOF)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def time_rk4(m, U, steps, warmup, torch):
    for _ in range(warmup):
        m.rk4_step(U, DT, 1)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        m.rk4_step(U, DT, 1)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _time_steps(m, U, steps, warmup, torch):
    Uc = U if m.prec == 0 else U.float()
    m.autotune(Uc, torch.empty_like(Uc))
    del Uc
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(warmup):
            m.rk4_step(U, DT, 1)
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        m.rk4_step(U, DT, steps)     # one captured CUDA graph per RK4 step
        e1.record(s)
        s.synchronize()
    return e0.elapsed_time(e1) / steps


def rhs_error(m64, mred, U0, blocks, torch):
    """Max per-variable relative L-inf error of a reduced-precision RHS: |R_red - R_64| over all
    points of the blocks [(first value, elements, points per element)], divided by max |R_64|, per
    conserved variable (blocks of one instance share the normalisation; the maximum over instances
    is returned). Both RHS are evaluated on the FP32-rounded state; R_64 is the FP64 GPU form, which
    the parity tests pin to the FP64 oracle at 1e-12."""
    U32 = torch.from_numpy(U0.astype(np.float32)).cuda()
    U64 = U32.double()
    R64, R32 = torch.empty_like(U64), torch.empty_like(U32)
    m64.rhs(U64, R64)
    mred.rhs(U32, R32)
    m64.sync_status()
    mred.sync_status()
    a, b = R32.double().cpu().numpy(), R64.cpu().numpy()
    worst = 0.0
    for inst in blocks:
        d, sc = np.zeros(5), np.zeros(5)
        for off, ne, nu in inst:
            x = a[off:off + ne * 5 * nu].reshape(ne, 5, nu)
            y = b[off:off + ne * 5 * nu].reshape(ne, 5, nu)
            d = np.maximum(d, np.abs(x - y).max(axis=(0, 2)))
            sc = np.maximum(sc, np.abs(y).max(axis=(0, 2)))
        worst = max(worst, float((d / sc).max()))
    return {"rhs_err_vs_fp64": worst, "within_2e-5": worst <= 2e-5}


def other_configs(args, torch, fr, W):
    """Mixed hex/prism TGV (40^3 box: 32,000 hexes + 64,000 prisms, p = 3), the 48^3 TGV without
    anti-aliasing and with full (flux + surface-flux) anti-aliasing, a tetrahedral and a pyramidal TGV
    box, a curved (trilinear) hexahedral TGV box, and the batched ensemble
    of 64 TGV instances (edges in {8,...,24}, p in {3,4}, M in [0.05,0.2], Re in [400,3200] from
    SplitMix64(20240111)), each timed over RK4 steps on a side stream (CUDA-graph replay)."""
    out = {}
    steps = 3
    mesh = W.mixed_box_mesh(40)
    p0 = W.tgv_p0()
    blocks = [(mesh["hex_v"].shape[0], 64), (mesh["pri_v"].shape[0], 40)]
    eb = [[(0, blocks[0][0], 64), (blocks[0][0] * 5 * 64, blocks[1][0], 40)]]
    m64 = None
    for prec in ("fp64", "fp32", "mixed_fp16", "mixed_bf16"):
        # reduced precisions in the low-Mach form (rho_ref = 1; FP64 ignores it)
        m = fr.FRMesh(mesh, fr.make_params(p=3, prec=prec, p_ref=p0, rho_ref=1.0))
        U0 = W.tgv_state(m.sol_coords(), blocks, perturb=1e-3)
        U = torch.from_numpy(U0).cuda()
        ms = _time_steps(m, U, steps, 2, torch)
        m.sync_status()
        out[f"mixed40_{prec}"] = {"gdof_rhs_per_s": U0.size * RHS_PER_STEP / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                                  "dof": int(U0.size), "elements": sum(b[0] for b in blocks)}
        if prec != "fp64":
            out[f"mixed40_{prec}"]["speedup_vs_fp64"] = out["mixed40_fp64"]["ms_per_step"] / ms
            out[f"mixed40_{prec}"].update(rhs_error(m64, m, U0, eb, torch))
            m.close()
        else:
            m64 = m
        del U
    m64.close()
    # the same 48^3 p = 3 TGV without flux anti-aliasing (flux at the solution points), the paper's
    # "AA off" discretisation, FP64 and FP32 low-Mach
    mesh48 = W.box_hex_mesh(N_EDGE)
    eb48 = [[(0, N_EDGE ** 3, (P + 1) ** 3)]]
    for prec in ("fp64", "fp32"):
        m = fr.FRMesh(mesh48, fr.make_params(p=P, nq1d=P + 1, prec=prec, p_ref=p0, rho_ref=1.0))
        U0 = W.tgv_state(m.sol_coords(), [(N_EDGE ** 3, (P + 1) ** 3)], perturb=1e-3)
        U = torch.from_numpy(U0).cuda()
        ms = _time_steps(m, U, steps, 2, torch)
        m.sync_status()
        out[f"aa_off48_{prec}"] = {"gdof_rhs_per_s": U0.size * RHS_PER_STEP / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                                   "dof": int(U0.size), "elements": N_EDGE ** 3}
        if prec == "fp64":
            m64 = m
        else:
            out[f"aa_off48_{prec}"].update(rhs_error(m64, m, U0, eb48, torch))
            m.close()
            m64.close()
        del U
    # ... and with full anti-aliasing (flux + surface flux), FP64 and the low-Mach FP32 form
    for prec in ("fp64", "fp32"):
        m = fr.FRMesh(mesh48, fr.make_params(p=P, prec=prec, p_ref=p0, rho_ref=1.0, surface_aa=True))
        U0 = W.tgv_state(m.sol_coords(), [(N_EDGE ** 3, (P + 1) ** 3)], perturb=1e-3)
        U = torch.from_numpy(U0).cuda()
        ms = _time_steps(m, U, steps, 2, torch)
        m.sync_status()
        out[f"aa_full48_{prec}"] = {"gdof_rhs_per_s": U0.size * RHS_PER_STEP / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                                    "dof": int(U0.size), "elements": N_EDGE ** 3}
        if prec == "fp64":
            m64 = m
        else:   # the low-Mach FP32 form (FP64 ignores rho_ref)
            out[f"aa_full48_{prec}"].update(rhs_error(m64, m, U0, eb48, torch))
            m.close()
            m64.close()
        del U
    # tetrahedra: the 24^3 box split into 82,944 Kuhn tetrahedra (p = 3, dense operators, collapsed
    # 5^3 quadrature), FP64, FP32 and the mixed FP16 form with the interpolation on the tensor cores
    # (reduced precisions in the low-Mach form: rho_ref = 1; FP64 ignores it)
    mesh_t = W.box_tet_mesh(24)
    nt = mesh_t["tet_v"].shape[0]
    for name, prec in (("fp64", "fp64"), ("fp32", "fp32"), ("mixed_fp16_tc", "mixed_fp16")):
        m = fr.FRMesh(mesh_t, fr.make_params(p=3, prec=prec, p_ref=p0, rho_ref=1.0))
        m.set_dense_tensor_cores(prec == "mixed_fp16")
        U0 = W.tgv_state(m.sol_coords(), [(nt, 20)], perturb=1e-3)
        U = torch.from_numpy(U0).cuda()
        ms = _time_steps(m, U, steps, 2, torch)
        m.sync_status()
        out[f"tet24_{name}"] = {"gdof_rhs_per_s": U0.size * RHS_PER_STEP / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                                "dof": int(U0.size), "elements": nt}
        # the volume kernel alone (CUDA events around its launches in one RHS)
        Uc = U if prec == "fp64" else U.float()
        Rc = torch.empty_like(Uc)
        m.set_timing(True)
        m.rhs(Uc, Rc)
        torch.cuda.synchronize()
        m.set_timing(False)
        kt = m.kernel_times()
        b_ms = kt[1][0] / max(1, kt[1][1])
        tfl = tet_phase_b_flops_per_element() * nt / (b_ms * 1e-3) / 1e12
        out[f"tet24_{name}"].update({"volume_kernel_ms": b_ms, "volume_tflops": tfl,
                                     "flops_per_element": tet_phase_b_flops_per_element()})
        if prec == "fp64":
            out[f"tet24_{name}"]["volume_frac_of_fp64_peak"] = tfl / FP64_PEAK_TFLOPS
        del Uc, Rc
        if prec != "fp64":
            out[f"tet24_{name}"]["speedup_vs_fp64"] = out["tet24_fp64"]["ms_per_step"] / ms
            out[f"tet24_{name}"].update(rhs_error(m64, m, U0, [[(0, nt, 20)]], torch))
            m.close()
        else:
            m64 = m
        del U
    # curved (trilinear) hexahedra, 48^3 p = 3: metric terms at every point; fused FP64 and the
    # low-Mach FP32 form, and the unfused FP64 form
    m64.close()
    mesh_c = W.curved_box_mesh(N_EDGE)
    for name, prec, form in (("fp64", "fp64", "fused"), ("fp32", "fp32", "fused"), ("unfused_fp64", "fp64", "unfused")):
        m = fr.FRMesh(mesh_c, fr.make_params(p=P, prec=prec, p_ref=p0, rho_ref=1.0))
        m.set_form(form)
        U0 = W.tgv_state(m.sol_coords(), [(N_EDGE ** 3, (P + 1) ** 3)], perturb=1e-3)
        U = torch.from_numpy(U0).cuda()
        ms = _time_steps(m, U, steps, 2, torch)
        m.sync_status()
        out[f"curved48_{name}"] = {"gdof_rhs_per_s": U0.size * RHS_PER_STEP / (ms * 1e-3) / 1e9,
                                   "ms_per_step": ms, "dof": int(U0.size), "elements": N_EDGE ** 3}
        if name == "fp64":
            m64 = m
        else:
            if name == "fp32":   # the low-Mach FP32 form (FP64 ignores rho_ref)
                out[f"curved48_{name}"].update(rhs_error(m64, m, U0, eb48, torch))
            m.close()
        del U
        torch.cuda.empty_cache()
    m64.close()
    # pyramids: the 20^3 box, every cell split into six pyramids (48,000 pyramids, 7.2M DOF)
    mesh_y = W.box_pyr_mesh(20)
    ny = mesh_y["pyr_v"].shape[0]
    fl_y = tet_phase_b_flops_per_element(30, 56, 5)
    for prec in ("fp64", "fp32"):
        m = fr.FRMesh(mesh_y, fr.make_params(p=3, prec=prec, p_ref=p0, rho_ref=1.0))
        U0 = W.tgv_state(m.sol_coords(), [(ny, 30)], perturb=1e-3)
        U = torch.from_numpy(U0).cuda()
        ms = _time_steps(m, U, steps, 2, torch)
        m.sync_status()
        Uc = U if prec == "fp64" else U.float()
        Rc = torch.empty_like(Uc)
        m.set_timing(True)
        m.rhs(Uc, Rc)
        torch.cuda.synchronize()
        m.set_timing(False)
        kt = m.kernel_times()
        b_ms = kt[1][0] / max(1, kt[1][1])
        out[f"pyr20_{prec}"] = {"gdof_rhs_per_s": U0.size * RHS_PER_STEP / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                                "dof": int(U0.size), "elements": ny, "volume_kernel_ms": b_ms,
                                "volume_tflops": fl_y * ny / (b_ms * 1e-3) / 1e12, "flops_per_element": fl_y}
        del Uc, Rc
        if prec == "fp64":
            out["pyr20_fp64"]["volume_frac_of_fp64_peak"] = out["pyr20_fp64"]["volume_tflops"] / FP64_PEAK_TFLOPS
            m64 = m
        else:
            out[f"pyr20_{prec}"]["speedup_vs_fp64"] = out["pyr20_fp64"]["ms_per_step"] / ms
            out[f"pyr20_{prec}"].update(rhs_error(m64, m, U0, [[(0, ny, 30)]], torch))
            m.close()
            m64.close()
        del U
    draws = W.ensemble_draws(64)
    meshes = [W.box_hex_mesh(d["edge"]) for d in draws]
    for prec in ("fp64", "fp32"):
        params = [fr.make_params(p=d["p"], mu=1.0 / d["re"], prec=prec, p_ref=W.tgv_p0(mach=d["mach"]), rho_ref=1.0)
                  for d in draws]
        m = fr.FRMesh(meshes, params)
        xyz = m.sol_coords()
        off = m.instance_offsets()
        parts = []
        for i, d in enumerate(draws):
            npts = (off[i + 1] - off[i]) // 5
            base = off[i] // 5
            parts.append(W.tgv_state(xyz[base:base + npts], [(d["edge"] ** 3, (d["p"] + 1) ** 3)], mach=d["mach"],
                                     perturb=1e-3, dof_offset=off[i]))
        U0 = np.concatenate(parts)
        U = torch.from_numpy(U0).cuda()
        ms = _time_steps(m, U, steps, 2, torch)
        m.sync_status()
        info = m.info()
        out[f"ensemble64_{prec}"] = {"gdof_rhs_per_s": U0.size * RHS_PER_STEP / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                                     "dof": int(U0.size), "elements": int(info["elements"]),
                                     "launches_per_rhs": int(info["launches_per_rhs"])}
        if prec != "fp64":
            out[f"ensemble64_{prec}"]["speedup_vs_fp64"] = out["ensemble64_fp64"]["ms_per_step"] / ms
            eb = [[(int(off[i]), d["edge"] ** 3, (d["p"] + 1) ** 3)] for i, d in enumerate(draws)]
            out[f"ensemble64_{prec}"].update(rhs_error(m64, m, U0, eb, torch))
            m.close()
            m64.close()
        else:
            m64 = m
        del U
        torch.cuda.empty_cache()
    return out


def run_partitioned(args, rank, world):
    """The 48^3 mesh split into `world` z slabs, one per GPU: every RHS evaluation of the RK4 step
    runs phase A, a halo exchange of the face solution, phase B, an exchange of the face viscous flux,
    phase C with the stage update (fr_rk4_stage; partition.py, NCCL send/recv under torchrun). A step
    is one RK4 step (4 RHS), as in the default mode; strong scaling: the whole mesh is the same for
    every N."""
    import torch

    from paper_2401_06132_gb300 import build as B
    from paper_2401_06132_gb300 import fr, partition, replicas, workloads as W

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    mesh = W.box_hex_mesh(N_EDGE)
    prm = fr.make_params(p=P, prec="fp64", p_ref=W.tgv_p0())
    m = fr.FRMesh.part(mesh, prm, world, rank)
    info = m.halo_info()
    e0, _ = info["elements"]
    U0 = W.tgv_state(m.sol_coords(), [(m.info()["elements"], (P + 1) ** 3)], perturb=1e-3,
                     dof_offset=e0 * FR_NV_DOF_PER_ELEMENT)
    U = torch.from_numpy(U0).cuda()
    pr = partition.PartRHS(m)

    def exchange(what):
        if world > 1:
            partition.dist_exchange(pr.send[what], pr.recv[what], pr.counts, pr.nvar[what], rank)

    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            pr.rk4_step(U, DT, exchange)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0v, e1v = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0v.record(s)
            for _ in range(args.steps):
                pr.rk4_step(U, DT, exchange)
            e1v.record(s)
            torch.cuda.synchronize()
    m.sync_status(stream=s)
    ms = replicas.max_over_ranks(e0v.elapsed_time(e1v) / args.steps, device="cuda")
    dof_total = N_EDGE ** 3 * FR_NV_DOF_PER_ELEMENT
    if rank != 0:
        return
    value = dof_total * RHS_PER_STEP / (ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(), "mode": "partitioned single mesh (z slabs)",
                       "parallelism": f"{world} parts, 2 halo exchanges per RHS", "halo_points": info["nhalo"],
                       "l2": "inputs larger than L2 (283 MB FP64 state, 129 MB L2)"},
            # per RHS: 3 phases, and a pack and an unpack per exchange and peer; the FP64 stage update is
            # folded into phase C
            "gpu_launches": RHS_PER_STEP * (3 + 4 * sum(1 for c in info["counts"] if c)) * args.steps,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_2401_06132_gb300 import build as B
    from paper_2401_06132_gb300 import fr, workloads as W

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    mesh = W.box_hex_mesh(N_EDGE)
    p0 = W.tgv_p0()
    prm = fr.make_params(p=P, prec="fp64", p_ref=p0)
    m = fr.FRMesh(mesh, prm)
    info = m.info()
    xyz = m.sol_coords()
    U0 = W.tgv_state(xyz, [(N_EDGE ** 3, (P + 1) ** 3)], perturb=1e-3)
    dof = U0.size
    U = torch.from_numpy(U0).cuda()

    # --- headline: FP64 fused, RK4 steps (one CUDA graph per step) on a side stream, timed with
    #     events on that stream, barrier + max over ranks; no per-kernel instrumentation -----------
    tuned = m.autotune(U, torch.empty_like(U))      # launch shape of the volume kernel
    s = torch.cuda.Stream()
    for _ in range(args.warmup):                    # the first step captures the graph
        m.rk4_step(U, DT, 1, stream=s)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(s)
        for _ in range(args.steps):
            m.rk4_step(U, DT, 1, stream=s)
        e1.record(s)
        torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / args.steps
    m.sync_status(stream=s)
    # --- kernel split: a second pass over the same number of steps with CUDA events recorded
    #     around every launch (plain launches; this pass is not the headline) ----------------------
    m.set_timing(True)
    for _ in range(args.steps):
        m.rk4_step(U, DT, 1, stream=s)
    torch.cuda.synchronize()
    m.set_timing(False)
    kt = m.kernel_times()
    m.sync_status(stream=s)
    from paper_2401_06132_gb300 import replicas
    ms_step = replicas.max_over_ranks(ms_step, device="cuda")    # slowest replica
    if world > 1:
        torch.distributed.barrier()
    value = replicas.replica_throughput(dof, RHS_PER_STEP, ms_step, world)
    # fused form: the RK4 stage update is folded into the last interface kernel of each RHS
    launches_per_step = RHS_PER_STEP * info["launches_per_rhs"]

    if rank != 0:
        return

    # --- dominant kernel and its roofline ----------------------------------------------------
    names = {0: "fused A (disu)", 1: "fused B (volume group)", 2: "fused C (interface group)",
             3: "fused C1 (pair flux)", 4: "fused C2 (lift + RK4 stage)", 30: "RK4 update"}
    share = {names.get(k, str(k)): v[0] / max(1e-9, sum(x[0] for x in kt.values())) for k, v in kt.items()}
    b_ms, b_n = kt.get(1, (0.0, 1))
    b_avg = b_ms / max(1, b_n)
    flops_b = phase_b_flops_per_element() * info["elements"]
    probe = fr.probe_fma()
    # FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA per clock x 2 FLOP x 2.07 GHz
    peak_fp64 = FP64_PEAK_TFLOPS
    achieved = flops_b / (b_avg * 1e-3) / 1e12
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else open(os.devnull) as f:
        try:
            peaks = json.load(f)
        except Exception:
            peaks = {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    compulsory = 2 * dof * 8  # U read + R written per RHS, FP64
    rhs_ms = ms_step / RHS_PER_STEP
    hbm_frac = compulsory / (rhs_ms * 1e-3) / 1e9 / hbm_peak

    # --- other forms (same workload): FP64 unfused, FP32 fused / unfused, mixed fused -----------
    forms = {"fused_fp64": value / world}
    ksteps = max(2, min(args.steps, 5))
    m.set_form("unfused")
    forms["unfused_fp64"] = dof * RHS_PER_STEP / (time_rk4(m, U, ksteps, 1, torch) * 1e-3) / 1e9
    m.set_form("fused")
    del U
    torch.cuda.empty_cache()
    errs = {}
    eb = [[(0, N_EDGE ** 3, (P + 1) ** 3)]]
    m32 = fr.FRMesh(mesh, fr.make_params(p=P, prec="fp32", p_ref=p0, rho_ref=1.0))
    U = torch.from_numpy(U0).cuda()
    U32 = U.float()
    m32.autotune(U32, torch.empty_like(U32))
    del U32
    # FP32 fused: low-Mach form (<= 2e-5 relative RHS error against the FP64 oracle)
    forms["fused_fp32"] = dof * RHS_PER_STEP / (time_rk4(m32, U, ksteps, 2, torch) * 1e-3) / 1e9
    errs["fused_fp32"] = rhs_error(m, m32, U0, eb, torch)
    # the same with the RK4 stage states and sum formed in FP64 (fr_set_rk_fp64_stages): the cost of
    # keeping FP64 in the stage arithmetic (its accuracy effect: the 100-step dissipation tests)
    m32.set_rk_fp64_stages(True)
    forms["fused_fp32_fp64_stage_sums"] = dof * RHS_PER_STEP / (time_rk4(m32, U, ksteps, 2, torch) * 1e-3) / 1e9
    m32.set_rk_fp64_stages(False)
    m32.set_form("unfused")   # plain FP32, one kernel per paper kernel
    forms["unfused_fp32"] = dof * RHS_PER_STEP / (time_rk4(m32, U, ksteps, 1, torch) * 1e-3) / 1e9
    errs["unfused_fp32"] = rhs_error(m, m32, U0, eb, torch)
    m32.close()
    del m32
    # mixed forms with the hexahedral x-y plane contractions moved to the tensor cores as split
    # FP16 / BF16 products (low-Mach form); without that switch a hex-only grid runs the FP32 kernels
    for prec in ("mixed_fp16", "mixed_bf16"):
        mm = fr.FRMesh(mesh, fr.make_params(p=P, prec=prec, p_ref=p0, rho_ref=1.0))
        mm.set_hex_tensor_cores(True)
        forms[f"fused_{prec}_hex_tensor_cores"] = dof * RHS_PER_STEP / (time_rk4(mm, U, ksteps, 2, torch) * 1e-3) / 1e9
        errs[f"fused_{prec}_hex_tensor_cores"] = rhs_error(m, mm, U0, eb, torch)
        mm.close()
        del mm
    m.close()
    del m, U
    torch.cuda.empty_cache()

    # --- the other workloads: mixed hex/prism grid and the batched ensemble -----------------------
    others = {}
    if not args.skip_configs:
        others = other_configs(args, torch, fr, W)

    # --- end to end through the host-buffer entry point (copies inside the timed region) ------
    m = fr.FRMesh(mesh, prm)
    Uh = torch.from_numpy(U0.copy()).pin_memory().numpy()
    m.rk4_step_host(Uh, DT, 1)
    t0 = time.perf_counter()
    ke = max(2, min(args.steps, 5))
    for _ in range(ke):
        m.rk4_step_host(Uh, DT, 1)
    e2e_s = (time.perf_counter() - t0) / ke
    e2e_value = dof * RHS_PER_STEP / e2e_s / 1e9
    m.close()

    cpu, _ = oracle_sample(seconds=args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(), "elements": info["elements"], "dof": dof, "rhs_per_step": RHS_PER_STEP,
                   "form": "fused", "volume_kernel_threads": tuned,
                   "timing": "headline: CUDA-graph RK4 steps without instrumentation; kernel split and the "
                             "roofline's launch duration: a second pass of the same steps with per-launch events",
                   "l2": "inputs larger than L2 (283 MB FP64 state, 129 MB L2)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"kernel": "fused B (volume group)", "bound": "alu", "achieved": achieved, "peak": peak_fp64,
                     "unit": "TFLOP/s", "frac": achieved / peak_fp64,
                     "traffic": VOLUME_FP64_DRAM_BYTES_PER_ELEMENT * info["elements"],
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 FLOP x 2.07 GHz",
                     "traffic_source": "ncu dram bytes of one volume-kernel launch on the 40^3 box, scaled by elements",
                     "probe_fp64_tflops": probe["fp64_gflops"] / 1e3,
                     "frac_of_probe": achieved / (probe["fp64_gflops"] / 1e3),
                     "flops_per_launch": flops_b, "avg_launch_ms": b_avg},
        "hbm_roofline": {"compulsory_bytes_per_rhs": compulsory, "peak_gbs": hbm_peak,
                         "frac": hbm_frac, "note": "compulsory bytes (U read + R written) / RHS time / measured copy peak"},
        "forms_gdof_rhs_per_s": forms,
        "forms_rhs_error": errs,
        "other_workloads": others,
        "kernel_share": share,
        "probe": probe,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": dof * 8, "d2h_bytes_per_step": dof * 8},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-configs", action="store_true", help="skip the mixed-grid and ensemble workloads")
    ap.add_argument("--mode", default="replicas", choices=["replicas", "partitioned"],
                    help="N > 1: independent replicas (weak scaling) or one mesh split over the GPUs (strong)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.mode == "partitioned":
        run_partitioned(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
