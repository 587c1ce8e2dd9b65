"""ctypes binding of the C ABI in include/fr_gb300.h (argument marshalling only).

Every step of the RHS and of RK4 runs in the CUDA kernels of libfrgb300.so; there is no CPU path.
Device buffers are torch CUDA tensors; the stream is torch's current stream unless given.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FR_LIBRARY=bounds selects the bounds-checking build (libfrgb300_bounds.so, build(variant="bounds"))
LIB_PATH = os.path.join(HERE, "libfrgb300_bounds.so" if os.environ.get("FR_LIBRARY") == "bounds" else "libfrgb300.so")

FR_OK, FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_EMESH, FR_ETIMEOUT, FR_ENONPHYS, FR_EUNSUPPORTED, FR_EBOUNDS = range(9)
STATUS_NAMES = ["FR_OK", "FR_EINVAL", "FR_ENOMEM", "FR_ECUDA", "FR_EMESH", "FR_ETIMEOUT", "FR_ENONPHYS",
                "FR_EUNSUPPORTED", "FR_EBOUNDS"]
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed_bf16": 2, "mixed_fp16": 3}
# volume-kernel launch shapes (fr_autotune, fr_set_volume_shape): threads per element, or elements per
# CTA with register-resident sweeps and the CTAs per SM
SHAPES = (64, 128, 256, "8/CTA x1", "8/CTA x2", "2/CTA split")
FORMS = {"fused": 0, "unfused": 1}


class FRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("Pr", C.c_double), ("mu", C.c_double), ("beta", C.c_double),
                ("tau", C.c_double), ("p", C.c_int), ("nq1d", C.c_int), ("tri_strength", C.c_int),
                ("prec", C.c_int), ("rusanov_mode", C.c_int), ("p_ref", C.c_double), ("rho_ref", C.c_double),
                ("surface_aa", C.c_int)]


class MeshDesc(C.Structure):
    _fields_ = [("n_hex", C.c_int), ("n_pri", C.c_int), ("n_verts", C.c_int), ("verts", C.POINTER(C.c_double)),
                ("hex_v", C.POINTER(C.c_int)), ("pri_v", C.POINTER(C.c_int)), ("period", C.c_double * 3),
                ("n_tet", C.c_int), ("tet_v", C.POINTER(C.c_int)), ("n_pyr", C.c_int), ("pyr_v", C.POINTER(C.c_int))]


_lib = None


def lib():
    """Loads the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, dp, llp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)
        sig = {
            "fr_mesh_create": ([C.POINTER(C.POINTER(MeshDesc)), C.c_int, C.POINTER(Params), C.POINTER(vp)], C.c_int),
            "fr_destroy": ([vp], C.c_int),
            "fr_set_form": ([vp, C.c_int], C.c_int),
            "fr_set_debug": ([vp, C.c_int], C.c_int),
            "fr_rhs": ([vp, vp, vp, vp], C.c_int),
            "fr_rhs_host": ([vp, vp, vp, vp], C.c_int),
            "fr_rk4_step": ([vp, vp, C.c_double, C.c_int, vp], C.c_int),
            "fr_rk4_step_host": ([vp, vp, C.c_double, C.c_int, vp], C.c_int),
            "fr_sync_status": ([vp, vp], C.c_int),
            "fr_mesh_info": ([vp, llp], C.c_int),
            "fr_num_values": ([vp], C.c_longlong),
            "fr_sol_coords": ([vp, dp], C.c_int),
            "fr_instance_offsets": ([vp, llp], C.c_int),
            "fr_diagnostics": ([vp, vp, vp, dp, vp], C.c_int),
            "fr_diagnostics_noalloc": ([vp, vp, vp, dp, vp], C.c_int),
            "fr_stage": ([vp, C.c_int, dp, C.c_longlong, llp], C.c_int),
            "fr_last_error": ([], C.c_char_p),
            "fr_set_timing": ([vp, C.c_int], C.c_int),
            "fr_set_graph": ([vp, C.c_int], C.c_int),
            "fr_set_hex_tensor_cores": ([vp, C.c_int], C.c_int),
            "fr_set_dense_tensor_cores": ([vp, C.c_int], C.c_int),
            "fr_autotune": ([vp, vp, vp, C.POINTER(C.c_int), C.c_int, vp], C.c_int),
            "fr_set_volume_shape": ([vp, C.c_int], C.c_int),
            "fr_set_merged": ([vp, C.c_int], C.c_int),
            "fr_set_rk_fp64_stages": ([vp, C.c_int], C.c_int),
            "fr_group_info": ([vp, C.c_int, llp], C.c_int),
            "fr_set_group_shape": ([vp, C.c_int, C.c_int], C.c_int),
            "fr_kernel_times": ([vp, C.POINTER(C.c_double), llp, C.c_int], C.c_int),
            "fr_probe_fma": ([dp, vp], C.c_int),
            "fr_partition_plan": ([C.POINTER(MeshDesc), C.POINTER(Params), C.c_int, C.c_int, llp, llp, llp, llp,
                                   C.c_longlong], C.c_int),
            "fr_mesh_create_part": ([C.POINTER(MeshDesc), C.POINTER(Params), C.c_int, C.c_int, C.POINTER(vp)], C.c_int),
            "fr_halo_info": ([vp, llp, llp], C.c_int),
            "fr_halo_pack": ([vp, C.c_int, vp, vp], C.c_int),
            "fr_halo_unpack": ([vp, C.c_int, vp, vp], C.c_int),
            "fr_rhs_phase": ([vp, C.c_int, vp, vp, vp], C.c_int),
            "fr_rk4_stage": ([vp, C.c_int, C.c_int, vp, C.c_double, vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes, fn.restype = args, res
        _lib = L
    return _lib


def _check(st):
    if st != FR_OK:
        raise FRError(st, lib().fr_last_error().decode())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_params(p=3, gamma=1.4, Pr=0.71, mu=1.0 / 1600, beta=0.5, tau=0.1, prec="fp64", nq1d=0, tri_strength=0,
                p_ref=0.0, rho_ref=0.0, surface_aa=False):
    return Params(gamma, Pr, mu, beta, tau, p, nq1d, tri_strength, PRECISIONS[prec], 0, p_ref, rho_ref,
                  int(bool(surface_aa)))


def _mesh_desc(m: dict, keep: list) -> MeshDesc:
    """fr_mesh_desc of a mesh dict; the arrays it points to are appended to `keep`."""
    verts = np.ascontiguousarray(m["verts"], dtype=np.float64)
    hex_v = np.ascontiguousarray(m.get("hex_v", np.zeros((0, 8))), dtype=np.int32)
    pri_v = np.ascontiguousarray(m.get("pri_v", np.zeros((0, 6))), dtype=np.int32)
    tet_v = np.ascontiguousarray(m.get("tet_v", np.zeros((0, 4))), dtype=np.int32)
    pyr_v = np.ascontiguousarray(m.get("pyr_v", np.zeros((0, 5))), dtype=np.int32)
    keep += [verts, hex_v, pri_v, tet_v, pyr_v]
    ip = C.POINTER(C.c_int)
    return MeshDesc(hex_v.shape[0], pri_v.shape[0], verts.shape[0], verts.ctypes.data_as(C.POINTER(C.c_double)),
                    hex_v.ctypes.data_as(ip), pri_v.ctypes.data_as(ip),
                    (C.c_double * 3)(*m.get("period", (0.0, 0.0, 0.0))), tet_v.shape[0], tet_v.ctypes.data_as(ip),
                    pyr_v.shape[0], pyr_v.ctypes.data_as(ip))


def partition_plan(mesh: dict, params: Params, nparts: int, part: int) -> dict:
    """fr_partition_plan (host only): own element range, per-peer counts, and the whole-mesh flux
    points this part sends and receives, in buffer order."""
    keep = []
    d = _mesh_desc(mesh, keep)
    info = (C.c_longlong * 6)()
    counts = (C.c_longlong * nparts)()
    _check(lib().fr_partition_plan(C.byref(d), C.byref(params), nparts, part, info, counts, None, None, 0))
    n = info[3]
    send = np.zeros(max(n, 1), dtype=np.int64)
    recv = np.zeros(max(n, 1), dtype=np.int64)
    llp = C.POINTER(C.c_longlong)
    _check(lib().fr_partition_plan(C.byref(d), C.byref(params), nparts, part, info, counts,
                                   send.ctypes.data_as(llp), recv.ctypes.data_as(llp), n))
    return dict(elements=(info[0], info[1]), nfpt_own=info[2], nhalo=n, ne_total=info[4], nfpt_total=info[5],
                counts=list(counts), send=send[:n].copy(), recv=recv[:n].copy())


class FRMesh:
    """One handle over one or more independent mesh instances (batched ensemble when several)."""

    def __init__(self, meshes: Sequence[dict] | dict, params: Sequence[Params] | Params):
        if isinstance(meshes, dict):
            meshes = [meshes]
        if isinstance(params, Params):
            params = [params] * len(meshes)
        assert len(params) == len(meshes)
        self._keep = []
        descs = [_mesh_desc(m, self._keep) for m in meshes]
        arr = (C.POINTER(MeshDesc) * len(descs))(*[C.pointer(d) for d in descs])
        self._descs = descs
        prm = (Params * len(params))(*params)
        h = C.c_void_p()
        _check(lib().fr_mesh_create(arr, len(descs), prm, C.byref(h)))
        self.h = h
        self.prec = params[0].prec
        self.n_inst = len(meshes)

    @classmethod
    def part(cls, mesh: dict, params: Params, nparts: int, part: int) -> "FRMesh":
        """fr_mesh_create_part: part `part` of nparts of a single-instance mesh (own elements only)."""
        self = cls.__new__(cls)
        self._keep = []
        self._descs = [_mesh_desc(mesh, self._keep)]
        h = C.c_void_p()
        _check(lib().fr_mesh_create_part(C.byref(self._descs[0]), C.byref(params), nparts, part, C.byref(h)))
        self.h = h
        self.prec = params.prec
        self.n_inst = 1
        return self

    def halo_info(self) -> dict:
        info = (C.c_longlong * 7)()
        n = max(1, int(self._halo_nparts()))
        counts = (C.c_longlong * n)()
        _check(lib().fr_halo_info(self.h, info, counts))
        return dict(nparts=info[0], part=info[1], elements=(info[2], info[3]), nhalo=info[4],
                    nvar=(info[5], info[6]), counts=list(counts)[:info[0]])

    def _halo_nparts(self) -> int:
        info = (C.c_longlong * 7)()
        _check(lib().fr_halo_info(self.h, info, None))
        return info[0]

    def halo_pack(self, what: int, send, stream=None):
        _check(lib().fr_halo_pack(self.h, what, C.c_void_p(send.data_ptr()), _stream_ptr(stream)))

    def halo_unpack(self, what: int, recv, stream=None):
        _check(lib().fr_halo_unpack(self.h, what, C.c_void_p(recv.data_ptr()), _stream_ptr(stream)))

    def rhs_phase(self, phase: int, U, R, stream=None):
        self._check_tensor(U)
        self._check_tensor(R)
        _check(lib().fr_rhs_phase(self.h, phase, C.c_void_p(U.data_ptr()), C.c_void_p(R.data_ptr()),
                                  _stream_ptr(stream)))

    def rk4_stage(self, stage: int, phase: int, U, dt: float, stream=None):
        """fr_rk4_stage: one phase of one RK4 stage on the FP64 master state U."""
        self._check_tensor(U, dtype=U.dtype)
        assert U.dtype.itemsize == 8, "the RK4 master state is FP64"
        _check(lib().fr_rk4_stage(self.h, stage, phase, C.c_void_p(U.data_ptr()), dt, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().fr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- properties -------------------------------------------------------------------------
    @property
    def dtype(self):
        import torch
        return torch.float64 if self.prec == 0 else torch.float32

    def info(self):
        a = (C.c_longlong * 7)()
        _check(lib().fr_mesh_info(self.h, a))
        keys = ["elements", "values", "flux_points", "pairs", "instances", "launches_per_rhs", "device_bytes"]
        return dict(zip(keys, list(a)))

    @property
    def num_values(self) -> int:
        return int(lib().fr_num_values(self.h))

    def instance_offsets(self):
        a = (C.c_longlong * (self.n_inst + 1))()
        _check(lib().fr_instance_offsets(self.h, a))
        return list(a)

    def sol_coords(self) -> np.ndarray:
        out = np.zeros((self.num_values // 5, 3))
        _check(lib().fr_sol_coords(self.h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def set_form(self, form: str):
        _check(lib().fr_set_form(self.h, FORMS[form]))

    def set_debug(self, flags: int):
        _check(lib().fr_set_debug(self.h, flags))

    # -- compute ----------------------------------------------------------------------------
    def _check_tensor(self, t, dtype=None):
        assert t.is_cuda and t.is_contiguous() and t.numel() == self.num_values, "bad tensor"
        assert t.dtype == (dtype or self.dtype), f"expected {dtype or self.dtype}, got {t.dtype}"

    def rhs(self, U, R, stream=None):
        self._check_tensor(U)
        self._check_tensor(R)
        _check(lib().fr_rhs(self.h, C.c_void_p(U.data_ptr()), C.c_void_p(R.data_ptr()), _stream_ptr(stream)))

    def rhs_host(self, U: np.ndarray, R: np.ndarray, stream=None):
        dt = np.float64 if self.prec == 0 else np.float32
        assert U.dtype == dt and R.dtype == dt and U.flags.c_contiguous and R.flags.c_contiguous
        _check(lib().fr_rhs_host(self.h, C.c_void_p(U.ctypes.data), C.c_void_p(R.ctypes.data), _stream_ptr(stream)))

    def rk4_step(self, U, dt: float, nsteps: int = 1, stream=None):
        import torch
        self._check_tensor(U, torch.float64)
        _check(lib().fr_rk4_step(self.h, C.c_void_p(U.data_ptr()), float(dt), int(nsteps), _stream_ptr(stream)))

    def rk4_step_host(self, U: np.ndarray, dt: float, nsteps: int = 1, stream=None):
        assert U.dtype == np.float64 and U.flags.c_contiguous
        _check(lib().fr_rk4_step_host(self.h, C.c_void_p(U.ctypes.data), float(dt), int(nsteps), _stream_ptr(stream)))

    def sync_status(self, stream=None):
        _check(lib().fr_sync_status(self.h, _stream_ptr(stream)))

    def diagnostics(self, U, R=None, stream=None):
        out = np.zeros(8 * self.n_inst)
        _check(lib().fr_diagnostics(self.h, C.c_void_p(U.data_ptr()), C.c_void_p(R.data_ptr() if R is not None else 0),
                                    out.ctypes.data_as(C.POINTER(C.c_double)), _stream_ptr(stream)))
        res = []
        for i in range(self.n_inst):
            o = out[8 * i:8 * i + 8]
            res.append(dict(volume=o[0], Ek=o[1], eps=o[2], sums=o[3:8].copy()))
        return res

    def groups(self) -> list[dict]:
        """fr_group_info of every kernel group."""
        out, info = [], (C.c_longlong * 6)()
        while lib().fr_group_info(self.h, len(out), info) == FR_OK:
            out.append(dict(type=info[0], p=info[1], m=info[2], elements=info[3], shape=info[4], shapes=info[5]))
        return out

    def autotune(self, U, R, stream=None, cache: str | None = None):
        """Pick the fastest volume-kernel launch shape per group on this state; returns the choices.
        With `cache` (a JSON file), a choice stored there for the same device, precision, element type
        and order is applied without timing, and new choices are added to it."""
        self._check_tensor(U)
        self._check_tensor(R)
        keys = self._shape_keys() if cache else None
        if cache:
            import json
            stored = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    stored = json.load(f)
            if all(k is None or k in stored for k in keys):
                for g, k in enumerate(keys):
                    if k is not None:
                        _check(lib().fr_set_group_shape(self.h, g, int(stored[k])))
                return [SHAPES[g["shape"]] for g in self.groups()]
        out = (C.c_int * 16)(*([-1] * 16))
        _check(lib().fr_autotune(self.h, C.c_void_p(U.data_ptr()), C.c_void_p(R.data_ptr()), out, 16,
                                 _stream_ptr(stream)))
        if cache:
            for g, k in enumerate(keys):
                if k is not None:
                    stored[k] = int(out[g])
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(stored, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return [SHAPES[v] for v in out if v >= 0]

    def _shape_keys(self):
        """Cache key of each group's volume-kernel shape (None for groups without a choice)."""
        import torch
        dev = torch.cuda.get_device_name()
        prec = {v: k for k, v in PRECISIONS.items()}[self.prec]
        return [f"{dev}|{prec}|type{g['type']}|p{g['p']}|m{g['m']}" if g["shapes"] > 1 else None for g in self.groups()]

    def set_merged(self, on: bool):
        """fr_set_merged: one launch per phase over all element groups."""
        _check(lib().fr_set_merged(self.h, int(bool(on))))

    def set_rk_fp64_stages(self, on: bool):
        """fr_set_rk_fp64_stages: reduced precisions form the RK4 stage states and sum in FP64."""
        _check(lib().fr_set_rk_fp64_stages(self.h, int(bool(on))))

    def set_volume_shape(self, shape: int):
        """fr_set_volume_shape: the volume-kernel launch shape of every hexahedral group (0..5)."""
        _check(lib().fr_set_volume_shape(self.h, shape))

    def set_graph(self, on: bool):
        _check(lib().fr_set_graph(self.h, int(on)))

    def set_hex_tensor_cores(self, on: bool):
        _check(lib().fr_set_hex_tensor_cores(self.h, int(on)))

    def set_dense_tensor_cores(self, on: bool):
        _check(lib().fr_set_dense_tensor_cores(self.h, int(on)))

    def set_timing(self, on: bool):
        _check(lib().fr_set_timing(self.h, int(on)))

    def kernel_times(self, n_ids: int = 32):
        """{kernel id: (total ms, launches)} for launches since the last call."""
        ms = (C.c_double * n_ids)()
        cnt = (C.c_longlong * n_ids)()
        _check(lib().fr_kernel_times(self.h, ms, cnt, n_ids))
        return {i: (ms[i], cnt[i]) for i in range(n_ids) if cnt[i]}

    def diagnostics_noalloc(self, U, R=None, stream=None):
        """fr_diagnostics_noalloc: the same sums through the entry point that allocates nothing. While
        another thread captures a stream in global mode, pass a non-blocking stream here (work on the
        legacy default stream would join that capture)."""
        out = np.zeros(8 * self.n_inst)
        _check(lib().fr_diagnostics_noalloc(self.h, C.c_void_p(U.data_ptr()),
                                            C.c_void_p(R.data_ptr() if R is not None else 0),
                                            out.ctypes.data_as(C.POINTER(C.c_double)), _stream_ptr(stream)))
        return [dict(volume=out[8 * i], Ek=out[8 * i + 1], eps=out[8 * i + 2], sums=out[8 * i + 3:8 * i + 8].copy())
                for i in range(self.n_inst)]

    def stage(self, which: int) -> np.ndarray:
        n = C.c_longlong(0)
        _check(lib().fr_stage(self.h, which, None, 0, C.byref(n)))
        out = np.zeros(n.value)
        _check(lib().fr_stage(self.h, which, out.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n)))
        return out


def probe_fma(stream=None):
    out = np.zeros(2)
    _check(lib().fr_probe_fma(out.ctypes.data_as(C.POINTER(C.c_double)), _stream_ptr(stream)))
    return dict(fp64_gflops=out[0], fp32_gflops=out[1])
