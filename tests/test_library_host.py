"""CPU-only checks of the GPU library's host side and of the shared input generators.

No compute call reaches a GPU here: the library is built, loaded and probed for its exported
symbols; mesh validation errors are raised by host code before any device work.
"""
import ctypes as C
import re
import shutil

import numpy as np
import pytest

from paper_2401_06132_gb300 import fr, workloads as W

HEADER = "include/fr_gb300.h"


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2401_06132_gb300 import build as B
    B.build()
    return fr.lib()


def test_library_exports_every_declared_symbol(lib):
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = open(os.path.join(root, HEADER)).read()
    names = re.findall(r"^\s*(?:fr_status|long long|const char \*)\s*\*?\s*(fr_\w+)\s*\(", hdr, re.M)
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_setters_reject_a_null_handle(lib):
    """The switches of a handle (form, graphs, tensor-core paths, timing, debug) check the handle on
    the host and return FR_EINVAL for a null one, with no device work."""
    for name in ("fr_set_form", "fr_set_graph", "fr_set_hex_tensor_cores", "fr_set_dense_tensor_cores",
                 "fr_set_timing"):
        f = getattr(lib, name)
        f.restype = C.c_int
        assert f(C.c_void_p(None), C.c_int(1)) == fr.FR_EINVAL, name


def _create(mesh, **kw):
    return fr.FRMesh(mesh, fr.make_params(**kw))


def test_host_validation_rejects_bad_meshes_before_any_device_work(lib):
    # non-periodic box: boundary faces have no partner
    with pytest.raises(fr.FRError) as e:
        _create(W.box_hex_mesh(2, periodic=False))
    assert e.value.status == fr.FR_EMESH
    # non-affine hex (one corner moved) is a curved element: with a non-affine prism beside it the
    # mesh is refused (prisms must be affine)
    mesh = W.mixed_box_mesh(2)
    mesh["verts"] = mesh["verts"].copy()
    mesh["verts"][mesh["pri_v"][0, 4]] += np.array([0.05, 0.0, 0.0])
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status in (fr.FR_EUNSUPPORTED, fr.FR_EMESH)
    # inverted element: swap two corners of the tensor order
    mesh = W.box_hex_mesh(1)
    mesh["hex_v"] = mesh["hex_v"][:, [1, 0, 3, 2, 5, 4, 7, 6]].copy()
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status == fr.FR_EMESH
    # vertex id out of range
    mesh = W.box_hex_mesh(1)
    mesh["hex_v"] = mesh["hex_v"].copy()
    mesh["hex_v"][0, 0] = 10 ** 6
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status == fr.FR_EMESH
    # unsupported order / quadrature
    with pytest.raises(fr.FRError) as e:
        _create(W.box_hex_mesh(1), p=7)
    assert e.value.status == fr.FR_EUNSUPPORTED
    with pytest.raises(fr.FRError) as e:
        _create(W.box_hex_mesh(1), p=3, nq1d=8)
    assert e.value.status == fr.FR_EUNSUPPORTED
    with pytest.raises(fr.FRError) as e:
        _create(W.box_hex_mesh(1), gamma=0.9)
    assert e.value.status == fr.FR_EINVAL
    # the collocation form (nq1d = p + 1) is built for hexahedra only
    with pytest.raises(fr.FRError) as e:
        _create(W.mixed_box_mesh(2), p=3, nq1d=4)
    assert e.value.status == fr.FR_EUNSUPPORTED and "anti-aliasing" in str(e.value)
    # surface-flux anti-aliasing: single-instance hexahedral meshes with m = p + 2
    with pytest.raises(fr.FRError) as e:
        _create(W.mixed_box_mesh(2), p=3, surface_aa=True)
    assert e.value.status == fr.FR_EUNSUPPORTED and "surface-flux" in str(e.value)
    with pytest.raises(fr.FRError) as e:
        _create(W.box_hex_mesh(2), p=3, nq1d=4, surface_aa=True)
    assert e.value.status == fr.FR_EUNSUPPORTED and "surface-flux" in str(e.value)


def test_splitmix64_reference_vectors():
    """SplitMix64 (Steele, Lea, Flood 2014; Vigna's reference C code) seeded with 1234567."""
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
              16408922859458223821]
    got = [int(v) for v in W.splitmix64(1234567, np.arange(5))]
    assert got == expect


def test_uniform_range_and_mean():
    u = W.uniform_pm1(W.SEED, np.arange(200000))
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 5e-3


def test_mesh_generators_counts_and_volume():
    for N in (1, 3, 8):
        m = W.box_hex_mesh(N)
        assert m["hex_v"].shape == (N ** 3, 8)
        m = W.sheared_box_mesh(N)
        assert m["hex_v"].shape == (N ** 3, 8)
    m = W.mixed_box_mesh(4)
    assert m["hex_v"].shape == (32, 8) and m["pri_v"].shape == (64, 6)


def test_ensemble_draws_ranges():
    d = W.ensemble_draws(64)
    assert len(d) == 64
    assert {x["edge"] for x in d} <= {8, 12, 16, 20, 24} and {x["p"] for x in d} <= {3, 4}
    assert all(0.05 <= x["mach"] <= 0.2 and 400 <= x["re"] <= 3200 for x in d)


def test_tgv_state_layout():
    xyz = np.random.default_rng(0).uniform(-3, 3, size=(2 * 64, 3))
    U = W.tgv_state(xyz, [(2, 64)])
    V = W.tgv_conserved(xyz)
    assert U.shape == (2 * 5 * 64,)
    np.testing.assert_array_equal(U.reshape(2, 5, 64)[1, 4], V[4, 64:])


def test_host_validation_prisms(lib):
    # prisms are built for p = 3 only
    with pytest.raises(fr.FRError) as e:
        _create(W.mixed_box_mesh(2), p=4)
    assert e.value.status == fr.FR_EUNSUPPORTED
    # a non-affine prism (top triangle sheared differently from the bottom one)
    mesh = W.mixed_box_mesh(2)
    mesh["verts"] = mesh["verts"].copy()
    top = mesh["pri_v"][0, 4]
    mesh["verts"][top] += np.array([0.05, 0.0, 0.0])
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status in (fr.FR_EUNSUPPORTED, fr.FR_EMESH)
    # a prism mesh with one prism removed leaves faces without partners
    mesh = W.mixed_box_mesh(2)
    mesh["pri_v"] = mesh["pri_v"][1:].copy()
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status == fr.FR_EMESH


def test_tet_mesh_generator_orientation_and_volume():
    """The Kuhn split: six positively oriented tetrahedra per cell filling the box."""
    for shear in (False, True):
        m = W.box_tet_mesh(3, shear=shear)
        v, t = m["verts"], m["tet_v"]
        assert t.shape == (6 * 27, 4)
        J = np.stack([v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]], v[t[:, 3]] - v[t[:, 0]]], axis=2)
        det = np.linalg.det(J)
        assert np.all(det > 0)
        assert abs(det.sum() / 6 - (2 * np.pi) ** 3) < 1e-9


def test_host_validation_tetrahedra(lib):
    mesh = W.box_tet_mesh(1)
    for kw in (dict(p=4), dict(p=3, nq1d=4), dict(p=3, surface_aa=True)):
        with pytest.raises(fr.FRError) as e:
            _create(mesh, **kw)
        assert e.value.status == fr.FR_EUNSUPPORTED, kw
    # one tetrahedron removed: faces without partners
    mesh = W.box_tet_mesh(2)
    mesh["tet_v"] = mesh["tet_v"][1:].copy()
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status == fr.FR_EMESH
    # an inverted tetrahedron (two vertices swapped)
    mesh = W.box_tet_mesh(2)
    mesh["tet_v"] = mesh["tet_v"].copy()
    mesh["tet_v"][0, [1, 2]] = mesh["tet_v"][0, [2, 1]]
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status == fr.FR_EMESH


def test_host_validation_curved(lib):
    """Curved (trilinear) hexahedra run single-instance hexahedral meshes with m = p + 2."""
    mesh = W.curved_box_mesh(3)
    for kw in (dict(p=3, nq1d=4), dict(p=3, surface_aa=True)):
        with pytest.raises(fr.FRError) as e:
            _create(mesh, **kw)
        assert e.value.status == fr.FR_EUNSUPPORTED, kw
    with pytest.raises(fr.FRError) as e:
        fr.FRMesh([mesh, mesh], fr.make_params(p=3))
    assert e.value.status == fr.FR_EUNSUPPORTED


def test_pyr_mesh_generator_orientation_and_volume():
    """Six positively oriented pyramids per cell, filling the box; bases in tensor order."""
    for hb in (0, 2):
        m = W.box_pyr_mesh(3, hex_below=hb)
        v, P = m["verts"], m["pyr_v"]
        assert P.shape == (6 * 9 * (3 - hb), 5) and m["hex_v"].shape[0] == 9 * hb
        J0 = 0.5 * (v[P[:, 1]] - v[P[:, 0]])
        J1 = 0.5 * (v[P[:, 2]] - v[P[:, 0]])
        J2 = 0.5 * (v[P[:, 4]] - v[P[:, 0]]) - 0.5 * (J0 + J1)
        det = np.einsum("ij,ij->i", J0, np.cross(J1, J2))
        assert np.all(det > 0)
        np.testing.assert_allclose(v[P[:, 3]], v[P[:, 1]] + v[P[:, 2]] - v[P[:, 0]], atol=1e-12)
        vol = det.sum() * 8 / 3 + 8 * (2 * np.pi / 3) ** 3 / 8 * m["hex_v"].shape[0]
        assert abs(vol - (2 * np.pi) ** 3) < 1e-9


def test_host_validation_pyramids(lib):
    mesh = W.box_pyr_mesh(1)
    for kw in (dict(p=4), dict(p=3, nq1d=4), dict(p=3, surface_aa=True)):
        with pytest.raises(fr.FRError) as e:
            _create(mesh, **kw)
        assert e.value.status == fr.FR_EUNSUPPORTED, kw
    mesh = W.box_pyr_mesh(2)
    mesh["pyr_v"] = mesh["pyr_v"][1:].copy()
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status == fr.FR_EMESH
    mesh = W.box_pyr_mesh(2)
    mesh["pyr_v"] = mesh["pyr_v"].copy()
    mesh["pyr_v"][0, [1, 2]] = mesh["pyr_v"][0, [2, 1]]
    with pytest.raises(fr.FRError) as e:
        _create(mesh)
    assert e.value.status == fr.FR_EMESH
