"""Seeded synthetic inputs shared by the GPU path, the tests and the benchmark.

This module holds no arithmetic of the FR method: only mesh geometry (vertex grids and element
connectivity of the Taylor-Green-vortex boxes), the analytic Taylor-Green initial condition as a
function of physical coordinates, and a counter-based SplitMix64 generator. Solution-point
coordinates are always supplied by the caller (the GPU library or the oracle), so no point set or
mapping of the method lives here.

Taylor-Green vortex (Sec. 6 of the paper, with reading G6 for the sign of v_y and G7 for a uniform
density): on [-pi L, pi L]^3, rho = 1, v = U0 (sin x cos y cos z, -cos x sin y cos z, 0),
p = p0 + rho0 U0^2/16 (cos 2x + cos 2y)(cos 2z + 2), p0 = rho0 U0^2 / (gamma M^2).
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20240111
MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------------------------
# Counter-based generator
# ---------------------------------------------------------------------------------------------

def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output number idx (0-based) of the stream started at ``seed`` (Steele, Lea and
    Flood, 2014): z = seed + (idx+1)*0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, idx: np.ndarray) -> np.ndarray:
    """U(-1, 1) from the top 53 bits of SplitMix64 number idx."""
    z = splitmix64(seed, idx)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def uniform01(seed: int, idx) -> np.ndarray:
    z = splitmix64(seed, np.asarray(idx))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------------------------
# Meshes (vertex grids and connectivity only)
# ---------------------------------------------------------------------------------------------

def box_hex_mesh(N: int, length: float = 2 * math.pi, origin: float = -math.pi, periodic: bool = True):
    """N^3 uniform hexahedra on [origin, origin+length]^3. Element index ex + N ey + N^2 ez;
    hex vertex order is tensor order (corner a + 2b + 4c for (a,b,c) in {0,1}^3)."""
    g = origin + length * np.arange(N + 1) / N
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")], axis=1)
    vid = lambda i, j, k: i + (N + 1) * (j + (N + 1) * k)  # noqa: E731
    e = np.arange(N ** 3)
    ex, ey, ez = e % N, (e // N) % N, e // (N * N)
    hex_v = np.stack([vid(ex + (c & 1), ey + ((c >> 1) & 1), ez + ((c >> 2) & 1)) for c in range(8)], axis=1)
    per = (length, length, length) if periodic else (0.0, 0.0, 0.0)
    return dict(verts=verts, hex_v=hex_v.astype(np.int32), pri_v=np.zeros((0, 6), np.int32), period=per)


def mixed_box_mesh(N: int, length: float = 2 * math.pi, origin: float = -math.pi):
    """N^3 box (N even): cells with x < 0 are hexahedra; each cell with x >= 0 is split along the
    xy-face diagonal into two prisms extruded along z. Prism vertex order: v0,v1,v2 at the lower z
    face mapped to the reference (-1,-1),(1,-1),(-1,1), and v3,v4,v5 above them."""
    assert N % 2 == 0
    g = origin + length * np.arange(N + 1) / N
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")], axis=1)
    vid = lambda i, j, k: i + (N + 1) * (j + (N + 1) * k)  # noqa: E731
    hexes, prisms = [], []
    for ez in range(N):
        for ey in range(N):
            for ex in range(N):
                c = [vid(ex + (q & 1), ey + ((q >> 1) & 1), ez + ((q >> 2) & 1)) for q in range(8)]
                if ex < N // 2:
                    hexes.append(c)
                else:
                    # lower triangle: right angle at corner (0,0)
                    prisms.append([c[0], c[1], c[2], c[4], c[5], c[6]])
                    # upper triangle: right angle at corner (1,1)
                    prisms.append([c[3], c[2], c[1], c[7], c[6], c[5]])
    return dict(verts=verts, hex_v=np.array(hexes, np.int32).reshape(-1, 8),
                pri_v=np.array(prisms, np.int32).reshape(-1, 6), period=(length, length, length))


# ---------------------------------------------------------------------------------------------
# Analytic Taylor-Green state
# ---------------------------------------------------------------------------------------------

def tgv_p0(gamma: float = 1.4, mach: float = 0.1, rho0: float = 1.0, U0: float = 1.0) -> float:
    return rho0 * U0 * U0 / (gamma * mach * mach)


def tgv_conserved(xyz: np.ndarray, gamma: float = 1.4, mach: float = 0.1, rho0: float = 1.0,
                  U0: float = 1.0, L: float = 1.0) -> np.ndarray:
    """Conserved variables (rho, rho v, E) of the Taylor-Green initial condition at points xyz
    [npts, 3]; returns [5, npts]."""
    x, y, z = xyz[:, 0] / L, xyz[:, 1] / L, xyz[:, 2] / L
    p0 = tgv_p0(gamma, mach, rho0, U0)
    vx = U0 * np.sin(x) * np.cos(y) * np.cos(z)
    vy = -U0 * np.cos(x) * np.sin(y) * np.cos(z)
    vz = np.zeros_like(x)
    p = p0 + rho0 * U0 * U0 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = np.full_like(x, rho0)
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return np.stack([rho, rho * vx, rho * vy, rho * vz, E])


def to_layout(values_per_point: np.ndarray, pts_per_elem) -> np.ndarray:
    """[5, sum_pts] point-major values -> flat [elem][var][pt] array. ``pts_per_elem`` is a
    list of (n_elements, n_points) blocks in element order."""
    out = []
    off = 0
    for ne, npt in pts_per_elem:
        blk = values_per_point[:, off:off + ne * npt].reshape(5, ne, npt).transpose(1, 0, 2)
        out.append(blk.reshape(-1))
        off += ne * npt
    return np.concatenate(out)


def tgv_state(xyz: np.ndarray, pts_per_elem, gamma=1.4, mach=0.1, perturb: float = 0.0,
              seed: int = SEED, dof_offset: int = 0) -> np.ndarray:
    """TGV state in the [elem][var][pt] layout; optionally times (1 + perturb*xi) per DOF with
    xi ~ U(-1,1) from SplitMix64(seed) indexed by the global DOF id."""
    U = to_layout(tgv_conserved(xyz, gamma, mach), pts_per_elem)
    if perturb:
        U = U * (1.0 + perturb * uniform_pm1(seed, np.arange(dof_offset, dof_offset + U.size)))
    return U


# ---------------------------------------------------------------------------------------------
# Batched ensemble of Taylor-Green instances
# ---------------------------------------------------------------------------------------------

def ensemble_draws(n_inst: int = 64, seed: int = SEED):
    """Per instance, in this draw order: edge ~ U{8,12,16,20,24}, p ~ U{3,4}, M ~ U[0.05,0.2],
    Re ~ U[400,3200]; four SplitMix64 numbers per instance."""
    out = []
    for i in range(n_inst):
        u = uniform01(seed, np.arange(4 * i, 4 * i + 4))
        edge = (8, 12, 16, 20, 24)[min(int(u[0] * 5), 4)]
        p = 3 if u[1] < 0.5 else 4
        mach = 0.05 + 0.15 * u[2]
        re = 400.0 + 2800.0 * u[3]
        out.append(dict(edge=edge, p=p, mach=float(mach), re=float(re)))
    return out


def sheared_box_mesh(N: int, length: float = 2 * math.pi, origin: float = -math.pi):
    """N^3 affine but non-orthogonal hexahedra tiling the periodic box: vertex (i,j,k) sits at
    x = origin + i h + (j + k) h/N, y = origin + j h, z = origin + k h. After N rows the shear adds
    up to one element, so faces still match across the axis-aligned periods."""
    h = length / N
    s = h / N
    i, j, k = np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1), indexing="ij")
    i, j, k = i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")
    verts = np.stack([origin + i * h + (j + k) * s, origin + j * h, origin + k * h], axis=1)
    vid = lambda a, b, c: a + (N + 1) * (b + (N + 1) * c)  # noqa: E731
    e = np.arange(N ** 3)
    ex, ey, ez = e % N, (e // N) % N, e // (N * N)
    hex_v = np.stack([vid(ex + (c & 1), ey + ((c >> 1) & 1), ez + ((c >> 2) & 1)) for c in range(8)], axis=1)
    return dict(verts=verts, hex_v=hex_v.astype(np.int32), pri_v=np.zeros((0, 6), np.int32),
                period=(length, length, length))


# Kuhn split of the unit cube into six tetrahedra, one per axis permutation: each walks from corner
# (0,0,0) to (1,1,1) along the axes in the permutation's order. Corners in tensor order a + 2b + 4c.
_KUHN_PERMS = ((0, 1, 2), (1, 2, 0), (2, 0, 1), (1, 0, 2), (0, 2, 1), (2, 1, 0))


def _kuhn_tets():
    out = []
    for k, perm in enumerate(_KUHN_PERMS):
        c0 = 0
        c1 = c0 | (1 << perm[0])
        c2 = c1 | (1 << perm[1])
        c3 = 7
        # the last three permutations are odd: swap two vertices to keep a positive orientation
        out.append((c0, c1, c2, c3) if k < 3 else (c0, c2, c1, c3))
    return out


def box_tet_mesh(N: int, length: float = 2 * math.pi, origin: float = -math.pi, shear: bool = False):
    """N^3 periodic box of cells, each split into six tetrahedra (Kuhn split, which every cell shares,
    so the faces of neighbouring cells match, also across the periods). Tetrahedron vertex order:
    v0..v3 map to the reference corners (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1). With
    ``shear`` the vertex grid is sheared as in ``sheared_box_mesh``."""
    h = length / N
    i, j, k = np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1), indexing="ij")
    i, j, k = i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")
    sx = (j + k) * (h / N) if shear else 0.0
    verts = np.stack([origin + i * h + sx, origin + j * h, origin + k * h], axis=1)
    vid = lambda a, b, c: a + (N + 1) * (b + (N + 1) * c)  # noqa: E731
    e = np.arange(N ** 3)
    ex, ey, ez = e % N, (e // N) % N, e // (N * N)
    corner = np.stack([vid(ex + (c & 1), ey + ((c >> 1) & 1), ez + ((c >> 2) & 1)) for c in range(8)], axis=1)
    tets = np.stack([corner[:, list(t)] for t in _kuhn_tets()], axis=1).reshape(-1, 4)
    return dict(verts=verts, hex_v=np.zeros((0, 8), np.int32), pri_v=np.zeros((0, 6), np.int32),
                tet_v=tets.astype(np.int32), period=(length, length, length))


def curved_box_mesh(N: int, amp: float = 0.1, length: float = 2 * math.pi, origin: float = -math.pi):
    """N^3 periodic box of non-affine (trilinear) hexahedra: the uniform vertex grid (X, Y, Z) moved
    by amp * h * (sin(2 pi Y/L) sin(2 pi Z/L), sin(2 pi Z/L) sin(2 pi X/L), sin(2 pi X/L) sin(2 pi Y/L)),
    a displacement that is periodic on the grid, so faces still match across the periods. Every
    element is a general hexahedron with straight edges whose metric terms vary inside it (for
    N >= 3; at N = 2 every vertex sits on a zero of the displacement)."""
    h = length / N
    g = origin + length * np.arange(N + 1) / N
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    X, Y, Z = X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")
    w = 2 * math.pi / length
    sx, sy, sz = np.sin(w * (X - origin)), np.sin(w * (Y - origin)), np.sin(w * (Z - origin))
    verts = np.stack([X + amp * h * sy * sz, Y + amp * h * sz * sx, Z + amp * h * sx * sy], axis=1)
    vid = lambda i, j, k: i + (N + 1) * (j + (N + 1) * k)  # noqa: E731
    e = np.arange(N ** 3)
    ex, ey, ez = e % N, (e // N) % N, e // (N * N)
    hex_v = np.stack([vid(ex + (c & 1), ey + ((c >> 1) & 1), ez + ((c >> 2) & 1)) for c in range(8)], axis=1)
    return dict(verts=verts, hex_v=hex_v.astype(np.int32), pri_v=np.zeros((0, 6), np.int32),
                period=(length, length, length))


def box_pyr_mesh(N: int, hex_below: int = 0, length: float = 2 * math.pi, origin: float = -math.pi):
    """N^3 periodic box of cells; cells with x index < hex_below are hexahedra, every other cell is
    split into six pyramids, one per cell face, with the face as base and the cell centre as apex
    (its triangular faces meet the neighbouring pyramids of the same cell; its base meets the next
    cell's face, a hexahedron's or another pyramid's base). Pyramid vertex order: the base corners in
    tensor order (reference (-1,-1,-1), (1,-1,-1), (-1,1,-1), (1,1,-1)), then the apex (0,0,1)."""
    g = origin + length * np.arange(N + 1) / N
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    verts = [np.stack([X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")], axis=1)]
    nv0 = (N + 1) ** 3
    vid = lambda i, j, k: i + (N + 1) * (j + (N + 1) * k)  # noqa: E731
    h = length / N
    hexes, pyrs, centres = [], [], []
    for ez in range(N):
        for ey in range(N):
            for ex in range(N):
                c = [vid(ex + (q & 1), ey + ((q >> 1) & 1), ez + ((q >> 2) & 1)) for q in range(8)]
                if ex < hex_below:
                    hexes.append(c)
                    continue
                ci = nv0 + len(centres)
                centres.append([origin + (ex + 0.5) * h, origin + (ey + 0.5) * h, origin + (ez + 0.5) * h])
                for d in range(3):
                    t1, t2 = [t for t in range(3) if t != d]
                    for side in (0, 1):
                        base = []
                        for b in (0, 1):
                            for a in (0, 1):
                                q = (side << d) | (a << t1) | (b << t2)
                                base.append(c[q])
                        # orientation: the apex must lie on the +z side of the reference base
                        if side == 1:
                            base = [base[0], base[2], base[1], base[3]]
                        pyrs.append(base + [ci])
    verts.append(np.array(centres, dtype=np.float64).reshape(-1, 3))
    verts = np.concatenate(verts)
    # fix orientation by the sign of the affine map's determinant
    P = np.array(pyrs, np.int64).reshape(-1, 5)
    if P.shape[0]:
        v = verts
        J0 = 0.5 * (v[P[:, 1]] - v[P[:, 0]])
        J1 = 0.5 * (v[P[:, 2]] - v[P[:, 0]])
        J2 = 0.5 * (v[P[:, 4]] - v[P[:, 0]]) - 0.5 * (J0 + J1)
        det = np.einsum("ij,ij->i", J0, np.cross(J1, J2))
        neg = det < 0
        P[neg] = P[neg][:, [0, 2, 1, 3, 4]]
    return dict(verts=verts, hex_v=np.array(hexes, np.int32).reshape(-1, 8), pri_v=np.zeros((0, 6), np.int32),
                tet_v=np.zeros((0, 4), np.int32), pyr_v=P.astype(np.int32), period=(length, length, length))
