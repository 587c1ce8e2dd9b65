"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names what it pins and which plausible mistakes it catches. Values printed in the paper
live under tests/golden/ with their citation.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_06132_gb300 import workloads as W
from tests.analytic_ns import tgv_rhs_function

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return np.array(rows)


def _layout(o, mesh):
    blocks = []
    if mesh["hex_v"].shape[0]:
        blocks.append((mesh["hex_v"].shape[0], o.dims(0)[0]))
    if mesh["pri_v"].shape[0]:
        blocks.append((mesh["pri_v"].shape[0], o.dims(1)[0]))
    if mesh.get("tet_v", np.zeros((0, 4))).shape[0]:
        blocks.append((mesh["tet_v"].shape[0], o.dims(2)[0]))
    if mesh.get("pyr_v", np.zeros((0, 5))).shape[0]:
        blocks.append((mesh["pyr_v"].shape[0], o.dims(3)[0]))
    return blocks


def _eval_poly3(coef, pts):
    """sum c[a,b,c] x^a y^b z^c at pts."""
    out = np.zeros(pts.shape[0])
    for (a, b, c), v in np.ndenumerate(coef):
        out += v * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c
    return out


def _eval_poly3_grad(coef, pts, d):
    out = np.zeros(pts.shape[0])
    for (a, b, c), v in np.ndenumerate(coef):
        e = [a, b, c]
        if e[d] == 0:
            continue
        k = e[d]
        e[d] -= 1
        out += v * k * pts[:, 0] ** e[0] * pts[:, 1] ** e[1] * pts[:, 2] ** e[2]
    return out


def _random_space_poly(rng, p, etype):
    """Random polynomial in the element's solution space: Q_p (hex), P_p(tri) x P_p(z) (prism) or
    P_p (tetrahedron)."""
    c = rng.standard_normal((p + 1, p + 1, p + 1))
    if etype == 1:
        for a in range(p + 1):
            for b in range(p + 1):
                if a + b > p:
                    c[a, b, :] = 0
    if etype == 2:
        for (a, b, cc), _ in np.ndenumerate(c):
            if a + b + cc > p:
                c[a, b, cc] = 0
    return c


class _SpaceFn:
    """A random function of an element's solution space: a polynomial (coefficient array) on
    hexahedra, prisms and tetrahedra; on pyramids a combination of the rational generators
    a^i b^j (1-c)^max(i,j) c^k (a = 2x/(1-z), b = 2y/(1-z), c = z), evaluated directly."""

    def __init__(self, rng, p, etype):
        self.etype = etype
        if etype == 3:
            self.terms = [(i, j, k, rng.standard_normal()) for m in range(p + 1) for k in range(p + 1 - m)
                          for j in range(m + 1) for i in range(m + 1) if max(i, j) == m]
        else:
            self.c = _random_space_poly(rng, p, etype)

    def __call__(self, X):
        if self.etype != 3:
            return _eval_poly3(self.c, X)
        om = 1.0 - X[:, 2]
        a, b, c = 2 * X[:, 0] / om, 2 * X[:, 1] / om, X[:, 2]
        return sum(v * a ** i * b ** j * om ** max(i, j) * c ** k for i, j, k, v in self.terms)


# ----------------------------------------------------------------------------------------------
# Point sets and quadrature
# ----------------------------------------------------------------------------------------------

def test_gl_nodes_match_paper():
    """GL nodes equal the paper's printed 3- and 4-point values (Sec. 4.1 figures)."""
    g = _golden("gl_nodes_paper.txt")
    for n in (3, 4):
        x, _ = O.gauss_legendre(n)
        np.testing.assert_allclose(x, g[g[:, 0] == n, 1], atol=2e-16)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_gl_exactness_is_2n_minus_1(n):
    """Weights sum to 2 and integrate x^k exactly for k <= 2n-1, and not for k = 2n."""
    x, w = O.gauss_legendre(n)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs((w * x ** k).sum() - exact) < 1e-14
    assert abs((w * x ** (2 * n)).sum() - 2.0 / (2 * n + 1)) > 1e-6


def test_triangle_points_match_paper_and_are_symmetric():
    """The prism's triangle points are the paper's printed Williams-Shunn points (Sec. 4.1), and the
    set is invariant under the six symmetries of the reference triangle."""
    g = _golden("ws_triangle_points_paper.txt")
    for p in (2, 3):
        xy = O.tri_solution_points(p)
        np.testing.assert_array_equal(xy, g[g[:, 0] == p, 1:])
        # barycentric coordinates; the symmetry group permutes them
        lam = np.stack([(xy[:, 0] + 1) / 2, (xy[:, 1] + 1) / 2, -(xy[:, 0] + xy[:, 1]) / 2], axis=1)
        for perm in ([1, 0, 2], [2, 1, 0], [0, 2, 1], [1, 2, 0], [2, 0, 1]):
            lp = lam[:, perm]
            img = np.stack([2 * lp[:, 0] - 1, 2 * lp[:, 1] - 1], axis=1)
            d = np.abs(img[:, None, :] - xy[None, :, :]).max(axis=2).min(axis=1)
            assert d.max() < 5e-15


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_collapsed_triangle_rule_strength(k):
    """Reading R8: the k x k collapsed rule integrates lambda1^a lambda2^b exactly for a+b <= 2k-2,
    with the closed form int_T ((x+1)/2)^a ((y+1)/2)^b dx dy = 4 a! b! / (a+b+2)!; it fails above."""
    xy, w = O.tri_rule(k)
    l1, l2 = (xy[:, 0] + 1) / 2, (xy[:, 1] + 1) / 2
    for a in range(2 * k - 1):
        for b in range(2 * k - 1 - a):
            exact = 4.0 * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs((w * l1 ** a * l2 ** b).sum() - exact) < 1e-14
    worst = max(abs((w * l1 ** a * l2 ** (2 * k - 1 - a)).sum()
                    - 4.0 * math.factorial(a) * math.factorial(2 * k - 1 - a) / math.factorial(2 * k + 1))
                for a in range(2 * k))
    assert worst > 1e-8


@pytest.mark.parametrize("p", [2, 3, 4])
def test_triangle_basis_orthonormal_and_complete(p):
    """Reading R11: the Gram-Schmidt triangle basis is orthonormal on the reference triangle (area 2)
    and spans P_p: every monomial of degree <= p is reproduced by its projection."""
    xy, w = O.tri_rule(p + 3)
    B = O.tri_basis_values(p, xy)
    G = B.T @ (w[:, None] * B)
    np.testing.assert_allclose(G, np.eye(B.shape[1]), atol=1e-13)
    for a in range(p + 1):
        for b in range(p + 1 - a):
            m = xy[:, 0] ** a * xy[:, 1] ** b
            proj = B @ (B.T @ (w * m))
            assert np.abs(proj - m).max() < 1e-12


def _jacobi_moment(alpha, k):
    """int_{-1}^{1} (1-x)^alpha x^k dx by the binomial expansion of (1-x)^alpha."""
    return sum(math.comb(alpha, j) * (-1) ** j * (2.0 / (j + k + 1) if (j + k) % 2 == 0 else 0.0)
               for j in range(alpha + 1))


@pytest.mark.parametrize("alpha", [0, 1, 2])
@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_gauss_jacobi_rule_exactness(alpha, n):
    """Reading T2's 1D rules: the n-point Gauss rule of the weight (1-x)^alpha integrates x^k
    exactly for k <= 2n-1 (closed-form moments) and not for k = 2n; alpha = 0 is Gauss-Legendre."""
    x, w = O.gauss_jacobi(n, alpha)
    assert np.all(np.diff(x) > 0) and np.all(np.abs(x) < 1) and np.all(w > 0)
    for k in range(2 * n):
        assert abs((w * x ** k).sum() - _jacobi_moment(alpha, k)) < 1e-14
    assert abs((w * x ** (2 * n)).sum() - _jacobi_moment(alpha, 2 * n)) > 1e-8
    if alpha == 0:
        np.testing.assert_allclose(x, O.gauss_legendre(n)[0], atol=1e-15)


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_collapsed_tetrahedron_rule_strength(k):
    """Reading T2: the k^3 collapsed rule integrates lambda1^a lambda2^b lambda3^c exactly for
    a+b+c <= 2k-1, with lambda_i = (x_i+1)/2 and the Dirichlet integral
    int_T lambda1^a lambda2^b lambda3^c dV = 8 a! b! c! / (a+b+c+3)! (8 = the map's Jacobian);
    it fails at degree 2k (catches a wrong Jacobian weight or a wrong Gauss-Jacobi exponent)."""
    xyz, w = O.tet_rule(k)
    lam = (xyz + 1) / 2
    assert np.all(lam > 0) and np.all(lam.sum(axis=1) < 1) and np.all(w > 0)
    f = math.factorial
    for a in range(2 * k):
        for b in range(2 * k - a):
            for c in range(2 * k - a - b):
                exact = 8.0 * f(a) * f(b) * f(c) / f(a + b + c + 3)
                got = (w * lam[:, 0] ** a * lam[:, 1] ** b * lam[:, 2] ** c).sum()
                assert abs(got - exact) < 1e-14
    worst = max(abs((w * lam[:, 0] ** a * lam[:, 2] ** (2 * k - a)).sum()
                    - 8.0 * f(a) * f(2 * k - a) / f(2 * k + 3)) for a in range(2 * k + 1))
    assert worst > 1e-10


@pytest.mark.parametrize("p", [2, 3])
def test_tetrahedron_points_symmetric_interior_unisolvent(p):
    """Reading T1: (p+1)(p+2)(p+3)/6 interior points, invariant under the 24 symmetries of the
    tetrahedron (permutations of the barycentric coordinates), unisolvent for P_p."""
    import itertools
    x = O.tet_solution_points(p)
    assert x.shape[0] == (p + 1) * (p + 2) * (p + 3) // 6
    lam = np.concatenate([(x + 1) / 2, 1 - ((x + 1) / 2).sum(axis=1, keepdims=True)], axis=1)
    assert lam.min() > 0.04
    for perm in itertools.permutations(range(4)):
        img = lam[:, list(perm)]
        d = np.abs(img[:, None, :] - lam[None, :, :]).max(axis=2).min(axis=1)
        assert d.max() < 1e-15
    V = np.stack([x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c for a in range(p + 1) for b in range(p + 1 - a)
                  for c in range(p + 1 - a - b)], axis=1)
    assert np.linalg.cond(V) < 1e4


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_collapsed_pyramid_rule_strength(k):
    """Reading P2: the k^3 collapsed pyramid rule integrates x^a y^b z^c exactly for a+b+c <= 2k-1,
    against int = 4/((a+1)(b+1)) int_{-1}^{1} z^c ((1-z)/2)^(a+b+2) dz for even a, b (zero otherwise),
    the last integral by the binomial expansion; it fails at degree 2k."""
    xyz, w = O.pyr_rule(k)
    assert np.all(w > 0) and np.all(np.abs(xyz[:, :2]) < (1 - xyz[:, 2:3]) / 2) and abs(w.sum() - 8 / 3) < 1e-14

    def exact(a, b, c):
        if a % 2 or b % 2:
            return 0.0
        n = a + b + 2
        zint = sum(math.comb(n, j) * (-1) ** j * (2.0 / (c + j + 1) if (c + j) % 2 == 0 else 0.0) for j in range(n + 1))
        return 4.0 / ((a + 1) * (b + 1)) * zint / 2 ** n

    for a in range(2 * k):
        for b in range(2 * k - a):
            for c in range(2 * k - a - b):
                got = (w * xyz[:, 0] ** a * xyz[:, 1] ** b * xyz[:, 2] ** c).sum()
                assert abs(got - exact(a, b, c)) < 1e-14, (a, b, c)
    worst = max(abs((w * xyz[:, 2] ** (2 * k)).sum() - exact(0, 0, 2 * k)),
                abs((w * xyz[:, 0] ** 2 * xyz[:, 2] ** (2 * k - 2)).sum() - exact(2, 0, 2 * k - 2)))
    assert worst > 1e-12


@pytest.mark.parametrize("p", [2, 3])
def test_pyramid_points_symmetric_interior_unisolvent(p):
    """Reading P1: (p+1)(p+2)(2p+3)/6 interior points, invariant under the eight symmetries of the
    square base, unisolvent for the rational pyramid space (its generators' Vandermonde matrix is
    well conditioned)."""
    x = O.pyr_solution_points(p)
    n = (p + 1) * (p + 2) * (2 * p + 3) // 6
    assert x.shape[0] == n
    assert np.all(x[:, 2] > -1) and np.all(x[:, 2] < 1) and np.all(np.abs(x[:, :2]).max(axis=1) < (1 - x[:, 2]) / 2)
    for sx, sy, swap in [(a, b, c) for a in (1, -1) for b in (1, -1) for c in (0, 1)]:
        img = x.copy()
        if swap:
            img[:, [0, 1]] = img[:, [1, 0]]
        img[:, 0] *= sx
        img[:, 1] *= sy
        d = np.abs(img[:, None, :] - x[None, :, :]).max(axis=2).min(axis=1)
        assert d.max() < 1e-15
    om = 1 - x[:, 2]
    a, b, c = 2 * x[:, 0] / om, 2 * x[:, 1] / om, x[:, 2]
    V = np.stack([a ** i * b ** j * om ** max(i, j) * c ** k for m in range(p + 1) for k in range(p + 1 - m)
                  for j in range(m + 1) for i in range(m + 1) if max(i, j) == m], axis=1)
    assert V.shape == (n, n) and np.linalg.cond(V) < 1e5


# ----------------------------------------------------------------------------------------------
# Element operators: exactness, projection, lift, sum factorisation
# ----------------------------------------------------------------------------------------------

def _oracle_for(etype, p, m=None):
    m = m or p + 2
    if etype == 0:
        return O.Oracle(W.box_hex_mesh(1), p, m)
    if etype == 2:
        return O.Oracle(W.box_tet_mesh(1), p, m)
    if etype == 3:
        return O.Oracle(W.box_pyr_mesh(1), p, m)
    return O.Oracle(W.mixed_box_mesh(2), p, m)


CASES = [(0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (2, 2), (2, 3), (3, 2), (3, 3)]
VOLUME = {0: 8.0, 1: 4.0, 2: 4.0 / 3.0, 3: 8.0 / 3.0}


@pytest.mark.parametrize("etype,p", CASES)
def test_interpolation_and_derivative_exact_on_space(etype, p):
    """Check (b): M0 (disu) and M7 (uqpts) reproduce every function of the solution space exactly,
    and the derivative matrices M4 = M1 every polynomial of it (on the pyramid, whose rational space
    is not closed under differentiation, reading P3: the polynomials P_p, where the projected
    derivative is exact). Catches a transposed operator or a wrong point set."""
    o = _oracle_for(etype, p)
    xu, xf, xq = o.op(etype, "xu"), o.op(etype, "xf"), o.op(etype, "xq")
    M0, M7, D = o.op(etype, "M0"), o.op(etype, "M7"), o.op(etype, "D")
    rng = np.random.default_rng(7)
    for _ in range(3):
        f = _SpaceFn(rng, p, etype)
        u = f(xu)
        assert np.abs(M0 @ u - f(xf)).max() < 1e-12
        assert np.abs(M7 @ u - f(xq)).max() < 1e-12
        c = _random_space_poly(rng, p, 2 if etype == 3 else etype)
        u = _eval_poly3(c, xu)
        for d in range(3):
            assert np.abs(D[d] @ u - _eval_poly3_grad(c, xu, d)).max() < 1e-11
    # one degree higher is not reproduced (the space is exactly the stated one)
    c = np.zeros((p + 2, p + 2, p + 2)); c[p + 1, 0, 0] = 1.0
    assert np.abs(M7 @ _eval_poly3(c, xu) - _eval_poly3(c, xq)).max() > 1e-6


@pytest.mark.parametrize("etype,p", CASES)
def test_volume_quadrature_and_projection(etype, p):
    """Check (c) and the M8 projection: the volume rule integrates degree-2p products of the space
    exactly; M8 M7 = I; and M8 g is the L2 projection of any g sampled at quadrature points (the
    residual is orthogonal to the space)."""
    o = _oracle_for(etype, p)
    xq, wq, M7, M8 = o.op(etype, "xq"), o.op(etype, "wq"), o.op(etype, "M7"), o.op(etype, "M8")
    assert abs(wq.sum() - VOLUME[etype]) < 1e-13
    np.testing.assert_allclose(M8 @ M7, np.eye(M7.shape[1]), atol=1e-13)
    rng = np.random.default_rng(3)
    g = np.cos(1.3 * xq[:, 0] + 0.7 * xq[:, 1] - 0.4 * xq[:, 2]) + xq[:, 2] ** (p + 1)
    r = g - M7 @ (M8 @ g)
    for _ in range(4):
        f = _SpaceFn(rng, p, etype)
        assert abs((wq * r * f(xq)).sum()) < 1e-13


def _radau_dg_lift(p, xi):
    """Derivative of the DG correction function g_R = (P_p + P_{p+1})/2 at xi (Huynh's Radau form)."""
    cR = np.zeros(p + 2); cR[p] = 0.5; cR[p + 1] = 0.5
    return np.polynomial.legendre.legval(xi, np.polynomial.legendre.legder(cR))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_hex_lift_equals_radau_dg_closed_form(p):
    """Reading R3 on hexahedra: the oracle's M^-1 E lift equals g_R'(xi_i) (right faces) and
    g_R'(-xi_i) (left faces) along the line through each flux point, zero elsewhere."""
    o = _oracle_for(0, p)
    xu, xf, nref, lift = o.op(0, "xu"), o.op(0, "xf"), o.op(0, "nref"), o.op(0, "lift")
    exp = np.zeros_like(lift)
    for s in range(xf.shape[0]):
        d = int(np.argmax(np.abs(nref[s])))
        side = nref[s, d]
        tang = [t for t in range(3) if t != d]
        on_line = np.all(np.abs(xu[:, tang] - xf[s, tang]) < 1e-14, axis=1)
        exp[on_line, s] = _radau_dg_lift(p, side * xu[on_line, d])
    np.testing.assert_allclose(lift, exp, atol=1e-12)


@pytest.mark.parametrize("etype,p", CASES)
def test_lift_is_dg_lift(etype, p):
    """Reading R3 on every face of both element types: the lifted polynomial l_sigma = sum_zeta
    Lift[zeta, sigma] l_zeta satisfies int_V v (sum_sigma l_sigma h_sigma) dV = int_face v h dS for
    every v in the volume space and every h in the face space (reference measure)."""
    o = _oracle_for(etype, p)
    xf, xq, wq = o.op(etype, "xf"), o.op(etype, "xq"), o.op(etype, "wq")
    M7, lift, face = o.op(etype, "M7"), o.op(etype, "lift"), o.op(etype, "fpt_face").astype(int)
    nref = o.op(etype, "nref")
    rng = np.random.default_rng(11)
    gx, gw = O.gauss_legendre(p + 3)
    txy, tw = O.tri_rule(p + 3)
    for f in np.unique(face):
        sel = face == f
        n = nref[sel][0]
        for _ in range(2):
            fv = _SpaceFn(rng, p, etype)
            fh = _SpaceFn(rng, p, etype)
            h_at_f = np.where(sel, fh(xf), 0.0)
            lhs = (wq * fv(xq) * (M7 @ (lift @ h_at_f))).sum()
            # face quadrature in the face parameters; X(s,t) built from the face's plane
            if etype == 3 and n[2] < -0.5:
                # pyramid base z = -1: the traces are Q_p
                S, T = np.meshgrid(gx, gx, indexing="ij")
                pts = np.stack([S.ravel(), T.ravel(), -np.ones(S.size)], 1)
                wts = np.outer(gw, gw).ravel()
            elif etype == 3:
                # pyramid triangle: the apex and the base edge the outward normal points to
                e0 = np.array([n[0], n[1]]) / max(abs(n[0]), abs(n[1]))
                t_ = np.array([-e0[1], e0[0]])
                P0 = np.array([e0[0] - t_[0], e0[1] - t_[1], -1.0])
                P1 = np.array([e0[0] + t_[0], e0[1] + t_[1], -1.0])
                P2 = np.array([0.0, 0.0, 1.0])
                s_, u_ = txy[:, 0], txy[:, 1]
                pts = P0 + np.outer((1 + s_) / 2, P1 - P0) + np.outer((1 + u_) / 2, P2 - P0)
                wts = tw * np.linalg.norm(np.cross(P1 - P0, P2 - P0)) / 4
            elif etype == 0:
                d = int(np.argmax(np.abs(n)))
                tang = [t for t in range(3) if t != d]
                S, T = np.meshgrid(gx, gx, indexing="ij")
                pts = np.zeros((S.size, 3)); pts[:, d] = n[d]; pts[:, tang[0]] = S.ravel(); pts[:, tang[1]] = T.ravel()
                wts = np.outer(gw, gw).ravel()
            elif etype == 2:
                # triangle faces of the tetrahedron, parametrised by the reference triangle (s, t)
                s_, t_ = txy[:, 0], txy[:, 1]
                one = np.ones_like(s_)
                if n[2] < -0.5:
                    pts = np.stack([s_, t_, -one], 1); wts = tw
                elif n[1] < -0.5:
                    pts = np.stack([s_, -one, t_], 1); wts = tw
                elif n[0] < -0.5:
                    pts = np.stack([-one, s_, t_], 1); wts = tw
                else:
                    pts = np.stack([-1 - s_ - t_, s_, t_], 1); wts = tw * math.sqrt(3.0)
            elif abs(n[2]) > 0.5:
                pts = np.zeros((txy.shape[0], 3)); pts[:, :2] = txy; pts[:, 2] = n[2]; wts = tw
            else:
                S, T = np.meshgrid(gx, gx, indexing="ij")
                s, t = S.ravel(), T.ravel()
                wts = np.outer(gw, gw).ravel()
                if n[1] < -0.5:
                    pts = np.stack([s, -np.ones_like(s), t], 1)
                elif n[0] < -0.5:
                    pts = np.stack([-np.ones_like(s), s, t], 1)
                else:
                    pts = np.stack([-s, s, t], 1); wts = wts * math.sqrt(2.0)
            rhs = (wts * fv(pts) * fh(pts)).sum()
            assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs))


@pytest.mark.parametrize("p,m", [(3, 5), (4, 6)])
def test_dense_equals_sum_factorised(p, m):
    """Check (d): the dense hex operators equal Kronecker products of 1D factors (interpolation
    n->m, projection m->n, derivative, face interpolation) to 1e-14 (Sec. 4)."""
    o = O.Oracle(W.box_hex_mesh(1), p, m)
    n = p + 1
    x, _ = O.gauss_legendre(n)
    xq, wq1 = O.gauss_legendre(m)

    def lag(xs, a, t):
        v = np.ones_like(t)
        for b in range(len(xs)):
            if b != a:
                v = v * (t - xs[b]) / (xs[a] - xs[b])
        return v

    B = np.stack([lag(x, a, xq) for a in range(n)], axis=1)            # m x n
    Dd = np.zeros((n, n))
    for a in range(n):
        c = np.poly1d([1.0])
        for b in range(n):
            if b != a:
                c = c * np.poly1d([1.0, -x[b]]) / (x[a] - x[b])
        Dd[:, a] = np.polyder(c)(x)
    V = np.stack([np.sqrt(r + 0.5) * np.polynomial.legendre.legval(x, np.eye(n)[r]) for r in range(n)], 1)
    Vq = np.stack([np.sqrt(r + 0.5) * np.polynomial.legendre.legval(xq, np.eye(n)[r]) for r in range(n)], 1)
    P = V @ (Vq * wq1[:, None]).T                                       # n x m
    I = np.eye(n)
    # tensor index a + n b + n^2 c -> kron(z, y, x)
    np.testing.assert_allclose(o.op(0, "M7"), np.kron(B, np.kron(B, B)), atol=1e-14)
    np.testing.assert_allclose(o.op(0, "M8"), np.kron(P, np.kron(P, P)), atol=1e-14)
    D = o.op(0, "D")
    np.testing.assert_allclose(D[0], np.kron(I, np.kron(I, Dd)), atol=2e-13)
    np.testing.assert_allclose(D[1], np.kron(I, np.kron(Dd, I)), atol=2e-13)
    np.testing.assert_allclose(D[2], np.kron(Dd, np.kron(I, I)), atol=2e-13)
    # face interpolation rows: each flux point's row is a 1D interpolation along its normal line
    xu, xf, M0 = o.op(0, "xu"), o.op(0, "xf"), o.op(0, "M0")
    for s in range(xf.shape[0]):
        row = np.zeros(xu.shape[0])
        d = [k for k in range(3) if abs(abs(xf[s, k]) - 1) < 1e-15 and all(abs(xf[s, t]) < 1 for t in range(3) if t != k)][0]
        tang = [t for t in range(3) if t != d]
        on = np.all(np.abs(xu[:, tang] - xf[s, tang]) < 1e-14, axis=1)
        row[on] = [lag(x, int(np.argmin(np.abs(x - xu[z, d]))), np.array([xf[s, d]]))[0] for z in np.where(on)[0]]
        assert np.abs(M0[s] - row).max() < 1e-14


@pytest.mark.parametrize("etype,p", CASES)
def test_corrected_derivatives_integrate_by_parts(etype, p):
    """Green's identity on every element type: with a zero common value the corrected gradient
    operator M4 - M6 M0 satisfies int v (Agrad_d u) dV = -int u (d_d v) dV, and the corrected
    divergence M1 - M3 M2 satisfies int v (Adiv F) dV = -sum_d int F_d (d_d v) dV, for u, v, F_d in
    the solution space. This pins the lift, the reference normals and the face measure of every
    face at once (a slanted face's sqrt 2, sqrt 3 or sqrt 5 / 2, a flipped normal or a transposed
    lift fail) and, on the pyramid, the projected derivative of reading P3 (the nodal derivative of
    its rational space fails it)."""
    o = _oracle_for(etype, p)
    xu, wq, M7, D = o.op(etype, "xu"), o.op(etype, "wq"), o.op(etype, "M7"), o.op(etype, "D")
    Ag, Ad = o.op(etype, "Agrad"), o.op(etype, "Adiv")
    rng = np.random.default_rng(5)
    ip = lambda a, b: (wq * (M7 @ a) * (M7 @ b)).sum()  # noqa: E731
    for _ in range(2):
        u = _SpaceFn(rng, p, etype)(xu)
        v = _SpaceFn(rng, p, etype)(xu)
        F = [_SpaceFn(rng, p, etype)(xu) for _ in range(3)]
        for d in range(3):
            lhs, rhs = ip(v, Ag[d] @ u), -ip(u, D[d] @ v)
            assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs))
        lhs = ip(v, np.einsum("zdk,dk->z", Ad, np.array(F)))
        rhs = -sum(ip(F[d], D[d] @ v) for d in range(3))
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs))


def test_operator_identities():
    """The rewrites of Eqs. (Qsubs) and (subs): tgradpcoru's M4 - M6 M0 and tdivtpcorf's M1 - M3 M2
    applied to a field equal the two-step forms."""
    o = _oracle_for(1, 3)
    for t in (0, 1, 2):
        if t == 2:
            o = _oracle_for(2, 3)
        D, M0, lift, nref = o.op(t, "D"), o.op(t, "M0"), o.op(t, "lift"), o.op(t, "nref")
        Ag, Ad = o.op(t, "Agrad"), o.op(t, "Adiv")
        u = np.random.default_rng(0).standard_normal(D.shape[1])
        for d in range(3):
            np.testing.assert_allclose(Ag[d] @ u, D[d] @ u - lift @ (nref[:, d] * (M0 @ u)), atol=1e-11)
        F = np.random.default_rng(1).standard_normal((3, D.shape[1]))
        two_step = sum(D[d] @ F[d] for d in range(3)) - lift @ sum(nref[:, d] * (M0 @ F[d]) for d in range(3))
        np.testing.assert_allclose(np.einsum("zdk,dk->z", Ad, F), two_step, atol=1e-11)


# ----------------------------------------------------------------------------------------------
# Whole RHS: freestream, conservation, physics
# ----------------------------------------------------------------------------------------------

FREESTREAM = np.array([1.1, 1.1 * 0.3, -1.1 * 0.2, 1.1 * 0.1, 1.0 / 0.4 + 0.5 * 1.1 * 0.14])

MESHES = {
    "hex1_self_periodic": lambda: W.box_hex_mesh(1),
    "hex2": lambda: W.box_hex_mesh(2),
    "hex3": lambda: W.box_hex_mesh(3),
    "sheared3": lambda: W.sheared_box_mesh(3),
    "mixed2": lambda: W.mixed_box_mesh(2),
    "mixed4": lambda: W.mixed_box_mesh(4),
    "curved3": lambda: W.curved_box_mesh(3, amp=0.15),
    "pyr2": lambda: W.box_pyr_mesh(2),
    "hexpyr2": lambda: W.box_pyr_mesh(2, hex_below=1),
    "tet2": lambda: W.box_tet_mesh(2),
    "tetshear2": lambda: W.box_tet_mesh(2, shear=True),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("p", [3, 4])
def test_freestream_preservation(name, p):
    """Check (a): a constant state gives a zero RHS to 1e-13 on affine meshes, including
    self-periodic, sheared and mixed hex/prism meshes, and on trilinear (curved) hexahedra, whose
    metric terms lie in the solution space for p >= 2 so that the discrete metric identities hold. Rounding in the divergence grows with the
    operator norm, so the bound is relative to the RHS scale max|f| (2/h) (p+1)^2."""
    mesh = MESHES[name]()
    if (mesh["pri_v"].shape[0] or mesh.get("tet_v", np.zeros((0, 4))).shape[0]
            or mesh.get("pyr_v", np.zeros((0, 5))).shape[0]) and p != 3:
        pytest.skip("printed triangle points exist for p=2,3 only")
    o = O.Oracle(mesh, p, p + 2)
    blocks = _layout(o, mesh)
    U = np.concatenate([np.tile(np.repeat(FREESTREAM, npt), ne) for ne, npt in blocks])
    R = o.rhs(U)
    N = round(mesh["verts"].shape[0] ** (1.0 / 3.0)) - 1
    fmax = 1.1  # largest inviscid flux component of FREESTREAM (p = 1, rho v^2 <= 0.1)
    scale = fmax * (2.0 / (2 * np.pi / N)) * (p + 1) ** 2
    assert np.abs(R).max() < 1e-13 * scale


def _tgv(o, mesh, perturb=0.0, mach=0.1):
    return W.tgv_state(o.sol_coords(), _layout(o, mesh), mach=mach, perturb=perturb)


@pytest.mark.parametrize("name", ["hex1_self_periodic", "hex3", "sheared3", "mixed4", "tetshear2", "curved3", "pyr2",
                                  "hexpyr2"])
def test_discrete_conservation(name):
    """Check (e): the quadrature-weighted RHS sums to zero to 1e-12 relative, per variable."""
    mesh = MESHES[name]()
    o = O.Oracle(mesh, 3, 5)
    U = _tgv(o, mesh, perturb=1e-2)
    d = o.diagnostics(U, o.rhs(U))
    assert np.all(np.abs(d["sums"]) <= 1e-12 * d["abs_sums"])


def test_ke_dissipation_rate_converges_to_closed_form():
    """At t=0 the TGV has div v = 0, so eps(0) = mu <|omega|^2> = 3 mu / 4 for rho = U0 = 1. The
    discrete eps from the RHS converges to it (a dropped or mis-signed viscous term fails)."""
    mu = 1.0 / 1600
    errs = []
    for N in (8, 16):
        mesh = W.box_hex_mesh(N)
        o = O.Oracle(mesh, 3, 5, threads=os.cpu_count())
        U = _tgv(o, mesh)
        d = o.diagnostics(U, o.rhs(U))
        assert abs(d["Ek"] - 0.125) < 1e-12
        errs.append(abs(d["eps"] / (0.75 * mu) - 1.0))
    assert errs[0] < 1e-3 and errs[1] < 2e-6 and errs[1] < errs[0] / 100


@pytest.mark.parametrize("meshfn,m,surf", [(W.box_hex_mesh, 5, False), (W.sheared_box_mesh, 5, False),
                                           (W.box_hex_mesh, 4, False), (W.sheared_box_mesh, 5, True),
                                           (W.curved_box_mesh, 5, False)])
def test_rhs_converges_to_analytic_navier_stokes(meshfn, m, surf):
    """Consistency on a compressible periodic field (div v != 0, non-uniform rho, M = 0.3): the
    inviscid RHS (mu = 0) converges to the exact -div f^e at order >= p - 0.5, and the viscous part
    R(mu) - R(0) (stress incl. the -2/3 mu div v term, viscous work and heat flux, Re = 10)
    converges to the exact -div(-f^v) at order >= p - 1.5 (second-derivative terms under LDG).
    On the sheared mesh this also pins the metric terms (a transposed J^-1 fails). m = 4 is the
    collocation form (no anti-aliasing), which converges at the same orders on this smooth field;
    surf = True adds surface-flux anti-aliasing (full anti-aliasing). The curved mesh (trilinear
    hexahedra) pins the per-point metric terms: an element-constant metric fails it."""
    from tests.analytic_ns import rhs_function, state_function
    mach, mu = 0.3, 0.1
    state = state_function("wave", 1.4, mach)
    ex_inv = rhs_function("wave", 1.4, mach, 0.0, 0.71)
    ex_vis = rhs_function("wave", 1.4, mach, mu, 0.71)
    e_inv, e_vis = [], []
    for N in (8, 16):
        mesh = meshfn(N)
        o0 = O.Oracle(mesh, 3, m, mu=0.0, threads=os.cpu_count(), surf=surf)
        o1 = O.Oracle(mesh, 3, m, mu=mu, threads=os.cpu_count(), surf=surf)
        x = o0.sol_coords()
        U = W.to_layout(state(x), [(N ** 3, 64)])
        r0 = o0.rhs(U).reshape(N ** 3, 5, 64).transpose(1, 0, 2).reshape(5, -1)
        r1 = o1.rhs(U).reshape(N ** 3, 5, 64).transpose(1, 0, 2).reshape(5, -1)
        x0, x1 = ex_inv(x), ex_vis(x)
        e_inv.append(np.abs(r0 - x0).max(axis=1) / np.abs(x0).max(axis=1))
        dv, dx = (r1 - r0)[1:], (x1 - x0)[1:]
        e_vis.append(np.abs(dv - dx).max(axis=1) / np.abs(dx).max(axis=1))
    e_inv, e_vis = np.array(e_inv), np.array(e_vis)
    assert np.all(np.log2(e_inv[0] / e_inv[1]) > 2.5), e_inv
    assert np.all(e_inv[1] < 1e-2), e_inv
    assert np.all(np.log2(e_vis[0] / e_vis[1]) > 1.5), e_vis
    assert np.all(e_vis[1] < 0.1), e_vis


def test_tetrahedra_rhs_converges_to_analytic_navier_stokes():
    """Consistency of the tetrahedral discretisation (readings T1, T2) on the sheared Kuhn mesh,
    whose elements have full, non-diagonal Jacobians: on the compressible wave field of the hex test
    the inviscid RHS converges at order >= p - 0.5 and the viscous part at order >= p - 1.5 between
    8^3 and 16^3 cells (3,072 and 24,576 tetrahedra)."""
    from tests.analytic_ns import rhs_function, state_function
    mach, mu = 0.3, 0.1
    state = state_function("wave", 1.4, mach)
    ex_inv = rhs_function("wave", 1.4, mach, 0.0, 0.71)
    ex_vis = rhs_function("wave", 1.4, mach, mu, 0.71)
    e_inv, e_vis = [], []
    for N in (8, 16):
        mesh = W.box_tet_mesh(N, shear=True)
        ne = mesh["tet_v"].shape[0]
        o0 = O.Oracle(mesh, 3, 5, mu=0.0, threads=os.cpu_count())
        o1 = O.Oracle(mesh, 3, 5, mu=mu, threads=os.cpu_count())
        x = o0.sol_coords()
        U = W.to_layout(state(x), [(ne, 20)])
        r0 = o0.rhs(U).reshape(ne, 5, 20).transpose(1, 0, 2).reshape(5, -1)
        r1 = o1.rhs(U).reshape(ne, 5, 20).transpose(1, 0, 2).reshape(5, -1)
        x0, x1 = ex_inv(x), ex_vis(x)
        e_inv.append(np.abs(r0 - x0).max(axis=1) / np.abs(x0).max(axis=1))
        dv, dx = (r1 - r0)[1:], (x1 - x0)[1:]
        e_vis.append(np.abs(dv - dx).max(axis=1) / np.abs(dx).max(axis=1))
    e_inv, e_vis = np.array(e_inv), np.array(e_vis)
    assert np.all(np.log2(e_inv[0] / e_inv[1]) > 2.5), e_inv
    assert np.all(e_inv[1] < 0.05), e_inv
    assert np.all(np.log2(e_vis[0] / e_vis[1]) > 1.5), e_vis
    assert np.all(e_vis[1] < 0.5), e_vis


def test_pyramids_rhs_converges_to_analytic_navier_stokes():
    """Consistency of the pyramidal discretisation (readings P1-P3) on the box of cells split into
    six pyramids each: inviscid order >= p - 0.5 and viscous order >= p - 1.5 between 8^3 and 16^3
    cells (3,072 and 24,576 pyramids)."""
    from tests.analytic_ns import rhs_function, state_function
    mach, mu = 0.3, 0.1
    state = state_function("wave", 1.4, mach)
    ex_inv = rhs_function("wave", 1.4, mach, 0.0, 0.71)
    ex_vis = rhs_function("wave", 1.4, mach, mu, 0.71)
    e_inv, e_vis = [], []
    for N in (8, 16):
        mesh = W.box_pyr_mesh(N)
        ne = mesh["pyr_v"].shape[0]
        o0 = O.Oracle(mesh, 3, 5, mu=0.0, threads=os.cpu_count())
        o1 = O.Oracle(mesh, 3, 5, mu=mu, threads=os.cpu_count())
        x = o0.sol_coords()
        U = W.to_layout(state(x), [(ne, 30)])
        r0 = o0.rhs(U).reshape(ne, 5, 30).transpose(1, 0, 2).reshape(5, -1)
        r1 = o1.rhs(U).reshape(ne, 5, 30).transpose(1, 0, 2).reshape(5, -1)
        x0, x1 = ex_inv(x), ex_vis(x)
        e_inv.append(np.abs(r0 - x0).max(axis=1) / np.abs(x0).max(axis=1))
        dv, dx = (r1 - r0)[1:], (x1 - x0)[1:]
        e_vis.append(np.abs(dv - dx).max(axis=1) / np.abs(dx).max(axis=1))
    e_inv, e_vis = np.array(e_inv), np.array(e_vis)
    assert np.all(np.log2(e_inv[0] / e_inv[1]) > 2.5), e_inv
    assert np.all(e_inv[1] < 0.01), e_inv
    assert np.all(np.log2(e_vis[0] / e_vis[1]) > 1.5), e_vis
    assert np.all(e_vis[1] < 0.2), e_vis


def test_penalty_term_is_dissipative_energy_identity():
    """Reading G3 on hexahedra: the LDG penalty changes the RHS by a term whose GL-weighted inner
    product with the state is -tau sum_pairs int |n_s| |uL - uR|^2 dS <= 0 (catches the penalty's
    sign, its |n_s| scaling and the lift scaling)."""
    N, p = 3, 3
    mesh = W.sheared_box_mesh(N)
    o1 = O.Oracle(mesh, p, 5, tau=0.1)
    o0 = O.Oracle(mesh, p, 5, tau=0.0)
    U = _tgv(o1, mesh, perturb=2e-2)
    st = o1.rhs_stages(U)
    dR = st["R"] - o0.rhs(U)
    Wu = o1.op(0, "Wu")
    nu = 64
    inner = 0.0
    for e in range(N ** 3):
        _, _, det = o1.geometry(e)
        inner += det * (Wu[None, :] * U.reshape(-1, 5, nu)[e] * dR.reshape(-1, 5, nu)[e]).sum()
    # face side: GL weights on each face point; |n_s| from each element's metric
    L, R = o1.pairs()
    uf = st["uf"].reshape(-1, 5, 96)
    _, gw = O.gauss_legendre(p + 1)
    wface = np.outer(gw, gw).ravel(order="F")
    nref = o1.op(0, "nref")
    jump = 0.0
    for gl, gr in zip(L, R):
        eL, sL = divmod(gl, 96)
        eR, sR = divmod(gr, 96)
        J, Ji, det = o1.geometry(eL)
        ns = det * Ji.T @ nref[sL]
        jump += wface[sL % 16] * np.linalg.norm(ns) * ((uf[eL, :, sL] - uf[eR, :, sR]) ** 2).sum()
    assert jump > 0
    np.testing.assert_allclose(inner, -0.1 * jump, rtol=1e-9)


def test_rk4_damps_interface_jumps():
    """Stability (readings G3 and R4): 150 RK4 steps (dt = 2e-3) of a TGV with 1e-2 noise on 4^3,
    p=3 stay finite, the inter-element jump energy sum |uL - uR|^2 falls by more than 100x (an
    anti-dissipative penalty or Rusanov term makes it grow), and after the first acoustic transient
    the kinetic energy decreases monotonically."""
    mesh = W.box_hex_mesh(4)
    o = O.Oracle(mesh, 3, 5, threads=os.cpu_count())
    U = _tgv(o, mesh, perturb=1e-2)
    L, R = o.pairs()
    eL, sL = np.divmod(L, 96)
    eR, sR = np.divmod(R, 96)

    def jump(U):
        uf = o.rhs_stages(U)["uf"].reshape(-1, 5, 96)
        return ((uf[eL, :, sL] - uf[eR, :, sR]) ** 2).sum()

    js, ek = [jump(U)], [o.diagnostics(U)["Ek"]]
    for _ in range(15):
        U = o.rk4(U, 2e-3, 10)
        js.append(jump(U))
        ek.append(o.diagnostics(U)["Ek"])
    js, ek = np.array(js), np.array(ek)
    assert np.all(np.isfinite(js)) and js[-1] < 1e-2 * js[0]
    assert np.all(np.diff(ek[1:]) < 0)


def test_rk4_is_fourth_order_in_time():
    """The oracle's time integrator (Sec. 3, classical RK4): on the 2^3 box, p = 3, a TGV state
    advanced to T = 0.08 with 8, 16 and 32 steps against 256 steps; halving dt divides the error by
    about 2^4 = 16 (measured 17.5 and 16.8). A wrong stage weight or stage time drops the order to
    three or less (ratio <= 8)."""
    mesh = W.box_hex_mesh(2)
    o = O.Oracle(mesh, 3, 5, threads=os.cpu_count())
    U0 = _tgv(o, mesh, perturb=1e-3)
    T = 0.08
    ref = o.rk4(U0, T / 256, 256)
    err = [np.abs(o.rk4(U0, T / n, n) - ref).max() / np.abs(ref).max() for n in (8, 16, 32)]
    r1, r2 = err[0] / err[1], err[1] / err[2]
    assert 12.0 < r1 < 22.0 and 12.0 < r2 < 22.0, (err, r1, r2)


def test_self_periodic_pairing_rule():
    """Reading R5 on the 1^3 self-periodic hex: every face pairs with the opposite face of the same
    element and the smaller local face (the -x, -y, -z faces) is L."""
    o = O.Oracle(W.box_hex_mesh(1), 3, 5)
    L, R = o.pairs()
    assert len(L) == 48
    face = o.op(0, "fpt_face").astype(int)
    assert set(face[L]) == {0, 2, 4} and set(face[R]) == {1, 3, 5}
    xf = o.flux_coords()
    d = xf[L] - xf[R]
    d -= 2 * np.pi * np.round(d / (2 * np.pi))
    assert np.abs(d).max() < 1e-12


def test_split_hex_into_prisms_matches_hex_on_linear_fields():
    """A periodic 2^3 box of prisms (mixed mesh) and of hexes give the same RHS for a state that both
    represent exactly with zero interface jumps is too strong in general; instead, both must have
    zero RHS for a freestream and agree on total mass flux: sum W detJ R_rho = 0."""
    mesh = W.mixed_box_mesh(2)
    o = O.Oracle(mesh, 3, 5)
    U = _tgv(o, mesh, perturb=1e-2)
    d = o.diagnostics(U, o.rhs(U))
    assert abs(d["sums"][0]) <= 1e-12 * d["abs_sums"][0]
    assert abs(d["volume"] - (2 * np.pi) ** 3) < 1e-10


@pytest.mark.parametrize("name", ["hex16", "mixed4", "sheared3"])
def test_reference_pressure_is_an_identity(name):
    """Removing a constant p_ref from the momentum flux, in the volume and at interfaces, changes the
    RHS only by rounding on affine meshes (a constant flux has zero divergence and its common flux
    equals its own normal flux). Removing it from the volume flux alone would change the RHS by
    O(p_ref (p+1)^2/h); here the change must stay at the plain oracle's rounding floor."""
    mesh = {"hex16": lambda: W.box_hex_mesh(16), "mixed4": lambda: W.mixed_box_mesh(4),
            "sheared3": lambda: W.sheared_box_mesh(3)}[name]()
    p0 = W.tgv_p0()
    o0 = O.Oracle(mesh, 3, 5, threads=os.cpu_count())
    o1 = O.Oracle(mesh, 3, 5, threads=os.cpu_count(), p_ref=p0)
    U = _tgv(o0, mesh, perturb=1e-3)
    R0, R1 = o0.rhs(U), o1.rhs(U)
    blocks = _layout(o0, mesh)
    off = 0
    for ne, nu in blocks:
        n = ne * 5 * nu
        a, b = R0[off:off + n].reshape(ne, 5, nu), R1[off:off + n].reshape(ne, 5, nu)
        rel = np.abs(a - b).max(axis=(0, 2)) / np.abs(a).max(axis=(0, 2))
        assert rel.max() < 5e-12, rel
        off += n


@pytest.mark.parametrize("p", [3, 4])
def test_collocation_form_is_identity_quadrature(p):
    """Without anti-aliasing the flux is evaluated at the solution points: with m = p + 1 GL points
    the quadrature points are the solution points, so M7 (interpolation) and M8 (the L2 projection,
    exact because the n-point GL rule integrates degree 2p products) are the identity, and the RHS
    is the collocation form. Pinned against that definition (identity operators, quadrature points
    at the solution points) and freestream preservation."""
    mesh = W.box_hex_mesh(2)
    o = O.Oracle(mesh, p, p + 1)
    nu = (p + 1) ** 3
    np.testing.assert_allclose(o.op(0, "M7"), np.eye(nu), atol=1e-14)
    np.testing.assert_allclose(o.op(0, "M8"), np.eye(nu), atol=1e-13)
    np.testing.assert_allclose(o.op(0, "xq"), o.op(0, "xu"), atol=1e-15)
    # freestream and conservation hold in the collocation form too
    U = np.tile(np.array([1.1, 0.2, -0.3, 0.1, 180.0]).repeat(nu), 8)
    R = o.rhs(U)
    assert np.abs(R).max() <= 1e-13 * 180.0 * (2 / np.pi) * (p + 1) ** 2


# --- surface-flux anti-aliasing (hexahedra): flux points replaced by the m x m face quadrature
@pytest.mark.parametrize("p", [3, 4])
def test_surface_aa_lift_is_the_dg_lift_of_the_projected_face_data(p):
    """With the face quadrature points as flux points, the DG lift M3' = M^-1 E' (reading R3) must
    equal the n x n flux-point lift applied after the face L2 projection from the m x m GL points
    to the n x n GL points: M3'[z][q] = sum_s M3[z][s] P(s, q), P = Pj (x) Pj with
    Pj[i][a] = w_a l_i(x_a) / w_i. Both sides come from different constructions (face quadrature
    of Lagrange products vs. 1D GL weights), so a wrong node set, weight or face mapping fails."""
    mesh = W.box_hex_mesh(1)
    o = O.Oracle(mesh, p, p + 2)
    os_ = O.Oracle(mesh, p, p + 2, surf=True)
    n, m = p + 1, p + 2
    M3 = o.op(0, "lift")
    M3s = os_.op(0, "lift")
    assert M3s.shape == (n ** 3, 6 * m * m)
    x, w = O.gauss_legendre(n)
    xq, wq = O.gauss_legendre(m)
    L = np.array([[np.prod([(xa - x[j]) / (x[i] - x[j]) for j in range(n) if j != i]) for xa in xq] for i in range(n)])
    Pj = L * wq[None, :] / w[:, None]
    P2 = np.kron(Pj, Pj)    # [(i + n j)][(a + m b)] on one face
    for f in range(6):
        np.testing.assert_allclose(M3s[:, f * m * m:(f + 1) * m * m], M3[:, f * n * n:(f + 1) * n * n] @ P2, atol=1e-13)


@pytest.mark.parametrize("name", ["hex1_self_periodic", "hex3", "sheared3"])
def test_surface_aa_freestream_and_conservation(name):
    """Checks (a) and (e) with surface-flux anti-aliasing: a constant state gives a zero RHS, and the
    quadrature-weighted RHS of a perturbed TGV sums to zero."""
    mesh = MESHES[name]()
    o = O.Oracle(mesh, 3, 5, surf=True)
    blocks = _layout(o, mesh)
    U = np.concatenate([np.tile(np.repeat(FREESTREAM, npt), ne) for ne, npt in blocks])
    N = round(mesh["verts"].shape[0] ** (1.0 / 3.0)) - 1
    assert np.abs(o.rhs(U)).max() < 1e-13 * 1.1 * (2.0 / (2 * np.pi / N)) * 16
    U = _tgv(o, mesh, perturb=1e-2)
    d = o.diagnostics(U, o.rhs(U))
    assert np.all(np.abs(d["sums"]) <= 1e-12 * d["abs_sums"])


def test_surface_aa_leaves_the_corrected_gradient_unchanged():
    """The common solution is linear in the two traces, and the traces are polynomials of degree p
    that the m x m face points interpolate and the face projection recovers exactly; so moving the
    interface terms to the face quadrature points leaves the corrected gradient unchanged (to
    rounding) and changes only the common flux. On the perturbed TGV the RHS does change (the
    interface quadrature of the nonlinear flux), while the common solution at the face quadrature
    points is the n x n common solution interpolated there."""
    mesh = W.sheared_box_mesh(3)
    o = O.Oracle(mesh, 3, 5)
    os_ = O.Oracle(mesh, 3, 5, surf=True)
    U = _tgv(o, mesh, perturb=1e-2)
    a, b = o.rhs_stages(U), os_.rhs_stages(U)
    scale = np.abs(a["qu"]).max()
    np.testing.assert_allclose(b["qu"], a["qu"], atol=1e-12 * scale)
    n, m = 4, 5
    x, w = O.gauss_legendre(n)
    xq, _ = O.gauss_legendre(m)
    B = np.array([[np.prod([(xa - x[j]) / (x[i] - x[j]) for j in range(n) if j != i]) for i in range(n)] for xa in xq])
    B2 = np.kron(B, B)      # [(a + m b)][(i + n j)]
    ne = 27
    cf = a["cf"].reshape(ne, 5, 6, n * n)
    cfs = b["cf"].reshape(ne, 5, 6, m * m)
    np.testing.assert_allclose(cfs, np.einsum("qs,evfs->evfq", B2, cf), atol=1e-12 * np.abs(cf).max())
    dR = np.abs(a["R"] - b["R"]).max() / np.abs(a["R"]).max()
    assert 1e-9 < dR < 1e-1, dR


def test_golden_dissipation_rate_matches_the_oracle_as_it_stands():
    """tests/golden/eps_tgv32_p4.txt (written by make_eps_32p4.py) holds the oracle's kinetic energy
    and dissipation rate of the 32^3 p = 4 sweep at step 0 and after 100 RK4 steps. The step-0 row
    must be what the oracle computes now (one RHS), so the stored trajectory cannot go stale after an
    oracle change unnoticed; the rates are near the closed form eps(0) = 3 mu / 4 (the 1e-3
    perturbation adds dissipation) and E_k near 1/8; both stored rates are positive and E_k decays."""
    path = os.path.join(os.path.dirname(__file__), "golden", "eps_tgv32_p4.txt")
    rows = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, ek, eps = line.split()
                rows[int(k)] = (float(ek), float(eps))
    assert set(rows) == {0, 100}
    mesh = W.box_hex_mesh(32)
    o = O.Oracle(mesh, 4, 6, threads=os.cpu_count(), p_ref=W.tgv_p0())
    U = W.tgv_state(o.sol_coords(), [(32 ** 3, 125)], perturb=1e-3)
    d = o.diagnostics(U, o.rhs(U))
    assert abs(d["Ek"] / rows[0][0] - 1) <= 1e-13 and abs(d["eps"] / rows[0][1] - 1) <= 1e-11, (d, rows[0])
    assert abs(rows[0][0] - 0.125) < 1e-3 and 0.75 / 1600 < rows[0][1] < 2 * 0.75 / 1600
    assert rows[100][0] < rows[0][0] and rows[100][1] > 0
