/*
 * fr_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 reference ("the oracle") for one right-hand-side (RHS) evaluation of the
 * flux-reconstruction (FR) discretisation of the compressible Navier-Stokes equations with flux
 * anti-aliasing (over-integration of the flux at element quadrature points), on affine or trilinear
 * hexahedra, affine prisms, tetrahedra and pyramids, plus the classical RK4 step around it.
 *
 * Only the test-suite, the package smoke check and the CPU-baseline leg of the benchmark may load
 * the library built from this file. It shares no code with the GPU library.
 *
 * How it follows the paper (Akkurt, Witherden, Vincent, "Cache blocking for flux reconstruction:
 * extension to Navier-Stokes equations and anti-aliasing"):
 *   - operators are DENSE per element type, built from a modal orthonormal basis and a nodal
 *     Vandermonde matrix (Sec. 2.2 operator definitions M0..M10); there is no sum factorisation;
 *   - one loop per paper kernel, in the paper's execution order (Sec. 3):
 *       disu, con_u, tgradpcoru, tgradcoru, gradcoru, gradcoru_fpts, gradcoru_qpts, uqpts,
 *       tdisf, tdivtpcorf, comm_flux, tdivtconf, negdivconf.
 *
 * Readings where the paper is silent or garbled (each one stated where it is used):
 *   G1  temperature T = p/(rho R); the heat flux is mu*gamma/((gamma-1)Pr) grad(p/rho).
 *   G3  the LDG penalty tau(uL-uR) is dissipative in the total flux f = fe - fv.
 *   G4  M7 is Nq x Nu and M8 is Nu x Nq (the index definitions, not the printed dims).
 *   G5  the gradient is of the physical solution u (equivalent for affine elements).
 *   R2  hex flux points: n x n Gauss-Legendre (GL) points per face. With surface-flux
 *       anti-aliasing (Sec. 2.2.1: the flux points at the interfaces are replaced by quadrature
 *       points) they are the m x m GL points of the face quadrature instead; every flux-point
 *       operator (M0, M3, M6, M2) then follows from the same definitions.
 *   R3  correction functions are the DG-equivalent ones: lift = M^-1 E with the exact mass
 *       matrix M and E = int_face l_zeta l^face_sigma dS (reference measure).
 *   R4  Rusanov: F = 1/2 n.(fe_L + fe_R) + 1/2 s (uL - uR), s = max(|vL.n|+cL, |vR.n|+cR).
 *   R5  the L side of a flux-point pair is the element with the smaller global index (hexes
 *       before prisms before tetrahedra before pyramids); a self-pair takes the smaller local face
 *       number as L.
 *   R6  transformed common flux D = |n_s| F with n_s = detJ J^-T n~; each side uses its own |n_s|.
 *   R7  prism solution points: the paper's Williams-Shunn triangle points x GL points in z.
 *   R8  prism quadrature: collapsed (Duffy) k x k GL triangle rule x m GL points in z.
 *   R11 orthonormal bases: normalised Legendre on lines; Gram-Schmidt of monomials on triangles
 *       and tetrahedra.
 *   T1  tetrahedra (Sec. 1 lists them among the supported types, with dense operators; the paper
 *       prints no point set for them): solution points are the order-p equispaced lattice shrunk by
 *       4/5 towards the centroid; each triangular face carries the printed Williams-Shunn triangle
 *       points (so p = 2, 3). With the DG-equivalent lift and the L2 projection of the flux, the RHS
 *       as a polynomial does not depend on the solution points, only its rounding does.
 *   C1  curved (non-affine) hexahedra (gradcoru reads per-point metric terms J^(u) in the
 *       appendix's data-movement table): the trilinear map of the 8 vertices; J^-T at each solution point for the gradient,
 *       det J J^-1 at each quadrature point for the flux, n_s = det J J^-T n~ at each flux point,
 *       R = -R~ / det J at each solution point. Prisms and tetrahedra stay affine.
 *   P1  pyramids (named in Sec. 1; no space or points printed): the rational pyramid space spanned by
 *       a^i b^j (1-c)^max(i,j) c^k in the collapsed coordinates (Q_p on the base, P_p on the
 *       triangles, so it conforms with hexahedra and tetrahedra); solution points: the order-p
 *       pyramid lattice shrunk by 4/5 towards the centroid; flux points: n x n GL points on the base,
 *       the printed Williams-Shunn triangle points on the four triangles (so p = 2, 3).
 *   P3  pyramid derivative: the space is not closed under differentiation (d/dx of a b (1-c) is
 *       2b, outside it), so the derivative operator is the L2 projection of the exact derivative,
 *       M^-1 int l_zeta d l_nu; with it the DG-equivalent scheme stays conservative (the nodal
 *       derivative would not integrate to the boundary flux). On the polynomial spaces of the
 *       other types the projection is the identity, so the nodal derivative is kept there.
 *   P2  pyramid quadrature: collapsed m^3 rule (GL in a and b, the Gauss rule of (1-c)^2 in c),
 *       exact to total degree 2m-1.
 *   T2  tetrahedron quadrature: collapsed m x m x m rule (GL in a, Gauss rules of the weights
 *       (1-b) and (1-c)^2 in b and c), exact to total degree 2m-1 -- with m = p + 2 the same
 *       degree 2p+3 that m GL points give per direction on the hexahedron.
 *
 * Parity pins: see tests/test_oracle_*.py. Parity for the prism and tetrahedron elements and for
 * the R4/R5 readings is pinned by invariants and identities (freestream, conservation, polynomial
 * exactness, integration by parts, grid convergence), not by printed values.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 5
#define ND 3

/* ---------------------------------------------------------------------------------------------
 * Small dense linear algebra
 * ------------------------------------------------------------------------------------------- */

/* In-place inverse of the n x n row-major matrix a by Gauss-Jordan elimination with partial
 * pivoting. Returns 0 on success, -1 if the matrix is numerically singular. */
static int mat_inverse(int n, double *a)
{
    double *b = (double *)calloc((size_t)n * 2 * n, sizeof(double));
    int w = 2 * n;
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) b[i * w + j] = a[i * n + j];
        b[i * w + n + i] = 1.0;
    }
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(b[r * w + c]) > fabs(b[piv * w + c])) piv = r;
        if (fabs(b[piv * w + c]) < 1e-300) { free(b); return -1; }
        if (piv != c)
            for (int j = 0; j < w; j++) { double t = b[c * w + j]; b[c * w + j] = b[piv * w + j]; b[piv * w + j] = t; }
        double d = b[c * w + c];
        for (int j = 0; j < w; j++) b[c * w + j] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            double f = b[r * w + c];
            if (f == 0.0) continue;
            for (int j = 0; j < w; j++) b[r * w + j] -= f * b[c * w + j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) a[i * n + j] = b[i * w + n + j];
    free(b);
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * One-dimensional building blocks
 * ------------------------------------------------------------------------------------------- */

/* Legendre polynomials P_0..P_n and their derivatives at x, from the three-term recurrence
 * (r+1) P_{r+1} = (2r+1) x P_r - r P_{r-1} and P'_{r+1} = P'_{r-1} + (2r+1) P_r. */
static void legendre_all(int n, double x, double *P, double *dP)
{
    P[0] = 1.0; dP[0] = 0.0;
    if (n >= 1) { P[1] = x; dP[1] = 1.0; }
    for (int r = 1; r < n; r++) {
        P[r + 1] = ((2 * r + 1) * x * P[r] - r * P[r - 1]) / (r + 1);
        dP[r + 1] = dP[r - 1] + (2 * r + 1) * P[r];
    }
}

/* n-point Gauss-Legendre rule on [-1,1]: nodes are the roots of P_n (Newton iteration from a
 * cosine guess), weights 2/((1-x^2) P_n'(x)^2). Nodes are returned in increasing order. */
void or_gauss_legendre(int n, double *x, double *w)
{
    double P[64], dP[64];
    for (int i = 0; i < n; i++) {
        double r = -cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; it++) {
            legendre_all(n, r, P, dP);
            double dr = P[n] / dP[n];
            r -= dr;
            if (fabs(dr) < 1e-16) break;
        }
        legendre_all(n, r, P, dP);
        x[i] = r;
        w[i] = 2.0 / ((1.0 - r * r) * dP[n] * dP[n]);
    }
}

/* Lagrange basis polynomial a on the nodes xs[0..n-1], evaluated at x (product formula). */
static double lagrange1d(int n, const double *xs, int a, double x)
{
    double v = 1.0;
    for (int b = 0; b < n; b++)
        if (b != a) v *= (x - xs[b]) / (xs[a] - xs[b]);
    return v;
}

static double ipow(double x, int k) { double v = 1.0; for (int i = 0; i < k; i++) v *= x; return v; }

/* Collapsed (Duffy) k x k rule on the reference triangle (-1,-1),(1,-1),(-1,1):
 * x = (1+a)(1-b)/2 - 1, y = b, weight w_a w_b (1-b)/2, exact for total degree 2k-2.
 * Point index ia + k*ib. */
void or_tri_rule(int k, double *xy, double *w)
{
    double g[32], gw[32];
    or_gauss_legendre(k, g, gw);
    for (int ib = 0; ib < k; ib++)
        for (int ia = 0; ia < k; ia++) {
            int q = ia + k * ib;
            double a = g[ia], b = g[ib];
            xy[2 * q + 0] = 0.5 * (1.0 + a) * (1.0 - b) - 1.0;
            xy[2 * q + 1] = b;
            w[q] = gw[ia] * gw[ib] * 0.5 * (1.0 - b);
        }
}

/* n-point Gauss rule for the weight (1-x)^alpha on [-1,1] (reading T2 uses alpha = 0, 1, 2).
 * The nodes are the roots of the degree-n polynomial orthogonal under that weight: it is built by
 * Gram-Schmidt of the Legendre polynomials P_0..P_n with inner products from a 40-point GL rule
 * (exact for these integrands), its n roots are bracketed on a fine grid and bisected; the weights
 * are those of the interpolatory rule on the nodes, w_j = int (1-x)^alpha l_j(x) dx. Returns 0, or
 * -1 if the n roots were not all found. Nodes in increasing order. */
int or_gauss_jacobi(int n, int alpha, double *x, double *w)
{
    enum { NG = 40 };
    double g[NG], gw[NG], wt[NG], P[64], dP[64];
    if (n < 1 || n > 16) return -1;
    or_gauss_legendre(NG, g, gw);
    for (int q = 0; q < NG; q++) wt[q] = gw[q] * ipow(1.0 - g[q], alpha);
    /* c[k][r]: polynomial k = sum_r c[k][r] P_r, orthogonal under the weight */
    double c[17][17], val[17][NG];
    memset(c, 0, sizeof c);
    for (int k = 0; k <= n; k++) {
        c[k][k] = 1.0;
        for (int q = 0; q < NG; q++) { legendre_all(k, g[q], P, dP); val[k][q] = P[k]; }
        for (int pass = 0; pass < 2; pass++)
            for (int j = 0; j < k; j++) {
                double ip = 0, nj = 0;
                for (int q = 0; q < NG; q++) { ip += wt[q] * val[k][q] * val[j][q]; nj += wt[q] * val[j][q] * val[j][q]; }
                double f = ip / nj;
                for (int r = 0; r <= n; r++) c[k][r] -= f * c[j][r];
                for (int q = 0; q < NG; q++) val[k][q] -= f * val[j][q];
            }
    }
    /* the roots of polynomial n */
    const int NS = 20000;
    int found = 0;
    double xa = -1.0, fa;
    legendre_all(n, xa, P, dP);
    fa = 0; for (int r = 0; r <= n; r++) fa += c[n][r] * P[r];
    for (int i = 1; i <= NS && found < n; i++) {
        double xb = -1.0 + 2.0 * i / NS, fb = 0;
        legendre_all(n, xb, P, dP);
        for (int r = 0; r <= n; r++) fb += c[n][r] * P[r];
        if ((fa < 0) != (fb < 0)) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200 && hi - lo > 0; it++) {
                double mid = 0.5 * (lo + hi), fm = 0;
                if (mid <= lo || mid >= hi) break;
                legendre_all(n, mid, P, dP);
                for (int r = 0; r <= n; r++) fm += c[n][r] * P[r];
                if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
            }
            x[found++] = 0.5 * (lo + hi);
        }
        xa = xb; fa = fb;
    }
    if (found != n) return -1;
    for (int j = 0; j < n; j++) {
        double v = 0;
        for (int q = 0; q < NG; q++) v += wt[q] * lagrange1d(n, x, j, g[q]);
        w[j] = v;
    }
    return 0;
}

/* Collapsed (Duffy) k x k x k rule on the reference tetrahedron (-1,-1,-1), (1,-1,-1), (-1,1,-1),
 * (-1,-1,1) (reading T2): for a, b, c in [-1,1], x = (1+a)(1-b)(1-c)/4 - 1, y = (1+b)(1-c)/2 - 1,
 * z = c, with Jacobian (1-b)(1-c)^2/8; a takes the k-point GL rule, b and c the k-point Gauss rules
 * of the weights (1-b) and (1-c)^2. A polynomial of total degree d in (x,y,z) is of degree <= d in
 * each of a, b, c, so the rule is exact for d <= 2k-1. Point index ia + k ib + k^2 ic. */
int or_tet_rule(int k, double *xyz, double *w)
{
    double ga[32], wa[32], gb[32], wb[32], gc[32], wc[32];
    if (k < 1 || k > 16) return -1;
    or_gauss_legendre(k, ga, wa);
    if (or_gauss_jacobi(k, 1, gb, wb) || or_gauss_jacobi(k, 2, gc, wc)) return -1;
    for (int ic = 0; ic < k; ic++)
        for (int ib = 0; ib < k; ib++)
            for (int ia = 0; ia < k; ia++) {
                int q = ia + k * ib + k * k * ic;
                double a = ga[ia], b = gb[ib], c = gc[ic];
                xyz[3 * q + 0] = 0.25 * (1.0 + a) * (1.0 - b) * (1.0 - c) - 1.0;
                xyz[3 * q + 1] = 0.5 * (1.0 + b) * (1.0 - c) - 1.0;
                xyz[3 * q + 2] = c;
                w[q] = wa[ia] * wb[ib] * wc[ic] / 8.0;
            }
    return 0;
}

/* Tetrahedron solution points (reading T1): the equispaced lattice of order p, (a, b, c)/p with
 * a + b + c <= p, mapped onto the reference tetrahedron and shrunk by the factor 4/5 towards its
 * centroid (-1/2, -1/2, -1/2), so that every point is interior. The set keeps the tetrahedron's
 * symmetries and is unisolvent for P_p (an affine image of the lattice). Index order: a fastest,
 * then b, then c. Returns the count (p+1)(p+2)(p+3)/6. */
int or_tet_solution_points(int p, double *xyz)
{
    const double s = 0.8;
    int k = 0;
    for (int c = 0; c <= p; c++)
        for (int b = 0; b <= p - c; b++)
            for (int a = 0; a <= p - b - c; a++) {
                double X[3] = {-1.0 + 2.0 * a / p, -1.0 + 2.0 * b / p, -1.0 + 2.0 * c / p};
                for (int d = 0; d < 3; d++) xyz[3 * k + d] = -0.5 + s * (X[d] + 0.5);
                k++;
            }
    return k;
}

/* Williams-Shunn triangle solution points as printed in the paper's prism figures
 * (Fig. "Solution points for prism elements with polynomial orders p=2 and p=3"). */
static const double WS_P2[6][2] = {
    {-0.81684757298044, 0.63369514596088},   {0.63369514596088, -0.81684757298044},
    {-0.81684757298044, -0.81684757298044},  {-0.108103018168072, -0.783793963663856},
    {-0.783793963663856, -0.108103018168072}, {-0.108103018168072, -0.108103018168072}};
static const double WS_P3[10][2] = {
    {-0.333333333333333, -0.333333333333333}, {-0.888871894660414, 0.777743789320828},
    {0.777743789320828, -0.888871894660414},  {-0.888871894660414, -0.888871894660414},
    {0.268421495491446, -0.408932576528214},  {-0.859488918963232, -0.408932576528214},
    {-0.408932576528214, -0.859488918963232}, {0.268421495491446, -0.859488918963232},
    {-0.859488918963232, 0.268421495491446},  {-0.408932576528214, 0.268421495491446}};

/* Copies the printed triangle points for order p into xy; returns the count or -1. */
int or_tri_solution_points(int p, double *xy)
{
    if (p == 2) { memcpy(xy, WS_P2, sizeof(WS_P2)); return 6; }
    if (p == 3) { memcpy(xy, WS_P3, sizeof(WS_P3)); return 10; }
    return -1;
}

/* Collapsed k x k x k rule on the reference pyramid (base [-1,1]^2 at z = -1, apex (0,0,1); reading
 * P2): x = a(1-c)/2, y = b(1-c)/2, z = c with Jacobian (1-c)^2/4; a and b take the k-point GL rule,
 * c the k-point Gauss rule of the weight (1-c)^2. A polynomial of total degree d in (x,y,z), and a
 * product of two functions of the pyramid space of order <= d/2, are polynomials of degree <= d in
 * each of a, b, c, so the rule is exact for d <= 2k-1. Index ia + k ib + k^2 ic. */
int or_pyr_rule(int k, double *xyz, double *w)
{
    double ga[32], wa[32], gc[32], wc[32];
    if (k < 1 || k > 16) return -1;
    or_gauss_legendre(k, ga, wa);
    if (or_gauss_jacobi(k, 2, gc, wc)) return -1;
    for (int ic = 0; ic < k; ic++)
        for (int ib = 0; ib < k; ib++)
            for (int ia = 0; ia < k; ia++) {
                int q = ia + k * ib + k * k * ic;
                double c = gc[ic];
                xyz[3 * q + 0] = 0.5 * ga[ia] * (1.0 - c);
                xyz[3 * q + 1] = 0.5 * ga[ib] * (1.0 - c);
                xyz[3 * q + 2] = c;
                w[q] = wa[ia] * wa[ib] * wc[ic] / 4.0;
            }
    return 0;
}

/* Pyramid solution points (reading P1): the pyramid lattice of order p -- layer k = 0..p at
 * z = -1 + 2k/p holds the (p+1-k)^2 points x, y = (1 - k/p)(-1 + 2i/(p-k)) (the apex for k = p) --
 * shrunk by 4/5 towards the centroid (0, 0, -1/2), so every point is interior. Index order: i
 * fastest (x), then j (y), then the layer k. Returns the count (p+1)(p+2)(2p+3)/6. */
int or_pyr_solution_points(int p, double *xyz)
{
    const double s = 0.8;
    int n = 0;
    for (int k = 0; k <= p; k++) {
        int m = p - k;
        double z = -1.0 + 2.0 * k / p, h = 1.0 - (double)k / p;
        for (int j = 0; j <= m; j++)
            for (int i = 0; i <= m; i++) {
                double X[3] = {m ? h * (-1.0 + 2.0 * i / m) : 0.0, m ? h * (-1.0 + 2.0 * j / m) : 0.0, z};
                xyz[3 * n + 0] = s * X[0];
                xyz[3 * n + 1] = s * X[1];
                xyz[3 * n + 2] = -0.5 + s * (X[2] + 0.5);
                n++;
            }
    }
    return n;
}

/* ---------------------------------------------------------------------------------------------
 * Orthonormal modal bases (reading R11)
 * ------------------------------------------------------------------------------------------- */

typedef struct {
    int p, nt;          /* order, number of triangle modes (p+1)(p+2)/2 */
    int *mi, *mj;       /* monomial exponents x^i y^j, graded order */
    double *c;          /* [nt][nt] coefficients: phi_t = sum_k c[t][k] x^mi[k] y^mj[k] */
} tri_basis;


static void tri_basis_eval(const tri_basis *tb, double x, double y, double *phi, double *dphx, double *dphy)
{
    for (int t = 0; t < tb->nt; t++) {
        double v = 0, vx = 0, vy = 0;
        for (int k = 0; k < tb->nt; k++) {
            int i = tb->mi[k], j = tb->mj[k];
            double ck = tb->c[t * tb->nt + k];
            v += ck * ipow(x, i) * ipow(y, j);
            if (i > 0) vx += ck * i * ipow(x, i - 1) * ipow(y, j);
            if (j > 0) vy += ck * j * ipow(x, i) * ipow(y, j - 1);
        }
        phi[t] = v;
        if (dphx) dphx[t] = vx;
        if (dphy) dphy[t] = vy;
    }
}

/* Gram-Schmidt (modified, two passes) of the monomials x^i y^j, i+j <= p, under the collapsed
 * rule of strength 2p+2 on the reference triangle. */
static void tri_basis_init(tri_basis *tb, int p)
{
    int nt = (p + 1) * (p + 2) / 2;
    tb->p = p; tb->nt = nt;
    tb->mi = (int *)malloc(nt * sizeof(int));
    tb->mj = (int *)malloc(nt * sizeof(int));
    tb->c = (double *)calloc((size_t)nt * nt, sizeof(double));
    int k = 0;
    for (int d = 0; d <= p; d++)
        for (int i = d; i >= 0; i--) { tb->mi[k] = i; tb->mj[k] = d - i; k++; }
    int kq = p + 2, nq = kq * kq;
    double *xy = (double *)malloc(2 * nq * sizeof(double)), *w = (double *)malloc(nq * sizeof(double));
    or_tri_rule(kq, xy, w);
    double *val = (double *)malloc((size_t)nt * nq * sizeof(double)); /* values of current vectors */
    for (int t = 0; t < nt; t++) {
        double *ct = tb->c + t * nt;
        ct[t] = 1.0;
        for (int q = 0; q < nq; q++) val[t * nq + q] = ipow(xy[2 * q], tb->mi[t]) * ipow(xy[2 * q + 1], tb->mj[t]);
        for (int pass = 0; pass < 2; pass++)
            for (int s = 0; s < t; s++) {
                double ip = 0;
                for (int q = 0; q < nq; q++) ip += w[q] * val[t * nq + q] * val[s * nq + q];
                for (int kk = 0; kk < nt; kk++) ct[kk] -= ip * tb->c[s * nt + kk];
                for (int q = 0; q < nq; q++) val[t * nq + q] -= ip * val[s * nq + q];
            }
        double nrm = 0;
        for (int q = 0; q < nq; q++) nrm += w[q] * val[t * nq + q] * val[t * nq + q];
        nrm = sqrt(nrm);
        for (int kk = 0; kk < nt; kk++) ct[kk] /= nrm;
        for (int q = 0; q < nq; q++) val[t * nq + q] /= nrm;
    }
    free(xy); free(w); free(val);
}

static void tri_basis_free(tri_basis *tb) { free(tb->mi); free(tb->mj); free(tb->c); }

/* Orthonormal basis of P_p on the reference tetrahedron (volume 4/3): Gram-Schmidt (modified, two
 * passes) of the monomials x^i y^j z^l, i+j+l <= p in graded order, under the collapsed rule with
 * p + 2 points per direction (strength 2p+3 >= 2p). */
typedef struct {
    int p, nt;
    int *e;             /* [nt][3] monomial exponents */
    double *c;          /* [nt][nt] coefficients: phi_t = sum_k c[t][k] x^e[k][0] y^e[k][1] z^e[k][2] */
} tet_basis;

static void tet_basis_eval(const tet_basis *tb, const double *X, double *phi, double *dphi /* [3][nt] or NULL */)
{
    int nt = tb->nt;
    for (int t = 0; t < nt; t++) {
        double v = 0, g[3] = {0, 0, 0};
        for (int k = 0; k < nt; k++) {
            const int *e = tb->e + 3 * k;
            double ck = tb->c[t * nt + k];
            v += ck * ipow(X[0], e[0]) * ipow(X[1], e[1]) * ipow(X[2], e[2]);
            for (int d = 0; d < 3; d++) {
                if (e[d] == 0) continue;
                double m = ck * e[d];
                for (int dd = 0; dd < 3; dd++) m *= ipow(X[dd], dd == d ? e[dd] - 1 : e[dd]);
                g[d] += m;
            }
        }
        phi[t] = v;
        if (dphi) for (int d = 0; d < 3; d++) dphi[d * nt + t] = g[d];
    }
}

static int tet_basis_init(tet_basis *tb, int p)
{
    int nt = (p + 1) * (p + 2) * (p + 3) / 6;
    tb->p = p; tb->nt = nt;
    tb->e = (int *)malloc(3 * nt * sizeof(int));
    tb->c = (double *)calloc((size_t)nt * nt, sizeof(double));
    int k = 0;
    for (int d = 0; d <= p; d++)
        for (int i = d; i >= 0; i--)
            for (int j = d - i; j >= 0; j--) { tb->e[3 * k] = i; tb->e[3 * k + 1] = j; tb->e[3 * k + 2] = d - i - j; k++; }
    int kq = p + 2, nq = kq * kq * kq;
    double *xyz = (double *)malloc(3 * nq * sizeof(double)), *w = (double *)malloc(nq * sizeof(double));
    if (or_tet_rule(kq, xyz, w)) { free(xyz); free(w); return -1; }
    double *val = (double *)malloc((size_t)nt * nq * sizeof(double));
    for (int t = 0; t < nt; t++) {
        double *ct = tb->c + t * nt;
        const int *e = tb->e + 3 * t;
        ct[t] = 1.0;
        for (int q = 0; q < nq; q++)
            val[t * nq + q] = ipow(xyz[3 * q], e[0]) * ipow(xyz[3 * q + 1], e[1]) * ipow(xyz[3 * q + 2], e[2]);
        for (int pass = 0; pass < 2; pass++)
            for (int s = 0; s < t; s++) {
                double ip = 0;
                for (int q = 0; q < nq; q++) ip += w[q] * val[t * nq + q] * val[s * nq + q];
                for (int kk = 0; kk < nt; kk++) ct[kk] -= ip * tb->c[s * nt + kk];
                for (int q = 0; q < nq; q++) val[t * nq + q] -= ip * val[s * nq + q];
            }
        double nrm = 0;
        for (int q = 0; q < nq; q++) nrm += w[q] * val[t * nq + q] * val[t * nq + q];
        nrm = sqrt(nrm);
        for (int kk = 0; kk < nt; kk++) ct[kk] /= nrm;
        for (int q = 0; q < nq; q++) val[t * nq + q] /= nrm;
    }
    free(xyz); free(w); free(val);
    return 0;
}

static void tet_basis_free(tet_basis *tb) { free(tb->e); free(tb->c); }

/* Orthonormal basis of the pyramid space of order p (reading P1): the span of the functions
 * g_ijk = a^i b^j (1-c)^max(i,j) c^k, 0 <= i, j <= p, 0 <= k <= p - max(i,j), in the collapsed
 * coordinates a = 2x/(1-z), b = 2y/(1-z), c = z -- rational in (x, y, z), with Q_p traces on the
 * base and P_p traces on the triangular faces; (p+1)(p+2)(2p+3)/6 functions. Gram-Schmidt
 * (modified, two passes) under the collapsed rule with p + 2 points per direction, exact for the
 * products (degree <= 2p in each collapsed coordinate). */
typedef struct {
    int p, nt;
    int *e;             /* [nt][3] exponents (i, j, k) */
    double *c;          /* [nt][nt] coefficients over the generators */
} pyr_basis;

/* Generator g_ijk and its (x, y, z) gradient at X (interior: z < 1). */
static void pyr_gen(const int *e, const double *X, double *g, double *dg)
{
    const double om = 1.0 - X[2], a = 2.0 * X[0] / om, b = 2.0 * X[1] / om, c = X[2];
    const int i = e[0], j = e[1], k = e[2], mm = i > j ? i : j;
    const double ai = ipow(a, i), bj = ipow(b, j), cm = ipow(om, mm), ck = ipow(c, k);
    *g = ai * bj * cm * ck;
    if (!dg) return;
    const double ga = i ? i * ipow(a, i - 1) * bj * cm * ck : 0.0;
    const double gb = j ? j * ai * ipow(b, j - 1) * cm * ck : 0.0;
    double gc = 0.0;
    if (mm) gc -= mm * ai * bj * ipow(om, mm - 1) * ck;
    if (k) gc += ai * bj * cm * k * ipow(c, k - 1);
    dg[0] = ga * 2.0 / om;
    dg[1] = gb * 2.0 / om;
    dg[2] = (ga * a + gb * b) / om + gc;
}

static void pyr_basis_eval(const pyr_basis *pb, const double *X, double *phi, double *dphi /* [3][nt] or NULL */)
{
    int nt = pb->nt;
    double g[64], dg[3 * 64];
    for (int k = 0; k < nt; k++) pyr_gen(pb->e + 3 * k, X, &g[k], dphi ? &dg[3 * k] : NULL);
    for (int t = 0; t < nt; t++) {
        double v = 0, d0 = 0, d1 = 0, d2 = 0;
        for (int k = 0; k < nt; k++) {
            double ck = pb->c[t * nt + k];
            v += ck * g[k];
            if (dphi) { d0 += ck * dg[3 * k]; d1 += ck * dg[3 * k + 1]; d2 += ck * dg[3 * k + 2]; }
        }
        phi[t] = v;
        if (dphi) { dphi[t] = d0; dphi[nt + t] = d1; dphi[2 * nt + t] = d2; }
    }
}

static int pyr_basis_init(pyr_basis *pb, int p)
{
    int nt = (p + 1) * (p + 2) * (2 * p + 3) / 6;
    if (nt > 64) return -1;
    pb->p = p; pb->nt = nt;
    pb->e = (int *)malloc(3 * nt * sizeof(int));
    pb->c = (double *)calloc((size_t)nt * nt, sizeof(double));
    int n = 0;
    for (int mm = 0; mm <= p; mm++)          /* graded by max(i,j), then k */
        for (int k = 0; k <= p - mm; k++)
            for (int j = 0; j <= mm; j++)
                for (int i = 0; i <= mm; i++) {
                    if ((i > j ? i : j) != mm) continue;
                    pb->e[3 * n] = i; pb->e[3 * n + 1] = j; pb->e[3 * n + 2] = k;
                    n++;
                }
    int kq = p + 2, nq = kq * kq * kq;
    double *xyz = (double *)malloc(3 * nq * sizeof(double)), *w = (double *)malloc(nq * sizeof(double));
    if (or_pyr_rule(kq, xyz, w)) { free(xyz); free(w); return -1; }
    double *val = (double *)malloc((size_t)nt * nq * sizeof(double));
    for (int t = 0; t < nt; t++) {
        double *ct = pb->c + t * nt;
        ct[t] = 1.0;
        for (int q = 0; q < nq; q++) pyr_gen(pb->e + 3 * t, xyz + 3 * q, &val[t * nq + q], NULL);
        for (int pass = 0; pass < 2; pass++)
            for (int s2 = 0; s2 < t; s2++) {
                double ip = 0;
                for (int q = 0; q < nq; q++) ip += w[q] * val[t * nq + q] * val[s2 * nq + q];
                for (int kk = 0; kk < nt; kk++) ct[kk] -= ip * pb->c[s2 * nt + kk];
                for (int q = 0; q < nq; q++) val[t * nq + q] -= ip * val[s2 * nq + q];
            }
        double nrm = 0;
        for (int q = 0; q < nq; q++) nrm += w[q] * val[t * nq + q] * val[t * nq + q];
        nrm = sqrt(nrm);
        for (int kk = 0; kk < nt; kk++) ct[kk] /= nrm;
        for (int q = 0; q < nq; q++) val[t * nq + q] /= nrm;
    }
    free(xyz); free(w); free(val);
    return 0;
}

static void pyr_basis_free(pyr_basis *pb) { free(pb->e); free(pb->c); }

/* ---------------------------------------------------------------------------------------------
 * Element types and their dense operators
 * ------------------------------------------------------------------------------------------- */

enum { ET_HEX = 0, ET_PRI = 1, ET_TET = 2, ET_PYR = 3, ET_COUNT = 4 };

typedef struct {
    int kind;           /* 0 = quad, 1 = triangle */
    int npts;
    double nref[3];     /* unit outward reference normal */
    double dS;          /* reference surface measure per unit (s,t) parameter area */
} face_info;

typedef struct {
    int type, p, n1, m1;    /* type, order, 1D solution points, 1D quadrature points */
    int nu, nf, nq, nmodes, nfaces;
    face_info faces[6];
    int *fpt_face;          /* [nf] face of each flux point */
    double *xu, *xf, *xq, *wq; /* ref coordinates [n][3], quadrature weights [nq] */
    double *fparam;         /* [nf][2] face parameters (s,t) of flux points */
    double *nref;           /* [nf][3] */
    double *M0;             /* [nf][nu]  disu: l_zeta(x^f_sigma) */
    double *Dm;             /* [3][nu][nu] d/dx~_d l_nu at x^u_zeta (M4 = M1) */
    double *M3;             /* [nu][nf]  DG-equivalent lift (div g), reading R3 */
    double *M7;             /* [nq][nu]  l_zeta(x^q_sigma) */
    double *M8;             /* [nu][nq]  sum_nu psi(x^u) w^q psi(x^q) */
    double *Agrad;          /* [3][nu][nu] M4 - M6 M0 (per direction) */
    double *Adiv;           /* [nu][3][nu] M1 - M3 M2 */
    double *Wu;             /* [nu] int l_zeta over the reference element */
    tri_basis tb;           /* prism and tetrahedron (their triangle faces) */
    tet_basis teb;          /* tetrahedron only */
    pyr_basis pyb;          /* pyramid only */
    double g1[16], g1w[16]; /* 1D GL solution nodes */
    int nfn;                /* 1D nodes of the hex face point grids: n, or m with surface-flux AA */
    double fg[32];          /* their coordinates */
} etype_t;

/* Modal orthonormal basis and its reference gradient at a point. */
static void modal_eval(const etype_t *et, const double *X, double *psi, double *dpsi /* [3][nmodes] or NULL */)
{
    int p = et->p, n1 = p + 1;
    double Px[32], dPx[32], Py[32], dPy[32], Pz[32], dPz[32];
    legendre_all(p, X[2], Pz, dPz);
    for (int r = 0; r <= p; r++) { double s = sqrt(r + 0.5); Pz[r] *= s; dPz[r] *= s; }
    if (et->type == ET_HEX) {
        legendre_all(p, X[0], Px, dPx);
        legendre_all(p, X[1], Py, dPy);
        for (int r = 0; r <= p; r++) {
            double s = sqrt(r + 0.5);
            Px[r] *= s; dPx[r] *= s; Py[r] *= s; dPy[r] *= s;
        }
        for (int c = 0; c < n1; c++)
            for (int b = 0; b < n1; b++)
                for (int a = 0; a < n1; a++) {
                    int nu = a + n1 * b + n1 * n1 * c;
                    psi[nu] = Px[a] * Py[b] * Pz[c];
                    if (dpsi) {
                        dpsi[0 * et->nmodes + nu] = dPx[a] * Py[b] * Pz[c];
                        dpsi[1 * et->nmodes + nu] = Px[a] * dPy[b] * Pz[c];
                        dpsi[2 * et->nmodes + nu] = Px[a] * Py[b] * dPz[c];
                    }
                }
    } else if (et->type == ET_TET) {
        tet_basis_eval(&et->teb, X, psi, dpsi);
    } else if (et->type == ET_PYR) {
        pyr_basis_eval(&et->pyb, X, psi, dpsi);
    } else {
        int nt = et->tb.nt;
        double phi[64], phx[64], phy[64];
        tri_basis_eval(&et->tb, X[0], X[1], phi, phx, phy);
        for (int c = 0; c < n1; c++)
            for (int t = 0; t < nt; t++) {
                int nu = t + nt * c;
                psi[nu] = phi[t] * Pz[c];
                if (dpsi) {
                    dpsi[0 * et->nmodes + nu] = phx[t] * Pz[c];
                    dpsi[1 * et->nmodes + nu] = phy[t] * Pz[c];
                    dpsi[2 * et->nmodes + nu] = phi[t] * dPz[c];
                }
            }
    }
}

/* Maps face parameters (s,t) of face f to reference coordinates X. */
static void face_map(const etype_t *et, int f, double s, double t, double *X)
{
    if (et->type == ET_HEX) {
        int d = f / 2; double side = (f % 2) ? 1.0 : -1.0;
        int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        X[d] = side; X[t1] = s; X[t2] = t;
    } else if (et->type == ET_TET) {
        switch (f) {
        case 0: X[0] = s; X[1] = t; X[2] = -1.0; break;        /* z = -1 */
        case 1: X[0] = s; X[1] = -1.0; X[2] = t; break;        /* y = -1 */
        case 2: X[0] = -1.0; X[1] = s; X[2] = t; break;        /* x = -1 */
        default: X[0] = -1.0 - s - t; X[1] = s; X[2] = t; break; /* x + y + z = -1 */
        }
    } else if (et->type == ET_PYR) {
        /* base (s, t) = (x, y); a triangle of vertices P0, P1, P2 at barycentric
         * ((-(s+t))/2, (1+s)/2, (1+t)/2) */
        static const double tri[4][3][3] = {
            {{-1, -1, -1}, {1, -1, -1}, {0, 0, 1}},    /* y = -(1-z)/2 */
            {{1, -1, -1}, {1, 1, -1}, {0, 0, 1}},      /* x = (1-z)/2 */
            {{1, 1, -1}, {-1, 1, -1}, {0, 0, 1}},      /* y = (1-z)/2 */
            {{-1, 1, -1}, {-1, -1, -1}, {0, 0, 1}}};   /* x = -(1-z)/2 */
        if (f == 0) { X[0] = s; X[1] = t; X[2] = -1.0; }
        else {
            const double l0 = -0.5 * (s + t), l1 = 0.5 * (1.0 + s), l2 = 0.5 * (1.0 + t);
            for (int d = 0; d < 3; d++) X[d] = l0 * tri[f - 1][0][d] + l1 * tri[f - 1][1][d] + l2 * tri[f - 1][2][d];
        }
    } else {
        switch (f) {
        case 0: X[0] = s; X[1] = t; X[2] = -1.0; break;   /* triangle z = -1 */
        case 1: X[0] = s; X[1] = t; X[2] = 1.0; break;    /* triangle z = +1 */
        case 2: X[0] = s; X[1] = -1.0; X[2] = t; break;   /* quad y = -1 */
        case 3: X[0] = -s; X[1] = s; X[2] = t; break;     /* quad x + y = 0 */
        default: X[0] = -1.0; X[1] = s; X[2] = t; break;  /* quad x = -1 */
        }
    }
}

/* Face nodal basis function j of face f (quad: GL Lagrange in s,t; triangle: nodal basis on the
 * triangle solution points), evaluated at face parameters (s,t). */
static double face_nodal(const etype_t *et, int f, int j, double s, double t, const double *TVinv)
{
    if (et->faces[f].kind == 0) {
        int k = et->nfn;
        return lagrange1d(k, et->fg, j % k, s) * lagrange1d(k, et->fg, j / k, t);
    }
    int nt = et->tb.nt;
    double phi[64];
    tri_basis_eval(&et->tb, s, t, phi, NULL, NULL);
    double v = 0;
    for (int k = 0; k < nt; k++) v += phi[k] * TVinv[k * nt + j];
    return v;
}

static int etype_init(etype_t *et, int type, int p, int m, int tri_k, int surf)
{
    memset(et, 0, sizeof(*et));
    et->type = type; et->p = p; et->n1 = p + 1; et->m1 = m;
    int n1 = p + 1;
    or_gauss_legendre(n1, et->g1, et->g1w);
    double gq[32], gqw[32];
    or_gauss_legendre(m, gq, gqw);
    if (surf && type != ET_HEX) return -1;   /* surface-flux AA: hexahedra only */
    et->nfn = surf ? m : n1;
    for (int i = 0; i < et->nfn; i++) et->fg[i] = surf ? gq[i] : et->g1[i];
    double txy[2 * 64];
    int nt = 0;
    if (type == ET_HEX) {
        et->nu = n1 * n1 * n1; et->nmodes = et->nu; et->nfaces = 6;
        et->nq = m * m * m;
        for (int f = 0; f < 6; f++) {
            et->faces[f].kind = 0; et->faces[f].npts = et->nfn * et->nfn; et->faces[f].dS = 1.0;
            memset(et->faces[f].nref, 0, sizeof(double) * 3);
            et->faces[f].nref[f / 2] = (f % 2) ? 1.0 : -1.0;
        }
    } else if (type == ET_PYR) {
        /* reading P1: p = 2, 3 (the triangular faces carry the printed triangle points) */
        nt = or_tri_solution_points(p, txy);
        if (nt < 0) return -1;
        tri_basis_init(&et->tb, p);
        if (pyr_basis_init(&et->pyb, p)) return -1;
        et->nu = (p + 1) * (p + 2) * (2 * p + 3) / 6; et->nmodes = et->nu; et->nfaces = 5;
        et->nq = m * m * m;
        double r5 = 1.0 / sqrt(5.0), dst = 0.5 * sqrt(5.0);
        face_info fi[5] = {
            {0, et->nfn * et->nfn, {0, 0, -1}, 1.0}, {1, nt, {0, -2 * r5, r5}, dst}, {1, nt, {2 * r5, 0, r5}, dst},
            {1, nt, {0, 2 * r5, r5}, dst}, {1, nt, {-2 * r5, 0, r5}, dst}};
        for (int f = 0; f < 5; f++) et->faces[f] = fi[f];
    } else if (type == ET_TET) {
        /* reading T1: p = 2, 3 (the faces carry the printed triangle points) */
        nt = or_tri_solution_points(p, txy);
        if (nt < 0) return -1;
        tri_basis_init(&et->tb, p);
        if (tet_basis_init(&et->teb, p)) return -1;
        et->nu = (p + 1) * (p + 2) * (p + 3) / 6; et->nmodes = et->nu; et->nfaces = 4;
        et->nq = m * m * m;
        double r3 = 1.0 / sqrt(3.0);
        face_info fi[4] = {
            {1, nt, {0, 0, -1}, 1.0}, {1, nt, {0, -1, 0}, 1.0}, {1, nt, {-1, 0, 0}, 1.0},
            {1, nt, {r3, r3, r3}, sqrt(3.0)}};
        for (int f = 0; f < 4; f++) et->faces[f] = fi[f];
    } else {
        nt = or_tri_solution_points(p, txy);
        if (nt < 0) return -1;
        tri_basis_init(&et->tb, p);
        et->nu = nt * n1; et->nmodes = et->nu; et->nfaces = 5;
        if (tri_k < 1) tri_k = m;
        et->nq = tri_k * tri_k * m;
        double r2 = 1.0 / sqrt(2.0);
        face_info fi[5] = {
            {1, nt, {0, 0, -1}, 1.0}, {1, nt, {0, 0, 1}, 1.0},
            {0, n1 * n1, {0, -1, 0}, 1.0}, {0, n1 * n1, {r2, r2, 0}, sqrt(2.0)},
            {0, n1 * n1, {-1, 0, 0}, 1.0}};
        for (int f = 0; f < 5; f++) et->faces[f] = fi[f];
    }
    int nf = 0;
    for (int f = 0; f < et->nfaces; f++) nf += et->faces[f].npts;
    et->nf = nf;
    int nu = et->nu, nq = et->nq;

    et->xu = (double *)malloc(nu * 3 * sizeof(double));
    et->xf = (double *)malloc(nf * 3 * sizeof(double));
    et->fparam = (double *)malloc(nf * 2 * sizeof(double));
    et->nref = (double *)malloc(nf * 3 * sizeof(double));
    et->fpt_face = (int *)malloc(nf * sizeof(int));
    et->xq = (double *)malloc(nq * 3 * sizeof(double));
    et->wq = (double *)malloc(nq * sizeof(double));

    /* solution points (R1, R7) */
    if (type == ET_HEX) {
        for (int k = 0; k < n1; k++)
            for (int j = 0; j < n1; j++)
                for (int i = 0; i < n1; i++) {
                    int z = i + n1 * j + n1 * n1 * k;
                    et->xu[3 * z] = et->g1[i]; et->xu[3 * z + 1] = et->g1[j]; et->xu[3 * z + 2] = et->g1[k];
                }
    } else if (type == ET_TET) {
        or_tet_solution_points(p, et->xu);
    } else if (type == ET_PYR) {
        or_pyr_solution_points(p, et->xu);
    } else {
        for (int k = 0; k < n1; k++)
            for (int t = 0; t < nt; t++) {
                int z = t + nt * k;
                et->xu[3 * z] = txy[2 * t]; et->xu[3 * z + 1] = txy[2 * t + 1]; et->xu[3 * z + 2] = et->g1[k];
            }
    }
    /* flux points (R2, R7) */
    {
        int s = 0;
        for (int f = 0; f < et->nfaces; f++) {
            for (int j = 0; j < et->faces[f].npts; j++, s++) {
                double ps, pt;
                if (et->faces[f].kind == 0) { ps = et->fg[j % et->nfn]; pt = et->fg[j / et->nfn]; }
                else { ps = txy[2 * j]; pt = txy[2 * j + 1]; }
                et->fparam[2 * s] = ps; et->fparam[2 * s + 1] = pt;
                face_map(et, f, ps, pt, et->xf + 3 * s);
                for (int d = 0; d < 3; d++) et->nref[3 * s + d] = et->faces[f].nref[d];
                et->fpt_face[s] = f;
            }
        }
    }
    /* volume quadrature (hex: GL^3; prism: R8) */
    if (type == ET_HEX) {
        for (int c = 0; c < m; c++)
            for (int b = 0; b < m; b++)
                for (int a = 0; a < m; a++) {
                    int q = a + m * b + m * m * c;
                    et->xq[3 * q] = gq[a]; et->xq[3 * q + 1] = gq[b]; et->xq[3 * q + 2] = gq[c];
                    et->wq[q] = gqw[a] * gqw[b] * gqw[c];
                }
    } else if (type == ET_TET) {
        /* reading T2: collapsed Gauss rules, m points per direction */
        if (or_tet_rule(m, et->xq, et->wq)) return -1;
    } else if (type == ET_PYR) {
        /* reading P2: collapsed Gauss rules, m points per direction */
        if (or_pyr_rule(m, et->xq, et->wq)) return -1;
    } else {
        int nt2 = tri_k * tri_k;
        double *txq = (double *)malloc(2 * nt2 * sizeof(double)), *twq = (double *)malloc(nt2 * sizeof(double));
        or_tri_rule(tri_k, txq, twq);
        for (int c = 0; c < m; c++)
            for (int t = 0; t < nt2; t++) {
                int q = t + nt2 * c;
                et->xq[3 * q] = txq[2 * t]; et->xq[3 * q + 1] = txq[2 * t + 1]; et->xq[3 * q + 2] = gq[c];
                et->wq[q] = twq[t] * gqw[c];
            }
        free(txq); free(twq);
    }

    /* Nodal basis: V[zeta][nu] = psi_nu(x_zeta); l_zeta(x) = sum_nu psi_nu(x) Vinv[nu][zeta]. */
    int nm = et->nmodes;
    double *V = (double *)malloc((size_t)nu * nm * sizeof(double));
    double *psi = (double *)malloc(nm * sizeof(double)), *dpsi = (double *)malloc(3 * nm * sizeof(double));
    for (int z = 0; z < nu; z++) {
        modal_eval(et, et->xu + 3 * z, psi, NULL);
        for (int v = 0; v < nm; v++) V[z * nm + v] = psi[v];
    }
    double *Vinv = (double *)malloc((size_t)nu * nm * sizeof(double));
    memcpy(Vinv, V, (size_t)nu * nm * sizeof(double));
    if (mat_inverse(nu, Vinv)) return -2;

    et->M0 = (double *)calloc((size_t)nf * nu, sizeof(double));
    et->Dm = (double *)calloc((size_t)3 * nu * nu, sizeof(double));
    et->M7 = (double *)calloc((size_t)nq * nu, sizeof(double));
    et->M8 = (double *)calloc((size_t)nu * nq, sizeof(double));
    et->M3 = (double *)calloc((size_t)nu * nf, sizeof(double));
    et->Wu = (double *)calloc(nu, sizeof(double));

    /* M0 (disu) */
    for (int s = 0; s < nf; s++) {
        modal_eval(et, et->xf + 3 * s, psi, NULL);
        for (int z = 0; z < nu; z++) {
            double v = 0;
            for (int k = 0; k < nm; k++) v += psi[k] * Vinv[k * nu + z];
            et->M0[s * nu + z] = v;
        }
    }
    /* M4 = M1: derivative of the nodal basis at solution points */
    for (int zp = 0; zp < nu; zp++) {
        modal_eval(et, et->xu + 3 * zp, psi, dpsi);
        for (int d = 0; d < 3; d++)
            for (int z = 0; z < nu; z++) {
                double v = 0;
                for (int k = 0; k < nm; k++) v += dpsi[d * nm + k] * Vinv[k * nu + z];
                et->Dm[(d * nu + zp) * nu + z] = v;
            }
    }
    /* Pyramid (reading P3): the rational space is not closed under differentiation, so the
     * derivative operator is the L2 projection of the exact derivative onto the space,
     * D_d = M^-1 S_d with S_d[zeta][nu] = int l_zeta d_d l_nu (the collapsed rule is exact for these
     * products). On the polynomial spaces of the other types this equals the nodal derivative. */
    if (type == ET_PYR) {
        double *S = (double *)calloc((size_t)3 * nu * nu, sizeof(double));
        double *lq = (double *)malloc(nu * sizeof(double)), *dlq = (double *)malloc(3 * nu * sizeof(double));
        for (int q = 0; q < nq; q++) {
            modal_eval(et, et->xq + 3 * q, psi, dpsi);
            for (int z = 0; z < nu; z++) {
                double v = 0, g[3] = {0, 0, 0};
                for (int k = 0; k < nm; k++) {
                    v += psi[k] * Vinv[k * nu + z];
                    for (int d = 0; d < 3; d++) g[d] += dpsi[d * nm + k] * Vinv[k * nu + z];
                }
                lq[z] = v;
                for (int d = 0; d < 3; d++) dlq[d * nu + z] = g[d];
            }
            for (int d = 0; d < 3; d++)
                for (int z = 0; z < nu; z++)
                    for (int j = 0; j < nu; j++) S[(d * nu + z) * nu + j] += et->wq[q] * lq[z] * dlq[d * nu + j];
        }
        for (int d = 0; d < 3; d++)
            for (int z = 0; z < nu; z++)
                for (int j = 0; j < nu; j++) {
                    double v = 0;
                    for (int zp = 0; zp < nu; zp++) {
                        double minv = 0;
                        for (int k = 0; k < nm; k++) minv += V[z * nm + k] * V[zp * nm + k];
                        v += minv * S[(d * nu + zp) * nu + j];
                    }
                    et->Dm[(d * nu + z) * nu + j] = v;
                }
        free(S); free(lq); free(dlq);
    }
    /* M7 (uqpts) and M8 (L2 projection, reading G4 for its shape) */
    double *PQ = (double *)malloc((size_t)nq * nm * sizeof(double));
    for (int q = 0; q < nq; q++) {
        modal_eval(et, et->xq + 3 * q, psi, NULL);
        for (int k = 0; k < nm; k++) PQ[q * nm + k] = psi[k];
        for (int z = 0; z < nu; z++) {
            double v = 0;
            for (int k = 0; k < nm; k++) v += psi[k] * Vinv[k * nu + z];
            et->M7[q * nu + z] = v;
        }
    }
    for (int z = 0; z < nu; z++)
        for (int q = 0; q < nq; q++) {
            double v = 0;
            for (int k = 0; k < nm; k++) v += V[z * nm + k] * et->wq[q] * PQ[q * nm + k];
            et->M8[z * nq + q] = v;
        }
    /* quadrature weights of the nodal basis: W_zeta = sum_q w_q l_zeta(x_q) */
    for (int z = 0; z < nu; z++) {
        double v = 0;
        for (int q = 0; q < nq; q++) v += et->wq[q] * et->M7[q * nu + z];
        et->Wu[z] = v;
    }

    /* Lift (reading R3): Minv = V V^T in the orthonormal basis; E by face quadrature. */
    {
        double *TVinv = NULL;
        if (type != ET_HEX) {
            TVinv = (double *)malloc(nt * nt * sizeof(double));
            double phi[64];
            for (int a = 0; a < nt; a++) {
                tri_basis_eval(&et->tb, txy[2 * a], txy[2 * a + 1], phi, NULL, NULL);
                for (int k = 0; k < nt; k++) TVinv[a * nt + k] = phi[k];
            }
            if (mat_inverse(nt, TVinv)) return -3;
        }
        double *E = (double *)calloc((size_t)nu * nf, sizeof(double));
        int kq = p + 2;
        double gf[32], gfw[32];
        or_gauss_legendre(kq, gf, gfw);
        double *tq = (double *)malloc(2 * kq * kq * sizeof(double)), *tw = (double *)malloc(kq * kq * sizeof(double));
        or_tri_rule(kq, tq, tw);
        int s0 = 0;
        for (int f = 0; f < et->nfaces; f++) {
            int npf = et->faces[f].npts;
            int nfq = (et->faces[f].kind == 0) ? kq * kq : kq * kq;
            for (int iq = 0; iq < nfq; iq++) {
                double s, t, wgt;
                if (et->faces[f].kind == 0) { s = gf[iq % kq]; t = gf[iq / kq]; wgt = gfw[iq % kq] * gfw[iq / kq]; }
                else { s = tq[2 * iq]; t = tq[2 * iq + 1]; wgt = tw[iq]; }
                wgt *= et->faces[f].dS;
                double X[3];
                face_map(et, f, s, t, X);
                modal_eval(et, X, psi, NULL);
                for (int j = 0; j < npf; j++) {
                    double lf = face_nodal(et, f, j, s, t, TVinv);
                    for (int z = 0; z < nu; z++) {
                        double lz = 0;
                        for (int k = 0; k < nm; k++) lz += psi[k] * Vinv[k * nu + z];
                        E[z * nf + s0 + j] += wgt * lz * lf;
                    }
                }
            }
            s0 += npf;
        }
        for (int z = 0; z < nu; z++)
            for (int s = 0; s < nf; s++) {
                double v = 0;
                for (int zp = 0; zp < nu; zp++) {
                    double minv = 0;
                    for (int k = 0; k < nm; k++) minv += V[z * nm + k] * V[zp * nm + k];
                    v += minv * E[zp * nf + s];
                }
                et->M3[z * nf + s] = v;
            }
        free(E); free(tq); free(tw); free(TVinv);
    }

    /* tgradpcoru operator M4 - M6 M0 with (M6)_d[zeta][sigma] = M3[zeta][sigma] n~_d(sigma) */
    et->Agrad = (double *)calloc((size_t)3 * nu * nu, sizeof(double));
    for (int d = 0; d < 3; d++)
        for (int z = 0; z < nu; z++)
            for (int zz = 0; zz < nu; zz++) {
                double v = et->Dm[(d * nu + z) * nu + zz];
                for (int s = 0; s < nf; s++) v -= et->M3[z * nf + s] * et->nref[3 * s + d] * et->M0[s * nu + zz];
                et->Agrad[(d * nu + z) * nu + zz] = v;
            }
    /* tdivtpcorf operator M1 - M3 M2 with (M2)[sigma][(d,zeta)] = l_zeta(x^f_sigma) n~_d(sigma) */
    et->Adiv = (double *)calloc((size_t)nu * 3 * nu, sizeof(double));
    for (int z = 0; z < nu; z++)
        for (int d = 0; d < 3; d++)
            for (int zz = 0; zz < nu; zz++) {
                double v = et->Dm[(d * nu + z) * nu + zz];
                for (int s = 0; s < nf; s++) v -= et->M3[z * nf + s] * et->M0[s * nu + zz] * et->nref[3 * s + d];
                et->Adiv[(z * 3 + d) * nu + zz] = v;
            }
    free(V); free(Vinv); free(psi); free(dpsi); free(PQ);
    return 0;
}

static void etype_free(etype_t *et)
{
    free(et->fpt_face); free(et->xu); free(et->xf); free(et->xq); free(et->wq); free(et->fparam);
    free(et->nref); free(et->M0); free(et->Dm); free(et->M3); free(et->M7); free(et->M8);
    free(et->Agrad); free(et->Adiv); free(et->Wu);
    if (et->type != ET_HEX) tri_basis_free(&et->tb);
    if (et->type == ET_TET) tet_basis_free(&et->teb);
    if (et->type == ET_PYR) pyr_basis_free(&et->pyb);
}

/* ---------------------------------------------------------------------------------------------
 * Mesh, metrics and interface pairs
 * ------------------------------------------------------------------------------------------- */

typedef struct {
    double gamma, Pr, mu, beta, tau;
    double p_ref;   /* constant reference pressure removed from the momentum flux (0 = none) */
} phys_params;

typedef struct {
    phys_params ph;
    etype_t et[ET_COUNT];
    int has[ET_COUNT];
    int n_hex, n_pri, n_tet, n_pyr, ne;
    double period[3];
    double *x0;     /* [ne][3] reference origin: x = x0 + J (xi + 1) */
    double *J;      /* [ne][9] row-major dx_i/dxi_j */
    double *Jinv;   /* [ne][9] dxi_i/dx_j */
    double *detJ;   /* [ne] */
    int *curved;    /* [ne] 1: a non-affine (trilinear) hexahedron, metric terms vary per point */
    double *vx;     /* [ne][8][3] hexahedron vertices (tensor order), for the trilinear map */
    long *uoff, *foff; /* per element offset into [elem][var][pt] solution and flux-point arrays */
    long nU, nF;       /* total solution and flux-point values (times NV) */
    long nfpt;         /* total flux points */
    long *fpt_base;    /* per element first global flux point */
    int *fpt_elem;     /* [nfpt] element of global flux point */
    long npair;
    long *pairL, *pairR; /* global flux points of each pair, L per reading R5 */
    /* work arrays */
    double *UF, *CF, *DF, *Q, *QF, *Rt;
    int nthreads;
} oracle_t;

/* Element order: hexahedra, then prisms, then tetrahedra. */
static int etype_of(const oracle_t *o, int e)
{
    return e < o->n_hex ? ET_HEX : (e < o->n_hex + o->n_pri ? ET_PRI : (e < o->n_hex + o->n_pri + o->n_tet ? ET_TET : ET_PYR));
}
static const etype_t *ET(const oracle_t *o, int e) { return &o->et[etype_of(o, e)]; }

static double pdist(const oracle_t *o, const double *a, const double *b)
{
    double s = 0;
    for (int d = 0; d < 3; d++) {
        double x = a[d] - b[d];
        if (o->period[d] > 0) x -= o->period[d] * floor(x / o->period[d] + 0.5);
        s += x * x;
    }
    return sqrt(s);
}

/* Trilinear map of hexahedron e (corners c = a + 2b + 4c, reference corner (+-1, +-1, +-1)):
 * x(X) = sum_c N_c(X) v_c with N_c = prod_d (1 + s_cd X_d)/2; its Jacobian dx_i/dX_j. */
static void trilinear(const oracle_t *o, int e, const double *X, double *x, double *J)
{
    const double *v = o->vx + 24 * (size_t)e;
    if (x) x[0] = x[1] = x[2] = 0.0;
    if (J) for (int k = 0; k < 9; k++) J[k] = 0.0;
    for (int c = 0; c < 8; c++) {
        double sg[3] = {(c & 1) ? 1.0 : -1.0, (c & 2) ? 1.0 : -1.0, (c & 4) ? 1.0 : -1.0};
        double f[3];
        for (int d = 0; d < 3; d++) f[d] = 0.5 * (1.0 + sg[d] * X[d]);
        double N = f[0] * f[1] * f[2];
        double dN[3] = {0.5 * sg[0] * f[1] * f[2], 0.5 * sg[1] * f[0] * f[2], 0.5 * sg[2] * f[0] * f[1]};
        for (int i = 0; i < 3; i++) {
            if (x) x[i] += N * v[3 * c + i];
            if (J) for (int j = 0; j < 3; j++) J[3 * i + j] += dN[j] * v[3 * c + i];
        }
    }
}

static void inv3(const double *a, double *b, double *det);

/* Inverse Jacobian (row-major dX_i/dx_j) and det J of element e at reference point X: the element
 * constants for affine elements, the trilinear map's values at X for curved hexahedra. */
static void point_geom(const oracle_t *o, int e, const double *X, double *Jinv, double *det)
{
    if (o->curved[e]) {
        double J[9];
        trilinear(o, e, X, NULL, J);
        inv3(J, Jinv, det);
        return;
    }
    memcpy(Jinv, o->Jinv + 9 * e, 9 * sizeof(double));
    *det = o->detJ[e];
}

static void phys_coord(const oracle_t *o, int e, const double *X, double *x)
{
    if (o->curved[e]) { trilinear(o, e, X, x, NULL); return; }
    for (int i = 0; i < 3; i++) {
        x[i] = o->x0[3 * e + i];
        for (int j = 0; j < 3; j++) x[i] += o->J[9 * e + 3 * i + j] * (X[j] + 1.0);
    }
}

static void inv3(const double *a, double *b, double *det)
{
    double d = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
    b[0] = (a[4] * a[8] - a[5] * a[7]) / d; b[1] = (a[2] * a[7] - a[1] * a[8]) / d; b[2] = (a[1] * a[5] - a[2] * a[4]) / d;
    b[3] = (a[5] * a[6] - a[3] * a[8]) / d; b[4] = (a[0] * a[8] - a[2] * a[6]) / d; b[5] = (a[2] * a[3] - a[0] * a[5]) / d;
    b[6] = (a[3] * a[7] - a[4] * a[6]) / d; b[7] = (a[1] * a[6] - a[0] * a[7]) / d; b[8] = (a[0] * a[4] - a[1] * a[3]) / d;
    *det = d;
}

/* Error codes (match the GPU library's status numbers for convenience in tests). */
#define OR_OK 0
#define OR_EINVAL 1
#define OR_EMESH 4
#define OR_EUNSUPPORTED 7

void or_destroy(void *h);

typedef struct { long long k[3]; int face; } or_facekey;

static int facekey_cmp_keys(const or_facekey *a, const or_facekey *b)
{
    for (int d = 0; d < 3; d++) {
        if (a->k[d] < b->k[d]) return -1;
        if (a->k[d] > b->k[d]) return 1;
    }
    return 0;
}

static int facekey_cmp(const void *a, const void *b)
{
    int c = facekey_cmp_keys((const or_facekey *)a, (const or_facekey *)b);
    if (c) return c;
    return ((const or_facekey *)a)->face - ((const or_facekey *)b)->face;
}

void *or_create4(int p, int m, int tri_k, int surf, double gamma, double Pr, double mu, double beta, double tau,
                 double p_ref, int n_hex, int n_pri, int n_tet, int n_pyr, int n_verts, const double *verts,
                 const int *hex_v, const int *pri_v, const int *tet_v, const int *pyr_v, const double *period, int *err);

void *or_create(int p, int m, int tri_k, double gamma, double Pr, double mu, double beta, double tau, double p_ref,
                int n_hex, int n_pri, int n_verts, const double *verts, const int *hex_v, const int *pri_v,
                const double *period, int *err)
{
    return or_create4(p, m, tri_k, 0, gamma, Pr, mu, beta, tau, p_ref, n_hex, n_pri, 0, 0, n_verts, verts, hex_v, pri_v,
                      NULL, NULL, period, err);
}

/* As or_create; surf = 1 selects surface-flux anti-aliasing (hexahedra only): the flux points of
 * every face are its m x m GL quadrature points. */
void *or_create2(int p, int m, int tri_k, int surf, double gamma, double Pr, double mu, double beta, double tau,
                 double p_ref, int n_hex, int n_pri, int n_verts, const double *verts, const int *hex_v,
                 const int *pri_v, const double *period, int *err)
{
    return or_create4(p, m, tri_k, surf, gamma, Pr, mu, beta, tau, p_ref, n_hex, n_pri, 0, 0, n_verts, verts, hex_v,
                      pri_v, NULL, NULL, period, err);
}

/* As or_create2, with n_tet tetrahedra (4 vertices each, tet_v) after the prisms. */
void *or_create3(int p, int m, int tri_k, int surf, double gamma, double Pr, double mu, double beta, double tau,
                 double p_ref, int n_hex, int n_pri, int n_tet, int n_verts, const double *verts, const int *hex_v,
                 const int *pri_v, const int *tet_v, const double *period, int *err)
{
    return or_create4(p, m, tri_k, surf, gamma, Pr, mu, beta, tau, p_ref, n_hex, n_pri, n_tet, 0, n_verts, verts,
                      hex_v, pri_v, tet_v, NULL, period, err);
}

/* As or_create3, with n_pyr pyramids (5 vertices each, pyr_v: the base corners in tensor order --
 * reference (-1,-1,-1), (1,-1,-1), (-1,1,-1), (1,1,-1) -- then the apex, reference (0,0,1)) after the
 * tetrahedra. */
void *or_create4(int p, int m, int tri_k, int surf, double gamma, double Pr, double mu, double beta, double tau,
                 double p_ref, int n_hex, int n_pri, int n_tet, int n_pyr, int n_verts, const double *verts,
                 const int *hex_v, const int *pri_v, const int *tet_v, const int *pyr_v, const double *period, int *err)
{
    *err = OR_OK;
    if (p < 1 || m < 1 || n_hex < 0 || n_pri < 0 || n_tet < 0 || n_pyr < 0 || n_hex + n_pri + n_tet + n_pyr == 0) {
        *err = OR_EINVAL;
        return NULL;
    }
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    o->ph.gamma = gamma; o->ph.Pr = Pr; o->ph.mu = mu; o->ph.beta = beta; o->ph.tau = tau; o->ph.p_ref = p_ref;
    o->n_hex = n_hex; o->n_pri = n_pri; o->n_tet = n_tet; o->n_pyr = n_pyr; o->ne = n_hex + n_pri + n_tet + n_pyr;
    for (int d = 0; d < 3; d++) o->period[d] = period ? period[d] : 0.0;
    o->nthreads = 1;
    const int counts[ET_COUNT] = {n_hex, n_pri, n_tet, n_pyr};
    for (int t = 0; t < ET_COUNT; t++) {
        if (counts[t] == 0) continue;
        if (etype_init(&o->et[t], t, p, m, tri_k, surf)) { *err = OR_EUNSUPPORTED; or_destroy(o); return NULL; }
        o->has[t] = 1;
    }
    int ne = o->ne;
    o->x0 = (double *)malloc(3 * ne * sizeof(double));
    o->J = (double *)malloc(9 * ne * sizeof(double));
    o->Jinv = (double *)malloc(9 * ne * sizeof(double));
    o->detJ = (double *)malloc(ne * sizeof(double));
    o->curved = (int *)calloc(ne, sizeof(int));
    o->vx = (double *)calloc((size_t)24 * ne, sizeof(double));
    o->uoff = (long *)malloc(ne * sizeof(long));
    o->foff = (long *)malloc(ne * sizeof(long));
    o->fpt_base = (long *)malloc(ne * sizeof(long));
    long uo = 0, fo = 0, fb = 0;
    for (int e = 0; e < ne; e++) {
        const etype_t *et = ET(o, e);
        o->uoff[e] = uo; o->foff[e] = fo; o->fpt_base[e] = fb;
        uo += (long)NV * et->nu; fo += (long)NV * et->nf; fb += et->nf;
        /* affine map from vertices; reject non-affine or inverted elements */
        const double *v[8];
        const int typ = etype_of(o, e);
        int nv = typ == ET_HEX ? 8 : (typ == ET_PRI ? 6 : (typ == ET_TET ? 4 : 5));
        for (int k = 0; k < nv; k++) {
            int vi = typ == ET_HEX ? hex_v[8 * e + k]
                     : typ == ET_PRI ? pri_v[6 * (e - n_hex) + k]
                     : typ == ET_TET ? tet_v[4 * (e - n_hex - n_pri) + k]
                                     : pyr_v[5 * (e - n_hex - n_pri - n_tet) + k];
            if (vi < 0 || vi >= n_verts) { *err = OR_EMESH; or_destroy(o); return NULL; }
            v[k] = verts + 3 * vi;
        }
        int c1 = 1, c2 = 2, c3 = (e < n_hex) ? 4 : 3;
        double scale = 0;
        for (int i = 0; i < 3; i++) {
            o->x0[3 * e + i] = v[0][i];
            o->J[9 * e + 3 * i + 0] = 0.5 * (v[c1][i] - v[0][i]);
            o->J[9 * e + 3 * i + 1] = 0.5 * (v[c2][i] - v[0][i]);
            /* pyramid: the apex (0,0,1) = corner (-1,-1,-1) + (1,1,2) */
            o->J[9 * e + 3 * i + 2] = typ == ET_PYR ? 0.5 * (v[4][i] - v[0][i]) - 0.25 * (v[c1][i] - v[0][i]) - 0.25 * (v[c2][i] - v[0][i])
                                                    : 0.5 * (v[c3][i] - v[0][i]);
            scale += fabs(v[c1][i] - v[0][i]) + fabs(v[c2][i] - v[0][i]) + fabs(v[typ == ET_PYR ? 4 : c3][i] - v[0][i]);
        }
        if (typ == ET_HEX)
            for (int k = 0; k < 8; k++)
                for (int i = 0; i < 3; i++) o->vx[24 * (size_t)e + 3 * k + i] = v[k][i];
        /* affinity: every vertex equals the affine image of its reference corner; a hexahedron that
         * is not affine is kept as a trilinear (curved) element, other types are rejected */
        for (int k = 0; k < nv; k++) {
            double X[3];
            if (e < n_hex) { X[0] = (k & 1) ? 1 : -1; X[1] = (k & 2) ? 1 : -1; X[2] = (k & 4) ? 1 : -1; }
            else if (typ == ET_PYR) {
                static const double pp[5][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {0, 0, 1}};
                X[0] = pp[k][0]; X[1] = pp[k][1]; X[2] = pp[k][2];
            } else {
                static const double pc[6][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}};
                X[0] = pc[k][0]; X[1] = pc[k][1]; X[2] = pc[k][2];
            }
            double x[3];
            phys_coord(o, e, X, x);
            int off = 0;
            for (int i = 0; i < 3; i++) off |= fabs(x[i] - v[k][i]) > 1e-10 * scale;
            if (off && typ != ET_HEX) { *err = OR_EUNSUPPORTED; or_destroy(o); return NULL; }
            if (off) o->curved[e] = 1;
        }
        inv3(o->J + 9 * e, o->Jinv + 9 * e, &o->detJ[e]);
        if (!(o->detJ[e] > 0)) { *err = OR_EMESH; or_destroy(o); return NULL; }
        if (o->curved[e]) {
            /* the trilinear map must be invertible at every point the method uses */
            const etype_t *et = ET(o, e);
            const double *sets[3] = {et->xu, et->xq, et->xf};
            const int counts[3] = {et->nu, et->nq, et->nf};
            for (int t = 0; t < 3; t++)
                for (int z = 0; z < counts[t]; z++) {
                    double Ji[9], dj;
                    point_geom(o, e, sets[t] + 3 * z, Ji, &dj);
                    if (!(dj > 0)) { *err = OR_EMESH; or_destroy(o); return NULL; }
                }
        }
    }
    o->nU = uo; o->nF = fo; o->nfpt = fb;
    o->fpt_elem = (int *)malloc(fb * sizeof(int));
    for (int e = 0; e < ne; e++)
        for (int s = 0; s < ET(o, e)->nf; s++) o->fpt_elem[o->fpt_base[e] + s] = e;

    /* Interface pairing by physical coordinates (bucketed faces, then brute force over points). */
    int nfaces_tot = 0;
    for (int e = 0; e < ne; e++) nfaces_tot += ET(o, e)->nfaces;
    int *fe = (int *)malloc(nfaces_tot * sizeof(int)), *ff = (int *)malloc(nfaces_tot * sizeof(int));
    int *fs0 = (int *)malloc(nfaces_tot * sizeof(int));
    double *fc = (double *)malloc(3 * nfaces_tot * sizeof(double));
    double *fsize = (double *)malloc(nfaces_tot * sizeof(double));
    int *mate = (int *)malloc(nfaces_tot * sizeof(int));
    {
        int k = 0;
        for (int e = 0; e < ne; e++) {
            const etype_t *et = ET(o, e);
            int s0 = 0;
            for (int f = 0; f < et->nfaces; f++) {
                fe[k] = e; ff[k] = f; fs0[k] = s0; mate[k] = -1;
                /* the physical face centroid is the affine image of the reference face centre */
                double Xc[3], c[3];
                if (et->type == ET_HEX) { Xc[0] = Xc[1] = Xc[2] = 0.0; Xc[f / 2] = (f % 2) ? 1.0 : -1.0; }
                else if (et->type == ET_TET) {
                    /* centroid of the face's three reference vertices */
                    double t3 = -1.0 / 3.0;
                    Xc[0] = Xc[1] = Xc[2] = t3;
                    if (f < 3) Xc[2 - f] = -1.0;
                }
                else if (et->type == ET_PYR) {
                    /* base: its centre; a triangle: the image of the reference triangle's centroid */
                    if (f == 0) face_map(et, 0, 0.0, 0.0, Xc);
                    else face_map(et, f, -1.0 / 3.0, -1.0 / 3.0, Xc);
                }
                else if (f < 2) { Xc[0] = Xc[1] = -1.0 / 3.0; Xc[2] = f ? 1.0 : -1.0; }
                else if (f == 2) { Xc[0] = 0.0; Xc[1] = -1.0; Xc[2] = 0.0; }
                else if (f == 3) { Xc[0] = 0.0; Xc[1] = 0.0; Xc[2] = 0.0; }
                else { Xc[0] = -1.0; Xc[1] = 0.0; Xc[2] = 0.0; }
                phys_coord(o, e, Xc, c);
                for (int d = 0; d < 3; d++) fc[3 * k + d] = c[d];
                fsize[k] = pow(fabs(o->detJ[e]), 1.0 / 3.0);
                s0 += et->faces[f].npts;
                k++;
            }
        }
    }
    /* Face matching: faces are bucketed by the cell (size a quarter of the smallest element) of
     * their centroid, wrapped into the periodic box; the bucket list is sorted and every face looks
     * for an unmatched partner in its own and the 26 neighbouring cells (binary search). */
    {
        double hmin = 1e300;
        for (int a = 0; a < nfaces_tot; a++) if (fsize[a] < hmin) hmin = fsize[a];
        double cell = 0.25 * hmin;
        long long ncell[3];
        for (int d = 0; d < 3; d++) ncell[d] = o->period[d] > 0 ? (long long)ceil(o->period[d] / cell) : 0;
        or_facekey *keys = (or_facekey *)malloc(nfaces_tot * sizeof(or_facekey));
        for (int a = 0; a < nfaces_tot; a++) {
            for (int d = 0; d < 3; d++) {
                double x = fc[3 * a + d];
                if (o->period[d] > 0) x -= o->period[d] * floor(x / o->period[d]);
                long long q = (long long)floor(x / cell);
                if (ncell[d] > 0) q = ((q % ncell[d]) + ncell[d]) % ncell[d];
                keys[a].k[d] = q;
            }
            keys[a].face = a;
        }
        qsort(keys, nfaces_tot, sizeof(or_facekey), facekey_cmp);
        for (int a = 0; a < nfaces_tot && !*err; a++) {
            int fa = keys[a].face;
            if (mate[fa] >= 0) continue;
            for (int nb = 0; nb < 27 && mate[fa] < 0; nb++) {
                or_facekey probe;
                for (int d = 0; d < 3; d++) {
                    long long q = keys[a].k[d] + (nb / (d == 0 ? 1 : d == 1 ? 3 : 9)) % 3 - 1;
                    if (ncell[d] > 0) q = ((q % ncell[d]) + ncell[d]) % ncell[d];
                    probe.k[d] = q;
                }
                /* first entry with key >= probe */
                int lo = 0, hi = nfaces_tot;
                while (lo < hi) {
                    int mid = (lo + hi) / 2;
                    if (facekey_cmp_keys(&keys[mid], &probe) < 0) lo = mid + 1; else hi = mid;
                }
                for (int b = lo; b < nfaces_tot && facekey_cmp_keys(&keys[b], &probe) == 0; b++) {
                    int fb = keys[b].face;
                    if (fb == fa || mate[fb] >= 0) continue;
                    if (pdist(o, fc + 3 * fa, fc + 3 * fb) < 1e-8 * fsize[fa]) { mate[fa] = fb; mate[fb] = fa; break; }
                }
            }
            if (mate[fa] < 0) *err = OR_EMESH;
        }
        free(keys);
        if (*err) { free(fe); free(ff); free(fs0); free(fc); free(fsize); free(mate); or_destroy(o); return NULL; }
    }
    o->npair = o->nfpt / 2;
    o->pairL = (long *)malloc(o->npair * sizeof(long));
    o->pairR = (long *)malloc(o->npair * sizeof(long));
    long ip = 0;
    for (int a = 0; a < nfaces_tot; a++) {
        int b = mate[a];
        if (b < a) continue;
        int ea = fe[a], eb = fe[b];
        const etype_t *ta = ET(o, ea), *tb = ET(o, eb);
        if (ta->faces[ff[a]].npts != tb->faces[ff[b]].npts) { *err = OR_EMESH; break; }
        int np = ta->faces[ff[a]].npts;
        /* reading R5: L = smaller element index; self-pair -> smaller local face */
        int aL = (ea < eb || (ea == eb && ff[a] < ff[b]));
        for (int j = 0; j < np; j++) {
            double xa[3];
            phys_coord(o, ea, ta->xf + 3 * (fs0[a] + j), xa);
            int found = -1;
            for (int jj = 0; jj < np; jj++) {
                double xb[3];
                phys_coord(o, eb, tb->xf + 3 * (fs0[b] + jj), xb);
                if (pdist(o, xa, xb) < 1e-8 * fsize[a]) { found = jj; break; }
            }
            if (found < 0) { *err = OR_EMESH; break; }
            long ga = o->fpt_base[ea] + fs0[a] + j, gb = o->fpt_base[eb] + fs0[b] + found;
            o->pairL[ip] = aL ? ga : gb;
            o->pairR[ip] = aL ? gb : ga;
            ip++;
        }
        if (*err) break;
    }
    free(fe); free(ff); free(fs0); free(fc); free(fsize); free(mate);
    if (*err || ip != o->npair) { if (!*err) *err = OR_EMESH; or_destroy(o); return NULL; }

    o->UF = (double *)calloc(o->nF, sizeof(double));
    o->CF = (double *)calloc(o->nF, sizeof(double));
    o->DF = (double *)calloc(o->nF, sizeof(double));
    o->QF = (double *)calloc(3 * o->nF, sizeof(double));
    o->Q = (double *)calloc(3 * o->nU, sizeof(double));
    o->Rt = (double *)calloc(o->nU, sizeof(double));
    return o;
}

void or_destroy(void *h)
{
    oracle_t *o = (oracle_t *)h;
    if (!o) return;
    for (int t = 0; t < ET_COUNT; t++) if (o->has[t]) etype_free(&o->et[t]);
    free(o->x0); free(o->J); free(o->Jinv); free(o->detJ); free(o->uoff); free(o->foff);
    free(o->curved); free(o->vx);
    free(o->fpt_base); free(o->fpt_elem); free(o->pairL); free(o->pairR);
    free(o->UF); free(o->CF); free(o->DF); free(o->QF); free(o->Q); free(o->Rt);
    free(o);
}

void or_set_threads(void *h, int n) { ((oracle_t *)h)->nthreads = n > 0 ? n : 1; }

long or_num_values(void *h) { return ((oracle_t *)h)->nU; }
long or_num_fvalues(void *h) { return ((oracle_t *)h)->nF; }
long or_num_pairs(void *h) { return ((oracle_t *)h)->npair; }

/* Physical coordinates of every solution point, layout [elem][pt][3]. */
void or_sol_coords(void *h, double *xyz)
{
    oracle_t *o = (oracle_t *)h;
    long k = 0;
    for (int e = 0; e < o->ne; e++) {
        const etype_t *et = ET(o, e);
        for (int z = 0; z < et->nu; z++, k++) phys_coord(o, e, et->xu + 3 * z, xyz + 3 * k);
    }
}

/* Physical coordinates of every flux point, layout [elem][fpt][3]. */
void or_flux_coords(void *h, double *xyz)
{
    oracle_t *o = (oracle_t *)h;
    long k = 0;
    for (int e = 0; e < o->ne; e++) {
        const etype_t *et = ET(o, e);
        for (int s = 0; s < et->nf; s++, k++) phys_coord(o, e, et->xf + 3 * s, xyz + 3 * k);
    }
}

/* Pair list (global flux point ids), for tests. */
void or_pairs(void *h, long *L, long *R)
{
    oracle_t *o = (oracle_t *)h;
    memcpy(L, o->pairL, o->npair * sizeof(long));
    memcpy(R, o->pairR, o->npair * sizeof(long));
}

/* ---------------------------------------------------------------------------------------------
 * Physics: inviscid and viscous fluxes (Sec. 2.1, Eqs. for f^e and f^v)
 * ------------------------------------------------------------------------------------------- */

/* f[d][alpha], d = direction. A constant p_ref removed from the momentum flux (volume and
 * interface alike) changes nothing in exact arithmetic on affine elements: a constant flux has zero
 * divergence and its common flux equals its own normal flux, so the lifted jump vanishes. */
static void flux_inviscid(const phys_params *ph, const double *u, double f[3][NV], double *p_out)
{
    double rho = u[0], vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho, E = u[4];
    double p = (ph->gamma - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy + vz * vz));
    double pm = p - ph->p_ref;
    double v[3] = {vx, vy, vz};
    for (int d = 0; d < 3; d++) {
        f[d][0] = rho * v[d];
        f[d][1] = rho * v[d] * vx + (d == 0 ? pm : 0.0);
        f[d][2] = rho * v[d] * vy + (d == 1 ? pm : 0.0);
        f[d][3] = rho * v[d] * vz + (d == 2 ? pm : 0.0);
        f[d][4] = v[d] * (E + p);
    }
    if (p_out) *p_out = p;
}

/* Viscous flux f^v(u, q), q[alpha][d] = physical gradient. Stress tensor per Sec. 2.1 and heat
 * flux per reading G1: phi = mu gamma/((gamma-1) Pr) grad(p/rho). */
static void flux_viscous(const phys_params *ph, const double *u, const double q[NV][3], double f[3][NV])
{
    double rho = u[0], v[3] = {u[1] / rho, u[2] / rho, u[3] / rho}, E = u[4];
    double dv[3][3]; /* dv[i][d] = d v_i / d x_d */
    for (int i = 0; i < 3; i++)
        for (int d = 0; d < 3; d++) dv[i][d] = (q[1 + i][d] - v[i] * q[0][d]) / rho;
    double div = dv[0][0] + dv[1][1] + dv[2][2];
    double mu = ph->mu, g = ph->gamma;
    double T[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            T[i][j] = mu * (dv[j][i] + dv[i][j]) - (i == j ? 2.0 / 3.0 * mu * div : 0.0);
    double phi[3];
    for (int d = 0; d < 3; d++) {
        double dEr = (q[4][d] - (E / rho) * q[0][d]) / rho;            /* d(E/rho) */
        double dke = v[0] * dv[0][d] + v[1] * dv[1][d] + v[2] * dv[2][d]; /* d(|v|^2/2) */
        double dpr = (g - 1.0) * (dEr - dke);                            /* d(p/rho) */
        phi[d] = mu * g / ((g - 1.0) * ph->Pr) * dpr;
    }
    for (int d = 0; d < 3; d++) {
        f[d][0] = 0.0;
        f[d][1] = T[0][d];
        f[d][2] = T[1][d];
        f[d][3] = T[2][d];
        f[d][4] = v[0] * T[0][d] + v[1] * T[1][d] + v[2] * T[2][d] + phi[d];
    }
}

/* Physical outward normal scaling at flux point X of element e: n_s = detJ J^-T n~ (the metric at
 * the flux point itself on curved elements). */
static void normal_scaled(const oracle_t *o, int e, const double *X, const double *nref, double *ns)
{
    double Ji[9], dj;
    point_geom(o, e, X, Ji, &dj);
    for (int k = 0; k < 3; k++) {
        ns[k] = 0;
        for (int d = 0; d < 3; d++) ns[k] += Ji[3 * d + k] * nref[d];
        ns[k] *= dj;
    }
}

/* ---------------------------------------------------------------------------------------------
 * The RHS: one loop per paper kernel, in the paper's execution order
 * ------------------------------------------------------------------------------------------- */

/* Optional intermediates for stage-level parity checks (all may be NULL):
 *   uf, cf, df: [elem][var][fpt]   qu: [elem][var][dim][pt] physical gradient at solution points
 *   qf: [elem][var][dim][fpt]      fu: [elem][var][dim][pt] projected transformed flux F~(u) */
typedef struct { double *uf, *cf, *qu, *qf, *fu, *df; } or_stages;

static int rhs_impl(oracle_t *o, const double *U, double *R, or_stages *st)
{
    const phys_params *ph = &o->ph;
    int ne = o->ne;
#ifdef _OPENMP
    omp_set_num_threads(o->nthreads);
#endif

    /* 1. disu: U^(f) = M0 U^(u) */
#pragma omp parallel for schedule(static)
    for (int e = 0; e < ne; e++) {
        const etype_t *et = ET(o, e);
        const double *u = U + o->uoff[e];
        double *uf = o->UF + o->foff[e];
        for (int a = 0; a < NV; a++)
            for (int s = 0; s < et->nf; s++) {
                double v = 0;
                for (int z = 0; z < et->nu; z++) v += et->M0[s * et->nu + z] * u[a * et->nu + z];
                uf[a * et->nf + s] = v;
            }
    }

    /* 2. con_u: C = (1/2 - beta) uL + (1/2 + beta) uR, assigned to both points of a pair */
#pragma omp parallel for schedule(static)
    for (long ip = 0; ip < o->npair; ip++) {
        long gL = o->pairL[ip], gR = o->pairR[ip];
        int eL = o->fpt_elem[gL], eR = o->fpt_elem[gR];
        int sL = (int)(gL - o->fpt_base[eL]), sR = (int)(gR - o->fpt_base[eR]);
        int nfL = ET(o, eL)->nf, nfR = ET(o, eR)->nf;
        for (int a = 0; a < NV; a++) {
            double uL = o->UF[o->foff[eL] + a * nfL + sL], uR = o->UF[o->foff[eR] + a * nfR + sR];
            double c = (0.5 - ph->beta) * uL + (0.5 + ph->beta) * uR;
            o->CF[o->foff[eL] + a * nfL + sL] = c;
            o->CF[o->foff[eR] + a * nfR + sR] = c;
        }
    }

    /* 3.-5. tgradpcoru (Q~ = (M4 - M6 M0) U), tgradcoru (Q~ += M6 C), gradcoru (q = J^-T q~) */
#pragma omp parallel for schedule(static)
    for (int e = 0; e < ne; e++) {
        const etype_t *et = ET(o, e);
        int nu = et->nu, nf = et->nf;
        const double *u = U + o->uoff[e];
        const double *cf = o->CF + o->foff[e];
        double *q = o->Q + 3 * o->uoff[e];
        double *qt = (double *)malloc(3 * nu * sizeof(double));
        for (int a = 0; a < NV; a++) {
            for (int d = 0; d < 3; d++)
                for (int z = 0; z < nu; z++) {
                    double v = 0;
                    for (int zz = 0; zz < nu; zz++) v += et->Agrad[(d * nu + z) * nu + zz] * u[a * nu + zz];
                    qt[d * nu + z] = v;
                }
            for (int d = 0; d < 3; d++)
                for (int z = 0; z < nu; z++) {
                    double v = 0;
                    for (int s = 0; s < nf; s++) v += et->M3[z * nf + s] * et->nref[3 * s + d] * cf[a * nf + s];
                    qt[d * nu + z] += v;
                }
            for (int z = 0; z < nu; z++) {
                double Ji[9], dj;
                point_geom(o, e, et->xu + 3 * z, Ji, &dj);
                for (int k = 0; k < 3; k++) {
                    double v = 0;
                    for (int d = 0; d < 3; d++) v += Ji[3 * d + k] * qt[d * nu + z];
                    q[(a * 3 + k) * nu + z] = v;
                }
            }
        }
        free(qt);
    }

    /* 6. gradcoru_fpts: Q^(f) = (I3 (x) M0) Q^(u) */
#pragma omp parallel for schedule(static)
    for (int e = 0; e < ne; e++) {
        const etype_t *et = ET(o, e);
        int nu = et->nu, nf = et->nf;
        const double *q = o->Q + 3 * o->uoff[e];
        double *qf = o->QF + 3 * o->foff[e];
        for (int ad = 0; ad < 3 * NV; ad++)
            for (int s = 0; s < nf; s++) {
                double v = 0;
                for (int z = 0; z < nu; z++) v += et->M0[s * nu + z] * q[ad * nu + z];
                qf[ad * nf + s] = v;
            }
    }

    /* 7.-10. gradcoru_qpts, uqpts, tdisf, tdivtpcorf (per element, with local work arrays) */
#pragma omp parallel for schedule(static)
    for (int e = 0; e < ne; e++) {
        const etype_t *et = ET(o, e);
        int nu = et->nu, nq = et->nq, nf = et->nf;
        const double *u = U + o->uoff[e];
        const double *q = o->Q + 3 * o->uoff[e];
        double *qq = (double *)malloc((size_t)3 * NV * nq * sizeof(double));
        double *uq = (double *)malloc((size_t)NV * nq * sizeof(double));
        double *fq = (double *)malloc((size_t)3 * NV * nq * sizeof(double));
        double *fu = (double *)malloc((size_t)3 * NV * nu * sizeof(double));
        /* 7. gradcoru_qpts: Q^(q) = (I3 (x) M7) Q^(u) */
        for (int ad = 0; ad < 3 * NV; ad++)
            for (int s = 0; s < nq; s++) {
                double v = 0;
                for (int z = 0; z < nu; z++) v += et->M7[s * nu + z] * q[ad * nu + z];
                qq[ad * nq + s] = v;
            }
        /* 8. uqpts: U^(q) = M7 U^(u) */
        for (int a = 0; a < NV; a++)
            for (int s = 0; s < nq; s++) {
                double v = 0;
                for (int z = 0; z < nu; z++) v += et->M7[s * nu + z] * u[a * nu + z];
                uq[a * nq + s] = v;
            }
        /* 9. tdisf: F~(q) = detJ J^-1 f(U^(q), Q^(q)), with f = fe - fv */
        for (int s = 0; s < nq; s++) {
            double us[NV], qs[NV][3], fe[3][NV], fv[3][NV];
            for (int a = 0; a < NV; a++) {
                us[a] = uq[a * nq + s];
                for (int d = 0; d < 3; d++) qs[a][d] = qq[(a * 3 + d) * nq + s];
            }
            flux_inviscid(ph, us, fe, NULL);
            flux_viscous(ph, us, qs, fv);
            double Ji[9], dj;
            point_geom(o, e, et->xq + 3 * s, Ji, &dj);
            for (int a = 0; a < NV; a++)
                for (int d = 0; d < 3; d++) {
                    double v = 0;
                    for (int k = 0; k < 3; k++) v += Ji[3 * d + k] * (fe[k][a] - fv[k][a]);
                    fq[(a * 3 + d) * nq + s] = dj * v;
                }
        }
        /* 10. tdivtpcorf: R~ = (M1 - M3 M2) M9 F~(q), with M9 = I3 (x) M8 */
        for (int ad = 0; ad < 3 * NV; ad++)
            for (int z = 0; z < nu; z++) {
                double v = 0;
                for (int s = 0; s < nq; s++) v += et->M8[z * nq + s] * fq[ad * nq + s];
                fu[ad * nu + z] = v;
            }
        double *rt = o->Rt + o->uoff[e];
        for (int a = 0; a < NV; a++)
            for (int z = 0; z < nu; z++) {
                double v = 0;
                for (int d = 0; d < 3; d++)
                    for (int zz = 0; zz < nu; zz++) v += et->Adiv[(z * 3 + d) * nu + zz] * fu[(a * 3 + d) * nu + zz];
                rt[a * nu + z] = v;
            }
        if (st && st->fu) memcpy(st->fu + 3 * o->uoff[e], fu, (size_t)3 * NV * nu * sizeof(double));
        (void)nf;
        free(qq); free(uq); free(fq); free(fu);
    }

    /* 11. comm_flux: Rusanov (reading R4) + LDG viscous flux (G3), D_L = |n_sL| F, D_R = -|n_sR| F */
#pragma omp parallel for schedule(static)
    for (long ip = 0; ip < o->npair; ip++) {
        long gL = o->pairL[ip], gR = o->pairR[ip];
        int eL = o->fpt_elem[gL], eR = o->fpt_elem[gR];
        int sL = (int)(gL - o->fpt_base[eL]), sR = (int)(gR - o->fpt_base[eR]);
        const etype_t *tL = ET(o, eL), *tR = ET(o, eR);
        int nfL = tL->nf, nfR = tR->nf;
        double uL[NV], uR[NV], qL[NV][3], qR[NV][3];
        for (int a = 0; a < NV; a++) {
            uL[a] = o->UF[o->foff[eL] + a * nfL + sL];
            uR[a] = o->UF[o->foff[eR] + a * nfR + sR];
            for (int d = 0; d < 3; d++) {
                qL[a][d] = o->QF[3 * o->foff[eL] + (a * 3 + d) * nfL + sL];
                qR[a][d] = o->QF[3 * o->foff[eR] + (a * 3 + d) * nfR + sR];
            }
        }
        double nsL[3], nsR[3];
        normal_scaled(o, eL, tL->xf + 3 * sL, tL->nref + 3 * sL, nsL);
        normal_scaled(o, eR, tR->xf + 3 * sR, tR->nref + 3 * sR, nsR);
        double magL = sqrt(nsL[0] * nsL[0] + nsL[1] * nsL[1] + nsL[2] * nsL[2]);
        double magR = sqrt(nsR[0] * nsR[0] + nsR[1] * nsR[1] + nsR[2] * nsR[2]);
        double n[3] = {nsL[0] / magL, nsL[1] / magL, nsL[2] / magL};
        double feL[3][NV], feR[3][NV], fvL[3][NV], fvR[3][NV], pL, pR;
        flux_inviscid(ph, uL, feL, &pL);
        flux_inviscid(ph, uR, feR, &pR);
        flux_viscous(ph, uL, qL, fvL);
        flux_viscous(ph, uR, qR, fvR);
        double vnL = (uL[1] * n[0] + uL[2] * n[1] + uL[3] * n[2]) / uL[0];
        double vnR = (uR[1] * n[0] + uR[2] * n[1] + uR[3] * n[2]) / uR[0];
        double cL = sqrt(ph->gamma * pL / uL[0]), cR = sqrt(ph->gamma * pR / uR[0]);
        double sL_ = fabs(vnL) + cL, sR_ = fabs(vnR) + cR;
        double smax = sL_ > sR_ ? sL_ : sR_;
        for (int a = 0; a < NV; a++) {
            double fnL = 0, fnR = 0, fvnL = 0, fvnR = 0;
            for (int d = 0; d < 3; d++) {
                fnL += n[d] * feL[d][a]; fnR += n[d] * feR[d][a];
                fvnL += n[d] * fvL[d][a]; fvnR += n[d] * fvR[d][a];
            }
            double Finv = 0.5 * (fnL + fnR) + 0.5 * smax * (uL[a] - uR[a]);
            double Fvis = (0.5 + ph->beta) * fvnL + (0.5 - ph->beta) * fvnR;
            double F = Finv - Fvis + ph->tau * (uL[a] - uR[a]);
            o->DF[o->foff[eL] + a * nfL + sL] = magL * F;
            o->DF[o->foff[eR] + a * nfR + sR] = -magR * F;
        }
    }

    /* 12.-13. tdivtconf (R~ += M3 D) and negdivconf (R = -R~ / detJ) */
#pragma omp parallel for schedule(static)
    for (int e = 0; e < ne; e++) {
        const etype_t *et = ET(o, e);
        int nu = et->nu, nf = et->nf;
        const double *df = o->DF + o->foff[e];
        double *rt = o->Rt + o->uoff[e];
        double *r = R + o->uoff[e];
        for (int a = 0; a < NV; a++)
            for (int z = 0; z < nu; z++) {
                double v = 0;
                for (int s = 0; s < nf; s++) v += et->M3[z * nf + s] * df[a * nf + s];
                rt[a * nu + z] += v;
                double Ji[9], dj;
                point_geom(o, e, et->xu + 3 * z, Ji, &dj);
                r[a * nu + z] = -rt[a * nu + z] / dj;
            }
    }

    if (st) {
        if (st->uf) memcpy(st->uf, o->UF, o->nF * sizeof(double));
        if (st->cf) memcpy(st->cf, o->CF, o->nF * sizeof(double));
        if (st->df) memcpy(st->df, o->DF, o->nF * sizeof(double));
        if (st->qu) memcpy(st->qu, o->Q, 3 * o->nU * sizeof(double));
        if (st->qf) memcpy(st->qf, o->QF, 3 * o->nF * sizeof(double));
    }
    return OR_OK;
}

int or_rhs(void *h, const double *U, double *R) { return rhs_impl((oracle_t *)h, U, R, NULL); }

int or_rhs_stages(void *h, const double *U, double *R, double *uf, double *cf, double *qu, double *qf,
                  double *fu, double *df)
{
    or_stages st = {uf, cf, qu, qf, fu, df};
    return rhs_impl((oracle_t *)h, U, R, &st);
}

/* Classical four-stage RK4 on the semi-discrete system du/dt = R(u). */
int or_rk4(void *h, double *U, double dt, int nsteps)
{
    oracle_t *o = (oracle_t *)h;
    long n = o->nU;
    double *k = (double *)malloc(n * sizeof(double)), *us = (double *)malloc(n * sizeof(double));
    double *acc = (double *)malloc(n * sizeof(double));
    static const double c[4] = {0.0, 0.5, 0.5, 1.0}, b[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
    for (int step = 0; step < nsteps; step++) {
        for (long i = 0; i < n; i++) acc[i] = 0.0;
        for (int s = 0; s < 4; s++) {
            if (s == 0) memcpy(us, U, n * sizeof(double));
            else for (long i = 0; i < n; i++) us[i] = U[i] + c[s] * dt * k[i];
            rhs_impl(o, us, k, NULL);
            for (long i = 0; i < n; i++) acc[i] += b[s] * k[i];
        }
        for (long i = 0; i < n; i++) U[i] += dt * acc[i];
    }
    free(k); free(us); free(acc);
    return OR_OK;
}

/* Diagnostics of a state U and its RHS R (R may be NULL):
 * out[0] = |Omega| = sum W detJ, out[1] = E_k = (1/|Omega|) sum W detJ rho|v|^2/2,
 * out[2] = eps = -dE_k/dt = -(1/|Omega|) sum W detJ (v.R_rhov - |v|^2/2 R_rho),
 * out[3..7] = sum W detJ R_alpha, out[8..12] = sum W detJ |R_alpha|. */
void or_diagnostics(void *h, const double *U, const double *R, double *out)
{
    oracle_t *o = (oracle_t *)h;
    for (int i = 0; i < 13; i++) out[i] = 0.0;
    for (int e = 0; e < o->ne; e++) {
        const etype_t *et = ET(o, e);
        const double *u = U + o->uoff[e];
        const double *r = R ? R + o->uoff[e] : NULL;
        for (int z = 0; z < et->nu; z++) {
            double Ji[9], dj;
            point_geom(o, e, et->xu + 3 * z, Ji, &dj);
            double w = et->Wu[z] * dj;
            double rho = u[z], v[3] = {u[et->nu + z] / rho, u[2 * et->nu + z] / rho, u[3 * et->nu + z] / rho};
            double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            out[0] += w;
            out[1] += w * 0.5 * rho * v2;
            if (r) {
                double dke = v[0] * r[et->nu + z] + v[1] * r[2 * et->nu + z] + v[2] * r[3 * et->nu + z] - 0.5 * v2 * r[z];
                out[2] -= w * dke;
                for (int a = 0; a < NV; a++) { out[3 + a] += w * r[a * et->nu + z]; out[8 + a] += w * fabs(r[a * et->nu + z]); }
            }
        }
    }
    out[1] /= out[0];
    out[2] /= out[0];
}

/* ---------------------------------------------------------------------------------------------
 * Operator export for pins
 * ------------------------------------------------------------------------------------------- */

/* dims[0..3] = nu, nf, nq, nfaces for element type t; returns -1 if absent. */
int or_etype_dims(void *h, int t, int *dims)
{
    oracle_t *o = (oracle_t *)h;
    if (t < 0 || t >= ET_COUNT || !o->has[t]) return -1;
    const etype_t *et = &o->et[t];
    dims[0] = et->nu; dims[1] = et->nf; dims[2] = et->nq; dims[3] = et->nfaces;
    return 0;
}

/* which: 0 xu[nu][3], 1 xf[nf][3], 2 nref[nf][3], 3 xq[nq][3], 4 wq[nq], 5 M0[nf][nu],
 * 6 D[3][nu][nu], 7 M3 lift[nu][nf], 8 M7[nq][nu], 9 M8[nu][nq], 10 Wu[nu],
 * 11 Agrad[3][nu][nu], 12 Adiv[nu][3][nu], 13 fpt_face[nf] (as doubles) */
int or_get_operator(void *h, int t, int which, double *out)
{
    oracle_t *o = (oracle_t *)h;
    if (t < 0 || t >= ET_COUNT || !o->has[t]) return -1;
    const etype_t *et = &o->et[t];
    int nu = et->nu, nf = et->nf, nq = et->nq;
    switch (which) {
    case 0: memcpy(out, et->xu, 3 * nu * sizeof(double)); break;
    case 1: memcpy(out, et->xf, 3 * nf * sizeof(double)); break;
    case 2: memcpy(out, et->nref, 3 * nf * sizeof(double)); break;
    case 3: memcpy(out, et->xq, 3 * nq * sizeof(double)); break;
    case 4: memcpy(out, et->wq, nq * sizeof(double)); break;
    case 5: memcpy(out, et->M0, (size_t)nf * nu * sizeof(double)); break;
    case 6: memcpy(out, et->Dm, (size_t)3 * nu * nu * sizeof(double)); break;
    case 7: memcpy(out, et->M3, (size_t)nu * nf * sizeof(double)); break;
    case 8: memcpy(out, et->M7, (size_t)nq * nu * sizeof(double)); break;
    case 9: memcpy(out, et->M8, (size_t)nu * nq * sizeof(double)); break;
    case 10: memcpy(out, et->Wu, nu * sizeof(double)); break;
    case 11: memcpy(out, et->Agrad, (size_t)3 * nu * nu * sizeof(double)); break;
    case 12: memcpy(out, et->Adiv, (size_t)3 * nu * nu * sizeof(double)); break;
    case 13: for (int s = 0; s < nf; s++) out[s] = et->fpt_face[s]; break;
    default: return -1;
    }
    return 0;
}

/* Element geometry export: J[9], Jinv[9], detJ for element e. */
int or_element_geometry(void *h, int e, double *J, double *Jinv, double *detJ)
{
    oracle_t *o = (oracle_t *)h;
    if (e < 0 || e >= o->ne) return -1;
    memcpy(J, o->J + 9 * e, 9 * sizeof(double));
    memcpy(Jinv, o->Jinv + 9 * e, 9 * sizeof(double));
    *detJ = o->detJ[e];
    return 0;
}

/* Orthonormal triangle basis values at (x,y), for pins (nt = (p+1)(p+2)/2 values). */
int or_tri_basis_values(int p, int npts, const double *xy, double *out)
{
    tri_basis tb;
    tri_basis_init(&tb, p);
    for (int i = 0; i < npts; i++) tri_basis_eval(&tb, xy[2 * i], xy[2 * i + 1], out + (size_t)i * tb.nt, NULL, NULL);
    tri_basis_free(&tb);
    return 0;
}
