// fr_basis.cpp -- host construction of the element operators used by the GPU kernels.
//
// Hexahedra are handled through 1D factors (sum factorisation, Sec. 4): every dense operator of
// Sec. 2.2 (M0, M4/M1, M6/M3, M7, M8) is a Kronecker product of the tables built here.
#include <cmath>
#include <cstring>

#include "fr_internal.h"

namespace frb {

// Cyclic Jacobi eigenvalue iteration for a small symmetric matrix a (row-major n x n). On return the
// diagonal of a holds the eigenvalues and the columns of v the orthonormal eigenvectors.
static void jacobi_eig(int n, double *a, double *v)
{
    for (int i = 0; i < n * n; i++) v[i] = 0.0;
    for (int i = 0; i < n; i++) v[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) off += a[i * n + j] * a[i * n + j];
        if (off < 1e-34) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = a[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < n; r++) {  // A <- A J (columns p, q)
                    double arp = a[r * n + p], arq = a[r * n + q];
                    a[r * n + p] = c * arp - s * arq;
                    a[r * n + q] = s * arp + c * arq;
                }
                for (int r = 0; r < n; r++) {  // A <- J^T A (rows p, q)
                    double apr = a[p * n + r], aqr = a[q * n + r];
                    a[p * n + r] = c * apr - s * aqr;
                    a[q * n + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < n; r++) {
                    double vrp = v[r * n + p], vrq = v[r * n + q];
                    v[r * n + p] = c * vrp - s * vrq;
                    v[r * n + q] = s * vrp + c * vrq;
                }
            }
    }
}

void gauss_legendre(int n, double *x, double *w)
{
    // Jacobi matrix of the monic Legendre recurrence: zero diagonal, off-diagonal k / sqrt(4k^2-1).
    double a[16 * 16], v[16 * 16];
    for (int i = 0; i < n * n; i++) a[i] = 0.0;
    for (int k = 1; k < n; k++) {
        double b = k / std::sqrt(4.0 * k * k - 1.0);
        a[(k - 1) * n + k] = b;
        a[k * n + k - 1] = b;
    }
    jacobi_eig(n, a, v);
    // sort ascending; weight = 2 * (first eigenvector component)^2
    int idx[16];
    for (int i = 0; i < n; i++) idx[i] = i;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++)
            if (a[idx[j] * n + idx[j]] < a[idx[i] * n + idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int i = 0; i < n; i++) {
        double xi = a[idx[i] * n + idx[i]];
        // two Newton polishing steps on P_n (recurrence) keep the nodes at full precision
        for (int it = 0; it < 2; it++) {
            double p0 = 1.0, p1 = xi;
            for (int k = 1; k < n; k++) { double p2 = ((2 * k + 1) * xi * p1 - k * p0) / (k + 1); p0 = p1; p1 = p2; }
            double dp = n * (xi * p1 - p0) / (xi * xi - 1.0);
            xi -= p1 / dp;
        }
        x[i] = xi;
        double v0 = v[0 * n + idx[i]];
        w[i] = 2.0 * v0 * v0;
    }
    // symmetrise (the rule is symmetric about 0)
    for (int i = 0; i < n / 2; i++) {
        double xs = 0.5 * (x[n - 1 - i] - x[i]), ws = 0.5 * (w[i] + w[n - 1 - i]);
        x[i] = -xs; x[n - 1 - i] = xs; w[i] = ws; w[n - 1 - i] = ws;
    }
    if (n % 2) x[n / 2] = 0.0;
}

// Barycentric Lagrange basis on nodes xs: values of every l_i at t.
static void lagrange_values(int n, const double *xs, double t, double *out)
{
    double lam[FR_MAXM + 2];
    for (int i = 0; i < n; i++) {
        lam[i] = 1.0;
        for (int j = 0; j < n; j++) if (j != i) lam[i] /= (xs[i] - xs[j]);
    }
    for (int i = 0; i < n; i++)
        if (t == xs[i]) { for (int j = 0; j < n; j++) out[j] = (i == j); return; }
    double den = 0.0;
    for (int i = 0; i < n; i++) den += lam[i] / (t - xs[i]);
    for (int i = 0; i < n; i++) out[i] = lam[i] / (t - xs[i]) / den;
}

int hex1d(int p, int m, Hex1D &h)
{
    int n = p + 1;
    if (n < 2 || n > FR_MAXN || m < 1 || m > FR_MAXM) return -1;
    std::memset(&h, 0, sizeof(h));
    h.n = n; h.m = m;
    gauss_legendre(n, h.x, h.w);
    gauss_legendre(m, h.xq, h.wq);
    double v[FR_MAXN];
    for (int a = 0; a < m; a++) {
        lagrange_values(n, h.x, h.xq[a], v);
        for (int i = 0; i < n; i++) h.B[a][i] = v[i];
    }
    lagrange_values(n, h.x, -1.0, h.lL);
    lagrange_values(n, h.x, 1.0, h.lR);
    // barycentric differentiation matrix D[a][i] = l_i'(x_a)
    double lam[FR_MAXN];
    for (int i = 0; i < n; i++) {
        lam[i] = 1.0;
        for (int j = 0; j < n; j++) if (j != i) lam[i] /= (h.x[i] - h.x[j]);
    }
    for (int a = 0; a < n; a++) {
        double diag = 0.0;
        for (int i = 0; i < n; i++) {
            if (i == a) continue;
            h.D[a][i] = (lam[i] / lam[a]) / (h.x[a] - h.x[i]);
            diag -= h.D[a][i];
        }
        h.D[a][a] = diag;
    }
    // DG-equivalent lift (GL mass matrix is diag(w) exactly): l_i(+-1) / w_i
    for (int i = 0; i < n; i++) { h.liftL[i] = h.lL[i] / h.w[i]; h.liftR[i] = h.lR[i] / h.w[i]; }
    // L2 projection onto P_p sampled at the solution points. The GL solution points make the mass
    // matrix diagonal, so the projection is diag(1/w) B^T diag(wq): Pj[i][a] = wq_a l_i(xq_a) / w_i.
    for (int i = 0; i < n; i++)
        for (int a = 0; a < m; a++) h.Pj[i][a] = h.wq[a] * h.B[a][i] / h.w[i];
    // corrected derivative of the factored forms M4 - M6 M0 and M1 - M3 M2 along one line
    for (int a = 0; a < n; a++)
        for (int i = 0; i < n; i++)
            h.Dh[a][i] = h.D[a][i] - h.liftR[a] * h.lR[i] + h.liftL[a] * h.lL[i];
    return 0;
}

// In-place inverse of a small dense matrix (Gauss-Jordan, partial pivoting); 0 on success.
static int invert(int n, double *a)
{
    double aug[FR_PT][2 * FR_PT];
    if (n > FR_PT) return -1;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++) aug[i][j] = j < n ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++) if (std::fabs(aug[r][c]) > std::fabs(aug[piv][c])) piv = r;
        if (std::fabs(aug[piv][c]) < 1e-300) return -1;
        for (int j = 0; j < 2 * n; j++) { double t = aug[c][j]; aug[c][j] = aug[piv][j]; aug[piv][j] = t; }
        double d = aug[c][c];
        for (int j = 0; j < 2 * n; j++) aug[c][j] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c || aug[r][c] == 0.0) continue;
            double f = aug[r][c];
            for (int j = 0; j < 2 * n; j++) aug[r][j] -= f * aug[c][j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) a[i * n + j] = aug[i][n + j];
    return 0;
}

// Monomials x^i y^j with i + j <= 3 (10 of them), their x- and y-derivatives.
static void monomials3(double x, double y, double *m, double *mx, double *my)
{
    int k = 0;
    for (int d = 0; d <= 3; d++)
        for (int j = 0; j <= d; j++) {
            int i = d - j;
            double xi = std::pow(x, i), yj = std::pow(y, j);
            m[k] = xi * yj;
            if (mx) mx[k] = i ? i * std::pow(x, i - 1) * yj : 0.0;
            if (my) my[k] = j ? j * xi * std::pow(y, j - 1) : 0.0;
            k++;
        }
}

int prism2d(Prism2D &P)
{
    std::memset(&P, 0, sizeof(P));
    // Williams-Shunn triangle points of order 3 as printed in the paper (Sec. 4.1 prism figures)
    static const double ws[FR_PT][2] = {
        {-0.333333333333333, -0.333333333333333}, {-0.888871894660414, 0.777743789320828},
        {0.777743789320828, -0.888871894660414},  {-0.888871894660414, -0.888871894660414},
        {0.268421495491446, -0.408932576528214},  {-0.859488918963232, -0.408932576528214},
        {-0.408932576528214, -0.859488918963232}, {0.268421495491446, -0.859488918963232},
        {-0.859488918963232, 0.268421495491446},  {-0.408932576528214, 0.268421495491446}};
    std::memcpy(P.xt, ws, sizeof ws);
    if (hex1d(3, 5, P.z)) return -1;
    // collapsed 5 x 5 rule: x = (1+a)(1-b)/2 - 1, y = b, w = wa wb (1-b)/2
    double g[5], gw[5];
    gauss_legendre(5, g, gw);
    for (int ib = 0; ib < 5; ib++)
        for (int ia = 0; ia < 5; ia++) {
            int q = ia + 5 * ib;
            P.xq[q][0] = 0.5 * (1.0 + g[ia]) * (1.0 - g[ib]) - 1.0;
            P.xq[q][1] = g[ib];
            P.wq[q] = gw[ia] * gw[ib] * 0.5 * (1.0 - g[ib]);
        }
    // nodal basis from the monomial Vandermonde matrix: l_t = sum_k m_k C[k][t]
    double V[FR_PT * FR_PT];
    for (int t = 0; t < FR_PT; t++) monomials3(P.xt[t][0], P.xt[t][1], &V[t * FR_PT], nullptr, nullptr);
    if (invert(FR_PT, V)) return -2;   // V now holds C = V^-1: C[k][t]
    auto nodal = [&](double x, double y, double *l, double *lx, double *ly) {
        double m[FR_PT], mx[FR_PT], my[FR_PT];
        monomials3(x, y, m, mx, my);
        for (int t = 0; t < FR_PT; t++) {
            double a = 0, b = 0, c = 0;
            for (int k = 0; k < FR_PT; k++) { a += m[k] * V[k * FR_PT + t]; b += mx[k] * V[k * FR_PT + t]; c += my[k] * V[k * FR_PT + t]; }
            l[t] = a;
            if (lx) lx[t] = b;
            if (ly) ly[t] = c;
        }
    };
    for (int q = 0; q < FR_PQ; q++) nodal(P.xq[q][0], P.xq[q][1], P.Bt[q], nullptr, nullptr);
    for (int t = 0; t < FR_PT; t++) {
        double l[FR_PT], lx[FR_PT], ly[FR_PT];
        nodal(P.xt[t][0], P.xt[t][1], l, lx, ly);
        for (int u = 0; u < FR_PT; u++) { P.Dx[t][u] = lx[u]; P.Dy[t][u] = ly[u]; }
    }
    // mass matrix (the rule is exact to degree 8 >= 6) and its inverse
    double M[FR_PT * FR_PT];
    for (int t = 0; t < FR_PT; t++)
        for (int u = 0; u < FR_PT; u++) {
            double v = 0;
            for (int q = 0; q < FR_PQ; q++) v += P.wq[q] * P.Bt[q][t] * P.Bt[q][u];
            M[t * FR_PT + u] = v;
        }
    for (int t = 0; t < FR_PT; t++) {
        double v = 0;
        for (int q = 0; q < FR_PQ; q++) v += P.wq[q] * P.Bt[q][t];
        P.wt[t] = v;
    }
    if (invert(FR_PT, M)) return -3;
    // L2 projection onto the nodal space: Pt = M^-1 Bt^T W
    for (int t = 0; t < FR_PT; t++)
        for (int q = 0; q < FR_PQ; q++) {
            double v = 0;
            for (int u = 0; u < FR_PT; u++) v += M[t * FR_PT + u] * P.Bt[q][u];
            P.Pt[t][q] = v * P.wq[q];
        }
    // quad faces 2 (y = -1), 3 (x + y = 0), 4 (x = -1): edge parameter s runs over the GL points
    const double r2 = 1.0 / std::sqrt(2.0);
    const double nrm[3][2] = {{0.0, -1.0}, {r2, r2}, {-1.0, 0.0}};
    const double jac[3] = {1.0, std::sqrt(2.0), 1.0};   // reference arc length per unit s
    for (int f = 0; f < 3; f++) {
        P.nf[f][0] = nrm[f][0];
        P.nf[f][1] = nrm[f][1];
        for (int a = 0; a < FR_PE; a++) {
            double s = P.z.x[a], x, y;
            if (f == 0) { x = s; y = -1.0; }
            else if (f == 1) { x = -s; y = s; }
            else { x = -1.0; y = s; }
            nodal(x, y, P.Ef[f][a], nullptr, nullptr);
        }
        // E_edge[t][a] = int_edge l_t l_a ds = jac w_a l_t(edge point a) (GL exact for degree 6);
        // lift L_f = M^-1 E_edge
        for (int t = 0; t < FR_PT; t++)
            for (int a = 0; a < FR_PE; a++) {
                double v = 0;
                for (int u = 0; u < FR_PT; u++) v += M[t * FR_PT + u] * jac[f] * P.z.w[a] * P.Ef[f][a][u];
                P.Lf[f][t][a] = v;
            }
    }
    // corrected in-plane derivatives (the factored M4 - M6 M0 and M1 - M3 M2 in the triangle plane)
    for (int t = 0; t < FR_PT; t++)
        for (int u = 0; u < FR_PT; u++) {
            double cx = 0, cy = 0;
            for (int f = 0; f < 3; f++)
                for (int a = 0; a < FR_PE; a++) {
                    cx += P.nf[f][0] * P.Lf[f][t][a] * P.Ef[f][a][u];
                    cy += P.nf[f][1] * P.Lf[f][t][a] * P.Ef[f][a][u];
                }
            P.Dhx[t][u] = P.Dx[t][u] - cx;
            P.Dhy[t][u] = P.Dy[t][u] - cy;
        }
    return 0;
}

// Gauss rule of the weight (1-x)^alpha on [-1,1]: the three-term recurrence of its monic orthogonal
// polynomials from the discretised Stieltjes procedure (inner products by the 16-point GL rule,
// exact for the degrees met here), then Golub-Welsch: the nodes are the eigenvalues of the Jacobi
// matrix and the weights mu_0 times the squared first eigenvector components; two Newton steps on
// the recurrence polish the nodes. Nodes ascending.
static int gauss_weight_rule(int n, int alpha, double *x, double *w)
{
    if (n < 1 || n > 8) return -1;
    double g[16], gw[16], ww[16], pm[16], pc[16];
    gauss_legendre(16, g, gw);
    for (int q = 0; q < 16; q++) {
        ww[q] = gw[q] * std::pow(1.0 - g[q], alpha);
        pm[q] = 0.0;
        pc[q] = 1.0;
    }
    double ak[8], bk[8], nprev = 1.0;
    for (int k = 0; k < n; k++) {
        double nk = 0, xk = 0;
        for (int q = 0; q < 16; q++) { nk += ww[q] * pc[q] * pc[q]; xk += ww[q] * g[q] * pc[q] * pc[q]; }
        ak[k] = xk / nk;
        bk[k] = k ? nk / nprev : nk;   // b_0 = mu_0
        nprev = nk;
        for (int q = 0; q < 16; q++) {
            double nx = (g[q] - ak[k]) * pc[q] - (k ? bk[k] : 0.0) * pm[q];
            pm[q] = pc[q];
            pc[q] = nx;
        }
    }
    double a[64], v[64];
    for (int i = 0; i < n * n; i++) a[i] = 0.0;
    for (int k = 0; k < n; k++) a[k * n + k] = ak[k];
    for (int k = 1; k < n; k++) a[(k - 1) * n + k] = a[k * n + k - 1] = std::sqrt(bk[k]);
    jacobi_eig(n, a, v);
    int idx[8];
    for (int i = 0; i < n; i++) idx[i] = i;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++)
            if (a[idx[j] * n + idx[j]] < a[idx[i] * n + idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int i = 0; i < n; i++) {
        double xi = a[idx[i] * n + idx[i]];
        for (int it = 0; it < 2; it++) {
            double p0 = 0.0, p1 = 1.0, d0 = 0.0, d1 = 0.0;
            for (int k = 0; k < n; k++) {
                double p2 = (xi - ak[k]) * p1 - (k ? bk[k] : 0.0) * p0;
                double d2 = p1 + (xi - ak[k]) * d1 - (k ? bk[k] : 0.0) * d0;
                p0 = p1; p1 = p2; d0 = d1; d1 = d2;
            }
            xi -= p1 / d1;
        }
        x[i] = xi;
        double v0 = v[0 * n + idx[i]];
        w[i] = bk[0] * v0 * v0;
    }
    return 0;
}

// Monomials x^i y^j z^k with i + j + k <= 3 (20 of them) and their gradients.
static void monomials3d(const double *X, double *m, double (*dm)[FR_TU])
{
    int k = 0;
    for (int d = 0; d <= 3; d++)
        for (int i = d; i >= 0; i--)
            for (int j = d - i; j >= 0; j--) {
                const int l = d - i - j, e[3] = {i, j, l};
                m[k] = std::pow(X[0], i) * std::pow(X[1], j) * std::pow(X[2], l);
                if (dm)
                    for (int c = 0; c < 3; c++) {
                        double v = e[c];
                        for (int cc = 0; cc < 3; cc++) v *= std::pow(X[cc], cc == c ? (e[cc] ? e[cc] - 1 : 0) : e[cc]);
                        dm[c][k] = e[c] ? v : 0.0;
                    }
                k++;
            }
}

// In-place inverse of an n x n matrix (n <= FR_YU), Gauss-Jordan with partial pivoting.
static int invert_n(int n, double *a)
{
    double aug[FR_YU][2 * FR_YU];
    if (n > FR_YU) return -1;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++) aug[i][j] = j < n ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++) if (std::fabs(aug[r][c]) > std::fabs(aug[piv][c])) piv = r;
        if (std::fabs(aug[piv][c]) < 1e-300) return -1;
        for (int j = 0; j < 2 * n; j++) { double t = aug[c][j]; aug[c][j] = aug[piv][j]; aug[piv][j] = t; }
        double d = aug[c][c];
        for (int j = 0; j < 2 * n; j++) aug[c][j] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c || aug[r][c] == 0.0) continue;
            double f = aug[r][c];
            for (int j = 0; j < 2 * n; j++) aug[r][j] -= f * aug[c][j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) a[i * n + j] = aug[i][n + j];
    return 0;
}

int tet3d(Tet3D &T)
{
    std::memset(&T, 0, sizeof(T));
    // solution points: order-3 lattice (a, b, c)/3, a fastest, shrunk by 4/5 towards (-1/2,-1/2,-1/2)
    int k = 0;
    for (int c = 0; c <= 3; c++)
        for (int b = 0; b <= 3 - c; b++)
            for (int a = 0; a <= 3 - b - c; a++) {
                const double X[3] = {-1.0 + 2.0 * a / 3.0, -1.0 + 2.0 * b / 3.0, -1.0 + 2.0 * c / 3.0};
                for (int d = 0; d < 3; d++) T.x[k][d] = -0.5 + 0.8 * (X[d] + 0.5);
                k++;
            }
    // flux points: the printed triangle points on each face, X = face map of (s, t)
    Prism2D P;
    if (prism2d(P)) return -1;
    const double r3 = 1.0 / std::sqrt(3.0);
    const double nrm[4][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0}, {r3, r3, r3}};
    const double dS[4] = {1.0, 1.0, 1.0, std::sqrt(3.0)};
    std::memcpy(T.nf, nrm, sizeof nrm);
    for (int f = 0; f <= 4; f++) T.foff[f] = 10 * f;
    for (int f = 0; f < 4; f++)
        for (int t = 0; t < 10; t++) {
            const double s = P.xt[t][0], u = P.xt[t][1];
            double *X = T.xf[10 * f + t];
            if (f == 0) { X[0] = s; X[1] = u; X[2] = -1.0; }
            else if (f == 1) { X[0] = s; X[1] = -1.0; X[2] = u; }
            else if (f == 2) { X[0] = -1.0; X[1] = s; X[2] = u; }
            else { X[0] = -1.0 - s - u; X[1] = s; X[2] = u; }
        }
    // collapsed rule: GL in a, the Gauss rules of (1-b) and (1-c)^2 in b and c
    double ga[5], wa[5], gb[5], wb[5], gc[5], wc[5];
    gauss_legendre(5, ga, wa);
    if (gauss_weight_rule(5, 1, gb, wb) || gauss_weight_rule(5, 2, gc, wc)) return -2;
    for (int ic = 0; ic < 5; ic++)
        for (int ib = 0; ib < 5; ib++)
            for (int ia = 0; ia < 5; ia++) {
                const int q = ia + 5 * ib + 25 * ic;
                T.xq[q][0] = 0.25 * (1.0 + ga[ia]) * (1.0 - gb[ib]) * (1.0 - gc[ic]) - 1.0;
                T.xq[q][1] = 0.5 * (1.0 + gb[ib]) * (1.0 - gc[ic]) - 1.0;
                T.xq[q][2] = gc[ic];
                T.wq[q] = wa[ia] * wb[ib] * wc[ic] / 8.0;
            }
    // nodal basis from the monomial Vandermonde matrix: l_z = sum_k m_k C[k][z]
    double C[FR_TU * FR_TU];
    for (int z = 0; z < FR_TU; z++) monomials3d(T.x[z], &C[z * FR_TU], nullptr);
    if (invert_n(FR_TU, C)) return -3;
    auto nodal = [&](const double *X, double *l, double (*dl)[FR_TU]) {
        double m[FR_TU], dm[3][FR_TU];
        monomials3d(X, m, dm);
        for (int z = 0; z < FR_TU; z++) {
            double v = 0, g0 = 0, g1 = 0, g2 = 0;
            for (int kk = 0; kk < FR_TU; kk++) {
                const double c = C[kk * FR_TU + z];
                v += m[kk] * c; g0 += dm[0][kk] * c; g1 += dm[1][kk] * c; g2 += dm[2][kk] * c;
            }
            l[z] = v;
            if (dl) { dl[0][z] = g0; dl[1][z] = g1; dl[2][z] = g2; }
        }
    };
    for (int q = 0; q < FR_TQ; q++) nodal(T.xq[q], T.B[q], nullptr);
    for (int s = 0; s < FR_TF; s++) nodal(T.xf[s], T.M0[s], nullptr);
    for (int z = 0; z < FR_TU; z++) {
        double l[FR_TU], dl[3][FR_TU];
        nodal(T.x[z], l, dl);
        for (int d = 0; d < 3; d++)
            for (int j = 0; j < FR_TU; j++) T.D[d][z][j] = dl[d][j];
    }
    // mass matrix (the rule is exact to degree 9 >= 6), its inverse, the point weights, projection
    double M[FR_TU * FR_TU];
    for (int z = 0; z < FR_TU; z++) {
        double wz = 0;
        for (int q = 0; q < FR_TQ; q++) wz += T.wq[q] * T.B[q][z];
        T.w[z] = wz;
        for (int j = 0; j < FR_TU; j++) {
            double v = 0;
            for (int q = 0; q < FR_TQ; q++) v += T.wq[q] * T.B[q][z] * T.B[q][j];
            M[z * FR_TU + j] = v;
        }
    }
    if (invert_n(FR_TU, M)) return -4;
    for (int z = 0; z < FR_TU; z++)
        for (int q = 0; q < FR_TQ; q++) {
            double v = 0;
            for (int j = 0; j < FR_TU; j++) v += M[z * FR_TU + j] * T.B[q][j];
            T.Pj[z][q] = v * T.wq[q];
        }
    // lift: E[z][10 f + t] = dS_f int_face l_z l^face_t; on a face l_z is a polynomial of the face
    // space, l_z = sum_t' l_z(x_t') l^face_t', so E = dS_f M0_f^T Mf with the face mass matrix Mf of
    // the triangle's nodal basis (collapsed 5 x 5 triangle rule, exact to degree 8 >= 6)
    double Mf[10][10];
    {
        double Vt[10 * 10];
        auto mono2 = [](double x, double y, double *m) {
            int kk = 0;
            for (int d = 0; d <= 3; d++)
                for (int j = 0; j <= d; j++) m[kk++] = std::pow(x, d - j) * std::pow(y, j);
        };
        for (int t = 0; t < 10; t++) mono2(P.xt[t][0], P.xt[t][1], &Vt[t * 10]);
        if (invert_n(10, Vt)) return -5;
        for (int t = 0; t < 10; t++)
            for (int u = 0; u < 10; u++) Mf[t][u] = 0.0;
        for (int q = 0; q < FR_PQ; q++) {
            double m[10], l[10];
            mono2(P.xq[q][0], P.xq[q][1], m);
            for (int t = 0; t < 10; t++) {
                double v = 0;
                for (int kk = 0; kk < 10; kk++) v += m[kk] * Vt[kk * 10 + t];
                l[t] = v;
            }
            for (int t = 0; t < 10; t++)
                for (int u = 0; u < 10; u++) Mf[t][u] += P.wq[q] * l[t] * l[u];
        }
    }
    for (int z = 0; z < FR_TU; z++)
        for (int f = 0; f < 4; f++)
            for (int t = 0; t < 10; t++) {
                double e = 0;
                for (int tp = 0; tp < 10; tp++) e += T.M0[10 * f + tp][z] * Mf[tp][t];
                T.L[z][10 * f + t] = dS[f] * e;   // E for now
            }
    {
        double E[FR_TU][FR_TF];
        std::memcpy(E, T.L, sizeof E);
        for (int z = 0; z < FR_TU; z++)
            for (int s = 0; s < FR_TF; s++) {
                double v = 0;
                for (int j = 0; j < FR_TU; j++) v += M[z * FR_TU + j] * E[j][s];
                T.L[z][s] = v;
            }
    }
    // corrected derivative
    for (int d = 0; d < 3; d++)
        for (int z = 0; z < FR_TU; z++)
            for (int j = 0; j < FR_TU; j++) {
                double c = 0;
                for (int s = 0; s < FR_TF; s++) c += T.L[z][s] * nrm[s / 10][d] * T.M0[s][j];
                T.Dh[d][z][j] = T.D[d][z][j] - c;
            }
    return 0;
}

// Generator g_ijk = a^i b^j (1-c)^max(i,j) c^k of the pyramid space (a = 2x/(1-z), b = 2y/(1-z),
// c = z) and its (x, y, z) gradient; ordered by max(i,j), then k, then j, then i (30 at order 3).
static void pyr_generators(const double *X, double *g, double (*dg)[FR_YU])
{
    const double om = 1.0 - X[2], a = 2.0 * X[0] / om, b = 2.0 * X[1] / om, c = X[2];
    int n = 0;
    for (int mm = 0; mm <= 3; mm++)
        for (int k = 0; k <= 3 - mm; k++)
            for (int j = 0; j <= mm; j++)
                for (int i = 0; i <= mm; i++) {
                    if ((i > j ? i : j) != mm) continue;
                    const double ai = std::pow(a, i), bj = std::pow(b, j), cm = std::pow(om, mm), ck = std::pow(c, k);
                    g[n] = ai * bj * cm * ck;
                    if (dg) {
                        const double ga = i ? i * std::pow(a, i - 1) * bj * cm * ck : 0.0;
                        const double gb = j ? j * ai * std::pow(b, j - 1) * cm * ck : 0.0;
                        double gc = (mm ? -mm * ai * bj * std::pow(om, mm - 1) * ck : 0.0) + (k ? ai * bj * cm * k * std::pow(c, k - 1) : 0.0);
                        dg[0][n] = 2.0 * ga / om;
                        dg[1][n] = 2.0 * gb / om;
                        dg[2][n] = (a * ga + b * gb) / om + gc;
                    }
                    n++;
                }
}

int pyr3d(Pyr3D &P)
{
    std::memset(&P, 0, sizeof(P));
    constexpr int NU = FR_YU, NF = FR_YF;
    // solution points: the order-3 pyramid lattice (layer k at z = -1 + 2k/3 holds (4-k)^2 points at
    // x, y = (1 - k/3)(-1 + 2i/(3-k))), shrunk by 4/5 towards (0, 0, -1/2); i fastest, then j, then k
    int n = 0;
    for (int k = 0; k <= 3; k++) {
        const int m = 3 - k;
        const double z = -1.0 + 2.0 * k / 3.0, h = 1.0 - k / 3.0;
        for (int j = 0; j <= m; j++)
            for (int i = 0; i <= m; i++) {
                const double x = m ? h * (-1.0 + 2.0 * i / m) : 0.0, y = m ? h * (-1.0 + 2.0 * j / m) : 0.0;
                P.x[n][0] = 0.8 * x; P.x[n][1] = 0.8 * y; P.x[n][2] = -0.5 + 0.8 * (z + 0.5);
                n++;
            }
    }
    // faces: the base (4 x 4 GL points, a + 4 b) and four triangles (the printed triangle points)
    Prism2D Pr;
    if (prism2d(Pr)) return -1;
    const double r5 = 1.0 / std::sqrt(5.0);
    const double nrm[5][3] = {{0, 0, -1}, {0, -2 * r5, r5}, {2 * r5, 0, r5}, {0, 2 * r5, r5}, {-2 * r5, 0, r5}};
    std::memcpy(P.nf, nrm, sizeof nrm);
    P.foff[0] = 0;
    P.foff[1] = 16;
    for (int f = 2; f <= 5; f++) P.foff[f] = 16 + 10 * (f - 1);
    static const double tri[4][3][3] = {{{-1, -1, -1}, {1, -1, -1}, {0, 0, 1}},
                                        {{1, -1, -1}, {1, 1, -1}, {0, 0, 1}},
                                        {{1, 1, -1}, {-1, 1, -1}, {0, 0, 1}},
                                        {{-1, 1, -1}, {-1, -1, -1}, {0, 0, 1}}};
    for (int b = 0; b < 4; b++)
        for (int a = 0; a < 4; a++) {
            P.xf[a + 4 * b][0] = Pr.z.x[a]; P.xf[a + 4 * b][1] = Pr.z.x[b]; P.xf[a + 4 * b][2] = -1.0;
        }
    for (int f = 0; f < 4; f++)
        for (int t = 0; t < 10; t++) {
            const double s = Pr.xt[t][0], u = Pr.xt[t][1];
            const double l0 = -0.5 * (s + u), l1 = 0.5 * (1.0 + s), l2 = 0.5 * (1.0 + u);
            for (int d = 0; d < 3; d++) P.xf[16 + 10 * f + t][d] = l0 * tri[f][0][d] + l1 * tri[f][1][d] + l2 * tri[f][2][d];
        }
    // collapsed rule: GL in a and b, the Gauss rule of (1-c)^2 in c; x = a(1-c)/2, y = b(1-c)/2
    double ga[5], wa[5], gc[5], wc[5];
    gauss_legendre(5, ga, wa);
    if (gauss_weight_rule(5, 2, gc, wc)) return -2;
    for (int ic = 0; ic < 5; ic++)
        for (int ib = 0; ib < 5; ib++)
            for (int ia = 0; ia < 5; ia++) {
                const int q = ia + 5 * ib + 25 * ic;
                P.xq[q][0] = 0.5 * ga[ia] * (1.0 - gc[ic]);
                P.xq[q][1] = 0.5 * ga[ib] * (1.0 - gc[ic]);
                P.xq[q][2] = gc[ic];
                P.wq[q] = wa[ia] * wa[ib] * wc[ic] / 4.0;
            }
    // nodal basis from the generators' Vandermonde matrix: l_z = sum_k g_k C[k][z]
    double C[NU * NU];
    for (int z = 0; z < NU; z++) pyr_generators(P.x[z], &C[z * NU], nullptr);
    if (invert_n(NU, C)) return -3;
    auto nodal = [&](const double *X, double *l, double (*dl)[NU]) {
        double g[NU], dg[3][NU];
        pyr_generators(X, g, dl ? dg : nullptr);
        for (int z = 0; z < NU; z++) {
            double v = 0, g0 = 0, g1 = 0, g2 = 0;
            for (int kk = 0; kk < NU; kk++) {
                const double c = C[kk * NU + z];
                v += g[kk] * c;
                if (dl) { g0 += dg[0][kk] * c; g1 += dg[1][kk] * c; g2 += dg[2][kk] * c; }
            }
            l[z] = v;
            if (dl) { dl[0][z] = g0; dl[1][z] = g1; dl[2][z] = g2; }
        }
    };
    static double dq[3][FR_TQ][NU];   // derivatives of the nodal basis at the quadrature points
    for (int q = 0; q < FR_TQ; q++) {
        double dl[3][NU];
        nodal(P.xq[q], P.B[q], dl);
        for (int d = 0; d < 3; d++)
            for (int z = 0; z < NU; z++) dq[d][q][z] = dl[d][z];
    }
    for (int s = 0; s < NF; s++) nodal(P.xf[s], P.M0[s], nullptr);
    // mass matrix (the rule is exact for the products), its inverse, point weights, projection
    double M[NU * NU];
    for (int z = 0; z < NU; z++) {
        double wz = 0;
        for (int q = 0; q < FR_TQ; q++) wz += P.wq[q] * P.B[q][z];
        P.w[z] = wz;
        for (int j = 0; j < NU; j++) {
            double v = 0;
            for (int q = 0; q < FR_TQ; q++) v += P.wq[q] * P.B[q][z] * P.B[q][j];
            M[z * NU + j] = v;
        }
    }
    if (invert_n(NU, M)) return -4;
    for (int z = 0; z < NU; z++)
        for (int q = 0; q < FR_TQ; q++) {
            double v = 0;
            for (int j = 0; j < NU; j++) v += M[z * NU + j] * P.B[q][j];
            P.Pj[z][q] = v * P.wq[q];
        }
    // derivative: the L2 projection of the exact derivative, D_d = Pj (d_d l_j at the quadrature points)
    for (int d = 0; d < 3; d++)
        for (int z = 0; z < NU; z++)
            for (int j = 0; j < NU; j++) {
                double v = 0;
                for (int q = 0; q < FR_TQ; q++) v += P.Pj[z][q] * dq[d][q][j];
                P.D[d][z][j] = v;
            }
    // lift: E = M0_f^T W_f on the base (the 4 x 4 GL rule is exact for the Q_3 traces' products)
    // and dS_f M0_f^T Mf on the triangles (face mass matrix of the triangle's nodal basis,
    // dS = sqrt(5)/2); L = M^-1 E
    double Mf[10][10];
    {
        double Vt[10 * 10];
        auto mono2 = [](double x, double y, double *mm) {
            int kk = 0;
            for (int d = 0; d <= 3; d++)
                for (int j = 0; j <= d; j++) mm[kk++] = std::pow(x, d - j) * std::pow(y, j);
        };
        for (int t = 0; t < 10; t++) mono2(Pr.xt[t][0], Pr.xt[t][1], &Vt[t * 10]);
        if (invert_n(10, Vt)) return -5;
        for (int t = 0; t < 10; t++)
            for (int u = 0; u < 10; u++) Mf[t][u] = 0.0;
        for (int q = 0; q < FR_PQ; q++) {
            double mm[10], l[10];
            mono2(Pr.xq[q][0], Pr.xq[q][1], mm);
            for (int t = 0; t < 10; t++) {
                double v = 0;
                for (int kk = 0; kk < 10; kk++) v += mm[kk] * Vt[kk * 10 + t];
                l[t] = v;
            }
            for (int t = 0; t < 10; t++)
                for (int u = 0; u < 10; u++) Mf[t][u] += Pr.wq[q] * l[t] * l[u];
        }
    }
    static double E[NU][NF];
    const double dst = 0.5 * std::sqrt(5.0);
    for (int z = 0; z < NU; z++) {
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 4; a++) E[z][a + 4 * b] = P.M0[a + 4 * b][z] * Pr.z.w[a] * Pr.z.w[b];
        for (int f = 0; f < 4; f++)
            for (int t = 0; t < 10; t++) {
                double e = 0;
                for (int tp = 0; tp < 10; tp++) e += P.M0[16 + 10 * f + tp][z] * Mf[tp][t];
                E[z][16 + 10 * f + t] = dst * e;
            }
    }
    for (int z = 0; z < NU; z++)
        for (int s = 0; s < NF; s++) {
            double v = 0;
            for (int j = 0; j < NU; j++) v += M[z * NU + j] * E[j][s];
            P.L[z][s] = v;
        }
    // corrected derivative
    for (int d = 0; d < 3; d++)
        for (int z = 0; z < NU; z++)
            for (int j = 0; j < NU; j++) {
                double c = 0;
                for (int s = 0; s < NF; s++) {
                    const int f = s < 16 ? 0 : 1 + (s - 16) / 10;
                    c += P.L[z][s] * nrm[f][d] * P.M0[s][j];
                }
                P.Dh[d][z][j] = P.D[d][z][j] - c;
            }
    return 0;
}

}  // namespace frb
