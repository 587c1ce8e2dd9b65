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

}  // namespace frb
