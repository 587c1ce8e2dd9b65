// fr_physics.cuh -- pointwise physics of the compressible Navier-Stokes equations (Sec. 2.1),
// shared by the hexahedral and prismatic kernels.
#pragma once

#include "fr_internal.h"

// ---------------------------------------------------------------------------------------------
// Point physics (Sec. 2.1): total flux f = f^e - f^v, viscous normal flux, Rusanov common flux
// ---------------------------------------------------------------------------------------------

// Physical total flux f[d][alpha] from the state u and its physical gradient g[alpha][d].
// Returns false for a non-physical state (rho <= 0, p <= 0 or non-finite).
template <typename T>
__device__ __forceinline__ bool total_flux(const Phys<T> &ph, const T *u, const T (*g)[3], T (*f)[5])
{
    const T rho = u[0], ir = T(1) / rho;
    const T v[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
    const T E = u[4];
    const T p = ph.gm1 * (E - T(0.5) * (u[1] * v[0] + u[2] * v[1] + u[3] * v[2]));
    T dv[3][3];  // dv[i][d] = d v_i / d x_d
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int d = 0; d < 3; d++) dv[i][d] = (g[1 + i][d] - v[i] * g[0][d]) * ir;
    const T div = dv[0][0] + dv[1][1] + dv[2][2];
    const T er = E * ir;
    const T pm = p - ph.pref;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        T tau[3];
#pragma unroll
        for (int i = 0; i < 3; i++) tau[i] = ph.mu * (dv[i][d] + dv[d][i]) - (i == d ? T(2.0 / 3.0) * ph.mu * div : T(0));
        // heat flux mu gamma/Pr [d(E/rho) - v.dv] = mu gamma/((gamma-1)Pr) d(p/rho)
        const T phi = ph.heat * ((g[4][d] - er * g[0][d]) * ir - (v[0] * dv[0][d] + v[1] * dv[1][d] + v[2] * dv[2][d]));
        f[d][0] = u[1 + d];
        f[d][1] = u[1] * v[d] + (d == 0 ? pm : T(0)) - tau[0];
        f[d][2] = u[2] * v[d] + (d == 1 ? pm : T(0)) - tau[1];
        f[d][3] = u[3] * v[d] + (d == 2 ? pm : T(0)) - tau[2];
        f[d][4] = v[d] * (E + p) - (v[0] * tau[0] + v[1] * tau[1] + v[2] * tau[2] + phi);
    }
    return rho > T(0) && p > T(0) && isfinite(p) && isfinite(f[0][4] + f[1][4] + f[2][4]);
}

// n . f^v for variables 1..4 (the mass component is zero).
template <typename T>
__device__ __forceinline__ void viscous_normal_flux(const Phys<T> &ph, const T *u, const T (*g)[3], const T *n, T *fvn)
{
    const T rho = u[0], ir = T(1) / rho;
    const T v[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
    T dv[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int d = 0; d < 3; d++) dv[i][d] = (g[1 + i][d] - v[i] * g[0][d]) * ir;
    const T div = dv[0][0] + dv[1][1] + dv[2][2];
    const T er = u[4] * ir;
    T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        T tau[3];
#pragma unroll
        for (int i = 0; i < 3; i++) tau[i] = ph.mu * (dv[i][d] + dv[d][i]) - (i == d ? T(2.0 / 3.0) * ph.mu * div : T(0));
        const T phi = ph.heat * ((g[4][d] - er * g[0][d]) * ir - (v[0] * dv[0][d] + v[1] * dv[1][d] + v[2] * dv[2][d]));
        acc[0] += n[d] * tau[0];
        acc[1] += n[d] * tau[1];
        acc[2] += n[d] * tau[2];
        acc[3] += n[d] * (v[0] * tau[0] + v[1] * tau[1] + v[2] * tau[2] + phi);
    }
#pragma unroll
    for (int a = 0; a < 4; a++) fvn[a] = acc[a];
}

// Common physical normal flux along nL (Rusanov inviscid part, LDG viscous part and penalty):
// F = 1/2 nL.(fe_L + fe_R) + 1/2 s (uL - uR) - [(1/2+beta) nL.fv_L + (1/2-beta) nL.fv_R] + tau (uL - uR)
// fvL = nL.fv_L (vars 1..4), fvR = nR.fv_R with nR = -nL.
template <typename T>
__device__ __forceinline__ bool common_flux(const Phys<T> &ph, const T *uL, const T *uR, const T *fvL, const T *fvR,
                                            const T *n, T *F)
{
    const T irL = T(1) / uL[0], irR = T(1) / uR[0];
    const T vnL = (uL[1] * n[0] + uL[2] * n[1] + uL[3] * n[2]) * irL;
    const T vnR = (uR[1] * n[0] + uR[2] * n[1] + uR[3] * n[2]) * irR;
    const T pL = ph.gm1 * (uL[4] - T(0.5) * irL * (uL[1] * uL[1] + uL[2] * uL[2] + uL[3] * uL[3]));
    const T pR = ph.gm1 * (uR[4] - T(0.5) * irR * (uR[1] * uR[1] + uR[2] * uR[2] + uR[3] * uR[3]));
    const T cL = sqrt(ph.gamma * pL * irL), cR = sqrt(ph.gamma * pR * irR);
    const T s = fmax(fabs(vnL) + cL, fabs(vnR) + cR);
    T fnL[5], fnR[5];
    fnL[0] = uL[0] * vnL; fnR[0] = uR[0] * vnR;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        fnL[1 + i] = uL[1 + i] * vnL + (pL - ph.pref) * n[i];
        fnR[1 + i] = uR[1 + i] * vnR + (pR - ph.pref) * n[i];
    }
    fnL[4] = vnL * (uL[4] + pL); fnR[4] = vnR * (uR[4] + pR);
    const T wl = T(0.5) + ph.beta, wr = T(0.5) - ph.beta;
#pragma unroll
    for (int a = 0; a < 5; a++) {
        const T du = uL[a] - uR[a];
        const T fv = (a == 0) ? T(0) : (wl * fvL[a - 1] - wr * fvR[a - 1]);
        F[a] = T(0.5) * (fnL[a] + fnR[a]) + T(0.5) * s * du - fv + ph.tau * du;
    }
    return pL > T(0) && pR > T(0) && uL[0] > T(0) && uR[0] > T(0) && isfinite(s);
}


__device__ __forceinline__ void flag_status(int *status, bool ok)
{
    if (!ok) atomicOr(status, 1);
}
