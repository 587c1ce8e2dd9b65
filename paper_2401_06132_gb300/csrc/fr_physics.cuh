// fr_physics.cuh -- pointwise physics of the compressible Navier-Stokes equations (Sec. 2.1),
// shared by the hexahedral and prismatic kernels.
#pragma once

#include "fr_internal.h"

// ---------------------------------------------------------------------------------------------
// Point physics (Sec. 2.1): total flux f = f^e - f^v, viscous normal flux, Rusanov common flux
// ---------------------------------------------------------------------------------------------

// rho times the velocity gradient, w[i][d] = rho dv_i/dx_d = d(rho v_i)/dx_d - v_i d(rho)/dx_d; the
// factor 1/rho is folded into the coefficients that multiply it (mu/rho, heat/rho).
template <typename T>
__device__ __forceinline__ void rho_dv(const T *v, const T (*g)[3], T (*w)[3])
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int d = 0; d < 3; d++) w[i][d] = g[1 + i][d] - v[i] * g[0][d];
}

// The symmetric viscous stress tau[i][d] = mu (dv_i/dx_d + dv_d/dx_i) - 2/3 mu div v delta_id from
// w = rho dv and mr = mu / rho (six distinct entries).
template <typename T>
__device__ __forceinline__ void viscous_stress(const T mr, const T (*w)[3], T (*tau)[3])
{
    const T lam = T(-2.0 / 3.0) * mr * (w[0][0] + w[1][1] + w[2][2]);
    const T m2 = mr + mr;
#pragma unroll
    for (int i = 0; i < 3; i++) tau[i][i] = m2 * w[i][i] + lam;
    tau[0][1] = tau[1][0] = mr * (w[0][1] + w[1][0]);
    tau[0][2] = tau[2][0] = mr * (w[0][2] + w[2][0]);
    tau[1][2] = tau[2][1] = mr * (w[1][2] + w[2][1]);
}

// Physical total flux f[d][alpha] from the state u and its physical gradient g[alpha][d].
// Returns false for a non-physical state (rho <= 0, p <= 0 or non-finite).
template <typename T>
__device__ __forceinline__ bool total_flux(const Phys<T> &ph, const T *u, const T (*g)[3], T (*f)[5])
{
    const T rho = u[0], ir = T(1) / rho;
    const T v[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
    const T E = u[4];
    const T p = ph.gm1 * (E - T(0.5) * (u[1] * v[0] + u[2] * v[1] + u[3] * v[2]));
    T w[3][3], tau[3][3];
    rho_dv(v, g, w);
    viscous_stress(ph.mu * ir, w, tau);
    const T er = E * ir, hr = ph.heat * ir, pm = p - ph.pref, ep = E + p;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        // heat flux mu gamma/Pr [d(E/rho) - v.dv] = mu gamma/((gamma-1)Pr) d(p/rho)
        const T phi = hr * ((g[4][d] - er * g[0][d]) - (v[0] * w[0][d] + v[1] * w[1][d] + v[2] * w[2][d]));
        f[d][0] = u[1 + d];
        f[d][1] = u[1] * v[d] + (d == 0 ? pm : T(0)) - tau[0][d];
        f[d][2] = u[2] * v[d] + (d == 1 ? pm : T(0)) - tau[1][d];
        f[d][3] = u[3] * v[d] + (d == 2 ? pm : T(0)) - tau[2][d];
        f[d][4] = v[d] * ep - (v[0] * tau[0][d] + v[1] * tau[1][d] + v[2] * tau[2][d] + phi);
    }
    return rho > T(0) && p > T(0) && isfinite(p) && isfinite(f[0][4] + f[1][4] + f[2][4]);
}

// n . f^v for variables 1..4 (the mass component is zero).
template <typename T>
__device__ __forceinline__ void viscous_normal_flux(const Phys<T> &ph, const T *u, const T (*g)[3], const T *n, T *fvn)
{
    const T rho = u[0], ir = T(1) / rho;
    const T v[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
    T w[3][3], tau[3][3];
    rho_dv(v, g, w);
    viscous_stress(ph.mu * ir, w, tau);
    const T er = u[4] * ir;
#pragma unroll
    for (int i = 0; i < 3; i++) fvn[i] = n[0] * tau[i][0] + n[1] * tau[i][1] + n[2] * tau[i][2];
    // n . (tau v + phi) = v . (tau n) + n . phi
    T nphi = T(0);
#pragma unroll
    for (int d = 0; d < 3; d++) nphi += n[d] * ((g[4][d] - er * g[0][d]) - (v[0] * w[0][d] + v[1] * w[1][d] + v[2] * w[2][d]));
    fvn[3] = v[0] * fvn[0] + v[1] * fvn[1] + v[2] * fvn[2] + ph.heat * ir * nphi;
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

// -------------------------------------------------------------------------------------------------
// Low-Mach FP32 form. The state is carried as deviations w = (rho - rref, rho v, E - eref) from a
// reference state at rest with (gamma - 1) eref = pref, and the energy equation is replaced by the
// reduced energy E - H0 rho (H0 = (eref + pref)/rref), whose flux is
//   v (E + p) - H0 rho v - f^v_E = v (E' + p' - H0 rho') - f^v_E,   p' = p - pref,
// a difference of O(1) terms instead of O(1/(gamma M^2)) ones. The mass equation is carried in FP64
// by the callers, and R_E = R_(E - H0 rho) + H0 R_rho. All of this is exact in exact arithmetic.
// -------------------------------------------------------------------------------------------------

// Fluxes f[d][a] of (rho, rho v, E - H0 rho) from the deviations w and the physical gradient g
// (gradients of deviations equal gradients of the conserved variables). The mass flux f[d][0] = rho v
// is written only with `mass` (elements whose mass equation runs through the FP32 flux path);
// otherwise it is 0 and the float-float mass channel carries it.
__device__ __forceinline__ bool total_flux_dev(const Phys<float> &ph, const float *w, const float (*g)[3], float (*f)[5],
                                               bool mass = false)
{
    const float rho = ph.rref + w[0], ir = 1.0f / rho;
    const float v[3] = {w[1] * ir, w[2] * ir, w[3] * ir};
    const float pd = ph.gm1 * (w[4] - 0.5f * (w[1] * v[0] + w[2] * v[1] + w[3] * v[2]));
    const float er = (ph.eref + w[4]) * ir, hr = ph.heat * ir;
    float rw[3][3], tau[3][3];
    rho_dv(v, g, rw);
    viscous_stress(ph.mu * ir, rw, tau);
    const float hred = w[4] + pd - ph.H0 * w[0];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float phi = hr * ((g[4][d] - er * g[0][d]) - (v[0] * rw[0][d] + v[1] * rw[1][d] + v[2] * rw[2][d]));
        f[d][0] = mass ? w[1 + d] : 0.0f;
        f[d][1] = w[1] * v[d] + (d == 0 ? pd : 0.0f) - tau[0][d];
        f[d][2] = w[2] * v[d] + (d == 1 ? pd : 0.0f) - tau[1][d];
        f[d][3] = w[3] * v[d] + (d == 2 ? pd : 0.0f) - tau[2][d];
        f[d][4] = v[d] * hred - (v[0] * tau[0][d] + v[1] * tau[1][d] + v[2] * tau[2][d] + phi);
    }
    return rho > 0.0f && ph.pref + pd > 0.0f && isfinite(pd) && isfinite(f[0][4] + f[1][4] + f[2][4]);
}

// Common normal flux of (rho v, E - H0 rho) (F[1..4]) from deviation states, with the same Rusanov
// and LDG rules as common_flux; returns the Rusanov wave speed in s for the FP64 mass flux.
__device__ __forceinline__ bool common_flux_dev(const Phys<float> &ph, const float *wL, const float *wR,
                                                const float *fvL, const float *fvR, const float *n, float *F, float &s)
{
    const float rL = ph.rref + wL[0], rR = ph.rref + wR[0];
    const float irL = 1.0f / rL, irR = 1.0f / rR;
    const float vnL = (wL[1] * n[0] + wL[2] * n[1] + wL[3] * n[2]) * irL;
    const float vnR = (wR[1] * n[0] + wR[2] * n[1] + wR[3] * n[2]) * irR;
    const float pdL = ph.gm1 * (wL[4] - 0.5f * irL * (wL[1] * wL[1] + wL[2] * wL[2] + wL[3] * wL[3]));
    const float pdR = ph.gm1 * (wR[4] - 0.5f * irR * (wR[1] * wR[1] + wR[2] * wR[2] + wR[3] * wR[3]));
    const float pL = ph.pref + pdL, pR = ph.pref + pdR;
    const float cL = sqrtf(ph.gamma * pL * irL), cR = sqrtf(ph.gamma * pR * irR);
    s = fmaxf(fabsf(vnL) + cL, fabsf(vnR) + cR);
    float fnL[5], fnR[5], du[5];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        fnL[1 + i] = wL[1 + i] * vnL + pdL * n[i];
        fnR[1 + i] = wR[1 + i] * vnR + pdR * n[i];
        du[1 + i] = wL[1 + i] - wR[1 + i];
    }
    fnL[4] = vnL * (wL[4] + pdL - ph.H0 * wL[0]);
    fnR[4] = vnR * (wR[4] + pdR - ph.H0 * wR[0]);
    du[4] = (wL[4] - wR[4]) - ph.H0 * (wL[0] - wR[0]);
    const float wl = 0.5f + ph.beta, wr = 0.5f - ph.beta;
    F[0] = 0.0f;
#pragma unroll
    for (int a = 1; a < 5; a++)
        F[a] = 0.5f * (fnL[a] + fnR[a]) + 0.5f * s * du[a] - (wl * fvL[a - 1] - wr * fvR[a - 1]) + ph.tau * du[a];
    return pL > 0.0f && pR > 0.0f && rL > 0.0f && rR > 0.0f && isfinite(s);
}

// The common normal mass flux in FP32 from deviation states (the Rusanov and penalty terms of
// common_flux; the mass has no viscous flux), with the wave speed s returned by common_flux_dev:
// 1/2 nL.(rho v_L + rho v_R) + (s/2 + tau)(rho_L - rho_R).
__device__ __forceinline__ float common_mass_flux_dev(const Phys<float> &ph, const float *wL, const float *wR,
                                                      const float *n, float s)
{
    const float mL = wL[1] * n[0] + wL[2] * n[1] + wL[3] * n[2], mR = wR[1] * n[0] + wR[2] * n[1] + wR[3] * n[2];
    const float du = wL[0] - wR[0];
    return 0.5f * (mL + mR) + 0.5f * s * du + ph.tau * du;
}
