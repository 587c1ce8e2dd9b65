// fr_pri.cu -- prismatic kernels (p = 3) of the anti-aliased Navier-Stokes FR right-hand side.
//
// A prism is the tensor product of a triangle and a line (Sec. 4.1): every operator is a dense
// triangle-plane block (10 x 10, 25 x 10, 10 x 25, 4 x 10, 10 x 4) applied per z level, times a 1D
// operator along z applied per triangle point. Point index t + 10 k; flux points: face 0 (z = -1)
// and face 1 (z = +1) carry the 10 triangle points, quad faces 2 (y = -1), 3 (x + y = 0) and
// 4 (x = -1) carry 4 x 4 points with local index a + 4 b (a along the edge, b = z level).
// Same three fused phases as the hexahedra: A face solution, B volume group, C interface group.
#include <cuda_runtime.h>

#include "fr_internal.h"
#include "fr_physics.cuh"

namespace {

constexpr int NT_ = FR_PT, NZ = FR_PE, MZ = 5, NQT = FR_PQ;
constexpr int NU = NT_ * NZ;                  // 40
constexpr int NF = 2 * NT_ + 3 * NZ * NZ;     // 68
constexpr int NQ = NQT * MZ;                  // 125
constexpr int FOFF[5] = {0, 10, 20, 36, 52};

__device__ __forceinline__ int face_of(int s) { return s < 10 ? 0 : s < 20 ? 1 : 2 + (s - 20) / 16; }

template <typename T>
__device__ __forceinline__ void pri_normal(const Geo<T> &g, int f, T *n, T &mag)
{
    const T r2 = T(0.70710678118654752440);
    T nr[3] = {T(0), T(0), T(0)};
    if (f == 0) nr[2] = T(-1);
    else if (f == 1) nr[2] = T(1);
    else if (f == 2) nr[1] = T(-1);
    else if (f == 3) { nr[0] = r2; nr[1] = r2; }
    else nr[0] = T(-1);
    T ns[3];
#pragma unroll
    for (int k = 0; k < 3; k++) ns[k] = g.det * (g.Ji[k] * nr[0] + g.Ji[3 + k] * nr[1] + g.Ji[6 + k] * nr[2]);
    mag = sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
    const T im = T(1) / mag;
#pragma unroll
    for (int k = 0; k < 3; k++) n[k] = ns[k] * im;
}

// Value at flux point s of a field stored at solution points (stride 1, index t + 10 k).
template <typename T>
__device__ __forceinline__ T face_value(const PriOps<T> &op, const T *fld, int s)
{
    T v = T(0);
    if (s < 20) {
        const int t = s % 10;
        const T *l = s < 10 ? op.lzL : op.lzR;
#pragma unroll
        for (int k = 0; k < NZ; k++) v += l[k] * fld[t + 10 * k];
    } else {
        const int f = (s - 20) / 16, loc = (s - 20) % 16, a = loc % 4, b = loc / 4;
#pragma unroll
        for (int t = 0; t < NT_; t++) v += op.Ef[f][a][t] * fld[t + 10 * b];
    }
    return v;
}

template <typename T, int NTH>
__device__ __forceinline__ void load_ops(const PriOps<T> *g, PriOps<T> &s)
{
    const int n = sizeof(PriOps<T>) / sizeof(T);
    const T *src = reinterpret_cast<const T *>(g);
    T *dst = reinterpret_cast<T *>(&s);
    for (int i = threadIdx.x; i < n; i += NTH) dst[i] = src[i];
}

// -------------------------------------------------------------------------------------------------
// Phase A: disu
// -------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_pri_disu(HexArgs<T> a, const PriOps<T> *gops)
{
    __shared__ PriOps<T> op;
    load_ops<T, 256>(gops, op);
    __syncthreads();
    const long long total = a.ne * FR_NV * NF;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(it % NF);
        const long long ea = it / NF;
        const int alpha = (int)(ea % FR_NV);
        const long long e = ea / FR_NV;
        a.UF[alpha * a.nfpt + elem_f0(a, e, NF) + s] = face_value(op, a.U + elem_u0(a, e, NU) + alpha * NU, s);
    }
}

// -------------------------------------------------------------------------------------------------
// Phase B: volume group
// -------------------------------------------------------------------------------------------------
template <typename T, int NTH>
__device__ __forceinline__ void pri_interp_5(const PriOps<T> &op, const T *src, T *tmp, T *dst)
{
    for (int it = threadIdx.x; it < 5 * NZ * NQT; it += NTH) {   // triangle plane: (fc, k, q)
        const int fc = it / (NZ * NQT), r = it % (NZ * NQT), k = r / NQT, q = r % NQT;
        T v = T(0);
#pragma unroll
        for (int t = 0; t < NT_; t++) v += op.Bt[q][t] * src[fc * NU + t + 10 * k];
        tmp[fc * NZ * NQT + q + NQT * k] = v;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 5 * MZ * NQT; it += NTH) {   // z: (fc, c, q)
        const int fc = it / (MZ * NQT), r = it % (MZ * NQT), c = r / NQT, q = r % NQT;
        T v = T(0);
#pragma unroll
        for (int k = 0; k < NZ; k++) v += op.Bz[c][k] * tmp[fc * NZ * NQT + q + NQT * k];
        dst[fc * NQ + q + NQT * c] = v;
    }
    __syncthreads();
}

template <typename T, int NTH>
__device__ __forceinline__ void pri_project_5(const PriOps<T> &op, const T *src, T *tmp, T *dst)
{
    for (int it = threadIdx.x; it < 5 * NZ * NQT; it += NTH) {   // z: (fc, k, q)
        const int fc = it / (NZ * NQT), r = it % (NZ * NQT), k = r / NQT, q = r % NQT;
        T v = T(0);
#pragma unroll
        for (int c = 0; c < MZ; c++) v += op.Pz[k][c] * src[fc * NQ + q + NQT * c];
        tmp[fc * NZ * NQT + q + NQT * k] = v;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 5 * NU; it += NTH) {          // triangle plane: (fc, k, t)
        const int fc = it / NU, r = it % NU, k = r / NT_, t = r % NT_;
        T v = T(0);
#pragma unroll
        for (int q = 0; q < NQT; q++) v += op.Pt[t][q] * tmp[fc * NZ * NQT + q + NQT * k];
        dst[fc * NU + t + 10 * k] = v;
    }
    __syncthreads();
}

template <typename T, int NTH>
__global__ void __launch_bounds__(NTH) k_pri_B(HexArgs<T> a, const PriOps<T> *gops)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PriOps<T> &op = *reinterpret_cast<PriOps<T> *>(smem_raw);
    T *s_u = reinterpret_cast<T *>(smem_raw + ((sizeof(PriOps<T>) + 15) / 16) * 16);
    T *s_q = s_u + 5 * NU;
    T *s_c = s_q + 15 * NU;
    T *s_w = s_c + 5 * NF;
    T *s_t = s_w + 20 * NQ;
    load_ops<T, NTH>(gops, op);
    for (long long e = blockIdx.x; e < a.ne; e += gridDim.x) {
        const Geo<T> g = a.geo[e];
        const Phys<T> ph = elem_phys(a, e);
        const T *U = a.U + elem_u0(a, e, NU);
        const long long gf0 = elem_f0(a, e, NF);
        for (int it = threadIdx.x; it < 5 * NU; it += NTH) s_u[it] = U[it];
        for (int it = threadIdx.x; it < 5 * NF; it += NTH) {   // con_u
            const int alpha = it / NF, s = it % NF;
            const uint32_t pc = a.partner[gf0 + s];
            const bool isL = (pc & FR_LFLAG) != 0;
            const long long pg = pc & ~FR_LFLAG;
            const T own = a.UF[alpha * a.nfpt + gf0 + s], oth = a.UF[alpha * a.nfpt + pg];
            const T uL = isL ? own : oth, uR = isL ? oth : own;
            s_c[it] = (T(0.5) - ph.beta) * uL + (T(0.5) + ph.beta) * uR;
        }
        __syncthreads();
        // corrected gradient: z lines (alpha, t) and triangle planes (alpha, k, t)
        for (int it = threadIdx.x; it < 5 * NT_; it += NTH) {
            const int alpha = it / NT_, t = it % NT_;
            T u[NZ];
#pragma unroll
            for (int k = 0; k < NZ; k++) u[k] = s_u[alpha * NU + t + 10 * k];
            const T cB = s_c[alpha * NF + t], cT = s_c[alpha * NF + 10 + t];
#pragma unroll
            for (int k = 0; k < NZ; k++) {
                T v = op.liftzR[k] * cT - op.liftzL[k] * cB;
#pragma unroll
                for (int j = 0; j < NZ; j++) v += op.Dhz[k][j] * u[j];
                s_q[(alpha * 3 + 2) * NU + t + 10 * k] = v;
            }
        }
        for (int it = threadIdx.x; it < 5 * NU; it += NTH) {
            const int alpha = it / NU, r = it % NU, k = r / NT_, t = r % NT_;
            const T *u = s_u + alpha * NU + 10 * k;
            T vx = T(0), vy = T(0);
#pragma unroll
            for (int j = 0; j < NT_; j++) { vx += op.Dhx[t][j] * u[j]; vy += op.Dhy[t][j] * u[j]; }
#pragma unroll
            for (int f = 0; f < 3; f++) {
                T l = T(0);
#pragma unroll
                for (int b = 0; b < NZ; b++) l += op.Lf[f][t][b] * s_c[alpha * NF + 20 + 16 * f + b + 4 * k];
                vx += op.nf[f][0] * l;
                vy += op.nf[f][1] * l;
            }
            s_q[(alpha * 3 + 0) * NU + t + 10 * k] = vx;
            s_q[(alpha * 3 + 1) * NU + t + 10 * k] = vy;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 5 * NU; it += NTH) {   // gradcoru
            const int alpha = it / NU, z = it % NU;
            T *q = s_q + alpha * 3 * NU + z;
            const T q0 = q[0], q1 = q[NU], q2 = q[2 * NU];
#pragma unroll
            for (int k = 0; k < 3; k++) q[k * NU] = g.Ji[k] * q0 + g.Ji[3 + k] * q1 + g.Ji[6 + k] * q2;
        }
        __syncthreads();
        for (int s = threadIdx.x; s < NF; s += NTH) {          // viscous normal flux at own flux points
            T uf[5], qf[5][3];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                uf[alpha] = face_value(op, s_u + alpha * NU, s);
#pragma unroll
                for (int d = 0; d < 3; d++) qf[alpha][d] = face_value(op, s_q + (alpha * 3 + d) * NU, s);
            }
            const T *nt = a.fnrm + (e * 6 + face_of(s)) * 4;
            T n[3] = {nt[0], nt[1], nt[2]};
            T fvn[4];
            viscous_normal_flux(ph, uf, qf, n, fvn);
#pragma unroll
            for (int k = 0; k < 4; k++) a.FV[k * a.nfpt + gf0 + s] = fvn[k];
        }
        pri_interp_5<T, NTH>(op, s_u, s_t, s_w);
#pragma unroll 1
        for (int c = 0; c < 3; c++) pri_interp_5<T, NTH>(op, s_q + 5 * c * NU, s_t, s_w + (5 + 5 * c) * NQ);
        bool ok = true;
        for (int q = threadIdx.x; q < NQ; q += NTH) {          // tdisf
            T u[5], gq[5][3], f[3][5];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                u[alpha] = s_w[alpha * NQ + q];
#pragma unroll
                for (int d = 0; d < 3; d++) gq[alpha][d] = s_w[(5 + alpha * 3 + d) * NQ + q];
            }
            ok &= total_flux(ph, u, gq, f);
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++)
#pragma unroll
                for (int d = 0; d < 3; d++)
                    s_w[(alpha * 3 + d) * NQ + q] = g.det * (g.Ji[3 * d] * f[0][alpha] + g.Ji[3 * d + 1] * f[1][alpha] + g.Ji[3 * d + 2] * f[2][alpha]);
        }
        flag_status(a.status, ok);
        __syncthreads();
#pragma unroll 1
        for (int c = 0; c < 3; c++) pri_project_5<T, NTH>(op, s_w + 5 * c * NQ, s_t, s_q + 5 * c * NU);
        T *R = a.R + elem_u0(a, e, NU);
        for (int it = threadIdx.x; it < 5 * NU; it += NTH) {   // corrected divergence
            const int alpha = it / NU, r = it % NU, k = r / NT_, t = r % NT_;
            const T *F = s_q + alpha * 3 * NU;
            T v = T(0);
#pragma unroll
            for (int j = 0; j < NT_; j++) v += op.Dhx[t][j] * F[j + 10 * k] + op.Dhy[t][j] * F[NU + j + 10 * k];
#pragma unroll
            for (int j = 0; j < NZ; j++) v += op.Dhz[k][j] * F[2 * NU + t + 10 * j];
            R[it] = v;
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------------------------------------
// Phase C: interface group
// -------------------------------------------------------------------------------------------------
template <typename T, int NTH>
__global__ void __launch_bounds__(NTH) k_pri_C(HexArgs<T> a, const PriOps<T> *gops)
{
    __shared__ PriOps<T> op;
    __shared__ T s_d[5 * NF];
    load_ops<T, NTH>(gops, op);
    __syncthreads();
    for (long long e = blockIdx.x; e < a.ne; e += gridDim.x) {
        const Geo<T> g = a.geo[e];
        const Phys<T> ph = elem_phys(a, e);
        const long long gf0 = elem_f0(a, e, NF);
        bool ok = true;
        for (int s = threadIdx.x; s < NF; s += NTH) {
            const uint32_t pc = a.partner[gf0 + s];
            const bool isL = (pc & FR_LFLAG) != 0;
            const long long pg = pc & ~FR_LFLAG, og = gf0 + s;
            T uo[5], up[5], fvo[4], fvp[4];
#pragma unroll
            for (int k = 0; k < 5; k++) { uo[k] = a.UF[k * a.nfpt + og]; up[k] = a.UF[k * a.nfpt + pg]; }
#pragma unroll
            for (int k = 0; k < 4; k++) { fvo[k] = a.FV[k * a.nfpt + og]; fvp[k] = a.FV[k * a.nfpt + pg]; }
            const T *nt = a.fnrm + (e * 6 + face_of(s)) * 4;
            T n[3] = {nt[0], nt[1], nt[2]};
            const T mag = nt[3];
            T nL[3] = {isL ? n[0] : -n[0], isL ? n[1] : -n[1], isL ? n[2] : -n[2]};
            T F[5];
            ok &= isL ? common_flux(ph, uo, up, fvo, fvp, nL, F) : common_flux(ph, up, uo, fvp, fvo, nL, F);
            const T sc = isL ? mag : -mag;
#pragma unroll
            for (int k = 0; k < 5; k++) s_d[k * NF + s] = sc * F[k];
        }
        flag_status(a.status, ok);
        __syncthreads();
        T *R = a.R + elem_u0(a, e, NU);
        const T idet = T(-1) / g.det;
        for (int it = threadIdx.x; it < 5 * NU; it += NTH) {
            const int alpha = it / NU, r = it % NU, k = r / NT_, t = r % NT_;
            const T *D = s_d + alpha * NF;
            T v = R[it] + op.liftzL[k] * D[t] + op.liftzR[k] * D[10 + t];
#pragma unroll
            for (int f = 0; f < 3; f++)
#pragma unroll
                for (int b = 0; b < NZ; b++) v += op.Lf[f][t][b] * D[20 + 16 * f + b + 4 * k];
            if (a.rkstage == 0) R[it] = v * idet;
            else rk_fold(a, elem_u0(a, e, NU) + it, v * idet);
        }
        __syncthreads();
    }
}

int grid_elems(long long ne, int per_sm)
{
    long long g = ne;
    if (g > 152LL * per_sm * 8) g = 152LL * per_sm * 8;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T>
int pri_fused_phase(int phase, const HexArgs<T> &a, const PriOps<T> *ops, cudaStream_t s)
{
    if (a.ne == 0) return 0;
    if (phase == 0) {
        long long work = a.ne * FR_NV * NF;
        long long g = (work + 255) / 256;
        if (g > 152LL * 64) g = 152LL * 64;
        k_pri_disu<T><<<(int)g, 256, 0, s>>>(a, ops);
    } else if (phase == 1) {
        constexpr int NTH = 128;
        const size_t smem = ((sizeof(PriOps<T>) + 15) / 16) * 16 + (size_t)(5 * NU + 15 * NU + 5 * NF + 20 * NQ + 5 * NZ * NQT) * sizeof(T);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_pri_B<T, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_pri_B<T, NTH><<<grid_elems(a.ne, 8), NTH, smem, s>>>(a, ops);
    } else {
        k_pri_C<T, 128><<<grid_elems(a.ne, 8), 128, 0, s>>>(a, ops);
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template int pri_fused_phase<double>(int, const HexArgs<double> &, const PriOps<double> *, cudaStream_t);
template int pri_fused_phase<float>(int, const HexArgs<float> &, const PriOps<float> *, cudaStream_t);
