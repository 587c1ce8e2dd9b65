// fr_pri_body.cuh -- the prismatic (p = 3) phase bodies of the anti-aliased Navier-Stokes FR
// right-hand side (face solution, volume group, interface group; Sec. 4.1 factorisation), as device
// functions over the elements first, first + stride, ... of a launch: fr_pri.cu launches them on
// their own, and fr_hex.cu inside the launches that serve several element groups at once.
#pragma once

#include <cuda_runtime.h>

#include "fr_internal.h"
#include "fr_physics.cuh"
#include "fr_tcgen05.cuh"

namespace pri {
namespace {

constexpr int NT_ = FR_PT, NZ = FR_PE, MZ = 5, NQT = FR_PQ;
constexpr int NU = NT_ * NZ;                  // 40
constexpr int NF = 2 * NT_ + 3 * NZ * NZ;     // 68
constexpr int NQ = NQT * MZ;                  // 125

__device__ __forceinline__ int face_of(int s) { return s < 10 ? 0 : s < 20 ? 1 : 2 + (s - 20) / 16; }

// The FP32 operator table in constant memory (one copy per translation unit that includes this
// file, filled by set_const_ops on each device): read with compile-time indices, its entries are
// constant-bank operands of the multiply-adds instead of a shared-memory load per coefficient.
__constant__ PriOps<float> c_pri32;

inline int set_const_ops(const PriOps<float> &h)
{
    return cudaMemcpyToSymbol(c_pri32, &h, sizeof(h)) == cudaSuccess ? 0 : -1;
}

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

// An entry of the float-float table: its hi part and the lo part at the same offset.
__device__ __forceinline__ ff ffop(const PriOpsFF &o, const float &hi)
{
    // the lo part sits at the same offset in the second table
    const float *h = &hi;
    return ff{hi, *(reinterpret_cast<const float *>(&o.lo) + (h - reinterpret_cast<const float *>(&o.hi)))};
}

// Same, of the field minus a constant, with the float-float table (a compensated dot product, Dot2):
// the face value to about 48 bits before its final rounding to FP32.
__device__ __forceinline__ ff face_value_ff_off(const PriOpsFF &o, const float *fld, int s, float off)
{
    float sh, c;
    if (s < 20) {
        const int t = s % 10;
        const float *l = s < 10 ? o.hi.lzL : o.hi.lzR;
        dot2_first(ffop(o, l[0]), fld[t] - off, sh, c);
#pragma unroll
        for (int k = 1; k < NZ; k++) dot2_next(ffop(o, l[k]), fld[t + 10 * k] - off, sh, c);
    } else {
        const int f = (s - 20) / 16, loc = (s - 20) % 16, a = loc % 4, b = loc / 4;
        dot2_first(ffop(o, o.hi.Ef[f][a][0]), fld[10 * b] - off, sh, c);
#pragma unroll
        for (int t = 1; t < NT_; t++) dot2_next(ffop(o, o.hi.Ef[f][a][t]), fld[t + 10 * b] - off, sh, c);
    }
    return fast_two_sum(sh, c);
}

template <typename T, int NTH>
__device__ __forceinline__ void load_ops(const PriOps<T> *g, PriOps<T> &s)
{
    const int n = sizeof(PriOps<T>) / sizeof(T);
    const T *src = reinterpret_cast<const T *>(g);
    T *dst = reinterpret_cast<T *>(&s);
    for (int i = threadIdx.x; i < n; i += NTH) dst[i] = src[i];
}


// Shared-memory operands of the tensor-core contractions (bytes, 128-byte aligned pieces), for the
// split form TCM (1: FP16 in three K segments, 2: BF16 in six; tc::SplitForm).
constexpr int TC_ROWS_I = 20 * MZ, TC_ROWS_P = 15 * MZ;    // 100 and 75 rows of M = 128
constexpr int TC_ST = 11;                                  // row stride of the projected rows
template <int TCM>
struct PriTC {
    static constexpr int KI = tc::split_k<TCM>(NT_), NI = 32;    // interpolation: K = segments x 10 (padded), N = 25 (+7)
    static constexpr int KP = tc::split_k<TCM>(NQT), NP = 16;    // projection: K = segments x 25 (padded), N = 10 (+6)
    static constexpr int SBO_I = KI / 8 * 128, SBO_P = KP / 8 * 128;
    // The A tile holds the rows an element writes (the larger layout of the two); the MMA reads
    // all 128 rows, and the ones past the element's last run on into the buffers that follow the
    // tile (the operator tiles and the kernel's arrays), feeding accumulator lanes never read.
    static constexpr int A_I = (TC_ROWS_I + 7) / 8 * SBO_I, A_P = (TC_ROWS_P + 7) / 8 * SBO_P;
    static constexpr int A_BYTES = ((A_I > A_P ? A_I : A_P) + 127) / 128 * 128;
    static constexpr int BI_BYTES = NI / 8 * SBO_I, BP_BYTES = NP / 8 * SBO_P;
    static constexpr int HEAD = A_BYTES + BI_BYTES + BP_BYTES + 128 * 4 + 16;   // tiles, row shifts, barrier, TMEM slot
    static constexpr int BYTES = HEAD + 128;                                     // + alignment slack
    static constexpr uint32_t IDESC_I = tc::idesc_f16(TCM - 1, 128, NI), IDESC_P = tc::idesc_f16(TCM - 1, 128, NP);
    static_assert(TC_ROWS_I <= 128 && TC_ROWS_P <= 128, "one M = 128 tile per element");
    static_assert(16 * SBO_I <= HEAD + (5 * NU + 15 * NU + 5 * NF + 20 * NQ) * 4 &&
                      16 * SBO_P <= HEAD + (5 * NU + 15 * NU + 5 * NF + 20 * NQ) * 4,
                  "the 128 rows an MMA reads stay inside the CTA's shared memory");
};

// -------------------------------------------------------------------------------------------------
// Phase A: disu
// -------------------------------------------------------------------------------------------------
// The reduced precisions evaluate the face values with the float-float operator table (compensated:
// exact products, TwoSum accumulation) and round once: the quad-face rows of the triangle
// interpolation extrapolate from interior points (row sums of |Ef| well above 1), and at low Mach
// the Rusanov dissipation (1/2)(|v.n| + c)(u_L - u_R), with c about 10 |v|, lifts any rounding of a
// face value into R. Low-Mach form (ph.dev): the face solution of the deviations from the reference
// state, and the own-normal mass flux n.(rho v) at every flux point in float-float.
template <typename T>
__device__ __forceinline__ void pri_disu_body(const HexArgs<T> &a, const PriOps<T> *gops, const PriOpsFF *opsff, long long first, long long stride)
{
    constexpr bool F32 = sizeof(T) == 4;
    __shared__ __align__(16) unsigned char raw[F32 ? sizeof(PriOpsFF) : sizeof(PriOps<T>)];
    if constexpr (F32) {
        const float *src = reinterpret_cast<const float *>(opsff);
        float *dst = reinterpret_cast<float *>(raw);
        for (int i = threadIdx.x; i < (int)(sizeof(PriOpsFF) / sizeof(float)); i += 256) dst[i] = src[i];
    } else {
        load_ops<T, 256>(gops, *reinterpret_cast<PriOps<T> *>(raw));
    }
    __syncthreads();
    const long long total = a.ne * NF;
    for (long long it = first * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)stride * blockDim.x) {
        // one thread per (element, flux point), all five variables
        const int s = (int)(it % NF);
        const long long e = it / NF;
#ifdef FR_DEBUG_BOUNDS
        {
            const long long u0 = elem_u0(a, e, NU), f0 = elem_f0(a, e, NF);
            if (u0 < 0 || u0 + (long long)FR_NV * NU > a.nU || f0 < 0 || f0 + NF > a.nfpt) {
                atomicOr(a.status, 4);
                continue;
            }
        }
#endif
        const T *u = a.U + elem_u0(a, e, NU);
        const long long fo = elem_f0(a, e, NF) + s;
        if constexpr (F32) {
            const PriOpsFF &o = *reinterpret_cast<const PriOpsFF *>(raw);
            const Phys<T> ph = elem_phys(a, e);
            const bool dev = ph.dev != 0;
            ff v[FR_NV];
#pragma unroll
            for (int alpha = 0; alpha < FR_NV; alpha++) {
                const float off = dev ? (alpha == 0 ? ph.rref : (alpha == 4 ? ph.eref : 0.0f)) : 0.0f;
                v[alpha] = face_value_ff_off(o, u + alpha * NU, s, off);
                a.UF[alpha * a.nfpt + fo] = v[alpha].hi + v[alpha].lo;
            }
            if (dev) {
                const ff *nt = a.fnrm64 + (e * 6 + face_of(s)) * 4;
                ff mf = ff_of(0.0f);
#pragma unroll
                for (int k = 0; k < 3; k++)
                    if (nt[k].hi != 0.0f) mf = ff_fma(nt[k], v[1 + k], mf);
                a.MF[fo] = mf;
            }
        } else {
            const PriOps<T> &op = *reinterpret_cast<const PriOps<T> *>(raw);
#pragma unroll
            for (int alpha = 0; alpha < FR_NV; alpha++) a.UF[alpha * a.nfpt + fo] = face_value(op, u + alpha * NU, s);
        }
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

// FP32 without tensor cores, all 20 fields: the triangle-plane factor with one thread per (field, z
// level) line, its 10 values in registers and all 25 quadrature points formed from them, then z with
// one thread per (field, triangle quadrature point); the operators from the constant-memory table
// with compile-time indices.
template <int NTH>
__device__ __forceinline__ void pri_interp_all_c(const float *src, float *tmp, float *dst)
{
    for (int it = threadIdx.x; it < 20 * NZ; it += NTH) {   // triangle plane: (f, k)
        const float *s = src + (it / NZ) * NU + 10 * (it % NZ);
        float u[NT_];
#pragma unroll
        for (int t = 0; t < NT_; t++) u[t] = s[t];
        float *d = tmp + it * NQT;   // (f NZ + k) NQT + q
#pragma unroll
        for (int q = 0; q < NQT; q++) {
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < NT_; t++) v += c_pri32.Bt[q][t] * u[t];
            d[q] = v;
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 20 * NQT; it += NTH) {   // z: (f, q)
        const int f = it / NQT, q = it % NQT;
        float u[NZ];
#pragma unroll
        for (int k = 0; k < NZ; k++) u[k] = tmp[(f * NZ + k) * NQT + q];
#pragma unroll
        for (int c = 0; c < MZ; c++) {
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < NZ; k++) v += c_pri32.Bz[c][k] * u[k];
            dst[f * NQ + q + NQT * c] = v;
        }
    }
    __syncthreads();
}

// The projection of the 15 flux fields in the same form: z with one thread per (field, triangle
// quadrature point), then the triangle plane with one thread per (field, z level) line, its 25
// values in registers.
template <int NTH>
__device__ __forceinline__ void pri_project_all_c(const float *src, float *tmp, float *dst)
{
    for (int it = threadIdx.x; it < 15 * NQT; it += NTH) {   // z: (f, q)
        const int f = it / NQT, q = it % NQT;
        float u[MZ];
#pragma unroll
        for (int c = 0; c < MZ; c++) u[c] = src[f * NQ + q + NQT * c];
#pragma unroll
        for (int k = 0; k < NZ; k++) {
            float v = 0.f;
#pragma unroll
            for (int c = 0; c < MZ; c++) v += c_pri32.Pz[k][c] * u[c];
            tmp[(f * NZ + k) * NQT + q] = v;
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 15 * NZ; it += NTH) {   // triangle plane: (f, k)
        const float *s = tmp + it * NQT;
        float u[NQT];
#pragma unroll
        for (int q = 0; q < NQT; q++) u[q] = s[q];
        float *d = dst + (it / NZ) * NU + 10 * (it % NZ);
#pragma unroll
        for (int t = 0; t < NT_; t++) {
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < NQT; q++) v += c_pri32.Pt[t][q] * u[q];
            d[t] = v;
        }
    }
    __syncthreads();
}

template <typename T, int NTH, int TCM>
__device__ __forceinline__ void pri_B_body(const HexArgs<T> &a, const PriOps<T> *gops, const PriOpsFF *opsff, long long first, long long stride)
{
    static_assert(TCM == 0 || (NTH == 128 && sizeof(T) == 4), "tensor-core form: FP32, one warpgroup per element");
    using PT = PriTC<TCM == 0 ? 1 : TCM>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ff s_mf[sizeof(T) == 4 ? 3 * NU : 1];   // low-Mach form: transformed mass flux
    __shared__ short s_plist[NF];                         // flux points that need the viscous flux
    __shared__ int s_pcnt;
    PriOps<T> &op = *reinterpret_cast<PriOps<T> *>(smem_raw);
    unsigned char *arr = smem_raw + ((sizeof(PriOps<T>) + 15) / 16) * 16;
    // tensor-core state (TCM != 0): the tiles come first, so that the MMA's rows past an element's
    // last run on into the arrays below
    unsigned char *tA = nullptr, *tBi = nullptr, *tBp = nullptr;
    int *s_sh = nullptr;
    uint64_t *mbar = nullptr;
    uint32_t *s_tmem = nullptr, tmem = 0, parity = 0;
    bool tc_fail = false, first_wait = true;
    if constexpr (TCM != 0) {
        const uint32_t raw = tc::smem_u32(arr);
        tA = arr + ((128 - (raw & 127)) & 127);
        tBi = tA + PT::A_BYTES;
        tBp = tBi + PT::BI_BYTES;
        s_sh = reinterpret_cast<int *>(tBp + PT::BP_BYTES);
        mbar = reinterpret_cast<uint64_t *>(s_sh + 128);
        s_tmem = reinterpret_cast<uint32_t *>(mbar + 1);
        arr = tA + PT::HEAD;
    }
    T *s_u = reinterpret_cast<T *>(arr);
    T *s_q = s_u + 5 * NU;
    T *s_c = s_q + 15 * NU;
    T *s_w = s_c + 5 * NF;
    T *s_t = s_w + 20 * NQ;
    load_ops<T, NTH>(gops, op);
    if constexpr (TCM != 0) {
        tc::setup(mbar, s_tmem, 32);
        __syncthreads();   // operators in shared memory
        // operator tiles in the split form's segments (FP16: [B_hi | B_hi | B_lo])
        using SF = tc::SplitForm<TCM>;
        for (int i = threadIdx.x; i < PT::NI * PT::KI; i += NTH) {
            const int n = i / PT::KI, k = i % PT::KI, sg = k / NT_;
            uint16_t pp[3] = {0, 0, 0};
            if (n < NQT && sg < SF::SEGS) tc::split_parts<TCM>((float)op.Bt[n][k % NT_], pp);
            *reinterpret_cast<uint16_t *>(tBi + tc::core_offset(n, k, PT::SBO_I)) = sg < SF::SEGS ? pp[SF::y_part(sg)] : (uint16_t)0;
        }
        for (int i = threadIdx.x; i < PT::NP * PT::KP; i += NTH) {
            const int n = i / PT::KP, k = i % PT::KP, sg = k / NQT;
            uint16_t pp[3] = {0, 0, 0};
            if (n < NT_ && sg < SF::SEGS) tc::split_parts<TCM>((float)op.Pt[n][k % NQT], pp);
            *reinterpret_cast<uint16_t *>(tBp + tc::core_offset(n, k, PT::SBO_P)) = sg < SF::SEGS ? pp[SF::y_part(sg)] : (uint16_t)0;
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tmem = *s_tmem;
    }
    for (long long e = first; e < a.ne; e += stride) {
        if (!fr_elem_ok(a, e, NU, NF)) continue;
        const Geo<T> g = a.geo[e];
        const Phys<T> ph = elem_phys(a, e);
        const T *U = a.U + elem_u0(a, e, NU);
        const long long gf0 = elem_f0(a, e, NF);
        bool dev = false;
        if constexpr (sizeof(T) == 4) dev = ph.dev != 0;
        for (int it = threadIdx.x; it < 5 * NU; it += NTH) {
            T v = U[it];
            if (dev) v -= it < NU ? ph.rref : (it >= 4 * NU ? ph.eref : T(0));
            s_u[it] = v;
        }
        if (threadIdx.x == 0) s_pcnt = 0;
        for (int it = threadIdx.x; it < 5 * NF; it += NTH) {   // con_u
            const int alpha = it / NF, s = it % NF;
            const uint32_t pc = a.partner[gf0 + s];
            const bool isL = (pc & FR_LFLAG) != 0;
            const long long pg = fr_partner(a, pc, gf0 + s);
            const T own = a.UF[alpha * a.nfpt + gf0 + s], oth = a.UF[alpha * a.nfpt + pg];
            const T uL = isL ? own : oth, uR = isL ? oth : own;
            s_c[it] = (T(0.5) - ph.beta) * uL + (T(0.5) + ph.beta) * uR;
        }
        __syncthreads();
        // low-Mach form: volume part of R~_rho in float-float (rho v lies in the solution space, so
        // its projection is itself and the corrected divergence applies at the solution points).
        // The tensor-core forms run it while the projection's MMA chain is in flight.
        auto mass_channel = [&]() {
            if constexpr (sizeof(T) == 4) {
                if (dev) {
                    const ff *cm = a.geo64[e].cm;   // det J J^-1, per element
                    for (int z = threadIdx.x; z < NU; z += NTH) {
                        const float m0 = s_u[NU + z], m1 = s_u[2 * NU + z], m2 = s_u[3 * NU + z];
#pragma unroll
                        for (int d = 0; d < 3; d++)
                            s_mf[d * NU + z] = ff_add(ff_add(ff_mul_f(cm[3 * d], m0), ff_mul_f(cm[3 * d + 1], m1)), ff_mul_f(cm[3 * d + 2], m2));
                    }
                    __syncthreads();
                    const PriOpsFF &o = *opsff;
                    const long long pbase = elem_u0(a, e, NU) / FR_NV;
                    for (int z = threadIdx.x; z < NU; z += NTH) {
                        const int k = z / NT_, t = z % NT_;
                        float sh = 0.0f, c = 0.0f;   // compensated dot product (Dot2)
#pragma unroll
                        for (int j = 0; j < NT_; j++) {
                            dot2ff_next(ffop(o, o.hi.Dhx[t][j]), s_mf[j + 10 * k], sh, c);
                            dot2ff_next(ffop(o, o.hi.Dhy[t][j]), s_mf[NU + j + 10 * k], sh, c);
                        }
#pragma unroll
                        for (int j = 0; j < NZ; j++) dot2ff_next(ffop(o, o.hi.Dhz[k][j]), s_mf[2 * NU + t + 10 * j], sh, c);
                        a.RL[pbase + z] = two_sum(sh, c);
                    }
                }
            }
        };
        if constexpr (TCM == 0) mass_channel();
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
        // viscous normal flux at own flux points, on the side whose LDG weight 1/2 +- beta is not
        // zero (the other side's is never used); the points are compacted so whole warps work
        // (the tensor-core forms run it while the interpolation's MMA chain is in flight)
        auto viscous_faces = [&]() {
            for (int s = threadIdx.x; s < NF; s += NTH) {
                const bool isL = (a.partner[gf0 + s] & FR_LFLAG) != 0;
                const T wgt = isL ? T(0.5) + ph.beta : T(0.5) - ph.beta;
                if (wgt == T(0)) {
#pragma unroll
                    for (int k = 0; k < 4; k++) a.FV[k * a.nfpt + gf0 + s] = T(0);
                } else {
                    s_plist[atomicAdd(&s_pcnt, 1)] = (short)s;
                }
            }
            __syncthreads();
            const int nplist = s_pcnt;
            for (int li = threadIdx.x; li < nplist; li += NTH) {
                const int s = s_plist[li];
                T uf[5], qf[5][3];
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    uf[alpha] = face_value(op, s_u + alpha * NU, s);
#pragma unroll
                    for (int d = 0; d < 3; d++) qf[alpha][d] = face_value(op, s_q + (alpha * 3 + d) * NU, s);
                }
                const T *nt = a.fnrm + (e * 6 + face_of(s)) * 4;
                T n[3] = {nt[0], nt[1], nt[2]};
                if (dev) { uf[0] += ph.rref; uf[4] += ph.eref; }
                T fvn[4];
                viscous_normal_flux(ph, uf, qf, n, fvn);
#pragma unroll
                for (int k = 0; k < 4; k++) a.FV[k * a.nfpt + gf0 + s] = fvn[k];
            }
        };
        if constexpr (TCM == 0) viscous_faces();
        if constexpr (TCM == 0 && sizeof(T) == 4) {
            pri_interp_all_c<NTH>(s_u, s_t, s_w);   // s_q follows s_u
        } else if constexpr (TCM == 0) {
            pri_interp_5<T, NTH>(op, s_u, s_t, s_w);
#pragma unroll 1
            for (int c = 0; c < 3; c++) pri_interp_5<T, NTH>(op, s_q + 5 * c * NU, s_t, s_w + (5 + 5 * c) * NQ);
        } else {
            // z first (CUDA cores): row r = 5 f + c holds field f (s_q follows s_u) at z level c on
            // the 10 triangle points; then the triangle interpolation of all 100 rows on the tensor core.
            const int r = threadIdx.x;
            if (r < TC_ROWS_I) {
                const int f = r / MZ, c = r % MZ;
                const T *src = s_u + f * NU;
                float x[NT_], mx = 0.f;
#pragma unroll
                for (int t = 0; t < NT_; t++) {
                    float v = 0.f;
#pragma unroll
                    for (int k = 0; k < NZ; k++) v += (float)op.Bz[c][k] * (float)src[t + 10 * k];
                    x[t] = v;
                    mx = fmaxf(mx, fabsf(v));
                }
                const int sh = tc::row_shift(mx);
                const float sc = tc::pow2f(sh);
#pragma unroll
                for (int t = 0; t < NT_; t++) x[t] *= sc;
                tc::store_split_parts<TCM, PT::KI, NT_>(tA, r, x);
                s_sh[r] = sh;
            }
            tc::mma_issue<PT::KI / 16>(tmem, tA, PT::SBO_I, tBi, PT::SBO_I, PT::IDESC_I, mbar);
            viscous_faces();   // CUDA-core work while the chain runs (touches no operand tile)
            if (!tc::mma_wait(mbar, parity, tc::first_limit(first_wait, a.dbg_wait0))) {
                tc_fail = true;
                break;
            }
            {
                float v0[16], v1[16];
                const uint32_t ta = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16);
                tc::ld16(ta, v0);
                tc::ld16(ta + 16, v1);
                if (r < TC_ROWS_I) {
                    const float isc = tc::pow2f(-s_sh[r]);
                    T *dst = s_w + NQT * r;                    // field f, level c: f NQ + 25 c = 25 r
#pragma unroll
                    for (int q = 0; q < 16; q++) dst[q] = (T)(v0[q] * isc);
#pragma unroll
                    for (int q = 16; q < NQT; q++) dst[q] = (T)(v1[q - 16] * isc);
                }
            }
            __syncthreads();
        }
        bool ok = true;
        for (int q = threadIdx.x; q < NQ; q += NTH) {          // tdisf
            T u[5], gq[5][3], f[3][5];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                u[alpha] = s_w[alpha * NQ + q];
#pragma unroll
                for (int d = 0; d < 3; d++) gq[alpha][d] = s_w[(5 + alpha * 3 + d) * NQ + q];
            }
            if constexpr (sizeof(T) == 4) {
                if (dev) ok &= total_flux_dev(ph, u, gq, f);
                else ok &= total_flux(ph, u, gq, f);
            } else {
                ok &= total_flux(ph, u, gq, f);
            }
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++)
#pragma unroll
                for (int d = 0; d < 3; d++)
                    s_w[(alpha * 3 + d) * NQ + q] = g.det * (g.Ji[3 * d] * f[0][alpha] + g.Ji[3 * d + 1] * f[1][alpha] + g.Ji[3 * d + 2] * f[2][alpha]);
        }
        flag_status(a.status, ok);
        __syncthreads();
        if constexpr (TCM == 0 && sizeof(T) == 4) {
            pri_project_all_c<NTH>(s_w, s_t, s_q);
        } else if constexpr (TCM == 0) {
#pragma unroll 1
            for (int c = 0; c < 3; c++) pri_project_5<T, NTH>(op, s_w + 5 * c * NQ, s_t, s_q + 5 * c * NU);
        } else {
            // triangle projection of the 75 rows (flux component f, quadrature level c) on the tensor
            // core, then z (CUDA cores)
            const int r = threadIdx.x;
            if (r < TC_ROWS_P) {
                const T *src = s_w + NQT * r;
                float x[NQT], mx = 0.f;
#pragma unroll
                for (int q = 0; q < NQT; q++) { x[q] = (float)src[q]; mx = fmaxf(mx, fabsf(x[q])); }
                const int sh = tc::row_shift(mx);
                const float sc = tc::pow2f(sh);
#pragma unroll
                for (int q = 0; q < NQT; q++) x[q] *= sc;
                tc::store_split_parts<TCM, PT::KP, NQT>(tA, r, x);
                s_sh[r] = sh;
            }
            tc::mma_issue<PT::KP / 16>(tmem, tA, PT::SBO_P, tBp, PT::SBO_P, PT::IDESC_P, mbar);
            // CUDA-core work while the chain runs: it reads the state and writes only static shared
            // memory and global memory, which the chain's rows (they run on past the operand tile
            // into the dynamic shared arrays) never reach
            mass_channel();
            if (!tc::mma_wait(mbar, parity, tc::first_limit(first_wait, a.dbg_wait0))) {
                tc_fail = true;
                break;
            }
            {
                float v0[16];
                tc::ld16(tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16), v0);
                if (r < TC_ROWS_P) {
                    const float isc = tc::pow2f(-s_sh[r]);
#pragma unroll
                    for (int t = 0; t < NT_; t++) s_t[TC_ST * r + t] = (T)(v0[t] * isc);
                }
            }
            __syncthreads();
            for (int it = threadIdx.x; it < 15 * NU; it += NTH) {
                const int f = it / NU, rr = it % NU, k = rr / NT_, t = rr % NT_;
                T v = T(0);
#pragma unroll
                for (int c = 0; c < MZ; c++) v += op.Pz[k][c] * s_t[TC_ST * (MZ * f + c) + t];
                s_q[f * NU + t + 10 * k] = v;
            }
            __syncthreads();
        }
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
    if constexpr (TCM != 0) {
        // a chain that did not complete within the bound is reported; the tensor memory is released
        if (tc_fail && threadIdx.x == 0) atomicOr(a.status, 2);
        tc::teardown(mbar, parity, tc_fail, tmem, 32);
    }
}


// -------------------------------------------------------------------------------------------------
// Phase C: interface group
// -------------------------------------------------------------------------------------------------
template <typename T, int NTH>
__device__ __forceinline__ void pri_C_body(const HexArgs<T> &a, const PriOps<T> *gops, const PriOpsFF *opsff, long long first, long long stride)
{
    __shared__ PriOps<T> op;
    __shared__ T s_d[5 * NF];
    __shared__ ff s_dff[sizeof(T) == 4 ? NF : 1];   // low-Mach form: transformed mass flux (float-float)
    load_ops<T, NTH>(gops, op);
    __syncthreads();
    for (long long e = first; e < a.ne; e += stride) {
        if (!fr_elem_ok(a, e, NU, NF)) continue;
        const Geo<T> g = a.geo[e];
        const Phys<T> ph = elem_phys(a, e);
        const long long gf0 = elem_f0(a, e, NF);
        bool dev = false;
        if constexpr (sizeof(T) == 4) dev = ph.dev != 0;
        bool ok = true;
        for (int s = threadIdx.x; s < NF; s += NTH) {
            const uint32_t pc = a.partner[gf0 + s];
            const bool isL = (pc & FR_LFLAG) != 0;
            const long long og = gf0 + s, pg = fr_partner(a, pc, og);
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
            if constexpr (sizeof(T) == 4) {
                if (dev) {
                    float sw;
                    ok &= isL ? common_flux_dev(ph, uo, up, fvo, fvp, nL, F, sw) : common_flux_dev(ph, up, uo, fvp, fvo, nL, F, sw);
                    // mass flux in float-float: 1/2 (mL - mR) + (s/2 + tau)(rho_L - rho_R),
                    // mX = own-normal n.(rho v)
                    const ff mo = a.MF[og], mp = a.MF[pg];
                    const ff mL = isL ? mo : mp, mR = isL ? mp : mo;
                    const float rL = isL ? uo[0] : up[0], rR = isL ? up[0] : uo[0];
                    const ff Fr = ff_add(ff_mul_f(ff_sub(mL, mR), 0.5f), ff_mul_f(two_sum(rL, -rR), 0.5f * sw + ph.tau));
                    const ff magf = a.fnrm64[(e * 6 + face_of(s)) * 4 + 3];
                    s_dff[s] = isL ? ff_mul(magf, Fr) : ff_neg(ff_mul(magf, Fr));
                } else {
                    ok &= isL ? common_flux(ph, uo, up, fvo, fvp, nL, F) : common_flux(ph, up, uo, fvp, fvo, nL, F);
                }
            } else {
                ok &= isL ? common_flux(ph, uo, up, fvo, fvp, nL, F) : common_flux(ph, up, uo, fvp, fvo, nL, F);
            }
            const T sc = isL ? mag : -mag;
#pragma unroll
            for (int k = 0; k < 5; k++) s_d[k * NF + s] = sc * F[k];
        }
        flag_status(a.status, ok);
        __syncthreads();
        T *R = a.R + elem_u0(a, e, NU);
        const T idet = g.nidet;
        if (!dev) {
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
        } else if constexpr (sizeof(T) == 4) {
            // low-Mach form: R_rho in float-float, R_E = R_(E - H0 rho) + H0 R_rho
            const PriOpsFF &o = *opsff;
            const ff idet64 = a.geo64[e].idet;
            const ff H0 = ph.H0ff;
            const long long pbase = elem_u0(a, e, NU) / FR_NV;
            for (int z = threadIdx.x; z < NU; z += NTH) {
                const int k = z / NT_, t = z % NT_;
                ff r = a.RL[pbase + z];
                r = ff_fma(ffop(o, o.hi.liftzL[k]), s_dff[t], r);
                r = ff_fma(ffop(o, o.hi.liftzR[k]), s_dff[10 + t], r);
#pragma unroll
                for (int f = 0; f < 3; f++)
#pragma unroll
                    for (int b = 0; b < NZ; b++) r = ff_fma(ffop(o, o.hi.Lf[f][t][b]), s_dff[20 + 16 * f + b + 4 * k], r);
                const ff Rrho = ff_mul(r, idet64);
                float out[5];
                out[0] = Rrho.hi + Rrho.lo;
#pragma unroll
                for (int alpha = 1; alpha < 5; alpha++) {
                    const T *D = s_d + alpha * NF;
                    T v = R[alpha * NU + z] + op.liftzL[k] * D[t] + op.liftzR[k] * D[10 + t];
#pragma unroll
                    for (int f = 0; f < 3; f++)
#pragma unroll
                        for (int b = 0; b < NZ; b++) v += op.Lf[f][t][b] * D[20 + 16 * f + b + 4 * k];
                    out[alpha] = v * idet;
                }
                const ff e4 = ff_fma(H0, Rrho, ff_of(out[4]));
                out[4] = e4.hi + e4.lo;
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    if (a.rkstage == 0) R[alpha * NU + z] = out[alpha];
                    else rk_fold(a, elem_u0(a, e, NU) + alpha * NU + z, out[alpha]);
                }
            }
        }
        __syncthreads();
    }
}


}  // namespace
}  // namespace pri
