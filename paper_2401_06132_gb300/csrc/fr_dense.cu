// fr_dense.cu -- kernels of the anti-aliased Navier-Stokes FR right-hand side for element types
// without tensor-product structure (p = 3): tetrahedra and pyramids.
//
// Sum factorisation (Sec. 4) serves hexahedra and prisms only; for tetrahedra and pyramids (Sec. 1)
// every operator is a dense matrix applied per element: NU solution points (20 / 30), NF flux points
// on NFACE faces (4 x 10 / a 16-point base and 4 x 10), 125 quadrature points. Same three fused
// phases as the other types: A face solution, B volume group, C interface group. The volume group
// evaluates, per element, the con_u average, the corrected gradient (Dh_d u plus the face lift of the
// common solution, then J^-T), the own-normal viscous flux at the flux points whose LDG weight is not
// zero, the interpolation of the 20 fields (u and its gradient) to the quadrature points, the
// pointwise flux and its transformation det J J^-1 f, and the L2 projection with the corrected
// divergence folded in (R~ = sum_d (Dh_d Pj) f~_d: one dense NU x 125 operator per direction).
//
// The operator tables (DenseOps: 100 KB / 160 KB in FP64) stay in global memory, read through the
// L1/L2 caches; they are stored with the output index fastest, so that a warp's lanes, which compute
// consecutive outputs, read consecutive entries while the field values they multiply are one
// shared-memory broadcast per warp (16-byte vector loads along the solution-point index, whose rows
// are padded to NUS with zero operator rows).
#include <cuda_runtime.h>

#include "fr_internal.h"
#include "fr_physics.cuh"
#include "fr_tcgen05.cuh"

namespace {

constexpr int NQ = FR_TQ, NQP = FR_TQP;

// Tensor-core interpolation of the mixed forms: D[q][f] = sum_j B[q][j] x_f[j] for the 20 fields
// (state and gradient) of one element, M = 128 quadrature-point rows (125 used), N = 32 field rows
// (20 used), K = the split form's NU-wide slices (tc::SplitForm; FP16: [B_hi | B_hi | B_lo] against
// [x_hi | x_lo | x_hi]; BF16: six slices of three parts), zero-padded to a multiple of 16. The
// operator tile is split once per CTA; each element writes its 20 field rows (scaled by a power of
// two per row) and reads its quadrature point's 20 values back from tensor memory, one lane per
// thread.
template <typename OPS, int TCM>
struct DenseTC {
    static constexpr int KI = tc::split_k<TCM>(OPS::NU);       // FP16: 64 (tetrahedron), 96 (pyramid)
    static constexpr int SBO = KI / 8 * 128;
    static constexpr int A_BYTES = 16 * SBO;                   // 128 rows
    static constexpr int B_BYTES = 4 * SBO;                    // 32 rows
    static constexpr int HEAD = A_BYTES + B_BYTES + 32 * 4 + 16;   // tiles, row shifts, barrier, TMEM slot
    static constexpr int BYTES = HEAD + 128;                   // + alignment slack
    static constexpr uint32_t IDESC = tc::idesc_f16(TCM - 1, 128, 32);
};

// 16 bytes of T (4 floats or 2 doubles): one vector shared-memory load
template <typename T>
struct alignas(16) V16 {
    static constexpr int n = 16 / sizeof(T);
    T v[n];
};
template <typename T>
__device__ __forceinline__ V16<T> ld16(const T *p)
{
    return *reinterpret_cast<const V16<T> *>(p);
}

// The float-float table type of an operator table, and one entry of it as a pair (the lo part sits
// at the same offset in the second table).
template <typename OPS>
using FFOf = DenseOpsFF<DenseOps<float, OPS::NU, OPS::NF, OPS::NFACE>>;
template <typename FF>
__device__ __forceinline__ ff ffat(const FF &o, const float &hi)
{
    const float *h0 = reinterpret_cast<const float *>(&o.hi);
    return ff{hi, reinterpret_cast<const float *>(&o.lo)[&hi - h0]};
}

// -------------------------------------------------------------------------------------------------
// Phase A: disu (U^f = M0 U)
// -------------------------------------------------------------------------------------------------
// EPB elements per CTA iteration, one thread per (element, flux point). The states of the EPB
// elements are staged in shared memory with coalesced loads; each thread keeps its column of M0 in
// registers for the whole persistent loop and reads the state with 16-byte broadcast loads.
// The reduced precisions evaluate every face value as a compensated dot product (Dot2 of Ogita, Rump
// and Oishi) of the float-float M0 row (hi + lo) with the FP32 state, rounded once: at low Mach the
// Rusanov dissipation (1/2)(|v.n| + c)(u_L - u_R), c about 10 |v|, lifts any rounding of a face
// value into R. Low-Mach FP32 form (ph.dev): the face solution of the deviations from the reference
// state, and the own-normal mass flux n.(rho v) at every flux point in float-float: first
// m_f = n_f . (rho v) at the solution points per face (the face normal is constant on an affine
// element), then the same compensated dot product with m_f.
// FP32 pyramids (224 threads per CTA): registers capped for five CTAs per SM, up from two at the
// compiler's 112 (a few spilled values; the tetrahedral form is faster uncapped). Otherwise (0) the
// compiler's own register count.
template <typename T, typename OPS, int EPB>
__global__ void __launch_bounds__(OPS::NF * EPB, (sizeof(T) == 4 && OPS::NF * EPB > 192) ? 1280 / (OPS::NF * EPB) : 0)
k_dense_disu(HexArgs<T> a, const OPS *__restrict__ op, const FFOf<OPS> *__restrict__ opsff)
{
    constexpr int NU = OPS::NU, NF = OPS::NF, NUS = OPS::NUS, NFACE = OPS::NFACE, NTH = NF * EPB;
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int VN = V16<T>::n;
    __shared__ __align__(16) T s_u[EPB][FR_NV * NUS];
    __shared__ __align__(16) ff s_m[F32 ? EPB : 1][F32 ? NFACE * NUS : 1];
    const int el = threadIdx.x / NF, s = threadIdx.x % NF;
    T col[NUS];
#pragma unroll
    for (int z = 0; z < NUS; z++) col[z] = op->M0t[z][s];   // pad rows are zero
    float col_lo[F32 ? NUS : 1];                              // lo parts of the FP32 column
    if constexpr (F32) {
#pragma unroll
        for (int z = 0; z < NUS; z++) col_lo[z] = opsff->lo.M0t[z][s];
    }
    if constexpr (NUS > NU) {
        for (int i = threadIdx.x; i < EPB * FR_NV * (NUS - NU); i += NTH) {
            const int l = i / (FR_NV * (NUS - NU)), r = i % (FR_NV * (NUS - NU));
            s_u[l][(r / (NUS - NU)) * NUS + NU + r % (NUS - NU)] = T(0);
        }
    }
    const long long ng = (a.ne + EPB - 1) / EPB;
    for (long long g = blockIdx.x; g < ng; g += gridDim.x) {
        const long long e0 = g * EPB;
        const int nel = (int)(a.ne - e0 < EPB ? a.ne - e0 : EPB);
        {
            bool blk_ok = true;
            for (int k = 0; k < nel; k++) blk_ok = blk_ok && fr_elem_ok(a, e0 + k, NU, NF);
            if (!blk_ok) continue;
        }
        for (int i = threadIdx.x; i < nel * FR_NV * NU; i += NTH) {
            const int l = i / (FR_NV * NU), r = i % (FR_NV * NU), alpha = r / NU;
            const long long e = e0 + l;
            T v = a.U[elem_u0(a, e, NU) + r];
            if constexpr (F32) {
                const Phys<T> ph = elem_phys(a, e);
                if (ph.dev) v -= alpha == 0 ? ph.rref : (alpha == 4 ? ph.eref : T(0));
            }
            s_u[l][alpha * NUS + r % NU] = v;
        }
        if constexpr (F32) {
            __syncthreads();
            for (int i = threadIdx.x; i < nel * NFACE * NU; i += NTH) {
                const int l = i / (NFACE * NU), r = i % (NFACE * NU), f = r / NU, z = r % NU;
                const long long e = e0 + l;
                if (!elem_phys(a, e).dev) continue;
                const ff *nt = a.fnrm64 + (e * 6 + f) * 4;
                const float *u = s_u[l];
                ff m = ff_mul_f(nt[0], u[NUS + z]);
                m = ff_add(m, ff_mul_f(nt[1], u[2 * NUS + z]));
                s_m[l][f * NUS + z] = ff_add(m, ff_mul_f(nt[2], u[3 * NUS + z]));
            }
        }
        __syncthreads();
        if (el < nel) {
            const long long e = e0 + el;
            const long long f0 = elem_f0(a, e, NF);
            const T *u = s_u[el];
            if constexpr (F32) {
                // sh + c = sum_z (col + col_lo)[z] x[z]: exact products (one FMA each), TwoSum
                // accumulation of the high parts, the errors summed in c
                float sh[FR_NV], c[FR_NV];
#pragma unroll
                for (int alpha = 0; alpha < FR_NV; alpha++) { sh[alpha] = 0.0f; c[alpha] = 0.0f; }
#pragma unroll
                for (int z = 0; z < NUS; z += VN) {
#pragma unroll
                    for (int alpha = 0; alpha < FR_NV; alpha++) {
                        const V16<T> x = ld16(u + alpha * NUS + z);
#pragma unroll
                        for (int j = 0; j < VN; j++) {
                            const float pr = col[z + j] * x.v[j];
                            const float er = __fmaf_rn(col_lo[z + j], x.v[j], __fmaf_rn(col[z + j], x.v[j], -pr));
                            const ff t = two_sum(sh[alpha], pr);
                            sh[alpha] = t.hi;
                            c[alpha] += t.lo + er;
                        }
                    }
                }
#pragma unroll
                for (int alpha = 0; alpha < FR_NV; alpha++) a.UF[alpha * a.nfpt + f0 + s] = sh[alpha] + c[alpha];
            } else {
                T v[FR_NV];
#pragma unroll
                for (int alpha = 0; alpha < FR_NV; alpha++) v[alpha] = T(0);
#pragma unroll
                for (int z = 0; z < NUS; z += VN) {
#pragma unroll
                    for (int alpha = 0; alpha < FR_NV; alpha++) {
                        const V16<T> x = ld16(u + alpha * NUS + z);
#pragma unroll
                        for (int j = 0; j < VN; j++) v[alpha] += col[z + j] * x.v[j];
                    }
                }
#pragma unroll
                for (int alpha = 0; alpha < FR_NV; alpha++) a.UF[alpha * a.nfpt + f0 + s] = v[alpha];
            }
            if constexpr (F32) {
                if (elem_phys(a, e).dev) {
                    const ff *m = s_m[el] + OPS::FACE(s) * NUS;
                    float sh = 0.0f, c = 0.0f;
#pragma unroll
                    for (int z = 0; z < NU; z++) {
                        const ff mz = m[z];
                        const float pr = col[z] * mz.hi;
                        const float er = __fmaf_rn(opsff->lo.M0t[z][s], mz.hi, __fmaf_rn(col[z], mz.lo, __fmaf_rn(col[z], mz.hi, -pr)));
                        const ff t = two_sum(sh, pr);
                        sh = t.hi;
                        c += t.lo + er;
                    }
                    a.MF[f0 + s] = two_sum(sh, c);
                }
            }
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------------------------------------
// Phase B: volume group, one element per CTA of NTH threads (persistent over elements)
// -------------------------------------------------------------------------------------------------
template <typename T, int NTH, typename OPS, int TCM>
__global__ void __launch_bounds__(NTH, sizeof(T) == 4 ? (TCM == 0 ? 8 : 6) : 0) k_dense_B(HexArgs<T> a, const OPS *__restrict__ op, const FFOf<OPS> *__restrict__ opsff)
{
    constexpr int NU = OPS::NU, NF = OPS::NF, NFACE = OPS::NFACE, NUS = OPS::NUS;
    static_assert(NTH >= NQ, "one thread per quadrature point");
    static_assert(TCM == 0 || (NTH == 128 && sizeof(T) == 4), "tensor-core form: FP32, one warpgroup per element");
    using TC = DenseTC<OPS, TCM == 0 ? 1 : TCM>;
    using SF = tc::SplitForm<TCM == 0 ? 1 : TCM>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ short s_plist[NF];
    __shared__ int s_pcnt;
    __shared__ __align__(8) double s_mfb[sizeof(T) == 4 ? 3 * NU : 1];   // low-Mach form: transformed mass flux
    __shared__ __align__(8) double s_rlb[sizeof(T) == 4 ? 3 * NU : 1];   // low-Mach form: Dh_d of it, per d
    constexpr int VW = V16<T>::n;
    constexpr int NCH = NTH / NU;                 // quadrature-point chunks of the projection
    unsigned char *arr = smem_raw;
    // tensor-core state (TCM != 0): operator tile, field tile, row shifts, barrier, TMEM address
    unsigned char *tA = nullptr, *tB = nullptr;
    int *s_sh = nullptr;
    uint64_t *mbar = nullptr;
    uint32_t *s_tmem = nullptr, tmem = 0, parity = 0;
    bool tc_fail = false, first_wait = true;
    if constexpr (TCM != 0) {
        const uint32_t raw = tc::smem_u32(arr);
        tA = arr + ((128 - (raw & 127)) & 127);
        tB = tA + TC::A_BYTES;
        s_sh = reinterpret_cast<int *>(tB + TC::B_BYTES);
        mbar = reinterpret_cast<uint64_t *>(s_sh + 32);
        s_tmem = reinterpret_cast<uint32_t *>(mbar + 1);
        arr = tA + TC::HEAD;
        tc::setup(mbar, s_tmem, 32);
        for (int i = threadIdx.x; i < 128 * TC::KI; i += NTH) {   // the split form's slices of B, rows q
            const int n = i / TC::KI, k = i % TC::KI, sg = k / NU;
            uint16_t pp[3] = {0, 0, 0};
            if (n < NQ && sg < SF::SEGS) tc::split_parts<TCM>((float)op->Bt[k % NU][n], pp);
            *reinterpret_cast<uint16_t *>(tA + tc::core_offset(n, k, TC::SBO)) = sg < SF::SEGS ? pp[SF::y_part(sg)] : (uint16_t)0;
        }
        for (int i = threadIdx.x; i < 32 * TC::KI; i += NTH)     // field rows 20..31 and the K pad stay zero
            *reinterpret_cast<uint16_t *>(tB + tc::core_offset(i / TC::KI, i % TC::KI, TC::SBO)) = 0;
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tmem = *s_tmem;
    }
    T *s_u = reinterpret_cast<T *>(arr);        // [5][NUS] state
    T *s_q = s_u + 5 * NUS;                       // [15][NUS] physical gradient (field 5 + 3 alpha + d of s_u)
    T *s_c = s_q + 15 * NUS;                      // [5][NF] common solution
    T *s_w = s_c + 5 * NF;                        // [20][NQP] fields at quadrature points, then f~
    T *s_red = s_w + 15 * NQP;                    // [NCH][5][NU] projection partial sums (fields 15-19 are dead by then)
    static_assert(NCH * 5 * NU <= 5 * NQP, "partial sums fit in the dead quadrature-point rows");
    static_assert(NUS % VW == 0 && (NUS * sizeof(T)) % 16 == 0 && (NQP * sizeof(T)) % 16 == 0 && (NF * sizeof(T)) % 16 == 0,
                  "16-byte rows");
    // pads that meet zero operator rows in the vector loads stay zero: s_w columns NQ.. and the
    // solution-point columns NU.. of the 20 fields
    for (int it = threadIdx.x; it < 20 * (NQP - NQ); it += NTH) s_w[(it / (NQP - NQ)) * NQP + NQ + it % (NQP - NQ)] = T(0);
    if constexpr (NUS > NU)
        for (int it = threadIdx.x; it < 20 * (NUS - NU); it += NTH) s_u[(it / (NUS - NU)) * NUS + NU + it % (NUS - NU)] = T(0);
    for (long long e = blockIdx.x; e < a.ne; e += gridDim.x) {
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
            s_u[(it / NU) * NUS + it % NU] = v;
        }
        if constexpr (sizeof(T) == 4) {
            // low-Mach form: the volume part of R~_rho, sum_d Dh_d (det J J^-1 rho v)_d, in about 48
            // bits or better (rho v lies in the solution space, so its L2 projection is itself and
            // the corrected divergence Dh applies at the solution points). First the transformed
            // mass flux (read from the state in global memory, so that it is ready at the first
            // barrier); the 3 NU products Dh_d m_d then ride along with the gradient items below.
            // The dense product costs 3 NU^2 multiply-adds per element: on the tetrahedron (NU = 20)
            // the FP64 pipe, idle in this kernel, does them faster than float-float arithmetic on
            // the busy FP32 pipe; on the pyramid (NU = 30) the FP64 pipe would become the limit, so
            // it stays in float-float.
            if (dev) {
                const GeoLM &g64 = a.geo64[e];
                for (int z = threadIdx.x; z < NU; z += NTH) {
                    const float m0 = U[NU + z], m1 = U[2 * NU + z], m2 = U[3 * NU + z];
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        if constexpr (NU <= 20) {
                            s_mfb[d * NU + z] = g64.det * (g64.Ji[3 * d] * (double)m0 + g64.Ji[3 * d + 1] * (double)m1 + g64.Ji[3 * d + 2] * (double)m2);
                        } else {
                            ff *s_mf = reinterpret_cast<ff *>(s_mfb);
                            s_mf[d * NU + z] = ff_add(ff_add(ff_mul_f(g64.cm[3 * d], m0), ff_mul_f(g64.cm[3 * d + 1], m1)), ff_mul_f(g64.cm[3 * d + 2], m2));
                        }
                    }
                }
            }
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
        // corrected gradient q~_d = Dh_d u + sum_f n_f,d (L_f c), then q = J^-T q~
        const int ngrad = 5 * NU + (dev ? 3 * NU : 0);
        for (int it = threadIdx.x; it < ngrad; it += NTH) {
            if constexpr (sizeof(T) == 4) {
                if (it >= 5 * NU) {   // low-Mach mass channel: (Dh_d m_d)[z]
                    const int d = (it - 5 * NU) / NU, z = (it - 5 * NU) % NU;
                    const FFOf<OPS> &o = *opsff;
                    if constexpr (NU <= 20) {
                        double v = 0.0;
#pragma unroll 5
                        for (int j = 0; j < NU; j++) v += o.Dht64[d][j][z] * s_mfb[d * NU + j];
                        s_rlb[d * NU + z] = v;
                    } else {
                        // compensated dot product (Dot2) of the float-float operator row and m_d
                        const ff *m = reinterpret_cast<const ff *>(s_mfb) + d * NU;
                        float sh = 0.0f, c = 0.0f;
#pragma unroll 5
                        for (int j = 0; j < NU; j++) {
                            const float h = o.hi.Dht[d][j][z], l = o.lo.Dht[d][j][z];
                            const ff mj = m[j];
                            const float pr = h * mj.hi;
                            const float er = __fmaf_rn(l, mj.hi, __fmaf_rn(h, mj.lo, __fmaf_rn(h, mj.hi, -pr)));
                            const ff t = two_sum(sh, pr);
                            sh = t.hi;
                            c += t.lo + er;
                        }
                        reinterpret_cast<ff *>(s_rlb)[d * NU + z] = two_sum(sh, c);
                    }
                    continue;
                }
            }
            const int alpha = it / NU, z = it % NU;
            const T *u = s_u + alpha * NUS;
            const T *c = s_c + alpha * NF;
            T q0 = T(0), q1 = T(0), q2 = T(0);
#pragma unroll 4
            for (int j = 0; j < NU; j++) {
                const T uj = u[j];
                q0 += op->Dht[0][j][z] * uj;
                q1 += op->Dht[1][j][z] * uj;
                q2 += op->Dht[2][j][z] * uj;
            }
#pragma unroll
            for (int f = 0; f < NFACE; f++) {
                T l = T(0);
#pragma unroll
                for (int s = OPS::F0(f); s < OPS::F0(f + 1); s++) l += op->Lt[s][z] * c[s];
                q0 += op->nf[f][0] * l;
                q1 += op->nf[f][1] * l;
                q2 += op->nf[f][2] * l;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) s_q[(alpha * 3 + k) * NUS + z] = g.Ji[k] * q0 + g.Ji[3 + k] * q1 + g.Ji[6 + k] * q2;
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
            if (dev) {
                const long long pbase = elem_u0(a, e, NU) / FR_NV;
                for (int z = threadIdx.x; z < NU; z += NTH) {
                    if constexpr (NU <= 20) {
                        a.RL[pbase + z] = ff_from_double(s_rlb[z] + s_rlb[NU + z] + s_rlb[2 * NU + z]);
                    } else {
                        const ff *r = reinterpret_cast<const ff *>(s_rlb);
                        a.RL[pbase + z] = ff_add(ff_add(r[z], r[NU + z]), r[2 * NU + z]);
                    }
                }
            }
        }
        // viscous normal flux at own flux points, on the side whose LDG weight 1/2 +- beta is not
        // zero (the other side's is never used); the points are compacted so whole warps work
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
        if constexpr (TCM != 0) {
            // the 20 field rows (s_q follows s_u) for the tensor-core interpolation, four threads per
            // row: [x_hi | x_lo | x_hi], scaled by 2^sh so that the row's largest magnitude lies in
            // [2^14, 2^15); the MMA then runs while the viscous flux below is evaluated
            if (threadIdx.x < 96) {   // warps 0-2, whole warps in the shuffles
                const int r = threadIdx.x >> 2, sub = threadIdx.x & 3;
                const bool row = r < 20;
                constexpr int NV = (NU + 3) / 4;
                float x[NV], mx = 0.f;
#pragma unroll
                for (int i = 0; i < NV; i++) {
                    const int j = sub + 4 * i;
                    x[i] = (row && j < NU) ? (float)s_u[r * NUS + j] : 0.f;
                    mx = fmaxf(mx, fabsf(x[i]));
                }
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
                if (row) {
                    const int sh = tc::row_shift(mx);
                    const float sc = tc::pow2f(sh);
#pragma unroll
                    for (int i = 0; i < NV; i++) {
                        const int j = sub + 4 * i;
                        if (j < NU) {
                            uint16_t pp[3];
                            tc::split_parts<TCM>(x[i] * sc, pp);
#pragma unroll
                            for (int sg = 0; sg < SF::SEGS; sg++)
                                *reinterpret_cast<uint16_t *>(tB + tc::core_offset(r, sg * NU + j, TC::SBO)) = pp[SF::x_part(sg)];
                        }
                    }
                    if (sub == 0) s_sh[r] = sh;
                }
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
        }
        __syncthreads();
        if constexpr (TCM != 0) {
            if (threadIdx.x == 0) {
                tc::fence_after_sync();
                const uint32_t aA = tc::smem_u32(tA), aB = tc::smem_u32(tB);
#pragma unroll
                for (int j = 0; j < TC::KI / 16; j++)
                    tc::mma_f16(tmem, tc::sdesc(aA + 256 * j, 128, TC::SBO), tc::sdesc(aB + 256 * j, 128, TC::SBO),
                                TC::IDESC, j);
                tc::commit(mbar);
            }
        }
        const int nplist = s_pcnt;
        for (int li = threadIdx.x; li < nplist; li += NTH) {
            const int s = s_plist[li];
            T v[20];
#pragma unroll
            for (int f = 0; f < 20; f++) v[f] = T(0);
#pragma unroll 1
            for (int z0 = 0; z0 < NUS; z0 += VW) {
                T m[VW];
#pragma unroll
                for (int k = 0; k < VW; k++) m[k] = op->M0t[z0 + k][s];
#pragma unroll
                for (int f = 0; f < 20; f++) {
                    const V16<T> x = ld16(s_u + f * NUS + z0);
#pragma unroll
                    for (int k = 0; k < VW; k++) v[f] += m[k] * x.v[k];
                }
            }
            T uf[5], qf[5][3];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                uf[alpha] = v[alpha];
#pragma unroll
                for (int d = 0; d < 3; d++) qf[alpha][d] = v[5 + alpha * 3 + d];
            }
            const T *nt = a.fnrm + (e * 6 + OPS::FACE(s)) * 4;
            T n[3] = {nt[0], nt[1], nt[2]};
            if (dev) { uf[0] += ph.rref; uf[4] += ph.eref; }
            T fvn[4];
            viscous_normal_flux(ph, uf, qf, n, fvn);
#pragma unroll
            for (int k = 0; k < 4; k++) a.FV[k * a.nfpt + gf0 + s] = fvn[k];
        }
        if constexpr (TCM != 0) {
            // the interpolation issued above: wait (bounded) and read lane q = this thread
            const bool done = tc::mbar_wait(mbar, parity, tc::first_limit(first_wait, a.dbg_wait0));
            if (!__syncthreads_and(done)) {
                tc_fail = true;
                break;
            }
            parity ^= 1;
            tc::fence_after_sync();
            float v0[16], v1[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16);   // lane = quadrature point
            tc::ld16(ta, v0);
            tc::ld16(ta + 16, v1);
            const int q = threadIdx.x;
            if (q < NQ) {
#pragma unroll
                for (int f = 0; f < 16; f++) s_w[f * NQP + q] = v0[f] * tc::pow2f(-s_sh[f]);
#pragma unroll
                for (int f = 16; f < 20; f++) s_w[f * NQP + q] = v1[f - 16] * tc::pow2f(-s_sh[f]);
            }
        } else {
            // interpolation of the 20 fields to the quadrature points: one point per thread
            for (int q = threadIdx.x; q < NQ; q += NTH) {
                T v[20];
#pragma unroll
                for (int f = 0; f < 20; f++) v[f] = T(0);
#pragma unroll 1
                for (int j0 = 0; j0 < NUS; j0 += VW) {
                    T b[VW];
#pragma unroll
                    for (int k = 0; k < VW; k++) b[k] = op->Bt[j0 + k][q];
#pragma unroll
                    for (int f = 0; f < 20; f++) {
                        const V16<T> x = ld16(s_u + f * NUS + j0);
#pragma unroll
                        for (int k = 0; k < VW; k++) v[f] += b[k] * x.v[k];
                    }
                }
#pragma unroll
                for (int f = 0; f < 20; f++) s_w[f * NQP + q] = v[f];
            }
        }
        __syncthreads();
        bool ok = true;
        for (int q = threadIdx.x; q < NQ; q += NTH) {          // tdisf, in place
            T u[5], gq[5][3], f[3][5];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                u[alpha] = s_w[alpha * NQP + q];
#pragma unroll
                for (int d = 0; d < 3; d++) gq[alpha][d] = s_w[(5 + alpha * 3 + d) * NQP + q];
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
                    s_w[(alpha * 3 + d) * NQP + q] = g.det * (g.Ji[3 * d] * f[0][alpha] + g.Ji[3 * d + 1] * f[1][alpha] + g.Ji[3 * d + 2] * f[2][alpha]);
        }
        flag_status(a.status, ok);
        __syncthreads();
        // projection with the corrected divergence: R~[alpha][z] = sum_d sum_q Dv_d[z][q] f~_d[alpha][q].
        // Thread (z, chunk c of the NQP/4 groups of 4 quadrature points) sums all 5 variables over its
        // chunk (one operator load per 5 FMAs, the flux values as 16-byte broadcasts); the NCH
        // partial sums are then added in shared memory.
        if (threadIdx.x < NU * NCH) {
            const int z = threadIdx.x % NU, c = threadIdx.x / NU;
            const int gb = c * (NQP / 4) / NCH, ge = (c + 1) * (NQP / 4) / NCH;
            T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll 1
            for (int d = 0; d < 3; d++)
#pragma unroll 1
                for (int gq4 = gb; gq4 < ge; gq4++) {
                    const int q0 = 4 * gq4;
                    T mv[4];
#pragma unroll
                    for (int k = 0; k < 4; k++) mv[k] = op->Dvt[d][q0 + k][z];
#pragma unroll
                    for (int alpha = 0; alpha < 5; alpha++) {
                        const T *F = s_w + (alpha * 3 + d) * NQP + q0;
#pragma unroll
                        for (int h = 0; h < 4; h += VW) {
                            const V16<T> x = ld16(F + h);
#pragma unroll
                            for (int k = 0; k < VW; k++) acc[alpha] += mv[h + k] * x.v[k];
                        }
                    }
                }
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) s_red[(c * 5 + alpha) * NU + z] = acc[alpha];
        }
        __syncthreads();
        T *R = a.R + elem_u0(a, e, NU);
        for (int it = threadIdx.x; it < 5 * NU; it += NTH) {
            T v = T(0);
#pragma unroll
            for (int c = 0; c < NCH; c++) v += s_red[c * 5 * NU + it];
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
// Phase C: interface group (common flux at every own flux point, lift and scale)
// -------------------------------------------------------------------------------------------------
// FP32: registers capped for 1280 resident threads per SM (eight tetrahedral or five pyramidal CTAs):
// the kernel waits on its partner gathers, and more warps keep more of them in flight.
template <typename T, typename OPS, int EPB>
__global__ void __launch_bounds__(OPS::NF * EPB, sizeof(T) == 4 ? 1280 / (OPS::NF * EPB) : 0) k_dense_C(HexArgs<T> a, const OPS *__restrict__ op, const FFOf<OPS> *__restrict__ opsff)
{
    constexpr int NU = OPS::NU, NF = OPS::NF, NTH = NF * EPB;
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int VN = V16<T>::n;
    static_assert(NF % VN == 0, "flux-point rows are whole 16-byte vectors");
    __shared__ __align__(16) T s_d[EPB][FR_NV * NF];
    __shared__ ff s_dff[F32 ? EPB : 1][F32 ? NF : 1];    // low-Mach form: scaled common mass flux (float-float)
    __shared__ ff s_rr[F32 ? EPB : 1][F32 ? NU : 1];     // low-Mach form: R_rho (float-float)
    __shared__ ff s_idet[F32 ? EPB : 1];                 // low-Mach form: -1 / det J (float-float)
    const int el = threadIdx.x / NF, s = threadIdx.x % NF;
    const long long ng = (a.ne + EPB - 1) / EPB;
    for (long long g = blockIdx.x; g < ng; g += gridDim.x) {
        const long long e0 = g * EPB;
        const int nel = (int)(a.ne - e0 < EPB ? a.ne - e0 : EPB);
        {
            bool blk_ok = true;
            for (int k = 0; k < nel; k++) blk_ok = blk_ok && fr_elem_ok(a, e0 + k, NU, NF);
            if (!blk_ok) continue;
        }
        bool ok = true;
        if (el < nel) {
            const long long e = e0 + el;
            const Phys<T> ph = elem_phys(a, e);
            const long long og = elem_f0(a, e, NF) + s;
            const uint32_t pc = a.partner[og];
            const bool isL = (pc & FR_LFLAG) != 0;
            const long long pg = fr_partner(a, pc, og);
            T uo[5], up[5], fvo[4], fvp[4];
#pragma unroll
            for (int k = 0; k < 5; k++) { uo[k] = a.UF[k * a.nfpt + og]; up[k] = a.UF[k * a.nfpt + pg]; }
#pragma unroll
            for (int k = 0; k < 4; k++) { fvo[k] = a.FV[k * a.nfpt + og]; fvp[k] = a.FV[k * a.nfpt + pg]; }
            const T *nt = a.fnrm + (e * 6 + OPS::FACE(s)) * 4;
            const T mag = nt[3];
            T nL[3] = {isL ? nt[0] : -nt[0], isL ? nt[1] : -nt[1], isL ? nt[2] : -nt[2]};
            T F[5];
            bool dev = false;
            if constexpr (F32) dev = ph.dev != 0;
            if (dev) {
                if constexpr (F32) {
                    float sw;
                    ok = isL ? common_flux_dev(ph, uo, up, fvo, fvp, nL, F, sw) : common_flux_dev(ph, up, uo, fvp, fvo, nL, F, sw);
                    // mass flux in float-float: 1/2 (mL - mR) + (s/2 + tau)(rho_L - rho_R), mX = own-normal n.(rho v)
                    const ff mo = a.MF[og], mp = a.MF[pg];
                    const ff mL = isL ? mo : mp, mR = isL ? mp : mo;
                    const float rL = isL ? uo[0] : up[0], rR = isL ? up[0] : uo[0];
                    const ff Fr = ff_add(ff_mul_f(ff_sub(mL, mR), 0.5f), ff_mul_f(two_sum(rL, -rR), 0.5f * sw + ph.tau));
                    const ff magf = a.fnrm64[(e * 6 + OPS::FACE(s)) * 4 + 3];
                    s_dff[el][s] = isL ? ff_mul(magf, Fr) : ff_neg(ff_mul(magf, Fr));
                    if (s == 0) s_idet[el] = a.geo64[e].idet;
                }
            } else {
                ok = isL ? common_flux(ph, uo, up, fvo, fvp, nL, F) : common_flux(ph, up, uo, fvp, fvo, nL, F);
            }
            const T sc = isL ? mag : -mag;
#pragma unroll
            for (int k = 0; k < 5; k++) s_d[el][k * NF + s] = sc * F[k];
        }
        flag_status(a.status, ok);
        __syncthreads();
        // lift and scale: R += L D, R *= -1/det; the mass rows of low-Mach elements in float-float,
        // then the energy rows, which add H0 R_rho
        for (int pass = 0; pass < 2; pass++) {
            const int nrow = pass == 0 ? 4 : 1;
            for (int i = threadIdx.x; i < nel * nrow * NU; i += NTH) {
                const int l = i / (nrow * NU), alpha = pass == 0 ? (i / NU) % 4 : 4, z = i % NU;
                const long long e = e0 + l;
                const long long ui = elem_u0(a, e, NU) + alpha * NU + z;
                bool dev = false;
                if constexpr (F32) dev = elem_phys(a, e).dev != 0;
                float outf = 0.0f;
                T out;
                if (F32 && dev && alpha == 0) {
                    if constexpr (F32) {
                        const ff r0 = a.RL[elem_u0(a, e, NU) / FR_NV + z];
                        float sh = r0.hi, c = r0.lo;
                        const ff *d = s_dff[l];
#pragma unroll 8
                        for (int s2 = 0; s2 < NF; s2++) {
                            const float lh = op->Lt[s2][z], ll = opsff->lo.Lt[s2][z];
                            const ff ds = d[s2];
                            const float pr = lh * ds.hi;
                            const float er = __fmaf_rn(ll, ds.hi, __fmaf_rn(lh, ds.lo, __fmaf_rn(lh, ds.hi, -pr)));
                            const ff t = two_sum(sh, pr);
                            sh = t.hi;
                            c += t.lo + er;
                        }
                        const ff Rrho = ff_mul(two_sum(sh, c), s_idet[l]);
                        s_rr[l][z] = Rrho;
                        outf = Rrho.hi + Rrho.lo;
                    }
                    out = (T)outf;
                } else {
                    const T *D = s_d[l] + alpha * NF;
                    T v = a.R[ui];
#pragma unroll 2
                    for (int s2 = 0; s2 < NF; s2 += VN) {
                        const V16<T> x = ld16(D + s2);
#pragma unroll
                        for (int j = 0; j < VN; j++) v += op->Lt[s2 + j][z] * x.v[j];
                    }
                    out = v * a.geo[e].nidet;
                    if constexpr (F32) {
                        if (dev && alpha == 4) {
                            const ff e4 = ff_fma(elem_phys(a, e).H0ff, s_rr[l][z], ff_of(out));
                            out = e4.hi + e4.lo;
                        }
                    }
                }
                if (a.rkstage == 0) a.R[ui] = out;
                else rk_fold(a, ui, out);
            }
            if (F32 && pass == 0) __syncthreads();
        }
        __syncthreads();
    }
}

// persistent grid over groups of epb elements: at most per_sm CTAs per SM, 8 waves
int grid_groups(long long ne, int epb, int per_sm)
{
    long long g = (ne + epb - 1) / epb;
    if (g > fr_sms() * per_sm * 8) g = fr_sms() * per_sm * 8;
    return (int)(g < 1 ? 1 : g);
}

int grid_elems(long long ne, int per_sm)
{
    long long g = ne;
    if (g > fr_sms() * per_sm * 8) g = fr_sms() * per_sm * 8;
    return (int)(g < 1 ? 1 : g);
}

template <typename T, typename OPS>
int dense_phase(int phase, const HexArgs<T> &a, const OPS *ops, const FFOf<OPS> *opsff, cudaStream_t s)
{
    constexpr int NU = OPS::NU, NF = OPS::NF, NUS = OPS::NUS;
    if (a.ne == 0) return 0;
    if (phase == 0) {
        k_dense_disu<T, OPS, 4><<<grid_groups(a.ne, 4, 8), NF * 4, 0, s>>>(a, ops, opsff);
    } else if (phase == 1) {
        constexpr int NTH = 128;
        const size_t base = (size_t)(20 * NUS + 5 * NF + 20 * NQP) * sizeof(T);
        bool tcdone = false;
        if constexpr (sizeof(T) == 4) {
            if (a.tcmode != 0) {
                tcdone = true;
                const size_t smem = base + (a.tcmode == 1 ? DenseTC<OPS, 1>::BYTES : DenseTC<OPS, 2>::BYTES);
                // persistent: as many CTAs as fit on the SMs (shared memory, registers, and the 512
                // tensor-memory columns at 32 per CTA)
                auto kern = a.tcmode == 1 ? k_dense_B<T, NTH, OPS, 1> : k_dense_B<T, NTH, OPS, 2>;
                static int occ[3] = {-1, -1, -1};
                int &o = occ[a.tcmode];
                if (o < 0) {
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    cudaFuncAttributes fa{};
                    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return -1;
                    const int by_smem = (int)(232448 / (smem + fa.sharedSizeBytes + 1024));
                    const int by_regs = 65536 / (((fa.numRegs + 7) / 8 * 8) * NTH);
                    int v = by_smem < by_regs ? by_smem : by_regs;
                    if (v > 512 / 32) v = 512 / 32;
                    if (v < 1) return -4;
                    o = v;
                }
                const long long g = a.ne < fr_sms() * o ? a.ne : fr_sms() * o;
                kern<<<(int)g, NTH, smem, s>>>(a, ops, opsff);
            }
        }
        if (!tcdone) {
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_dense_B<T, NTH, OPS, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base);
                attr = true;
            }
            k_dense_B<T, NTH, OPS, 0><<<grid_elems(a.ne, 8), NTH, base, s>>>(a, ops, opsff);
        }
    } else {
        k_dense_C<T, OPS, 4><<<grid_groups(a.ne, 4, 8), NF * 4, 0, s>>>(a, ops, opsff);
    }
    (void)NU;
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

template <typename T>
int tet_fused_phase(int phase, const HexArgs<T> &a, const TetOps<T> *ops, const DenseOpsFF<TetOps<float>> *opsff, cudaStream_t s)
{
    return dense_phase<T, TetOps<T>>(phase, a, ops, opsff, s);
}

template <typename T>
int pyr_fused_phase(int phase, const HexArgs<T> &a, const PyrOps<T> *ops, const DenseOpsFF<PyrOps<float>> *opsff, cudaStream_t s)
{
    return dense_phase<T, PyrOps<T>>(phase, a, ops, opsff, s);
}

template int tet_fused_phase<double>(int, const HexArgs<double> &, const TetOps<double> *, const DenseOpsFF<TetOps<float>> *, cudaStream_t);
template int tet_fused_phase<float>(int, const HexArgs<float> &, const TetOps<float> *, const DenseOpsFF<TetOps<float>> *, cudaStream_t);
template int pyr_fused_phase<double>(int, const HexArgs<double> &, const PyrOps<double> *, const DenseOpsFF<PyrOps<float>> *, cudaStream_t);
template int pyr_fused_phase<float>(int, const HexArgs<float> &, const PyrOps<float> *, const DenseOpsFF<PyrOps<float>> *, cudaStream_t);
