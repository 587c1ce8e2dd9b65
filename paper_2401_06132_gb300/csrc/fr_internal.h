// fr_internal.h -- internal types of the GB300 flux-reconstruction library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/fr_gb300.h"
#include "fr_ff.cuh"

#define FR_NV 5
#define FR_MAXN 6          // max 1D solution points (p <= 5)
#define FR_MAXM 7          // max 1D quadrature points
#define FR_LFLAG 0x80000000u

// ---------------------------------------------------------------------------------------------
// Host-side basis construction (fr_basis.cpp)
// ---------------------------------------------------------------------------------------------
namespace frb {

// Gauss-Legendre nodes (ascending) and weights on [-1,1], from the eigen-decomposition of the
// Jacobi matrix of the Legendre recurrence (Golub-Welsch).
void gauss_legendre(int n, double *x, double *w);

// 1D operators of a hex element of order p with m quadrature points per direction.
struct Hex1D {
    int n, m;
    double x[FR_MAXN], w[FR_MAXN];          // solution points / GL weights
    double xq[FR_MAXM], wq[FR_MAXM];        // quadrature points / weights
    double B[FR_MAXM][FR_MAXN];             // interpolation solution -> quadrature: l_i(xq_a)
    double Pj[FR_MAXN][FR_MAXM];            // L2 projection quadrature -> solution
    double D[FR_MAXN][FR_MAXN];             // derivative: l_i'(x_a)
    double Dh[FR_MAXN][FR_MAXN];            // corrected derivative D - liftR lR^T + liftL lL^T
    double lL[FR_MAXN], lR[FR_MAXN];        // l_i(-1), l_i(+1)
    double liftL[FR_MAXN], liftR[FR_MAXN];  // DG-equivalent lift l_i(-+1)/w_i
};
int hex1d(int p, int m, Hex1D &h);

// Prism of order 3: 10 triangle points (the paper's Williams-Shunn set) x 4 GL levels in z;
// quadrature: collapsed 5 x 5 triangle rule x 5 GL points in z (125 points).
#define FR_PT 10      // triangle solution points
#define FR_PQ 25      // triangle quadrature points
#define FR_PE 4       // points per triangle edge (and z levels)
struct Prism2D {
    double xt[FR_PT][2];          // triangle solution points
    double wt[FR_PT];             // int l_t over the reference triangle
    double xq[FR_PQ][2], wq[FR_PQ];
    double Bt[FR_PQ][FR_PT];      // triangle interpolation solution -> quadrature points
    double Pt[FR_PT][FR_PQ];      // triangle L2 projection quadrature -> solution points
    double Dx[FR_PT][FR_PT], Dy[FR_PT][FR_PT];   // in-plane derivatives d l_t'/dx (x_t)
    double Dhx[FR_PT][FR_PT], Dhy[FR_PT][FR_PT]; // corrected: D - sum_f n_f L_f E_f
    double Ef[3][FR_PE][FR_PT];   // interpolation to the edge points of quad faces 2, 3, 4
    double Lf[3][FR_PT][FR_PE];   // DG lift of quad faces 2, 3, 4 (triangle part; identity in z)
    double nf[3][2];              // unit reference normals (x, y) of quad faces 2, 3, 4
    Hex1D z;                      // 1D operators along z (p = 3, m = 5)
};
int prism2d(Prism2D &P);

// Element types without tensor-product structure (Sec. 1: tetrahedra and pyramids use no sum
// factorisation), order 3, with dense per-element operators: NU solution points, NF flux points on
// NFACE faces (face f holds points foff[f] .. foff[f+1]-1), 125 collapsed Gauss-Jacobi quadrature
// points (exact to total degree 9).
//   tetrahedron: 20 solution points (the order-3 equispaced lattice shrunk by 4/5 towards the
//     centroid), 4 faces x 10 flux points (the paper's printed Williams-Shunn triangle points);
//     faces 0 z = -1, 1 y = -1, 2 x = -1, 3 x+y+z = -1.
//   pyramid (base [-1,1]^2 at z = -1, apex (0,0,1)): the rational pyramid space (Q_3 traces on the
//     base, P_3 on the triangles), 30 solution points (the order-3 pyramid lattice shrunk by 4/5
//     towards the centroid (0,0,-1/2)), base 4 x 4 GL flux points (a + 4 b) then 4 triangles x 10
//     Williams-Shunn points; faces 0 base, 1 y = -(1-z)/2, 2 x = (1-z)/2, 3 y = (1-z)/2,
//     4 x = -(1-z)/2. Its derivative operator is the L2 projection of the exact derivative (the
//     rational space is not closed under differentiation).
#define FR_TQ 125     // quadrature points
#define FR_TQP 128    // quadrature points padded to whole 16-byte vectors (the pad rows are zero)
template <int NU_, int NF_, int NFACE_>
struct DenseRef {
    static constexpr int NU = NU_, NF = NF_, NFACE = NFACE_;
    double x[NU][3];               // solution points (reference coordinates)
    double w[NU];                  // int l_z over the reference element
    double xf[NF][3];              // flux points
    double nf[NFACE][3];           // unit outward reference normals
    int foff[NFACE + 1];           // first flux point of each face
    double xq[FR_TQ][3], wq[FR_TQ];
    double B[FR_TQ][NU];           // interpolation to quadrature points (M7)
    double M0[NF][NU];             // interpolation to flux points
    double D[3][NU][NU];           // D[d][z][j]: derivative of l_j at x_z (projected on the pyramid)
    double L[NU][NF];              // DG-equivalent lift M^-1 E
    double Dh[3][NU][NU];          // D_d - L diag(n_d) M0: the operator of M4 - M6 M0 and of M1 - M3 M2
    double Pj[NU][FR_TQ];          // L2 projection (M8)
};
using Tet3D = DenseRef<20, 40, 4>;
using Pyr3D = DenseRef<30, 56, 5>;
#define FR_TU 20      // tetrahedron solution points
#define FR_TF 40      // tetrahedron flux points
#define FR_YU 30      // pyramid solution points
#define FR_YF 56      // pyramid flux points
int tet3d(Tet3D &T);
int pyr3d(Pyr3D &P);

}  // namespace frb

// ---------------------------------------------------------------------------------------------
// Device-side operator tables (constant memory, one slot per hex order p = 2, 3, 4)
// ---------------------------------------------------------------------------------------------
// A line operator A (R outputs x C inputs) whose Gauss-Legendre node sets are symmetric about 0, so
// that A[R-1-r][C-1-c] = S A[r][c] (S = +1 for interpolation and projection, -1 for operators with
// one derivative), in even/odd form: with x_e[c] = x[c] + x[C-1-c] and x_o[c] = x[c] - x[C-1-c]
// (c < C/2), E[r] = sum_c e[r][c] x_e[c] (+ m[r] x[C/2] for odd C) and O[r] = sum_c o[r][c] x_o[c]
// give y[r] = E + O and y[R-1-r] = S (E - O) for r < R/2 (the middle row of odd R is E or O alone):
// about half the multiply-adds of the plain product.
template <typename T>
struct HexEO {
    T e[FR_MAXM][FR_MAXM];    // (A[r][c] + A[r][C-1-c]) / 2
    T o[FR_MAXM][FR_MAXM];    // (A[r][c] - A[r][C-1-c]) / 2
    T m[FR_MAXM];             // A[r][(C-1)/2] (odd C)
};

template <typename T>
struct HexOps {
    HexEO<T> Beo, Peo, DPeo;  // B, Pj and DP in even/odd form
    T B[FR_MAXM][FR_MAXN];
    T Pj[FR_MAXN][FR_MAXM];
    T DP[FR_MAXN][FR_MAXM];   // Dh Pj: projection followed by the corrected derivative
    T Dh[FR_MAXN][FR_MAXN];
    T lL[FR_MAXN], lR[FR_MAXN];
    T liftL[FR_MAXN], liftR[FR_MAXN];
    T w[FR_MAXN];
};

// Prism (p = 3) operator tables: triangle part dense, z part 1D.
template <typename T>
struct PriOps {
    T Bt[FR_PQ][FR_PT];
    T Pt[FR_PT][FR_PQ];
    T Dhx[FR_PT][FR_PT], Dhy[FR_PT][FR_PT];
    T Ef[3][FR_PE][FR_PT];
    T Lf[3][FR_PT][FR_PE];
    T nf[3][2];
    T Bz[5][FR_PE], Pz[FR_PE][5], Dhz[FR_PE][FR_PE];
    T lzL[FR_PE], lzR[FR_PE], liftzL[FR_PE], liftzR[FR_PE];
};

// Dense-element (p = 3) operator tables, transposed so that the output index runs fastest (a warp's
// lanes compute consecutive outputs and read consecutive entries). Rows of the solution-point index
// are padded to NUS (a multiple of 4) for 16-byte vector loads; the pad rows are zero.
template <typename T, int NU_, int NF_, int NFACE_>
struct DenseOps {
    static constexpr int NU = NU_, NF = NF_, NFACE = NFACE_, NUS = (NU_ + 3) / 4 * 4;
    // face f holds flux points F0(f) .. F0(f+1)-1: the first face has NF - 10 (NFACE - 1) points
    // (10 on the tetrahedron, the 16-point base on the pyramid), every other face the 10 triangle points
    static constexpr int FIRST = NF_ - 10 * (NFACE_ - 1);
    static constexpr __host__ __device__ int F0(int f) { return f == 0 ? 0 : FIRST + 10 * (f - 1); }
    static constexpr __host__ __device__ int FACE(int s) { return s < FIRST ? 0 : 1 + (s - FIRST) / 10; }
    T Bt[NUS][FR_TQ];              // B^T: [j][q]
    T M0t[NUS][NF];                // M0^T: [z][s]
    T Dht[3][NU][NU];              // [d][j][z] = Dh[d][z][j]
    T Lt[NF][NU];                  // [s][z] = L[z][s]
    T Dvt[3][FR_TQP][NU];          // (Dh_d Pj)^T: projection with the corrected divergence, [d][q][z]
    T nf[NFACE][3];
    int foff[NFACE + 1];           // F0(f), kept with the table
};
template <typename T> using TetOps = DenseOps<T, 20, 40, 4>;
template <typename T> using PyrOps = DenseOps<T, 30, 56, 5>;
// The FP32 tables as float-float pairs (value = hi + lo): the low-Mach FP32 form's mass channel.
template <typename OPS32>
struct DenseOpsFF {
    OPS32 hi, lo;
    double Dht64[3][OPS32::NU][OPS32::NU];   // Dh in FP64, [d][j][z]: the mass channel's volume term
};

// Prism operators as float-float pairs: value = hi + lo (the low-Mach mass channel).
struct PriOpsFF {
    PriOps<float> hi, lo;
};

// Physical constants of an instance, in the compute precision.
template <typename T>
struct Phys {
    T gamma, gm1, mu, beta, tau;
    T heat;       // mu gamma / ((gamma - 1) Pr)
    T pref;       // reference pressure removed from the momentum flux
    // low-Mach FP32 form: deviations from (rref, 0, 0, 0, eref), reduced energy E - H0 rho
    T rref, eref, H0;
    double H0d, rrefd;
    ff H0ff;      // H0 as a float-float pair
    int dev;
};

// Geometry of one affine element: inverse Jacobian (row-major dxi_i/dx_j) and its determinant.
template <typename T>
struct Geo {
    T Ji[9];
    T det;
    T nidet;      // -1 / det, formed on the host (a division per thread and element costs FP64-pipe slots)
};
// The low-Mach form's geometry of one element: the FP64 inverse Jacobian and determinant, and the
// float-float pairs its mass channel multiplies by, det J J^-1 (row-major) and -1 / det J, formed on
// the host (FP64 arithmetic and conversions run at 1/64 of the FP32 rate on GB300).
struct GeoLM {
    double Ji[9];
    double det;
    ff cm[9];
    ff idet;
};

// One block of elements of one type and order inside one instance.
struct Block {
    int inst;                 // instance index
    int type;                 // 0 hex, 1 prism, 2 tetrahedron, 3 pyramid
    int p, m;                 // order, 1D quadrature points
    int nu, nf;               // points per element, flux points per element
    long long ne;             // elements
    long long elem0;          // first global element
    long long u0;             // first value in U
    long long f0;             // first global flux point
};

// Everything a hex kernel of one element block needs. Face arrays are var-major over the global
// flux-point index of the whole handle: A[var * nfpt + gfpt].
template <typename T>
struct HexArgs {
    long long ne;             // elements in the block
    long long u0;             // first value of the block in U/R
    long long f0;             // first global flux point of the block
    long long nfpt;           // flux points of the whole handle
    const Geo<T> *geo;        // [ne], block-local
    const uint32_t *partner;  // [nfpt] partner gfpt, FR_LFLAG set when this point is the L side
    Phys<T> ph;
    const T *U;               // state, block starts at U + u0
    T *R;                     // RHS
    T *UF;                    // [5][nfpt] solution at flux points
    T *FV;                    // fused: [4][nfpt] own-normal viscous flux n.fv (vars 1..4)
    T *CF;                    // unfused: [5][nfpt] common solution
    T *QF;                    // unfused: [15][nfpt] gradient at flux points
    T *DF;                    // unfused: [5][nfpt] transformed common normal flux
    T *Qu;                    // unfused: [elem][5][3][nu] gradient, later projected flux
    T *UQ;                    // unfused: [elem][5][nq] solution at quadrature points
    T *QQ;                    // unfused: [elem][5][3][nq] gradient, later transformed flux, at qpts
    T *Rt;                    // unfused: [elem][5][nu] R~
    int *status;              // device status word (bit 0: non-physical state; bit 1: a bounded wait gave up)
    // Batched launch over several blocks of one element type and order (all null for one block):
    // per element its first value in U/R, its first global flux point and its instance's physics.
    const long long *eu0;
    const long long *ef0;
    const int *eph;
    const Phys<T> *phtab;
    // RK4 stage fused into the interface kernel: rkstage = 0 writes R; rkstage = s + 1 folds the
    // value k = R(u_s) of stage s in directly: acc = (s ? acc : 0) + b_s k and us = U + c_{s+1} dt k
    // for s < 3; U += dt (acc + b_3 k) for s = 3.
    // Low-Mach FP32 form (ph.dev): FP64 geometry, own-normal mass flux n.(rho v) at flux points,
    // and the volume part of R~_rho per solution point, all in FP64
    const GeoLM *geo64;
    ff *MF;                   // float-float (about 48 bits; FP64 rates are 1/70 of FP32 on this chip)
    ff *RL;
    // Per element and face (6 slots; prisms use 5): unit outward normal and |n_s|, n_s = detJ J^-T n~
    const T *fnrm;            // [elem][6][4] in the compute precision
    const ff *fnrm64;         // [elem][6][4] in float-float (low-Mach mass channel)
    // Split interface phase (FP64): C1 evaluates each pair once from its L point (list lpts, entries
    // element_in_launch * 256 + local flux point) into DF; C2 lifts per element.
    const uint32_t *lpts;
    long long nlpts;
    int rkstage;
    double rkdt;
    double *rkU;
    double *rkacc;
    T *rkus;
    // Prism volume kernel in the FP32 compute precision: 0 = CUDA-core operators; 1 / 2 = the dense
    // triangle interpolation and projection as split hi + lo FP16 / BF16 products on the tensor cores.
    int tcmode;
    // Hexahedral volume kernel without anti-aliasing: the flux is evaluated at the solution points
    // (quadrature points = solution points, so interpolation and projection are the identity).
    int aa_off;
    // Surface-flux anti-aliasing (single hexahedral block): m x m quadrature points per face, element
    // e's at e * 6 m^2 + face * m^2 + a + m b; partner codes as for flux points; the face solution
    // and own-normal viscous flux there, var-major over the nqf points.
    int surf;
    const uint32_t *qpartner;
    T *UFQ;
    T *FVQ;
    T *DQ;                    // [5][nqf] transformed common flux per side
    const uint32_t *qlpts;    // L quadrature points (one per pair)
    long long nqf, nqlpts;
    // Curved (trilinear) hexahedra, unfused form: metric terms at every point (null on affine meshes)
    const T *mu;              // [elem][nu][10]: J^-1 (row-major dxi_i/dx_j) and det J at solution points
    const T *mq;              // [elem][nq][9]: det J J^-1 at quadrature points
    const T *mfn;             // [elem][nf][4]: unit outward normal and |n_s| at flux points
    // Debug: the first bounded wait of every CTA (tensor-core completion or state prefetch) gives up
    // at once, so that the FR_ETIMEOUT path runs without any fault; the drain wait keeps its bound.
    int dbg_wait0;
    long long nU;             // values of U and R in the handle (index checks of the bounds-checking build)
};

// SM count of the calling thread's current device, cached per device: the kernels' grids are sized
// in multiples of it (resident CTAs per SM times the SMs, or a few waves of them)
inline long long fr_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 152;
        cache[dev] = v;
    }
    return cache[dev];
}

#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ void rk_fold(const HexArgs<T> &a, long long i, T val)
{
    const double kv = (double)val;
    const int st = a.rkstage - 1;
    if (st == 3) {
        a.rkU[i] += a.rkdt * (a.rkacc[i] + (1.0 / 6.0) * kv);
    } else {
        const double b = st == 0 ? 1.0 / 6.0 : 1.0 / 3.0;
        const double c = st == 2 ? 1.0 : 0.5;
        a.rkacc[i] = (st == 0 ? 0.0 : a.rkacc[i]) + b * kv;
        a.rkus[i] = (T)(a.rkU[i] + c * a.rkdt * kv);
    }
}
#endif

#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ long long elem_u0(const HexArgs<T> &a, long long e, int nu)
{
    return a.eu0 ? a.eu0[e] : a.u0 + e * FR_NV * nu;
}
template <typename T>
__device__ __forceinline__ long long elem_f0(const HexArgs<T> &a, long long e, int nf)
{
    return a.ef0 ? a.ef0[e] : a.f0 + e * nf;
}
template <typename T>
__device__ __forceinline__ Phys<T> elem_phys(const HexArgs<T> &a, long long e)
{
    return a.eph ? a.phtab[a.eph[e]] : a.ph;
}

// Index checks of the bounds-checking build (compiled with FR_DEBUG_BOUNDS; a release build compiles
// them away). A failed check sets bit 2 of the status word (reported as FR_EBOUNDS) and the access is
// redirected or skipped, so the check itself never touches memory out of bounds.
// The partner flux point of partner code pc (own: this point's index, used if the partner is outside
// the handle's face arrays).
template <typename T>
__device__ __forceinline__ long long fr_partner(const HexArgs<T> &a, uint32_t pc, long long own)
{
    const long long pg = pc & ~FR_LFLAG;
#ifdef FR_DEBUG_BOUNDS
    if (pg >= a.nfpt) {
        atomicOr(a.status, 4);
        return own;
    }
#endif
    return pg;
}

// Element e's values and flux points lie inside U/R and the face arrays (call with every thread of
// the CTA; the first thread reports a failure).
template <typename T>
__device__ __forceinline__ bool fr_elem_ok(const HexArgs<T> &a, long long e, int nu, int nf)
{
#ifdef FR_DEBUG_BOUNDS
    const long long u0 = elem_u0(a, e, nu), f0 = elem_f0(a, e, nf);
    if (u0 < 0 || u0 + (long long)FR_NV * nu > a.nU || f0 < 0 || f0 + nf > a.nfpt) {
        if (threadIdx.x == 0) atomicOr(a.status, 4);
        return false;
    }
#else
    (void)a; (void)e; (void)nu; (void)nf;
#endif
    return true;
}
#endif

// One launch per phase over several element groups (fr_hex.cu): hexahedra p = 3 (kind 3), p = 4
// (kind 4) and prisms (kind 1), flux anti-aliasing on the CUDA cores; every CTA takes its share of
// each group in turn (elements first, first + grid, ... of the group).
#define FR_MULTI_MAX 4
template <typename T>
struct MultiArgs {
    int ng;
    int kind[FR_MULTI_MAX];
    HexArgs<T> a[FR_MULTI_MAX];
    const PriOps<T> *pops;        // prism operator tables (prism groups)
    const PriOpsFF *pff;
};
template <typename T> int multi_phase(int phase, const MultiArgs<T> &ma, cudaStream_t s);

// Launchers (fr_hex.cu). phase: 0 = A (face solution), 1 = B (volume group), 2 = C (interfaces),
// 3 = C1 (common flux once per pair, into DF), 4 = C2 (lift and scale from DF).
// variant: launch shape of the volume kernel (0, 1, 2 = 64, 128, 256 threads per element)
template <typename T> int hex_fused_phase(int p, int phase, const HexArgs<T> &a, cudaStream_t s, int variant = 1);
// kernel: 1..13 in the paper's order (disu .. negdivconf)
template <typename T> int hex_unfused_kernel(int p, int kernel, const HexArgs<T> &a, cudaStream_t s);
int hex_upload_ops(int p, int m, const frb::Hex1D &h);
// Prism kernels (fr_pri.cu); the operator tables are passed by device pointer (opsff: the
// float-float table of the low-Mach FP32 form's mass channel; null otherwise).
template <typename T> int pri_fused_phase(int phase, const HexArgs<T> &a, const PriOps<T> *ops, const PriOpsFF *opsff, cudaStream_t s);
// The FP32 prism operator table in the constant memory of the current device, for the prism kernels
// (fr_pri.cu) and the launches that serve several element groups (fr_hex.cu); 0 on success.
int pri_set_const_ops(const PriOps<float> *h);
int multi_set_pri_const_ops(const PriOps<float> *h);
// Dense-element kernels (fr_dense.cu): tetrahedra and pyramids, operator table by device pointer.
// (opsff: the float-float FP32 table of the low-Mach form's mass channel; null otherwise).
template <typename T>
int tet_fused_phase(int phase, const HexArgs<T> &a, const TetOps<T> *ops, const DenseOpsFF<TetOps<float>> *opsff, cudaStream_t s);
template <typename T>
int pyr_fused_phase(int phase, const HexArgs<T> &a, const PyrOps<T> *ops, const DenseOpsFF<PyrOps<float>> *opsff, cudaStream_t s);
