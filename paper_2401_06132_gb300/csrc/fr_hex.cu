// fr_hex.cu -- hexahedral kernels of the anti-aliased Navier-Stokes FR right-hand side.
//
// Two forms of the same computation (Sec. 2.2 and 2.2.1 kernels, sum-factorised per Sec. 4):
//
//   fused   A: disu                   -> U^(f) at every flux point (global, read by neighbours)
//           B: con_u + tgradpcoru + tgradcoru + gradcoru + gradcoru_fpts (viscous part) +
//              uqpts + gradcoru_qpts + tdisf + tdivtpcorf, per element, intermediates in shared
//              memory; writes R~ into R and the own-normal viscous flux at flux points
//           C: comm_flux + tdivtconf + negdivconf, per element (each side evaluates the common flux
//              of its own flux points with the L/R roles of the pair, so both sides agree bitwise)
//   unfused K1..K13: one kernel per paper kernel with global intermediates (Sec. 3 order).
//
// Hex point index i + n j + n^2 k; the face-local index of a flux point is a + n b over the two
// tangential axes in increasing axis order; flux point sigma = face * n^2 + local.
#include <cuda_runtime.h>

#include <type_traits>

#include "fr_internal.h"
#include "fr_physics.cuh"
#include "fr_tcgen05.cuh"
#include "fr_pri_body.cuh"   // the prism phase bodies, for the launches that serve several groups

__constant__ HexOps<double> c_hex64[3];  // slot p - 2
__constant__ HexOps<float> c_hex32[3];

// Float-float copies of the operators of the low-Mach form's mass channel.
struct HexOpsFF {
    ff lL[FR_MAXN], lR[FR_MAXN], liftL[FR_MAXN], liftR[FR_MAXN];
    ff Dh[FR_MAXN][FR_MAXN];
};
__constant__ HexOpsFF c_hexff[3];

template <typename T> __device__ __forceinline__ const HexOps<T> &OPS(int slot);
template <> __device__ __forceinline__ const HexOps<double> &OPS<double>(int slot) { return c_hex64[slot]; }
template <> __device__ __forceinline__ const HexOps<float> &OPS<float>(int slot) { return c_hex32[slot]; }

// Even/odd form of the R x C line operator A (row stride ld) in both precisions.
static void eo_fill(const double *A, int ld, int R, int C, HexEO<double> &d, HexEO<float> &f)
{
    for (int r = 0; r < (R + 1) / 2; r++) {
        for (int c = 0; c < C / 2; c++) {
            const double e = 0.5 * (A[r * ld + c] + A[r * ld + C - 1 - c]), o = 0.5 * (A[r * ld + c] - A[r * ld + C - 1 - c]);
            d.e[r][c] = e; d.o[r][c] = o; f.e[r][c] = (float)e; f.o[r][c] = (float)o;
        }
        if (C % 2) { d.m[r] = A[r * ld + C / 2]; f.m[r] = (float)A[r * ld + C / 2]; }
    }
}

int hex_upload_ops(int p, int m, const frb::Hex1D &h)
{
    if (p < 2 || p > 4 || m != p + 2) return -1;
    HexOps<double> d{};
    HexOps<float> f{};
    for (int a = 0; a < FR_MAXM; a++)
        for (int i = 0; i < FR_MAXN; i++) { d.B[a][i] = h.B[a][i]; f.B[a][i] = (float)h.B[a][i]; }
    for (int i = 0; i < FR_MAXN; i++) {
        for (int a = 0; a < FR_MAXM; a++) { d.Pj[i][a] = h.Pj[i][a]; f.Pj[i][a] = (float)h.Pj[i][a]; }
        for (int a = 0; a < FR_MAXM; a++) {
            double v = 0.0;
            for (int b = 0; b < FR_MAXN; b++) v += h.Dh[i][b] * h.Pj[b][a];
            d.DP[i][a] = v; f.DP[i][a] = (float)v;
        }
        for (int j = 0; j < FR_MAXN; j++) { d.Dh[i][j] = h.Dh[i][j]; f.Dh[i][j] = (float)h.Dh[i][j]; }
        d.lL[i] = h.lL[i]; d.lR[i] = h.lR[i]; d.liftL[i] = h.liftL[i]; d.liftR[i] = h.liftR[i]; d.w[i] = h.w[i];
        f.lL[i] = (float)h.lL[i]; f.lR[i] = (float)h.lR[i]; f.liftL[i] = (float)h.liftL[i];
        f.liftR[i] = (float)h.liftR[i]; f.w[i] = (float)h.w[i];
    }
    const int n = p + 1;
    eo_fill(&h.B[0][0], FR_MAXN, m, n, d.Beo, f.Beo);
    eo_fill(&h.Pj[0][0], FR_MAXM, n, m, d.Peo, f.Peo);
    eo_fill(&d.DP[0][0], FR_MAXM, n, m, d.DPeo, f.DPeo);
    HexOpsFF x{};
    for (int i = 0; i < FR_MAXN; i++) {
        x.lL[i] = ff_from_double(h.lL[i]); x.lR[i] = ff_from_double(h.lR[i]);
        x.liftL[i] = ff_from_double(h.liftL[i]); x.liftR[i] = ff_from_double(h.liftR[i]);
        for (int j = 0; j < FR_MAXN; j++) x.Dh[i][j] = ff_from_double(h.Dh[i][j]);
    }
    if (cudaMemcpyToSymbol(c_hex64, &d, sizeof(d), (p - 2) * sizeof(d)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(c_hex32, &f, sizeof(f), (p - 2) * sizeof(f)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(c_hexff, &x, sizeof(x), (p - 2) * sizeof(x)) != cudaSuccess) return -2;
    return 0;
}

// Physical outward unit normal and |n_s| (n_s = detJ J^-T n~) of hex face f.
template <typename T>
__device__ __forceinline__ void face_normal(const Geo<T> &g, int f, T *n, T &mag)
{
    const int d = f >> 1;
    const T sgn = (f & 1) ? T(1) : T(-1);
    T ns[3];
#pragma unroll
    for (int k = 0; k < 3; k++) ns[k] = g.det * sgn * g.Ji[3 * d + k];
    mag = sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
    const T im = T(1) / mag;
#pragma unroll
    for (int k = 0; k < 3; k++) n[k] = ns[k] * im;
}

// Unit normal and |n_s| of face f of element e from the per-element face table.
template <typename T, typename V>
__device__ __forceinline__ void face_nrm(const V *tab, long long e, int f, V *n, V &mag)
{
    const V *t = tab + (e * 6 + f) * 4;
    n[0] = t[0]; n[1] = t[1]; n[2] = t[2]; mag = t[3];
}

// Same line in a padded shared-memory layout (x-line stride XS, plane stride PS).
template <int N, int XS, int PS>
__device__ __forceinline__ void face_line_p(int f, int local, int &base, int &stride)
{
    const int d = f >> 1, a = local % N, b = local / N;
    if (d == 0) { base = XS * a + PS * b; stride = 1; }
    else if (d == 1) { base = a + PS * b; stride = XS; }
    else { base = a + XS * b; stride = PS; }
}

// y = A x along one line for an operator in even/odd form (HexEO), S = +1 symmetric, -1 antisymmetric.
template <typename T, int C, int R, int S>
__device__ __forceinline__ void line_eo(const HexEO<T> &A, const T (&x)[C], T (&y)[R])
{
    constexpr int CH = C / 2, RH = R / 2;
    T xe[CH], xo[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) { xe[c] = x[c] + x[C - 1 - c]; xo[c] = x[c] - x[C - 1 - c]; }
#pragma unroll
    for (int r = 0; r < RH; r++) {
        T E = (C % 2) ? A.m[r] * x[CH] : T(0), O = T(0);
#pragma unroll
        for (int c = 0; c < CH; c++) { E += A.e[r][c] * xe[c]; O += A.o[r][c] * xo[c]; }
        y[r] = E + O;
        y[R - 1 - r] = S > 0 ? E - O : O - E;
    }
    if constexpr (R % 2) {   // middle row: the even part alone (S = +1) or the odd part alone (S = -1)
        T v = (S > 0 && (C % 2)) ? A.m[RH] * x[CH] : T(0);
#pragma unroll
        for (int c = 0; c < CH; c++) v += S > 0 ? A.e[RH][c] * xe[c] : A.o[RH][c] * xo[c];
        y[RH] = v;
    }
}

// y = A x along one line for a constant operator with R <= FR_MAXN rows (indices fixed at compile time)
template <typename T, int R, int C>
__device__ __forceinline__ void line_rows(const T (&A)[FR_MAXN][FR_MAXM], const T (&x)[C], T (&y)[R])
{
#pragma unroll
    for (int r = 0; r < R; r++) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < C; c++) v += A[r][c] * x[c];
        y[r] = v;
    }
}

template <int N>
__device__ __forceinline__ void face_line(int f, int local, int &base, int &stride)
{
    // solution-point index of the line through face point `local` of face f: base + i * stride
    const int d = f >> 1, a = local % N, b = local / N;
    if (d == 0) { base = N * a + N * N * b; stride = 1; }
    else if (d == 1) { base = a + N * N * b; stride = N; }
    else { base = a + N * b; stride = N * N; }
}


// ---------------------------------------------------------------------------------------------
// Fused phase A / unfused K1: disu, U^(f) = M0 U
// ---------------------------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(256) k_disu(HexArgs<T> a)
{
    constexpr int N = P + 1, NU = N * N * N, NF = 6 * N * N;
    const HexOps<T> &op = OPS<T>(P - 2);
    const long long total = a.ne * FR_NV * NF;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(it % NF);
        const long long ea = it / NF;
        const int alpha = (int)(ea % FR_NV);
        const long long e = ea / FR_NV;
        const int f = s / (N * N), loc = s % (N * N);
        int base, stride;
        face_line<N>(f, loc, base, stride);
        const T *u = a.U + elem_u0(a, e, NU) + alpha * NU + base;
        const T *l = (f & 1) ? op.lR : op.lL;
        T v = T(0);
#pragma unroll
        for (int i = 0; i < N; i++) v += l[i] * u[i * stride];
        a.UF[alpha * a.nfpt + elem_f0(a, e, NF) + s] = v;
    }
}

// Fused phase A: the same disu over blocks of EB elements. The block's solution is staged in shared
// memory with coalesced loads (each element's 5 x n^3 values are contiguous), then every thread
// writes one flux-point value; consecutive threads write consecutive flux points of one variable.
template <typename T, int P, int EB, int NT>
__device__ __forceinline__ void disu_blk_body(const HexArgs<T> &a, long long first, long long stride)
{
    constexpr int N = P + 1, NU = N * N * N, NF = 6 * N * N;
    __shared__ T s_u[EB * FR_NV * NU];
    // the trace rows, selected by each flux point's run-time face side, from shared memory (a
    // constant-memory load is serialised over the distinct addresses of a warp)
    __shared__ T s_l[2 * N];
    __shared__ ff s_lff[std::is_same<T, float>::value ? 2 * N : 1];
    {
        const HexOps<T> &op = OPS<T>(P - 2);
        for (int i = threadIdx.x; i < 2 * N; i += NT) {
            s_l[i] = i < N ? op.lL[i] : op.lR[i - N];
            if constexpr (std::is_same<T, float>::value) s_lff[i] = i < N ? c_hexff[P - 2].lL[i] : c_hexff[P - 2].lR[i - N];
        }
        __syncthreads();
    }
    for (long long e0 = (long long)first * EB; e0 < a.ne; e0 += (long long)stride * EB) {
        const int nb = (int)((a.ne - e0) < EB ? (a.ne - e0) : EB);
        {
            bool blk_ok = true;
            for (int k = 0; k < nb; k++) blk_ok = blk_ok && fr_elem_ok(a, e0 + k, NU, NF);
            if (!blk_ok) continue;
        }
        for (int i = threadIdx.x; i < nb * FR_NV * NU; i += NT) {
            const int el = i / (FR_NV * NU), r = i % (FR_NV * NU);
            T v = a.eu0 == nullptr ? a.U[a.u0 + e0 * FR_NV * NU + i] : a.U[a.eu0[e0 + el] + r];
            if constexpr (std::is_same<T, float>::value) {
                const Phys<T> ph = elem_phys(a, e0 + el);
                if (ph.dev) {   // deviations from the reference state (exact in FP32)
                    if (r < NU) v -= ph.rref;
                    else if (r >= 4 * NU) v -= ph.eref;
                }
            }
            s_u[i] = v;
        }
        __syncthreads();
        // one thread per (element, flux point), all five variables: the face line is located once.
        // FP32: the face values are evaluated with the float-float line operator (exact products,
        // TwoSum accumulation) and rounded once; at low Mach the Rusanov dissipation
        // (1/2)(|v.n| + c)(u_L - u_R), with c about 10 |v|, lifts any rounding of a face value into R.
        for (int it = threadIdx.x; it < nb * NF; it += NT) {
            const int el = it / NF, sp = it % NF, f = sp / (N * N);
            int base, stride;
            face_line<N>(f, sp % (N * N), base, stride);
            const long long fo = elem_f0(a, e0 + el, NF) + sp;
            if constexpr (std::is_same<T, float>::value) {
                const ff *lf = s_lff + (f & 1) * N;
                ff v[FR_NV];
#pragma unroll
                for (int alpha = 0; alpha < FR_NV; alpha++) {
                    const T *u = s_u + (el * FR_NV + alpha) * NU + base;
                    float sh, c;
                    dot2_first(lf[0], u[0], sh, c);
#pragma unroll
                    for (int i = 1; i < N; i++) dot2_next(lf[i], u[i * stride], sh, c);
                    const ff w = fast_two_sum(sh, c);
                    v[alpha] = w;
                    a.UF[alpha * a.nfpt + fo] = w.hi + w.lo;
                }
                // low-Mach form: own-normal mass flux n.(rho v) at every flux point, in float-float
                // (curved elements carry their mass flux through the FP32 flux path instead)
                if (elem_phys(a, e0 + el).dev && !a.mu && !a.surf) {
                    const ff *nt = a.fnrm64 + ((e0 + el) * 6 + f) * 4;
                    ff mf = ff_of(0.0f);
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const ff nk = nt[k];
                        if (nk.hi == 0.0f) continue;   // axis-aligned faces need one component
                        mf = ff_fma(nk, v[1 + k], mf);
                    }
                    a.MF[fo] = mf;
                }
            } else {
                const T *l = s_l + (f & 1) * N;
#pragma unroll
                for (int alpha = 0; alpha < FR_NV; alpha++) {
                    const T *u = s_u + (el * FR_NV + alpha) * NU + base;
                    T v = T(0);
#pragma unroll
                    for (int i = 0; i < N; i++) v += l[i] * u[i * stride];
                    a.UF[alpha * a.nfpt + fo] = v;
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int P, int EB, int NT>
__global__ void __launch_bounds__(NT) k_disu_blk(HexArgs<T> a)
{
    disu_blk_body<T, P, EB, NT>(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------------------------
// Fused phase B: the per-element volume group
// ---------------------------------------------------------------------------------------------
template <typename T, int P>
struct HexSmem {
    static constexpr int N = P + 1, M = P + 2, NU = N * N * N, NF = 6 * N * N, NQ = M * M * M;
    // solution-point fields are padded so that x-lines of even length do not start on the same banks
    static constexpr int XS = (N % 2 == 0) ? N + 1 : N, PS = XS * N, FS = PS * N;
    // the sweeps take all 20 (15) fields per pass with one staging buffer (the first sweep's output
    // goes to the quadrature-point buffer): fewer barriers, and work-item counts (20 n^2, 20 m n,
    // 20 m^2 lines) that fill whole warps, which FP64, bound by its pipe, needs more than resident CTAs
    // s_u, s_q, s_c (the state, the gradient, the common solution): free once the interpolation's
    // first sweep has read them, so its second sweep and the projection stage their outputs there
    // (the region is sized for the larger of the two uses)
    static constexpr int LOW = (20 * FS + 5 * NF) > 20 * M * M * N ? 20 * FS + 5 * NF : 20 * M * M * N;
    // the next element's state, fetched by the bulk-copy engine while this one computes (the copy
    // must be a whole number of 16-byte units)
    static constexpr bool TMA = (5 * NU * sizeof(T)) % 16 == 0;
    static constexpr int PF = TMA ? 5 * NU : 0;
    static constexpr int SIZE = LOW + PF + 20 * NQ;
};

// Mixed forms (tcmode 1 = FP16, 2 = BF16 halves): the x-y factor of the interpolation, B (x) B
// (M^2 x N^2), and of the projection, Pj (x) Pj (N^2 x M^2), are applied as dense blocks on the
// tensor cores to all 20 (15) fields and all z quadrature levels of an element in one M = 128 MMA
// chain each, as split products [x_hi | x_lo | x_hi] . [y_hi | y_hi | y_lo]; the z factor stays on
// the CUDA cores. The dense block takes N M / (N + M) times the multiply-adds of two 1D sweeps (and
// three for the split), paid on a unit with about 30 times the FP32 rate of the CUDA cores.
template <int P, int TCM>
struct HexTc {
    static constexpr int N = P + 1, M = P + 2, N2 = N * N, M2 = M * M;
    static constexpr int RI = 20 * M, RP = 15 * M;                 // rows: field x z quadrature level
    // K: the split form's segments (tc::SplitForm: FP16 three, BF16 six) of N^2 or M^2 values
    static constexpr int KI = tc::split_k<TCM>(N2), KP = tc::split_k<TCM>(M2);
    static constexpr int NI = (M2 + 15) / 16 * 16, NP = (N2 + 15) / 16 * 16;
    static constexpr int SBO_I = KI / 8 * 128, SBO_P = KP / 8 * 128;
    static constexpr int A_I = (RI + 7) / 8 * SBO_I, A_P = (RP + 7) / 8 * SBO_P;
    static constexpr int A_BYTES = ((A_I > A_P ? A_I : A_P) + 127) / 128 * 128;
    static constexpr int BI_BYTES = NI / 8 * SBO_I, BP_BYTES = NP / 8 * SBO_P;
    static constexpr int ST = N2 | 1;                               // odd row stride of staged rows
    static constexpr int TT = (RI > RP ? RI : RP) * ST;             // staged rows (floats)
    static constexpr int COLS = NI > 32 ? 64 : 32;                  // tensor-memory columns
    static constexpr int HEAD = 128 + A_BYTES + BI_BYTES + BP_BYTES;  // before the kernel's arrays
    static_assert(RI <= 128 && RP <= 128, "one M = 128 tile per element");
};

// Scales the L values x of one operand row by 2^sh (its largest magnitude into [2^14, 2^15)) and
// writes their split parts as row r of the tile (K values); returns sh.
template <int TCM, int K, int L>
__device__ __forceinline__ int split_store_row(unsigned char *base, int r, float (&x)[L])
{
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < L; i++) mx = fmaxf(mx, fabsf(x[i]));
    const int sh = tc::row_shift(mx);
    const float sc = tc::pow2f(sh);
#pragma unroll
    for (int i = 0; i < L; i++) x[i] *= sc;
    tc::store_split_parts<TCM, K, L>(base, r, x);
    return sh;
}

// Sum-factorised interpolation of 5 fields (src, stride NU) to quadrature points (dst, stride NQ).
template <typename T, int P, int NT, int XS = P + 1, int PS = (P + 1) * (P + 1), int FS = (P + 1) * (P + 1) * (P + 1)>
__device__ __forceinline__ void interp_5(const HexOps<T> &op, const T *src, T *t1, T *t2, T *dst)
{
    constexpr int N = P + 1, M = P + 2, NQ = M * M * M;
    for (int it = threadIdx.x; it < 5 * N * N; it += NT) {  // x: (fc, j, k)
        const int fc = it / (N * N), jk = it % (N * N);
        const int sb = fc * FS + XS * (jk % N) + PS * (jk / N);
        T u[N], v[M];
#pragma unroll
        for (int i = 0; i < N; i++) u[i] = src[sb + i];
        line_eo<T, N, M, 1>(op.Beo, u, v);
#pragma unroll
        for (int q = 0; q < M; q++) t1[fc * M * N * N + q + M * jk] = v[q];
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 5 * M * N; it += NT) {  // y: (fc, qa, k)
        const int fc = it / (M * N), r = it % (M * N), qa = r % M, k = r / M;
        T u[N], v[M];
#pragma unroll
        for (int j = 0; j < N; j++) u[j] = t1[fc * M * N * N + qa + M * j + M * N * k];
        line_eo<T, N, M, 1>(op.Beo, u, v);
#pragma unroll
        for (int q = 0; q < M; q++) t2[fc * M * M * N + qa + M * q + M * M * k] = v[q];
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 5 * M * M; it += NT) {  // z: (fc, qa, qb)
        const int fc = it / (M * M), ab = it % (M * M);
        T u[N], v[M];
#pragma unroll
        for (int k = 0; k < N; k++) u[k] = t2[fc * M * M * N + ab + M * M * k];
        line_eo<T, N, M, 1>(op.Beo, u, v);
#pragma unroll
        for (int q = 0; q < M; q++) {
            dst[fc * NQ + ab + M * M * q] = v[q];
        }
    }
    __syncthreads();
}

// Sum-factorised interpolation of all 20 fields at once (src: fields at stride FS, padded layout)
// to the quadrature points (dst, stride NQ), x then y then z; the x sweep is staged in dst itself,
// the y sweep in tmp (20 M^2 N values). Three barriers instead of twelve. FP64 applies B in its
// even/odd form (B is centro-symmetric), FP32 the plain rows.
template <typename T, int P, int NT, int XS, int PS, int FS>
__device__ __forceinline__ void interp_all(const HexOps<T> &op, const T *src, T *tmp, T *dst)
{
    constexpr int N = P + 1, M = P + 2, NQ = M * M * M, NF_ = 20;
    T *xs = dst;   // [f][qa + M (j + N k)]
    for (int it = threadIdx.x; it < NF_ * N * N; it += NT) {
        const int f = it / (N * N), jk = it % (N * N);
        const int sb = f * FS + XS * (jk % N) + PS * (jk / N);
        T u[N];
#pragma unroll
        for (int i = 0; i < N; i++) u[i] = src[sb + i];
        if constexpr (sizeof(T) == 8) {
            T v[M];
            line_eo<T, N, M, 1>(op.Beo, u, v);
#pragma unroll
            for (int q = 0; q < M; q++) xs[f * M * N * N + q + M * jk] = v[q];
        } else {
#pragma unroll
        for (int q = 0; q < M; q++) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < N; i++) v += op.B[q][i] * u[i];
            xs[f * M * N * N + q + M * jk] = v;
        }
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < NF_ * M * N; it += NT) {   // (f, qa, k)
        const int f = it / (M * N), r = it % (M * N), qa = r % M, k = r / M;
        T u[N];
#pragma unroll
        for (int j = 0; j < N; j++) u[j] = xs[f * M * N * N + qa + M * j + M * N * k];
        if constexpr (sizeof(T) == 8) {
            T v[M];
            line_eo<T, N, M, 1>(op.Beo, u, v);
#pragma unroll
            for (int q = 0; q < M; q++) tmp[f * M * M * N + qa + M * q + M * M * k] = v[q];
        } else {
#pragma unroll
        for (int q = 0; q < M; q++) {
            T v = T(0);
#pragma unroll
            for (int j = 0; j < N; j++) v += op.B[q][j] * u[j];
            tmp[f * M * M * N + qa + M * q + M * M * k] = v;
        }
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < NF_ * M * M; it += NT) {   // (f, qa, qb)
        const int f = it / (M * M), ab = it % (M * M);
        T u[N];
#pragma unroll
        for (int k = 0; k < N; k++) u[k] = tmp[f * M * M * N + ab + M * M * k];
        if constexpr (sizeof(T) == 8) {
            T v[M];
            line_eo<T, N, M, 1>(op.Beo, u, v);
#pragma unroll
            for (int q = 0; q < M; q++) dst[f * NQ + ab + M * M * q] = v[q];
        } else {
#pragma unroll
        for (int q = 0; q < M; q++) {
            T v = T(0);
#pragma unroll
            for (int k = 0; k < N; k++) v += op.B[q][k] * u[k];
            dst[f * NQ + ab + M * M * q] = v;
        }
        }
    }
    __syncthreads();
}

// tdivtpcorf with the corrected divergence folded into the projection: the projection of the
// flux component along direction d uses Dh Pj instead of Pj along d, and the last (x) sweep sums
// the three components, so R~[alpha] = sum_d Dh_d (Pj x Pj x Pj) F~[alpha][d] lands in R directly.
// src: the 15 transformed-flux fields at the quadrature points (field alpha 3 + d, stride NQ), all
// in one pass through tmp (15 M^2 N values); every sweep stages its output where its input has been
// consumed. The loops over the three directions are unrolled, so that each sweep's operator is known
// at compile time: its coefficients are constant-bank operands of the multiply-adds, not run-time
// loads from constant memory (one per coefficient and line, serialised over the distinct addresses
// of a warp). FP64 applies the even/odd forms (Pj symmetric, Dh Pj antisymmetric: fewer
// multiply-adds on its slow pipe), FP32 the plain rows.
template <typename T, int P, int NT>
__device__ __forceinline__ void project_div_all(const HexOps<T> &op, T *src, T *tmp, T *R)
{
    constexpr int N = P + 1, M = P + 2, NQ = M * M * M, NU = N * N * N;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const T(&Z)[FR_MAXN][FR_MAXM] = d == 2 ? op.DP : op.Pj;
        for (int it = threadIdx.x; it < 5 * M * M; it += NT) {   // z: (alpha, qa qb) -> k
            const int alpha = it / (M * M), ab = it % (M * M);
            T u[M], v[N];
#pragma unroll
            for (int c = 0; c < M; c++) u[c] = src[(alpha * 3 + d) * NQ + ab + M * M * c];
            if constexpr (sizeof(T) == 8) {
                if (d == 2) line_eo<T, M, N, -1>(op.DPeo, u, v);
                else line_eo<T, M, N, 1>(op.Peo, u, v);
            } else line_rows<T, N, M>(Z, u, v);
#pragma unroll
            for (int k = 0; k < N; k++) tmp[(d * 5 + alpha) * M * M * N + ab + M * M * k] = v[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const T(&Y)[FR_MAXN][FR_MAXM] = d == 1 ? op.DP : op.Pj;
        for (int it = threadIdx.x; it < 5 * M * N; it += NT) {   // y: (alpha, qa, k) -> j
            const int alpha = it / (M * N), r2 = it % (M * N), qa = r2 % M, k = r2 / M;
            T u[M], v[N];
#pragma unroll
            for (int b = 0; b < M; b++) u[b] = tmp[(d * 5 + alpha) * M * M * N + qa + M * b + M * M * k];
            if constexpr (sizeof(T) == 8) {
                if (d == 1) line_eo<T, M, N, -1>(op.DPeo, u, v);
                else line_eo<T, M, N, 1>(op.Peo, u, v);
            } else line_rows<T, N, M>(Y, u, v);
#pragma unroll
            for (int j = 0; j < N; j++) src[(alpha * 3 + d) * NQ + qa + M * j + M * N * k] = v[j];   // over the consumed input
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 5 * N * N; it += NT) {   // x: (alpha, j, k), sum over d -> i
        const int alpha = it / (N * N), jk = it % (N * N);
        T v[N];
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = T(0);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const T(&X)[FR_MAXN][FR_MAXM] = d == 0 ? op.DP : op.Pj;
            T u[M], y[N];
#pragma unroll
            for (int q = 0; q < M; q++) u[q] = src[(alpha * 3 + d) * NQ + q + M * jk];
            if constexpr (sizeof(T) == 8) {
                if (d == 0) line_eo<T, M, N, -1>(op.DPeo, u, y);
                else line_eo<T, M, N, 1>(op.Peo, u, y);
            } else line_rows<T, N, M>(X, u, y);
#pragma unroll
            for (int i = 0; i < N; i++) v[i] += y[i];
        }
#pragma unroll
        for (int i = 0; i < N; i++) R[alpha * NU + i + N * jk] = v[i];
    }
}

// Sum-factorised L2 projection of 5 fields from quadrature points (src, stride NQ) to solution
// points (dst, stride NU).
template <typename T, int P, int NT, int XS = P + 1, int PS = (P + 1) * (P + 1), int FS = (P + 1) * (P + 1) * (P + 1)>
__device__ __forceinline__ void project_5(const HexOps<T> &op, const T *src, T *t1, T *t2, T *dst)
{
    constexpr int N = P + 1, M = P + 2, NQ = M * M * M;
    for (int it = threadIdx.x; it < 5 * M * M; it += NT) {  // z: (fc, qa, qb) -> k
        const int fc = it / (M * M), ab = it % (M * M);
        T u[M];
#pragma unroll
        for (int c = 0; c < M; c++) u[c] = src[fc * NQ + ab + M * M * c];
#pragma unroll
        for (int k = 0; k < N; k++) {
            T v = T(0);
#pragma unroll
            for (int c = 0; c < M; c++) v += op.Pj[k][c] * u[c];
            t2[fc * M * M * N + ab + M * M * k] = v;
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 5 * M * N; it += NT) {  // y: (fc, qa, k) -> j
        const int fc = it / (M * N), r = it % (M * N), qa = r % M, k = r / M;
        T u[M];
#pragma unroll
        for (int b = 0; b < M; b++) u[b] = t2[fc * M * M * N + qa + M * b + M * M * k];
#pragma unroll
        for (int j = 0; j < N; j++) {
            T v = T(0);
#pragma unroll
            for (int b = 0; b < M; b++) v += op.Pj[j][b] * u[b];
            t1[fc * M * N * N + qa + M * j + M * N * k] = v;
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 5 * N * N; it += NT) {  // x: (fc, j, k) -> i
        const int fc = it / (N * N), jk = it % (N * N);
        T u[M];
#pragma unroll
        for (int q = 0; q < M; q++) u[q] = t1[fc * M * N * N + q + M * jk];
        const int db = fc * FS + XS * (jk % N) + PS * (jk / N);
#pragma unroll
        for (int i = 0; i < N; i++) {
            T v = T(0);
#pragma unroll
            for (int q = 0; q < M; q++) v += op.Pj[i][q] * u[q];
            dst[db + i] = v;
        }
    }
    __syncthreads();
}

template <typename T, int P, int NT, int TCM = 0, bool AA = true, bool SURF = false, bool CURV = false>
__device__ __forceinline__ void fused_B_body(const HexArgs<T> &a, long long first, long long stride)
{
    static_assert(AA || TCM == 0, "the collocation form has no interpolation or projection");
    static_assert(!SURF || (AA && TCM == 0), "surface-flux anti-aliasing runs with flux anti-aliasing on the CUDA cores");
    // CURV: curved (trilinear) elements of a single block, metric terms per point from a.mu, a.mq, a.mfn
    static_assert(!CURV || (AA && !SURF && TCM == 0), "curved elements: flux anti-aliasing on the CUDA cores");
    using S = HexSmem<T, P>;
    using TC = HexTc<P, TCM == 0 ? 1 : TCM>;
    static_assert(TCM == 0 || (NT == 128 && std::is_same<T, float>::value), "tensor-core form: FP32, one warpgroup");
    constexpr int N = S::N, M = S::M, NU = S::NU, NF = S::NF, NQ = S::NQ;
    constexpr int XS = S::XS, PS = S::PS, FS = S::FS;
    (void)M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // tensor-core form: operand tiles first (the MMA reads 128 rows of A; rows past the element's
    // last run on into the following buffers and only feed unread accumulator lanes)
    unsigned char *tA = nullptr, *tBi = nullptr, *tBp = nullptr;
    unsigned char *arr = smem_raw;
    if constexpr (TCM != 0) {
        const uint32_t raw = tc::smem_u32(smem_raw);
        tA = smem_raw + ((128 - (raw & 127)) & 127);
        tBi = tA + TC::A_BYTES;
        tBp = tBi + TC::BI_BYTES;
        arr = smem_raw + TC::HEAD;
    }
    T *s_u = reinterpret_cast<T *>(arr);
    T *s_q = s_u + 5 * FS;
    T *s_c = s_q + 15 * FS;
    T *s_pf = s_u + S::LOW;                    // prefetched state of the next element
    T *s_w = s_pf + S::PF;
    T *s_t1 = s_w + 20 * NQ;                   // scratch of the surface-flux and tensor-core paths
    __shared__ short s_list[NF];
    __shared__ int s_cnt;
    __shared__ int s_sh[TCM ? 128 : 1];
    __shared__ uint64_t s_mbar[1];
    __shared__ uint32_t s_tmem[1];
    const HexOps<T> &op = OPS<T>(P - 2);
    uint32_t tmem = 0, parity = 0;
    bool tc_fail = false;
    // The next element's state is fetched by the bulk-copy engine while this element computes: the
    // copy goes into s_pf (issued as soon as this element's state has been read from it) and lands on
    // s_ubar. Needs the tile to be a whole number of 16-byte units (p = 3) and 16-byte aligned in
    // memory (checked per element).
    constexpr bool TMA_U = S::TMA;
    __shared__ uint64_t s_ubar;
    bool pending = false;
    uint32_t uparity = 0;
    bool first_wait = true;
    if constexpr (TMA_U) {
        if (threadIdx.x == 0) tc::mbar_init(&s_ubar, 1);
        __syncthreads();
    }
    if constexpr (TCM != 0) {
        tc::setup(s_mbar, s_tmem, TC::COLS);
        // operator blocks in the split form's segments (FP16: [hi | hi | lo]) from the FP64 1D operators
        using SF = tc::SplitForm<TCM>;
        const HexOps<double> &o64 = OPS<double>(P - 2);
        for (int i = threadIdx.x; i < TC::NI * TC::KI; i += NT) {
            const int n = i / TC::KI, k = i % TC::KI, sg = k / TC::N2;
            uint16_t pp[3] = {0, 0, 0};
            if (n < TC::M2 && sg < SF::SEGS) {
                const int kk = k % TC::N2;
                tc::split_parts<TCM>((float)(o64.B[n % M][kk % N] * o64.B[n / M][kk / N]), pp);
            }
            *reinterpret_cast<uint16_t *>(tBi + tc::core_offset(n, k, TC::SBO_I)) = sg < SF::SEGS ? pp[SF::y_part(sg)] : (uint16_t)0;
        }
        for (int i = threadIdx.x; i < TC::NP * TC::KP; i += NT) {
            const int n = i / TC::KP, k = i % TC::KP, sg = k / TC::M2;
            uint16_t pp[3] = {0, 0, 0};
            if (n < TC::N2 && sg < SF::SEGS) {
                const int kk = k % TC::M2;
                tc::split_parts<TCM>((float)(o64.Pj[n % N][kk % M] * o64.Pj[n / N][kk / M]), pp);
            }
            *reinterpret_cast<uint16_t *>(tBp + tc::core_offset(n, k, TC::SBO_P)) = sg < SF::SEGS ? pp[SF::y_part(sg)] : (uint16_t)0;
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tmem = s_tmem[0];
    }

    for (long long e = first; e < a.ne; e += stride) {
        const Geo<T> g = a.geo[e];
        const Phys<T> ph = elem_phys(a, e);
        const T *U = a.U + elem_u0(a, e, NU);
        const long long gf0 = elem_f0(a, e, NF);
        // 1. load the element's solution (deviations from the reference state in the low-Mach form)
        bool dev = false;
        if constexpr (std::is_same<T, float>::value) dev = ph.dev != 0;
        const T *usrc = U;
        if constexpr (TMA_U) {
            if (pending) {
                const bool landed = tc::mbar_wait(&s_ubar, uparity, tc::first_limit(first_wait, a.dbg_wait0));
                uparity ^= 1;
                pending = false;
                if (__syncthreads_and(landed)) {
                    usrc = s_pf;
                } else {
                    // the copy did not land within the bound: report it, give it one more bounded
                    // wait, and read the state from global memory
                    if (threadIdx.x == 0) atomicOr(a.status, 2);
                    tc::mbar_wait(&s_ubar, uparity ^ 1);
                }
            }
        }
        // (after any prefetch of this element has landed: nothing is left in flight when it is skipped)
        if (!fr_elem_ok(a, e, NU, NF)) continue;
        for (int it = threadIdx.x; it < 5 * NU; it += NT) {
            T v = usrc[it];
            if constexpr (std::is_same<T, float>::value) {
                if (dev) v -= (it < NU) ? ph.rref : (it >= 4 * NU ? ph.eref : T(0));
            }
            const int alpha = it / NU, z = it % NU;
            s_u[alpha * FS + z % N + XS * ((z / N) % N) + PS * (z / (N * N))] = v;
        }
        if constexpr (TMA_U) {
            tc::fence_async_smem();   // this element's reads of s_pf before the copy that overwrites it
            __syncthreads();
            // prefetch the next element's state into s_pf
            const long long en = e + stride;
            bool en_ok = en < a.ne;
#ifdef FR_DEBUG_BOUNDS
            if (en_ok) {   // the bounds-checking build prefetches only elements inside U
                const long long un = elem_u0(a, en, NU);
                en_ok = un >= 0 && un + (long long)FR_NV * NU <= a.nU;
            }
#endif
            if (en_ok) {
                const T *Un = a.U + elem_u0(a, en, NU);
                if ((reinterpret_cast<uintptr_t>(Un) & 15) == 0) {
                    if (threadIdx.x == 0) tc::bulk_g2s(s_pf, Un, 5 * NU * sizeof(T), &s_ubar);
                    pending = true;
                }
            }
        }
        // 2. con_u: common solution at own flux points, C = (1/2 - beta) uL + (1/2 + beta) uR
        for (int it = threadIdx.x; it < 5 * NF; it += NT) {
            const int alpha = it / NF, s = it % NF;
            const uint32_t pc = a.partner[gf0 + s];
            const bool isL = (pc & FR_LFLAG) != 0;
            const long long pg = fr_partner(a, pc, gf0 + s);
            const T own = a.UF[alpha * a.nfpt + gf0 + s], oth = a.UF[alpha * a.nfpt + pg];
            const T uL = isL ? own : oth, uR = isL ? oth : own;
            s_c[it] = (T(0.5) - ph.beta) * uL + (T(0.5) + ph.beta) * uR;
        }
        __syncthreads();
        // 3. tgradpcoru + tgradcoru along lines: q~ = Dh u + liftR C_R - liftL C_L
        for (int it = threadIdx.x; it < 15 * N * N; it += NT) {
            const int alpha = it / (3 * N * N), r = it % (3 * N * N), d = r / (N * N), loc = r % (N * N);
            int base, stride;
            face_line_p<N, XS, PS>(2 * d, loc, base, stride);
            T u[N];
#pragma unroll
            for (int i = 0; i < N; i++) u[i] = s_u[alpha * FS + base + i * stride];
            const T cL = s_c[alpha * NF + (2 * d) * N * N + loc], cR = s_c[alpha * NF + (2 * d + 1) * N * N + loc];
#pragma unroll
            for (int i = 0; i < N; i++) {
                T v = op.liftR[i] * cR - op.liftL[i] * cL;
#pragma unroll
                for (int j = 0; j < N; j++) v += op.Dh[i][j] * u[j];
                s_q[(alpha * 3 + d) * FS + base + i * stride] = v;
            }
        }
        __syncthreads();
        // 4. gradcoru: q = J^-T q~ (per point, all three components; diagonal J^-1 is common)
        const bool diagJ = g.Ji[1] == T(0) && g.Ji[2] == T(0) && g.Ji[3] == T(0) && g.Ji[5] == T(0) &&
                           g.Ji[6] == T(0) && g.Ji[7] == T(0);
        for (int it = threadIdx.x; it < 5 * NU; it += NT) {
            const int alpha = it / NU, z = it % NU;
            T *q = s_q + alpha * 3 * FS + z % N + XS * ((z / N) % N) + PS * (z / (N * N));
            if constexpr (CURV) {   // J^-T at this solution point
                const T *Ji = a.mu + (e * NU + z) * 10;
                const T q0 = q[0], q1 = q[FS], q2 = q[2 * FS];
#pragma unroll
                for (int k = 0; k < 3; k++) q[k * FS] = Ji[k] * q0 + Ji[3 + k] * q1 + Ji[6 + k] * q2;
            } else if (diagJ) {
                q[0] *= g.Ji[0]; q[FS] *= g.Ji[4]; q[2 * FS] *= g.Ji[8];
            } else {
                const T q0 = q[0], q1 = q[FS], q2 = q[2 * FS];
#pragma unroll
                for (int k = 0; k < 3; k++) q[k * FS] = g.Ji[k] * q0 + g.Ji[3 + k] * q1 + g.Ji[6 + k] * q2;
            }
        }
        // 5. gradcoru_fpts + the viscous part of comm_flux: own-normal n.f^v at own flux points.
        //    The LDG flux weighs the two sides by 1/2 + beta (L) and 1/2 - beta (R); a side whose
        //    weight is exactly zero (beta = +-1/2) is not evaluated. The needed points are compacted
        //    so that whole warps do the work.
        if constexpr (SURF) {
            // surface-flux anti-aliasing: the face solution and the own-normal viscous flux at the
            // m x m quadrature points of each face, interpolated in-plane from the n x n traces
            // (along the first face direction into s_t1, then per point along the second). A face
            // is wholly the L or the R side of its pair; only L faces need the gradient (LDG weight
            // 1/2 + beta; the R side's weight 1/2 - beta is zero at beta = 1/2, checked per point).
            T *tr = s_w;    // [face][field 0..19][n^2] traces (free until step 6; s_q follows s_u)
            T *ti = s_t1;   // [face][field][qa][k] = sum_j B[qa][j] tr[j + n k]
            __syncthreads();   // the physical gradient (step 4) is complete
            for (int it = threadIdx.x; it < 6 * 20 * N * N; it += NT) {
                const int f = it / (20 * N * N), r = it % (20 * N * N), fld = r / (N * N), loc = r % (N * N);
                int base, stride;
                face_line_p<N, XS, PS>(f, loc, base, stride);
                const T *l = (f & 1) ? op.lR : op.lL;
                const T *src = s_u + fld * FS + base;
                if constexpr (std::is_same<T, float>::value) {
                    if (fld < 5) {
                        // the state's traces as compensated products (float-float line operator),
                        // rounded once: the face values feed the Rusanov dissipation
                        const HexOpsFF &off = c_hexff[P - 2];
                        const ff *lf = (f & 1) ? off.lR : off.lL;
                        float sh, c;
                        dot2_first(lf[0], src[0], sh, c);
#pragma unroll
                        for (int i = 1; i < N; i++) dot2_next(lf[i], src[i * stride], sh, c);
                        const ff w = fast_two_sum(sh, c);
                        tr[it] = w.hi + w.lo;
                        continue;
                    }
                }
                T v = T(0);
#pragma unroll
                for (int i = 0; i < N; i++) v += l[i] * src[i * stride];
                tr[it] = v;
            }
            __syncthreads();
            for (int it = threadIdx.x; it < 6 * 20 * M * N; it += NT) {
                const int f = it / (20 * M * N), r = it % (20 * M * N), fld = r / (M * N), qk = r % (M * N);
                const int qa = qk % M, k = qk / M;
                if (fld >= 5 && !(a.qpartner[e * 6LL * M * M + f * M * M] & FR_LFLAG)) continue;   // R face
                const T *t = tr + (f * 20 + fld) * N * N + N * k;
                T v = T(0);
#pragma unroll
                for (int j = 0; j < N; j++) v += op.B[qa][j] * t[j];
                ti[it] = v;
            }
            __syncthreads();
            for (int it = threadIdx.x; it < 6 * M * M; it += NT) {
                const int f = it / (M * M), t = it % (M * M), qa = t % M, qb = t / M;
                const long long gq = e * 6LL * M * M + it;
                const bool isL = (a.qpartner[gq] & FR_LFLAG) != 0;
                const T wgt = isL ? T(0.5) + ph.beta : T(0.5) - ph.beta;
                const T *tf = ti + f * 20 * M * N + qa;
                T uf[5];
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    T v = T(0);
#pragma unroll
                    for (int k = 0; k < N; k++) v += op.B[qb][k] * tf[alpha * M * N + M * k];
                    uf[alpha] = v;
                    a.UFQ[alpha * a.nqf + gq] = v;
                }
                if constexpr (std::is_same<T, float>::value) {
                    // low-Mach form: the face values are deviations; the viscous flux takes the state
                    if (dev) { uf[0] += ph.rref; uf[4] += ph.eref; }
                }
                if (wgt == T(0)) {
#pragma unroll
                    for (int k = 0; k < 4; k++) a.FVQ[k * a.nqf + gq] = T(0);
                    continue;
                }
                if (!isL) {
                    // an R face needs its gradient only if beta != 1/2: evaluate it from the traces
                    const T *tr_f = tr + f * 20 * N * N;
                    T qf[5][3];
#pragma unroll
                    for (int c = 0; c < 15; c++) {
                        T v = T(0);
#pragma unroll
                        for (int k = 0; k < N; k++) {
                            T w = T(0);
#pragma unroll
                            for (int j = 0; j < N; j++) w += op.B[qa][j] * tr_f[(5 + c) * N * N + j + N * k];
                            v += op.B[qb][k] * w;
                        }
                        qf[c / 3][c % 3] = v;
                    }
                    T n[3], mag;
                    face_nrm<T, T>(a.fnrm, e, f, n, mag);
                    T fvn[4];
                    viscous_normal_flux(ph, uf, qf, n, fvn);
#pragma unroll
                    for (int k = 0; k < 4; k++) a.FVQ[k * a.nqf + gq] = fvn[k];
                    continue;
                }
                T qf[5][3];
#pragma unroll
                for (int c = 0; c < 15; c++) {
                    T v = T(0);
#pragma unroll
                    for (int k = 0; k < N; k++) v += op.B[qb][k] * tf[(5 + c) * M * N + M * k];
                    qf[c / 3][c % 3] = v;
                }
                T n[3], mag;
                face_nrm<T, T>(a.fnrm, e, f, n, mag);
                T fvn[4];
                viscous_normal_flux(ph, uf, qf, n, fvn);
#pragma unroll
                for (int k = 0; k < 4; k++) a.FVQ[k * a.nqf + gq] = fvn[k];
            }
            __syncthreads();
        } else {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (int s = threadIdx.x; s < NF; s += NT) {
            const bool isL = (a.partner[gf0 + s] & FR_LFLAG) != 0;
            const T wgt = isL ? T(0.5) + ph.beta : T(0.5) - ph.beta;
            if (wgt == T(0)) {
#pragma unroll
                for (int k = 0; k < 4; k++) a.FV[k * a.nfpt + gf0 + s] = T(0);
            } else {
                s_list[atomicAdd(&s_cnt, 1)] = (short)s;
            }
        }
        __syncthreads();
        const int nlist = s_cnt;
        for (int li = threadIdx.x; li < nlist; li += NT) {
            const int s = s_list[li];
            const int f = s / (N * N), loc = s % (N * N);
            int base, stride;
            face_line_p<N, XS, PS>(f, loc, base, stride);
            const T *l = (f & 1) ? op.lR : op.lL;
            T uf[5], qf[5][3];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                T v = T(0);
#pragma unroll
                for (int i = 0; i < N; i++) v += l[i] * s_u[alpha * FS + base + i * stride];
                uf[alpha] = v;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    T w = T(0);
#pragma unroll
                    for (int i = 0; i < N; i++) w += l[i] * s_q[(alpha * 3 + d) * FS + base + i * stride];
                    qf[alpha][d] = w;
                }
            }
            T n[3], mag;
            if constexpr (CURV) {   // the normal at this flux point
                const T *t = a.mfn + (e * NF + s) * 4;
                n[0] = t[0]; n[1] = t[1]; n[2] = t[2]; mag = t[3];
            } else {
                face_nrm<T, T>(a.fnrm, e, f, n, mag);
            }
            if constexpr (std::is_same<T, float>::value) {
                if (dev) { uf[0] += ph.rref; uf[4] += ph.eref; }
            }
            T fvn[4];
            viscous_normal_flux(ph, uf, qf, n, fvn);
#pragma unroll
            for (int k = 0; k < 4; k++) a.FV[k * a.nfpt + gf0 + s] = fvn[k];
        }
        }   // surface-flux anti-aliasing or not
        if constexpr (std::is_same<T, float>::value) {
            // low-Mach form: volume part of R~_rho in float-float (the mass flux rho v is a
            // polynomial of the solution space, so its L2 projection is itself: no quadrature points).
            // Curved elements: det J J^-1 varies over the element, so the mass flux takes the FP32
            // quadrature-point path with the other fluxes instead.
            if (dev && !CURV && !SURF) {
                const HexOpsFF &off = c_hexff[P - 2];
                const ff *cm = a.geo64[e].cm;   // det J J^-1, per element
                // the transformed mass flux (3 NU float-float values) over the common solution
                // (5 NF values), consumed by the gradient step
                static_assert(3 * NU * sizeof(ff) <= 5 * NF * sizeof(T), "mass flux over s_c");
                ff *s_mf = reinterpret_cast<ff *>(s_c);
                // the upper half of the CTA takes the solution points first: the lower half is still
                // on the viscous flux of the flux-point list (at most 96 points), so the two overlap
                const int tr = (threadIdx.x + NT / 2) % NT;
                for (int it = tr; it < NU; it += NT) {
                    const int pz = it % N + XS * ((it / N) % N) + PS * (it / (N * N));
                    const float m0 = s_u[FS + pz], m1 = s_u[2 * FS + pz], m2 = s_u[3 * FS + pz];
                    if (diagJ) {
                        s_mf[it] = ff_mul_f(cm[0], m0);
                        s_mf[NU + it] = ff_mul_f(cm[4], m1);
                        s_mf[2 * NU + it] = ff_mul_f(cm[8], m2);
                    } else {
#pragma unroll
                        for (int d = 0; d < 3; d++)
                            s_mf[d * NU + it] = ff_add(ff_add(ff_mul_f(cm[3 * d], m0), ff_mul_f(cm[3 * d + 1], m1)), ff_mul_f(cm[3 * d + 2], m2));
                    }
                }
                __syncthreads();
                const long long pbase = elem_u0(a, e, NU) / FR_NV;
                for (int z = tr; z < NU; z += NT) {
                    const int i = z % N, j = (z / N) % N, k = z / (N * N);
                    float sh = 0.0f, c = 0.0f;   // compensated dot product (Dot2)
#pragma unroll
                    for (int b = 0; b < N; b++) {
                        dot2ff_next(off.Dh[i][b], s_mf[b + N * j + N * N * k], sh, c);
                        dot2ff_next(off.Dh[j][b], s_mf[NU + i + N * b + N * N * k], sh, c);
                        dot2ff_next(off.Dh[k][b], s_mf[2 * NU + i + N * j + N * N * b], sh, c);
                    }
                    a.RL[pbase + z] = two_sum(sh, c);
                }
            }
        }
        // 6. uqpts + gradcoru_qpts: 20 fields to quadrature points, 5 at a time
        if constexpr (!AA) {
            // collocation form: the flux is evaluated at the solution points (step 7b below)
        } else if constexpr (TCM == 0) {
            interp_all<T, P, NT, XS, PS, FS>(op, s_u, s_u, s_w);   // s_q follows s_u; staged over them
        } else {
            // z factor on the CUDA cores: row r = f M + c holds field f (s_q follows s_u) at z
            // quadrature level c on the N^2 in-plane points
            T *s_tt = s_t1;
            for (int it = threadIdx.x; it < TC::RI * TC::N2; it += NT) {
                const int r = it / TC::N2, n = it % TC::N2, f = r / M, c = r % M;
                const T *src = s_u + f * FS + n % N + XS * (n / N);
                T v = T(0);
#pragma unroll
                for (int k = 0; k < N; k++) v += op.B[c][k] * src[PS * k];
                s_tt[r * TC::ST + n] = v;
            }
            __syncthreads();
            if (threadIdx.x < TC::RI) {
                const int r = threadIdx.x;
                float x[TC::N2];
#pragma unroll
                for (int n = 0; n < TC::N2; n++) x[n] = s_tt[r * TC::ST + n];
                s_sh[r] = split_store_row<TCM, TC::KI, TC::N2>(tA, r, x);
            }
            if (!tc::mma_chain<TC::KI / 16>(tmem, tA, TC::SBO_I, tBi, TC::SBO_I, tc::idesc_f16(TCM - 1, 128, TC::NI), s_mbar, parity,
                                            tc::first_limit(first_wait, a.dbg_wait0))) {
                tc_fail = true;
                break;
            }
            {
                const int r = threadIdx.x;
                const uint32_t ta = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16);
                float v[TC::NI];
#pragma unroll
                for (int cb = 0; cb < TC::NI / 16; cb++) {
                    float w[16];
                    tc::ld16(ta + 16 * cb, w);
#pragma unroll
                    for (int q = 0; q < 16; q++) v[16 * cb + q] = w[q];
                }
                if (r < TC::RI) {
                    const float isc = tc::pow2f(-s_sh[r]);
#pragma unroll
                    for (int q = 0; q < TC::M2; q++) s_w[TC::M2 * r + q] = v[q] * isc;   // f NQ + M^2 c = M^2 r
                }
            }
            __syncthreads();
        }
        // 7. tdisf: transformed flux at each quadrature point, in place
        bool ok = true;
        if constexpr (!AA) {
            // 7b. collocation form: flux at the solution points from s_u and the gradient in s_q,
            //     written over the gradient (the projection is the identity) once every thread is
            //     done reading the gradient at the flux points
            __syncthreads();
            for (int z = threadIdx.x; z < NU; z += NT) {
                const int pz = z % N + XS * ((z / N) % N) + PS * (z / (N * N));
                T u[5], gq[5][3], f[3][5];
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    u[alpha] = s_u[alpha * FS + pz];
#pragma unroll
                    for (int d = 0; d < 3; d++) gq[alpha][d] = s_q[(alpha * 3 + d) * FS + pz];
                }
                if constexpr (std::is_same<T, float>::value) {
                    if (dev) ok &= total_flux_dev(ph, u, gq, f);
                    else ok &= total_flux(ph, u, gq, f);
                } else {
                    ok &= total_flux(ph, u, gq, f);
                }
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++)
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        s_q[(alpha * 3 + d) * FS + pz] =
                            g.det * (g.Ji[3 * d] * f[0][alpha] + g.Ji[3 * d + 1] * f[1][alpha] + g.Ji[3 * d + 2] * f[2][alpha]);
            }
        }
        for (int q = threadIdx.x; AA && q < NQ; q += NT) {
            T u[5], gq[5][3], f[3][5];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                u[alpha] = s_w[alpha * NQ + q];
#pragma unroll
                for (int d = 0; d < 3; d++) gq[alpha][d] = s_w[(5 + alpha * 3 + d) * NQ + q];
            }
            if constexpr (std::is_same<T, float>::value) {
                if (dev) ok &= total_flux_dev(ph, u, gq, f, CURV || SURF);
                else ok &= total_flux(ph, u, gq, f);
            } else {
                ok &= total_flux(ph, u, gq, f);
            }
            if constexpr (CURV) {   // det J J^-1 at this quadrature point
                const T *c = a.mq + (e * NQ + q) * 9;
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++)
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        s_w[(alpha * 3 + d) * NQ + q] = c[3 * d] * f[0][alpha] + c[3 * d + 1] * f[1][alpha] + c[3 * d + 2] * f[2][alpha];
            } else if (diagJ) {
                const T s0 = g.det * g.Ji[0], s1 = g.det * g.Ji[4], s2 = g.det * g.Ji[8];
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    s_w[(alpha * 3 + 0) * NQ + q] = s0 * f[0][alpha];
                    s_w[(alpha * 3 + 1) * NQ + q] = s1 * f[1][alpha];
                    s_w[(alpha * 3 + 2) * NQ + q] = s2 * f[2][alpha];
                }
            } else {
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++)
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        s_w[(alpha * 3 + d) * NQ + q] = g.det * (g.Ji[3 * d] * f[0][alpha] + g.Ji[3 * d + 1] * f[1][alpha] + g.Ji[3 * d + 2] * f[2][alpha]);
            }
        }
        flag_status(a.status, ok);
        __syncthreads();
        // 8. tdivtpcorf, first factor: projection of the 15 transformed-flux fields (into s_q);
        //    on the CUDA-core paths the corrected divergence (step 9) is folded into it
        T *R = a.R + elem_u0(a, e, NU);
        if constexpr (!AA) {
            // collocation form: the flux already sits at the solution points
        } else if constexpr (TCM == 0) {
            project_div_all<T, P, NT>(op, s_w, s_u, R);   // staged over s_u, s_q, s_c
        } else {
            // x-y factor on the tensor cores: row r = f M + c holds flux component f at quadrature
            // level c on the M^2 in-plane points; then the z factor on the CUDA cores
            T *s_tt = s_t1;
            if (threadIdx.x < TC::RP) {
                const int r = threadIdx.x;
                float x[TC::M2];
#pragma unroll
                for (int q = 0; q < TC::M2; q++) x[q] = s_w[TC::M2 * r + q];
                s_sh[r] = split_store_row<TCM, TC::KP, TC::M2>(tA, r, x);
            }
            if (!tc::mma_chain<TC::KP / 16>(tmem, tA, TC::SBO_P, tBp, TC::SBO_P, tc::idesc_f16(TCM - 1, 128, TC::NP), s_mbar, parity,
                                            tc::first_limit(first_wait, a.dbg_wait0))) {
                tc_fail = true;
                break;
            }
            {
                const int r = threadIdx.x;
                const uint32_t ta = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16);
                float v[TC::NP];
#pragma unroll
                for (int cb = 0; cb < TC::NP / 16; cb++) {
                    float w[16];
                    tc::ld16(ta + 16 * cb, w);
#pragma unroll
                    for (int q = 0; q < 16; q++) v[16 * cb + q] = w[q];
                }
                if (r < TC::RP) {
                    const float isc = tc::pow2f(-s_sh[r]);
#pragma unroll
                    for (int n = 0; n < TC::N2; n++) s_tt[r * TC::ST + n] = v[n] * isc;
                }
            }
            __syncthreads();
            for (int it = threadIdx.x; it < 15 * NU; it += NT) {
                const int f = it / NU, z = it % NU, n = z % TC::N2, k = z / TC::N2;
                T v = T(0);
#pragma unroll
                for (int c = 0; c < M; c++) v += op.Pj[k][c] * s_tt[(f * M + c) * TC::ST + n];
                s_q[f * FS + n % N + XS * (n / N) + PS * k] = v;
            }
            __syncthreads();
        }
        // 9. tdivtpcorf, second factor: R~ = sum_d Dh_d F~_d, written to R (finished in phase C)
        for (int it = threadIdx.x; (!AA || TCM != 0) && it < 5 * NU; it += NT) {
            const int alpha = it / NU, z = it % NU, i = z % N, j = (z / N) % N, k = z / (N * N);
            const T *F = s_q + alpha * 3 * FS;
            T v = T(0);
#pragma unroll
            for (int b = 0; b < N; b++) {
                v += op.Dh[i][b] * F[b + XS * j + PS * k];
                v += op.Dh[j][b] * F[FS + i + XS * b + PS * k];
                v += op.Dh[k][b] * F[2 * FS + i + XS * j + PS * b];
            }
            R[it] = v;
        }
        __syncthreads();
    }
    if constexpr (TCM != 0) {
        // a chain that did not complete within the bound is reported; the tensor memory is released
        if (tc_fail && threadIdx.x == 0) atomicOr(a.status, 2);
        tc::teardown(s_mbar, parity, tc_fail, tmem, TC::COLS);
    }
}

// The FP32 affine p = 3 volume kernel is capped at 48 registers per thread: ten CTAs of 128 threads
// per SM (more warps to hide its shared-memory latency; an eleventh, which its shared memory would
// allow, needs 40 registers, spills and measured slower). A minimum of 0 CTAs leaves the register
// count to the compiler (an explicit 1 lets it take up to 255).
template <typename T, int P, int NT, int TCM, bool AA, bool SURF, bool CURV>
constexpr int fused_B_min_ctas()
{
    return (sizeof(T) == 4 && TCM == 0 && AA && !SURF && !CURV && P == 3) ? 10 * 128 / NT : 0;
}

template <typename T, int P, int NT, int TCM = 0, bool AA = true, bool SURF = false, bool CURV = false>
__global__ void __launch_bounds__(NT, (fused_B_min_ctas<T, P, NT, TCM, AA, SURF, CURV>())) k_fused_B(HexArgs<T> a)
{
    fused_B_body<T, P, NT, TCM, AA, SURF, CURV>(a, blockIdx.x, gridDim.x);
}

// FP32 with surface-flux anti-aliasing: registers capped so that 896 threads' worth of CTAs (seven
// of 128) stay resident, as many as its shared memory allows at 128 threads
template <int P, int NT>
__global__ void __launch_bounds__(NT, 896 / NT) k_fused_B_surf32(HexArgs<float> a)
{
    fused_B_body<float, P, NT, 0, true, true, false>(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------------------------
// Fused phase C: comm_flux + tdivtconf + negdivconf per element
// ---------------------------------------------------------------------------------------------
template <typename T, int P, int NT, bool CURV = false>
__device__ __forceinline__ void fused_C_body(const HexArgs<T> &a, long long first, long long stride)
{
    constexpr int N = P + 1, NU = N * N * N, NF = 6 * N * N;
    __shared__ T s_d[5 * NF];
    __shared__ ff s_dff[std::is_same<T, float>::value ? NF : 1];   // low-Mach form: transformed mass flux
    // the lift rows, read with each solution point's run-time (i, j, k), from shared memory: a
    // constant-memory load is serialised over the distinct addresses of a warp
    __shared__ T s_lift[2 * N];                                          // liftL | liftR
    __shared__ ff s_liftff[std::is_same<T, float>::value ? 2 * N : 1];
    {
        const HexOps<T> &op = OPS<T>(P - 2);
        for (int i = threadIdx.x; i < 2 * N; i += NT) {
            s_lift[i] = i < N ? op.liftL[i] : op.liftR[i - N];
            if constexpr (std::is_same<T, float>::value) s_liftff[i] = i < N ? c_hexff[P - 2].liftL[i] : c_hexff[P - 2].liftR[i - N];
        }
        __syncthreads();
    }
    const T *liftL = s_lift, *liftR = s_lift + N;
    for (long long e = first; e < a.ne; e += stride) {
        if (!fr_elem_ok(a, e, (P + 1) * (P + 1) * (P + 1), 6 * (P + 1) * (P + 1))) continue;
        const Geo<T> g = a.geo[e];
        const Phys<T> ph = elem_phys(a, e);
        bool dev = false;
        if constexpr (std::is_same<T, float>::value) dev = ph.dev != 0;
        const long long gf0 = elem_f0(a, e, NF);
        bool ok = true;
        for (int s = threadIdx.x; s < NF; s += NT) {
            const int f = s / (N * N);
            const uint32_t pc = a.partner[gf0 + s];
            const bool isL = (pc & FR_LFLAG) != 0;
            const long long og = gf0 + s, pg = fr_partner(a, pc, og);
            T uo[5], up[5], fvo[4], fvp[4];
#pragma unroll
            for (int k = 0; k < 5; k++) { uo[k] = a.UF[k * a.nfpt + og]; up[k] = a.UF[k * a.nfpt + pg]; }
#pragma unroll
            for (int k = 0; k < 4; k++) { fvo[k] = a.FV[k * a.nfpt + og]; fvp[k] = a.FV[k * a.nfpt + pg]; }
            T n[3], mag;
            if constexpr (CURV) {   // curved elements: the normal at this flux point
                const T *t = a.mfn + (e * NF + s) * 4;
                n[0] = t[0]; n[1] = t[1]; n[2] = t[2]; mag = t[3];
            } else {
                face_nrm<T, T>(a.fnrm, e, f, n, mag);
            }
            T nL[3] = {isL ? n[0] : -n[0], isL ? n[1] : -n[1], isL ? n[2] : -n[2]};
            T F[5];
            if constexpr (std::is_same<T, float>::value) {
                if (dev) {
                    float sw;
                    ok &= isL ? common_flux_dev(ph, uo, up, fvo, fvp, nL, F, sw) : common_flux_dev(ph, up, uo, fvp, fvo, nL, F, sw);
                    if constexpr (CURV) {
                        // curved elements: the mass equation runs through the FP32 flux path
                        F[0] = isL ? common_mass_flux_dev(ph, uo, up, nL, sw) : common_mass_flux_dev(ph, up, uo, nL, sw);
                    } else {
                        // mass flux in float-float: 1/2 (mL - mR) + (s/2 + tau)(rho_L - rho_R),
                        // mX = own-normal n.(rho v)
                        const ff mo = a.MF[og], mp = a.MF[pg];
                        const ff mL = isL ? mo : mp, mR = isL ? mp : mo;
                        const float rL = isL ? uo[0] : up[0], rR = isL ? up[0] : uo[0];
                        const ff Fr = ff_add(ff_mul_f(ff_sub(mL, mR), 0.5f), ff_mul_f(two_sum(rL, -rR), 0.5f * sw + ph.tau));
                        const ff mag = a.fnrm64[(e * 6 + f) * 4 + 3];
                        s_dff[s] = isL ? ff_mul(mag, Fr) : ff_neg(ff_mul(mag, Fr));
                    }
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
            for (int it = threadIdx.x; it < 5 * NU; it += NT) {
                const int alpha = it / NU, z = it % NU, i = z % N, j = (z / N) % N, k = z / (N * N);
                const T *D = s_d + alpha * NF;
                T v = R[it];
                v += liftL[i] * D[0 * N * N + j + N * k] + liftR[i] * D[1 * N * N + j + N * k];
                v += liftL[j] * D[2 * N * N + i + N * k] + liftR[j] * D[3 * N * N + i + N * k];
                v += liftL[k] * D[4 * N * N + i + N * j] + liftR[k] * D[5 * N * N + i + N * j];
                // curved elements: det J at this solution point
                const T sc = CURV ? T(-1) / a.mu[(e * NU + z) * 10 + 9] : idet;
                if (a.rkstage == 0) R[it] = v * sc;
                else rk_fold(a, elem_u0(a, e, NU) + it, v * sc);
            }
        } else if constexpr (std::is_same<T, float>::value && CURV) {
            // low-Mach form on curved elements: every variable in FP32, then R_E = R_(E - H0 rho) + H0 R_rho
            for (int z = threadIdx.x; z < NU; z += NT) {
                const int i = z % N, j = (z / N) % N, k = z / (N * N);
                const T sc = T(-1) / a.mu[(e * NU + z) * 10 + 9];
                float out[5];
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    const T *D = s_d + alpha * NF;
                    T v = R[alpha * NU + z];
                    v += liftL[i] * D[0 * N * N + j + N * k] + liftR[i] * D[1 * N * N + j + N * k];
                    v += liftL[j] * D[2 * N * N + i + N * k] + liftR[j] * D[3 * N * N + i + N * k];
                    v += liftL[k] * D[4 * N * N + i + N * j] + liftR[k] * D[5 * N * N + i + N * j];
                    out[alpha] = v * sc;
                }
                out[4] += ph.H0 * out[0];
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    if (a.rkstage == 0) R[alpha * NU + z] = out[alpha];
                    else rk_fold(a, elem_u0(a, e, NU) + alpha * NU + z, out[alpha]);
                }
            }
        } else if constexpr (std::is_same<T, float>::value) {
            // low-Mach form: R_rho in float-float, R_E = R_(E - H0 rho) + H0 R_rho
            const ff *fliftL = s_liftff, *fliftR = s_liftff + N;
            const ff idet64 = a.geo64[e].idet;
            const ff H0 = ph.H0ff;
            const long long pbase = elem_u0(a, e, NU) / FR_NV;
            for (int z = threadIdx.x; z < NU; z += NT) {
                const int i = z % N, j = (z / N) % N, k = z / (N * N);
                ff r = a.RL[pbase + z];
                r = ff_fma(fliftL[i], s_dff[0 * N * N + j + N * k], r);
                r = ff_fma(fliftR[i], s_dff[1 * N * N + j + N * k], r);
                r = ff_fma(fliftL[j], s_dff[2 * N * N + i + N * k], r);
                r = ff_fma(fliftR[j], s_dff[3 * N * N + i + N * k], r);
                r = ff_fma(fliftL[k], s_dff[4 * N * N + i + N * j], r);
                r = ff_fma(fliftR[k], s_dff[5 * N * N + i + N * j], r);
                const ff Rrho = ff_mul(r, idet64);
                float out[5];
                out[0] = Rrho.hi + Rrho.lo;
#pragma unroll
                for (int alpha = 1; alpha < 5; alpha++) {
                    const T *D = s_d + alpha * NF;
                    T v = R[alpha * NU + z];
                    v += liftL[i] * D[0 * N * N + j + N * k] + liftR[i] * D[1 * N * N + j + N * k];
                    v += liftL[j] * D[2 * N * N + i + N * k] + liftR[j] * D[3 * N * N + i + N * k];
                    v += liftL[k] * D[4 * N * N + i + N * j] + liftR[k] * D[5 * N * N + i + N * j];
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

// FP32: registers capped for 960 resident threads per SM (ten CTAs of 96, one thread per flux point
// of a p = 3 element): the kernel waits on its partner gathers, and more warps keep more of them in
// flight. FP64 (0): the compiler's own register count.
template <typename T, int P, int NT, bool CURV = false>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 960 / NT : 0) k_fused_C(HexArgs<T> a)
{
    fused_C_body<T, P, NT, CURV>(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------------------------
// Interface phase with surface-flux anti-aliasing, split like C1/C2: the common flux once per
// pair of face quadrature points, from its L point (list qlpts), written to both sides' slots of DQ
// with each side's |n_s| (k_surf_pair); then per element the face L2 projection of DQ to the n x n
// face points (Pj (x) Pj, which makes the DG lift of the quadrature-point data the n x n lift of the
// projected data), the lift and the scaling (k_surf_lift).
// ---------------------------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(128) k_surf_pair(HexArgs<T> a)
{
    constexpr int M = P + 2, NQF = 6 * M * M;
    bool ok = true;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < a.nqlpts; it += (long long)gridDim.x * blockDim.x) {
        const long long gl = a.qlpts[it];
        const long long gr = a.qpartner[gl] & ~FR_LFLAG;
        const long long eL = gl / NQF, eR = gr / NQF;
        const int fL = (int)(gl % NQF) / (M * M), fR = (int)(gr % NQF) / (M * M);
        const Phys<T> ph = elem_phys(a, eL);
        T uL[5], uR[5], fvL[4], fvR[4];
#pragma unroll
        for (int k = 0; k < 5; k++) { uL[k] = a.UFQ[k * a.nqf + gl]; uR[k] = a.UFQ[k * a.nqf + gr]; }
#pragma unroll
        for (int k = 0; k < 4; k++) { fvL[k] = a.FVQ[k * a.nqf + gl]; fvR[k] = a.FVQ[k * a.nqf + gr]; }
        T n[3], magL, nR[3], magR;
        face_nrm<T, T>(a.fnrm, eL, fL, n, magL);
        face_nrm<T, T>(a.fnrm, eR, fR, nR, magR);
        T F[5];
        bool dev = false;
        if constexpr (std::is_same<T, float>::value) dev = ph.dev != 0;
        if (dev) {
            if constexpr (std::is_same<T, float>::value) {
                // low-Mach form: deviation states, reduced energy; the mass in FP32 here
                float sw;
                ok &= common_flux_dev(ph, uL, uR, fvL, fvR, n, F, sw);
                F[0] = common_mass_flux_dev(ph, uL, uR, n, sw);
            }
        } else {
            ok &= common_flux(ph, uL, uR, fvL, fvR, n, F);
        }
#pragma unroll
        for (int k = 0; k < 5; k++) {
            a.DQ[k * a.nqf + gl] = magL * F[k];
            a.DQ[k * a.nqf + gr] = -magR * F[k];
        }
    }
    flag_status(a.status, ok);
}

template <typename T, int P, int NT>
__global__ void __launch_bounds__(NT) k_surf_lift(HexArgs<T> a)
{
    constexpr int N = P + 1, M = P + 2, NU = N * N * N, NF = 6 * N * N, NQF = 6 * M * M;
    __shared__ T s_dq[5 * NQF];
    __shared__ T s_t[5 * 6 * N * M];
    __shared__ T s_d[5 * NF];
    const HexOps<T> &op = OPS<T>(P - 2);
    for (long long e = blockIdx.x; e < a.ne; e += gridDim.x) {
        if (!fr_elem_ok(a, e, (P + 1) * (P + 1) * (P + 1), 6 * (P + 1) * (P + 1))) continue;
        const Geo<T> g = a.geo[e];
        for (int it = threadIdx.x; it < 5 * NQF; it += NT) {
            const int alpha = it / NQF, s = it % NQF;
            s_dq[it] = a.DQ[alpha * a.nqf + e * NQF + s];
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 5 * 6 * N * M; it += NT) {   // (alpha, face, i, b): along a
            const int af = it / (N * M), r = it % (N * M), i = r % N, b = r / N;
            const T *D = s_dq + af * M * M + M * b;
            T v = T(0);
#pragma unroll
            for (int qa = 0; qa < M; qa++) v += op.Pj[i][qa] * D[qa];
            s_t[it] = v;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 5 * NF; it += NT) {   // (alpha, face, i + N j): along b
            const int af = it / (N * N), loc = it % (N * N), i = loc % N, j = loc / N;
            const T *t = s_t + af * N * M + i;
            T v = T(0);
#pragma unroll
            for (int b = 0; b < M; b++) v += op.Pj[j][b] * t[N * b];
            s_d[it] = v;
        }
        __syncthreads();
        T *R = a.R + elem_u0(a, e, NU);
        const T idet = g.nidet;
        bool dev = false;
        if constexpr (std::is_same<T, float>::value) dev = elem_phys(a, e).dev != 0;
        if (!dev) {
            for (int it = threadIdx.x; it < 5 * NU; it += NT) {
                const int alpha = it / NU, z = it % NU, i = z % N, j = (z / N) % N, k = z / (N * N);
                const T *D = s_d + alpha * NF;
                T v = R[it];
                v += op.liftL[i] * D[0 * N * N + j + N * k] + op.liftR[i] * D[1 * N * N + j + N * k];
                v += op.liftL[j] * D[2 * N * N + i + N * k] + op.liftR[j] * D[3 * N * N + i + N * k];
                v += op.liftL[k] * D[4 * N * N + i + N * j] + op.liftR[k] * D[5 * N * N + i + N * j];
                if (a.rkstage == 0) R[it] = v * idet;
                else rk_fold(a, elem_u0(a, e, NU) + it, v * idet);
            }
        } else {
            // low-Mach form: every variable in FP32, then R_E = R_(E - H0 rho) + H0 R_rho
            const T H0 = elem_phys(a, e).H0;
            for (int z = threadIdx.x; z < NU; z += NT) {
                const int i = z % N, j = (z / N) % N, k = z / (N * N);
                T out[5];
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    const T *D = s_d + alpha * NF;
                    T v = R[alpha * NU + z];
                    v += op.liftL[i] * D[0 * N * N + j + N * k] + op.liftR[i] * D[1 * N * N + j + N * k];
                    v += op.liftL[j] * D[2 * N * N + i + N * k] + op.liftR[j] * D[3 * N * N + i + N * k];
                    v += op.liftL[k] * D[4 * N * N + i + N * j] + op.liftR[k] * D[5 * N * N + i + N * j];
                    out[alpha] = v * idet;
                }
                out[4] += H0 * out[0];
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

// ---------------------------------------------------------------------------------------------
// Split interface phase: C1 common flux once per pair, C2 lift
// ---------------------------------------------------------------------------------------------
template <typename T, int P, bool CURV = false>
__global__ void __launch_bounds__(128) k_pair_flux(HexArgs<T> a)
{
    constexpr int N = P + 1, NF = 6 * N * N;
    bool ok = true;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < a.nlpts; it += (long long)gridDim.x * blockDim.x) {
        const uint32_t code = a.lpts[it];
        const long long e = code >> 8;
        const int s = code & 255, f = s / (N * N);
        const long long gl = elem_f0(a, e, NF) + s;
        const long long gr = fr_partner(a, a.partner[gl], gl);
        const Phys<T> ph = elem_phys(a, e);
        T uL[5], uR[5], fvL[4], fvR[4];
#pragma unroll
        for (int k = 0; k < 5; k++) { uL[k] = a.UF[k * a.nfpt + gl]; uR[k] = a.UF[k * a.nfpt + gr]; }
#pragma unroll
        for (int k = 0; k < 4; k++) { fvL[k] = a.FV[k * a.nfpt + gl]; fvR[k] = a.FV[k * a.nfpt + gr]; }
        T n[3], mag;
        if constexpr (CURV) {   // curved elements: the normal at this flux point
            const T *t = a.mfn + (e * NF + s) * 4;
            n[0] = t[0]; n[1] = t[1]; n[2] = t[2]; mag = t[3];
        } else {
            face_nrm<T, T>(a.fnrm, e, f, n, mag);
        }
        T F[5];
        ok &= common_flux(ph, uL, uR, fvL, fvR, n, F);
#pragma unroll
        for (int k = 0; k < 5; k++) a.DF[k * a.nfpt + gl] = F[k];
    }
    flag_status(a.status, ok);
}

template <typename T, int P, int NT, bool CURV = false>
__global__ void __launch_bounds__(NT) k_lift(HexArgs<T> a)
{
    constexpr int N = P + 1, NU = N * N * N, NF = 6 * N * N;
    __shared__ T s_d[5 * NF];
    __shared__ T s_lift[2 * N];   // liftL | liftR, read with run-time (i, j, k)
    {
        const HexOps<T> &op = OPS<T>(P - 2);
        for (int i = threadIdx.x; i < 2 * N; i += NT) s_lift[i] = i < N ? op.liftL[i] : op.liftR[i - N];
        __syncthreads();
    }
    const T *liftL = s_lift, *liftR = s_lift + N;
    for (long long e = blockIdx.x; e < a.ne; e += gridDim.x) {
        if (!fr_elem_ok(a, e, (P + 1) * (P + 1) * (P + 1), 6 * (P + 1) * (P + 1))) continue;
        const Geo<T> g = a.geo[e];
        const long long gf0 = elem_f0(a, e, NF);
        for (int s = threadIdx.x; s < NF; s += NT) {
            const uint32_t pc = a.partner[gf0 + s];
            const bool isL = (pc & FR_LFLAG) != 0;
            const long long src = isL ? gf0 + s : fr_partner(a, pc, gf0 + s);
            const T mag = CURV ? a.mfn[(e * NF + s) * 4 + 3] : a.fnrm[(e * 6 + s / (N * N)) * 4 + 3];
            const T sc = isL ? mag : -mag;
#pragma unroll
            for (int k = 0; k < 5; k++) s_d[k * NF + s] = sc * a.DF[k * a.nfpt + src];
        }
        __syncthreads();
        T *R = a.R + elem_u0(a, e, NU);
        const T idet = g.nidet;
        for (int it = threadIdx.x; it < 5 * NU; it += NT) {
            const int alpha = it / NU, z = it % NU, i = z % N, j = (z / N) % N, k = z / (N * N);
            const T *D = s_d + alpha * NF;
            T v = R[it];
            v += liftL[i] * D[0 * N * N + j + N * k] + liftR[i] * D[1 * N * N + j + N * k];
            v += liftL[j] * D[2 * N * N + i + N * k] + liftR[j] * D[3 * N * N + i + N * k];
            v += liftL[k] * D[4 * N * N + i + N * j] + liftR[k] * D[5 * N * N + i + N * j];
            // curved elements: det J at this solution point
            const T sc = CURV ? T(-1) / a.mu[(e * NU + z) * 10 + 9] : idet;
            if (a.rkstage == 0) R[it] = v * sc;
            else rk_fold(a, elem_u0(a, e, NU) + it, v * sc);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Unfused kernels K2..K13 (global intermediates)
// ---------------------------------------------------------------------------------------------

// K2 con_u: each pair visited once (from its L point); the common value is written to both points.
template <typename T, int P>
__global__ void __launch_bounds__(256) k_con_u(HexArgs<T> a)
{
    constexpr int N = P + 1, NF = 6 * N * N;
    const long long total = a.ne * NF;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const long long gl = a.f0 + it;
        const uint32_t pc = a.partner[gl];
        if (!(pc & FR_LFLAG)) continue;
        const long long gr = fr_partner(a, pc, gl);
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const T c = (T(0.5) - a.ph.beta) * a.UF[k * a.nfpt + gl] + (T(0.5) + a.ph.beta) * a.UF[k * a.nfpt + gr];
            a.CF[k * a.nfpt + gl] = c;
            a.CF[k * a.nfpt + gr] = c;
        }
    }
}

// K3 tgradpcoru (mode 0): Q~ = (M4 - M6 M0) U;  K4 tgradcoru (mode 1): Q~ += M6 C.
template <typename T, int P, int MODE>
__global__ void __launch_bounds__(256) k_tgrad(HexArgs<T> a)
{
    constexpr int N = P + 1, NU = N * N * N, NF = 6 * N * N;
    const HexOps<T> &op = OPS<T>(P - 2);
    const long long total = a.ne * 15 * N * N;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const long long e = it / (15 * N * N);
        const int r = (int)(it % (15 * N * N)), alpha = r / (3 * N * N), d = (r / (N * N)) % 3, loc = r % (N * N);
        int base, stride;
        face_line<N>(2 * d, loc, base, stride);
        T *q = a.Qu + ((e * 5 + alpha) * 3 + d) * NU + base;
        if (MODE == 0) {
            const T *u = a.U + a.u0 + (e * 5 + alpha) * NU + base;
            T uu[N];
#pragma unroll
            for (int i = 0; i < N; i++) uu[i] = u[i * stride];
#pragma unroll
            for (int i = 0; i < N; i++) {
                T v = T(0);
#pragma unroll
                for (int j = 0; j < N; j++) v += op.Dh[i][j] * uu[j];
                q[i * stride] = v;
            }
        } else {
            const long long g0 = a.f0 + e * NF;
            const T cL = a.CF[alpha * a.nfpt + g0 + (2 * d) * N * N + loc];
            const T cR = a.CF[alpha * a.nfpt + g0 + (2 * d + 1) * N * N + loc];
#pragma unroll
            for (int i = 0; i < N; i++) q[i * stride] += op.liftR[i] * cR - op.liftL[i] * cL;
        }
    }
}

// K5 gradcoru: q = J^-T q~
template <typename T, int P>
__global__ void __launch_bounds__(256) k_gradcoru(HexArgs<T> a)
{
    constexpr int N = P + 1, NU = N * N * N;
    const long long total = a.ne * 5 * NU;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const long long e = it / (5 * NU);
        const int r = (int)(it % (5 * NU)), alpha = r / NU, z = r % NU;
        // the element's metric, or (curved elements) the metric at this solution point
        const T *Ji = a.mu ? a.mu + (e * NU + z) * 10 : a.geo[e].Ji;
        T *q = a.Qu + (e * 5 + alpha) * 3 * NU + z;
        const T q0 = q[0], q1 = q[NU], q2 = q[2 * NU];
#pragma unroll
        for (int k = 0; k < 3; k++) q[k * NU] = Ji[k] * q0 + Ji[3 + k] * q1 + Ji[6 + k] * q2;
    }
}

// K6 gradcoru_fpts: Q^(f) = (I3 x M0) Q^(u)
template <typename T, int P>
__global__ void __launch_bounds__(256) k_gradcoru_fpts(HexArgs<T> a)
{
    constexpr int N = P + 1, NU = N * N * N, NF = 6 * N * N;
    const HexOps<T> &op = OPS<T>(P - 2);
    const long long total = a.ne * 15 * NF;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const long long e = it / (15 * NF);
        const int r = (int)(it % (15 * NF)), ad = r / NF, s = r % NF, f = s / (N * N);
        int base, stride;
        face_line<N>(f, s % (N * N), base, stride);
        const T *q = a.Qu + (e * 15 + ad) * NU + base;
        const T *l = (f & 1) ? op.lR : op.lL;
        T v = T(0);
#pragma unroll
        for (int i = 0; i < N; i++) v += l[i] * q[i * stride];
        a.QF[ad * a.nfpt + a.f0 + e * NF + s] = v;
    }
}

// K7 gradcoru_qpts (15 fields, Qu -> QQ) and K8 uqpts (5 fields, U -> UQ); one CTA per element.
template <typename T, int P, int NT, int NFLD>
__global__ void __launch_bounds__(NT) k_qpts(HexArgs<T> a)
{
    constexpr int N = P + 1, M = P + 2, NU = N * N * N, NQ = M * M * M;
    __shared__ T s_src[5 * NU], s_t1[5 * M * N * N], s_t2[5 * M * M * N], s_dst[5 * NQ];
    const HexOps<T> &op = OPS<T>(P - 2);
    for (long long e = blockIdx.x; e < a.ne; e += gridDim.x) {
        if (!fr_elem_ok(a, e, (P + 1) * (P + 1) * (P + 1), 6 * (P + 1) * (P + 1))) continue;
        for (int c = 0; c < NFLD / 5; c++) {
            const T *src = (NFLD == 5) ? a.U + a.u0 + e * 5 * NU : a.Qu + (e * 15 + 5 * c) * NU;
            T *dst = (NFLD == 5) ? a.UQ + e * 5 * NQ : a.QQ + (e * 15 + 5 * c) * NQ;
            for (int it = threadIdx.x; it < 5 * NU; it += NT) s_src[it] = src[it];
            __syncthreads();
            interp_5<T, P, NT>(op, s_src, s_t1, s_t2, s_dst);
            for (int it = threadIdx.x; it < 5 * NQ; it += NT) dst[it] = s_dst[it];
            __syncthreads();
        }
    }
}

// K9 tdisf: QQ <- detJ J^-1 f(UQ, QQ), in place
template <typename T, int P>
__global__ void __launch_bounds__(128) k_tdisf(HexArgs<T> a)
{
    constexpr int M = P + 2, NQ = M * M * M;
    const long long total = a.ne * NQ;
    bool ok = true;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const long long e = it / NQ;
        const int q = (int)(it % NQ);
        const Geo<T> &g = a.geo[e];
        T u[5], gq[5][3], f[3][5];
        T *Q = a.QQ + e * 15 * NQ + q;
#pragma unroll
        for (int alpha = 0; alpha < 5; alpha++) {
            u[alpha] = a.UQ[(e * 5 + alpha) * NQ + q];
#pragma unroll
            for (int d = 0; d < 3; d++) gq[alpha][d] = Q[(alpha * 3 + d) * NQ];
        }
        ok &= total_flux(a.ph, u, gq, f);
        if (a.mq) {   // curved elements: det J J^-1 at this quadrature point
            const T *c = a.mq + (e * NQ + q) * 9;
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++)
#pragma unroll
                for (int d = 0; d < 3; d++)
                    Q[(alpha * 3 + d) * NQ] = c[3 * d] * f[0][alpha] + c[3 * d + 1] * f[1][alpha] + c[3 * d + 2] * f[2][alpha];
        } else {
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++)
#pragma unroll
                for (int d = 0; d < 3; d++)
                    Q[(alpha * 3 + d) * NQ] = g.det * (g.Ji[3 * d] * f[0][alpha] + g.Ji[3 * d + 1] * f[1][alpha] + g.Ji[3 * d + 2] * f[2][alpha]);
        }
    }
    flag_status(a.status, ok);
}

// K10 tdivtpcorf: F~u = M9 F~q (written to Qu), R~ = (M1 - M3 M2) F~u (written to Rt)
template <typename T, int P, int NT>
__global__ void __launch_bounds__(NT) k_tdivtpcorf(HexArgs<T> a)
{
    constexpr int N = P + 1, M = P + 2, NU = N * N * N, NQ = M * M * M;
    __shared__ T s_src[5 * NQ], s_t1[5 * M * N * N], s_t2[5 * M * M * N], s_F[15 * NU];
    const HexOps<T> &op = OPS<T>(P - 2);
    for (long long e = blockIdx.x; e < a.ne; e += gridDim.x) {
        if (!fr_elem_ok(a, e, (P + 1) * (P + 1) * (P + 1), 6 * (P + 1) * (P + 1))) continue;
        for (int c = 0; c < 3; c++) {
            const T *src = a.QQ + (e * 15 + 5 * c) * NQ;
            for (int it = threadIdx.x; it < 5 * NQ; it += NT) s_src[it] = src[it];
            __syncthreads();
            project_5<T, P, NT>(op, s_src, s_t1, s_t2, s_F + 5 * c * NU);
        }
        for (int it = threadIdx.x; it < 15 * NU; it += NT) a.Qu[e * 15 * NU + it] = s_F[it];
        for (int it = threadIdx.x; it < 5 * NU; it += NT) {
            const int alpha = it / NU, z = it % NU, i = z % N, j = (z / N) % N, k = z / (N * N);
            const T *F = s_F + alpha * 3 * NU;
            T v = T(0);
#pragma unroll
            for (int b = 0; b < N; b++) {
                v += op.Dh[i][b] * F[b + N * j + N * N * k];
                v += op.Dh[j][b] * F[NU + i + N * b + N * N * k];
                v += op.Dh[k][b] * F[2 * NU + i + N * j + N * N * b];
            }
            a.Rt[e * 5 * NU + it] = v;
        }
        __syncthreads();
    }
}

// K11 comm_flux: per pair (from its L point), D~_L = |n_sL| F, D~_R = -|n_sR| F
template <typename T, int P>
__global__ void __launch_bounds__(128) k_comm_flux(HexArgs<T> a)
{
    constexpr int N = P + 1, NF = 6 * N * N;
    const long long total = a.ne * NF;
    bool ok = true;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const long long gl = a.f0 + it;
        const uint32_t pc = a.partner[gl];
        if (!(pc & FR_LFLAG)) continue;
        const long long gr = fr_partner(a, pc, gl);
        const long long e = it / NF;
        const int f = (int)(it % NF) / (N * N);
        T uL[5], uR[5], qL[5][3], qR[5][3];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            uL[k] = a.UF[k * a.nfpt + gl]; uR[k] = a.UF[k * a.nfpt + gr];
#pragma unroll
            for (int d = 0; d < 3; d++) { qL[k][d] = a.QF[(k * 3 + d) * a.nfpt + gl]; qR[k][d] = a.QF[(k * 3 + d) * a.nfpt + gr]; }
        }
        T n[3], magL;
        // the R side's |n_s| comes from its own element (global flux point -> element of this handle's
        // hex blocks; the unfused form supports single-block hex meshes)
        const long long eR = (gr - a.f0) / NF;
        const int fR = (int)((gr - a.f0) % NF) / (N * N);
        T nR[3], magR;
        if (a.mfn) {   // curved elements: the normal at the flux point itself, from each side
            const T *tl = a.mfn + (gl - a.f0) * 4, *tr = a.mfn + (gr - a.f0) * 4;
            n[0] = tl[0]; n[1] = tl[1]; n[2] = tl[2]; magL = tl[3];
            nR[0] = tr[0]; nR[1] = tr[1]; nR[2] = tr[2]; magR = tr[3];
        } else {
            face_normal(a.geo[e], f, n, magL);
            face_normal(a.geo[eR], fR, nR, magR);
        }
        T fvL[4], fvR[4], mnR[3] = {-n[0], -n[1], -n[2]};
        viscous_normal_flux(a.ph, uL, qL, n, fvL);
        viscous_normal_flux(a.ph, uR, qR, mnR, fvR);
        T F[5];
        ok &= common_flux(a.ph, uL, uR, fvL, fvR, n, F);
#pragma unroll
        for (int k = 0; k < 5; k++) { a.DF[k * a.nfpt + gl] = magL * F[k]; a.DF[k * a.nfpt + gr] = -magR * F[k]; }
    }
    flag_status(a.status, ok);
}

// K12 tdivtconf (R~ += M3 D) and K13 negdivconf (R = -R~/detJ); MODE 0 = K12, 1 = K13
template <typename T, int P, int MODE>
__global__ void __launch_bounds__(256) k_tdivtconf(HexArgs<T> a)
{
    constexpr int N = P + 1, NU = N * N * N, NF = 6 * N * N;
    const HexOps<T> &op = OPS<T>(P - 2);
    const long long total = a.ne * 5 * NU;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
        const long long e = it / (5 * NU);
        const int r = (int)(it % (5 * NU)), alpha = r / NU, z = r % NU, i = z % N, j = (z / N) % N, k = z / (N * N);
        if (MODE == 0) {
            const T *D = a.DF + alpha * a.nfpt + a.f0 + e * NF;
            T v = a.Rt[it];
            v += op.liftL[i] * D[0 * N * N + j + N * k] + op.liftR[i] * D[1 * N * N + j + N * k];
            v += op.liftL[j] * D[2 * N * N + i + N * k] + op.liftR[j] * D[3 * N * N + i + N * k];
            v += op.liftL[k] * D[4 * N * N + i + N * j] + op.liftR[k] * D[5 * N * N + i + N * j];
            a.Rt[it] = v;
        } else {
            a.R[a.u0 + it] = -a.Rt[it] / (a.mu ? a.mu[(e * NU + z) * 10 + 9] : a.geo[e].det);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// FP32 volume group, p = 3, several elements per CTA with register-resident line sweeps
//
// The same computation as k_fused_B<float, 3, ...> (flux anti-aliasing, affine elements, CUDA
// cores), organised for the FP32 pipe: a CTA takes EPB elements at a time, and every sum-factorised
// operator is applied by one thread to one whole field of one element from registers -- the
// interpolation of field f (4^3 -> 5^3: x and y sweeps plane by plane, then z) and the projection
// of transformed-flux component (alpha, d) (5^3 -> 4^3: first along d with the corrected derivative
// folded in, Dh Pj, then along the other two directions with Pj; the 1D factors of the tensor
// product commute). Every thread of a warp then applies the same operator entry at the same time, so
// the coefficients are uniform constant-memory operands; shared memory only carries the
// transpositions between a field-per-thread and a point-per-thread view (the pointwise flux), and
// a CTA crosses about eleven barriers per EPB elements instead of about twenty per element.
// Per element the shared workspace is one region of 2580 floats: the state and gradient (20 fields
// at stride 65), the common solution, then the 20 fields at the 125 quadrature points (stride 129),
// then the projected components; field strides of 1 modulo 32 keep a warp's (element, field)
// threads on distinct banks.
// ---------------------------------------------------------------------------------------------
namespace b32 {
constexpr int N = 4, M = 5, NU = 64, NF = 96, NQ = 125;
constexpr int FS = 65;      // field stride of the solution-point fields
constexpr int QS = 129;     // field stride of the quadrature-point fields
constexpr int CO = 20 * FS; // common solution C^(f): 5 x 96
constexpr int MO = CO + 5 * NF;   // low-Mach mass channel: 3 x 64 float-float values
constexpr int ES = 20 * QS; // element stride (2580 = 20 mod 32)
static_assert(MO + 3 * NU * 2 <= ES, "the mass channel fits below the quadrature-point fields' end");
}

// SPLIT: the interpolation of a field is shared by five threads (one per z quadrature level: the
// z sweep of that level, then its y and x sweeps) and the projection of a component by four (one
// per solution level along d), with the same multiply-adds in total and each operator row that
// differs between the threads held in registers.
template <int EPB, int NT, int MB, bool SPLIT = false>
__global__ void __launch_bounds__(NT, MB) k_hex_B32(HexArgs<float> a)
{
    using namespace b32;
    extern __shared__ __align__(16) float s_ws[];
    __shared__ Geo<float> s_geo[EPB];
    __shared__ Phys<float> s_ph[EPB];
    __shared__ long long s_u0[EPB], s_f0[EPB];
    __shared__ unsigned char s_diag[EPB];
    __shared__ short s_list[EPB * NF];
    __shared__ int s_cnt;
    const HexOps<float> &op = OPS<float>(1);
    const int tid = threadIdx.x;
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < a.ne; e0 += (long long)gridDim.x * EPB) {
        const int nb = (int)((a.ne - e0) < EPB ? (a.ne - e0) : EPB);
        {
            bool blk_ok = true;
            for (int k = 0; k < nb; k++) blk_ok = blk_ok && fr_elem_ok(a, e0 + k, NU, NF);
            if (!blk_ok) continue;
        }
        if (tid < nb) {
            const long long e = e0 + tid;
            const Geo<float> g = a.geo[e];
            s_geo[tid] = g;
            s_ph[tid] = elem_phys(a, e);
            s_u0[tid] = elem_u0(a, e, NU);
            s_f0[tid] = elem_f0(a, e, NF);
            s_diag[tid] = g.Ji[1] == 0.f && g.Ji[2] == 0.f && g.Ji[3] == 0.f && g.Ji[5] == 0.f && g.Ji[6] == 0.f &&
                          g.Ji[7] == 0.f;
        }
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        // 1. the state (deviations from the reference state in the low-Mach form), coalesced
        for (int i = tid; i < nb * 5 * NU; i += NT) {
            const int el = i / (5 * NU), r = i % (5 * NU), alpha = r / NU, z = r % NU;
            const Phys<float> &ph = s_ph[el];
            float v = a.U[s_u0[el] + r];
            if (ph.dev) v -= alpha == 0 ? ph.rref : (alpha == 4 ? ph.eref : 0.f);
            s_ws[el * ES + alpha * FS + z] = v;
        }
        // 2. con_u: common solution at the own flux points, (1/2 - beta) uL + (1/2 + beta) uR
        for (int i = tid; i < nb * 5 * NF; i += NT) {
            const int el = i / (5 * NF), r = i % (5 * NF), alpha = r / NF, s = r % NF;
            const long long gf = s_f0[el] + s;
            const uint32_t pc = a.partner[gf];
            const bool isL = (pc & FR_LFLAG) != 0;
            const float own = a.UF[alpha * a.nfpt + gf], oth = a.UF[alpha * a.nfpt + fr_partner(a, pc, gf)];
            const float beta = s_ph[el].beta;
            s_ws[el * ES + CO + r] = (0.5f - beta) * (isL ? own : oth) + (0.5f + beta) * (isL ? oth : own);
        }
        __syncthreads();
        // 3. corrected gradient along lines, q~ = Dh u + liftR C_R - liftL C_L, and J^-T on diagonal
        //    metrics (the other elements take the full J^-T in a pass of their own below)
        for (int i = tid; i < nb * 15 * N * N; i += NT) {
            const int el = i / (15 * N * N), r = i % (15 * N * N), alpha = r / (3 * N * N), r2 = r % (3 * N * N);
            const int d = r2 / (N * N), loc = r2 % (N * N);
            int base, stride;
            face_line<N>(2 * d, loc, base, stride);
            float *w = s_ws + el * ES;
            float u[N];
#pragma unroll
            for (int k = 0; k < N; k++) u[k] = w[alpha * FS + base + k * stride];
            const float cL = w[CO + alpha * NF + 2 * d * N * N + loc], cR = w[CO + alpha * NF + (2 * d + 1) * N * N + loc];
            const float sc = s_diag[el] ? s_geo[el].Ji[4 * d] : 1.f;
#pragma unroll
            for (int k = 0; k < N; k++) {
                float v = op.liftR[k] * cR - op.liftL[k] * cL;
#pragma unroll
                for (int j = 0; j < N; j++) v += op.Dh[k][j] * u[j];
                w[(5 + alpha * 3 + d) * FS + base + k * stride] = v * sc;
            }
        }
        if (__syncthreads_or(tid < nb && !s_diag[tid])) {
            for (int i = tid; i < nb * 5 * NU; i += NT) {
                const int el = i / (5 * NU), r = i % (5 * NU), alpha = r / NU, z = r % NU;
                if (s_diag[el]) continue;
                const float *Ji = s_geo[el].Ji;
                float *q = s_ws + el * ES + (5 + alpha * 3) * FS + z;
                const float q0 = q[0], q1 = q[FS], q2 = q[2 * FS];
#pragma unroll
                for (int k = 0; k < 3; k++) q[k * FS] = Ji[k] * q0 + Ji[3 + k] * q1 + Ji[6 + k] * q2;
            }
            __syncthreads();
        }
        // 4. own-normal viscous flux at the own flux points on the side whose LDG weight is not zero
        //    (compacted over the EPB elements so that whole warps work)
        for (int i = tid; i < nb * NF; i += NT) {
            const int el = i / NF, s = i % NF;
            const long long gf = s_f0[el] + s;
            const bool isL = (a.partner[gf] & FR_LFLAG) != 0;
            const float wgt = isL ? 0.5f + s_ph[el].beta : 0.5f - s_ph[el].beta;
            if (wgt == 0.f) {
#pragma unroll
                for (int k = 0; k < 4; k++) a.FV[k * a.nfpt + gf] = 0.f;
            } else {
                s_list[atomicAdd(&s_cnt, 1)] = (short)i;
            }
        }
        __syncthreads();
        const int nlist = s_cnt;
        for (int li = tid; li < nlist; li += NT) {
            const int i = s_list[li], el = i / NF, s = i % NF, f = s / (N * N);
            int base, stride;
            face_line<N>(f, s % (N * N), base, stride);
            const float *l = (f & 1) ? op.lR : op.lL;
            const float *w = s_ws + el * ES + base;
            float uf[5], qf[5][3];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                float v = 0.f;
#pragma unroll
                for (int k = 0; k < N; k++) v += l[k] * w[alpha * FS + k * stride];
                uf[alpha] = v;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    float x = 0.f;
#pragma unroll
                    for (int k = 0; k < N; k++) x += l[k] * w[(5 + alpha * 3 + d) * FS + k * stride];
                    qf[alpha][d] = x;
                }
            }
            const Phys<float> &ph = s_ph[el];
            if (ph.dev) { uf[0] += ph.rref; uf[4] += ph.eref; }
            float n[3], mag;
            face_nrm<float, float>(a.fnrm, e0 + el, f, n, mag);
            float fvn[4];
            viscous_normal_flux(ph, uf, qf, n, fvn);
            const long long gf = s_f0[el] + s;
#pragma unroll
            for (int k = 0; k < 4; k++) a.FV[k * a.nfpt + gf] = fvn[k];
        }
        // 5. low-Mach form: the volume part of R~_rho in float-float (rho v lies in the solution
        //    space: its L2 projection is itself), Dh applied along each direction at the solution points
        if (s_ph[0].dev) {
            const HexOpsFF &off = c_hexff[1];
            for (int i = tid; i < nb * NU; i += NT) {
                const int el = i / NU, z = i % NU;
                const ff *cm = a.geo64[e0 + el].cm;
                float *w = s_ws + el * ES;
                ff *mf = reinterpret_cast<ff *>(w + MO);
                const float m0 = w[FS + z], m1 = w[2 * FS + z], m2 = w[3 * FS + z];
                if (s_diag[el]) {
                    mf[z] = ff_mul_f(cm[0], m0);
                    mf[NU + z] = ff_mul_f(cm[4], m1);
                    mf[2 * NU + z] = ff_mul_f(cm[8], m2);
                } else {
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        mf[d * NU + z] = ff_add(ff_add(ff_mul_f(cm[3 * d], m0), ff_mul_f(cm[3 * d + 1], m1)), ff_mul_f(cm[3 * d + 2], m2));
                }
            }
            __syncthreads();
            for (int i = tid; i < nb * NU; i += NT) {
                const int el = i / NU, z = i % NU, x = z % N, y = (z / N) % N, k = z / (N * N);
                const ff *mf = reinterpret_cast<const ff *>(s_ws + el * ES + MO);
                float sh = 0.0f, c = 0.0f;   // compensated dot product (Dot2)
#pragma unroll
                for (int b = 0; b < N; b++) {
                    dot2ff_next(off.Dh[x][b], mf[b + N * y + N * N * k], sh, c);
                    dot2ff_next(off.Dh[y][b], mf[NU + x + N * b + N * N * k], sh, c);
                    dot2ff_next(off.Dh[k][b], mf[2 * NU + x + N * y + N * N * b], sh, c);
                }
                a.RL[s_u0[el] / FR_NV + z] = two_sum(sh, c);
            }
        }
        // 6. uqpts + gradcoru_qpts: one thread per (element, field) interpolates the field to the
        //    125 quadrature points from registers: the z sweep column by column (4 -> 5; every
        //    input read), then, once every thread has read its inputs, the y and x sweeps plane by
        //    plane straight into the quadrature-point layout over the consumed inputs
        if constexpr (SPLIT) {
            // x index i outermost: per i the z sweep of the x-line i at level qc, its y sweep, and
            // the x sweep accumulated into the level's 25 outputs (i ascending, as a dense sum)
            const bool itask = tid < nb * 5 * 20;
            const int iel = tid / 100, ifld = (tid % 100) / 5, qc = tid % 5;
            float out[M][M];   // [qa][qb]
#pragma unroll
            for (int qa = 0; qa < M; qa++)
#pragma unroll
                for (int qb = 0; qb < M; qb++) out[qa][qb] = 0.f;
            if (itask) {
                float bz[N];
#pragma unroll
                for (int k = 0; k < N; k++) bz[k] = op.B[qc][k];
                const float *w = s_ws + iel * ES + ifld * FS;
#pragma unroll 1
                for (int i = 0; i < N; i++) {
                    float zi[N];   // [j]
#pragma unroll
                    for (int j = 0; j < N; j++) {
                        float v = 0.f;
#pragma unroll
                        for (int k = 0; k < N; k++) v += bz[k] * w[i + N * j + N * N * k];
                        zi[j] = v;
                    }
#pragma unroll
                    for (int qb = 0; qb < M; qb++) {
                        float v = 0.f;
#pragma unroll
                        for (int j = 0; j < N; j++) v += op.B[qb][j] * zi[j];
#pragma unroll
                        for (int qa = 0; qa < M; qa++) out[qa][qb] += op.B[qa][i] * v;
                    }
                }
            }
            __syncthreads();
            if (itask) {
                float *w = s_ws + iel * ES + ifld * QS + M * M * qc;
#pragma unroll
                for (int qb = 0; qb < M; qb++)
#pragma unroll
                    for (int qa = 0; qa < M; qa++) w[qa + M * qb] = out[qa][qb];
            }
            __syncthreads();
        } else {
        float zt[N][N][M];   // [i][j][qc]
            const bool itask = tid < nb * 20;
            const int iel = tid / 20, ifld = tid % 20;
            if (itask) {
                const float *w = s_ws + iel * ES + ifld * FS;
    #pragma unroll
                for (int i = 0; i < N; i++)
    #pragma unroll
                    for (int j = 0; j < N; j++) {
                        float u[N];
    #pragma unroll
                        for (int k = 0; k < N; k++) u[k] = w[i + N * j + N * N * k];
    #pragma unroll
                        for (int qc = 0; qc < M; qc++) {
                            float v = 0.f;
    #pragma unroll
                            for (int k = 0; k < N; k++) v += op.B[qc][k] * u[k];
                            zt[i][j][qc] = v;
                        }
                    }
            }
            __syncthreads();
            if (itask) {
                float *w = s_ws + iel * ES + ifld * QS;
    #pragma unroll
                for (int qc = 0; qc < M; qc++) {
                    float yt[N][M];   // [i][qb]
    #pragma unroll
                    for (int i = 0; i < N; i++)
    #pragma unroll
                        for (int qb = 0; qb < M; qb++) {
                            float v = 0.f;
    #pragma unroll
                            for (int j = 0; j < N; j++) v += op.B[qb][j] * zt[i][j][qc];
                            yt[i][qb] = v;
                        }
    #pragma unroll
                    for (int qb = 0; qb < M; qb++)
    #pragma unroll
                        for (int qa = 0; qa < M; qa++) {
                            float v = 0.f;
    #pragma unroll
                            for (int i = 0; i < N; i++) v += op.B[qa][i] * yt[i][qb];
                            w[qa + M * qb + M * M * qc] = v;
                        }
                }
            }
            __syncthreads();
        }
        // 7. tdisf: transformed flux at each quadrature point, in place (fields alpha 3 + d)
        bool ok = true;
        for (int i = tid; i < nb * NQ; i += NT) {
            const int el = i / NQ, q = i % NQ;
            float *w = s_ws + el * ES + q;
            const Phys<float> &ph = s_ph[el];
            const Geo<float> &g = s_geo[el];
            float u[5], gq[5][3], f[3][5];
#pragma unroll
            for (int alpha = 0; alpha < 5; alpha++) {
                u[alpha] = w[alpha * QS];
#pragma unroll
                for (int d = 0; d < 3; d++) gq[alpha][d] = w[(5 + alpha * 3 + d) * QS];
            }
            if (ph.dev) ok &= total_flux_dev(ph, u, gq, f);
            else ok &= total_flux(ph, u, gq, f);
            if (s_diag[el]) {
                const float s0 = g.det * g.Ji[0], s1 = g.det * g.Ji[4], s2 = g.det * g.Ji[8];
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++) {
                    w[(alpha * 3 + 0) * QS] = s0 * f[0][alpha];
                    w[(alpha * 3 + 1) * QS] = s1 * f[1][alpha];
                    w[(alpha * 3 + 2) * QS] = s2 * f[2][alpha];
                }
            } else {
#pragma unroll
                for (int alpha = 0; alpha < 5; alpha++)
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        w[(alpha * 3 + d) * QS] = g.det * (g.Ji[3 * d] * f[0][alpha] + g.Ji[3 * d + 1] * f[1][alpha] + g.Ji[3 * d + 2] * f[2][alpha]);
            }
        }
        flag_status(a.status, ok);
        __syncthreads();
        // 8. tdivtpcorf: one thread per (element, alpha, d) projects component d of the flux of
        //    variable alpha, first along d with Dh Pj (projection and corrected derivative), then
        //    along the other two directions p < r with Pj, into solution-point component slots
        if constexpr (SPLIT) {
            // four threads per component: thread k2 produces the solution level k2 along d
            const bool ptask = tid < nb * 60;
            const int pel = tid / 60, pc = (tid % 60) / 4, k2 = tid % 4, pd = pc % 3;
            const int qd = pd == 0 ? 1 : (pd == 1 ? M : M * M), qp = pd == 0 ? M : 1, qr = pd == 2 ? M : M * M;
            const int zd = pd == 0 ? 1 : (pd == 1 ? N : N * N), zp = pd == 0 ? N : 1, zr = pd == 2 ? N : N * N;
            // r index outermost: per ir the d sweep of the slice, its p sweep, and the r sweep
            // accumulated into the 16 outputs (ir ascending, as a dense sum)
            float out[N][N];   // [jp][jr]
#pragma unroll
            for (int jp = 0; jp < N; jp++)
#pragma unroll
                for (int jr = 0; jr < N; jr++) out[jp][jr] = 0.f;
            if (ptask) {
                float dp[M];
#pragma unroll
                for (int m = 0; m < M; m++) dp[m] = op.DP[k2][m];
                const float *w = s_ws + pel * ES + pc * QS;
#pragma unroll 1
                for (int ir = 0; ir < M; ir++) {
                    const float *wr = w + ir * qr;
                    float pt[M];   // [ip]
#pragma unroll
                    for (int ip = 0; ip < M; ip++) {
                        float v = 0.f;
#pragma unroll
                        for (int m = 0; m < M; m++) v += dp[m] * wr[m * qd + ip * qp];
                        pt[ip] = v;
                    }
#pragma unroll
                    for (int jp = 0; jp < N; jp++) {
                        float v = 0.f;
#pragma unroll
                        for (int ip = 0; ip < M; ip++) v += op.Pj[jp][ip] * pt[ip];
#pragma unroll
                        for (int jr = 0; jr < N; jr++) out[jp][jr] += op.Pj[jr][ir] * v;
                    }
                }
            }
            __syncthreads();
            if (ptask) {
                float *w = s_ws + pel * ES + pc * FS + k2 * zd;
#pragma unroll
                for (int jp = 0; jp < N; jp++)
#pragma unroll
                    for (int jr = 0; jr < N; jr++) w[jp * zp + jr * zr] = out[jp][jr];
            }
            __syncthreads();
        } else {
        const bool ptask = tid < nb * 15;
            const int pel = tid / 15, pc = tid % 15, pd = pc % 3;
            // quadrature strides (1, M, M^2) and solution strides (1, N, N^2) of d, p and r
            const int qd = pd == 0 ? 1 : (pd == 1 ? M : M * M), qp = pd == 0 ? M : 1, qr = pd == 2 ? M : M * M;
            const int zd = pd == 0 ? 1 : (pd == 1 ? N : N * N), zp = pd == 0 ? N : 1, zr = pd == 2 ? N : N * N;
            // the r sweep accumulates slice by slice (ir ascending, as a dense sum would), so only the
            // 64 outputs, one slice and one column stay in registers
            float acc[N][N][N];   // [jp][jr][k along d]
    #pragma unroll
            for (int jp = 0; jp < N; jp++)
    #pragma unroll
                for (int jr = 0; jr < N; jr++)
    #pragma unroll
                    for (int k = 0; k < N; k++) acc[jp][jr][k] = 0.f;
            if (ptask) {
                const float *w = s_ws + pel * ES + pc * QS;
    #pragma unroll 1
                for (int ir = 0; ir < M; ir++) {
                    const float *wr = w + ir * qr;
                    float pt[M][N];   // [ip][k]
    #pragma unroll
                    for (int ip = 0; ip < M; ip++) {
                        float c[M];
    #pragma unroll
                        for (int m = 0; m < M; m++) c[m] = wr[m * qd + ip * qp];
    #pragma unroll
                        for (int k = 0; k < N; k++) {
                            float v = 0.f;
    #pragma unroll
                            for (int m = 0; m < M; m++) v += op.DP[k][m] * c[m];
                            pt[ip][k] = v;
                        }
                    }
    #pragma unroll
                    for (int jp = 0; jp < N; jp++)
    #pragma unroll
                        for (int k = 0; k < N; k++) {
                            float v = 0.f;
    #pragma unroll
                            for (int ip = 0; ip < M; ip++) v += op.Pj[jp][ip] * pt[ip][k];
    #pragma unroll
                            for (int jr = 0; jr < N; jr++) acc[jp][jr][k] += op.Pj[jr][ir] * v;
                        }
                }
            }
            __syncthreads();
            if (ptask) {
                float *w = s_ws + pel * ES + pc * FS;
    #pragma unroll
                for (int jp = 0; jp < N; jp++)
    #pragma unroll
                    for (int jr = 0; jr < N; jr++)
    #pragma unroll
                        for (int k = 0; k < N; k++) w[k * zd + jp * zp + jr * zr] = acc[jp][jr][k];
            }
            __syncthreads();
        }
        // 9. R~[alpha] = sum over d of the projected components, written to R (finished in phase C)
        for (int i = tid; i < nb * 5 * NU; i += NT) {
            const int el = i / (5 * NU), r = i % (5 * NU), alpha = r / NU, z = r % NU;
            const float *w = s_ws + el * ES + alpha * 3 * FS + z;
            a.R[s_u0[el] + r] = (w[0] + w[FS]) + w[2 * FS];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------------
static int grid_for(long long work, int threads)
{
    long long g = (work + threads - 1) / threads;
    if (g > fr_sms() * 64) g = fr_sms() * 64;
    return (int)(g < 1 ? 1 : g);
}

static int grid_elems(long long ne, int per_sm)
{
    long long g = ne;
    if (g > fr_sms() * per_sm * 8) g = fr_sms() * per_sm * 8;
    return (int)(g < 1 ? 1 : g);
}

template <typename T, int P, int NT, bool AA = true, bool SURF = false, bool CURV = false>
static void launch_B(const HexArgs<T> &a, cudaStream_t s)
{
    using S = HexSmem<T, P>;
    // the collocation form needs no quadrature-point buffers; surface-flux anti-aliasing stages its
    // in-plane interpolation (6 faces x 20 fields x m x n values) after the quadrature-point buffer
    constexpr int TI = 6 * 20 * S::M * S::N;
    const size_t smem = (!AA ? S::LOW + S::PF : (SURF ? S::SIZE + TI : S::SIZE)) * sizeof(T);
    static bool attr = false;
    if constexpr (SURF && sizeof(T) == 4) {
        if (!attr) {
            cudaFuncSetAttribute(k_fused_B_surf32<P, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_fused_B_surf32<P, NT><<<grid_elems(a.ne, 8), NT, smem, s>>>(a);
    } else {
        if (!attr) {
            cudaFuncSetAttribute(k_fused_B<T, P, NT, 0, AA, SURF, CURV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_fused_B<T, P, NT, 0, AA, SURF, CURV><<<grid_elems(a.ne, 8), NT, smem, s>>>(a);
    }
}

// Tensor-core form of the volume kernel (FP32, 128 threads, persistent: at most as many CTAs as
// fit on the SMs, each holding its tensor-memory columns for its lifetime).
template <int P, int TCM>
static int launch_B_tc(const HexArgs<float> &a, cudaStream_t s)
{
    using TC = HexTc<P, TCM>;
    static_assert(16 * (TC::SBO_I > TC::SBO_P ? TC::SBO_I : TC::SBO_P) <=
                      TC::A_BYTES + TC::BI_BYTES + TC::BP_BYTES + HexSmem<float, P>::SIZE * (int)sizeof(float),
                  "the 128 rows an MMA reads stay inside the CTA's shared memory");
    // the staged rows of the plane contractions sit after the quadrature-point buffer
    const size_t tt = (size_t)TC::TT;
    const size_t smem = TC::HEAD + (HexSmem<float, P>::SIZE + tt) * sizeof(float);
    static int occ = -1;
    if (occ < 0) {
        // resident CTAs per SM from the kernel's shared memory and registers (232,448 B of shared
        // memory and 64K registers per SM, 1 KB reserved per CTA); each CTA holds COLS of the 512
        // tensor-memory columns, which bounds the count too
        cudaFuncSetAttribute(k_fused_B<float, P, 128, TCM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, k_fused_B<float, P, 128, TCM>) != cudaSuccess) return -1;
        const int by_smem = (int)(232448 / (smem + fa.sharedSizeBytes + 1024));
        const int by_regs = 65536 / (((fa.numRegs + 7) / 8 * 8) * 128);
        int o = by_smem < by_regs ? by_smem : by_regs;
        if (o > 512 / TC::COLS) o = 512 / TC::COLS;
        if (o < 1) return -4;
        occ = o;
    }
    long long g = a.ne < fr_sms() * occ ? a.ne : fr_sms() * occ;
    k_fused_B<float, P, 128, TCM><<<(int)g, 128, smem, s>>>(a);
    return 0;
}

template <int EPB, int NT, int MB, bool SPLIT = false>
static int launch_B32(const HexArgs<float> &a, cudaStream_t s)
{
    const size_t smem = (size_t)EPB * b32::ES * sizeof(float);
    static int occ = -1, nsm = 0;
    if (occ < 0) {
        cudaFuncSetAttribute(k_hex_B32<EPB, NT, MB, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return -1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hex_B32<EPB, NT, MB, SPLIT>, NT, smem) != cudaSuccess || occ < 1)
            return -4;
    }
    long long g = (a.ne + EPB - 1) / EPB;   // persistent: at most the resident CTAs
    if (g > (long long)nsm * occ) g = (long long)nsm * occ;
    k_hex_B32<EPB, NT, MB, SPLIT><<<(int)g, NT, smem, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int P>
static int fused_phase(int phase, const HexArgs<T> &a, cudaStream_t s, int variant)
{
    if (a.ne == 0) return 0;
    if (phase == 0) {
        constexpr int EB = 8;
        long long g = (a.ne + EB - 1) / EB;
        if (g > fr_sms() * 16) g = fr_sms() * 16;
        k_disu_blk<T, P, EB, 256><<<(int)g, 256, 0, s>>>(a);
    } else if (phase == 1) {
        if constexpr (std::is_same<T, float>::value) {
            if (a.tcmode != 0) {
                const int r = a.tcmode == 1 ? launch_B_tc<P, 1>(a, s) : launch_B_tc<P, 2>(a, s);
                if (r) return r;
                return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
            }
        }
        if (a.mu) {   // curved elements: per-point metric terms (one launch shape)
            launch_B<T, P, 128, true, false, true>(a, s);
            return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
        }
        // launch shape chosen by the autotuner: 64, 128 or 256 threads per element
        if (a.surf) {
            if (variant == 0) launch_B<T, P, 64, true, true>(a, s);
            else if (variant == 2) launch_B<T, P, 256, true, true>(a, s);
            else launch_B<T, P, 128, true, true>(a, s);
            return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
        }
        if (a.aa_off) {
            if (variant == 0) launch_B<T, P, 64, false>(a, s);
            else if (variant == 2) launch_B<T, P, 256, false>(a, s);
            else launch_B<T, P, 128, false>(a, s);
            return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
        }
        if constexpr (std::is_same<T, float>::value && P == 3) {
            // several elements per CTA, register-resident line sweeps: 3 = one CTA of 8 elements
            // per SM (all 255 registers), 4 = two per SM (registers capped at 204)
            if (variant == 3) return launch_B32<8, 160, 1>(a, s);
            if (variant == 4) return launch_B32<8, 160, 2>(a, s);
            if (variant == 5) return launch_B32<2, 224, 3, true>(a, s);
        }
        if (variant == 0) launch_B<T, P, 64>(a, s);
        else if (variant == 2) launch_B<T, P, 256>(a, s);
        else launch_B<T, P, 128>(a, s);
    } else if (phase == 2) {
        if (a.mu) k_fused_C<T, P, 128, true><<<grid_elems(a.ne, 8), 128, 0, s>>>(a);
        else if (P == 3) k_fused_C<T, P, 96><<<grid_elems(a.ne, 10), 96, 0, s>>>(a);
        else k_fused_C<T, P, 128><<<grid_elems(a.ne, 8), 128, 0, s>>>(a);
    } else if (phase == 3) {
        if (a.surf) { if (a.nqlpts > 0) k_surf_pair<T, P><<<grid_for(a.nqlpts, 128), 128, 0, s>>>(a); }
        else if (a.nlpts > 0 && a.mu) k_pair_flux<T, P, true><<<grid_for(a.nlpts, 128), 128, 0, s>>>(a);
        else if (a.nlpts > 0) k_pair_flux<T, P><<<grid_for(a.nlpts, 128), 128, 0, s>>>(a);
    } else {
        if (a.surf) k_surf_lift<T, P, 128><<<grid_elems(a.ne, 8), 128, 0, s>>>(a);
        else if (a.mu) k_lift<T, P, 128, true><<<grid_elems(a.ne, 8), 128, 0, s>>>(a);
        else k_lift<T, P, 128><<<grid_elems(a.ne, 8), 128, 0, s>>>(a);
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------------------------
// One launch per phase over several element groups (hexahedra p = 3 / 4 and prisms, CUDA cores):
// every CTA runs each group's phase body on its share of that group's elements in turn. The
// dynamic shared memory is the largest group's; each body uses it from the start.
// ---------------------------------------------------------------------------------------------
int multi_set_pri_const_ops(const PriOps<float> *h) { return pri::set_const_ops(*h); }

template <typename T>
__global__ void __launch_bounds__(256) k_multi_A(MultiArgs<T> ma)
{
    for (int g = 0; g < ma.ng; g++) {
        if (ma.kind[g] == 3) disu_blk_body<T, 3, 8, 256>(ma.a[g], blockIdx.x, gridDim.x);
        else if (ma.kind[g] == 4) disu_blk_body<T, 4, 8, 256>(ma.a[g], blockIdx.x, gridDim.x);
        else pri::pri_disu_body<T>(ma.a[g], ma.pops, ma.pff, blockIdx.x, gridDim.x);
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_multi_B(MultiArgs<T> ma)
{
    for (int g = 0; g < ma.ng; g++) {
        if (ma.kind[g] == 3) fused_B_body<T, 3, 128>(ma.a[g], blockIdx.x, gridDim.x);
        else if (ma.kind[g] == 4) fused_B_body<T, 4, 128>(ma.a[g], blockIdx.x, gridDim.x);
        else pri::pri_B_body<T, 128, 0>(ma.a[g], ma.pops, ma.pff, blockIdx.x, gridDim.x);
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_multi_C(MultiArgs<T> ma)
{
    for (int g = 0; g < ma.ng; g++) {
        if (ma.kind[g] == 3) fused_C_body<T, 3, 128>(ma.a[g], blockIdx.x, gridDim.x);
        else if (ma.kind[g] == 4) fused_C_body<T, 4, 128>(ma.a[g], blockIdx.x, gridDim.x);
        else pri::pri_C_body<T, 128>(ma.a[g], ma.pops, ma.pff, blockIdx.x, gridDim.x);
        __syncthreads();
    }
}

// Dynamic shared memory of the volume bodies: a hexahedral group of order P, and the prism group
// (its operator table, the element arrays, the 20-field staging buffer of the FP32 interpolation).
template <typename T>
static size_t multi_B_smem(const MultiArgs<T> &ma)
{
    size_t need = 0;
    for (int g = 0; g < ma.ng; g++) {
        size_t v;
        if (ma.kind[g] == 3) v = HexSmem<T, 3>::SIZE * sizeof(T);
        else if (ma.kind[g] == 4) v = HexSmem<T, 4>::SIZE * sizeof(T);
        else v = ((sizeof(PriOps<T>) + 15) / 16) * 16 +
                 (size_t)(5 * pri::NU + 15 * pri::NU + 5 * pri::NF + 20 * pri::NQ) * sizeof(T) +
                 (size_t)((sizeof(T) == 4 ? 20 : 5) * pri::NZ * pri::NQT) * sizeof(T);
        need = v > need ? v : need;
    }
    return need;
}

template <typename T>
int multi_phase(int phase, const MultiArgs<T> &ma, cudaStream_t s)
{
    if (ma.ng < 1 || ma.ng > FR_MULTI_MAX) return -1;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    int occ = 0;
    if (phase == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_multi_A<T>, 256, 0) != cudaSuccess || occ < 1) return -4;
        k_multi_A<T><<<nsm * occ, 256, 0, s>>>(ma);
    } else if (phase == 1) {
        const size_t smem = multi_B_smem(ma);
        if (cudaFuncSetAttribute(k_multi_B<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_multi_B<T>, 128, smem) != cudaSuccess || occ < 1) return -4;
        k_multi_B<T><<<nsm * occ, 128, smem, s>>>(ma);
    } else {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_multi_C<T>, 128, 0) != cudaSuccess || occ < 1) return -4;
        k_multi_C<T><<<nsm * occ, 128, 0, s>>>(ma);
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template int multi_phase<double>(int, const MultiArgs<double> &, cudaStream_t);
template int multi_phase<float>(int, const MultiArgs<float> &, cudaStream_t);

template <typename T, int P>
static int unfused_kernel(int k, const HexArgs<T> &a, cudaStream_t s)
{
    constexpr int N = P + 1, NU = N * N * N, NF = 6 * N * N, NQ = (P + 2) * (P + 2) * (P + 2);
    if (a.ne == 0) return 0;
    switch (k) {
    case 1: k_disu<T, P><<<grid_for(a.ne * 5 * NF, 256), 256, 0, s>>>(a); break;
    case 2: k_con_u<T, P><<<grid_for(a.ne * NF, 256), 256, 0, s>>>(a); break;
    case 3: k_tgrad<T, P, 0><<<grid_for(a.ne * 15 * N * N, 256), 256, 0, s>>>(a); break;
    case 4: k_tgrad<T, P, 1><<<grid_for(a.ne * 15 * N * N, 256), 256, 0, s>>>(a); break;
    case 5: k_gradcoru<T, P><<<grid_for(a.ne * 5 * NU, 256), 256, 0, s>>>(a); break;
    case 6: k_gradcoru_fpts<T, P><<<grid_for(a.ne * 15 * NF, 256), 256, 0, s>>>(a); break;
    case 7: k_qpts<T, P, 128, 15><<<grid_elems(a.ne, 8), 128, 0, s>>>(a); break;
    case 8: k_qpts<T, P, 128, 5><<<grid_elems(a.ne, 8), 128, 0, s>>>(a); break;
    case 9: k_tdisf<T, P><<<grid_for(a.ne * NQ, 128), 128, 0, s>>>(a); break;
    case 10: k_tdivtpcorf<T, P, 128><<<grid_elems(a.ne, 8), 128, 0, s>>>(a); break;
    case 11: k_comm_flux<T, P><<<grid_for(a.ne * NF, 128), 128, 0, s>>>(a); break;
    case 12: k_tdivtconf<T, P, 0><<<grid_for(a.ne * 5 * NU, 256), 256, 0, s>>>(a); break;
    case 13: k_tdivtconf<T, P, 1><<<grid_for(a.ne * 5 * NU, 256), 256, 0, s>>>(a); break;
    default: return -2;
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename T>
int hex_fused_phase(int p, int phase, const HexArgs<T> &a, cudaStream_t s, int variant)
{
    switch (p) {
    case 3: return fused_phase<T, 3>(phase, a, s, variant);
    case 4: return fused_phase<T, 4>(phase, a, s, variant);
    default: return -3;
    }
}

template <typename T>
int hex_unfused_kernel(int p, int k, const HexArgs<T> &a, cudaStream_t s)
{
    switch (p) {
    case 3: return unfused_kernel<T, 3>(k, a, s);
    case 4: return unfused_kernel<T, 4>(k, a, s);
    default: return -3;
    }
}

template int hex_fused_phase<double>(int, int, const HexArgs<double> &, cudaStream_t, int);
template int hex_fused_phase<float>(int, int, const HexArgs<float> &, cudaStream_t, int);
template int hex_unfused_kernel<double>(int, int, const HexArgs<double> &, cudaStream_t);
template int hex_unfused_kernel<float>(int, int, const HexArgs<float> &, cudaStream_t);
