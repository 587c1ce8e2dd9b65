// fr_pri.cu -- prismatic kernels (p = 3) of the anti-aliased Navier-Stokes FR right-hand side.
//
// A prism is the tensor product of a triangle and a line (Sec. 4.1): every operator is a dense
// triangle-plane block (10 x 10, 25 x 10, 10 x 25, 4 x 10, 10 x 4) applied per z level, times a 1D
// operator along z applied per triangle point. Point index t + 10 k; flux points: face 0 (z = -1)
// and face 1 (z = +1) carry the 10 triangle points, quad faces 2 (y = -1), 3 (x + y = 0) and
// 4 (x = -1) carry 4 x 4 points with local index a + 4 b (a along the edge, b = z level).
// Same three fused phases as the hexahedra: A face solution, B volume group, C interface group.
//
// Mixed-precision forms: in phase B the two dense triangle-plane contractions that dominate the
// operator work -- interpolation to the 25 triangle quadrature points and the L2 projection back --
// run on the tensor cores as split products. Each operand x is split into x_hi + x_lo (FP16 or
// BF16, x_lo = round(x - x_hi)), and x.y is formed as x_hi y_hi + x_lo y_hi + x_hi y_lo with FP32
// accumulation in tensor memory: the three products are one MMA chain over a K dimension that holds
// [x_hi | x_lo | x_hi] against [y_hi | y_hi | y_lo]. Rows (element field x z level) are scaled by a
// power of two that brings their largest magnitude into [2^14, 2^15), so FP16 keeps full precision
// in x_lo; the scale is removed exactly after the product.
#include <cuda_runtime.h>

#include "fr_internal.h"
#include "fr_physics.cuh"
#include "fr_tcgen05.cuh"
#include "fr_pri_body.cuh"

namespace pri {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_pri_disu(HexArgs<T> a, const PriOps<T> *gops, const PriOpsFF *opsff)
{
    pri_disu_body<T>(a, gops, opsff, blockIdx.x, gridDim.x);
}

// FP32 on the CUDA cores: registers capped for eight CTAs of 128 threads per SM, as many as its
// shared memory allows (64 registers, a few spilled values in L1; 72 registers measured slower).
// Otherwise (0) the compiler's own register count.
template <typename T, int NTH, int TCM>
__global__ void __launch_bounds__(NTH, sizeof(T) == 4 && TCM == 0 ? 8 : 0) k_pri_B(HexArgs<T> a, const PriOps<T> *gops, const PriOpsFF *opsff)
{
    pri_B_body<T, NTH, TCM>(a, gops, opsff, blockIdx.x, gridDim.x);
}

// FP32: registers capped for 960 resident threads per SM (ten CTAs of 96), as for the hexahedra
template <typename T, int NTH>
__global__ void __launch_bounds__(NTH, sizeof(T) == 4 ? 960 / NTH : 0) k_pri_C(HexArgs<T> a, const PriOps<T> *gops, const PriOpsFF *opsff)
{
    pri_C_body<T, NTH>(a, gops, opsff, blockIdx.x, gridDim.x);
}

int grid_elems(long long ne, int per_sm)
{
    long long g = ne;
    if (g > fr_sms() * per_sm * 8) g = fr_sms() * per_sm * 8;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace pri

using namespace pri;

int pri_set_const_ops(const PriOps<float> *h) { return pri::set_const_ops(*h); }

template <typename T>
int pri_fused_phase(int phase, const HexArgs<T> &a, const PriOps<T> *ops, const PriOpsFF *ops64, cudaStream_t s)
{
    if (a.ne == 0) return 0;
    if (phase == 0) {
        long long work = a.ne * NF;
        long long g = (work + 255) / 256;
        if (g > fr_sms() * 64) g = fr_sms() * 64;
        k_pri_disu<T><<<(int)g, 256, 0, s>>>(a, ops, ops64);
    } else if (phase == 1) {
        constexpr int NTH = 128;
        const size_t base = ((sizeof(PriOps<T>) + 15) / 16) * 16 + (size_t)(5 * NU + 15 * NU + 5 * NF + 20 * NQ) * sizeof(T);
        bool tcdone = false;
        if constexpr (sizeof(T) == 4) {
          if (a.tcmode != 0) {
            tcdone = true;
            const int tcnt = TC_ROWS_P * TC_ST > 5 * NZ * NQT ? TC_ROWS_P * TC_ST : 5 * NZ * NQT;
            const size_t smem = base + (size_t)tcnt * sizeof(T) + (a.tcmode == 1 ? PriTC<1>::BYTES : PriTC<2>::BYTES);
            // persistent: as many CTAs as fit on the SMs (shared memory, registers, and the 512
            // tensor-memory columns at 32 per CTA)
            auto kern = a.tcmode == 1 ? k_pri_B<T, NTH, 1> : k_pri_B<T, NTH, 2>;
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
            kern<<<(int)g, NTH, smem, s>>>(a, ops, ops64);
          }
        }
        if (!tcdone) {
            // FP32 interpolates all 20 fields per pass (staging 20 x 4 x 25 values)
            const size_t smem = base + (size_t)((sizeof(T) == 4 ? 20 : 5) * NZ * NQT) * sizeof(T);
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_pri_B<T, NTH, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                attr = true;
            }
            k_pri_B<T, NTH, 0><<<grid_elems(a.ne, 8), NTH, smem, s>>>(a, ops, ops64);
        }
    } else {
        if constexpr (sizeof(T) == 4) k_pri_C<T, 96><<<grid_elems(a.ne, 10), 96, 0, s>>>(a, ops, ops64);
        else k_pri_C<T, 128><<<grid_elems(a.ne, 8), 128, 0, s>>>(a, ops, ops64);
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template int pri_fused_phase<double>(int, const HexArgs<double> &, const PriOps<double> *, const PriOpsFF *, cudaStream_t);
template int pri_fused_phase<float>(int, const HexArgs<float> &, const PriOps<float> *, const PriOpsFF *, cudaStream_t);
