// fr_tcgen05.cuh -- inline-PTX wrappers for the Blackwell asynchronous units of sm_100a/sm_103a:
// the fifth-generation tensor cores (tensor-memory allocation, shared-memory matrix descriptors,
// kind::f16 MMA issue by one thread, completion through an mbarrier, TMEM loads back to registers)
// and the bulk-copy (TMA) engine (global -> shared copies that complete on an mbarrier).
//
// Operand layout used throughout: K-major, no swizzle. A matrix of R rows x K 16-bit values is
// stored as core matrices of 8 rows x 8 values (16 bytes per row, 128 contiguous bytes per core
// matrix); value (r, k) sits at byte
//     (r / 8) * sbo + (k / 8) * lbo + (r % 8) * 16 + (k % 8) * 2
// with lbo = 128 (core matrices adjacent along K) and sbo = (K / 8) * 128.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__host__ __device__ constexpr uint32_t core_offset(int r, int k, int sbo)
{
    return (uint32_t)((r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (no swizzle): start address, leading (K) and stride (M/N) byte
// offsets, each encoded >> 4; bit 46 is the descriptor version of the fifth-generation tensor core.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16 with an FP32 accumulator; fmt 0 = FP16, 1 = BF16 for both
// A and B; both K-major; dense, no negation.
__host__ __device__ constexpr uint32_t idesc_f16(int fmt, int M, int N)
{
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Executed by one whole warp. Writes the TMEM base address to *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Executed by one whole warp.
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Makes this thread's ordinary shared-memory stores visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A B^T for one K = 16 slice; A, B described by shared-memory descriptors.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier receives one arrival when every MMA issued before by this thread has completed.
__device__ __forceinline__ void commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Polls (non-blocking test, short sleeps) until the phase of parity `parity` has completed.
// Gives up after `limit` polls (about a second at the default) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t limit = 1u << 24)
{
    const uint32_t a = smem_u32(mbar);
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global memory into
// this CTA's shared memory, completing on *mbar, whose phase also takes one arrival from this call.
// Issued by one thread.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (lane = 32 * (warp % 4) + lane id),
// starting at taddr; waits for the load to land before returning.
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Split hi + lo operands (TCM = 1: FP16, 2: BF16): x_hi = round(x), x_lo = round(x - x_hi).
template <int TCM>
__device__ __forceinline__ void split16(float x, uint16_t &h, uint16_t &l)
{
    if constexpr (TCM == 1) {
        const __half hh = __float2half_rn(x);
        h = __half_as_ushort(hh);
        l = __half_as_ushort(__float2half_rn(x - __half2float(hh)));
    } else {
        const __nv_bfloat16 hh = __float2bfloat16_rn(x);
        h = __bfloat16_as_ushort(hh);
        l = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hh)));
    }
}

// The split forms of the operands, by K segment. FP16 (TCM = 1): x = x_hi + x_lo, three products
// x_hi y_hi + x_lo y_hi + x_hi y_lo (segments [x_hi | x_lo | x_hi] against [y_hi | y_hi | y_lo]).
// BF16 (TCM = 2), whose 8-bit significands leave about 16 bits in two terms: x = x_1 + x_2 + x_3,
// y likewise, and the six products whose parts' orders sum to at most two (x_1 y_1, x_1 y_2,
// x_2 y_1, x_1 y_3, x_2 y_2, x_3 y_1), about 24 bits like FP32. `x` is the data operand (the rows
// split per element), `y` the operator.
template <int TCM>
struct SplitForm {
    static constexpr int PARTS = TCM == 2 ? 3 : 2;
    static constexpr int SEGS = TCM == 2 ? 6 : 3;
    // the part of x, and of y, that K segment s holds
    __host__ __device__ static constexpr int x_part(int s) { return TCM == 2 ? (s == 2 || s == 4 ? 1 : (s == 5 ? 2 : 0)) : (s == 1 ? 1 : 0); }
    __host__ __device__ static constexpr int y_part(int s) { return TCM == 2 ? (s == 1 || s == 4 ? 1 : (s == 3 ? 2 : 0)) : (s == 2 ? 1 : 0); }
};

// Each product x_i y_j whose parts' orders sum to at most PARTS - 1 appears in exactly one segment,
// and no other product appears (checked at compile time for both forms).
template <int TCM>
constexpr bool split_form_complete()
{
    using SF = SplitForm<TCM>;
    int seen[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int s = 0; s < SF::SEGS; s++) seen[SF::x_part(s)][SF::y_part(s)]++;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (seen[i][j] != ((i < SF::PARTS && j < SF::PARTS && i + j <= SF::PARTS - 1) ? 1 : 0)) return false;
    return true;
}
static_assert(split_form_complete<1>() && split_form_complete<2>(), "split forms: every product of order <= 1 (FP16) or <= 2 (BF16) once");

// The parts of x in the split form (FP16: hi, lo; BF16: x_1, x_2, x_3, each the rounding of what
// the previous ones leave; the differences are exact in FP32).
template <int TCM>
__device__ __forceinline__ void split_parts(float x, uint16_t (&p)[3])
{
    if constexpr (TCM == 1) {
        split16<1>(x, p[0], p[1]);
        p[2] = 0;
    } else {
        const __nv_bfloat16 b1 = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(b1);
        const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(b2);
        p[0] = __bfloat16_as_ushort(b1);
        p[1] = __bfloat16_as_ushort(b2);
        p[2] = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
    }
}

// K of a split operand row: SEGS segments of K0 values, padded to the MMA's K step of 16.
template <int TCM>
__host__ __device__ constexpr int split_k(int k0) { return (SplitForm<TCM>::SEGS * k0 + 15) / 16 * 16; }

// Exponent s with max|x| 2^s in [2^14, 2^15) (0 for zero, subnormal or non-finite maxima).
__device__ __forceinline__ int row_shift(float mx)
{
    const int eb = (int)((__float_as_uint(mx) >> 23) & 0xFF);
    if (eb == 0 || eb == 255) return 0;
    const int sh = 141 - eb;
    return sh < -120 ? -120 : (sh > 120 ? 120 : sh);
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// Row r of a split data operand: the parts of the L values x (already scaled) in the K segments
// of the split form, zero-padded to K, as K/8 core-matrix rows of 16 bytes.
template <int TCM, int K, int L>
__device__ __forceinline__ void store_split_parts(unsigned char *base, int r, const float (&x)[L])
{
    using SF = SplitForm<TCM>;
    uint16_t pp[L][3];
#pragma unroll
    for (int i = 0; i < L; i++) split_parts<TCM>(x[i], pp[i]);
#pragma unroll
    for (int ch = 0; ch < K / 8; ch++) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            uint16_t v[2];
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const int k = 8 * ch + 2 * h + j, sg = k / L, i = k % L;
                v[j] = sg < SF::SEGS ? pp[i][SF::x_part(sg)] : (uint16_t)0;
            }
            w[h] = pack2(v[0], v[1]);
        }
        *reinterpret_cast<uint4 *>(base + core_offset(r, 8 * ch, (K / 8) * 128)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// One MMA chain D = A B^T over KSTEPS slices of K = 16 (M = 128 rows of A, N rows of B, both K-major
// with lbo = 128), issued by thread 0 after every thread's operand stores are made visible to the
// tensor core; then every thread waits (at most `limit` polls) for completion. Returns false,
// uniformly across the CTA, if the wait gave up; the phase parity advances only on success.
template <int KSTEPS>
__device__ __forceinline__ bool mma_chain(uint32_t tmem, const unsigned char *A, int sbo_a, const unsigned char *B, int sbo_b,
                                          uint32_t idesc, uint64_t *mbar, uint32_t &parity, uint32_t limit = 1u << 24)
{
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_after_sync();
        const uint32_t aA = smem_u32(A), aB = smem_u32(B);
#pragma unroll
        for (int j = 0; j < KSTEPS; j++)
            mma_f16(tmem, sdesc(aA + 256 * j, 128, sbo_a), sdesc(aB + 256 * j, 128, sbo_b), idesc, j);
        commit(mbar);
    }
    const bool done = mbar_wait(mbar, parity, limit);
    if (!__syncthreads_and(done)) return false;
    parity ^= 1;
    fence_after_sync();
    return true;
}

// The two halves of mma_chain, for callers that do independent CUDA-core work while the chain runs:
// mma_issue makes every thread's operand stores visible and issues the chain from thread 0 (call with
// every thread); mma_wait waits for it as mma_chain does (the caller must not write the operand
// tiles, or shared memory the chain's rows run into, between the two).
template <int KSTEPS>
__device__ __forceinline__ void mma_issue(uint32_t tmem, const unsigned char *A, int sbo_a, const unsigned char *B, int sbo_b,
                                          uint32_t idesc, uint64_t *mbar)
{
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_after_sync();
        const uint32_t aA = smem_u32(A), aB = smem_u32(B);
#pragma unroll
        for (int j = 0; j < KSTEPS; j++)
            mma_f16(tmem, sdesc(aA + 256 * j, 128, sbo_a), sdesc(aB + 256 * j, 128, sbo_b), idesc, j);
        commit(mbar);
    }
}

__device__ __forceinline__ bool mma_wait(uint64_t *mbar, uint32_t &parity, uint32_t limit = 1u << 24)
{
    const bool done = mbar_wait(mbar, parity, limit);
    if (!__syncthreads_and(done)) return false;
    parity ^= 1;
    fence_after_sync();
    return true;
}

// Per-CTA setup: mbarrier (thread 0) and tensor-memory columns (warp 0). Call with every thread.
__device__ __forceinline__ void setup(uint64_t *mbar, uint32_t *s_tmem, uint32_t ncols)
{
    if (threadIdx.x == 0) mbar_init(mbar, 1);
    __syncwarp();
    if (threadIdx.x < 32) tmem_alloc(s_tmem, ncols);
}

// Poll limit of a CTA's first bounded wait: 0 when the debug switch that makes it give up at once is on
// (exercises the give-up path: report, drain with the normal bound, release, return).
__device__ __forceinline__ uint32_t first_limit(bool &first, int give_up)
{
    const uint32_t l = (first && give_up) ? 0u : (1u << 24);
    first = false;
    return l;
}

// Per-CTA teardown; `failed`: a chain gave up, so its completion gets one more bounded wait first.
__device__ __forceinline__ void teardown(uint64_t *mbar, uint32_t parity, bool failed, uint32_t tmem, uint32_t ncols)
{
    if (failed) mbar_wait(mbar, parity);
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        fence_after_sync();
        tmem_free(tmem, ncols);
    }
}

}  // namespace tc
