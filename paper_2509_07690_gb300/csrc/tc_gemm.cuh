// Tensor-core tile engine of the precision form's sup-sup update (HYLU
// Sec. 2.2, Fig. 1c: a supernode destination takes the updates of its source
// supernodes as dense matrix products).  On sm_103a the products run on the
// 5th-generation tensor cores: tcgen05.mma kind::f16 with BF16 operands and
// FP32 accumulators in tensor memory (TMEM).  FP32 operands are split into
// NS BF16 terms, x = x_0 + x_1 (+ x_2), each the BF16 rounding of what the
// earlier terms leave (the splitting of Henry, Tang and Heinecke, 2019), and
// the product is the sum of the term products whose combined order is below
// NS (3 products for NS = 2, 6 for NS = 3: about FP32 accuracy).
//
// One tile is M = 128 rows (TMEM lanes) x N = 64 columns (TMEM columns) of
// the destination, accumulated over K chunks of 32:
//   - A (128 x 32 per term) is loaded by TMA (cp.async.bulk.tensor.2d) as
//     four boxes of 8 K-elements x 128 rows: without swizzling a box is a
//     column of 8x8 core matrices (16 bytes per row), the canonical K-major
//     layout (core matrices 128 B apart along M, 2 KB apart along K);
//   - B (32 x 64 per term) is written by the threads into the same layout
//     (core matrices 128 B apart along N, 1 KB apart along K), gathered from
//     wherever the caller's rows live and split on the way;
//   - one thread issues the MMAs and commits them to an mbarrier; the
//     epilogue reads the accumulator with tcgen05.ld (each warp its 32 lanes).
// Every wait is bounded; an expired wait reports through the caller's status.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace hylu {
namespace tc {

constexpr int TM = 128;               // tile rows (TMEM lanes)
constexpr int TN = 64;                // tile columns (TMEM columns, FP32)
constexpr int TK = 32;                // K chunk
constexpr int KB = 8;                 // K elements per core-matrix column (16 bytes of BF16)
constexpr int A_BOX_BYTES = KB * TM * 2;            // one TMA box: 2 KB
constexpr int A_TERM_BYTES = TK * TM * 2;           // 8 KB per term and chunk
constexpr int B_TERM_BYTES = TK * TN * 2;           // 4 KB per term and chunk
constexpr uint32_t TMEM_COLS = 64;

template <int NS>
struct TileSmem {
    alignas(1024) __nv_bfloat16 a[NS][TK * TM];
    alignas(1024) __nv_bfloat16 b[NS][TK * TN];
    alignas(8) unsigned long long bar_tma;
    alignas(8) unsigned long long bar_mma;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------- TMA
// 2D tiled load of one box into shared memory, completing bytes on `bar`.
// x (innermost, in elements) must be a multiple of 8 for 16-bit elements.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// generic-proxy writes to shared memory made visible to the async proxy
// (the tensor core reads B written by the threads)
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]; accumulate = 0 overwrites D
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on `bar` once every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory matrix descriptor, no swizzling, K-major: start address,
// leading (K-direction) and stride (M/N-direction) byte offsets between 8x8
// core matrices; bit 46 is the descriptor version of this architecture.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16
// at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Split x into NS BF16 terms (rounded to nearest; each term the rounding of
// what the earlier terms leave).
template <int NS>
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16* t) {
    float r = x;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        t[s] = __float2bfloat16_rn(r);
        r -= __bfloat162float(t[s]);
    }
}

// Byte offset of element (n, k) of a 32 x 64 B chunk (K-major core matrices:
// 8 n-rows of 16 bytes each, 128 B apart along N, 1 KB apart along K).
__device__ __forceinline__ int b_off(int n, int k) { return (k >> 3) * (TN * 16) + n * 16 + (k & 7) * 2; }

// Issue the MMAs of one K chunk (one thread).  Term products (i, j) with
// i + j < NS: the larger terms first.
template <int NS>
__device__ __forceinline__ void issue_chunk(TileSmem<NS>& sm, uint32_t tmem_d, bool first) {
    constexpr uint32_t idesc = idesc_bf16(TM, TN);
    bool acc = !first;
#pragma unroll
    for (int kk = 0; kk < TK / 16; ++kk) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                if (i + j >= NS) continue;
                // A: K-adjacent core matrices 2 KB apart (one TMA box each),
                // M-adjacent 128 B; B: K-adjacent 1 KB, N-adjacent 128 B
                const uint64_t ad = smem_desc(smem_u32(&sm.a[i][0]) + kk * 2 * A_BOX_BYTES, A_BOX_BYTES, 128);
                const uint64_t bd = smem_desc(smem_u32(&sm.b[j][0]) + kk * 2 * (TN * 16), TN * 16, 128);
                mma_bf16(tmem_d, ad, bd, idesc, acc ? 1u : 0u);
                acc = true;
            }
        }
    }
}

}  // namespace tc
}  // namespace hylu
