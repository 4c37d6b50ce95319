// Host side of the tensor-core tile engine (tc_gemm.cuh): TMA tensor maps of
// split BF16 operands, and the engine applied to plain dense matrices
// (hylu_split_gemm), which checks the engine in isolation: C -= A B with A
// M x K, B K x N and C M x N in FP32, every product on the tensor cores.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "tc_gemm.cuh"
#include "../../include/hylu.h"

namespace hylu {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// A (M x K, row stride lda) -> NS BF16 terms, each a zero-padded Mp x Kp
// row-major array at out + s * Mp * Kp.
template <int NS>
__global__ void split_rows_kernel(const float* __restrict__ A, int M, int K, int lda,
                                  __nv_bfloat16* __restrict__ out, int Mp, int Kp) {
    const int64_t tot = (int64_t)Mp * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / Kp), k = (int)(e % Kp);
        const float v = (m < M && k < K) ? A[(int64_t)m * lda + k] : 0.f;
        __nv_bfloat16 t[NS];
        tc::split_bf16<NS>(v, t);
#pragma unroll
        for (int s = 0; s < NS; ++s) out[s * tot + e] = t[s];
    }
}

struct DenseMaps {
    CUtensorMap m[3];
};

// One 128 x 64 tile of C -= A B per block (128 threads).
template <int NS>
__global__ void __launch_bounds__(128) dense_tile_kernel(const __grid_constant__ DenseMaps maps,
                                                         const float* __restrict__ B, int K, int N, int ldb,
                                                         float* __restrict__ C, int M, int ldc, int Kp,
                                                         int* status, long long limit) {
    extern __shared__ unsigned char smem_raw[];
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
    tc::TileSmem<NS>& sm = *reinterpret_cast<tc::TileSmem<NS>*>(base);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * tc::TM, n0 = blockIdx.y * tc::TN;
    if (tid == 0) {
        tc::mbar_init(&sm.bar_tma, 1);
        tc::mbar_init(&sm.bar_mma, 1);
        tc::mbar_fence_init();
        sm.abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(&sm.tmem_base, tc::TMEM_COLS);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    const int nchunks = Kp / tc::TK;
    uint32_t phase = 0;
    bool issued = false;
    for (int c = 0; c < nchunks; ++c) {
        if (tid == 0) {
            tc::mbar_expect_tx(&sm.bar_tma, NS * tc::A_TERM_BYTES);
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int j = 0; j < tc::TK / tc::KB; ++j)
                    tc::tma_load_2d(&sm.a[s][j * tc::KB * tc::TM], &maps.m[s], c * tc::TK + j * tc::KB, m0,
                                    &sm.bar_tma);
        }
        // B chunk: rows c * TK .. + TK, columns n0 .. n0 + TN, split on the way
        for (int e = tid; e < tc::TK * tc::TN; e += 128) {
            const int k = e / tc::TN, n = e % tc::TN;
            const int gk = c * tc::TK + k, gn = n0 + n;
            const float v = (gk < K && gn < N) ? B[(int64_t)gk * ldb + gn] : 0.f;
            __nv_bfloat16 t[NS];
            tc::split_bf16<NS>(v, t);
#pragma unroll
            for (int s = 0; s < NS; ++s)
                *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(sm.b[s]) + tc::b_off(n, k)) = t[s];
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (!tc::mbar_wait(&sm.bar_tma, phase, limit)) {
                sm.abort = 1;
                atomicCAS(status, 0, HYLU_ERR_DEVICE_TIMEOUT);
                tc::mbar_wait(&sm.bar_tma, phase, limit);     // copies still in flight
            } else {
                tc::tc_fence_after();
                tc::issue_chunk<NS>(sm, tmem, c == 0);
                tc::mma_commit(&sm.bar_mma);
            }
        }
        __syncthreads();
        if (sm.abort) break;
        issued = true;
        if (!tc::mbar_wait(&sm.bar_mma, phase, limit)) {
            if (tid == 0) atomicCAS(status, 0, HYLU_ERR_DEVICE_TIMEOUT);
            tc::mbar_wait(&sm.bar_mma, phase, limit);
            sm.abort = 1;
            break;
        }
        phase ^= 1u;
    }
    __syncthreads();
    if (issued && !sm.abort) {
        tc::tc_fence_after();
        const int m = m0 + warp * 32 + lane;
#pragma unroll
        for (int j = 0; j < tc::TN / 16; ++j) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 16), v);
            if (m < M) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = n0 + j * 16 + q;
                    if (n < N) C[(int64_t)m * ldc + n] -= v[q];
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tc::TMEM_COLS);
}

template <int NS>
int run_dense(const float* A, const float* B, float* C, int M, int N, int K, int lda, int ldb, int ldc,
              cudaStream_t st) {
    auto enc = encode_fn();
    if (!enc) return HYLU_ERR_CUDA;
    const int Mp = (M + tc::TM - 1) / tc::TM * tc::TM;
    const int Kp = (K + tc::TK - 1) / tc::TK * tc::TK;
    __nv_bfloat16* split = nullptr;
    int* status = nullptr;
    if (cudaMalloc(&split, sizeof(__nv_bfloat16) * (size_t)NS * Mp * Kp) != cudaSuccess) return HYLU_ERR_NOMEM;
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) { cudaFree(split); return HYLU_ERR_NOMEM; }
    int rc = HYLU_OK;
    DenseMaps maps{};
    for (int s = 0; s < NS && rc == HYLU_OK; ++s) {
        cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Mp};
        cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
        cuuint32_t box[2] = {(cuuint32_t)tc::KB, (cuuint32_t)tc::TM};
        cuuint32_t estr[2] = {1, 1};
        if (enc(&maps.m[s], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, split + (size_t)s * Mp * Kp, dims, strides, box,
                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            rc = HYLU_ERR_CUDA;
    }
    if (rc == HYLU_OK && cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) rc = HYLU_ERR_CUDA;
    if (rc == HYLU_OK && Mp > 0 && Kp > 0) {
        split_rows_kernel<NS><<<std::min<int64_t>(4096, ((int64_t)Mp * Kp + 255) / 256), 256, 0, st>>>(
            A, M, K, lda, split, Mp, Kp);
        count_launch();
        const size_t smem = sizeof(tc::TileSmem<NS>) + 1024;
        cudaFuncSetAttribute(dense_tile_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid(Mp / tc::TM, (N + tc::TN - 1) / tc::TN);
        dense_tile_kernel<NS><<<grid, 128, smem, st>>>(maps, B, K, N, ldb, C, M, ldc, Kp, status, 1LL << 24);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) rc = HYLU_ERR_CUDA;
    }
    int hs = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = HYLU_ERR_CUDA;
    else if (rc == HYLU_OK && cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && hs)
        rc = hs;
    cudaFree(split);
    cudaFree(status);
    return rc;
}

}  // namespace

bool tensor_maps_available() { return encode_fn() != nullptr; }

size_t tensor_map_bytes() { return sizeof(CUtensorMap); }

int encode_a_maps(int32_t ngd, const int32_t* Mp, const int32_t* Kp, const int64_t* a_off, uint16_t* const* a_term,
                  void* out) {
    auto enc = encode_fn();
    if (!enc) return HYLU_ERR_CUDA;
    CUtensorMap* m = static_cast<CUtensorMap*>(out);
    for (int32_t g = 0; g < ngd; ++g)
        for (int s = 0; s < 3; ++s) {
            CUtensorMap& t = m[3 * g + s];
            std::memset(&t, 0, sizeof(t));
            if (Kp[g] == 0) continue;          // no pair: never loaded
            cuuint64_t dims[2] = {(cuuint64_t)Kp[g], (cuuint64_t)Mp[g]};
            cuuint64_t strides[1] = {(cuuint64_t)Kp[g] * 2};
            cuuint32_t box[2] = {(cuuint32_t)tc::KB, (cuuint32_t)tc::TM};
            cuuint32_t estr[2] = {1, 1};
            if (enc(&t, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a_term[s] + a_off[g], dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return HYLU_ERR_CUDA;
        }
    return HYLU_OK;
}

}  // namespace hylu

extern "C" int hylu_split_gemm(const float* d_a, const float* d_b, float* d_c, int m, int n, int k, int lda,
                               int ldb, int ldc, int nsplit, void* stream) {
    if (m < 0 || n < 0 || k < 0 || (nsplit != 2 && nsplit != 3)) return HYLU_ERR_ARG;
    if (m == 0 || n == 0 || k == 0) return HYLU_OK;
    if (!d_a || !d_b || !d_c || lda < k || ldb < n || ldc < n) return HYLU_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return nsplit == 2 ? hylu::run_dense<2>(d_a, d_b, d_c, m, n, k, lda, ldb, ldc, st)
                       : hylu::run_dense<3>(d_a, d_b, d_c, m, n, k, lda, ldb, ldc, st);
}
