// BF16 GEMM with FP32 accumulation on the fifth-generation tensor cores, for
// the training passes of the proposal network:
//
//     C[m][n] (+)= sum_k A[m][k] B[n][k]        (A: M x K, B: N x K, both K-major)
//
// One block of 128 threads computes a 128 x BN tile of C (BN 128, or 64 when
// that gives the SMs more blocks, or 16 for the output layer).  Thread 0
// streams the K dimension in chunks of 64 through three shared-memory stages,
// each chunk's copy issued two chunks ahead of its MMAs: each chunk of A
// and B arrives by TMA as eight 16-byte-wide column slices (one box of 8 x 128
// or 8 x BN elements each), which is exactly the no-swizzle K-major core-matrix
// layout the MMA descriptors expect (adjacent 8-row groups 128 bytes apart,
// adjacent 8-column slices rows * 16 bytes apart).  It issues four
// tcgen05.mma (K = 16) per chunk into one TMEM accumulator and commits them to
// the stage's mbarrier, which frees the stage for the copy three chunks later.
// A product split over K runs about two blocks per SM, which add their tiles.
// After the last commit the four warps read their 32 TMEM lanes and store (or,
// split over K, atomically add) the FP32 tile.  Rows and columns past the
// matrices' ends are filled with zeros by the copies and never stored.  Every
// wait is bounded: a wait that gives up raises the caller's error flag and the
// block leaves without storing.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "gamma_internal.h"
#include "gamma_tc.cuh"

namespace gk {

using bf16 = __nv_bfloat16;

namespace {

constexpr int kGemmBM = 128;             // rows per tile (MMA M)
constexpr int kGemmBK = 64;              // K per stage
constexpr int kGemmStages = 3;           // stages in flight

template <int BN>
struct GemmSmem {
    bf16 A[kGemmStages][kGemmBM * kGemmBK];   // per stage: 8 slices of 128 rows x 16 bytes
    bf16 B[kGemmStages][BN * kGemmBK];        // per stage: 8 slices of BN rows x 16 bytes
    uint64_t full[kGemmStages], empty[kGemmStages], done;
    uint32_t tmem;
    int ok;
};

template <int BN, bool ATOMIC>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
              int M, int N, int nchunks, int chunks_per_split, float* __restrict__ C, int ldc,
              unsigned* flags)
{
    static_assert(BN == 16 || BN == 64 || BN == 128, "tile width");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the stages start on a 1 KB boundary (TMA destinations: 128 bytes)
    unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    GemmSmem<BN>& S = *reinterpret_cast<GemmSmem<BN>*>(base);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kGemmBM, n0 = blockIdx.x * BN;
    const int c0 = blockIdx.z * chunks_per_split;
    const int c1 = min(nchunks, c0 + chunks_per_split);
    if (c0 >= c1) return;                                 // block-uniform: an empty K split
    constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;
    if (tid == 0) {
        for (int b = 0; b < kGemmStages; ++b) {
            mbar_init(&S.full[b], 1);
            mbar_init(&S.empty[b], 1);
        }
        mbar_init(&S.done, 1);
        mbar_fence_init();
        S.ok = 1;
    }
    if (warp == 0) {
        tmem_alloc(&S.tmem, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tm = S.tmem;
    if (tid == 0) {
        constexpr uint32_t kId = idesc_bf16_f32(kGemmBM, BN);
        constexpr uint32_t kBytes = (kGemmBM + BN) * kGemmBK * 2;
        uint32_t nfull[kGemmStages] = {}, nempty[kGemmStages] = {};
        bool pending[kGemmStages] = {};                   // a copy issued but not yet seen landed
        bool ok = true;
        // chunk i (from c0) goes to stage i % kGemmStages; its copy is issued
        // kGemmStages - 1 chunks ahead of its MMAs
        auto load = [&](int i) {
            const int s = i % kGemmStages;
            if (i >= kGemmStages) {                       // the MMAs of chunk i - kGemmStages read it
                ok = mbar_wait_bounded(&S.empty[s], nempty[s] & 1u);
                ++nempty[s];
                if (!ok) return;
            }
            mbar_arrive_expect_tx(&S.full[s], kBytes);
            pending[s] = true;
            const int k0 = (c0 + i) * kGemmBK;
#pragma unroll
            for (int j = 0; j < kGemmBK / 8; ++j) {
                tma_load_2d(&S.A[s][j * kGemmBM * 8], &amap, k0 + 8 * j, m0, &S.full[s]);
                tma_load_2d(&S.B[s][j * BN * 8], &bmap, k0 + 8 * j, n0, &S.full[s]);
            }
        };
        const int nloc = c1 - c0;
        for (int i = 0; i < kGemmStages - 1 && i < nloc && ok; ++i) load(i);
        for (int c = c0; c < c1 && ok; ++c) {
            const int i = c - c0, s = i % kGemmStages;
            if (i + kGemmStages - 1 < nloc) load(i + kGemmStages - 1);
            if (!ok) break;
            ok = mbar_wait_bounded(&S.full[s], nfull[s] & 1u);
            if (!ok) break;
            pending[s] = false;
            ++nfull[s];
            tc_fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kGemmBK; kk += 16) {
                const uint32_t la = kGemmBM * 16u, lb = BN * 16u;    // bytes between 8-column slices
                const uint64_t ad = smem_desc(smem_addr(&S.A[s][0]) + (uint32_t)(kk >> 3) * la, la, 128u);
                const uint64_t bd = smem_desc(smem_addr(&S.B[s][0]) + (uint32_t)(kk >> 3) * lb, lb, 128u);
                tc_mma_bf16(tm, ad, bd, kId, (c > c0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(&S.empty[s]);
        }
        tc_commit(&S.done);
        if (!ok) {
            S.ok = 0;
            // let this block's copies land before it leaves
            for (int b = 0; b < kGemmStages; ++b)
                if (pending[b]) mbar_wait_bounded(&S.full[b], nfull[b] & 1u);
        }
    }
    // every thread waits for the accumulator (bounded), then the epilogue
    const bool landed = mbar_wait_bounded(&S.done, 0u);
    const bool ok = __syncthreads_and(landed) && S.ok;      // block-uniform
    tc_fence_after_sync();
    if (ok) {
        const int row = m0 + 32 * warp + lane;
#pragma unroll 1
        for (int j = 0; j < BN; j += 16) {
            float v[16];
            tmem_ld16(tm + ((uint32_t)(32 * warp) << 16) + (uint32_t)j, v);
            if (row < M) {
                float* dst = C + (long long)row * ldc + n0 + j;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    if (n0 + j + u < N) {
                        if (ATOMIC) atomicAdd(dst + u, v[u]);
                        else dst[u] = v[u];
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(flags, kFlagTimeout);
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    if (warp == 0) tmem_dealloc(tm, kTmemCols);
}

}  // namespace

template <int BN, bool ATOMIC>
static cudaError_t launch_gemm_tc_k(const CUtensorMap& am, const CUtensorMap& bm, long long M, int N,
                                    int nchunks, int per, int splits, float* C, int ldc,
                                    unsigned* flags, cudaStream_t s)
{
    const size_t smem = sizeof(GemmSmem<BN>) + 1024;      // room to align the base to 1 KB
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<BN, ATOMIC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + kGemmBM - 1) / kGemmBM),
                    (unsigned)splits);
    k_gemm_tc<BN, ATOMIC><<<grid, 128, smem, s>>>(am, bm, (int)M, N, nchunks, per, C, ldc, flags);
    return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const bf16* A, long long M, long long lda, const bf16* B, int N,
                           long long ldb, long long K, float* C, int ldc, int splits,
                           unsigned* flags, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0 || splits < 1) return cudaErrorInvalidValue;
    if ((lda % 8) || (ldb % 8) || (((uintptr_t)A | (uintptr_t)B) & 15u)) return cudaErrorInvalidValue;
    const long long mtiles = (M + kGemmBM - 1) / kGemmBM;
    // the widest tile that still gives every SM a block (else 64 columns)
    const int bn = N <= 16 ? 16 : (mtiles * ((N + 127) / 128) >= device_sm_count() ? 128 : 64);
    CUtensorMap am, bm;
    // A: K x M elements (inner, rows), boxes of 8 x 128; B: K x N, boxes of 8 x bn
    if (!encode_bf16_2d(&am, A, (unsigned long long)K, (unsigned long long)M,
                        (unsigned long long)lda * 2, 8, kGemmBM) ||
        !encode_bf16_2d(&bm, B, (unsigned long long)K, (unsigned long long)N,
                        (unsigned long long)ldb * 2, 8, (unsigned)bn))
        return cudaErrorInvalidValue;
    const int nchunks = (int)((K + kGemmBK - 1) / kGemmBK);
    if (splits > 1) {
        // a split-K product: about two blocks per SM
        const long long tiles = mtiles * ((N + bn - 1) / bn);
        splits = (int)std::max<long long>(splits, (2LL * device_sm_count() + tiles - 1) / tiles);
        splits = std::min(splits, std::max(1, nchunks / 4));   // at least 4 chunks a block
    }
    splits = std::min(splits, nchunks);
    const int per = (nchunks + splits - 1) / splits;
    splits = (nchunks + per - 1) / per;
    const bool atomic = splits > 1;
    if (bn == 16) {
        return atomic ? launch_gemm_tc_k<16, true>(am, bm, M, N, nchunks, per, splits, C, ldc, flags, s)
                      : launch_gemm_tc_k<16, false>(am, bm, M, N, nchunks, per, splits, C, ldc, flags, s);
    }
    if (bn == 64) {
        return atomic ? launch_gemm_tc_k<64, true>(am, bm, M, N, nchunks, per, splits, C, ldc, flags, s)
                      : launch_gemm_tc_k<64, false>(am, bm, M, N, nchunks, per, splits, C, ldc, flags, s);
    }
    return atomic ? launch_gemm_tc_k<128, true>(am, bm, M, N, nchunks, per, splits, C, ldc, flags, s)
                  : launch_gemm_tc_k<128, false>(am, bm, M, N, nchunks, per, splits, C, ldc, flags, s);
}

// Transpose of a bf16 matrix: src [rows][cols] (row stride lds) -> dst
// [cols][rows] (row stride ldd >= rows; columns rows .. ldd - 1 are zeroed).
__global__ void __launch_bounds__(256) k_transpose_bf16(const bf16* __restrict__ src, long long rows,
                                                        int cols, long long lds, bf16* __restrict__ dst,
                                                        long long ldd)
{
    __shared__ bf16 t[32][33];
    const long long r0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const long long r = r0 + j;
        const int c = c0 + tx;
        t[j][tx] = (r < rows && c < cols) ? src[r * lds + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int c = c0 + j;
        const long long r = r0 + tx;
        if (c < cols && r < ldd) dst[(long long)c * ldd + r] = t[tx][j];
    }
}

cudaError_t launch_transpose_bf16(const bf16* src, long long rows, int cols, long long lds, bf16* dst,
                                  long long ldd, cudaStream_t s)
{
    const dim3 grid((unsigned)((ldd + 31) / 32), (unsigned)((cols + 31) / 32));
    k_transpose_bf16<<<grid, 256, 0, s>>>(src, rows, cols, lds, dst, ldd);
    return cudaGetLastError();
}

}  // namespace gk
