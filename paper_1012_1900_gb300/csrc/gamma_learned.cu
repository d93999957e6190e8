// Learned proposal for the gamma search: patch features, labels from the exact
// search, a 375-128-128-4 BF16 network trained and run with hand-written
// tensor-core kernels, and the seeding pass that turns its proposal into an
// exact upper bound before the table walk.
//
// None of this is in the paper.  The network never decides a result: its
// proposed nearest point only selects cells whose faces are evaluated
// exactly, and the distance found is a true distance to the evaluation
// surface, hence a valid upper bound on gamma.  The exact walk (Algorithm A1
// step 4) then runs unchanged from that bound.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gamma.h"
#include "gamma_cell.cuh"
#include "gamma_internal.h"
#include "gamma_mlp.cuh"
#include "gamma_tc.cuh"

namespace gk {

using bf16 = __nv_bfloat16;

// --------------------------------------------------------------------------
// Features
// --------------------------------------------------------------------------

// Gradient magnitude of dose D at grid point p, in normalised units
// (dose / dD per length / dta): central differences inside, one-sided at the
// grid edge.
template <int N>
__device__ __forceinline__ float grad_norm(const float* __restrict__ D, const Problem& P, int px,
                                           int py, int pz, long long p)
{
    const int c[3] = {px, py, pz};
    const int n[3] = {P.nx, P.ny, P.nz};
    const long long st[3] = {1, (long long)P.nx, (long long)P.nx * P.ny};
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) {
        // the same arithmetic as the seeding pass's features (box_grad2)
        float d;
        if (c[a] > 0 && c[a] < n[a] - 1) d = (__ldg(D + p + st[a]) - __ldg(D + p - st[a])) * (0.5f / P.hn[a]);
        else if (c[a] == 0) d = (__ldg(D + p + st[a]) - __ldg(D + p)) * (1.f / P.hn[a]);
        else d = (__ldg(D + p) - __ldg(D + p - st[a])) * (1.f / P.hn[a]);
        s = fmaf(d, d, s);
    }
    return sqrtf(s);
}

// Feature f (0..kInPad-1) of reference voxel (x, y, z): channel f / 125 over
// the 5^N patch p = v + o, o in {-2..2}^N (patch index f % 125, x fastest):
//   0: (D_e(p) - D_r(v)) / dD          clamped to [-16, 16]
//   1: |grad D_e(p)| * dta / dD        clamped to [0, 32]
//   2: |grad D_r(p)| * dta / dD        clamped to [0, 32]
// zero outside the grid and for f >= 375 (2D uses the first 25 of each 125).
template <int N>
__device__ __forceinline__ float voxel_feature(const Problem& P, int x, int y, int z, float dr,
                                               float inv, int f)
{
    if (f >= kIn) return 0.f;
    const int ch = f / 125, pi = f % 125;
    const int ox = pi % 5 - 2, oy = (pi / 5) % 5 - 2, oz = pi / 25 - 2;
    if (N == 2 && oz != -2) return 0.f;
    const int px = x + ox, py = y + oy, pz = N == 3 ? z + oz : 0;
    if ((unsigned)px >= (unsigned)P.nx || (unsigned)py >= (unsigned)P.ny ||
        (N == 3 && (unsigned)pz >= (unsigned)P.nz))
        return 0.f;
    const long long p = ((long long)pz * P.ny + py) * P.nx + px;
    if (ch == 0) return fminf(fmaxf((__ldg(P.ev + p) - dr) * inv, -16.f), 16.f);
    return fminf(grad_norm<N>(ch == 1 ? P.ev : P.ref, P, px, py, pz, p) * inv, 32.f);
}

// Queue items past the cost gate (bucket >= min_bucket), into P.seed_list.
__global__ void __launch_bounds__(256) k_seed_select(const __grid_constant__ Problem P, int min_bucket)
{
    const unsigned total = min(P.ctr->tail_count, P.tail_cap);
    const int lane = threadIdx.x & 31;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned c0 = blockIdx.x * blockDim.x; c0 < total; c0 += stride) {
        const unsigned i = c0 + threadIdx.x;
        const bool take = i < total && (int)P.tail_bucket[i] >= min_bucket;
        const unsigned m = __ballot_sync(0xffffffffu, take);
        unsigned base = 0;
        if (lane == 0 && m) base = atomicAdd(&P.ctr->seed_count, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (take) P.seed_list[base + __popc(m & ((1u << lane) - 1u))] = i;
    }
}

// Features f0 .. f0 + 7 of reference voxel v (f0 a multiple of 8), computed
// point by point (their loads independent, so the compiler keeps them in
// flight together).  v = 0xffffffff: zeros.
template <int N>
__device__ __forceinline__ void features8(const Problem& P, unsigned v, float dr, float inv, int f0,
                                          float (&val)[8])
{
#pragma unroll
    for (int u = 0; u < 8; ++u) val[u] = 0.f;
    if (v == 0xffffffffu || f0 >= kIn) return;
    const int x = (int)(v % (unsigned)P.nx);
    const unsigned r1 = v / (unsigned)P.nx;
    const int y = (int)(r1 % (unsigned)P.ny), z = (int)(r1 / (unsigned)P.ny);
#pragma unroll
    for (int u = 0; u < 8; ++u) val[u] = voxel_feature<N>(P, x, y, z, dr, inv, f0 + u);
}

template <int N>
__global__ void __launch_bounds__(256) k_features(const __grid_constant__ Problem P,
                                                  const unsigned* __restrict__ vox, long long n,
                                                  bf16* __restrict__ X)
{
    const float dnorm = P.dose_norm > 0.f ? P.dose_norm : fdec(P.ctr->dnorm_enc);
    const long long total = n * (kInPad / 8);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / (kInPad / 8);
        const int f0 = (int)(e % (kInPad / 8)) * 8;
        const unsigned v = vox[i];
        const float dr = __ldg(P.ref + v);
        const float dD = P.dd_frac * (P.local ? dr : dnorm);
        const float inv = dD > 0.f ? 1.0f / dD : 0.f;
        float val[8];
        features8<N>(P, v, dr, inv, f0, val);
#pragma unroll
        for (int u = 0; u < 8; ++u) X[i * kInPad + f0 + u] = __float2bfloat16(val[u]);
    }
}

// --------------------------------------------------------------------------
// Cells around an arbitrary offset (labels and seeds)
// --------------------------------------------------------------------------

template <int N>
__device__ __forceinline__ bool load_cell(const Problem& P, int x, int y, int z, int cx, int cy,
                                          int cz, float dr, float inv, float (&q)[8], uint32_t& ok)
{
    const int px = x + cx, py = y + cy, pz = z + cz;
    if ((unsigned)px >= (unsigned)P.nx || (unsigned)py >= (unsigned)P.ny ||
        (N == 3 && (unsigned)pz >= (unsigned)P.nz))
        return false;
    const bool ex = px + 1 < P.nx, ey = py + 1 < P.ny, ez = N == 3 && pz + 1 < P.nz;
    const long long sy = P.nx, sz = (long long)P.nx * P.ny;
    const long long p = (long long)pz * sz + (long long)py * sy + px;
    ok = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        q[u] = 0.f;
        if (u < (1 << N)) {
            const bool present = (!(u & 1) || ex) && (!(u & 2) || ey) && (!(u & 4) || ez);
            if (present) {
                const long long o = p + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) + ((u & 4) ? sz : 0);
                q[u] = (__ldg(P.ev + o) - dr) * inv;
                ok |= 1u << u;
            }
        }
    }
    return true;
}

// Labels: for each listed voxel, the nearest point of the evaluation surface
// (re-walking the table up to the gamma already computed) as an offset in
// normalised spatial units, and log(gamma + 1e-3).  Rows whose search would
// leave the table, or whose voxel is not evaluated, get NaN.
template <int N>
__global__ void __launch_bounds__(128) k_labels(const __grid_constant__ Problem P,
                                                const float* __restrict__ gmap,
                                                const unsigned* __restrict__ vox, long long n,
                                                float* __restrict__ T)
{
    const float dnorm = P.dose_norm > 0.f ? P.dose_norm : fdec(P.ctr->dnorm_enc);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned v = vox[i];
        const float gs = gmap[v];
        float* t = T + 4 * i;
        if (!(gs >= 0.f) || gs > P.r_cover) {
            t[0] = t[1] = t[2] = t[3] = __int_as_float(0x7fc00000);
            continue;
        }
        const int x = (int)(v % (unsigned)P.nx);
        const unsigned r1 = v / (unsigned)P.nx;
        const int y = (int)(r1 % (unsigned)P.ny), z = (int)(r1 / (unsigned)P.ny);
        const float dr = __ldg(P.ref + v);
        const float inv = 1.0f / (P.dd_frac * (P.local ? dr : dnorm));
        const float lim = gs * (1.f + 1e-5f) + 1e-6f;
        float best = kInf, foot[3] = {0.f, 0.f, 0.f}, fv[3] = {0.f, 0.f, 0.f};
        // the 2^N cells whose box contains the voxel first (the table keys
        // them by their faces off the voxel only), then the table
        for (int k = -(1 << N); k < P.ntable; ++k) {
            int cx, cy, cz;
            if (k < 0) {
                const int s = k + (1 << N);
                cx = -(s & 1);
                cy = -((s >> 1) & 1);
                cz = N == 3 ? -((s >> 2) & 1) : 0;
            } else {
                const TableEntry e = P.table[k];
                if (e.key > lim) break;
                cx = unpack10(e.off, 0);
                cy = unpack10(e.off, 10);
                cz = unpack10(e.off, 20);
                if (cx >= -1 && cx <= 0 && cy >= -1 && cy <= 0 && cz >= -1 && cz <= 0) continue;
            }
            float q[8];
            uint32_t ok;
            if (!load_cell<N>(P, x, y, z, cx, cy, cz, dr, inv, q, ok)) continue;
            CellGeom<float> g;
            cell_geom<N, float>(cx, cy, cz, P.mt, g);
            const float before = best;
            cell_argmin<N, float>(q, ok, g, P.mt, best, foot);
            if (best < before) {
                fv[0] = cx + foot[0];
                fv[1] = cy + foot[1];
                fv[2] = cz + foot[2];
            }
        }
        t[0] = fv[0] * P.hn[0];
        t[1] = fv[1] * P.hn[1];
        t[2] = N == 3 ? fv[2] * P.hn[2] : 0.f;
        t[3] = logf(gs + 1e-3f);
    }
}

// --------------------------------------------------------------------------
// Training passes around the tensor-core GEMMs (gamma_gemm_tc.cu)
// --------------------------------------------------------------------------

// Z (M x N, fp32) += bias; H = bf16(relu(Z)) (or bf16(Z) without relu).
__global__ void k_bias_act(long long M, int N, float* __restrict__ Z, const float* __restrict__ bias,
                           bf16* __restrict__ H, int ldh, int relu)
{
    const long long total = M * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % N);
        const float z = Z[e] + bias[c];
        Z[e] = z;
        if (H) H[(e / N) * ldh + c] = __float2bfloat16(relu ? fmaxf(z, 0.f) : z);
    }
}

// Huber loss (delta 1) per output, averaged over the rows with finite
// targets; dY = dloss / dy.  Y: M x kOutPad, T: M x kOut.
__global__ void k_huber(long long M, const float* __restrict__ Y, const float* __restrict__ T,
                        float* __restrict__ dY, float* __restrict__ loss, float inv_count)
{
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (long long)gridDim.x * blockDim.x) {
        const bool valid = isfinite(T[4 * i + 3]);
#pragma unroll
        for (int j = 0; j < kOut; ++j) {
            const float r = valid ? Y[i * kOutPad + j] - T[4 * i + j] : 0.f;
            const float a = fabsf(r);
            acc += a <= 1.f ? 0.5f * r * r : a - 0.5f;
            dY[4 * i + j] = (a <= 1.f ? r : copysignf(1.f, r)) * inv_count;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv_count);
}

// Output layer backward on CUDA cores (K = 4 is too thin for the tensor
// cores): dZ2 = (dY W3) * [Z2 > 0] (bf16), and the partial sums of
// dW3 = dY^T H2, db3 = sum dY.
__global__ void k_out_back(long long M, const float* __restrict__ dY, const float* __restrict__ W3,
                           const float* __restrict__ Z2, const bf16* __restrict__ H2,
                           bf16* __restrict__ dZ2, float* __restrict__ gW3, float* __restrict__ gb3)
{
    __shared__ float sW3[kOut * kH];
    __shared__ float sg[kOut * kH + kOut];
    for (int i = threadIdx.x; i < kOut * kH; i += blockDim.x) {
        sW3[i] = W3[i];
        sg[i] = 0.f;
    }
    if (threadIdx.x < kOut) sg[kOut * kH + threadIdx.x] = 0.f;
    __syncthreads();
    const int c = threadIdx.x % kH;                  // blockDim.x is a multiple of kH
    const int rstep = blockDim.x / kH;
    float gw[kOut] = {0.f, 0.f, 0.f, 0.f}, gb[kOut] = {0.f, 0.f, 0.f, 0.f};
    for (long long m = (long long)blockIdx.x * rstep + threadIdx.x / kH; m < M;
         m += (long long)gridDim.x * rstep) {
        float d = 0.f;
#pragma unroll
        for (int j = 0; j < kOut; ++j) d = fmaf(dY[4 * m + j], sW3[j * kH + c], d);
        dZ2[m * kH + c] = __float2bfloat16(Z2[m * kH + c] > 0.f ? d : 0.f);
        const float h = __bfloat162float(H2[m * kH + c]);
#pragma unroll
        for (int j = 0; j < kOut; ++j) {
            gw[j] = fmaf(dY[4 * m + j], h, gw[j]);
            if (c == 0) gb[j] += dY[4 * m + j];
        }
    }
#pragma unroll
    for (int j = 0; j < kOut; ++j) {
        atomicAdd(&sg[j * kH + c], gw[j]);
        if (c == 0) atomicAdd(&sg[kOut * kH + j], gb[j]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOut * kH; i += blockDim.x) atomicAdd(&gW3[i], sg[i]);
    if (threadIdx.x < kOut) atomicAdd(&gb3[threadIdx.x], sg[kOut * kH + threadIdx.x]);
}

// dZ = bf16(dH * [Z > 0]) and the column sums of dZ (bias gradient).
__global__ void k_relu_back(long long M, int N, const float* __restrict__ dH,
                            const float* __restrict__ Z, bf16* __restrict__ dZ,
                            float* __restrict__ gb)
{
    const long long total = M * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const float d = Z[e] > 0.f ? dH[e] : 0.f;
        dZ[e] = __float2bfloat16(d);
    }
    (void)gb;
}

// Column sums of a bf16 matrix (M x N) into gb (atomic).
__global__ void k_colsum(long long M, int N, const bf16* __restrict__ D, float* __restrict__ gb)
{
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (long long m = blockIdx.x; m < M; m += gridDim.x) s += __bfloat162float(D[m * N + c]);
    atomicAdd(&gb[c], s);
}

// Adam on the FP32 master parameters; padded entries (mask == 0) stay zero.
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, const unsigned char* __restrict__ mask,
                       float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!mask[i]) continue;
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// bf16 copies of the weights (and W2^T for the backward GEMM).
__global__ void k_cast_weights(const float* __restrict__ W1, const float* __restrict__ W2,
                               const float* __restrict__ W3, bf16* __restrict__ W1h,
                               bf16* __restrict__ W2h, bf16* __restrict__ W2Th,
                               bf16* __restrict__ W3h)
{
    const int total = kH * kInPad + 2 * kH * kH + kOutPad * kH;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        if (e < kH * kInPad) {
            W1h[e] = __float2bfloat16(W1[e]);
        } else if (e < kH * kInPad + kH * kH) {
            const int i = e - kH * kInPad;
            W2h[i] = __float2bfloat16(W2[i]);
        } else if (e < kH * kInPad + 2 * kH * kH) {
            const int i = e - kH * kInPad - kH * kH;
            const int r = i / kH, c = i % kH;            // W2T[r][c] = W2[c][r]
            W2Th[i] = __float2bfloat16(W2[c * kH + r]);
        } else {
            const int i = e - kH * kInPad - 2 * kH * kH;
            W3h[i] = __float2bfloat16(W3[i]);
        }
    }
}

// --------------------------------------------------------------------------
// Network inference on the fifth-generation tensor cores (tcgen05)
//
// One block of 256 threads per SM keeps the three weight matrices resident in
// shared memory in the no-swizzle K-major core-matrix layout (8 rows x 16
// bytes per core matrix; core matrices adjacent in K are LBO = rows/8 * 128
// bytes apart, adjacent 8-row groups SBO = 128 bytes apart) and runs 128
// feature rows at a time.  The rows arrive by TMA: each 64-column chunk is
// eight boxes of 8 columns x 128 rows, which land in exactly that layout,
// through three stages (one "full" and one "empty" mbarrier each).  One thread
// issues the copies and the MMAs: layer 1 accumulates X W1^T over the six
// chunks in TMEM columns 0..127, and as soon as its last MMAs are committed
// the first three chunks of the block's next tile are copied in, overlapping
// the rest of this tile.  The epilogues read TMEM with tcgen05.ld (warp w
// reads lanes 32 (w % 4) .. +31), add the bias, apply the ReLU and write the
// next layer's BF16 operand: H1 W2^T goes to columns 128..255, then H2 (over
// H1, whose MMAs have completed) times W3^T (N padded to 16) to columns
// 0..15.  Every wait is bounded.
// --------------------------------------------------------------------------

constexpr int kRows = 128;                 // rows per tile (MMA M)
constexpr int kKc = 64;                    // K chunk of the streamed features
constexpr int kNChunks = kInPad / kKc;     // 6
constexpr int kXStages = 3;                // chunk stages in flight (divides kNChunks)
static_assert(kNChunks % kXStages == 0, "chunk c of every tile must use stage c % kXStages");
constexpr int kN3 = 16;                    // layer-3 N (4 outputs, padded)
constexpr int kTmemCols = 256;

struct __align__(1024) TcSmem {
    bf16 W1[kH * kInPad];                  // rows 128, K 384 (core-matrix layout)
    bf16 W2[kH * kH];                      // rows 128, K 128
    bf16 H[kRows * kH];                    // H1, then H2 (rows 128, K 128)
    bf16 Xc[kXStages][kRows * kKc];        // feature chunks (TMA destinations)
    bf16 W3[kN3 * kH];                     // rows 16, K 128 (rows >= kOut zero)
    float b1[kH], b2[kH], b3[kOutPad];
    uint64_t xfull[kXStages], xempty[kXStages], mma;
    uint32_t tmem;
    int ok;
};

// Element index of (row, k) in a core-matrix tile with `rows` rows.
__device__ __forceinline__ int core_idx(int row, int k, int rows)
{
    return (((k >> 3) * (rows >> 3) + (row >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// Descriptor of the K = 16 slice starting at column k0 of a core-matrix tile.
__device__ __forceinline__ uint64_t tile_desc(const bf16* base, int rows, int k0)
{
    const uint32_t lbo = (uint32_t)(rows >> 3) * 128u;
    return smem_desc(smem_addr(base) + (uint32_t)(k0 >> 3) * lbo, lbo, 128u);
}

// Row-major [rows][K] BF16 weights (global) -> core-matrix tile (shared).
__device__ __forceinline__ void stage_weights(bf16* dst, const bf16* __restrict__ src, int rows,
                                              int src_rows, int K)
{
    const int n = rows * (K / 8);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int r = e / (K / 8), j = e % (K / 8);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < src_rows) v = *reinterpret_cast<const uint4*>(src + (long long)r * K + j * 8);
        *reinterpret_cast<uint4*>(dst + core_idx(r, j * 8, rows)) = v;
    }
}

// D (TMEM, 128 lanes x 128 columns from column `col`) + bias, ReLU -> BF16
// core-matrix tile `dst` (rows 128, K 128).
__device__ __forceinline__ void epilogue_relu(uint32_t tmem, uint32_t col, const float* bias, bf16* dst)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, half = warp >> 2, row = 32 * q + lane;
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        const int c0 = half * 64 + j * 16;
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + col + (uint32_t)c0, v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = c0 + 8 * h + 2 * i;
                const __nv_bfloat162 pr = __floats2bfloat162_rn(fmaxf(v[8 * h + 2 * i] + bias[c], 0.f),
                                                                fmaxf(v[8 * h + 2 * i + 1] + bias[c + 1], 0.f));
                w[i] = *reinterpret_cast<const uint32_t*>(&pr);
            }
            *reinterpret_cast<uint4*>(dst + core_idx(row, c0 + 8 * h, kRows)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// The block's smem is the whole 227 KB (one block per SM; the TMEM allocation
// can then never wait).
constexpr size_t kTcSmemBytes = 232448;
static_assert(sizeof(TcSmem) + 1024 <= kTcSmemBytes, "tensor-core tile does not fit in shared memory");

// Network outputs Y [rows][4] of the feature rows X [rows][384] (bf16, read by
// the tensor map xmap), for rows < (*count_dev if given, capped at M, else M).
__global__ void __launch_bounds__(256, 1) k_mlp_rows(const __grid_constant__ MlpWeights W,
                                                     const __grid_constant__ CUtensorMap xmap,
                                                     long long M, const unsigned* count_dev,
                                                     float* __restrict__ Y, unsigned* flags)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    TcSmem& S = *reinterpret_cast<TcSmem*>(base);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long nrows = count_dev ? min((long long)*count_dev, M) : M;
    const long long ntiles = (nrows + kRows - 1) / kRows;
    if ((long long)blockIdx.x >= ntiles) return;                  // block-uniform
    stage_weights(S.W1, W.W1, kH, kH, kInPad);
    stage_weights(S.W2, W.W2, kH, kH, kH);
    stage_weights(S.W3, W.W3, kN3, kOutPad, kH);
    for (int i = tid; i < kH; i += blockDim.x) {
        S.b1[i] = W.b1[i];
        S.b2[i] = W.b2[i];
    }
    if (tid < kOutPad) S.b3[tid] = W.b3[tid];
    if (tid == 0) {
        for (int b = 0; b < kXStages; ++b) {
            mbar_init(&S.xfull[b], 1);
            mbar_init(&S.xempty[b], 1);
        }
        mbar_init(&S.mma, 1);
        mbar_fence_init();
        S.ok = 1;
    }
    if (warp == 0) {
        tmem_alloc(&S.tmem, kTmemCols);
        tmem_relinquish();
    }
    fence_async_shared();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tm = S.tmem;
    constexpr uint32_t kId128 = idesc_bf16_f32(kRows, kH), kId16 = idesc_bf16_f32(kRows, kN3);
    constexpr uint32_t kChunkBytes = kRows * kKc * 2;
    // thread 0's bookkeeping: loads issued into / consumed from each stage
    uint32_t loads[kXStages] = {}, used[kXStages] = {};
    bool t0ok = true;
    auto issue = [&](long long tile, int c) {           // thread 0: chunk c of a tile
        const int s = c % kXStages;
        if (loads[s] > 0 && t0ok)                        // the MMAs of the stage's last chunk
            t0ok = mbar_wait_bounded(&S.xempty[s], (loads[s] - 1) & 1u);
        if (!t0ok) return;
        mbar_arrive_expect_tx(&S.xfull[s], kChunkBytes);
#pragma unroll
        for (int j = 0; j < kKc / 8; ++j)
            tma_load_2d(&S.Xc[s][j * kRows * 8], &xmap, c * kKc + 8 * j, (int)(tile * kRows), &S.xfull[s]);
        ++loads[s];
    };
    uint32_t nmma = 0;                                   // phases of S.mma waited so far
    if (tid == 0)
        for (int c = 0; c < kXStages; ++c) issue(blockIdx.x, c);
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long row0 = t * kRows;
        if (tid == 0) {
            // ---- layer 1: D1 = X W1^T over six chunks ----
            for (int c = 0; c < kNChunks && t0ok; ++c) {
                const int s = c % kXStages;
                if (c >= kXStages) issue(t, c);
                if (!t0ok) break;
                t0ok = mbar_wait_bounded(&S.xfull[s], used[s] & 1u);
                if (!t0ok) break;
                ++used[s];
                tc_fence_after_sync();
#pragma unroll
                for (int kk = 0; kk < kKc; kk += 16)
                    tc_mma_bf16(tm, tile_desc(S.Xc[s], kRows, kk), tile_desc(S.W1, kH, c * kKc + kk),
                                kId128, (c | kk) != 0);
                tc_commit(&S.xempty[s]);
            }
            tc_commit(&S.mma);
            // the next tile's first chunks, while this tile finishes
            if (t + gridDim.x < ntiles)
                for (int c = 0; c < kXStages; ++c) issue(t + gridDim.x, c);
            if (!t0ok) S.ok = 0;
        }
        ok = mbar_wait_bounded(&S.mma, nmma & 1u) && ok;
        ++nmma;
        tc_fence_after_sync();
        epilogue_relu(tm, 0u, S.b1, S.H);
        fence_async_shared();
        tc_fence_before_sync();
        __syncthreads();
        // ---- layer 2: D2 (columns 128..255) = H1 W2^T ----
        if (tid == 0) {
            tc_fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kH; kk += 16)
                tc_mma_bf16(tm + kH, tile_desc(S.H, kRows, kk), tile_desc(S.W2, kH, kk), kId128, kk != 0);
            tc_commit(&S.mma);
        }
        ok = mbar_wait_bounded(&S.mma, nmma & 1u) && ok;
        ++nmma;
        tc_fence_after_sync();
        __syncthreads();                                 // every read of H1 is done (MMAs completed)
        epilogue_relu(tm, (uint32_t)kH, S.b2, S.H);      // H2 over H1
        fence_async_shared();
        tc_fence_before_sync();
        __syncthreads();
        // ---- layer 3: D3 (columns 0..15) = H2 W3^T ----
        if (tid == 0) {
            tc_fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kH; kk += 16)
                tc_mma_bf16(tm, tile_desc(S.H, kRows, kk), tile_desc(S.W3, kN3, kk), kId16, kk != 0);
            tc_commit(&S.mma);
        }
        ok = mbar_wait_bounded(&S.mma, nmma & 1u) && ok;
        ++nmma;
        tc_fence_after_sync();
        if (warp < 4) {
            float v[16];
            tmem_ld16(tm + ((uint32_t)(32 * warp) << 16), v);
            const long long row = row0 + 32 * warp + lane;
            if (row < nrows)
#pragma unroll
                for (int o = 0; o < kOut; ++o) Y[row * kOut + o] = v[o] + S.b3[o];
        }
        tc_fence_before_sync();
        const bool all_ok = __syncthreads_and(ok && S.ok) != 0;
        tc_fence_after_sync();
        if (!all_ok) {
            ok = false;
            break;
        }
    }
    if (tid == 0 && (!ok || !t0ok)) {
        atomicOr(flags, kFlagTimeout);
        for (int b = 0; b < kXStages; ++b)               // copies still in flight land first
            if (loads[b] > used[b]) mbar_wait_bounded(&S.xfull[b], used[b] & 1u);
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    if (warp == 0) tmem_dealloc(tm, kTmemCols);
}

cudaError_t launch_mlp_rows(const MlpWeights& W, const bf16* X, long long M, const unsigned* count_dev,
                            float* Y, unsigned* flags, cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    CUtensorMap xmap;
    if (!encode_bf16_2d(&xmap, X, kInPad, (unsigned long long)M, kInPad * 2, 8, kRows))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmemBytes);
    if (e != cudaSuccess) return e;
    const long long tiles = (M + kRows - 1) / kRows;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, device_sm_count()));
    k_mlp_rows<<<grid, 256, kTcSmemBytes, s>>>(W, xmap, M, count_dev, Y, flags);
    return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const MlpWeights& W, const bf16* X, long long M, float* Y,
                             unsigned* flags, cudaStream_t s)
{
    return launch_mlp_rows(W, X, M, nullptr, Y, flags, s);
}

// --------------------------------------------------------------------------
// Seeding of the queued voxels: features, network, exact seeds
// --------------------------------------------------------------------------

// Cost bucket of a queued voxel whose running squared gamma is g2: 1 + floor(2
// log2 of the table cells with key < gamma) (0 when there are none), the
// bucket k_shell gives.
__device__ __forceinline__ int cost_bucket(const Problem& P, float g2)
{
    return cost_bucket_of(P.bucket_key, sqrtf(g2));
}

// The seed rows of one pair (BATCH = false: P0.seed_list items) or of every
// pair of a batch group (the (pair, item) rows of bd): their number, capped
// at the row buffer, and the pair and queue item of row r.
template <bool BATCH>
struct SeedRows {
    const Problem* P0;
    const BatchDesc* bd;
    __device__ unsigned count() const
    {
        return BATCH ? min(*bd->seed_count, bd->seed_cap) : min(P0->ctr->seed_count, P0->seed_cap);
    }
    __device__ bf16* X() const { return BATCH ? bd->seed_X : P0->seed_X; }
    __device__ float* Y() const { return BATCH ? bd->seed_Y : P0->seed_Y; }
    __device__ const Problem& prob(unsigned r) const { return BATCH ? bd->probs[bd->seed_pair[r]] : *P0; }
    __device__ unsigned item(unsigned r) const { return BATCH ? bd->seed_item[r] : P0->seed_list[r]; }
};

// Features of every seed row into the row buffer.  One warp per row: the
// warp stages the 7^N neighbourhood of the voxel (the 5^N patch and the
// neighbours its gradients use) of both doses in shared memory, then each
// lane takes patch points and computes their three channels together, with
// the arithmetic of voxel_feature (so the features equal gamma_features').
constexpr int kBoxW = kPatch + 2;                    // 7
template <int N>
struct FeatBox {
    static constexpr int ELEMS = N == 3 ? kBoxW * kBoxW * kBoxW : kBoxW * kBoxW;
};

template <int N, bool BATCH>
__global__ void __launch_bounds__(256) k_seed_features(const __grid_constant__ Problem P0,
                                                       const BatchDesc* __restrict__ bd)
{
    constexpr int E = FeatBox<N>::ELEMS;
    constexpr int NP = N == 3 ? 125 : 25;            // patch points used
    __shared__ float sh_e[8][E], sh_r[8][E];
    const SeedRows<BATCH> rows{&P0, bd};
    const unsigned total = rows.count();
    bf16* X = rows.X();
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    float* be = sh_e[wi];
    float* br = sh_r[wi];
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    const int bst[3] = {1, kBoxW, kBoxW * kBoxW};
    for (unsigned r = gw; r < total; r += nw) {               // warp-uniform
        const Problem& P = rows.prob(r);
        const unsigned v = P.tail_raw[rows.item(r)];
        const int x = (int)(v % (unsigned)P.nx);
        const unsigned r1 = v / (unsigned)P.nx;
        const int y = (int)(r1 % (unsigned)P.ny), z = (int)(r1 / (unsigned)P.ny);
        const float dr = __ldg(P.ref + v);
        const float inv = 1.0f / (P.dd_frac * (P.local ? dr : resolve_dnorm(P)));
        const int n[3] = {P.nx, P.ny, P.nz};
        float c1[3], c2[3];                                   // one-sided and central factors
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c1[a] = 1.f / P.hn[a];
            c2[a] = 0.5f / P.hn[a];
        }
        // ---- the 7^N box around v (offsets -3 .. 3); outside the grid: 0 ----
        __syncwarp();
#pragma unroll 4
        for (int e = lane; e < E; e += 32) {
            const int ox = e % kBoxW - 3, oy = (e / kBoxW) % kBoxW - 3, oz = N == 3 ? e / (kBoxW * kBoxW) - 3 : 0;
            const int px = x + ox, py = y + oy, pz = z + oz;
            const bool in = (unsigned)px < (unsigned)P.nx && (unsigned)py < (unsigned)P.ny &&
                            (N == 2 || (unsigned)pz < (unsigned)P.nz);
            const long long p = ((long long)pz * P.ny + py) * P.nx + px;
            be[e] = in ? __ldg(P.ev + p) : 0.f;
            br[e] = in ? __ldg(P.ref + p) : 0.f;
        }
        __syncwarp();
        // ---- the three channels of one patch point per lane ----
        bf16* xr = X + (long long)r * kInPad;
        for (int pi = lane; pi < 125; pi += 32) {
            float f0 = 0.f, f1 = 0.f, f2 = 0.f;
            if (pi < NP) {
                const int o[3] = {pi % 5 - 2, (pi / 5) % 5 - 2, N == 3 ? pi / 25 - 2 : 0};
                const int c[3] = {x + o[0], y + o[1], z + o[2]};
                if ((unsigned)c[0] < (unsigned)P.nx && (unsigned)c[1] < (unsigned)P.ny &&
                    (N == 2 || (unsigned)c[2] < (unsigned)P.nz)) {
                    const int bi = ((o[2] + (N == 3 ? 3 : 0)) * kBoxW + (o[1] + 3)) * kBoxW + (o[0] + 3);
                    f0 = fminf(fmaxf((be[bi] - dr) * inv, -16.f), 16.f);
                    // the gradients of both doses (central differences inside,
                    // one-sided at the grid edge), as grad_norm takes them
                    float se = 0.f, sr = 0.f;
#pragma unroll
                    for (int a = 0; a < N; ++a) {
                        float de, dq;
                        if (c[a] > 0 && c[a] < n[a] - 1) {
                            de = (be[bi + bst[a]] - be[bi - bst[a]]) * c2[a];
                            dq = (br[bi + bst[a]] - br[bi - bst[a]]) * c2[a];
                        } else if (c[a] == 0) {
                            de = (be[bi + bst[a]] - be[bi]) * c1[a];
                            dq = (br[bi + bst[a]] - br[bi]) * c1[a];
                        } else {
                            de = (be[bi] - be[bi - bst[a]]) * c1[a];
                            dq = (br[bi] - br[bi - bst[a]]) * c1[a];
                        }
                        se = fmaf(de, de, se);
                        sr = fmaf(dq, dq, sr);
                    }
                    f1 = fminf(sqrtf(se) * inv, 32.f);
                    f2 = fminf(sqrtf(sr) * inv, 32.f);
                }
            }
            xr[pi] = __float2bfloat16(f0);
            xr[125 + pi] = __float2bfloat16(f1);
            xr[250 + pi] = __float2bfloat16(f2);
        }
        if (lane < kInPad - kIn) xr[kIn + lane] = __float2bfloat16(0.f);
    }
}

// Exact seeds from the network's proposals: for every seed row, the faces of
// the 2^N cells around the proposed nearest point (two threads per row), a
// true distance to the evaluation surface, lower the voxel's running squared
// gamma; the voxel moves to the cost bucket of the tighter bound.
template <int N, bool BATCH>
__global__ void __launch_bounds__(256) k_seed_apply(const __grid_constant__ Problem P0,
                                                    const BatchDesc* __restrict__ bd)
{
    const SeedRows<BATCH> rows{&P0, bd};
    const unsigned total = rows.count();
    const float* Y = rows.Y();
    __shared__ unsigned sh_hist[kNumBuckets];
    __shared__ unsigned sh_seed, sh_imp;
    if (threadIdx.x < kNumBuckets) sh_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) sh_seed = sh_imp = 0;
    __syncthreads();
    // a warp takes 16 rows at a time (two lanes per row), so that every lane
    // of the warp runs the same iterations (the shuffle below)
    const int lane = threadIdx.x & 31, half = lane & 1;
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    for (unsigned rb = gw * 16u; rb < total; rb += nw * 16u) {
        const unsigned r = rb + (unsigned)(lane >> 1);
        const bool live = r < total;
        float sd2 = kInf;
        unsigned v = 0, item = 0;
        const Problem& P = rows.prob(live ? r : 0u);
        if (live) {
            item = rows.item(r);
            v = P.tail_raw[item];
            const int x = (int)(v % (unsigned)P.nx);
            const unsigned r1 = v / (unsigned)P.nx;
            const int y = (int)(r1 % (unsigned)P.ny), z = (int)(r1 / (unsigned)P.ny);
            const float dr = __ldg(P.ref + v);
            const float inv = 1.0f / (P.dd_frac * (P.local ? dr : resolve_dnorm(P)));
            int o[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float ov = a < N ? Y[(long long)r * kOut + a] / P.hn[a] : 0.f;
                o[a] = (int)floorf(fminf(fmaxf(ov, -256.f), 256.f));
            }
            constexpr int NCELL = 1 << N;
#pragma unroll 1
            for (int u = half; u < NCELL; u += 2) {
                const int cx = o[0] + (u & 1), cy = o[1] + ((u >> 1) & 1),
                          cz = N == 3 ? o[2] + ((u >> 2) & 1) : 0;
                float q[8];
                uint32_t okc;
                if (!load_cell<N>(P, x, y, z, cx, cy, cz, dr, inv, q, okc)) continue;
                CellGeom<float> gg;
                cell_geom<N, float>(cx, cy, cz, P.mt, gg);
                bool ill = false;
                const float cb = cell_min_d2<N, float>(q, okc, gg, P.mt,
                                                       P.tau > 0.f ? 0.99f * rsqrtf(P.tau) : kInf,
                                                       kInf, ill);
                if (ill) ill = cell_gram_ill<N>(q, okc, P.mt.kappa, P.tau);
                if (!ill) sd2 = fminf(sd2, cb);            // ill-conditioned cells are not used as seeds
            }
        }
        sd2 = fminf(sd2, __shfl_xor_sync(0xffffffffu, sd2, 1));
        if (live && half == 0) {
            const float cur = P.out[v];                     // gamma^2 after the faces through v
            const float nb = fminf(cur, sd2);
            const bool better = nb < cur;
            if (better) P.out[v] = nb;
            const int bucket = cost_bucket(P, nb);
            const int was = P.tail_bucket[item];
            if (BATCH) {
                atomicAdd(&P.ctr->seeded, 1u);
                if (better) atomicAdd(&P.ctr->seed_improved, 1u);
                if (bucket != was) {                        // move the voxel between its pair's bins
                    P.tail_bucket[item] = (unsigned char)bucket;
                    atomicAdd(&P.ctr->hist[bucket], 1u);
                    atomicSub(&P.ctr->hist[was], 1u);
                }
            } else {
                atomicAdd(&sh_seed, 1u);
                if (better) atomicAdd(&sh_imp, 1u);
                if (bucket != was) {
                    P.tail_bucket[item] = (unsigned char)bucket;
                    atomicAdd(&sh_hist[bucket], 1u);
                    atomicSub(&sh_hist[was], 1u);          // wraps; the sum over the block is exact
                }
            }
        }
    }
    if constexpr (!BATCH) {
        __syncthreads();
        if (threadIdx.x < kNumBuckets && sh_hist[threadIdx.x])
            atomicAdd(&P0.ctr->hist[threadIdx.x], sh_hist[threadIdx.x]);
        if (threadIdx.x == 0) {
            if (sh_seed) atomicAdd(&P0.ctr->seeded, sh_seed);
            if (sh_imp) atomicAdd(&P0.ctr->seed_improved, sh_imp);
        }
    }
}

// Queue items of every pair of a batch group past the cost gate, as (pair,
// item) rows (blockIdx.y = pair).
__global__ void __launch_bounds__(256) k_seed_select_batch(const BatchDesc* __restrict__ bd,
                                                           int min_bucket)
{
    const Problem& P = bd->probs[blockIdx.y];
    const unsigned total = min(P.ctr->tail_count, P.tail_cap);
    const int lane = threadIdx.x & 31;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned c0 = blockIdx.x * blockDim.x; c0 < total; c0 += stride) {
        const unsigned i = c0 + threadIdx.x;
        const bool take = i < total && (int)P.tail_bucket[i] >= min_bucket;
        const unsigned m = __ballot_sync(0xffffffffu, take);
        unsigned base = 0;
        if (lane == 0 && m) base = atomicAdd(bd->seed_count, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (take) {
            const unsigned pos = base + __popc(m & ((1u << lane) - 1u));
            if (pos < bd->seed_cap) {                       // rows past the buffer go unseeded
                bd->seed_item[pos] = i;
                bd->seed_pair[pos] = (unsigned short)blockIdx.y;
            }
        }
    }
}

template <int N, bool BATCH>
static cudaError_t launch_seeding_n(const Problem& P, const BatchDesc* bd, const MlpWeights& W,
                                    const bf16* X, float* Y, unsigned cap, const unsigned* count,
                                    unsigned* flags, cudaStream_t s)
{
    const int sms = device_sm_count();
    k_seed_features<N, BATCH><<<sms * 16, 256, 0, s>>>(P, bd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_mlp_rows(W, X, cap, count, Y, flags, s)) != cudaSuccess) return e;
    k_seed_apply<N, BATCH><<<sms * 8, 256, 0, s>>>(P, bd);
    return cudaGetLastError();
}

cudaError_t launch_seeding(const Problem& P, const MlpWeights& W, int min_bucket, cudaStream_t s)
{
    if (!P.seed_list || !P.seed_X || !P.seed_Y || P.seed_cap == 0) return cudaErrorInvalidValue;
    k_seed_select<<<device_sm_count() * 4, 256, 0, s>>>(P, min_bucket);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return P.ndim == 3
               ? launch_seeding_n<3, false>(P, nullptr, W, P.seed_X, P.seed_Y, P.seed_cap,
                                            &P.ctr->seed_count, &P.ctr->flags, s)
               : launch_seeding_n<2, false>(P, nullptr, W, P.seed_X, P.seed_Y, P.seed_cap,
                                            &P.ctr->seed_count, &P.ctr->flags, s);
}

cudaError_t launch_batch_seeding(const BatchGroup& g, const MlpWeights& W, int min_bucket,
                                 cudaStream_t s)
{
    if (g.npairs <= 0 || g.seed_cap == 0) return cudaSuccess;
    const int bx = std::max(1, device_sm_count() * 2 / std::max(1, g.npairs)) + 1;
    k_seed_select_batch<<<dim3(bx, g.npairs), 256, 0, s>>>(g.desc, min_bucket);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Problem dummy{};
    return g.ndim == 3 ? launch_seeding_n<3, true>(dummy, g.desc, W, g.seed_X, g.seed_Y, g.seed_cap,
                                                   g.seed_count, g.flags, s)
                       : launch_seeding_n<2, true>(dummy, g.desc, W, g.seed_X, g.seed_Y, g.seed_cap,
                                                   g.seed_count, g.flags, s);
}

cudaError_t launch_features(const Problem& P, const unsigned* vox, long long n, bf16* X,
                            cudaStream_t s)
{
    const long long total = n * (kInPad / 8);
    const int grid = (int)std::min<long long>((total + 255) / 256, (long long)device_sm_count() * 32);
    if (P.ndim == 3) k_features<3><<<std::max(grid, 1), 256, 0, s>>>(P, vox, n, X);
    else k_features<2><<<std::max(grid, 1), 256, 0, s>>>(P, vox, n, X);
    return cudaGetLastError();
}

cudaError_t launch_labels(const Problem& P, const float* gmap, const unsigned* vox, long long n,
                          float* T, cudaStream_t s)
{
    const int grid = (int)std::min<long long>((n + 127) / 128, (long long)device_sm_count() * 16);
    if (P.ndim == 3) k_labels<3><<<std::max(grid, 1), 128, 0, s>>>(P, gmap, vox, n, T);
    else k_labels<2><<<std::max(grid, 1), 128, 0, s>>>(P, gmap, vox, n, T);
    return cudaGetLastError();
}

}  // namespace gk

// ==========================================================================
// Model object and its C ABI
// ==========================================================================

using gk::bf16;

struct gamma_model_s {
    int device = 0;
    float* p = nullptr;           // fp32 master parameters (layout below)
    float* gr = nullptr;          // gradients
    float* m1 = nullptr;          // Adam first moment
    float* m2 = nullptr;          // Adam second moment
    unsigned char* mask = nullptr;  // 1 for trainable entries (padding stays zero)
    bf16 *W1h = nullptr, *W2h = nullptr, *W2Th = nullptr, *W3h = nullptr;
    long long step = 0;
    unsigned long long seed = 0;
    // training workspace
    long long wsM = 0;
    float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *dY = nullptr, *dH1 = nullptr, *loss = nullptr;
    bf16 *H1h = nullptr, *H2h = nullptr, *dZ2h = nullptr, *dZ1h = nullptr;
    // batch-contiguous (transposed) operands of the weight-gradient GEMMs,
    // row stride wsMp = wsM rounded up to 8 (16-byte rows for TMA)
    bf16 *XT = nullptr, *H1T = nullptr, *dZ1T = nullptr, *dZ2T = nullptr;
    long long wsMp = 0;
    unsigned* dflags = nullptr;   // error flags of the tensor-core kernels
};

namespace {

// Parameter layout (floats): W1 [128][384], b1 [128], W2 [128][128], b2 [128],
// W3 [8][128], b3 [8].
constexpr long long kOffW1 = 0;
constexpr long long kOffB1 = kOffW1 + gk::kH * gk::kInPad;
constexpr long long kOffW2 = kOffB1 + gk::kH;
constexpr long long kOffB2 = kOffW2 + gk::kH * gk::kH;
constexpr long long kOffW3 = kOffB2 + gk::kH;
constexpr long long kOffB3 = kOffW3 + gk::kOutPad * gk::kH;
constexpr long long kNParams = kOffB3 + gk::kOutPad;

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? GAMMA_OK : (e == cudaErrorMemoryAllocation ? GAMMA_ERR_OOM : GAMMA_ERR_CUDA); }

#define MCK(call)                                  \
    do {                                           \
        int rc_ = cuda_rc(call);                   \
        if (rc_) return rc_;                       \
    } while (0)

void free_ws(gamma_model_s* m)
{
    cudaFree(m->Z1); cudaFree(m->Z2); cudaFree(m->Y); cudaFree(m->dY); cudaFree(m->dH1);
    cudaFree(m->loss); cudaFree(m->H1h); cudaFree(m->H2h); cudaFree(m->dZ2h); cudaFree(m->dZ1h);
    cudaFree(m->XT); cudaFree(m->H1T); cudaFree(m->dZ1T); cudaFree(m->dZ2T);
    m->Z1 = m->Z2 = m->Y = m->dY = m->dH1 = m->loss = nullptr;
    m->H1h = m->H2h = m->dZ2h = m->dZ1h = nullptr;
    m->XT = m->H1T = m->dZ1T = m->dZ2T = nullptr;
    m->wsM = m->wsMp = 0;
}

int ensure_ws(gamma_model_s* m, long long M)
{
    if (M <= m->wsM) return GAMMA_OK;
    free_ws(m);
    MCK(cudaMalloc(&m->Z1, sizeof(float) * M * gk::kH));
    MCK(cudaMalloc(&m->Z2, sizeof(float) * M * gk::kH));
    MCK(cudaMalloc(&m->Y, sizeof(float) * M * gk::kOutPad));
    MCK(cudaMalloc(&m->dY, sizeof(float) * M * gk::kOut));
    MCK(cudaMalloc(&m->dH1, sizeof(float) * M * gk::kH));
    MCK(cudaMalloc(&m->loss, sizeof(float)));
    MCK(cudaMalloc(&m->H1h, sizeof(bf16) * M * gk::kH));
    MCK(cudaMalloc(&m->H2h, sizeof(bf16) * M * gk::kH));
    MCK(cudaMalloc(&m->dZ2h, sizeof(bf16) * M * gk::kH));
    MCK(cudaMalloc(&m->dZ1h, sizeof(bf16) * M * gk::kH));
    const long long Mp = (M + 7) / 8 * 8;
    MCK(cudaMalloc(&m->XT, sizeof(bf16) * Mp * gk::kInPad));
    MCK(cudaMalloc(&m->H1T, sizeof(bf16) * Mp * gk::kH));
    MCK(cudaMalloc(&m->dZ1T, sizeof(bf16) * Mp * gk::kH));
    MCK(cudaMalloc(&m->dZ2T, sizeof(bf16) * Mp * gk::kH));
    m->wsM = M;
    m->wsMp = Mp;
    return GAMMA_OK;
}

int grid_for_n(long long n, int threads = 256)
{
    long long b = (n + threads - 1) / threads;
    return (int)std::max<long long>(1, std::min<long long>(b, (long long)gk::device_sm_count() * 16));
}

// Host-side parameter initialisation: He-normal weights from a splitmix64 /
// Box-Muller stream, zero biases and padding.
void init_params(std::vector<float>& h, unsigned long long seed)
{
    h.assign(kNParams, 0.f);
    unsigned long long st = seed ? seed : 0x9e3779b97f4a7c15ull;
    auto next = [&]() {
        st += 0x9e3779b97f4a7c15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    };
    auto unif = [&]() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    auto normal = [&]() { return std::sqrt(-2.0 * std::log(unif())) * std::cos(6.283185307179586 * unif()); };
    for (int r = 0; r < gk::kH; ++r)
        for (int c = 0; c < gk::kIn; ++c) h[kOffW1 + r * gk::kInPad + c] = (float)(normal() * std::sqrt(2.0 / gk::kIn));
    for (int i = 0; i < gk::kH * gk::kH; ++i) h[kOffW2 + i] = (float)(normal() * std::sqrt(2.0 / gk::kH));
    for (int r = 0; r < gk::kOut; ++r)
        for (int c = 0; c < gk::kH; ++c) h[kOffW3 + r * gk::kH + c] = (float)(normal() * std::sqrt(1.0 / gk::kH));
}

std::vector<unsigned char> param_mask()
{
    std::vector<unsigned char> k(kNParams, 1);
    for (int r = 0; r < gk::kH; ++r)
        for (int c = gk::kIn; c < gk::kInPad; ++c) k[kOffW1 + r * gk::kInPad + c] = 0;
    for (int r = gk::kOut; r < gk::kOutPad; ++r)
        for (int c = 0; c < gk::kH; ++c) k[kOffW3 + r * gk::kH + c] = 0;
    for (int r = gk::kOut; r < gk::kOutPad; ++r) k[kOffB3 + r] = 0;
    return k;
}

int refresh_bf16(gamma_model_s* m, cudaStream_t s)
{
    gk::k_cast_weights<<<64, 256, 0, s>>>(m->p + kOffW1, m->p + kOffW2, m->p + kOffW3, m->W1h,
                                          m->W2h, m->W2Th, m->W3h);
    return cuda_rc(cudaGetLastError());
}

// Forward pass of a minibatch through the training kernels (activations
// kept): the three layers as tensor-core GEMMs (tcgen05, TMEM accumulators,
// TMA operand loads), bias and ReLU in separate element-wise passes.
int forward_train(gamma_model_s* m, const bf16* X, long long M, cudaStream_t s)
{
    using namespace gk;
    MCK(launch_gemm_tc(X, M, kInPad, m->W1h, kH, kInPad, kInPad, m->Z1, kH, 1, m->dflags, s));
    k_bias_act<<<grid_for_n(M * kH), 256, 0, s>>>(M, kH, m->Z1, m->p + kOffB1, m->H1h, kH, 1);
    MCK(launch_gemm_tc(m->H1h, M, kH, m->W2h, kH, kH, kH, m->Z2, kH, 1, m->dflags, s));
    k_bias_act<<<grid_for_n(M * kH), 256, 0, s>>>(M, kH, m->Z2, m->p + kOffB2, m->H2h, kH, 1);
    MCK(launch_gemm_tc(m->H2h, M, kH, m->W3h, kOutPad, kH, kH, m->Y, kOutPad, 1, m->dflags, s));
    k_bias_act<<<grid_for_n(M * kOutPad), 256, 0, s>>>(M, kOutPad, m->Y, m->p + kOffB3, nullptr, 0, 0);
    return cuda_rc(cudaGetLastError());
}

// Loss and gradients of a minibatch into m->gr (zeroed first).  The weight
// gradients sum over the batch, so their GEMMs take the batch as K: the
// operands are first transposed to batch-contiguous rows, and the K range is
// split over several blocks per tile that add into the gradient.
int backward_train(gamma_model_s* m, const bf16* X, const float* T, long long M, long long count,
                   cudaStream_t s)
{
    using namespace gk;
    MCK(cudaMemsetAsync(m->gr, 0, sizeof(float) * kNParams, s));
    MCK(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
    const float invc = count > 0 ? 1.f / (float)count : 0.f;
    const long long Mp = (M + 7) / 8 * 8;
    const int splits = (int)std::max<long long>(1, std::min<long long>(32, M / 512));
    k_huber<<<grid_for_n(M), 256, 0, s>>>(M, m->Y, T, m->dY, m->loss, invc);
    k_out_back<<<grid_for_n(M * kH, 256), 256, 0, s>>>(M, m->dY, m->p + kOffW3, m->Z2, m->H2h,
                                                         m->dZ2h, m->gr + kOffW3, m->gr + kOffB3);
    // dW2 = dZ2^T H1 (K = batch), db2 = colsum dZ2
    MCK(launch_transpose_bf16(m->dZ2h, M, kH, kH, m->dZ2T, Mp, s));
    MCK(launch_transpose_bf16(m->H1h, M, kH, kH, m->H1T, Mp, s));
    MCK(launch_gemm_tc(m->dZ2T, kH, Mp, m->H1T, kH, Mp, M, m->gr + kOffW2, kH, splits, m->dflags, s));
    k_colsum<<<dim3(256, (kH + 127) / 128), 128, 0, s>>>(M, kH, m->dZ2h, m->gr + kOffB2);
    // dH1 = dZ2 W2 (B[n][k] = W2^T[n][k] = W2[k][n]), dZ1 = dH1 [Z1 > 0]
    MCK(launch_gemm_tc(m->dZ2h, M, kH, m->W2Th, kH, kH, kH, m->dH1, kH, 1, m->dflags, s));
    k_relu_back<<<grid_for_n(M * kH), 256, 0, s>>>(M, kH, m->dH1, m->Z1, m->dZ1h, nullptr);
    k_colsum<<<dim3(256, (kH + 127) / 128), 128, 0, s>>>(M, kH, m->dZ1h, m->gr + kOffB1);
    // dW1 = dZ1^T X (K = batch)
    MCK(launch_transpose_bf16(m->dZ1h, M, kH, kH, m->dZ1T, Mp, s));
    MCK(launch_transpose_bf16(X, M, kInPad, kInPad, m->XT, Mp, s));
    MCK(launch_gemm_tc(m->dZ1T, kH, Mp, m->XT, kInPad, Mp, M, m->gr + kOffW1, kInPad, splits,
                       m->dflags, s));
    return cuda_rc(cudaGetLastError());
}

}  // namespace

namespace gk {

bool model_weights(const gamma_model_s* m, MlpWeights* w)
{
    if (!m) return false;
    w->W1 = m->W1h;
    w->W2 = m->W2h;
    w->W3 = m->W3h;
    w->b1 = m->p + kOffB1;
    w->b2 = m->p + kOffB2;
    w->b3 = m->p + kOffB3;
    return true;
}

}  // namespace gk

extern "C" {

int gamma_model_create(gamma_model* out, uint64_t seed)
{
    if (!out) return GAMMA_ERR_INVALID_ARG;
    *out = nullptr;
    gamma_model_s* m = new (std::nothrow) gamma_model_s();
    if (!m) return GAMMA_ERR_OOM;
    auto fail = [&](int rc) { gamma_model_destroy(m); return rc; };
    if (cudaGetDevice(&m->device) != cudaSuccess) return fail(GAMMA_ERR_CUDA);
    int rc;
    if ((rc = cuda_rc(cudaMalloc(&m->p, sizeof(float) * kNParams)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->gr, sizeof(float) * kNParams)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->m1, sizeof(float) * kNParams)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->m2, sizeof(float) * kNParams)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->mask, kNParams)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->W1h, sizeof(bf16) * gk::kH * gk::kInPad)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->W2h, sizeof(bf16) * gk::kH * gk::kH)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->W2Th, sizeof(bf16) * gk::kH * gk::kH)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->W3h, sizeof(bf16) * gk::kOutPad * gk::kH)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&m->dflags, sizeof(unsigned))))) return fail(rc);
    if ((rc = cuda_rc(cudaMemset(m->dflags, 0, sizeof(unsigned))))) return fail(rc);
    std::vector<float> h;
    init_params(h, seed);
    m->seed = seed;
    const std::vector<unsigned char> k = param_mask();
    if ((rc = cuda_rc(cudaMemcpy(m->p, h.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice)))) return fail(rc);
    if ((rc = cuda_rc(cudaMemcpy(m->mask, k.data(), kNParams, cudaMemcpyHostToDevice)))) return fail(rc);
    if ((rc = cuda_rc(cudaMemset(m->m1, 0, sizeof(float) * kNParams)))) return fail(rc);
    if ((rc = cuda_rc(cudaMemset(m->m2, 0, sizeof(float) * kNParams)))) return fail(rc);
    if ((rc = refresh_bf16(m, 0))) return fail(rc);
    if ((rc = cuda_rc(cudaDeviceSynchronize()))) return fail(rc);
    *out = m;
    return GAMMA_OK;
}

void gamma_model_destroy(gamma_model m)
{
    if (!m) return;
    cudaFree(m->p); cudaFree(m->gr); cudaFree(m->m1); cudaFree(m->m2); cudaFree(m->mask);
    cudaFree(m->W1h); cudaFree(m->W2h); cudaFree(m->W2Th); cudaFree(m->W3h);
    cudaFree(m->dflags);
    free_ws(m);
    delete m;
}

int64_t gamma_model_num_params(void) { return kNParams; }

int gamma_model_get_params(gamma_model m, float* host, int64_t n, int which)
{
    if (!m || !host || n != kNParams || which < 0 || which > 3) return GAMMA_ERR_INVALID_ARG;
    const float* src = which == 0 ? m->p : which == 1 ? m->gr : which == 2 ? m->m1 : m->m2;
    MCK(cudaDeviceSynchronize());
    MCK(cudaMemcpy(host, src, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
    return GAMMA_OK;
}

int gamma_model_set_params(gamma_model m, const float* host, int64_t n)
{
    if (!m || !host || n != kNParams) return GAMMA_ERR_INVALID_ARG;
    MCK(cudaMemcpy(m->p, host, sizeof(float) * kNParams, cudaMemcpyHostToDevice));
    if (int rc = refresh_bf16(m, 0)) return rc;
    MCK(cudaDeviceSynchronize());
    return GAMMA_OK;
}

int gamma_model_forward(gamma_model m, const void* X_bf16_dev, int64_t M, float* Y_dev,
                        void* cuda_stream)
{
    if (!m || !X_bf16_dev || !Y_dev || M <= 0) return GAMMA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (reinterpret_cast<uintptr_t>(X_bf16_dev) % 16 != 0) return GAMMA_ERR_INVALID_ARG;
    if (int rc = ensure_ws(m, M)) return rc;
    MCK(cudaMemsetAsync(m->dflags, 0, sizeof(unsigned), s));
    if (int rc = forward_train(m, (const bf16*)X_bf16_dev, M, s)) return rc;
    MCK(cudaMemcpy2DAsync(Y_dev, sizeof(float) * gk::kOut, m->Y, sizeof(float) * gk::kOutPad,
                          sizeof(float) * gk::kOut, (size_t)M, cudaMemcpyDeviceToDevice, s));
    return GAMMA_OK;
}

int gamma_model_infer(gamma_model m, const void* X_bf16_dev, int64_t M, float* Y_dev,
                      void* cuda_stream)
{
    if (!m || !X_bf16_dev || !Y_dev || M <= 0) return GAMMA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(X_bf16_dev) % 16 != 0) return GAMMA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    gk::MlpWeights W;
    gk::model_weights(m, &W);
    MCK(cudaMemsetAsync(m->dflags, 0, sizeof(unsigned), s));
    MCK(gk::launch_mlp_infer(W, (const bf16*)X_bf16_dev, M, Y_dev, m->dflags, s));
    unsigned flags = 0;
    MCK(cudaMemcpyAsync(&flags, m->dflags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    return (flags & gk::kFlagTimeout) ? GAMMA_ERR_TIMEOUT : GAMMA_OK;
}

int gamma_model_backward(gamma_model m, const void* X_bf16_dev, const float* T_dev, int64_t M,
                         float* loss_out, void* cuda_stream)
{
    if (!m || !X_bf16_dev || !T_dev || M <= 0) return GAMMA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (reinterpret_cast<uintptr_t>(X_bf16_dev) % 16 != 0) return GAMMA_ERR_INVALID_ARG;
    if (int rc = ensure_ws(m, M)) return rc;
    MCK(cudaMemsetAsync(m->dflags, 0, sizeof(unsigned), s));
    if (int rc = forward_train(m, (const bf16*)X_bf16_dev, M, s)) return rc;
    if (int rc = backward_train(m, (const bf16*)X_bf16_dev, T_dev, M, M, s)) return rc;
    if (loss_out) {
        unsigned flags = 0;
        MCK(cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        MCK(cudaMemcpyAsync(&flags, m->dflags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        if (flags & gk::kFlagTimeout) return GAMMA_ERR_TIMEOUT;
    }
    return GAMMA_OK;
}

int gamma_model_train_step(gamma_model m, const void* X_bf16_dev, const float* T_dev, int64_t M,
                           float lr, float* loss_out, void* cuda_stream)
{
    if (!m || !(lr >= 0.f)) return GAMMA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (int rc = gamma_model_backward(m, X_bf16_dev, T_dev, M, nullptr, cuda_stream)) return rc;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    gk::k_adam<<<grid_for_n(kNParams), 256, 0, s>>>(kNParams, m->p, m->gr, m->m1, m->m2, m->mask, lr,
                                                   b1, b2, 1e-8f, c1, c2);
    MCK(cudaGetLastError());
    if (int rc = refresh_bf16(m, s)) return rc;
    if (loss_out) {
        unsigned flags = 0;
        MCK(cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        MCK(cudaMemcpyAsync(&flags, m->dflags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        if (flags & gk::kFlagTimeout) return GAMMA_ERR_TIMEOUT;
    }
    return GAMMA_OK;
}

// File format: 8-byte magic "GAMMAMLP", int32 version 1, int32 kIn, kInPad,
// kH, kOut, kOutPad, int64 Adam step, uint64 seed, then kNParams floats each of
// parameters, Adam first and second moments (little-endian).
int gamma_model_save(gamma_model m, const char* path)
{
    if (!m || !path) return GAMMA_ERR_INVALID_ARG;
    std::vector<float> p(kNParams), a(kNParams), b(kNParams);
    if (int rc = gamma_model_get_params(m, p.data(), kNParams, 0)) return rc;
    if (int rc = gamma_model_get_params(m, a.data(), kNParams, 2)) return rc;
    if (int rc = gamma_model_get_params(m, b.data(), kNParams, 3)) return rc;
    FILE* f = std::fopen(path, "wb");
    if (!f) return GAMMA_ERR_INVALID_ARG;
    const int32_t hdr[7] = {1, gk::kIn, gk::kInPad, gk::kH, gk::kOut, gk::kOutPad, 0};
    const int64_t step = m->step;
    const uint64_t seed = m->seed;
    bool ok = std::fwrite("GAMMAMLP", 1, 8, f) == 8 && std::fwrite(hdr, 4, 6, f) == 6 &&
              std::fwrite(&step, 8, 1, f) == 1 && std::fwrite(&seed, 8, 1, f) == 1 &&
              std::fwrite(p.data(), 4, kNParams, f) == (size_t)kNParams &&
              std::fwrite(a.data(), 4, kNParams, f) == (size_t)kNParams &&
              std::fwrite(b.data(), 4, kNParams, f) == (size_t)kNParams;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? GAMMA_OK : GAMMA_ERR_INVALID_ARG;
}

int gamma_model_load(gamma_model m, const char* path)
{
    if (!m || !path) return GAMMA_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return GAMMA_ERR_MODEL;
    char magic[8];
    int32_t hdr[6];
    int64_t step = 0;
    uint64_t seed = 0;
    std::vector<float> p(kNParams), a(kNParams), b(kNParams);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "GAMMAMLP", 8) == 0 &&
              std::fread(hdr, 4, 6, f) == 6 && hdr[0] == 1 && hdr[1] == gk::kIn &&
              hdr[2] == gk::kInPad && hdr[3] == gk::kH && hdr[4] == gk::kOut &&
              hdr[5] == gk::kOutPad && std::fread(&step, 8, 1, f) == 1 &&
              std::fread(&seed, 8, 1, f) == 1 &&
              std::fread(p.data(), 4, kNParams, f) == (size_t)kNParams &&
              std::fread(a.data(), 4, kNParams, f) == (size_t)kNParams &&
              std::fread(b.data(), 4, kNParams, f) == (size_t)kNParams;
    std::fclose(f);
    if (!ok) return GAMMA_ERR_MODEL;
    for (float x : p)
        if (!std::isfinite(x)) return GAMMA_ERR_MODEL;
    MCK(cudaMemcpy(m->p, p.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->m1, a.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->m2, b.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice));
    m->step = step;
    m->seed = seed;
    if (int rc = refresh_bf16(m, 0)) return rc;
    MCK(cudaDeviceSynchronize());
    return GAMMA_OK;
}

}  // extern "C"
