// CUDA kernels of the gamma search (sm_103a).
//
// One run over a dose pair is four stream-ordered launches:
//   k_prepare   max of the reference dose (the global dose norm) and its
//               finite check (k_shell checks the evaluation dose, every value
//               of which is the centre of one tile voxel)  (Algorithm A2 step 2)
//   k_shell     per reference voxel: criteria, low-dose cutoff, gamma0 =
//               DD/dD (A1 step 4a) and every face through the voxel's node
//               (reduced closed form), from a TMA-staged tile; voxels whose
//               running gamma still exceeds the distance to any other face
//               are queued with a cost bucket
//   k_scatter   order the queue by estimated cost, most expensive first (the
//               role the paper's DD sort plays, Section 2.2 and Table 2)
//   k_tail      persistent: a group of G lanes takes one queued voxel and
//               walks the sorted cell table G cells at a time, with the exact
//               early exit of A1 step 4b-ii (key >= gamma) and a per-cell
//               lower bound sqrt(key^2 + dose gap^2)
// No kernel waits on another block or allocates memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>

#include "gamma_cell.cuh"
#include "gamma_internal.h"
#include "gamma_near.cuh"
#include "gamma_tma.cuh"

namespace gk {

// --------------------------------------------------------------------------
// k_prepare: dose norm and finite check
// --------------------------------------------------------------------------

// part: bit 0 = maximum and finite check of the reference dose, bit 1 =
// finite check of the evaluation dose (a part left out reads as zeros).
template <bool BATCH>
__global__ void __launch_bounds__(256)
    k_prepare(const __grid_constant__ Problem P0, const BatchDesc* __restrict__ bd, int part)
{
    const Problem& P = BATCH ? bd->probs[blockIdx.y] : P0;
    if constexpr (BATCH) {
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
            *bd->shell_next = 0u;
            if (bd->seed_count) {
                *bd->seed_count = 0u;
                *bd->seed_head = 0u;
            }
        }
    }
    float m = -kInf;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const float* ref = (part & 1) ? P.ref : nullptr;
    const float* ev = (part & 2) ? P.ev : nullptr;
    long long done = 0;
    if ((((uintptr_t)P.ref | (uintptr_t)P.ev) & 15u) == 0) {      // 16-byte vector reads
        const long long n4 = P.nvox / 4;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4* r4p = (const float4*)ref;
        const float4* e4p = (const float4*)ev;
        auto r4 = [&](long long i) { return r4p ? __ldg(r4p + i) : zero4; };
        auto e4 = [&](long long i) { return e4p ? __ldg(e4p + i) : zero4; };
        auto take = [&](const float4 r, const float4 e) {
            bad |= !(isfinite(r.x) && isfinite(r.y) && isfinite(r.z) && isfinite(r.w) &&
                     isfinite(e.x) && isfinite(e.y) && isfinite(e.z) && isfinite(e.w));
            m = fmaxf(m, fmaxf(fmaxf(r.x, r.y), fmaxf(r.z, r.w)));
        };
        long long i = first;
        for (; i + stride < n4; i += 2 * stride) {          // four 16-byte reads in flight
            const float4 ra = r4(i), ea = e4(i);
            const float4 rb = r4(i + stride), eb = e4(i + stride);
            take(ra, ea);
            take(rb, eb);
        }
        if (i < n4) take(r4(i), e4(i));
        done = n4 * 4;
    }
    for (long long i = done + first; i < P.nvox; i += stride) {
        const float r = ref ? __ldg(ref + i) : 0.f, e = ev ? __ldg(ev + i) : 0.f;
        bad |= !(isfinite(r) && isfinite(e));
        m = fmaxf(m, r);
    }
    // one atomic per block: same-address atomics serialise in L2
    __shared__ float sh_m[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) sh_m[threadIdx.x >> 5] = m;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh_m[w]);
        if (part & 1) atomicMax(&P.ctr->dnorm_enc, fenc(m));
        if (bad) atomicOr(&P.ctr->flags, kFlagNonFinite);
    }
}

// --------------------------------------------------------------------------
// k_shell: gamma0 and the key-0 cells, one block per tile of voxels
// --------------------------------------------------------------------------

// Tile of voxels per block (x fastest; a warp is one x row) and its halo box
// in shared memory.  The box starts 4 voxels left of the tile so that the TMA
// x coordinate stays a multiple of 4 floats (16 bytes).
template <int N>
struct ShellTile {
    static constexpr int TX = 32, TY = N == 3 ? 4 : 8, TZ = N == 3 ? 2 : 1;
    static constexpr int BX = 40, BY = TY + 2, BZ = N == 3 ? TZ + 2 : 1;
    static constexpr int ELEMS = BX * BY * BZ;
    // each staging buffer starts on a 128-byte boundary (TMA destination rule)
    static constexpr int STRIDE = (ELEMS + 31) / 32 * 32;
    static_assert(STRIDE * 4 % 128 == 0, "TMA destination must stay 128-byte aligned");
};

template <int N, int MINB, bool BATCH>
__global__ void __launch_bounds__(256, MINB)
    k_shell(const __grid_constant__ Problem P0, const __grid_constant__ CUtensorMap tmap0,
            int use_tma0, int t_first, int ntiles, unsigned* tile_next,
            const __grid_constant__ SlabGate gate, const BatchDesc* __restrict__ bd)
{
    using T = ShellTile<N>;
    __shared__ __align__(128) float tile[2][T::STRIDE];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ unsigned int sh_hist[kNumBuckets];
    __shared__ unsigned long long sh_eval, sh_pass;
    __shared__ unsigned int sh_rmax;
    __shared__ __align__(16) Problem sh_P;     // the current pair (batched launches)
    __shared__ int sh_next[2];                 // the block's next tile, per staging buffer
    __shared__ unsigned sh_tb[2];              // 1 + largest cost bucket queued in the tile (0: none)

    const int lane = threadIdx.x & 31;
    const int lx = lane, ly = (threadIdx.x >> 5) % T::TY, lz = (threadIdx.x >> 5) / T::TY;

    if (threadIdx.x < kNumBuckets) sh_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        sh_eval = 0;
        sh_pass = 0;
        sh_rmax = 0;
        sh_tb[0] = sh_tb[1] = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // global tile -> (pair, tile of that pair)
    auto locate = [&](int t, int& pr, int& lt) {
        if constexpr (!BATCH) {
            pr = 0;
            lt = t;
        } else {
            int lo = 0, hi = bd->npairs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bd->tile_start[mid] <= t) lo = mid; else hi = mid - 1;
            }
            pr = lo;
            lt = t - bd->tile_start[lo];
        }
    };
    auto pair_tma = [&](int pr) { return BATCH ? bd->use_tma[pr] : use_tma0; };
    auto tile_origin = [&](int nx, int ny, int lt, int& x0, int& y0, int& z0) {
        const int ntx = (nx + T::TX - 1) / T::TX, nty = (ny + T::TY - 1) / T::TY;
        x0 = (lt % ntx) * T::TX;
        y0 = ((lt / ntx) % nty) * T::TY;
        z0 = (lt / ntx / nty) * T::TZ;
    };
    bool gate_failed = false;            // thread 0: a slab wait gave up
    auto issue = [&](int t, int b) {
        if (t >= ntiles) return;
        int pr, lt;
        locate(t, pr, lt);
        if (!pair_tma(pr)) return;
        const Problem& Q = BATCH ? bd->probs[pr] : P0;
        const CUtensorMap* map = BATCH ? &bd->maps[pr] : &tmap0;
        int x0, y0, z0;
        tile_origin(Q.nx, Q.ny, lt, x0, y0, z0);
        if (!BATCH && gate.flag && !gate_failed) {
            // the box reads slices z0 - 1 .. z0 + TZ, from at most two slabs
            const int zlo = max(z0 - 1, 0), zhi = min(z0 + T::TZ, Q.nz - 1);
            if (!flag_wait_bounded(gate.flag + zlo / gate.depth, gate.epoch) ||
                !flag_wait_bounded(gate.flag + zhi / gate.depth, gate.epoch)) {
                atomicOr(&Q.ctr->flags, kFlagTimeout);     // the run reports a timeout
                gate_failed = true;                        // and this block waits no more
            }
            fence_async_global();
        }
        mbar_arrive_expect_tx(&bar[b], T::ELEMS * (uint32_t)sizeof(float));
        if (N == 3) tma_load_3d(tile[b], map, x0 - 4, y0 - 1, z0 - 1, &bar[b]);
        else tma_load_2d(tile[b], map, x0 - 4, y0 - 1, &bar[b]);
    };
    if (threadIdx.x == 0) issue(t_first + blockIdx.x, 0);
    uint32_t parity = 0;                 // bit b: phase of bar[b] to wait for
    unsigned my_eval = 0, my_pass = 0;
    float my_rmax = 0.f;
    bool bad_ev = false;                 // a non-finite evaluation dose was seen
    int buf = 0;
    int cur = -1;                        // pair whose counters my_* accumulate

    // per-block counters -> the pair's global counters
    auto flush = [&](const Problem& Q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            my_eval += __shfl_xor_sync(kFull, my_eval, o);
            my_pass += __shfl_xor_sync(kFull, my_pass, o);
            my_rmax = fmaxf(my_rmax, __shfl_xor_sync(kFull, my_rmax, o));
        }
        if (__any_sync(kFull, bad_ev) && lane == 0) atomicOr(&Q.ctr->flags, kFlagNonFinite);
        bad_ev = false;
        if (lane == 0) {
            if (my_eval) atomicAdd(&sh_eval, (unsigned long long)my_eval);
            if (my_pass) atomicAdd(&sh_pass, (unsigned long long)my_pass);
            atomicMax(&sh_rmax, fenc(my_rmax));
        }
        my_eval = my_pass = 0;
        my_rmax = 0.f;
        __syncthreads();
        if (threadIdx.x < kNumBuckets && sh_hist[threadIdx.x]) {
            atomicAdd(&Q.ctr->hist[threadIdx.x], sh_hist[threadIdx.x]);
            sh_hist[threadIdx.x] = 0;
        }
        if (threadIdx.x == 0) {
            if (sh_eval) atomicAdd(&Q.ctr->n_eval, sh_eval);
            if (sh_pass) atomicAdd(&Q.ctr->n_pass, sh_pass);
            atomicMax(&Q.ctr->rmax_enc, sh_rmax);
            sh_eval = 0;
            sh_pass = 0;
            sh_rmax = 0;
        }
        __syncthreads();
    };

    // Tiles after the first come from a work counter when one is given (the
    // block that finishes first takes the next tile), else in grid stride.
    for (int t = t_first + blockIdx.x; t < ntiles; buf ^= 1) {
        int pr, lt;
        locate(t, pr, lt);
        if constexpr (BATCH) {
            if (pr != cur) {                       // block-uniform
                if (cur >= 0) flush(sh_P);
                const int* src = (const int*)&bd->probs[pr];
                int* dst = (int*)&sh_P;
                for (int i = threadIdx.x; i < (int)(sizeof(Problem) / 4); i += blockDim.x)
                    dst[i] = src[i];
                __syncthreads();
                cur = pr;
            }
        }
        const Problem& P = BATCH ? sh_P : P0;
        const bool use_tma = pair_tma(pr) != 0;
        const float dnorm = resolve_dnorm(P);
        const float thr = cutoff_threshold(P.local, P.cutoff_frac, dnorm);
        // every face not through the voxel is at spatial distance >= the
        // first table key, or >= the cover radius when the table was cut
        const float k0 = P.ntable > 0 ? P.table[0].key : kInf;
        const float qlim = fminf(k0 * k0, P.r_cover * P.r_cover);
        int x0, y0, z0;
        tile_origin(P.nx, P.ny, lt, x0, y0, z0);
        float* tl = tile[buf];
        // ---- stage: prefetch the next tile, wait for this one ----
        // Every thread waits on the tile's mbarrier itself; a wait that gives
        // up is reported at the end-of-tile barrier, where the block leaves
        // together (the smem reads in between stay in bounds).
        if (threadIdx.x == 0) {
            const int nt = tile_next ? t_first + (int)gridDim.x + (int)atomicAdd(tile_next, 1u)
                                     : t + (int)gridDim.x;
            sh_next[buf] = nt;                 // read by every thread after this tile's barrier
            issue(nt, buf ^ 1);
        }
        bool timed_out = false;
        if (use_tma) {
            timed_out = !mbar_wait_bounded(&bar[buf], (parity >> buf) & 1u);
            parity ^= 1u << buf;
        } else {
            for (int i = threadIdx.x; i < T::ELEMS; i += blockDim.x) {
                const int bx = i % T::BX, by = (i / T::BX) % T::BY, bz = i / (T::BX * T::BY);
                const int gx = x0 - 4 + bx, gy = y0 - 1 + by, gz = (N == 3 ? z0 - 1 : 0) + bz;
                const bool in = (unsigned)gx < (unsigned)P.nx && (unsigned)gy < (unsigned)P.ny &&
                                (N == 2 || (unsigned)gz < (unsigned)P.nz);
                tl[i] = in ? __ldg(P.ev + ((long long)gz * P.ny + gy) * P.nx + gx) : 0.f;
            }
            __syncthreads();
        }

        // ---- gamma0 and the faces that contain the voxel ----
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        const bool inside = x < P.nx && y < P.ny && z < P.nz;
        const long long v = inside ? ((long long)z * P.ny + y) * P.nx + x : 0;
        const int tix0 = ((N == 3 ? lz + 1 : 0) * T::BY + (ly + 1)) * T::BX + (lx + 4);
        float dr = 0.f, best = 0.f;
        bool act = false;
        if (inside) {
            dr = __ldg(P.ref + v);
            act = is_evaluated(P, dr, thr);
            if (!act) P.out[v] = __int_as_float(0x7fc00000);
            bad_ev |= !isfinite(tl[tix0]);           // every evaluation dose is some tile's centre
        }
        const int tix = tix0;
        uint32_t inm = 0, inp = 0;       // neighbours at -1 / +1 inside the grid, per axis
        inm |= (x > 0) ? 1u : 0u;
        inp |= (x + 1 < P.nx) ? 1u : 0u;
        inm |= (y > 0) ? 2u : 0u;
        inp |= (y + 1 < P.ny) ? 2u : 0u;
        if (N == 3) {
            inm |= (z > 0) ? 4u : 0u;
            inp |= (z + 1 < P.nz) ? 4u : 0u;
        }
        if (act) {
            const float dD = P.dd_frac * (P.local ? dr : dnorm);
            const float q0 = (tl[tix] - dr) / dD;
            best = q0 * q0;
            my_rmax = fmaxf(my_rmax, fabsf(q0));
            if (best > 0.f) best = near_gamma2<N, T::BX, T::BX * T::BY>(tl, tix, inm, inp, dr, dD, P.mt.kappa);
        }

        // ---- finish or queue ----
        bool tail = false;
        int bucket = 0;
        if (act) {
            tail = best > qlim;
            if (tail) {
                P.out[v] = best;                       // gamma^2, finished by k_tail
                // 1 + floor(2 log2 of the table cells with key < gamma)
                bucket = cost_bucket_of(P.bucket_key, sqrtf(best));
            } else {
                const float gam = sqrtf(best);
                P.out[v] = gam;
                ++my_eval;
                my_pass += gam <= 1.f;                 // decided on the value written
            }
        }
        const unsigned tm = __ballot_sync(kFull, tail);
        if (!BATCH && P.tile_mask) {
            // the tile's queue for the tile-staged walk: one bit per voxel
            if (lane == 0) P.tile_mask[(size_t)lt * 8 + (threadIdx.x >> 5)] = tm;
            if (tm) {
                unsigned bm = tail ? (unsigned)bucket + 1u : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bm = max(bm, __shfl_xor_sync(kFull, bm, o));
                if (lane == 0) atomicMax(&sh_tb[buf], bm);
            }
        }
        if (!BATCH && P.row_items && tm) {
            // this warp row's item for the row-staged walk
            unsigned bm = tail ? (unsigned)bucket : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bm = max(bm, __shfl_xor_sync(kFull, bm, o));
            if (lane == 0) {
                const unsigned ip = atomicAdd(&P.ctr->row_count, 1u);
                P.row_items[ip] = ((unsigned long long)((unsigned)lt * 8u + (threadIdx.x >> 5)) << 32) | tm;
                P.row_bkt[ip] = (unsigned char)bm;
                atomicAdd(&P.ctr->row_hist[bm], 1u);
            }
        }
        if (tm) {
            unsigned pos0 = 0;
            if (lane == 0) pos0 = atomicAdd(&P.ctr->tail_count, (unsigned)__popc(tm));
            pos0 = __shfl_sync(kFull, pos0, 0);
            if (tail) {
                const unsigned pos = pos0 + __popc(tm & ((1u << lane) - 1u));
                if (pos < P.tail_cap) {
                    P.tail_raw[pos] = (unsigned)v;
                    P.tail_bucket[pos] = (unsigned char)bucket;
                    atomicAdd(&sh_hist[bucket], 1u);
                } else {
                    atomicOr(&P.ctr->flags, kFlagTailFull);
                }
            }
        }
        // tile[buf] is free for reuse once every thread has passed this point
        if (__syncthreads_or(timed_out)) {
            if (threadIdx.x == 0) {
                atomicOr(&P.ctr->flags, kFlagTimeout);
                // let this block's own copies land before it leaves
                mbar_wait_bounded(&bar[buf], (parity >> buf) & 1u);
                mbar_wait_bounded(&bar[buf ^ 1], (parity >> (buf ^ 1)) & 1u);
            }
            break;
        }
        if (!BATCH && P.tile_mask && threadIdx.x == 0) {
            const unsigned b1 = sh_tb[buf];
            if (b1) {
                const unsigned pos = atomicAdd(&P.ctr->tile_count, 1u);
                P.tile_list[pos] = (unsigned)lt;
                P.tile_bkt[pos] = (unsigned char)(b1 - 1u);
                atomicAdd(&P.ctr->tile_hist[b1 - 1u], 1u);
            }
            sh_tb[buf] = 0;            // the next tile of this buffer comes after the next barrier
        }
        t = sh_next[buf];
    }
    if (!BATCH || cur >= 0) flush(BATCH ? sh_P : P0);
}

// --------------------------------------------------------------------------
// k_shell_w: the same per-voxel work, one warp per tile, no block barriers
// --------------------------------------------------------------------------

// In k_shell the eight warps of a block share one staged tile and meet at a
// block barrier per tile, so a tile takes as long as its slowest warp row.
// Here each warp stages its own smaller tile (32 x 2 x 2 voxels in 3D, 32 x 4
// in 2D, with a one-voxel halo) into a double buffer of its own, with its own
// TMA copies and mbarriers (or plain loads when the grid takes no TMA map),
// and takes its next tile from the work counter by itself: warps never wait
// for one another until the end of the kernel.  Batched launches number the
// tiles of all pairs of a group in one range; a warp keeps a copy of its
// current pair's Problem in shared memory.
template <int N>
struct WarpTile {
    static constexpr int TX = 32, TY = N == 3 ? 2 : 4, TZ = N == 3 ? 2 : 1;
    static constexpr int BX = 40, BY = TY + 2, BZ = N == 3 ? TZ + 2 : 1;
    static constexpr int ELEMS = BX * BY * BZ;
    static constexpr int STRIDE = (ELEMS + 31) / 32 * 32;   // 128-byte aligned buffers
    static_assert(STRIDE * 4 % 128 == 0, "TMA destination must stay 128-byte aligned");
};

template <int N, int MINB, bool BATCH>
__global__ void __launch_bounds__(256, MINB)
    k_shell_w(const __grid_constant__ Problem P0, const __grid_constant__ CUtensorMap tmap0,
              int use_tma0, int t_first, int ntiles, unsigned* tile_next,
              const __grid_constant__ SlabGate gate, const BatchDesc* __restrict__ bd)
{
    using T = WarpTile<N>;
    __shared__ __align__(128) float tiles[8][2][T::STRIDE];
    __shared__ __align__(8) uint64_t bar[8][2];
    __shared__ __align__(16) Problem sh_P[BATCH ? 8 : 1];   // batched: each warp's current pair
    __shared__ unsigned int sh_hist[kNumBuckets];
    __shared__ unsigned long long sh_eval, sh_pass;
    __shared__ unsigned int sh_rmax, sh_bad;
    // each warp's queued voxels (and cost buckets) not yet in the run's queue:
    // one atomic on the queue counter per kShellQ of them, not one per row
    constexpr int kShellQ = BATCH ? 64 : 128;     // (the batched kernel keeps 8 Problems too)
    __shared__ unsigned qv[8][kShellQ];
    __shared__ unsigned char qb[8][kShellQ];

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < kNumBuckets) sh_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        sh_eval = sh_pass = 0;
        sh_rmax = sh_bad = 0;
    }
    if (lane == 0) {
        mbar_init(&bar[w][0], 1);
        mbar_init(&bar[w][1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // global tile -> (pair, tile of that pair)
    auto locate = [&](int t, int& pr, int& lt) {
        if constexpr (!BATCH) {
            pr = 0;
            lt = t;
        } else {
            int lo = 0, hi = bd->npairs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bd->tile_start[mid] <= t) lo = mid; else hi = mid - 1;
            }
            pr = lo;
            lt = t - bd->tile_start[lo];
        }
    };
    auto origin = [&](int nx, int ny, int lt, int& x0, int& y0, int& z0) {
        const int ntx = (nx + T::TX - 1) / T::TX, nty = (ny + T::TY - 1) / T::TY;
        x0 = (lt % ntx) * T::TX;
        y0 = ((lt / ntx) % nty) * T::TY;
        z0 = (lt / ntx / nty) * T::TZ;
    };
    bool gate_failed = false;                 // lane 0: a slab wait gave up
    // the copy of tile t's box into buffer b, by the whole warp: one TMA copy
    // issued by lane 0, or, for a grid without a TMA map (its rows are not
    // 16-byte aligned), 4-byte asynchronous copies by every lane; either way
    // the box of the next tile is in flight while this one is computed.  One
    // cp.async group per call (empty for TMA tiles), so that the group of
    // the tile to compute is the second most recent one.  (Slab gates come
    // only with a TMA map.)
    auto issue = [&](int t, int b) {
        if (t < ntiles) {
            int pr, lt;
            locate(t, pr, lt);
            const Problem& Q = BATCH ? bd->probs[pr] : P0;
            int x0, y0, z0;
            origin(Q.nx, Q.ny, lt, x0, y0, z0);
            if (BATCH ? bd->use_tma[pr] : use_tma0) {
                if (lane == 0) {
                    const CUtensorMap* map = BATCH ? &bd->maps[pr] : &tmap0;
                    if (!BATCH && gate.flag && !gate_failed) {
                        // the box reads slices z0 - 1 .. z0 + TZ, from at most two slabs
                        const int zlo = max(z0 - 1, 0), zhi = min(z0 + T::TZ, Q.nz - 1);
                        if (!flag_wait_bounded(gate.flag + zlo / gate.depth, gate.epoch) ||
                            !flag_wait_bounded(gate.flag + zhi / gate.depth, gate.epoch)) {
                            atomicOr(&Q.ctr->flags, kFlagTimeout);     // the run reports a timeout
                            gate_failed = true;                        // and this warp waits no more
                        }
                        fence_async_global();
                    }
                    mbar_arrive_expect_tx(&bar[w][b], T::ELEMS * (uint32_t)sizeof(float));
                    if (N == 3) tma_load_3d(tiles[w][b], map, x0 - 4, y0 - 1, z0 - 1, &bar[w][b]);
                    else tma_load_2d(tiles[w][b], map, x0 - 4, y0 - 1, &bar[w][b]);
                }
            } else {
                const int nx = Q.nx, ny = Q.ny, nz = Q.nz;
                const float* ev = Q.ev;
                float* dst = tiles[w][b];
                for (int i = lane; i < T::ELEMS; i += 32) {
                    const int bx = i % T::BX, by = (i / T::BX) % T::BY, bz = i / (T::BX * T::BY);
                    const int gx = x0 - 4 + bx, gy = y0 - 1 + by, gz = (N == 3 ? z0 - 1 : 0) + bz;
                    const bool in = (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny &&
                                    (N == 2 || (unsigned)gz < (unsigned)nz);
                    cp_async_f32(dst + i, ev + (in ? ((long long)gz * ny + gy) * nx + gx : 0), in);
                }
            }
        }
        cp_async_commit();
    };
    const int nwarps = (int)gridDim.x * 8;
    int t = t_first + (int)blockIdx.x * 8 + w;     // the first tile of every warp, then the counter
    issue(t, 0);

    unsigned my_eval = 0, my_pass = 0;
    float my_rmax = 0.f;
    bool bad_ev = false, timed_out = false;
    uint32_t parity = 0;                      // bit b: phase of bar[w][b] to wait for
    int b = 0;
    int cur = -1;                             // batched: the pair in sh_P[w] and counted in my_*
    // the current pair's constants: dose norm, cutoff, and the bound below
    // which a voxel is final (every face not through the voxel is at spatial
    // distance >= the first table key, or >= the cover radius when the table
    // was cut)
    float dnorm = 0.f, thr = 0.f, qlim = 0.f;
    auto constants = [&](const Problem& Q) {
        dnorm = resolve_dnorm(Q);
        thr = cutoff_threshold(Q.local, Q.cutoff_frac, dnorm);
        const float k0 = Q.ntable > 0 ? Q.table[0].key : kInf;
        qlim = fminf(k0 * k0, Q.r_cover * Q.r_cover);
    };
    if constexpr (!BATCH) constants(P0);

    // a warp's counts -> its pair's counters (batched: when its pair changes)
    auto flush_counts = [&](const Problem& Q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            my_eval += __shfl_xor_sync(kFull, my_eval, o);
            my_pass += __shfl_xor_sync(kFull, my_pass, o);
            my_rmax = fmaxf(my_rmax, __shfl_xor_sync(kFull, my_rmax, o));
        }
        if (__any_sync(kFull, bad_ev) && lane == 0) atomicOr(&Q.ctr->flags, kFlagNonFinite);
        if (lane == 0) {
            if (my_eval) atomicAdd(&Q.ctr->n_eval, (unsigned long long)my_eval);
            if (my_pass) atomicAdd(&Q.ctr->n_pass, (unsigned long long)my_pass);
            if (my_rmax > 0.f) atomicMax(&Q.ctr->rmax_enc, fenc(my_rmax));
        }
        my_eval = my_pass = 0;
        my_rmax = 0.f;
        bad_ev = false;
    };

    int qn = 0;                               // entries in qv[w] (warp-uniform)
    auto flush_queue = [&](const Problem& Q) {
        if (qn == 0) return;
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&Q.ctr->tail_count, (unsigned)qn);
        base = __shfl_sync(kFull, base, 0);
        for (int i0 = 0; i0 < qn; i0 += 32) {
            const int i = i0 + lane;
            bool counted = false;
            int bk = 0;
            if (i < qn) {
                const unsigned pos = base + (unsigned)i;
                bk = qb[w][i];
                if (pos < Q.tail_cap) {
                    Q.tail_raw[pos] = qv[w][i];
                    Q.tail_bucket[pos] = (unsigned char)bk;
                    counted = true;
                } else {
                    atomicOr(&Q.ctr->flags, kFlagTailFull);
                }
            }
            if constexpr (BATCH) {
                // the pair's histogram, one atomic per distinct bucket of the 32
                const unsigned peers = __match_any_sync(kFull, counted ? bk : -1);
                if (counted && lane == __ffs(peers) - 1)
                    atomicAdd(&Q.ctr->hist[bk], (unsigned)__popc(peers));
            } else {
                if (counted) atomicAdd(&sh_hist[bk], 1u);
            }
        }
        __syncwarp();
        qn = 0;
    };

    while (t < ntiles) {
        int nt = 0;
        if (lane == 0) nt = t_first + nwarps + (int)atomicAdd(tile_next, 1u);
        nt = __shfl_sync(kFull, nt, 0);
        issue(nt, b ^ 1);
        int pr, lt;
        locate(t, pr, lt);
        if constexpr (BATCH) {
            if (pr != cur) {                   // warp-uniform
                if (cur >= 0) {
                    flush_queue(sh_P[w]);
                    flush_counts(sh_P[w]);
                }
                __syncwarp();
                const int* src = (const int*)&bd->probs[pr];
                int* dst = (int*)&sh_P[w];
                for (int i = lane; i < (int)(sizeof(Problem) / 4); i += 32) dst[i] = src[i];
                __syncwarp();
                cur = pr;
                constants(sh_P[w]);
            }
        }
        const Problem& P = BATCH ? sh_P[w] : P0;
        float* tl = tiles[w][b];
        int x0, y0, z0;
        origin(P.nx, P.ny, lt, x0, y0, z0);
        // the tile's reference doses, loaded while its staged box may still
        // be in flight (row r in drq[0] when row r is processed)
        constexpr int ROWS = T::TY * T::TZ;
        float drq[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int x = x0 + lane, y = y0 + r % T::TY, z = z0 + r / T::TY;
            drq[r] = (x < P.nx && y < P.ny && z < P.nz) ? __ldg(P.ref + ((long long)z * P.ny + y) * P.nx + x)
                                                         : 0.f;
        }
        if (BATCH ? bd->use_tma[pr] : use_tma0) {
            if (!mbar_wait_bounded(&bar[w][b], (parity >> b) & 1u)) {
                timed_out = true;              // (warp-uniform: every lane polls the same phase)
                break;
            }
            parity ^= 1u << b;
        } else {
            cp_async_wait<1>();                // this tile's copies (the next tile's may be in flight)
            __syncwarp();
        }
#pragma unroll 1
        for (int r = 0; r < ROWS; ++r) {
            const int ly = r % T::TY, lz = r / T::TY;
            const int x = x0 + lane, y = y0 + ly, z = z0 + lz;
            const bool inside = x < P.nx && y < P.ny && z < P.nz;
            const long long v = inside ? ((long long)z * P.ny + y) * P.nx + x : 0;
            const int tix = ((N == 3 ? lz + 1 : 0) * T::BY + (ly + 1)) * T::BX + (lane + 4);
            const float dr = drq[0];
#pragma unroll
            for (int k = 0; k + 1 < ROWS; ++k) drq[k] = drq[k + 1];
            float best = 0.f;
            bool act = false;
            if (inside) {
                act = is_evaluated(P, dr, thr);
                if (!act) P.out[v] = __int_as_float(0x7fc00000);
                bad_ev |= !isfinite(tl[tix]);       // every evaluation dose is some tile's centre
            }
            uint32_t inm = 0, inp = 0;         // neighbours at -1 / +1 inside the grid, per axis
            inm |= (x > 0) ? 1u : 0u;
            inp |= (x + 1 < P.nx) ? 1u : 0u;
            inm |= (y > 0) ? 2u : 0u;
            inp |= (y + 1 < P.ny) ? 2u : 0u;
            if (N == 3) {
                inm |= (z > 0) ? 4u : 0u;
                inp |= (z + 1 < P.nz) ? 4u : 0u;
            }
            if (act) {
                const float dD = P.dd_frac * (P.local ? dr : dnorm);
                const float q0 = (tl[tix] - dr) / dD;
                best = q0 * q0;
                my_rmax = fmaxf(my_rmax, fabsf(q0));
                if (best > 0.f) best = near_gamma2<N, T::BX, T::BX * T::BY>(tl, tix, inm, inp, dr, dD, P.mt.kappa);
            }
            bool tail = false;
            int bucket = 0;
            if (act) {
                tail = best > qlim;
                if (tail) {
                    P.out[v] = best;                   // gamma^2, finished by the table walk
                    // 1 + floor(2 log2 of the table cells with key < gamma)
                    bucket = cost_bucket_of(P.bucket_key, sqrtf(best));
                } else {
                    const float gam = sqrtf(best);
                    P.out[v] = gam;
                    ++my_eval;
                    my_pass += gam <= 1.f;             // decided on the value written
                }
            }
            const unsigned tm = __ballot_sync(kFull, tail);
            if (tm) {
                if (qn + 32 > kShellQ) flush_queue(P);
                if (tail) {
                    const int i = qn + __popc(tm & ((1u << lane) - 1u));
                    qv[w][i] = (unsigned)v;
                    qb[w][i] = (unsigned char)bucket;
                }
                qn += __popc(tm);
                __syncwarp();
            }
        }
        __syncwarp();                          // tiles[w][b] is free for the copy after next
        t = nt;
        b ^= 1;
    }
    cp_async_wait<0>();                        // no copy into this block's memory outlives it
    if (timed_out) {
        if (lane == 0) {
            if constexpr (BATCH) atomicOr(&bd->probs[cur < 0 ? 0 : cur].ctr->flags, kFlagTimeout);
            else atomicOr(&P0.ctr->flags, kFlagTimeout);
            // let this warp's own copies land before the block leaves
            mbar_wait_bounded(&bar[w][0], parity & 1u);
            mbar_wait_bounded(&bar[w][1], (parity >> 1) & 1u);
        }
        __syncwarp();
    }
    if constexpr (BATCH) {
        if (cur >= 0) {
            flush_queue(sh_P[w]);
            flush_counts(sh_P[w]);
        }
    } else {
        flush_queue(P0);
        // per block, then one atomic each: same-address atomics serialise in L2
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            my_eval += __shfl_xor_sync(kFull, my_eval, o);
            my_pass += __shfl_xor_sync(kFull, my_pass, o);
            my_rmax = fmaxf(my_rmax, __shfl_xor_sync(kFull, my_rmax, o));
        }
        const bool bad = __any_sync(kFull, bad_ev);
        if (lane == 0) {
            if (my_eval) atomicAdd(&sh_eval, (unsigned long long)my_eval);
            if (my_pass) atomicAdd(&sh_pass, (unsigned long long)my_pass);
            atomicMax(&sh_rmax, fenc(my_rmax));
            if (bad) sh_bad = 1;
        }
        __syncthreads();
        if (threadIdx.x < kNumBuckets && sh_hist[threadIdx.x])
            atomicAdd(&P0.ctr->hist[threadIdx.x], sh_hist[threadIdx.x]);
        if (threadIdx.x == 0) {
            if (sh_eval) atomicAdd(&P0.ctr->n_eval, sh_eval);
            if (sh_pass) atomicAdd(&P0.ctr->n_pass, sh_pass);
            atomicMax(&P0.ctr->rmax_enc, sh_rmax);
            if (sh_bad) atomicOr(&P0.ctr->flags, kFlagNonFinite);
        }
    }
}

// The queue's parts chosen from the queue itself (option group_bucket < 0):
// a queued voxel of cost bucket b is estimated to key c(b) = 2^((2b - 1) / 4)
// table cells (the middle of the bucket), the walk's W = sum of c over the
// queue, spread over its L lanes, ideally takes T = W / L steps per lane.  A
// voxel walks alone unless that takes longer than s T; it walks 4 lanes
// above s T, 8 above 4 s T and a whole warp above 8 s T, so that no voxel's
// own walk sets the kernel's length while the lanes stay busy.  Called by a
// full warp, lane b holding the count of bucket b; every lane gets the
// three thresholds.
__device__ __forceinline__ void auto_part_buckets(unsigned count, unsigned lanes, float scale, int& b4,
                                                  int& b8, int& b32)
{
    const int lane = threadIdx.x & 31;
    const float c = lane > 0 ? exp2f((2 * lane - 1) * 0.25f) : 0.f;
    float w = (float)count * c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
    const float t = scale * w / (float)max(lanes, 1u);
    auto first_above = [&](float lim) {
        const unsigned m = __ballot_sync(kFull, lane > 0 && c > lim);
        return m ? __ffs(m) - 1 : kNumBuckets;
    };
    b4 = first_above(t);
    b8 = first_above(4.f * t);
    b32 = first_above(8.f * t);
}

// --------------------------------------------------------------------------
// Queue ordering: bucket offsets (most expensive first) and scatter
// --------------------------------------------------------------------------

// Scatter queued voxels into bucket order.  Every block derives the bucket
// starts from the histogram itself (32 values), then reserves one range per
// bucket per block-chunk with a single atomic on a per-bucket cursor.
__global__ void __launch_bounds__(256) k_scatter(const __grid_constant__ Problem P)
{
    __shared__ unsigned start[kNumBuckets], cnt[kNumBuckets], base[kNumBuckets];
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = kNumBuckets - 1; b >= 0; --b) {
            start[b] = acc;
            acc += P.ctr->hist[b];
        }
    }
    const unsigned total = min(P.ctr->tail_count, P.tail_cap);
    for (unsigned c0 = blockIdx.x * blockDim.x; c0 < total; c0 += gridDim.x * blockDim.x) {
        if (threadIdx.x < kNumBuckets) cnt[threadIdx.x] = 0;
        __syncthreads();
        const unsigned i = c0 + threadIdx.x;
        int b = -1;
        unsigned rank = 0;
        if (i < total) {
            b = P.tail_bucket[i];
            rank = atomicAdd(&cnt[b], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kNumBuckets && cnt[threadIdx.x])
            base[threadIdx.x] = start[threadIdx.x] + atomicAdd(&P.ctr->cursor[threadIdx.x], cnt[threadIdx.x]);
        __syncthreads();
        if (b >= 0) P.tail_sorted[base[b] + rank] = P.tail_raw[i];
        __syncthreads();
    }
}

// The tiles with queued voxels in order of their largest cost bucket, most
// expensive first (same scheme as k_scatter).
__global__ void __launch_bounds__(256) k_scatter_tiles(const __grid_constant__ Problem P)
{
    __shared__ unsigned start[kNumBuckets], cnt[kNumBuckets], base[kNumBuckets];
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = kNumBuckets - 1; b >= 0; --b) {
            start[b] = acc;
            acc += P.ctr->tile_hist[b];
        }
    }
    const unsigned total = P.ctr->tile_count;
    for (unsigned c0 = blockIdx.x * blockDim.x; c0 < total; c0 += gridDim.x * blockDim.x) {
        if (threadIdx.x < kNumBuckets) cnt[threadIdx.x] = 0;
        __syncthreads();
        const unsigned i = c0 + threadIdx.x;
        int b = -1;
        unsigned rank = 0;
        if (i < total) {
            b = P.tile_bkt[i];
            rank = atomicAdd(&cnt[b], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kNumBuckets && cnt[threadIdx.x])
            base[threadIdx.x] = start[threadIdx.x] + atomicAdd(&P.ctr->tile_cursor[threadIdx.x], cnt[threadIdx.x]);
        __syncthreads();
        if (b >= 0) P.tile_sorted[base[b] + rank] = P.tile_list[i];
        __syncthreads();
    }
}

// The warp rows with queued voxels in order of their largest cost bucket,
// most expensive first (same scheme as k_scatter).
__global__ void __launch_bounds__(256) k_scatter_rows(const __grid_constant__ Problem P)
{
    __shared__ unsigned start[kNumBuckets], cnt[kNumBuckets], base[kNumBuckets];
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = kNumBuckets - 1; b >= 0; --b) {
            start[b] = acc;
            acc += P.ctr->row_hist[b];
        }
    }
    const unsigned total = P.ctr->row_count;
    for (unsigned c0 = blockIdx.x * blockDim.x; c0 < total; c0 += gridDim.x * blockDim.x) {
        if (threadIdx.x < kNumBuckets) cnt[threadIdx.x] = 0;
        __syncthreads();
        const unsigned i = c0 + threadIdx.x;
        int b = -1;
        unsigned rank = 0;
        if (i < total) {
            b = P.row_bkt[i];
            rank = atomicAdd(&cnt[b], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kNumBuckets && cnt[threadIdx.x])
            base[threadIdx.x] = start[threadIdx.x] + atomicAdd(&P.ctr->row_cursor[threadIdx.x], cnt[threadIdx.x]);
        __syncthreads();
        if (b >= 0) P.row_sorted[base[b] + rank] = P.row_items[i];
        __syncthreads();
    }
}

// Global order of a batch group's queued voxels, in four parts by cost
// bucket: b >= group32_bucket, then b >= group8_bucket, then b >=
// group_bucket, then the rest (the thresholds made non-increasing); within a
// part pair by pair (so that the walks in flight share one pair's doses in
// L2), most expensive bucket first within a pair.  All thresholds 0 give one
// pair-major order.  Each pair's cursor[b] starts at its range in that order;
// item_start holds those starts, the total and the ends of the first three
// parts, and the walk's work counters restart.  One block.
__global__ void __launch_bounds__(256) k_bucket_scan_batch(const BatchDesc* __restrict__ bd)
{
    __shared__ unsigned tot[4];
    __shared__ unsigned sc[4][256];
    __shared__ unsigned hsum[kNumBuckets];
    __shared__ int sh_b[3];
    const int np = bd->npairs, tid = threadIdx.x;
    if (bd->group_bucket < 0) {
        // parts chosen from the group's queue (auto_part_buckets over every pair's histogram)
        if (tid < kNumBuckets) hsum[tid] = 0;
        __syncthreads();
        for (int i = tid; i < np * kNumBuckets; i += blockDim.x) {
            const unsigned v = bd->probs[i / kNumBuckets].ctr->hist[i % kNumBuckets];
            if (v) atomicAdd(&hsum[i % kNumBuckets], v);
        }
        __syncthreads();
        if (tid < 32) {
            int a4, a8, a32;
            auto_part_buckets(hsum[tid], bd->walk_lanes, bd->auto_scale, a4, a8, a32);
            if (tid == 0) {
                sh_b[0] = a4;
                sh_b[1] = a8;
                sh_b[2] = a32;
            }
        }
        __syncthreads();
    }
    const bool autop = bd->group_bucket < 0;
    const int b32 = autop ? sh_b[2] : bd->group32_bucket, b8 = min(autop ? sh_b[1] : bd->group8_bucket, b32),
              b4 = min(autop ? sh_b[0] : bd->group_bucket, b8);
    auto part_of = [&](int b) { return b >= b32 ? 0 : (b >= b8 ? 1 : (b >= b4 ? 2 : 3)); };
    auto sums = [&](int p, unsigned (&u)[4]) {
        u[0] = u[1] = u[2] = u[3] = 0;
        if (p >= np) return;
        const Counters* c = bd->probs[p].ctr;
        for (int b = 0; b < kNumBuckets; ++b) u[part_of(b)] += c->hist[b];
    };
    if (tid < 4) tot[tid] = 0;
    __syncthreads();
    for (int p = tid; p < np; p += blockDim.x) {
        unsigned u[4];
        sums(p, u);
        for (int r = 0; r < 4; ++r)
            if (u[r]) atomicAdd(&tot[r], u[r]);
    }
    __syncthreads();
    unsigned rb[4], carry[4] = {0, 0, 0, 0};
    rb[0] = 0;
    for (int r = 1; r < 4; ++r) rb[r] = rb[r - 1] + tot[r - 1];
    for (int c0 = 0; c0 < np; c0 += blockDim.x) {
        const int p = c0 + tid;
        unsigned u[4];
        sums(p, u);
        for (int r = 0; r < 4; ++r) sc[r][tid] = u[r];
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {      // inclusive scans, per part
            unsigned v[4];
            for (int r = 0; r < 4; ++r) v[r] = tid >= o ? sc[r][tid - o] : 0u;
            __syncthreads();
            for (int r = 0; r < 4; ++r) sc[r][tid] += v[r];
            __syncthreads();
        }
        if (p < np) {
            Counters* c = bd->probs[p].ctr;
            unsigned start[4];
            for (int r = 0; r < 4; ++r) start[r] = rb[r] + carry[r] + sc[r][tid] - u[r];
            for (int b = kNumBuckets - 1; b >= 0; --b) {
                const int r = part_of(b);
                bd->item_start[p * kNumBuckets + (kNumBuckets - 1 - b)] = start[r];
                c->cursor[b] = start[r];
                start[r] += c->hist[b];
            }
        }
        for (int r = 0; r < 4; ++r) carry[r] += sc[r][blockDim.x - 1];
        __syncthreads();
    }
    if (tid == 0) {
        const int nb = np * kNumBuckets;
        bd->item_start[nb] = rb[3] + tot[3];
        bd->item_start[nb + 1] = rb[1];
        bd->item_start[nb + 2] = rb[2];
        bd->item_start[nb + 3] = rb[3];
        *bd->head = 0;
        if (bd->part_head) {
            for (int r = 0; r < 4; ++r) bd->part_head[r] = 0;
            *bd->fix_count = 0;
        }
    }
}

// Scatter one pair (blockIdx.y) of a batch group into the group order: per
// chunk of 256 queued voxels one atomic per cost bucket on the pair's cursor
// (as k_scatter), not one per voxel.
__global__ void __launch_bounds__(256) k_scatter_batch(const BatchDesc* __restrict__ bd)
{
    __shared__ unsigned cnt[kNumBuckets], base[kNumBuckets];
    const Problem& P = bd->probs[blockIdx.y];
    const unsigned total = min(P.ctr->tail_count, P.tail_cap);
    for (unsigned c0 = blockIdx.x * blockDim.x; c0 < total; c0 += gridDim.x * blockDim.x) {
        if (threadIdx.x < kNumBuckets) cnt[threadIdx.x] = 0;
        __syncthreads();
        const unsigned i = c0 + threadIdx.x;
        int b = -1;
        unsigned rank = 0;
        if (i < total) {
            b = P.tail_bucket[i];
            rank = atomicAdd(&cnt[b], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kNumBuckets && cnt[threadIdx.x])
            base[threadIdx.x] = atomicAdd(&P.ctr->cursor[threadIdx.x], cnt[threadIdx.x]);
        __syncthreads();
        if (b >= 0) {
            const unsigned pos = base[b] + rank;
            bd->items_v[pos] = P.tail_raw[i];
            bd->items_p[pos] = (unsigned short)blockIdx.y;
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// k_tail: persistent, G lanes per voxel, walk of the sorted cell table
// --------------------------------------------------------------------------

struct TailStats {
    unsigned long long visited = 0, pruned = 0, keyed = 0;
};

template <int N>
__device__ __forceinline__ float visit_cell(const Problem& P, int x, int y, int z, int cx, int cy,
                                            int cz, float key, float dr, float inv, float dnorm,
                                            float best, TailStats& st)
{
    const int px = x + cx, py = y + cy, pz = z + cz;
    if ((unsigned)px >= (unsigned)P.nx || (unsigned)py >= (unsigned)P.ny ||
        (N == 3 && (unsigned)pz >= (unsigned)P.nz))
        return best;
    const bool ex = px + 1 < P.nx, ey = py + 1 < P.ny, ez = N == 3 && pz + 1 < P.nz;
    const long long sy = P.nx, sz = (long long)P.nx * P.ny;
    const long long p = (long long)pz * sz + (long long)py * sy + px;
    float q[8];
    uint32_t ok = 0;
    float qmin = kInf, qmax = -kInf;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        q[u] = 0.f;
        if (u < (1 << N)) {
            const bool present = (!(u & 1) || ex) && (!(u & 2) || ey) && (!(u & 4) || ez);
            if (present) {
                const long long o = p + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) + ((u & 4) ? sz : 0);
                q[u] = (__ldg(P.ev + o) - dr) * inv;
                qmin = fminf(qmin, q[u]);
                qmax = fmaxf(qmax, q[u]);
                ok |= 1u << u;
            }
        }
    }
    // every point of the cell's faces has spatial distance >= key and a dose
    // coordinate in [qmin, qmax]
    const float gap = qmin > 0.f ? qmin : (qmax < 0.f ? -qmax : 0.f);
    if (fmaf(gap, gap, key * key) >= best) {
        if (P.stats) ++st.pruned;
        return best;
    }
    if (P.stats) ++st.visited;
    const float cb = cell_all_faces<N>(P, q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], ok, cx, cy,
                                       cz, p, dr, dnorm);
    return fminf(best, cb);
}

template <int G>
__device__ __forceinline__ float group_min(float v, unsigned gmask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(gmask, v, o));
    return v;
}

// The walk ran past a truncated table with the running bound still above
// the cover radius: scan every cell of the remaining search box, G lanes
// together (rare; keeps the result exact).
template <int N, int G>
__device__ __forceinline__ float tail_box_scan(const Problem& P, int x, int y, int z, float dr,
                                            float inv, float dnorm, float best, int gl,
                                            unsigned gmask, TailStats& st)
{
    const float rc2 = P.r_cover * P.r_cover;
    const float g = sqrtf(best);
    const int ax = (int)ceilf(g / P.hn[0]) + 1;
    const int ay = (int)ceilf(g / P.hn[1]) + 1;
    const int az = N == 3 ? (int)ceilf(g / P.hn[2]) + 1 : 0;
    const int x0 = max(-ax - 1, -x), x1 = min(ax, P.nx - 1 - x);
    const int y0 = max(-ay - 1, -y), y1 = min(ay, P.ny - 1 - y);
    const int z0 = N == 3 ? max(-az - 1, -z) : 0, z1 = N == 3 ? min(az, P.nz - 1 - z) : 0;
    const long long bx = x1 - x0 + 1, by = y1 - y0 + 1, bz = z1 - z0 + 1;
    const long long tot = bx * by * bz;
    const float lim = rc2 * 0.99999f;
    float lb = best;
    for (long long b = gl; b < tot; b += G) {
        const int cx = x0 + (int)(b % bx);
        const long long rr = b / bx;
        const int cy = y0 + (int)(rr % by);
        const int cz = z0 + (int)(rr / by);
        const float axd = (float)max(max(cx, -cx - 1), 0) * P.hn[0];
        const float ayd = (float)max(max(cy, -cy - 1), 0) * P.hn[1];
        const float azd = N == 3 ? (float)max(max(cz, -cz - 1), 0) * P.hn[2] : 0.f;
        float k2 = axd * axd + ayd * ayd + azd * azd;
        if (k2 == 0.f)       // key-0 cell: only its faces off the voxel remain
            k2 = P.key0_far2[(cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2)];
        if (k2 < lim || k2 >= lb) continue;
        lb = visit_cell<N>(P, x, y, z, cx, cy, cz, sqrtf(k2), dr, inv, dnorm, lb, st);
    }
    return group_min<G>(lb, gmask);
}

template <int N, int G, int MINB, bool BATCH>
__global__ void __launch_bounds__(256, MINB)
    k_tail(const __grid_constant__ Problem P0, const BatchDesc* __restrict__ bd)
{
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << gbase);
    const unsigned total = BATCH ? bd->item_start[kNumBuckets * bd->npairs]
                                 : min(P0.ctr->tail_count, P0.tail_cap);
    unsigned* head = BATCH ? bd->head : &P0.ctr->head;
    unsigned int my_eval = 0, my_pass = 0, my_over = 0;
    int my_pair = -1;          // batched: pair whose counts my_* hold
    TailStats st;
    // batched launches: hand this lane's counts to their pair
    auto flush_pair = [&]() {
        if (my_pair >= 0 && gl == 0) {
            Counters* c = bd->probs[my_pair].ctr;
            if (my_eval) atomicAdd(&c->n_eval, (unsigned long long)my_eval);
            if (my_pass) atomicAdd(&c->n_pass, (unsigned long long)my_pass);
            if (my_over) atomicAdd(&c->overflow_count, my_over);
        }
        my_eval = my_pass = my_over = 0;
    };

    for (;;) {
        unsigned item = 0;
        if (gl == 0) item = atomicAdd(head, 1u);
        item = __shfl_sync(gmask, item, gbase);
        if (item >= total) break;
        int pr = 0;
        unsigned v;
        if constexpr (BATCH) {
            v = bd->items_v[item];
            pr = bd->items_p[item];
            if (pr != my_pair) {                 // uniform over the group
                flush_pair();
                my_pair = pr;
            }
        } else {
            v = P0.sort_tail ? P0.tail_sorted[item] : P0.tail_raw[item];
        }
        const Problem& P = BATCH ? bd->probs[pr] : P0;
        const float dnorm = resolve_dnorm(P);
        const float rc2 = P.r_cover * P.r_cover;
        const int x = (int)(v % (unsigned)P.nx);
        const unsigned r1 = v / (unsigned)P.nx;
        const int y = (int)(r1 % (unsigned)P.ny);
        const int z = (int)(r1 / (unsigned)P.ny);
        const float dr = __ldg(P.ref + v);
        const float dD = P.dd_frac * (P.local ? dr : dnorm);
        const float inv = 1.0f / dD;
        float best = P.out[v];                       // gamma^2 over the faces through v
        int t = 0;
        while (t < P.ntable) {
            const int idx = t + gl;
            float key = kInf;
            uint32_t off = 0;
            if (idx < P.ntable) {
                const TableEntry e = P.table[idx];
                key = e.key;
                off = e.off;
            }
            const float k0 = __shfl_sync(gmask, key, gbase);
            if (k0 * k0 >= best) break;                   // A1 step 4b-ii, exact
            float cb = best;
            if (key * key < best) {
                if (P.stats) ++st.keyed;
                cb = visit_cell<N>(P, x, y, z, unpack10(off, 0), unpack10(off, 10),
                                   unpack10(off, 20), key, dr, inv, dnorm, best, st);
            }
            best = group_min<G>(cb, gmask);
            t += G;
        }
        if (t >= P.ntable && best > rc2) {
            if (gl == 0) ++my_over;
            best = tail_box_scan<N, G>(P, x, y, z, dr, inv, dnorm, best, gl, gmask, st);
        }
        if (gl == 0) {
            const float gam = sqrtf(best);
            P.out[v] = gam;
            ++my_eval;
            my_pass += gam <= 1.f;
        }
    }
    if constexpr (BATCH) flush_pair();
    if constexpr (!BATCH) {      // single-pair totals (batched ones went out per pair run)
        const Problem& P = P0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            my_eval += __shfl_xor_sync(kFull, my_eval, o);
            my_pass += __shfl_xor_sync(kFull, my_pass, o);
            my_over += __shfl_xor_sync(kFull, my_over, o);
            if (P.stats) {
                st.visited += __shfl_xor_sync(kFull, st.visited, o);
                st.pruned += __shfl_xor_sync(kFull, st.pruned, o);
                st.keyed += __shfl_xor_sync(kFull, st.keyed, o);
            }
        }
        if (lane == 0) {
            if (my_eval) atomicAdd(&P.ctr->n_eval, (unsigned long long)my_eval);
            if (my_pass) atomicAdd(&P.ctr->n_pass, (unsigned long long)my_pass);
            if (my_over) atomicAdd(&P.ctr->overflow_count, my_over);
            if (P.stats) {
                atomicAdd(&P.ctr->cells_visited, st.visited);
                atomicAdd(&P.ctr->cells_pruned, st.pruned);
                atomicAdd(&P.ctr->cells_keyed, st.keyed);
            }
        }
    }
}

// --------------------------------------------------------------------------
// k_tail_cq: surviving cells of the walks evaluated 32 at a time by the warp
// --------------------------------------------------------------------------

// In k_tail the face evaluation of a cell (the bulk of the work) runs with
// only the lanes whose cell passed the dose-gap test active.  Here a voxel's
// walk appends each cell that passes the test, with its vertex doses, to a
// ring buffer of the warp instead of evaluating it; whenever 32 cells wait,
// the whole warp evaluates them together, one per lane, and lowers each
// owner's running bound in shared memory (atomicMin on the bits of a
// non-negative float).  A walk may therefore key and test a few cells against
// a bound that is not yet the lowest: the stop (key >= bound) and the prune
// (key^2 + gap^2 >= bound) stay exact with any bound that is at least the
// true minimum, and each cell is evaluated with the arithmetic of k_tail, so
// the map is the one k_tail writes.  A voxel is final once every cell it
// appended has been evaluated; a walker has two voxel slots so that it can
// start its next voxel while the cells of the previous one still wait.
//
// The queue is ordered by cost bucket, most expensive first: the voxels of
// bucket cq_group8_bucket and above walk 8 lanes each (8 table entries per
// step), those of bucket cq_group_bucket and above 4 lanes each, which
// shortens the longest walks; the rest walk one lane each.  The
// rare paths (a cell whose Gram matrix is near singular, a walk that runs past
// a truncated table) are not taken here: such a voxel goes to fix_list with
// its bound, and k_tail_fix finishes it, so that this kernel's registers stay
// those of the FP32 evaluation.
constexpr int kCqRing = 64;               // ring of pending cells per warp
constexpr int kCqMinWalking = 16;         // flush a partial batch below this many walking lanes

// Per-warp shared state.  A walker's state (one lane, or the first lane of a
// group) lives here rather than in registers.
struct CqWarp {
    float q[8][kCqRing];       // vertex doses of a pending cell (relative, normalised)
    unsigned off[kCqRing];     // its offset from the voxel, packed as in the table
    unsigned meta[kCqRing];    // owner slot (bits 0-5), vertices inside the grid (bits 8-15)
    unsigned best[64];         // running squared gamma per voxel slot (float bits)
    unsigned vox[64];          // voxel index per slot
    float dr[64];              // reference dose per slot
    float inv[64];             // 1 / Delta D per slot
    unsigned fixm[2];          // slots whose voxel goes to the finishing pass
    int xyz[3][32];            // the walking voxel's grid position, per walker
    int t[32];                 // its next table entry
    unsigned wseq[32];         // sequence number of the last cell it appended
    unsigned dseq[32];         // the same for the voxel in the drain slot
    unsigned state[32];        // kCq* bits below
    unsigned cnt[2][32];       // voxels finished and passed
    int cpair[32];             // batched: the pair those counts belong to
    unsigned short pair[64];   // batched: the pair of each voxel slot
    unsigned long long stat[3][32];    // cells visited, pruned, keyed (option "stats")
};
// Batched launches: the walking voxel's grid and table, per walker, cached
// when it takes the voxel (a pair's Problem lives in global memory).
struct CqWalkDims {
    int dim[4][32];            // nx, ny, nz, table length
    const TableEntry* tab[32];
    const float* ev[32];
};
constexpr unsigned kCqWalk = 1u, kCqEnded = 2u, kCqWPend = 4u, kCqDBusy = 8u, kCqDPend = 16u,
                   kCqDOver = 32u, kCqSlot = 64u;     // slot bit: the walking slot is walker + 32

// Lanes per voxel of the four parts of the queue.
constexpr int kCqParts = 4;
__device__ __forceinline__ int cq_part_lanes(int part)
{
    return part == 0 ? 32 : (part == 1 ? 8 : (part == 2 ? 4 : 1));
}

// The problem a voxel slot belongs to: the launch's own, or (batched) that of
// the slot's pair.
template <bool BATCH>
__device__ __forceinline__ const Problem& cq_prob(const Problem& P0, const BatchDesc* bd,
                                                  volatile const CqWarp& V, int slot)
{
    if constexpr (BATCH) return bd->probs[V.pair[slot]];
    else return P0;
}

// Hands a walker's counts to their pair (batched launches).
__device__ __forceinline__ void cq_flush_counts(const BatchDesc* bd, volatile CqWarp& V, int w)
{
    const int pr = V.cpair[w];
    if (pr >= 0) {
        Counters* c = bd->probs[pr].ctr;
        if (V.cnt[0][w]) atomicAdd(&c->n_eval, (unsigned long long)V.cnt[0][w]);
        if (V.cnt[1][w]) atomicAdd(&c->n_pass, (unsigned long long)V.cnt[1][w]);
    }
    V.cnt[0][w] = 0;
    V.cnt[1][w] = 0;
}

template <int N, int MINB, bool BATCH>
__global__ void __launch_bounds__(256, MINB)
    k_tail_cq(const __grid_constant__ Problem P0, const BatchDesc* __restrict__ bd)
{
    __shared__ CqWarp cqw[8];
    __shared__ CqWalkDims cqd[BATCH ? 8 : 1];
    __shared__ unsigned s_end[kCqParts];   // the parts of the queue end at these items
    __shared__ float s_dnorm;              // single pair: its dose norm
    CqWarp& W = cqw[threadIdx.x >> 5];
    volatile CqWarp& V = cqw[threadIdx.x >> 5];
    volatile CqWalkDims& VD = cqd[BATCH ? threadIdx.x >> 5 : 0];
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (threadIdx.x < 32) {
        if constexpr (BATCH) {
            // the group's queue: voxels of bucket >= the group bucket of every
            // pair first, then the rest (k_bucket_scan_batch)
            if (lane == 0) {
                const int nb = kNumBuckets * bd->npairs;
                s_end[0] = bd->item_start[nb + 1];
                s_end[1] = bd->item_start[nb + 2];
                s_end[2] = bd->item_start[nb + 3];
                s_end[3] = bd->item_start[nb];
            }
        } else {
            // the cost-ordered queue: items of bucket >= cq_group32_bucket
            // first, then those of bucket >= cq_group8_bucket, then >=
            // cq_group_bucket, then the rest
            const Problem& P = P0;
            const unsigned total = min(P.ctr->tail_count, P.tail_cap);
            const unsigned hb = P.sort_tail ? P.ctr->hist[lane] : 0u;
            int b32 = P.cq_group32_bucket, b8 = min(P.cq_group8_bucket, b32), b4 = min(P.cq_group_bucket, b8);
            if (P.cq_group_bucket < 0)
                auto_part_buckets(hb, gridDim.x * blockDim.x, P.cq_auto_scale, b4, b8, b32);
            unsigned h32 = lane >= b32 ? hb : 0u, h8 = lane >= b8 ? hb : 0u, h4 = lane >= b4 ? hb : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                h32 += __shfl_xor_sync(kFull, h32, o);
                h8 += __shfl_xor_sync(kFull, h8, o);
                h4 += __shfl_xor_sync(kFull, h4, o);
            }
            if (lane == 0) {
                s_dnorm = resolve_dnorm(P);
                s_end[0] = min(h32, total);
                s_end[1] = min(h8, total);
                s_end[2] = min(h4, total);
                s_end[3] = total;
            }
        }
    }
    W.state[lane] = 0;
    W.wseq[lane] = W.dseq[lane] = 0;
    W.cnt[0][lane] = W.cnt[1][lane] = 0;
    W.cpair[lane] = -1;
    W.pair[lane] = W.pair[lane + 32] = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) W.stat[k][lane] = 0;
    if (lane < 2) W.fixm[lane] = 0;
    __syncthreads();
    unsigned* const heads = BATCH ? bd->part_head : P0.ctr->head_part;

    int part = 0;                      // the part of the queue this warp takes voxels from
    while (part < kCqParts - 1 && s_end[part] == (part ? s_end[part - 1] : 0u)) ++part;
    int g = cq_part_lanes(part);       // its lanes per voxel
    unsigned head = 0, count = 0;      // the ring: pending cells are [head, head + count)
    bool queue_done = false;           // warp-uniform, for the current part
    unsigned long long steps = 0;      // loop steps of this warp (option "stats")
    for (;;) {
        if (!BATCH && P0.stats) ++steps;
        const int gl = lane & (g - 1), ld = lane - gl;
        const bool leader = gl == 0;
        const unsigned gmask = g == 32 ? kFull : ((1u << g) - 1u) << ld;
        unsigned sta = V.state[ld];
        if (leader) {
            // 1. a drained voxel whose cells are all evaluated is final
            if ((sta & kCqDBusy) && (!(sta & kCqDPend) || (int)(head - V.dseq[ld]) > 0)) {
                const int ds = ld + ((sta & kCqSlot) ? 0 : 32);
                const Problem& Q = cq_prob<BATCH>(P0, bd, V, ds);
                const float best = __uint_as_float(V.best[ds]);
                const unsigned v = V.vox[ds];
                if (((V.fixm[ds >> 5] >> (ds & 31)) & 1u) ||
                    ((sta & kCqDOver) && best > Q.r_cover * Q.r_cover)) {
                    Q.out[v] = best;                        // gamma^2: k_tail_fix completes it
                    if constexpr (BATCH) {
                        const unsigned k = atomicAdd(bd->fix_count, 1u);
                        bd->fix_v[k] = v;
                        bd->fix_p[k] = V.pair[ds];
                    } else {
                        Q.fix_list[atomicAdd(&Q.ctr->fix_count, 1u)] = v;
                    }
                } else {
                    const float gam = sqrtf(best);
                    Q.out[v] = gam;
                    if constexpr (BATCH) {
                        if (V.cpair[ld] != (int)V.pair[ds]) {
                            cq_flush_counts(bd, V, ld);
                            V.cpair[ld] = V.pair[ds];
                        }
                    }
                    ++V.cnt[0][ld];
                    if (gam <= 1.f) ++V.cnt[1][ld];
                }
                sta &= ~kCqDBusy;
            }
            // 2. an ended walk becomes the drain slot; the walker takes a new voxel
            if ((sta & kCqEnded) && !(sta & kCqDBusy)) {
                const int ws = ld + ((sta & kCqSlot) ? 32 : 0);
                unsigned d = kCqDBusy;
                if (sta & kCqWPend) d |= kCqDPend;
                if (V.t[ld] >= (BATCH ? VD.dim[3][ld] : P0.ntable)) d |= kCqDOver;
                V.dseq[ld] = V.wseq[ld];
                sta = d | ((sta & kCqSlot) ^ kCqSlot);
            }
        }
        // 3. refill the empty walkers from the current part of the queue
        const bool empty = leader && !(sta & (kCqWalk | kCqEnded));
        const unsigned need = __ballot_sync(kFull, empty);
        if (need && !queue_done) {
            const unsigned lo = part ? s_end[part - 1] : 0u, hi = s_end[part];
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&heads[part], (unsigned)__popc(need));
            base = __shfl_sync(kFull, base, 0) + lo;
            if (base + (unsigned)__popc(need) >= hi) queue_done = true;
            if (empty) {
                const unsigned item = base + (unsigned)__popc(need & lt_mask);
                if (item < hi) {
                    const int ws = ld + ((sta & kCqSlot) ? 32 : 0);
                    unsigned v;
                    if constexpr (BATCH) {
                        v = bd->items_v[item];
                        V.pair[ws] = bd->items_p[item];
                    } else {
                        v = P0.sort_tail ? P0.tail_sorted[item] : P0.tail_raw[item];
                    }
                    const Problem& Q = cq_prob<BATCH>(P0, bd, V, ws);
                    V.xyz[0][ld] = (int)(v % (unsigned)Q.nx);
                    const unsigned r1 = v / (unsigned)Q.nx;
                    V.xyz[1][ld] = (int)(r1 % (unsigned)Q.ny);
                    V.xyz[2][ld] = (int)(r1 / (unsigned)Q.ny);
                    const float dr = __ldg(Q.ref + v);
                    V.dr[ws] = dr;
                    V.inv[ws] = 1.0f / (Q.dd_frac * (Q.local ? dr : (BATCH ? resolve_dnorm(Q) : s_dnorm)));
                    V.best[ws] = __float_as_uint(Q.out[v]);  // gamma^2 over the faces through v
                    V.vox[ws] = v;
                    if constexpr (BATCH) {
                        VD.dim[0][ld] = Q.nx;
                        VD.dim[1][ld] = Q.ny;
                        VD.dim[2][ld] = Q.nz;
                        VD.dim[3][ld] = Q.ntable;
                        VD.tab[ld] = Q.table;
                        VD.ev[ld] = Q.ev;
                    }
                    atomicAnd(&W.fixm[ws >> 5], ~(1u << (ws & 31)));
                    V.t[ld] = 0;
                    sta = (sta & ~kCqWPend) | kCqWalk;
                }
            }
        }
        if (leader) V.state[ld] = sta;
        __syncwarp();
        sta = V.state[ld];                 // the group's lanes follow their walker
        if (queue_done && !__any_sync(kFull, (sta & (kCqWalk | kCqEnded | kCqDBusy)) != 0)) {
            if (part == kCqParts - 1) break;
            ++part;                        // this part is done: the next, with fewer lanes per voxel
            g = cq_part_lanes(part);
            queue_done = false;
            V.state[lane] = 0;
            __syncwarp();
            continue;
        }

        // 4. one table step of every walking group: entries t .. t + g - 1
        const bool walking = (sta & kCqWalk) != 0;
        const int ws = ld + ((sta & kCqSlot) ? 32 : 0);
        // the walking voxel's grid and table (batched: cached at its refill)
        const int qnx = BATCH ? VD.dim[0][ld] : P0.nx, qny = BATCH ? VD.dim[1][ld] : P0.ny;
        const int qnz = BATCH ? VD.dim[2][ld] : P0.nz, qnt = BATCH ? VD.dim[3][ld] : P0.ntable;
        const TableEntry* qtab = BATCH ? VD.tab[ld] : P0.table;
        const float* qev = BATCH ? VD.ev[ld] : P0.ev;
        const bool qstats = !BATCH && P0.stats;
        const int t0 = walking ? V.t[ld] : 0;
        float key = kInf;
        uint32_t off = 0;
        if (walking && t0 + gl < qnt) {
            const TableEntry e = qtab[t0 + gl];
            key = e.key;
            off = e.off;
        }
        const float k0 = __shfl_sync(kFull, key, ld);
        bool cand = false, ended = false;
        float q[8];
        uint32_t ok = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = 0.f;
        if (walking) {
            const float bst = __uint_as_float(V.best[ws]);
            ended = t0 >= qnt || k0 * k0 >= bst;              // A1 step 4b-ii, exact
            if (!ended && key * key < bst) {
                if (qstats) ++V.stat[2][lane];
                const int px = V.xyz[0][ld] + unpack10(off, 0);
                const int py = V.xyz[1][ld] + unpack10(off, 10);
                const int pz = V.xyz[2][ld] + unpack10(off, 20);
                if ((unsigned)px < (unsigned)qnx && (unsigned)py < (unsigned)qny &&
                    (N == 2 || (unsigned)pz < (unsigned)qnz)) {
                    const long long sy = qnx, sz = (long long)qnx * qny;
                    const bool ex = px + 1 < qnx, ey = py + 1 < qny, ez = N == 3 && pz + 1 < qnz;
                    const long long p = (long long)pz * sz + (long long)py * sy + px;
                    const float dr = V.dr[ws], inv = V.inv[ws];
                    float qmin = kInf, qmax = -kInf;
#pragma unroll
                    for (int u = 0; u < (1 << N); ++u) {
                        const bool present = (!(u & 1) || ex) && (!(u & 2) || ey) && (!(u & 4) || ez);
                        if (present) {
                            const long long o = p + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) +
                                                ((u & 4) ? sz : 0);
                            q[u] = (__ldg(qev + o) - dr) * inv;
                            qmin = fminf(qmin, q[u]);
                            qmax = fmaxf(qmax, q[u]);
                            ok |= 1u << u;
                        }
                    }
                    const float gap = qmin > 0.f ? qmin : (qmax < 0.f ? -qmax : 0.f);
                    if (fmaf(gap, gap, key * key) >= bst) {
                        if (qstats) ++V.stat[1][lane];
                    } else {
                        cand = true;
                    }
                }
            }
        }
        // 5. append the surviving cells to the ring
        const unsigned cm = __ballot_sync(kFull, cand);
        if (cand) {
            const unsigned seq = head + count + (unsigned)__popc(cm & lt_mask);
            const int slot = (int)(seq & (kCqRing - 1));
#pragma unroll
            for (int u = 0; u < (1 << N); ++u) V.q[u][slot] = q[u];
            V.off[slot] = off;
            V.meta[slot] = (unsigned)ws | (ok << 8);
        }
        if (leader && walking) {
            if (ended) {
                sta = (sta & ~kCqWalk) | kCqEnded;
            } else {
                V.t[ld] = t0 + g;
                const unsigned gm = cm & gmask;
                if (gm) {                   // the group's last appended cell
                    const int hl = 31 - __clz(gm);
                    V.wseq[ld] = head + count + (unsigned)__popc(cm & ((1u << hl) - 1u));
                    sta |= kCqWPend;
                }
            }
            V.state[ld] = sta;
        }
        count += (unsigned)__popc(cm);
        const int nwalk = g * __popc(__ballot_sync(kFull, leader && (sta & kCqWalk) && !ended));
        __syncwarp();
        // 6. evaluate the oldest 32 pending cells (or fewer, when few lanes walk)
        if (count >= 32u || (count > 0u && nwalk < kCqMinWalking)) {
            const unsigned n = min(count, 32u);
            if ((unsigned)lane < n) {
                const int slot = (int)((head + (unsigned)lane) & (kCqRing - 1));
                const unsigned meta = V.meta[slot];
                const int owner = (int)(meta & 63u);
                const unsigned cok = meta >> 8;
                const unsigned coff = V.off[slot];
                float cq[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) cq[u] = u < (1 << N) ? V.q[u][slot] : 0.f;
                auto evaluate = [&](const Metric& mt, float dmax, float tau) {
                    CellGeom<float> cg;
                    cell_geom<N, float>(unpack10(coff, 0), unpack10(coff, 10), unpack10(coff, 20), mt, cg);
                    bool ill = false;
                    const float cb = cell_min_d2<N, float>(cq, cok, cg, mt, dmax, kInf, ill);
                    if (ill && cell_gram_ill<N>(cq, cok, mt.kappa, tau))
                        atomicOr(&W.fixm[owner >> 5], 1u << (owner & 31));   // k_tail_fix redoes it
                    else
                        atomicMin(&W.best[owner], __float_as_uint(cb + 0.f));   // -0 -> +0
                };
                if constexpr (BATCH) {
                    // the owner's pair's metric: three 16-byte loads
                    const float4* m4 = bd->metric4 + 3 * (int)V.pair[owner];
                    const float4 a = m4[0], b = m4[1], c = m4[2];
                    Metric mt;
                    mt.hn2[0] = a.x; mt.hn2[1] = a.y; mt.hn2[2] = a.z;
                    mt.kappa[0] = 0.f;
                    mt.kappa[1] = b.x; mt.kappa[2] = b.y; mt.kappa[3] = b.z; mt.kappa[4] = b.w;
                    mt.kappa[5] = c.x; mt.kappa[6] = c.y; mt.kappa[7] = c.z;
                    evaluate(mt, a.w > 0.f ? 0.99f * rsqrtf(a.w) : kInf, a.w);   // bound as ill_dmax
                } else {
                    evaluate(P0.mt, ill_dmax(P0), P0.tau);
                }
                if (!BATCH && P0.stats) ++V.stat[0][lane];
            }
            head += n;
            count -= n;
        }
        __syncwarp();
    }
    if constexpr (BATCH) {
        cq_flush_counts(bd, V, lane);          // per-pair counts of every walker
    } else {
        // per-warp totals
        const Problem& P = P0;
        unsigned c0 = W.cnt[0][lane], c1 = W.cnt[1][lane];
        unsigned long long s0 = W.stat[0][lane], s1 = W.stat[1][lane], s2 = W.stat[2][lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c0 += __shfl_xor_sync(kFull, c0, o);
            c1 += __shfl_xor_sync(kFull, c1, o);
            s0 += __shfl_xor_sync(kFull, s0, o);
            s1 += __shfl_xor_sync(kFull, s1, o);
            s2 += __shfl_xor_sync(kFull, s2, o);
        }
        if (lane == 0) {
            if (c0) atomicAdd(&P.ctr->n_eval, (unsigned long long)c0);
            if (c1) atomicAdd(&P.ctr->n_pass, (unsigned long long)c1);
            if (P.stats) {
                atomicAdd(&P.ctr->cells_visited, s0);
                atomicAdd(&P.ctr->cells_pruned, s1);
                atomicAdd(&P.ctr->cells_keyed, s2);
                atomicAdd(&P.ctr->lane_steps, 32ull * steps);
            }
        }
    }
}

// Finishing pass of k_tail_cq: one warp per voxel of the fix list, whose
// bound (gamma^2, an upper bound of the result) is in out.  The walk of
// k_tail (32 lanes, FP64 redo of near-singular cells) from that bound, then
// the box scan when it runs past the table.
template <int N, bool BATCH>
__global__ void __launch_bounds__(256) k_tail_fix(const __grid_constant__ Problem P0,
                                                  const BatchDesc* __restrict__ bd)
{
    const int lane = threadIdx.x & 31;
    const unsigned nfix = BATCH ? *bd->fix_count : P0.ctr->fix_count;
    unsigned my_eval = 0, my_pass = 0, my_over = 0;
    TailStats st;
    for (unsigned i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nfix;
         i += (gridDim.x * blockDim.x) >> 5) {
        const Problem& P = BATCH ? bd->probs[bd->fix_p[i]] : P0;
        const unsigned v = BATCH ? bd->fix_v[i] : P.fix_list[i];
        const float dnorm = resolve_dnorm(P);
        const int x = (int)(v % (unsigned)P.nx);
        const unsigned r1 = v / (unsigned)P.nx;
        const int y = (int)(r1 % (unsigned)P.ny), z = (int)(r1 / (unsigned)P.ny);
        const float dr = __ldg(P.ref + v);
        const float inv = 1.0f / (P.dd_frac * (P.local ? dr : dnorm));
        float best = P.out[v];
        int t = 0;
        while (t < P.ntable) {
            const int idx = t + lane;
            float key = kInf;
            uint32_t off = 0;
            if (idx < P.ntable) {
                const TableEntry e = P.table[idx];
                key = e.key;
                off = e.off;
            }
            const float k0 = __shfl_sync(kFull, key, 0);
            if (k0 * k0 >= best) break;
            float cb = best;
            if (key * key < best) {
                if (P.stats) ++st.keyed;
                cb = visit_cell<N>(P, x, y, z, unpack10(off, 0), unpack10(off, 10), unpack10(off, 20),
                                   key, dr, inv, dnorm, best, st);
            }
            best = group_min<32>(cb, kFull);
            t += 32;
        }
        const bool over = t >= P.ntable && best > P.r_cover * P.r_cover;
        if (over) best = tail_box_scan<N, 32>(P, x, y, z, dr, inv, dnorm, best, lane, kFull, st);
        if (lane == 0) {
            const float gam = sqrtf(best);
            P.out[v] = gam;
            if constexpr (BATCH) {
                atomicAdd(&P.ctr->n_eval, 1ull);
                if (gam <= 1.f) atomicAdd(&P.ctr->n_pass, 1ull);
                if (over) atomicAdd(&P.ctr->overflow_count, 1u);
            } else {
                ++my_eval;
                my_pass += gam <= 1.f;
                my_over += over;
            }
        }
    }
    if constexpr (!BATCH) {
        const Problem& P = P0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            my_eval += __shfl_xor_sync(kFull, my_eval, o);
            my_pass += __shfl_xor_sync(kFull, my_pass, o);
            my_over += __shfl_xor_sync(kFull, my_over, o);
            if (P.stats) {
                st.visited += __shfl_xor_sync(kFull, st.visited, o);
                st.pruned += __shfl_xor_sync(kFull, st.pruned, o);
                st.keyed += __shfl_xor_sync(kFull, st.keyed, o);
            }
        }
        if (lane == 0) {
            if (my_eval) atomicAdd(&P.ctr->n_eval, (unsigned long long)my_eval);
            if (my_pass) atomicAdd(&P.ctr->n_pass, (unsigned long long)my_pass);
            if (my_over) atomicAdd(&P.ctr->overflow_count, my_over);
            if (P.stats) {
                atomicAdd(&P.ctr->cells_visited, st.visited);
                atomicAdd(&P.ctr->cells_pruned, st.pruned);
                atomicAdd(&P.ctr->cells_keyed, st.keyed);
            }
        }
    }
}

// --------------------------------------------------------------------------
// k_walk: tile-staged walk of the queued voxels, one shell tile per block
// --------------------------------------------------------------------------

// Halo box of a walk tile in shared memory: the shell tile plus H voxels on
// every side (the x start stays a multiple of 4 floats for the TMA copy).
// Every cell whose corner lies within H - 1 voxels of a tile voxel (cells
// with box distance up to (H - 1) h) reads its eight doses from the box;
// cells further out read global memory.
template <int N>
struct WalkBox {
    using T = ShellTile<N>;
    static constexpr int H = 4;
    static constexpr int BX = T::TX + 2 * H, BY = T::TY + 2 * H, BZ = N == 3 ? T::TZ + 2 * H : 1;
    static constexpr int ELEMS = BX * BY * BZ;
    static constexpr int STRIDE = (ELEMS + 31) / 32 * 32;
    static_assert(STRIDE * 4 % 128 == 0, "TMA destination must stay 128-byte aligned");
    static_assert(H % 4 == 0, "the box's x start must stay 16-byte aligned");
};

constexpr int kWalkTableCache = 1024;        // first table entries kept in shared memory

// visit_cell with the eight doses from the staged box B when the whole cell
// lies inside it (b0x, b0y, b0z: grid coordinates of the box's first element).
template <int N, class B = WalkBox<N>>
__device__ __forceinline__ float visit_cell_box(const Problem& P, const float* __restrict__ bx,
                                                int b0x, int b0y, int b0z, int x, int y, int z,
                                                int cx, int cy, int cz, float key, float dr,
                                                float inv, float dnorm, float best, TailStats& st)
{
    const int px = x + cx, py = y + cy, pz = z + cz;
    if ((unsigned)px >= (unsigned)P.nx || (unsigned)py >= (unsigned)P.ny ||
        (N == 3 && (unsigned)pz >= (unsigned)P.nz))
        return best;
    const bool ex = px + 1 < P.nx, ey = py + 1 < P.ny, ez = N == 3 && pz + 1 < P.nz;
    const int lx = px - b0x, ly = py - b0y, lz = N == 3 ? pz - b0z : 0;
    const bool inbox = (unsigned)lx <= (unsigned)(B::BX - 2) && (unsigned)ly <= (unsigned)(B::BY - 2) &&
                       (N == 2 || (unsigned)lz <= (unsigned)(B::BZ - 2));
    const long long sy = P.nx, sz = (long long)P.nx * P.ny;
    const long long p = (long long)pz * sz + (long long)py * sy + px;
    const int lp = (lz * B::BY + ly) * B::BX + lx;
    float q[8];
    uint32_t ok = 0;
    float qmin = kInf, qmax = -kInf;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        q[u] = 0.f;
        if (u < (1 << N)) {
            const bool present = (!(u & 1) || ex) && (!(u & 2) || ey) && (!(u & 4) || ez);
            if (present) {
                const int lo = ((u & 1) ? 1 : 0) + ((u & 2) ? B::BX : 0) + ((u & 4) ? B::BX * B::BY : 0);
                const long long o = p + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) + ((u & 4) ? sz : 0);
                const float d = inbox ? bx[lp + lo] : __ldg(P.ev + o);
                q[u] = (d - dr) * inv;
                qmin = fminf(qmin, q[u]);
                qmax = fmaxf(qmax, q[u]);
                ok |= 1u << u;
            }
        }
    }
    const float gap = qmin > 0.f ? qmin : (qmax < 0.f ? -qmax : 0.f);
    if (fmaf(gap, gap, key * key) >= best) {
        if (P.stats) ++st.pruned;
        return best;
    }
    if (P.stats) ++st.visited;
    const float cb = cell_all_faces<N>(P, q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], ok, cx, cy,
                                       cz, p, dr, dnorm);
    return fminf(best, cb);
}

// Minimum over the G lanes of a group (G a power of two <= 32, lanes gbase ..
// gbase + G - 1 of the warp, mask gmask).
__device__ __forceinline__ float group_min_rt(float v, int G, unsigned gmask)
{
    for (int o = G >> 1; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(gmask, v, o));
    return v;
}

// One block per tile with queued voxels, in cost order: the halo box of the
// tile arrives by TMA (double-buffered, the next tile's copy in flight while
// this one is walked); the tile's queued voxels are read from its bit mask;
// G lanes per voxel (G chosen per tile from the number of queued voxels so
// that the block's 256 threads are used) walk the sorted cell table G cells
// at a time with the exact stop of Algorithm A1 step 4b-ii and the dose-gap
// bound, reading cell doses from the box.
template <int N, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_walk(const __grid_constant__ Problem P, const __grid_constant__ CUtensorMap wmap, int use_tma)
{
    using T = ShellTile<N>;
    using B = WalkBox<N>;
    __shared__ __align__(128) float box[2][B::STRIDE];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ TableEntry sh_table[kWalkTableCache];
    __shared__ unsigned short sh_q[T::TX * T::TY * T::TZ];
    __shared__ int sh_nq;
    __shared__ int sh_next[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned ntiles = P.ctr->tile_count;
    const unsigned* order = P.sort_tail ? P.tile_sorted : P.tile_list;
    const int ncache = min(P.ntable, kWalkTableCache);
    for (int i = tid; i < ncache; i += blockDim.x) sh_table[i] = P.table[i];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const float dnorm = resolve_dnorm(P);
    const float rc2 = P.r_cover * P.r_cover;
    const int ntx = (P.nx + T::TX - 1) / T::TX, nty = (P.ny + T::TY - 1) / T::TY;
    auto origin = [&](unsigned lt, int& x0, int& y0, int& z0) {
        x0 = (int)(lt % (unsigned)ntx) * T::TX;
        y0 = (int)((lt / (unsigned)ntx) % (unsigned)nty) * T::TY;
        z0 = N == 3 ? (int)(lt / (unsigned)ntx / (unsigned)nty) * T::TZ : 0;
    };
    auto issue = [&](unsigned i, int b) {
        if (i >= ntiles || !use_tma) return;
        int x0, y0, z0;
        origin(order[i], x0, y0, z0);
        mbar_arrive_expect_tx(&bar[b], B::ELEMS * (uint32_t)sizeof(float));
        if (N == 3) tma_load_3d(box[b], &wmap, x0 - B::H, y0 - B::H, z0 - B::H, &bar[b]);
        else tma_load_2d(box[b], &wmap, x0 - B::H, y0 - B::H, &bar[b]);
    };
    unsigned my_eval = 0, my_pass = 0, my_over = 0;
    TailStats st;
    uint32_t parity = 0;
    int buf = 0;
    unsigned i = blockIdx.x;
    if (tid == 0) issue(i, 0);
    for (; i < ntiles; buf ^= 1) {
        const unsigned lt = order[i];
        int x0, y0, z0;
        origin(lt, x0, y0, z0);
        const int b0x = x0 - B::H, b0y = y0 - B::H, b0z = N == 3 ? z0 - B::H : 0;
        if (tid == 0) {
            const unsigned nt = gridDim.x + atomicAdd(&P.ctr->tile_head, 1u);
            sh_next[buf] = (int)min(nt, ntiles);
            issue(nt, buf ^ 1);
        }
        // the tile's queued voxels, in voxel order (warp 0)
        if (warp == 0) {
            const unsigned w = lane < 8 ? P.tile_mask[(size_t)lt * 8 + lane] : 0u;
            const int c = __popc(w);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            int pos = incl - c;
            for (unsigned m = w; m; m &= m - 1) sh_q[pos++] = (unsigned short)(lane * 32 + __ffs(m) - 1);
            if (lane == 7) sh_nq = incl;
        }
        float* bx = box[buf];
        bool timed_out = false;
        if (use_tma) {
            timed_out = !mbar_wait_bounded(&bar[buf], (parity >> buf) & 1u);
            parity ^= 1u << buf;
        } else {
            for (int e = tid; e < B::ELEMS; e += blockDim.x) {
                const int ex_ = e % B::BX, ey_ = (e / B::BX) % B::BY, ez_ = e / (B::BX * B::BY);
                const int gx = b0x + ex_, gy = b0y + ey_, gz = b0z + ez_;
                const bool in = (unsigned)gx < (unsigned)P.nx && (unsigned)gy < (unsigned)P.ny &&
                                (N == 2 || (unsigned)gz < (unsigned)P.nz);
                bx[e] = in ? __ldg(P.ev + ((long long)gz * P.ny + gy) * P.nx + gx) : 0.f;
            }
        }
        __syncthreads();
        const int nq = sh_nq;
        int G = 32;
        while (G > 2 && nq * G > (int)blockDim.x) G >>= 1;
        const int slots = (int)blockDim.x / G;
        const int gl = tid & (G - 1);
        const int gbase = lane & ~(G - 1);
        const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << gbase);
        for (int k = tid / G; k < nq && !timed_out; k += slots) {
            const int q = sh_q[k];
            const int x = x0 + (q & 31), y = y0 + (q >> 5) % T::TY, z = z0 + (q >> 5) / T::TY;
            const unsigned v = (unsigned)(((long long)z * P.ny + y) * P.nx + x);
            const float dr = __ldg(P.ref + v);
            const float dD = P.dd_frac * (P.local ? dr : dnorm);
            const float inv = 1.0f / dD;
            float best = P.out[v];                       // gamma^2 over the faces through v
            int t = 0;
            while (t < P.ntable) {
                const int idx = t + gl;
                float key = kInf;
                uint32_t off = 0;
                if (idx < P.ntable) {
                    const TableEntry e = idx < kWalkTableCache ? sh_table[idx] : P.table[idx];
                    key = e.key;
                    off = e.off;
                }
                const float k0 = __shfl_sync(gmask, key, gbase);
                if (k0 * k0 >= best) break;               // A1 step 4b-ii, exact
                float cb = best;
                if (key * key < best) {
                    if (P.stats) ++st.keyed;
                    cb = visit_cell_box<N>(P, bx, b0x, b0y, b0z, x, y, z, unpack10(off, 0),
                                           unpack10(off, 10), unpack10(off, 20), key, dr, inv, dnorm,
                                           best, st);
                }
                best = group_min_rt(cb, G, gmask);
                t += G;
            }
            if (t >= P.ntable && best > rc2) {
                // past a truncated table: the exact scan of the remaining box
                if (gl == 0) ++my_over;
                const float g = sqrtf(best);
                const int ax = (int)ceilf(g / P.hn[0]) + 1;
                const int ay = (int)ceilf(g / P.hn[1]) + 1;
                const int az = N == 3 ? (int)ceilf(g / P.hn[2]) + 1 : 0;
                const int xa = max(-ax - 1, -x), xb = min(ax, P.nx - 1 - x);
                const int ya = max(-ay - 1, -y), yb = min(ay, P.ny - 1 - y);
                const int za = N == 3 ? max(-az - 1, -z) : 0, zb = N == 3 ? min(az, P.nz - 1 - z) : 0;
                const long long wx = xb - xa + 1, wy = yb - ya + 1, wz = zb - za + 1;
                const long long tot = wx * wy * wz;
                const float lim = rc2 * 0.99999f;
                float lb = best;
                for (long long b = gl; b < tot; b += G) {
                    const int cx = xa + (int)(b % wx);
                    const long long rr = b / wx;
                    const int cy = ya + (int)(rr % wy);
                    const int cz = za + (int)(rr / wy);
                    const float axd = (float)max(max(cx, -cx - 1), 0) * P.hn[0];
                    const float ayd = (float)max(max(cy, -cy - 1), 0) * P.hn[1];
                    const float azd = N == 3 ? (float)max(max(cz, -cz - 1), 0) * P.hn[2] : 0.f;
                    float k2 = axd * axd + ayd * ayd + azd * azd;
                    if (k2 == 0.f)
                        k2 = P.key0_far2[(cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2)];
                    if (k2 < lim || k2 >= lb) continue;
                    lb = visit_cell_box<N>(P, bx, b0x, b0y, b0z, x, y, z, cx, cy, cz, sqrtf(k2), dr,
                                           inv, dnorm, lb, st);
                }
                best = group_min_rt(lb, G, gmask);
            }
            if (gl == 0) {
                const float gam = sqrtf(best);
                P.out[v] = gam;
                ++my_eval;
                my_pass += gam <= 1.f;
            }
        }
        // box[buf] and sh_q are free for reuse once every thread is here
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) {
                atomicOr(&P.ctr->flags, kFlagTimeout);
                mbar_wait_bounded(&bar[buf], (parity >> buf) & 1u);
                mbar_wait_bounded(&bar[buf ^ 1], (parity >> (buf ^ 1)) & 1u);
            }
            break;
        }
        i = (unsigned)sh_next[buf];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_eval += __shfl_xor_sync(kFull, my_eval, o);
        my_pass += __shfl_xor_sync(kFull, my_pass, o);
        my_over += __shfl_xor_sync(kFull, my_over, o);
        if (P.stats) {
            st.visited += __shfl_xor_sync(kFull, st.visited, o);
            st.pruned += __shfl_xor_sync(kFull, st.pruned, o);
            st.keyed += __shfl_xor_sync(kFull, st.keyed, o);
        }
    }
    if (lane == 0) {
        if (my_eval) atomicAdd(&P.ctr->n_eval, (unsigned long long)my_eval);
        if (my_pass) atomicAdd(&P.ctr->n_pass, (unsigned long long)my_pass);
        if (my_over) atomicAdd(&P.ctr->overflow_count, my_over);
        if (P.stats) {
            atomicAdd(&P.ctr->cells_visited, st.visited);
            atomicAdd(&P.ctr->cells_pruned, st.pruned);
            atomicAdd(&P.ctr->cells_keyed, st.keyed);
        }
    }
}

// --------------------------------------------------------------------------
// k_walk_rows: row-staged walk, one shell warp row per warp at a time
// --------------------------------------------------------------------------

// Halo box of one shell warp row (32 voxels along x): 4 voxels on each side in
// x (the x start stays a multiple of 4 floats for the TMA copy) and RH in y
// and z.  Cells whose corner lies within 3 voxels in x and RH - 1 in y and z
// of the row's voxels read their doses from the box; others global memory.
template <int N>
struct RowBox {
    static constexpr int RH = 3;
    static constexpr int BX = 32 + 8, BY = 2 * RH + 1, BZ = N == 3 ? 2 * RH + 1 : 1;
    static constexpr int ELEMS = BX * BY * BZ;
    static constexpr int STRIDE = (ELEMS + 31) / 32 * 32;
    static_assert(STRIDE * 4 % 128 == 0, "TMA destination must stay 128-byte aligned");
};

// Every warp, independently: take the next row item in cost order, stage the
// row's halo box by one TMA copy into its own buffer (bounded wait), and walk
// the table for the row's queued voxels, G lanes each (G chosen from the
// number of queued voxels so that the warp's lanes are used), with the exact
// stop of Algorithm A1 step 4b-ii and the dose-gap bound.  No block barrier:
// a warp moves on as soon as its row is done, as in k_tail.
template <int N, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_walk_rows(const __grid_constant__ Problem P, const __grid_constant__ CUtensorMap rmap, int use_tma)
{
    using T = ShellTile<N>;
    using B = RowBox<N>;
    // the warps' boxes in dynamic shared memory (8 x B::STRIDE floats, from a
    // 128-byte boundary: TMA destinations)
    extern __shared__ __align__(128) unsigned char dyn_raw[];
    float* boxes = reinterpret_cast<float*>(dyn_raw + ((128u - (smem_addr(dyn_raw) & 127u)) & 127u));
    __shared__ __align__(8) uint64_t bar[8];
    __shared__ TableEntry sh_table[kWalkTableCache];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned nrows = P.ctr->row_count;
    const unsigned long long* order = P.sort_tail ? P.row_sorted : P.row_items;
    const int ncache = min(P.ntable, kWalkTableCache);
    for (int i = tid; i < ncache; i += blockDim.x) sh_table[i] = P.table[i];
    if (tid == 0) {
        for (int i = 0; i < 8; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const float dnorm = resolve_dnorm(P);
    const float rc2 = P.r_cover * P.r_cover;
    const int ntx = (P.nx + T::TX - 1) / T::TX, nty = (P.ny + T::TY - 1) / T::TY;
    float* bx = boxes + (size_t)w * B::STRIDE;
    unsigned my_eval = 0, my_pass = 0, my_over = 0;
    TailStats st;
    uint32_t phase = 0;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(&P.ctr->row_head, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= nrows) break;
        const unsigned long long item = order[it];
        const unsigned mask = (unsigned)item, rid = (unsigned)(item >> 32);
        const unsigned lt = rid >> 3, wr = rid & 7u;
        const int x0 = (int)(lt % (unsigned)ntx) * T::TX;
        const int y = (int)((lt / (unsigned)ntx) % (unsigned)nty) * T::TY + (int)(wr % T::TY);
        const int z = N == 3 ? (int)(lt / (unsigned)ntx / (unsigned)nty) * T::TZ + (int)(wr / T::TY) : 0;
        const int b0x = x0 - 4, b0y = y - B::RH, b0z = N == 3 ? z - B::RH : 0;
        // ---- the row's halo box ----
        bool ok = true;
        if (use_tma) {
            if (lane == 0) {
                fence_async_shared();                 // the box's previous reads come first
                mbar_arrive_expect_tx(&bar[w], B::ELEMS * (uint32_t)sizeof(float));
                if (N == 3) tma_load_3d(bx, &rmap, b0x, b0y, b0z, &bar[w]);
                else tma_load_2d(bx, &rmap, b0x, b0y, &bar[w]);
            }
            ok = mbar_wait_bounded(&bar[w], phase & 1u);
            ++phase;
        } else {
            for (int e = lane; e < B::ELEMS; e += 32) {
                const int ex_ = e % B::BX, ey_ = (e / B::BX) % B::BY, ez_ = e / (B::BX * B::BY);
                const int gx = b0x + ex_, gy = b0y + ey_, gz = b0z + ez_;
                const bool in = (unsigned)gx < (unsigned)P.nx && (unsigned)gy < (unsigned)P.ny &&
                                (N == 2 || (unsigned)gz < (unsigned)P.nz);
                bx[e] = in ? __ldg(P.ev + ((long long)gz * P.ny + gy) * P.nx + gx) : 0.f;
            }
            __syncwarp();
        }
        if (!__all_sync(kFull, ok)) {
            if (lane == 0) {
                atomicOr(&P.ctr->flags, kFlagTimeout);
                mbar_wait_bounded(&bar[w], (phase - 1) & 1u);     // its copy lands before the warp leaves
            }
            break;
        }
        // ---- the row's queued voxels, G lanes each ----
        const int nq = __popc(mask);
        int G = 32;
        while (G > 2 && nq * G > 32) G >>= 1;
        const int slots = 32 / G;
        const int gl = lane & (G - 1);
        const int gbase = lane & ~(G - 1);
        const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << gbase);
        for (int k = lane / G; k < nq; k += slots) {           // group-uniform
            unsigned mk = mask;                                // the k-th queued voxel of the row
            for (int j = 0; j < k; ++j) mk &= mk - 1u;         // (k < popc(mask): mk stays non-zero)
            const int xi = __ffs(mk) - 1;
            const int x = x0 + xi;
            const unsigned v = (unsigned)(((long long)z * P.ny + y) * P.nx + x);
            const float dr = __ldg(P.ref + v);
            const float dD = P.dd_frac * (P.local ? dr : dnorm);
            const float inv = 1.0f / dD;
            float best = P.out[v];                             // gamma^2 over the faces through v
            int t = 0;
            while (t < P.ntable) {
                const int idx = t + gl;
                float key = kInf;
                uint32_t off = 0;
                if (idx < P.ntable) {
                    const TableEntry e = idx < kWalkTableCache ? sh_table[idx] : P.table[idx];
                    key = e.key;
                    off = e.off;
                }
                const float k0 = __shfl_sync(gmask, key, gbase);
                if (k0 * k0 >= best) break;                     // A1 step 4b-ii, exact
                float cb = best;
                if (key * key < best) {
                    if (P.stats) ++st.keyed;
                    cb = visit_cell_box<N, B>(P, bx, b0x, b0y, b0z, x, y, z, unpack10(off, 0),
                                              unpack10(off, 10), unpack10(off, 20), key, dr, inv,
                                              dnorm, best, st);
                }
                best = group_min_rt(cb, G, gmask);
                t += G;
            }
            if (t >= P.ntable && best > rc2) {
                // past a truncated table: the exact scan of the remaining box
                if (gl == 0) ++my_over;
                const float g = sqrtf(best);
                const int ax = (int)ceilf(g / P.hn[0]) + 1;
                const int ay = (int)ceilf(g / P.hn[1]) + 1;
                const int az = N == 3 ? (int)ceilf(g / P.hn[2]) + 1 : 0;
                const int xa = max(-ax - 1, -x), xb = min(ax, P.nx - 1 - x);
                const int ya = max(-ay - 1, -y), yb = min(ay, P.ny - 1 - y);
                const int za = N == 3 ? max(-az - 1, -z) : 0, zb = N == 3 ? min(az, P.nz - 1 - z) : 0;
                const long long wx = xb - xa + 1, wy = yb - ya + 1, wz = zb - za + 1;
                const long long tot = wx * wy * wz;
                const float lim = rc2 * 0.99999f;
                float lb = best;
                for (long long b = gl; b < tot; b += G) {
                    const int cx = xa + (int)(b % wx);
                    const long long rr = b / wx;
                    const int cy = ya + (int)(rr % wy);
                    const int cz = za + (int)(rr / wy);
                    const float axd = (float)max(max(cx, -cx - 1), 0) * P.hn[0];
                    const float ayd = (float)max(max(cy, -cy - 1), 0) * P.hn[1];
                    const float azd = N == 3 ? (float)max(max(cz, -cz - 1), 0) * P.hn[2] : 0.f;
                    float k2 = axd * axd + ayd * ayd + azd * azd;
                    if (k2 == 0.f)
                        k2 = P.key0_far2[(cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2)];
                    if (k2 < lim || k2 >= lb) continue;
                    lb = visit_cell_box<N, B>(P, bx, b0x, b0y, b0z, x, y, z, cx, cy, cz, sqrtf(k2), dr,
                                              inv, dnorm, lb, st);
                }
                best = group_min_rt(lb, G, gmask);
            }
            if (gl == 0) {
                const float gam = sqrtf(best);
                P.out[v] = gam;
                ++my_eval;
                my_pass += gam <= 1.f;
            }
        }
        __syncwarp();                                          // the box is free again
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_eval += __shfl_xor_sync(kFull, my_eval, o);
        my_pass += __shfl_xor_sync(kFull, my_pass, o);
        my_over += __shfl_xor_sync(kFull, my_over, o);
        if (P.stats) {
            st.visited += __shfl_xor_sync(kFull, st.visited, o);
            st.pruned += __shfl_xor_sync(kFull, st.pruned, o);
            st.keyed += __shfl_xor_sync(kFull, st.keyed, o);
        }
    }
    if (lane == 0) {
        if (my_eval) atomicAdd(&P.ctr->n_eval, (unsigned long long)my_eval);
        if (my_pass) atomicAdd(&P.ctr->n_pass, (unsigned long long)my_pass);
        if (my_over) atomicAdd(&P.ctr->overflow_count, my_over);
        if (P.stats) {
            atomicAdd(&P.ctr->cells_visited, st.visited);
            atomicAdd(&P.ctr->cells_pruned, st.pruned);
            atomicAdd(&P.ctr->cells_keyed, st.keyed);
        }
    }
}

// --------------------------------------------------------------------------
// Launchers
// --------------------------------------------------------------------------

int device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

static int grid_for(long long n, int threads, int cap)
{
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

cudaError_t launch_prepare(const Problem& P, cudaStream_t s, int part)
{
    const int sms = device_sm_count();
    k_prepare<false><<<grid_for((P.nvox + 3) / 4, 256, sms * 8), 256, 0, s>>>(P, nullptr, part);
    return cudaGetLastError();
}

// Distance from the origin to the closed simplex with vertices W[0..nv-1] in
// R^3 (KKT enumeration over its faces), for the host-side shell constants.
static double simplex_dist_host(const double (*W)[3], int nv)
{
    double best = INFINITY;
    for (int mask = 1; mask < (1 << nv); ++mask) {
        int idx[4], k = 0;
        for (int i = 0; i < nv; ++i)
            if (mask & (1 << i)) idx[k++] = i;
        const double* w0 = W[idx[0]];
        double E[3][3], G[3][3], r[3], mu[3] = {0, 0, 0};
        const int m = k - 1;
        for (int i = 0; i < m; ++i)
            for (int a = 0; a < 3; ++a) E[i][a] = W[idx[i + 1]][a] - w0[a];
        for (int i = 0; i < m; ++i) {
            r[i] = 0;
            for (int a = 0; a < 3; ++a) r[i] -= E[i][a] * w0[a];
            for (int j = 0; j < m; ++j) {
                G[i][j] = 0;
                for (int a = 0; a < 3; ++a) G[i][j] += E[i][a] * E[j][a];
            }
        }
        // Gaussian elimination (G is symmetric positive definite here)
        bool okk = true;
        for (int c = 0; c < m && okk; ++c) {
            if (!(fabs(G[c][c]) > 1e-300)) { okk = false; break; }
            for (int rr = c + 1; rr < m; ++rr) {
                const double f = G[rr][c] / G[c][c];
                for (int j = c; j < m; ++j) G[rr][j] -= f * G[c][j];
                r[rr] -= f * r[c];
            }
        }
        if (!okk) continue;
        for (int c = m - 1; c >= 0; --c) {
            double acc = r[c];
            for (int j = c + 1; j < m; ++j) acc -= G[c][j] * mu[j];
            mu[c] = acc / G[c][c];
        }
        double sum = 0;
        bool valid = true;
        for (int i = 0; i < m; ++i) {
            sum += mu[i];
            if (mu[i] < -1e-12) valid = false;
        }
        if (sum > 1 + 1e-12) valid = false;
        if (!valid) continue;
        double d2 = 0;
        for (int a = 0; a < 3; ++a) {
            double p = w0[a];
            for (int i = 0; i < m; ++i) p += mu[i] * E[i][a];
            d2 += p * p;
        }
        best = fmin(best, sqrt(d2));
    }
    return best;
}

void key0_far(const double hn_in[3], int nd, double far[8])
{
    const double hn[3] = {hn_in[0], hn_in[1], nd == 3 ? hn_in[2] : 0.0};
    const int full = (1 << nd) - 1;
    for (int s = 0; s < 8; ++s) far[s] = INFINITY;
    for (int s = 1; s <= full; ++s) {
        const int c[3] = {-(s & 1), -((s >> 1) & 1), -((s >> 2) & 1)};
        double f = INFINITY;
        // every owned face is a chain 0 = u0 < u1 < ... < um of axis masks
        for (int u1 = 1; u1 <= full; ++u1)
            for (int u2 = 0; u2 <= full; ++u2)
                for (int u3 = 0; u3 <= full; ++u3) {
                    int chain[4] = {0, u1, u2, u3};
                    int m = 1;
                    if (u2) {
                        if ((u2 & u1) != u1 || u2 == u1) continue;
                        m = 2;
                        if (u3) {
                            if ((u3 & u2) != u2 || u3 == u2) continue;
                            m = 3;
                        }
                    } else if (u3) {
                        continue;
                    }
                    bool has = false;
                    for (int i = 0; i <= m; ++i) has = has || chain[i] == s;
                    if (has) continue;
                    double W[4][3];
                    for (int i = 0; i <= m; ++i)
                        for (int a = 0; a < 3; ++a)
                            W[i][a] = (a < nd) ? (c[a] + ((chain[i] >> a) & 1)) * hn[a] : 0.0;
                    f = fmin(f, simplex_dist_host(W, m + 1));
                }
        double W[1][3];                       // the cell's own corner vertex
        for (int a = 0; a < 3; ++a) W[0][a] = (a < nd) ? c[a] * hn[a] : 0.0;
        f = fmin(f, simplex_dist_host(W, 1));
        far[s] = f * (1.0 - 1e-6);            // absorbs the rounding of the projection
    }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder (looked up once), or null.
static EncodeFn tensor_map_encoder()
{
    static EncodeFn encode = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = (EncodeFn)fn;
    }
    return encode;
}

bool encode_bf16_2d(CUtensorMap* map, const void* base, unsigned long long inner,
                    unsigned long long rows, unsigned long long row_stride_bytes,
                    unsigned box_inner, unsigned box_rows)
{
    const EncodeFn encode = tensor_map_encoder();
    if (!encode || ((uintptr_t)base & 15u) || (row_stride_bytes & 15u) || (box_inner * 2) % 16) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)row_stride_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    std::memset(map, 0, sizeof(*map));
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                  es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of the evaluation dose with a tile box of (bx, by, bz) floats;
// false when TMA cannot be used for it.
static bool encode_box_map(const Problem& P, CUtensorMap* map, int bx, int by, int bz)
{
    const EncodeFn encode = tensor_map_encoder();
    if (!encode) return false;
    if (((uintptr_t)P.ev & 15u) != 0 || (P.nx % 4) != 0) return false;   // TMA alignment rules
    if (P.ndim == 3) {
        const cuuint64_t dims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)P.nz};
        const cuuint64_t strides[2] = {(cuuint64_t)P.nx * 4, (cuuint64_t)P.nx * P.ny * 4};
        const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
        const cuuint32_t es[3] = {1, 1, 1};
        return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)P.ev, dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny};
    const cuuint64_t strides[1] = {(cuuint64_t)P.nx * 4};
    const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    const cuuint32_t es[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)P.ev, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// The shell of a run uses k_shell_w (warp tiles) unless a staged walk needs
// k_shell's tile layout for its queue.
static bool warp_tiled(const Problem& P) { return !P.tile_mask && !P.row_items; }

bool encode_tile_map(const Problem& P, CUtensorMap* map)
{
    if (warp_tiled(P))
        return P.ndim == 3 ? encode_box_map(P, map, WarpTile<3>::BX, WarpTile<3>::BY, WarpTile<3>::BZ)
                           : encode_box_map(P, map, WarpTile<2>::BX, WarpTile<2>::BY, 1);
    return P.ndim == 3 ? encode_box_map(P, map, ShellTile<3>::BX, ShellTile<3>::BY, ShellTile<3>::BZ)
                       : encode_box_map(P, map, ShellTile<2>::BX, ShellTile<2>::BY, 1);
}

template <class T>
static long long tile_count(const Problem& P)
{
    const long long nxy = (long long)((P.nx + T::TX - 1) / T::TX) * ((P.ny + T::TY - 1) / T::TY);
    return P.ndim == 3 ? nxy * ((P.nz + T::TZ - 1) / T::TZ) : nxy;
}

int block_tiles(const Problem& P)
{
    const long long tiles = P.ndim == 3 ? tile_count<ShellTile<3>>(P) : tile_count<ShellTile<2>>(P);
    return tiles > 0x3fffffffLL ? -1 : (int)tiles;
}

int shell_tiles(const Problem& P)
{
    if (!warp_tiled(P)) return block_tiles(P);
    const long long tiles = P.ndim == 3 ? tile_count<WarpTile<3>>(P) : tile_count<WarpTile<2>>(P);
    return tiles > 0x3fffffffLL ? -1 : (int)tiles;
}

// k_shell with its register budget chosen for `per_sm` resident blocks.
template <int N, bool BATCH>
static void launch_shell_k(int per_sm, unsigned grid, cudaStream_t s, const Problem& P,
                           const CUtensorMap& map, int use_tma, int t_first, int tiles,
                           unsigned* next, const SlabGate& gate, const BatchDesc* bd)
{
    switch (per_sm) {
    case 1: k_shell<N, 1, BATCH><<<grid, 256, 0, s>>>(P, map, use_tma, t_first, tiles, next, gate, bd); break;
    case 2: k_shell<N, 2, BATCH><<<grid, 256, 0, s>>>(P, map, use_tma, t_first, tiles, next, gate, bd); break;
    case 3: k_shell<N, 3, BATCH><<<grid, 256, 0, s>>>(P, map, use_tma, t_first, tiles, next, gate, bd); break;
    default: k_shell<N, 4, BATCH><<<grid, 256, 0, s>>>(P, map, use_tma, t_first, tiles, next, gate, bd); break;
    }
}

bool shell_gate_ok(const Problem& P)
{
    CUtensorMap map;
    return encode_tile_map(P, &map);
}

template <class T>
static void layers_of(const Problem& P, int* tiles_per_layer, int* layers, int* layer_depth)
{
    *tiles_per_layer = ((P.nx + T::TX - 1) / T::TX) * ((P.ny + T::TY - 1) / T::TY);
    *layers = P.ndim == 3 ? (P.nz + T::TZ - 1) / T::TZ : 1;
    *layer_depth = P.ndim == 3 ? T::TZ : 1;
}

void shell_layers(const Problem& P, int* tiles_per_layer, int* layers, int* layer_depth)
{
    if (warp_tiled(P)) {
        if (P.ndim == 3) layers_of<WarpTile<3>>(P, tiles_per_layer, layers, layer_depth);
        else layers_of<WarpTile<2>>(P, tiles_per_layer, layers, layer_depth);
    } else {
        if (P.ndim == 3) layers_of<ShellTile<3>>(P, tiles_per_layer, layers, layer_depth);
        else layers_of<ShellTile<2>>(P, tiles_per_layer, layers, layer_depth);
    }
}

template <int N, bool BATCH>
static void launch_shell_w_k(int per_sm, unsigned grid, cudaStream_t s, const Problem& P,
                             const CUtensorMap& map, int use_tma, int t_first, int tiles,
                             unsigned* next, const SlabGate& gate, const BatchDesc* bd)
{
    switch (per_sm) {
    case 1: k_shell_w<N, 1, BATCH><<<grid, 256, 0, s>>>(P, map, use_tma, t_first, tiles, next, gate, bd); break;
    case 2: k_shell_w<N, 2, BATCH><<<grid, 256, 0, s>>>(P, map, use_tma, t_first, tiles, next, gate, bd); break;
    case 3: k_shell_w<N, 3, BATCH><<<grid, 256, 0, s>>>(P, map, use_tma, t_first, tiles, next, gate, bd); break;
    default: k_shell_w<N, 4, BATCH><<<grid, 256, 0, s>>>(P, map, use_tma, t_first, tiles, next, gate, bd); break;
    }
}

cudaError_t launch_shell_range(const Problem& P, int tile_first, int tile_end, int slot,
                               const SlabGate& gate, cudaStream_t s)
{
    if (slot < 0 || slot >= kShellSlots) return cudaErrorInvalidValue;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    const int use_tma = encode_tile_map(P, &map) ? 1 : 0;
    if (gate.flag && (!use_tma || gate.depth <= 0)) return cudaErrorInvalidValue;
    const int sms = device_sm_count();
    const int per_sm = std::min(4, std::max(1, P.shell_minblocks));
    const int tiles = shell_tiles(P);
    if (tiles < 0 || tile_first < 0 || tile_end > tiles || tile_first > tile_end)
        return cudaErrorInvalidValue;
    if (tile_first == tile_end) return cudaSuccess;
    unsigned* next = &P.ctr->shell_next[slot];
    if (warp_tiled(P)) {
        // eight tiles per block in flight
        const unsigned grid = (unsigned)std::min<long long>((tile_end - tile_first + 7) / 8,
                                                            (long long)sms * per_sm);
        if (P.ndim == 3)
            launch_shell_w_k<3, false>(per_sm, grid, s, P, map, use_tma, tile_first, tile_end, next, gate,
                                       nullptr);
        else
            launch_shell_w_k<2, false>(per_sm, grid, s, P, map, use_tma, tile_first, tile_end, next, gate,
                                       nullptr);
        return cudaGetLastError();
    }
    const unsigned grid =
        (unsigned)std::min<long long>(tile_end - tile_first, (long long)sms * per_sm);
    if (P.ndim == 3)
        launch_shell_k<3, false>(per_sm, grid, s, P, map, use_tma, tile_first, tile_end, next, gate,
                                 nullptr);
    else
        launch_shell_k<2, false>(per_sm, grid, s, P, map, use_tma, tile_first, tile_end, next, gate,
                                 nullptr);
    return cudaGetLastError();
}

cudaError_t launch_shell(const Problem& P, cudaStream_t s)
{
    const int tiles = shell_tiles(P);
    if (tiles < 0) return cudaErrorInvalidValue;
    return launch_shell_range(P, 0, tiles, 0, SlabGate{nullptr, 0u, 0}, s);
}

// Copy the final gamma of every queued voxel from the device map into a
// host map (through its device-mapped pointer) that already holds the rest.
// Block 0 also copies the run's final counters into `host_ctr` (mapped), so
// that reading them needs no copy of its own.
__global__ void __launch_bounds__(256) k_patch_host(const __grid_constant__ Problem P, float* host_out,
                                                    Counters* host_ctr)
{
    if (blockIdx.x == 0 && host_ctr) {
        const unsigned* src = (const unsigned*)P.ctr;
        unsigned* dst = (unsigned*)host_ctr;
        for (unsigned i = threadIdx.x; i < sizeof(Counters) / 4; i += blockDim.x) dst[i] = src[i];
    }
    const unsigned n = min(P.ctr->tail_count, P.tail_cap);
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned v = P.tail_raw[i];
        host_out[v] = P.out[v];
    }
}

cudaError_t launch_patch_host(const Problem& P, float* host_out_mapped, Counters* host_ctr_mapped,
                              cudaStream_t s)
{
    k_patch_host<<<device_sm_count() * 4, 256, 0, s>>>(P, host_out_mapped, host_ctr_mapped);
    return cudaGetLastError();
}

cudaError_t launch_order_tail(const Problem& P, cudaStream_t s)
{
    if (!P.sort_tail) return cudaSuccess;
    const int sms = device_sm_count();
    k_scatter<<<sms * 8, 256, 0, s>>>(P);
    return cudaGetLastError();
}

template <int N, int MINB, bool BATCH>
static void launch_tail_g(const Problem& P, const BatchDesc* bd, int G, int grid, cudaStream_t s)
{
    switch (G) {
    case 2: k_tail<N, 2, MINB, BATCH><<<grid, 256, 0, s>>>(P, bd); break;
    case 4: k_tail<N, 4, MINB, BATCH><<<grid, 256, 0, s>>>(P, bd); break;
    case 8: k_tail<N, 8, MINB, BATCH><<<grid, 256, 0, s>>>(P, bd); break;
    case 16: k_tail<N, 16, MINB, BATCH><<<grid, 256, 0, s>>>(P, bd); break;
    default: k_tail<N, 32, MINB, BATCH><<<grid, 256, 0, s>>>(P, bd); break;
    }
}

// k_tail with G lanes per queued voxel and its register budget sized for
// `per_sm` resident blocks (1 to 3; 3 spills a little and is still the
// fastest on the benchmark workload).
template <int N, bool BATCH>
static void launch_tail_n(const Problem& P, const BatchDesc* bd, int G, int per_sm, int grid,
                          cudaStream_t s)
{
    if (per_sm >= 3) launch_tail_g<N, 3, BATCH>(P, bd, G, grid, s);
    else if (per_sm == 2) launch_tail_g<N, 2, BATCH>(P, bd, G, grid, s);
    else launch_tail_g<N, 1, BATCH>(P, bd, G, grid, s);
}

cudaError_t launch_tail(const Problem& P, int lanes_per_voxel, int tail_minblocks, cudaStream_t s)
{
    const int sms = device_sm_count();
    const int grid = sms * 8;      // persistent: enough warps to fill every SM
    if (P.ndim == 3) launch_tail_n<3, false>(P, nullptr, lanes_per_voxel, tail_minblocks, grid, s);
    else launch_tail_n<2, false>(P, nullptr, lanes_per_voxel, tail_minblocks, grid, s);
    return cudaGetLastError();
}

template <int N, bool BATCH>
static void launch_tail_cq_n(const Problem& P, const BatchDesc* bd, int per_sm, cudaStream_t s)
{
    const int grid = device_sm_count() * per_sm;      // persistent: one wave of resident blocks
    if (per_sm >= 4) k_tail_cq<N, 4, BATCH><<<grid, 256, 0, s>>>(P, bd);
    else if (per_sm == 3) k_tail_cq<N, 3, BATCH><<<grid, 256, 0, s>>>(P, bd);
    else if (per_sm == 2) k_tail_cq<N, 2, BATCH><<<grid, 256, 0, s>>>(P, bd);
    else k_tail_cq<N, 1, BATCH><<<grid, 256, 0, s>>>(P, bd);
    k_tail_fix<N, BATCH><<<device_sm_count() * 2, 256, 0, s>>>(P, bd);
}

cudaError_t launch_tail_cq(const Problem& P, int tail_minblocks, cudaStream_t s)
{
    if (!P.fix_list) return cudaErrorInvalidValue;
    const int per_sm = std::min(4, std::max(1, tail_minblocks));
    if (P.ndim == 3) launch_tail_cq_n<3, false>(P, nullptr, per_sm, s);
    else launch_tail_cq_n<2, false>(P, nullptr, per_sm, s);
    return cudaGetLastError();
}

cudaError_t launch_order_tiles(const Problem& P, cudaStream_t s)
{
    if (!P.sort_tail) return cudaSuccess;
    k_scatter_tiles<<<device_sm_count() * 2, 256, 0, s>>>(P);
    return cudaGetLastError();
}

template <int N>
static void launch_walk_n(const Problem& P, const CUtensorMap& map, int use_tma, int per_sm,
                          int grid, cudaStream_t s)
{
    if (per_sm >= 3) k_walk<N, 3><<<grid, 256, 0, s>>>(P, map, use_tma);
    else if (per_sm == 2) k_walk<N, 2><<<grid, 256, 0, s>>>(P, map, use_tma);
    else k_walk<N, 1><<<grid, 256, 0, s>>>(P, map, use_tma);
}

cudaError_t launch_walk(const Problem& P, int walk_minblocks, cudaStream_t s)
{
    if (!P.tile_mask) return cudaErrorInvalidValue;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    int use_tma;
    if (P.ndim == 3) use_tma = encode_box_map(P, &map, WalkBox<3>::BX, WalkBox<3>::BY, WalkBox<3>::BZ);
    else use_tma = encode_box_map(P, &map, WalkBox<2>::BX, WalkBox<2>::BY, 1);
    const int per_sm = std::min(3, std::max(1, walk_minblocks));
    const int grid = device_sm_count() * per_sm;     // persistent; blocks past the tile list exit
    if (P.ndim == 3) launch_walk_n<3>(P, map, use_tma, per_sm, grid, s);
    else launch_walk_n<2>(P, map, use_tma, per_sm, grid, s);
    return cudaGetLastError();
}

cudaError_t launch_order_rows(const Problem& P, cudaStream_t s)
{
    if (!P.sort_tail) return cudaSuccess;
    k_scatter_rows<<<device_sm_count() * 2, 256, 0, s>>>(P);
    return cudaGetLastError();
}

template <int N, int MINB>
static cudaError_t launch_walk_rows_k(const Problem& P, const CUtensorMap& map, int use_tma, int grid,
                                      cudaStream_t s)
{
    const int smem = 8 * RowBox<N>::STRIDE * (int)sizeof(float) + 128;
    cudaError_t e = cudaFuncSetAttribute(k_walk_rows<N, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_walk_rows<N, MINB><<<grid, 256, smem, s>>>(P, map, use_tma);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_walk_rows_n(const Problem& P, const CUtensorMap& map, int use_tma, int per_sm,
                                      int grid, cudaStream_t s)
{
    if (per_sm >= 3) return launch_walk_rows_k<N, 3>(P, map, use_tma, grid, s);
    if (per_sm == 2) return launch_walk_rows_k<N, 2>(P, map, use_tma, grid, s);
    return launch_walk_rows_k<N, 1>(P, map, use_tma, grid, s);
}

cudaError_t launch_walk_rows(const Problem& P, int walk_minblocks, cudaStream_t s)
{
    if (!P.row_items) return cudaErrorInvalidValue;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    int use_tma;
    if (P.ndim == 3) use_tma = encode_box_map(P, &map, RowBox<3>::BX, RowBox<3>::BY, RowBox<3>::BZ);
    else use_tma = encode_box_map(P, &map, RowBox<2>::BX, RowBox<2>::BY, 1);
    const int per_sm = std::min(3, std::max(1, walk_minblocks));
    const int grid = device_sm_count() * per_sm;     // persistent
    return P.ndim == 3 ? launch_walk_rows_n<3>(P, map, use_tma, per_sm, grid, s)
                       : launch_walk_rows_n<2>(P, map, use_tma, per_sm, grid, s);
}

// --------------------------------------------------------------------------
// Batched launches (one group = pairs of one dimension)
// --------------------------------------------------------------------------

cudaError_t launch_batch_prepare(const BatchGroup& g, cudaStream_t s)
{
    if (g.npairs <= 0) return cudaSuccess;
    const int sms = device_sm_count();
    const int bx = grid_for(g.max_nvox, 256, std::max(1, sms * 8 / std::max(1, g.npairs)) + 1);
    Problem dummy{};
    k_prepare<true><<<dim3(bx, g.npairs), 256, 0, s>>>(dummy, g.desc, 1);   // k_shell checks the evaluation dose
    return cudaGetLastError();
}

cudaError_t launch_batch_shell(const BatchGroup& g, int shell_minblocks, cudaStream_t s)
{
    if (g.npairs <= 0 || g.total_tiles <= 0) return cudaSuccess;
    const int sms = device_sm_count();
    const int per_sm = std::min(4, std::max(1, shell_minblocks));
    const unsigned grid = (unsigned)std::min<long long>((g.total_tiles + 7) / 8, (long long)sms * per_sm);
    Problem dummy{};
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if (g.ndim == 3) launch_shell_w_k<3, true>(per_sm, grid, s, dummy, map, 0, 0, g.total_tiles, g.shell_next,
                                          SlabGate{nullptr, 0u, 0}, g.desc);
    else launch_shell_w_k<2, true>(per_sm, grid, s, dummy, map, 0, 0, g.total_tiles, g.shell_next,
                                          SlabGate{nullptr, 0u, 0}, g.desc);
    return cudaGetLastError();
}

cudaError_t launch_batch_order(const BatchGroup& g, cudaStream_t s)
{
    if (g.npairs <= 0) return cudaSuccess;
    k_bucket_scan_batch<<<1, 256, 0, s>>>(g.desc);
    // enough blocks per pair for the largest queue (one 256-voxel chunk per
    // block and pass); the blocks of small pairs leave at once
    const int sms = device_sm_count();
    k_scatter_batch<<<dim3(sms * 4, g.npairs), 256, 0, s>>>(g.desc);
    return cudaGetLastError();
}

cudaError_t launch_batch_tail(const BatchGroup& g, int walk, int lanes_per_voxel, int tail_minblocks,
                              cudaStream_t s)
{
    if (g.npairs <= 0) return cudaSuccess;
    const int sms = device_sm_count();
    Problem dummy{};
    if (walk == 3) {
        const int per_sm = std::min(4, std::max(1, tail_minblocks));
        if (g.ndim == 3) launch_tail_cq_n<3, true>(dummy, g.desc, per_sm, s);
        else launch_tail_cq_n<2, true>(dummy, g.desc, per_sm, s);
        return cudaGetLastError();
    }
    if (g.ndim == 3) launch_tail_n<3, true>(dummy, g.desc, lanes_per_voxel, tail_minblocks, sms * 8, s);
    else launch_tail_n<2, true>(dummy, g.desc, lanes_per_voxel, tail_minblocks, sms * 8, s);
    return cudaGetLastError();
}

}  // namespace gk
