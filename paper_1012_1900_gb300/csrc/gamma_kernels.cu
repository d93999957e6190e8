// CUDA kernels of the gamma search (sm_103a).
//
// One run over a dose pair is five stream-ordered launches:
//   k_prepare   max of the reference dose (the global dose norm) and a
//               finite-input check                       (Algorithm A2 step 2)
//   k_shell     per reference voxel: criteria, low-dose cutoff, gamma0 =
//               DD/dD (A1 step 4a) and every face of the 2^n key-0 cells
//               around the voxel, from its 3^n neighbourhood held in
//               registers; voxels whose running gamma still exceeds the next
//               table key are queued with a cost bucket
//   k_bucket_scan / k_scatter
//               order the queue by estimated cost, most expensive first (the
//               role the paper's DD sort plays, Section 2.2 and Table 2)
//   k_tail      persistent: a group of G lanes takes one queued voxel and
//               walks the sorted cell table G cells at a time, with the exact
//               early exit of A1 step 4b-ii (key >= gamma) and a per-cell
//               lower bound sqrt(key^2 + dose gap^2)
// No kernel waits on another block or allocates memory.
#include <cuda_runtime.h>
#include <math.h>

#include "gamma_internal.h"

namespace gk {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float resolve_dnorm(const Problem& P)
{
    return P.dose_norm > 0.f ? P.dose_norm : fdec(P.ctr->dnorm_enc);
}

__device__ __forceinline__ bool is_evaluated(const Problem& P, float dr, float thr)
{
    return dr >= thr && (!P.local || dr > 0.f);
}

// --------------------------------------------------------------------------
// k_prepare: dose norm and finite check
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_prepare(const __grid_constant__ Problem P)
{
    float m = -kInf;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.nvox; i += stride) {
        const float r = __ldg(P.ref + i), e = __ldg(P.ev + i);
        bad |= !(isfinite(r) && isfinite(e));
        m = fmaxf(m, r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    bad = __any_sync(kFull, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&P.ctr->dnorm_enc, fenc(m));
        if (bad) atomicOr(&P.ctr->flags, kFlagNonFinite);
    }
}

// --------------------------------------------------------------------------
// FP64 redo of one cell whose Gram matrices are near singular
// --------------------------------------------------------------------------

template <int N>
__device__ __noinline__ float cell_redo_f64(const float* __restrict__ ev, long long p, long long sy,
                                            long long sz, uint32_t ok, int cx, int cy, int cz,
                                            double drd, double invd, MetricT<double> mtd,
                                            unsigned int* fp64_counter)
{
    double q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        q[u] = 0.0;
        if (u < (1 << N) && ((ok >> u) & 1u)) {
            const long long o = p + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) + ((u & 4) ? sz : 0);
            q[u] = ((double)ev[o] - drd) * invd;
        }
    }
    CellGeom<double> g;
    cell_geom<N, double>(cx, cy, cz, mtd, g);
    bool ill = false;
    const double b = cell_min_d2<N, double>(q, ok, g, mtd, 0.0, (double)kInf, ill);
    atomicAdd(fp64_counter, 1u);
    return (float)b;
}

// --------------------------------------------------------------------------
// k_shell: gamma0 and the key-0 cells, thread per voxel
// --------------------------------------------------------------------------

template <int N>
__global__ void __launch_bounds__(256) k_shell(const __grid_constant__ Problem P)
{
    constexpr int NB = N == 3 ? 27 : 9;
    __shared__ unsigned int sh_hist[kNumBuckets];
    __shared__ unsigned long long sh_eval, sh_pass;
    __shared__ unsigned int sh_rmax;
    if (threadIdx.x < kNumBuckets) sh_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) { sh_eval = 0; sh_pass = 0; sh_rmax = 0; }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const float dnorm = resolve_dnorm(P);
    const float thr = P.cutoff_frac * dnorm;
    const float k1 = P.t1 < P.ntable ? P.table[P.t1].key : kInf;
    const float k1sq = k1 * k1;
    const float rc2 = P.r_cover * P.r_cover;
    const bool table_ends = P.t1 >= P.ntable;
    const long long sy = P.nx, sz = (long long)P.nx * P.ny;
    unsigned int my_eval = 0, my_pass = 0;
    float my_rmax = 0.f;

    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < P.nvox;
         base += stride) {
        const long long v = base + lane;
        bool tail = false;
        int bucket = 0;
        if (v < P.nvox) {
            const int x = (int)(v % P.nx);
            const long long r1 = v / P.nx;
            const int y = (int)(r1 % P.ny);
            const int z = (int)(r1 / P.ny);
            const float dr = __ldg(P.ref + v);
            if (!is_evaluated(P, dr, thr)) {
                P.out[v] = __int_as_float(0x7fc00000);
            } else {
                const float dD = P.dd_frac * (P.local ? dr : dnorm);
                const float inv = 1.0f / dD;
                float nb[NB];
                uint32_t inb = 0;
#pragma unroll
                for (int dz = (N == 3 ? -1 : 0); dz <= (N == 3 ? 1 : 0); ++dz)
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int k = (N == 3 ? (dz + 1) * 9 : 0) + (dy + 1) * 3 + (dx + 1);
                            const bool in = (unsigned)(x + dx) < (unsigned)P.nx &&
                                            (unsigned)(y + dy) < (unsigned)P.ny &&
                                            (N == 2 || (unsigned)(z + dz) < (unsigned)P.nz);
                            nb[k] = in ? (__ldg(P.ev + v + dx + dy * sy + dz * sz) - dr) * inv : 0.f;
                            inb |= (in ? 1u : 0u) << k;
                        }
                constexpr int C = N == 3 ? 13 : 4;           // the voxel itself
                float best = nb[C] * nb[C];
                my_rmax = fmaxf(my_rmax, fabsf(nb[C]));
                if (best > 0.f) {
#pragma unroll
                    for (int cz = (N == 3 ? -1 : 0); cz <= 0; ++cz)
#pragma unroll
                        for (int cy = -1; cy <= 0; ++cy)
#pragma unroll
                            for (int cx = -1; cx <= 0; ++cx) {
                                float q[8];
                                uint32_t ok = 0;
#pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    q[u] = 0.f;
                                    if (u < (1 << N)) {
                                        const int ux = u & 1, uy = (u >> 1) & 1, uz = (u >> 2) & 1;
                                        const int k = (N == 3 ? (cz + uz + 1) * 9 : 0) +
                                                      (cy + uy + 1) * 3 + (cx + ux + 1);
                                        q[u] = nb[k];
                                        ok |= ((inb >> k) & 1u) << u;
                                    }
                                }
                                if (!(ok & 1u)) continue;
                                CellGeom<float> g;
                                cell_geom<N, float>(cx, cy, cz, P.mt, g);
                                bool ill = false;
                                float cb = cell_min_d2<N, float>(q, ok, g, P.mt, P.tau, kInf, ill);
                                if (ill) {
                                    const double drd = dr;
                                    const double invd =
                                        1.0 / ((double)P.dd_frac * (P.local ? drd : (double)dnorm));
                                    const long long p = v + cx + cy * sy + cz * sz;
                                    cb = cell_redo_f64<N>(P.ev, p, sy, sz, ok, cx, cy, cz, drd, invd,
                                                          P.mtd, &P.ctr->fp64_cells);
                                }
                                best = fminf(best, cb);
                            }
                }
                tail = (best > k1sq) || (table_ends && best > rc2);
                if (tail) {
                    P.out[v] = best;                       // gamma^2, finished by k_tail
                    // estimated cost: table cells past the shell with key < gamma
                    const float gk_ = sqrtf(best);
                    int lo = P.t1, hi = P.ntable;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (P.table[mid].key < gk_) lo = mid + 1; else hi = mid;
                    }
                    const int cost = lo - P.t1;
                    bucket = cost <= 0 ? 0 : min(kNumBuckets - 1, 1 + (int)(2.f * __log2f((float)cost)));
                } else {
                    const float gam = sqrtf(best);
                    P.out[v] = gam;
                    ++my_eval;
                    my_pass += gam <= 1.f;             // decided on the value written
                }
            }
        }
        const unsigned tm = __ballot_sync(kFull, tail);
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
    }
    // block reductions
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_eval += __shfl_xor_sync(kFull, my_eval, o);
        my_pass += __shfl_xor_sync(kFull, my_pass, o);
        my_rmax = fmaxf(my_rmax, __shfl_xor_sync(kFull, my_rmax, o));
    }
    if (lane == 0) {
        atomicAdd(&sh_eval, (unsigned long long)my_eval);
        atomicAdd(&sh_pass, (unsigned long long)my_pass);
        atomicMax(&sh_rmax, fenc(my_rmax));
    }
    __syncthreads();
    if (threadIdx.x < kNumBuckets && sh_hist[threadIdx.x])
        atomicAdd(&P.ctr->hist[threadIdx.x], sh_hist[threadIdx.x]);
    if (threadIdx.x == 0) {
        if (sh_eval) atomicAdd(&P.ctr->n_eval, sh_eval);
        if (sh_pass) atomicAdd(&P.ctr->n_pass, sh_pass);
        atomicMax(&P.ctr->rmax_enc, sh_rmax);
    }
}

// --------------------------------------------------------------------------
// Queue ordering: bucket offsets (most expensive first) and scatter
// --------------------------------------------------------------------------

__global__ void k_bucket_scan(Counters* ctr)
{
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = kNumBuckets - 1; b >= 0; --b) {
            ctr->cursor[b] = acc;
            acc += ctr->hist[b];
        }
    }
}

__global__ void __launch_bounds__(256) k_scatter(const __grid_constant__ Problem P)
{
    const unsigned total = min(P.ctr->tail_count, P.tail_cap);
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const unsigned pos = atomicAdd(&P.ctr->cursor[P.tail_bucket[i]], 1u);
        P.tail_sorted[pos] = P.tail_raw[i];
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
                                            int cz, float key, float dr, float inv, double drd,
                                            double invd, float best, TailStats& st)
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
    CellGeom<float> g;
    cell_geom<N, float>(cx, cy, cz, P.mt, g);
    bool ill = false;
    float cb = cell_min_d2<N, float>(q, ok, g, P.mt, P.tau, kInf, ill);
    if (ill)
        cb = cell_redo_f64<N>(P.ev, p, sy, sz, ok, cx, cy, cz, drd, invd, P.mtd, &P.ctr->fp64_cells);
    return fminf(best, cb);
}

template <int G>
__device__ __forceinline__ float group_min(float v, unsigned gmask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(gmask, v, o));
    return v;
}

template <int N, int G>
__global__ void __launch_bounds__(256) k_tail(const __grid_constant__ Problem P)
{
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << gbase);
    const float dnorm = resolve_dnorm(P);
    const unsigned total = min(P.ctr->tail_count, P.tail_cap);
    const float rc2 = P.r_cover * P.r_cover;
    unsigned int my_eval = 0, my_pass = 0, my_over = 0;
    TailStats st;

    for (;;) {
        unsigned item = 0;
        if (gl == 0) item = atomicAdd(&P.ctr->head, 1u);
        item = __shfl_sync(gmask, item, gbase);
        if (item >= total) break;
        const unsigned v = P.sort_tail ? P.tail_sorted[item] : P.tail_raw[item];
        const int x = (int)(v % (unsigned)P.nx);
        const unsigned r1 = v / (unsigned)P.nx;
        const int y = (int)(r1 % (unsigned)P.ny);
        const int z = (int)(r1 / (unsigned)P.ny);
        const float dr = __ldg(P.ref + v);
        const float dD = P.dd_frac * (P.local ? dr : dnorm);
        const float inv = 1.0f / dD;
        const double drd = dr;
        const double invd = 1.0 / ((double)P.dd_frac * (P.local ? drd : (double)dnorm));
        float best = P.out[v];                       // gamma^2 after the key-0 cells
        int t = P.t1;
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
                                   unpack10(off, 20), key, dr, inv, drd, invd, best, st);
            }
            best = group_min<G>(cb, gmask);
            t += G;
        }
        if (t >= P.ntable && best > rc2) {
            // The walk ran past a truncated table: scan every cell of the
            // remaining search box (rare; keeps the result exact).
            ++my_over;
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
                const float k2 = axd * axd + ayd * ayd + azd * azd;
                if (k2 < lim || k2 >= lb) continue;
                lb = visit_cell<N>(P, x, y, z, cx, cy, cz, sqrtf(k2), dr, inv, drd, invd, lb, st);
            }
            best = group_min<G>(lb, gmask);
        }
        if (gl == 0) {
            const float gam = sqrtf(best);
            P.out[v] = gam;
            ++my_eval;
            my_pass += gam <= 1.f;
        }
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
        if (my_over) atomicAdd(&P.ctr->overflow_count, my_over / G);
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

cudaError_t launch_prepare(const Problem& P, cudaStream_t s)
{
    const int sms = device_sm_count();
    k_prepare<<<grid_for(P.nvox, 256, sms * 8), 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_shell(const Problem& P, cudaStream_t s)
{
    const int sms = device_sm_count();
    const int grid = grid_for(P.nvox, 256, sms * 64);
    if (P.ndim == 3) k_shell<3><<<grid, 256, 0, s>>>(P);
    else k_shell<2><<<grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_order_tail(const Problem& P, cudaStream_t s)
{
    if (!P.sort_tail) return cudaSuccess;
    k_bucket_scan<<<1, 32, 0, s>>>(P.ctr);
    const int sms = device_sm_count();
    k_scatter<<<sms * 2, 256, 0, s>>>(P);
    return cudaGetLastError();
}

template <int N>
static void launch_tail_n(const Problem& P, int G, int grid, cudaStream_t s)
{
    switch (G) {
    case 4: k_tail<N, 4><<<grid, 256, 0, s>>>(P); break;
    case 8: k_tail<N, 8><<<grid, 256, 0, s>>>(P); break;
    case 16: k_tail<N, 16><<<grid, 256, 0, s>>>(P); break;
    default: k_tail<N, 32><<<grid, 256, 0, s>>>(P); break;
    }
}

cudaError_t launch_tail(const Problem& P, int lanes_per_voxel, cudaStream_t s)
{
    const int sms = device_sm_count();
    const int grid = sms * 8;      // persistent: enough warps to fill every SM
    if (P.ndim == 3) launch_tail_n<3>(P, lanes_per_voxel, grid, s);
    else launch_tail_n<2>(P, lanes_per_voxel, grid, s);
    return cudaGetLastError();
}

}  // namespace gk
