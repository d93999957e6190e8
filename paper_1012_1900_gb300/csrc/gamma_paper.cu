// The paper's own GPU design (Algorithm A2), kept as a measured ablation of
// this library's two-phase search:
//   k_paper_dd    Kernel 1: DD = |D_e - D_r| / dD per reference voxel and the
//                 low-dose cutoff (A2 steps 2-3); evaluated voxels get their
//                 DD as sort key, the others the largest key
//   (sort)        the {DD, voxel} pairs sorted by DD, as the paper's Thrust
//                 sort (a library radix sort; skipped in the unsorted variant)
//   k_paper_walk  Kernel 3: one thread per voxel in that order walks the
//                 radially sorted cell table with the break of A1 step 4b-ii
//                 and evaluates every simplex of every cell it reaches, either
//                 all faces in closed form (Section 2.2, the paper's choice)
//                 or the full simplices with Ju's recursion (Section 2.1)
// The results equal those of the two-phase search (both are exact).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include <cub/device/device_radix_sort.cuh>

#include "gamma_cell.cuh"
#include "gamma_internal.h"

namespace gk {

// --------------------------------------------------------------------------
// Kernel 1: DD keys
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_paper_dd(const __grid_constant__ Problem P,
                                                  unsigned* __restrict__ keys,
                                                  unsigned* __restrict__ ids)
{
    const float dnorm = resolve_dnorm(P);
    const float thr = cutoff_threshold(P.local, P.cutoff_frac, dnorm);
    float my_rmax = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < P.nvox; v += stride) {
        const float dr = __ldg(P.ref + v);
        unsigned key = 0xffffffffu;
        if (is_evaluated(P, dr, thr)) {
            const float dD = P.dd_frac * (P.local ? dr : dnorm);
            const float g0 = fabsf(__ldg(P.ev + v) - dr) / dD;
            my_rmax = fmaxf(my_rmax, g0);
            key = __float_as_uint(g0);             // order-preserving for g0 >= 0
        } else {
            P.out[v] = __int_as_float(0x7fc00000);
        }
        keys[v] = key;
        ids[v] = (unsigned)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_rmax = fmaxf(my_rmax, __shfl_xor_sync(kFull, my_rmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&P.ctr->rmax_enc, fenc(my_rmax));
}

// --------------------------------------------------------------------------
// Ju's recursion on a closed simplex (FP32)
// --------------------------------------------------------------------------

// Squared distance from the reference point to the closed full simplex of
// the cell (lower corner c, voxel units from the voxel) whose vertices are
// the chain masks ch[0] = 0 < ch[1] < ... < ch[N] (q: their relative doses
// by mask), by Ju's recursion (Section 2.1): project onto the affine hull;
// if a barycentric weight is negative, search the facets opposite those
// vertices instead.  Every sub-simplex of a chain is a chain, whose
// increments are axis-disjoint, so each projection takes the closed form of
// the normal equations (Gram matrix diag(sigma^2) + d d^T) from its own
// lowest vertex.  Vertex subsets are bit masks over chain positions, each
// solved at most once, larger masks first (a facet's mask is smaller).
// `ill` is raised when a Gram matrix may be near singular (see face_core).
template <int N, typename T>
__device__ T ju_chain_d2(const T (&q)[8], const int (&ch)[4], const int (&c)[3],
                         const MetricT<T>& mt, T dmax, bool& ill)
{
    T best = T(kInf);
    uint32_t pending = 1u << ((1u << (N + 1)) - 1u);
    uint32_t visited = 0;
    while (pending) {
        const int m = 31 - __clz(pending);
        pending &= ~(1u << m);
        if ((visited >> m) & 1u) continue;
        visited |= 1u << m;
        int pos[4] = {0, 0, 0, 0};
        int k = 0;
#pragma unroll
        for (int i = 0; i <= N; ++i)
            if ((m >> i) & 1) pos[k++] = i;
        const int u0 = ch[pos[0]];
        // spatial position of the lowest vertex (voxel units) and |s0|^2
        T s0[3], s02 = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s0[a] = a < N ? T(c[a] + ((u0 >> a) & 1)) : T(0);
            s02 = fma_(mt.hn2[a] * s0[a], s0[a], s02);
        }
        if (k == 1) {
            best = min_(best, fma_(q[u0], q[u0], s02));
            continue;
        }
        // rho^2 (squared spatial distance to the face's spatial hull) as a sum
        // of non-negative terms: the axes no increment spans, plus Lagrange's
        // identity within each multi-axis increment
        T D = T(1), L = q[u0], rho2 = T(0);
        T dk[3] = {T(0), T(0), T(0)}, beta[3] = {T(0), T(0), T(0)};
        int covered = 0;
        for (int i = 1; i < k; ++i) {
            const int A = ch[pos[i]] ^ ch[pos[i - 1]];
            covered |= A;
            const T kap = mt.kappa[A];
            const T d = q[ch[pos[i]]] - q[ch[pos[i - 1]]];
            T sa = T(0);                             // s0 . e_i (spatial), in hn^2 units
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if ((A >> a) & 1) sa = fma_(mt.hn2[a], s0[a], sa);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = a + 1; b < 3; ++b)
                    if (((A >> a) & 1) && ((A >> b) & 1)) {
                        const T ds = s0[a] - s0[b];
                        rho2 = fma_(mt.hn2[a] * mt.hn2[b] * ds * ds, kap, rho2);
                    }
            beta[i - 1] = -sa * kap;
            dk[i - 1] = d * kap;
            D = fma_(d, dk[i - 1], D);
            L = fma_(d, beta[i - 1], L);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (!((covered >> a) & 1)) rho2 = fma_(mt.hn2[a] * s0[a], s0[a], rho2);
        if (k >= 3 && D > dmax) ill = true;
        const T r = L / D;
        // weights of the vertices: 1 - mu_1, mu_1 - mu_2, ..., mu_(k-1)
        T mu_prev = T(1);
        bool inside = true;
        T lam[4];
        for (int i = 1; i < k; ++i) {
            const T mu = fma_(-r, dk[i - 1], beta[i - 1]);
            lam[i - 1] = mu_prev - mu;
            mu_prev = mu;
        }
        lam[k - 1] = mu_prev;
        for (int j = 0; j < k; ++j) inside = inside && lam[j] >= T(0);
        if (inside) {
            best = min_(best, fma_(L, r, rho2));
        } else {
            for (int j = 0; j < k; ++j)
                if (lam[j] < T(0)) pending |= 1u << (m & ~(1 << pos[j]));
        }
    }
    return best;
}

// Every simplex of one cell.  JU: the n! full simplices of a cube inside the
// grid by Ju's recursion (the faces of boundary cubes are faces of interior
// ones); else every face the cell owns in closed form.  Cells whose Gram
// matrices are near singular are redone in FP64.
template <int N, bool JU>
__device__ __forceinline__ float paper_cell(const Problem& P, int x, int y, int z, int cx, int cy,
                                            int cz, float dr, float inv, float dnorm)
{
    const int px = x + cx, py = y + cy, pz = z + cz;
    if ((unsigned)px >= (unsigned)P.nx || (unsigned)py >= (unsigned)P.ny ||
        (N == 3 && (unsigned)pz >= (unsigned)P.nz))
        return kInf;
    const bool ex = px + 1 < P.nx, ey = py + 1 < P.ny, ez = N == 3 && pz + 1 < P.nz;
    const long long sy = P.nx, sz = (long long)P.nx * P.ny;
    const long long p = (long long)pz * sz + (long long)py * sy + px;
    float q[8];
    uint32_t ok = 0;
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
    if constexpr (!JU) {
        return cell_all_faces<N>(P, q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], ok, cx, cy, cz,
                                 p, dr, dnorm);
    } else {
        constexpr int full = (1 << N) - 1;
        if (((ok >> full) & 1u) == 0) return kInf;          // the cube leaves the grid
        constexpr int nperm = N == 3 ? 6 : 2;
        const int perm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        const int c[3] = {cx, cy, cz};
        float best = kInf;
        bool ill = false;
#pragma unroll 1
        for (int s = 0; s < nperm; ++s) {
            int ch[4] = {0, 0, 0, 0};
#pragma unroll
            for (int v = 1; v <= N; ++v)
                ch[v] = ch[v - 1] | (1 << (N == 3 ? perm3[s][v - 1] : (s == 0 ? v - 1 : 2 - v)));
            best = fminf(best, ju_chain_d2<N, float>(q, ch, c, P.mt, ill_dmax(P), ill));
        }
        if (ill && P.tau > 0.f) {
            // the same simplices by the same recursion in FP64 (the closed
            // redo of the owned faces would not cover the same faces)
            const double drd = dr;
            const double invd = 1.0 / ((double)P.dd_frac * (P.local ? drd : (double)dnorm));
            double qd[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                qd[u] = 0.0;
                if (u < (1 << N)) {
                    const long long o = p + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) + ((u & 4) ? sz : 0);
                    qd[u] = ((double)P.ev[o] - drd) * invd;
                }
            }
            double bd = (double)kInf;
            bool ill64 = false;
#pragma unroll 1
            for (int s = 0; s < nperm; ++s) {
                int ch[4] = {0, 0, 0, 0};
#pragma unroll
                for (int v = 1; v <= N; ++v)
                    ch[v] = ch[v - 1] | (1 << (N == 3 ? perm3[s][v - 1] : (s == 0 ? v - 1 : 2 - v)));
                bd = fmin(bd, ju_chain_d2<N, double>(qd, ch, c, P.mtd, (double)kInf, ill64));
            }
            atomicAdd(&P.ctr->fp64_cells, 1u);
            best = (float)bd;
        }
        return best;
    }
}

// --------------------------------------------------------------------------
// Kernel 3: one thread per voxel
// --------------------------------------------------------------------------

template <int N, bool JU, bool SORTED>
__global__ void __launch_bounds__(256) k_paper_walk(const __grid_constant__ Problem P,
                                                    const unsigned* __restrict__ keys,
                                                    const unsigned* __restrict__ ids)
{
    const float dnorm = resolve_dnorm(P);
    const float thr = cutoff_threshold(P.local, P.cutoff_frac, dnorm);
    const float rc2 = P.r_cover * P.r_cover;
    unsigned my_eval = 0, my_pass = 0, my_over = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.nvox; i += stride) {
        unsigned v;
        float dr;
        if constexpr (SORTED) {
            if (keys[i] == 0xffffffffu) continue;           // not evaluated (sorted last)
            v = ids[i];
            dr = __ldg(P.ref + v);
        } else {
            v = (unsigned)i;
            dr = __ldg(P.ref + v);
            if (!is_evaluated(P, dr, thr)) {
                P.out[v] = __int_as_float(0x7fc00000);
                continue;
            }
        }
        const int x = (int)(v % (unsigned)P.nx);
        const unsigned r1 = v / (unsigned)P.nx;
        const int y = (int)(r1 % (unsigned)P.ny), z = (int)(r1 / (unsigned)P.ny);
        const float dD = P.dd_frac * (P.local ? dr : dnorm);
        const float inv = 1.0f / dD;
        const float q0 = (__ldg(P.ev + v) - dr) * inv;
        float best = q0 * q0;                                // A1 step 4a
        // the 2^n cells whose box contains the voxel, then the table (step 4b)
#pragma unroll 1
        for (int s = 0; s < (1 << N); ++s)
            best = fminf(best, paper_cell<N, JU>(P, x, y, z, -(s & 1), -((s >> 1) & 1),
                                                 N == 3 ? -((s >> 2) & 1) : 0, dr, inv, dnorm));
        int t = 0;
        for (; t < P.ntable; ++t) {
            const TableEntry e = P.table[t];
            const int cx = unpack10(e.off, 0), cy = unpack10(e.off, 10), cz = unpack10(e.off, 20);
            if (cx >= -1 && cx <= 0 && cy >= -1 && cy <= 0 && cz >= -1 && cz <= 0) continue;
            if (e.key * e.key >= best) break;                // A1 step 4b-ii, exact
            best = fminf(best, paper_cell<N, JU>(P, x, y, z, cx, cy, cz, dr, inv, dnorm));
        }
        if (t >= P.ntable && best > rc2) {
            // past a truncated table: every remaining cell of the search box
            ++my_over;
            const float g = sqrtf(best);
            const int ax = (int)ceilf(g / P.hn[0]) + 1;
            const int ay = (int)ceilf(g / P.hn[1]) + 1;
            const int az = N == 3 ? (int)ceilf(g / P.hn[2]) + 1 : 0;
            const float lim = rc2 * 0.99999f;
            for (int cz = (N == 3 ? max(-az - 1, -z) : 0); cz <= (N == 3 ? min(az, P.nz - 1 - z) : 0); ++cz)
                for (int cy = max(-ay - 1, -y); cy <= min(ay, P.ny - 1 - y); ++cy)
                    for (int cx = max(-ax - 1, -x); cx <= min(ax, P.nx - 1 - x); ++cx) {
                        const float axd = (float)max(max(cx, -cx - 1), 0) * P.hn[0];
                        const float ayd = (float)max(max(cy, -cy - 1), 0) * P.hn[1];
                        const float azd = N == 3 ? (float)max(max(cz, -cz - 1), 0) * P.hn[2] : 0.f;
                        const float k2 = axd * axd + ayd * ayd + azd * azd;
                        if (k2 == 0.f || k2 < lim || k2 >= best) continue;   // key-0 cells done above
                        best = fminf(best, paper_cell<N, JU>(P, x, y, z, cx, cy, cz, dr, inv, dnorm));
                    }
        }
        const float gam = sqrtf(best);
        P.out[v] = gam;
        ++my_eval;
        my_pass += gam <= 1.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_eval += __shfl_xor_sync(kFull, my_eval, o);
        my_pass += __shfl_xor_sync(kFull, my_pass, o);
        my_over += __shfl_xor_sync(kFull, my_over, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (my_eval) atomicAdd(&P.ctr->n_eval, (unsigned long long)my_eval);
        if (my_pass) atomicAdd(&P.ctr->n_pass, (unsigned long long)my_pass);
        if (my_over) atomicAdd(&P.ctr->overflow_count, my_over);
    }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------

size_t paper_sort_bytes(long long nvox)
{
    size_t bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, bytes, (const unsigned*)nullptr, (unsigned*)nullptr,
                                    (const unsigned*)nullptr, (unsigned*)nullptr, (int)nvox);
    return bytes;
}

template <int N, bool JU>
static void launch_walk(const Problem& P, bool sorted, const unsigned* keys, const unsigned* ids,
                        int grid, cudaStream_t s)
{
    if (sorted) k_paper_walk<N, JU, true><<<grid, 256, 0, s>>>(P, keys, ids);
    else k_paper_walk<N, JU, false><<<grid, 256, 0, s>>>(P, keys, ids);
}

cudaError_t launch_paper(const Problem& P, const PaperScratch& w, bool sorted, bool ju,
                         cudaEvent_t after_sort, cudaStream_t s)
{
    if (P.nvox > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int n = (int)P.nvox;
    const int grid_dd = (int)std::min<long long>((P.nvox + 255) / 256, (long long)device_sm_count() * 32);
    const unsigned* keys = w.keys;
    const unsigned* ids = w.ids;
    if (sorted) {
        k_paper_dd<<<std::max(grid_dd, 1), 256, 0, s>>>(P, w.keys, w.ids);
        size_t bytes = w.temp_bytes;
        cudaError_t e = cub::DeviceRadixSort::SortPairs(w.temp, bytes, w.keys, w.keys_alt, w.ids,
                                                        w.ids_alt, n, 0, 32, s);
        if (e != cudaSuccess) return e;
        keys = w.keys_alt;
        ids = w.ids_alt;
    }
    if (after_sort) cudaEventRecord(after_sort, s);
    const int grid = (int)std::max<long long>(1, (P.nvox + 255) / 256);
    if (P.ndim == 3) {
        if (ju) launch_walk<3, true>(P, sorted, keys, ids, grid, s);
        else launch_walk<3, false>(P, sorted, keys, ids, grid, s);
    } else {
        if (ju) launch_walk<2, true>(P, sorted, keys, ids, grid, s);
        else launch_walk<2, false>(P, sorted, keys, ids, grid, s);
    }
    return cudaGetLastError();
}

}  // namespace gk
