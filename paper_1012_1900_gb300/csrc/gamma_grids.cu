// Reference and evaluation doses on different grids (each grid with its own
// shape, spacing and origin; same axes).  Eq. 1 as for coincident grids: the
// evaluation surface is the Freudenthal interpolant of the evaluation grid,
// and each reference voxel searches it from its own position, which is in
// general not an evaluation node.
//
//   k_grid_prepare  max of the reference dose (the global dose norm) and a
//                   finite check of both grids
//   k_grid_walk     a group of lanes per reference voxel (eight by default)
//                   walks the cell table in key order, a cell per lane and
//                   round, from the evaluation cell
//                   that holds the voxel (clamped to the grid), with the exact
//                   stop of A1 step 4b-ii; a cell is skipped when the distance
//                   from the reference point to its box, with its dose gap,
//                   already reaches the running gamma, else every face of it
//                   is evaluated (real-valued cell offsets; FP64 redo when a
//                   Gram matrix is near singular)
//
// The table is keyed by the distance between the box of the voxel's cell and
// the box of the other cell, divided by the DTA: a lower bound on the distance
// from any point of the first box to any face of the second.  It stays a
// lower bound for a voxel outside the evaluation grid, whose clamped cell is
// the grid cell nearest to it: per axis, its distance to any cell is at least
// that cell's gap to the clamped one.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/gamma.h"
#include "gamma_cell.cuh"
#include "gamma_internal.h"

namespace gk {

// Table key of cell offset c along one axis, in cells: the smallest distance
// from a point in its own cell to cell c.  Variant 8 holds for any point of
// the cell (and, per axis, for a point outside the grid, from its clamped
// cell); variants 0-7 for a point in one half of its cell per axis (bit a of
// the variant: the upper half [0.5, 1) of axis a, else the lower [0, 0.5)).
__host__ __device__ inline double grid_axis_key(int c, int variant, int a)
{
    if (variant == 8 || c == 0) return c == 0 ? 0.0 : (double)(c > 0 ? c - 1 : -c - 1);
    const bool upper = (variant >> a) & 1;
    return c > 0 ? (double)(c - 1) + (upper ? 0.0 : 0.5) : (double)(-c - 1) + (upper ? 0.5 : 0.0);
}

// The table variant for a point at fraction fr of its cell (0-7: its half of
// the cell per axis; 8: outside [0, 1) on some axis, beyond the grid).
__device__ __forceinline__ int grid_variant(const float (&fr)[3], int nd)
{
    int v = 0;
    for (int a = 0; a < nd; ++a) {
        if (!(fr[a] >= 0.f && fr[a] < 1.f)) return 8;
        if (fr[a] >= 0.5f) v |= 1 << a;
    }
    return v;
}

// --------------------------------------------------------------------------
// Prepare: dose norm over the reference grid, finite checks
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_grid_prepare(const __grid_constant__ GridProblem G)
{
    float m = -kInf;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = first; i < G.nref; i += stride) {
        const float r = __ldg(G.ref + i);
        bad |= !isfinite(r);
        m = fmaxf(m, r);
    }
    for (long long i = first; i < G.neval; i += stride) bad |= !isfinite(__ldg(G.ev + i));
    __shared__ float sh_m[8];                  // one atomic per block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) sh_m[threadIdx.x >> 5] = m;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh_m[w]);
        atomicMax(&G.ctr->dnorm_enc, fenc(m));
        if (bad) atomicOr(&G.ctr->flags, kFlagNonFinite);
    }
}

// --------------------------------------------------------------------------
// The walk
// --------------------------------------------------------------------------

// Every face of evaluation cell p (its lower corner, grid coordinates) for a
// reference point at u (evaluation voxel units, real), unless the cell's
// key and dose range already keep it at least sqrt(best) away.
template <int N>
__device__ __forceinline__ float grid_cell(const GridProblem& G, const int (&p)[3],
                                           const double (&u)[3], const float (&cf)[3], float key,
                                           float dr, float inv, float dnorm, float best)
{
    const long long sy = G.en[0], sz = (long long)G.en[0] * G.en[1];
    const long long pidx = (long long)p[2] * sz + (long long)p[1] * sy + p[0];
    const bool ex = p[0] + 1 < G.en[0], ey = p[1] + 1 < G.en[1], ez = N == 3 && p[2] + 1 < G.en[2];
    float q[8];
    uint32_t ok = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        q[w] = 0.f;
        if (w < (1 << N)) {
            const bool present = (!(w & 1) || ex) && (!(w & 2) || ey) && (!(w & 4) || ez);
            if (present) {
                const long long o = pidx + ((w & 1) ? 1 : 0) + ((w & 2) ? sy : 0) + ((w & 4) ? sz : 0);
                q[w] = (__ldg(G.ev + o) - dr) * inv;
                ok |= 1u << w;
            }
        }
    }
    float qmin = kInf, qmax = -kInf;
#pragma unroll
    for (int w = 0; w < 8; ++w)
        if ((ok >> w) & 1u) {
            qmin = fminf(qmin, q[w]);
            qmax = fmaxf(qmax, q[w]);
        }
    const float gap = qmin > 0.f ? qmin : (qmax < 0.f ? -qmax : 0.f);
    if (fmaf(gap, gap, key * key) >= best) return best;
    // the cell's corner relative to the point (voxel units), cf = d - fraction
    CellGeom<float> g;
    cell_geom<N, float>(cf[0], cf[1], N == 3 ? cf[2] : 0.f, G.mt, g);
    bool ill = false;
    const float dmax = G.tau > 0.f ? 0.99f * rsqrtf(G.tau) : kInf;
    float cb = cell_min_d2<N, float>(q, ok, g, G.mt, dmax, kInf, ill);
    if (ill) ill = cell_gram_ill<N>(q, ok, G.mt.kappa, G.tau);
    if (ill) {
        const double drd = dr;
        const double invd = 1.0 / ((double)G.dd_frac * (G.local ? drd : (double)dnorm));
        cb = cell_redo_f64<N, double>(G.ev, pidx, sy, sz, ok, (double)p[0] - u[0],
                                      (double)p[1] - u[1], N == 3 ? (double)p[2] - u[2] : 0.0,
                                      drd, invd, G.mtd, &G.ctr->fp64_cells);
    }
    return fminf(best, cb);
}

// GL lanes per reference voxel (GL-aligned groups of a warp; 2 .. 32).  The
// table starts with the voxel's own cell (offset 0), so the first round of G
// cells gives a finite bound; later cells are skipped when the distance from
// the point itself to the cell's box, with the dose gap, already reaches the
// running gamma.  The exact stop (A1 step 4b-ii) takes the table's key.
template <int N, int GL>
__global__ void __launch_bounds__(256, 2) k_grid_walk(const __grid_constant__ GridProblem G)
{
    const int lane = threadIdx.x & 31, gl = lane & (GL - 1), gbase = lane & ~(GL - 1);
    const unsigned gmask = GL == 32 ? kFull : (((1u << GL) - 1u) << gbase);
    const float dnorm = G.dose_norm > 0.f ? G.dose_norm : fdec(G.ctr->dnorm_enc);
    const float thr = cutoff_threshold(G.local, G.cutoff_frac, dnorm);
    unsigned my_eval = 0, my_pass = 0, my_over = 0;
    const long long ngroups = ((long long)gridDim.x * blockDim.x) / GL;
    // every reference voxel, or (from_list) those k_grid_cq left in walk_list
    const long long nwork = G.from_list ? (long long)G.ctr->fix_count : G.nref;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / GL; i < nwork;
         i += ngroups) {                                     // group-uniform
        const long long v = G.from_list ? (long long)G.walk_list[i] : i;
        const float dr = __ldg(G.ref + v);
        if (!(dr >= thr && (!G.local || dr > 0.f))) {
            if (gl == 0) G.out[v] = __int_as_float(0x7fc00000);
            continue;
        }
        const long long ix[3] = {v % G.rn[0], (v / G.rn[0]) % G.rn[1], v / ((long long)G.rn[0] * G.rn[1])};
        // the point in evaluation voxel units: its cell c0 (clamped to the
        // grid) and its position fr in that cell (outside [0, 1) beyond the
        // grid), from FP64 on one lane
        double u[3] = {0.0, 0.0, 0.0};
        int c0[3] = {0, 0, 0};
        float fr[3] = {0.f, 0.f, 0.f}, ehf[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < N; ++a) {
            double ua = 0.0, f = 0.0;
            if (gl == 0) {
                ua = (G.ro[a] + (double)ix[a] * G.rh[a] - G.eo[a]) / G.eh[a];
                f = fmin(fmax(floor(ua), 0.0), (double)(G.en[a] - 2));
            }
            u[a] = __shfl_sync(gmask, ua, gbase);
            c0[a] = (int)__shfl_sync(gmask, f, gbase);
            fr[a] = (float)(u[a] - (double)c0[a]);
            ehf[a] = (float)G.eh[a];
        }
        const float dD = G.dd_frac * (G.local ? dr : dnorm);
        const float inv = 1.0f / dD;
        // the table for the point's half of its cell per axis
        const int var = grid_variant(fr, N);
        const TableEntry* table = G.table + G.toff[var];
        const int ntable = G.tlen[var];
        const float rc2 = G.tcover[var] * G.tcover[var];
        float best = kInf;
        int t = 0;
        while (t < ntable) {
            const int idx = t + gl;
            float key = kInf;
            uint32_t off = 0;
            if (idx < ntable) {
                const TableEntry e = table[idx];
                key = e.key;
                off = e.off;
            }
            const float k0 = __shfl_sync(gmask, key, gbase);
            if (k0 * k0 >= best) break;                       // A1 step 4b-ii, exact
            float cb = best;
            if (key * key < best) {
                const int d[3] = {unpack10(off, 0), unpack10(off, 10), N == 3 ? unpack10(off, 20) : 0};
                const int p[3] = {c0[0] + d[0], c0[1] + d[1], c0[2] + d[2]};
                bool in = true;
                // the distance from the point to the cell's box: a lower bound
                // in FP32 from the integer offset and the point's fraction,
                // each axis lowered by its rounding (4 ulp of its operands) and
                // the sum by 1e-5
                float k2 = 0.f;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    in = in && p[a] >= 0 && p[a] < G.en[a];
                    const float lo = (float)d[a] - fr[a], hi = fr[a] - (float)(d[a] + 1);
                    const float slack = 4.8e-7f * (fabsf(fr[a]) + fabsf((float)d[a]) + 2.f);
                    const float gap = fmaxf(fmaxf(lo, hi) - slack, 0.f) * ehf[a];
                    k2 = fmaf(gap, gap, k2);
                }
                k2 *= 0.99999f;
                if (in && k2 < best) {
                    const float cf[3] = {(float)d[0] - fr[0], (float)d[1] - fr[1], (float)d[2] - fr[2]};
                    cb = grid_cell<N>(G, p, u, cf, sqrtf(fmaxf(k2, key * key)), dr, inv, dnorm, best);
                }
            }
#pragma unroll
            for (int o = GL / 2; o > 0; o >>= 1) cb = fminf(cb, __shfl_xor_sync(gmask, cb, o));
            best = cb;
            t += GL;
        }
        if (t >= ntable && best > rc2) {
            // past a truncated table: every remaining cell of the search box
            if (gl == 0) ++my_over;
            const float gm = sqrtf(best);
            int dlo[3] = {0, 0, 0}, dhi[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const float l = gm / (float)G.eh[a] + 2.f;
                const int lim = l < (float)G.en[a] ? (int)ceilf(l) : G.en[a];
                dlo[a] = max(-lim, -c0[a]);
                dhi[a] = min(lim, G.en[a] - 1 - c0[a]);
            }
            const long long wx = dhi[0] - dlo[0] + 1, wy = dhi[1] - dlo[1] + 1, wz = dhi[2] - dlo[2] + 1;
            const long long tot = wx * wy * wz;
            const float cut = rc2 * 0.99999f;
            float lb = best;
            for (long long b = gl; b < tot; b += GL) {
                const int d[3] = {dlo[0] + (int)(b % wx), dlo[1] + (int)((b / wx) % wy), dlo[2] + (int)(b / (wx * wy))};
                const int p[3] = {c0[0] + d[0], c0[1] + d[1], c0[2] + d[2]};
                bool in = true;
                float k2 = 0.f;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    in = in && p[a] >= 0 && p[a] < G.en[a];
                    const float gap = (float)grid_axis_key(d[a], var, a) * (float)G.eh[a];
                    k2 = fmaf(gap, gap, k2);
                }
                if (!in || k2 < cut || k2 >= lb) continue;
                const float cf[3] = {(float)d[0] - fr[0], (float)d[1] - fr[1], (float)d[2] - fr[2]};
                lb = grid_cell<N>(G, p, u, cf, sqrtf(k2), dr, inv, dnorm, lb);
            }
#pragma unroll
            for (int o = GL / 2; o > 0; o >>= 1) lb = fminf(lb, __shfl_xor_sync(gmask, lb, o));
            best = lb;
        }
        if (gl == 0) {
            const float gam = sqrtf(best);
            G.out[v] = gam;
            ++my_eval;
            my_pass += gam <= 1.f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_eval += __shfl_xor_sync(kFull, my_eval, o);
        my_pass += __shfl_xor_sync(kFull, my_pass, o);
        my_over += __shfl_xor_sync(kFull, my_over, o);
    }
    if (lane == 0) {
        if (my_eval) atomicAdd(&G.ctr->n_eval, (unsigned long long)my_eval);
        if (my_pass) atomicAdd(&G.ctr->n_pass, (unsigned long long)my_pass);
        if (my_over) atomicAdd(&G.ctr->overflow_count, my_over);
    }
}

// --------------------------------------------------------------------------
// The warp-evaluated walk (default): cells collected per warp, evaluated 32
// at a time
// --------------------------------------------------------------------------

// As for coincident grids (k_tail_cq), the face evaluation of a cell is not
// done by the lane that reached it: a cell that passes the box and dose-gap
// bounds is appended, with its vertex doses and its offset from the point, to
// a ring of the warp, and the whole warp evaluates 32 such cells at once, one
// per lane, lowering each owner's running bound in shared memory (atomicMin
// on the bits of a non-negative float).  GL lanes walk one reference voxel's
// table together (GL entries per step); a walker keeps two voxel slots so that
// it starts its next voxel while the cells of its last one wait.  Every stop
// and prune stays exact with a lagging bound, and each cell is evaluated with
// the arithmetic of grid_cell, so the map is k_grid_walk's.  A voxel with a
// near-singular cell, or whose walk runs past a truncated table, goes to
// walk_list; k_grid_walk then searches it again from scratch (FP64 redo, box
// scan), so that this kernel keeps the registers of the FP32 evaluation.
constexpr int kGqRing = 64;

struct GqWarp {
    float q[8][kGqRing];       // vertex doses of a pending cell (relative, normalised)
    float cf[3][kGqRing];      // its lower corner relative to the point (evaluation voxels)
    unsigned meta[kGqRing];    // owner slot (bits 0-5), vertices inside the grid (bits 8-15)
    unsigned best[64];         // running squared gamma per voxel slot (float bits)
    unsigned vox[64];          // reference voxel per slot
    float dr[32], inv[32];     // the walking voxel's reference dose and 1 / Delta D, per walker
    float fr[3][32];           // its position in its evaluation cell
    int c0[3][32];             // that cell
    int t[32];                 // its next table entry
    unsigned wseq[32], dseq[32], state[32];
    unsigned fixm[2];          // slots whose voxel is searched again by k_grid_walk
    unsigned cnt[2][32];       // voxels finished and passed
    unsigned pend[64];         // evaluated reference voxels not yet taken by a walker
    int tv[64];                // table variant of each slot's voxel
};
constexpr unsigned kGqWalk = 1u, kGqEnded = 2u, kGqWPend = 4u, kGqDBusy = 8u, kGqDPend = 16u,
                   kGqDOver = 32u, kGqSlot = 64u;     // slot bit: the walking slot is walker + 32

template <int N, int GL>
__global__ void __launch_bounds__(256, 2) k_grid_cq(const __grid_constant__ GridProblem G)
{
    __shared__ GqWarp gqw[8];
    GqWarp& W = gqw[threadIdx.x >> 5];
    volatile GqWarp& V = gqw[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31, gl = lane & (GL - 1), ld = lane - gl;
    const bool leader = gl == 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned gmask = GL == 32 ? kFull : ((1u << GL) - 1u) << ld;
    const float dnorm = G.dose_norm > 0.f ? G.dose_norm : fdec(G.ctr->dnorm_enc);
    const float thr = cutoff_threshold(G.local, G.cutoff_frac, dnorm);
    const float ehf[3] = {(float)G.eh[0], (float)G.eh[1], (float)G.eh[2]};
    W.state[lane] = 0;
    W.wseq[lane] = W.dseq[lane] = 0;
    W.cnt[0][lane] = W.cnt[1][lane] = 0;
    W.tv[lane] = W.tv[lane + 32] = 8;
    if (lane < 2) W.fixm[lane] = 0;
    __syncwarp();

    unsigned head = 0, count = 0;      // the ring: pending cells are [head, head + count)
    unsigned pend_n = 0;               // entries of W.pend (warp-uniform)
    bool queue_done = false;           // warp-uniform
    for (;;) {
        unsigned sta = V.state[ld];
        if (leader) {
            // 1. a drained voxel whose cells are all evaluated is final
            if ((sta & kGqDBusy) && (!(sta & kGqDPend) || (int)(head - V.dseq[ld]) > 0)) {
                const int ds = ld + ((sta & kGqSlot) ? 0 : 32);
                const float best = __uint_as_float(V.best[ds]);
                const unsigned v = V.vox[ds];
                const float rc = G.tcover[V.tv[ds]];
                if (((V.fixm[ds >> 5] >> (ds & 31)) & 1u) || ((sta & kGqDOver) && best > rc * rc)) {
                    G.walk_list[atomicAdd(&G.ctr->fix_count, 1u)] = v;   // k_grid_walk finishes it
                } else {
                    const float gam = sqrtf(best);
                    G.out[v] = gam;
                    ++V.cnt[0][ld];
                    if (gam <= 1.f) ++V.cnt[1][ld];
                }
                sta &= ~kGqDBusy;
            }
            // 2. an ended walk becomes the drain slot; the walker takes a new voxel
            if ((sta & kGqEnded) && !(sta & kGqDBusy)) {
                unsigned d = kGqDBusy;
                if (sta & kGqWPend) d |= kGqDPend;
                if (V.t[ld] >= G.tlen[V.tv[ld + ((sta & kGqSlot) ? 32 : 0)]]) d |= kGqDOver;
                V.dseq[ld] = V.wseq[ld];
                sta = d | ((sta & kGqSlot) ^ kGqSlot);
            }
        }
        // 3. refill the empty walkers, from a per-warp list of evaluated voxels
        //    that the warp fills 32 grid voxels at a time (one atomic each)
        const bool empty = leader && !(sta & (kGqWalk | kGqEnded));
        const unsigned need = __ballot_sync(kFull, empty);
        while (__popc(need) > (int)pend_n && !queue_done) {      // warp-uniform
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&G.ctr->head, 32u);
            base = __shfl_sync(kFull, base, 0);
            const long long v = (long long)base + lane;
            bool take = false;
            if (v < G.nref) {
                const float r = __ldg(G.ref + v);
                take = r >= thr && (!G.local || r > 0.f);
                if (!take) G.out[v] = __int_as_float(0x7fc00000);
            }
            const unsigned tk = __ballot_sync(kFull, take);
            if (take) V.pend[pend_n + __popc(tk & lt_mask)] = (unsigned)v;
            pend_n += __popc(tk);
            if ((long long)base + 32 >= G.nref) queue_done = true;
            __syncwarp();
        }
        if (empty) {
            const int k = __popc(need & lt_mask);
            if (k < (int)pend_n) {
                const unsigned v = V.pend[pend_n - 1 - k];
                const int ws = ld + ((sta & kGqSlot) ? 32 : 0);
                const long long ix[3] = {v % G.rn[0], (v / G.rn[0]) % G.rn[1], v / ((long long)G.rn[0] * G.rn[1])};
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    // the point in evaluation voxel units: its cell (clamped to
                    // the grid) and its position in that cell (FP64, once)
                    const double ua = (G.ro[a] + (double)ix[a] * G.rh[a] - G.eo[a]) / G.eh[a];
                    const double f = fmin(fmax(floor(ua), 0.0), (double)(G.en[a] - 2));
                    V.c0[a][ld] = (int)f;
                    V.fr[a][ld] = (float)(ua - f);
                }
                for (int a = N; a < 3; ++a) {
                    V.c0[a][ld] = 0;
                    V.fr[a][ld] = 0.f;
                }
                {
                    float frr[3];
                    for (int a = 0; a < 3; ++a) frr[a] = V.fr[a][ld];
                    V.tv[ws] = grid_variant(frr, N);
                }
                const float dr = __ldg(G.ref + v);
                V.dr[ld] = dr;
                V.inv[ld] = 1.0f / (G.dd_frac * (G.local ? dr : dnorm));
                V.best[ws] = __float_as_uint(kInf);
                V.vox[ws] = v;
                atomicAnd(&W.fixm[ws >> 5], ~(1u << (ws & 31)));
                V.t[ld] = 0;
                sta = (sta & ~kGqWPend) | kGqWalk;
            }
        }
        pend_n -= min((unsigned)__popc(need), pend_n);
        if (leader) V.state[ld] = sta;
        __syncwarp();
        sta = V.state[ld];                 // the group's lanes follow their walker
        if (queue_done && pend_n == 0 &&
            !__any_sync(kFull, (sta & (kGqWalk | kGqEnded | kGqDBusy)) != 0))
            break;

        // 4. one table step of every walking group: entries t .. t + GL - 1
        const bool walking = (sta & kGqWalk) != 0;
        const int ws = ld + ((sta & kGqSlot) ? 32 : 0);
        const int t0 = walking ? V.t[ld] : 0;
        float key = kInf;
        uint32_t off = 0;
        const int var = V.tv[ws];
        const int ntable = G.tlen[var];
        if (walking && t0 + gl < ntable) {
            const TableEntry e = G.table[G.toff[var] + t0 + gl];
            key = e.key;
            off = e.off;
        }
        const float k0 = __shfl_sync(kFull, key, ld);
        bool cand = false, ended = false;
        float q[8], cf[3] = {0.f, 0.f, 0.f};
        uint32_t ok = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = 0.f;
        if (walking) {
            const float bst = __uint_as_float(V.best[ws]);
            ended = t0 >= ntable || k0 * k0 >= bst;           // A1 step 4b-ii, exact
            if (!ended && key * key < bst) {
                const int d[3] = {unpack10(off, 0), unpack10(off, 10), N == 3 ? unpack10(off, 20) : 0};
                int p[3];
                bool in = true;
                // the distance from the point to the cell's box: a lower bound
                // in FP32 from the integer offset and the point's fraction,
                // each axis lowered by its rounding and the sum by 1e-5
                float k2 = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    p[a] = V.c0[a][ld] + d[a];
                    const float fr = V.fr[a][ld];
                    cf[a] = (float)d[a] - fr;
                    if (a < N) {
                        in = in && p[a] >= 0 && p[a] < G.en[a];
                        const float lo = (float)d[a] - fr, hi = fr - (float)(d[a] + 1);
                        const float slack = 4.8e-7f * (fabsf(fr) + fabsf((float)d[a]) + 2.f);
                        const float gap = fmaxf(fmaxf(lo, hi) - slack, 0.f) * ehf[a];
                        k2 = fmaf(gap, gap, k2);
                    }
                }
                k2 *= 0.99999f;
                if (in && k2 < bst) {
                    const long long sy = G.en[0], sz = (long long)G.en[0] * G.en[1];
                    const long long pidx = (long long)p[2] * sz + (long long)p[1] * sy + p[0];
                    const bool ex = p[0] + 1 < G.en[0], ey = p[1] + 1 < G.en[1], ez = N == 3 && p[2] + 1 < G.en[2];
                    const float dr = V.dr[ld], inv = V.inv[ld];
                    float qmin = kInf, qmax = -kInf;
#pragma unroll
                    for (int u = 0; u < (1 << N); ++u) {
                        const bool present = (!(u & 1) || ex) && (!(u & 2) || ey) && (!(u & 4) || ez);
                        if (present) {
                            const long long o = pidx + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) + ((u & 4) ? sz : 0);
                            q[u] = (__ldg(G.ev + o) - dr) * inv;
                            qmin = fminf(qmin, q[u]);
                            qmax = fmaxf(qmax, q[u]);
                            ok |= 1u << u;
                        }
                    }
                    const float gap = qmin > 0.f ? qmin : (qmax < 0.f ? -qmax : 0.f);
                    const float kb = sqrtf(fmaxf(k2, key * key));
                    cand = fmaf(gap, gap, kb * kb) < bst;
                }
            }
        }
        // 5. append the surviving cells to the ring
        const unsigned cm = __ballot_sync(kFull, cand);
        if (cand) {
            const unsigned seq = head + count + (unsigned)__popc(cm & lt_mask);
            const int slot = (int)(seq & (kGqRing - 1));
#pragma unroll
            for (int u = 0; u < (1 << N); ++u) V.q[u][slot] = q[u];
#pragma unroll
            for (int a = 0; a < 3; ++a) V.cf[a][slot] = cf[a];
            V.meta[slot] = (unsigned)ws | (ok << 8);
        }
        if (leader && walking) {
            if (ended) {
                sta = (sta & ~kGqWalk) | kGqEnded;
            } else {
                V.t[ld] = t0 + GL;
                const unsigned gm = cm & gmask;
                if (gm) {                   // the group's last appended cell
                    const int hl = 31 - __clz(gm);
                    V.wseq[ld] = head + count + (unsigned)__popc(cm & ((1u << hl) - 1u));
                    sta |= kGqWPend;
                }
            }
            V.state[ld] = sta;
        }
        count += (unsigned)__popc(cm);
        const int nwalk = GL * __popc(__ballot_sync(kFull, leader && (sta & kGqWalk) && !ended));
        __syncwarp();
        // 6. evaluate the oldest 32 pending cells (or fewer, when few lanes walk)
        if (count >= 32u || (count > 0u && nwalk < 16)) {
            const unsigned n = min(count, 32u);
            if ((unsigned)lane < n) {
                const int slot = (int)((head + (unsigned)lane) & (kGqRing - 1));
                const unsigned meta = V.meta[slot];
                const int owner = (int)(meta & 63u);
                const unsigned cok = meta >> 8;
                float cq[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) cq[u] = u < (1 << N) ? V.q[u][slot] : 0.f;
                CellGeom<float> cg;
                cell_geom<N, float>(V.cf[0][slot], V.cf[1][slot], N == 3 ? V.cf[2][slot] : 0.f, G.mt, cg);
                bool ill = false;
                const float dmax = G.tau > 0.f ? 0.99f * rsqrtf(G.tau) : kInf;
                const float cb = cell_min_d2<N, float>(cq, cok, cg, G.mt, dmax, kInf, ill);
                if (ill && cell_gram_ill<N>(cq, cok, G.mt.kappa, G.tau))
                    atomicOr(&W.fixm[owner >> 5], 1u << (owner & 31));   // searched again
                else
                    atomicMin(&W.best[owner], __float_as_uint(cb + 0.f));   // -0 -> +0
            }
            head += n;
            count -= n;
        }
        __syncwarp();
    }
    unsigned c0 = W.cnt[0][lane], c1 = W.cnt[1][lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_xor_sync(kFull, c0, o);
        c1 += __shfl_xor_sync(kFull, c1, o);
    }
    if (lane == 0) {
        if (c0) atomicAdd(&G.ctr->n_eval, (unsigned long long)c0);
        if (c1) atomicAdd(&G.ctr->n_pass, (unsigned long long)c1);
    }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------

int build_grid_table(int nd, const double hn[3], const int en[3], long long cap, int variant,
                     std::vector<TableEntry>& table, double& r_cover)
{
    // radius from a ball-volume estimate of about 2 * cap cells
    const double cellvol = hn[0] * hn[1] * (nd == 3 ? hn[2] : 1.0);
    double R = nd == 3 ? std::cbrt(2.0 * (double)cap * cellvol * 3.0 / (4.0 * M_PI))
                       : std::sqrt(2.0 * (double)cap * cellvol / M_PI);
    bool whole = false, packing = false;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    double diag = 0;
    for (int a = 0; a < nd; ++a) diag += (double)en[a] * en[a] * hn[a] * hn[a];
    diag = std::sqrt(diag) + 1.0;
    if (R > diag) { R = diag; whole = true; }
    for (int a = 0; a < nd; ++a) {
        long long l = (long long)std::ceil(R / hn[a]) + 2;
        l = std::min<long long>(l, en[a]);
        if (l > 511) { l = 511; packing = true; }
        lo[a] = -(int)l;
        hi[a] = (int)l;
    }
    struct Tmp { double key; int x, y, z; };
    std::vector<Tmp> all;
    try {
        for (int z = lo[2]; z <= hi[2]; ++z)
            for (int y = lo[1]; y <= hi[1]; ++y)
                for (int x = lo[0]; x <= hi[0]; ++x) {
                    const int c[3] = {x, y, z};
                    double k2 = 0;
                    for (int a = 0; a < nd; ++a) {
                        const double gap = grid_axis_key(c[a], variant, a) * hn[a];
                        k2 += gap * gap;
                    }
                    const double key = std::sqrt(k2);
                    if (key < R) all.push_back({key, x, y, z});
                }
    } catch (const std::bad_alloc&) {
        return GAMMA_ERR_OOM;
    }
    std::sort(all.begin(), all.end(), [](const Tmp& a, const Tmp& b) {
        if (a.key != b.key) return a.key < b.key;
        // the voxel's own cell first among the key-0 cells (a finite bound
        // from the walk's first round), then z, y, x
        const bool a0 = (a.x | a.y | a.z) == 0, b0 = (b.x | b.y | b.z) == 0;
        if (a0 != b0) return a0;
        if (a.z != b.z) return a.z < b.z;
        if (a.y != b.y) return a.y < b.y;
        return a.x < b.x;
    });
    double cover = whole ? INFINITY : R;
    if (packing) {
        double m = INFINITY;
        for (int a = 0; a < nd; ++a) m = std::min(m, 509.0 * hn[a]);
        cover = std::min(cover, m);
    }
    size_t keep = all.size();
    if ((long long)keep > cap) {
        keep = (size_t)cap;
        cover = std::min(cover, all[keep].key);
    }
    table.resize(keep);
    for (size_t i = 0; i < keep; ++i) {
        table[i].off = pack10(all[i].x, all[i].y, all[i].z);
        float f = (float)all[i].key;
        if ((double)f > all[i].key) f = std::nextafterf(f, -INFINITY);
        table[i].key = f;
    }
    r_cover = cover;
    return GAMMA_OK;
}

template <int N>
static void launch_grid_walk_n(const GridProblem& G, int gl, int grid, cudaStream_t s)
{
    switch (gl) {
    case 2: k_grid_walk<N, 2><<<grid, 256, 0, s>>>(G); break;
    case 4: k_grid_walk<N, 4><<<grid, 256, 0, s>>>(G); break;
    case 16: k_grid_walk<N, 16><<<grid, 256, 0, s>>>(G); break;
    case 32: k_grid_walk<N, 32><<<grid, 256, 0, s>>>(G); break;
    default: k_grid_walk<N, 8><<<grid, 256, 0, s>>>(G); break;
    }
}

cudaError_t launch_grids(const GridProblem& G, cudaStream_t s)
{
    const int sms = device_sm_count();
    const long long nmax = std::max(G.nref, G.neval);
    const int gp = (int)std::max<long long>(1, std::min<long long>((nmax + 255) / 256, (long long)sms * 8));
    k_grid_prepare<<<gp, 256, 0, s>>>(G);
    if (G.walk == 3 && G.walk_list) {
        // the warp-evaluated walk, then a 32-lane search of the voxels it left
        if (G.ndim == 3) k_grid_cq<3, 8><<<sms * 2, 256, 0, s>>>(G);
        else k_grid_cq<2, 8><<<sms * 2, 256, 0, s>>>(G);
        GridProblem F = G;
        F.from_list = 1;
        if (G.ndim == 3) launch_grid_walk_n<3>(F, 32, sms * 2, s);
        else launch_grid_walk_n<2>(F, 32, sms * 2, s);
        return cudaGetLastError();
    }
    const int gl = G.lanes;
    const int gw = (int)std::max<long long>(1, std::min<long long>((G.nref * gl + 255) / 256,
                                                                   (long long)sms * 16));
    if (G.ndim == 3) launch_grid_walk_n<3>(G, gl, gw, s);
    else launch_grid_walk_n<2>(G, gl, gw, s);
    return cudaGetLastError();
}

}  // namespace gk
