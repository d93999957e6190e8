// Internal structures shared by the CUDA kernels and the C-ABI layer.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "gamma_face.cuh"
#include "gamma_mlp.cuh"

struct gamma_model_s;

namespace gk {

constexpr int kNumBuckets = 32;
constexpr int kShellSlots = 8;       // shell launches of one run with their own tile counter

// Launch shapes a new handle starts with (options "lanes_per_voxel",
// "shell_blocks_per_sm", "tail_blocks_per_sm"); gamma_run_noalloc, which has
// no options, always uses them.
constexpr int kDefaultLanesPerVoxel = 8;
constexpr int kDefaultShellBlocksPerSm = 2;
constexpr int kDefaultTailBlocksPerSm = 2;

// Flags raised by kernels (Counters::flags).
enum : uint32_t {
    kFlagNonFinite = 1u,     // a NaN or Inf dose was seen
    kFlagTailFull = 2u,      // the tail queue overflowed its capacity
    kFlagTimeout = 4u,       // a bounded wait on a tile copy gave up
};

// One entry of the radially sorted cell table (Algorithm A1 steps 2-3):
// the cell's lower-corner offset relative to the reference voxel, packed as
// three signed 10-bit fields (x | y << 10 | z << 20), and the key: a lower
// bound, divided by the DTA and rounded down to float, on the spatial
// distance from the voxel to every face of the cell the table walk still has
// to evaluate.  That is the distance to the cell box, except for the cells
// whose box contains the voxel (key-0 cells): their faces through the voxel
// are done before the walk, so their key is the distance to their other
// faces, and the cell whose corner is the voxel (all its faces contain it) is
// not in the table.
struct TableEntry {
    uint32_t off;
    float key;
};

__host__ __device__ inline int unpack10(uint32_t v, int shift)
{
    int f = int((v >> shift) & 1023u);
    return f >= 512 ? f - 1024 : f;
}

__host__ __device__ inline uint32_t pack10(int x, int y, int z)
{
    return (uint32_t(x) & 1023u) | ((uint32_t(y) & 1023u) << 10) | ((uint32_t(z) & 1023u) << 20);
}

// Device-side counters; zeroed at the start of every run.
struct Counters {
    unsigned long long n_eval;
    unsigned long long n_pass;
    unsigned long long cells_visited;   // stats mode: cells whose faces were evaluated
    unsigned long long cells_pruned;    // stats mode: cells skipped by the lower bound
    unsigned long long cells_keyed;     // stats mode: table cells reached before the break
    unsigned int dnorm_enc;             // max reference dose, order-preserving int code
    unsigned int rmax_enc;              // max gamma0 over evaluated voxels (same code)
    unsigned int flags;
    unsigned int tail_count;
    unsigned int head;
    unsigned int overflow_count;        // voxels that needed the box scan
    unsigned int fp64_cells;            // cells redone in FP64
    unsigned int seed_head;             // work counter of the learned seeding pass
    unsigned int seeded;                // queued voxels the proposal network seeded
    unsigned int seed_improved;         // ... whose bound the seed lowered
    unsigned int seed_count;            // queued voxels past the seeding cost gate
    unsigned int shell_next[kShellSlots];   // tile work counters of the shell launches
    unsigned int hist[kNumBuckets];
    unsigned int cursor[kNumBuckets];
    unsigned int tile_count;            // shell tiles with at least one queued voxel
    unsigned int tile_head;             // work counter of the tile-staged walk
    unsigned int tile_hist[kNumBuckets];    // those tiles by their largest cost bucket
    unsigned int tile_cursor[kNumBuckets];
    unsigned int row_count;             // shell warp rows with at least one queued voxel
    unsigned int row_head;              // work counter of the row-staged walk
    unsigned int row_hist[kNumBuckets]; // those rows by their largest cost bucket
    unsigned int row_cursor[kNumBuckets];
    unsigned int head_part[4];          // warp-evaluated walk: work counters of the queue's parts
    unsigned int fix_count;             // ... voxels it leaves to the finishing pass
    unsigned long long lane_steps;      // stats mode: lane slots of its loop steps, idle lanes included
};

// The cost bucket thresholds of a sorted table (Problem::bucket_key).
inline void fill_bucket_keys(const TableEntry* table, int ntable, float* out)
{
    out[0] = -__builtin_huge_valf();
    for (int b = 1; b < kNumBuckets; ++b) {
        const double c = std::ceil(std::pow(2.0, 0.5 * (b - 1)));
        out[b] = c <= (double)ntable ? table[(long long)c - 1].key : __builtin_huge_valf();
    }
}

// The cost bucket of a voxel whose search radius (normalised) is g: the
// number of thresholds below g, by bisection over the non-decreasing keys.
__host__ __device__ inline int cost_bucket_of(const float* bucket_key, float g)
{
    int b = 0;
    for (int step = kNumBuckets / 2; step > 0; step >>= 1)
        if (b + step < kNumBuckets && bucket_key[b + step] < g) b += step;
    return b;
}

// Order-preserving encoding of a float into an unsigned int (for atomicMax).
__host__ __device__ inline unsigned int fenc(float f)
{
    union { float f; unsigned int u; } c;
    c.f = f;
    return (c.u & 0x80000000u) ? ~c.u : (c.u | 0x80000000u);
}
__host__ __device__ inline float fdec(unsigned int e)
{
    union { float f; unsigned int u; } c;
    c.u = (e & 0x80000000u) ? (e & 0x7fffffffu) : ~e;
    return c.f;
}

// Everything a launch needs about one dose pair.
struct Problem {
    const float* ref;
    const float* ev;
    float* out;
    long long nvox;
    int ndim;
    int nx, ny, nz;
    float hn[3];             // h_a / dta
    Metric mt;               // FP32 metric constants
    MetricT<double> mtd;     // FP64 copies for the ill-conditioned redo
    float dd_frac;
    float cutoff_frac;
    float dose_norm;         // > 0: fixed; else the device max of the reference
    int local;
    float tau;               // FP64 redo when det(G)/prod(G_ii) < tau (0: never)
    int stats;               // count cells in the tail search
    const TableEntry* table;
    int ntable;
    // cost bucket thresholds: bucket_key[b] (b >= 1) is the key of table entry
    // ceil(2^((b - 1) / 2)) - 1 (+inf past the table), so that the cost bucket
    // 1 + floor(2 log2 c) of a voxel with c table keys below g is the number
    // of b >= 1 with bucket_key[b] < g (0 when c = 0); bucket_key[0] = -inf
    float bucket_key[kNumBuckets];
    float r_cover;           // every cell with key < r_cover is in the table
    unsigned int tail_cap;
    Counters* ctr;
    unsigned int* tail_raw;      // unsorted tail voxels
    unsigned char* tail_bucket;  // their cost buckets
    unsigned int* tail_sorted;   // tail voxels, most expensive bucket first
    int sort_tail;               // 0: keep discovery order (ablation)
    int shell_minblocks;         // k_shell register budget: resident blocks per SM, 1..4
    // squared spatial distance from the voxel to the faces of key-0 cell S
    // (lower corner at -S) that do not contain it, rounded down; +inf for S = 0
    float key0_far2[8];
    // learned seeding: the queue items past the cost gate, and the row
    // buffers of the network (features, outputs) for up to seed_cap of them
    unsigned* seed_list;
    __nv_bfloat16* seed_X;         // [seed_cap][kInPad]
    float* seed_Y;                 // [seed_cap][kOut]
    unsigned seed_cap;
    // tile-staged walk (null: the queue is walked voxel by voxel, k_tail):
    // per shell tile one bit per voxel of the tile that is queued (8 words,
    // word = warp of the tile, bit = lane), the tiles with any queued voxel
    // (unordered, with their largest cost bucket) and the same tiles ordered
    // by that bucket, most expensive first
    unsigned* tile_mask;
    unsigned* tile_list;
    unsigned char* tile_bkt;
    unsigned* tile_sorted;
    // row-staged walk (null: not used): per shell warp row with queued voxels
    // one item (row id = tile * 8 + warp in the high word, queue mask in the
    // low word) with its largest cost bucket, and the items in cost order
    unsigned long long* row_items;
    unsigned char* row_bkt;
    unsigned long long* row_sorted;
    // warp-evaluated walk (k_tail_cq): queued voxels of cost bucket
    // cq_group32_bucket and above walk 32 lanes each, of cq_group8_bucket and
    // above 8, of cq_group_bucket and above 4; fix_list (tail_cap entries)
    // holds the voxels whose exact result the finishing pass completes
    int cq_group_bucket;         // < 0: the walk chooses the three from the queue (auto_part_buckets)
    int cq_group8_bucket;
    int cq_group32_bucket;
    float cq_auto_scale;         // ... with this slack
    unsigned* fix_list;
};

// Readiness of the evaluation dose by z slab, for a shell launch that starts
// while the dose is still being copied in: slab k (voxel slices
// [k * depth, (k + 1) * depth)) has landed once flag[k] has reached epoch
// (slabs may land in any order).  flag == nullptr: the whole dose is present.
struct SlabGate {
    const unsigned* flag;
    unsigned epoch;
    int depth;
};

// Device-side description of the pairs of one batched launch group (pairs of
// the same dimension).  All arrays live in device memory.
struct BatchDesc {
    int npairs;
    const Problem* probs;          // [npairs], shell constants filled in
    const CUtensorMap* maps;       // [npairs] evaluation-dose tile maps
    const int* use_tma;            // [npairs] 1: the map is valid for TMA loads
    const int* tile_start;         // [npairs + 1] first global shell tile of each pair
    unsigned* item_start;          // [npairs * kNumBuckets + 4] start of each (pair, cost
                                   // bucket) range of the queued voxels, their total, and
                                   // the ends of the first three parts (k_bucket_scan_batch)
    unsigned* items_v;             // [sum of tail_cap] queued voxels in that order
    unsigned short* items_p;       // [sum of tail_cap] their pair
    unsigned* head;                // work counter of the group's table walk
    // warp-evaluated walk: cost buckets from which the queued voxels walk 4,
    // 8 and 32 lanes each (the queue's parts, costliest first; all 0 keeps one
    // pair-major order), the work counters of the parts, and the voxels (with
    // their pair) left to the finishing pass
    int group_bucket, group8_bucket, group32_bucket;   // group_bucket < 0: chosen from the queue
    float auto_scale;              // ... with this slack, for a walk of walk_lanes lanes
    unsigned walk_lanes;
    unsigned* part_head;           // [4]
    const float4* metric4;         // [npairs][3] per pair: hn2 x, y, z, tau; kappa 1-4;
                                   // kappa 5-7, 0
    unsigned* fix_v;               // [sum of tail_cap]
    unsigned short* fix_p;
    unsigned* fix_count;
    unsigned* shell_next;          // tile counter of the group's shell (zeroed by its prepare)
    // learned seeding (null without a model): queue items of every pair past
    // the cost gate, as (pair, item) rows, their count and the work counter of
    // the seeding pass (both zeroed by the group's prepare)
    unsigned* seed_item;           // [seed_cap]
    unsigned short* seed_pair;     // [seed_cap]
    unsigned* seed_count;
    unsigned* seed_head;
    __nv_bfloat16* seed_X;         // [seed_cap][kInPad] network inputs
    float* seed_Y;                 // [seed_cap][kOut] network outputs
    unsigned seed_cap;             // rows past it go unseeded
};

// Host view of one batched launch group.
struct BatchGroup {
    int ndim;
    int npairs;
    long long max_nvox;            // largest pair, for the prepare grid
    int total_tiles;               // shell tiles over all pairs
    const BatchDesc* desc;         // device copy of the descriptor
    unsigned* shell_next;          // device: the descriptor's shell tile counter
    // learned seeding (seed_cap 0: no model): the descriptor's row buffers and
    // row count, and where a timed-out wait of the network is reported
    __nv_bfloat16* seed_X;
    float* seed_Y;
    unsigned seed_cap;
    unsigned* seed_count;
    unsigned* flags;
};

// Launchers (gamma_kernels.cu).  All are stream-ordered and allocate nothing.
// part: 1 = reference dose only (norm, finite check), 2 = evaluation dose only
// (finite check), 3 = both.
cudaError_t launch_prepare(const Problem& P, cudaStream_t s, int part = 3);
cudaError_t launch_shell(const Problem& P, cudaStream_t s);
// Shell over tiles [tile_first, tile_end).  Tiles run x fastest, then y, then
// z: shell_layers gives the tiles of one z layer, the number of layers and the
// voxel depth of a layer, so that a z slab of layers is one tile range.
// Each launch of one run takes its own tile counter, slot 0 .. kShellSlots - 1.
// A gate makes the launch wait, tile by tile, for the z slabs its tiles read
// (only with TMA tile loads; false from shell_gate_ok otherwise).
cudaError_t launch_shell_range(const Problem& P, int tile_first, int tile_end, int slot,
                               const SlabGate& gate, cudaStream_t s);
bool shell_gate_ok(const Problem& P);
void shell_layers(const Problem& P, int* tiles_per_layer, int* layers, int* layer_depth);
// Final gamma of every queued voxel into a host map, through its
// device-mapped pointer, and (when given) the run's counters into mapped
// host memory.
cudaError_t launch_patch_host(const Problem& P, float* host_out_mapped, Counters* host_ctr_mapped,
                              cudaStream_t s);
cudaError_t launch_order_tail(const Problem& P, cudaStream_t s);
cudaError_t launch_tail(const Problem& P, int lanes_per_voxel, int tail_minblocks, cudaStream_t s);
// one lane per queued voxel, surviving cells evaluated by the whole warp
cudaError_t launch_tail_cq(const Problem& P, int tail_minblocks, cudaStream_t s);
// Tile-staged walk (P.tile_mask set): order the tiles with queued voxels by
// cost, then one block per tile stages the tile's evaluation-dose halo box in
// shared memory and walks the table for the tile's queued voxels.
cudaError_t launch_order_tiles(const Problem& P, cudaStream_t s);
cudaError_t launch_walk(const Problem& P, int walk_minblocks, cudaStream_t s);
// Row-staged walk (P.row_items set): order the shell's warp rows with queued
// voxels by cost, then every warp takes one row at a time, stages the row's
// evaluation-dose halo box in shared memory and walks the table for the
// row's queued voxels.
cudaError_t launch_order_rows(const Problem& P, cudaStream_t s);
cudaError_t launch_walk_rows(const Problem& P, int walk_minblocks, cudaStream_t s);
int device_sm_count();

// Host-side constants a Problem needs before it is uploaded for a batch.
// Spatial distance (DTA units, rounded down) from the voxel to the faces of
// key-0 cell S that do not contain it, for S = 1 .. 2^nd - 1; far[0] = +inf.
void key0_far(const double hn[3], int nd, double far[8]);
// Tile-load map for a Problem; false when TMA cannot be used for it.
bool encode_tile_map(const Problem& P, CUtensorMap* map);
int shell_tiles(const Problem& P);
// Tiles of k_shell's layout (the staged walks' units).
int block_tiles(const Problem& P);

// Learned proposal (gamma_learned.cu).
bool model_weights(const gamma_model_s* m, MlpWeights* w);
// Seeding of one pair's queued voxels: the items whose cost bucket is at
// least min_bucket (into P.seed_list), their features (P.seed_X), the network
// on the tensor cores (P.seed_Y) and the exact seeds from the proposals.
cudaError_t launch_seeding(const Problem& P, const MlpWeights& W, int min_bucket, cudaStream_t s);
// Network outputs for M feature rows (row-major [M][384] BF16, 16-byte aligned).
cudaError_t launch_mlp_infer(const MlpWeights& W, const __nv_bfloat16* X, long long M, float* Y,
                             unsigned* flags, cudaStream_t s);

// Reference and evaluation doses on different grids (gamma_grids.cu).
// Positions and spacings are in DTA units, axes (x, y, z).
struct GridProblem {
    const float* ref;
    const float* ev;
    float* out;
    int ndim;
    int rn[3], en[3];            // reference / evaluation grid sizes (z = 1 in 2D)
    double ro[3], rh[3];         // reference origin and spacing
    double eo[3], eh[3];         // evaluation origin and spacing
    long long nref, neval;
    Metric mt;                   // evaluation-grid metric (hn = eh)
    MetricT<double> mtd;
    float dd_frac, cutoff_frac, dose_norm;
    int local;
    float tau;
    // nine cell tables, concatenated: variant 8 keyed by the gap between cell
    // boxes (any point of the voxel's cell, or a point outside the grid),
    // variants 0-7 by the smallest distance from a point in one half of its
    // cell per axis (bit a: the upper half of axis a); entries toff[k] ..
    // toff[k] + tlen[k] - 1, every cell with key < tcover[k] included
    const TableEntry* table;
    int toff[9], tlen[9];
    float tcover[9];
    Counters* ctr;
    int lanes;                   // lanes per reference voxel (2 .. 32)
    int walk;                    // 3: the warp-evaluated walk (k_grid_cq), else k_grid_walk
    unsigned* walk_list;         // voxels k_grid_cq leaves to k_grid_walk (nref entries)
    int from_list;               // k_grid_walk: walk only walk_list[0 .. ctr->fix_count)
};
int build_grid_table(int nd, const double hn[3], const int en[3], long long cap, int variant,
                     std::vector<TableEntry>& table, double& r_cover);
cudaError_t launch_grids(const GridProblem& G, cudaStream_t s);

// Paper-design ablation (gamma_paper.cu): one thread per voxel, optionally in
// DD order, all simplices of every cell reached (closed form or Ju's recursion).
struct PaperScratch {
    unsigned *keys = nullptr, *ids = nullptr, *keys_alt = nullptr, *ids_alt = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0;
};
size_t paper_sort_bytes(long long nvox);
cudaError_t launch_paper(const Problem& P, const PaperScratch& w, bool sorted, bool ju,
                         cudaEvent_t after_sort, cudaStream_t s);
cudaError_t launch_features(const Problem& P, const unsigned* vox, long long n, __nv_bfloat16* X,
                            cudaStream_t s);
cudaError_t launch_labels(const Problem& P, const float* gmap, const unsigned* vox, long long n,
                          float* T, cudaStream_t s);

// Batched launches over one group: prepare, shell, ordering, table walk.
cudaError_t launch_batch_prepare(const BatchGroup& g, cudaStream_t s);
cudaError_t launch_batch_shell(const BatchGroup& g, int shell_minblocks, cudaStream_t s);
cudaError_t launch_batch_order(const BatchGroup& g, cudaStream_t s);
// walk: 3 the warp-evaluated walk, else the voxel walk with lanes_per_voxel.
cudaError_t launch_batch_tail(const BatchGroup& g, int walk, int lanes_per_voxel, int tail_minblocks,
                              cudaStream_t s);
// Tensor map of a row-major bf16 matrix (inner elements x rows, row stride in
// bytes) with boxes of box_inner x box_rows elements; false when the driver's
// encoder is missing or the alignment rules fail.
bool encode_bf16_2d(CUtensorMap* map, const void* base, unsigned long long inner,
                    unsigned long long rows, unsigned long long row_stride_bytes,
                    unsigned box_inner, unsigned box_rows);
// C (+)= A B^T on the tensor cores (gamma_gemm_tc.cu): A [M][K] and B [N][K]
// bf16 with K contiguous (row strides lda, ldb: multiples of 8 elements, bases
// 16-byte aligned), C fp32 [M][ldc].  With splits > 1 the K range is split over
// that many blocks per tile, which add into C (it must hold the initial value,
// normally zero); else C is overwritten.  flags receives kFlagTimeout if a
// bounded wait gave up.
cudaError_t launch_gemm_tc(const __nv_bfloat16* A, long long M, long long lda, const __nv_bfloat16* B,
                           int N, long long ldb, long long K, float* C, int ldc, int splits,
                           unsigned* flags, cudaStream_t s);
// dst [cols][ldd] = transpose of src [rows][cols] (row stride lds); the
// columns rows .. ldd - 1 of dst are zeroed.
cudaError_t launch_transpose_bf16(const __nv_bfloat16* src, long long rows, int cols, long long lds,
                                  __nv_bfloat16* dst, long long ldd, cudaStream_t s);

// Learned seeding of a batch group (gamma_learned.cu): the queue items of every
// pair whose cost bucket is at least min_bucket as (pair, item) rows, then the
// features, network and exact seeds of all of them, one launch each.
cudaError_t launch_batch_seeding(const BatchGroup& g, const MlpWeights& W, int min_bucket,
                                 cudaStream_t s);

}  // namespace gk
