// C ABI of the gamma library: handle management, the host-side cell table
// (Algorithm A1 steps 2-3) and the launch sequence of one run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/gamma.h"
#include "gamma_internal.h"

using gk::Counters;
using gk::Problem;
using gk::TableEntry;

namespace {

thread_local std::string g_last_cuda;

int cuda_fail(cudaError_t e)
{
    g_last_cuda = cudaGetErrorString(e);
    // the runtime also keeps a failed call's error as its last error; clear
    // it (a sticky error stays), so that the launch checks of the next call
    // do not report it again
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GAMMA_ERR_OOM : GAMMA_ERR_CUDA;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// Keeps the caller's current device across a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Largest float not above x (keys must stay lower bounds after rounding).
float round_down(double x)
{
    float f = (float)x;
    if ((double)f > x) f = std::nextafterf(f, -INFINITY);
    return f;
}

double axis_gap(int i) { return i >= 0 ? (double)i : (double)(-i - 1); }

}  // namespace

struct BatchState;
void free_batch(BatchState* b);

// Reference and evaluation on different grids: the launch description and
// its cell table (device).
struct GridState {
    gk::GridProblem G{};
    TableEntry* table_dev = nullptr;
    unsigned* walk_list = nullptr;     // voxels the warp-evaluated walk leaves to k_grid_walk
};

// Evaluation-dose z slabs of a host-buffer run: the shell starts on a slab
// while the next ones are still being copied.
constexpr int kPipeChunks = gk::kShellSlots;
// Queued voxels one run (or one batch group) seeds at most with an attached
// model: the network's row buffers hold this many rows (784 bytes each);
// further voxels past the cost gate are walked without a seed.
constexpr unsigned kSeedRowsMax = 1u << 19;

struct gamma_ctx {
    BatchState* batch = nullptr;      // non-null for batch handles
    GridState* grids = nullptr;       // non-null for handles over two different grids
    int graph = 1;                    // batch: capture and replay a CUDA graph
    int device = 0;
    int ndim = 3;
    int64_t nz = 1, ny = 1, nx = 1, nvox = 0;
    double h[3] = {1, 1, 1};          // hx, hy, hz in mm
    gamma_criteria crit{};
    const float* ref = nullptr;
    const float* ev = nullptr;
    float* own_ref = nullptr;
    float* own_ev = nullptr;
    float* own_out = nullptr;
    // cell table
    std::vector<TableEntry> table;
    TableEntry* table_dev = nullptr;
    float key0_far2[8] = {};
    double r_cover = 0;
    int64_t table_cap = 1 << 17;
    // scratch
    Counters* ctr = nullptr;
    unsigned* tail_raw = nullptr;
    unsigned char* tail_bucket = nullptr;
    unsigned* tail_sorted = nullptr;
    unsigned tail_cap = 0;
    // tile-staged walk: queue bit masks per shell tile, tiles with queued voxels
    unsigned* tile_mask = nullptr;
    unsigned* tile_list = nullptr;
    unsigned char* tile_bkt = nullptr;
    unsigned* tile_sorted = nullptr;
    // row-staged walk: one item per shell warp row with queued voxels
    unsigned long long* row_items = nullptr;
    unsigned char* row_bkt = nullptr;
    unsigned long long* row_sorted = nullptr;
    // warp-evaluated walk: voxels left to its finishing pass (tail_cap entries)
    unsigned* fix_list = nullptr;
    int group_bucket = 9;             // ... queued voxels of this cost bucket and above walk 4 lanes each
                                      //     (< 0: the walk chooses the parts from the queue)
    int group_auto_pct = 100;         // ... with this slack (percent)
    int group8_bucket = 32;           // ... and of this one and above 8 lanes each (32: none)
    int group32_bucket = 32;          // ... and of this one and above 32 lanes each (32: none)
    int walk = 3;                     // 0: voxel queue walk (k_tail); 1: tile-staged (k_walk);
                                      // 2: row-staged (k_walk_rows); 3: voxel queue walk with
                                      // the warp evaluating surviving cells together (k_tail_cq)
    // options
    int lanes = gk::kDefaultLanesPerVoxel;
    double tau = 1e-6;
    int stats = 0;
    int sort_tail = 1;
    int timing = 0;
    int shell_minblocks = gk::kDefaultShellBlocksPerSm;
    int tail_minblocks = gk::kDefaultTailBlocksPerSm;
    int pipeline = 8;        // gamma_run_host: z slabs of the overlapped path (0: run in order)
    int design = 0;          // 0: two-phase search; 1 / 2: the paper's A2 with / without DD sort
    int face_eval = 0;       // design 1 / 2: 0 closed-form faces, 1 Ju's recursion
    gk::PaperScratch paper;
    gamma_model model = nullptr;      // attached proposal network (may be null)
    unsigned* seed_list = nullptr;    // with a model: queue items past the cost gate (tail_cap)
    __nv_bfloat16* seed_X = nullptr;  // with a model: network input rows (seed_cap x 384)
    float* seed_Y = nullptr;          // with a model: network output rows (seed_cap x 4)
    unsigned seed_cap = 0;
    int seed_min_bucket = 13;         // cost gate of the seeding pass (bucket of >= 64 cells)
    bool own_model = false;
    // per-phase events: 0 start, 1 after h2d, 2 after prepare, 3 after shell,
    // 4 after order, 5 after tail, 6 after d2h
    cudaEvent_t tev[7] = {};
    bool ev_h2d = false;     // the last run copied inputs from the host
    // host-buffer pipeline (gamma_run_host): compute and copy-out streams and
    // the events that order them against the caller's stream
    cudaStream_t pipe_s[2] = {};
    cudaEvent_t pipe_ev[7] = {};
    cudaEvent_t slab_ev[kPipeChunks] = {};
    unsigned* slab_flags = nullptr;   // device, kPipeChunks: last run whose slab k landed
    unsigned epoch = 0;               // number of the current overlapped run
    cudaEvent_t tev_out = nullptr;    // timing: end of the overlapped map copy-out
    int overlapped = 0;               // last run: 0 in order, 1 overlapped, 2 overlapped + slab gate
    // graph replay of single-pair gamma_run (option "graph"): captured once the
    // same output has been run twice with no option or input change between
    cudaStream_t sg_cap = nullptr;
    cudaGraph_t sg_graph = nullptr;
    cudaGraphExec_t sg_exec = nullptr;
    float* sg_out = nullptr;          // output the captured graph writes
    float* sg_seen = nullptr;         // output of the last direct run
    bool sg_dirty = true;             // options or inputs changed since that run
    Counters* host_ctr = nullptr;     // page-locked, mapped: counters an overlapped run leaves
    Counters* host_ctr_dev = nullptr; // its device address
    int drop_slab_flag = 0;           // test hook: k + 1 leaves slab k's flag unwritten
    // state
    cudaStream_t last_stream = nullptr;
    bool ran = false;
};

namespace {

// Algorithm A1 steps 2-3 for the cells of the Freudenthal triangulation: every
// lower-corner offset c whose cell can hold faces for some voxel, keyed by the
// distance from the reference voxel to the closed cell box [c, c + 1] divided
// by the DTA (for the key-0 cells: to their faces off the voxel), sorted
// ascending (ties by z, y, x), cut to `cap` entries.
int build_table(gamma_ctx* h)
{
    const double dta = h->crit.dta_mm;
    const double hn[3] = {h->h[0] / dta, h->h[1] / dta, h->h[2] / dta};
    const int nd = h->ndim;
    const int64_t n[3] = {h->nx, h->ny, h->nz};
    const int64_t cap = h->table_cap;
    if (cap < (1 << nd)) return GAMMA_ERR_INVALID_ARG;
    // radius from a ball-volume estimate of about 2 * cap cells
    double cellvol = hn[0] * hn[1] * (nd == 3 ? hn[2] : 1.0);
    double R = nd == 3 ? std::cbrt(2.0 * (double)cap * cellvol * 3.0 / (4.0 * M_PI))
                       : std::sqrt(2.0 * (double)cap * cellvol / M_PI);
    // the whole grid seen from any voxel
    double diag = 0;
    for (int a = 0; a < nd; ++a) diag += (double)(n[a] * n[a]) * hn[a] * hn[a];
    diag = std::sqrt(diag) + 1.0;
    bool clipped_by_grid = false;
    if (R > diag) { R = diag; clipped_by_grid = true; }
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    bool packing_limited = false;
    for (int a = 0; a < nd; ++a) {
        int64_t lim = (int64_t)std::ceil(R / hn[a]) + 1;
        lo[a] = std::max<int64_t>(-(n[a] - 1), -lim - 1);
        hi[a] = std::min<int64_t>(n[a] - 1, lim);
        if (lo[a] < -511) { lo[a] = -511; packing_limited = true; }
        if (hi[a] > 511) { hi[a] = 511; packing_limited = true; }
    }
    double far[8];
    gk::key0_far(hn, nd, far);
    for (int s = 0; s < 8; ++s) {
        const double f2 = far[s] * far[s];
        float r = (float)f2;
        if ((double)r > f2) r = std::nextafterf(r, -INFINITY);
        h->key0_far2[s] = r;
    }
    struct Tmp { double key; int x, y, z; };
    std::vector<Tmp> all;
    try {
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    double ax = axis_gap((int)x) * hn[0], ay = axis_gap((int)y) * hn[1];
                    double az = nd == 3 ? axis_gap((int)z) * hn[2] : 0.0;
                    double key = std::sqrt(ax * ax + ay * ay + az * az);
                    if (key == 0.0) key = far[(x & 1) | ((y & 1) << 1) | ((z & 1) << 2)];
                    if (key < R) all.push_back({key, (int)x, (int)y, (int)z});
                }
    } catch (const std::bad_alloc&) {
        return GAMMA_ERR_OOM;
    }
    std::sort(all.begin(), all.end(), [](const Tmp& a, const Tmp& b) {
        if (a.key != b.key) return a.key < b.key;
        if (a.z != b.z) return a.z < b.z;
        if (a.y != b.y) return a.y < b.y;
        return a.x < b.x;
    });
    double cover = clipped_by_grid ? INFINITY : R;
    if (packing_limited) {
        double m = INFINITY;
        for (int a = 0; a < nd; ++a) m = std::min(m, 510.0 * hn[a]);
        cover = std::min(cover, m);
    }
    size_t keep = all.size();
    if ((int64_t)keep > cap) {
        keep = (size_t)cap;
        cover = std::min(cover, all[keep].key);
    }
    h->table.resize(keep);
    for (size_t i = 0; i < keep; ++i) {
        h->table[i].off = gk::pack10(all[i].x, all[i].y, all[i].z);
        h->table[i].key = round_down(all[i].key);
    }
    h->r_cover = cover;
    if (h->table_dev) { cudaFree(h->table_dev); h->table_dev = nullptr; }
    if (keep) {
        CK(cudaMalloc(&h->table_dev, keep * sizeof(TableEntry)));
        CK(cudaMemcpy(h->table_dev, h->table.data(), keep * sizeof(TableEntry),
                      cudaMemcpyHostToDevice));
    }
    return GAMMA_OK;
}

Problem make_problem(const gamma_ctx* h, float* out)
{
    Problem P{};
    P.ref = h->ref;
    P.ev = h->ev;
    P.out = out;
    P.nvox = h->nvox;
    P.ndim = h->ndim;
    P.nx = (int)h->nx;
    P.ny = (int)h->ny;
    P.nz = (int)h->nz;
    const double dta = h->crit.dta_mm;
    double hn2[3];
    for (int a = 0; a < 3; ++a) {
        const double hn = h->h[a] / dta;
        P.hn[a] = (float)hn;
        hn2[a] = hn * hn;
        P.mt.hn2[a] = (float)hn2[a];
        P.mtd.hn2[a] = hn2[a];
    }
    P.mt.kappa[0] = 0.f;
    P.mtd.kappa[0] = 0.0;
    for (int A = 1; A < 8; ++A) {
        double s = 0;
        for (int a = 0; a < 3; ++a)
            if (A & (1 << a)) s += hn2[a];
        P.mt.kappa[A] = (float)(1.0 / s);
        P.mtd.kappa[A] = 1.0 / s;
    }
    P.dd_frac = h->crit.dd_frac;
    P.cutoff_frac = h->crit.cutoff_frac;
    P.dose_norm = h->crit.dose_norm;
    P.local = h->crit.mode == GAMMA_LOCAL;
    P.tau = (float)h->tau;
    P.stats = h->stats;
    P.table = h->table_dev;
    P.ntable = (int)h->table.size();
    gk::fill_bucket_keys(h->table.data(), P.ntable, P.bucket_key);
    for (int s = 0; s < 8; ++s) P.key0_far2[s] = h->key0_far2[s];
    P.r_cover = std::isinf(h->r_cover) ? INFINITY : round_down(h->r_cover);
    P.tail_cap = h->tail_cap;
    P.ctr = h->ctr;
    P.tail_raw = h->tail_raw;
    P.tail_bucket = h->tail_bucket;
    P.tail_sorted = h->tail_sorted;
    P.sort_tail = h->sort_tail;
    P.shell_minblocks = h->shell_minblocks;
    P.seed_list = h->seed_list;
    P.seed_X = h->seed_X;
    P.seed_Y = h->seed_Y;
    P.seed_cap = h->seed_cap;
    P.fix_list = h->fix_list;
    P.cq_group_bucket = h->group_bucket;
    P.cq_group8_bucket = h->group8_bucket;
    P.cq_group32_bucket = h->group32_bucket;
    P.cq_auto_scale = 0.01f * (float)h->group_auto_pct;
    if (h->walk == 1 && h->tile_mask) {
        P.tile_mask = h->tile_mask;
        P.tile_list = h->tile_list;
        P.tile_bkt = h->tile_bkt;
        P.tile_sorted = h->tile_sorted;
    }
    if (h->walk == 2 && h->row_items) {
        P.row_items = h->row_items;
        P.row_bkt = h->row_bkt;
        P.row_sorted = h->row_sorted;
    }
    return P;
}

void free_ctx(gamma_ctx* h)
{
    if (!h) return;
    if (h->batch) free_batch(h->batch);
    if (h->grids) {
        cudaFree(h->grids->table_dev);
        cudaFree(h->grids->walk_list);
        delete h->grids;
    }
    if (h->own_model) gamma_model_destroy(h->model);
    for (auto& e : h->tev)
        if (e) cudaEventDestroy(e);
    for (auto& e : h->pipe_ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : h->slab_ev)
        if (e) cudaEventDestroy(e);
    if (h->tev_out) cudaEventDestroy(h->tev_out);
    if (h->sg_exec) cudaGraphExecDestroy(h->sg_exec);
    if (h->sg_graph) cudaGraphDestroy(h->sg_graph);
    if (h->sg_cap) cudaStreamDestroy(h->sg_cap);
    if (h->host_ctr) cudaFreeHost(h->host_ctr);
    cudaFree(h->slab_flags);
    for (auto& st : h->pipe_s)
        if (st) cudaStreamDestroy(st);
    cudaFree(h->table_dev);
    cudaFree(h->ctr);
    cudaFree(h->tail_raw);
    cudaFree(h->tail_bucket);
    cudaFree(h->tail_sorted);
    cudaFree(h->tile_mask);
    cudaFree(h->tile_list);
    cudaFree(h->tile_bkt);
    cudaFree(h->tile_sorted);
    cudaFree(h->row_items);
    cudaFree(h->row_bkt);
    cudaFree(h->row_sorted);
    cudaFree(h->fix_list);
    cudaFree(h->seed_list);
    cudaFree(h->seed_X);
    cudaFree(h->seed_Y);
    cudaFree(h->own_ref);
    cudaFree(h->own_ev);
    cudaFree(h->own_out);
    cudaFree(h->paper.keys);
    cudaFree(h->paper.ids);
    cudaFree(h->paper.keys_alt);
    cudaFree(h->paper.ids_alt);
    cudaFree(h->paper.temp);
    delete h;
}

int check_criteria(const gamma_criteria* c)
{
    if (!c) return GAMMA_ERR_INVALID_ARG;
    if (!(c->dd_frac > 0.f) || !std::isfinite(c->dd_frac)) return GAMMA_ERR_INVALID_ARG;
    if (!(c->dta_mm > 0.f) || !std::isfinite(c->dta_mm)) return GAMMA_ERR_INVALID_ARG;
    if (c->mode != GAMMA_GLOBAL && c->mode != GAMMA_LOCAL) return GAMMA_ERR_INVALID_ARG;
    if (!std::isfinite(c->cutoff_frac) || !std::isfinite(c->dose_norm)) return GAMMA_ERR_INVALID_ARG;
    return GAMMA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Batched runs
// ---------------------------------------------------------------------------

struct BatchState {
    int n = 0;
    std::vector<gamma_ctx*> pairs;     // per-pair tables and scratch
    std::vector<float*> outs;
    std::vector<int> members[2];       // pair indices of group 0 (2D) and 1 (3D)
    Counters* ctrs = nullptr;          // [n], contiguous: one memset per run
    struct Group {
        gk::Problem* probs = nullptr;
        CUtensorMap* maps = nullptr;
        int* use_tma = nullptr;
        int* tile_start = nullptr;
        unsigned* item_start = nullptr;
        unsigned* items_v = nullptr;
        unsigned short* items_p = nullptr;
        unsigned* head = nullptr;          // walk, shell tiles, seed rows, seeding work,
                                           // warp-evaluated walk parts (3), its fix count
        float4* metric4 = nullptr;         // per pair: metric constants of the warp-evaluated walk
        unsigned* fix_v = nullptr;         // warp-evaluated walk: voxels for its finishing pass
        unsigned short* fix_p = nullptr;
        unsigned* seed_item = nullptr;     // with a model: (pair, item) rows past the gate
        unsigned short* seed_pair = nullptr;
        __nv_bfloat16* seed_X = nullptr;   // ... their network inputs and outputs
        float* seed_Y = nullptr;
        unsigned seed_cap = 0;
        gk::BatchDesc* desc = nullptr;
        gk::BatchGroup host{};
    } grp[2];
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool dirty = true;                 // device problems / graph out of date
};

namespace {

void free_group(BatchState::Group& g)
{
    cudaFree(g.probs);
    cudaFree(g.maps);
    cudaFree(g.use_tma);
    cudaFree(g.tile_start);
    cudaFree(g.item_start);
    cudaFree(g.items_v);
    cudaFree(g.items_p);
    cudaFree(g.head);
    cudaFree(g.fix_v);
    cudaFree(g.metric4);
    cudaFree(g.fix_p);
    cudaFree(g.seed_item);
    cudaFree(g.seed_pair);
    cudaFree(g.seed_X);
    cudaFree(g.seed_Y);
    cudaFree(g.desc);
    g = BatchState::Group{};
}

}  // namespace

void free_batch(BatchState* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (auto& g : b->grp) free_group(g);
    for (gamma_ctx* c : b->pairs) {
        if (c) c->ctr = nullptr;           // points into b->ctrs
        free_ctx(c);
    }
    cudaFree(b->ctrs);
    delete b;
}

namespace {

// (Re)build every pair's Problem with the batch handle's options and upload
// the per-group descriptors.
int batch_upload(gamma_ctx* h)
{
    BatchState* b = h->batch;
    for (int gi = 0; gi < 2; ++gi) {
        auto& G = b->grp[gi];
        const auto& mem = b->members[gi];
        const int np = (int)mem.size();
        if (np == 0) continue;
        std::vector<gk::Problem> probs(np);
        std::vector<CUtensorMap> maps(np);
        std::vector<int> use(np), tstart(np + 1, 0);
        long long maxv = 0;
        for (int k = 0; k < np; ++k) {
            gamma_ctx* c = b->pairs[mem[k]];
            c->tau = h->tau;
            c->stats = 0;
            c->sort_tail = 1;
            c->shell_minblocks = h->shell_minblocks;
            probs[k] = make_problem(c, b->outs[mem[k]]);
            std::memset(&maps[k], 0, sizeof(CUtensorMap));
            use[k] = gk::encode_tile_map(probs[k], &maps[k]) ? 1 : 0;
            const int tiles = gk::shell_tiles(probs[k]);
            if (tiles < 0) return GAMMA_ERR_SHAPE;
            if ((long long)tstart[k] + tiles > 0x3fffffffLL) return GAMMA_ERR_SHAPE;
            tstart[k + 1] = tstart[k] + tiles;
            maxv = std::max<long long>(maxv, c->nvox);
        }
        if (!G.probs) {
            CK(cudaMalloc(&G.probs, sizeof(gk::Problem) * np));
            CK(cudaMalloc(&G.maps, sizeof(CUtensorMap) * np));
            CK(cudaMalloc(&G.use_tma, sizeof(int) * np));
            CK(cudaMalloc(&G.tile_start, sizeof(int) * (np + 1)));
            CK(cudaMalloc(&G.item_start, sizeof(unsigned) * (gk::kNumBuckets * np + 4)));
            size_t cap = 0;
            for (int k = 0; k < np; ++k) cap += b->pairs[mem[k]]->tail_cap;
            CK(cudaMalloc(&G.items_v, sizeof(unsigned) * std::max<size_t>(cap, 1)));
            CK(cudaMalloc(&G.items_p, sizeof(unsigned short) * std::max<size_t>(cap, 1)));
            CK(cudaMalloc(&G.fix_v, sizeof(unsigned) * std::max<size_t>(cap, 1)));
            CK(cudaMalloc(&G.metric4, sizeof(float4) * 3 * np));
            CK(cudaMalloc(&G.fix_p, sizeof(unsigned short) * std::max<size_t>(cap, 1)));
            CK(cudaMalloc(&G.head, 12 * sizeof(unsigned)));
            CK(cudaMemset(G.head, 0, 12 * sizeof(unsigned)));
            CK(cudaMalloc(&G.desc, sizeof(gk::BatchDesc)));
        }
        if (h->model && !G.seed_item) {
            size_t cap = 0;
            for (int k = 0; k < np; ++k) cap += b->pairs[mem[k]]->tail_cap;
            G.seed_cap = (unsigned)std::max<size_t>(1, std::min<size_t>(cap, kSeedRowsMax));
            CK(cudaMalloc(&G.seed_item, sizeof(unsigned) * G.seed_cap));
            CK(cudaMalloc(&G.seed_pair, sizeof(unsigned short) * G.seed_cap));
            CK(cudaMalloc(&G.seed_X, sizeof(__nv_bfloat16) * gk::kInPad * (size_t)G.seed_cap));
            CK(cudaMalloc(&G.seed_Y, sizeof(float) * gk::kOut * (size_t)G.seed_cap));
        }
        CK(cudaMemcpy(G.probs, probs.data(), sizeof(gk::Problem) * np, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(G.maps, maps.data(), sizeof(CUtensorMap) * np, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(G.use_tma, use.data(), sizeof(int) * np, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(G.tile_start, tstart.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice));
        std::vector<float4> m4(3 * (size_t)np);
        for (int k = 0; k < np; ++k) {
            const gk::Metric& mt = probs[k].mt;
            m4[3 * k] = make_float4(mt.hn2[0], mt.hn2[1], mt.hn2[2], probs[k].tau);
            m4[3 * k + 1] = make_float4(mt.kappa[1], mt.kappa[2], mt.kappa[3], mt.kappa[4]);
            m4[3 * k + 2] = make_float4(mt.kappa[5], mt.kappa[6], mt.kappa[7], 0.f);
        }
        CK(cudaMemcpy(G.metric4, m4.data(), sizeof(float4) * m4.size(), cudaMemcpyHostToDevice));
        gk::BatchDesc d{};
        d.npairs = np;
        d.probs = G.probs;
        d.maps = G.maps;
        d.use_tma = G.use_tma;
        d.tile_start = G.tile_start;
        d.item_start = G.item_start;
        d.items_v = G.items_v;
        d.items_p = G.items_p;
        d.head = G.head;
        d.shell_next = G.head + 1;
        d.group_bucket = h->walk == 3 ? h->group_bucket : 0;
        d.group8_bucket = h->walk == 3 ? h->group8_bucket : 0;
        d.group32_bucket = h->walk == 3 ? h->group32_bucket : 0;
        d.auto_scale = 0.01f * (float)h->group_auto_pct;
        d.walk_lanes = (unsigned)(gk::device_sm_count() * std::min(4, std::max(1, h->tail_minblocks)) * 256);
        d.part_head = G.head + 4;
        d.metric4 = G.metric4;
        d.fix_v = G.fix_v;
        d.fix_p = G.fix_p;
        d.fix_count = G.head + 8;
        if (h->model) {
            d.seed_item = G.seed_item;
            d.seed_pair = G.seed_pair;
            d.seed_count = G.head + 2;
            d.seed_head = G.head + 3;
            d.seed_X = G.seed_X;
            d.seed_Y = G.seed_Y;
            d.seed_cap = G.seed_cap;
        }
        CK(cudaMemcpy(G.desc, &d, sizeof(d), cudaMemcpyHostToDevice));
        G.host.ndim = gi == 0 ? 2 : 3;
        G.host.npairs = np;
        G.host.max_nvox = maxv;
        G.host.total_tiles = tstart[np];
        G.host.desc = G.desc;
        G.host.shell_next = G.head + 1;
        G.host.seed_X = h->model ? G.seed_X : nullptr;
        G.host.seed_Y = h->model ? G.seed_Y : nullptr;
        G.host.seed_cap = h->model ? G.seed_cap : 0u;
        G.host.seed_count = G.head + 2;
        G.host.flags = &b->ctrs[mem[0]].flags;
    }
    return GAMMA_OK;
}

// The launch sequence of one batched run, on stream s.
int batch_enqueue(gamma_ctx* h, cudaStream_t s)
{
    BatchState* b = h->batch;
    const bool tm = h->timing != 0;
    if (tm) {
        CK(cudaEventRecord(h->tev[0], s));
        CK(cudaEventRecord(h->tev[1], s));
    }
    CK(cudaMemsetAsync(b->ctrs, 0, sizeof(Counters) * b->n, s));
    for (auto& G : b->grp) CK(gk::launch_batch_prepare(G.host, s));
    if (tm) CK(cudaEventRecord(h->tev[2], s));
    for (auto& G : b->grp) CK(gk::launch_batch_shell(G.host, h->shell_minblocks, s));
    if (h->model) {
        // learned seeding of every pair's queued voxels past the cost gate
        gk::MlpWeights W;
        gk::model_weights(h->model, &W);
        for (auto& G : b->grp) CK(gk::launch_batch_seeding(G.host, W, h->seed_min_bucket, s));
    }
    if (tm) CK(cudaEventRecord(h->tev[3], s));
    for (auto& G : b->grp) CK(gk::launch_batch_order(G.host, s));
    if (tm) CK(cudaEventRecord(h->tev[4], s));
    for (auto& G : b->grp) CK(gk::launch_batch_tail(G.host, h->walk, h->lanes, h->tail_minblocks, s));
    if (tm) {
        CK(cudaEventRecord(h->tev[5], s));
        CK(cudaEventRecord(h->tev[6], s));
    }
    return GAMMA_OK;
}

Counters sum_counters(const std::vector<Counters>& cs)
{
    Counters t;
    std::memset(&t, 0, sizeof(t));
    for (const Counters& c : cs) {
        t.n_eval += c.n_eval;
        t.n_pass += c.n_pass;
        t.cells_visited += c.cells_visited;
        t.cells_pruned += c.cells_pruned;
        t.cells_keyed += c.cells_keyed;
        t.lane_steps += c.lane_steps;
        t.flags |= c.flags;
        t.tail_count += c.tail_count;
        t.overflow_count += c.overflow_count;
        t.fp64_cells += c.fp64_cells;
        t.seeded += c.seeded;
        t.seed_improved += c.seed_improved;
        if (gk::fdec(c.rmax_enc) > gk::fdec(t.rmax_enc) || t.rmax_enc == 0) t.rmax_enc = c.rmax_enc;
    }
    return t;
}

}  // namespace

extern "C" {

int gamma_create(gamma_handle* out, const float* ref_dev, const float* eval_dev, int ndim,
                 const int64_t shape[3], const float spacing_mm[3], const gamma_criteria* crit)
{
    if (!out || !shape || !spacing_mm) return GAMMA_ERR_INVALID_ARG;
    *out = nullptr;
    if ((ref_dev == nullptr) != (eval_dev == nullptr)) return GAMMA_ERR_INVALID_ARG;
    if (int rc = check_criteria(crit)) return rc;
    if (ndim != 2 && ndim != 3) return GAMMA_ERR_SHAPE;
    const int64_t nz = ndim == 3 ? shape[0] : 1, ny = shape[1], nx = shape[2];
    if (ndim == 2 && shape[0] != 1) return GAMMA_ERR_SHAPE;
    if (nx < 2 || ny < 2 || (ndim == 3 && nz < 2)) return GAMMA_ERR_SHAPE;
    if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30)) return GAMMA_ERR_SHAPE;
    const int64_t nvox = nx * ny * nz;
    if (nvox >= (int64_t(1) << 31)) return GAMMA_ERR_SHAPE;
    for (int a = (ndim == 3 ? 0 : 1); a < 3; ++a)
        if (!(spacing_mm[a] > 0.f) || !std::isfinite(spacing_mm[a])) return GAMMA_ERR_INVALID_ARG;

    gamma_ctx* h = new (std::nothrow) gamma_ctx();
    if (!h) return GAMMA_ERR_OOM;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return GAMMA_ERR_CUDA; }
    h->ndim = ndim;
    h->nz = nz; h->ny = ny; h->nx = nx; h->nvox = nvox;
    h->h[0] = spacing_mm[2];
    h->h[1] = spacing_mm[1];
    h->h[2] = ndim == 3 ? spacing_mm[0] : 1.0;
    h->crit = *crit;
    h->ref = ref_dev;
    h->ev = eval_dev;
    int rc = GAMMA_OK;
    auto fail = [&](int code) { free_ctx(h); return code; };
    if ((rc = build_table(h)) != GAMMA_OK) return fail(rc);
    cudaError_t e;
    for (auto& te : h->tev)
        if ((e = cudaEventCreate(&te)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMalloc(&h->ctr, sizeof(Counters))) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaStreamCreateWithFlags(&h->sg_cap, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(cuda_fail(e));
    h->tail_cap = (unsigned)nvox;
    if ((e = cudaMalloc(&h->tail_raw, sizeof(unsigned) * nvox)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMalloc(&h->tail_sorted, sizeof(unsigned) * nvox)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMalloc(&h->tail_bucket, nvox)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMalloc(&h->fix_list, sizeof(unsigned) * nvox)) != cudaSuccess) return fail(cuda_fail(e));
    {
        Problem P0 = make_problem(h, nullptr);
        const int tiles = gk::block_tiles(P0);
        if (tiles < 0) return fail(GAMMA_ERR_SHAPE);
        const size_t nt = (size_t)std::max(tiles, 1);
        if ((e = cudaMalloc(&h->tile_mask, sizeof(unsigned) * 8 * nt)) != cudaSuccess ||
            (e = cudaMalloc(&h->tile_list, sizeof(unsigned) * nt)) != cudaSuccess ||
            (e = cudaMalloc(&h->tile_bkt, nt)) != cudaSuccess ||
            (e = cudaMalloc(&h->tile_sorted, sizeof(unsigned) * nt)) != cudaSuccess ||
            (e = cudaMalloc(&h->row_items, sizeof(unsigned long long) * 8 * nt)) != cudaSuccess ||
            (e = cudaMalloc(&h->row_bkt, 8 * nt)) != cudaSuccess ||
            (e = cudaMalloc(&h->row_sorted, sizeof(unsigned long long) * 8 * nt)) != cudaSuccess)
            return fail(cuda_fail(e));
    }
    if (!ref_dev) {
        if ((e = cudaMalloc(&h->own_ref, sizeof(float) * nvox)) != cudaSuccess) return fail(cuda_fail(e));
        if ((e = cudaMalloc(&h->own_ev, sizeof(float) * nvox)) != cudaSuccess) return fail(cuda_fail(e));
        if ((e = cudaMalloc(&h->own_out, sizeof(float) * nvox)) != cudaSuccess) return fail(cuda_fail(e));
        h->ref = h->own_ref;
        h->ev = h->own_ev;
    }
    *out = h;
    return GAMMA_OK;
}

// The nine cell tables of a two-grid handle (variants of gk::build_grid_table,
// each capped at `cap` entries), concatenated in one device array.
static int upload_grid_tables(gamma_ctx* h, long long cap)
{
    gk::GridProblem& G = h->grids->G;
    const double hn[3] = {G.eh[0], G.eh[1], G.eh[2]};
    std::vector<TableEntry> all, table;
    int off[9], len[9];
    float cov[9];
    for (int k = 0; k < 9; ++k) {
        double cover = 0;
        table.clear();
        if (int rc = gk::build_grid_table(G.ndim, hn, G.en, cap, k, table, cover)) return rc;
        off[k] = (int)all.size();
        len[k] = (int)table.size();
        cov[k] = std::isinf(cover) ? INFINITY : round_down(cover);
        all.insert(all.end(), table.begin(), table.end());
    }
    if (all.size() > (size_t)0x7fffffff) return GAMMA_ERR_TABLE_TOO_LARGE;
    TableEntry* dev = nullptr;
    CK(cudaMalloc(&dev, sizeof(TableEntry) * std::max<size_t>(all.size(), 1)));
    if (!all.empty()) {
        const cudaError_t e = cudaMemcpy(dev, all.data(), sizeof(TableEntry) * all.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(dev);
            return cuda_fail(e);
        }
    }
    cudaFree(h->grids->table_dev);
    h->grids->table_dev = dev;
    G.table = dev;
    for (int k = 0; k < 9; ++k) {
        G.toff[k] = off[k];
        G.tlen[k] = len[k];
        G.tcover[k] = cov[k];
    }
    return GAMMA_OK;
}

int gamma_create_grids(gamma_handle* out, const float* ref_dev, const float* eval_dev, int ndim,
                       const int64_t ref_shape[3], const float ref_spacing_mm[3],
                       const float ref_origin_mm[3], const int64_t eval_shape[3],
                       const float eval_spacing_mm[3], const float eval_origin_mm[3],
                       const gamma_criteria* crit)
{
    if (!out || !ref_dev || !eval_dev || !ref_shape || !ref_spacing_mm || !ref_origin_mm ||
        !eval_shape || !eval_spacing_mm || !eval_origin_mm)
        return GAMMA_ERR_INVALID_ARG;
    *out = nullptr;
    if (int rc = check_criteria(crit)) return rc;
    if (ndim != 2 && ndim != 3) return GAMMA_ERR_SHAPE;
    if (ndim == 2 && (ref_shape[0] != 1 || eval_shape[0] != 1)) return GAMMA_ERR_SHAPE;
    const int first = ndim == 3 ? 0 : 1;
    bool same = true;
    for (int a = first; a < 3; ++a) {
        if (ref_shape[a] < 1 || eval_shape[a] < 2) return GAMMA_ERR_SHAPE;
        if (ref_shape[a] > (1 << 30) || eval_shape[a] > (1 << 30)) return GAMMA_ERR_SHAPE;
        if (!(ref_spacing_mm[a] > 0.f) || !std::isfinite(ref_spacing_mm[a]) ||
            !(eval_spacing_mm[a] > 0.f) || !std::isfinite(eval_spacing_mm[a]) ||
            !std::isfinite(ref_origin_mm[a]) || !std::isfinite(eval_origin_mm[a]))
            return GAMMA_ERR_INVALID_ARG;
        same = same && ref_shape[a] == eval_shape[a] && ref_spacing_mm[a] == eval_spacing_mm[a] &&
               ref_origin_mm[a] == eval_origin_mm[a];
    }
    int64_t nref = 1, neval = 1;
    for (int a = first; a < 3; ++a) {
        nref *= ref_shape[a];
        neval *= eval_shape[a];
    }
    if (nref >= (int64_t(1) << 31) || neval >= (int64_t(1) << 31)) return GAMMA_ERR_SHAPE;
    if (same) return gamma_create(out, ref_dev, eval_dev, ndim, ref_shape, ref_spacing_mm, crit);

    gamma_ctx* h = new (std::nothrow) gamma_ctx();
    if (!h) return GAMMA_ERR_OOM;
    auto fail = [&](int code) { free_ctx(h); return code; };
    h->grids = new (std::nothrow) GridState();
    if (!h->grids) return fail(GAMMA_ERR_OOM);
    h->walk = 0;       // the lane walk: the warp-evaluated one measured slower on two grids
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(GAMMA_ERR_CUDA);
    h->ndim = ndim;
    h->nz = ndim == 3 ? ref_shape[0] : 1;
    h->ny = ref_shape[1];
    h->nx = ref_shape[2];
    h->nvox = nref;
    h->crit = *crit;
    h->ref = ref_dev;
    h->ev = eval_dev;
    gk::GridProblem& G = h->grids->G;
    const double dta = crit->dta_mm;
    G.ndim = ndim;
    G.nref = nref;
    G.neval = neval;
    for (int a = 0; a < 3; ++a) {
        const int src = 2 - a;                          // (z, y, x) -> (x, y, z)
        const bool used = a < ndim;
        G.rn[a] = used ? (int)ref_shape[src] : 1;
        G.en[a] = used ? (int)eval_shape[src] : 1;
        G.rh[a] = used ? ref_spacing_mm[src] / dta : 1.0;
        G.ro[a] = used ? ref_origin_mm[src] / dta : 0.0;
        G.eh[a] = used ? eval_spacing_mm[src] / dta : 1.0;
        G.eo[a] = used ? eval_origin_mm[src] / dta : 0.0;
        G.mt.hn2[a] = (float)(G.eh[a] * G.eh[a]);
        G.mtd.hn2[a] = G.eh[a] * G.eh[a];
    }
    G.mt.kappa[0] = 0.f;
    G.mtd.kappa[0] = 0.0;
    for (int A = 1; A < 8; ++A) {
        double s = 0;
        for (int a = 0; a < 3; ++a)
            if (A & (1 << a)) s += G.mtd.hn2[a];
        G.mt.kappa[A] = (float)(1.0 / s);
        G.mtd.kappa[A] = 1.0 / s;
    }
    G.dd_frac = crit->dd_frac;
    G.cutoff_frac = crit->cutoff_frac;
    G.dose_norm = crit->dose_norm;
    G.local = crit->mode == GAMMA_LOCAL;
    if (int rc = upload_grid_tables(h, h->table_cap)) return fail(rc);
    cudaError_t e;
    if ((e = cudaMalloc(&h->grids->walk_list, sizeof(unsigned) * (size_t)nref)) != cudaSuccess)
        return fail(cuda_fail(e));
    for (auto& te : h->tev)
        if ((e = cudaEventCreate(&te)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaMalloc(&h->ctr, sizeof(Counters))) != cudaSuccess) return fail(cuda_fail(e));
    *out = h;
    return GAMMA_OK;
}

int gamma_set_inputs(gamma_handle h, const float* ref_dev, const float* eval_dev)
{
    if (!h || !ref_dev || !eval_dev || h->own_ref) return GAMMA_ERR_INVALID_ARG;
    h->ref = ref_dev;
    h->ev = eval_dev;
    h->sg_dirty = true;
    return GAMMA_OK;
}

// Order and walk the queued voxels: tile by tile or row by row from staged
// halo boxes (k_walk, k_walk_rows) or voxel by voxel (k_tail, k_tail_cq).
// tm: record the "order" event between.
static int enqueue_walk(gamma_handle h, const Problem& P, cudaStream_t s, bool tm)
{
    if (P.row_items) {
        CK(gk::launch_order_rows(P, s));
        if (tm) CK(cudaEventRecord(h->tev[4], s));
        CK(gk::launch_walk_rows(P, h->tail_minblocks, s));
    } else if (P.tile_mask) {
        CK(gk::launch_order_tiles(P, s));
        if (tm) CK(cudaEventRecord(h->tev[4], s));
        CK(gk::launch_walk(P, h->tail_minblocks, s));
    } else {
        CK(gk::launch_order_tail(P, s));
        if (tm) CK(cudaEventRecord(h->tev[4], s));
        if (h->walk == 3) CK(gk::launch_tail_cq(P, h->tail_minblocks, s));
        else CK(gk::launch_tail(P, h->lanes, h->tail_minblocks, s));
    }
    return GAMMA_OK;
}

// The search of one run with no timing events, model or paper design: what
// the graph replay captures.
static int enqueue_search(gamma_handle h, const Problem& P, cudaStream_t s)
{
    CK(cudaMemsetAsync(h->ctr, 0, sizeof(Counters), s));
    CK(gk::launch_prepare(P, s, 1));
    CK(gk::launch_shell(P, s));
    return enqueue_walk(h, P, s, false);
}

int gamma_run(gamma_handle h, float* gamma_out_dev, void* cuda_stream)
{
    if (!h || !gamma_out_dev) return GAMMA_ERR_INVALID_ARG;
    h->overlapped = 0;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool tm = h->timing != 0;
    if (h->grids) {
        gk::GridProblem G = h->grids->G;
        G.ref = h->ref;
        G.ev = h->ev;
        G.out = gamma_out_dev;
        G.ctr = h->ctr;
        G.tau = (float)h->tau;
        G.lanes = h->lanes;
        G.walk = h->walk;
        G.walk_list = h->grids->walk_list;
        G.from_list = 0;
        if (tm) {
            CK(cudaEventRecord(h->tev[0], s));
            CK(cudaEventRecord(h->tev[1], s));
            CK(cudaEventRecord(h->tev[2], s));
            CK(cudaEventRecord(h->tev[3], s));
            CK(cudaEventRecord(h->tev[4], s));
        }
        CK(cudaMemsetAsync(h->ctr, 0, sizeof(Counters), s));
        CK(gk::launch_grids(G, s));
        if (tm) {
            CK(cudaEventRecord(h->tev[5], s));
            CK(cudaEventRecord(h->tev[6], s));
        }
        h->last_stream = s;
        h->ran = true;
        return GAMMA_OK;
    }
    const Problem P = make_problem(h, gamma_out_dev);
    if (h->graph && h->sg_cap && !tm && h->design == 0 && !h->model) {
        if (h->sg_exec && (h->sg_dirty || h->sg_out != gamma_out_dev)) {
            cudaGraphExecDestroy(h->sg_exec);         // freed once a replay in flight ends
            cudaGraphDestroy(h->sg_graph);
            h->sg_exec = nullptr;
            h->sg_graph = nullptr;
        }
        if (!h->sg_exec && !h->sg_dirty && h->sg_seen == gamma_out_dev) {
            CK(cudaStreamBeginCapture(h->sg_cap, cudaStreamCaptureModeThreadLocal));
            const int rc = enqueue_search(h, P, h->sg_cap);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(h->sg_cap, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (ec != cudaSuccess) return cuda_fail(ec);
            h->sg_graph = g;
            CK(cudaGraphInstantiate(&h->sg_exec, h->sg_graph, 0));
            h->sg_out = gamma_out_dev;
        }
        if (h->sg_exec) {
            CK(cudaGraphLaunch(h->sg_exec, s));
            h->last_stream = s;
            h->ran = true;
            return GAMMA_OK;
        }
        h->sg_seen = gamma_out_dev;
        h->sg_dirty = false;
        if (int rc = enqueue_search(h, P, s)) return rc;
        h->last_stream = s;
        h->ran = true;
        return GAMMA_OK;
    }
    if (tm && !h->ev_h2d) {
        CK(cudaEventRecord(h->tev[0], s));
        CK(cudaEventRecord(h->tev[1], s));
    }
    CK(cudaMemsetAsync(h->ctr, 0, sizeof(Counters), s));
    // the search's shell checks the evaluation dose itself; the paper's design does not
    CK(gk::launch_prepare(P, s, h->design != 0 ? 3 : 1));
    if (tm) CK(cudaEventRecord(h->tev[2], s));
    if (h->design != 0) {
        // the paper's design: DD keys and sort ("shell" phase), then the walk ("tail")
        CK(gk::launch_paper(P, h->paper, h->design == 1, h->face_eval == 1, tm ? h->tev[3] : nullptr, s));
        if (tm) {
            CK(cudaEventRecord(h->tev[4], s));
            CK(cudaEventRecord(h->tev[5], s));
            if (!h->ev_h2d) CK(cudaEventRecord(h->tev[6], s));
        }
        h->last_stream = s;
        h->ran = true;
        return GAMMA_OK;
    }
    CK(gk::launch_shell(P, s));
    if (h->model) {
        gk::MlpWeights W;
        gk::model_weights(h->model, &W);
        CK(gk::launch_seeding(P, W, h->seed_min_bucket, s));
    }
    if (tm) CK(cudaEventRecord(h->tev[3], s));
    if (int rc = enqueue_walk(h, P, s, tm)) return rc;
    if (tm) {
        CK(cudaEventRecord(h->tev[5], s));
        if (!h->ev_h2d) CK(cudaEventRecord(h->tev[6], s));
    }
    h->last_stream = s;
    h->ran = true;
    return GAMMA_OK;
}

namespace {

// Device address of a page-locked, mapped host buffer of `bytes` bytes, or
// null when either end of it is not such memory.
void* mapped_host(const void* p, size_t bytes)
{
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        cudaPointerGetAttributes(&b, (const char*)p + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer ||
        (const char*)b.devicePointer != (const char*)a.devicePointer + bytes - 1)
        return nullptr;
    return a.devicePointer;
}

// Stream write of a 32-bit value into device memory, ordered after the
// stream's earlier work with a memory fence (driver entry point; null when
// the driver does not offer it).
using WriteValueFn = CUresult (*)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
WriteValueFn write_value_fn()
{
    static WriteValueFn fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (WriteValueFn)p;
    }
    return fn;
}

// Host-buffer run with the copies overlapped.  The reference dose is copied
// first (the caller has queued it) and its norm taken on the compute stream
// while the evaluation dose follows in z slabs on the same copy stream.  The
// shell is one launch that starts once the norm is known: once a slab's copy
// has completed, a stream write on a second stream raises that slab's flag,
// and each tile waits (bounded) for the slabs its box reads.  The map is
// copied out while the queued voxels are searched, and their final values are
// then written into the host map directly, with the run's counters.  Without
// TMA tile loads or the stream write, the shell waits for the whole dose.
int run_host_pipelined(gamma_handle h, const float* eval_host, float* gamma_out_host,
                       float* out_mapped, cudaStream_t s)
{
    for (auto& e : h->slab_ev)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (!h->host_ctr) {
        CK(cudaHostAlloc(&h->host_ctr, sizeof(Counters), cudaHostAllocMapped));
        CK(cudaHostGetDevicePointer((void**)&h->host_ctr_dev, h->host_ctr, 0));
    }
    if (!h->slab_flags) {
        CK(cudaMalloc(&h->slab_flags, sizeof(unsigned) * kPipeChunks));
        CK(cudaMemset(h->slab_flags, 0, sizeof(unsigned) * kPipeChunks));
    }
    const bool tm = h->timing != 0;
    if (tm && !h->tev_out) CK(cudaEventCreate(&h->tev_out));
    cudaStream_t c = h->pipe_s[0], o = h->pipe_s[1];
    // start, reference in, evaluation in (s / o), shell done, map out, done
    cudaEvent_t* E = h->pipe_ev;
    const Problem P = make_problem(h, h->own_out);
    int per_layer = 0, layers = 0, depth = 0;
    gk::shell_layers(P, &per_layer, &layers, &depth);
    WriteValueFn wv = write_value_fn();
    bool gated = h->pipeline > 1 && P.ndim == 3 && layers > 1 && wv && gk::shell_gate_ok(P);
    const int want = gated ? std::min(h->pipeline, layers) : 1;
    const int slab_layers = (layers + want - 1) / want;
    const int64_t slab_depth = (int64_t)slab_layers * depth;           // voxel slices per slab
    const int K = (int)((h->nz + slab_depth - 1) / slab_depth);
    const size_t slice = sizeof(float) * (size_t)h->nx * (size_t)h->ny;
    const size_t bytes = sizeof(float) * (size_t)h->nvox;
    const unsigned epoch = ++h->epoch == 0 ? ++h->epoch : h->epoch;    // 0 is the flags' initial value

    // the caller has already recorded E[0] (earlier work on s) and queued the
    // reference dose's copy after it
    CK(cudaStreamWaitEvent(c, E[0], 0));
    CK(cudaStreamWaitEvent(o, E[0], 0));
    CK(cudaMemsetAsync(h->ctr, 0, sizeof(Counters), c));
    CK(cudaEventRecord(E[1], s));
    CK(cudaStreamWaitEvent(c, E[1], 0));
    CK(gk::launch_prepare(P, c, 1));
    // slabs back to back on s; each slab's flag is written on o once the
    // slab's event has fired, so the copies see no fence between them
    for (int k = 0; k < K; ++k) {
        const int64_t za = k * slab_depth, zb = std::min<int64_t>(za + slab_depth, h->nz);
        const int64_t off = za * h->nx * h->ny;
        CK(cudaMemcpyAsync(h->own_ev + off, eval_host + off, slice * (size_t)(zb - za),
                           cudaMemcpyHostToDevice, s));
        if (gated) {
            CK(cudaEventRecord(h->slab_ev[k], s));
            CK(cudaStreamWaitEvent(o, h->slab_ev[k], 0));
            if (h->drop_slab_flag != k + 1 &&
                wv(o, (CUdeviceptr)(h->slab_flags + k), epoch, 0) != CUDA_SUCCESS)
                gated = false;       // not offered here: the shell waits for the whole dose
        }
    }
    CK(cudaEventRecord(E[2], s));
    CK(cudaEventRecord(E[3], o));
    if (tm) CK(cudaEventRecord(h->tev[1], s));
    if (tm) CK(cudaEventRecord(h->tev[2], c));
    const int tiles = gk::shell_tiles(P);
    if (gated) {
        CK(gk::launch_shell_range(P, 0, tiles, 0, gk::SlabGate{h->slab_flags, epoch, (int)slab_depth}, c));
        CK(cudaStreamWaitEvent(c, E[2], 0));
        CK(cudaStreamWaitEvent(c, E[3], 0));
    } else {
        CK(cudaStreamWaitEvent(c, E[2], 0));
        CK(cudaStreamWaitEvent(c, E[3], 0));
        CK(gk::launch_shell_range(P, 0, tiles, 0, gk::SlabGate{nullptr, 0u, 0}, c));
    }
    if (tm) CK(cudaEventRecord(h->tev[3], c));
    CK(cudaEventRecord(E[4], c));
    CK(cudaStreamWaitEvent(o, E[4], 0));
    CK(cudaMemcpyAsync(gamma_out_host, h->own_out, bytes, cudaMemcpyDeviceToHost, o));
    if (tm) CK(cudaEventRecord(h->tev_out, o));
    CK(cudaEventRecord(E[5], o));
    if (int rc = enqueue_walk(h, P, c, tm)) return rc;
    if (tm) CK(cudaEventRecord(h->tev[5], c));
    CK(cudaStreamWaitEvent(c, E[5], 0));
    CK(gk::launch_patch_host(P, out_mapped, h->host_ctr_dev, c));
    if (tm) CK(cudaEventRecord(h->tev[6], c));
    CK(cudaEventRecord(E[6], c));
    CK(cudaStreamWaitEvent(s, E[6], 0));
    h->last_stream = s;
    h->ran = true;
    h->overlapped = gated ? 2 : 1;
    return GAMMA_OK;
}

}  // namespace

int gamma_run_host(gamma_handle h, const float* ref_host, const float* eval_host,
                   float* gamma_out_host, void* cuda_stream)
{
    if (!h || !ref_host || !eval_host || !gamma_out_host || !h->own_ref) return GAMMA_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t bytes = sizeof(float) * (size_t)h->nvox;
    const bool tm = h->timing != 0;
    // both paths start with the reference dose: queue it before choosing one;
    // E[0] marks the work already on s, which the overlapped path's own
    // streams wait for (not for this copy)
    if (tm) CK(cudaEventRecord(h->tev[0], s));
    const bool may_overlap = !h->grids && !h->batch && h->design == 0 && !h->model && h->pipeline;
    if (may_overlap) {
        for (auto& st : h->pipe_s)
            if (!st) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        for (auto& e : h->pipe_ev)
            if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        CK(cudaEventRecord(h->pipe_ev[0], s));
    }
    CK(cudaMemcpyAsync(h->own_ref, ref_host, bytes, cudaMemcpyHostToDevice, s));
    {
        float* out_mapped = nullptr;
        if (may_overlap && mapped_host(ref_host, bytes) && mapped_host(eval_host, bytes) &&
            (out_mapped = (float*)mapped_host(gamma_out_host, bytes)) != nullptr)
            return run_host_pipelined(h, eval_host, gamma_out_host, out_mapped, s);
    }
    CK(cudaMemcpyAsync(h->own_ev, eval_host, bytes, cudaMemcpyHostToDevice, s));
    if (tm) CK(cudaEventRecord(h->tev[1], s));
    h->ev_h2d = true;
    int rc = gamma_run(h, h->own_out, cuda_stream);
    h->ev_h2d = false;
    if (rc) return rc;
    CK(cudaMemcpyAsync(gamma_out_host, h->own_out, bytes, cudaMemcpyDeviceToHost, s));
    if (tm) CK(cudaEventRecord(h->tev[6], s));
    return GAMMA_OK;
}

static int read_counters(gamma_handle h, Counters* c, int pair = -1)
{
    if (!h->ran) return GAMMA_ERR_NOT_RUN;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    CK(cudaStreamSynchronize(h->last_stream));
    if (!h->batch && h->overlapped) {            // the final patch left them in host memory
        std::memcpy(c, h->host_ctr, sizeof(Counters));
        return GAMMA_OK;
    }
    if (!h->batch) {
        CK(cudaMemcpy(c, h->ctr, sizeof(Counters), cudaMemcpyDeviceToHost));
        return GAMMA_OK;
    }
    std::vector<Counters> cs(h->batch->n);
    CK(cudaMemcpy(cs.data(), h->batch->ctrs, sizeof(Counters) * cs.size(), cudaMemcpyDeviceToHost));
    *c = pair >= 0 ? cs[pair] : sum_counters(cs);
    return GAMMA_OK;
}

// Global criteria whose run found no positive dose norm (no norm given and
// no positive reference dose) evaluated no voxel (the kernels' cutoff).
static bool missing_norm(const gamma_criteria& crit, const Counters& c)
{
    return crit.mode == GAMMA_GLOBAL && !(crit.dose_norm > 0.f) && !(gk::fdec(c.dnorm_enc) > 0.f);
}

int gamma_pass_rate(gamma_handle h, double* rate, int64_t* n_eval, int64_t* n_pass)
{
    if (!h) return GAMMA_ERR_INVALID_ARG;
    Counters c;
    if (int rc = read_counters(h, &c)) return rc;
    if (c.flags & gk::kFlagNonFinite) return GAMMA_ERR_NAN_INPUT;
    if (c.flags & gk::kFlagTimeout) return GAMMA_ERR_TIMEOUT;
    if (c.flags & gk::kFlagTailFull) return GAMMA_ERR_QUEUE_FULL;
    if (!h->batch && missing_norm(h->crit, c)) return GAMMA_ERR_DOSE_NORM;
    for (int k = 0; h->batch && k < h->batch->n; ++k) {
        Counters ck;
        if (int rc = read_counters(h, &ck, k)) return rc;
        if (missing_norm(h->batch->pairs[k]->crit, ck)) return GAMMA_ERR_DOSE_NORM;
    }
    if (n_eval) *n_eval = (int64_t)c.n_eval;
    if (n_pass) *n_pass = (int64_t)c.n_pass;
    if (rate) *rate = c.n_eval ? (double)c.n_pass / (double)c.n_eval : 0.0;
    return GAMMA_OK;
}

int gamma_get_stats(gamma_handle h, gamma_stats* out)
{
    if (!h || !out) return GAMMA_ERR_INVALID_ARG;
    Counters c;
    if (int rc = read_counters(h, &c)) return rc;
    std::memset(out, 0, sizeof(*out));
    if (h->batch) {
        out->n_voxels = 0;
        for (gamma_ctx* c2 : h->batch->pairs) out->n_voxels += c2->nvox;
    } else {
        out->n_voxels = h->nvox;
    }
    out->n_eval = (int64_t)c.n_eval;
    out->n_pass = (int64_t)c.n_pass;
    out->tail_voxels = (int64_t)c.tail_count;
    out->overflow_voxels = (int64_t)c.overflow_count;
    out->fp64_cells = (int64_t)c.fp64_cells;
    out->seeded = (int64_t)c.seeded;
    out->seed_improved = (int64_t)c.seed_improved;
    out->cells_keyed = (int64_t)c.cells_keyed;
    out->cells_visited = (int64_t)c.cells_visited;
    out->cells_pruned = (int64_t)c.cells_pruned;
    out->lane_slot_steps = (int64_t)c.lane_steps;
    out->d_norm = h->crit.dose_norm > 0 ? (double)h->crit.dose_norm : (double)gk::fdec(c.dnorm_enc);
    out->r_max = (double)gk::fdec(c.rmax_enc);
    out->table_entries = (int64_t)h->table.size();
    out->table_radius = h->r_cover;
    out->flags = c.flags;
    return GAMMA_OK;
}

int gamma_get_timings(gamma_handle h, gamma_timings* out)
{
    if (!h || !out) return GAMMA_ERR_INVALID_ARG;
    if (!h->ran) return GAMMA_ERR_NOT_RUN;
    if (!h->timing) return GAMMA_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    CK(cudaStreamSynchronize(h->last_stream));
    out->overlapped = h->overlapped;
    if (h->overlapped) {             // phase end times from the start of the run
        float* f[6] = {&out->h2d_ms, &out->prepare_ms, &out->shell_ms, &out->order_ms,
                       &out->tail_ms, &out->total_ms};
        for (int i = 0; i < 6; ++i) CK(cudaEventElapsedTime(f[i], h->tev[0], h->tev[i + 1]));
        CK(cudaEventElapsedTime(&out->d2h_ms, h->tev[0], h->tev_out));
        return GAMMA_OK;
    }
    float t[6];
    for (int i = 0; i < 6; ++i) CK(cudaEventElapsedTime(&t[i], h->tev[i], h->tev[i + 1]));
    out->h2d_ms = t[0];
    out->prepare_ms = t[1];
    out->shell_ms = t[2];
    out->order_ms = t[3];
    out->tail_ms = t[4];
    out->d2h_ms = t[5];
    CK(cudaEventElapsedTime(&out->total_ms, h->tev[0], h->tev[6]));
    return GAMMA_OK;
}

int gamma_get_option(gamma_handle h, const char* key, int64_t* value)
{
    if (!h || !key || !value) return GAMMA_ERR_INVALID_ARG;
    const struct { const char* k; int v; } opts[] = {
        {"lanes_per_voxel", h->lanes}, {"shell_blocks_per_sm", h->shell_minblocks},
        {"tail_blocks_per_sm", h->tail_minblocks}, {"walk", h->walk}, {"group_bucket", h->group_bucket},
        {"group8_bucket", h->group8_bucket}, {"group32_bucket", h->group32_bucket},
        {"group_auto_pct", h->group_auto_pct}};
    for (const auto& o : opts)
        if (!std::strcmp(key, o.k)) {
            *value = o.v;
            return GAMMA_OK;
        }
    return GAMMA_ERR_INVALID_ARG;
}

int gamma_set_option(gamma_handle h, const char* key, int64_t value)
{
    if (!h || !key) return GAMMA_ERR_INVALID_ARG;
    h->sg_dirty = true;
    if (h->grids && !std::strcmp(key, "table_cap")) {
        // every cell next to the voxel's own (3^n of them) must be in the table
        if (value < 27 || value > (int64_t(1) << 26)) return GAMMA_ERR_INVALID_ARG;
        DeviceGuard dg(h->device);
        if (!dg.ok) return GAMMA_ERR_CUDA;
        if (h->ran) { CK(cudaStreamSynchronize(h->last_stream)); }
        if (int rc = upload_grid_tables(h, value)) return rc;
        h->table_cap = value;
        return GAMMA_OK;
    }
    if (h->grids && std::strcmp(key, "timing") && std::strcmp(key, "fp64_tau_exp10") &&
        std::strcmp(key, "lanes_per_voxel") && std::strcmp(key, "walk"))
        return GAMMA_ERR_INVALID_ARG;                   // the other options tune the coincident-grid search
    if (h->grids && !std::strcmp(key, "walk")) {
        if (value != 0 && value != 3) return GAMMA_ERR_INVALID_ARG;   // lane walk or warp-evaluated
        h->walk = (int)value;
        return GAMMA_OK;
    }
    if (h->batch) {
        h->batch->dirty = true;
        if (!std::strcmp(key, "graph")) {
            if (value != 0 && value != 1) return GAMMA_ERR_INVALID_ARG;
            h->graph = (int)value;
            return GAMMA_OK;
        }
        if (!std::strcmp(key, "table_cap")) {
            for (gamma_ctx* c : h->batch->pairs)
                if (int rc = gamma_set_option(c, key, value)) return rc;
            return GAMMA_OK;
        }
        if (!std::strcmp(key, "sort_tail") || !std::strcmp(key, "stats"))
            return value == 0 || value == 1 ? GAMMA_OK : GAMMA_ERR_INVALID_ARG;  // fixed in batches
    }
    if (!std::strcmp(key, "graph")) {                  // single-pair handles
        if (value != 0 && value != 1) return GAMMA_ERR_INVALID_ARG;
        h->graph = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "walk")) {
        // batch handles walk voxel by voxel: with (3) or without (0) the warp evaluation
        if (value < 0 || value > 3 || (h->batch && value != 0 && value != 3)) return GAMMA_ERR_INVALID_ARG;
        h->walk = (int)value;
        if (h->batch) h->batch->dirty = true;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "group_auto_pct")) {
        if (value < 1 || value > 100000) return GAMMA_ERR_INVALID_ARG;
        h->group_auto_pct = (int)value;
        if (h->batch) h->batch->dirty = true;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "group_bucket") || !std::strcmp(key, "group8_bucket") ||
        !std::strcmp(key, "group32_bucket")) {
        if (value < (key[5] == '_' ? -1 : 0) || value > gk::kNumBuckets) return GAMMA_ERR_INVALID_ARG;
        (key[5] == '8' ? h->group8_bucket : key[5] == '3' ? h->group32_bucket : h->group_bucket) = (int)value;
        if (h->batch) h->batch->dirty = true;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "lanes_per_voxel")) {
        if (value != 2 && value != 4 && value != 8 && value != 16 && value != 32) return GAMMA_ERR_INVALID_ARG;
        h->lanes = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "table_cap")) {
        if (value < 8 || value > (int64_t(1) << 26)) return GAMMA_ERR_INVALID_ARG;
        DeviceGuard dg(h->device);
        if (!dg.ok) return GAMMA_ERR_CUDA;
        if (h->ran) { CK(cudaStreamSynchronize(h->last_stream)); }
        h->table_cap = value;
        return build_table(h);
    }
    if (!std::strcmp(key, "fp64_tau_exp10")) {
        if (value > 30) return GAMMA_ERR_INVALID_ARG;
        h->tau = value <= 0 ? 0.0 : std::pow(10.0, -(double)value);
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "stats")) {
        if (value != 0 && value != 1) return GAMMA_ERR_INVALID_ARG;
        h->stats = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "design")) {
        if (h->batch || value < 0 || value > 3) return GAMMA_ERR_INVALID_ARG;
        if (value != 0 && !h->paper.keys) {
            DeviceGuard dg(h->device);
            if (!dg.ok) return GAMMA_ERR_CUDA;
            if (h->ran) { CK(cudaStreamSynchronize(h->last_stream)); }
            const size_t n = (size_t)h->nvox;
            gk::PaperScratch& w = h->paper;
            w.temp_bytes = gk::paper_sort_bytes(h->nvox);
            CK(cudaMalloc(&w.keys, sizeof(unsigned) * n));
            CK(cudaMalloc(&w.ids, sizeof(unsigned) * n));
            CK(cudaMalloc(&w.keys_alt, sizeof(unsigned) * n));
            CK(cudaMalloc(&w.ids_alt, sizeof(unsigned) * n));
            CK(cudaMalloc(&w.temp, std::max<size_t>(w.temp_bytes, 16)));
        }
        h->design = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "pipeline")) {
        if (h->batch || value < 0 || value > kPipeChunks) return GAMMA_ERR_INVALID_ARG;
        h->pipeline = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "drop_slab_flag")) {
        if (h->batch || value < 0 || value > kPipeChunks) return GAMMA_ERR_INVALID_ARG;
        h->drop_slab_flag = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "face_eval")) {
        if (h->batch || value < 0 || value > 1) return GAMMA_ERR_INVALID_ARG;
        h->face_eval = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "seed_min_bucket")) {
        if (value < 0 || value >= gk::kNumBuckets) return GAMMA_ERR_INVALID_ARG;
        h->seed_min_bucket = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "tail_blocks_per_sm")) {
        if (value < 1 || value > 4) return GAMMA_ERR_INVALID_ARG;
        h->tail_minblocks = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "shell_blocks_per_sm")) {
        if (value < 1 || value > 4) return GAMMA_ERR_INVALID_ARG;
        h->shell_minblocks = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "timing")) {
        if (value != 0 && value != 1) return GAMMA_ERR_INVALID_ARG;
        h->timing = (int)value;
        return GAMMA_OK;
    }
    if (!std::strcmp(key, "sort_tail")) {
        if (value != 0 && value != 1) return GAMMA_ERR_INVALID_ARG;
        h->sort_tail = (int)value;
        return GAMMA_OK;
    }
    return GAMMA_ERR_INVALID_ARG;
}

void gamma_destroy(gamma_handle h)
{
    if (!h) return;
    DeviceGuard dg(h->device);
    if (h->ran) cudaStreamSynchronize(h->last_stream);
    free_ctx(h);
}

int gamma_batch_create(gamma_handle* out, int n_pairs, const gamma_pair_desc* pairs)
{
    if (!out || n_pairs <= 0 || n_pairs > 65535 || !pairs) return GAMMA_ERR_INVALID_ARG;
    *out = nullptr;
    gamma_ctx* h = new (std::nothrow) gamma_ctx();
    if (!h) return GAMMA_ERR_OOM;
    h->batch = new (std::nothrow) BatchState();
    if (!h->batch) { delete h; return GAMMA_ERR_OOM; }
    BatchState* b = h->batch;
    auto fail = [&](int code) { free_ctx(h); return code; };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(GAMMA_ERR_CUDA);
    cudaError_t e;
    for (auto& te : h->tev)
        if ((e = cudaEventCreate(&te)) != cudaSuccess) return fail(cuda_fail(e));
    b->n = n_pairs;
    b->pairs.assign(n_pairs, nullptr);
    b->outs.assign(n_pairs, nullptr);
    if ((e = cudaMalloc(&b->ctrs, sizeof(Counters) * n_pairs)) != cudaSuccess)
        return fail(cuda_fail(e));
    for (int i = 0; i < n_pairs; ++i) {
        const gamma_pair_desc& d = pairs[i];
        if (!d.ref_dev || !d.eval_dev || !d.gamma_out_dev) return fail(GAMMA_ERR_INVALID_ARG);
        gamma_ctx* c = nullptr;
        if (int rc = gamma_create(&c, d.ref_dev, d.eval_dev, d.ndim, d.shape, d.spacing_mm, &d.crit))
            return fail(rc);
        cudaFree(c->ctr);                        // counters live in one shared array
        c->ctr = b->ctrs + i;
        b->pairs[i] = c;
        b->outs[i] = d.gamma_out_dev;
        b->members[d.ndim == 2 ? 0 : 1].push_back(i);
    }
    if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(cuda_fail(e));
    if (int rc = batch_upload(h)) return fail(rc);
    b->dirty = false;
    *out = h;
    return GAMMA_OK;
}

int gamma_batch_run(gamma_handle h, void* cuda_stream)
{
    if (!h || !h->batch) return GAMMA_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    BatchState* b = h->batch;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (b->dirty) {
        if (h->ran) CK(cudaStreamSynchronize(h->last_stream));
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        if (int rc = batch_upload(h)) return rc;
        b->dirty = false;
    }
    if (h->graph && !h->timing) {            // phase events are recorded by direct launches
        if (!b->exec) {
            CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            const int rc = batch_enqueue(h, b->cap);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (ec != cudaSuccess) return cuda_fail(ec);
            b->graph = g;
            CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
        }
        CK(cudaGraphLaunch(b->exec, s));
    } else {
        if (int rc = batch_enqueue(h, s)) return rc;
    }
    h->last_stream = s;
    h->ran = true;
    for (gamma_ctx* c : b->pairs) {
        c->ran = true;
        c->last_stream = s;
    }
    return GAMMA_OK;
}

int gamma_batch_pass_rate(gamma_handle h, int pair, double* rate, int64_t* n_eval, int64_t* n_pass)
{
    if (!h || !h->batch || pair < 0 || pair >= h->batch->n) return GAMMA_ERR_INVALID_ARG;
    Counters c;
    if (int rc = read_counters(h, &c, pair)) return rc;
    if (c.flags & gk::kFlagNonFinite) return GAMMA_ERR_NAN_INPUT;
    if (c.flags & gk::kFlagTimeout) return GAMMA_ERR_TIMEOUT;
    if (c.flags & gk::kFlagTailFull) return GAMMA_ERR_QUEUE_FULL;
    if (missing_norm(h->batch->pairs[pair]->crit, c)) return GAMMA_ERR_DOSE_NORM;
    if (n_eval) *n_eval = (int64_t)c.n_eval;
    if (n_pass) *n_pass = (int64_t)c.n_pass;
    if (rate) *rate = c.n_eval ? (double)c.n_pass / (double)c.n_eval : 0.0;
    return GAMMA_OK;
}

int gamma_batch_get_stats(gamma_handle h, int pair, gamma_stats* out)
{
    if (!h || !h->batch || !out || pair < 0 || pair >= h->batch->n) return GAMMA_ERR_INVALID_ARG;
    gamma_ctx* c = h->batch->pairs[pair];
    Counters k;
    if (int rc = read_counters(h, &k, pair)) return rc;
    std::memset(out, 0, sizeof(*out));
    out->n_voxels = c->nvox;
    out->n_eval = (int64_t)k.n_eval;
    out->n_pass = (int64_t)k.n_pass;
    out->tail_voxels = (int64_t)k.tail_count;
    out->overflow_voxels = (int64_t)k.overflow_count;
    out->fp64_cells = (int64_t)k.fp64_cells;
    out->seeded = (int64_t)k.seeded;
    out->seed_improved = (int64_t)k.seed_improved;
    out->d_norm = c->crit.dose_norm > 0 ? (double)c->crit.dose_norm : (double)gk::fdec(k.dnorm_enc);
    out->r_max = (double)gk::fdec(k.rmax_enc);
    out->table_entries = (int64_t)c->table.size();
    out->table_radius = c->r_cover;
    out->flags = k.flags;
    return GAMMA_OK;
}

int gamma_autotune(gamma_handle h, float* gamma_out_dev, void* cuda_stream, int reps,
                   int64_t* lanes_per_voxel, int64_t* shell_blocks_per_sm,
                   int64_t* tail_blocks_per_sm, float* best_ms)
{
    if (!h || reps <= 0 || (!h->batch && !gamma_out_dev)) return GAMMA_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int lanes[5] = {2, 4, 8, 16, 32};
    int best_l = h->lanes, best_b = h->shell_minblocks, best_t = h->tail_minblocks;
    float best = INFINITY;
    int rc = GAMMA_OK;
    auto run = [&]() { return h->batch ? gamma_batch_run(h, s) : gamma_run(h, gamma_out_dev, s); };
    // the staged walks and the warp-evaluated queue walk do not take a lane
    // count: only the block budgets vary
    const bool tile_walk = !h->grids && h->walk != 0;
    const int nl = tile_walk ? 1 : 5;
    const int tb_max = tile_walk && h->walk == 3 ? 4 : 3;
    for (int li = 0; li < nl && rc == GAMMA_OK; ++li)
        for (int bl = 1; bl <= 4 && rc == GAMMA_OK; ++bl)
            for (int tb = 1; tb <= tb_max && rc == GAMMA_OK; ++tb) {
                h->lanes = tile_walk ? best_l : lanes[li];
                h->shell_minblocks = bl;
                h->tail_minblocks = tb;
                h->sg_dirty = true;                    // a captured graph holds the old shapes
                if (h->batch) h->batch->dirty = true;
                if ((rc = run()) || (rc = run())) break; // direct run, then graph capture

                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && rc == GAMMA_OK; ++r) rc = run();
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = GAMMA_ERR_CUDA; break; }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
                if (ms < best) { best = ms; best_l = h->lanes; best_b = bl; best_t = tb; }
            }
    h->lanes = best_l;
    h->shell_minblocks = best_b;
    h->tail_minblocks = best_t;
    // the warp-evaluated walk's queue parts: the fixed thresholds or the
    // choice from the queue (long queues of global criteria walk faster one
    // lane per voxel), whichever runs faster at the best shapes
    if (rc == GAMMA_OK && !h->grids && h->walk == 3 && best < INFINITY) {
        const int keep = h->group_bucket;
        h->group_bucket = keep >= 0 ? -1 : 9;
        h->sg_dirty = true;
        if (h->batch) h->batch->dirty = true;
        float ms = INFINITY;
        if (!(rc = run()) && !(rc = run())) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && rc == GAMMA_OK; ++r) rc = run();
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = GAMMA_ERR_CUDA;
            else {
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
            }
        }
        if (rc == GAMMA_OK && ms < best) best = ms;
        else h->group_bucket = keep;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->sg_dirty = true;
    if (h->batch) h->batch->dirty = true;
    if (rc) return rc;
    if (lanes_per_voxel) *lanes_per_voxel = best_l;
    if (shell_blocks_per_sm) *shell_blocks_per_sm = best_b;
    if (tail_blocks_per_sm) *tail_blocks_per_sm = best_t;
    if (best_ms) *best_ms = best;
    return GAMMA_OK;
}

int gamma_features(gamma_handle h, const uint32_t* voxels_dev, int64_t n, void* X_bf16_dev,
                   void* cuda_stream)
{
    if (!h || h->batch || !voxels_dev || !X_bf16_dev || n < 0) return GAMMA_ERR_INVALID_ARG;
    if (n == 0) return GAMMA_OK;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    const Problem P = make_problem(h, nullptr);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CK(gk::launch_features(P, voxels_dev, n, (__nv_bfloat16*)X_bf16_dev, s));
    return GAMMA_OK;
}

int gamma_labels(gamma_handle h, const float* gamma_map_dev, const uint32_t* voxels_dev, int64_t n,
                 float* targets_dev, void* cuda_stream)
{
    if (!h || h->batch || !gamma_map_dev || !voxels_dev || !targets_dev || n < 0)
        return GAMMA_ERR_INVALID_ARG;
    if (n == 0) return GAMMA_OK;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    const Problem P = make_problem(h, nullptr);
    CK(gk::launch_labels(P, gamma_map_dev, voxels_dev, n, targets_dev, (cudaStream_t)cuda_stream));
    return GAMMA_OK;
}

// Buffers the seeding pass needs once a model is attached.
static int seed_buffers(gamma_handle h)
{
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    if (!h->seed_list) CK(cudaMalloc(&h->seed_list, sizeof(unsigned) * (size_t)h->tail_cap));
    if (!h->seed_X) {
        h->seed_cap = std::min<unsigned>(h->tail_cap, kSeedRowsMax);
        CK(cudaMalloc(&h->seed_X, sizeof(__nv_bfloat16) * gk::kInPad * (size_t)h->seed_cap));
        CK(cudaMalloc(&h->seed_Y, sizeof(float) * gk::kOut * (size_t)h->seed_cap));
    }
    return GAMMA_OK;
}

// A model attached to (or detached from) a batch handle changes its launch
// sequence: the descriptors are uploaded again (with the seeding rows) and the
// graph is captured again at the next run.
static int batch_model_changed(gamma_handle h)
{
    BatchState* b = h->batch;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    if (h->ran) CK(cudaStreamSynchronize(h->last_stream));
    b->dirty = true;
    return GAMMA_OK;
}

int gamma_set_model(gamma_handle h, gamma_model m)
{
    if (!h || h->grids) return GAMMA_ERR_INVALID_ARG;
    if (m && !h->batch)
        if (int rc = seed_buffers(h)) return rc;
    if (h->batch)
        if (int rc = batch_model_changed(h)) return rc;
    if (h->own_model) gamma_model_destroy(h->model);
    h->sg_dirty = true;
    h->model = m;
    h->own_model = false;
    return GAMMA_OK;
}

int gamma_load_model(gamma_handle h, const char* path)
{
    if (!h || !path) return GAMMA_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    if (!dg.ok) return GAMMA_ERR_CUDA;
    if (h->grids) return GAMMA_ERR_INVALID_ARG;
    if (h->batch) {
        if (int rc = batch_model_changed(h)) return rc;
    } else if (int rc = seed_buffers(h)) {
        return rc;
    }
    gamma_model m = nullptr;
    if (int rc = gamma_model_create(&m, 0)) return rc;
    if (int rc = gamma_model_load(m, path)) {
        gamma_model_destroy(m);
        return rc;
    }
    if (h->own_model) gamma_model_destroy(h->model);
    h->sg_dirty = true;
    h->model = m;
    h->own_model = true;
    return GAMMA_OK;
}

const char* gamma_strerror(int code)
{
    switch (code) {
    case GAMMA_OK: return "ok";
    case GAMMA_ERR_INVALID_ARG: return "invalid argument";
    case GAMMA_ERR_SHAPE: return "invalid shape";
    case GAMMA_ERR_NAN_INPUT: return "non-finite dose in input";
    case GAMMA_ERR_OOM: return "out of memory";
    case GAMMA_ERR_TABLE_TOO_LARGE: return "cell table too large";
    case GAMMA_ERR_TIMEOUT: return "device wait timed out";
    case GAMMA_ERR_CUDA: return "CUDA error";
    case GAMMA_ERR_NOT_RUN: return "no run yet";
    case GAMMA_ERR_MODEL: return "bad model";
    case GAMMA_ERR_QUEUE_FULL: return "work queue overflow";
    case GAMMA_ERR_TOO_LARGE: return "grid exceeds the fixed scratch of gamma_run_noalloc";
    case GAMMA_ERR_DOSE_NORM: return "global criteria need a positive dose norm: the reference has no positive dose";
    default: return "unknown error";
    }
}

namespace {

__device__ float g_fma_sink;

// FP32 FMA throughput probe: eight independent multiply-add chains per
// thread, 128 FMAs per chain and round.  With 0 < b < 1 and c > 0 every chain
// stays positive, so the sum is never stored; the store keeps the chains live.
__global__ void __launch_bounds__(256) k_fma_probe(float b, float c, int rounds)
{
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (float)threadIdx.x * 1e-3f + (float)i;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) sum += a[i];
    if (sum < 0.f) g_fma_sink = sum;
}

struct EventPair {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~EventPair()
    {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
};

}  // namespace

int gamma_measure_fp32_peak(double* tflops, double* ms, void* cuda_stream)
{
    if (!tflops) return GAMMA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, rounds = 1000;
    EventPair ev;
    CK(cudaEventCreate(&ev.e[0]));
    CK(cudaEventCreate(&ev.e[1]));
    k_fma_probe<<<blocks, threads, 0, s>>>(0.999f, 1e-3f, rounds / 10);
    CK(cudaGetLastError());
    float best = INFINITY;
    for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(ev.e[0], s));
        k_fma_probe<<<blocks, threads, 0, s>>>(0.999f, 1e-3f, rounds);
        CK(cudaGetLastError());
        CK(cudaEventRecord(ev.e[1], s));
        CK(cudaEventSynchronize(ev.e[1]));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ev.e[0], ev.e[1]));
        best = std::min(best, t);
    }
    const double flop = (double)blocks * threads * rounds * 16.0 * 8.0 * 2.0;
    *tflops = best > 0.f ? flop / (best * 1e-3) / 1e12 : 0.0;
    if (ms) *ms = best;
    return GAMMA_OK;
}

const char* gamma_last_cuda_error(void) { return g_last_cuda.c_str(); }

const char* gamma_version(void) { return "gamma_gb300 0.1 (sm_103a)"; }

}  // extern "C"
