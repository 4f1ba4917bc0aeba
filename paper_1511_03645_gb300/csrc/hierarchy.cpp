// Host side of libadjamr: the AMR hierarchy on one GB300.
//
// Fields and medium coefficients live in one device arena per level
// (structure of arrays: [field][cell], every patch a contiguous block with a
// 2-cell ghost ring).  The host keeps only metadata: patch boxes, lookup
// buckets, and the device descriptor tables (ghost map, average-down map,
// tile work-list) rebuilt at each regrid.  Between regrids a level step is
// three kernel launches on the context's stream (ghost fill, fused step,
// average-down); regrids flag on the device, copy the flag bitmap to the
// host, cluster there (Berger-Rigoutsos, Sec. 3) and initialise the new
// patches on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace adjamr;

namespace {

struct Box {
    int i0, i1, j0, j1;  // inclusive
};

struct HPatch {
    int ilo, jlo, nx, ny, sx, sy;
    long long base;
};

struct Level {
    int N = 0, M = 0;
    double dx = 0, dy = 0, dt = 0;
    long long nstep = 0;
    int cur = 0;
    std::vector<HPatch> patches;
    long long ncell = 0, ninterior = 0;
    double *q[2] = {nullptr, nullptr};
    double *aux = nullptr, *med = nullptr;
    double *d_arena = nullptr;  // the one allocation q[0], q[1], aux and med point into
    PatchDesc *d_patches = nullptr;
    WorkItem *d_work = nullptr;
    int nwork = 0, work_tx = 0, work_ty = 0;
    bool work_lpt = false, work_deps = false;
    // substep launches: dependency rows of the work list ([nwork][kDepRow]
    // tile indices, then nwork counts) and the tile of every arena cell
    int *d_dep = nullptr, *d_tile_of = nullptr;
    // coefficient table of the whole index space (AuxTable), kept across rebuilds
    double *d_auxtab = nullptr;
    std::vector<WorkItem> h_work;
    GhostDesc *d_ghost = nullptr;
    long long nghost = 0;
    // coarse stencil values of the kind-1 ghost cells (k_cpre), recomputed
    // after every step of level l - 1: d_cpre[((k * m + f) * cpre_sc + src) * 3 + j]
    // for substep k; d_clist lists one ghost cell per distinct coarse cell
    int *d_cmark = nullptr;
    size_t cmark_cap = 0;
    unsigned long long *d_clist = nullptr;
    double *d_cpre = nullptr;
    long long cpre_sc = 0;
    AvgDesc *d_avg = nullptr;
    long long navg = 0;
    long long *d_prefix = nullptr;   // interior cells per patch (prefix)
    long long *d_gprefix = nullptr;  // ghost cells per patch (prefix)
    long long *d_sprefix = nullptr;  // storage cells per patch (prefix)
    long long *d_aprefix = nullptr;  // coarse-footprint cells per patch (prefix)
    long long nstore = 0, nghost_cells = 0, navg_cells = 0;
    int *d_owner = nullptr;          // [M][N] arena index of each interior cell, or -1
    char *d_meta = nullptr;          // one allocation holding d_patches and the prefix arrays
    MediumDev *d_med = nullptr;
    // lookup buckets (cells per bucket side)
    int bs = 16, nbx = 0, nby = 0;
    std::vector<std::vector<int>> buckets;
    // conservation fix-up (refluxing), rebuilt after every regrid: the table
    // of the level's taking-part cells (coarse-role entries first) and its
    // arena map, keyed on the host by J * N + I; for the pair (l, l + 1) the
    // coarse-role records, the fine records of every substep and the fine
    // cell each fine record belongs to
    std::unordered_map<long long, int> rkey;
    int nrcell = 0, nrcoarse = 0;
    RefluxCell *d_rcells = nullptr;
    int *d_rmap = nullptr;
    double *d_lc = nullptr, *d_lf = nullptr;
    long long nfrec = 0;
    long long *d_fidx = nullptr;
};

// Row-major bitmap of a window of an index space: cell (i, j) is bit i & 63 of
// word i >> 6 of row j.
struct Bits {
    int N = 0, M = 0, nw = 0;
    std::vector<uint64_t> w;
    void reset(int n, int m)
    {
        N = n;
        M = m;
        nw = (n + 63) >> 6;
        w.assign((size_t)nw * m, 0);
    }
    uint64_t *row(int j) { return &w[(size_t)j * nw]; }
    const uint64_t *row(int j) const { return &w[(size_t)j * nw]; }
    uint64_t tail() const { return (N & 63) ? ((1ull << (N & 63)) - 1) : ~0ull; }
};

}  // namespace

struct adjamr_ctx {
    adjamr_params P;
    int m = 0, naux = 0, nmed = 0, gy = 0;
    Level L[ADJAMR_MAX_LEVELS];
    long long T[ADJAMR_MAX_LEVELS] = {};
    long long rebuilt_tick[ADJAMR_MAX_LEVELS];
    cudaStream_t s = nullptr;
    // side stream of the adjoint flags that overlap the step of their level
    // (high priority: the host waits for them), and the event that orders
    // them after the work already queued on s
    cudaStream_t s_flag = nullptr;
    cudaEvent_t ev_flag = nullptr;
    bool on_side = false;  // s is the side stream (inside the overlapped flags)
    std::string err;
    bool have_medium = false;
    MediumDev mh[ADJAMR_MAX_LEVELS];
    std::vector<double *> dense_dev;
    adjamr_adjoint *adj = nullptr;
    unsigned long long *d_cfl = nullptr;
    // flag head (kPinHead bytes: count, bounding box, list counters) of the
    // flag calls that make no bitmap; a regrid's head sits in front of its bitmap
    unsigned long long *d_fhead = nullptr;
    int *d_err = nullptr;  // device-side invariant violations (nesting), checked after syncs
    Bits h_fl, h_unc;               // host clustering scratch (regrid window)
    std::vector<int> h_sort_cnt;    // work-list ordering scratch
    std::vector<WorkItem> h_sort_tmp;
    std::vector<uint64_t> h_tmp;
    std::vector<int> h_cnt;
    // pinned staging ring of the descriptor uploads: slots used in turn, each
    // reused once the copy recorded by its event has completed; 4 slots cover
    // the uploads of one regrid of two levels, so the host does not wait for
    // the stream in the middle of a regrid
    static constexpr int kStageSlots = 4;
    char *h_stage[kStageSlots] = {};
    size_t h_stage_bytes[kStageSlots] = {};
    cudaEvent_t stage_ev[kStageSlots] = {};
    int stage_slot = 0;
    // device blocks released by regrids, reused by later ones (the stream
    // orders every use, as with cudaFreeAsync): sizes of every block handed
    // out, and the cached ones
    std::unordered_map<void *, size_t> blk_size;
    std::vector<std::pair<size_t, void *>> blk_free;
    size_t blk_free_bytes = 0;
    size_t blk_cache_cap = (size_t)512 << 20;  // bytes the cache may hold (0: no caching)
    uint64_t *d_flagall = nullptr;  // flag head + bitmap of the level being regridded
    uint64_t *d_flagbuf = nullptr;  // the bitmap: d_flagall + kPinHead / 8
    // pinned readback of the flag count, bounding box and (when small) the
    // whole bitmap: one synchronisation per flagged level
    char *h_pin = nullptr;
    size_t h_pin_bytes = 0;
    bool pin_has_bits = false;
    // work list of the two-pass flags
    unsigned long long *d_fitems = nullptr;
    long long fcap = 0;
    // per-level bilinear tables of the adjoint grid for the dense flag kernel
    char *d_ftab[ADJAMR_MAX_LEVELS] = {};
    int ftab_ax[ADJAMR_MAX_LEVELS] = {}, ftab_ay[ADJAMR_MAX_LEVELS] = {};
    size_t ftab_off[ADJAMR_MAX_LEVELS][6] = {};
    size_t flagbuf_bytes = 0;
    double *d_fscratch = nullptr, *d_fout = nullptr;
    size_t fscratch_n = 0;
    adjamr_stats st = {};
    int tx = 32, ty = 8, launch_mode = 0, grid_persistent = 0, nsm = 0;
    // per level: tile extents the patches are cut to, the compiled kernel tile
    // that holds them, the persistent grid
    int ltx[ADJAMR_MAX_LEVELS] = {}, lty[ADJAMR_MAX_LEVELS] = {}, lgrid[ADJAMR_MAX_LEVELS] = {};
    int lkx[ADJAMR_MAX_LEVELS] = {}, lky[ADJAMR_MAX_LEVELS] = {};
    int lfuse[ADJAMR_MAX_LEVELS] = {};  // ghost ring computed inside the step kernel
    int lmode[ADJAMR_MAX_LEVELS] = {};  // ADJAMR_LAUNCH_* per level
    unsigned long long *d_wctr = nullptr;  // tile counter of the dynamic launch mode
    unsigned long long wbase = 0;          // its value at the start of the next dynamic launch
    // substep launches: grid per level (0: the level's kernel tile has no
    // substep kernel), per-tile completion counters and their epoch
    int lgrid_sub[ADJAMR_MAX_LEVELS] = {};
    unsigned long long *d_done = nullptr;
    size_t done_cap = 0;
    unsigned long long done_base = 0;
    int cgen = 0;  // generation of the coarse-stencil marks
    bool aux_tables = true;  // per-level coefficient tables (off in the serving loop)
    bool timing = false;
    // gauges: cell indices per level (device), records on the device
    int ngauge = 0;
    int *d_gij = nullptr;           // [2][nlevels][ngauge]: I then J
    double *d_grec = nullptr;       // [gcap][ngauge][1 + m]
    long long ngrec = 0, gcap = 0;
    // the builders of the level a regrid is rebuilding, recorded (pend_on)
    // instead of launched and then launched together by launch_rebuild
    bool pend_on = false;
    adjamr::OwnerFillArgs pend_o{};
    adjamr::AuxPatchesArgs pend_x{};
    adjamr::InitNewArgs pend_in{};
    adjamr::GhostBuildArgs pend_gb{};
    adjamr::AvgBuildArgs pend_ab{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // step-kernel timing without host synchronisation: event pairs recorded
    // around every step launch, read when the stream is synchronised
    std::vector<cudaEvent_t> tev;
    std::vector<int> tev_level;
    size_t tev_used = 0;
};

namespace {

// device block from the context's cache (best fit up to twice the size),
// else a new stream-ordered allocation
template <typename T>
cudaError_t cget(adjamr_ctx *c, T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    const size_t bytes = (n * sizeof(T) + 255) / 256 * 256;
    int best = -1;
    // (a cached block was released in the order of the main stream: work on
    // the side stream takes fresh stream-ordered memory instead)
    for (int k = 0; k < (int)c->blk_free.size() && !c->on_side; k++) {
        const size_t b = c->blk_free[k].first;
        if (b >= bytes && b <= 2 * bytes + 65536 && (best < 0 || b < c->blk_free[best].first)) best = k;
    }
    if (best >= 0) {
        *p = static_cast<T *>(c->blk_free[best].second);
        c->blk_free_bytes -= c->blk_free[best].first;
        c->blk_free.erase(c->blk_free.begin() + best);
        return cudaSuccess;
    }
    void *q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, bytes, c->s);
    if (e != cudaSuccess) return e;
    c->blk_size[q] = bytes;
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

// return a block to the cache (blocks not from cget are freed)
constexpr size_t kBlockCacheMax = 48;
template <typename T>
void cput(adjamr_ctx *c, T *&p)
{
    if (!p) return;
    void *q = (void *)p;
    p = nullptr;
    auto it = c->blk_size.find(q);
    if (it == c->blk_size.end()) {
        cudaFreeAsync(q, c->s);
        return;
    }
    c->blk_free.push_back({it->second, q});
    c->blk_free_bytes += it->second;
    while (!c->blk_free.empty() && (c->blk_free.size() > kBlockCacheMax || c->blk_free_bytes > c->blk_cache_cap)) {
        void *old = c->blk_free.front().second;
        c->blk_free_bytes -= c->blk_free.front().first;
        c->blk_free.erase(c->blk_free.begin());
        c->blk_size.erase(old);
        cudaFreeAsync(old, c->on_side ? c->s_flag : c->s);  // in the main stream's order
    }
}

}  // namespace

namespace adjamr {
void ctx_set_block_cache(adjamr_ctx *c, size_t cap_bytes) { c->blk_cache_cap = cap_bytes; }
void ctx_set_aux_tables(adjamr_ctx *c, bool on) { c->aux_tables = on; }

// index-space cells of level l's coefficient table (0: none is kept)
long long aux_table_cells(const adjamr_ctx *c, int l)
{
    constexpr long long kMaxCells = 1ll << 23;  // <= 8.4 M cells (400 MB at 6 fields)
    const long long n = (long long)(c->L[l].N + 4) * (c->P.dim == 2 ? c->L[l].M + 4 : 1);
    return (c->aux_tables && n <= kMaxCells) ? n : 0;
}

bool pdl_enabled()
{
    static const bool on = [] {
        const char *v = std::getenv("ADJAMR_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}
}  // namespace adjamr

namespace {

void cache_drain(adjamr_ctx *c)
{
    for (auto &b : c->blk_free) {
        c->blk_size.erase(b.second);
        cudaFreeAsync(b.second, c->s);
    }
    c->blk_free.clear();
    c->blk_free_bytes = 0;
}


#define CKR(ctx, x)                                                                                   \
    do {                                                                                              \
        cudaError_t _e = (x);                                                                         \
        if (_e != cudaSuccess) {                                                                      \
            (ctx)->err = std::string(#x) + ": " + cudaGetErrorString(_e);                             \
            return ADJAMR_ECUDA;                                                                      \
        }                                                                                             \
    } while (0)

#define TRY(x)                                                                                        \
    do {                                                                                              \
        adjamr_status _s = (x);                                                                       \
        if (_s != ADJAMR_OK) return _s;                                                               \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n, cudaStream_t s)
{
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    return cudaMallocAsync((void **)p, n * sizeof(T), s);
}

template <typename T>
void dfree(T *&p, cudaStream_t s)
{
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

template <typename T>
cudaError_t upload(T **p, const std::vector<T> &v, cudaStream_t s)
{
    cudaError_t e = dalloc(p, v.size(), s);
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

int part_len(int n, int p, int k) { return n / p + (k < n % p ? 1 : 0); }
int part_off(int n, int p, int k)
{
    int o = 0;
    for (int q = 0; q < k; q++) o += part_len(n, p, q);
    return o;
}

long long cell_of(const adjamr_ctx *c, const HPatch &p, int i, int j)
{
    return p.base + (long long)(j + c->gy) * p.sx + (i + 2);
}

void build_buckets(Level &L)
{
    L.nbx = (L.N + L.bs - 1) / L.bs;
    L.nby = (L.M + L.bs - 1) / L.bs;
    L.buckets.assign((size_t)L.nbx * L.nby, {});
    for (int k = 0; k < (int)L.patches.size(); k++) {
        const HPatch &p = L.patches[k];
        for (int by = p.jlo / L.bs; by <= (p.jlo + p.ny - 1) / L.bs; by++)
            for (int bx = p.ilo / L.bs; bx <= (p.ilo + p.nx - 1) / L.bs; bx++)
                L.buckets[(size_t)by * L.nbx + bx].push_back(k);
    }
}

int find_patch(Level &L, int I, int J)
{
    if (L.buckets.empty() && !L.patches.empty()) build_buckets(L);
    if (I < 0 || J < 0 || I >= L.N || J >= L.M || L.buckets.empty()) return -1;
    const std::vector<int> &b = L.buckets[(size_t)(J / L.bs) * L.nbx + I / L.bs];
    for (int k : b) {
        const HPatch &p = L.patches[k];
        if (I >= p.ilo && I < p.ilo + p.nx && J >= p.jlo && J < p.jlo + p.ny) return k;
    }
    return -1;
}

// the level's patches are exactly the boxes b, in order
bool same_layout(const Level &L, const std::vector<Box> &b)
{
    if (L.patches.size() != b.size()) return false;
    for (size_t k = 0; k < b.size(); k++) {
        const HPatch &p = L.patches[k];
        if (p.ilo != b[k].i0 || p.jlo != b[k].j0 || p.nx != b[k].i1 - b[k].i0 + 1 || p.ny != b[k].j1 - b[k].j0 + 1)
            return false;
    }
    return true;
}

void reflux_release(adjamr_ctx *c, Level &L)
{
    cput(c, L.d_rcells);
    cput(c, L.d_rmap);
    cput(c, L.d_lc);
    cput(c, L.d_lf);
    cput(c, L.d_fidx);
    L.rkey.clear();
    L.nrcell = L.nrcoarse = 0;
    L.nfrec = 0;
}

void free_level(adjamr_ctx *c, Level &L)
{
    cudaStream_t s = c->s;
    cput(c, L.d_arena);
    L.q[0] = L.q[1] = nullptr;
    L.aux = L.med = nullptr;
    if (L.d_meta) {
        cput(c, L.d_meta);
        L.d_patches = nullptr;
        L.d_prefix = L.d_gprefix = L.d_sprefix = L.d_aprefix = nullptr;
    } else {
        dfree(L.d_patches, s);
        dfree(L.d_prefix, s);
        dfree(L.d_gprefix, s);
        dfree(L.d_sprefix, s);
        dfree(L.d_aprefix, s);
    }
    cput(c, L.d_work);
    cput(c, L.d_dep);
    cput(c, L.d_tile_of);
    cput(c, L.d_ghost);
    cput(c, L.d_cmark);
    L.cmark_cap = 0;
    cput(c, L.d_clist);
    cput(c, L.d_cpre);
    cput(c, L.d_avg);
    cput(c, L.d_owner);
    reflux_release(c, L);
    L.patches.clear();
    L.h_work.clear();
    L.buckets.clear();
    L.ncell = L.ninterior = 0;
    L.nwork = 0;
    L.nghost = L.navg = 0;
    L.work_tx = L.work_ty = 0;
}

// (re)build the tile work-list of a level for tile (tx, ty)

cudaError_t upload_packed(adjamr_ctx *c, const std::vector<std::pair<const void *, size_t>> &chunks, char **dev,
                          std::vector<size_t> &offs);

adjamr_status build_work(adjamr_ctx *c, int l, int tx, int ty)
{
    Level &L = c->L[l];
    const bool deps = c->lmode[l] == ADJAMR_LAUNCH_SUBSTEPS && c->P.dim == 2;
    // substep launches keep the spatial (patch, row) order: a tile's
    // neighbours are then taken close to it in the previous substep
    const bool lpt = c->lmode[l] != ADJAMR_LAUNCH_PER_PATCH && !deps;
    if (L.work_tx == tx && L.work_ty == ty && L.d_work && L.work_lpt == lpt && L.work_deps == deps) return ADJAMR_OK;
    cput(c, L.d_work);
    L.h_work.clear();
    const int tyy0 = (c->P.dim == 2) ? ty : 1;
    int txx = tx, tyy = tyy0;
    if (c->P.dim == 2 && c->lmode[l] == ADJAMR_LAUNCH_WORKLIST && c->nsm > 0) {
        // A small layout cut at the level's tile size leaves SMs with one or
        // two CTAs (or none), which cannot keep the FP64 pipe busy: cut it
        // finer, down to 8x8, until every SM has about three tiles.  The
        // kernel is the level's (it runs any tile up to its shape), and every
        // cut gives the same bits.
        auto count = [&](int a, int b) {
            long long n = 0;
            for (const HPatch &p : L.patches) n += (long long)tile_count(p.nx, a) * tile_count(p.ny, b);
            return n;
        };
        const long long want = 3LL * c->nsm;
        static const int cuts[3][2] = {{12, 12}, {12, 8}, {8, 8}};
        if (count(txx, tyy) < want)
            for (const auto &cu : cuts) {
                if (cu[0] * cu[1] >= txx * tyy) continue;
                txx = std::min(txx, cu[0]);
                tyy = std::min(tyy, cu[1]);
                if (count(txx, tyy) >= want) break;
            }
    }
    if (c->P.dim == 1 && c->lmode[l] == ADJAMR_LAUNCH_WORKLIST && c->nsm > 0) {
        // A small 1D level cut at the level's tile leaves each phase's FP64
        // work to one or two SMs, whose narrow FP64 pipe then serialises
        // several warps: cut it finer, down to 24 cells (one warp per phase),
        // until the tiles reach the SM count.  Every cut gives the same bits.
        auto count1 = [&](int a) {
            long long n = 0;
            for (const HPatch &p : L.patches) n += (long long)tile_count(p.nx, a);
            return n;
        };
        static const int cuts1[3] = {64, 32, 24};
        if (count1(txx) < c->nsm)
            for (int cu : cuts1) {
                if (cu >= txx) continue;
                txx = cu;
                if (count1(txx) >= c->nsm) break;
            }
    }
    for (int k = 0; k < (int)L.patches.size(); k++) {
        const HPatch &p = L.patches[k];
        const int nx = tile_count(p.nx, txx), ny = tile_count(p.ny, tyy);
        for (int b = 0; b < ny; b++)
            for (int a = 0; a < nx; a++)
                L.h_work.push_back({k, tile_off(p.nx, nx, a), tile_off(p.ny, ny, b),
                                    (unsigned short)tile_len(p.nx, nx, a), (unsigned short)tile_len(p.ny, ny, b)});
    }
    // one launch over the level: largest tiles first, so that the last CTAs
    // to start are the short ones (one launch per patch keeps patch order)
    if (lpt && L.h_work.size() > 1) {
        // stable counting sort by tile area, largest first (areas <= 64 x 16)
        int amax = 0;
        for (const WorkItem &w : L.h_work) amax = std::max(amax, (int)w.tx * w.ty);
        std::vector<int> &start = c->h_sort_cnt;
        start.assign((size_t)amax + 2, 0);
        for (const WorkItem &w : L.h_work) start[(size_t)(amax - (int)w.tx * w.ty) + 1]++;
        for (size_t k = 1; k < start.size(); k++) start[k] += start[k - 1];
        std::vector<WorkItem> &out = c->h_sort_tmp;
        out.resize(L.h_work.size());
        for (const WorkItem &w : L.h_work) out[(size_t)start[(size_t)(amax - (int)w.tx * w.ty)]++] = w;
        L.h_work.swap(out);
    }
    L.nwork = (int)L.h_work.size();
    std::vector<size_t> offs;
    char *dw = nullptr;
    CKR(c, upload_packed(c, {{L.h_work.data(), sizeof(WorkItem) * L.h_work.size()}}, &dw, offs));
    L.d_work = reinterpret_cast<WorkItem *>(dw);
    cput(c, L.d_dep);
    cput(c, L.d_tile_of);
    if (deps && L.nwork > 0) {
        // dependency rows built on the device from the level's owner map
        CKR(c, cget(c, &L.d_dep, (size_t)L.nwork * (kDepRow + 1)));
        CKR(c, cget(c, &L.d_tile_of, (size_t)L.ncell));
        CKR(c, launch_tile_deps(L.d_patches, L.d_work, L.nwork, L.d_owner, L.N, L.M, c->P.bc, L.d_tile_of, L.d_dep,
                                L.d_dep + (size_t)L.nwork * kDepRow, c->s));
        c->st.kernel_launches += 2;
    }
    L.work_tx = tx;
    L.work_ty = ty;
    L.work_lpt = lpt;
    L.work_deps = deps;
    return ADJAMR_OK;
}

// Copy host chunks into one new device allocation through the pinned
// staging buffer; returns the device base, chunk k at offs[k].
cudaError_t upload_packed(adjamr_ctx *c, const std::vector<std::pair<const void *, size_t>> &chunks, char **dev,
                          std::vector<size_t> &offs)
{
    size_t total = 0;
    offs.clear();
    for (auto &ch : chunks) {
        offs.push_back(total);
        total += (ch.second + 255) / 256 * 256;
    }
    *dev = nullptr;
    if (total == 0) return cudaSuccess;
    const int sl = c->stage_slot;
    c->stage_slot = (sl + 1) % adjamr_ctx::kStageSlots;
    cudaError_t e;
    if (c->stage_ev[sl]) {
        e = cudaEventSynchronize(c->stage_ev[sl]);  // the slot's previous copy is done
        if (e != cudaSuccess) return e;
    } else {
        e = cudaEventCreateWithFlags(&c->stage_ev[sl], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    if (c->h_stage_bytes[sl] < total) {
        if (c->h_stage[sl]) cudaFreeHost(c->h_stage[sl]);
        c->h_stage[sl] = nullptr;
        size_t want = std::max(total, (size_t)1 << 20);
        e = cudaMallocHost((void **)&c->h_stage[sl], want);
        if (e != cudaSuccess) {
            c->h_stage_bytes[sl] = 0;
            return e;
        }
        c->h_stage_bytes[sl] = want;
    }
    for (size_t k = 0; k < chunks.size(); k++)
        if (chunks[k].second) std::memcpy(c->h_stage[sl] + offs[k], chunks[k].first, chunks[k].second);
    e = cget(c, dev, total);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(*dev, c->h_stage[sl], total, cudaMemcpyHostToDevice, c->s);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(c->stage_ev[sl], c->s);
}

// Copy a host vector into an existing device block through the pinned
// staging ring (no host wait for the stream unless the slot is still busy).
template <typename T>
cudaError_t upload_now(adjamr_ctx *c, T *dst, const std::vector<T> &v)
{
    const size_t total = v.size() * sizeof(T);
    if (total == 0) return cudaSuccess;
    const int sl = c->stage_slot;
    c->stage_slot = (sl + 1) % adjamr_ctx::kStageSlots;
    cudaError_t e;
    if (c->stage_ev[sl]) {
        e = cudaEventSynchronize(c->stage_ev[sl]);
        if (e != cudaSuccess) return e;
    } else {
        e = cudaEventCreateWithFlags(&c->stage_ev[sl], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    if (c->h_stage_bytes[sl] < total) {
        if (c->h_stage[sl]) cudaFreeHost(c->h_stage[sl]);
        c->h_stage[sl] = nullptr;
        const size_t want = std::max(total, (size_t)1 << 20);
        e = cudaMallocHost((void **)&c->h_stage[sl], want);
        if (e != cudaSuccess) {
            c->h_stage_bytes[sl] = 0;
            return e;
        }
        c->h_stage_bytes[sl] = want;
    }
    std::memcpy(c->h_stage[sl], v.data(), total);
    e = cudaMemcpyAsync(dst, c->h_stage[sl], total, cudaMemcpyHostToDevice, c->s);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(c->stage_ev[sl], c->s);
}

LevelIdx idx_of(const adjamr_ctx *c, int l)
{
    LevelIdx g;
    g.dim = c->P.dim;
    g.N = c->L[l].N;
    g.M = c->L[l].M;
    g.gy = c->gy;
    for (int k = 0; k < 4; k++) g.bc[k] = c->P.bc[k];
    return g;
}

// A builder kernel of a level's layout: launched now, or recorded for the
// combined launches of the rebuild in progress (flush_rebuild).
template <typename Args>
adjamr_status run_builder(adjamr_ctx *c, const Args &a)
{
    if (c->pend_on) {
        if constexpr (std::is_same_v<Args, OwnerFillArgs>) c->pend_o = a;
        else if constexpr (std::is_same_v<Args, AuxPatchesArgs>) c->pend_x = a;
        else if constexpr (std::is_same_v<Args, InitNewArgs>) c->pend_in = a;
        else if constexpr (std::is_same_v<Args, GhostBuildArgs>) c->pend_gb = a;
        else c->pend_ab = a;
        return ADJAMR_OK;
    }
    cudaError_t e;
    if constexpr (std::is_same_v<Args, OwnerFillArgs>) e = launch_owner_fill(a, c->s);
    else if constexpr (std::is_same_v<Args, AuxPatchesArgs>) e = launch_aux_patches(a, c->s);
    else if constexpr (std::is_same_v<Args, InitNewArgs>) e = launch_init_new(a, c->s);
    else if constexpr (std::is_same_v<Args, GhostBuildArgs>) e = launch_ghost_build(a, c->s);
    else e = launch_avg_build(a, c->s);
    CKR(c, e);
    if (a.n > 0) c->st.kernel_launches++;
    return ADJAMR_OK;
}

void pend_clear(adjamr_ctx *c)
{
    c->pend_on = false;
    c->pend_o = {};
    c->pend_x = {};
    c->pend_in = {};
    c->pend_gb = {};
    c->pend_ab = {};
}

// Launch the recorded builders (two kernels at most) and stop recording.
adjamr_status flush_rebuild(adjamr_ctx *c)
{
    int nl = 0;
    const cudaError_t e = launch_rebuild(c->pend_o, c->pend_x, c->pend_in, c->pend_gb, c->pend_ab, c->s, &nl);
    c->st.kernel_launches += nl;
    pend_clear(c);
    CKR(c, e);
    return ADJAMR_OK;
}

// allocate the arena of a level for the given boxes (level index space)
adjamr_status alloc_level(adjamr_ctx *c, int l, const std::vector<Box> &boxes)
{
    Level &L = c->L[l];
    L.patches.clear();
    long long off = 0;
    for (const Box &b : boxes) {
        HPatch p;
        p.ilo = b.i0;
        p.jlo = b.j0;
        p.nx = b.i1 - b.i0 + 1;
        p.ny = b.j1 - b.j0 + 1;
        p.sx = p.nx + 4;
        p.sy = p.ny + 2 * c->gy;
        p.base = off;
        off += ((long long)p.sx * p.sy + 3) / 4 * 4;  // 32-byte aligned blocks
        L.patches.push_back(p);
    }
    L.ncell = off;
    L.ninterior = 0;
    std::vector<PatchDesc> pd;
    std::vector<long long> prefix{0}, gprefix{0}, sprefix{0}, aprefix{0};
    double dtdx = L.dt / L.dx, dtdy = (c->P.dim == 2) ? L.dt / L.dy : 0.0;
    int rc = (l > 0) ? c->P.ratio[l - 1] : 1;
    L.nstore = L.nghost_cells = L.navg_cells = 0;
    for (const HPatch &p : L.patches) {
        PatchDesc d;
        d.ilo = p.ilo; d.jlo = p.jlo; d.nx = p.nx; d.ny = p.ny; d.sx = p.sx; d.sy = p.sy; d.base = p.base;
        d.dtdx = dtdx; d.dtdy = dtdy; d.hx = 0.5 * dtdx; d.hy = 0.5 * dtdy;
        d.gbase = L.nghost_cells;
        pd.push_back(d);
        L.ninterior += (long long)p.nx * p.ny;
        L.nstore += (long long)p.sx * p.sy;
        L.nghost_cells += (long long)p.sx * p.sy - (long long)p.nx * p.ny;
        L.navg_cells += (l > 0) ? (long long)(p.nx / rc) * (c->P.dim == 2 ? p.ny / rc : 1) : 0;
        prefix.push_back(L.ninterior);
        gprefix.push_back(L.nghost_cells);
        sprefix.push_back(L.nstore);
        aprefix.push_back(L.navg_cells);
    }
    // (no clearing: every ghost cell is written by the ghost fill before it is
    // read, every interior cell by the initialisation or the step)
    // one allocation: q[0] | q[1] | aux | med
    CKR(c, cget(c, &L.d_arena, (size_t)(2 * c->m + c->naux + c->nmed) * L.ncell));
    L.q[0] = L.d_arena;
    L.q[1] = L.d_arena ? L.q[0] + (size_t)c->m * L.ncell : nullptr;
    L.aux = L.d_arena ? L.q[1] + (size_t)c->m * L.ncell : nullptr;
    L.med = L.d_arena ? L.aux + (size_t)c->naux * L.ncell : nullptr;
    {
        std::vector<size_t> offs;
        const size_t pb = sizeof(long long) * prefix.size();
        CKR(c, upload_packed(c, {{pd.data(), sizeof(PatchDesc) * pd.size()}, {prefix.data(), pb}, {gprefix.data(), pb},
                                 {sprefix.data(), pb}, {aprefix.data(), pb}},
                             &L.d_meta, offs));
        L.d_patches = pd.empty() ? nullptr : (PatchDesc *)(L.d_meta + offs[0]);
        L.d_prefix = (long long *)(L.d_meta + offs[1]);
        L.d_gprefix = (long long *)(L.d_meta + offs[2]);
        L.d_sprefix = (long long *)(L.d_meta + offs[3]);
        L.d_aprefix = (long long *)(L.d_meta + offs[4]);
    }
    CKR(c, cget(c, &L.d_owner, (size_t)L.N * L.M));
    CKR(c, cudaMemsetAsync(L.d_owner, 0xff, sizeof(int) * (size_t)L.N * L.M, c->s));
    if (!L.patches.empty())
        TRY(run_builder(c, OwnerFillArgs{L.d_patches, L.d_prefix, (int)L.patches.size(), L.ninterior, idx_of(c, l),
                                         L.d_owner}));
    L.buckets.clear();  // rebuilt on demand by the host lookups
    L.work_tx = L.work_ty = 0;
    return build_work(c, l, c->ltx[l], c->lty[l]);
}

LevelGeom geom_of(const adjamr_ctx *c, int l)
{
    LevelGeom g;
    g.dim = c->P.dim;
    g.N = c->L[l].N;
    g.M = c->L[l].M;
    g.lo0 = c->P.lo[0];
    g.lo1 = c->P.lo[1];
    g.dx = c->L[l].dx;
    g.dy = c->L[l].dy;
    for (int k = 0; k < 4; k++) g.bc[k] = c->P.bc[k];
    return g;
}

// medium coefficients of every storage cell of a level
// (old: the level's previous arena during a rebuild, whose interior cells
// give their coefficients to the new storage cells at the same (I, J))
adjamr_status fill_aux(adjamr_ctx *c, int l, const Level *old = nullptr)
{
    Level &L = c->L[l];
    if (!c->have_medium || L.patches.empty()) return ADJAMR_OK;
    AuxReuse ru{nullptr, nullptr, nullptr, 0, c->naux, c->nmed};
    const long long tn = aux_table_cells(c, l);
    const AuxTable tb{L.d_auxtab, tn, L.N + 4};
    if (!tb.tab && old && !old->patches.empty() && old->d_owner && old->aux) {
        ru.owner = old->d_owner;
        ru.aux = old->aux;
        ru.med = old->med;
        ru.stride = old->ncell;
    }
    return run_builder(c, AuxPatchesArgs{c->P.eqn, L.d_patches, L.d_sprefix, (int)L.patches.size(), L.nstore,
                                         idx_of(c, l), L.aux, L.med, L.ncell, L.d_med, geom_of(c, l), ru, tb});
}

// ghost map of level l (needs level l-1 when l > 0), built on the device
adjamr_status build_ghost_map(adjamr_ctx *c, int l)
{
    Level &L = c->L[l];
    cput(c, L.d_ghost);
    L.nghost = L.nghost_cells;
    if (L.nghost == 0) return ADJAMR_OK;
    CKR(c, cget(c, &L.d_ghost, (size_t)L.nghost));
    const int *oc = (l > 0) ? c->L[l - 1].d_owner : nullptr;
    LevelIdx gc = (l > 0) ? idx_of(c, l - 1) : idx_of(c, l);
    int r = (l > 0) ? c->P.ratio[l - 1] : 1;
    // the coarse stencil list and values (levels > 0): the marks persist with
    // the level (zeroed when allocated) and are compared with a fresh
    // generation number, so they need no clearing per build
    cput(c, L.d_clist);
    cput(c, L.d_cpre);
    L.cpre_sc = 0;
    int gen = 0;
    if (l > 0) {
        const Level &C = c->L[l - 1];
        if (L.cmark_cap < (size_t)C.ncell) {
            cput(c, L.d_cmark);
            L.cmark_cap = 0;
            const size_t want = std::max((size_t)C.ncell, 2 * L.cmark_cap);
            CKR(c, cget(c, &L.d_cmark, want));
            CKR(c, cudaMemsetAsync(L.d_cmark, 0, sizeof(int) * want, c->s));
            L.cmark_cap = want;
        }
        CKR(c, cget(c, &L.d_clist, (size_t)L.nghost + 1));
        CKR(c, cget(c, &L.d_cpre, (size_t)r * c->m * C.ncell * 3));
        CKR(c, cudaMemsetAsync(L.d_clist, 0, sizeof(unsigned long long), c->s));
        if (++c->cgen <= 0) c->cgen = 1;  // (2^31 builds)
        gen = c->cgen;
        L.cpre_sc = C.ncell;
    }
    return run_builder(c, GhostBuildArgs{L.d_patches, L.d_gprefix, (int)L.patches.size(), L.nghost, idx_of(c, l),
                                         L.d_owner, oc, gc, r, L.d_ghost, c->d_err, l > 0 ? L.d_cmark : nullptr, gen,
                                         l > 0 ? L.d_clist : nullptr});
}

// Coarse stencil values of level l's kind-1 ghost cells for all substeps of
// the step level l - 1 has just taken (its old and new states final until the
// average-down); the substeps' ghost fills and ghost rings read them.
bool substeps_ok(const adjamr_ctx *c, int l);

// Whether level l's first ghost fill of a coarse step also computes the
// stored stencil values of the later substeps (separate fill, one launch per
// substep): then coarse_pre does nothing for it.
bool fill_makes_pre(const adjamr_ctx *c, int l) { return l > 0 && !c->lfuse[l] && !substeps_ok(c, l); }

// Step-kernel timing without host synchronisation: an event pair around a
// launch, tagged with its level and kind (0: step kernel; 1: ghost work of the
// level -- its separate ghost fill or coarse stencil values), harvested once
// the stream has passed them.  Records the first event; returns the second.
cudaError_t time_begin(adjamr_ctx *c, int l, int kind, cudaEvent_t *end)
{
    *end = nullptr;
    if (!c->timing) return cudaSuccess;
    while (c->tev.size() < c->tev_used + 2) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        c->tev.push_back(e);
        c->tev_level.push_back(0);
    }
    c->tev_level[c->tev_used] = l + kind * ADJAMR_MAX_LEVELS;
    *end = c->tev[c->tev_used + 1];
    cudaError_t err = cudaEventRecord(c->tev[c->tev_used], c->s);
    c->tev_used += 2;
    return err;
}

adjamr_status coarse_pre(adjamr_ctx *c, int l)
{
    Level &L = c->L[l];
    const Level &C = c->L[l - 1];
    if (!L.d_cpre || L.nghost == 0 || fill_makes_pre(c, l)) return ADJAMR_OK;
    // timed as level l's ghost work (a fill at substep 0 computes the same
    // values there otherwise)
    cudaEvent_t te = nullptr;
    CKR(c, time_begin(c, l, 1, &te));
    CKR(c, launch_cpre(L.d_ghost, L.d_clist, L.nghost, c->m, c->P.ratio[l - 1], c->P.dim, C.q[C.cur],
                       C.q[1 - C.cur], L.cpre_sc, L.d_cpre, c->nsm * 8, c->s));
    if (te) CKR(c, cudaEventRecord(te, c->s));
    c->st.kernel_launches++;
    return ADJAMR_OK;
}

// average-down map of level l (fine) into level l-1, built on the device
adjamr_status build_avg_map(adjamr_ctx *c, int l)
{
    Level &F = c->L[l];
    cput(c, F.d_avg);
    F.navg = F.navg_cells;
    if (F.navg == 0) return ADJAMR_OK;
    CKR(c, cget(c, &F.d_avg, (size_t)F.navg));
    return run_builder(c, AvgBuildArgs{F.d_patches, F.d_aprefix, (int)F.patches.size(), F.navg, c->P.dim,
                                       c->P.ratio[l - 1], c->L[l - 1].d_owner, idx_of(c, l - 1), F.d_avg, c->d_err});
}

// ---------------------------------------------------------------- clustering
// Berger-Rigoutsos on a flag field [M][N] with a nesting mask, using
// integral images for box counts and signatures.

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

// number of set bits i0..i1 (inclusive) of a row
inline int row_count(const uint64_t *r, int i0, int i1)
{
    const int k0 = i0 >> 6, k1 = i1 >> 6;
    const uint64_t m0 = ~0ull << (i0 & 63), m1 = ~0ull >> (63 - (i1 & 63));
    if (k0 == k1) return popc(r[k0] & m0 & m1);
    int c = popc(r[k0] & m0);
    for (int k = k0 + 1; k < k1; k++) c += popc(r[k]);
    return c + popc(r[k1] & m1);
}

inline bool row_any(const uint64_t *r, int i0, int i1)
{
    const int k0 = i0 >> 6, k1 = i1 >> 6;
    const uint64_t m0 = ~0ull << (i0 & 63), m1 = ~0ull >> (63 - (i1 & 63));
    if (k0 == k1) return (r[k0] & m0 & m1) != 0;
    if (r[k0] & m0) return true;
    for (int k = k0 + 1; k < k1; k++)
        if (r[k]) return true;
    return (r[k1] & m1) != 0;
}

inline void row_clear(uint64_t *r, int i0, int i1)
{
    const int k0 = i0 >> 6, k1 = i1 >> 6;
    const uint64_t m0 = ~0ull << (i0 & 63), m1 = ~0ull >> (63 - (i1 & 63));
    if (k0 == k1) {
        r[k0] &= ~(m0 & m1);
        return;
    }
    r[k0] &= ~m0;
    for (int k = k0 + 1; k < k1; k++) r[k] = 0;
    r[k1] &= ~m1;
}

// Chebyshev dilation by w cells along rows and wy cells along columns; cells
// outside the window count as clear.  t: scratch.
void dilate_bits(Bits &f, int w, int wy, std::vector<uint64_t> &t)
{
    const int nw = f.nw;
    const uint64_t tail = f.tail();
    if (w > 0) {
        t.resize((size_t)nw);
        for (int j = 0; j < f.M; j++) {
            uint64_t *r = f.row(j);
            for (int pass = 0; pass < w; pass += 63) {  // shifts of at most 63 per pass
                const int ws = std::min(63, w - pass);
                std::copy(r, r + nw, t.begin());
                for (int sft = 1; sft <= ws; sft++)
                    for (int k = 0; k < nw; k++) {
                        uint64_t up = (t[k] << sft) | (k > 0 ? t[k - 1] >> (64 - sft) : 0);
                        uint64_t dn = (t[k] >> sft) | (k + 1 < nw ? t[k + 1] << (64 - sft) : 0);
                        r[k] |= up | dn;
                    }
                r[nw - 1] &= tail;
            }
        }
    }
    if (wy > 0) {
        t.assign(f.w.begin(), f.w.end());
        for (int j = 0; j < f.M; j++) {
            uint64_t *r = f.row(j);
            for (int d = 1; d <= wy; d++) {
                if (j - d >= 0) {
                    const uint64_t *q = &t[(size_t)(j - d) * nw];
                    for (int k = 0; k < nw; k++) r[k] |= q[k];
                }
                if (j + d < f.M) {
                    const uint64_t *q = &t[(size_t)(j + d) * nw];
                    for (int k = 0; k < nw; k++) r[k] |= q[k];
                }
            }
        }
    }
}

// 64x64 bit-matrix transpose in place: bit c of a[r] <-> bit r of a[c]
// (swaps of the off-diagonal blocks of width 32, 16, ..., 1)
void transpose64(uint64_t *a)
{
    uint64_t m = 0x00000000FFFFFFFFull;
    for (int j = 32; j != 0; j >>= 1, m ^= (m << j)) {
        for (int k = 0; k < 64; k = (k + j + 1) & ~j) {
            uint64_t t = ((a[k] >> j) ^ a[k + j]) & m;
            a[k + j] ^= t;
            a[k] ^= t << j;
        }
    }
}

// T = transpose of f (T.N = f.M, T.M = f.N)
void transpose_bits(const Bits &f, Bits &T)
{
    T.reset(f.M, f.N);
    uint64_t blk[64];
    const int nbj = (f.M + 63) >> 6;
    for (int bj = 0; bj < nbj; bj++)
        for (int bi = 0; bi < f.nw; bi++) {
            for (int r = 0; r < 64; r++) {
                int j = bj * 64 + r;
                blk[r] = (j < f.M) ? f.row(j)[bi] : 0;
            }
            transpose64(blk);
            for (int c = 0; c < 64; c++) {
                int i = bi * 64 + c;
                if (i < f.N) T.row(i)[bj] = blk[c];
            }
        }
}

// Berger-Rigoutsos clustering (Sec. 3, regridding) on a flag bitmap with the
// non-nestable cells marked in U; row and column signatures of a box are bit
// counts of the bitmap and of its transpose.
struct Clusterer {
    int N, M, dim, mc;
    double eff;
    const Bits *F = nullptr, *U = nullptr;
    Bits T;                         // transpose of *F
    std::vector<Box> out;
    std::vector<long long> cs, rs;  // signature scratch (split() is not recursive)
    std::vector<Box> stack;

    void init(const Bits &flags, const Bits &unnest)
    {
        F = &flags;
        U = &unnest;
        transpose_bits(flags, T);
    }

    void run(Box b)
    {
        out.clear();
        stack.assign(1, b);
        while (!stack.empty()) {
            Box x = stack.back();
            stack.pop_back();
            Box l, r;
            if (split(x, l, r)) {
                stack.push_back(r);
                stack.push_back(l);
            }
        }
    }

    // returns true and the two halves if x must be split; false if x was
    // accepted (pushed to out) or holds no flag
    bool split(Box x, Box &L, Box &R)
    {
        rs.resize(x.j1 - x.j0 + 1);
        long long tot = 0;
        for (int j = x.j0; j <= x.j1; j++) tot += (rs[j - x.j0] = row_count(F->row(j), x.i0, x.i1));
        if (tot == 0) return false;
        cs.resize(x.i1 - x.i0 + 1);
        for (int i = x.i0; i <= x.i1; i++) cs[i - x.i0] = row_count(T.row(i), x.j0, x.j1);
        int a = 0, bb = (int)cs.size() - 1, c0 = 0, c1 = (int)rs.size() - 1;
        while (cs[a] == 0) a++;
        while (cs[bb] == 0) bb--;
        while (rs[c0] == 0) c0++;
        while (rs[c1] == 0) c1--;
        Box b{x.i0 + a, x.i0 + bb, x.j0 + c0, x.j0 + c1};
        // signatures of the shrunk box: the removed rows and columns hold no flag
        const long long *sxp = cs.data() + a, *syp = rs.data() + c0;
        long long nf = 0;
        for (int k = 0; k <= bb - a; k++) nf += sxp[k];
        int lx = b.i1 - b.i0 + 1, ly = b.j1 - b.j0 + 1;
        long long area = (long long)lx * ly;
        bool nestable = true;
        for (int j = b.j0; j <= b.j1 && nestable; j++) nestable = !row_any(U->row(j), b.i0, b.i1);
        if (nestable && (double)nf / (double)area >= eff) {
            out.push_back(b);
            return false;
        }
        int m = nestable ? mc : 1;
        int ndim = (dim == 2) ? 2 : 1;
        const long long *sig[2] = {sxp, syp};
        int los[2] = {b.i0, b.j0}, his[2] = {b.i1, b.j1};
        // (1) zero signature closest to the centre
        int bd = -1, bp = 0, bdist = 0;
        for (int d = 0; d < ndim; d++) {
            const long long *s = sig[d];
            for (int k = los[d] + 1; k < his[d]; k++) {
                if (s[k - los[d]] != 0) continue;
                int dist = std::abs(2 * k - (los[d] + his[d]));
                if (bd < 0 || dist < bdist) { bd = d; bp = k; bdist = dist; }
            }
        }
        if (bd >= 0) {
            L = b; R = b;
            if (bd == 0) { L.i1 = bp - 1; R.i0 = bp + 1; }
            else { L.j1 = bp - 1; R.j0 = bp + 1; }
            return true;
        }
        // (2) strongest sign change of the second difference
        long long bstr = -1;
        for (int d = 0; d < ndim; d++) {
            const long long *s = sig[d];
            int lo = los[d], hi = his[d];
            for (int k = lo + 1; k <= hi - 2; k++) {
                long long d0 = s[k - 1 - lo] - 2 * s[k - lo] + s[k + 1 - lo];
                long long d1 = s[k - lo] - 2 * s[k + 1 - lo] + s[k + 2 - lo];
                bool change = (d0 < 0 && d1 > 0) || (d0 > 0 && d1 < 0);
                if (!change || k - lo + 1 < m || hi - k < m) continue;
                long long str = d1 > d0 ? d1 - d0 : d0 - d1;
                int dist = std::abs(2 * k + 1 - (lo + hi));
                if (str > bstr || (str == bstr && dist < bdist)) { bstr = str; bdist = dist; bd = d; bp = k; }
            }
        }
        if (bd >= 0) {
            L = b; R = b;
            if (bd == 0) { L.i1 = bp; R.i0 = bp + 1; }
            else { L.j1 = bp; R.j0 = bp + 1; }
            return true;
        }
        // (3) bisect the longer side (x on ties), else the other one
        int order[2] = {0, 1};
        if (ndim == 2 && ly > lx) { order[0] = 1; order[1] = 0; }
        for (int q = 0; q < ndim; q++) {
            int d = order[q];
            int len = d ? ly : lx, lo = d ? b.j0 : b.i0;
            if (len / 2 < m || len - len / 2 < m) continue;
            int mid = lo + len / 2;
            L = b; R = b;
            if (d == 0) { L.i1 = mid - 1; R.i0 = mid; }
            else { L.j1 = mid - 1; R.j0 = mid; }
            return true;
        }
        out.push_back(b);
        return false;
    }
};

// separable Chebyshev dilation of a 0/1 field [M][N] by w cells in x and wy
// in y, in place, with sliding window counts (t and cnt are scratch)
constexpr size_t kPinHead = 64;          // count, bounding box and list counters ahead of the bitmap
constexpr long long kFlagItemsMax = (long long)1 << 26;  // longest (cell, block) list of the two-pass flags
constexpr size_t kPinBits = 256 << 10;   // bitmaps up to this size come back with the count

// Scratch of one error estimate: the estimate itself (the level's arena
// layout, m fields) and the buffers its kernels work in.  The caller releases
// it (errest_release) once the stream that ran the estimate has been
// synchronised: on the flag side stream the block cache orders its frees on
// the main stream, so blocks still in use there must not go back earlier.
struct ErrEstScratch {
    double *tau = nullptr, *buf = nullptr;
    unsigned long long *cfl = nullptr;
    char *meta = nullptr;
};

void errest_release(adjamr_ctx *c, ErrEstScratch &x)
{
    cput(c, x.tau);
    cput(c, x.buf);
    cput(c, x.cfl);
    cput(c, x.meta);
}

// Richardson error estimate of level l at its current time (flag modes
// ADJAMR_FLAG_ERROR, _RICHARDSON): into x.tau.  Every patch is
// extended to even extents with a ring of 4 cells (values as ghost cells get
// them), advanced two steps of dt by the step kernel (the first over the
// region widened by 2, the second over the even patch), coarsened by 2 and
// advanced one step of 2 dt (dt/dx unchanged), and tau = (coarsened two-step
// state - coarse step) / 6 on every 2^d block.
adjamr_status error_estimate(adjamr_ctx *c, int l, ErrEstScratch &x)
{
    Level &L = c->L[l];
    const adjamr_params &P = c->P;
    const int dim = P.dim, m = c->m;
    if (L.patches.empty()) return ADJAMR_OK;
    const int kx = (dim == 2) ? 16 : 128, ky = (dim == 2) ? 8 : 1;
    std::vector<ErrEstPatch> ep;
    std::vector<long long> epre{0}, cpre{0};
    std::vector<PatchDesc> p1, p2, pc;
    std::vector<WorkItem> w1, w2, wc;
    const double dtdx = L.dt / L.dx, dtdy = (dim == 2) ? L.dt / L.dy : 0.0;
    auto tiles = [&](std::vector<WorkItem> &w, int k, int nx, int ny) {
        const int tx = tile_count(nx, kx), ty = tile_count(ny, ky);
        for (int b = 0; b < ty; b++)
            for (int a = 0; a < tx; a++)
                w.push_back({k, tile_off(nx, tx, a), tile_off(ny, ty, b), (unsigned short)tile_len(nx, tx, a),
                             (unsigned short)tile_len(ny, ty, b)});
    };
    long long nE = 0, nC = 0;
    for (const HPatch &h : L.patches) {
        ErrEstPatch e{};
        e.ilo = h.ilo;
        e.jlo = h.jlo;
        e.nx = h.nx;
        e.ny = h.ny;
        e.ne = h.nx + (h.nx & 1);
        e.me = (dim == 2) ? h.ny + (h.ny & 1) : 1;
        e.asx = h.sx;
        e.abase = h.base;
        const int ex = e.ne + 8, ey = (dim == 2) ? e.me + 8 : 1;
        const int cx = e.ne / 2 + 4, cy = (dim == 2) ? e.me / 2 + 4 : 1;
        e.ebase = nE;
        e.cbase = nC;
        PatchDesc d{};
        d.dtdx = dtdx;
        d.dtdy = dtdy;
        d.hx = 0.5 * dtdx;
        d.hy = 0.5 * dtdy;
        // first fine step: the even patch widened by 2 cells, ring = E's outer 2
        d.ilo = h.ilo - 2;
        d.jlo = (dim == 2) ? h.jlo - 2 : 0;
        d.nx = e.ne + 4;
        d.ny = (dim == 2) ? e.me + 4 : 1;
        d.sx = ex;
        d.sy = ey;
        d.base = e.ebase;
        tiles(w1, (int)p1.size(), d.nx, d.ny);
        p1.push_back(d);
        // second fine step: the even patch, its ring = the first step's border
        d.ilo = h.ilo;
        d.jlo = h.jlo;
        d.nx = e.ne;
        d.ny = e.me;
        d.sy = (dim == 2) ? e.me + 4 : 1;
        d.base = e.ebase + ((dim == 2) ? 2LL * ex : 0LL) + 2;
        tiles(w2, (int)p2.size(), d.nx, d.ny);
        p2.push_back(d);
        // coarse step (2 dt over 2 dx: the same dt/dx)
        d.nx = e.ne / 2;
        d.ny = (dim == 2) ? e.me / 2 : 1;
        d.sx = cx;
        d.sy = cy;
        d.base = e.cbase;
        tiles(wc, (int)pc.size(), d.nx, d.ny);
        pc.push_back(d);
        ep.push_back(e);
        nE += (long long)ex * ey;
        nC += (long long)cx * cy;
        epre.push_back(nE);
        cpre.push_back(nC);
    }
    std::vector<size_t> offs;
    char *meta = nullptr;
    CKR(c, upload_packed(c,
                         {{ep.data(), sizeof(ErrEstPatch) * ep.size()},
                          {epre.data(), sizeof(long long) * epre.size()},
                          {cpre.data(), sizeof(long long) * cpre.size()},
                          {p1.data(), sizeof(PatchDesc) * p1.size()},
                          {p2.data(), sizeof(PatchDesc) * p2.size()},
                          {pc.data(), sizeof(PatchDesc) * pc.size()},
                          {w1.data(), sizeof(WorkItem) * w1.size()},
                          {w2.data(), sizeof(WorkItem) * w2.size()},
                          {wc.data(), sizeof(WorkItem) * wc.size()}},
                         &meta, offs));
    const int per = 2 * m + c->naux + c->nmed;
    x.meta = meta;
    cudaError_t ea = cget(c, &x.buf, (size_t)per * (nE + nC));
    if (ea == cudaSuccess) ea = cget(c, &x.cfl, 1);
    if (ea == cudaSuccess) ea = cget(c, &x.tau, (size_t)m * L.ncell);
    if (ea != cudaSuccess) {
        c->err = std::string("error estimate: ") + cudaGetErrorString(ea);
        return ADJAMR_ECUDA;
    }
    double *buf = x.buf, *t = x.tau;
    unsigned long long *cfl = x.cfl;
    ErrEstArgs a{};
    a.ep = reinterpret_cast<const ErrEstPatch *>(meta + offs[0]);
    a.eprefix = reinterpret_cast<const long long *>(meta + offs[1]);
    a.cprefix = reinterpret_cast<const long long *>(meta + offs[2]);
    a.np = (int)ep.size();
    a.dim = dim;
    a.m = m;
    a.eqn = P.eqn;
    a.nE = nE;
    a.nC = nC;
    a.E = buf;
    a.F = a.E + (size_t)m * nE;
    a.auxE = a.F + (size_t)m * nE;
    a.medE = a.auxE + (size_t)c->naux * nE;
    a.C = a.medE + (size_t)c->nmed * nE;
    a.C1 = a.C + (size_t)m * nC;
    a.auxC = a.C1 + (size_t)m * nC;
    a.medC = a.auxC + (size_t)c->naux * nC;
    const int *oc = nullptr;
    const double *qo = nullptr, *qn = nullptr;
    long long sc = 0;
    int r = 1, k = 0;
    LevelIdx gc = idx_of(c, l);
    if (l > 0) {
        Level &C = c->L[l - 1];
        oc = C.d_owner;
        gc = idx_of(c, l - 1);
        qo = C.q[C.cur];
        qn = C.q[1 - C.cur];
        sc = C.ncell;
        r = P.ratio[l - 1];
        k = (int)(L.nstep - C.nstep * r);
    }
    cudaError_t e = launch_errest_fill(a, idx_of(c, l), L.d_owner, L.q[L.cur], L.ncell, oc, gc, r, qo, qn, sc, k,
                                       L.d_med, geom_of(c, l), c->d_err, c->s);
    const PatchDesc *d1 = reinterpret_cast<const PatchDesc *>(meta + offs[3]);
    const PatchDesc *d2 = reinterpret_cast<const PatchDesc *>(meta + offs[4]);
    const PatchDesc *dc = reinterpret_cast<const PatchDesc *>(meta + offs[5]);
    if (e == cudaSuccess)
        e = launch_step(dim, P.eqn, kx, ky, a.E, a.F, a.auxE, nE, d1,
                        reinterpret_cast<const WorkItem *>(meta + offs[6]), (int)w1.size(), 0, cfl, c->s);
    if (e == cudaSuccess)
        e = launch_step(dim, P.eqn, kx, ky, a.F, a.E, a.auxE, nE, d2,
                        reinterpret_cast<const WorkItem *>(meta + offs[7]), (int)w2.size(), 0, cfl, c->s);
    if (e == cudaSuccess)
        e = launch_step(dim, P.eqn, kx, ky, a.C, a.C1, a.auxC, nC, dc,
                        reinterpret_cast<const WorkItem *>(meta + offs[8]), (int)wc.size(), 0, cfl, c->s);
    if (e == cudaSuccess) e = launch_errest_tau(a, L.d_prefix, L.ninterior, t, L.ncell, c->s);
    c->st.kernel_launches += 6;
    if (e != cudaSuccess) {
        c->err = std::string("error estimate: ") + cudaGetErrorString(e);
        return ADJAMR_ECUDA;
    }
    return ADJAMR_OK;
}

adjamr_status flag_dense(adjamr_ctx *c, int l, double tol, uint64_t *d_bits, int pitch64, unsigned char *d_patchflags,
                         long long *nflag_out, int *bbox_out = nullptr);
adjamr_status flag_readback(adjamr_ctx *c, int l, uint64_t *d_bits, int pitch64, bool twopass, long long *nflag_out,
                            int *bbox_out);

// work list of the two-pass flags with room for n (cell, block) pairs
adjamr_status grow_flag_list(adjamr_ctx *c, long long n)
{
    cput(c, c->d_fitems);
    c->fcap = 0;
    CKR(c, cget(c, &c->d_fitems, (size_t)n));
    c->fcap = n;
    return ADJAMR_OK;
}

// Rebuild levels base+1 .. nlevels-1 top-down (Sec. 3, regridding).
void harvest_timing(adjamr_ctx *c);

// Proper-nesting distance of a refinement by r, in cells of the coarser
// level: the ghost ring of 2 fine cells needs 2; the error estimate's ring of
// 4 fine cells (flag modes ADJAMR_FLAG_ERROR, _RICHARDSON) ceil(4 / r) + 1, so that its
// interpolation stencils stay on the coarser level.
int nest_width(const adjamr_ctx *c, int r)
{
    int nw = 2;
    if ((c->P.flag_mode == ADJAMR_FLAG_ERROR || c->P.flag_mode == ADJAMR_FLAG_RICHARDSON) && r > 0)
        nw = std::max(nw, (4 + r - 1) / r + 1);
    return nw;
}

adjamr_status regrid_body(adjamr_ctx *c, int base, int init, bool side_flags = false);

double ms_since(std::chrono::steady_clock::time_point t)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

adjamr_status build_reflux(adjamr_ctx *c, int base);

adjamr_status regrid_from(adjamr_ctx *c, int base, int init, bool side_flags = false)
{
    c->st.regrids++;
    auto t0 = std::chrono::steady_clock::now();
    adjamr_status st = regrid_body(c, base, init, side_flags);
    if (st == ADJAMR_OK) st = build_reflux(c, base);
    c->st.regrid_host_ms += ms_since(t0);
    return st;
}

// Conservation fix-up tables of levels base .. nlevels - 1 (their layouts
// or the layouts of the next finer levels changed).  Coarse role of level
// l: every uncovered cell beside a level-(l + 1) patch, found by walking the
// ring of cells around each fine patch's footprint; side s of that cell
// faces the patch and gets record id 4 e + s.  Fine role of level l: every
// patch-edge cell whose neighbour across side s is inside the domain and in
// no patch of the level; its coarse cell C (the neighbour divided by r) is a
// coarse-role entry e_C of level l - 1 with side s ^ 1 facing this patch,
// and the fine record id is (4 e_C + (s ^ 1)) nseg + (the cell's offset
// along that side inside C).
adjamr_status build_reflux(adjamr_ctx *c, int base)
{
    const adjamr_params &P = c->P;
    if (!P.reflux) return ADJAMR_OK;
    const int nl = P.nlevels, dim = P.dim, ns = dim == 2 ? 4 : 2;
    for (int l = base; l < nl; l++) reflux_release(c, c->L[l]);
    std::vector<std::vector<RefluxCell>> ent(nl);
    auto entry_of = [&](int l, int I, int J) -> int {
        Level &L = c->L[l];
        const long long key = (long long)J * L.N + I;
        auto it = L.rkey.find(key);
        if (it != L.rkey.end()) return it->second;
        const int k = find_patch(L, I, J);
        if (k < 0) return -1;
        RefluxCell rc;
        rc.idx = cell_of(c, L.patches[k], I - L.patches[k].ilo, J - L.patches[k].jlo);
        for (int q = 0; q < 4; q++) rc.c[q] = rc.f[q] = -1;
        const int e = (int)ent[l].size();
        ent[l].push_back(rc);
        L.rkey.emplace(key, e);
        return e;
    };
    for (int l = base; l + 1 < nl; l++) {
        Level &L = c->L[l], &F = c->L[l + 1];
        if (L.patches.empty() || F.patches.empty()) continue;
        const int r = P.ratio[l];
        auto visit = [&](int I, int J, int side) -> bool {
            if (I < 0 || I >= L.N || J < 0 || J >= L.M) return true;
            if (find_patch(F, I * r, J * r) >= 0) return true;  // covered: not an interface
            const int e = entry_of(l, I, J);
            if (e < 0) return false;
            ent[l][e].c[side] = 4 * e + side;
            return true;
        };
        bool ok = true;
        for (const HPatch &fp : F.patches) {
            const int a0 = fp.ilo / r, a1 = (fp.ilo + fp.nx) / r - 1;
            const int b0 = dim == 2 ? fp.jlo / r : 0, b1 = dim == 2 ? (fp.jlo + fp.ny) / r - 1 : 0;
            for (int J = b0; J <= b1; J++) ok = visit(a0 - 1, J, 1) && visit(a1 + 1, J, 0) && ok;
            if (dim == 2)
                for (int I = a0; I <= a1; I++) ok = visit(I, b0 - 1, 3) && visit(I, b1 + 1, 2) && ok;
        }
        if (!ok) {
            c->err = "refluxing: a cell beside a level-" + std::to_string(l + 1) + " patch is not a level-" +
                     std::to_string(l) + " cell";
            return ADJAMR_ENEST;
        }
        L.nrcoarse = (int)ent[l].size();
    }
    for (int l = std::max(base, 1); l < nl; l++) {
        Level &L = c->L[l], &C = c->L[l - 1];
        if (L.patches.empty() || C.nrcoarse == 0) continue;
        const int r = P.ratio[l - 1], nseg = dim == 2 ? r : 1;
        const long long nfrec = (long long)C.nrcoarse * 4 * nseg;
        std::vector<long long> fidx((size_t)nfrec, -1);
        for (const HPatch &p : L.patches)
            for (int j = 0; j < p.ny; j++)
                for (int i = 0; i < p.nx; i++) {
                    if (i > 0 && i < p.nx - 1 && (dim == 1 || (j > 0 && j < p.ny - 1))) continue;
                    const int I = p.ilo + i, J = p.jlo + j;
                    for (int sd = 0; sd < ns; sd++) {
                        const int nI = I + (sd == 0 ? -1 : sd == 1 ? 1 : 0);
                        const int nJ = J + (sd == 2 ? -1 : sd == 3 ? 1 : 0);
                        const int li = nI - p.ilo, lj = nJ - p.jlo;
                        if (li >= 0 && li < p.nx && lj >= 0 && lj < p.ny) continue;
                        if (nI < 0 || nI >= L.N || nJ < 0 || nJ >= L.M) continue;
                        if (find_patch(L, nI, nJ) >= 0) continue;
                        const int Ci = nI / r, Cj = dim == 2 ? nJ / r : 0, cs = sd ^ 1;
                        auto it = C.rkey.find((long long)Cj * C.N + Ci);
                        const int ec = it == C.rkey.end() ? -1 : it->second;
                        if (ec < 0 || ec >= C.nrcoarse) {
                            c->err = "refluxing: no coarse record beside a level-" + std::to_string(l) + " patch";
                            return ADJAMR_ENEST;
                        }
                        const int seg = dim == 1 ? 0 : (sd < 2 ? J - Cj * r : I - Ci * r);
                        const long long fr = ((long long)ec * 4 + cs) * nseg + seg;
                        fidx[(size_t)fr] = cell_of(c, p, i, j);
                        const int e = entry_of(l, I, J);
                        ent[l][e].f[sd] = (int)fr;
                    }
                }
        if (C.nfrec != nfrec || !C.d_fidx) {
            cput(c, C.d_fidx);
            cput(c, C.d_lf);
            cput(c, C.d_lc);
            CKR(c, cget(c, &C.d_fidx, (size_t)nfrec));
            CKR(c, cget(c, &C.d_lf, (size_t)r * nfrec * 4));
            CKR(c, cget(c, &C.d_lc, (size_t)C.nrcoarse * 8));
            C.nfrec = nfrec;
        }
        CKR(c, upload_now(c, C.d_fidx, fidx));
    }
    for (int l = base; l < nl; l++) {
        Level &L = c->L[l];
        L.nrcell = (int)ent[l].size();
        if (L.nrcell == 0) continue;
        CKR(c, cget(c, &L.d_rcells, ent[l].size()));
        CKR(c, upload_now(c, L.d_rcells, ent[l]));
        CKR(c, cget(c, &L.d_rmap, (size_t)L.ncell));
        CKR(c, cudaMemsetAsync(L.d_rmap, 0xff, (size_t)L.ncell * sizeof(int), c->s));
        CKR(c, launch_reflux_map(L.d_rcells, L.nrcell, L.d_rmap, c->s));
        c->st.kernel_launches++;
    }
    return ADJAMR_OK;
}

// fix-up records of a step of level l at substep `sub` of the coarser step
RefluxArgs reflux_args(adjamr_ctx *c, int l, int sub)
{
    RefluxArgs rx{};
    Level &L = c->L[l];
    if (!c->P.reflux || L.nrcell == 0) return rx;
    rx.rmap = L.d_rmap;
    rx.cells = L.d_rcells;
    rx.lc = L.d_lc;
    if (l > 0) {
        rx.lf = c->L[l - 1].d_lf;
        rx.nfrec = c->L[l - 1].nfrec;
    }
    rx.sub = sub;
    return rx;
}

// the fix-up of level l's coarse-role cells after its finer level's substeps
// and average-down (Sec. 3, AMR after Berger and LeVeque)
adjamr_status reflux_apply(adjamr_ctx *c, int l)
{
    Level &L = c->L[l], &F = c->L[l + 1];
    if (!c->P.reflux || L.nrcoarse == 0) return ADJAMR_OK;
    RefluxApply a{};
    a.cells = L.d_rcells;
    a.ncoarse = L.nrcoarse;
    a.qc_old = L.q[L.cur];
    a.qc_new = L.q[1 - L.cur];
    a.medc = L.med;
    a.sc = L.ncell;
    a.lc = L.d_lc;
    a.lf = L.d_lf;
    a.nfrec = L.nfrec;
    a.fidx = L.d_fidx;
    a.medf = F.med;
    a.sf = F.ncell;
    a.r = c->P.ratio[l];
    a.nseg = c->P.dim == 2 ? a.r : 1;
    a.w = 1.0 / (double)(a.r * a.nseg);
    a.dtdx = L.dt / L.dx;
    a.dtdy = c->P.dim == 2 ? L.dt / L.dy : 0.0;
    a.err = c->d_err;
    CKR(c, launch_reflux_apply(c->P.dim, c->P.eqn, a, c->s));
    c->st.kernel_launches++;
    return ADJAMR_OK;
}

// flags of level lev into d_flagbuf (count, bounding box and bitmap read back)
adjamr_status regrid_flags(adjamr_ctx *c, int lev, long long *nf, int *bb)
{
    const Level &C = c->L[lev];
    const int pitch64 = (C.N + 63) >> 6;
    size_t nb = (size_t)pitch64 * C.M * sizeof(uint64_t);
    if (c->flagbuf_bytes < nb) {
        dfree(c->d_flagall, c->s);
        c->d_flagbuf = nullptr;
        CKR(c, dalloc(&c->d_flagall, (kPinHead + nb) / sizeof(uint64_t), c->s));
        c->d_flagbuf = c->d_flagall + kPinHead / sizeof(uint64_t);
        c->flagbuf_bytes = nb;
    }
    // one memset clears the head (count, box, list counters) and the bitmap
    CKR(c, cudaMemsetAsync(c->d_flagall, 0, kPinHead + nb, c->s));
    return flag_dense(c, lev, c->P.tol, c->d_flagbuf, pitch64, nullptr, nf, bb);
}

adjamr_status regrid_body(adjamr_ctx *c, int base, int init, bool side_flags)
{
    const adjamr_params &P = c->P;
    bool coarser_rebuilt = false;  // level lev was rebuilt earlier in this call
    for (int lev = base; lev < P.nlevels - 1; lev++) {
        Level &C = c->L[lev];
        Level &F = c->L[lev + 1];
        const int r = P.ratio[lev], N = C.N, M = C.M, dim = P.dim;
        const long long tick = C.nstep * c->T[lev];
        // ---- adjoint flags of level lev on its index space (device bitmap) ----
        const int pitch64 = (N + 63) >> 6;
        long long nf = 0;
        int bb[4];
        auto tp = std::chrono::steady_clock::now();
        if (lev == base && side_flags) {
            // on the side stream, after the work queued before ev_flag
            CKR(c, cudaStreamWaitEvent(c->s_flag, c->ev_flag, 0));
            std::swap(c->s, c->s_flag);
            c->on_side = true;
            const adjamr_status fs = regrid_flags(c, lev, &nf, bb);
            c->on_side = false;
            std::swap(c->s, c->s_flag);
            TRY(fs);
            // later work on s that reuses the flag buffers comes after them
            CKR(c, cudaEventRecord(c->ev_flag, c->s_flag));
            CKR(c, cudaStreamWaitEvent(c->s, c->ev_flag, 0));
        } else {
            TRY(regrid_flags(c, lev, &nf, bb));
        }
        c->st.regrid_phase_ms[0] += ms_since(tp);
        harvest_timing(c);
        auto tc = std::chrono::steady_clock::now();
        std::vector<Box> fin;
        if (nf > 0) {
            // Window = bounding box of the flags grown by the buffer and the
            // nesting distance, clipped to the domain, its first column on a
            // word boundary.  Clustering starts by shrinking to the flags'
            // bounding box, so any such window gives the same boxes as the
            // whole index space.
            const int nw = nest_width(c, r);
            const int grow = P.buffer + nw;
            const int wi0 = std::max(0, bb[0] - grow) & ~63, wi1 = std::min(N - 1, bb[1] + grow);
            const int wj0 = (dim == 2) ? std::max(0, bb[2] - grow) : 0;
            const int wj1 = (dim == 2) ? std::min(M - 1, bb[3] + grow) : 0;
            const int k0 = wi0 >> 6, nwords = (wi1 >> 6) - k0 + 1;
            const int wN = std::min(N - wi0, 64 * nwords), wM = wj1 - wj0 + 1;
            Bits &fl = c->h_fl, &unc = c->h_unc;
            fl.reset(wN, wM);
            tp = std::chrono::steady_clock::now();
            if (c->pin_has_bits) {
                const uint64_t *all = reinterpret_cast<const uint64_t *>(c->h_pin + kPinHead);
                for (int j = 0; j < wM; j++)
                    std::memcpy(fl.row(j), all + (size_t)(wj0 + j) * pitch64 + k0, (size_t)fl.nw * sizeof(uint64_t));
            } else {
                CKR(c, cudaMemcpy2DAsync(fl.w.data(), (size_t)fl.nw * sizeof(uint64_t),
                                         c->d_flagbuf + (size_t)wj0 * pitch64 + k0, (size_t)pitch64 * sizeof(uint64_t),
                                         (size_t)fl.nw * sizeof(uint64_t), (size_t)wM, cudaMemcpyDeviceToHost, c->s));
                CKR(c, cudaStreamSynchronize(c->s));
            }
            double wcopy = ms_since(tp);
            c->st.regrid_phase_ms[1] += wcopy;
            c->st.cluster_host_ms -= wcopy;
            auto ts = std::chrono::steady_clock::now();
            // buffer, nesting mask (every cell within nw cells covered by this level)
            dilate_bits(fl, P.buffer, dim == 2 ? P.buffer : 0, c->h_tmp);
            unc.reset(wN, wM);
            for (int j = 0; j < wM; j++) {
                uint64_t *r = unc.row(j);
                std::fill(r, r + unc.nw, ~0ull);
                r[unc.nw - 1] &= unc.tail();
            }
            for (const HPatch &p : C.patches) {
                int a0 = std::max(p.ilo, wi0), a1 = std::min(p.ilo + p.nx - 1, wi0 + wN - 1);
                int b0 = std::max(p.jlo, wj0), b1 = std::min(p.jlo + p.ny - 1, wj1);
                if (a0 > a1 || b0 > b1) continue;
                for (int j = b0; j <= b1; j++) row_clear(unc.row(j - wj0), a0 - wi0, a1 - wi0);
            }
            // cells beyond the window but inside the domain: the window reaches
            // nw cells past every flag the buffer can create, so they never
            // decide a flagged cell's nesting
            dilate_bits(unc, nw, dim == 2 ? nw : 0, c->h_tmp);
            for (size_t k = 0; k < fl.w.size(); k++) fl.w[k] &= ~unc.w[k];
            c->st.cluster_phase_ms[0] += ms_since(ts);
            ts = std::chrono::steady_clock::now();
            static thread_local Clusterer cl;  // reused scratch (one context per host thread)
            cl.N = wN;
            cl.M = wM;
            cl.dim = dim;
            cl.mc = (P.min_patch + r - 1) / r;
            cl.eff = P.cluster_eff;
            cl.init(fl, unc);
            c->st.cluster_phase_ms[1] += ms_since(ts);
            ts = std::chrono::steady_clock::now();
            cl.run(Box{0, wN - 1, 0, wM - 1});
            c->st.cluster_phase_ms[2] += ms_since(ts);
            ts = std::chrono::steady_clock::now();
            for (Box b : cl.out) {
                b.i0 += wi0;
                b.i1 += wi0;
                b.j0 += wj0;
                b.j1 += wj0;
                int lx = b.i1 - b.i0 + 1, ly = b.j1 - b.j0 + 1;
                int px = 1, py = 1;
                while (r * ((lx + px - 1) / px) > P.max_patch) px++;
                if (dim == 2)
                    while (r * ((ly + py - 1) / py) > P.max_patch) py++;
                for (int bj = 0; bj < py; bj++)
                    for (int bi = 0; bi < px; bi++) {
                        Box s;
                        s.i0 = b.i0 + part_off(lx, px, bi);
                        s.i1 = s.i0 + part_len(lx, px, bi) - 1;
                        s.j0 = (dim == 2) ? b.j0 + part_off(ly, py, bj) : 0;
                        s.j1 = (dim == 2) ? s.j0 + part_len(ly, py, bj) - 1 : 0;
                        fin.push_back(s);
                    }
            }
            std::sort(fin.begin(), fin.end(), [](const Box &a, const Box &b) {
                return a.j0 != b.j0 ? a.j0 < b.j0 : a.i0 < b.i0;
            });
            c->st.cluster_phase_ms[3] += ms_since(ts);
        }
        c->st.cluster_host_ms += ms_since(tc);
        c->st.regrid_phase_ms[2] = c->st.cluster_host_ms;
        // ---- new level lev+1 (refined boxes) ----
        std::vector<Box> fb;
        for (const Box &b : fin)
            fb.push_back(Box{b.i0 * r, (b.i1 + 1) * r - 1, dim == 2 ? b.j0 * r : 0, dim == 2 ? (b.j1 + 1) * r - 1 : 0});
        // The boxes the level has now, over a coarser level this call left as
        // it was: the rebuild would give every cell its old value at its old
        // storage index (new patches take the old fine values wherever they
        // exist), the same ghost and average-down maps and the same work
        // lists, so the level stays as it is.  An empty level stays empty.
        if (!init && !coarser_rebuilt && F.d_owner && same_layout(F, fb)) {
            F.nstep = C.nstep * r;
            if (F.patches.empty()) F.cur = 0;
            c->rebuilt_tick[lev + 1] = tick;
            c->st.level_rebuilds_skipped++;
            if (F.patches.empty()) break;
            continue;
        }
        coarser_rebuilt = true;
        Level old;
        std::swap(old.patches, F.patches);
        std::swap(old.buckets, F.buckets);
        old.N = F.N; old.M = F.M; old.bs = F.bs; old.nbx = F.nbx; old.nby = F.nby;
        old.q[0] = F.q[0]; old.q[1] = F.q[1]; old.ncell = F.ncell; old.cur = F.cur; old.d_arena = F.d_arena;
        F.d_arena = nullptr;
        old.aux = F.aux; old.med = F.med; old.d_patches = F.d_patches; old.d_work = F.d_work;
        old.d_ghost = F.d_ghost; old.d_avg = F.d_avg; old.d_prefix = F.d_prefix;
        old.d_gprefix = F.d_gprefix; old.d_sprefix = F.d_sprefix; old.d_aprefix = F.d_aprefix; old.d_owner = F.d_owner;
        old.d_meta = F.d_meta;
        F.d_meta = nullptr;
        F.q[0] = F.q[1] = nullptr;
        F.aux = F.med = nullptr;
        F.d_patches = nullptr; F.d_work = nullptr; F.d_ghost = nullptr; F.d_avg = nullptr; F.d_prefix = nullptr;
        F.d_gprefix = F.d_sprefix = F.d_aprefix = nullptr;
        F.d_owner = nullptr;
        tp = std::chrono::steady_clock::now();
        // The level's builders go out as two launches (launch_rebuild), except
        // under substep launches, whose work list reads the new owner map as it
        // is built.  Recording stops, and a record left by an error is dropped,
        // on every way out of this iteration.
        struct PendOff {
            adjamr_ctx *c;
            ~PendOff() { pend_clear(c); }
        } pend_off{c};
        c->pend_on = c->lmode[lev + 1] != ADJAMR_LAUNCH_SUBSTEPS;
        TRY(alloc_level(c, lev + 1, fb));
        c->st.regrid_phase_ms[3] += ms_since(tp);
        tp = std::chrono::steady_clock::now();
        F.cur = 0;
        F.nstep = C.nstep * r;
        TRY(fill_aux(c, lev + 1, &old));
        if (!F.patches.empty()) {
            if (init && P.qinit) {
                long long n = F.ninterior;
                std::vector<double> xc(n), yc(n), qv((size_t)n * c->m);
                long long o = 0;
                for (const HPatch &p : F.patches)
                    for (int j = 0; j < p.ny; j++)
                        for (int i = 0; i < p.nx; i++, o++) {
                            xc[o] = P.lo[0] + ((double)(p.ilo + i) + 0.5) * F.dx;
                            yc[o] = (dim == 2) ? P.lo[1] + ((double)(p.jlo + j) + 0.5) * F.dy : 0.0;
                        }
                P.qinit(lev + 1, (int)n, xc.data(), yc.data(), qv.data(), P.qinit_user);
                std::vector<double> host((size_t)c->m * F.ncell, 0.0);
                o = 0;
                for (const HPatch &p : F.patches)
                    for (int j = 0; j < p.ny; j++)
                        for (int i = 0; i < p.nx; i++, o++)
                            for (int f = 0; f < c->m; f++) host[(size_t)f * F.ncell + cell_of(c, p, i, j)] = qv[(size_t)f * n + o];
                CKR(c, cudaMemcpyAsync(F.q[0], host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
            } else {
                TRY(run_builder(c, InitNewArgs{F.d_patches, F.d_prefix, (int)F.patches.size(), F.ninterior,
                                               idx_of(c, lev + 1), c->m, F.q[0], F.ncell,
                                               old.patches.empty() ? nullptr : old.d_owner,
                                               old.q[0] ? old.q[old.cur] : F.q[0], old.ncell, C.d_owner,
                                               idx_of(c, lev), C.q[C.cur], C.ncell, r, c->d_err}));
            }
            TRY(build_ghost_map(c, lev + 1));
            TRY(build_avg_map(c, lev + 1));
        }
        // (before the old arena goes back to the cache: the new cells read it)
        if (c->pend_on) TRY(flush_rebuild(c));
        c->st.regrid_phase_ms[4] += ms_since(tp);
        tp = std::chrono::steady_clock::now();
        free_level(c, old);
        c->st.regrid_phase_ms[5] += ms_since(tp);
        c->rebuilt_tick[lev + 1] = tick;
        c->st.level_rebuilds++;
        if (F.patches.empty()) {
            for (int q = lev + 2; q < P.nlevels; q++) free_level(c, c->L[q]);
            break;
        }
    }
    return ADJAMR_OK;
}

constexpr int kFlagBlocksPerThread = 1;
constexpr long long kFlagOnePassMax = 1ll << 16;  // (cell, snapshot block) pairs decided in one pass

// Per-column and per-row bilinear tables of the attached adjoint grid for
// level l (the same arithmetic as the flag kernel's per-cell setup: cell
// centre x = lo + (I + 1/2) dx; u = (x - lo) / dxa; stencil index and
// weight from u - 1/2 clamped to the outermost centres; containing cell
// floor(u) clamped).  Rebuilt when the adjoint grid changes.
adjamr_status flag_tables(adjamr_ctx *c, int l)
{
    const adjamr_params &P = c->P;
    Level &L = c->L[l];
    const int ax = c->adj->ax, ay = c->adj->ay;
    if (c->d_ftab[l] && c->ftab_ax[l] == ax && c->ftab_ay[l] == ay) return ADJAMR_OK;
    cput(c, c->d_ftab[l]);
    const int N = L.N, M = (P.dim == 2) ? L.M : 1;
    std::vector<int> ta(N), tac(N), tb(M), tbc(M);
    std::vector<double> twx(N), twy(M);
    auto axis = [](double x, double lo, double hi, int na, int &a, double &w, int &acell) {
        double dxa = (hi - lo) / (double)na;
        double u = (x - lo) / dxa;
        double xi = u - 0.5;
        xi = std::fmin(std::fmax(xi, 0.0), (double)(na - 1));
        a = (int)std::floor(xi);
        if (a > na - 2) a = na - 2;
        if (a < 0) a = 0;
        w = xi - (double)a;
        acell = (int)std::floor(u);
        if (acell < 0) acell = 0;
        if (acell > na - 1) acell = na - 1;
    };
    for (int I = 0; I < N; I++) {
        double x = P.lo[0] + ((double)I + 0.5) * L.dx;
        axis(x, P.lo[0], P.hi[0], ax, ta[I], twx[I], tac[I]);
    }
    for (int J = 0; J < M; J++) {
        if (P.dim == 2) {
            double y = P.lo[1] + ((double)J + 0.5) * L.dy;
            axis(y, P.lo[1], P.hi[1], ay, tb[J], twy[J], tbc[J]);
        } else {
            tb[J] = tbc[J] = 0;
            twy[J] = 0.0;
        }
    }
    std::vector<size_t> offs;
    CKR(c, upload_packed(c, {{ta.data(), sizeof(int) * N}, {tac.data(), sizeof(int) * N}, {twx.data(), sizeof(double) * N},
                             {tb.data(), sizeof(int) * M}, {tbc.data(), sizeof(int) * M}, {twy.data(), sizeof(double) * M}},
                         &c->d_ftab[l], offs));
    for (int k = 0; k < 6; k++) c->ftab_off[l][k] = offs[k];
    c->ftab_ax[l] = ax;
    c->ftab_ay[l] = ay;
    return ADJAMR_OK;
}

adjamr_status ghost_fill(adjamr_ctx *c, int l, int k, bool early = false, bool stored = false);

adjamr_status flag_dense(adjamr_ctx *c, int l, double tol, uint64_t *d_bits, int pitch64, unsigned char *d_patchflags,
                         long long *nflag_out, int *bbox_out)
{
    Level &L = c->L[l];
    *nflag_out = 0;
    if (L.patches.empty()) return ADJAMR_OK;
    const adjamr_params &P = c->P;
    FlagArgs a;
    std::memset(&a, 0, sizeof a);
    a.q = L.q[L.cur];
    a.stride = L.ncell;
    a.patches = L.d_patches;
    a.cell_prefix = L.d_prefix;
    a.np = (int)L.patches.size();
    a.dim = P.dim;
    a.m = c->m;
    a.mode = P.flag_mode;
    a.ncells = L.ninterior;
    a.lo0 = P.lo[0]; a.lo1 = P.lo[1]; a.hi0 = P.hi[0]; a.hi1 = P.hi[1];
    a.dx = L.dx; a.dy = L.dy;
    a.tol = tol;
    a.flags_patch = d_patchflags;
    a.flags_bits = reinterpret_cast<unsigned long long *>(d_bits);
    a.pitch64 = pitch64;
    a.N = L.N;
    // head: count (word 0), bounding box (words 1-2), list counters (words 3-4)
    unsigned long long *head = d_bits ? reinterpret_cast<unsigned long long *>(d_bits) - kPinHead / 8 : c->d_fhead;
    a.count = head;
    double t = P.t0 + (double)L.nstep * L.dt;
    double T = std::fmin(t + (P.tf - P.ts), P.tf);
    a.t = t;
    a.T = T;
    a.t0 = P.t0;
    if (c->adj) {
        int S = c->adj->S;
        a.S = S;
        a.snaps = c->adj->d_snaps;
        a.wet = c->adj->d_wet;
        a.ax = c->adj->ax;
        a.ay = c->adj->ay;
        a.dts = (P.tf - P.t0) / (double)(S - 1);
        int nlo = 0, nhi = S - 1;
        for (int n = 0; n < S; n++)
            if (P.t0 + (double)n * a.dts <= t) nlo = n;
        for (int n = S - 1; n >= 0; n--)
            if (P.t0 + (double)n * a.dts >= T) nhi = n;
        a.nlo = nlo;
        a.nhi = nhi;
        a.bmax = c->adj->d_bmax;
    } else {
        a.S = 0;
        a.ax = a.ay = 1;
    }
    a.bbox = reinterpret_cast<int *>(head + 1);
    unsigned long long *fctr = head + 3;
    // (a regrid's head was cleared with its bitmap)
    if (!d_bits) CKR(c, cudaMemsetAsync(head, 0, kPinHead, c->s));
    // regrid flags (dense only, bracket max, block maxima present): one thread
    // per (cell, group of snapshot blocks) over the level's index space
    if (P.flag_mode == ADJAMR_FLAG_DIFFERENCE) {
        // centred differences read the ghost ring of the current state
        const int sub = l > 0 ? (int)(L.nstep - c->L[l - 1].nstep * P.ratio[l - 1]) : 0;
        TRY(ghost_fill(c, l, sub));
    }
    // error flagging: the bracket rule on the error estimate instead of the state;
    // Richardson flagging: the estimate's largest component
    // (released on every return path, all of which come after the stream's
    // synchronisation in flag_readback or after an error)
    ErrEstScratch ex;
    struct Release {
        adjamr_ctx *c;
        ErrEstScratch &x;
        ~Release()
        {
            if (!x.tau && !x.buf && !x.cfl && !x.meta) return;
            cudaStreamSynchronize(c->s);
            errest_release(c, x);
        }
    } release{c, ex};
    if (P.flag_mode == ADJAMR_FLAG_ERROR || P.flag_mode == ADJAMR_FLAG_RICHARDSON) {
        TRY(error_estimate(c, l, ex));
        a.q = ex.tau;
        a.mode = P.flag_mode == ADJAMR_FLAG_ERROR ? ADJAMR_FLAG_BRACKET_MAX : ADJAMR_FLAG_RICHARDSON;
    }
    const bool dense = d_bits && !d_patchflags && a.mode == ADJAMR_FLAG_BRACKET_MAX && c->adj &&
                       c->adj->d_bmax && a.S >= 2;
    if (dense) {
        TRY(flag_tables(c, l));
        const size_t *off = c->ftab_off[l];
        char *base = c->d_ftab[l];
        a.owner = L.d_owner;
        a.M = L.M;
        a.tab_a = (const int *)(base + off[0]);
        a.tab_ac = (const int *)(base + off[1]);
        a.tab_wx = (const double *)(base + off[2]);
        a.tab_b = (const int *)(base + off[3]);
        a.tab_bc = (const int *)(base + off[4]);
        a.tab_wy = (const double *)(base + off[5]);
        a.gblk = kFlagBlocksPerThread;
        const long long nblk = (a.nlo <= a.nhi) ? a.nhi / kSnapBlock - a.nlo / kSnapBlock + 1 : 1;
        // two passes through a work list of (cell, block) pairs; a list too
        // short for this call is grown (up to kFlagItemsMax) and the call redone,
        // beyond that the one-pass kernel decides
        // A level of few (cell, block) pairs (a 1D level of a few hundred
        // cells) is decided by the one-pass kernel alone: its single launch
        // costs less than the two passes' two there (the same decisions).
        const bool tiny = (long long)L.N * L.M * nblk <= kFlagOnePassMax;
        const long long want = std::min((long long)L.N * L.M * nblk, kFlagItemsMax);
        if (!tiny && c->fcap < std::min(want, (long long)1 << 20))
            TRY(grow_flag_list(c, std::min(want, (long long)1 << 20)));
        for (int attempt = 0;; attempt++) {
            if (attempt > 0)
                CKR(c, cudaMemsetAsync(head, 0, kPinHead + (size_t)pitch64 * L.M * sizeof(uint64_t), c->s));
            const bool twopass = !tiny && (attempt == 0 || c->fcap >= (long long)L.N * L.M * nblk);
            if (twopass) {
                CKR(c, launch_flag_twopass(a, FlagWork{c->d_fitems, fctr, c->fcap}, c->nsm * 8, c->s));
                c->st.kernel_launches += 2;
            } else {
                CKR(c, launch_flag_dense(a, (int)((nblk + a.gblk - 1) / a.gblk), c->s));
                c->st.kernel_launches++;
            }
            TRY(flag_readback(c, l, d_bits, pitch64, twopass, nflag_out, bbox_out));
            unsigned long long ovf = 0;
            if (twopass) std::memcpy(&ovf, c->h_pin + 32, sizeof ovf);
            if (!ovf) break;
            if (c->fcap < want) TRY(grow_flag_list(c, want));
        }
        return ADJAMR_OK;
    }
    CKR(c, launch_flag(a, c->s));
    c->st.kernel_launches++;
    return flag_readback(c, l, d_bits, pitch64, false, nflag_out, bbox_out);
}

// count, box, (twopass) the work-list counters and (up to kPinBits bytes) the
// bitmap into pinned memory, then one synchronisation
adjamr_status flag_readback(adjamr_ctx *c, int l, uint64_t *d_bits, int pitch64, bool twopass, long long *nflag_out,
                            int *bbox_out)
{
    Level &L = c->L[l];
    const size_t bits_bytes = d_bits ? (size_t)pitch64 * (size_t)L.M * sizeof(uint64_t) : 0;
    const bool with_bits = d_bits && bits_bytes <= kPinBits;
    const size_t need = kPinHead + (with_bits ? bits_bytes : 0);
    if (c->h_pin_bytes < need) {
        if (c->h_pin) cudaFreeHost(c->h_pin);
        c->h_pin = nullptr;
        c->h_pin_bytes = 0;
        CKR(c, cudaMallocHost((void **)&c->h_pin, std::max(need, (size_t)kPinHead + 4096)));
        c->h_pin_bytes = std::max(need, (size_t)kPinHead + 4096);
    }
    // the head (and a small bitmap right behind it) in one copy
    const unsigned long long *head =
        d_bits ? reinterpret_cast<const unsigned long long *>(d_bits) - kPinHead / 8 : c->d_fhead;
    CKR(c, cudaMemcpyAsync(c->h_pin, head, need, cudaMemcpyDeviceToHost, c->s));
    (void)twopass;
    c->pin_has_bits = with_bits;
    CKR(c, cudaStreamSynchronize(c->s));
    unsigned long long cnt = 0;
    std::memcpy(&cnt, c->h_pin, sizeof cnt);
    *nflag_out = (long long)cnt;
    if (bbox_out) {
        int v[4];
        std::memcpy(v, c->h_pin + 8, sizeof v);
        bbox_out[0] = 0x7fffffff - v[0];  // (no flag: INT_MAX, -1, INT_MAX, -1)
        bbox_out[1] = v[1] - 1;
        bbox_out[2] = 0x7fffffff - v[2];
        bbox_out[3] = v[3] - 1;
    }
    return ADJAMR_OK;
}

// early: the caller knows that the kernel ahead in the stream writes only
// interior cells of level l or cells of finer levels, and that level l - 1 is
// final for this substep (see k_ghost_fill).  stored: the coarse stencil
// values of this coarse step are current (coarse_pre ran after the step of
// level l - 1); otherwise the fill interpolates from the coarse states.
adjamr_status ghost_fill(adjamr_ctx *c, int l, int k, bool early, bool stored)
{
    Level &L = c->L[l];
    if (L.nghost == 0) return ADJAMR_OK;
    const double *qo = nullptr, *qn = nullptr;
    long long sc = 0;
    int r = 1;
    if (l > 0) {
        Level &C = c->L[l - 1];
        qo = C.q[C.cur];
        qn = C.q[1 - C.cur];
        sc = C.ncell;
        r = c->P.ratio[l - 1];
    }
    const bool stored_ok = stored && l > 0 && L.d_cpre;
    CpreArgs cp{};
    const double *pre_k = nullptr;
    if (stored_ok && k == 0 && fill_makes_pre(c, l)) {
        // substep 0 interpolates directly and computes the later substeps' values
        cp.list = L.d_clist;
        cp.pre = L.d_cpre;
        cp.sc = L.cpre_sc;
        cp.r = r;
    } else if (stored_ok) {
        pre_k = L.d_cpre + (long long)k * c->m * L.cpre_sc * 3;
        sc = L.cpre_sc;
    }
    CKR(c, launch_ghost_fill(c->P.dim, c->m, L.d_ghost, L.nghost, L.q[L.cur], L.ncell, qo, qn, sc, k, r, c->s,
                             early && l > 0 && k > 0, pre_k, cp, c->nsm * 2));
    c->st.kernel_launches++;
    return ADJAMR_OK;
}

// Ghost arguments of a step that computes the level's ghost ring while it
// stages its tiles (same descriptors and arithmetic as ghost_fill); k is the
// fine substep within the coarser level's step.
GhostArgs fused_ghosts(adjamr_ctx *c, int l, int k)
{
    Level &L = c->L[l];
    GhostArgs ga{L.d_ghost, nullptr, 0, 0, k};
    if (l > 0) {
        ga.pre = L.d_cpre;
        ga.sc = L.cpre_sc;
        ga.pstride = (long long)c->m * L.cpre_sc * 3;
    }
    return ga;
}

enum GhostMode { GHOST_READY = 0, GHOST_FUSED = 1, GHOST_FILL = 2 };

// One step of every patch of level l at fine substep k: q[cur] -> q[1-cur].
// GHOST_FUSED: the step kernel computes the ghost ring while staging;
// GHOST_FILL: the ghost-fill kernel runs first; GHOST_READY: the ring of
// q[cur] was filled beforehand.  Both ways give the same bits.
adjamr_status step_patches(adjamr_ctx *c, int l, int k, GhostMode gm, bool early_ghosts = false)
{
    Level &L = c->L[l];
    if (L.patches.empty()) return ADJAMR_OK;
    GhostArgs ga = (gm == GHOST_FUSED) ? fused_ghosts(c, l, k) : GhostArgs{};
    ga.rx = reflux_args(c, l, k);
    TRY(build_work(c, l, c->ltx[l], c->lty[l]));
    cudaEvent_t te = nullptr;
    if (gm == GHOST_FILL) {
        CKR(c, time_begin(c, l, 1, &te));
        TRY(ghost_fill(c, l, k, early_ghosts, true));
        if (te) CKR(c, cudaEventRecord(te, c->s));
    }
    CKR(c, time_begin(c, l, 0, &te));
    const double *q = L.q[L.cur];
    double *qn = L.q[1 - L.cur];
    const int mode = c->lmode[l];
    if (mode == ADJAMR_LAUNCH_PER_PATCH) {
        int w0 = 0;
        for (int k = 0; k < (int)L.patches.size(); k++) {
            int w1 = w0;
            while (w1 < L.nwork && L.h_work[w1].patch == k) w1++;
            CKR(c, launch_step(c->P.dim, c->P.eqn, c->lkx[l], c->lky[l], q, qn, L.aux, L.ncell, L.d_patches,
                               L.d_work + w0, w1 - w0, 0, c->d_cfl, c->s, ga));
            c->st.kernel_launches++;
            c->st.step_kernel_launches++;
            c->st.level_step_launches[l]++;
            w0 = w1;
        }
    } else {
        int grid = 0;
        TileSched sc{nullptr, 0};
        // SUBSTEPS on a level that cannot take substep launches runs as DYNAMIC
        const bool dyn = mode == ADJAMR_LAUNCH_DYNAMIC || mode == ADJAMR_LAUNCH_SUBSTEPS;
        if (mode == ADJAMR_LAUNCH_PERSISTENT || dyn) grid = std::min(L.nwork, c->lgrid[l]);
        if (dyn) {
            sc.ctr = c->d_wctr;
            sc.base = c->wbase;
            c->wbase += (unsigned long long)L.nwork + (unsigned long long)grid;
        }
        CKR(c, launch_step(c->P.dim, c->P.eqn, c->lkx[l], c->lky[l], q, qn, L.aux, L.ncell, L.d_patches, L.d_work,
                           L.nwork, grid, c->d_cfl, c->s, ga, sc));
        c->st.kernel_launches++;
        c->st.step_kernel_launches++;
        c->st.level_step_launches[l]++;
    }
    if (c->timing) CKR(c, cudaEventRecord(te, c->s));
    c->st.cell_updates += L.ninterior;
    c->st.level_cell_updates[l] += L.ninterior;
    return ADJAMR_OK;
}

// Whether the r substeps of level l within one step of level l - 1 run as one
// substep launch: the finest level of a 2D hierarchy whose kernel tile has a
// substep kernel (no regrid and no finer level come between its substeps).
bool substeps_ok(const adjamr_ctx *c, int l)
{
    return l > 0 && l == c->P.nlevels - 1 && c->P.dim == 2 && c->lmode[l] == ADJAMR_LAUNCH_SUBSTEPS &&
           c->lgrid_sub[l] > 0 && c->P.ratio[l - 1] <= kMaxSubsteps;
}

// One substep launch of r substeps of level l (work list already built)
// with the given dependency lists; r * ninterior cell updates.
adjamr_status launch_substeps(adjamr_ctx *c, int l, int r, const int *dep_idx, const int *dep_cnt)
{
    Level &L = c->L[l];
    {
        if (c->done_cap < (size_t)L.nwork + 1) {
            const size_t want = std::max((size_t)L.nwork + 1, 2 * c->done_cap);
            if (c->d_done) CKR(c, cudaFreeAsync(c->d_done, c->s));
            c->d_done = nullptr;
            c->done_cap = 0;
            CKR(c, cudaMallocAsync((void **)&c->d_done, want * sizeof(unsigned long long), c->s));
            CKR(c, cudaMemsetAsync(c->d_done, 0, want * sizeof(unsigned long long), c->s));
            c->done_cap = want;
        }
        GhostArgs ga = fused_ghosts(c, l, 0);
        ga.rx = reflux_args(c, l, 0);
        SubstepArgs sa{};
        sa.dep_idx = dep_idx;
        sa.dep_cnt = dep_cnt;
        sa.done = c->d_done;
        sa.base = c->done_base;
        sa.nsub = r;
        sa.err = c->d_err;
        c->done_base += (unsigned long long)r;
        const int nitems = r * L.nwork;
        const int grid = std::min(nitems, c->lgrid_sub[l]);
        TileSched sc{c->d_wctr, c->wbase};
        c->wbase += (unsigned long long)nitems + (unsigned long long)grid;
        cudaEvent_t te = nullptr;
        CKR(c, time_begin(c, l, 0, &te));
        CKR(c, launch_step_substeps(c->P.eqn, c->lkx[l], c->lky[l], L.q[L.cur], L.q[1 - L.cur], L.aux, L.ncell,
                                    L.d_patches, L.d_work, L.nwork, grid, c->d_cfl, c->s, ga, sc, sa));
        if (c->timing) CKR(c, cudaEventRecord(te, c->s));
        c->st.kernel_launches++;
        c->st.step_kernel_launches++;
        c->st.level_step_launches[l]++;
        c->st.cell_updates += (long long)r * L.ninterior;
        c->st.level_cell_updates[l] += (long long)r * L.ninterior;
    }
    return ADJAMR_OK;
}

// All r substeps of level l (Sec. 3 subcycling) in one launch of
// k_step2d_sub: q[cur] -> ... -> the final state, in q[cur] again for even r.
adjamr_status step_level_substeps(adjamr_ctx *c, int l, int r)
{
    Level &L = c->L[l];
    if (!L.patches.empty()) {
        TRY(build_work(c, l, c->ltx[l], c->lty[l]));
        TRY(launch_substeps(c, l, r, L.d_dep, L.d_dep + (size_t)L.nwork * kDepRow));
    }
    if (r & 1) L.cur = 1 - L.cur;
    L.nstep += r;
    return ADJAMR_OK;
}

adjamr_status average_down(adjamr_ctx *c, int lf)
{
    Level &F = c->L[lf];
    Level &C = c->L[lf - 1];
    if (F.navg == 0) return ADJAMR_OK;
    CKR(c, launch_average_down(c->P.dim, c->m, F.d_avg, F.navg, F.q[F.cur], F.ncell, C.q[1 - C.cur], C.ncell,
                               c->P.ratio[lf - 1], c->s));
    c->st.kernel_launches++;
    return ADJAMR_OK;
}

// device-side invariant violations recorded by the regrid builders
adjamr_status check_err(adjamr_ctx *c)
{
    int e = 0;
    CKR(c, cudaMemcpyAsync(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost, c->s));
    CKR(c, cudaStreamSynchronize(c->s));
    if (e & kSubstepErrBit) {
        c->err = "a substep launch gave up waiting for a neighbouring tile";
        return ADJAMR_ETIMEOUT;
    }
    if (e & kRefluxErrBit) {
        c->err = "conservation fix-up: a coarse-fine side without its fine records";
        return ADJAMR_ENEST;
    }
    if (e) {
        c->err = "hierarchy not properly nested (device check " + std::to_string(e) + ")";
        return ADJAMR_ENEST;
    }
    return ADJAMR_OK;
}

// sum the recorded step-kernel event pairs (stream already synchronised)
// (pairs whose end event has not completed yet stay for a later harvest)
void harvest_timing(adjamr_ctx *c)
{
    size_t k = 0;
    for (; k + 1 < c->tev_used; k += 2) {
        if (cudaEventQuery(c->tev[k + 1]) == cudaErrorNotReady) break;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->tev[k], c->tev[k + 1]) == cudaSuccess) {
            const int lev = c->tev_level[k] % ADJAMR_MAX_LEVELS;
            if (c->tev_level[k] < ADJAMR_MAX_LEVELS) {
                c->st.step_kernel_ms += ms;
                c->st.level_step_ms[lev] += ms;
            } else {
                c->st.level_ghost_ms[lev] += ms;
            }
        }
    }
    (void)cudaGetLastError();
    for (size_t j = k; j < c->tev_used; j++) {
        std::swap(c->tev[j - k], c->tev[j]);
        std::swap(c->tev_level[j - k], c->tev_level[j]);
    }
    c->tev_used -= k;
}

// Berger-Oliger recursion (Sec. 3, time stepping with subcycling)
adjamr_status step_level(adjamr_ctx *c, int l)
{
    Level &L = c->L[l];
    const adjamr_params &P = c->P;
    int k = P.regrid_interval;
    const bool regrid =
        l < P.nlevels - 1 && k > 0 && L.nstep > 0 && L.nstep % k == 0 && c->rebuilt_tick[l + 1] != L.nstep * c->T[l];
    int sub = 0;
    if (l > 0) sub = (int)(L.nstep - c->L[l - 1].nstep * P.ratio[l - 1]);
    const GhostMode gm = c->lfuse[l] ? GHOST_FUSED : GHOST_FILL;
    // (with the fix-up the step records for the new finer level: regrid first)
    if (regrid && c->s_flag && !P.reflux &&
        (P.flag_mode == ADJAMR_FLAG_BRACKET_MAX || P.flag_mode == ADJAMR_FLAG_LINEAR ||
         P.flag_mode == ADJAMR_FLAG_ERROR || P.flag_mode == ADJAMR_FLAG_RICHARDSON)) {
        // The adjoint flags of level l read its current interior state, which
        // its step leaves alone (it writes the other buffer): the flags run on
        // the side stream while the step runs, so the host clusters and builds
        // level l + 1 during the step.  The rebuilt levels come after the step
        // in stream order, as their first use does.  The error estimate reads
        // the same state and the coarser level's two states, which stay as
        // they are until the average-down; it writes only buffers of its own.
        CKR(c, cudaEventRecord(c->ev_flag, c->s));
        TRY(step_patches(c, l, sub, gm, false));
        TRY(regrid_from(c, l, 0, true));
    } else {
        if (regrid) TRY(regrid_from(c, l, 0));
        // After the first substep and without a rebuild in between, the kernel
        // ahead is this level's previous step, the average-down into it or a
        // finer level's kernel; none of them touches this level's ghost cells.
        TRY(step_patches(c, l, sub, gm, sub > 0 && !regrid));
    }
    if (l < P.nlevels - 1 && !c->L[l + 1].patches.empty()) {
        int r = P.ratio[l];
        TRY(coarse_pre(c, l + 1));
        c->L[l + 1].nstep = L.nstep * r;
        if (substeps_ok(c, l + 1)) TRY(step_level_substeps(c, l + 1, r));
        else
            for (int s = 0; s < r; s++) TRY(step_level(c, l + 1));
        TRY(average_down(c, l + 1));
        TRY(reflux_apply(c, l));
    }
    L.cur = 1 - L.cur;
    L.nstep++;
    return ADJAMR_OK;
}

adjamr_status set_medium_impl(adjamr_ctx *c, const adjamr_medium *m)
{
    if (!m) return ADJAMR_EINVAL;
    for (double *p : c->dense_dev) cudaFreeAsync(p, c->s);
    c->dense_dev.clear();
    for (int l = 0; l < c->P.nlevels; l++) {
        MediumDev &md = c->mh[l];
        std::memset(&md, 0, sizeof md);
        md.kind = m->kind;
        md.nmed = c->nmed;
        md.N = c->L[l].N;
        md.M = c->L[l].M;
        if (m->kind == ADJAMR_MEDIUM_LAYERED) {
            if (m->nlayers < 1 || m->nlayers > 32 || !m->f0 || !m->f1 || (m->nlayers > 1 && !m->iface)) {
                c->err = "layered medium: bad layer table";
                return ADJAMR_EINVAL;
            }
            md.axis = m->axis;
            md.nl = m->nlayers;
            for (int k = 0; k < m->nlayers; k++)
                if (!(m->f0[k] > 0.0) || (c->nmed > 1 && !(m->f1[k] > 0.0))) {
                    c->err = "medium must be positive (rho, K > 0; hbar > 0)";
                    return ADJAMR_EINVAL;
                }
            for (int k = 0; k < m->nlayers - 1; k++) md.iface[k] = m->iface[k];
            for (int k = 0; k < m->nlayers; k++) {
                md.f0[k] = m->f0[k];
                md.f1[k] = m->f1[k];
            }
        } else if (m->kind == ADJAMR_MEDIUM_DENSE) {
            if (!m->dense || m->ndense < c->P.nlevels || !m->dense[l]) {
                c->err = "dense medium: one array per level required";
                return ADJAMR_EINVAL;
            }
            size_t n = (size_t)c->nmed * md.N * md.M;
            for (size_t k = 0; k < n; k++)
                if (!(m->dense[l][k] > 0.0)) {
                    c->err = "medium must be positive (rho, K > 0; hbar > 0)";
                    return ADJAMR_EINVAL;
                }
            double *d = nullptr;
            CKR(c, dalloc(&d, n, c->s));
            CKR(c, cudaMemcpyAsync(d, m->dense[l], n * sizeof(double), cudaMemcpyHostToDevice, c->s));
            c->dense_dev.push_back(d);
            md.dense = d;
        } else {
            c->err = "unknown medium kind";
            return ADJAMR_EINVAL;
        }
        Level &L = c->L[l];
        dfree(L.d_med, c->s);
        CKR(c, dalloc(&L.d_med, 1, c->s));
        CKR(c, cudaMemcpyAsync(L.d_med, &md, sizeof md, cudaMemcpyHostToDevice, c->s));
    }
    // coefficient tables: the medium does not change in time, so the
    // coefficients of a cell depend on (level, I, J) only
    for (int l = 0; l < c->P.nlevels; l++) {
        Level &L = c->L[l];
        dfree(L.d_auxtab, c->s);
        const long long tn = aux_table_cells(c, l);
        if (tn == 0) continue;
        CKR(c, dalloc(&L.d_auxtab, (size_t)(c->naux + c->nmed) * tn, c->s));
        CKR(c, launch_aux_table(c->P.eqn, L.d_med, geom_of(c, l), L.d_auxtab, c->s));
        c->st.kernel_launches++;
    }
    CKR(c, cudaStreamSynchronize(c->s));
    c->have_medium = true;
    for (int l = 0; l < c->P.nlevels; l++) TRY(fill_aux(c, l));
    return ADJAMR_OK;
}

// level 0's state from qinit at its cell centres (zero without qinit), into
// q[0]; synchronises
adjamr_status sample_level0(adjamr_ctx *c)
{
    const adjamr_params *p = &c->P;
    Level &L0 = c->L[0];
    L0.cur = 0;
    std::vector<double> host(p->qinit ? (size_t)c->m * L0.ncell : 0, 0.0);
    if (p->qinit) {
        long long n = L0.ninterior;
        std::vector<double> xc(n), yc(n), qv((size_t)n * c->m);
        long long o = 0;
        for (const HPatch &q : L0.patches)
            for (int j = 0; j < q.ny; j++)
                for (int i = 0; i < q.nx; i++, o++) {
                    xc[o] = p->lo[0] + ((double)(q.ilo + i) + 0.5) * L0.dx;
                    yc[o] = (p->dim == 2) ? p->lo[1] + ((double)(q.jlo + j) + 0.5) * L0.dy : 0.0;
                }
        p->qinit(0, (int)n, xc.data(), yc.data(), qv.data(), p->qinit_user);
        o = 0;
        for (const HPatch &q : L0.patches)
            for (int j = 0; j < q.ny; j++)
                for (int i = 0; i < q.nx; i++, o++)
                    for (int f = 0; f < c->m; f++) host[(size_t)f * L0.ncell + cell_of(c, q, i, j)] = qv[(size_t)f * n + o];
    }
    if (p->qinit)
        CKR(c, cudaMemcpyAsync(L0.q[0], host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
    else if (L0.ncell > 0)
        CKR(c, cudaMemsetAsync(L0.q[0], 0, sizeof(double) * (size_t)c->m * L0.ncell, c->s));
    CKR(c, cudaStreamSynchronize(c->s));
    return ADJAMR_OK;
}

adjamr_status create_impl(const adjamr_params *p, adjamr_ctx **out)
{
    if (!p || !out) return ADJAMR_EINVAL;
    *out = nullptr;
    if (p->dim < 1 || p->dim > 2 || p->nlevels < 1 || p->nlevels > ADJAMR_MAX_LEVELS || p->n0[0] < 1 ||
        (p->dim == 2 && p->n0[1] < 1) || p->eqn < 0 || p->eqn > 3 || (p->dim == 1 && p->eqn > 1) ||
        !(p->hi[0] > p->lo[0]) || (p->dim == 2 && !(p->hi[1] > p->lo[1])) || p->max_patch0 < 1 ||
        p->max_patch < 1 || (p->dt0 <= 0.0 && !(p->cmax > 0.0)) || !(p->tf > p->t0))
        return ADJAMR_EINVAL;
    for (int l = 0; l < p->nlevels - 1; l++)
        if (p->ratio[l] < 2 || p->ratio[l] > kMaxSubsteps) return ADJAMR_EINVAL;
    for (int k = 0; k < 4; k++)
        if (p->bc[k] < 0 || p->bc[k] > 2) return ADJAMR_EINVAL;
    if (p->flag_mode < ADJAMR_FLAG_BRACKET_MAX || p->flag_mode > ADJAMR_FLAG_RICHARDSON) return ADJAMR_EINVAL;
    if (p->launch_mode < ADJAMR_LAUNCH_WORKLIST || p->launch_mode > ADJAMR_LAUNCH_SUBSTEPS) return ADJAMR_EINVAL;
    if (p->reflux != 0 && p->reflux != 1) return ADJAMR_EINVAL;
    adjamr_ctx *c = new (std::nothrow) adjamr_ctx();
    if (!c) return ADJAMR_ENOMEM;
    c->P = *p;
    c->s = (cudaStream_t)p->stream;
    c->m = (p->dim == 2) ? 3 : 2;
    c->naux = naux_of(p->eqn);
    c->nmed = nmed_of(p->eqn);
    c->gy = (p->dim == 2) ? 2 : 0;
    // default 2D tile 16 x 12: the fastest cut measured for the adjoint grids
    // and the finest levels of the workloads (any tile gives the same bits)
    c->tx = p->tile_x > 0 ? p->tile_x : (p->dim == 2 ? 16 : 256);
    c->ty = p->tile_y > 0 ? p->tile_y : (p->dim == 2 ? 12 : 1);
    c->launch_mode = p->launch_mode;
    for (int l = 0; l < ADJAMR_MAX_LEVELS; l++) c->rebuilt_tick[l] = -1;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete c;
        return ADJAMR_ECUDA;
    }
    {
        // keep freed arena blocks in the stream-ordered pool across syncs:
        // regrids free and re-allocate level arenas every few steps
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            unsigned long long thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    int kx = 0, ky = 0;
    if (!step_kernel_shape(p->dim, c->tx, c->ty, &kx, &ky)) {
        delete c;
        return ADJAMR_EINVAL;  // no compiled tile holds tiles of this size
    }
    int occ = step_occupancy(p->dim, p->eqn, kx, ky);
    if (p->dim == 2 && occ <= 0) {
        delete c;
        return ADJAMR_EINVAL;
    }
    c->grid_persistent = nsm * std::max(occ, 1);
    c->nsm = nsm;
    for (int l = 0; l < ADJAMR_MAX_LEVELS; l++) {
        c->ltx[l] = c->tx;
        c->lty[l] = c->ty;
        c->lkx[l] = kx;
        c->lky[l] = ky;
        c->lgrid[l] = c->grid_persistent;
        c->lgrid_sub[l] = p->dim == 2 ? nsm * substep_occupancy(p->eqn, kx, ky) : 0;
        c->lfuse[l] = 1;
        c->lmode[l] = p->launch_mode;
    }
    int N = p->n0[0], M = (p->dim == 2) ? p->n0[1] : 1;
    for (int l = 0; l < p->nlevels; l++) {
        Level &L = c->L[l];
        L.N = N;
        L.M = M;
        L.dx = (p->hi[0] - p->lo[0]) / (double)N;
        L.dy = (p->dim == 2) ? (p->hi[1] - p->lo[1]) / (double)M : 1.0;
        if (l < p->nlevels - 1) {
            N *= p->ratio[l];
            if (p->dim == 2) M *= p->ratio[l];
        }
    }
    double dt0 = p->dt0;
    if (dt0 <= 0.0) {
        double dmin = (p->dim == 2) ? std::fmin(c->L[0].dx, c->L[0].dy) : c->L[0].dx;
        double dtc = p->cfl * dmin / p->cmax;
        double ns = std::ceil((p->tf - p->t0) / dtc);
        dt0 = (p->tf - p->t0) / ns;
    }
    c->L[0].dt = dt0;
    for (int l = 1; l < p->nlevels; l++) c->L[l].dt = c->L[l - 1].dt / (double)p->ratio[l - 1];
    long long T = 1;
    for (int l = p->nlevels - 1; l >= 0; l--) {
        c->T[l] = T;
        if (l > 0) T *= p->ratio[l - 1];
    }
    adjamr_status st;
#define FAIL(x)                                                                                       \
    do {                                                                                              \
        st = (x);                                                                                     \
        if (st != ADJAMR_OK) {                                                                        \
            adjamr_destroy(c);                                                                        \
            return st;                                                                                \
        }                                                                                             \
    } while (0)
    if (cudaMalloc(&c->d_cfl, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_fhead, kPinHead) != cudaSuccess ||
        cudaMalloc(&c->d_fout, sizeof(double)) != cudaSuccess || cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_wctr, sizeof(unsigned long long)) != cudaSuccess) {
        adjamr_destroy(c);
        return ADJAMR_ENOMEM;
    }
    {
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->s_flag, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_flag, cudaEventDisableTiming) != cudaSuccess) {
            adjamr_destroy(c);
            return ADJAMR_ECUDA;
        }
    }
    cudaMemsetAsync(c->d_cfl, 0, sizeof(unsigned long long), c->s);
    cudaMemsetAsync(c->d_wctr, 0, sizeof(unsigned long long), c->s);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->s);
    cudaEventCreate(&c->ev0);
    cudaEventCreate(&c->ev1);
    // level 0 tiles the domain
    Level &L0 = c->L[0];
    int px = (L0.N + p->max_patch0 - 1) / p->max_patch0;
    int py = (p->dim == 2) ? (L0.M + p->max_patch0 - 1) / p->max_patch0 : 1;
    std::vector<Box> boxes;
    for (int b = 0; b < py; b++)
        for (int a = 0; a < px; a++) {
            Box x;
            x.i0 = part_off(L0.N, px, a);
            x.i1 = x.i0 + part_len(L0.N, px, a) - 1;
            x.j0 = (p->dim == 2) ? part_off(L0.M, py, b) : 0;
            x.j1 = (p->dim == 2) ? x.j0 + part_len(L0.M, py, b) - 1 : 0;
            boxes.push_back(x);
        }
    FAIL(alloc_level(c, 0, boxes));
    FAIL(build_ghost_map(c, 0));
    FAIL(sample_level0(c));
#undef FAIL
    if (cudaStreamSynchronize(c->s) != cudaSuccess) {
        adjamr_destroy(c);
        return ADJAMR_ECUDA;
    }
    *out = c;
    return ADJAMR_OK;
}

// interior of a level, patch by patch, field-major per patch
adjamr_status read_level_impl(adjamr_ctx *c, int l, double *dst, size_t cap, bool write, const double *src,
                              const double *from = nullptr)
{
    Level &L = c->L[l];
    size_t need = (size_t)c->m * L.ninterior;
    if (cap < need) {
        c->err = "buffer too small";
        return ADJAMR_EINVAL;
    }
    if (L.ncell == 0) return ADJAMR_OK;
    std::vector<double> host((size_t)c->m * L.ncell);
    const double *buf = from ? from : L.q[L.cur];
    CKR(c, cudaMemcpyAsync(host.data(), buf, host.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CKR(c, cudaStreamSynchronize(c->s));
    size_t o = 0;
    for (const HPatch &p : L.patches)
        for (int f = 0; f < c->m; f++)
            for (int j = 0; j < p.ny; j++)
                for (int i = 0; i < p.nx; i++, o++) {
                    size_t idx = (size_t)f * L.ncell + cell_of(c, p, i, j);
                    if (write) host[idx] = src[o];
                    else dst[o] = host[idx];
                }
    if (write) {
        CKR(c, cudaMemcpyAsync(L.q[L.cur], host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
        CKR(c, cudaStreamSynchronize(c->s));
    }
    return ADJAMR_OK;
}

}  // namespace

// culling table of a snapshot set (see k_flag)
cudaError_t attach_block_max(adjamr_adjoint *a, cudaStream_t s)
{
    a->nblk = (a->S + kSnapBlock - 1) / kSnapBlock;
    size_t n = (size_t)a->nblk * a->m * a->ax * a->ay;
    cudaError_t e = cudaMalloc(&a->d_bmax, n * sizeof(double));
    if (e != cudaSuccess) {
        a->d_bmax = nullptr;
        return e;
    }
    a->bytes += n * sizeof(double);
    return launch_block_max(a->d_snaps, a->S, a->m, a->ax, a->ay, a->dim, a->d_bmax, s);
}

// ====================================================================== ABI
extern "C" {

adjamr_status adjamr_init_grid_hierarchy(const adjamr_params *p, adjamr_ctx **out)
{
    try {
        return create_impl(p, out);
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_set_medium(adjamr_ctx *ctx, const adjamr_medium *m)
{
    if (!ctx) return ADJAMR_EINVAL;
    try {
        return set_medium_impl(ctx, m);
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_load_adjoint_snapshots(adjamr_ctx *ctx, const double *snaps, int nsnap, int ax, int ay,
                                            const unsigned char *wet, int on_device, adjamr_adjoint **out)
{
    if (!ctx || !snaps || nsnap < 2 || ax < 1) return ADJAMR_EINVAL;
    if (ctx->P.dim == 1) ay = 1;
    if (ay < 1 || (ctx->P.dim == 2 && ax < 2) || (ctx->P.dim == 2 && ay < 2)) return ADJAMR_EINVAL;
    adjamr_adjoint *cur = ctx->adj;
    if (cur && cur->refs.load() == 1 && cur->S == nsnap && cur->m == ctx->m && cur->ax == ax && cur->ay == ay &&
        cur->dim == ctx->P.dim && cur->d_bmax) {
        // The context's own set of the same shape, held by nothing else: it is
        // refilled in place once no kernel of the context reads it, instead of
        // a new device allocation per set and a release of the old one.
        const size_t n = (size_t)nsnap * cur->m * ax * ay;
        cudaError_t e = cudaStreamSynchronize(ctx->s);
        if (e == cudaSuccess && ctx->s_flag) e = cudaStreamSynchronize(ctx->s_flag);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cur->d_snaps, snaps, n * sizeof(double),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->s);
        if (e == cudaSuccess) {
            if (wet) e = cudaMemcpyAsync(cur->d_wet, wet, (size_t)ax * ay, cudaMemcpyHostToDevice, ctx->s);
            else e = cudaMemsetAsync(cur->d_wet, 1, (size_t)ax * ay, ctx->s);
        }
        if (e == cudaSuccess) e = launch_block_max(cur->d_snaps, cur->S, cur->m, ax, ay, cur->dim, cur->d_bmax, ctx->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
        if (e != cudaSuccess) {
            // the set's contents are unknown now: the context lets it go
            ctx->err = cudaGetErrorString(e);
            ctx->adj = nullptr;
            adjamr_adjoint_release(cur);
            return ADJAMR_ECUDA;
        }
        if (out) {
            cur->refs++;
            *out = cur;
        }
        return ADJAMR_OK;
    }
    adjamr_adjoint *a = new (std::nothrow) adjamr_adjoint();
    if (!a) return ADJAMR_ENOMEM;
    a->S = nsnap;
    a->m = ctx->m;
    a->ax = ax;
    a->ay = ay;
    a->dim = ctx->P.dim;
    size_t n = (size_t)nsnap * a->m * ax * ay;
    a->bytes = n * sizeof(double) + (size_t)ax * ay;
    if (cudaMalloc(&a->d_snaps, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&a->d_wet, (size_t)ax * ay) != cudaSuccess) {
        adjamr_adjoint_release(a);
        return ADJAMR_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(a->d_snaps, snaps, n * sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->s);
    if (e == cudaSuccess) {
        if (wet) e = cudaMemcpyAsync(a->d_wet, wet, (size_t)ax * ay, cudaMemcpyHostToDevice, ctx->s);
        else e = cudaMemsetAsync(a->d_wet, 1, (size_t)ax * ay, ctx->s);
    }
    if (e == cudaSuccess) e = attach_block_max(a, ctx->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
    if (e != cudaSuccess) {
        ctx->err = cudaGetErrorString(e);
        adjamr_adjoint_release(a);
        return ADJAMR_ECUDA;
    }
    if (ctx->adj) adjamr_adjoint_release(ctx->adj);
    ctx->adj = a;
    if (out) {
        a->refs++;
        *out = a;
    }
    return ADJAMR_OK;
}

adjamr_status adjamr_set_adjoint(adjamr_ctx *ctx, adjamr_adjoint *adj)
{
    if (!ctx || !adj || adj->m != ctx->m || adj->dim != ctx->P.dim) return ADJAMR_EINVAL;
    adj->refs++;
    if (ctx->adj) adjamr_adjoint_release(ctx->adj);
    ctx->adj = adj;
    return ADJAMR_OK;
}

adjamr_status adjamr_adjoint_read(adjamr_adjoint *adj, double *dst, size_t cap)
{
    if (!adj || !dst) return ADJAMR_EINVAL;
    size_t n = (size_t)adj->S * adj->m * adj->ax * adj->ay;
    if (cap < n) return ADJAMR_EINVAL;
    if (cudaMemcpy(dst, adj->d_snaps, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return ADJAMR_ECUDA;
    return ADJAMR_OK;
}

void adjamr_adjoint_release(adjamr_adjoint *adj)
{
    if (!adj) return;
    if (--adj->refs > 0) return;
    if (adj->d_snaps) cudaFree(adj->d_snaps);
    if (adj->d_wet) cudaFree(adj->d_wet);
    if (adj->d_bmax) cudaFree(adj->d_bmax);
    delete adj;
}

adjamr_status adjamr_solve_adjoint(adjamr_ctx *ctx, const adjamr_params *ap, const adjamr_medium *am,
                                   const double *phi, int nsnap, adjamr_adjoint **out)
{
    if (!ap || !am || !phi || nsnap < 2 || ap->nlevels < 1 || (ap->eqn != ADJAMR_ACOUSTICS_ADJOINT &&
                                                                ap->eqn != ADJAMR_SW_ADJOINT))
        return ADJAMR_EINVAL;
    const bool amr = ap->nlevels > 1;
    if (amr && ap->flag_mode != ADJAMR_FLAG_DIFFERENCE && ap->flag_mode != ADJAMR_FLAG_SURFACE &&
        ap->flag_mode != ADJAMR_FLAG_RICHARDSON)
        return ADJAMR_EINVAL;
    if (!(ap->cmax > 0.0) || ap->n0[0] < 1 || (ap->dim == 2 && ap->n0[1] < 1) || !(ap->tf > ap->t0))
        return ADJAMR_EINVAL;
    try {
        // level-0 step dT / ceil(dT / dt_cfl), dT = the snapshot interval, so
        // that steps land on the snapshots (finer levels: dt_0 / prod r)
        const double dx0 = (ap->hi[0] - ap->lo[0]) / (double)ap->n0[0];
        const double dmin = (ap->dim == 2) ? std::fmin(dx0, (ap->hi[1] - ap->lo[1]) / (double)ap->n0[1]) : dx0;
        const double dts = (ap->tf - ap->t0) / (double)(nsnap - 1);
        const double dtc = ap->cfl * dmin / ap->cmax;
        const int nsub = (int)std::ceil(dts / dtc);
        adjamr_params q = *ap;
        q.qinit = nullptr;
        q.dt0 = dts / (double)nsub;
        q.stream = ctx ? (void *)ctx->s : ap->stream;
        adjamr_ctx *a = nullptr;
        TRY(create_impl(&q, &a));
        adjamr_status st = set_medium_impl(a, am);
        if (st != ADJAMR_OK) {
            if (ctx) ctx->err = a->err;
            adjamr_destroy(a);
            return st;
        }
        Level &L = a->L[0];
        int nx = L.N, ny = L.M, m = a->m;
        // phi into the interior (patch order)
        {
            std::vector<double> pv((size_t)m * L.ninterior);
            size_t o = 0;
            for (const HPatch &p : L.patches)
                for (int f = 0; f < m; f++)
                    for (int j = 0; j < p.ny; j++)
                        for (int i = 0; i < p.nx; i++) pv[o++] = phi[((size_t)f * ny + p.jlo + j) * nx + p.ilo + i];
            st = read_level_impl(a, 0, nullptr, pv.size(), true, pv.data());
            // adjoint with AMR: the finer levels flagged by the standard
            // flagger from phi, their cells interpolated from level 0
            if (st == ADJAMR_OK && amr) st = regrid_from(a, 0, 0);
            if (st != ADJAMR_OK) {
                if (ctx) ctx->err = a->err;
                adjamr_destroy(a);
                return st;
            }
        }
        // dense cell map for snapshot gathers
        std::vector<long long> map((size_t)nx * ny);
        for (const HPatch &p : L.patches)
            for (int j = 0; j < p.ny; j++)
                for (int i = 0; i < p.nx; i++) map[(size_t)(p.jlo + j) * nx + p.ilo + i] = cell_of(a, p, i, j);
        long long *d_map = nullptr;
        adjamr_adjoint *h = new adjamr_adjoint();
        h->S = nsnap;
        h->m = m;
        h->ax = nx;
        h->ay = ny;
        h->dim = ap->dim;
        size_t per = (size_t)m * nx * ny;
        h->bytes = per * nsnap * sizeof(double) + (size_t)nx * ny;
        cudaError_t e = cudaMalloc(&h->d_snaps, per * nsnap * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->d_wet, (size_t)nx * ny);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->d_wet, 1, (size_t)nx * ny, a->s);
        if (e == cudaSuccess) e = upload(&d_map, map, a->s);
        for (int sidx = 0; sidx < nsnap && e == cudaSuccess; sidx++) {
            if (sidx > 0)
                for (int k = 0; k < nsub && st == ADJAMR_OK; k++) {
                    if (amr) {
                        // a Berger-Oliger step: level 0 then holds the composite
                        // solution averaged onto the snapshot grid
                        st = step_level(a, 0);
                    } else {
                        st = step_patches(a, 0, 0, a->lfuse[0] ? GHOST_FUSED : GHOST_FILL);
                        L.cur = 1 - L.cur;
                        L.nstep++;
                    }
                }
            if (st != ADJAMR_OK) break;
            e = launch_gather_interior(m, d_map, (long long)nx * ny, L.q[L.cur], L.ncell,
                                       h->d_snaps + (size_t)(nsnap - 1 - sidx) * per, a->s);
        }
        if (e == cudaSuccess && st == ADJAMR_OK) e = attach_block_max(h, a->s);
        if (e == cudaSuccess && st == ADJAMR_OK) e = cudaStreamSynchronize(a->s);
        dfree(d_map, a->s);
        long long adj_updates = a->st.cell_updates;
        if (e != cudaSuccess || st != ADJAMR_OK) {
            if (ctx) ctx->err = e != cudaSuccess ? cudaGetErrorString(e) : a->err;
            adjamr_destroy(a);
            adjamr_adjoint_release(h);
            return e != cudaSuccess ? ADJAMR_ECUDA : st;
        }
        adjamr_destroy(a);
        if (ctx) {
            ctx->st.adjoint_cell_updates += adj_updates;
            if (ctx->adj) adjamr_adjoint_release(ctx->adj);
            ctx->adj = h;
            if (out) {
                h->refs++;
                *out = h;
            }
        } else if (out) {
            *out = h;
        } else {
            adjamr_adjoint_release(h);
        }
        return ADJAMR_OK;
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_regrid(adjamr_ctx *ctx, int base_level, int init)
{
    if (!ctx || base_level < 0 || base_level >= ctx->P.nlevels) return ADJAMR_EINVAL;
    if (!ctx->have_medium) return ADJAMR_ESTATE;
    try {
        TRY(regrid_from(ctx, base_level, init));
        CKR(ctx, cudaStreamSynchronize(ctx->s));
        return check_err(ctx);
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

// one gauge record at the current level-0 time (device, stream-ordered)
adjamr_status record_gauges(adjamr_ctx *c)
{
    if (c->ngauge == 0) return ADJAMR_OK;
    const int w = 1 + c->m;
    if (c->ngrec == c->gcap) {
        long long ncap = c->gcap ? 2 * c->gcap : 256;
        double *nb = nullptr;
        CKR(c, dalloc(&nb, (size_t)ncap * c->ngauge * w, c->s));
        if (c->ngrec) CKR(c, cudaMemcpyAsync(nb, c->d_grec, sizeof(double) * (size_t)c->ngrec * c->ngauge * w,
                                              cudaMemcpyDeviceToDevice, c->s));
        dfree(c->d_grec, c->s);
        c->d_grec = nb;
        c->gcap = ncap;
    }
    GaugeArgs g;
    std::memset(&g, 0, sizeof g);
    g.n = c->ngauge;
    g.m = c->m;
    g.nlev = c->P.nlevels;
    g.gi = c->d_gij;
    g.gj = c->d_gij + (size_t)c->P.nlevels * c->ngauge;
    for (int l = 0; l < c->P.nlevels; l++) {
        const Level &L = c->L[l];
        g.owner[l] = L.patches.empty() ? nullptr : L.d_owner;
        g.q[l] = L.q[L.cur];
        g.stride[l] = L.ncell;
        g.N[l] = L.N;
    }
    g.t = c->P.t0 + (double)c->L[0].nstep * c->L[0].dt;
    g.out = c->d_grec + (size_t)c->ngrec * c->ngauge * w;
    CKR(c, launch_gauges(g, c->s));
    c->st.kernel_launches++;
    c->ngrec++;
    return ADJAMR_OK;
}

adjamr_status adjamr_set_gauges(adjamr_ctx *ctx, int n, const double *x, const double *y)
{
    if (!ctx || n < 0 || (n > 0 && (!x || (ctx->P.dim == 2 && !y)))) return ADJAMR_EINVAL;
    try {
        const adjamr_params &P = ctx->P;
        const int nl = P.nlevels;
        std::vector<int> ij((size_t)2 * nl * n);
        for (int l = 0; l < nl; l++) {
            const Level &L = ctx->L[l];
            for (int g = 0; g < n; g++) {
                int I = (int)std::floor((x[g] - P.lo[0]) / L.dx);
                I = std::min(std::max(I, 0), L.N - 1);
                int J = 0;
                if (P.dim == 2) {
                    J = (int)std::floor((y[g] - P.lo[1]) / L.dy);
                    J = std::min(std::max(J, 0), L.M - 1);
                }
                ij[(size_t)l * n + g] = I;
                ij[(size_t)(nl + l) * n + g] = J;
            }
        }
        cput(ctx, ctx->d_gij);
        dfree(ctx->d_grec, ctx->s);
        ctx->ngrec = ctx->gcap = 0;
        ctx->ngauge = n;
        if (n > 0) {
            std::vector<size_t> offs;
            char *d = nullptr;
            CKR(ctx, upload_packed(ctx, {{ij.data(), sizeof(int) * ij.size()}}, &d, offs));
            ctx->d_gij = reinterpret_cast<int *>(d);
        }
        return ADJAMR_OK;
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_read_gauges(adjamr_ctx *ctx, double *out, long long cap, long long *nrec)
{
    if (!ctx || cap < 0 || (cap > 0 && !out)) return ADJAMR_EINVAL;
    const long long n = std::min(cap, ctx->ngrec);
    if (n > 0)
        CKR(ctx, cudaMemcpyAsync(out, ctx->d_grec, sizeof(double) * (size_t)n * ctx->ngauge * (1 + ctx->m),
                                 cudaMemcpyDeviceToHost, ctx->s));
    CKR(ctx, cudaStreamSynchronize(ctx->s));
    if (nrec) *nrec = ctx->ngrec;
    return ADJAMR_OK;
}

adjamr_status adjamr_advance_level(adjamr_ctx *ctx, int level, int nsteps)
{
    if (!ctx || level != 0 || nsteps < 0) return ADJAMR_EINVAL;
    if (!ctx->have_medium) return ADJAMR_ESTATE;
    try {
        CKR(ctx, cudaMemsetAsync(ctx->d_cfl, 0, sizeof(unsigned long long), ctx->s));
        for (int s = 0; s < nsteps; s++) {
            TRY(step_level(ctx, 0));
            TRY(record_gauges(ctx));
        }
        unsigned long long bits = 0;
        CKR(ctx, cudaMemcpyAsync(&bits, ctx->d_cfl, sizeof bits, cudaMemcpyDeviceToHost, ctx->s));
        CKR(ctx, cudaStreamSynchronize(ctx->s));
        harvest_timing(ctx);
        TRY(check_err(ctx));
        double cfl;
        std::memcpy(&cfl, &bits, sizeof cfl);
        ctx->st.cfl_max_seen = std::fmax(ctx->st.cfl_max_seen, cfl);
        if (cfl > ctx->P.cfl_max) {
            ctx->err = "CFL number exceeded cfl_max";
            return ADJAMR_ECFL;
        }
        return ADJAMR_OK;
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_flag_cells(adjamr_ctx *ctx, int level, double tol, double t_s, unsigned char *flags_out,
                                long long *nflag)
{
    if (!ctx || level < 0 || level >= ctx->P.nlevels) return ADJAMR_EINVAL;
    if (!(t_s >= ctx->P.t0 && t_s <= ctx->P.tf)) return ADJAMR_EINVAL;
    try {
        Level &L = ctx->L[level];
        unsigned char *d = nullptr;
        CKR(ctx, dalloc(&d, (size_t)std::max<long long>(L.ninterior, 1), ctx->s));
        long long n = 0;
        // the window of this call starts at t_s; the run's own ts (the
        // regrids' window) is put back afterwards
        const double ts_run = ctx->P.ts;
        ctx->P.ts = t_s;
        adjamr_status st = flag_dense(ctx, level, tol, nullptr, 0, d, &n);
        ctx->P.ts = ts_run;
        if (st == ADJAMR_OK && flags_out && L.ninterior > 0) {
            CKR(ctx, cudaMemcpyAsync(flags_out, d, (size_t)L.ninterior, cudaMemcpyDeviceToHost, ctx->s));
            CKR(ctx, cudaStreamSynchronize(ctx->s));
        }
        dfree(d, ctx->s);
        if (nflag) *nflag = n;
        return st;
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_integrate_functional(adjamr_ctx *ctx, const adjamr_target *t, double *J_out)
{
    if (!ctx || !t || !J_out) return ADJAMR_EINVAL;
    try {
        const adjamr_params &P = ctx->P;
        std::vector<std::vector<long long>> idx(P.nlevels);
        std::vector<std::vector<double>> area(P.nlevels);
        size_t total = 0;
        for (int l = 0; l < P.nlevels; l++) {
            const Level &L = ctx->L[l];
            if (L.patches.empty()) break;
            int r = (l < P.nlevels - 1) ? P.ratio[l] : 1;
            Level *F = (l < P.nlevels - 1 && !ctx->L[l + 1].patches.empty()) ? &ctx->L[l + 1] : nullptr;
            for (const HPatch &p : L.patches)
                for (int j = 0; j < p.ny; j++)
                    for (int i = 0; i < p.nx; i++) {
                        int I = p.ilo + i, J = p.jlo + j;
                        double xl = P.lo[0] + (double)I * L.dx, xr = P.lo[0] + (double)(I + 1) * L.dx;
                        double ox = std::fmin(xr, t->x1) - std::fmax(xl, t->x0);
                        if (!(ox > 0.0)) continue;
                        double a = ox;
                        if (P.dim == 2) {
                            double yl = P.lo[1] + (double)J * L.dy, yr = P.lo[1] + (double)(J + 1) * L.dy;
                            double oy = std::fmin(yr, t->y1) - std::fmax(yl, t->y0);
                            if (!(oy > 0.0)) continue;
                            a = ox * oy;
                        }
                        if (F && find_patch(*F, I * r, P.dim == 2 ? J * r : 0) >= 0) continue;
                        idx[l].push_back(cell_of(ctx, p, i, j));
                        area[l].push_back(a);
                    }
            total += idx[l].size();
        }
        if (ctx->fscratch_n < total + 1) {
            dfree(ctx->d_fscratch, ctx->s);
            CKR(ctx, dalloc(&ctx->d_fscratch, total + 1, ctx->s));
            ctx->fscratch_n = total + 1;
        }
        size_t off = 0;
        std::vector<long long *> tmp_i;
        std::vector<double *> tmp_a;
        for (int l = 0; l < P.nlevels; l++) {
            if (idx[l].empty()) continue;
            long long *di = nullptr;
            double *da = nullptr;
            CKR(ctx, upload(&di, idx[l], ctx->s));
            CKR(ctx, upload(&da, area[l], ctx->s));
            Level &L = ctx->L[l];
            // terms of this level; the tree reduction runs once over all levels
            CKR(ctx, launch_func_terms(di, da, (long long)idx[l].size(), L.q[L.cur], t->weight, ctx->d_fscratch + off,
                                       ctx->s));
            ctx->st.kernel_launches++;
            off += idx[l].size();
            tmp_i.push_back(di);
            tmp_a.push_back(da);
        }
        CKR(ctx, launch_pairwise(ctx->d_fscratch, (long long)total, ctx->d_fout, ctx->s));
        ctx->st.kernel_launches++;
        for (long long *p : tmp_i) dfree(p, ctx->s);
        for (double *p : tmp_a) dfree(p, ctx->s);
        double J = 0.0;
        CKR(ctx, cudaMemcpyAsync(&J, ctx->d_fout, sizeof J, cudaMemcpyDeviceToHost, ctx->s));
        CKR(ctx, cudaStreamSynchronize(ctx->s));
        *J_out = J;
        return ADJAMR_OK;
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

}  // extern "C"

extern "C" {

adjamr_status adjamr_get_patches(adjamr_ctx *ctx, int level, adjamr_patch *out, int cap, int *n)
{
    if (!ctx || level < 0 || level >= ctx->P.nlevels) return ADJAMR_EINVAL;
    const Level &L = ctx->L[level];
    int np = (int)L.patches.size();
    if (n) *n = np;
    if (!out) return ADJAMR_OK;
    if (cap < np) return ADJAMR_EINVAL;
    for (int k = 0; k < np; k++) {
        const HPatch &p = L.patches[k];
        out[k].level = level;
        out[k].ilo = p.ilo;
        out[k].jlo = p.jlo;
        out[k].nx = p.nx;
        out[k].ny = p.ny;
    }
    return ADJAMR_OK;
}

adjamr_status adjamr_read_level(adjamr_ctx *ctx, int level, double *dst, size_t cap)
{
    if (!ctx || level < 0 || level >= ctx->P.nlevels || (!dst && cap)) return ADJAMR_EINVAL;
    try {
        return read_level_impl(ctx, level, dst, cap, false, nullptr);
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_write_level(adjamr_ctx *ctx, int level, const double *src, size_t count)
{
    if (!ctx || level < 0 || level >= ctx->P.nlevels || (!src && count)) return ADJAMR_EINVAL;
    try {
        return read_level_impl(ctx, level, nullptr, count, true, src);
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_reset(adjamr_ctx *ctx)
{
    if (!ctx) return ADJAMR_EINVAL;
    try {
        CKR(ctx, cudaStreamSynchronize(ctx->s));
        if (ctx->s_flag) CKR(ctx, cudaStreamSynchronize(ctx->s_flag));
        for (int l = ctx->P.nlevels - 1; l >= 1; l--) free_level(ctx, ctx->L[l]);
        reflux_release(ctx, ctx->L[0]);
        for (int l = 0; l < ctx->P.nlevels; l++) {
            ctx->L[l].nstep = 0;
            ctx->L[l].cur = 0;
        }
        for (int l = 0; l < ADJAMR_MAX_LEVELS; l++) ctx->rebuilt_tick[l] = -1;
        ctx->ngrec = 0;
        ctx->st = adjamr_stats{};
        CKR(ctx, cudaMemsetAsync(ctx->d_cfl, 0, sizeof(unsigned long long), ctx->s));
        CKR(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
        return sample_level0(ctx);
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_error_estimate(adjamr_ctx *ctx, int level, double *dst, size_t cap)
{
    if (!ctx || level < 0 || level >= ctx->P.nlevels || (!dst && cap)) return ADJAMR_EINVAL;
    if (!ctx->have_medium) {
        ctx->err = "error estimate: no medium set";
        return ADJAMR_ESTATE;
    }
    try {
        // a level nested only as the other flag modes nest it may leave the
        // estimate's ring without coarse cells: reported for this call, the
        // context's error word is then put back
        TRY(check_err(ctx));
        ErrEstScratch ex;
        adjamr_status st = error_estimate(ctx, level, ex);
        if (st == ADJAMR_OK) st = read_level_impl(ctx, level, dst, cap, false, nullptr, ex.tau);  // synchronises
        cudaStreamSynchronize(ctx->s);
        errest_release(ctx, ex);
        if (st != ADJAMR_OK) return st;
        st = check_err(ctx);
        if (st == ADJAMR_ENEST) {
            CKR(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
            CKR(ctx, cudaStreamSynchronize(ctx->s));
            ctx->err = "error estimate: the level is not nested deeply enough for the estimate's ring "
                       "(nest it as ADJAMR_FLAG_ERROR does)";
        }
        return st;
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_fill_ghosts(adjamr_ctx *ctx, int level)
{
    if (!ctx || level < 0 || level >= ctx->P.nlevels) return ADJAMR_EINVAL;
    int sub = 0;
    if (level > 0) sub = (int)(ctx->L[level].nstep - ctx->L[level - 1].nstep * ctx->P.ratio[level - 1]);
    TRY(ghost_fill(ctx, level, sub));
    CKR(ctx, cudaStreamSynchronize(ctx->s));
    return ADJAMR_OK;
}

adjamr_status adjamr_read_patch_ghosted(adjamr_ctx *ctx, int level, int k, double *q, double *med)
{
    if (!ctx || level < 0 || level >= ctx->P.nlevels) return ADJAMR_EINVAL;
    Level &L = ctx->L[level];
    if (k < 0 || k >= (int)L.patches.size()) return ADJAMR_EINVAL;
    const HPatch &p = L.patches[k];
    size_t n = (size_t)p.sx * p.sy;
    for (int f = 0; f < ctx->m && q; f++)
        CKR(ctx, cudaMemcpyAsync(q + f * n, L.q[L.cur] + (size_t)f * L.ncell + p.base, n * sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->s));
    for (int f = 0; f < ctx->nmed && med; f++)
        CKR(ctx, cudaMemcpyAsync(med + f * n, L.med + (size_t)f * L.ncell + p.base, n * sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->s));
    CKR(ctx, cudaStreamSynchronize(ctx->s));
    return ADJAMR_OK;
}

adjamr_status adjamr_step_level_only(adjamr_ctx *ctx, int level)
{
    if (!ctx || level < 0 || level >= ctx->P.nlevels) return ADJAMR_EINVAL;
    if (!ctx->have_medium) return ADJAMR_ESTATE;
    Level &L = ctx->L[level];
    TRY(step_patches(ctx, level, 0, GHOST_READY));
    L.cur = 1 - L.cur;
    L.nstep++;
    CKR(ctx, cudaStreamSynchronize(ctx->s));
    return ADJAMR_OK;
}

adjamr_status adjamr_cluster_boxes(const unsigned char *flags, const unsigned char *nestable, int N, int M, int dim,
                                   int min_cells, double efficiency, int *boxes, int cap, int *nboxes)
{
    if (!flags || N < 1 || M < 1 || (dim != 1 && dim != 2) || (dim == 1 && M != 1) || min_cells < 1 || cap < 0 ||
        (cap > 0 && !boxes) || !nboxes)
        return ADJAMR_EINVAL;
    try {
        Bits fl, un;
        fl.reset(N, M);
        un.reset(N, M);
        for (int j = 0; j < M; j++)
            for (int i = 0; i < N; i++) {
                const size_t k = (size_t)j * N + i;
                if (flags[k]) fl.row(j)[i >> 6] |= 1ull << (i & 63);
                if (nestable && !nestable[k]) un.row(j)[i >> 6] |= 1ull << (i & 63);
            }
        Clusterer cl;
        cl.N = N;
        cl.M = M;
        cl.dim = dim;
        cl.mc = min_cells;
        cl.eff = efficiency;
        cl.init(fl, un);
        cl.run(Box{0, N - 1, 0, M - 1});
        std::vector<Box> out = cl.out;
        std::sort(out.begin(), out.end(),
                  [](const Box &a, const Box &b) { return a.j0 != b.j0 ? a.j0 < b.j0 : a.i0 < b.i0; });
        *nboxes = (int)out.size();
        for (int k = 0; k < (int)out.size() && k < cap; k++) {
            boxes[4 * k + 0] = out[k].i0;
            boxes[4 * k + 1] = out[k].i1;
            boxes[4 * k + 2] = out[k].j0;
            boxes[4 * k + 3] = out[k].j1;
        }
        return ADJAMR_OK;
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_set_level_kernel(adjamr_ctx *ctx, int level, int tile_x, int tile_y, int fuse_ghosts,
                                      int launch_mode)
{
    if (!ctx || level < -1 || level >= ctx->P.nlevels) return ADJAMR_EINVAL;
    if (launch_mode < -1 || launch_mode > ADJAMR_LAUNCH_SUBSTEPS) return ADJAMR_EINVAL;
    int ty = (ctx->P.dim == 2) ? tile_y : 1;
    int kx = 0, ky = 0;
    if (!step_kernel_shape(ctx->P.dim, tile_x, ty, &kx, &ky)) return ADJAMR_EINVAL;
    const int occ = step_occupancy(ctx->P.dim, ctx->P.eqn, kx, ky);
    if (occ <= 0) return ADJAMR_EINVAL;
    for (int l = 0; l < ctx->P.nlevels; l++) {
        if (level >= 0 && l != level) continue;
        ctx->ltx[l] = tile_x;
        ctx->lty[l] = ty;
        ctx->lkx[l] = kx;
        ctx->lky[l] = ky;
        ctx->lgrid[l] = ctx->nsm * std::max(occ, 1);
        ctx->lgrid_sub[l] = ctx->P.dim == 2 ? ctx->nsm * substep_occupancy(ctx->P.eqn, kx, ky) : 0;
        ctx->lfuse[l] = fuse_ghosts != 0;
        if (launch_mode >= 0) ctx->lmode[l] = launch_mode;
    }
    return ADJAMR_OK;
}

adjamr_status adjamr_substep_wait_selftest(adjamr_ctx *ctx, double *wait_ms)
{
    if (!ctx) return ADJAMR_EINVAL;
    const int l = ctx->P.nlevels - 1;
    if (!substeps_ok(ctx, l) || ctx->L[l].patches.empty() || !ctx->have_medium) return ADJAMR_ESTATE;
    try {
        Level &L = ctx->L[l];
        TRY(build_work(ctx, l, ctx->ltx[l], ctx->lty[l]));
        // every tile waits for counter nwork, which no tile advances
        std::vector<int> idx((size_t)L.nwork * kDepRow, L.nwork), cnt((size_t)L.nwork, 1);
        std::vector<size_t> offs;
        char *d = nullptr;
        CKR(ctx, upload_packed(ctx, {{idx.data(), sizeof(int) * idx.size()}, {cnt.data(), sizeof(int) * cnt.size()}},
                               &d, offs));
        const adjamr_stats keep = ctx->st;
        CKR(ctx, cudaEventRecord(ctx->ev0, ctx->s));
        adjamr_status st = launch_substeps(ctx, l, 2, reinterpret_cast<const int *>(d + offs[0]),
                                           reinterpret_cast<const int *>(d + offs[1]));
        ctx->st = keep;
        if (st != ADJAMR_OK) return st;
        CKR(ctx, cudaEventRecord(ctx->ev1, ctx->s));
        int e = 0;
        CKR(ctx, cudaMemcpyAsync(&e, ctx->d_err, sizeof e, cudaMemcpyDeviceToHost, ctx->s));
        CKR(ctx, cudaStreamSynchronize(ctx->s));
        float ms = 0.f;
        CKR(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        if (wait_ms) *wait_ms = ms;
        cput(ctx, d);
        if (!(e & kSubstepErrBit)) return ADJAMR_OK;
        const int rest = e & ~kSubstepErrBit;
        CKR(ctx, cudaMemcpyAsync(ctx->d_err, &rest, sizeof rest, cudaMemcpyHostToDevice, ctx->s));
        CKR(ctx, cudaStreamSynchronize(ctx->s));
        ctx->err = "a substep launch gave up waiting for a neighbouring tile (self test)";
        return ADJAMR_ETIMEOUT;
    } catch (...) {
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_get_stats(adjamr_ctx *ctx, adjamr_stats *out)
{
    if (!ctx || !out) return ADJAMR_EINVAL;
    *out = ctx->st;
    return ADJAMR_OK;
}

adjamr_status adjamr_set_timing(adjamr_ctx *ctx, int enable)
{
    if (!ctx) return ADJAMR_EINVAL;
    ctx->timing = enable != 0;
    return ADJAMR_OK;
}

adjamr_status adjamr_time_info(adjamr_ctx *ctx, double *dt0, int *nsteps)
{
    if (!ctx) return ADJAMR_EINVAL;
    double dt = ctx->L[0].dt;
    if (dt0) *dt0 = dt;
    if (nsteps) *nsteps = (int)std::llround((ctx->P.tf - ctx->P.t0) / dt);
    return ADJAMR_OK;
}

const char *adjamr_last_error(adjamr_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void adjamr_destroy(adjamr_ctx *ctx)
{
    if (!ctx) return;
    for (int l = 0; l < ADJAMR_MAX_LEVELS; l++) {
        free_level(ctx, ctx->L[l]);
        dfree(ctx->L[l].d_med, ctx->s);
        dfree(ctx->L[l].d_auxtab, ctx->s);
    }
    for (double *p : ctx->dense_dev) cudaFreeAsync(p, ctx->s);
    dfree(ctx->d_flagall, ctx->s);
    ctx->d_flagbuf = nullptr;
    for (int l = 0; l < ADJAMR_MAX_LEVELS; l++) cput(ctx, ctx->d_ftab[l]);
    cput(ctx, ctx->d_fitems);
    cput(ctx, ctx->d_gij);
    dfree(ctx->d_grec, ctx->s);
    dfree(ctx->d_fscratch, ctx->s);
    dfree(ctx->d_done, ctx->s);
    cache_drain(ctx);
    cudaStreamSynchronize(ctx->s);
    if (ctx->s_flag) {
        cudaStreamSynchronize(ctx->s_flag);
        cudaStreamDestroy(ctx->s_flag);
    }
    if (ctx->ev_flag) cudaEventDestroy(ctx->ev_flag);
    if (ctx->d_cfl) cudaFree(ctx->d_cfl);
    if (ctx->d_fhead) cudaFree(ctx->d_fhead);
    if (ctx->d_fout) cudaFree(ctx->d_fout);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_wctr) cudaFree(ctx->d_wctr);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
    for (int k = 0; k < adjamr_ctx::kStageSlots; k++) {
        if (ctx->stage_ev[k]) cudaEventDestroy(ctx->stage_ev[k]);
        if (ctx->h_stage[k]) cudaFreeHost(ctx->h_stage[k]);
    }
    if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
    if (ctx->adj) adjamr_adjoint_release(ctx->adj);
    delete ctx;
}

}  // extern "C"
