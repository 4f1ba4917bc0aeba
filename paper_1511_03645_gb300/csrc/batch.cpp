// Batched independent patches: many 2D acoustics patches of uneven sizes and
// mixed resolutions advance together.  Each patch is its own domain with
// extrapolation ghost cells and its own dt.  A step is two launches: the
// ghost fill over every ghost cell of every patch, and the fused step kernel
// over a tile work-list of all patches (one launch, or a persistent grid),
// or one step launch per patch for comparison.  A pair of steps can be
// captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

using namespace adjamr;

namespace {
struct BPatch {
    int nx, ny, sx, sy, mid;
    long long base;
    double x0, y0, dx, dy, dt;
};
}  // namespace

struct adjamr_batch {
    int np = 0;
    cudaStream_t s = nullptr;
    std::vector<BPatch> patches;
    long long ncell = 0, ninterior = 0;
    double *q[2] = {nullptr, nullptr};
    double *aux = nullptr, *med = nullptr;
    int cur = 0;
    PatchDesc *d_patches = nullptr;
    GhostDesc *d_ghost = nullptr;
    long long nghost = 0;
    int fuse = 0;  // ghost ring computed inside the step kernel
    WorkItem *d_work = nullptr;
    int nwork = 0, wtx = 0, wty = 0;
    std::vector<WorkItem> h_work;
    std::vector<int> order;
    MediumDev *d_media = nullptr;
    unsigned long long *d_cfl = nullptr;
    unsigned long long *d_wctr = nullptr;  // tile counter of the dynamic launch mode
    int nsm = 0;
    std::map<std::tuple<int, int, int, int, int>, cudaGraphExec_t> graphs;
    std::string err;
};

namespace {

cudaError_t build_work(adjamr_batch *b, int tx, int ty)
{
    if (b->d_work && b->wtx == tx && b->wty == ty) return cudaSuccess;
    if (b->d_work) cudaFreeAsync(b->d_work, b->s);
    b->d_work = nullptr;
    b->h_work.clear();
    for (int k : b->order) {
        const BPatch &p = b->patches[k];
        const int nx = tile_count(p.nx, tx), ny = tile_count(p.ny, ty);
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                b->h_work.push_back({k, tile_off(p.nx, nx, i), tile_off(p.ny, ny, j),
                                     (unsigned short)tile_len(p.nx, nx, i), (unsigned short)tile_len(p.ny, ny, j)});
    }
    b->nwork = (int)b->h_work.size();
    cudaError_t e = cudaMallocAsync((void **)&b->d_work, sizeof(WorkItem) * b->h_work.size(), b->s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(b->d_work, b->h_work.data(), sizeof(WorkItem) * b->h_work.size(), cudaMemcpyHostToDevice,
                        b->s);
    b->wtx = tx;
    b->wty = ty;
    return e;
}

void drop_graphs(adjamr_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// one step of every patch; swaps buffers.  The extrapolated ghost ring comes
// from the ghost descriptors, either inside the step kernel while it stages
// its tiles (b->fuse) or from the ghost-fill kernel launched first.
cudaError_t one_step(adjamr_batch *b, int mode, int tx, int ty)
{
    int kx = 0, ky = 0;  // the compiled kernel tile that holds tx x ty tiles
    if (!step_kernel_shape(2, tx, ty, &kx, &ky)) return cudaErrorInvalidValue;
    const double *q = b->q[b->cur];
    double *qn = b->q[1 - b->cur];
    GhostArgs ga{};
    cudaError_t e = cudaSuccess;
    if (b->fuse) {
        ga.gd = b->d_ghost;
    } else {
        e = launch_ghost_fill(2, 3, b->d_ghost, b->nghost, b->q[b->cur], b->ncell, nullptr, nullptr, 0, 0, 1, b->s);
        if (e != cudaSuccess) return e;
    }
    if (mode == ADJAMR_LAUNCH_PER_PATCH) {
        int w0 = 0;
        while (w0 < b->nwork) {
            int w1 = w0, k = b->h_work[w0].patch;
            while (w1 < b->nwork && b->h_work[w1].patch == k) w1++;
            e = launch_step(2, 0, kx, ky, q, qn, b->aux, b->ncell, b->d_patches, b->d_work + w0, w1 - w0, 0, b->d_cfl,
                            b->s, ga);
            if (e != cudaSuccess) return e;
            w0 = w1;
        }
    } else {
        int grid = 0;
        if (mode == ADJAMR_LAUNCH_PERSISTENT || mode == ADJAMR_LAUNCH_DYNAMIC)
            grid = std::min(b->nwork, b->nsm * std::max(1, step_occupancy(2, 0, kx, ky)));
        TileSched sc{nullptr, 0};
        if (mode == ADJAMR_LAUNCH_DYNAMIC) {
            // counter reset in the stream, so that a captured step replays as is
            e = cudaMemsetAsync(b->d_wctr, 0, sizeof(unsigned long long), b->s);
            if (e != cudaSuccess) return e;
            sc.ctr = b->d_wctr;
        }
        e = launch_step(2, 0, kx, ky, q, qn, b->aux, b->ncell, b->d_patches, b->d_work, b->nwork, grid, b->d_cfl, b->s,
                        ga, sc);
        if (e != cudaSuccess) return e;
    }
    b->cur = 1 - b->cur;
    return cudaSuccess;
}

}  // namespace

extern "C" {

adjamr_status adjamr_batch_create(int npatch, const int *nx, const int *ny, const double *x0, const double *y0,
                                  const double *x1, const double *y1, const double *dt, const int *medium_id,
                                  const adjamr_medium *media, int nmedia, const double *q0, void *stream,
                                  adjamr_batch **out)
{
    if (npatch < 1 || !nx || !ny || !x0 || !y0 || !x1 || !y1 || !dt || !medium_id || !media || nmedia < 1 || !out)
        return ADJAMR_EINVAL;
    for (int k = 0; k < nmedia; k++)
        if (media[k].kind != ADJAMR_MEDIUM_LAYERED || media[k].nlayers < 1 || media[k].nlayers > 32)
            return ADJAMR_EINVAL;
    adjamr_batch *b = new (std::nothrow) adjamr_batch();
    if (!b) return ADJAMR_ENOMEM;
    try {
        b->np = npatch;
        b->s = (cudaStream_t)stream;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
        long long off = 0, gcount = 0;
        std::vector<PatchDesc> pd;
        for (int k = 0; k < npatch; k++) {
            if (nx[k] < 1 || ny[k] < 1 || medium_id[k] < 0 || medium_id[k] >= nmedia || !(x1[k] > x0[k]) ||
                !(y1[k] > y0[k]) || !(dt[k] > 0.0)) {
                delete b;
                return ADJAMR_EINVAL;
            }
            BPatch p;
            p.nx = nx[k];
            p.ny = ny[k];
            p.sx = nx[k] + 4;
            p.sy = ny[k] + 4;
            p.mid = medium_id[k];
            p.base = off;
            p.x0 = x0[k];
            p.y0 = y0[k];
            p.dx = (x1[k] - x0[k]) / (double)nx[k];
            p.dy = (y1[k] - y0[k]) / (double)ny[k];
            p.dt = dt[k];
            off += ((long long)p.sx * p.sy + 3) / 4 * 4;
            b->patches.push_back(p);
            b->ninterior += (long long)p.nx * p.ny;
            PatchDesc d;
            d.ilo = 0; d.jlo = 0; d.nx = p.nx; d.ny = p.ny; d.sx = p.sx; d.sy = p.sy; d.base = p.base;
            d.dtdx = p.dt / p.dx; d.dtdy = p.dt / p.dy; d.hx = 0.5 * d.dtdx; d.hy = 0.5 * d.dtdy;
            d.gbase = gcount;
            gcount += (long long)p.sx * p.sy - (long long)p.nx * p.ny;
            pd.push_back(d);
            b->order.push_back(k);
        }
        b->ncell = off;
        cudaError_t e = cudaSuccess;
        auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
        chk(cudaMallocAsync((void **)&b->q[0], sizeof(double) * 3 * off, b->s));
        chk(cudaMallocAsync((void **)&b->q[1], sizeof(double) * 3 * off, b->s));
        chk(cudaMallocAsync((void **)&b->aux, sizeof(double) * naux_of(0) * off, b->s));
        chk(cudaMallocAsync((void **)&b->med, sizeof(double) * 2 * off, b->s));
        chk(cudaMallocAsync((void **)&b->d_patches, sizeof(PatchDesc) * pd.size(), b->s));
        chk(cudaMallocAsync((void **)&b->d_media, sizeof(MediumDev) * nmedia, b->s));
        chk(cudaMallocAsync((void **)&b->d_cfl, sizeof(unsigned long long), b->s));
        chk(cudaMallocAsync((void **)&b->d_wctr, sizeof(unsigned long long), b->s));
        if (e != cudaSuccess) {
            adjamr_batch_destroy(b);
            return ADJAMR_ENOMEM;
        }
        chk(cudaMemsetAsync(b->q[0], 0, sizeof(double) * 3 * off, b->s));
        chk(cudaMemsetAsync(b->q[1], 0, sizeof(double) * 3 * off, b->s));
        chk(cudaMemsetAsync(b->d_cfl, 0, sizeof(unsigned long long), b->s));
        chk(cudaMemcpyAsync(b->d_patches, pd.data(), sizeof(PatchDesc) * pd.size(), cudaMemcpyHostToDevice, b->s));
        std::vector<MediumDev> mh(nmedia);
        for (int k = 0; k < nmedia; k++) {
            MediumDev &m = mh[k];
            std::memset(&m, 0, sizeof m);
            m.kind = ADJAMR_MEDIUM_LAYERED;
            m.axis = media[k].axis;
            m.nl = media[k].nlayers;
            m.nmed = 2;
            for (int q = 0; q < m.nl - 1; q++) m.iface[q] = media[k].iface[q];
            for (int q = 0; q < m.nl; q++) {
                m.f0[q] = media[k].f0[q];
                m.f1[q] = media[k].f1[q];
            }
        }
        chk(cudaMemcpyAsync(b->d_media, mh.data(), sizeof(MediumDev) * nmedia, cudaMemcpyHostToDevice, b->s));
        // ghost map (extrapolation: nearest interior cell of the same patch),
        // medium coefficients, initial state
        std::vector<GhostDesc> gd;
        std::vector<double> host((size_t)3 * off, 0.0);
        size_t o = 0;
        for (int k = 0; k < npatch; k++) {
            const BPatch &p = b->patches[k];
            std::vector<AuxDesc> ad;
            for (int j = -2; j < p.ny + 2; j++)
                for (int i = -2; i < p.nx + 2; i++) {
                    long long cell = p.base + (long long)(j + 2) * p.sx + (i + 2);
                    ad.push_back({cell, i, j});
                    if (i >= 0 && i < p.nx && j >= 0 && j < p.ny) continue;
                    int ii = std::min(std::max(i, 0), p.nx - 1), jj = std::min(std::max(j, 0), p.ny - 1);
                    GhostDesc g;
                    std::memset(&g, 0, sizeof g);
                    g.dst = cell;
                    g.src = p.base + (long long)(jj + 2) * p.sx + (ii + 2);
                    g.kind = 0;
                    gd.push_back(g);
                }
            AuxDesc *dad = nullptr;
            chk(cudaMallocAsync((void **)&dad, sizeof(AuxDesc) * ad.size(), b->s));
            chk(cudaMemcpyAsync(dad, ad.data(), sizeof(AuxDesc) * ad.size(), cudaMemcpyHostToDevice, b->s));
            LevelGeom g;
            g.dim = 2;
            g.N = p.nx;
            g.M = p.ny;
            g.lo0 = p.x0;
            g.lo1 = p.y0;
            g.dx = p.dx;
            g.dy = p.dy;
            for (int q = 0; q < 4; q++) g.bc[q] = ADJAMR_BC_EXTRAP;
            chk(launch_aux_fill(0, 2, dad, (long long)ad.size(), b->aux, b->med, off, b->d_media + p.mid, g, b->s));
            chk(cudaFreeAsync(dad, b->s));
            if (q0)
                for (int f = 0; f < 3; f++)
                    for (int j = 0; j < p.ny; j++)
                        for (int i = 0; i < p.nx; i++)
                            host[(size_t)f * off + p.base + (size_t)(j + 2) * p.sx + (i + 2)] = q0[o++];
        }
        b->nghost = (long long)gd.size();
        chk(cudaMallocAsync((void **)&b->d_ghost, sizeof(GhostDesc) * gd.size(), b->s));
        chk(cudaMemcpyAsync(b->d_ghost, gd.data(), sizeof(GhostDesc) * gd.size(), cudaMemcpyHostToDevice, b->s));
        chk(cudaMemcpyAsync(b->q[0], host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, b->s));
        chk(build_work(b, 32, 8));
        chk(cudaStreamSynchronize(b->s));
        if (e != cudaSuccess) {
            adjamr_batch_destroy(b);
            return ADJAMR_ECUDA;
        }
        *out = b;
        return ADJAMR_OK;
    } catch (...) {
        adjamr_batch_destroy(b);
        return ADJAMR_ENOMEM;
    }
}

adjamr_status adjamr_batch_set_order(adjamr_batch *b, const int *order)
{
    if (!b || !order) return ADJAMR_EINVAL;
    std::vector<char> seen(b->np, 0);
    for (int k = 0; k < b->np; k++) {
        if (order[k] < 0 || order[k] >= b->np || seen[order[k]]) return ADJAMR_EINVAL;
        seen[order[k]] = 1;
    }
    b->order.assign(order, order + b->np);
    if (b->d_work) cudaFreeAsync(b->d_work, b->s);
    b->d_work = nullptr;
    b->wtx = b->wty = 0;
    drop_graphs(b);
    return ADJAMR_OK;
}

adjamr_status adjamr_batch_set_ghost_fusion(adjamr_batch *b, int fuse_ghosts)
{
    if (!b) return ADJAMR_EINVAL;
    b->fuse = fuse_ghosts != 0;
    return ADJAMR_OK;
}

adjamr_status adjamr_batch_step(adjamr_batch *b, int nsteps, int mode, int tx, int ty)
{
    if (!b || nsteps < 0 || mode < ADJAMR_LAUNCH_WORKLIST || mode > ADJAMR_LAUNCH_DYNAMIC) return ADJAMR_EINVAL;
    int kx = 0, ky = 0;
    if (!step_kernel_shape(2, tx, ty, &kx, &ky) || step_occupancy(2, 0, kx, ky) <= 0) return ADJAMR_EINVAL;
    if (build_work(b, tx, ty) != cudaSuccess) return ADJAMR_ECUDA;
    for (int s = 0; s < nsteps; s++) {
        cudaError_t e = one_step(b, mode, tx, ty);
        if (e != cudaSuccess) {
            b->err = cudaGetErrorString(e);
            return ADJAMR_ECUDA;
        }
    }
    return ADJAMR_OK;
}

adjamr_status adjamr_batch_step_graph(adjamr_batch *b, int nsteps, int mode, int tx, int ty)
{
    if (!b || nsteps < 0 || mode < ADJAMR_LAUNCH_WORKLIST || mode > ADJAMR_LAUNCH_DYNAMIC) return ADJAMR_EINVAL;
    int kx = 0, ky = 0;
    if (!step_kernel_shape(2, tx, ty, &kx, &ky) || step_occupancy(2, 0, kx, ky) <= 0) return ADJAMR_EINVAL;
    if (build_work(b, tx, ty) != cudaSuccess) return ADJAMR_ECUDA;
    if (b->s == nullptr) return ADJAMR_ESTATE;  // capture needs a non-default stream
    auto key = std::make_tuple(mode, tx, ty, b->cur, b->fuse);
    cudaGraphExec_t exec = nullptr;
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaGraph_t g = nullptr;
        int cur0 = b->cur;
        cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = one_step(b, mode, tx, ty);
        if (e == cudaSuccess) e = one_step(b, mode, tx, ty);
        cudaError_t e2 = cudaStreamEndCapture(b->s, &g);
        b->cur = cur0;  // capture does not execute
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            b->err = cudaGetErrorString(e != cudaSuccess ? e : e2);
            return ADJAMR_ECUDA;
        }
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->err = cudaGetErrorString(e);
            return ADJAMR_ECUDA;
        }
        b->graphs[key] = exec;
    } else {
        exec = it->second;
    }
    for (int s = 0; s + 1 < nsteps; s += 2) {
        cudaError_t e = cudaGraphLaunch(exec, b->s);
        if (e != cudaSuccess) {
            b->err = cudaGetErrorString(e);
            return ADJAMR_ECUDA;
        }
    }
    if (nsteps & 1) {
        cudaError_t e = one_step(b, mode, tx, ty);
        if (e != cudaSuccess) return ADJAMR_ECUDA;
    }
    return ADJAMR_OK;
}

adjamr_status adjamr_batch_read(adjamr_batch *b, double *dst, size_t cap)
{
    if (!b || !dst || cap < (size_t)3 * b->ninterior) return ADJAMR_EINVAL;
    std::vector<double> host((size_t)3 * b->ncell);
    if (cudaMemcpyAsync(host.data(), b->q[b->cur], host.size() * sizeof(double), cudaMemcpyDeviceToHost, b->s) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->s) != cudaSuccess)
        return ADJAMR_ECUDA;
    size_t o = 0;
    for (const BPatch &p : b->patches)
        for (int f = 0; f < 3; f++)
            for (int j = 0; j < p.ny; j++)
                for (int i = 0; i < p.nx; i++)
                    dst[o++] = host[(size_t)f * b->ncell + p.base + (size_t)(j + 2) * p.sx + (i + 2)];
    return ADJAMR_OK;
}

adjamr_status adjamr_batch_cells(adjamr_batch *b, long long *cells)
{
    if (!b || !cells) return ADJAMR_EINVAL;
    *cells = b->ninterior;
    return ADJAMR_OK;
}

void adjamr_batch_destroy(adjamr_batch *b)
{
    if (!b) return;
    drop_graphs(b);
    cudaStream_t s = b->s;
    void *ptrs[] = {b->q[0], b->q[1], b->aux, b->med, b->d_patches, b->d_ghost, b->d_work, b->d_media, b->d_cfl,
                    b->d_wctr};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
    delete b;
}

}  // extern "C"
