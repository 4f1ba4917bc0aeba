// AMR kernels (Sec. 3 and Sec. 4), FP64, sm_103a:
//  - ghost fill: same-level copy / physical boundary (via a boundary-mapped
//    source cell) / coarse space-time interpolation (linear in time between
//    the coarse old and new states, minmod-limited linear in space);
//  - regrid init of new patches (copy from the old arena or space
//    interpolation from the coarser level);
//  - averaging fine -> coarse;
//  - medium coefficients of new patches;
//  - adjoint flagging (bilinear interpolation in space; bracketing
//    snapshots or linear-in-time window maximum) with a warp-ballot count;
//  - the functional J with a fixed pairwise summation tree.
// Operation order follows the canonical operations (compiled with
// --fmad=false), as does the CPU oracle.
#include <algorithm>

#include <cuda_runtime.h>

#include "internal.h"
#include "device_common.cuh"

namespace adjamr {
namespace {

constexpr int kT = 256;

// One thread per (ghost cell, field): short load chains, more of them in
// flight.  early != 0 (a fine substep after the first, so the coarser level's
// states are final and the kernel ahead in the stream is a step of this level,
// which writes only interior cells): the coarse interpolations are written
// before waiting for that step, so they overlap its tail; the same-level copies
// read its output and come after the wait.  pre_k != nullptr: coarse
// interpolations from the stored stencil values of this substep.
__device__ __forceinline__ double fill_value(const GhostDesc &g, const double *qf, long long sf,
                                             const double *__restrict__ qo, const double *__restrict__ qn_,
                                             long long sc, int f, int k, double th, int dim,
                                             const double *__restrict__ pre_k)
{
    return pre_k ? ghost_value(g, qf, sf, pre_k, sc, f, dim) : ghost_value_direct(g, qf, sf, qo, qn_, sc, f, k, th, dim);
}

// cp.list != nullptr (substep 0): the CTAs past the fill's also compute the
// coarse stencil values of substeps 1 .. r - 1 (k_cpre's work) for the later
// substeps' fills
__global__ void k_ghost_fill(int dim, int m, const GhostDesc *__restrict__ gd, long long n, double *qf, long long sf,
                             const double *__restrict__ qo, const double *__restrict__ qn_, long long sc, int k,
                             double th, int early, const double *__restrict__ pre_k, CpreArgs cp)
{
    const unsigned fill_blocks = (unsigned)((n * m + kT - 1) / kT);
    if (cp.list && blockIdx.x >= fill_blocks) {
        pdl_wait();
        pdl_launch_dependents();
        const long long per = (long long)(cp.r - 1) * m;
        const long long total = (long long)cp.list[0] * per;
        const long long stride = (long long)(gridDim.x - fill_blocks) * blockDim.x;
        for (long long t = (long long)(blockIdx.x - fill_blocks) * blockDim.x + threadIdx.x; t < total; t += stride) {
            const long long e = t / per;
            const int rest = (int)(t - e * per), s = 1 + rest / m, f = rest - (s - 1) * m;
            const GhostDesc g = gd[cp.list[1 + e]];
            double v[3];
            coarse_stencil(g, qo, qn_, sc, f, s, cp.tt.th[s], dim, v);
            double *p = cp.pre + (((long long)s * m + f) * cp.sc + g.src) * 3;
            p[0] = v[0];
            p[1] = v[1];
            p[2] = v[2];
        }
        return;
    }
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < n * m;
    const long long gi = valid ? t / m : 0;
    const int f = (int)(t - gi * m);
    // early: the descriptor (fixed since the level's rebuild) is read before
    // the wait too, so that a copy waits for one load of the step's output only
    GhostDesc g{};
    if (early && valid) {
        g = gd[gi];
        if (g.kind != 0) qf[(long long)f * sf + g.dst] = fill_value(g, qf, sf, qo, qn_, sc, f, k, th, dim, pre_k);
    }
    pdl_wait();
    pdl_launch_dependents();
    if (!valid || (early && g.kind != 0)) return;
    if (!early) g = gd[gi];
    qf[(long long)f * sf + g.dst] = fill_value(g, qf, sf, qo, qn_, sc, f, k, th, dim, pre_k);
}

// Coarse stencil values of the listed coarse cells for every substep s < r of
// the coarse step (time fraction th[s]) and field: computed once per coarse
// cell instead of once per fine ghost cell.
__global__ void k_cpre(const GhostDesc *__restrict__ gd, const unsigned long long *__restrict__ list, int m, int r,
                       int dim, const double *__restrict__ qo, const double *__restrict__ qn_, long long sc,
                       double *pre, SubstepTimes tt)
{
    pdl_wait();
    pdl_launch_dependents();
    const long long per = (long long)r * m;
    const long long n = (long long)list[0] * per;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long e = t / per;
        const int rest = (int)(t - e * per), s = rest / m, f = rest - s * m;
        const GhostDesc g = gd[list[1 + e]];
        double v[3];
        coarse_stencil(g, qo, qn_, sc, f, s, tt.th[s], dim, v);
        double *p = pre + (((long long)s * m + f) * sc + g.src) * 3;
        p[0] = v[0];
        p[1] = v[1];
        p[2] = v[2];
    }
}

// one thread per (coarse cell, field): the sum of its r^d fine values in row
// order, times 1/r^d
__global__ void k_average_down(int dim, int m, const AvgDesc *__restrict__ ad, long long n,
                               const double *__restrict__ qf, long long sf, double *qc, long long sc, int r)
{
    pdl_wait();
    pdl_launch_dependents();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * m) return;
    const long long e = t / m;
    const int f = (int)(t - e * m);
    const AvgDesc a = ad[e];
    const int rr = (dim == 2) ? r : 1;
    const double inv = 1.0 / (double)(r * rr);
    const double *src = qf + (long long)f * sf + a.src;
    double s = 0.0;
    for (int jj = 0; jj < rr; jj++)
        for (int ii = 0; ii < r; ii++) s = s + src[(long long)jj * a.fsx + ii];
    qc[(long long)f * sc + a.dst] = s * inv;
}

// boundary map of a level index (no signs: the medium is even)
// (the final clamp only matters for the left neighbour of the outermost ghost
// cell on grids narrower than 3 cells, a value no step reads)
__device__ __forceinline__ int map_index(int I, int N, int bclo, int bchi)
{
    if (I < 0) {
        if (bclo == ADJAMR_BC_EXTRAP) I = 0;
        else if (bclo == ADJAMR_BC_WALL) I = -1 - I;
        else I = I + N;
    } else if (I >= N) {
        if (bchi == ADJAMR_BC_EXTRAP) I = N - 1;
        else if (bchi == ADJAMR_BC_WALL) I = 2 * N - 1 - I;
        else I = I - N;
    }
    return min(max(I, 0), N - 1);
}

__device__ void medium_at(const MediumDev &md, const LevelGeom &g, int I, int J, double *out)
{
    I = map_index(I, g.N, g.bc[0], g.bc[1]);
    if (g.dim == 2) J = map_index(J, g.M, g.bc[2], g.bc[3]);
    else J = 0;
    if (md.kind == ADJAMR_MEDIUM_LAYERED) {
        double c = (md.axis == 0) ? g.lo0 + ((double)I + 0.5) * g.dx : g.lo1 + ((double)J + 0.5) * g.dy;
        int k = 0;
        while (k < md.nl - 1 && md.iface[k] <= c) k++;
        out[0] = md.f0[k];
        out[1] = md.f1[k];
    } else {
        long long idx = (long long)J * md.N + I;
        out[0] = md.dense[idx];
        if (md.nmed > 1) out[1] = md.dense[(long long)md.N * md.M + idx];
    }
}

// coefficients of a cell from the primary medium of the cell (c0), of its
// x-neighbour below (cl) and of its y-neighbour below (cb)
__device__ void aux_from_medium(int eqn, int dim, const double *c0, const double *cl, const double *cb, long long idx,
                                double *aux, double *med, long long stride)
{
    med[idx] = c0[0];
    if (eqn == 0 || eqn == 1) med[stride + idx] = c0[1];
    if (eqn == 0 || eqn == 1) {
        double c = sqrt(c0[1] / c0[0]);
        double Z = c0[0] * c;
        double ccl = sqrt(cl[1] / cl[0]);
        double Zl = cl[0] * ccl;
        aux[idx] = c;
        aux[stride + idx] = Z;
        aux[2 * stride + idx] = 1.0 / (Zl + Z);
        if (dim == 2) {
            double ccb = sqrt(cb[1] / cb[0]);
            double Zb = cb[0] * ccb;
            aux[3 * stride + idx] = 1.0 / (Zb + Z);
        } else {
            aux[3 * stride + idx] = 0.0;
        }
        if (eqn == 1) {
            aux[4 * stride + idx] = 1.0 / c0[0];
            aux[5 * stride + idx] = c0[1];
        }
    } else {
        double hx = 0.5 * (cl[0] + c0[0]);
        double ghx = kGrav * hx;
        double cex = sqrt(ghx);
        double hy = (dim == 2) ? 0.5 * (cb[0] + c0[0]) : hx;
        double ghy = kGrav * hy;
        double cey = sqrt(ghy);
        if (eqn == 2) {
            aux[idx] = cex;
            aux[stride + idx] = 1.0 / cex;
            aux[2 * stride + idx] = ghx;
            aux[3 * stride + idx] = cey;
            aux[4 * stride + idx] = 1.0 / cey;
            aux[5 * stride + idx] = ghy;
        } else {
            aux[idx] = cex;
            aux[stride + idx] = 1.0 / cex;
            aux[2 * stride + idx] = cey;
            aux[3 * stride + idx] = 1.0 / cey;
            aux[4 * stride + idx] = kGrav * c0[0];
        }
    }
}

__device__ void aux_cell(int eqn, int dim, const MediumDev &md, const LevelGeom &g, int I, int J, long long idx,
                         double *aux, double *med, long long stride)
{
    double c0[2] = {0, 0}, cl[2] = {0, 0}, cb[2] = {0, 0};
    medium_at(md, g, I, J, c0);
    medium_at(md, g, I - 1, J, cl);
    if (dim == 2) medium_at(md, g, I, J - 1, cb);
    aux_from_medium(eqn, dim, c0, cl, cb, idx, aux, med, stride);
}

// the coefficients of every cell of the bordered index space (aux_cell's
// arithmetic, so the table holds the bits the per-cell path computes)
__global__ void k_aux_table(int eqn, const MediumDev *__restrict__ mdp, LevelGeom g, double *tab, long long n, int W,
                            int naux)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int j = (int)(t / W), i = (int)(t - (long long)j * W);
    const int I = i - 2, J = (g.dim == 2) ? j - 2 : 0;
    aux_cell(eqn, g.dim, *mdp, g, I, J, t, tab, tab + (long long)naux * n, n);
}

__global__ void k_aux_fill(int eqn, int dim, const AuxDesc *__restrict__ ad, long long n, double *aux, double *med,
                           long long stride, const MediumDev *__restrict__ mdp, LevelGeom g)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    AuxDesc d = ad[t];
    aux_cell(eqn, dim, *mdp, g, d.I, d.J, d.idx, aux, med, stride);
}

// ---------------------------------------------------------------- device-side regrid support
__device__ __forceinline__ int find_in_prefix(const long long *__restrict__ prefix, int np, long long t)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// boundary map with the sign flags of components 1 (x-normal) and 2 (y-normal)
__device__ __forceinline__ void bc_map_dev(const LevelIdx &g, int &I, int &J, int &f1, int &f2)
{
    f1 = f2 = 0;
    if (I < 0) {
        if (g.bc[0] == ADJAMR_BC_EXTRAP) I = 0;
        else if (g.bc[0] == ADJAMR_BC_WALL) { I = -1 - I; f1 = 1; }
        else I += g.N;
    } else if (I >= g.N) {
        if (g.bc[1] == ADJAMR_BC_EXTRAP) I = g.N - 1;
        else if (g.bc[1] == ADJAMR_BC_WALL) { I = 2 * g.N - 1 - I; f1 = 1; }
        else I -= g.N;
    }
    if (g.dim == 2) {
        if (J < 0) {
            if (g.bc[2] == ADJAMR_BC_EXTRAP) J = 0;
            else if (g.bc[2] == ADJAMR_BC_WALL) { J = -1 - J; f2 = 1; }
            else J += g.M;
        } else if (J >= g.M) {
            if (g.bc[3] == ADJAMR_BC_EXTRAP) J = g.M - 1;
            else if (g.bc[3] == ADJAMR_BC_WALL) { J = 2 * g.M - 1 - J; f2 = 1; }
            else J -= g.M;
        }
    } else {
        J = 0;
    }
}

__device__ __forceinline__ int owner_at(const int *__restrict__ owner, const LevelIdx &g, int I, int J)
{
    if (I < 0 || I >= g.N || J < 0 || J >= g.M) return -1;
    return owner[(long long)J * g.N + I];
}

// coarse-interpolation descriptor at in-domain fine cell (I, J); false if a
// coarse reference is not a cell of the coarser level (nesting violated)
__device__ bool coarse_desc_dev(int I, int J, int r, const int *__restrict__ owner_c, const LevelIdx &gc,
                                GhostDesc &g)
{
    int ic = I / r, jc = (gc.dim == 2) ? J / r : 0;
    g.kind = 1;
    g.fx = (double)(2 * (I - ic * r) + 1 - r) / (double)(2 * r);
    g.fy = (gc.dim == 2) ? (double)(2 * (J - jc * r) + 1 - r) / (double)(2 * r) : 0.0;
    const int di[5] = {0, -1, 1, 0, 0}, dj[5] = {0, 0, 0, -1, 1};
    long long ref[5] = {0, 0, 0, 0, 0};
    int nref = (gc.dim == 2) ? 5 : 3;
    bool ok = true;
    for (int k = 0; k < nref; k++) {
        int a = ic + di[k], b = jc + dj[k], f1, f2;
        bc_map_dev(gc, a, b, f1, f2);
        int o = owner_at(owner_c, gc, a, b);
        if (o < 0) {
            ok = false;
            o = 0;
        }
        ref[k] = o;
        g.signs |= (f1 << (2 + 2 * k)) | (f2 << (3 + 2 * k));
    }
    g.src = ref[0];
    g.cxm = ref[1];
    g.cxp = ref[2];
    g.cym = ref[3];
    g.cyp = ref[4];
    return ok;
}

__device__ __forceinline__ void owner_fill_at(const OwnerFillArgs &a, long long t)
{
    int p = find_in_prefix(a.prefix, a.np, t);
    const PatchDesc P = a.pd[p];
    long long k = t - a.prefix[p];
    int j = (int)(k / P.nx), i = (int)(k - (long long)j * P.nx);
    a.owner[(long long)(P.jlo + j) * a.g.N + P.ilo + i] = (int)(P.base + (long long)(j + a.g.gy) * P.sx + (i + 2));
}

__device__ __forceinline__ void ghost_build_at(const GhostBuildArgs &a, long long t)
{
    const LevelIdx &g = a.g;
    int p = find_in_prefix(a.gprefix, a.np, t);
    const PatchDesc P = a.pd[p];
    long long k = t - a.gprefix[p];
    const long long bottom = (long long)g.gy * P.sx, mid = (long long)P.ny * 4;
    int si, sj;
    if (k < bottom) {
        sj = (int)(k / P.sx);
        si = (int)(k - (long long)sj * P.sx);
    } else if (k < bottom + mid) {
        long long kk = k - bottom;
        int c = (int)(kk & 3);
        sj = g.gy + (int)(kk >> 2);
        si = (c < 2) ? c : P.nx + c;
    } else {
        long long kk = k - bottom - mid;
        int rr = (int)(kk / P.sx);
        sj = g.gy + P.ny + rr;
        si = (int)(kk - (long long)rr * P.sx);
    }
    int I = P.ilo + si - 2, J = P.jlo + sj - g.gy, f1, f2;
    bc_map_dev(g, I, J, f1, f2);
    GhostDesc d;
    d.dst = P.base + (long long)sj * P.sx + si;
    d.src = d.cxm = d.cxp = d.cym = d.cyp = 0;
    d.kind = 0;
    d.signs = 0;
    d.fx = d.fy = 0.0;
    int o = owner_at(a.owner, g, I, J);
    if (o >= 0) {
        d.src = o;
    } else if (a.owner_c) {
        if (!coarse_desc_dev(I, J, a.r, a.owner_c, a.gc, d)) atomicOr(a.err, 1);
    } else {
        atomicOr(a.err, 2);
        d.src = d.dst;  // harmless self-copy
    }
    d.signs |= f1 | (f2 << 1);
    a.out[t] = d;
    // list the coarse cell once (which of its ghost cells is listed is immaterial)
    if (d.kind != 0 && a.cmark && atomicExch(&a.cmark[d.src], a.cgen) != a.cgen)
        a.clist[1 + atomicAdd(&a.clist[0], 1ull)] = (unsigned long long)t;
}

__device__ __forceinline__ void avg_build_at(const AvgBuildArgs &a, long long t)
{
    const int r = a.r, dim = a.dim;
    int p = find_in_prefix(a.aprefix, a.np, t);
    const PatchDesc P = a.pd[p];
    long long k = t - a.aprefix[p];
    int na = P.nx / r;
    int bj = (int)(k / na), ai = (int)(k - (long long)bj * na);
    int ca = P.ilo / r + ai, cb = (dim == 2) ? P.jlo / r + bj : 0;
    int o = owner_at(a.owner_c, a.gc, ca, cb);
    if (o < 0) {
        atomicOr(a.err, 4);
        o = 0;
    }
    AvgDesc d;
    d.dst = o;
    int gy = (dim == 2) ? 2 : 0;
    int fj = (dim == 2) ? cb * r - P.jlo : 0;
    d.src = P.base + (long long)(fj + gy) * P.sx + (ca * r - P.ilo + 2);
    d.fsx = P.sx;
    d.pad = 0;
    a.out[t] = d;
}

__device__ __forceinline__ void init_new_at(const InitNewArgs &a, long long t)
{
    int p = find_in_prefix(a.prefix, a.np, t);
    const PatchDesc P = a.pd[p];
    long long k = t - a.prefix[p];
    int j = (int)(k / P.nx), i = (int)(k - (long long)j * P.nx);
    int I = P.ilo + i, J = P.jlo + j;
    long long dst = P.base + (long long)(j + a.g.gy) * P.sx + (i + 2);
    int o = a.owner_old ? owner_at(a.owner_old, a.g, I, J) : -1;
    if (o >= 0) {
        for (int f = 0; f < a.m; f++) a.qf[(long long)f * a.sf + dst] = a.qold[(long long)f * a.so + o];
        return;
    }
    GhostDesc d;
    d.signs = 0;
    if (!coarse_desc_dev(I, J, a.r, a.owner_c, a.gc, d)) atomicOr(a.err, 8);
    for (int f = 0; f < a.m; f++) a.qf[(long long)f * a.sf + dst] = interp_field(d, a.qc, a.qc, a.sc, f, 0, 0.0, a.g.dim);
}

__device__ __forceinline__ void aux_patches_at(const AuxPatchesArgs &a, long long t)
{
    const LevelIdx &g = a.g;
    int p = find_in_prefix(a.sprefix, a.np, t);
    const PatchDesc P = a.pd[p];
    long long k = t - a.sprefix[p];
    int sj = (int)(k / P.sx), si = (int)(k - (long long)sj * P.sx);
    const int I = P.ilo + si - 2, J = P.jlo + sj - g.gy;
    const long long idx = P.base + k;
    const AuxReuse &ru = a.ru;
    if (a.tb.tab) {
        const long long ti = (long long)(J + g.gy) * a.tb.width + (I + 2);
        for (int f = 0; f < ru.naux; f++)
            a.aux[(long long)f * a.stride + idx] = a.tb.tab[(long long)f * a.tb.stride + ti];
        for (int f = 0; f < ru.nmed; f++)
            a.med[(long long)f * a.stride + idx] = a.tb.tab[(long long)(ru.naux + f) * a.tb.stride + ti];
        return;
    }
    if (ru.owner) {
        const int o = owner_at(ru.owner, g, I, J);
        if (o >= 0) {
            for (int f = 0; f < ru.naux; f++)
                a.aux[(long long)f * a.stride + idx] = ru.aux[(long long)f * ru.stride + o];
            for (int f = 0; f < ru.nmed; f++)
                a.med[(long long)f * a.stride + idx] = ru.med[(long long)f * ru.stride + o];
            return;
        }
    }
    aux_cell(a.eqn, g.dim, *a.mdp, a.geom, I, J, idx, a.aux, a.med, a.stride);
}

// thread index of the calling thread within a part of a grid that starts at
// block b0; -1 outside it
__device__ __forceinline__ long long part_thread(unsigned b0, long long n)
{
    const long long t = (long long)(blockIdx.x - b0) * blockDim.x + threadIdx.x;
    return t < n ? t : -1;
}

__global__ void k_owner_fill(OwnerFillArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    const long long t = part_thread(0, a.n);
    if (t >= 0) owner_fill_at(a, t);
}

__global__ void k_ghost_build(GhostBuildArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    const long long t = part_thread(0, a.n);
    if (t >= 0) ghost_build_at(a, t);
}

__global__ void k_avg_build(AvgBuildArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    const long long t = part_thread(0, a.n);
    if (t >= 0) avg_build_at(a, t);
}

__global__ void k_init_new(InitNewArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    const long long t = part_thread(0, a.n);
    if (t >= 0) init_new_at(a, t);
}

__global__ void k_aux_patches(AuxPatchesArgs a)
{
    pdl_wait();
    pdl_launch_dependents();
    const long long t = part_thread(0, a.n);
    if (t >= 0) aux_patches_at(a, t);
}

// A level's rebuild, first launch: blocks [0, b1) fill the owner map, [b1,
// b2) the coefficients, [b2, grid) the new interior state.
__global__ void k_rebuild_a(OwnerFillArgs o, AuxPatchesArgs x, InitNewArgs in, unsigned b1, unsigned b2)
{
    pdl_wait();
    pdl_launch_dependents();
    if (blockIdx.x < b1) {
        const long long t = part_thread(0, o.n);
        if (t >= 0) owner_fill_at(o, t);
    } else if (blockIdx.x < b2) {
        const long long t = part_thread(b1, x.n);
        if (t >= 0) aux_patches_at(x, t);
    } else {
        const long long t = part_thread(b2, in.n);
        if (t >= 0) init_new_at(in, t);
    }
}

// second launch: blocks [0, b1) the ghost descriptors, [b1, grid) the
// average-down descriptors (both read the owner map of the first)
__global__ void k_rebuild_b(GhostBuildArgs gb, AvgBuildArgs ab, unsigned b1)
{
    pdl_wait();
    pdl_launch_dependents();
    if (blockIdx.x < b1) {
        const long long t = part_thread(0, gb.n);
        if (t >= 0) ghost_build_at(gb, t);
    } else {
        const long long t = part_thread(b1, ab.n);
        if (t >= 0) avg_build_at(ab, t);
    }
}

// ---------------------------------------------------------------- error estimate (Sec. 7)
// One thread per storage cell of the extended patches: the value as a ghost
// cell gets it (the level's own cell where it has one, else the coarse
// space-time interpolation), boundary-mapped, and the cell's coefficients.
__global__ void k_errest_ext(ErrEstArgs a, LevelIdx g, const int *__restrict__ owner, const double *__restrict__ q,
                             long long sq, const int *__restrict__ owner_c, LevelIdx gc, int r,
                             const double *__restrict__ qo, const double *__restrict__ qn, long long sc, int k,
                             double th, const MediumDev *__restrict__ md, LevelGeom geom, int *err)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nE) return;
    const int p = find_in_prefix(a.eprefix, a.np, t);
    const ErrEstPatch P = a.ep[p];
    const long long e = t - a.eprefix[p];
    const int ex = P.ne + 8, ge = (a.dim == 2) ? 4 : 0;
    const int sj = (int)(e / ex), si = (int)(e - (long long)sj * ex);
    const int I0 = P.ilo + si - 4, J0 = (a.dim == 2) ? P.jlo + sj - ge : 0;
    int I = I0, J = J0, f1, f2;
    bc_map_dev(g, I, J, f1, f2);
    GhostDesc d;
    d.dst = 0;
    d.src = d.cxm = d.cxp = d.cym = d.cyp = 0;
    d.kind = 0;
    d.signs = 0;
    d.fx = d.fy = 0.0;
    const int o = owner_at(owner, g, I, J);
    if (o >= 0) {
        d.src = o;
    } else if (owner_c) {
        if (!coarse_desc_dev(I, J, r, owner_c, gc, d)) atomicOr(err, 1);
    } else {
        atomicOr(err, 2);
    }
    d.signs |= f1 | (f2 << 1);
    const long long idx = P.ebase + e;
    for (int f = 0; f < a.m; f++) a.E[(long long)f * a.nE + idx] = ghost_value_direct(d, q, sq, qo, qn, sc, f, k, th, a.dim);
    aux_cell(a.eqn, a.dim, *md, geom, I0, J0, idx, a.auxE, a.medE, a.nE);
}

// primary medium of coarsened cell (a, b) of patch P (coarse storage
// coordinates): the mean of its children's, summed row by row
__device__ void errest_coarse_medium(const ErrEstPatch &P, int dim, int nmed, const MediumDev &md,
                                     const LevelGeom &geom, int ca, int cb, double *out)
{
    const int rr = (dim == 2) ? 2 : 1, ge = (dim == 2) ? 4 : 0;
    const double inv = 1.0 / (double)(2 * rr);
    double s[2] = {0.0, 0.0};
    for (int jj = 0; jj < rr; jj++)
        for (int ii = 0; ii < 2; ii++) {
            double v[2] = {0.0, 0.0};
            const int I = P.ilo + 2 * ca + ii - 4, J = (dim == 2) ? P.jlo + 2 * cb + jj - ge : 0;
            medium_at(md, geom, I, J, v);
            for (int f = 0; f < nmed; f++) s[f] = s[f] + v[f];
        }
    for (int f = 0; f < nmed; f++) out[f] = s[f] * inv;
    if (nmed < 2) out[1] = 0.0;
}

// One thread per storage cell of the coarsened patches: the mean of the
// children's state and medium, and the coefficients of that medium.
__global__ void k_errest_coarse(ErrEstArgs a, const MediumDev *__restrict__ md, LevelGeom geom)
{
    pdl_wait();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nC) return;
    const int p = find_in_prefix(a.cprefix, a.np, t);
    const ErrEstPatch P = a.ep[p];
    const long long e = t - a.cprefix[p];
    const int cx = P.ne / 2 + 4, ex = P.ne + 8, rr = (a.dim == 2) ? 2 : 1;
    const int b = (int)(e / cx), ca = (int)(e - (long long)b * cx);
    const double inv = 1.0 / (double)(2 * rr);
    const long long idx = P.cbase + e;
    for (int f = 0; f < a.m; f++) {
        double s = 0.0;
        for (int jj = 0; jj < rr; jj++)
            for (int ii = 0; ii < 2; ii++)
                s = s + a.E[(long long)f * a.nE + P.ebase + (long long)(b * rr + jj) * ex + 2 * ca + ii];
        a.C[(long long)f * a.nC + idx] = s * inv;
    }
    const int nmed = nmed_of(a.eqn);
    double c0[2], cl[2], cb_[2] = {0.0, 0.0};
    errest_coarse_medium(P, a.dim, nmed, *md, geom, ca, b, c0);
    errest_coarse_medium(P, a.dim, nmed, *md, geom, ca - 1, b, cl);
    if (a.dim == 2) errest_coarse_medium(P, a.dim, nmed, *md, geom, ca, b - 1, cb_);
    aux_from_medium(a.eqn, a.dim, c0, cl, cb_, idx, a.auxC, a.medC, a.nC);
}

// One thread per interior cell of the level: tau of its 2 x 2 (1D: 2) block.
__global__ void k_errest_tau(ErrEstArgs a, const long long *__restrict__ iprefix, long long n, double *tau,
                             long long st)
{
    pdl_wait();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int p = find_in_prefix(iprefix, a.np, t);
    const ErrEstPatch P = a.ep[p];
    const long long e = t - iprefix[p];
    const int j = (int)(e / P.nx), i = (int)(e - (long long)j * P.nx);
    const int ca = i / 2, cb = (a.dim == 2) ? j / 2 : 0;
    const int rr = (a.dim == 2) ? 2 : 1, ge = (a.dim == 2) ? 4 : 0, gc = (a.dim == 2) ? 2 : 0, gy = gc;
    const int ex = P.ne + 8, cx = P.ne / 2 + 4;
    const double inv = 1.0 / (double)(2 * rr);
    const long long dst = P.abase + (long long)(j + gy) * P.asx + (i + 2);
    for (int f = 0; f < a.m; f++) {
        double s = 0.0;
        for (int jj = 0; jj < rr; jj++)
            for (int ii = 0; ii < 2; ii++)
                s = s + a.E[(long long)f * a.nE + P.ebase + (long long)(cb * rr + jj + ge) * ex + 2 * ca + ii + 4];
        const double fc = s * inv;
        const double c1 = a.C1[(long long)f * a.nC + P.cbase + (long long)(cb + gc) * cx + ca + 2];
        tau[(long long)f * st + dst] = (fc - c1) / 6.0;
    }
}

// ---------------------------------------------------------------- flagging
__device__ __forceinline__ void bilinear_setup(double x, double lo, double hi, int na, int &a, double &w)
{
    double dxa = (hi - lo) / (double)na;
    double xi = (x - lo) / dxa - 0.5;
    xi = fmin(fmax(xi, 0.0), (double)(na - 1));
    a = (int)floor(xi);
    if (a > na - 2) a = na - 2;
    if (a < 0) a = 0;
    w = xi - (double)a;
}

__device__ __forceinline__ double adj_interp(const FlagArgs &A, int n, int f, int a, double wx, int b, double wy)
{
    const double *s = A.snaps + ((long long)n * A.m + f) * (long long)A.ax * A.ay;
    if (A.dim == 1) {
        if (A.ax == 1) return s[0];
        return (1.0 - wx) * s[a] + wx * s[a + 1];
    }
    double omx = 1.0 - wx;
    long long r0 = (long long)b * A.ax, r1 = (long long)(b + 1) * A.ax;
    double v0 = omx * s[r0 + a] + wx * s[r0 + a + 1];
    double v1 = omx * s[r1 + a] + wx * s[r1 + a + 1];
    return (1.0 - wy) * v0 + wy * v1;
}

__device__ __forceinline__ double snap_time(const FlagArgs &A, int n) { return A.t0 + (double)n * A.dts; }

__global__ void k_flag(FlagArgs A)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool flagged = false;
    int fI = 0x7fffffff, fJ = 0x7fffffff, gI = -1, gJ = -1;  // bounding-box contributions
    if (t < A.ncells) {
        // patch containing interior cell t (binary search on the prefix)
        int lo = 0, hi = A.np - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (A.cell_prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const PatchDesc P = A.patches[lo];
        long long k = t - A.cell_prefix[lo];
        int j = (int)(k / P.nx), i = (int)(k - (long long)j * P.nx);
        int gy = (A.dim == 2) ? 2 : 0;
        long long cell = P.base + (long long)(j + gy) * P.sx + (i + 2);
        int I = P.ilo + i, J = P.jlo + j;
        double x = A.lo0 + ((double)I + 0.5) * A.dx;
        double y = (A.dim == 2) ? A.lo1 + ((double)J + 0.5) * A.dy : 0.0;
        double Q[3];
        for (int f = 0; f < A.m; f++) Q[f] = A.q[(long long)f * A.stride + cell];
        // flag iff the window maximum of |q^ . q| exceeds tol: the scan stops
        // at the first term above tol (the decision is that of the full max);
        // a dry adjoint cell sets the inner product to zero (Sec. 5.3)
        bool hit = false;
        if (A.mode == ADJAMR_FLAG_DIFFERENCE) {
            // undivided centred differences from the ghost-filled arena
            double val = 0.0;
            for (int f = 0; f < A.m; f++) {
                const double *qf = A.q + (long long)f * A.stride;
                val = fmax(val, fabs(qf[cell + 1] - qf[cell - 1]));
                if (A.dim == 2) val = fmax(val, fabs(qf[cell + P.sx] - qf[cell - P.sx]));
            }
            hit = val > A.tol;
        } else if (A.mode == ADJAMR_FLAG_SURFACE) {
            hit = fabs(Q[0]) > A.tol;
        } else if (A.mode == ADJAMR_FLAG_RICHARDSON) {
            // q holds the error estimate: its largest component
            double val = 0.0;
            for (int f = 0; f < A.m; f++) val = fmax(val, fabs(Q[f]));
            hit = val > A.tol;
        } else if (A.S >= 2) {
            double dxa = (A.hi0 - A.lo0) / (double)A.ax;
            int ac = (int)floor((x - A.lo0) / dxa);
            ac = min(max(ac, 0), A.ax - 1);
            int bc = 0;
            if (A.dim == 2) {
                double dya = (A.hi1 - A.lo1) / (double)A.ay;
                bc = (int)floor((y - A.lo1) / dya);
                bc = min(max(bc, 0), A.ay - 1);
            }
            bool dry = A.wet && !A.wet[(long long)bc * A.ax + ac];
            int a, b = 0;
            double wx, wy = 0.0;
            bilinear_setup(x, A.lo0, A.hi0, A.ax, a, wx);
            if (A.dim == 2) bilinear_setup(y, A.lo1, A.hi1, A.ay, b, wy);
            if (dry) {
                hit = 0.0 > A.tol;
            } else if (A.mode == ADJAMR_FLAG_BRACKET_MAX) {
                // Blocks of snapshots whose bound sum_f |q_f| max_f |q^| cannot
                // exceed tol are skipped: every computed |q^_n . q| of the block
                // is at most the bound times (1 + 12 ulp), far inside the 1e-12
                // margin, so the decision is that of the full scan.
                const long long plane = (long long)A.ax * A.ay;
                const long long cell = (long long)b * A.ax + a;
                for (int blk = A.nlo / kSnapBlock; blk <= A.nhi / kSnapBlock && !hit; blk++) {
                    if (A.bmax) {
                        double B = 0.0;
                        for (int f = 0; f < A.m; f++)
                            B = fma(fabs(Q[f]), A.bmax[((long long)blk * A.m + f) * plane + cell], B);
                        if (B * (1.0 + 1e-12) <= A.tol) continue;
                    }
                    int n0 = max(A.nlo, blk * kSnapBlock), n1 = min(A.nhi, blk * kSnapBlock + kSnapBlock - 1);
                    for (int n = n0; n <= n1 && !hit; n++) {
                        double d = 0.0;
                        for (int f = 0; f < A.m; f++) {
                            double av = adj_interp(A, n, f, a, wx, b, wy);
                            d = (f == 0) ? av * Q[0] : d + av * Q[f];
                        }
                        hit = fabs(d) > A.tol;
                    }
                }
                if (A.nlo > A.nhi) hit = 0.0 > A.tol;
            } else {
                // q^ linear in time: values at t, at T, and snapshots strictly inside
                for (int pass = 0; pass < 2 && !hit; pass++) {
                    double tau = pass == 0 ? A.t : A.T;
                    int n = 0;
                    while (n < A.S - 2 && snap_time(A, n + 1) <= tau) n++;
                    double w = (tau - snap_time(A, n)) / A.dts;
                    double d = 0.0;
                    for (int f = 0; f < A.m; f++) {
                        double a0 = adj_interp(A, n, f, a, wx, b, wy), a1 = adj_interp(A, n + 1, f, a, wx, b, wy);
                        double av = (1.0 - w) * a0 + w * a1;
                        d = (f == 0) ? av * Q[0] : d + av * Q[f];
                    }
                    hit = fabs(d) > A.tol;
                }
                for (int n = 0; n < A.S && !hit; n++) {
                    double tn = snap_time(A, n);
                    if (!(tn > A.t && tn < A.T)) continue;
                    double d = 0.0;
                    for (int f = 0; f < A.m; f++) {
                        double av = adj_interp(A, n, f, a, wx, b, wy);
                        d = (f == 0) ? av * Q[0] : d + av * Q[f];
                    }
                    hit = fabs(d) > A.tol;
                }
            }
        } else {
            hit = 0.0 > A.tol;
        }
        flagged = hit;
        if (A.flags_patch) A.flags_patch[t] = flagged ? 1 : 0;
        if (A.flags_bits && flagged) atomicOr(A.flags_bits + (long long)J * A.pitch64 + (I >> 6), 1ull << (I & 63));
        if (flagged) {
            fI = gI = I;
            fJ = gJ = J;
        }
    }
    unsigned bal = __ballot_sync(0xffffffffu, flagged);
    if (bal) {
        fI = __reduce_min_sync(0xffffffffu, fI);
        fJ = __reduce_min_sync(0xffffffffu, fJ);
        gI = __reduce_max_sync(0xffffffffu, gI);
        gJ = __reduce_max_sync(0xffffffffu, gJ);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(A.count, (unsigned long long)__popc(bal));
            if (A.bbox) {
                atomicMax(A.bbox + 0, 0x7fffffff - fI);
                atomicMax(A.bbox + 1, gI + 1);
                atomicMax(A.bbox + 2, 0x7fffffff - fJ);
                atomicMax(A.bbox + 3, gJ + 1);
            }
        }
    }
}

// Bracket-max flagging over the level's dense index space: thread (cell,
// group) scans the group's snapshot blocks of the window.  A cell is flagged
// iff some |q^_n . q| of the window exceeds tol (Sec. 4; the decision does not
// depend on the order the snapshots are visited, so the window may be split
// among threads); blocks whose bound cannot exceed tol are skipped as in
// k_flag.  The first thread to set a cell's flag counts it; warp shuffles
// reduce the count and the bounding box of the flags.
// Gauge record: for every gauge, the level-0 time and the values of the cell
// holding the point on the finest level with a patch there.
__global__ void k_gauges(GaugeArgs G)
{
    pdl_wait();
    pdl_launch_dependents();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G.n) return;
    double *o = G.out + (long long)g * (1 + G.m);
    o[0] = G.t;
    for (int f = 0; f < G.m; f++) o[1 + f] = 0.0;
    for (int l = G.nlev - 1; l >= 0; l--) {
        if (!G.owner[l]) continue;
        const int I = G.gi[l * G.n + g], J = G.gj[l * G.n + g];
        const int c = G.owner[l][(long long)J * G.N[l] + I];
        if (c < 0) continue;
        for (int f = 0; f < G.m; f++) o[1 + f] = G.q[l][(long long)f * G.stride[l] + c];
        break;
    }
}

template <int MF>
__global__ void k_flag_dense(FlagArgs A)
{
    const long long NM = (long long)A.N * A.M;
    const long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y;
    bool hit = false, fresh = false;
    int fI = 0x7fffffff, fJ = 0x7fffffff, gI = -1, gJ = -1;
    if (cidx < NM) {
        const int o = A.owner[cidx];
        if (o >= 0) {
            const int J = (int)(cidx / A.N), I = (int)(cidx - (long long)J * A.N);
            const int ac = A.tab_ac[I], bc = (A.dim == 2) ? A.tab_bc[J] : 0;
            const bool dry = A.wet && !A.wet[(long long)bc * A.ax + ac];
            if (A.S < 2 || dry || A.nlo > A.nhi) {
                hit = (grp == 0) && (0.0 > A.tol);
            } else {
                double Q[MF];
#pragma unroll
                for (int f = 0; f < MF; f++) Q[f] = A.q[(long long)f * A.stride + o];
                const int a = A.tab_a[I], b = (A.dim == 2) ? A.tab_b[J] : 0;
                const double wx = A.tab_wx[I], wy = (A.dim == 2) ? A.tab_wy[J] : 0.0;
                const long long plane = (long long)A.ax * A.ay;
                const long long acell = (long long)b * A.ax + a;
                const volatile unsigned long long *done = A.flags_bits + (long long)J * A.pitch64 + (I >> 6);
                const unsigned long long bit = 1ull << (I & 63);
                const int blo = A.nlo / kSnapBlock + grp * A.gblk;
                const int bhi = min(A.nhi / kSnapBlock, blo + A.gblk - 1);
                for (int blk = blo; blk <= bhi && !hit; blk++) {
                    if (*done & bit) break;  // set by another group: nothing left to decide
                    double B = 0.0;
#pragma unroll
                    for (int f = 0; f < MF; f++)
                        B = fma(fabs(Q[f]), A.bmax[((long long)blk * MF + f) * plane + acell], B);
                    if (B * (1.0 + 1e-12) <= A.tol) continue;
                    // the block's snapshots without an early exit, so that their
                    // loads are in flight together
                    const int n0 = blk * kSnapBlock;
#pragma unroll
                    for (int k = 0; k < kSnapBlock; k++) {
                        const int n = n0 + k;
                        if (n < A.nlo || n > A.nhi) continue;
                        double d = 0.0;
#pragma unroll
                        for (int f = 0; f < MF; f++) {
                            double av = adj_interp(A, n, f, a, wx, b, wy);
                            d = (f == 0) ? av * Q[0] : d + av * Q[f];
                        }
                        hit = hit || fabs(d) > A.tol;
                    }
                }
            }
            if (hit) {
                const unsigned long long bit = 1ull << (I & 63);
                fresh = (atomicOr(A.flags_bits + (long long)J * A.pitch64 + (I >> 6), bit) & bit) == 0;
                fI = gI = I;
                fJ = gJ = J;
            }
        }
    }
    const unsigned fr = __ballot_sync(0xffffffffu, fresh);
    if (__any_sync(0xffffffffu, hit)) {
        fI = __reduce_min_sync(0xffffffffu, fI);
        fJ = __reduce_min_sync(0xffffffffu, fJ);
        gI = __reduce_max_sync(0xffffffffu, gI);
        gJ = __reduce_max_sync(0xffffffffu, gJ);
        if ((threadIdx.x & 31) == 0) {
            if (fr) atomicAdd(A.count, (unsigned long long)__popc(fr));
            atomicMax(A.bbox + 0, 0x7fffffff - fI);
            atomicMax(A.bbox + 1, gI + 1);
            atomicMax(A.bbox + 2, 0x7fffffff - fJ);
            atomicMax(A.bbox + 3, gJ + 1);
        }
    }
}

// count and bounding box of this warp's flags: a shuffle reduction and one
// set of atomics per warp (every lane calls it)
__device__ __forceinline__ void flag_reduce(const FlagArgs &A, bool any_hit, unsigned nfresh, int fI, int gI, int fJ,
                                            int gJ)
{
    const unsigned total = __reduce_add_sync(0xffffffffu, nfresh);
    if (__any_sync(0xffffffffu, any_hit)) {
        fI = __reduce_min_sync(0xffffffffu, fI);
        fJ = __reduce_min_sync(0xffffffffu, fJ);
        gI = __reduce_max_sync(0xffffffffu, gI);
        gJ = __reduce_max_sync(0xffffffffu, gJ);
        if ((threadIdx.x & 31) == 0) {
            if (total) atomicAdd(A.count, (unsigned long long)total);
            atomicMax(A.bbox + 0, 0x7fffffff - fI);
            atomicMax(A.bbox + 1, gI + 1);
            atomicMax(A.bbox + 2, 0x7fffffff - fJ);
            atomicMax(A.bbox + 3, gJ + 1);
        }
    }
}

// Pass 1 of the two-pass flagging: one thread per cell of the level's index
// space.  Cells whose test needs no snapshot (dry adjoint cell, fewer than 2
// snapshots, empty window) are decided here; for the others every snapshot
// block of the window whose bound sum_f |q_f| max |q^_f| can exceed tol (see
// k_flag) is appended to the work list, a warp at a time.
template <int MF>
__global__ void k_flag_bound(FlagArgs A, FlagWork W)
{
    const long long NM = (long long)A.N * A.M;
    const long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool hit = false, active = false;
    unsigned fresh = 0;
    int fI = 0x7fffffff, fJ = 0x7fffffff, gI = -1, gJ = -1;
    double Q[MF];
#pragma unroll
    for (int f = 0; f < MF; f++) Q[f] = 0.0;
    long long acell = 0;
    if (cidx < NM) {
        const int o = A.owner[cidx];
        if (o >= 0) {
            const int J = (int)(cidx / A.N), I = (int)(cidx - (long long)J * A.N);
            const int ac = A.tab_ac[I], bc = (A.dim == 2) ? A.tab_bc[J] : 0;
            const bool dry = A.wet && !A.wet[(long long)bc * A.ax + ac];
            if (A.S < 2 || dry || A.nlo > A.nhi) {
                hit = 0.0 > A.tol;
                if (hit) {
                    const unsigned long long bit = 1ull << (I & 63);
                    fresh = (atomicOr(A.flags_bits + (long long)J * A.pitch64 + (I >> 6), bit) & bit) == 0;
                    fI = gI = I;
                    fJ = gJ = J;
                }
            } else {
                active = true;
#pragma unroll
                for (int f = 0; f < MF; f++) Q[f] = A.q[(long long)f * A.stride + o];
                const int a = A.tab_a[I], b = (A.dim == 2) ? A.tab_b[J] : 0;
                acell = (long long)b * A.ax + a;
            }
        }
    }
    // the window's blocks are the same for every thread of the launch
    const long long plane = (long long)A.ax * A.ay;
    const int b1 = (A.nlo <= A.nhi) ? A.nhi / kSnapBlock : -1;
    for (int blk = A.nlo / kSnapBlock; blk <= b1; blk++) {
        bool push = false;
        if (active) {
            double B = 0.0;
#pragma unroll
            for (int f = 0; f < MF; f++) B = fma(fabs(Q[f]), A.bmax[((long long)blk * MF + f) * plane + acell], B);
            push = B * (1.0 + 1e-12) > A.tol;
        }
        const unsigned m = __ballot_sync(0xffffffffu, push);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(W.ctr, (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (push) {
                const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
                if (slot < (unsigned long long)W.cap) W.items[slot] = ((unsigned long long)cidx << 16) | (unsigned)blk;
                else W.ctr[1] = 1;
            }
        }
    }
    flag_reduce(A, hit, fresh, fI, gI, fJ, gJ);
}

// Pass 2: thread t evaluates snapshot t % 8 of listed block t / 8 (a grid
// striding over the list), skipping cells already flagged.
template <int MF>
__global__ void k_flag_eval(FlagArgs A, FlagWork W)
{
    const unsigned long long listed = W.ctr[0];
    const unsigned long long nitem = listed < (unsigned long long)W.cap ? listed : (unsigned long long)W.cap;
    const unsigned long long total = nitem * kSnapBlock;
    bool any = false;
    unsigned fresh = 0;
    int fI = 0x7fffffff, fJ = 0x7fffffff, gI = -1, gJ = -1;
    for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long item = W.items[t / kSnapBlock];
        const int n = (int)(item & 0xffff) * kSnapBlock + (int)(t % kSnapBlock);
        if (n < A.nlo || n > A.nhi) continue;
        const long long cidx = (long long)(item >> 16);
        const int J = (int)(cidx / A.N), I = (int)(cidx - (long long)J * A.N);
        unsigned long long *word = A.flags_bits + (long long)J * A.pitch64 + (I >> 6);
        const unsigned long long bit = 1ull << (I & 63);
        if (*(volatile unsigned long long *)word & bit) continue;  // decided by another snapshot
        const int o = A.owner[cidx];
        const int a = A.tab_a[I], b = (A.dim == 2) ? A.tab_b[J] : 0;
        const double wx = A.tab_wx[I], wy = (A.dim == 2) ? A.tab_wy[J] : 0.0;
        double d = 0.0;
#pragma unroll
        for (int f = 0; f < MF; f++) {
            const double av = adj_interp(A, n, f, a, wx, b, wy);
            const double qf = A.q[(long long)f * A.stride + o];
            d = (f == 0) ? av * qf : d + av * qf;
        }
        if (fabs(d) > A.tol) {
            any = true;
            if ((atomicOr(word, bit) & bit) == 0) fresh++;
            fI = min(fI, I);
            gI = max(gI, I);
            fJ = min(fJ, J);
            gJ = max(gJ, J);
        }
    }
    flag_reduce(A, any, fresh, fI, gI, fJ, gJ);
}

__global__ void k_block_max(const double *__restrict__ snaps, int S, int m, int ax, int ay, int dim, int nblk,
                            double *bmax)
{
    long long plane = (long long)ax * ay;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nblk * m * plane) return;
    long long cell = t % plane;
    int f = (int)((t / plane) % m);
    int blk = (int)(t / (plane * m));
    int a = (int)(cell % ax), b = (int)(cell / ax);
    int a1 = min(a + 1, ax - 1), b1 = (dim == 2) ? min(b + 1, ay - 1) : b;
    double mx = 0.0;
    for (int n = blk * kSnapBlock; n < min(S, blk * kSnapBlock + kSnapBlock); n++) {
        const double *sp = snaps + ((long long)n * m + f) * plane;
        mx = fmax(mx, fabs(sp[(long long)b * ax + a]));
        mx = fmax(mx, fabs(sp[(long long)b * ax + a1]));
        mx = fmax(mx, fabs(sp[(long long)b1 * ax + a]));
        mx = fmax(mx, fabs(sp[(long long)b1 * ax + a1]));
    }
    bmax[t] = mx;
}

// ---------------------------------------------------------------- functional
__global__ void k_func_terms(const long long *__restrict__ idx, const double *__restrict__ area, long long n,
                             const double *__restrict__ q, double weight, double *out)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = weight * (q[idx[t]] * area[t]);
}

// one CTA: repeated pairwise passes a[i] = a[2i] + a[2i+1], odd tail carried.
// Chunks of blockDim pairs are processed with a uniform trip count, so every
// thread meets every barrier; within a chunk all pairs are read before any
// result is written (chunk c writes [cB, (c+1)B), later chunks read >= 2(c+1)B).
__global__ void k_pairwise(double *a, long long n, double *out)
{
    const long long B = blockDim.x;
    while (n > 1) {
        long long h = n / 2;
        for (long long base = 0; base < h; base += B) {
            long long i = base + threadIdx.x;
            double s = 0.0;
            if (i < h) s = a[2 * i] + a[2 * i + 1];
            __syncthreads();
            if (i < h) a[i] = s;
            __syncthreads();
        }
        if (threadIdx.x == 0 && (n & 1)) a[h] = a[n - 1];
        __syncthreads();
        n = (n + 1) / 2;
    }
    if (threadIdx.x == 0) *out = (n == 1) ? a[0] : 0.0;
}

__global__ void k_gather(int m, const long long *__restrict__ map, long long n, const double *__restrict__ q,
                         long long stride, double *dst)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    for (int f = 0; f < m; f++) dst[(long long)f * n + t] = q[(long long)f * stride + map[t]];
}

inline unsigned nblk(long long n) { return (unsigned)((n + kT - 1) / kT); }
constexpr int kEB = 64;  // block size of the error-estimate kernels
inline unsigned nblk_of(long long n) { return nblk(n); }

}  // namespace

cudaError_t launch_ghost_fill(int dim, int m, const GhostDesc *g, long long n, double *qf, long long sf,
                              const double *qc_old, const double *qc_new, long long sc, int k, int r, cudaStream_t s,
                              bool early, const double *pre_k, CpreArgs cp, int cp_blocks)
{
    if (n <= 0) return cudaSuccess;
    const double th = (double)k / (double)r;  // same division as the oracle's, on the host
    unsigned grid = nblk(n * m);
    if (cp.list) {
        if (cp.r < 2 || cp.r > kMaxSubsteps || cp_blocks < 1) return cudaErrorInvalidValue;
        for (int j = 0; j < cp.r; j++) cp.tt.th[j] = (double)j / (double)cp.r;  // as the oracle's, on the host
        grid += (unsigned)cp_blocks;
    }
    return launch_pdl(k_ghost_fill, dim3(grid), dim3(kT), 0, s, dim, m, g, n, qf, sf, qc_old, qc_new, sc, k, th,
                      early && pdl_enabled() ? 1 : 0, pre_k, cp);
}

cudaError_t launch_cpre(const GhostDesc *g, const unsigned long long *list, long long nmax, int m, int r, int dim,
                        const double *qc_old, const double *qc_new, long long sc, double *pre, int grid,
                        cudaStream_t s)
{
    if (nmax <= 0) return cudaSuccess;
    if (r < 1 || r > kMaxSubsteps) return cudaErrorInvalidValue;
    SubstepTimes tt{};
    for (int k = 0; k < r; k++) tt.th[k] = (double)k / (double)r;  // same division as the oracle's, on the host
    const long long need = nblk(nmax * r * m);
    const int g_ = (int)std::max(1ll, std::min(need, (long long)grid));
    return launch_pdl(k_cpre, dim3(g_), dim3(kT), 0, s, g, list, m, r, dim, qc_old, qc_new, sc, pre, tt);
}

cudaError_t launch_average_down(int dim, int m, const AvgDesc *a, long long n, const double *qf, long long sf,
                                double *qc, long long sc, int r, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    return launch_pdl(k_average_down, dim3(nblk(n * m)), dim3(kT), 0, s, dim, m, a, n, qf, sf, qc, sc, r);
}

cudaError_t launch_aux_fill(int eqn, int dim, const AuxDesc *d, long long n, double *aux, double *med,
                            long long stride, const MediumDev *mdev, LevelGeom geom, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_aux_fill<<<nblk(n), kT, 0, s>>>(eqn, dim, d, n, aux, med, stride, mdev, geom);
    return cudaGetLastError();
}

cudaError_t launch_owner_fill(const OwnerFillArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    return launch_pdl(k_owner_fill, dim3(nblk(a.n)), dim3(kT), 0, s, a);
}

cudaError_t launch_ghost_build(const GhostBuildArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    if (a.cmark && (a.cgen <= 0 || !a.clist)) return cudaErrorInvalidValue;
    return launch_pdl(k_ghost_build, dim3(nblk(a.n)), dim3(kT), 0, s, a);
}

cudaError_t launch_avg_build(const AvgBuildArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    return launch_pdl(k_avg_build, dim3(nblk(a.n)), dim3(kT), 0, s, a);
}

cudaError_t launch_rebuild(const OwnerFillArgs &o, const AuxPatchesArgs &x, const InitNewArgs &in,
                           const GhostBuildArgs &gb, const AvgBuildArgs &ab, cudaStream_t s, int *nlaunch)
{
    *nlaunch = 0;
    if (gb.n > 0 && gb.cmark && (gb.cgen <= 0 || !gb.clist)) return cudaErrorInvalidValue;
    auto blocks = [](long long n) { return n > 0 ? nblk(n) : 0u; };
    const unsigned a1 = blocks(o.n), a2 = a1 + blocks(x.n), a3 = a2 + blocks(in.n);
    if (a3 > 0) {
        const cudaError_t e = launch_pdl(k_rebuild_a, dim3(a3), dim3(kT), 0, s, o, x, in, a1, a2);
        if (e != cudaSuccess) return e;
        ++*nlaunch;
    }
    const unsigned b1 = blocks(gb.n), b2 = b1 + blocks(ab.n);
    if (b2 > 0) {
        const cudaError_t e = launch_pdl(k_rebuild_b, dim3(b2), dim3(kT), 0, s, gb, ab, b1);
        if (e != cudaSuccess) return e;
        ++*nlaunch;
    }
    return cudaSuccess;
}

cudaError_t launch_errest_fill(const ErrEstArgs &a, LevelIdx g, const int *owner, const double *q, long long sq,
                               const int *owner_c, LevelIdx gc, int r, const double *qo, const double *qn,
                               long long sc, int k, const MediumDev *md, LevelGeom geom, int *err, cudaStream_t s)
{
    if (a.nE <= 0 || a.nC <= 0) return cudaSuccess;
    const double th = (r > 0) ? (double)k / (double)r : 0.0;  // as the ghost fill's, on the host
    // blocks of 64: these kernels are FP64-latency bound on levels of a few
    // thousand cells, so they are spread over as many SMs as possible
    k_errest_ext<<<(unsigned)((a.nE + kEB - 1) / kEB), kEB, 0, s>>>(a, g, owner, q, sq, owner_c, gc, r, qo, qn, sc, k,
                                                                    th, md, geom, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pdl(k_errest_coarse, dim3((unsigned)((a.nC + kEB - 1) / kEB)), dim3(kEB), 0, s, a, md, geom);
}

cudaError_t launch_errest_tau(const ErrEstArgs &a, const long long *iprefix, long long ninterior, double *tau,
                              long long st, cudaStream_t s)
{
    if (ninterior <= 0) return cudaSuccess;
    return launch_pdl(k_errest_tau, dim3((unsigned)((ninterior + kEB - 1) / kEB)), dim3(kEB), 0, s, a, iprefix,
                      ninterior, tau, st);
}

cudaError_t launch_init_new(const InitNewArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    return launch_pdl(k_init_new, dim3(nblk(a.n)), dim3(kT), 0, s, a);
}

cudaError_t launch_aux_patches(const AuxPatchesArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    return launch_pdl(k_aux_patches, dim3(nblk(a.n)), dim3(kT), 0, s, a);
}

cudaError_t launch_aux_table(int eqn, const MediumDev *mdev, LevelGeom geom, double *tab, cudaStream_t s)
{
    const int W = geom.N + 4, H = (geom.dim == 2) ? geom.M + 4 : 1;
    const long long n = (long long)W * H;
    k_aux_table<<<nblk(n), kT, 0, s>>>(eqn, mdev, geom, tab, n, W, naux_of(eqn));
    return cudaGetLastError();
}

cudaError_t launch_block_max(const double *snaps, int S, int m, int ax, int ay, int dim, double *bmax, cudaStream_t s)
{
    int nblk = (S + kSnapBlock - 1) / kSnapBlock;
    long long n = (long long)nblk * m * ax * ay;
    if (n <= 0) return cudaSuccess;
    k_block_max<<<nblk_of(n), kT, 0, s>>>(snaps, S, m, ax, ay, dim, nblk, bmax);
    return cudaGetLastError();
}

cudaError_t launch_gauges(const GaugeArgs &g, cudaStream_t s)
{
    if (g.n <= 0) return cudaSuccess;
    return launch_pdl(k_gauges, dim3((g.n + kT - 1) / kT), dim3(kT), 0, s, g);
}

cudaError_t launch_flag_twopass(const FlagArgs &a, const FlagWork &w, int eval_grid, cudaStream_t s)
{
    const long long nm = (long long)a.N * a.M;
    if (nm <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((nm + kT - 1) / kT);
    if (a.m == 3) {
        k_flag_bound<3><<<nb, kT, 0, s>>>(a, w);
        k_flag_eval<3><<<eval_grid, kT, 0, s>>>(a, w);
    } else if (a.m == 2) {
        k_flag_bound<2><<<nb, kT, 0, s>>>(a, w);
        k_flag_eval<2><<<eval_grid, kT, 0, s>>>(a, w);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_flag_dense(const FlagArgs &a, int ngroup, cudaStream_t s)
{
    const long long nm = (long long)a.N * a.M;
    if (nm <= 0 || ngroup <= 0) return cudaSuccess;
    dim3 grid((unsigned)((nm + kT - 1) / kT), (unsigned)ngroup);
    if (a.m == 3) k_flag_dense<3><<<grid, kT, 0, s>>>(a);
    else if (a.m == 2) k_flag_dense<2><<<grid, kT, 0, s>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_flag(const FlagArgs &a, cudaStream_t s)
{
    if (a.ncells <= 0) return cudaSuccess;
    k_flag<<<nblk(a.ncells), kT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_func_terms(const long long *idx, const double *area, long long n, const double *q, double weight,
                              double *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_func_terms<<<nblk(n), kT, 0, s>>>(idx, area, n, q, weight, out);
    return cudaGetLastError();
}

cudaError_t launch_pairwise(double *a, long long n, double *out, cudaStream_t s)
{
    k_pairwise<<<1, 1024, 0, s>>>(a, n, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_interior(int m, const long long *map, long long n, const double *q, long long stride,
                                   double *dst, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_gather<<<nblk(n), kT, 0, s>>>(m, map, n, q, stride, dst);
    return cudaGetLastError();
}

}  // namespace adjamr
