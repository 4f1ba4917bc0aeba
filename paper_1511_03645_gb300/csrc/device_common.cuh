// Device helpers shared by the AMR kernels and the fused step kernel:
// boundary signs and the coarse-to-fine space-time interpolation of a ghost
// (or new) cell (Sec. 3: linear in time between the coarser level's old and
// new states, minmod-limited linear in space), in the canonical order.
#pragma once
#include "internal.h"

namespace adjamr {
namespace {

// Programmatic dependent launch (sm_90 and later): a kernel launched with the
// programmatic-serialization attribute may start before the kernel ahead of it
// in the stream has finished; pdl_wait() returns once that kernel has
// completed and its writes are visible (at once for a normal launch).  Every
// kernel launched that way calls it before its first global memory access, so
// completions stay in stream order.  pdl_launch_dependents() lets the next
// such kernel launch as soon as every CTA of this grid has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return fmin(a, b);
    if (a < 0.0 && b < 0.0) return fmax(a, b);
    return 0.0;
}

__device__ __forceinline__ double sgn(double v, int signs, int comp, int ref)
{
    // comp 0 is never flipped; comps 1, 2 by bits (2*ref + comp - 1)
    if (comp == 0) return v;
    return ((signs >> (2 * ref + comp - 1)) & 1) ? -v : v;
}

// value of field f at coarse reference `ref` (cell index c), at time th = k/r
// of the coarse step (k = 0: the old state alone)
__device__ __forceinline__ double coarse_val(const double *__restrict__ qo, const double *__restrict__ qn_,
                                             long long sc, long long c, int f, int k, double th, int signs, int ref)
{
    double v0 = qo[(long long)f * sc + c];
    double v;
    if (k == 0) {
        v = v0;
    } else {
        double v1 = qn_[(long long)f * sc + c];
        v = (1.0 - th) * v0 + th * v1;
    }
    return sgn(v, signs, f, ref + 1);
}

__device__ __forceinline__ double interp_field(const GhostDesc &g, const double *__restrict__ qo,
                                               const double *__restrict__ qn_, long long sc, int f, int k, double th,
                                               int dim)
{
    double q0 = coarse_val(qo, qn_, sc, g.src, f, k, th, g.signs, 0);
    double qxm = coarse_val(qo, qn_, sc, g.cxm, f, k, th, g.signs, 1);
    double qxp = coarse_val(qo, qn_, sc, g.cxp, f, k, th, g.signs, 2);
    double sx = minmod(qxp - q0, q0 - qxm);
    double v = q0 + sx * g.fx;
    if (dim == 2) {
        double qym = coarse_val(qo, qn_, sc, g.cym, f, k, th, g.signs, 3);
        double qyp = coarse_val(qo, qn_, sc, g.cyp, f, k, th, g.signs, 4);
        double sy = minmod(qyp - q0, q0 - qym);
        v = v + sy * g.fy;
    }
    return v;
}

// load of the level's state; CG: through L2 only, for state written by other
// CTAs of the running launch
template <bool CG>
__device__ __forceinline__ double ldq(const double *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// The coarse stencil values of interp_field (q0 and the minmod slopes sx, sy
// of field f at time fraction th), stored for reuse by every fine cell of
// the coarse cell: p[0..2].
__device__ __forceinline__ void coarse_stencil(const GhostDesc &g, const double *__restrict__ qo,
                                               const double *__restrict__ qn_, long long sc, int f, int k, double th,
                                               int dim, double *p)
{
    double q0 = coarse_val(qo, qn_, sc, g.src, f, k, th, g.signs, 0);
    double qxm = coarse_val(qo, qn_, sc, g.cxm, f, k, th, g.signs, 1);
    double qxp = coarse_val(qo, qn_, sc, g.cxp, f, k, th, g.signs, 2);
    p[0] = q0;
    p[1] = minmod(qxp - q0, q0 - qxm);
    p[2] = 0.0;
    if (dim == 2) {
        double qym = coarse_val(qo, qn_, sc, g.cym, f, k, th, g.signs, 3);
        double qyp = coarse_val(qo, qn_, sc, g.cyp, f, k, th, g.signs, 4);
        p[2] = minmod(qyp - q0, q0 - qym);
    }
}

// interp_field from stored coarse stencil values (same operations, same bits)
__device__ __forceinline__ double pre_field(const GhostDesc &g, const double *__restrict__ pre, long long sc, int f,
                                            int dim)
{
    const double *p = pre + ((long long)f * sc + g.src) * 3;
    double v = p[0] + p[1] * g.fx;
    if (dim == 2) v = v + p[2] * g.fy;
    return v;
}

// value of field f of the ghost cell described by g (same-level copy, or the
// coarse space-time interpolation from the stored stencil values pre_k of
// its substep), with the boundary sign of the result
template <bool CG = false>
__device__ __forceinline__ double ghost_value(const GhostDesc &g, const double *__restrict__ qf, long long sf,
                                              const double *__restrict__ pre_k, long long sc, int f, int dim)
{
    double v;
    if (g.kind == 0) v = ldq<CG>(qf + (long long)f * sf + g.src);
    else v = pre_field(g, pre_k, sc, f, dim);
    return sgn(v, g.signs, f, 0);
}

// the same, interpolating directly from the coarse states
__device__ __forceinline__ double ghost_value_direct(const GhostDesc &g, const double *__restrict__ qf, long long sf,
                                                     const double *__restrict__ qo, const double *__restrict__ qn_,
                                                     long long sc, int f, int k, double th, int dim)
{
    double v;
    if (g.kind == 0) v = qf[(long long)f * sf + g.src];
    else v = interp_field(g, qo, qn_, sc, f, k, th, dim);
    return sgn(v, g.signs, f, 0);
}

// index, within its patch, of the ghost cell at storage (si, sj): bottom rows,
// then the 4 side cells of each interior row, then top rows
__device__ __forceinline__ long long ghost_local_index(const PatchDesc &P, int si, int sj, int gy)
{
    if (sj < gy) return (long long)sj * P.sx + si;
    if (sj < gy + P.ny) return (long long)gy * P.sx + (long long)(sj - gy) * 4 + (si < 2 ? si : si - P.nx);
    return (long long)gy * P.sx + (long long)P.ny * 4 + (long long)(sj - gy - P.ny) * P.sx + si;
}

}  // namespace
}  // namespace adjamr
