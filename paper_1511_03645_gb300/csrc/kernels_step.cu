// High-resolution wave-propagation step (Sec. 3; LeVeque 1997 unsplit
// method with transverse Riemann problems), FP64, sm_103a.
//
// One CTA advances one tile of one patch from a tile work-list.  The tile's
// state and medium coefficients plus a 2-cell halo are staged in shared
// memory; every edge quantity of the tile (waves, fluctuations, limited
// corrections, transverse terms) lives in shared memory; the new state is
// written once.  The same kernel serves a one-launch-per-level work-list, a
// persistent grid looping over the work-list, and one launch per patch.
//
// Operation order follows the canonical operations of the design record
// exactly (compiled with --fmad=false, so only the explicit fma() calls of
// that order fuse): the CPU oracle evaluates the same IEEE operations in the
// same order, so results agree bit for bit.
//
// Systems: 0 acoustics (wave form, eigenvectors of A: (-Z_l,1) at -c_l,
// (Z_r,1) at +c_r), 1 adjoint acoustics (f-wave, eigenvectors of -A^T:
// (1,Z_l) at -c_l, (1,-Z_r) at +c_r), 2 linearised shallow water (f-wave,
// df = (d mu, g h_e d eta), eigenvectors (1,-+c_e)), 3 adjoint shallow water
// (f-wave, eigenvectors (c_e,1) at -c_e, (-c_e,1) at +c_e).
#include <cuda_runtime.h>

#include "internal.h"
#include "device_common.cuh"

namespace adjamr {
namespace {

constexpr int kThreads = 256;

// Edge coefficients gathered from the per-cell aux arrays.
struct Edge {
    double s1, s2;       // speeds of the left- and right-going waves
    double Zl, Zr, izs;  // acoustics
    double ce, ice, ghe; // shallow water
};

// aux index layout per system (see internal.h)
template <int EQN, int DIR>
__device__ __forceinline__ void load_edge(const double *__restrict__ sa, int stride, int l, int r, Edge &e)
{
    if constexpr (EQN == 0 || EQN == 1) {
        e.s1 = -sa[l];               // c at left cell
        e.s2 = sa[r];                // c at right cell
        e.Zl = sa[stride + l];
        e.Zr = sa[stride + r];
        e.izs = sa[(2 + DIR) * stride + r];
    } else if constexpr (EQN == 2) {
        e.ce = sa[(3 * DIR) * stride + r];
        e.ice = sa[(3 * DIR + 1) * stride + r];
        e.ghe = sa[(3 * DIR + 2) * stride + r];
        e.s1 = -e.ce;
        e.s2 = e.ce;
    } else {
        e.ce = sa[(2 * DIR) * stride + r];
        e.ice = sa[(2 * DIR + 1) * stride + r];
        e.s1 = -e.ce;
        e.s2 = e.ce;
    }
}

// eigen-decomposition of d = (d0, dn) at the edge (canonical order)
template <int EQN>
__device__ __forceinline__ void decompose(const Edge &e, double d0, double dn, double *w1, double *w2)
{
    if constexpr (EQN == 0) {
        double a1 = fma(e.Zr, dn, -d0) * e.izs;
        double a2 = fma(e.Zl, dn, d0) * e.izs;
        w1[0] = -(e.Zl * a1);
        w1[1] = a1;
        w2[0] = e.Zr * a2;
        w2[1] = a2;
    } else if constexpr (EQN == 1) {
        double b1 = fma(e.Zr, d0, dn) * e.izs;
        double b2 = fma(e.Zl, d0, -dn) * e.izs;
        w1[0] = b1;
        w1[1] = e.Zl * b1;
        w2[0] = b2;
        w2[1] = -(e.Zr * b2);
    } else if constexpr (EQN == 2) {
        double b1 = fma(-dn, e.ice, d0) * 0.5;
        double b2 = fma(dn, e.ice, d0) * 0.5;
        w1[0] = b1;
        w1[1] = -(e.ce * b1);
        w2[0] = b2;
        w2[1] = e.ce * b2;
    } else {
        double b1 = fma(d0, e.ice, dn) * 0.5;
        double b2 = fma(-d0, e.ice, dn) * 0.5;
        w1[0] = e.ce * b1;
        w1[1] = b1;
        w2[0] = -(e.ce * b2);
        w2[1] = b2;
    }
}

// jump (wave form) or flux difference (f-wave forms) across the edge;
// NRM = index of the normal component (1 = u, 2 = v); DIR selects aux.
template <int EQN>
__device__ __forceinline__ void edge_jump(const Edge &e, const double *__restrict__ sa, int stride, int l, int r,
                                          double ql0, double qln, double qr0, double qrn, double &d0, double &dn)
{
    if constexpr (EQN == 0) {
        d0 = qr0 - ql0;
        dn = qrn - qln;
    } else if constexpr (EQN == 2) {
        d0 = qrn - qln;
        dn = e.ghe * (qr0 - ql0);
    } else if constexpr (EQN == 1) {
        double fl0 = -(sa[4 * stride + l] * qln), fln = -(sa[5 * stride + l] * ql0);
        double fr0 = -(sa[4 * stride + r] * qrn), frn = -(sa[5 * stride + r] * qr0);
        d0 = fr0 - fl0;
        dn = frn - fln;
    } else {
        double fl0 = -(sa[4 * stride + l] * qln), fln = -ql0;
        double fr0 = -(sa[4 * stride + r] * qrn), frn = -qr0;
        d0 = fr0 - fl0;
        dn = frn - fln;
    }
}

// Transverse split of a fluctuation (d0, 0) whose normal component is 0:
// left-going part s1*w1 and right-going part s2*w2 of its decomposition.
// Equal to decompose(e, d0, 0.0, ...) except possibly for the sign of a zero
// (terms like Z*0.0 are dropped), which no later operation can turn into a
// different non-zero value.
template <int EQN>
__device__ __forceinline__ void trans_split(const Edge &e, double d0, double *am, double *ap)
{
    if constexpr (EQN == 0) {
        // a1 = (-d0) izs = -a2 exactly (rounding is sign-symmetric), so
        // -(Zl a1) = Zl a2 and s1 a1 = -(s1 a2): one product fewer, same bits
        double a2 = d0 * e.izs;
        am[0] = e.s1 * (e.Zl * a2);
        am[1] = -(e.s1 * a2);
        ap[0] = e.s2 * (e.Zr * a2);
        ap[1] = e.s2 * a2;
    } else if constexpr (EQN == 1) {
        double b1 = (e.Zr * d0) * e.izs;
        double b2 = (e.Zl * d0) * e.izs;
        am[0] = e.s1 * b1;
        am[1] = e.s1 * (e.Zl * b1);
        ap[0] = e.s2 * b2;
        ap[1] = e.s2 * (-(e.Zr * b2));
    } else if constexpr (EQN == 2) {
        double b = d0 * 0.5;
        am[0] = e.s1 * b;
        am[1] = e.s1 * (-(e.ce * b));
        ap[0] = e.s2 * b;
        ap[1] = e.s2 * (e.ce * b);
    } else {
        double t = d0 * e.ice;
        double b1 = t * 0.5;
        double b2 = (-t) * 0.5;
        am[0] = e.s1 * (e.ce * b1);
        am[1] = e.s1 * b1;
        ap[0] = e.s2 * (-(e.ce * b2));
        ap[1] = e.s2 * b2;
    }
}

// MC limiter phi(theta), theta = (W_upwind . W)/(W . W), in the canonical
// form  wn == 0 ? 0 : fmax(0, fmin(fmin(fma(0.5, th, 0.5), 2), 2*th)).
// Exact shortcuts skip the division: dot <= 0 gives theta <= 0 and phi = 0
// (up to the sign of zero); dot >= 4 wn gives a rounded theta >= 4 and
// phi = 2.  The tests and the min run on the integer pipe: a sum of squares
// is never -0, and past the early exits every value compared (dot, 4 wn,
// fma(0.5, th, 0.5), 2, 2 th) is a non-negative double, which orders like its
// bit pattern (products by 2 and 4 are exponent increments); the outer
// fmax(0, .) is the identity on those values.
// bits of x * 2^k for a positive double x: an exponent increment when x is
// normal and stays finite (exact), else the multiplication
template <int K>
__device__ __forceinline__ long long scaled_bits(double x)
{
    const long long b = __double_as_longlong(x);
    const long long e = b >> 52;
    if (e >= 1 && e <= 2046 - K) return b + ((long long)K << 52);
    return __double_as_longlong(x * (double)(1 << K));
}

// 0.5 * x: an exponent decrement when x and x/2 are normal (exact), else the
// multiplication
__device__ __forceinline__ double half(double x)
{
    const long long b = __double_as_longlong(x);
    const long long e = (b >> 52) & 0x7ff;
    if (e >= 2 && e <= 2046) return __longlong_as_double(b - (1ll << 52));
    return 0.5 * x;
}

__device__ __forceinline__ double mc_phi(double w0, double w1, double u0, double u1)
{
    const double wn = fma(w0, w0, w1 * w1);
    if (__double_as_longlong(wn) == 0) return 0.0;
    const double dot = fma(u0, w0, u1 * w1);
    const long long idot = __double_as_longlong(dot);
    if (idot <= 0) return 0.0;
    if (idot >= scaled_bits<2>(wn)) return 2.0;
    const double th = dot / wn;
    const long long ia = __double_as_longlong(fma(0.5, th, 0.5));
    const long long ib = scaled_bits<1>(th);
    const long long i2 = 0x4000000000000000ll;  // 2.0
    long long m = ia < i2 ? ia : i2;
    m = m < ib ? m : ib;
    return __longlong_as_double(m);
}

// s > 0.0 and s < 0.0 decided on the integer pipe (identical to the FP64
// comparisons for every non-NaN double, signed zeros included)
__device__ __forceinline__ bool positive(double s) { return __double_as_longlong(s) > 0; }
__device__ __forceinline__ bool negative(double s)
{
    long long b = __double_as_longlong(s);
    return b < 0 && b != (long long)0x8000000000000000ull;
}

// correction coefficient of a wave of speed s: |s| fma(-dtd, |s|, 1) for the
// wave form, sign(s) fma(-dtd, |s|, 1) for the f-wave forms
template <int EQN>
__device__ __forceinline__ double corr_coef(double s, double dtd)
{
    double a = fabs(s);
    if constexpr (EQN == 0) {
        return a * fma(-dtd, a, 1.0);
    } else {
        double t = fma(-dtd, a, 1.0);
        return negative(s) ? -t : t;
    }
}

// fmax(|a|, |b|) by comparing bit patterns on the integer pipe (non-NaN)
__device__ __forceinline__ double maxabs(double a, double b)
{
    long long x = __double_as_longlong(a) & 0x7fffffffffffffffll;
    long long y = __double_as_longlong(b) & 0x7fffffffffffffffll;
    return __longlong_as_double(x > y ? x : y);
}

// max of non-negative doubles through their bit patterns (integer pipe)
__device__ __forceinline__ long long bmax(long long a, double v)
{
    long long b = __double_as_longlong(v);
    return b > a ? b : a;
}

__device__ __forceinline__ void cfl_reduce(long long c, unsigned long long *cfl_bits)
{
    for (int o = 16; o > 0; o >>= 1) {
        long long x = __shfl_xor_sync(0xffffffffu, c, o);
        c = x > c ? x : c;
    }
    if ((threadIdx.x & 31) == 0 && c > 0) atomicMax(cfl_bits, (unsigned long long)c);
}

// Asynchronous 8-byte global -> shared copies for the tile staging: all of a
// thread's copies are in flight at once instead of one load-store round trip
// each (cp.async.ca: through L1; used only for data no other CTA of the launch
// writes).
__device__ __forceinline__ void cp_async8(double *smem, const double *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}

// fetch the line holding p into L1 (no register result)
__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// next tile of this CTA (see TileSched); w_static = the strided choice
__device__ __forceinline__ int fetch_tile(const TileSched &sc, int *slot, int w_static)
{
    if (!sc.ctr) return w_static;
    if (threadIdx.x == 0) *slot = (int)(atomicAdd(sc.ctr, 1ull) - sc.base);
    __syncthreads();
    return *slot;
}

// ---------------------------------------------------------------- 2D
template <int EQN, int TX, int TY>
struct Smem2D {
    static constexpr int NA = naux_of(EQN);
    static constexpr int PX = TX + 4, PY = TY + 4;          // staged tile + halo
    static constexpr int XEX = TX + 3, XEY = TY + 2;        // x-edges [-1, tx+1] x rows [-1, ty]
    static constexpr int YEX = TX + 2, YEY = TY + 3;        // y-edges: cols [-1, tx] x [-1, ty+1]
    static constexpr int XNX = TX + 1, XNY = TY + 2;        // Fn: x-edges [0, tx] x rows [-1, ty]
    static constexpr int YNX = TX + 2, YNY = TY + 1;        // Gn: cols [-1, tx] x y-edges [0, ty]
    static constexpr int nQ = 3 * PX * PY, nA = NA * PX * PY;
    static constexpr int nXW = 4 * XEX * XEY, nXF = 4 * XEX * XEY;
    static constexpr int nYW = 4 * YEX * YEY, nYF = 4 * YEX * YEY;
    static constexpr int nXN = 2 * XNX * XNY, nYN = 2 * YNX * YNY;
    // the second-order fluxes Fn, Gn live from the limiter to the transverse
    // phase, when the staged state is not read: they take its place where
    // they fit (the update then reads the tile's cells from global memory)
    static constexpr bool kAlias = nXN + nYN <= nQ;
    static constexpr int total = nQ + nA + nXW + nXF + nYW + nYF + (kAlias ? 0 : nXN + nYN);
    static constexpr size_t bytes = sizeof(double) * (size_t)total;
};

// One tile of one step: stage, Riemann problems, limiter, transverse
// corrections, update of the tile's cells in qn.  CG: the state is read
// through L2 only (it was written by other CTAs of the same launch).
template <int EQN, int TX, int TY, bool CG>
__device__ __forceinline__ void step2d_tile(const double *__restrict__ q, double *__restrict__ qn,
                                            const double *__restrict__ aux, long long stride, const PatchDesc P,
                                            const WorkItem wi, const GhostArgs &ga, double *sm, long long &cfl)
{
    using S = Smem2D<EQN, TX, TY>;
    double *sQ = sm;
    double *sA = sQ + S::nQ;
    double *XW = sA + S::nA;   // waves w1_0, w1_n, w2_0, w2_n at x-edges; later SX + FF
    double *XF = XW + S::nXW;  // fluctuations am_0, am_n, ap_0, ap_n at x-edges
    double *YW = XF + S::nXF;  // same at y-edges; later SY + GG
    double *YF = YW + S::nYW;
    double *XN = S::kAlias ? sQ : YF + S::nYF;  // Fn (2 comps)
    double *YN = XN + S::nXN;                   // Gn (2 comps)
    constexpr int PX = S::PX, PY = S::PY, PS = PX * PY;
    constexpr int XEX = S::XEX, XEY = S::XEY, XES = XEX * XEY;
    constexpr int YEX = S::YEX, YEY = S::YEY, YES = YEX * YEY;
    constexpr int XNX = S::XNX, XNS = XNX * S::XNY;
    constexpr int YNX = S::YNX, YNS = YNX * S::YNY;
    // reuse of the wave arrays after the limiter phase
    double *SX = XW;                       // [2][TY+2][TX]   cells [0,tx) x rows [-1,ty]
    double *FF = XW + 2 * (TY + 2) * TX;   // [2][TY][TX+1]   x-edges [0,tx] x rows [0,ty)
    double *SY = YW;                       // [2][TY][TX+2]   cols [-1,tx] x rows [0,ty)
    double *GG = YW + 2 * TY * (TX + 2);   // [2][TY+1][TX]   cols [0,tx) x y-edges [0,ty]
    constexpr int SXS = (TY + 2) * TX, FFS = TY * (TX + 1), SYS = TY * (TX + 2), GGS = (TY + 1) * TX;

    const int tid = threadIdx.x;
    {
        const int x0 = wi.x0, y0 = wi.y0;
        const int tx = wi.tx, ty = wi.ty;
        const int rx = tx + 4, ry = ty + 4;
        const double dtdx = P.dtdx, dtdy = P.dtdy, hx = P.hx, hy = P.hy;
        // ---- stage state and coefficients (tile + 2-cell halo) ----
        // With ga.gd set, the ghost-ring cells of the state are not read from
        // q but computed from their ghost descriptors (same-level copy or
        // coarse space-time interpolation, Sec. 3) in a second pass over the
        // staged region; without it the ring of q was filled beforehand.
        {
            const long long gb = P.base + (long long)y0 * P.sx + x0;
            const int nrow = rx;
            // the staged storage columns [x0, x0+tx+4) reach the ghost ring when x0 < 2
            // or x0 + tx + 3 >= nx + 2 (rows alike)
            const bool ring = ga.gd && (x0 < 2 || y0 < 2 || x0 + tx + 1 >= P.nx || y0 + ty + 1 >= P.ny);
            for (int k = tid; k < (3 + S::NA) * ry * nrow; k += kThreads) {
                int f = k / (ry * nrow), rem = k - f * ry * nrow;
                int r = rem / nrow, c = rem - r * nrow;
                long long g = gb + (long long)r * P.sx + c;
                if (f < 3) {
                    const int si = x0 + c, sj = y0 + r;
                    if (!(ring && (si < 2 || si >= P.nx + 2 || sj < 2 || sj >= P.ny + 2))) {
                        // the state of a substep launch was written by other CTAs
                        // of the launch: read it through L2 only
                        if constexpr (CG) sQ[f * PS + r * PX + c] = ldq<CG>(q + (long long)f * stride + g);
                        else cp_async8(&sQ[f * PS + r * PX + c], q + (long long)f * stride + g);
                    }
                } else {
                    cp_async8(&sA[(f - 3) * PS + r * PX + c], aux + (long long)(f - 3) * stride + g);
                }
            }
            cp_async_wait_all();
            if (ring) {
                for (int k = tid; k < ry * nrow; k += kThreads) {
                    int r = k / nrow, c = k - r * nrow;
                    const int si = x0 + c, sj = y0 + r;
                    if (!(si < 2 || si >= P.nx + 2 || sj < 2 || sj >= P.ny + 2)) continue;
                    const GhostDesc gdsc = ga.gd[P.gbase + ghost_local_index(P, si, sj, 2)];
                    double v[3];
#pragma unroll
                    for (int f = 0; f < 3; f++)
                        v[f] = ghost_value<CG>(gdsc, q, stride, ga.pre + ga.k * ga.pstride, ga.sc, f, 2);
#pragma unroll
                    for (int f = 0; f < 3; f++) sQ[f * PS + r * PX + c] = v[f];
                }
            }
        }
        __syncthreads();
        // ---- normal Riemann problems at x-edges and y-edges ----
        for (int k = tid; k < (tx + 3) * (ty + 2) + (tx + 2) * (ty + 3); k += kThreads) {
            if (k < (tx + 3) * (ty + 2)) {
                int er = k / (tx + 3), ec = k - er * (tx + 3);     // row ry = er-1, edge ex = ec-1
                int l = (er + 1) * PX + ec, r = l + 1;             // cells (ex-1, ry) and (ex, ry) staged
                Edge e;
                load_edge<EQN, 0>(sA, PS, l, r, e);
                double d0, dn, w1[2], w2[2];
                edge_jump<EQN>(e, sA, PS, l, r, sQ[l], sQ[PS + l], sQ[r], sQ[PS + r], d0, dn);
                decompose<EQN>(e, d0, dn, w1, w2);
                int o = er * XEX + ec;
                XW[o] = w1[0]; XW[XES + o] = w1[1]; XW[2 * XES + o] = w2[0]; XW[3 * XES + o] = w2[1];
                if constexpr (EQN == 0) {
                    XF[o] = e.s1 * w1[0]; XF[XES + o] = e.s1 * w1[1];
                    XF[2 * XES + o] = e.s2 * w2[0]; XF[3 * XES + o] = e.s2 * w2[1];
                } else {
                    XF[o] = w1[0]; XF[XES + o] = w1[1]; XF[2 * XES + o] = w2[0]; XF[3 * XES + o] = w2[1];
                }
            } else {
                int kk = k - (tx + 3) * (ty + 2);
                int er = kk / (tx + 2), ec = kk - er * (tx + 2);  // y-edge ey = er-1, column cx = ec-1
                int l = er * PX + ec + 1, r = l + PX;              // cells (cx, ey-1) and (cx, ey)
                Edge e;
                load_edge<EQN, 1>(sA, PS, l, r, e);
                double d0, dn, w1[2], w2[2];
                edge_jump<EQN>(e, sA, PS, l, r, sQ[l], sQ[2 * PS + l], sQ[r], sQ[2 * PS + r], d0, dn);
                decompose<EQN>(e, d0, dn, w1, w2);
                int o = er * YEX + ec;
                YW[o] = w1[0]; YW[YES + o] = w1[1]; YW[2 * YES + o] = w2[0]; YW[3 * YES + o] = w2[1];
                if constexpr (EQN == 0) {
                    YF[o] = e.s1 * w1[0]; YF[YES + o] = e.s1 * w1[1];
                    YF[2 * YES + o] = e.s2 * w2[0]; YF[3 * YES + o] = e.s2 * w2[1];
                } else {
                    YF[o] = w1[0]; YF[YES + o] = w1[1]; YF[2 * YES + o] = w2[0]; YF[3 * YES + o] = w2[1];
                }
            }
        }
        __syncthreads();
        // ---- MC-limited second-order corrections Fn (x) and Gn (y) ----
        for (int k = tid; k < (tx + 1) * (ty + 2) + (tx + 2) * (ty + 1); k += kThreads) {
            if (k < (tx + 1) * (ty + 2)) {
                int er = k / (tx + 1), ec = k - er * (tx + 1);      // row ry = er-1, edge ex = ec
                int o = er * XEX + ec + 1;                          // edge ex in XW
                int l = (er + 1) * PX + ec + 1, r = l + 1;
                Edge e;
                load_edge<EQN, 0>(sA, PS, l, r, e);
                int u1 = positive(e.s1) ? o - 1 : o + 1;
                int u2 = positive(e.s2) ? o - 1 : o + 1;
                double w10 = XW[o], w1n = XW[XES + o], w20 = XW[2 * XES + o], w2n = XW[3 * XES + o];
                double p1 = mc_phi(w10, w1n, XW[u1], XW[XES + u1]);
                double p2 = mc_phi(w20, w2n, XW[2 * XES + u2], XW[3 * XES + u2]);
                double cf1 = corr_coef<EQN>(e.s1, dtdx), cf2 = corr_coef<EQN>(e.s2, dtdx);
                int on = er * XNX + ec;
                XN[on] = half(cf1 * (p1 * w10) + cf2 * (p2 * w20));
                XN[XNS + on] = half(cf1 * (p1 * w1n) + cf2 * (p2 * w2n));
            } else {
                int kk = k - (tx + 1) * (ty + 2);
                int er = kk / (tx + 2), ec = kk - er * (tx + 2);   // y-edge ey = er, column cx = ec-1
                int o = (er + 1) * YEX + ec;
                int l = (er + 1) * PX + ec + 1, r = l + PX;
                Edge e;
                load_edge<EQN, 1>(sA, PS, l, r, e);
                int u1 = positive(e.s1) ? o - YEX : o + YEX;
                int u2 = positive(e.s2) ? o - YEX : o + YEX;
                double w10 = YW[o], w1n = YW[YES + o], w20 = YW[2 * YES + o], w2n = YW[3 * YES + o];
                double p1 = mc_phi(w10, w1n, YW[u1], YW[YES + u1]);
                double p2 = mc_phi(w20, w2n, YW[2 * YES + u2], YW[3 * YES + u2]);
                double cf1 = corr_coef<EQN>(e.s1, dtdy), cf2 = corr_coef<EQN>(e.s2, dtdy);
                int on = er * YNX + ec;
                YN[on] = half(cf1 * (p1 * w10) + cf2 * (p2 * w20));
                YN[YNS + on] = half(cf1 * (p1 * w1n) + cf2 * (p2 * w2n));
            }
        }
        __syncthreads();
        // ---- fluctuations entering each cell, corrections included ----
        for (int k = tid; k < tx * (ty + 2) + (tx + 2) * ty; k += kThreads) {
            if (k < tx * (ty + 2)) {
                int er = k / tx, c = k - er * tx;                  // cell (c, ry = er-1)
                int oL = er * XEX + c + 1, oR = oL + 1;            // x-edges c and c+1
                int nL = er * XNX + c, nR = nL + 1;
                // component 0 only: the transverse split of this fluctuation
                // takes (Sx_0, 0) (the y-direction sees no x-velocity jump)
                const double apT = XF[2 * XES + oL] - XN[nL];
                const double amT = XF[oR] + XN[nR];
                SX[er * TX + c] = apT + amT;
            } else {
                int kk0 = k - tx * (ty + 2);
                int r = kk0 / (tx + 2), ec = kk0 - r * (tx + 2);  // cell (cx = ec-1, r)
                int oB = (r + 1) * YEX + ec, oT = oB + YEX;        // y-edges r and r+1
                int nB = r * YNX + ec, nT = nB + YNX;
                const double bpT = YF[2 * YES + oB] - YN[nB];
                const double bmT = YF[oT] + YN[nT];
                SY[r * (TX + 2) + ec] = bpT + bmT;
            }
        }
        __syncthreads();
        // ---- transverse corrections: full edge fluxes F and G, and CFL ----
        // (the CFL number max_e (dtd |s|_e) is dtd * max_e |s|_e exactly: a
        // product by a positive constant is monotone, so the maxima of |s| are
        // taken on the integer pipe and multiplied once per direction)
        long long smx = 0, smy = 0;
        for (int k = tid; k < (tx + 1) * ty + tx * (ty + 1); k += kThreads) {
            if (k < (tx + 1) * ty) {
                int r = k / (tx + 1), ec = k - r * (tx + 1);       // x-edge ex = ec, row r
                int l = (r + 2) * PX + ec + 1, rr = l + 1;
                Edge e;
                load_edge<EQN, 0>(sA, PS, l, rr, e);
                double dR = SY[r * (TX + 2) + ec + 1];            // Sy of the cell right of the edge
                double dL = SY[r * (TX + 2) + ec];                // Sy of the cell left of the edge
                double am[2], ap[2], bm[2], bp[2];
                trans_split<EQN>(e, dR, am, ap);
                trans_split<EQN>(e, dL, bm, bp);
                int on = (r + 1) * XNX + ec;
                for (int kk = 0; kk < 2; kk++)
                    FF[kk * FFS + r * (TX + 1) + ec] = fma(-hy, am[kk] + bp[kk], XN[kk * XNS + on]);
                smx = bmax(smx, maxabs(e.s1, e.s2));
            } else {
                int kk0 = k - (tx + 1) * ty;
                int er = kk0 / tx, c = kk0 - er * tx;              // y-edge ey = er, column c
                int l = (er + 1) * PX + c + 2, rr = l + PX;
                Edge e;
                load_edge<EQN, 1>(sA, PS, l, rr, e);
                double dU = SX[(er + 1) * TX + c];                 // Sx of the cell above the edge
                double dD = SX[er * TX + c];                       // Sx of the cell below
                double am[2], ap[2], bm[2], bp[2];
                trans_split<EQN>(e, dU, am, ap);
                trans_split<EQN>(e, dD, bm, bp);
                int on = er * YNX + c + 1;
                for (int kk = 0; kk < 2; kk++)
                    GG[kk * GGS + er * TX + c] = fma(-hx, am[kk] + bp[kk], YN[kk * YNS + on]);
                smy = bmax(smy, maxabs(e.s1, e.s2));
            }
        }
        if (smx > 0) cfl = bmax(cfl, dtdx * __longlong_as_double(smx));
        if (smy > 0) cfl = bmax(cfl, dtdy * __longlong_as_double(smy));
        __syncthreads();
        // ---- cell update q - (X + Y) ----
        for (int k = tid; k < tx * ty; k += kThreads) {
            int r = k / tx, c = k - r * tx;
            int oL = (r + 1) * XEX + c + 1, oR = oL + 1;
            int oB = (r + 1) * YEX + c + 1, oT = oB + YEX;
            int fL = r * (TX + 1) + c, fR = fL + 1;
            int gB = r * TX + c, gT = gB + TX;
            double A0 = (XF[2 * XES + oL] + XF[oR]) + (FF[fR] - FF[fL]);
            double A1 = (XF[3 * XES + oL] + XF[XES + oR]) + (FF[FFS + fR] - FF[FFS + fL]);
            double B0 = (YF[2 * YES + oB] + YF[oT]) + (GG[gT] - GG[gB]);
            double B1 = (YF[3 * YES + oB] + YF[YES + oT]) + (GG[GGS + gT] - GG[GGS + gB]);
            int s = (r + 2) * PX + c + 2;
            long long g = P.base + (long long)(y0 + r + 2) * P.sx + (x0 + c + 2);
            const double p0 = S::kAlias ? ldq<CG>(q + g) : sQ[s];
            const double u0 = S::kAlias ? ldq<CG>(q + stride + g) : sQ[PS + s];
            const double v0 = S::kAlias ? ldq<CG>(q + 2 * stride + g) : sQ[2 * PS + s];
            qn[g] = p0 - (dtdx * A0 + dtdy * B0);
            qn[stride + g] = fma(-dtdx, A1, u0);        // u sees the x-edges only
            qn[2 * stride + g] = fma(-dtdy, B1, v0);    // v sees the y-edges only
        }
        // ---- fix-up records (coarse-fine sides of the listed cells) ----
        // A loop of its own after the update: the edge arrays are intact until
        // the barrier, and the update keeps its registers.
        if (ga.rx.rmap) {
            for (int k = tid; k < tx * ty; k += kThreads) {
                const int r = k / tx, c = k - r * tx;
                const long long g = P.base + (long long)(y0 + r + 2) * P.sx + (x0 + c + 2);
                const int e = ga.rx.rmap[g];
                if (e < 0) continue;
                const int oL = (r + 1) * XEX + c + 1, oR = oL + 1;
                const int oB = (r + 1) * YEX + c + 1, oT = oB + YEX;
                const int fL = r * (TX + 1) + c, fR = fL + 1;
                const int gB = r * TX + c, gT = gB + TX;
                const RefluxCell rc = ga.rx.cells[e];
                // what each side puts into the cell: the fluctuation entering
                // through it with the full (transverse-corrected) flux of that edge
#pragma unroll
                for (int sd = 0; sd < 4; sd++) {
                    if (rc.c[sd] < 0 && rc.f[sd] < 0) continue;
                    double a, b;
                    if (sd == 0) {
                        a = XF[2 * XES + oL] - FF[fL];
                        b = XF[3 * XES + oL] - FF[FFS + fL];
                    } else if (sd == 1) {
                        a = XF[oR] + FF[fR];
                        b = XF[XES + oR] + FF[FFS + fR];
                    } else if (sd == 2) {
                        a = YF[2 * YES + oB] - GG[gB];
                        b = YF[3 * YES + oB] - GG[GGS + gB];
                    } else {
                        a = YF[oT] + GG[gT];
                        b = YF[YES + oT] + GG[GGS + gT];
                    }
                    if (rc.c[sd] >= 0) {
                        ga.rx.lc[2 * (long long)rc.c[sd]] = a;
                        ga.rx.lc[2 * (long long)rc.c[sd] + 1] = b;
                    }
                    if (rc.f[sd] >= 0) {
                        // the cell's state at the start of the step (not yet
                        // overwritten: q and qn are different buffers)
                        const int s = (r + 2) * PX + c + 2;
                        double *o = ga.rx.lf + ((long long)ga.rx.sub * ga.rx.nfrec + rc.f[sd]) * 4;
                        o[0] = a;
                        o[1] = b;
                        o[2] = S::kAlias ? ldq<CG>(q + g) : sQ[s];
                        o[3] = sd < 2 ? (S::kAlias ? ldq<CG>(q + stride + g) : sQ[PS + s])
                                      : (S::kAlias ? ldq<CG>(q + 2 * stride + g) : sQ[2 * PS + s]);
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <int EQN, int TX, int TY>
__global__ void __launch_bounds__(kThreads) k_step2d(const double *__restrict__ q, double *__restrict__ qn,
                                                     const double *__restrict__ aux, long long stride,
                                                     const PatchDesc *__restrict__ patches,
                                                     const WorkItem *__restrict__ work, int nwork,
                                                     unsigned long long *cfl_bits, GhostArgs ga, TileSched sc)
{
    extern __shared__ double sm[];
    long long cfl = 0;
    __shared__ int s_next;
    // One tile per CTA (the work-list launch): the tile's work-list entry,
    // fixed since the level's rebuild, is read before the wait for the kernel
    // ahead and its patch descriptor fetched towards L1 meanwhile; the state
    // that kernel writes is read after the wait.
    const bool single = !sc.ctr && (long long)gridDim.x >= nwork;
    WorkItem wi{};
    if (single && (int)blockIdx.x < nwork) {
        wi = work[blockIdx.x];
        prefetch_l1(patches + wi.patch);
    }
    pdl_wait();
    pdl_launch_dependents();
    for (int w = fetch_tile(sc, &s_next, blockIdx.x); w < nwork; w = fetch_tile(sc, &s_next, w + gridDim.x)) {
        if (!single) wi = work[w];
        step2d_tile<EQN, TX, TY, false>(q, qn, aux, stride, patches[wi.patch], wi, ga, sm, cfl);
        if (single) break;
    }
    cfl_reduce(cfl, cfl_bits);
}

// ---------------------------------------------------------------- substeps
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Warp 0 waits until every tile on w's dependency row (all nwork tiles when
// the row overflowed) has completed `target` substeps.  Each wait is bounded
// (time and polls); it gives up early when another CTA has already reported
// a failure.  Uniform over the CTA.
__device__ __forceinline__ bool wait_deps(const SubstepArgs &sa, int w, int nwork, unsigned long long target,
                                          int *s_ok)
{
    if (threadIdx.x < 32) {
        bool ok = true;
        const int n = sa.dep_cnt[w];
        const bool all = n > kDepRow;
        const int cnt = all ? nwork : n;
        unsigned long long t0 = 0;
        unsigned int spins = 0;
        for (int j = (int)threadIdx.x; ok && j < cnt; j += 32) {
            const int u = all ? j : sa.dep_idx[(long long)w * kDepRow + j];
            const unsigned long long *f = sa.done + u;
            while (ld_acquire(f) < target) {
                if (spins == 0) t0 = global_ns();
                if ((++spins & 255u) == 0 &&
                    (global_ns() - t0 > kSubstepWaitNs || spins > kSubstepWaitSpins ||
                     (*(volatile const int *)sa.err & kSubstepErrBit) != 0)) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) {
            if (!ok) atomicOr(sa.err, kSubstepErrBit);
            *s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ int claim_item(const TileSched &sc)
{
    return (int)(atomicAdd(sc.ctr, 1ull) - sc.base);
}

// nsub consecutive steps of one level in one launch (the substeps of the
// finest level within a coarser step, Sec. 3 time stepping with
// subcycling).  Work item i is tile w = i mod nwork of substep s = i / nwork;
// CTAs take items in increasing order from the atomic counter, and item
// (s, w) first waits until the tiles whose cells its staged region reads
// (2-cell halo and ghost-ring sources) have completed substep s - 1.  Every
// such tile has a smaller item index, so the smallest unfinished item can
// always proceed.  Substep s reads buffer (s & 1 ? qb : qa) and writes the
// other; its ghost ring takes the stored coarse stencil values of substep s.
template <int EQN, int TX, int TY>
__global__ void __launch_bounds__(kThreads) k_step2d_sub(double *qa, double *qb, const double *__restrict__ aux,
                                                         long long stride, const PatchDesc *__restrict__ patches,
                                                         const WorkItem *__restrict__ work, int nwork,
                                                         unsigned long long *cfl_bits, GhostArgs ga, TileSched sc,
                                                         SubstepArgs sa)
{
    pdl_wait();
    pdl_launch_dependents();
    extern __shared__ double sm[];
    long long cfl = 0;
    // s_next[it & 1]: the item taken during iteration it - 1 (a thread of
    // warp 1 takes the next item while the CTA works on the current one, off
    // the path of warp 0, which runs the dependency waits)
    constexpr int kClaimer = 32;
    __shared__ int s_next[2], s_ok;
    const int nitems = sa.nsub * nwork;
    if (threadIdx.x == kClaimer) s_next[0] = claim_item(sc);
    __syncthreads();
    int i = s_next[0];
    // After a failed wait the CTA keeps taking items without working on them,
    // so that the counter advances by exactly nitems + gridDim.x.
    bool failed = false;
    for (int it = 0; i < nitems; it++) {
        const int nb = (it + 1) & 1;
        if (threadIdx.x == kClaimer) s_next[nb] = claim_item(sc);
        if (failed || i < 0) {
            if (!failed && threadIdx.x == 0) atomicOr(sa.err, kSubstepErrBit);
            failed = true;
        } else {
            const int s = i / nwork, w = i - s * nwork;
            if (s > 0 && !wait_deps(sa, w, nwork, sa.base + (unsigned long long)s, &s_ok)) {
                failed = true;
            } else {
                GhostArgs g = ga;
                g.k = ga.k + s;
                g.rx.sub = ga.rx.sub + s;
                const WorkItem wi = work[w];
                step2d_tile<EQN, TX, TY, true>((s & 1) ? qb : qa, (s & 1) ? qa : qb, aux, stride,
                                               patches[wi.patch], wi, g, sm, cfl);
                // the tile's stores precede the barrier that ends step2d_tile
                if (threadIdx.x == 0) {
                    __threadfence();
                    st_release(sa.done + w, sa.base + (unsigned long long)s + 1);
                }
            }
        }
        __syncthreads();  // s_next[nb] is written
        i = s_next[nb];
    }
    cfl_reduce(cfl, cfl_bits);
}

// ---------------------------------------------------------------- 1D
template <int EQN, int TX>
struct Smem1D {
    static constexpr int NA = naux_of(EQN);
    static constexpr int PX = TX + 4, XE = TX + 3, XN = TX + 1;
    static constexpr int total = 2 * PX + NA * PX + 8 * XE + 2 * XN;
    static constexpr size_t bytes = sizeof(double) * (size_t)total;
};

// One tile of one 1D step: stage, Riemann problems, limiter, update of the
// tile's cells in qn (and the fix-up records of listed cells).
template <int EQN, int TX>
__device__ __forceinline__ void step1d_tile(const double *__restrict__ q, double *__restrict__ qn,
                                            const double *__restrict__ aux, long long stride, const PatchDesc P,
                                            const WorkItem wi, const GhostArgs &ga, double *sm, long long &cfl)
{
    using S = Smem1D<EQN, TX>;
    constexpr int PX = S::PX, XE = S::XE, XNn = S::XN;
    double *sQ = sm;
    double *sA = sQ + 2 * PX;
    double *XW = sA + S::NA * PX;
    double *XF = XW + 4 * XE;
    double *XN = XF + 4 * XE;
    const int tid = threadIdx.x;
    const int x0 = wi.x0;
    const int tx = wi.tx, rx = tx + 4;
    const double dtdx = P.dtdx;
    const bool ring = ga.gd && (x0 < 2 || x0 + tx + 1 >= P.nx);  // staged [x0, x0+tx+4) meets the ring
    for (int k = tid; k < (2 + S::NA) * rx; k += kThreads) {
        int f = k / rx, c = k - f * rx;
        long long g = P.base + x0 + c;
        if (f < 2) {
            const int si = x0 + c;
            if (!(ring && (si < 2 || si >= P.nx + 2))) sQ[f * PX + c] = q[(long long)f * stride + g];
        } else {
            sA[(f - 2) * PX + c] = aux[(long long)(f - 2) * stride + g];
        }
    }
    for (int c = tid; ring && c < rx; c += kThreads) {
        const int si = x0 + c;
        if (si < 2 || si >= P.nx + 2) {
            const GhostDesc gdsc = ga.gd[P.gbase + ghost_local_index(P, si, 0, 0)];
            double v0 = ghost_value(gdsc, q, stride, ga.pre + ga.k * ga.pstride, ga.sc, 0, 1);
            double v1 = ghost_value(gdsc, q, stride, ga.pre + ga.k * ga.pstride, ga.sc, 1, 1);
            sQ[c] = v0;
            sQ[PX + c] = v1;
        }
    }
    __syncthreads();
    for (int k = tid; k < tx + 3; k += kThreads) {    // edge ex = k-1 between staged cells k, k+1
        int l = k, r = k + 1;
        Edge e;
        load_edge<EQN, 0>(sA, PX, l, r, e);
        double d0, dn, w1[2], w2[2];
        edge_jump<EQN>(e, sA, PX, l, r, sQ[l], sQ[PX + l], sQ[r], sQ[PX + r], d0, dn);
        decompose<EQN>(e, d0, dn, w1, w2);
        XW[k] = w1[0]; XW[XE + k] = w1[1]; XW[2 * XE + k] = w2[0]; XW[3 * XE + k] = w2[1];
        if constexpr (EQN == 0) {
            XF[k] = e.s1 * w1[0]; XF[XE + k] = e.s1 * w1[1];
            XF[2 * XE + k] = e.s2 * w2[0]; XF[3 * XE + k] = e.s2 * w2[1];
        } else {
            XF[k] = w1[0]; XF[XE + k] = w1[1]; XF[2 * XE + k] = w2[0]; XF[3 * XE + k] = w2[1];
        }
    }
    __syncthreads();
    long long smx = 0;  // max |s| over this thread's edges (see the 2D kernel)
    for (int k = tid; k < tx + 1; k += kThreads) {    // edge ex = k
        int o = k + 1, l = k + 1, r = k + 2;
        Edge e;
        load_edge<EQN, 0>(sA, PX, l, r, e);
        int u1 = positive(e.s1) ? o - 1 : o + 1;
        int u2 = positive(e.s2) ? o - 1 : o + 1;
        double w10 = XW[o], w1n = XW[XE + o], w20 = XW[2 * XE + o], w2n = XW[3 * XE + o];
        double p1 = mc_phi(w10, w1n, XW[u1], XW[XE + u1]);
        double p2 = mc_phi(w20, w2n, XW[2 * XE + u2], XW[3 * XE + u2]);
        double cf1 = corr_coef<EQN>(e.s1, dtdx), cf2 = corr_coef<EQN>(e.s2, dtdx);
        XN[k] = half(cf1 * (p1 * w10) + cf2 * (p2 * w20));
        XN[XNn + k] = half(cf1 * (p1 * w1n) + cf2 * (p2 * w2n));
        smx = bmax(smx, maxabs(e.s1, e.s2));
    }
    if (smx > 0) cfl = bmax(cfl, dtdx * __longlong_as_double(smx));
    __syncthreads();
    for (int c = tid; c < tx; c += kThreads) {
        int oL = c + 1, oR = c + 2;
        double A0 = (XF[2 * XE + oL] + XF[oR]) + (XN[c + 1] - XN[c]);
        double A1 = (XF[3 * XE + oL] + XF[XE + oR]) + (XN[XNn + c + 1] - XN[XNn + c]);
        long long g = P.base + x0 + c + 2;
        qn[g] = sQ[c + 2] - dtdx * A0;
        qn[stride + g] = fma(-dtdx, A1, sQ[PX + c + 2]);
        if (ga.rx.rmap) {
            const int e = ga.rx.rmap[g];
            if (e >= 0) {
                const RefluxCell rc = ga.rx.cells[e];
                for (int sd = 0; sd < 2; sd++) {
                    if (rc.c[sd] < 0 && rc.f[sd] < 0) continue;
                    const double a = sd == 0 ? XF[2 * XE + oL] - XN[c] : XF[oR] + XN[c + 1];
                    const double b = sd == 0 ? XF[3 * XE + oL] - XN[XNn + c] : XF[XE + oR] + XN[XNn + c + 1];
                    if (rc.c[sd] >= 0) {
                        ga.rx.lc[2 * (long long)rc.c[sd]] = a;
                        ga.rx.lc[2 * (long long)rc.c[sd] + 1] = b;
                    }
                    if (rc.f[sd] >= 0) {
                        double *o = ga.rx.lf + ((long long)ga.rx.sub * ga.rx.nfrec + rc.f[sd]) * 4;
                        o[0] = a;
                        o[1] = b;
                        o[2] = sQ[c + 2];
                        o[3] = sQ[PX + c + 2];
                    }
                }
            }
        }
    }
    __syncthreads();
}

template <int EQN, int TX>
__global__ void __launch_bounds__(kThreads) k_step1d(const double *__restrict__ q, double *__restrict__ qn,
                                                     const double *__restrict__ aux, long long stride,
                                                     const PatchDesc *__restrict__ patches,
                                                     const WorkItem *__restrict__ work, int nwork,
                                                     unsigned long long *cfl_bits, GhostArgs ga, TileSched sc)
{
    extern __shared__ double sm[];
    long long cfl = 0;
    __shared__ int s_next;
    // one tile per CTA: its work-list entry is read before the wait (as in k_step2d)
    const bool single = !sc.ctr && (long long)gridDim.x >= nwork;
    WorkItem wi{};
    if (single && (int)blockIdx.x < nwork) {
        wi = work[blockIdx.x];
        prefetch_l1(patches + wi.patch);
    }
    pdl_wait();
    pdl_launch_dependents();
    for (int w = fetch_tile(sc, &s_next, blockIdx.x); w < nwork; w = fetch_tile(sc, &s_next, w + gridDim.x)) {
        if (!single) wi = work[w];
        step1d_tile<EQN, TX>(q, qn, aux, stride, patches[wi.patch], wi, ga, sm, cfl);
        if (single) break;
    }
    cfl_reduce(cfl, cfl_bits);
}

// the dynamic shared-memory limit is raised once per kernel (outside any
// stream capture: the first launch of each kernel happens uncaptured)
template <auto Kern>
cudaError_t ensure_smem_attr(size_t smem)
{
    static cudaError_t state = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return state;
}

template <auto Kern>
cudaError_t launch_kernel(size_t smem, int nwork, int grid, const double *q, double *qn, const double *aux,
                          long long stride, const PatchDesc *patches, const WorkItem *work,
                          unsigned long long *cfl_bits, cudaStream_t s, const GhostArgs &ga, const TileSched &sc)
{
    auto kern = Kern;
    cudaError_t e = ensure_smem_attr<Kern>(smem);
    if (e != cudaSuccess) return e;
    if (nwork <= 0) return cudaSuccess;
    int g = grid > 0 ? grid : nwork;
    return launch_pdl(kern, dim3(g), dim3(kThreads), smem, s, q, qn, aux, stride, patches, work, nwork, cfl_bits, ga,
                      sc);
}

template <int EQN>
cudaError_t dispatch2d(int tx, int ty, int nwork, int grid, const double *q, double *qn, const double *aux,
                       long long stride, const PatchDesc *p, const WorkItem *w, unsigned long long *c,
                       cudaStream_t s, const GhostArgs &ga, const TileSched &sc)
{
#define ADJ_TILE(X, Y)                                                                                    \
    if (tx == X && ty == Y)                                                                               \
        return launch_kernel<k_step2d<EQN, X, Y>>(Smem2D<EQN, X, Y>::bytes, nwork, grid, q, qn, aux, stride, p, w, \
                                                  c, s, ga, sc);
    ADJ_TILE(32, 8)
    ADJ_TILE(16, 8)
    ADJ_TILE(16, 12)
    ADJ_TILE(16, 16)
    ADJ_TILE(32, 16)
    ADJ_TILE(64, 8)
    ADJ_TILE(8, 8)
#undef ADJ_TILE
    return cudaErrorInvalidValue;
}

template <int EQN>
cudaError_t dispatch1d(int tx, int nwork, int grid, const double *q, double *qn, const double *aux, long long stride,
                       const PatchDesc *p, const WorkItem *w, unsigned long long *c, cudaStream_t s,
                       const GhostArgs &ga, const TileSched &sc)
{
    if (tx == 256)
        return launch_kernel<k_step1d<EQN, 256>>(Smem1D<EQN, 256>::bytes, nwork, grid, q, qn, aux, stride, p, w, c, s,
                                                 ga, sc);
    if (tx == 128)
        return launch_kernel<k_step1d<EQN, 128>>(Smem1D<EQN, 128>::bytes, nwork, grid, q, qn, aux, stride, p, w, c, s,
                                                 ga, sc);
    return cudaErrorInvalidValue;
}

template <int EQN>
int occ2d(int tx, int ty)
{
    int n = 0;
#define ADJ_OCC(X, Y)                                                                                   \
    if (tx == X && ty == Y) {                                                                           \
        if (ensure_smem_attr<k_step2d<EQN, X, Y>>(Smem2D<EQN, X, Y>::bytes) == cudaSuccess)            \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2d<EQN, X, Y>, kThreads,            \
                                                          Smem2D<EQN, X, Y>::bytes);                    \
    }
    ADJ_OCC(32, 8)
    ADJ_OCC(16, 8)
    ADJ_OCC(16, 12)
    ADJ_OCC(16, 16)
    ADJ_OCC(32, 16)
    ADJ_OCC(64, 8)
    ADJ_OCC(8, 8)
#undef ADJ_OCC
    return n;
}

// tile of every interior cell of the level (one CTA per tile)
__global__ void k_tile_map(const PatchDesc *__restrict__ patches, const WorkItem *__restrict__ work, int nwork,
                           int *tile_of)
{
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const WorkItem wi = work[w];
    const PatchDesc P = patches[wi.patch];
    for (int k = threadIdx.x; k < (int)wi.tx * wi.ty; k += blockDim.x) {
        const int j = k / wi.tx, i = k - j * wi.tx;
        tile_of[P.base + (long long)(wi.y0 + j + 2) * P.sx + (wi.x0 + i + 2)] = w;
    }
}

// Dependency row of each tile (one CTA per tile): the distinct tiles owning
// a cell of its cells + 2-cell halo, collected in a shared open-addressing
// set with bounded probing.  Halo cells beyond a periodic boundary are taken
// at their images; beyond the other boundaries the ghost values come from
// cells inside the halo, so those cells are skipped.
constexpr int kDepSet = 128;
__global__ void k_tile_deps(const PatchDesc *__restrict__ patches, const WorkItem *__restrict__ work, int nwork,
                            const int *__restrict__ owner, int N, int M, int4 bc, const int *__restrict__ tile_of,
                            int *dep_idx, int *dep_cnt)
{
    __shared__ int set[kDepSet];
    __shared__ int s_over;
    const int w = blockIdx.x;
    if (w >= nwork) return;
    for (int k = threadIdx.x; k < kDepSet; k += blockDim.x) set[k] = -1;
    if (threadIdx.x == 0) s_over = 0;
    __syncthreads();
    const WorkItem wi = work[w];
    const PatchDesc P = patches[wi.patch];
    const int W = wi.tx + 4, H = wi.ty + 4, i0 = P.ilo + wi.x0 - 2, j0 = P.jlo + wi.y0 - 2;
    for (int k = threadIdx.x; k < W * H; k += blockDim.x) {
        int J = j0 + k / W, I = i0 + k % W;
        if (I < 0) { if (bc.x != ADJAMR_BC_PERIODIC) continue; I += N; }
        if (I >= N) { if (bc.y != ADJAMR_BC_PERIODIC) continue; I -= N; }
        if (J < 0) { if (bc.z != ADJAMR_BC_PERIODIC) continue; J += M; }
        if (J >= M) { if (bc.w != ADJAMR_BC_PERIODIC) continue; J -= M; }
        const int o = owner[(long long)J * N + I];
        if (o < 0) continue;
        const int u = tile_of[o];
        int h = (int)(((unsigned)u * 2654435761u) >> 25);  // 7 bits
        bool in = false;
        for (int p = 0; p < kDepSet; p++) {
            const int prev = atomicCAS(&set[h], -1, u);
            if (prev == -1 || prev == u) {
                in = true;
                break;
            }
            h = (h + 1) & (kDepSet - 1);
        }
        if (!in) s_over = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int n = 0;
        for (int k = 0; k < kDepSet; k++)
            if (set[k] >= 0) {
                if (n < kDepRow) dep_idx[(long long)w * kDepRow + n] = set[k];
                n++;
            }
        dep_cnt[w] = (s_over || n > kDepRow) ? kDepRow + 1 : n;
    }
}

template <int EQN>
cudaError_t dispatch_sub(int tx, int ty, int nwork, int grid, double *qa, double *qb, const double *aux,
                         long long stride, const PatchDesc *p, const WorkItem *w, unsigned long long *c, cudaStream_t s,
                         const GhostArgs &ga, const TileSched &sc, const SubstepArgs &sa, int *occ)
{
#define ADJ_SUB(X, Y)                                                                                          \
    if (tx == X && ty == Y) {                                                                                  \
        constexpr size_t smem = Smem2D<EQN, X, Y>::bytes;                                                      \
        cudaError_t e = ensure_smem_attr<k_step2d_sub<EQN, X, Y>>(smem);                                      \
        if (e != cudaSuccess) return e;                                                                        \
        if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_step2d_sub<EQN, X, Y>, kThreads, \
                                                                      smem);                                   \
        return launch_pdl(k_step2d_sub<EQN, X, Y>, dim3(grid), dim3(kThreads), smem, s, qa, qb, aux, stride, p, \
                          w, nwork, c, ga, sc, sa);                                                            \
    }
    ADJ_SUB(16, 16)
    ADJ_SUB(16, 12)
    ADJ_SUB(16, 8)
    ADJ_SUB(8, 8)
#undef ADJ_SUB
    return cudaErrorInvalidValue;
}

cudaError_t sub_switch(int eqn, int tx, int ty, int nwork, int grid, double *qa, double *qb, const double *aux,
                       long long stride, const PatchDesc *p, const WorkItem *w, unsigned long long *c, cudaStream_t s,
                       const GhostArgs &ga, const TileSched &sc, const SubstepArgs &sa, int *occ)
{
    switch (eqn) {
    case 0: return dispatch_sub<0>(tx, ty, nwork, grid, qa, qb, aux, stride, p, w, c, s, ga, sc, sa, occ);
    case 1: return dispatch_sub<1>(tx, ty, nwork, grid, qa, qb, aux, stride, p, w, c, s, ga, sc, sa, occ);
    case 2: return dispatch_sub<2>(tx, ty, nwork, grid, qa, qb, aux, stride, p, w, c, s, ga, sc, sa, occ);
    case 3: return dispatch_sub<3>(tx, ty, nwork, grid, qa, qb, aux, stride, p, w, c, s, ga, sc, sa, occ);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- refluxing
// (A-dQ + A+dQ) of the Riemann problem between a left cell (primary medium
// ml, state (l0, ln)) and a right cell (mr, (r0, rn)): the edge coefficients
// from the primary media as the per-cell coefficient fill computes them
// (c = sqrt(K / rho), Z = rho c, 1 / (Z_l + Z_r); shallow water: the edge
// depth 0.5 (h_l + h_r), c_e = sqrt(g h_e), 1 / c_e), then the jump or flux
// difference, the decomposition and the fluctuations of the step kernel.
template <int EQN>
__device__ __forceinline__ void riemann_total(const double *ml, const double *mr, double l0, double ln, double r0,
                                              double rn, double *tot)
{
    Edge e;
    if constexpr (EQN == 0 || EQN == 1) {
        const double cl = sqrt(ml[1] / ml[0]), cr = sqrt(mr[1] / mr[0]);
        e.Zl = ml[0] * cl;
        e.Zr = mr[0] * cr;
        e.izs = 1.0 / (e.Zl + e.Zr);
        e.s1 = -cl;
        e.s2 = cr;
    } else {
        const double he = 0.5 * (ml[0] + mr[0]);
        e.ghe = kGrav * he;
        e.ce = sqrt(e.ghe);
        e.ice = 1.0 / e.ce;
        e.s1 = -e.ce;
        e.s2 = e.ce;
    }
    double d0, dn;
    if constexpr (EQN == 0) {
        d0 = r0 - l0;
        dn = rn - ln;
    } else if constexpr (EQN == 2) {
        d0 = rn - ln;
        dn = e.ghe * (r0 - l0);
    } else if constexpr (EQN == 1) {
        const double irl = 1.0 / ml[0], irr = 1.0 / mr[0];
        const double fl0 = -(irl * ln), fln = -(ml[1] * l0);
        const double fr0 = -(irr * rn), frn = -(mr[1] * r0);
        d0 = fr0 - fl0;
        dn = frn - fln;
    } else {
        const double gl = kGrav * ml[0], gr = kGrav * mr[0];
        const double fl0 = -(gl * ln), fln = -l0;
        const double fr0 = -(gr * rn), frn = -r0;
        d0 = fr0 - fl0;
        dn = frn - fln;
    }
    double w1[2], w2[2];
    decompose<EQN>(e, d0, dn, w1, w2);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        if constexpr (EQN == 0) tot[k] = e.s1 * w1[k] + e.s2 * w2[k];
        else tot[k] = w1[k] + w2[k];
    }
}

// One thread per coarse-role cell: its sides in the order 0..3, each summing
// L* over the substeps (outer) and the fine edges along the side (inner).
template <int EQN, int DIM>
__global__ void __launch_bounds__(256) k_reflux_apply(RefluxApply a)
{
    pdl_wait();
    pdl_launch_dependents();
    constexpr int NM = nmed_of(EQN);
    constexpr int NS = DIM == 2 ? 4 : 2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.ncoarse; e += gridDim.x * blockDim.x) {
        const RefluxCell rc = a.cells[e];
        const long long ic = rc.idx;
        double mC[2] = {0.0, 0.0};
#pragma unroll
        for (int f = 0; f < NM; f++) mC[f] = a.medc[f * a.sc + ic];
        for (int sd = 0; sd < NS; sd++) {
            if (rc.c[sd] < 0) continue;
            const int n = sd < 2 ? 1 : 2;
            const double c0 = a.qc_old[ic], cn = a.qc_old[n * a.sc + ic];
            double acc0 = 0.0, acc1 = 0.0;
            for (int sb = 0; sb < a.r; sb++)
                for (int g = 0; g < a.nseg; g++) {
                    const long long fr = (long long)rc.c[sd] * a.nseg + g;
                    const double *rec = a.lf + ((long long)sb * a.nfrec + fr) * 4;
                    const long long fi = a.fidx[fr];
                    if (fi < 0) {  // every fine edge of a recorded side has a record: a broken table
                        atomicOr(a.err, kRefluxErrBit);
                        continue;
                    }
                    double mf[2] = {0.0, 0.0};
#pragma unroll
                    for (int f = 0; f < NM; f++) mf[f] = a.medf[f * a.sf + fi];
                    double tot[2];
                    if (sd == 1 || sd == 3) riemann_total<EQN>(mC, mf, c0, cn, rec[2], rec[3], tot);  // C below/left
                    else riemann_total<EQN>(mf, mC, rec[2], rec[3], c0, cn, tot);                  // C above/right
                    acc0 = acc0 + (tot[0] - rec[0]);
                    acc1 = acc1 + (tot[1] - rec[1]);
                }
            const double dtd = sd < 2 ? a.dtdx : a.dtdy;
            const long long lcr = 2 * (long long)rc.c[sd];
            a.qc_new[ic] = a.qc_new[ic] - dtd * (acc0 * a.w - a.lc[lcr]);
            a.qc_new[n * a.sc + ic] = a.qc_new[n * a.sc + ic] - dtd * (acc1 * a.w - a.lc[lcr + 1]);
        }
    }
}

__global__ void k_reflux_map(const RefluxCell *__restrict__ cells, int n, int *rmap)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) rmap[cells[e].idx] = e;
}

}  // namespace

cudaError_t launch_reflux_apply(int dim, int eqn, const RefluxApply &a, cudaStream_t s)
{
    if (a.ncoarse <= 0) return cudaSuccess;
    const dim3 grid((a.ncoarse + 255) / 256), block(256);
    if (dim == 1) {
        switch (eqn) {
        case 0: return launch_pdl(k_reflux_apply<0, 1>, grid, block, 0, s, a);
        case 1: return launch_pdl(k_reflux_apply<1, 1>, grid, block, 0, s, a);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (eqn) {
    case 0: return launch_pdl(k_reflux_apply<0, 2>, grid, block, 0, s, a);
    case 1: return launch_pdl(k_reflux_apply<1, 2>, grid, block, 0, s, a);
    case 2: return launch_pdl(k_reflux_apply<2, 2>, grid, block, 0, s, a);
    case 3: return launch_pdl(k_reflux_apply<3, 2>, grid, block, 0, s, a);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_reflux_map(const RefluxCell *cells, int n, int *rmap, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_reflux_map<<<(n + 255) / 256, 256, 0, s>>>(cells, n, rmap);
    return cudaGetLastError();
}

cudaError_t launch_step_substeps(int eqn, int tx, int ty, double *qa, double *qb, const double *aux, long long stride,
                                 const PatchDesc *patches, const WorkItem *work, int nwork, int grid,
                                 unsigned long long *cfl_bits, cudaStream_t s, const GhostArgs &ga,
                                 const TileSched &sc, const SubstepArgs &sa)
{
    if (!sc.ctr || !ga.gd || sa.nsub < 1 || sa.nsub > kMaxSubsteps || grid < 1) return cudaErrorInvalidValue;
    if (nwork <= 0) return cudaSuccess;
    return sub_switch(eqn, tx, ty, nwork, grid, qa, qb, aux, stride, patches, work, cfl_bits, s, ga, sc, sa, nullptr);
}

cudaError_t launch_tile_deps(const PatchDesc *patches, const WorkItem *work, int nwork, const int *owner, int N, int M,
                             const int *bc, int *tile_of, int *dep_idx, int *dep_cnt, cudaStream_t s)
{
    if (nwork <= 0) return cudaSuccess;
    k_tile_map<<<nwork, 256, 0, s>>>(patches, work, nwork, tile_of);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tile_deps<<<nwork, 256, 0, s>>>(patches, work, nwork, owner, N, M, make_int4(bc[0], bc[1], bc[2], bc[3]),
                                      tile_of, dep_idx, dep_cnt);
    return cudaGetLastError();
}

int substep_occupancy(int eqn, int tx, int ty)
{
    int n = 0;
    const GhostArgs ga{};
    const TileSched sc{};
    const SubstepArgs sa{};
    if (sub_switch(eqn, tx, ty, 0, 0, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, ga, sc, sa,
                   &n) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_step(int dim, int eqn, int tx, int ty, const double *q, double *qn, const double *aux,
                        long long stride, const PatchDesc *patches, const WorkItem *work, int nwork, int grid,
                        unsigned long long *cfl_bits, cudaStream_t s, GhostArgs ga, TileSched sc)
{
    if (dim == 1) {
        switch (eqn) {
        case 0: return dispatch1d<0>(tx, nwork, grid, q, qn, aux, stride, patches, work, cfl_bits, s, ga, sc);
        case 1: return dispatch1d<1>(tx, nwork, grid, q, qn, aux, stride, patches, work, cfl_bits, s, ga, sc);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (eqn) {
    case 0: return dispatch2d<0>(tx, ty, nwork, grid, q, qn, aux, stride, patches, work, cfl_bits, s, ga, sc);
    case 1: return dispatch2d<1>(tx, ty, nwork, grid, q, qn, aux, stride, patches, work, cfl_bits, s, ga, sc);
    case 2: return dispatch2d<2>(tx, ty, nwork, grid, q, qn, aux, stride, patches, work, cfl_bits, s, ga, sc);
    case 3: return dispatch2d<3>(tx, ty, nwork, grid, q, qn, aux, stride, patches, work, cfl_bits, s, ga, sc);
    default: return cudaErrorInvalidValue;
    }
}

bool step_kernel_shape(int dim, int tx, int ty, int *kx, int *ky)
{
    if (tx < 1 || ty < 1) return false;
    if (dim == 1) {
        if (tx > 256) return false;
        *kx = tx <= 128 ? 128 : 256;
        *ky = 1;
        return true;
    }
    static const int shapes[7][2] = {{8, 8}, {16, 8}, {16, 12}, {32, 8}, {16, 16}, {64, 8}, {32, 16}};
    for (const auto &sh : shapes)
        if (tx <= sh[0] && ty <= sh[1]) {
            *kx = sh[0];
            *ky = sh[1];
            return true;
        }
    return false;
}

int step_occupancy(int dim, int eqn, int tx, int ty)
{
    if (dim == 1) return 4;
    switch (eqn) {
    case 0: return occ2d<0>(tx, ty);
    case 1: return occ2d<1>(tx, ty);
    case 2: return occ2d<2>(tx, ty);
    case 3: return occ2d<3>(tx, ty);
    default: return 0;
    }
}

}  // namespace adjamr
