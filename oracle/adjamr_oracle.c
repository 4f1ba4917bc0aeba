/*
 * Plain, slow, single-threaded CPU FP64 oracle of adjoint-guided
 * block-structured AMR for linear hyperbolic waves (Davis & LeVeque,
 * "Adjoint methods for guiding adaptive mesh refinement in wave propagation
 * problems").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA implementation; the two agree
 * because both follow the same written operation order (the "canonical
 * operations"), not because they share source.
 *
 * Compile with -O2 -ffp-contract=off: every floating-point operation below
 * is a single IEEE-754 operation (+ - * / sqrt fma fmin fmax fabs; fma is the
 * C99 fused multiply-add, rounded once), evaluated in the order written.
 *
 * What it computes, by paper section:
 *  - Sec. 2, Eq. (eq:qtAqx), (adjoint1): forward q_t + A q_x (+ B q_y) = 0
 *    and the time-reversed adjoint  q~_t - (A^T q~)_x (- (B^T q~)_y) = 0
 *    (Sec. 4).  Acoustics: Sec. 5.1 (1D) and Sec. 5.2 (2D) matrices;
 *    linearised shallow water: Sec. 5.3 matrices.
 *  - Sec. 3: high-resolution wave propagation (Riemann solves at every
 *    edge, limited second-order corrections, transverse Riemann problems),
 *    f-wave form for the adjoint (conservative) systems and for the
 *    bathymetry-dependent shallow-water flux.
 *  - Sec. 3: nested patches refined in space and time, coarse-first
 *    recursion, ghost cells from same-level neighbours or space-time
 *    interpolation from the coarser level; flag -> cluster
 *    (Berger-Rigoutsos) -> properly nested patches, regridded every few
 *    steps.
 *  - Sec. 4: adjoint solved once on a fixed grid, snapshots at regular
 *    intervals, bilinear interpolation in space, both bracketing snapshots
 *    in time; Sec. 5.1.2: maximum over the time window of interest.
 *  - Sec. 2, Eq. (eq:J_general): the functional J.
 *  - Sec. 5.2.4 and Sec. 5.3: the standard flagging the paper compares
 *    against (undivided differences of every component; surface elevation)
 *    and gauges (time series at points, finest level covering the point).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OMAXLEV 8
#define OGRAV 9.81

enum { O_ACOU = 0, O_ACOU_ADJ = 1, O_SW = 2, O_SW_ADJ = 3 };
enum { O_EXTRAP = 0, O_WALL = 1, O_PERIODIC = 2 };
enum { O_BRACKET = 0, O_LINEAR = 1, O_DIFF = 2, O_SURFACE = 3, O_ERROR = 4, O_RICHARDSON = 5 };
enum { O_MED_NONE = 0, O_MED_LAYERED = 1, O_MED_DENSE = 2 };

typedef void (*orc_qinit_fn)(int level, int n, const double *xc, const double *yc, double *q_out, void *user);

typedef struct {
    int dim, eqn;
    double lo[2], hi[2];
    int n0[2];
    int nlevels;
    int ratio[OMAXLEV];
    int bc[4];
    double cfl, cfl_max, cmax, dt0;
    double t0, tf, ts, tol;
    int regrid_interval, buffer;
    double cluster_eff;
    int min_patch, max_patch, max_patch0;
    int flag_mode;
    orc_qinit_fn qinit;
    void *qinit_user;
    int reflux;   /* conservation fix-up at coarse-fine interfaces (Sec. 3; Berger-LeVeque) */
} orc_params;

typedef struct {
    int ilo, jlo, nx, ny;
    double *q[2];
    double *med;
} OPatch;

typedef struct {
    int np;
    OPatch *p;
    int N, M;
    double dx, dy, dt;
    long nstep;
    int cur;
} OLevel;

typedef struct {
    int kind, axis, nl;
    double iface[32], f0[32], f1[32];
    double *dense[OMAXLEV][2];
    int dn[OMAXLEV][2];
} OMedium;

/* conservation fix-up register of one coarse level l: one entry per
   (uncovered level-l cell C, side of C that faces a level-(l+1) patch) */
typedef struct {
    int pk, i, j, side; /* coarse patch, local cell, side 0..3 = x-left, x-right, y-bottom, y-top */
    double Lc[2];       /* what the coarse step put into C through that side */
    double *Lf;         /* [substep][segment][2]: the fine-side values L* */
} OReg;

typedef struct {
    int active, n, cap, N, M;
    OReg *e;
    int *idx;           /* [4][M][N]: entry of (cell, side), -1 if none */
    unsigned char *cov; /* [M][N]: cell covered by level l+1 */
} ORegs;

typedef struct {
    orc_params P;
    int m, nmed, gx, gy;
    ORegs reg[OMAXLEV];
    OLevel L[OMAXLEV];
    OMedium med;
    long T[OMAXLEV];
    long rebuilt_tick[OMAXLEV];
    /* adjoint snapshots in forward time order: snaps[n][f][j][i] */
    int nsnap, an[2];
    double *snaps;
    unsigned char *wet;
    long long cell_updates;
    /* gauges: points recorded after every level-0 step, grec[n][g][1 + m] =
       (t, q of the cell holding the point on the finest level covering it) */
    int ngauge;
    double *gxs, *gys;
    long ngrec, gcap;
    double *grec;
    /* adjoint-weighted error flagging: the error estimate of the level being
       flagged, [cell in patch order, row-major within a patch][m] */
    double *tau;
    long ntau;
    char err[256];
} OHier;

static void reg_clear(ORegs *R);

/* ------------------------------------------------------------------ */
/* storage helpers                                                     */
/* ------------------------------------------------------------------ */
static int sxof(const OHier *h, const OPatch *p) { return p->nx + 2 * h->gx; }
static int syof(const OHier *h, const OPatch *p) { return p->ny + 2 * h->gy; }
/* index of field f, local cell (i, j), i in [-gx, nx+gx), j in [-gy, ny+gy) */
static long qidx(const OHier *h, const OPatch *p, int f, int i, int j)
{
    return ((long)f * syof(h, p) + (j + h->gy)) * sxof(h, p) + (i + h->gx);
}

static void *xcalloc(size_t n, size_t s)
{
    void *v = calloc(n ? n : 1, s);
    if (!v) {
        fprintf(stderr, "oracle: out of memory\n");
        abort();
    }
    return v;
}

static double level_time(const OHier *h, int l) { return h->P.t0 + (double)h->L[l].nstep * h->L[l].dt; }

/* ------------------------------------------------------------------ */
/* medium                                                              */
/* ------------------------------------------------------------------ */
/* primary medium at an in-domain cell (I, J) of level l:
   acoustics (rho, K); shallow water (hbar). */
static void medium_at(const OHier *h, int l, int I, int J, double *out)
{
    const OMedium *m = &h->med;
    if (m->kind == O_MED_LAYERED) {
        double c = (m->axis == 0) ? h->P.lo[0] + ((double)I + 0.5) * h->L[l].dx
                                  : h->P.lo[1] + ((double)J + 0.5) * h->L[l].dy;
        int k = 0;
        while (k < m->nl - 1 && m->iface[k] <= c) k++;
        out[0] = m->f0[k];
        out[1] = m->f1[k];
    } else {
        long idx = (long)J * m->dn[l][0] + I;
        out[0] = m->dense[l][0][idx];
        if (h->nmed > 1) out[1] = m->dense[l][1][idx];
    }
}

/* ------------------------------------------------------------------ */
/* boundary-condition index map: (I, J) possibly outside the domain ->  */
/* in-domain cell and per-field sign.  Extrapolation: nearest interior; */
/* wall: mirror with the normal velocity negated; periodic: wrap.       */
/* ------------------------------------------------------------------ */
static void map_bc(const OHier *h, int l, int *I, int *J, double *sign)
{
    int N = h->L[l].N, M = h->L[l].M;
    for (int f = 0; f < h->m; f++) sign[f] = 1.0;
    if (*I < 0) {
        int bc = h->P.bc[0];
        if (bc == O_EXTRAP) *I = 0;
        else if (bc == O_WALL) { *I = -1 - *I; sign[1] = -sign[1]; }
        else *I += N;
    } else if (*I >= N) {
        int bc = h->P.bc[1];
        if (bc == O_EXTRAP) *I = N - 1;
        else if (bc == O_WALL) { *I = 2 * N - 1 - *I; sign[1] = -sign[1]; }
        else *I -= N;
    }
    if (h->P.dim == 2) {
        if (*J < 0) {
            int bc = h->P.bc[2];
            if (bc == O_EXTRAP) *J = 0;
            else if (bc == O_WALL) { *J = -1 - *J; sign[2] = -sign[2]; }
            else *J += M;
        } else if (*J >= M) {
            int bc = h->P.bc[3];
            if (bc == O_EXTRAP) *J = M - 1;
            else if (bc == O_WALL) { *J = 2 * M - 1 - *J; sign[2] = -sign[2]; }
            else *J -= M;
        }
    }
}

static void fill_patch_medium(OHier *h, int l, OPatch *p)
{
    double sg[3], v[2];
    for (int j = -h->gy; j < p->ny + h->gy; j++)
        for (int i = -h->gx; i < p->nx + h->gx; i++) {
            int I = p->ilo + i, J = p->jlo + j;
            map_bc(h, l, &I, &J, sg);
            medium_at(h, l, I, J, v);
            for (int f = 0; f < h->nmed; f++) p->med[qidx(h, p, f, i, j)] = v[f];
        }
}

/* ------------------------------------------------------------------ */
/* Riemann solvers (Sec. 3 + the matrices of Secs. 5.1-5.3).            */
/* All work on the two active components of a direction: component 0   */
/* (pressure / surface) and the normal velocity/momentum component n.   */
/* ------------------------------------------------------------------ */
typedef struct {
    double s1, s2;     /* left-going and right-going speeds */
    double Zl, Zr, izs; /* acoustics: impedances, 1/(Zl+Zr) */
    double ce, ice;    /* shallow water: edge speed and its reciprocal */
    double ghe;        /* shallow water: g * (edge depth) */
} OEdge;

/* medium-only coefficients at the edge between cells with primary medium ml, mr */
static void edge_coef(int eqn, const double *ml, const double *mr, OEdge *e)
{
    if (eqn == O_ACOU || eqn == O_ACOU_ADJ) {
        double cl = sqrt(ml[1] / ml[0]);
        double cr = sqrt(mr[1] / mr[0]);
        e->Zl = ml[0] * cl;
        e->Zr = mr[0] * cr;
        e->izs = 1.0 / (e->Zl + e->Zr);
        e->s1 = -cl;
        e->s2 = cr;
        e->ce = e->ice = e->ghe = 0.0;
    } else {
        double he = 0.5 * (ml[0] + mr[0]);
        e->ghe = OGRAV * he;
        e->ce = sqrt(e->ghe);
        e->ice = 1.0 / e->ce;
        e->s1 = -e->ce;
        e->s2 = e->ce;
        e->Zl = e->Zr = e->izs = 0.0;
    }
}

/* Decompose a 2-vector d = (d0, dn) into the eigenvectors of the edge.
 *  acoustics (wave form, eigenvectors of A):   d = a1 (-Zl, 1) + a2 (Zr, 1)
 *  adjoint acoustics (f-wave, eigvecs of -A^T): d = b1 (1, Zl) + b2 (1, -Zr)
 *  shallow water (f-wave, edge speed ce):      d = b1 (1, -ce) + b2 (1, ce)
 *  adjoint shallow water (f-wave):             d = b1 (ce, 1) + b2 (-ce, 1)
 * d is the jump dQ (wave form) or the flux difference df (f-wave forms). */
static void decompose(int eqn, const OEdge *e, double d0, double dn, double *w1, double *w2)
{
    if (eqn == O_ACOU) {
        double a1 = fma(e->Zr, dn, -d0) * e->izs;
        double a2 = fma(e->Zl, dn, d0) * e->izs;
        w1[0] = -(e->Zl * a1);
        w1[1] = a1;
        w2[0] = e->Zr * a2;
        w2[1] = a2;
    } else if (eqn == O_ACOU_ADJ) {
        double b1 = fma(e->Zr, d0, dn) * e->izs;
        double b2 = fma(e->Zl, d0, -dn) * e->izs;
        w1[0] = b1;
        w1[1] = e->Zl * b1;
        w2[0] = b2;
        w2[1] = -(e->Zr * b2);
    } else if (eqn == O_SW) {
        double b1 = fma(-dn, e->ice, d0) * 0.5;
        double b2 = fma(dn, e->ice, d0) * 0.5;
        w1[0] = b1;
        w1[1] = -(e->ce * b1);
        w2[0] = b2;
        w2[1] = e->ce * b2;
    } else {
        double b1 = fma(d0, e->ice, dn) * 0.5;
        double b2 = fma(-d0, e->ice, dn) * 0.5;
        w1[0] = e->ce * b1;
        w1[1] = b1;
        w2[0] = -(e->ce * b2);
        w2[1] = b2;
    }
}

/* flux of an f-wave (adjoint) system in one cell, components (0, n):
 *  adjoint acoustics: f = -A^T q = (-(u_n / rho), -(K p));
 *  adjoint shallow water: f = (-(g hbar mu_n), -eta). */
static void cell_flux(int eqn, const double *med, double q0, double qn, double *f)
{
    if (eqn == O_ACOU_ADJ) {
        double irho = 1.0 / med[0];
        f[0] = -(irho * qn);
        f[1] = -(med[1] * q0);
    } else {
        double gh = OGRAV * med[0];
        f[0] = -(gh * qn);
        f[1] = -q0;
    }
}

/* Normal Riemann problem at one edge: waves, speeds and fluctuations. */
typedef struct {
    OEdge e;
    double w1[2], w2[2];
    double am[2], ap[2];
    double Fn[2];
} OEdgeRes;

static void normal_solve(int eqn, const double *ml, const double *mr, double ql0, double qln, double qr0,
                         double qrn, OEdgeRes *r)
{
    edge_coef(eqn, ml, mr, &r->e);
    double d0, dn;
    if (eqn == O_ACOU) {
        d0 = qr0 - ql0;
        dn = qrn - qln;
    } else if (eqn == O_SW) {
        /* linearised shallow water: df = (d mu, g hbar_edge d eta) */
        d0 = qrn - qln;
        dn = r->e.ghe * (qr0 - ql0);
    } else {
        double fl[2], fr[2];
        cell_flux(eqn, ml, ql0, qln, fl);
        cell_flux(eqn, mr, qr0, qrn, fr);
        d0 = fr[0] - fl[0];
        dn = fr[1] - fl[1];
    }
    decompose(eqn, &r->e, d0, dn, r->w1, r->w2);
    if (eqn == O_ACOU) {
        for (int k = 0; k < 2; k++) {
            r->am[k] = r->e.s1 * r->w1[k];
            r->ap[k] = r->e.s2 * r->w2[k];
        }
    } else {
        for (int k = 0; k < 2; k++) {
            r->am[k] = r->w1[k];
            r->ap[k] = r->w2[k];
        }
    }
    r->Fn[0] = r->Fn[1] = 0.0;
}

/* Transverse split of a fluctuation delta = (d0, dn) at an edge:
 * left-going part s1*w1(delta) and right-going part s2*w2(delta). */
static void trans_minus(int eqn, const OEdge *e, double d0, double dn, double *out)
{
    double w1[2], w2[2];
    decompose(eqn, e, d0, dn, w1, w2);
    out[0] = e->s1 * w1[0];
    out[1] = e->s1 * w1[1];
}
static void trans_plus(int eqn, const OEdge *e, double d0, double dn, double *out)
{
    double w1[2], w2[2];
    decompose(eqn, e, d0, dn, w1, w2);
    out[0] = e->s2 * w2[0];
    out[1] = e->s2 * w2[1];
}

/* MC limiter (monotonized centred): phi(th) = max(0, min((1+th)/2, 2, 2 th)),
 * th = (W_upwind . W) / (W . W); phi = 0 when W . W = 0. */
static double mc_phi(const double *w, const double *wu)
{
    double wn = fma(w[0], w[0], w[1] * w[1]);
    if (wn == 0.0) return 0.0;
    double dot = fma(wu[0], w[0], wu[1] * w[1]);
    double th = dot / wn;
    return fmax(0.0, fmin(fmin(fma(0.5, th, 0.5), 2.0), 2.0 * th));
}

/* second-order correction flux Fn = 1/2 sum_p cf_p phi_p W_p at edge r, with
 * upwind neighbours rm (edge - 1) and rp (edge + 1) in the normal direction. */
static void limit_edge(int eqn, double dtdx, OEdgeRes *r, const OEdgeRes *rm, const OEdgeRes *rp)
{
    const double *wu1 = (r->e.s1 > 0.0) ? rm->w1 : rp->w1;
    const double *wu2 = (r->e.s2 > 0.0) ? rm->w2 : rp->w2;
    double phi1 = mc_phi(r->w1, wu1);
    double phi2 = mc_phi(r->w2, wu2);
    double a1 = fabs(r->e.s1), a2 = fabs(r->e.s2);
    double cf1, cf2;
    if (eqn == O_ACOU) {
        cf1 = a1 * fma(-dtdx, a1, 1.0);
        cf2 = a2 * fma(-dtdx, a2, 1.0);
    } else {
        double t1 = fma(-dtdx, a1, 1.0), t2 = fma(-dtdx, a2, 1.0);
        cf1 = (r->e.s1 < 0.0) ? -t1 : t1;
        cf2 = (r->e.s2 < 0.0) ? -t2 : t2;
    }
    for (int k = 0; k < 2; k++) {
        double wl1 = phi1 * r->w1[k];
        double wl2 = phi2 * r->w2[k];
        r->Fn[k] = 0.5 * (cf1 * wl1 + cf2 * wl2);
    }
}

/* ------------------------------------------------------------------ */
/* one step of one patch                                               */
/* q, med: ghosted storage (gx = 2; gy = 2 in 2D, 0 in 1D) of extents  */
/* sx = nx + 4 and sy; qout: interior only, field-major [f][j][i].     */
/* ------------------------------------------------------------------ */
static double step_patch(int dim, int eqn, int nx, int ny, const double *q, const double *med, double dt,
                         double dx, double dy, double *qout, double *side)
{
    const int gx = 2, gy = (dim == 2) ? 2 : 0;
    const int sx = nx + 2 * gx, sy = ny + 2 * gy;
    const int m = (dim == 2) ? 3 : 2, nmed = (eqn == O_SW || eqn == O_SW_ADJ) ? 1 : 2;
    const double dtdx = dt / dx, dtdy = (dim == 2) ? dt / dy : 0.0;
    const double hx = 0.5 * dtdx, hy = 0.5 * dtdy;
#define Q(f, i, j) q[((long)(f) * sy + (j) + gy) * sx + (i) + gx]
#define MED(i, j, out)                                                                         \
    do {                                                                                       \
        for (int _f = 0; _f < nmed; _f++) (out)[_f] = med[((long)_f * sy + (j) + gy) * sx + (i) + gx]; \
    } while (0)
    double cfl = 0.0;

    if (dim == 1) {
        /* x-edges e in [-1, nx+1]; edge e separates cells e-1 and e */
        int ne = nx + 3;
        OEdgeRes *X = xcalloc(ne, sizeof(OEdgeRes));
        for (int e = -1; e <= nx + 1; e++) {
            double ml[2], mr[2];
            MED(e - 1, 0, ml);
            MED(e, 0, mr);
            normal_solve(eqn, ml, mr, Q(0, e - 1, 0), Q(1, e - 1, 0), Q(0, e, 0), Q(1, e, 0), &X[e + 1]);
        }
        for (int e = 0; e <= nx; e++) {
            limit_edge(eqn, dtdx, &X[e + 1], &X[e], &X[e + 2]);
            double c = dtdx * fmax(fabs(X[e + 1].e.s1), fabs(X[e + 1].e.s2));
            cfl = fmax(cfl, c);
        }
        for (int i = 0; i < nx; i++) {
            const OEdgeRes *L = &X[i + 1], *R = &X[i + 2];
            double A0 = (L->ap[0] + R->am[0]) + (R->Fn[0] - L->Fn[0]);
            double A1 = (L->ap[1] + R->am[1]) + (R->Fn[1] - L->Fn[1]);
            qout[i] = Q(0, i, 0) - dtdx * A0;
            qout[(long)nx + i] = fma(-dtdx, A1, Q(1, i, 0));
            if (side)
                for (int k = 0; k < 2; k++) {
                    side[(long)(0 * 2 + k) * nx + i] = L->ap[k] - L->Fn[k];
                    side[(long)(1 * 2 + k) * nx + i] = R->am[k] + R->Fn[k];
                }
        }
        free(X);
        return cfl;
    }

    /* ---- 2D ---- */
    /* x-edges: e in [-1, nx+1], rows j in [-1, ny] */
    int nex = nx + 3, nrx = ny + 2;
    OEdgeRes *X = xcalloc((size_t)nex * nrx, sizeof(OEdgeRes));
#define XE(e, j) X[((j) + 1) * nex + (e) + 1]
    for (int j = -1; j <= ny; j++)
        for (int e = -1; e <= nx + 1; e++) {
            double ml[2], mr[2];
            MED(e - 1, j, ml);
            MED(e, j, mr);
            normal_solve(eqn, ml, mr, Q(0, e - 1, j), Q(1, e - 1, j), Q(0, e, j), Q(1, e, j), &XE(e, j));
        }
    for (int j = -1; j <= ny; j++)
        for (int e = 0; e <= nx; e++) limit_edge(eqn, dtdx, &XE(e, j), &XE(e - 1, j), &XE(e + 1, j));
    /* y-edges: e in [-1, ny+1], columns i in [-1, nx] */
    int ney = ny + 3, ncy = nx + 2;
    OEdgeRes *Y = xcalloc((size_t)ney * ncy, sizeof(OEdgeRes));
#define YE(i, e) Y[((e) + 1) * ncy + (i) + 1]
    for (int e = -1; e <= ny + 1; e++)
        for (int i = -1; i <= nx; i++) {
            double ml[2], mr[2];
            MED(i, e - 1, ml);
            MED(i, e, mr);
            normal_solve(eqn, ml, mr, Q(0, i, e - 1), Q(2, i, e - 1), Q(0, i, e), Q(2, i, e), &YE(i, e));
        }
    for (int e = 0; e <= ny; e++)
        for (int i = -1; i <= nx; i++) limit_edge(eqn, dtdy, &YE(i, e), &YE(i, e - 1), &YE(i, e + 1));

    /* Sx(i, j): x-fluctuations entering cell (i, j), including the
       second-order corrections (A+dQ - Fn from the left edge, A-dQ + Fn
       from the right edge); comps (0, u).  i in [0, nx), j in [-1, ny]. */
    double *Sx = xcalloc((size_t)2 * nx * (ny + 2), sizeof(double));
#define SX(k, i, j) Sx[((long)(k) * (ny + 2) + (j) + 1) * nx + (i)]
    for (int j = -1; j <= ny; j++)
        for (int i = 0; i < nx; i++) {
            const OEdgeRes *L = &XE(i, j), *R = &XE(i + 1, j);
            for (int k = 0; k < 2; k++) {
                double apT = L->ap[k] - L->Fn[k];
                double amT = R->am[k] + R->Fn[k];
                SX(k, i, j) = apT + amT;
            }
        }
    /* Sy(i, j): y-fluctuations entering cell (i, j); comps (0, v).
       i in [-1, nx], j in [0, ny). */
    double *Sy = xcalloc((size_t)2 * (nx + 2) * ny, sizeof(double));
#define SY(k, i, j) Sy[((long)(k) * ny + (j)) * (nx + 2) + (i) + 1]
    for (int j = 0; j < ny; j++)
        for (int i = -1; i <= nx; i++) {
            const OEdgeRes *B = &YE(i, j), *T = &YE(i, j + 1);
            for (int k = 0; k < 2; k++) {
                double bpT = B->ap[k] - B->Fn[k];
                double bmT = T->am[k] + T->Fn[k];
                SY(k, i, j) = bpT + bmT;
            }
        }
    /* full x-edge fluxes: F = Fn - (dt/2dy) (A-(Sy right cell) + A+(Sy left cell));
       the y-fluctuation has zero x-normal (u) component.  e in [0, nx], j in [0, ny). */
    double *F = xcalloc((size_t)2 * (nx + 1) * ny, sizeof(double));
#define FF(k, e, j) F[((long)(k) * ny + (j)) * (nx + 1) + (e)]
    for (int j = 0; j < ny; j++)
        for (int e = 0; e <= nx; e++) {
            const OEdgeRes *r = &XE(e, j);
            double tm[2], tp[2];
            trans_minus(eqn, &r->e, SY(0, e, j), 0.0, tm);
            trans_plus(eqn, &r->e, SY(0, e - 1, j), 0.0, tp);
            for (int k = 0; k < 2; k++) FF(k, e, j) = fma(-hy, tm[k] + tp[k], r->Fn[k]);
            double c = dtdx * fmax(fabs(r->e.s1), fabs(r->e.s2));
            cfl = fmax(cfl, c);
        }
    /* full y-edge fluxes: G = Gn - (dt/2dx) (B-(Sx upper cell) + B+(Sx lower cell)). */
    double *G = xcalloc((size_t)2 * nx * (ny + 1), sizeof(double));
#define GG(k, i, e) G[((long)(k) * (ny + 1) + (e)) * nx + (i)]
    for (int e = 0; e <= ny; e++)
        for (int i = 0; i < nx; i++) {
            const OEdgeRes *r = &YE(i, e);
            double tm[2], tp[2];
            trans_minus(eqn, &r->e, SX(0, i, e), 0.0, tm);
            trans_plus(eqn, &r->e, SX(0, i, e - 1), 0.0, tp);
            for (int k = 0; k < 2; k++) GG(k, i, e) = fma(-hx, tm[k] + tp[k], r->Fn[k]);
            double c = dtdy * fmax(fabs(r->e.s1), fabs(r->e.s2));
            cfl = fmax(cfl, c);
        }
    /* cell update: p - (X_p + Y_p) with X = dtdx*A from the x-edges and Y =
       dtdy*B from the y-edges; the velocities see one direction each:
       u - dtdx*A_u and v - dtdy*B_v, each with one rounding. */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const OEdgeRes *L = &XE(i, j), *R = &XE(i + 1, j);
            const OEdgeRes *B = &YE(i, j), *T = &YE(i, j + 1);
            double Ax[2], By[2];
            for (int k = 0; k < 2; k++) {
                Ax[k] = (L->ap[k] + R->am[k]) + (FF(k, i + 1, j) - FF(k, i, j));
                By[k] = (B->ap[k] + T->am[k]) + (GG(k, i, j + 1) - GG(k, i, j));
            }
            qout[((long)0 * ny + j) * nx + i] = Q(0, i, j) - (dtdx * Ax[0] + dtdy * By[0]);
            qout[((long)1 * ny + j) * nx + i] = fma(-dtdx, Ax[1], Q(1, i, j));
            qout[((long)2 * ny + j) * nx + i] = fma(-dtdy, By[1], Q(2, i, j));
            if (side) {
                long nc = (long)nx * ny, c = (long)j * nx + i;
                for (int k = 0; k < 2; k++) {
                    side[(0 * 2 + k) * nc + c] = L->ap[k] - FF(k, i, j);
                    side[(1 * 2 + k) * nc + c] = R->am[k] + FF(k, i + 1, j);
                    side[(2 * 2 + k) * nc + c] = B->ap[k] - GG(k, i, j);
                    side[(3 * 2 + k) * nc + c] = T->am[k] + GG(k, i, j + 1);
                }
            }
        }
    free(X);
    free(Y);
    free(Sx);
    free(Sy);
    free(F);
    free(G);
#undef Q
#undef MED
#undef XE
#undef YE
#undef SX
#undef SY
#undef FF
#undef GG
    (void)m;
    return cfl;
}


/* exported: one step of a standalone ghosted patch */
int orc_step_patch(int dim, int eqn, int nx, int ny, const double *q, const double *med, double dt, double dx,
                   double dy, double *qout, double *cfl)
{
    if (dim == 1) ny = 1;
    double c = step_patch(dim, eqn, nx, ny, q, med, dt, dx, dy, qout, NULL);
    if (cfl) *cfl = c;
    return 0;
}

/* ------------------------------------------------------------------ */
/* hierarchy                                                           */
/* ------------------------------------------------------------------ */
static void free_patch(OPatch *p)
{
    free(p->q[0]);
    free(p->q[1]);
    free(p->med);
    p->q[0] = p->q[1] = p->med = NULL;
}

static void alloc_patch(OHier *h, OPatch *p)
{
    long n = (long)sxof(h, p) * syof(h, p);
    p->q[0] = xcalloc((size_t)n * h->m, sizeof(double));
    p->q[1] = xcalloc((size_t)n * h->m, sizeof(double));
    p->med = xcalloc((size_t)n * h->nmed, sizeof(double));
}

static int find_patch(const OHier *h, int l, int I, int J)
{
    const OLevel *L = &h->L[l];
    for (int k = 0; k < L->np; k++) {
        const OPatch *p = &L->p[k];
        if (I >= p->ilo && I < p->ilo + p->nx && J >= p->jlo && J < p->jlo + p->ny) return k;
    }
    return -1;
}

/* split a length into p near-equal parts: the first (n % p) get one more */
static int part_len(int n, int p, int k) { return n / p + (k < n % p ? 1 : 0); }
static int part_off(int n, int p, int k)
{
    int o = 0;
    for (int q = 0; q < k; q++) o += part_len(n, p, q);
    return o;
}

void *orc_create(const orc_params *P)
{
    if (P->dim < 1 || P->dim > 2 || P->nlevels < 1 || P->nlevels > OMAXLEV) return NULL;
    OHier *h = xcalloc(1, sizeof(OHier));
    h->P = *P;
    h->m = (P->dim == 2) ? 3 : 2;
    h->nmed = (P->eqn == O_SW || P->eqn == O_SW_ADJ) ? 1 : 2;
    h->gx = 2;
    h->gy = (P->dim == 2) ? 2 : 0;
    int N = P->n0[0], M = (P->dim == 2) ? P->n0[1] : 1;
    for (int l = 0; l < P->nlevels; l++) {
        OLevel *L = &h->L[l];
        L->N = N;
        L->M = M;
        L->dx = (P->hi[0] - P->lo[0]) / (double)N;
        L->dy = (P->dim == 2) ? (P->hi[1] - P->lo[1]) / (double)M : 1.0;
        if (l < P->nlevels - 1) {
            N *= P->ratio[l];
            if (P->dim == 2) M *= P->ratio[l];
        }
        h->rebuilt_tick[l] = -1;
    }
    /* time steps: dt0 = (tf-t0)/ceil((tf-t0)/dt_cfl), dt_l = dt_{l-1}/r */
    double dt0 = P->dt0;
    if (dt0 <= 0.0) {
        double dmin = (P->dim == 2) ? fmin(h->L[0].dx, h->L[0].dy) : h->L[0].dx;
        double dtc = P->cfl * dmin / P->cmax;
        double ns = ceil((P->tf - P->t0) / dtc);
        dt0 = (P->tf - P->t0) / ns;
    }
    h->L[0].dt = dt0;
    for (int l = 1; l < P->nlevels; l++) h->L[l].dt = h->L[l - 1].dt / (double)P->ratio[l - 1];
    long T = 1;
    for (int l = P->nlevels - 1; l >= 0; l--) {
        h->T[l] = T;
        if (l > 0) T *= P->ratio[l - 1];
    }
    /* level 0 tiles the domain with near-equal patches of at most max_patch0 cells */
    OLevel *L0 = &h->L[0];
    int px = (L0->N + P->max_patch0 - 1) / P->max_patch0;
    int py = (P->dim == 2) ? (L0->M + P->max_patch0 - 1) / P->max_patch0 : 1;
    L0->np = px * py;
    L0->p = xcalloc(L0->np, sizeof(OPatch));
    for (int b = 0; b < py; b++)
        for (int a = 0; a < px; a++) {
            OPatch *p = &L0->p[b * px + a];
            p->ilo = part_off(L0->N, px, a);
            p->nx = part_len(L0->N, px, a);
            p->jlo = (P->dim == 2) ? part_off(L0->M, py, b) : 0;
            p->ny = (P->dim == 2) ? part_len(L0->M, py, b) : 1;
            alloc_patch(h, p);
        }
    /* initial data from qinit at cell centres */
    if (P->qinit) {
        for (int k = 0; k < L0->np; k++) {
            OPatch *p = &L0->p[k];
            int n = p->nx * p->ny;
            double *xc = xcalloc(n, sizeof(double)), *yc = xcalloc(n, sizeof(double));
            double *qv = xcalloc((size_t)n * h->m, sizeof(double));
            for (int j = 0; j < p->ny; j++)
                for (int i = 0; i < p->nx; i++) {
                    xc[j * p->nx + i] = P->lo[0] + ((double)(p->ilo + i) + 0.5) * L0->dx;
                    yc[j * p->nx + i] = (P->dim == 2) ? P->lo[1] + ((double)(p->jlo + j) + 0.5) * L0->dy : 0.0;
                }
            P->qinit(0, n, xc, yc, qv, P->qinit_user);
            for (int f = 0; f < h->m; f++)
                for (int j = 0; j < p->ny; j++)
                    for (int i = 0; i < p->nx; i++) p->q[0][qidx(h, p, f, i, j)] = qv[(long)f * n + j * p->nx + i];
            free(xc);
            free(yc);
            free(qv);
        }
    }
    return h;
}

void orc_destroy(void *hv)
{
    OHier *h = hv;
    if (!h) return;
    for (int l = 0; l < h->P.nlevels; l++) {
        for (int k = 0; k < h->L[l].np; k++) free_patch(&h->L[l].p[k]);
        free(h->L[l].p);
        for (int f = 0; f < 2; f++) free(h->med.dense[l][f]);
        reg_clear(&h->reg[l]);
        free(h->reg[l].e);
        free(h->reg[l].idx);
        free(h->reg[l].cov);
    }
    free(h->snaps);
    free(h->wet);
    free(h->gxs);
    free(h->gys);
    free(h->grec);
    free(h->tau);
    free(h);
}

int orc_set_medium_layered(void *hv, int axis, int nl, const double *iface, const double *f0, const double *f1)
{
    OHier *h = hv;
    if (nl < 1 || nl > 32) return 1;
    h->med.kind = O_MED_LAYERED;
    h->med.axis = axis;
    h->med.nl = nl;
    for (int k = 0; k < nl - 1; k++) h->med.iface[k] = iface[k];
    for (int k = 0; k < nl; k++) {
        h->med.f0[k] = f0[k];
        h->med.f1[k] = f1 ? f1[k] : 0.0;
    }
    for (int k = 0; k < h->L[0].np; k++) fill_patch_medium(h, 0, &h->L[0].p[k]);
    return 0;
}

/* dense medium of one level: fields [nmed][M_l][N_l] */
int orc_set_medium_dense(void *hv, int level, const double *fields)
{
    OHier *h = hv;
    if (level < 0 || level >= h->P.nlevels) return 1;
    long n = (long)h->L[level].N * h->L[level].M;
    h->med.kind = O_MED_DENSE;
    h->med.dn[level][0] = h->L[level].N;
    h->med.dn[level][1] = h->L[level].M;
    for (int f = 0; f < h->nmed; f++) {
        free(h->med.dense[level][f]);
        h->med.dense[level][f] = xcalloc(n, sizeof(double));
        memcpy(h->med.dense[level][f], fields + (long)f * n, (size_t)n * sizeof(double));
    }
    if (level == 0)
        for (int k = 0; k < h->L[0].np; k++) fill_patch_medium(h, 0, &h->L[0].p[k]);
    return 0;
}

/* snapshots [nsnap][m][ay][ax] in forward time order; wet [ay][ax] or NULL */
int orc_set_adjoint(void *hv, int nsnap, int ax, int ay, const double *snaps, const unsigned char *wet)
{
    OHier *h = hv;
    if (nsnap < 2) return 1;
    if (h->P.dim == 1) ay = 1;
    free(h->snaps);
    free(h->wet);
    long n = (long)nsnap * h->m * ax * ay;
    h->snaps = xcalloc(n, sizeof(double));
    memcpy(h->snaps, snaps, (size_t)n * sizeof(double));
    h->wet = xcalloc((size_t)ax * ay, 1);
    if (wet) memcpy(h->wet, wet, (size_t)ax * ay);
    else memset(h->wet, 1, (size_t)ax * ay);
    h->nsnap = nsnap;
    h->an[0] = ax;
    h->an[1] = ay;
    return 0;
}

/* ------------------------------------------------------------------ */
/* composite values and space-time interpolation (Sec. 3)              */
/* ------------------------------------------------------------------ */
static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return fmin(a, b);
    if (a < 0.0 && b < 0.0) return fmax(a, b);
    return 0.0;
}

/* value of field f at coarse cell (a, b) of level c, time-interpolated with
   th = k/r between the level's current and new states (k = 0: current). */
static int coarse_value(OHier *h, int c, int a, int b, int k, int r, int f, double *out)
{
    double sg[3];
    map_bc(h, c, &a, &b, sg);
    int pk = find_patch(h, c, a, b);
    if (pk < 0) {
        snprintf(h->err, sizeof h->err, "nesting violated: level %d cell (%d,%d) not covered", c, a, b);
        return 1;
    }
    const OPatch *p = &h->L[c].p[pk];
    int cur = h->L[c].cur;
    double v0 = p->q[cur][qidx(h, p, f, a - p->ilo, b - p->jlo)];
    double v;
    if (k == 0) {
        v = v0;
    } else {
        double th = (double)k / (double)r;
        double v1 = p->q[1 - cur][qidx(h, p, f, a - p->ilo, b - p->jlo)];
        v = (1.0 - th) * v0 + th * v1;
    }
    *out = sg[f] < 0.0 ? -v : v;
    return 0;
}

/* conservative piecewise-linear (minmod-limited) space interpolation from
   level l-1 at fine in-domain cell (I, J) of level l, time fraction k/r. */
static int coarse_interp(OHier *h, int l, int I, int J, int k, double *vals)
{
    int r = h->P.ratio[l - 1];
    int c = l - 1;
    int ic = I / r, jc = (h->P.dim == 2) ? J / r : 0;
    double fx = (double)(2 * (I - ic * r) + 1 - r) / (double)(2 * r);
    double fy = (h->P.dim == 2) ? (double)(2 * (J - jc * r) + 1 - r) / (double)(2 * r) : 0.0;
    for (int f = 0; f < h->m; f++) {
        double q0, qxm, qxp;
        if (coarse_value(h, c, ic, jc, k, r, f, &q0)) return 1;
        if (coarse_value(h, c, ic - 1, jc, k, r, f, &qxm)) return 1;
        if (coarse_value(h, c, ic + 1, jc, k, r, f, &qxp)) return 1;
        double sx = minmod(qxp - q0, q0 - qxm);
        double v = q0 + sx * fx;
        if (h->P.dim == 2) {
            double qym, qyp;
            if (coarse_value(h, c, ic, jc - 1, k, r, f, &qym)) return 1;
            if (coarse_value(h, c, ic, jc + 1, k, r, f, &qyp)) return 1;
            double sy = minmod(qyp - q0, q0 - qym);
            v = v + sy * fy;
        }
        vals[f] = v;
    }
    return 0;
}

/* ghost cells of every patch of level l at substep k of the coarser step */
static int fill_ghosts(OHier *h, int l, int k)
{
    OLevel *L = &h->L[l];
    int cur = L->cur;
    for (int pk = 0; pk < L->np; pk++) {
        OPatch *p = &L->p[pk];
        for (int j = -h->gy; j < p->ny + h->gy; j++)
            for (int i = -h->gx; i < p->nx + h->gx; i++) {
                if (i >= 0 && i < p->nx && j >= 0 && j < p->ny) continue;
                int I = p->ilo + i, J = p->jlo + j;
                double sg[3], v[3];
                map_bc(h, l, &I, &J, sg);
                int sk = find_patch(h, l, I, J);
                if (sk >= 0) {
                    const OPatch *s = &L->p[sk];
                    for (int f = 0; f < h->m; f++) v[f] = s->q[cur][qidx(h, s, f, I - s->ilo, J - s->jlo)];
                } else {
                    if (l == 0) {
                        snprintf(h->err, sizeof h->err, "level 0 does not cover cell (%d,%d)", I, J);
                        return 1;
                    }
                    if (coarse_interp(h, l, I, J, k, v)) return 1;
                }
                for (int f = 0; f < h->m; f++) p->q[cur][qidx(h, p, f, i, j)] = sg[f] < 0.0 ? -v[f] : v[f];
            }
    }
    return 0;
}

/* substep of level l within the current step of level l-1 (0 on level 0) */
static int level_sub(const OHier *h, int l)
{
    return l > 0 ? (int)(h->L[l].nstep - h->L[l - 1].nstep * h->P.ratio[l - 1]) : 0;
}

/* fine -> coarse: mean of the r^d children, summed row by row */
static int average_down(OHier *h, int lf)
{
    int lc = lf - 1, r = h->P.ratio[lc];
    OLevel *F = &h->L[lf], *C = &h->L[lc];
    int fcur = F->cur, cnew = 1 - C->cur;
    int rr = (h->P.dim == 2) ? r : 1;
    double inv = 1.0 / (double)(r * rr);
    for (int pk = 0; pk < F->np; pk++) {
        const OPatch *p = &F->p[pk];
        int a0 = p->ilo / r, a1 = (p->ilo + p->nx) / r;
        int b0 = (h->P.dim == 2) ? p->jlo / r : 0, b1 = (h->P.dim == 2) ? (p->jlo + p->ny) / r : 1;
        for (int b = b0; b < b1; b++)
            for (int a = a0; a < a1; a++) {
                int ck = find_patch(h, lc, a, b);
                if (ck < 0) {
                    snprintf(h->err, sizeof h->err, "average_down: coarse cell (%d,%d) not covered", a, b);
                    return 1;
                }
                OPatch *c = &C->p[ck];
                for (int f = 0; f < h->m; f++) {
                    double s = 0.0;
                    for (int jj = 0; jj < rr; jj++)
                        for (int ii = 0; ii < r; ii++) {
                            int fi = a * r + ii - p->ilo, fj = (h->P.dim == 2) ? b * r + jj - p->jlo : 0;
                            s = s + p->q[fcur][qidx(h, p, f, fi, fj)];
                        }
                    c->q[cnew][qidx(h, c, f, a - c->ilo, b - c->jlo)] = s * inv;
                }
            }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* conservation fix-up at coarse-fine interfaces (refluxing).           */
/*                                                                      */
/* The coarse step updates an uncovered coarse cell C beside a fine     */
/* patch with what it computes at the shared edge (Lc: the fluctuation */
/* plus correction flux entering C from that side).  The fine patch     */
/* meanwhile advances with ghost values interpolated from the coarse    */
/* level, so what leaves the fine side through the edge is not what C   */
/* received.  Written as fluxes of a linear conservative system f = Aq: */
/* the fine cell f beside the edge receives F_fine - f(Q_f) (its side   */
/* value "fin"), so the flux through the edge seen from the fine side   */
/* is f(Q_f) -/+ fin; C should have received the time and edge average  */
/* of that flux less f(Q_C), i.e.                                       */
/*   L* = (A-dQ + A+dQ)(Riemann problem between C and f) - fin,         */
/* with C on its own side of the problem and Q_C its value at the start */
/* of the coarse step (C's other edges telescope with that value).      */
/* After the fine substeps and the average-down,                        */
/*   Q_C <- Q_C - (dt/dx)_coarse * (mean(L*) - Lc)                      */
/* for every such side of C.  For homogeneous acoustics and for the     */
/* f-wave systems (adjoints, the surface row of shallow water) this     */
/* makes the composite sums of the conserved fields change only through */
/* the physical boundary; elsewhere it is the same consistent           */
/* correction.  Sec. 3 (AMR following Berger and LeVeque).              */
/* ------------------------------------------------------------------ */
static int opposite_side(int s) { return s ^ 1; }

static void side_neighbour(int s, int I, int J, int *nI, int *nJ)
{
    *nI = I + (s == 0 ? -1 : s == 1 ? 1 : 0);
    *nJ = J + (s == 2 ? -1 : s == 3 ? 1 : 0);
}

static void reg_clear(ORegs *R)
{
    for (int q = 0; q < R->n; q++) free(R->e[q].Lf);
    R->n = 0;
    R->active = 0;
}

static void reg_begin(OHier *h, int l)
{
    ORegs *R = &h->reg[l];
    reg_clear(R);
    int N = h->L[l].N, M = h->L[l].M, r = h->P.ratio[l];
    if (R->N != N || R->M != M) {
        free(R->idx);
        free(R->cov);
        R->idx = xcalloc((size_t)4 * N * M, sizeof(int));
        R->cov = xcalloc((size_t)N * M, 1);
        R->N = N;
        R->M = M;
    }
    for (long q = 0; q < 4L * N * M; q++) R->idx[q] = -1;
    memset(R->cov, 0, (size_t)N * M);
    const OLevel *F = &h->L[l + 1];
    for (int k = 0; k < F->np; k++) {
        const OPatch *p = &F->p[k];
        int a0 = p->ilo / r, a1 = (p->ilo + p->nx) / r;
        int b0 = (h->P.dim == 2) ? p->jlo / r : 0, b1 = (h->P.dim == 2) ? (p->jlo + p->ny) / r : 1;
        for (int b = b0; b < b1; b++)
            for (int a = a0; a < a1; a++) R->cov[(long)b * N + a] = 1;
    }
    R->active = 1;
}

/* coarse side: every uncovered cell of patch pk with a covered neighbour */
static void reg_coarse(OHier *h, int l, int pk, const double *side)
{
    ORegs *R = &h->reg[l];
    const OPatch *p = &h->L[l].p[pk];
    int N = R->N, M = R->M, ns = (h->P.dim == 2) ? 4 : 2;
    int r = h->P.ratio[l], nseg = (h->P.dim == 2) ? r : 1;
    long nc = (long)p->nx * p->ny;
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) {
            int I = p->ilo + i, J = p->jlo + j;
            if (R->cov[(long)J * N + I]) continue;
            for (int s = 0; s < ns; s++) {
                int nI, nJ;
                side_neighbour(s, I, J, &nI, &nJ);
                if (nI < 0 || nI >= N || nJ < 0 || nJ >= M) continue;
                if (!R->cov[(long)nJ * N + nI]) continue;
                if (R->n == R->cap) {
                    R->cap = R->cap ? 2 * R->cap : 256;
                    R->e = realloc(R->e, (size_t)R->cap * sizeof(OReg));
                }
                OReg *e = &R->e[R->n];
                e->pk = pk;
                e->i = i;
                e->j = j;
                e->side = s;
                for (int k = 0; k < 2; k++) e->Lc[k] = side[(long)(s * 2 + k) * nc + (long)j * p->nx + i];
                e->Lf = xcalloc((size_t)r * nseg * 2, sizeof(double));
                R->idx[((long)s * M + J) * N + I] = R->n;
                R->n++;
            }
        }
}

/* fine side: patch pk of level l (fine) at its current substep; the cells
   whose neighbour across a side is a coarse-interpolated ghost cell */
static int reg_fine(OHier *h, int l, int pk, const double *side)
{
    int c = l - 1, r = h->P.ratio[c];
    ORegs *R = &h->reg[c];
    const OLevel *L = &h->L[l], *C = &h->L[c];
    const OPatch *p = &L->p[pk];
    int ns = (h->P.dim == 2) ? 4 : 2, nseg = (h->P.dim == 2) ? r : 1;
    int sub = level_sub(h, l);
    long nc = (long)p->nx * p->ny;
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) {
            if (i > 0 && i < p->nx - 1 && (h->P.dim == 1 || (j > 0 && j < p->ny - 1))) continue;
            int I = p->ilo + i, J = p->jlo + j;
            for (int s = 0; s < ns; s++) {
                int nI, nJ;
                side_neighbour(s, I, J, &nI, &nJ);
                int li = nI - p->ilo, lj = nJ - p->jlo;
                if (li >= 0 && li < p->nx && lj >= 0 && lj < p->ny) continue;    /* inside the patch */
                if (nI < 0 || nI >= L->N || nJ < 0 || nJ >= L->M) continue;   /* physical boundary */
                if (find_patch(h, l, nI, nJ) >= 0) continue;                     /* same-level neighbour */
                int Ci = nI / r, Cj = (h->P.dim == 2) ? nJ / r : 0;
                int cs = opposite_side(s);
                int q = R->idx[((long)cs * R->M + Cj) * R->N + Ci];
                int ck = find_patch(h, c, Ci, Cj);
                if (q < 0 || ck < 0) {
                    snprintf(h->err, sizeof h->err, "reflux: no register for coarse cell (%d,%d) side %d", Ci, Cj, cs);
                    return 1;
                }
                const OPatch *cp = &C->p[ck];
                int n = (s < 2) ? 1 : 2;
                double QC0 = cp->q[C->cur][qidx(h, cp, 0, Ci - cp->ilo, Cj - cp->jlo)];
                double QCn = cp->q[C->cur][qidx(h, cp, n, Ci - cp->ilo, Cj - cp->jlo)];
                double Qf0 = p->q[L->cur][qidx(h, p, 0, i, j)];
                double Qfn = p->q[L->cur][qidx(h, p, n, i, j)];
                double mC[2], mf[2];
                for (int f = 0; f < h->nmed; f++) {
                    mC[f] = cp->med[qidx(h, cp, f, Ci - cp->ilo, Cj - cp->jlo)];
                    mf[f] = p->med[qidx(h, p, f, i, j)];
                }
                OEdgeRes er;
                if (s == 0 || s == 2) normal_solve(h->P.eqn, mC, mf, QC0, QCn, Qf0, Qfn, &er);   /* C below/left of f */
                else normal_solve(h->P.eqn, mf, mC, Qf0, Qfn, QC0, QCn, &er);                  /* C above/right of f */
                int kseg = (h->P.dim == 1) ? 0 : (s < 2 ? J - Cj * r : I - Ci * r);
                double *o = R->e[q].Lf + ((long)sub * nseg + kseg) * 2;
                for (int k = 0; k < 2; k++) {
                    double tot = er.am[k] + er.ap[k];
                    o[k] = tot - side[(long)(s * 2 + k) * nc + (long)j * p->nx + i];
                }
            }
        }
    return 0;
}

/* apply the fix-up to the new state of coarse level l (after average-down) */
static void reg_apply(OHier *h, int l)
{
    ORegs *R = &h->reg[l];
    OLevel *L = &h->L[l];
    int r = h->P.ratio[l], nseg = (h->P.dim == 2) ? r : 1;
    double w = 1.0 / (double)(r * nseg);
    double dtdx = L->dt / L->dx, dtdy = (h->P.dim == 2) ? L->dt / L->dy : 0.0;
    for (int q = 0; q < R->n; q++) {
        const OReg *e = &R->e[q];
        OPatch *p = &L->p[e->pk];
        int n = (e->side < 2) ? 1 : 2;
        double dtd = (e->side < 2) ? dtdx : dtdy;
        for (int k = 0; k < 2; k++) {
            double acc = 0.0;
            for (int sb = 0; sb < r; sb++)
                for (int g = 0; g < nseg; g++) acc = acc + e->Lf[((long)sb * nseg + g) * 2 + k];
            double *v = &p->q[1 - L->cur][qidx(h, p, k == 0 ? 0 : n, e->i, e->j)];
            *v = *v - dtd * (acc * w - e->Lc[k]);
        }
    }
    reg_clear(R);
}

static double step_level_patches(OHier *h, int l, int *err)
{
    OLevel *L = &h->L[l];
    int cur = L->cur;
    double cfl = 0.0;
    int coarse_reg = h->P.reflux && l < h->P.nlevels - 1 && h->L[l + 1].np > 0;
    int fine_reg = h->P.reflux && l > 0 && h->reg[l - 1].active;
    if (coarse_reg) reg_begin(h, l);
    for (int pk = 0; pk < L->np; pk++) {
        OPatch *p = &L->p[pk];
        double *qo = xcalloc((size_t)h->m * p->nx * p->ny, sizeof(double));
        double *side = (coarse_reg || fine_reg) ? xcalloc((size_t)8 * p->nx * p->ny, sizeof(double)) : NULL;
        double c = step_patch(h->P.dim, h->P.eqn, p->nx, p->ny, p->q[cur], p->med, L->dt, L->dx, L->dy, qo, side);
        cfl = fmax(cfl, c);
        h->cell_updates += (long long)p->nx * p->ny;
        if (coarse_reg) reg_coarse(h, l, pk, side);
        if (fine_reg && reg_fine(h, l, pk, side)) *err = 1;
        for (int f = 0; f < h->m; f++)
            for (int j = 0; j < p->ny; j++)
                for (int i = 0; i < p->nx; i++)
                    p->q[1 - cur][qidx(h, p, f, i, j)] = qo[((long)f * p->ny + j) * p->nx + i];
        free(qo);
        free(side);
    }
    return cfl;
}

/* ------------------------------------------------------------------ */
/* adjoint flagging (Sec. 4; time range: Sec. 5.1.2)                    */
/* ------------------------------------------------------------------ */
/* bilinear interpolation of snapshot n, field f, at (x, y); positions
   outside the outermost adjoint cell centres are clamped to them */
static double adj_interp(const OHier *h, int n, int f, double x, double y)
{
    int ax = h->an[0], ay = h->an[1];
    double dxa = (h->P.hi[0] - h->P.lo[0]) / (double)ax;
    double xi = (x - h->P.lo[0]) / dxa - 0.5;
    xi = fmin(fmax(xi, 0.0), (double)(ax - 1));
    int a = (int)floor(xi);
    if (a > ax - 2) a = ax - 2;
    if (a < 0) a = 0;
    double wx = xi - (double)a;
    const double *s = h->snaps + ((long)n * h->m + f) * ax * ay;
    if (h->P.dim == 1) {
        if (ax == 1) return s[0];
        return (1.0 - wx) * s[a] + wx * s[a + 1];
    }
    double dya = (h->P.hi[1] - h->P.lo[1]) / (double)ay;
    double yi = (y - h->P.lo[1]) / dya - 0.5;
    yi = fmin(fmax(yi, 0.0), (double)(ay - 1));
    int b = (int)floor(yi);
    if (b > ay - 2) b = ay - 2;
    if (b < 0) b = 0;
    double wy = yi - (double)b;
    double omx = 1.0 - wx;
    double v0 = omx * s[(long)b * ax + a] + wx * s[(long)b * ax + a + 1];
    double v1 = omx * s[(long)(b + 1) * ax + a] + wx * s[(long)(b + 1) * ax + a + 1];
    return (1.0 - wy) * v0 + wy * v1;
}

static int adj_wet(const OHier *h, double x, double y)
{
    int ax = h->an[0], ay = h->an[1];
    double dxa = (h->P.hi[0] - h->P.lo[0]) / (double)ax;
    int a = (int)floor((x - h->P.lo[0]) / dxa);
    if (a < 0) a = 0;
    if (a > ax - 1) a = ax - 1;
    int b = 0;
    if (h->P.dim == 2) {
        double dya = (h->P.hi[1] - h->P.lo[1]) / (double)ay;
        b = (int)floor((y - h->P.lo[1]) / dya);
        if (b < 0) b = 0;
        if (b > ay - 1) b = ay - 1;
    }
    return h->wet[(long)b * ax + a] != 0;
}

static double snap_time(const OHier *h, int n)
{
    double dts = (h->P.tf - h->P.t0) / (double)(h->nsnap - 1);
    return h->P.t0 + (double)n * dts;
}

/* inner product |qhat . Q| with qhat from snapshot n (dot order p, u, v) */
static double adj_dot_snap(const OHier *h, int n, double x, double y, const double *Q)
{
    double d = 0.0;
    for (int f = 0; f < h->m; f++) {
        double a = adj_interp(h, n, f, x, y);
        d = (f == 0) ? a * Q[0] : d + a * Q[f];
    }
    return fabs(d);
}

/* |qhat(tau) . Q| with qhat linear in time between bracketing snapshots */
static double adj_dot_time(const OHier *h, double tau, double x, double y, const double *Q)
{
    int S = h->nsnap;
    double dts = (h->P.tf - h->P.t0) / (double)(S - 1);
    int n = 0;
    while (n < S - 2 && snap_time(h, n + 1) <= tau) n++;
    double w = (tau - snap_time(h, n)) / dts;
    double d = 0.0;
    for (int f = 0; f < h->m; f++) {
        double a0 = adj_interp(h, n, f, x, y), a1 = adj_interp(h, n + 1, f, x, y);
        double a = (1.0 - w) * a0 + w * a1;
        d = (f == 0) ? a * Q[0] : d + a * Q[f];
    }
    return fabs(d);
}

/* ------------------------------------------------------------------ */
/* adjoint-weighted error estimate (Sec. 7: the forward solution's      */
/* pointwise error estimated by Richardson extrapolation, its effect on */
/* J by the adjoint).                                                   */
/*                                                                      */
/* For every patch of level l at the level's current time t: take the   */
/* patch extended to an even size (ne x me) with a ring of 4 cells, the */
/* values outside the patch filled as ghost cells are (same level where */
/* it has a patch, else the interpolation from level l-1 at the same    */
/* substep, boundary-mapped); advance it two steps of dt (the first     */
/* over the region widened by 2 cells, the second over the even patch); */
/* coarsen the extended patch by 2 in every direction (mean of the      */
/* children, medium included) and advance it one step of 2 dt.  With a  */
/* second-order method one fine step's local error is C dx^3 and the    */
/* coarse step's 8 C dx^3, so coarse minus (coarsened) fine after the   */
/* two is 6 C dx^3 and                                                  */
/*   tau = (coarsen(fine) - coarse) / 6 = -(local error of one step),   */
/* per component, on every 2 x 2 (1D: 2) block of the patch.  A cell   */
/* is flagged where max over the flagging window's snapshots of         */
/* |qhat . tau| exceeds the tolerance (the bracket rule of Sec. 4 with  */
/* tau in place of q).                                                  */
/* ------------------------------------------------------------------ */
/* value of level l at index (I, J) (boundary-mapped) at substep k of the
   coarser step: the level's own patch where it has one, else the
   interpolation from level l - 1, as a ghost cell gets it */
static int level_value(OHier *h, int l, int I, int J, int k, double *v)
{
    double sg[3], w[3];
    map_bc(h, l, &I, &J, sg);
    int sk = find_patch(h, l, I, J);
    if (sk >= 0) {
        const OPatch *s = &h->L[l].p[sk];
        for (int f = 0; f < h->m; f++) w[f] = s->q[h->L[l].cur][qidx(h, s, f, I - s->ilo, J - s->jlo)];
    } else {
        if (l == 0) {
            snprintf(h->err, sizeof h->err, "level 0 does not cover cell (%d,%d)", I, J);
            return 1;
        }
        if (coarse_interp(h, l, I, J, k, w)) return 1;
    }
    for (int f = 0; f < h->m; f++) v[f] = sg[f] < 0.0 ? -w[f] : w[f];
    return 0;
}

/* mean of the 2 x 2 (1D: 2) children of every cell of a coarsened array:
   src [nf][sy][sx] -> dst [nf][sy/2][sx/2] (1D: sy = 1 stays 1), children
   summed row by row */
static void coarsen2(int dim, int nf, int sx, int sy, const double *src, double *dst)
{
    int cx = sx / 2, cy = (dim == 2) ? sy / 2 : 1, rr = (dim == 2) ? 2 : 1;
    double inv = 1.0 / (double)(2 * rr);
    for (int f = 0; f < nf; f++)
        for (int b = 0; b < cy; b++)
            for (int a = 0; a < cx; a++) {
                double s = 0.0;
                for (int jj = 0; jj < rr; jj++)
                    for (int ii = 0; ii < 2; ii++) s = s + src[((long)f * sy + b * rr + jj) * sx + 2 * a + ii];
                dst[((long)f * cy + b) * cx + a] = s * inv;
            }
}

static int error_estimate(OHier *h, int l)
{
    OLevel *L = &h->L[l];
    const int dim = h->P.dim, eqn = h->P.eqn, m = h->m, nmed = h->nmed;
    const int k = level_sub(h, l);
    long n = 0;
    for (int pk = 0; pk < L->np; pk++) n += (long)L->p[pk].nx * L->p[pk].ny;
    free(h->tau);
    h->tau = xcalloc((size_t)(n > 0 ? n : 1) * m, sizeof(double));
    h->ntau = n;
    long o = 0;
    for (int pk = 0; pk < L->np; pk++) {
        const OPatch *p = &L->p[pk];
        const int ne = p->nx + (p->nx & 1), me = (dim == 2) ? p->ny + (p->ny & 1) : 1;
        const int g = (dim == 2) ? 4 : 0;
        const int ex = ne + 8, ey = me + 2 * g;
        double *E = xcalloc((size_t)m * ex * ey, sizeof(double));
        double *EM = xcalloc((size_t)nmed * ex * ey, sizeof(double));
        for (int sj = 0; sj < ey; sj++)
            for (int si = 0; si < ex; si++) {
                int I = p->ilo + si - 4, J = p->jlo + sj - g;
                double v[3], sg[3], md[2];
                if (level_value(h, l, I, J, k, v)) {
                    free(E);
                    free(EM);
                    return 1;
                }
                for (int f = 0; f < m; f++) E[((long)f * ey + sj) * ex + si] = v[f];
                map_bc(h, l, &I, &J, sg);
                medium_at(h, l, I, J, md);
                for (int f = 0; f < nmed; f++) EM[((long)f * ey + sj) * ex + si] = md[f];
            }
        /* fine: two steps of dt */
        const int f1x = ne + 4, f1y = (dim == 2) ? me + 4 : 1;
        double *F1 = xcalloc((size_t)m * f1x * f1y, sizeof(double));
        step_patch(dim, eqn, f1x, f1y, E, EM, L->dt, L->dx, L->dy, F1, NULL);
        double *M1 = xcalloc((size_t)nmed * f1x * f1y, sizeof(double));
        for (int f = 0; f < nmed; f++)
            for (int j = 0; j < f1y; j++)
                for (int i = 0; i < f1x; i++)
                    M1[((long)f * f1y + j) * f1x + i] = EM[((long)f * ey + j + (g ? 2 : 0)) * ex + i + 2];
        double *F2 = xcalloc((size_t)m * ne * me, sizeof(double));
        step_patch(dim, eqn, ne, me, F1, M1, L->dt, L->dx, L->dy, F2, NULL);
        /* coarse: one step of 2 dt on the extended patch coarsened by 2 */
        const int cx = ex / 2, cy = (dim == 2) ? ey / 2 : 1;
        double *C = xcalloc((size_t)m * cx * cy, sizeof(double));
        double *CM = xcalloc((size_t)nmed * cx * cy, sizeof(double));
        coarsen2(dim, m, ex, ey, E, C);
        coarsen2(dim, nmed, ex, ey, EM, CM);
        const int nc = ne / 2, mc = (dim == 2) ? me / 2 : 1;
        double *C1 = xcalloc((size_t)m * nc * mc, sizeof(double));
        step_patch(dim, eqn, nc, mc, C, CM, 2.0 * L->dt, 2.0 * L->dx, 2.0 * L->dy, C1, NULL);
        double *FC = xcalloc((size_t)m * nc * mc, sizeof(double));
        coarsen2(dim, m, ne, me, F2, FC);
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                int a = i / 2, b = (dim == 2) ? j / 2 : 0;
                for (int f = 0; f < m; f++) {
                    long c = ((long)f * mc + b) * nc + a;
                    h->tau[(o + (long)j * p->nx + i) * m + f] = (FC[c] - C1[c]) / 6.0;
                }
            }
        o += (long)p->nx * p->ny;
        free(E);
        free(EM);
        free(F1);
        free(M1);
        free(F2);
        free(C);
        free(CM);
        free(C1);
        free(FC);
    }
    return 0;
}

/* exported: the error estimate of level l at its current time, laid out as
   orc_read_level lays out the state (per patch [m][ny][nx], patches in
   order); n = capacity in doubles; returns 0, or 1 on error */
int orc_error_estimate(void *hv, int level, double *tau_out, long n)
{
    OHier *h = hv;
    if (level < 0 || level >= h->P.nlevels) return 1;
    if (error_estimate(h, level)) return 1;
    if (n < h->ntau * h->m) return 1;
    long o = 0, c = 0;
    for (int pk = 0; pk < h->L[level].np; pk++) {
        const OPatch *p = &h->L[level].p[pk];
        long np = (long)p->nx * p->ny;
        for (int f = 0; f < h->m; f++)
            for (long e = 0; e < np; e++) tau_out[o++] = h->tau[(c + e) * h->m + f];
        c += np;
    }
    return 0;
}

/* flags of the interior cells of level l at its current time, in patch
   order, row-major within a patch.  Window: tau in [t, T],
   T = min(t + tf - ts, tf); value = max over the window of |qhat . q|. */
static long flag_level(OHier *h, int l, double tol, unsigned char *flags)
{
    OLevel *L = &h->L[l];
    double t = level_time(h, l);
    double T = fmin(t + (h->P.tf - h->P.ts), h->P.tf);
    int S = h->nsnap;
    int nlo = 0, nhi = S - 1;
    for (int n = 0; n < S; n++)
        if (snap_time(h, n) <= t) nlo = n;
    for (int n = S - 1; n >= 0; n--)
        if (snap_time(h, n) >= T) nhi = n;
    long cnt = 0, o = 0;
    for (int pk = 0; pk < L->np; pk++) {
        const OPatch *p = &L->p[pk];
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                double x = h->P.lo[0] + ((double)(p->ilo + i) + 0.5) * L->dx;
                double y = (h->P.dim == 2) ? h->P.lo[1] + ((double)(p->jlo + j) + 0.5) * L->dy : 0.0;
                double Q[3];
                for (int f = 0; f < h->m; f++) Q[f] = p->q[L->cur][qidx(h, p, f, i, j)];
                double val = 0.0;
                if (h->P.flag_mode == O_DIFF) {
                    /* undivided centred difference of every component in
                       every direction, from the ghost-filled patch */
                    const double *qq = p->q[L->cur];
                    for (int f = 0; f < h->m; f++) {
                        val = fmax(val, fabs(qq[qidx(h, p, f, i + 1, j)] - qq[qidx(h, p, f, i - 1, j)]));
                        if (h->P.dim == 2)
                            val = fmax(val, fabs(qq[qidx(h, p, f, i, j + 1)] - qq[qidx(h, p, f, i, j - 1)]));
                    }
                } else if (h->P.flag_mode == O_SURFACE) {
                    val = fabs(Q[0]);  /* perturbation of the surface (first component) */
                } else if (h->P.flag_mode == O_RICHARDSON) {
                    /* the standard Richardson flagger (Sec. 1): the error estimate
                       itself, largest component */
                    for (int f = 0; f < h->m; f++) val = fmax(val, fabs(h->tau[o * h->m + f]));
                } else if (S >= 2 && h->snaps) {
                    if (h->P.flag_mode == O_ERROR) {
                        const double *tq = &h->tau[o * h->m];
                        for (int n = nlo; n <= nhi; n++) val = fmax(val, adj_dot_snap(h, n, x, y, tq));
                    } else if (h->P.flag_mode == O_BRACKET) {
                        for (int n = nlo; n <= nhi; n++) val = fmax(val, adj_dot_snap(h, n, x, y, Q));
                    } else {
                        val = fmax(adj_dot_time(h, t, x, y, Q), adj_dot_time(h, T, x, y, Q));
                        for (int n = 0; n < S; n++) {
                            double tn = snap_time(h, n);
                            if (tn > t && tn < T) val = fmax(val, adj_dot_snap(h, n, x, y, Q));
                        }
                    }
                    if (!adj_wet(h, x, y)) val = 0.0;
                }
                unsigned char fl = (val > tol) ? 1 : 0;
                flags[o++] = fl;
                cnt += fl;
            }
    }
    return cnt;
}

int orc_flag(void *hv, int level, double tol, unsigned char *flags, long *nflag)
{
    OHier *h = hv;
    if (level < 0 || level >= h->P.nlevels) return 1;
    if (h->P.flag_mode == O_DIFF && fill_ghosts(h, level, level_sub(h, level))) return 1;
    if ((h->P.flag_mode == O_ERROR || h->P.flag_mode == O_RICHARDSON) && error_estimate(h, level)) return 1;
    long c = flag_level(h, level, tol, flags);
    if (nflag) *nflag = c;
    return 0;
}

/* ------------------------------------------------------------------ */
/* clustering: Berger-Rigoutsos on a dense flag bitmap (Sec. 3)         */
/* ------------------------------------------------------------------ */
typedef struct { int i0, i1, j0, j1; } OBox;
typedef struct {
    OBox *b;
    int n, cap;
} OBoxList;

static void box_push(OBoxList *L, OBox b)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->b = realloc(L->b, (size_t)L->cap * sizeof(OBox));
    }
    L->b[L->n++] = b;
}

typedef struct {
    const unsigned char *flag, *nest;
    int N, M, dim, mc;
    double eff;
} OBR;

static void br(const OBR *c, OBox b, OBoxList *out)
{
    /* shrink to the bounding box of the flags inside b */
    int i0 = b.i1 + 1, i1 = b.i0 - 1, j0 = b.j1 + 1, j1 = b.j0 - 1;
    long nf = 0;
    for (int j = b.j0; j <= b.j1; j++)
        for (int i = b.i0; i <= b.i1; i++)
            if (c->flag[(long)j * c->N + i]) {
                nf++;
                if (i < i0) i0 = i;
                if (i > i1) i1 = i;
                if (j < j0) j0 = j;
                if (j > j1) j1 = j;
            }
    if (nf == 0) return;
    b.i0 = i0; b.i1 = i1; b.j0 = j0; b.j1 = j1;
    int lx = i1 - i0 + 1, ly = j1 - j0 + 1;
    long area = (long)lx * ly;
    int nestable = 1;
    for (int j = j0; j <= j1 && nestable; j++)
        for (int i = i0; i <= i1; i++)
            if (!c->nest[(long)j * c->N + i]) { nestable = 0; break; }
    double eff = (double)nf / (double)area;
    if (nestable && eff >= c->eff) { box_push(out, b); return; }
    int mc = nestable ? c->mc : 1;
    /* signatures */
    long *sx = xcalloc(lx, sizeof(long)), *sy = xcalloc(ly, sizeof(long));
    for (int j = j0; j <= j1; j++)
        for (int i = i0; i <= i1; i++)
            if (c->flag[(long)j * c->N + i]) { sx[i - i0]++; sy[j - j0]++; }
    int dims = (c->dim == 2) ? 2 : 1;
    /* 1. a hole (zero signature) closest to the centre; ties: x, then lower index */
    int bd = -1, bpos = 0, bdist = 0;
    for (int d = 0; d < dims; d++) {
        int lo = d ? j0 : i0, hi = d ? j1 : i1;
        long *s = d ? sy : sx;
        for (int k = lo + 1; k < hi; k++)
            if (s[k - lo] == 0) {
                int dist = abs(2 * k - (lo + hi));
                if (bd < 0 || dist < bdist) { bd = d; bpos = k; bdist = dist; }
            }
    }
    OBox L, R;
    int have = 0;
    if (bd >= 0) {
        L = b; R = b;
        if (bd == 0) { L.i1 = bpos - 1; R.i0 = bpos + 1; }
        else { L.j1 = bpos - 1; R.j0 = bpos + 1; }
        have = 1;
    }
    /* 2. the strongest sign change of the signature's second difference;
          split between k and k+1; ties: closer to centre, x, lower index */
    if (!have) {
        long bstr = -1;
        for (int d = 0; d < dims; d++) {
            int lo = d ? j0 : i0, hi = d ? j1 : i1;
            long *s = d ? sy : sx;
            for (int k = lo + 1; k + 1 <= hi - 1; k++) {
                long l0 = s[k - 1 - lo] - 2 * s[k - lo] + s[k + 1 - lo];
                long l1 = s[k - lo] - 2 * s[k + 1 - lo] + s[k + 2 - lo];
                if (!((l0 < 0 && l1 > 0) || (l0 > 0 && l1 < 0))) continue;
                if (k - lo + 1 < mc || hi - k < mc) continue;
                long str = labs(l1 - l0);
                int dist = abs(2 * k + 1 - (lo + hi));
                if (str > bstr || (str == bstr && dist < bdist)) {
                    bstr = str; bdist = dist; bd = d; bpos = k;
                }
            }
        }
        if (bd >= 0) {
            L = b; R = b;
            if (bd == 0) { L.i1 = bpos; R.i0 = bpos + 1; }
            else { L.j1 = bpos; R.j0 = bpos + 1; }
            have = 1;
        }
    }
    /* 3. bisect the longer side (ties: x), else the other side */
    if (!have) {
        int order[2] = {0, 1};
        if (dims == 2 && ly > lx) { order[0] = 1; order[1] = 0; }
        for (int q = 0; q < dims && !have; q++) {
            int d = order[q];
            int len = d ? ly : lx, lo = d ? j0 : i0;
            if (len / 2 < mc || len - len / 2 < mc) continue;
            int mid = lo + len / 2;
            L = b; R = b;
            if (d == 0) { L.i1 = mid - 1; R.i0 = mid; }
            else { L.j1 = mid - 1; R.j0 = mid; }
            have = 1;
        }
    }
    free(sx);
    free(sy);
    if (!have) { box_push(out, b); return; }
    br(c, L, out);
    br(c, R, out);
}

static int cmp_box(const void *a, const void *b)
{
    const OBox *x = a, *y = b;
    if (x->j0 != y->j0) return x->j0 < y->j0 ? -1 : 1;
    if (x->i0 != y->i0) return x->i0 < y->i0 ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* regrid: flag -> buffer -> nest -> cluster -> split -> new patches    */
/* ------------------------------------------------------------------ */
static int init_new_patch(OHier *h, int l, OPatch *np, const OLevel *old, int init)
{
    int cur = 0;
    (void)cur;
    if (init && h->P.qinit) {
        int n = np->nx * np->ny;
        double *xc = xcalloc(n, sizeof(double)), *yc = xcalloc(n, sizeof(double));
        double *qv = xcalloc((size_t)n * h->m, sizeof(double));
        for (int j = 0; j < np->ny; j++)
            for (int i = 0; i < np->nx; i++) {
                xc[j * np->nx + i] = h->P.lo[0] + ((double)(np->ilo + i) + 0.5) * h->L[l].dx;
                yc[j * np->nx + i] = (h->P.dim == 2) ? h->P.lo[1] + ((double)(np->jlo + j) + 0.5) * h->L[l].dy : 0.0;
            }
        h->P.qinit(l, n, xc, yc, qv, h->P.qinit_user);
        for (int f = 0; f < h->m; f++)
            for (int j = 0; j < np->ny; j++)
                for (int i = 0; i < np->nx; i++) np->q[0][qidx(h, np, f, i, j)] = qv[(long)f * n + j * np->nx + i];
        free(xc);
        free(yc);
        free(qv);
        return 0;
    }
    for (int j = 0; j < np->ny; j++)
        for (int i = 0; i < np->nx; i++) {
            int I = np->ilo + i, J = np->jlo + j;
            int ok = -1;
            for (int k = 0; k < old->np; k++) {
                const OPatch *p = &old->p[k];
                if (I >= p->ilo && I < p->ilo + p->nx && J >= p->jlo && J < p->jlo + p->ny) { ok = k; break; }
            }
            if (ok >= 0) {
                const OPatch *p = &old->p[ok];
                for (int f = 0; f < h->m; f++) np->q[0][qidx(h, np, f, i, j)] = p->q[old->cur][qidx(h, p, f, I - p->ilo, J - p->jlo)];
            } else {
                double v[3];
                if (coarse_interp(h, l, I, J, 0, v)) return 1;
                for (int f = 0; f < h->m; f++) np->q[0][qidx(h, np, f, i, j)] = v[f];
            }
        }
    return 0;
}

static int regrid_from(OHier *h, int l, int init)
{
    for (int lev = l; lev < h->P.nlevels - 1; lev++) {
        OLevel *C = &h->L[lev], *F = &h->L[lev + 1];
        int r = h->P.ratio[lev];
        int N = C->N, M = C->M, dim = h->P.dim;
        long tick = C->nstep * h->T[lev];
        /* flags on the level index space */
        long ncell = 0;
        for (int k = 0; k < C->np; k++) ncell += (long)C->p[k].nx * C->p[k].ny;
        unsigned char *pf = xcalloc(ncell, 1);
        if ((h->P.flag_mode == O_DIFF && fill_ghosts(h, lev, level_sub(h, lev))) ||
            ((h->P.flag_mode == O_ERROR || h->P.flag_mode == O_RICHARDSON) && error_estimate(h, lev))) {
            free(pf);
            return 1;
        }
        flag_level(h, lev, h->P.tol, pf);
        unsigned char *fl = xcalloc((size_t)N * M, 1);
        unsigned char *cov = xcalloc((size_t)N * M, 1);
        long o = 0;
        for (int k = 0; k < C->np; k++) {
            const OPatch *p = &C->p[k];
            for (int j = 0; j < p->ny; j++)
                for (int i = 0; i < p->nx; i++) {
                    fl[(long)(p->jlo + j) * N + p->ilo + i] = pf[o++];
                    cov[(long)(p->jlo + j) * N + p->ilo + i] = 1;
                }
        }
        free(pf);
        /* buffer: dilate by b cells (Chebyshev), clipped to the domain */
        int bw = h->P.buffer, bwy = (dim == 2) ? bw : 0;
        unsigned char *fb = xcalloc((size_t)N * M, 1);
        for (int j = 0; j < M; j++)
            for (int i = 0; i < N; i++) {
                if (!fl[(long)j * N + i]) continue;
                for (int jj = j - bwy; jj <= j + bwy; jj++)
                    for (int ii = i - bw; ii <= i + bw; ii++)
                        if (ii >= 0 && ii < N && jj >= 0 && jj < M) fb[(long)jj * N + ii] = 1;
            }
        /* proper nesting: a cell may be refined only if every cell within
           nw cells of it is covered by this level (outside the domain counts
           as covered): nw = 2 for the ghost ring of 2 fine cells; the error
           estimate's ring of 4 fine cells takes nw = ceil(4 / r) + 1 (3 for
           r = 2, 3), so that its interpolation stencils stay on this level */
        unsigned char *nest = xcalloc((size_t)N * M, 1);
        int nw = 2;
        if ((h->P.flag_mode == O_ERROR || h->P.flag_mode == O_RICHARDSON) && (4 + r - 1) / r + 1 > nw)
            nw = (4 + r - 1) / r + 1;
        int nwy = (dim == 2) ? nw : 0;
        for (int j = 0; j < M; j++)
            for (int i = 0; i < N; i++) {
                int ok = 1;
                for (int jj = j - nwy; jj <= j + nwy && ok; jj++)
                    for (int ii = i - nw; ii <= i + nw; ii++) {
                        if (ii < 0 || ii >= N || jj < 0 || jj >= M) continue;
                        if (!cov[(long)jj * N + ii]) { ok = 0; break; }
                    }
                nest[(long)j * N + i] = (unsigned char)ok;
                if (!ok) fb[(long)j * N + i] = 0;
            }
        OBR c = {fb, nest, N, M, dim, (h->P.min_patch + r - 1) / r, h->P.cluster_eff};
        OBoxList boxes = {0};
        OBox all = {0, N - 1, 0, M - 1};
        br(&c, all, &boxes);
        /* split boxes whose refinement exceeds max_patch into near-equal parts */
        OBoxList fin = {0};
        for (int q = 0; q < boxes.n; q++) {
            OBox b = boxes.b[q];
            int lx = b.i1 - b.i0 + 1, ly = b.j1 - b.j0 + 1;
            int px = 1, py = 1;
            while (r * ((lx + px - 1) / px) > h->P.max_patch) px++;
            if (dim == 2)
                while (r * ((ly + py - 1) / py) > h->P.max_patch) py++;
            for (int bj = 0; bj < py; bj++)
                for (int bi = 0; bi < px; bi++) {
                    OBox s;
                    s.i0 = b.i0 + part_off(lx, px, bi);
                    s.i1 = s.i0 + part_len(lx, px, bi) - 1;
                    s.j0 = (dim == 2) ? b.j0 + part_off(ly, py, bj) : 0;
                    s.j1 = (dim == 2) ? s.j0 + part_len(ly, py, bj) - 1 : 0;
                    box_push(&fin, s);
                }
        }
        free(boxes.b);
        qsort(fin.b, fin.n, sizeof(OBox), cmp_box);
        /* build the new level lev+1 */
        OLevel old = *F;
        OPatch *np = xcalloc(fin.n ? fin.n : 1, sizeof(OPatch));
        for (int q = 0; q < fin.n; q++) {
            OPatch *p = &np[q];
            p->ilo = fin.b[q].i0 * r;
            p->nx = (fin.b[q].i1 - fin.b[q].i0 + 1) * r;
            p->jlo = (dim == 2) ? fin.b[q].j0 * r : 0;
            p->ny = (dim == 2) ? (fin.b[q].j1 - fin.b[q].j0 + 1) * r : 1;
            alloc_patch(h, p);
            fill_patch_medium(h, lev + 1, p);
        }
        int rc = 0;
        for (int q = 0; q < fin.n && !rc; q++) rc = init_new_patch(h, lev + 1, &np[q], &old, init);
        for (int k = 0; k < old.np; k++) free_patch(&old.p[k]);
        free(old.p);
        F->p = np;
        F->np = fin.n;
        F->cur = 0;
        F->nstep = C->nstep * r;
        h->rebuilt_tick[lev + 1] = tick;
        free(fin.b);
        free(fl);
        free(cov);
        free(fb);
        free(nest);
        if (rc) return rc;
        if (F->np == 0) {
            for (int q = lev + 2; q < h->P.nlevels; q++) {
                for (int k = 0; k < h->L[q].np; k++) free_patch(&h->L[q].p[k]);
                free(h->L[q].p);
                h->L[q].p = NULL;
                h->L[q].np = 0;
            }
            break;
        }
    }
    return 0;
}

/* exported for tests: replace the patches of `level` by the given boxes
   ([np][4] = ilo, jlo, nx, ny on the level's index space), state zero,
   medium filled as a regrid fills it (checks of another implementation's
   ghost cells and coefficients on its own layout) */
int orc_set_layout(void *hv, int level, int np, const int *boxes)
{
    OHier *h = hv;
    if (level < 0 || level >= h->P.nlevels || np < 0) return 1;
    OLevel *L = &h->L[level];
    for (int k = 0; k < L->np; k++) free_patch(&L->p[k]);
    free(L->p);
    L->p = xcalloc(np ? np : 1, sizeof(OPatch));
    L->np = np;
    L->cur = 0;
    for (int k = 0; k < np; k++) {
        OPatch *p = &L->p[k];
        p->ilo = boxes[4 * k + 0];
        p->jlo = boxes[4 * k + 1];
        p->nx = boxes[4 * k + 2];
        p->ny = boxes[4 * k + 3];
        if (p->nx < 1 || p->ny < 1 || p->ilo < 0 || p->jlo < 0 || p->ilo + p->nx > L->N || p->jlo + p->ny > L->M)
            return 1;
        alloc_patch(h, p);
        fill_patch_medium(h, level, p);
    }
    return 0;
}

/* exported: set the step counter of a level (its time t0 + nstep * dt) */
int orc_set_nstep(void *hv, int level, long nstep)
{
    OHier *h = hv;
    if (level < 0 || level >= h->P.nlevels || nstep < 0) return 1;
    h->L[level].nstep = nstep;
    return 0;
}

int orc_regrid(void *hv, int level, int init)
{
    OHier *h = hv;
    if (level < 0 || level >= h->P.nlevels) return 1;
    return regrid_from(h, level, init);
}

/* ------------------------------------------------------------------ */
/* Berger-Oliger time stepping (Sec. 3): coarse first, then r fine     */
/* steps with ghost cells interpolated in time, then average down.     */
/* ------------------------------------------------------------------ */
static int step_level(OHier *h, int l, double *cflmax)
{
    OLevel *L = &h->L[l];
    int k = h->P.regrid_interval;
    if (l < h->P.nlevels - 1 && k > 0 && L->nstep > 0 && L->nstep % k == 0 &&
        h->rebuilt_tick[l + 1] != L->nstep * h->T[l]) {
        if (regrid_from(h, l, 0)) return 1;
    }
    int sub = 0;
    if (l > 0) sub = (int)(L->nstep - h->L[l - 1].nstep * h->P.ratio[l - 1]);
    if (fill_ghosts(h, l, sub)) return 1;
    int err = 0;
    double c = step_level_patches(h, l, &err);
    if (err) return 1;
    *cflmax = fmax(*cflmax, c);
    if (l < h->P.nlevels - 1 && h->L[l + 1].np > 0) {
        int r = h->P.ratio[l];
        h->L[l + 1].nstep = L->nstep * r;
        for (int s = 0; s < r; s++)
            if (step_level(h, l + 1, cflmax)) return 1;
        if (average_down(h, l + 1)) return 1;
        if (h->reg[l].active) reg_apply(h, l);
    }
    L->cur = 1 - L->cur;
    L->nstep++;
    return 0;
}

/* advance the hierarchy by nsteps coarse steps; returns 0, or 1 on error,
   or 2 if the CFL number exceeded cfl_max */
/* gauge record at the current level-0 time: for every gauge, the cell that
   holds the point on the finest level covering it (cell index floor((x -
   lo)/dx), clamped to the level) */
static void record_gauges(OHier *h)
{
    if (h->ngauge == 0) return;
    const int w = 1 + h->m;
    if (h->ngrec == h->gcap) {
        h->gcap = h->gcap ? 2 * h->gcap : 64;
        h->grec = realloc(h->grec, (size_t)h->gcap * h->ngauge * w * sizeof(double));
    }
    double *rec = h->grec + (size_t)h->ngrec * h->ngauge * w;
    for (int g = 0; g < h->ngauge; g++) {
        double *o = rec + (size_t)g * w;
        o[0] = level_time(h, 0);
        for (int f = 0; f < h->m; f++) o[1 + f] = 0.0;
        for (int l = h->P.nlevels - 1; l >= 0; l--) {
            const OLevel *L = &h->L[l];
            if (L->np == 0) continue;
            int I = (int)floor((h->gxs[g] - h->P.lo[0]) / L->dx);
            if (I < 0) I = 0;
            if (I > L->N - 1) I = L->N - 1;
            int J = 0;
            if (h->P.dim == 2) {
                J = (int)floor((h->gys[g] - h->P.lo[1]) / L->dy);
                if (J < 0) J = 0;
                if (J > L->M - 1) J = L->M - 1;
            }
            int k = find_patch(h, l, I, J);
            if (k < 0) continue;
            const OPatch *p = &L->p[k];
            for (int f = 0; f < h->m; f++) o[1 + f] = p->q[L->cur][qidx(h, p, f, I - p->ilo, J - p->jlo)];
            break;
        }
    }
    h->ngrec++;
}

int orc_set_gauges(void *hv, int n, const double *x, const double *y)
{
    OHier *h = hv;
    if (n < 0) return 1;
    free(h->gxs);
    free(h->gys);
    free(h->grec);
    h->gxs = n ? xcalloc((size_t)n, sizeof(double)) : NULL;
    h->gys = n ? xcalloc((size_t)n, sizeof(double)) : NULL;
    for (int g = 0; g < n; g++) {
        h->gxs[g] = x[g];
        h->gys[g] = (h->P.dim == 2) ? y[g] : 0.0;
    }
    h->ngauge = n;
    h->grec = NULL;
    h->ngrec = h->gcap = 0;
    return 0;
}

/* records so far (each ngauge x (1 + m) doubles); copies at most cap */
long orc_read_gauges(void *hv, double *out, long cap)
{
    OHier *h = hv;
    long n = h->ngrec < cap ? h->ngrec : cap;
    if (n > 0) memcpy(out, h->grec, (size_t)n * h->ngauge * (1 + h->m) * sizeof(double));
    return h->ngrec;
}

int orc_advance(void *hv, int nsteps, double *cfl_out)
{
    OHier *h = hv;
    double cfl = 0.0;
    for (int s = 0; s < nsteps; s++) {
        if (step_level(h, 0, &cfl)) return 1;
        record_gauges(h);
    }
    if (cfl_out) *cfl_out = cfl;
    return cfl > h->P.cfl_max ? 2 : 0;
}

/* ------------------------------------------------------------------ */
/* queries                                                             */
/* ------------------------------------------------------------------ */
int orc_npatches(void *hv, int level) { return ((OHier *)hv)->L[level].np; }

int orc_get_patches(void *hv, int level, int *boxes /* [np][4]: ilo, jlo, nx, ny */)
{
    OHier *h = hv;
    for (int k = 0; k < h->L[level].np; k++) {
        const OPatch *p = &h->L[level].p[k];
        boxes[4 * k + 0] = p->ilo;
        boxes[4 * k + 1] = p->jlo;
        boxes[4 * k + 2] = p->nx;
        boxes[4 * k + 3] = p->ny;
    }
    return h->L[level].np;
}

double orc_level_dt(void *hv, int level) { return ((OHier *)hv)->L[level].dt; }
long long orc_cell_updates(void *hv) { return ((OHier *)hv)->cell_updates; }
long orc_level_nstep(void *hv, int level) { return ((OHier *)hv)->L[level].nstep; }
const char *orc_error(void *hv) { return ((OHier *)hv)->err; }

/* interior data of level l, patch by patch, field-major within a patch */
long orc_read_level(void *hv, int level, double *dst)
{
    OHier *h = hv;
    const OLevel *L = &h->L[level];
    long o = 0;
    for (int k = 0; k < L->np; k++) {
        const OPatch *p = &L->p[k];
        for (int f = 0; f < h->m; f++)
            for (int j = 0; j < p->ny; j++)
                for (int i = 0; i < p->nx; i++) dst[o++] = p->q[L->cur][qidx(h, p, f, i, j)];
    }
    return o;
}

long orc_write_level(void *hv, int level, const double *src)
{
    OHier *h = hv;
    OLevel *L = &h->L[level];
    long o = 0;
    for (int k = 0; k < L->np; k++) {
        OPatch *p = &L->p[k];
        for (int f = 0; f < h->m; f++)
            for (int j = 0; j < p->ny; j++)
                for (int i = 0; i < p->nx; i++) p->q[L->cur][qidx(h, p, f, i, j)] = src[o++];
    }
    return o;
}

/* ghosted storage of one patch (current state), field-major, then medium */
long orc_read_patch_ghosted(void *hv, int level, int k, double *q, double *med)
{
    OHier *h = hv;
    const OLevel *L = &h->L[level];
    const OPatch *p = &L->p[k];
    long n = (long)sxof(h, p) * syof(h, p);
    if (q) memcpy(q, p->q[L->cur], (size_t)n * h->m * sizeof(double));
    if (med) memcpy(med, p->med, (size_t)n * h->nmed * sizeof(double));
    return n;
}

int orc_fill_ghosts(void *hv, int level)
{
    OHier *h = hv;
    int sub = 0;
    if (level > 0) sub = (int)(h->L[level].nstep - h->L[level - 1].nstep * h->P.ratio[level - 1]);
    return fill_ghosts(h, level, sub);
}

/* pairwise sum: repeatedly add neighbours (2i, 2i+1); an odd tail element
   is carried up unchanged */
static double pairwise_sum(double *a, long n)
{
    if (n == 0) return 0.0;
    while (n > 1) {
        long h = n / 2;
        for (long i = 0; i < h; i++) a[i] = a[2 * i] + a[2 * i + 1];
        if (n & 1) a[h] = a[n - 1];
        n = (n + 1) / 2;
    }
    return a[0];
}

/* J = sum over the composite grid (finest level covering each point) of
   weight * q0 * |cell ∩ box|  (Eq. eq:J_general with phi = weight * I_box
   on field 0); contributions in (level, patch, j, i) order, pairwise sum. */
double orc_functional(void *hv, double x0, double x1, double y0, double y1, double weight)
{
    OHier *h = hv;
    long cap = 1024, n = 0;
    double *c = xcalloc(cap, sizeof(double));
    for (int l = 0; l < h->P.nlevels; l++) {
        const OLevel *L = &h->L[l];
        if (L->np == 0) break;
        int r = (l < h->P.nlevels - 1) ? h->P.ratio[l] : 1;
        const OLevel *Fn = (l < h->P.nlevels - 1) ? &h->L[l + 1] : NULL;
        for (int k = 0; k < L->np; k++) {
            const OPatch *p = &L->p[k];
            for (int j = 0; j < p->ny; j++)
                for (int i = 0; i < p->nx; i++) {
                    int I = p->ilo + i, J = p->jlo + j;
                    double xl = h->P.lo[0] + (double)I * L->dx, xr = h->P.lo[0] + (double)(I + 1) * L->dx;
                    double ox = fmin(xr, x1) - fmax(xl, x0);
                    if (!(ox > 0.0)) continue;
                    double area = ox;
                    if (h->P.dim == 2) {
                        double yl = h->P.lo[1] + (double)J * L->dy, yr = h->P.lo[1] + (double)(J + 1) * L->dy;
                        double oy = fmin(yr, y1) - fmax(yl, y0);
                        if (!(oy > 0.0)) continue;
                        area = ox * oy;
                    }
                    if (Fn && Fn->np > 0) {
                        int covered = 0;
                        int FI = I * r, FJ = (h->P.dim == 2) ? J * r : 0;
                        for (int q = 0; q < Fn->np && !covered; q++) {
                            const OPatch *f = &Fn->p[q];
                            if (FI >= f->ilo && FI < f->ilo + f->nx && FJ >= f->jlo && FJ < f->jlo + f->ny) covered = 1;
                        }
                        if (covered) continue;
                    }
                    if (n == cap) {
                        cap *= 2;
                        c = realloc(c, (size_t)cap * sizeof(double));
                    }
                    c[n++] = weight * (p->q[L->cur][qidx(h, p, 0, i, j)] * area);
                }
        }
    }
    double J = pairwise_sum(c, n);
    free(c);
    return J;
}

/* ------------------------------------------------------------------ */
/* adjoint solve (Sec. 4): q~_t - (A^T q~)_x = 0 forward in time from  */
/* q~(x, 0) = phi on one fixed grid; snapshots at t_f - t_n stored in   */
/* forward time order.                                                 */
/* ------------------------------------------------------------------ */
/* P describes the adjoint grid (nlevels = 1, eqn = adjoint variant).
   medium: layered (axis, nl, iface, f0, f1) when dense == NULL, else dense
   [nmed][ny][nx].  phi: [m][ny][nx].  snaps out: [nsnap][m][ny][nx]. */
int orc_adjoint_solve(const orc_params *P, int axis, int nl, const double *iface, const double *f0,
                      const double *f1, const double *dense, const double *phi, int nsnap, double *snaps)
{
    orc_params Q = *P;
    Q.nlevels = 1;
    Q.qinit = NULL;
    Q.dt0 = 1.0;
    OHier *h = orc_create(&Q);
    if (!h) return 1;
    if (dense) orc_set_medium_dense(h, 0, dense);
    else orc_set_medium_layered(h, axis, nl, iface, f0, f1);
    OLevel *L = &h->L[0];
    int nx = L->N, ny = L->M;
    double dmin = (P->dim == 2) ? fmin(L->dx, L->dy) : L->dx;
    double dts = (P->tf - P->t0) / (double)(nsnap - 1);
    double dtc = P->cfl * dmin / P->cmax;
    int nsub = (int)ceil(dts / dtc);
    L->dt = dts / (double)nsub;
    /* scatter phi into the patches */
    for (int k = 0; k < L->np; k++) {
        OPatch *p = &L->p[k];
        for (int f = 0; f < h->m; f++)
            for (int j = 0; j < p->ny; j++)
                for (int i = 0; i < p->nx; i++)
                    p->q[L->cur][qidx(h, p, f, i, j)] = phi[((long)f * ny + p->jlo + j) * nx + p->ilo + i];
    }
    long per = (long)h->m * nx * ny;
    for (int s = 0; s < nsnap; s++) {
        if (s > 0)
            for (int q = 0; q < nsub; q++) {
                int err = 0;
                if (fill_ghosts(h, 0, 0)) { orc_destroy(h); return 1; }
                step_level_patches(h, 0, &err);
                L->cur = 1 - L->cur;
                L->nstep++;
            }
        double *dst = snaps + (long)(nsnap - 1 - s) * per;
        for (int k = 0; k < L->np; k++) {
            const OPatch *p = &L->p[k];
            for (int f = 0; f < h->m; f++)
                for (int j = 0; j < p->ny; j++)
                    for (int i = 0; i < p->nx; i++)
                        dst[((long)f * ny + p->jlo + j) * nx + p->ilo + i] = p->q[L->cur][qidx(h, p, f, i, j)];
        }
    }
    orc_destroy(h);
    return 0;
}

/* The adjoint solved on an AMR hierarchy of its own (Sec. 7 names this as a
   way to a more accurate inner product): P describes the adjoint hierarchy
   (eqn = adjoint system, nlevels >= 1, ratios, a standard flag mode and its
   tolerance, regrid interval and buffer); its level 0 is the snapshot grid.
   q~(x, 0) = phi on level 0 and, on the finer levels the initial regrid
   creates, the coarse-fine interpolation of it (a target box aligned to
   level-0 cell edges is reproduced exactly).  Level-0 steps of dt = dT /
   ceil(dT / dt_cfl), dT = (tf - t0)/(nsnap - 1), each a full Berger-Oliger
   step (regrids, substeps, average-down: level 0 holds the composite
   solution averaged onto it); snapshot s is level 0 at tau_s, stored at
   index nsnap - 1 - s (forward time order).  medium: dense [nmed][ny][nx]
   per level in `dense` (nlevels arrays back to back) or layered. */
int orc_adjoint_solve_amr(const orc_params *P, int axis, int nl, const double *iface, const double *f0,
                          const double *f1, const double *dense, const double *phi, int nsnap, double *snaps)
{
    if (nsnap < 2 || P->nlevels < 1) return 1;
    orc_params Q = *P;
    Q.qinit = NULL;
    double dmin0;
    {
        int N = P->n0[0], M = (P->dim == 2) ? P->n0[1] : 1;
        double dx = (P->hi[0] - P->lo[0]) / (double)N;
        double dy = (P->dim == 2) ? (P->hi[1] - P->lo[1]) / (double)M : dx;
        dmin0 = (P->dim == 2) ? fmin(dx, dy) : dx;
    }
    double dts = (P->tf - P->t0) / (double)(nsnap - 1);
    double dtc = P->cfl * dmin0 / P->cmax;
    int nsub = (int)ceil(dts / dtc);
    Q.dt0 = dts / (double)nsub;
    OHier *h = orc_create(&Q);
    if (!h) return 1;
    if (dense) {
        long off = 0;
        int N = P->n0[0], M = (P->dim == 2) ? P->n0[1] : 1;
        for (int l = 0; l < P->nlevels; l++) {
            orc_set_medium_dense(h, l, dense + off);
            off += (long)h->nmed * N * M;
            if (l < P->nlevels - 1) {
                N *= P->ratio[l];
                if (P->dim == 2) M *= P->ratio[l];
            }
        }
    } else {
        orc_set_medium_layered(h, axis, nl, iface, f0, f1);
    }
    OLevel *L = &h->L[0];
    int nx = L->N, ny = L->M;
    for (int k = 0; k < L->np; k++) {
        OPatch *p = &L->p[k];
        for (int f = 0; f < h->m; f++)
            for (int j = 0; j < p->ny; j++)
                for (int i = 0; i < p->nx; i++)
                    p->q[L->cur][qidx(h, p, f, i, j)] = phi[((long)f * ny + p->jlo + j) * nx + p->ilo + i];
    }
    if (P->nlevels > 1 && regrid_from(h, 0, 0)) {
        orc_destroy(h);
        return 1;
    }
    long per = (long)h->m * nx * ny;
    double cfl = 0.0;
    for (int s = 0; s < nsnap; s++) {
        if (s > 0)
            for (int q = 0; q < nsub; q++)
                if (step_level(h, 0, &cfl)) {
                    orc_destroy(h);
                    return 1;
                }
        double *dst = snaps + (long)(nsnap - 1 - s) * per;
        for (int k = 0; k < L->np; k++) {
            const OPatch *p = &L->p[k];
            for (int f = 0; f < h->m; f++)
                for (int j = 0; j < p->ny; j++)
                    for (int i = 0; i < p->nx; i++)
                        dst[((long)f * ny + p->jlo + j) * nx + p->ilo + i] = p->q[L->cur][qidx(h, p, f, i, j)];
        }
    }
    orc_destroy(h);
    return 0;
}

/* exported for tests: Berger-Rigoutsos clustering of a dense flag field
   [M][N] with nesting mask (NULL = everything nestable); boxes out as
   [n][4] = (i0, i1, j0, j1), inclusive, sorted by (j0, i0).  Returns the
   number of boxes, or -1 if cap is too small. */
int orc_cluster(const unsigned char *flags, const unsigned char *nest, int N, int M, int dim, int mc, double eff,
                int *boxes, int cap)
{
    unsigned char *ones = NULL;
    if (!nest) {
        ones = xcalloc((size_t)N * M, 1);
        memset(ones, 1, (size_t)N * M);
        nest = ones;
    }
    OBR c = {flags, nest, N, M, dim, mc, eff};
    OBoxList L = {0};
    OBox all = {0, N - 1, 0, M - 1};
    br(&c, all, &L);
    qsort(L.b, L.n, sizeof(OBox), cmp_box);
    int n = L.n;
    if (n <= cap)
        for (int k = 0; k < n; k++) {
            boxes[4 * k + 0] = L.b[k].i0;
            boxes[4 * k + 1] = L.b[k].i1;
            boxes[4 * k + 2] = L.b[k].j0;
            boxes[4 * k + 3] = L.b[k].j1;
        }
    free(L.b);
    free(ones);
    return n <= cap ? n : -1;
}
