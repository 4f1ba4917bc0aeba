// Internal structures of libadjamr: device descriptors shared by the host
// hierarchy code (hierarchy.cpp) and the CUDA kernels (kernels_*.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifdef __cplusplus
#include <atomic>
#endif

#include "adjamr.h"

#ifndef __CUDACC__
// A device-resident adjoint snapshot set, shared by reference count
// (contexts and serving slots on several host threads hold references).
struct adjamr_adjoint {
    std::atomic<int> refs{1};
    int S = 0, m = 0, ax = 0, ay = 0, dim = 0;
    double *d_snaps = nullptr;
    unsigned char *d_wet = nullptr;
    double *d_bmax = nullptr;  // [nblk][m][ay][ax]: max |q^| over a snapshot block and a bilinear stencil
    int nblk = 0;
    size_t bytes = 0;
};
#endif

namespace adjamr {

constexpr double kGrav = 9.81;

// Per-cell coefficient arrays ("aux"), hoisted medium-only quantities.
// Edge coefficients are stored at the cell on the high side of the edge
// (x-edge i-1/2 at cell i, y-edge j-1/2 at cell j).
//  ACOUSTICS:          c, Z, 1/(Z_{i-1}+Z_i), 1/(Z_{j-1}+Z_j)
//  ACOUSTICS_ADJOINT:  c, Z, izs_x, izs_y, 1/rho, K
//  SW:                 ce_x, 1/ce_x, g*he_x, ce_y, 1/ce_y, g*he_y
//  SW_ADJOINT:         ce_x, 1/ce_x, ce_y, 1/ce_y, g*hbar
__host__ __device__ constexpr int naux_of(int eqn) { return eqn == 0 ? 4 : (eqn == 3 ? 5 : 6); }
__host__ __device__ constexpr int nmed_of(int eqn) { return (eqn == 2 || eqn == 3) ? 1 : 2; }

// A patch in a level arena.  Storage cell (si, sj) (si in [0, sx), sj in
// [0, sy)) of field f lives at f*stride + base + sj*sx + si; interior cell
// (i, j) is storage (i + 2, j + gy), gy = 2 in 2D and 0 in 1D.
struct PatchDesc {
    int ilo, jlo, nx, ny;
    int sx, sy;
    long long base;
    double dtdx, dtdy, hx, hy;
    long long gbase;  // index of the patch's first ghost descriptor
};

// One tile of the step work-list.
// One tile of a patch: interior cells [x0, x0+tx) x [y0, y0+ty), tx <= TX and
// ty <= TY of the kernel.  A patch is cut into near-equal tiles (extents
// differ by at most one cell per direction) so that the tiles of a level
// carry near-equal work.
struct WorkItem {
    int patch, x0, y0;
    unsigned short tx, ty;
};

// near-equal split of len cells into ceil(len / t) pieces: piece k's offset
// and length
inline int tile_count(int len, int t) { return (len + t - 1) / t; }
inline int tile_off(int len, int n, int k) { return k * (len / n) + (k < len % n ? k : len % n); }
inline int tile_len(int len, int n, int k) { return len / n + (k < len % n ? 1 : 0); }

// One ghost cell (or one new cell at regrid).
//  kind 0: copy the cell `src` of the same arena (with sign flips);
//  kind 1: minmod-limited linear interpolation from the coarser level around
//          coarse cell `src` with neighbours cxm, cxp, cym, cyp (each with
//          its own boundary sign), fine offset (mx, my) inside the coarse cell;
//  kind 2 (regrid only): copy cell `src` of the OLD arena of this level.
// signs: bits 0,1 = negate components 1,2 of the result; bits 2+2k, 3+2k =
// negate components 1,2 of coarse reference k (0 centre, 1 xm, 2 xp, 3 ym, 4 yp).
struct GhostDesc {
    long long dst;
    long long src, cxm, cxp, cym, cyp;
    int kind, signs;
    double fx, fy;  // offsets (2m+1-r)/(2r) of the fine cell within its coarse cell
};

// Average-down of one coarse cell: dst in the coarse arena, src = fine child
// (0, 0) in the fine arena, fsx = fine row pitch.
struct AvgDesc {
    long long dst, src;
    int fsx, pad;
};

// Aux-fill of one storage cell of a new patch: arena index and the global
// level index of the cell (may lie outside the domain: boundary-mapped on
// the device).
struct AuxDesc {
    long long idx;
    int I, J;
};

struct MediumDev {
    int kind, axis, nl, nmed;
    double iface[32], f0[32], f1[32];
    const double *dense;   // [nmed][M][N] of this level (DENSE)
    int N, M;
};

struct LevelGeom {
    int dim, N, M;
    double lo0, lo1, dx, dy;
    int bc[4];
};

// Conservation fix-up at coarse-fine interfaces (refluxing).  A cell of a
// level that takes part has an entry in the level's table: its arena index,
// for each side s (0 x-low, 1 x-high, 2 y-low, 3 y-high) the coarse-role
// record c[s] (the cell is an uncovered cell and its neighbour across s is
// covered by the finer level) and the fine-role record f[s] (the cell is on
// a patch edge and its neighbour across s is a ghost cell interpolated from
// the coarser level), -1 where none.
struct RefluxCell {
    long long idx;
    int c[4], f[4];
};

// What a step launch records for the fix-up (rmap == nullptr: nothing).
// rmap[arena cell] = entry of the level's table or -1.  A coarse-role record
// c receives lc[2c + k] = the value side s put into the cell (component 0,
// then the normal component); a fine-role record f of substep `sub`
// receives lf[(sub * nfrec + f) * 4 + {0, 1, 2, 3}] = those two values and
// the cell's state (component 0, normal component) at the start of the step.
struct RefluxArgs {
    const int *rmap;
    const RefluxCell *cells;
    double *lc, *lf;
    long long nfrec;
    int sub;
};

// Ghost cells computed inside the step kernel while staging a tile: the
// ghost descriptors of the level and the coarser level's two time levels.
// gd == nullptr: the ghost ring is read from q (filled beforehand).  rx: the
// fix-up records of the launch (they travel with the ghost arguments, which
// every step launch carries).
struct GhostArgs {
    const GhostDesc *gd;
    // coarse stencil values of the level's kind-1 ghost cells (k_cpre) for
    // substep 0; substep k at pre + k * pstride; sc = the coarse arena stride
    const double *pre;
    long long sc, pstride;
    int k;  // fine substep within the coarse step
    RefluxArgs rx;
};

// The fix-up of the coarse-role cells of level l after the fine substeps and
// the average-down: for every side s with c[s] >= 0, the mean over the r
// substeps and nseg fine edges of L* = (A-dQ + A+dQ)(Riemann problem between
// the cell, at its old state, and the fine cell) - (what the fine cell
// received through the edge), and qc_new -= dtd * (mean L* - lc).
struct RefluxApply {
    const RefluxCell *cells;
    int ncoarse;
    const double *qc_old;
    double *qc_new;
    const double *medc;     // primary medium of level l
    long long sc;
    const double *lc, *lf;
    long long nfrec;
    const long long *fidx;  // [nfrec]: arena index of the fine cell of a fine record
    const double *medf;     // primary medium of level l + 1
    long long sf;
    int r, nseg;
    double w;               // 1 / (r * nseg)
    double dtdx, dtdy;
    int *err;               // kRefluxErrBit or-ed in if a fine edge of a recorded side has no record
};
constexpr int kRefluxErrBit = 1 << 29;
cudaError_t launch_reflux_apply(int dim, int eqn, const RefluxApply &a, cudaStream_t s);
// rmap[cells[e].idx] = e for every entry (rmap set to -1 beforehand)
cudaError_t launch_reflux_map(const RefluxCell *cells, int n, int *rmap, cudaStream_t s);

// Tile schedule of a step launch.  ctr == nullptr: CTA b takes tiles b,
// b + grid, ...  Otherwise every CTA takes the next tile from the counter
// (dynamic balancing); tile = counter - base, and the launch advances the
// counter by exactly nwork + grid (its tiles plus one fetch past the end per
// CTA), so consecutive launches on a stream chain their bases.
struct TileSched {
    unsigned long long *ctr;
    unsigned long long base;
};

// Several substeps of one level in one launch (k_step2d_sub).  Row w of
// dep_idx (stride kDepRow) lists the tiles whose interior cells tile w's
// staged region reads, itself included; dep_cnt[w] entries, or more than
// kDepRow when the row overflowed (then the tile waits for every tile).
// done[w] = base + substeps tile w has completed in this launch (values from
// earlier launches are <= base).
constexpr int kMaxSubsteps = 16;
constexpr int kDepRow = 48;
constexpr unsigned long long kSubstepWaitNs = 1000000000ull;  // a wait gives up after 1 s
constexpr unsigned int kSubstepWaitSpins = 1u << 24;
constexpr int kSubstepErrBit = 1 << 30;  // recorded in the context's device error word
struct SubstepArgs {
    const int *dep_idx, *dep_cnt;
    unsigned long long *done;
    unsigned long long base;
    int nsub;
    int *err;                  // kSubstepErrBit is or-ed in when a wait gave up
};

// time fractions k / r of the substeps of a coarse step, divided on the host
struct SubstepTimes {
    double th[kMaxSubsteps];
};

// Programmatic dependent launch of the kernels of the stepping sequence (step,
// ghost fill, average-down, gauges): on unless the environment sets
// ADJAMR_PDL=0 (read once).  Results are the same either way.
bool pdl_enabled();
#ifdef __CUDACC__
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<A &&>(args)...);
}
#endif

// ---- kernel launchers (kernels_step.cu / kernels_amr.cu) ----
cudaError_t launch_step(int dim, int eqn, int tx, int ty, const double *q, double *qn, const double *aux,
                        long long stride, const PatchDesc *patches, const WorkItem *work, int nwork, int grid,
                        unsigned long long *cfl_bits, cudaStream_t s, GhostArgs ga = GhostArgs{},
                        TileSched sc = TileSched{nullptr, 0});
int step_occupancy(int dim, int eqn, int tx, int ty);
// sa.nsub steps of a 2D level in one launch of `grid` CTAs that take items
// from sc (sc.ctr required; the counter advances by nsub * nwork + grid).
// Kernel tiles 8x8, 16x8, 16x12 and 16x16 only; ga.gd required (the ghost ring is
// computed in the kernel), ga.k = the first substep.
cudaError_t launch_step_substeps(int eqn, int tx, int ty, double *qa, double *qb, const double *aux, long long stride,
                                 const PatchDesc *patches, const WorkItem *work, int nwork, int grid,
                                 unsigned long long *cfl_bits, cudaStream_t s, const GhostArgs &ga,
                                 const TileSched &sc, const SubstepArgs &sa);
int substep_occupancy(int eqn, int tx, int ty);  // 0: no such kernel
// dependency rows of a 2D level's work list for substep launches: tile_of
// (one int per arena cell) receives the tile of every interior cell, then
// each tile lists the tiles met by its cells and 2-cell halo (periodic
// images across periodic boundaries; owner = the level's [M][N] owner map)
cudaError_t launch_tile_deps(const PatchDesc *patches, const WorkItem *work, int nwork, const int *owner, int N, int M,
                             const int *bc, int *tile_of, int *dep_idx, int *dep_cnt, cudaStream_t s);
// compiled step-kernel tile (kx, ky) that holds tiles of tx x ty cells: the
// smallest by area among 8x8, 16x8, 16x12, 32x8, 16x16, 64x8, 32x16 (1D: 128 or 256);
// false if none does
bool step_kernel_shape(int dim, int tx, int ty, int *kx, int *ky);

// early: the kernel ahead in the stream is a step of this level and the
// coarser level's states are final (see k_ghost_fill).  pre_k != nullptr: the
// kind-1 ghost cells take the precomputed coarse stencil values of substep k
// (k_cpre) instead of interpolating from qc_old / qc_new.
// cp.list != nullptr: cp_blocks extra CTAs also compute the stored stencil
// values of substeps 1 .. cp.r - 1 into cp.pre (as launch_cpre; the fill
// itself then interpolates directly, pre_k = nullptr)
struct CpreArgs {
    const unsigned long long *list;
    double *pre;
    long long sc;
    int r;
    SubstepTimes tt;  // filled by the launcher
};
cudaError_t launch_ghost_fill(int dim, int m, const GhostDesc *g, long long n, double *qf, long long sf,
                              const double *qc_old, const double *qc_new, long long sc, int k, int r,
                              cudaStream_t s, bool early = false, const double *pre_k = nullptr,
                              CpreArgs cp = CpreArgs{}, int cp_blocks = 0);
// coarse stencil values (q0, sx, sy) of every listed coarse cell, field and
// substep s < r: pre[((s * m + f) * sc + src) * 3 + {0, 1, 2}]
cudaError_t launch_cpre(const GhostDesc *g, const unsigned long long *list, long long nmax, int m, int r, int dim,
                        const double *qc_old, const double *qc_new, long long sc, double *pre, int grid,
                        cudaStream_t s);
cudaError_t launch_average_down(int dim, int m, const AvgDesc *a, long long n, const double *qf, long long sf,
                                double *qc, long long sc, int r, cudaStream_t s);
// Fill primary medium (med) and derived coefficients (aux) of the listed
// storage cells of one level.  mdev: device copy of the level's medium.
cudaError_t launch_aux_fill(int eqn, int dim, const AuxDesc *d, long long n, double *aux, double *med,
                            long long stride, const MediumDev *mdev, LevelGeom geom, cudaStream_t s);

struct FlagArgs {
    const double *q;
    long long stride;
    const PatchDesc *patches;
    const long long *cell_prefix;   // [np+1] interior-cell prefix over patches
    int np, dim, m, mode;
    long long ncells;
    double lo0, lo1, hi0, hi1, dx, dy;
    const double *snaps;            // [S][m][ay][ax]
    const unsigned char *wet;       // [ay][ax]
    int ax, ay, nlo, nhi, S;
    double t, T, t0, dts, tol;
    unsigned char *flags_patch;     // [ncells] (may be null)
    unsigned long long *flags_bits; // [M][pitch64]: bit I & 63 of word I >> 6 of row J (may be null; zeroed)
    int pitch64;
    int N;
    unsigned long long *count;
    int *bbox;                      // [4]: bounding box of the flagged cells, as atomic maxima of
                                    // INT_MAX - min I, max I + 1, INT_MAX - min J, max J + 1 (zero: none)
    const double *bmax;             // block maxima for culling (may be null)
    // dense bracket-max variant: the level's owner map ([M][N] storage index
    // or -1) and per-column / per-row bilinear tables of the adjoint grid
    const int *owner;
    int M, gblk;                    // index-space rows; snapshot blocks per thread
    const int *tab_a, *tab_ac;      // [N]: stencil column, column of the containing cell
    const double *tab_wx;           // [N]
    const int *tab_b, *tab_bc;      // [M]
    const double *tab_wy;           // [M]
};
constexpr int kSnapBlock = 8;       // snapshots per culling block
// block maxima of a snapshot set: bmax[blk][f][b][a] = max over the block's
// snapshots and the cells (a..a+1, b..b+1) of |snap|
cudaError_t launch_block_max(const double *snaps, int S, int m, int ax, int ay, int dim, double *bmax,
                             cudaStream_t s);
cudaError_t launch_flag(const FlagArgs &a, cudaStream_t s);
// gauge record: out[g][1 + m] for every gauge (see k_gauges)
struct GaugeArgs {
    int n, m, nlev;
    const int *gi, *gj;             // [nlev][n]: cell index of every gauge on every level
    const int *owner[ADJAMR_MAX_LEVELS];
    const double *q[ADJAMR_MAX_LEVELS];
    long long stride[ADJAMR_MAX_LEVELS];
    int N[ADJAMR_MAX_LEVELS];
    double t;
    double *out;
};
cudaError_t launch_gauges(const GaugeArgs &g, cudaStream_t s);

// bytes of released device blocks a context keeps for reuse by later regrids
// (0: every block is freed at once; the serving loop, which admits requests by
// their projected bytes, uses 0)
void ctx_set_block_cache(adjamr_ctx *c, size_t cap_bytes);
// per-level coefficient tables on (default) or off; set before adjamr_set_medium
void ctx_set_aux_tables(adjamr_ctx *c, bool on);

// bracket-max flags over the level's index space, one thread per (cell, group
// of a.gblk snapshot blocks), into the zeroed bitmap a.flags_bits
cudaError_t launch_flag_dense(const FlagArgs &a, int ngroup, cudaStream_t s);
// The same flags in two passes: a bound pass lists the (cell, snapshot block)
// pairs whose bound can exceed tol, an evaluation pass takes one snapshot of a
// listed block per thread.  ctr[0] = listed pairs, ctr[1] = nonzero when the
// list overflowed cap (the flags are then incomplete; ctr zeroed beforehand).
struct FlagWork {
    unsigned long long *items;  // (cell index << 16) | block
    unsigned long long *ctr;
    long long cap;
};
cudaError_t launch_flag_twopass(const FlagArgs &a, const FlagWork &w, int eval_grid, cudaStream_t s);

// terms weight*(q0*area) of the functional into out[0..n)
cudaError_t launch_func_terms(const long long *idx, const double *area, long long n, const double *q, double weight,
                              double *out, cudaStream_t s);
// fixed pairwise tree sum of a[0..n) (destroys a) into *out
cudaError_t launch_pairwise(double *a, long long n, double *out, cudaStream_t s);

cudaError_t launch_gather_interior(int m, const long long *map, long long n, const double *q, long long stride,
                                   double *dst, cudaStream_t s);

}  // namespace adjamr

namespace adjamr {

// Geometry of a level for device-side index work (boundary maps, owners).
struct LevelIdx {
    int dim, N, M, gy;
    int bc[4];
};

// Richardson error estimate of one level (flag mode ADJAMR_FLAG_ERROR).
// Every patch of the level is extended to even extents (ne, me) (1D: me = 1)
// with a ring of 4 cells: storage "E", pitch ne + 8, me + 8 rows (1D: one),
// at ebase; the same coarsened by 2: storage "C", pitch ne/2 + 4, me/2 + 4
// rows (1D: one), at cbase.  abase/asx: the patch in the level arena.
struct ErrEstPatch {
    int ilo, jlo, nx, ny;
    int ne, me, asx, pad;
    long long ebase, cbase, abase;
};
struct ErrEstArgs {
    const ErrEstPatch *ep;
    const long long *eprefix, *cprefix;  // [np + 1]: E / C storage cells before patch p
    int np, dim, m, eqn;
    long long nE, nC;                    // E / C storage cells (the buffers' field strides)
    double *E, *F, *auxE, *medE;         // E storage: state, first-step state, coefficients
    double *C, *C1, *auxC, *medC;        // C storage
};
// the extended patches (state as ghost cells get it at substep k with time
// fraction th of level l - 1: q the level's current state, owner its owner
// map; qo / qn, owner_c the coarser level's) and their coefficients; then the
// coarsened copies (mean of the children, medium included).  err |= 1 where
// an interpolation stencil leaves the coarser level.
cudaError_t launch_errest_fill(const ErrEstArgs &a, LevelIdx g, const int *owner, const double *q, long long sq,
                               const int *owner_c, LevelIdx gc, int r, const double *qo, const double *qn,
                               long long sc, int k, const MediumDev *md, LevelGeom geom, int *err, cudaStream_t s);
// tau[f * st + arena cell] = (mean of the 2^d children of the two-step state
// (in E) - the coarse step's (C1)) / 6 for every interior cell of the level
cudaError_t launch_errest_tau(const ErrEstArgs &a, const long long *iprefix, long long ninterior, double *tau,
                              long long st, cudaStream_t s);

// Device-side regrid support: the kernels that build a level's new layout,
// one thread per interior cell, storage cell, ghost cell or coarse cell under
// the level (n = 0: nothing to do).  Prefix arrays have np+1 entries.
//
// owner[J*N + I] = arena index of interior cell (I, J) of the level, or -1
// (the map is set to -1 beforehand).
struct OwnerFillArgs {
    const PatchDesc *pd;
    const long long *prefix;
    int np;
    long long n;
    LevelIdx g;
    int *owner;
};
// ghost descriptors of every patch of a level; gprefix = ghost-cell prefix.
// owner_c / gc describe the coarser level (owner_c null on level 0).
// cmark / clist (levels > 0): also lists one kind-1 ghost cell per distinct
// coarse cell, clist[0] = count (zeroed beforehand), clist[1 + e] = ghost
// index; a coarse cell is taken when its mark was not yet cgen (> 0)
struct GhostBuildArgs {
    const PatchDesc *pd;
    const long long *gprefix;
    int np;
    long long n;
    LevelIdx g;
    const int *owner, *owner_c;
    LevelIdx gc;
    int r;
    GhostDesc *out;
    int *err;
    int *cmark;
    int cgen;
    unsigned long long *clist;
};
// average-down descriptors; aprefix = prefix of coarse-footprint cells per fine patch
struct AvgBuildArgs {
    const PatchDesc *pd;
    const long long *aprefix;
    int np;
    long long n;
    int dim, r;
    const int *owner_c;
    LevelIdx gc;
    AvgDesc *out;
    int *err;
};
// new interior cells: copy from the old arena (owner_old) or interpolate from
// the coarser level (owner_c, qc) at its current time
struct InitNewArgs {
    const PatchDesc *pd;
    const long long *prefix;
    int np;
    long long n;
    LevelIdx g;
    int m;
    double *qf;
    long long sf;
    const int *owner_old;
    const double *qold;
    long long so;
    const int *owner_c;
    LevelIdx gc;
    const double *qc;
    long long sc;
    int r;
    int *err;
};
cudaError_t launch_owner_fill(const OwnerFillArgs &a, cudaStream_t s);
cudaError_t launch_ghost_build(const GhostBuildArgs &a, cudaStream_t s);
cudaError_t launch_avg_build(const AvgBuildArgs &a, cudaStream_t s);
cudaError_t launch_init_new(const InitNewArgs &a, cudaStream_t s);
// coefficients a rebuilt level may copy from its previous arena: a storage
// cell whose (I, J) was an interior cell of the previous patches takes that
// cell's values (they depend on (I, J) only); owner == nullptr: compute all
struct AuxReuse {
    const int *owner;
    const double *aux, *med;
    long long stride;
    int naux, nmed;
};
// Coefficient table of a level: aux then med fields of every cell of the
// index space with a 2-cell border ([naux + nmed][rows][N + 4], rows = M + 4
// in 2D, 1 in 1D), computed once per medium by launch_aux_table.
struct AuxTable {
    const double *tab;
    long long stride;  // cells per field
    int width;         // N + 4
};
cudaError_t launch_aux_table(int eqn, const MediumDev *mdev, LevelGeom geom, double *tab, cudaStream_t s);
// coefficients of every storage cell (sprefix = storage-cell prefix);
// tb.tab != nullptr: copied from the table
struct AuxPatchesArgs {
    int eqn;
    const PatchDesc *pd;
    const long long *sprefix;
    int np;
    long long n;
    LevelIdx g;
    double *aux, *med;
    long long stride;
    const MediumDev *mdp;
    LevelGeom geom;
    AuxReuse ru;
    AuxTable tb;
};
cudaError_t launch_aux_patches(const AuxPatchesArgs &a, cudaStream_t s);
// The five builders of one level in two launches: the owner map, the
// coefficients and the new interior state (none reads another's output) side
// by side in one grid, then the ghost and average-down maps (which read the
// new owner map) in the next.  *nlaunch = kernels launched (0 to 2).
cudaError_t launch_rebuild(const OwnerFillArgs &o, const AuxPatchesArgs &x, const InitNewArgs &in,
                           const GhostBuildArgs &gb, const AvgBuildArgs &ab, cudaStream_t s, int *nlaunch);

}  // namespace adjamr
