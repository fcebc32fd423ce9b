// Device engine of the coupled lattice Boltzmann step with the general local
// reactive boundary condition (arXiv 2306.10794).  Templated over the storage
// type T (float: deviation storage, double) and the flow / solute lattices.
//
// Storage ("AA pattern", one population array per lattice, in place):
//   population slot A[i][cell] for every cell of a padded dense grid (x
//   fastest, rows padded to 32 cells, ghost layers on non-periodic axes),
//   the cells grouped in blocks of 32 whose Q populations are stored one
//   after the other (pslot).  After an
//   even step the post-collision value f*_i(x) sits in A[opp(i)][x]; after
//   an odd step in A[i][x + e_i], whatever lies at x + e_i (fluid, solid or
//   ghost).  Writes never depend on the geometry; the boundary rules are
//   applied when a node READS a population whose source x - e_i is inactive:
//   the plain value there is its own f*_opp(i) (halfway bounce-back), which
//   the open-boundary rules then modify.  Phase changes therefore never move
//   populations: the next step simply reads with the new node classes.
//
// Per step: k_fluid (dense sweep, fluid cells: flow + solute), k_bound (the
// compacted list of wet boundary cells: solute streaming, Eq. general_RBC on
// every link to a fluid cell, ledger, collision with u = 0, solid-fraction
// update), k_fend (fluid cells next to reactive boundary cells gather their
// precipitation shares), and, with phase change, the event kernels that
// apply Sec. 2.4 and rebuild the node words and both lists on the device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lattice.cuh"
#include "sim_iface.h"

namespace lbrbc {

enum : uint32_t { CLS_FLUID = 0, CLS_BOUND = 1, CLS_SOLID = 2 };
enum : uint8_t { KIND_FLUID = 0, KIND_REACTIVE = 1, KIND_DIRICHLET = 2, KIND_OUTSIDE = 3 };
enum : int { EV_DISSOLVE = 1, EV_PRECIPITATE = 2 };
enum : int { ERR_NUMERIC = 1, ERR_OVERFLOW = 2 };
// fluid sweep: dense grid or compacted fluid list
enum : int { SWEEP_DENSE = 0, SWEEP_LIST = 1 };

// node word of a fluid cell: bits 0-1 class, bits FBIT.. "flow source
// x - e_i is not fluid" for i = 1..QF-1, bits GBIT.. "solute source
// x - e_i is inactive" for i = 1..QG-1.
constexpr int FBIT = 2;
constexpr int GBIT = 20;
// word of a boundary-list entry: bits 0.. source inactive (i = 1..QG-1),
// bits 8.. link towards a fluid cell (o = 1..QG-1), bit 16 Dirichlet cell.
constexpr int BW_LINK = 8;
constexpr uint32_t BW_DIRICHLET = 1u << 16;
constexpr uint32_t BW_DEAD = 1u << 17;  // entry of a cell that is no longer a wet boundary cell

#ifndef LBRBC_FLUID_BLOCK
#define LBRBC_FLUID_BLOCK 128
#endif
// Population loads / stores of the fluid sweep: 0 default caching, 1
// evict-first (each population is touched once per step).
#ifndef LBRBC_STREAM_HINT
#define LBRBC_STREAM_HINT 1
#endif
// Active-cell sweep: cache policy of the odd step's loads and stores through
// the neighbour table (1 evict-first like the other population accesses, 0
// the default policy, which keeps partly used lines for the neighbouring
// warps: measured 17 % faster for the loads on a 512^3 sphere pack) and
// resident blocks of 128 threads per SM it is compiled for.
#ifndef LBRBC_SP_NBR_HINT
#define LBRBC_SP_NBR_HINT 0
#endif
#ifndef LBRBC_SP_NBR_STORE_HINT
#define LBRBC_SP_NBR_STORE_HINT 1
#endif
#ifndef LBRBC_BOUND_BLOCKS
#define LBRBC_BOUND_BLOCKS 5  // resident blocks per SM of the boundary kernel (register cap)
#endif
#ifndef LBRBC_SP_L2PF
// odd active-cell sweep: L2 prefetch distance in blocks (0: none); one wave
// of resident blocks on GB300 (152 SMs x 8): 2.29 -> 2.23 ms per launch at
// 512^3 (608: 2.24, 2432: 2.31; prefetching the block's populations as
// well: 2.44)
#define LBRBC_SP_L2PF 1216
#endif

#ifndef LBRBC_SP_BLOCKS
#define LBRBC_SP_BLOCKS 8
#endif
constexpr int FLUID_BLOCK = LBRBC_FLUID_BLOCK;
constexpr int LIST_BLOCK = 256;
constexpr int SCAN_CHUNK = 1024;

struct Geo {
    int nx, ny, nz;
    int SX, SY, SZ;      // padded extents
    int py, pz;          // ghost layers in y / z (0 when periodic)
    int per_x, per_y, per_z, open_x;
    long long OFF, NP;   // offset of the padded origin, slots per population
    __host__ __device__ long long idx(int x, int y, int z) const {
        return OFF + x + (long long)SX * ((long long)(y + py) + (long long)SY * (z + pz));
    }
};

struct Nbr {
    long long xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Nbr nbr_deltas(const Geo& g, int x, int y, int z) {
    Nbr d;
    const long long sy = g.SX, sz = (long long)g.SX * g.SY;
    d.xp = (g.per_x && x == g.nx - 1) ? -(long long)(g.nx - 1) : 1;
    d.xm = (g.per_x && x == 0) ? (long long)(g.nx - 1) : -1;
    d.yp = (g.per_y && y == g.ny - 1) ? -(long long)(g.ny - 1) * sy : sy;
    d.ym = (g.per_y && y == 0) ? (long long)(g.ny - 1) * sy : -sy;
    d.zp = (g.per_z && z == g.nz - 1) ? -(long long)(g.nz - 1) * sz : sz;
    d.zm = (g.per_z && z == 0) ? (long long)(g.nz - 1) * sz : -sz;
    return d;
}

template <class L>
__device__ __forceinline__ long long off(const Nbr& d, int i) {
    return (L::cx(i) > 0 ? d.xp : (L::cx(i) < 0 ? d.xm : 0)) + (L::cy(i) > 0 ? d.yp : (L::cy(i) < 0 ? d.ym : 0)) +
           (L::cz(i) > 0 ? d.zp : (L::cz(i) < 0 ? d.zm : 0));
}

// Is (x,y,z) + e inside the grid after periodic wrapping?  Writes the wrapped
// coordinates.
__device__ __forceinline__ bool wrap_inside(const Geo& g, int& x, int& y, int& z) {
    if (x < 0 || x >= g.nx) {
        if (!g.per_x) return false;
        x = (x + g.nx) % g.nx;
    }
    if (y < 0 || y >= g.ny) {
        if (!g.per_y) return false;
        y = (y + g.ny) % g.ny;
    }
    if (z < 0 || z >= g.nz) {
        if (!g.per_z) return false;
        z = (z + g.nz) % g.nz;
    }
    return true;
}

__device__ __forceinline__ void coords(const Geo& g, long long id, int& x, int& y, int& z) {
    long long r = id - g.OFF;
    x = (int)(r % g.SX);
    long long t = r / g.SX;
    y = (int)(t % g.SY) - g.py;
    z = (int)(t / g.SY) - g.pz;
}

struct Phys {
    double of_sym, of_anti;  // flow: 1/tau (symmetric), 1/tau^- (antisymmetric)
    double og_sym, og_anti;  // solute: antisymmetric part relaxes with 1/tau_D
    int trt_f, trt_g;
    double gw0, gw1, gcs2;   // solute weights (rest / moving) and cs^2
    double cref;             // reference concentration of the deviation storage
    double c_inlet, rho_out, c_dir, c_eq, k_r, gamma, Vm, rho_init;
    int scheme, phase_change;
};

// The same parameters in the storage precision, precomputed on the host so
// that per-cell arithmetic never converts from FP64 (FP64 is slow on GB300).
template <typename T>
struct PhysT {
    T f_sym, f_anti;   // flow relaxation rates
    T g_sym, g_anti;   // solute relaxation rates
    T gw[9];           // solute weights per direction
    T ics2;            // 1 / cs^2 of the solute lattice
    T cref;            // deviation reference
    T c_in_d, c_dir_d, c_eq_d;  // c_inlet, c_dirichlet, c_eq minus cref
    T rho_out, k_r, gamma, neg_vm;
    T rho_out_d;       // rho_out - 1 (the outlet rule in deviation form, no cancellation)
};

template <typename T>
struct Dev {
    Geo geo;
    T* F;                 // flow populations  (QF * NP)
    T* G;                 // solute populations (QG * NP)
    uint32_t* nw;         // node words (NP)
    uint8_t* kind;        // cell kinds (NP)
    double* phi;          // solid fraction (NP)
    double* kfield;       // per-voxel k_r (NP) or null
    double* inlet_ux;     // ny*nz
    double* side;         // outlet: previous u (3 per cell) and C, 4*ny*nz
    // wet boundary cells
    int cap_b;
    int* nb;
    int* b_idx;
    uint32_t* b_word;
    uint64_t* b_xyz;      // packed cell coordinates (21 bits each)
    T* b_kappa;           // (QG-1) * cap_b
    double* b_krate;      // cap_b or null
    T* b_share;           // (QG-1) * cap_b: precipitation share of link o (written by k_bound, list order)
    int* bmap;            // NP
    // fluid cells receiving precipitation shares
    int cap_f;
    int* nf;
    int* f_idx;
    int* f_src;           // (QG-1) * cap_f: index in b_share of the share from the boundary cell at x - e_o, or -1
    // compacted fluid cells (packed x | y << 11 | z << 22), when the sweep
    // runs over a list instead of the dense grid
    int use_fl;
    int cap_fl;
    int* nfl;
    uint32_t* fl_xyz;
    // adjoint recomputation tape (null in ordinary steps): fluid velocity
    // per cell (3 floats) and the streamed h_obar of each reactive link
    float* tape_u;
    T* tape_h;            // (QG-1) * cap_b
    // phase-change events of the current step
    int cap_e;
    int* nev;
    int* ev_node;
    int* ev_kind;
    double* ev_val;       // 3 * cap_e
    double* ev_w;         // (QG-1) * cap_e
    int* evidx;           // NP, -1 when not an event
    // event log
    long long cap_log;
    long long* nlog;
    long long* log_step;
    long long* log_node;
    int* log_kind;
    long long* step;      // completed steps
    double* acc;          // [0] reacted (unused: k_bound keeps per-block partials)
    unsigned long long* facc;  // event-path sums in 64.64 fixed point: [0..1] Dirichlet inflow, [2..3] unpaid
    double* bacc;         // per-block partial ledger of k_bound: 2 * gridDim.x
    int* err;
    // compaction scratch
    int* blk;             // per chunk counts / offsets
    // Active-cell ("sparse") population storage: populations only for the
    // stored cells S (fluid, wet boundary and a margin of solid cells next to
    // them), numbered in three row-major ranges (cells fluid at the last
    // packing, boundary cells, margin) and blocked by 32 like the dense
    // layout.  Null / 0 for the dense layout.
    int sparse;
    long long cap_s;      // capacity of the stored-cell arrays (multiple of 32)
    int* ns;              // number of stored cells
    int* cmap;            // NP: compact index of a padded cell, -1 if not stored
    int* cid;             // cap_s: padded index of compact cell n
    uint32_t* nwc;        // cap_s: node word of compact cell n
    uint32_t* etab;       // neighbour table of each stored cell (see sp_cell_tables), blocked by 32
                          // cells: QF - 1 entries per cell (QG - 1 without a flow lattice)
    int* b_cn;            // cap_b: compact index of each wet boundary cell
    int* rown;            // NP: owner of a cell of the event region (RNONE outside), event path
    // local maintenance of the classes and lists after phase-change events
    // (null without phase change, or with LBRBC_LOCAL_LISTS=0): fluid-end
    // position of every cell (-1: none), the step's candidates, counters,
    // and the cells of the step's region
    int* fmap;            // NP
    int* candb;           // LOC_CAND_CAP: new wet boundary cells of the step
    int* candf;           // LOC_CAND_CAP: new fluid ends of the step
    int* lcnt;            // LC_N counters (LC_*)
    uint32_t* lmark;      // NP: step stamp of the cells of the region
    int* rlist;           // LOC_EV_MAX * cube: cells of the region
    int* repack;          // [0] set when a cell needs storage it does not have
    int* nrepack;         // repackings done
    // repacking targets (phase change only): new numbering and populations
    int* ns2;
    int* cmap2;
    int* cid2;
    uint8_t* scode;       // NP: range of each cell in the stored set
    int* stot;            // [3]: cells per range
    T* F2;
    T* G2;
};

template <class LG>
__device__ __forceinline__ double gweight(const Phys& p, int i) {
    if constexpr (LG::Q == 9) return LG::w(i);
    else return i == 0 ? p.gw0 : p.gw1;
}

template <class LG>
__device__ __forceinline__ double gcs2(const Phys& p) {
    if constexpr (LG::Q == 9) return 1.0 / 3.0;
    else return p.gcs2;
}

// ---------------------------------------------------------------------------
// Collision helpers (deviation form: a_i stores value_i - w_i * ref).
// ---------------------------------------------------------------------------
template <class L, typename T>
__device__ __forceinline__ void collide_flow(T (&f)[L::Q], T rho, T ux, T uy, T uz, const Phys& p,
                                             const PhysT<T>& q) {
    const T usq = ux * ux + uy * uy + uz * uz;
    const T drho = rho - T(1);
    if (!p.trt_f) {
        const T om = q.f_sym;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const T eu = T(L::cx(i)) * ux + T(L::cy(i)) * uy + T(L::cz(i)) * uz;
            const T feq = T(L::w(i)) * (drho + rho * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * usq));
            f[i] = f[i] - om * (f[i] - feq);
        }
    } else {
        const T op = q.f_sym, om = q.f_anti;
        {
            const T feq = T(L::w(0)) * (drho - rho * T(1.5) * usq);
            f[0] = f[0] - op * (f[0] - feq);
        }
#pragma unroll
        for (int i = 1; i <= L::H; ++i) {
            const int j = L::opp(i);
            const T eu = T(L::cx(i)) * ux + T(L::cy(i)) * uy + T(L::cz(i)) * uz;
            const T ep = T(L::w(i)) * (drho + rho * (T(4.5) * eu * eu - T(1.5) * usq));
            const T em = T(L::w(i)) * rho * T(3) * eu;
            const T fp = T(0.5) * (f[i] + f[j]), fm = T(0.5) * (f[i] - f[j]);
            const T dp = op * (fp - ep), dm = om * (fm - em);
            f[i] = f[i] - dp - dm;
            f[j] = f[j] - dp + dm;
        }
    }
}

template <class L, typename T>
__device__ __forceinline__ void collide_solute(T (&g)[L::Q], T C, T ux, T uy, T uz, const Phys& p,
                                               const PhysT<T>& q) {
    const T dc = C - q.cref;
    const T ics2 = q.ics2;
    if (!p.trt_g) {
        const T om = q.g_anti;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const T eu = T(L::cx(i)) * ux + T(L::cy(i)) * uy + T(L::cz(i)) * uz;
            const T w = q.gw[i];
            const T geq = w * dc + w * C * eu * ics2;
            g[i] = g[i] - om * (g[i] - geq);
        }
    } else {
        const T os = q.g_sym, oa = q.g_anti;
        g[0] = g[0] - os * (g[0] - q.gw[0] * dc);
#pragma unroll
        for (int i = 1; i <= L::H; ++i) {
            const int j = L::opp(i);
            const T eu = T(L::cx(i)) * ux + T(L::cy(i)) * uy + T(L::cz(i)) * uz;
            const T w = q.gw[i];
            const T ep = w * dc, em = w * C * eu * ics2;
            const T gp = T(0.5) * (g[i] + g[j]), gm = T(0.5) * (g[i] - g[j]);
            const T dp = os * (gp - ep), dm = oa * (gm - em);
            g[i] = g[i] - dp - dm;
            g[j] = g[j] - dp + dm;
        }
    }
}

}  // namespace lbrbc
#include "pairs.cuh"
namespace lbrbc {

// ---------------------------------------------------------------------------
// Fluid cells: stream (read side), boundary rules, moments, collide, write.
// Element indices are 32-bit (checked at creation: Q * NP < 2^32), all loads
// of both lattices are issued before any arithmetic, and cells without an
// inactive source take a path with no per-direction tests.
// ---------------------------------------------------------------------------
struct Nbr32 {
    int xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Nbr32 nbr32(const Geo& g, int x, int y, int z) {
    Nbr32 d;
    const int sy = g.SX, sz = g.SX * g.SY;
    d.xp = (g.per_x && x == g.nx - 1) ? -(g.nx - 1) : 1;
    d.xm = (g.per_x && x == 0) ? (g.nx - 1) : -1;
    d.yp = (g.per_y && y == g.ny - 1) ? -(g.ny - 1) * sy : sy;
    d.ym = (g.per_y && y == 0) ? (g.ny - 1) * sy : -sy;
    d.zp = (g.per_z && z == g.nz - 1) ? -(g.nz - 1) * sz : sz;
    d.zm = (g.per_z && z == 0) ? (g.nz - 1) * sz : -sz;
    return d;
}

template <class L>
__device__ __forceinline__ uint32_t off32(const Nbr32& d, int i) {
    return (uint32_t)((L::cx(i) > 0 ? d.xp : (L::cx(i) < 0 ? d.xm : 0)) +
                      (L::cy(i) > 0 ? d.yp : (L::cy(i) < 0 ? d.ym : 0)) +
                      (L::cz(i) > 0 ? d.zp : (L::cz(i) < 0 ? d.zm : 0)));
}

// Population layout: cells in blocks of 32 consecutive padded indices (a
// row segment: rows start at multiples of 32), the Q populations of a block
// stored one after the other, 32 values each.  Slot of population i of cell
// id: (id - id % 32) Q + 32 i + id % 32.  A warp's 32 cells read and write
// one 128-byte line per population, and the Q lines of a block are
// contiguous, so a warp streams Q * 128 bytes from one region instead of
// one line from each of Q arrays.
template <class L>
__host__ __device__ __forceinline__ uint32_t pslot(int i, uint32_t id) {
    return (id & ~31u) * (uint32_t)L::Q + (uint32_t)i * 32u + (id & 31u);
}
template <class L>
__host__ __device__ __forceinline__ long long pslot64(int i, long long id) {
    return (id & ~31LL) * (long long)L::Q + (long long)i * 32 + (id & 31LL);
}

// Slots of a cell and of its neighbours in the blocked layout.  Rows start
// at multiples of 32 and y / z neighbour offsets are multiples of the row
// length, so a y / z shift moves whole blocks: the slot of population j at
// id + e is the slot of j at the x-shifted cell plus the y / z offset times
// Q.  Per cell: the population-0 slots of the cell and of its x neighbours
// (periodic wrap included) and the y / z offsets scaled by Q.
template <class L>
struct Blk {
    uint32_t b0, bxp, bxm;
    uint32_t yp, ym, zp, zm;
};

template <class L>
__device__ __forceinline__ Blk<L> blk_of(uint32_t id, const Nbr32& d) {
    Blk<L> k;
    k.b0 = pslot<L>(0, id);
    k.bxp = pslot<L>(0, id + (uint32_t)d.xp);
    k.bxm = pslot<L>(0, id + (uint32_t)d.xm);
    k.yp = (uint32_t)d.yp * (uint32_t)L::Q;
    k.ym = (uint32_t)d.ym * (uint32_t)L::Q;
    k.zp = (uint32_t)d.zp * (uint32_t)L::Q;
    k.zm = (uint32_t)d.zm * (uint32_t)L::Q;
    return k;
}

// slot of population j at the neighbour id + e_n
template <class L>
__device__ __forceinline__ uint32_t nslot(const Blk<L>& k, int j, int n) {
    uint32_t s = (L::cx(n) > 0 ? k.bxp : (L::cx(n) < 0 ? k.bxm : k.b0)) + (uint32_t)j * 32u;
    if (L::cy(n) > 0) s += k.yp;
    else if (L::cy(n) < 0) s += k.ym;
    if (L::cz(n) > 0) s += k.zp;
    else if (L::cz(n) < 0) s += k.zm;
    return s;
}

// Slot read by a cell for direction i: its own slot i (even step) or the
// slot opp(i) of the source x - e_i (odd step); an inactive source swaps
// the two (the value there is the cell's own f*_opp(i)).
template <class L, bool ODD>
__device__ __forceinline__ uint32_t read_slot(const Blk<L>& k, int i, bool inactive) {
    const uint32_t own = k.b0 + (uint32_t)i * 32u;
    const uint32_t nbr = nslot<L>(k, L::opp(i), L::opp(i));
    return (ODD == inactive) ? own : nbr;
}

template <class L, bool ODD>
__device__ __forceinline__ uint32_t write_slot(const Blk<L>& k, int i) {
    return ODD ? nslot<L>(k, i, i) : k.b0 + (uint32_t)L::opp(i) * 32u;
}

template <typename T>
__device__ __forceinline__ T ld_pop(const T* p) {
#if LBRBC_STREAM_HINT
    return __ldcs(p);
#else
    return *p;
#endif
}
template <typename T>
__device__ __forceinline__ void st_pop(T* p, T v) {
#if LBRBC_STREAM_HINT
    __stcs(p, v);
#else
    *p = v;
#endif
}

// Node-word flags of fluid cells on the inlet (x = 0) and outlet (x = nx - 1)
// faces of an open x axis.
constexpr uint32_t NW_INLET = 1u << 30;
constexpr uint32_t NW_OUTLET = 1u << 31;

// Where a fluid cell's pre-collision populations come from and where its
// post-collision ones go.  GlobalSrc: the dense AA layout (writes never
// depend on the geometry).
template <typename T, class LF, class LG, bool ODD>
struct GlobalSrc {
    static constexpr bool kTargets = false;  // writes do not depend on the neighbours' classes
    static constexpr bool kBranchFree = false;  // reads pick a slot per direction
    const T* __restrict__ F;
    const T* __restrict__ G;
    Blk<LF> kF;
    Blk<LG> kG;
    T* Fw;
    T* Gw;
    __device__ __forceinline__ T f(int i, bool inactive) const { return ld_pop(F + read_slot<LF, ODD>(kF, i, inactive)); }
    __device__ __forceinline__ T g(int i, bool inactive) const { return ld_pop(G + read_slot<LG, ODD>(kG, i, inactive)); }
    __device__ __forceinline__ void fput(int i, T v, bool) const { st_pop(Fw + write_slot<LF, ODD>(kF, i), v); }
    __device__ __forceinline__ void gput(int i, T v, bool) const { st_pop(Gw + write_slot<LG, ODD>(kG, i), v); }
};

// Stencil of the neighbour table of the active-cell layout: the flow lattice
// when there is one (its directions include the solute lattice's), else the
// solute lattice.
template <class LF, class LG>
struct Stencil {
    using L = LF;
};
template <class LG>
struct Stencil<NoFlow, LG> {
    using L = LG;
};

// Stencil direction with the velocity of direction j of lattice L.
template <class LS, class L>
__host__ __device__ constexpr int sdir(int j) {
    for (int s = 0; s < LS::Q; ++s)
        if (LS::cx(s) == L::cx(j) && LS::cy(s) == L::cy(j) && LS::cz(s) == L::cz(j)) return s;
    return -1;
}

// Active-cell layout, own-slot convention.  Even step: a cell reads its own
// slot i and writes f*_i into its own slot opp(i).  Odd step: it reads
// f_i from slot opp(i) of the source x - e_i (its own slot i when the source
// is inactive: the value there is its own f*_opp(i), halfway bounce-back) and
// writes f*_i into slot i of x + e_i (its own slot opp(i) when that target
// is inactive).  No population ever lives in an inactive cell, so the
// storage holds the stored cells only.
//
// The odd step's addresses come from the effective-base table: for each
// neighbour direction d, E[d] is the neighbour's block base (m - m % 32) Q +
// m % 32 when the neighbour is active for the lattice, else the cell's own
// base plus 32 (opp(d) - d).  The read of direction opp(d) and the write of
// direction d then both use slot E[d] + 32 d, active neighbour or not, so
// the odd step needs no per-direction test.
template <class L>
__host__ __device__ __forceinline__ uint32_t pbase(uint32_t n) {
    return (n & ~31u) * (uint32_t)L::Q + (n & 31u);
}

// Position of entry k of cell n in the blocked effective-base table.
__device__ __forceinline__ size_t etab_at(uint32_t n, int nt, int k) {
    return (size_t)(n & ~31u) * (size_t)nt + (size_t)k * 32u + (n & 31u);
}

// Table entries per stored cell: one per flow direction (with a flow
// lattice), else one per solute direction.  A flow direction whose velocity
// is also a solute velocity ("shared", the 6 axis directions of D3Q19 /
// D3Q7) holds the compact index of the neighbour when it is not solid (it is
// then stored), and the reads and writes of both lattices along it test the
// node word; every other direction holds the folded effective base of its
// lattice.  One table thus serves both lattices (96 -> 72 B per cell in 3D).
template <class LF, class LG>
__host__ __device__ constexpr int tab_entries() {
    return LF::Q > 0 ? LF::Q - 1 : LG::Q - 1;
}
template <class LF, class LG>
__host__ __device__ constexpr bool shared_dir(int k) {
    if constexpr (LF::Q == 0) {
        return false;
    } else {
        for (int j = 1; j < LG::Q; ++j)
            if (LG::cx(j) == LF::cx(k) && LG::cy(j) == LF::cy(k) && LG::cz(j) == LF::cz(k)) return true;
        return false;
    }
}

template <typename T, class LF, class LG, bool ODD>
struct SparseSrc {
    static constexpr bool kTargets = false;  // inactive targets are handled inside (table or node word)
    static constexpr bool kBranchFree = true;  // no branch: per-direction selects of addresses
    static constexpr int NT = tab_entries<LF, LG>();
    const T* __restrict__ F;
    const T* __restrict__ G;
    const uint32_t* __restrict__ et;  // this cell's table entries (entry k at et[32 k])
    uint32_t n;
    T* Fw;
    T* Gw;
    uint32_t w;  // node word: inactive sources of both lattices
    __device__ __forceinline__ uint32_t e(int k) const { return __ldg(et + 32 * k); }
    // slot E[k] + 32 d of a folded entry: the sum is formed in 32-bit
    // unsigned arithmetic (an inactive neighbour's entry wraps around and the
    // sum comes back to the own slot) before it offsets a pointer
    __device__ __forceinline__ uint32_t slot(int k, int d) const { return e(k) + 32u * (uint32_t)d; }
    // slot of direction d of lattice L in the neighbour of shared flow
    // direction k, or the own slot `own` when inactive
    template <class L>
    __device__ __forceinline__ uint32_t shared(int k, int d, bool inactive, uint32_t own) const {
        const uint32_t m = e(k);
        return inactive ? own : pbase<L>(m) + 32u * (uint32_t)d;
    }
    __device__ __forceinline__ T ld_nbr(const T* p) const {
#if LBRBC_SP_NBR_HINT
        return ld_pop(p);
#else
        return *p;
#endif
    }
    __device__ __forceinline__ T f(int i, bool) const {
        if (!ODD || i == 0) return ld_pop(F + pslot<LF>(i, n));
        const int d = LF::opp(i);
        if (shared_dir<LF, LG>(d))
            return ld_nbr(F + shared<LF>(d - 1, d, (w >> (FBIT + i - 1)) & 1u, pslot<LF>(i, n)));
        return ld_nbr(F + slot(d - 1, d));
    }
    __device__ __forceinline__ T g(int i, bool) const {
        if (!ODD || i == 0) return ld_pop(G + pslot<LG>(i, n));
        const int d = LG::opp(i);
        if constexpr (LF::Q > 0) {
            const int k = sdir<LF, LG>(d);
            return ld_nbr(G + shared<LG>(k - 1, d, (w >> (GBIT + i - 1)) & 1u, pslot<LG>(i, n)));
        } else {
            return ld_nbr(G + slot(d - 1, d));
        }
    }
    __device__ __forceinline__ void st_nbr(T* p, T v) const {
#if LBRBC_SP_NBR_STORE_HINT
        st_pop(p, v);
#else
        *p = v;
#endif
    }
    __device__ __forceinline__ void fput(int i, T v, bool) const {
        if (!ODD || i == 0) {
            st_pop(Fw + pslot<LF>(LF::opp(i), n), v);
        } else if (shared_dir<LF, LG>(i)) {
            st_nbr(Fw + shared<LF>(i - 1, i, (w >> (FBIT + LF::opp(i) - 1)) & 1u, pslot<LF>(LF::opp(i), n)), v);
        } else {
            st_nbr(Fw + slot(i - 1, i), v);
        }
    }
    __device__ __forceinline__ void gput(int i, T v, bool) const {
        if (!ODD || i == 0) {
            st_pop(Gw + pslot<LG>(LG::opp(i), n), v);
        } else if constexpr (LF::Q > 0) {
            const int k = sdir<LF, LG>(i);
            st_nbr(Gw + shared<LG>(k - 1, i, (w >> (GBIT + LG::opp(i) - 1)) & 1u, pslot<LG>(LG::opp(i), n)), v);
        } else {
            st_nbr(Gw + slot(i - 1, i), v);
        }
    }
};

// One fluid cell of one step with node word w: stream (read side), open
// boundaries, moments, collision, write.  id is the cell's padded index
// (used for the adjoint tape), (y, z) its position (used on open x faces).
// Shared by the dense, active-cell and batched sweeps.
template <typename T, class LF, class LG, bool ODD, class Src>
__device__ __forceinline__ void fluid_cell_src(const Dev<T>& a, const Phys& p, const PhysT<T>& q, uint32_t id,
                                               uint32_t w, const Src& src, bool inlet, bool outlet, int y, int z) {
    constexpr int QF = LF::Q, QG = LG::Q;
    const Geo& g = a.geo;
    const bool plain = ((w & ~(NW_INLET | NW_OUTLET)) >> FBIT) == 0u && !inlet && !outlet;

    // Warps whose cells all read the plain slots take a path with no
    // per-direction tests; the others pick, per direction, the plain slot or
    // the swapped one of an inactive source.  (All sources active means all
    // targets active too: the sources of a cell are all its neighbours.)
    const bool wplain = Src::kBranchFree || __all_sync(__activemask(), plain);
    T f[QF > 0 ? QF : 1];
    T gg[QG];
    if (wplain) {
#pragma unroll
        for (int i = 0; i < QF; ++i) f[i] = src.f(i, false);
#pragma unroll
        for (int i = 0; i < QG; ++i) gg[i] = src.g(i, false);
    } else {
#pragma unroll
        for (int i = 0; i < QF; ++i) {
            const bool wall = i > 0 && ((w >> (FBIT + i - 1)) & 1u);
            f[i] = src.f(i, wall);
        }
#pragma unroll
        for (int i = 0; i < QG; ++i) {
            const bool wall = i > 0 && ((w >> (GBIT + i - 1)) & 1u);
            gg[i] = src.g(i, wall);
        }
    }
    if (!plain) {
        const int face = y + g.ny * z;
        if constexpr (QF > 0) {
            if (inlet) {
                // moving-wall bounce-back with the inlet velocity (rho_w = 1):
                // f_i += 2 (w_i / cs^2) c_x u_in, with the exact-sum coefficients
                // so that the injected mass is exactly u_in per cell and step
                const T uin = T(a.inlet_ux[face]);
#pragma unroll
                for (int i = 1; i < QF; ++i)
                    if (LF::cx(i) > 0) f[i] += T(2 * LF::cx(i)) * mom_coef<LF, T>(i) * uin;
            }
            if (outlet) {
                // pressure anti-bounce-back at rho_out with the previous velocity,
                // in deviation form: rho_out (1 + X) - 1 = (rho_out - 1) + rho_out X
                // (the plain form loses all but ~1e-2 of X ~ u^2 in FP32)
                const T uo0 = T(a.side[4 * face + 0]), uo1 = T(a.side[4 * face + 1]), uo2 = T(a.side[4 * face + 2]);
                const T uq = uo0 * uo0 + uo1 * uo1 + uo2 * uo2;
#pragma unroll
                for (int i = 1; i < QF; ++i)
                    if (LF::cx(i) < 0) {
                        const T eu = T(LF::cx(i)) * uo0 + T(LF::cy(i)) * uo1 + T(LF::cz(i)) * uo2;
                        f[i] = -f[i] + T(2.0 * LF::w(i)) * (q.rho_out_d + q.rho_out * (T(4.5) * eu * eu - T(1.5) * uq));
                    }
            }
        }
        if (inlet) {
#pragma unroll
            for (int i = 1; i < QG; ++i)
                if (LG::cx(i) > 0) gg[i] = -gg[i] + T(2) * q.gw[i] * q.c_in_d;
        }
        if (outlet) {
            const T co_d = T(a.side[4 * face + 3] - p.cref);  // previous C minus the reference, in FP64
#pragma unroll
            for (int i = 1; i < QG; ++i)
                if (LG::cx(i) < 0) gg[i] = -gg[i] + T(2) * q.gw[i] * co_d;
        }
    }

    T ux = T(0), uy = T(0), uz = T(0), rho = T(1);
    if constexpr (QF > 0) {
        flow_pairs<LF, T>(reinterpret_cast<T(&)[QF]>(f), rho, ux, uy, uz, p, q);
        if (!Src::kTargets || wplain) {
#pragma unroll
            for (int i = 0; i < QF; ++i) src.fput(i, f[i], false);
        } else {
#pragma unroll
            for (int i = 0; i < QF; ++i) src.fput(i, f[i], i > 0 && ((w >> (FBIT + LF::opp(i) - 1)) & 1u));
        }
    }
    T C;
    solute_pairs<LG, T>(gg, C, ux, uy, uz, p, q);
    if (!(rho > T(0)) || !isfinite(C)) *a.err |= ERR_NUMERIC;
    if (a.tape_u) {
        a.tape_u[3 * (size_t)id] = (float)ux;
        a.tape_u[3 * (size_t)id + 1] = (float)uy;
        a.tape_u[3 * (size_t)id + 2] = (float)uz;
    }
    if (!Src::kTargets || wplain) {
#pragma unroll
        for (int i = 0; i < QG; ++i) src.gput(i, gg[i], false);
    } else {
#pragma unroll
        for (int i = 0; i < QG; ++i) src.gput(i, gg[i], i > 0 && ((w >> (GBIT + LG::opp(i) - 1)) & 1u));
    }
    if (outlet) {
        const int face = y + g.ny * z;
        a.side[4 * face + 0] = (double)ux;
        a.side[4 * face + 1] = (double)uy;
        a.side[4 * face + 2] = (double)uz;
        a.side[4 * face + 3] = (double)C;
    }
}

template <typename T, class LF, class LG, bool ODD>
__device__ __forceinline__ void fluid_cell(const Dev<T>& a, const Phys& p, const PhysT<T>& q, int x, int y, int z) {
    const Geo& g = a.geo;
    const uint32_t id = (uint32_t)g.idx(x, y, z);
    const uint32_t w = a.nw[id];
    if ((w & 3u) != CLS_FLUID) return;
    const Nbr32 d = nbr32(g, x, y, z);
    const GlobalSrc<T, LF, LG, ODD> src{a.F, a.G, blk_of<LF>(id, d), blk_of<LG>(id, d), a.F, a.G};
    const bool inlet = g.open_x && x == 0;
    const bool outlet = g.open_x && x == g.nx - 1;
    fluid_cell_src<T, LF, LG, ODD>(a, p, q, id, w, src, inlet, outlet, y, z);
}

template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(FLUID_BLOCK, sizeof(T) == 4 ? 8 : 5) k_fluid(const Dev<T> a, const Phys p, const PhysT<T> q) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.geo.nx) return;
    fluid_cell<T, LF, LG, ODD>(a, p, q, x, blockIdx.y, blockIdx.z);
}

// The fluid sweep of the active-cell layout: one thread per stored cell in
// compact order (cells fluid at the last packing first, row-major), so a
// warp's 32 cells read and write whole 128-byte population lines whatever
// the geometry.
// One stored cell n of the active-cell layout (nothing unless it is fluid);
// shared by the single-domain and batched sweeps.
template <typename T, class LF, class LG, bool ODD>
__device__ __forceinline__ void sparse_cell(const Dev<T>& a, const Phys& p, const PhysT<T>& q, int n) {
    const uint32_t w = a.nwc[n];
    if ((w & 3u) != CLS_FLUID) return;
    const bool inlet = (w & NW_INLET) != 0u, outlet = (w & NW_OUTLET) != 0u;
    uint32_t id = 0;
    int x = 0, y = 0, z = 0;
    if (inlet || outlet || a.tape_u) {
        id = (uint32_t)a.cid[n];
        coords(a.geo, id, x, y, z);
    }
    constexpr int NT = SparseSrc<T, LF, LG, ODD>::NT;
    const SparseSrc<T, LF, LG, ODD> src{a.F, a.G, a.etab + etab_at((uint32_t)n, NT, 0), (uint32_t)n, a.F, a.G, w};
    fluid_cell_src<T, LF, LG, ODD>(a, p, q, id, w, src, inlet, outlet, y, z);
}

template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(FLUID_BLOCK, sizeof(T) == 4 ? LBRBC_SP_BLOCKS : 5) k_fluid_sp(const Dev<T> a, const Phys p, const PhysT<T> q) {
    const int ns = *a.ns;
#if LBRBC_SP_L2PF
    // odd step: ask the L2 for the table rows and node words of the block
    // LBRBC_SP_L2PF blocks ahead, which the scheduler starts about one wave
    // later (a hint: nothing waits on it; rows inside the allocation, every
    // range 16-byte aligned and a multiple of 16 bytes)
    if (ODD && threadIdx.x == 0) {
        constexpr int NT = tab_entries<LF, LG>();
        const long long c0 = ((long long)blockIdx.x + LBRBC_SP_L2PF) * blockDim.x;
        if (c0 < ns) {
            const long long rows = min((long long)blockDim.x, a.cap_s - c0);  // a multiple of 64
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.etab + (size_t)c0 * NT),
                         "r"((unsigned)(rows * NT * 4)) : "memory");
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.nwc + c0), "r"((unsigned)(rows * 4))
                         : "memory");
        }
    }
#endif
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < ns; n += gridDim.x * blockDim.x)
        sparse_cell<T, LF, LG, ODD>(a, p, q, n);
}

// The same sweep over the compacted fluid cells: every lane of a warp has a
// fluid cell, which pays off in porous media where most 32-cell row
// segments of the dense grid are partly solid.
__device__ __forceinline__ void unpack32(uint32_t v, int& x, int& y, int& z) {
    x = (int)(v & 2047u);
    y = (int)((v >> 11) & 2047u);
    z = (int)(v >> 22);
}

template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(FLUID_BLOCK) k_fluid_list(const Dev<T> a, const Phys p, const PhysT<T> q) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= *a.nfl) return;
    int x, y, z;
    unpack32(a.fl_xyz[e], x, y, z);
    fluid_cell<T, LF, LG, ODD>(a, p, q, x, y, z);
}

// ---------------------------------------------------------------------------
// Order-independent sums of the event path: each term is rounded once to a
// 128-bit two's-complement fixed-point number with 64 fractional bits
// (truncating below 2^-64, |term| < 2^63) and added with integer atomics, so
// the total does not depend on the order in which threads add their terms.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fx_add(unsigned long long* a, double v) {
    if (v == 0.0) return;
    const double m = fabs(v);
    unsigned long long hi = (unsigned long long)floor(m);
    unsigned long long lo = (unsigned long long)((m - (double)hi) * 18446744073709551616.0);
    if (v < 0.0) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const unsigned long long old = atomicAdd(&a[0], lo);
    atomicAdd(&a[1], hi + (old + lo < old ? 1ull : 0ull));
}

__host__ __device__ __forceinline__ double fx_value(const unsigned long long* a) {
    return (double)(long long)a[1] + (double)a[0] * (1.0 / 18446744073709551616.0);
}

// ---------------------------------------------------------------------------
// Event queue with warp-aggregated atomics.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void push_event(int* nev, int cap, int* ev_node, int* ev_kind, int* err, int node,
                                           int kind) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(nev, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    const int pos = base + __popc(mask & ((1u << lane) - 1u));
    if (pos < cap) {
        ev_node[pos] = node;
        ev_kind[pos] = kind;
    } else {
        atomicOr(err, ERR_OVERFLOW);
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Exact sum of differences of stored populations.  FP64 storage: plain FP64.
// FP32 storage: float-float accumulation (TwoSum), exact for the differences
// and accurate to ~2^-48 for the sum, converted to FP64 once per cell, so the
// FP32 path issues almost no FP64 instructions (GB300 runs FP64 at a small
// fraction of the FP32 rate).
template <typename T>
struct DiffSum {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s += a - b; }
    __device__ __forceinline__ void merge(const DiffSum& o) { s += o.s; }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ int sign() const { return s > 0.0 ? 1 : (s < 0.0 ? -1 : 0); }
    __device__ __forceinline__ double approx() const { return s; }
    __device__ __forceinline__ void shfl_down(int off) { s = __shfl_down_sync(0xffffffffu, s, off); }
};
template <>
struct DiffSum<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float d = a - b;  // a - b = d + e exactly
        const float bv = d - a;
        const float e = (a - (d - bv)) + (-b - bv);
        const float s2 = hi + d;  // hi + d = s2 + t exactly
        const float bb = s2 - hi;
        const float t = (hi - (s2 - bb)) + (d - bb);
        const float tl = t + (lo + e);
        hi = s2 + tl;
        lo = tl - (hi - s2);
    }
    __device__ __forceinline__ void merge(const DiffSum& o) {
        const float s2 = hi + o.hi;
        const float bb = s2 - hi;
        const float t = (hi - (s2 - bb)) + (o.hi - bb);
        const float tl = t + (lo + o.lo);
        hi = s2 + tl;
        lo = tl - (hi - s2);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ int sign() const {
        const float v = hi != 0.f ? hi : lo;
        return v > 0.f ? 1 : (v < 0.f ? -1 : 0);
    }
    __device__ __forceinline__ float approx() const { return hi + lo; }
    __device__ __forceinline__ void shfl_down(int off) {
        hi = __shfl_down_sync(0xffffffffu, hi, off);
        lo = __shfl_down_sync(0xffffffffu, lo, off);
    }
};

template <typename T>
__device__ __forceinline__ DiffSum<T> warp_merge(DiffSum<T> v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DiffSum<T> w = v;
        w.shfl_down(o);
        v.merge(w);
    }
    return v;
}

// phi <= 0 and phi >= 1 on the bit pattern of a (non-NaN) double: integer
// compares, no FP64 instruction.
__device__ __forceinline__ bool dle0(double v) { return __double_as_longlong(v) <= 0LL; }
__device__ __forceinline__ bool dge1(double v) { return __double_as_longlong(v) >= 0x3FF0000000000000LL; }

// ---------------------------------------------------------------------------
// Wet boundary cells (compacted list): solute stream, Eq. general_RBC on each
// link to a fluid cell (all links from the streamed values), ledger
// m_l = g_o(new) - g_o(streamed), collision with u = 0, Eq.
// solidFractionUpdate (adjacent growth, conserving sign).  FP64 is used only
// where the ledger needs it (GB300 runs FP64 at a small fraction of FP32):
// each m_l is the exact FP64 difference of two stored values, the shares
// need one division per cell.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t pack_xyz(int x, int y, int z) {
    return (uint64_t)(uint32_t)x | ((uint64_t)(uint32_t)y << 21) | ((uint64_t)(uint32_t)z << 42);
}
__device__ __forceinline__ void unpack_xyz(uint64_t v, int& x, int& y, int& z) {
    x = (int)(v & 0x1fffffu);
    y = (int)((v >> 21) & 0x1fffffu);
    z = (int)((v >> 42) & 0x1fffffu);
}

// One wet boundary cell (list entry e) of one step; adds its reacted mass
// (or Dirichlet inflow) to racc (dacc).
// Solute slots of a wet boundary cell: dense AA layout (from the cell's
// coordinates) or active-cell layout (from its compact index and the
// neighbour table; LF only names the table's stencil).
template <typename T, class LF, class LG, bool ODD, bool SP>
struct BoundSlots {
    Blk<LG> kb;
    uint32_t n;
    const uint32_t* et;
    __device__ __forceinline__ BoundSlots(const Dev<T>& a, int e) {
        if constexpr (SP) {
            n = (uint32_t)a.b_cn[e];
            et = a.etab + etab_at(n, tab_entries<LF, LG>(), 0);
        } else {
            int x, y, z;
            unpack_xyz(a.b_xyz[e], x, y, z);
            const uint32_t b = (uint32_t)a.geo.idx(x, y, z);
            kb = blk_of<LG>(b, nbr32(a.geo, x, y, z));
        }
    }
    // (active-cell layout with a flow lattice: the solute directions are
    // shared table entries holding the neighbour's compact index, selected by
    // the cell's inactive-source bits; without one, folded solute entries)
    __device__ __forceinline__ uint32_t rd(int i, bool inactive) const {
        if constexpr (SP) {
            if (!ODD || i == 0) return pslot<LG>(i, n);
            const int d = LG::opp(i);
            if constexpr (LF::Q > 0) {
                const uint32_t m = et[32 * (sdir<LF, LG>(d) - 1)];
                return inactive ? pslot<LG>(i, n) : pbase<LG>(m) + 32u * (uint32_t)d;
            } else {
                return et[32 * (d - 1)] + 32u * (uint32_t)d;
            }
        } else {
            return read_slot<LG, ODD>(kb, i, inactive);
        }
    }
    __device__ __forceinline__ uint32_t wr(int i, bool inactive) const {
        if constexpr (SP) {
            if (!ODD || i == 0) return pslot<LG>(LG::opp(i), n);
            if constexpr (LF::Q > 0) {
                const uint32_t m = et[32 * (sdir<LF, LG>(i) - 1)];
                return inactive ? pslot<LG>(LG::opp(i), n) : pbase<LG>(m) + 32u * (uint32_t)i;
            } else {
                return et[32 * (i - 1)] + 32u * (uint32_t)i;
            }
        } else {
            return write_slot<LG, ODD>(kb, i);
        }
    }
};

template <typename T, class LF, class LG, bool ODD, bool SP>
__device__ __forceinline__ void bound_entry(const Dev<T>& a, const Phys& p, const PhysT<T>& q, int e, DiffSum<T>& racc,
                                            DiffSum<T>& dacc) {
    constexpr int Q = LG::Q;
    T* __restrict__ G = a.G;
    const T cref = q.cref;
    const T gam = q.gamma, ics2 = q.ics2;
    const uint32_t bw = a.b_word[e];
    if (bw & BW_DEAD) return;
    const BoundSlots<T, LF, LG, ODD, SP> kb(a, e);
    const uint32_t b = (uint32_t)a.b_idx[e];
    T gp[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool inactive = i > 0 && ((bw >> (i - 1)) & 1u);
        gp[i] = G[kb.rd(i, inactive)];
    }
    T gq[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) gq[i] = gp[i];
    const bool dir = (bw & BW_DIRICHLET) != 0u;
    const T kr = a.b_krate ? T(a.b_krate[e]) : q.k_r;
    T mabs[Q];
    DiffSum<T> ms;
    T S = T(0);
#pragma unroll
    for (int o = 1; o < Q; ++o) {
        mabs[o] = T(0);
        if (!((bw >> (BW_LINK + o - 1)) & 1u)) continue;
        const T gt = gp[LG::opp(o)];
        const T w2 = T(2) * q.gw[o];
        T val;
        if (dir) {
            val = -gt + w2 * q.c_dir_d;  // anti-bounce-back, C_wall = c_dirichlet
        } else {
            const T kap = a.b_kappa[(long long)(o - 1) * a.cap_b + e];
            T k = T(0);
            bool inf = false;
            if (p.scheme == 0) k = gam * kr * kap * ics2;
            else if (p.scheme == 1) k = kr * kap * ics2;
            else if (p.scheme == 2) {
                if (kap > T(0)) k = gam * kr * ics2 / kap;
                else inf = true;
            } else inf = true;
            if (kr == T(0)) {  // k_r = 0: inert under every scheme
                k = T(0);
                inf = false;
            }
            if (inf) val = -gt + w2 * q.c_eq_d;
            else {
                const T ik = T(1) / (T(1) + k);
                val = k * ik * w2 * q.c_eq_d + (T(1) - k) * ik * gt;
            }
        }
        ms.add(val, gp[o]);
        mabs[o] = fabs(val - gp[o]);
        if (a.tape_h) a.tape_h[(long long)(o - 1) * a.cap_b + e] = gt;
        S += mabs[o];
        gq[o] = val;
    }
    T sc = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) sc += gq[i];
    const T C = cref + sc;
    if (!isfinite(C)) *a.err |= ERR_NUMERIC;
    collide_solute<LG, T>(gq, C, T(0), T(0), T(0), p, q);
    {
        // the collision conserves C: the rest population takes the remainder
        // (rounded weights would otherwise create solute in proportion to C)
        T rest = sc;
#pragma unroll
        for (int i = 1; i < Q; ++i) rest -= gq[i];
        gq[0] = rest;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) G[kb.wr(i, i > 0 && ((bw >> (LG::opp(i) - 1)) & 1u))] = gq[i];
    const int sg = ms.sign();
    if (dir) {
        dacc.merge(ms);
        return;
    }
    racc.merge(ms);
    double ph = 0.0;
    if (sg > 0 || p.phase_change) ph = a.phi[b];
    if (sg > 0) {  // dissolution: the boundary cell loses solid (the only FP64 arithmetic here)
        ph -= p.Vm * ms.value();
        a.phi[b] = ph;
    }
    const T r = (sg < 0 && S > T(0)) ? q.neg_vm * T(ms.approx()) / S : T(0);
    // shares in list order; each fluid end gathers its own.  Every direction
    // is written (0 without a link), so a warp writes whole sectors and the
    // L2 need not fetch partly written ones from DRAM.
#pragma unroll
    for (int o = 1; o < Q; ++o) a.b_share[(long long)(o - 1) * a.cap_b + e] = r * mabs[o];
    if (p.phase_change && dle0(ph)) push_event(a.nev, a.cap_e, a.ev_node, a.ev_kind, a.err, (int)b, EV_DISSOLVE);
}

template <typename T, class LF, class LG, bool ODD, bool SP>
__global__ void __launch_bounds__(LIST_BLOCK, LBRBC_BOUND_BLOCKS) k_bound(const Dev<T> a, const Phys p, const PhysT<T> q) {
    const int n = *a.nb;
    DiffSum<T> racc, dacc;  // reacted mass and Dirichlet inflow of this thread
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        bound_entry<T, LF, LG, ODD, SP>(a, p, q, e, racc, dacc);
    // each block owns its two accumulators (fixed grid): no atomics and a
    // fixed summation order
    __shared__ __align__(16) unsigned char red_raw[2 * (LIST_BLOCK / 32) * sizeof(DiffSum<T>)];
    DiffSum<T>* red = reinterpret_cast<DiffSum<T>*>(red_raw);  // [2][LIST_BLOCK / 32]
    racc = warp_merge(racc);
    dacc = warp_merge(dacc);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = racc;
        red[LIST_BLOCK / 32 + (threadIdx.x >> 5)] = dacc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        DiffSum<T> r = red[0], d = red[LIST_BLOCK / 32];
        for (int k = 1; k < LIST_BLOCK / 32; ++k) {
            r.merge(red[k]);
            d.merge(red[LIST_BLOCK / 32 + k]);
        }
        if (r.sign() != 0 || d.sign() != 0) {
            a.bacc[2 * blockIdx.x] += r.value();
            a.bacc[2 * blockIdx.x + 1] += d.value();
        }
    }
}

// Fluid cells at the ends of reactive links gather their precipitation
// shares (fixed direction order) and test the phi >= 1 threshold.
// One fluid cell at the end of reactive links (list entry e): gathers its
// precipitation shares in fixed direction order and tests phi >= 1.
template <typename T, class LG>
__device__ __forceinline__ void fend_entry(const Dev<T>& a, const Phys& p, int e) {
    const long long f = a.f_idx[e];
    if (f < 0) return;  // no longer a fluid end
    T acc = T(0);
#pragma unroll
    for (int o = 1; o < LG::Q; ++o) {
        const int s = a.f_src[(long long)(o - 1) * a.cap_f + e];
        if (s >= 0) acc += a.b_share[s];
    }
    double ph = a.phi[f];
    if (acc != T(0)) {
        ph += (double)acc;
        a.phi[f] = ph;
    }
    if (p.phase_change && dge1(ph)) push_event(a.nev, a.cap_e, a.ev_node, a.ev_kind, a.err, (int)f, EV_PRECIPITATE);
}

template <typename T, class LG>
__global__ void __launch_bounds__(LIST_BLOCK) k_fend(const Dev<T> a, const Phys p) {
    const int n = *a.nf;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) fend_entry<T, LG>(a, p, e);
}

// ---------------------------------------------------------------------------
// Post-collision populations at their plain AA positions.
// ---------------------------------------------------------------------------
// Slot of the post-collision population f*_i of cell id in the current state
// (lastodd: the last step was odd).  Dense layout: the AA position.  Active-
// cell layout (own-slot convention): after an even step the cell's own slot
// opp(i); after an odd step slot i of the neighbour id + e_i when that
// neighbour is active for the lattice (flow: fluid; solute: not solid), else
// the own slot opp(i).  FLOW: L is the flow lattice.
template <class L, bool FLOW, typename T>
__device__ __forceinline__ long long post_slot(const Dev<T>& a, long long id, const Nbr& d, int i, bool lastodd) {
    if (!a.sparse) return lastodd ? pslot64<L>(i, id + off<L>(d, i)) : pslot64<L>(L::opp(i), id);
    if (lastodd && i != 0) {
        const long long nb = id + off<L>(d, i);
        const uint32_t c = a.nw[nb] & 3u;
        if (FLOW ? c == CLS_FLUID : c != CLS_SOLID) return pslot64<L>(i, a.cmap[nb]);
    }
    return pslot64<L>(L::opp(i), a.cmap[id]);
}

template <class L, bool FLOW, typename T>
__device__ __forceinline__ T post_sum(const Dev<T>& a, const T* A, long long id, const Nbr& d, bool lastodd) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) s += A[post_slot<L, FLOW, T>(a, id, d, i, lastodd)];
    return s;
}

__device__ __forceinline__ Nbr nbr_of(const Geo& g, long long id) {
    int x, y, z;
    coords(g, id, x, y, z);
    return nbr_deltas(g, x, y, z);
}

// Solid indicator for the wall normal: solid cells and positions beyond a
// wall axis are 1; an open x axis is extended by clamping.
__device__ __forceinline__ double solid_ind(const Geo& g, const uint8_t* kind, int x, int y, int z) {
    if (x < 0 || x >= g.nx) {
        if (g.per_x) x = (x + g.nx) % g.nx;
        else if (g.open_x) x = x < 0 ? 0 : g.nx - 1;
        else return 1.0;
    }
    if (y < 0 || y >= g.ny) {
        if (g.per_y) y = (y + g.ny) % g.ny;
        else return 1.0;
    }
    if (z < 0 || z >= g.nz) {
        if (g.per_z) z = (z + g.nz) % g.nz;
        else return 1.0;
    }
    return kind[g.idx(x, y, z)] != KIND_FLUID ? 1.0 : 0.0;
}

// Unit normal n = -grad s / |grad s| of the isotropic gradient
// cs^-2 sum_i w_i s(x + e_i) e_i (D3Q19 / D2Q9 weights), accumulated exactly
// as the integer vector sum_i (36 w_i) s e_i; false if it vanishes.  Exact
// accumulation keeps symmetric components exactly zero, which the
// precipitation-excess split depends on.
template <int DIM>
__device__ bool wall_normal(const Geo& g, const uint8_t* kind, int x, int y, int z, double n[3]) {
    using L = typename NormalStencil<DIM>::L;
    int gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const int s = (int)solid_ind(g, kind, x + L::cx(i), y + L::cy(i), z + L::cz(i));
        const int wi = (int)(36.0 * L::w(i) + 0.5);
        gx += wi * s * L::cx(i);
        gy += wi * s * L::cy(i);
        gz += wi * s * L::cz(i);
    }
    if (gx == 0 && gy == 0 && gz == 0) {
        n[0] = n[1] = n[2] = 0.0;
        return false;
    }
    const double len = sqrt((double)(gx * gx + gy * gy + gz * gz));
    n[0] = -(double)gx / len;
    n[1] = -(double)gy / len;
    n[2] = -(double)gz / len;
    return true;
}

// Class of an in-grid cell from the kinds: fluid, or solid with / without a
// fluid neighbour along the solute lattice.
template <class LG>
__device__ uint32_t class_of(const Geo& g, const uint8_t* kind, int x, int y, int z) {
    const uint8_t k = kind[g.idx(x, y, z)];
    if (k == KIND_FLUID) return CLS_FLUID;
#pragma unroll
    for (int o = 1; o < LG::Q; ++o) {
        int xx = x + LG::cx(o), yy = y + LG::cy(o), zz = z + LG::cz(o);
        if (wrap_inside(g, xx, yy, zz) && kind[g.idx(xx, yy, zz)] == KIND_FLUID) return CLS_BOUND;
    }
    return CLS_SOLID;
}

template <class LG>
__device__ __forceinline__ uint32_t class_at(const Geo& g, const uint8_t* kind, int x, int y, int z) {
    if (!wrap_inside(g, x, y, z)) return CLS_SOLID;
    return class_of<LG>(g, kind, x, y, z);
}

#include "events.cuh"

// Initial state: equilibrium populations written as an odd step would write
// them, so the first step (even) reads them as streamed values.
template <typename T, class LF, class LG>
__global__ void k_init(const Dev<T> a, const Phys p, const double* __restrict__ c0, const double* __restrict__ u0) {
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        const uint32_t cls = a.nw[id] & 3u;
        const Nbr d = nbr_deltas(g, x, y, z);
        double ux = 0.0, uy = 0.0, uz = 0.0;
        if (cls == CLS_FLUID && u0) {
            ux = u0[3 * t];
            uy = u0[3 * t + 1];
            uz = u0[3 * t + 2];
        }
        const double C = c0[t];
        if constexpr (LF::Q > 0) {
            if (cls == CLS_FLUID) {
                const double rho = p.rho_init, usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
                for (int i = 0; i < LF::Q; ++i) {
                    const double eu = LF::cx(i) * ux + LF::cy(i) * uy + LF::cz(i) * uz;
                    const double feq = LF::w(i) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
                    a.F[post_slot<LF, true, T>(a, id, d, i, true)] = T(feq - LF::w(i));
                }
            }
        }
        if (cls != CLS_SOLID) {
            const double ics2 = 1.0 / gcs2<LG>(p);
#pragma unroll
            for (int i = 0; i < LG::Q; ++i) {
                const double eu = LG::cx(i) * ux + LG::cy(i) * uy + LG::cz(i) * uz;
                const double w = gweight<LG>(p, i);
                a.G[post_slot<LG, false, T>(a, id, d, i, true)] = T(C * w * (1.0 + eu * ics2) - w * p.cref);
            }
        }
        if (g.open_x && x == g.nx - 1) {
            const int face = y + g.ny * z;
            a.side[4 * face + 0] = ux;
            a.side[4 * face + 1] = uy;
            a.side[4 * face + 2] = uz;
            a.side[4 * face + 3] = C;
        }
    }
}

// Moments of the current state into caller-layout FP64 arrays.
template <typename T, class LF, class LG>
__global__ void k_fields(const Dev<T> a, const Phys p, int lastodd, double* u, double* rho, double* c, double* phi) {
    const Geo& g = a.geo;
    const long long NP = g.NP;
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        const uint32_t cls = a.nw[id] & 3u;
        const Nbr d = nbr_deltas(g, x, y, z);
        double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, C = 0.0;
        if constexpr (LF::Q > 0) {
            if (cls == CLS_FLUID) {
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < LF::Q; ++i) {
                    const double v = (double)a.F[post_slot<LF, true, T>(a, id, d, i, lastodd)];
                    s += v;
                    jx += LF::cx(i) * v;
                    jy += LF::cy(i) * v;
                    jz += LF::cz(i) * v;
                }
                r = 1.0 + s;
                jx /= r;
                jy /= r;
                jz /= r;
            }
        }
        if (cls != CLS_SOLID) C = p.cref + (double)post_sum<LG, false, T>(a, a.G, id, d, lastodd);
        if (u) {
            u[3 * t] = jx;
            u[3 * t + 1] = jy;
            u[3 * t + 2] = jz;
        }
        if (rho) rho[t] = r;
        if (c) c[t] = C;
        if (phi) phi[t] = a.phi[id];
    }
}

template <typename T>
__global__ void k_classes(const Dev<T> a, uint8_t* out) {
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        out[t] = (uint8_t)(a.nw[g.idx(x, y, z)] & 3u);
    }
}

// Deterministic two-pass reduction: per-block partial sums (fixed block
// partition and tree order), then one block sums the partials in order.
constexpr int RED_BLOCK = 256;
template <typename T, class LG>
__global__ void __launch_bounds__(RED_BLOCK) k_reduce_partial(const Dev<T> a, const Phys p, int lastodd, double* part) {
    const Geo& g = a.geo;
    const long long NP = g.NP;
    const long long total = (long long)g.nx * g.ny * g.nz;
    double sc = 0.0, sp = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        if ((a.nw[id] & 3u) != CLS_SOLID) {
            const Nbr d = nbr_deltas(g, x, y, z);
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < LG::Q; ++i) s += (double)a.G[post_slot<LG, false, T>(a, id, d, i, lastodd)];
            sc += p.cref + s;
        }
        sp += a.phi[id];
    }
    __shared__ double s1[RED_BLOCK], s2[RED_BLOCK];
    s1[threadIdx.x] = sc;
    s2[threadIdx.x] = sp;
    __syncthreads();
    for (int k = RED_BLOCK / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            s1[threadIdx.x] += s1[threadIdx.x + k];
            s2[threadIdx.x] += s2[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

template <int UNUSED = 0>
__global__ void k_reduce_final(const double* part, int nblocks, double* out) {
    // one warp, fixed order: lane-strided partial sums, then a shuffle tree
    double s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        s1 += part[2 * b];
        s2 += part[2 * b + 1];
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (threadIdx.x == 0) {
        out[0] = s1;
        out[1] = s2;
    }
}

// Sum of k_bound's per-block ledger partials and the event-path accumulators
// (one warp, fixed order): out[0] reacted, out[1] Dirichlet inflow, out[2]
// unpaid.
template <int UNUSED = 0>
__global__ void k_sum_partials(const double* bacc, int nblocks, const double* acc, const unsigned long long* facc,
                               double* out) {
    double r = 0.0, q = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        r += bacc[2 * b];
        q += bacc[2 * b + 1];
    }
    r = warp_sum(r);
    q = warp_sum(q);
    if (threadIdx.x == 0) {
        out[0] = acc[0] + r;
        out[1] = fx_value(facc) + q;
        out[2] = fx_value(facc + 2);
    }
}

}  // namespace lbrbc
#include "adjoint.cuh"
#include "engine_host.cuh"
