// Device engine of the coupled lattice Boltzmann step with the general local
// reactive boundary condition (arXiv 2306.10794).  Templated over the storage
// type T (float: deviation storage, double) and the flow / solute lattices.
//
// Storage ("AA pattern", one population array per lattice, in place):
//   every population slot A[i][cell] of a padded dense grid (SoA, x fastest,
//   rows padded to 32 cells, ghost layers on non-periodic axes).  After an
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
#include <thread>
#include <vector>

#include "lattice.cuh"
#include "sim_iface.h"

namespace lbrbc {

enum : uint32_t { CLS_FLUID = 0, CLS_BOUND = 1, CLS_SOLID = 2 };
enum : uint8_t { KIND_FLUID = 0, KIND_REACTIVE = 1, KIND_DIRICHLET = 2, KIND_OUTSIDE = 3 };
enum : int { EV_DISSOLVE = 1, EV_PRECIPITATE = 2 };
enum : int { ERR_NUMERIC = 1, ERR_OVERFLOW = 2, ERR_TIMEOUT = 4 };
// fluid sweep: dense grid, compacted fluid list, or staged row tiles
enum : int { SWEEP_DENSE = 0, SWEEP_LIST = 1, SWEEP_STAGED = 2 };

// node word of a fluid cell: bits 0-1 class, bits FBIT.. "flow source
// x - e_i is not fluid" for i = 1..QF-1, bits GBIT.. "solute source
// x - e_i is inactive" for i = 1..QG-1.
constexpr int FBIT = 2;
constexpr int GBIT = 20;
// word of a boundary-list entry: bits 0.. source inactive (i = 1..QG-1),
// bits 8.. link towards a fluid cell (o = 1..QG-1), bit 16 Dirichlet cell.
constexpr int BW_LINK = 8;
constexpr uint32_t BW_DIRICHLET = 1u << 16;

#ifndef LBRBC_FLUID_BLOCK
#define LBRBC_FLUID_BLOCK 128
#endif
// Population loads / stores of the fluid sweep: 0 default caching, 1
// evict-first (each population is touched once per step).
#ifndef LBRBC_STREAM_HINT
#define LBRBC_STREAM_HINT 1
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
    int* b_fslot;         // (QG-1) * cap_b: slot in f_share of the fluid end of link o, or -1
    int* bmap;            // NP
    // fluid cells receiving precipitation shares
    int cap_f;
    int* nf;
    int* f_idx;
    T* f_share;           // (QG-1) * cap_f: share received from the boundary cell at x - e_o
    // compacted fluid cells (packed x | y << 11 | z << 22), when the sweep
    // runs over a list instead of the dense grid
    int use_fl;
    int cap_fl;
    int* nfl;
    uint32_t* fl_xyz;
    // staged sweep: one flag per row tile (1 = the tile has a fluid cell)
    int ntiles;
    uint8_t* tile_on;
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
    double* acc;          // [0] reacted, [1] Dirichlet inflow, [2] unpaid (event path)
    double* bacc;         // per-block partial ledger of k_bound: 2 * gridDim.x
    int* err;
    // compaction scratch
    int* blk;             // per chunk counts / offsets
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

// Slot read by a cell for direction i: its own slot i (even step) or the
// slot opp(i) of the source x - e_i (odd step); an inactive source swaps
// the two (the value there is the cell's own f*_opp(i)).
template <class L, bool ODD>
__device__ __forceinline__ uint32_t read_slot(uint32_t id, const Nbr32& d, uint32_t NP, int i, bool inactive) {
    const uint32_t own = (uint32_t)i * NP + id;
    const uint32_t nbr = (uint32_t)L::opp(i) * NP + id + off32<L>(d, L::opp(i));
    return (ODD == inactive) ? own : nbr;
}

template <class L, bool ODD>
__device__ __forceinline__ uint32_t write_slot(uint32_t id, const Nbr32& d, uint32_t NP, int i) {
    return ODD ? (uint32_t)i * NP + id + off32<L>(d, i) : (uint32_t)L::opp(i) * NP + id;
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

// Where a fluid cell's pre-collision populations come from.  GlobalSrc reads
// the AA slot (read_slot) directly; the staged sweep reads the plain slots
// from shared memory and only the swapped slots of inactive sources from HBM.
template <typename T, class LF, class LG, bool ODD>
struct GlobalSrc {
    const T* __restrict__ F;
    const T* __restrict__ G;
    uint32_t id, NP;
    Nbr32 d;
    __device__ __forceinline__ bool general() const { return false; }
    __device__ __forceinline__ T f(int i, bool inactive) const {
        return ld_pop(F + read_slot<LF, ODD>(id, d, NP, i, inactive));
    }
    __device__ __forceinline__ T g(int i, bool inactive) const {
        return ld_pop(G + read_slot<LG, ODD>(id, d, NP, i, inactive));
    }
};

// One fluid cell (x, y, z) of one step with node word w; shared by the
// single-domain, staged and batched sweeps.
template <typename T, class LF, class LG, bool ODD, class Src>
__device__ __forceinline__ void fluid_cell_src(const Dev<T>& a, const Phys& p, const PhysT<T>& q, int x, int y, int z,
                                               uint32_t id, uint32_t w, const Nbr32& d, const Src& src) {
    constexpr int QF = LF::Q, QG = LG::Q;
    const Geo& g = a.geo;
    const uint32_t NP = (uint32_t)g.NP;
    T* __restrict__ F = a.F;
    T* __restrict__ G = a.G;
    const bool inlet = g.open_x && x == 0;
    const bool outlet = g.open_x && x == g.nx - 1;
    const bool plain = (w >> FBIT) == 0u && !inlet && !outlet && !src.general();

    // Warps whose cells all read the plain slots take a path with no
    // per-direction tests; the others pick, per direction, the plain slot or
    // the swapped one of an inactive source.
    T f[QF > 0 ? QF : 1];
    T gg[QG];
    if (__all_sync(__activemask(), plain)) {
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
                // moving-wall bounce-back with the inlet velocity (rho_w = 1)
                const T uin = T(a.inlet_ux[face]);
#pragma unroll
                for (int i = 1; i < QF; ++i)
                    if (LF::cx(i) > 0) f[i] += T(6.0 * LF::w(i) * LF::cx(i)) * uin;
            }
            if (outlet) {
                // pressure anti-bounce-back at rho_out with the previous velocity
                const T uo0 = T(a.side[4 * face + 0]), uo1 = T(a.side[4 * face + 1]), uo2 = T(a.side[4 * face + 2]);
                const T uq = uo0 * uo0 + uo1 * uo1 + uo2 * uo2;
#pragma unroll
                for (int i = 1; i < QF; ++i)
                    if (LF::cx(i) < 0) {
                        const T eu = T(LF::cx(i)) * uo0 + T(LF::cy(i)) * uo1 + T(LF::cz(i)) * uo2;
                        f[i] = -f[i] + T(2.0 * LF::w(i)) * (q.rho_out * (T(1) + T(4.5) * eu * eu - T(1.5) * uq) - T(1));
                    }
            }
        }
        if (inlet) {
#pragma unroll
            for (int i = 1; i < QG; ++i)
                if (LG::cx(i) > 0) gg[i] = -gg[i] + T(2) * q.gw[i] * q.c_in_d;
        }
        if (outlet) {
            const T co = T(a.side[4 * face + 3]);
#pragma unroll
            for (int i = 1; i < QG; ++i)
                if (LG::cx(i) < 0) gg[i] = -gg[i] + T(2) * q.gw[i] * (co - q.cref);
        }
    }

    T ux = T(0), uy = T(0), uz = T(0), rho = T(1);
    if constexpr (QF > 0) {
        flow_pairs<LF, T>(reinterpret_cast<T(&)[QF]>(f), rho, ux, uy, uz, p, q);
#pragma unroll
        for (int i = 0; i < QF; ++i) st_pop(F + write_slot<LF, ODD>(id, d, NP, i), f[i]);
    }
    T C;
    solute_pairs<LG, T>(gg, C, ux, uy, uz, p, q);
    if (!(rho > T(0)) || !isfinite(C)) *a.err |= ERR_NUMERIC;
    if (a.tape_u) {
        a.tape_u[3 * (size_t)id] = (float)ux;
        a.tape_u[3 * (size_t)id + 1] = (float)uy;
        a.tape_u[3 * (size_t)id + 2] = (float)uz;
    }
#pragma unroll
    for (int i = 0; i < QG; ++i) st_pop(G + write_slot<LG, ODD>(id, d, NP, i), gg[i]);
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
    const GlobalSrc<T, LF, LG, ODD> src{a.F, a.G, id, (uint32_t)g.NP, d};
    fluid_cell_src<T, LF, LG, ODD>(a, p, q, x, y, z, id, w, d, src);
}

template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(FLUID_BLOCK, sizeof(T) == 4 ? 8 : 5) k_fluid(const Dev<T> a, const Phys p, const PhysT<T> q) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.geo.nx) return;
    fluid_cell<T, LF, LG, ODD>(a, p, q, x, blockIdx.y, blockIdx.z);
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
template <typename T, class LG, bool ODD>
__device__ __forceinline__ void bound_entry(const Dev<T>& a, const Phys& p, const PhysT<T>& q, int e, DiffSum<T>& racc,
                                            DiffSum<T>& dacc) {
    constexpr int Q = LG::Q;
    const Geo& g = a.geo;
    const uint32_t NP = (uint32_t)g.NP;
    T* __restrict__ G = a.G;
    const T cref = q.cref;
    const T gam = q.gamma, ics2 = q.ics2;
    int x, y, z;
    unpack_xyz(a.b_xyz[e], x, y, z);
    const uint32_t b = (uint32_t)g.idx(x, y, z);
    const Nbr32 d = nbr32(g, x, y, z);
    const uint32_t bw = a.b_word[e];
    T gp[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool inactive = i > 0 && ((bw >> (i - 1)) & 1u);
        gp[i] = G[read_slot<LG, ODD>(b, d, NP, i, inactive)];
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
#pragma unroll
    for (int i = 0; i < Q; ++i) G[write_slot<LG, ODD>(b, d, NP, i)] = gq[i];
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
#pragma unroll
    for (int o = 1; o < Q; ++o) {
        const int slot = a.b_fslot[(long long)(o - 1) * a.cap_b + e];
        if (slot >= 0) a.f_share[slot] = r * mabs[o];
    }
    if (p.phase_change && dle0(ph)) push_event(a.nev, a.cap_e, a.ev_node, a.ev_kind, a.err, (int)b, EV_DISSOLVE);
}

template <typename T, class LG, bool ODD>
__global__ void __launch_bounds__(LIST_BLOCK) k_bound(const Dev<T> a, const Phys p, const PhysT<T> q) {
    const int n = *a.nb;
    DiffSum<T> racc, dacc;  // reacted mass and Dirichlet inflow of this thread
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        bound_entry<T, LG, ODD>(a, p, q, e, racc, dacc);
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
    T acc = T(0);
#pragma unroll
    for (int o = 1; o < LG::Q; ++o) acc += a.f_share[(long long)(o - 1) * a.cap_f + e];
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
template <class L, typename T>
__device__ __forceinline__ long long post_slot(long long id, const Nbr& d, int i, long long NP, bool lastodd) {
    return lastodd ? (long long)i * NP + id + off<L>(d, i) : (long long)L::opp(i) * NP + id;
}

template <class L, typename T>
__device__ __forceinline__ T post_sum(const T* A, long long id, const Nbr& d, long long NP, bool lastodd) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) s += A[post_slot<L, T>(id, d, i, NP, lastodd)];
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

// ---------------------------------------------------------------------------
// Phase change (Sec. 2.4), applied to all cells that crossed a threshold in
// this step at once.  Every cell that receives something gathers it in a
// fixed direction order, so the result does not depend on thread timing.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_ev_mark(const Dev<T> a) {
    const int n = *a.nev;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n && e < a.cap_e; e += gridDim.x * blockDim.x) {
        const int node = a.ev_node[e];
        const int kd = a.ev_kind[e];
        a.evidx[node] = e;
        a.kind[node] = kd == EV_DISSOLVE ? KIND_FLUID : KIND_REACTIVE;
        if (a.cap_log > 0) {
            const long long pos = atomicAdd((unsigned long long*)a.nlog, 1ull);
            if (pos < a.cap_log) {
                int x, y, z;
                coords(a.geo, node, x, y, z);
                a.log_step[pos] = *a.step;
                a.log_node[pos] = x + (long long)a.geo.nx * (y + (long long)a.geo.ny * z);
                a.log_kind[pos] = kd;
            }
        }
    }
}

template <typename T, class LF, class LG>
__global__ void k_ev_compute(const Dev<T> a, const Phys p, int lastodd) {
    const int n = min(*a.nev, a.cap_e);
    const Geo& g = a.geo;
    const long long NP = g.NP;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const long long id = a.ev_node[e];
        int x, y, z;
        coords(g, id, x, y, z);
        const Nbr d = nbr_deltas(g, x, y, z);
        const double Cself = p.cref + (double)post_sum<LG, T>(a.G, id, d, NP, lastodd);
        if (a.ev_kind[e] == EV_DISSOLVE) {
            double sc = 0.0, sr = 0.0;
            int nfl = 0, ns = 0;
#pragma unroll
            for (int o = 1; o < LG::Q; ++o) {
                int xx = x + LG::cx(o), yy = y + LG::cy(o), zz = z + LG::cz(o);
                if (!wrap_inside(g, xx, yy, zz)) continue;
                const long long nb = g.idx(xx, yy, zz);
                if ((a.nw[nb] & 3u) == CLS_FLUID) {
                    const Nbr dn = nbr_deltas(g, xx, yy, zz);
                    sc += p.cref + (double)post_sum<LG, T>(a.G, nb, dn, NP, lastodd);
                    if constexpr (LF::Q > 0) sr += 1.0 + (double)post_sum<LF, T>(a.F, nb, dn, NP, lastodd);
                    else sr += 1.0;
                    nfl++;
                }
                if (a.kind[nb] == KIND_REACTIVE) ns++;
            }
            const double cinit = nfl ? sc / nfl : Cself;
            const double rinit = nfl ? sr / nfl : p.rho_init;
            const double Q = p.Vm * (cinit - Cself) - a.phi[id];
            a.ev_val[e] = cinit;
            a.ev_val[a.cap_e + e] = rinit;
            a.ev_val[2 * a.cap_e + e] = ns ? Q / ns : 0.0;
            if (!ns) atomicAdd(&a.acc[2], -Q / p.Vm);
        } else {
            const double phic = a.phi[id] + p.Vm * Cself;
            const double excess = phic - 1.0;
            double nrm[3];
            const bool ok = wall_normal<LG::DIM>(g, a.kind, x, y, z, nrm);
            double kap[LG::Q];
            double sk = 0.0;
            int nfl = 0;
#pragma unroll
            for (int o = 1; o < LG::Q; ++o) {
                kap[o] = 0.0;
                int xx = x + LG::cx(o), yy = y + LG::cy(o), zz = z + LG::cz(o);
                if (!wrap_inside(g, xx, yy, zz)) continue;
                if (a.kind[g.idx(xx, yy, zz)] != KIND_FLUID) continue;
                double kk = 1.0;
                if (ok) {
                    kk = LG::cx(o) * nrm[0] + LG::cy(o) * nrm[1] + LG::cz(o) * nrm[2];
                    kk = kk > 0.0 ? kk : 0.0;
                }
                kap[o] = kk;
                sk += kk;
                nfl++;
            }
#pragma unroll
            for (int o = 1; o < LG::Q; ++o) {
                int xx = x + LG::cx(o), yy = y + LG::cy(o), zz = z + LG::cz(o);
                bool fl = wrap_inside(g, xx, yy, zz) && a.kind[g.idx(xx, yy, zz)] == KIND_FLUID;
                double share = fl ? (sk > 0.0 ? kap[o] / sk : 1.0 / nfl) : 0.0;
                a.ev_w[(long long)(o - 1) * a.cap_e + e] = nfl ? excess / p.Vm * share : 0.0;
            }
            a.ev_val[e] = nfl ? 1.0 : phic;
        }
    }
}

template <typename T, class LF, class LG>
__global__ void k_ev_apply_self(const Dev<T> a, const Phys p, int lastodd) {
    const int n = min(*a.nev, a.cap_e);
    const Geo& g = a.geo;
    const long long NP = g.NP;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const long long id = a.ev_node[e];
        const Nbr d = nbr_of(g, id);
        if (a.ev_kind[e] == EV_DISSOLVE) {
            const double cinit = a.ev_val[e], rinit = a.ev_val[a.cap_e + e];
#pragma unroll
            for (int i = 0; i < LG::Q; ++i)
                a.G[post_slot<LG, T>(id, d, i, NP, lastodd)] = T(gweight<LG>(p, i) * (cinit - p.cref));
            if constexpr (LF::Q > 0) {
#pragma unroll
                for (int i = 0; i < LF::Q; ++i) a.F[post_slot<LF, T>(id, d, i, NP, lastodd)] = T(LF::w(i) * (rinit - 1.0));
            }
            a.phi[id] = 0.0;
        } else {
#pragma unroll
            for (int i = 0; i < LG::Q; ++i)
                a.G[post_slot<LG, T>(id, d, i, NP, lastodd)] = T(-gweight<LG>(p, i) * p.cref);
            a.phi[id] = a.ev_val[e];
        }
    }
}

// One thread per (event, direction); the cell x_e + e_o is handled by the
// event found first when scanning its own neighbours in direction order.
template <typename T, class LG>
__global__ void k_ev_neighbours(const Dev<T> a, const Phys p, int lastodd) {
    constexpr int NQ = LG::Q - 1;
    const int n = min(*a.nev, a.cap_e);
    const Geo& g = a.geo;
    const long long NP = g.NP;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * NQ;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / NQ), o = 1 + (int)(t % NQ);
        const long long src = a.ev_node[e];
        int x, y, z;
        coords(g, src, x, y, z);
        x += LG::cx(o);
        y += LG::cy(o);
        z += LG::cz(o);
        // note: LG::cx(o) with a run-time o; fine outside the hot path
        if (!wrap_inside(g, x, y, z)) continue;
        const long long tgt = g.idx(x, y, z);
        int first = -1;
        for (int q = 1; q < LG::Q; ++q) {
            int xx = x + LG::cx(q), yy = y + LG::cy(q), zz = z + LG::cz(q);
            if (!wrap_inside(g, xx, yy, zz)) continue;
            if (a.evidx[g.idx(xx, yy, zz)] >= 0) {
                first = q;
                break;
            }
        }
        if (first != LG::opp(o)) continue;
        double charge = 0.0, dC = 0.0;
        const uint8_t kt = a.kind[tgt];
        for (int q = 1; q < LG::Q; ++q) {
            int xx = x + LG::cx(q), yy = y + LG::cy(q), zz = z + LG::cz(q);
            if (!wrap_inside(g, xx, yy, zz)) continue;
            const int ee = a.evidx[g.idx(xx, yy, zz)];
            if (ee < 0) continue;
            if (a.ev_kind[ee] == EV_DISSOLVE && kt == KIND_REACTIVE) charge += a.ev_val[2 * a.cap_e + ee];
            if (a.ev_kind[ee] == EV_PRECIPITATE && kt == KIND_FLUID)
                dC += a.ev_w[(long long)(LG::opp(q) - 1) * a.cap_e + ee];
        }
        if (charge != 0.0) a.phi[tgt] -= charge;
        if (dC != 0.0) {
            const Nbr d = nbr_deltas(g, x, y, z);
            for (int i = 0; i < LG::Q; ++i) {
                const long long s = post_slot<LG, T>(tgt, d, i, NP, lastodd);
                a.G[s] = T((double)a.G[s] + gweight<LG>(p, i) * dC);
            }
        }
    }
}

// New classes and node words from the kinds (whole grid); boundary cells
// that lost their last fluid neighbour convert their solute into phi, solid
// cells that gained one start empty.
template <typename T, class LF, class LG>
__global__ void k_reclassify(const Dev<T> a, const Phys p, int lastodd, int force) {
    if (!force && *a.nev == 0) return;
    const Geo& g = a.geo;
    const long long NP = g.NP;
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        const uint32_t cls = class_of<LG>(g, a.kind, x, y, z);
        const uint32_t old = a.nw[id] & 3u;
        if (!force && old != cls && a.evidx[id] < 0) {
            const Nbr d = nbr_deltas(g, x, y, z);
            if (old == CLS_BOUND && cls == CLS_SOLID) {
                const double C = p.cref + (double)post_sum<LG, T>(a.G, id, d, NP, lastodd);
                if (a.kind[id] == KIND_REACTIVE) a.phi[id] += p.Vm * C;
                else atomicAdd(&a.acc[1], -C);
            }
            if (cls != CLS_FLUID) {
#pragma unroll
                for (int i = 0; i < LG::Q; ++i)
                    a.G[post_slot<LG, T>(id, d, i, NP, lastodd)] = T(-gweight<LG>(p, i) * p.cref);
            }
        }
        uint32_t w = cls;
        if (cls == CLS_FLUID) {
            if constexpr (LF::Q > 0) {
#pragma unroll
                for (int i = 1; i < LF::Q; ++i) {
                    int xx = x - LF::cx(i), yy = y - LF::cy(i), zz = z - LF::cz(i);
                    if (class_at<LG>(g, a.kind, xx, yy, zz) != CLS_FLUID) w |= 1u << (FBIT + i - 1);
                }
            }
#pragma unroll
            for (int i = 1; i < LG::Q; ++i) {
                int xx = x - LG::cx(i), yy = y - LG::cy(i), zz = z - LG::cz(i);
                if (class_at<LG>(g, a.kind, xx, yy, zz) == CLS_SOLID) w |= 1u << (GBIT + i - 1);
            }
        }
        a.nw[id] = w;
    }
}

// Stream compaction of the wet boundary cells (order = cell index).
// Pass 1: counts per chunk of SCAN_CHUNK cells.
template <typename T, class LG>
__global__ void k_count(const Dev<T> a, int which, int force) {
    if (!force && *a.nev == 0) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    const long long chunk = blockIdx.x;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int local = 0;
    for (long long t = chunk * SCAN_CHUNK + threadIdx.x; t < min(total, (chunk + 1) * SCAN_CHUNK); t += blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        const uint32_t cls = a.nw[id] & 3u;
        if (which == 0) local += cls == CLS_BOUND;
        else if (which == 2) local += cls == CLS_FLUID;
        else if (cls == CLS_FLUID) {
#pragma unroll
            for (int o = 1; o < LG::Q; ++o) {
                int xx = x - LG::cx(o), yy = y - LG::cy(o), zz = z - LG::cz(o);
                if (!wrap_inside(g, xx, yy, zz)) continue;
                const long long nb = g.idx(xx, yy, zz);
                if ((a.nw[nb] & 3u) == CLS_BOUND && a.kind[nb] == KIND_REACTIVE) {
                    local++;
                    break;
                }
            }
        }
    }
    atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) a.blk[chunk] = cnt;
}

// Pass 2: exclusive scan of the chunk counts (one block); total -> *count.
template <typename T>
__global__ void k_scan(const Dev<T> a, int nchunks, int which, int force) {
    if (!force && *a.nev == 0) return;
    __shared__ int part[1024];
    const int per = (nchunks + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(nchunks, lo + per);
    int s = 0;
    for (int c = lo; c < hi; ++c) s += a.blk[c];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const int v = part[k];
            part[k] = run;
            run += v;
        }
        const int cap = which == 0 ? a.cap_b : (which == 1 ? a.cap_f : a.cap_fl);
        if (run > cap) atomicOr(a.err, ERR_OVERFLOW);
        *(which == 0 ? a.nb : (which == 1 ? a.nf : a.nfl)) = min(run, cap);
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int c = lo; c < hi; ++c) {
        const int v = a.blk[c];
        a.blk[c] = run;
        run += v;
    }
}

// Pass 3: write the entries in cell order.
template <typename T, class LG>
__global__ void k_write_lists(const Dev<T> a, const Phys p, int which, int force) {
    if (!force && *a.nev == 0) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    const long long chunk = blockIdx.x;
    __shared__ int warp_tot[32];
    __shared__ int base_s;
    if (threadIdx.x == 0) base_s = a.blk[chunk];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw_ = blockDim.x >> 5;
    for (long long t0 = chunk * SCAN_CHUNK; t0 < min(total, (chunk + 1) * SCAN_CHUNK); t0 += blockDim.x) {
        const long long t = t0 + threadIdx.x;
        bool sel = false;
        int x = 0, y = 0, z = 0;
        long long id = 0;
        int src[LG::Q];
        if (t < min(total, (chunk + 1) * SCAN_CHUNK)) {
            x = (int)(t % g.nx);
            y = (int)((t / g.nx) % g.ny);
            z = (int)(t / ((long long)g.nx * g.ny));
            id = g.idx(x, y, z);
            const uint32_t cls = a.nw[id] & 3u;
            if (which == 0) {
                sel = cls == CLS_BOUND;
                a.bmap[id] = -1;
            } else if (which == 2) {
                sel = cls == CLS_FLUID;
            } else if (cls == CLS_FLUID) {
#pragma unroll
                for (int o = 1; o < LG::Q; ++o) {
                    src[o] = -1;
                    int xx = x - LG::cx(o), yy = y - LG::cy(o), zz = z - LG::cz(o);
                    if (!wrap_inside(g, xx, yy, zz)) continue;
                    const long long nb = g.idx(xx, yy, zz);
                    if ((a.nw[nb] & 3u) == CLS_BOUND && a.kind[nb] == KIND_REACTIVE) {
                        src[o] = a.bmap[nb];
                        sel = true;
                    }
                }
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, sel);
        if (lane == 0) warp_tot[wid] = __popc(bal);
        __syncthreads();
        int woff = 0, tot = 0;
        for (int k = 0; k < nw_; ++k) {
            if (k < wid) woff += warp_tot[k];
            tot += warp_tot[k];
        }
        const int pos = base_s + woff + __popc(bal & ((1u << lane) - 1u));
        if (sel) {
            if (which == 0 && pos < a.cap_b) {
                a.b_idx[pos] = (int)id;
                a.b_xyz[pos] = pack_xyz(x, y, z);
                a.bmap[id] = pos;
                uint32_t bw = 0;
                const uint8_t kd = a.kind[id];
                if (kd == KIND_DIRICHLET) bw |= BW_DIRICHLET;
                double nrm[3];
                const bool ok = wall_normal<LG::DIM>(g, a.kind, x, y, z, nrm);
#pragma unroll
                for (int o = 1; o < LG::Q; ++o) {
                    int xs = x - LG::cx(o), ys = y - LG::cy(o), zs = z - LG::cz(o);
                    if (class_at<LG>(g, a.kind, xs, ys, zs) == CLS_SOLID) bw |= 1u << (o - 1);
                    int xf = x + LG::cx(o), yf = y + LG::cy(o), zf = z + LG::cz(o);
                    T kap = T(0);
                    if (wrap_inside(g, xf, yf, zf) && a.kind[g.idx(xf, yf, zf)] == KIND_FLUID) {
                        bw |= 1u << (BW_LINK + o - 1);
                        double kk = 1.0;
                        if (ok) {
                            kk = LG::cx(o) * nrm[0] + LG::cy(o) * nrm[1] + LG::cz(o) * nrm[2];
                            kk = kk > 0.0 ? kk : 0.0;
                        }
                        kap = T(kk);
                    }
                    a.b_kappa[(long long)(o - 1) * a.cap_b + pos] = kap;
                }
                a.b_word[pos] = bw;
                if (a.b_krate) a.b_krate[pos] = a.kfield ? a.kfield[id] : p.k_r;
#pragma unroll
                for (int o = 1; o < LG::Q; ++o) a.b_fslot[(long long)(o - 1) * a.cap_b + pos] = -1;
            } else if (which == 2 && pos < a.cap_fl) {
                a.fl_xyz[pos] = (uint32_t)x | ((uint32_t)y << 11) | ((uint32_t)z << 22);
            } else if (which == 1 && pos < a.cap_f) {
                a.f_idx[pos] = (int)id;
#pragma unroll
                for (int o = 1; o < LG::Q; ++o) {
                    const long long slot = (long long)(o - 1) * a.cap_f + pos;
                    a.f_share[slot] = T(0);
                    if (src[o] >= 0) a.b_fslot[(long long)(o - 1) * a.cap_b + src[o]] = (int)slot;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base_s += tot;
        __syncthreads();
    }
}

template <typename T>
__global__ void k_ev_reset(const Dev<T> a) {
    const int n = min(*a.nev, a.cap_e);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) a.evidx[a.ev_node[e]] = -1;
}

template <typename T>
__global__ void k_step_end(const Dev<T> a) {
    *a.nev = 0;
    *a.step += 1;
}

// Initial state: equilibrium populations written as an odd step would write
// them, so the first step (even) reads them as streamed values.
template <typename T, class LF, class LG>
__global__ void k_init(const Dev<T> a, const Phys p, const double* __restrict__ c0, const double* __restrict__ u0) {
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
                    a.F[(long long)i * NP + id + off<LF>(d, i)] = T(feq - LF::w(i));
                }
            }
        }
        if (cls != CLS_SOLID) {
            const double ics2 = 1.0 / gcs2<LG>(p);
#pragma unroll
            for (int i = 0; i < LG::Q; ++i) {
                const double eu = LG::cx(i) * ux + LG::cy(i) * uy + LG::cz(i) * uz;
                const double w = gweight<LG>(p, i);
                a.G[(long long)i * NP + id + off<LG>(d, i)] = T(C * w * (1.0 + eu * ics2) - w * p.cref);
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
                    const double v = (double)a.F[post_slot<LF, T>(id, d, i, NP, lastodd)];
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
        if (cls != CLS_SOLID) C = p.cref + (double)post_sum<LG, T>(a.G, id, d, NP, lastodd);
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
            for (int i = 0; i < LG::Q; ++i) s += (double)a.G[post_slot<LG, T>(id, d, i, NP, lastodd)];
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
__global__ void k_sum_partials(const double* bacc, int nblocks, const double* acc, double* out) {
    double r = 0.0, q = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        r += bacc[2 * b];
        q += bacc[2 * b + 1];
    }
    r = warp_sum(r);
    q = warp_sum(q);
    if (threadIdx.x == 0) {
        out[0] = acc[0] + r;
        out[1] = acc[1] + q;
        out[2] = acc[2];
    }
}

}  // namespace lbrbc
#include "staged.cuh"
#include "adjoint.cuh"
namespace lbrbc {

// ---------------------------------------------------------------------------
// Host side of the engine.
// ---------------------------------------------------------------------------
#define LB_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
            return 2;                                                                     \
        }                                                                                 \
    } while (0)

template <typename T, class LF, class LG>
class Engine final : public ISim {
   public:
    ~Engine() override { release(); }

    int init(const lbrbc_params& P, const uint8_t* mask, const lbrbc_init* ini, std::string& err) override {
        (void)cudaGetLastError();  // do not report an error left by earlier, unrelated calls
        prm_ = P;
        Geo& g = d_.geo;
        g.nx = P.nx;
        g.ny = P.ny;
        g.nz = P.dim == 2 ? 1 : P.nz;
        g.per_x = P.bc[0] == LBRBC_PERIODIC;
        g.per_y = P.bc[1] == LBRBC_PERIODIC;
        g.per_z = P.dim == 2 ? 1 : P.bc[2] == LBRBC_PERIODIC;
        g.open_x = P.bc[0] == LBRBC_OPEN;
        g.py = g.per_y ? 0 : 1;
        g.pz = g.per_z ? 0 : 1;
        g.SX = ((g.nx + 2 + 31) / 32) * 32;
        g.SY = g.ny + 2 * g.py;
        g.SZ = g.nz + 2 * g.pz;
        g.OFF = 32;
        g.NP = ((g.OFF + (long long)g.SX * g.SY * g.SZ + 64 + 63) / 64) * 64;
        ncell_ = (long long)g.nx * g.ny * g.nz;
        if (g.nx >= (1 << 21) || g.ny >= (1 << 21) || g.nz >= (1 << 21)) {
            err = "grid extent must be below 2^21 cells per axis";
            return 1;
        }
        {
            const long long qmax = std::max(LF::Q, LG::Q);
            if (g.NP >= (1LL << 31) || qmax * g.NP >= (1LL << 32)) {
                err = "grid too large for 32-bit population indices";
                return 1;
            }
        }
        // physics
        Phys& p = ph_;
        const bool trt_f = P.magic_flow >= 0.0, trt_g = P.magic_solute >= 0.0;
        p.trt_f = trt_f;
        p.trt_g = trt_g;
        p.of_sym = 1.0 / P.tau_flow;
        p.of_anti = trt_f ? 1.0 / (0.5 + P.magic_flow / (P.tau_flow - 0.5)) : p.of_sym;
        p.og_anti = 1.0 / P.tau_solute;
        p.og_sym = trt_g ? 1.0 / (0.5 + P.magic_solute / (P.tau_solute - 0.5)) : p.og_anti;
        if (LG::Q == 9) {
            p.gcs2 = 1.0 / 3.0;
            p.gw0 = 4.0 / 9.0;
            p.gw1 = 1.0 / 9.0;
        } else {
            double J0 = P.rest_fraction;
            if (J0 < 0.0) J0 = (LG::DIM == 2) ? 1.0 / 3.0 : 0.25;
            p.gcs2 = (1.0 - J0) / LG::DIM;
            p.gw0 = J0;
            p.gw1 = p.gcs2 / 2.0;
            if (P.rest_fraction < 0.0 && LG::DIM == 2) {
                p.gw0 = 1.0 / 3.0;
                p.gw1 = 1.0 / 6.0;
                p.gcs2 = 1.0 / 3.0;
            }
        }
        p.cref = P.c_init != 0.0 ? P.c_init : (P.c_eq != 0.0 ? P.c_eq : P.c_dirichlet);
        p.c_inlet = P.c_inlet;
        p.rho_out = P.rho_outlet;
        p.c_dir = P.c_dirichlet;
        p.c_eq = P.c_eq;
        p.k_r = P.k_r;
        p.gamma = P.tau_solute / (P.tau_solute - 0.5);
        p.Vm = P.molar_volume;
        p.rho_init = P.rho_init;
        p.scheme = P.scheme;
        p.phase_change = P.phase_change;
        {
            PhysT<T>& q = pt_;
            q.f_sym = T(p.of_sym);
            q.f_anti = T(p.of_anti);
            q.g_sym = T(p.og_sym);
            q.g_anti = T(p.og_anti);
            for (int i = 0; i < 9; ++i) q.gw[i] = T(0);
            for (int i = 0; i < LG::Q; ++i) q.gw[i] = T(LG::Q == 9 ? LG::w(i) : (i == 0 ? p.gw0 : p.gw1));
            q.ics2 = T(1.0 / p.gcs2);
            q.cref = T(p.cref);
            q.c_in_d = T(p.c_inlet - p.cref);
            q.c_dir_d = T(p.c_dir - p.cref);
            q.c_eq_d = T(p.c_eq - p.cref);
            q.rho_out = T(p.rho_out);
            q.k_r = T(p.k_r);
            q.gamma = T(p.gamma);
            q.neg_vm = T(-p.Vm);
        }

        // kinds with ghosts, host side
        const long long NP = g.NP;
        std::vector<uint8_t> kind(NP, KIND_OUTSIDE);
        long long nsolid = 0, nfluid = 0;
        for (int z = 0; z < g.nz; ++z)
            for (int y = 0; y < g.ny; ++y)
                for (int x = 0; x < g.nx; ++x) {
                    const uint8_t m = mask[x + (long long)g.nx * (y + (long long)g.ny * z)];
                    kind[g.idx(x, y, z)] = m;
                    if (m == KIND_FLUID) nfluid++;
                    else nsolid++;
                }
        nfluid_ = nfluid;
        // list capacities: the initial counts with head room for growth
        long long nb0 = 0, nf0 = 0;
        count_lists_host(kind, nb0, nf0);
        nb0_ = nb0;
        nf0_ = nf0;
        auto grow = [&](long long n0) {
            long long c = std::max<long long>(4 * n0, n0 + ncell_ / 16) + 1024;
            return (int)std::min<long long>(c, ncell_ + 1024);
        };
        d_.cap_b = grow(nb0);
        d_.cap_f = grow(nf0);
        d_.cap_e = (int)std::min<long long>(ncell_ + 64, std::max<long long>(1 << 16, ncell_ / 64));
        // Sweep over the dense grid (default), over a compacted fluid-cell
        // list (LBRBC_FLUID_SWEEP=list, or a batch schedule) or over staged
        // row tiles (LBRBC_FLUID_SWEEP=staged).  Measured on GB300 both
        // alternatives are slower: a warp's 32 list cells span several rows,
        // so every population load touches more lines; the staged tiles
        // leave fewer warps to issue an issue-bound cell update.
        {
            long long active = 0;
            for (int z = 0; z < g.nz; ++z)
                for (int y = 0; y < g.ny; ++y)
                    for (int x0 = 0; x0 < g.nx; x0 += 32) {
                        bool any = false;
                        for (int x = x0; x < std::min(g.nx, x0 + 32) && !any; ++x)
                            any = mask[x + (long long)g.nx * (y + (long long)g.ny * z)] == KIND_FLUID;
                        active += any;
                    }
            lane_eff_ = active ? (double)nfluid / (32.0 * active) : 1.0;
            const bool fits = g.nx <= 2048 && g.ny <= 2048 && g.nz <= 1024;
            const char* env = getenv("LBRBC_FLUID_SWEEP");
            int want = SWEEP_DENSE;
            if (env && !strcmp(env, "list")) want = SWEEP_LIST;
            if (env && !strcmp(env, "dense")) want = SWEEP_DENSE;
            if (env && !strcmp(env, "staged")) want = SWEEP_STAGED;
            if (force_list_) want = SWEEP_LIST;
            // (the list sweep is not combined with phase change)
            if (want == SWEEP_LIST && !(fits && !P.phase_change)) want = SWEEP_DENSE;
            sweep_ = want;
            d_.use_fl = want == SWEEP_LIST;
            d_.cap_fl = (int)std::min<long long>(ncell_, std::max<long long>(2 * nfluid, nfluid + ncell_ / 8) + 1024);
        }
        d_.cap_log = P.event_log_capacity > 0 ? P.event_log_capacity : 0;
        nchunks_ = (int)((ncell_ + SCAN_CHUNK - 1) / SCAN_CHUNK);

        // device allocations
        constexpr int QF = LF::Q > 0 ? LF::Q : 0, QG = LG::Q;
        if (QF) LB_CUDA(dalloc(&d_.F, (size_t)QF * NP));
        else d_.F = nullptr;
        LB_CUDA(dalloc(&d_.G, (size_t)QG * NP));
        LB_CUDA(dalloc(&d_.nw, (size_t)NP));
        LB_CUDA(dalloc(&d_.kind, (size_t)NP));
        LB_CUDA(dalloc(&d_.phi, (size_t)NP));
        LB_CUDA(dalloc(&d_.inlet_ux, (size_t)g.ny * g.nz));
        LB_CUDA(dalloc(&d_.side, (size_t)4 * g.ny * g.nz));
        LB_CUDA(dalloc(&d_.nb, 1));
        LB_CUDA(dalloc(&d_.b_idx, (size_t)d_.cap_b));
        LB_CUDA(dalloc(&d_.b_word, (size_t)d_.cap_b));
        LB_CUDA(dalloc(&d_.b_xyz, (size_t)d_.cap_b));
        LB_CUDA(dalloc(&d_.b_kappa, (size_t)(QG - 1) * d_.cap_b));
        LB_CUDA(dalloc(&d_.b_fslot, (size_t)(QG - 1) * d_.cap_b));
        LB_CUDA(dalloc(&d_.bmap, (size_t)NP));
        LB_CUDA(dalloc(&d_.nf, 1));
        LB_CUDA(dalloc(&d_.f_idx, (size_t)d_.cap_f));
        LB_CUDA(dalloc(&d_.f_share, (size_t)(QG - 1) * d_.cap_f));
        LB_CUDA(dalloc(&d_.nfl, 1));
        d_.ntiles = 0;
        d_.tile_on = nullptr;
        if (sweep_ == SWEEP_STAGED) {
            const long long nt = (long long)((g.nx + TILE_X - 1) / TILE_X) * g.ny * g.nz;
            if (nt >= (1LL << 31)) {
                err = "too many row tiles for the staged sweep";
                return 1;
            }
            d_.ntiles = (int)nt;
            LB_CUDA(dalloc(&d_.tile_on, (size_t)nt));
            if (setup_staged(err)) return 2;
        }
        if (d_.use_fl) LB_CUDA(dalloc(&d_.fl_xyz, (size_t)d_.cap_fl));
        else d_.fl_xyz = nullptr;
        LB_CUDA(cudaMemset(d_.nfl, 0, sizeof(int)));
        LB_CUDA(dalloc(&d_.nev, 1));
        LB_CUDA(dalloc(&d_.ev_node, (size_t)d_.cap_e));
        LB_CUDA(dalloc(&d_.ev_kind, (size_t)d_.cap_e));
        LB_CUDA(dalloc(&d_.ev_val, (size_t)3 * d_.cap_e));
        LB_CUDA(dalloc(&d_.ev_w, (size_t)(QG - 1) * d_.cap_e));
        LB_CUDA(dalloc(&d_.evidx, (size_t)NP));
        LB_CUDA(dalloc(&d_.nlog, 1));
        if (d_.cap_log) {
            LB_CUDA(dalloc(&d_.log_step, (size_t)d_.cap_log));
            LB_CUDA(dalloc(&d_.log_node, (size_t)d_.cap_log));
            LB_CUDA(dalloc(&d_.log_kind, (size_t)d_.cap_log));
        } else {
            d_.log_step = d_.log_node = nullptr;
            d_.log_kind = nullptr;
        }
        LB_CUDA(dalloc(&d_.step, 1));
        LB_CUDA(dalloc(&d_.acc, 4));
        nbacc_ = list_grid(d_.cap_b);
        LB_CUDA(dalloc(&d_.bacc, (size_t)2 * nbacc_));
        LB_CUDA(cudaMemset(d_.bacc, 0, 2 * nbacc_ * sizeof(double)));
        LB_CUDA(dalloc(&d_.err, 1));
        LB_CUDA(dalloc(&d_.blk, (size_t)nchunks_ + 1));
        LB_CUDA(cudaStreamCreateWithFlags(&own_, cudaStreamNonBlocking));
        {
            // the boundary branch runs beside the fluid sweep; the highest
            // priority lets its few blocks start first instead of queueing
            // behind the sweep's
            int lo = 0, hi = 0;
            LB_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            LB_CUDA(cudaStreamCreateWithPriority(&aux_, cudaStreamNonBlocking, hi));
        }
        LB_CUDA(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming));
        LB_CUDA(cudaEventCreateWithFlags(&join_, cudaEventDisableTiming));

        // uploads
        std::vector<double> phi(NP, 0.0);
        std::vector<double> c0((size_t)ncell_);
        for (int z = 0; z < g.nz; ++z)
            for (int y = 0; y < g.ny; ++y)
                for (int x = 0; x < g.nx; ++x) {
                    const long long t = x + (long long)g.nx * (y + (long long)g.ny * z);
                    const uint8_t m = mask[t];
                    phi[g.idx(x, y, z)] = (ini && ini->phi_init) ? ini->phi_init[t] : (m == KIND_REACTIVE ? 1.0 : 0.0);
                    c0[t] = (ini && ini->c_init) ? ini->c_init[t] : (m == KIND_DIRICHLET ? P.c_dirichlet : P.c_init);
                }
        LB_CUDA(cudaMemcpy(d_.kind, kind.data(), NP, cudaMemcpyHostToDevice));
        LB_CUDA(cudaMemcpy(d_.phi, phi.data(), NP * sizeof(double), cudaMemcpyHostToDevice));
        if (ini && ini->k_field) {
            std::vector<double> kf(NP, 0.0);
            for (int z = 0; z < g.nz; ++z)
                for (int y = 0; y < g.ny; ++y)
                    for (int x = 0; x < g.nx; ++x)
                        kf[g.idx(x, y, z)] = ini->k_field[x + (long long)g.nx * (y + (long long)g.ny * z)];
            LB_CUDA(dalloc(&d_.kfield, (size_t)NP));
            LB_CUDA(dalloc(&d_.b_krate, (size_t)d_.cap_b));
            LB_CUDA(cudaMemcpy(d_.kfield, kf.data(), NP * sizeof(double), cudaMemcpyHostToDevice));
        } else {
            d_.kfield = nullptr;
            d_.b_krate = nullptr;
        }
        {
            std::vector<double> inl((size_t)g.ny * g.nz);
            for (size_t i = 0; i < inl.size(); ++i) inl[i] = (ini && ini->inlet_ux) ? ini->inlet_ux[i] : P.u_inlet;
            LB_CUDA(cudaMemcpy(d_.inlet_ux, inl.data(), inl.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
        LB_CUDA(cudaMemset(d_.nw, 0, NP * sizeof(uint32_t)));
        LB_CUDA(cudaMemset(d_.evidx, 0xff, NP * sizeof(int)));
        LB_CUDA(cudaMemset(d_.bmap, 0xff, NP * sizeof(int)));
        LB_CUDA(cudaMemset(d_.nev, 0, sizeof(int)));
        LB_CUDA(cudaMemset(d_.nb, 0, sizeof(int)));
        LB_CUDA(cudaMemset(d_.nf, 0, sizeof(int)));
        LB_CUDA(cudaMemset(d_.nlog, 0, sizeof(long long)));
        LB_CUDA(cudaMemset(d_.step, 0, sizeof(long long)));
        LB_CUDA(cudaMemset(d_.acc, 0, 4 * sizeof(double)));
        LB_CUDA(cudaMemset(d_.err, 0, sizeof(int)));
        LB_CUDA(cudaMemset(d_.side, 0, 4 * sizeof(double) * g.ny * g.nz));
        if (QF) LB_CUDA(cudaMemset(d_.F, 0, (size_t)QF * NP * sizeof(T)));
        LB_CUDA(cudaMemset(d_.G, 0, (size_t)QG * NP * sizeof(T)));
        // ghost cells are solid for every lattice
        {
            std::vector<uint32_t> nwh(NP, CLS_SOLID);
            LB_CUDA(cudaMemcpy(d_.nw, nwh.data(), NP * sizeof(uint32_t), cudaMemcpyHostToDevice));
        }
        // classes, lists, initial populations
        if (rebuild(own_, 0, 1, err)) return 2;
        double *dc0 = nullptr, *du0 = nullptr;
        LB_CUDA(talloc(&dc0, (size_t)ncell_));
        LB_CUDA(cudaMemcpy(dc0, c0.data(), ncell_ * sizeof(double), cudaMemcpyHostToDevice));
        if (ini && ini->u_init) {
            LB_CUDA(talloc(&du0, (size_t)3 * ncell_));
            LB_CUDA(cudaMemcpy(du0, ini->u_init, 3 * ncell_ * sizeof(double), cudaMemcpyHostToDevice));
        }
        k_init<T, LF, LG><<<grid_for(ncell_, 256), 256, 0, own_>>>(d_, ph_, dc0, du0);
        LB_CUDA(cudaGetLastError());
        LB_CUDA(cudaStreamSynchronize(own_));
        cudaFree(dc0);
        if (du0) cudaFree(du0);
        int hnb = 0, hnf = 0, herr = 0;
        LB_CUDA(cudaMemcpy(&hnb, d_.nb, sizeof(int), cudaMemcpyDeviceToHost));
        LB_CUDA(cudaMemcpy(&hnf, d_.nf, sizeof(int), cudaMemcpyDeviceToHost));
        LB_CUDA(cudaMemcpy(&herr, d_.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr & ERR_OVERFLOW) {
            err = "internal list capacity exceeded at creation";
            return 5;
        }
        if (hnb != nb0) {
            err = "device boundary list disagrees with the host count";
            return 5;
        }
        lastodd_ = 1;
        steps_ = 0;
        if (build_graphs(err)) return 2;
        return 0;
    }

    int step(int64_t n, cudaStream_t s, std::string& err) override {
        if (batched_) {
            err = "this domain belongs to a batch: step it with lbrbc_batch_step";
            return 5;
        }
        cudaStream_t st = s ? s : own_;
        int64_t k = 0;
        // the state's parity decides which graph comes first
        while (k < n) {
            if (!lastodd_ || n - k < 2) {
                // single step of the pending parity
                LB_CUDA(cudaGraphLaunch(lastodd_ ? g_even_ : g_odd_, st));
                lastodd_ ^= 1;
                k += 1;
            } else {
                LB_CUDA(cudaGraphLaunch(g_pair_, st));
                k += 2;
            }
        }
        steps_ += n;
        last_stream_ = st;
        if (!s) LB_CUDA(cudaStreamSynchronize(own_));
        return 0;
    }

    int fields(double* u, double* rho, double* c, double* phi, int device, std::string& err) override {
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        double *du = u, *dr = rho, *dc = c, *dp = phi;
        double* tmp = nullptr;
        if (!device) {
            int nf = (u ? 3 : 0) + (rho ? 1 : 0) + (c ? 1 : 0) + (phi ? 1 : 0);
            if (nf == 0) return 0;
            LB_CUDA(talloc(&tmp, (size_t)nf * ncell_));
            double* q = tmp;
            du = u ? q : nullptr;
            q += u ? 3 * ncell_ : 0;
            dr = rho ? q : nullptr;
            q += rho ? ncell_ : 0;
            dc = c ? q : nullptr;
            q += c ? ncell_ : 0;
            dp = phi ? q : nullptr;
        }
        k_fields<T, LF, LG><<<grid_for(ncell_, 256), 256, 0, own_>>>(d_, ph_, lastodd_, du, dr, dc, dp);
        LB_CUDA(cudaGetLastError());
        LB_CUDA(cudaStreamSynchronize(own_));
        if (!device) {
            if (u) LB_CUDA(cudaMemcpy(u, du, 3 * ncell_ * sizeof(double), cudaMemcpyDeviceToHost));
            if (rho) LB_CUDA(cudaMemcpy(rho, dr, ncell_ * sizeof(double), cudaMemcpyDeviceToHost));
            if (c) LB_CUDA(cudaMemcpy(c, dc, ncell_ * sizeof(double), cudaMemcpyDeviceToHost));
            if (phi) LB_CUDA(cudaMemcpy(phi, dp, ncell_ * sizeof(double), cudaMemcpyDeviceToHost));
            cudaFree(tmp);
        }
        return 0;
    }

    int classes(uint8_t* out, std::string& err) override {
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        uint8_t* tmp = nullptr;
        LB_CUDA(talloc(&tmp, (size_t)ncell_));
        k_classes<T><<<grid_for(ncell_, 256), 256, 0, own_>>>(d_, tmp);
        LB_CUDA(cudaGetLastError());
        LB_CUDA(cudaMemcpyAsync(out, tmp, ncell_, cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaStreamSynchronize(own_));
        cudaFree(tmp);
        return 0;
    }

    int ledger(double* out, std::string& err) override {
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        const int nblk = red_blocks();
        double* part = nullptr;
        LB_CUDA(talloc(&part, (size_t)2 * nblk + 2));
        k_reduce_partial<T, LG><<<nblk, RED_BLOCK, 0, own_>>>(d_, ph_, lastodd_, part);
        k_reduce_final<0><<<1, 32, 0, own_>>>(part, nblk, part + 2 * nblk);
        LB_CUDA(cudaGetLastError());
        double sums[2], acc[4];
        std::vector<double> bacc((size_t)2 * nbacc_);
        LB_CUDA(cudaMemcpyAsync(sums, part + 2 * nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaMemcpyAsync(acc, d_.acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaMemcpyAsync(bacc.data(), d_.bacc, bacc.size() * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaStreamSynchronize(own_));
        for (int b = 0; b < nbacc_; ++b) {
            acc[0] += bacc[2 * b];
            acc[1] += bacc[2 * b + 1];
        }
        cudaFree(part);
        out[0] = sums[0];
        out[1] = prm_.molar_volume > 0.0 ? sums[1] / prm_.molar_volume : 0.0;
        out[2] = acc[2];
        out[3] = acc[1];
        out[4] = acc[0];
        out[5] = (double)steps_;
        return 0;
    }

    // Same reduction on caller-provided scratch (2 * red_blocks() + 2 doubles).
    int ledger_with_scratch(double* out, double* part, std::string& err) {
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        const int nblk = red_blocks();
        k_reduce_partial<T, LG><<<nblk, RED_BLOCK, 0, own_>>>(d_, ph_, lastodd_, part);
        k_reduce_final<0><<<1, 32, 0, own_>>>(part, nblk, part + 2 * nblk);
        LB_CUDA(cudaGetLastError());
        double sums[2], acc[4];
        std::vector<double> bacc((size_t)2 * nbacc_);
        LB_CUDA(cudaMemcpyAsync(sums, part + 2 * nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaMemcpyAsync(acc, d_.acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaMemcpyAsync(bacc.data(), d_.bacc, bacc.size() * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaStreamSynchronize(own_));
        for (int b = 0; b < nbacc_; ++b) {
            acc[0] += bacc[2 * b];
            acc[1] += bacc[2 * b + 1];
        }
        out[0] = sums[0];
        out[1] = prm_.molar_volume > 0.0 ? sums[1] / prm_.molar_volume : 0.0;
        out[2] = acc[2];
        out[3] = acc[1];
        out[4] = acc[0];
        out[5] = (double)steps_;
        return 0;
    }

    // Mass balance with caller-provided device scratch and no allocation:
    // one partial pair per block of cells_per_block cells, then the final
    // sums; scratch holds 2 * max_blocks + 8 doubles.
    int ledger_scratch(double* out, double* scratch, int max_blocks, long long cells_per_block,
                       std::string& err) override {
        const long long nblk = (ncell_ + cells_per_block - 1) / cells_per_block;
        if (nblk > max_blocks) {
            err = "grid of " + std::to_string(ncell_) + " cells exceeds the static scratch of this entry point (" +
                  std::to_string((long long)max_blocks * cells_per_block) + " cells)";
            return 1;
        }
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        double* tail = scratch + 2 * (size_t)max_blocks;
        k_reduce_partial<T, LG><<<(int)nblk, RED_BLOCK, 0, own_>>>(d_, ph_, lastodd_, scratch);
        k_reduce_final<0><<<1, 32, 0, own_>>>(scratch, (int)nblk, tail);
        k_sum_partials<0><<<1, 32, 0, own_>>>(d_.bacc, nbacc_, d_.acc, tail + 2);
        LB_CUDA(cudaGetLastError());
        double h[5];
        LB_CUDA(cudaMemcpyAsync(h, tail, 5 * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaStreamSynchronize(own_));
        out[0] = h[0];
        out[1] = prm_.molar_volume > 0.0 ? h[1] / prm_.molar_volume : 0.0;
        out[2] = h[4];
        out[3] = h[3];
        out[4] = h[2];
        out[5] = (double)steps_;
        return 0;
    }

    int events(int64_t* count, int64_t capacity, int64_t* stp, int64_t* node, int32_t* kind, std::string& err) override {
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        long long n = 0;
        LB_CUDA(cudaMemcpy(&n, d_.nlog, sizeof(long long), cudaMemcpyDeviceToHost));
        n = std::min<long long>(n, d_.cap_log);
        *count = n;
        const long long m = std::min<long long>(n, capacity);
        if (m > 0 && stp) LB_CUDA(cudaMemcpy(stp, d_.log_step, m * sizeof(long long), cudaMemcpyDeviceToHost));
        if (m > 0 && node) LB_CUDA(cudaMemcpy(node, d_.log_node, m * sizeof(long long), cudaMemcpyDeviceToHost));
        if (m > 0 && kind) LB_CUDA(cudaMemcpy(kind, d_.log_kind, m * sizeof(int), cudaMemcpyDeviceToHost));
        return 0;
    }

    int check(std::string& err) override {
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        LB_CUDA(cudaDeviceSynchronize());
        int herr = 0;
        LB_CUDA(cudaMemcpy(&herr, d_.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr & ERR_OVERFLOW) {
            err = "an internal list (events / boundary cells) exceeded its capacity";
            return 5;
        }
        if (herr & ERR_NUMERIC) {
            err = "non-finite concentration or non-positive density encountered";
            return 3;
        }
        if (herr & ERR_TIMEOUT) {
            err = "a bounded device wait of the staged sweep gave up";
            return 4;
        }
        return 0;
    }

    // Accessors used by the batched engine.
    const PhysT<T>& physt() const { return pt_; }
    int nbacc() const { return nbacc_; }
    const Geo& geo() const { return d_.geo; }
    int host_nb() const { return (int)nb0_; }
    int host_nf() const { return (int)nf0_; }
    void set_batched() { batched_ = true; }
    void force_list(bool v) { force_list_ = v; }
    bool uses_list() const { return d_.use_fl != 0; }
    double lane_efficiency() const { return lane_eff_; }
    int host_nfl() const { return (int)nfluid_; }
    // Record n steps taken by the batched kernels (parity after them: lastodd).
    void advance(int64_t n, int lastodd, cudaStream_t st) {
        steps_ += n;
        lastodd_ = lastodd;
        last_stream_ = st;
    }

    long long fluid_cells() const override { return nfluid_; }
    long long boundary_cells() const override { return nb0_; }
    int red_blocks() const { return (int)std::min<long long>(1024, (ncell_ + RED_BLOCK - 1) / RED_BLOCK); }
    const Dev<T>& dev() const { return d_; }
    const Phys& phys() const { return ph_; }
    int last_odd() const { return lastodd_; }
    cudaStream_t own_stream() const { return own_; }
    cudaStream_t last_stream() const { return last_stream_; }

    // Gradient of the reacted mass J over the next n steps (the steps are
    // taken: the simulation ends n steps later, as after lbrbc_step) with
    // respect to k_r (scalar: sum over cells), c_eq and the per-cell k_r.
    // sqrt(n) checkpoints of the full state, per-segment recomputation onto
    // a tape, reverse sweep of the adjoint kernels.
    int adjoint(int64_t n, double* J, double* dk, double* dceq, double* dk_field, std::string& err) override {
        if (ph_.phase_change) {
            err = "the adjoint needs phase change off (events are not differentiable)";
            return 1;
        }
        if (n < 1) {
            err = "n must be >= 1";
            return 1;
        }
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        cudaStream_t st = own_;
        const long long NP = d_.geo.NP;
        constexpr int QF = LF::Q > 0 ? LF::Q : 0, QG = LG::Q;
        const int64_t S = std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)n)));
        const int64_t nseg = (n + S - 1) / S;
        const size_t fbytes = (size_t)QF * NP * sizeof(T), gbytes = (size_t)QG * NP * sizeof(T);
        const size_t sbytes = (size_t)4 * d_.geo.ny * d_.geo.nz * sizeof(double);
        std::vector<void*> tmp;
        auto get = [&](size_t bytes, void** p) -> cudaError_t {
            cudaError_t e = cudaMalloc(p, bytes + 16);
            if (e == cudaSuccess) tmp.push_back(*p);
            return e;
        };
        auto cleanup = [&]() {
            cudaStreamSynchronize(st);
            for (void* p : tmp) cudaFree(p);
        };
#define LB_ACUDA(call)                                                      \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) {                                            \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            cleanup();                                                      \
            return 2;                                                       \
        }                                                                   \
    } while (0)
        const int nbk = list_grid(d_.cap_b);
        void *ck = nullptr, *gtape = nullptr, *utape = nullptr, *lam = nullptr, *nu = nullptr, *dkf = nullptr;
        void *part = nullptr, *save_phi = nullptr, *save_bacc = nullptr, *save_acc = nullptr, *fin = nullptr;
        const size_t ckb = fbytes + gbytes + sbytes;
        LB_ACUDA(get(ckb * (size_t)nseg, &ck));
        const size_t hbytes = (size_t)(QG - 1) * d_.cap_b * sizeof(T);
        LB_ACUDA(get(hbytes * (size_t)(S + 1), &gtape));
        LB_ACUDA(get((size_t)3 * NP * sizeof(float) * (size_t)(S + 1), &utape));
        LB_ACUDA(get(gbytes, &lam));
        LB_ACUDA(get(gbytes, &nu));
        LB_ACUDA(get((size_t)NP * sizeof(double), &dkf));
        LB_ACUDA(get((size_t)2 * nbk * sizeof(double), &part));
        LB_ACUDA(get((size_t)NP * sizeof(double), &save_phi));
        LB_ACUDA(get((size_t)2 * nbacc_ * sizeof(double), &save_bacc));
        LB_ACUDA(get(4 * sizeof(double), &save_acc));
        LB_ACUDA(get(ckb, &fin));
        auto save_state = [&](char* dst) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            if (QF) e = cudaMemcpyAsync(dst, d_.F, fbytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst + fbytes, d_.G, gbytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst + fbytes + gbytes, d_.side, sbytes, cudaMemcpyDeviceToDevice, st);
            return e;
        };
        auto load_state = [&](const char* src) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            if (QF) e = cudaMemcpyAsync(d_.F, src, fbytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_.G, src + fbytes, gbytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_.side, src + fbytes + gbytes, sbytes, cudaMemcpyDeviceToDevice, st);
            return e;
        };
        double led0[6];
        if (int rc = ledger(led0, err)) {
            cleanup();
            return rc;
        }
        // forward pass with checkpoints
        std::vector<int> ck_odd(nseg);
        for (int64_t sgi = 0; sgi < nseg; ++sgi) {
            LB_ACUDA(save_state((char*)ck + ckb * sgi));
            ck_odd[sgi] = lastodd_;
            const int64_t len = std::min<int64_t>(S, n - sgi * S);
            if (int rc = step(len, st, err)) {
                cleanup();
                return rc;
            }
        }
        double led1[6];
        if (int rc = ledger(led1, err)) {
            cleanup();
            return rc;
        }
        const int fin_odd = lastodd_;
        const int64_t fin_steps = steps_;
        LB_ACUDA(save_state((char*)fin));
        LB_ACUDA(cudaMemcpyAsync(save_phi, d_.phi, NP * sizeof(double), cudaMemcpyDeviceToDevice, st));
        LB_ACUDA(cudaMemcpyAsync(save_bacc, d_.bacc, 2 * nbacc_ * sizeof(double), cudaMemcpyDeviceToDevice, st));
        LB_ACUDA(cudaMemcpyAsync(save_acc, d_.acc, 4 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        // reverse sweep
        LB_ACUDA(cudaMemsetAsync(lam, 0, gbytes, st));
        LB_ACUDA(cudaMemsetAsync(dkf, 0, NP * sizeof(double), st));
        LB_ACUDA(cudaMemsetAsync(part, 0, 2 * nbk * sizeof(double), st));
        const dim3 g3((d_.geo.nx + FLUID_BLOCK - 1) / FLUID_BLOCK, d_.geo.ny, d_.geo.nz);
        for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
            LB_ACUDA(load_state((const char*)ck + ckb * sgi));
            lastodd_ = ck_odd[sgi];
            const int64_t len = std::min<int64_t>(S, n - sgi * S);
            T* ht = (T*)gtape;
            float* ut = (float*)utape;
            const size_t hstride = (size_t)(QG - 1) * d_.cap_b;
            // recompute the segment; the step kernels write the tape as they go
            for (int64_t j = 1; j <= len; ++j) {
                Dev<T> dv = d_;
                dv.tape_u = QF ? ut + (size_t)j * 3 * NP : nullptr;
                dv.tape_h = ht + (size_t)j * hstride;
                if (enqueue_step(st, !lastodd_, err, nullptr, &dv)) {
                    cleanup();
                    return 2;
                }
                lastodd_ ^= 1;
            }
            for (int64_t j = len; j >= 1; --j) {
                k_adj_fluid<T, LG><<<g3, FLUID_BLOCK, 0, st>>>(d_, ph_, pt_, (const T*)lam, (T*)nu,
                                                               QF ? ut + (size_t)j * 3 * NP : nullptr);
                k_adj_bound<T, LG><<<nbk, LIST_BLOCK, 0, st>>>(d_, ph_, pt_, (const T*)lam, (T*)nu,
                                                               ht + (size_t)j * hstride, (double*)dkf, (double*)part);
                k_adj_stream<T, LG><<<g3, FLUID_BLOCK, 0, st>>>(d_, ph_, pt_, (const T*)nu, (T*)lam);
            }
            LB_ACUDA(cudaGetLastError());
        }
        // the recomputation re-accumulated phi and the ledger: restore the
        // state reached by the forward pass
        LB_ACUDA(load_state((const char*)fin));
        LB_ACUDA(cudaMemcpyAsync(d_.phi, save_phi, NP * sizeof(double), cudaMemcpyDeviceToDevice, st));
        LB_ACUDA(cudaMemcpyAsync(d_.bacc, save_bacc, 2 * nbacc_ * sizeof(double), cudaMemcpyDeviceToDevice, st));
        LB_ACUDA(cudaMemcpyAsync(d_.acc, save_acc, 4 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        lastodd_ = fin_odd;
        steps_ = fin_steps;
        std::vector<double> hp((size_t)2 * nbk);
        LB_ACUDA(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        std::vector<double> hk;
        if (dk_field) {
            hk.resize(NP);
            LB_ACUDA(cudaMemcpyAsync(hk.data(), dkf, NP * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        LB_ACUDA(cudaStreamSynchronize(st));
        double sk = 0.0, sc = 0.0;
        for (int b = 0; b < nbk; ++b) {
            sk += hp[2 * b];
            sc += hp[2 * b + 1];
        }
        if (J) *J = led1[4] - led0[4];
        if (dk) *dk = sk;
        if (dceq) *dceq = sc;
        if (dk_field) {
            const Geo& g = d_.geo;
            for (int z = 0; z < g.nz; ++z)
                for (int y = 0; y < g.ny; ++y)
                    for (int x = 0; x < g.nx; ++x)
                        dk_field[x + (long long)g.nx * (y + (long long)g.ny * z)] = hk[g.idx(x, y, z)];
        }
#undef LB_ACUDA
        cleanup();
        return 0;
    }

   private:
    // Allocation owned by the simulation until release().
    template <typename U>
    cudaError_t dalloc(U** p, size_t n) {
        cudaError_t e = cudaMalloc((void**)p, n * sizeof(U) + 16);
        if (e == cudaSuccess) allocs_.push_back((void*)*p);
        return e;
    }
    // Temporary allocation, freed by the caller.
    template <typename U>
    static cudaError_t talloc(U** p, size_t n) {
        return cudaMalloc((void**)p, n * sizeof(U) + 16);
    }

    static int grid_for(long long n, int block) {
        long long b = (n + block - 1) / block;
        return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 16));
    }

    // Initial sizes of the wet-boundary list (non-fluid cells with a fluid
    // solute-lattice neighbour) and of the fluid-end list (fluid cells with a
    // reactive neighbour at x - e_o), counted on the host to size the lists.
    // The kinds are copied into a grid with one ghost layer (periodic axes
    // wrapped, others marked outside) so the count runs with fixed neighbour
    // offsets, split over host threads by z.
    void count_lists_host(const std::vector<uint8_t>& kind, long long& nb, long long& nf) const {
        const Geo& g = d_.geo;
        const int X = g.nx + 2, Y = g.ny + 2, Z = g.nz + 2;
        const uint8_t OUT = 255;
        std::vector<uint8_t> K((size_t)X * Y * Z, OUT);
        auto wrap = [](int v, int n, bool per) { return per ? (v + n) % n : v; };
        for (int z = -1; z <= g.nz; ++z)
            for (int y = -1; y <= g.ny; ++y)
                for (int x = -1; x <= g.nx; ++x) {
                    const int xs = wrap(x, g.nx, g.per_x), ys = wrap(y, g.ny, g.per_y), zs = wrap(z, g.nz, g.per_z);
                    if (xs < 0 || xs >= g.nx || ys < 0 || ys >= g.ny || zs < 0 || zs >= g.nz) continue;
                    K[(size_t)(x + 1) + (size_t)X * ((y + 1) + (size_t)Y * (z + 1))] = kind[g.idx(xs, ys, zs)];
                }
        long long off[LG::Q];
        for (int o = 0; o < LG::Q; ++o) off[o] = LG::cx(o) + (long long)X * (LG::cy(o) + (long long)Y * LG::cz(o));
        const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<long long> cb(nt, 0), cf(nt, 0);
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t)
            pool.emplace_back([&, t]() {
                long long b = 0, f = 0;
                for (int z = t; z < g.nz; z += nt)
                    for (int y = 0; y < g.ny; ++y) {
                        const uint8_t* row = K.data() + (size_t)X * ((y + 1) + (size_t)Y * (z + 1)) + 1;
                        for (int x = 0; x < g.nx; ++x) {
                            const uint8_t* c = row + x;
                            if (*c == KIND_FLUID) {
                                for (int o = 1; o < LG::Q; ++o)
                                    if (c[-off[o]] == KIND_REACTIVE) {
                                        ++f;
                                        break;
                                    }
                            } else {
                                for (int o = 1; o < LG::Q; ++o)
                                    if (c[off[o]] == KIND_FLUID) {
                                        ++b;
                                        break;
                                    }
                            }
                        }
                    }
                cb[t] = b;
                cf[t] = f;
            });
        for (auto& th : pool) th.join();
        nb = nf = 0;
        for (int t = 0; t < nt; ++t) {
            nb += cb[t];
            nf += cf[t];
        }
    }

    // Reclassification and list rebuild (force = 1 at creation: unconditional).
    int rebuild(cudaStream_t st, int lastodd, int force, std::string& err) {
        k_reclassify<T, LF, LG><<<grid_for(ncell_, 256), 256, 0, st>>>(d_, ph_, lastodd, force);
        if (sweep_ == SWEEP_STAGED) k_tile_flags<T><<<grid_for((long long)d_.ntiles * 32, 256), 256, 0, st>>>(d_, force);
        for (int which = 0; which < (d_.use_fl ? 3 : 2); ++which) {
            k_count<T, LG><<<nchunks_, 256, 0, st>>>(d_, which, force);
            k_scan<T><<<1, 1024, 0, st>>>(d_, nchunks_, which, force);
            k_write_lists<T, LG><<<nchunks_, 256, 0, st>>>(d_, ph_, which, force);
        }
        LB_CUDA(cudaGetLastError());
        return 0;
    }

    // One time step; with `ev` (5 events) the kernel groups are bracketed by
    // event records: fluid sweep, boundary list, fluid ends, phase change.
    int enqueue_step(cudaStream_t st, bool odd, std::string& err, cudaEvent_t* ev = nullptr,
                     const Dev<T>* dv = nullptr) {
        const Dev<T>& d_ = dv ? *dv : this->d_;
        const Geo& g = d_.geo;
        dim3 grid((g.nx + FLUID_BLOCK - 1) / FLUID_BLOCK, g.ny, g.nz);
        if (ev) LB_CUDA(cudaEventRecord(ev[0], st));
        // Without per-group timing the boundary list and the fluid ends run
        // on a second stream beside the fluid sweep: the three kernels touch
        // disjoint population slots (each slot is read and written by one
        // cell per step), and the fluid ends depend only on the boundary list.
        const bool fork = ev == nullptr;
        if (fork) {
            LB_CUDA(cudaEventRecord(fork_, st));
            LB_CUDA(cudaStreamWaitEvent(aux_, fork_, 0));
            const int lg = list_grid(d_.cap_b);
            if (odd) k_bound<T, LG, true><<<lg, LIST_BLOCK, 0, aux_>>>(d_, ph_, pt_);
            else k_bound<T, LG, false><<<lg, LIST_BLOCK, 0, aux_>>>(d_, ph_, pt_);
            k_fend<T, LG><<<list_grid(d_.cap_f), LIST_BLOCK, 0, aux_>>>(d_, ph_);
            LB_CUDA(cudaEventRecord(join_, aux_));
        }
        if (sweep_ == SWEEP_STAGED) {
            const size_t sm = (size_t)staged_stages<T>() * staged_stage_bytes<T, LF, LG>();
            if (odd) k_fluid_staged<T, LF, LG, true><<<sgrid_, TILE_X, sm, st>>>(d_, ph_, pt_);
            else k_fluid_staged<T, LF, LG, false><<<sgrid_, TILE_X, sm, st>>>(d_, ph_, pt_);
        } else if (d_.use_fl) {
            const int gl = (int)((d_.cap_fl + FLUID_BLOCK - 1) / FLUID_BLOCK);
            if (odd) k_fluid_list<T, LF, LG, true><<<gl, FLUID_BLOCK, 0, st>>>(d_, ph_, pt_);
            else k_fluid_list<T, LF, LG, false><<<gl, FLUID_BLOCK, 0, st>>>(d_, ph_, pt_);
        } else {
            if (odd) k_fluid<T, LF, LG, true><<<grid, FLUID_BLOCK, 0, st>>>(d_, ph_, pt_);
            else k_fluid<T, LF, LG, false><<<grid, FLUID_BLOCK, 0, st>>>(d_, ph_, pt_);
        }
        if (fork) {
            LB_CUDA(cudaStreamWaitEvent(st, join_, 0));
        } else {
            LB_CUDA(cudaEventRecord(ev[1], st));
            const int lg = list_grid(d_.cap_b);
            if (odd) k_bound<T, LG, true><<<lg, LIST_BLOCK, 0, st>>>(d_, ph_, pt_);
            else k_bound<T, LG, false><<<lg, LIST_BLOCK, 0, st>>>(d_, ph_, pt_);
            LB_CUDA(cudaEventRecord(ev[2], st));
            k_fend<T, LG><<<list_grid(d_.cap_f), LIST_BLOCK, 0, st>>>(d_, ph_);
            LB_CUDA(cudaEventRecord(ev[3], st));
        }
        if (ph_.phase_change) {
            const int eg = 152 * 2;
            const int lo = odd ? 1 : 0;
            k_ev_mark<T><<<eg, 256, 0, st>>>(d_);
            k_ev_compute<T, LF, LG><<<eg, 256, 0, st>>>(d_, ph_, lo);
            k_ev_apply_self<T, LF, LG><<<eg, 256, 0, st>>>(d_, ph_, lo);
            k_ev_neighbours<T, LG><<<eg, 256, 0, st>>>(d_, ph_, lo);
            if (rebuild(st, lo, 0, err)) return 2;
            k_ev_reset<T><<<eg, 256, 0, st>>>(d_);
            k_step_end<T><<<1, 1, 0, st>>>(d_);
        }
        if (ev) LB_CUDA(cudaEventRecord(ev[4], st));
        LB_CUDA(cudaGetLastError());
        return 0;
    }

   public:
    // Number of kernel launches of one step.
    int launches_per_step() const override { return 3 + (ph_.phase_change ? 5 + 3 * 2 + 2 + 1 : 0); }

    // Run n steps without graphs, timing each kernel group with CUDA events on
    // the stream the kernels run on; ms[g] = mean duration of group g.
    int profile(int64_t n, cudaStream_t s, double* ms, std::string& err) override {
        cudaStream_t st = s ? s : own_;
        n = std::max<int64_t>(1, std::min<int64_t>(n, 4096));
        std::vector<cudaEvent_t> ev((size_t)5 * n);
        for (auto& e : ev) LB_CUDA(cudaEventCreate(&e));
        for (int64_t k = 0; k < n; ++k) {
            const bool odd = !lastodd_;
            if (enqueue_step(st, odd, err, &ev[(size_t)5 * k])) return 2;
            lastodd_ ^= 1;
        }
        steps_ += n;
        last_stream_ = st;
        LB_CUDA(cudaStreamSynchronize(st));
        double acc[4] = {0, 0, 0, 0};
        for (int64_t k = 0; k < n; ++k)
            for (int q = 0; q < 4; ++q) {
                float t = 0.f;
                LB_CUDA(cudaEventElapsedTime(&t, ev[(size_t)5 * k + q], ev[(size_t)5 * k + q + 1]));
                acc[q] += t;
            }
        for (int q = 0; q < 4; ++q) ms[q] = acc[q] / (double)n;
        for (auto& e : ev) cudaEventDestroy(e);
        return 0;
    }

   private:
    // Shared memory and persistent grid of the staged sweep: as many CTAs as
    // fit on the device at once (never more than there are tiles).
    int setup_staged(std::string& err) {
        const size_t sm = (size_t)staged_stages<T>() * staged_stage_bytes<T, LF, LG>();
        int occ = 64;
        int dev = 0, nsm = 0;
        LB_CUDA(cudaGetDevice(&dev));
        LB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        auto occ_of = [&](auto kern) -> int {
            int o = 0;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
            // the persistent grid assumes every CTA of the occupancy
            // estimate is resident: ask for the largest shared-memory carveout
            if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
                return -1;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, TILE_X, sm) != cudaSuccess) return -1;
            return o;
        };
        const int o[2] = {occ_of(k_fluid_staged<T, LF, LG, false>), occ_of(k_fluid_staged<T, LF, LG, true>)};
        for (int k = 0; k < 2; ++k) {
            if (o[k] < 0) {
                err = std::string("staged sweep setup: ") + cudaGetErrorString(cudaGetLastError());
                return 2;
            }
            occ = std::min(occ, o[k]);
        }
        occ = std::max(1, occ);
        sgrid_ = (int)std::max<long long>(1, std::min<long long>((long long)nsm * occ, d_.ntiles));
        return 0;
    }

    static int list_grid(int cap) {
        return (int)std::max(1, std::min(152 * 8, (cap + LIST_BLOCK - 1) / LIST_BLOCK));
    }

    int build_graphs(std::string& err) {
        cudaStream_t cs;
        LB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        auto cap = [&](cudaGraphExec_t* out, int mode) -> int {
            cudaGraph_t gr;
            LB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            int r = 0;
            if (mode == 0) r = enqueue_step(cs, false, err);
            else if (mode == 1) r = enqueue_step(cs, true, err);
            else {
                r = enqueue_step(cs, false, err);
                if (!r) r = enqueue_step(cs, true, err);
            }
            cudaError_t e = cudaStreamEndCapture(cs, &gr);
            if (r) return r;
            if (e != cudaSuccess) {
                err = std::string("graph capture: ") + cudaGetErrorString(e);
                return 2;
            }
            LB_CUDA(cudaGraphInstantiate(out, gr, 0));
            cudaGraphDestroy(gr);
            return 0;
        };
        if (cap(&g_even_, 0) || cap(&g_odd_, 1) || cap(&g_pair_, 2)) {
            cudaStreamDestroy(cs);
            return 2;
        }
        graphs_ = true;
        cudaStreamDestroy(cs);
        return 0;
    }

    void release() {
        if (graphs_) {
            cudaGraphExecDestroy(g_even_);
            cudaGraphExecDestroy(g_odd_);
            cudaGraphExecDestroy(g_pair_);
            graphs_ = false;
        }
        if (own_) cudaStreamSynchronize(own_);
        for (void* p : allocs_) cudaFree(p);
        allocs_.clear();
        if (own_) cudaStreamDestroy(own_);
        own_ = nullptr;
        if (aux_) cudaStreamDestroy(aux_);
        aux_ = nullptr;
        if (fork_) cudaEventDestroy(fork_);
        if (join_) cudaEventDestroy(join_);
        fork_ = join_ = nullptr;
    }

    lbrbc_params prm_{};
    Dev<T> d_{};
    Phys ph_{};
    PhysT<T> pt_{};
    long long ncell_ = 0, nfluid_ = 0, nb0_ = 0, nf0_ = 0;
    int nchunks_ = 0;
    int nbacc_ = 0;
    int lastodd_ = 1;
    int64_t steps_ = 0;
    cudaStream_t own_ = nullptr, last_stream_ = nullptr, aux_ = nullptr;
    cudaEvent_t fork_ = nullptr, join_ = nullptr;
    int sweep_ = SWEEP_DENSE;
    int sgrid_ = 1;
    cudaGraphExec_t g_even_{}, g_odd_{}, g_pair_{};
    bool graphs_ = false;
    bool batched_ = false;
    bool force_list_ = false;
    double lane_eff_ = 1.0;
    std::vector<void*> allocs_;
};

#undef LB_CUDA

}  // namespace lbrbc
