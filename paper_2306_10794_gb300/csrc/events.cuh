// Phase change (Sec. 2.4) and what follows it on the device: the event
// kernels, the reclassification of cells, the local and full maintenance of
// the boundary and fluid-end lists, and the active-cell layout's stored-set
// numbering, neighbour tables, link swaps and repacking.  Included by
// engine.cuh at this point of its definitions (namespace lbrbc).
#pragma once

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
        const double Cself = p.cref + (double)post_sum<LG, false, T>(a, a.G, id, d, lastodd);
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
                    sc += p.cref + (double)post_sum<LG, false, T>(a, a.G, nb, dn, lastodd);
                    if constexpr (LF::Q > 0) sr += 1.0 + (double)post_sum<LF, true, T>(a, a.F, nb, dn, lastodd);
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
            if (!ns) fx_add(a.facc + 2, -Q / p.Vm);
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
                a.G[post_slot<LG, false, T>(a, id, d, i, lastodd)] = T(gweight<LG>(p, i) * (cinit - p.cref));
            if constexpr (LF::Q > 0) {
#pragma unroll
                for (int i = 0; i < LF::Q; ++i) a.F[post_slot<LF, true, T>(a, id, d, i, lastodd)] = T(LF::w(i) * (rinit - 1.0));
            }
            a.phi[id] = 0.0;
        } else {
#pragma unroll
            for (int i = 0; i < LG::Q; ++i)
                a.G[post_slot<LG, false, T>(a, id, d, i, lastodd)] = T(-gweight<LG>(p, i) * p.cref);
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
                const long long s = post_slot<LG, false, T>(a, tgt, d, i, lastodd);
                a.G[s] = T((double)a.G[s] + gweight<LG>(p, i) * dC);
            }
        }
    }
}

// New class of in-grid cell (x, y, z) from the kinds; a boundary cell that
// lost its last fluid neighbour converts its solute into phi, a solid cell
// that gained one starts empty.  force: creation (no state to convert).
template <typename T, class LF, class LG>
__device__ uint32_t reclass_transition(const Dev<T>& a, const Phys& p, int x, int y, int z, long long id,
                                       int lastodd, int force) {
    const Geo& g = a.geo;
    const uint32_t cls = class_of<LG>(g, a.kind, x, y, z);
    const uint32_t old = a.nw[id] & 3u;
    if (!force && old != cls && a.evidx[id] < 0) {
        const Nbr d = nbr_deltas(g, x, y, z);
        if (old == CLS_BOUND && cls == CLS_SOLID) {
            const double C = p.cref + (double)post_sum<LG, false, T>(a, a.G, id, d, lastodd);
            if (a.kind[id] == KIND_REACTIVE) a.phi[id] += p.Vm * C;
            else fx_add(a.facc, -C);
        }
        if (cls != CLS_FLUID) {
            if (a.sparse && a.cmap[id] < 0) {
                // a solid cell outside the stored set gained a fluid
                // neighbour: the layout is repacked before the next step,
                // and the repacking gives it its starting populations
                *a.repack = 1;
            } else {
#pragma unroll
                for (int i = 0; i < LG::Q; ++i)
                    a.G[post_slot<LG, false, T>(a, id, d, i, lastodd)] = T(-gweight<LG>(p, i) * p.cref);
            }
        }
    }
    return cls;
}

// Node word of cell (x, y, z) of class cls: for a fluid cell the inactive
// sources of both lattices (flow: not fluid; solute: solid) and the open
// faces.  cls_at(x, y, z) gives the class of any position (solid outside a
// wall axis).
template <class LF, class LG, class ClassAt>
__device__ __forceinline__ uint32_t node_word(const Geo& g, int x, int y, int z, uint32_t cls, const ClassAt& cls_at) {
    uint32_t w = cls;
    if (cls == CLS_FLUID) {
        if constexpr (LF::Q > 0) {
#pragma unroll
            for (int i = 1; i < LF::Q; ++i)
                if (cls_at(x - LF::cx(i), y - LF::cy(i), z - LF::cz(i)) != CLS_FLUID) w |= 1u << (FBIT + i - 1);
        }
#pragma unroll
        for (int i = 1; i < LG::Q; ++i)
            if (cls_at(x - LG::cx(i), y - LG::cy(i), z - LG::cz(i)) == CLS_SOLID) w |= 1u << (GBIT + i - 1);
        if (g.open_x && x == 0) w |= NW_INLET;
        if (g.open_x && x == g.nx - 1) w |= NW_OUTLET;
    }
    return w;
}

template <typename T>
__device__ __forceinline__ void store_word(const Dev<T>& a, long long id, uint32_t w) {
    a.nw[id] = w;
    if (a.sparse) {
        const int c = a.cmap[id];
        if (c >= 0) a.nwc[c] = w;
    }
}

// New class and node word of in-grid cell (x, y, z) with the neighbours'
// classes taken from the kinds (their node words may be changing in the same
// pass): the local reclassification.
template <typename T, class LF, class LG>
__device__ void reclassify_cell(const Dev<T>& a, const Phys& p, int x, int y, int z, long long id, int lastodd,
                                int force) {
    const Geo& g = a.geo;
    const uint32_t cls = reclass_transition<T, LF, LG>(a, p, x, y, z, id, lastodd, force);
    const uint32_t w = node_word<LF, LG>(g, x, y, z, cls, [&](int xx, int yy, int zz) {
        return class_at<LG>(g, a.kind, xx, yy, zz);
    });
    store_word(a, id, w);
}

// Local list maintenance: counters in Dev::lcnt.
enum {
    LC_CANDB = 0,   // new wet boundary cells of this step
    LC_CANDF = 1,   // new fluid ends of this step
    LC_DEADB = 2,   // dead boundary entries since the last compaction
    LC_DEADF = 3,   // dead fluid-end entries since the last compaction
    LC_FULL = 4,    // this step reclassifies the whole grid / compacts the lists
    LC_LOCAL = 5,   // this step updates the region around the events only
    LC_BASEB = 6,   // list lengths before this step's appends
    LC_BASEF = 7,
    LC_NREG = 8,    // cells of this step's region
    LC_EVMAX = 9,   // events of a step handled locally (at most LOC_EV_MAX; more: whole grid)
    LC_N = 16
};
// Cells that a change of kind at an event cell can affect: a cell's class
// depends on the kinds of its solute-lattice neighbours, a node word on the
// classes of its flow- and solute-lattice neighbours, a boundary entry on the
// kinds within two solute links and the wall normal's D3Q19 / D2Q9 stencil,
// and a cell's fluid-end status on the classes of its solute-lattice
// neighbours.  Every such offset lies in the cube of half width 2.
constexpr int LOC_HALF = 2;
constexpr int LOC_CAND_CAP = 8192;    // appends per list and step (more: full compaction)
constexpr int LOC_EV_MAX = 16384;     // largest limit of events handled locally (region list size)

template <int DIM>
__host__ __device__ constexpr int loc_cube() {
    return DIM == 3 ? (2 * LOC_HALF + 1) * (2 * LOC_HALF + 1) * (2 * LOC_HALF + 1)
                    : (2 * LOC_HALF + 1) * (2 * LOC_HALF + 1);
}

// List entry of wet boundary cell (x, y, z) at position pos: its index,
// coordinates and compact index, its word (inactive sources, links to fluid
// cells, Dirichlet flag), the link coefficients (e_o . n)+ of the wall normal
// and its rate, from the current kinds and node words.  The share sources
// are set by the fluid ends.
template <typename T, class LG>
__device__ void bound_entry_data(const Dev<T>& a, const Phys& p, int x, int y, int z, long long id, int pos) {
    const Geo& g = a.geo;
    a.b_idx[pos] = (int)id;
    if (a.sparse) a.b_cn[pos] = a.cmap[id];
    a.b_xyz[pos] = pack_xyz(x, y, z);
    uint32_t bw = 0;
    const uint8_t kd = a.kind[id];
    if (kd == KIND_DIRICHLET) bw |= BW_DIRICHLET;
    double nrm[3];
    const bool ok = wall_normal<LG::DIM>(g, a.kind, x, y, z, nrm);
#pragma unroll
    for (int o = 1; o < LG::Q; ++o) {
        int xs = x - LG::cx(o), ys = y - LG::cy(o), zs = z - LG::cz(o);
        if (!wrap_inside(g, xs, ys, zs) || (a.nw[g.idx(xs, ys, zs)] & 3u) == CLS_SOLID) bw |= 1u << (o - 1);
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
}

// Whether the full compaction of the lists runs: at creation, when the
// local maintenance asked for it, or (without local maintenance) on every
// step with events.
template <typename T>
__device__ __forceinline__ bool full_lists(const Dev<T>& a, int force) {
    return force || (a.lcnt ? a.lcnt[LC_FULL] != 0 : *a.nev != 0);
}

// New classes and node words over the whole grid (at creation, and in a
// step whose events are too many for the local update), in two passes:
// the classes from the kinds, then the node words from the neighbours'
// classes (a few byte loads per direction instead of recomputing each
// neighbour's class from its kinds).
template <typename T>
__device__ __forceinline__ bool full_reclass(const Dev<T>& a, int force) {
    return force || (a.lcnt ? a.lcnt[LC_FULL] != 0 : *a.nev != 0);
}

template <typename T, class LF, class LG>
__global__ void k_reclassify(const Dev<T> a, const Phys p, int lastodd, int force) {
    if (!full_reclass(a, force)) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        a.nw[id] = reclass_transition<T, LF, LG>(a, p, x, y, z, id, lastodd, force);
    }
}

template <typename T, class LF, class LG>
__global__ void k_recl_words(const Dev<T> a, int force) {
    if (!full_reclass(a, force)) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        const uint32_t w = node_word<LF, LG>(g, x, y, z, a.nw[id] & 3u, [&](int xx, int yy, int zz) {
            return wrap_inside(g, xx, yy, zz) ? (a.nw[g.idx(xx, yy, zz)] & 3u) : CLS_SOLID;
        });
        store_word(a, id, w);
    }
}

// Whether this step's events are handled locally (one thread).
template <typename T>
__global__ void k_loc_decide(const Dev<T> a) {
    int* c = a.lcnt;
    c[LC_CANDB] = c[LC_CANDF] = c[LC_NREG] = 0;
    const int nev = *a.nev;
    const bool any = nev > 0;
    const bool local = any && nev <= c[LC_EVMAX] && nev <= a.cap_e;
    c[LC_LOCAL] = local;
    c[LC_FULL] = any && !local;
}

// Cell of the region: offset t of the cube around event e, wrapped into the
// grid; false outside it.
template <class LG>
__device__ __forceinline__ bool loc_cell(const Geo& g, const int* ev_node, long long t, int& x, int& y, int& z) {
    constexpr int W = 2 * LOC_HALF + 1, NC = loc_cube<LG::DIM>();
    const int e = (int)(t / NC), j = (int)(t % NC);
    coords(g, ev_node[e], x, y, z);
    x += j % W - LOC_HALF;
    y += (j / W) % W - LOC_HALF;
    if (LG::DIM == 3) z += j / (W * W) - LOC_HALF;
    return wrap_inside(g, x, y, z);
}

// Local reclassification: every cell of the cubes around the events once
// (a per-step stamp claims it), recorded in the region list.
template <typename T, class LF, class LG>
__global__ void k_loc_recl(const Dev<T> a, const Phys p, int lastodd) {
    if (!a.lcnt[LC_LOCAL]) return;
    const Geo& g = a.geo;
    const long long total = (long long)*a.nev * loc_cube<LG::DIM>();
    const uint32_t stamp = (uint32_t)*a.step + 1u;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        if (!loc_cell<LG>(g, a.ev_node, t, x, y, z)) continue;
        const long long id = g.idx(x, y, z);
        if (atomicExch(&a.lmark[id], stamp) == stamp) continue;
        reclassify_cell<T, LF, LG>(a, p, x, y, z, id, lastodd, 0);
        a.rlist[atomicAdd(&a.lcnt[LC_NREG], 1)] = (int)id;
    }
}

// Whether fluid cell (x, y, z) is a fluid end: a reactive wet boundary cell
// upstream along a solute link.
template <typename T, class LG>
__device__ __forceinline__ bool is_fluid_end(const Dev<T>& a, int x, int y, int z) {
    const Geo& g = a.geo;
#pragma unroll
    for (int o = 1; o < LG::Q; ++o) {
        int xx = x - LG::cx(o), yy = y - LG::cy(o), zz = z - LG::cz(o);
        if (!wrap_inside(g, xx, yy, zz)) continue;
        const long long nb = g.idx(xx, yy, zz);
        if ((a.nw[nb] & 3u) == CLS_BOUND && a.kind[nb] == KIND_REACTIVE) return true;
    }
    return false;
}

// Region cells against the lists: boundary entries of cells that stay wet
// boundary cells are recomputed in place, entries of cells that left a list
// are marked dead, cells that joined one become candidates.
template <typename T, class LG>
__global__ void k_loc_lists(const Dev<T> a, const Phys p) {
    if (!a.lcnt[LC_LOCAL] || a.lcnt[LC_FULL]) return;
    const Geo& g = a.geo;
    const int n = a.lcnt[LC_NREG];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const long long id = a.rlist[r];
        int x, y, z;
        coords(g, id, x, y, z);
        const uint32_t cls = a.nw[id] & 3u;
        const int pb = a.bmap[id];
        if (cls == CLS_BOUND) {
            if (pb >= 0) {
                bound_entry_data<T, LG>(a, p, x, y, z, id, pb);
            } else {
                const int k = atomicAdd(&a.lcnt[LC_CANDB], 1);
                if (k < LOC_CAND_CAP) a.candb[k] = (int)id;
            }
        } else if (pb >= 0) {
            a.b_word[pb] = BW_DEAD;
            a.bmap[id] = -1;
            atomicAdd(&a.lcnt[LC_DEADB], 1);
        }
        const bool fe = cls == CLS_FLUID && is_fluid_end<T, LG>(a, x, y, z);
        const int pf = a.fmap[id];
        if (fe && pf < 0) {
            const int k = atomicAdd(&a.lcnt[LC_CANDF], 1);
            if (k < LOC_CAND_CAP) a.candf[k] = (int)id;
        } else if (!fe && pf >= 0) {
            a.f_idx[pf] = -1;
            a.fmap[id] = -1;
            atomicAdd(&a.lcnt[LC_DEADF], 1);
        }
    }
}

// Room for the appends, or a full compaction instead (too many candidates,
// no capacity left, or more than an eighth of a list dead); one thread.
template <typename T>
__global__ void k_loc_plan(const Dev<T> a) {
    int* c = a.lcnt;
    if (!c[LC_LOCAL] || c[LC_FULL]) return;
    const int cb = c[LC_CANDB], cf = c[LC_CANDF];
    const long long nb = *a.nb, nf = *a.nf;
    if (cb > LOC_CAND_CAP || cf > LOC_CAND_CAP || nb + cb > a.cap_b || nf + cf > a.cap_f ||
        8LL * c[LC_DEADB] > nb + cb || 8LL * c[LC_DEADF] > nf + cf) {
        c[LC_FULL] = 1;
        return;
    }
    c[LC_BASEB] = (int)nb;
    c[LC_BASEF] = (int)nf;
    *a.nb = (int)(nb + cb);
    *a.nf = (int)(nf + cf);
}

// Appends in cell order (rank among the candidates), so that the lists do
// not depend on thread timing.
template <typename T, class LG>
__global__ void k_loc_append(const Dev<T> a, const Phys p) {
    if (!a.lcnt[LC_LOCAL] || a.lcnt[LC_FULL]) return;
    const Geo& g = a.geo;
    const int cb = a.lcnt[LC_CANDB], cf = a.lcnt[LC_CANDF];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cb + cf; t += gridDim.x * blockDim.x) {
        const bool isb = t < cb;
        const int* cand = isb ? a.candb : a.candf;
        const int nc = isb ? cb : cf;
        const int id = cand[isb ? t : t - cb];
        int rank = 0;
        for (int k = 0; k < nc; ++k) rank += cand[k] < id;
        if (isb) {
            const int pos = a.lcnt[LC_BASEB] + rank;
            int x, y, z;
            coords(g, id, x, y, z);
            a.bmap[id] = pos;
            bound_entry_data<T, LG>(a, p, x, y, z, id, pos);
        } else {
            const int pos = a.lcnt[LC_BASEF] + rank;
            a.f_idx[pos] = id;
            a.fmap[id] = pos;
#pragma unroll
            for (int o = 1; o < LG::Q; ++o) a.f_src[(long long)(o - 1) * a.cap_f + pos] = -1;
        }
    }
}

// Share sources of the fluid ends of the region: link o gathers from the
// reactive wet boundary cell at x - e_o.  Fluid ends outside the region keep
// theirs: a source entry moves only when it is appended or dies, both within
// one cell of an event, and its fluid ends then lie in the region.
template <typename T, class LG>
__global__ void k_loc_fsrc(const Dev<T> a) {
    if (!a.lcnt[LC_LOCAL] || a.lcnt[LC_FULL]) return;
    const Geo& g = a.geo;
    const int n = a.lcnt[LC_NREG];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const long long id = a.rlist[r];
        const int pf = a.fmap[id];
        if (pf < 0) continue;
        int x, y, z;
        coords(g, id, x, y, z);
#pragma unroll
        for (int o = 1; o < LG::Q; ++o) {
            int xs = x - LG::cx(o), ys = y - LG::cy(o), zs = z - LG::cz(o);
            int src = -1;
            if (wrap_inside(g, xs, ys, zs)) {
                const long long nb = g.idx(xs, ys, zs);
                const int pb = a.bmap[nb];
                if (pb >= 0 && (a.nw[nb] & 3u) == CLS_BOUND && a.kind[nb] == KIND_REACTIVE) src = (o - 1) * a.cap_b + pb;
            }
            a.f_src[(long long)(o - 1) * a.cap_f + pf] = src;
        }
    }
}

// Stream compaction of the wet boundary cells (order = cell index).
// Pass 1: counts per chunk of SCAN_CHUNK cells.
template <typename T, class LG>
__global__ void k_count(const Dev<T> a, int which, int force, int nchunks) {
    if (!full_lists(a, force)) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    __shared__ int cnt;
    for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        int local = 0;
        for (long long t = chunk * SCAN_CHUNK + threadIdx.x; t < min(total, (chunk + 1) * SCAN_CHUNK);
             t += blockDim.x) {
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
        __syncthreads();
    }
}

// Pass 2: exclusive scan of the chunk counts (one block); total -> *count.
template <typename T>
__global__ void k_scan(const Dev<T> a, int nchunks, int which, int force) {
    if (!full_lists(a, force)) return;
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
__global__ void k_write_lists(const Dev<T> a, const Phys p, int which, int force, int nchunks) {
    if (!full_lists(a, force)) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    __shared__ int warp_tot[32];
    __shared__ int base_s;
    for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
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
            } else if (a.fmap) {
                a.fmap[id] = -1;
            }
            if (which == 1 && cls == CLS_FLUID) {
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
                a.bmap[id] = pos;
                bound_entry_data<T, LG>(a, p, x, y, z, id, pos);
            } else if (which == 2 && pos < a.cap_fl) {
                a.fl_xyz[pos] = (uint32_t)x | ((uint32_t)y << 11) | ((uint32_t)z << 22);
            } else if (which == 1 && pos < a.cap_f) {
                a.f_idx[pos] = (int)id;
                if (a.fmap) a.fmap[id] = pos;
#pragma unroll
                for (int o = 1; o < LG::Q; ++o) {
                    a.f_src[(long long)(o - 1) * a.cap_f + pos] = src[o] >= 0 ? (o - 1) * a.cap_b + src[o] : -1;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base_s += tot;
        __syncthreads();
    }
    }
}

// ---------------------------------------------------------------------------
// Active-cell layout: the stored set, its numbering and neighbour table, and
// the event path's link swaps.
// ---------------------------------------------------------------------------
constexpr int RNONE = 0x7f7f7f7f;  // rown of a cell outside the event region (byte-filled)

// Range of every in-grid cell in the stored set from the current classes:
// 0 fluid, 1 wet boundary, 2 solid with a wet-boundary neighbour along the
// solute lattice (the margin a dissolution can turn into boundary cells),
// 3 not stored.
template <typename T, class LG>
__global__ void k_sp_mark(const Dev<T> a, uint8_t* __restrict__ code, const int* __restrict__ go) {
    if (go && *go == 0) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx);
        const int y = (int)((t / g.nx) % g.ny);
        const int z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        const uint32_t c = a.nw[id] & 3u;
        uint8_t r = c == CLS_FLUID ? 0 : (c == CLS_BOUND ? 1 : 3);
        if (r == 3) {
#pragma unroll
            for (int o = 1; o < LG::Q; ++o) {
                int xx = x + LG::cx(o), yy = y + LG::cy(o), zz = z + LG::cz(o);
                if (wrap_inside(g, xx, yy, zz) && (a.nw[g.idx(xx, yy, zz)] & 3u) == CLS_BOUND) r = 2;
            }
        }
        code[id] = r;
    }
}

// Per chunk of SCAN_CHUNK cells (x-fastest order): cells of range r.
template <typename T>
__global__ void k_sp_count(const Dev<T> a, const uint8_t* __restrict__ code, int r, const int* __restrict__ go,
                           int nchunks) {
    if (go && *go == 0) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    __shared__ int cnt;
    for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        int local = 0;
        for (long long t = chunk * SCAN_CHUNK + threadIdx.x; t < min(total, (chunk + 1) * SCAN_CHUNK);
             t += blockDim.x) {
            const int x = (int)(t % g.nx);
            const int y = (int)((t / g.nx) % g.ny);
            const int z = (int)(t / ((long long)g.nx * g.ny));
            local += code[g.idx(x, y, z)] == r;
        }
        atomicAdd(&cnt, local);
        __syncthreads();
        if (threadIdx.x == 0) a.blk[chunk] = cnt;
        __syncthreads();
    }
}

// Exclusive scan of the chunk counts (one block); the range total goes to
// tot[r].
template <typename T>
__global__ void k_sp_scan(const Dev<T> a, int nchunks, int r, int* __restrict__ tot, const int* __restrict__ go) {
    if (go && *go == 0) return;
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
        tot[r] = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int c = lo; c < hi; ++c) {
        const int v = a.blk[c];
        a.blk[c] = run;
        run += v;
    }
}

// Compact indices of range r in chunk order after the ranges before it
// (cmap_out must hold -1 for every cell beforehand).  Positions beyond the
// capacity raise ERR_OVERFLOW and are not written.
template <typename T>
__global__ void k_sp_write(const Dev<T> a, const uint8_t* __restrict__ code, int r, const int* __restrict__ tot,
                           int* __restrict__ cmap_out, int* __restrict__ cid_out, const int* __restrict__ go,
                           int nchunks) {
    if (go && *go == 0) return;
    const Geo& g = a.geo;
    const long long total = (long long)g.nx * g.ny * g.nz;
    __shared__ int warp_tot[32];
    __shared__ int base_s;
    for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    if (threadIdx.x == 0) {
        int b = a.blk[chunk];
        for (int k = 0; k < r; ++k) b += tot[k];
        base_s = b;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw_ = blockDim.x >> 5;
    const long long end = min(total, (chunk + 1) * SCAN_CHUNK);
    for (long long t0 = chunk * SCAN_CHUNK; t0 < end; t0 += blockDim.x) {
        const long long t = t0 + threadIdx.x;
        bool sel = false;
        long long id = 0;
        if (t < end) {
            const int x = (int)(t % g.nx);
            const int y = (int)((t / g.nx) % g.ny);
            const int z = (int)(t / ((long long)g.nx * g.ny));
            id = g.idx(x, y, z);
            sel = code[id] == r;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, sel);
        if (lane == 0) warp_tot[wid] = __popc(bal);
        __syncthreads();
        int woff = 0, tt = 0;
        for (int k = 0; k < nw_; ++k) {
            if (k < wid) woff += warp_tot[k];
            tt += warp_tot[k];
        }
        const int pos = base_s + woff + __popc(bal & ((1u << lane) - 1u));
        if (sel) {
            if (pos < a.cap_s) {
                cmap_out[id] = pos;
                cid_out[pos] = (int)id;
            } else {
                atomicOr(a.err, ERR_OVERFLOW);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base_s += tt;
        __syncthreads();
    }
    }
}

// Stored-cell count from the range totals.
template <typename T>
__global__ void k_sp_total(const Dev<T> a, const int* __restrict__ tot, int* __restrict__ ns_out,
                           const int* __restrict__ go) {
    if (go && *go == 0) return;
    const long long n = (long long)tot[0] + tot[1] + tot[2];
    *ns_out = (int)min(n, a.cap_s);
}

// Node word and table entries of stored cell n (padded index id).  With a
// flow lattice one entry per flow direction k: for a shared direction (also a
// solute velocity) the neighbour's compact index when it is not solid (else
// the cell's own index; the sweep then takes its own slot from the node
// word), for the others the folded effective base -- the neighbour's block
// base when it is fluid, else the cell's own base plus 32 (opp(k) - k), so
// that slot E[k] + 32 k is the own slot opp(k).  Without a flow lattice the
// folded entries of the solute directions (active: not solid).
template <typename T, class LF, class LG>
__device__ __forceinline__ void sp_cell_tables(const Dev<T>& a, uint32_t n, long long id) {
    constexpr int NT = tab_entries<LF, LG>();
    a.nwc[n] = a.nw[id];
    const Nbr d = nbr_of(a.geo, id);
    if constexpr (LF::Q > 0) {
        const uint32_t own = pbase<LF>(n);
#pragma unroll
        for (int k = 1; k < LF::Q; ++k) {
            const long long nb = id + off<LF>(d, k);
            const uint32_t cls = a.nw[nb] & 3u;
            const int cm = a.cmap[nb];
            // an active neighbour is always stored; should one not be, the
            // entry points at the cell itself and the run reports an error
            if (cls != CLS_SOLID && cm < 0) atomicOr(a.err, ERR_OVERFLOW);
            uint32_t v;
            if (shared_dir<LF, LG>(k)) v = cls != CLS_SOLID && cm >= 0 ? (uint32_t)cm : n;
            else v = cls == CLS_FLUID && cm >= 0 ? pbase<LF>((uint32_t)cm) : own + 32u * (uint32_t)(LF::opp(k) - k);
            a.etab[etab_at(n, NT, k - 1)] = v;
        }
    } else {
        const uint32_t own = pbase<LG>(n);
#pragma unroll
        for (int k = 1; k < LG::Q; ++k) {
            const long long nb = id + off<LG>(d, k);
            const int cm = a.cmap[nb];
            const bool act = (a.nw[nb] & 3u) != CLS_SOLID;
            if (act && cm < 0) atomicOr(a.err, ERR_OVERFLOW);
            a.etab[etab_at(n, NT, k - 1)] =
                act && cm >= 0 ? pbase<LG>((uint32_t)cm) : own + 32u * (uint32_t)(LG::opp(k) - k);
        }
    }
}

template <typename T, class LF, class LG>
__global__ void k_sp_tables(const Dev<T> a, const int* __restrict__ go) {
    if (go && *go == 0) return;
    const int ns = *a.ns;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < ns; n += (long long)gridDim.x * blockDim.x)
        sp_cell_tables<T, LF, LG>(a, (uint32_t)n, a.cid[n]);
}

// After the classes changed: the table entries of every stored cell within
// one flow-lattice step of the event region (the cells whose neighbours may
// have changed activity).  A cell reached from several items is recomputed
// from the same classes each time.
template <typename T, class LF, class LG>
__global__ void k_sp_retab(const Dev<T> a) {
    using LS = typename Stencil<LF, LG>::L;
    const int n = min(*a.nev, a.cap_e);
    const Geo& g = a.geo;
    const long long items = (long long)n * LG::Q * LS::Q;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < items;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / (LG::Q * LS::Q));
        const int r = (int)(t % (LG::Q * LS::Q));
        const int o = r / LS::Q, sdx = r % LS::Q;
        int x, y, z;
        coords(g, a.ev_node[e], x, y, z);
        x += LG::cx(o) + LS::cx(sdx);
        y += LG::cy(o) + LS::cy(sdx);
        z += LG::cz(o) + LS::cz(sdx);
        if (!wrap_inside(g, x, y, z)) continue;
        const long long c = g.idx(x, y, z);
        const int cn = a.cmap[c];
        if (cn >= 0) sp_cell_tables<T, LF, LG>(a, (uint32_t)cn, c);
    }
}

// Event region of a step: the event cells and their neighbours along the
// solute lattice.  A cell's owner is the smallest (event, direction) item
// that reaches it.
template <typename T, class LG>
__global__ void k_sp_rmark(const Dev<T> a) {
    const int n = min(*a.nev, a.cap_e);
    const Geo& g = a.geo;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * LG::Q;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / LG::Q), o = (int)(t % LG::Q);
        int x, y, z;
        coords(g, a.ev_node[e], x, y, z);
        x += LG::cx(o);
        y += LG::cy(o);
        z += LG::cz(o);
        if (!wrap_inside(g, x, y, z)) continue;
        atomicMin(&a.rown[g.idx(x, y, z)], (int)t);
    }
}

// Swap the two slots of every link with an end in the event region whose
// two ends are both active for the lattice under the classes in the node
// words: after an odd step this turns the region into the even-step form
// (each cell's f*_i in its own slot opp(i)), and back after the classes
// change.  Each link is handled once: by its end in the region, or by the
// end whose direction lies in the first half when both are.
template <typename T, class L, bool FLOW>
__device__ __forceinline__ void swap_links(const Dev<T>& a, T* A, long long c, const Nbr& d) {
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const long long nb = c + off<L>(d, i);
        if (i > L::H && a.rown[nb] != RNONE) continue;
        const uint32_t cc = a.nw[c] & 3u, cn = a.nw[nb] & 3u;
        const bool act = FLOW ? (cc == CLS_FLUID && cn == CLS_FLUID) : (cc != CLS_SOLID && cn != CLS_SOLID);
        if (!act) continue;
        const long long s1 = pslot64<L>(i, a.cmap[nb]), s2 = pslot64<L>(L::opp(i), a.cmap[c]);
        const T v = A[s1];
        A[s1] = A[s2];
        A[s2] = v;
    }
}

template <typename T, class LF, class LG>
__global__ void k_sp_swap(const Dev<T> a) {
    const int n = min(*a.nev, a.cap_e);
    const Geo& g = a.geo;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * LG::Q;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / LG::Q), o = (int)(t % LG::Q);
        int x, y, z;
        coords(g, a.ev_node[e], x, y, z);
        x += LG::cx(o);
        y += LG::cy(o);
        z += LG::cz(o);
        if (!wrap_inside(g, x, y, z)) continue;
        const long long c = g.idx(x, y, z);
        if (a.rown[c] != (int)t) continue;
        const Nbr d = nbr_deltas(g, x, y, z);
        if constexpr (LF::Q > 0) swap_links<T, LF, true>(a, a.F, c, d);
        swap_links<T, LG, false>(a, a.G, c, d);
    }
}

template <typename T, class LG>
__global__ void k_sp_rreset(const Dev<T> a) {
    const int n = min(*a.nev, a.cap_e);
    const Geo& g = a.geo;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * LG::Q;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / LG::Q), o = (int)(t % LG::Q);
        int x, y, z;
        coords(g, a.ev_node[e], x, y, z);
        x += LG::cx(o);
        y += LG::cy(o);
        z += LG::cz(o);
        if (!wrap_inside(g, x, y, z)) continue;
        a.rown[g.idx(x, y, z)] = RNONE;
    }
}

// Repacking (when a cell outside the stored set must be stored): the new
// numbering is written to cmap2 / cid2 / ns2 by the k_sp_* kernels above,
// then the populations move cell by cell into F2 / G2 (new cells start with
// C = 0 and flow at rest) and everything is copied back.  Every kernel
// returns at once unless a repacking is pending.
template <typename T, class LF, class LG>
__global__ void k_sp_gather(const Dev<T> a, const Phys p) {
    if (*a.repack == 0) return;
    constexpr int QF = LF::Q, QG = LG::Q;
    const int ns2 = *a.ns2;
    for (long long n2 = blockIdx.x * (long long)blockDim.x + threadIdx.x; n2 < ns2;
         n2 += (long long)gridDim.x * blockDim.x) {
        const int n = a.cmap[a.cid2[n2]];
        if constexpr (QF > 0) {
#pragma unroll
            for (int i = 0; i < QF; ++i) a.F2[pslot64<LF>(i, n2)] = n >= 0 ? a.F[pslot64<LF>(i, n)] : T(0);
        }
#pragma unroll
        for (int i = 0; i < QG; ++i)
            a.G2[pslot64<LG>(i, n2)] = n >= 0 ? a.G[pslot64<LG>(i, n)] : T(-gweight<LG>(p, i) * p.cref);
    }
}

template <typename T, class LF, class LG>
__global__ void k_sp_commit(const Dev<T> a) {
    if (*a.repack == 0) return;
    constexpr int QF = LF::Q, QG = LG::Q;
    const int ns2 = *a.ns2;
    const long long NP = a.geo.NP;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long k = t0; k < (long long)QF * ns2; k += stride) {
        const long long n = k % ns2, i = k / ns2;
        a.F[pslot64<LF>((int)i, n)] = a.F2[pslot64<LF>((int)i, n)];
    }
    for (long long k = t0; k < (long long)QG * ns2; k += stride) {
        const long long n = k % ns2, i = k / ns2;
        a.G[pslot64<LG>((int)i, n)] = a.G2[pslot64<LG>((int)i, n)];
    }
    for (long long k = t0; k < ns2; k += stride) a.cid[k] = a.cid2[k];
    for (long long k = t0; k < NP; k += stride) a.cmap[k] = a.cmap2[k];
}

template <typename T>
__global__ void k_sp_commit_end(const Dev<T> a) {
    if (*a.repack == 0) return;
    *a.ns = *a.ns2;
}

template <typename T>
__global__ void k_sp_repack_done(const Dev<T> a) {
    if (*a.repack == 0) return;
    *a.repack = 0;
    *a.nrepack += 1;
}

// Compact indices of the boundary entries after a repacking (the local list
// maintenance keeps the entries and their order).
template <typename T>
__global__ void k_sp_recn(const Dev<T> a) {
    if (*a.repack == 0) return;
    const int n = *a.nb;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        if (!(a.b_word[e] & BW_DEAD)) a.b_cn[e] = a.cmap[a.b_idx[e]];
}

// -1 everywhere (cmap2 before a repacking), when one is pending.
template <typename T>
__global__ void k_sp_clear2(const Dev<T> a) {
    if (*a.repack == 0) return;
    const long long NP = a.geo.NP;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < NP; k += (long long)gridDim.x * blockDim.x)
        a.cmap2[k] = -1;
}

template <typename T>
__global__ void k_ev_reset(const Dev<T> a) {
    const int n = min(*a.nev, a.cap_e);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) a.evidx[a.ev_node[e]] = -1;
}

// Condition of the graph node that holds the step's phase-change path (and
// the step counter); a step without events is counted here.
template <typename T>
__global__ void k_ev_gate(const Dev<T> a, cudaGraphConditionalHandle h) {
    const bool any = *a.nev > 0;
    cudaGraphSetConditional(h, any ? 1u : 0u);
    if (!any) *a.step += 1;
}

template <typename T>
__global__ void k_step_end(const Dev<T> a) {
    *a.nev = 0;
    *a.step += 1;
    if (a.lcnt) {
        if (a.lcnt[LC_FULL]) a.lcnt[LC_DEADB] = a.lcnt[LC_DEADF] = 0;
        a.lcnt[LC_FULL] = a.lcnt[LC_LOCAL] = 0;
    }
}

