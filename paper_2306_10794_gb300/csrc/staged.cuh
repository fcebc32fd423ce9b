// Staged fluid sweep: persistent CTAs walk row tiles of TILE_X cells along x
// (one thread per cell).  The lanes of warp 0 stage a tile's population rows
// and node words into shared memory with bulk asynchronous copies
// (cp.async.bulk, one row per lane, completion on an mbarrier), STAGES tiles
// ahead of the compute; no thread holds loads in flight in registers, so the
// bytes in flight per SM are set by the shared-memory stages, not by the
// register-limited occupancy of a one-cell-per-thread sweep.  On GB300 the
// cell update is issue-bound rather than latency-bound, and the five
// resident CTAs per SM this allows (20 warps) issue more slowly than the
// dense sweep's 32 warps: the dense sweep is the default, this one is
// selected with LBRBC_FLUID_SWEEP=staged.
//
// What is staged is the slot every cell reads unless one of its sources is
// inactive: its own slots (even steps, the row of the cell itself) or the
// source-side slots (odd steps: for direction i the row of population
// opp(i) at (y - e_iy, z - e_iz), with a halo of 4 cells on each side for
// the x shift).  Swapped reads of inactive sources, and the two cells of a
// periodic x row that wrap, read HBM directly (GlobalSrc).  Writes go from
// registers to HBM as in the dense sweep.  Each slot is read and written by
// one cell per step (AA pattern), so prefetching tile k+1 while tile k
// writes is race-free; halo elements belong to other cells and are never
// used.
#pragma once

namespace lbrbc {

constexpr int TILE_X = 128;            // cells per tile = threads per CTA
constexpr int TILE_W = TILE_X + 8;     // staged row width: x0 - 4 .. x0 + TILE_X + 4
constexpr unsigned long long STAGE_WAIT_NS = 2000000000ull;  // bound of one mbarrier wait

template <typename T>
constexpr int staged_stages() {
    return sizeof(T) == 4 ? 3 : 2;
}

template <typename T, class LF, class LG>
constexpr size_t staged_stage_bytes() {
    // population rows of both lattices, then the node words of the tile
    return (size_t)(LF::Q + LG::Q) * TILE_W * sizeof(T) + (size_t)TILE_W * sizeof(uint32_t);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16), completing `bytes` transactions on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// y / z part of the offset to the neighbour in direction j (periodic wrap
// included; the x shift is taken from the staged halo).
template <class L>
__device__ __forceinline__ int yz_off32(const Nbr32& d, int j) {
    return (L::cy(j) > 0 ? d.yp : (L::cy(j) < 0 ? d.ym : 0)) + (L::cz(j) > 0 ? d.zp : (L::cz(j) < 0 ? d.zm : 0));
}

template <typename T, class LF, class LG, bool ODD>
struct StagedSrc {
    GlobalSrc<T, LF, LG, ODD> gl;
    const T* sF;  // staged rows of the flow lattice, TILE_W apart
    const T* sG;  // staged rows of the solute lattice
    int lx;       // the cell's column in the staged rows
    bool wrap;    // periodic x row end: every read from HBM
    __device__ __forceinline__ bool general() const { return wrap; }
    __device__ __forceinline__ T f(int i, bool inactive) const {
        if (inactive || wrap) return gl.f(i, inactive);
        return sF[i * TILE_W + lx - (ODD ? LF::cx(i) : 0)];
    }
    __device__ __forceinline__ T g(int i, bool inactive) const {
        if (inactive || wrap) return gl.g(i, inactive);
        return sG[i * TILE_W + lx - (ODD ? LG::cx(i) : 0)];
    }
};

// Tile t -> (x0, y, z), tiles ordered x-tile fastest, then y, then z.
__device__ __forceinline__ void tile_coords(const Geo& g, int t, int& x0, int& y, int& z) {
    const int ntx = (g.nx + TILE_X - 1) / TILE_X;
    const int r = t / ntx;
    x0 = (t - r * ntx) * TILE_X;
    y = r % g.ny;
    z = r / g.ny;
}

// Row r of a stage: population rows of the flow lattice (r < QF), of the
// solute lattice (QF <= r < QF + QG), then the node words (r = QF + QG).
struct RowInfo {
    int lat;       // 0 flow, 1 solute, 2 node words
    int pop;       // population whose slots the row holds
    int cy, cz;    // odd steps: the row sits at (y + cy, z + cz)
};

template <class LF, class LG, bool ODD>
__device__ __forceinline__ void fill_rows(RowInfo* ri) {
    constexpr int QF = LF::Q, QG = LG::Q;
#pragma unroll
    for (int i = 0; i < QF; ++i) {
        const int j = LF::opp(i);
        ri[i] = RowInfo{0, ODD ? j : i, ODD ? LF::cy(j) : 0, ODD ? LF::cz(j) : 0};
    }
#pragma unroll
    for (int i = 0; i < QG; ++i) {
        const int j = LG::opp(i);
        ri[QF + i] = RowInfo{1, ODD ? j : i, ODD ? LG::cy(j) : 0, ODD ? LG::cz(j) : 0};
    }
    ri[QF + QG] = RowInfo{2, 0, 0, 0};
}

// First copied element of row r of the tile at `base` (population rows of
// odd steps start 4 cells before x0).
template <typename T, bool ODD>
__device__ __forceinline__ const void* row_src(const Dev<T>& a, const RowInfo& r, uint32_t base, const Nbr32& d) {
    if (r.lat == 2) return a.nw + base;
    const T* L = r.lat == 0 ? a.F : a.G;
    if (!ODD) return L + (size_t)r.pop * a.geo.NP + base;
    const int yz = (r.cy > 0 ? d.yp : (r.cy < 0 ? d.ym : 0)) + (r.cz > 0 ? d.zp : (r.cz < 0 ? d.zm : 0));
    return L + (size_t)r.pop * a.geo.NP + base + yz - 4;
}

template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(TILE_X) k_fluid_staged(const Dev<T> a, const Phys p, const PhysT<T> q) {
    constexpr int QF = LF::Q, QG = LG::Q, NR = QF + QG;
    constexpr int S = staged_stages<T>();
    constexpr size_t SB = staged_stage_bytes<T, LF, LG>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ int stile[S];
    __shared__ RowInfo rows[NR + 1];
    const Geo& g = a.geo;
    const int ntiles = a.ntiles;
    const uint32_t NP = (uint32_t)g.NP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int next = blockIdx.x;  // tile cursor (lane 0 of warp 0)

    auto next_tile = [&]() {
        while (next < ntiles && !a.tile_on[next]) next += gridDim.x;
        const int t = next < ntiles ? next : -1;
        if (t >= 0) next += gridDim.x;
        return t;
    };
    auto geometry = [&](int t, uint32_t& base, Nbr32& d, uint32_t& row, uint32_t& nwb) {
        int x0, y, z;
        tile_coords(g, t, x0, y, z);
        const int n = min(TILE_X, g.nx - x0);
        base = (uint32_t)g.idx(x0, y, z);
        d = nbr32(g, x0, y, z);
        row = (uint32_t)(((ODD ? n + 8 : n) + 3) & ~3) * (uint32_t)sizeof(T);
        nwb = (uint32_t)((n + 3) & ~3) * 4u;
    };
    // warp 0: stage the next tile of this CTA into stage s
    auto issue = [&](int s) {
        if (warp != 0) return;
        unsigned char* st = smem_raw + (size_t)s * SB;
        int t = 0;
        if (lane == 0) t = next_tile();
        t = __shfl_sync(0xffffffffu, t, 0);
        if (lane == 0) stile[s] = t;
        if (t < 0) return;
        uint32_t base, row, nwb;
        Nbr32 d;
        geometry(t, base, d, row, nwb);
        if (lane == 0) mbar_expect_tx(&full[s], (uint32_t)NR * row + nwb);
        __syncwarp();
        for (int r = lane; r <= NR; r += 32)
            bulk_g2s(st + (size_t)r * TILE_W * sizeof(T), row_src<T, ODD>(a, rows[r], base, d), r == NR ? nwb : row,
                     &full[s]);
    };

    if (threadIdx.x == 0) {
        fill_rows<LF, LG, ODD>(rows);
#pragma unroll
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    for (int s = 0; s < S; ++s) issue(s);
    __syncthreads();

    for (int k = 0;; ++k) {
        const int s = k % S;
        const int t = stile[s];
        if (t < 0) break;
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k / S) & 1), STAGE_WAIT_NS);
        if (ok) {
            int x0, y, z;
            tile_coords(g, t, x0, y, z);
            const int x = x0 + (int)threadIdx.x;
            const T* sr = reinterpret_cast<const T*>(smem_raw + (size_t)s * SB);
            if (x < g.nx) {
                const uint32_t w = reinterpret_cast<const uint32_t*>(sr + NR * TILE_W)[threadIdx.x];
                if ((w & 3u) == CLS_FLUID) {
                    const uint32_t id = (uint32_t)g.idx(x, y, z);
                    const Nbr32 d = nbr32(g, x, y, z);
                    const StagedSrc<T, LF, LG, ODD> src{{a.F, a.G, id, NP, d},
                                                        sr,
                                                        sr + QF * TILE_W,
                                                        (int)threadIdx.x + (ODD ? 4 : 0),
                                                        g.per_x && (x == 0 || x == g.nx - 1)};
                    fluid_cell_src<T, LF, LG, ODD>(a, p, q, x, y, z, id, w, d, src);
                }
            }
        }
        // every thread is done with stage s (and agrees whether a wait failed)
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(a.err, ERR_TIMEOUT);
                // let the copies still in flight land before the CTA exits
                for (int j = 0; j < S; ++j) {
                    const int kk = k + j, ss = kk % S;
                    if (stile[ss] >= 0) mbar_wait_bounded(&full[ss], (uint32_t)((kk / S) & 1), STAGE_WAIT_NS);
                }
            }
            return;
        }
        issue(s);
    }
}

// Tile flags of the staged sweep: a tile is active when one of its cells is
// fluid (one warp per tile; after reclassification only when events
// happened).
template <typename T>
__global__ void k_tile_flags(const Dev<T> a, int force) {
    if (!force && *a.nev == 0) return;
    const Geo& g = a.geo;
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int t = warp; t < a.ntiles; t += nwarps) {
        int x0, y, z;
        tile_coords(g, t, x0, y, z);
        bool any = false;
        for (int j = lane; j < TILE_X; j += 32) {
            const int x = x0 + j;
            if (x < g.nx) any |= (a.nw[g.idx(x, y, z)] & 3u) == CLS_FLUID;
        }
        any = __any_sync(0xffffffffu, any);
        if (lane == 0) a.tile_on[t] = any ? 1 : 0;
    }
}

}  // namespace lbrbc
