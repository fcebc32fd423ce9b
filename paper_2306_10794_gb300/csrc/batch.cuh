// Batched time stepping of many independent domains (uneven sizes, own
// parameters) with one launch per kernel phase for the whole batch: the
// fluid sweep, the wet-boundary list and the fluid-end gather each run as a
// persistent kernel over a precomputed schedule of work items drawn from
// every domain, and a pair of steps is replayed from one CUDA graph.  An
// autotuner times candidate schedules (tile shape along x, tile order, grid
// size) on the batch itself and keeps the fastest.
#pragma once

#include <algorithm>
#include <memory>
#include <numeric>
#include <vector>

#include "engine.cuh"

namespace lbrbc {

// Resident blocks per SM the batched active-cell sweep is compiled for
// (FP32, even and odd steps): the register cap that lets them reside.  The
// domain's parameters live in registers here (in the single-domain sweep
// they are constant-bank operands): uncapped the even step takes 136
// registers (3 blocks); capped at 80 it spills 188 B to L1 but measured
// fastest over 256 domains (2.80 ms per step against 3.26 uncapped).
#ifndef LBRBC_KB_SP_BLOCKS_EVEN
#define LBRBC_KB_SP_BLOCKS_EVEN 6
#endif
#ifndef LBRBC_KB_SP_BLOCKS_ODD
#define LBRBC_KB_SP_BLOCKS_ODD 6
#endif

template <typename T>
struct DomainDesc {
    Dev<T> a;
    Phys p;
    PhysT<T> q;
};

// Fluid tile: 128 threads over tw cells along x times 128/tw rows along y at
// one z.  x: domain, y: x0 | (log2(tw) << 24), z: y0, w: z.
template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(FLUID_BLOCK) kb_fluid(const DomainDesc<T>* __restrict__ dd, const int4* __restrict__ tiles,
                                                     int ntiles) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const DomainDesc<T>& D = dd[tl.x];
        const int lw = tl.y >> 24;
        const int tw = 1 << lw;
        const int x = (tl.y & 0xffffff) + (threadIdx.x & (tw - 1));
        const int y = tl.z + (threadIdx.x >> lw);
        if (x < D.a.geo.nx && y < D.a.geo.ny) fluid_cell<T, LF, LG, ODD>(D.a, D.p, D.q, x, y, tl.w);
    }
}

// Fluid-list chunk: FLUID_BLOCK consecutive entries of one domain's
// compacted fluid-cell list.
template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(FLUID_BLOCK) kb_fluid_list4(const DomainDesc<T>* __restrict__ dd,
                                                           const int4* __restrict__ chunks, int nchunks) {
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int4 ch = chunks[c];
        const DomainDesc<T>& D = dd[ch.x];
        const int e = ch.y * FLUID_BLOCK + threadIdx.x;
        if (e < *D.a.nfl) {
            int x, y, z;
            unpack32(D.a.fl_xyz[e], x, y, z);
            fluid_cell<T, LF, LG, ODD>(D.a, D.p, D.q, x, y, z);
        }
    }
}

// Active-cell chunk: FLUID_BLOCK consecutive stored cells of one domain on
// the active-cell layout.  x: domain, y: chunk.
template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(FLUID_BLOCK, sizeof(T) == 4 ? (ODD ? LBRBC_KB_SP_BLOCKS_ODD : LBRBC_KB_SP_BLOCKS_EVEN) : 4) kb_fluid_sp(const DomainDesc<T>* __restrict__ dd,
                                                        const int2* __restrict__ chunks, int nchunks) {
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int2 ch = chunks[c];
        const DomainDesc<T>& D = dd[ch.x];
        const int n = ch.y * FLUID_BLOCK + threadIdx.x;
        if (n < *D.a.ns) sparse_cell<T, LF, LG, ODD>(D.a, D.p, D.q, n);
    }
}

// Boundary chunk: LIST_BLOCK consecutive list entries of one domain; the
// chunk's ledger partial goes to the domain's slot for that chunk.
template <typename T, class LF, class LG, bool ODD>
__global__ void __launch_bounds__(LIST_BLOCK) kb_bound(const DomainDesc<T>* __restrict__ dd, const int2* __restrict__ chunks,
                                                    int nchunks) {
    __shared__ __align__(16) unsigned char red_raw[2 * (LIST_BLOCK / 32) * sizeof(DiffSum<T>)];
    DiffSum<T>* red = reinterpret_cast<DiffSum<T>*>(red_raw);
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int2 ch = chunks[c];
        const DomainDesc<T>& D = dd[ch.x];
        const int e = ch.y * LIST_BLOCK + threadIdx.x;
        DiffSum<T> racc, dacc;
        if (e < *D.a.nb) {
            if (D.a.sparse) bound_entry<T, LF, LG, ODD, true>(D.a, D.p, D.q, e, racc, dacc);
            else bound_entry<T, LF, LG, ODD, false>(D.a, D.p, D.q, e, racc, dacc);
        }
        racc = warp_merge(racc);
        dacc = warp_merge(dacc);
        __syncthreads();
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
                D.a.bacc[2 * ch.y] += r.value();
                D.a.bacc[2 * ch.y + 1] += d.value();
            }
        }
    }
}

template <typename T, class LG>
__global__ void __launch_bounds__(LIST_BLOCK) kb_fend(const DomainDesc<T>* __restrict__ dd, const int2* __restrict__ chunks,
                                                   int nchunks) {
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int2 ch = chunks[c];
        const DomainDesc<T>& D = dd[ch.x];
        const int e = ch.y * LIST_BLOCK + threadIdx.x;
        if (e < *D.a.nf) fend_entry<T, LG>(D.a, D.p, e);
    }
}

#define LB_BCUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
            return 2;                                                                     \
        }                                                                                 \
    } while (0)

template <typename T, class LF, class LG>
class BatchEngine final : public IBatch {
   public:
    ~BatchEngine() override { release(); }

    int init(int n, const lbrbc_params* P, const uint8_t* const* masks, const lbrbc_init* inits,
             std::string& err) override {
        (void)cudaGetLastError();
        for (int i = 0; i < n; ++i) {
            if (P[i].phase_change) {
                err = "batched domains do not support phase change (domain " + std::to_string(i) + ")";
                return 1;
            }
            auto* e = new Engine<T, LF, LG>();
            e->set_batched();
            e->force_list(true);
            doms_.emplace_back(e);
            const int rc = e->init(P[i], masks[i], inits ? &inits[i] : nullptr, err);
            if (rc) {
                err = "domain " + std::to_string(i) + ": " + err;
                return rc;
            }
            if ((e->host_nb() + LIST_BLOCK - 1) / LIST_BLOCK > e->nbacc()) {
                err = "domain " + std::to_string(i) + " has too many boundary cells for batching";
                return 1;
            }
        }
        std::vector<DomainDesc<T>> h(n);
        for (int i = 0; i < n; ++i) {
            h[i].a = doms_[i]->dev();
            h[i].p = doms_[i]->phys();
            h[i].q = doms_[i]->physt();
        }
        LB_BCUDA(cudaMalloc((void**)&dd_, sizeof(DomainDesc<T>) * n));
        LB_BCUDA(cudaMemcpy(dd_, h.data(), sizeof(DomainDesc<T>) * n, cudaMemcpyHostToDevice));
        // list chunks (fixed: no phase change)
        std::vector<int2> bch, fch;
        for (int i = 0; i < n; ++i) {
            for (int c = 0; c * LIST_BLOCK < doms_[i]->host_nb(); ++c) bch.push_back(make_int2(i, c));
            for (int c = 0; c * LIST_BLOCK < doms_[i]->host_nf(); ++c) fch.push_back(make_int2(i, c));
        }
        nbch_ = (int)bch.size();
        nfch_ = (int)fch.size();
        // fluid chunks of the domains on the active-cell layout (fixed: no
        // phase change, the stored set never changes)
        {
            std::vector<std::vector<int2>> per(n);
            for (int i = 0; i < n; ++i)
                if (doms_[i]->sparse())  // the fluid cells are the first range of the stored set
                    for (long long c = 0; c * FLUID_BLOCK < doms_[i]->fluid_cells(); ++c)
                        per[i].push_back(make_int2(i, (int)c));
            std::vector<int2> sch;
            // largest domains first, chunks interleaved round-robin
            std::vector<int> idx(n);
            std::iota(idx.begin(), idx.end(), 0);
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return per[a].size() > per[b].size(); });
            for (size_t k = 0, more = 1; more; ++k) {
                more = 0;
                for (int i : idx)
                    if (k < per[i].size()) {
                        sch.push_back(per[i][k]);
                        more = 1;
                    }
            }
            nsch_ = (int)sch.size();
            LB_BCUDA(cudaMalloc((void**)&sch_, sizeof(int2) * std::max(1, nsch_)));
            if (nsch_) LB_BCUDA(cudaMemcpy(sch_, sch.data(), sizeof(int2) * nsch_, cudaMemcpyHostToDevice));
        }
        LB_BCUDA(cudaMalloc((void**)&bch_, sizeof(int2) * std::max(1, nbch_)));
        LB_BCUDA(cudaMalloc((void**)&fch_, sizeof(int2) * std::max(1, nfch_)));
        if (nbch_) LB_BCUDA(cudaMemcpy(bch_, bch.data(), sizeof(int2) * nbch_, cudaMemcpyHostToDevice));
        if (nfch_) LB_BCUDA(cudaMemcpy(fch_, fch.data(), sizeof(int2) * nfch_, cudaMemcpyHostToDevice));
        LB_BCUDA(cudaStreamCreateWithFlags(&own_, cudaStreamNonBlocking));
        {
            int lo = 0, hi = 0;
            LB_BCUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            LB_BCUDA(cudaStreamCreateWithPriority(&aux_, cudaStreamNonBlocking, hi));
        }
        LB_BCUDA(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming));
        LB_BCUDA(cudaEventCreateWithFlags(&join_, cudaEventDisableTiming));
        // default schedule until autotuned: fluid-list chunks, largest domains
        // first, 8 blocks per SM
        if (set_schedule(3, 1, 8, err)) return 2;
        return 0;
    }

    int step(int64_t n, cudaStream_t s, std::string& err) override {
        cudaStream_t st = s ? s : own_;
        int64_t k = 0;
        while (k < n) {
            if (multi_ && lastodd_ && n - k >= MSTEP) {
                LB_BCUDA(cudaGraphLaunch(g_multi_, st));  // MSTEP (even) steps, parity kept
                k += MSTEP;
            } else if (!lastodd_ || n - k < 2) {
                LB_BCUDA(cudaGraphLaunch(lastodd_ ? g_even_ : g_odd_, st));
                lastodd_ ^= 1;
                k += 1;
            } else {
                LB_BCUDA(cudaGraphLaunch(g_pair_, st));
                k += 2;
            }
        }
        for (auto& d : doms_) d->advance(n, lastodd_, st);
        if (!s) LB_BCUDA(cudaStreamSynchronize(own_));
        return 0;
    }

    // Time each candidate schedule for `pairs` step pairs (real steps of every
    // domain) and keep the fastest.  choice: [tile policy, order, blocks/SM].
    int autotune(int pairs, cudaStream_t s, int64_t* choice, double* best_ms, std::string& err) override {
        cudaStream_t st = s ? s : own_;
        const int policies[] = {0, 1, 2, 3, 4}, orders[] = {0, 1}, per_sm[] = {4, 8, 16};
        double best = 1e30;
        int bp = 0, bo = 1, bs = 8;
        cudaEvent_t e0, e1;
        LB_BCUDA(cudaEventCreate(&e0));
        LB_BCUDA(cudaEventCreate(&e1));
        for (int pol : policies)
            for (int ord : orders)
                for (int ps : per_sm) {
                    if (pol == 4 && ord != 0) continue;  // order does not apply; ps = branches / 4
                    if (set_schedule(pol, ord, ps, err)) return 2;
                    if (step(2, st, err)) return 2;  // warm-up pair
                    LB_BCUDA(cudaEventRecord(e0, st));
                    if (step(2 * (int64_t)pairs, st, err)) return 2;
                    LB_BCUDA(cudaEventRecord(e1, st));
                    LB_BCUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    LB_BCUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best) {
                        best = ms;
                        bp = pol;
                        bo = ord;
                        bs = ps;
                    }
                }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (set_schedule(bp, bo, bs, err)) return 2;
        if (choice) {
            choice[0] = bp;
            choice[1] = bo;
            choice[2] = bs;
        }
        if (best_ms) *best_ms = best / (2.0 * pairs);
        return 0;
    }

    int schedule(int policy, int order, int per_sm, std::string& err) override {
        return set_schedule(policy, order, per_sm, err);
    }

    int size() const override { return (int)doms_.size(); }
    ISim* domain(int i) override { return doms_[i].get(); }
    long long fluid_cells() const override {
        long long s = 0;
        for (auto& d : doms_) s += d->fluid_cells();
        return s;
    }

   private:
    // Tile policy 0: width min(128, pow2 >= nx); 1: 64; 2: 32; 3: chunks of
    // each domain's compacted fluid-cell list instead of dense tiles; 4: no
    // persistent kernels, the domains' own kernels side by side in one graph.  Order
    // 0: domain by domain; 1: largest domains first with the work items of
    // all domains interleaved round-robin.
    int set_schedule(int policy, int order, int per_sm, std::string& err) {
        policy_ = policy;
        std::vector<std::vector<int4>> per(doms_.size());
        for (size_t i = 0; i < doms_.size() && policy == 3; ++i)
            if (!doms_[i]->sparse())
                for (int c = 0; c * FLUID_BLOCK < doms_[i]->host_nfl(); ++c) per[i].push_back(make_int4((int)i, c, 0, 0));
        for (size_t i = 0; i < doms_.size() && policy < 3; ++i) {
            if (doms_[i]->sparse()) continue;  // its fluid chunks are fixed (sch_)
            const Geo& g = doms_[i]->geo();
            int tw = 128;
            if (policy == 0)
                while (tw > 32 && tw / 2 >= g.nx) tw /= 2;
            else tw = policy == 1 ? 64 : 32;
            int lw = 0;
            while ((1 << lw) < tw) ++lw;
            const int rows = FLUID_BLOCK / tw;
            for (int z = 0; z < g.nz; ++z)
                for (int y0 = 0; y0 < g.ny; y0 += rows)
                    for (int x0 = 0; x0 < g.nx; x0 += tw) per[i].push_back(make_int4((int)i, x0 | (lw << 24), y0, z));
        }
        std::vector<int4> tiles;
        if (order == 0) {
            for (auto& v : per) tiles.insert(tiles.end(), v.begin(), v.end());
        } else {
            std::vector<size_t> idx(per.size());
            std::iota(idx.begin(), idx.end(), 0);
            std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return per[a].size() > per[b].size(); });
            size_t k = 0;
            bool more = true;
            while (more) {
                more = false;
                for (size_t i : idx)
                    if (k < per[i].size()) {
                        tiles.push_back(per[i][k]);
                        more = true;
                    }
                ++k;
            }
        }
        ntiles_ = (int)tiles.size();
        if (tiles_) cudaFree(tiles_);
        tiles_ = nullptr;
        LB_BCUDA(cudaMalloc((void**)&tiles_, sizeof(int4) * std::max(1, ntiles_)));
        LB_BCUDA(cudaMemcpy(tiles_, tiles.data(), sizeof(int4) * ntiles_, cudaMemcpyHostToDevice));
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        grid_ = std::max(1, nsm * per_sm);
        nbr_ = 8 * per_sm;  // schedule 4: branch streams of the domain graph (32, 64, 128)
        return build_graphs(err);
    }

    // One step of every domain.  The wet-boundary chunks and the fluid-end
    // gather run on a second stream beside the fluid phase: within each
    // domain the three touch disjoint population slots, and the gather
    // depends only on the boundary phase.
    int enqueue(cudaStream_t st, bool odd, std::string& err) {
        if (policy_ == 4) return enqueue_domains(st, odd, err);
        const int gf = std::min(grid_, std::max(1, ntiles_));
        const int gs = std::min(grid_, std::max(1, nsch_));
        const int gb = std::min(grid_, std::max(1, nbch_));
        const int ge = std::min(grid_, std::max(1, nfch_));
        LB_BCUDA(cudaEventRecord(fork_, st));
        LB_BCUDA(cudaStreamWaitEvent(aux_, fork_, 0));
        if (nbch_) {
            if (odd) kb_bound<T, LF, LG, true><<<gb, LIST_BLOCK, 0, aux_>>>(dd_, bch_, nbch_);
            else kb_bound<T, LF, LG, false><<<gb, LIST_BLOCK, 0, aux_>>>(dd_, bch_, nbch_);
        }
        if (nfch_) kb_fend<T, LG><<<ge, LIST_BLOCK, 0, aux_>>>(dd_, fch_, nfch_);
        LB_BCUDA(cudaEventRecord(join_, aux_));
        if (nsch_) {
            if (odd) kb_fluid_sp<T, LF, LG, true><<<gs, FLUID_BLOCK, 0, st>>>(dd_, sch_, nsch_);
            else kb_fluid_sp<T, LF, LG, false><<<gs, FLUID_BLOCK, 0, st>>>(dd_, sch_, nsch_);
        }
        if (ntiles_ && policy_ == 3) {
            // list chunks are stored in the tile array as {domain, chunk, 0, 0}
            if (odd) kb_fluid_list4<T, LF, LG, true><<<gf, FLUID_BLOCK, 0, st>>>(dd_, tiles_, ntiles_);
            else kb_fluid_list4<T, LF, LG, false><<<gf, FLUID_BLOCK, 0, st>>>(dd_, tiles_, ntiles_);
        } else if (ntiles_) {
            if (odd) kb_fluid<T, LF, LG, true><<<gf, FLUID_BLOCK, 0, st>>>(dd_, tiles_, ntiles_);
            else kb_fluid<T, LF, LG, false><<<gf, FLUID_BLOCK, 0, st>>>(dd_, tiles_, ntiles_);
        }
        LB_BCUDA(cudaStreamWaitEvent(st, join_, 0));
        LB_BCUDA(cudaGetLastError());
        return 0;
    }

    // Schedule 4: every domain's own step kernels (parameters in the launch's
    // constant bank, the single-domain register budget) as independent
    // branches of one graph: nbr_ branch streams, the domains dealt largest
    // first to the branch with the fewest fluid cells so far; each domain's
    // boundary list forks onto its own second stream.
    // nsteps steps of every domain, chained per domain on its branch.
    int enqueue_domains(cudaStream_t st, bool odd, std::string& err, int nsteps = 1) {
        while ((int)br_.size() < nbr_) {
            cudaStream_t b;
            cudaEvent_t e;
            LB_BCUDA(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
            LB_BCUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            br_.push_back(b);
            bj_.push_back(e);
        }
        const int nb = std::min<int>(nbr_, (int)doms_.size());
        std::vector<int> idx(doms_.size()), owner(doms_.size());
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int a, int b) { return doms_[a]->fluid_cells() > doms_[b]->fluid_cells(); });
        std::vector<long long> load(nb, 0);
        for (int i : idx) {
            const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            owner[i] = j;
            load[j] += doms_[i]->fluid_cells() + 1;
        }
        LB_BCUDA(cudaEventRecord(fork_, st));
        for (int j = 0; j < nb; ++j) LB_BCUDA(cudaStreamWaitEvent(br_[j], fork_, 0));
        // several steps: each domain's next step follows its own previous
        // step on its branch, with no barrier across domains in between
        for (int i : idx)
            for (int t = 0; t < nsteps; ++t)
                if (int rc = doms_[i]->enqueue_own_step(br_[owner[i]], (t & 1) ? !odd : odd, err)) return rc;
        for (int j = 0; j < nb; ++j) {
            LB_BCUDA(cudaEventRecord(bj_[j], br_[j]));
            LB_BCUDA(cudaStreamWaitEvent(st, bj_[j], 0));
        }
        LB_BCUDA(cudaGetLastError());
        return 0;
    }

    int build_graphs(std::string& err) {
        drop_graphs();
        cudaStream_t cs;
        LB_BCUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        auto cap = [&](cudaGraphExec_t* out, int mode) -> int {
            cudaGraph_t gr;
            LB_BCUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            int r = 0;
            if (mode == 0) r = enqueue(cs, false, err);
            else if (mode == 1) r = enqueue(cs, true, err);
            else if (policy_ == 4) r = enqueue_domains(cs, false, err, mode == 2 ? 2 : MSTEP);
            else {
                r = enqueue(cs, false, err);
                if (!r) r = enqueue(cs, true, err);
            }
            cudaError_t e = cudaStreamEndCapture(cs, &gr);
            if (r) return r;
            if (e != cudaSuccess) {
                err = std::string("graph capture: ") + cudaGetErrorString(e);
                return 2;
            }
            LB_BCUDA(cudaGraphInstantiate(out, gr, 0));
            cudaGraphDestroy(gr);
            return 0;
        };
        int r = cap(&g_even_, 0) || cap(&g_odd_, 1) || cap(&g_pair_, 2);
        multi_ = false;
        if (!r && policy_ == 4) {
            r = cap(&g_multi_, 3);
            multi_ = r == 0;
        }
        cudaStreamDestroy(cs);
        if (r) return 2;
        graphs_ = true;
        return 0;
    }

    void drop_graphs() {
        if (!graphs_) return;
        cudaGraphExecDestroy(g_even_);
        cudaGraphExecDestroy(g_odd_);
        cudaGraphExecDestroy(g_pair_);
        if (multi_) cudaGraphExecDestroy(g_multi_);
        multi_ = false;
        graphs_ = false;
    }

    void release() {
        if (own_) cudaStreamSynchronize(own_);
        drop_graphs();
        for (auto b : br_) cudaStreamDestroy(b);
        for (auto e : bj_) cudaEventDestroy(e);
        br_.clear();
        bj_.clear();
        if (dd_) cudaFree(dd_);
        if (tiles_) cudaFree(tiles_);
        if (bch_) cudaFree(bch_);
        if (fch_) cudaFree(fch_);
        if (sch_) cudaFree(sch_);
        sch_ = nullptr;
        dd_ = nullptr;
        tiles_ = nullptr;
        bch_ = fch_ = nullptr;
        doms_.clear();
        if (own_) cudaStreamDestroy(own_);
        own_ = nullptr;
        if (aux_) cudaStreamDestroy(aux_);
        aux_ = nullptr;
        if (fork_) cudaEventDestroy(fork_);
        if (join_) cudaEventDestroy(join_);
        fork_ = join_ = nullptr;
    }

    std::vector<std::unique_ptr<Engine<T, LF, LG>>> doms_;
    DomainDesc<T>* dd_ = nullptr;
    int4* tiles_ = nullptr;
    int2 *bch_ = nullptr, *fch_ = nullptr, *sch_ = nullptr;
    int ntiles_ = 0, nbch_ = 0, nfch_ = 0, nsch_ = 0, grid_ = 0, policy_ = 0;
    int lastodd_ = 1;
    cudaStream_t own_ = nullptr, aux_ = nullptr;
    cudaEvent_t fork_ = nullptr, join_ = nullptr;
    int nbr_ = 32;
    std::vector<cudaStream_t> br_;  // branch streams of the domain-graph schedule
    std::vector<cudaEvent_t> bj_;
    cudaGraphExec_t g_even_{}, g_odd_{}, g_pair_{};
    // schedule 4: MSTEP steps per graph launch (fewer joins across domains)
    static constexpr int MSTEP = 8;
    cudaGraphExec_t g_multi_{};
    bool multi_ = false;
    bool graphs_ = false;
};

#undef LB_BCUDA

}  // namespace lbrbc
