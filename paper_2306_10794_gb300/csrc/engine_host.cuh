// Host side of the device engine (engine.cuh holds the kernels): creation,
// list sizing, graphs of the step, fields, ledger, events, the adjoint
// driver and the measurement helper.
#pragma once

#include <algorithm>
#include <thread>
#include <vector>

namespace lbrbc {

// Creation-time fills on the device (the padded per-cell arrays would
// otherwise be built and copied from the host, ~3 GB at 512^3).
static __global__ void k_fill_u32(uint32_t* __restrict__ a, long long n, uint32_t v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

// Scatter of a caller-layout (x-fastest, nx * ny * nz) FP64 field into the
// padded grid; src null: v_reactive on reactive cells, 0 elsewhere.
static __global__ void k_scatter_cells(double* __restrict__ dst, const double* __restrict__ src, const uint8_t* __restrict__ kind,
                                Geo g, double v_reactive) {
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx), y = (int)((t / g.nx) % g.ny), z = (int)(t / ((long long)g.nx * g.ny));
        const long long id = g.idx(x, y, z);
        dst[id] = src ? src[t] : (kind[id] == KIND_REACTIVE ? v_reactive : 0.0);
    }
}

// Initial concentration in the caller layout: c_dirichlet on Dirichlet
// cells, c_init elsewhere.
static __global__ void k_c0_cells(double* __restrict__ c0, const uint8_t* __restrict__ kind, Geo g, double c_init, double c_dir) {
    const long long total = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.nx), y = (int)((t / g.nx) % g.ny), z = (int)(t / ((long long)g.nx * g.ny));
        c0[t] = kind[g.idx(x, y, z)] == KIND_DIRICHLET ? c_dir : c_init;
    }
}

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
            q.rho_out_d = T(p.rho_out - 1.0);
            q.k_r = T(p.k_r);
            q.gamma = T(p.gamma);
            q.neg_vm = T(-p.Vm);
        }

        // kinds with ghosts, host side (z-slabs on host threads)
        const long long NP = g.NP;
        std::vector<uint8_t> kind(NP, KIND_OUTSIDE);
        std::vector<long long> nfl_z(g.nz, 0);
        par_for(g.nz, [&](int z) {
            long long c = 0;
            for (int y = 0; y < g.ny; ++y) {
                const uint8_t* row = mask + (long long)g.nx * (y + (long long)g.ny * z);
                uint8_t* dst = kind.data() + g.idx(0, y, z);
                for (int x = 0; x < g.nx; ++x) {
                    dst[x] = row[x];
                    c += row[x] == KIND_FLUID;
                }
            }
            nfl_z[z] = c;
        });
        long long nfluid = 0;
        for (long long c : nfl_z) nfluid += c;
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
        // the share sources index the (QG - 1) x cap_b share array with an int
        if ((long long)(LG::Q - 1) * std::max(d_.cap_b, d_.cap_f) >= (1LL << 31)) {
            err = "grid too large: boundary-list capacity exceeds the 32-bit share index";
            return 1;
        }
        d_.cap_e = (int)std::min<long long>(ncell_ + 64, std::max<long long>(1 << 16, ncell_ / 64));
        // Sweep over the dense grid (default), over a compacted fluid-cell
        // list (LBRBC_FLUID_SWEEP=list, or a batch schedule).  Measured on
        // GB300 the list is slower: a warp's 32 list cells span several rows,
        // so every population load touches more lines.
        {
            std::vector<long long> act_z(g.nz, 0);
            par_for(g.nz, [&](int z) {
                long long c = 0;
                for (int y = 0; y < g.ny; ++y) {
                    const uint8_t* row = mask + (long long)g.nx * (y + (long long)g.ny * z);
                    for (int x0 = 0; x0 < g.nx; x0 += 32) {
                        bool any = false;
                        for (int x = x0; x < std::min(g.nx, x0 + 32) && !any; ++x) any = row[x] == KIND_FLUID;
                        c += any;
                    }
                }
                act_z[z] = c;
            });
            long long active = 0;
            for (long long c : act_z) active += c;
            lane_eff_ = active ? (double)nfluid / (32.0 * active) : 1.0;
            const bool fits = g.nx <= 2048 && g.ny <= 2048 && g.nz <= 1024;
            const char* env = getenv("LBRBC_FLUID_SWEEP");
            int want = SWEEP_DENSE;
            if (env && !strcmp(env, "list")) want = SWEEP_LIST;
            if (env && !strcmp(env, "dense")) want = SWEEP_DENSE;
            if (force_list_) want = SWEEP_LIST;
            // (the list sweep is not combined with phase change)
            if (want == SWEEP_LIST && !(fits && !P.phase_change)) want = SWEEP_DENSE;
            // population layout: the active-cell layout in porous media
            // (batched domains keep the dense layout)
            int lay = P.layout;
            if (force_dense_) lay = LBRBC_LAYOUT_DENSE;
            if (lay == LBRBC_LAYOUT_AUTO) lay = lane_eff_ < 0.85 ? LBRBC_LAYOUT_SPARSE : LBRBC_LAYOUT_DENSE;
            d_.sparse = lay == LBRBC_LAYOUT_SPARSE;
            if (d_.sparse) want = SWEEP_DENSE;
            sweep_ = want;
            d_.use_fl = want == SWEEP_LIST;
            d_.cap_fl = (int)std::min<long long>(ncell_, std::max<long long>(2 * nfluid, nfluid + ncell_ / 8) + 1024);
        }
        d_.cap_log = P.event_log_capacity > 0 ? P.event_log_capacity : 0;
        nchunks_ = (int)((ncell_ + SCAN_CHUNK - 1) / SCAN_CHUNK);

        // device allocations
        constexpr int QF = LF::Q > 0 ? LF::Q : 0, QG = LG::Q;
        d_.F = d_.G = nullptr;
        if (!d_.sparse) {
            if (QF) LB_CUDA(dalloc(&d_.F, (size_t)QF * NP));
            LB_CUDA(dalloc(&d_.G, (size_t)QG * NP));
            popn_ = NP;
        } else {
            LB_CUDA(dalloc(&d_.cmap, (size_t)NP));
            LB_CUDA(cudaMemset(d_.cmap, 0xff, NP * sizeof(int)));
            LB_CUDA(dalloc(&d_.ns, 1));
            LB_CUDA(dalloc(&d_.repack, 1));
            LB_CUDA(dalloc(&d_.nrepack, 1));
            LB_CUDA(cudaMemset(d_.ns, 0, sizeof(int)));
            LB_CUDA(cudaMemset(d_.repack, 0, sizeof(int)));
            LB_CUDA(cudaMemset(d_.nrepack, 0, sizeof(int)));
            LB_CUDA(dalloc(&d_.scode, (size_t)NP));
            LB_CUDA(cudaMemset(d_.scode, 3, NP));
            LB_CUDA(dalloc(&d_.stot, 4));
            if (P.phase_change) {
                LB_CUDA(dalloc(&d_.rown, (size_t)NP));
                LB_CUDA(cudaMemset(d_.rown, 0x7f, NP * sizeof(int)));
                LB_CUDA(dalloc(&d_.ns2, 1));
                LB_CUDA(dalloc(&d_.cmap2, (size_t)NP));
            }
        }
        {
            const char* env = getenv("LBRBC_COND_GRAPH");
            cond_graphs_ = !(env && !strcmp(env, "0"));
        }
        // local maintenance of classes and lists after events (default on;
        // LBRBC_LOCAL_LISTS=0 reclassifies the whole grid and compacts the
        // lists in every step with events)
        d_.fmap = d_.candb = d_.candf = d_.lcnt = d_.rlist = nullptr;
        d_.lmark = nullptr;
        {
            const char* env = getenv("LBRBC_LOCAL_LISTS");
            if (P.phase_change && !(env && !strcmp(env, "0"))) {
                LB_CUDA(dalloc(&d_.fmap, (size_t)NP));
                LB_CUDA(cudaMemset(d_.fmap, 0xff, NP * sizeof(int)));
                LB_CUDA(dalloc(&d_.lmark, (size_t)NP));
                LB_CUDA(cudaMemset(d_.lmark, 0, NP * sizeof(uint32_t)));
                LB_CUDA(dalloc(&d_.candb, (size_t)LOC_CAND_CAP));
                LB_CUDA(dalloc(&d_.candf, (size_t)LOC_CAND_CAP));
                LB_CUDA(dalloc(&d_.lcnt, (size_t)LC_N));
                LB_CUDA(cudaMemset(d_.lcnt, 0, LC_N * sizeof(int)));
                LB_CUDA(dalloc(&d_.rlist, (size_t)LOC_EV_MAX * loc_cube<LG::DIM>()));
                // LBRBC_LOCAL_EV_MAX lowers the limit (tests mix local and
                // whole-grid steps in small runs)
                const char* lim = getenv("LBRBC_LOCAL_EV_MAX");
                const int evmax = lim ? std::max(0, std::min(LOC_EV_MAX, atoi(lim))) : LOC_EV_MAX;
                LB_CUDA(cudaMemcpy(d_.lcnt + LC_EVMAX, &evmax, sizeof(int), cudaMemcpyHostToDevice));
            }
        }
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
        LB_CUDA(dalloc(&d_.b_share, (size_t)(QG - 1) * d_.cap_b));
        LB_CUDA(cudaMemset(d_.b_share, 0, (size_t)(QG - 1) * d_.cap_b * sizeof(T)));
        if (d_.sparse) LB_CUDA(dalloc(&d_.b_cn, (size_t)d_.cap_b));
        LB_CUDA(dalloc(&d_.bmap, (size_t)NP));
        LB_CUDA(dalloc(&d_.nf, 1));
        LB_CUDA(dalloc(&d_.f_idx, (size_t)d_.cap_f));
        LB_CUDA(dalloc(&d_.f_src, (size_t)(QG - 1) * d_.cap_f));
        LB_CUDA(dalloc(&d_.nfl, 1));
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
        LB_CUDA(dalloc(&d_.facc, 4));
        nbacc_ = list_grid(d_.cap_b);
        // Grids of the boundary-list and fluid-end kernels: sized to the
        // lists at creation with 25 % head room (a grid-stride loop covers
        // any growth).  A grid sized to the capacity would hold most of the
        // GPU's thread slots with idle threads while the fluid sweep runs.
        bgrid_ = (int)std::min<long long>(nbacc_, std::max<long long>(1, (nb0_ * 5 / 4 + LIST_BLOCK - 1) / LIST_BLOCK));
        fgrid_ = (int)std::min<long long>(list_grid(d_.cap_f),
                                          std::max<long long>(1, (nf0_ * 5 / 4 + LIST_BLOCK - 1) / LIST_BLOCK));
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

        // uploads: the kinds; phi, the initial concentration and the k field
        // are formed on the device from them (or scattered from the caller's
        // arrays)
        LB_CUDA(cudaMemcpy(d_.kind, kind.data(), NP, cudaMemcpyHostToDevice));
        const int gf = grid_for(ncell_, 256);
        double* dtmp = nullptr;  // one caller-layout field at a time
        LB_CUDA(talloc(&dtmp, (size_t)ncell_));
        auto scatter = [&](double* dst, const double* host, double v_reactive) -> cudaError_t {
            cudaError_t e = cudaMemset(dst, 0, NP * sizeof(double));
            if (e == cudaSuccess && host) e = cudaMemcpy(dtmp, host, ncell_ * sizeof(double), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) k_scatter_cells<<<gf, 256, 0, own_>>>(dst, host ? dtmp : nullptr, d_.kind, g, v_reactive);
            if (e == cudaSuccess) e = cudaStreamSynchronize(own_);
            return e;
        };
        if (cudaError_t e = scatter(d_.phi, (ini && ini->phi_init) ? ini->phi_init : nullptr, 1.0); e != cudaSuccess) {
            cudaFree(dtmp);
            err = std::string("phi upload: ") + cudaGetErrorString(e);
            return 2;
        }
        if (ini && ini->k_field) {
            LB_CUDA(dalloc(&d_.kfield, (size_t)NP));
            LB_CUDA(dalloc(&d_.b_krate, (size_t)d_.cap_b));
            if (cudaError_t e = scatter(d_.kfield, ini->k_field, 0.0); e != cudaSuccess) {
                cudaFree(dtmp);
                err = std::string("k field upload: ") + cudaGetErrorString(e);
                return 2;
            }
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
        LB_CUDA(cudaMemset(d_.facc, 0, 4 * sizeof(unsigned long long)));
        LB_CUDA(cudaMemset(d_.err, 0, sizeof(int)));
        LB_CUDA(cudaMemset(d_.side, 0, 4 * sizeof(double) * g.ny * g.nz));
        if (!d_.sparse) {
            if (QF) LB_CUDA(cudaMemset(d_.F, 0, (size_t)QF * NP * sizeof(T)));
            LB_CUDA(cudaMemset(d_.G, 0, (size_t)QG * NP * sizeof(T)));
        }
        // ghost cells are solid for every lattice
        k_fill_u32<<<grid_for(NP, 256), 256, 0, own_>>>(d_.nw, NP, CLS_SOLID);
        LB_CUDA(cudaGetLastError());
        // classes, stored set (active-cell layout), lists, initial populations
        if (!d_.sparse) {
            if (rebuild(own_, 0, 1, err)) return 2;
        } else {
            enqueue_reclassify(own_, 0, 1);
            if (build_stored(err)) return 2;
            enqueue_lists(own_, 1);
            LB_CUDA(cudaGetLastError());
        }
        double *dc0 = dtmp, *du0 = nullptr;
        if (ini && ini->c_init) LB_CUDA(cudaMemcpy(dc0, ini->c_init, ncell_ * sizeof(double), cudaMemcpyHostToDevice));
        else k_c0_cells<<<grid_for(ncell_, 256), 256, 0, own_>>>(dc0, d_.kind, g, P.c_init, P.c_dirichlet);
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
        unsigned long long facc[4];
        std::vector<double> bacc((size_t)2 * nbacc_);
        LB_CUDA(cudaMemcpyAsync(sums, part + 2 * nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaMemcpyAsync(acc, d_.acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaMemcpyAsync(facc, d_.facc, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaMemcpyAsync(bacc.data(), d_.bacc, bacc.size() * sizeof(double), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaStreamSynchronize(own_));
        acc[1] = fx_value(facc);
        acc[2] = fx_value(facc + 2);
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

    // Mass balance with caller-provided device scratch and no allocation:
    // one partial pair per block of cells_per_block cells, then the final
    // sums; scratch holds 2 * max_blocks + 8 doubles.
    int ledger_scratch(double* out, double* scratch, int max_blocks, long long cells_per_block,
                       std::string& err) override {
        if (int rc = noalloc_size_check(ncell_, max_blocks, cells_per_block, err)) return rc;
        const long long nblk = (ncell_ + cells_per_block - 1) / cells_per_block;
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        double* tail = scratch + 2 * (size_t)max_blocks;
        k_reduce_partial<T, LG><<<(int)nblk, RED_BLOCK, 0, own_>>>(d_, ph_, lastodd_, scratch);
        k_reduce_final<0><<<1, 32, 0, own_>>>(scratch, (int)nblk, tail);
        k_sum_partials<0><<<1, 32, 0, own_>>>(d_.bacc, nbacc_, d_.acc, d_.facc, tail + 2);
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
    void force_dense(bool v) { force_dense_ = v; }
    bool sparse() const { return d_.sparse != 0; }
    long long stored0() const { return ns0_; }
    bool uses_list() const { return d_.use_fl != 0; }
    double lane_efficiency() const { return lane_eff_; }
    int host_nfl() const { return (int)nfluid_; }
    // One step of this domain's own kernels on st (the batched engine's
    // domain-graph schedule captures these side by side).
    int enqueue_own_step(cudaStream_t st, bool odd, std::string& err) { return enqueue_step(st, odd, err); }
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
        const size_t fbytes = (size_t)QF * popn_ * sizeof(T), gbytes = (size_t)QG * popn_ * sizeof(T);
        const size_t lbytes = (size_t)QG * NP * sizeof(T);  // adjoint arrays: plain layout over the padded grid
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
        LB_ACUDA(get(lbytes, &lam));
        LB_ACUDA(get(lbytes, &nu));
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
        LB_ACUDA(cudaMemsetAsync(lam, 0, lbytes, st));
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

    // Grid of the chunked compaction kernels: a fixed number of blocks
    // looping over the chunks, so that a step without events pays one small
    // wave of early exits instead of one block per chunk.
    int cgrid() const { return (int)std::max<long long>(1, std::min<long long>(nchunks_, 152LL * 8)); }

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
    // f(i) for i in [0, n) over up to 16 host threads (i interleaved).
    template <class F>
    static void par_for(int n, F&& f) {
        const int nt = (int)std::max(1u, std::min({16u, std::thread::hardware_concurrency(), (unsigned)std::max(1, n)}));
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t)
            pool.emplace_back([&, t]() {
                for (int i = t; i < n; i += nt) f(i);
            });
        for (auto& th : pool) th.join();
    }

    void count_lists_host(const std::vector<uint8_t>& kind, long long& nb, long long& nf) const {
        const Geo& g = d_.geo;
        const int X = g.nx + 2, Y = g.ny + 2, Z = g.nz + 2;
        const uint8_t OUT = 255;
        std::vector<uint8_t> K((size_t)X * Y * Z, OUT);
        auto wrap = [](int v, int n, bool per) { return per ? (v + n) % n : v; };
        par_for(g.nz + 2, [&](int zi) {
            const int z = zi - 1;
            for (int y = -1; y <= g.ny; ++y)
                for (int x = -1; x <= g.nx; ++x) {
                    const int xs = wrap(x, g.nx, g.per_x), ys = wrap(y, g.ny, g.per_y), zs = wrap(z, g.nz, g.per_z);
                    if (xs < 0 || xs >= g.nx || ys < 0 || ys >= g.ny || zs < 0 || zs >= g.nz) continue;
                    K[(size_t)(x + 1) + (size_t)X * ((y + 1) + (size_t)Y * (z + 1))] = kind[g.idx(xs, ys, zs)];
                }
        });
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
        enqueue_reclassify(st, lastodd, force);
        enqueue_lists(st, force);
        LB_CUDA(cudaGetLastError());
        return 0;
    }

    void enqueue_reclassify(cudaStream_t st, int form, int force) {
        k_reclassify<T, LF, LG><<<grid_for(ncell_, 256), 256, 0, st>>>(d_, ph_, form, force);
        k_recl_words<T, LF, LG><<<grid_for(ncell_, 256), 256, 0, st>>>(d_, force);
    }

    void enqueue_lists(cudaStream_t st, int force) {
        for (int which = 0; which < (d_.use_fl ? 3 : 2); ++which) {
            k_count<T, LG><<<cgrid(), 256, 0, st>>>(d_, which, force, nchunks_);
            k_scan<T><<<1, 1024, 0, st>>>(d_, nchunks_, which, force);
            k_write_lists<T, LG><<<cgrid(), 256, 0, st>>>(d_, ph_, which, force, nchunks_);
        }
    }

    // Numbering of the stored set into (cmap_out, cid_out, ns_out): range
    // codes from the current classes, then per range count / scan / write.
    // go: null (unconditional) or a device flag the kernels test first.
    void enqueue_numbering(cudaStream_t st, int* cmap_out, int* cid_out, int* ns_out, const int* go) {
        k_sp_mark<T, LG><<<grid_for(ncell_, 256), 256, 0, st>>>(d_, d_.scode, go);
        for (int r = 0; r < 3; ++r) {
            k_sp_count<T><<<cgrid(), 256, 0, st>>>(d_, d_.scode, r, go, nchunks_);
            k_sp_scan<T><<<1, 1024, 0, st>>>(d_, nchunks_, r, d_.stot, go);
            k_sp_write<T><<<cgrid(), 256, 0, st>>>(d_, d_.scode, r, d_.stot, cmap_out, cid_out, go, nchunks_);
        }
        k_sp_total<T><<<1, 1, 0, st>>>(d_, d_.stot, ns_out, go);
    }

    // Creation of the active-cell layout: count the stored set, size and
    // allocate the population storage, number the cells, build the tables.
    int build_stored(std::string& err) {
        constexpr int QF = LF::Q > 0 ? LF::Q : 0, QG = LG::Q;
        using LS = typename Stencil<LF, LG>::L;
        k_sp_mark<T, LG><<<grid_for(ncell_, 256), 256, 0, own_>>>(d_, d_.scode, nullptr);
        for (int r = 0; r < 3; ++r) {
            k_sp_count<T><<<cgrid(), 256, 0, own_>>>(d_, d_.scode, r, nullptr, nchunks_);
            k_sp_scan<T><<<1, 1024, 0, own_>>>(d_, nchunks_, r, d_.stot, nullptr);
        }
        LB_CUDA(cudaGetLastError());
        int tot[3] = {0, 0, 0};
        LB_CUDA(cudaMemcpyAsync(tot, d_.stot, 3 * sizeof(int), cudaMemcpyDeviceToHost, own_));
        LB_CUDA(cudaStreamSynchronize(own_));
        const long long ns = (long long)tot[0] + tot[1] + tot[2];
        // With phase change the stored set can grow (dissolution) up to the
        // whole grid; the storage is sized for that, so a repacking can never
        // run out of room (it costs memory only: the sweeps touch the stored
        // cells alone).  Without phase change the set never changes.
        long long cap = prm_.phase_change ? ncell_ : ns;
        cap = std::max<long long>(64, ((cap + 63) / 64) * 64);
        ns0_ = ns;
        if ((long long)std::max(QF, QG) * cap >= (1LL << 32)) {
            err = "stored set too large for 32-bit population indices";
            return 1;
        }
        d_.cap_s = cap;
        popn_ = cap;
        if (QF) LB_CUDA(dalloc(&d_.F, (size_t)QF * cap));
        LB_CUDA(dalloc(&d_.G, (size_t)QG * cap));
        if (QF) LB_CUDA(cudaMemset(d_.F, 0, (size_t)QF * cap * sizeof(T)));
        LB_CUDA(cudaMemset(d_.G, 0, (size_t)QG * cap * sizeof(T)));
        LB_CUDA(dalloc(&d_.cid, (size_t)cap));
        LB_CUDA(dalloc(&d_.nwc, (size_t)cap));
        LB_CUDA(dalloc(&d_.etab, (size_t)tab_entries<LF, LG>() * cap));
        LB_CUDA(cudaMemset(d_.nwc, 0, cap * sizeof(uint32_t)));
        if (prm_.phase_change) {
            LB_CUDA(dalloc(&d_.cid2, (size_t)cap));
            if (QF) LB_CUDA(dalloc(&d_.F2, (size_t)QF * cap));
            LB_CUDA(dalloc(&d_.G2, (size_t)QG * cap));
        }
        enqueue_numbering(own_, d_.cmap, d_.cid, d_.ns, nullptr);
        k_sp_tables<T, LF, LG><<<grid_for(cap, 256), 256, 0, own_>>>(d_, nullptr);
        LB_CUDA(cudaGetLastError());
        return 0;
    }

    // Repacking inside the step graph: every kernel returns at once unless a
    // reclassification found a cell that needs storage it does not have.
    void enqueue_repack(cudaStream_t st) {
        k_sp_clear2<T><<<grid_for(d_.geo.NP, 256), 256, 0, st>>>(d_);
        enqueue_numbering(st, d_.cmap2, d_.cid2, d_.ns2, d_.repack);
        k_sp_gather<T, LF, LG><<<grid_for(d_.cap_s, 256), 256, 0, st>>>(d_, ph_);
        k_sp_commit<T, LF, LG><<<grid_for(d_.geo.NP, 256), 256, 0, st>>>(d_);
        k_sp_commit_end<T><<<1, 1, 0, st>>>(d_);
        k_sp_tables<T, LF, LG><<<grid_for(d_.cap_s, 256), 256, 0, st>>>(d_, d_.repack);
        k_sp_recn<T><<<list_grid(d_.cap_b), LIST_BLOCK, 0, st>>>(d_);
        k_sp_repack_done<T><<<1, 1, 0, st>>>(d_);
    }

    // One time step; with `ev` (5 events) the kernel groups are bracketed by
    // event records: fluid sweep, boundary list, fluid ends, phase change.
    int enqueue_step(cudaStream_t st, bool odd, std::string& err, cudaEvent_t* ev = nullptr,
                     const Dev<T>* dv = nullptr) {
        const Dev<T>& d_ = dv ? *dv : this->d_;
        const Geo& g = d_.geo;
        const bool sp = d_.sparse != 0;
        dim3 grid((g.nx + FLUID_BLOCK - 1) / FLUID_BLOCK, g.ny, g.nz);
        // one thread per stored cell at creation; the sweep strides over any
        // growth of the set
        const int gsp = sp ? (int)std::max<long long>(1, (ns0_ + FLUID_BLOCK - 1) / FLUID_BLOCK) : 1;
        if (ev) LB_CUDA(cudaEventRecord(ev[0], st));
        // Without per-group timing the boundary list and the fluid ends run
        // on a second stream beside the fluid sweep: the three kernels touch
        // disjoint population slots (each slot is read and written by one
        // cell per step), and the fluid ends depend only on the boundary list.
        const bool fork = ev == nullptr;
        // Inside a graph the phase-change path is the body of a conditional
        // node: the gate after the fluid ends (the last kernel that raises
        // events) sets its condition, and in a step without events also
        // counts the step, so such a step launches nothing after the sweep.
        bool cond = false;
        cudaGraphConditionalHandle h{};
        if (ph_.phase_change && fork && cond_graphs_) {
            cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
            LB_CUDA(cudaStreamIsCapturing(st, &cst));
            if (cst == cudaStreamCaptureStatusActive) {
                cudaGraph_t gr = nullptr;
                LB_CUDA(cudaStreamGetCaptureInfo(st, &cst, nullptr, &gr, nullptr, nullptr, nullptr));
                LB_CUDA(cudaGraphConditionalHandleCreate(&h, gr, 0, 0));
                cond = true;
            }
        }
        if (fork) {
            LB_CUDA(cudaEventRecord(fork_, st));
            LB_CUDA(cudaStreamWaitEvent(aux_, fork_, 0));
            launch_bound(aux_, odd, d_);
            k_fend<T, LG><<<fgrid_, LIST_BLOCK, 0, aux_>>>(d_, ph_);
            if (cond) k_ev_gate<T><<<1, 1, 0, aux_>>>(d_, h);
            LB_CUDA(cudaEventRecord(join_, aux_));
        }
        if (sp) {
            if (odd) k_fluid_sp<T, LF, LG, true><<<gsp, FLUID_BLOCK, 0, st>>>(d_, ph_, pt_);
            else k_fluid_sp<T, LF, LG, false><<<gsp, FLUID_BLOCK, 0, st>>>(d_, ph_, pt_);
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
            launch_bound(st, odd, d_);
            LB_CUDA(cudaEventRecord(ev[2], st));
            k_fend<T, LG><<<fgrid_, LIST_BLOCK, 0, st>>>(d_, ph_);
            LB_CUDA(cudaEventRecord(ev[3], st));
        }
        if (ph_.phase_change) {
            if (cond) {
                if (enqueue_events_conditional(st, odd, d_, h, err)) return 2;
            } else {
                enqueue_events(st, odd, d_);
                k_step_end<T><<<1, 1, 0, st>>>(d_);
            }
        }
        if (ev) LB_CUDA(cudaEventRecord(ev[4], st));
        LB_CUDA(cudaGetLastError());
        return 0;
    }

    // The phase-change path of one step: events, classes, stored set, lists.
    void enqueue_events(cudaStream_t st, bool odd, const Dev<T>& d_) {
        const bool sp = d_.sparse != 0;
        const int eg = 152 * 2;
        // The event kernels read and write post-collision populations.
        // Dense layout: at their AA positions after this step.  Active-
        // cell layout: in the even-step form (each cell's own slots);
        // after an odd step the links of the event region are swapped
        // into that form first, and back once the classes have changed.
        const int form = sp ? 0 : (odd ? 1 : 0);
        k_ev_mark<T><<<eg, 256, 0, st>>>(d_);
        if (sp && odd) {
            k_sp_rmark<T, LG><<<eg, 256, 0, st>>>(d_);
            k_sp_swap<T, LF, LG><<<eg, 256, 0, st>>>(d_);
        }
        k_ev_compute<T, LF, LG><<<eg, 256, 0, st>>>(d_, ph_, form);
        k_ev_apply_self<T, LF, LG><<<eg, 256, 0, st>>>(d_, ph_, form);
        k_ev_neighbours<T, LG><<<eg, 256, 0, st>>>(d_, ph_, form);
        // Classes and lists: locally around the events (the cube of half
        // width 2 around each), or over the whole grid when the events
        // are many, the stored set was repacked or the lists need a
        // compaction.
        const bool loc = d_.lcnt != nullptr;
        if (loc) k_loc_decide<T><<<1, 1, 0, st>>>(d_);
        enqueue_reclassify(st, form, 0);
        if (loc) k_loc_recl<T, LF, LG><<<eg, 256, 0, st>>>(d_, ph_, form);
        if (sp) enqueue_repack(st);
        if (sp) k_sp_retab<T, LF, LG><<<eg, 256, 0, st>>>(d_);
        if (sp && odd) {
            k_sp_swap<T, LF, LG><<<eg, 256, 0, st>>>(d_);
            k_sp_rreset<T, LG><<<eg, 256, 0, st>>>(d_);
        }
        if (loc) {
            k_loc_lists<T, LG><<<eg, 256, 0, st>>>(d_, ph_);
            k_loc_plan<T><<<1, 1, 0, st>>>(d_);
            k_loc_append<T, LG><<<eg, 256, 0, st>>>(d_, ph_);
            k_loc_fsrc<T, LG><<<eg, 256, 0, st>>>(d_);
        }
        enqueue_lists(st, 0);
        k_ev_reset<T><<<eg, 256, 0, st>>>(d_);
    }

    // The same path and the step counter as the body of an IF node (handle
    // h, set by the gate) of the graph being captured on st.
    int enqueue_events_conditional(cudaStream_t st, bool odd, const Dev<T>& d_, cudaGraphConditionalHandle h,
                                   std::string& err) {
        cudaStreamCaptureStatus cst;
        cudaGraph_t gr = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        LB_CUDA(cudaStreamGetCaptureInfo(st, &cst, nullptr, &gr, &deps, nullptr, &nd));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        LB_CUDA(cudaGraphAddNode(&node, gr, deps, nullptr, nd, &np));
        LB_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        if (!body_) LB_CUDA(cudaStreamCreateWithFlags(&body_, cudaStreamNonBlocking));
        LB_CUDA(cudaStreamBeginCaptureToGraph(body_, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
        enqueue_events(body_, odd, d_);
        k_step_end<T><<<1, 1, 0, body_>>>(d_);
        cudaGraph_t bg = nullptr;
        const cudaError_t e1 = cudaGetLastError();
        const cudaError_t e2 = cudaStreamEndCapture(body_, &bg);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            err = std::string("capture of the event path: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2);
            return 2;
        }
        return 0;
    }

    void launch_bound(cudaStream_t st, bool odd, const Dev<T>& d) {
        if (d.sparse) {
            if (odd) k_bound<T, LF, LG, true, true><<<bgrid_, LIST_BLOCK, 0, st>>>(d, ph_, pt_);
            else k_bound<T, LF, LG, false, true><<<bgrid_, LIST_BLOCK, 0, st>>>(d, ph_, pt_);
        } else {
            if (odd) k_bound<T, LF, LG, true, false><<<bgrid_, LIST_BLOCK, 0, st>>>(d, ph_, pt_);
            else k_bound<T, LF, LG, false, false><<<bgrid_, LIST_BLOCK, 0, st>>>(d, ph_, pt_);
        }
    }

   public:
    // Kernel launches of the phase-change path of one step (mean of an even
    // and an odd step).
    int event_path_launches() const override {
        if (!ph_.phase_change) return 0;
        int n = 4 + 2 + 3 * (d_.use_fl ? 3 : 2) + 1 + (cond_graphs_ ? 1 : 0);  // events, reclassification,
                                                                             // lists, reset (+ step counter)
        if (d_.sparse) n += 1 + (1 + 9 + 1) + 6 + 1 + 2;  // repacking (conditional), table refresh, swaps of odd steps / 2
        if (d_.lcnt) n += 6;                              // local reclassification and list maintenance
        return n;
    }

    // Kernel launches of one step of the step graphs without phase-change
    // events: the fluid sweep, the boundary list and the fluid ends, and with
    // phase change the gate of the event path and the step counter (the path
    // itself runs only in steps with events, or always without conditional
    // graph nodes).
    int launches_per_step() const override {
        int n = 3;
        if (ph_.phase_change) n += cond_graphs_ ? 1 : 1 + event_path_launches();
        return n;
    }

    int layout_info(int64_t* out, std::string& err) override {
        LB_CUDA(cudaStreamSynchronize(last_stream_ ? last_stream_ : own_));
        constexpr int QF = LF::Q > 0 ? LF::Q : 0, QG = LG::Q;
        out[0] = d_.sparse ? LBRBC_LAYOUT_SPARSE : LBRBC_LAYOUT_DENSE;
        out[1] = d_.geo.NP;
        out[2] = 0;
        if (d_.sparse) {
            int h[2] = {0, 0};
            LB_CUDA(cudaMemcpy(&h[0], d_.ns, sizeof(int), cudaMemcpyDeviceToHost));
            LB_CUDA(cudaMemcpy(&h[1], d_.nrepack, sizeof(int), cudaMemcpyDeviceToHost));
            out[1] = h[0];
            out[2] = h[1];
        }
        out[3] = (int64_t)(QF + QG) * popn_ * (int64_t)sizeof(T);
        return 0;
    }

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
        if (body_) cudaStreamDestroy(body_);
        body_ = nullptr;
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
    int nbacc_ = 0, bgrid_ = 1, fgrid_ = 1;
    int lastodd_ = 1;
    int64_t steps_ = 0;
    cudaStream_t own_ = nullptr, last_stream_ = nullptr, aux_ = nullptr;
    cudaEvent_t fork_ = nullptr, join_ = nullptr;
    cudaStream_t body_ = nullptr;   // capture stream of the conditional event path
    bool cond_graphs_ = true;       // LBRBC_COND_GRAPH=0: the event path always runs (early exits)
    int sweep_ = SWEEP_DENSE;
    cudaGraphExec_t g_even_{}, g_odd_{}, g_pair_{};
    bool graphs_ = false;
    bool batched_ = false;
    bool force_list_ = false;
    bool force_dense_ = false;
    long long popn_ = 0;  // population slots per direction (padded grid or stored-cell capacity)
    long long ns0_ = 0;   // stored cells at creation (active-cell layout)
    double lane_eff_ = 1.0;
    std::vector<void*> allocs_;
};

#undef LB_CUDA

}  // namespace lbrbc
