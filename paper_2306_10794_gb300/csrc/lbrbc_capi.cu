// C ABI of the library: argument validation, dispatch to the engines, error
// messages.  The declarations and their documentation are in include/lbrbc.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sim_iface.h"


namespace {

thread_local std::string g_create_error;

lbrbc_status fail(lbrbc_sim* s, int code, const std::string& msg) {
    if (s) s->err = msg;
    else g_create_error = msg;
    return (lbrbc_status)code;
}

}  // namespace

std::string lbrbc_validate_params(const lbrbc_params& p);

namespace {

std::string validate(const lbrbc_params& p) { return lbrbc_validate_params(p); }

}  // namespace

std::string lbrbc_validate_params(const lbrbc_params& p) {
    if (p.dim != 2 && p.dim != 3) return "dim must be 2 or 3";
    if (p.nx < 1 || p.ny < 1 || (p.dim == 3 && p.nz < 1)) return "grid sizes must be positive";
    if (p.dim == 2 && p.nz != 1 && p.nz != 0) return "2D grids need nz = 1";
    if (p.dim == 3 && !((p.flow_q == 19 || p.flow_q == 0) && p.solute_q == 7))
        return "3D needs flow_q in {19, 0} and solute_q = 7";
    if (p.dim == 2 && !((p.flow_q == 9 && p.solute_q == 5) || (p.flow_q == 0 && (p.solute_q == 5 || p.solute_q == 9))))
        return "2D needs (flow_q, solute_q) in {(9, 5), (0, 5), (0, 9)}";
    for (int a = 0; a < 3; ++a) {
        if (p.bc[a] < LBRBC_PERIODIC || p.bc[a] > LBRBC_OPEN) return "bc must be PERIODIC, WALL or OPEN";
        if (a > 0 && p.bc[a] == LBRBC_OPEN) return "only the x axis may be OPEN";
    }
    if (p.bc[0] == LBRBC_OPEN && p.nx < 2) return "an OPEN x axis needs nx >= 2";
    if (!(p.tau_solute > 0.5)) return "tau_solute must exceed 1/2";
    if (p.flow_q && !(p.tau_flow > 0.5)) return "tau_flow must exceed 1/2";
    if (p.magic_flow == 0.0 || p.magic_solute == 0.0) return "Lambda = 0 is singular (use < 0 for BGK)";
    if (p.rest_fraction >= 1.0) return "rest_fraction must be < 1";
    if (p.rest_fraction >= 0.0 && p.solute_q == 9) return "the rest fraction applies to D2Q5 / D3Q7 only";
    if (!(p.k_r >= 0.0) || !(p.c_eq >= 0.0)) return "k_r and c_eq must be >= 0";
    if (!(p.molar_volume >= 0.0)) return "molar_volume must be >= 0";
    if (p.phase_change && !(p.molar_volume > 0.0)) return "phase change needs molar_volume > 0";
    if (p.scheme < LBRBC_SCHEME_NEW || p.scheme > LBRBC_SCHEME_ANTI_BB) return "unknown scheme";
    if (p.precision != LBRBC_FP32 && p.precision != LBRBC_FP64) return "precision must be FP32 or FP64";
    if (!(p.rho_init > 0.0)) return "rho_init must be positive";
    if (p.event_log_capacity < 0) return "event_log_capacity must be >= 0";
    if (p.layout < LBRBC_LAYOUT_AUTO || p.layout > LBRBC_LAYOUT_SPARSE) return "layout must be AUTO, DENSE or SPARSE";
    return "";
}

extern "C" {

lbrbc_status lbrbc_create(const lbrbc_params* params, const uint8_t* mask, const lbrbc_init* init, lbrbc_sim** out) {
    if (!params || !mask || !out) return fail(nullptr, LBRBC_ERR_ARG, "params, mask and out must be non-NULL");
    *out = nullptr;
    lbrbc_params p = *params;
    if (p.dim == 2) p.nz = 1;
    std::string why = validate(p);
    if (!why.empty()) return fail(nullptr, LBRBC_ERR_ARG, why);
    const long long n = (long long)p.nx * p.ny * p.nz;
    for (long long i = 0; i < n; ++i)
        if (mask[i] > LBRBC_CELL_DIRICHLET) return fail(nullptr, LBRBC_ERR_ARG, "mask values must be 0, 1 or 2");
    if (init && init->phi_init && p.phase_change)
        for (long long i = 0; i < n; ++i)
            if (mask[i] == LBRBC_CELL_FLUID && init->phi_init[i] >= 1.0)
                return fail(nullptr, LBRBC_ERR_ARG, "fluid cells must start with phi < 1");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(nullptr, LBRBC_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
    lbrbc::ISim* impl = p.dim == 3 ? lbrbc::make_sim_3d(p.precision, p.flow_q, p.solute_q)
                                   : lbrbc::make_sim_2d(p.precision, p.flow_q, p.solute_q);
    if (!impl) return fail(nullptr, LBRBC_ERR_UNSUPPORTED, "lattice combination not built");
    lbrbc_sim* s = new (std::nothrow) lbrbc_sim();
    if (!s) {
        delete impl;
        return fail(nullptr, LBRBC_ERR_ARG, "out of host memory");
    }
    s->impl = impl;
    cudaGetDevice(&s->device);
    std::string err;
    int rc = impl->init(p, mask, init, err);
    if (rc) {
        delete s->impl;
        delete s;
        return fail(nullptr, rc, err);
    }
    *out = s;
    return LBRBC_OK;
}

lbrbc_status lbrbc_step(lbrbc_sim* sim, int64_t n, void* stream) {
    if (!sim) return fail(nullptr, LBRBC_ERR_ARG, "NULL simulation");
    if (n < 0) return fail(sim, LBRBC_ERR_ARG, "n must be >= 0");
    std::string err;
    int rc = sim->impl->step(n, (cudaStream_t)stream, err);
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_fields(lbrbc_sim* sim, double* u, double* rho, double* c, double* phi, int device) {
    if (!sim) return fail(nullptr, LBRBC_ERR_ARG, "NULL simulation");
    std::string err;
    int rc = sim->impl->fields(u, rho, c, phi, device, err);
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_classes(lbrbc_sim* sim, uint8_t* out) {
    if (!sim || !out) return fail(sim, LBRBC_ERR_ARG, "NULL argument");
    std::string err;
    int rc = sim->impl->classes(out, err);
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_mass_ledger(lbrbc_sim* sim, double* out) {
    if (!sim || !out) return fail(sim, LBRBC_ERR_ARG, "NULL argument");
    std::string err;
    int rc = sim->impl->ledger(out, err);
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_events(lbrbc_sim* sim, int64_t* count, int64_t capacity, int64_t* step, int64_t* node,
                          int32_t* kind) {
    if (!sim || !count) return fail(sim, LBRBC_ERR_ARG, "NULL argument");
    if (capacity < 0) return fail(sim, LBRBC_ERR_ARG, "capacity must be >= 0");
    std::string err;
    int rc = sim->impl->events(count, capacity, step, node, kind, err);
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_adjoint(lbrbc_sim* sim, int64_t n_steps, double* J, double* dJ_dk, double* dJ_dceq,
                           double* dJ_dkfield) {
    if (!sim) return fail(nullptr, LBRBC_ERR_ARG, "NULL simulation");
    if (sim->borrowed) return fail(sim, LBRBC_ERR_STATE, "the adjoint of a batched domain is not available");
    std::string err;
    int rc = sim->impl->adjoint(n_steps, J, dJ_dk, dJ_dceq, dJ_dkfield, err);
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_profile_step(lbrbc_sim* sim, int64_t n, void* stream, double* ms_out, int64_t* launches) {
    if (!sim || !ms_out) return fail(sim, LBRBC_ERR_ARG, "NULL argument");
    if (n < 1) return fail(sim, LBRBC_ERR_ARG, "n must be >= 1");
    std::string err;
    int rc = sim->impl->profile(n, (cudaStream_t)stream, ms_out, err);
    if (!rc && launches) *launches = sim->impl->launches_per_step();
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_info(lbrbc_sim* sim, int64_t* out) {
    if (!sim || !out) return fail(sim, LBRBC_ERR_ARG, "NULL argument");
    out[0] = sim->impl->fluid_cells();
    out[1] = sim->impl->boundary_cells();
    out[2] = sim->impl->launches_per_step();
    return LBRBC_OK;
}

lbrbc_status lbrbc_launch_counts(lbrbc_sim* sim, int64_t* out) {
    if (!sim || !out) return fail(sim, LBRBC_ERR_ARG, "NULL argument");
    out[0] = sim->impl->launches_per_step();
    out[1] = sim->impl->event_path_launches();
    return LBRBC_OK;
}

lbrbc_status lbrbc_layout_info(lbrbc_sim* sim, int64_t* out) {
    if (!sim || !out) return fail(sim, LBRBC_ERR_ARG, "NULL argument");
    std::string err;
    int rc = sim->impl->layout_info(out, err);
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_check(lbrbc_sim* sim) {
    if (!sim) return fail(nullptr, LBRBC_ERR_ARG, "NULL simulation");
    std::string err;
    int rc = sim->impl->check(err);
    return rc ? fail(sim, rc, err) : LBRBC_OK;
}

lbrbc_status lbrbc_batch_create(int32_t n, const lbrbc_params* params, const uint8_t* const* masks,
                                const lbrbc_init* inits, lbrbc_batch** out) {
    if (!params || !masks || !out || n < 1) return fail(nullptr, LBRBC_ERR_ARG, "need n >= 1, params, masks and out");
    *out = nullptr;
    std::vector<lbrbc_params> ps(params, params + n);
    for (int i = 0; i < n; ++i) {
        lbrbc_params& p = ps[i];
        if (p.dim == 2) p.nz = 1;
        std::string why = validate(p);
        if (!why.empty()) return fail(nullptr, LBRBC_ERR_ARG, "domain " + std::to_string(i) + ": " + why);
        if (p.dim != 3 || p.flow_q != ps[0].flow_q || p.solute_q != ps[0].solute_q || p.precision != ps[0].precision)
            return fail(nullptr, LBRBC_ERR_ARG, "batched domains must be 3D with the same lattices and precision");
        if (!masks[i]) return fail(nullptr, LBRBC_ERR_ARG, "NULL mask");
        const long long nc = (long long)p.nx * p.ny * p.nz;
        for (long long c = 0; c < nc; ++c)
            if (masks[i][c] > LBRBC_CELL_DIRICHLET) return fail(nullptr, LBRBC_ERR_ARG, "mask values must be 0, 1 or 2");
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(nullptr, LBRBC_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
    lbrbc::IBatch* impl = lbrbc::make_batch_3d(ps[0].precision, ps[0].flow_q, ps[0].solute_q);
    if (!impl) return fail(nullptr, LBRBC_ERR_UNSUPPORTED, "batched lattice combination not built");
    lbrbc_batch* b = new (std::nothrow) lbrbc_batch();
    if (!b) {
        delete impl;
        return fail(nullptr, LBRBC_ERR_ARG, "out of host memory");
    }
    b->impl = impl;
    std::string err;
    int rc = impl->init(n, ps.data(), masks, inits, err);
    if (rc) {
        delete b->impl;
        delete b;
        return fail(nullptr, rc, err);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    b->views.resize(n);
    for (int i = 0; i < n; ++i) {
        b->views[i].impl = impl->domain(i);
        b->views[i].device = dev;
        b->views[i].borrowed = true;
    }
    *out = b;
    return LBRBC_OK;
}

lbrbc_status lbrbc_batch_step(lbrbc_batch* b, int64_t n, void* stream) {
    if (!b) return fail(nullptr, LBRBC_ERR_ARG, "NULL batch");
    if (n < 0) {
        b->err = "n must be >= 0";
        return LBRBC_ERR_ARG;
    }
    int rc = b->impl->step(n, (cudaStream_t)stream, b->err);
    return (lbrbc_status)rc;
}

lbrbc_status lbrbc_batch_autotune(lbrbc_batch* b, int32_t pairs, void* stream, int64_t* choice, double* ms_per_step) {
    if (!b || pairs < 1) {
        if (b) b->err = "pairs must be >= 1";
        return LBRBC_ERR_ARG;
    }
    int rc = b->impl->autotune(pairs, (cudaStream_t)stream, choice, ms_per_step, b->err);
    return (lbrbc_status)rc;
}

lbrbc_status lbrbc_batch_schedule(lbrbc_batch* b, int32_t policy, int32_t order, int32_t blocks_per_sm) {
    if (!b) return LBRBC_ERR_ARG;
    if (policy < 0 || policy > 4 || order < 0 || order > 1 || blocks_per_sm < 1 || blocks_per_sm > 64) {
        b->err = "schedule out of range (policy 0-4, order 0-1, blocks per SM 1-64)";
        return LBRBC_ERR_ARG;
    }
    return (lbrbc_status)b->impl->schedule(policy, order, blocks_per_sm, b->err);
}

lbrbc_status lbrbc_batch_info(lbrbc_batch* b, int64_t* out) {
    if (!b || !out) return LBRBC_ERR_ARG;
    out[0] = b->impl->size();
    out[1] = b->impl->fluid_cells();
    return LBRBC_OK;
}

lbrbc_sim* lbrbc_batch_domain(lbrbc_batch* b, int32_t i) {
    if (!b || i < 0 || i >= (int32_t)b->views.size()) return nullptr;
    return &b->views[i];
}

const char* lbrbc_batch_last_error(lbrbc_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

void lbrbc_batch_destroy(lbrbc_batch* b) {
    if (!b) return;
    delete b->impl;
    delete b;
}

const char* lbrbc_last_error(lbrbc_sim* sim) {
    if (sim) return sim->err.c_str();
    return g_create_error.c_str();
}

void lbrbc_destroy(lbrbc_sim* sim) {
    if (!sim || sim->borrowed) return;
    delete sim->impl;
    delete sim;
}

}  // extern "C"
