// lbrbc_mass_ledger_noalloc: the mass balance of lbrbc_mass_ledger computed
// without allocating device memory.  The reduction's partial sums live in a
// file-scope device array, shared by every call on a device (see the
// declaration in include/lbrbc.h for the contract).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "sim_iface.h"

#define LBRBC_NOALLOC_MAX_BLOCKS 4096
#define LBRBC_NOALLOC_CELLS_PER_BLOCK 65536LL

namespace {

// Partial sums (two per block) plus eight result slots: 65.6 KB per device,
// held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_ledger_scratch[2 * LBRBC_NOALLOC_MAX_BLOCKS + 8];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so kernels are always given
// this address.  It is looked up on every call (no cache): after a device
// reset or a new primary context the module is reloaded and the array may
// move, and the lookup costs little next to the call's stream synchronisation.
int scratch_here(double** out, std::string& err) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_ledger_scratch);
    if (e != cudaSuccess) {
        err = std::string("cudaGetSymbolAddress(static ledger scratch): ") + cudaGetErrorString(e);
        return LBRBC_ERR_CUDA;
    }
    *out = (double*)p;
    return LBRBC_OK;
}

}  // namespace


extern "C" lbrbc_status lbrbc_mass_ledger_noalloc(lbrbc_sim* sim, double* out) {
    if (!sim || !out) {
        if (sim) sim->err = "NULL argument";
        return LBRBC_ERR_ARG;
    }
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) {
        sim->err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return LBRBC_ERR_CUDA;
    }
    if (cur != sim->device && (e = cudaSetDevice(sim->device)) != cudaSuccess) {
        sim->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return LBRBC_ERR_CUDA;
    }
    std::string err;
    double* scratch = nullptr;
    int rc = scratch_here(&scratch, err);
    if (rc == LBRBC_OK)
        rc = sim->impl->ledger_scratch(out, scratch, LBRBC_NOALLOC_MAX_BLOCKS, LBRBC_NOALLOC_CELLS_PER_BLOCK, err);
    if (cur != sim->device) cudaSetDevice(cur);
    if (rc != LBRBC_OK) sim->err = err;
    return (lbrbc_status)rc;
}

extern "C" lbrbc_status lbrbc_noalloc_size_check(int64_t n_cells, int32_t max_blocks, int64_t cells_per_block,
                                                 char* msg, int32_t msg_len) {
    std::string err;
    const int rc = lbrbc::noalloc_size_check((long long)n_cells, (int)max_blocks, (long long)cells_per_block, err);
    if (msg && msg_len > 0) {
        const size_t n = std::min<size_t>(err.size(), (size_t)msg_len - 1);
        memcpy(msg, err.data(), n);
        msg[n] = '\0';
    }
    return (lbrbc_status)rc;
}
