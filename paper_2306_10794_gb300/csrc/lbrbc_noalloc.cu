// lbrbc_mass_ledger_noalloc: the mass balance of lbrbc_mass_ledger computed
// without allocating device memory.  The reduction's partial sums live in a
// file-scope device array, shared by every call on a device (see the
// declaration in include/lbrbc.h for the contract).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sim_iface.h"

#define LBRBC_NOALLOC_MAX_BLOCKS 4096
#define LBRBC_NOALLOC_CELLS_PER_BLOCK 65536LL

namespace {

// Partial sums (two per block) plus eight result slots: 65.6 KB per device,
// held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_ledger_scratch[2 * LBRBC_NOALLOC_MAX_BLOCKS + 8];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev`, looked up once per device
// with that device current.  In host code the array's name is only a
// host-side stand-in, so kernels are always given this address.
int scratch_on(int dev, double** out, std::string& err) {
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device index out of range for the static ledger scratch";
        return LBRBC_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_ledger_scratch);
        if (e != cudaSuccess) {
            err = std::string("cudaGetSymbolAddress(static ledger scratch): ") + cudaGetErrorString(e);
            return LBRBC_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
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
    int rc = scratch_on(sim->device, &scratch, err);
    if (rc == LBRBC_OK)
        rc = sim->impl->ledger_scratch(out, scratch, LBRBC_NOALLOC_MAX_BLOCKS, LBRBC_NOALLOC_CELLS_PER_BLOCK, err);
    if (cur != sim->device) cudaSetDevice(cur);
    if (rc != LBRBC_OK) sim->err = err;
    return (lbrbc_status)rc;
}
