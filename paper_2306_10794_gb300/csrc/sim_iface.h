// Internal interface between the C ABI and the templated device engines.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbrbc.h"

namespace lbrbc {

// Return codes follow lbrbc_status.
class ISim {
   public:
    virtual ~ISim() {}
    virtual int init(const lbrbc_params& p, const uint8_t* mask, const lbrbc_init* ini, std::string& err) = 0;
    virtual int step(int64_t n, cudaStream_t s, std::string& err) = 0;
    virtual int fields(double* u, double* rho, double* c, double* phi, int device, std::string& err) = 0;
    virtual int classes(uint8_t* out, std::string& err) = 0;
    virtual int ledger(double* out, std::string& err) = 0;
    virtual int events(int64_t* count, int64_t capacity, int64_t* step, int64_t* node, int32_t* kind,
                       std::string& err) = 0;
    virtual int check(std::string& err) = 0;
    virtual int profile(int64_t n, cudaStream_t s, double* ms, std::string& err) = 0;
    virtual int ledger_scratch(double* out, double* scratch, int max_blocks, long long cells_per_block,
                               std::string& err) = 0;
    virtual int launches_per_step() const = 0;
    virtual int event_path_launches() const = 0;
    virtual int adjoint(int64_t n, double* J, double* dk, double* dceq, double* dk_field, std::string& err) = 0;
    virtual long long fluid_cells() const = 0;
    virtual long long boundary_cells() const = 0;
    virtual int layout_info(int64_t* out, std::string& err) = 0;
};

// Many independent domains stepped together (same lattices and precision).
class IBatch {
   public:
    virtual ~IBatch() {}
    virtual int init(int n, const lbrbc_params* p, const uint8_t* const* masks, const lbrbc_init* inits,
                     std::string& err) = 0;
    virtual int step(int64_t n, cudaStream_t s, std::string& err) = 0;
    virtual int autotune(int pairs, cudaStream_t s, int64_t* choice, double* ms_per_step, std::string& err) = 0;
    virtual int schedule(int policy, int order, int per_sm, std::string& err) = 0;
    virtual int size() const = 0;
    virtual ISim* domain(int i) = 0;
    virtual long long fluid_cells() const = 0;
};

// Size rule of the scratch-based ledger: one partial pair per block of
// cells_per_block cells, at most max_blocks blocks.  Returns LBRBC_OK or
// LBRBC_ERR_ARG with a message naming the limit.
inline int noalloc_size_check(long long ncell, int max_blocks, long long cells_per_block, std::string& err) {
    if (ncell < 0 || max_blocks < 1 || cells_per_block < 1) {
        err = "invalid size arguments";
        return LBRBC_ERR_ARG;
    }
    const long long nblk = (ncell + cells_per_block - 1) / cells_per_block;
    if (nblk > max_blocks) {
        err = "grid of " + std::to_string(ncell) + " cells exceeds the static scratch of this entry point (" +
              std::to_string((long long)max_blocks * cells_per_block) + " cells)";
        return LBRBC_ERR_ARG;
    }
    err.clear();
    return LBRBC_OK;
}

// Factories, one per translation unit; nullptr if the combination is not built.
ISim* make_sim_3d(int precision, int flow_q, int solute_q);
ISim* make_sim_2d(int precision, int flow_q, int solute_q);
IBatch* make_batch_3d(int precision, int flow_q, int solute_q);

}  // namespace lbrbc

// The opaque handles of the C ABI.  A domain handle handed out by a batch is
// borrowed: its engine belongs to the batch.
struct lbrbc_sim {
    lbrbc::ISim* impl = nullptr;
    std::string err;
    int device = 0;
    bool borrowed = false;
};

struct lbrbc_batch {
    lbrbc::IBatch* impl = nullptr;
    std::string err;
    std::vector<lbrbc_sim> views;
};
