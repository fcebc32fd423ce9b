// 3D engines: D3Q19 flow + D3Q7 solute, and D3Q7 solute alone.
#include "batch.cuh"

namespace lbrbc {

ISim* make_sim_3d(int precision, int flow_q, int solute_q) {
    if (solute_q != 7) return nullptr;
    if (flow_q == 19) {
        if (precision == LBRBC_FP64) return new Engine<double, D3Q19, D3Q7>();
        return new Engine<float, D3Q19, D3Q7>();
    }
    if (flow_q == 0) {
        if (precision == LBRBC_FP64) return new Engine<double, NoFlow, D3Q7>();
        return new Engine<float, NoFlow, D3Q7>();
    }
    return nullptr;
}

IBatch* make_batch_3d(int precision, int flow_q, int solute_q) {
    if (flow_q != 19 || solute_q != 7) return nullptr;
    if (precision == LBRBC_FP64) return new BatchEngine<double, D3Q19, D3Q7>();
    return new BatchEngine<float, D3Q19, D3Q7>();
}

}  // namespace lbrbc
