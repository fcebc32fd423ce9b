// 2D engines: D2Q9 flow + D2Q5 solute, D2Q5 or D2Q9 solute alone.
#include "engine.cuh"

namespace lbrbc {

ISim* make_sim_2d(int precision, int flow_q, int solute_q) {
    const bool f64 = precision == LBRBC_FP64;
    if (flow_q == 9 && solute_q == 5) {
        if (f64) return new Engine<double, D2Q9, D2Q5>();
        return new Engine<float, D2Q9, D2Q5>();
    }
    if (flow_q == 0 && solute_q == 5) {
        if (f64) return new Engine<double, NoFlow, D2Q5>();
        return new Engine<float, NoFlow, D2Q5>();
    }
    if (flow_q == 0 && solute_q == 9) {
        if (f64) return new Engine<double, NoFlow, D2Q9>();
        return new Engine<float, NoFlow, D2Q9>();
    }
    return nullptr;
}

}  // namespace lbrbc
