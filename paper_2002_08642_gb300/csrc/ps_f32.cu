// ps_f32.cu -- float instantiations of the step engine for every built-in grid size.
#include "ps_engine.cuh"

namespace ps {

#define PS_OPS_ENTRY(n)                                  \
    case n: {                                            \
        static const Ops o = Engine<float, n>::ops();       \
        return &o;                                       \
    }

const Ops* ops_f32(int n) {
    switch (n) {
        PS_SIZES(PS_OPS_ENTRY)
        default: return nullptr;
    }
}

}  // namespace ps
