// ps_f64_b.cu -- double instantiations of the step engine for the grid sizes
// of chain B (cubic, and N x N x N/2 where N/2 is in the chain too).
#include "ps_engine.cuh"

namespace ps {

#define PS_OPS_ENTRY(n) \
    case n:             \
        return ops_for_nz<double, n>(nz);

const Ops* ops_f64_b(int n, int nz) {
    switch (n) {
        PS_SIZES_B(PS_OPS_ENTRY)
        default: return nullptr;
    }
}

}  // namespace ps
