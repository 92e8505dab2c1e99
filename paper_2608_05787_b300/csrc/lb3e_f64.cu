// FP64 build of the step: compiled with --fmad=false, so every multiply and add
// rounds separately, as in a plain C evaluation of the same formulas.
#include "lb3e_params.cuh"
#include "lb3e_sim.cuh"

namespace lb3e {
size_t workspace_bytes_f64(const lb3e_params& p) { return Sim<double, double>::layout(p).total; }
SimBase* make_sim_f64(const lb3e_params& p, void* ws, void* stream) {
    return new Sim<double, double>(p, ws, static_cast<cudaStream_t>(stream));
}
}  // namespace lb3e
