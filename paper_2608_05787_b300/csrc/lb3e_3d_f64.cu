// FP64 build of the three-dimensional (D3Q15) step: compiled with --fmad=false, so
// every multiply and add rounds separately, as in a plain C evaluation.
#include "lb3e_3d.cuh"

namespace lb3e {
size_t workspace_bytes_3d_f64(const lb3e_params& p) { return Sim3<double>::layout(p).total; }
SimBase* make_sim_3d_f64(const lb3e_params& p, void* ws, void* stream) {
    return new Sim3<double>(p, ws, static_cast<cudaStream_t>(stream));
}
}  // namespace lb3e
