// FP32 build of the three-dimensional (D3Q15) step.
#include "lb3e_3d.cuh"

namespace lb3e {
size_t workspace_bytes_3d_f32(const lb3e_params& p) { return Sim3<float>::layout(p).total; }
SimBase* make_sim_3d_f32(const lb3e_params& p, void* ws, void* stream) {
    return new Sim3<float>(p, ws, static_cast<cudaStream_t>(stream));
}
}  // namespace lb3e
