// FP32 builds of the step: FP32 arithmetic with FP32-stored populations, and
// FP32 arithmetic with FP16-stored populations (FP64 kept for reductions).
#include "lb3e_params.cuh"
#include "lb3e_sim.cuh"

namespace lb3e {
size_t workspace_bytes_f32(const lb3e_params& p) { return Sim<float, float>::layout(p).total; }
SimBase* make_sim_f32(const lb3e_params& p, void* ws, void* stream) {
    return new Sim<float, float>(p, ws, static_cast<cudaStream_t>(stream));
}
size_t workspace_bytes_f16s(const lb3e_params& p) { return Sim<float, __half>::layout(p).total; }
SimBase* make_sim_f16s(const lb3e_params& p, void* ws, void* stream) {
    return new Sim<float, __half>(p, ws, static_cast<cudaStream_t>(stream));
}
}  // namespace lb3e
