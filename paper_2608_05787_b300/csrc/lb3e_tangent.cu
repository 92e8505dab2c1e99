// Tangent (forward-mode) builds of the step: arithmetic on dual numbers, FP32
// with three derivative directions (precision 3) and FP64 with one (precision 4,
// a validation build: three FP64 directions would need 96 KB of static shared
// memory in the fused tile).  The kernels are the same templates as the plain builds.
#include "lb3e_params.cuh"
#include "lb3e_sim.cuh"

namespace lb3e {
using D3f = Dual<float, 3>;
using D1d = Dual<double, 1>;
size_t workspace_bytes_t32(const lb3e_params& p) { return Sim<D3f, D3f>::layout(p).total; }
SimBase* make_sim_t32(const lb3e_params& p, void* ws, void* stream) {
    return new Sim<D3f, D3f>(p, ws, static_cast<cudaStream_t>(stream));
}
size_t workspace_bytes_t64(const lb3e_params& p) { return Sim<D1d, D1d>::layout(p).total; }
SimBase* make_sim_t64(const lb3e_params& p, void* ws, void* stream) {
    return new Sim<D1d, D1d>(p, ws, static_cast<cudaStream_t>(stream));
}
}  // namespace lb3e
