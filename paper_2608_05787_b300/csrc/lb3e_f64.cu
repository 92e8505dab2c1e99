// FP64 build of the step: compiled with --fmad=false, so every multiply and add
// rounds separately, as in a plain C evaluation of the same formulas.
#include "lb3e_params.cuh"
#include "lb3e_sim.cuh"

namespace lb3e {
size_t workspace_bytes_f64(const lb3e_params& p) { return Sim<double, double>::layout(p).total; }
SimBase* make_sim_f64(const lb3e_params& p, void* ws, void* stream) {
    return new Sim<double, double>(p, ws, static_cast<cudaStream_t>(stream));
}
size_t batch_bytes_f64(const lb3e_params* ps, int n) { return Batch<double, double>::bytes(ps, n); }
BatchBase* new_batch_f64(const lb3e_params* ps, int n, void* ws, void* stream) {
    return new Batch<double, double>(ps, n, ws, static_cast<cudaStream_t>(stream));
}
int init_batch_f64(BatchBase* b, const double* const* phis) { return static_cast<Batch<double, double>*>(b)->init(phis); }
}  // namespace lb3e
