// FP32 builds of the step: FP32 arithmetic with FP32-stored populations, and
// FP32 arithmetic with FP16- or BF16-stored populations (FP64 kept for reductions).
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
size_t batch_bytes_f32(const lb3e_params* ps, int n) { return Batch<float, float>::bytes(ps, n); }
BatchBase* new_batch_f32(const lb3e_params* ps, int n, void* ws, void* stream) {
    return new Batch<float, float>(ps, n, ws, static_cast<cudaStream_t>(stream));
}
int init_batch_f32(BatchBase* b, const double* const* phis) { return static_cast<Batch<float, float>*>(b)->init(phis); }
size_t batch_bytes_f16s(const lb3e_params* ps, int n) { return Batch<float, __half>::bytes(ps, n); }
BatchBase* new_batch_f16s(const lb3e_params* ps, int n, void* ws, void* stream) {
    return new Batch<float, __half>(ps, n, ws, static_cast<cudaStream_t>(stream));
}
int init_batch_f16s(BatchBase* b, const double* const* phis) { return static_cast<Batch<float, __half>*>(b)->init(phis); }
size_t workspace_bytes_bf16s(const lb3e_params& p) { return Sim<float, __nv_bfloat16>::layout(p).total; }
SimBase* make_sim_bf16s(const lb3e_params& p, void* ws, void* stream) {
    return new Sim<float, __nv_bfloat16>(p, ws, static_cast<cudaStream_t>(stream));
}
size_t batch_bytes_bf16s(const lb3e_params* ps, int n) { return Batch<float, __nv_bfloat16>::bytes(ps, n); }
BatchBase* new_batch_bf16s(const lb3e_params* ps, int n, void* ws, void* stream) {
    return new Batch<float, __nv_bfloat16>(ps, n, ws, static_cast<cudaStream_t>(stream));
}
int init_batch_bf16s(BatchBase* b, const double* const* phis) {
    return static_cast<Batch<float, __nv_bfloat16>*>(b)->init(phis);
}
}  // namespace lb3e
