// gk_batched_bf16.cu -- the batched solver's kernel for bf16 operators (one instantiation per
// translation unit, so that the storage types compile in parallel).
#include "gk_batched_kernel.cuh"

namespace gk {

const void *batched_kernel_bf16() { return reinterpret_cast<const void *>(&k_batched<__nv_bfloat16>); }

}  // namespace gk
