// gk_batched_f32.cu -- the batched solver's kernel for f32 operators (one instantiation per
// translation unit, so that the storage types compile in parallel).
#include "gk_batched_kernel.cuh"

namespace gk {

const void *batched_kernel_f32() { return reinterpret_cast<const void *>(&k_batched<float>); }

}  // namespace gk
