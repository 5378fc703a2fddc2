// gk_batched_f16.cu -- the batched solver's kernel for f16 operators (one instantiation per
// translation unit, so that the storage types compile in parallel).
#include "gk_batched_kernel.cuh"

namespace gk {

const void *batched_kernel_f16() { return reinterpret_cast<const void *>(&k_batched<__half>); }

}  // namespace gk
