// gk_batched_f64.cu -- the batched solver's kernel for f64 operators (one instantiation per
// translation unit, so that the storage types compile in parallel).
#include "gk_batched_kernel.cuh"

namespace gk {

const void *batched_kernel_f64() { return reinterpret_cast<const void *>(&k_batched<double>); }

}  // namespace gk
