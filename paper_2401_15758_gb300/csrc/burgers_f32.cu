// FP32 instantiations of the Burgers sweeps (see burgers_impl.cuh).
#include "burgers_impl.cuh"

namespace sc4 {
template int burgers_tlm<float>(const ModelGeom&, const float*, const float*, int, int, float*, int,
                                cudaStream_t);
template int burgers_adj<float>(const ModelGeom&, const float*, const float*, int, int, float*, int,
                                cudaStream_t);
}  // namespace sc4
