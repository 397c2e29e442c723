// FP64 instantiations of the Burgers sweeps (see burgers_impl.cuh).
#include "burgers_impl.cuh"

namespace sc4 {
template int burgers_fwd<double>(const ModelGeom&, const double*, double*, float*, const double*,
                                 double*, double*, double*, cudaStream_t);
template int burgers_tlm<double>(const ModelGeom&, const double*, const double*, int, int, double*,
                                 int, cudaStream_t);
template int burgers_adj<double>(const ModelGeom&, const double*, const double*, int, int, double*,
                                 int, cudaStream_t);
}  // namespace sc4
