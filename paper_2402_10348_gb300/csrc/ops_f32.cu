// Float32 instantiations of the element operators (the FSI_FP32 path used inside
// mixed-precision iterative refinement).
#include "ops_impl.cuh"

namespace fsi {

template int launch_ns<float>(fsi_mesh*, int, const double*, double*, unsigned);
template int launch_nsq<float>(fsi_mesh*, const double*, double*, unsigned);
template int launch_ac<float>(fsi_mesh*, int, int, const double*, double*);
template int launch_b<float>(fsi_mesh*, int, int, const double*, double*);

}  // namespace fsi
