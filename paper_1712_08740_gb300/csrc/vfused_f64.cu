// Fused V(1,1) level kernels instantiated for the complex128 V-cycle (precision F64).
#include "vfused.cuh"

namespace helm {

void vfused_attr_f64() { set_attr<double, double2>(); }

HELM_INST_V(double, double2)

}  // namespace helm
