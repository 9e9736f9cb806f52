// Fused V(1,1) level kernels instantiated for the complex64 V-cycle on a complex128 basis (MIXED).
#include "vfused.cuh"

namespace helm {

void vfused_attr_mixed() { set_attr<float, double2>(); }

HELM_INST_V(float, double2)

}  // namespace helm
