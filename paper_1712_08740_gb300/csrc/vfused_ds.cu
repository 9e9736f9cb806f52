// Fused V(1,1) level kernels instantiated for the complex64 V-cycle on a double-single basis (MIXED_DS).
#include "vfused.cuh"

namespace helm {

void vfused_attr_ds() { set_attr<float, float4>(); }

HELM_INST_V(float, float4)

}  // namespace helm
