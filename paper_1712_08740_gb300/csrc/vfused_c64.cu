// Fused V(1,1) level kernels instantiated for the complex64 V-cycle on a complex64 basis (MIXED_C64).
#include "vfused.cuh"

namespace helm {

void vfused_attr_c64() { set_attr<float, float2>(); }

HELM_INST_V(float, float2)

}  // namespace helm
