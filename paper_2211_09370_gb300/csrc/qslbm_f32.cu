// FP32 instantiation of the qslbm kernels and launchers.
#include "qslbm_launch.cuh"

namespace qslbm {
const Ops& ops_f32() { return Launch<float>::table(); }
}  // namespace qslbm
