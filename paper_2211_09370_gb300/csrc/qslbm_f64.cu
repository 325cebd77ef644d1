// FP64 instantiation of the qslbm kernels and launchers.
#include "qslbm_launch.cuh"

namespace qslbm {
const Ops& ops_f64() { return Launch<double>::table(); }
}  // namespace qslbm
