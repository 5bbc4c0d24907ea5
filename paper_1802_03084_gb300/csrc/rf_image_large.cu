// Imaging kernels for image sides 1024 .. 8192.
#include "rf_image.cuh"

namespace rf {
RF_INSTANTIATE_IMAGE(1024)
RF_INSTANTIATE_IMAGE(2048)
RF_INSTANTIATE_IMAGE(4096)
RF_INSTANTIATE_IMAGE(8192)
}  // namespace rf
