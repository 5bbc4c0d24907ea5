// Imaging kernels for image sides 16 .. 512.
#include "rf_image.cuh"

namespace rf {
RF_INSTANTIATE_IMAGE(16)
RF_INSTANTIATE_IMAGE(32)
RF_INSTANTIATE_IMAGE(64)
RF_INSTANTIATE_IMAGE(128)
RF_INSTANTIATE_IMAGE(256)
RF_INSTANTIATE_IMAGE(512)
}  // namespace rf
