// The fused column + row imaging pass for image sides 1024 .. 4096.
#include "rf_image.cuh"

namespace rf {
RF_INSTANTIATE_FUSED(1024)
RF_INSTANTIATE_FUSED(2048)
RF_INSTANTIATE_FUSED(4096)
}  // namespace rf
