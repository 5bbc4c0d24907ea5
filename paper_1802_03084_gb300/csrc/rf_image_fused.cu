// The fused column + row imaging pass for image sides 1024 .. 4096 (2048
// only when its row pass holds 32 values a thread, see RF_ROW_VALUES_2048).
#include "rf_image.cuh"

namespace rf {
RF_INSTANTIATE_FUSED(1024)
#if RF_ROW_VALUES_2048 == 32
RF_INSTANTIATE_FUSED(2048)
#endif
RF_INSTANTIATE_FUSED(4096)
}  // namespace rf
