// Instantiations of the lane kernel with kLevSlots queries per warp, protein (5 bit planes, 20 symbols).
#include "lev_kernels.cuh"

namespace msa {
#define SLOT(WC)                                                                                                 \
    {0, WC, MSA_PROTEIN, lane_smem_words(WC, 20, kLevSlots) * sizeof(uint32_t), launch_lane<WC, 5, 20, kLevSlots>, \
     (const void *)lev_lane_kernel<WC, 5, 20, kLevSlots>}
const LevKernelInfo kLevSlotProt[] = {SLOT(1),  SLOT(2),  SLOT(3),  SLOT(4),  SLOT(5),  SLOT(6),
                                     SLOT(8),  SLOT(10), SLOT(12), SLOT(14), SLOT(16), SLOT(20),
                                     SLOT(24), SLOT(28), SLOT(32), SLOT(36), SLOT(40), SLOT(44),
                                     SLOT(48), SLOT(52), SLOT(56), SLOT(60), SLOT(64)};
const int kLevSlotProtCount = sizeof(kLevSlotProt) / sizeof(kLevSlotProt[0]);
}  // namespace msa
