// Instantiations of the lane kernel with kLevSlots queries per warp, DNA (2 bit planes, 4 symbols).
#include "lev_kernels.cuh"

namespace msa {
#define SLOT(WC)                                                                                                 \
    {0, WC, MSA_DNA, lane_smem_words(WC, 4, kLevSlots) * sizeof(uint32_t), launch_lane<WC, 2, 4, kLevSlots>, \
     (const void *)lev_lane_kernel<WC, 2, 4, kLevSlots>}
const LevKernelInfo kLevSlotDna[] = {SLOT(1),  SLOT(2),  SLOT(3),  SLOT(4),  SLOT(5),  SLOT(6),
                                     SLOT(8),  SLOT(10), SLOT(12), SLOT(14), SLOT(16), SLOT(20),
                                     SLOT(24), SLOT(28), SLOT(32), SLOT(36), SLOT(40), SLOT(44),
                                     SLOT(48), SLOT(52), SLOT(56), SLOT(60), SLOT(64)};
const int kLevSlotDnaCount = sizeof(kLevSlotDna) / sizeof(kLevSlotDna[0]);
}  // namespace msa
