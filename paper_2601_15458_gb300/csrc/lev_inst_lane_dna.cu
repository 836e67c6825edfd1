// Instantiations of the lane kernel for DNA (2 bit planes, 4 symbols).
#include "lev_kernels.cuh"

namespace msa {
#define LANE(WC) {0, WC, MSA_DNA, lane_peq_stride(WC) * 4 * sizeof(uint32_t), launch_lane<WC, 2, 4>, (const void *)lev_lane_kernel<WC, 2, 4>}
const LevKernelInfo kLevLaneDna[] = {LANE(1),  LANE(2),  LANE(3),  LANE(4),  LANE(5),  LANE(6),
                                     LANE(8),  LANE(10), LANE(12), LANE(14), LANE(16), LANE(20),
                                     LANE(24), LANE(28), LANE(32), LANE(36), LANE(40), LANE(44),
                                     LANE(48), LANE(52), LANE(56), LANE(60), LANE(64)};
const int kLevLaneDnaCount = sizeof(kLevLaneDna) / sizeof(kLevLaneDna[0]);
}  // namespace msa
