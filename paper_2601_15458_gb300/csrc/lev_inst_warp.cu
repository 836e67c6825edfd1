// Instantiations of the warp kernel (32 lanes per pair) for both alphabets.
#include "lev_kernels.cuh"

namespace msa {
#define WARPK(WPL, A, B, S) {1, WPL, A, ((WPL) * (S) * 32 + 3 * kRing + 2) * sizeof(uint32_t), launch_warp<WPL, B, S>, (const void *)lev_warp_kernel<WPL, B, S>}
const LevKernelInfo kLevWarpDna[] = {WARPK(1, MSA_DNA, 2, 4),  WARPK(2, MSA_DNA, 2, 4),  WARPK(3, MSA_DNA, 2, 4),
                                     WARPK(4, MSA_DNA, 2, 4),  WARPK(5, MSA_DNA, 2, 4),  WARPK(6, MSA_DNA, 2, 4),
                                     WARPK(8, MSA_DNA, 2, 4),  WARPK(10, MSA_DNA, 2, 4), WARPK(12, MSA_DNA, 2, 4),
                                     WARPK(16, MSA_DNA, 2, 4)};
const int kLevWarpDnaCount = sizeof(kLevWarpDna) / sizeof(kLevWarpDna[0]);
const LevKernelInfo kLevWarpProt[] = {WARPK(1, MSA_PROTEIN, 5, 20), WARPK(2, MSA_PROTEIN, 5, 20),
                                      WARPK(3, MSA_PROTEIN, 5, 20), WARPK(4, MSA_PROTEIN, 5, 20),
                                      WARPK(5, MSA_PROTEIN, 5, 20), WARPK(6, MSA_PROTEIN, 5, 20),
                                      WARPK(8, MSA_PROTEIN, 5, 20), WARPK(10, MSA_PROTEIN, 5, 20),
                                      WARPK(12, MSA_PROTEIN, 5, 20), WARPK(16, MSA_PROTEIN, 5, 20)};
const int kLevWarpProtCount = sizeof(kLevWarpProt) / sizeof(kLevWarpProt[0]);
}  // namespace msa
