// epie_fused_128.cu -- fused ePIE kernel for 128x128 frames: 2 CTA(s) of 512
// threads per frame (see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

cudaError_t launch_fused_128(int itype, const GroupArgs &a, cudaStream_t st) {
  if (itype == 0) return launch_fused_t<128, 2, 512, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<128, 2, 512, __half>(a, st);
  return launch_fused_t<128, 2, 512, float>(a, st);
}

size_t fused_smem_128(int itype) {
  if (itype == 0) return FusedCfg<128, 2, 512, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<128, 2, 512, __half>::SMEM;
  return FusedCfg<128, 2, 512, float>::SMEM;
}

}  // namespace epie
