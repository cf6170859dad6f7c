// epie_fused_256.cu -- fused ePIE kernel for 256x256 frames: 8 CTA(s) of 512
// threads per frame (see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

cudaError_t launch_fused_256(int itype, const GroupArgs &a, cudaStream_t st) {
  if (itype == 0) return launch_fused_t<256, 8, 512, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<256, 8, 512, __half>(a, st);
  return launch_fused_t<256, 8, 512, float>(a, st);
}

size_t fused_smem_256(int itype) {
  if (itype == 0) return FusedCfg<256, 8, 512, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<256, 8, 512, __half>::SMEM;
  return FusedCfg<256, 8, 512, float>::SMEM;
}

}  // namespace epie
