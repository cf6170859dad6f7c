// epie_fused_64.cu -- fused ePIE kernel for 64x64 frames: 1 CTA(s) of 256
// threads per frame (see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

cudaError_t launch_fused_64(int itype, const GroupArgs &a, cudaStream_t st) {
  if (itype == 0) return launch_fused_t<64, 1, 256, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<64, 1, 256, __half>(a, st);
  return launch_fused_t<64, 1, 256, float>(a, st);
}

size_t fused_smem_64(int itype) {
  if (itype == 0) return FusedCfg<64, 1, 256, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<64, 1, 256, __half>::SMEM;
  return FusedCfg<64, 1, 256, float>::SMEM;
}

}  // namespace epie
