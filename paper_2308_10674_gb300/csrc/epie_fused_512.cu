// epie_fused_512.cu -- fused ePIE kernel for 512x512 frames: 16 CTA(s) of 1024
// threads per frame (see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

cudaError_t launch_fused_512(int itype, const GroupArgs &a, cudaStream_t st) {
  if (itype == 0) return launch_fused_t<512, 16, 1024, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<512, 16, 1024, __half>(a, st);
  return launch_fused_t<512, 16, 1024, float>(a, st);
}

size_t fused_smem_512(int itype) {
  if (itype == 0) return FusedCfg<512, 16, 1024, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<512, 16, 1024, __half>::SMEM;
  return FusedCfg<512, 16, 1024, float>::SMEM;
}

}  // namespace epie
