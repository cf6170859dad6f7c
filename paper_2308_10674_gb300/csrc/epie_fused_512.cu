// epie_fused_512.cu -- fused ePIE kernel for 512x512 frames: EPIE_CTAS_512 CTAs of
// N*N/(16*CTAs) threads per frame (see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

namespace {
constexpr int CL = EPIE_CTAS_512;
constexpr int NT = 512 * 512 / (CL * 16);
}  // namespace

cudaError_t launch_fused_512(int itype, const GroupArgs &a, cudaStream_t st) {
  if (itype == 0) return launch_fused_t<512, CL, NT, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<512, CL, NT, __half>(a, st);
  return launch_fused_t<512, CL, NT, float>(a, st);
}

size_t fused_smem_512(int itype) {
  if (itype == 0) return FusedCfg<512, CL, NT, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<512, CL, NT, __half>::SMEM;
  return FusedCfg<512, CL, NT, float>::SMEM;
}

}  // namespace epie
