// epie_fused_128.cu -- fused ePIE kernel for 128x128 frames: EPIE_CTAS_128 CTAs of
// N*N/(16*CTAs) threads per frame (see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

namespace {
constexpr int CL = EPIE_CTAS_128;
constexpr int NT = 128 * 128 / (CL * 16);
}  // namespace

cudaError_t launch_fused_128(int itype, const GroupArgs &a, cudaStream_t st) {
  if (itype == 0) return launch_fused_t<128, CL, NT, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<128, CL, NT, __half>(a, st);
  return launch_fused_t<128, CL, NT, float>(a, st);
}

size_t fused_smem_128(int itype) {
  if (itype == 0) return FusedCfg<128, CL, NT, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<128, CL, NT, __half>::SMEM;
  return FusedCfg<128, CL, NT, float>::SMEM;
}

}  // namespace epie
