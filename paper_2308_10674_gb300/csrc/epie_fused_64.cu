// epie_fused_64.cu -- fused ePIE kernel for 64x64 frames: EPIE_CTAS_64 CTAs of
// N*N/(16*CTAs) threads per frame (see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

namespace {
constexpr int CL = EPIE_CTAS_64;
constexpr int NT = 64 * 64 / (CL * 16);
}  // namespace

cudaError_t launch_fused_64(int itype, const GroupArgs &a, cudaStream_t st) {
  if (itype == 0) return launch_fused_t<64, CL, NT, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<64, CL, NT, __half>(a, st);
  return launch_fused_t<64, CL, NT, float>(a, st);
}

size_t fused_smem_64(int itype) {
  if (itype == 0) return FusedCfg<64, CL, NT, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<64, CL, NT, __half>::SMEM;
  return FusedCfg<64, CL, NT, float>::SMEM;
}

}  // namespace epie
