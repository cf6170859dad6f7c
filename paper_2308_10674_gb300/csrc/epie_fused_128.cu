// epie_fused_128.cu -- fused ePIE kernel for 128x128 frames in three tile
// shapes: 1, 2 (the default) or 4 CTAs per frame, each thread holding 16
// values (1024, 512 or 256 threads per CTA; see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

namespace {
template <int CL>
cudaError_t launch_cl(int itype, const GroupArgs &a, cudaStream_t st) {
  constexpr int NT = 128 * 128 / (CL * 16);
  if (itype == 0) return launch_fused_t<128, CL, NT, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<128, CL, NT, __half>(a, st);
  return launch_fused_t<128, CL, NT, float>(a, st);
}
}  // namespace

cudaError_t launch_fused_128(int itype, const GroupArgs &a, cudaStream_t st, int cl) {
  switch (cl == 0 ? EPIE_CTAS_128 : cl) {
    case 1: return launch_cl<1>(itype, a, st);
    case 2: return launch_cl<2>(itype, a, st);
    case 4: return launch_cl<4>(itype, a, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t fused_smem_128(int itype) {
  constexpr int CL = EPIE_CTAS_128, NT = 128 * 128 / (CL * 16);
  if (itype == 0) return FusedCfg<128, CL, NT, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<128, CL, NT, __half>::SMEM;
  return FusedCfg<128, CL, NT, float>::SMEM;
}

}  // namespace epie
