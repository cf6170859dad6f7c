// epie_fused_256.cu -- fused ePIE kernel for 256x256 frames: EPIE_CTAS_256 CTAs of
// N*N/(16*CTAs) threads per frame (see epie_fused.cuh).
#include "epie_fused.cuh"

namespace epie {

namespace {
constexpr int CL = EPIE_CTAS_256;
constexpr int NT = 256 * 256 / (CL * 16);
}  // namespace

cudaError_t launch_fused_256(int itype, const GroupArgs &a, cudaStream_t st) {
  if (itype == 0) return launch_fused_t<256, CL, NT, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<256, CL, NT, __half>(a, st);
  return launch_fused_t<256, CL, NT, float>(a, st);
}

size_t fused_smem_256(int itype) {
  if (itype == 0) return FusedCfg<256, CL, NT, uint16_t>::SMEM;
  if (itype == 1) return FusedCfg<256, CL, NT, __half>::SMEM;
  return FusedCfg<256, CL, NT, float>::SMEM;
}

}  // namespace epie

#ifdef EPIE_PHASE_CLOCKS
// profiling builds: copy the per-CTA phase clocks of the last launch to the host
extern "C" __attribute__((visibility("default"))) int epie_read_phase_clocks(long long *host,
                                                                            int n_ctas) {
  return static_cast<int>(
      cudaMemcpyFromSymbol(host, epie::g_phase_clocks, sizeof(long long) * 16 * n_ctas));
}
#endif
