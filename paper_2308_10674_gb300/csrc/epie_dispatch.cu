// epie_dispatch.cu -- frame-size dispatch of the fused ePIE kernel.
#include "epie_internal.h"

namespace epie {

cudaError_t launch_fused_64(int itype, const GroupArgs &a, cudaStream_t st);
cudaError_t launch_fused_128(int itype, const GroupArgs &a, cudaStream_t st);
cudaError_t launch_fused_256(int itype, const GroupArgs &a, cudaStream_t st);
cudaError_t launch_fused_512(int itype, const GroupArgs &a, cudaStream_t st);
size_t fused_smem_64(int itype);
size_t fused_smem_128(int itype);
size_t fused_smem_256(int itype);
size_t fused_smem_512(int itype);

cudaError_t launch_fused(int N, int itype, const GroupArgs &a, cudaStream_t st) {
  switch (N) {
    case 64: return launch_fused_64(itype, a, st);
    case 128: return launch_fused_128(itype, a, st);
    case 256: return launch_fused_256(itype, a, st);
    case 512: return launch_fused_512(itype, a, st);
    default: return cudaErrorInvalidValue;
  }
}

int fused_ctas_per_frame(int N) {
  switch (N) {
    case 64: return EPIE_CTAS_64;
    case 128: return EPIE_CTAS_128;
    case 256: return EPIE_CTAS_256;
    case 512: return EPIE_CTAS_512;
    default: return 0;
  }
}

size_t fused_smem_bytes(int N, int itype) {
  switch (N) {
    case 64: return fused_smem_64(itype);
    case 128: return fused_smem_128(itype);
    case 256: return fused_smem_256(itype);
    case 512: return fused_smem_512(itype);
    default: return 0;
  }
}

}  // namespace epie
