// epie_dispatch.cu -- frame-size dispatch of the fused ePIE kernel.
#include "epie_internal.h"

namespace epie {

cudaError_t launch_fused_64(int itype, const GroupArgs &a, cudaStream_t st);
cudaError_t launch_fused_128(int itype, const GroupArgs &a, cudaStream_t st, int cl);
cudaError_t launch_fused_256(int itype, const GroupArgs &a, cudaStream_t st);
cudaError_t launch_fused_512(int itype, const GroupArgs &a, cudaStream_t st);
size_t fused_smem_64(int itype);
size_t fused_smem_128(int itype);
size_t fused_smem_256(int itype);
size_t fused_smem_512(int itype);

cudaError_t launch_fused(int N, int itype, const GroupArgs &a, cudaStream_t st, int cl) {
  if (fused_ctas_per_frame(N, cl) == 0) return cudaErrorInvalidValue;
  switch (N) {
    case 64: return launch_fused_64(itype, a, st);
    case 128: return launch_fused_128(itype, a, st, cl);
    case 256: return launch_fused_256(itype, a, st);
    case 512: return launch_fused_512(itype, a, st);
    default: return cudaErrorInvalidValue;
  }
}

int fused_ctas_per_frame(int N, int cl) {
  switch (N) {
    case 64: return cl == 0 || cl == EPIE_CTAS_64 ? EPIE_CTAS_64 : 0;
    case 128: return cl == 0 ? EPIE_CTAS_128 : (cl == 1 || cl == 2 || cl == 4 ? cl : 0);
    case 256: return cl == 0 || cl == EPIE_CTAS_256 ? EPIE_CTAS_256 : 0;
    case 512: return cl == 0 || cl == EPIE_CTAS_512 ? EPIE_CTAS_512 : 0;
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
