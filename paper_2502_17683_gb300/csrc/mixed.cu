// Placeholder until the tcgen05 path lands: reports the split precisions as unavailable.
#include "mixed.cuh"

namespace thc {
bool mixed_supported() { return false; }
size_t mixed_ws_bytes(int, int, int, int) { return 0; }
void mixed_ws_carve(MixedWs&, Arena&, int, int, int, int) {}
void mixed_project(MixedWs&, cudaStream_t, int, int, int, int, int, const double*, double* const*, const double*, int) {}
void mixed_zgemm(MixedWs&, cudaStream_t, int, int, int, double* const*, int) {}
void mixed_partner(MixedWs&, cudaStream_t, int, int, int, double* const*, int) {}
void mixed_backproject(MixedWs&, cudaStream_t, int, int, int, int, int, double*, int) {}
}  // namespace thc
