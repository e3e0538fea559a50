// Split-precision (BF16x3 / TF32x3) MTTKRP on tcgen05 tensor cores: launchers.
#pragma once
#include "common.cuh"

namespace thc {

struct MixedWs {
    int ready = 0;
};

bool mixed_supported();
size_t mixed_ws_bytes(int o, int v, int Rt, int R);
void mixed_ws_carve(MixedWs& mx, Arena& ar, int o, int v, int Rt, int R);
void mixed_project(MixedWs& mx, cudaStream_t st, int o, int v, int Rt, int R, int k,
                   const double* Ak, double* const* W, const double* Y, int prec);
void mixed_zgemm(MixedWs& mx, cudaStream_t st, int Rt, int R, int half, double* const* W, int prec);
void mixed_partner(MixedWs& mx, cudaStream_t st, int Rt, int R, int mode, double* const* W, int prec);
void mixed_backproject(MixedWs& mx, cudaStream_t st, int o, int v, int Rt, int R, int k,
                       double* M, int prec);

}  // namespace thc
