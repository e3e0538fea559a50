// Device helpers shared by the LDL^T factorisations (blocked and dataflow).
#pragma once
#include <cuda_runtime.h>

namespace thc {

// Reciprocal 1/d of a positive normal double: the hardware's approximate FP64 reciprocal
// (one instruction; measured on this part: relative error below 2^-19 over log-uniform d)
// refined by one third-order Newton step y <- y (1 + e + e^2), e = 1 - d y (cubic
// convergence: 2^-19 -> below 2^-57; measured within 1 ulp of IEEE division over 1.5e8
// samples). Three dependent FP64 operations after the seed. The result is used only for
// d > 0 with 2^-998 < d < 2^998 (the pivot test); other inputs give a discarded value.
__device__ __forceinline__ double recip_nr(double d) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    const double t = fma(-d, y, 1.0);
    const double u = fma(t, t, t);
    return fma(y, u, y);
}

// d > tau with d, tau >= 0 finite-or-not, decided on the integer pipe: non-negative
// doubles order like their bit patterns; NaN / inf / negative fail.
__device__ __forceinline__ bool pivot_ok(double d, double tau) {
    const long long bd = __double_as_longlong(d), bt = __double_as_longlong(tau);
    const bool finite_pos = bd > 0 && bd < 0x7FF0000000000000LL;
    return finite_pos && bd > bt && ((bd >> 52) & 0x7FF) > 24 && ((bd >> 52) & 0x7FF) < 2022;
}

// Pairs (r, s), c < s <= r < N, ordered by s descending: the group of s = N - 1 - k holds
// the k + 1 rows r = s..N-1 and starts at k (k + 1) / 2, so the pairs with s > c form the
// prefix of length (N - 1 - c)(N - c) / 2. Closed-form inverse of the group start (FP32
// sqrt is exact for these small integers; the two checks correct any rounding of the
// estimate).
template <int N>
__device__ __forceinline__ unsigned short pair_code(int e) {
    int k = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    if ((k + 1) * (k + 2) / 2 <= e) ++k;
    if (k * (k + 1) / 2 > e) --k;
    const int s = N - 1 - k;
    const int r = s + (e - k * (k + 1) / 2);
    return (unsigned short)((r << 8) | s);
}

}  // namespace thc
