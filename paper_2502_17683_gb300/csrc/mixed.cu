// Split-precision MTTKRP orchestration on the tcgen05 GEMM (see mixed.cuh).
#include <algorithm>

#include "mixed.cuh"
#include "prof.cuh"

namespace thc {

bool mixed_supported() { return tc_available(); }

namespace {
constexpr int kBackSplits = 10;  // at most this many K slices in the back-projection
size_t split_bytes(bool tf32, int rows, int cols) {
    return 2 * Arena::need<uint8_t>((size_t)rows * split_pitch(tf32, cols) * (tf32 ? 4 : 2));
}
void carve_split(Arena& ar, bool tf32, SplitMat& m, int rows, int cols) {
    const int pitch = split_pitch(tf32, cols);
    const size_t bytes = (size_t)rows * pitch * (tf32 ? 4 : 2);
    m.hi = ar.take<uint8_t>(bytes);
    m.lo = ar.take<uint8_t>(bytes);
    m.rows = rows;
    m.cols = cols;
    m.pitch = pitch;
}
}  // namespace

size_t mixed_ws_bytes(bool tf32, int o, int v, int Rt, int R) {
    size_t b = 0;
    b += 2 * split_bytes(tf32, Rt, Rt);
    b += split_bytes(tf32, Rt, o) + split_bytes(tf32, Rt, v);
    b += split_bytes(tf32, o, Rt) + split_bytes(tf32, v, Rt);
    b += 2 * split_bytes(tf32, R, o) + 2 * split_bytes(tf32, R, v);
    b += 2 * split_bytes(tf32, R, Rt);
    b += 5 * Arena::need<float>((size_t)R * Rt);
    b += Arena::need<double>((size_t)kBackSplits * std::max(o, v) * R);
    return b;
}

void mixed_ws_carve(MixedWs& mx, Arena& ar, bool tf32, int o, int v, int Rt, int R) {
    mx.tf32 = tf32;
    mx.o = o;
    mx.v = v;
    mx.Rt = Rt;
    mx.R = R;
    carve_split(ar, tf32, mx.Zs, Rt, Rt);
    carve_split(ar, tf32, mx.ZTs, Rt, Rt);
    carve_split(ar, tf32, mx.XT[0], Rt, o);
    carve_split(ar, tf32, mx.XT[1], Rt, v);
    carve_split(ar, tf32, mx.Xs[0], o, Rt);
    carve_split(ar, tf32, mx.Xs[1], v, Rt);
    carve_split(ar, tf32, mx.At[0], R, o);
    carve_split(ar, tf32, mx.At[1], R, v);
    carve_split(ar, tf32, mx.At[2], R, o);
    carve_split(ar, tf32, mx.At[3], R, v);
    carve_split(ar, tf32, mx.Pt, R, Rt);
    carve_split(ar, tf32, mx.Et, R, Rt);
    for (int k = 0; k < 4; ++k) mx.Wt[k] = ar.take<float>((size_t)R * Rt);
    mx.Yf = ar.take<float>((size_t)R * Rt);
    mx.part_cap = (size_t)kBackSplits * std::max(o, v) * R;
    mx.part = ar.take<double>(mx.part_cap);
}

cudaError_t mixed_setup(MixedWs& mx, cudaStream_t st, const double* Xo, const double* Xv,
                        const double* Z) {
    const bool t = mx.tf32;
    const int Rt = mx.Rt;
    split_rows(st, t, Z, Rt, Rt, Rt, mx.Zs);
    split_transpose(st, t, Z, Rt, Rt, Rt, mx.ZTs);
    split_transpose(st, t, Xo, Rt, mx.o, Rt, mx.XT[0]);
    split_transpose(st, t, Xv, Rt, mx.v, Rt, mx.XT[1]);
    split_rows(st, t, Xo, Rt, mx.o, Rt, mx.Xs[0]);
    split_rows(st, t, Xv, Rt, mx.v, Rt, mx.Xs[1]);
    return cudaGetLastError();
}

cudaError_t mixed_project(MixedWs& mx, cudaStream_t st, int k, const double* Ak, bool in_sweep) {
    const int n = (k % 2 == 0) ? mx.o : mx.v;
    split_transpose(st, mx.tf32, Ak, mx.R, n, mx.R, mx.At[k]);
    TcEpilogue ep;
    ep.out_f32 = mx.Wt[k];
    ep.ld_f32 = mx.Rt;
    if (k == 1 || k == 3) {  // P = W_{k-1} o W_k for the next Z-GEMM
        ep.mul = mx.Wt[k - 1];
        ep.ld_mul = mx.Rt;
        ep.out_split = &mx.Pt;
    } else if (in_sweep) {  // E = W_k o Y for the partner mode's back-projection
        ep.mul = mx.Yf;
        ep.ld_mul = mx.Rt;
        ep.out_split = &mx.Et;
    }
    return tc_gemm(st, mx.tf32, mx.At[k], mx.XT[k % 2], mx.R, mx.Rt, n, ep);
}

cudaError_t mixed_zgemm(MixedWs& mx, cudaStream_t st, int half) {
    TcEpilogue ep;
    ep.prof_class = KC_TCZ;
    ep.out_f32 = mx.Yf;
    ep.ld_f32 = mx.Rt;
    ep.mul = half == 0 ? mx.Wt[1] : mx.Wt[3];
    ep.ld_mul = mx.Rt;
    ep.out_split = &mx.Et;
    return tc_gemm(st, mx.tf32, mx.Pt, half == 0 ? mx.Zs : mx.ZTs, mx.R, mx.Rt, mx.Rt, ep);
}

cudaError_t mixed_partner(MixedWs& mx, cudaStream_t st, int mode) {
    const float* w = mode == 1 ? mx.Wt[0] : mx.Wt[2];
    split_hadamard(st, mx.tf32, w, mx.Yf, mx.Rt, mx.R, mx.Rt, mx.Et);
    return cudaGetLastError();
}

cudaError_t mixed_backproject(MixedWs& mx, cudaStream_t st, int k, double* M) {
    const int n = (k % 2 == 0) ? mx.o : mx.v;
    TcEpilogue ep;
    ep.out_f64t = M;
    ep.ld_f64t = mx.R;
    return tc_gemm(st, mx.tf32, mx.Et, mx.Xs[k % 2], mx.R, n, mx.Rt, ep, mx.part, mx.part_cap);
}

int mixed_take_error() { return tc_take_error(); }

}  // namespace thc
