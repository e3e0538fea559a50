// tcgen05 split-operand GEMM for sm_103a (see tc_gemm.cuh).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>

#include "common.cuh"
#include "prof.cuh"
#include "tc_gemm.cuh"
#include "tcgen05.cuh"

namespace thc {

__device__ int g_tc_error = 0;

namespace {

constexpr int BM = 128;             // MMA M (one CTA, cta_group::1)
constexpr int KBYTES = 128;         // bytes of K per stage (one 128-byte swizzle atom)
constexpr int TILE_A = BM * KBYTES;  // 16 KB
constexpr int ACC_COLS = 256;        // one FP32 accumulator (tile N <= 256)
constexpr int TMEM_COLS = 2 * ACC_COLS;  // two: the epilogue drains one while the next fills
constexpr int EPI_WARPS = 8;       // two per TMEM lane quarter, alternate 16-column slices
constexpr int EPI_PITCH = 20;      // floats per staged row (16 + 4: 16-byte rows, no conflicts)
constexpr int EPI_STAGE_BYTES = EPI_WARPS * 32 * EPI_PITCH * 4;
constexpr uint32_t WAIT_LIMIT = 1u << 22;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;  // warp 0: TMA, warp 1: MMA + TMEM, then epilogue

// Bounded wait: records `code` in the error word and returns false when it gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int code) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(&g_tc_error, code);
    return false;
}

struct KArgs {
    int M, N, nkb, BN, stages;
    int tn, tm, ntiles;  // tiles along N and M, and tn x tm x K splits in all
    int kper;          // k-blocks per tile along the K split (split-K of the FP64-out epilogue)
    double* part;      // split-K partials [z][N][ld_f64t] (when gridDim.z > 1)
    TcEpilogue ep;
    void* out_hi;
    void* out_lo;
    int ld_split;
    int vec;           // bit 0: out_f32, bit 1: mul, bit 2: split outputs take 16-/8-byte vectors
};

template <bool TF32>
__device__ __forceinline__ void store_split(void* hi, void* lo, size_t idx, float x) {
    if (TF32) {
        // round to the 10-bit TF32 mantissa (nearest, ties away), residual likewise
        const uint32_t u = __float_as_uint(x);
        const float h = __uint_as_float((u + 0x1000u) & 0xFFFFE000u);
        const float r = x - h;
        const uint32_t ur = __float_as_uint(r);
        const float l = __uint_as_float((ur + 0x1000u) & 0xFFFFE000u);
        ((float*)hi)[idx] = h;
        ((float*)lo)[idx] = l;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        ((__nv_bfloat16*)hi)[idx] = h;
        ((__nv_bfloat16*)lo)[idx] = l;
    }
}

// Four consecutive outputs split(e) at idx .. idx + lim - 1 (lim < 4 at the column tail); one
// vector store per half when `vec` (16 bytes TF32, 8 bytes BF16).
template <bool TF32>
__device__ __forceinline__ void store_split4(void* hi, void* lo, size_t idx, const float4& e,
                                             bool vec, int lim) {
    const float x[4] = {e.x, e.y, e.z, e.w};
    if (vec && lim >= 4) {
        if (TF32) {
            float h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t b = __float_as_uint(x[u]);
                h[u] = __uint_as_float((b + 0x1000u) & 0xFFFFE000u);
                const uint32_t br = __float_as_uint(x[u] - h[u]);
                l[u] = __uint_as_float((br + 0x1000u) & 0xFFFFE000u);
            }
            *(float4*)((float*)hi + idx) = make_float4(h[0], h[1], h[2], h[3]);
            *(float4*)((float*)lo + idx) = make_float4(l[0], l[1], l[2], l[3]);
        } else {
            __nv_bfloat16 h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                h[u] = __float2bfloat16_rn(x[u]);
                l[u] = __float2bfloat16_rn(x[u] - __bfloat162float(h[u]));
            }
            uint2 ph, pl;
            ph.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
            ph.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
            pl.x = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
            pl.y = (uint32_t)__bfloat16_as_ushort(l[2]) | ((uint32_t)__bfloat16_as_ushort(l[3]) << 16);
            *(uint2*)((__nv_bfloat16*)hi + idx) = ph;
            *(uint2*)((__nv_bfloat16*)lo + idx) = pl;
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < lim) store_split<TF32>(hi, lo, idx + u, x[u]);
    }
}

// Persistent split GEMM: each CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... of the
// (N tile, M tile, K split) grid. Warp 0 streams the operand tiles through the TMA ring
// without stopping between tiles; warp 1 issues the MMAs of tile i into TMEM accumulator
// i & 1 and commits it; the eight epilogue warps drain accumulator i & 1 while the MMAs of
// tile i + 1 run into the other one, then release it. An epilogue warp reads 32 rows x 16
// columns from TMEM (one row per lane) and, for the row-major outputs, restages them in
// shared memory so that each lane holds 4 consecutive columns of 4 rows: partner loads and
// output stores are then 16-byte (8-byte for BF16 halves) vectors, 8 rows per instruction.
// Every wait is bounded and records a code when it gives up.
template <bool TF32>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
          const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
          const KArgs args) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment for the swizzled tiles
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int BN = args.BN, S = args.stages;
    const int tileB = BN * KBYTES;
    const int stage_bytes = 2 * TILE_A + 2 * tileB;
    float* epi = (float*)(smem + (size_t)S * stage_bytes);
    uint64_t* full = (uint64_t*)((uint8_t*)epi + EPI_STAGE_BYTES);
    uint64_t* empty = full + S;
    uint64_t* acc_full = empty + S;   // [2]
    uint64_t* acc_empty = acc_full + 2;  // [2]
    uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kel = TF32 ? 32 : 64;  // elements per 128-byte K block
    const int tnm = args.tn * args.tm;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS);  // one arrive per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer ----
        const uint32_t tx = (uint32_t)stage_bytes;
        int it = 0;  // position in the ring, over all tiles of this CTA
        bool ok = true;
        for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x) {
            const int z = t / tnm, r = t % tnm, m0 = (r / args.tn) * BM, n0 = (r % args.tn) * BN;
            const int kb0 = z * args.kper, nk = min(args.nkb, kb0 + args.kper) - kb0;
            for (int kb = 0; kb < nk; ++kb, ++it) {
                const int s = it % S;
                if (!mbar_wait(&empty[s], ((it / S) & 1) ^ 1, 1)) {
                    ok = false;
                    break;
                }
                uint8_t* st = smem + (size_t)s * stage_bytes;
                const int kx = (kb0 + kb) * kel;
                mbar_expect_tx(&full[s], tx);
                tma_load_2d(st, &tAh, &full[s], kx, m0);
                tma_load_2d(st + TILE_A, &tAl, &full[s], kx, m0);
                tma_load_2d(st + 2 * TILE_A, &tBh, &full[s], kx, n0);
                tma_load_2d(st + 2 * TILE_A + tileB, &tBl, &full[s], kx, n0);
            }
        }
        // drain: wait until the MMAs released every stage still in flight
        for (int j = max(0, it - S); j < it; ++j) mbar_wait(&empty[j % S], (j / S) & 1, 2);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        const uint32_t idesc = make_idesc(TF32, BM, BN);
        int it = 0, i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x, ++i) {
            const int z = t / tnm;
            const int kb0 = z * args.kper, nk = min(args.nkb, kb0 + args.kper) - kb0;
            const int b = i & 1;
            // accumulator b is free once the epilogue has drained tile i - 2
            if (i >= 2 && !mbar_wait(&acc_empty[b], ((i >> 1) - 1) & 1, 5)) break;
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)(b * ACC_COLS);
            for (int kb = 0; kb < nk; ++kb, ++it) {
                const int s = it % S;
                if (!mbar_wait(&full[s], (it / S) & 1, 3)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint8_t* st = smem + (size_t)s * stage_bytes;
                const uint64_t ah = sw128_desc(smem_u32(st));
                const uint64_t al = sw128_desc(smem_u32(st + TILE_A));
                const uint64_t bh = sw128_desc(smem_u32(st + 2 * TILE_A));
                const uint64_t bl = sw128_desc(smem_u32(st + 2 * TILE_A + tileB));
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {  // 4 MMAs of 32 bytes of K per stage
                    const uint64_t o = (uint64_t)(kk * 32) >> 4;
                    tc_mma<TF32>(acc, ah + o, bh + o, idesc, (kb | kk) ? 1u : 0u);
                    tc_mma<TF32>(acc, ah + o, bl + o, idesc, 1u);
                    tc_mma<TF32>(acc, al + o, bh + o, idesc, 1u);
                }
                tc_commit(&empty[s]);
            }
            if (!ok) break;
            tc_commit(&acc_full[b]);
        }
    } else if (warp >= 2) {
        // ---- epilogue: TMEM -> registers -> fused outputs ----
        const int q = warp & 3;          // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;   // slices 16 h, 16 h + 32, ...
        const TcEpilogue& ep = args.ep;
        float* stg = epi + (warp - 2) * 32 * EPI_PITCH;  // this warp's 32 x 16 staging
        const bool rowmajor = ep.out_f32 || ep.mul;
        const bool vf32 = args.vec & 1, vmul = args.vec & 2, vsplit = args.vec & 4;
        const int rl = lane >> 2, cg = lane & 3;  // restaged: rows rl + 8k, columns 4cg..4cg+3
        int i = 0;
        for (int t = blockIdx.x; t < args.ntiles; t += gridDim.x, ++i) {
            const int z = t / tnm, r = t % tnm, m0 = (r / args.tn) * BM, n0 = (r % args.tn) * BN;
            const int b = i & 1;
            const int mq = m0 + 32 * q;  // first row of this warp's quarter
            const int m = mq + lane;
            double* f64t = args.part ? args.part + (size_t)z * args.N * ep.ld_f64t : ep.out_f64t;
            float4 cur[4], nxt[4];
            auto load_partner = [&](int c, float4* dst) {
                const int n = n0 + c + 4 * cg;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int mm = mq + rl + 8 * k;
                    const float* src = ep.mul + (size_t)mm * ep.ld_mul + n;
                    if (mm < args.M && n + 3 < args.N && vmul) {
                        dst[k] = __ldg((const float4*)src);
                    } else {
                        float e[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            e[u] = (mm < args.M && n + u < args.N) ? __ldg(src + u) : 0.f;
                        dst[k] = make_float4(e[0], e[1], e[2], e[3]);
                    }
                }
            };
            const int c0 = 16 * h;
            // the first slice's partner loads overlap the main loop
            if (ep.mul && c0 < BN) load_partner(c0, cur);
            if (!mbar_wait(&acc_full[b], (i >> 1) & 1, 4)) break;
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)(b * ACC_COLS) + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
            for (int c = c0; c < BN; c += 32) {
                float v[16];
                tmem_ld16(acc + (uint32_t)c, v);
                // software pipeline: the next slice's partner loads are in flight while this
                // slice is written
                if (ep.mul && c + 32 < BN) load_partner(c + 32, nxt);
                if (f64t && m < args.M) {
                    // transposed FP64 output: consecutive lanes hold consecutive m (coalesced)
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = n0 + c + j;
                        if (n < args.N) f64t[(size_t)n * ep.ld_f64t + m] = (double)v[j];
                    }
                }
                if (rowmajor) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        *(float4*)&stg[lane * EPI_PITCH + 4 * k] =
                            make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                    __syncwarp();
                    const int n = n0 + c + 4 * cg;
                    const int lim = args.N - n;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int mm = mq + rl + 8 * k;
                        if (mm >= args.M || lim <= 0) continue;
                        const float4 d = *(const float4*)&stg[(rl + 8 * k) * EPI_PITCH + 4 * cg];
                        if (ep.out_f32) {
                            float* dst = ep.out_f32 + (size_t)mm * ep.ld_f32 + n;
                            if (vf32 && lim >= 4) {
                                *(float4*)dst = d;
                            } else {
                                const float x[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                                for (int u = 0; u < 4; ++u)
                                    if (u < lim) dst[u] = x[u];
                            }
                        }
                        if (ep.mul) {
                            const float4 p = cur[k];
                            const float4 e = make_float4(d.x * p.x, d.y * p.y, d.z * p.z, d.w * p.w);
                            store_split4<TF32>(args.out_hi, args.out_lo,
                                               (size_t)mm * args.ld_split + n, e, vsplit, lim);
                        }
                    }
                    __syncwarp();
                }
                if (ep.mul) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
                }
            }
            // every TMEM read of this tile has completed (tcgen05.wait::ld in tmem_ld16)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// fixed-order sum of the split-K partials into the FP64 output
__global__ void k_tc_splitk_reduce(const double* __restrict__ part, int splits, long total,
                                   double* __restrict__ out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
         i += (long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * total + i];
        out[i] = s;
    }
}

// ---- host side ---------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool load_encode() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode != nullptr;
}

bool make_map(CUtensorMap* map, bool tf32, const void* base, int rows, int cols, int pitch,
              int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const int esz = tf32 ? 4 : 2;
    cuuint64_t strides[1] = {(cuuint64_t)pitch * esz};
    cuuint32_t box[2] = {(cuuint32_t)(KBYTES / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int g_max_smem = 0;

}  // namespace

bool tc_available() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return false;
    if (!(p.major == 10 && p.minor == 3)) return false;
    g_max_smem = (int)p.sharedMemPerBlockOptin;
    return load_encode();
}

int tc_take_error() {
    int h = 0, z = 0;
    cudaMemcpyFromSymbol(&h, g_tc_error, sizeof(int));
    if (h) cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
    return h;
}

namespace {

// Launch one GEMM with tile N = BN (a multiple of 16, at most 256).
cudaError_t tc_launch(cudaStream_t st, bool tf32, const SplitMat& A, const SplitMat& B, int M,
                      int N, int K, const TcEpilogue& ep, double* part, size_t part_cap, int BN) {
    const int mt = cdiv(M, BM);
    const int tileB = BN * KBYTES;
    const int stage_bytes = 2 * TILE_A + 2 * tileB;
    const int nkb = std::max(1, cdiv((long)K * (tf32 ? 4 : 2), KBYTES));
    const int avail = g_max_smem - 1024 - EPI_STAGE_BYTES - 256;
    const int stages = std::max(2, std::min(6, avail / stage_bytes));
    const size_t smem = 1024 + (size_t)stages * stage_bytes + EPI_STAGE_BYTES + 256;
    CUtensorMap mAh, mAl, mBh, mBl;
    if (!make_map(&mAh, tf32, A.hi, M, K, A.pitch, BM) || !make_map(&mAl, tf32, A.lo, M, K, A.pitch, BM) ||
        !make_map(&mBh, tf32, B.hi, N, K, B.pitch, BN) || !make_map(&mBl, tf32, B.lo, N, K, B.pitch, BN))
        return cudaErrorInvalidValue;
    // split-K (deterministic, via FP64 partials) when only the transposed FP64 output is
    // wanted and the tile grid is far smaller than the SM count
    int splits = 1;
    const long tiles = (long)cdiv(N, BN) * mt;
    if (!ep.out_f32 && !ep.mul && ep.out_f64t && part && tiles * 2 <= num_sms() && nkb >= 4) {
        splits = (int)std::min<long>(std::min<long>(num_sms() / tiles, nkb / 2),
                                     (long)(part_cap / ((size_t)N * ep.ld_f64t)));
        splits = std::max(1, splits);
    }
    const int kper = cdiv(nkb, splits);
    splits = cdiv(nkb, kper);
    KArgs args;
    args.M = M;
    args.N = N;
    args.nkb = nkb;
    args.BN = BN;
    args.stages = stages;
    args.tn = cdiv(N, BN);
    args.tm = mt;
    args.ntiles = args.tn * mt * splits;
    args.kper = kper;
    args.part = splits > 1 ? part : nullptr;
    args.ep = ep;
    args.out_hi = ep.out_split ? ep.out_split->hi : nullptr;
    args.out_lo = ep.out_split ? ep.out_split->lo : nullptr;
    args.ld_split = ep.out_split ? ep.out_split->pitch : 0;
    auto al = [](const void* p, int bytes) { return ((uintptr_t)p % bytes) == 0; };
    args.vec = ((ep.out_f32 && al(ep.out_f32, 16) && ep.ld_f32 % 4 == 0) ? 1 : 0) |
               ((ep.mul && al(ep.mul, 16) && ep.ld_mul % 4 == 0) ? 2 : 0) |
               ((args.out_hi && al(args.out_hi, tf32 ? 16 : 8) && al(args.out_lo, tf32 ? 16 : 8) &&
                 args.ld_split % 4 == 0)
                    ? 4
                    : 0);
    const int grid = std::min(args.ntiles, num_sms());  // persistent: at most one CTA per SM
    ProfScope prof(st, ep.prof_class, 2.0 * M * (double)N * K);
    count_launch(splits > 1 ? 2 : 1);
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        // once per process, outside any stream capture: allow the largest ring
        cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem);
        cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem);
    });
    if (tf32)
        k_tc_gemm<true><<<grid, NTHREADS, smem, st>>>(mAh, mAl, mBh, mBl, args);
    else
        k_tc_gemm<false><<<grid, NTHREADS, smem, st>>>(mAh, mAl, mBh, mBl, args);
    if (splits > 1) {
        const long total = (long)N * ep.ld_f64t;
        k_tc_splitk_reduce<<<(int)std::min<long>(cdiv(total, 256), 4L * num_sms()), 256, 0, st>>>(
            part, splits, total, ep.out_f64t);
    }
    return cudaGetLastError();
}

// Default tile N: a multiple of 16 up to 256, as wide as keeps about one CTA per SM busy.
int heuristic_bn(int M, int N) {
    const int mt = cdiv(M, BM);
    int cap = 64;
    for (int cand : {256, 128}) {
        if ((long)mt * cdiv(N, cand) >= 120) {
            cap = cand;
            break;
        }
    }
    if (N <= cap) cap = std::max(16, ((N + 15) / 16) * 16);
    return std::min(256, (cdiv(N, cdiv(N, cap)) + 15) / 16 * 16);
}

// ---- autotuner: per (M, N, K, kind, epilogue) the fastest tile N, process-wide ----
struct TuneKey {
    int M, N, K, kind;
    bool operator<(const TuneKey& o) const {
        if (M != o.M) return M < o.M;
        if (N != o.N) return N < o.N;
        if (K != o.K) return K < o.K;
        return kind < o.kind;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;
std::atomic<int> g_tuning{0};

int epi_kind(bool tf32, const TcEpilogue& ep) {
    return (tf32 ? 1 : 0) | (ep.out_f32 ? 2 : 0) | (ep.mul ? 4 : 0) | (ep.out_f64t ? 8 : 0);
}

}  // namespace

void tc_set_tuning(bool on) { g_tuning.store(on ? 1 : 0); }

int tc_tuned_entries() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int)g_tuned.size();
}

cudaError_t tc_gemm(cudaStream_t st, bool tf32, const SplitMat& A, const SplitMat& B, int M, int N,
                    int K, const TcEpilogue& ep, double* part, size_t part_cap) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (!g_encode && !load_encode()) return cudaErrorNotSupported;
    if (g_max_smem == 0) tc_available();
    const TuneKey key{M, N, K, epi_kind(tf32, ep)};
    int BN = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) BN = it->second;
    }
    if (BN == 0 && g_tuning.load()) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (cs == cudaStreamCaptureStatusNone) {
            // time every candidate on the live operands (outputs are rewritten identically)
            const int nmax = std::min(256, ((N + 15) / 16) * 16);
            int cands[6], nc = 0;
            for (int c : {32, 64, 96, 128, 192, 256})
                if (c <= nmax) cands[nc++] = c;
            if (nc == 0) cands[nc++] = nmax;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            float best = 1e30f;
            for (int i = 0; i < nc; ++i) {
                cudaError_t err = tc_launch(st, tf32, A, B, M, N, K, ep, part, part_cap, cands[i]);
                if (err != cudaSuccess) continue;
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3; ++r) tc_launch(st, tf32, A, B, M, N, K, ep, part, part_cap, cands[i]);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    BN = cands[i];
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (BN) {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tuned[key] = BN;
            }
        }
    }
    if (BN == 0) BN = heuristic_bn(M, N);
    return tc_launch(st, tf32, A, B, M, N, K, ep, part, part_cap, BN);
}

// ---- split conversions ---------------------------------------------------------------
int split_kblock(bool tf32) { return tf32 ? 32 : 64; }
int split_pitch(bool tf32, int cols) {
    const int kb = split_kblock(tf32);
    return std::max(kb, ((cols + kb - 1) / kb) * kb);
}

template <bool TF32>
__device__ __forceinline__ void store_split_d(void* hi, void* lo, size_t idx, double x) {
    if (TF32) {
        const float xf = (float)x;
        const uint32_t u = __float_as_uint(xf);
        const float h = __uint_as_float((u + 0x1000u) & 0xFFFFE000u);
        const float r = (float)(x - (double)h);
        const float l = __uint_as_float((__float_as_uint(r) + 0x1000u) & 0xFFFFE000u);
        ((float*)hi)[idx] = h;
        ((float*)lo)[idx] = l;
    } else {
        const __nv_bfloat16 h = __double2bfloat16(x);
        const __nv_bfloat16 l = __double2bfloat16(x - (double)__bfloat162float(h));
        ((__nv_bfloat16*)hi)[idx] = h;
        ((__nv_bfloat16*)lo)[idx] = l;
    }
}

template <bool TF32>
__global__ void k_split_rows(const double* __restrict__ src, int ld, int rows, int cols, void* hi,
                             void* lo, int pitch) {
    const long n = (long)rows * cols;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        store_split_d<TF32>(hi, lo, (size_t)r * pitch + c, src[(size_t)r * ld + c]);
    }
}

// 32 x 32 tiles through shared memory so that reads and writes are both coalesced
template <bool TF32>
__global__ void k_split_transpose(const double* __restrict__ src, int ld, int rows, int cols,
                                  void* hi, void* lo, int pitch) {
    __shared__ double t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * ld + c] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) store_split_d<TF32>(hi, lo, (size_t)c * pitch + r, t[threadIdx.x][i]);
    }
}

template <bool TF32>
__global__ void k_split_hadamard(const float* __restrict__ a, const float* __restrict__ b, int ld,
                                 int rows, int cols, void* hi, void* lo, int pitch) {
    const long n = (long)rows * cols;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const size_t o = (size_t)r * ld + c;
        store_split<TF32>(hi, lo, (size_t)r * pitch + c, a[o] * b[o]);
    }
}

void split_rows(cudaStream_t st, bool tf32, const double* src, int ld, int rows, int cols,
                SplitMat& d) {
    const long n = (long)rows * cols;
    const int blocks = (int)std::min<long>(cdiv(n, 256), 4L * num_sms());
    count_launch();
    if (tf32)
        k_split_rows<true><<<blocks, 256, 0, st>>>(src, ld, rows, cols, d.hi, d.lo, d.pitch);
    else
        k_split_rows<false><<<blocks, 256, 0, st>>>(src, ld, rows, cols, d.hi, d.lo, d.pitch);
}

void split_transpose(cudaStream_t st, bool tf32, const double* src, int ld, int rows, int cols,
                     SplitMat& d) {
    dim3 grid(cdiv(cols, 32), cdiv(rows, 32)), block(32, 8);
    count_launch();
    if (tf32)
        k_split_transpose<true><<<grid, block, 0, st>>>(src, ld, rows, cols, d.hi, d.lo, d.pitch);
    else
        k_split_transpose<false><<<grid, block, 0, st>>>(src, ld, rows, cols, d.hi, d.lo, d.pitch);
}

void split_hadamard(cudaStream_t st, bool tf32, const float* a, const float* b, int ld, int rows,
                    int cols, SplitMat& d) {
    const long n = (long)rows * cols;
    const int blocks = (int)std::min<long>(cdiv(n, 256), 4L * num_sms());
    count_launch();
    if (tf32)
        k_split_hadamard<true><<<blocks, 256, 0, st>>>(a, b, ld, rows, cols, d.hi, d.lo, d.pitch);
    else
        k_split_hadamard<false><<<blocks, 256, 0, st>>>(a, b, ld, rows, cols, d.hi, d.lo, d.pitch);
}

}  // namespace thc
