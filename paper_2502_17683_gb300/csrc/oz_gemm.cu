// FP64-accurate emulated products on the BF16 tensor cores and the two-level LDL^T built
// on them (see oz.cuh for the arithmetic).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "f64.cuh"
#include "oz.cuh"
#include "prof.cuh"
#include "tcgen05.cuh"

namespace thc {

__device__ int g_oz_error = 0;

namespace {

constexpr int S = kOzSlices;
constexpr int KP = kOzPanel;                 // K elements per operand row (2 x 64)
constexpr int BM = 128;                      // MMA M: rows of the left operand per tile
constexpr int BN = 32;                       // MMA N: rows of the right operand per tile
constexpr int A_TILE = BM * 128;             // bytes of one 128 x 64 BF16 slice (one K half)
constexpr int A_DEPTH = 2;                   // slices per left-operand TMA box and ring stage
constexpr int A_STAGE = A_DEPTH * A_TILE;    // 32 KB
constexpr int A_GROUPS = (S + A_DEPTH - 1) / A_DEPTH;  // stages per K half (the last one half used)
constexpr int B_HALF = S * BN * 128;         // all right-operand slices of one K half (28 KB)
constexpr int A_STAGES = 4;
constexpr int B_STAGES = 2;
constexpr int SMEM_BYTES = 1024 + A_STAGES * A_STAGE + B_STAGES * B_HALF + 256;
constexpr int ACC_SET = S * BN;              // TMEM columns of one set of S accumulators (224)
constexpr int TMEM_COLS = 512;               // two sets: the epilogue drains one, the MMAs fill the other
constexpr int EPI_WARPS = 16;                // four per TMEM lane quarter, 8 columns each
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;  // warp 0 TMA, warp 1 MMA + TMEM, then the epilogue
constexpr uint32_t WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ bool oz_wait(uint64_t* bar, uint32_t parity, int code) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(&g_oz_error, code);
    return false;
}

__device__ __forceinline__ double pow2(int e) {
    return __longlong_as_double((long long)(e + 1023) << 52);  // e in [-1022, 1023]
}

// Exponent E of a normal double, |x| in [2^(E-1), 2^E); -2000 for zero, subnormal, inf, NaN.
__device__ __forceinline__ int exp_of(double x) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    return (ex == 0 || ex == 0x7FF) ? -2000 : ex - 1022;
}

// The S digits of x relative to the row exponent erow: x ~ 2^erow sum_a d_a 2^(-7-8a),
// formed exactly in integer arithmetic from the bits of x (X = round(x 2^(55 - erow)),
// then signed base-256 digits from the least significant one up).
__device__ __forceinline__ void digits_of(double x, int erow, int (&d)[S]) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    long long X = 0;
    if (ex != 0 && ex != 0x7FF) {
        const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
        const int sh = (ex - 1022) - erow + 2;  // <= 2
        if (sh >= 0)
            X = m * (1LL << sh);
        else if (sh > -54)
            X = (m + (1LL << (-sh - 1))) >> (-sh);
        if (b < 0) X = -X;
    }
#pragma unroll
    for (int a = S - 1; a > 0; --a) {
        const long long da = ((X + 128) & 255) - 128;
        d[a] = (int)da;
        X = (X - da) >> 8;  // exact: X - da is a multiple of 256 (arithmetic shift)
    }
    d[0] = (int)X;
}

// V 2^e rounded once to FP64 (to nearest, ties to even), its sign flipped by neg (0 or the
// sign bit): the IEEE 754 binary64 encoding of the normalised magnitude assembled in integer
// arithmetic, so that of each output element only the final addition runs on the FP64 pipe
// (an int64 conversion costs as much there as an FMA). |V| < 2^63. Below the normal range
// the term is dropped (signed zero), above it the result is infinite.
__device__ __forceinline__ double scaled_i64(long long V, int e, unsigned long long neg) {
    const unsigned long long sgn = ((unsigned long long)V & 0x8000000000000000ULL) ^ neg;
    const unsigned long long u = V < 0 ? 0ULL - (unsigned long long)V : (unsigned long long)V;
    if (u == 0) return __longlong_as_double((long long)sgn);
    const int lz = __clzll((long long)u);
    const unsigned long long m = u << lz;   // leading one at bit 63
    unsigned long long mant = m >> 11;      // 53 bits, leading one at bit 52
    const unsigned rem = (unsigned)(m & 0x7FFULL);
    mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ULL))) ? 1ULL : 0ULL;
    const int be = 1023 + 63 - lz + e;      // biased exponent of the result
    if (be < 1) return __longlong_as_double((long long)sgn);
    if (be > 2046) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ULL));
    // a rounding carry into bit 53 moves into the exponent field
    return __longlong_as_double((long long)(sgn | (((unsigned long long)(be - 1) << 52) + mant)));
}

__device__ __forceinline__ uint16_t bf16_int(int d) {
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)d));
}

// Row exponent of a row held by a group of 128 threads (4 warps, one value each): the max
// of the exponent fields, -2000 (no normal value) giving 0. sh: 4 ints per group; every
// thread of the block must call it (it holds a block barrier).
__device__ __forceinline__ int group_row_exp(int e, int* sh, int group, int wig) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0) sh[group * 4 + wig] = e;
    __syncthreads();
    e = max(max(sh[group * 4], sh[group * 4 + 1]), max(sh[group * 4 + 2], sh[group * 4 + 3]));
    return e == -2000 ? 0 : e;
}

// The S digits of one value into slices out[a][row][k] (one BF16 each).
__device__ __forceinline__ void store_digits(double x, int erow, uint16_t* __restrict__ out, int rows_alloc,
                                             int row, int k) {
    int d[S];
    digits_of(x, erow, d);
#pragma unroll
    for (int a = 0; a < S; ++a) out[((size_t)a * rows_alloc + row) * KP + k] = bf16_int(d[a]);
}

constexpr int SPLIT_ROWS = 2;  // rows per block of the row splits: 128 threads, one value each, per row

// Row r < rows: the values src[r * ld + k] (k < K, zero beyond), their row exponent and
// their S digit slices out[a][r][k] (k < KP). 128 threads per row, one value each. K chunk
// c = blockIdx.y (values KP c ..) goes to slices out[S c + a] and exponents exps[rows_alloc c ..].
__global__ void __launch_bounds__(128 * SPLIT_ROWS)
k_oz_split(const double* __restrict__ src, int ld, int rows, int K, uint16_t* __restrict__ out,
           int rows_alloc, int* __restrict__ exps) {
    __shared__ int sh[4 * SPLIT_ROWS];
    const int group = threadIdx.x >> 7, k = threadIdx.x & 127, wig = k >> 5;
    const int r = blockIdx.x * SPLIT_ROWS + group;
    const int ch = blockIdx.y;
    src += (size_t)ch * KP;
    K -= ch * KP;
    out += (size_t)ch * S * rows_alloc * KP;
    exps += (size_t)ch * rows_alloc;
    const bool live = r < rows;
    const double x = (live && k < K) ? src[(size_t)r * ld + k] : 0.0;
    const int erow = group_row_exp(exp_of(x), sh, group, wig);
    if (!live) return;
    store_digits(x, erow, out, rows_alloc, r, k);
    if (k == 0) exps[r] = erow;
}

// The two operands of an LDL^T trailing update from one read of the rows below the panel:
// row r < mA of src (its first K entries) gives the left-operand row r, scaled per column k
// by D_k 2^-m_k, and, for r < mB, the right-operand row r, scaled by 2^m_k (m_k =
// floor(E(D_k) / 2), D_k = diag[k * (ldd + 1)]), each cut into its S digit slices.
// 128 threads per row, one column each.
__global__ void __launch_bounds__(128 * SPLIT_ROWS)
k_oz_split_ldl(const double* __restrict__ src, int ld, int mA, int mB, int K,
               const double* __restrict__ diag, int ldd, uint16_t* __restrict__ outA, int rowsA,
               int* __restrict__ expsA, uint16_t* __restrict__ outB, int rowsB, int* __restrict__ expsB) {
    __shared__ int sha[4 * SPLIT_ROWS], shb[4 * SPLIT_ROWS];
    const int group = threadIdx.x >> 7, k = threadIdx.x & 127, wig = k >> 5;
    const int r = blockIdx.x * SPLIT_ROWS + group;
    // K chunk ch = blockIdx.y of a wider panel: its columns, their D, its slices and exponents
    const int ch = blockIdx.y;
    src += (size_t)ch * KP;
    diag += (size_t)ch * KP * (ldd + 1);
    K -= ch * KP;
    outA += (size_t)ch * S * rowsA * KP;
    expsA += (size_t)ch * rowsA;
    outB += (size_t)ch * S * rowsB * KP;
    expsB += (size_t)ch * rowsB;
    const bool live = r < mA;
    double a = 0.0, b = 0.0;
    if (live && k < K) {
        const double v = src[(size_t)r * ld + k];
        const double dk = diag[(size_t)k * (ldd + 1)];
        const int Ek = exp_of(dk);
        const int mk = (Ek == -2000) ? 0 : (Ek >> 1);
        a = v * (dk * pow2(-mk));
        b = v * pow2(mk);
    }
    const int ea = group_row_exp(exp_of(a), sha, group, wig);
    const int eb = group_row_exp(exp_of(b), shb, group, wig);
    if (!live) return;
    store_digits(a, ea, outA, rowsA, r, k);
    const bool hasB = r < mB;
    if (hasB) store_digits(b, eb, outB, rowsB, r, k);
    if (k == 0) {
        expsA[r] = ea;
        if (hasB) expsB[r] = eb;
    }
}

constexpr int SPLIT_T_ROWS = 8;  // output rows per block of the transposed split (1024 threads)

// Transposed source: output row n < N takes the K chunk [k0, k0 + kb) of column n of the
// K x N row-major matrix S (ld), times S2 element by element when given (a Hadamard
// operand): values S[(k0 + k) * ld + n] (* S2[...]). A 128 x 8 slab is staged in shared
// memory (8 consecutive columns per source row), then 128 threads per output row form its
// exponent and digits, one value each. Chunk c = blockIdx.y takes rows k0 + KP c .. (of the
// kb left) into slices out[S c + a] and exponents exps[rows_alloc c ..].
__global__ void __launch_bounds__(128 * SPLIT_T_ROWS)
k_oz_split_t(const double* __restrict__ S, const double* __restrict__ S2, int ld, int N, int k0,
             int kb, uint16_t* __restrict__ out, int rows_alloc, int* __restrict__ exps) {
    __shared__ double tile[KP][SPLIT_T_ROWS + 1];
    __shared__ int sh[4 * SPLIT_T_ROWS];
    const int ch = blockIdx.y;
    k0 += ch * KP;
    kb -= ch * KP;
    out += (size_t)ch * kOzSlices * rows_alloc * KP;  // (S is the source matrix here)
    exps += (size_t)ch * rows_alloc;
    const int n0 = blockIdx.x * SPLIT_T_ROWS;
    {
        const int kk = threadIdx.x / SPLIT_T_ROWS, nn = threadIdx.x % SPLIT_T_ROWS;
        const int n = n0 + nn;
        double v = 0.0;
        if (kk < kb && n < N) {
            const size_t o = (size_t)(k0 + kk) * ld + n;
            v = S[o];
            if (S2) v *= S2[o];
        }
        tile[kk][nn] = v;
    }
    __syncthreads();
    const int group = threadIdx.x >> 7, k = threadIdx.x & 127, wig = k >> 5;
    const int n = n0 + group;
    const double x = tile[k][group];
    const int erow = group_row_exp(exp_of(x), sh, group, wig);
    if (n >= N) return;
    store_digits(x, erow, out, rows_alloc, n, k);
    if (k == 0) exps[n] = erow;
}

// C[j][i] = C[i][j] for j > i (the upper triangle of a symmetric result from its lower one)
__global__ void k_oz_mirror(int n, double* __restrict__ C, int ldc) {
    __shared__ double t[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;  // tile row, tile column (bj > bi mirrored)
    if (bj < bi) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        const int i = bj * 32 + r, j = bi * 32 + tx;  // lower element (i, j), i >= j
        t[r][tx] = (i < n && j < n) ? C[(size_t)i * ldc + j] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = bi * 32 + r, j = bj * 32 + tx;  // upper element (i, j) = lower (j, i)
        if (i < n && j < n && j > i) C[(size_t)i * ldc + j] = t[tx][r];
    }
}

struct UpdArgs {
    double* C;     // C[i][j] at C[i * ldc + j]
    int ldc;
    int mA, mB;    // rows of C (left operand rows) and columns (right operand rows)
    const int* eA;
    const int* eB;
    int tiles_m;   // tiles along mA
    int tiles_n;   // tiles along mB
    int lower;     // 1: rows i < mB only on and below the diagonal (LDL^T trailing block)
    double sign;   // C (+)= sign * E o (A B^T); +1 or -1
    int accumulate;  // 0: C is overwritten
    const double* E;  // optional Hadamard factor of the product, indexed like C
    int khalves;      // 64-wide K halves that hold data in the last chunk (1 when its K <= 64)
    int nchunks;      // K chunks of KP; chunk c's slices are planes S c .. S c + S - 1 of the maps
    int eA_cs, eB_cs; // offsets between the chunks' exponent rows
    int nactive;      // active tiles (tile_of's index range)
    int kgroups;      // split K: work item (group g, tile) takes chunks [g cpg, (g + 1) cpg); group 0
    int cpg;          // adds into C, group g > 0 writes its sum to part + (g - 1) mA mB (ld mB)
    double* part;     // (kgroups > 1 only without E and lower)
};

// Active tiles of row block tm: on a lower-only (symmetric or LDL^T trailing) block, rows
// that lie within the first mB stop at the diagonal; below them every tile is active.
__host__ __device__ __forceinline__ int row_tiles(int tm, int tiles_n, int mB, bool lower) {
    const int m0 = tm * BM;
    return (lower && m0 + BM - 1 < mB) ? min(tiles_n, (m0 + BM - 1) / BN + 1) : tiles_n;
}

// The active tile of compact index u (row by row, so that the CTAs' shares of a lower block
// differ by at most one tile; tiles above the diagonal are never handed out). Only the rows
// of a lower block that end within its first mB columns (at most mB / BM of them) have
// fewer tiles than tiles_n; they are walked, every later row is full.
__device__ __forceinline__ void tile_of(const UpdArgs& a, int u, int& m0, int& n0) {
    int tm = 0;
    if (a.lower) {
        for (; tm < a.tiles_m && tm * BM + BM - 1 < a.mB; ++tm) {
            const int c = row_tiles(tm, a.tiles_n, a.mB, true);
            if (u < c) {
                m0 = tm * BM;
                n0 = u * BN;
                return;
            }
            u -= c;
        }
    }
    tm += u / a.tiles_n;
    m0 = tm * BM;
    n0 = (u % a.tiles_n) * BN;
}

// C (+)= sign * E o (A B^T) from the digit slices, one 128 x 32 output tile at a time, each
// CTA (one per SM) walking tiles blockIdx.x, blockIdx.x + gridDim.x, ...: warp 0 streams,
// per tile and K half, the right operand's S boxes (one 28 KB stage) and the left
// operand's S boxes (16 KB stages) by 3-D TMA; warp 1 issues, per left slice a and K step,
// one BF16 MMA against the stacked right slices b <= S - 1 - a whose result columns fall
// into accumulators a + b of the tile's set (two sets of S x 32 TMEM columns alternate
// between tiles): 7 MMAs of N = 32 (S - a) per K step instead of 28; eight epilogue warps (a lane
// quarter and 16 columns each) turn the previous tile's S integer accumulators into one
// FP64 value per element and apply it, overlapping the MMAs of the next tile. Rows of C
// below mB on a lower-only block are updated on and below the diagonal only. Every wait is
// bounded.
__global__ void __launch_bounds__(NTHREADS, 1)
k_oz_update(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
            const UpdArgs args) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* asm_ = smem;                               // [A_STAGES] x A_STAGE
    uint8_t* bsm = smem + A_STAGES * A_STAGE;           // [B_STAGES] x B_HALF
    uint64_t* afull = (uint64_t*)(bsm + B_STAGES * B_HALF);
    uint64_t* aempty = afull + A_STAGES;
    uint64_t* bfull = aempty + A_STAGES;
    uint64_t* bempty = bfull + B_STAGES;
    uint64_t* accfull = bempty + B_STAGES;              // [2]
    uint64_t* accempty = accfull + 2;                   // [2]
    uint32_t* tmem_slot = (uint32_t*)(accempty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = args.nactive;
    const int nwork = ntiles * args.kgroups;

    if (threadIdx.x == 0) {
        for (int i = 0; i < A_STAGES; ++i) {
            mbar_init(&afull[i], 1);
            mbar_init(&aempty[i], 1);
        }
        for (int i = 0; i < B_STAGES; ++i) {
            mbar_init(&bfull[i], 1);
            mbar_init(&bempty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accempty[i], EPI_WARPS);
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
        int ia = 0, ib = 0;  // positions in the two rings, over all tiles of this CTA
        bool ok = true;
        for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
            const int t = w % ntiles, g0 = (w / ntiles) * args.cpg, g1 = min(args.nchunks, g0 + args.cpg);
            int m0, n0;
            tile_of(args, t, m0, n0);
            for (int ch = g0; ch < g1 && ok; ++ch) {
            const int nh = ch == args.nchunks - 1 ? args.khalves : 2;
            for (int c = 0; c < nh && ok; ++c) {
                const int sb = ib % B_STAGES;
                if (!oz_wait(&bempty[sb], ((ib / B_STAGES) & 1) ^ 1, 1)) { ok = false; break; }
                mbar_expect_tx(&bfull[sb], (uint32_t)B_HALF);
                // all S right slices in one box, stacked (slice b at rows 32 b ..)
                tma_load_3d(bsm + sb * B_HALF, &mapB, &bfull[sb], 64 * c, n0, S * ch);
                ++ib;
                for (int g = 0; g < A_GROUPS; ++g, ++ia) {
                    // slices 2g, 2g + 1 in one box (past the chunk's last slice the box holds
                    // the next chunk's first, or zeros; its bytes still count, the MMAs skip it)
                    const int sa = ia % A_STAGES;
                    if (!oz_wait(&aempty[sa], ((ia / A_STAGES) & 1) ^ 1, 1)) { ok = false; break; }
                    mbar_expect_tx(&afull[sa], (uint32_t)A_STAGE);
                    tma_load_3d(asm_ + sa * A_STAGE, &mapA, &afull[sa], 64 * c, m0, S * ch + A_DEPTH * g);
                }
            }
            }
        }
        // every copy issued has landed before the CTA may leave
        for (int j = max(0, ia - A_STAGES); j < ia; ++j) oz_wait(&afull[j % A_STAGES], (j / A_STAGES) & 1, 2);
        for (int j = max(0, ib - B_STAGES); j < ib; ++j) oz_wait(&bfull[j % B_STAGES], (j / B_STAGES) & 1, 2);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        int ia = 0, ib = 0, i = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
            const int t = w % ntiles, g0 = (w / ntiles) * args.cpg, g1 = min(args.nchunks, g0 + args.cpg);
            int m0, n0;
            tile_of(args, t, m0, n0);
            // one accumulator set per (tile, K chunk), alternating
            for (int ch = g0; ch < g1 && ok; ++ch) {
            const int nh = ch == args.nchunks - 1 ? args.khalves : 2;
            const int set = i & 1;
            // accumulator set `set` is free once the epilogue has drained tile-chunk i - 2
            if (i >= 2 && !oz_wait(&accempty[set], ((i >> 1) - 1) & 1, 5)) { ok = false; break; }
            tc_fence_after();
            const uint32_t acc0 = tmem + (uint32_t)(set * ACC_SET);
            for (int c = 0; c < nh && ok; ++c) {
                const int sb = ib % B_STAGES;
                if (!oz_wait(&bfull[sb], (ib / B_STAGES) & 1, 3)) { ok = false; break; }
                const uint64_t bd = sw128_desc(smem_u32(bsm + sb * B_HALF));
                for (int g = 0; g < A_GROUPS; ++g, ++ia) {
                    const int sa = ia % A_STAGES;
                    if (!oz_wait(&afull[sa], (ia / A_STAGES) & 1, 4)) { ok = false; break; }
                    tc_fence_after();
#pragma unroll
                    for (int s2 = 0; s2 < A_DEPTH; ++s2) {
                        const int a = A_DEPTH * g + s2;
                        if (a >= S) break;
                        // the right slices b = 0..S-1-a lie stacked in the stage (rows 32 b ..), so
                        // one MMA of N = 32 (S - a) with its accumulator base at column 32 a puts
                        // A_a B_b^T at columns 32 (a + b): accumulator a + b, for every b at once
                        const uint64_t ad = sw128_desc(smem_u32(asm_ + sa * A_STAGE + s2 * A_TILE));
                        const uint32_t idesc_a = make_idesc(false, BM, BN * (S - a));
                        const uint32_t acc = acc0 + (uint32_t)(a * BN);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {  // 4 x 16 elements (32 bytes) per 64-wide box
                            const uint64_t o = (uint64_t)(kk * 32) >> 4;
                            tc_mma<false>(acc, ad + o, bd + o, idesc_a, (c | a | kk) ? 1u : 0u);
                        }
                    }
                    tc_commit(&aempty[sa]);
                }
                tc_commit(&bempty[sb]);
                ++ib;
            }
            tc_commit(&accfull[set]);  // also after a failed wait: arrives once the issued MMAs are done
            ++i;
            }
        }
    } else if (warp >= 2) {
        // ---- epilogue: a lane quarter q and 8 columns h of each tile ----
        const int q = warp & 3, h = (warp - 2) >> 2;  // h = 0..3
        const unsigned long long sign_bit = args.sign < 0.0 ? 0x8000000000000000ULL : 0ULL;
        int i = 0;
        for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
            const int t = w % ntiles, grp = w / ntiles, g0 = grp * args.cpg, g1 = min(args.nchunks, g0 + args.cpg);
            int m0, n0;
            tile_of(args, t, m0, n0);
            // group 0 into C, the others into their partial sums
            double* const cbase = grp == 0 ? args.C : args.part + (size_t)(grp - 1) * args.mA * args.mB;
            const int cld = grp == 0 ? args.ldc : args.mB;
            for (int ch = g0; ch < g1; ++ch) {
            // chunks after the group's first add to what the previous one wrote (same thread, same elements)
            const bool accum = (grp == 0 && args.accumulate) || ch > g0;
            const int* eBc = args.eB + (size_t)ch * args.eB_cs;
            const int set = i & 1;
            const bool ok = oz_wait(&accfull[set], (i >> 1) & 1, 6);
            tc_fence_after();
            const int row = m0 + 32 * q + lane;
            const bool rowok = row < args.mA;
            const int ea = rowok ? args.eA[(size_t)ch * args.eA_cs + row] : 0;
            double* crow = cbase + (size_t)row * cld;
            const uint32_t tbase = tmem + (uint32_t)(set * ACC_SET + 8 * h) + ((uint32_t)(32 * q) << 16);
            // two halves of 4 columns; every lane takes part in each tensor-memory load (a
            // warp-wide instruction), only the arithmetic and the stores are masked per lane
#pragma unroll 1
            for (int hh = 0; hh < 2; ++hh) {
                const int jc = n0 + 8 * h + 4 * hh;
                uint32_t r[S][4];
#pragma unroll
                for (int g = 0; g < S; ++g) tmem_ld4_nowait(tbase + (uint32_t)(g * BN + 4 * hh), r[g]);
                double cv[4];
                int eb[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int j = jc + jj;
                    cv[jj] = (ok && rowok && j < args.mB && accum) ? crow[j] : 0.0;
                    eb[jj] = j < args.mB ? __ldg(eBc + j) : 0;
                }
                tmem_ld_wait(r);
                if (rowok && ok) {
                    double tv[4];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        long long acc[S];
#pragma unroll
                        for (int g = 0; g < S; ++g) acc[g] = (long long)__float2int_rn(__uint_as_float(r[g][jj]));
                        const long long hi = acc[0] * 65536 + acc[1] * 256 + acc[2];
                        const long long lo = acc[3] * 16777216 + acc[4] * 65536 + acc[5] * 256 + acc[6];
                        const int sh = (hi >= (1LL << 29) || hi <= -(1LL << 29)) ? 8 : 0;
                        tv[jj] = scaled_i64(hi * (1LL << (32 - sh)) + (lo >> sh), ea + eb[jj] - 62 + sh, sign_bit);
                    }
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = jc + jj;
                        double out;
                        if (args.E) {
                            const double f = args.E[(size_t)row * args.ldc + min(j, args.mB - 1)];
                            out = accum ? fma(f, tv[jj], cv[jj]) : f * tv[jj];
                        } else {
                            out = accum ? cv[jj] + tv[jj] : tv[jj];
                        }
                        if (j < args.mB && !(args.lower && row < args.mB && j > row)) crow[j] = out;
                    }
                }
                __syncwarp();
            }
            // every TMEM read of this tile has completed (tcgen05.wait::ld)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[set]);
            ++i;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// C[i][j] += part[0][i][j] + part[1][i][j] + ... (the split-K partial sums, fixed order)
__global__ void k_oz_add_parts(double* __restrict__ C, int ldc, int M, int N, const double* __restrict__ part,
                               int nparts) {
    const long total = (long)M * N;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        double* c = C + (e / N) * (long)ldc + e % N;
        double v = *c;
        for (int p = 0; p < nparts; ++p) v += part[p * total + e];
        *c = v;
    }
}

// ---- host ----------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;
bool g_ready = false;
int g_num_sm = 148;

bool oz_init() {
    std::call_once(g_once, [] {
        int dev = 0;
        cudaDeviceProp p;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return;
        if (!(p.major == 10 && p.minor == 3) || (int)p.sharedMemPerBlockOptin < SMEM_BYTES) return;
        g_num_sm = p.multiProcessorCount;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        if (cudaFuncSetAttribute(k_oz_update, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
            cudaSuccess)
            return;
        g_ready = true;
    });
    return g_ready;
}

// 3-D map over the digit slices [planes][rows_alloc][KP] (BF16; S planes per K chunk):
// box 64 (K) x box_rows x depth.
bool slice_map(CUtensorMap* m, const uint16_t* base, int rows, int rows_alloc, int box_rows, int depth,
               int planes = S) {
    cuuint64_t dims[3] = {(cuuint64_t)KP, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)KP * 2, (cuuint64_t)rows_alloc * KP * 2};
    cuuint32_t box[3] = {64, (cuuint32_t)box_rows, (cuuint32_t)depth};
    cuuint32_t estr[3] = {1, 1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void split(cudaStream_t st, const double* src, int ld, int rows, int K, uint16_t* out, int rows_alloc,
           int* exps) {
    if (rows <= 0) return;
    k_oz_split<<<cdiv(rows, SPLIT_ROWS), 128 * SPLIT_ROWS, 0, st>>>(src, ld, rows, K, out, rows_alloc, exps);
    count_launch();
}

// same_ab: the left operand is the right one (a Gram A^T A): its slices and exponents are
// read from the right operand's buffers.
// nchunks > 1: K = KP (nchunks - 1) + kb in one launch, the chunks' slices laid out
// [chunk][S][mA][KP] and [chunk][S][mB][KP] (exponents [chunk][mA], [chunk][mB]).
// kgroups > 1 (with nchunks > 1, no E, not lower): the chunks in kgroups groups on separate
// CTAs, all groups but the first summed in ws.part, then added to C in order.
cudaError_t update(cudaStream_t st, int mA, int mB, int kb, double* C, int ldc, const OzWs& ws, bool lower,
                   double sign, bool accumulate = true, const double* E = nullptr, bool same_ab = false,
                   int nchunks = 1, int kgroups = 1) {
    if (mA <= 0 || mB <= 0) return cudaSuccess;
    CUtensorMap ma, mb;
    const uint16_t* sa = same_ab ? ws.sB : ws.sA;
    const int ra = nchunks > 1 ? mA : (same_ab ? ws.rowsB : ws.rowsA);
    const int rb = nchunks > 1 ? mB : ws.rowsB;
    if (!slice_map(&ma, sa, mA, ra, BM, A_DEPTH, S * nchunks) || !slice_map(&mb, ws.sB, mB, rb, BN, S, S * nchunks))
        return cudaErrorInvalidValue;
    if (kgroups > 1 && (E || lower || nchunks < 2 || !ws.part ||
                        (size_t)(kgroups - 1) * mA * mB > ws.part_cap))
        kgroups = 1;
    const int cpg = cdiv(nchunks, std::max(1, kgroups));
    kgroups = cdiv(nchunks, cpg);
    const int tiles_m = cdiv(mA, BM), tiles_n = cdiv(mB, BN);
    long active = 0;
    for (int tm = 0; tm < tiles_m; ++tm) active += row_tiles(tm, tiles_n, mB, lower);
    UpdArgs a{C, ldc, mA, mB, same_ab ? ws.eB : ws.eA, ws.eB, tiles_m, tiles_n, lower ? 1 : 0,
              sign, accumulate ? 1 : 0, E, kb > 64 ? 2 : 1, nchunks, ra, rb, (int)active, kgroups, cpg, ws.part};
    // persistent: one CTA per SM, at most one per active (tile, K group) work item
    const int grid = (int)std::max<long>(1, std::min<long>(active * kgroups, g_num_sm));
    k_oz_update<<<grid, NTHREADS, SMEM_BYTES, st>>>(ma, mb, a);
    count_launch();
    if (kgroups > 1) {
        k_oz_add_parts<<<(int)std::min<long>(cdiv((long)mA * mB, 256), 4L * g_num_sm), 256, 0, st>>>(
            C, ldc, mA, mB, ws.part, kgroups - 1);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace

size_t oz_ws_bytes(int rowsA, int rowsB, size_t part_doubles) {
    return Arena::need<uint16_t>((size_t)S * rowsA * KP) + Arena::need<uint16_t>((size_t)S * rowsB * KP) +
           Arena::need<int>(rowsA) + Arena::need<int>(rowsB) + (part_doubles ? Arena::need<double>(part_doubles) : 0);
}

bool oz_available() { return oz_init(); }

void oz_ws_carve(OzWs& w, Arena& ar, int rowsA, int rowsB, size_t part_doubles) {
    w.rowsA = rowsA;
    w.rowsB = rowsB;
    w.sA = ar.take<uint16_t>((size_t)S * w.rowsA * KP);
    w.sB = ar.take<uint16_t>((size_t)S * w.rowsB * KP);
    w.eA = ar.take<int>(w.rowsA);
    w.eB = ar.take<int>(w.rowsB);
    w.part = part_doubles ? ar.take<double>(part_doubles) : nullptr;
    w.part_cap = part_doubles;
}

// Once at most this many columns are left, the rest of the factorisation runs as one
// dataflow launch (its FP64 trailing updates still hide behind its pivot chain there)
// instead of further panels, each followed by a digit split and an update launch that the
// next panel waits for. Measured on GB300 with 128-column panels, BF16x3 sweeps/s: 106.9 /
// 108.5 / 110.1 / 110.1 / 105.7 at R_cp = 1800 for 8 (none) / 264 / 520 / 776 / 1032
// columns, 221.9 / 226.5 / 233.7 at R_cp = 1080 for 56 / 312 / 440.
constexpr int kTailCols = 520;

// From R = 1536, panels of two K chunks: half as many panel boundaries (digit split and
// update launch, which the next panel waits for), each update over both chunks in one
// launch. BF16x3 sweeps/s on GB300: 120.2 / 121.3 / 115.6 at R_cp = 1800 for 128 / 256 / 384
// columns (the panel's FP64 substitution work outgrows its pivot chain at 384), 235.8 /
// 238.1 at R_cp = 1080; but the 64-problem batch (R_cp <= 1440, panels on at most 32 CTAs
// beside the other problems, where that FP64 work is no longer hidden) took 3.86 s with
// 256 against 3.73 s with 128. The width depends on R alone, so a problem factorises the
// same way (same bits) in the batched driver and alone.
int panel_cols(int R) { return R >= 1536 ? 2 * KP : KP; }

// Width of the panel that starts at column j0: panel_cols(R), or everything left once at
// most kTailCols columns remain.
int panel_width(int R, int j0) {
    return R - j0 <= kTailCols ? R - j0 : std::min(panel_cols(R), R - j0);
}

void oz_ldl_ws_rows(int R, int nmax, int* rowsA, int* rowsB) {
    const int pc = std::min(panel_cols(R), R);
    const long nch = cdiv(pc, KP);
    if (nch < 2 || R - pc <= 0) return;
    *rowsA = (int)std::max<long>(*rowsA, nch * (R + nmax - pc));
    *rowsB = (int)std::max<long>(*rowsB, nch * (R - pc));
}

bool oz_prepare(int R, int n) {
    if (!oz_init()) return false;
    for (int j0 = 0; j0 < R;) {
        const int bw = panel_width(R, j0);
        if (!flow_prepare(bw, R + n - j0 - bw)) return false;
        j0 += bw;
    }
    return true;
}

cudaError_t ldl_oz(cudaStream_t st, int R, int n, double* Haug, double* P, double* dinv,
                   DevScalars* sc, int mode, int* sync, const OzWs& ws, int max_ctas) {
    for (int j0 = 0; j0 < R; j0 += panel_width(R, j0)) {
        const int bw = panel_width(R, j0);
        const int j1 = j0 + bw;
        const int mA = R + n - j1, mB = R - j1;
        cudaError_t e;
        {
            // the panel's LDL^T and the substitution of every row below it
            ProfScope prof(st, KC_CHOL, (double)bw * bw * bw / 3.0 + (double)mA * bw * bw);
            e = ldl_flow_panel(st, R, n, j0, bw, Haug, P, dinv, sc, mode, sync, max_ctas);
        }
        if (e != cudaSuccess) return e;
        if (j1 >= R) break;
        const double* below = Haug + (size_t)j1 * R + j0;   // rows j1.., panel columns
        const double* diag = Haug + (size_t)j0 * R + j0;
        {
            ProfScope prof(st, KC_OZ, (double)mB * (mB + 1) * bw + 2.0 * (mA - mB) * mB * bw);
            const int nch = cdiv(bw, KP);
            if (nch > 1 && (long)nch * mA <= ws.rowsA && (long)nch * mB <= ws.rowsB) {
                // a wider panel: all its chunks split at once, one update launch over them
                k_oz_split_ldl<<<dim3(cdiv(mA, SPLIT_ROWS), nch), 128 * SPLIT_ROWS, 0, st>>>(
                    below, R, mA, mB, bw, diag, R, ws.sA, mA, ws.eA, ws.sB, mB, ws.eB);
                count_launch();
                e = update(st, mA, mB, bw - KP * (nch - 1), Haug + (size_t)j1 * R + j1, R, ws, true, -1.0, true,
                           nullptr, false, nch);
            } else {
                for (int k0 = 0; k0 < bw && e == cudaSuccess; k0 += KP) {
                    const int kb = std::min(KP, bw - k0);
                    k_oz_split_ldl<<<cdiv(mA, SPLIT_ROWS), 128 * SPLIT_ROWS, 0, st>>>(
                        below + k0, R, mA, mB, kb, diag + (size_t)k0 * (R + 1), R, ws.sA, ws.rowsA, ws.eA, ws.sB,
                        ws.rowsB, ws.eB);
                    count_launch();
                    e = update(st, mA, mB, kb, Haug + (size_t)j1 * R + j1, R, ws, true, -1.0);
                }
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t oz_gemm(cudaStream_t st, int M, int N, int K, const double* A, int lda, const double* B,
                    int ldb, double* C, int ldc, double sign, bool lower, const OzWs& ws) {
    if (!oz_init()) return cudaErrorNotSupported;
    if (M > ws.rowsA || N > ws.rowsB) return cudaErrorInvalidValue;
    const int nch = cdiv(K, KP);
    if (nch > 1 && (long)nch * M <= ws.rowsA && (long)nch * N <= ws.rowsB) {
        // every chunk's digits at once, then one update launch over all chunks
        k_oz_split<<<dim3(cdiv(M, SPLIT_ROWS), nch), 128 * SPLIT_ROWS, 0, st>>>(A, lda, M, K, ws.sA, M, ws.eA);
        k_oz_split<<<dim3(cdiv(N, SPLIT_ROWS), nch), 128 * SPLIT_ROWS, 0, st>>>(B, ldb, N, K, ws.sB, N, ws.eB);
        count_launch(2);
        const cudaError_t e = update(st, M, N, K - KP * (nch - 1), C, ldc, ws, lower, sign, true, nullptr, false, nch);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    for (int k0 = 0; k0 < K; k0 += KP) {
        const int kb = std::min(KP, K - k0);
        split(st, A + k0, lda, M, kb, ws.sA, ws.rowsA, ws.eA);
        split(st, B + k0, ldb, N, kb, ws.sB, ws.rowsB, ws.eB);
        const cudaError_t e = update(st, M, N, kb, C, ldc, ws, lower, sign);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t oz_dgemm(cudaStream_t st, bool trans_a, int M, int N, int K, const double* A, int lda,
                     const double* B, const double* B2, int ldb, double* C, int ldc, const double* E,
                     bool symm, const OzWs& ws) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (!oz_init()) return cudaErrorNotSupported;
    if (M > ws.rowsA || N > ws.rowsB || (symm && M != N)) return cudaErrorInvalidValue;
    if (K <= 0) return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * N, M, st);
    ProfScope prof(st, KC_OZ, (symm ? 1.0 : 2.0) * M * (double)N * K);
    // A^T A (a Gram): one operand split serves both sides
    const bool same_ab = trans_a && A == B && !B2 && lda == ldb && M == N;
    const int nch = cdiv(K, KP);
    if (nch > 1 && (same_ab || (long)nch * M <= ws.rowsA) && (long)nch * N <= ws.rowsB) {
        // every chunk's digits at once, then one update launch over all chunks
        if (!same_ab) {
            if (trans_a)
                k_oz_split_t<<<dim3(cdiv(M, SPLIT_T_ROWS), nch), 128 * SPLIT_T_ROWS, 0, st>>>(A, nullptr, lda, M, 0, K,
                                                                                             ws.sA, M, ws.eA);
            else
                k_oz_split<<<dim3(cdiv(M, SPLIT_ROWS), nch), 128 * SPLIT_ROWS, 0, st>>>(A, lda, M, K, ws.sA, M, ws.eA);
            count_launch();
        }
        k_oz_split_t<<<dim3(cdiv(N, SPLIT_T_ROWS), nch), 128 * SPLIT_T_ROWS, 0, st>>>(B, B2, ldb, N, 0, K, ws.sB,
                                                                                     N, ws.eB);
        count_launch();
        const cudaError_t e = update(st, M, N, K - KP * (nch - 1), C, ldc, ws, symm, 1.0, false, E, same_ab, nch);
        if (e != cudaSuccess) return e;
    } else
    for (int k0 = 0; k0 < K; k0 += KP) {
        const int kb = std::min(KP, K - k0);
        if (same_ab) {
            // nothing: the left operand is read from the right operand's slices
        } else if (trans_a) {
            k_oz_split_t<<<cdiv(M, SPLIT_T_ROWS), 128 * SPLIT_T_ROWS, 0, st>>>(A, nullptr, lda, M, k0, kb, ws.sA,
                                                                               ws.rowsA, ws.eA);
            count_launch();
        } else {
            split(st, A + k0, lda, M, kb, ws.sA, ws.rowsA, ws.eA);
        }
        k_oz_split_t<<<cdiv(N, SPLIT_T_ROWS), 128 * SPLIT_T_ROWS, 0, st>>>(B, B2, ldb, N, k0, kb, ws.sB, ws.rowsB,
                                                                           ws.eB);
        count_launch();
        const cudaError_t e = update(st, M, N, kb, C, ldc, ws, symm, 1.0, k0 > 0, E, same_ab);
        if (e != cudaSuccess) return e;
    }
    if (symm && N > 1) {
        const int nt = cdiv(N, 32);
        k_oz_mirror<<<dim3(nt, nt), 256, 0, st>>>(N, C, ldc);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t oz_gemm_sub(cudaStream_t st, int M, int N, int K, const double* A, int lda, const double* B,
                        int ldb, double* C, int ldc, const OzWs& ws) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (!oz_init()) return cudaErrorNotSupported;
    if (M > ws.rowsA || N > ws.rowsB) return cudaErrorInvalidValue;
    ProfScope prof(st, KC_OZ, 2.0 * M * (double)N * K);
    const int nch = cdiv(K, KP);
    if (nch > 1 && (long)nch * M <= ws.rowsA && (long)nch * N <= ws.rowsB) {
        // every chunk's digits at once, then one update launch over all chunks
        k_oz_split<<<dim3(cdiv(M, SPLIT_ROWS), nch), 128 * SPLIT_ROWS, 0, st>>>(A, lda, M, K, ws.sA, M, ws.eA);
        k_oz_split_t<<<dim3(cdiv(N, SPLIT_T_ROWS), nch), 128 * SPLIT_T_ROWS, 0, st>>>(B, nullptr, ldb, N, 0, K,
                                                                                     ws.sB, N, ws.eB);
        count_launch(2);
        // split K over CTAs when the tiles alone leave most SMs idle
        const long tiles = (long)cdiv(M, BM) * cdiv(N, BN);
        const int groups = (int)std::min<long>(nch, std::max<long>(1, g_num_sm / tiles));
        const cudaError_t e =
            update(st, M, N, K - KP * (nch - 1), C, ldc, ws, false, -1.0, true, nullptr, false, nch, groups);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    for (int k0 = 0; k0 < K; k0 += KP) {
        const int kb = std::min(KP, K - k0);
        split(st, A + k0, lda, M, kb, ws.sA, ws.rowsA, ws.eA);
        // right operand row j = column j of B over the chunk's K rows
        k_oz_split_t<<<cdiv(N, SPLIT_T_ROWS), 128 * SPLIT_T_ROWS, 0, st>>>(B, nullptr, ldb, N, k0, kb, ws.sB,
                                                                           ws.rowsB, ws.eB);
        count_launch();
        const cudaError_t e = update(st, M, N, kb, C, ldc, ws, false, -1.0, true);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

int oz_take_error() {
    int h = 0, z = 0;
    cudaMemcpyFromSymbol(&h, g_oz_error, sizeof(int));
    if (h) cudaMemcpyToSymbol(g_oz_error, &z, sizeof(int));
    return h;
}

}  // namespace thc
