// Dataflow LDL^T of the normal matrix with the forward solve fused (the rows of M are
// carried along as extra rows), in one persistent launch per solve.
//
// Why: the factorisation has one pivot per column on its critical path, and GB300 runs
// FP64 at about two FMA per clock per SM (one warp-instruction per SM sub-partition every
// 64 clocks). A launch per block step serialises the diagonal factorisation, the panel
// substitution and the trailing update, and the diagonal factorisation shares its SM with
// update CTAs that saturate the FP64 pipe. Here one CTA (the chain) owns the critical
// path on an SM of its own, and the other CTAs work through the off-path tiles while it
// runs, so the trailing update of step k overlaps the diagonal work of steps k+1, k+2...
//
// Tiles are FB x FB (FB = 16). With T = ceil(R / FB) column tiles, row tiles 0..T-1 are
// the rows of H and row tiles T.. the appended rows of M. Tasks:
//   F(s)      LDL^T of the diagonal tile (s, s)                       [chain]
//   S(t, k)   X L_kk^T = B for tile (t, k), then L = X D_k^-1            [chain if t = k+1]
//   U(t,j,k)  tile (t, j) -= L(t, k) X(j, k)^T (lower half if t = j)   [chain if t = j = k+1]
// Chain step s runs S(s, s-1), U(s, s, s-1), F(s) back to back in shared memory (warps 0-7
// of the chain CTA; warps 8-14 prefetch its next two tiles, warp 15 publishes its
// progress). The other tasks form one list in a fixed order, split into the critical
// tasks (row tile s on panels s-2, s-3), served by CTAs of their own, and the rest; worker
// groups (128 threads) claim entries with an atomic ticket and wait for their inputs on
// per-tile progress counters:
//   sdone[t] = k + 1 once S(t, k) is stored; cnt[t][j] = number of panels applied to tile
//   (t, j); fdone = s + 1 once F(s) is stored.
// Every tile receives its updates in panel order (a U task waits for the previous panel's
// update of the same tile), so the result does not depend on the schedule: bit-identical
// from run to run.
//
// Progress without deadlock, whatever the number of resident CTAs: the chain role goes to
// the first CTA that starts, tickets are claimed in list order only by running groups, and
// the list order (checked on the host before the first launch) puts every task that the
// chain or a task waits for before the waiting task. So the lowest unfinished ticket can
// always run. Every wait is bounded (1 s); on expiry the kernel raises an abort flag that
// ends all waits, and the host reports ERR_TIMEOUT.
//
// Result layout (same as the blocked factorisation): strictly-lower L and diag(D) in H,
// D^-1 in dinv, Y = M L^-T D^-1 in the appended rows; P (R x R) holds X = L D per tile.
#include <float.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "thc_cpd.h"
#include "f64.cuh"
#include "ldl_common.cuh"
#include "prof.cuh"

namespace thc {

__device__ int g_flow_error = 0;

namespace {

constexpr int FB = 16;
constexpr int kGroups = 4;                 // worker groups (128 threads) per CTA
constexpr int kFlowThreads = 128 * kGroups;
constexpr int kFlowSmem = 120 * 1024;      // more than half an SM: one CTA per SM
constexpr unsigned long long kWaitNs = 1000000000ull;  // default limit of every wait (1 s)
constexpr int kSyncHead = 6;  // ticket, arrivals, fdone, abort, critical ticket, CTAs done
constexpr int kMaxTiles = 256;             // largest schedule the host builds
// Up to 128 tiles (R <= 2048) the dataflow kernel is at least as fast as the blocked
// launches (BF16x3 sweeps measured 5.00 vs 6.28 ms at R = 1080, 9.66 vs 10.54 at 1440,
// 17.55 vs 17.67 at 1800, where the solve turns FP64-throughput bound); beyond, the blocked
// factorisation runs.
constexpr int kFlowMaxTiles = 128;

struct FlowTask {
    short type, t, j, k;                   // type 0: S(t, k); 1: U(t, j, k)
};

// The tasks on the two panels just behind chain step s in row tile s: S(s, s-2),
// U(s, s-1, s-2), U(s, s, s-2), which feed step s directly, and S(s, s-3), U(s, j, s-3)
// (j = s-2, s-1, s), which feed those. They are served by worker groups of their own that
// run alone on their SMs, so that the FP64 pipes they issue to are not shared with three
// other groups (which makes a task several times slower and, here, holds up the chain).
__host__ __device__ __forceinline__ bool critical_task(const FlowTask& x, int nT) {
    return x.t < nT && x.k >= x.t - 3;
}

struct ChainSmem {
    double Lp[FB][FB + 1];   // L of the previous diagonal tile (strictly lower)
    double dp[FB];           // its D^-1
    double Xs[FB][FB + 1];   // X(s, s-1)
    double Ls[FB][FB + 1];   // L(s, s-1)
    double D[FB][FB + 1];    // diagonal tile being factorised
    double L[FB][FB + 1];
    double dinv[FB];
    double x2[FB];           // x2[r] = a(r, r-1)^2 once column r-2 has been applied to it
    double Bn[2][FB][FB + 1];  // tile (s, s-1) for step s, buffer s & 1 (from the producer)
    double Dn[2][FB][FB + 1];  // tile (s, s)
    unsigned short pairs[FB * (FB + 1) / 2];
    int bad;
    int ok;
    int pstat;               // producer: inputs of its current step ready
    volatile int valid[2];   // buffer holds complete tiles (0: the launch is aborting)
    volatile int full[2];    // last step written to buffer b
    volatile int empty[2];   // last step the chain has taken out of buffer b
    volatile int live;       // 0 once the chain is aborting: the publisher releases nothing
    volatile int pub;        // steps whose two barriers (7 and 8) the publisher has passed
};

struct WorkerSmem {
    double A[FB][FB + 1];
    double B[FB][FB + 1];
    int ticket;
    int ok;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void group_sync(int id) {
    asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}

// *p[i] >= v[i] for every i (true), or the launch is aborting / this wait gave up (false).
// The counters are read together: one round trip per poll.
template <int N>
__device__ bool flow_wait(const int* const (&p)[N], const int (&v)[N], int* abort_flag,
                          unsigned long long limit_ns) {
    auto ready = [&]() {
        int x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = ld_acquire(p[i]);
        bool ok = true;
#pragma unroll
        for (int i = 0; i < N; ++i) ok = ok && x[i] >= v[i];
        return ok;
    };
    if (ready()) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0;; ++it) {
        if (it > 8) __nanosleep(40);
        if (ready()) return true;
        if ((it & 31) == 31) {
            if (ld_acquire(abort_flag)) return false;
            if (global_ns() - t0 > limit_ns) {
                atomicExch(abort_flag, 1);
                atomicExch(&g_flow_error, 1);
                return false;
            }
        }
    }
}

constexpr int kPublisher = 224;  // chain thread that reports a failed pivot
constexpr int kProducerThreads = 224;  // warps 8-14 prefetch the chain's tiles
// Warp 15 publishes the chain's progress: after bar.arrive 7 / 8 by the 256 chain threads
// (tile (s, s-1) substituted; tile (s, s) factorised) it fences and releases sdone[s] /
// fdone, so that the fence's latency is not on the chain's path.

// The chain arrives at barriers 7 and 8 without waiting, so before its arrivals of step s
// it makes sure that the publisher has passed both barriers of step s - 1 (S.pub >= s):
// arriving again at a named barrier whose previous phase the publisher has not yet joined
// would complete that phase without the publisher and leave it waiting on a later one.
// The publisher gets there within a fence and a store once the chain has arrived, so the
// wait is normally over at once; it is bounded all the same (error code 2 when it gives
// up).
template <class S_t>
__device__ __forceinline__ void wait_publisher(S_t& S, int s) {
    for (unsigned it = 0; S.pub < s; ++it) {
        if (it == (1u << 26)) {
            atomicExch(&g_flow_error, 2);
            break;
        }
    }
}

// Barrier of the chain's compute threads 0..255 (producer and publisher warps run apart).
__device__ __forceinline__ void chain_sync() { asm volatile("bar.sync 5, 256;" ::: "memory"); }
__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 6, 224;" ::: "memory"); }
__device__ __forceinline__ void chain_arrive_subst() { asm volatile("bar.arrive 7, 288;" ::: "memory"); }
__device__ __forceinline__ void chain_arrive_factor() { asm volatile("bar.arrive 8, 288;" ::: "memory"); }

// Bounded wait for a shared-memory step counter written by the other half of the chain
// CTA: *p >= v (true), or the launch aborts / the wait gives up (false).
__device__ bool smem_wait(const volatile int* p, int v, int* abort_flag, unsigned long long limit_ns) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; *p < v; ++it) {
        if ((it & 63) == 63) {
            if (ld_acquire(abort_flag)) return false;
            if (global_ns() - t0 > limit_ns) {
                atomicExch(abort_flag, 1);
                atomicExch(&g_flow_error, 1);
                return false;
            }
        }
    }
    __threadfence_block();  // what was written before the flag is read after it
    return true;
}

// LDL^T of the jb x jb tile in S.D (lower triangle) into S.L (strictly lower), S.D's
// diagonal and S.dinv. Threads 0..127 compute with a barrier of their own per column.
// Thread 0 carries only the pivot chain, one column ahead: d(c+1) = a(c+1, c+1) -
// a(c+1, c)^2 / d(c) and its reciprocal, with 1/d(c) in a register and a(c+1, c)^2 formed,
// one column earlier, by the thread that finished a(c+1, c). (Each FP64 instruction of a
// warp costs tens of clocks of issue on this part, so the chain thread issues four per
// column and nothing else.) Warps 1-3 apply column c to the rest of the tile over the
// packed pair list, at most two pairs per thread whose operands are all read before
// either is written. A pivot <= tau sets S.bad and continues with 1 (the caller then
// replays the mode with the pseudo-inverse). Ends with a barrier of the chain's threads
// 0..255.
__device__ void factor_tile(ChainSmem& S, int jb, double tau) {
    const int tid = threadIdx.x;
    if (tid < 128) {
        double inv = 0.0;  // thread 0: 1/d(c) of the current column
        if (tid == 0) {
            S.bad = 0;
            double d = S.D[0][0];
            if (!pivot_ok(d, tau)) {
                S.bad = 1;
                d = 1.0;
                S.D[0][0] = d;
            }
            inv = recip_nr(d);
            S.dinv[0] = inv;
            if (jb > 1) {
                const double x = S.D[1][0];
                S.x2[1] = x * x;
            }
        }
        for (int c = 0; c < jb; ++c) {
            asm volatile("bar.sync 1, 128;" ::: "memory");  // dinv[c] and column c are final
            if (tid == 0) {
                if (c + 1 < jb) {
                    double d1 = fma(-S.x2[c + 1], inv, S.D[c + 1][c + 1]);
                    // the check runs beside the reciprocal, off the chain
                    const bool ok = pivot_ok(d1, tau);
                    double r = recip_nr(d1);
                    if (!ok) {
                        S.bad = 1;
                        d1 = 1.0;
                        r = 1.0;
                    }
                    S.D[c + 1][c + 1] = d1;
                    S.dinv[c + 1] = r;
                    inv = r;
                }
            } else if (tid >= 32) {
                // pair (r, s), c < s <= r: L(r, c) = a(r, c) / d(c) when s = c + 1, and
                // a(r, s) -= L(r, c) a(s, c) except for the pivot (c+1, c+1), thread 0's.
                // Column c is read-only in this step and every pair writes its own entry.
                const double inv_c = S.dinv[c];
                const int hi = FB - 1 - c;
                const int npair = hi * (hi + 1) / 2;
                int r[2], ss[2];
                double x[2], y[2], z[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int e = tid - 32 + 96 * k;
                    r[k] = FB;
                    ss[k] = 0;
                    if (e < npair) {
                        const int rs = S.pairs[e];
                        r[k] = rs >> 8;
                        ss[k] = rs & 0xFF;
                    }
                    x[k] = y[k] = z[k] = 0.0;
                    if (r[k] < jb) {
                        x[k] = S.D[r[k]][c];
                        y[k] = S.D[ss[k]][c];
                        if (r[k] != c + 1) z[k] = S.D[r[k]][ss[k]];
                    }
                }
                const double l0 = x[0] * inv_c, l1 = x[1] * inv_c;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (r[k] >= jb) continue;
                    const double l = k ? l1 : l0;
                    if (ss[k] == c + 1) S.L[r[k]][c] = l;
                    if (r[k] == c + 1) continue;
                    const double a = fma(-l, y[k], z[k]);
                    S.D[r[k]][ss[k]] = a;
                    if (r[k] == c + 2 && ss[k] == c + 1) S.x2[r[k]] = a * a;
                }
            }
        }
    }
    chain_sync();
}

struct FlowArgs {
    double* H;              // element (0, 0) of the factorised block; rows ld doubles apart
    double* P;              // X = L D of the block's H rows, same indexing as H
    double* dinv;           // D^-1 of the block's R columns
    int R, nrows, nT, nM;   // columns (and H rows) of the block, all its rows, tile counts
    int ld;                 // row pitch of H and P (R for a whole solve)
    int R_tau;              // order of the whole normal matrix (the pivot threshold's R)
    const FlowTask* tasks;  // [0, nmain): served by the worker CTAs; [nmain, ntasks): the
    int ntasks, nmain;      // critical tasks, served by the critical CTAs
    int ncrit;              // critical CTAs (one group each), roles 1..ncrit
    int* sync;              // nsync progress ints, zero at entry; the last CTA out re-zeroes them
    int nsync;
    DevScalars* sc;
    int mode;
    unsigned long long wait_ns;  // limit of every wait
};

__device__ __forceinline__ int* sdone_of(const FlowArgs& a) { return a.sync + kSyncHead; }
__device__ __forceinline__ int* cnt_of(const FlowArgs& a) {
    return a.sync + kSyncHead + a.nT + a.nM;
}

// Producer warps of the chain CTA (8-14): for steps s = 1..T-1, waits until tiles
// (s, s-1) and (s, s) hold all updates through panel s-2, copies them into buffer s & 1 and
// flags it, so the chain finds them in shared memory; a buffer is reused once the chain
// has taken its previous content out.
__device__ void flow_producer(const FlowArgs& a, ChainSmem& S) {
    const int t2 = threadIdx.x - 256, R = a.R, nT = a.nT;  // 0 .. kProducerThreads - 1
    const size_t ld = a.ld;
    int* abort_flag = a.sync + 3;
    int* cnt = cnt_of(a);
    for (int sn = 1; sn < nT; ++sn) {
        const int b = sn & 1;
        if (t2 == 0) {
            bool ok = sn < 3 || smem_wait(&S.empty[b], sn - 2, abort_flag, a.wait_ns);
            if (ok) {
                const int* const pc[2] = {&cnt[sn * nT + sn - 1], &cnt[sn * nT + sn]};
                const int vc[2] = {sn - 1, sn - 1};
                ok = flow_wait(pc, vc, abort_flag, a.wait_ns);
            }
            S.pstat = ok;
        }
        producer_sync();
        const bool ok = S.pstat;
        if (ok) {
            const int n0 = sn * FB, nb = min(FB, R - n0);
            for (int e = t2; e < FB * FB; e += kProducerThreads) {
                const int rr = e >> 4, cc = e & 15;
                S.Bn[b][rr][cc] = rr < nb ? __ldcg(a.H + (size_t)(n0 + rr) * ld + n0 - FB + cc) : 0.0;
                S.Dn[b][rr][cc] =
                    (rr < nb && cc <= rr) ? __ldcg(a.H + (size_t)(n0 + rr) * ld + n0 + cc) : 0.0;
            }
        }
        producer_sync();
        if (t2 == 0) {
            S.valid[b] = ok;
            __threadfence_block();
            S.full[b] = sn;
        }
        if (!ok) break;
    }
}

// The critical path (threads 0..255): for s = 0..T-1, S(s, s-1), U(s, s, s-1), F(s).
__device__ void flow_chain(const FlowArgs& a, ChainSmem& S) {
    const int tid = threadIdx.x, R = a.R, nT = a.nT;
    const size_t ld = a.ld;
    int* abort_flag = a.sync + 3;
    const double tau = (double)a.R_tau * DBL_EPSILON * a.sc->maxdiag;
    const int r = tid >> 4, c = tid & 15;  // element of a tile
    int bad = 0;
    int s_end = nT;  // the step the loop stopped at (nT: all done)
    for (int s = 0; s < nT; ++s) {
        const int s0 = s * FB, sb = min(FB, R - s0), b = s & 1;
        double dss = 0.0, x = 0.0;
        if (s == 0) {
            if (r < sb && c <= r) dss = __ldcg(a.H + (size_t)r * ld + c);
        } else {
            if (tid == 0) S.ok = smem_wait(&S.full[b], s, abort_flag, a.wait_ns) && S.valid[b];
            chain_sync();
            if (!S.ok) {
                s_end = s;
                break;
            }
            dss = S.Dn[b][r][c];
            x = S.Bn[b][r][c];
            // X L_{s-1}^T = B: column sweep, x[r][q] passed along the row's half-warp
#pragma unroll
            for (int q = 0; q < FB - 1; ++q) {
                const double xq = __shfl_sync(0xffffffffu, x, (tid & 16) | q);
                if (c > q) x = fma(-xq, S.Lp[c][q], x);
            }
            const double l = x * S.dp[c];
            if (r < sb) {
                a.H[(size_t)(s0 + r) * ld + s0 - FB + c] = l;
                a.P[(size_t)(s0 + r) * ld + s0 - FB + c] = x;
            }
            S.Xs[r][c] = x;
            S.Ls[r][c] = l;
            if (tid == 0) wait_publisher(S, s);
            chain_sync();
            if (tid == 0) S.empty[b] = s;  // buffer b read out (before the barrier above)
            chain_arrive_subst();          // the publisher warp releases sdone[s]
            if (c <= r) {
                double a0 = 0.0, a1 = 0.0;
#pragma unroll
                for (int q = 0; q < FB; q += 2) {
                    a0 = fma(S.Ls[r][q], S.Xs[c][q], a0);
                    a1 = fma(S.Ls[r][q + 1], S.Xs[c][q + 1], a1);
                }
                dss -= (a0 + a1);
            }
        }
        S.D[r][c] = dss;
        chain_sync();
        factor_tile(S, sb, tau);
        if (r < sb && c <= r)
            a.H[(size_t)(s0 + r) * ld + s0 + c] = (c < r) ? S.L[r][c] : S.D[r][r];
        if (tid < sb) a.dinv[s0 + tid] = S.dinv[tid];
        S.Lp[r][c] = (c < r && r < sb) ? S.L[r][c] : 0.0;
        if (tid < FB) S.dp[tid] = tid < sb ? S.dinv[tid] : 0.0;
        bad |= S.bad;
        chain_sync();
        chain_arrive_factor();  // the publisher warp releases fdone = s + 1
    }
    if (s_end < nT) {
        // aborting (a wait gave up): run out the publisher's barriers, releasing nothing
        if (tid == 0) S.live = 0;
        for (int s2 = s_end; s2 < nT; ++s2) {
            if (s2 > 0) {
                if (tid == 0) wait_publisher(S, s2);
                chain_sync();
                chain_arrive_subst();
            }
            chain_arrive_factor();
        }
    }
    if (tid == kPublisher && bad) atomicOr(&a.sc->fail_mask, 1 << a.mode);
}

// Warp 15: releases the chain's progress flags (see chain_arrive_*); the fences run here.
__device__ void flow_publisher(const FlowArgs& a, ChainSmem& S) {
    const int lane = threadIdx.x & 31;
    int* fdone = a.sync + 2;
    int* sdone = sdone_of(a);
    for (int s = 0; s < a.nT; ++s) {
        if (s > 0) {
            asm volatile("bar.sync 7, 288;" ::: "memory");
            if (lane == 0 && S.live) {
                __threadfence();
                st_release(&sdone[s], s);
            }
        }
        asm volatile("bar.sync 8, 288;" ::: "memory");
        if (lane == 0 && S.live) {
            __threadfence();
            st_release(fdone, s + 1);
        }
        if (lane == 0) S.pub = s + 1;  // both barriers of step s passed
    }
}

// Rows of row tile t: [r0, rlim) with r0 = first row (H rows, then M rows).
__device__ __forceinline__ void tile_rows(const FlowArgs& a, int t, int& r0, int& rlim) {
    if (t < a.nT) {
        r0 = t * FB;
        rlim = a.R;
    } else {
        r0 = a.R + (t - a.nT) * FB;
        rlim = a.nrows;
    }
}

// S(t, k) by one worker group: thread gt owns column c of rows rr and rr + 8.
__device__ void task_S(const FlowArgs& a, WorkerSmem& W, int gt, int bar, int t, int k) {
    const int R = a.R;
    const size_t ld = a.ld;
    int* sdone = sdone_of(a);
    if (gt == 0) {
        const int* const pc[2] = {a.sync + 2, &cnt_of(a)[t * a.nT + k]};
        const int vc[2] = {k + 1, k};
        W.ok = flow_wait(pc, vc, a.sync + 3, a.wait_ns);
    }
    group_sync(bar);
    if (!W.ok) return;
    int r0, rlim;
    tile_rows(a, t, r0, rlim);
    const int k0 = k * FB, kb = min(FB, R - k0);
    const int c = gt & 15, rr = gt >> 4;
    const int row0 = r0 + rr, row1 = r0 + rr + 8;
    const bool cv = c < kb;
    double b0 = (cv && row0 < rlim) ? __ldcg(a.H + (size_t)row0 * ld + k0 + c) : 0.0;
    double b1 = (cv && row1 < rlim) ? __ldcg(a.H + (size_t)row1 * ld + k0 + c) : 0.0;
    double lr[FB];
#pragma unroll
    for (int q = 0; q < FB; ++q)
        lr[q] = (q < c && cv) ? __ldcg(a.H + (size_t)(k0 + c) * ld + k0 + q) : 0.0;
    const double di = cv ? __ldcg(a.dinv + k0 + c) : 0.0;
    const int src = gt & 16;
#pragma unroll
    for (int q = 0; q < FB - 1; ++q) {
        const double x0 = __shfl_sync(0xffffffffu, b0, src | q);
        const double x1 = __shfl_sync(0xffffffffu, b1, src | q);
        if (c > q) {
            b0 = fma(-x0, lr[q], b0);
            b1 = fma(-x1, lr[q], b1);
        }
    }
    const bool hrow = t < a.nT;
    if (cv && row0 < rlim) {
        a.H[(size_t)row0 * ld + k0 + c] = b0 * di;
        if (hrow) a.P[(size_t)row0 * ld + k0 + c] = b0;
    }
    if (cv && row1 < rlim) {
        a.H[(size_t)row1 * ld + k0 + c] = b1 * di;
        if (hrow) a.P[(size_t)row1 * ld + k0 + c] = b1;
    }
    group_sync(bar);
    if (gt == 0) {
        __threadfence();
        st_release(&sdone[t], k + 1);
    }
}

// U(t, j, k) by one worker group: tile (t, j) -= L(t, k) X(j, k)^T.
__device__ void task_U(const FlowArgs& a, WorkerSmem& W, int gt, int bar, int t, int j, int k) {
    const int R = a.R;
    const size_t ld = a.ld;
    int* sdone = sdone_of(a);
    int* cnt = cnt_of(a);
    if (gt == 0) {
        const int* const pc[3] = {&sdone[t], &sdone[j], &cnt[t * a.nT + j]};
        const int vc[3] = {k + 1, k + 1, k};
        W.ok = flow_wait(pc, vc, a.sync + 3, a.wait_ns);
    }
    group_sync(bar);
    if (!W.ok) return;
    int r0, rlim;
    tile_rows(a, t, r0, rlim);
    const int k0 = k * FB, kb = min(FB, R - k0), c0 = j * FB;
    const int c = gt & 15, rr = gt >> 4;
    const int row0 = r0 + rr, row1 = r0 + rr + 8, col = c0 + c;
    const bool cv = c < kb;
    W.A[rr][c] = (cv && row0 < rlim) ? __ldcg(a.H + (size_t)row0 * ld + k0 + c) : 0.0;
    W.A[rr + 8][c] = (cv && row1 < rlim) ? __ldcg(a.H + (size_t)row1 * ld + k0 + c) : 0.0;
    W.B[rr][c] = (cv && c0 + rr < R) ? __ldcg(a.P + (size_t)(c0 + rr) * ld + k0 + c) : 0.0;
    W.B[rr + 8][c] = (cv && c0 + rr + 8 < R) ? __ldcg(a.P + (size_t)(c0 + rr + 8) * ld + k0 + c) : 0.0;
    const bool diag = t == j;
    const bool v0 = row0 < rlim && col < R && !(diag && c > rr);
    const bool v1 = row1 < rlim && col < R && !(diag && c > rr + 8);
    const double h0 = v0 ? __ldcg(a.H + (size_t)row0 * ld + col) : 0.0;
    const double h1 = v1 ? __ldcg(a.H + (size_t)row1 * ld + col) : 0.0;
    group_sync(bar);
    double s0 = 0.0, s1 = 0.0, u0 = 0.0, u1 = 0.0;
#pragma unroll
    for (int q = 0; q < FB; q += 2) {
        const double b0 = W.B[c][q], b1 = W.B[c][q + 1];
        s0 = fma(W.A[rr][q], b0, s0);
        s1 = fma(W.A[rr][q + 1], b1, s1);
        u0 = fma(W.A[rr + 8][q], b0, u0);
        u1 = fma(W.A[rr + 8][q + 1], b1, u1);
    }
    if (v0) a.H[(size_t)row0 * ld + col] = h0 - (s0 + s1);
    if (v1) a.H[(size_t)row1 * ld + col] = h1 - (u0 + u1);
    group_sync(bar);
    if (gt == 0) {
        __threadfence();
        st_release(&cnt[t * a.nT + j], k + 1);
    }
}

// Worker group loop over tickets [0, count) of `list`, handed out by `counter` in order.
__device__ void flow_worker(const FlowArgs& a, WorkerSmem& W, int g, const FlowTask* list,
                            int count, int* counter) {
    const int gt = threadIdx.x & 127, bar = 1 + g;
    if (gt == 0) W.ticket = atomicAdd(counter, 1);
    group_sync(bar);
    for (;;) {
        const int ti = W.ticket;
        if (ti >= count) break;
        // claim the next ticket while this one runs (holding one in reserve keeps the
        // lowest unfinished ticket runnable: a group works on its lower ticket first)
        int nxt = 0;
        if (gt == 0) nxt = atomicAdd(counter, 1);
        const FlowTask tk = list[ti];
        if (tk.type == 0)
            task_S(a, W, gt, bar, tk.t, tk.k);
        else
            task_U(a, W, gt, bar, tk.t, tk.j, tk.k);
        if (gt == 0) W.ticket = nxt;
        group_sync(bar);
    }
}

__global__ void __launch_bounds__(kFlowThreads, 1) k_ldl_flow(FlowArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int role;
    if (threadIdx.x == 0) role = atomicAdd(a.sync + 1, 1);
    __syncthreads();
    if (role == 0) {
        ChainSmem& S = *reinterpret_cast<ChainSmem*>(smem);
        for (int e = threadIdx.x; e < FB * (FB + 1) / 2; e += blockDim.x) S.pairs[e] = pair_code<FB>(e);
        if (threadIdx.x < FB * FB) S.L[threadIdx.x >> 4][threadIdx.x & 15] = 0.0;
        if (threadIdx.x == 0) {
            S.live = 1;
            S.pub = 0;
        }
        if (threadIdx.x < 2) {
            S.full[threadIdx.x] = 0;
            S.empty[threadIdx.x] = 0;
        }
        __syncthreads();
        if (threadIdx.x < 256)
            flow_chain(a, S);
        else if (threadIdx.x < 256 + kProducerThreads)
            flow_producer(a, S);
        else
            flow_publisher(a, S);
    } else {
        WorkerSmem* ws = reinterpret_cast<WorkerSmem*>(smem);
        const int g = threadIdx.x >> 7;
        if (role <= a.ncrit) {
            // a critical CTA: one group, alone on its SM
            if (g == 0)
                flow_worker(a, ws[0], 0, a.tasks + a.nmain, a.ntasks - a.nmain, a.sync + 4);
        } else {
            flow_worker(a, ws[g], g, a.tasks, a.nmain, a.sync);
        }
    }
    // the last CTA out clears this launch's counters for the next one (no memset node)
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(a.sync + 5, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        for (int i = threadIdx.x; i < a.nsync; i += blockDim.x) a.sync[i] = 0;
    }
}

constexpr size_t kFlowSmemUsed = sizeof(ChainSmem) > kGroups * sizeof(WorkerSmem)
                                     ? sizeof(ChainSmem)
                                     : kGroups * sizeof(WorkerSmem);
static_assert(sizeof(ChainSmem) <= kFlowSmem, "chain shared memory");
static_assert(kGroups * sizeof(WorkerSmem) <= kFlowSmem, "worker shared memory");

// ---- backward solve A L = Y by column slices -------------------------------------------
// Row r of A: a_J = (y_J - sum_{K > J} a_K L_{K,J}) L_JJ^-1 over 32-column blocks J from the
// last to the first (unit lower L). Work item = (row, slice of 4 blocks); each of the 128
// threads owns one column of the slice (its y in a register) and the warp that owns block J
// runs that block's substitution. An item first applies the a_K of all higher blocks as the
// items above publish them (per-row counter prog[r] = blocks solved from the top), then
// solves its own blocks and publishes each. Items are claimed highest slice first, so an item
// only waits for items claimed before it: progress for any number of resident CTAs. Each
// row's work (R^2 / 2 FMA) is spread over R / 128 SMs instead of one.
constexpr int BB = 32;
constexpr int kSliceBlocks = 4;
constexpr int kSlice = BB * kSliceBlocks;
constexpr int kBsThreads = kSlice;

struct BsArgs {
    const double* Yf;
    double* A;
    const double* H;
    int R, n, nJ, C;
    int ld;     // row pitch of Yf, A and H (R for a whole solve)
    int* sync;  // [0] ticket, [1] abort, [2] CTAs done, [3 + r] prog of row r; zero at entry
    unsigned long long wait_ns;
};

// 32-term dot product in four independent FMA chains (fixed order)
__device__ __forceinline__ double dot32(const double* x, const double* h) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
    for (int k = 0; k < BB; k += 4) {
        s0 = fma(x[k], h[k], s0);
        s1 = fma(x[k + 1], h[k + 1], s1);
        s2 = fma(x[k + 2], h[k + 2], s2);
        s3 = fma(x[k + 3], h[k + 3], s3);
    }
    return (s0 + s1) + (s2 + s3);
}

__global__ void __launch_bounds__(kBsThreads) k_bsolve_slices(BsArgs a) {
    __shared__ double as[2][BB];
    __shared__ int tk, kmin, ok, last;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, R = a.R;
    int* abort_flag = a.sync + 1;
    int* prog = a.sync + 3;
    for (;;) {
        if (tid == 0) tk = atomicAdd(a.sync, 1);
        __syncthreads();
        const int t = tk;
        if (t >= a.n * a.C) break;
        const int c = a.C - 1 - t / a.n, r = t % a.n;  // highest slices first
        const int cs = c * kSlice, ce = min(R, cs + kSlice);
        const int Jlo = c * kSliceBlocks, Jhi = min(a.nJ, Jlo + kSliceBlocks);
        const int q = cs + tid;  // this thread's column
        const bool qv = q < ce;
        const size_t ld = a.ld;
        double y = qv ? a.Yf[(size_t)r * ld + q] : 0.0;
        // this warp's diagonal block (if it owns one): column `lane` of L_JJ, in registers
        const int Jw = Jlo + w, c0w = Jw * BB, jbw = min(BB, R - c0w);
        double lc[BB];
#pragma unroll
        for (int k = 0; k < BB; ++k)
            lc[k] = (Jw < Jhi && k > lane && k < jbw) ? __ldg(a.H + (size_t)(c0w + k) * ld + c0w + lane)
                                                     : 0.0;
        // a_K of the higher blocks, as they are published; the L rows are loaded first
        bool good = true;
        int published = a.nJ;  // blocks K >= published are known to be solved
        for (int K = a.nJ - 1; K >= Jhi; --K) {
            const int k0 = K * BB, kb = min(BB, R - k0);
            double hv[BB], av[BB];
#pragma unroll
            for (int k = 0; k < BB; ++k)
                hv[k] = (k < kb && qv) ? __ldg(a.H + (size_t)(k0 + k) * ld + q) : 0.0;
            if (K < published) {
                if (tid == 0) {
                    const int* const pc[1] = {&prog[r]};
                    const int vc[1] = {a.nJ - K};
                    ok = flow_wait(pc, vc, abort_flag, a.wait_ns);
                    kmin = a.nJ - ld_acquire(&prog[r]);
                }
                __syncthreads();
                good = ok;
                published = kmin;
                __syncthreads();  // ok / kmin are rewritten at the next wait
                if (!good) break;
            }
#pragma unroll
            for (int k = 0; k < BB; ++k) av[k] = k < kb ? __ldcg(a.A + (size_t)r * ld + k0 + k) : 0.0;
            y -= dot32(av, hv);
        }
        if (!good) break;
        // own blocks, top to bottom; one barrier per block (a_J double-buffered), the solving
        // warp publishes after the barrier while the next block's warp goes on
        for (int J = Jhi - 1; J >= Jlo; --J) {
            const int c0 = J * BB, jb = min(BB, R - c0), b = J & 1;
            const bool mine = w == J - Jlo;
            if (mine) {
                double v = y;
#pragma unroll
                for (int k = BB - 1; k > 0; --k) {
                    if (k < jb) {  // uniform over the warp
                        const double ak = __shfl_sync(0xffffffffu, v, k);
                        if (lane < k) v = fma(-ak, lc[k], v);
                    }
                }
                y = v;
                as[b][lane] = v;
                if (lane < jb) a.A[(size_t)r * ld + c0 + lane] = v;
            }
            __syncthreads();
            if (mine) {
                if (lane == 0) {
                    __threadfence();
                    st_release(&prog[r], a.nJ - J);
                }
            } else if (qv && q < c0) {
                double hv[BB];
#pragma unroll
                for (int k = 0; k < BB; ++k)
                    hv[k] = k < jb ? __ldg(a.H + (size_t)(c0 + k) * ld + q) : 0.0;
                y -= dot32(as[b], hv);
            }
        }
        __syncthreads();  // tk is rewritten by the next claim
    }
    // the last CTA out clears the counters for the next launch (no memset node)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(a.sync + 2, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        for (int i = tid; i < 3 + a.n; i += blockDim.x) a.sync[i] = 0;
    }
}

// ---- host: the task list ---------------------------------------------------------------
// Ticket order: a diagonal wavefront. S(t, k) sorts at 2k + 1 and U(t, j, k) at j + k, so
// the updates near the diagonal (which the chain needs first) come early and those of
// far columns later, while consecutive updates of one tile stay one position apart (they
// never pile up behind each other). Ties: substitutions first, rows of H before rows of M,
// then panel, column, row. Every task sorts after the tasks it waits for (the check below
// confirms it): a U task's inputs S(t, k), S(j, k) sort at 2k + 1 <= j + k and its previous
// update at j + k - 1; the chain's inputs for step s sort at most at 2s - 2, below the
// tasks that wait for that step (2s + 1 and up).
bool build_tasks(int R, int n, std::vector<FlowTask>& out, int& nT, int& nM) {
    nT = cdiv(R, FB);
    nM = cdiv(n, FB);
    const int nRT = nT + nM;
    std::vector<FlowTask> it;
    auto push = [&](int type, int t, int j, int k) {
        it.push_back(FlowTask{(short)type, (short)t, (short)j, (short)k});
    };
    for (int k = 0; k < nT; ++k) {
        for (int t = k + 2; t < nT; ++t) push(0, t, 0, k);
        for (int t = nT; t < nRT; ++t) push(0, t, 0, k);
        for (int j = k + 1; j < nT; ++j) {
            for (int t = j; t < nT; ++t)
                if (!(t == j && j == k + 1)) push(1, t, j, k);
            for (int t = nT; t < nRT; ++t) push(1, t, j, k);
        }
    }
    auto key = [&](const FlowTask& x) {
        const int tau = x.type == 0 ? 2 * x.k + 1 : x.j + x.k;
        return std::make_tuple(tau, (int)x.type, x.t >= nT ? 1 : 0, (int)x.k, (int)x.j, (int)x.t);
    };
    std::stable_sort(it.begin(), it.end(),
                     [&](const FlowTask& x, const FlowTask& y) { return key(x) < key(y); });
    if (it.size() >= 0x7fffffff) return false;
    // index of every ticket task, -1 for chain tasks or tasks that do not exist
    std::vector<int> sidx((size_t)nRT * nT, -1), uidx((size_t)nRT * nT * nT, -1);
    for (size_t i = 0; i < it.size(); ++i) {
        const FlowTask& x = it[i];
        if (x.type == 0)
            sidx[(size_t)x.t * nT + x.k] = (int)i;
        else
            uidx[((size_t)x.t * nT + x.j) * nT + x.k] = (int)i;
    }
    auto U = [&](int t, int j, int k) { return uidx[((size_t)t * nT + j) * nT + k]; };
    // every row tile below the chain is substituted with every panel (the updates are then
    // complete too: each S task depends on all updates of its tile)
    for (int k = 0; k < nT; ++k)
        for (int t = k + 2; t < nRT; ++t)
            if (sidx[(size_t)t * nT + k] < 0) return false;
    // chain step s waits for U(s, s-1, m) and U(s, s, m), m <= s - 2; wmax[s] = the largest
    // ticket any chain step up to s waits for
    std::vector<int> wmax(nT, -1);
    for (int s = 0; s < nT; ++s) {
        int w = s ? wmax[s - 1] : -1;
        for (int m = 0; m + 2 <= s; ++m) {
            const int a = U(s, s - 1, m), b = U(s, s, m);
            if (a < 0 || b < 0) return false;
            w = std::max(w, std::max(a, b));
        }
        wmax[s] = w;
    }
    // every task's inputs come earlier in the list; a task that waits for chain step s comes
    // after everything chain steps 0..s wait for
    for (size_t i = 0; i < it.size(); ++i) {
        const FlowTask& x = it[i];
        const int me = (int)i;
        if (x.type == 0) {
            for (int m = 0; m < x.k; ++m) {
                const int d = U(x.t, x.k, m);
                if (d < 0 || d >= me) return false;
            }
            if (wmax[x.k] >= me) return false;
        } else {
            const int t = x.t, j = x.j, k = x.k;
            const bool s_t_chain = t < nT && t == k + 1, s_j_chain = j == k + 1;
            if (!s_t_chain) {
                const int d = sidx[(size_t)t * nT + k];
                if (d < 0 || d >= me) return false;
            }
            if (!s_j_chain) {
                const int d = sidx[(size_t)j * nT + k];
                if (d < 0 || d >= me) return false;
            }
            if (k >= 1) {
                const int d = U(t, j, k - 1);
                if (d < 0 || d >= me) return false;
            }
            if (s_j_chain && wmax[k + 1] >= me) return false;
        }
    }
    out.swap(it);
    return true;
}

struct Plan {
    FlowTask* tasks = nullptr;  // main tasks, then the critical ones, each in list order
    int ntasks = 0, nmain = 0, nT = 0, nM = 0, grid = 0, ncrit = 0;
    bool ok = false;
};

thread_local unsigned long long t_wait_ns = kWaitNs;

std::mutex g_plan_mu;
std::map<std::tuple<int, int, int>, Plan> g_plans;  // (device, R, n) -> plan (kept)

const Plan* get_plan(int R, int n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto key = std::make_tuple(dev, R, n);
    auto f = g_plans.find(key);
    if (f != g_plans.end()) return f->second.ok ? &f->second : nullptr;
    Plan& p = g_plans[key];
    if (cdiv(R, FB) > kFlowMaxTiles || cdiv(n, FB) > kMaxTiles) return nullptr;
    std::vector<FlowTask> h;
    if (!build_tasks(R, n, h, p.nT, p.nM)) return nullptr;
    p.ntasks = (int)h.size();
    // split the list into the main and the critical subsequences; each keeps the list
    // order, so the argument for progress (every task comes after all it waits for; a
    // group works on its lower ticket first) holds for each, given one group serves it
    std::stable_partition(h.begin(), h.end(),
                          [&](const FlowTask& x) { return !critical_task(x, p.nT); });
    p.nmain = 0;
    while (p.nmain < p.ntasks && !critical_task(h[p.nmain], p.nT)) ++p.nmain;
    if (p.ntasks > 0) {
        if (cudaMalloc(&p.tasks, sizeof(FlowTask) * h.size()) != cudaSuccess) return nullptr;
        if (cudaMemcpy(p.tasks, h.data(), sizeof(FlowTask) * h.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return nullptr;
    }
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // every SM (measured: 152 CTAs beat 120 and 80 at R = 720; the chain's waits for
    // workers shrink), fewer only when there are fewer tasks than worker groups
    p.grid = (int)std::min<long>(nsm, 1 + std::max<long>(1, ((long)p.nmain + kGroups - 1) / kGroups));
    // four critical CTAs on a full grid (seven critical tasks per chain step), else one
    p.ncrit = p.ntasks > p.nmain ? (p.grid >= 16 ? 4 : 1) : 0;
    p.grid = std::min(nsm, p.grid + p.ncrit);
    if (p.grid < 1 + p.ncrit + (p.nmain > 0 ? 1 : 0)) return nullptr;
    if (cudaFuncSetAttribute(k_ldl_flow, cudaFuncAttributeMaxDynamicSharedMemorySize, kFlowSmem) !=
        cudaSuccess)
        return nullptr;
    p.ok = true;
    return &p;
}

}  // namespace

size_t flow_sync_ints(int R, int nmax) {
    const size_t nT = cdiv(R, FB), nRT = nT + cdiv(nmax, FB);
    return kSyncHead + nRT + nRT * nT;
}

bool flow_prepare(int R, int n) { return get_plan(R, n) != nullptr; }

cudaError_t ldl_flow(cudaStream_t st, int R, int n, double* Haug, double* P, double* dinv,
                     DevScalars* sc, int mode, int* sync, int max_ctas) {
    const Plan* p = get_plan(R, n);
    if (!p) return cudaErrorInvalidValue;
    const int nsync = kSyncHead + (p->nT + p->nM) * (1 + p->nT);
    // alone on the GPU: one CTA per SM (the chain's SM is not shared); next to other
    // problems (max_ctas > 0): a few CTAs with just the shared memory they use, one of them
    // for the critical tasks
    const int ncrit = max_ctas > 0 ? std::min(p->ncrit, 1) : p->ncrit;
    const int grid = max_ctas > 0 ? std::max(2 + ncrit, std::min(p->grid, max_ctas)) : p->grid;
    FlowArgs a{Haug, P, dinv, R, R + n, p->nT, p->nM, R, R, p->tasks, p->ntasks, p->nmain, ncrit,
               sync, nsync, sc, mode, t_wait_ns};
    const int smem = max_ctas > 0 ? (int)kFlowSmemUsed : kFlowSmem;
    k_ldl_flow<<<grid, kFlowThreads, smem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t ldl_flow_tasks(cudaStream_t st, int R, int n, double* Haug, double* P, double* dinv,
                           DevScalars* sc, int mode, int* sync, const short* host_tasks,
                           int ntasks, void* dev_tasks) {
    const Plan* p = get_plan(R, n);  // grid, shared-memory attribute and tile counts
    if (!p || ntasks < 0) return cudaErrorInvalidValue;
    std::vector<FlowTask> h((size_t)ntasks);
    for (int i = 0; i < ntasks; ++i)
        h[i] = FlowTask{host_tasks[4 * i], host_tasks[4 * i + 1], host_tasks[4 * i + 2],
                        host_tasks[4 * i + 3]};
    std::stable_partition(h.begin(), h.end(),
                          [&](const FlowTask& x) { return !critical_task(x, p->nT); });
    int nmain = 0;
    while (nmain < ntasks && !critical_task(h[nmain], p->nT)) ++nmain;
    if (ntasks > 0) {
        const cudaError_t e = cudaMemcpyAsync(dev_tasks, h.data(), sizeof(FlowTask) * h.size(),
                                              cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        // the host vector goes out of scope: the copy must have left it
        const cudaError_t e2 = cudaStreamSynchronize(st);
        if (e2 != cudaSuccess) return e2;
    }
    const int nsync = kSyncHead + (p->nT + p->nM) * (1 + p->nT);
    const int ncrit = ntasks > nmain ? p->ncrit : 0;
    FlowArgs a{Haug, P, dinv, R, R + n, p->nT, p->nM, R, R, (const FlowTask*)dev_tasks, ntasks,
               nmain, ncrit, sync, nsync, sc, mode, t_wait_ns};
    k_ldl_flow<<<p->grid, kFlowThreads, kFlowSmem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

int flow_task_check(int R, int n, const short* tasks, int ntasks) {
    const int nT = cdiv(R, FB), nRT = nT + cdiv(n, FB);
    for (int i = 0; i < ntasks; ++i) {
        const short* x = tasks + 4 * i;
        if (x[0] != 0 && x[0] != 1) return i;
        if (x[1] < 0 || x[1] >= nRT || x[3] < 0 || x[3] >= nT) return i;
        if (x[0] == 1 && (x[2] < 0 || x[2] >= nT)) return i;
    }
    return -1;
}

void flow_set_wait_ns(unsigned long long ns) { t_wait_ns = ns ? ns : kWaitNs; }

cudaError_t ldl_flow_panel(cudaStream_t st, int R, int n, int j0, int bw, double* Haug, double* P,
                           double* dinv, DevScalars* sc, int mode, int* sync, int max_ctas) {
    const int below = R + n - j0 - bw;
    const Plan* p = get_plan(bw, below);
    if (!p) return cudaErrorInvalidValue;
    const int nsync = kSyncHead + (p->nT + p->nM) * (1 + p->nT);
    const size_t off = (size_t)j0 * R + j0;
    // as ldl_flow: next to other problems (max_ctas > 0) a few CTAs with just the shared
    // memory they use, one of them for the critical tasks
    const int ncrit = max_ctas > 0 ? std::min(p->ncrit, 1) : p->ncrit;
    const int grid = max_ctas > 0 ? std::max(2 + ncrit, std::min(p->grid, max_ctas)) : p->grid;
    const int smem = max_ctas > 0 ? (int)kFlowSmemUsed : kFlowSmem;
    FlowArgs a{Haug + off, P + off, dinv + j0, bw, bw + below, p->nT, p->nM, R, R, p->tasks,
               p->ntasks, p->nmain, ncrit, sync, nsync, sc, mode, t_wait_ns};
    k_ldl_flow<<<grid, kFlowThreads, smem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

size_t bsolve_sync_ints(int nmax) { return 3 + (size_t)nmax; }

cudaError_t bsolve_slices(cudaStream_t st, int R, int n, const double* Yf, double* A,
                          const double* H, int* sync, int ld) {
    if (n <= 0) return cudaSuccess;
    const int nJ = cdiv(R, BB), C = cdiv(R, kSlice);
    BsArgs a{Yf, A, H, R, n, nJ, C, ld > 0 ? ld : R, sync, t_wait_ns};
    const int grid = std::min(n * C, num_sms() * 4);
    k_bsolve_slices<<<grid, kBsThreads, 0, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

int flow_take_error() {
    int h = 0, z = 0;
    cudaMemcpyFromSymbol(&h, g_flow_error, sizeof(int));
    if (h) cudaMemcpyToSymbol(g_flow_error, &z, sizeof(int));
    return h;
}

}  // namespace thc

extern "C" int thc_cpd_ldl_schedule(int R, int n, short* out, int cap) {
    using namespace thc;
    if (R < 1 || n < 0 || cdiv(R, FB) > kMaxTiles || cdiv(n, FB) > kMaxTiles) return -1;
    std::vector<FlowTask> h;
    int nT = 0, nM = 0;
    if (!build_tasks(R, n, h, nT, nM)) return -1;
    if (out) {
        const size_t m = std::min(h.size(), (size_t)std::max(cap, 0));
        for (size_t i = 0; i < m; ++i) {
            out[4 * i] = h[i].type;
            out[4 * i + 1] = h[i].t;
            out[4 * i + 2] = h[i].j;
            out[4 * i + 3] = h[i].k;
        }
    }
    return (int)h.size();
}
