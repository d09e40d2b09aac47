// spiir_plain.cu -- FP32 per-sample SPIIR kernels for sm_103a.
//
//   prologue   move each level's strain history to the front of its buffer
//              and append the pushed base-rate samples;
//   decimate   the x2 decimation cascade (Sec. 2.2, Eq. kaiser_window_filtering,
//              causal T-tap form);
//   recur      the filter recursion y_k[n] = a_k y_k[n-1] + b_k x[n-d_k]
//              (Eq. iireq0) and the sum over a template's filters
//              (Eq. iireq1), every level in one launch;
//   combine    sum of a unit's parts, x2 upsampling of the next lower rate
//              and the upstream sum, level by level (Sec. 2.2, Fig. 1), and
//              the 2*dt scale.
//
// Recursion kernel layout. A CTA stages its level's strain window (history
// plus a segment of the push) into shared memory with one bulk async copy
// (cp.async.bulk + mbarrier). Each lane owns F filter slots whose state
// (y), pole and gain sit in registers for the whole push; two slots are
// updated together with packed f32x2 FMA. Each filter reads its delayed input
// straight from the window at its own offset (the packer spreads the offsets
// of one round over the 32 shared-memory banks). Every lane accumulates its
// filters' sum for T consecutive samples, then the lanes of a unit reduce
// those T sums with a butterfly reduce-scatter (shuffles in a fixed order,
// no atomics; a full-warp unit with T = 32 goes through the warp's shared-
// memory rows instead), which leaves each lane holding whole sums for T/G
// samples.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "spiir_internal.h"

// Reduction of a unit's per-lane sums, chosen at compile time so that the
// paper's alternatives (Sec. 3.1.3: shuffle or shared-memory reduction,
// cross-warp direct atomics) can be rebuilt and timed against the adopted
// one:
//   0  adopted: shared-memory column sums for full-warp units of 32-sample
//      tiles, shuffle butterfly for smaller groups, ordered hand-off across
//      the warps of a unit;
//   1  shuffle butterfly for every group size;
//   2  shared-memory column sums for every group of 2 or more lanes
//      (32-sample tiles);
//   3  as 0, but the warps of a multi-warp unit add their sums into the
//      output row with atomics (the rows are zeroed before the kernel; the
//      order of the additions, and so the last bits, vary from run to run).
#ifndef SPIIR_REDUCE_ABLATION
#define SPIIR_REDUCE_ABLATION 0
#endif

namespace {

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy helpers (inline PTX)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(m))
        : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for an mbarrier phase for at most ~2 s; on timeout record it in the
// status word and report failure instead of hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *m, uint32_t parity,
                                                  unsigned int *status) {
    if (mbar_try_wait(m, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(m, parity)) return true;
        if (globaltimer_ns() - t0 > 2000000000ull) {
            atomicExch(status, SPIIR_DEV_TIMEOUT);
            return false;
        }
    }
}

// ---------------------------------------------------------------------------
// Prologue: strain history + new base-rate samples
// ---------------------------------------------------------------------------

// One CTA per (level, stream) moves the level's history; the new base-rate
// samples, whose places overlap the history's sources, are copied by the
// next kernel with a grid wide enough for the push.
__global__ void prologue_kernel(const PrologueArgs a) {
    const int lev = blockIdx.x;
    const int s = a.stream0 + blockIdx.y;
    if (lev == 0 && a.prog) {
        // fresh work queue and segment progress for this push
        if (threadIdx.x == 0) a.queue[s] = 0u;
        for (int k = threadIdx.x; k < a.n_items; k += blockDim.x)
            a.prog[(int64_t)s * a.n_items + k] = 0u;
    }
    const LevelArgs L = a.lev[lev];
    float *buf = a.xbuf + (int64_t)s * a.xbuf_stream_stride + L.xbuf_off;
    const int hist = L.hist, np = L.n_prev;
    if (np > 0 && hist > 0) {
        // buf[0, hist) <- buf[np, np + hist); chunks of np samples so that a
        // chunk's sources are read before the next chunk overwrites them.
        for (int c0 = 0; c0 < hist; c0 += np) {
            const int len = min(np, hist - c0);
            for (int k = threadIdx.x; k < len; k += blockDim.x) buf[c0 + k] = buf[c0 + np + k];
            __syncthreads();
        }
    }
}

// The push's base-rate samples behind level 0's history, every stream.
__global__ void prologue_copy_kernel(const PrologueArgs a) {
    const LevelArgs L = a.lev[0];
    float *buf = a.xbuf + (int64_t)(a.stream0 + blockIdx.y) * a.xbuf_stream_stride + L.xbuf_off + L.hist;
    const float *src = a.x_in + (int64_t)blockIdx.y * a.x_in_stream_stride;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L.n; k += gridDim.x * blockDim.x) buf[k] = src[k];
}

// ---------------------------------------------------------------------------
// Decimation cascade: x_{i+1}[m] = sum_j h[j] x_i[2m - j]
// ---------------------------------------------------------------------------

__global__ void decimate_kernel(const DecimArgs a) {
    const int s = a.stream0 + blockIdx.x;
    float *base = a.xbuf + (int64_t)s * a.xbuf_stream_stride;
    __shared__ float h[SPIIR_MAX_DOWN_TAPS];
    for (int j = threadIdx.x; j < a.n_taps; j += blockDim.x) h[j] = a.h_down[j];
    __syncthreads();
    for (int i = 1; i < a.n_levels; ++i) {
        const LevelArgs Ls = a.lev[i - 1], Ld = a.lev[i];
        const float *src = base + Ls.xbuf_off + Ls.hist;
        float *dst = base + Ld.xbuf_off + Ld.hist;
        for (int m = threadIdx.x; m < Ld.n; m += blockDim.x) {
            const float *p = src + 2 * m;
            // two interleaved partial sums (taps are even in number): shorter
            // dependency chains for long decimators
            float acc0 = 0.f, acc1 = 0.f;
            for (int j = 0; j < a.n_taps; j += 2) {
                acc0 = fmaf(h[j], p[-j], acc0);
                acc1 = fmaf(h[j + 1], p[-j - 1], acc1);
            }
            dst[m] = acc0 + acc1;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Recursion kernel (persistent, dynamically scheduled)
//
// Work items are (CTA item, time segment) pairs taken from a per-stream
// atomic queue in segment-major order. Segment s of an item starts only after
// segment s-1 of the same item has finished (a progress counter with
// acquire/release ordering); the filter state travels through global memory
// between segments, so an item's segments may run on different SMs. This
// keeps every SM busy whatever the number and size of the items, and every
// wait is on an item that a running CTA took earlier from the queue.
// ---------------------------------------------------------------------------

constexpr int kRedBytes = 2 * SPIIR_CTA_WARPS * 32 * 2 * 4;   // cross-warp sums, 2 buffers
constexpr int kRowPitch = 33;                                  // float2 per staged row (padded)
constexpr int kScratchBytes = SPIIR_CTA_WARPS * 32 * kRowPitch * 8;   // small-unit output rows

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void named_bar(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Wait (at most ~2 s) until *p >= want; on timeout record it and go on.
__device__ __forceinline__ bool wait_counter(const unsigned int *p, unsigned int want,
                                             unsigned int *status) {
    if (ld_acquire(p) >= want) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        __nanosleep(100);
        if (ld_acquire(p) >= want) return true;
        if (globaltimer_ns() - t0 > 2000000000ull) {
            atomicExch(status, SPIIR_DEV_TIMEOUT);
            return false;
        }
    }
}

template <int PMAX>
struct Regs {
    float2 are[PMAX], aim[PMAX], naim[PMAX], bre[PMAX], bim[PMAX], yre[PMAX], yim[PMAX];
    int off0[PMAX], off1[PMAX];
};

// Pairwise (tree-ordered) sum of v[LO..HI): a log-depth dependency chain.
template <int LO, int HI>
__device__ __forceinline__ float2 tree_sum(const float2 *v) {
    if constexpr (HI - LO == 1) {
        return v[LO];
    } else {
        constexpr int MID = (LO + HI) / 2;
        return __fadd2_rn(tree_sum<LO, MID>(v), tree_sum<MID, HI>(v));
    }
}

// One time tile of T samples for P slot pairs; sre/sim receive this lane's
// per-sample sums over its filters. tl < T marks a ragged last tile.
template <int T, int PMAX, int P, bool FULL>
__device__ __forceinline__ void tile(const float *__restrict__ xs, int tb, int tl,
                                     Regs<PMAX> &r, float (&sre)[T], float (&sim)[T]) {
#pragma unroll
    for (int j = 0; j < T; ++j) {
        if (FULL || j < tl) {
            float2 nr[P], ni[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float2 X = make_float2(xs[r.off0[p] + tb + j], xs[r.off1[p] + tb + j]);
                const float2 tr = __fmul2_rn(r.bre[p], X);
                const float2 ti = __fmul2_rn(r.bim[p], X);
                float2 a = __ffma2_rn(r.are[p], r.yre[p], tr);
                a = __ffma2_rn(r.naim[p], r.yim[p], a);
                float2 b = __ffma2_rn(r.are[p], r.yim[p], ti);
                b = __ffma2_rn(r.aim[p], r.yre[p], b);
                r.yre[p] = a;
                r.yim[p] = b;
                nr[p] = a;
                ni[p] = b;
            }
            const float2 accr = tree_sum<0, P>(nr);
            const float2 acci = tree_sum<0, P>(ni);
            sre[j] = accr.x + accr.y;
            sim[j] = acci.x + acci.y;
        } else {
            sre[j] = 0.f;
            sim[j] = 0.f;
        }
    }
}

// Butterfly reduce-scatter over lane groups: round with stride S exchanges
// half of the LEN live values with lane^S and adds; once one value is left
// the remaining rounds are plain pairwise sums.
template <int T, int LEN, int S>
__device__ __forceinline__ void rs_round(float (&re)[T], float (&im)[T], int lane) {
    if constexpr (S >= 1) {
        if constexpr (LEN >= 2) {
            const bool up = (lane & S) != 0;
#pragma unroll
            for (int i = 0; i < LEN / 2; ++i) {
                const float sr = up ? re[i] : re[i + LEN / 2];
                const float kr = up ? re[i + LEN / 2] : re[i];
                const float si = up ? im[i] : im[i + LEN / 2];
                const float ki = up ? im[i + LEN / 2] : im[i];
                re[i] = kr + __shfl_xor_sync(0xffffffffu, sr, S);
                im[i] = ki + __shfl_xor_sync(0xffffffffu, si, S);
            }
            rs_round<T, LEN / 2, S / 2>(re, im, lane);
        } else {
            re[0] += __shfl_xor_sync(0xffffffffu, re[0], S);
            im[0] += __shfl_xor_sync(0xffffffffu, im[0], S);
            rs_round<T, 1, S / 2>(re, im, lane);
        }
    }
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// Where one warp's reduction ends up and what it spans.
struct OutCtx {
    float2 *row;      // destination row at this segment's first sample
    float scale;
    bool valid;
    int xw_log2, xw_rank, warp;
    int n_tiles;      // tiles in this segment (for the cross-warp hand-off)
    float *red;       // cross-warp buffers in shared memory
    float2 *scratch;  // per-warp rows: small units' output staging, full-warp sums
};

// After the reduce-scatter for group size G a lane holds CH = max(T/G, 1)
// consecutive sums; when G > T, 2^NR lanes hold the same sums and the first
// of them writes. Units spanning several warps hand their sums to rank 0
// through two shared-memory buffers: the other ranks arrive on FULL[b]
// without waiting, rank 0 waits on FULL[b], adds in rank order, and arrives on
// EMPTY[b]; a rank waits on EMPTY[b] only before reusing buffer b.
template <int T, int G>
__device__ __forceinline__ void reduce_write(float (&re)[T], float (&im)[T], int lane, int tl,
                                             int t0, int tile, const OutCtx &o) {
    constexpr int kAbl = SPIIR_REDUCE_ABLATION;
    if constexpr (kAbl == 2 && T == 32 && G >= 2 && G < 32) {
        // shared-memory column sums for a group of G lanes: lane l of group g
        // sums columns (l % G) CH .. (l % G) CH + CH - 1 over the group's rows
        constexpr int CHs = T / G;
        float2 *sc = o.scratch + o.warp * (32 * kRowPitch);
#pragma unroll
        for (int i = 0; i < T; ++i) sc[lane * kRowPitch + i] = make_float2(re[i], im[i]);
        __syncwarp();
        const int g0 = lane & ~(G - 1), c0 = (lane & (G - 1)) * CHs;
        float ar[CHs], ai[CHs];
#pragma unroll
        for (int i = 0; i < CHs; ++i) ar[i] = ai[i] = 0.f;
#pragma unroll
        for (int q = 0; q < G; ++q)
#pragma unroll
            for (int i = 0; i < CHs; ++i) {
                const float2 v = sc[(g0 + q) * kRowPitch + c0 + i];
                ar[i] += v.x;
                ai[i] += v.y;
            }
#pragma unroll
        for (int i = 0; i < CHs; ++i) {
            re[i] = ar[i];
            im[i] = ai[i];
        }
        __syncwarp();
    } else if constexpr (kAbl != 1 && T == 32 && G == 32) {
        // A whole warp sums each of the 32 samples: through the warp's
        // shared-memory rows (lane l stores its 32 sums in row l, then sums
        // column l over the rows in lane order) this takes 32 stores, 32 loads
        // and 31 adds per lane and value pair, about half the instructions of
        // the five-round butterfly.
        float2 *sc = o.scratch + o.warp * (32 * kRowPitch);
#pragma unroll
        for (int i = 0; i < T; ++i) sc[lane * kRowPitch + i] = make_float2(re[i], im[i]);
        __syncwarp();
        float ar = 0.f, ai = 0.f;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const float2 v = sc[q * kRowPitch + lane];
            ar += v.x;
            ai += v.y;
        }
        re[0] = ar;
        im[0] = ai;
        __syncwarp();
    } else {
        rs_round<T, T, G / 2>(re, im, lane);
    }
    constexpr int NS = ilog2(G < T ? G : T);
    constexpr int NR = ilog2(G) - NS;
    constexpr int CH = (T / G) > 1 ? (T / G) : 1;
    if constexpr (G == 32 && kAbl == 3) {
        if (o.xw_log2 > 0) {
            // every warp of the unit adds its sums into the zeroed row (each
            // rank has the unit's destination in this build)
            if (!o.valid) return;
            if ((lane & ((1 << NR) - 1)) != 0) return;
            float2 *row = o.row + t0;
            const int tc = ((lane & (G - 1)) >> NR) * CH;
#pragma unroll
            for (int i = 0; i < CH; ++i)
                if (tc + i < tl) {
                    atomicAdd(&row[tc + i].x, o.scale * re[i]);
                    atomicAdd(&row[tc + i].y, o.scale * im[i]);
                }
            return;
        }
    }
    if constexpr (G == 32 && kAbl != 3) {
        if (o.xw_log2 > 0) {
            const int nw = 1 << o.xw_log2;
            const int first = o.warp - o.xw_rank;
            const int b = tile & 1;
            const int base = 1 + 4 * (first >> 1);     // FULL0, FULL1, EMPTY0, EMPTY1
            const int n = 32 * nw;
            if (o.xw_rank > 0) {
                if (tile >= 2) named_bar(base + 2 + b, n);      // buffer b free again
                float *mine = o.red + ((b * SPIIR_CTA_WARPS + o.warp) * 32 + lane) * (2 * CH);
#pragma unroll
                for (int i = 0; i < CH; ++i) {
                    mine[2 * i] = re[i];
                    mine[2 * i + 1] = im[i];
                }
                named_arrive(base + b, n);
                return;
            }
            named_bar(base + b, n);
            for (int w = 1; w < nw; ++w) {
                const float *other =
                    o.red + ((b * SPIIR_CTA_WARPS + first + w) * 32 + lane) * (2 * CH);
#pragma unroll
                for (int i = 0; i < CH; ++i) {
                    re[i] += other[2 * i];
                    im[i] += other[2 * i + 1];
                }
            }
            if (tile + 2 < o.n_tiles) named_arrive(base + 2 + b, n);
        }
    }
    if constexpr (T == 32 && G <= 4) {
        // Groups of up to 4 lanes: a lane holds CH = 32 / G consecutive sums
        // of its group's row, so a direct store would scatter over 8 to 32
        // rows at a stride of CH samples. Stage the warp's rows in shared
        // memory and write each row with one 256-byte store of the whole
        // warp. (Larger groups gain nothing from it.)
        float2 *sc = o.scratch + o.warp * (32 * kRowPitch);
        const int grp = lane / G, tcs = (lane & (G - 1)) * CH;
#pragma unroll
        for (int i = 0; i < CH; ++i)
            sc[grp * kRowPitch + tcs + i] = make_float2(o.scale * re[i], o.scale * im[i]);
        __syncwarp();
        const unsigned long long rowbits = reinterpret_cast<unsigned long long>(o.row);
#pragma unroll
        for (int r = 0; r < 32 / G; ++r) {
            const unsigned long long rb = __shfl_sync(0xffffffffu, rowbits, r * G);
            const int v = __shfl_sync(0xffffffffu, (int)o.valid, r * G);
            if (v && lane < tl) reinterpret_cast<float2 *>(rb)[t0 + lane] = sc[r * kRowPitch + lane];
        }
        __syncwarp();
        return;
    }
    if (!o.valid) return;
    if ((lane & ((1 << NR) - 1)) != 0) return;
    const int tc = ((lane & (G - 1)) >> NR) * CH;
    float2 *row = o.row + t0;
#pragma unroll
    for (int i = 0; i < CH; ++i)
        if (tc + i < tl) row[tc + i] = make_float2(o.scale * re[i], o.scale * im[i]);
}

template <int T, int PMAX, int P>
__device__ __forceinline__ void run_segment(const float *__restrict__ xs, int seg_len,
                                            Regs<PMAX> &r, int lane, int g, const OutCtx &o) {
    int k = 0;
    for (int t0 = 0; t0 < seg_len; t0 += T, ++k) {
        const int tl = min(T, seg_len - t0);
        float sre[T], sim[T];
        if (tl == T)
            tile<T, PMAX, P, true>(xs, t0, T, r, sre, sim);
        else
            tile<T, PMAX, P, false>(xs, t0, tl, r, sre, sim);
        switch (g) {
            case 0: reduce_write<T, 1>(sre, sim, lane, tl, t0, k, o); break;
            case 1: reduce_write<T, 2>(sre, sim, lane, tl, t0, k, o); break;
            case 2: reduce_write<T, 4>(sre, sim, lane, tl, t0, k, o); break;
            case 3: reduce_write<T, 8>(sre, sim, lane, tl, t0, k, o); break;
            case 4: reduce_write<T, 16>(sre, sim, lane, tl, t0, k, o); break;
            default: reduce_write<T, 32>(sre, sim, lane, tl, t0, k, o); break;
        }
    }
}

template <int T, int PMAX, int P>
__device__ __forceinline__ void dispatch_segment(int p_runtime, const float *xs, int seg_len,
                                                 Regs<PMAX> &r, int lane, int g,
                                                 const OutCtx &o) {
    if constexpr (P <= PMAX) {
        if (p_runtime == P)
            run_segment<T, PMAX, P>(xs, seg_len, r, lane, g, o);
        else
            dispatch_segment<T, PMAX, P + 1>(p_runtime, xs, seg_len, r, lane, g, o);
    }
}

template <int T, int FMAX, int MINB>
__global__ void __launch_bounds__(SPIIR_CTA_WARPS * 32, MINB) recur_kernel(const RecurArgs a) {
    constexpr int PMAX = FMAX / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    float *red = reinterpret_cast<float *>(smem + 16);
    float2 *scratch = reinterpret_cast<float2 *>(smem + 16 + kRedBytes);
    float *xs = reinterpret_cast<float *>(smem + 16 + kRedBytes + kScratchBytes);
    __shared__ int s_item;

    const int stream = a.stream0 + blockIdx.y;
    unsigned int *queue = a.queue + stream;
    unsigned int *prog = a.prog + (int64_t)stream * a.n_items;
    const int total = a.n_segs * a.n_items;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *st = a.state + (int64_t)stream * a.n_slots;

    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int q = s_item;
        if (q >= total) break;
        const int seg = q / a.n_items;
        const int gi = a.order[q - seg * a.n_items];
        const CtaItem item = a.items[gi];
        const LevelArgs L = a.lev[item.level];
        const int s0 = seg * L.seg;
        const int sl = min(L.seg, L.n - s0);
        // in the failure-detection test the first item is dropped, so the
        // wait of the item after it has to give up
        const bool dropped = a.stall_test && q == 0;
        if (seg > 0 && threadIdx.x == 0) wait_counter(prog + gi, (unsigned)seg, a.status);
        __syncthreads();
        if (sl > 0 && !dropped) {
            const float *xlev = a.xbuf + (int64_t)stream * a.xbuf_stream_stride + L.xbuf_off;
            if (threadIdx.x == 0) {
                const uint32_t bytes = (uint32_t)(((L.hist + sl) * 4 + 15) & ~15);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(mbar, bytes);
                bulk_g2s(xs, xlev + s0, bytes, mbar);
            }
            const bool ok = mbar_wait_bounded(mbar, phase, a.status);
            phase ^= 1u;
            const bool active = ok && warp < item.task_count;
            if (active) {
                const WarpTask wt = a.tasks[item.task_begin + warp];
                const int P = wt.F / 2;
                Regs<PMAX> r;
#pragma unroll
                for (int p = 0; p < PMAX; ++p) {
                    if (p < P) {
                        const int64_t i0 = wt.slot_base + (int64_t)(2 * p) * 32 + lane, i1 = i0 + 32;
                        r.are[p] = make_float2(a.a_re[i0], a.a_re[i1]);
                        r.aim[p] = make_float2(a.a_im[i0], a.a_im[i1]);
                        r.naim[p] = make_float2(-r.aim[p].x, -r.aim[p].y);
                        r.bre[p] = make_float2(a.b_re[i0], a.b_re[i1]);
                        r.bim[p] = make_float2(a.b_im[i0], a.b_im[i1]);
                        const float2 y0 = __ldcg(st + i0), y1 = __ldcg(st + i1);
                        r.yre[p] = make_float2(y0.x, y1.x);
                        r.yim[p] = make_float2(y0.y, y1.y);
                        r.off0[p] = a.xoff[i0];
                        r.off1[p] = a.xoff[i1];
                    } else {
                        r.are[p] = r.aim[p] = r.naim[p] = r.bre[p] = r.bim[p] = make_float2(0.f, 0.f);
                        r.yre[p] = r.yim[p] = make_float2(0.f, 0.f);
                        r.off0[p] = r.off1[p] = 0;
                    }
                }
                OutCtx o;
                o.row = nullptr;
                o.scale = 1.f;
                o.valid = false;
                o.xw_log2 = wt.xw_log2;
                o.xw_rank = wt.xw_rank;
                o.warp = warp;
                o.n_tiles = (sl + T - 1) / T;
                o.red = red;
                o.scratch = scratch;
                const int grp = lane >> wt.g_log2;
                if (grp < wt.n_groups && (wt.xw_rank == 0 || SPIIR_REDUCE_ABLATION == 3)) {
                    const int dst = a.task_out[wt.out_base + grp];
                    o.valid = true;
                    if (dst >= 0) {
                        o.row = a.z + (int64_t)stream * a.z_stream_stride + (int64_t)dst * a.z_row_stride;
                        o.scale = a.scale;
                    } else {
                        o.row = a.partial + (int64_t)stream * a.partial_stream_stride + L.part_base +
                                (int64_t)(-dst - 1) * L.part_stride;
                    }
                    o.row += s0;
                }
                if (P > 0) dispatch_segment<T, PMAX, 1>(P, xs, sl, r, lane, wt.g_log2, o);
#pragma unroll
                for (int p = 0; p < PMAX; ++p) {
                    if (p < P) {
                        const int64_t i0 = wt.slot_base + (int64_t)(2 * p) * 32 + lane, i1 = i0 + 32;
                        st[i0] = make_float2(r.yre[p].x, r.yim[p].x);
                        st[i1] = make_float2(r.yre[p].y, r.yim[p].y);
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && !dropped) {
            __threadfence();
            st_release(prog + gi, (unsigned)(seg + 1));
        }
    }
}

// ---------------------------------------------------------------------------
// Combine: parts + upsample(next lower rate) + scale
// ---------------------------------------------------------------------------

// One CTA per (template, stream) runs the whole level chain of a push in
// time chunks of C base-rate samples (C >> H a multiple of 4). Level i >= 1
// keeps its upsampler input in shared memory as [SPIIR_UHIST history |
// C >> i samples]; the history carries across chunks in shared memory and
// across pushes in a SPIIR_UHIST-long global row. At the start of a chunk one
// thread stages the first unit part of every level into shared memory with
// bulk async copies (all levels in flight at once); then, from the lowest
// rate up:
//   u_H[n] = sum of the unit parts
//   u_i[n] = sum of the unit parts + 2 sum_j h_up[2j + (n&1)] u_{i+1}[n/2 - j]
//   z[n]   = scale * u_0[n]
// A thread makes 4 consecutive outputs 4q..4q+3 (lower-rate samples 2q and
// 2q+1) from one window of the lower level held in registers, so only the
// unit parts and z touch HBM.
constexpr int kCombThreads = 256;

// Shared-memory layout of the combine CTA, in float2 units after a 16-byte
// mbarrier slot: the upsampler buffers of levels 1..H, each SPIIR_UHIST + 2 +
// (C >> i) long, then the part stage of levels 0..H, C >> i each. C is a
// multiple of 4 << H, so every length is a multiple of 2 (16-byte aligned).
__host__ __device__ __forceinline__ int comb_ubuf_off(int chunk, int i) {   // i >= 1
    return (i - 1) * (SPIIR_UHIST + 2) + chunk - (chunk >> (i - 1));
}
__host__ __device__ __forceinline__ int comb_stage_off(int chunk, int H, int i) {
    return comb_ubuf_off(chunk, H + 1) + 2 * chunk - 2 * (chunk >> i);
}

// u_lo: lower-level buffer at its sample 0 (history at negative indices).
template <int HT>
__device__ __forceinline__ void upsample_quad(const float2 *u_lo, int q, const float (&h0)[32],
                                              const float (&h1)[32], int ht,
                                              float2 (&o)[4]) {
    if constexpr (HT > 0 && (HT % 2) == 0) {
        // w[k] = u[2q - HT + k], k < HT + 2, loaded two samples at a time
        float2 w[HT + 2];
        const float4 *src = reinterpret_cast<const float4 *>(u_lo + 2 * q - HT);
#pragma unroll
        for (int k = 0; k < HT / 2 + 1; ++k) {
            const float4 v = src[k];
            w[2 * k] = make_float2(v.x, v.y);
            w[2 * k + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int j = 0; j < HT; ++j) {
            const float2 a0 = w[HT - j], a1 = w[HT + 1 - j];   // u[2q - j], u[2q + 1 - j]
            o[0].x = fmaf(h0[j], a0.x, o[0].x);
            o[0].y = fmaf(h0[j], a0.y, o[0].y);
            o[1].x = fmaf(h1[j], a0.x, o[1].x);
            o[1].y = fmaf(h1[j], a0.y, o[1].y);
            o[2].x = fmaf(h0[j], a1.x, o[2].x);
            o[2].y = fmaf(h0[j], a1.y, o[2].y);
            o[3].x = fmaf(h1[j], a1.x, o[3].x);
            o[3].y = fmaf(h1[j], a1.y, o[3].y);
        }
    } else {
        for (int j = 0; j < ht; ++j) {
            const float2 a0 = u_lo[2 * q - j], a1 = u_lo[2 * q + 1 - j];
            o[0].x = fmaf(h0[j], a0.x, o[0].x);
            o[0].y = fmaf(h0[j], a0.y, o[0].y);
            o[1].x = fmaf(h1[j], a0.x, o[1].x);
            o[1].y = fmaf(h1[j], a0.y, o[1].y);
            o[2].x = fmaf(h0[j], a1.x, o[2].x);
            o[2].y = fmaf(h0[j], a1.y, o[2].y);
            o[3].x = fmaf(h1[j], a1.x, o[3].x);
            o[3].y = fmaf(h1[j], a1.y, o[3].y);
        }
    }
}

template <int HT>
__global__ void __launch_bounds__(kCombThreads, 4) combine_kernel(const CombineArgs a, int chunk) {
    extern __shared__ __align__(16) unsigned char csm[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(csm);
    float2 *cbuf = reinterpret_cast<float2 *>(csm + 16);
    const int t = a.rows ? a.rows[blockIdx.x] : (int)blockIdx.x;
    const int s = a.stream0 + blockIdx.y, tid = threadIdx.x;
    const int H = a.n_levels - 1, ht = a.n_taps / 2;
    const float2 *part = a.partial + (int64_t)s * a.partial_stream_stride;
    float2 *hist = a.ubuf + (int64_t)s * a.ubuf_stream_stride;
    float2 *zrow = a.z + (int64_t)s * a.z_stream_stride + (int64_t)t * a.z_row_stride;
    const int32_t *cptr = a.comb_ptr + t * a.n_levels;

    float h0[32], h1[32];   // even / odd polyphase branches of 2 h_up
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        h0[j] = (j < ht) ? a.h_up2[2 * j] : 0.f;
        h1[j] = (j < ht) ? a.h_up2[2 * j + 1] : 0.f;
    }
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    for (int k = tid; k < H * SPIIR_UHIST; k += kCombThreads) {
        const int i = 1 + k / SPIIR_UHIST, j = k % SPIIR_UHIST;
        cbuf[comb_ubuf_off(chunk, i) + j] = hist[a.lev[i].ubuf_off + (int64_t)t * SPIIR_UHIST + j];
    }
    __syncthreads();

    const int n0 = a.lev[0].n;
    uint32_t phase = 0;
    for (int c0 = 0; c0 < n0; c0 += chunk) {
        const int cn = min(chunk, n0 - c0);
        uint32_t bytes = 0;
        for (int i = 0; i <= H; ++i)
            if (cptr[i + 1] > cptr[i]) bytes += (uint32_t)(cn >> i) * 8u;
        bool ok = true;
        if (bytes) {
            if (tid == 0) {
                // the previous chunk's reads of the stage before this copy's writes
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(mbar, bytes);
                for (int i = 0; i <= H; ++i)
                    if (cptr[i + 1] > cptr[i]) {
                        const LevelArgs &L = a.lev[i];
                        bulk_g2s(cbuf + comb_stage_off(chunk, H, i),
                                 part + L.part_base + (int64_t)a.comb_rows[cptr[i]] * L.part_stride +
                                     (c0 >> i),
                                 (uint32_t)(cn >> i) * 8u, mbar);
                    }
            }
            ok = mbar_wait_bounded(mbar, phase, a.status);
            phase ^= 1u;
        }
        if (!__syncthreads_and(ok)) {
            // a copy did not land in time (status word set): wait once more,
            // bounded, so that no copy is left writing this CTA's memory
            mbar_wait_bounded(mbar, phase ^ 1u, a.status);
            return;
        }
        for (int i = H; i >= 0; --i) {
            const LevelArgs &L = a.lev[i];
            const int ni = cn >> i, off = c0 >> i;
            const int r0 = cptr[i], r1 = cptr[i + 1];
            const float2 *pl = part + L.part_base + off;
            const float4 *stg = reinterpret_cast<const float4 *>(cbuf + comb_stage_off(chunk, H, i));
            float2 *u_hi = (i > 0) ? cbuf + comb_ubuf_off(chunk, i) + SPIIR_UHIST : nullptr;
            const float2 *u_lo = (i < H) ? cbuf + comb_ubuf_off(chunk, i + 1) + SPIIR_UHIST : nullptr;
            for (int q = tid; 4 * q < ni; q += kCombThreads) {
                float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
                if (r1 > r0) {
                    p0 = stg[2 * q];
                    p1 = stg[2 * q + 1];
                }
                for (int r = r0 + 1; r < r1; ++r) {   // further parts (large units)
                    const float4 *pr = reinterpret_cast<const float4 *>(
                        pl + (int64_t)a.comb_rows[r] * L.part_stride + 4 * q);
                    const float4 v0 = __ldg(pr), v1 = __ldg(pr + 1);
                    p0.x += v0.x; p0.y += v0.y; p0.z += v0.z; p0.w += v0.w;
                    p1.x += v1.x; p1.y += v1.y; p1.z += v1.z; p1.w += v1.w;
                }
                float2 o[4] = {make_float2(p0.x, p0.y), make_float2(p0.z, p0.w),
                               make_float2(p1.x, p1.y), make_float2(p1.z, p1.w)};
                if (u_lo) upsample_quad<HT>(u_lo, q, h0, h1, ht, o);
                if (u_hi) {
                    float4 *d = reinterpret_cast<float4 *>(u_hi + 4 * q);
                    d[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                    d[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
                } else {
                    const float sc = a.scale;
                    float4 *d = reinterpret_cast<float4 *>(zrow + c0 + 4 * q);
                    d[0] = make_float4(sc * o[0].x, sc * o[0].y, sc * o[1].x, sc * o[1].y);
                    d[1] = make_float4(sc * o[2].x, sc * o[2].y, sc * o[3].x, sc * o[3].y);
                }
            }
            __syncthreads();
        }
        // keep the last SPIIR_UHIST samples of every level as its history
        constexpr int kPer = (SPIIR_MAX_LEVELS * SPIIR_UHIST + kCombThreads - 1) / kCombThreads;
        float2 keep[kPer];
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            const int k = tid + e * kCombThreads;
            if (k < H * SPIIR_UHIST) {
                const int i = 1 + k / SPIIR_UHIST, j = k % SPIIR_UHIST;
                keep[e] = cbuf[comb_ubuf_off(chunk, i) + (cn >> i) + j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            const int k = tid + e * kCombThreads;
            if (k < H * SPIIR_UHIST) {
                const int i = 1 + k / SPIIR_UHIST, j = k % SPIIR_UHIST;
                cbuf[comb_ubuf_off(chunk, i) + j] = keep[e];
            }
        }
        __syncthreads();
    }
    for (int k = tid; k < H * SPIIR_UHIST; k += kCombThreads) {
        const int i = 1 + k / SPIIR_UHIST, j = k % SPIIR_UHIST;
        hist[a.lev[i].ubuf_off + (int64_t)t * SPIIR_UHIST + j] = cbuf[comb_ubuf_off(chunk, i) + j];
    }
}

// ---------------------------------------------------------------------------
// Variants
// ---------------------------------------------------------------------------

struct Variant {
    int T, FMAX;
    void (*fn)(const RecurArgs);
};

const Variant kVariants[] = {
    {16, 8, recur_kernel<16, 8, 3>},
    {16, 16, recur_kernel<16, 16, 2>},
    {32, 4, recur_kernel<32, 4, 3>},
    {32, 8, recur_kernel<32, 8, 2>},
    {16, 4, recur_kernel<16, 4, 4>},
    {32, 8, recur_kernel<32, 8, 3>},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

int spiir_recur_variant_count() { return kNumVariants; }

void spiir_recur_variant_shape(int v, int *time_tile, int *fmax) {
    *time_tile = kVariants[v].T;
    *fmax = kVariants[v].FMAX;
}

cudaError_t spiir_recur_prepare(int v, int smem_bytes, int *ctas_per_sm) {
    // The limit is a property of the kernel shared by every bank: set it once
    // to the device maximum; each launch passes its own (smaller) size.
    int dev = 0, max_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kVariants[v].fn);
    if (e != cudaSuccess) return e;
    const int dyn_max = max_optin - (int)fa.sharedSizeBytes;
    if (smem_bytes > dyn_max) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kVariants[v].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kVariants[v].fn, SPIIR_CTA_WARPS * 32,
                                                      smem_bytes);
    *ctas_per_sm = n > 0 ? n : 1;
    return e;
}

int spiir_recur_red_bytes() { return kRedBytes + kScratchBytes; }

cudaError_t spiir_launch_prologue(const PrologueArgs &a, int n_streams, cudaStream_t s) {
    prologue_kernel<<<dim3(a.n_levels, n_streams), 512, 0, s>>>(a);
    const int n = a.lev[0].n;
    if (n > 0) {
        const unsigned gx = (unsigned)std::min(1024, std::max(1, (n + 1023) / 1024));
        prologue_copy_kernel<<<dim3(gx, n_streams), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t spiir_launch_decimate(const DecimArgs &a, int n_streams, cudaStream_t s) {
    decimate_kernel<<<n_streams, 512, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t spiir_launch_recur(const RecurArgs &a, int variant, int n_ctas, int n_streams,
                               int smem_bytes, cudaStream_t s) {
#if SPIIR_REDUCE_ABLATION == 3
    // the atomics build adds into its destination rows: zero them first
    for (int q = 0; q < n_streams; ++q) {
        cudaError_t e = cudaMemset2DAsync(a.z + (int64_t)(a.stream0 + q) * a.z_stream_stride,
                                          a.z_row_stride * sizeof(float2), 0, (size_t)a.lev[0].n * sizeof(float2),
                                          (size_t)(a.z_stream_stride / a.z_row_stride), s);
        if (e == cudaSuccess && a.partial && a.partial_stream_stride)
            e = cudaMemsetAsync(a.partial + (int64_t)(a.stream0 + q) * a.partial_stream_stride, 0,
                                (size_t)a.partial_stream_stride * sizeof(float2), s);
        if (e != cudaSuccess) return e;
    }
#endif
    kVariants[variant].fn<<<dim3(n_ctas, n_streams), SPIIR_CTA_WARPS * 32, smem_bytes, s>>>(a);
    return cudaGetLastError();
}

namespace {

// |z| / norm_t, one thread per output sample (the SNR of Sec. 2.1 is the
// modulus of z over the template's normalisation constant).
__global__ void abs_kernel(const float2 *z, int64_t ring, int64_t n, const float *norm, float *out) {
    const int t = blockIdx.y;
    const float nt = norm ? norm[t] : 1.0f;
    const float2 *zr = z + (int64_t)t * ring;
    float *o = out + (int64_t)t * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = zr[i];
        o[i] = hypotf(v.x, v.y) / nt;
    }
}

}  // namespace

cudaError_t spiir_launch_abs(const float2 *z, int64_t ring, int T, int64_t n, const float *norm,
                             float *out, cudaStream_t s) {
    if (T <= 0 || n <= 0) return cudaSuccess;
    const int bx = (int)std::min<int64_t>((n + 255) / 256, 64);
    for (int t0 = 0; t0 < T; t0 += 65535) {
        const int tn = std::min(65535, T - t0);
        abs_kernel<<<dim3(bx, tn), 256, 0, s>>>(z + (int64_t)t0 * ring, ring, n, norm ? norm + t0 : nullptr,
                                              out + (int64_t)t0 * n);
    }
    return cudaGetLastError();
}

int spiir_combine_chunk(int n_levels, int64_t push_max) {
    const int64_t c = std::max<int64_t>(2048, (int64_t)4 << (n_levels - 1));
    return (int)std::min<int64_t>(c, push_max);
}

int spiir_combine_smem(int n_levels, int chunk) {
    const int H = n_levels - 1;
    return 16 + comb_stage_off(chunk, H, H + 1) * (int)sizeof(float2);
}

cudaError_t spiir_launch_combine(const CombineArgs &a, int chunk, int n_streams, cudaStream_t s) {
    const int smem = spiir_combine_smem(a.n_levels, chunk);
    const dim3 grid(a.n_templates, n_streams);
    const int ht = a.n_taps / 2;
    switch (a.n_levels > 1 ? ht : 0) {
        case 8: combine_kernel<8><<<grid, kCombThreads, smem, s>>>(a, chunk); break;
        case 16: combine_kernel<16><<<grid, kCombThreads, smem, s>>>(a, chunk); break;
        case 32: combine_kernel<32><<<grid, kCombThreads, smem, s>>>(a, chunk); break;
        default: combine_kernel<-1><<<grid, kCombThreads, smem, s>>>(a, chunk); break;
    }
    return cudaGetLastError();
}

cudaError_t spiir_combine_prepare() {
    // like the recursion kernel: one kernel-wide limit, the device maximum
    int dev = 0, optin = 0;
    cudaError_t r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const void *fns[] = {(const void *)combine_kernel<8>, (const void *)combine_kernel<16>,
                         (const void *)combine_kernel<32>, (const void *)combine_kernel<-1>};
    for (const void *f : fns)
        if (r == cudaSuccess) r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    return r;
}
