// spiir_tc.cu -- block-parallel tensor-core form of single-rate SPIIR banks.
//
// Exact chunked decomposition (chunks of L samples, n0 = c*L, F > max d_k):
//
//   z_t[n0+j] = scale * ( sum_{q=0}^{F+L-1} h_t[q] xt[n0+j-q]
//                        + sum_{k in t} a_k^{j+1} s_k(c) ),        0 <= j < L
//
//   h_t[q]  = sum_k 1[q >= d_k] b_k a_k^(q-d_k)   (template impulse response)
//   xt[m]   = x[m] for m >= n0-F, else 0          (older input is in the state)
//   v_k[p]  = a_k v_k[p-1] + x[p]                 (undelayed unit filter)
//   s_k(c)  = a_k^(F-d_k) b_k v_k[n0-F-1]
//   v_k     <- a_k^L v_k + sum_{i<L} a_k^(L-1-i) x[n0-F+i]   (chunk to chunk)
//
// It follows from Eq. (iireq0) solved as Eq. (equ:first-order2): inputs older
// than n0-F reach every filter after its delay, so their whole effect is the
// filter state; newer inputs are a finite convolution with h_t.
//
// Three tensor-core contractions (tcgen05.mma, operands in shared memory,
// accumulators in tensor memory) and one FP64 recurrence:
//   FIR    D[(t,re/im), j] = H[(t,re/im), q] x Toeplitz(xt)[q, j]. The Toeplitz
//          operand is a shared-memory descriptor over a reversed strain window
//          stored 8 times with one-sample shifts: every 8x8 core matrix
//          (n-block g, k-block kb) is block g+kb, so both descriptor strides
//          are 128 bytes and no Toeplitz matrix is ever built.
//   STATE  G_k(c, i2) = sum_{i1<64} a_k^i1 x[e_c - 64 i2 - i1]: power panel
//          R[k][i] = a_k^i, i < 64 (K-major, contraction over powers) times
//          strain segments; U_k = sum_i2 a_k^(64 i2) G_k(c, i2).
//   CARRY  (FP32 inside a batch of chunks, FP64 from batch to batch; one
//          thread per filter and stream) s = c_k v, v <- a^L v + U.
//   OUTPUT D[j1, (c, j2, re/im)] = sum_k R[k][j1] w_k(c, j2) with
//          w = a_k^(64 j2) a_k s_k(c): the same panel R read MN-major
//          (contraction over filters); the FIR adds its term to it in z.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "spiir_internal.h"
#include "spiir_tc.h"

namespace {

thread_local std::string g_tc_err;

spiir_status tc_fail(spiir_status st, const char *msg) {
    g_tc_err = msg;
    return st;
}

#define TC_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            g_tc_err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
            return e_ == cudaErrorMemoryAllocation ? SPIIR_ENOMEM : SPIIR_ECUDA;        \
        }                                                                               \
    } while (0)

constexpr int kJ = 64;            // power-panel length (STATE/OUTPUT factorisation)
constexpr int kTile = 128;        // filters per carry tile (MMA M)
constexpr int kGroup = 64;        // templates per FIR tile (M = 128 rows re/im)
constexpr int kKs = 64;           // FIR K slice
constexpr int kStages = 4;        // FIR A-operand pipeline depth
constexpr int kSliceBytes = 128 * kKs * 2;   // 16 KB

// ---------------------------------------------------------------------------
// Device helpers: mbarrier, bulk copy, tcgen05
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t s32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(m)), "r"(c) : "memory");
}

// Test of an mbarrier phase that may suspend the thread until the phase
// completes, for at most kSuspendNs (the hint): a waiting warp then takes no
// issue slots from the warps doing the work, and the bounded waits below
// still look at the clock and the abort flag between tries.
constexpr uint32_t kSuspendNs = 100000;
__device__ __forceinline__ bool mbar_try(uint64_t *m, uint32_t ph) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(s32(m)), "r"(ph), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded wait (~2 s): on timeout record it and report false.
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t ph, unsigned int *status) {
    if (mbar_try(m, ph)) return true;
    const uint64_t t0 = gtime();
    while (!mbar_try(m, ph)) {
        if (gtime() - t0 > 2000000000ull) {
            atomicExch(status, SPIIR_DEV_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_expect(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(m)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            s32(dst)),
        "l"(src), "r"(bytes), "r"(s32(m))
        : "memory");
}

// Bring [src, src + bytes) into L2 (16-byte aligned, a multiple of 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Whole warp: allocate ncols tensor-memory columns; address written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start, LBO (stride between
// core matrices along K), SBO (stride between 8-row groups along M/N).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16, FP32 accumulate.
__host__ __device__ constexpr uint32_t idesc(int M, int N, bool bf16, bool a_mn, bool b_mn) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *m) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     s32(m))
                 : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%"
        "15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if constexpr (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&h);
    } else {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
}

template <bool BF16>
__device__ __forceinline__ uint4 pack8(const float (&v)[8]) {
    uint4 r;
    r.x = pack2<BF16>(v[0], v[1]);
    r.y = pack2<BF16>(v[2], v[3]);
    r.z = pack2<BF16>(v[4], v[5]);
    r.w = pack2<BF16>(v[6], v[7]);
    return r;
}

// ---------------------------------------------------------------------------
// Kernel arguments
// ---------------------------------------------------------------------------

// Strain operands of one push, staged once in global memory in the exact
// shared-memory layouts the contractions read (fetched with bulk copies).
struct TcStageArgs {
    const float *xbuf;        // [stream][xbuf_stride]: hist then the push
    int64_t xbuf_stride;
    int32_t hist, F, L, K, n_chunks, n_streams, stream0;
    int32_t cpb, n_batches;   // carry: chunks per batch, batches
    uint4 *hank;              // [s][c][hank_bytes/16]  FIR Toeplitz source
    uint4 *hank_lo;           // NULL, or the same layout: x - bf16(x), the low
                              // part of a split-bf16 operand
    int32_t hank_bytes;
    uint4 *xseg;              // [batch][kXsegBytes/16] STATE strain segments
};

constexpr int kNii = 64;                       // STATE columns per carry batch
constexpr int kXsegBytes = kNii * kJ * 2;      // 8 KB

struct TcFirArgs {
    const uint4 *H;           // [group][slice][16 KB] pre-tiled impulse responses
    const float *row_scale;   // per template: snr_scale * 2^-e_t
    const uint8_t *has_carry; // per template: z already holds the state term
    const int32_t *groups;    // NULL: template groups 0 .. n_groups-1; else
                              // the groups to run (n_groups entries)
    const uint4 *hank;        // staged Toeplitz sources
    int32_t hank_bytes;
    int32_t L, K;
    int32_t n_groups, n_chunks, n_streams, n_templates;
    int32_t stream0;
    float2 *z;
    int64_t z_row_stride, z_stream_stride;
    unsigned int *status;
};

struct TcCarryArgs {
    const int32_t *tile_ptr;  // [t], [t+1]: carry tiles of template t
    const int32_t *tile_end;  // NULL, or [t]: end of template t's tiles
                              // (tile_ptr[t] is then their start)
    const int32_t *tmpl_of;   // templates that own tiles
    int32_t n_carry;
    const float2 *a;          // [slot] a_k
    const float2 *aJ;         // [slot] a_k^kJ
    const uint4 *aL;          // [slot] a_k^L: FP64 double2 or double-float float4 (carry mode)
    const float2 *aLf;        // [slot] a_k^L rounded to FP32
    const uint4 *aLb;         // [slot] a_k^(L * cpb), same type, cpb of this launch
    const float2 *c;          // [slot] a_k^(F-d_k) b_k
    uint4 *v;                 // [stream][n_slots] undelayed unit-filter state, same type
    const uint4 *panel;       // [tile] power panels (layout below), precomputed
    int64_t n_slots;
    const uint4 *xseg;        // staged STATE strain segments
    int32_t L, n_chunks, n_streams, stream0, cpb, n_batches;
    float scale;
    float2 *z;
    int64_t z_row_stride, z_stream_stride;
    unsigned int *status;
};

// ---------------------------------------------------------------------------
// Staging kernel: one thread per 16-byte chunk of either operand
// ---------------------------------------------------------------------------

template <bool BF16>
__global__ void tc_stage_kernel(const TcStageArgs a) {
    const int64_t hank_chunks = (int64_t)a.n_streams * a.n_chunks * (a.hank_bytes / 16);
    const int64_t xseg_chunks = (int64_t)a.n_batches * (kXsegBytes / 16);
    const int LJ = a.L / kJ;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hank_chunks + xseg_chunks;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v[8];
        if (i < hank_chunks) {
            // Toeplitz source of chunk c: xr[p] = xt[n0 + L - 1 - p]; 16-byte
            // chunk (blk, r) holds xr[8 blk + r + 0..7]
            const int per = a.hank_bytes / 16;
            const int sc = (int)(i / per), w = (int)(i % per);
            const int ss = sc / a.n_chunks, c = sc % a.n_chunks;
            const int blk = w >> 3, r = w & 7;
            const float *x = a.xbuf + (int64_t)(a.stream0 + ss) * a.xbuf_stride + a.hist;
            const int n0 = c * a.L;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int p = 8 * blk + r + q;
                const int m = n0 + a.L - 1 - p;
                v[q] = (p < a.L + a.K - 1 && m >= n0 - a.F) ? x[m] : 0.f;
            }
            a.hank[i] = pack8<BF16>(v);
            if (a.hank_lo) {
                float lo[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) lo[q] = v[q] - __bfloat162float(__float2bfloat16_rn(v[q]));
                a.hank_lo[i] = pack8<BF16>(lo);
            }
        } else {
            // STATE segments of batch b: row n = (s, i2, c) (the chunks of a
            // stream and power block adjacent), K = i1:
            // x_s[e_c - kJ i2 - i1], e_c = c L - F + L - 1; layout
            // [n/8][i1/8][n%8][i1%8]
            const int64_t j = i - hank_chunks;
            const int b = (int)(j / (kXsegBytes / 16)), w = (int)(j % (kXsegBytes / 16));
            constexpr int kKB = kJ / 8;
            const int n = (w / (8 * kKB)) * 8 + (w % 8), kb = (w / 8) % kKB;
            const int nb = min(a.cpb, a.n_chunks - b * a.cpb);
            const int cc = n % a.cpb, i2 = (n / a.cpb) % LJ, ss = n / a.cpb / LJ;
            if (ss < a.n_streams && cc < nb) {
                const float *x = a.xbuf + (int64_t)(a.stream0 + ss) * a.xbuf_stride + a.hist;
                const int e = (b * a.cpb + cc) * a.L - a.F + a.L - 1 - kJ * i2;
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = x[e - (8 * kb + q)];
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = 0.f;
            }
            a.xseg[j] = pack8<BF16>(v);
        }
    }
}

// ---------------------------------------------------------------------------
// FIR kernel: persistent, warp-specialised
//   warp 0 lane 0: bulk-copy producer (impulse-response slices, Toeplitz source)
//   warp 1 lane 0: MMA issuer into two tensor-memory accumulators
//   warps 2-9    : epilogue (tensor memory -> z), overlapping the next MMAs;
//                  two warps per tensor-memory lane quadrant, each taking
//                  every other 16-column step
// Items (template group, stream, chunk), chunk fastest so that CTAs working at
// the same time share impulse-response tiles in L2.
// ---------------------------------------------------------------------------

// Template group of the FIR items with group index sg / n_streams, the last
// group first: the carry kernel ends on the highest templates, whose state
// terms are then the likeliest to be still in L2 when the FIR reads them.
__device__ __forceinline__ int fir_group(const TcFirArgs &a, int sg) {
    const int gi = a.n_groups - 1 - sg / a.n_streams;
    return a.groups ? a.groups[gi] : gi;
}

constexpr int kFirEpiWarps = 8;
constexpr int kFirThreads = (2 + kFirEpiWarps) * 32;

template <bool BF16>
__global__ void __launch_bounds__(kFirThreads, 1) tc_fir_kernel(const TcFirArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t a_full[kStages], a_empty[kStages], h_full[2], h_empty[2], acc_full[2],
        acc_empty[2];
    __shared__ uint32_t s_tmem;
    const int L = a.L, K = a.K;
    const int n_slices = K / kKs;
    const int n_items = a.n_groups * a.n_streams * a.n_chunks;
    unsigned char *stage_mem = smem;                                   // kStages x 16 KB
    unsigned char *hank = smem + kStages * kSliceBytes;                // 2 x hank_bytes
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&h_full[i], 1);
            mbar_init(&h_empty[i], 1);
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kFirEpiWarps * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&s_tmem, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0 && lane == 0) {
        // producer
        int64_t gc = 0;     // global slice counter (A ring)
        int li = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++li) {
            const int c = it % a.n_chunks, sg = it / a.n_chunks;
            const int ss = sg % a.n_streams;
            const int g = fir_group(a, sg);
            const int hb = li & 1;
            if (li >= 2) {
                ok = mbar_wait(&h_empty[hb], ((li >> 1) - 1) & 1, a.status);
                if (!ok) break;
            }
            mbar_expect(&h_full[hb], a.hank_bytes);
            bulk_load(hank + (size_t)hb * a.hank_bytes,
                      a.hank + ((size_t)ss * a.n_chunks + c) * (a.hank_bytes / 16), a.hank_bytes,
                      &h_full[hb]);
            const uint4 *A = a.H + (size_t)g * n_slices * (kSliceBytes / 16);
            for (int ks = 0; ks < n_slices; ++ks, ++gc) {
                const int st = (int)(gc % kStages);
                const int64_t use = gc / kStages;
                if (use >= 1) {
                    ok = mbar_wait(&a_empty[st], (uint32_t)((use - 1) & 1), a.status);
                    if (!ok) break;
                }
                mbar_expect(&a_full[st], kSliceBytes);
                bulk_load(stage_mem + st * kSliceBytes, A + (size_t)ks * (kSliceBytes / 16),
                          kSliceBytes, &a_full[st]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t id = idesc(128, L, BF16, false, false);
        int64_t gc = 0;
        int li = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++li) {
            const int ab = li & 1, hb = li & 1;
            if (li >= 2) {
                ok = mbar_wait(&acc_empty[ab], ((li >> 1) - 1) & 1, a.status);
                if (!ok) break;
            }
            ok = mbar_wait(&h_full[hb], (li >> 1) & 1, a.status);
            if (!ok) break;
            tc_fence_after();
            const uint32_t d = tmem + ab * 256;
            const uint32_t bbase = s32(hank + (size_t)hb * a.hank_bytes);
            for (int ks = 0; ks < n_slices; ++ks, ++gc) {
                const int st = (int)(gc % kStages);
                ok = mbar_wait(&a_full[st], (uint32_t)((gc / kStages) & 1), a.status);
                if (!ok) break;
                tc_fence_after();
                const uint32_t abase = s32(stage_mem + st * kSliceBytes);
#pragma unroll
                for (int kk = 0; kk < kKs / 16; ++kk) {
                    const uint64_t ad = sdesc(abase + kk * 256, 128, 1024);
                    const uint64_t bd = sdesc(bbase + (ks * (kKs / 8) + 2 * kk) * 128, 128, 128);
                    mma(d, ad, bd, id, (ks | kk) ? 1u : 0u);
                }
                mma_commit(&a_empty[st]);
            }
            mma_commit(&h_empty[hb]);
            mma_commit(&acc_full[ab]);
        }
    } else if (warp >= 2) {
        // epilogue: lane row r = template 64g + r/2, re (even) / im (odd);
        // column n' is time n = L - 1 - n'
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;      // steps half, half + 2, ...
        const int r = q * 32 + lane;
        int li = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < n_items; it += gridDim.x, ++li) {
            const int c = it % a.n_chunks, sg = it / a.n_chunks;
            const int ss = sg % a.n_streams;
            const int g = fir_group(a, sg);
            const int ab = li & 1;
            const int t = g * kGroup + (r >> 1);
            const float sc = (t < a.n_templates) ? a.row_scale[t] : 0.f;
            float2 *zrow = a.z + (int64_t)(a.stream0 + ss) * a.z_stream_stride +
                           (int64_t)min(t, a.n_templates - 1) * a.z_row_stride + (int64_t)c * L;
            const bool is_re = (r & 1) == 0;
            const bool add = (t < a.n_templates) && a.has_carry[t];
            const int i0 = is_re ? 0 : 8;
            // A lane writes the 8 samples of its 8 columns of a 16-column step:
            // column c is sample L - 1 - c, so they are the contiguous samples
            // from L - 8 - (16 cc + i0), moved as four 16-byte vectors. The
            // state term (written by the carry kernel) of the warp's next kD
            // steps is in flight at any time, the first ones fetched before
            // the accumulator is ready, so the global latency overlaps the
            // contraction and the earlier steps.
            const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
            auto zv = [&](int cc) {
                return reinterpret_cast<float4 *>(zrow + (L - 8 - (cc * 16 + i0)));
            };
            constexpr int kD = 3;
            float4 pf[kD][4];
#pragma unroll
            for (int d = 0; d < kD; ++d)
#pragma unroll
                for (int i = 0; i < 4; ++i) pf[d][i] = (add && half + 2 * d < L / 16) ? zv(half + 2 * d)[i] : zero4;
            ok = ok && mbar_wait(&acc_full[ab], (li >> 1) & 1, a.status);
            tc_fence_after();
            for (int cc = half; cc < L / 16; cc += 2) {
                float4 prev[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    prev[i] = pf[0][i];
#pragma unroll
                    for (int d = 0; d + 1 < kD; ++d) pf[d][i] = pf[d + 1][i];
                    pf[kD - 1][i] = (add && cc + 2 * kD < L / 16) ? zv(cc + 2 * kD)[i] : zero4;
                }
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + ab * 256 + cc * 16, v);
                float o[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) o[i] = __shfl_xor_sync(0xffffffffu, v[i], 1);
                if (ok && t < a.n_templates) {
                    // even lanes own columns 0..7 of the step, odd lanes 8..15
                    // (compile-time register indices on both sides); sample
                    // sb + u holds column 7 - u
                    float re[8], im[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        re[i] = is_re ? v[i] : o[8 + i];
                        im[i] = is_re ? o[i] : v[8 + i];
                    }
                    float4 *dst = zv(cc);
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const int i_lo = 7 - 2 * w, i_hi = 6 - 2 * w;   // samples 2w, 2w + 1
                        dst[w] = make_float4(fmaf(sc, re[i_lo], prev[w].x), fmaf(sc, im[i_lo], prev[w].y),
                                             fmaf(sc, re[i_hi], prev[w].z), fmaf(sc, im[i_hi], prev[w].w));
                    }
                }
            }
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s32(&acc_empty[ab])) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 512);
}

// ---------------------------------------------------------------------------
// Carry kernel: one CTA per SM, persistent over templates. A CTA's work is a
// sequence of jobs (template, chunk batch, 128-filter tile) on four power
// panel slots and two OUTPUT-operand (W) slots in shared memory and two carry
// groups, spread over warp roles:
//   warp 0, lane 0   issues the STATE contractions in job order as soon as
//                    each one's inputs are ready, and the strain-segment copies
//   last warp, lane 0  issues the OUTPUT contractions in job order (a
//                    separate warp, on another scheduler: a single issuer sharing a
//                    scheduler with the arithmetic warps was slow to react)
//   next-to-last warp, lane 0  bulk copy of each job's precomputed power
//                    panel into its slot (up to four jobs ahead)
//   warps 1-4        the epilogue of each (template, batch) in order:
//                    OUTPUT accumulators -> z (a separate role: taken by the
//                    copying warps, the epilogues delayed the next panel)
//   warps 5 ..       carry groups 0 and 1 of 4 S warps each, one thread per
//                    filter and stream: STATE (tensor memory) -> FP32 carry
//                    inside a batch, FP64 (or double-float) from batch to batch
//                    -> OUTPUT operand W of the job's slot. With two streams a
//                    filter's two chains run in two threads, which halves each
//                    group's dependent chain per job (the groups' latency, not
//                    the tensor pipe, sets the kernel's pace)
// Panel of a 128-filter tile: 128 rows m of powers, layout
// [k/8][m/8][k%8][m%8], in row groups of 8: group 2 p holds Re a_k^j and
// group 2 p + 1 Im a_k^j for the powers j = 8 p .. 8 p + 7. STATE reads it
// K-major (filters x powers: the re powers 16 i .. 16 i + 15 are groups 4 i
// and 4 i + 2, the im powers groups 4 i + 1 and 4 i + 3); OUTPUT reads it
// MN-major along M = 128:
//   D[m][2c]     = sum_k R[k][m] Re w_k(c),  D[m][2c + 1] = sum_k R[k][m] Im w_k(c)
//   z_re(j) = D[re j][2c] - D[im j][2c + 1],  z_im(j) = D[re j][2c + 1] + D[im j][2c]
// The two rows of power j are tensor-memory lanes 8 apart, so one 16-lane
// load (shape 16x256b) gives each epilogue thread all four terms of z(j, c).
// Every hand-off between roles is an mbarrier: tcgen05.commit for
// contractions, one arrive per thread for the 128-thread roles; every wait is
// bounded and gives up at once when another role has given up (the epilogue
// role agrees on it with a barrier reduction, so it leaves as a whole).
// Tensor memory (512 columns): STATE of carry group g at 128 g (re 64, im 64
// columns); OUTPUT of (template, batch) e at 256 + 128 (e % 2).
// ---------------------------------------------------------------------------

// Warps of the carry kernel for S streams: the two issuers, the panel
// copier, the four epilogue warps and two carry groups of 4 S warps (one
// thread per filter and stream).
constexpr int carry_warps(int S) { return 7 + 8 * S; }
constexpr int kPanelSlots = 4;     // power panels in flight
constexpr int kWSlots = 2;         // OUTPUT operands W in flight
constexpr int kPanelBytes = kTile * 2 * kJ * 2;                 // 32 KB
constexpr int kWBytes = kTile * 2 * kNii * 2;                   // 32 KB
constexpr int kCarrySmem = kPanelSlots * kPanelBytes + kWSlots * kWBytes + 2 * kXsegBytes;   // 208 KB

__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s32(m)) : "memory");
}

// Bounded wait that also gives up when *abort is set; a timeout sets *abort.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t *m, uint32_t ph, unsigned int *status,
                                             volatile int *abort) {
    if (mbar_try(m, ph)) return true;
    const uint64_t t0 = gtime();
    while (!mbar_try(m, ph)) {
        if (*abort) return false;
        if (gtime() - t0 > 2000000000ull) {
            atomicExch(status, SPIIR_DEV_TIMEOUT);
            *abort = 1;
            return false;
        }
    }
    return true;
}

// 16 lanes x 256 bits, 16 times along the columns: thread t gets rows
// t / 4 and t / 4 + 8, columns 2 (t % 4) and 2 (t % 4) + 1 of each 8.
__device__ __forceinline__ void tmem_ld16x256_x16(uint32_t taddr, uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
}

// The same, 8 times along the columns (64 columns).
__device__ __forceinline__ void tmem_ld16x256_x8(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// 32 lanes x N consecutive columns (N = 4 or 8), without waiting.
__device__ __forceinline__ void tmem_ld_n(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_n(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The 128 threads of the epilogue role (named barrier 1): synchronise, and
// agree on v (true only if every thread passes true), so that the role
// leaves its loop as a whole.
__device__ __forceinline__ bool panel_role_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

struct CarryJob {
    int t, b0, tile;
    bool first_tile, last_tile;
    int j, e;   // job index and (template, batch) index within this CTA
    int s, w, g;   // panel slot, W slot and carry group (STATE columns)
};

// The job sequence of this CTA: jobs cycle through the panel and W slots and
// alternate between the two carry groups. When a template has several
// batches, the filter state v of a tile passes from one batch to the next,
// so a tile keeps its carry group for all of them. Every listed template
// owns at least one tile.
struct CarryJobs {
    const TcCarryArgs *a;
    int ti, b0, tile, tile0, tile1, t, j, e;
    bool multi, valid;
    __device__ explicit CarryJobs(const TcCarryArgs &A)
        : a(&A), ti(blockIdx.x), j(0), e(0), multi(A.n_batches > 1) {
        start();
    }
    __device__ void start() {
        valid = ti < a->n_carry;
        if (valid) {
            t = a->tmpl_of[ti];
            tile0 = a->tile_ptr[t];
            tile1 = a->tile_end ? a->tile_end[t] : a->tile_ptr[t + 1];
            b0 = 0;
            tile = tile0;
        }
    }
    __device__ CarryJob cur() const {
        const int g = multi ? ((tile - tile0) & 1) : (j & 1);
        return CarryJob{t, b0, tile, tile == tile0, tile == tile1 - 1, j, e, j % kPanelSlots, j % kWSlots, g};
    }
    __device__ void next() {
        ++j;
        if (++tile < tile1) return;
        tile = tile0;
        ++e;
        if (++b0 < a->n_batches) return;
        ti += gridDim.x;
        start();
    }
};

template <class Fn>
__device__ __forceinline__ void carry_jobs(const TcCarryArgs &a, Fn &&fn) {
    for (CarryJobs it(a); it.valid; it.next())
        if (!fn(it.cur())) return;
}

__device__ __forceinline__ float2 cmul(float2 x, float2 y) {
    return make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}

// Double-float complex numbers: float4 {re hi, im hi, re lo, im lo}, value
// hi + lo with |lo| <= ulp(hi) / 2 (about 48 significant bits), on the FP32
// pipe: GB300's FP64 rate is 2 DFMA per SM and clock. Built from the
// error-free sum (Knuth's TwoSum), product (FMA residual) and the
// normalising fast sum (Dekker); the _rn intrinsics keep the compiler from
// contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// One component of x y + d: x1 y1 + sg x2 y2 + d (x, y double-float parts
// (hi, lo); sg = +1 or -1), returned as (hi, lo).
__device__ __forceinline__ float2 df_dot2_add(float x1h, float x1l, float y1h, float y1l, float x2h,
                                              float x2l, float y2h, float y2l, float sg, float d) {
    const float p1 = __fmul_rn(x1h, y1h);
    const float e1 = __fmaf_rn(x1h, y1h, -p1);
    const float nx2h = sg * x2h, nx2l = sg * x2l;
    const float p2 = __fmul_rn(nx2h, y2h);
    const float e2 = __fmaf_rn(nx2h, y2h, -p2);
    float s, t1, t2;
    two_sum(p1, p2, s, t1);
    two_sum(s, d, s, t2);
    float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(t1, t2));
    lo = __fmaf_rn(x1h, y1l, lo);
    lo = __fmaf_rn(x1l, y1h, lo);
    lo = __fmaf_rn(nx2h, y2l, lo);
    lo = __fmaf_rn(nx2l, y2h, lo);
    const float hi = __fadd_rn(s, lo);
    return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}

// x y + d for double-float x, y and FP32 d.
__device__ __forceinline__ float4 cdf_mul_add(float4 x, float4 y, float2 d) {
    const float2 re = df_dot2_add(x.x, x.z, y.x, y.z, x.y, x.w, y.y, y.w, -1.f, d.x);
    const float2 im = df_dot2_add(x.x, x.z, y.y, y.w, x.y, x.w, y.x, y.z, 1.f, d.y);
    return make_float4(re.x, im.x, re.y, im.y);
}

// The inter-batch anchor in either carry arithmetic: FP64 complex (double2)
// or double-float (float4). Its FP32 value, x y + d, and x y.
__device__ __forceinline__ float2 anchor_f32(const double2 &v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ float2 anchor_f32(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ double2 anchor_madd(double2 x, double2 y, float2 d) {
    return make_double2(fma(x.x, y.x, fma(-x.y, y.y, (double)d.x)), fma(x.x, y.y, fma(x.y, y.x, (double)d.y)));
}
__device__ __forceinline__ float4 anchor_madd(float4 x, float4 y, float2 d) { return cdf_mul_add(x, y, d); }

// MODE: arithmetic of the carried filter state. 0: FP64 anchor per chunk
// batch with FP32 offsets inside it; 1: the same with a double-float anchor;
// 2: FP64 state updated at every chunk.
template <bool BF16, int LJ, int S, int MODE>
__global__ void __launch_bounds__(carry_warps(S) * 32, 1) tc_carry_kernel(const TcCarryArgs a) {
    constexpr bool DF = MODE == 1, CH = MODE == 2;
    constexpr int kCarryWarps = carry_warps(S), kGW = 4 * S;   // warps, warps per carry group
    using Anchor = typename std::conditional<DF, float4, double2>::type;   // carry arithmetic
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t panel_full[kPanelSlots], panel_free[kPanelSlots], w_full[kWSlots], w_free[kWSlots],
        state_full[2], state_free[2], out_full[2], out_free[2], xs_full[2], drain, drain_o;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    // panel slot s at s * kPanelBytes, W slot w at kPanelSlots * kPanelBytes + w * kWBytes
    unsigned char *Wb = smem + kPanelSlots * kPanelBytes;
    unsigned char *Xs = Wb + kWSlots * kWBytes;                    // strain segments of batches b % 2
    // OUTPUT operand W, MN-major [k/8][n/8][k%8][n%8] (n = column, k = filter):
    // 8-column groups 128 bytes apart, 8-filter groups kWK apart; column 2c =
    // Re w(c), 2c + 1 = Im w(c) of chunk column c = (stream, chunk, j2)
    constexpr uint32_t kWK = (2 * kNii / 8) * 128;
    const int L = LJ * kJ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = &s_abort;     // S (1 or 2) = a.n_streams

    if (threadIdx.x == 0) {
        for (int i = 0; i < kPanelSlots; ++i) {
            mbar_init(&panel_full[i], 1);
            mbar_init(&panel_free[i], 1);
        }
        for (int i = 0; i < kWSlots; ++i) {
            mbar_init(&w_full[i], 32 * kGW);
            mbar_init(&w_free[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&state_full[i], 1);
            mbar_init(&state_free[i], 32 * kGW);
            mbar_init(&out_full[i], 1);
            mbar_init(&out_free[i], 128);
        }
        mbar_init(&xs_full[0], 1);
        mbar_init(&xs_full[1], 1);
        mbar_init(&drain, 1);
        mbar_init(&drain_o, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&s_tmem, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- STATE issuer ----------------
            // STATE of each job in job order, as soon as its strain segment,
            // its carry group's STATE columns and its panel are ready; the
            // strain-segment copies. Phase parities and use flags are bits
            // of ph; slot phases follow from the job index (use j / kPanelSlots).
            constexpr uint32_t kSF = 0, kUsed = 2;
            uint32_t ph = 0, ph_d = 0;
            // strain-segment buffers (batch b in buffer b % 2): batch held or
            // being loaded, job of the last STATE that read it, load in flight,
            // and the phase of the next load's completion
            int held0 = -1, held1 = -1, last0 = -1000, last1 = -1000;
            uint32_t loading = 0, xs_ph = 0;
            int last_pf = -1;   // latest job whose panel was ready: every STATE up
                                // to kPanelSlots jobs before it has finished (its
                                // slot was freed by that job's OUTPUT)
            auto start_load = [&](int x, int batch) {
                mbar_expect(&xs_full[x], kXsegBytes);
                bulk_load(Xs + x * kXsegBytes, a.xseg + (size_t)batch * (kXsegBytes / 16), kXsegBytes,
                          &xs_full[x]);
                if (x) held1 = batch;
                else held0 = batch;
                loading |= 1u << x;
            };
            bool issued = false, ok = true;
            const uint32_t id_state = idesc(128, kNii, BF16, false, false);
            const uint32_t smem0 = s32(smem), xs0 = s32(Xs);
            for (CarryJobs st(a); ok && st.valid; st.next()) {
                const CarryJob J = st.cur();
                const uint32_t g = (uint32_t)J.g, sl = (uint32_t)J.s;
                const int xb = J.b0 & 1;
                if ((xb ? held1 : held0) != J.b0 && !((loading >> xb) & 1u)) {
                    // the buffer's readers must be done before it is refilled:
                    // certain kPanelSlots jobs on, else drain the tensor pipe
                    // (rare: templates of one or two tiles with several batches)
                    if (issued && (xb ? last1 : last0) > last_pf - kPanelSlots) {
                        mma_commit(&drain);
                        ok = mbar_wait_ab(&drain, ph_d, a.status, abort);
                        ph_d ^= 1u;
                        if (!ok) break;
                    }
                    start_load(xb, J.b0);
                }
                if ((loading >> xb) & 1u) {
                    if (!(ok = mbar_wait_ab(&xs_full[xb], (xs_ph >> xb) & 1u, a.status, abort))) break;
                    loading &= ~(1u << xb);
                    xs_ph ^= 1u << xb;
                }
                if ((ph >> (kUsed + g)) & 1u) {
                    if (!(ok = mbar_wait_ab(&state_free[g], (ph >> (kSF + g)) & 1u, a.status, abort))) break;
                    ph ^= 1u << (kSF + g);
                }
                ph |= 1u << (kUsed + g);
                if (!(ok = mbar_wait_ab(&panel_full[sl], (uint32_t)(J.j / kPanelSlots) & 1u, a.status, abort)))
                    break;
                last_pf = J.j;
                if (xb) last1 = J.j;
                else last0 = J.j;
                tc_fence_after();
                // descriptors advance by 16-byte units in their low bits;
                // re powers 16 kk .. 16 kk + 15 are panel row groups 4 kk and
                // 4 kk + 2, the im powers groups 4 kk + 1 and 4 kk + 3
                const uint64_t dr0 = sdesc(smem0 + sl * kPanelBytes, 256, 2048);
                const uint64_t di0 = dr0 + (128 >> 4);
                const uint64_t dx0 = sdesc(xs0 + xb * kXsegBytes, 128, (kJ / 8) * 128);
                const uint32_t d = tmem + 128 * g;
#pragma unroll
                for (int kk = 0; kk < kJ / 16; ++kk) {
                    const uint64_t o = (uint64_t)(kk * 512) >> 4;
                    const uint64_t ox = (uint64_t)(kk * 256) >> 4;
                    mma(d, dr0 + o, dx0 + ox, id_state, kk ? 1u : 0u);
                    mma(d + kNii, di0 + o, dx0 + ox, id_state, kk ? 1u : 0u);
                }
                mma_commit(&state_full[g]);
                issued = true;
                // prefetch the template's next batch into the other buffer
                // once that buffer's readers are certainly done
                const int nb2 = J.b0 + 1, x2 = nb2 & 1;
                if (nb2 < a.n_batches && (x2 ? held1 : held0) != nb2 && !((loading >> x2) & 1u) &&
                    (x2 ? last1 : last0) <= last_pf - kPanelSlots)
                    start_load(x2, nb2);
            }
            // nothing may still run when the tensor memory is released, and no
            // copy may still be writing shared memory
            if (issued) {
                mma_commit(&drain);
                mbar_wait(&drain, ph_d, a.status);
            }
            for (int x = 0; x < 2; ++x)
                if ((loading >> x) & 1u) mbar_wait(&xs_full[x], (xs_ph >> x) & 1u, a.status);
        }
    } else if (warp == kCarryWarps - 1) {
        if (lane == 0) {
            // ---------------- OUTPUT issuer ----------------
            // OUTPUT of each job in job order (the first tile of a (template,
            // batch) overwrites the accumulator) once its W is written and,
            // for a first tile, the accumulator's previous epilogue is done.
            // W complete implies the job's STATE has finished.
            uint32_t of_ph = 0;                 // out_free phase per buffer
            bool issued = false;
            const uint32_t id_out = idesc(128, 2 * kNii, BF16, true, true);
            const uint32_t smem0 = s32(smem), wb0 = s32(Wb);
            for (CarryJobs ot(a); ot.valid; ot.next()) {
                const CarryJob J = ot.cur();
                const uint32_t sl = (uint32_t)J.s, wl = (uint32_t)J.w, ob = (uint32_t)(J.e & 1);
                if (J.first_tile && J.e >= 2) {
                    if (!mbar_wait_ab(&out_free[ob], (of_ph >> ob) & 1u, a.status, abort)) break;
                    of_ph ^= 1u << ob;
                }
                if (!mbar_wait_ab(&w_full[wl], (uint32_t)(J.j / kWSlots) & 1u, a.status, abort)) break;
                tc_fence_after();
                // D = R^T W over the tile's filters
                const uint64_t a0 = sdesc(smem0 + sl * kPanelBytes, 2048, 128);
                const uint64_t b0 = sdesc(wb0 + wl * kWBytes, kWK, 128);
                const uint32_t dz = tmem + 256 + 128 * ob;
                const uint32_t acc0 = J.first_tile ? 0u : 1u;
#pragma unroll
                for (int kk = 0; kk < kTile / 16; ++kk) {
                    const uint64_t oa = (uint64_t)(kk * 2 * 2048) >> 4;
                    const uint64_t ow = (uint64_t)(kk * 2 * kWK) >> 4;
                    mma(dz, a0 + oa, b0 + ow, id_out, kk ? 1u : acc0);
                }
                mma_commit(&w_free[wl]);
                mma_commit(&panel_free[sl]);
                if (J.last_tile) mma_commit(&out_full[ob]);
                issued = true;
            }
            if (issued) {
                mma_commit(&drain_o);
                mbar_wait(&drain_o, 0, a.status);
            }
        }
    } else if (warp == kCarryWarps - 2) {
        if (lane == 0) {
            // ---------------- panel copies ----------------
            // each job's precomputed power panel, one bulk copy into its slot
            // as soon as the OUTPUT kPanelSlots jobs back has freed the slot
            int last_copy = -1;
            for (CarryJobs pt(a); pt.valid; pt.next()) {
                const CarryJob J = pt.cur();
                const int sl = J.s, use = J.j / kPanelSlots;
                if (use > 0 && !mbar_wait_ab(&panel_free[sl], (use - 1) & 1, a.status, abort)) break;
                mbar_expect(&panel_full[sl], kPanelBytes);
                bulk_load(smem + sl * kPanelBytes, a.panel + (size_t)J.tile * (kPanelBytes / 16), kPanelBytes,
                          &panel_full[sl]);
                last_copy = J.j;
                if (J.b0 == 0) {
                    // the tile's coefficients and states, which its carry
                    // group reads when it starts the job, into L2 ahead of it
                    const int64_t s0 = (int64_t)J.tile * kTile;
                    prefetch_l2(a.a + s0, kTile * 8);
                    prefetch_l2(a.aJ + s0, kTile * 8);
                    prefetch_l2(a.c + s0, kTile * 8);
                    prefetch_l2(a.aLf + s0, kTile * 8);
                    prefetch_l2(a.aLb + s0, kTile * 16);
                    for (int q = 0; q < S; ++q) prefetch_l2(a.v + (int64_t)(a.stream0 + q) * a.n_slots + s0, kTile * 16);
                }
            }
            // no copy may still be writing shared memory when the CTA exits
            for (int j = max(0, last_copy - kPanelSlots + 1); j <= last_copy; ++j)
                mbar_wait(&panel_full[j % kPanelSlots], (uint32_t)(j / kPanelSlots) & 1u, a.status);
        }
    } else if (warp <= 4) {
        // ---------------- epilogue ----------------
        // each (template, batch) in order, once its last OUTPUT has finished:
        // OUTPUT accumulators -> z. Each warp reads its tensor-memory quadrant
        // q (powers 16 q .. 16 q + 15) as two 16-lane halves.
        const uint32_t lane_base = ((uint32_t)((warp & 3) * 32)) << 16;
        carry_jobs(a, [&](const CarryJob &J) -> bool {
            if (!J.last_tile) return true;
            const int ob = J.e & 1;
            if (!panel_role_all(mbar_wait_ab(&out_full[ob], (J.e >> 1) & 1, a.status, abort))) return false;
            tc_fence_after();
            const int b = J.b0;
            const int nb = min(a.cpb, a.n_chunks - b * a.cpb);
            const int nii = S * nb * LJ;                // columns of this batch
            const uint32_t tb = tmem + lane_base + 256 + 128 * ob;
            // z of stream 0 and 1 at this batch's first sample
            float2 *zb0 = a.z + (int64_t)a.stream0 * a.z_stream_stride + (int64_t)J.t * a.z_row_stride +
                          (int64_t)b * a.cpb * L;
            float2 *zb1 = zb0 + a.z_stream_stride;
            // chunk column c = 4 cb + t % 4 = (chunk S + stream) LJ + j2
            const int tm = lane & 3, qo = tm / LJ, j2 = tm % LJ;
            // 8-column groups per load: all 16 at once, or two loads of 8
            // where the larger carry groups leave fewer registers per thread
            constexpr int kEp = S == 2 ? 8 : 16;
#pragma unroll 1
            for (int hp = 0; hp < 2 * (16 / kEp); ++hp) {
                const int hf = hp / (16 / kEp), cp = hp % (16 / kEp);
                // lanes 16 hf .. 16 hf + 15 of the quadrant: thread t gets the
                // re row of power jj (lane t / 4) and its im row (lane t / 4 + 8),
                // columns 2 (t % 4) and 2 (t % 4) + 1 of every 8
                const int jj = (warp & 3) * 16 + 8 * hf + (lane >> 2);
                uint32_t v[4 * kEp];
                const uint32_t ta = tb + ((uint32_t)(16 * hf) << 16) + (uint32_t)(8 * kEp * cp);
                if constexpr (kEp == 16) tmem_ld16x256_x16(ta, v);
                else tmem_ld16x256_x8(ta, v);
                tmem_wait_ld();
#pragma unroll
                for (int cl = 0; cl < kEp; ++cl) {
                    const int cb = cp * kEp + cl;
                    const int c = 4 * cb + tm;
                    if (c < nii) {
                        const int q = (4 * cb) / LJ + qo;
                        float2 *zp = ((q % S) ? zb1 : zb0) + (q / S) * L + kJ * j2 + jj;
                        const float r0 = __uint_as_float(v[4 * cl]), r1 = __uint_as_float(v[4 * cl + 1]);
                        const float r2 = __uint_as_float(v[4 * cl + 2]), r3 = __uint_as_float(v[4 * cl + 3]);
                        *zp = make_float2(a.scale * (r0 - r3), a.scale * (r1 + r2));
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&out_free[ob]);
            return true;
        });
    } else {
        // ---------------- carry groups ----------------
        // group g = warps 5 + g kGW .. 5 + g kGW + kGW - 1; a thread owns
        // filter k of the tile (its tensor-memory lane) in stream ss
        const int grp = (warp - 5) / kGW;
        const int ss = ((warp - 5) % kGW) >> 2;
        const int k = (warp & 3) * 32 + lane;                 // tensor-memory lane = filter
        const uint32_t lane_base = ((uint32_t)((warp & 3) * 32)) << 16;
        const uint32_t kofs = (uint32_t)(k >> 3) * kWK + (k & 7) * 16;
        uint32_t n_state = 0;
        carry_jobs(a, [&](const CarryJob &J) -> bool {
            if (J.g != grp) return true;
            const int wl = J.w;
            const int64_t slot = (int64_t)J.tile * kTile + k;
            const float2 ak = a.a[slot], aJ = a.aJ[slot], ck = a.c[slot], aLf = a.aLf[slot];
            const Anchor aLb = reinterpret_cast<const Anchor *>(a.aLb)[slot];
            Anchor *vp = reinterpret_cast<Anchor *>(a.v) + (int64_t)(a.stream0 + ss) * a.n_slots + slot;
            // per job: aJ^i2 for the state sums, a^(kJ j2) a c for the outputs
            float2 pj[LJ], cj[LJ];
            pj[0] = make_float2(1.f, 0.f);
            cj[0] = cmul(ak, ck);
#pragma unroll
            for (int i = 1; i < LJ; ++i) {
                pj[i] = cmul(pj[i - 1], aJ);
                cj[i] = cmul(cj[i - 1], aJ);
            }
            // the same factors as packed pairs (j2, j2 + 1) for f32x2 products
            float2 cjr[LJ / 2], cji[LJ / 2], ncji[LJ / 2];
#pragma unroll
            for (int i = 0; i < LJ / 2; ++i) {
                cjr[i] = make_float2(cj[2 * i].x, cj[2 * i + 1].x);
                cji[i] = make_float2(cj[2 * i].y, cj[2 * i + 1].y);
                ncji[i] = make_float2(-cj[2 * i].y, -cj[2 * i + 1].y);
            }
            Anchor v = *vp;
            if (!mbar_wait_ab(&state_full[grp], n_state & 1, a.status, abort)) return false;
            ++n_state;
            tc_fence_after();
            const int b = J.b0;
            const int nb = min(a.cpb, a.n_chunks - b * a.cpb);
            // Carry across this batch. The batch's starting state v is an
            // FP64 (or double-float) anchor; chunk states inside the batch are
            // FP32 offsets from it:
            //   v_c = a^(cL) v + d_c,  d_{c+1} = a^L d_c + U_c,  d_0 = 0,
            // and the next batch starts from a^(nb L) v + d_nb in the anchor's
            // arithmetic: p = a^(cL) v, dd = d_c (MODE 2: vc = the chunk's
            // starting state in FP64, v_{c+1} = a^L v_c + U_c).
            float2 p = anchor_f32(v), dd = make_float2(0.f, 0.f);
            double2 vc = CH ? reinterpret_cast<const double2 &>(v) : make_double2(0.0, 0.0);
            const double2 aL64 = CH ? reinterpret_cast<const double2 *>(a.aL)[slot] : make_double2(0.0, 0.0);
            // Chunk c's sums G(i2) for this stream are STATE columns
            // (ss LJ + i2) kMaxC + c (re; im kNii further on): the chunks of a
            // power block are adjacent, so the sums of two chunks form one
            // packed f32x2 operand. Its W goes to columns 2 (c S + ss) LJ ..
            // + 2 LJ - 1: 4 LJ contiguous bytes at (k/8) kWK + n / 8 * 128 +
            // (n % 8) * 2 + (k%8) 16, n = 2 (c S + ss) LJ.
            const uint32_t tb = tmem + lane_base + 128 * grp;
            constexpr int kMaxC = kNii / (S * LJ);
            // Two streams: first every chunk's U = sum_i2 aJ^i2 G(i2), then the
            // group's STATE columns are released and W is made, so that the
            // group's next STATE contraction runs meanwhile. One stream: U and
            // W chunk by chunk (its sixteen U would not fit the registers) and
            // the columns are released at the last read.
            constexpr bool kUFirst = S == 2;
            constexpr int kR = 16 / LJ;                     // chunks per tensor-memory round trip
            // a round: every power block's sums of chunks pp kR .. pp kR + kR - 1
            auto load_round = [&](int pp, uint32_t(&rr)[LJ][kR], uint32_t(&ri)[LJ][kR]) {
#pragma unroll
                for (int i2 = 0; i2 < LJ; ++i2) {
                    const uint32_t col = (uint32_t)((ss * LJ + i2) * kMaxC + pp * kR);
                    tmem_ld_n(tb + col, rr[i2]);
                    tmem_ld_n(tb + kNii + col, ri[i2]);
                }
                tmem_wait_ld();
            };
            // U of the round's chunks i, i + 1 (i even), two chunks per packed
            // operation; each element takes the scalar order
            // u = fma(Re aJ^i2, g, fma(-+Im aJ^i2, g', u)) over i2 = 1 ..
            auto u_pair = [&](const uint32_t(&rr)[LJ][kR], const uint32_t(&ri)[LJ][kR], int i, float2 &u0,
                              float2 &u1) {
                float2 ur = make_float2(__uint_as_float(rr[0][i]), __uint_as_float(rr[0][i + 1]));
                float2 ui = make_float2(__uint_as_float(ri[0][i]), __uint_as_float(ri[0][i + 1]));
#pragma unroll
                for (int i2 = 1; i2 < LJ; ++i2) {
                    const float2 gr = make_float2(__uint_as_float(rr[i2][i]), __uint_as_float(rr[i2][i + 1]));
                    const float2 gi = make_float2(__uint_as_float(ri[i2][i]), __uint_as_float(ri[i2][i + 1]));
                    const float2 px = make_float2(pj[i2].x, pj[i2].x), py = make_float2(pj[i2].y, pj[i2].y);
                    const float2 npy = make_float2(-pj[i2].y, -pj[i2].y);
                    ur = __ffma2_rn(px, gr, __ffma2_rn(npy, gi, ur));
                    ui = __ffma2_rn(px, gi, __ffma2_rn(py, gr, ui));
                }
                u0 = make_float2(ur.x, ui.x);
                u1 = make_float2(ur.y, ui.y);
            };
            // W of chunk c, then the carry to chunk c + 1
            auto w_step = [&](unsigned char *W, int c, float2 Uc) {
                const int n = 2 * (c * S + ss) * LJ;
                const uint32_t off = kofs + (uint32_t)(n >> 3) * 128 + (n & 7) * 2;
                float wr[LJ], wi[LJ];
                if (c < nb) {
                    const float2 vv = CH ? make_float2((float)vc.x, (float)vc.y)
                                         : make_float2(p.x + dd.x, p.y + dd.y);
                    const float2 vx = make_float2(vv.x, vv.x), vy = make_float2(vv.y, vv.y);
#pragma unroll
                    for (int i3 = 0; i3 < LJ / 2; ++i3) {      // w = a^(kJ j2) a c vv
                        const float2 r = __ffma2_rn(ncji[i3], vy, __fmul2_rn(cjr[i3], vx));
                        const float2 m = __ffma2_rn(cji[i3], vx, __fmul2_rn(cjr[i3], vy));
                        wr[2 * i3] = r.x;
                        wr[2 * i3 + 1] = r.y;
                        wi[2 * i3] = m.x;
                        wi[2 * i3 + 1] = m.y;
                    }
                    if constexpr (CH) {
                        vc = make_double2(fma(aL64.x, vc.x, fma(-aL64.y, vc.y, (double)Uc.x)),
                                          fma(aL64.x, vc.y, fma(aL64.y, vc.x, (double)Uc.y)));
                    } else {
                        dd = make_float2(fmaf(aLf.x, dd.x, fmaf(-aLf.y, dd.y, Uc.x)),
                                         fmaf(aLf.x, dd.y, fmaf(aLf.y, dd.x, Uc.y)));
                        p = cmul(aLf, p);
                    }
                } else {
                    // columns past this batch contribute nothing
#pragma unroll
                    for (int j2 = 0; j2 < LJ; ++j2) wr[j2] = wi[j2] = 0.f;
                }
                if constexpr (LJ == 4) {
                    *reinterpret_cast<uint4 *>(W + off) =
                        make_uint4(pack2<BF16>(wr[0], wi[0]), pack2<BF16>(wr[1], wi[1]),
                                   pack2<BF16>(wr[2], wi[2]), pack2<BF16>(wr[3], wi[3]));
                } else {
                    *reinterpret_cast<uint2 *>(W + off) =
                        make_uint2(pack2<BF16>(wr[0], wi[0]), pack2<BF16>(wr[1], wi[1]));
                }
            };
            // W's slot is free once the OUTPUT two jobs back has finished
            const int use = J.j / kWSlots;
            unsigned char *W = Wb + wl * kWBytes;
            if constexpr (kUFirst) {
                float2 U[kMaxC];
#pragma unroll
                for (int pp = 0; pp < kMaxC / kR; ++pp) {
                    uint32_t rr[LJ][kR], ri[LJ][kR];
                    load_round(pp, rr, ri);
#pragma unroll
                    for (int i = 0; i < kR; i += 2) u_pair(rr, ri, i, U[pp * kR + i], U[pp * kR + i + 1]);
                }
                tc_fence_before();
                mbar_arrive(&state_free[grp]);
                if (use > 0 && !mbar_wait_ab(&w_free[wl], (use - 1) & 1, a.status, abort)) return false;
#pragma unroll
                for (int c = 0; c < kMaxC; ++c) w_step(W, c, U[c]);
            } else {
                if (use > 0 && !mbar_wait_ab(&w_free[wl], (use - 1) & 1, a.status, abort)) return false;
#pragma unroll
                for (int pp = 0; pp < kMaxC / kR; ++pp) {
                    uint32_t rr[LJ][kR], ri[LJ][kR];
                    load_round(pp, rr, ri);
                    if (pp == kMaxC / kR - 1) {
                        tc_fence_before();
                        mbar_arrive(&state_free[grp]);
                    }
#pragma unroll
                    for (int i = 0; i < kR; i += 2) {
                        float2 u0, u1;
                        u_pair(rr, ri, i, u0, u1);
                        w_step(W, pp * kR + i, u0);
                        w_step(W, pp * kR + i + 1, u1);
                    }
                }
            }
            // W is complete: the OUTPUT contraction may start during the
            // state update below
            fence_async_smem();
            mbar_arrive(&w_full[wl]);
            if constexpr (CH) {
                *vp = reinterpret_cast<const Anchor &>(vc);
                return true;
            }
            // v <- a^(nb L) v + d_nb in the anchor's arithmetic
            Anchor pw;
            if (nb == a.cpb) {
                pw = aLb;
            } else {
                const Anchor aL = reinterpret_cast<const Anchor *>(a.aL)[slot];
                pw = aL;
                for (int i = 1; i < nb; ++i) pw = anchor_madd(pw, aL, make_float2(0.f, 0.f));
            }
            *vp = anchor_madd(pw, v, dd);
            return true;
        });
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free(tmem, 512);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct TcBank {
    int T = 0, S = 0, L = 256, F = 0, K = 0, n_groups = 0, n_slices = 0;
    int n_carry_ctas = 0, n_tiles = 0;
    int64_t n_slots = 0;
    int64_t max_n = 0, ring_len = 0, xbuf_stride = 0;
    bool bf16 = false;
    float scale = 0.f;
    int max_delay = 0;
    // device
    uint4 *H = nullptr;
    float *row_scale = nullptr;
    int32_t *tile_ptr = nullptr, *tmpl_of = nullptr;
    uint8_t *has_carry = nullptr;
    float2 *a = nullptr, *aJ = nullptr, *c = nullptr, *aLf = nullptr;
    uint4 *aL = nullptr, *v = nullptr, *aLb1 = nullptr, *aLb2 = nullptr;   // FP64 or double-float
    bool df = false;                          // double-float carry
    int carry_mode = 0;                       // 0 FP64 per batch, 1 double-float, 2 FP64 per chunk
    float *xbuf = nullptr, *stage = nullptr;
    float2 *z = nullptr;
    unsigned int *status = nullptr;
    uint4 *hank = nullptr, *xseg = nullptr;   // staged strain operands
    bool split = false;                       // split bf16: FIR in three passes
    uint4 *H_lo = nullptr, *hank_lo = nullptr;
    uint8_t *all_rows = nullptr;
    uint4 *panel = nullptr;                   // carry tiles' power panels
    std::vector<int64_t> slot_k;              // filter of each carry slot (-1: padding)
    int64_t n_filters = 0;
    int hank_bytes = 0;
    int n_sms = 1;
    std::vector<int64_t> last_n;
    int64_t footprint = 0;
};

namespace {

constexpr int kFirSmem = kStages * kSliceBytes;
int hank_bytes_of(int L, int K) { return (L + K) / 8 * 128; }
int fir_smem_of(int L, int K) { return kFirSmem + 2 * hank_bytes_of(L, K); }
int carry_cpb(int streams, int L) { return std::max(1, kNii / (streams * (L / kJ))); }

struct TcPlan {
    int T, L, F, K, n_groups, n_slices, n_tiles;
    int64_t n_slots, max_n, ring_len, xbuf_stride;
    int max_delay;
};

spiir_status tc_plan(const spiir_bank_desc *d, TcPlan &p) {
    p.L = d->chunk_len ? d->chunk_len : 256;
    if (p.L != 128 && p.L != 256)
        return tc_fail(SPIIR_EUNSUPPORTED, "tensor-core form: chunk_len must be 128 or 256");
    if (d->block_len % p.L != 0)
        return tc_fail(SPIIR_EINVAL, "tensor-core form: block_len must be a multiple of chunk_len");
    p.T = d->n_templates;
    int md = 0;
    std::vector<int64_t> cnt(p.T, 0);
    for (int64_t k = 0; k < d->n_filters; ++k) {
        md = std::max(md, d->delay[k]);
        cnt[d->template_id[k]]++;
    }
    p.max_delay = md;
    p.F = (int)(((int64_t)md + 1 + 63) / 64 * 64);
    p.K = p.F + p.L;
    if (fir_smem_of(p.L, p.K) > 220 * 1024)
        return tc_fail(SPIIR_EUNSUPPORTED, "tensor-core form: delays too long for the FIR tile");
    p.n_groups = (p.T + kGroup - 1) / kGroup;
    p.n_slices = p.K / kKs;
    p.n_tiles = 0;
    for (int t = 0; t < p.T; ++t) p.n_tiles += (int)((cnt[t] + kTile - 1) / kTile);
    p.n_slots = (int64_t)p.n_tiles * kTile;
    p.max_n = (int64_t)d->block_len * d->max_push_blocks;
    p.ring_len = (p.max_n + 1) / 2 * 2;
    p.xbuf_stride = (p.F + p.max_n + 64 + 3) / 4 * 4;
    return SPIIR_OK;
}

int64_t tc_bytes(const spiir_bank_desc *d, const TcPlan &p) {
    const int64_t S = d->n_streams;
    int64_t b = 0;
    b += (int64_t)p.n_groups * p.n_slices * kSliceBytes;
    b += (int64_t)p.T * 4 + (p.T + 1) * 4 + p.T * 4;
    b += p.n_slots * (8 * 4 + 16 * 3);
    b += (int64_t)p.n_tiles * kPanelBytes;
    b += S * p.n_slots * 16;
    b += S * p.xbuf_stride * 4 + S * p.ring_len * 4;
    b += S * (int64_t)p.T * p.ring_len * 8;
    const int64_t C = p.max_n / p.L;
    b += S * C * hank_bytes_of(p.L, p.K);
    b += (C * S * (p.L / kJ) / kNii + 2) * kXsegBytes;
    if (d->mode == SPIIR_TC_BF16X2)     // low parts of H and of the Toeplitz sources
        b += (int64_t)p.n_groups * p.n_slices * kSliceBytes + S * C * hank_bytes_of(p.L, p.K) + p.T;
    return b + 256;
}

// An anchor value as the carry kernel reads it: FP64 {re, im}, or the
// double-float split {re hi, im hi, re lo, im lo}.
uint4 host_anchor(std::complex<double> x, bool df) {
    uint4 r;
    if (df) {
        const float rh = (float)x.real(), ih = (float)x.imag();
        const float4 f = make_float4(rh, ih, (float)(x.real() - (double)rh), (float)(x.imag() - (double)ih));
        std::memcpy(&r, &f, sizeof r);
    } else {
        const double2 f = make_double2(x.real(), x.imag());
        std::memcpy(&r, &f, sizeof r);
    }
    return r;
}

// The carry kernel's instantiations, indexed 12 bf16 + 6 (L = 128) + 3 (two
// streams) + carry mode (0 FP64 anchor per batch, 1 double-float anchor, 2
// FP64 per chunk).
using CarryFn = void (*)(const TcCarryArgs);
constexpr int kCarryFns = 24;
CarryFn carry_kernel(int i) {
    static const CarryFn k[kCarryFns] = {
        tc_carry_kernel<false, 4, 1, 0>, tc_carry_kernel<false, 4, 1, 1>, tc_carry_kernel<false, 4, 1, 2>,
        tc_carry_kernel<false, 4, 2, 0>, tc_carry_kernel<false, 4, 2, 1>, tc_carry_kernel<false, 4, 2, 2>,
        tc_carry_kernel<false, 2, 1, 0>, tc_carry_kernel<false, 2, 1, 1>, tc_carry_kernel<false, 2, 1, 2>,
        tc_carry_kernel<false, 2, 2, 0>, tc_carry_kernel<false, 2, 2, 1>, tc_carry_kernel<false, 2, 2, 2>,
        tc_carry_kernel<true, 4, 1, 0>,  tc_carry_kernel<true, 4, 1, 1>,  tc_carry_kernel<true, 4, 1, 2>,
        tc_carry_kernel<true, 4, 2, 0>,  tc_carry_kernel<true, 4, 2, 1>,  tc_carry_kernel<true, 4, 2, 2>,
        tc_carry_kernel<true, 2, 1, 0>,  tc_carry_kernel<true, 2, 1, 1>,  tc_carry_kernel<true, 2, 1, 2>,
        tc_carry_kernel<true, 2, 2, 0>,  tc_carry_kernel<true, 2, 2, 1>,  tc_carry_kernel<true, 2, 2, 2>,
    };
    return k[i];
}

uint16_t host16(float x, bool bf16) {
    if (bf16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}

template <typename T>
spiir_status tc_upload(T **dst, const std::vector<T> &src, cudaStream_t s) {
    *dst = nullptr;
    if (src.empty()) return SPIIR_OK;
    TC_CUDA(cudaMalloc((void **)dst, src.size() * sizeof(T)));
    TC_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return SPIIR_OK;
}

}  // namespace

int spiir_tc_hank_bytes(int L, int K) { return hank_bytes_of(L, K); }
int spiir_tc_xseg_bytes() { return kXsegBytes; }
int spiir_tc_cpb(int streams, int L) { return carry_cpb(streams, L); }

spiir_status spiir_tc_pack(const spiir_bank_desc *d, int level, int F, int L, double row_mult, bool bf16,
                           bool df, TcPack &pk, bool split) {
    split = split && bf16;
    pk = TcPack();
    const int T = d->n_templates;
    const int K = F + L;
    pk.T = T;
    pk.F = F;
    pk.L = L;
    pk.K = K;
    pk.n_groups = (T + kGroup - 1) / kGroup;
    pk.n_slices = K / kKs;
    // filters per template in input order
    std::vector<std::vector<int64_t>> fl(T);
    for (int64_t k = 0; k < d->n_filters; ++k) {
        if (level >= 0 && (d->level ? d->level[k] : 0) != level) continue;
        if (d->delay[k] >= F) return tc_fail(SPIIR_EINVAL, "tensor-core form: a delay is not below F");
        fl[d->template_id[k]].push_back(k);
    }

    // Impulse responses h_t[q], q < K, in FP64; rows scaled by 2^e_t into the
    // 16-bit range; tiles [group][slice][r/8][k/8][r%8][k%8].
    pk.H.assign((size_t)pk.n_groups * pk.n_slices * (kSliceBytes / 2), 0);
    if (split) pk.H_lo.assign(pk.H.size(), 0);
    pk.row_scale.assign(T, 0.f);
    auto work = [&](int t0, int t1) {
        std::vector<std::complex<double>> h(K);
        for (int t = t0; t < t1; ++t) {
            std::fill(h.begin(), h.end(), std::complex<double>(0, 0));
            for (int64_t k : fl[t]) {
                const std::complex<double> a(d->a_re[k], d->a_im[k]);
                std::complex<double> pw(d->b_re[k], d->b_im[k]);
                for (int q = d->delay[k]; q < K; ++q) {
                    h[q] += pw;
                    pw *= a;
                }
            }
            double mx = 0.0;
            for (int q = 0; q < K; ++q) mx = std::max(mx, std::max(std::fabs(h[q].real()), std::fabs(h[q].imag())));
            int e = 0;
            if (mx > 0.0) {
                int ex;
                std::frexp(mx, &ex);          // mx in [2^(ex-1), 2^ex)
                e = 10 - ex;                  // max |h| * 2^e in [2^9, 2^10)
            }
            const double sc = std::ldexp(1.0, e);
            pk.row_scale[t] = (float)(row_mult * std::ldexp(1.0, -e));
            const int g = t / kGroup;
            for (int comp = 0; comp < 2; ++comp) {
                const int r = 2 * (t % kGroup) + comp;
                for (int q = 0; q < K; ++q) {
                    const double val = (comp ? h[q].imag() : h[q].real()) * sc;
                    const int sl = q / kKs, kq = q % kKs;
                    const size_t off = ((size_t)g * pk.n_slices + sl) * (kSliceBytes / 2) +
                                       (size_t)(r >> 3) * 512 + (kq >> 3) * 64 + (r & 7) * 8 + (kq & 7);
                    pk.H[off] = host16((float)val, bf16);
                    if (split) {
                        // hi + lo carries about 16 significant bits of h
                        const double hi = (double)__bfloat162float(__ushort_as_bfloat16(pk.H[off]));
                        pk.H_lo[off] = host16((float)(val - hi), true);
                    }
                }
            }
        }
    };
    const int nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    {
        std::vector<std::thread> th;
        for (int i = 0; i < nth; ++i) {
            const int t0 = (int)((int64_t)T * i / nth), t1 = (int)((int64_t)T * (i + 1) / nth);
            th.emplace_back(work, t0, t1);
        }
        for (auto &x : th) x.join();
    }

    // Carry tiles: 128 filter slots each, template-major.
    int n_tiles = 0;
    for (int t = 0; t < T; ++t) n_tiles += (int)((fl[t].size() + kTile - 1) / kTile);
    pk.n_tiles = n_tiles;
    const int64_t n_slots = (int64_t)n_tiles * kTile;
    pk.tile_ptr.assign(T + 1, 0);
    pk.has_carry.assign(T, 0);
    pk.a.assign(n_slots, make_float2(0.f, 0.f));
    pk.aJ = pk.c = pk.aLf = pk.a;
    pk.aL.assign(n_slots, make_uint4(0u, 0u, 0u, 0u));
    pk.aLb1 = pk.aLb2 = pk.aL;
    pk.slot_k.assign(n_slots, -1);
    const int cpb1 = carry_cpb(1, L), cpb2 = carry_cpb(2, L);
    int tile = 0;
    for (int t = 0; t < T; ++t) {
        pk.tile_ptr[t] = tile;
        const int nt = (int)((fl[t].size() + kTile - 1) / kTile);
        if (nt) pk.has_carry[t] = 1;
        for (int i = 0; i < (int)fl[t].size(); ++i) {
            const int64_t slot = (int64_t)tile * kTile + i;
            const int64_t k = fl[t][i];
            pk.slot_k[slot] = k;
            const std::complex<double> a(d->a_re[k], d->a_im[k]), bb(d->b_re[k], d->b_im[k]);
            auto pw = [&](int n) {
                std::complex<double> r(1, 0), x = a;
                while (n) {
                    if (n & 1) r *= x;
                    x *= x;
                    n >>= 1;
                }
                return r;
            };
            const std::complex<double> aL = pw(L), ck = pw(F - d->delay[k]) * bb;
            pk.a[slot] = make_float2(d->a_re[k], d->a_im[k]);
            const auto pJ = pw(kJ);
            pk.aJ[slot] = make_float2((float)pJ.real(), (float)pJ.imag());
            pk.aL[slot] = host_anchor(aL, df);
            pk.aLf[slot] = make_float2((float)aL.real(), (float)aL.imag());
            pk.aLb1[slot] = host_anchor(pw(L * cpb1), df);
            pk.aLb2[slot] = host_anchor(pw(L * cpb2), df);
            pk.c[slot] = make_float2((float)ck.real(), (float)ck.imag());
        }
        tile += nt;
    }
    pk.tile_ptr[T] = tile;
    // Power panel of each tile (the layout the carry kernel copies into a
    // slot): a_k^j, j < kJ, in FP64 and rounded once to the operand type.
    pk.panel.assign((size_t)n_tiles * (kPanelBytes / 2), 0);
    {
        auto pwork = [&](int64_t t0, int64_t t1) {
            for (int64_t tl = t0; tl < t1; ++tl)
                for (int kk = 0; kk < kTile; ++kk) {
                    const int64_t k = pk.slot_k[tl * kTile + kk];
                    const std::complex<double> a =
                        k >= 0 ? std::complex<double>(d->a_re[k], d->a_im[k]) : std::complex<double>(0, 0);
                    std::complex<double> x(1, 0);
                    // [k/8][m/8][k%8][m%8]: row group 2 (j/8) = Re, 2 (j/8) + 1 = Im
                    uint16_t *P = pk.panel.data() + (size_t)tl * (kPanelBytes / 2) + (kk >> 3) * 1024 + (kk & 7) * 8;
                    for (int j = 0; j < kJ; ++j) {
                        const int g = 2 * (j >> 3);
                        P[g * 64 + (j & 7)] = host16((float)x.real(), bf16);
                        P[(g + 1) * 64 + (j & 7)] = host16((float)x.imag(), bf16);
                        x *= a;
                    }
                }
        };
        std::vector<std::thread> th;
        for (int i = 0; i < nth; ++i)
            th.emplace_back(pwork, (int64_t)n_tiles * i / nth, (int64_t)n_tiles * (i + 1) / nth);
        for (auto &x : th) x.join();
    }
    return SPIIR_OK;
}

spiir_status spiir_tc_prepare(int L, int K) {
    int dev = 0, max_optin = 0;
    TC_CUDA(cudaGetDevice(&dev));
    TC_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const void *fns[2 + kCarryFns];
    int need[2 + kCarryFns];
    fns[0] = (const void *)tc_fir_kernel<true>;
    fns[1] = (const void *)tc_fir_kernel<false>;
    need[0] = need[1] = fir_smem_of(L, K);
    for (int i = 0; i < kCarryFns; ++i) {
        fns[2 + i] = (const void *)carry_kernel(i);
        need[2 + i] = kCarrySmem;
    }
    // kernel-wide limits shared by every bank: the device maximum
    for (int i = 0; i < 2 + kCarryFns; ++i) {
        cudaFuncAttributes fa;
        TC_CUDA(cudaFuncGetAttributes(&fa, fns[i]));
        const int dyn_max = max_optin - (int)fa.sharedSizeBytes;
        if (need[i] > dyn_max)
            return tc_fail(SPIIR_EUNSUPPORTED, "tensor-core form: shared memory above the device limit");
        TC_CUDA(cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
    }
    return SPIIR_OK;
}

spiir_status spiir_tc_launch(const TcLaunch &l, cudaStream_t s, KernelTimer *timer) {
    const int C = l.n_chunks, count = l.n_streams;
    const int cpb = carry_cpb(count, l.L);
    const int n_batches = (C + cpb - 1) / cpb;
    const int hb = hank_bytes_of(l.L, l.K);
    TcStageArgs sa{};
    sa.xbuf = l.xbuf;
    sa.xbuf_stride = l.xbuf_stride;
    sa.hist = l.hist;
    sa.F = l.F;
    sa.L = l.L;
    sa.K = l.K;
    sa.n_chunks = C;
    sa.n_streams = count;
    sa.stream0 = l.stream0;
    sa.cpb = cpb;
    sa.n_batches = n_batches;
    sa.hank = l.hank;
    sa.hank_lo = l.H_lo ? l.hank_lo : nullptr;
    sa.hank_bytes = hb;
    sa.xseg = l.xseg;
    {
        const int64_t chunks = (int64_t)count * C * (hb / 16) + (int64_t)n_batches * (kXsegBytes / 16);
        const int grid = (int)std::min<int64_t>((chunks + 255) / 256, 8LL * l.n_sms);
        if (timer) timer->begin(SPIIR_K_TC_STAGE, s);
        if (l.bf16)
            tc_stage_kernel<true><<<grid, 256, 0, s>>>(sa);
        else
            tc_stage_kernel<false><<<grid, 256, 0, s>>>(sa);
        TC_CUDA(cudaGetLastError());
        if (timer) timer->end(s);
    }
    // the carry kernel writes the state term into z; the FIR kernel adds to it
    if (l.n_carry > 0) {
        TcCarryArgs ca{};
        ca.tile_ptr = l.tile_ptr;
        ca.tile_end = l.tile_end;
        ca.tmpl_of = l.tmpl_of;
        ca.n_carry = l.n_carry;
        ca.a = l.a;
        ca.aJ = l.aJ;
        ca.aL = l.aL;
        ca.aLf = l.aLf;
        ca.aLb = count == 1 ? l.aLb1 : l.aLb2;
        ca.c = l.c;
        ca.v = l.v;
        ca.n_slots = l.n_slots;
        ca.xseg = l.xseg;
        ca.L = l.L;
        ca.n_chunks = C;
        ca.n_streams = count;
        ca.stream0 = l.stream0;
        ca.cpb = cpb;
        ca.n_batches = n_batches;
        ca.scale = l.carry_scale;
        ca.z = l.z;
        ca.z_row_stride = l.z_row_stride;
        ca.z_stream_stride = l.z_stream_stride;
        ca.status = l.status;
        ca.panel = l.panel;
        const int grid = std::min(l.n_carry, l.n_sms);
        if (timer) timer->begin(SPIIR_K_TC_CARRY, s);
        const bool l2 = l.L == 2 * kJ, two = count == 2;
        carry_kernel(12 * l.bf16 + 6 * l2 + 3 * two + l.carry_mode)<<<grid, carry_warps(count) * 32, kCarrySmem, s>>>(ca);
        TC_CUDA(cudaGetLastError());
        if (timer) timer->end(s);
    }
    if (l.n_groups > 0) {
        TcFirArgs fa{};
        fa.H = l.H;
        fa.row_scale = l.row_scale;
        fa.has_carry = l.has_carry;
        fa.groups = l.groups;
        fa.hank = l.hank;
        fa.hank_bytes = hb;
        fa.L = l.L;
        fa.K = l.K;
        fa.n_groups = l.n_groups;
        fa.n_chunks = C;
        fa.n_streams = count;
        fa.n_templates = l.n_rows;
        fa.stream0 = l.stream0;
        fa.z = l.z;
        fa.z_row_stride = l.z_row_stride;
        fa.z_stream_stride = l.z_stream_stride;
        fa.status = l.status;
        const int items = l.n_groups * C * count;
        const int grid = std::min(items, l.n_sms);
        const int smem = fir_smem_of(l.L, l.K);
        // split bf16: H x_hi, then H x_lo and H_lo x_hi added to z (the
        // product of the two low parts, about 2^-16 of the result, is left out)
        const int passes = l.H_lo ? 3 : 1;
        if (timer) timer->begin(SPIIR_K_TC_FIR, s);
        for (int pass = 0; pass < passes; ++pass) {
            if (pass > 0) {
                fa.has_carry = l.all_rows;
                fa.hank = pass == 1 ? l.hank_lo : l.hank;
                fa.H = pass == 1 ? l.H : l.H_lo;
            }
            if (l.bf16)
                tc_fir_kernel<true><<<grid, kFirThreads, smem, s>>>(fa);
            else
                tc_fir_kernel<false><<<grid, kFirThreads, smem, s>>>(fa);
            TC_CUDA(cudaGetLastError());
        }
        if (timer) timer->end(s, passes);
    }
    return SPIIR_OK;
}

spiir_status spiir_tc_create(const spiir_bank_desc *d, float scale, cudaStream_t s, TcBank **out,
                             int64_t *footprint) {
    *out = nullptr;
    TcPlan p;
    spiir_status st = tc_plan(d, p);
    if (st) return st;
    const int64_t bytes = tc_bytes(d, p);
    if (d->hbm_budget_bytes > 0 && bytes > d->hbm_budget_bytes)
        return tc_fail(SPIIR_EBUDGET, "tensor-core bank above hbm_budget_bytes");
    TcBank *b = new TcBank();
    b->T = p.T;
    b->S = d->n_streams;
    b->L = p.L;
    b->F = p.F;
    b->K = p.K;
    b->n_groups = p.n_groups;
    b->n_slices = p.n_slices;
    b->n_tiles = p.n_tiles;
    b->n_slots = p.n_slots;
    b->max_n = p.max_n;
    b->ring_len = p.ring_len;
    b->xbuf_stride = p.xbuf_stride;
    b->bf16 = d->mode != SPIIR_TC_FP16;
    b->split = d->mode == SPIIR_TC_BF16X2;
    b->df = d->carry == 1;
    b->carry_mode = d->carry;
    b->scale = scale;
    b->max_delay = p.max_delay;
    b->last_n.assign(d->n_streams, 0);
    b->footprint = bytes;
    *footprint = bytes;
    *out = b;

    TcPack pk;
    if ((st = spiir_tc_pack(d, -1, p.F, p.L, scale, b->bf16, b->df, pk, b->split))) return st;
    std::vector<int32_t> tmpl_of;
    for (int t = 0; t < p.T; ++t)
        if (pk.has_carry[t]) tmpl_of.push_back(t);
    b->n_carry_ctas = (int)tmpl_of.size();
    b->n_filters = d->n_filters;
    if ((st = tc_upload(&b->H, std::vector<uint4>((uint4 *)pk.H.data(), (uint4 *)(pk.H.data() + pk.H.size())), s)))
        return st;
    if (b->split) {
        if ((st = tc_upload(&b->H_lo, std::vector<uint4>((uint4 *)pk.H_lo.data(),
                                                         (uint4 *)(pk.H_lo.data() + pk.H_lo.size())), s)))
            return st;
        if ((st = tc_upload(&b->all_rows, std::vector<uint8_t>(std::max(1, p.T), 1), s))) return st;
    }
    if ((st = tc_upload(&b->row_scale, pk.row_scale, s))) return st;
    if ((st = tc_upload(&b->tile_ptr, pk.tile_ptr, s))) return st;
    if ((st = tc_upload(&b->tmpl_of, tmpl_of, s))) return st;
    if ((st = tc_upload(&b->has_carry, pk.has_carry, s))) return st;
    if ((st = tc_upload(&b->a, pk.a, s))) return st;
    if ((st = tc_upload(&b->aJ, pk.aJ, s))) return st;
    if ((st = tc_upload(&b->c, pk.c, s))) return st;
    if ((st = tc_upload(&b->aL, pk.aL, s))) return st;
    if ((st = tc_upload(&b->aLf, pk.aLf, s))) return st;
    if ((st = tc_upload(&b->aLb1, pk.aLb1, s))) return st;
    if ((st = tc_upload(&b->aLb2, pk.aLb2, s))) return st;
    if ((st = tc_upload(&b->panel,
                        std::vector<uint4>((uint4 *)pk.panel.data(), (uint4 *)(pk.panel.data() + pk.panel.size())),
                        s)))
        return st;
    b->slot_k = std::move(pk.slot_k);
    const int64_t S = d->n_streams;
    TC_CUDA(cudaMalloc((void **)&b->v, std::max<int64_t>(1, S * p.n_slots) * sizeof(uint4)));
    TC_CUDA(cudaMemsetAsync(b->v, 0, std::max<int64_t>(1, S * p.n_slots) * sizeof(uint4), s));
    TC_CUDA(cudaMalloc((void **)&b->xbuf, S * p.xbuf_stride * sizeof(float)));
    TC_CUDA(cudaMemsetAsync(b->xbuf, 0, S * p.xbuf_stride * sizeof(float), s));
    TC_CUDA(cudaMalloc((void **)&b->stage, S * p.ring_len * sizeof(float)));
    TC_CUDA(cudaMalloc((void **)&b->z, S * (int64_t)p.T * p.ring_len * sizeof(float2)));
    TC_CUDA(cudaMemsetAsync(b->z, 0, S * (int64_t)p.T * p.ring_len * sizeof(float2), s));
    TC_CUDA(cudaMalloc((void **)&b->status, sizeof(unsigned int)));
    TC_CUDA(cudaMemsetAsync(b->status, 0, sizeof(unsigned int), s));
    b->hank_bytes = hank_bytes_of(p.L, p.K);
    const int64_t Cmax = p.max_n / p.L;
    TC_CUDA(cudaMalloc((void **)&b->hank, S * Cmax * b->hank_bytes));
    if (b->split) TC_CUDA(cudaMalloc((void **)&b->hank_lo, S * Cmax * b->hank_bytes));
    const int64_t nbmax = (Cmax + carry_cpb(std::min<int64_t>(S, 2), p.L) - 1) / carry_cpb(std::min<int64_t>(S, 2), p.L) + 1;
    TC_CUDA(cudaMalloc((void **)&b->xseg, std::max<int64_t>(nbmax, Cmax) * kXsegBytes));
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    TC_CUDA(cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, dev));
    if ((st = spiir_tc_prepare(p.L, p.K))) return st;
    TC_CUDA(cudaStreamSynchronize(s));
    return SPIIR_OK;
}

spiir_status spiir_tc_push(TcBank *b, int s0, int count, const float *x, int64_t x_stride, int64_t n,
                           cudaStream_t s, KernelTimer *timer, int64_t zoff) {
    if (n % b->L != 0) return tc_fail(SPIIR_EINVAL, "push length must be a multiple of chunk_len");
    const int64_t n_prev = b->last_n[s0];
    for (int q = s0; q < s0 + count; ++q)
        if (b->last_n[q] != n_prev) {
            for (int i = 0; i < count; ++i) {
                spiir_status st = spiir_tc_push(b, s0 + i, 1, x + i * x_stride, x_stride, n, s, timer, zoff);
                if (st) return st;
            }
            return SPIIR_OK;
        }
    // streams are carried two at a time (the carry kernel's thread layout);
    // each pair runs its own prologue
    if (count > 2) {
        for (int i = 0; i < count; i += 2) {
            const int cnt = std::min(2, count - i);
            spiir_status st = spiir_tc_push(b, s0 + i, cnt, x + i * x_stride, x_stride, n, s, timer, zoff);
            if (st) return st;
        }
        return SPIIR_OK;
    }
    // strain history + new samples (single-level prologue)
    PrologueArgs pa{};
    pa.xbuf = b->xbuf;
    pa.xbuf_stream_stride = b->xbuf_stride;
    pa.x_in = x;
    pa.x_in_stream_stride = x_stride;
    pa.stream0 = s0;
    pa.n_levels = 1;
    pa.lev[0].hist = b->F;
    pa.lev[0].n = (int32_t)n;
    pa.lev[0].n_prev = (int32_t)n_prev;
    pa.lev[0].xbuf_off = 0;
    timer->begin(SPIIR_K_TC_STAGE, s);
    TC_CUDA(spiir_launch_prologue(pa, count, s));
    timer->end(s, kPrologueLaunches);

    TcLaunch l{};
    l.xbuf = b->xbuf;
    l.xbuf_stride = b->xbuf_stride;
    l.hist = b->F;
    l.F = b->F;
    l.L = b->L;
    l.K = b->K;
    l.n_chunks = (int)(n / b->L);
    l.n_streams = count;
    l.stream0 = s0;
    l.hank = b->hank;
    l.xseg = b->xseg;
    l.tile_ptr = b->tile_ptr;
    l.tile_end = nullptr;
    l.tmpl_of = b->tmpl_of;
    l.n_carry = b->n_carry_ctas;
    l.a = b->a;
    l.aJ = b->aJ;
    l.aLf = b->aLf;
    l.c = b->c;
    l.aL = b->aL;
    l.aLb1 = b->aLb1;
    l.aLb2 = b->aLb2;
    l.panel = b->panel;
    l.v = b->v;
    l.n_slots = b->n_slots;
    l.carry_scale = b->scale;
    l.H = b->H;
    l.row_scale = b->row_scale;
    l.has_carry = b->has_carry;
    l.H_lo = b->H_lo;
    l.hank_lo = b->hank_lo;
    l.all_rows = b->all_rows;
    l.groups = nullptr;
    l.n_groups = b->n_groups;
    l.n_rows = b->T;
    l.z = b->z + zoff;
    l.z_row_stride = b->ring_len;
    l.z_stream_stride = (int64_t)b->T * b->ring_len;
    l.bf16 = b->bf16;
    l.df = b->df;
    l.carry_mode = b->carry_mode;
    l.status = b->status;
    l.n_sms = b->n_sms;
    spiir_status st = spiir_tc_launch(l, s, timer);
    if (st) return st;
    for (int q = s0; q < s0 + count; ++q) b->last_n[q] = n;
    return SPIIR_OK;
}

spiir_status spiir_tc_reset(TcBank *b, int s0, int count, cudaStream_t s) {
    if (b->n_slots)
        TC_CUDA(cudaMemsetAsync(b->v + (int64_t)s0 * b->n_slots, 0, count * b->n_slots * sizeof(uint4), s));
    TC_CUDA(cudaMemsetAsync(b->xbuf + (int64_t)s0 * b->xbuf_stride, 0, count * b->xbuf_stride * sizeof(float), s));
    for (int q = s0; q < s0 + count; ++q) b->last_n[q] = 0;
    return SPIIR_OK;
}

int64_t spiir_tc_xbuf_len(TcBank *b) { return b->xbuf_stride; }

std::vector<int64_t> &spiir_tc_last_n(TcBank *b) { return b->last_n; }

spiir_status spiir_tc_state_get(TcBank *b, int q, double *v, float *xbuf, int64_t *last_n, cudaStream_t s) {
    std::vector<uint4> raw(b->n_slots);
    if (b->n_slots)
        TC_CUDA(cudaMemcpyAsync(raw.data(), b->v + (int64_t)q * b->n_slots, b->n_slots * sizeof(uint4),
                                cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaMemcpyAsync(xbuf, b->xbuf + (int64_t)q * b->xbuf_stride, b->xbuf_stride * sizeof(float),
                            cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    for (int64_t sl = 0; sl < b->n_slots; ++sl) {
        const int64_t k = b->slot_k[sl];
        if (k < 0) continue;
        double re, im;
        if (b->df) {
            float4 f;
            std::memcpy(&f, &raw[sl], sizeof f);
            re = (double)f.x + (double)f.z;
            im = (double)f.y + (double)f.w;
        } else {
            double2 f;
            std::memcpy(&f, &raw[sl], sizeof f);
            re = f.x;
            im = f.y;
        }
        v[2 * k] = re;
        v[2 * k + 1] = im;
    }
    *last_n = b->last_n[q];
    return SPIIR_OK;
}

spiir_status spiir_tc_state_set(TcBank *b, int q, const double *v, const float *xbuf, int64_t last_n,
                                cudaStream_t s) {
    std::vector<uint4> raw(b->n_slots, make_uint4(0u, 0u, 0u, 0u));
    for (int64_t sl = 0; sl < b->n_slots; ++sl) {
        const int64_t k = b->slot_k[sl];
        if (k >= 0) raw[sl] = host_anchor(std::complex<double>(v[2 * k], v[2 * k + 1]), b->df);
    }
    if (b->n_slots)
        TC_CUDA(cudaMemcpyAsync(b->v + (int64_t)q * b->n_slots, raw.data(), b->n_slots * sizeof(uint4),
                                cudaMemcpyHostToDevice, s));
    TC_CUDA(cudaMemcpyAsync(b->xbuf + (int64_t)q * b->xbuf_stride, xbuf, b->xbuf_stride * sizeof(float),
                            cudaMemcpyHostToDevice, s));
    TC_CUDA(cudaStreamSynchronize(s));
    b->last_n[q] = last_n;
    return SPIIR_OK;
}

const float2 *spiir_tc_output(TcBank *b, int stream, int64_t *ring_len) {
    *ring_len = b->ring_len;
    return b->z + (int64_t)stream * b->T * b->ring_len;
}

float *spiir_tc_stage(TcBank *b) { return b->stage; }

unsigned int *spiir_tc_status(TcBank *b) { return b->status; }

void spiir_tc_info(TcBank *b, spiir_bank_info *info) {
    info->n_slots = b->n_slots;
    info->filter_samples_per_block = 0;
    info->n_warp_tasks = 0;
    info->n_cta_items = b->n_groups;
    info->filters_per_lane = 0;
    info->time_tile = b->L;
    info->kernel_variant = b->split ? 3 : b->bf16 ? 2 : 1;
    info->max_delay = b->max_delay;
    info->tc_fir_len = b->F;
    info->graph_captured = 0;
    info->n_units = b->n_tiles;
    info->smem_ways = 1.f;
    info->slot_fill = 1.f;
}

int64_t spiir_tc_footprint(const spiir_bank_desc *d) {
    TcPlan p;
    if (tc_plan(d, p)) return -1;
    return tc_bytes(d, p);
}

void spiir_tc_destroy(TcBank *b) {
    if (!b) return;
    void *ptrs[] = {b->H, b->row_scale, b->tile_ptr, b->tmpl_of, b->has_carry, b->a, b->aJ, b->c,
                    b->aL, b->v, b->xbuf, b->stage, b->z, b->status, b->hank, b->xseg,
                    b->aLf, b->aLb1, b->aLb2, b->panel, b->H_lo, b->hank_lo, b->all_rows};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete b;
}

const char *spiir_tc_last_error() { return g_tc_err.c_str(); }
