// spiir_internal.h -- structures shared by the host side and the kernels of
// libspiir. Not part of the public ABI (include/spiir.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SPIIR_MAX_LEVELS 12
#define SPIIR_MAX_TAPS 64        // interpolator taps
#define SPIIR_MAX_DOWN_TAPS 512  // decimator taps
#define SPIIR_UHIST 32   // history kept per upsampler input row (>= n_taps/2)
#define SPIIR_CTA_WARPS 4

// Device status word values (written by kernels, read by the host).
#define SPIIR_DEV_OK 0u
#define SPIIR_DEV_TIMEOUT 1u

// One warp's work in the FP32 recursion kernel: 32 lanes x F rounds of
// filter slots (slot = slot_base + round*32 + lane). Lanes form groups of
// 2^g_log2 consecutive lanes; each group is one unit (a template's filters at
// one level, or a part of them) whose per-sample sum the group reduces. A unit
// larger than one warp spans 2^xw_log2 consecutive warps of the CTA (then
// g_log2 = 5); its warps add their sums in shared memory and rank 0 writes.
struct WarpTask {
    int32_t slot_base;
    int8_t F;         // rounds, even, <= the kernel variant's FMAX
    int8_t g_log2;    // lane group size = 1 << g_log2 (<= 32)
    int8_t level;
    int8_t xw_log2;   // warps per unit (0 = unit inside this warp)
    int32_t out_base; // task_out[out_base + group] = destination of the group
    int16_t n_groups; // groups that hold a unit (the rest are padding)
    int8_t xw_rank;   // this warp's rank in its multi-warp unit
    int8_t pad;
};

// One CTA's work: up to SPIIR_CTA_WARPS warp tasks of the same level.
struct CtaItem {
    int32_t level;
    int32_t task_begin;
    int32_t task_count;
    int32_t F;        // max F among the tasks (for variant dispatch)
};

// Per-level sizes of one push.
struct LevelArgs {
    int32_t hist;     // strain history samples in front of the block (mult. of 4)
    int32_t n;        // samples of this level in this push
    int32_t seg;      // samples per time segment (multiple of 4)
    int32_t n_prev;   // samples of the previous push at this level
    int64_t part_base;   // float2 offset of this level's partial rows
    int64_t part_stride; // float2 per partial row
    int64_t xbuf_off;    // float offset of this level's strain buffer (per stream)
    int64_t ubuf_off;    // float2 offset of this level's upsampler rows
    int32_t ubuf_stride; // float2 per upsampler history row (SPIIR_UHIST)
    int32_t pad;
};

struct RecurArgs {
    const WarpTask *tasks;
    const CtaItem *items;
    const int32_t *order;      // queue order of the CTA items (heaviest first)
    int32_t n_items;           // CTA items (groups) per stream
    int32_t n_segs;            // time segments per push; queue = n_segs * n_items
    unsigned int *queue;       // [stream] work counter, zeroed by the prologue
    unsigned int *prog;        // [stream][n_items] segments finished this push
    int32_t stall_test;        // 1: queue item 0 neither works nor publishes
                               // its progress (failure-detection test)
    const int32_t *task_out;   // >= 0: direct z row; < 0: partial row -(v+1)
    const float *a_re, *a_im, *b_re, *b_im;
    const int32_t *xoff;       // per slot: hist - delay (window offset)
    float2 *state;             // [stream][n_slots]
    int64_t n_slots;
    float *xbuf;               // [stream][xbuf_stream_stride]
    int64_t xbuf_stream_stride;
    float2 *partial;           // [stream][partial_stream_stride]
    int64_t partial_stream_stride;
    float2 *z;                 // output ring [stream][n_templates][ring_len]
    int64_t z_row_stride;      // ring_len
    int64_t z_stream_stride;
    float scale;
    int32_t stream0;           // first stream of this launch (grid.y adds)
    int32_t n_levels;
    unsigned int *status;
    LevelArgs lev[SPIIR_MAX_LEVELS];
};

struct PrologueArgs {
    unsigned int *queue;        // zeroed for the recursion kernel's work queue
    unsigned int *prog;         // [stream][n_items] zeroed
    int32_t n_items;
    int32_t pad;
    float *xbuf;
    int64_t xbuf_stream_stride;
    const float *x_in;          // [n_streams_in_push][n] device, level 0 samples
    int64_t x_in_stream_stride;
    int32_t stream0;
    int32_t n_levels;
    LevelArgs lev[SPIIR_MAX_LEVELS];
};

struct DecimArgs {
    float *xbuf;
    int64_t xbuf_stream_stride;
    int32_t stream0;
    int32_t n_levels;
    int32_t n_taps;
    float h_down[SPIIR_MAX_DOWN_TAPS];
    LevelArgs lev[SPIIR_MAX_LEVELS];
};

struct CombineArgs {
    const int32_t *comb_ptr;   // [(t * n_levels + i)] CSR into comb_rows
    const int32_t *comb_rows;  // partial rows per (template, level), fixed order
    float2 *partial;
    int64_t partial_stream_stride;
    float2 *ubuf;              // upsampler histories [stream][level][template][SPIIR_UHIST]
    int64_t ubuf_stream_stride;
    float2 *z;
    int64_t z_row_stride;
    int64_t z_stream_stride;
    float scale;
    int32_t n_templates;
    int32_t n_levels;
    int32_t n_taps;
    int32_t stream0;
    unsigned int *status;          // device status word (bounded waits)
    const int32_t *rows;           // NULL: CTA x combines template row x; else
                                   // row rows[x] (n_templates entries)
    float h_up2[SPIIR_MAX_TAPS];   // 2 * h_up (gain 2 of the zero-stuffed series)
    LevelArgs lev[SPIIR_MAX_LEVELS];
};

// Per-kernel CUDA-event timing (tracing), owned by a bank.
struct KernelTimer {
    bool on = false;
    struct Rec {
        int kind;
        int n;                 // kernels launched between the two events
        cudaEvent_t a, b;
    };
    Rec recs[4096];
    int n_recs = 0;
    double ms[8] = {};
    long long launches[8] = {};
    int open_kind = -1;
    cudaEvent_t pool[8192];
    int n_pool = 0;

    cudaEvent_t get() {
        if (n_pool > 0) return pool[--n_pool];
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void begin(int kind, cudaStream_t s) {
        if (!on) return;
        if (n_recs == 4096) flush();
        recs[n_recs].kind = kind;
        recs[n_recs].a = get();
        recs[n_recs].b = get();
        cudaEventRecord(recs[n_recs].a, s);
        open_kind = kind;
    }
    void end(cudaStream_t s, int n_launches = 1) {
        if (!on || open_kind < 0) return;
        recs[n_recs].n = n_launches;
        cudaEventRecord(recs[n_recs].b, s);
        ++n_recs;
        open_kind = -1;
    }
    void flush() {
        for (int i = 0; i < n_recs; ++i) {
            cudaEventSynchronize(recs[i].b);
            float t = 0.f;
            cudaEventElapsedTime(&t, recs[i].a, recs[i].b);
            ms[recs[i].kind] += t;
            launches[recs[i].kind] += recs[i].n;
            if (n_pool < 8190) {
                pool[n_pool++] = recs[i].a;
                pool[n_pool++] = recs[i].b;
            } else {
                cudaEventDestroy(recs[i].a);
                cudaEventDestroy(recs[i].b);
            }
        }
        n_recs = 0;
    }
    void release() {
        flush();
        for (int i = 0; i < n_pool; ++i) cudaEventDestroy(pool[i]);
        n_pool = 0;
    }
};

// Kernel launchers (spiir_plain.cu).
// Kernels spiir_launch_prologue launches (history move, then the new samples).
constexpr int kPrologueLaunches = 2;
cudaError_t spiir_launch_prologue(const PrologueArgs &a, int n_streams, cudaStream_t s);
cudaError_t spiir_launch_decimate(const DecimArgs &a, int n_streams, cudaStream_t s);
cudaError_t spiir_launch_recur(const RecurArgs &a, int variant, int n_ctas,
                               int n_streams, int smem_bytes, cudaStream_t s);
cudaError_t spiir_launch_combine(const CombineArgs &a, int chunk, int n_streams, cudaStream_t s);
// out[t][i] = |z[t][i]| / norm[t] (norm NULL: 1) for T rows of n samples, z rows ring apart.
cudaError_t spiir_launch_abs(const float2 *z, int64_t ring, int T, int64_t n, const float *norm,
                             float *out, cudaStream_t s);
// Base-rate samples per combine time chunk, and the combine CTA's shared memory.
int spiir_combine_chunk(int n_levels, int64_t push_max);
int spiir_combine_smem(int n_levels, int chunk);
cudaError_t spiir_combine_prepare();
int spiir_recur_variant_count();
void spiir_recur_variant_shape(int variant, int *time_tile, int *fmax);
// Sets the dynamic shared memory limit and returns resident CTAs per SM.
cudaError_t spiir_recur_prepare(int variant, int smem_bytes, int *ctas_per_sm);
int spiir_recur_red_bytes();
