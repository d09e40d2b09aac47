// spiir_plan.h -- host-side planner of libspiir shared by the bank
// (spiir_api.cu) and the server (spiir_server.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "spiir.h"
#include "spiir_internal.h"

namespace spiir_host {

// Message of the calling thread's last failure (spiir_last_error).
extern thread_local std::string g_err;
spiir_status fail(spiir_status st, const char *fmt, ...);

#define CUDA_TRY(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return spiir_host::fail(e_ == cudaErrorMemoryAllocation ? SPIIR_ENOMEM       \
                                                                    : SPIIR_ECUDA,       \
                                    "%s: %s", #call, cudaGetErrorString(e_));            \
    } while (0)

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Sizes and packed arrays of one bank for one recursion-kernel variant.
struct Plan {
    int variant = 0, T = 32, FMAX = 8;
    int seg_base = 4096;          // base-rate samples per time segment (tunable)
    int n_levels = 1, H = 0, n_taps = 32, n_taps_up = 32, align = 0;   // decimator, interpolator
    int hist[SPIIR_MAX_LEVELS] = {};
    int seg[SPIIR_MAX_LEVELS] = {};
    int64_t max_n[SPIIR_MAX_LEVELS] = {};
    int64_t xbuf_off[SPIIR_MAX_LEVELS] = {};
    int64_t part_rows[SPIIR_MAX_LEVELS] = {};
    int64_t part_base[SPIIR_MAX_LEVELS] = {};
    int64_t part_stride[SPIIR_MAX_LEVELS] = {};
    int64_t ubuf_off[SPIIR_MAX_LEVELS] = {};
    int32_t ubuf_stride[SPIIR_MAX_LEVELS] = {};
    int64_t xbuf_stream_stride = 0, part_stream_stride = 0, ubuf_stream_stride = 0;
    int64_t ring_len = 0;
    int smem_bytes = 0;
    bool need_combine = false;
    int max_F = 0, max_delay = 0;
    int64_t n_slots = 0;
    int64_t fs_per_block = 0;
    // packed arrays
    std::vector<float> are, aim, bre, bim;
    std::vector<int32_t> xoff;
    std::vector<WarpTask> tasks;
    std::vector<CtaItem> items;
    std::vector<int32_t> task_out;
    std::vector<int32_t> comb_ptr, comb_rows;
    std::vector<int32_t> order;
    std::vector<int64_t> slot_filter;   // filter of each slot (-1: padding)
    int64_t lds_rounds = 0, lds_wavefronts = 0;
    int64_t n_units = 0;
};


spiir_status validate(const spiir_bank_desc *d);
int chosen_variant(const spiir_bank_desc *d);
spiir_status make_plan(const spiir_bank_desc *d, int variant, bool arrays, Plan &p,
                       const int *hist_fixed = nullptr, int seg_base = 4096);
int64_t plan_footprint(const spiir_bank_desc *d, const Plan &p);
int64_t align_delay(int level, int n_levels, int n_taps, int n_taps_up, int align);
int push_segments_n(int64_t n, int seg_base = 4096);
int64_t segment_len(int64_t n, int i, int S);
void lib_kaiser_taps(int n, double A, float *out);

}  // namespace spiir_host
