// spiir_tc.h -- block-parallel tensor-core form of single-rate SPIIR banks
// (internal interface between spiir_api.cu and spiir_tc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "spiir.h"

struct TcBank;

spiir_status spiir_tc_create(const spiir_bank_desc *desc, float scale, cudaStream_t s,
                             TcBank **out, int64_t *footprint);
struct KernelTimer;
// zoff: first output-ring column the push writes (0 for an ordinary push).
spiir_status spiir_tc_push(TcBank *b, int s0, int count, const float *x, int64_t x_stride,
                           int64_t n, cudaStream_t s, KernelTimer *timer, int64_t zoff = 0);
spiir_status spiir_tc_reset(TcBank *b, int s0, int count, cudaStream_t s);
const float2 *spiir_tc_output(TcBank *b, int stream, int64_t *ring_len);
float *spiir_tc_stage(TcBank *b);
unsigned int *spiir_tc_status(TcBank *b);
void spiir_tc_info(TcBank *b, spiir_bank_info *info);
int64_t spiir_tc_footprint(const spiir_bank_desc *desc);
// Filter state of stream q in filter order (FP64 {re, im} per filter, whatever
// the carry arithmetic), its strain history (xbuf_len floats) and the length
// of its last push. Synchronous on s.
int64_t spiir_tc_xbuf_len(TcBank *b);
// Length of each stream's last push (host state a push reads and updates).
std::vector<int64_t> &spiir_tc_last_n(TcBank *b);
spiir_status spiir_tc_state_get(TcBank *b, int q, double *v, float *xbuf, int64_t *last_n,
                                cudaStream_t s);
spiir_status spiir_tc_state_set(TcBank *b, int q, const double *v, const float *xbuf, int64_t last_n,
                                cudaStream_t s);
void spiir_tc_destroy(TcBank *b);
const char *spiir_tc_last_error();

// ---------------------------------------------------------------------------
// Building blocks shared with the server (spiir_server.cu)
// ---------------------------------------------------------------------------

// Sizes of the block-parallel form.
constexpr int kTcGroup = 64;          // templates per impulse-response group (FIR rows / 2)
constexpr int kTcTile = 128;          // filter slots per carry tile
constexpr int kTcSliceBytes = 16384;  // one K slice of a group's impulse responses
constexpr int kTcPanelBytes = 32768;  // one tile's power panel
int spiir_tc_hank_bytes(int L, int K);            // Toeplitz source of one chunk
int spiir_tc_xseg_bytes();                        // STATE strain segments of one batch
int spiir_tc_cpb(int streams, int L);             // chunks per carry batch

// Host-side packing of a set of single-rate filters (all of a bank, or one
// level of a multi-rate bank) for a FIR length F and chunk length L: the
// impulse-response groups, per-template row scales, the carry tiles and their
// precomputed power panels, in the layouts the kernels read. Template t of
// the set is FIR row 2 (t % 64) (+1) of group t / 64; its tiles are
// tile_ptr[t] .. tile_ptr[t + 1] - 1.
struct TcPack {
    int T = 0, F = 0, L = 0, K = 0, n_groups = 0, n_slices = 0, n_tiles = 0;
    std::vector<uint16_t> H;          // [group][slice][kTcSliceBytes / 2]
    std::vector<uint16_t> H_lo;       // split bf16 only: h - bf16(h), same layout
    std::vector<float> row_scale;     // [T]: row_mult * 2^-e_t
    std::vector<int32_t> tile_ptr;    // [T + 1]
    std::vector<uint8_t> has_carry;   // [T]
    std::vector<float2> a, aJ, c, aLf;      // [tile * 128 + lane]
    std::vector<uint4> aL, aLb1, aLb2;      // [tile * 128 + lane]: FP64 or double-float
    std::vector<int64_t> slot_k;            // filter of each slot (-1: padding)
    std::vector<uint16_t> panel;      // [tile][kTcPanelBytes / 2]
};
// level < 0: every filter (single rate); else the filters with level[k] ==
// level. Delays must be < F. row_mult scales every output row (the SNR scale,
// or 1 for a level sum that a later pass scales). split (with bf16): also the
// low bf16 part of every impulse-response value, H_lo.
spiir_status spiir_tc_pack(const spiir_bank_desc *d, int level, int F, int L, double row_mult, bool bf16,
                           bool df, TcPack &pk, bool split = false);

// One batched launch sequence of the block-parallel form for up to two
// streams: strain staging, the carry kernel (state term into z) and the FIR
// kernel (adds the FIR term), over the groups and carry templates listed.
struct TcLaunch {
    // strain: xbuf + (stream0 + s) * xbuf_stride + hist is the push's first
    // sample; hist >= F
    const float *xbuf;
    int64_t xbuf_stride;
    int hist, F, L, K, n_chunks, n_streams, stream0;
    uint4 *hank, *xseg;                // staging buffers
    // carry
    const int32_t *tile_ptr, *tile_end, *tmpl_of;
    int n_carry;                       // templates listed in tmpl_of
    const float2 *a, *aJ, *aLf, *c;
    const uint4 *aL, *aLb1, *aLb2, *panel;
    uint4 *v;                          // [stream][n_slots]
    int64_t n_slots;
    float carry_scale;
    // FIR
    const uint4 *H;
    const float *row_scale;
    const uint8_t *has_carry;
    // split bf16 (H_lo non-NULL): the FIR runs three accumulating passes,
    // H x + H x_lo + H_lo x, over the low parts H_lo and hank_lo (staged
    // here); all_rows: n_rows ones, so that the later passes add to z
    const uint4 *H_lo;
    uint4 *hank_lo;
    const uint8_t *all_rows;
    const int32_t *groups;             // NULL: groups 0 .. n_groups-1
    int n_groups, n_rows;              // groups to run; rows addressable in z
    // output rows (row t of stream s at z + s * z_stream_stride + t * z_row_stride)
    float2 *z;
    int64_t z_row_stride, z_stream_stride;
    bool bf16, df;                     // operand type; double-float anchor
    int carry_mode;                    // 0 FP64 anchor per batch, 1 double-float, 2 FP64 per chunk
    unsigned int *status;
    int n_sms;
};
spiir_status spiir_tc_launch(const TcLaunch &l, cudaStream_t s, KernelTimer *timer);
// Sets the kernels' shared-memory limits (once per process and device).
spiir_status spiir_tc_prepare(int L, int K);
