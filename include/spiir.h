/*
 * spiir.h -- C ABI of libspiir, a GB300 (sm_103a) implementation of Summed
 * Parallel IIR (SPIIR) filtering and its multi-rate scheme (arXiv:1702.02256).
 *
 * What is computed (Sec. 2.1, Eqs. iireq0 and iireq1): every template t is a
 * bank of complex first-order filters k with pole a_k, gain b_k and integer
 * delay d_k driven by the real strain x,
 *
 *     y_k[n] = a_k * y_k[n-1] + b_k * x[n - d_k],
 *     z_t[n] = snr_scale * sum_{k in t} y_k[n],      snr_scale = 2*dt,
 *
 * and, when n_levels > 1, the multi-rate scheme of Sec. 2.2 (Fig. 1): the
 * strain is decimated by 2 in succession (Kaiser-window low-pass, Eq.
 * kaiser_window_filtering), a filter at level i runs at base_rate/2^i on the
 * level-i strain, and from the lowest rate up each rate's sum is upsampled by
 * 2 and added to the next rate's sum; level i's own sum is delayed by
 * D_i = (Td-1)/2 + (Tu-1)/2 + 2*D_{i+1} (D_H = 0; Td, Tu the decimator and
 * interpolator lengths, whose linear-phase round trip this is) so that the
 * levels line up.
 *
 * Conventions shared by every call:
 *   - Complex arrays on the device are complex64: interleaved (re, im) float32.
 *   - "Device pointer" means memory the caller allocated on the current CUDA
 *     device (e.g. a torch tensor). The caller owns it; it must stay valid
 *     until the work queued on `cuda_stream` has reached it.
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Calls do not throw. Each returns a spiir_status; spiir_last_error()
 *     then holds a one-line message for the calling thread.
 *   - A bank is used by one host thread at a time.
 *   - Filter state, strain history and resampler history live on the device
 *     in the bank between calls: a long series can be pushed in pieces and
 *     gives the same SNR as one push of the whole series.
 */
#ifndef SPIIR_H
#define SPIIR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spiir_bank *spiir_bank_t;

typedef enum {
    SPIIR_OK = 0,
    SPIIR_EINVAL = 1,      /* bad argument: null pointer, size, ordering, range */
    SPIIR_ENOMEM = 2,      /* a device or host allocation failed */
    SPIIR_EBUDGET = 3,     /* footprint above desc->hbm_budget_bytes */
    SPIIR_ECUDA = 4,       /* a CUDA runtime call failed (message has its name) */
    SPIIR_ETIMEOUT = 5,    /* a bounded device-side wait gave up; results of
                              that push are not valid, the bank stays usable */
    SPIIR_ESTATE = 6,      /* call out of order (read before any push, ...) */
    SPIIR_EUNSUPPORTED = 7 /* valid request this library does not provide */
} spiir_status;

/* Compute form. PLAIN_FP32 is the per-sample FP32 recursion (all n_levels).
 * The TC_* forms are the block-parallel tensor-core form for single-rate
 * banks: over chunks of chunk_len samples the bank is a dense contraction of
 * the template impulse responses with a Toeplitz view of x, plus per-filter
 * power panels a_k^j applied to filter states carried between chunks in FP64
 * (or double-float, desc->carry).
 * TC_FP16 / TC_BF16 round the panel and strain operands to that type (FP32
 * accumulation). TC_BF16X2 splits both operands of the FIR contraction (the
 * template impulse responses and the strain) into a bf16 high part and a
 * bf16 low part (the rounding residual) and runs it as three accumulating
 * passes, hi*hi + hi*lo + lo*hi: about three times the FIR's tensor work, for
 * an error near that of 16-bit significands. Its carry contractions (states
 * of inputs older than the FIR window) stay single-pass bf16; their share of
 * the SNR is small when the filters decay within a few FIR lengths (for
 * time constants log-uniform in 10-2000 samples and F = 1024, about 9% of
 * the RMS), so their rounding adds roughly that share of the single-pass
 * bf16 error. Banks only (the server takes PLAIN_FP32, TC_FP16, TC_BF16).
 * The tensor-core modes take single-rate banks (n_levels = 1; a multi-rate
 * bank is EUNSUPPORTED). Multi-rate banks run the block form at the rates
 * whose block holds whole chunks through the server (spiir_server_*), where
 * a member added before the first push has the SNR of a bank of its own. */
typedef enum {
    SPIIR_PLAIN_FP32 = 0,
    SPIIR_TC_FP16 = 1,
    SPIIR_TC_BF16 = 2,
    SPIIR_TC_BF16X2 = 3
} spiir_mode;

/* Bank description. All arrays are host memory owned by the caller and are
 * copied during spiir_bank_create; they may be freed when it returns. */
typedef struct {
    int32_t n_templates;    /* >= 1 */
    int32_t n_levels;       /* 1 = single rate; up to 12 */
    int32_t base_rate;      /* Hz of level 0 (the input rate), e.g. 4096 */
    int32_t n_streams;      /* independent detector streams, >= 1 */
    int32_t block_len;      /* samples per push unit at the base rate; a
                               multiple of 2^(n_levels-1) */
    int32_t max_push_blocks;/* largest push, in blocks (output ring size) */
    int64_t n_filters;      /* >= 0; templates may have zero filters */
    const float *a_re, *a_im;     /* pole a_k, at the filter's own rate */
    const float *b_re, *b_im;     /* gain b_k */
    const int32_t *delay;         /* d_k >= 0, samples at the filter's rate */
    const int32_t *template_id;   /* in [0, n_templates) */
    const int8_t *level;          /* in [0, n_levels); NULL = all level 0.
                                     There is no "assign at create" value
                                     (-1 is EINVAL): running a designed
                                     filter at a lower rate changes its
                                     pole, gain and delay, which is filter
                                     design; spiir_assign_level gives the
                                     Sec. 2.2 rule to callers that convert
                                     their filters themselves */
    const float *h_down, *h_up;   /* decimator taps (n_taps of them) and
                                     interpolator taps (n_taps_up); NULL =
                                     built-in 60 dB Kaiser low-passes */
    int32_t n_taps;               /* decimator length: even, 2..512; 0 = 32 */
    int32_t align;                /* 1 = delay level sums by D_i (default
                                     when n_levels > 1), 0 = no delay */
    float snr_scale;              /* 0 = 2/base_rate (2*dt, Eq. iireq1) */
    spiir_mode mode;
    int32_t chunk_len;            /* TC forms: chunk length L (0 = 256) */
    int32_t tune;                 /* 0 = built-in tile choice (plain: 4
                                     filters per lane when the non-empty
                                     (template, level) units hold at most
                                     128 filters on average, else 8; 32-
                                     sample time tiles); 1 = autotune
                                     at create: time candidate tilings on
                                     pushes of zeros and keep the fastest
                                     (plain: every compiled recursion
                                     variant, then the time-segment length
                                     and resident CTAs per SM; TC: the
                                     chunk length 128 or 256, overriding
                                     chunk_len); -(v+1) = recursion variant v */
    int64_t hbm_budget_bytes;     /* 0 = no limit; else create fails with
                                     SPIIR_EBUDGET above it */
    int32_t n_taps_up;            /* interpolator length: even, 2..64; 0 =
                                     n_taps (Sec. 2.2 pairs a long 100 dB
                                     decimator with a 32-tap interpolator) */
    int32_t carry;                /* TC forms: arithmetic of the filter state
                                     carried from chunk to chunk: 0 = FP64
                                     at every batch of chunks, FP32 offsets
                                     from it inside a batch (default); 1 =
                                     the same with double-float pairs on the
                                     FP32 pipe (about 48 significant bits;
                                     faster on parts with a low FP64 rate);
                                     2 = FP64 at every chunk (slowest).
                                     Ignored by PLAIN_FP32; other values:
                                     EINVAL */
} spiir_bank_desc;

/* Read-only facts about a created bank. */
typedef struct {
    int64_t footprint_bytes;   /* device bytes the bank holds */
    int64_t n_slots;           /* filter slots after packing (>= n_filters) */
    int64_t filter_samples_per_block; /* sum over filters of own-rate samples
                                         in one block, per stream */
    int32_t n_warp_tasks;
    int32_t n_cta_items;
    int32_t filters_per_lane;  /* largest F chosen by the packer */
    int32_t time_tile;         /* T of the recursion kernel */
    int32_t kernel_variant;    /* index of the compiled recursion variant */
    int32_t max_delay;         /* largest d_k (+ alignment) over levels */
    int32_t tc_fir_len;        /* TC forms: F (> max delay), else 0 */
    int32_t graph_captured;    /* 1 if pushes replay a CUDA graph */
    int32_t n_units;           /* (template, level, part) units */
    float smem_ways;           /* mean shared-memory wavefronts per round of
                                  32 delayed-input reads (1 = no conflicts) */
    float slot_fill;           /* n_filters / n_slots */
    int32_t segment_base;      /* plain form: base-rate samples per time
                                  segment of the recursion's work queue */
    int32_t ctas_per_sm;       /* plain form: resident recursion CTAs per SM */
    float tune_ms;             /* wall time the autotuner took (0: not run) */
} spiir_bank_info;

/* Create a bank: validate the description, place filters into warp tasks
 * (template-major per level, lane groups sized to the template's filter
 * count), upload coefficients, allocate device state, history and output
 * ring, and zero the state (Sec. 2.1: the recursion starts from y = 0 with
 * x[n < 0] = 0). Work is queued on cuda_stream and synchronised before return.
 * Errors: EINVAL (description), EBUDGET, ENOMEM, ECUDA, EUNSUPPORTED. */
spiir_status spiir_bank_create(const spiir_bank_desc *desc, void *cuda_stream,
                               spiir_bank_t *out);

/* Filter n_samples more samples of one stream (stream_id in [0, n_streams))
 * or of all streams (stream_id = -1; x_dev is then [n_streams][n_samples]).
 * x_dev: device float32, contiguous. n_samples: a positive multiple of
 * block_len, at most block_len * max_push_blocks. Asynchronous on
 * cuda_stream; the SNR of these samples replaces the bank's output ring for
 * the pushed stream(s). Errors: EINVAL; ETIMEOUT/ECUDA from an earlier push. */
spiir_status spiir_push_block(spiir_bank_t bank, int32_t stream_id,
                              const float *x_dev, int64_t n_samples,
                              void *cuda_stream);

/* Copy the SNR of the most recent push of stream_id (or of every stream for
 * -1) into z_dev: complex64 [n_templates][n_samples] per stream, streams
 * outermost, the last n_samples samples of that push, z = snr_scale * sum.
 * Asynchronous device-to-device copy on cuda_stream.
 * Errors: EINVAL, ESTATE (nothing pushed on that stream since create, reset
 * or state import). */
spiir_status spiir_read_snr(spiir_bank_t bank, int32_t stream_id, void *z_dev,
                            int64_t n_samples, void *cuda_stream);

/* Zero the filter state, strain history and resampler history of one stream
 * (or all, -1): the next push behaves like the first push of a new bank. */
spiir_status spiir_state_reset(spiir_bank_t bank, int32_t stream_id,
                               void *cuda_stream);

/* The SNR of Sec. 2.1 as the modulus of z over a per-template normalisation
 * constant: out_dev[stream][template][i] = |z| / norm_dev[template] for the
 * last n_samples samples of the most recent push of stream_id (or every
 * stream, -1), float32, streams outermost. norm_dev: device float
 * [n_templates] (the caller's constants, > 0), or NULL for |z|. Asynchronous
 * on cuda_stream. Errors: EINVAL, ESTATE (no push since create, reset or
 * state import). */
spiir_status spiir_read_snr_abs(spiir_bank_t bank, int32_t stream_id, float *out_dev,
                                int64_t n_samples, const float *norm_dev, void *cuda_stream);

/* Checkpoint and resume. A state blob holds, per stream, everything a push
 * depends on: the filter states (in filter order, so it does not depend on
 * the kernel variant), the strain and resampler histories and the length of
 * the last push. spiir_state_bytes: size of the blob of one stream (or all,
 * -1), -1 on a bad argument. spiir_state_export writes it to host memory dst
 * (at least that many bytes; the call waits for the copies). spiir_state_import
 * reads a blob of the same number of streams into stream_id (or all, -1) of a
 * bank created from the same description (same filters, rates, resampler,
 * block length, maximum push and form; the tensor-core carry arithmetic may
 * differ: its state is stored in FP64); later pushes then continue the
 * stream as if it had never stopped. The output ring is not part of the
 * state: read the SNR after the next push. Errors: EINVAL (NULL pointer,
 * short buffer, blob of another description or form, stream count).
 * The caller owns dst/src. */
int64_t spiir_state_bytes(spiir_bank_t bank, int32_t stream_id);
spiir_status spiir_state_export(spiir_bank_t bank, int32_t stream_id, void *dst, int64_t bytes,
                                void *cuda_stream);
spiir_status spiir_state_import(spiir_bank_t bank, int32_t stream_id, const void *src,
                                int64_t bytes, void *cuda_stream);

/* End-to-end call on host buffers: copy x_host [n_streams or 1][n_samples]
 * to the device, push, and copy the SNR back into z_host (layout of
 * spiir_read_snr). Pinned host memory makes the copies asynchronous; the
 * call returns after the SNR is in z_host. */
spiir_status spiir_push_block_host(spiir_bank_t bank, int32_t stream_id,
                                   const float *x_host, int64_t n_samples,
                                   void *z_host, void *cuda_stream);

/* The same push, returning once its copies and kernels are queued: the SNR
 * is in z_host, and x_host may be reused, only after spiir_bank_host_sync
 * returns. Arguments and errors as for spiir_push_block_host; x_host and
 * z_host must stay valid until then, and must be pinned for the copies to
 * overlap anything. When the output ring holds two pushes of n_samples
 * (block_len * max_push_blocks >= 2 * n_samples), consecutive asynchronous
 * pushes write alternate halves of it, so a push's kernels run while the SNR
 * of the push before it is still being copied out; otherwise each waits,
 * on the device, for that copy. Every call that writes the ring (pushes,
 * host pushes) waits on the device for the copies still reading it, so the
 * calls may be mixed. spiir_read_snr and spiir_read_snr_abs read the last
 * push wherever it sits in the ring. The SNR of the pushes of the tensor-core
 * and plain forms is the same as from spiir_push_block_host, bit for bit. */
spiir_status spiir_push_block_host_async(spiir_bank_t bank, int32_t stream_id,
                                         const float *x_host, int64_t n_samples,
                                         void *z_host, void *cuda_stream);

/* Waits (on the host) until every asynchronous host push of the bank has its
 * SNR in host memory. EINVAL for a NULL bank, ECUDA if a copy failed. */
spiir_status spiir_bank_host_sync(spiir_bank_t bank);

/* Device bytes a bank with this description would hold (filters, state,
 * history, scratch, output ring), for admission control. -1 on a bad desc. */
int64_t spiir_bank_footprint(const spiir_bank_desc *desc);

/* Facts about a created bank. */
spiir_status spiir_bank_get_info(spiir_bank_t bank, spiir_bank_info *info);

/* The packing a description would get, computed on the host only (no device
 * work, no CUDA call): the fields of spiir_bank_get_info for the variant that
 * desc->tune selects (the built-in choice when tune >= 0). */
spiir_status spiir_bank_plan(const spiir_bank_desc *desc, spiir_bank_info *info);

/* Wait for the bank's queued work and report the device status word: OK, or
 * ETIMEOUT if a bounded device wait gave up since the last call (the word is
 * then cleared). */
spiir_status spiir_bank_sync_status(spiir_bank_t bank);

/* Kernel kinds for per-kernel timing. */
typedef enum {
    SPIIR_K_PROLOGUE = 0, /* strain history shift + new samples */
    SPIIR_K_DECIMATE = 1, /* x2 decimation cascade */
    SPIIR_K_RECUR = 2,    /* FP32 recursion + per-template sum */
    SPIIR_K_COMBINE = 3,  /* parts + x2 upsample + upstream sum + scale */
    SPIIR_K_TC_STAGE = 4, /* TC form: strain operand staging */
    SPIIR_K_TC_FIR = 5,   /* TC form: impulse-response x Toeplitz(x) GEMM */
    SPIIR_K_TC_CARRY = 6, /* TC form: power panels, FP64 carry, state GEMMs */
    SPIIR_K_OTHER = 7,
    SPIIR_K_COUNT = 8
} spiir_kernel_kind;

typedef struct {
    double ms[SPIIR_K_COUNT];        /* summed device time per kind */
    int64_t launches[SPIIR_K_COUNT]; /* launches per kind */
} spiir_kernel_times;

/* Tracing: while enabled, every push records a CUDA event pair on its own
 * stream around each kernel it launches. */
spiir_status spiir_bank_enable_timing(spiir_bank_t bank, int32_t enable);

/* Wait for the recorded events, return the per-kind sums since the previous
 * call (or since timing was enabled), and start a new count. */
spiir_status spiir_bank_kernel_times(spiir_bank_t bank, spiir_kernel_times *out);

/* Failure-detection test (plain form): one push of the first stream in which
 * the first work item of the recursion kernel neither runs nor publishes its
 * progress, so the item that depends on it waits until the bounded device
 * wait (about 2 s) gives up and records SPIIR_ETIMEOUT in the status word.
 * No fault, trap or hang: the kernel finishes, the SNR of that push is not
 * valid, the next spiir_bank_sync_status returns SPIIR_ETIMEOUT and clears
 * it, and the bank keeps working. n_samples >= 8192 (two time segments). */
spiir_status spiir_bank_test_stall(spiir_bank_t bank, const float *x_dev, int64_t n_samples,
                                   void *cuda_stream);

/* Release everything the bank holds. NULL is ignored. */
void spiir_bank_destroy(spiir_bank_t bank);

/* The library's own resampling taps (Sec. 2.2): n_taps-tap Kaiser-window
 * low-pass with cutoff at half the input Nyquist frequency, window parameter
 * from Kaiser's formula for atten_db, unit DC gain, float32. */
spiir_status spiir_kaiser_taps(int32_t n_taps, double atten_db, float *out);

/* The rate-assignment rule of Sec. 2.2 on a base-rate pole a: the level
 * whose rate base_rate/2^i is the smallest that is >= twice the filter's band
 * edge |arg a| * base_rate / (2 pi). Returns -1 for n_levels outside [1, 30]
 * or base_rate <= 0. */
int32_t spiir_assign_level(float a_re, float a_im, int32_t base_rate,
                           int32_t n_levels);

/* The same rule with a passband margin: the smallest available rate that is
 * >= 2 f (1 + margin), keeping the band edge clear of the resamplers'
 * transition band (margin = 0 is spiir_assign_level). Returns -1 for
 * margin < 0 or not finite, n_levels outside [1, 30] or base_rate <= 0. */
int32_t spiir_assign_level_margin(float a_re, float a_im, int32_t base_rate,
                                  int32_t n_levels, float margin);

/* One-shot filtering that allocates no device memory. The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc, such as a
 * host framework whose real-time thread must not allocate device memory (an
 * allocation can block on the driver for an unbounded time), or a process
 * whose device memory is divided up in advance, so that an allocation outside
 * its own pools fails.
 *
 * Filters x_dev (device float32 [n_samples], one stream) with the bank that
 * desc describes (plain FP32 form, n_streams = 1), starting from zero filter
 * state and zero strain history, and writes z_dev (device complex64
 * [n_templates][n_samples], the layout of spiir_read_snr) -- the SNR that
 * spiir_bank_create + spiir_push_block + spiir_read_snr would give for the
 * same description and samples. n_samples: a positive multiple of
 * 4 * 2^(n_levels-1). desc->block_len, max_push_blocks and tune >= 0 are
 * ignored (one push of n_samples, built-in tile choice; tune < 0 still
 * forces a variant). The caller owns x_dev and z_dev.
 *
 * All device memory it uses is one fixed 32 MiB __device__ array that every
 * GPU loading the library reserves until the process exits. A bank and length
 * whose packed coefficients, state and buffers need more fail with EINVAL and a
 * message giving both sizes. Every call shares that array and leaves its
 * contents behind (it clears what must start at zero), so calls whose work
 * overlaps on the GPU -- on two streams, or from two host threads -- race and
 * must be serialised by the caller. A bounded device-side wait that gives up
 * (possible only when such calls overlap) leaves a wrong z and is not
 * reported by this call. The first call on a device, with that device
 * current, looks up the array's device address (first calls from several
 * host threads are safe); make that first call before any stream capture.
 * The coefficients are packed in ordinary host memory and copied in on
 * cuda_stream. */
spiir_status spiir_filter_noalloc(const spiir_bank_desc *desc, const float *x_dev,
                                  int64_t n_samples, void *z_dev, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Serving: many banks filtered together.
 *
 * A server holds the strain of n_streams detector streams and any number of
 * member banks (template-bank requests of a serving loop). Every push filters
 * one block of every stream through all members at once: one shared history
 * update and decimation cascade of the strain (Sec. 2.2), one recursion
 * launch over the work items of every member and level (Eqs. iireq0,
 * iireq1), one upsample-and-add launch over every member's templates; the
 * tensor-core modes run the levels whose block holds whole chunks in the
 * block-parallel form, batched over all members (for each template with
 * enough filters at the level, tc_min_filters), and the rest in the plain
 * form. Members join and leave between pushes; their filter states and
 * resampler histories stay on the device between pushes, in pooled arrays
 * that grow as needed and are reused after a member leaves.
 *
 * A member added before push k takes part from push k on: its filter states
 * and upsampler histories start at zero there, while its delayed inputs
 * x[n - d_k] read the server's continuous strain history (for a member
 * added before the first push that is the zero history of a new bank, and
 * its SNR equals that of a bank of its own). In the levels run in the block
 * form the first chunk's FIR window reaches F samples back (F = max_delay + 1
 * rounded up to 64), so there a late member's filters start F - d_k samples
 * before its first sample: the start-up transients of the two forms differ
 * by a term that decays with each filter's time constant. Each member's SNR
 * is the same whatever other members share the server (fixed summation
 * order).
 * ------------------------------------------------------------------------ */
typedef struct spiir_server *spiir_server_t;

typedef struct {
    int32_t n_streams;     /* detector streams pushed together, >= 1 */
    int32_t n_levels;      /* rates of every member, 1..12 */
    int32_t base_rate;     /* Hz of level 0 */
    int32_t block_len;     /* base-rate samples per push and stream; a
                              multiple of 4 * 2^(n_levels-1) */
    int32_t max_delay;     /* largest delay d_k (own-rate samples) any member
                              may have; sets the strain history kept */
    const float *h_down, *h_up;   /* resampler taps as in spiir_bank_desc */
    int32_t n_taps, n_taps_up;
    int32_t align;         /* as in spiir_bank_desc (1 when n_levels > 1) */
    float snr_scale;       /* 0 = 2/base_rate */
    spiir_mode mode;       /* PLAIN_FP32, TC_FP16 or TC_BF16 */
    int32_t chunk_len;     /* TC modes: chunk length (0 = 256) */
    int32_t carry;         /* TC modes: as in spiir_bank_desc */
    int32_t tune;          /* recursion variant: -(v+1) forces v, else built-in */
    int32_t tc_min_filters;/* TC modes: a template runs a block-form level in
                              the block form when it has at least this many
                              filters there, else in the plain form (the
                              block form's cost per template-sample does not
                              shrink with the filter count); 0 = 24, 1 =
                              every template with filters */
} spiir_server_desc;

/* Facts about a server. */
typedef struct {
    int32_t n_members;         /* members taking part in pushes */
    int32_t n_templates;       /* their templates */
    int64_t n_filters;         /* their filters */
    int64_t filter_samples_per_push;  /* sum over filters of own-rate samples
                                         in one push of one stream */
    int64_t device_bytes;      /* device memory the server holds (pools) */
    int32_t n_cta_items;       /* recursion work items per stream */
    int32_t kernel_variant;    /* recursion variant */
    int32_t tc_levels;         /* levels run in the block-parallel form */
    int32_t launches_per_push; /* kernels one push launches */
} spiir_server_info;

/* Create an empty server. Errors: EINVAL, ENOMEM, ECUDA, EUNSUPPORTED. */
spiir_status spiir_server_create(const spiir_server_desc *desc, void *cuda_stream,
                                 spiir_server_t *out);

/* Add a member. Of *member only the filters (a, b, delay, template_id,
 * level), n_templates, n_filters, n_levels (must equal the server's) and
 * base_rate (must equal the server's) are used; streams, block length,
 * resampler, scale and form are the server's. The arrays are copied before
 * return. *member_id receives the member's handle (>= 0). The member takes
 * part from the next push. Errors: EINVAL (description, a delay above
 * max_delay), ENOMEM. */
spiir_status spiir_server_add(spiir_server_t srv, const spiir_bank_desc *member,
                              int32_t *member_id);

/* Remove a member: it takes no part in later pushes and its memory is
 * reused. Errors: EINVAL (unknown id). */
spiir_status spiir_server_remove(spiir_server_t srv, int32_t member_id);

/* Device bytes a member would add to the server's pools (for admission
 * control; pools grow geometrically, so the server may hold up to about
 * half as much again). -1 on a bad description. */
int64_t spiir_server_member_footprint(spiir_server_t srv, const spiir_bank_desc *member);

/* Apply the pending additions and removals now, so that the next push only
 * filters: place the new members in the pools and upload their coefficients
 * (on a stream of the server's, after the work of earlier pushes), rebuild
 * the work lists and capture the next push's launches. Work is queued on
 * cuda_stream, which the next push must follow (pass the same stream). A
 * serving loop calls it between blocks, while it waits for the next block.
 * Optional: a push applies pending changes itself. Errors: ENOMEM, ECUDA. */
spiir_status spiir_server_prepare(spiir_server_t srv, void *cuda_stream);

/* Filter one block of every stream: x_dev device float32
 * [n_streams][block_len]. Applies pending additions and removals first. A
 * push without members still takes the block into the strain history, so
 * that members joining later read the continuous stream. Asynchronous on
 * cuda_stream. Errors: ECUDA, ENOMEM; ETIMEOUT from an earlier push shows in
 * spiir_server_sync_status. */
spiir_status spiir_server_push(spiir_server_t srv, const float *x_dev, void *cuda_stream);

/* The SNR of the last push for one member: z_dev device complex64
 * [n_streams][n_templates of the member][block_len]. Asynchronous device
 * copy on cuda_stream. Errors: EINVAL (unknown id), ESTATE (the member has
 * not taken part in a push yet). */
spiir_status spiir_server_read(spiir_server_t srv, int32_t member_id, void *z_dev,
                               void *cuda_stream);

spiir_status spiir_server_get_info(spiir_server_t srv, spiir_server_info *info);

/* Wait for the server's queued work and report its device status word (OK,
 * or ETIMEOUT once after a bounded device wait gave up). */
spiir_status spiir_server_sync_status(spiir_server_t srv);

/* Tracing, as for banks: while enabled, pushes launch their kernels one by
 * one (no graph) with a CUDA event pair around each; spiir_server_kernel_times
 * waits for them and returns the per-kind sums since the previous call. */
spiir_status spiir_server_enable_timing(spiir_server_t srv, int32_t enable);
spiir_status spiir_server_kernel_times(spiir_server_t srv, spiir_kernel_times *out);

/* Release everything the server holds. NULL is ignored. */
void spiir_server_destroy(spiir_server_t srv);

/* ------------------------------------------------------------------------
 * Replicas: one bank split by templates over several devices.
 *
 * Templates are independent (Eqs. iireq0, iireq1), so the bank of desc is
 * cut into contiguous template ranges of about equal filter-samples, one
 * ordinary bank per listed device (a device may be listed more than once),
 * with no exchange between devices. Each push copies the host strain to every
 * device, the devices filter at the same time (one host thread each), and the
 * SNR rows are gathered into one host array in template order.
 * ------------------------------------------------------------------------ */
typedef struct spiir_replicas *spiir_replicas_t;

/* Create the replicas. devices: n_devices device ordinals (1 <= n_devices <=
 * n_templates). desc as for spiir_bank_create (its arrays are copied).
 * Errors: EINVAL (description, a device not present), ENOMEM, ECUDA, and any
 * error of spiir_bank_create on a device. */
spiir_status spiir_replicas_create(const spiir_bank_desc *desc, const int32_t *devices,
                                   int32_t n_devices, spiir_replicas_t *out);

/* Push n_samples of every stream from host memory x_host [n_streams][n_samples]
 * (n_samples as for spiir_push_block) through every replica and write the SNR
 * to host memory z_host: complex64 [n_streams][n_templates][n_samples], the
 * layout of spiir_read_snr for the whole bank. Returns when z_host is written.
 * The caller owns both buffers. Errors: EINVAL, and those of
 * spiir_push_block_host on a device. */
spiir_status spiir_replicas_push_host(spiir_replicas_t rp, const float *x_host, int64_t n_samples,
                                      void *z_host);

/* Replica i's device and template range [template0, template0 + n_templates). */
spiir_status spiir_replicas_get(spiir_replicas_t rp, int32_t i, int32_t *device,
                                int32_t *template0, int32_t *n_templates);

/* Release every replica. NULL is ignored. */
void spiir_replicas_destroy(spiir_replicas_t rp);

/* Message of the last failed call on this thread ("" if none). */
const char *spiir_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPIIR_H */
