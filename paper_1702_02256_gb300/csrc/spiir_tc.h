// spiir_tc.h -- block-parallel tensor-core form of single-rate SPIIR banks
// (internal interface between spiir_api.cu and spiir_tc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
spiir_status spiir_tc_state_get(TcBank *b, int q, double *v, float *xbuf, int64_t *last_n,
                                cudaStream_t s);
spiir_status spiir_tc_state_set(TcBank *b, int q, const double *v, const float *xbuf, int64_t last_n,
                                cudaStream_t s);
void spiir_tc_destroy(TcBank *b);
const char *spiir_tc_last_error();
