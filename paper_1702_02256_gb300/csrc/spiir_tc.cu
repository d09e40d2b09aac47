// spiir_tc.cu -- block-parallel tensor-core form (not built yet in this file).
#include "spiir_tc.h"

struct TcBank {
    int unused;
};

static const char *kMsg = "tensor-core form not available in this build";

spiir_status spiir_tc_create(const spiir_bank_desc *, float, cudaStream_t, TcBank **out,
                             int64_t *) {
    *out = nullptr;
    return SPIIR_EUNSUPPORTED;
}
spiir_status spiir_tc_push(TcBank *, int, int, const float *, int64_t, int64_t, cudaStream_t,
                           KernelTimer *) {
    return SPIIR_EUNSUPPORTED;
}
spiir_status spiir_tc_reset(TcBank *, int, int, cudaStream_t) { return SPIIR_EUNSUPPORTED; }
const float2 *spiir_tc_output(TcBank *, int, int64_t *ring_len) {
    *ring_len = 0;
    return nullptr;
}
float *spiir_tc_stage(TcBank *) { return nullptr; }
unsigned int *spiir_tc_status(TcBank *) { return nullptr; }
void spiir_tc_info(TcBank *, spiir_bank_info *) {}
int64_t spiir_tc_footprint(const spiir_bank_desc *) { return -1; }
void spiir_tc_destroy(TcBank *b) { delete b; }
const char *spiir_tc_last_error() { return kMsg; }
