// spiir_replicas.cu -- a bank split by templates over several devices
// (spiir_replicas_* of include/spiir.h).
//
// Templates are independent (Eqs. iireq0, iireq1: a template's SNR depends on
// its own filters and the shared strain only), so a bank splits into
// contiguous template ranges, one ordinary bank per device, with no exchange
// between devices: a push copies the host strain to every device, each
// filters its templates, and their SNR rows are gathered into one host array.
// The ranges are balanced by filter-samples (filters weighted by the samples
// of their rate). Each device is driven by a host thread of its own, so the
// devices work at the same time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "spiir.h"
#include "spiir_plan.h"

using namespace spiir_host;

namespace {

struct Replica {
    int device = 0;
    int t0 = 0, T = 0;              // template range of the full bank
    spiir_bank_t bank = nullptr;
    cudaStream_t stream = nullptr;
    float2 *z_host = nullptr;       // pinned [n_streams][T][max_n]
    float *x_host = nullptr;        // pinned [n_streams][max_n]
    spiir_status st = SPIIR_OK;
    std::string err;
};

}  // namespace

struct spiir_replicas {
    int S = 1, T = 0;
    int64_t max_n = 0;
    std::vector<Replica> r;
};

namespace {

void release(spiir_replicas *rp) {
    for (Replica &q : rp->r) {
        if (q.device >= 0) cudaSetDevice(q.device);
        if (q.bank) spiir_bank_destroy(q.bank);
        if (q.stream) cudaStreamDestroy(q.stream);
        if (q.z_host) cudaFreeHost(q.z_host);
        if (q.x_host) cudaFreeHost(q.x_host);
        q.bank = nullptr;
        q.stream = nullptr;
        q.z_host = nullptr;
        q.x_host = nullptr;
    }
}

}  // namespace

extern "C" {

spiir_status spiir_replicas_create(const spiir_bank_desc *desc, const int32_t *devices, int32_t n_devices,
                                   spiir_replicas_t *out) {
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!devices || n_devices < 1) return fail(SPIIR_EINVAL, "need at least one device");
    spiir_status st = validate(desc);
    if (st) return st;
    int n_dev = 0;
    CUDA_TRY(cudaGetDeviceCount(&n_dev));
    for (int i = 0; i < n_devices; ++i)
        if (devices[i] < 0 || devices[i] >= n_dev) return fail(SPIIR_EINVAL, "device %d not present", devices[i]);
    const int T = desc->n_templates;
    if (n_devices > T) return fail(SPIIR_EINVAL, "more devices than templates");
    // filter-samples per template (a filter at level i runs at 1/2^i of the rate)
    std::vector<double> w(T, 0.0);
    for (int64_t k = 0; k < desc->n_filters; ++k)
        w[desc->template_id[k]] += std::ldexp(1.0, -(desc->level ? desc->level[k] : 0));
    double total = 0.0;
    for (double v : w) total += v + 1e-9;
    // contiguous ranges with about total / n_devices each, at least one template
    std::vector<int> cut(n_devices + 1, 0);
    cut[n_devices] = T;
    {
        double acc = 0.0;
        int t = 0;
        for (int i = 1; i < n_devices; ++i) {
            const double target = total * i / n_devices;
            while (t < T - (n_devices - i) && acc + w[t] + 1e-9 <= target) acc += w[t++] + 1e-9;
            t = std::max(t, cut[i - 1] + 1);
            cut[i] = t;
        }
    }
    spiir_replicas *rp = new (std::nothrow) spiir_replicas();
    if (!rp) return fail(SPIIR_ENOMEM, "host allocation failed");
    rp->S = desc->n_streams;
    rp->T = T;
    rp->max_n = (int64_t)desc->block_len * desc->max_push_blocks;
    rp->r.resize(n_devices);
    int prev = 0;
    cudaGetDevice(&prev);
    for (int i = 0; i < n_devices; ++i) {
        Replica &q = rp->r[i];
        q.device = devices[i];
        q.t0 = cut[i];
        q.T = cut[i + 1] - cut[i];
        // the sub-bank: filters of templates [t0, t0 + T), renumbered
        std::vector<float> ar, ai, br, bi;
        std::vector<int32_t> dl, tid;
        std::vector<int8_t> lv;
        for (int64_t k = 0; k < desc->n_filters; ++k) {
            const int t = desc->template_id[k];
            if (t < q.t0 || t >= q.t0 + q.T) continue;
            ar.push_back(desc->a_re[k]);
            ai.push_back(desc->a_im[k]);
            br.push_back(desc->b_re[k]);
            bi.push_back(desc->b_im[k]);
            dl.push_back(desc->delay[k]);
            tid.push_back(t - q.t0);
            lv.push_back(desc->level ? desc->level[k] : 0);
        }
        spiir_bank_desc d = *desc;
        d.n_templates = q.T;
        d.n_filters = (int64_t)ar.size();
        d.a_re = ar.data();
        d.a_im = ai.data();
        d.b_re = br.data();
        d.b_im = bi.data();
        d.delay = dl.data();
        d.template_id = tid.data();
        d.level = lv.data();
        cudaError_t e = cudaSetDevice(q.device);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&q.z_host, (size_t)rp->S * q.T * rp->max_n * sizeof(float2));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&q.x_host, (size_t)rp->S * rp->max_n * sizeof(float));
        if (e != cudaSuccess) {
            release(rp);
            delete rp;
            cudaSetDevice(prev);
            return fail(SPIIR_ENOMEM, "replica %d: %s", i, cudaGetErrorString(e));
        }
        if ((st = spiir_bank_create(&d, q.stream, &q.bank))) {
            const std::string m = spiir_last_error();
            release(rp);
            delete rp;
            cudaSetDevice(prev);
            return fail(st, "replica %d: %s", i, m.c_str());
        }
    }
    cudaSetDevice(prev);
    *out = rp;
    return SPIIR_OK;
}

spiir_status spiir_replicas_push_host(spiir_replicas_t rp, const float *x_host, int64_t n_samples,
                                      void *z_host) {
    if (!rp || !x_host || !z_host) return fail(SPIIR_EINVAL, "NULL argument");
    if (n_samples <= 0 || n_samples > rp->max_n) return fail(SPIIR_EINVAL, "bad n_samples");
    const int S = rp->S;
    std::vector<std::thread> th;
    for (Replica &q : rp->r) {
        th.emplace_back([&q, S, x_host, n_samples]() {
            q.st = SPIIR_OK;
            if (cudaSetDevice(q.device) != cudaSuccess) {
                q.st = SPIIR_ECUDA;
                q.err = "cudaSetDevice failed";
                return;
            }
            std::memcpy(q.x_host, x_host, (size_t)S * n_samples * sizeof(float));
            q.st = spiir_push_block_host(q.bank, -1, q.x_host, n_samples, q.z_host, q.stream);
            if (q.st) q.err = spiir_last_error();
        });
    }
    for (auto &t : th) t.join();
    for (size_t i = 0; i < rp->r.size(); ++i)
        if (rp->r[i].st) return fail(rp->r[i].st, "replica %zu: %s", i, rp->r[i].err.c_str());
    // gather: replica rows [t0, t0 + T) of every stream
    float2 *z = static_cast<float2 *>(z_host);
    for (const Replica &q : rp->r)
        for (int s = 0; s < S; ++s)
            std::memcpy(z + ((int64_t)s * rp->T + q.t0) * n_samples, q.z_host + (int64_t)s * q.T * n_samples,
                        (size_t)q.T * n_samples * sizeof(float2));
    return SPIIR_OK;
}

spiir_status spiir_replicas_get(spiir_replicas_t rp, int32_t i, int32_t *device, int32_t *template0,
                                int32_t *n_templates) {
    if (!rp || i < 0 || i >= (int32_t)rp->r.size() || !device || !template0 || !n_templates)
        return fail(SPIIR_EINVAL, "bad argument");
    *device = rp->r[i].device;
    *template0 = rp->r[i].t0;
    *n_templates = rp->r[i].T;
    return SPIIR_OK;
}

void spiir_replicas_destroy(spiir_replicas_t rp) {
    if (!rp) return;
    for (Replica &q : rp->r)
        if (cudaSetDevice(q.device) == cudaSuccess && q.stream) cudaStreamSynchronize(q.stream);
    release(rp);
    delete rp;
}

}  // extern "C"
