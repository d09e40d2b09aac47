// spiir_api.cu -- host side of libspiir: the C ABI of include/spiir.h.
//
// Bank creation turns the filter list into warp tasks for the FP32 recursion
// kernel (spiir_plain.cu):
//   * per level, each template's filters form a unit (split into parts of at
//     most 32*FMAX filters);
//   * a unit gets a group of G = 2^g lanes (the smallest with G*FMAX >= its
//     filter count) and F rounds, F = ceil(count/G) rounded up to even;
//   * units of the same (level, G, F) share a warp, 32/G units per warp;
//   * within a warp, each round's 32 filters are picked so that their strain
//     window offsets fall in distinct shared-memory banks where the pools
//     allow it (all lanes read x[n - d_k] in the same instruction);
//   * up to SPIIR_CTA_WARPS warps of one level and F form a CTA item.
// The level alignment delays D_i of the multi-rate scheme are folded into
// the filter delays (a delayed sum is the sum of delayed filters), so the
// upsample-and-add step needs no delay line.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "spiir.h"
#include "spiir_internal.h"
#include "spiir_plan.h"
#include "spiir_tc.h"

namespace spiir_host {

thread_local std::string g_err;

spiir_status fail(spiir_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

constexpr int kSmemMax = 227 * 1024;

// The library's resampling taps: Kaiser-window-tapered ideal low-pass with
// cutoff at half the input Nyquist frequency (Sec. 2.2). I0 by its series.
double lib_i0(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 1000; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term <= sum * 1e-18) break;
    }
    return sum;
}

double lib_kaiser_beta(double A) {
    if (A > 50.0) return 0.1102 * (A - 8.7);
    if (A >= 21.0) return 0.5842 * std::pow(A - 21.0, 0.4) + 0.07886 * (A - 21.0);
    return 0.0;
}

void lib_kaiser_taps(int n, double A, float *out) {
    const double beta = lib_kaiser_beta(A), norm = lib_i0(beta);
    std::vector<double> h(n);
    double s = 0.0;
    const double c = 0.5 * (n - 1);
    for (int i = 0; i < n; ++i) {
        const double m = i - c;
        const double x = m * M_PI * 0.5;
        const double ideal = (m == 0.0) ? 0.5 : std::sin(x) / (M_PI * m);
        const double u = (i - c) / c;
        const double w = lib_i0(beta * std::sqrt(std::max(0.0, 1.0 - u * u))) / norm;
        h[i] = ideal * w;
        s += h[i];
    }
    for (int i = 0; i < n; ++i) out[i] = (float)(h[i] / s);
}

// ---------------------------------------------------------------------------
// Plan: sizes and packed arrays for one kernel variant
// ---------------------------------------------------------------------------

struct Unit {
    int level, tmpl;
    std::vector<int64_t> filt;
    int G, F;
    int32_t dest;
};

// A push of n base-rate samples is cut into S time segments (S the smallest
// power of two with S * seg_base >= n, seg_base 4096 unless tuned); level
// i's segments are segment_len samples long (a multiple of 4, at most
// max(seg_base >> i, 4)), so at the lower
// rates the last segments may be short or empty.
int push_segments_n(int64_t n, int seg_base) {
    int S = 1;
    while ((int64_t)S * seg_base < n) S *= 2;
    return S;
}

int64_t segment_len(int64_t n, int i, int S) { return round_up(((n >> i) + S - 1) / S, 4); }

int64_t align_delay(int level, int n_levels, int n_taps, int n_taps_up, int align) {
    if (!align) return 0;
    int64_t D = 0;
    // a down/up round trip: the two linear-phase group delays at the higher rate
    const int64_t R = (n_taps + n_taps_up) / 2 - 1;
    for (int i = n_levels - 2; i >= level; --i) D = R + 2 * D;
    return D;
}

spiir_status validate(const spiir_bank_desc *d) {
    if (!d) return fail(SPIIR_EINVAL, "desc is NULL");
    if (d->n_templates < 1) return fail(SPIIR_EINVAL, "n_templates must be >= 1");
    if (d->n_levels < 1 || d->n_levels > SPIIR_MAX_LEVELS)
        return fail(SPIIR_EINVAL, "n_levels must be in [1, %d]", SPIIR_MAX_LEVELS);
    if (d->base_rate <= 0) return fail(SPIIR_EINVAL, "base_rate must be > 0");
    if (d->n_streams < 1) return fail(SPIIR_EINVAL, "n_streams must be >= 1");
    if (d->block_len < 1) return fail(SPIIR_EINVAL, "block_len must be >= 1");
    if (d->block_len % (1 << (d->n_levels - 1)) != 0)
        return fail(SPIIR_EINVAL, "block_len must be a multiple of 2^(n_levels-1)");
    if ((d->block_len >> (d->n_levels - 1)) % 4 != 0)
        return fail(SPIIR_EINVAL, "block_len / 2^(n_levels-1) must be a multiple of 4");
    if (d->max_push_blocks < 1) return fail(SPIIR_EINVAL, "max_push_blocks must be >= 1");
    if ((int64_t)d->block_len * d->max_push_blocks > (1ll << 30))
        return fail(SPIIR_EINVAL, "block_len * max_push_blocks too large");
    if (d->n_filters < 0) return fail(SPIIR_EINVAL, "n_filters must be >= 0");
    if (d->n_filters > 0 && (!d->a_re || !d->a_im || !d->b_re || !d->b_im || !d->delay ||
                             !d->template_id))
        return fail(SPIIR_EINVAL, "filter arrays must not be NULL");
    const int nt = d->n_taps ? d->n_taps : 32;
    if (nt < 2 || nt > SPIIR_MAX_DOWN_TAPS || (nt & 1))
        return fail(SPIIR_EINVAL, "n_taps must be even and in [2, %d]", SPIIR_MAX_DOWN_TAPS);
    const int ntu = d->n_taps_up ? d->n_taps_up : nt;
    if (ntu < 2 || ntu > SPIIR_MAX_TAPS || (ntu & 1))
        return fail(SPIIR_EINVAL, "interpolator taps must be even and in [2, %d]", SPIIR_MAX_TAPS);
    if ((d->h_down == nullptr) != (d->h_up == nullptr))
        return fail(SPIIR_EINVAL, "give both h_down and h_up or neither");
    if (d->mode < SPIIR_PLAIN_FP32 || d->mode > SPIIR_TC_BF16X2)
        return fail(SPIIR_EINVAL, "unknown mode %d", (int)d->mode);
    if (d->mode != SPIIR_PLAIN_FP32 && d->n_levels != 1)
        return fail(SPIIR_EUNSUPPORTED, "tensor-core forms take single-rate banks");
    if (d->hbm_budget_bytes < 0) return fail(SPIIR_EINVAL, "hbm_budget_bytes must be >= 0");
    if (d->carry < 0 || d->carry > 2)
        return fail(SPIIR_EINVAL, "carry must be 0 (FP64 per batch), 1 (double-float) or 2 (FP64 per chunk)");
    for (int64_t k = 0; k < d->n_filters; ++k) {
        if (d->template_id[k] < 0 || d->template_id[k] >= d->n_templates)
            return fail(SPIIR_EINVAL, "template_id[%lld] out of range", (long long)k);
        if (d->delay[k] < 0 || d->delay[k] > (1 << 20))
            return fail(SPIIR_EINVAL, "delay[%lld] out of range", (long long)k);
        if (d->level && (d->level[k] < 0 || d->level[k] >= d->n_levels))
            return fail(SPIIR_EINVAL, "level[%lld] out of range", (long long)k);
        if (!std::isfinite(d->a_re[k]) || !std::isfinite(d->a_im[k]) ||
            !std::isfinite(d->b_re[k]) || !std::isfinite(d->b_im[k]))
            return fail(SPIIR_EINVAL, "filter %lld has a non-finite coefficient", (long long)k);
    }
    return SPIIR_OK;
}

int default_variant(const spiir_bank_desc *d);

// Variant requested by desc->tune < 0, or the built-in choice.
int chosen_variant(const spiir_bank_desc *d) {
    if (d->tune < 0) {
        const int v = -d->tune - 1;
        if (v < spiir_recur_variant_count()) return v;
    }
    return default_variant(d);
}

void plan_info(const spiir_bank_desc *d, const Plan &p, spiir_bank_info *info) {
    info->n_slots = p.n_slots;
    info->filter_samples_per_block = p.fs_per_block;
    info->n_warp_tasks = (int32_t)p.tasks.size();
    info->n_cta_items = (int32_t)p.items.size();
    info->filters_per_lane = p.max_F;
    info->time_tile = p.T;
    info->kernel_variant = p.variant;
    info->max_delay = p.max_delay;
    info->tc_fir_len = 0;
    info->graph_captured = 0;
    info->n_units = (int32_t)p.n_units;
    info->smem_ways = p.lds_rounds ? (float)p.lds_wavefronts / (float)p.lds_rounds : 1.f;
    info->slot_fill = p.n_slots ? (float)d->n_filters / (float)p.n_slots : 1.f;
    info->segment_base = p.seg_base;
}

int default_variant(const spiir_bank_desc *d) {
    // By the mean number of filters in a bank's non-empty (template, rate)
    // units (d is validated). Up to 128: T = 32 with 4 filters per lane and
    // three CTAs per SM (variant 2), within 4% of the best compiled variant on
    // single-rate banks of 4 to 128 filters per template and the fastest on
    // multi-rate banks, whose units are small; 8 per lane loses up to 20%
    // there (4-lane units at 32 filters). Larger units: T = 32, 8 filters per
    // lane, two CTAs per SM (variant 3): units above 256 filters span 2-4
    // warps, twice as many independent chains as with 16 per lane, and the
    // 32-sample tile halves the reduction's share per sample.
    if (d->n_filters <= 0) return 3;
    std::vector<uint8_t> seen((size_t)d->n_templates * d->n_levels, 0);
    int64_t units = 0;
    for (int64_t k = 0; k < d->n_filters; ++k) {
        const size_t u = (size_t)d->template_id[k] * d->n_levels + (d->level ? d->level[k] : 0);
        units += seen[u] == 0;
        seen[u] = 1;
    }
    return d->n_filters <= 128 * units ? 2 : 3;
}

// Builds the plan. With arrays == false only the sizes are computed.
// hist_fixed (optional, n_levels entries): strain history per level to use
// instead of the bank's own (a server's shared strain buffers); it must hold
// every filter's delay plus the level's alignment delay.
spiir_status make_plan(const spiir_bank_desc *d, int variant, bool arrays, Plan &p,
                       const int *hist_fixed, int seg_base) {
    p = Plan();
    p.variant = variant;
    p.seg_base = seg_base;
    spiir_recur_variant_shape(variant, &p.T, &p.FMAX);
    p.n_levels = d->n_levels;
    p.H = d->n_levels - 1;
    p.n_taps = d->n_taps ? d->n_taps : 32;
    p.n_taps_up = d->n_taps_up ? d->n_taps_up : p.n_taps;
    p.align = (d->n_levels > 1) ? (d->align != 0) : 0;
    const int L = p.n_levels;
    const int64_t push_max = (int64_t)d->block_len * d->max_push_blocks;

    // filters per (level, template)
    std::vector<std::vector<int64_t>> lists((size_t)L * d->n_templates);
    std::vector<int> maxd(L, 0);
    for (int64_t k = 0; k < d->n_filters; ++k) {
        const int lv = d->level ? d->level[k] : 0;
        lists[(size_t)lv * d->n_templates + d->template_id[k]].push_back(k);
        maxd[lv] = std::max(maxd[lv], d->delay[k]);
    }
    int64_t off = 0;
    for (int i = 0; i < L; ++i) {
        const int64_t D = align_delay(i, L, p.n_taps, p.n_taps_up, p.align);
        int64_t h = (int64_t)maxd[i] + D;
        if (i < p.H) h = std::max<int64_t>(h, p.n_taps - 1);
        h = round_up(h, 4);
        if (hist_fixed) {
            if (hist_fixed[i] < h)
                return fail(SPIIR_EINVAL, "a delay at level %d (%lld samples with alignment) is above "
                                          "the server's strain history", i, (long long)h);
            h = hist_fixed[i];
        }
        p.hist[i] = (int)h;
        p.max_delay = std::max<int>(p.max_delay, (int)(maxd[i] + D));
        p.max_n[i] = push_max >> i;
        // the window holds the history plus the longest segment
        const int64_t sg = std::min<int64_t>(round_up(p.max_n[i], 4), round_up(std::max(p.seg_base >> i, 4), 4));
        if (16 + spiir_recur_red_bytes() + 4 * (h + sg) + 64 > kSmemMax - 1024)
            return fail(SPIIR_EUNSUPPORTED, "delay %lld at level %d does not fit shared memory",
                        (long long)h, i);
        p.seg[i] = (int)sg;
        p.smem_bytes = std::max<int>(p.smem_bytes,
                                     (int)(16 + spiir_recur_red_bytes() + 4 * (h + sg) + 64));
        p.xbuf_off[i] = off;
        off += round_up(h + p.max_n[i] + 64, 4);
    }
    p.xbuf_stream_stride = off;
    p.ring_len = round_up(push_max, 2);

    // units
    std::vector<Unit> units;
    int64_t rows[SPIIR_MAX_LEVELS] = {};
    bool all_single = true;
    for (int i = 0; i < L; ++i)
        for (int t = 0; t < d->n_templates; ++t) {
            const auto &f = lists[(size_t)i * d->n_templates + t];
            if ((int64_t)f.size() > 32ll * SPIIR_CTA_WARPS * p.FMAX) all_single = false;
        }
    p.need_combine = (L > 1) || !all_single;
    p.comb_ptr.assign((size_t)d->n_templates * L + 1, 0);
    std::vector<std::vector<int32_t>> comb((size_t)d->n_templates * L);
    for (int i = 0; i < L; ++i) {
        for (int t = 0; t < d->n_templates; ++t) {
            const auto &f = lists[(size_t)i * d->n_templates + t];
            const int64_t M = (int64_t)f.size();
            p.fs_per_block += M * (d->block_len >> i);
            if (M == 0) continue;
            const int64_t cap = 32ll * SPIIR_CTA_WARPS * p.FMAX;
            const int64_t parts = (M + cap - 1) / cap;
            // lanes x slots of a unit of m filters: G = smallest power of two
            // with G FMAX >= m, F = ceil(m / G) rounded up to even
            auto shape = [&](int64_t m, int &G, int &F) {
                G = 1;
                while ((int64_t)G * p.FMAX < m) G *= 2;
                F = (int)((m + G - 1) / G);
                F += F & 1;
                if (F < 2) F = 2;
            };
            auto add_unit = [&](int64_t b0, int64_t b1) {
                Unit u;
                u.level = i;
                u.tmpl = t;
                u.filt.assign(f.begin() + b0, f.begin() + b1);
                shape(b1 - b0, u.G, u.F);
                if (!p.need_combine) {
                    u.dest = t;
                } else {
                    const int64_t row = rows[i]++;
                    u.dest = -(int32_t)(row + 1);
                    comb[(size_t)t * L + i].push_back((int32_t)row);
                }
                units.push_back(std::move(u));
            };
            for (int64_t q = 0; q < parts; ++q) {
                const int64_t b0 = M * q / parts, b1 = M * (q + 1) / parts;
                const int64_t m = b1 - b0;
                int G, F;
                shape(m, G, F);
                // Where a combine pass runs anyway, split off the filters above
                // the largest full block of G' lanes x FMAX slots when that saves
                // more padded slots than an extra partial row costs: a row is
                // 16 bytes of HBM traffic per sample (written, read back), about
                // 12 slot-updates of FP32 time at the measured peaks.
                int64_t full = 0;
                for (int64_t g2 = 1; g2 * p.FMAX <= m; g2 *= 2) full = g2 * p.FMAX;
                if (p.need_combine && full > 0 && full < m) {
                    int Gr, Fr;
                    shape(m - full, Gr, Fr);
                    if ((int64_t)G * F - (full + (int64_t)Gr * Fr) > 12) {
                        add_unit(b0, b0 + full);
                        add_unit(b0 + full, b1);
                        continue;
                    }
                }
                add_unit(b0, b1);
            }
        }
    }
    for (size_t j = 0; j < comb.size(); ++j) {
        p.comb_ptr[j + 1] = p.comb_ptr[j] + (int32_t)comb[j].size();
        for (auto r : comb[j]) p.comb_rows.push_back(r);
    }
    int64_t poff = 0, uoff = 0;
    for (int i = 0; i < L; ++i) {
        p.part_rows[i] = rows[i];
        p.part_stride[i] = round_up(p.max_n[i], 2);
        p.part_base[i] = poff;
        poff += rows[i] * p.part_stride[i];
        if (i > 0) {
            p.ubuf_stride[i] = SPIIR_UHIST;
            p.ubuf_off[i] = uoff;
            uoff += (int64_t)d->n_templates * p.ubuf_stride[i];
        }
    }
    p.part_stream_stride = poff;
    p.ubuf_stream_stride = uoff;

    // Bundles: one warp of small units (32/G units of G <= 32 lanes), or the
    // 2^xw warps of one unit larger than a warp; all of one (level, G, F).
    std::stable_sort(units.begin(), units.end(), [](const Unit &a, const Unit &b) {
        if (a.level != b.level) return a.level < b.level;
        if (a.F != b.F) return a.F > b.F;
        return a.G < b.G;
    });
    struct Bundle {
        int level, G, F, W;       // W warps; G <= 32 when W == 1
        std::vector<int> units;
    };
    std::vector<Bundle> bundles;
    for (size_t u = 0; u < units.size();) {
        if (units[u].G > 32) {
            bundles.push_back(Bundle{units[u].level, 32, units[u].F, units[u].G / 32, {(int)u}});
            ++u;
            continue;
        }
        Bundle b{units[u].level, units[u].G, units[u].F, 1, {}};
        const int per = 32 / b.G;
        while (u < units.size() && (int)b.units.size() < per && units[u].level == b.level &&
               units[u].G == b.G && units[u].F == b.F)
            b.units.push_back((int)u++);
        bundles.push_back(std::move(b));
    }
    // CTA items: bundles of one (level, F, W) filling SPIIR_CTA_WARPS warps
    std::vector<int> bo(bundles.size());
    for (size_t i = 0; i < bo.size(); ++i) bo[i] = (int)i;
    std::stable_sort(bo.begin(), bo.end(), [&](int a, int b) {
        const Bundle &x = bundles[a], &y = bundles[b];
        if (x.level != y.level) return x.level < y.level;
        if (x.F != y.F) return x.F > y.F;
        return x.W > y.W;
    });
    std::vector<std::vector<int>> item_bundles;
    for (size_t i = 0; i < bo.size();) {
        std::vector<int> it;
        const Bundle &b0 = bundles[bo[i]];
        int warps_used = 0;
        while (i < bo.size() && warps_used + bundles[bo[i]].W <= SPIIR_CTA_WARPS &&
               bundles[bo[i]].level == b0.level && bundles[bo[i]].F == b0.F &&
               bundles[bo[i]].W == b0.W) {
            warps_used += bundles[bo[i]].W;
            it.push_back(bo[i++]);
        }
        item_bundles.push_back(std::move(it));
    }

    p.n_units = (int64_t)units.size();
    int64_t n_slots = 0;
    size_t n_warps = 0;
    for (auto &b : bundles) {
        n_slots += 32ll * b.F * b.W;
        n_warps += b.W;
        p.max_F = std::max(p.max_F, b.F);
    }
    p.n_slots = n_slots;
    // queue order of the items: most work first
    p.order.resize(item_bundles.size());
    {
        std::vector<int64_t> work(item_bundles.size(), 0);
        for (size_t i = 0; i < item_bundles.size(); ++i)
            for (int bi : item_bundles[i])
                work[i] += (int64_t)bundles[bi].F * bundles[bi].W * p.max_n[bundles[bi].level];
        for (size_t i = 0; i < p.order.size(); ++i) p.order[i] = (int32_t)i;
        std::stable_sort(p.order.begin(), p.order.end(),
                         [&](int32_t a, int32_t b) { return work[a] > work[b]; });
    }
    if (!arrays) {
        p.tasks.resize(n_warps);
        p.items.resize(item_bundles.size());
        return SPIIR_OK;
    }

    p.are.assign(n_slots, 0.f);
    p.aim.assign(n_slots, 0.f);
    p.bre.assign(n_slots, 0.f);
    p.bim.assign(n_slots, 0.f);
    p.xoff.assign(n_slots, 0);
    p.slot_filter.assign(n_slots, -1);
    int64_t slot_base = 0;
    for (auto &ib : item_bundles) {
        CtaItem ci;
        ci.level = bundles[ib[0]].level;
        ci.task_begin = (int32_t)p.tasks.size();
        ci.task_count = 0;
        ci.F = bundles[ib[0]].F;
        for (int bi : ib) {
            const Bundle &b = bundles[bi];
            const int g = b.G, F = b.F, lv = b.level, W = b.W;
            const int64_t D = align_delay(lv, L, p.n_taps, p.n_taps_up, p.align);
            const int hist = p.hist[lv];
            int gl = 0;
            while ((1 << gl) < g) ++gl;
            int xw = 0;
            while ((1 << xw) < W) ++xw;
            const int out_base = (int32_t)p.task_out.size();
            for (int u : b.units) p.task_out.push_back(units[u].dest);
            // pools bucketed by the shared-memory bank of the window offset:
            // one per group (W == 1) or one shared by the unit's warps
            const int ng = (int)b.units.size();
            std::vector<std::vector<std::vector<int64_t>>> pool(
                ng, std::vector<std::vector<int64_t>>(32));
            std::vector<int> rot(ng, 0);
            for (int q = 0; q < ng; ++q)
                for (int64_t k : units[b.units[q]].filt) {
                    const int64_t xo = hist - (d->delay[k] + D);
                    pool[q][xo & 31].push_back(k);
                }
            const int64_t base0 = slot_base;
            for (int w = 0; w < W; ++w) {
                WarpTask wt;
                wt.slot_base = (int32_t)(base0 + 32ll * F * w);
                wt.F = (int8_t)F;
                wt.g_log2 = (int8_t)gl;
                wt.level = (int8_t)lv;
                wt.xw_log2 = (int8_t)xw;
                wt.out_base = out_base;
                wt.n_groups = (int16_t)(W > 1 ? 1 : ng);
                wt.xw_rank = (int8_t)w;
                wt.pad = 0;
                p.tasks.push_back(wt);
                ci.task_count++;
            }
            // rounds of all warps interleaved so the shared pool drains evenly
            for (int r = 0; r < F; ++r) {
                for (int w = 0; w < W; ++w) {
                    uint32_t used = 0;
                    int per_bank[32] = {};
                    for (int l = 0; l < 32; ++l) {
                        const int64_t s = base0 + 32ll * F * w + (int64_t)r * 32 + l;
                        const int q = W > 1 ? 0 : l / g;
                        int64_t pick = -1;
                        if (q < ng) {
                            // fullest bank not yet read this round, else the
                            // fullest bank (a conflict); drawing from the fullest
                            // keeps the pools even for the later rounds
                            auto &pl = pool[q];
                            int best = -1;
                            for (int pass = 0; pass < 2 && best < 0; ++pass) {
                                size_t most = 0;
                                for (int c = 0; c < 32; ++c) {
                                    const int bk = (rot[q] + c) & 31;
                                    if (pass == 0 && (used >> bk & 1u)) continue;
                                    if (pl[bk].size() > most) {
                                        most = pl[bk].size();
                                        best = bk;
                                    }
                                }
                            }
                            if (best >= 0) {
                                pick = pl[best].back();
                                pl[best].pop_back();
                                rot[q] = (best + 1) & 31;
                            }
                        }
                        int32_t xo;
                        if (pick >= 0) {
                            p.slot_filter[s] = pick;
                            p.are[s] = d->a_re[pick];
                            p.aim[s] = d->a_im[pick];
                            p.bre[s] = d->b_re[pick];
                            p.bim[s] = d->b_im[pick];
                            xo = (int32_t)(hist - (d->delay[pick] + D));
                        } else {
                            // inert padding slot: read a free bank inside the window
                            int bk = 0;
                            while (bk < 32 && (used >> bk & 1u)) ++bk;
                            bk &= 31;
                            xo = hist - ((hist - bk) & 31);
                            if (xo < 0) xo = hist;
                        }
                        p.xoff[s] = xo;
                        used |= 1u << (xo & 31);
                        per_bank[xo & 31]++;
                    }
                    int wave = 0;
                    for (int bk = 0; bk < 32; ++bk) wave = std::max(wave, per_bank[bk]);
                    p.lds_rounds++;
                    p.lds_wavefronts += wave;
                }
            }
            slot_base += 32ll * F * W;
        }
        p.items.push_back(ci);
    }
    return SPIIR_OK;
}

int64_t plan_footprint(const spiir_bank_desc *d, const Plan &p) {
    const int64_t S = d->n_streams;
    int64_t b = 0;
    b += p.n_slots * (4 * 4 + 4);                        // coefficients + offsets
    b += (int64_t)p.tasks.size() * sizeof(WarpTask);
    b += (int64_t)p.items.size() * sizeof(CtaItem);
    b += (int64_t)p.tasks.size() * 32 * 4;               // task_out (upper bound)
    b += ((int64_t)d->n_templates * p.n_levels + 1) * 4 + p.n_slots * 4;  // comb lists (bound)
    b += (int64_t)p.items.size() * 4 * (1 + S) + S * 4;   // queue order, progress
    b += S * p.n_slots * 8;                              // state
    b += S * p.xbuf_stream_stride * 4;                   // strain windows
    b += S * p.part_stream_stride * 8;                   // partial sums
    b += S * p.ubuf_stream_stride * 8;                   // upsampler rows
    b += S * (int64_t)d->n_templates * p.ring_len * 8;   // output ring
    b += S * p.ring_len * 4;                             // host-call staging
    b += 256;
    return b;
}

template <typename T>
spiir_status upload(T **dst, const std::vector<T> &src, cudaStream_t s) {
    *dst = nullptr;
    if (src.empty()) return SPIIR_OK;
    CUDA_TRY(cudaMalloc((void **)dst, src.size() * sizeof(T)));
    CUDA_TRY(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return SPIIR_OK;
}

}  // namespace spiir_host

using namespace spiir_host;

// ---------------------------------------------------------------------------
// The bank
// ---------------------------------------------------------------------------

struct GraphEntry {
    int s0, count;
    int64_t n, n_prev, zoff;
    cudaGraphExec_t exec;
    std::vector<int64_t> prev;   // block form: previous push length of every pushed stream
};

struct spiir_bank {
    spiir_bank_desc d;
    Plan p;
    float scale = 0.f;
    std::vector<float> h_down, h_up;
    int device = 0;
    // device arrays
    float *are = nullptr, *aim = nullptr, *bre = nullptr, *bim = nullptr;
    int32_t *xoff = nullptr;
    WarpTask *tasks = nullptr;
    CtaItem *items = nullptr;
    int32_t *task_out = nullptr, *comb_ptr = nullptr, *comb_rows = nullptr;
    float2 *state = nullptr, *partial = nullptr, *ubuf = nullptr, *z = nullptr;
    float *xbuf = nullptr, *xstage = nullptr;
    unsigned int *status = nullptr;
    int32_t *order = nullptr;
    unsigned int *queue = nullptr, *prog = nullptr;
    int ctas_per_sm = 1, n_sms = 1;
    int ctas_cap = 0;                       // tuned CTAs per SM (0: the occupancy limit)
    float tune_ms = 0.f;                    // wall time the autotuner took
    cudaStream_t cap = nullptr;             // private stream for graph capture
    cudaStream_t copy[2] = {nullptr, nullptr};   // host push: device-to-host copies
    cudaEvent_t piece_done[4] = {};         // host push: a piece's SNR is in the ring
    // asynchronous host pushes alternate between ring columns [0, n) and
    // [n, 2n) when the ring holds two pushes: half_free[h][c] is recorded on
    // copy stream c after the last copy-back out of half h, which covered
    // ring columns [half_lo[h], half_hi[h]); a later write there waits on it
    cudaEvent_t half_free[2][2] = {};
    int64_t half_lo[2] = {0, 0}, half_hi[2] = {0, 0};
    int async_half = 0;                     // half the next asynchronous push writes
    std::vector<GraphEntry> graphs;
    std::vector<int64_t> last_n;            // samples of the last kernel push (strain history)
    std::vector<int64_t> ring_n;            // samples of the last call's push held in the ring
    std::vector<int64_t> ring_base;         // ring column where that push starts
    std::vector<char> out_valid;            // the output ring holds a push of the stream
    uint64_t fingerprint = 0;               // of the description, for state import
    int64_t footprint = 0;
    int64_t n_filters = 0;
    TcBank *tc = nullptr;
    KernelTimer *timer = nullptr;

    void free_device() {
        void *ptrs[] = {are, aim, bre, bim, xoff, tasks, items, task_out, comb_ptr, comb_rows,
                        state, partial, ubuf, z, xbuf, xstage, status, order, queue, prog};
        for (void *q : ptrs)
            if (q) cudaFree(q);
        are = aim = bre = bim = nullptr;
        xoff = nullptr;
        tasks = nullptr;
        items = nullptr;
        task_out = comb_ptr = comb_rows = nullptr;
        state = partial = ubuf = z = nullptr;
        xbuf = xstage = nullptr;
        status = nullptr;
        order = nullptr;
        queue = prog = nullptr;
        if (tc) {
            spiir_tc_destroy(tc);
            tc = nullptr;
        }
        if (timer) {
            timer->release();
            delete timer;
            timer = nullptr;
        }
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
        if (cap) {
            cudaStreamDestroy(cap);
            cap = nullptr;
        }
        for (auto &c : copy)
            if (c) {
                cudaStreamDestroy(c);
                c = nullptr;
            }
        for (auto &e : piece_done)
            if (e) {
                cudaEventDestroy(e);
                e = nullptr;
            }
        for (auto &h : half_free)
            for (auto &e : h)
                if (e) {
                    cudaEventDestroy(e);
                    e = nullptr;
                }
    }
};

namespace {

spiir_status alloc_plain(spiir_bank *b, cudaStream_t s) {
    const Plan &p = b->p;
    const int64_t S = b->d.n_streams;
    spiir_status st;
    if ((st = upload(&b->are, p.are, s))) return st;
    if ((st = upload(&b->aim, p.aim, s))) return st;
    if ((st = upload(&b->bre, p.bre, s))) return st;
    if ((st = upload(&b->bim, p.bim, s))) return st;
    if ((st = upload(&b->xoff, p.xoff, s))) return st;
    if ((st = upload(&b->tasks, p.tasks, s))) return st;
    if ((st = upload(&b->items, p.items, s))) return st;
    if ((st = upload(&b->task_out, p.task_out, s))) return st;
    if ((st = upload(&b->comb_ptr, p.comb_ptr, s))) return st;
    if ((st = upload(&b->comb_rows, p.comb_rows, s))) return st;
    if ((st = upload(&b->order, p.order, s))) return st;
    CUDA_TRY(cudaMalloc((void **)&b->queue, S * sizeof(unsigned int)));
    CUDA_TRY(cudaMalloc((void **)&b->prog, std::max<int64_t>(1, S * (int64_t)p.items.size()) *
                                              sizeof(unsigned int)));
    CUDA_TRY(cudaMalloc((void **)&b->state, std::max<int64_t>(1, S * p.n_slots) * sizeof(float2)));
    CUDA_TRY(cudaMalloc((void **)&b->xbuf, S * p.xbuf_stream_stride * sizeof(float)));
    if (p.part_stream_stride)
        CUDA_TRY(cudaMalloc((void **)&b->partial, S * p.part_stream_stride * sizeof(float2)));
    if (p.ubuf_stream_stride)
        CUDA_TRY(cudaMalloc((void **)&b->ubuf, S * p.ubuf_stream_stride * sizeof(float2)));
    CUDA_TRY(cudaMalloc((void **)&b->z, S * (int64_t)b->d.n_templates * p.ring_len * sizeof(float2)));
    CUDA_TRY(cudaMalloc((void **)&b->xstage, S * p.ring_len * sizeof(float)));
    CUDA_TRY(cudaMalloc((void **)&b->status, sizeof(unsigned int)));
    CUDA_TRY(cudaMemsetAsync(b->state, 0, std::max<int64_t>(1, S * p.n_slots) * sizeof(float2), s));
    CUDA_TRY(cudaMemsetAsync(b->xbuf, 0, S * p.xbuf_stream_stride * sizeof(float), s));
    if (b->ubuf) CUDA_TRY(cudaMemsetAsync(b->ubuf, 0, S * p.ubuf_stream_stride * sizeof(float2), s));
    CUDA_TRY(cudaMemsetAsync(b->z, 0, S * (int64_t)b->d.n_templates * p.ring_len * sizeof(float2), s));
    CUDA_TRY(cudaMemsetAsync(b->status, 0, sizeof(unsigned int), s));
    CUDA_TRY(spiir_recur_prepare(p.variant, p.smem_bytes, &b->ctas_per_sm));
    if (p.need_combine) CUDA_TRY(spiir_combine_prepare());
    CUDA_TRY(cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, b->device));
    CUDA_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    return SPIIR_OK;
}

// Time segments per push: about 4096 base-rate samples each, a power of two,
// at least 4 samples at the lowest level.
int push_segments(const Plan &p, int64_t n) { return push_segments_n(n, p.seg_base); }

void level_args(const spiir_bank *b, int64_t n, int64_t n_prev, LevelArgs *lev) {
    const Plan &p = b->p;
    const int S = push_segments(p, n);
    for (int i = 0; i < p.n_levels; ++i) {
        LevelArgs &L = lev[i];
        L.hist = p.hist[i];
        L.n = (int32_t)(n >> i);
        L.seg = (int32_t)segment_len(n, i, S);
        L.n_prev = (int32_t)(n_prev >> i);
        L.part_base = p.part_base[i];
        L.part_stride = p.part_stride[i];
        L.xbuf_off = p.xbuf_off[i];
        L.ubuf_off = p.ubuf_off[i];
        L.ubuf_stride = p.ubuf_stride[i];
        L.pad = 0;
    }
}

// The kernels of one push (no host state changes).
// zoff: first output-ring column this push writes (0 for an ordinary push;
// the pieces of a pipelined host push write consecutive column ranges).
spiir_status launch_sequence(spiir_bank *b, int s0, int count, const float *x, int64_t x_stride,
                             int64_t n, int64_t n_prev, cudaStream_t st, bool stall_test,
                             int64_t zoff = 0) {
    const Plan &p = b->p;
    PrologueArgs pa{};
    pa.queue = b->queue;
    pa.prog = b->prog;
    pa.n_items = (int32_t)p.items.size();
    pa.xbuf = b->xbuf;
    pa.xbuf_stream_stride = p.xbuf_stream_stride;
    pa.x_in = x;
    pa.x_in_stream_stride = x_stride;
    pa.stream0 = s0;
    pa.n_levels = p.n_levels;
    level_args(b, n, n_prev, pa.lev);
    KernelTimer &tm = *b->timer;
    tm.begin(SPIIR_K_PROLOGUE, st);
    CUDA_TRY(spiir_launch_prologue(pa, count, st));
    tm.end(st, kPrologueLaunches);
    if (p.n_levels > 1) {
        DecimArgs da{};
        da.xbuf = b->xbuf;
        da.xbuf_stream_stride = p.xbuf_stream_stride;
        da.stream0 = s0;
        da.n_levels = p.n_levels;
        da.n_taps = p.n_taps;
        for (int j = 0; j < p.n_taps; ++j) da.h_down[j] = b->h_down[j];
        level_args(b, n, n_prev, da.lev);
        tm.begin(SPIIR_K_DECIMATE, st);
        CUDA_TRY(spiir_launch_decimate(da, count, st));
        tm.end(st);
    }
    if (!p.items.empty()) {
        RecurArgs ra{};
        ra.tasks = b->tasks;
        ra.items = b->items;
        ra.order = b->order;
        ra.n_items = (int32_t)p.items.size();
        ra.n_segs = push_segments(p, n);
        ra.queue = b->queue;
        ra.prog = b->prog;
        ra.stall_test = stall_test ? 1 : 0;
        ra.task_out = b->task_out;
        ra.a_re = b->are;
        ra.a_im = b->aim;
        ra.b_re = b->bre;
        ra.b_im = b->bim;
        ra.xoff = b->xoff;
        ra.state = b->state;
        ra.n_slots = p.n_slots;
        ra.xbuf = b->xbuf;
        ra.xbuf_stream_stride = p.xbuf_stream_stride;
        ra.partial = b->partial;
        ra.partial_stream_stride = p.part_stream_stride;
        ra.z = b->z + zoff;
        ra.z_row_stride = p.ring_len;
        ra.z_stream_stride = (int64_t)b->d.n_templates * p.ring_len;
        ra.scale = b->scale;
        ra.stream0 = s0;
        ra.n_levels = p.n_levels;
        ra.status = b->status;
        level_args(b, n, n_prev, ra.lev);
        tm.begin(SPIIR_K_RECUR, st);
        const int64_t total = (int64_t)ra.n_segs * ra.n_items;
        const int per_sm = b->ctas_cap > 0 ? std::min(b->ctas_cap, b->ctas_per_sm) : b->ctas_per_sm;
        const int64_t resident = std::max<int64_t>(1, (int64_t)per_sm * b->n_sms / count);
        const int ctas = (int)std::min<int64_t>(total, resident);
        CUDA_TRY(spiir_launch_recur(ra, p.variant, ctas, count, p.smem_bytes, st));
        tm.end(st);
    }
    if (p.need_combine) {
        CombineArgs ca{};
        ca.comb_ptr = b->comb_ptr;
        ca.comb_rows = b->comb_rows;
        ca.partial = b->partial;
        ca.partial_stream_stride = p.part_stream_stride;
        ca.ubuf = b->ubuf;
        ca.ubuf_stream_stride = p.ubuf_stream_stride;
        ca.z = b->z + zoff;
        ca.z_row_stride = p.ring_len;
        ca.z_stream_stride = (int64_t)b->d.n_templates * p.ring_len;
        ca.scale = b->scale;
        ca.n_templates = b->d.n_templates;
        ca.n_levels = p.n_levels;
        ca.n_taps = p.n_taps_up;
        ca.stream0 = s0;
        ca.status = b->status;
        for (int j = 0; j < p.n_taps_up; ++j) ca.h_up2[j] = 2.0f * b->h_up[j];
        level_args(b, n, n_prev, ca.lev);
        tm.begin(SPIIR_K_COMBINE, st);
        CUDA_TRY(spiir_launch_combine(ca, spiir_combine_chunk(p.n_levels, p.ring_len), count, st));
        tm.end(st);
    }
    return SPIIR_OK;
}

// A push replayed from a CUDA graph: the strain is copied into the bank's
// staging buffer on the caller's stream and one graph (captured once per
// stream set, length and previous length) launches all kernels.
spiir_status push_graph(spiir_bank *b, int s0, int count, const float *x, int64_t x_stride,
                        int64_t n, cudaStream_t st, int64_t zoff) {
    const int64_t n_prev = b->last_n[s0];
    GraphEntry *ge = nullptr;
    for (auto &g : b->graphs)
        if (g.s0 == s0 && g.count == count && g.n == n && g.n_prev == n_prev && g.zoff == zoff) ge = &g;
    if (!ge) {
        if (b->graphs.size() >= 16) {
            cudaGraphExecDestroy(b->graphs.front().exec);
            b->graphs.erase(b->graphs.begin());
        }
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        spiir_status stc = launch_sequence(b, s0, count, b->xstage + (int64_t)s0 * n, n, n, n_prev,
                                           b->cap, false, zoff);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (stc) {
            if (g) cudaGraphDestroy(g);
            return stc;
        }
        if (e != cudaSuccess) return fail(SPIIR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(SPIIR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        b->graphs.push_back(GraphEntry{s0, count, n, n_prev, zoff, exec, {}});
        ge = &b->graphs.back();
    }
    float *dst = b->xstage + (int64_t)s0 * n;
    if (x != dst) {
        if (x_stride == n) {
            CUDA_TRY(cudaMemcpyAsync(dst, x, count * n * sizeof(float), cudaMemcpyDeviceToDevice, st));
        } else {
            CUDA_TRY(cudaMemcpy2DAsync(dst, n * sizeof(float), x, x_stride * sizeof(float),
                                       n * sizeof(float), count, cudaMemcpyDeviceToDevice, st));
        }
    }
    CUDA_TRY(cudaGraphLaunch(ge->exec, st));
    return SPIIR_OK;
}

// A block-form push replayed from a CUDA graph (captured once per stream
// set, length, previous lengths and output offset): the strain is copied into
// the bank's staging buffer, which the graph reads.
spiir_status push_tc(spiir_bank *b, int s0, int count, const float *x, int64_t n, cudaStream_t st,
                     int64_t zoff) {
    std::vector<int64_t> &last = spiir_tc_last_n(b->tc);
    if (!b->cap || b->timer->on) {
        spiir_status r = spiir_tc_push(b->tc, s0, count, x, n, n, st, b->timer, zoff);
        return r ? fail(r, "%s", spiir_tc_last_error()) : SPIIR_OK;
    }
    std::vector<int64_t> prev(last.begin() + s0, last.begin() + s0 + count);
    GraphEntry *ge = nullptr;
    for (auto &g : b->graphs)
        if (g.s0 == s0 && g.count == count && g.n == n && g.zoff == zoff && g.prev == prev) ge = &g;
    float *stage = spiir_tc_stage(b->tc);
    if (!ge) {
        if (b->graphs.size() >= 16) {
            cudaGraphExecDestroy(b->graphs.front().exec);
            b->graphs.erase(b->graphs.begin());
        }
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        spiir_status stc = spiir_tc_push(b->tc, s0, count, stage, n, n, b->cap, b->timer, zoff);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        // capturing ran the push's host logic: put its state back
        std::copy(prev.begin(), prev.end(), last.begin() + s0);
        if (stc) {
            if (g) cudaGraphDestroy(g);
            return fail(stc, "%s", spiir_tc_last_error());
        }
        if (e != cudaSuccess) return fail(SPIIR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(SPIIR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        b->graphs.push_back(GraphEntry{s0, count, n, prev.empty() ? 0 : prev[0], zoff, exec, prev});
        ge = &b->graphs.back();
    }
    if (x != stage) CUDA_TRY(cudaMemcpyAsync(stage, x, (size_t)count * n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaGraphLaunch(ge->exec, st));
    for (int q = s0; q < s0 + count; ++q) last[q] = n;
    return SPIIR_OK;
}

spiir_status push_plain(spiir_bank *b, int s0, int count, const float *x, int64_t x_stride,
                        int64_t n, cudaStream_t st, bool stall_test = false, int64_t zoff = 0) {
    spiir_status r;
    if (b->cap && !b->timer->on && !stall_test)
        r = push_graph(b, s0, count, x, x_stride, n, st, zoff);
    else
        r = launch_sequence(b, s0, count, x, x_stride, n, b->last_n[s0], st, stall_test, zoff);
    if (r) return r;
    for (int q = s0; q < s0 + count; ++q) b->last_n[q] = n;
    return SPIIR_OK;
}

// FNV-1a over everything in a description that the filter state's meaning
// and layout depend on (the carry arithmetic of the tensor-core forms is left
// out: their state is exported in FP64).
uint64_t desc_fingerprint(const spiir_bank_desc *d) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    };
    const int32_t sc[] = {d->n_templates, d->n_levels, d->base_rate, d->block_len,
                          d->max_push_blocks, d->n_taps ? d->n_taps : 32,
                          d->n_taps_up ? d->n_taps_up : (d->n_taps ? d->n_taps : 32), d->align,
                          (int32_t)(d->mode != SPIIR_PLAIN_FP32), d->mode == SPIIR_PLAIN_FP32 ? 0 :
                          (d->chunk_len ? d->chunk_len : 256)};
    mix(sc, sizeof sc);
    mix(&d->n_filters, sizeof d->n_filters);
    const int64_t n = d->n_filters;
    if (n > 0) {
        mix(d->a_re, n * sizeof(float));
        mix(d->a_im, n * sizeof(float));
        mix(d->b_re, n * sizeof(float));
        mix(d->b_im, n * sizeof(float));
        mix(d->delay, n * sizeof(int32_t));
        mix(d->template_id, n * sizeof(int32_t));
        if (d->level) mix(d->level, n * sizeof(int8_t));
    }
    if (d->h_down) {
        const int nt = d->n_taps ? d->n_taps : 32, ntu = d->n_taps_up ? d->n_taps_up : nt;
        mix(d->h_down, nt * sizeof(float));
        mix(d->h_up, ntu * sizeof(float));
    }
    return h;
}

// Tile choices of a bank: the recursion variant, its time-segment length and
// CTAs per SM (plain form), the chunk length (block form).
struct Tuning {
    int variant = 3;
    int seg_base = 4096;
    int ctas = 0;
    int chunk_len = 0;
};

spiir_status build_bank(const spiir_bank_desc *desc_in, const Tuning &tn, cudaStream_t s,
                        spiir_bank *b) {
    spiir_bank_desc dd = *desc_in;
    if (tn.chunk_len) dd.chunk_len = tn.chunk_len;
    const spiir_bank_desc *desc = &dd;
    const int variant = tn.variant;
    b->ctas_cap = tn.ctas;
    b->d = *desc;
    b->n_filters = desc->n_filters;
    b->d.a_re = b->d.a_im = b->d.b_re = b->d.b_im = nullptr;
    b->d.delay = b->d.template_id = nullptr;
    b->d.level = nullptr;
    b->d.h_down = b->d.h_up = nullptr;
    if (b->d.n_taps == 0) b->d.n_taps = 32;
    if (b->d.n_taps_up == 0) b->d.n_taps_up = b->d.n_taps;
    if (b->d.chunk_len == 0) b->d.chunk_len = 256;
    b->scale = desc->snr_scale != 0.f ? desc->snr_scale : 2.0f / (float)desc->base_rate;
    const int nt = b->d.n_taps, ntu = b->d.n_taps_up;
    b->h_down.resize(nt);
    b->h_up.resize(ntu);
    if (desc->h_down) {
        std::copy(desc->h_down, desc->h_down + nt, b->h_down.begin());
        std::copy(desc->h_up, desc->h_up + ntu, b->h_up.begin());
    } else {
        lib_kaiser_taps(nt, 60.0, b->h_down.data());
        lib_kaiser_taps(ntu, 60.0, b->h_up.data());
    }
    b->last_n.assign(desc->n_streams, 0);
    b->ring_n.assign(desc->n_streams, 0);
    b->ring_base.assign(desc->n_streams, 0);
    b->out_valid.assign(desc->n_streams, 0);
    b->fingerprint = desc_fingerprint(desc);
    if (!b->timer) b->timer = new KernelTimer();
    spiir_status st;
    if (desc->mode != SPIIR_PLAIN_FP32) {
        st = spiir_tc_create(desc, b->scale, s, &b->tc, &b->footprint);
        if (st) return fail(st, "%s", spiir_tc_last_error());
        CUDA_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        return SPIIR_OK;
    }
    if ((st = make_plan(desc, variant, true, b->p, nullptr, tn.seg_base))) return st;
    b->footprint = plan_footprint(desc, b->p);
    if (desc->hbm_budget_bytes > 0 && b->footprint > desc->hbm_budget_bytes)
        return fail(SPIIR_EBUDGET, "bank needs %lld bytes, budget %lld",
                    (long long)b->footprint, (long long)desc->hbm_budget_bytes);
    if ((st = alloc_plain(b, s))) return st;
    CUDA_TRY(cudaStreamSynchronize(s));
    return SPIIR_OK;
}

// Device time of a few pushes of zeros through a built bank (one push to
// warm up, three timed), on its own kernels.
spiir_status time_pushes(spiir_bank *b, const spiir_bank_desc *desc, cudaStream_t s, float *ms) {
    const int S = desc->n_streams;
    const int64_t n = (int64_t)desc->block_len * std::min(desc->max_push_blocks, 4);
    float *x = b->tc ? spiir_tc_stage(b->tc) : b->xstage;
    CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)S * n * sizeof(float), s));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    spiir_status st = SPIIR_OK;
    for (int r = 0; r < 4 && !st; ++r) {
        if (r == 1) cudaEventRecord(e0, s);
        st = b->tc ? spiir_tc_push(b->tc, 0, S, x, n, n, s, b->timer) : push_plain(b, 0, S, x, n, n, s);
    }
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (e != cudaSuccess) return fail(SPIIR_ECUDA, "autotune: %s", cudaGetErrorString(e));
    *ms = t;
    return SPIIR_OK;
}

// Time one tuning; keep it in *best when faster. Banks that cannot be built
// with it (shared memory, ...) are skipped.
spiir_status try_tuning(const spiir_bank_desc *desc, const Tuning &tn, cudaStream_t s, Tuning *best,
                        float *best_ms) {
    spiir_bank tmp;
    spiir_status st = build_bank(desc, tn, s, &tmp);
    float ms = 0.f;
    if (!st) st = time_pushes(&tmp, desc, s, &ms);
    tmp.free_device();
    if (st == SPIIR_ENOMEM || st == SPIIR_EBUDGET || st == SPIIR_ECUDA) return st;
    if (!st && ms < *best_ms) {
        *best_ms = ms;
        *best = tn;
    }
    return SPIIR_OK;
}

// The autotuner (desc->tune == 1). Plain form: every compiled recursion
// variant (time tile, filters per lane, CTAs per SM it is built for), then
// for the fastest the time-segment length of the persistent queue (2048,
// 4096, 8192 base-rate samples) and then fewer resident CTAs per SM. Block
// form: the chunk length (128 or 256). Each candidate builds the bank and
// times pushes of zeros of the bank's own push length.
spiir_status autotune(const spiir_bank_desc *desc, cudaStream_t s, Tuning *best) {
    float best_ms = 1e30f;
    spiir_status st;
    if (desc->mode != SPIIR_PLAIN_FP32) {
        best->chunk_len = desc->chunk_len ? desc->chunk_len : 256;
        for (int Lc : {256, 128}) {
            if (desc->block_len % Lc) continue;
            Tuning tn;
            tn.chunk_len = Lc;
            if ((st = try_tuning(desc, tn, s, best, &best_ms))) return st;
        }
        return SPIIR_OK;
    }
    *best = Tuning();
    best->variant = default_variant(desc);
    const int nv = spiir_recur_variant_count();
    for (int v = 0; v < nv; ++v) {
        Tuning tn;
        tn.variant = v;
        if ((st = try_tuning(desc, tn, s, best, &best_ms))) return st;
    }
    for (int sb : {2048, 8192}) {
        Tuning tn = *best;
        tn.seg_base = sb;
        if ((st = try_tuning(desc, tn, s, best, &best_ms))) return st;
    }
    int occ = 1;
    {
        Plan p;
        if (make_plan(desc, best->variant, false, p, nullptr, best->seg_base) == SPIIR_OK)
            spiir_recur_prepare(best->variant, p.smem_bytes, &occ);
    }
    for (int c = occ - 1; c >= 1 && c >= occ - 2; --c) {
        Tuning tn = *best;
        tn.ctas = c;
        if ((st = try_tuning(desc, tn, s, best, &best_ms))) return st;
    }
    return SPIIR_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

spiir_status spiir_bank_create(const spiir_bank_desc *desc, void *cuda_stream, spiir_bank_t *out) {
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    spiir_status st = validate(desc);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Tuning tn;
    tn.variant = chosen_variant(desc);
    float tune_ms = 0.f;
    if (desc->tune > 0) {
        const auto t0 = std::chrono::steady_clock::now();
        if ((st = autotune(desc, s, &tn))) return st;
        tune_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    spiir_bank *b = new (std::nothrow) spiir_bank();
    if (!b) return fail(SPIIR_ENOMEM, "host allocation failed");
    cudaGetDevice(&b->device);
    b->tune_ms = tune_ms;
    st = build_bank(desc, tn, s, b);
    if (st) {
        b->free_device();
        delete b;
        return st;
    }
    *out = b;
    g_err.clear();
    return SPIIR_OK;
}

// Makes stream s wait until no asynchronous copy-back still reads ring
// columns that overlap [lo, hi).
static spiir_status fence_ring(spiir_bank *b, cudaStream_t s, int64_t lo, int64_t hi) {
    for (int h = 0; h < 2; ++h)
        if (b->half_hi[h] > lo && b->half_lo[h] < hi)
            for (cudaEvent_t e : b->half_free[h])
                if (e) CUDA_TRY(cudaStreamWaitEvent(s, e, 0));
    return SPIIR_OK;
}

spiir_status spiir_push_block(spiir_bank_t b, int32_t stream_id, const float *x_dev,
                              int64_t n_samples, void *cuda_stream) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (!x_dev) return fail(SPIIR_EINVAL, "x_dev is NULL");
    if (stream_id < -1 || stream_id >= b->d.n_streams)
        return fail(SPIIR_EINVAL, "stream_id %d out of range", stream_id);
    if (n_samples <= 0 || n_samples % b->d.block_len != 0 ||
        n_samples > (int64_t)b->d.block_len * b->d.max_push_blocks)
        return fail(SPIIR_EINVAL, "n_samples must be a positive multiple of block_len, at most "
                                  "block_len * max_push_blocks");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int s0 = stream_id < 0 ? 0 : stream_id;
    const int cnt = stream_id < 0 ? b->d.n_streams : 1;
    if (spiir_status st = fence_ring(b, s, 0, n_samples)) return st;
    for (int q = s0; q < s0 + cnt; ++q) b->ring_base[q] = 0;
    if (b->tc) {
        spiir_status st = push_tc(b, s0, cnt, x_dev, n_samples, s, 0);
        if (st) return st;
        for (int q = s0; q < s0 + cnt; ++q) {
            b->last_n[q] = b->ring_n[q] = n_samples;
            b->out_valid[q] = 1;
        }
        return SPIIR_OK;
    }
    bool same = true;
    for (int q = s0; q < s0 + cnt; ++q) same &= (b->last_n[q] == b->last_n[s0]);
    if (same) {
        spiir_status st = push_plain(b, s0, cnt, x_dev, n_samples, n_samples, s);
        if (st) return st;
    } else {
        for (int q = 0; q < cnt; ++q) {
            spiir_status st = push_plain(b, s0 + q, 1, x_dev + q * n_samples, n_samples, n_samples, s);
            if (st) return st;
        }
    }
    for (int q = s0; q < s0 + cnt; ++q) {
        b->ring_n[q] = n_samples;
        b->out_valid[q] = 1;
    }
    return SPIIR_OK;
}

spiir_status spiir_read_snr(spiir_bank_t b, int32_t stream_id, void *z_dev, int64_t n_samples,
                            void *cuda_stream) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (!z_dev) return fail(SPIIR_EINVAL, "z_dev is NULL");
    if (stream_id < -1 || stream_id >= b->d.n_streams)
        return fail(SPIIR_EINVAL, "stream_id %d out of range", stream_id);
    const int s0 = stream_id < 0 ? 0 : stream_id;
    const int cnt = stream_id < 0 ? b->d.n_streams : 1;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    for (int q = s0; q < s0 + cnt; ++q) {
        if (b->last_n[q] == 0) return fail(SPIIR_ESTATE, "nothing pushed on stream %d", q);
        if (!b->out_valid[q])
            return fail(SPIIR_ESTATE, "no push on stream %d since its state was imported", q);
        if (n_samples <= 0 || n_samples > b->ring_n[q])
            return fail(SPIIR_EINVAL, "n_samples must be in [1, samples of the last push]");
    }
    const int T = b->d.n_templates;
    for (int q = s0; q < s0 + cnt; ++q) {
        const float2 *src;
        int64_t ring;
        if (b->tc) {
            src = spiir_tc_output(b->tc, q, &ring);
        } else {
            ring = b->p.ring_len;
            src = b->z + (int64_t)q * T * ring;
        }
        src += b->ring_base[q] + b->ring_n[q] - n_samples;
        char *dst = (char *)z_dev + (int64_t)(q - s0) * T * n_samples * sizeof(float2);
        CUDA_TRY(cudaMemcpy2DAsync(dst, n_samples * sizeof(float2), src, ring * sizeof(float2),
                                   n_samples * sizeof(float2), T, cudaMemcpyDeviceToDevice, s));
    }
    return SPIIR_OK;
}

spiir_status spiir_state_reset(spiir_bank_t b, int32_t stream_id, void *cuda_stream) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (stream_id < -1 || stream_id >= b->d.n_streams)
        return fail(SPIIR_EINVAL, "stream_id %d out of range", stream_id);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int s0 = stream_id < 0 ? 0 : stream_id;
    const int cnt = stream_id < 0 ? b->d.n_streams : 1;
    if (b->tc) {
        spiir_status st = spiir_tc_reset(b->tc, s0, cnt, s);
        if (st) return fail(st, "%s", spiir_tc_last_error());
    } else {
        const Plan &p = b->p;
        if (p.n_slots)
            CUDA_TRY(cudaMemsetAsync(b->state + (int64_t)s0 * p.n_slots, 0,
                                     cnt * p.n_slots * sizeof(float2), s));
        CUDA_TRY(cudaMemsetAsync(b->xbuf + (int64_t)s0 * p.xbuf_stream_stride, 0,
                                 cnt * p.xbuf_stream_stride * sizeof(float), s));
        if (b->ubuf)
            CUDA_TRY(cudaMemsetAsync(b->ubuf + (int64_t)s0 * p.ubuf_stream_stride, 0,
                                     cnt * p.ubuf_stream_stride * sizeof(float2), s));
    }
    for (int q = s0; q < s0 + cnt; ++q) {
        b->last_n[q] = b->ring_n[q] = b->ring_base[q] = 0;
        b->out_valid[q] = 0;
    }
    return SPIIR_OK;
}

// State blob: a header, then one record per stream: the length of its last
// push, the filter states in filter order (plain: FP32 {re, im}; tensor-core:
// FP64 {re, im}), the strain history (xbuf) and, for the plain form, the
// upsampler histories (ubuf).
struct StateHeader {
    char magic[8];
    uint32_t form, n_streams;
    uint64_t fingerprint;
    int64_t n_filters, xbuf_len, ubuf_len, elem_bytes;
};
constexpr char kStateMagic[8] = {'S', 'P', 'I', 'I', 'R', 'S', 'T', '1'};

static void state_shape(spiir_bank_t b, StateHeader &h) {
    std::memcpy(h.magic, kStateMagic, 8);
    h.form = b->tc ? 1u : 0u;
    h.fingerprint = b->fingerprint;
    h.n_filters = b->n_filters;
    h.xbuf_len = b->tc ? spiir_tc_xbuf_len(b->tc) : b->p.xbuf_stream_stride;
    h.ubuf_len = b->tc ? 0 : b->p.ubuf_stream_stride;
    h.elem_bytes = b->tc ? 16 : 8;
}

static int64_t state_record_bytes(const StateHeader &h) {
    return 8 + h.n_filters * h.elem_bytes + h.xbuf_len * 4 + h.ubuf_len * 8;
}

int64_t spiir_state_bytes(spiir_bank_t b, int32_t stream_id) {
    if (!b || stream_id < -1 || stream_id >= b->d.n_streams) return -1;
    StateHeader h;
    state_shape(b, h);
    const int cnt = stream_id < 0 ? b->d.n_streams : 1;
    return (int64_t)sizeof(StateHeader) + cnt * state_record_bytes(h);
}

spiir_status spiir_state_export(spiir_bank_t b, int32_t stream_id, void *dst, int64_t bytes,
                                void *cuda_stream) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (!dst) return fail(SPIIR_EINVAL, "dst is NULL");
    if (stream_id < -1 || stream_id >= b->d.n_streams)
        return fail(SPIIR_EINVAL, "stream_id %d out of range", stream_id);
    if (bytes < spiir_state_bytes(b, stream_id))
        return fail(SPIIR_EINVAL, "buffer of %lld bytes, %lld needed", (long long)bytes,
                    (long long)spiir_state_bytes(b, stream_id));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int s0 = stream_id < 0 ? 0 : stream_id;
    const int cnt = stream_id < 0 ? b->d.n_streams : 1;
    StateHeader h;
    state_shape(b, h);
    h.n_streams = (uint32_t)cnt;
    char *out = (char *)dst;
    std::memcpy(out, &h, sizeof h);
    out += sizeof h;
    for (int q = s0; q < s0 + cnt; ++q) {
        int64_t last_n = b->last_n[q];
        char *rec = out;
        out += state_record_bytes(h);
        double *v64 = nullptr;
        float2 *v32 = nullptr;
        float *xb = (float *)(rec + 8 + h.n_filters * h.elem_bytes);
        if (b->tc) {
            v64 = (double *)(rec + 8);
            spiir_status st = spiir_tc_state_get(b->tc, q, v64, xb, &last_n, s);
            if (st) return fail(st, "%s", spiir_tc_last_error());
        } else {
            const Plan &p = b->p;
            std::vector<float2> raw(p.n_slots);
            if (p.n_slots)
                CUDA_TRY(cudaMemcpyAsync(raw.data(), b->state + (int64_t)q * p.n_slots,
                                         p.n_slots * sizeof(float2), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaMemcpyAsync(xb, b->xbuf + (int64_t)q * p.xbuf_stream_stride,
                                     p.xbuf_stream_stride * sizeof(float), cudaMemcpyDeviceToHost, s));
            if (h.ubuf_len)
                CUDA_TRY(cudaMemcpyAsync(xb + h.xbuf_len, b->ubuf + (int64_t)q * p.ubuf_stream_stride,
                                         p.ubuf_stream_stride * sizeof(float2), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            v32 = (float2 *)(rec + 8);
            for (int64_t sl = 0; sl < p.n_slots; ++sl)
                if (p.slot_filter[sl] >= 0) v32[p.slot_filter[sl]] = raw[sl];
        }
        std::memcpy(rec, &last_n, 8);
    }
    return SPIIR_OK;
}

spiir_status spiir_state_import(spiir_bank_t b, int32_t stream_id, const void *src, int64_t bytes,
                                void *cuda_stream) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (!src) return fail(SPIIR_EINVAL, "src is NULL");
    if (stream_id < -1 || stream_id >= b->d.n_streams)
        return fail(SPIIR_EINVAL, "stream_id %d out of range", stream_id);
    const int s0 = stream_id < 0 ? 0 : stream_id;
    const int cnt = stream_id < 0 ? b->d.n_streams : 1;
    StateHeader want, got;
    state_shape(b, want);
    if (bytes < (int64_t)sizeof got) return fail(SPIIR_EINVAL, "state blob too short");
    std::memcpy(&got, src, sizeof got);
    if (std::memcmp(got.magic, kStateMagic, 8) != 0) return fail(SPIIR_EINVAL, "not a state blob");
    if (got.form != want.form || got.fingerprint != want.fingerprint || got.n_filters != want.n_filters ||
        got.xbuf_len != want.xbuf_len || got.ubuf_len != want.ubuf_len || got.elem_bytes != want.elem_bytes)
        return fail(SPIIR_EINVAL, "state blob of another bank description or form");
    if ((int)got.n_streams != cnt)
        return fail(SPIIR_EINVAL, "blob holds %u streams, %d requested", got.n_streams, cnt);
    if (bytes < (int64_t)sizeof got + cnt * state_record_bytes(got))
        return fail(SPIIR_EINVAL, "state blob truncated");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const char *in = (const char *)src + sizeof got;
    for (int q = s0; q < s0 + cnt; ++q) {
        const char *rec = in;
        in += state_record_bytes(got);
        int64_t last_n;
        std::memcpy(&last_n, rec, 8);
        if (last_n < 0 || last_n > (int64_t)b->d.block_len * b->d.max_push_blocks ||
            last_n % b->d.block_len != 0)
            return fail(SPIIR_EINVAL, "state blob: bad push length");
        const float *xb = (const float *)(rec + 8 + got.n_filters * got.elem_bytes);
        if (b->tc) {
            spiir_status st = spiir_tc_state_set(b->tc, q, (const double *)(rec + 8), xb, last_n, s);
            if (st) return fail(st, "%s", spiir_tc_last_error());
        } else {
            const Plan &p = b->p;
            const float2 *v32 = (const float2 *)(rec + 8);
            std::vector<float2> raw(p.n_slots, make_float2(0.f, 0.f));
            for (int64_t sl = 0; sl < p.n_slots; ++sl)
                if (p.slot_filter[sl] >= 0) raw[sl] = v32[p.slot_filter[sl]];
            if (p.n_slots)
                CUDA_TRY(cudaMemcpyAsync(b->state + (int64_t)q * p.n_slots, raw.data(),
                                         p.n_slots * sizeof(float2), cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(b->xbuf + (int64_t)q * p.xbuf_stream_stride, xb,
                                     p.xbuf_stream_stride * sizeof(float), cudaMemcpyHostToDevice, s));
            if (got.ubuf_len)
                CUDA_TRY(cudaMemcpyAsync(b->ubuf + (int64_t)q * p.ubuf_stream_stride, xb + got.xbuf_len,
                                         p.ubuf_stream_stride * sizeof(float2), cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaStreamSynchronize(s));
        }
        b->last_n[q] = last_n;
        b->ring_n[q] = b->ring_base[q] = 0;
        b->out_valid[q] = 0;
    }
    return SPIIR_OK;
}

spiir_status spiir_read_snr_abs(spiir_bank_t b, int32_t stream_id, float *out_dev, int64_t n_samples,
                                const float *norm_dev, void *cuda_stream) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (!out_dev) return fail(SPIIR_EINVAL, "out_dev is NULL");
    if (stream_id < -1 || stream_id >= b->d.n_streams)
        return fail(SPIIR_EINVAL, "stream_id %d out of range", stream_id);
    const int s0 = stream_id < 0 ? 0 : stream_id;
    const int cnt = stream_id < 0 ? b->d.n_streams : 1;
    for (int q = s0; q < s0 + cnt; ++q) {
        if (b->last_n[q] == 0) return fail(SPIIR_ESTATE, "nothing pushed on stream %d", q);
        if (!b->out_valid[q])
            return fail(SPIIR_ESTATE, "no push on stream %d since its state was imported", q);
        if (n_samples <= 0 || n_samples > b->ring_n[q])
            return fail(SPIIR_EINVAL, "n_samples must be in [1, samples of the last push]");
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int T = b->d.n_templates;
    for (int q = s0; q < s0 + cnt; ++q) {
        const float2 *src;
        int64_t ring;
        if (b->tc) {
            src = spiir_tc_output(b->tc, q, &ring);
        } else {
            ring = b->p.ring_len;
            src = b->z + (int64_t)q * T * ring;
        }
        CUDA_TRY(spiir_launch_abs(src + b->ring_base[q] + b->ring_n[q] - n_samples, ring, T, n_samples, norm_dev,
                                  out_dev + (int64_t)(q - s0) * T * n_samples, s));
    }
    return SPIIR_OK;
}

// The host-buffer push behind spiir_push_block_host (async = false: returns
// once z_host holds the SNR) and spiir_push_block_host_async (returns once
// the work is queued; the push goes into the ring half the previous
// asynchronous push did not use when the ring holds two pushes, so its
// kernels run while that push's SNR is still being copied out).
static spiir_status host_push(spiir_bank_t b, int32_t stream_id, const float *x_host, int64_t n_samples,
                       void *z_host, cudaStream_t s, bool async) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (!x_host || !z_host) return fail(SPIIR_EINVAL, "host buffers must not be NULL");
    if (stream_id < -1 || stream_id >= b->d.n_streams)
        return fail(SPIIR_EINVAL, "stream_id %d out of range", stream_id);
    if (n_samples <= 0 || n_samples % b->d.block_len != 0 ||
        n_samples > (int64_t)b->d.block_len * b->d.max_push_blocks)
        return fail(SPIIR_EINVAL, "bad n_samples");
    const int s0 = stream_id < 0 ? 0 : stream_id;
    const int cnt = stream_id < 0 ? b->d.n_streams : 1;
    const int T = b->d.n_templates;
    int64_t ring_len = b->p.ring_len;
    if (b->tc) spiir_tc_output(b->tc, 0, &ring_len);
    const bool two = async && ring_len >= 2 * n_samples;
    const int half = two ? b->async_half : 0;
    const int64_t base = half ? n_samples : 0;    // first ring column of this push
    // A push of several blocks runs as up to four pieces of whole blocks.
    // Piece i writes output-ring columns [base + off_i, base + off_i + n_i)
    // (pushes compose exactly: block-split invariance), and its SNR is copied
    // back while piece i + 1 computes, the template rows split over two copy
    // streams (two copy engines: one device-to-host stream does not fill the
    // link). The ring then holds the whole push, as after one push of n_samples.
    const int64_t n_blocks = n_samples / b->d.block_len;
    const int n_pieces = (int)std::min<int64_t>(4, n_blocks);
    if (!b->copy[0]) {
        for (auto &c : b->copy) CUDA_TRY(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
        for (auto &e : b->piece_done) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto &h : b->half_free)
            for (auto &e : h) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // no earlier asynchronous copy-back may still read what this push writes
    if (spiir_status st = fence_ring(b, s, base, base + n_samples)) return st;
    int64_t off = 0;
    for (int i = 0; i < n_pieces; ++i) {
        bool same = true;
        for (int q = s0; q < s0 + cnt; ++q) same &= (b->last_n[q] == b->last_n[s0]);
        const int64_t n_i = (n_blocks * (i + 1) / n_pieces - n_blocks * i / n_pieces) * b->d.block_len;
        // strain of this piece, [cnt][n_i], into the staging buffer (the
        // plain form's graphs read it there; stream order keeps the previous
        // piece's kernels ahead of the overwrite)
        float *stage = b->tc ? spiir_tc_stage(b->tc) : b->xstage + (int64_t)s0 * n_i;
        CUDA_TRY(cudaMemcpy2DAsync(stage, n_i * sizeof(float), x_host + off, n_samples * sizeof(float),
                                   n_i * sizeof(float), cnt, cudaMemcpyHostToDevice, s));
        if (b->tc) {
            spiir_status st = push_tc(b, s0, cnt, stage, n_i, s, base + off);
            if (st) return st;
            for (int q = s0; q < s0 + cnt; ++q) b->last_n[q] = n_i;
        } else if (same) {
            spiir_status st = push_plain(b, s0, cnt, stage, n_i, n_i, s, false, base + off);
            if (st) return st;
        } else {
            for (int q = 0; q < cnt; ++q) {
                spiir_status st = push_plain(b, s0 + q, 1, stage + q * n_i, n_i, n_i, s, false, base + off);
                if (st) return st;
            }
        }
        const int n_cs = 2;
        CUDA_TRY(cudaEventRecord(b->piece_done[i], s));
        for (auto &c : b->copy) CUDA_TRY(cudaStreamWaitEvent(c, b->piece_done[i], 0));
        for (int q = s0; q < s0 + cnt; ++q) {
            const float2 *src;
            int64_t ring;
            if (b->tc) {
                src = spiir_tc_output(b->tc, q, &ring);
            } else {
                ring = b->p.ring_len;
                src = b->z + (int64_t)q * T * ring;
            }
            for (int h = 0; h < n_cs; ++h) {
                const int r0 = T * h / n_cs, r1 = T * (h + 1) / n_cs;
                if (r1 <= r0) continue;
                char *dst = (char *)z_host + ((int64_t)(q - s0) * T * n_samples + (int64_t)r0 * n_samples + off) *
                                                 sizeof(float2);
                CUDA_TRY(cudaMemcpy2DAsync(dst, n_samples * sizeof(float2), src + (int64_t)r0 * ring + base + off,
                                           ring * sizeof(float2), n_i * sizeof(float2), r1 - r0,
                                           cudaMemcpyDeviceToHost, b->copy[h]));
            }
        }
        off += n_i;
    }
    for (int q = s0; q < s0 + cnt; ++q) {
        b->ring_n[q] = n_samples;
        b->ring_base[q] = base;
        b->out_valid[q] = 1;
    }
    if (async) {
        for (int c = 0; c < 2; ++c) CUDA_TRY(cudaEventRecord(b->half_free[half][c], b->copy[c]));
        b->half_lo[half] = base;
        b->half_hi[half] = base + n_samples;
        if (two) b->async_half ^= 1;
        return SPIIR_OK;
    }
    for (auto &c : b->copy)
        if (c) CUDA_TRY(cudaStreamSynchronize(c));
    CUDA_TRY(cudaStreamSynchronize(s));
    // every copy-back, asynchronous ones included, has finished
    b->half_lo[0] = b->half_hi[0] = b->half_lo[1] = b->half_hi[1] = 0;
    return SPIIR_OK;
}

spiir_status spiir_push_block_host(spiir_bank_t b, int32_t stream_id, const float *x_host,
                                   int64_t n_samples, void *z_host, void *cuda_stream) {
    return host_push(b, stream_id, x_host, n_samples, z_host, (cudaStream_t)cuda_stream, false);
}

spiir_status spiir_push_block_host_async(spiir_bank_t b, int32_t stream_id, const float *x_host,
                                         int64_t n_samples, void *z_host, void *cuda_stream) {
    return host_push(b, stream_id, x_host, n_samples, z_host, (cudaStream_t)cuda_stream, true);
}

spiir_status spiir_bank_host_sync(spiir_bank_t b) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    for (auto &c : b->copy)
        if (c) CUDA_TRY(cudaStreamSynchronize(c));
    b->half_lo[0] = b->half_hi[0] = b->half_lo[1] = b->half_hi[1] = 0;
    return SPIIR_OK;
}

int64_t spiir_bank_footprint(const spiir_bank_desc *desc) {
    if (validate(desc)) return -1;
    if (desc->mode != SPIIR_PLAIN_FP32) return spiir_tc_footprint(desc);
    Plan p;
    if (make_plan(desc, chosen_variant(desc), false, p)) return -1;
    return plan_footprint(desc, p);
}

spiir_status spiir_bank_plan(const spiir_bank_desc *desc, spiir_bank_info *info) {
    if (!info) return fail(SPIIR_EINVAL, "info is NULL");
    spiir_status st = validate(desc);
    if (st) return st;
    if (desc->mode != SPIIR_PLAIN_FP32) return fail(SPIIR_EUNSUPPORTED, "plan of the plain form only");
    Plan p;
    if ((st = make_plan(desc, chosen_variant(desc), true, p))) return st;
    std::memset(info, 0, sizeof(*info));
    info->footprint_bytes = plan_footprint(desc, p);
    plan_info(desc, p, info);
    return SPIIR_OK;
}

spiir_status spiir_bank_get_info(spiir_bank_t b, spiir_bank_info *info) {
    if (!b || !info) return fail(SPIIR_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->footprint_bytes = b->footprint;
    if (b->tc) {
        spiir_tc_info(b->tc, info);
        info->tune_ms = b->tune_ms;
        info->graph_captured = b->graphs.empty() ? 0 : 1;
        return SPIIR_OK;
    }
    plan_info(&b->d, b->p, info);
    info->slot_fill = b->p.n_slots ? (float)b->n_filters / (float)b->p.n_slots : 1.f;
    info->graph_captured = b->graphs.empty() ? 0 : 1;
    info->segment_base = b->p.seg_base;
    info->ctas_per_sm = b->ctas_cap > 0 ? std::min(b->ctas_cap, b->ctas_per_sm) : b->ctas_per_sm;
    info->tune_ms = b->tune_ms;
    return SPIIR_OK;
}

spiir_status spiir_bank_sync_status(spiir_bank_t b) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    CUDA_TRY(cudaDeviceSynchronize());
    unsigned int *dst = b->tc ? spiir_tc_status(b->tc) : b->status;
    unsigned int v = 0;
    CUDA_TRY(cudaMemcpy(&v, dst, sizeof(v), cudaMemcpyDeviceToHost));
    if (v != SPIIR_DEV_OK) {
        CUDA_TRY(cudaMemset(dst, 0, sizeof(unsigned int)));
        return fail(SPIIR_ETIMEOUT, "a device-side wait timed out (status %u)", v);
    }
    return SPIIR_OK;
}

spiir_status spiir_bank_test_stall(spiir_bank_t b, const float *x_dev, int64_t n_samples,
                                   void *cuda_stream) {
    if (!b || !x_dev) return fail(SPIIR_EINVAL, "NULL argument");
    if (b->tc) return fail(SPIIR_EUNSUPPORTED, "stall test runs on the plain form");
    if (n_samples < 8192 || n_samples % b->d.block_len != 0 ||
        n_samples > (int64_t)b->d.block_len * b->d.max_push_blocks)
        return fail(SPIIR_EINVAL, "stall test needs a push of at least two 4096-sample segments");
    return push_plain(b, 0, 1, x_dev, n_samples, n_samples, (cudaStream_t)cuda_stream, true);
}

spiir_status spiir_bank_enable_timing(spiir_bank_t b, int32_t enable) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    b->timer->flush();
    b->timer->on = enable != 0;
    for (int k = 0; k < SPIIR_K_COUNT; ++k) {
        b->timer->ms[k] = 0.0;
        b->timer->launches[k] = 0;
    }
    return SPIIR_OK;
}

spiir_status spiir_bank_kernel_times(spiir_bank_t b, spiir_kernel_times *out) {
    if (!b || !out) return fail(SPIIR_EINVAL, "NULL argument");
    b->timer->flush();
    for (int k = 0; k < SPIIR_K_COUNT; ++k) {
        out->ms[k] = b->timer->ms[k];
        out->launches[k] = b->timer->launches[k];
        b->timer->ms[k] = 0.0;
        b->timer->launches[k] = 0;
    }
    return SPIIR_OK;
}

void spiir_bank_destroy(spiir_bank_t b) {
    if (!b) return;
    cudaDeviceSynchronize();
    b->free_device();
    delete b;
}

spiir_status spiir_kaiser_taps(int32_t n_taps, double atten_db, float *out) {
    if (!out || n_taps < 2 || n_taps > 4096) return fail(SPIIR_EINVAL, "bad n_taps or out");
    lib_kaiser_taps(n_taps, atten_db, out);
    return SPIIR_OK;
}

int32_t spiir_assign_level(float a_re, float a_im, int32_t base_rate, int32_t n_levels) {
    return spiir_assign_level_margin(a_re, a_im, base_rate, n_levels, 0.f);
}

int32_t spiir_assign_level_margin(float a_re, float a_im, int32_t base_rate, int32_t n_levels,
                                  float margin) {
    if (!(margin >= 0.f) || !std::isfinite(margin) || n_levels < 1 || n_levels > 30 || base_rate <= 0)
        return -1;
    const double f = std::fabs(std::atan2((double)a_im, (double)a_re)) * base_rate / (2.0 * M_PI);
    const double need = 2.0 * f * (1.0 + (double)margin);
    int32_t lv = 0;
    for (int32_t i = 0; i < n_levels; ++i)
        if ((double)base_rate / (double)(1 << i) >= need) lv = i;
    return lv;
}

const char *spiir_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// One-shot filtering without device allocation (spiir_filter_noalloc).
//
// Some callers cannot call cudaMalloc: a host framework that hands the
// library a real-time thread on which device allocation is forbidden (an
// allocation can block on the driver for an unbounded time), or a process
// whose device memory is carved up in advance by someone else, so that any
// allocation outside its own pools fails. This entry point serves them: all
// the device memory it needs lives in one file-scope __device__ array of
// fixed size, which the module reserves on every GPU that loads the library
// and keeps until the process exits.
// ---------------------------------------------------------------------------

#define SPIIR_NOALLOC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_spiir_noalloc_scratch[SPIIR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
// Per-device address of the scratch array, filled in by the first call on
// that device. Atomic so that first calls from several host threads do not
// race; two of them may both look the address up, which is harmless.
std::atomic<void *> g_noalloc_ptr[kMaxDevices] = {};
KernelTimer g_noalloc_timer;  // stays off: pushes record no events

// Device address of the scratch array on the current device. The array's
// name is only a host-side stand-in; the address comes from the runtime, once
// per device, with that device current.
spiir_status noalloc_scratch(void **out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SPIIR_EUNSUPPORTED, "device %d out of range", dev);
    void *p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        CUDA_TRY(cudaGetSymbolAddress(&p, g_spiir_noalloc_scratch));
        g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return SPIIR_OK;
}

struct Carve {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

template <typename T>
spiir_status put(T *dst, const std::vector<T> &src, cudaStream_t s) {
    if (src.empty()) return SPIIR_OK;
    CUDA_TRY(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return SPIIR_OK;
}

}  // namespace

extern "C" spiir_status spiir_filter_noalloc(const spiir_bank_desc *desc, const float *x_dev,
                                             int64_t n_samples, void *z_dev, void *cuda_stream) {
    if (!x_dev || !z_dev) return fail(SPIIR_EINVAL, "x_dev and z_dev must not be NULL");
    if (!desc) return fail(SPIIR_EINVAL, "desc is NULL");
    if (desc->mode != SPIIR_PLAIN_FP32)
        return fail(SPIIR_EUNSUPPORTED, "spiir_filter_noalloc runs the plain FP32 form only");
    if (desc->n_streams != 1) return fail(SPIIR_EINVAL, "spiir_filter_noalloc takes one stream");
    if (desc->n_levels < 1 || desc->n_levels > SPIIR_MAX_LEVELS)
        return fail(SPIIR_EINVAL, "n_levels must be in [1, %d]", SPIIR_MAX_LEVELS);
    const int H = desc->n_levels - 1;
    if (n_samples <= 0 || n_samples % (4ll << H) != 0 || n_samples > (1ll << 30))
        return fail(SPIIR_EINVAL, "n_samples must be a positive multiple of 4*2^(n_levels-1)");

    // Plan for one push of n_samples from zero state: the description's
    // block_len, max_push_blocks and autotuning request are replaced before
    // it is validated, so a caller need not fill them in.
    spiir_bank_desc d = *desc;
    d.block_len = (int32_t)n_samples;
    d.max_push_blocks = 1;
    d.tune = desc->tune < 0 ? desc->tune : 0;
    spiir_status st = validate(&d);
    if (st) return st;
    spiir_bank b;
    b.d = d;
    b.n_filters = d.n_filters;
    if ((st = make_plan(&d, chosen_variant(&d), true, b.p))) return st;
    const Plan &p = b.p;

    // Size check before any device work.
    size_t need = 0;
    {
        Carve c{nullptr};
        c.take<float>(p.n_slots);
        c.take<float>(p.n_slots);
        c.take<float>(p.n_slots);
        c.take<float>(p.n_slots);
        c.take<int32_t>(p.n_slots);
        c.take<WarpTask>(p.tasks.size());
        c.take<CtaItem>(p.items.size());
        c.take<int32_t>(p.task_out.size());
        c.take<int32_t>(p.comb_ptr.size());
        c.take<int32_t>(p.comb_rows.size());
        c.take<int32_t>(p.order.size());
        c.take<unsigned int>(1);
        c.take<unsigned int>(std::max<size_t>(1, p.items.size()));
        c.take<float2>(std::max<int64_t>(1, p.n_slots));
        c.take<float>(p.xbuf_stream_stride);
        c.take<float2>(p.part_stream_stride);
        c.take<float2>(p.ubuf_stream_stride);
        c.take<unsigned int>(1);
        need = c.off;
    }
    if (need > SPIIR_NOALLOC_SCRATCH_BYTES)
        return fail(SPIIR_EINVAL,
                    "spiir_filter_noalloc: this bank and length need %zu bytes of scratch, above "
                    "the fixed %u bytes; use spiir_bank_create instead",
                    need, (unsigned)SPIIR_NOALLOC_SCRATCH_BYTES);

    void *base = nullptr;
    if ((st = noalloc_scratch(&base))) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Carve c{static_cast<char *>(base)};
    b.are = c.take<float>(p.n_slots);
    b.aim = c.take<float>(p.n_slots);
    b.bre = c.take<float>(p.n_slots);
    b.bim = c.take<float>(p.n_slots);
    b.xoff = c.take<int32_t>(p.n_slots);
    b.tasks = c.take<WarpTask>(p.tasks.size());
    b.items = c.take<CtaItem>(p.items.size());
    b.task_out = c.take<int32_t>(p.task_out.size());
    b.comb_ptr = c.take<int32_t>(p.comb_ptr.size());
    b.comb_rows = c.take<int32_t>(p.comb_rows.size());
    b.order = c.take<int32_t>(p.order.size());
    b.queue = c.take<unsigned int>(1);
    b.prog = c.take<unsigned int>(std::max<size_t>(1, p.items.size()));
    b.state = c.take<float2>(std::max<int64_t>(1, p.n_slots));
    b.xbuf = c.take<float>(p.xbuf_stream_stride);
    b.partial = p.part_stream_stride ? c.take<float2>(p.part_stream_stride) : nullptr;
    b.ubuf = p.ubuf_stream_stride ? c.take<float2>(p.ubuf_stream_stride) : nullptr;
    b.status = c.take<unsigned int>(1);
    b.z = static_cast<float2 *>(z_dev);   // row stride p.ring_len == n_samples

    if ((st = put(b.are, p.are, s)) || (st = put(b.aim, p.aim, s)) || (st = put(b.bre, p.bre, s)) ||
        (st = put(b.bim, p.bim, s)) || (st = put(b.xoff, p.xoff, s)) ||
        (st = put(b.tasks, p.tasks, s)) || (st = put(b.items, p.items, s)) ||
        (st = put(b.task_out, p.task_out, s)) || (st = put(b.comb_ptr, p.comb_ptr, s)) ||
        (st = put(b.comb_rows, p.comb_rows, s)) || (st = put(b.order, p.order, s)))
        return st;
    // The array keeps the previous call's contents: zero the state, the strain
    // history, the upsampler history and the status word.
    CUDA_TRY(cudaMemsetAsync(b.state, 0, std::max<int64_t>(1, p.n_slots) * sizeof(float2), s));
    CUDA_TRY(cudaMemsetAsync(b.xbuf, 0, p.xbuf_stream_stride * sizeof(float), s));
    if (b.ubuf) CUDA_TRY(cudaMemsetAsync(b.ubuf, 0, p.ubuf_stream_stride * sizeof(float2), s));
    CUDA_TRY(cudaMemsetAsync(b.status, 0, sizeof(unsigned int), s));
    // Templates without filters are never written by the kernels.
    CUDA_TRY(cudaMemsetAsync(z_dev, 0, (size_t)d.n_templates * n_samples * sizeof(float2), s));
    CUDA_TRY(spiir_recur_prepare(p.variant, p.smem_bytes, &b.ctas_per_sm));
    if (p.need_combine) CUDA_TRY(spiir_combine_prepare());
    CUDA_TRY(cudaGetDevice(&b.device));
    CUDA_TRY(cudaDeviceGetAttribute(&b.n_sms, cudaDevAttrMultiProcessorCount, b.device));

    b.scale = desc->snr_scale != 0.f ? desc->snr_scale : 2.0f / (float)desc->base_rate;
    const int nt = d.n_taps ? d.n_taps : 32;
    const int ntu = d.n_taps_up ? d.n_taps_up : nt;
    b.d.n_taps = nt;
    b.d.n_taps_up = ntu;
    b.h_down.resize(nt);
    b.h_up.resize(ntu);
    if (desc->h_down) {
        std::copy(desc->h_down, desc->h_down + nt, b.h_down.begin());
        std::copy(desc->h_up, desc->h_up + ntu, b.h_up.begin());
    } else {
        lib_kaiser_taps(nt, 60.0, b.h_down.data());
        lib_kaiser_taps(ntu, 60.0, b.h_up.data());
    }
    b.last_n.assign(1, 0);
    b.ring_n.assign(1, 0);
    b.timer = &g_noalloc_timer;
    st = push_plain(&b, 0, 1, x_dev, n_samples, n_samples, s);
    // The bank object only borrows these pointers: clear them so that it
    // frees nothing when it goes out of scope.
    b.are = b.aim = b.bre = b.bim = nullptr;
    b.xoff = nullptr;
    b.tasks = nullptr;
    b.items = nullptr;
    b.task_out = b.comb_ptr = b.comb_rows = nullptr;
    b.state = b.partial = b.ubuf = b.z = nullptr;
    b.xbuf = nullptr;
    b.status = nullptr;
    b.order = nullptr;
    b.queue = b.prog = nullptr;
    b.timer = nullptr;
    return st;
}
