// spiir_server.cu -- many banks filtered together (spiir_server_* of
// include/spiir.h): the batched serving form of the SPIIR hot path.
//
// Every push runs one prologue (strain history update) and one decimation
// cascade for all members (Sec. 2.2), one persistent recursion launch over the
// work items of every member and level that runs in the plain form (Eqs.
// iireq0, iireq1), in the tensor-core modes one batched block-form launch
// sequence per level (and pair of streams) over every member's filters at
// that level, and one upsample-and-add launch over every member's templates;
// the launches are replayed from a CUDA graph while the membership is
// unchanged. Each member is planned like a bank of its own (make_plan with
// the server's strain history; spiir_tc_pack per block-form level) and placed
// in pooled device arrays:
//   * plain filter slots (pole, gain, window offset, state per stream),
//   * template rows (output ring, upsampler histories),
//   * partial rows per level (per-push scratch of the level sums), the
//     plain units' rows first, then 64 rows per impulse-response group,
//   * per block-form level: impulse-response groups (64 templates) and carry
//     tiles (128 filters: coefficients, power panel, FP64 state per stream);
// each pool hands out contiguous ranges first-fit, reuses the ranges of
// members that left, and grows geometrically (keeping every member's place
// and its state). The work lists (warp tasks, CTA items, queue order,
// destinations, group and carry lists, combine lists) are rebuilt on the host
// and uploaded whenever the membership changes; the kernels are the bank's.
//
// In the block form a level's alignment delay D_i (Sec. 2.2) is a delay of
// the strain the level reads (its window starts D_i samples earlier), so the
// FIR length stays the largest filter delay plus one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "spiir.h"
#include "spiir_internal.h"
#include "spiir_plan.h"
#include "spiir_tc.h"

using namespace spiir_host;

namespace {

// First-fit allocator of index ranges in [0, cap).
class RangeAlloc {
  public:
    int64_t cap() const { return cap_; }
    // Start of a free range of n indices, or -1 (n == 0 takes nothing).
    int64_t take(int64_t n) {
        if (n <= 0) return 0;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const int64_t s = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[s + n] = len - n;
                return s;
            }
        }
        return -1;
    }
    void give(int64_t s, int64_t n) {
        if (n <= 0) return;
        auto it = free_.emplace(s, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    // Capacity at which a range of n fits (extending a free tail if any).
    int64_t need_for(int64_t n) const {
        if (!free_.empty()) {
            auto last = std::prev(free_.end());
            if (last->first + last->second == cap_) return last->first + n;
        }
        return cap_ + n;
    }
    void grow(int64_t new_cap) {
        if (new_cap > cap_) {
            give(cap_, new_cap - cap_);
            cap_ = new_cap;
        }
    }

  private:
    std::map<int64_t, int64_t> free_;
    int64_t cap_ = 0;
};

// A device array that grows on demand (elements, not bytes).
template <typename T>
struct DevVec {
    T *p = nullptr;
    int64_t cap = 0;
    // At least n elements; the old contents are not kept. The old array is
    // freed once the work queued on s (which follows every push that read
    // it) has finished.
    spiir_status reserve(int64_t n, cudaStream_t s) {
        if (n <= cap) return SPIIR_OK;
        const int64_t c = std::max<int64_t>(n, cap + cap / 2);
        if (p) {
            CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(p);
        }
        p = nullptr;
        cap = 0;
        CUDA_TRY(cudaMalloc((void **)&p, std::max<int64_t>(1, c) * sizeof(T)));
        cap = c;
        return SPIIR_OK;
    }
    spiir_status upload(const std::vector<T> &v, cudaStream_t s) {
        spiir_status st = reserve((int64_t)v.size(), s);
        if (st) return st;
        if (!v.empty())
            CUDA_TRY(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        return SPIIR_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// A member's part at one block-form level.
struct MemberTc {
    bool used = false;           // some of the member's templates run this level in the block form
    std::vector<int32_t> row;    // per member template: its row among them, or -1 (plain form)
    int nT = 0;                  // templates routed to the block form
    int64_t g0 = 0, ng = 0;      // impulse-response groups
    int64_t t0 = 0, nt = 0;      // carry tiles
    TcPack pk;                   // host packing (only has_carry kept once uploaded)
};

struct Member {
    int id = 0;
    int T = 0;
    Plan p;                      // plan of the member's plain-form levels
    int64_t slot0 = 0;           // first pooled filter slot
    int64_t row0 = 0;            // first pooled template row
    int64_t prow0[SPIIR_MAX_LEVELS] = {};   // first pooled partial row per level
    MemberTc tc[SPIIR_MAX_LEVELS];
    bool combine = false;        // its templates go through the combine pass
    int64_t n_filters = 0;
    int64_t fs_per_push = 0;     // filter-samples of one push per stream
    bool pushed = false;         // has taken part in a push
};

// One block-form level of the server: pools and per-push lists.
struct TcPool {
    bool on = false;
    int hist_read = 0;           // strain history before the push, minus D_i
    RangeAlloc group_alloc, tile_alloc;
    uint4 *H = nullptr;          // [group][slice][16 KB]
    float *row_scale = nullptr;  // [group * 64 + r]
    uint8_t *has_carry = nullptr;
    int32_t *tile_ptr = nullptr, *tile_end = nullptr;
    float2 *a = nullptr, *aJ = nullptr, *c = nullptr, *aLf = nullptr;   // [tile * 128 + k]
    uint4 *aL = nullptr, *aLb1 = nullptr, *aLb2 = nullptr;
    uint4 *v = nullptr;          // [stream][tile * 128 + k]
    uint4 *panel = nullptr;      // [tile][32 KB]
    DevVec<int32_t> groups, tmpl_of;
    int n_groups = 0, n_carry = 0;
};

}  // namespace

struct spiir_server {
    spiir_server_desc d{};
    int S = 1, L = 1, H = 0, block = 0, variant = 0;
    float scale = 0.f;
    std::vector<float> h_down, h_up;
    Plan geo;                    // sizes of an empty member: strain layout,
                                 // segment lengths, partial strides, history
    int smem_bytes = 0, ctas_per_sm = 1, n_sms = 1;
    // block form
    bool tc_mode = false, bf16 = false, df = false;
    int tcL = 256, tcF = 0, tcK = 0, n_slices = 0, n_tc_levels = 0;
    int tc_min = 24;             // filters a template needs at a level to run it in the block form
    TcPool tcp[SPIIR_MAX_LEVELS];
    uint4 *hank = nullptr, *xseg = nullptr;
    // shared strain
    float *xbuf = nullptr, *xstage = nullptr;
    unsigned int *status = nullptr;
    // pools
    RangeAlloc slot_alloc, row_alloc, prow_alloc[SPIIR_MAX_LEVELS];
    float *are = nullptr, *aim = nullptr, *bre = nullptr, *bim = nullptr;
    int32_t *xoff = nullptr;
    float2 *state = nullptr;     // [stream][slot cap]
    float2 *z = nullptr;         // [stream][row cap][block]
    float2 *ubuf = nullptr;      // [stream][level 1..H][row cap][SPIIR_UHIST]
    float2 *partial = nullptr;   // [stream][level][rows][stride]
    int64_t part_base[SPIIR_MAX_LEVELS] = {}, part_stream_stride = 0;
    // work lists
    DevVec<WarpTask> tasks;
    DevVec<CtaItem> items;
    DevVec<int32_t> order, task_out, comb_ptr, comb_rows, comb_list;
    DevVec<unsigned int> queue, prog;
    int n_items = 0, n_comb = 0, n_tasks = 0;
    // members
    std::map<int, Member> members;
    std::vector<Member> pending_add;
    std::vector<int> pending_remove;
    int next_id = 0;
    bool dirty = false;
    int64_t pushes = 0;
    // graph of one push (by previous push length: 0 for the first)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int launches = 0;
    // membership changes run on io after the last push (ev_push) and the
    // next push waits for them (ev_io)
    cudaStream_t io = nullptr;
    cudaEvent_t ev_push = nullptr, ev_io = nullptr;
    bool pushed_once = false, io_pending = false;
    KernelTimer *timer = nullptr;

    // rows of partial level i before its block-form rows
    int64_t tc_row_base(int i) const { return prow_alloc[i].cap(); }
    int64_t level_rows(int i) const { return prow_alloc[i].cap() + 64 * tcp[i].group_alloc.cap(); }

    void drop_graphs() {
        for (auto &g : graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    void release() {
        drop_graphs();
        void *ptrs[] = {xbuf, xstage, status, are, aim, bre, bim, xoff, state, z, ubuf, partial, hank, xseg};
        for (void *q : ptrs)
            if (q) cudaFree(q);
        xbuf = xstage = nullptr;
        status = nullptr;
        are = aim = bre = bim = nullptr;
        xoff = nullptr;
        state = z = ubuf = partial = nullptr;
        hank = xseg = nullptr;
        for (auto &t : tcp) {
            void *tp[] = {t.H, t.row_scale, t.has_carry, t.tile_ptr, t.tile_end, t.a, t.aJ, t.c, t.aLf,
                          t.aL, t.aLb1, t.aLb2, t.v, t.panel};
            for (void *q : tp)
                if (q) cudaFree(q);
            t.H = nullptr;
            t.row_scale = nullptr;
            t.has_carry = nullptr;
            t.tile_ptr = t.tile_end = nullptr;
            t.a = t.aJ = t.c = t.aLf = nullptr;
            t.aL = t.aLb1 = t.aLb2 = t.v = t.panel = nullptr;
            t.groups.release();
            t.tmpl_of.release();
        }
        tasks.release();
        items.release();
        order.release();
        task_out.release();
        comb_ptr.release();
        comb_rows.release();
        comb_list.release();
        queue.release();
        prog.release();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        cap_stream = nullptr;
        if (io) cudaStreamDestroy(io);
        io = nullptr;
        if (ev_push) cudaEventDestroy(ev_push);
        if (ev_io) cudaEventDestroy(ev_io);
        ev_push = ev_io = nullptr;
        if (timer) {
            timer->release();
            delete timer;
            timer = nullptr;
        }
    }
};

namespace {

// The description a member's plain levels are planned with: its filters at
// those levels, the server's shape.
spiir_bank_desc plain_desc(const spiir_server *sv, const spiir_bank_desc *m) {
    spiir_bank_desc d = *m;
    d.n_streams = sv->S;
    d.block_len = sv->block;
    d.max_push_blocks = 1;
    d.h_down = sv->h_down.data();
    d.h_up = sv->h_up.data();
    d.n_taps = (int32_t)sv->h_down.size();
    d.n_taps_up = (int32_t)sv->h_up.size();
    d.align = sv->d.align;
    d.snr_scale = sv->scale;
    d.mode = SPIIR_PLAIN_FP32;
    d.chunk_len = 0;
    d.tune = -(sv->variant + 1);
    d.hbm_budget_bytes = 0;
    d.carry = 0;
    return d;
}

// Grow a [outer][cap * inner] array to [outer][new_cap * inner], keeping the
// first cap entries of each row; new entries are zero.
template <typename T>
spiir_status grow_rows(T **p, int64_t outer, int64_t cap, int64_t new_cap, int64_t inner, cudaStream_t s) {
    T *q = nullptr;
    CUDA_TRY(cudaMalloc((void **)&q, std::max<int64_t>(1, outer * new_cap * inner) * sizeof(T)));
    CUDA_TRY(cudaMemsetAsync(q, 0, std::max<int64_t>(1, outer * new_cap * inner) * sizeof(T), s));
    if (*p && cap > 0)
        CUDA_TRY(cudaMemcpy2DAsync(q, new_cap * inner * sizeof(T), *p, cap * inner * sizeof(T),
                                   cap * inner * sizeof(T), outer, cudaMemcpyDeviceToDevice, s));
    if (*p) {
        CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(*p);
    }
    *p = q;
    return SPIIR_OK;
}

int64_t grown(int64_t need, int64_t cap) { return std::max<int64_t>(need, cap + cap / 2); }

spiir_status grow_slots(spiir_server *sv, int64_t need, cudaStream_t s) {
    const int64_t cap = sv->slot_alloc.cap(), nc = grown(need, cap);
    spiir_status st;
    if ((st = grow_rows(&sv->are, 1, cap, nc, 1, s)) || (st = grow_rows(&sv->aim, 1, cap, nc, 1, s)) ||
        (st = grow_rows(&sv->bre, 1, cap, nc, 1, s)) || (st = grow_rows(&sv->bim, 1, cap, nc, 1, s)) ||
        (st = grow_rows(&sv->xoff, 1, cap, nc, 1, s)) || (st = grow_rows(&sv->state, sv->S, cap, nc, 1, s)))
        return st;
    sv->slot_alloc.grow(nc);
    return SPIIR_OK;
}

spiir_status grow_template_rows(spiir_server *sv, int64_t need, cudaStream_t s) {
    const int64_t cap = sv->row_alloc.cap(), nc = grown(need, cap);
    spiir_status st;
    // the output ring is per-push: no contents to keep
    if (sv->z) {
        CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(sv->z);
        sv->z = nullptr;
    }
    CUDA_TRY(cudaMalloc((void **)&sv->z, std::max<int64_t>(1, sv->S * nc * sv->block) * sizeof(float2)));
    CUDA_TRY(cudaMemsetAsync(sv->z, 0, std::max<int64_t>(1, sv->S * nc * sv->block) * sizeof(float2), s));
    if (sv->H > 0 && (st = grow_rows(&sv->ubuf, (int64_t)sv->S * sv->H, cap, nc, SPIIR_UHIST, s))) return st;
    sv->row_alloc.grow(nc);
    return SPIIR_OK;
}

// Partial rows are per-push scratch: a new layout reallocates without copying.
spiir_status relayout_partial(spiir_server *sv, cudaStream_t s) {
    int64_t off = 0;
    for (int i = 0; i < sv->L; ++i) {
        sv->part_base[i] = off;
        off += sv->level_rows(i) * sv->geo.part_stride[i];
    }
    sv->part_stream_stride = off;
    if (sv->partial) {
        CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(sv->partial);
        sv->partial = nullptr;
    }
    CUDA_TRY(cudaMalloc((void **)&sv->partial, std::max<int64_t>(1, sv->S * off) * sizeof(float2)));
    return SPIIR_OK;
}

spiir_status grow_groups(spiir_server *sv, TcPool &t, int64_t need, cudaStream_t s) {
    const int64_t cap = t.group_alloc.cap(), nc = grown(need, cap);
    spiir_status st;
    const int64_t slice16 = (int64_t)sv->n_slices * (kTcSliceBytes / 16);
    if ((st = grow_rows(&t.H, 1, cap, nc, slice16, s)) || (st = grow_rows(&t.row_scale, 1, cap, nc, 64, s)) ||
        (st = grow_rows(&t.has_carry, 1, cap, nc, 64, s)) || (st = grow_rows(&t.tile_ptr, 1, cap, nc, 64, s)) ||
        (st = grow_rows(&t.tile_end, 1, cap, nc, 64, s)))
        return st;
    t.group_alloc.grow(nc);
    return relayout_partial(sv, s);
}

spiir_status grow_tiles(spiir_server *sv, TcPool &t, int64_t need, cudaStream_t s) {
    const int64_t cap = t.tile_alloc.cap(), nc = grown(need, cap);
    spiir_status st;
    if ((st = grow_rows(&t.a, 1, cap, nc, kTcTile, s)) || (st = grow_rows(&t.aJ, 1, cap, nc, kTcTile, s)) ||
        (st = grow_rows(&t.c, 1, cap, nc, kTcTile, s)) || (st = grow_rows(&t.aLf, 1, cap, nc, kTcTile, s)) ||
        (st = grow_rows(&t.aL, 1, cap, nc, kTcTile, s)) || (st = grow_rows(&t.aLb1, 1, cap, nc, kTcTile, s)) ||
        (st = grow_rows(&t.aLb2, 1, cap, nc, kTcTile, s)) ||
        (st = grow_rows(&t.v, sv->S, cap, nc, kTcTile, s)) ||
        (st = grow_rows(&t.panel, 1, cap, nc, kTcPanelBytes / 16, s)))
        return st;
    t.tile_alloc.grow(nc);
    return SPIIR_OK;
}

template <typename T>
spiir_status put(T *dst, const std::vector<T> &src, cudaStream_t s) {
    if (!src.empty())
        CUDA_TRY(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return SPIIR_OK;
}

// Place a member's block-form part at level i.
spiir_status place_tc(spiir_server *sv, Member &m, int i, cudaStream_t s) {
    MemberTc &mt = m.tc[i];
    TcPool &t = sv->tcp[i];
    const TcPack &pk = mt.pk;
    spiir_status st;
    mt.ng = pk.n_groups;
    mt.nt = pk.n_tiles;
    int64_t at = t.group_alloc.take(mt.ng);
    if (at < 0) {
        if ((st = grow_groups(sv, t, t.group_alloc.need_for(mt.ng), s))) return st;
        at = t.group_alloc.take(mt.ng);
    }
    mt.g0 = at;
    at = t.tile_alloc.take(mt.nt);
    if (at < 0) {
        if ((st = grow_tiles(sv, t, t.tile_alloc.need_for(mt.nt), s))) return st;
        at = t.tile_alloc.take(mt.nt);
    }
    mt.t0 = at;
    const int64_t slice16 = (int64_t)sv->n_slices * (kTcSliceBytes / 16);
    CUDA_TRY(cudaMemcpyAsync(t.H + mt.g0 * slice16, pk.H.data(), pk.H.size() * sizeof(uint16_t),
                             cudaMemcpyHostToDevice, s));
    // per row of the member's groups (rows past its templates are inert)
    const int64_t nr = mt.ng * 64;
    std::vector<float> rs(nr, 0.f);
    std::vector<uint8_t> hc(nr, 0);
    std::vector<int32_t> tp(nr, 0), te(nr, 0);
    for (int r = 0; r < mt.nT; ++r) {
        rs[r] = pk.row_scale[r];
        hc[r] = pk.has_carry[r];
        tp[r] = (int32_t)(mt.t0 + pk.tile_ptr[r]);
        te[r] = (int32_t)(mt.t0 + pk.tile_ptr[r + 1]);
    }
    const int64_t r0 = mt.g0 * 64;
    if ((st = put(t.row_scale + r0, rs, s)) || (st = put(t.has_carry + r0, hc, s)) ||
        (st = put(t.tile_ptr + r0, tp, s)) || (st = put(t.tile_end + r0, te, s)))
        return st;
    const int64_t k0 = mt.t0 * kTcTile;
    if ((st = put(t.a + k0, pk.a, s)) || (st = put(t.aJ + k0, pk.aJ, s)) || (st = put(t.c + k0, pk.c, s)) ||
        (st = put(t.aLf + k0, pk.aLf, s)) || (st = put(t.aL + k0, pk.aL, s)) ||
        (st = put(t.aLb1 + k0, pk.aLb1, s)) || (st = put(t.aLb2 + k0, pk.aLb2, s)))
        return st;
    if (mt.nt > 0) {
        CUDA_TRY(cudaMemcpyAsync(t.panel + mt.t0 * (kTcPanelBytes / 16), pk.panel.data(),
                                 pk.panel.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemset2DAsync(t.v + k0, t.tile_alloc.cap() * kTcTile * sizeof(uint4), 0,
                                   mt.nt * kTcTile * sizeof(uint4), sv->S, s));
    }
    return SPIIR_OK;
}

// Place a new member: ranges in every pool, coefficients uploaded, state,
// output rows and upsampler histories zeroed.
spiir_status place(spiir_server *sv, Member &m, cudaStream_t s) {
    spiir_status st;
    const Plan &p = m.p;
    int64_t at = sv->slot_alloc.take(p.n_slots);
    if (at < 0) {
        if ((st = grow_slots(sv, sv->slot_alloc.need_for(p.n_slots), s))) return st;
        at = sv->slot_alloc.take(p.n_slots);
    }
    m.slot0 = at;
    at = sv->row_alloc.take(m.T);
    if (at < 0) {
        if ((st = grow_template_rows(sv, sv->row_alloc.need_for(m.T), s))) return st;
        at = sv->row_alloc.take(m.T);
    }
    m.row0 = at;
    for (int i = 0; i < sv->L; ++i) {
        at = sv->prow_alloc[i].take(p.part_rows[i]);
        if (at < 0) {
            sv->prow_alloc[i].grow(grown(sv->prow_alloc[i].need_for(p.part_rows[i]), sv->prow_alloc[i].cap()));
            if ((st = relayout_partial(sv, s))) return st;
            at = sv->prow_alloc[i].take(p.part_rows[i]);
        }
        m.prow0[i] = at;
    }
    for (int i = 0; i < sv->L; ++i)
        if (m.tc[i].used && (st = place_tc(sv, m, i, s))) return st;
    const int64_t n = p.n_slots, cap = sv->slot_alloc.cap(), rcap = sv->row_alloc.cap();
    if (n > 0) {
        CUDA_TRY(cudaMemcpyAsync(sv->are + m.slot0, p.are.data(), n * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(sv->aim + m.slot0, p.aim.data(), n * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(sv->bre + m.slot0, p.bre.data(), n * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(sv->bim + m.slot0, p.bim.data(), n * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(sv->xoff + m.slot0, p.xoff.data(), n * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemset2DAsync(sv->state + m.slot0, cap * sizeof(float2), 0, n * sizeof(float2), sv->S, s));
    }
    CUDA_TRY(cudaMemset2DAsync(sv->z + m.row0 * sv->block, rcap * sv->block * sizeof(float2), 0,
                               (size_t)m.T * sv->block * sizeof(float2), sv->S, s));
    if (sv->H > 0)
        CUDA_TRY(cudaMemset2DAsync(sv->ubuf + m.row0 * SPIIR_UHIST, rcap * SPIIR_UHIST * sizeof(float2), 0,
                                   (size_t)m.T * SPIIR_UHIST * sizeof(float2), (size_t)sv->S * sv->H, s));
    return SPIIR_OK;
}

void unplace(spiir_server *sv, const Member &m) {
    sv->slot_alloc.give(m.slot0, m.p.n_slots);
    sv->row_alloc.give(m.row0, m.T);
    for (int i = 0; i < sv->L; ++i) {
        sv->prow_alloc[i].give(m.prow0[i], m.p.part_rows[i]);
        if (m.tc[i].used) {
            sv->tcp[i].group_alloc.give(m.tc[i].g0, m.tc[i].ng);
            sv->tcp[i].tile_alloc.give(m.tc[i].t0, m.tc[i].nt);
        }
    }
}

// Work lists of all members, in member order, with pooled indices.
spiir_status rebuild_lists(spiir_server *sv, cudaStream_t s) {
    std::vector<WarpTask> tasks;
    std::vector<CtaItem> items;
    std::vector<int32_t> task_out, order;
    std::vector<int64_t> work;
    const int64_t rcap = sv->row_alloc.cap();
    std::vector<int32_t> owner(rcap, -1);      // member (index in mv) of each pooled row
    std::vector<const Member *> mv;
    for (auto &kv : sv->members) mv.push_back(&kv.second);
    for (size_t mi = 0; mi < mv.size(); ++mi) {
        const Member &m = *mv[mi];
        const Plan &p = m.p;
        const int32_t task0 = (int32_t)tasks.size(), out0 = (int32_t)task_out.size();
        // level of each destination entry (from the task that owns it)
        std::vector<int8_t> lvl(p.task_out.size(), 0);
        for (const WarpTask &wt : p.tasks)
            for (int g = 0; g < wt.n_groups; ++g) lvl[wt.out_base + g] = wt.level;
        for (size_t j = 0; j < p.task_out.size(); ++j) {
            const int32_t dst = p.task_out[j];
            if (dst >= 0)
                task_out.push_back((int32_t)(m.row0 + dst));
            else
                task_out.push_back(-(int32_t)(m.prow0[lvl[j]] + (-dst - 1)) - 1);
        }
        for (WarpTask wt : p.tasks) {
            wt.slot_base = (int32_t)(wt.slot_base + m.slot0);
            wt.out_base += out0;
            tasks.push_back(wt);
        }
        for (CtaItem ci : p.items) {
            int64_t w = 0;
            for (int k = 0; k < ci.task_count; ++k) {
                const WarpTask &wt = p.tasks[ci.task_begin + k];
                w += (int64_t)wt.F * (sv->block >> wt.level);
            }
            ci.task_begin += task0;
            items.push_back(ci);
            work.push_back(w);
        }
        for (int t = 0; t < m.T; ++t) owner[m.row0 + t] = (int32_t)mi;
    }
    if ((int64_t)tasks.size() > INT32_MAX || (int64_t)sv->slot_alloc.cap() > INT32_MAX)
        return fail(SPIIR_EUNSUPPORTED, "server above 2^31 filter slots");
    order.resize(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
    // combine lists over the pooled template rows: the plain units' partial
    // rows, then the template's block-form row of each block-form level
    std::vector<int32_t> cptr((size_t)rcap * sv->L + 1, 0), crows, clist;
    for (int64_t r = 0; r < rcap; ++r) {
        const int mi = owner[r];
        const Member *m = mi >= 0 ? mv[mi] : nullptr;
        const bool comb = m && m->combine;
        if (comb) clist.push_back((int32_t)r);
        for (int i = 0; i < sv->L; ++i) {
            const size_t j = (size_t)r * sv->L + i;
            if (comb) {
                const int t = (int)(r - m->row0);
                const Plan &p = m->p;
                if (!p.comb_ptr.empty())
                    for (int32_t q = p.comb_ptr[(size_t)t * sv->L + i]; q < p.comb_ptr[(size_t)t * sv->L + i + 1]; ++q)
                        crows.push_back((int32_t)(m->prow0[i] + p.comb_rows[q]));
                if (m->tc[i].used && m->tc[i].row[t] >= 0)
                    crows.push_back((int32_t)(sv->tc_row_base(i) + m->tc[i].g0 * 64 + m->tc[i].row[t]));
            }
            cptr[j + 1] = (int32_t)crows.size();
        }
    }
    spiir_status st;
    if ((st = sv->tasks.upload(tasks, s)) || (st = sv->items.upload(items, s)) ||
        (st = sv->order.upload(order, s)) || (st = sv->task_out.upload(task_out, s)) ||
        (st = sv->comb_ptr.upload(cptr, s)) || (st = sv->comb_rows.upload(crows, s)) ||
        (st = sv->comb_list.upload(clist, s)))
        return st;
    if ((st = sv->prog.reserve((int64_t)sv->S * std::max<size_t>(1, items.size()), s))) return st;
    sv->n_items = (int)items.size();
    sv->n_tasks = (int)tasks.size();
    sv->n_comb = (int)clist.size();
    // block-form lists: the groups of every member at the level, and the
    // pooled rows of the templates that own carry tiles
    for (int i = 0; i < sv->L; ++i) {
        TcPool &t = sv->tcp[i];
        if (!t.on) continue;
        std::vector<int32_t> gl, tl;
        for (const Member *m : mv) {
            const MemberTc &mt = m->tc[i];
            if (!mt.used) continue;
            for (int64_t g = 0; g < mt.ng; ++g) gl.push_back((int32_t)(mt.g0 + g));
            for (int r = 0; r < mt.nT && r < (int)mt.pk.has_carry.size(); ++r)
                if (mt.pk.has_carry[r]) tl.push_back((int32_t)(mt.g0 * 64 + r));
        }
        if ((st = t.groups.upload(gl, s)) || (st = t.tmpl_of.upload(tl, s))) return st;
        t.n_groups = (int)gl.size();
        t.n_carry = (int)tl.size();
    }
    return SPIIR_OK;
}

spiir_status apply_changes(spiir_server *sv) {
    cudaStream_t s = sv->io;
    // nothing may change under a push still in flight
    if (sv->pushed_once) CUDA_TRY(cudaStreamWaitEvent(s, sv->ev_push, 0));
    for (int id : sv->pending_remove) {
        auto it = sv->members.find(id);
        if (it == sv->members.end()) continue;
        unplace(sv, it->second);
        sv->members.erase(it);
    }
    sv->pending_remove.clear();
    for (Member &m : sv->pending_add) {
        spiir_status st = place(sv, m, s);
        if (st) return st;
        // the packed coefficients are on the device now; keep the lists
        const int id = m.id;
        sv->members.emplace(id, std::move(m));
        Member &mm = sv->members[id];
        Plan &p = mm.p;
        std::vector<float>().swap(p.are);
        std::vector<float>().swap(p.aim);
        std::vector<float>().swap(p.bre);
        std::vector<float>().swap(p.bim);
        std::vector<int32_t>().swap(p.xoff);
        std::vector<int64_t>().swap(p.slot_filter);
        for (auto &mt : mm.tc) {
            // keep only which templates own tiles (for the carry lists)
            std::vector<uint8_t> hc = std::move(mt.pk.has_carry);
            mt.pk = TcPack();
            mt.pk.has_carry = std::move(hc);
        }
    }
    sv->pending_add.clear();
    spiir_status st = rebuild_lists(sv, s);
    if (st) return st;
    CUDA_TRY(cudaEventRecord(sv->ev_io, s));
    sv->io_pending = true;
    sv->drop_graphs();
    sv->dirty = false;
    return SPIIR_OK;
}

spiir_status launch_push(spiir_server *sv, int64_t n_prev, cudaStream_t st);

// The graph of the next push (captured once per membership and per first or
// later push).
spiir_status ensure_graph(spiir_server *sv) {
    const int gi = sv->pushes > 0 ? 1 : 0;
    if (sv->graph[gi]) return SPIIR_OK;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(sv->cap_stream, cudaStreamCaptureModeThreadLocal));
    KernelTimer *keep = sv->timer;
    sv->timer = nullptr;                 // no events inside the graph
    spiir_status stc = launch_push(sv, gi ? sv->block : 0, sv->cap_stream);
    sv->timer = keep;
    cudaError_t e = cudaStreamEndCapture(sv->cap_stream, &g);
    if (stc) {
        if (g) cudaGraphDestroy(g);
        return stc;
    }
    if (e != cudaSuccess) return fail(SPIIR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&sv->graph[gi], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(SPIIR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return SPIIR_OK;
}

void level_args(const spiir_server *sv, int64_t n_prev, LevelArgs *lev) {
    const Plan &g = sv->geo;
    const int segs = push_segments_n(sv->block);
    for (int i = 0; i < sv->L; ++i) {
        LevelArgs &L = lev[i];
        L.hist = g.hist[i];
        L.n = (int32_t)(sv->block >> i);
        L.seg = (int32_t)segment_len(sv->block, i, segs);
        L.n_prev = (int32_t)(n_prev >> i);
        L.part_base = sv->part_base[i];
        L.part_stride = g.part_stride[i];
        L.xbuf_off = g.xbuf_off[i];
        L.ubuf_off = i > 0 ? (int64_t)(i - 1) * sv->row_alloc.cap() * SPIIR_UHIST : 0;
        L.ubuf_stride = i > 0 ? SPIIR_UHIST : 0;
        L.pad = 0;
    }
}

// The kernels of one push (reading the strain from xstage).
spiir_status launch_push(spiir_server *sv, int64_t n_prev, cudaStream_t st) {
    const int S = sv->S;
    int launches = 0;
    PrologueArgs pa{};
    pa.queue = sv->queue.p;
    pa.prog = sv->prog.p;
    pa.n_items = sv->n_items;
    pa.xbuf = sv->xbuf;
    pa.xbuf_stream_stride = sv->geo.xbuf_stream_stride;
    pa.x_in = sv->xstage;
    pa.x_in_stream_stride = sv->block;
    pa.stream0 = 0;
    pa.n_levels = sv->L;
    level_args(sv, n_prev, pa.lev);
    KernelTimer *tm = (sv->timer && sv->timer->on) ? sv->timer : nullptr;
    if (tm) tm->begin(SPIIR_K_PROLOGUE, st);
    CUDA_TRY(spiir_launch_prologue(pa, S, st));
    if (tm) tm->end(st, kPrologueLaunches);
    launches += kPrologueLaunches;
    if (sv->L > 1) {
        DecimArgs da{};
        da.xbuf = sv->xbuf;
        da.xbuf_stream_stride = sv->geo.xbuf_stream_stride;
        da.stream0 = 0;
        da.n_levels = sv->L;
        da.n_taps = (int)sv->h_down.size();
        for (size_t j = 0; j < sv->h_down.size(); ++j) da.h_down[j] = sv->h_down[j];
        level_args(sv, n_prev, da.lev);
        if (tm) tm->begin(SPIIR_K_DECIMATE, st);
        CUDA_TRY(spiir_launch_decimate(da, S, st));
        if (tm) tm->end(st);
        ++launches;
    }
    if (sv->n_items > 0) {
        RecurArgs ra{};
        ra.tasks = sv->tasks.p;
        ra.items = sv->items.p;
        ra.order = sv->order.p;
        ra.n_items = sv->n_items;
        ra.n_segs = push_segments_n(sv->block);
        ra.queue = sv->queue.p;
        ra.prog = sv->prog.p;
        ra.stall_test = 0;
        ra.task_out = sv->task_out.p;
        ra.a_re = sv->are;
        ra.a_im = sv->aim;
        ra.b_re = sv->bre;
        ra.b_im = sv->bim;
        ra.xoff = sv->xoff;
        ra.state = sv->state;
        ra.n_slots = sv->slot_alloc.cap();
        ra.xbuf = sv->xbuf;
        ra.xbuf_stream_stride = sv->geo.xbuf_stream_stride;
        ra.partial = sv->partial;
        ra.partial_stream_stride = sv->part_stream_stride;
        ra.z = sv->z;
        ra.z_row_stride = sv->block;
        ra.z_stream_stride = sv->row_alloc.cap() * sv->block;
        ra.scale = sv->scale;
        ra.stream0 = 0;
        ra.n_levels = sv->L;
        ra.status = sv->status;
        level_args(sv, n_prev, ra.lev);
        const int64_t total = (int64_t)ra.n_segs * ra.n_items;
        const int64_t resident = std::max<int64_t>(1, (int64_t)sv->ctas_per_sm * sv->n_sms / S);
        const int ctas = (int)std::min<int64_t>(total, resident);
        if (tm) tm->begin(SPIIR_K_RECUR, st);
        CUDA_TRY(spiir_launch_recur(ra, sv->variant, ctas, S, sv->smem_bytes, st));
        if (tm) tm->end(st);
        ++launches;
    }
    // block-form levels: each level's sums into its partial rows (unscaled;
    // the combine pass applies the SNR scale), streams two at a time
    for (int i = 0; i < sv->L; ++i) {
        const TcPool &t = sv->tcp[i];
        if (!t.on || t.n_groups == 0) continue;
        for (int q0 = 0; q0 < S; q0 += 2) {
            TcLaunch l{};
            l.xbuf = sv->xbuf + sv->geo.xbuf_off[i];
            l.xbuf_stride = sv->geo.xbuf_stream_stride;
            l.hist = t.hist_read;
            l.F = sv->tcF;
            l.L = sv->tcL;
            l.K = sv->tcK;
            l.n_chunks = (sv->block >> i) / sv->tcL;
            l.n_streams = std::min(2, S - q0);
            l.stream0 = q0;
            l.hank = sv->hank;
            l.xseg = sv->xseg;
            l.tile_ptr = t.tile_ptr;
            l.tile_end = t.tile_end;
            l.tmpl_of = t.tmpl_of.p;
            l.n_carry = t.n_carry;
            l.a = t.a;
            l.aJ = t.aJ;
            l.aLf = t.aLf;
            l.c = t.c;
            l.aL = t.aL;
            l.aLb1 = t.aLb1;
            l.aLb2 = t.aLb2;
            l.panel = t.panel;
            l.v = t.v;
            l.n_slots = t.tile_alloc.cap() * kTcTile;
            l.carry_scale = 1.0f;
            l.H = t.H;
            l.row_scale = t.row_scale;
            l.has_carry = t.has_carry;
            l.groups = t.groups.p;
            l.n_groups = t.n_groups;
            l.n_rows = (int)(64 * t.group_alloc.cap());
            l.z = sv->partial + sv->part_base[i] + sv->tc_row_base(i) * sv->geo.part_stride[i];
            l.z_row_stride = sv->geo.part_stride[i];
            l.z_stream_stride = sv->part_stream_stride;
            l.bf16 = sv->bf16;
            l.df = sv->df;
            l.carry_mode = sv->d.carry;
            l.status = sv->status;
            l.n_sms = sv->n_sms;
            spiir_status r = spiir_tc_launch(l, st, tm);
            if (r) return fail(r, "%s", spiir_tc_last_error());
            launches += 2 + (t.n_carry > 0);
        }
    }
    if (sv->n_comb > 0) {
        CombineArgs ca{};
        ca.comb_ptr = sv->comb_ptr.p;
        ca.comb_rows = sv->comb_rows.p;
        ca.partial = sv->partial;
        ca.partial_stream_stride = sv->part_stream_stride;
        ca.ubuf = sv->ubuf;
        ca.ubuf_stream_stride = (int64_t)sv->H * sv->row_alloc.cap() * SPIIR_UHIST;
        ca.z = sv->z;
        ca.z_row_stride = sv->block;
        ca.z_stream_stride = sv->row_alloc.cap() * sv->block;
        ca.scale = sv->scale;
        ca.n_templates = sv->n_comb;
        ca.n_levels = sv->L;
        ca.n_taps = (int)sv->h_up.size();
        ca.stream0 = 0;
        ca.status = sv->status;
        ca.rows = sv->comb_list.p;
        for (size_t j = 0; j < sv->h_up.size(); ++j) ca.h_up2[j] = 2.0f * sv->h_up[j];
        level_args(sv, n_prev, ca.lev);
        if (tm) tm->begin(SPIIR_K_COMBINE, st);
        CUDA_TRY(spiir_launch_combine(ca, spiir_combine_chunk(sv->L, sv->block), S, st));
        if (tm) tm->end(st);
        ++launches;
    }
    sv->launches = launches;
    return SPIIR_OK;
}

int64_t member_bytes(const spiir_server *sv, const Member &m) {
    const Plan &p = m.p;
    const int64_t S = sv->S;
    int64_t b = p.n_slots * (4 * 4 + 4 + 8 * S);
    b += (int64_t)m.T * S * ((int64_t)sv->block + (int64_t)sv->H * SPIIR_UHIST) * 8;
    for (int i = 0; i < sv->L; ++i) b += p.part_rows[i] * S * sv->geo.part_stride[i] * 8;
    b += (int64_t)p.tasks.size() * (sizeof(WarpTask) + 32 * 4) + (int64_t)p.items.size() * (sizeof(CtaItem) + 4 + 4 * S);
    b += (int64_t)m.T * sv->L * 4 + p.n_slots * 4;
    for (int i = 0; i < sv->L; ++i) {
        const MemberTc &mt = m.tc[i];
        if (!mt.used) continue;
        b += mt.pk.n_groups * ((int64_t)sv->n_slices * kTcSliceBytes + 64 * (4 + 1 + 8) + 64 * S * sv->geo.part_stride[i] * 8);
        b += (int64_t)mt.pk.n_tiles * (kTcPanelBytes + kTcTile * (32 + 48 + 16 * S));
    }
    return b;
}

spiir_status check_member(const spiir_server *sv, const spiir_bank_desc *m) {
    if (!m) return fail(SPIIR_EINVAL, "member is NULL");
    if (m->n_levels != sv->L)
        return fail(SPIIR_EINVAL, "member has %d levels, the server %d", m->n_levels, sv->L);
    if (m->base_rate != sv->d.base_rate) return fail(SPIIR_EINVAL, "member base_rate differs from the server's");
    if (m->n_filters > 0 && !m->delay) return fail(SPIIR_EINVAL, "filter arrays must not be NULL");
    for (int64_t k = 0; k < m->n_filters; ++k)
        if (m->delay[k] > sv->d.max_delay)
            return fail(SPIIR_EINVAL, "delay[%lld] = %d above the server's max_delay %d", (long long)k,
                        m->delay[k], sv->d.max_delay);
    return SPIIR_OK;
}

// Plan a member: its plain levels with make_plan, each block-form level with
// spiir_tc_pack (arrays == false: sizes only, for the footprint).
spiir_status build_member(const spiir_server *sv, const spiir_bank_desc *member, bool arrays, Member &m) {
    spiir_status st = check_member(sv, member);
    if (st) return st;
    spiir_bank_desc d = plain_desc(sv, member);
    if ((st = validate(&d))) return st;
    m.T = d.n_templates;
    m.n_filters = d.n_filters;
    m.fs_per_push = 0;
    for (int64_t k = 0; k < d.n_filters; ++k) m.fs_per_push += sv->block >> (d.level ? d.level[k] : 0);
    // Routing: at a block-form level a template runs in the block form when
    // it has at least tc_min filters there (the block form's cost per
    // template-sample is fixed by F + L, the plain recursion's grows with the
    // filters), else with its other filters in the plain form.
    const int thr = sv->tc_min;
    bool any_tc = false;
    for (int i = 0; i < sv->L; ++i) {
        MemberTc &mt = m.tc[i];
        mt.used = false;
        mt.nT = 0;
        mt.row.clear();
        if (!sv->tcp[i].on) continue;
        std::vector<int32_t> cnt(m.T, 0);
        for (int64_t k = 0; k < d.n_filters; ++k)
            if ((d.level ? d.level[k] : 0) == i) cnt[d.template_id[k]]++;
        mt.row.assign(m.T, -1);
        for (int t = 0; t < m.T; ++t)
            if (cnt[t] > 0 && cnt[t] >= thr) mt.row[t] = mt.nT++;
        mt.used = mt.nT > 0;
        any_tc |= mt.used;
    }
    auto to_tc = [&](int64_t k) {
        const int l = d.level ? d.level[k] : 0;
        return m.tc[l].used && m.tc[l].row[d.template_id[k]] >= 0;
    };
    // the filters of the plain form
    std::vector<float> ar, ai, br, bi;
    std::vector<int32_t> dl, tid;
    std::vector<int8_t> lv;
    for (int64_t k = 0; k < d.n_filters; ++k) {
        if (to_tc(k)) continue;
        ar.push_back(d.a_re[k]);
        ai.push_back(d.a_im[k]);
        br.push_back(d.b_re[k]);
        bi.push_back(d.b_im[k]);
        dl.push_back(d.delay[k]);
        tid.push_back(d.template_id[k]);
        lv.push_back((int8_t)(d.level ? d.level[k] : 0));
    }
    spiir_bank_desc dp = d;
    dp.n_filters = (int64_t)ar.size();
    dp.a_re = ar.data();
    dp.a_im = ai.data();
    dp.b_re = br.data();
    dp.b_im = bi.data();
    dp.delay = dl.data();
    dp.template_id = tid.data();
    dp.level = lv.data();
    if ((st = make_plan(&dp, sv->variant, arrays, m.p, sv->geo.hist))) return st;
    if (m.p.smem_bytes > sv->smem_bytes)
        return fail(SPIIR_EINVAL, "member needs more shared memory than the server's kernel setup");
    m.combine = m.p.need_combine || any_tc;
    // each block-form level: its routed templates, renumbered
    for (int i = 0; i < sv->L; ++i) {
        MemberTc &mt = m.tc[i];
        if (!mt.used) continue;
        std::vector<float> qr, qi, cr, ci;
        std::vector<int32_t> qd, qt;
        std::vector<int64_t> tcnt(mt.nT, 0);
        for (int64_t k = 0; k < d.n_filters; ++k) {
            if ((d.level ? d.level[k] : 0) != i || mt.row[d.template_id[k]] < 0) continue;
            qr.push_back(d.a_re[k]);
            qi.push_back(d.a_im[k]);
            cr.push_back(d.b_re[k]);
            ci.push_back(d.b_im[k]);
            qd.push_back(d.delay[k]);
            qt.push_back(mt.row[d.template_id[k]]);
            tcnt[mt.row[d.template_id[k]]]++;
        }
        if (arrays) {
            spiir_bank_desc dt = d;
            dt.n_templates = mt.nT;
            dt.n_filters = (int64_t)qr.size();
            dt.a_re = qr.data();
            dt.a_im = qi.data();
            dt.b_re = cr.data();
            dt.b_im = ci.data();
            dt.delay = qd.data();
            dt.template_id = qt.data();
            dt.level = nullptr;
            if ((st = spiir_tc_pack(&dt, -1, sv->tcF, sv->tcL, 1.0, sv->bf16, sv->df, mt.pk)))
                return fail(st, "%s", spiir_tc_last_error());
        } else {
            // sizes only: groups of 64 templates, tiles of 128 filters per template
            mt.pk.n_groups = (mt.nT + 63) / 64;
            int nt = 0;
            for (int t = 0; t < mt.nT; ++t) nt += (int)((tcnt[t] + kTcTile - 1) / kTcTile);
            mt.pk.n_tiles = nt;
        }
    }
    return SPIIR_OK;
}

}  // namespace

extern "C" {

spiir_status spiir_server_create(const spiir_server_desc *desc, void *cuda_stream, spiir_server_t *out) {
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(SPIIR_EINVAL, "desc is NULL");
    if (desc->mode != SPIIR_PLAIN_FP32 && desc->mode != SPIIR_TC_FP16 && desc->mode != SPIIR_TC_BF16)
        return fail(SPIIR_EUNSUPPORTED, "server: mode must be PLAIN_FP32, TC_FP16 or TC_BF16");
    if (desc->max_delay < 0 || desc->max_delay > (1 << 20))
        return fail(SPIIR_EINVAL, "max_delay must be in [0, 2^20]");
    if (desc->n_levels < 1 || desc->n_levels > SPIIR_MAX_LEVELS)
        return fail(SPIIR_EINVAL, "n_levels must be in [1, %d]", SPIIR_MAX_LEVELS);
    if (desc->carry < 0 || desc->carry > 2) return fail(SPIIR_EINVAL, "carry must be 0, 1 or 2");
    const bool tc = desc->mode != SPIIR_PLAIN_FP32;
    const int tcL = desc->chunk_len ? desc->chunk_len : 256;
    if (tc && tcL != 128 && tcL != 256) return fail(SPIIR_EUNSUPPORTED, "chunk_len must be 128 or 256");
    const int tcF = (int)(((int64_t)desc->max_delay + 1 + 63) / 64 * 64);
    // the shape is checked by planning an empty bank of it
    spiir_bank_desc e{};
    e.n_templates = 1;
    e.n_levels = desc->n_levels;
    e.base_rate = desc->base_rate;
    e.n_streams = desc->n_streams;
    e.block_len = desc->block_len;
    e.max_push_blocks = 1;
    e.h_down = desc->h_down;
    e.h_up = desc->h_up;
    e.n_taps = desc->n_taps;
    e.n_taps_up = desc->n_taps_up;
    e.align = desc->n_levels > 1 ? desc->align : 0;
    e.snr_scale = desc->snr_scale;
    e.mode = SPIIR_PLAIN_FP32;
    e.tune = desc->tune;
    spiir_status st = validate(&e);
    if (st) return st;
    if ((desc->block_len >> (desc->n_levels - 1)) % 4 != 0)
        return fail(SPIIR_EINVAL, "block_len must be a multiple of 4 * 2^(n_levels-1)");
    spiir_server *sv = new (std::nothrow) spiir_server();
    if (!sv) return fail(SPIIR_ENOMEM, "host allocation failed");
    sv->d = *desc;
    sv->d.h_down = sv->d.h_up = nullptr;
    sv->d.align = e.align;
    sv->S = desc->n_streams;
    sv->L = desc->n_levels;
    sv->H = desc->n_levels - 1;
    sv->block = desc->block_len;
    sv->scale = desc->snr_scale != 0.f ? desc->snr_scale : 2.0f / (float)desc->base_rate;
    const int nt = desc->n_taps ? desc->n_taps : 32;
    const int ntu = desc->n_taps_up ? desc->n_taps_up : nt;
    sv->h_down.resize(nt);
    sv->h_up.resize(ntu);
    if (desc->h_down) {
        std::copy(desc->h_down, desc->h_down + nt, sv->h_down.begin());
        std::copy(desc->h_up, desc->h_up + ntu, sv->h_up.begin());
    } else {
        lib_kaiser_taps(nt, 60.0, sv->h_down.data());
        lib_kaiser_taps(ntu, 60.0, sv->h_up.data());
    }
    // built-in variant: T = 32 with 4 filters per lane for multi-rate
    // members (small units), 8 for single rate
    sv->variant = desc->tune < 0 ? std::min(-desc->tune - 1, spiir_recur_variant_count() - 1)
                                 : (desc->n_levels > 1 ? 2 : 3);
    // block form: the levels whose push holds whole chunks
    sv->tc_mode = tc;
    sv->bf16 = desc->mode == SPIIR_TC_BF16;
    sv->df = desc->carry == 1;
    sv->tcL = tcL;
    sv->tc_min = desc->tc_min_filters > 0 ? desc->tc_min_filters : 24;
    sv->tcF = tcF;
    sv->tcK = tcF + tcL;
    sv->n_slices = sv->tcK / 64;
    if (tc)
        for (int i = 0; i < sv->L; ++i)
            if ((sv->block >> i) >= tcL && (sv->block >> i) % tcL == 0) {
                sv->tcp[i].on = true;
                sv->n_tc_levels++;
            }
    // the strain history every member can use: the largest delay (the FIR
    // length in the block form) plus the level's alignment delay
    {
        spiir_bank_desc g = e;
        g.h_down = sv->h_down.data();
        g.h_up = sv->h_up.data();
        g.n_taps = nt;
        g.n_taps_up = ntu;
        std::vector<float> one(sv->L, 0.f);
        std::vector<int32_t> dl(sv->L, tc ? tcF : desc->max_delay), tid(sv->L, 0);
        std::vector<int8_t> lv(sv->L);
        for (int i = 0; i < sv->L; ++i) lv[i] = (int8_t)i;
        g.n_filters = sv->L;
        g.a_re = g.a_im = g.b_re = g.b_im = one.data();
        g.delay = dl.data();
        g.template_id = tid.data();
        g.level = lv.data();
        if ((st = make_plan(&g, sv->variant, false, sv->geo))) {
            delete sv;
            return st;
        }
    }
    for (int i = 0; i < sv->L; ++i)
        if (sv->tcp[i].on)
            sv->tcp[i].hist_read = sv->geo.hist[i] - (int)align_delay(i, sv->L, nt, ntu, sv->d.align);
    sv->smem_bytes = sv->geo.smem_bytes;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    auto bail = [&](spiir_status r) {
        sv->release();
        delete sv;
        return r;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return bail(fail(SPIIR_ECUDA, "cudaGetDevice failed"));
    if (cudaDeviceGetAttribute(&sv->n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(fail(SPIIR_ECUDA, "cudaDeviceGetAttribute failed"));
    cudaError_t e1 = spiir_recur_prepare(sv->variant, sv->smem_bytes, &sv->ctas_per_sm);
    if (e1 == cudaSuccess) e1 = spiir_combine_prepare();
    if (e1 != cudaSuccess) return bail(fail(SPIIR_ECUDA, "kernel setup: %s", cudaGetErrorString(e1)));
    if (sv->n_tc_levels > 0) {
        if ((st = spiir_tc_prepare(sv->tcL, sv->tcK))) return bail(fail(st, "%s", spiir_tc_last_error()));
        // staging buffers for the largest level (level 0 holds the most chunks)
        int64_t cmax = 0;
        for (int i = 0; i < sv->L; ++i)
            if (sv->tcp[i].on) cmax = std::max<int64_t>(cmax, (sv->block >> i) / sv->tcL);
        const int64_t hb = spiir_tc_hank_bytes(sv->tcL, sv->tcK);
        const int cpb = spiir_tc_cpb(2, sv->tcL);
        const int64_t nb = std::max<int64_t>((cmax + cpb - 1) / cpb + 1, cmax);
        if (cudaMalloc((void **)&sv->hank, 2 * cmax * hb) != cudaSuccess ||
            cudaMalloc((void **)&sv->xseg, nb * spiir_tc_xseg_bytes()) != cudaSuccess)
            return bail(fail(SPIIR_ENOMEM, "server staging buffers"));
    }
    const int64_t xs = sv->S * sv->geo.xbuf_stream_stride;
    if (cudaMalloc((void **)&sv->xbuf, xs * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&sv->xstage, (int64_t)sv->S * sv->block * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&sv->status, sizeof(unsigned int)) != cudaSuccess)
        return bail(fail(SPIIR_ENOMEM, "server strain buffers"));
    if (cudaMemsetAsync(sv->xbuf, 0, xs * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(sv->status, 0, sizeof(unsigned int), s) != cudaSuccess)
        return bail(fail(SPIIR_ECUDA, "server setup"));
    if ((st = sv->queue.reserve(sv->S, s)) || (st = sv->prog.reserve(sv->S, s))) return bail(st);
    if ((st = relayout_partial(sv, s))) return bail(st);
    if (cudaStreamCreateWithFlags(&sv->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->io, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sv->ev_push, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sv->ev_io, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(SPIIR_ECUDA, "stream or event creation failed"));
    sv->timer = new KernelTimer();
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(SPIIR_ECUDA, "server setup"));
    *out = sv;
    g_err.clear();
    return SPIIR_OK;
}

spiir_status spiir_server_add(spiir_server_t sv, const spiir_bank_desc *member, int32_t *member_id) {
    if (!sv || !member_id) return fail(SPIIR_EINVAL, "NULL argument");
    Member m;
    m.id = sv->next_id;
    spiir_status st = build_member(sv, member, true, m);
    if (st) return st;
    sv->pending_add.push_back(std::move(m));
    *member_id = sv->next_id++;
    sv->dirty = true;
    return SPIIR_OK;
}

spiir_status spiir_server_remove(spiir_server_t sv, int32_t member_id) {
    if (!sv) return fail(SPIIR_EINVAL, "server is NULL");
    for (size_t i = 0; i < sv->pending_add.size(); ++i)
        if (sv->pending_add[i].id == member_id) {
            sv->pending_add.erase(sv->pending_add.begin() + i);
            return SPIIR_OK;
        }
    if (!sv->members.count(member_id) ||
        std::find(sv->pending_remove.begin(), sv->pending_remove.end(), member_id) != sv->pending_remove.end())
        return fail(SPIIR_EINVAL, "no member %d", member_id);
    sv->pending_remove.push_back(member_id);
    sv->dirty = true;
    return SPIIR_OK;
}

int64_t spiir_server_member_footprint(spiir_server_t sv, const spiir_bank_desc *member) {
    if (!sv) return -1;
    Member m;
    if (build_member(sv, member, false, m)) return -1;
    return member_bytes(sv, m);
}

spiir_status spiir_server_prepare(spiir_server_t sv, void *cuda_stream) {
    if (!sv) return fail(SPIIR_EINVAL, "server is NULL");
    spiir_status st;
    if (sv->dirty && (st = apply_changes(sv))) return st;
    if (!(sv->timer && sv->timer->on) && (st = ensure_graph(sv))) return st;
    if (sv->io_pending) {
        CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)cuda_stream, sv->ev_io, 0));
        sv->io_pending = false;
    }
    return SPIIR_OK;
}

spiir_status spiir_server_push(spiir_server_t sv, const float *x_dev, void *cuda_stream) {
    if (!sv || !x_dev) return fail(SPIIR_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    spiir_status st;
    if ((st = spiir_server_prepare(sv, cuda_stream))) return st;
    CUDA_TRY(cudaMemcpyAsync(sv->xstage, x_dev, (int64_t)sv->S * sv->block * sizeof(float),
                             cudaMemcpyDeviceToDevice, s));
    if (sv->timer && sv->timer->on) {
        if ((st = launch_push(sv, sv->pushes > 0 ? sv->block : 0, s))) return st;
    } else {
        CUDA_TRY(cudaGraphLaunch(sv->graph[sv->pushes > 0 ? 1 : 0], s));
    }
    CUDA_TRY(cudaEventRecord(sv->ev_push, s));
    sv->pushed_once = true;
    ++sv->pushes;
    for (auto &kv : sv->members) kv.second.pushed = true;
    return SPIIR_OK;
}

spiir_status spiir_server_enable_timing(spiir_server_t sv, int32_t enable) {
    if (!sv) return fail(SPIIR_EINVAL, "server is NULL");
    sv->timer->flush();
    sv->timer->on = enable != 0;
    for (int k = 0; k < SPIIR_K_COUNT; ++k) {
        sv->timer->ms[k] = 0.0;
        sv->timer->launches[k] = 0;
    }
    return SPIIR_OK;
}

spiir_status spiir_server_kernel_times(spiir_server_t sv, spiir_kernel_times *out) {
    if (!sv || !out) return fail(SPIIR_EINVAL, "NULL argument");
    sv->timer->flush();
    for (int k = 0; k < SPIIR_K_COUNT; ++k) {
        out->ms[k] = sv->timer->ms[k];
        out->launches[k] = sv->timer->launches[k];
        sv->timer->ms[k] = 0.0;
        sv->timer->launches[k] = 0;
    }
    return SPIIR_OK;
}

spiir_status spiir_server_read(spiir_server_t sv, int32_t member_id, void *z_dev, void *cuda_stream) {
    if (!sv || !z_dev) return fail(SPIIR_EINVAL, "NULL argument");
    auto it = sv->members.find(member_id);
    if (it == sv->members.end()) {
        for (const Member &m : sv->pending_add)
            if (m.id == member_id) return fail(SPIIR_ESTATE, "member %d has not taken part in a push", member_id);
        return fail(SPIIR_EINVAL, "no member %d", member_id);
    }
    const Member &m = it->second;
    if (!m.pushed) return fail(SPIIR_ESTATE, "member %d has not taken part in a push", member_id);
    const int64_t row_bytes = (int64_t)sv->block * sizeof(float2);
    CUDA_TRY(cudaMemcpy2DAsync(z_dev, m.T * row_bytes, sv->z + m.row0 * sv->block,
                               sv->row_alloc.cap() * row_bytes, m.T * row_bytes, sv->S,
                               cudaMemcpyDeviceToDevice, (cudaStream_t)cuda_stream));
    return SPIIR_OK;
}

spiir_status spiir_server_get_info(spiir_server_t sv, spiir_server_info *info) {
    if (!sv || !info) return fail(SPIIR_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->n_members = (int32_t)sv->members.size();
    for (auto &kv : sv->members) {
        info->n_templates += kv.second.T;
        info->n_filters += kv.second.n_filters;
        info->filter_samples_per_push += kv.second.fs_per_push;
    }
    int64_t b = sv->S * sv->geo.xbuf_stream_stride * 4 + (int64_t)sv->S * sv->block * 4;
    b += sv->slot_alloc.cap() * (4 * 4 + 4 + 8 * (int64_t)sv->S);
    b += sv->row_alloc.cap() * sv->S * ((int64_t)sv->block + (int64_t)sv->H * SPIIR_UHIST) * 8;
    b += sv->S * sv->part_stream_stride * 8;
    b += sv->tasks.cap * sizeof(WarpTask) + sv->items.cap * sizeof(CtaItem) +
         4 * (sv->order.cap + sv->task_out.cap + sv->comb_ptr.cap + sv->comb_rows.cap + sv->comb_list.cap +
              sv->queue.cap + sv->prog.cap);
    for (int i = 0; i < sv->L; ++i) {
        const TcPool &t = sv->tcp[i];
        if (!t.on) continue;
        b += t.group_alloc.cap() * ((int64_t)sv->n_slices * kTcSliceBytes + 64 * 13);
        b += t.tile_alloc.cap() * (kTcPanelBytes + kTcTile * (32 + 48 + 16 * (int64_t)sv->S));
    }
    info->device_bytes = b;
    info->n_cta_items = sv->n_items;
    info->kernel_variant = sv->variant;
    info->tc_levels = sv->n_tc_levels;
    info->launches_per_push = sv->launches;
    return SPIIR_OK;
}

spiir_status spiir_server_sync_status(spiir_server_t sv) {
    if (!sv) return fail(SPIIR_EINVAL, "server is NULL");
    CUDA_TRY(cudaDeviceSynchronize());
    unsigned int v = 0;
    CUDA_TRY(cudaMemcpy(&v, sv->status, sizeof(v), cudaMemcpyDeviceToHost));
    if (v != SPIIR_DEV_OK) {
        CUDA_TRY(cudaMemset(sv->status, 0, sizeof(unsigned int)));
        return fail(SPIIR_ETIMEOUT, "a device-side wait timed out (status %u)", v);
    }
    return SPIIR_OK;
}

void spiir_server_destroy(spiir_server_t sv) {
    if (!sv) return;
    cudaDeviceSynchronize();
    sv->release();
    delete sv;
}

}  // extern "C"
