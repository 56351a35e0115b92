// C ABI of the batched parametric grid max-flow solver (declared in pmf.h).
// Host-side logic only: argument checks, workspace layout, set-up copies,
// the solve launch sequence (optionally captured once as a CUDA graph and
// replayed), and reading back results.  Every step of the solve itself runs in
// the kernels of pmf_kernels.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "pmf.h"
#include "pmf_internal.h"

using namespace pmf;

namespace {

constexpr size_t ALIGN = 256;
size_t align_up(size_t v, size_t a = ALIGN) { return (v + a - 1) / a * a; }
int round_up_i(int v, int a) { return (v + a - 1) / a * a; }

struct Layout {
    size_t img_planes, inst_planes, masks, dev_inst, ist, tiles, tile_inst, ring, lambdas, flows,
        globals, staging, img_flags, inst_flags, scratch, trace, strip_cache, tmaps, total;
    size_t ring_cap;
    size_t max_tiles;
    size_t max_strips;                          // relabel strips (tile columns x 32-row bands)
    size_t max_hw;
    std::vector<int> rows, pitch;               // per image
    std::vector<int64_t> img_off;               // per image, int32 elements
    std::vector<int64_t> plane_off, mask_off;   // per instance
};

bool desc_ok(const pmf_batch_desc *d) {
    if (!d || d->n_images < 1 || d->n_inst < 1 || d->max_lambdas < 1) return false;
    if (!d->img_h || !d->img_w || !d->inst_image) return false;
    for (int i = 0; i < d->n_images; ++i)
        if (d->img_h[i] < 1 || d->img_w[i] < 1 || (int64_t)d->img_h[i] * d->img_w[i] > (1 << 28)) return false;
    for (int i = 0; i < d->n_inst; ++i)
        if (d->inst_image[i] < 0 || d->inst_image[i] >= d->n_images) return false;
    return true;
}

Layout make_layout(const pmf_batch_desc *d) {
    Layout L;
    L.rows.resize(d->n_images);
    L.pitch.resize(d->n_images);
    L.img_off.resize(d->n_images);
    size_t img_elems = 0;
    L.max_hw = 0;
    for (int i = 0; i < d->n_images; ++i) {
        L.rows[i] = round_up_i(d->img_h[i], ROW_ALIGN);
        L.pitch[i] = round_up_i(d->img_w[i], TILE_W);
        L.img_off[i] = (int64_t)img_elems;
        img_elems += (size_t)N_IMG_PLANES * L.rows[i] * L.pitch[i];
        L.max_hw = std::max(L.max_hw, (size_t)d->img_h[i] * d->img_w[i]);
    }
    L.plane_off.resize(d->n_inst);
    L.mask_off.resize(d->n_inst);
    size_t inst_elems = 0, mask_bytes = 0;
    L.max_tiles = 0;
    L.max_strips = 0;
    for (int i = 0; i < d->n_inst; ++i) {
        const int im = d->inst_image[i];
        const size_t ps = (size_t)L.rows[im] * L.pitch[im];
        L.plane_off[i] = (int64_t)inst_elems;
        inst_elems += (size_t)N_INST_PLANES * ps;
        L.mask_off[i] = (int64_t)mask_bytes;
        mask_bytes += (size_t)d->max_lambdas * ps;
        L.max_tiles += (size_t)(L.rows[im] / 4) * ((d->img_w[im] + TILE_IN - 1) / TILE_IN);   // smallest tile height
        L.max_strips += (size_t)((L.rows[im] + BFS_ROWS - 1) / BFS_ROWS) * ((d->img_w[im] + TILE_IN - 1) / TILE_IN);
    }
    // every tile can be queued once, and every resident warp may hold a ticket
    L.ring_cap = 1;
    while (L.ring_cap < L.max_tiles + 16384) L.ring_cap <<= 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes); return o; };
    L.img_planes = take(img_elems * 4);
    L.inst_planes = take(inst_elems * 4);
    L.masks = take(mask_bytes);
    L.dev_inst = take(sizeof(DevInst) * d->n_inst);
    L.ist = take(sizeof(InstState) * d->n_inst);
    L.tiles = take(sizeof(TileState) * L.max_tiles);
    L.tile_inst = take(sizeof(int32_t) * L.max_tiles);
    L.ring = take(sizeof(int32_t) * L.ring_cap);
    L.lambdas = take(sizeof(int32_t) * (size_t)d->n_inst * d->max_lambdas);
    L.flows = take(sizeof(int64_t) * (size_t)d->n_inst * d->max_lambdas);
    L.globals = take(sizeof(Globals));
    L.staging = take(sizeof(int32_t) * 3 * L.max_hw);
    L.img_flags = take(sizeof(int32_t) * d->n_images);
    L.inst_flags = take(sizeof(int32_t) * d->n_inst);
    L.scratch = take(256);                        // small device results (status words)
    L.trace = take(sizeof(TraceEvent) * TRACE_CAP);
    L.strip_cache = take(sizeof(int32_t) * STRIP_REC_WORDS * L.max_strips);
    L.tmaps = take((size_t)TMAP_BYTES * (d->n_inst + d->n_images));
    L.total = off;
    return L;
}

// Pinned host memory for the batches' small result mirrors comes from one
// process-wide arena: page-locked allocation and release synchronise the whole
// device, so a batch created or destroyed while others run on the GPU must not
// call cudaHostAlloc / cudaFreeHost.  Chunks are allocated once and reused.
class PinnedArena {
public:
    void *alloc(size_t n) {
        n = align_up(n);
        std::lock_guard<std::mutex> g(mu_);
        for (Chunk &c : chunks_) {
            for (size_t i = 0; i < c.free.size(); ++i) {
                if (c.free[i].second >= n) {
                    char *p = c.base + c.free[i].first;
                    c.free[i].first += n;
                    c.free[i].second -= n;
                    if (c.free[i].second == 0) c.free.erase(c.free.begin() + (long)i);
                    return p;
                }
            }
        }
        const size_t sz = std::max<size_t>(n, (size_t)16 << 20);
        void *base = nullptr;
        if (cudaHostAlloc(&base, sz, cudaHostAllocPortable) != cudaSuccess) return nullptr;
        chunks_.push_back(Chunk{(char *)base, sz, {{n, sz - n}}});
        if (chunks_.back().free.back().second == 0) chunks_.back().free.pop_back();
        return base;
    }
    void release(void *p, size_t n) {
        if (!p) return;
        n = align_up(n);
        std::lock_guard<std::mutex> g(mu_);
        for (Chunk &c : chunks_) {
            char *q = (char *)p;
            if (q < c.base || q >= c.base + c.size) continue;
            const size_t off = (size_t)(q - c.base);
            auto it = c.free.begin();
            while (it != c.free.end() && it->first < off) ++it;
            it = c.free.insert(it, {off, n});
            // merge with the following and the preceding free block
            if (it + 1 != c.free.end() && it->first + it->second == (it + 1)->first) {
                it->second += (it + 1)->second;
                c.free.erase(it + 1);
            }
            if (it != c.free.begin() && (it - 1)->first + (it - 1)->second == it->first) {
                (it - 1)->second += it->second;
                c.free.erase(it);
            }
            return;
        }
    }

private:
    struct Chunk {
        char *base;
        size_t size;
        std::vector<std::pair<size_t, size_t>> free;   // (offset, length), sorted
    };
    std::mutex mu_;
    std::vector<Chunk> chunks_;
};

PinnedArena &pinned_arena() {
    static PinnedArena *a = new PinnedArena();   // lives until exit (chunks are never returned)
    return *a;
}

struct DeviceGuard {
    int old = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&old) != cudaSuccess) old = -1;
        if (old != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (old >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != old) cudaSetDevice(old);
    }
};

}  // namespace

struct pmf_batch {
    pmf_batch_desc desc{};
    std::vector<int32_t> img_h, img_w, inst_image;
    Layout L;
    char *ws = nullptr;
    Params P{};
    pmf_tuning tune{};
    int n_sm = 0;
    int device = 0;
    cudaStream_t setup_stream = nullptr;   // caller's stream for set-up copies
    cudaStream_t cap_stream = nullptr;     // private stream used for graph capture
    cudaEvent_t done = nullptr;
    cudaEvent_t ev_t0 = nullptr, ev_w0 = nullptr, ev_w1 = nullptr, ev_t1 = nullptr;   // timing
    float worker_ms_rounds = 0.f;
    bool in_flight = false;
    bool solved = false;
    bool forks_changed = false;            // pmf_set_fork since the last geometry upload
    std::vector<int32_t> n_lam;            // schedule length of each instance in the last solve
    std::vector<DevInst> dinst;            // host copy of the descriptors
    // pinned host mirrors
    int32_t *lam_h = nullptr;
    InstState *ist_h = nullptr;
    long long *flows_h = nullptr;
    Globals *glob_h = nullptr;
    DevInst *dinst_h = nullptr;
    int32_t *done_h = nullptr;             // written by the kernel: 1 + status of each finished instance
    size_t pinned_bytes[6] = {0, 0, 0, 0, 0, 0};
    // captured graph
    cudaGraphExec_t gexec = nullptr;
    bool graph_valid = false;
    int worker_grid = 0;
    bool stage_ok = false;                 // tensor maps encoded: staged strip loads available
};

namespace pmf {

thread_local char g_last_error[256] = "";

pmf_status cuda_err_at(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return PMF_OK;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    return PMF_ERR_CUDA;
}

}  // namespace pmf

namespace {

#define cuda_err(e) cuda_err_at((e), __func__)

void apply_defaults(pmf_tuning *t) {
    if (t->tile_h != 4 && t->tile_h != 8) t->tile_h = 8;
    if (t->sweeps <= 0) t->sweeps = 8;
    if (t->relabel_every <= 0) t->relabel_every = 800;
    if (t->max_visits_per_tile <= 0) t->max_visits_per_tile = 2000;
    if (t->mode != 1) t->mode = 0;
    if (t->use_graph != 0) t->use_graph = 1;
    t->trace = t->trace ? 1 : 0;
    if (t->poll_ns <= 0) t->poll_ns = 256;
    if (t->label_slack == 0) t->label_slack = 16;
    if (t->label_slack < 0) t->label_slack = -1;
    if (t->push_order != 1) t->push_order = 0;
    if (t->relabel_extra < 0) t->relabel_extra = 0;
    if (t->relabel_reach < 0) t->relabel_reach = 0;
    if (t->strip_stage != 1) t->strip_stage = -1;
}

// per-instance tile geometry for the current tile height; uploads the table
pmf_status refresh_geometry(pmf_batch *b, cudaStream_t s) {
    const int th = b->tune.tile_h;
    const int span = BFS_ROWS / th;
    int base = 0;
    for (int i = 0; i < b->desc.n_inst; ++i) {
        const int im = b->inst_image[i];
        DevInst &d = b->dinst[i];
        d.H = b->img_h[im];
        d.W = b->img_w[im];
        d.rows = b->L.rows[im];
        d.pitch = b->L.pitch[im];
        d.image = im;
        d.tiles_x = (d.W + TILE_IN - 1) / TILE_IN;
        d.tiles_y = d.rows / th;
        d.n_tiles = d.tiles_x * d.tiles_y;
        d.tile_base = base;
        base += d.n_tiles;
        d.n_leads = d.tiles_x * ((d.tiles_y + span - 1) / span);
        d.hcap = d.H * d.W + 1;
        d.plane_off = b->L.plane_off[i];
        d.img_off = b->L.img_off[im];
        d.mask_off = b->L.mask_off[i];
        b->dinst_h[i] = d;
    }
    // the first relabel strips enter the queue largest instance first (a
    // longest-processing-time order: the biggest grids start earliest, so the
    // small ones fill in at the end instead of a big one running alone);
    // forked instances, which wait for their parent, are numbered last
    std::vector<int> order(b->desc.n_inst);
    for (int i = 0; i < b->desc.n_inst; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const bool wa = b->dinst_h[a].fork_parent >= 0, wc = b->dinst_h[c].fork_parent >= 0;
        if (wa != wc) return wc;
        return b->dinst_h[a].n_tiles > b->dinst_h[c].n_tiles;
    });
    int lbase = 0, queued = 0;
    for (int i : order) {
        b->dinst_h[i].lead_base = lbase;
        b->dinst[i].lead_base = lbase;
        lbase += b->dinst_h[i].n_leads;
        if (b->dinst_h[i].fork_parent < 0) queued = lbase;
    }
    b->P.n_tiles_total = base;
    b->P.n_leads_total = lbase;
    b->P.n_leads_queued = queued;
    b->forks_changed = false;
    b->P.tile_h = th;
    return cuda_err(cudaMemcpyAsync(b->ws + b->L.dev_inst, b->dinst_h, sizeof(DevInst) * b->desc.n_inst,
                                    cudaMemcpyHostToDevice, s));
}

int grid_size(pmf_batch *b) {
    if (b->tune.grid_blocks > 0) return b->tune.grid_blocks;
    int bps = b->tune.blocks_per_sm;
    if (bps <= 0) {
        if (worker_occupancy(b->tune.tile_h, &bps, b->P.strip_stage != 0) != cudaSuccess || bps <= 0) bps = 4;
    }
    return bps * b->n_sm;
}

// the launch sequence of one solve (persistent mode)
pmf_status enqueue_solve(pmf_batch *b, cudaStream_t s, bool capturing) {
    // inside a stream capture the timing events become event-record nodes
    auto rec = [&](cudaEvent_t ev) {
        return capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
    };
    const size_t lam_bytes = sizeof(int32_t) * (size_t)b->desc.n_inst * b->desc.max_lambdas;
    cudaError_t e = cudaMemcpyAsync(b->ws + b->L.lambdas, b->lam_h, lam_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = rec(b->ev_t0);
    if (e == cudaSuccess) e = launch_reset(b->P, s);
    int maxpix = 0;
    for (int i = 0; i < b->desc.n_inst; ++i) maxpix = std::max(maxpix, b->dinst[i].rows * b->dinst[i].pitch);
    if (e == cudaSuccess) e = launch_init(b->P, maxpix, s);
    if (e == cudaSuccess) e = rec(b->ev_w0);
    if (e == cudaSuccess) e = launch_worker(b->P, b->worker_grid, s);
    if (e == cudaSuccess) e = rec(b->ev_w1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ist_h, b->ws + b->L.ist, sizeof(InstState) * b->desc.n_inst, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->flows_h, b->ws + b->L.flows, sizeof(long long) * (size_t)b->desc.n_inst * b->desc.max_lambdas,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->glob_h, b->ws + b->L.globals, sizeof(Globals), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = rec(b->ev_t1);
    return cuda_err(e);
}

}  // namespace

extern "C" {

const char *pmf_version(void) { return "pmf 0.1.0 sm_103a"; }

const char *pmf_last_error(void) { return g_last_error; }

const char *pmf_status_string(pmf_status s) {
    switch (s) {
        case PMF_OK: return "ok";
        case PMF_ERR_INVALID_ARG: return "invalid argument";
        case PMF_ERR_OUT_OF_MEMORY: return "workspace too small";
        case PMF_ERR_NOT_MONOTONE: return "lambda schedule decreasing or negative slope";
        case PMF_ERR_OVERFLOW: return "capacity above the supported maximum";
        case PMF_ERR_CUDA: return "CUDA runtime error";
        case PMF_ERR_NOT_CONVERGED: return "watchdog stopped the solve";
        case PMF_ERR_NOT_READY: return "no finished solve";
    }
    return "unknown status";
}

pmf_status pmf_workspace_size(const pmf_batch_desc *desc, size_t *bytes) {
    if (!desc_ok(desc) || !bytes) return PMF_ERR_INVALID_ARG;
    *bytes = make_layout(desc).total;
    return PMF_OK;
}

pmf_status pmf_create_batch(const pmf_batch_desc *desc, void *dev_workspace, size_t bytes,
                            void *cuda_stream, pmf_batch **out) {
    if (!out) return PMF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc_ok(desc) || !dev_workspace) return PMF_ERR_INVALID_ARG;
    if (((uintptr_t)dev_workspace) % ALIGN) return PMF_ERR_INVALID_ARG;
    Layout L = make_layout(desc);
    if (bytes < L.total) return PMF_ERR_OUT_OF_MEMORY;
    DeviceGuard dg(desc->device);
    pmf_batch *b = new (std::nothrow) pmf_batch();
    if (!b) return PMF_ERR_OUT_OF_MEMORY;
    b->desc = *desc;
    b->img_h.assign(desc->img_h, desc->img_h + desc->n_images);
    b->img_w.assign(desc->img_w, desc->img_w + desc->n_images);
    b->inst_image.assign(desc->inst_image, desc->inst_image + desc->n_inst);
    b->desc.img_h = b->img_h.data();
    b->desc.img_w = b->img_w.data();
    b->desc.inst_image = b->inst_image.data();
    b->L = L;
    b->ws = (char *)dev_workspace;
    b->device = desc->device;
    b->setup_stream = (cudaStream_t)cuda_stream;
    b->dinst.resize(desc->n_inst);
    for (DevInst &d : b->dinst) {
        std::memset(&d, 0, sizeof(d));
        d.fork_parent = d.fork_child = d.fork_k = -1;
    }
    b->n_lam.assign(desc->n_inst, 0);
    apply_defaults(&b->tune);
    cudaError_t e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    const size_t nl = (size_t)desc->n_inst * desc->max_lambdas;
    b->pinned_bytes[0] = sizeof(int32_t) * nl;
    b->pinned_bytes[1] = sizeof(InstState) * desc->n_inst;
    b->pinned_bytes[2] = sizeof(long long) * nl;
    b->pinned_bytes[3] = sizeof(Globals);
    b->pinned_bytes[4] = sizeof(DevInst) * desc->n_inst;
    b->pinned_bytes[5] = sizeof(int32_t) * desc->n_inst;
    void **dst[6] = {(void **)&b->lam_h, (void **)&b->ist_h, (void **)&b->flows_h, (void **)&b->glob_h,
                     (void **)&b->dinst_h, (void **)&b->done_h};
    for (int j = 0; j < 6 && e == cudaSuccess; ++j) {
        *dst[j] = pinned_arena().alloc(b->pinned_bytes[j]);
        if (!*dst[j]) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_w0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_w1);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_t1);
    if (e != cudaSuccess) {
        pmf_destroy_batch(b);
        return PMF_ERR_CUDA;
    }
    Params &P = b->P;
    P.planes = (int32_t *)(b->ws + L.inst_planes);
    P.img = (const int32_t *)(b->ws + L.img_planes);
    P.masks = (uint8_t *)(b->ws + L.masks);
    P.inst = (const DevInst *)(b->ws + L.dev_inst);
    P.ist = (InstState *)(b->ws + L.ist);
    P.tiles = (TileState *)(b->ws + L.tiles);
    P.tile_inst = (const int32_t *)(b->ws + L.tile_inst);
    P.ring = (int32_t *)(b->ws + L.ring);
    P.strip_cache = (int32_t *)(b->ws + L.strip_cache);
    P.lambdas = (const int32_t *)(b->ws + L.lambdas);
    P.flows = (long long *)(b->ws + L.flows);
    P.g = (Globals *)(b->ws + L.globals);
    P.img_flags = (const int32_t *)(b->ws + L.img_flags);
    P.inst_flags = (int32_t *)(b->ws + L.inst_flags);
    {
        // pinned host memory is addressable from the device (unified addressing)
        void *dp = nullptr;
        P.done_flags = cudaHostGetDevicePointer(&dp, b->done_h, 0) == cudaSuccess ? (int32_t *)dp : nullptr;
        std::memset(b->done_h, 0, b->pinned_bytes[5]);
    }
    P.ring_mask = (unsigned long long)(L.ring_cap - 1);
    P.n_inst = desc->n_inst;
    P.max_lambdas = desc->max_lambdas;
    P.stall_ns = 5000000000LL;
    P.max_ns = 120000000000LL;
    if (const char *ev = getenv("PMF_MAX_SECONDS")) {
        const double sec = atof(ev);
        if (sec > 0) P.max_ns = (long long)(sec * 1e9);
    }
    // zero the parts that are read before being written: planes (capacities
    // not set stay zero), flags
    cudaStream_t s = b->setup_stream;
    e = cudaMemsetAsync(b->ws + L.img_planes, 0, L.masks - L.img_planes, s);
    // flags, scratch and trace start zeroed (the strip records after them are
    // always written by a strip's first visit of an epoch before they are read)
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + L.img_flags, 0, L.strip_cache - L.img_flags, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + L.globals, 0, sizeof(Globals), s);
    if (e == cudaSuccess) {
        const pmf_status st = refresh_geometry(b, s);
        if (st != PMF_OK) e = cudaErrorUnknown;
    }
    // tensor maps of the planes for staged strip loads (the workspace does not
    // move for the batch's lifetime); without an encoder the loads stay per lane
    std::vector<unsigned char> maps((size_t)TMAP_BYTES * (desc->n_inst + desc->n_images));
    if (e == cudaSuccess) {
        std::vector<int> rows(L.rows.begin(), L.rows.end()), pitch(L.pitch.begin(), L.pitch.end());
        b->stage_ok = encode_plane_maps(maps.data(), P.planes, P.img, desc->n_inst, L.plane_off.data(),
                                        b->inst_image.data(), desc->n_images, L.img_off.data(), rows.data(),
                                        pitch.data()) &&
                      prepare_stage_kernels() == cudaSuccess;
        (void)cudaGetLastError();
        if (b->stage_ok) e = cudaMemcpyAsync(b->ws + L.tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice, s);
    }
    P.tmaps = (const unsigned char *)(b->ws + L.tmaps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        pmf_destroy_batch(b);
        return PMF_ERR_CUDA;
    }
    *out = b;
    return PMF_OK;
}

pmf_status pmf_set_tuning(pmf_batch *b, const pmf_tuning *t) {
    if (!b || !t) return PMF_ERR_INVALID_ARG;
    if (t->tile_h != 0 && t->tile_h != 4 && t->tile_h != 8) return PMF_ERR_INVALID_ARG;
    if (t->sweeps < 0 || t->relabel_every < 0 || t->max_visits_per_tile < 0 || t->blocks_per_sm < 0 ||
        t->grid_blocks < 0)
        return PMF_ERR_INVALID_ARG;
    if (b->in_flight) {
        DeviceGuard dg(b->device);
        cudaEventSynchronize(b->done);
        b->in_flight = false;
    }
    pmf_tuning n = *t;
    apply_defaults(&n);
    b->tune = n;
    b->graph_valid = false;   // re-capture on next solve
    return PMF_OK;
}

pmf_status pmf_get_tuning(const pmf_batch *b, pmf_tuning *t) {
    if (!b || !t) return PMF_ERR_INVALID_ARG;
    *t = b->tune;
    return PMF_OK;
}

// status of the padding kernels' validation flags, in the order the device
// reports them (a negative slope first, then a capacity out of range, then a
// negative capacity)
static pmf_status host_flags_status(int32_t f) {
    if (f & VF_SLOPE) return PMF_ERR_NOT_MONOTONE;
    if (f & VF_OVERFLOW) return PMF_ERR_OVERFLOW;
    if (f & VF_NEG) return PMF_ERR_INVALID_ARG;
    return PMF_OK;
}

pmf_status pmf_set_capacities(pmf_batch *b, int32_t image, const int32_t *w_h, const int32_t *w_v,
                              int on_device) {
    if (!b || !w_h || !w_v || image < 0 || image >= b->desc.n_images) return PMF_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    if (b->in_flight) { cudaEventSynchronize(b->done); b->in_flight = false; }
    const int H = b->img_h[image], W = b->img_w[image];
    const size_t n = (size_t)H * W;
    cudaStream_t s = b->setup_stream;
    const int32_t *src_h = w_h, *src_v = w_v;
    if (!on_device) {
        // checked on the device by the padding kernel, the result read back below
        int32_t *stg = (int32_t *)(b->ws + b->L.staging);
        cudaError_t e = cudaMemcpyAsync(stg, w_h, n * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(stg + n, w_v, n * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return PMF_ERR_CUDA;
        src_h = stg;
        src_v = stg + n;
    }
    DevInst d{};
    d.H = H;
    d.W = W;
    d.rows = b->L.rows[image];
    d.pitch = b->L.pitch[image];
    d.img_off = b->L.img_off[image];
    int32_t *flags = (int32_t *)(b->ws + b->L.img_flags) + image;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_pad_image(b->P, image, d, src_h, src_v, flags, s);
    b->solved = false;
    if (e != cudaSuccess || on_device) return cuda_err(e);
    int32_t f = 0;
    e = cudaMemcpyAsync(&f, flags, sizeof(f), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    return host_flags_status(f);
}

pmf_status pmf_copy_terminals(pmf_batch *b, int32_t dst, int32_t src) {
    if (!b || dst < 0 || dst >= b->desc.n_inst || src < 0 || src >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    if (b->inst_image[dst] != b->inst_image[src]) return PMF_ERR_INVALID_ARG;
    if (dst == src) return PMF_OK;
    DeviceGuard dg(b->device);
    if (b->in_flight) { cudaEventSynchronize(b->done); b->in_flight = false; }
    const DevInst &ds = b->dinst[src], &dd = b->dinst[dst];
    const size_t ps = (size_t)ds.rows * ds.pitch;
    // src0, slope and ct are consecutive planes of an instance: one copy, and
    // the validation flags with them (pmf_sync reports them as for src)
    int32_t *planes = (int32_t *)(b->ws + b->L.inst_planes);
    int32_t *flags = (int32_t *)(b->ws + b->L.inst_flags);
    cudaStream_t s = b->setup_stream;
    cudaError_t e = cudaMemcpyAsync(planes + dd.plane_off + P_SRC0 * ps, planes + ds.plane_off + P_SRC0 * ps,
                                    3 * ps * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(flags + dst, flags + src, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    b->solved = false;
    return cuda_err(e);
}

pmf_status pmf_set_cut_rule(pmf_batch *b, int32_t inst, int32_t rule) {
    if (!b || inst < 0 || inst >= b->desc.n_inst || (rule != 0 && rule != 1)) return PMF_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    if (b->in_flight) { cudaEventSynchronize(b->done); b->in_flight = false; }
    b->dinst[inst].cut_rule = (int16_t)rule;
    b->dinst_h[inst].cut_rule = (int16_t)rule;
    cudaStream_t s = b->setup_stream;
    cudaError_t e = cudaMemcpyAsync(b->ws + b->L.dev_inst + sizeof(DevInst) * inst, &b->dinst_h[inst],
                                    sizeof(DevInst), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_err(e);
}

pmf_status pmf_set_slope_side(pmf_batch *b, int32_t inst, int32_t side) {
    if (!b || inst < 0 || inst >= b->desc.n_inst || (side != 0 && side != 1)) return PMF_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    if (b->in_flight) { cudaEventSynchronize(b->done); b->in_flight = false; }
    b->dinst[inst].slope_side = (int16_t)side;
    b->dinst_h[inst].slope_side = (int16_t)side;
    b->graph_valid = false;   // the worker kernel is chosen by whether any instance has side 1
    cudaStream_t s = b->setup_stream;
    cudaError_t e = cudaMemcpyAsync(b->ws + b->L.dev_inst + sizeof(DevInst) * inst, &b->dinst_h[inst],
                                    sizeof(DevInst), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_err(e);
}

pmf_status pmf_set_fork(pmf_batch *b, int32_t child, int32_t parent, int32_t parent_step) {
    if (!b || child < 0 || child >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    if (parent >= 0) {
        if (parent >= b->desc.n_inst || parent == child || parent_step < 0) return PMF_ERR_INVALID_ARG;
        if (b->inst_image[parent] != b->inst_image[child]) return PMF_ERR_INVALID_ARG;
        const int other = b->dinst[parent].fork_child;
        if (other >= 0 && other != child) return PMF_ERR_INVALID_ARG;   // one child per parent
    }
    DeviceGuard dg(b->device);
    if (b->in_flight) { cudaEventSynchronize(b->done); b->in_flight = false; }
    const int old = b->dinst[child].fork_parent;
    if (old >= 0) {
        b->dinst[old].fork_child = -1;
        b->dinst[old].fork_k = -1;
    }
    b->dinst[child].fork_parent = parent >= 0 ? parent : -1;
    if (parent >= 0) {
        b->dinst[parent].fork_child = child;
        b->dinst[parent].fork_k = parent_step;
    }
    b->forks_changed = true;   // uploaded with the descriptors at the next solve
    b->solved = false;
    return PMF_OK;
}

pmf_status pmf_set_terminals(pmf_batch *b, int32_t inst, const int32_t *src0, const int32_t *slope,
                             const int32_t *sink, int on_device) {
    if (!b || !src0 || !slope || !sink || inst < 0 || inst >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    if (b->in_flight) { cudaEventSynchronize(b->done); b->in_flight = false; }
    const int im = b->inst_image[inst];
    const int H = b->img_h[im], W = b->img_w[im];
    const size_t n = (size_t)H * W;
    cudaStream_t s = b->setup_stream;
    const int32_t *a = src0, *c = slope, *k = sink;
    if (!on_device) {
        // host arrays are checked on the device by the padding kernel (a host
        // loop is memory-bound at ~10 GB/s on one core) and the result is
        // read back before returning
        int32_t *stg = (int32_t *)(b->ws + b->L.staging);
        cudaError_t e = cudaMemcpyAsync(stg, src0, n * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(stg + n, slope, n * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(stg + 2 * n, sink, n * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return PMF_ERR_CUDA;
        a = stg;
        c = stg + n;
        k = stg + 2 * n;
    }
    DevInst d = b->dinst[inst];
    int32_t *flag_d = (int32_t *)(b->ws + b->L.inst_flags) + inst;
    cudaError_t e = cudaMemsetAsync(flag_d, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_pad_terminals(b->P, inst, d, a, c, k, s);
    b->solved = false;
    if (e != cudaSuccess || on_device) return cuda_err(e);
    int32_t flags = 0;
    e = cudaMemcpyAsync(&flags, flag_d, sizeof(flags), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    return host_flags_status(flags);
}

// Both entry points: instance i solves lambdas[i * stride + 0 .. len(i) - 1],
// len(i) = lengths ? lengths[i] : stride.
static pmf_status solve_impl(pmf_batch *b, const int32_t *lambdas, const int32_t *lengths, int32_t stride,
                             void *cuda_stream) {
    if (!b || !lambdas || stride < 1 || stride > b->desc.max_lambdas) return PMF_ERR_INVALID_ARG;
    auto len = [&](int i) { return lengths ? lengths[i] : stride; };
    for (int i = 0; i < b->desc.n_inst; ++i)
        if (len(i) < 1 || len(i) > stride) return PMF_ERR_INVALID_ARG;
    for (int i = 0; i < b->desc.n_inst; ++i)
        for (int k = 1; k < len(i); ++k)
            if (lambdas[(size_t)i * stride + k] < lambdas[(size_t)i * stride + k - 1]) return PMF_ERR_NOT_MONOTONE;
    // forks: the parent has the step it forks at, the child's schedule goes on
    // from the parent's lambda there (a decrease is PMF_ERR_NOT_MONOTONE), both
    // follow lambda on the same side with the same cut rule, and no chain of
    // forks closes on itself (its instances would all wait)
    for (int c = 0; c < b->desc.n_inst; ++c) {
        const int par = b->dinst[c].fork_parent;
        if (par < 0) continue;
        const int k = b->dinst[par].fork_k;
        if (k < 0 || k >= len(par)) return PMF_ERR_INVALID_ARG;
        if (b->dinst[par].slope_side != b->dinst[c].slope_side || b->dinst[par].cut_rule != b->dinst[c].cut_rule)
            return PMF_ERR_INVALID_ARG;
        int a = par, steps = 0;
        while (a >= 0 && a != c && steps <= b->desc.n_inst) { a = b->dinst[a].fork_parent; ++steps; }
        if (a == c) return PMF_ERR_INVALID_ARG;
    }
    for (int c = 0; c < b->desc.n_inst; ++c) {
        const int par = b->dinst[c].fork_parent;
        if (par >= 0 && lambdas[(size_t)c * stride] < lambdas[(size_t)par * stride + b->dinst[par].fork_k])
            return PMF_ERR_NOT_MONOTONE;
    }
    DeviceGuard dg(b->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (b->in_flight) { cudaEventSynchronize(b->done); b->in_flight = false; }
    std::memset(b->done_h, 0, b->pinned_bytes[5]);
    // lambda table [n_inst][max_lambdas] in pinned staging (the last value
    // repeated past an instance's length)
    for (int i = 0; i < b->desc.n_inst; ++i)
        for (int k = 0; k < b->desc.max_lambdas; ++k)
            b->lam_h[(size_t)i * b->desc.max_lambdas + k] = lambdas[(size_t)i * stride + std::min(k, len(i) - 1)];
    bool len_changed = false;
    for (int i = 0; i < b->desc.n_inst; ++i) len_changed |= b->n_lam[i] != len(i);
    b->P.trace = b->tune.trace ? (TraceEvent *)(b->ws + b->L.trace) : nullptr;
    b->P.sweeps = b->tune.sweeps;
    b->P.poll_ns = b->tune.poll_ns;
    b->P.label_slack = b->tune.label_slack < 0 ? 0 : b->tune.label_slack;
    b->P.chain_push = b->tune.push_order;
    b->P.relabel_pct = b->tune.relabel_every;
    b->P.relabel_extra = b->tune.relabel_extra;
    b->P.relabel_reach = b->tune.relabel_reach;
    b->P.any_sink_side = 0;
    for (int i = 0; i < b->desc.n_inst; ++i) b->P.any_sink_side |= b->dinst[i].slope_side != 0;
    b->P.max_visits_per_tile = b->tune.max_visits_per_tile;
    b->P.strip_stage = (b->tune.strip_stage == 1 && b->stage_ok) ? 1 : 0;
    const bool geo_changed = (b->P.tile_h != b->tune.tile_h) || len_changed || b->forks_changed;
    if (geo_changed) {
        // tile geometry and schedule lengths live in the descriptor table
        for (int i = 0; i < b->desc.n_inst; ++i) b->dinst[i].n_lambda = b->n_lam[i] = len(i);
        const pmf_status st = refresh_geometry(b, s);
        if (st != PMF_OK) return st;
        b->graph_valid = false;
    }
    b->worker_grid = grid_size(b);
    // grids of 1-3 blocks per SM at tile height 4 run the build that spends
    // the registers the fourth block would have had (no spills)
    b->P.wide_regs = (b->tune.tile_h == 4 && b->tune.grid_blocks <= 0 && b->tune.blocks_per_sm >= 1 &&
                      b->tune.blocks_per_sm <= 3) ? 1 : 0;
    b->solved = false;
    cudaError_t e = cudaSuccess;
    if (b->tune.mode == 1) {
        // host-polled rounds: one worker launch per round, the host reads the
        // number of finished instances after each (the one-call-per-iteration form)
        const size_t lam_bytes = sizeof(int32_t) * (size_t)b->desc.n_inst * b->desc.max_lambdas;
        e = cudaMemcpyAsync(b->ws + b->L.lambdas, b->lam_h, lam_bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_t0, s);
        b->worker_ms_rounds = 0.f;
        if (e == cudaSuccess) e = launch_reset(b->P, s);
        int maxpix = 0;
        for (int i = 0; i < b->desc.n_inst; ++i) maxpix = std::max(maxpix, b->dinst[i].rows * b->dinst[i].pitch);
        if (e == cudaSuccess) e = launch_init(b->P, maxpix, s);
        const auto t0 = std::chrono::steady_clock::now();
        for (long long round = 0; e == cudaSuccess && round < (1LL << 24); ++round) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el * 1e9 > (double)b->P.max_ns) break;
            e = launch_begin_round(b->P, s);
            if (e == cudaSuccess) e = cudaEventRecord(b->ev_w0, s);
            if (e == cudaSuccess) e = launch_worker(b->P, b->worker_grid, s);
            if (e == cudaSuccess) e = cudaEventRecord(b->ev_w1, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(b->glob_h, b->ws + b->L.globals, sizeof(Globals), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            float ms = 0.f;
            if (e == cudaSuccess && cudaEventElapsedTime(&ms, b->ev_w0, b->ev_w1) == cudaSuccess) b->worker_ms_rounds += ms;
            if (e != cudaSuccess || b->glob_h->inst_done >= b->desc.n_inst || b->glob_h->err) break;
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->ist_h, b->ws + b->L.ist, sizeof(InstState) * b->desc.n_inst, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->flows_h, b->ws + b->L.flows, sizeof(long long) * (size_t)b->desc.n_inst * b->desc.max_lambdas,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->glob_h, b->ws + b->L.globals, sizeof(Globals), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_t1, s);
    } else if (b->tune.use_graph) {
        // the kernel parameters are baked into the graph: set_tuning and a
        // geometry change invalidate it (graph_valid = false)
        if (!b->graph_valid || !b->gexec) {
            if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const pmf_status st = enqueue_solve(b, b->cap_stream, true);
                const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
                e = (st != PMF_OK) ? cudaErrorUnknown : e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) { b->gexec = nullptr; return cuda_err_at(e, "graph capture"); }
            b->graph_valid = true;
        }
        e = cudaGraphLaunch(b->gexec, s);
    } else {
        const pmf_status st = enqueue_solve(b, s, false);
        if (st != PMF_OK) return st;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->done, s);
    if (e != cudaSuccess) return cuda_err_at(e, "solve launch");
    b->in_flight = true;
    return PMF_OK;
}

pmf_status pmf_solve_schedule(pmf_batch *b, const int32_t *lambdas, int32_t n_lambda, void *cuda_stream) {
    return solve_impl(b, lambdas, nullptr, n_lambda, cuda_stream);
}

pmf_status pmf_solve_schedules(pmf_batch *b, const int32_t *lambdas, const int32_t *lengths, int32_t stride,
                               void *cuda_stream) {
    if (!lengths) return PMF_ERR_INVALID_ARG;
    return solve_impl(b, lambdas, lengths, stride, cuda_stream);
}

pmf_status pmf_sync(pmf_batch *b, pmf_status *per_instance) {
    if (!b) return PMF_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    if (!b->in_flight && !b->solved) return PMF_ERR_NOT_READY;
    if (b->in_flight) {
        const cudaError_t e = cudaEventSynchronize(b->done);
        b->in_flight = false;
        if (e != cudaSuccess) return PMF_ERR_CUDA;
        b->solved = true;
    }
    pmf_status all = PMF_OK;
    const bool gerr = b->glob_h->err != 0;
    const bool internal = (b->glob_h->err & GE_INTERNAL_MASK) != 0;
    for (int i = 0; i < b->desc.n_inst; ++i) {
        pmf_status st = (pmf_status)b->ist_h[i].status;
        if (internal && st == PMF_OK) st = PMF_ERR_NOT_CONVERGED;
        if (st == PMF_OK && (b->ist_h[i].phase != PH_DONE || b->ist_h[i].k < b->n_lam[i]))
            st = PMF_ERR_NOT_CONVERGED;
        if (gerr && st == PMF_OK && b->ist_h[i].phase != PH_DONE) st = PMF_ERR_NOT_CONVERGED;
        if (per_instance) per_instance[i] = st;
        if (st != PMF_OK && all == PMF_OK) all = st;
    }
    return all;
}

// Whether an instance's results can be read: after pmf_sync from the copied
// instance states; while the solve runs, once the kernel has flagged the
// instance finished and converged (its results are then final in device
// memory; flows are read from there).
enum Ready { NOT_READY = 0, READY_SYNCED, READY_IN_FLIGHT };
static Ready ready(const pmf_batch *b, int inst, int k_needed) {
    if (!b->in_flight) {
        if (!b->solved) return NOT_READY;
        const InstState &s = b->ist_h[inst];
        return s.status == PMF_OK && s.k >= k_needed ? READY_SYNCED : NOT_READY;
    }
    const int f = *(volatile const int32_t *)(b->done_h + inst);
    return f == 1 + PMF_OK ? READY_IN_FLIGHT : NOT_READY;
}

pmf_status pmf_poll(pmf_batch *b, uint8_t *done, int32_t *n_done) {
    if (!b) return PMF_ERR_INVALID_ARG;
    int n = 0;
    for (int i = 0; i < b->desc.n_inst; ++i) {
        const bool d = b->in_flight ? *(volatile const int32_t *)(b->done_h + i) != 0
                                    : (b->solved && b->ist_h[i].phase == PH_DONE);
        if (done) done[i] = d ? 1 : 0;
        n += d;
    }
    if (n_done) *n_done = n;
    return PMF_OK;
}

pmf_status pmf_get_cut(pmf_batch *b, int32_t inst, int32_t k, uint8_t *mask, int on_device) {
    if (!b || !mask || inst < 0 || inst >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    if (k < 0 || k >= std::max(b->n_lam[inst], 1)) return PMF_ERR_INVALID_ARG;
    if (ready(b, inst, k + 1) == NOT_READY) return PMF_ERR_NOT_READY;
    DeviceGuard dg(b->device);
    const DevInst &d = b->dinst[inst];
    const char *src = b->ws + b->L.masks + d.mask_off + (size_t)k * d.rows * d.pitch;
    cudaError_t e = cudaMemcpy2DAsync(mask, d.W, src, d.pitch, d.W, d.H,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                      b->cap_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap_stream);
    return cuda_err(e);
}

// the flow values of a ready instance, from the host mirror or, while the
// solve runs, from device memory
static pmf_status read_flows(pmf_batch *b, int inst, Ready r, int64_t *out, int k0, int n) {
    const size_t at = (size_t)inst * b->desc.max_lambdas + k0;
    if (r == READY_SYNCED) {
        for (int k = 0; k < n; ++k) out[k] = b->flows_h[at + k];
        return PMF_OK;
    }
    DeviceGuard dg(b->device);
    cudaError_t e = cudaMemcpyAsync(out, b->ws + b->L.flows + sizeof(long long) * at, sizeof(int64_t) * n,
                                    cudaMemcpyDeviceToHost, b->cap_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap_stream);
    return cuda_err(e);
}

pmf_status pmf_get_flow(pmf_batch *b, int32_t inst, int32_t k, int64_t *flow) {
    if (!b || !flow || inst < 0 || inst >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    if (k < 0 || k >= std::max(b->n_lam[inst], 1)) return PMF_ERR_INVALID_ARG;
    const Ready r = ready(b, inst, k + 1);
    if (r == NOT_READY) return PMF_ERR_NOT_READY;
    return read_flows(b, inst, r, flow, k, 1);
}

pmf_status pmf_get_cuts(pmf_batch *b, int32_t inst, uint8_t *masks, int on_device) {
    if (!b || !masks || inst < 0 || inst >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    if (ready(b, inst, b->n_lam[inst]) == NOT_READY) return PMF_ERR_NOT_READY;
    DeviceGuard dg(b->device);
    const DevInst &d = b->dinst[inst];
    // all lambdas in one 3-D copy: source slices rows x pitch, destination H x W
    cudaMemcpy3DParms p = {};
    p.srcPtr = make_cudaPitchedPtr(b->ws + b->L.masks + d.mask_off, (size_t)d.pitch, (size_t)d.W, (size_t)d.rows);
    p.dstPtr = make_cudaPitchedPtr(masks, (size_t)d.W, (size_t)d.W, (size_t)d.H);
    p.extent = make_cudaExtent((size_t)d.W, (size_t)d.H, (size_t)b->n_lam[inst]);
    p.kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpy3DAsync(&p, b->cap_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap_stream);
    return cuda_err(e);
}

pmf_status pmf_get_flows(pmf_batch *b, int32_t inst, int64_t *flows) {
    if (!b || !flows || inst < 0 || inst >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    const Ready r = ready(b, inst, b->n_lam[inst]);
    if (r == NOT_READY) return PMF_ERR_NOT_READY;
    return read_flows(b, inst, r, flows, 0, b->n_lam[inst]);
}

pmf_status pmf_get_flow_arcs(pmf_batch *b, int32_t inst, int32_t *f_h, int32_t *f_v, int32_t *f_s,
                             int32_t *f_t) {
    if (!b || !f_h || !f_v || !f_s || !f_t || inst < 0 || inst >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    if (b->in_flight || !b->solved) return PMF_ERR_NOT_READY;
    if (b->ist_h[inst].status != PMF_OK || b->ist_h[inst].k < b->n_lam[inst]) return PMF_ERR_NOT_READY;
    DeviceGuard dg(b->device);
    const DevInst &d = b->dinst[inst];
    const int lambda = b->lam_h[(size_t)inst * b->desc.max_lambdas + b->n_lam[inst] - 1];
    int32_t *status_d = (int32_t *)(b->ws + b->L.scratch);
    cudaStream_t s = b->cap_stream;
    cudaError_t e = launch_return_excess(b->P, d, lambda, 1 << 17, f_h, f_v, f_s, f_t, status_d, status_d + 4, s);
    int32_t status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, status_d, sizeof(status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    return status == 0 ? PMF_OK : PMF_ERR_NOT_CONVERGED;
}

pmf_status pmf_get_timing(pmf_batch *b, float *solve_ms, float *worker_ms) {
    if (!b || !solve_ms || !worker_ms) return PMF_ERR_INVALID_ARG;
    if (b->in_flight || !b->solved) return PMF_ERR_NOT_READY;
    DeviceGuard dg(b->device);
    if (cudaEventElapsedTime(solve_ms, b->ev_t0, b->ev_t1) != cudaSuccess) return PMF_ERR_CUDA;
    if (b->tune.mode == 1) {
        *worker_ms = b->worker_ms_rounds;
    } else if (cudaEventElapsedTime(worker_ms, b->ev_w0, b->ev_w1) != cudaSuccess) {
        return PMF_ERR_CUDA;
    }
    return PMF_OK;
}

pmf_status pmf_get_trace(pmf_batch *b, pmf_trace_event *out, int32_t cap, int32_t *n) {
    if (!b || !n || cap < 0 || (cap > 0 && !out)) return PMF_ERR_INVALID_ARG;
    if (b->in_flight || !b->solved) return PMF_ERR_NOT_READY;
    static_assert(sizeof(pmf_trace_event) == sizeof(TraceEvent), "trace record layout");
    const unsigned long long total = b->tune.trace ? b->glob_h->trace_n : 0;
    const int32_t have = (int32_t)std::min<unsigned long long>(total, (unsigned long long)TRACE_CAP);
    *n = have;
    const int32_t m = std::min(have, cap);
    if (m == 0) return PMF_OK;
    DeviceGuard dg(b->device);
    return cuda_err(cudaMemcpy(out, b->ws + b->L.trace, sizeof(TraceEvent) * m, cudaMemcpyDeviceToHost));
}

pmf_status pmf_get_profile(pmf_batch *b, uint64_t *out) {
    if (!b || !out) return PMF_ERR_INVALID_ARG;
    if (b->in_flight || !b->solved) return PMF_ERR_NOT_READY;
    for (int j = 0; j < PMF_PROFILE_COUNTERS; ++j) out[j] = b->tune.trace ? b->glob_h->prof[j] : 0;
    return PMF_OK;
}

pmf_status pmf_get_stats(pmf_batch *b, int32_t inst, pmf_stats *out) {
    if (!b || !out || inst < 0 || inst >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    if (b->in_flight || !b->solved) return PMF_ERR_NOT_READY;
    const InstState &s = b->ist_h[inst];
    out->pr_visits = (int64_t)s.pr_visits;
    out->bfs_visits = (int64_t)s.bfs_visits;
    out->global_relabels = (int64_t)s.epochs;
    out->lambdas_done = s.k;
    out->status = s.status;
    out->warm_visits = (int64_t)s.warm_visits;
    return PMF_OK;
}

pmf_status pmf_get_mask_layout(pmf_batch *b, int32_t inst, const uint8_t **dev_masks, int32_t *rows,
                               int32_t *pitch) {
    if (!b || !dev_masks || !rows || !pitch || inst < 0 || inst >= b->desc.n_inst) return PMF_ERR_INVALID_ARG;
    const DevInst &d = b->dinst[inst];
    *dev_masks = (const uint8_t *)(b->ws + b->L.masks + d.mask_off);
    *rows = d.rows;
    *pitch = d.pitch;
    return PMF_OK;
}

void pmf_destroy_batch(pmf_batch *b) {
    if (!b) return;
    DeviceGuard dg(b->device);
    if (b->in_flight && b->done) cudaEventSynchronize(b->done);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->done) cudaEventDestroy(b->done);
    for (cudaEvent_t ev : {b->ev_t0, b->ev_w0, b->ev_w1, b->ev_t1})
        if (ev) cudaEventDestroy(ev);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    pinned_arena().release(b->lam_h, b->pinned_bytes[0]);
    pinned_arena().release(b->ist_h, b->pinned_bytes[1]);
    pinned_arena().release(b->flows_h, b->pinned_bytes[2]);
    pinned_arena().release(b->glob_h, b->pinned_bytes[3]);
    pinned_arena().release(b->dinst_h, b->pinned_bytes[4]);
    pinned_arena().release(b->done_h, b->pinned_bytes[5]);
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// server mode: one persistent kernel that admits instances while it runs
// ---------------------------------------------------------------------------
namespace {

struct ServerLayout {
    int rows_max, pitch_max;
    size_t slot_px, max_tiles, max_strips, ring_cap;
    size_t img_planes, inst_planes, masks, dev_inst, ist, tiles, tile_inst, ring, lambdas, flows, globals,
        strip_cache, total;
};

bool server_desc_ok(const pmf_server_desc *d) {
    return d && d->n_slots >= 1 && d->n_slots <= MB_CAP && d->max_h >= 1 && d->max_w >= 1 &&
           (int64_t)d->max_h * d->max_w <= (1 << 26) && d->max_lambdas >= 1;
}

ServerLayout server_layout(const pmf_server_desc *d) {
    ServerLayout L;
    L.rows_max = round_up_i(d->max_h, ROW_ALIGN);
    L.pitch_max = round_up_i(d->max_w, TILE_W);
    L.slot_px = (size_t)L.rows_max * L.pitch_max;
    const size_t tx = (size_t)((d->max_w + TILE_IN - 1) / TILE_IN);
    L.max_tiles = tx * (size_t)(L.rows_max / 4);
    L.max_strips = tx * (size_t)((L.rows_max + BFS_ROWS - 1) / BFS_ROWS);
    L.ring_cap = 1;
    while (L.ring_cap < L.max_tiles * d->n_slots + 16384) L.ring_cap <<= 1;
    const size_t n = (size_t)d->n_slots;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes); return o; };
    L.img_planes = take(n * N_IMG_PLANES * L.slot_px * 4);
    L.inst_planes = take(n * N_INST_PLANES * L.slot_px * 4);
    L.masks = take(n * (size_t)d->max_lambdas * L.slot_px);
    L.dev_inst = take(sizeof(DevInst) * n);
    L.ist = take(sizeof(InstState) * n);
    L.tiles = take(sizeof(TileState) * n * L.max_tiles);
    L.tile_inst = take(sizeof(int32_t) * n * L.max_tiles);
    L.ring = take(sizeof(int32_t) * L.ring_cap);
    L.lambdas = take(sizeof(int32_t) * n * d->max_lambdas);
    L.flows = take(sizeof(int64_t) * n * d->max_lambdas);
    L.globals = take(sizeof(Globals));
    L.strip_cache = take(sizeof(int32_t) * STRIP_REC_WORDS * n * L.max_strips);
    L.total = off;
    return L;
}

}  // namespace

struct pmf_server {
    pmf_server_desc desc{};
    ServerLayout L{};
    char *ws = nullptr;
    Params P{};
    pmf_tuning tune{};
    int n_sm = 0;
    cudaStream_t kern = nullptr, copy = nullptr;
    bool running = false;
    Mailbox *mb = nullptr;                 // mapped host memory
    int32_t *done_h = nullptr;             // mapped: 1 + status of a slot's finished instance
    DevInst *dinst_h = nullptr;            // pinned staging of the slots' descriptors
    int32_t *lam_h = nullptr;              // pinned staging of the slots' schedules
    char *stage = nullptr;                 // pinned staging of one slot's inputs or results
    size_t pinned_bytes[5] = {0, 0, 0, 0, 0};
    std::vector<int> state;                // 0 free, 1 loaded, 2 posted
    int32_t posted = 0;                    // mailbox entries written
};

extern "C" {

pmf_status pmf_server_workspace_size(const pmf_server_desc *d, size_t *bytes) {
    if (!server_desc_ok(d) || !bytes) return PMF_ERR_INVALID_ARG;
    *bytes = server_layout(d).total;
    return PMF_OK;
}

void pmf_server_destroy(pmf_server *s);

pmf_status pmf_server_create(const pmf_server_desc *d, void *dev_workspace, size_t bytes, pmf_server **out) {
    if (!out) return PMF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!server_desc_ok(d) || !dev_workspace || ((uintptr_t)dev_workspace) % ALIGN) return PMF_ERR_INVALID_ARG;
    const ServerLayout L = server_layout(d);
    if (bytes < L.total) return PMF_ERR_OUT_OF_MEMORY;
    DeviceGuard dg(d->device);
    pmf_server *s = new (std::nothrow) pmf_server();
    if (!s) return PMF_ERR_OUT_OF_MEMORY;
    s->desc = *d;
    s->L = L;
    s->ws = (char *)dev_workspace;
    s->state.assign(d->n_slots, 0);
    apply_defaults(&s->tune);
    s->tune.tile_h = 4;
    s->tune.push_order = 1;
    cudaError_t e = cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, d->device);
    s->pinned_bytes[0] = sizeof(Mailbox);
    s->pinned_bytes[1] = sizeof(int32_t) * d->n_slots;
    s->pinned_bytes[2] = sizeof(DevInst) * d->n_slots;
    s->pinned_bytes[3] = sizeof(int32_t) * (size_t)d->n_slots * d->max_lambdas;
    // copies to and from pageable memory in the padded layout go row by row;
    // through pinned staging they are single transfers
    s->pinned_bytes[4] = std::max(sizeof(int32_t) * 5 * (size_t)d->max_h * d->max_w,
                                  (size_t)d->max_lambdas * L.slot_px + sizeof(int64_t) * d->max_lambdas);
    void **dst[5] = {(void **)&s->mb, (void **)&s->done_h, (void **)&s->dinst_h, (void **)&s->lam_h,
                     (void **)&s->stage};
    for (int j = 0; j < 5 && e == cudaSuccess; ++j) {
        *dst[j] = pinned_arena().alloc(s->pinned_bytes[j]);
        if (!*dst[j]) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->kern, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        pmf_server_destroy(s);
        return cuda_err_at(e, "pmf_server_create");
    }
    std::memset(s->mb, 0, sizeof(Mailbox));
    std::memset(s->done_h, 0, s->pinned_bytes[1]);
    Params &P = s->P;
    P.planes = (int32_t *)(s->ws + L.inst_planes);
    P.img = (const int32_t *)(s->ws + L.img_planes);
    P.masks = (uint8_t *)(s->ws + L.masks);
    P.inst = (const DevInst *)(s->ws + L.dev_inst);
    P.ist = (InstState *)(s->ws + L.ist);
    P.tiles = (TileState *)(s->ws + L.tiles);
    P.tile_inst = (const int32_t *)(s->ws + L.tile_inst);
    P.ring = (int32_t *)(s->ws + L.ring);
    P.strip_cache = (int32_t *)(s->ws + L.strip_cache);
    P.lambdas = (const int32_t *)(s->ws + L.lambdas);
    P.flows = (long long *)(s->ws + L.flows);
    P.g = (Globals *)(s->ws + L.globals);
    P.ring_mask = (unsigned long long)(L.ring_cap - 1);
    P.n_inst = d->n_slots;
    P.n_tiles_total = (int32_t)(L.max_tiles * d->n_slots);
    P.max_lambdas = d->max_lambdas;
    P.tile_h = 4;
    P.stall_ns = 5000000000LL;
    void *dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, s->mb, 0);
    P.mailbox = e == cudaSuccess ? (Mailbox *)dp : nullptr;
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dp, s->done_h, 0);
    P.done_flags = e == cudaSuccess ? (int32_t *)dp : nullptr;
    if (e != cudaSuccess) {
        pmf_server_destroy(s);
        return cuda_err_at(e, "pmf_server_create: mapped memory");
    }
    *out = s;
    return PMF_OK;
}

pmf_status pmf_server_set_tuning(pmf_server *s, const pmf_tuning *t) {
    if (!s || !t || s->running) return PMF_ERR_INVALID_ARG;
    if ((t->tile_h != 0 && t->tile_h != 4) || (t->push_order != 0 && t->push_order != 1) || t->sweeps < 0 ||
        t->relabel_every < 0 || t->max_visits_per_tile < 0 || t->blocks_per_sm < 0 || t->grid_blocks < 0 ||
        t->mode != 0)
        return PMF_ERR_INVALID_ARG;
    pmf_tuning n = *t;
    apply_defaults(&n);
    n.tile_h = 4;
    n.push_order = 1;
    s->tune = n;
    return PMF_OK;
}

pmf_status pmf_server_start(pmf_server *s, double max_seconds) {
    if (!s || s->running || !(max_seconds > 0)) return PMF_ERR_INVALID_ARG;
    DeviceGuard dg(s->desc.device);
    Params &P = s->P;
    P.trace = nullptr;
    P.sweeps = s->tune.sweeps;
    P.poll_ns = s->tune.poll_ns;
    P.label_slack = s->tune.label_slack < 0 ? 0 : s->tune.label_slack;
    P.chain_push = 1;
    P.relabel_pct = s->tune.relabel_every;
    P.relabel_extra = s->tune.relabel_extra;
    P.relabel_reach = s->tune.relabel_reach;
    P.max_visits_per_tile = s->tune.max_visits_per_tile;
    P.max_ns = (long long)(max_seconds * 1e9);
    std::memset(s->mb, 0, sizeof(Mailbox));
    std::memset(s->done_h, 0, s->pinned_bytes[1]);
    s->posted = 0;
    int grid = s->tune.grid_blocks;
    if (grid <= 0) {
        int bps = s->tune.blocks_per_sm;
        if (bps <= 0 && (server_occupancy(&bps) != cudaSuccess || bps <= 0)) bps = 4;
        grid = bps * s->n_sm;
    }
    cudaError_t e = launch_server_reset(P, (int)s->L.max_tiles, s->kern);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->kern);
    if (e == cudaSuccess) e = launch_server_worker(P, grid, s->kern);
    if (e != cudaSuccess) return cuda_err_at(e, "pmf_server_start");
    std::fill(s->state.begin(), s->state.end(), 0);
    s->running = true;
    return PMF_OK;
}

pmf_status pmf_server_load(pmf_server *s, int32_t slot, int32_t image_slot, int32_t H, int32_t W,
                           const int32_t *w_h, const int32_t *w_v, const int32_t *src0, const int32_t *slope,
                           const int32_t *sink, const int32_t *lambdas, int32_t n_lambda) {
    if (!s || slot < 0 || slot >= s->desc.n_slots || image_slot < 0 || image_slot >= s->desc.n_slots)
        return PMF_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || H > s->desc.max_h || W > s->desc.max_w || n_lambda < 1 || n_lambda > s->desc.max_lambdas)
        return PMF_ERR_INVALID_ARG;
    if (!src0 || !slope || !sink || !lambdas || (image_slot == slot && (!w_h || !w_v))) return PMF_ERR_INVALID_ARG;
    if (s->state[slot] == 2) return PMF_ERR_NOT_READY;     // posted and not yet read back
    for (int k = 1; k < n_lambda; ++k)
        if (lambdas[k] < lambdas[k - 1]) return PMF_ERR_NOT_MONOTONE;
    DeviceGuard dg(s->desc.device);
    const ServerLayout &L = s->L;
    DevInst &d = s->dinst_h[slot];
    std::memset(&d, 0, sizeof(d));
    d.H = H;
    d.W = W;
    d.rows = round_up_i(H, ROW_ALIGN);
    d.pitch = round_up_i(W, TILE_W);
    d.image = image_slot;
    d.tiles_x = (W + TILE_IN - 1) / TILE_IN;
    d.tiles_y = d.rows / 4;
    d.n_tiles = d.tiles_x * d.tiles_y;
    d.tile_base = (int32_t)(L.max_tiles * slot);
    d.n_lambda = n_lambda;
    d.hcap = H * W + 1;
    d.lead_base = (int32_t)(L.max_strips * slot);
    d.plane_off = (int64_t)((size_t)slot * N_INST_PLANES * L.slot_px);
    d.img_off = (int64_t)((size_t)image_slot * N_IMG_PLANES * L.slot_px);
    d.mask_off = (int64_t)((size_t)slot * s->desc.max_lambdas * L.slot_px);
    d.n_leads = d.tiles_x * ((d.tiles_y + BFS_ROWS / 4 - 1) / (BFS_ROWS / 4));
    d.fork_parent = d.fork_child = d.fork_k = -1;
    int32_t *lrow = s->lam_h + (size_t)slot * s->desc.max_lambdas;
    for (int k = 0; k < s->desc.max_lambdas; ++k) lrow[k] = lambdas[std::min(k, n_lambda - 1)];
    const size_t ps = (size_t)d.rows * d.pitch;
    cudaStream_t c = s->copy;
    // the inputs in the padded layout (rows x pitch), through pinned staging;
    // the kernel's set-up pass zeroes the padding and checks every value
    const size_t n = (size_t)H * W;
    int32_t *stg = (int32_t *)s->stage;
    const bool own_image = image_slot == slot;
    std::memcpy(stg, src0, n * 4);
    std::memcpy(stg + n, slope, n * 4);
    std::memcpy(stg + 2 * n, sink, n * 4);
    if (own_image) {
        std::memcpy(stg + 3 * n, w_h, n * 4);
        std::memcpy(stg + 4 * n, w_v, n * 4);
    }
    auto put = [&](char *dst_, const int32_t *src) {
        return cudaMemcpy2DAsync(dst_, (size_t)d.pitch * 4, src, (size_t)W * 4, (size_t)W * 4, H,
                                 cudaMemcpyHostToDevice, c);
    };
    char *ip = s->ws + L.inst_planes + (size_t)d.plane_off * 4;
    cudaError_t e = put(ip + (size_t)P_SRC0 * ps * 4, stg);
    if (e == cudaSuccess) e = put(ip + (size_t)P_SLOPE * ps * 4, stg + n);
    if (e == cudaSuccess) e = put(ip + (size_t)P_CT * ps * 4, stg + 2 * n);
    if (e == cudaSuccess && own_image) {
        char *im = s->ws + L.img_planes + (size_t)d.img_off * 4;
        e = put(im, stg + 3 * n);
        if (e == cudaSuccess) e = put(im + ps * 4, stg + 4 * n);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->ws + L.lambdas + sizeof(int32_t) * (size_t)slot * s->desc.max_lambdas, lrow,
                            sizeof(int32_t) * s->desc.max_lambdas, cudaMemcpyHostToDevice, c);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->ws + L.dev_inst + sizeof(DevInst) * slot, &d, sizeof(DevInst), cudaMemcpyHostToDevice, c);
    // the staging buffer is reused by the next call
    if (e == cudaSuccess) e = cudaStreamSynchronize(c);
    if (e != cudaSuccess) return cuda_err_at(e, "pmf_server_load");
    s->state[slot] = 1;
    return PMF_OK;
}

pmf_status pmf_server_post(pmf_server *s, const int32_t *slots, int32_t n) {
    if (!s || !slots || n < 1 || !s->running) return PMF_ERR_INVALID_ARG;
    for (int j = 0; j < n; ++j)
        if (slots[j] < 0 || slots[j] >= s->desc.n_slots || s->state[slots[j]] != 1) return PMF_ERR_INVALID_ARG;
    DeviceGuard dg(s->desc.device);
    // the slots' inputs are in device memory before the kernel may read them
    const cudaError_t e = cudaStreamSynchronize(s->copy);
    if (e != cudaSuccess) return cuda_err_at(e, "pmf_server_post");
    for (int j = 0; j < n; ++j) {
        const int slot = slots[j];
        *(volatile int32_t *)(s->done_h + slot) = 0;
        s->mb->ring[(s->posted + j) % MB_CAP] = slot;
        s->state[slot] = 2;
    }
    s->posted += n;
    std::atomic_thread_fence(std::memory_order_seq_cst);      // entries before the tail
    *(volatile int32_t *)&s->mb->tail = s->posted;
    return PMF_OK;
}

pmf_status pmf_server_poll(pmf_server *s, uint8_t *done, int32_t *n_done) {
    if (!s) return PMF_ERR_INVALID_ARG;
    int n = 0;
    for (int i = 0; i < s->desc.n_slots; ++i) {
        const bool d = s->state[i] == 2 && *(volatile int32_t *)(s->done_h + i) != 0;
        if (done) done[i] = d ? 1 : 0;
        n += d;
    }
    if (n_done) *n_done = n;
    return PMF_OK;
}

pmf_status pmf_server_read(pmf_server *s, int32_t slot, uint8_t *masks, int64_t *flows) {
    if (!s || slot < 0 || slot >= s->desc.n_slots || !masks || !flows) return PMF_ERR_INVALID_ARG;
    if (s->state[slot] != 2) return PMF_ERR_NOT_READY;
    const int f = *(volatile int32_t *)(s->done_h + slot);
    if (f == 0) return PMF_ERR_NOT_READY;
    s->state[slot] = 0;                                     // the slot may be loaded again
    const pmf_status st = (pmf_status)(f - 1);
    if (st != PMF_OK) return st;
    DeviceGuard dg(s->desc.device);
    const DevInst &d = s->dinst_h[slot];
    // the slot's masks as stored (n_lambda x rows x pitch) and its flows in one
    // pinned transfer each, then the padding dropped on the host
    const size_t ps = (size_t)d.rows * d.pitch;
    char *stg = s->stage;
    int64_t *fstg = (int64_t *)(stg + (size_t)s->desc.max_lambdas * s->L.slot_px);
    cudaError_t e = cudaMemcpyAsync(stg, s->ws + s->L.masks + d.mask_off, ps * d.n_lambda, cudaMemcpyDeviceToHost,
                                    s->copy);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(fstg, s->ws + s->L.flows + sizeof(int64_t) * (size_t)slot * s->desc.max_lambdas,
                            sizeof(int64_t) * d.n_lambda, cudaMemcpyDeviceToHost, s->copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy);
    if (e != cudaSuccess) return cuda_err_at(e, "pmf_server_read");
    for (int k = 0; k < d.n_lambda; ++k)
        for (int y = 0; y < d.H; ++y)
            std::memcpy(masks + ((size_t)k * d.H + y) * d.W, stg + (size_t)k * ps + (size_t)y * d.pitch, d.W);
    std::memcpy(flows, fstg, sizeof(int64_t) * d.n_lambda);
    return PMF_OK;
}

pmf_status pmf_server_stop(pmf_server *s) {
    if (!s || !s->running) return PMF_ERR_INVALID_ARG;
    DeviceGuard dg(s->desc.device);
    *(volatile int32_t *)&s->mb->stop = 1;
    cudaError_t e = cudaStreamSynchronize(s->kern);
    s->running = false;
    if (e != cudaSuccess) return cuda_err_at(e, "pmf_server_stop");
    Globals g;
    e = cudaMemcpy(&g, s->ws + s->L.globals, sizeof(Globals), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err_at(e, "pmf_server_stop: read state");
    return g.err ? PMF_ERR_NOT_CONVERGED : PMF_OK;
}

void pmf_server_destroy(pmf_server *s) {
    if (!s) return;
    DeviceGuard dg(s->desc.device);
    if (s->running) (void)pmf_server_stop(s);
    if (s->kern) cudaStreamDestroy(s->kern);
    if (s->copy) cudaStreamDestroy(s->copy);
    pinned_arena().release(s->mb, s->pinned_bytes[0]);
    pinned_arena().release(s->done_h, s->pinned_bytes[1]);
    pinned_arena().release(s->dinst_h, s->pinned_bytes[2]);
    pinned_arena().release(s->lam_h, s->pinned_bytes[3]);
    pinned_arena().release(s->stage, s->pinned_bytes[4]);
    delete s;
}

}  // extern "C"
