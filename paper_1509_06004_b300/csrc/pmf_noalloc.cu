// pmf_solve_noalloc: a single-instance solve that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// that owns the whole device-memory budget and hands out only pre-reserved
// buffers, or latency-critical paths where cudaMalloc's implicit device-wide
// synchronisation is not allowed.  For them this entry point keeps all the
// solver's scratch (state planes, masks, queue, tile and instance records) in a
// fixed, file-scope device array that the library reserves when it is loaded;
// the caller passes only its input capacities and its output buffers.
//
// The array is shared by every call in the process and keeps the last call's
// contents; each call re-initialises the parts that must start from zero.  Two
// calls whose GPU work overlapped would race on the array, so calls are
// serialised by a process-wide lock held until the call's stream work is done.
#include <atomic>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "pmf.h"
#include "pmf_internal.h"

using namespace pmf;

// the scratch: every GPU that loads the library holds it until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[(size_t)PMF_NOALLOC_SCRATCH_MB << 20];

namespace {

constexpr size_t kScratchBytes = (size_t)PMF_NOALLOC_SCRATCH_MB << 20;
constexpr int kMaxDevices = 64;
// solver knobs: the autotuner's choice for one-instance workloads (tile
// height 4, pushes along columns and rows, 8 sweeps per visit, relabel
// cadence 800 %, label slack 16)
constexpr int kTileH = 4;
constexpr int kPushOrder = 1;
constexpr int kSweeps = 8;
constexpr int kRelabelPct = 800;
constexpr int kLabelSlack = 16;

std::mutex g_lock;
void *g_addr[kMaxDevices];   // device address of the array, per device, looked up once
// test hook (pmf_testing_fail_noalloc_call): the n-th CUDA call of the next
// pmf_solve_noalloc reports a failure instead of being made; 0 = none
std::atomic<int> g_fail_at{0};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// the array's device address on the current device (set-up on first use)
pmf_status scratch_address(int dev, char **out) {
    if (dev < 0 || dev >= kMaxDevices) return PMF_ERR_INVALID_ARG;
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_err_at(e, "pmf_solve_noalloc: cudaGetSymbolAddress");
        if (p == nullptr) return cuda_err_at(cudaErrorInvalidSymbol, "pmf_solve_noalloc: cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = static_cast<char *>(g_addr[dev]);
    return PMF_OK;
}

}  // namespace

extern "C" PMF_API pmf_status pmf_solve_noalloc(int32_t H, int32_t W, const int32_t *w_h,
                                                const int32_t *w_v, const int32_t *src0,
                                                const int32_t *slope, const int32_t *sink,
                                                const int32_t *lambdas, int32_t n_lambda,
                                                uint8_t *masks, int64_t *flows, void *cuda_stream) {
    if (H < 1 || W < 1 || !w_h || !w_v || !src0 || !slope || !sink || !lambdas || !masks || !flows)
        return PMF_ERR_INVALID_ARG;
    if (n_lambda < 1) return PMF_ERR_INVALID_ARG;
    for (int k = 1; k < n_lambda; ++k)
        if (lambdas[k] < lambdas[k - 1]) return PMF_ERR_NOT_MONOTONE;
    const int rows = (H + ROW_ALIGN - 1) / ROW_ALIGN * ROW_ALIGN;
    const int pitch = (W + TILE_W - 1) / TILE_W * TILE_W;
    const size_t PS = (size_t)rows * pitch;
    // stated limits (see pmf.h)
    if (PS > (size_t)PMF_NOALLOC_MAX_PIXELS || n_lambda > PMF_NOALLOC_MAX_LAMBDAS) return PMF_ERR_OUT_OF_MEMORY;

    // layout inside the array
    const int tiles_x = (W + TILE_IN - 1) / TILE_IN, tiles_y = rows / kTileH;
    const int n_tiles = tiles_x * tiles_y;
    size_t ring_cap = 1;
    while (ring_cap < (size_t)n_tiles + 16384) ring_cap <<= 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = up256(off + bytes); return o; };
    const size_t o_img = take(PS * 4 * N_IMG_PLANES);
    const size_t o_inst = take(PS * 4 * N_INST_PLANES);
    const size_t o_masks = take(PS * (size_t)n_lambda);
    const size_t o_dinst = take(sizeof(DevInst));
    const size_t o_ist = take(sizeof(InstState));
    const size_t o_tiles = take(sizeof(TileState) * n_tiles);
    const size_t o_tinst = take(sizeof(int32_t) * n_tiles);
    const size_t o_ring = take(sizeof(int32_t) * ring_cap);
    const size_t o_lam = take(sizeof(int32_t) * n_lambda);
    const size_t o_flows = take(sizeof(int64_t) * n_lambda);
    const size_t o_glob = take(sizeof(Globals));
    const size_t o_flags = take(sizeof(int32_t) * 2);
    const size_t n_strips = (size_t)tiles_x * ((rows + BFS_ROWS - 1) / BFS_ROWS);
    const size_t o_strips = take(sizeof(int32_t) * STRIP_REC_WORDS * n_strips);
    if (off > kScratchBytes) return PMF_ERR_OUT_OF_MEMORY;

    std::lock_guard<std::mutex> guard(g_lock);
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int fail_at = g_fail_at.exchange(0);
    int n_calls = 0;
    cudaError_t e = cudaSuccess;
    const char *where = "";
    bool enqueued = false;   // stream work of this call may be in flight
    // one CUDA call: skipped after a failure; the test hook may fail it
    auto step = [&](const char *site, auto &&call) {
        if (e != cudaSuccess) return;
        if (++n_calls == fail_at) {
            e = cudaErrorUnknown;
            where = "pmf_solve_noalloc: injected failure";
            return;
        }
        e = call();
        if (e != cudaSuccess) where = site;
    };
    // an error return first waits for this call's queued work: the next call
    // must not start while it could still touch the shared array
    auto fail = [&]() -> pmf_status {
        if (enqueued) (void)cudaStreamSynchronize(s);
        return cuda_err_at(e, where);
    };

    int dev = 0;
    step("pmf_solve_noalloc: cudaGetDevice", [&] { return cudaGetDevice(&dev); });
    if (e != cudaSuccess) return fail();
    char *ws = nullptr;
    pmf_status st = scratch_address(dev, &ws);
    if (st != PMF_OK) return st;
    int n_sm = 0, bps = 0;
    step("pmf_solve_noalloc: cudaDeviceGetAttribute",
         [&] { return cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev); });
    if (e != cudaSuccess) return fail();
    if (n_sm < 1) return cuda_err_at(cudaErrorInvalidDevice, "pmf_solve_noalloc: multiprocessor count");
    if (worker_occupancy(kTileH, &bps) != cudaSuccess || bps < 1) bps = 1;

    DevInst d;
    std::memset(&d, 0, sizeof(d));
    d.H = H;
    d.W = W;
    d.pitch = pitch;
    d.rows = rows;
    d.tiles_x = tiles_x;
    d.tiles_y = tiles_y;
    d.n_tiles = n_tiles;
    d.n_lambda = n_lambda;
    d.hcap = H * W + 1;
    d.lead_base = 0;
    d.n_leads = tiles_x * ((tiles_y + BFS_ROWS / kTileH - 1) / (BFS_ROWS / kTileH));
    d.fork_parent = d.fork_child = d.fork_k = -1;

    Params P;
    std::memset(&P, 0, sizeof(P));
    P.trace = nullptr;
    P.planes = reinterpret_cast<int32_t *>(ws + o_inst);
    P.img = reinterpret_cast<const int32_t *>(ws + o_img);
    P.masks = reinterpret_cast<uint8_t *>(ws + o_masks);
    P.inst = reinterpret_cast<const DevInst *>(ws + o_dinst);
    P.ist = reinterpret_cast<InstState *>(ws + o_ist);
    P.tiles = reinterpret_cast<TileState *>(ws + o_tiles);
    P.tile_inst = reinterpret_cast<const int32_t *>(ws + o_tinst);
    P.ring = reinterpret_cast<int32_t *>(ws + o_ring);
    P.strip_cache = reinterpret_cast<int32_t *>(ws + o_strips);
    P.lambdas = reinterpret_cast<const int32_t *>(ws + o_lam);
    P.flows = reinterpret_cast<long long *>(ws + o_flows);
    P.g = reinterpret_cast<Globals *>(ws + o_glob);
    P.img_flags = reinterpret_cast<const int32_t *>(ws + o_flags);
    P.inst_flags = reinterpret_cast<int32_t *>(ws + o_flags) + 1;
    P.ring_mask = (unsigned long long)(ring_cap - 1);
    P.n_inst = 1;
    P.n_tiles_total = n_tiles;
    P.n_leads_total = d.n_leads;
    P.n_leads_queued = d.n_leads;
    P.max_lambdas = n_lambda;
    P.sweeps = kSweeps;
    P.chain_push = kPushOrder;
    P.relabel_pct = kRelabelPct;
    P.label_slack = kLabelSlack;
    P.tile_h = kTileH;
    P.poll_ns = 256;
    P.max_visits_per_tile = 2000;
    P.stall_ns = 5000000000LL;
    P.max_ns = 120000000000LL;

    // everything the solve reads before writing starts from zero; the rest is
    // written in full by the set-up kernels
    enqueued = true;
    step("pmf_solve_noalloc: clear flags", [&] { return cudaMemsetAsync(ws + o_flags, 0, sizeof(int32_t) * 2, s); });
    step("pmf_solve_noalloc: clear globals", [&] { return cudaMemsetAsync(ws + o_glob, 0, sizeof(Globals), s); });
    step("pmf_solve_noalloc: clear flows",
         [&] { return cudaMemsetAsync(ws + o_flows, 0, sizeof(int64_t) * n_lambda, s); });
    step("pmf_solve_noalloc: descriptor",
         [&] { return cudaMemcpyAsync(ws + o_dinst, &d, sizeof(d), cudaMemcpyHostToDevice, s); });
    step("pmf_solve_noalloc: schedule", [&] {
        return cudaMemcpyAsync(ws + o_lam, lambdas, sizeof(int32_t) * n_lambda, cudaMemcpyHostToDevice, s);
    });
    step("pmf_solve_noalloc: pad_image",
         [&] { return launch_pad_image(P, 0, d, w_h, w_v, reinterpret_cast<int32_t *>(ws + o_flags), s); });
    step("pmf_solve_noalloc: pad_terminals", [&] { return launch_pad_terminals(P, 0, d, src0, slope, sink, s); });
    step("pmf_solve_noalloc: reset", [&] { return launch_reset(P, s); });
    step("pmf_solve_noalloc: init", [&] { return launch_init(P, (int)PS, s); });
    step("pmf_solve_noalloc: worker", [&] { return launch_worker(P, bps * n_sm, s); });
    InstState ist;
    Globals glob;
    step("pmf_solve_noalloc: read state",
         [&] { return cudaMemcpyAsync(&ist, ws + o_ist, sizeof(ist), cudaMemcpyDeviceToHost, s); });
    step("pmf_solve_noalloc: read globals",
         [&] { return cudaMemcpyAsync(&glob, ws + o_glob, sizeof(glob), cudaMemcpyDeviceToHost, s); });
    step("pmf_solve_noalloc: synchronise", [&] { return cudaStreamSynchronize(s); });
    if (e != cudaSuccess) return fail();
    enqueued = false;
    if (ist.status != PMF_OK) return (pmf_status)ist.status;
    if (glob.err || ist.phase != PH_DONE || ist.k < n_lambda) return PMF_ERR_NOT_CONVERGED;

    // outputs: flow values to the caller's host array, masks to its device buffer
    enqueued = true;
    step("pmf_solve_noalloc: copy flows", [&] {
        return cudaMemcpyAsync(flows, ws + o_flows, sizeof(int64_t) * n_lambda, cudaMemcpyDeviceToHost, s);
    });
    for (int k = 0; k < n_lambda; ++k)
        step("pmf_solve_noalloc: copy masks", [&] {
            return cudaMemcpy2DAsync(masks + (size_t)k * H * W, W, ws + o_masks + (size_t)k * PS, pitch, W, H,
                                     cudaMemcpyDeviceToDevice, s);
        });
    step("pmf_solve_noalloc: synchronise", [&] { return cudaStreamSynchronize(s); });
    if (e != cudaSuccess) return fail();
    return PMF_OK;
}

extern "C" PMF_API void pmf_testing_fail_noalloc_call(int32_t n) { g_fail_at.store(n > 0 ? n : 0); }
