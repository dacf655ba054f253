// Multi-asset lookup serving: resident assets under a device-memory budget,
// continuous batching of requests of uneven sizes from different assets,
// batches launched as instantiated CUDA graphs.
//
// A scheduler thread owns the device side.  Each pass it
//   1. retires finished batches (event query) and records the completion
//      time of every request whose last queries were in them;
//   2. admits requests whose asset is resident, and small requests at
//      once: until their asset is resident their batches read the asset's
//      page-locked, mapped host copy across the CPU-GPU link; assets that
//      unfinished requests need are uploaded (asynchronously, from that
//      host copy), most requested first, as far as the budget allows after
//      evicting the least recently used assets that no unfinished request
//      needs;
//   3. fills every free batch slot from the admitted requests, shortest
//      remaining work first with ageing (a request's remaining query count
//      shrinks with the time it has waited, so small requests overtake
//      large ones and no request starves), at most 'request_chunk' queries
//      of one request per batch, so requests that arrive while others run
//      join the next batch;
//   4. launches the batch: query copies in, the slot's graph (a memcpy node
//      for the batch's descriptor table, then one persistent kernel per
//      texel format whose blocks pull 4096-query tiles of any item through
//      an atomic counter), result copies out, a completion event.  A
//      request whose buffers are page-locked, mapped into the device's
//      address space and 16-byte aligned skips both copies: its items point
//      the kernel at the host buffers themselves.
// Every query is computed by the same per-query code as htex_lookup, so a
// request's results do not depend on what else shares its batches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "lookup_core.cuh"

namespace htex {

constexpr int kFormats = 20;        // 5 texel formats x 1..4 channels
constexpr int kMaxItems = 256;      // batch items (request chunks) per batch
constexpr int kServeTile = 4096;    // queries per work tile
constexpr int kServeThreads = 256;
constexpr int kMaxAssets = 1024;

struct ItemDesc {                   // one request chunk inside a batch
    const uint8_t* rec;
    const uint8_t* hdr;
    const uint8_t* scale;
    const uint8_t* pool;
    const htex_query* q;
    float* out;
    int32_t H, uniform_log2n;
    uint32_t uniform_stride16;
    int32_t n;
};

struct ServeTable {
    uint32_t counter[kFormats];     // tiles handed out (zero at launch)
    uint32_t first_item[kFormats];  // items of format f: [first_item, first_item + num_items)
    uint32_t num_items[kFormats];
    uint32_t total_tiles[kFormats];
    uint32_t tile_start[kMaxItems]; // first tile of each item within its format
    ItemDesc items[kMaxItems];
};

template <int DT, int C>
__global__ void __launch_bounds__(kServeThreads) k_serve(ServeTable* tab, int fmt) {
    __shared__ uint32_t s_tile;
    const uint32_t ntiles = tab->total_tiles[fmt];
    if (ntiles == 0) return;
    const uint32_t first = tab->first_item[fmt], nitems = tab->num_items[fmt];
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&tab->counter[fmt], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        __syncthreads();
        if (tile >= ntiles) break;
        // the item holding this tile: last k with tile_start[k] <= tile
        uint32_t lo = first, hi = first + nitems - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) / 2;
            if (tab->tile_start[mid] <= tile) lo = mid; else hi = mid - 1;
        }
        const ItemDesc& it = tab->items[lo];
        Asset<GlobalSpace> A;
        A.rec.base = it.rec;
        A.hdr.base = it.hdr;
        A.scale.base = it.scale;
        A.pool.base = it.pool;
        A.H = it.H;
        A.uniform_log2n = it.uniform_log2n;
        A.uniform_stride16 = it.uniform_stride16;
        const FwdParams p{it.q, it.n, it.out, nullptr, nullptr};
        const int64_t start = int64_t(tile - tab->tile_start[lo]) * kServeTile;
        const int64_t end = start + kServeTile < int64_t(it.n) ? start + kServeTile : int64_t(it.n);
        for (int64_t i = start + threadIdx.x; i < end; i += blockDim.x) {
            const int4 raw = ld_query(p.q, i);
            lookup_one<DT, C, Raw<DT, C>::PACKED>(A, p, raw, record_of(A, raw), i);
        }
    }
}

}  // namespace htex

using namespace htex;
using Clock = std::chrono::steady_clock;

namespace {

int format_of(htex_dtype dt, int C) { return int(dt) * 4 + (C - 1); }

template <int DT, int C>
void launch_serve(ServeTable* tab, int fmt, int grid, cudaStream_t s) {
    k_serve<DT, C><<<grid, kServeThreads, 0, s>>>(tab, fmt);
}

template <int DT, int C>
int serve_grid(int sms) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_serve<DT, C>, kServeThreads, 0) != cudaSuccess || b < 1) b = 1;
    return sms * b;
}

using LaunchFn = void (*)(ServeTable*, int, int, cudaStream_t);
using GridFn = int (*)(int);

template <int DT>
void fill_tables(LaunchFn* L, GridFn* G) {
    const int b = DT * 4;
    L[b + 0] = launch_serve<DT, 1>; G[b + 0] = serve_grid<DT, 1>;
    L[b + 1] = launch_serve<DT, 2>; G[b + 1] = serve_grid<DT, 2>;
    L[b + 2] = launch_serve<DT, 3>; G[b + 2] = serve_grid<DT, 3>;
    L[b + 3] = launch_serve<DT, 4>; G[b + 3] = serve_grid<DT, 4>;
}

struct Request {
    int64_t id = 0;
    int32_t asset = 0;
    const htex_query* q = nullptr;
    float* out = nullptr;
    const htex_query* dq = nullptr;   // device addresses of mapped host buffers,
    float* dout = nullptr;            // or null: staged through the slot's buffers
    int64_t n = 0, issued = 0, done = 0;
    Clock::time_point t_submit;
    bool active = false;
};

struct ServeAsset {
    HtexAssetArrays arrays;
    // page-locked, mapped host copy: records, headers, scales, pool (each
    // 256-byte aligned); the device addresses of its parts serve requests
    // while the asset is not resident, the host addresses feed uploads
    void* host = nullptr;
    size_t off_hdr = 0, off_scale = 0, off_pool = 0;
    const uint8_t* dev_host = nullptr;
    int64_t bytes = 0;
    int fmt = 0;
    htex_textures* tex = nullptr;   // resident when set
    cudaEvent_t uploaded = nullptr;
    bool uploading = false;
    int64_t pins = 0;               // admitted or waiting, unfinished requests (demand)
    uint64_t last_use = 0;
};

struct ItemRef {
    Request* req;
    int64_t count;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t graph_formats = 0;     // formats the instantiated graph launches
    ServeTable* h_table = nullptr;  // page-locked
    ServeTable* d_table = nullptr;
    htex_query* d_q = nullptr;
    float* d_out = nullptr;
    bool busy = false;
    std::vector<ItemRef> items;
};

}  // namespace

struct htex_server {
    htex_server_config cfg{};
    int device = 0, sms = 0;
    LaunchFn launch[kFormats] = {};
    GridFn grid[kFormats] = {};

    std::mutex mu;                      // guards everything below it that the client touches
    std::condition_variable cv;
    std::deque<Request*> incoming;
    std::vector<std::pair<int64_t, double>> completed;
    int64_t next_id = 1, submitted = 0, finished = 0;
    htex_status error = HTEX_OK;
    bool stop = false;

    // assets: appended by the client under 'mu', published through the
    // atomic count; the scheduler only reads entries below the count
    ServeAsset* assets[kMaxAssets] = {};
    std::atomic<int32_t> num_assets{0};
    std::atomic<uint32_t> formats{0};   // formats of the registered assets (bit set)

    // scheduler-owned
    std::vector<Request*> waiting, admitted;
    std::vector<Slot> slots;
    cudaStream_t upload_stream = nullptr;
    cudaMemPool_t asset_pool = nullptr; // resident assets' device memory, released stream-ordered
    int64_t resident_bytes = 0;
    uint64_t tick = 0;
    htex_server_stats stats{};
    std::thread worker;
};

namespace {

void fail(htex_server* s, htex_status st) {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->error == HTEX_OK) s->error = st;
    s->cv.notify_all();
}

bool build_graph(htex_server* s, Slot& sl) {
    if (sl.exec) {
        cudaGraphExecDestroy(sl.exec);
        sl.exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    cudaMemcpyAsync(sl.d_table, sl.h_table, sizeof(ServeTable), cudaMemcpyHostToDevice, sl.stream);
    const uint32_t fm = s->formats.load();
    for (int f = 0; f < kFormats; ++f)
        if (fm & (1u << f)) s->launch[f](sl.d_table, f, s->grid[f](s->sms), sl.stream);
    if (cudaStreamEndCapture(sl.stream, &graph) != cudaSuccess) return false;
    const bool ok = cudaGraphInstantiate(&sl.exec, graph, 0) == cudaSuccess;
    cudaGraphDestroy(graph);
    sl.graph_formats = fm;
    return ok;
}

// Retire finished batches.
bool retire(htex_server* s) {
    bool progress = false;
    for (Slot& sl : s->slots) {
        if (!sl.busy) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) {
            fail(s, HTEX_ERR_CUDA);
            return false;
        }
        const Clock::time_point now = Clock::now();
        std::lock_guard<std::mutex> g(s->mu);
        for (const ItemRef& it : sl.items) {
            Request* r = it.req;
            r->done += it.count;
            if (r->done == r->n) {
                s->completed.emplace_back(r->id, std::chrono::duration<double>(now - r->t_submit).count());
                s->assets[r->asset]->pins -= 1;
                ++s->finished;
                ++s->stats.completed;
                delete r;
            }
        }
        sl.items.clear();
        sl.busy = false;
        progress = true;
        s->cv.notify_all();
    }
    return progress;
}

// Make room for 'need' bytes by evicting idle assets, least recently used first.
bool make_room(htex_server* s, int64_t need) {
    while (s->resident_bytes + need > s->cfg.budget_bytes) {
        ServeAsset* victim = nullptr;
        const int32_t na = s->num_assets.load();
        for (int32_t k = 0; k < na; ++k) {
            ServeAsset* a = s->assets[k];
            if (a->tex && !a->uploading && a->pins == 0 && (!victim || a->last_use < victim->last_use)) victim = a;
        }
        if (!victim) return false;
        // no request needs it, so every batch that read it has retired; its
        // buffers go back to the pool stream-ordered (no device-wide wait)
        htex_textures_destroy(victim->tex);
        victim->tex = nullptr;
        s->resident_bytes -= victim->bytes;
        std::lock_guard<std::mutex> g(s->mu);
        ++s->stats.evictions;
    }
    return true;
}

// The four parts of an asset's host copy to its device buffers.
htex_status copy_host_copy(const ServeAsset* a, htex_textures* t, cudaStream_t stream) {
    const uint8_t* h = static_cast<const uint8_t*>(a->host);
    const size_t rec_b = a->arrays.rec.size() * 4, hdr_b = a->arrays.hdr.size() * 4, sc_b = a->arrays.scale.size() * 4;
    if ((rec_b && cudaMemcpyAsync(t->d_rec, h, rec_b, cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
        (hdr_b && cudaMemcpyAsync(t->d_hdr, h + a->off_hdr, hdr_b, cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
        (sc_b && cudaMemcpyAsync(t->d_scale, h + a->off_scale, sc_b, cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
        (a->arrays.pool_bytes && cudaMemcpyAsync(t->d_pool, h + a->off_pool, size_t(a->arrays.pool_bytes),
                                                 cudaMemcpyHostToDevice, stream) != cudaSuccess)) {
        cudaGetLastError();
        return HTEX_ERR_CUDA;
    }
    return HTEX_OK;
}

// A request is admitted when its asset is resident.  A small request
// (at most kHostServeQueries) whose asset is not resident, or still
// uploading, is admitted at once: its batches read the asset's page-locked
// host copy across the CPU-GPU link, with the same kernel code and bytes.
// (Texel reads across the link cost several times the bytes of the query
// and result, so large requests wait for the upload instead.)  Assets with
// unfinished requests are uploaded, most requested first, as far as the
// budget allows after evicting idle assets.
constexpr int64_t kHostServeQueries = 65536;

bool admit(htex_server* s) {
    bool progress = false;
    const int32_t na = s->num_assets.load();
    for (int32_t k = 0; k < na; ++k) {      // finished uploads
        ServeAsset* a = s->assets[k];
        if (!a->uploading) continue;
        const cudaError_t e = cudaEventQuery(a->uploaded);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) {
            fail(s, HTEX_ERR_CUDA);
            return false;
        }
        a->uploading = false;
        progress = true;
    }
    for (size_t k = 0; k < s->waiting.size();) {
        Request* r = s->waiting[k];
        ServeAsset* a = s->assets[r->asset];
        if (!(a->tex && !a->uploading) && r->n > kHostServeQueries) {
            ++k;
            continue;
        }
        r->active = true;
        a->last_use = ++s->tick;
        s->admitted.push_back(r);
        s->waiting.erase(s->waiting.begin() + long(k));
        progress = true;
    }
    std::vector<ServeAsset*> want;
    for (int32_t k = 0; k < na; ++k)
        if (!s->assets[k]->tex && s->assets[k]->pins > 0) want.push_back(s->assets[k]);
    std::stable_sort(want.begin(), want.end(), [](const ServeAsset* x, const ServeAsset* y) { return x->pins > y->pins; });
    for (ServeAsset* a : want) {
        if (!make_room(s, a->bytes)) continue;
        htex_textures* t = nullptr;
        if (htex_asset_allocate_async(a->arrays, s->asset_pool, s->upload_stream, &t) != HTEX_OK) continue;
        if (copy_host_copy(a, t, s->upload_stream) != HTEX_OK ||
            cudaEventRecord(a->uploaded, s->upload_stream) != cudaSuccess) {
            htex_textures_destroy(t);
            fail(s, HTEX_ERR_CUDA);
            return false;
        }
        a->tex = t;
        a->uploading = true;
        s->resident_bytes += a->bytes;
        {
            std::lock_guard<std::mutex> g(s->mu);
            ++s->stats.uploads;
        }
        progress = true;
    }
    return progress;
}

// Order in which admitted requests fill a batch: shortest remaining work
// first, aged -- a request's remaining query count is divided by
// 1 + wait / kAgeScale, so small requests overtake large ones that arrived
// earlier, and a large request that has waited moves forward until it is
// served (no starvation).
constexpr double kAgeScale = 1e-3;   // seconds

void order_admitted(htex_server* s) {
    const Clock::time_point now = Clock::now();
    std::vector<std::pair<double, Request*>> keyed;
    keyed.reserve(s->admitted.size());
    for (Request* r : s->admitted) {
        const double wait = std::chrono::duration<double>(now - r->t_submit).count();
        keyed.emplace_back(double(r->n - r->issued) / (1.0 + wait / kAgeScale), r);
    }
    std::stable_sort(keyed.begin(), keyed.end(),
                     [](const auto& x, const auto& y) { return x.first < y.first; });
    for (size_t k = 0; k < keyed.size(); ++k) s->admitted[k] = keyed[k].second;
}

bool launch_batch(htex_server* s, Slot& sl) {
    // requests by aged remaining work, at most request_chunk queries each
    order_admitted(s);
    std::vector<std::pair<Request*, int64_t>> take;
    int64_t used = 0;
    for (Request* r : s->admitted) {
        const int64_t rem = r->n - r->issued;
        if (rem <= 0) continue;
        const int64_t c = std::min({rem, s->cfg.request_chunk, s->cfg.batch_queries - used});
        if (c <= 0) break;
        take.emplace_back(r, c);
        used += c;
        if (int(take.size()) >= s->cfg.max_items || used >= s->cfg.batch_queries) break;
    }
    if (take.empty()) return false;
    if (sl.graph_formats != s->formats.load() && !build_graph(s, sl)) {
        fail(s, HTEX_ERR_CUDA);
        return false;
    }
    // group the items by texel format for the per-format kernels
    std::stable_sort(take.begin(), take.end(), [&](const auto& x, const auto& y) {
        return s->assets[x.first->asset]->fmt < s->assets[y.first->asset]->fmt;
    });
    ServeTable* T = sl.h_table;
    int64_t host_queries = 0;
    std::memset(T->counter, 0, sizeof(T->counter));
    std::memset(T->num_items, 0, sizeof(T->num_items));
    std::memset(T->total_tiles, 0, sizeof(T->total_tiles));
    int64_t qoff = 0, ooff = 0;
    for (size_t k = 0; k < take.size(); ++k) {
        Request* r = take[k].first;
        const int64_t c = take[k].second;
        ServeAsset* a = s->assets[r->asset];
        const htex_textures* t = (a->tex && !a->uploading) ? a->tex : nullptr;   // resident, else the host copy
        const HtexAssetArrays& ar = a->arrays;
        const int f = a->fmt;
        if (T->num_items[f] == 0) T->first_item[f] = uint32_t(k);
        T->num_items[f] += 1;
        T->tile_start[k] = T->total_tiles[f];
        T->total_tiles[f] += uint32_t((c + kServeTile - 1) / kServeTile);
        ItemDesc& d = T->items[k];
        d.rec = t ? static_cast<const uint8_t*>(t->d_rec) : a->dev_host;
        d.hdr = t ? static_cast<const uint8_t*>(t->d_hdr) : a->dev_host + a->off_hdr;
        d.scale = t ? static_cast<const uint8_t*>(t->d_scale) : a->dev_host + a->off_scale;
        d.pool = t ? static_cast<const uint8_t*>(t->d_pool) : a->dev_host + a->off_pool;
        d.q = r->dq ? r->dq + r->issued : sl.d_q + qoff;
        d.out = r->dout ? r->dout + r->issued * ar.C : sl.d_out + ooff;
        d.H = ar.H;
        d.uniform_log2n = ar.uniform_log2n;
        d.uniform_stride16 = uint32_t(ar.uniform_stride / 16);
        d.n = int32_t(c);
        if (!t) host_queries += c;
        if (!r->dq) {
            if (cudaMemcpyAsync(sl.d_q + qoff, r->q + r->issued, size_t(c) * sizeof(htex_query),
                                cudaMemcpyHostToDevice, sl.stream) != cudaSuccess) {
                fail(s, HTEX_ERR_CUDA);
                return false;
            }
            qoff += c;
        }
        if (!r->dout) ooff += c * ar.C;
        a->last_use = ++s->tick;
    }
    if (cudaGraphLaunch(sl.exec, sl.stream) != cudaSuccess) {
        fail(s, HTEX_ERR_CUDA);
        return false;
    }
    ooff = 0;
    for (size_t k = 0; k < take.size(); ++k) {
        Request* r = take[k].first;
        const int64_t c = take[k].second;
        const int C = s->assets[r->asset]->arrays.C;
        if (!r->dout) {
            if (cudaMemcpyAsync(r->out + r->issued * C, sl.d_out + ooff, size_t(c) * C * sizeof(float),
                                cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess) {
                fail(s, HTEX_ERR_CUDA);
                return false;
            }
            ooff += c * C;
        }
        r->issued += c;
        sl.items.push_back({r, c});
    }
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) {
        fail(s, HTEX_ERR_CUDA);
        return false;
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        ++s->stats.batches;
        s->stats.queries += used;
        s->stats.host_queries += host_queries;
    }
    sl.busy = true;
    // requests with everything issued leave the admitted list (their
    // completion is recorded when their last batch retires)
    s->admitted.erase(std::remove_if(s->admitted.begin(), s->admitted.end(),
                                     [](Request* r) { return r->issued == r->n; }),
                      s->admitted.end());
    return true;
}

void run(htex_server* s) {
    if (cudaSetDevice(s->device) != cudaSuccess) {
        fail(s, HTEX_ERR_CUDA);
        return;
    }
    while (true) {
        {
            std::unique_lock<std::mutex> g(s->mu);
            if (s->stop || s->error != HTEX_OK) break;
            while (!s->incoming.empty()) {
                Request* r = s->incoming.front();
                s->assets[r->asset]->pins += 1;     // demand from the moment it arrives
                s->waiting.push_back(r);
                s->incoming.pop_front();
            }
        }
        bool progress = retire(s);
        progress |= admit(s);
        for (Slot& sl : s->slots)
            if (!sl.busy) progress |= launch_batch(s, sl);
        if (!progress) {
            // idle time: instantiate the graphs of slots whose format set is
            // stale, so that the first batches after new assets do not wait
            // for it
            const uint32_t fm = s->formats.load();
            for (Slot& sl : s->slots) {
                if (sl.busy || sl.graph_formats == fm) continue;
                if (!build_graph(s, sl)) {
                    fail(s, HTEX_ERR_CUDA);
                    return;
                }
                progress = true;
            }
        }
        if (!progress) {
            bool idle = s->waiting.empty() && s->admitted.empty();
            for (const Slot& sl : s->slots) idle = idle && !sl.busy;
            std::unique_lock<std::mutex> g(s->mu);
            if (idle && s->incoming.empty() && !s->stop)
                s->cv.wait_for(g, std::chrono::milliseconds(50));
            else if (!s->stop)
                s->cv.wait_for(g, std::chrono::microseconds(20));
        }
    }
}

void release(htex_server* s) {
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.h_table);
        cudaFree(sl.d_table);
        cudaFree(sl.d_q);
        cudaFree(sl.d_out);
    }
    for (int32_t k = 0; k < s->num_assets.load(); ++k) {
        ServeAsset* a = s->assets[k];
        htex_textures_destroy(a->tex);
        if (a->uploaded) cudaEventDestroy(a->uploaded);
        cudaFreeHost(a->host);
        delete a;
    }
    if (s->upload_stream) {
        cudaStreamSynchronize(s->upload_stream);
        cudaStreamDestroy(s->upload_stream);
        s->upload_stream = nullptr;
    }
    if (s->asset_pool) cudaMemPoolDestroy(s->asset_pool);
    for (Request* r : s->waiting) delete r;
    for (Request* r : s->incoming) delete r;
    // admitted requests are also referenced by unretired slots only through
    // 'admitted' or slot items; delete each once
    std::vector<Request*> rest(s->admitted.begin(), s->admitted.end());
    for (Slot& sl : s->slots)
        for (ItemRef& it : sl.items) rest.push_back(it.req);
    std::sort(rest.begin(), rest.end());
    rest.erase(std::unique(rest.begin(), rest.end()), rest.end());
    for (Request* r : rest) delete r;
}

}  // namespace

extern "C" htex_status htex_server_create(const htex_server_config* cfg, htex_server** out) {
    if (!cfg || !out) return HTEX_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->budget_bytes <= 0 || cfg->batch_queries < kServeTile || cfg->batch_queries >= (int64_t(1) << 31) ||
        cfg->batch_slots < 1 || cfg->batch_slots > 8 || cfg->max_items < 1 || cfg->max_items > kMaxItems ||
        cfg->request_chunk < 1)
        return HTEX_ERR_INVALID_ARG;
    htex_server* s = new (std::nothrow) htex_server;
    if (!s) return HTEX_ERR_OUT_OF_MEMORY;
    s->cfg = *cfg;
    fill_tables<HTEX_F32>(s->launch, s->grid);
    fill_tables<HTEX_U8>(s->launch, s->grid);
    fill_tables<HTEX_F16>(s->launch, s->grid);
    fill_tables<HTEX_BF16>(s->launch, s->grid);
    fill_tables<HTEX_E4M3>(s->launch, s->grid);
    bool ok = cudaGetDevice(&s->device) == cudaSuccess &&
              cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->upload_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        ok = cudaMemPoolCreate(&s->asset_pool, &props) == cudaSuccess;
        uint64_t keep = uint64_t(cfg->budget_bytes);
        if (ok) cudaMemPoolSetAttribute(s->asset_pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s->slots.resize(size_t(cfg->batch_slots));
    for (Slot& sl : s->slots) {
        ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
             cudaHostAlloc(reinterpret_cast<void**>(&sl.h_table), sizeof(ServeTable), cudaHostAllocDefault) == cudaSuccess &&
             cudaMalloc(&sl.d_table, sizeof(ServeTable)) == cudaSuccess &&
             cudaMalloc(&sl.d_q, size_t(cfg->batch_queries) * sizeof(htex_query)) == cudaSuccess &&
             cudaMalloc(&sl.d_out, size_t(cfg->batch_queries) * 4 * sizeof(float)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        release(s);
        delete s;
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    s->worker = std::thread(run, s);
    *out = s;
    return HTEX_OK;
}

extern "C" htex_status htex_server_add_asset(htex_server* s, const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                             const int32_t* log2_res, const void* pool, const float* scales,
                                             int32_t* asset_id) {
    if (!s || !m || !log2_res || !pool || !asset_id || channels < 1 || channels > 4 || !htex_dtype_valid(dtype))
        return HTEX_ERR_INVALID_ARG;
    if ((dtype == HTEX_F16 || dtype == HTEX_BF16 || dtype == HTEX_E4M3) && !scales) return HTEX_ERR_INVALID_ARG;
    for (int32_t e = 0; e < m->E; ++e)
        if (log2_res[e] < 0 || log2_res[e] > kMaxLog2Res) return HTEX_ERR_BAD_TEXTURE;
    ServeAsset* a = new (std::nothrow) ServeAsset;
    if (!a) return HTEX_ERR_OUT_OF_MEMORY;
    htex_status st;
    try {
        st = htex_asset_arrays(m, channels, dtype, log2_res, scales, &a->arrays);
    } catch (const std::bad_alloc&) {
        st = HTEX_ERR_OUT_OF_MEMORY;
    }
    if (st != HTEX_OK) {
        delete a;
        return st;
    }
    a->bytes = htex_asset_device_bytes(a->arrays);
    a->fmt = format_of(dtype, channels);
    if (a->bytes > s->cfg.budget_bytes) {
        delete a;
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    const auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t rec_b = a->arrays.rec.size() * 4, hdr_b = a->arrays.hdr.size() * 4, sc_b = a->arrays.scale.size() * 4;
    a->off_hdr = up(rec_b);
    a->off_scale = a->off_hdr + up(hdr_b);
    a->off_pool = a->off_scale + up(sc_b);
    const size_t total = a->off_pool + up(size_t(std::max<int64_t>(a->arrays.pool_bytes, 16)));
    void* dev = nullptr;
    if (cudaHostAlloc(&a->host, total, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&dev, a->host, 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&a->uploaded, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(a->host);
        delete a;
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    a->dev_host = static_cast<const uint8_t*>(dev);
    uint8_t* h = static_cast<uint8_t*>(a->host);
    std::memcpy(h, a->arrays.rec.data(), rec_b);
    std::memcpy(h + a->off_hdr, a->arrays.hdr.data(), hdr_b);
    std::memcpy(h + a->off_scale, a->arrays.scale.data(), sc_b);
    std::memcpy(h + a->off_pool, pool, size_t(a->arrays.pool_bytes));
    std::lock_guard<std::mutex> g(s->mu);
    if (s->error != HTEX_OK) {
        cudaEventDestroy(a->uploaded);
        cudaFreeHost(a->host);
        delete a;
        return s->error;
    }
    const int32_t k = s->num_assets.load();
    if (k >= kMaxAssets) {
        cudaEventDestroy(a->uploaded);
        cudaFreeHost(a->host);
        delete a;
        return HTEX_ERR_UNSUPPORTED;
    }
    s->assets[k] = a;
    s->formats.fetch_or(1u << a->fmt);
    s->num_assets.store(k + 1);
    *asset_id = k;
    return HTEX_OK;
}

// Device address of a page-locked, mapped host buffer, else null.
static const void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

extern "C" htex_status htex_server_submit(htex_server* s, int32_t asset_id, const htex_query* q, int64_t n,
                                          float* out, int64_t* request_id) {
    if (!s || !request_id || n < 0 || n >= (int64_t(1) << 40)) return HTEX_ERR_INVALID_ARG;
    if (n > 0 && (!q || !out)) return HTEX_ERR_INVALID_ARG;
    Request* r = new (std::nothrow) Request;
    if (!r) return HTEX_ERR_OUT_OF_MEMORY;
    r->asset = asset_id;
    r->q = q;
    r->out = out;
    r->n = n;
    if (n > 0) {
        const void* mq = mapped_host(q);
        void* mo = const_cast<void*>(mapped_host(out));
        if (mq && mo && ((reinterpret_cast<uintptr_t>(mq) | reinterpret_cast<uintptr_t>(mo)) & 15u) == 0) {
            r->dq = static_cast<const htex_query*>(mq);
            r->dout = static_cast<float*>(mo);
        }
    }
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> g(s->mu);
    if (s->error != HTEX_OK) {
        delete r;
        return s->error;
    }
    if (asset_id < 0 || asset_id >= s->num_assets.load()) {
        delete r;
        return HTEX_ERR_INVALID_ARG;
    }
    r->id = s->next_id++;
    *request_id = r->id;
    ++s->submitted;
    if (n == 0) {
        s->completed.emplace_back(r->id, 0.0);
        ++s->finished;
        ++s->stats.completed;
        delete r;
    } else {
        s->incoming.push_back(r);
    }
    s->cv.notify_all();
    return HTEX_OK;
}

extern "C" htex_status htex_server_poll(htex_server* s, int64_t* ids, double* latency_s, int32_t capacity,
                                        int32_t* count) {
    if (!s || !count || capacity < 0 || (capacity > 0 && (!ids || !latency_s))) return HTEX_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    const int32_t k = int32_t(std::min<size_t>(size_t(capacity), s->completed.size()));
    for (int32_t i = 0; i < k; ++i) {
        ids[i] = s->completed[size_t(i)].first;
        latency_s[i] = s->completed[size_t(i)].second;
    }
    s->completed.erase(s->completed.begin(), s->completed.begin() + k);
    *count = k;
    return s->error;
}

extern "C" htex_status htex_server_drain(htex_server* s, double timeout_s) {
    if (!s || !(timeout_s >= 0)) return HTEX_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> g(s->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (s->finished < s->submitted && s->error == HTEX_OK) {
        if (s->cv.wait_until(g, deadline) == std::cv_status::timeout && s->finished < s->submitted)
            return HTEX_ERR_TIMEOUT;
    }
    return s->error;
}

extern "C" htex_status htex_server_get_stats(htex_server* s, htex_server_stats* st) {
    if (!s || !st) return HTEX_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    *st = s->stats;
    st->resident_bytes = s->resident_bytes;
    return s->error;
}

extern "C" void htex_server_destroy(htex_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    release(s);
    delete s;
}
