// rs_serve.cu -- continuous-batching server over the pipeline (the serving form).
//
// Requests (one stream each, in host memory) arrive at any time.  A request is admitted
// when its inputs, outputs and resident state fit in the free part of a caller-provided
// device arena; its inputs are copied in on a copy stream of the server's own.  From
// then on the request is active: its data and its planning state stay on the device
// until it finishes.  The server advances every active request a slice at a time: one
// launch (rs_run over the active requests, each submitted with rs_stream_submit_slice)
// runs at most `slice_units` work units of each, so a request that arrives while others
// are on the GPU joins the next launch, and a long request holds a short one back by at
// most one slice.  Up to `max_inflight` slices are queued on the server's compute stream
// and the copies overlap them on the device: admissions' inputs go up on one copy
// stream, and the results of the requests a slice finishes come back on another (one
// gather kernel packing their output arrays into one arena region, one device-to-host
// copy into a page-locked staging buffer, scattered into the requests' host buffers when
// the copy has landed; when that path has no room, one copy per array).
//
// Nothing here allocates device memory; the arena is the caller's (a first-fit free
// list, so requests may finish in any order).  The staging buffers are host memory,
// allocated when a slice first needs one that large and reused.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <vector>

#include "rs_internal.h"

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// first-fit free list over [0, cap) with coalescing
struct FreeList {
    std::map<uint64_t, uint64_t> free;   // offset -> bytes
    uint64_t live = 0, peak = 0;
    void reset(uint64_t cap)
    {
        free.clear();
        if (cap) free[0] = cap;
        live = peak = 0;
    }
    bool alloc(uint64_t b, uint64_t *off)
    {
        for (auto it = free.begin(); it != free.end(); ++it) {
            if (it->second < b) continue;
            *off = it->first;
            const uint64_t rest = it->second - b;
            const uint64_t o2 = it->first + b;
            free.erase(it);
            if (rest) free[o2] = rest;
            live += b;
            if (live > peak) peak = live;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t b)
    {
        live -= b;
        auto it = free.emplace(off, b).first;
        auto nx = std::next(it);
        if (nx != free.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free.erase(nx);
        }
        if (it != free.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free.erase(it);
            }
        }
    }
};

struct Req {
    uint64_t id = 0;
    rs_request r;
    uint64_t off = 0, bytes = 0;        // arena chunk: inputs, outputs, resident state
    rs_stream_desc d;                   // device view of the request
    void *state = nullptr;
    uint64_t state_bytes = 0;
    uint64_t units = 0, next = 0;       // its work units; the next one to run
    uint64_t round = 0;                 // admission round (whose copy-in event covers it)
};

// one output array to gather: device source, device destination, 4-byte words
struct GatherItem {
    const uint4 *src;
    uint4 *dst;
    unsigned long long words;
};

// one output array to hand back: the request's host buffer, its offset in the staging
// buffer, bytes
struct Scatter {
    void *dst;
    uint64_t off, bytes;
};

// page-locked host staging buffer
struct Stage {
    unsigned char *p = nullptr;
    uint64_t cap = 0;
};

// one launch, and the requests whose last unit it runs
struct Slice {
    rs_pipeline *p = nullptr;
    uint64_t ws_off = 0, ws_bytes = 0, res_off = 0, res_bytes = 0;   // arena chunks of the slice
    std::vector<Req> finishing;
    cudaEvent_t done = nullptr;       // their results have landed in host memory
    Stage stage;
    std::vector<Scatter> scat;
};

// Each CTA copies whole items, 16 bytes per thread and step.  Sources and destinations
// are 16-byte aligned and padded to 256 bytes in the arena, so rounding an item up to
// 16 bytes stays inside its allocation.
__global__ void __launch_bounds__(128) rs_gather_kernel(const GatherItem *items, uint32_t n)
{
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const GatherItem it = items[i];
        const unsigned long long n16 = (it.words + 3) / 4;
        for (unsigned long long k = threadIdx.x; k < n16; k += blockDim.x) it.dst[k] = it.src[k];
    }
}

}  // namespace

struct rs_server {
    rs_stage_desc st[RS_MAX_STAGES];
    uint32_t n_stages = 0;
    rs_pipeline_opts opts;
    unsigned char *arena = nullptr;
    uint64_t cap = 0;
    FreeList fl;
    std::deque<Req> queued;
    std::vector<Req> active;
    std::deque<Slice> inflight;
    std::vector<rs_pipeline *> pool;
    rs_pipeline *probe = nullptr;           // sizes requests' resident state
    std::vector<cudaEvent_t> free_events;
    std::vector<Stage> free_stages;
    std::vector<uint64_t> completed;
    // admission rounds not yet waited on by the compute stream: {round, copy-in event}
    std::deque<std::pair<uint64_t, cudaEvent_t>> rounds;
    uint64_t round = 0;
    uint64_t next_id = 1;
    uint32_t max_batch = 4096, max_inflight = 2;
    uint32_t slice_units = 64;
    cudaStream_t stream = nullptr;                // slices (the caller's stream)
    cudaStream_t cin = nullptr, cout = nullptr;   // copy-in, results
    rs_server_stats stats;
};

static rs_status take_event(rs_server *s, cudaEvent_t *e)
{
    if (!s->free_events.empty()) {
        *e = s->free_events.back();
        s->free_events.pop_back();
        return RS_OK;
    }
    return cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

static uint64_t request_io_bytes(const rs_request &r)
{
    const uint64_t R = r.n_regions;
    uint64_t b = 0;
    if (r.parents) b += a256(R * 4);
    if (r.region_len) b += a256(R * 4);
    if (r.elements) b += a256(r.n_elements * 4);
    if (r.ctx) b += a256(R * 4);
    if (r.out_count) b += a256(R * 4);
    if (r.out_sum) b += a256(R * 8);
    if (r.out_min) b += a256(R * 4);
    return b < 256 ? 256 : b;
}

// the request's device view: inputs and outputs laid out in its chunk, then its state
static void layout_request(rs_server *s, Req &q)
{
    unsigned char *base = s->arena + q.off;
    size_t o = 0;
    rs_stream_desc &d = q.d;
    memset(&d, 0, sizeof d);
    d.n_regions = q.r.n_regions;
    const uint64_t R = q.r.n_regions;
    auto put = [&](const void *src, size_t bytes) -> void * {
        if (!src) return nullptr;
        void *p = base + o;
        o += a256(bytes);
        return p;
    };
    d.parents = (const uint32_t *)put(q.r.parents, R * 4);
    d.region_len = (const uint32_t *)put(q.r.region_len, R * 4);
    d.elements = (const uint32_t *)put(q.r.elements, q.r.n_elements * 4);
    d.ctx = (const uint32_t *)put(q.r.ctx, R * 4);
    d.n_elements = q.r.elements ? q.r.n_elements : 0;
    d.out_count = (uint32_t *)put(q.r.out_count, R * 4);
    d.out_sum = (uint64_t *)put(q.r.out_sum, R * 8);
    d.out_min = (uint32_t *)put(q.r.out_min, R * 4);
    d.total_elements_hint = q.r.total_elements_hint;
    q.state = base + a256(o);
}

static rs_status copy_in(rs_server *s, const Req &q)
{
    const uint64_t R = q.r.n_regions;
    struct {
        const void *src;
        const void *dst;
        uint64_t bytes;
    } c[4] = {{q.r.parents, q.d.parents, R * 4},
              {q.r.region_len, q.d.region_len, R * 4},
              {q.r.elements, q.d.elements, q.r.n_elements * 4},
              {q.r.ctx, q.d.ctx, R * 4}};
    for (auto &x : c)
        if (x.src && x.bytes &&
            cudaMemcpyAsync(const_cast<void *>(x.dst), x.src, x.bytes, cudaMemcpyHostToDevice, s->cin) != cudaSuccess)
            return RS_ERR_CUDA;
    return RS_OK;
}

// Queue the finishing requests' results back to the host on the results stream: one
// gather into an arena region and one copy into a staging buffer (scattered on the host
// at retire).  False, with nothing queued, when no arena room or staging buffer can be
// had: the caller copies each array.
static bool gather_results(rs_server *s, Slice &b)
{
    std::vector<Scatter> scat;
    uint64_t rbytes = 0;
    size_t n_items = 0;
    for (const Req &q : b.finishing) {
        const uint64_t R = q.r.n_regions;
        const void *hd[3] = {q.r.out_count, q.r.out_sum, q.r.out_min};
        const uint64_t by[3] = {R * 4, R * 8, R * 4};
        for (int k = 0; k < 3; ++k) {
            if (!hd[k] || R == 0) continue;
            scat.push_back(Scatter{const_cast<void *>(hd[k]), rbytes, by[k]});
            rbytes += (by[k] + 15) & ~(uint64_t)15;
            ++n_items;
        }
    }
    if (n_items == 0) return true;
    const uint64_t tbytes = a256(n_items * sizeof(GatherItem));
    const uint64_t total = tbytes + a256(rbytes);
    Stage sg;
    for (size_t i = 0; i < s->free_stages.size(); ++i) {
        if (s->free_stages[i].cap >= total) {
            sg = s->free_stages[i];
            s->free_stages.erase(s->free_stages.begin() + i);
            break;
        }
    }
    if (!sg.p) {
        uint64_t cap = 1u << 16;
        while (cap < total) cap <<= 1;
        if (cudaMallocHost((void **)&sg.p, cap) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        sg.cap = cap;
    }
    uint64_t off = 0;
    if (!s->fl.alloc(a256(total), &off)) {
        s->free_stages.push_back(sg);
        return false;
    }
    unsigned char *dev = s->arena + off;
    GatherItem *items = reinterpret_cast<GatherItem *>(sg.p);
    size_t k = 0;
    for (const Req &q : b.finishing) {
        if (q.r.n_regions == 0) continue;
        const void *src[3] = {q.d.out_count, q.d.out_sum, q.d.out_min};
        const void *hd[3] = {q.r.out_count, q.r.out_sum, q.r.out_min};
        const uint64_t words[3] = {q.r.n_regions, 2 * q.r.n_regions, q.r.n_regions};
        for (int j = 0; j < 3; ++j) {
            if (!hd[j]) continue;
            items[k].src = reinterpret_cast<const uint4 *>(src[j]);
            items[k].dst = reinterpret_cast<uint4 *>(dev + tbytes + scat[k].off);
            items[k].words = words[j];
            ++k;
        }
    }
    const uint32_t grid = n_items < 1024 ? (uint32_t)n_items : 1024u;
    if (cudaMemcpyAsync(dev, sg.p, n_items * sizeof(GatherItem), cudaMemcpyHostToDevice, s->cout) != cudaSuccess ||
        (rs_gather_kernel<<<grid, 128, 0, s->cout>>>(reinterpret_cast<const GatherItem *>(dev), (uint32_t)n_items),
         cudaGetLastError() != cudaSuccess) ||
        cudaMemcpyAsync(sg.p + tbytes, dev + tbytes, rbytes, cudaMemcpyDeviceToHost, s->cout) != cudaSuccess) {
        s->fl.release(off, a256(total));
        s->free_stages.push_back(sg);
        return false;
    }
    for (Scatter &c : scat) c.off += tbytes;
    b.stage = sg;
    b.scat.swap(scat);
    b.res_off = off;
    b.res_bytes = a256(total);
    return true;
}

// Launch one slice over the active requests: each runs its next slice_units units (all of
// them when slice_units is 0).  RS_ERR_NOT_READY when the arena has no room for the
// slice's workspace now.
static rs_status launch_slice(rs_server *s)
{
    Slice b;
    if (!s->pool.empty()) {
        b.p = s->pool.back();
        s->pool.pop_back();
        rs_clear_streams(b.p);
    } else {
        rs_status st = rs_pipeline_create(s->st, s->n_stages, &s->opts, &b.p);
        if (st != RS_OK) return st;
        // the stream table's pinned copy for a whole batch now, not grown mid-stream
        st = rs_pipeline_reserve_streams(b.p, s->max_batch);
        if (st != RS_OK) {
            rs_pipeline_destroy(b.p);
            return st;
        }
    }
    std::vector<size_t> members;
    uint64_t need_round = 0;
    for (size_t i = 0; i < s->active.size() && members.size() < s->max_batch; ++i) {
        Req &q = s->active[i];
        if (q.next >= q.units) continue;
        const uint64_t n = s->slice_units ? s->slice_units : q.units;
        rs_status st = rs_stream_submit_slice(b.p, &q.d, q.state, q.state_bytes, q.next, n, nullptr);
        if (st != RS_OK) {
            s->pool.push_back(b.p);
            return st;
        }
        members.push_back(i);
        if (q.round > need_round) need_round = q.round;
    }
    if (members.empty()) {
        s->pool.push_back(b.p);
        return RS_OK;
    }
    uint64_t wsb = 0;
    rs_status st = rs_run_workspace_bytes(b.p, &wsb);
    if (st != RS_OK) {
        s->pool.push_back(b.p);
        return st;
    }
    uint64_t woff = 0;
    if (!s->fl.alloc(a256(wsb), &woff)) {
        s->pool.push_back(b.p);
        return s->inflight.empty() ? RS_ERR_CAPACITY : RS_ERR_NOT_READY;
    }
    b.ws_off = woff;
    b.ws_bytes = a256(wsb);
    // the slice reads the inputs of every admission round up to its newest member's
    // (an event may be recorded again once a wait on it is enqueued)
    while (!s->rounds.empty() && s->rounds.front().first <= need_round) {
        if (cudaStreamWaitEvent(s->stream, s->rounds.front().second, 0) != cudaSuccess) return RS_ERR_CUDA;
        s->free_events.push_back(s->rounds.front().second);
        s->rounds.pop_front();
    }
    st = rs_run(b.p, s->arena + woff, b.ws_bytes, (rs_cuda_stream)s->stream);
    if (st != RS_OK) return st;
    // requests whose last unit ran: their results go back on the results stream
    std::vector<Req> keep;
    keep.reserve(s->active.size());
    size_t mi = 0;
    for (size_t i = 0; i < s->active.size(); ++i) {
        Req &q = s->active[i];
        if (mi < members.size() && members[mi] == i) {
            ++mi;
            q.next += s->slice_units ? s->slice_units : q.units;
            if (q.next >= q.units) {
                b.finishing.push_back(q);
                continue;
            }
        }
        keep.push_back(q);
    }
    s->active.swap(keep);
    cudaEvent_t ran;
    if (take_event(s, &ran) != RS_OK) return RS_ERR_CUDA;
    if (cudaEventRecord(ran, s->stream) != cudaSuccess) return RS_ERR_CUDA;
    if (cudaStreamWaitEvent(s->cout, ran, 0) != cudaSuccess) return RS_ERR_CUDA;
    s->free_events.push_back(ran);
    if (!b.finishing.empty()) {
        if (gather_results(s, b)) {
            s->stats.gathered++;
        } else {
            s->stats.per_array++;
            for (const Req &q : b.finishing) {
                const uint64_t R = q.r.n_regions;
                if (!R) continue;
                if ((q.r.out_count && cudaMemcpyAsync(q.r.out_count, q.d.out_count, R * 4, cudaMemcpyDeviceToHost,
                                                      s->cout) != cudaSuccess) ||
                    (q.r.out_sum && cudaMemcpyAsync(q.r.out_sum, q.d.out_sum, R * 8, cudaMemcpyDeviceToHost,
                                                    s->cout) != cudaSuccess) ||
                    (q.r.out_min && cudaMemcpyAsync(q.r.out_min, q.d.out_min, R * 4, cudaMemcpyDeviceToHost,
                                                    s->cout) != cudaSuccess))
                    return RS_ERR_CUDA;
            }
        }
    }
    if (take_event(s, &b.done) != RS_OK) return RS_ERR_CUDA;
    if (cudaEventRecord(b.done, s->cout) != cudaSuccess) return RS_ERR_CUDA;
    s->stats.batches++;
    if (members.size() > s->stats.largest_batch) s->stats.largest_batch = members.size();
    s->inflight.push_back(b);
    return RS_OK;
}

extern "C" {

rs_status rs_server_create(const rs_stage_desc *stages, uint32_t n_stages, const rs_pipeline_opts *opts,
                           void *arena, uint64_t arena_bytes, uint32_t max_batch, uint32_t max_inflight,
                           rs_cuda_stream stream, rs_server **out)
{
    if (!out || !arena || arena_bytes < 4096 || ((uintptr_t)arena & 255)) return RS_ERR_INVALID;
    *out = nullptr;
    // requests carry per-region outputs only: a pipeline ending in an emit sink is not served
    if (!stages || n_stages < 2 || n_stages > RS_MAX_STAGES || stages[n_stages - 1].kind == RS_EMIT)
        return RS_ERR_INVALID;
    // ... and a request has one leaf's results: linear pipelines only
    for (uint32_t i = 1; i < n_stages; ++i)
        if (stages[i].input && stages[i].input != i - 1) return RS_ERR_INVALID;
    // validate the stage list and options once, through the pipeline's own checks; a
    // request's units and state are sized for one strategy, so AUTO becomes TAG
    rs_pipeline_opts o;
    if (opts) o = *opts; else rs_default_opts(&o);
    if (o.strategy == RS_STRATEGY_AUTO) o.strategy = RS_STRATEGY_TAG;
    rs_pipeline *probe = nullptr;
    rs_status st = rs_pipeline_create(stages, n_stages, &o, &probe);
    if (st != RS_OK) return st;
    rs_server *s = new (std::nothrow) rs_server();
    if (!s) {
        rs_pipeline_destroy(probe);
        return RS_ERR_NOMEM;
    }
    memcpy(s->st, stages, n_stages * sizeof(rs_stage_desc));
    s->n_stages = n_stages;
    rs_pipeline_get_opts(probe, &s->opts);
    s->probe = probe;
    s->arena = (unsigned char *)arena;
    s->cap = arena_bytes & ~(uint64_t)255;
    s->fl.reset(s->cap);
    s->max_batch = max_batch ? max_batch : 4096;
    s->max_inflight = max_inflight ? max_inflight : 2;
    s->stream = (cudaStream_t)stream;
    memset(&s->stats, 0, sizeof s->stats);
    *out = s;
    return RS_OK;
}

rs_status rs_server_set_slice_units(rs_server *s, uint32_t units)
{
    if (!s) return RS_ERR_INVALID;
    s->slice_units = units;
    return RS_OK;
}

rs_status rs_server_submit(rs_server *s, const rs_request *r, uint64_t *req_id)
{
    if (!s || !r) return RS_ERR_INVALID;
    if (r->n_regions >= (1ull << 32) || r->n_elements >= (1ull << 32)) return RS_ERR_CAPACITY;
    if (r->n_regions && !r->region_len) return RS_ERR_INVALID;
    Req q;
    q.id = s->next_id++;
    q.r = *r;
    // the resident state this request's sliced runs need, sized like its device stream
    rs_stream_desc d;
    memset(&d, 0, sizeof d);
    d.n_regions = r->n_regions;
    d.region_len = r->region_len;
    d.n_elements = r->elements ? r->n_elements : 0;
    d.total_elements_hint = r->total_elements_hint;
    rs_status st = rs_stream_state_size(s->probe, &d, &q.state_bytes, &q.units);
    if (st != RS_OK) return st;
    q.bytes = a256(request_io_bytes(*r)) + a256(q.state_bytes);
    if (q.bytes > s->cap / 2) return RS_ERR_CAPACITY;   // could never be admitted beside a workspace
    try {
        if (q.units == 0) s->completed.push_back(q.id);   // nothing to run: done at once
        else s->queued.push_back(q);
    } catch (...) {
        return RS_ERR_NOMEM;
    }
    s->stats.submitted++;
    if (q.units == 0) {
        s->stats.admitted++;
        s->stats.completed++;
    }
    if (req_id) *req_id = q.id;
    return RS_OK;
}

rs_status rs_server_progress(rs_server *s)
{
    if (!s) return RS_ERR_INVALID;
    // the copy streams, made on first use (creating the server makes no CUDA call)
    if (!s->cin && cudaStreamCreateWithFlags(&s->cin, cudaStreamNonBlocking) != cudaSuccess) return RS_ERR_CUDA;
    if (!s->cout && cudaStreamCreateWithFlags(&s->cout, cudaStreamNonBlocking) != cudaSuccess) return RS_ERR_CUDA;
    // 1. retire slices whose finished requests' results have landed (in launch order)
    while (!s->inflight.empty()) {
        Slice &b = s->inflight.front();
        cudaError_t e = cudaEventQuery(b.done);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return RS_ERR_CUDA;
        for (const Scatter &c : b.scat) memcpy(c.dst, b.stage.p + c.off, c.bytes);
        if (b.stage.p) s->free_stages.push_back(b.stage);
        for (const Req &q : b.finishing) {
            s->completed.push_back(q.id);
            s->fl.release(q.off, q.bytes);
        }
        s->stats.completed += b.finishing.size();
        if (b.res_bytes) s->fl.release(b.res_off, b.res_bytes);
        s->fl.release(b.ws_off, b.ws_bytes);
        s->free_events.push_back(b.done);
        s->pool.push_back(b.p);
        s->inflight.pop_front();
    }
    // 2. admit queued requests while the arena has room for them; their inputs go up on
    //    the copy-in stream, and one event per round marks the copies done
    bool admitted = false;
    while (!s->queued.empty() && s->active.size() < s->max_batch) {
        Req &q = s->queued.front();
        uint64_t off = 0;
        if (!s->fl.alloc(q.bytes, &off)) break;
        q.off = off;
        q.round = s->round + 1;
        layout_request(s, q);
        rs_status st = copy_in(s, q);
        if (st != RS_OK) return st;
        s->active.push_back(q);
        s->queued.pop_front();
        s->stats.admitted++;
        admitted = true;
    }
    if (admitted) {
        cudaEvent_t ev;
        if (take_event(s, &ev) != RS_OK) return RS_ERR_CUDA;
        if (cudaEventRecord(ev, s->cin) != cudaSuccess) return RS_ERR_CUDA;
        s->rounds.push_back({++s->round, ev});
    }
    // 3. launch slices while fewer than max_inflight are queued
    while (s->inflight.size() < s->max_inflight) {
        bool work = false;
        for (const Req &q : s->active) work = work || q.next < q.units;
        if (!work) break;
        rs_status st = launch_slice(s);
        if (st == RS_ERR_NOT_READY) break;
        if (st != RS_OK) return st;
    }
    s->stats.in_flight = s->inflight.size();
    s->stats.queued = s->queued.size();
    s->stats.arena_live = s->fl.live;
    s->stats.arena_peak = s->fl.peak;
    return RS_OK;
}

rs_status rs_server_poll(rs_server *s, uint64_t *ids, uint32_t max, uint32_t *n)
{
    if (!s || !n) return RS_ERR_INVALID;
    uint32_t k = 0;
    while (k < max && k < s->completed.size()) {
        if (ids) ids[k] = s->completed[k];
        ++k;
    }
    s->completed.erase(s->completed.begin(), s->completed.begin() + k);
    *n = k;
    return RS_OK;
}

rs_status rs_server_get_stats(const rs_server *s, rs_server_stats *out)
{
    if (!s || !out) return RS_ERR_INVALID;
    *out = s->stats;
    return RS_OK;
}

rs_status rs_server_destroy(rs_server *s)
{
    if (!s) return RS_ERR_INVALID;
    cudaStreamSynchronize(s->stream);
    if (s->cin) cudaStreamSynchronize(s->cin);
    if (s->cout) cudaStreamSynchronize(s->cout);
    for (auto &b : s->inflight) {
        if (b.done) cudaEventDestroy(b.done);
        if (b.p) rs_pipeline_destroy(b.p);
        if (b.stage.p) cudaFreeHost(b.stage.p);
    }
    for (auto *p : s->pool) rs_pipeline_destroy(p);
    if (s->probe) rs_pipeline_destroy(s->probe);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    for (auto &r : s->rounds) cudaEventDestroy(r.second);
    for (Stage &g : s->free_stages) cudaFreeHost(g.p);
    if (s->cin) cudaStreamDestroy(s->cin);
    if (s->cout) cudaStreamDestroy(s->cout);
    delete s;
    return RS_OK;
}

}  // extern "C"
