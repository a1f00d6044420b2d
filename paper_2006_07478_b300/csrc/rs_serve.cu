// rs_serve.cu -- continuous-batching server over the pipeline (the serving form).
//
// Requests (one stream each, in host memory) arrive at any time.  The server admits a
// request when its inputs and outputs fit in the free part of a caller-provided device
// arena (a ring), copies it in, and groups every admitted request that is not yet
// running into the next batch: one rs_run over all of them.  Up to `max_inflight`
// batches are queued on the server's CUDA stream at once, so requests that arrive while
// others are on the GPU join the next batch and their work overlaps on the device.
// A batch's results come back with one gather kernel (every member's output arrays into
// one contiguous region of the arena) and one device-to-host copy into a page-locked
// staging buffer of the server's; when the batch's completion event fires they are
// copied on the host into the requests' output buffers, its arena space is released and
// its request ids are reported by rs_server_poll.  (A batch whose results do not fit
// that path falls back to one copy per output array.)
//
// Nothing here allocates device memory; the arena is the caller's.  The staging buffers
// are host memory, allocated when a batch first needs one that large and reused.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <deque>
#include <new>
#include <vector>

#include "rs_internal.h"

namespace {

struct Req {
    uint64_t id;
    rs_request r;
    uint64_t off, bytes;         // arena chunk
    uint32_t *d_count;           // the request's device outputs (in its arena chunk)
    unsigned long long *d_sum;
    uint32_t *d_min;
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

struct Batch {
    rs_pipeline *p = nullptr;
    std::vector<uint64_t> ids;
    uint64_t ws_bound = 0;       // workspace this batch will need, bounded from above
    uint64_t head_after = 0;     // ring head after this batch's last allocation
    uint64_t live_bytes = 0;     // bytes this batch holds in the ring
    cudaEvent_t ev = nullptr;
    Stage stage;                 // results staging (gathered path), returned at retire
    std::vector<Scatter> scat;   // where each staged output array goes
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

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct rs_server {
    rs_stage_desc st[RS_MAX_STAGES];
    uint32_t n_stages = 0;
    rs_pipeline_opts opts;
    unsigned char *arena = nullptr;
    uint64_t cap = 0;
    // ring allocator: live bytes occupy [tail, head) modulo cap
    uint64_t head = 0, tail = 0, live = 0, peak = 0;
    std::deque<Req> queued;
    Batch forming;
    std::vector<Req> forming_members;
    std::deque<Batch> inflight;
    std::vector<rs_pipeline *> pool;
    std::vector<cudaEvent_t> free_events;   // completion events of retired batches, reused
    std::vector<Stage> free_stages;         // staging buffers of retired batches, reused
    std::vector<uint64_t> completed;
    uint64_t next_id = 1;
    uint32_t max_batch = 4096, max_inflight = 2;
    cudaStream_t stream = nullptr;
    rs_server_stats stats;
};

// Contiguous allocation of b bytes from the ring.  Live bytes occupy [tail, head)
// modulo cap.  When the end of the arena is too short, the allocation wraps to 0 and
// the skipped end is charged to the caller (*charged) until the tail passes it.
static bool ring_alloc(rs_server *s, uint64_t b, uint64_t *off, uint64_t *charged)
{
    if (b > s->cap) return false;
    if (s->live == 0) s->head = s->tail = 0;
    uint64_t skip = 0;
    if (s->live == 0 || s->head > s->tail) {
        if (s->cap - s->head >= b) {
            *off = s->head;
        } else if (s->tail >= b) {
            skip = s->cap - s->head;
            *off = 0;
        } else {
            return false;
        }
    } else {   // wrapped (head < tail) or full (head == tail, live > 0)
        if (s->tail - s->head >= b) *off = s->head;
        else return false;
    }
    s->head = *off + b;
    s->live += b + skip;
    if (s->live > s->peak) s->peak = s->live;
    *charged = b + skip;
    return true;
}

// Upper bound of the workspace bytes one more stream adds to a batch (the layout of
// rs_workspace_size: merge slots, unit count, planner words and unit records for loaded
// streams, one stream-table entry for every stream, each piece 256-byte aligned).
static uint64_t stream_ws_bound(const rs_server *s, const rs_request &r)
{
    uint64_t b = a256(sizeof(DevStream)) + 256;
    if (s->st[0].kind == RS_ENUM_LOAD && r.n_regions) {
        const uint64_t kp = s->opts.regions_per_unit ? s->opts.regions_per_unit : 128;
        const uint64_t c = s->opts.region_cost ? s->opts.region_cost : RS_STEP_REGION;
        const uint64_t D = c * kp;
        const uint64_t units = (c * r.n_regions + r.n_elements + D - 1) / D;
        const uint64_t tiles = (r.n_regions + RS_PLAN_TILE_SMALL - 1) / RS_PLAN_TILE_SMALL;   // at most
        b += a256(units * sizeof(Slot)) + 256 + a256(tiles * 8) + a256((units + 1) * sizeof(UnitRec));
    }
    return b;
}

static uint64_t request_bytes(const rs_server *s, const rs_request &r)
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
    (void)s;
    return b < 256 ? 256 : b;
}

// Copy a request into its arena chunk and register it with the forming batch.
static rs_status admit(rs_server *s, Req &q)
{
    if (!s->forming.p) {
        if (!s->pool.empty()) {
            s->forming.p = s->pool.back();
            s->pool.pop_back();
            rs_clear_streams(s->forming.p);
        } else {
            rs_status st = rs_pipeline_create(s->st, s->n_stages, &s->opts, &s->forming.p);
            if (st != RS_OK) return st;
        }
    }
    unsigned char *base = s->arena + q.off;
    size_t o = 0;
    rs_stream_desc d;
    memset(&d, 0, sizeof d);
    d.n_regions = q.r.n_regions;
    const uint64_t R = q.r.n_regions;
    auto put = [&](const void *src, size_t bytes, const void **dst) -> bool {
        *dst = base + o;
        if (bytes && cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            return false;
        o += a256(bytes);
        return true;
    };
    if (q.r.parents && !put(q.r.parents, R * 4, (const void **)&d.parents)) return RS_ERR_CUDA;
    if (q.r.region_len && !put(q.r.region_len, R * 4, (const void **)&d.region_len)) return RS_ERR_CUDA;
    if (q.r.elements && !put(q.r.elements, q.r.n_elements * 4, (const void **)&d.elements)) return RS_ERR_CUDA;
    if (q.r.ctx && !put(q.r.ctx, R * 4, (const void **)&d.ctx)) return RS_ERR_CUDA;
    d.n_elements = q.r.elements ? q.r.n_elements : 0;
    if (q.r.out_count) { d.out_count = (uint32_t *)(base + o); o += a256(R * 4); }
    if (q.r.out_sum) { d.out_sum = (uint64_t *)(base + o); o += a256(R * 8); }
    if (q.r.out_min) { d.out_min = (uint32_t *)(base + o); o += a256(R * 4); }
    q.d_count = d.out_count;
    q.d_sum = (unsigned long long *)d.out_sum;
    q.d_min = d.out_min;
    d.total_elements_hint = q.r.total_elements_hint;
    uint64_t sid = 0;
    rs_status st = rs_stream_submit(s->forming.p, &d, &sid);
    if (st != RS_OK) return st;
    s->forming.ids.push_back(q.id);
    s->forming.head_after = s->head;
    s->stats.admitted++;
    return RS_OK;
}

// Queue the batch's results as one gather into an arena region and one copy into a
// staging buffer (host side scattered at retire).  False, with nothing queued, when the
// arena has no room or no staging buffer can be had: the caller copies per array.
static bool gather_results(rs_server *s, Batch &b, const std::vector<Req> &members)
{
    std::vector<Scatter> scat;
    uint64_t rbytes = 0;
    size_t n_items = 0;
    for (const Req &q : members) {
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
    if (n_items == 0) return true;   // nothing to hand back
    const uint64_t tbytes = a256(n_items * sizeof(GatherItem));
    const uint64_t total = tbytes + a256(rbytes);
    // a staging buffer at least this large: reuse one, else allocate (rounded up to a
    // power of two, so that few sizes are ever allocated)
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
    uint64_t off = 0, charged = 0;
    if (!ring_alloc(s, total, &off, &charged)) {
        s->free_stages.push_back(sg);
        return false;
    }
    b.head_after = s->head;
    b.live_bytes += charged;
    unsigned char *dev = s->arena + off;
    GatherItem *items = reinterpret_cast<GatherItem *>(sg.p);
    size_t k = 0;
    for (const Req &q : members) {
        if (q.r.n_regions == 0) continue;
        const void *src[3] = {q.d_count, q.d_sum, q.d_min};
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
    if (cudaMemcpyAsync(dev, sg.p, n_items * sizeof(GatherItem), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        (rs_gather_kernel<<<grid, 128, 0, s->stream>>>(reinterpret_cast<const GatherItem *>(dev), (uint32_t)n_items),
         cudaGetLastError() != cudaSuccess) ||
        cudaMemcpyAsync(sg.p + tbytes, dev + tbytes, rbytes, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) {
        // the arena charge stays with the batch; the copies are not queued: fall back
        s->free_stages.push_back(sg);
        return false;
    }
    for (Scatter &c : scat) c.off += tbytes;
    b.stage = sg;
    b.scat.swap(scat);
    return true;
}

// Launch the forming batch: workspace from the ring, one rs_run, result copies back
// to each request's host buffers, then a completion event.
static rs_status launch(rs_server *s, std::vector<Req> &members)
{
    Batch &b = s->forming;
    uint64_t wsb = 0;
    rs_status st = rs_workspace_size(b.p, &wsb);
    if (st != RS_OK) return st;
    uint64_t woff = 0, charged = 0;
    if (!ring_alloc(s, a256(wsb), &woff, &charged)) {
        // no room for the workspace: wait for a batch to finish, unless none is running
        return s->inflight.empty() ? RS_ERR_CAPACITY : RS_ERR_NOT_READY;
    }
    b.head_after = s->head;
    b.live_bytes += charged;
    st = rs_run(b.p, s->arena + woff, a256(wsb), (rs_cuda_stream)s->stream);
    if (st != RS_OK) return st;
    if (gather_results(s, b, members)) {
        s->stats.gathered++;
    } else {
        for (size_t i = 0; i < members.size(); ++i) {
            rs_region_results dst;
            dst.count = members[i].r.out_count;
            dst.sum = members[i].r.out_sum;
            dst.min = members[i].r.out_min;
            st = rs_fetch_region_results(b.p, i, &dst, (rs_cuda_stream)s->stream);
            if (st != RS_OK) return st;
        }
    }
    if (!b.ev && !s->free_events.empty()) {
        b.ev = s->free_events.back();
        s->free_events.pop_back();
    }
    if (!b.ev && cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) return RS_ERR_CUDA;
    if (cudaEventRecord(b.ev, s->stream) != cudaSuccess) return RS_ERR_CUDA;
    s->stats.batches++;
    s->stats.largest_batch = b.ids.size() > s->stats.largest_batch ? b.ids.size() : s->stats.largest_batch;
    s->inflight.push_back(b);
    s->forming = Batch();
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
    // validate the stage list and options once, through the pipeline's own checks
    rs_pipeline *probe = nullptr;
    rs_status st = rs_pipeline_create(stages, n_stages, opts, &probe);
    if (st != RS_OK) return st;
    rs_server *s = new (std::nothrow) rs_server();
    if (!s) {
        rs_pipeline_destroy(probe);
        return RS_ERR_NOMEM;
    }
    memcpy(s->st, stages, n_stages * sizeof(rs_stage_desc));
    s->n_stages = n_stages;
    rs_pipeline_get_opts(probe, &s->opts);
    s->pool.push_back(probe);
    s->arena = (unsigned char *)arena;
    s->cap = arena_bytes & ~(uint64_t)255;
    s->max_batch = max_batch ? max_batch : 4096;
    s->max_inflight = max_inflight ? max_inflight : 2;
    s->stream = (cudaStream_t)stream;
    memset(&s->stats, 0, sizeof s->stats);
    *out = s;
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
    q.off = 0;
    q.bytes = a256(request_bytes(s, *r));
    if (q.bytes > s->cap / 2) return RS_ERR_CAPACITY;   // could never be admitted beside a workspace
    try {
        s->queued.push_back(q);
    } catch (...) {
        return RS_ERR_NOMEM;
    }
    s->stats.submitted++;
    if (req_id) *req_id = q.id;
    return RS_OK;
}

rs_status rs_server_progress(rs_server *s)
{
    if (!s) return RS_ERR_INVALID;
    // 1. retire finished batches (in order)
    while (!s->inflight.empty()) {
        Batch &b = s->inflight.front();
        cudaError_t e = cudaEventQuery(b.ev);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return RS_ERR_CUDA;
        // gathered results: from the staging buffer into the requests' output buffers
        for (const Scatter &c : b.scat) memcpy(c.dst, b.stage.p + c.off, c.bytes);
        if (b.stage.p) s->free_stages.push_back(b.stage);
        b.stage = Stage();
        b.scat.clear();
        for (uint64_t id : b.ids) s->completed.push_back(id);
        s->stats.completed += b.ids.size();
        // release the batch's ring space: everything up to its last allocation
        s->tail = b.head_after;
        s->live -= b.live_bytes;
        if (s->live == 0) s->head = s->tail = 0;
        s->free_events.push_back(b.ev);   // reused by a later batch (no driver call per batch)
        b.ev = nullptr;
        s->pool.push_back(b.p);
        s->inflight.pop_front();
    }
    // 2. admit queued requests while the arena has room
    while (!s->queued.empty() && s->forming.ids.size() < s->max_batch) {
        Req &q = s->queued.front();
        // admission by free device memory: the request and the batch's grown workspace
        // must both fit (the workspace is taken from the ring when the batch launches)
        const uint64_t ws_next = s->forming.ws_bound + stream_ws_bound(s, q.r) + 512;
        const uint64_t h0 = s->head, t0 = s->tail, l0 = s->live, p0 = s->peak;
        uint64_t off = 0, charged = 0, woff = 0, wch = 0;
        if (!ring_alloc(s, q.bytes, &off, &charged)) break;
        const uint64_t h1 = s->head, t1 = s->tail, l1 = s->live, p1 = s->peak;
        const bool ws_fits = ring_alloc(s, a256(ws_next), &woff, &wch);
        if (!ws_fits) {
            s->head = h0; s->tail = t0; s->live = l0; s->peak = p0;   // undo the request's allocation
            break;
        }
        s->head = h1; s->tail = t1; s->live = l1; s->peak = p1;       // keep only the request's
        q.off = off;
        s->forming.live_bytes += charged;
        s->forming.ws_bound = ws_next - 512;
        rs_status st = admit(s, q);
        if (st != RS_OK) return st;
        s->forming_members.push_back(q);
        s->queued.pop_front();
    }
    // 3. launch the forming batch if a slot is free
    if (!s->forming.ids.empty() && s->inflight.size() < s->max_inflight) {
        rs_status st = launch(s, s->forming_members);
        if (st == RS_OK) {
            s->forming_members.clear();
        } else if (st != RS_ERR_NOT_READY) {
            return st;
        }
    }
    s->stats.in_flight = s->inflight.size();
    s->stats.queued = s->queued.size();
    s->stats.arena_live = s->live;
    s->stats.arena_peak = s->peak;
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
    for (auto &b : s->inflight) {
        if (b.ev) cudaEventDestroy(b.ev);
        if (b.p) rs_pipeline_destroy(b.p);
    }
    if (s->forming.p) rs_pipeline_destroy(s->forming.p);
    if (s->forming.ev) cudaEventDestroy(s->forming.ev);
    for (auto *p : s->pool) rs_pipeline_destroy(p);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    for (auto &b : s->inflight)
        if (b.stage.p) cudaFreeHost(b.stage.p);
    for (Stage &g : s->free_stages) cudaFreeHost(g.p);
    delete s;
    return RS_OK;
}

}  // extern "C"
