// rs_api.cu -- host side of the C ABI declared in include/rs.h.
//
// Validates stage lists and streams, sizes the caller's workspace, lays out each
// processor's shared memory, picks the persistent grid, launches the kernel of
// rs_kernel.cu, reads counters back, captures runs into CUDA graphs and times
// candidate configurations for the autotuner (Section 5: the strategy should be
// chosen from measurements of the workload).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "rs_internal.h"

#define RS_VERSION 1u
#define RS_NOALLOC_MAX_STREAMS 64
#define RS_TAG_MAX_K 65536u         // parents per unit (tag strategy; the signal strategy's
                                    // per-parent shared memory limits it to RS_MAX_K)
#define RS_TAG_UNIT_STEPS 4096u     // tag strategy: default merge-path steps per unit
#define RS_TAG_UNIT_ELEMS 8192.0    // tag strategy: hashed units of about this many elements

static thread_local int g_last_cuda = 0;

static rs_status cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return RS_ERR_CUDA;
}

struct StreamPlan {
    uint32_t mode, K, n_units, plan_tiles, D, c;
    size_t slots_off, ucount_off, planlb_off, rec_off;
    // this run's share of the stream: units [slice_lo, slice_lo + slice_n) of full_units,
    // run_tiles planner tiles (all of them, or none when a sliced stream was planned
    // earlier); a sliced stream's scratch lives in its own state (offsets above relative to
    // it): st_zero bytes cleared when it is planned, st_total bytes in all
    uint32_t full_units, slice_lo, slice_n, run_tiles;
    bool sliced, plan_now;
    bool usum;    // fixed-parent units of a loaded stream of lengths (short regions)
    size_t usum_off, grp_off;
    size_t st_zero, st_total;
};

// A stream submitted for a sliced run (rs_stream_submit_slice): its resident state and the
// units the next run takes.
struct SliceInfo {
    bool on = false;
    void *state = nullptr;
    uint64_t state_bytes = 0, begin = 0, count = 0;
};

// The workspace layout of make_plan in fixed arrays, for rs_run_noalloc (no allocation).
struct FixedPlan {
    uint64_t total_units, plan_tiles;
    uint32_t Kmax;
    size_t zero_end, table_off, total;
    StreamPlan sp[RS_NOALLOC_MAX_STREAMS];
};

// rs_run_noalloc's stream table, passed by value as a kernel parameter (9.7 KB, within
// the 32 KB parameter space of sm_70 and later)
struct NoallocTable {
    DevStream s[RS_NOALLOC_MAX_STREAMS];
};

struct rs_pipeline {
    rs_stage_desc stages[RS_MAX_STAGES];
    uint32_t n_stages;
    rs_pipeline_opts opts;
    std::vector<rs_stream_desc> streams;
    std::vector<SliceInfo> slices;   // one per stream
    std::vector<uint32_t> stream_K;
    // pinned copy of the device stream table
    DevStream *table_host = nullptr;
    size_t table_cap = 0;
    bool table_dirty = true;
    void *table_ws = nullptr;      // workspace the table's pointers refer to
    uint64_t table_bal = 0;        // balanced unit count the table was built for (0: none)
    void *table_in_ws = nullptr;   // workspace holding the current table (private workspaces)
    cudaEvent_t upload_done = nullptr;
    bool upload_pending = false;
    // graph
    cudaGraphExec_t graph = nullptr;
    // device facts
    int n_sm = 0;
    size_t smem_max = 0;   // largest dynamic shared memory a CTA may opt in to
    // per-launch timing ring
    std::vector<cudaEvent_t> tev;   // 2 events per slot
    uint32_t t_cap = 0, t_count = 0;
    // stream table and plan for rs_run_noalloc, part of the pipeline object so that call
    // needs no allocation of its own
    NoallocTable noalloc_table;
    FixedPlan noalloc_plan;
    // launch shape of the last prepared launch (reported by rs_get_stats)
    uint32_t last_grid = 0, last_block = 0, last_smem = 0, last_bps = 0, last_cp = 0;
    // the automatic processors-per-CTA choice, for the kernel and per-processor bytes
    // it was made for
    const void *auto_key_fn = nullptr;
    uint32_t auto_key_bytes = 0, auto_wpb = 0;
};

static void timing_free(rs_pipeline *p)
{
    for (cudaEvent_t e : p->tev)
        if (e) cudaEventDestroy(e);
    p->tev.clear();
    p->t_cap = p->t_count = 0;
}

static uint32_t host_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

static bool is_pow2(uint32_t x) { return x && !(x & (x - 1)); }

static uint32_t max_fanout_of(const rs_stage_desc *st, uint32_t n)
{
    uint32_t k = 1;
    for (uint32_t i = 1; i < n; ++i)
        if (st[i].kind == RS_EXPAND && st[i].max_fanout > k) k = st[i].max_fanout;
    return k;
}

// the stage whose output stage i reads (0 = the enumeration)
static uint32_t stage_input(const rs_stage_desc *st, uint32_t i) { return st[i].input ? st[i].input : i - 1; }

static bool is_element_stage(uint32_t kind) { return kind == RS_FILTER || kind == RS_MAP || kind == RS_EXPAND; }

// segment slots per element of an emit sink: the product of the element stages' maximum
// fan-outs (at most 8^4)
static uint32_t fanout_product(const rs_stage_desc *st, uint32_t n)
{
    uint32_t f = 1;
    for (uint32_t i = 1; i + 1 < n; ++i) f *= st[i].max_fanout ? st[i].max_fanout : 1u;
    return f;
}

static bool is_emit(const rs_pipeline *p) { return p->stages[p->n_stages - 1].kind == RS_EMIT; }

// aggregate / emit leaves of the stage list
static uint32_t n_leaves(const rs_stage_desc *st, uint32_t n)
{
    uint32_t k = 0;
    for (uint32_t i = 1; i < n; ++i) k += (st[i].kind == RS_AGGREGATE || st[i].kind == RS_EMIT) ? 1u : 0u;
    return k;
}

// Topology and per-edge boundary modes as the kernels take them.  `strategy` is the
// resolved pipeline strategy (RS_BOUNDARY_DEFAULT edges follow it).  mix: the pipeline
// runs on the per-edge kernel (a tree, or any mode set per edge).
struct Topo {
    bool mix;
    uint32_t n_sinks;
    uint8_t emode[RS_MAX_STAGES], up[RS_MAX_STAGES], kids[RS_MAX_STAGES], sink_of[RS_MAX_STAGES];
};

static rs_status make_topo(const rs_stage_desc *st, uint32_t n, uint32_t modes, int strategy, Topo *t)
{
    memset(t, 0, sizeof *t);
    if (modes & 3u) return RS_ERR_INVALID;                     // the enumeration has no input edge
    if (n < RS_MAX_STAGES && (modes >> (2 * n)) != 0) return RS_ERR_INVALID;   // beyond the last stage
    bool linear = true;
    for (uint32_t i = 1; i < n; ++i) linear = linear && stage_input(st, i) == i - 1;
    t->mix = !linear || modes != 0;
    for (uint32_t i = 0; i < RS_MAX_STAGES; ++i) t->sink_of[i] = 0xFF;
    for (uint32_t c = 1; c < n; ++c) {
        const uint32_t u = stage_input(st, c);
        t->up[c] = (uint8_t)u;
        t->kids[u] |= (uint8_t)(1u << c);
        if (st[c].kind == RS_AGGREGATE || st[c].kind == RS_EMIT) t->sink_of[c] = (uint8_t)t->n_sinks++;
        uint32_t m = (modes >> (2 * c)) & 3u;
        if (m == RS_BOUNDARY_DEFAULT) m = strategy == RS_STRATEGY_TAG ? RS_BOUNDARY_TAG : RS_BOUNDARY_SIGNAL;
        t->emode[c] = (uint8_t)(m == RS_BOUNDARY_TAG ? EM_TAG : m == RS_BOUNDARY_LANE ? EM_LANE : EM_SIG);
        if (m == RS_BOUNDARY_LANE && st[c].kind == RS_EXPAND) return RS_ERR_INVALID;   // fan-out 1 only
    }
    // tags never turn back into signals: every reader of a tagged edge's consumer is tagged
    for (uint32_t c = 2; c < n; ++c)
        if (t->emode[t->up[c]] == EM_TAG && t->up[c] != 0 && t->emode[c] != EM_TAG) return RS_ERR_INVALID;
    return RS_OK;
}

static void set_topo(KParams &P, const Topo &t)
{
    P.mix = t.mix;
    P.n_sinks = t.n_sinks;
    memcpy(P.emode, t.emode, sizeof P.emode);
    memcpy(P.up, t.up, sizeof P.up);
    memcpy(P.kids, t.kids, sizeof P.kids);
    memcpy(P.sink_of, t.sink_of, sizeof P.sink_of);
}

static rs_status fill_defaults(rs_pipeline_opts *o, uint32_t fan)
{
    if (o->ensemble_width == 0) o->ensemble_width = 4 * RS_W;
    if (o->queue_capacity == 0) {
        uint32_t c = 64;
        while (c < o->ensemble_width * (fan + 1)) c <<= 1;
        o->queue_capacity = c;
    }
    if (o->signal_capacity == 0) {
        // a node that selects contexts per lane consumes the signals of a whole ensemble at
        // once: with short regions that is many signals
        bool lane = false;
        for (int c = 1; c < RS_MAX_STAGES; ++c) lane = lane || ((o->boundary_modes >> (2 * c)) & 3u) == RS_BOUNDARY_LANE;
        o->signal_capacity = lane ? 256 : 32;
    }
    if (o->tile_elements == 0) o->tile_elements = o->ensemble_width < 128 ? o->ensemble_width : 128;
    // tiles_in_flight 0: the tag strategy reads elements directly (no staging tiles);
    // the signal strategy stages 4 tiles
    if (o->tiles_in_flight == 0 && o->strategy != RS_STRATEGY_TAG) o->tiles_in_flight = 4;
    // region_cost 0 stays 0: resolved per strategy when units are planned
    if (o->device_budget == 0) o->device_budget = 1ull << 22;
    return RS_OK;
}

// log2 x when x is a power of two, else RS_NOT_POW2 (divisions by x become shifts)
static uint32_t log2_if_pow2(uint32_t x)
{
    if (x == 0 || (x & (x - 1)) != 0) return RS_NOT_POW2;
    uint32_t k = 0;
    while ((1u << k) != x) ++k;
    return k;
}

static rs_status check_opts(const rs_pipeline_opts *o, uint32_t fan)
{
    const uint32_t W = o->ensemble_width;
    if (W != RS_W && W != 2 * RS_W && W != 4 * RS_W && W != 8 * RS_W) return RS_ERR_INVALID;
    if (!is_pow2(o->queue_capacity) || o->queue_capacity < W * (fan + 1) || o->queue_capacity > 4096)
        return RS_ERR_INVALID;
    if (!is_pow2(o->signal_capacity) || o->signal_capacity < 4 || o->signal_capacity > 1024)
        return RS_ERR_INVALID;
    if (o->strategy > RS_STRATEGY_AUTO) return RS_ERR_INVALID;
    if (o->regions_per_unit > RS_TAG_MAX_K) return RS_ERR_INVALID;
    const uint32_t Wt = W < 128 ? W : 128;   // signal-strategy tiles hold at least one ensemble
    if (!is_pow2(o->tile_elements) || o->tile_elements < Wt || o->tile_elements > 4096) return RS_ERR_INVALID;
    if (o->tiles_in_flight != 0 && o->tiles_in_flight != 2 && o->tiles_in_flight != 4) return RS_ERR_INVALID;
    if (o->warps_per_block > 8) return RS_ERR_INVALID;   // 0: chosen per launch
    if (o->region_cost != 0 && (!is_pow2(o->region_cost) || o->region_cost > 256)) return RS_ERR_INVALID;
    if (o->flags & ~(RS_FLAG_UNBALANCED_UNITS | RS_FLAG_PRIVATE_WORKSPACE)) return RS_ERR_INVALID;
    return RS_OK;
}

// A linear pipeline (every stage reads the one before it) or a tree: stage 1 reads the
// enumeration, every later stage an earlier element stage; the leaves are exactly the
// sinks (at most RS_MAX_SINKS aggregates, or one emit sink ending a linear pipeline).
static rs_status check_stages(const rs_stage_desc *st, uint32_t n)
{
    if (!st || n < 2 || n > RS_MAX_STAGES) return RS_ERR_INVALID;
    if (st[0].kind != RS_ENUM_HASH && st[0].kind != RS_ENUM_LOAD) return RS_ERR_INVALID;
    bool linear = true;
    uint32_t leaves = 0;
    for (uint32_t i = 1; i < n; ++i) {
        const uint32_t u = stage_input(st, i);
        if (i == 1 ? u != 0 : (u < 1 || u >= i || !is_element_stage(st[u].kind))) return RS_ERR_INVALID;
        linear = linear && u == i - 1;
        bool read = false;
        for (uint32_t c = i + 1; c < n; ++c) read = read || stage_input(st, c) == i;
        const bool sink = st[i].kind == RS_AGGREGATE || st[i].kind == RS_EMIT;
        if (read == sink) return RS_ERR_INVALID;   // sinks are exactly the leaves
        leaves += sink ? 1u : 0u;
    }
    if (leaves > RS_MAX_SINKS) return RS_ERR_INVALID;
    for (uint32_t i = 1; i < n; ++i)
        if (st[i].kind == RS_EMIT && (!linear || i != n - 1)) return RS_ERR_INVALID;
    for (uint32_t i = 1; i < n; ++i) {
        const rs_stage_desc &s = st[i];
        if (s.kind == RS_AGGREGATE || s.kind == RS_EMIT) continue;
        switch (s.kind) {
        case RS_FILTER:
            if (s.max_fanout != 1) return RS_ERR_INVALID;
            if (s.op == RS_OP_MOD_EQ) {
                if (s.params[0] == 0) return RS_ERR_INVALID;
            } else if (s.op != RS_OP_HASH_CTX_LT && s.op != RS_OP_WEIGHT_LT) {
                return RS_ERR_INVALID;
            }
            break;
        case RS_MAP:
            if (s.max_fanout != 1 || s.op != RS_OP_MUL_ADD) return RS_ERR_INVALID;
            break;
        case RS_EXPAND:
            if (s.op != RS_OP_HASH_FANOUT || s.max_fanout < 1 || s.max_fanout > 8) return RS_ERR_INVALID;
            break;
        default:
            return RS_ERR_INVALID;
        }
    }
    return RS_OK;
}

static DevStage to_dev(const rs_stage_desc &s)
{
    DevStage d;
    memset(&d, 0, sizeof d);
    d.fanout = s.max_fanout ? s.max_fanout : 1;
    d.p0 = s.params[0];
    d.p1 = s.params[1];
    d.c0 = host_fmix32(s.params[0] ^ RS_GOLD);
    d.c0s = d.c0 ^ (d.c0 >> 16);
    switch (s.kind) {
    case RS_ENUM_HASH: d.op = D_ENUM_HASH; break;
    case RS_ENUM_LOAD: d.op = D_ENUM_LOAD; break;
    case RS_AGGREGATE: d.op = D_AGG; break;
    case RS_EMIT: d.op = D_EMIT; break;
    case RS_MAP: d.op = D_MAP_MULADD; break;
    case RS_EXPAND: d.op = D_EXPAND; break;
    case RS_FILTER:
        if (s.op == RS_OP_MOD_EQ) {
            if (is_pow2(s.params[0])) {
                d.op = D_FILT_MASK;
                d.p0 = s.params[0] - 1u;
                // x mod m == c with c >= m can never hold; keep the comparison exact
                d.p1 = s.params[1] < s.params[0] ? s.params[1] : 0xFFFFFFFFu;
            } else {
                d.op = D_FILT_MOD;
            }
        } else if (s.op == RS_OP_HASH_CTX_LT) {
            d.op = D_FILT_HASH_CTX;
        } else {
            d.op = D_FILT_WEIGHT;
        }
        break;
    }
    return d;
}

extern "C" {

const char *rs_status_string(rs_status s)
{
    switch (s) {
    case RS_OK: return "ok";
    case RS_ERR_INVALID: return "invalid argument";
    case RS_ERR_NOMEM: return "host out of memory";
    case RS_ERR_CUDA: return "CUDA error";
    case RS_ERR_NOT_READY: return "not ready";
    case RS_ERR_STALL: return "device iteration budget exhausted";
    case RS_ERR_CAPACITY: return "capacity exceeded";
    case RS_ERR_STATE: return "call out of order";
    case RS_ERR_DEVICE_INPUT: return "device found inconsistent input";
    }
    return "unknown status";
}

rs_status rs_calibrate_cascade(const uint32_t *elements, uint64_t n, uint32_t ctx, const uint32_t *salts,
                               const uint32_t *thetas, uint64_t *out, rs_cuda_stream stream)
{
    if (!out || !salts || !thetas || (n > 0 && !elements)) return RS_ERR_INVALID;
    if (((uintptr_t)out & 7u) != 0) return RS_ERR_INVALID;
    int dev = 0, n_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(out, 0, 2 * sizeof(uint64_t), (cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e);
    if (n == 0) return RS_OK;
    uint32_t c0[3];
    for (int i = 0; i < 3; ++i) c0[i] = host_fmix32(salts[i] ^ RS_GOLD);
    const int le = rs_launch_calib(elements, (unsigned long long)n, ctx, c0, thetas, (unsigned long long *)out, n_sm,
                                   (void *)stream);
    if (le != 0) return cuda_fail((cudaError_t)le);
    return RS_OK;
}

int rs_last_cuda_error(void) { return g_last_cuda; }

uint32_t rs_version(void) { return RS_VERSION; }

uint32_t rs_struct_sizes(uint64_t *sizes, uint32_t max)
{
    const uint64_t z[] = {sizeof(rs_stage_desc), sizeof(rs_pipeline_opts), sizeof(rs_stream_desc),
                          sizeof(rs_region_results), sizeof(rs_stats), sizeof(rs_request), sizeof(rs_server_stats)};
    const uint32_t n = (uint32_t)(sizeof z / sizeof z[0]);
    for (uint32_t i = 0; i < n && i < max && sizes; ++i) sizes[i] = z[i];
    return n;
}

rs_status rs_default_opts(rs_pipeline_opts *o)
{
    if (!o) return RS_ERR_INVALID;
    memset(o, 0, sizeof *o);
    o->strategy = RS_STRATEGY_TAG;
    fill_defaults(o, 1);
    return RS_OK;
}

rs_status rs_pipeline_create(const rs_stage_desc *stages, uint32_t n_stages, const rs_pipeline_opts *opts,
                             rs_pipeline **out)
{
    if (!out) return RS_ERR_INVALID;
    *out = nullptr;
    rs_status st = check_stages(stages, n_stages);
    if (st != RS_OK) return st;
    rs_pipeline_opts o;
    if (opts) o = *opts; else { memset(&o, 0, sizeof o); o.strategy = RS_STRATEGY_TAG; }
    uint32_t fan = max_fanout_of(stages, n_stages);
    fill_defaults(&o, fan);
    st = check_opts(&o, fan);
    if (st != RS_OK) return st;
    Topo topo;   // boundary modes against the strategy (RS_STRATEGY_AUTO is checked per run)
    if (make_topo(stages, n_stages, o.boundary_modes, o.strategy == RS_STRATEGY_TAG ? RS_STRATEGY_TAG : RS_STRATEGY_SIGNAL,
                  &topo) != RS_OK)
        return RS_ERR_INVALID;
    rs_pipeline *p = new (std::nothrow) rs_pipeline();
    if (!p) return RS_ERR_NOMEM;
    memcpy(p->stages, stages, n_stages * sizeof(rs_stage_desc));
    p->n_stages = n_stages;
    p->opts = o;
    *out = p;
    return RS_OK;
}

rs_status rs_pipeline_destroy(rs_pipeline *p)
{
    if (!p) return RS_ERR_INVALID;
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->upload_done) {
        if (p->upload_pending) cudaEventSynchronize(p->upload_done);
        cudaEventDestroy(p->upload_done);
    }
    if (p->table_host) cudaFreeHost(p->table_host);
    timing_free(p);
    delete p;
    return RS_OK;
}

rs_status rs_pipeline_set_opts(rs_pipeline *p, const rs_pipeline_opts *opts)
{
    if (!p || !opts) return RS_ERR_INVALID;
    rs_pipeline_opts o = *opts;
    uint32_t fan = max_fanout_of(p->stages, p->n_stages);
    fill_defaults(&o, fan);
    rs_status st = check_opts(&o, fan);
    if (st != RS_OK) return st;
    Topo topo;
    if (make_topo(p->stages, p->n_stages, o.boundary_modes,
                  o.strategy == RS_STRATEGY_TAG ? RS_STRATEGY_TAG : RS_STRATEGY_SIGNAL, &topo) != RS_OK)
        return RS_ERR_INVALID;
    p->opts = o;
    p->table_dirty = true;   // regions_per_unit may change the unit split
    return RS_OK;
}

rs_status rs_pipeline_get_opts(const rs_pipeline *p, rs_pipeline_opts *opts)
{
    if (!p || !opts) return RS_ERR_INVALID;
    *opts = p->opts;
    return RS_OK;
}

rs_status rs_stream_submit(rs_pipeline *p, const rs_stream_desc *s, uint64_t *stream_id)
{
    if (!p || !s) return RS_ERR_INVALID;
    if (p->graph) return RS_ERR_STATE;
    if (s->n_regions >= (1ull << 32)) return RS_ERR_CAPACITY;
    if (s->n_regions > 0) {
        if (!s->region_len && !s->region_offsets) return RS_ERR_INVALID;
        if (p->stages[0].kind == RS_ENUM_LOAD && (!s->elements || s->n_elements == 0)) return RS_ERR_INVALID;
        if (s->n_elements >= (1ull << 32) - 4096) return RS_ERR_CAPACITY;   // positions stay 32-bit
        if (is_emit(p) && (!s->region_offsets || !s->out_count || !s->out_values || s->out_values_len == 0))
            return RS_ERR_INVALID;   // the emit sink's segments follow the CSR offsets
        // a tree's second leaf fills the same outputs as the first
        if (n_leaves(p->stages, p->n_stages) > 1 &&
            ((!s->out_count != !s->out2_count) || (!s->out_sum != !s->out2_sum) || (!s->out_min != !s->out2_min)))
            return RS_ERR_INVALID;
        for (uint32_t i = 1; i + 1 < p->n_stages; ++i)
            if (p->stages[i].kind == RS_FILTER && p->stages[i].op == RS_OP_HASH_CTX_LT) {
                // ctx may be NULL (t_r = 0)
            }
    }
    try {
        p->streams.push_back(*s);
        p->slices.push_back(SliceInfo());
    } catch (...) {
        if (p->streams.size() > p->slices.size()) p->streams.pop_back();
        return RS_ERR_NOMEM;
    }
    p->table_dirty = true;
    if (stream_id) *stream_id = p->streams.size() - 1;
    return RS_OK;
}

rs_status rs_clear_streams(rs_pipeline *p)
{
    if (!p) return RS_ERR_INVALID;
    if (p->graph) return RS_ERR_STATE;
    p->streams.clear();
    p->slices.clear();
    p->table_dirty = true;
    return RS_OK;
}

}  // extern "C"

static rs_status state_need(const rs_pipeline *p, const rs_stream_desc *s, uint64_t *bytes, uint64_t *n_units);

extern "C" {

rs_status rs_stream_state_size(const rs_pipeline *p, const rs_stream_desc *s, uint64_t *state_bytes,
                               uint64_t *n_units)
{
    if (!p || !s) return RS_ERR_INVALID;
    uint64_t b = 0, u = 0;
    rs_status st = state_need(p, s, &b, &u);
    if (st != RS_OK) return st;
    if (state_bytes) *state_bytes = b;
    if (n_units) *n_units = u;
    return RS_OK;
}

rs_status rs_stream_submit_slice(rs_pipeline *p, const rs_stream_desc *s, void *state, uint64_t state_bytes,
                                 uint64_t unit_begin, uint64_t unit_count, uint64_t *stream_id)
{
    if (!p || !s) return RS_ERR_INVALID;
    if (state && ((uintptr_t)state & 255) != 0) return RS_ERR_INVALID;
    uint64_t id = 0;
    rs_status st = rs_stream_submit(p, s, &id);
    if (st != RS_OK) return st;
    SliceInfo &si = p->slices.back();
    si.on = true;
    si.state = state;
    si.state_bytes = state_bytes;
    si.begin = unit_begin;
    si.count = unit_count;
    if (stream_id) *stream_id = id;
    return RS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------

// whole-parent units (hashed enumeration): about 2048 elements per unit for the signal
// strategy (its per-parent shared memory caps K at RS_MAX_K), about 8192 for the tag
// strategy
static uint32_t choose_K(const rs_pipeline *p, const rs_pipeline_opts &o, const rs_stream_desc &s, int strategy)
{
    if (o.regions_per_unit) return o.regions_per_unit;
    if (s.n_regions == 0) return 1;
    uint64_t tot = s.total_elements_hint;
    if (!tot && p->stages[0].kind == RS_ENUM_LOAD) tot = s.n_elements;
    double mean = tot ? (double)tot / (double)s.n_regions : 32.0;
    const bool tag = strategy == RS_STRATEGY_TAG;
    double want = (tag ? RS_TAG_UNIT_ELEMS : 2048.0) / (mean > 1e-9 ? mean : 1e-9);
    const uint32_t kmax = tag ? RS_TAG_MAX_K : RS_MAX_K;
    uint32_t K = 1;
    while (K * 2 <= want && K * 2 <= kmax) K *= 2;
    return K;
}

// merge-path unit shape: c steps per parent, D steps per unit
static void merge_shape(const rs_pipeline_opts &o, int strategy, uint32_t *c, uint32_t *D, uint32_t *K)
{
    if (strategy == RS_STRATEGY_TAG) {
        // a parent costs region_cost steps (default 1); a unit is region_cost x
        // regions_per_unit steps (default 4096)
        const uint32_t cc = o.region_cost ? o.region_cost : 1u;
        uint32_t k = o.regions_per_unit;
        if (!k) k = RS_TAG_UNIT_STEPS / cc ? RS_TAG_UNIT_STEPS / cc : 1u;
        *c = cc;
        *D = cc * k;
        *K = k;
    } else {
        const uint32_t kp = o.regions_per_unit ? o.regions_per_unit : 128u;
        *c = o.region_cost ? o.region_cost : RS_STEP_REGION;
        *D = *c * kp;      // a unit owns <= kp parents and holds <= D elements
        *K = kp + 1;       // plus the parent continued from an earlier unit
    }
}

// Parents per planner tile: with fewer than 2^20 regions over the loaded streams, tiles
// of 128 parents (one per lane and round), so that the planner has enough warps (a
// mean-4096 stream of 2^26 elements has only 16 K regions) to write its unit records.
static uint32_t plan_tile_parents(const rs_pipeline *p)
{
    uint64_t regions = 0;
    if (p->stages[0].kind == RS_ENUM_LOAD)
        for (const auto &s : p->streams) regions += s.n_regions;
    return regions < (1ull << 20) ? RS_PLAN_TILE_SMALL : RS_PLAN_TILE;
}

// the work decomposition of one stream
static void plan_stream(const rs_pipeline *p, const rs_pipeline_opts &o, int strategy, const rs_stream_desc &s,
                        StreamPlan &q, bool allow_usum = false, uint64_t bal = 0)
{
    memset(&q, 0, sizeof q);
    const double mean = s.n_regions ? (double)s.n_elements / (double)s.n_regions : 0.0;
    if (allow_usum && strategy == RS_STRATEGY_TAG && p->stages[0].kind == RS_ENUM_LOAD && !s.region_offsets &&
        s.n_regions > 0 && mean < RS_USUM_MEAN) {
        // short regions: units of K whole parents (the sum of K short lengths varies
        // little, so they stay balanced) whose offsets come from per-unit length sums, with
        // K the parents that fill the unit shape's D steps at this mean
        uint32_t c, D, K0;
        merge_shape(o, strategy, &c, &D, &K0);
        const double want = (double)D / (1.0 + (mean > 1.0 ? mean : 1.0));
        uint32_t K = 32;
        while ((double)K * 2 <= want && K * 2 <= RS_TAG_MAX_K) K *= 2;
        // balanced units: bal units in all (at most as many as the shape gives)
        if (bal && bal < (s.n_regions + K - 1) / K) K = (uint32_t)((s.n_regions + bal - 1) / bal);
        q.mode = UNIT_REGIONS;
        q.K = K;
        q.n_units = (uint32_t)((s.n_regions + K - 1) / K);
        q.usum = true;
        return;
    }
    if (p->stages[0].kind == RS_ENUM_LOAD) {
        q.mode = UNIT_MERGE;
        merge_shape(o, strategy, &q.c, &q.D, &q.K);
        uint64_t steps = (uint64_t)q.c * s.n_regions + s.n_elements;
        // balanced units: D grows so that the stream has bal units (never more than the
        // shape gives: the workspace was sized for those)
        if (bal && bal < (steps + q.D - 1) / q.D && (steps + bal - 1) / bal < (1ull << 32))
            q.D = (uint32_t)((steps + bal - 1) / bal);
        q.n_units = s.n_regions ? (uint32_t)((steps + q.D - 1) / q.D) : 0u;
        const uint32_t tile = plan_tile_parents(p);
        q.plan_tiles = (uint32_t)((s.n_regions + tile - 1) / tile);
    } else {
        q.mode = UNIT_REGIONS;
        q.K = choose_K(p, o, s, strategy);
        q.n_units = (uint32_t)((s.n_regions + q.K - 1) / q.K);
    }
}

// bytes of a stream's per-run scratch: merge slots (signal strategy only), unit count,
// planner look-back words; then its unit records
static size_t stream_zeroed_bytes(const StreamPlan &q, int strategy, uint32_t nsinks)
{
    if (q.mode != UNIT_MERGE) return 0;
    size_t b = 0;
    // one array of slots per leaf (a tree's second leaf merges through its own)
    if (strategy != RS_STRATEGY_TAG) b += (size_t)q.n_units * sizeof(Slot) * (nsinks > 1 ? nsinks : 1u);
    return b;
}

struct Plan {
    uint64_t total_units, plan_tiles;
    uint32_t Kmax;
    size_t hdr_bytes, zero_end, table_off, table_bytes, total;
    std::vector<StreamPlan> sp;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

// Lay out the workspace for a list of stream plans:
// [header | per stream: slots, unit count, planner look-back words | per stream: unit
//  records | stream table].  Everything before zero_end is cleared by every run.
template <class SP>
static void layout_plan(SP *sp, size_t ns, int strategy, uint32_t nsinks, uint64_t *total_units,
                        uint64_t *plan_tiles, uint32_t *Kmax, size_t *zero_end, size_t *table_off, size_t *total)
{
    *total_units = *plan_tiles = 0;
    *Kmax = 1;
    size_t off = align256(sizeof(WsHeader));
    for (size_t i = 0; i < ns; ++i) {
        StreamPlan &q = sp[i];
        if (q.K > *Kmax) *Kmax = q.K;
        *total_units += q.slice_n;
        *plan_tiles += q.run_tiles;
        if (q.usum) {   // per-unit length sums and group prefixes (zeroed: atomics)
            q.usum_off = off;
            off = align256(off + (size_t)q.n_units * 4);
            q.grp_off = off;
            off = align256(off + (size_t)((q.n_units + 31) / 32) * 4);
        }
        if (q.mode == UNIT_MERGE && !q.sliced) {   // a sliced stream's scratch is its state
            q.slots_off = off;
            off = align256(off + stream_zeroed_bytes(q, strategy, nsinks));
            q.ucount_off = off;
            off = align256(off + 4);
            q.planlb_off = off;
            off = align256(off + (size_t)q.plan_tiles * 8);
        }
    }
    *zero_end = off;
    for (size_t i = 0; i < ns; ++i) {
        StreamPlan &q = sp[i];
        if (q.mode == UNIT_MERGE && !q.sliced) {
            q.rec_off = off;
            off = align256(off + ((size_t)q.n_units + 1) * sizeof(UnitRec));
        }
    }
    *table_off = off;
    *total = off + align256(ns * sizeof(DevStream));
}

// A sliced stream's state: merge slots, unit count and planner words (cleared when the
// stream is planned), then its unit records.
static void state_layout(StreamPlan &q, int strategy, uint32_t nsinks)
{
    q.st_zero = q.st_total = 0;
    if (q.mode != UNIT_MERGE) return;
    size_t off = 0;
    q.slots_off = off;
    off = align256(off + stream_zeroed_bytes(q, strategy, nsinks));
    q.ucount_off = off;
    off = align256(off + 4);
    q.planlb_off = off;
    off = align256(off + (size_t)q.plan_tiles * 8);
    q.st_zero = off;
    q.rec_off = off;
    off = align256(off + ((size_t)q.n_units + 1) * sizeof(UnitRec));
    q.st_total = off;
}

// this run's share of a stream (all of it unless it was submitted for a sliced run)
static void apply_slice(const SliceInfo &si, StreamPlan &q, int strategy, uint32_t nsinks)
{
    q.full_units = q.n_units;
    q.sliced = si.on;
    q.slice_lo = 0;
    q.slice_n = q.n_units;
    q.plan_now = true;
    q.run_tiles = q.plan_tiles;
    if (!si.on) return;
    const uint64_t b = si.begin < q.n_units ? si.begin : q.n_units;
    const uint64_t n = si.count < q.n_units - b ? si.count : q.n_units - b;
    q.slice_lo = (uint32_t)b;
    q.slice_n = (uint32_t)n;
    q.plan_now = b == 0;
    q.run_tiles = q.plan_now ? q.plan_tiles : 0u;
    state_layout(q, strategy, nsinks);
}

static Plan make_plan(const rs_pipeline *p, int strategy, const rs_pipeline_opts &o, uint64_t bal = 0)
{
    Plan pl;
    pl.hdr_bytes = align256(sizeof(WsHeader));
    pl.sp.resize(p->streams.size());
    const uint32_t nsinks = n_leaves(p->stages, p->n_stages);
    for (size_t i = 0; i < p->streams.size(); ++i) {
        plan_stream(p, o, strategy, p->streams[i], pl.sp[i], !p->slices[i].on, bal);
        apply_slice(p->slices[i], pl.sp[i], strategy, nsinks);
    }
    layout_plan(pl.sp.data(), pl.sp.size(), strategy, n_leaves(p->stages, p->n_stages), &pl.total_units,
                &pl.plan_tiles, &pl.Kmax, &pl.zero_end, &pl.table_off, &pl.total);
    pl.table_bytes = pl.total - pl.table_off;
    return pl;
}

static int run_strategy(const rs_pipeline *p, Topo *t);

// the state a sliced run of stream s needs under the current options, and its units
static rs_status state_need(const rs_pipeline *p, const rs_stream_desc *s, uint64_t *bytes, uint64_t *n_units)
{
    Topo topo;
    const int strategy = run_strategy(p, &topo);
    if (strategy < 0) return RS_ERR_INVALID;
    StreamPlan q;
    plan_stream(p, p->opts, strategy, *s, q);
    SliceInfo si;
    si.on = true;
    apply_slice(si, q, strategy, n_leaves(p->stages, p->n_stages));
    *bytes = q.st_total;
    *n_units = q.full_units;
    return RS_OK;
}

// Per-processor shared memory of the tag kernel: counters, window marks (W words, hashed
// enumeration only: with loaded elements node 1 marks in the staging slot it has just
// read), node 1's staging ring of four element windows (loaded enumeration only),
// the rings of edges 1..n-3 (8-byte slots of {value, region tag}; edge n-2 too when node
// n-2 is an expansion), and the parent records
// (PR entries each of {region id, operand}, start offset, and parent id for hashed
// enumeration).  PR >= W + 64 cpl covers every record node 1 can still need: the parents
// of one window, plus one chunk of 32 cpl loaded beyond it.
static SmemLayout make_tag_layout(const rs_pipeline *p, uint32_t cpl)
{
    const rs_pipeline_opts &o = p->opts;
    const uint32_t W = o.ensemble_width;
    SmemLayout L;
    memset(&L, 0, sizeof L);
    size_t off = 0;
    L.o_prof = (uint32_t)off;
#ifdef RS_PROFILE
    off += 8 * RS_PROF_SLOTS;
#endif
    L.o_cnt = (uint32_t)off;      // 32-bit node statistics
    off += 4 * 4 * RS_MAX_STAGES;
    off = align_up(off, 16);
    L.o_pend = (uint32_t)off;     // the next unit's description (7 words), at byte 32 the
    off += 72;                    // 8-byte scratch slot of the ring stores, at byte 48 the
                                  // aggregate's pending fold (3 words, the sum at byte 64)
    off = align_up(off, 16);
    L.o_scr = (uint32_t)off;      // window marks, hashed enumeration only (loaded
    off += p->stages[0].kind == RS_ENUM_LOAD ? 0 : (size_t)4 * W;   // elements: a staging slot)
    off = align_up(off, 16);
    L.o_tiles = (uint32_t)off;    // node 1's staged element windows (4 x W)
    off += p->stages[0].kind == RS_ENUM_LOAD ? (size_t)4 * W * 4 : 0;
    // rings of edges 1..n-2, less the edge into the aggregate when its producer is not an
    // expansion: that node folds its kept items into the aggregate directly
    const uint32_t ns = p->n_stages;
    const bool fused = ns >= 3 && p->stages[ns - 2].kind != RS_EXPAND;
    const size_t rings = ns - 2 - (fused ? 1u : 0u);
    off = align_up(off, 16);
    L.o_qv = (uint32_t)off;       // ring slots {value, region id}, 8 bytes each
    L.o_qt = L.o_qv;
    off += rings * o.queue_capacity * 8;
    uint32_t pr = 128;
    while (pr < W + 64 * cpl) pr <<= 1;
    L.pr = pr;
    L.o_nra = (uint32_t)off;      // {region, operand} (PR entries)
    off += (size_t)pr * 8;
    L.o_nst = (uint32_t)off;      // start offsets (PR entries)
    off += (size_t)pr * 4;
    L.o_npar = (uint32_t)off;     // parent ids, hashed enumeration only (PR entries)
    off += p->stages[0].kind == RS_ENUM_HASH ? (size_t)pr * 4 : 0;
    L.per_warp = (uint32_t)align_up(off, 128);
    return L;
}

// Parents per lane in the tag kernel's parent chunks: two when the loaded streams' regions
// average fewer than 7 elements (chunk loads then recur every window or two and each one
// carries twice the parents; measured faster up to a mean of 6, even from 8), else one.  Hashed streams give no element count: one.
static uint32_t tag_chunk_cpl(const rs_pipeline *p)
{
    if (p->stages[0].kind != RS_ENUM_LOAD) return 1;
    uint64_t el = 0, regions = 0;
    for (const auto &s : p->streams) {
        el += s.n_elements;
        regions += s.n_regions;
    }
    return regions > 0 && el < 7 * regions ? 2u : 1u;
}

// every merge-path stream of a plan has a power-of-two D (the planner then divides by
// shifts; every tag-strategy unit shape has one)
template <class PL>
static uint32_t plan_pow2(const PL &pl, size_t ns)
{
    for (size_t i = 0; i < ns; ++i)
        if (pl.sp[i].mode == UNIT_MERGE && log2_if_pow2(pl.sp[i].D) == RS_NOT_POW2) return 0;
    return 1;
}

static SmemLayout make_layout(const rs_pipeline *p, int strategy, uint32_t Kmax, bool any_load, bool need_ctx,
                              bool need_par, bool want_min, const Topo &topo)
{
    const rs_pipeline_opts &o = p->opts;
    SmemLayout L;
    memset(&L, 0, sizeof L);
    size_t off = 0;
    L.o_prof = (uint32_t)off;
#ifdef RS_PROFILE
    off += 8 * RS_PROF_SLOTS;
#endif
    L.o_cnt = (uint32_t)off;
    off += 8 * 4 * RS_MAX_STAGES;
    L.o_pend = (uint32_t)off;
    off += 128;   // the prefetched next unit's descriptor (a Pending record)
    L.o_mmeta = (uint32_t)off;
    off += 16;
    L.o_mbar = (uint32_t)off;
    off += any_load ? 8 * o.tiles_in_flight : 0;
    off = align_up(off, 16);
    L.o_scr = (uint32_t)off;
    off += (size_t)4 * (o.ensemble_width > 32 ? o.ensemble_width : 32);   // window marks (tag strategy)
    off = align_up(off, 128);
    L.o_tiles = (uint32_t)off;
    off += any_load ? (size_t)o.tiles_in_flight * o.tile_elements * 4 : 0;
    // per-parent accumulators: every parent for the signal strategy; the tag strategy
    // updates the outputs directly and keeps only the two pieces a unit may share with
    // its neighbours (the continued first parent and a last parent running past it)
    const size_t nacc = strategy == RS_STRATEGY_TAG ? 2 : (size_t)Kmax;
    L.o_rs = (uint32_t)off;
    off += nacc * 8;
    for (int b = 0; b < 2; ++b) {
        // the unit-local offsets are built in place over the loaded lengths / offsets
        L.o_raw[b] = (uint32_t)off;
        L.o_moff[b] = (uint32_t)off;
        off += (size_t)(Kmax + 1) * 4;
        L.o_ctxb[b] = (uint32_t)off;
        off += need_ctx ? (size_t)Kmax * 4 : 0;
        L.o_parb[b] = (uint32_t)off;
        off += need_par ? (size_t)Kmax * 4 : 0;
    }
    L.o_rc = (uint32_t)off;
    off += nacc * 4;
    L.o_rm = (uint32_t)off;
    off += want_min ? nacc * 4 : 0;
    // a tree's second leaf: per-parent accumulators of its own
    L.o_rs2 = L.o_rs;
    L.o_rc2 = L.o_rc;
    L.o_rm2 = L.o_rm;
    if (topo.mix && topo.n_sinks > 1) {
        off = align_up(off, 8);
        L.o_rs2 = (uint32_t)off;
        off += nacc * 8;
        L.o_rc2 = (uint32_t)off;
        off += nacc * 4;
        L.o_rm2 = (uint32_t)off;
        off += want_min ? nacc * 4 : 0;
    }
    off = align_up(off, 16);
    // rings for edges 1..n-2 (edge 0 carries element positions, staged in the tiles)
    const uint32_t nr = p->n_stages - 2;
    // tag strategy: one 64-bit slot {value, tag} per item; signal strategy: 32-bit values
    L.o_qv = (uint32_t)off;
    off += (size_t)nr * o.queue_capacity * (strategy == RS_STRATEGY_TAG ? 8 : 4);
    L.o_qt = (uint32_t)off;
    // the per-edge kernel: a 16-bit parent tag per slot for the edges that carry tags
    off += topo.mix ? (size_t)nr * o.queue_capacity * 2 : 0;
    off = align_up(off, 16);
    // signal rings for edges 0..n-2
    L.o_sq = (uint32_t)off;
    off += strategy == RS_STRATEGY_SIGNAL ? (size_t)(p->n_stages - 1) * o.signal_capacity * 8 : 0;
    L.per_warp = (uint32_t)align_up(off, 128);
    return L;
}

static int resolve_strategy(const rs_pipeline *p)
{
    if (p->opts.strategy != RS_STRATEGY_AUTO) return (int)p->opts.strategy;
    // mean region length across the submitted streams; long regions favour signals
    uint64_t R = 0, N = 0;
    for (const auto &s : p->streams) {
        R += s.n_regions;
        uint64_t t = s.total_elements_hint;
        if (!t && p->stages[0].kind == RS_ENUM_LOAD) t = s.n_elements;
        N += t;
    }
    double mean = R ? (double)N / (double)R : 0.0;
    return mean >= 1024.0 ? RS_STRATEGY_SIGNAL : RS_STRATEGY_TAG;
}

// The strategy a run's kernels follow: the per-edge kernel (signal-strategy units and
// layout) for trees and per-edge boundary modes, else the resolved strategy; -1 when the
// modes are inconsistent for the resolved strategy.  *t gets the topology.
static int run_strategy(const rs_pipeline *p, Topo *t)
{
    const int strategy = resolve_strategy(p);
    if (make_topo(p->stages, p->n_stages, p->opts.boundary_modes, strategy, t) != RS_OK) return -1;
    return t->mix ? RS_STRATEGY_SIGNAL : strategy;
}

// Unit shapes (regions_per_unit, region_cost) rs_autotune tries for the tag strategy on
// merge-path streams.
static const uint32_t k_tag_shapes[][2] = {{4096, 1}, {8192, 1}, {16384, 1}, {2048, 1}, {1024, 4}, {256, 16},
                                            {2048, 4}, {4096, 2}};

// Workspace for either strategy with the current options and for every configuration
// rs_autotune may try, so one workspace serves them all.
static size_t workspace_need(const rs_pipeline *p)
{
    size_t need = 0;
    for (int strategy : {RS_STRATEGY_TAG, RS_STRATEGY_SIGNAL}) {
        const size_t t = make_plan(p, strategy, p->opts).total;
        if (t > need) need = t;
    }
    rs_pipeline_opts o = p->opts;
    for (const auto &sh : k_tag_shapes) {
        o.regions_per_unit = sh[0];
        o.region_cost = sh[1];
        const size_t t = make_plan(p, RS_STRATEGY_TAG, o).total;
        if (t > need) need = t;
    }
    o = p->opts;
    o.regions_per_unit = 0;
    for (int strategy : {RS_STRATEGY_TAG, RS_STRATEGY_SIGNAL}) {
        const size_t t = make_plan(p, strategy, o).total;
        if (t > need) need = t;
    }
    return need;
}

rs_status rs_run_workspace_bytes(const rs_pipeline *p, uint64_t *bytes)
{
    if (!p || !bytes) return RS_ERR_INVALID;
    Topo topo;
    const int strategy = run_strategy(p, &topo);
    if (strategy < 0) return RS_ERR_INVALID;
    *bytes = make_plan(p, strategy, p->opts).total;
    return RS_OK;
}

extern "C" rs_status rs_workspace_size(const rs_pipeline *p, uint64_t *bytes)
{
    if (!p || !bytes) return RS_ERR_INVALID;
    *bytes = workspace_need(p);
    return RS_OK;
}

// warps_per_block = 0: the processors per CTA (8, 4, 2 or 1) giving the most resident
// processors per SM for this kernel and per-processor shared memory (host-side
// occupancy queries only; remembered for the same kernel and size)
static rs_status auto_wpb(rs_pipeline *p, const KParams &P, uint32_t *out)
{
    const void *kf = rs_kernel_entry(P);
    if (p->auto_key_fn == kf && p->auto_key_bytes == P.L.per_warp) {
        *out = p->auto_wpb;
        return RS_OK;
    }
    uint32_t best_w = 0, best_res = 0;
    for (uint32_t cand = 8; cand >= 1; cand >>= 1) {
        if ((size_t)P.L.per_warp * cand > p->smem_max) continue;
        int bps = 0;
        int ce = rs_kernel_occupancy(P, (int)cand * 32, (size_t)P.L.per_warp * cand, &bps);
        if (ce != 0) return cuda_fail((cudaError_t)ce);
        if ((uint32_t)bps * cand > best_res) {
            best_res = (uint32_t)bps * cand;
            best_w = cand;
        }
    }
    if (best_w == 0) return RS_ERR_CAPACITY;
    p->auto_key_fn = kf;
    p->auto_key_bytes = P.L.per_warp;
    p->auto_wpb = best_w;
    *out = best_w;
    return RS_OK;
}

// The device stream table of a run: the streams' arrays, their unit split and this run's
// share of their units, and their scratch in the workspace wsd (a sliced stream's in its
// own state).
static void fill_table(const rs_pipeline *p, const StreamPlan *sp, size_t ns, unsigned char *wsd, DevStream *out)
{
    uint32_t base = 0, pbase = 0;
    for (size_t i = 0; i < ns; ++i) {
        const rs_stream_desc &s = p->streams[i];
        const StreamPlan &q = sp[i];
        DevStream &d = out[i];
        memset(&d, 0, sizeof d);
        d.parents = s.parents;
        d.len = s.region_len;
        d.offsets = s.region_offsets;
        d.elements = s.elements;
        d.ctx = s.ctx;
        d.out_count = s.out_count;
        d.out_sum = (unsigned long long *)s.out_sum;
        d.out_min = s.out_min;
        d.out_values = s.out_values;
        d.out_values_len = s.out_values_len;
        d.out2_count = s.out2_count;
        d.out2_sum = (unsigned long long *)s.out2_sum;
        d.out2_min = s.out2_min;
        d.n_elements = s.n_elements;
        d.R = (uint32_t)s.n_regions;
        d.K = q.K;
        d.n_units = q.slice_n;
        d.slice_lo = q.slice_lo;
        d.slot_units = q.full_units;
        d.finalize = q.slice_lo + q.slice_n >= q.full_units ? 1u : 0u;
        if (q.usum) {
            d.usum = (uint32_t *)(wsd + q.usum_off);
            d.usum_grp = (uint32_t *)(wsd + q.grp_off);
        }
        d.unit_base = base;
        // every stream's planner-tile base, planned or not, so that the tiles' bases never
        // decrease along the table (the planner finds a tile's stream by binary search: a
        // stream without tiles holds the base of the next one that has some)
        d.plan_base = pbase;
        d.tma_ok = s.elements && (((uintptr_t)s.elements & 15) == 0);
        d.mode = q.mode;
        if (q.mode == UNIT_MERGE) {
            unsigned char *b = q.sliced ? (unsigned char *)p->slices[i].state : wsd;
            d.rec = (UnitRec *)(b + q.rec_off);
            d.slots = (Slot *)(b + q.slots_off);
            d.u_count = (uint32_t *)(b + q.ucount_off);
            d.plan_lb = (unsigned long long *)(b + q.planlb_off);
            d.plan_tiles = q.run_tiles;
            d.plan_base = pbase;
            d.D = q.D;
            d.dsh = log2_if_pow2(q.D);
            d.c = q.c;
            pbase += q.run_tiles;
        }
        base += d.n_units;
    }
}

// some merge-path stream runs units in this run
static bool any_merge(const StreamPlan *sp, size_t ns)
{
    for (size_t i = 0; i < ns; ++i)
        if (sp[i].mode == UNIT_MERGE && sp[i].slice_n > 0) return true;
    return false;
}

// some stream runs fixed-parent units over lengths (their offsets are computed first)
static bool any_usum(const StreamPlan *sp, size_t ns, uint64_t *units)
{
    bool any = false;
    *units = 0;
    for (size_t i = 0; i < ns; ++i)
        if (sp[i].usum && sp[i].slice_n > 0) {
            any = true;
            *units += sp[i].n_units;
        }
    return any;
}

// every sliced stream's state holds its layout under the current options
static rs_status check_states(const rs_pipeline *p, const StreamPlan *sp, size_t ns)
{
    for (size_t i = 0; i < ns; ++i) {
        const StreamPlan &q = sp[i];
        if (!q.sliced || q.mode != UNIT_MERGE) continue;
        const SliceInfo &si = p->slices[i];
        if (!si.state || ((uintptr_t)si.state & 255) != 0) return RS_ERR_INVALID;
        if (si.state_bytes < q.st_total) return RS_ERR_CAPACITY;
    }
    return RS_OK;
}

// clear the scratch of the sliced streams this run plans
static rs_status clear_states(const rs_pipeline *p, const StreamPlan *sp, size_t ns, cudaStream_t stream)
{
    for (size_t i = 0; i < ns; ++i) {
        const StreamPlan &q = sp[i];
        if (!q.sliced || !q.plan_now || q.mode != UNIT_MERGE || q.slice_n == 0) continue;
        const cudaError_t e = cudaMemsetAsync(p->slices[i].state, 0, q.st_zero, stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return RS_OK;
}

struct Launch {
    KParams P;
    Plan pl;
    int grid, block;
    size_t smem;
};

// Host-only preparation: stream table in pinned memory, kernel parameters, grid.
// Makes no stream-ordered call, so it may run before a stream capture begins.
// The balanced unit count for a run (0: none): with the tag kernel on a persistent grid and
// one stream, the units of the plan made without balancing (n of them) are regrouped into
// r = floor(n / procs) whole rounds over the resident processors `procs`, so that the last
// round does not leave most of them idle.  Needs r >= 2: with one round every processor
// holds a single large unit and nothing evens out the processors' speeds.  Derived once,
// from the unbalanced plan; a plan made with the count may hold a few units fewer (each
// unit takes ceil(regions / count) parents), which the caller keeps as it is.
static uint64_t balanced_units(const rs_pipeline *p, int strategy, const Topo &topo, const Plan &pl, uint64_t procs)
{
    if (strategy != RS_STRATEGY_TAG || topo.mix || p->opts.grid != 0 || (p->opts.flags & RS_FLAG_UNBALANCED_UNITS))
        return 0;
    int with_units = 0;
    for (const StreamPlan &q : pl.sp) {
        if (q.slice_n == 0) continue;
        if (q.sliced) return 0;
        ++with_units;
    }
    if (with_units != 1 || procs == 0) return 0;
    const uint64_t n = pl.total_units;
    const uint64_t r = n / procs;
    if (r < 2 || r * procs == n) return 0;
    return r * procs;
}

// Room for n streams in the pinned host copy of the stream table, grown to a power of two
// (at least 16): freeing page-locked memory waits for the device, so it happens seldom.
static rs_status reserve_table(rs_pipeline *p, size_t n)
{
    if (p->table_cap >= n) return RS_OK;
    cudaError_t e;
    if (p->upload_pending) {
        if ((e = cudaEventSynchronize(p->upload_done)) != cudaSuccess) return cuda_fail(e);
        p->upload_pending = false;
    }
    if (p->table_host) cudaFreeHost(p->table_host);
    p->table_host = nullptr;
    p->table_cap = 0;
    p->table_dirty = true;
    size_t cap = 16;
    while (cap < n) cap <<= 1;
    if ((e = cudaMallocHost((void **)&p->table_host, cap * sizeof(DevStream))) != cudaSuccess) return cuda_fail(e);
    p->table_cap = cap;
    return RS_OK;
}

rs_status rs_pipeline_reserve_streams(rs_pipeline *p, uint64_t n_streams)
{
    if (!p) return RS_ERR_INVALID;
    return reserve_table(p, (size_t)n_streams);
}

static rs_status prepare(rs_pipeline *p, void *ws, uint64_t ws_bytes, Launch *out)
{
    if (!p || !ws) return RS_ERR_INVALID;
    if (p->streams.empty()) return RS_ERR_NOT_READY;
    Launch &Lc = *out;
    Topo topo;
    const int strategy = run_strategy(p, &topo);
    if (strategy < 0) return RS_ERR_INVALID;
    if (strategy != RS_STRATEGY_TAG && p->opts.ensemble_width > 4 * RS_W) return RS_ERR_INVALID;
    // a balanced unit count decided by an earlier run on the same streams and options
    uint64_t bal = (p->table_dirty || p->table_ws != ws) ? 0 : p->table_bal;
    cudaError_t e;
    const rs_pipeline_opts &o = p->opts;
    unsigned char *wsb = (unsigned char *)ws;
    const size_t ns = p->streams.size();
    for (int pass = 0;; ++pass) {
        Lc.pl = make_plan(p, strategy, p->opts, bal);
        const Plan &pl = Lc.pl;
        if (ws_bytes < pl.total) return RS_ERR_CAPACITY;
        rs_status sst = check_states(p, pl.sp.data(), pl.sp.size());
        if (sst != RS_OK) return sst;
        if (((uintptr_t)ws & 255) != 0) return RS_ERR_INVALID;
        if (pl.total_units >= (1ull << 31)) return RS_ERR_CAPACITY;
        if (!p->n_sm) {
            int dev = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e);
            if ((e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return cuda_fail(e);
        }

        // ---- kernel parameters ----
        KParams &P = Lc.P;
        memset(&P, 0, sizeof P);
        bool need_ctx = false, need_par = p->stages[0].kind == RS_ENUM_HASH;
        for (uint32_t i = 0; i < p->n_stages; ++i) {
            P.st[i] = to_dev(p->stages[i]);
            if (p->stages[i].kind == RS_FILTER && p->stages[i].op == RS_OP_HASH_CTX_LT) need_ctx = true;
            if (p->stages[i].kind == RS_FILTER && p->stages[i].op == RS_OP_WEIGHT_LT) need_par = true;
        }
        P.n_stages = (int)p->n_stages;
        P.strategy = strategy;
        P.n_streams = (uint32_t)ns;
        P.total_units = (uint32_t)pl.total_units;
        P.plan_tiles = (uint32_t)pl.plan_tiles;
        P.plan_pow2 = plan_pow2(pl, p->streams.size());
        P.plan_tile = plan_tile_parents(p);
        P.streams = (const DevStream *)(wsb + pl.table_off);
        P.hdr = (WsHeader *)wsb;
        P.V = o.ensemble_width / RS_W;
        P.C = o.queue_capacity;
        P.SC = o.signal_capacity;
        P.TE = o.tile_elements;
        P.NT = o.tiles_in_flight;
        P.need_ctx = need_ctx;
        P.need_par = need_par;
        bool wc = false, wsum = false, wm = false;
        for (const auto &s : p->streams) {
            wc |= s.out_count != nullptr;
            wsum |= s.out_sum != nullptr;
            wm |= s.out_min != nullptr;
        }
        // every non-empty stream must provide each output any stream asks for
        for (const auto &s : p->streams) {
            if (s.n_regions == 0) continue;
            if ((wc && !s.out_count) || (wsum && !s.out_sum) || (wm && !s.out_min)) return RS_ERR_INVALID;
        }
        // an emit sink claims positions with atomics on the counts, which every run zeroes
        // first: no identity results are written
        P.emit = is_emit(p);
        P.emit_f = fanout_product(p->stages, p->n_stages);
        P.want_count = wc && !P.emit;
        P.want_sum = wsum && !P.emit;
        P.want_min = wm && !P.emit;
        P.any_load = p->stages[0].kind == RS_ENUM_LOAD;
        P.budget = o.device_budget;
        P.spin_limit = 2000000000ull;   // 2 s on the global timer
        P.cpl = tag_chunk_cpl(p);
        P.L = strategy == RS_STRATEGY_TAG ? make_tag_layout(p, P.cpl)
                                          : make_layout(p, strategy, pl.Kmax, P.any_load, need_ctx, need_par, wm, topo);
        P.plan_fill = strategy == RS_STRATEGY_TAG;
        P.m16 = 1u << 16;
        P.m19 = 1u << 19;
        set_topo(P, topo);

        // processors per CTA: as asked, but no more than fit the per-block shared memory;
        // 0 = the count (8, 4, 2 or 1) giving the most resident processors per SM
        uint32_t wpb = o.warps_per_block;
        if (!p->smem_max) {
            int dev = 0, v = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e);
            if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
                return cuda_fail(e);
            p->smem_max = (size_t)v;
        }
        if (wpb == 0) {
            rs_status ws = auto_wpb(p, P, &wpb);
            if (ws != RS_OK) return ws;
        }
        while (wpb > 1 && (size_t)P.L.per_warp * wpb > p->smem_max) --wpb;
        if ((size_t)P.L.per_warp * wpb > p->smem_max) return RS_ERR_CAPACITY;
        Lc.block = (int)wpb * 32;
        Lc.smem = (size_t)P.L.per_warp * wpb;
        Lc.grid = (int)o.grid;
        if (pl.total_units == 0) break;   // only empty streams: nothing to launch
        if (Lc.grid == 0) {
            int bps = 0;
            int ce = rs_kernel_occupancy(P, Lc.block, Lc.smem, &bps);
            if (ce != 0) return cuda_fail((cudaError_t)ce);
            if (bps == 0) return RS_ERR_CAPACITY;
            p->last_bps = (uint32_t)bps;
            Lc.grid = bps * p->n_sm;
            uint64_t warps = (uint64_t)Lc.grid * wpb;   // no more processors than units
            if (warps > pl.total_units) {
                Lc.grid = (int)((pl.total_units + wpb - 1) / wpb);
                if (Lc.grid < 1) Lc.grid = 1;
            }
        } else {
            int ce = rs_kernel_max_smem_optin(P, Lc.smem);
            if (ce != 0) return cuda_fail((cudaError_t)ce);
            int bps = 0;
            ce = rs_kernel_occupancy(P, Lc.block, Lc.smem, &bps);
            if (ce != 0) return cuda_fail((cudaError_t)ce);
            p->last_bps = (uint32_t)bps;
        }

        // a count taken from an earlier run, or this pass's, stands: it is never derived
        // again from a plan made with it
        if (pass == 1 || bal != 0) break;
        const uint64_t want =
            balanced_units(p, strategy, topo, Lc.pl, (uint64_t)Lc.grid * (uint64_t)(Lc.block / 32));
        if (want == 0) break;
        bal = want;
    }
    const Plan &pl = Lc.pl;

    // ---- stream table (pinned host copy, uploaded by every run) ----
    if (p->table_dirty || !p->table_host || p->table_ws != ws || p->table_bal != bal) {
        if (p->upload_pending) {
            if ((e = cudaEventSynchronize(p->upload_done)) != cudaSuccess) return cuda_fail(e);
            p->upload_pending = false;
        }
        if (p->table_cap < ns) {
            const rs_status rst = reserve_table(p, ns);
            if (rst != RS_OK) return rst;
        }
        fill_table(p, pl.sp.data(), ns, (unsigned char *)ws, p->table_host);
        p->table_in_ws = nullptr;
        p->table_dirty = false;
        p->table_ws = ws;
        p->table_bal = bal;
    }

    p->last_grid = (uint32_t)Lc.grid;
    p->last_block = (uint32_t)Lc.block;
    p->last_smem = (uint32_t)Lc.smem;
    p->last_cp = strategy == RS_STRATEGY_TAG ? 32 * Lc.P.cpl : 0;
    return RS_OK;
}

// Stream-ordered part: workspace reset, table upload, kernel launch.
static rs_status enqueue(rs_pipeline *p, void *ws, const Launch &Lc, cudaStream_t stream, bool capturing)
{
    if (Lc.pl.total_units == 0) return RS_OK;   // only empty streams: nothing to launch
    cudaError_t e;
    unsigned char *wsb = (unsigned char *)ws;
    if ((e = cudaMemsetAsync(wsb, 0, Lc.pl.zero_end, stream)) != cudaSuccess) return cuda_fail(e);
    // a private workspace keeps the table an earlier run uploaded, until it is rebuilt
    const bool priv = (p->opts.flags & RS_FLAG_PRIVATE_WORKSPACE) != 0;
    if (capturing || !priv || p->table_in_ws != ws) {
        if ((e = cudaMemcpyAsync(wsb + Lc.pl.table_off, p->table_host, p->streams.size() * sizeof(DevStream),
                                 cudaMemcpyHostToDevice, stream)) != cudaSuccess)
            return cuda_fail(e);
        if (!capturing) {
            if (!p->upload_done) {
                if ((e = cudaEventCreateWithFlags(&p->upload_done, cudaEventDisableTiming)) != cudaSuccess)
                    return cuda_fail(e);
            }
            if ((e = cudaEventRecord(p->upload_done, stream)) != cudaSuccess) return cuda_fail(e);
            p->upload_pending = true;
            p->table_in_ws = priv ? ws : nullptr;
        }
    }
    if (Lc.P.emit) {
        for (const auto &s : p->streams)
            if (s.n_regions && (e = cudaMemsetAsync(s.out_count, 0, s.n_regions * 4, stream)) != cudaSuccess)
                return cuda_fail(e);
    }
    rs_status cst = clear_states(p, Lc.pl.sp.data(), Lc.pl.sp.size(), stream);
    if (cst != RS_OK) return cst;
    const bool timed = !capturing && p->t_cap > 0;
    const uint32_t slot = timed ? (p->t_count % p->t_cap) : 0;
    if (timed && (e = cudaEventRecord(p->tev[2 * slot], stream)) != cudaSuccess) return cuda_fail(e);
    uint64_t uu = 0;
    if (any_usum(Lc.pl.sp.data(), Lc.pl.sp.size(), &uu)) {
        int ug = (int)((uu + 7) / 8);
        if (ug > p->n_sm * 8) ug = p->n_sm * 8;
        if (ug < 1) ug = 1;
        int le2 = rs_launch_unit_offsets(Lc.P, ug, (void *)stream);
        if (le2 != 0) return cuda_fail((cudaError_t)le2);
    }
    if (Lc.P.plan_tiles > 0) {
        // planner: offsets and merge-path unit records for every UNIT_MERGE stream
        int pg = (int)((Lc.P.plan_tiles + 7) / 8);
        int cap = p->n_sm * 8;
        if (pg > cap) pg = cap;
        if (pg < 1) pg = 1;
        int le = rs_launch_planner(Lc.P, pg, (void *)stream);
        if (le != 0) return cuda_fail((cudaError_t)le);
    }
    int le = rs_launch_kernel(Lc.P, Lc.grid, Lc.block, Lc.smem, (void *)stream);
    if (le != 0) return cuda_fail((cudaError_t)le);
    if (any_merge(Lc.pl.sp.data(), Lc.pl.sp.size()) && !Lc.P.plan_fill) {
        // signal strategy: parents processed in pieces get their merged results (a sliced
        // stream's in the run holding its last unit)
        int fg = p->n_sm * 4;
        le = rs_launch_finalize(Lc.P, fg, (void *)stream);
        if (le != 0) return cuda_fail((cudaError_t)le);
    }
    if (timed) {
        if ((e = cudaEventRecord(p->tev[2 * slot + 1], stream)) != cudaSuccess) return cuda_fail(e);
        p->t_count++;
    }
    return RS_OK;
}

static rs_status run_impl(rs_pipeline *p, void *ws, uint64_t ws_bytes, cudaStream_t stream)
{
    Launch Lc;
    rs_status st = prepare(p, ws, ws_bytes, &Lc);
    if (st != RS_OK) return st;
    return enqueue(p, ws, Lc, stream, false);
}

extern "C" {

rs_status rs_run(rs_pipeline *p, void *workspace, uint64_t workspace_bytes, rs_cuda_stream stream)
{
    return run_impl(p, workspace, workspace_bytes, (cudaStream_t)stream);
}

rs_status rs_fetch_region_results(rs_pipeline *p, uint64_t stream_id, const rs_region_results *dst,
                                  rs_cuda_stream stream)
{
    if (!p || !dst || stream_id >= p->streams.size()) return RS_ERR_INVALID;
    const rs_stream_desc &s = p->streams[stream_id];
    const size_t R = s.n_regions;
    if (R == 0) return RS_OK;
    cudaError_t e;
    cudaStream_t cs = (cudaStream_t)stream;
    if (dst->count) {
        if (!s.out_count) return RS_ERR_INVALID;
        if (dst->count != s.out_count &&
            (e = cudaMemcpyAsync(dst->count, s.out_count, R * 4, cudaMemcpyDefault, cs)) != cudaSuccess)
            return cuda_fail(e);
    }
    if (dst->sum) {
        if (!s.out_sum) return RS_ERR_INVALID;
        if (dst->sum != s.out_sum &&
            (e = cudaMemcpyAsync(dst->sum, s.out_sum, R * 8, cudaMemcpyDefault, cs)) != cudaSuccess)
            return cuda_fail(e);
    }
    if (dst->min) {
        if (!s.out_min) return RS_ERR_INVALID;
        if (dst->min != s.out_min &&
            (e = cudaMemcpyAsync(dst->min, s.out_min, R * 4, cudaMemcpyDefault, cs)) != cudaSuccess)
            return cuda_fail(e);
    }
    return RS_OK;
}

rs_status rs_stream_upload(rs_pipeline *p, uint64_t stream_id, const rs_host_inputs *src, rs_cuda_stream stream)
{
    if (!p || !src || stream_id >= p->streams.size()) return RS_ERR_INVALID;
    const rs_stream_desc &s = p->streams[stream_id];
    const uint64_t R = s.n_regions;
    struct {
        const uint32_t *from;
        const uint32_t *to;
        uint64_t n;
    } c[5] = {{src->parents, s.parents, R},
              {src->region_len, s.region_len, R},
              {src->region_offsets, s.region_offsets, R ? R + 1 : 0},
              {src->elements, s.elements, s.n_elements},
              {src->ctx, s.ctx, R}};
    for (auto &x : c) {
        if (!x.from) continue;
        if (!x.to) return RS_ERR_INVALID;
        if (!x.n) continue;
        const cudaError_t e = cudaMemcpyAsync(const_cast<uint32_t *>(x.to), x.from, x.n * 4, cudaMemcpyHostToDevice,
                                              (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return RS_OK;
}

rs_status rs_get_stats(rs_pipeline *p, const void *workspace, rs_cuda_stream stream, rs_stats *out)
{
    if (!p || !workspace || !out) return RS_ERR_INVALID;
    cudaError_t e;
    if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e);
    WsHeader h;
    if ((e = cudaMemcpy(&h, workspace, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e);
    memset(out, 0, sizeof *out);
    out->device_status = h.status;
    out->n_nodes = p->n_stages;
    out->units = h.units;
    for (uint32_t i = 0; i < p->n_stages; ++i) {
        out->ensembles[i] = h.counters[4 * i + 0];
        out->items[i] = h.counters[4 * i + 1];
        out->signals[i] = h.counters[4 * i + 2];
        out->firings[i] = h.counters[4 * i + 3];
    }
    for (int i = 0; i < RS_PROF_SLOTS && i < 16; ++i) out->cycles[i] = h.cyc[i];
    out->grid = p->last_grid;
    out->block = p->last_block;
    out->smem_per_block = p->last_smem;
    out->blocks_per_sm = p->last_bps;
    out->chunk_parents = p->last_cp;
    if (h.status & (ST_STALL | ST_LOOKBACK_TIMEOUT | ST_COPY_TIMEOUT | ST_OVERFLOW)) return RS_ERR_STALL;
    if (h.status & ST_BAD_INPUT) return RS_ERR_DEVICE_INPUT;
    return RS_OK;
}

rs_status rs_graph_capture(rs_pipeline *p, void *workspace, uint64_t workspace_bytes, rs_cuda_stream stream)
{
    if (!p || !stream) return RS_ERR_INVALID;
    if (p->graph) return RS_ERR_STATE;
    for (const SliceInfo &si : p->slices)
        if (si.on) return RS_ERR_STATE;   // a slice runs once; its successor is another submission
    cudaError_t e;
    // the table upload inside the graph reads the pinned buffer at every replay:
    // build it now, outside the capture
    if (p->upload_pending) {
        if ((e = cudaEventSynchronize(p->upload_done)) != cudaSuccess) return cuda_fail(e);
        p->upload_pending = false;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    Launch Lc;
    rs_status st = prepare(p, workspace, workspace_bytes, &Lc);
    if (st != RS_OK) return st;
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return cuda_fail(e);
    st = enqueue(p, workspace, Lc, cs, true);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (st != RS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e);
    p->graph = ex;
    return RS_OK;
}

rs_status rs_graph_launch(rs_pipeline *p, rs_cuda_stream stream)
{
    if (!p) return RS_ERR_INVALID;
    if (!p->graph) return RS_ERR_NOT_READY;
    cudaError_t e = cudaGraphLaunch(p->graph, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return RS_OK;
}

rs_status rs_graph_release(rs_pipeline *p)
{
    if (!p) return RS_ERR_INVALID;
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    return RS_OK;
}

rs_status rs_timing_enable(rs_pipeline *p, uint32_t capacity)
{
    if (!p) return RS_ERR_INVALID;
    timing_free(p);
    if (capacity == 0) return RS_OK;
    try {
        p->tev.assign(2 * (size_t)capacity, nullptr);
    } catch (...) {
        return RS_ERR_NOMEM;
    }
    for (auto &e : p->tev) {
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) {
            timing_free(p);
            return cuda_fail(ce);
        }
    }
    p->t_cap = capacity;
    p->t_count = 0;
    return RS_OK;
}

rs_status rs_timing_read(rs_pipeline *p, float *ms, uint32_t max, uint32_t *n)
{
    if (!p || !n) return RS_ERR_INVALID;
    *n = 0;
    if (p->t_cap == 0) return RS_ERR_NOT_READY;
    uint32_t cnt = p->t_count < p->t_cap ? p->t_count : p->t_cap;
    uint32_t first = p->t_count - cnt;
    uint32_t w = 0;
    for (uint32_t i = 0; i < cnt && w < max; ++i) {
        uint32_t slot = (first + i) % p->t_cap;
        cudaError_t e = cudaEventSynchronize(p->tev[2 * slot + 1]);
        if (e != cudaSuccess) return cuda_fail(e);
        float t = 0.f;
        e = cudaEventElapsedTime(&t, p->tev[2 * slot], p->tev[2 * slot + 1]);
        if (e != cudaSuccess) return cuda_fail(e);
        if (ms) ms[w] = t;
        ++w;
    }
    *n = w;
    p->t_count = 0;
    return RS_OK;
}

rs_status rs_autotune(rs_pipeline *p, void *workspace, uint64_t workspace_bytes, rs_cuda_stream stream,
                      uint32_t trials, rs_pipeline_opts *best, float *best_ms)
{
    if (!p || !workspace) return RS_ERR_INVALID;
    if (p->graph) return RS_ERR_STATE;
    if (p->streams.empty()) return RS_ERR_NOT_READY;
    if (trials == 0) trials = 3;
    const rs_pipeline_opts base = p->opts;
    const uint32_t fan = max_fanout_of(p->stages, p->n_stages);
    const bool merge = p->stages[0].kind == RS_ENUM_LOAD;
    // whole-parent units (hashed streams) sized from the mean region length, per strategy
    rs_pipeline_opts probe = base;
    probe.regions_per_unit = 0;
    uint32_t K0[2] = {1, 1};
    for (const auto &s : p->streams) {
        for (int si = 0; si < 2; ++si) {
            const uint32_t k = choose_K(p, probe, s, si == 0 ? RS_STRATEGY_TAG : RS_STRATEGY_SIGNAL);
            if (k > K0[si]) K0[si] = k;
        }
    }

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&ev0)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaEventCreate(&ev1)) != cudaSuccess) { cudaEventDestroy(ev0); return cuda_fail(e); }
    rs_status result = RS_OK;
    // mean time of `trials` runs of configuration c; +inf when it does not fit or stalls
    // qmul: queue capacity as a multiple of the smallest legal one for the width
    auto time_of = [&](rs_pipeline_opts c, uint32_t qmul = 1) -> float {
        c.queue_capacity = 0;
        c.grid = 0;
        fill_defaults(&c, fan);
        c.queue_capacity *= qmul;
        if (check_opts(&c, fan) != RS_OK) return 1e30f;
        Topo tp;
        if (make_topo(p->stages, p->n_stages, c.boundary_modes,
                      c.strategy == RS_STRATEGY_TAG ? RS_STRATEGY_TAG : RS_STRATEGY_SIGNAL, &tp) != RS_OK)
            return 1e30f;
        p->opts = c;
        p->table_dirty = true;
        Topo topo;
        const int strategy = run_strategy(p, &topo);
        if (strategy < 0) return 1e30f;
        if (make_plan(p, strategy, c).total > workspace_bytes) return 1e30f;
        rs_status st = run_impl(p, workspace, workspace_bytes, (cudaStream_t)stream);
        if (st == RS_ERR_CAPACITY) return 1e30f;
        if (st != RS_OK) { result = st; return 1e30f; }
        cudaEventRecord(ev0, (cudaStream_t)stream);
        for (uint32_t t = 0; t < trials && st == RS_OK; ++t)
            st = run_impl(p, workspace, workspace_bytes, (cudaStream_t)stream);
        cudaEventRecord(ev1, (cudaStream_t)stream);
        if (st != RS_OK) { result = st; return 1e30f; }
        if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) { result = cuda_fail(e); return 1e30f; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        rs_stats stt;
        if (rs_get_stats(p, workspace, stream, &stt) != RS_OK) return 1e30f;   // never choose a stall
        return ms / (float)trials;
    };

    // Per strategy, a search from a starting point (128 items per ensemble, the first unit
    // shape): unit shape and ensemble width, then processors per CTA and (signal
    // strategy) tile size, each change kept when it is faster.  A strategy whose starting
    // point is over three times the best found so far is dropped.
    float best_t = 1e30f;
    rs_pipeline_opts best_o = base;
    uint32_t best_q = 1;
    const uint32_t strategies[2] = {RS_STRATEGY_TAG, RS_STRATEGY_SIGNAL};
    for (uint32_t si = 0; si < 2 && result == RS_OK; ++si) {
        // a strategy fixed in the options is the only one searched
        if (base.strategy != RS_STRATEGY_AUTO && strategies[si] != base.strategy) continue;
        const bool tag = strategies[si] == RS_STRATEGY_TAG;
        // (regions per unit, steps per parent)
        uint32_t shapes[12][2];
        static_assert(sizeof(k_tag_shapes) / sizeof(k_tag_shapes[0]) <= 12, "unit shapes fit the search");
        int n_shapes = 0;
        if (merge && tag) {
            for (const auto &sh : k_tag_shapes) {
                shapes[n_shapes][0] = sh[0];
                shapes[n_shapes++][1] = sh[1];
            }
        } else if (merge) {
            const uint32_t sh[6][2] = {{128, 16}, {256, 16}, {512, 16}, {128, 32}, {64, 64}, {32, 128}};
            for (int i = 0; i < 6; ++i) { shapes[i][0] = sh[i][0]; shapes[i][1] = sh[i][1]; }
            n_shapes = 6;
        } else {
            const uint32_t k0 = K0[si], kmax = tag ? RS_TAG_MAX_K : RS_MAX_K;
            shapes[n_shapes][0] = k0;
            shapes[n_shapes++][1] = 0;
            if (k0 * 2 <= kmax) { shapes[n_shapes][0] = k0 * 2; shapes[n_shapes++][1] = 0; }
            if (k0 > 1) { shapes[n_shapes][0] = k0 / 2; shapes[n_shapes++][1] = 0; }
        }
        rs_pipeline_opts cur = base;
        cur.strategy = strategies[si];
        cur.ensemble_width = 4 * RS_W;
        cur.warps_per_block = 0;
        cur.tile_elements = 0;
        cur.tiles_in_flight = 0;
        cur.regions_per_unit = shapes[0][0];
        cur.region_cost = shapes[0][1];
        float cur_t = time_of(cur);
        if (cur_t > 3.f * best_t) continue;
        // tag strategy: every unit shape at each ensemble width (128, 256, 64 items), since
        // the best shape depends on the width; signal strategy: shapes at 128, then 64
        const uint32_t widths[3] = {4u, 8u, 2u};
        for (int wi = 0; wi < (tag ? 3 : 1) && result == RS_OK; ++wi) {
            for (int i = 0; i < n_shapes && result == RS_OK; ++i) {
                if (wi == 0 && i == 0) continue;   // the starting point, timed above
                rs_pipeline_opts c = cur;
                c.ensemble_width = widths[wi] * RS_W;
                c.regions_per_unit = shapes[i][0];
                c.region_cost = shapes[i][1];
                const float t = time_of(c);
                if (t < cur_t) { cur_t = t; cur = c; }
            }
        }
        if (!tag) {
            rs_pipeline_opts c = cur;
            c.ensemble_width = 2 * RS_W;
            c.tile_elements = 0;
            const float t = time_of(c);
            if (t < cur_t) { cur_t = t; cur = c; }
        }
        for (uint32_t wb : {4u, 8u}) {
            rs_pipeline_opts c = cur;
            c.warps_per_block = wb;
            const float t = time_of(c);
            if (t < cur_t) { cur_t = t; cur = c; }
        }
        if (merge && !tag) {
            // element staging: tiles of W against 2 W elements
            for (uint32_t m : {2u}) {
                rs_pipeline_opts c = cur;
                c.tile_elements = m * cur.ensemble_width;
                const float t = time_of(c);
                if (t < cur_t) { cur_t = t; cur = c; }
            }
        }
        // queue capacity: 2 and 4 times the smallest legal one (deeper queues let a node
        // fire several ensembles in a row, and cost shared memory, hence occupancy)
        uint32_t cur_q = 1;
        for (uint32_t qm : {2u, 4u}) {
            const float t = time_of(cur, qm);
            if (t < cur_t) { cur_t = t; cur_q = qm; }
        }
        if (cur_t < best_t) {
            best_t = cur_t;
            best_o = cur;
            best_q = cur_q;
        }
    }
    // Per-edge boundary modes (Section 5: the best representation of regional context can
    // differ per stage, and should be chosen from measurements): for a linear pipeline,
    // signals into the first stages and tags from stage sw on, at every switch point sw;
    // per-lane selection (Section 6) on every edge; and per-lane selection into stage 1
    // with tags after it.  Each at 128 and 64 items per ensemble, on the per-edge kernel.
    bool linear = true;
    for (uint32_t i = 1; i < p->n_stages; ++i) linear = linear && stage_input(p->stages, i) == i - 1;
    if (base.strategy == RS_STRATEGY_AUTO && linear && p->n_stages >= 3 && result == RS_OK) {
        const uint32_t n = p->n_stages;
        uint32_t cand[RS_MAX_STAGES + 2];
        int nc = 0;
        for (uint32_t sw = 2; sw < n; ++sw) {
            uint32_t m = 0;
            for (uint32_t c = 1; c < n; ++c) m |= RS_BOUNDARY(c, c < sw ? RS_BOUNDARY_SIGNAL : RS_BOUNDARY_TAG);
            cand[nc++] = m;
        }
        uint32_t lane_all = 0, lane_tag = 0;
        for (uint32_t c = 1; c < n; ++c) {
            const uint32_t lm = p->stages[c].kind == RS_EXPAND ? RS_BOUNDARY_SIGNAL : RS_BOUNDARY_LANE;
            lane_all |= RS_BOUNDARY(c, lm);
            lane_tag |= RS_BOUNDARY(c, c == 1 ? lm : RS_BOUNDARY_TAG);
        }
        cand[nc++] = lane_all;
        cand[nc++] = lane_tag;
        for (int i = 0; i < nc && result == RS_OK; ++i) {
            for (uint32_t W : {4u, 2u}) {
                rs_pipeline_opts c = base;
                c.strategy = RS_STRATEGY_SIGNAL;
                c.boundary_modes = cand[i];
                c.ensemble_width = W * RS_W;
                c.signal_capacity = 0;
                c.regions_per_unit = 0;
                c.region_cost = 0;
                c.warps_per_block = 0;
                c.tile_elements = 0;
                c.tiles_in_flight = 0;
                const float t = time_of(c);
                if (t < best_t) {
                    best_t = t;
                    best_o = c;
                    best_q = 1;
                }
            }
        }
    }
    best_o.queue_capacity = 0;
    best_o.grid = 0;
    fill_defaults(&best_o, fan);
    best_o.queue_capacity *= best_q;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    p->opts = best_o;
    p->table_dirty = true;
    if (result != RS_OK) return result;
    if (best) *best = best_o;
    if (best_ms) *best_ms = best_t;
    return RS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// rs_run_noalloc: the same work as rs_run, with its scratch memory in a fixed array
// compiled into this library instead of a workspace passed by the caller.
//
// Some callers cannot allocate device memory when they run the pipeline: a host
// application that owns the whole device-memory budget through its own allocator or a
// hard cap, or a latency-critical loop in which an allocation (which may synchronise
// the device) is not acceptable.  This entry point lets them run without a workspace:
// it allocates nothing (no cudaMalloc / cudaFree / cudaMallocHost, no library that
// allocates), and uses the scratch array below.  The array is RS_NOALLOC_WS_BYTES on
// every GPU that loads the library, held until the process exits.

#define RS_NOALLOC_WS_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[RS_NOALLOC_WS_BYTES];

// Device address of the scratch array, looked up once per device (with that device
// current) on the first rs_run_noalloc call made while it is current.
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];

static rs_status noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 256) return RS_ERR_CAPACITY;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        g_noalloc_addr[dev] = ptr;
    }
    *out = g_noalloc_addr[dev];
    return RS_OK;
}

// copies the first n entries of the table (8-byte words; sizeof(DevStream) is a multiple
// of 8) into the scratch array
__global__ void __launch_bounds__(256) rs_noalloc_table_kernel(const __grid_constant__ NoallocTable t, DevStream *dst,
                                                               uint32_t n)
{
    const uint32_t words = n * (uint32_t)(sizeof(DevStream) / 8);
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&t.s[0]);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) d[i] = src[i];
}

static_assert(sizeof(DevStream) % 8 == 0, "the table copy moves 8-byte words");

static void make_plan_fixed(const rs_pipeline *p, int strategy, FixedPlan *pl)
{
    const size_t ns = p->streams.size();
    const uint32_t nsinks = n_leaves(p->stages, p->n_stages);
    for (size_t i = 0; i < ns; ++i) {
        plan_stream(p, p->opts, strategy, p->streams[i], pl->sp[i], !p->slices[i].on);
        apply_slice(p->slices[i], pl->sp[i], strategy, nsinks);
    }
    layout_plan(pl->sp, ns, strategy, n_leaves(p->stages, p->n_stages), &pl->total_units, &pl->plan_tiles,
                &pl->Kmax, &pl->zero_end, &pl->table_off, &pl->total);
}

extern "C" rs_status rs_run_noalloc(rs_pipeline *p, rs_cuda_stream stream)
{
    if (!p) return RS_ERR_INVALID;
    if (p->streams.empty()) return RS_ERR_NOT_READY;
    if (p->streams.size() > RS_NOALLOC_MAX_STREAMS) return RS_ERR_CAPACITY;
    Topo topo;
    const int strategy = run_strategy(p, &topo);
    if (strategy < 0) return RS_ERR_INVALID;
    if (strategy != RS_STRATEGY_TAG && p->opts.ensemble_width > 4 * RS_W) return RS_ERR_INVALID;
    rs_status st0;
    FixedPlan &pl = p->noalloc_plan;
    make_plan_fixed(p, strategy, &pl);
    if (pl.total > RS_NOALLOC_WS_BYTES) return RS_ERR_CAPACITY;   // beyond the fixed scratch
    if ((st0 = check_states(p, pl.sp, p->streams.size())) != RS_OK) return st0;
    if (pl.total_units >= (1ull << 31)) return RS_ERR_CAPACITY;
    void *ws = nullptr;
    rs_status st = noalloc_scratch(&ws);
    if (st != RS_OK) return st;
    cudaError_t e;
    if (!p->n_sm) {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e);
    }
    const rs_pipeline_opts &o = p->opts;
    unsigned char *wsb = (unsigned char *)ws;
    const size_t ns = p->streams.size();

    // stream table in the pipeline's own host memory (pointers into the scratch array)
    fill_table(p, pl.sp, ns, wsb, p->noalloc_table.s);
    if (pl.total_units == 0) return RS_OK;

    KParams P;
    memset(&P, 0, sizeof P);
    bool need_ctx = false, need_par = p->stages[0].kind == RS_ENUM_HASH;
    for (uint32_t i = 0; i < p->n_stages; ++i) {
        P.st[i] = to_dev(p->stages[i]);
        if (p->stages[i].kind == RS_FILTER && p->stages[i].op == RS_OP_HASH_CTX_LT) need_ctx = true;
        if (p->stages[i].kind == RS_FILTER && p->stages[i].op == RS_OP_WEIGHT_LT) need_par = true;
    }
    P.n_stages = (int)p->n_stages;
    P.strategy = strategy;
    P.n_streams = (uint32_t)ns;
    P.total_units = (uint32_t)pl.total_units;
    P.plan_tiles = (uint32_t)pl.plan_tiles;
    P.plan_pow2 = plan_pow2(pl, p->streams.size());
    P.plan_tile = plan_tile_parents(p);
    P.streams = (const DevStream *)(wsb + pl.table_off);
    P.hdr = (WsHeader *)wsb;
    P.V = o.ensemble_width / RS_W;
    P.C = o.queue_capacity;
    P.SC = o.signal_capacity;
    P.TE = o.tile_elements;
    P.NT = o.tiles_in_flight;
    P.need_ctx = need_ctx;
    P.need_par = need_par;
    bool wc = false, wsum = false, wm = false;
    for (const auto &s : p->streams) {
        wc |= s.out_count != nullptr;
        wsum |= s.out_sum != nullptr;
        wm |= s.out_min != nullptr;
    }
    for (const auto &s : p->streams) {
        if (s.n_regions == 0) continue;
        if ((wc && !s.out_count) || (wsum && !s.out_sum) || (wm && !s.out_min)) return RS_ERR_INVALID;
    }
    P.emit = is_emit(p);
    P.emit_f = fanout_product(p->stages, p->n_stages);
    P.want_count = wc && !P.emit;
    P.want_sum = wsum && !P.emit;
    P.want_min = wm && !P.emit;
    P.any_load = p->stages[0].kind == RS_ENUM_LOAD;
    P.budget = o.device_budget;
    P.spin_limit = 2000000000ull;
    P.cpl = tag_chunk_cpl(p);
    P.L = strategy == RS_STRATEGY_TAG ? make_tag_layout(p, P.cpl)
                                      : make_layout(p, strategy, pl.Kmax, P.any_load, need_ctx, need_par, wm, topo);
    P.plan_fill = strategy == RS_STRATEGY_TAG;
    P.m16 = 1u << 16;
    P.m19 = 1u << 19;
    set_topo(P, topo);
    if (!p->smem_max) {
        int dev = 0, v = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
            return cuda_fail(e);
        p->smem_max = (size_t)v;
    }
    uint32_t wpb = o.warps_per_block;
    if (wpb == 0) {
        rs_status ws = auto_wpb(p, P, &wpb);
        if (ws != RS_OK) return ws;
    }
    while (wpb > 1 && (size_t)P.L.per_warp * wpb > p->smem_max) --wpb;
    if ((size_t)P.L.per_warp * wpb > p->smem_max) return RS_ERR_CAPACITY;
    const int block = (int)wpb * 32;
    const size_t smem = (size_t)P.L.per_warp * wpb;
    int grid = (int)o.grid;
    if (grid == 0) {
        int bps = 0;
        int ce = rs_kernel_occupancy(P, block, smem, &bps);
        if (ce != 0) return cuda_fail((cudaError_t)ce);
        if (bps == 0) return RS_ERR_CAPACITY;
        grid = bps * p->n_sm;
        uint64_t warps = (uint64_t)grid * wpb;
        if (warps > pl.total_units) grid = (int)((pl.total_units + wpb - 1) / wpb);
        if (grid < 1) grid = 1;
    } else {
        int ce = rs_kernel_max_smem_optin(P, smem);
        if (ce != 0) return cuda_fail((cudaError_t)ce);
    }

    // the scratch keeps the previous call's contents: clear the part that must start at 0
    cudaStream_t cs = (cudaStream_t)stream;
    if ((e = cudaMemsetAsync(wsb, 0, pl.zero_end, cs)) != cudaSuccess) return cuda_fail(e);
    // the stream table reaches the device as the parameter of a copy kernel: no staging
    // buffer and no copy from pageable host memory
    rs_noalloc_table_kernel<<<1, 256, 0, cs>>>(p->noalloc_table, (DevStream *)(wsb + pl.table_off), (uint32_t)ns);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    if (P.emit) {
        for (const auto &s : p->streams)
            if (s.n_regions && (e = cudaMemsetAsync(s.out_count, 0, s.n_regions * 4, cs)) != cudaSuccess)
                return cuda_fail(e);
    }
    if ((st0 = clear_states(p, pl.sp, ns, cs)) != RS_OK) return st0;
    uint64_t uu = 0;
    if (any_usum(pl.sp, ns, &uu)) {
        int ug = (int)((uu + 7) / 8);
        if (ug > p->n_sm * 8) ug = p->n_sm * 8;
        if (ug < 1) ug = 1;
        int le2 = rs_launch_unit_offsets(P, ug, (void *)cs);
        if (le2 != 0) return cuda_fail((cudaError_t)le2);
    }
    if (P.plan_tiles > 0) {
        int pg = (int)((P.plan_tiles + 7) / 8);
        if (pg > p->n_sm * 8) pg = p->n_sm * 8;
        if (pg < 1) pg = 1;
        int le = rs_launch_planner(P, pg, (void *)cs);
        if (le != 0) return cuda_fail((cudaError_t)le);
    }
    int le = rs_launch_kernel(P, grid, block, smem, (void *)cs);
    if (le != 0) return cuda_fail((cudaError_t)le);
    if (any_merge(pl.sp, ns) && !P.plan_fill) {
        le = rs_launch_finalize(P, p->n_sm * 4, (void *)cs);
        if (le != 0) return cuda_fail((cudaError_t)le);
    }
    return RS_OK;
}
