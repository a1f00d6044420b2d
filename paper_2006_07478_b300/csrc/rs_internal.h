// rs_internal.h -- structures shared by the host API (rs_api.cu) and the device
// kernels (rs_kernel.cu).  Not part of the public ABI.
#pragma once
#include <stdint.h>

#include "rs.h"

#define RS_W 32                       // lanes of one SIMD processor (a warp)
#define RS_MAX_EDGES (RS_MAX_STAGES - 1)
#define RS_MAX_K 512                  // parents per work unit
#define RS_GOLD 0x9E3779B9u

// Device operation codes: the public (kind, op) pair flattened, with variants the
// host picks (e.g. a power-of-two modulus becomes a mask).
enum DevOp : uint32_t {
    D_ENUM_HASH = 1,
    D_ENUM_LOAD = 2,
    D_FILT_MOD = 3,
    D_FILT_MASK = 4,     // modulus is a power of two: keep (x & p0) == p1
    D_FILT_HASH_CTX = 5,
    D_FILT_WEIGHT = 6,
    D_MAP_MULADD = 7,
    D_EXPAND = 8,
    D_AGG = 9,
    D_EMIT = 10,         // sink: survivors into their region's segment of out_values
};

struct DevStage {
    uint32_t op;
    uint32_t fanout;
    uint32_t p0, p1;
    uint32_t c0;         // fmix32(p0 ^ RS_GOLD): the per-stage half of hash32, precomputed
    uint32_t c0s;        // c0 ^ (c0 >> 16): fmix32(x ^ c0) starts from x ^ (x >> 16) ^ c0s
    uint32_t pad[2];
};

// How region boundaries travel over an edge (per-edge boundary modes).
enum : uint32_t {
    EM_SIG = 0,    // Begin/End signals with credits; ensembles cut at every signal (Section 3)
    EM_TAG = 1,    // every item carries its region (Section 2.3 / Section 5)
    EM_LANE = 2,   // signals with credits, ensembles not cut: each lane selects the pre- or
                   // post-signal context of its own item (Section 6, future work)
};
// Work decomposition of a stream.
enum : uint32_t {
    UNIT_REGIONS = 0,   // a unit is K whole consecutive parents (hashed elements: no offsets needed)
    UNIT_MERGE = 1,     // merge-path units: a parent costs DevStream::c steps, an element 1 step,
                        // a unit is D steps (DevStream.D); parents straddling units are split
};
#define RS_STEP_REGION 16u   // default merge-path steps per parent (rs_pipeline_opts.region_cost)
#define RS_NOT_POW2 0xFFu
#define RS_PLAN_TILE 1024u                                  // parents per planner tile
#define RS_PLAN_TILE_SMALL 128u                             // ... when the streams hold few regions
#define RS_USUM_MEAN 8.0                                    // loaded streams of lengths whose regions
                                                            // average below this use fixed-parent units

// Start of merge-path unit u: i = parents whose header step lies before u*D, j = absolute
// index of the unit's first element, head_off / first_off = absolute offsets of parents
// i-1 and i.
struct UnitRec {
    uint32_t i, j, head_off, first_off;
};

// Partial aggregate of a parent processed in pieces (indexed by the unit owning it).
struct Slot {
    unsigned long long sum;
    uint32_t count, min_inv;   // min_inv = max of ~value: 0 is the identity
    uint32_t region;           // parent id + 1, set by the owning unit; 0 = slot unused
    uint32_t pad;
};

// Stream table entry (lives in the workspace).
struct DevStream {
    const uint32_t *parents;
    const uint32_t *len;
    const uint32_t *offsets;
    const uint32_t *elements;
    const uint32_t *ctx;
    uint32_t *out_count;
    unsigned long long *out_sum;
    uint32_t *out_min;
    uint64_t n_elements;
    uint32_t R;
    uint32_t K;          // parents per unit (UNIT_REGIONS)
    uint32_t n_units;    // units (UNIT_MERGE: an upper bound; the planner records the count)
    uint32_t unit_base;  // first global ticket of this stream
    uint32_t tma_ok;     // elements pointer 16-byte aligned: stage tiles with bulk copies
    uint32_t mode;       // UNIT_REGIONS or UNIT_MERGE
    // UNIT_MERGE only (workspace arrays)
    UnitRec *rec;        // n_units + 1 records
    Slot *slots;         // n_units slots
    uint32_t *u_count;   // units actually used, written by the planner
    unsigned long long *plan_lb;   // planner look-back words, one per planner tile
    uint32_t plan_tiles, plan_base;
    uint32_t D;          // merge-path steps per unit
    uint32_t dsh;        // log2 D when D is a power of two, else RS_NOT_POW2
    uint32_t c;          // merge-path steps per parent (an element costs one)
    // emit sink: region r's survivors go to out_values[emit_f * (offsets[r] - offsets[0]) ...]
    uint32_t *out_values;
    unsigned long long out_values_len;
    // tree topologies: the second leaf's per-region results
    uint32_t *out2_count;
    unsigned long long *out2_sum;
    uint32_t *out2_min;
    // sliced runs: this run processes units [slice_lo, slice_lo + n_units) of the stream;
    // slot_units = the stream's whole unit count (the length of each leaf's slot array);
    // finalize: this run holds the stream's last unit (the signal strategy then writes the
    // merged results of the parents processed in pieces)
    uint32_t slice_lo, slot_units, finalize;
    // fixed-parent units of a stream of lengths (UNIT_REGIONS over loaded elements): each
    // unit's length sum, and per group of 32 units the exclusive prefix of the group sums
    uint32_t *usum, *usum_grp;
};

// Status bits written by the device.
enum : uint32_t {
    ST_STALL = 1u,
    ST_LOOKBACK_TIMEOUT = 2u,
    ST_COPY_TIMEOUT = 4u,
    ST_BAD_INPUT = 8u,
    ST_OVERFLOW = 16u,
};
#define ST_ANY_STALL (ST_STALL | ST_LOOKBACK_TIMEOUT | ST_COPY_TIMEOUT | ST_OVERFLOW)

// Cycle-breakdown slots (optional profiling counters).
enum : int {
    PF_SETUP = 0,      // claim + stream lookup + lengths/offsets + context loads
    PF_LOOKBACK = 1,   // waiting on predecessors' prefix words
    PF_TILEWAIT = 2,   // waiting for bulk copies to land
    PF_ENUM = 3,       // enumeration (signal emission)
    PF_NODE0 = 4,      // PF_NODE0 + i: firing node i (1..5), minus tile waits
    PF_FLUSH = 10,     // writing per-parent results
    PF_TOTAL = 11,     // whole warp lifetime
    PF_GATHER1 = 12,   // node 1: parents and elements of an ensemble (inside node 1)
    PF_COMPUTE = 13,   // element stages: the stage's op on the ensemble (inside nodes)
    PF_COMPACT = 14,   // element stages: ballot compaction into the next ring (inside nodes)
    PF_TILES = 15,     // node 1: recycling tiles and issuing bulk copies (inside node 1)
    RS_PROF_SLOTS = 16
};

// Workspace header (reset by a memset before every run).
struct WsHeader {
    unsigned int cursor;
    unsigned int status;
    unsigned int plan_cursor;
    unsigned int pad[13];
    unsigned long long units;
    unsigned long long counters[4 * RS_MAX_STAGES];   // ensembles, items, signals, firings
    // optional cycle breakdown (KParams.profile): SM clock cycles summed over warps
    unsigned long long cyc[RS_PROF_SLOTS];
};

// Per-warp shared-memory layout (byte offsets from the warp's base).
struct SmemLayout {
    uint32_t per_warp;
    uint32_t o_prof, o_cnt, o_pend, o_mbar, o_mmeta, o_tiles, o_rc, o_rs, o_rm, o_qv, o_qt, o_sq, o_scr;
    uint32_t o_raw[2], o_moff[2], o_ctxb[2], o_parb[2];   // double-buffered unit metadata
    // tag kernel: rings of records of the non-empty parents node 1 is reading (PR
    // entries; the {region, operand} ring is mirrored to 2 PR)
    uint32_t o_nra, o_nst, o_npar, pr;
    // second leaf's per-parent accumulators (tree topologies)
    uint32_t o_rc2, o_rs2, o_rm2;
};

struct KParams {
    DevStage st[RS_MAX_STAGES];
    int n_stages;
    int strategy;                 // RS_STRATEGY_SIGNAL or RS_STRATEGY_TAG
    uint32_t n_streams;
    uint32_t total_units;
    uint32_t plan_tiles;          // planner tickets over all UNIT_MERGE streams
    const DevStream *streams;
    WsHeader *hdr;
    uint32_t V;                   // items per lane per ensemble (W = 32 V)
    uint32_t C, SC, TE, NT;       // queue slots, signal slots, tile elements, tiles
    uint32_t need_ctx, need_par, want_count, want_sum, want_min;
    uint32_t any_load;
    unsigned long long budget;
    unsigned long long spin_limit;
    uint32_t profile;             // accumulate the cycle breakdown
    uint32_t plan_fill;           // tag strategy: identity results written by the planner (regions a unit
                                  // starts inside) and by the pipeline kernel (every other region)
    uint32_t cpl;                 // tag strategy: parents per lane in node 1's parent chunks (1 or 2)
    uint32_t plan_pow2;           // every merge-path stream's D is a power of two (planner divides by shifts)
    uint32_t plan_tile;           // parents per planner tile (RS_PLAN_TILE or RS_PLAN_TILE_SMALL)
    uint32_t m16, m19;            // 2^16 and 2^19: x >> 16 = umulhi(x, m16), x >> 13 = umulhi(x, m19)
                                  // (run-time values, so the shifts stay multiplies)
    uint32_t emit;                // the last stage is the emit sink (results per item, not per region)
    uint32_t emit_f;              // its segment slots per element: the product of the maximum fan-outs
    // per-edge boundary modes and tree topologies (the generic per-edge kernel only):
    // node c's input edge carries region boundaries as emode[c] (EM_SIG, EM_TAG or EM_LANE);
    // node c reads the output of node up[c]; kids[i] has bit c set for each child c of node i;
    // sink_of[c] numbers the aggregate / emit leaves in stage order (0xFF: not a leaf)
    uint32_t mix;
    uint32_t n_sinks;
    uint8_t emode[RS_MAX_STAGES], up[RS_MAX_STAGES], kids[RS_MAX_STAGES], sink_of[RS_MAX_STAGES];
    SmemLayout L;
};

// Workspace bytes of the next rs_run alone (rs_workspace_size also covers every option
// set the autotuner may try); used by the server for each launch (rs_api.cu).
rs_status rs_run_workspace_bytes(const rs_pipeline *p, uint64_t *bytes);

// Launch helpers implemented in rs_kernel.cu.
int rs_launch_kernel(const KParams &P, int grid, int block, size_t smem, void *stream);
int rs_launch_planner(const KParams &P, int grid, void *stream);
int rs_launch_unit_offsets(const KParams &P, int grid, void *stream);   // fixed-parent units' offsets
// pinned room for the stream table of n streams, ahead of the first run that needs it
// (the server reserves its batch size, so no run frees page-locked memory mid-stream)
rs_status rs_pipeline_reserve_streams(rs_pipeline *p, uint64_t n_streams);
// the calibration kernel (rs_calib.cu): the cascade's element arithmetic over one region
int rs_launch_calib(const uint32_t *elements, unsigned long long n, uint32_t ctx, const uint32_t c0[3],
                    const uint32_t theta[3], unsigned long long *out, int n_sm, void *stream);
int rs_launch_finalize(const KParams &P, int grid, void *stream);
int rs_kernel_max_smem_optin(const KParams &P, size_t smem);
int rs_kernel_occupancy(const KParams &P, int block, size_t smem, int *blocks_per_sm);
const void *rs_kernel_entry(const KParams &P);   // the kernel a launch with P would use
int rs_kernel_is_specialised(const KParams &P);
// the tag strategy's kernel (rs_tag.cu, rs_tag2.cu)
const void *rs_tag_kernel_entry(const KParams &P);
int rs_tag_kernel_is_specialised(const KParams &P);
