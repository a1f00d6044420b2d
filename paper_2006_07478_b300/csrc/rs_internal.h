// rs_internal.h -- structures shared by the host API (rs_api.cu) and the device
// kernels (rs_kernel.cu).  Not part of the public ABI.
#pragma once
#include <stdint.h>

#include "rs.h"

#define RS_W 32                       // lanes of one SIMD processor (a warp)
#define RS_MAX_EDGES (RS_MAX_STAGES - 1)
#define RS_MAX_K 256                  // parents per work unit
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
};

struct DevStage {
    uint32_t op;
    uint32_t fanout;
    uint32_t p0, p1;
    uint32_t c0;         // fmix32(p0 ^ RS_GOLD): the per-stage half of hash32, precomputed
    uint32_t pad[3];
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
    uint32_t K;          // parents per unit
    uint32_t n_units;
    uint32_t unit_base;  // first global ticket of this stream
    uint32_t tma_ok;     // elements pointer 16-byte aligned: stage tiles with bulk copies
    uint32_t pad;
};

// Status bits written by the device.
enum : uint32_t {
    ST_STALL = 1u,
    ST_LOOKBACK_TIMEOUT = 2u,
    ST_COPY_TIMEOUT = 4u,
    ST_BAD_INPUT = 8u,
    ST_OVERFLOW = 16u,
};

// Workspace header (reset by a memset before every run).
struct WsHeader {
    unsigned int cursor;
    unsigned int status;
    unsigned int pad[14];
    unsigned long long units;
    unsigned long long counters[4 * RS_MAX_STAGES];   // ensembles, items, signals, firings
};

// Per-warp shared-memory layout (byte offsets from the warp's base).
struct SmemLayout {
    uint32_t per_warp;
    uint32_t o_mbar, o_tiles, o_off, o_ctx, o_par, o_rc, o_rs, o_rm, o_qv, o_qt, o_sq, o_scr;
};

struct KParams {
    DevStage st[RS_MAX_STAGES];
    int n_stages;
    int strategy;                 // RS_STRATEGY_SIGNAL or RS_STRATEGY_TAG
    uint32_t n_streams;
    uint32_t total_units;
    const DevStream *streams;
    WsHeader *hdr;
    unsigned long long *lookback; // one word per unit
    uint32_t V;                   // items per lane per ensemble (W = 32 V)
    uint32_t C, SC, TE, NT;       // queue slots, signal slots, tile elements, tiles
    uint32_t need_ctx, need_par, want_count, want_sum, want_min;
    uint32_t any_load;
    unsigned long long budget;
    unsigned long long spin_limit;
    SmemLayout L;
};

// Launch helper implemented in rs_kernel.cu.
int rs_launch_kernel(const KParams &P, int grid, int block, size_t smem, void *stream);
int rs_kernel_max_smem_optin(int strategy, int V, size_t smem);
int rs_kernel_occupancy(int strategy, int V, int block, size_t smem, int *blocks_per_sm);
