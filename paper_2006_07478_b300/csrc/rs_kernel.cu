// rs_kernel.cu -- persistent pipeline kernel for region-segmented streams (sm_103a).
//
// Mapping of the paper's model (Timcheck & Buhler, Sections 2-4) onto B300:
//   * SIMD processor (Section 2.2) = one warp.  The paper treats a CUDA block as
//     the SIMD width; here the hardware's own 32-lane SIMD unit is the processor, so
//     a node firing needs only __syncwarp, never a block barrier, and an SM holds
//     many independent pipeline instances.
//   * Processors compete for the input with one global atomic ticket (Section 2.2):
//     each ticket is a work unit of up to K consecutive parents of one stream.
//   * Each processor runs the non-preemptive scheduler of Section 2.1 over its own
//     pipeline: data queues are shared-memory rings, one per edge; a node fires on an
//     ensemble of <= 32 items gathered from its input ring with consecutive
//     (bank-conflict-free) loads; outputs are compacted with __ballot_sync/__popc.
//   * Enumeration (Section 4): parents open into elements.  Loaded elements are
//     staged from HBM into shared memory by 1-D bulk asynchronous copies (TMA,
//     cp.async.bulk + mbarrier), several tiles ahead of the enumerating node.
//   * Strategy SIGNAL (Sections 3-4): Begin/End signals on a signal ring per edge
//     with the credit protocol of Section 3.1, two-phase firing of Section 3.2 and
//     the ensemble <= credit rule of Section 3.3.
//   * Strategy TAG (Section 2.3 / Section 5): every queued item carries its region
//     tag; ensembles stay full across region boundaries; the aggregate reduces runs
//     of equal tags with a segmented warp scan.
//   * Region offsets: from CSR offsets, or for region lengths by a single-pass
//     decoupled look-back scan (Merrill & Garland 2016) fused into work claiming.
//   * Every wait is bounded (global timer); on expiry the kernel records a status
//     bit and the warp leaves its loop.  No trap, no unbounded spin.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_internal.h"

#include "rs_device.cuh"

// Cycle breakdown, compiled in only for the profiling build (-DRS_PROFILE=1): lane 0
// of each warp adds SM clock cycles per phase into a per-warp shared-memory array,
// folded into the workspace header at exit.
#ifdef RS_PROFILE
#define PROF_NOW() clock64()
#define PROF_ADD(slot, t0)                                   \
    do {                                                     \
        if (lane == 0) M.prof[slot] += clock64() - (t0);     \
    } while (0)
#else
#define PROF_NOW() 0ll
#define PROF_ADD(slot, t0) \
    do {                   \
    } while (0)
#endif
#define LB_AGG (1ull << 62)
#define LB_INCL (2ull << 62)
#define LB_VAL ((1ull << 62) - 1)
#define SIG_END 0x80000000u


// ---------------------------------------------------------------------------
// per-warp (per-processor) state, all warp-uniform, held in registers

struct Warp {
    // queue cursors (free-running).  Edge 0 (enumerate -> node 1) carries element
    // positions of the unit: qh[0] is node 1's next position, qt[0] the enumerated limit.
    // Edges e >= 1 are shared-memory rings of C slots (slot = cursor & (C-1)).
    uint32_t qh[RS_MAX_EDGES], qt[RS_MAX_EDGES];
    // signal rings and the sender's emitted-since-last-signal counter (Section 3.1)
    uint32_t sh[RS_MAX_EDGES], st[RS_MAX_EDGES], em[RS_MAX_EDGES];
    // receiver state per node: current credit counter and current parent (local index)
    uint32_t credit[RS_MAX_STAGES], ctxk[RS_MAX_STAGES];
    // aggregate accumulator (signal strategy), and the second leaf's in a tree
    uint32_t acc_c, acc_m;
    unsigned long long acc_s;
    uint32_t acc2_c, acc2_m;
    unsigned long long acc2_s;
};

struct Smem {
    SArr<unsigned long long> prof, mbar, mmeta, rs, cnt;   // cnt: per node {ensembles, items, signals, firings}
    SArr<uint32_t> tiles, moff, mctx, mpar, rc, rm, qv, sq, scr;
    SArr<uint16_t> qtag;
    SArr<unsigned long long> q64;   // tag strategy: ring slots packing {value, tag}
    SArr<uint32_t> mraw0, mraw1, mmoff0, mmoff1, mctx0, mctx1, mpar0, mpar1;
    SArr<uint32_t> rc2, rm2;           // the second leaf's per-parent accumulators (trees)
    SArr<unsigned long long> rs2;
    __device__ __forceinline__ SArr<uint32_t> raw(uint32_t b) const { return b ? mraw1 : mraw0; }
    __device__ __forceinline__ SArr<uint32_t> moffb(uint32_t b) const { return b ? mmoff1 : mmoff0; }
    __device__ __forceinline__ SArr<uint32_t> ctxb(uint32_t b) const { return b ? mctx1 : mctx0; }
    __device__ __forceinline__ SArr<uint32_t> parb(uint32_t b) const { return b ? mpar1 : mpar0; }
};

// element staging for one unit
struct Stage {
    const uint32_t *elements;
    uint32_t A, B;          // bulk-copied element range [A, B) (absolute, 16-byte aligned)
    uint32_t ntiles, t_issued, t_ready, t_freed;
    uint32_t ready_lim;     // every element below this (absolute) is readable
    uint32_t free_lim;      // node 1 reading at or past this frees the oldest tile
    uint32_t phase;         // bit s = parity of slot s's next completion
    bool tma;
    bool failed;
};

// ---------------------------------------------------------------------------

// A claimed work unit.  UNIT_REGIONS: K whole consecutive parents starting at r0.
// UNIT_MERGE: the elements [j0, j1) of the stream and the parents whose header step
// lies in the unit ([i0, i1)), preceded by the parent continued from an earlier unit
// (the head) when some of its elements fall in [j0, j1).
struct Unit {
    uint32_t ticket, stream, lu, r0, nk;
    uint32_t i0, i1, j0, j1, head_off, first_off, ebase;
    bool valid, skip, has_head;
};

// The next unit, prefetched while the current one runs: its parents' lengths (or CSR
// offsets), context words and ids land in metadata buffer `buf` by cp.async and are
// turned into unit-local offsets once they have landed.
struct Pending {
    Unit u;
    uint32_t buf, phase;     // metadata buffer; mbarrier parity of each buffer (bit b)
    bool scanned, bad, split_tail;
    uint32_t total, E0;      // elements in the unit and absolute index of its first one
    uint32_t tail_off, tail_len;   // absolute offset and length of the last owned parent
};

static_assert(sizeof(Pending) <= 128, "the prefetched unit record must fit its shared-memory slot");

__device__ __forceinline__ Unit describe_unit(const KParams &P, uint32_t ticket)
{
    Unit u;
    u.ticket = ticket;
    u.valid = ticket < P.total_units;
    u.skip = false;
    u.has_head = false;
    u.stream = u.lu = u.r0 = u.nk = 0;
    u.i0 = u.i1 = u.j0 = u.j1 = u.head_off = u.first_off = u.ebase = 0;
    if (!u.valid) return u;
    // stream owning this ticket: the last one whose unit_base <= ticket
    uint32_t lo = 0, hi = P.n_streams - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (P.streams[mid].unit_base <= ticket) lo = mid; else hi = mid - 1;
    }
    const DevStream &S = P.streams[lo];
    u.stream = lo;
    u.lu = ticket - S.unit_base + S.slice_lo;
    if (S.mode == UNIT_MERGE) {
        if (u.lu >= *S.u_count) {   // beyond the units the planner laid out
            u.skip = true;
            return u;
        }
        const UnitRec a = S.rec[u.lu], b = S.rec[u.lu + 1];
        u.i0 = a.i;
        u.j0 = a.j;
        u.head_off = a.head_off;
        u.first_off = a.first_off;
        u.i1 = b.i;
        u.j1 = b.j;
        u.ebase = S.rec[0].j;
        u.has_head = u.j0 < u.first_off;
        u.r0 = u.has_head ? u.i0 - 1 : u.i0;
        u.nk = (u.has_head ? 1u : 0u) + (u.i1 - u.i0);
        if (u.nk > S.D / S.c + 1 || u.j1 < u.j0 || u.i1 < u.i0) u.skip = true;   // inconsistent records
    } else {
        u.r0 = u.lu * S.K;
        if (u.r0 >= S.R) {
            u.skip = true;
            return u;
        }
        u.nk = min(S.K, S.R - u.r0);
    }
    return u;
}

// issue the unit's metadata copies into buffer b; every lane arrives on mmeta[b]
__device__ __forceinline__ void prefetch_meta(const KParams &P, Smem &M, const Unit &u, uint32_t b,
                                              uint32_t lane)
{
    const DevStream &S = P.streams[u.stream];
    if (!u.skip) {
        if (S.mode == UNIT_MERGE) {
            const uint32_t hh = u.has_head ? 1u : 0u, no = u.i1 - u.i0;
            if (S.offsets) {
                for (uint32_t q = lane; q <= no; q += 32) cp_async4(M.raw(b).ptr() + hh + q, S.offsets + u.i0 + q);
            } else {
                for (uint32_t q = lane; q < no; q += 32) cp_async4(M.raw(b).ptr() + hh + q, S.len + u.i0 + q);
            }
        } else if (S.offsets) {
            for (uint32_t k = lane; k <= u.nk; k += 32) cp_async4(M.raw(b).ptr() + k, S.offsets + u.r0 + k);
        } else {
            for (uint32_t k = lane; k < u.nk; k += 32) cp_async4(M.raw(b).ptr() + k, S.len + u.r0 + k);
        }
        if (P.need_ctx && S.ctx)
            for (uint32_t k = lane; k < u.nk; k += 32) cp_async4(M.ctxb(b).ptr() + k, S.ctx + u.r0 + k);
        if (P.need_par && S.parents)
            for (uint32_t k = lane; k < u.nk; k += 32) cp_async4(M.parb(b).ptr() + k, S.parents + u.r0 + k);
    }
    cp_async_arrive(&M.mmeta[b]);
}

// Metadata of `pu` has landed: build the unit-local offsets moff[0..nk] (positions of
// each parent's first element relative to the unit's first element, clamped to the
// unit) and note whether the last owned parent continues into later units.
__device__ __forceinline__ void scan_meta(Pending &pu, const KParams &P, Smem &M, uint32_t lane)
{
    const DevStream &S = P.streams[pu.u.stream];
    const SArr<uint32_t> raw = M.raw(pu.buf);
    const SArr<uint32_t> mo = M.moffb(pu.buf);
    const uint32_t nk = pu.u.nk;
    pu.bad = false;
    pu.split_tail = false;
    pu.tail_off = pu.tail_len = 0;
    if (pu.u.skip) {
        pu.total = 0;
        pu.E0 = 0;
        pu.scanned = true;
        return;
    }
    if (S.mode == UNIT_MERGE) {
        const uint32_t hh = pu.u.has_head ? 1u : 0u, no = pu.u.i1 - pu.u.i0;
        const uint32_t j0 = pu.u.j0, tot = pu.u.j1 - pu.u.j0;
        uint32_t carry = pu.u.first_off;   // absolute offset of the first owned parent
        bool dec = false;
        for (uint32_t b = 0; b < no; b += 32) {
            const uint32_t q = b + lane;
            uint32_t start, L = 0;
            if (S.offsets) {
                // raw and mo share storage: every lane reads its pair before any writes
                start = q < no ? raw[hh + q] : 0u;
                const uint32_t nx = q < no ? raw[hh + q + 1] : 0u;
                L = nx - start;
                dec |= q < no && nx < start;
                __syncwarp();
            } else {
                L = q < no ? raw[hh + q] : 0u;
                const uint32_t incl = warp_incl_scan_u32(L, lane);
                start = carry + incl - L;
                carry += __shfl_sync(FULLMASK, incl, 31);
            }
            if (q < no) {
                const uint32_t rel = start > j0 ? start - j0 : 0u;
                mo[hh + q] = min(rel, tot);
                if (q == no - 1) {
                    pu.tail_off = start;   // lane-local; broadcast below
                    pu.tail_len = L;
                }
            }
        }
        // the last owned parent's offset and length, from the lane that saw it
        if (no > 0) {
            const uint32_t src = (no - 1) & 31u;
            pu.tail_off = __shfl_sync(FULLMASK, pu.tail_off, src);
            pu.tail_len = __shfl_sync(FULLMASK, pu.tail_len, src);
            pu.split_tail = (unsigned long long)pu.tail_off + pu.tail_len > pu.u.j1;
        }
        if (lane == 0) {
            if (hh) mo[0] = 0;
            mo[nk] = tot;
        }
        pu.bad = __any_sync(FULLMASK, dec);
        pu.total = tot;
        pu.E0 = j0;
    } else if (S.offsets) {
        const uint32_t ob = raw[0];
        __syncwarp();   // raw and mo share storage
        bool dec = false;
        for (uint32_t k = lane; k <= nk; k += 32) {
            const uint32_t o = raw[k];
            dec |= o < ob;
            mo[k] = o - ob;
        }
        __syncwarp();
        for (uint32_t k = lane; k < nk; k += 32) dec |= mo[k + 1] < mo[k];
        pu.bad = __any_sync(FULLMASK, dec);
        pu.total = mo[nk];
        pu.E0 = ob;
    } else {
        uint32_t carry = 0;
        for (uint32_t b = 0; b < nk; b += 32) {
            const uint32_t k = b + lane;
            const uint32_t L = (k < nk) ? raw[k] : 0u;
            const uint32_t incl = warp_incl_scan_u32(L, lane);
            if (k < nk) mo[k] = carry + incl - L;
            carry += __shfl_sync(FULLMASK, incl, 31);
        }
        if (lane == 0) mo[nk] = carry;
        pu.total = carry;
        pu.E0 = 0;
    }
    __syncwarp();
    pu.scanned = true;
}

// non-blocking: build the pending unit's offsets if its metadata has landed
__device__ __forceinline__ void poll_next(Pending &pu, const KParams &P, Smem &M, uint32_t lane)
{
    if (!pu.u.valid || pu.scanned) return;
    if (!__all_sync(FULLMASK, mbar_test_wait(&M.mmeta[pu.buf], (pu.phase >> pu.buf) & 1u))) return;
    pu.phase ^= 1u << pu.buf;
    scan_meta(pu, P, M, lane);
}

// A parent processed in pieces: fold this piece's partial aggregate into the slot of
// the unit owning the parent (reductions, no returned value, no fence); the owner also
// records the parent id, and the finalize kernel writes the merged result after this
// kernel.  Integer count / sum / min are associative and commutative, so the result
// does not depend on the order of the pieces.
__device__ __forceinline__ void merge_piece(const DevStream &S, uint32_t r, uint32_t off_abs, uint32_t ebase,
                                            bool owner_piece, uint32_t cnt, unsigned long long sum, uint32_t mn,
                                            uint32_t sink = 0)
{
    const unsigned long long D = S.D, c = S.c;
    const unsigned long long Pr = c * r + (off_abs - ebase);
    // a tree's second leaf merges through a second array of slots
    Slot *sl = &S.slots[(unsigned long long)sink * S.slot_units + Pr / D];
    if (cnt) {
        atomicAdd(&sl->count, cnt);
        atomicAdd(&sl->sum, sum);
        atomicMax(&sl->min_inv, ~mn);
    }
    if (owner_piece) sl->region = r + 1;
}

// ---------------------------------------------------------------------------
// Planner: parent offsets (a single-pass decoupled look-back scan of the lengths, or
// the CSR offsets as given) and the merge-path unit records of every UNIT_MERGE stream.
// One warp per tile of 128 ROUNDS parents (ROUNDS = 8, or 1 when the streams hold few
// regions, so that the tiles are many), read in rounds of 128: in round k lane l
// holds the four parents r_lo + 128 k + 4 l .. + 3, so each load instruction of the warp
// covers one contiguous 512-byte row, and every round's loads are issued before the
// first is used.  Unit u starts inside the merge-path span (P_r, P_r + c + L_r] of the
// parent r that contains u D (P_r = c r + offset of r, c = the stream's parent cost); positions
// are taken relative to the tile, so locating the units costs one 32-bit division per
// lane and round instead of two 64-bit divisions per parent.
// A tile's look-back word holds its flag and its value in one 64-bit word and carries
// nothing else, so it is written and read relaxed (gpu scope): no fence, so publishing
// it never waits for the tile's identity-result stores to drain.


// x / d: a shift when every stream's d is a power of two (POW2, dsh = log2 d, as for
// every tag-strategy unit shape), else a 32-bit division when x < 2^32 (d = c K <= 2^16)
template <bool POW2>
__device__ __forceinline__ unsigned long long plan_div(unsigned long long x, uint32_t d, uint32_t dsh)
{
    if (POW2) return x >> dsh;
    if ((x >> 32) == 0) return (uint32_t)x / d;
    return x / d;
}

// a parent with more unit starts than this has its unit records written by the whole warp
constexpr unsigned long long PLAN_HEAVY = 4;

template <bool POW2, int PLAN_ROUNDS>
__global__ void __launch_bounds__(256) rs_plan_kernel(const __grid_constant__ KParams P)
{
    const uint32_t lane = threadIdx.x & 31u;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&P.hdr->plan_cursor, 1u);
        t = __shfl_sync(FULLMASK, t, 0);
        if (t >= P.plan_tiles) break;
        uint32_t lo = 0, hi = P.n_streams - 1;
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (P.streams[mid].plan_base <= t) lo = mid; else hi = mid - 1;
        }
        const DevStream &S = P.streams[lo];
        const uint32_t D = S.D, c = S.c, dsh = S.dsh;
        const uint32_t tile = t - S.plan_base;
        constexpr uint32_t TILE = 128u * PLAN_ROUNDS;
        const uint32_t r_lo = tile * TILE;
        const uint32_t r_hi = min(r_lo + TILE, S.R);
        const uint32_t base_abs = S.offsets ? S.offsets[0] : 0u;

        // lengths of the lane's four parents in every round (0 past the tile's end)
        uint32_t L[PLAN_ROUNDS][4];
        if (S.offsets) {
#pragma unroll
            for (int k = 0; k < PLAN_ROUNDS; ++k) {
                const uint32_t r = r_lo + 128u * k + 4u * lane;
                uint32_t a[5];
#pragma unroll
                for (int j = 0; j < 5; ++j) a[j] = S.offsets[min(r + j, r_hi)];
#pragma unroll
                for (int j = 0; j < 4; ++j) L[k][j] = a[j + 1] - a[j];
            }
        } else {
            const bool vec = ((uintptr_t)S.len & 15u) == 0;
#pragma unroll
            for (int k = 0; k < PLAN_ROUNDS; ++k) {
                const uint32_t r = r_lo + 128u * k + 4u * lane;
                if (vec && r + 4u <= r_hi) {
                    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(S.len + r));
                    L[k][0] = v.x;
                    L[k][1] = v.y;
                    L[k][2] = v.z;
                    L[k][3] = v.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) L[k][j] = (r + j < r_hi) ? __ldg(S.len + r + j) : 0u;
                }
            }
        }
        // per round: the lane's element count, its inclusive scan, the round total
        uint32_t ls[PLAN_ROUNDS], incl[PLAN_ROUNDS];
        uint32_t tsum = 0;
#pragma unroll
        for (int k = 0; k < PLAN_ROUNDS; ++k) {
            ls[k] = L[k][0] + L[k][1] + L[k][2] + L[k][3];
            incl[k] = warp_incl_scan_u32(ls[k], lane);
            tsum += __shfl_sync(FULLMASK, incl[k], 31);
        }

        uint32_t E = 0;   // offset of parent r_lo relative to the stream's first element
        bool stop = false;
        if (S.offsets) {
            E = S.offsets[r_lo] - base_abs;
        } else {
            unsigned long long *lb = S.plan_lb;
            if (tile == 0) {
                if (lane == 0) st_relaxed_u64(&lb[0], LB_INCL | (unsigned long long)tsum);
            } else {
                if (lane == 0) st_relaxed_u64(&lb[tile], LB_AGG | (unsigned long long)tsum);
                unsigned long long excl = 0;
                int jt = (int)tile - 1;
                unsigned long long t0 = global_ns();
                uint32_t it = 0;
                for (;;) {
                    const int idx = jt - (int)lane;
                    const unsigned long long wv = (idx >= 0) ? ld_relaxed_u64(&lb[idx]) : LB_INCL;
                    const uint32_t flag = (uint32_t)(wv >> 62);
                    const uint32_t notready = __ballot_sync(FULLMASK, flag == 0u);
                    const uint32_t inclm = __ballot_sync(FULLMASK, flag == 2u);
                    const uint32_t stopm = notready | inclm;
                    if (stopm == 0u) {
                        excl += warp_sum_u64(wv & LB_VAL);
                        jt -= 32;
                        continue;
                    }
                    const uint32_t first = __ffs(stopm) - 1;
                    if (notready & (1u << first)) {
                        if ((++it & 15u) == 0 && global_ns() - t0 > P.spin_limit) {
                            if (lane == 0) atomicOr(&P.hdr->status, ST_LOOKBACK_TIMEOUT);
                            stop = true;
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    excl += warp_sum_u64(lane <= first ? (wv & LB_VAL) : 0ull);
                    break;
                }
                E = (uint32_t)excl;
                if (lane == 0) st_relaxed_u64(&lb[tile], LB_INCL | (excl + tsum));
            }
        }
        if (stop) break;

        // unit records.  Frame: X = P - qt D, where qt = floor(P_{r_lo} / D), so the
        // tile starts at X = rem < D and unit qt + m starts at X = m D.
        bool bad = false;
        const unsigned long long Pt = (unsigned long long)c * r_lo + E;
        const unsigned long long qt = plan_div<POW2>(Pt, D, dsh);
        const uint32_t rem = (uint32_t)(Pt - qt * D);
        uint32_t pre = 0;   // elements of the tile before this round
#pragma unroll
        for (int k = 0; k < PLAN_ROUNDS; ++k) {
            const uint32_t rloc = 128u * k + 4u * lane;        // first parent, tile-relative
            const uint32_t r = r_lo + rloc;
            const uint32_t nl = r < r_hi ? min(4u, r_hi - r) : 0u;
            const uint32_t offl = pre + incl[k] - ls[k];        // its element offset in the tile
            const unsigned long long xa = rem + (unsigned long long)c * rloc + offl;
            const unsigned long long xb = xa + (unsigned long long)c * nl + ls[k];
            unsigned long long m = plan_div<POW2>(xa, D, dsh);
            uint32_t heavy = 0;   // bit j: parent j holds more than PLAN_HEAVY unit starts
            if (nl && plan_div<POW2>(xb, D, dsh) > m) {
                unsigned long long x = xa;
                uint32_t off = offl;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if ((uint32_t)j < nl) {
                        const uint32_t Lr = L[k][j];
                        const unsigned long long xn = x + c + Lr;
                        const unsigned long long mend = plan_div<POW2>(xn, D, dsh);
                        if (mend - m > PLAN_HEAVY) {
                            // many units start inside this parent: the warp writes them below
                            heavy |= 1u << j;
                            m = mend;
                        }
                        while ((m + 1) * D <= xn) {
                            ++m;
                            const unsigned long long u = qt + m;
                            if (u > S.slot_units) {   // the whole stream's records (a slice runs fewer units)
                                bad = true;
                                break;
                            }
                            const long long into = (long long)(m * D) - (long long)(x + c);
                            const uint32_t je = (uint32_t)(into <= 0 ? 0 : (into >= (long long)Lr ? Lr : into));
                            const uint32_t oa = base_abs + E + off;
                            UnitRec rc;
                            rc.i = r + j + 1;
                            rc.j = oa + je;
                            rc.head_off = oa;
                            rc.first_off = oa + Lr;
                            S.rec[u] = rc;
                            // tag strategy: a region the unit starts inside is shared by two
                            // units; its identity result is written here, before the pipeline
                            // kernel (every other region's by the one processor that owns it)
                            if (P.plan_fill && je < Lr) {
                                if (P.want_count) S.out_count[r + j] = 0u;
                                if (P.want_sum) S.out_sum[r + j] = 0ull;
                                if (P.want_min) S.out_min[r + j] = 0xFFFFFFFFu;
                            }
                        }
                        x = xn;
                        off += Lr;
                    }
                }
            }
            // the parents with many unit starts (a region much longer than a unit): the
            // whole warp writes each one's records, one per lane, instead of its lane alone
            for (uint32_t hv = __ballot_sync(FULLMASK, heavy != 0); hv; hv &= hv - 1) {
                const uint32_t src = __ffs(hv) - 1;
                const uint32_t hs = __shfl_sync(FULLMASK, heavy, src);
                unsigned long long xj = xa;
                uint32_t offj = offl;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t Lj = L[k][j];
                    const unsigned long long xs = __shfl_sync(FULLMASK, xj, src);
                    const uint32_t os = __shfl_sync(FULLMASK, offj, src);
                    const uint32_t Ls = __shfl_sync(FULLMASK, Lj, src);
                    if ((hs >> j) & 1u) {
                        const unsigned long long m0 = plan_div<POW2>(xs, D, dsh);
                        const unsigned long long me = plan_div<POW2>(xs + c + Ls, D, dsh);
                        const uint32_t rj = r_lo + 128u * k + 4u * src + j;
                        const uint32_t oa = base_abs + E + os;
                        for (unsigned long long mm = m0 + 1 + lane; mm <= me; mm += 32) {
                            const unsigned long long u = qt + mm;
                            if (u > S.slot_units) {
                                bad = true;
                                break;
                            }
                            const long long into = (long long)(mm * D) - (long long)(xs + c);
                            const uint32_t je = (uint32_t)(into <= 0 ? 0 : (into >= (long long)Ls ? Ls : into));
                            UnitRec rc;
                            rc.i = rj + 1;
                            rc.j = oa + je;
                            rc.head_off = oa;
                            rc.first_off = oa + Ls;
                            S.rec[u] = rc;
                            // the first unit start decides whether a unit starts inside the
                            // region (only the last can start exactly at its end)
                            if (P.plan_fill && mm == m0 + 1 && je < Ls) {
                                if (P.want_count) S.out_count[rj] = 0u;
                                if (P.want_sum) S.out_sum[rj] = 0ull;
                                if (P.want_min) S.out_min[rj] = 0xFFFFFFFFu;
                            }
                        }
                    }
                    xj += c + Lj;
                    offj += Lj;
                }
            }
            pre += __shfl_sync(FULLMASK, incl[k], 31);
        }
        if (tile == 0 && lane == 0) {
            UnitRec rc;
            rc.i = 0;
            rc.j = rc.head_off = rc.first_off = base_abs;
            S.rec[0] = rc;
        }
        if (tile + 1 == S.plan_tiles && lane == 0) {
            const uint32_t N = E + tsum;
            const unsigned long long U = ((unsigned long long)c * S.R + N + D - 1) / D;
            if (U > S.slot_units) {
                bad = true;
            } else {
                UnitRec rc;
                rc.i = S.R;
                rc.j = rc.first_off = base_abs + N;
                rc.head_off = base_abs + N;
                S.rec[U] = rc;
                *S.u_count = (uint32_t)U;
            }
        }
        if (__any_sync(FULLMASK, bad) && lane == 0) atomicOr(&P.hdr->status, ST_BAD_INPUT);
    }
}

// ---------------------------------------------------------------------------
// Unit offsets of fixed-parent units (streams of lengths with short regions): unit t holds
// parents [t K, (t + 1) K), so it needs only its first element's offset, the sum of the
// lengths before it.  Pass 1 (one warp per unit) writes each unit's length sum and adds it
// to its group of 32 units; pass 2 (one CTA per stream) scans the group sums; a unit's
// offset is then its group's prefix plus the sums of the units before it in the group,
// one warp-wide read (usum_offset).  No look-back and no unit records.

__global__ void __launch_bounds__(256) rs_unit_sum_kernel(const __grid_constant__ KParams P)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t si = 0; si < P.n_streams; ++si) {
        const DevStream &S = P.streams[si];
        if (!S.usum) continue;
        const bool vec = ((uintptr_t)S.len & 15u) == 0 && (S.K & 3u) == 0;
        for (uint32_t t = gw; t < S.n_units; t += nw) {
            const uint32_t r_lo = t * S.K, r_hi = min(r_lo + S.K, S.R);
            unsigned long long sum = 0;
            // 16-byte loads, eight in flight per lane
            for (uint32_t base = r_lo; base < r_hi; base += 8u * 128u) {
                uint4 v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t r = base + 128u * k + 4u * lane;
                    if (vec && r + 4u <= r_hi) {
                        v[k] = __ldg(reinterpret_cast<const uint4 *>(S.len + r));
                    } else {
                        v[k].x = r < r_hi ? __ldg(S.len + r) : 0u;
                        v[k].y = r + 1 < r_hi ? __ldg(S.len + r + 1) : 0u;
                        v[k].z = r + 2 < r_hi ? __ldg(S.len + r + 2) : 0u;
                        v[k].w = r + 3 < r_hi ? __ldg(S.len + r + 3) : 0u;
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) sum += (unsigned long long)v[k].x + v[k].y + v[k].z + v[k].w;
            }
            sum = warp_sum_u64(sum);
            if (lane == 0) {
                S.usum[t] = (uint32_t)sum;
                atomicAdd(S.usum_grp + (t >> 5), (uint32_t)sum);
            }
        }
    }
}

// pass 2: CTA b turns stream b's group sums into exclusive prefixes (two per thread and
// round, coalesced)
__global__ void __launch_bounds__(1024) rs_unit_scan_kernel(const __grid_constant__ KParams P)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry_s;
    if (blockIdx.x >= P.n_streams) return;
    const DevStream &S = P.streams[blockIdx.x];
    if (!S.usum) return;
    const uint32_t ng = (S.n_units + 31) >> 5, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (uint32_t b = 0; b < ng; b += blockDim.x) {
        const uint32_t i = b + tid;
        const uint32_t v = i < ng ? S.usum_grp[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULLMASK, incl, d);
            if (lane >= (uint32_t)d) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(FULLMASK, w, d);
                if (lane >= (uint32_t)d) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const uint32_t c0 = carry_s;
        if (i < ng) S.usum_grp[i] = c0 + incl - v + (warp ? wsum[warp - 1] : 0u);
        __syncthreads();
        if (tid == 0) carry_s = c0 + wsum[31];
        __syncthreads();
    }
}

int rs_launch_unit_offsets(const KParams &P, int grid, void *stream)
{
    void *args[] = {(void *)&P};
    cudaError_t e = cudaLaunchKernel((const void *)rs_unit_sum_kernel, dim3(grid), dim3(256), args, 0,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) return (int)e;
    e = cudaLaunchKernel((const void *)rs_unit_scan_kernel, dim3(P.n_streams), dim3(1024), args, 0,
                         (cudaStream_t)stream);
    return (int)e;
}

// ---------------------------------------------------------------------------
// Element staging: bulk copies (TMA) of the unit's elements into a ring of NT tiles of
// TE elements in the processor's shared memory, each tile's arrival counted on its own
// mbarrier.

__device__ __forceinline__ void tiles_issue(const KParams &P, Smem &M, Stage &g, uint32_t lane)
{
    const uint32_t TE = P.TE, NT = P.NT;
    while (g.t_issued < g.ntiles && g.t_issued < g.t_freed + NT) {
        uint32_t t = g.t_issued;
        uint32_t start = g.A + t * TE;
        uint32_t cnt = min(TE, g.B - start);
        uint32_t slot = t & (NT - 1);
        if (lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&M.mbar[slot], cnt * 4u);
            bulk_g2s(M.tiles.ptr() + slot * TE, g.elements + start, cnt * 4u, &M.mbar[slot]);
        }
        g.t_issued++;
    }
}

// make the staged elements below e_hi (absolute) readable; false (with the status bit
// set) when a copy has not landed within the spin limit
__device__ __forceinline__ bool tiles_ready(const KParams &P, Smem &M, Stage &g, uint32_t lane, uint32_t e_hi)
{
    if (!g.tma) return true;
    const uint32_t TE = P.TE, NT = P.NT;
    uint32_t lim = min(e_hi, g.B);
    while (g.t_ready < g.t_issued && g.A + g.t_ready * TE < lim) {
        uint32_t slot = g.t_ready & (NT - 1);
        uint32_t par = (g.phase >> slot) & 1u;
        if (!mbar_try_wait(&M.mbar[slot], par)) {
            const long long pt = PROF_NOW();
            unsigned long long t0 = global_ns();
            uint32_t it = 0;
            while (!mbar_try_wait(&M.mbar[slot], par)) {
                if ((++it & 63u) == 0 && global_ns() - t0 > P.spin_limit) {
                    g.failed = true;
                    break;
                }
            }
            PROF_ADD(PF_TILEWAIT, pt);
            (void)pt;
            if (g.failed) {
                if (lane == 0) atomicOr(&P.hdr->status, ST_COPY_TIMEOUT);
                return false;
            }
        }
        g.phase ^= 1u << slot;
        g.t_ready++;
    }
    g.ready_lim = (g.t_ready >= g.ntiles) ? 0xFFFFFFFFu : g.A + g.t_ready * TE;
    return true;
}

// every element below e_read (absolute) has been consumed: recycle tiles, refill them
__device__ __forceinline__ void tiles_release(const KParams &P, Smem &M, Stage &g, uint32_t lane, uint32_t e_read)
{
    if (!g.tma) return;
    const uint32_t TE = P.TE;
    bool freed = false;
    while (g.t_freed < g.t_ready && g.A + (g.t_freed + 1) * TE <= e_read) {
        g.t_freed++;
        freed = true;
    }
    g.free_lim = g.A + (g.t_freed + 1) * TE;
    if (freed) {
        __syncwarp();
        tiles_issue(P, M, g, lane);
    }
}

// the parent containing unit-local position pos (< moff[nk]), searching from `from`
// (which starts at or before pos); empty parents are skipped
__device__ __forceinline__ uint32_t parent_at(const Smem &M, uint32_t from, uint32_t pos, uint32_t nk,
                                              uint32_t lane)
{
    uint32_t k = from;
    for (;;) {
        const uint32_t e2 = M.moff[min(k + lane + 1, nk)];
        const uint32_t cnt = __popc(__ballot_sync(FULLMASK, e2 <= pos));
        k += cnt;
        if (cnt < 32) break;
    }
    return k;
}


// per-node counters live in the processor's shared memory (lane 0 updates them)
#define CNT_ADD(node, field, v)                                       \
    do {                                                              \
        if (lane == 0) M.cnt[4 * (node) + (field)] += (unsigned long long)(v); \
    } while (0)

template <int STRAT, int V, class S, bool MIX = false, int UM = -1>
struct Proc {
    static constexpr uint32_t W = 32u * V;   // ensemble width (items per firing)
    const KParams &P;
    Smem &M;
    Warp &w;
    Stage &g;
    const uint32_t lane;
    Pending *nxt;    // the prefetched next unit, in this processor's shared memory
    bool nxt_open;   // its metadata still has to be turned into offsets
    // current unit
    uint32_t nk, total, E0;
    uint32_t ek;     // enumerate: next parent to open (signal strategy)
    uint32_t ek1;    // node 1: parent containing its next position (tag strategy)
    bool stop;
    // the unit's stream and its first parent (the emit sink addresses outputs by region)
    const DevStream *ds = nullptr;
    uint32_t r0 = 0;

    __device__ __forceinline__ Proc(const KParams &P_, Smem &M_, Warp &w_, Stage &g_, uint32_t lane_)
        : P(P_), M(M_), w(w_), g(g_), lane(lane_), nk(0), total(0), E0(0), ek(0), ek1(0), stop(false)
    {
        nxt = nullptr;
        nxt_open = false;
    }

    __device__ __forceinline__ int nst() const { return S::generic ? P.n_stages : S::n; }
    template <int I>
    __device__ __forceinline__ uint32_t op() const
    {
        if constexpr (S::generic) return P.st[I].op;
        else return (uint32_t)S::template op<I>();
    }

    // How region boundaries reach node c over its input edge, and the topology.  Without
    // MIX every edge carries signals (tags for STRAT == TAG) along a linear pipeline; the
    // per-edge kernel (MIX) reads both from the parameters, except that a per-edge kernel
    // compiled for one mode on every edge (UM >= 0) has it at compile time.
    __device__ __forceinline__ uint32_t emode(int c) const
    {
        if constexpr (MIX) {
            if constexpr (UM >= 0) return (uint32_t)UM;
            else return P.emode[c];
        } else {
            return STRAT == RS_STRATEGY_TAG ? EM_TAG : EM_SIG;
        }
    }
    // The topology (MIX only): node i's children, whether it is a sink and which, its
    // producer.  A specialised per-edge kernel serves linear pipelines only (the host
    // checks), so there they are compile-time facts and the loops over children fold.
    static constexpr bool LIN = MIX && !S::generic;
    __device__ __forceinline__ uint32_t kids(int i) const
    {
        if constexpr (LIN) return i + 1 < S::n ? (1u << (i + 1)) : 0u;
        else return P.kids[i];
    }
    __device__ __forceinline__ bool is_sink(int i) const
    {
        if constexpr (LIN) return i == S::n - 1;
        else return P.sink_of[i] != 0xFFu;
    }
    __device__ __forceinline__ uint32_t sink_idx(int i) const
    {
        if constexpr (LIN) return 0u;
        else return P.sink_of[i];
    }
    __device__ __forceinline__ uint32_t up_of(int i) const
    {
        if constexpr (LIN) return (uint32_t)(i - 1);
        else return P.up[i];
    }
    // the per-parent accumulators of leaf q (a tree has two)
    __device__ __forceinline__ SArr<uint32_t> rcq(uint32_t q) const { return q ? M.rc2 : M.rc; }
    __device__ __forceinline__ SArr<unsigned long long> rsq(uint32_t q) const { return q ? M.rs2 : M.rs; }
    __device__ __forceinline__ SArr<uint32_t> rmq(uint32_t q) const { return q ? M.rm2 : M.rm; }

    // ---- tile staging ----
    __device__ __forceinline__ void issue_tiles() { tiles_issue(P, M, g, lane); }
    __device__ __forceinline__ void ensure_ready(uint32_t e_hi)
    {
        if (!tiles_ready(P, M, g, lane, e_hi)) stop = true;
    }
    __device__ __forceinline__ void release_below(uint32_t e_read) { tiles_release(P, M, g, lane, e_read); }

    __device__ __forceinline__ uint32_t load_elem(uint32_t e) const
    {
        if (g.tma && e < g.B) return M.tiles[(e - g.A) & (P.NT * P.TE - 1)];
        return __ldg(g.elements + e);
    }

    __device__ __forceinline__ void finish_tiles()
    {
        if (!g.tma) return;
        ensure_ready(0xFFFFFFFFu);
        g.t_freed = g.t_ready;
    }

    // ---- signal rings: slot j of edge e holds {word, credit} ----
    __device__ __forceinline__ uint32_t sidx(int e, uint32_t cursor) const
    {
        return 2u * (e * P.SC + (cursor & (P.SC - 1)));
    }

    // ---- enumeration (Section 4.2) ----
    // Signal strategy: for each parent k, Begin(k), its L_k element positions, End(k).
    // A batch of up to 32 parents is emitted at once, lane j handling parent ek + j; the
    // credits follow the sender rules of Section 3.1 exactly as if emitted one by one:
    // the first signal gets |Q| if the signal queue was empty, else the items emitted
    // since the previous signal; a Begin after an End carries 0; End(k) carries L_k.
    __device__ __forceinline__ void enum_signal()
    {
        const uint32_t SC = P.SC;
        while (ek < nk) {
            uint32_t room = (SC - (w.st[0] - w.sh[0])) >> 1;
            uint32_t m = min(min(32u, room), nk - ek);
            if (m == 0) break;
            uint32_t k = ek + lane;
            bool mine = lane < m;
            uint32_t L = mine ? (M.moff[k + 1] - M.moff[k]) : 0u;
            uint32_t Lsum = __reduce_add_sync(FULLMASK, L);
            // enumeration ensembles: each parent's positions are cut into W-wide pieces
            const uint32_t ens = __reduce_add_sync(FULLMASK, (L + W - 1) / W);
            uint32_t first = (w.sh[0] == w.st[0]) ? (w.qt[0] - w.qh[0]) : w.em[0];
            if (mine) {
                uint32_t b = sidx(0, w.st[0] + 2 * lane), e = sidx(0, w.st[0] + 2 * lane + 1);
                M.sq[b] = k;
                M.sq[b + 1] = lane == 0 ? first : 0u;
                M.sq[e] = SIG_END | k;
                M.sq[e + 1] = L;
            }
            __syncwarp();
            w.st[0] += 2 * m;
            w.qt[0] += Lsum;
            w.em[0] = 0;
            ek += m;
            CNT_ADD(0, 0, ens);
            CNT_ADD(0, 1, Lsum);
        }
    }

    // ---- parent of each of the positions [P0, P0+n) (tag strategy, node 1) ----
    // ek1 contains P0.  Every non-empty parent starting inside the window marks its
    // start; each lane takes the last mark at or before its position.
    __device__ __forceinline__ uint32_t assign_parents(uint32_t P0, uint32_t n)
    {
        uint32_t end0 = M.moff[ek1 + 1];
        if (end0 >= P0 + n) return ek1;   // the whole window lies in one parent
        uint32_t D = 0;
        uint32_t base = ek1 + 1;
        for (;;) {
            uint32_t k = base + lane;
            bool in = k < nk;
            uint32_t st = in ? M.moff[k] : total;
            uint32_t en = in ? M.moff[k + 1] : total;
            bool mark = in && en > st && st < P0 + n;
            if (mark) M.scr[st - P0] = k;
            D |= __reduce_or_sync(FULLMASK, mark ? (1u << (st - P0)) : 0u);
            uint32_t st31 = __shfl_sync(FULLMASK, st, 31);
            if (!(base + 32 < nk && st31 < P0 + n)) break;
            base += 32;
        }
        __syncwarp();
        uint32_t mk = D & ((2u << lane) - 1u);
        uint32_t myk = mk ? M.scr[31 - __clz(mk)] : ek1;
        __syncwarp();
        return myk;
    }

    // advance ek1 from parent `from` to the parent containing position pos (< total)
    __device__ __forceinline__ void advance_ek1(uint32_t from, uint32_t pos) { ek1 = parent_at(M, from, pos, nk, lane); }

    // ---- gather one ensemble of node I: x[s], k[s] for lane's items 32 s + lane ----
    // returns true when every item of the ensemble has the same parent (k[0])
    // F: a full ensemble (take == W), compiled without per-item guards
    template <int I, bool F>
    __device__ __forceinline__ bool gather(uint32_t take, uint32_t (&x)[V], uint32_t (&k)[V])
    {
        if (F) take = W;
        bool uni = true;
        if constexpr (I == 1) {
            const uint32_t q0 = w.qh[0];
            const bool hashed = op<0>() == D_ENUM_HASH;
            // parent of every item
            if (emode(1) == EM_TAG) {
                const uint32_t end0 = M.moff[ek1 + 1];
                if (end0 >= q0 + take) {
                    // the whole ensemble lies in one parent
#pragma unroll
                    for (int s = 0; s < V; ++s) k[s] = ek1;
                    if (end0 == q0 + take && q0 + take < total) advance_ek1(ek1, q0 + take);
                } else {
                    uni = false;
#pragma unroll
                    for (int s = 0; s < V; ++s) {
                        const uint32_t sb = 32u * s;
                        k[s] = ek1;
                        if (sb < take) {
                            const uint32_t n = min(32u, take - sb);
                            const uint32_t kk = assign_parents(q0 + sb, n);
                            const uint32_t klast = __shfl_sync(FULLMASK, kk, n - 1);
                            if (q0 + sb + n < total && M.moff[klast + 1] <= q0 + sb + n)
                                advance_ek1(klast, q0 + sb + n);
                            else
                                ek1 = klast;
                            k[s] = kk;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < V; ++s) k[s] = w.ctxk[1];
            }
            // the elements themselves (getItem(i) of Figure 4)
            if (hashed) {
#pragma unroll
                for (int s = 0; s < V; ++s) {
                    const uint32_t q = 32u * s + lane;
                    x[s] = (F || q < take) ? fmix32(M.mpar[k[s]] ^ fmix32((q0 + q - M.moff[k[s]]) ^ RS_GOLD)) : 0u;
                }
            } else {
                const uint32_t e_lo = E0 + q0;
                if (e_lo + take > g.ready_lim) ensure_ready(e_lo + take);
                if (g.tma && e_lo + take <= g.B) {
                    const uint32_t base = e_lo - g.A, mask = P.NT * P.TE - 1;
#pragma unroll
                    for (int s = 0; s < V; ++s) {
                        const uint32_t q = 32u * s + lane;
                        x[s] = (F || q < take) ? M.tiles[(base + q) & mask] : 0u;
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < V; ++s) {
                        const uint32_t q = 32u * s + lane;
                        x[s] = q < take ? load_elem(e_lo + q) : 0u;
                    }
                }
            }
        } else {
            const uint32_t C = P.C, cm = C - 1;
            const uint32_t rb = (I - 2) * C;   // input edge I-1 is ring I-2
            const uint32_t h = w.qh[I - 1];
            if (emode(I) == EM_TAG) {
                // tags are non-decreasing along a queue: equal ends mean one parent
                const uint32_t k0 = M.qtag[rb + (h & cm)];
                uni = k0 == M.qtag[rb + ((h + take - 1) & cm)];
#pragma unroll
                for (int s = 0; s < V; ++s) k[s] = k0;
            } else {
#pragma unroll
                for (int s = 0; s < V; ++s) k[s] = w.ctxk[I];
            }
#pragma unroll
            for (int s = 0; s < V; ++s) {
                const uint32_t q = 32u * s + lane;
                x[s] = 0;
                if (F || q < take) {
                    const uint32_t slot = rb + ((h + q) & cm);
                    x[s] = M.qv[slot];
                    if (emode(I) == EM_TAG && !uni) k[s] = M.qtag[slot];
                }
            }
        }
        return uni;
    }

    // ---- one ensemble through element stage I (filter / map / expand) ----
    template <int I, bool F>
    __device__ __forceinline__ void element_stage(uint32_t take)
    {
        if constexpr (MIX) {
            uint32_t x[V], k[V], bal[V];
            const bool uni = gather<I, F>(take, x, k);
            (void)mix_stage<I>(x, k, uni, take, bal);
            return;
        }
        if (F) take = W;
        const DevStage &sd = P.st[I];
        const uint32_t opc = op<I>();
        const uint32_t C = P.C, cm = C - 1;
        const uint32_t orb = (I - 1) * C;   // output edge I is ring I-1
        uint32_t x[V], k[V];
        const long long pg = PROF_NOW();
        (void)pg;
        const bool uni = gather<I, F>(take, x, k);
        if constexpr (I == 1) {
#ifdef RS_PROFILE
            // make the gather's loads complete before reading the clock
            uint32_t sink = 0;
            for (int s2 = 0; s2 < V; ++s2) sink ^= x[s2];
            if (sink == 0xFFFFFFFFu && lane == 99) M.scr[0] = sink;
#endif
            PROF_ADD(PF_GATHER1, pg);
        }
        if (opc == D_EXPAND) {
#pragma unroll
            for (int s = 0; s < V; ++s) {
                if (32u * s < take) {
                    const bool act = 32u * s + lane < take;
                    uint32_t nout = act ? fmix32(x[s] ^ sd.c0) % (sd.fanout + 1u) : 0u;
                    uint32_t incl = warp_incl_scan_u32(nout, lane);
                    uint32_t tot = __shfl_sync(FULLMASK, incl, 31);
                    uint32_t base = w.qt[I] + incl - nout;
                    for (uint32_t j = 0; j < nout; ++j) {
                        uint32_t y = fmix32(x[s] ^ fmix32((sd.p0 + 1u + j) ^ RS_GOLD));
                        uint32_t slot = orb + ((base + j) & cm);
                        M.qv[slot] = y;
                        if (STRAT == RS_STRATEGY_TAG) M.qtag[slot] = (uint16_t)k[s];
                    }
                    w.qt[I] += tot;
                    w.em[I] += tot;
                }
            }
            return;
        }
        const long long pc = PROF_NOW();
        (void)pc;
        bool keep[V];
        uint32_t y[V];
        // the parent's context word (t_r) or hashed id, once per ensemble when uniform
        uint32_t cu = 0;
        if (opc == D_FILT_HASH_CTX && uni) cu = M.mctx[k[0]];
        if (opc == D_FILT_WEIGHT && uni) cu = fmix32(M.mpar[k[0]] ^ sd.c0);
#pragma unroll
        for (int s = 0; s < V; ++s) {
            const uint32_t xs = x[s];
            bool kp;
            uint32_t ys = xs;
            switch (opc) {
            case D_FILT_MASK: kp = (xs & sd.p0) == sd.p1; break;
            case D_FILT_MOD: kp = (xs % sd.p0) == sd.p1; break;
            case D_FILT_HASH_CTX: kp = (fmix32(xs ^ sd.c0) ^ (uni ? cu : M.mctx[k[s]])) < sd.p1; break;
            case D_FILT_WEIGHT:
                kp = fmix32(xs ^ sd.c0) < (uni ? cu : fmix32(M.mpar[k[s]] ^ sd.c0));
                break;
            case D_MAP_MULADD: ys = xs * sd.p0 + sd.p1; kp = true; break;
            default: kp = false; break;
            }
            keep[s] = kp && (F || 32u * s + lane < take);
            y[s] = ys;
        }
#ifdef RS_PROFILE
        {
            uint32_t sink = 0;
            for (int s2 = 0; s2 < V; ++s2) sink ^= keep[s2] ? y[s2] : 0u;
            if (sink == 0xFFFFFFFFu && lane == 99) M.scr[0] = sink;
        }
#endif
        PROF_ADD(PF_COMPUTE, pc);
        const long long pp = PROF_NOW();
        (void)pp;
        const uint32_t lt = lanemask_lt();
        // all ballots first, then every kept item's slot from one running base
        uint32_t bal[V];
#pragma unroll
        for (int s = 0; s < V; ++s) bal[s] = (F || 32u * s < take) ? __ballot_sync(FULLMASK, keep[s]) : 0u;
        uint32_t base = w.qt[I];
#pragma unroll
        for (int s = 0; s < V; ++s) {
            if (keep[s]) {
                const uint32_t slot = orb + ((base + __popc(bal[s] & lt)) & cm);
                M.qv[slot] = y[s];
                if (STRAT == RS_STRATEGY_TAG) M.qtag[slot] = (uint16_t)k[s];
            }
            base += __popc(bal[s]);
        }
        w.em[I] += base - w.qt[I];
        w.qt[I] = base;
        PROF_ADD(PF_COMPACT, pp);
    }

    // ---- one ensemble into the emit sink (Section 4: survivors stripped of their
    // parent): the ensemble belongs to one parent (Section 3.3), so one atomic add on the
    // region's count claims its positions in the region's segment of the value array ----
    __device__ __forceinline__ void emit_ensemble(const uint32_t (&x)[V], uint32_t take)
    {
        const uint32_t r = r0 + w.ctxk[nst() - 1];
        uint32_t base = 0, seg = 0;
        if (lane == 0) {
            base = atomicAdd(ds->out_count + r, take);
            seg = __ldg(ds->offsets + r) - __ldg(ds->offsets);
        }
        base = __shfl_sync(FULLMASK, base, 0);
        seg = __shfl_sync(FULLMASK, seg, 0);
        const unsigned long long b = (unsigned long long)P.emit_f * seg + base;
#pragma unroll
        for (int s = 0; s < V; ++s) {
            const uint32_t q = 32u * s + lane;
            if (q < take) {
                if (b + q < ds->out_values_len) ds->out_values[b + q] = x[s];
                else atomicOr(&P.hdr->status, ST_BAD_INPUT);
            }
        }
    }

    // ---- one ensemble into the aggregate (node I = n-1) ----
    template <int I, bool F>
    __device__ __forceinline__ void aggregate(uint32_t take)
    {
        if (F) take = W;
        uint32_t x[V], k[V];
        if constexpr (MIX) {
            const bool uni = gather<I, F>(take, x, k);
            mix_sink<I>(x, k, uni, take);
            return;
        }
        (void)gather<I, F>(take, x, k);
        if constexpr (STRAT == RS_STRATEGY_SIGNAL) {
            if (S::generic && P.emit) {
                emit_ensemble(x, take);
                return;
            }
            // the whole ensemble belongs to the current parent (Section 3.3)
            unsigned long long part = 0;
            uint32_t mn = 0xFFFFFFFFu;
#pragma unroll
            for (int s = 0; s < V; ++s) {
                if (32u * s + lane < take) {
                    part += x[s];
                    mn = min(mn, x[s]);
                }
            }
            uint32_t lo = __reduce_add_sync(FULLMASK, (uint32_t)(part & 0xFFFFu));
            uint32_t hi = __reduce_add_sync(FULLMASK, (uint32_t)(part >> 16));
            w.acc_c += take;
            w.acc_s += ((unsigned long long)hi << 16) + lo;
            w.acc_m = min(w.acc_m, __reduce_min_sync(FULLMASK, mn));
            return;
        } else {
#pragma unroll
        for (int s = 0; s < V; ++s) {
            const uint32_t sb = 32u * s;
            if (sb >= take) break;
            const uint32_t n = min(32u, take - sb);
            const bool act = lane < n;
            const uint32_t v = act ? x[s] : 0u;
            const uint32_t kk = act ? k[s] : 0xFFFFFFFFu;
            const uint32_t k0 = __shfl_sync(FULLMASK, kk, 0);
            const uint32_t kl = __shfl_sync(FULLMASK, kk, n - 1);
            if (k0 == kl) {
                // one parent in the whole sub-ensemble (tags are non-decreasing)
                unsigned long long sm = warp_sum_u32_wide(v);
                uint32_t mn = __reduce_min_sync(FULLMASK, act ? v : 0xFFFFFFFFu);
                if (lane == 0) {
                    M.rc[k0] += n;
                    M.rs[k0] += sm;
                    if (P.want_min) M.rm[k0] = min(M.rm[k0], mn);
                }
            } else {
                uint32_t kprev = __shfl_up_sync(FULLMASK, kk, 1);
                uint32_t knext = __shfl_down_sync(FULLMASK, kk, 1);
                bool head = (lane == 0) || (kk != kprev);
                bool tail = (lane == 31) || (kk != knext);
                uint32_t heads = __ballot_sync(FULLMASK, head);
                uint32_t hl = 31 - __clz(heads & ((2u << lane) - 1u));
                unsigned long long ps = v;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    unsigned long long t = __shfl_up_sync(FULLMASK, ps, d);
                    if (lane >= (uint32_t)d) ps += t;
                }
                unsigned long long before = __shfl_sync(FULLMASK, ps, hl > 0 ? hl - 1 : 0);
                if (hl == 0) before = 0;
                uint32_t m = act ? v : 0xFFFFFFFFu;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    uint32_t t = __shfl_up_sync(FULLMASK, m, d);
                    if (lane >= (uint32_t)d && lane - d >= hl) m = min(m, t);
                }
                if (act && tail) {
                    M.rc[kk] += lane - hl + 1;
                    M.rs[kk] += ps - before;
                    if (P.want_min) M.rm[kk] = min(M.rm[kk], m);
                }
            }
            __syncwarp();
        }
        }
    }

    // ---- signal phase of node I (Section 3.2), receiver rule 2b ----
    // While the counter is 0: if the head signal carries credit, move it to the counter
    // and stop; otherwise consume the run of zero-credit signals at the head, up to 32
    // at a time, one lane each.  Consuming a run in parallel gives the same state as
    // consuming it one by one: the parent context is the last Begin's; the aggregate's
    // End(k) reports the running accumulator unless a Begin precedes it in the run (an
    // empty parent: identity); forwarded signals carry fresh credit by the sender rules
    // (the first one |Q_out| or the items emitted since the last signal, the rest 0).
    template <int I>
    __device__ __forceinline__ bool signal_phase(bool last)
    {
        if constexpr (MIX) return mix_signal_phase<I>(last);
        const uint32_t SC = P.SC;
        bool progress = false;
        while (w.credit[I] == 0 && w.sh[I - 1] != w.st[I - 1]) {
            const uint32_t h = sidx(I - 1, w.sh[I - 1]);
            const uint32_t hcr = M.sq[h + 1];
            if (hcr > 0) {
                w.credit[I] = hcr;
                __syncwarp();
                if (lane == 0) M.sq[h + 1] = 0;
                __syncwarp();
                progress = true;
                break;
            }
            uint32_t room = 32u;
            if constexpr (S::template maybe_elem<I>()) {
                if (!last) room = SC - (w.st[I] - w.sh[I]);
            }
            const uint32_t mmax = min(min(32u, w.st[I - 1] - w.sh[I - 1]), room);
            if (mmax == 0) break;
            const bool in = lane < mmax;
            const uint32_t j = sidx(I - 1, w.sh[I - 1] + lane);
            const uint32_t word = in ? M.sq[j] : 0u;
            const uint32_t cr = in ? M.sq[j + 1] : 1u;
            const uint32_t nz = __ballot_sync(FULLMASK, cr != 0u);
            const uint32_t m = nz ? (uint32_t)(__ffs(nz) - 1) : 32u;
            const bool mine = lane < m;
            const bool is_begin = mine && !(word & SIG_END);
            const uint32_t begins = __ballot_sync(FULLMASK, is_begin);
            if (begins) {
                const uint32_t lb = 31 - __clz(begins);
                w.ctxk[I] = __shfl_sync(FULLMASK, word, lb);
            }
            if (last) {
                if (mine && (word & SIG_END)) {
                    const uint32_t kk = word & ~SIG_END;
                    const bool fresh = (begins & lanemask_lt()) != 0u;
                    M.rc[kk] = fresh ? 0u : w.acc_c;
                    M.rs[kk] = fresh ? 0ull : w.acc_s;
                    if (P.want_min) M.rm[kk] = fresh ? 0xFFFFFFFFu : w.acc_m;
                }
                if (begins) {
                    w.acc_c = 0;
                    w.acc_s = 0;
                    w.acc_m = 0xFFFFFFFFu;
                }
            } else {
                if constexpr (S::template maybe_elem<I>()) {
                    const uint32_t c0 = (w.sh[I] == w.st[I]) ? (w.qt[I] - w.qh[I]) : w.em[I];
                    if (mine) {
                        const uint32_t o = sidx(I, w.st[I] + lane);
                        M.sq[o] = word;
                        M.sq[o + 1] = lane == 0 ? c0 : 0u;
                    }
                    w.st[I] += m;
                    w.em[I] = 0;
                }
            }
            __syncwarp();
            w.sh[I - 1] += m;
            CNT_ADD(I, 2, m);
            progress = true;
        }
        return progress;
    }

    // ---- fire node I (1 <= I < n) ----
    // drain: nothing more will arrive on node I's input (everything upstream is done),
    // so partial ensembles are fired; otherwise only full ensembles, or ensembles cut
    // by a pending signal's credit.
    template <int I>
    __device__ __forceinline__ void fire(bool drain)
    {
        if constexpr (S::template present<I>()) {
            if (I >= nst() || stop) return;
            const long long pt = PROF_NOW();
            (void)pt;
            if constexpr (MIX) mix_fire<I>(drain);
            else fire_body<I>(drain);
            PROF_ADD(PF_NODE0 + I, pt);
        }
    }

    template <int I>
    __device__ __forceinline__ void fire_body(bool drain)
    {
        constexpr bool can_push = S::template maybe_elem<I>();
        const bool last = !can_push || (I == nst() - 1);
        // a-priori maximum outputs per input (Section 3.2): 1 unless the stage expands
        const uint32_t fan = (S::generic || S::template op<I>() == (int)D_EXPAND) ? P.st[I].fanout : 1u;
        bool fired = false;
        uint32_t n_ens = 0, n_items = 0;   // folded into the shared counters once per firing
        for (;;) {
            const bool sigp = (STRAT == RS_STRATEGY_SIGNAL) && (w.sh[I - 1] != w.st[I - 1]);
            const uint32_t avail0 = w.qt[I - 1] - w.qh[I - 1];
            if (!(drain ? (avail0 > 0 || sigp) : (avail0 >= W || sigp))) break;
            if (!fired) {
                CNT_ADD(I, 3, 1);
                fired = true;
            }
            bool progress = false;
            // data phase: min(queued, downstream space, credit while a signal is pending)
            for (;;) {
                uint32_t want = min(w.qt[I - 1] - w.qh[I - 1], W);
                if (sigp) want = min(want, w.credit[I]);
                uint32_t take = want;
                if constexpr (can_push) {
                    if (!last) {
                        const uint32_t space = P.C - (w.qt[I] - w.qh[I]);
                        take = min(take, fan == 1u ? space : space / fan);
                    }
                }
                if (take == 0) break;
                if (take < want) break;                       // wait for downstream space
                if (!drain && !sigp && take < W) break;       // wait for a full ensemble
                if (last) {
                    if constexpr (S::template maybe_last<I>()) {
                        aggregate<I, false>(take);
                    }
                } else {
                    if constexpr (can_push) {
                        element_stage<I, false>(take);
                    }
                }
                if (stop) break;
                __syncwarp();
                w.qh[I - 1] += take;
                if (sigp) w.credit[I] -= take;
                n_ens++;
                n_items += take;
                progress = true;
                if constexpr (I == 1) {
                    if (op<0>() == D_ENUM_LOAD && E0 + w.qh[0] >= g.free_lim) {
                        const long long pt2 = PROF_NOW();
                        (void)pt2;
                        release_below(E0 + w.qh[0]);
                        PROF_ADD(PF_TILES, pt2);
                    }
                }
            }
            if (stop) break;
            if (STRAT == RS_STRATEGY_SIGNAL) progress |= signal_phase<I>(last);
            if (!progress) break;
        }
        if (n_ens) {
            CNT_ADD(I, 0, n_ens);
            CNT_ADD(I, 1, n_items);
        }
    }

    __device__ __forceinline__ bool edge_empty(int e) const
    {
        return (w.qh[e] == w.qt[e]) && (w.sh[e] == w.st[e]);
    }

    // edge_empty for a run-time edge index, by a compile-time select over the edges (so the
    // queue cursors stay in registers)
    __device__ __forceinline__ bool edge_empty_at(uint32_t e) const
    {
        bool r = true;
#pragma unroll
        for (int j = 0; j < RS_MAX_EDGES; ++j)
            if ((uint32_t)j == e) r = edge_empty(j);
        return r;
    }

    // =====================================================================================
    // The per-edge kernel (MIX): every edge carries region boundaries its own way (EM_SIG,
    // EM_TAG or EM_LANE, as the parameters say) and a node may feed several children (a
    // tree, Figure 1(b): its output stream, and with it every region boundary, is
    // replicated to each child).  Tags never turn back into signals: below an EM_TAG edge
    // every edge is EM_TAG (checked by the host).

    // node I's operation on one ensemble (per-item contexts unless uni) and the push of its
    // outputs to every child's ring, with tags for the children fed by tags.  bal[s] is the
    // ballot of slot s's kept items (fan-out 1); returns the outputs pushed.
    template <int I>
    __device__ __forceinline__ uint32_t mix_stage(const uint32_t (&x)[V], const uint32_t (&k)[V], bool uni,
                                                  uint32_t take, uint32_t (&bal)[V])
    {
        const DevStage &sd = P.st[I];
        const uint32_t opc = op<I>();
        const uint32_t C = P.C, cm = C - 1;
        const uint32_t km = kids(I);
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int s = 0; s < V; ++s) bal[s] = 0;
        if (opc == D_EXPAND) {
            uint32_t total = 0;
#pragma unroll
            for (int s = 0; s < V; ++s) {
                if (32u * s < take) {
                    const bool act = 32u * s + lane < take;
                    const uint32_t nout = act ? fmix32(x[s] ^ sd.c0) % (sd.fanout + 1u) : 0u;
                    const uint32_t incl = warp_incl_scan_u32(nout, lane);
                    const uint32_t tot = __shfl_sync(FULLMASK, incl, 31);
#pragma unroll
                    for (int c = 2; c < RS_MAX_STAGES; ++c) {
                        if (!(km & (1u << c))) continue;
                        const uint32_t orb = (c - 2) * C;
                        const bool tagc = emode(c) == EM_TAG;
                        const uint32_t base = w.qt[c - 1] + incl - nout;
                        for (uint32_t j = 0; j < nout; ++j) {
                            const uint32_t slot = orb + ((base + j) & cm);
                            M.qv[slot] = fmix32(x[s] ^ fmix32((sd.p0 + 1u + j) ^ RS_GOLD));
                            if (tagc) M.qtag[slot] = (uint16_t)k[s];
                        }
                        w.qt[c - 1] += tot;
                        w.em[c - 1] += tot;
                    }
                    total += tot;
                }
            }
            return total;
        }
        bool keep[V];
        uint32_t y[V];
        uint32_t cu = 0;
        if (opc == D_FILT_HASH_CTX && uni) cu = M.mctx[k[0]];
        if (opc == D_FILT_WEIGHT && uni) cu = fmix32(M.mpar[k[0]] ^ sd.c0);
#pragma unroll
        for (int s = 0; s < V; ++s) {
            const uint32_t xs = x[s];
            bool kp;
            uint32_t ys = xs;
            switch (opc) {
            case D_FILT_MASK: kp = (xs & sd.p0) == sd.p1; break;
            case D_FILT_MOD: kp = (xs % sd.p0) == sd.p1; break;
            case D_FILT_HASH_CTX: kp = (fmix32(xs ^ sd.c0) ^ (uni ? cu : M.mctx[k[s]])) < sd.p1; break;
            case D_FILT_WEIGHT: kp = fmix32(xs ^ sd.c0) < (uni ? cu : fmix32(M.mpar[k[s]] ^ sd.c0)); break;
            case D_MAP_MULADD: ys = xs * sd.p0 + sd.p1; kp = true; break;
            default: kp = false; break;
            }
            keep[s] = kp && 32u * s + lane < take;
            y[s] = ys;
        }
        uint32_t tot = 0;
#pragma unroll
        for (int s = 0; s < V; ++s) {
            bal[s] = 32u * s < take ? __ballot_sync(FULLMASK, keep[s]) : 0u;
            tot += __popc(bal[s]);
        }
#pragma unroll
        for (int c = 2; c < RS_MAX_STAGES; ++c) {
            if (!(km & (1u << c))) continue;
            const uint32_t orb = (c - 2) * C;
            const bool tagc = emode(c) == EM_TAG;
            uint32_t base = w.qt[c - 1];
#pragma unroll
            for (int s = 0; s < V; ++s) {
                if (keep[s]) {
                    const uint32_t slot = orb + ((base + __popc(bal[s] & lt)) & cm);
                    M.qv[slot] = y[s];
                    if (tagc) M.qtag[slot] = (uint16_t)k[s];
                }
                base += __popc(bal[s]);
            }
            w.qt[c - 1] = base;
            w.em[c - 1] += tot;
        }
        return tot;
    }

    // the emit sink fed by tags or per-lane contexts: one position claimed per item
    __device__ __forceinline__ void emit_items(const uint32_t (&x)[V], const uint32_t (&k)[V], uint32_t take)
    {
        const uint32_t o0 = __ldg(ds->offsets);
#pragma unroll
        for (int s = 0; s < V; ++s) {
            if (32u * s + lane < take) {
                const uint32_t r = r0 + k[s];
                const unsigned long long pos =
                    (unsigned long long)P.emit_f * (__ldg(ds->offsets + r) - o0) + atomicAdd(ds->out_count + r, 1u);
                if (pos < ds->out_values_len) ds->out_values[pos] = x[s];
                else atomicOr(&P.hdr->status, ST_BAD_INPUT);
            }
        }
    }

    // leaf I (an aggregate or the emit sink) takes one ensemble: fed by signals, the whole
    // ensemble belongs to the leaf's current parent (Section 3.3) and folds into its
    // running accumulator; fed by tags or per-lane contexts, runs of equal parents fold
    // into the per-parent accumulators (segmented warp reduction)
    template <int I>
    __device__ __forceinline__ void mix_sink(const uint32_t (&x)[V], const uint32_t (&k)[V], bool uni, uint32_t take)
    {
        const uint32_t q = sink_idx(I);
        if (emode(I) == EM_SIG) {
            if (P.emit) {
                emit_ensemble(x, take);
                return;
            }
            unsigned long long part = 0;
            uint32_t mn = 0xFFFFFFFFu;
#pragma unroll
            for (int s = 0; s < V; ++s) {
                if (32u * s + lane < take) {
                    part += x[s];
                    mn = min(mn, x[s]);
                }
            }
            const uint32_t lo = __reduce_add_sync(FULLMASK, (uint32_t)(part & 0xFFFFu));
            const uint32_t hi = __reduce_add_sync(FULLMASK, (uint32_t)(part >> 16));
            const unsigned long long sm = ((unsigned long long)hi << 16) + lo;
            mn = __reduce_min_sync(FULLMASK, mn);
            if (q == 0) {
                w.acc_c += take;
                w.acc_s += sm;
                w.acc_m = min(w.acc_m, mn);
            } else {
                w.acc2_c += take;
                w.acc2_s += sm;
                w.acc2_m = min(w.acc2_m, mn);
            }
            return;
        }
        if (P.emit) {
            emit_items(x, k, take);
            return;
        }
        const SArr<uint32_t> rc = rcq(q), rm = rmq(q);
        const SArr<unsigned long long> rs = rsq(q);
        (void)uni;
#pragma unroll
        for (int s = 0; s < V; ++s) {
            const uint32_t sb = 32u * s;
            if (sb >= take) break;
            const uint32_t n = min(32u, take - sb);
            const bool act = lane < n;
            const uint32_t v = act ? x[s] : 0u;
            const uint32_t kk = act ? k[s] : 0xFFFFFFFFu;
            // runs of equal parents: per-lane contexts never decrease along the ensemble
            const uint32_t kprev = __shfl_up_sync(FULLMASK, kk, 1);
            const uint32_t knext = __shfl_down_sync(FULLMASK, kk, 1);
            const bool head = lane == 0 || kk != kprev;
            const bool tail = lane == 31 || kk != knext;
            const uint32_t heads = __ballot_sync(FULLMASK, head);
            const uint32_t hl = 31 - __clz(heads & ((2u << lane) - 1u));
            unsigned long long ps = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long t = __shfl_up_sync(FULLMASK, ps, d);
                if (lane >= (uint32_t)d) ps += t;
            }
            unsigned long long before = __shfl_sync(FULLMASK, ps, hl > 0 ? hl - 1 : 0);
            if (hl == 0) before = 0;
            uint32_t m = act ? v : 0xFFFFFFFFu;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(FULLMASK, m, d);
                if (lane >= (uint32_t)d && lane - d >= hl) m = min(m, t);
            }
            if (act && tail) {
                rc[kk] += lane - hl + 1;
                rs[kk] += ps - before;
                if (P.want_min) rm[kk] = min(rm[kk], m);
            }
            __syncwarp();
        }
    }

    // the signal phase of a node fed by signals (receiver rule 2b, as signal_phase), with
    // the signals forwarded to every child that takes signals, each with the credit of its
    // own edge's sender rules, and an End at a leaf reporting that leaf's accumulator
    template <int I>
    __device__ __forceinline__ bool mix_signal_phase(bool last)
    {
        const uint32_t SC = P.SC;
        const uint32_t km = kids(I);
        const uint32_t q = last ? sink_idx(I) : 0u;
        bool progress = false;
        while (w.credit[I] == 0 && w.sh[I - 1] != w.st[I - 1]) {
            const uint32_t h = sidx(I - 1, w.sh[I - 1]);
            const uint32_t hcr = M.sq[h + 1];
            if (hcr > 0) {
                w.credit[I] = hcr;
                __syncwarp();
                if (lane == 0) M.sq[h + 1] = 0;
                __syncwarp();
                progress = true;
                break;
            }
            uint32_t room = 32u;
            if (!last) {
#pragma unroll
                for (int c = 2; c < RS_MAX_STAGES; ++c)
                    if ((km & (1u << c)) && emode(c) != EM_TAG) room = min(room, SC - (w.st[c - 1] - w.sh[c - 1]));
            }
            const uint32_t mmax = min(min(32u, w.st[I - 1] - w.sh[I - 1]), room);
            if (mmax == 0) break;
            const bool in = lane < mmax;
            const uint32_t j = sidx(I - 1, w.sh[I - 1] + lane);
            const uint32_t word = in ? M.sq[j] : 0u;
            const uint32_t cr = in ? M.sq[j + 1] : 1u;
            const uint32_t nz = __ballot_sync(FULLMASK, cr != 0u);
            const uint32_t m = nz ? (uint32_t)(__ffs(nz) - 1) : 32u;
            const bool mine = lane < m;
            const bool is_begin = mine && !(word & SIG_END);
            const uint32_t begins = __ballot_sync(FULLMASK, is_begin);
            if (begins) w.ctxk[I] = __shfl_sync(FULLMASK, word, 31 - __clz(begins));
            if (last) {
                uint32_t ac = q ? w.acc2_c : w.acc_c, am = q ? w.acc2_m : w.acc_m;
                unsigned long long as = q ? w.acc2_s : w.acc_s;
                if (mine && (word & SIG_END)) {
                    const uint32_t kk = word & ~SIG_END;
                    const bool fresh = (begins & lanemask_lt()) != 0u;
                    rcq(q)[kk] = fresh ? 0u : ac;
                    rsq(q)[kk] = fresh ? 0ull : as;
                    if (P.want_min) rmq(q)[kk] = fresh ? 0xFFFFFFFFu : am;
                }
                if (begins) {
                    if (q) {
                        w.acc2_c = 0;
                        w.acc2_s = 0;
                        w.acc2_m = 0xFFFFFFFFu;
                    } else {
                        w.acc_c = 0;
                        w.acc_s = 0;
                        w.acc_m = 0xFFFFFFFFu;
                    }
                }
            } else {
#pragma unroll
                for (int c = 2; c < RS_MAX_STAGES; ++c) {
                    if (!(km & (1u << c)) || emode(c) == EM_TAG) continue;
                    const uint32_t c0 = (w.sh[c - 1] == w.st[c - 1]) ? (w.qt[c - 1] - w.qh[c - 1]) : w.em[c - 1];
                    if (mine) {
                        const uint32_t o = sidx(c - 1, w.st[c - 1] + lane);
                        M.sq[o] = word;
                        M.sq[o + 1] = lane == 0 ? c0 : 0u;
                    }
                    w.st[c - 1] += m;
                    w.em[c - 1] = 0;
                }
            }
            __syncwarp();
            w.sh[I - 1] += m;
            CNT_ADD(I, 2, m);
            progress = true;
        }
        return progress;
    }

    // Per-lane state selection (Section 6): node I's input edge carries signals, but its
    // ensembles are not cut at them.  The signals whose position falls inside the
    // ensemble are consumed with it (up to LANE_MAX_SIG, read 32 at a time).  Positions
    // come from the credits: the head signal's counts the items before it (w.credit[I]
    // holds it once taken off the ring), each later one the items since the signal before.
    // Every lane takes the context of the last Begin at or before its item; each consumed
    // signal is forwarded to the children that take signals with the credit the sender
    // rules give it at its place among the outputs (the first: |Q| or the count since the
    // child's last signal, plus the outputs before it; the others: the outputs since the
    // signal before).  Fan-out 1 only (the host rejects an expansion fed this way).
    // Until its input is drained the node waits for full ensembles, unless its signal
    // ring is nearly full: then the producer waits on it, and it takes what it has.  An
    // ensemble waits for room for all of it in every child's ring.
    // Returns false when nothing was consumed.
    static constexpr uint32_t LANE_MAX_SIG = 256;

    // signal j (from the head) of edge e: its word and credit
    __device__ __forceinline__ uint32_t sig_word(uint32_t e, uint32_t j) const { return M.sq[sidx(e, w.sh[e] + j)]; }

    template <int I>
    __device__ __forceinline__ bool lane_step(bool drain, uint32_t &took, uint32_t &nsig)
    {
        const uint32_t e = I - 1;
        const uint32_t C = P.C, SC = P.SC;
        const bool last = is_sink(I);
        const uint32_t km = last ? 0u : kids(I);
        uint32_t space = W, sroom = SC;
        bool fwd = false;
#pragma unroll
        for (int c = 2; c < RS_MAX_STAGES; ++c) {
            if (!(km & (1u << c))) continue;
            space = min(space, C - (w.qt[c - 1] - w.qh[c - 1]));
            if (emode(c) != EM_TAG) {
                sroom = min(sroom, SC - (w.st[c - 1] - w.sh[c - 1]));
                fwd = true;
            }
        }
        const uint32_t avail = w.qt[e] - w.qh[e];
        const uint32_t pend = w.st[e] - w.sh[e];
        // an ensemble fires only when the children have room for all of it (like the
        // data phase of fire_body, which waits for downstream space rather than cut it)
        uint32_t take = min(avail, W);
        if (space < take) take = 0;
        if (!drain && take < W && SC - pend >= 2) take = 0;
        // pass 1: how many signals this step consumes -- those at or before the
        // ensemble's end, as many as fit the children's signal rings
        const uint32_t mmax = min(fwd ? sroom : SC, LANE_MAX_SIG);
        uint32_t m = 0, stop_pos = 0xFFFFFFFFu, last_pos = 0, pbase = w.credit[I];
        while (m < pend && m < mmax) {
            const uint32_t np = min(32u, pend - m);
            const bool in = lane < np;
            const uint32_t cr = in ? M.sq[sidx(e, w.sh[e] + m + lane) + 1] : 0u;
            const uint32_t pos = pbase + warp_incl_scan_u32(cr, lane);
            uint32_t mc = __popc(__ballot_sync(FULLMASK, in && pos <= take));
            mc = min(mc, mmax - m);
            if (mc < np) stop_pos = __shfl_sync(FULLMASK, pos, mc);
            if (mc > 0) last_pos = __shfl_sync(FULLMASK, pos, mc - 1);
            pbase = __shfl_sync(FULLMASK, pos, 31);
            m += mc;
            if (mc < 32) break;
        }
        // the items of this step stop at the first signal left on the ring
        if (stop_pos != 0xFFFFFFFFu) take = min(take, stop_pos);
        else if (m < pend) take = min(take, last_pos);
        if (take == 0 && m == 0) return false;
        uint32_t x[V], k[V];
#pragma unroll
        for (int s = 0; s < V; ++s) {
            x[s] = 0;
            k[s] = w.ctxk[I];
        }
        if (take > 0) (void)gather<I, false>(take, x, k);
        if (stop) return false;
        // pass 2: mark the item of every consumed Begin strictly inside the ensemble with
        // its index + 1 (the later Begin wins at one position), then a running maximum over
        // the items gives each lane the signal whose word is its context
        uint32_t lastb = 0xFFFFFFFFu;   // index of the last consumed Begin
        bool inside = false;
        if (m > 0) {
            if (take > 0) {
#pragma unroll
                for (int s = 0; s < V; ++s) M.scr[32u * s + lane] = 0u;
                __syncwarp();
            }
            pbase = w.credit[I];
            for (uint32_t b = 0; b < m; b += 32) {
                const bool in = b + lane < m;
                const uint32_t j = sidx(e, w.sh[e] + b + lane);
                const uint32_t word = in ? M.sq[j] : SIG_END;
                const uint32_t pos = pbase + warp_incl_scan_u32(in ? M.sq[j + 1] : 0u, lane);
                const bool begin = in && !(word & SIG_END);
                const uint32_t bb = __ballot_sync(FULLMASK, begin);
                if (bb) lastb = b + 31 - __clz(bb);
                if (begin && pos < take) atomicMax(&M.scr[pos], b + lane + 1u);
                inside = inside || __any_sync(FULLMASK, begin && pos < take);
                pbase = __shfl_sync(FULLMASK, pos, 31);
            }
            __syncwarp();
            if (inside) {
                uint32_t carry = 0;
#pragma unroll
                for (int s = 0; s < V; ++s) {
                    uint32_t inc = M.scr[32u * s + lane];
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) inc = max(inc, __shfl_up_sync(FULLMASK, inc, d));
                    const uint32_t rel = max(carry, inc);
                    carry = max(carry, __shfl_sync(FULLMASK, inc, 31));
                    if (rel && 32u * s + lane < take) k[s] = sig_word(e, rel - 1u);
                }
                __syncwarp();
            }
        }
        if constexpr (I == 1) {
            // hashed enumeration: an element is a function of its parent, which the lane
            // knows only now
            if (op<0>() == D_ENUM_HASH && inside) {
                const uint32_t q0 = w.qh[0];
#pragma unroll
                for (int s = 0; s < V; ++s) {
                    const uint32_t q = 32u * s + lane;
                    if (q < take) x[s] = fmix32(M.mpar[k[s]] ^ fmix32((q0 + q - M.moff[k[s]]) ^ RS_GOLD));
                }
            }
        }
        if (last) {
            if constexpr (S::template maybe_last<I>())
                if (take > 0) mix_sink<I>(x, k, !inside, take);
        } else if constexpr (S::template maybe_elem<I>()) {
            // the children's queues before this step's outputs (for the first credit)
            uint32_t first[RS_MAX_STAGES];
#pragma unroll
            for (int c = 2; c < RS_MAX_STAGES; ++c) {
                first[c] = 0;
                if ((km & (1u << c)) && emode(c) != EM_TAG)
                    first[c] = (w.sh[c - 1] == w.st[c - 1]) ? (w.qt[c - 1] - w.qh[c - 1]) : w.em[c - 1];
            }
            uint32_t bal[V];
            uint32_t tot = 0;
            if (take > 0) {
                tot = mix_stage<I>(x, k, !inside, take, bal);
            } else {
#pragma unroll
                for (int s = 0; s < V; ++s) bal[s] = 0;
            }
            if (m > 0 && fwd) {
                // pass 3: forward; ob = outputs of the items before a signal's position
                pbase = w.credit[I];
                uint32_t ob_prev = 0;
                for (uint32_t b = 0; b < m; b += 32) {
                    const bool in = b + lane < m;
                    const uint32_t j = sidx(e, w.sh[e] + b + lane);
                    const uint32_t word = in ? M.sq[j] : 0u;
                    const uint32_t pos = pbase + warp_incl_scan_u32(in ? M.sq[j + 1] : 0u, lane);
                    uint32_t ob = 0;
#pragma unroll
                    for (int s = 0; s < V; ++s) {
                        const uint32_t lo = 32u * s;
                        if (pos >= lo + 32u) ob += __popc(bal[s]);
                        else if (pos > lo) ob += __popc(bal[s] & ((1u << (pos - lo)) - 1u));
                    }
                    uint32_t obp = __shfl_up_sync(FULLMASK, ob, 1);
                    if (lane == 0) obp = ob_prev;
#pragma unroll
                    for (int c = 2; c < RS_MAX_STAGES; ++c) {
                        if (!(km & (1u << c)) || emode(c) == EM_TAG) continue;
                        if (in) {
                            const uint32_t o = sidx(c - 1, w.st[c - 1] + b + lane);
                            M.sq[o] = word;
                            M.sq[o + 1] = (b + lane == 0) ? first[c] + ob : ob - obp;
                        }
                    }
                    const uint32_t nin = min(32u, m - b);
                    ob_prev = __shfl_sync(FULLMASK, ob, nin - 1);
                    pbase = __shfl_sync(FULLMASK, pos, 31);
                }
#pragma unroll
                for (int c = 2; c < RS_MAX_STAGES; ++c) {
                    if (!(km & (1u << c)) || emode(c) == EM_TAG) continue;
                    w.st[c - 1] += m;
                    w.em[c - 1] = tot - ob_prev;
                }
            }
        }
        if (lastb != 0xFFFFFFFFu) w.ctxk[I] = sig_word(e, lastb);
        // the signal now at the head: the items still before it
        if (m < pend && stop_pos != 0xFFFFFFFFu) {
            if (lane == 0) M.sq[sidx(e, w.sh[e] + m) + 1] = 0;
            w.credit[I] = stop_pos - take;
        } else {
            w.credit[I] = 0;
        }
        __syncwarp();
        w.qh[e] += take;
        w.sh[e] += m;
        if constexpr (I == 1) {
            if (op<0>() == D_ENUM_LOAD && E0 + w.qh[0] >= g.free_lim) release_below(E0 + w.qh[0]);
        }
        CNT_ADD(I, 2, m);
        took = take;
        nsig = m;
        return true;
    }

    // fire node I (MIX): per-lane selection steps for an EM_LANE input, else the data and
    // signal phases of fire_body with the children's room and modes
    template <int I>
    __device__ __forceinline__ void mix_fire(bool drain)
    {
        const uint32_t mode = emode(I);
        const bool last = is_sink(I);
        const uint32_t km = last ? 0u : kids(I);
        bool fired = false;
        uint32_t n_ens = 0, n_items = 0;
        if (mode == EM_LANE) {
            for (;;) {
                uint32_t took = 0, nsig = 0;
                if (!lane_step<I>(drain, took, nsig)) break;
                if (!fired) {
                    CNT_ADD(I, 3, 1);
                    fired = true;
                }
                if (took) {
                    n_ens++;
                    n_items += took;
                }
                if (stop) break;
            }
        } else {
            const uint32_t fan = op<I>() == D_EXPAND ? P.st[I].fanout : 1u;
            for (;;) {
                const bool sigp = mode == EM_SIG && w.sh[I - 1] != w.st[I - 1];
                const uint32_t avail0 = w.qt[I - 1] - w.qh[I - 1];
                if (!(drain ? (avail0 > 0 || sigp) : (avail0 >= W || sigp))) break;
                if (!fired) {
                    CNT_ADD(I, 3, 1);
                    fired = true;
                }
                bool progress = false;
                for (;;) {
                    uint32_t want = min(w.qt[I - 1] - w.qh[I - 1], W);
                    if (sigp) want = min(want, w.credit[I]);
                    uint32_t take = want;
                    if (!last) {
                        uint32_t space = 0xFFFFFFFFu;
#pragma unroll
                        for (int c = 2; c < RS_MAX_STAGES; ++c)
                            if (km & (1u << c)) space = min(space, P.C - (w.qt[c - 1] - w.qh[c - 1]));
                        take = min(take, fan == 1u ? space : space / fan);
                    }
                    if (take == 0) break;
                    if (take < want) break;                       // wait for downstream space
                    if (!drain && !sigp && take < W) break;       // wait for a full ensemble
                    if (last) {
                        if constexpr (S::template maybe_last<I>()) aggregate<I, false>(take);
                    } else {
                        if constexpr (S::template maybe_elem<I>()) element_stage<I, false>(take);
                    }
                    if (stop) break;
                    __syncwarp();
                    w.qh[I - 1] += take;
                    if (sigp) w.credit[I] -= take;
                    n_ens++;
                    n_items += take;
                    progress = true;
                    if constexpr (I == 1) {
                        if (op<0>() == D_ENUM_LOAD && E0 + w.qh[0] >= g.free_lim) release_below(E0 + w.qh[0]);
                    }
                }
                if (stop) break;
                if (mode == EM_SIG) progress |= signal_phase<I>(last);
                if (!progress) break;
            }
        }
        if (n_ens) {
            CNT_ADD(I, 0, n_ens);
            CNT_ADD(I, 1, n_items);
        }
    }

    // one unit through the per-edge pipeline: the scheduler of run_unit over the tree,
    // upstream first; a node drains once its producer has drained and its producer's
    // input edge is empty
    __device__ __forceinline__ void mix_run_unit()
    {
#pragma unroll
        for (int i = 0; i < RS_MAX_EDGES; ++i) w.qh[i] = w.qt[i] = w.sh[i] = w.st[i] = w.em[i] = 0;
#pragma unroll
        for (int i = 0; i < RS_MAX_STAGES; ++i) w.credit[i] = w.ctxk[i] = 0;
        w.acc_c = w.acc2_c = 0;
        w.acc_s = w.acc2_s = 0;
        w.acc_m = w.acc2_m = 0xFFFFFFFFu;
        ek = 0;
        const int n = nst();
        // leaves fed by tags or per-lane contexts fold into per-parent accumulators, which
        // start at the identity; an emit sink uses none, and the minima exist only when a
        // stream asks for them (the layout gives them no room otherwise)
        for (int i = 1; i < n; ++i) {
            if (!is_sink(i) || emode(i) == EM_SIG || P.emit) continue;
            const uint32_t q = sink_idx(i);
            for (uint32_t kk = lane; kk < nk; kk += 32) {
                rcq(q)[kk] = 0u;
                rsq(q)[kk] = 0ull;
                if (P.want_min) rmq(q)[kk] = 0xFFFFFFFFu;
            }
        }
        __syncwarp();
        const bool tag0 = emode(1) == EM_TAG;
        if (tag0) {
            w.qt[0] = total;
            CNT_ADD(0, 0, (total + W - 1) / W);
            CNT_ADD(0, 1, total);
            ek1 = 0;
            if (total > 0) advance_ek1(0, 0);
        }
        for (unsigned long long sweep = 0;; ++sweep) {
            CNT_ADD(0, 3, 1);
            if (nxt_open) {
                poll_next(*nxt, P, M, lane);
                nxt_open = !nxt->scanned;
            }
            if (!tag0) enum_signal();
            const bool done0 = tag0 || ek >= nk;
            uint32_t dm = 0;   // bit i: node i drains
#define RS_MIX_FIRE(I)                                                                            \
            if (I < n) {                                                                          \
                const uint32_t u = up_of(I);                                                      \
                const bool d = u == 0 ? done0 : (((dm >> u) & 1u) && edge_empty_at(u - 1));       \
                if (d) dm |= 1u << I;                                                             \
                fire<I>(d);                                                                       \
            }
            RS_MIX_FIRE(1)
            RS_MIX_FIRE(2)
            RS_MIX_FIRE(3)
            RS_MIX_FIRE(4)
            RS_MIX_FIRE(5)
#undef RS_MIX_FIRE
            if (stop) return;
            bool all = done0;
#pragma unroll
            for (int e2 = 0; e2 < RS_MAX_EDGES; ++e2)
                if (e2 + 1 < n) all = all && edge_empty(e2);
            if (all) break;
            if (sweep >= P.budget) {
                if (lane == 0) atomicOr(&P.hdr->status, ST_STALL);
                stop = true;
                return;
            }
        }
    }

    // ---- run one unit to completion: the non-preemptive scheduler of Section 2.1 ----
    // Each sweep offers every node a firing, upstream first.
    __device__ __forceinline__ void run_unit()
    {
#pragma unroll
        for (int i = 0; i < RS_MAX_EDGES; ++i) w.qh[i] = w.qt[i] = w.sh[i] = w.st[i] = w.em[i] = 0;
#pragma unroll
        for (int i = 0; i < RS_MAX_STAGES; ++i) w.credit[i] = w.ctxk[i] = 0;
        w.acc_c = 0;
        w.acc_s = 0;
        w.acc_m = 0xFFFFFFFFu;
        ek = 0;
        if (STRAT == RS_STRATEGY_TAG) {
            // enumeration emits every position of the unit at once; node 1 derives tags
            w.qt[0] = total;
            CNT_ADD(0, 0, (total + W - 1) / W);
            CNT_ADD(0, 1, total);
            ek1 = 0;
            if (total > 0) advance_ek1(0, 0);
        }
        for (unsigned long long sweep = 0;; ++sweep) {
            CNT_ADD(0, 3, 1);
            if (nxt_open) {
                poll_next(*nxt, P, M, lane);
                nxt_open = !nxt->scanned;
            }
            if (STRAT == RS_STRATEGY_SIGNAL) {
                const long long pt = PROF_NOW();
                (void)pt;
                enum_signal();
                PROF_ADD(PF_ENUM, pt);
            }
            bool d = (STRAT == RS_STRATEGY_TAG) || ek >= nk;
            fire<1>(d);
            d = d && edge_empty(0);
            fire<2>(d);
            d = d && (nst() <= 2 || edge_empty(1));
            fire<3>(d);
            d = d && (nst() <= 3 || edge_empty(2));
            fire<4>(d);
            d = d && (nst() <= 4 || edge_empty(3));
            fire<5>(d);
            d = d && (nst() <= 5 || edge_empty(4));
            if (stop) return;
            if (d) break;
            if (sweep >= P.budget) {
                if (lane == 0) atomicOr(&P.hdr->status, ST_STALL);
                stop = true;
                return;
            }
        }
    }
};

// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------

template <int STRAT, int V, class SG, bool MIX = false, int UM = -1>
__global__ void __launch_bounds__(256, 2) rs_pipeline_kernel(const __grid_constant__ KParams P)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t wb = warp * P.L.per_warp;   // this processor's byte offset in shared memory
    Smem M;
    M.prof = sarr<unsigned long long>(wb + P.L.o_prof);
    M.cnt = sarr<unsigned long long>(wb + P.L.o_cnt);
    Pending *const pend = reinterpret_cast<Pending *>(smem_raw + wb + P.L.o_pend);
    M.mbar = sarr<unsigned long long>(wb + P.L.o_mbar);
    M.mmeta = sarr<unsigned long long>(wb + P.L.o_mmeta);
    M.tiles = sarr<uint32_t>(wb + P.L.o_tiles);
    M.mraw0 = sarr<uint32_t>(wb + P.L.o_raw[0]);
    M.mraw1 = sarr<uint32_t>(wb + P.L.o_raw[1]);
    M.mmoff0 = sarr<uint32_t>(wb + P.L.o_moff[0]);
    M.mmoff1 = sarr<uint32_t>(wb + P.L.o_moff[1]);
    M.mctx0 = sarr<uint32_t>(wb + P.L.o_ctxb[0]);
    M.mctx1 = sarr<uint32_t>(wb + P.L.o_ctxb[1]);
    M.mpar0 = sarr<uint32_t>(wb + P.L.o_parb[0]);
    M.mpar1 = sarr<uint32_t>(wb + P.L.o_parb[1]);
    M.moff = M.mmoff0;
    M.mctx = M.mctx0;
    M.mpar = M.mpar0;
    M.rc = sarr<uint32_t>(wb + P.L.o_rc);
    M.rs = sarr<unsigned long long>(wb + P.L.o_rs);
    M.rm = sarr<uint32_t>(wb + P.L.o_rm);
    M.rc2 = sarr<uint32_t>(wb + P.L.o_rc2);
    M.rs2 = sarr<unsigned long long>(wb + P.L.o_rs2);
    M.rm2 = sarr<uint32_t>(wb + P.L.o_rm2);
    M.qv = sarr<uint32_t>(wb + P.L.o_qv);
    M.qtag = sarr<uint16_t>(wb + P.L.o_qt);
    M.q64 = sarr<unsigned long long>(wb + P.L.o_qv);
    M.sq = sarr<uint32_t>(wb + P.L.o_sq);
    M.scr = sarr<uint32_t>(wb + P.L.o_scr);

    if (lane == 0) {
        if (P.any_load)
            for (uint32_t s = 0; s < P.NT; ++s) mbar_init(&M.mbar[s], 1);
        mbar_init(&M.mmeta[0], 32);   // one arrival per lane per metadata prefetch
        mbar_init(&M.mmeta[1], 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
#ifdef RS_PROFILE
    if (lane < RS_PROF_SLOTS) M.prof[lane] = 0;
#endif
    const long long t_start = PROF_NOW();
    (void)t_start;
    __syncwarp();

    Warp w;
    if (lane < 4 * RS_MAX_STAGES) M.cnt[lane] = 0;
    Stage g;
    g.phase = 0;
    g.failed = false;
    unsigned long long units = 0;
    bool stop = false;
    const bool load = (SG::generic ? P.st[0].op : (uint32_t)SG::template op<0>()) == D_ENUM_LOAD;

    // first unit: claim and prefetch
    Pending cur;
    {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&P.hdr->cursor, 1u);
        t = __shfl_sync(FULLMASK, t, 0);
        cur.u = describe_unit(P, t);
        cur.buf = 0;
        cur.phase = 0;
        cur.scanned = false;
        cur.bad = false;
        cur.split_tail = false;
        cur.total = cur.E0 = cur.tail_off = cur.tail_len = 0;
        if (cur.u.valid) prefetch_meta(P, M, cur.u, 0, lane);
    }

    while (cur.u.valid && !stop) {
        long long pt_setup = PROF_NOW();
        (void)pt_setup;
        units++;
        // claim the next unit now; its ticket is read after this unit's setup
        uint32_t next_ticket = 0;
        if (lane == 0) next_ticket = atomicAdd(&P.hdr->cursor, 1u);

        const DevStream &S = P.streams[cur.u.stream];
        const uint32_t r0 = cur.u.r0, nk = cur.u.nk;
        const uint32_t b = cur.buf;
        if (!cur.scanned) {
            // wait (bounded) for this unit's metadata
            const uint32_t par = (cur.phase >> b) & 1u;
            if (!mbar_try_wait(&M.mmeta[b], par)) {
                unsigned long long t0 = global_ns();
                uint32_t it = 0;
                while (!mbar_try_wait(&M.mmeta[b], par)) {
                    if ((++it & 63u) == 0 && global_ns() - t0 > P.spin_limit) {
                        if (lane == 0) atomicOr(&P.hdr->status, ST_COPY_TIMEOUT);
                        stop = true;
                        break;
                    }
                }
                if (stop) break;
            }
            cur.phase ^= 1u << b;
            scan_meta(cur, P, M, lane);
        }
        const uint32_t E0 = cur.E0;
        const uint32_t total = cur.total;
        bool bad = cur.bad;
        if (load && !bad && (unsigned long long)E0 + total > S.n_elements) bad = true;

        // the prefetched next unit (its copies overlap this unit's work)
        Pending &nxt = *pend;
        __syncwarp();
        {
            const uint32_t t = __shfl_sync(FULLMASK, next_ticket, 0);
            nxt.u = describe_unit(P, t);
            nxt.buf = b ^ 1u;
            nxt.phase = cur.phase;
            nxt.scanned = false;
            nxt.bad = false;
            nxt.split_tail = false;
            nxt.total = nxt.E0 = nxt.tail_off = nxt.tail_len = 0;
            if (nxt.u.valid) prefetch_meta(P, M, nxt.u, nxt.buf, lane);
        }

        if (bad || cur.u.skip) {
            if (bad && lane == 0) atomicOr(&P.hdr->status, ST_BAD_INPUT);
            cur = nxt;
            continue;
        }
        M.moff = M.moffb(b);
        M.mctx = M.ctxb(b);
        M.mpar = M.parb(b);
        if (P.need_ctx && !S.ctx)
            for (uint32_t k = lane; k < nk; k += 32) M.mctx[k] = 0u;
        if (P.need_par && !S.parents)
            for (uint32_t k = lane; k < nk; k += 32) M.mpar[k] = r0 + k;
        const bool split_head = cur.u.has_head;
        const bool split_tail = cur.split_tail;
        __syncwarp();

        // ---- element staging: bulk copies of [A, B) in tiles ----
        g.elements = S.elements;
        g.tma = load && S.tma_ok && P.NT > 0;
        g.A = E0 & ~3u;
        g.B = (E0 + total) & ~3u;
        if (g.B < g.A) g.B = g.A;
        g.ntiles = g.tma ? (g.B - g.A + P.TE - 1) / P.TE : 0u;
        g.t_issued = g.t_ready = g.t_freed = 0;
        g.ready_lim = g.tma ? (g.ntiles ? g.A : 0xFFFFFFFFu) : 0xFFFFFFFFu;
        g.free_lim = g.A + P.TE;

        PROF_ADD(PF_SETUP, pt_setup);
        bool pstop;
        {
            Proc<STRAT, V, SG, MIX, UM> pr(P, M, w, g, lane);
            pr.nxt = pend;
            pr.nxt_open = nxt.u.valid && !nxt.scanned;
            pr.nk = nk;
            pr.total = total;
            pr.E0 = E0;
            pr.ds = &S;
            pr.r0 = r0;
            if (g.tma) pr.issue_tiles();
            if constexpr (MIX) pr.mix_run_unit();
            else pr.run_unit();
            pr.finish_tiles();
            pstop = pr.stop;
        }
        if (pstop) {
            stop = true;
            break;
        }
        __syncwarp();

        // ---- per-parent results, coalesced ----
        const long long pt_fl = PROF_NOW();
        (void)pt_fl;
        // parents processed in pieces (the continued head, a last parent running past
        // the unit) merge through their owner's slot; the rest are written directly (tag
        // strategy: already updated in place)
        {
            for (uint32_t k = lane; k < nk; k += 32) {
                if ((k == 0 && split_head) || (k == nk - 1 && split_tail)) continue;
                if (P.want_count) S.out_count[r0 + k] = M.rc[k];
                if (P.want_sum) S.out_sum[r0 + k] = M.rs[k];
                if (P.want_min) S.out_min[r0 + k] = M.rm[k];
                if (MIX && P.n_sinks > 1) {
                    // a tree's second leaf
                    if (P.want_count) S.out2_count[r0 + k] = M.rc2[k];
                    if (P.want_sum) S.out2_sum[r0 + k] = M.rs2[k];
                    if (P.want_min) S.out2_min[r0 + k] = M.rm2[k];
                }
            }
        }
        // accumulator of the first and the last parent: index 0 and nk - 1 (signal
        // strategy), slots 0 and 1 (tag strategy; one slot when they are the same parent)
        const uint32_t ah = 0, at = nk - 1;
        if (lane == 0) {
            if (split_head)
                merge_piece(S, r0, cur.u.head_off, cur.u.ebase, false, M.rc[ah], M.rs[ah],
                            P.want_min ? M.rm[ah] : 0xFFFFFFFFu);
            if (split_tail && !(split_head && nk == 1))
                merge_piece(S, r0 + nk - 1, cur.tail_off, cur.u.ebase, true, M.rc[at], M.rs[at],
                            P.want_min ? M.rm[at] : 0xFFFFFFFFu);
            if (MIX && P.n_sinks > 1) {
                if (split_head)
                    merge_piece(S, r0, cur.u.head_off, cur.u.ebase, false, M.rc2[ah], M.rs2[ah],
                                P.want_min ? M.rm2[ah] : 0xFFFFFFFFu, 1);
                if (split_tail && !(split_head && nk == 1))
                    merge_piece(S, r0 + nk - 1, cur.tail_off, cur.u.ebase, true, M.rc2[at], M.rs2[at],
                                P.want_min ? M.rm2[at] : 0xFFFFFFFFu, 1);
            }
        }
        __syncwarp();
        PROF_ADD(PF_FLUSH, pt_fl);
        cur = nxt;
    }
    // a prefetch may still be in flight when the loop ends (error exit): let it land
    if (cur.u.valid && !cur.scanned) {
        const uint32_t par = (cur.phase >> cur.buf) & 1u;
        unsigned long long t0 = global_ns();
        uint32_t it = 0;
        while (!mbar_try_wait(&M.mmeta[cur.buf], par)) {
            if ((++it & 63u) == 0 && global_ns() - t0 > P.spin_limit) break;
        }
    }

    // ---- counters ----
    PROF_ADD(PF_TOTAL, t_start);
    __syncwarp();
#ifdef RS_PROFILE
    if (lane < RS_PROF_SLOTS) atomicAdd(&P.hdr->cyc[lane], M.prof[lane]);
#endif
    if (lane == 0) {
        atomicAdd(&P.hdr->units, units);
        for (int i = 0; i < 4 * P.n_stages; ++i) atomicAdd(&P.hdr->counters[i], M.cnt[i]);
    }
}

// ---------------------------------------------------------------------------
// host-side launch helpers

// Kernel table: specialised signatures for the pipelines the workloads use, plus the
// generic kernel for any other stage list.
struct KEntry {
    int strategy, V, oe, o1, o2, o3, o4;
    const void *fn;
    int um;   // per-edge kernels: the mode of every edge, compiled in (-1: read per edge)
};

#define RS_KSIG(ST, V, OE, O1, O2, O3, O4) \
    {ST, V, OE, O1, O2, O3, O4, (const void *)rs_pipeline_kernel<ST, V, Sig<OE, O1, O2, O3, O4>>, -1}
#define RS_KALLV(ST, OE, O1, O2, O3, O4) \
    RS_KSIG(ST, 1, OE, O1, O2, O3, O4), RS_KSIG(ST, 2, OE, O1, O2, O3, O4), RS_KSIG(ST, 4, OE, O1, O2, O3, O4)
#define RS_KBOTH(OE, O1, O2, O3, O4) RS_KALLV(RS_STRATEGY_SIGNAL, OE, O1, O2, O3, O4)

// the per-edge kernel (boundary modes per edge, tree topologies): generic ops, and the
// workloads' linear pipelines at 128 items per ensemble specialised (the generic one's
// code overflows the instruction cache)
#define RS_KMIX(V) {-1, V, 0, 0, 0, 0, 0, (const void *)rs_pipeline_kernel<RS_STRATEGY_SIGNAL, V, GenericSig, true>, -1}
#define RS_KMIXS(V, OE, O1, O2, O3, O4) \
    {-1, V, OE, O1, O2, O3, O4, (const void *)rs_pipeline_kernel<RS_STRATEGY_SIGNAL, V, Sig<OE, O1, O2, O3, O4>, true>, -1}
#define RS_KMIXU(V, UM, OE, O1, O2, O3, O4)                                                                          \
    {-1, V, OE, O1, O2, O3, O4, (const void *)rs_pipeline_kernel<RS_STRATEGY_SIGNAL, V, Sig<OE, O1, O2, O3, O4>, true, UM>, \
     UM}

static const KEntry g_kernels[] = {
    RS_KMIX(1), RS_KMIX(2), RS_KMIX(4),
    // the cascade (three context hash filters) and the lines pipeline (two context hash
    // filters and a multiply-add map)
    RS_KMIXS(4, D_ENUM_LOAD, D_FILT_HASH_CTX, D_FILT_HASH_CTX, D_FILT_HASH_CTX, 0),
    RS_KMIXS(4, D_ENUM_LOAD, D_FILT_HASH_CTX, D_FILT_HASH_CTX, D_MAP_MULADD, 0),
    // ... with per-lane selection on every edge
    RS_KMIXU(4, EM_LANE, D_ENUM_LOAD, D_FILT_HASH_CTX, D_FILT_HASH_CTX, D_FILT_HASH_CTX, 0),
    RS_KMIXU(4, EM_LANE, D_ENUM_LOAD, D_FILT_HASH_CTX, D_FILT_HASH_CTX, D_MAP_MULADD, 0),
    // loaded elements -> three context hash filters -> aggregate
    RS_KBOTH(D_ENUM_LOAD, D_FILT_HASH_CTX, D_FILT_HASH_CTX, D_FILT_HASH_CTX, 0),
    // hashed elements -> power-of-two modulus filter -> multiply-add map -> aggregate
    RS_KBOTH(D_ENUM_HASH, D_FILT_MASK, D_MAP_MULADD, 0, 0),
    // loaded elements (edges) -> weight comparison -> aggregate
    RS_KBOTH(D_ENUM_LOAD, D_FILT_WEIGHT, 0, 0, 0),
    // loaded elements -> aggregate (the region-sum benchmark), 128 items per ensemble
    RS_KSIG(RS_STRATEGY_SIGNAL, 4, D_ENUM_LOAD, 0, 0, 0, 0),
    // any other stage list
    RS_KBOTH(0, 0, 0, 0, 0),
};

static const void *kernel_ptr(const KParams &P)
{
    int ops[5] = {0, 0, 0, 0, 0};
    ops[0] = (int)P.st[0].op;
    for (int i = 1; i < P.n_stages - 1 && i < 5; ++i) ops[i] = (int)P.st[i].op;
    if (P.mix) {
        // a specialised per-edge kernel serves a linear pipeline ending in the aggregate
        bool linear = P.n_sinks <= 1 && !P.emit;
        for (int i = 1; i < P.n_stages; ++i) linear = linear && P.up[i] == i - 1;
        // one mode on every edge: the kernel compiled for it, if any
        int um = P.n_stages > 1 ? (int)P.emode[1] : -1;
        for (int i = 2; i < P.n_stages; ++i)
            if ((int)P.emode[i] != um) um = -1;
        const void *generic = nullptr, *spec = nullptr;
        for (const KEntry &e : g_kernels) {
            if (e.strategy != -1 || e.V != (int)P.V) continue;
            if (e.oe == 0) {
                generic = e.fn;
            } else if (linear && e.oe == ops[0] && e.o1 == ops[1] && e.o2 == ops[2] && e.o3 == ops[3] &&
                       e.o4 == ops[4]) {
                if (e.um >= 0 && e.um == um) return e.fn;
                if (e.um < 0) spec = e.fn;
            }
        }
        return spec ? spec : generic;
    }
    if (P.strategy == RS_STRATEGY_TAG) return rs_tag_kernel_entry(P);
    const void *generic = nullptr;
    for (const KEntry &e : g_kernels) {
        if (e.strategy != P.strategy || e.V != (int)P.V) continue;
        if (e.oe == 0) {
            generic = e.fn;
            continue;
        }
        // specialised kernels end in the aggregate: an emit sink takes the generic one
        if (!P.emit && e.oe == ops[0] && e.o1 == ops[1] && e.o2 == ops[2] && e.o3 == ops[3] && e.o4 == ops[4])
            return e.fn;
    }
    return generic;
}

const void *rs_kernel_entry(const KParams &P) { return kernel_ptr(P); }

int rs_kernel_occupancy(const KParams &P, int block, size_t smem, int *blocks_per_sm)
{
    const void *f = kernel_ptr(P);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
    return (int)e;
}

int rs_kernel_max_smem_optin(const KParams &P, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(kernel_ptr(P), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return (int)e;
}

int rs_kernel_is_specialised(const KParams &P)
{
    if (P.strategy == RS_STRATEGY_TAG) return rs_tag_kernel_is_specialised(P);
    for (const KEntry &e : g_kernels)
        if (e.fn == kernel_ptr(P)) return e.oe != 0;
    return 0;
}

// ---------------------------------------------------------------------------
// Finalize: write the merged result of every parent that was processed in pieces.

__global__ void __launch_bounds__(256) rs_finalize_kernel(const __grid_constant__ KParams P)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (uint32_t si = 0; si < P.n_streams; ++si) {
        const DevStream &S = P.streams[si];
        if (S.mode != UNIT_MERGE || S.R == 0 || !S.finalize) continue;   // a sliced stream: after its last slice
        const uint32_t U = *S.u_count;
        for (uint32_t u = tid; u < U; u += nth) {
            const Slot sl = S.slots[u];
            if (sl.region == 0) continue;
            const uint32_t r = sl.region - 1;
            if (P.want_count) S.out_count[r] = sl.count;
            if (P.want_sum) S.out_sum[r] = sl.sum;
            if (P.want_min) S.out_min[r] = ~sl.min_inv;
            if (P.mix && P.n_sinks > 1) {
                // a tree's second leaf: its own slots, after the first leaf's
                const Slot s2 = S.slots[S.slot_units + u];
                if (P.want_count) S.out2_count[r] = s2.count;
                if (P.want_sum) S.out2_sum[r] = s2.sum;
                if (P.want_min) S.out2_min[r] = ~s2.min_inv;
            }
        }
    }
}

int rs_launch_finalize(const KParams &P, int grid, void *stream)
{
    void *args[] = {(void *)&P};
    cudaError_t e = cudaLaunchKernel((const void *)rs_finalize_kernel, dim3(grid), dim3(256), args, 0,
                                     (cudaStream_t)stream);
    return (int)e;
}

static const void *planner_ptr(const KParams &P)
{
    constexpr int BIG = RS_PLAN_TILE / 128, SMALL = RS_PLAN_TILE_SMALL / 128;
    static_assert(SMALL == 1, "small planner tiles hold one round");
    if (P.plan_tile == RS_PLAN_TILE_SMALL)
        return P.plan_pow2 ? (const void *)rs_plan_kernel<true, SMALL> : (const void *)rs_plan_kernel<false, SMALL>;
    return P.plan_pow2 ? (const void *)rs_plan_kernel<true, BIG> : (const void *)rs_plan_kernel<false, BIG>;
}

int rs_launch_planner(const KParams &P, int grid, void *stream)
{
    void *args[] = {(void *)&P};
    cudaError_t e = cudaLaunchKernel(planner_ptr(P), dim3(grid), dim3(256), args, 0,
                                     (cudaStream_t)stream);
    return (int)e;
}

int rs_launch_kernel(const KParams &P, int grid, int block, size_t smem, void *stream)
{
    const void *f = kernel_ptr(P);
    void *args[] = {(void *)&P};
    cudaError_t e = cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, (cudaStream_t)stream);
    return (int)e;
}
