// rs_tag.cuh -- the tag strategy (Section 2.3 and Section 5) on sm_103a: the engine and
// the kernel template, instantiated by rs_tag.cu and rs_tag2.cu.
//
// A persistent kernel in which every warp is one SIMD processor (Section 2.2) running
// the whole pipeline over the work units it claims with one global atomic ticket.
// Every queued item carries its region (its tag), so ensembles stay full across region
// boundaries and no signal queues exist.  Per processor:
//
//   * Node 1 reads the unit's elements in windows of W = 32 V consecutive positions.
//     Enumeration is zero-copy: the enumerate node's output queue is the element array
//     itself (getItem(i) of Section 4 is node 1's load).  A window is split into slices
//     of 32 VS positions; in each slice lane l takes VS consecutive positions.  They are
//     copied into a shared-memory ring of four windows by one 16-byte asynchronous copy
//     per lane and slice (cp.async), three windows ahead of node 1, so every copy
//     instruction of the warp reads one contiguous 512-byte row.
//   * The unit's parents are streamed in chunks of 32 CPL, CPL = 1 or 2 per lane (length
//     or CSR offsets, context word and id; two per lane halve the chunk loads when
//     regions are short on average).  A warp scan gives their offsets, and the non-empty
//     ones are appended to a small ring of parent records in shared memory: region id,
//     the value node 1's operation needs (context word or parent weight) and start
//     offset (plus the parent id for hashed enumeration).
//   * A window inside one parent takes its tag from registers.  A window that crosses
//     parent starts writes each start's record index at its position, and a warp
//     max-scan of these marks gives every position its parent.
//   * Nodes 2.. fire on full ensembles of W items taken from shared-memory rings of
//     64-bit {value, region} slots (Section 2.1's queues; a node fires only when its
//     output ring can take W times its maximum fan-out, Section 3.2).  The 0..1 outputs
//     of a filter or map are compacted slot by slot: each of the lane's V item slots is
//     placed by its own ballot, so a ring holds an ensemble's kept items in slot-major
//     order (an expansion's 0..k outputs keep item order, by one warp scan of the lanes'
//     output counts).  Tags along a ring are therefore not ordered; a one-region ensemble
//     is recognised by a warp vote.
//   * The aggregate (Section 4.2's begin/run/end per parent) folds each ensemble into
//     the region outputs with integer reductions: one per ensemble when it holds a
//     single region, otherwise one per run of equal tags in a lane.  count, sum and min
//     are associative and commutative, so the result is bit-exact in any order.  Every
//     region's output holds the identity result before its first fold: the planner
//     writes it for a region two units share (the one a unit starts inside), and the
//     processor whose unit owns a region writes it when it loads that region's parent,
//     before any fold into it; this also covers empty regions.  Folds are red.global
//     reductions (no value comes back).
//   * Enumeration straight into the aggregate (the region-sum stage list, compiled on its
//     own) needs no tag per item: runs of full windows inside one parent keep per-lane
//     partials and reduce once per run, and a window crossing parent starts folds each
//     region's piece as a difference of two warp prefix sums, or, when every start in it
//     falls on a lane boundary, each lane's items (which then lie in one region) at once.
//
// Rings and the parent stream are drained when a processor moves to a unit of another
// stream and when it runs out of units.  Nothing waits on another warp: the kernel has
// no spin loop, and every loop that depends on the input is bounded.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_device.cuh"

namespace {

constexpr uint32_t NONE = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long pack2(uint32_t lo, uint32_t hi)
{
    return ((unsigned long long)hi << 32) | lo;
}

// fmix32(x ^ c0) where c0s = c0 ^ (c0 >> 16): the first xor-shift distributes over the
// xor with the stage constant.  Two of the three right shifts are taken as the high
// word of a multiply by a power of two (m16 = 2^16, m19 = 2^19, so umulhi(h, m16) =
// h >> 16 and umulhi(h, m19) = h >> 13): they run on the multiply pipe, which the
// hash otherwise leaves idle, instead of the integer pipe that carries the rest.
__device__ __forceinline__ uint32_t fmix32_x(uint32_t x, uint32_t c0s, uint32_t m16, uint32_t m19)
{
    uint32_t h = x ^ __umulhi(x, m16) ^ c0s;
    h *= 0x85EBCA6Bu;
    h ^= __umulhi(h, m19);
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// fmix32 (MurmurHash3's 32-bit finalizer) with the same split of its shifts
__device__ __forceinline__ uint32_t fmix32_m(uint32_t h, uint32_t m16, uint32_t m19)
{
    h ^= __umulhi(h, m16);
    h *= 0x85EBCA6Bu;
    h ^= __umulhi(h, m19);
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// inclusive warp scan (sum): the shuffle's own predicate says whether the source lane
// exists, so each step is one shuffle and one predicated add
__device__ __forceinline__ uint32_t scan_add(uint32_t v)
{
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        asm("{\n\t.reg .b32 t;\n\t.reg .pred p;\n\t"
            "shfl.sync.up.b32 t|p, %0, %1, 0, -1;\n\t"
            "@p add.u32 %0, %0, t;\n\t}"
            : "+r"(v)
            : "r"(d));
    }
    return v;
}

// inclusive warp scan (max); a lane with no source lane gets its own value back,
// and max(v, v) = v
__device__ __forceinline__ uint32_t scan_max(uint32_t v)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) v = max(v, __shfl_up_sync(FULLMASK, v, d));
    return v;
}

// the stream being processed: what node 1 and the per-ensemble operands read, held in
// registers (the rest is read from the stream table when needed)
struct StreamRegs {
    const uint32_t *elements, *ctx;
    const uint32_t *meta;   // CSR offsets, or lengths
    uint32_t n_el;          // element count, clamped to 32 bits
    bool csr;               // meta holds offsets
    bool vec;               // elements 16-byte aligned: vector copies
};

// A claimed ticket: its stream and merge-path unit.
struct TicketUnit {
    uint32_t stream, rs, base, rend, j0, j1;
    bool valid, work, fill;
    // identity results this unit writes (merge-path units): its parents except the one it
    // starts inside (skip_head) and the one the next unit starts inside (skip_tail), which
    // the planner wrote
    bool own, skip_head, skip_tail;
};

// stream of ticket t: the last stream whose unit_base <= t, by a 32-way warp search
__device__ __forceinline__ uint32_t stream_of(const KParams &P, uint32_t t, uint32_t lane)
{
    uint32_t lo = 0, n = P.n_streams;
    while (n > 1) {
        const uint32_t step = (n + 31) / 32;
        const uint32_t idx = lo + lane * step;
        const bool le = idx < lo + n && P.streams[idx].unit_base <= t;
        const uint32_t b = __ballot_sync(FULLMASK, le);
        const uint32_t k = 31 - __clz(b | 1u);
        lo += k * step;
        n = min(step, n - k * step);
    }
    return lo;
}

// element offset of fixed-parent unit lu of a stream of lengths: its group's prefix plus
// the length sums of the units before it in the group (warp-collective, one read each)
__device__ __forceinline__ uint32_t usum_offset(const DevStream &S, uint32_t lu, uint32_t lane)
{
    const uint32_t g0 = lu & ~31u;
    const uint32_t v = (g0 + lane < lu) ? __ldg(S.usum + g0 + lane) : 0u;
    return __ldg(S.usum_grp + (lu >> 5)) + __reduce_add_sync(FULLMASK, v);
}

__device__ __forceinline__ TicketUnit describe(const KParams &P, uint32_t t, uint32_t lane)
{
    TicketUnit u;
    u.valid = t < P.total_units;
    u.work = u.fill = u.own = u.skip_head = u.skip_tail = false;
    u.stream = u.rs = u.base = u.rend = u.j0 = u.j1 = 0;
    if (!u.valid) return u;
    u.stream = stream_of(P, t, lane);
    const DevStream &S = P.streams[u.stream];
    const uint32_t lu = t - S.unit_base + S.slice_lo;
    if (S.mode == UNIT_REGIONS) {
        // K whole parents; their elements end where the last one ends
        u.rs = lu * S.K;
        u.rend = min(u.rs + S.K, S.R);
        // CSR offsets, or the fixed-parent units' offsets of a loaded stream of lengths;
        // hashed elements of a stream of lengths count positions from the unit's start
        u.base = S.offsets ? __ldg(S.offsets + u.rs) : (S.usum ? usum_offset(S, lu, lane) : 0u);
        u.j0 = u.base;
        u.j1 = NONE;
        u.fill = true;
        u.work = u.rs < u.rend;
        return u;
    }
    if (lu >= *S.u_count) return u;   // beyond the planner's units
    const UnitRec ra = S.rec[lu], rb = S.rec[lu + 1];
    u.j0 = ra.j;
    u.j1 = rb.j;
    const bool head = ra.j < ra.first_off;
    u.rs = head ? ra.i - 1 : ra.i;
    u.base = head ? ra.head_off : ra.first_off;
    u.rend = min(rb.i, S.R);
    u.own = P.plan_fill != 0;
    u.skip_head = head;
    u.skip_tail = rb.j < rb.first_off;
    if (u.j1 <= u.j0) return u;   // no elements: only identity results to write
    const bool bad = rb.i < ra.i || u.rs >= u.rend || (S.elements && u.j1 > S.n_elements);
    if (bad) {
        if (lane == 0) atomicOr(&P.hdr->status, ST_BAD_INPUT);
        return u;
    }
    u.work = true;
    return u;
}

// asynchronous 16-byte copy global -> shared of src_bytes (0..16) bytes, the rest of
// the 16 zero-filled (the source is 16-byte aligned); and its 4-byte form
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4z(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// st.shared of v at byte address a when k != 0, as one predicated store (no branch)
__device__ __forceinline__ void st_shared_if(uint32_t a, uint32_t v, uint32_t k)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.shared.u32 [%0], %1;\n\t}" ::"r"(a), "r"(v),
                 "r"(k)
                 : "memory");
}

// words p[r] and p[r + 1] of a read-only array (0 when not wanted): with VEC (r even),
// one 8-byte load when both are wanted and the array is 8-byte aligned, else one load each.
// The loads allocate in L1: the downstream nodes read the same context words by region.
template <bool VEC>
__device__ __forceinline__ void ld_pair(const uint32_t *p, uint32_t r, bool in0, bool in1, uint32_t &a, uint32_t &b)
{
    if (VEC && in0 && in1 && ((uintptr_t)p & 7u) == 0) {
        const uint2 v = ld_nc_v2(p + r);
        a = v.x;
        b = v.y;
    } else {
        a = in0 ? __ldg(p + r) : 0u;
        b = in1 ? __ldg(p + r + 1) : 0u;
    }
}

// node 1's element windows in flight per processor (a shared-memory ring of NB windows)
constexpr uint32_t NB = 4;   // a power of two (slot = window count & (NB - 1))

template <int V, class SG, int CPL>
struct TagEngine {
    static_assert(CPL == 1 || CPL == 2, "one or two parents per lane and chunk");
    static constexpr uint32_t CP = 32u * CPL;      // parents per chunk
    static constexpr int VS = V < 4 ? V : 4;       // consecutive positions per lane and slice
    static constexpr int NS = V / VS;              // slices per window
    static constexpr uint32_t SW = 32u * VS;       // positions per slice
    static constexpr uint32_t W = 32u * V;         // ensemble width

    const KParams &P;
    const uint32_t lane;
    const uint32_t wb;   // this processor's byte offset in dynamic shared memory
    // shared-memory arrays: byte offsets from the kernel parameters, so only wb lives in
    // a register
    // node statistics (32-bit per processor; a field about to pass 2^31 goes to the
    // header's 64-bit counters at once)
    __device__ __forceinline__ SArr<uint32_t> cnt() const { return sarr<uint32_t>(wb + P.L.o_cnt); }
    // the aggregate's pending fold (lane 0): region (NONE: none), count, min, then the sum
    __device__ __forceinline__ SArr<uint32_t> accw() const { return sarr<uint32_t>(wb + P.L.o_pend + 48); }
    __device__ __forceinline__ SArr<unsigned long long> accs() const
    {
        return sarr<unsigned long long>(wb + P.L.o_pend + 64);
    }
    __device__ __forceinline__ SArr<unsigned long long> nra() const { return sarr<unsigned long long>(wb + P.L.o_nra); }
    // ring slots {value, region tag}, 8 bytes each
    __device__ __forceinline__ SArr<uint2> rq() const { return sarr<uint2>(wb + P.L.o_qv); }
    __device__ __forceinline__ SArr<uint32_t> nst() const { return sarr<uint32_t>(wb + P.L.o_nst); }
    __device__ __forceinline__ SArr<uint32_t> npar() const { return sarr<uint32_t>(wb + P.L.o_npar); }
    // node 1's window marks: with loaded elements, the staging slot node 1 has just read
    // (free until the copy issued at the next window), else an array of their own
    __device__ __forceinline__ SArr<uint32_t> marks() const
    {
        return hashed() ? sarr<uint32_t>(wb + P.L.o_scr)
                        : sarr<uint32_t>(wb + P.L.o_tiles + ((wc - 1) & (NB - 1)) * W * 4);
    }
    __device__ __forceinline__ SArr<uint32_t> stg() const { return sarr<uint32_t>(wb + P.L.o_tiles); }
    __device__ __forceinline__ SArr<uint32_t> nxs() const { return sarr<uint32_t>(wb + P.L.o_pend); }
    // ring capacity and record-ring size (powers of two), from the kernel parameters
    __device__ __forceinline__ uint32_t C() const { return P.C; }
    __device__ __forceinline__ uint32_t CM() const { return P.C - 1; }
    __device__ __forceinline__ uint32_t PR() const { return P.L.pr; }
    __device__ __forceinline__ uint32_t PRM() const { return P.L.pr - 1; }

    // free-running cursors of the rings; edge e (node e -> node e + 1, e >= 1) is ring e - 1
    uint32_t qh[RS_MAX_STAGES], qt[RS_MAX_STAGES];
    StreamRegs S;
    uint32_t sidx;

    // the unit node 1 is reading: elements [j0, j1), next window at a
    uint32_t j0, j1, a;
    // its parent stream: next parent to load (cb), limit (re), offset of parent cb
    // (length streams), offset of the first parent not loaded yet (NONE: all loaded),
    // parent-record counters (free-running), the record node 1 is in, and the start of
    // the record after it (NONE while not loaded)
    uint32_t cb, re, cstart, load_start, ord_loaded, ord_cur, s_nx;
    uint32_t rlo;   // the unit's first parent (chunks start on multiples of CP parents)
    // windows [a, a + W) with a >= j0 and a + W <= flim are full, inside the current
    // parent and need no parent loads (flim = min(s_nx, j1, load_start))
    uint32_t flim, nfast;
    // node 1's staging ring: start of the next window to copy, windows copied and used
    uint32_t ia, wi, wc;
    uint32_t clim;   // elements below min(j1, element count): windows ending there copy whole
    // the next unit: its claimed ticket (lane 0) and, once described (during this unit's
    // last windows), its description
    uint32_t nt;
    bool nxt_done;
    uint32_t r_cur, aux_cur, st_cur, par_cur;
    // the next chunk, loaded ahead: this lane's parents cb + CPL lane (and, for CPL = 2,
    // the one after it): length or start offset (and the second's, which for CSR is also
    // the first's end), the second's end offset for CSR, context words, ids
    uint32_t pl0, pl0b, pl1b, pc, pcb, pp, ppb;
    // node statistics: lane k holds counter k (node k / 4, field k % 4: ensembles,
    // items, signals, firings), folded into shared memory after every unit
    uint32_t ctr;
    bool stop, unit_bad, fill;
    // identity results this unit writes: none (0), or its parents in [rlo + bit 1, re - bit 2)
    // (bit 0 set); whole-parent units write all of theirs
    uint32_t ownf;

    __device__ __forceinline__ TagEngine(const KParams &P_, uint32_t lane_, uint32_t wb_)
        : P(P_), lane(lane_), wb(wb_)
    {
#pragma unroll
        for (int e = 0; e < RS_MAX_STAGES; ++e) qh[e] = qt[e] = 0;
        sidx = NONE;
        j0 = j1 = a = 0;
        cb = re = cstart = rlo = 0;
        load_start = s_nx = NONE;
        flim = 0;
        nfast = 0;
        ia = wi = wc = 0;
        clim = 0;
        nt = 0;
        nxt_done = false;
        ord_loaded = ord_cur = 0;
        r_cur = aux_cur = st_cur = par_cur = 0;
        pl0 = pl0b = pl1b = pc = pcb = pp = ppb = 0;
        ctr = 0;
        stop = unit_bad = fill = false;
        ownf = 0;
        S.elements = S.ctx = S.meta = nullptr;
        S.n_el = 0;
        S.csr = S.vec = false;
    }

    __device__ __forceinline__ int n_st() const { return SG::generic ? P.n_stages : SG::n; }
    template <int I>
    __device__ __forceinline__ uint32_t op() const
    {
        if constexpr (SG::generic) return P.st[I].op;
        else return (uint32_t)SG::template op<I>();
    }
    __device__ __forceinline__ bool hashed() const { return op<0>() == D_ENUM_HASH; }
    template <int I>
    __device__ __forceinline__ uint32_t fanout() const
    {
        if (!SG::generic && SG::template op<I>() != (int)D_EXPAND) return 1u;
        return P.st[I].fanout;
    }

    // node I fired n_ens ensembles holding n_items items in one firing
    __device__ __forceinline__ void count_firing(int I, uint32_t n_ens, uint32_t n_items)
    {
        const uint32_t k = lane - 4u * I;
        ctr += k == 0 ? n_ens : (k == 1 ? n_items : (k == 3 ? 1u : 0u));
    }

    __device__ __forceinline__ void flush_counters()
    {
        if (lane < 4 * RS_MAX_STAGES) {
            uint32_t v = cnt()[lane];
            if (v + (unsigned long long)ctr >= (1ull << 31)) {
                atomicAdd(&P.hdr->counters[lane], (unsigned long long)v + ctr);
                v = 0;
            } else {
                v += ctr;
            }
            cnt()[lane] = v;
        }
        ctr = 0;
    }

    __device__ __forceinline__ const DevStream &D() const { return P.streams[sidx]; }

    __device__ __forceinline__ void set_stream(uint32_t si)
    {
        const DevStream &D = P.streams[si];
        S.elements = D.elements;
        S.ctx = D.ctx;
        S.csr = D.offsets != nullptr;
        S.meta = S.csr ? D.offsets : D.len;
        S.n_el = D.n_elements < 0xFFFFFFFFull ? (uint32_t)D.n_elements : 0xFFFFFFFFu;
        S.vec = D.tma_ok != 0;
        sidx = si;
    }

    // ---------------------------------------------------------------------------
    // parent stream (Section 4: findCount and getParent of each parent)

    // load this lane's parents of the chunk at cb (consumed by the next load_chunk);
    // chunks are aligned to CP parents, so each warp load reads whole 128-byte lines
    __device__ __forceinline__ void issue_chunk()
    {
        const uint32_t r = cb + CPL * lane;
        const bool in0 = r >= rlo && r < re, in1 = CPL == 2 && r + 1 >= rlo && r + 1 < re;
        if (S.csr) {
            // offsets r and r + 1 (the first parent's end, also the second's start), r + 2
            ld_pair<CPL == 2>(S.meta, r, in0, in0 || in1, pl0, pl0b);
            if (CPL == 2) pl1b = in1 ? __ldg(S.meta + r + 2) : 0u;
        } else {
            ld_pair<CPL == 2>(S.meta, r, in0, in1, pl0, pl0b);
        }
        const uint32_t o1 = op<1>();
        if (o1 == D_FILT_HASH_CTX && S.ctx) ld_pair<CPL == 2>(S.ctx, r, in0, in1, pc, pcb);
        if (o1 == D_FILT_WEIGHT || hashed()) {
            const uint32_t *pa = D().parents;
            if (pa) ld_pair<CPL == 2>(pa, r, in0, in1, pp, ppb);
        }
    }

    __device__ __forceinline__ void bad_unit()
    {
        if (lane == 0) atomicOr(&P.hdr->status, ST_BAD_INPUT);
        unit_bad = true;
        load_start = NONE;
    }

    // turn the loaded chunk into parent records (non-empty parents of the unit only); a
    // whole-parent unit (fill) also writes each parent's identity result
    __device__ __forceinline__ void load_chunk()
    {
        // consistent input never holds more records than one window's parents plus a
        // chunk (fewer than PR - CP before this load): anything else is inconsistent
        if (ord_loaded - ord_cur > PR() - CP) {
            bad_unit();
            return;
        }
        const uint32_t r = cb + CPL * lane;
        const bool in0 = r >= rlo && r < re, in1 = CPL == 2 && r + 1 >= rlo && r + 1 < re;
        uint32_t st0, L0, st1, L1;
        bool bad = false;
        if (S.csr) {
            st0 = pl0;
            L0 = pl0b - pl0;
            st1 = pl0b;
            L1 = pl1b - pl0b;
            bad = (in0 && pl0b < pl0) || (in1 && pl1b < pl0b);
        } else {
            L0 = in0 ? pl0 : 0u;
            L1 = in1 ? pl0b : 0u;
            const uint32_t s2 = L0 + L1;
            const uint32_t incl = scan_add(s2);
            st0 = cstart + incl - s2;
            st1 = st0 + L0;
            cstart += __shfl_sync(FULLMASK, incl, 31);
        }
        if (ownf) {
            const uint32_t lo_own = rlo + ((ownf >> 1) & 1u), hi_own = re - ((ownf >> 2) & 1u);
            if (in0 && r >= lo_own && r < hi_own) write_identity(r);
            if (in1 && r + 1 >= lo_own && r + 1 < hi_own) write_identity(r + 1);
        }
        // end of the chunk's last parent (the start of parent cb + nin)
        const uint32_t last = min(CP, re - cb) - 1;
        const uint32_t e_sel = (CPL == 2 && (last & 1u)) ? st1 + L1 : st0 + L0;
        const uint32_t end_last = __shfl_sync(FULLMASK, e_sel, last / CPL);
        const bool nz0 = in0 && !bad && L0 > 0 && st0 + L0 > j0 && st0 < j1;
        const bool nz1 = in1 && !bad && L1 > 0 && st1 + L1 > j0 && st1 < j1;
        const uint32_t b0 = __ballot_sync(FULLMASK, nz0), b1 = CPL == 2 ? __ballot_sync(FULLMASK, nz1) : 0u;
        if (nz0 || nz1) {
            // records in parent order: the lower lanes' parents, then this lane's first
            const uint32_t lt = lanemask_lt();
            const uint32_t o0 = ord_loaded + __popc(b0 & lt) + __popc(b1 & lt);
            const uint32_t o1r = o0 + (nz0 ? 1u : 0u);
            if (nz0) put_record(o0 & PRM(), r, st0, pc, pp);
            if (nz1) put_record(o1r & PRM(), r + 1, st1, pcb, ppb);
        }
        ord_loaded += __popc(b0) + __popc(b1);
        __syncwarp();   // records (and identity results) precede their readers
        if (__any_sync(FULLMASK, bad)) {
            bad_unit();
            return;
        }
        cb += CP;
        if (cb >= re) {
            if (j1 == NONE) j1 = end_last;   // a whole-parent unit ends with its last parent
            load_start = NONE;
        } else {
            // past the unit's last element only empty parents remain: loaded only when the
            // unit writes their identity results
            load_start = (end_last >= j1 && !(ownf & 1u)) ? NONE : end_last;
        }
        if (load_start != NONE) issue_chunk();
        if (s_nx == NONE && ord_cur + 1 != ord_loaded) s_nx = nst()[(ord_cur + 1) & PRM()];
        flim = min(min(s_nx, j1), load_start);
    }

    __device__ __forceinline__ void write_identity(uint32_t r) const
    {
        const DevStream &d = D();
        if (P.want_count) d.out_count[r] = 0u;
        if (P.want_sum) d.out_sum[r] = 0ull;
        if (P.want_min) d.out_min[r] = NONE;
    }

    // record o: region r starting at offset st, with node 1's operand from the context
    // word c or the parent id p
    __device__ __forceinline__ void put_record(uint32_t o, uint32_t r, uint32_t st, uint32_t c, uint32_t p)
    {
        const uint32_t o1 = op<1>();
        uint32_t aux = 0, par = 0;
        if (o1 == D_FILT_WEIGHT || hashed()) par = D().parents ? p : r;
        if (o1 == D_FILT_HASH_CTX) aux = S.ctx ? c : 0u;
        if (o1 == D_FILT_WEIGHT) aux = fmix32_x(par, P.st[1].c0s, P.m16, P.m19);
        nra()[o] = pack2(r, aux);
        nst()[o] = st;
        if (hashed()) npar()[o] = par;
    }

    // describe the next unit while this one still has work, so that the descriptor's
    // loads overlap this unit's last windows; the description waits in shared memory
    __device__ __forceinline__ void resolve_next()
    {
        const TicketUnit u = describe(P, __shfl_sync(FULLMASK, nt, 0), lane);
        if (lane == 0) {
            SArr<uint32_t> x = nxs();
            x[0] = u.stream;
            x[1] = u.rs;
            x[2] = u.base;
            x[3] = u.rend;
            x[4] = u.j0;
            x[5] = u.j1;
            x[6] = (u.valid ? 1u : 0u) | (u.work ? 2u : 0u) | (u.fill ? 4u : 0u) | (u.own ? 8u : 0u) |
                   (u.skip_head ? 16u : 0u) | (u.skip_tail ? 32u : 0u);
        }
        __syncwarp();
        nxt_done = true;
    }

    __device__ __forceinline__ TicketUnit next_unit()
    {
        if (!nxt_done) resolve_next();
        const SArr<uint32_t> x = nxs();
        TicketUnit u;
        u.stream = x[0];
        u.rs = x[1];
        u.base = x[2];
        u.rend = x[3];
        u.j0 = x[4];
        u.j1 = x[5];
        const uint32_t f = x[6];
        u.valid = f & 1u;
        u.work = f & 2u;
        u.fill = f & 4u;
        u.own = f & 8u;
        u.skip_head = f & 16u;
        u.skip_tail = f & 32u;
        __syncwarp();
        return u;
    }

    // make record o the current one
    __device__ __forceinline__ void take_record(uint32_t o)
    {
        ord_cur = o;
        const uint32_t i = o & PRM();
        const unsigned long long e = nra()[i];
        r_cur = (uint32_t)e;
        aux_cur = (uint32_t)(e >> 32);
        if (hashed()) {
            st_cur = nst()[i];
            par_cur = npar()[i];
        }
        s_nx = (o + 1 != ord_loaded) ? nst()[(o + 1) & PRM()] : NONE;
        flim = min(min(s_nx, j1), load_start);
    }

    // ---------------------------------------------------------------------------
    // node 1's element loads

    // copy the next window's elements (this lane's VS positions of every slice) into its
    // slot of the staging ring; positions past the unit's end or the array are
    // zero-filled (they are never valid).  One commit group per window, empty ones too.
    __device__ __forceinline__ void issue_window()
    {
        const uint32_t wa = ia;
        const uint32_t sb = smem_addr(stg().ptr() + (wi & (NB - 1)) * W);
        if (VS == 4 && S.vec && wa + W <= clim) {
            // the whole window lies inside the unit and the array: plain 16-byte copies
#pragma unroll
            for (int t = 0; t < NS; ++t)
                cp_async16(sb + 4u * (t * SW + VS * lane), S.elements + wa + t * SW + VS * lane, 16u);
        } else if (wa < j1) {
            const uint32_t lim = min(j1, S.n_el);
#pragma unroll
            for (int t = 0; t < NS; ++t) {
                const uint32_t e = wa + t * SW + VS * lane;
                const uint32_t n = e < lim ? min(lim - e, (uint32_t)VS) : 0u;
                const uint32_t dst = sb + 4u * (t * SW + VS * lane);
                if (VS == 4 && S.vec) {
                    cp_async16(dst, n ? S.elements + e : S.elements, 4u * n);
                } else {
#pragma unroll
                    for (int i = 0; i < VS; ++i)
                        cp_async4z(dst + 4u * i, (uint32_t)i < n ? S.elements + e + i : S.elements, (uint32_t)i < n ? 4u : 0u);
                }
            }
        }
        cp_async_commit();
        ia += W;
        ++wi;
    }

    // this lane's elements of the current window (its copy group has landed: the lane
    // reads only what it copied itself)
    __device__ __forceinline__ void staged_window(uint32_t (&x)[V])
    {
        issue_window();
        cp_async_wait<NB - 1>();
        const uint32_t *sp = stg().ptr() + (wc & (NB - 1)) * W;
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            if constexpr (VS == 4) {
                const uint4 v = *reinterpret_cast<const uint4 *>(sp + t * SW + VS * lane);
                x[t * VS + 0] = v.x;
                x[t * VS + 1 % VS] = v.y;
                x[t * VS + 2 % VS] = v.z;
                x[t * VS + 3 % VS] = v.w;
            } else {
#pragma unroll
                for (int i = 0; i < VS; ++i) x[t * VS + i] = sp[t * SW + VS * lane + i];
            }
        }
        ++wc;
    }

    // ---------------------------------------------------------------------------
    // stage operations (Section 2.1: 0..k outputs per input)

    template <int I>
    __device__ __forceinline__ void apply(const uint32_t (&x)[V], const uint32_t (&aux)[V], const bool (&valid)[V],
                                          bool (&keep)[V], uint32_t (&y)[V]) const
    {
        const DevStage &sd = P.st[I];
        const uint32_t opc = op<I>();
#pragma unroll
        for (int j = 0; j < V; ++j) {
            bool kp;
            uint32_t ys = x[j];
            switch (opc) {
            case D_FILT_MASK: kp = (x[j] & sd.p0) == sd.p1; break;
            case D_FILT_MOD: kp = (x[j] % sd.p0) == sd.p1; break;
            case D_FILT_HASH_CTX: kp = (fmix32_x(x[j], sd.c0s, P.m16, P.m19) ^ aux[j]) < sd.p1; break;
            case D_FILT_WEIGHT: kp = fmix32_x(x[j], sd.c0s, P.m16, P.m19) < aux[j]; break;
            case D_MAP_MULADD: ys = x[j] * sd.p0 + sd.p1; kp = true; break;
            default: kp = false; break;
            }
            keep[j] = kp && valid[j];
            y[j] = ys;
        }
    }

    // Append kept items to the ring of edge I, slot by slot: the kept items of slot j of
    // all lanes take the next consecutive slots, in lane order, placed by one ballot (the
    // lanes' earlier kept items of that slot) and one popcount (all of them).  The caller
    // guarantees room for W items.
    template <int I>
    __device__ __forceinline__ void push(const bool (&keep)[V], const uint32_t (&y)[V], const uint32_t (&r)[V])
    {
        const uint32_t lt = lanemask_lt();
        const uint32_t qb = smem_addr(rq().ptr()) + 8u * (I - 1) * C();
        const uint32_t cm = CM();
        uint32_t t = qt[I];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const uint32_t b = __ballot_sync(FULLMASK, keep[j]);
            if (keep[j]) {
                const uint32_t qa = qb + 8u * ((t + __popc(b & lt)) & cm);
                asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(qa), "r"(y[j]), "r"(r[j]) : "memory");
            }
            t += __popc(b);
        }
        qt[I] = t;
    }

    // node I's kept items: into the ring of edge I, or, when node I is the last node
    // before the aggregate and not an expansion, straight into the aggregate (no ring on
    // that edge; the aggregate fires once per ensemble of node I, on its kept items)
    template <int I, int NG, int GV>
    __device__ __forceinline__ void emit(const bool (&keep)[V], const uint32_t (&y)[V], const uint32_t (&r)[V],
                                         bool uni, uint32_t r0)
    {
        if (I == n_st() - 2) {
            uint32_t k = 0;
#pragma unroll
            for (int j = 0; j < V; ++j) k += keep[j] ? 1u : 0u;
            const uint32_t n = __reduce_add_sync(FULLMASK, k);
            aggregate(y, r, keep, uni, r0, n);
            count_firing(I + 1, 1u, n);
        } else {
            push<I>(keep, y, r);
        }
    }

    // expansion (0..fanout outputs per item): item x emits n = hash32(x, p0) mod
    // (fanout + 1) values hash32(x, p0 + 1 + i), i < n, in order
    template <int I, int NG, int GV>
    __device__ __forceinline__ void expand(const uint32_t (&x)[V], const uint32_t (&r)[V], const bool (&valid)[V])
    {
        const DevStage &sd = P.st[I];
        const uint32_t rb = (I - 1) * C();
        uint32_t nout[V], c = 0;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            nout[j] = valid[j] ? fmix32_x(x[j], sd.c0s, P.m16, P.m19) % (sd.fanout + 1u) : 0u;
            c += nout[j] << (16 * (j / GV));
        }
        const uint32_t incl = scan_add(c);
        const uint32_t tot = __shfl_sync(FULLMASK, incl, 31);
        const uint32_t ex = incl - c;
        uint32_t gb = qt[I];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            uint32_t pos = gb + ((ex >> (16 * g)) & 0xFFFFu);
#pragma unroll
            for (int i = 0; i < GV; ++i) {
                const int j = g * GV + i;
                for (uint32_t o = 0; o < nout[j]; ++o) {
                    const uint32_t yv = fmix32(x[j] ^ fmix32((sd.p0 + 1u + o) ^ RS_GOLD));
                    rq()[rb + (pos & CM())] = make_uint2(yv, r[j]);
                    ++pos;
                }
            }
            gb += (tot >> (16 * g)) & 0xFFFFu;
        }
        qt[I] = gb;
    }

    __device__ __forceinline__ void fold(uint32_t rr, uint32_t n, unsigned long long s, uint32_t mn) const
    {
        const DevStream &d = D();
        if (P.want_count) red_add_u32(d.out_count + rr, n);
        if (P.want_sum) red_add_u64(d.out_sum + rr, s);
        if (P.want_min) red_min_u32(d.out_min + rr, mn);
    }

    // One-region ensembles fold into the processor's pending fold (lane 0, shared memory),
    // which goes to the region's outputs when an ensemble of another region arrives and
    // before the processor changes stream or finishes: a region long enough to span many
    // ensembles costs one atomic per output per processor and run of its ensembles, not
    // one per ensemble (with one region in a whole stream, every processor's folds would
    // otherwise meet on one address).  Deferring a fold keeps it after the region's
    // identity result: the owner writes that when it loads the parent, before any item
    // of it, and the planner before the kernel for a region two units share.
    __device__ __forceinline__ void acc_add(uint32_t rr, uint32_t n, unsigned long long s, uint32_t mn) const
    {
        const uint32_t ar = accw()[0];
        if (ar == rr) {
            accw()[1] += n;
            accs()[0] += s;
            accw()[2] = min(accw()[2], mn);
        } else {
            if (ar != NONE) fold(ar, accw()[1], accs()[0], accw()[2]);
            accw()[0] = rr;
            accw()[1] = n;
            accs()[0] = s;
            accw()[2] = mn;
        }
    }

    // the pending fold to the outputs (warp-collective; lane 0 holds it)
    __device__ __forceinline__ void acc_flush() const
    {
        if (lane == 0) {
            const uint32_t ar = accw()[0];
            if (ar != NONE) fold(ar, accw()[1], accs()[0], accw()[2]);
            accw()[0] = NONE;
        }
        __syncwarp();
    }

    // one emitted value at position pos of the stream's value array (bounds-checked)
    __device__ __forceinline__ void put_value(const DevStream &d, unsigned long long pos, uint32_t v) const
    {
        if (pos < d.out_values_len) d.out_values[pos] = v;
        else atomicOr(&P.hdr->status, ST_BAD_INPUT);
    }

    // the emit sink (Section 4: results derived from single elements, stripped of their
    // parent): each kept value goes to its region's segment of the value array, at a
    // position claimed by an atomic add on the region's count (zeroed before the run), so
    // a region's values keep no particular order.  A one-region ensemble claims all its
    // positions with one atomic and places the values by a warp prefix.
    __device__ __forceinline__ void emit_values(const uint32_t (&x)[V], const uint32_t (&r)[V],
                                                const bool (&valid)[V], bool uni, uint32_t r0, uint32_t n_valid) const
    {
        const DevStream &d = D();
        const uint32_t o0 = __ldg(d.offsets);
        if (uni) {
            if (n_valid == 0) return;
            uint32_t c = 0;
#pragma unroll
            for (int j = 0; j < V; ++j) c += valid[j] ? 1u : 0u;
            const uint32_t incl = scan_add(c);
            uint32_t base = 0, seg = 0;
            if (lane == 0) {
                base = atomicAdd(d.out_count + r0, n_valid);
                seg = __ldg(d.offsets + r0) - o0;
            }
            base = __shfl_sync(FULLMASK, base, 0);
            seg = __shfl_sync(FULLMASK, seg, 0);
            unsigned long long pos = (unsigned long long)P.emit_f * seg + base + (incl - c);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                if (valid[j]) {
                    put_value(d, pos, x[j]);
                    ++pos;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                if (valid[j]) {
                    const uint32_t b = atomicAdd(d.out_count + r[j], 1u);
                    put_value(d, (unsigned long long)P.emit_f * (__ldg(d.offsets + r[j]) - o0) + b, x[j]);
                }
            }
        }
    }

    // the aggregate (Section 4.2): count, sum and min of each region's surviving items
    // (or, for an emit sink, the items themselves)
    __device__ __forceinline__ void aggregate(const uint32_t (&x)[V], const uint32_t (&r)[V], const bool (&valid)[V],
                                              bool uni, uint32_t r0, uint32_t n_valid) const
    {
        if ((SG::generic && P.emit) || SG::emit) {
            emit_values(x, r, valid, uni, r0, n_valid);
            return;
        }
        if (uni) {
            uint32_t lo = 0, hi = 0, mn = NONE;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                if (valid[j]) {
                    lo += x[j] & 0xFFFFu;
                    hi += x[j] >> 16;
                    mn = min(mn, x[j]);
                }
            }
            if (P.want_sum) {
                lo = __reduce_add_sync(FULLMASK, lo);
                hi = __reduce_add_sync(FULLMASK, hi);
            }
            if (P.want_min) mn = __reduce_min_sync(FULLMASK, mn);
            if (lane == 0 && n_valid) acc_add(r0, n_valid, ((unsigned long long)hi << 16) + lo, mn);
        } else {
            // runs of equal consecutive tags among the lane's items (any order of regions:
            // the reductions commute)
            uint32_t cr = NONE, cn = 0, cm = NONE;
            unsigned long long cs = 0;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                if (valid[j]) {
                    if (r[j] != cr) {
                        if (cn) fold(cr, cn, cs, cm);
                        cr = r[j];
                        cn = 0;
                        cs = 0;
                        cm = NONE;
                    }
                    cn++;
                    cs += x[j];
                    cm = min(cm, x[j]);
                }
            }
            if (cn) fold(cr, cn, cs, cm);
        }
    }

    // the value node I's operation needs per item, from its region (nodes >= 2)
    template <int I>
    __device__ __forceinline__ void aux_of(const uint32_t (&r)[V], const bool (&valid)[V], bool uni, uint32_t r0,
                                           uint32_t (&aux)[V]) const
    {
        const uint32_t opc = op<I>();
#pragma unroll
        for (int j = 0; j < V; ++j) aux[j] = 0;
        if (opc == D_FILT_HASH_CTX) {
            if (!S.ctx) return;
            if (uni) {
                const uint32_t c = __ldg(S.ctx + r0);
#pragma unroll
                for (int j = 0; j < V; ++j) aux[j] = c;
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (valid[j]) aux[j] = __ldg(S.ctx + r[j]);
            }
        } else if (opc == D_FILT_WEIGHT) {
            const uint32_t c0s = P.st[I].c0s;
            if (uni) {
                const uint32_t *pa = D().parents;
                const uint32_t w = fmix32_x(pa ? __ldg(pa + r0) : r0, c0s, P.m16, P.m19);
#pragma unroll
                for (int j = 0; j < V; ++j) aux[j] = w;
            } else {
                const uint32_t *pa = D().parents;
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (valid[j]) aux[j] = fmix32_x(pa ? __ldg(pa + r[j]) : r[j], c0s, P.m16, P.m19);
            }
        }
    }

    // ---------------------------------------------------------------------------
    // node 1's steady state: a window that is full, inside the current parent and needs
    // no parent loads (a >= j0, a + W <= flim)

    __device__ __forceinline__ void fast_window()
    {
        uint32_t x[V], r[V], aux[V];
        bool valid[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            r[j] = r_cur;
            aux[j] = aux_cur;
            valid[j] = true;
        }
        if (hashed()) {
#pragma unroll
            for (int t = 0; t < NS; ++t)
#pragma unroll
                for (int i = 0; i < VS; ++i) {
                    const uint32_t p = a + t * SW + VS * lane + i;
                    x[t * VS + i] = fmix32_m(par_cur ^ fmix32_m((p - st_cur) ^ RS_GOLD, P.m16, P.m19), P.m16, P.m19);
                }
        } else {
            staged_window(x);
        }
        if (n_st() == 2) {
            if constexpr (SG::template maybe_last<1>()) aggregate(x, r, valid, true, r_cur, W);
        } else {
            if constexpr (SG::template maybe_elem<1>()) {
                if (op<1>() == D_EXPAND) {
                    expand<1, NS, VS>(x, r, valid);
                } else {
                    uint32_t y[V];
                    bool keep[V];
                    apply<1>(x, aux, valid, keep, y);
                    emit<1, NS, VS>(keep, y, r, true, r_cur);
                }
            }
        }
        a += W;
        ++nfast;
    }

    // Enumeration straight into the aggregate (loaded elements, two nodes): a run of full
    // windows inside the current parent.  Each lane keeps its own 64-bit sum (and minimum)
    // across the run; the warp reduces them and folds into the pending fold once per run,
    // not once per window.  Every window of the run is full, so the count is the run's
    // window count times W.  The run stops where the fast windows end and, while the next
    // unit is still to be described, 8 windows before the unit's end, as step() does.
    static constexpr bool RUN = !SG::generic && SG::n == 2 && !SG::emit && SG::template op<0>() == D_ENUM_LOAD;

    template <bool MIN>
    __device__ __forceinline__ void fast_run()
    {
        unsigned long long s = 0;
        uint32_t mn = NONE, k = 0;
        // the last window start of the run: a + W <= flim and, while the next unit is
        // undescribed, a + 8 W < j1 (neither bound moves during the run)
        uint32_t lim = flim - W;
        if (!nxt_done) lim = min(lim, j1 > 8 * W ? j1 - 8 * W - 1 : 0u);
        do {
            uint32_t x[V];
            staged_window(x);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                s += x[j];
                if (MIN) mn = min(mn, x[j]);
            }
            a += W;
            ++k;
        } while (a <= lim);
        nfast += k;
        s = warp_sum_u64(s);
        if (MIN) mn = __reduce_min_sync(FULLMASK, mn);
        if (lane == 0) acc_add(r_cur, k * W, s, mn);
    }

    // Enumeration straight into the aggregate over a window that crosses parent starts
    // (count and sum; lanes hold consecutive positions): no region id per item.  Lane k
    // reads the start of record ord_cur + k (the current record's piece starts at lo).
    //   * Every start on a lane boundary: each lane's V items lie in one region, the
    //     record of the last start at or below the lane's first position (a count of the
    //     lanes holding a start, from one OR-reduction of their bits), and the lane folds
    //     its valid items' count and sum.
    //   * Otherwise, inclusive prefix sums over the window's positions, of the values' low
    //     and high 16-bit halves, go one after the other through the window's staging slot
    //     (free until the next copy); each region's piece of the window,
    //     [max(start, lo), min(next start, hi)), is the difference of two prefix values,
    //     and one lane per piece folds it: one fold per region and window.
    // A window with more than 32 pieces is left to node1's general path: returns false
    // before touching anything.
    __device__ __forceinline__ bool agg_window(const uint32_t (&x)[V], uint32_t lo, uint32_t hi)
    {
        static_assert(NS == 1, "positions a + V lane + i");
        const uint32_t nrec = ord_loaded - ord_cur, o = ord_cur + lane;
        const uint32_t st = lane == 0 ? lo : (lane < nrec ? nst()[o & PRM()] : NONE);
        const bool w = st < hi;
        const uint32_t bw = __ballot_sync(FULLMASK, w);
        if (bw >> 31) return false;
        ctr += (lane == 0 || lane == 4 || lane == 7) ? 1u : (lane == 5 ? hi - lo : 0u);
        // record k >= 1 starts in (lo, hi): on a lane boundary, at lane (st - a) / V in 1..31
        const uint32_t d = st - a;
        if (__all_sync(FULLMASK, !w || lane == 0 || (d & (V - 1)) == 0)) {
            const uint32_t m = __reduce_or_sync(FULLMASK, (w && lane > 0) ? 1u << (d / V) : 0u);
            const uint32_t rel = __popc(m & (FULLMASK >> (31 - lane)));
            uint32_t n = 0;
            unsigned long long sum = 0;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const uint32_t p = a + V * lane + i;
                const bool in = p >= lo && p < hi;
                n += in ? 1u : 0u;
                sum += in ? x[i] : 0u;
            }
            if (n) fold((uint32_t)nra()[(ord_cur + rel) & PRM()], n, sum, NONE);
        } else {
            // inclusive prefixes of both halves at the lane's positions (invalid ones add 0)
            uint32_t pl[V], ph[V];
            uint32_t cl = 0, ch = 0;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const uint32_t p = a + V * lane + i;
                const uint32_t v = (p >= lo && p < hi) ? x[i] : 0u;
                cl += v & 0xFFFFu;
                ch += v >> 16;
                pl[i] = cl;
                ph[i] = ch;
            }
            const uint32_t il = scan_add(cl), ih = scan_add(ch);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                pl[i] += il - cl;
                ph[i] += ih - ch;
            }
            const uint32_t s = max(st, lo);
            const uint32_t e = (w && lane + 1 < nrec) ? min(hi, nst()[(o + 1) & PRM()]) : hi;
            const bool piece = w && e > s;
            uint32_t sl = 0, sh = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __syncwarp();
                uint32_t q[V];
#pragma unroll
                for (int i = 0; i < V; ++i) q[i] = h ? ph[i] : pl[i];
                if constexpr (V == 4) {
                    reinterpret_cast<uint4 *>(marks().ptr())[lane] = make_uint4(q[0], q[1 % V], q[2 % V], q[3 % V]);
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i) marks()[V * lane + i] = q[i];
                }
                __syncwarp();
                if (piece) {
                    const uint32_t df = marks()[e - 1 - a] - (s > a ? marks()[s - 1 - a] : 0u);
                    if (h) sh = df;
                    else sl = df;
                }
            }
            if (piece) fold((uint32_t)nra()[o & PRM()], e - s, ((unsigned long long)sh << 16) + sl, NONE);
        }
        __syncwarp();
        // the last record starting before hi becomes the current one
        take_record(ord_cur + 31 - __clz(bw));
        a += W;
        return true;
    }

    // ---------------------------------------------------------------------------
    // node 1: the window [a, a + W) of the unit (any case: partial windows, parent
    // starts inside the window, parents still to load)

    __device__ __forceinline__ void node1()
    {
        // every parent starting before the window's end is loaded (for a whole-parent
        // unit this also finds the unit's end once its last parent is loaded)
        while (load_start < a + W) {
            load_chunk();
            if (unit_bad) {
                a = NONE;
                return;
            }
        }
        if (a >= j1) return;
        // the elements (getItem of Section 4); loaded ones first, so that the marks can
        // take the staging slot they came from
        uint32_t x[V];
        if (!hashed()) staged_window(x);
        const uint32_t lo = max(a, j0), hi = min(a + W, j1);
        uint32_t r[V], aux[V], st[V], par[V];
        const bool uni = s_nx >= hi;
        if constexpr (RUN && NS == 1) {
            if (!uni && !P.want_min && agg_window(x, lo, hi)) return;
        }
        if (uni) {
            // every position of the window lies in the current parent
#pragma unroll
            for (int j = 0; j < V; ++j) {
                r[j] = r_cur;
                aux[j] = aux_cur;
                st[j] = st_cur;
                par[j] = par_cur;
            }
        } else {
            // mark each parent start in the window with its record index (relative to
            // the current record), then a running maximum gives each position's parent
            __syncwarp();
            uint4 *mk = reinterpret_cast<uint4 *>(marks().ptr());
#pragma unroll
            for (uint32_t k = 0; k < W / 128; ++k) mk[k * 32 + lane] = make_uint4(0u, 0u, 0u, 0u);
            if constexpr (W < 128) {
                if (lane < W / 4) mk[lane] = make_uint4(0u, 0u, 0u, 0u);
            }
            __syncwarp();
            const uint32_t nx = ord_cur + 1;
            for (uint32_t base = nx;; base += 32) {
                const uint32_t o = base + lane;
                const bool in = (o - nx) < (ord_loaded - nx);
                const uint32_t s = in ? nst()[o & PRM()] : NONE;
                const bool w = s < hi;
                if (w && s >= a) marks()[s - a] = o - ord_cur;
                if (!__shfl_sync(FULLMASK, w, 31)) break;
            }
            __syncwarp();
            uint32_t rel[V];
            uint32_t carry = 0;
#pragma unroll
            for (int t = 0; t < NS; ++t) {
                uint32_t m[VS];
                const uint32_t mo = t * SW + VS * lane;
                if constexpr (VS == 4) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(marks().ptr() + mo);
                    m[0] = v.x;
                    m[1 % VS] = v.y;
                    m[2 % VS] = v.z;
                    m[3 % VS] = v.w;
                } else if constexpr (VS == 2) {
                    const uint2 v = *reinterpret_cast<const uint2 *>(marks().ptr() + mo);
                    m[0] = v.x;
                    m[1 % VS] = v.y;
                } else {
                    m[0] = marks()[mo];
                }
                uint32_t lm = m[0];
#pragma unroll
                for (int i = 1; i < VS; ++i) lm = max(lm, m[i]);
                const uint32_t incl = scan_max(lm);
                const uint32_t ex = __shfl_up_sync(FULLMASK, incl, 1);
                uint32_t c = max(carry, lane ? ex : 0u);
#pragma unroll
                for (int i = 0; i < VS; ++i) {
                    c = max(c, m[i]);
                    rel[t * VS + i] = c;
                }
                carry = max(carry, __shfl_sync(FULLMASK, incl, 31));
            }
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const unsigned long long e = nra()[(ord_cur + rel[j]) & PRM()];
                r[j] = (uint32_t)e;
                aux[j] = (uint32_t)(e >> 32);
                if (hashed()) {
                    st[j] = nst()[(ord_cur + rel[j]) & PRM()];
                    par[j] = npar()[(ord_cur + rel[j]) & PRM()];
                } else {
                    st[j] = par[j] = 0;
                }
            }
            take_record(ord_cur + carry);
        }
        // valid positions: all of them except in a unit's first and last windows
        bool valid[V];
        if (lo == a && hi == a + W) {
#pragma unroll
            for (int j = 0; j < V; ++j) valid[j] = true;
        } else {
#pragma unroll
            for (int t = 0; t < NS; ++t)
#pragma unroll
                for (int i = 0; i < VS; ++i) {
                    const uint32_t p = a + t * SW + VS * lane + i;
                    valid[t * VS + i] = p >= lo && p < hi;
                }
        }
        if (hashed()) {
#pragma unroll
            for (int t = 0; t < NS; ++t)
#pragma unroll
                for (int i = 0; i < VS; ++i) {
                    const int j = t * VS + i;
                    const uint32_t p = a + t * SW + VS * lane + i;
                    x[j] = valid[j] ? fmix32_m(par[j] ^ fmix32_m((p - st[j]) ^ RS_GOLD, P.m16, P.m19), P.m16, P.m19) : 0u;
                }
        }
        const uint32_t n_valid = hi - lo;
        // node 0 and node 1 each ran one ensemble; node 1 consumed n_valid items in one firing
        ctr += (lane == 0 || lane == 4 || lane == 7) ? 1u : (lane == 5 ? n_valid : 0u);
        // node 1's operation; with a two-stage pipeline node 1 is the aggregate
        if (n_st() == 2) {
            if constexpr (SG::template maybe_last<1>()) aggregate(x, r, valid, uni, r_cur, n_valid);
        } else {
            if constexpr (SG::template maybe_elem<1>()) {
                if (op<1>() == D_EXPAND) {
                    expand<1, NS, VS>(x, r, valid);
                } else {
                    uint32_t y[V];
                    bool keep[V];
                    apply<1>(x, aux, valid, keep, y);
                    emit<1, NS, VS>(keep, y, r, uni, r_cur);
                }
            }
        }
        a += W;
    }

    // ---------------------------------------------------------------------------
    // nodes I >= 2: ensembles from the ring of edge I - 1

    // ensemble of node I: `take` items at the head of the ring of edge I - 1 (FULL: take
    // == W and the head is V-aligned, as in every non-draining firing)
    template <int I, bool FULL>
    __device__ __forceinline__ void gather(uint32_t take, uint32_t (&x)[V], uint32_t (&r)[V], bool (&valid)[V],
                                           bool &uni, uint32_t &r0) const
    {
        const uint32_t rb = (I - 2) * C();
        const uint32_t h = qh[I - 1];
        if (FULL || (h & (V - 1)) == 0) {
            // the lane's V slots are contiguous (C is a multiple of V)
            const uint32_t s = rb + ((h + V * lane) & CM());
            // two slots per 16-byte load (s is even: h and C are multiples of V)
            if constexpr (VS == 4) {
#pragma unroll
                for (int t = 0; t < NS; ++t) {
                    const uint4 p0 = *reinterpret_cast<const uint4 *>(rq().ptr() + s + 4 * t);
                    const uint4 p1 = *reinterpret_cast<const uint4 *>(rq().ptr() + s + 4 * t + 2);
                    x[4 * t + 0] = p0.x;
                    r[4 * t + 0] = p0.y;
                    x[4 * t + 1 % V] = p0.z;
                    r[4 * t + 1 % V] = p0.w;
                    x[4 * t + 2 % V] = p1.x;
                    r[4 * t + 2 % V] = p1.y;
                    x[4 * t + 3 % V] = p1.z;
                    r[4 * t + 3 % V] = p1.w;
                }
            } else if constexpr (VS == 2) {
                const uint4 p0 = *reinterpret_cast<const uint4 *>(rq().ptr() + s);
                x[0] = p0.x;
                r[0] = p0.y;
                x[1 % V] = p0.z;
                r[1 % V] = p0.w;
            } else {
                const uint2 p0 = rq()[s];
                x[0] = p0.x;
                r[0] = p0.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const uint2 p0 = rq()[rb + ((h + V * lane + j) & CM())];
                x[j] = p0.x;
                r[j] = p0.y;
            }
        }
#pragma unroll
        for (int j = 0; j < V; ++j) valid[j] = FULL || V * lane + j < take;
        // one region: every valid item carries the first item's tag (a warp vote; tags along
        // a ring are in slot-major order of each pushed ensemble, not sorted)
        r0 = __shfl_sync(FULLMASK, r[0], 0);
        bool same = true;
#pragma unroll
        for (int j = 0; j < V; ++j) same = same && (!valid[j] || r[j] == r0);
        uni = __all_sync(FULLMASK, same);
    }

    template <int I, bool FULL>
    __device__ __forceinline__ void ensemble(uint32_t take)
    {
        uint32_t x[V], r[V], r0;
        bool valid[V], uni;
        gather<I, FULL>(take, x, r, valid, uni, r0);
        if (I == n_st() - 1) {
            if constexpr (SG::template maybe_last<I>()) aggregate(x, r, valid, uni, r0, take);
        } else {
            if constexpr (SG::template maybe_elem<I>()) {
                if (op<I>() == D_EXPAND) {
                    expand<I, 1, V>(x, r, valid);
                } else {
                    uint32_t aux[V], y[V];
                    bool keep[V];
                    aux_of<I>(r, valid, uni, r0, aux);
                    apply<I>(x, aux, valid, keep, y);
                    emit<I, 1, V>(keep, y, r, uni, r0);
                }
            }
        }
    }

    // node I fires on full ensembles while its input holds one and its output has room
    template <int I>
    __device__ __forceinline__ void fire()
    {
        if constexpr (SG::template present<I>() && I < RS_MAX_STAGES) {
            if (I >= n_st()) return;
            const bool last = I == n_st() - 1;
            const uint32_t need = W * fanout<I>();
            uint32_t n_ens = 0;
            while (qt[I - 1] - qh[I - 1] >= W && (last || C() - (qt[I] - qh[I]) >= need)) {
                ensemble<I, true>(W);
                qh[I - 1] += W;
                ++n_ens;
            }
            if (n_ens) count_firing(I, n_ens, n_ens * W);
        }
    }

    // node I fires on whatever its input holds (partial ensembles), while its output has
    // room; a drained ring restarts on a V-aligned slot
    template <int I>
    __device__ __forceinline__ void fire_drain()
    {
        if constexpr (SG::template present<I>() && I < RS_MAX_STAGES) {
            if (I >= n_st()) return;
            const bool last = I == n_st() - 1;
            const uint32_t need = W * fanout<I>();
            uint32_t n_ens = 0, n_items = 0;
            for (;;) {
                const uint32_t avail = qt[I - 1] - qh[I - 1];
                if (avail == 0 || (!last && C() - (qt[I] - qh[I]) < need)) break;
                const uint32_t take = min(avail, W);
                ensemble<I, false>(take);
                qh[I - 1] += take;
                ++n_ens;
                n_items += take;
            }
            if (n_ens) count_firing(I, n_ens, n_items);
            if (qh[I - 1] == qt[I - 1]) qh[I - 1] = qt[I - 1] = (qt[I - 1] + V - 1) & ~(uint32_t)(V - 1);
        }
    }

    // offer the downstream nodes the processor, upstream first; a node is visited only
    // when its input ring holds a full ensemble (which also holds for every node whose
    // output ring is too full for node 1 or an upstream node to fire)
    __device__ __forceinline__ void pump()
    {
        if (n_st() <= 2 || qt[1] - qh[1] < W) return;
        fire<2>();
        if (n_st() <= 3 || qt[2] - qh[2] < W) return;
        fire<3>();
        if (n_st() <= 4 || qt[3] - qh[3] < W) return;
        fire<4>();
        if (n_st() <= 5 || qt[4] - qh[4] < W) return;
        fire<5>();
    }

    __device__ __forceinline__ bool rings_empty() const
    {
        bool e = true;
#pragma unroll
        for (int k = 1; k < RS_MAX_STAGES - 1; ++k)
            if (k < n_st() - 1) e = e && qh[k] == qt[k];
        return e;
    }

    // fire the downstream nodes on partial ensembles until every ring is empty
    __device__ __forceinline__ void drain_all()
    {
        for (unsigned long long it = 0; !rings_empty(); ++it) {
            if (it > P.budget) {
                if (lane == 0) atomicOr(&P.hdr->status, ST_STALL);
                stop = true;
                return;
            }
            fire_drain<2>();
            fire_drain<3>();
            fire_drain<4>();
            fire_drain<5>();
        }
    }

    // node 1 fires on one window (after making room downstream, Section 3.2); false
    // when the processor must stop
    __device__ __forceinline__ bool step()
    {
        // positions stay below 2^32 - 4 W, so no window end wraps around (the host
        // rejects larger element arrays; lengths summing beyond it are bad input)
        if (a > NONE - 4 * W) {
            bad_unit();
            return false;
        }
        if (n_st() > 2) {
            const uint32_t need = W * fanout<1>();
            uint64_t guard = 0;
            while (C() - (qt[1] - qh[1]) < need) {
                pump();
                if (++guard > P.budget) {
                    if (lane == 0) atomicOr(&P.hdr->status, ST_STALL);
                    stop = true;
                    return false;
                }
            }
        }
        if (a >= j0 && a + W <= flim) {
            if constexpr (RUN) {
                if (P.want_min) fast_run<true>();
                else fast_run<false>();
            } else {
                fast_window();
            }
        } else {
            node1();
        }
        if (!nxt_done && a + 8 * W >= j1) resolve_next();
        pump();
        return true;
    }

    // identity results of parents [lo, hi) of a unit with no elements
    __device__ __forceinline__ void own_fill(uint32_t lo, uint32_t hi) const
    {
        for (uint32_t r = lo + lane; r < hi; r += 32) write_identity(r);
    }

    // ---------------------------------------------------------------------------
    // one work unit: elements [rj0, rj1) of the stream (rj1 = NONE: up to the end of its
    // last parent), parents from rs (whose first element is at offset base) below rend;
    // whole-parent units (wfill) also write every parent's identity result

    __device__ __forceinline__ void run_unit(uint32_t rs, uint32_t base, uint32_t rend, uint32_t rj0, uint32_t rj1,
                                             bool wfill, uint32_t rownf)
    {
        ownf = rownf;
        j0 = rj0;
        j1 = rj1;
        cb = rs & ~(CP - 1);
        rlo = rs;
        re = rend;
        cstart = base;
        fill = wfill;
        unit_bad = false;
        load_start = (rs < rend && base < j1) ? base : NONE;
        a = j0 & ~3u;
        if (load_start != NONE) issue_chunk();
        ia = a;
        wi = wc = 0;
        clim = min(j1, S.n_el);
        if (!hashed())
            for (uint32_t k = 0; k + 1 < NB; ++k) issue_window();
        // the first non-empty parent (the one holding position j0)
        ord_cur = ord_loaded;
        s_nx = NONE;
        flim = 0;
        nfast = 0;
        while (ord_loaded == ord_cur && load_start != NONE) load_chunk();
        if (!unit_bad) {
            if (ord_loaded != ord_cur) {
                take_record(ord_cur);
                while (a < j1 && !stop)
                    if (!step()) break;
            } else if (!fill && lane == 0) {
                // merge-path units always hold elements: inconsistent input
                atomicOr(&P.hdr->status, ST_BAD_INPUT);
            }
        }
        // parents after the unit's last element (empty ones) still get their identity results
        while (ownf && !fill && !unit_bad && !stop && load_start != NONE) load_chunk();
        if (!unit_bad && j1 != NONE) ctr += lane == 1 ? j1 - j0 : (lane == 3 ? 1u : 0u);
        // fast windows: one ensemble each at nodes 0 and 1, W items, one firing of node 1
        ctr += (lane == 0 || lane == 4 || lane == 7) ? nfast : (lane == 5 ? nfast * W : 0u);
        flush_counters();
    }
};

}  // namespace

template <int V, class SG, int CPL>
// up to 4 items per lane: at most 80 registers, so that three CTAs of 8 processors fit
// an SM; 8 items per lane: 128
__global__ void __launch_bounds__(256, (V <= 4 ? 3 : 2)) rs_tag_kernel(const __grid_constant__ KParams P)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t wb = warp * P.L.per_warp;
    TagEngine<V, SG, CPL> E(P, lane, wb);
    if (lane < 4 * RS_MAX_STAGES) E.cnt()[lane] = 0;
    if (lane == 0) E.accw()[0] = NONE;
    __syncwarp();

    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&P.hdr->cursor, 1u);
    t = __shfl_sync(FULLMASK, t, 0);
    TicketUnit u = describe(P, t, lane);
    unsigned long long units = 0;
    while (u.valid && !E.stop) {
        if (lane == 0) E.nt = atomicAdd(&P.hdr->cursor, 1u);
        E.nxt_done = false;
        units++;
        if (u.work) {
            if (u.stream != E.sidx) {
                E.drain_all();
                E.acc_flush();
                E.set_stream(u.stream);
            }
            const uint32_t ownf =
                u.fill ? 1u : (u.own ? (1u | (u.skip_head ? 2u : 0u) | (u.skip_tail ? 4u : 0u)) : 0u);
            E.run_unit(u.rs, u.base, u.rend, u.j0, u.j1, u.fill, ownf);
        } else if (u.own) {
            // a unit with no elements: only its parents' identity results
            if (u.stream != E.sidx) {
                E.drain_all();
                E.acc_flush();
                E.set_stream(u.stream);
            }
            const uint32_t lo = u.rs + (u.skip_head ? 1u : 0u);
            const uint32_t hi = u.rend >= (u.skip_tail ? 1u : 0u) ? u.rend - (u.skip_tail ? 1u : 0u) : 0u;
            E.own_fill(lo, hi);
        }
        u = E.next_unit();
    }
    if (!E.stop) E.drain_all();
    E.acc_flush();
    E.flush_counters();

    __syncwarp();
    if (lane == 0) {
        atomicAdd(&P.hdr->units, units);
        for (int i = 0; i < 4 * P.n_stages; ++i) atomicAdd(&P.hdr->counters[i], (unsigned long long)E.cnt()[i]);
    }
}

// ---------------------------------------------------------------------------
// kernel tables (one per CPL, in rs_tag.cu and rs_tag2.cu): the workload pipelines'
// signatures, specialised, plus the generic one

struct TagEntry {
    int V, oe, o1, o2, o3, o4;
    const void *fn;
    int emit;   // the stage list ends in an emit sink, not an aggregate
};

#define RS_TSIG(V, CPL, OE, O1, O2, O3, O4) \
    {V, OE, O1, O2, O3, O4, (const void *)rs_tag_kernel<V, Sig<OE, O1, O2, O3, O4>, CPL>, 0}
#define RS_TSIGE(V, CPL, OE, O1, O2, O3, O4) \
    {V, OE, O1, O2, O3, O4, (const void *)rs_tag_kernel<V, Sig<OE, O1, O2, O3, O4, D_EMIT>, CPL>, 1}
#define RS_TALLV(CPL, OE, O1, O2, O3, O4)                                                          \
    RS_TSIG(1, CPL, OE, O1, O2, O3, O4), RS_TSIG(2, CPL, OE, O1, O2, O3, O4),                      \
        RS_TSIG(4, CPL, OE, O1, O2, O3, O4), RS_TSIG(8, CPL, OE, O1, O2, O3, O4)
#define RS_TAG_TABLE(CPL)                                                                           \
    {/* loaded elements -> three context hash filters -> aggregate */                               \
     RS_TALLV(CPL, D_ENUM_LOAD, D_FILT_HASH_CTX, D_FILT_HASH_CTX, D_FILT_HASH_CTX, 0),              \
     /* ... ending in an emit sink instead, at 128 items per ensemble */                             \
     RS_TSIGE(4, CPL, D_ENUM_LOAD, D_FILT_HASH_CTX, D_FILT_HASH_CTX, D_FILT_HASH_CTX, 0),            \
     /* hashed elements -> power-of-two modulus filter -> multiply-add map -> aggregate */          \
     RS_TALLV(CPL, D_ENUM_HASH, D_FILT_MASK, D_MAP_MULADD, 0, 0),                                    \
     /* loaded elements -> aggregate (the region-sum benchmark), 128 items per ensemble */         \
     RS_TSIG(4, CPL, D_ENUM_LOAD, 0, 0, 0, 0),                                                       \
     /* loaded elements (edges) -> weight comparison -> aggregate */                                 \
     RS_TALLV(CPL, D_ENUM_LOAD, D_FILT_WEIGHT, 0, 0, 0),                                             \
     /* any other stage list */                                                                      \
     RS_TALLV(CPL, 0, 0, 0, 0, 0)}

// the table of rs_tag2.cu (two parents per lane)
const TagEntry *rs_tag_table2(size_t *n);
