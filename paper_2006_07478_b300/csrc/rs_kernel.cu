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

#define FULLMASK 0xFFFFFFFFu
#define LB_AGG (1ull << 62)
#define LB_INCL (2ull << 62)
#define LB_VAL ((1ull << 62) - 1)
#define SIG_END 0x80000000u

// ---------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    // MurmurHash3 32-bit finalizer
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global -> shared, completion counted on an mbarrier (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULLMASK, v, d);
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v, uint32_t lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULLMASK, v, d);
        if (lane >= (uint32_t)d) v += y;
    }
    return v;
}

// sum of 32-bit values over the warp as a 64-bit total (inactive lanes pass 0)
__device__ __forceinline__ unsigned long long warp_sum_u32_wide(uint32_t v)
{
    uint32_t lo = __reduce_add_sync(FULLMASK, v & 0xFFFFu);
    uint32_t hi = __reduce_add_sync(FULLMASK, v >> 16);
    return ((unsigned long long)hi << 16) + lo;
}

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
    // aggregate accumulator (signal strategy)
    uint32_t acc_c, acc_m;
    unsigned long long acc_s;
    // counters
    unsigned long long c_ens[RS_MAX_STAGES], c_items[RS_MAX_STAGES], c_sig[RS_MAX_STAGES],
        c_fire[RS_MAX_STAGES];
};

struct Smem {
    unsigned long long *mbar;
    uint32_t *tiles, *moff, *mctx, *mpar, *rc, *rm, *qv, *sq, *scr;
    uint16_t *qtag;
    unsigned long long *rs;
};

// element staging for one unit
struct Stage {
    const uint32_t *elements;
    uint32_t A, B;          // bulk-copied element range [A, B) (absolute, 16-byte aligned)
    uint32_t ntiles, t_issued, t_ready, t_freed;
    uint32_t phase;         // bit s = parity of slot s's next completion
    bool tma;
    bool failed;
};

// ---------------------------------------------------------------------------

template <int STRAT, int V>
struct Proc {
    static constexpr uint32_t W = 32u * V;   // ensemble width (items per firing)
    const KParams &P;
    Smem &M;
    Warp &w;
    Stage &g;
    const uint32_t lane;
    // current unit
    uint32_t nk, total, E0;
    uint32_t ek;     // enumerate: next parent to open (signal strategy)
    uint32_t ek1;    // node 1: parent containing its next position (tag strategy)
    bool stop;

    __device__ __forceinline__ Proc(const KParams &P_, Smem &M_, Warp &w_, Stage &g_, uint32_t lane_)
        : P(P_), M(M_), w(w_), g(g_), lane(lane_), nk(0), total(0), E0(0), ek(0), ek1(0), stop(false) {}

    __device__ __forceinline__ bool loading() const { return P.st[0].op == D_ENUM_LOAD; }

    // ---- tile staging (TMA bulk copies into a ring of NT*TE elements) ----
    __device__ __forceinline__ void issue_tiles()
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
                bulk_g2s(M.tiles + slot * TE, g.elements + start, cnt * 4u, &M.mbar[slot]);
            }
            g.t_issued++;
        }
    }

    // make elements below e_hi (absolute) readable from the ring
    __device__ __forceinline__ void ensure_ready(uint32_t e_hi)
    {
        if (!g.tma) return;
        const uint32_t TE = P.TE, NT = P.NT;
        uint32_t lim = min(e_hi, g.B);
        while (g.t_ready < g.t_issued && g.A + g.t_ready * TE < lim) {
            uint32_t slot = g.t_ready & (NT - 1);
            uint32_t par = (g.phase >> slot) & 1u;
            if (!mbar_try_wait(&M.mbar[slot], par)) {
                unsigned long long t0 = global_ns();
                uint32_t it = 0;
                while (!mbar_try_wait(&M.mbar[slot], par)) {
                    if ((++it & 63u) == 0 && global_ns() - t0 > P.spin_limit) {
                        g.failed = true;
                        break;
                    }
                }
                if (g.failed) {
                    if (lane == 0) atomicOr(&P.hdr->status, ST_COPY_TIMEOUT);
                    stop = true;
                    return;
                }
            }
            g.phase ^= 1u << slot;
            g.t_ready++;
        }
    }

    // node 1 has consumed every element below e_read (absolute): recycle tiles
    __device__ __forceinline__ void release_below(uint32_t e_read)
    {
        if (!g.tma) return;
        const uint32_t TE = P.TE;
        bool freed = false;
        while (g.t_freed < g.t_ready && g.A + (g.t_freed + 1) * TE <= e_read) {
            g.t_freed++;
            freed = true;
        }
        if (freed) {
            __syncwarp();
            issue_tiles();
        }
    }

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
            w.c_ens[0]++;
            w.c_items[0] += Lsum;
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
    __device__ __forceinline__ void advance_ek1(uint32_t from, uint32_t pos)
    {
        ek1 = from;
        for (;;) {
            uint32_t e2 = M.moff[min(ek1 + lane + 1, nk)];
            uint32_t cnt = __popc(__ballot_sync(FULLMASK, e2 <= pos));
            ek1 += cnt;
            if (cnt < 32) break;
        }
    }

    // ---- gather one ensemble of node I: x[s], k[s] for lane's items 32 s + lane ----
    template <int I>
    __device__ __forceinline__ void gather(uint32_t take, uint32_t (&x)[V], uint32_t (&k)[V])
    {
        if constexpr (I == 1) {
            const uint32_t q0 = w.qh[0];
            const bool hashed = P.st[0].op == D_ENUM_HASH;
            if (!hashed) {
                ensure_ready(E0 + q0 + take);
            }
#pragma unroll
            for (int s = 0; s < V; ++s) {
                const uint32_t sb = 32u * s;
                k[s] = 0;
                x[s] = 0;
                if (sb < take) {
                    const uint32_t n = min(32u, take - sb);
                    const uint32_t pos = q0 + sb + lane;
                    uint32_t kk;
                    if (STRAT == RS_STRATEGY_TAG) {
                        kk = assign_parents(q0 + sb, n);
                        uint32_t klast = __shfl_sync(FULLMASK, kk, n - 1);
                        if (q0 + sb + n < total && M.moff[klast + 1] <= q0 + sb + n)
                            advance_ek1(klast, q0 + sb + n);
                        else
                            ek1 = klast;
                    } else {
                        kk = w.ctxk[1];
                    }
                    k[s] = kk;
                    if (lane < n) {
                        if (hashed)
                            x[s] = fmix32(M.mpar[kk] ^ fmix32((pos - M.moff[kk]) ^ RS_GOLD));
                        else
                            x[s] = load_elem(E0 + pos);
                    }
                }
            }
        } else {
            const uint32_t C = P.C, cm = C - 1;
            const uint32_t rb = (I - 2) * C;   // input edge I-1 is ring I-2
#pragma unroll
            for (int s = 0; s < V; ++s) {
                const uint32_t q = 32u * s + lane;
                x[s] = 0;
                k[s] = (STRAT == RS_STRATEGY_TAG) ? 0u : w.ctxk[I];
                if (q < take) {
                    const uint32_t slot = rb + ((w.qh[I - 1] + q) & cm);
                    x[s] = M.qv[slot];
                    if (STRAT == RS_STRATEGY_TAG) k[s] = M.qtag[slot];
                }
            }
        }
    }

    // ---- one ensemble through element stage I (filter / map / expand) ----
    template <int I>
    __device__ __forceinline__ void element_stage(uint32_t take)
    {
        const DevStage &sd = P.st[I];
        const uint32_t C = P.C, cm = C - 1;
        const uint32_t orb = (I - 1) * C;   // output edge I is ring I-1
        uint32_t x[V], k[V];
        gather<I>(take, x, k);
        if (sd.op == D_EXPAND) {
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
        bool keep[V];
        uint32_t y[V];
#pragma unroll
        for (int s = 0; s < V; ++s) {
            const uint32_t xs = x[s];
            bool kp;
            uint32_t ys = xs;
            switch (sd.op) {
            case D_FILT_MASK: kp = (xs & sd.p0) == sd.p1; break;
            case D_FILT_MOD: kp = (xs % sd.p0) == sd.p1; break;
            case D_FILT_HASH_CTX: kp = (fmix32(xs ^ sd.c0) ^ M.mctx[k[s]]) < sd.p1; break;
            case D_FILT_WEIGHT: kp = fmix32(xs ^ sd.c0) < fmix32(M.mpar[k[s]] ^ sd.c0); break;
            case D_MAP_MULADD: ys = xs * sd.p0 + sd.p1; kp = true; break;
            default: kp = false; break;
            }
            keep[s] = kp && (32u * s + lane < take);
            y[s] = ys;
        }
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int s = 0; s < V; ++s) {
            if (32u * s < take) {
                uint32_t b = __ballot_sync(FULLMASK, keep[s]);
                if (keep[s]) {
                    uint32_t slot = orb + ((w.qt[I] + __popc(b & lt)) & cm);
                    M.qv[slot] = y[s];
                    if (STRAT == RS_STRATEGY_TAG) M.qtag[slot] = (uint16_t)k[s];
                }
                uint32_t np = __popc(b);
                w.qt[I] += np;
                w.em[I] += np;
            }
        }
    }

    // ---- one ensemble into the aggregate (node I = n-1) ----
    template <int I>
    __device__ __forceinline__ void aggregate(uint32_t take)
    {
        uint32_t x[V], k[V];
        gather<I>(take, x, k);
        if (STRAT == RS_STRATEGY_SIGNAL) {
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
        }
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
                    M.rm[k0] = min(M.rm[k0], mn);
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
                    M.rm[kk] = min(M.rm[kk], m);
                }
            }
            __syncwarp();
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
            if constexpr (I + 1 < RS_MAX_STAGES) {
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
                    M.rm[kk] = fresh ? 0xFFFFFFFFu : w.acc_m;
                }
                if (begins) {
                    w.acc_c = 0;
                    w.acc_s = 0;
                    w.acc_m = 0xFFFFFFFFu;
                }
            } else {
                if constexpr (I + 1 < RS_MAX_STAGES) {
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
            w.c_sig[I] += m;
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
        if (I >= P.n_stages || stop) return;
        constexpr bool can_push = I + 1 < RS_MAX_STAGES;
        const bool last = !can_push || (I == P.n_stages - 1);
        const uint32_t fan = P.st[I].fanout;
        bool fired = false;
        for (;;) {
            const bool sigp = (STRAT == RS_STRATEGY_SIGNAL) && (w.sh[I - 1] != w.st[I - 1]);
            const uint32_t avail0 = w.qt[I - 1] - w.qh[I - 1];
            if (!(drain ? (avail0 > 0 || sigp) : (avail0 >= W || sigp))) break;
            if (!fired) {
                w.c_fire[I]++;
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
                    aggregate<I>(take);
                } else {
                    if constexpr (can_push) element_stage<I>(take);
                }
                if (stop) return;
                __syncwarp();
                w.qh[I - 1] += take;
                if (sigp) w.credit[I] -= take;
                w.c_ens[I]++;
                w.c_items[I] += take;
                progress = true;
                if constexpr (I == 1) {
                    if (P.st[0].op == D_ENUM_LOAD) release_below(E0 + w.qh[0]);
                }
            }
            if (STRAT == RS_STRATEGY_SIGNAL) progress |= signal_phase<I>(last);
            if (!progress) break;
        }
    }

    __device__ __forceinline__ bool edge_empty(int e) const
    {
        return (w.qh[e] == w.qt[e]) && (w.sh[e] == w.st[e]);
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
            w.c_ens[0]++;
            w.c_items[0] += total;
            ek1 = 0;
            if (total > 0) advance_ek1(0, 0);
        }
        for (unsigned long long sweep = 0;; ++sweep) {
            w.c_fire[0]++;
            if (STRAT == RS_STRATEGY_SIGNAL) enum_signal();
            bool d = (STRAT == RS_STRATEGY_TAG) || ek >= nk;
            fire<1>(d);
            d = d && edge_empty(0);
            fire<2>(d);
            d = d && (P.n_stages <= 2 || edge_empty(1));
            fire<3>(d);
            d = d && (P.n_stages <= 3 || edge_empty(2));
            fire<4>(d);
            d = d && (P.n_stages <= 4 || edge_empty(3));
            fire<5>(d);
            d = d && (P.n_stages <= 5 || edge_empty(4));
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

template <int STRAT, int V>
__global__ void __launch_bounds__(256) rs_pipeline_kernel(const __grid_constant__ KParams P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned char *wb = smem_raw + (size_t)warp * P.L.per_warp;
    Smem M;
    M.mbar = (unsigned long long *)(wb + P.L.o_mbar);
    M.tiles = (uint32_t *)(wb + P.L.o_tiles);
    M.moff = (uint32_t *)(wb + P.L.o_off);
    M.mctx = (uint32_t *)(wb + P.L.o_ctx);
    M.mpar = (uint32_t *)(wb + P.L.o_par);
    M.rc = (uint32_t *)(wb + P.L.o_rc);
    M.rs = (unsigned long long *)(wb + P.L.o_rs);
    M.rm = (uint32_t *)(wb + P.L.o_rm);
    M.qv = (uint32_t *)(wb + P.L.o_qv);
    M.qtag = (uint16_t *)(wb + P.L.o_qt);
    M.sq = (uint32_t *)(wb + P.L.o_sq);
    M.scr = (uint32_t *)(wb + P.L.o_scr);

    if (P.any_load && lane == 0) {
        for (uint32_t s = 0; s < P.NT; ++s) mbar_init(&M.mbar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    Warp w;
#pragma unroll
    for (int i = 0; i < RS_MAX_STAGES; ++i) w.c_ens[i] = w.c_items[i] = w.c_sig[i] = w.c_fire[i] = 0;
    Stage g;
    g.phase = 0;
    g.failed = false;
    unsigned long long units = 0;
    bool stop = false;

    while (!stop) {
        uint32_t ticket = 0;
        if (lane == 0) ticket = atomicAdd(&P.hdr->cursor, 1u);
        ticket = __shfl_sync(FULLMASK, ticket, 0);
        if (ticket >= P.total_units) break;
        units++;
        // stream owning this ticket: the last one whose unit_base <= ticket
        uint32_t lo = 0, hi = P.n_streams - 1;
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (P.streams[mid].unit_base <= ticket) lo = mid; else hi = mid - 1;
        }
        const DevStream &S = P.streams[lo];
        const uint32_t lu = ticket - S.unit_base;
        const uint32_t K = S.K;
        const uint32_t r0 = lu * K;
        const uint32_t nk = min(K, S.R - r0);
        const bool load = P.st[0].op == D_ENUM_LOAD;
        bool bad = false;
        uint32_t E0 = 0, total = 0;

        // ---- parents of this unit: lengths -> local offsets ----
        if (S.offsets) {
            uint32_t ob = S.offsets[r0];
            for (uint32_t k = lane; k <= nk; k += 32) M.moff[k] = S.offsets[r0 + k] - ob;
            __syncwarp();
            bool dec = false;
            for (uint32_t k = lane; k < nk; k += 32) dec |= M.moff[k + 1] < M.moff[k];
            bad = __any_sync(FULLMASK, dec);
            E0 = ob;
            total = M.moff[nk];
        } else {
            uint32_t carry = 0;
            for (uint32_t b = 0; b < nk; b += 32) {
                uint32_t k = b + lane;
                uint32_t L = (k < nk) ? S.len[r0 + k] : 0u;
                uint32_t incl = warp_incl_scan_u32(L, lane);
                if (k < nk) M.moff[k] = carry + incl - L;
                carry += __shfl_sync(FULLMASK, incl, 31);
            }
            if (lane == 0) M.moff[nk] = carry;
            total = carry;
            if (load) {
                // decoupled look-back over this stream's units
                unsigned long long *lb = P.lookback + S.unit_base;
                if (lu == 0) {
                    if (lane == 0) st_release_u64(&lb[0], LB_INCL | (unsigned long long)total);
                } else {
                    if (lane == 0) st_release_u64(&lb[lu], LB_AGG | (unsigned long long)total);
                    unsigned long long excl = 0;
                    int j = (int)lu - 1;
                    unsigned long long t0 = global_ns();
                    uint32_t it = 0;
                    for (;;) {
                        int idx = j - (int)lane;
                        unsigned long long wv = (idx >= 0) ? ld_acquire_u64(&lb[idx]) : LB_INCL;
                        uint32_t flag = (uint32_t)(wv >> 62);
                        uint32_t notready = __ballot_sync(FULLMASK, flag == 0u);
                        uint32_t incl = __ballot_sync(FULLMASK, flag == 2u);
                        uint32_t stopm = notready | incl;
                        if (stopm == 0u) {
                            excl += warp_sum_u64(wv & LB_VAL);
                            j -= 32;
                            continue;
                        }
                        uint32_t first = __ffs(stopm) - 1;
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
                    E0 = (uint32_t)excl;
                    if (lane == 0) st_release_u64(&lb[lu], LB_INCL | (excl + total));
                    if (stop) break;
                }
            }
        }
        if (load && !bad && (unsigned long long)E0 + total > S.n_elements) bad = true;
        if (bad) {
            if (lane == 0) atomicOr(&P.hdr->status, ST_BAD_INPUT);
            continue;
        }
        if (P.need_ctx)
            for (uint32_t k = lane; k < nk; k += 32) M.mctx[k] = S.ctx ? S.ctx[r0 + k] : 0u;
        if (P.need_par)
            for (uint32_t k = lane; k < nk; k += 32) M.mpar[k] = S.parents ? S.parents[r0 + k] : r0 + k;
        if (STRAT == RS_STRATEGY_TAG) {
            for (uint32_t k = lane; k < nk; k += 32) {
                M.rc[k] = 0;
                M.rs[k] = 0;
                M.rm[k] = 0xFFFFFFFFu;
            }
        }
        __syncwarp();

        // ---- element staging: bulk copies of [A, B) in tiles ----
        g.elements = S.elements;
        g.tma = load && S.tma_ok;
        g.A = E0 & ~3u;
        g.B = (E0 + total) & ~3u;
        if (g.B < g.A) g.B = g.A;
        g.ntiles = g.tma ? (g.B - g.A + P.TE - 1) / P.TE : 0u;
        g.t_issued = g.t_ready = g.t_freed = 0;

        Proc<STRAT, V> pr(P, M, w, g, lane);
        pr.nk = nk;
        pr.total = total;
        pr.E0 = E0;
        if (g.tma) pr.issue_tiles();
        pr.run_unit();
        pr.finish_tiles();
        if (pr.stop) {
            stop = true;
            break;
        }
        __syncwarp();

        // ---- per-parent results, coalesced ----
        for (uint32_t k = lane; k < nk; k += 32) {
            if (P.want_count) S.out_count[r0 + k] = M.rc[k];
            if (P.want_sum) S.out_sum[r0 + k] = M.rs[k];
            if (P.want_min) S.out_min[r0 + k] = M.rm[k];
        }
        __syncwarp();
    }

    // ---- counters ----
    if (lane == 0) {
        atomicAdd(&P.hdr->units, units);
#pragma unroll
        for (int i = 0; i < RS_MAX_STAGES; ++i) {
            if (i < P.n_stages) {
                atomicAdd(&P.hdr->counters[4 * i + 0], w.c_ens[i]);
                atomicAdd(&P.hdr->counters[4 * i + 1], w.c_items[i]);
                atomicAdd(&P.hdr->counters[4 * i + 2], w.c_sig[i]);
                atomicAdd(&P.hdr->counters[4 * i + 3], w.c_fire[i]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host-side launch helpers

static const void *kernel_ptr(int strategy, int V)
{
    if (strategy == RS_STRATEGY_SIGNAL) {
        if (V == 1) return (const void *)rs_pipeline_kernel<RS_STRATEGY_SIGNAL, 1>;
        if (V == 2) return (const void *)rs_pipeline_kernel<RS_STRATEGY_SIGNAL, 2>;
        return (const void *)rs_pipeline_kernel<RS_STRATEGY_SIGNAL, 4>;
    }
    if (V == 1) return (const void *)rs_pipeline_kernel<RS_STRATEGY_TAG, 1>;
    if (V == 2) return (const void *)rs_pipeline_kernel<RS_STRATEGY_TAG, 2>;
    return (const void *)rs_pipeline_kernel<RS_STRATEGY_TAG, 4>;
}

int rs_kernel_occupancy(int strategy, int V, int block, size_t smem, int *blocks_per_sm)
{
    const void *f = kernel_ptr(strategy, V);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
    return (int)e;
}

int rs_kernel_max_smem_optin(int strategy, int V, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(kernel_ptr(strategy, V), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    return (int)e;
}

int rs_launch_kernel(const KParams &P, int grid, int block, size_t smem, void *stream)
{
    const void *f = kernel_ptr(P.strategy, (int)P.V);
    void *args[] = {(void *)&P};
    cudaError_t e = cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, (cudaStream_t)stream);
    return (int)e;
}
