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
// per-warp state

struct Warp {
    // queue cursors (free-running; slot = cursor & (C-1))
    uint32_t qh[RS_MAX_EDGES], qt[RS_MAX_EDGES];
    // signal rings and the sender's emitted-since-last-signal counter (Section 3.1)
    uint32_t sh[RS_MAX_EDGES], st[RS_MAX_EDGES], em[RS_MAX_EDGES];
    // receiver state: current credit counter and current parent (local index)
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
    uint32_t *tiles, *moff, *mctx, *mpar, *rc, *rm, *qv, *qtag, *sq, *scr;
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

template <int STRAT>
struct Kern {
    const KParams &P;
    Smem &M;
    Warp &w;
    Stage &g;
    uint32_t lane;
    // unit
    uint32_t nk, total, E0, r0;
    bool stop;

    __device__ __forceinline__ Kern(const KParams &P_, Smem &M_, Warp &w_, Stage &g_, uint32_t lane_)
        : P(P_), M(M_), w(w_), g(g_), lane(lane_), nk(0), total(0), E0(0), r0(0), stop(false) {}

    // ---- tile staging (TMA bulk copies into a ring of NT*TE elements) ----
    __device__ __forceinline__ void issue_tiles()
    {
        const uint32_t TE = P.TE, NT = P.NT;
        bool any = false;
        while (g.t_issued < g.ntiles && g.t_issued < g.t_freed + NT) {
            any = true;
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
        (void)any;
    }

    // make elements [.., e_hi) (absolute) readable from the ring
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

    // the enumerating node has read everything below e_read (absolute)
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

    // drain outstanding copies (they must land before the shared memory is reused or
    // the CTA exits); bounded like every wait
    __device__ __forceinline__ void finish_tiles()
    {
        if (!g.tma) return;
        ensure_ready(0xFFFFFFFFu);
        g.t_freed = g.t_ready;
    }

    // ---- signal ring helpers ----
    __device__ __forceinline__ void push_signal(int e, uint32_t word)
    {
        // Section 3.1 sender rules: empty signal queue -> credit = items queued now;
        // else -> items emitted since the previous signal.
        uint32_t credit = (w.sh[e] == w.st[e]) ? (w.qt[e] - w.qh[e]) : w.em[e];
        if (lane == 0) {
            uint32_t idx = e * P.SC + (w.st[e] & (P.SC - 1));
            M.sq[2 * idx] = word;
            M.sq[2 * idx + 1] = credit;
        }
        w.st[e]++;
        w.em[e] = 0;
    }

    // ---- enumeration, tag strategy ----
    // fills queue 0 with (element, local region) pairs, ensembles cut only by space
    __device__ __forceinline__ void enum_tag(uint32_t &epos, uint32_t &ek)
    {
        const uint32_t C = P.C, cm = C - 1;
        const DevStage &s0 = P.st[0];
        while (epos < total && !stop) {
            uint32_t space = C - (w.qt[0] - w.qh[0]);
            if (space == 0) break;
            uint32_t take = min(min((uint32_t)RS_W, space), total - epos);
            // window of the next 32 region ends after ek
            uint32_t kk = ek + lane + 1;
            uint32_t endj = M.moff[min(kk, nk)];
            uint32_t end31 = __shfl_sync(FULLMASK, endj, 31);
            if (ek + 32 <= nk) take = min(take, end31 - epos);
            uint32_t nxt = __shfl_down_sync(FULLMASK, endj, 1);
            uint32_t pj = endj - epos;
            bool valid = (pj < take) && (lane == 31 || endj != nxt);
            if (valid) M.scr[pj] = lane + 1;
            uint32_t D = __reduce_or_sync(FULLMASK, valid ? (1u << pj) : 0u);
            __syncwarp();
            uint32_t myk = ek;
            uint32_t mk = D & ((2u << lane) - 1u);
            if (lane < take && mk) myk = ek + M.scr[31 - __clz(mk)];
            uint32_t pos = epos + lane;
            uint32_t x = 0;
            if (s0.op == D_ENUM_HASH) {
                if (lane < take) x = fmix32(M.mpar[myk] ^ fmix32((pos - M.moff[myk]) ^ RS_GOLD));
            } else {
                ensure_ready(E0 + epos + take);
                if (stop) return;
                if (lane < take) x = load_elem(E0 + pos);
            }
            if (lane < take) {
                uint32_t slot = (w.qt[0] + lane) & cm;
                M.qv[slot] = x;
                M.qtag[slot] = myk;
            }
            __syncwarp();
            w.qt[0] += take;
            epos += take;
            w.c_ens[0]++;
            w.c_items[0] += take;
            ek = __shfl_sync(FULLMASK, myk, take - 1);
            if (epos < total) {
                // advance to the region containing epos (skipping empty regions)
                for (;;) {
                    uint32_t e2 = M.moff[min(ek + lane + 1, nk)];
                    uint32_t cnt = __popc(__ballot_sync(FULLMASK, e2 <= epos));
                    ek += cnt;
                    if (cnt < 32) break;
                }
            }
            if (s0.op == D_ENUM_LOAD) release_below(E0 + epos);
        }
    }

    // ---- enumeration, signal strategy ----
    // per parent: Begin(k), its elements, End(k) (Section 4.2)
    __device__ __forceinline__ void enum_signal(uint32_t &epos, uint32_t &ek, bool &begun)
    {
        const uint32_t C = P.C, cm = C - 1, SC = P.SC;
        const DevStage &s0 = P.st[0];
        while (ek < nk && !stop) {
            if (!begun) {
                if (w.st[0] - w.sh[0] >= SC) return;
                push_signal(0, ek);
                begun = true;
            }
            uint32_t re = M.moff[ek + 1];
            while (epos < re) {
                uint32_t space = C - (w.qt[0] - w.qh[0]);
                if (space == 0) return;
                uint32_t take = min(min((uint32_t)RS_W, space), re - epos);
                uint32_t pos = epos + lane;
                uint32_t x = 0;
                if (s0.op == D_ENUM_HASH) {
                    if (lane < take) x = fmix32(M.mpar[ek] ^ fmix32((pos - M.moff[ek]) ^ RS_GOLD));
                } else {
                    ensure_ready(E0 + epos + take);
                    if (stop) return;
                    if (lane < take) x = load_elem(E0 + pos);
                }
                if (lane < take) M.qv[(w.qt[0] + lane) & cm] = x;
                __syncwarp();
                w.qt[0] += take;
                w.em[0] += take;
                epos += take;
                w.c_ens[0]++;
                w.c_items[0] += take;
                if (s0.op == D_ENUM_LOAD) release_below(E0 + epos);
            }
            if (w.st[0] - w.sh[0] >= SC) return;
            push_signal(0, SIG_END | ek);
            __syncwarp();
            ek++;
            begun = false;
        }
    }

    // ---- one ensemble through an element stage (filter / map / expand) ----
    template <int I>
    __device__ __forceinline__ void run_element_stage(uint32_t take)
    {
        const DevStage &s = P.st[I];
        const uint32_t C = P.C, cm = C - 1;
        const bool active = lane < take;
        const uint32_t islot = (I - 1) * C + ((w.qh[I - 1] + lane) & cm);
        uint32_t x = active ? M.qv[islot] : 0u;
        uint32_t k = (STRAT == RS_STRATEGY_TAG) ? (active ? M.qtag[islot] : 0u) : w.ctxk[I];
        if (s.op == D_EXPAND) {
            uint32_t nout = active ? fmix32(x ^ s.c0) % (s.fanout + 1u) : 0u;
            uint32_t incl = warp_incl_scan_u32(nout, lane);
            uint32_t tot = __shfl_sync(FULLMASK, incl, 31);
            uint32_t base = w.qt[I] + incl - nout;
            for (uint32_t j = 0; j < nout; ++j) {
                uint32_t y = fmix32(x ^ fmix32((s.p0 + 1u + j) ^ RS_GOLD));
                uint32_t slot = I * C + ((base + j) & cm);
                M.qv[slot] = y;
                if (STRAT == RS_STRATEGY_TAG) M.qtag[slot] = k;
            }
            w.qt[I] += tot;
            w.em[I] += tot;
        } else {
            bool keep;
            uint32_t y = x;
            switch (s.op) {
            case D_FILT_MASK: keep = (x & s.p0) == s.p1; break;
            case D_FILT_MOD: keep = (x % s.p0) == s.p1; break;
            case D_FILT_HASH_CTX: keep = (fmix32(x ^ s.c0) ^ M.mctx[k]) < s.p1; break;
            case D_FILT_WEIGHT: keep = fmix32(x ^ s.c0) < fmix32(M.mpar[k] ^ s.c0); break;
            case D_MAP_MULADD: y = x * s.p0 + s.p1; keep = true; break;
            default: keep = false; break;
            }
            keep = keep && active;
            uint32_t b = __ballot_sync(FULLMASK, keep);
            if (keep) {
                uint32_t slot = I * C + ((w.qt[I] + __popc(b & lanemask_lt())) & cm);
                M.qv[slot] = y;
                if (STRAT == RS_STRATEGY_TAG) M.qtag[slot] = k;
            }
            uint32_t np = __popc(b);
            w.qt[I] += np;
            w.em[I] += np;
        }
    }

    // ---- one ensemble into the aggregate ----
    template <int I>
    __device__ __forceinline__ void run_aggregate(uint32_t take)
    {
        const uint32_t C = P.C, cm = C - 1;
        const bool active = lane < take;
        const uint32_t islot = (I - 1) * C + ((w.qh[I - 1] + lane) & cm);
        uint32_t v = active ? M.qv[islot] : 0u;
        if (STRAT == RS_STRATEGY_SIGNAL) {
            // every item of the ensemble belongs to the current parent (Section 3.3)
            w.acc_c += take;
            w.acc_s += warp_sum_u32_wide(v);
            w.acc_m = min(w.acc_m, __reduce_min_sync(FULLMASK, active ? v : 0xFFFFFFFFu));
        } else {
            uint32_t k = active ? M.qtag[islot] : 0xFFFFFFFFu;
            uint32_t kprev = __shfl_up_sync(FULLMASK, k, 1);
            uint32_t knext = __shfl_down_sync(FULLMASK, k, 1);
            bool head = (lane == 0) || (k != kprev);
            bool tail = (lane == 31) || (k != knext);
            uint32_t heads = __ballot_sync(FULLMASK, head);
            uint32_t k0 = __shfl_sync(FULLMASK, k, 0);
            uint32_t amask = (take >= 32) ? FULLMASK : ((1u << take) - 1u);
            if ((heads & amask) == 1u) {
                // one region in the whole ensemble
                unsigned long long s = warp_sum_u32_wide(v);
                uint32_t m = __reduce_min_sync(FULLMASK, active ? v : 0xFFFFFFFFu);
                if (lane == 0) {
                    M.rc[k0] += take;
                    M.rs[k0] += s;
                    M.rm[k0] = min(M.rm[k0], m);
                }
            } else {
                uint32_t hl = 31 - __clz(heads & ((2u << lane) - 1u));
                unsigned long long ps = v;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    unsigned long long y = __shfl_up_sync(FULLMASK, ps, d);
                    if (lane >= (uint32_t)d) ps += y;
                }
                unsigned long long before = __shfl_sync(FULLMASK, ps, hl > 0 ? hl - 1 : 0);
                if (hl == 0) before = 0;
                uint32_t m = active ? v : 0xFFFFFFFFu;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    uint32_t y = __shfl_up_sync(FULLMASK, m, d);
                    if (lane >= (uint32_t)d && lane - d >= hl) m = min(m, y);
                }
                if (active && tail) {
                    M.rc[k] += lane - hl + 1;
                    M.rs[k] += ps - before;
                    M.rm[k] = min(M.rm[k], m);
                }
            }
        }
        __syncwarp();
    }

    // ---- fire node I (1 <= I < n): data phase(s) and signal phase(s) ----
    template <int I>
    __device__ __forceinline__ void fire(bool drain)
    {
        if (I >= P.n_stages || stop) return;
        const DevStage &s = P.st[I];
        constexpr bool can_push = I + 1 < RS_MAX_STAGES;   // node I has an output queue slot
        const bool last = !can_push || (I == P.n_stages - 1);
        const uint32_t C = P.C, SC = P.SC;
        bool fired = false;
        for (;;) {
            bool progress = false;
            const bool sig_pending = (STRAT == RS_STRATEGY_SIGNAL) && (w.sh[I - 1] != w.st[I - 1]);
            uint32_t avail = w.qt[I - 1] - w.qh[I - 1];
            bool ready = drain ? (avail > 0 || sig_pending) : (avail >= RS_W || sig_pending);
            if (!ready) break;
            if (!fired) {
                w.c_fire[I]++;
                fired = true;
            }
            // data phase (Section 3.2): min(queued, downstream space, credit if a signal is pending)
            for (;;) {
                avail = w.qt[I - 1] - w.qh[I - 1];
                uint32_t lim = sig_pending ? w.credit[I] : avail;
                uint32_t take = min(min(avail, lim), (uint32_t)RS_W);
                if constexpr (can_push) {
                    if (!last) {
                        uint32_t space = C - (w.qt[I] - w.qh[I]);
                        uint32_t fit = (s.fanout == 1u) ? space : space / s.fanout;
                        take = min(take, fit);
                    }
                }
                if (take == 0) break;
                // keep ensembles full unless a signal forces the cut or the unit drains
                if (!drain && !sig_pending && take < RS_W) break;
                if (last) {
                    run_aggregate<I>(take);
                } else {
                    if constexpr (can_push) run_element_stage<I>(take);
                }
                __syncwarp();
                w.qh[I - 1] += take;
                if (sig_pending) w.credit[I] -= take;
                w.c_ens[I]++;
                w.c_items[I] += take;
                progress = true;
            }
            // signal phase: while the counter is 0 (receiver rules 2b)
            if (STRAT == RS_STRATEGY_SIGNAL) {
                while (w.credit[I] == 0 && w.sh[I - 1] != w.st[I - 1]) {
                    uint32_t idx = (I - 1) * SC + (w.sh[I - 1] & (SC - 1));
                    uint32_t word = M.sq[2 * idx];
                    uint32_t cr = M.sq[2 * idx + 1];
                    if (cr > 0) {
                        w.credit[I] = cr;          // move the head signal's credit to the counter
                        __syncwarp();
                        if (lane == 0) M.sq[2 * idx + 1] = 0;
                        __syncwarp();
                        progress = true;
                        break;
                    }
                    if constexpr (can_push) {
                        if (!last && w.st[I] - w.sh[I] >= SC) break;   // no room to forward
                    }
                    w.sh[I - 1]++;
                    w.c_sig[I]++;
                    uint32_t k = word & ~SIG_END;
                    if (!(word & SIG_END)) {
                        w.ctxk[I] = k;             // Begin: switch parent context
                        if (last) {
                            w.acc_c = 0;
                            w.acc_s = 0;
                            w.acc_m = 0xFFFFFFFFu; // begin()
                        }
                    } else if (last) {
                        if (lane == 0) {           // end(): one result per parent
                            M.rc[k] = w.acc_c;
                            M.rs[k] = w.acc_s;
                            M.rm[k] = w.acc_m;
                        }
                    }
                    __syncwarp();
                    if constexpr (can_push) {
                        if (!last) push_signal(I, word);   // forward with fresh credit
                    }
                    __syncwarp();
                    progress = true;
                }
            }
            if (!progress) break;
        }
    }

    __device__ __forceinline__ bool queues_empty() const
    {
        bool e = true;
#pragma unroll
        for (int i = 0; i < RS_MAX_EDGES; ++i)
            if (i < P.n_stages - 1) e = e && (w.qh[i] == w.qt[i]) && (w.sh[i] == w.st[i]);
        return e;
    }

    // ---- run one unit to completion ----
    __device__ __forceinline__ void run_unit()
    {
        uint32_t epos = 0, ek = 0;
        bool begun = false;
#pragma unroll
        for (int i = 0; i < RS_MAX_EDGES; ++i) {
            w.qh[i] = w.qt[i] = w.sh[i] = w.st[i] = w.em[i] = 0;
        }
#pragma unroll
        for (int i = 0; i < RS_MAX_STAGES; ++i) w.credit[i] = w.ctxk[i] = 0;
        if (STRAT == RS_STRATEGY_TAG && total > 0) {
            // first non-empty region
            for (;;) {
                uint32_t e2 = M.moff[min(ek + lane + 1, nk)];
                uint32_t cnt = __popc(__ballot_sync(FULLMASK, e2 <= 0u));
                ek += cnt;
                if (cnt < 32) break;
            }
        }
        w.acc_c = 0;
        w.acc_s = 0;
        w.acc_m = 0xFFFFFFFFu;
        for (unsigned long long sweep = 0;; ++sweep) {
            bool drain;
            if (STRAT == RS_STRATEGY_TAG) {
                enum_tag(epos, ek);
                drain = epos >= total;
            } else {
                enum_signal(epos, ek, begun);
                drain = ek >= nk;
            }
            if (stop) return;
            w.c_fire[0]++;
            fire<1>(drain);
            fire<2>(drain);
            fire<3>(drain);
            fire<4>(drain);
            fire<5>(drain);
            if (drain && queues_empty()) break;
            if (sweep >= P.budget) {
                if (lane == 0) atomicOr(&P.hdr->status, ST_STALL);
                stop = true;
                return;
            }
        }
    }
};

// ---------------------------------------------------------------------------

template <int STRAT>
__global__ void __launch_bounds__(512) rs_pipeline_kernel(const __grid_constant__ KParams P)
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
    M.qtag = (uint32_t *)(wb + P.L.o_qt);
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

        // ---- parents of this unit: lengths -> local offsets (a1) ----
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

        Kern<STRAT> kern(P, M, w, g, lane);
        kern.nk = nk;
        kern.total = total;
        kern.E0 = E0;
        kern.r0 = r0;
        if (g.tma) kern.issue_tiles();
        kern.run_unit();
        kern.finish_tiles();
        if (kern.stop) {
            stop = true;
            break;
        }
        __syncwarp();

        // ---- per-region results, coalesced (a7) ----
        for (uint32_t k = lane; k < nk; k += 32) {
            if (P.want_count) S.out_count[r0 + k] = M.rc[k];
            if (P.want_sum) S.out_sum[r0 + k] = M.rs[k];
            if (P.want_min) S.out_min[r0 + k] = M.rm[k];
        }
        __syncwarp();
    }

    // ---- counters (a8) ----
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

static const void *kernel_ptr(int strategy)
{
    return strategy == RS_STRATEGY_SIGNAL ? (const void *)rs_pipeline_kernel<RS_STRATEGY_SIGNAL>
                                          : (const void *)rs_pipeline_kernel<RS_STRATEGY_TAG>;
}

int rs_kernel_occupancy(int strategy, int block, size_t smem, int *blocks_per_sm)
{
    const void *f = kernel_ptr(strategy);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
    return (int)e;
}

int rs_kernel_max_smem_optin(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(kernel_ptr(RS_STRATEGY_SIGNAL), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(kernel_ptr(RS_STRATEGY_TAG), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return (int)e;
}

int rs_launch_kernel(const KParams &P, int grid, int block, size_t smem, void *stream)
{
    const void *f = kernel_ptr(P.strategy);
    void *args[] = {(void *)&P};
    cudaError_t e = cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, (cudaStream_t)stream);
    return (int)e;
}
