/*
 * rs_oracle.c -- sequential CPU oracle for region-segmented streaming pipelines.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header or constant table with the CUDA
 * library; the two agree only through the mathematics written down here.
 *
 * What it computes (Timcheck & Buhler, "Streaming Computations with Region-Based
 * State on SIMD Architectures"):
 *   - Section 4: a stream of composite objects (parents); each parent r holds L_r
 *     elements.  Enumeration opens parent r into elements i = 0..L_r-1 (sequential
 *     indices, Section 4.1); nodes downstream may consult the parent (getParent()).
 *   - Section 2.1: a linear pipeline; each node turns one input into 0..k outputs.
 *     Tree topologies (Figure 1(b), ora_run_tree) replicate a stage's output stream to
 *     each of its children; every leaf is an aggregate with results of its own.
 *   - Section 4 / Figure 4: aggregation closes the parent: begin() resets the
 *     accumulator, run() folds each surviving item in, end() emits one result per
 *     parent -- including parents none of whose elements survive.  Section 4's other
 *     option, results derived from individual elements stripped of their parent, is
 *     the emit sink (ora_run_emit): the survivors themselves, grouped by region.
 *   - Lemma 1 (precise delivery) says the signal/credit protocol only delivers
 *     region boundaries; it never changes which items meet which context.  So the
 *     method's result is exactly the plain definition below: walk the regions in
 *     order, walk each region's elements in order, push every element through the
 *     stages, fold survivors into that region's accumulator.
 *
 * The integer operations available to a stage (hash32, the filter predicates,
 * the maps, the bounded fan-out expansion) are this project's concrete choices for
 * the paper's user-supplied run() bodies; each is written out where it is defined.
 *
 * Parity: pinned.  fmix32 is checked against published MurmurHash3_x86_32 test
 * vectors and against its algebraic inverse; ora_run is checked against closed
 * forms, algebraic invariants (region splitting, permutation within a region,
 * threshold monotonicity), a separate Python model of the paper's queue/credit
 * machinery (oracle/protosim.py) and pass-rate statistics.  See tests/.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* Stage operations.  Values are this file's own; the Python wrapper maps names to them. */
enum {
    ORA_ENUM_HASH = 1,      /* x(r,i) = hash32(p_r, i)                          */
    ORA_ENUM_LOAD = 2,      /* x(r,i) = elements[off_r + i]                     */
    ORA_FILTER_MOD = 10,    /* keep x mod m == c                   (p0=m, p1=c) */
    ORA_FILTER_HASH_CTX = 11, /* keep (hash32(x,salt) ^ t_r) < theta (p0=salt, p1=theta) */
    ORA_FILTER_WEIGHT_LT = 12, /* keep hash32(x,salt) < hash32(p_r,salt) (p0=salt) */
    ORA_MAP_MUL = 20,       /* x <- a*x + b mod 2^32               (p0=a, p1=b) */
    ORA_EXPAND = 30,        /* n = hash32(x,salt) mod (k+1) outputs hash32(x, salt+1+j) (p0=salt, fanout=k) */
    ORA_AGGREGATE = 40,     /* count, sum (u64), min                            */
    ORA_EMIT = 50           /* each survivor, stripped of its parent, into the
                               region's segment of the output array (Section 4's
                               alternative to aggregation)                       */
};

typedef struct {
    int32_t op;
    uint32_t fanout;
    uint32_t p0, p1, p2, p3;
} ora_stage;

/* MurmurHash3 32-bit finalizer (Appleby, public domain): xor-shift 16, multiply by
 * 0x85EBCA6B, xor-shift 13, multiply by 0xC2B2AE35, xor-shift 16, all mod 2^32. */
uint32_t ora_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* Two-argument hash used by every hashed element, filter and expansion:
 * hash32(a, b) = fmix32(a XOR fmix32(b XOR 0x9E3779B9)). */
uint32_t ora_hash32(uint32_t a, uint32_t b)
{
    return ora_fmix32(a ^ ora_fmix32(b ^ 0x9E3779B9u));
}

typedef struct {
    uint64_t R;
    const uint32_t *parents;   /* p_r; NULL means p_r = r                       */
    const uint32_t *len;       /* L_r; used when offsets == NULL                */
    const uint32_t *offsets;   /* R+1 CSR offsets; NULL means derive from len   */
    const uint32_t *elements;  /* for ORA_ENUM_LOAD                             */
    const uint32_t *ctx;       /* t_r; NULL means t_r = 0                       */
} ora_stream;

typedef struct {
    uint32_t count;
    uint64_t sum;
    uint32_t min;
    uint32_t *seg;   /* ORA_EMIT: the region's segment of the output array, else NULL */
} ora_acc;

/* Push one item x (already produced by stage s-1) through stages s..n-1 of region r,
 * folding survivors into acc.  Depth-first; with commutative folds the order in
 * which an item's expansions are visited does not affect the result. */
static void push_item(const ora_stage *st, int n, int s, uint32_t x, uint64_t r,
                      uint32_t parent, uint32_t t, ora_acc *acc)
{
    for (; s < n; ++s) {
        const ora_stage *g = &st[s];
        switch (g->op) {
        case ORA_FILTER_MOD:
            if (x % g->p0 != g->p1) return;
            break;
        case ORA_FILTER_HASH_CTX:
            if ((ora_hash32(x, g->p0) ^ t) >= g->p1) return;
            break;
        case ORA_FILTER_WEIGHT_LT:
            if (!(ora_hash32(x, g->p0) < ora_hash32(parent, g->p0))) return;
            break;
        case ORA_MAP_MUL:
            x = g->p0 * x + g->p1;
            break;
        case ORA_EXPAND: {
            uint32_t nout = ora_hash32(x, g->p0) % (g->fanout + 1u);
            for (uint32_t j = 0; j < nout; ++j)
                push_item(st, n, s + 1, ora_hash32(x, g->p0 + 1u + j), r, parent, t, acc);
            return;
        }
        case ORA_AGGREGATE:
            acc->count += 1u;
            acc->sum += (uint64_t)x;
            if (x < acc->min) acc->min = x;
            return;
        case ORA_EMIT:
            /* results derived from individual elements, in stream order; the count
             * says how many the region produced */
            if (acc->seg) acc->seg[acc->count] = x;
            acc->count += 1u;
            return;
        default:
            return;
        }
    }
}

/* Validate a stage list: an enumeration first, an aggregate last, element ops between. */
static int check_stages(const ora_stage *st, int n)
{
    if (n < 2 || n > 8) return -1;
    if (st[0].op != ORA_ENUM_HASH && st[0].op != ORA_ENUM_LOAD) return -1;
    if (st[n - 1].op != ORA_AGGREGATE && st[n - 1].op != ORA_EMIT) return -1;
    for (int s = 1; s < n - 1; ++s) {
        int op = st[s].op;
        if (op == ORA_FILTER_MOD && st[s].p0 == 0) return -1;
        if (op != ORA_FILTER_MOD && op != ORA_FILTER_HASH_CTX && op != ORA_FILTER_WEIGHT_LT &&
            op != ORA_MAP_MUL && op != ORA_EXPAND)
            return -1;
    }
    return 0;
}

/* The plain definition for regions [r_begin, r_end): begin, run over every element
 * in order, end.  off[] holds each region's first element index (R+1 entries). */
static void run_range(const ora_stage *st, int n, const ora_stream *s, const uint64_t *off,
                      uint64_t r_begin, uint64_t r_end,
                      uint32_t *count, uint64_t *sum, uint32_t *mn)
{
    for (uint64_t r = r_begin; r < r_end; ++r) {
        ora_acc acc = {0u, 0u, 0xFFFFFFFFu, NULL};         /* begin() */
        uint32_t parent = s->parents ? s->parents[r] : (uint32_t)r;
        uint32_t t = s->ctx ? s->ctx[r] : 0u;
        uint64_t L = off[r + 1] - off[r];
        for (uint64_t i = 0; i < L; ++i) {                 /* run() per element */
            uint32_t x = (st[0].op == ORA_ENUM_HASH) ? ora_hash32(parent, (uint32_t)i)
                                                     : s->elements[off[r] + i];
            push_item(st, n, 1, x, r, parent, t, &acc);
        }
        if (count) count[r] = acc.count;                  /* end(): one result per parent */
        if (sum) sum[r] = acc.sum;
        if (mn) mn[r] = acc.min;
    }
}

static uint64_t *make_offsets(const ora_stream *s)
{
    uint64_t *off = (uint64_t *)malloc((s->R + 1) * sizeof(uint64_t));
    if (!off) return NULL;
    off[0] = s->offsets ? s->offsets[0] : 0u;
    for (uint64_t r = 0; r < s->R; ++r)
        off[r + 1] = s->offsets ? (uint64_t)s->offsets[r + 1] : off[r] + s->len[r];
    return off;
}

typedef struct {
    const ora_stage *st; int n; const ora_stream *s; const uint64_t *off;
    uint64_t b, e; uint32_t *count; uint64_t *sum; uint32_t *mn;
} ora_job;

static void *job_main(void *arg)
{
    ora_job *j = (ora_job *)arg;
    run_range(j->st, j->n, j->s, j->off, j->b, j->e, j->count, j->sum, j->mn);
    return NULL;
}

/* Whole stream, on `threads` host threads taking contiguous blocks of regions
 * (regions are independent, so the split does not change any result).
 * Returns 0, or -1 for an invalid stage list / allocation failure. */
int ora_run(const ora_stage *st, int n, uint64_t R, const uint32_t *parents,
            const uint32_t *len, const uint32_t *offsets, const uint32_t *elements,
            const uint32_t *ctx, uint32_t *count, uint64_t *sum, uint32_t *mn, int threads)
{
    if (check_stages(st, n)) return -1;
    if (!len && !offsets && R > 0) return -1;
    if (st[0].op == ORA_ENUM_LOAD && !elements && R > 0) return -1;
    ora_stream s = {R, parents, len, offsets, elements, ctx};
    uint64_t *off = make_offsets(&s);
    if (!off) return -1;
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > R) threads = R > 0 ? (int)R : 1;
    if (threads == 1) {
        run_range(st, n, &s, off, 0, R, count, sum, mn);
    } else {
        pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
        ora_job *jobs = (ora_job *)malloc(sizeof(ora_job) * threads);
        for (int k = 0; k < threads; ++k) {
            uint64_t b = R * (uint64_t)k / threads, e = R * (uint64_t)(k + 1) / threads;
            jobs[k] = (ora_job){st, n, &s, off, b, e, count, sum, mn};
            pthread_create(&tid[k], NULL, job_main, &jobs[k]);
        }
        for (int k = 0; k < threads; ++k) pthread_join(tid[k], NULL);
        free(tid);
        free(jobs);
    }
    free(off);
    return 0;
}

/* Only the regions listed in idx[0..m): results go to out_*[k] for region idx[k].
 * Used to check sampled regions of streams too large for a full oracle pass. */
int ora_run_sampled(const ora_stage *st, int n, uint64_t R, const uint32_t *parents,
                    const uint32_t *len, const uint32_t *offsets, const uint32_t *elements,
                    const uint32_t *ctx, const uint64_t *idx, uint64_t m,
                    uint32_t *count, uint64_t *sum, uint32_t *mn)
{
    if (check_stages(st, n)) return -1;
    if (!len && !offsets && R > 0) return -1;
    ora_stream s = {R, parents, len, offsets, elements, ctx};
    uint64_t *off = make_offsets(&s);
    if (!off) return -1;
    for (uint64_t k = 0; k < m; ++k) {
        uint64_t r = idx[k];
        if (r >= R) { free(off); return -1; }
        /* a one-region stream whose only region is r */
        uint32_t p1 = parents ? parents[r] : (uint32_t)r;
        uint32_t t1 = ctx ? ctx[r] : 0u;
        uint64_t off1[2] = {off[r], off[r + 1]};
        ora_stream s1 = {1u, &p1, NULL, NULL, elements, &t1};
        uint32_t c1; uint64_t su1; uint32_t mi1;
        run_range(st, n, &s1, off1, 0, 1, &c1, &su1, &mi1);
        if (count) count[k] = c1;
        if (sum) sum[k] = su1;
        if (mn) mn[k] = mi1;
    }
    free(off);
    return 0;
}

/* Sink ORA_EMIT: every surviving value of region r goes, in stream order, to
 * values[F * (off_r - off_0) + j], j = 0..count[r]-1, where off_r is the region's first
 * element index and F the product of the element stages' maximum fan-outs (so region r
 * owns F * L_r slots, enough for any survivors).  values holds F * N entries. */
int ora_run_emit(const ora_stage *st, int n, uint64_t R, const uint32_t *parents,
                 const uint32_t *len, const uint32_t *offsets, const uint32_t *elements,
                 const uint32_t *ctx, uint32_t F, uint32_t *values, uint32_t *count)
{
    if (check_stages(st, n) || st[n - 1].op != ORA_EMIT) return -1;
    if (!len && !offsets && R > 0) return -1;
    if (st[0].op == ORA_ENUM_LOAD && !elements && R > 0) return -1;
    ora_stream s = {R, parents, len, offsets, elements, ctx};
    uint64_t *off = make_offsets(&s);
    if (!off) return -1;
    for (uint64_t r = 0; r < R; ++r) {
        ora_acc acc = {0u, 0u, 0xFFFFFFFFu, values + (uint64_t)F * (off[r] - off[0])};
        uint32_t parent = parents ? parents[r] : (uint32_t)r;
        uint32_t t = ctx ? ctx[r] : 0u;
        uint64_t L = off[r + 1] - off[r];
        for (uint64_t i = 0; i < L; ++i) {
            uint32_t x = (st[0].op == ORA_ENUM_HASH) ? ora_hash32(parent, (uint32_t)i) : elements[off[r] + i];
            push_item(st, n, 1, x, r, parent, t, &acc);
        }
        count[r] = acc.count;
    }
    free(off);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Tree topologies (Section 2.1, Figure 1(b)): stage s >= 1 reads the output stream of
 * stage up[s] (up[1] = 0, the enumeration; 1 <= up[s] < s otherwise).  Every output of
 * a stage goes to each of its children -- the stream is replicated at a branch, and so
 * is every region boundary -- and each leaf is an aggregate with results of its own.
 * sink_of[s] numbers the leaves in stage order. */

static void push_tree(const ora_stage *st, const int *up, const int *sink_of, int n, int s, uint32_t x,
                      uint32_t parent, uint32_t t, ora_acc *acc)
{
    const ora_stage *g = &st[s];
    switch (g->op) {
    case ORA_FILTER_MOD:
        if (x % g->p0 != g->p1) return;
        break;
    case ORA_FILTER_HASH_CTX:
        if ((ora_hash32(x, g->p0) ^ t) >= g->p1) return;
        break;
    case ORA_FILTER_WEIGHT_LT:
        if (!(ora_hash32(x, g->p0) < ora_hash32(parent, g->p0))) return;
        break;
    case ORA_MAP_MUL:
        x = g->p0 * x + g->p1;
        break;
    case ORA_EXPAND: {
        uint32_t nout = ora_hash32(x, g->p0) % (g->fanout + 1u);
        for (uint32_t j = 0; j < nout; ++j) {
            uint32_t y = ora_hash32(x, g->p0 + 1u + j);
            for (int c = s + 1; c < n; ++c)
                if (up[c] == s) push_tree(st, up, sink_of, n, c, y, parent, t, acc);
        }
        return;
    }
    case ORA_AGGREGATE: {
        ora_acc *a = &acc[sink_of[s]];
        a->count += 1u;
        a->sum += (uint64_t)x;
        if (x < a->min) a->min = x;
        return;
    }
    default:
        return;
    }
    for (int c = s + 1; c < n; ++c)
        if (up[c] == s) push_tree(st, up, sink_of, n, c, x, parent, t, acc);
}

/* Results of sink k go to count[k][r], sum[k][r], mn[k][r] (any may be NULL).
 * Returns the number of sinks, or -1 for an invalid tree (a sink with children, an
 * element stage without, more than 4 sinks). */
int ora_run_tree(const ora_stage *st, const int32_t *up, int n, uint64_t R, const uint32_t *parents,
                 const uint32_t *len, const uint32_t *offsets, const uint32_t *elements, const uint32_t *ctx,
                 uint32_t **count, uint64_t **sum, uint32_t **mn)
{
    int upi[16], sink_of[16], n_sinks = 0;
    if (n < 2 || n > 16) return -1;
    if (st[0].op != ORA_ENUM_HASH && st[0].op != ORA_ENUM_LOAD) return -1;
    for (int s = 1; s < n; ++s) {
        upi[s] = up[s];
        if (s == 1 ? up[s] != 0 : (up[s] < 1 || up[s] >= s)) return -1;
        if (st[up[s]].op == ORA_AGGREGATE) return -1;   /* a sink has no children */
    }
    for (int s = 1; s < n; ++s) {
        int kids = 0;
        for (int c = s + 1; c < n; ++c) kids += up[c] == s;
        const int op = st[s].op;
        if (op == ORA_AGGREGATE) {
            if (n_sinks >= 4) return -1;
            sink_of[s] = n_sinks++;
        } else {
            if (kids == 0) return -1;                     /* every leaf is a sink */
            if (op != ORA_FILTER_MOD && op != ORA_FILTER_HASH_CTX && op != ORA_FILTER_WEIGHT_LT &&
                op != ORA_MAP_MUL && op != ORA_EXPAND)
                return -1;
            if (op == ORA_FILTER_MOD && st[s].p0 == 0) return -1;
            sink_of[s] = -1;
        }
    }
    if (!len && !offsets && R > 0) return -1;
    if (st[0].op == ORA_ENUM_LOAD && !elements && R > 0) return -1;
    ora_stream s = {R, parents, len, offsets, elements, ctx};
    uint64_t *off = make_offsets(&s);
    if (!off) return -1;
    for (uint64_t r = 0; r < R; ++r) {
        ora_acc acc[4];
        for (int k = 0; k < 4; ++k) acc[k] = (ora_acc){0u, 0u, 0xFFFFFFFFu, NULL};   /* begin() per sink */
        uint32_t parent = parents ? parents[r] : (uint32_t)r;
        uint32_t t = ctx ? ctx[r] : 0u;
        uint64_t L = off[r + 1] - off[r];
        for (uint64_t i = 0; i < L; ++i) {
            uint32_t x = (st[0].op == ORA_ENUM_HASH) ? ora_hash32(parent, (uint32_t)i) : elements[off[r] + i];
            push_tree(st, upi, sink_of, n, 1, x, parent, t, acc);
        }
        for (int k = 0; k < n_sinks; ++k) {                /* end(): one result per parent and sink */
            if (count && count[k]) count[k][r] = acc[k].count;
            if (sum && sum[k]) sum[k][r] = acc[k].sum;
            if (mn && mn[k]) mn[k][r] = acc[k].min;
        }
    }
    free(off);
    return n_sinks;
}
