/*
 * rs.h -- C ABI of librs, a B300 (sm_103a) engine for streaming pipelines whose
 * input is cut into variably sized regions (Timcheck & Buhler, "Streaming
 * Computations with Region-Based State on SIMD Architectures").
 *
 * The problem, as the paper states it:
 *   - Section 4: the input is a stream of composite objects ("parents"); parent r
 *     holds L_r elements (findCount() in Figure 4).  Enumeration opens each parent
 *     into the stream of its elements i = 0..L_r-1; downstream nodes can consult the
 *     parent (getParent()).  Aggregation closes it again: one result per parent,
 *     including parents none of whose elements survive.
 *   - Section 2.1: the computation is a linear pipeline of nodes joined by
 *     fixed-size queues; each input makes a node emit 0..k outputs, k known a
 *     priori per node (Section 3.2 uses it to decide fireability).
 *   - Section 2.2: one pipeline instance per SIMD processor; processors compete for
 *     the common input with atomics; a node consumes ensembles of up to W items.
 *   - Section 3: region boundaries travel as signals on a separate queue per edge,
 *     synchronised with the data by credits (Lemma 1: precise delivery), and no
 *     ensemble mixes items from both sides of a signal (Section 3.3).  The
 *     alternative of Section 2.3 / Section 5 tags every item with its region instead.
 *
 * Conventions (every entry point):
 *   - returns rs_status; nothing else crosses the ABI on failure;
 *   - pointers named "device" must be device memory of the current CUDA device,
 *     owned by the caller and kept alive until the work enqueued on the given CUDA
 *     stream has finished (the same rule as cudaMemcpyAsync);
 *   - the library allocates no device memory: scratch space is a caller-owned
 *     workspace sized by rs_workspace_size();
 *   - a pipeline object is not thread-safe; use one per host thread;
 *   - CUDA streams are passed as rs_cuda_stream (the same handle as cudaStream_t);
 *     NULL means the legacy default stream.
 */
#ifndef RS_H
#define RS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rs_cuda_stream;
typedef struct rs_pipeline rs_pipeline;

typedef enum {
    RS_OK = 0,
    RS_ERR_INVALID = 1,     /* bad argument, stage list, option or stream description */
    RS_ERR_NOMEM = 2,       /* host allocation failed                                 */
    RS_ERR_CUDA = 3,        /* a CUDA runtime call failed (see rs_last_cuda_error)    */
    RS_ERR_NOT_READY = 4,   /* nothing submitted / not captured yet                   */
    RS_ERR_STALL = 5,       /* a device loop ran out of its iteration budget          */
    RS_ERR_CAPACITY = 6,    /* workspace too small, or a size beyond a stated limit   */
    RS_ERR_STATE = 7,       /* call out of order (e.g. submit while a graph is live)  */
    RS_ERR_DEVICE_INPUT = 8 /* the device found inconsistent input (offsets, bounds)  */
} rs_status;

/* ---- stages (Section 2.1 nodes; Section 4 enumeration / aggregation) ---------- */

typedef enum {
    RS_ENUM_HASH = 1,   /* enumerate: element i of parent r is hash32(p_r, i)             */
    RS_ENUM_LOAD = 2,   /* enumerate: element i of parent r is elements[off_r + i]        */
    RS_FILTER = 3,      /* 0 or 1 output per input                                        */
    RS_MAP = 4,         /* exactly 1 output per input                                     */
    RS_EXPAND = 5,      /* 0..max_fanout outputs per input                                */
    RS_AGGREGATE = 6,   /* per-region count / sum / min of the surviving values           */
    RS_EMIT = 7         /* the surviving values themselves, stripped of their parent
                           (Section 4's alternative to aggregation): region r's survivors
                           land in its own segment of the stream's out_values array,
                           out_values[F * (off_r - off_0) ...], F = the product of the
                           element stages' max_fanout, in an unspecified order, and
                           out_count[r] says how many.  Needs CSR region_offsets.        */
} rs_stage_kind;

/* Operations.  hash32(a, b) = fmix32(a XOR fmix32(b XOR 0x9E3779B9)) where fmix32 is
 * the MurmurHash3 32-bit finalizer; all arithmetic is modulo 2^32.  t_r is the
 * parent's context word (ctx[r], 0 when no ctx array is given) and p_r its id. */
typedef enum {
    RS_OP_NONE = 0,
    RS_OP_MOD_EQ = 1,       /* FILTER: keep x mod params[0] == params[1]  (params[0] > 0) */
    RS_OP_HASH_CTX_LT = 2,  /* FILTER: keep (hash32(x, params[0]) XOR t_r) < params[1]    */
    RS_OP_WEIGHT_LT = 3,    /* FILTER: keep hash32(x, params[0]) < hash32(p_r, params[0]) */
    RS_OP_MUL_ADD = 4,      /* MAP:    x <- params[0] * x + params[1]                     */
    RS_OP_HASH_FANOUT = 5   /* EXPAND: n = hash32(x, params[0]) mod (max_fanout + 1)
                               outputs hash32(x, params[0] + 1 + j), j = 0..n-1           */
} rs_op;

typedef struct {
    uint32_t kind;          /* rs_stage_kind                                    */
    uint32_t op;            /* rs_op (RS_OP_NONE for enumerate / aggregate)     */
    uint32_t max_fanout;    /* a-priori maximum outputs per input (Section 3.2) */
    uint32_t params[4];
    uint32_t input;         /* tree topologies (Section 2.1, Figure 1(b)): index of the
                               stage whose output this stage reads; 0 = the stage before
                               it (a linear pipeline).  Stage 1 reads the enumeration;
                               every other stage reads an earlier FILTER / MAP / EXPAND
                               stage, whose output stream -- and with it every region
                               boundary -- is replicated to each of its readers.  The
                               leaves are the AGGREGATE stages (at most RS_MAX_SINKS;
                               an emit sink only ends a linear pipeline).            */
} rs_stage_desc;

#define RS_MAX_SINKS 2      /* aggregate leaves of a tree */

#define RS_MAX_STAGES 6     /* enumerate + up to 4 element stages + aggregate or emit */

/* ---- options ----------------------------------------------------------------- */

typedef enum {
    RS_STRATEGY_SIGNAL = 0, /* signal-delimited ensembles: Begin/End signals with credits
                               (Sections 3-4); ensembles never cross a region boundary   */
    RS_STRATEGY_TAG = 1,    /* per-item region tags (Section 2.3 / Section 5): ensembles
                               stay full across region boundaries                        */
    RS_STRATEGY_AUTO = 2    /* pick by mean region length at run time (see rs_autotune)  */
} rs_strategy;

typedef struct {
    uint32_t ensemble_width;    /* W, items per ensemble: 32, 64 or 128; a warp is one SIMD
                                   processor and each lane takes W/32 items; 0 = 128         */
    uint32_t queue_capacity;    /* data-queue slots per edge; power of two,
                                   >= W * (max fan-out + 1) so a blocked node always leaves
                                   room for one full ensemble downstream; 0 = the smallest
                                   legal power of two >= 64                                  */
    uint32_t signal_capacity;   /* signal-queue slots per edge; power of two >= 4; 0 = 32 (256
                                   when an edge selects contexts per lane)                   */
    uint32_t strategy;          /* rs_strategy                                                 */
    uint32_t regions_per_unit;  /* parents claimed per atomic step, <= 512; 0 = from the mean
                                   region length (about 2048 elements per claim)              */
    uint32_t tile_elements;     /* elements per bulk-copy tile for RS_ENUM_LOAD, a power of
                                   two in W..4096; 0 = W                                      */
    uint32_t tiles_in_flight;   /* staging tiles per processor, 2 or 4; or 0: no staging --
                                   each lane reads its elements with 16-byte loads issued
                                   two ensembles ahead.  0 is the tag strategy's default;
                                   for the signal strategy 0 means 4                        */
    uint32_t warps_per_block;   /* processors per CTA, 1..8; 0 = the count (8, 4, 2 or 1)
                                   giving the most resident processors per SM; fewer when
                                   their shared memory would not fit one CTA                */
    uint32_t grid;              /* CTAs; 0 = a persistent grid (SMs x resident CTAs per SM)   */
    uint32_t region_cost;       /* RS_ENUM_LOAD streams are cut into merge-path work units in
                                   which a parent costs region_cost steps and an element one;
                                   a unit holds <= regions_per_unit parents and <=
                                   region_cost * regions_per_unit elements.  Power of two in
                                   1..256; 0 = 16                                            */
    uint64_t device_budget;     /* scheduler sweeps allowed per claimed unit before the device
                                   reports RS_ERR_STALL; 0 = 2^22                            */
    uint32_t boundary_modes;    /* per-edge region boundaries: bits 2c..2c+1 say how stage c
                                   (1..5) learns the region of each input item --
                                   RS_BOUNDARY_DEFAULT (from `strategy`), _SIGNAL, _TAG or
                                   _LANE.  0 everywhere: `strategy` decides for the whole
                                   pipeline.  Anything else, or a tree topology, runs the
                                   per-edge kernel (units of <= 512 parents, as the signal
                                   strategy's).  Below a tagged edge every edge is tagged;
                                   an EXPAND stage takes no RS_BOUNDARY_LANE input.        */
    uint32_t flags;             /* RS_FLAG_* below                                              */
} rs_pipeline_opts;

/* The tag strategy with a persistent grid (grid = 0) and one stream: when the stream has at
 * least two rounds of units over the resident processors, the unit count is rounded down to
 * a whole number of rounds (units grow a little), so that the last round does not leave
 * most processors idle.  The count is decided by the first run after a submit or an option
 * change and kept by the runs after it.  This flag keeps the unit shape as given. */
#define RS_FLAG_UNBALANCED_UNITS 1u
/* The caller gives rs_run the workspace of this pipeline alone: nothing else writes into it
 * between two runs of the pipeline.  A run then leaves in place the stream table (the
 * per-stream array pointers and unit split that every run reads) an earlier run uploaded
 * into the same workspace, and uploads it again only after a submit, an option change or a
 * change of workspace.  Without the flag every run copies the table from host memory first.
 * Graph capture always records the copy.  Breaking the promise is undefined behaviour: the
 * kernels would follow whatever pointers the workspace then holds where the table was. */
#define RS_FLAG_PRIVATE_WORKSPACE 2u

typedef enum {
    RS_BOUNDARY_DEFAULT = 0,
    RS_BOUNDARY_SIGNAL = 1, /* Begin/End signals with credits; ensembles cut at each (Section 3)  */
    RS_BOUNDARY_TAG = 2,    /* the producer tags each item with its region (Section 2.3 / 5):
                               mixing signals upstream and tags downstream is the per-stage
                               choice of Section 5 (the taxi application)                        */
    RS_BOUNDARY_LANE = 3    /* signals with credits, but ensembles span them: each lane selects
                               the context before or after a signal for its own item (the
                               per-lane state selection proposed in Section 6)                    */
} rs_boundary;

#define RS_BOUNDARY(stage, mode) ((uint32_t)(mode) << (2 * (stage)))

/* Fill *opts with the defaults above (strategy = RS_STRATEGY_TAG). */
rs_status rs_default_opts(rs_pipeline_opts *opts);

/* Create a pipeline from a stage list: stages[0] is RS_ENUM_HASH or RS_ENUM_LOAD,
 * stages[n-1] is RS_AGGREGATE or RS_EMIT, the ones between are FILTER / MAP / EXPAND.
 * Checks (RS_ERR_INVALID): 2 <= n <= RS_MAX_STAGES; kinds/ops/params legal; FILTER
 * and MAP have max_fanout 1, EXPAND 1..8; the queue capacity holds one ensemble's
 * worst-case output (Section 3.2).  No CUDA call is made. */
rs_status rs_pipeline_create(const rs_stage_desc *stages, uint32_t n_stages,
                             const rs_pipeline_opts *opts, rs_pipeline **out);
rs_status rs_pipeline_destroy(rs_pipeline *p);
/* Replace the options of an existing pipeline (same checks as create). */
rs_status rs_pipeline_set_opts(rs_pipeline *p, const rs_pipeline_opts *opts);
rs_status rs_pipeline_get_opts(const rs_pipeline *p, rs_pipeline_opts *opts);

/* ---- streams (Section 4 composite objects) ------------------------------------- */

typedef struct {
    uint64_t n_regions;             /* R, < 2^32                                             */
    const uint32_t *parents;        /* device, R ids p_r; NULL means p_r = r                 */
    const uint32_t *region_len;     /* device, R lengths L_r; or NULL when offsets are given */
    const uint32_t *region_offsets; /* device, R+1 non-decreasing CSR offsets (element index
                                       of each parent's first element); NULL = from lengths */
    const uint32_t *elements;       /* device, element array for RS_ENUM_LOAD, else NULL     */
    uint64_t n_elements;            /* entries in `elements` (bounds check), < 2^32 - 4096   */
    const uint32_t *ctx;            /* device, R context words t_r, or NULL (t_r = 0)        */
    uint32_t *out_count;            /* device, R; count of survivors per region (or NULL)    */
    uint64_t *out_sum;              /* device, R; sum of survivors per region (or NULL)      */
    uint32_t *out_min;              /* device, R; min survivor, 0xFFFFFFFF if none (or NULL) */
    uint64_t total_elements_hint;   /* sum of L_r if the caller knows it, else 0; only used to
                                       size work units (regions_per_unit = 0)               */
    uint32_t *out_values;           /* device, RS_EMIT pipelines only (else NULL): at least
                                       F * (offsets[R] - offsets[0]) entries; out_count is
                                       then required and is zeroed by every run             */
    uint64_t out_values_len;        /* entries in out_values (the device checks every write
                                       against it and reports RS_ERR_DEVICE_INPUT beyond)   */
    uint32_t *out2_count;           /* tree pipelines with two leaves: the second leaf's   */
    uint64_t *out2_sum;             /* results, R entries each (the same arrays as the     */
    uint32_t *out2_min;             /* first leaf's are required); else NULL               */
} rs_stream_desc;

/* Register a stream with the pipeline; it is processed by every later rs_run until
 * rs_clear_streams.  Only pointers are recorded; nothing is read now.  Empty streams
 * (R = 0) are accepted.  *stream_id is the index used by rs_fetch_region_results. */
rs_status rs_stream_submit(rs_pipeline *p, const rs_stream_desc *s, uint64_t *stream_id);
rs_status rs_clear_streams(rs_pipeline *p);

/* ---- sliced runs over resident per-stream state (bounded launches) ------------------
 * A stream's work is a sequence of n_units merge-path units (whole-parent units for
 * hashed enumeration); every unit can run in any launch once the stream is planned,
 * because the aggregate folds each unit's items into the region outputs with integer
 * reductions (Section 4's begin/run/end, merged across pieces).  A sliced run keeps the
 * stream's planning state -- its unit records, planner words and merge slots -- in a
 * caller-owned device buffer that outlives the launch, and each launch processes a
 * bounded number of the stream's units.  This is the serving form: many streams advance
 * a slice at a time and new ones join between launches. */

/* Bytes of resident state a sliced run of stream s needs (0 for hashed enumeration, which
 * needs none) and its number of units, under the pipeline's current options (units of
 * loaded streams are an upper bound: the planner may use fewer; units past the last one
 * are skipped).  Host-only. */
rs_status rs_stream_state_size(const rs_pipeline *p, const rs_stream_desc *s, uint64_t *state_bytes,
                               uint64_t *n_units);

/* Submit stream s for the next rs_run with only its units [unit_begin, unit_begin +
 * unit_count) (clamped to the stream's units).  `state` (device, 256-byte aligned,
 * caller-owned, at least rs_stream_state_size bytes; may be NULL for hashed enumeration)
 * must be the same buffer for every slice of the stream and must not change in between.
 * unit_begin == 0 plans the stream: the run clears the state and writes the stream's unit
 * records (and the identity results the planner owns) before its units run.  The
 * region results are complete once every unit has run (the signal strategy writes the
 * merged results of split parents in the run holding the last unit); the options must not
 * change between slices of one stream.  Sliced streams cannot be captured in a graph
 * (RS_ERR_STATE): each slice is a submission of its own.  Errors as rs_stream_submit;
 * rs_run returns RS_ERR_CAPACITY if a state is too small. */
rs_status rs_stream_submit_slice(rs_pipeline *p, const rs_stream_desc *s, void *state, uint64_t state_bytes,
                                 uint64_t unit_begin, uint64_t unit_count, uint64_t *stream_id);

/* Bytes of caller-owned device workspace rs_run needs for the streams submitted so
 * far (work cursor, look-back words, stream table, counters, status word). */
rs_status rs_workspace_size(const rs_pipeline *p, uint64_t *bytes);

/* Enqueue one pass over every submitted stream on `stream`: one persistent kernel
 * launch (plus a memset of the workspace header).  Asynchronous; results land in
 * each stream's out_* arrays.  RS_ERR_CAPACITY if workspace_bytes is too small,
 * RS_ERR_NOT_READY if nothing is submitted, RS_ERR_CUDA on a launch failure. */
rs_status rs_run(rs_pipeline *p, void *workspace, uint64_t workspace_bytes, rs_cuda_stream stream);

/* Host copies of a submitted stream's inputs (any may be NULL: not copied). */
typedef struct {
    const uint32_t *parents;         /* R entries     */
    const uint32_t *region_len;      /* R entries     */
    const uint32_t *region_offsets;  /* R + 1 entries */
    const uint32_t *elements;        /* n_elements    */
    const uint32_t *ctx;             /* R entries     */
} rs_host_inputs;

/* Enqueue host-to-device copies of stream `stream_id`'s inputs from `src` into the device
 * arrays it was submitted with (sizes from its description), on `stream`: with
 * rs_run and rs_fetch_region_results, one pass from host buffers to host results through
 * this ABI.  Page-locked sources make the copies asynchronous (the cudaMemcpyAsync rule:
 * keep them unchanged until the copies have run).  RS_ERR_INVALID for an array the
 * stream was submitted without. */
rs_status rs_stream_upload(rs_pipeline *p, uint64_t stream_id, const rs_host_inputs *src, rs_cuda_stream stream);

typedef struct {
    uint32_t *count;    /* destination (host or device), R entries, or NULL */
    uint64_t *sum;
    uint32_t *min;
} rs_region_results;

/* Enqueue copies of stream `stream_id`'s per-region results into dst (any memory
 * cudaMemcpyAsync accepts).  Asynchronous like rs_run. */
rs_status rs_fetch_region_results(rs_pipeline *p, uint64_t stream_id, const rs_region_results *dst,
                                  rs_cuda_stream stream);

/* ---- statistics and device status ---------------------------------------------- */

typedef struct {
    uint32_t device_status;            /* bit 0 stall, 1 look-back timeout, 2 copy timeout,
                                          3 bad offsets/bounds, 4 internal queue overflow   */
    uint32_t n_nodes;
    uint64_t units;                    /* work units claimed                                */
    uint64_t ensembles[RS_MAX_STAGES]; /* ensembles fired per node (node 0 = enumerate)     */
    uint64_t items[RS_MAX_STAGES];     /* items consumed per node (active lanes)            */
    uint64_t signals[RS_MAX_STAGES];   /* signals consumed per node                         */
    uint64_t firings[RS_MAX_STAGES];   /* scheduler firings per node                        */
    uint64_t cycles[16];               /* profiling build only (else 0): SM cycles summed over
                                          processors in setup, look-back, tile waits, signal
                                          emission, nodes 1..5 (slots 5..9, tile waits
                                          included in node 1), result flush, lifetime, and
                                          inside the nodes: node 1's gather, stage compute,
                                          compaction, tile recycling                       */
    /* launch shape of the last enqueued pipeline kernel (host-side facts) */
    uint32_t grid;                     /* CTAs                                              */
    uint32_t block;                    /* threads per CTA (32 per processor)                */
    uint32_t smem_per_block;           /* dynamic shared memory per CTA, bytes              */
    uint32_t blocks_per_sm;            /* resident CTAs per SM (occupancy calculator)       */
    uint32_t chunk_parents;            /* tag strategy: parents node 1 loads per chunk, 32
                                          (one per lane) or 64 (two per lane, chosen when the
                                          loaded streams' regions average under 7 elements);
                                          0 for the signal strategy                         */
} rs_stats;

/* Synchronise `stream`, read the workspace counters of the last rs_run and return
 * RS_ERR_STALL / RS_ERR_DEVICE_INPUT if the device flagged a problem (stats filled
 * either way).  Active-lane fraction of node i = items[i] / (W * ensembles[i]). */
rs_status rs_get_stats(rs_pipeline *p, const void *workspace, rs_cuda_stream stream, rs_stats *out);

/* ---- batching in a CUDA graph (many streams, one launch, replayed) ------------- */

/* Capture rs_run for the submitted streams into a CUDA graph owned by the pipeline. */
rs_status rs_graph_capture(rs_pipeline *p, void *workspace, uint64_t workspace_bytes, rs_cuda_stream stream);
/* Replay the captured graph on `stream`. */
rs_status rs_graph_launch(rs_pipeline *p, rs_cuda_stream stream);
rs_status rs_graph_release(rs_pipeline *p);

/* ---- autotuning (Section 5: choose per workload, from measurements) ------------ */

/* Choose options by timed trials on the submitted streams (the profile-guided choice
 * of Section 5): for each strategy (both when the pipeline's strategy option is
 * RS_STRATEGY_AUTO, else only the one it names), a coordinate search from the defaults over the
 * unit shape (regions_per_unit x region_cost, or whole-parent unit sizes for hashed
 * streams), then ensemble width, processors per CTA, tile size and queue capacity (1, 2
 * and 4 times the smallest legal one), each change kept when faster; a strategy starting
 * above three times the best so far is dropped.  With RS_STRATEGY_AUTO and a linear
 * pipeline it then tries per-edge boundary modes: signals into the first stages and tags
 * from stage s on, for every s (the per-stage choice of Section 5), per-lane selection on
 * every edge, and per-lane selection into stage 1 with tags after it.
 * Each trial is one warm-up and `trials` timed runs (CUDA events).  The fastest is
 * kept in the pipeline and returned in *best (mean milliseconds in *best_ms).
 * Overwrites the streams' outputs. */
rs_status rs_autotune(rs_pipeline *p, void *workspace, uint64_t workspace_bytes, rs_cuda_stream stream,
                      uint32_t trials, rs_pipeline_opts *best, float *best_ms);

/* ---- per-launch kernel timing --------------------------------------------------- */

/* When enabled (capacity > 0), every rs_run records a pair of CUDA events on its
 * stream immediately before and after its kernel launch, into a ring of `capacity`
 * slots owned by the pipeline (capacity 0 disables and frees them).  Not recorded
 * inside rs_graph_capture. */
rs_status rs_timing_enable(rs_pipeline *p, uint32_t capacity);
/* Wait for the recorded events, write up to `max` kernel durations in milliseconds
 * (launch order) to ms[], their number to *n, and empty the ring. */
rs_status rs_timing_read(rs_pipeline *p, float *ms, uint32_t max, uint32_t *n);

/* ---- serving: continuous batching of arriving streams --------------------------- */

typedef struct rs_server rs_server;

/* One request: a whole stream in HOST memory (page-locked for asynchronous copies).
 * The input arrays must stay valid, and the output arrays must not be read, until the
 * request id comes back from rs_server_poll. */
typedef struct {
    uint64_t n_regions;
    const uint32_t *parents;     /* host, R ids, or NULL (p_r = r)                  */
    const uint32_t *region_len;  /* host, R lengths                                 */
    const uint32_t *elements;    /* host, for RS_ENUM_LOAD, else NULL               */
    uint64_t n_elements;
    const uint32_t *ctx;         /* host, R context words, or NULL                  */
    uint32_t *out_count;         /* host outputs, R entries each, or NULL           */
    uint64_t *out_sum;
    uint32_t *out_min;
    uint64_t total_elements_hint;
} rs_request;

typedef struct {
    uint64_t submitted, admitted, completed;
    uint64_t batches, largest_batch;     /* launches (slices), most requests in one          */
    uint64_t in_flight, queued;          /* launches queued on the GPU, requests waiting for
                                            memory                                           */
    uint64_t arena_live, arena_peak;     /* bytes of the arena in use now / at most          */
    uint64_t gathered;                   /* launches whose finished requests' results came
                                            back with one gather kernel and one copy        */
    uint64_t per_array;                  /* ... with one copy per output array (no room)    */
} rs_server_stats;

/* A server over one linear stage list (not ending in an emit sink).  `arena` (device,
 * caller-owned, 256-byte aligned) is the device memory budget: a request is admitted only
 * when its inputs, outputs and resident state (rs_stream_state_size) fit in the arena's
 * free part, and stays there until it finishes; every launch's workspace comes from it
 * too.  Each launch (a slice) advances every active request -- up to max_batch of them
 * (0 = 4096) -- by at most the slice budget of work units (rs_server_set_slice_units),
 * so requests arriving meanwhile join the next launch.  Up to max_inflight (0 = 2)
 * launches are queued on `stream`; admissions' copies and finished requests' result
 * copies run on two streams of the server's own, so they overlap the launches on the
 * device.  RS_STRATEGY_AUTO serves with the tag strategy (a request's units are sized
 * once, at submission).  No CUDA call is made here. */
rs_status rs_server_create(const rs_stage_desc *stages, uint32_t n_stages, const rs_pipeline_opts *opts,
                           void *arena, uint64_t arena_bytes, uint32_t max_batch, uint32_t max_inflight,
                           rs_cuda_stream stream, rs_server **out);
/* Work units each active request runs per launch (default 64); 0 runs every request to
 * completion in the launch it joins. */
rs_status rs_server_set_slice_units(rs_server *s, uint32_t units);
/* Queue a request (host-side only; admitted by a later rs_server_progress).
 * RS_ERR_CAPACITY if it needs more than half the arena. */
rs_status rs_server_submit(rs_server *s, const rs_request *r, uint64_t *req_id);
/* Non-blocking step: retire launches whose finished requests' results have landed
 * (copied into the requests' host outputs here; their arena space is freed), admit queued
 * requests while the arena has room (their inputs copied on the server's copy-in stream),
 * and launch slices while fewer than max_inflight are queued.  The results of the
 * requests a launch finishes come back with one gather kernel and one device-to-host copy
 * into a page-locked staging buffer of the server's (host memory, allocated with
 * cudaMallocHost when a launch first needs one that large, reused afterwards); if that
 * cannot be had, with one copy per output array.  The first call creates the two copy
 * streams. */
rs_status rs_server_progress(rs_server *s);
/* Ids of requests completed since the last poll (up to max; *n = how many). */
rs_status rs_server_poll(rs_server *s, uint64_t *ids, uint32_t max, uint32_t *n);
rs_status rs_server_get_stats(const rs_server *s, rs_server_stats *out);
/* Synchronise the server's stream and free the server. */
rs_status rs_server_destroy(rs_server *s);

/* ---- running without a caller workspace ------------------------------------------ */

/* The paper has no counterpart to this entry point; it serves callers that cannot
 * allocate device memory when they run the pipeline (a host application that owns the
 * device-memory budget through its own allocator or a hard cap, or a latency-critical
 * loop where an allocation could synchronise the device).
 *
 * Same work and results as rs_run, but the scratch memory (work cursor, planner words,
 * unit records, merge slots, stream table) lives in a fixed 16 MiB array compiled into
 * the library (every GPU that loads the library holds it until the process exits).
 * The call allocates nothing: no cudaMalloc, cudaFree or cudaMallocHost, and no
 * allocating library routine.
 *   - The first call on a device (with that device current) looks up the array's
 *     device address once; make that first call before any stream capture.  The
 *     address is kept until the process exits, so resetting a device
 *     (cudaDeviceReset) while the library is loaded is not supported here.
 *   - RS_ERR_CAPACITY, with nothing enqueued, if the submitted streams need more than
 *     16 MiB of scratch (rs_workspace_size reports the need) or more than 64 streams
 *     are submitted.
 *   - Every call shares the one array and clears what must start at zero; calls whose
 *     work overlaps on the GPU (other CUDA streams, other host threads, other
 *     pipelines) race on it and must be serialised by the caller.
 *   - rs_get_stats reads a caller workspace and does not apply to these runs. */
rs_status rs_run_noalloc(rs_pipeline *p, rs_cuda_stream stream);

/* ---- calibration ---------------------------------------------------------------- */

/* A measurement aid, not part of the pipeline: the cascade's element arithmetic over ONE
 * region with no region handling at all.  elements[0..n) (device memory, any alignment;
 * 16-byte aligned arrays are read with vector loads) pass three filters in a row, each
 * keeping x when (hash32(x, salts[i]) XOR ctx) < thetas[i] -- the context-hash filter of
 * Section 5's cascade, every element under the one context word ctx -- with the ensemble
 * queues and compaction of the pipeline kernels between them; out[0] (device, 8-byte
 * aligned, two words) receives the survivors' count and out[1] their sum (zeroed first
 * on `stream`).  The results equal a pipeline run on a stream of one region of n elements
 * with context word ctx; the time bounds from above what the pipeline kernels can reach
 * on the same elements.  salts and thetas are host arrays of 3.  RS_ERR_INVALID on a null
 * or misaligned argument, RS_ERR_CUDA on a launch failure. */
rs_status rs_calibrate_cascade(const uint32_t *elements, uint64_t n, uint32_t ctx, const uint32_t *salts,
                               const uint32_t *thetas, uint64_t *out, rs_cuda_stream stream);

/* ---- misc ---------------------------------------------------------------------- */

const char *rs_status_string(rs_status s);
/* Last CUDA error code seen by the library on this thread (0 if none). */
int rs_last_cuda_error(void);
/* Library version, for the binding's load check. */
uint32_t rs_version(void);
/* sizeof of the ABI structs, so a binding can check its mirrors: writes up to `max`
 * entries in this order -- rs_stage_desc, rs_pipeline_opts, rs_stream_desc,
 * rs_region_results, rs_stats, rs_request, rs_server_stats -- and returns how many it
 * knows (7).  Host-only; needs no GPU. */
uint32_t rs_struct_sizes(uint64_t *sizes, uint32_t max);

#ifdef __cplusplus
}
#endif
#endif /* RS_H */
