/*
 * rv.h -- C ABI of librv, B300-native runtime verification of LTL4-C formulas.
 *
 * LTL4-C ("Accelerated Runtime Verification of LTL Specifications with
 * Counting Semantics", Medhat, Joshi, Bonakdarpour, Fischmeister) is LTL with
 * four-valued runtime semantics (Def. "LTL4 semantics", Sec. 2.2.2) under a
 * string of counting quantifiers: A (percentage of instances) and E (number
 * of instances), each with a numeric constraint (Def. 1, Sec. 2.1).  A trace
 * verdict is one of six truth values (Sec. 2.3, Def. "LTL4-C Semantics").
 *
 * The library implements Algorithm 1 (Sec. 4.2) on one GPU:
 *   map      (SortTrace)          events grouped by binding key,
 *   monitor  (Distribute)         each binding's LTL4 Moore monitor steps over
 *                                 its projected sub-trace,
 *   reduce   (ApplyQuantifiers)   per-parent verdict counts, then each
 *                                 quantifier's constraint in exact integers.
 *
 * Conventions for every entry point:
 *   - Return an rv_status; RV_OK (0) means success.  rv_last_error() gives a
 *     thread-local message for the last failure.  No C++ exception and no
 *     process exit crosses this interface; device-side faults are reported
 *     through a device status word, never by trapping.
 *   - The caller owns every input and output buffer.  The library owns the
 *     objects it returns (rv_formula, rv_service, rv_stream) and frees them in
 *     the matching *_free / *_close call.
 *   - "device pointer" means memory of the current CUDA device; "host
 *     pointer" means ordinary (or pinned) host memory.
 *   - Timestamps are optional everywhere: the order of a trace is its array
 *     order (Sec. 2, Def. "Trace"); when a ts array is given it is checked to
 *     be non-decreasing and a violation returns RV_EINVAL.
 */
#ifndef RV_H
#define RV_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RV_OK = 0,
  RV_EPARSE = 1,        /* formula text does not follow Def. 1 */
  RV_EUNSUPPORTED = 2,  /* more than 16 monitor states, > 2 quantifiers, too large a body */
  RV_EINVAL = 3,        /* bad argument or bad trace (predicate code out of range, ts decreasing) */
  RV_ENOMEM = 4,        /* workspace too small or allocation failed */
  RV_EAGAIN = 5,        /* streaming: chunk not admitted now (memory budget), retry later */
  RV_ETIMEOUT = 6,      /* poll timed out, or a bounded device wait gave up */
  RV_ECUDA = 7,         /* a CUDA runtime call failed */
  RV_EINTERNAL = 8      /* device status word reports an internal limit/bug */
} rv_status;

/* Six truth values in their lattice order F < Fc < Fp < Tp < Tc < T (Sec. 2.3). */
typedef enum {
  RV_BOT = 0, RV_BOT_C = 1, RV_BOT_P = 2, RV_TOP_P = 3, RV_TOP_C = 4, RV_TOP = 5
} rv_verdict;

enum { RV_ONEHOT = 0, RV_BITMASK = 1 };          /* alphabet modes */
enum { RV_Q_A = 0, RV_Q_E = 1 };                 /* quantifier kinds (Eq. bigq) */
enum { RV_LT = 0, RV_LE = 1, RV_GT = 2, RV_GE = 3, RV_EQ = 4 };  /* comparison ~ */

#define RV_MAX_STATES 16
#define RV_MAX_LETTERS 256
#define RV_MAX_CMP 4

/* Interpretation of the predicate byte of an event (Sec. 2: events are sets
 * of predicates).  RV_ONEHOT: code c is the single predicate code_names[c]
 * (n_codes <= 256).  RV_BITMASK: bit i of the byte means code_names[i] holds
 * (n_codes <= 8), so one event can carry several predicates.
 * key_bits: width of the key column, 32 or 64.  With two quantified variables
 * the key must be 64-bit and holds (d0 << 32) | d1.
 * value_name (may be NULL): name of an optional uint32 value column of the
 * events, a program variable such as case study 2's average chunk size of a
 * user's session (Sec. 5.1).  Body atoms "value_name ~ c" or
 * "value_name(args) ~ c" (~ one of < <= > >= =, c an integer constant in
 * [0, 2^32)) are interpreted predicates: true at an event iff its value
 * compares so with c. */
typedef struct {
  int n_codes;
  const char* const* code_names;
  int alphabet;
  int key_bits;
  const char* value_name;
} rv_schema;

typedef struct rv_formula rv_formula;

typedef struct {
  int n_quant;     /* 0, 1 or 2 counting quantifiers */
  int n_states;    /* states of the minimal LTL4 Moore monitor of the body (<= 16) */
  int n_letters;   /* number of distinct predicate bytes: n_codes or 2^n_codes */
  int q0;          /* initial monitor state */
  int key_bits;
  int alphabet;
  int n_base;      /* letters of the predicate byte alone */
  int n_cmp;       /* comparison atoms (letter = code + n_base * outcome bits) */
} rv_formula_info;

/* Parse `text` (Def. 1 syntax, defaults A = A_{=1}, E = E_{>=1}) and
 * synthesise the LTL4 monitor of its body over the schema's alphabet
 * (Def. "LTL4 Monitor", Sec. 2.2.3).  Concrete grammar: a formula is zero to
 * two binders `Q_{~c} x: p(x) =>` followed by the body; Q is A (c a decimal
 * or percentage in [0,1]) or E (c an integer >= 0), ~ one of < <= > >= =;
 * the body is LTL over the schema's code names with ! && || -> <-> (also
 * & | and =>), X F G, and infix U R W, tightest first: unary operators,
 * U/R/W, &&, ||, ->, <->.
 * On error returns RV_EPARSE / RV_EUNSUPPORTED / RV_EINVAL and writes a
 * message into err[errlen] (may be NULL).  *out is owned by the caller and
 * released with rv_formula_free.  Host only; no GPU work. */
rv_status rv_compile_formula(const char* text, const rv_schema* schema, rv_formula** out,
                             char* err, size_t errlen);
rv_status rv_formula_get_info(const rv_formula* f, rv_formula_info* info);
/* Monitor tables (host copies): maps[l] for each letter l < n_letters holds the
 * transition map of letter l with nibble s = delta(s, l); labels[s] is the
 * verdict lambda(s) in rv_verdict coding (one of F, Fp, Tp, T). */
rv_status rv_formula_tables(const rv_formula* f, uint64_t* maps, int n_maps, uint8_t labels[16]);
/* Quantifier tuple <Q_i, ~_i, c_i> of level i (Eq. bigq): kind RV_Q_A/E,
 * op RV_LT..RV_EQ, constant num/den (den = 1 for E). */
rv_status rv_formula_quantifier(const rv_formula* f, int level, int* kind, int* op,
                                uint64_t* num, uint64_t* den);
void rv_formula_free(rv_formula* f);

/* Six-valued valuation of one quantifier node from its child-verdict counts
 * v[0..5] (Eq. S and Def. "LTL4-C Semantics").  The cases are tried
 * top-down in lattice order; for >=/> the count sums are the printed ones,
 * for <=/< the mirrored ones (the children that could still be true push the
 * count up), '=' is an exact integer equality under the same rungs, and the
 * permanence rules are Table 1 (E) and, for A, what holds for every
 * continuation that adds children of any verdict.  Host entry of the same
 * function the reduce kernels run. */
rv_status rv_valuate(int kind, int op, uint64_t num, uint64_t den, const uint64_t v[6], int* verdict);

/* ------------------------------------------------------------------ offline verification */

/* A trace as a structure of arrays in trace order: key (uint32 or uint64 per
 * key_bits), pred (uint8 predicate byte), optional ts (uint32, may be NULL),
 * value (uint32, the schema's value column; needed only by formulas with
 * comparison atoms, which the offline and timeline entry points accept). */
typedef struct {
  const void* key;
  const uint8_t* pred;
  const uint32_t* ts;
  uint64_t n;
  const uint32_t* value;
} rv_trace;

typedef struct {
  int32_t root;               /* [u |=_6 phi] as rv_verdict */
  int32_t status;             /* rv_status of the device work */
  uint64_t root_counts[6];    /* the root's child-verdict vector v (Sec. 3.4) */
  uint64_t level_counts[2][6];/* verdict histogram of the level-1 and level-2 nodes */
  uint64_t n_nodes[2];        /* number of distinct D|^1 and D|^2 (value-vector prefixes) */
  uint64_t events;
} rv_result;

/* Optional per-binding outputs (device pointers, caller-owned).  keys/verdicts
 * receive one entry per innermost binding (LTL4 verdict); outer_* one entry per
 * level-1 node of a two-quantifier formula (six-valued verdict).  The order is
 * unspecified.  Capacity n (events) always suffices. */
typedef struct {
  uint64_t* keys;
  uint8_t* verdicts;
  uint64_t capacity;
  uint64_t* outer_keys;
  uint8_t* outer_verdicts;
  uint64_t outer_capacity;
} rv_bindings;

/* Tuning knobs; zero means "choose automatically". */
typedef struct {
  int bucket_bits;       /* log2 of the first-level key buckets, 8..11 */
  int sub_bucket_bits;   /* log2 of the second-level split, 0..7 (0..8 without heavy-key routing:
                            two variables, no_heavy) */
  int unit_records;      /* records folded by one CTA, multiple of 256 */
  int no_heavy;          /* nonzero: no own sub-buckets for bindings that a sample of
                            the trace shows to be heavy (one-variable formulas) */
  int test_wait_polls;   /* test aid, 0 in normal use: > 0 makes the last kernel wait
                            for a device flag that nothing sets, giving up after this
                            many polls; the result's status is then RV_ETIMEOUT, the
                            verdicts are still computed and the context stays usable
                            (exercises the bounded-wait path without a GPU fault) */
} rv_verify_opts;

/* Device memory the offline path needs for a trace of n events
 * (host_input != 0 adds room to stage host arrays on the device). */
size_t rv_verify_workspace_size(const rv_formula* f, uint64_t n, int host_input,
                                const rv_verify_opts* opts);

/* Verify one trace against one formula (Algorithm 1: SortTrace, SpawnMonitors,
 * Distribute, ApplyQuantifiers).  on_device != 0: t's arrays are device
 * pointers; otherwise host pointers that are copied in on stream s.  ws is a
 * device workspace of at least rv_verify_workspace_size bytes (NULL: the
 * library allocates and frees one).  Blocks until the result is in *out.
 * Errors: RV_EINVAL (bad trace), RV_ENOMEM (workspace), RV_ECUDA. */
rv_status rv_verify_trace(const rv_formula* f, const rv_trace* t, int on_device, void* ws,
                          size_t ws_bytes, rv_result* out, const rv_bindings* bindings,
                          const rv_verify_opts* opts, cudaStream_t s);

/* Asynchronous form for device-resident traces: enqueues all work on s and
 * writes the result into the device struct *dev_out; no host synchronisation.
 * The caller reads dev_out after synchronising s.  Device-side outcomes are in
 * dev_out->status: RV_EINVAL for a bad trace (predicate code out of range,
 * timestamps decreasing); RV_EAGAIN, for two-quantifier formulas only, when
 * more distinct outer values fell into one key bucket than a fold unit can
 * count (256; the default split uses 2^16 buckets by hash of the outer value,
 * so only keys crafted to collide reach it) -- rerun through rv_verify_trace,
 * which reports it as an error with a message. */
rv_status rv_verify_trace_async(const rv_formula* f, const rv_trace* t, void* ws, size_t ws_bytes,
                                rv_result* dev_out, const rv_bindings* bindings,
                                const rv_verify_opts* opts, cudaStream_t s);

/* ------------------------------------------------------------------ per-event timeline
 * The online mode of Algorithm 1 (Sec. 4.2) yields an evolving verdict; this
 * gives it at event granularity.  For event j whose innermost binding is D
 * (its key: the 32- or 64-bit key, (d0 << 32) | d1 with two variables, one
 * binding for an unquantified property), event_verdicts[j] is the LTL4
 * verdict (Def. "LTL4 semantics", Sec. 2.2.2; rv_verdict code F, Fp, Tp or T)
 * of D's projection (Sec. 2.4.3) cut after event j.  Every binding whose
 * verdict becomes F adds one pair (viol_keys[i], viol_index[i]): its key and
 * the trace index of its first F event (F is permanent); *n_viol receives the
 * number of pairs, in unspecified order.
 * t holds device arrays; event_verdicts (n bytes), viol_keys (uint64[n]),
 * viol_index (uint32[n]) and n_viol (one uint64) are device memory owned by
 * the caller; ws is a device workspace of rv_timeline_workspace_size bytes.
 * Runs on stream s and returns when the results are complete (it reads a
 * small status back).  The events are grouped by a stable radix sort of (key,
 * index) and each binding's states come from a segmented scan of composed
 * 64-bit transition maps, so long bindings spread over the whole GPU.
 * Errors: RV_EINVAL (null arrays, predicate code out of range), RV_ENOMEM
 * (workspace), RV_ECUDA. */
size_t rv_timeline_workspace_size(const rv_formula* f, uint64_t n);
rv_status rv_verify_timeline(const rv_formula* f, const rv_trace* t, void* ws, size_t ws_bytes,
                             uint8_t* event_verdicts, uint64_t* viol_keys, uint32_t* viol_index,
                             uint64_t* n_viol, cudaStream_t s);

/* ------------------------------------------------------------------ front end: strace text -> events
 * The paper monitors programs through strace; its parsing module translates
 * strace strings into a numerical table (Sec. 5).  rv_parse_strace does that
 * on the GPU.  Each line of `text` (device memory, `bytes` long, lines ended
 * by '\n', a last unterminated line included) has the form
 *     [pid] TIME NAME(ARGS...) = RET [ERRNO (text)]
 * with the pid optional ("[pid N] " or "N ") and TIME either
 * seconds.microseconds (strace -ttt) or HH:MM:SS.microseconds (-tt).  A line
 * whose NAME matches a rule becomes one event: pred = the rule's code, key =
 * the first argument (RV_KEY_ARG0, e.g. the descriptor a read or close works
 * on) or the return value (RV_KEY_RET, e.g. the descriptor socket or accept
 * makes), ts = TIME in microseconds.  A call that strace -f splits into
 * "NAME(ARGS <unfinished ...>" and "<... NAME resumed> ...) = RET" yields one
 * event, from the line that holds its key.  Lines of other calls, signals and
 * exits, calls whose key is missing, and failed calls (RET < 0) when the rule
 * sets ok_only (RV_KEY_RET rules always need RET >= 0) are dropped.  Events
 * keep the order of their lines.
 * key_out (uint32), pred_out (uint8) and ts_out (uint64, may be NULL) are
 * device arrays of `capacity` entries; *n_events (host) receives the number
 * of events; more than capacity returns RV_ENOMEM after writing the first
 * capacity.  ws: device workspace of rv_parse_workspace_size(bytes) bytes
 * (8 bytes per 8 KiB of text plus a few words); text may start at any byte
 * address (16-byte aligned text is read with wider loads).  Runs on s and
 * returns when the table is complete.  1..16 rules, names of at most 23
 * characters.  Errors: RV_EINVAL, RV_ENOMEM, RV_ETIMEOUT (a bounded device
 * wait between text tiles gave up; the table is then not valid), RV_ECUDA. */
#define RV_PARSE_MAX_RULES 16
#define RV_PARSE_NAME_LEN 24
enum { RV_KEY_ARG0 = 0, RV_KEY_RET = 1 };
typedef struct {
  const char* name;   /* system call name, e.g. "recvfrom" */
  int code;           /* predicate code of its events */
  int key_from;       /* RV_KEY_ARG0 or RV_KEY_RET */
  int ok_only;        /* nonzero: drop calls that returned a negative value */
} rv_syscall_rule;
size_t rv_parse_workspace_size(uint64_t bytes);
rv_status rv_parse_strace(const char* text, uint64_t bytes, const rv_syscall_rule* rules, int n_rules,
                          void* ws, size_t ws_bytes, uint32_t* key_out, uint8_t* pred_out, uint64_t* ts_out,
                          uint64_t capacity, uint64_t* n_events, cudaStream_t s);

/* ------------------------------------------------------------------ one trace over several ranks
 * Algorithm 1 (Sec. 4.2) evaluates every binding on its own projection
 * (Sec. 2.4.3); all bindings of one outer value d_0 form one subtree of the
 * submonitor tree (Sec. 3.3), and the only step that joins subtrees,
 * ApplyQuantifiers, counts verdicts per level (the vectors v of Sec. 3.4),
 * which are sums.  So a trace splits by its outermost quantified value into
 * parts that are verified independently (one per rank), and the parts' counts
 * add up to the whole trace's.  Rank of an event: a hash of its outer value
 * (the key with one variable, key >> 32 with two) scaled to [0, world); it is
 * independent of the key mixing inside the verifier.
 *   rv_shard_of: the rank of each of n host keys (key_bits of f), written to
 *     the host array rank_out[n].  Host only; no GPU work.
 *   rv_shard_workspace_size / rv_shard_trace: device form.  t holds device
 *     arrays; the events are written to key_out/pred_out (ts_out when t has
 *     timestamps, value_out when it has values), device arrays of n entries, grouped into world
 *     contiguous segments in rank order, trace order kept inside every
 *     segment; counts_out (device uint64[world]) receives the segment sizes.
 *     ws: device workspace of at least rv_shard_workspace_size bytes.  Work is
 *     queued on s; nothing is synchronised.  1 <= world <= 256.
 *   rv_combine_results: the result of the whole trace from the results of its
 *     parts (host structs): counts, node numbers and events summed, the root
 *     valuated on the summed root counts, the first failed part's status.  A
 *     single part that already holds summed counts (an all-reduce) is
 *     re-valuated the same way.
 * Errors: RV_EINVAL (null arguments, world out of range, an unquantified
 * property -- its one binding is the whole trace -- with world > 1),
 * RV_ENOMEM (workspace), RV_ECUDA. */
rv_status rv_shard_of(const rv_formula* f, const void* key, uint64_t n, int world, uint32_t* rank_out);
size_t rv_shard_workspace_size(uint64_t n, int world);
rv_status rv_shard_trace(const rv_formula* f, const rv_trace* t, int world, void* ws, size_t ws_bytes,
                         void* key_out, uint8_t* pred_out, uint32_t* ts_out, uint32_t* value_out,
                         uint64_t* counts_out, cudaStream_t s);
rv_status rv_combine_results(const rv_formula* f, const rv_result* parts, int n_parts, rv_result* out);

/* ------------------------------------------------------------------ batched verification
 * Many traces of uneven length, each checked against its own list of nf
 * single-quantifier formulas (nf <= 32), in one fixed sequence of launches
 * captured in a CUDA graph (Algorithm 1, with the grouping of a trace shared
 * by all of its formulas).  The traces are concatenated: key uint32[n] and
 * pred uint8[n] hold trace t at [offsets[t], offsets[t+1]).  Formula j of
 * trace t is f[t * nf + j]; all formulas of a trace must have one quantifier,
 * 32-bit keys and the trace's alphabet (at most 16 letters).
 *   rv_batch_create: validate, copy the monitor tables, plan buckets and warp
 *     tiles from the offsets (host arrays; copied).  Device memory for the
 *     plan comes from the registered allocator (or cudaMalloc).
 *   rv_batch_run: key/pred/ws/dev_results are device pointers; results
 *     rv_result[nt * nf] land in dev_results after s completes.  The launch
 *     sequence is captured once per argument set and replayed as a graph.
 *     Cluster thresholds: a trace's bindings are hashed into buckets of about
 *     bucket_records records (16 to 2048 buckets per trace, so a short
 *     trace's buckets are smaller), whose bindings one CTA folds (lane = formula,
 *     in passes of at most 512 bindings each); a bucket longer than
 *     long_records (its runs too long for one CTA) is cut into segments of
 *     long_records records: later segments are folded by CTAs of their own
 *     into composed 64-bit transition maps (Sec. 4.2 composes monitors per
 *     binding; here per segment), which the bucket's fold applies in order.
 *     A result's status: RV_EINVAL (predicate code out of range),
 *     RV_ETIMEOUT (a bounded device wait gave up), RV_EINTERNAL.
 *   rv_batch_autotune: times the candidate bucket sizes and warp-tile lengths
 *     on the given inputs, then the candidate long_records with the best of
 *     those, keeps the fastest and reports it in *chosen. */
typedef struct rv_batch rv_batch;
typedef struct {
  int bucket_records;   /* target records per bucket (per trace), default 4096 */
  int tile_events;      /* events per warp tile of the split, default 16384 */
  int long_records;     /* segment length of long buckets, default 65536; < 0: never split */
} rv_batch_opts;
rv_status rv_batch_create(const rv_formula* const* f, int nf, int nt, const uint64_t* offsets,
                          const rv_batch_opts* opts, rv_batch** out);
size_t rv_batch_workspace_size(const rv_batch* b);
rv_status rv_batch_run(rv_batch* b, const uint32_t* key, const uint8_t* pred, void* ws, size_t ws_bytes,
                       rv_result* dev_results, cudaStream_t s);
rv_status rv_batch_autotune(rv_batch* b, const uint32_t* key, const uint8_t* pred, void* ws, size_t ws_bytes,
                            rv_result* dev_results, cudaStream_t s, rv_batch_opts* chosen);
void rv_batch_free(rv_batch* b);

/* ------------------------------------------------------------------ online serving
 * The online mode of Algorithm 1 (Sec. 4.2): repeated invocations on newly
 * arrived events update the submonitor tree, whose state stays on the GPU.
 * A service owns one formula (one or two quantifiers; one-quantifier streams
 * use 32-bit keys, two-quantifier streams 64-bit (d0 << 32) | d1 keys) and up
 * to max_streams open streams, each an independent trace.  Continuous batching: a
 * push only stages the chunk (host copy) and returns; a worker thread batches
 * every staged chunk (at most one per stream per batch) onto the GPU while
 * newer chunks keep arriving.  Every processed chunk yields one
 * rv_stream_verdict: the stream's six-valued verdict for its whole prefix up to
 * and including that chunk, and the push -> verdict latency.
 *   rv_stream_push: chunk arrays are host pointers, copied before return.
 *     RV_EAGAIN: not admitted (staging budget max_staged_events, or the
 *     worst case of one new binding per event would exceed max_bindings /
 *     max_outer); retry later.  RV_EINVAL: closed stream, decreasing ts.
 *   rv_stream_poll: up to max verdicts in ticket order; waits up to
 *     timeout_us; RV_ETIMEOUT when none arrived.
 *   rv_stream_close: drops the stream's queued chunks and verdicts and ends
 *     the handle (no call may use it afterwards).  Once no batch on the GPU
 *     carries its chunks, its bindings and outer nodes are retired on the
 *     device (their table entries and ids are reused by later bindings, so
 *     their memory counts toward admission again) and its slot is given back
 *     to rv_stream_open.
 *   Batches overlap: the worker stages and copies batch k+1 (its own pinned
 *   and device buffers, a copy stream) while batch k's kernels run; kernels
 *   run in batch order on one stream, so every chunk's verdict is that of its
 *   stream's prefix.  A batch that fails on the device gives its chunks that
 *   status and fails only the streams it carried (their later pushes return
 *   RV_EINVAL); other streams go on.  A failed CUDA call fails the service.
 *   rv_service_close: drains the worker and frees everything (device memory
 *     through the registered allocator). */
typedef struct rv_service rv_service;
typedef struct rv_stream rv_stream;
typedef struct {
  uint64_t max_bindings;      /* innermost bindings over all streams (default 2^24) */
  uint64_t max_outer;         /* outer nodes over all streams (default 2^22) */
  uint64_t max_batch_events;  /* events per device batch, also the largest chunk (default 2^22) */
  uint64_t max_staged_events; /* events admitted but not yet processed (default 2^25) */
  int max_streams;            /* default 64 */
} rv_service_cfg;
typedef struct {
  uint64_t ticket;            /* 1, 2, ... per stream, in push order */
  int32_t root;               /* rv_verdict of the stream prefix */
  int32_t status;             /* rv_status of the batch that carried the chunk */
  uint64_t root_counts[6];
  uint64_t events;            /* events of the stream up to this chunk */
  double latency_us;          /* push -> verdict visible to poll */
} rv_stream_verdict;
typedef struct {
  uint64_t batches, admitted, refused, events, bindings, outer_nodes, staged_events;
} rv_service_counters;
rv_status rv_service_open(const rv_formula* f, const rv_service_cfg* cfg, rv_service** out);
rv_status rv_service_close(rv_service* svc);
rv_status rv_stream_open(rv_service* svc, rv_stream** out);
rv_status rv_stream_push(rv_stream* st, const rv_trace* chunk, uint64_t* ticket);
rv_status rv_stream_poll(rv_stream* st, rv_stream_verdict* out, int max, int* n, int timeout_us);
rv_status rv_stream_close(rv_stream* st);
rv_status rv_service_stats(rv_service* svc, rv_service_counters* out);

/* ------------------------------------------------------------------ instrumentation
 * The paper times whole monitor runs (Sec. 5.2); these calls time each kernel.
 * rv_profile_enable(1): every kernel launch of the library is bracketed by a
 * pair of CUDA events recorded on the launching stream.  rv_profile_collect
 * waits for the recorded events, adds their durations into per-kernel totals
 * and copies up to max entries into out; it returns the number of distinct
 * kernels and clears the totals.  rv_launch_count: kernels launched by the
 * library in this process (profiling on or off). */
typedef struct {
  char name[48];
  uint64_t launches;
  double total_ms;
} rv_kernel_stat;
void rv_profile_enable(int on);
int rv_profile_collect(rv_kernel_stat* out, int max);
uint64_t rv_launch_count(void);

/* Offline verification that allocates no device memory (the paper has no
 * counterpart; this is a convenience of the library).  It is for callers that
 * cannot allocate when they verify: code running during CUDA graph capture,
 * where cudaMalloc is not allowed; hosts whose device memory is all owned by
 * another allocator; monitoring loops that must never block or fail on an
 * allocation.  Same arguments and result as rv_verify_trace_async (t holds
 * device arrays, *dev_out is a device struct, work is queued on s), but the
 * workspace is a fixed 64 MiB array inside the library, which every GPU that
 * loads librv keeps until the process exits.
 * Limits: traces of at most 1,000,000 events (and whose workspace fits the
 * 64 MiB); longer ones return RV_EINVAL with a message, nothing is queued.
 * Device-side outcomes are in dev_out->status exactly as for
 * rv_verify_trace_async (RV_EAGAIN there: outer values crafted to collide in
 * one key bucket; rerun through rv_verify_trace with a workspace).
 * The first call on a device looks up the array's device address (set-up,
 * once per device, with that device current) and keeps it for the life of
 * the process; make that first call before any stream capture.  A
 * cudaDeviceReset of that device invalidates the kept address: do not call
 * this entry point on a device after resetting it in the same process.  All
 * calls share the one array and each call clears what must start at zero:
 * calls whose work overlaps on the GPU (different streams, or host threads
 * without ordering) race and give wrong results. */
rv_status rv_verify_trace_noalloc(const rv_formula* f, const rv_trace* t, rv_result* dev_out, cudaStream_t s);

/* Last error message of the calling thread (never NULL). */
const char* rv_last_error(void);

/* Device allocator used when the library needs device memory of its own
 * (ws == NULL, streaming service).  NULL restores cudaMalloc/cudaFree. */
typedef void* (*rv_alloc_fn)(size_t bytes, void* ctx);
typedef void (*rv_free_fn)(void* ptr, void* ctx);
void rv_set_allocator(rv_alloc_fn alloc, rv_free_fn free_fn, void* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RV_H */
