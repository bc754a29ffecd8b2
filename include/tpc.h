/*
 * tpc — GB300 (sm_103a) clustering of Timepix hits into connected components.
 *
 * C ABI of the CUDA library libtpc.so.  The problem is the one of
 * Celko, Mraz, Bergmann, Manek, "Parallel CPU- and GPU-based connected
 * component algorithms for event building for hybrid pixel detectors"
 * (arXiv:2412.11809), Section 2: group zero-suppressed hits (x, y, ToA, ToT)
 * into clusters that are maximal (i), spatially 8-connected (ii) and satisfy a
 * temporal condition (iii):
 *   TPC_LOCAL  (iii)(a)  every step of a connecting path has |dToA| <= dt;
 *   TPC_GLOBAL (iii)(b)  every hit but the first has a cluster hit <= dt earlier;
 *   TPC_STATIC (iii)(c)  all ToAs of a cluster lie within dt.
 * A pixel counts as its own neighbour (Section 4.1: "the 8 neighbouring pixels
 * plus the pixel itself"); ToA comparisons are inclusive.  (b) and (c) are
 * evaluated as the time sweep of Algorithm 1 in (ToA, index) order: a hit
 * merges every still-open cluster with a member on one of its 9 pixels;
 * (b) open = last ToA >= toa - dt, (c) open = first ToA >= toa - dt.
 *
 * Conventions for every call:
 *   - All functions return 0 (TPC_OK) or a negative tpc_status; no call
 *     throws, aborts or traps.  tpc_strerror() names a status.
 *   - Hit indices are global stream indices: 0-based positions in the order
 *     of all tpc_push() calls on a context.
 *   - A label is the smallest global index in its cluster (canonical).
 *   - `where` says whether a pointer is host (TPC_HOST) or device
 *     (TPC_DEVICE, memory of the context's CUDA device) memory.
 *   - The caller owns every buffer it passes.  The library owns all device
 *     state it allocates and frees it in tpc_destroy().
 *   - Work is ordered on the context's CUDA stream (TPC_OPT_STREAM).  A
 *     context must not be used from two host threads at once; different
 *     contexts are independent and may run concurrently.
 */
#ifndef TPC_H
#define TPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One hit, 16 bytes, little endian.  ToA in 1.5625 ns ticks. */
typedef struct tpc_hit {
    uint16_t x;         /* column, < width */
    uint16_t y;         /* row, < height */
    uint16_t tot;       /* time over threshold (weight of the centroid) */
    uint16_t reserved;  /* ignored */
    uint64_t toa;       /* time of arrival */
} tpc_hit;

/* One cluster record, 40 bytes. */
typedef struct tpc_cluster {
    uint64_t label;     /* smallest global hit index in the cluster */
    int64_t size;       /* number of hits */
    int64_t sum_tot;    /* sum of ToT, exact */
    uint64_t first_toa; /* smallest ToA */
    float cx, cy;       /* ToT-weighted centroid sum(tot*x)/sum(tot), integer
                           pixel coordinates: both exact integer sums taken to
                           fp32 and divided in fp32 (relative error at most
                           3 * 2^-24); NaN when sum_tot == 0 */
} tpc_cluster;

typedef enum {
    TPC_OK = 0,
    TPC_ERR_ARG = -1,     /* null pointer, bad variant/key/where, sensor too large */
    TPC_ERR_RANGE = -2,   /* a hit with x >= width or y >= height (found on device) */
    TPC_ERR_NOMEM = -3,   /* device or pinned allocation failed */
    TPC_ERR_BUSY = -4,    /* admission refused: the memory budget would be exceeded */
    TPC_ERR_TIMEOUT = -5, /* a bounded device-side wait gave up */
    TPC_ERR_CUDA = -6,    /* a CUDA runtime call failed */
    TPC_ERR_CAP = -7,     /* output buffer too small; *n_out holds the size needed */
    TPC_ERR_SPAN = -8,    /* ToA span of one processing step is >= 2^32 ticks */
    TPC_ERR_LATE = -9,    /* streaming: a hit arrived later than max_disorder allows */
    TPC_ERR_STATE = -10   /* call not valid in the context's current state */
} tpc_status;

typedef enum { TPC_LOCAL = 0, TPC_GLOBAL = 1, TPC_STATIC = 2 } tpc_variant;
typedef enum { TPC_HOST = 0, TPC_DEVICE = 1 } tpc_where;

typedef enum {
    /* Streaming (Algorithm 2's t, Section 3.1's t-ordered streams): the
       largest amount by which a later hit may precede an earlier one.  When
       set (< UINT64_MAX), every tpc_push() clusters the new chunk together
       with the open clusters carried on the device and finalises every
       cluster whose last ToA <= max_toa_seen - max_disorder - dt.  Default
       UINT64_MAX: pushes only buffer, tpc_flush() clusters everything. */
    TPC_OPT_MAX_DISORDER = 1,
    /* Device-memory budget in bytes for this context's working set; a push
       that would exceed it fails with TPC_ERR_BUSY and changes nothing.
       Default 0 = unlimited. */
    TPC_OPT_MEM_BUDGET = 2,
    /* cudaStream_t (cast to uint64_t) on which all work is ordered.
       Default 0 = a stream the context creates. */
    TPC_OPT_STREAM = 3,
    /* At most this many CTAs per SM for the persistent kernels (each kernel's
       grid is one wave: SMs x its occupancy).  0 (default) = as many as fit;
       a smaller value leaves room for other work on the GPU. */
    TPC_OPT_CTAS_PER_SM = 4,
    /* Fault injection on the host, for tests of error handling: value N > 0
       makes the N-th device or pinned allocation this context makes from
       now on fail as an out-of-memory would (the call reports
       TPC_ERR_NOMEM); it fires once, then the option is off.  0 = off.  No
       CUDA call fails and no GPU is faulted: the allocation is not made.
       After any TPC_ERR_NOMEM the context stays usable and the failed call
       may be repeated; the result of the step before is dropped. */
    TPC_OPT_FAIL_ALLOC = 5
} tpc_option;

typedef struct tpc_ctx tpc_ctx;

/* Create a context for one sensor of width x height pixels (width*height <=
   2^20) with time window dt (ticks) and a variant.  Uses the current CUDA
   device.  *out receives the context; on error *out is NULL. */
int tpc_create(uint32_t width, uint32_t height, uint64_t dt, int variant, tpc_ctx **out);

/* Set an option (see tpc_option).  Options may change only while no hits
   are pending (TPC_ERR_STATE otherwise). */
int tpc_set_option(tpc_ctx *ctx, int key, uint64_t value);

/* Append n hits (a chunk) to the stream.  Host hits are copied (through a
   pinned staging buffer) before the call returns.  Device hits are read by
   work queued on the context stream: the caller must keep them unchanged
   until tpc_sync() (or a retrieval call) returns.  In streaming mode the
   chunk is clustered at once; otherwise it is buffered for tpc_flush(). */
int tpc_push(tpc_ctx *ctx, const tpc_hit *hits, size_t n, int where);

/* Cluster everything pending and close every cluster (the end of the
   stream).  Asynchronous for TPC_LOCAL: errors found on the device are
   reported by tpc_sync() and the retrieval calls.  TPC_GLOBAL and
   TPC_STATIC are clustered here too (TPC_GLOBAL waits for the device
   between its merge rounds); streaming (max_disorder) and batching accept
   TPC_LOCAL only. */
int tpc_flush(tpc_ctx *ctx);

/* Wait for the context's queued work; returns the first device-side error
   of the last processing step, if any. */
int tpc_sync(tpc_ctx *ctx);

/* Labels of the hits finalised by the last processing step (the last push
   in streaming mode, or tpc_flush), in increasing global index.  After a
   plain push...push, flush these are all hits.  labels[k] is the label of
   global hit indices[k]; `indices` may be NULL.  Both buffers hold at least
   cap entries and live in `where` memory.  *n_out = number of hits
   finalised; if it exceeds cap, nothing is written and TPC_ERR_CAP is
   returned. */
int tpc_labels(tpc_ctx *ctx, uint64_t *labels, uint64_t *indices, size_t cap,
               size_t *n_out, int where);

/* Queue, without waiting, the copy of the labels of the last one-shot step
   (tpc_flush or tpc_batch_flush of a non-streaming context) into `labels`
   (at least cap entries in `where` memory), on the context stream.  After
   push...push, flush these are the labels of every hit pushed since the
   previous flush, in push order, so their number is known on the host
   without reading the device; *n_out receives it.  The buffer holds the
   labels once tpc_sync() or a later retrieval call on the context has
   returned, and device-side errors of the step are reported there.  Lets a
   caller overlap one step's copies with another context's kernels.
   TPC_ERR_STATE for a streaming result or before the first step;
   TPC_ERR_CAP (nothing queued) if cap < *n_out. */
int tpc_labels_async(tpc_ctx *ctx, uint64_t *labels, size_t cap, size_t *n_out, int where);

/* Bind caller device buffers (memory of the context's device) that every
   following one-shot step of the context (tpc_flush of a non-streaming
   context, any variant, or a tpc_batch_flush it takes part in) writes its
   results into directly: labels[i] for the i-th hit pushed since the
   previous step, records[k] ordered by label, cap entries each, so that no
   retrieval copy is needed (tpc_counts gives the cluster count; tpc_labels
   and tpc_cluster_features still work, copying from these buffers).  A
   step with more hits than cap fails with TPC_ERR_CAP before doing
   anything (the hits stay pending); more clusters than cap is reported as
   TPC_ERR_NOMEM by tpc_sync, as for the context's own buffers.  The caller
   keeps the buffers alive and unread until the step's work is done (after
   tpc_sync or a retrieval call).  labels = records = NULL unbinds.
   TPC_ERR_ARG for host or foreign-device pointers, one NULL of two or cap
   0; TPC_ERR_STATE for a streaming context. */
int tpc_bind_outputs(tpc_ctx *ctx, uint64_t *labels, tpc_cluster *records, size_t cap);

/* Cluster records finalised by the last processing step, ordered by label.
   Same size protocol as tpc_labels. */
int tpc_cluster_features(tpc_ctx *ctx, tpc_cluster *out, size_t cap, size_t *n_out,
                         int where);

/* Cluster the pending hits of n contexts in one batch: every kernel of the
   pipeline runs once over all contexts (persistent CTAs over (context, tile)
   work items), replayed from one CUDA graph.  All contexts must be on the
   same device, non-streaming, with pending hits pushed; results are read
   per context with tpc_labels / tpc_cluster_features.  Work is ordered on the
   first context's stream; every context's stream waits for it. */
int tpc_batch_flush(tpc_ctx **ctxs, int n);

/* Launch choices of a context's processing steps and of the batches it
   leads (tpc_batch_flush uses the first context's).  Results never depend
   on them; only the time does.  The paper sizes its GPU work by hand (at
   least 10,000 hits per thread, Section 4.1); here the work per CTA is a
   tile of 4096 hits and these choices set how the launches fill the GPU. */
typedef struct tpc_tuning {
    uint8_t ctas_sort;    /* CTAs per SM of the tile sort and merge, 0 = as many as fit */
    uint8_t ctas_link;    /* CTAs per SM of the link kernels, 0 = as many as fit */
    uint8_t ctas_acc;     /* CTAs per SM of the feature kernel, 0 = as many as fit */
    uint8_t ctas_out;     /* CTAs per SM of the label and record kernels, 0 = as many as fit */
    uint16_t acc_span;    /* positions per pass of the feature kernel: 512, 1024 or 2048
                             (0 = 1024, the default) */
    uint8_t general_link; /* bit 0: sensors the shared-memory pixel table covers at once,
                             bit 1: sensors it covers in bands, take the general link kernel */
    uint8_t order;        /* batches: 0 = contexts in the given order, 1 = most hits first */
} tpc_tuning;             /* 8 bytes; all zero = the defaults */

/* Set (t, or the defaults if t is NULL) / read a context's launch choices.
   TPC_ERR_ARG for a value outside the ranges above (CTA counts <= 64). */
int tpc_set_tuning(tpc_ctx *ctx, const tpc_tuning *t);
int tpc_get_tuning(tpc_ctx *ctx, tpc_tuning *t);

typedef struct tpc_tune_report {
    tpc_tuning chosen;    /* the choices now set on ctxs[0] */
    uint32_t from_cache;  /* 1: taken from the cache file; nothing was timed */
    uint32_t trials;      /* launch choices timed */
    double untuned_ms;    /* median device time of the batch with the defaults */
    double tuned_ms;      /* with the chosen ones (from the cache: as stored) */
    char key[192];        /* the cache key of this batch */
} tpc_tune_report;

#define TPC_TUNE_FORCE 1  /* time the candidates even if the cache has the key */

/* Autotuner of the batched step: with the same arguments and preconditions
   as tpc_batch_flush (every context has pending hits), look the batch's key
   up in the cache file (GPU name and SM count, each sensor geometry with the
   bucket floor(log2(hits)) of its pending hits, the number of contexts) or,
   if absent (or with TPC_TUNE_FORCE), time the pending batch itself, which
   stays pending: the defaults, then coordinate descent over the fields of
   tpc_tuning, two passes, three timed runs per candidate, a change kept if
   its median improves by more than 1 %.  Sets the choice on ctxs[0] and
   appends it to the cache file (cache_path NULL: no cache).  Work is
   ordered on ctxs[0]'s stream and waited for. */
int tpc_tune_batch(tpc_ctx **ctxs, int n, const char *cache_path, int flags, tpc_tune_report *rep);

/* The tuner's cache file, host only (no CUDA call): one line per entry,
   "key<TAB>ctas_sort ctas_link ctas_acc ctas_out acc_span general_link
   order<TAB>ms", the last line with a key winning; lines that do not parse
   are skipped.  lookup: TPC_ERR_STATE if the file or the key is absent;
   *ms (may be NULL) receives the stored time.  store appends a line;
   TPC_ERR_ARG for an invalid tuning, an empty key or one holding a tab or
   newline, or a file that cannot be written. */
int tpc_tune_cache_lookup(const char *path, const char *key, tpc_tuning *out, double *ms);
int tpc_tune_cache_store(const char *path, const char *key, const tpc_tuning *t, double ms);

/* Number of hits finalised, clusters finalised and hits carried (open) by
   the last processing step.  Waits for the context's work. */
int tpc_counts(tpc_ctx *ctx, size_t *n_hits, size_t *n_clusters, size_t *n_open);

/* Diagnostics: tpc_flush() with the kernels launched one by one (no CUDA
   graph) and an event after each; names[k] (static strings) and ms[k]
   receive each kernel's device time in launch order, *n_out the number of
   kernels in one processing step.  Waits for completion.  TPC_ERR_CAP if
   cap < *n_out (the first cap entries are written); TPC_ERR_STATE for a
   streaming context.  Not part of the paper: per-kernel timing in the
   spirit of its wall-clock measurements (Section 4, benchmark set-up). */
int tpc_profile_flush(tpc_ctx *ctx, const char **names, float *ms, int cap, int *n_out);

/* Diagnostics: the union-find forest of the last processing step of this
   context (tpc_flush or a streaming push; not a batch), the structure of
   Section 4.1.  Hits are numbered by position in the step's (ToA, input)
   order; parent[p] is the position of p's parent (p itself for a root) and
   input_pos[p] the input index of the hit at position p (0-based within the
   step: the carried open hits first when streaming, then the new chunk).
   Both host arrays hold at least cap entries; *n_out = hits in the step;
   TPC_ERR_CAP if that exceeds cap; TPC_ERR_STATE after a batch or before
   any step.  Waits for the context's work.  Every parent precedes its child
   in (ToA, input) order, so toa(parent(h)) <= toa(h), the time invariant of
   Section 4.1, and each root is its cluster's earliest hit. */
int tpc_forest(tpc_ctx *ctx, uint32_t *parent, uint32_t *input_pos, size_t cap, size_t *n_out);

/* Diagnostics of the context's last TPC_GLOBAL or TPC_STATIC flush (zero
   otherwise): (b) rounds of merges on the device, of which full passes over
   every hit (the first, and any after the list of open edges overflowed),
   exact recomputations of the groups' last ToA, and the edges the first
   round left open (capped at the list's size); (c) components longer
   than a warp's shared-memory staging (512 hits), swept by one warp
   through a sliding window of 512 hits; of those, the ones swept again by a
   whole CTA (more hits within dt than that window holds), and of those the
   ones too long (over 8192 hits) to stage in shared memory, swept from
   global memory.  Waits for the context's work. */
typedef struct tpc_variant_stats {
    uint32_t rounds, full_rounds, exact_checks;
    uint32_t windowed, window_fallbacks, global_sweeps;
    uint32_t first_open_edges;
} tpc_variant_stats;
int tpc_variant_stats_get(tpc_ctx *ctx, tpc_variant_stats *out);

/* Bytes of device memory the context currently holds. */
int tpc_device_bytes(tpc_ctx *ctx, size_t *bytes);

/* Checkpoint of a streaming context (TPC_OPT_MAX_DISORDER set): everything
   the next push depends on — the open hits carried on the device with their
   global indices, the largest ToA seen, the watermark and the global index
   of the next hit.  The paper's pipeline hands buffers over between
   processing steps (Algorithm 2 and Algorithm 3, steps 1 and 9); a snapshot
   taken between two pushes lets the stream continue in another context,
   process or machine with results identical to an uninterrupted stream.
   Byte layout (host order, little endian on every supported host):
   tpc_snapshot_header, then n_carry tpc_hit records, then n_carry uint64
   global indices, in the order the device keeps them. */
#define TPC_SNAPSHOT_MAGIC 0x53435054u   /* "TPCS" */
#define TPC_SNAPSHOT_VERSION 1u
typedef struct tpc_snapshot_header {
    uint32_t magic;         /* TPC_SNAPSHOT_MAGIC */
    uint32_t version;       /* TPC_SNAPSHOT_VERSION */
    uint32_t width, height; /* sensor of the context */
    uint64_t dt;            /* time window of the context */
    uint64_t max_disorder;  /* TPC_OPT_MAX_DISORDER of the context */
    uint64_t pushed;        /* global index of the next hit to be pushed */
    uint64_t seen_max;      /* largest ToA pushed so far (valid if has_seen) */
    uint64_t watermark;     /* clusters whose last ToA <= watermark are final */
    uint32_t has_seen;      /* 1 once any hit has been pushed */
    uint32_t n_carry;       /* open hits carried into the next push */
} tpc_snapshot_header;      /* 64 bytes */

/* Write the snapshot of a streaming context into host memory `buf` (cap
   bytes).  Waits for the context's queued work.  *n_out = bytes the
   snapshot takes (64 + 24 * n_carry); if that exceeds cap (buf may then be
   NULL), nothing is written and TPC_ERR_CAP is returned.  TPC_ERR_STATE for
   a context not in streaming mode; a device-side error of the last push
   (for example TPC_ERR_LATE) is returned instead of a snapshot.  The
   context is left unchanged and may keep streaming. */
int tpc_snapshot(tpc_ctx *ctx, void *buf, size_t cap, size_t *n_out);

/* Load a snapshot (host memory, n bytes) into a TPC_LOCAL context created
   with the same width, height and dt that holds no open hits and no
   pending hits (new, or after tpc_flush).  Sets TPC_OPT_MAX_DISORDER to
   the snapshot's and makes the context continue that stream: the next
   push clusters its hits with the restored open hits, and global indices
   continue from the header's `pushed`.  Results of earlier steps are
   dropped (retrieval calls report nothing until the next push or flush).
   TPC_ERR_ARG for a malformed snapshot (magic, version, size) or a sensor
   or dt mismatch; TPC_ERR_STATE if the context is busy; the context is
   unchanged on any error but TPC_ERR_CUDA and TPC_ERR_NOMEM. */
int tpc_restore(tpc_ctx *ctx, const void *buf, size_t n);

/* Hit buffer filling (Algorithm 2, Section 4.1): host-side ingestion that
   cuts a t-ordered hit stream (Section 3.1: toa_i < toa_j + t for every
   earlier hit i and later hit j) into buffers for the device.  A buffer
   takes hits freely while it holds fewer than b - b_t; then only hits
   earlier than toa_max + t_closing (and while it holds fewer than b); other
   hits go to the next buffer.  A hit later than toa_max + t + t_closing
   sends the buffer, and the next buffer becomes the current one.  toa_max
   is the largest ToA of the hits taken while a buffer had room, one value
   for the whole stream.  On a t-ordered stream whose closing windows fit in
   b_t, and whose buffers take their first b - b_t hits over more than t
   ticks, buffer k holds exactly the hits earlier than its cut toa_max +
   t_closing, so clusters are split only across a cut, within dt of it; in
   every case the buffers, taken in the order they are sent, form a
   t-ordered stream again.  Buffers keep arrival order inside; the next
   buffer has no size cap, so a buffer can start with more than b hits when
   b_t is too small for the stream.  Host memory only (no CUDA call); a
   filler must not be used from two host threads at once. */
typedef struct tpc_filler tpc_filler;

/* b > b_t >= 0 (TPC_ERR_ARG otherwise); t, t_closing in ToA ticks. */
int tpc_filler_create(uint64_t b, uint64_t b_t, uint64_t t, uint64_t t_closing,
                      tpc_filler **out);

/* storeHit for each of the n host hits, in order.  Hits are numbered in
   arrival order over all calls (0-based).  TPC_ERR_STATE after
   tpc_filler_finish(). */
int tpc_filler_store(tpc_filler *f, const tpc_hit *hits, size_t n);

/* End of the stream: send the current buffer, then a non-empty next
   buffer (their cut is UINT64_MAX). */
int tpc_filler_finish(tpc_filler *f);

/* Number of sent buffers waiting, and the size in hits of the oldest (0 if
   none); either pointer may be NULL. */
int tpc_filler_ready(tpc_filler *f, size_t *n_buffers, size_t *front_hits);

/* Take the oldest sent buffer: its hits into `hits` (host, cap records),
   their arrival numbers into `indices` (host, cap entries, may be NULL) and
   its cut into *cut (may be NULL).  *n_out = its size; TPC_ERR_CAP (nothing
   taken) if that exceeds cap; TPC_ERR_STATE if no buffer is waiting. */
int tpc_filler_take(tpc_filler *f, tpc_hit *hits, uint64_t *indices, size_t cap,
                    size_t *n_out, uint64_t *cut);

/* sendToDevice: push the oldest sent buffer into a context (tpc_push of
   host hits, so the same ordering and errors) and take it; arrival numbers,
   size and cut as tpc_filler_take.  On an error of tpc_push the buffer
   stays waiting. */
int tpc_filler_send(tpc_filler *f, tpc_ctx *ctx, uint64_t *indices, size_t cap,
                    size_t *n_out, uint64_t *cut);

void tpc_filler_destroy(tpc_filler *f);

/* Largest batch tpc_cluster_static() accepts. */
#define TPC_STATIC_MAX_HITS 65536

/* Error bits tpc_cluster_static() writes to counts[1] (0 = none). */
#define TPC_STATIC_E_RANGE 1u   /* a hit outside the sensor (its pixel is clamped) */
#define TPC_STATIC_E_SPAN 2u    /* the batch's ToA span is 2^32 ticks or more */
#define TPC_STATIC_E_CAP 16u    /* more clusters than record_cap (> 0): records truncated */

/* One-shot clustering (variant TPC_LOCAL) of at most TPC_STATIC_MAX_HITS
   hits that allocates nothing.  The paper has no counterpart; it is an
   addition of this library, for callers that cannot call cudaMalloc:
   real-time readout loops that must not block (cudaMalloc can synchronise
   the device), and code under a fixed memory plan that may only use
   buffers it was given.
     hits        device pointer, n records (same layout as tpc_push)
     labels      device pointer, n entries: labels[i] = smallest index i'
                 in hit i's cluster (indices 0..n-1 of this call)
     records     device pointer, record_cap cluster records ordered by label
                 (as tpc_cluster_features); may be NULL if record_cap == 0
     counts      device pointer, 2 entries written by the call:
                 counts[0] = number of clusters, counts[1] = TPC_STATIC_E_*
                 bits (0 = none).  With record_cap == 0 (labels only) the
                 cap bit is never set; with 0 < record_cap < counts[0] it is,
                 and the first record_cap records are written.
     stream      cudaStream_t (as void *) the work is queued on; 0 = legacy
   Asynchronous: returns after queueing.  TPC_ERR_ARG for n >
   TPC_STATIC_MAX_HITS, null pointers or a sensor larger than tpc_create
   allows.  Working memory is one fixed device array of the library
   (about 4.5 MB per GPU that loads it, held until exit), shared by every
   call and keeping the last call's contents: calls whose work overlaps on
   the GPU race on it, so order them on one stream.  The first call on a
   device does set-up (looks up that array's device address with
   cudaGetSymbolAddress and sets kernel attributes); make that first call
   before any stream capture. */
int tpc_cluster_static(const tpc_hit *hits, size_t n, uint32_t width, uint32_t height,
                       uint64_t dt, uint64_t *labels, tpc_cluster *records, size_t record_cap,
                       uint64_t *counts, void *stream);

/* Serving loop: detector streams clustered on one GPU under one device-memory
   budget.  The paper keeps every buffer "in use until retrieved" and hands a
   thread the next buffer only when one is free (Algorithm 2; Algorithm 3
   steps 1 and 9, Section 4.1); here a submitted chunk waits in one queue, in
   submission order, until its stream is idle and the device memory the
   stream will hold while the chunk runs fits in the budget next to what the
   other streams hold.  Admitted chunks run at once on their stream's own CUDA
   stream (chunks of different streams overlap on the GPU), each through a
   streaming TPC_LOCAL context (open clusters carried on the device,
   finalised by the ToA watermark, as TPC_OPT_MAX_DISORDER), and their
   results are copied into the caller's host buffers.  When the chunk at the
   head of the queue does not fit, the work arrays of idle streams are freed
   (stream-ordered, without synchronising the device) before it waits;
   later chunks do not overtake it.  Each stream has a host worker thread. */
typedef struct tpc_server tpc_server;

typedef struct tpc_server_result {
    uint64_t tag;        /* the tag the chunk was submitted with */
    int32_t stream;      /* its stream */
    int32_t status;      /* TPC_OK, or the chunk's error (TPC_ERR_BUSY: it can
                            never fit in the budget; TPC_ERR_CAP: cap too small,
                            n_hits / n_clusters give the sizes needed and the
                            results are lost; a device error of the step) */
    uint64_t n_hits;     /* hits finalised by the chunk: labels[k] is the label
                            of global hit indices[k], k < n_hits, increasing */
    uint64_t n_clusters; /* cluster records finalised, records[0..n_clusters) */
    double queue_ms;     /* submission to admission */
    double latency_ms;   /* submission to results in the caller's buffers */
} tpc_server_result;

typedef struct tpc_server_stats {
    uint64_t budget;     /* bytes */
    uint64_t in_use;     /* bytes held by idle streams plus reserved by running chunks */
    uint64_t peak;       /* largest in_use so far */
    uint64_t streams, submitted, admitted, completed, failed, rejected;
    uint64_t queued;     /* chunks waiting now */
    uint64_t in_flight;  /* chunks running now */
    uint64_t waits;      /* chunks that waited at the head of the queue for memory */
    uint64_t releases;   /* idle streams whose work arrays were freed to make room */
} tpc_server_stats;

/* A server for the current CUDA device with a budget in bytes (> 0). */
int tpc_server_create(uint64_t mem_budget, tpc_server **out);

/* Add a detector stream: sensor, time window and the stream's disorder
   bound t (Section 3.1; 0 < max_disorder < UINT64_MAX).  *id receives its
   number (0, 1, ...). */
int tpc_server_add_stream(tpc_server *s, uint32_t width, uint32_t height, uint64_t dt,
                          uint64_t max_disorder, int *id);

/* Queue a chunk of n host hits of stream id (copied to the device when it is
   admitted), or, with end_of_stream != 0 and n == 0, the end of the stream
   (closes every open cluster; no chunk may follow).  The caller keeps
   `hits` unchanged and the host buffers labels, indices (may be NULL) and
   records (cap entries each) alive until tpc_server_wait() returns this
   chunk's result; cap must cover the hits the chunk finalises (at most its
   own hits plus the stream's open hits).  Chunks of one stream run in
   submission order.  Never blocks on the device. */
int tpc_server_submit(tpc_server *s, int id, const tpc_hit *hits, size_t n, uint64_t *labels,
                      uint64_t *indices, tpc_cluster *records, size_t cap, uint64_t tag,
                      int end_of_stream);

/* Wait up to timeout_us microseconds (< 0: no limit) for the next completed
   chunk, in completion order.  TPC_ERR_TIMEOUT if none completed in time;
   TPC_ERR_STATE if nothing is queued, running or waiting to be returned. */
int tpc_server_wait(tpc_server *s, tpc_server_result *res, int64_t timeout_us);

/* Counters and memory figures of the server. */
int tpc_server_stats_get(tpc_server *s, tpc_server_stats *out);

/* Drop queued chunks, let running ones finish, end the worker threads and
   destroy the streams' contexts. */
void tpc_server_destroy(tpc_server *s);

const char *tpc_strerror(int status);
void tpc_destroy(tpc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* TPC_H */
