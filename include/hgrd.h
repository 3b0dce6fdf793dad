/*
 * hgrd.h — C ABI of libhgrd.so, the B300 (sm_103a) exhaustive host-guided
 * GPU data-race check.
 *
 * Model (the paper's race definition, made concrete by the host binding):
 *   A kernel descriptor lists a kernel's memory accesses as quasi-affine
 *   index expressions over threadIdx, blockIdx, loop counters and kernel
 *   parameters, each with guards, a read/write/atomic flag, an access width
 *   and a barrier-interval id.  A binding supplies every parameter and the
 *   launch dimensions, as the launching host code does (Sec. 4 and Sec. 5.1,
 *   host classes (1)-(5)).  Two instances race when they come from different
 *   threads, touch a common byte granule, at least one writes, they are not
 *   both atomic with enough scope, and they are unordered: in shared memory
 *   only inside one block and one barrier interval, in global memory also
 *   across blocks in any interval, because block barriers do not order blocks
 *   (Sec. 2 "Data races on GPUs", Sec. 6.1, Table 2, Appendix A).
 *
 * Pipeline behind hgrd_check (all on one GPU, stream ordered): instance
 * expansion into 64-bit keys, a stable onesweep LSD radix sort on the key's
 * (array, granule, interval) bits, a segmented conflict scan over runs of
 * equal (array, granule), and witness compaction + canonicalisation.
 *
 * Conventions for every entry point:
 *   * Return value: HGRD_OK (0), HGRD_ETRUNCATED (1: more witnesses than the
 *     caller's capacity; the verdict's counts stay exact and the first `cap`
 *     canonical witnesses are written), or a negative error.  No entry point
 *     aborts or exits; hgrd_last_error() returns a thread-local message about
 *     the last failure on the calling thread.
 *   * Ownership: descriptors are created and freed by the library.  Device
 *     workspace and CUDA streams are owned by the caller (the Python binding
 *     allocates them with PyTorch).  Host output arrays are owned by the caller.
 *   * Pointers named d_* are device pointers; all others are host pointers.
 *   * The library keeps no device state between calls.
 */
#ifndef HGRD_H
#define HGRD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HGRD_OK = 0,
  HGRD_ETRUNCATED = 1,
  HGRD_EINVAL = -1,          /* null pointer, bad option, descriptor not bound */
  HGRD_EPARSE = -2,          /* descriptor text malformed or not quasi-affine */
  HGRD_EBIND = -3,           /* parameter count, launch dims, divisor <= 0, negative size */
  HGRD_EHOSTCONSTRAINT = -4, /* a host `assert` of the descriptor is false for the binding */
  HGRD_EOVERFLOW = -5,       /* an index expression can leave int64, or the key exceeds 64 bits */
  HGRD_ENOMEM = -6,          /* workspace smaller than hgrd_workspace_size, or raw witness cap hit */
  HGRD_EDEVICE = -7,         /* a CUDA call failed */
  HGRD_ETIMEOUT = -8,        /* a bounded device-side wait gave up */
  HGRD_EUNSUPPORTED = -9     /* descriptor exceeds a fixed limit of this build */
};

enum { HGRD_SPACE_GLOBAL = 0, HGRD_SPACE_SHARED = 1 };
/* kind_mask bits: race type of a witness (Sec. 2, Table 2) */
enum { HGRD_INTER_BLOCK = 1, HGRD_INTRA_BLOCK = 2, HGRD_INTRA_WARP = 4 };

typedef struct hgrd_desc hgrd_desc; /* opaque, library owned */

/* Host binding (Sec. 5.1, classes (1)-(5)): launch dims and parameter values
 * in the descriptor's `param` order. */
typedef struct {
  int32_t grid[3], block[3];
  uint32_t nparams;
  const int64_t* params;
} hgrd_binding;

/* One racy (access pair, location) — the paper's report unit (Sec. 5, Sec. 6
 * component 5): array, byte address of the granule (the in-block offset for
 * shared memory, merged over blocks), the two access ids (acc_lo <= acc_hi,
 * descriptor order), and the race types seen there. */
typedef struct {
  uint8_t space, array, acc_lo, acc_hi, kind_mask, pad[3];
  uint64_t byte_addr;
} hgrd_witness;

/* One concrete access instance: linear block, linear thread (tx + ty*bdx +
 * tz*bdx*bdy), loop counters (outermost first), access id. */
typedef struct {
  uint32_t lin_block, lin_thread;
  uint32_t iter[4];
  uint8_t access, pad[3];
} hgrd_inst;

/* Verdict.  Witnesses are ordered by (space, array, byte_addr, acc_lo,
 * acc_hi); min_w is the first.  min_x/min_y is the lexicographically smallest
 * racing instance pair realising min_w (x of acc_lo, y of acc_hi, keys
 * (lin_block, lin_thread, iter...)), valid when pair_found is 1.
 * n_instances counts every (block, thread, loop vector, access) tuple before
 * guards; n_keys the granule keys of live in-bounds instances; n_oob the live
 * instances outside their array. */
typedef struct {
  int32_t racy, pair_found;
  uint64_t n_witness, n_by_kind[3], n_instances, n_keys, n_oob;
  hgrd_witness min_w;
  hgrd_inst min_x, min_y;
  /* racy access pairs, the paper's report unit (Sec. 5, Sec. 6 component 5):
   * bit b of pair_kind[k][a] is set when accesses a and b race with kind
   * 1 << k somewhere (symmetric in a, b) */
  uint32_t pair_kind[3][32];
} hgrd_verdict;

/* Options.  Zero-initialised means defaults. */
typedef struct {
  uint64_t max_raw_witness; /* device buffer for per-run witnesses before merging;
                               0 = twice the key bound, between 1<<12 and 1<<24 */
  uint32_t pair_cap;        /* instances gathered to find min_x/min_y; 0 = min(key bound, 1<<20) */
  uint32_t flags;           /* HGRD_NO_PAIR: skip the canonical instance pair;
                               HGRD_PROFILE: time every pipeline stage with CUDA events;
                               HGRD_STOP_FIRST: stop the exact scan once one race is confirmed
                               (the verdict is racy/clean exactly; witnesses and counts are then
                               a subset, each witness a real race);
                               HGRD_NO_SPLIT: sort the keys of shared arrays with the global ones
                               instead of checking them in per-block bins (same result; for
                               comparison and testing);
                               HGRD_JIT / HGRD_NO_JIT: always / never expand with kernels
                               specialised to the program's structure, compiled at run time
                               (default: when hgrd_jit_compile or an HGRD_JIT check already
                               compiled them for this binding); same result;
                               HGRD_NO_SMALL: never run a small binding (at most 4096 keys, 1024
                               simulated warps) whole in one CTA; by default it does, and falls
                               back to the device-wide pipeline when it keeps too few witnesses;
                               HGRD_NO_CELL_FILTER / HGRD_CELL_FILTER: never / always (when its
                               table fits: at most 2^23 cells) sort only the keys of locations
                               that two threads touch with a writer among them, found with a
                               per-location table the count pass fills (default: when at least
                               2^16 keys may be sorted); same result;
                               HGRD_GRAPH: run the check as one CUDA graph launch, the graph
                               captured by the first such check of this binding with this
                               workspace, these options and this device, and replayed by the
                               later ones (same result; the graph's kernels read the program
                               from the graph's own device copy, filled from a pinned copy
                               taken at capture: once by hgrd_check_enqueue, before every
                               replay by hgrd_check; ignored with HGRD_PROFILE; a rebind
                               makes a new binding);
                               HGRD_ALL_KEYS: write and sort the keys of every live access,
                               also of those the pair rule shows can race with nothing, in one
                               global sort on the interpreted kernels (implies HGRD_NO_SPLIT,
                               HGRD_NO_JIT, HGRD_NO_SMALL); same result: a measurement mode that
                               puts every key of the check through the sort and the scan;
                               HGRD_SCAN_BALLOT: run the first phase of the conflict scan as
                               32-key warp steps (one key per lane, ballots per step) instead of
                               rows of 16 keys per lane staged by tensor copies; same result */
  uint32_t only_accesses;   /* nonzero: check only the accesses whose bit is set (a restricted
                               check: every witness is a real race of the full kernel, but a
                               clean result says nothing about the other accesses) */
  uint32_t max_shared_keys; /* block-local mode: room for keys of shared-memory bins that can
                               race (a writer and two threads); 0 = all kept shared keys up to
                               2^24, a sixteenth of them beyond.  HGRD_ENOMEM names the count
                               when short */
} hgrd_check_opts;
enum {
  HGRD_NO_PAIR = 1,
  HGRD_PROFILE = 2,
  HGRD_STOP_FIRST = 4,
  HGRD_NO_SPLIT = 8,
  HGRD_JIT = 16,
  HGRD_NO_JIT = 32,
  HGRD_NO_SMALL = 64,
  HGRD_GRAPH = 128,
  HGRD_NO_CELL_FILTER = 256,
  HGRD_CELL_FILTER = 512,
  HGRD_ALL_KEYS = 1024,
  HGRD_SCAN_BALLOT = 2048
};

/* One timed pipeline stage (HGRD_PROFILE): events recorded on the check's
 * stream around the stage's kernels. */
typedef struct {
  char name[24];
  float ms;
} hgrd_stage_time;

/* Per-call counters of the last hgrd_check* on the calling thread. */
typedef struct {
  uint64_t kernel_launches; /* kernels of this library enqueued by the call */
  uint64_t n_candidates;    /* runs the exact conflict scan examined */
  uint64_t n_raw_witness;   /* per-run witnesses before the cross-block merge */
  uint32_t sort_passes;     /* radix passes over the instance keys */
  uint32_t int64_path;      /* 1 when index arithmetic needed 64-bit integers */
  uint64_t h2d_bytes;       /* host->device bytes the call copied (the compiled program) */
  uint64_t d2h_bytes;       /* device->host bytes the call copied (counters, witnesses, pair search) */
  uint64_t n_sorted_keys;   /* keys that went through the radix sort */
  uint64_t n_binned_keys;   /* shared-array keys written into candidate bins (block-local mode) */
  uint32_t shared_bins;     /* 1 when the shared-array keys were checked in per-block bins */
  uint32_t jit;             /* 1 when the expansion ran specialised kernels (HGRD_JIT) */
  uint64_t eval_ops;        /* integer operations of the count pass's evaluation (guards,
                               index, bound tests, interval, the ops they read; a term is one
                               multiply-add, a division by a constant 3, a remainder 5); on
                               specialised kernels loop-invariant and loop-guarded accesses
                               count once per thread */
  uint32_t small;           /* 1 when the check ran whole in one CTA */
  uint32_t cell_filter;     /* 1 when only keys of cells with a writer and two threads were sorted */
  uint64_t n_written_keys;  /* global-array keys the expansion wrote (the first sort pass reads
                               them all; with the cell filter it keeps n_sorted_keys of them) */
  uint64_t cuda_objects_created; /* process-wide, not per call: CUDA objects and buffers this
                               library has created since it was loaded (streams, events,
                               instantiated graphs, pinned host buffers, loaded modules) */
} hgrd_stats;

/* Parse a descriptor (format: kernel/param/loop/array/let/access/assert lines,
 * documented in the project's workload module).  A descriptor states what the
 * paper's front end extracts from the kernel code (Sec. 6.2, Table 1): per
 * access its address expression over thread ids, block ids, loop counters and
 * parameters, its guards, its read/write/atomic kind and width, and the block-
 * and warp-barrier intervals it falls in (Sec. 6.1, Sec. 5.2); `param` and
 * `assert` lines carry the host code's facts (Sec. 4).  Static checks: names, at
 * most 32 accesses, 32 arrays, 4 loops, quasi-affine expressions (a product
 * needs one uniform factor, divisors are uniform), intervals free of thread
 * and block ids, uniform loop bounds, sizes and asserts.  `text` need not be
 * NUL terminated.  On success *out owns a new descriptor. */
int hgrd_load_desc(const char* text, size_t len, hgrd_desc** out);

/* Bind host values (Sec. 5.1, classes (1)-(5); Sec. 6.3): checks the
 * parameter count, 1 <= dims, <= 1024 threads per block, every divisor > 0,
 * array sizes >= 0 and every `assert` (HGRD_EHOSTCONSTRAINT when one fails),
 * folds the values into per-access coefficient tables, bounds every
 * expression over the instance box (HGRD_EOVERFLOW when int64 can
 * overflow) and plans the key layout.  Acquire-release guards (`sync`
 * fields, Sec. 6.5 with the scopes of Appendix A) are decided here, per pair
 * of guarded accesses on one lock array, when both guard elements are
 * constant or each access is guarded at its own index with equal widths;
 * pairs whose elements can differ between instances (constant, affine in
 * thread and block ids, or the access's own element) are left to the exact
 * scan, instance pair by instance pair; guard elements with a loop counter,
 * or with a division or remainder other than the access's own index, are
 * HGRD_EUNSUPPORTED.  Rebinding replaces the old binding. */
int hgrd_bind_host_params(hgrd_desc* d, const hgrd_binding* b);

/* Device workspace bytes hgrd_check needs for the bound descriptor: the
 * instance keys, their sorted copy and the witness buffers of the exhaustive
 * decision that stands in for the paper's constraint solve (Sec. 6.4).  The
 * workspace must be 256-byte aligned. */
int hgrd_workspace_size(const hgrd_desc* d, const hgrd_check_opts* o, size_t* bytes);

/* Exhaustive check of the bound descriptor on `cuda_stream` (a cudaStream_t,
 * NULL = legacy default stream).  Decides the paper's race (Sec. 2: two
 * threads, an overlapping address, at least one write, not both atomic,
 * unordered by barriers; shared memory within a block, global memory across
 * the grid) for the bound host values, with the trivially race-free pairs of
 * Sec. 6.1 and Table 2's constraints for the three race types (inter-block,
 * intra-block, intra-warp), and reports racy access pairs with their types
 * (Sec. 5) plus per-location witnesses.  Synchronous on return: writes up to `cap`
 * canonical witnesses to host_out (may be NULL when cap is 0) and the verdict
 * to *v.  The workspace contents are scratch. */
int hgrd_check(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, void* cuda_stream,
               hgrd_witness* host_out, uint64_t cap, hgrd_verdict* v);

/* Same pipeline, enqueue only: no host synchronisation and no host copies.
 * The verdict (without the instance pair) and the canonical witnesses stay in
 * the workspace; hgrd_check_collect reads them after the stream reaches
 * this point.  Used to time the device path alone. */
int hgrd_check_enqueue(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, void* cuda_stream);
int hgrd_check_collect(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, void* cuda_stream,
                       hgrd_witness* host_out, uint64_t cap, hgrd_verdict* v);

/* Radix-sort autotuner.  The onesweep pass comes in several shapes: the
 * early-count kernels (shapes 0-6: 256 threads x 32 or 28 keys, 384 x 16;
 * warp ranking by shared atomic-OR peer masks, the match instruction, or per
 * warp by its digit diversity; shape 0 is the default) and the earlier ones
 * (shapes 7-19: 256x16, 256x12, 512x8, 384x12, 256x24, 128x16 with several
 * rankings).  hgrd_sort_tune times one pass of each on up to 2^25 random keys
 * in the given device workspace (about 17.4 bytes per key), keeps the fastest
 * for the current device and writes per-shape times (ms) to ms[0 .. cap).
 * hgrd_sort_variant selects a shape (set >= 0) or queries it (set < 0). */
int hgrd_sort_tune(void* d_ws, size_t ws_bytes, void* cuda_stream, int* best, float* ms, int cap);
int hgrd_sort_variant(int set, int* current, int* count);
/* The shape of one pass of the key sort (pass 0 = the lowest digit) on the
 * current device: set >= 0 selects a shape for that pass, -1 returns it to
 * the device's shape, below -1 only queries; *current (may be NULL) = the
 * pass's shape, -1 when it follows the device's.  Lets a tuner pick a shape
 * per pass on the check's own keys (digit diversity differs by pass). */
int hgrd_sort_pass_variant(int pass, int set, int* current);

/* Counters of the last check on this thread. */
int hgrd_last_stats(hgrd_stats* s);

/* Stage times of the last check enqueued with HGRD_PROFILE on this thread;
 * waits for the stream to reach the last stage.  Writes up to `cap` entries
 * and the number of stages to *n. */
int hgrd_last_profile(hgrd_stage_time* out, uint32_t cap, uint32_t* n);

/* ---- Batched check of many (kernel, binding) items ------------------------
 * The host-code classes of Sec. 4 (a host loop bounding a parameter, class
 * (4); several launch sites of one kernel) give many bound descriptors to
 * check.  A batch runs them together: items whose keys fit on chip go to one
 * persistent, work-queued kernel (a CTA checks a whole item in shared memory,
 * largest items first); the others run the device-wide pipeline, spread over
 * streams longest-first.  Verdicts are per item and exact (the same as
 * hgrd_check on the item); only the first `witness_cap` canonical witnesses
 * of each item are kept.  Items must stay alive and bound as they were at
 * hgrd_batch_create until hgrd_batch_free. */
typedef struct hgrd_batch hgrd_batch; /* opaque, library owned */
typedef struct {
  uint32_t small_keys;  /* items with at most this many keys run on chip (0 = 4096, the maximum) */
  uint32_t streams;     /* streams: one for the on-chip kernel plus large-item streams (0 = 4, 2..16) */
  uint32_t witness_cap; /* canonical witnesses kept per item (0 = 64) */
  uint32_t flags;       /* HGRD_BATCH_GRAPH: capture the whole batch into a CUDA graph on the first
                           run and replay it on later runs with the same workspace and stream;
                           HGRD_BATCH_JIT: at creation, compile specialised expansion kernels
                           (hgrd_jit_compile) for the items too large for the on-chip kernel,
                           once per program structure (a sweep of one kernel shares one) */
} hgrd_batch_opts;
enum { HGRD_BATCH_GRAPH = 1, HGRD_BATCH_JIT = 2 };
typedef struct {
  int32_t status;   /* HGRD_OK, or HGRD_ENOMEM (a witness buffer overflowed: rerun with hgrd_check) */
  int32_t racy, small, n_copied;
  uint64_t n_witness, n_by_kind[3], n_instances, n_keys, n_oob;
  uint32_t pair_kind[3][32]; /* racy access pairs, as in hgrd_verdict */
} hgrd_item_verdict;

int hgrd_batch_create(const hgrd_desc* const* items, uint32_t n, const hgrd_batch_opts* o, hgrd_batch** out);
int hgrd_batch_workspace_size(const hgrd_batch* b, size_t* bytes);
/* Enqueue the whole batch on `cuda_stream` (no host synchronisation). */
int hgrd_batch_run(hgrd_batch* b, void* d_ws, size_t ws_bytes, void* cuda_stream);
/* Wait for the stream and read every item's verdict (v[n]) and its first
 * min(wcap, witness_cap) witnesses (w[n * wcap], item i at w + i * wcap). */
int hgrd_batch_collect(hgrd_batch* b, void* d_ws, size_t ws_bytes, void* cuda_stream, hgrd_item_verdict* v,
                       hgrd_witness* w, uint32_t wcap);
/* Autotuner: times the batch under each (small-item threshold, stream count)
 * in {0, 1024, 4096} x {2, 4, 8, 16}, keeps the fastest for later runs and
 * reports it in *chosen (may be NULL). */
int hgrd_batch_tune(hgrd_batch* b, void* d_ws, size_t ws_bytes, void* cuda_stream, hgrd_batch_opts* chosen);
void hgrd_batch_free(hgrd_batch* b);

/* Ranked batch (the learned ranker over a whole batch; the paper has no
 * learned part).  hgrd_batch_rank_prepare lists every item's eligible access
 * pairs with their 96 features (as hgrd_pair_features; static per binding,
 * computed once on the host).  hgrd_batch_check_ranked then, on the stream:
 *   1. scores every pair of every item in one inference (hgrd_mlp_predict)
 *      and takes each item's top-k pairs on the device (ties to the lower
 *      pair index); an item with at most k eligible pairs takes them all,
 *      one whose best logit is below min_score is not ranked;
 *   2. runs the batch once, each ranked large item restricted to the
 *      accesses of its top pairs (small items run whole on chip);
 *   3. runs the whole check of every ranked item that stage 2 found clean,
 *      unless its checked accesses covered every eligible pair.
 * Verdicts (racy) are exact for every item.  An item decided racy by its
 * restricted check reports the races found there (each a race of the item,
 * Sec. 6.1: races are pairwise), not its full witness set.  stage[n] (may be
 * NULL): 0 whole check in the first run, 1 race found by the restricted
 * check, 2 whole check in the second run, 3 clean on a restricted check
 * covering every eligible pair.  Features are uploaded into the workspace on
 * the first call with it.  Synchronous on return (two host round trips). */
typedef struct {
  uint32_t n_pairs, ranked, confirmed, second; /* pairs scored, items ranked, races confirmed, second-run items */
  float ms_score, ms_stage1, ms_stage2;        /* host wall time of each part */
  float pad;
} hgrd_batch_rank_info;
int hgrd_batch_rank_prepare(hgrd_batch* b);
int hgrd_batch_ranked_workspace_size(const hgrd_batch* b, size_t* bytes);
int hgrd_batch_check_ranked(hgrd_batch* b, const void* d_model, uint32_t topk, float min_score, void* d_ws,
                            size_t ws_bytes, void* cuda_stream, hgrd_item_verdict* v, hgrd_witness* w, uint32_t wcap,
                            uint8_t* stage, hgrd_batch_rank_info* info);

/* ---- The learned ranker (an AI-systems addition; the paper has no learned part)
 * An MLP 96 -> 256 -> 256 -> 1 (ReLU) scores access pairs of a bound kernel
 * so that likely races are checked first.  BF16 operands, FP32 accumulation
 * and FP32 master weights; trained with weighted binary cross-entropy and
 * AdamW by the library's own forward and backward kernels on labels from the
 * exact check.  It never changes a verdict. */
enum { HGRD_MLP_IN = 96, HGRD_MLP_HIDDEN = 256, HGRD_MLP_PARAMS = 90881 };

/* The eligible pairs a <= b of a bound descriptor (same array, not both loads,
 * not both atomics of sufficient scope: the pair rule of Sec. 6.1 and
 * Appendix A; neither access dead) with 96 features each: per access, its kind
 * and scope, width, memory space, the folded coefficients on thread, block
 * and loop ids, div/mod and guard counts, its index range against the array;
 * per pair, interval overlap and identical interval ranges, race kinds the
 * pair rule allows, byte-range overlap, coefficient differences, launch and array sizes.  Host memory:
 * out[cap * 96], pairs[cap * 2]; *n = number of eligible pairs (ETRUNCATED
 * when it exceeds cap). */
int hgrd_pair_features(const hgrd_desc* d, float* out, uint8_t* pairs, uint32_t cap, uint32_t* n);

/* Model buffer (device, caller allocated, 256-byte aligned): FP32 parameters,
 * gradients, AdamW moments, then BF16 parameters.  Workspace for a batch of
 * n samples: activations. */
size_t hgrd_mlp_model_bytes(void);
size_t hgrd_mlp_workspace_bytes(uint32_t n);
/* Uniform(+-1/sqrt(fan_in)) weights from a counter-based generator, zero biases and moments. */
int hgrd_mlp_init(void* d_model, uint64_t seed, void* cuda_stream);
/* Logits of n feature rows d_x[n * 96] (FP32, converted to BF16) into d_logits[n]. */
int hgrd_mlp_predict(const void* d_model, const float* d_x, uint32_t n, float* d_logits, void* d_ws,
                     size_t ws_bytes, void* cuda_stream);
/* Gradients (into the model buffer) of the weighted mean BCE loss
 * sum_i w_i * bce(z_i, y_i) / wsum; d_w may be NULL (all weights 1). */
int hgrd_mlp_grad(void* d_model, const float* d_x, const float* d_y, const float* d_w, float wsum, uint32_t n,
                  void* d_ws, size_t ws_bytes, void* cuda_stream);
/* hgrd_mlp_grad, then one AdamW step (beta 0.9 / 0.999, eps 1e-8, decoupled
 * weight decay); the batch loss is written to *d_loss (device) when given. */
int hgrd_mlp_train_step(void* d_model, const float* d_x, const float* d_y, const float* d_w, float wsum, uint32_t n,
                        float lr, float weight_decay, uint32_t step, void* d_ws, size_t ws_bytes, void* cuda_stream,
                        float* d_loss);
/* Device pointers of the FP32 parameters and gradients inside the model buffer. */
int hgrd_mlp_params(const void* d_model, float** d_params, float** d_grads);
/* Refresh the BF16 copies after the FP32 parameters were written directly. */
int hgrd_mlp_sync_bf16(void* d_model, void* cuda_stream);

/* Ranked check.  Scores the eligible pairs (with the model, or with
 * host_scores[n_pairs] in hgrd_pair_features order when given), runs a
 * restricted exact check of the accesses of the top `topk` pairs that stops
 * at its first race, and only if that finds none runs the full check (also
 * stopping at its first race).  The ranked check runs only when the best
 * pair's score (a logit) reaches min_score, so kernels the model deems clean
 * go straight to the full check.  With at most `topk` eligible pairs no
 * scores are computed: every pair is checked at once.  When the checked
 * accesses cover every eligible pair, the restricted check is the whole
 * verdict (accesses in no eligible pair race with nothing, Sec. 6.1); its
 * n_keys / n_oob then count the checked accesses only.  The racy flag is
 * exact; when racy, the witnesses are the races found (each a real race),
 * not the full set.  A restricted check small enough for one CTA runs there,
 * and a kernel whose full check runs in one CTA is not ranked at all.  The
 * first call on a host thread allocates 200 KB of pinned host memory for the
 * features and scores, kept for the thread's lifetime.
 * Workspace: hgrd_ranked_workspace_size. */
typedef struct {
  uint32_t n_pairs, stage; /* stage 1: race found by the ranked check; 2: the full check decided */
  uint32_t access_mask, pad;
  uint64_t keys_ranked, keys_full; /* keys the two checks expanded */
  float ms_rank, pad2;             /* host time of features + scoring */
} hgrd_rank_info;
int hgrd_ranked_workspace_size(const hgrd_desc* d, const hgrd_check_opts* o, size_t* bytes);
int hgrd_check_ranked(const hgrd_desc* d, const hgrd_check_opts* o, const void* d_model, const float* host_scores,
                      uint32_t topk, float min_score, void* d_ws, size_t ws_bytes, void* cuda_stream,
                      hgrd_witness* host_out, uint64_t cap, hgrd_verdict* v, hgrd_rank_info* info);

/* hgrd_check without a caller workspace, for callers that cannot allocate
 * device memory: code running while another component owns all device memory
 * (a caching allocator or pool that must not be bypassed), code called from
 * inside such an allocator, or embedders without access to cudaMalloc.  The
 * paper has no counterpart; this is a deployment convenience.
 *   * Scratch: a 64 MiB array compiled into the library.  Every device that
 *     loads the library holds it until the process exits.
 *   * Bindings whose hgrd_workspace_size exceeds 64 MiB are rejected with
 *     HGRD_ENOMEM before any work is enqueued.
 *   * The call allocates nothing: no cudaMalloc/cudaFree, no streams, events
 *     or graphs (the witness merge is launched directly, never through a
 *     cached graph), no pinned host staging (witnesses are widened in place
 *     inside host_out); hgrd_stats.cuda_objects_created does not move.
 *   * The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (once per device, with that device current).
 *   * Never on a capturing stream: the call reads its results back and
 *     synchronises the stream, so a capturing stream gets HGRD_EINVAL.
 *   * All calls share the one array, which keeps the previous call's data;
 *     each call clears what must start at zero.  Calls whose GPU work
 *     overlaps (other host threads, other streams) race on the array.
 *   * Outputs as hgrd_check (witnesses, counts, racy-pair matrices), except
 *     that the canonical instance pair is not searched (pair_found = 0).
 *     Synchronous on return. */
int hgrd_check_noalloc(const hgrd_desc* d, const hgrd_check_opts* o, void* cuda_stream, hgrd_witness* host_out,
                       uint64_t cap, hgrd_verdict* v);

/* ---- Specialised expansion ---------------------------------------------------
 * The expansion (every instance's guards, index and interval, Sec. 6.2's
 * addr / tb / id) normally interprets the bound program.  These calls build
 * kernels specialised to the program's structure instead: CUDA source where
 * each op, guard, index and interval is straight-line code, with the bound
 * values (coefficients, divisors, sizes) read from the kernel's parameters,
 * compiled for sm_103a at run time (seconds) and cached for the process, so
 * bindings of one structure share a module.  Results are identical to the
 * interpreted kernels.  Once compiled for a bound descriptor, every check of
 * it uses them unless HGRD_NO_JIT is set.
 *   hgrd_jit_compile: compile now (or find in the cache) for the bound
 *     descriptor `d` and the pipeline `o` selects (o->flags HGRD_NO_SPLIT;
 *     o may be NULL); *compile_ms (may be NULL) = time this call spent
 *     compiling (0 on a cache hit).  HGRD_EUNSUPPORTED with the compiler's
 *     log (hgrd_last_error) when compiling or loading fails, e.g. without a
 *     device.  Needs a current CUDA device to load the module.
 *   hgrd_jit_source: the generated source for the same choice,
 *     NUL-terminated into out[0, cap); *len = its full length (out may be
 *     NULL to size it). */
int hgrd_jit_compile(const hgrd_desc* d, const hgrd_check_opts* o, double* compile_ms);
int hgrd_jit_source(const hgrd_desc* d, const hgrd_check_opts* o, char* out, size_t cap, size_t* len);

/* ---- Host-admissible inputs (the paper's question: a race under some input) --
 * A race "under some host-admissible input" (Sec. 3, Sec. 5.1) is decided here
 * by checking a set of admissible bindings (the batched path), not
 * symbolically.
 *   hgrd_desc_params: the parameters of a loaded descriptor, in declaration
 *     order, with the bounds its asserts put on each parameter alone (asserts
 *     affine in one parameter after folding constants: `N > 0`, `2*N <= 8192`;
 *     others, e.g. those with launch dimensions, are enforced at bind time).
 *     Writes min(cap, n) entries; *n = the parameter count.
 *   hgrd_bound_hash: a 64-bit hash of everything a check of the bound
 *     descriptor reads (compiled program, array sizes and granules): two
 *     bindings with equal hashes have equal verdicts, so a sweep checks one. */
typedef struct {
  char name[32];
  int64_t lo, hi;          /* inclusive; INT64_MIN / INT64_MAX when unbounded */
  uint32_t has_lo, has_hi;
} hgrd_param_info;
int hgrd_desc_params(const hgrd_desc* d, hgrd_param_info* out, uint32_t cap, uint32_t* n);
/* Size of a bound check, known at bind time without a device: the
 * (block, thread, loop vector, access) instances it enumerates (Sec. 6.2's
 * instance space under the host binding, before guards) and the most keys
 * its live instances can make.  Cost model for splitting batches. */
int hgrd_bound_info(const hgrd_desc* d, uint64_t* n_instances, uint64_t* max_keys);
int hgrd_bound_hash(const hgrd_desc* d, uint64_t* h);

void hgrd_free_desc(hgrd_desc* d);
const char* hgrd_last_error(void);

/* Self-test hook for the division-by-constant method used by the kernels
 * (Granlund & Montgomery 1994, Thm. 4.2, with C truncation for negative
 * numerators): q = n / d, r = n % d for d > 0; wide selects the 64-bit form.
 * Host-side computation of exactly the arithmetic the device performs. */
int hgrd_debug_divmod(int64_t n, int64_t d, int wide, int64_t* q, int64_t* r);

/* Failure-path self-test of the bounded device waits: one sort pass over
 * 12288 random keys whose first tile is never taken (its tile ticket starts
 * past it), so every other tile's look-back waits on a status nothing will
 * publish.  Each wait gives up after its iteration limit (a few seconds at
 * most), the kernel records the timeout and returns, and this call returns
 * HGRD_ETIMEOUT with the context still usable; HGRD_OK would mean the wait
 * did not run out.  Workspace: at least 256 KB, 256-byte aligned.  Has no
 * counterpart in the paper: it exercises this library's own error path. */
int hgrd_debug_lookback_timeout(void* d_ws, size_t ws_bytes, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* HGRD_H */
