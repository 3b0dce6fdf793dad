// hgrd_check and friends: workspace layout and the stream-ordered pipeline
//   expand(count) -> scan -> expand(write) -> onesweep passes ->
//   candidates -> exact -> witness sort -> merge -> kind counts
// All sizes the kernels need at run time are read from device counters, so
// nothing between the first and the last kernel waits on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "hgrd_host.h"
#include "jit.h"
#include "kernels.cuh"

namespace hgrd {
// the batch's on-chip kernel for one small check (batch.cu)
bool small_single_ok(const Bound& B, uint32_t only);
cudaError_t launch_small_single(const Launch& L, const DProg* d_prog, uint64_t* counters, uint64_t* scratch,
                                uint64_t* uniq);
}  // namespace hgrd

namespace hgrd {

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// HGRD_ALL_KEYS runs one global sort on the interpreted kernels: the flags
// it implies are set here, once, at every entry point that takes options
const hgrd_check_opts* norm_opts(const hgrd_check_opts* o, hgrd_check_opts* tmp) {
  if (!o || !(o->flags & HGRD_ALL_KEYS)) return o;
  *tmp = *o;
  tmp->flags |= HGRD_NO_SPLIT | HGRD_NO_JIT | HGRD_NO_SMALL;
  tmp->flags &= ~(uint32_t)HGRD_JIT;
  return tmp;
}

struct Layout {
  size_t counters, prog, unit_cnt, unit_off, partials, hist, status, keysA, keysB, raw, raw2, flags, excl,
      pairs, stbl, sbase, cells, total;
  bool cfilter;        // the cell filter's table exists (the filter runs in the first sort pass)
  uint64_t raw_cap, pair_cap, status_words;
  uint64_t scap;       // room for keys of candidate shared bins (block-local mode)
  uint64_t key_words;  // length of each key buffer
  uint64_t cand_cap;   // candidate entries (two words each) the spare key buffer holds
  uint64_t nsort;      // most keys the global sort can see
};

Layout layout(const Bound& B, const hgrd_check_opts* o) {
  Layout L{};
  const DProg& P = B.prog;
  const uint64_t nk = std::max<uint64_t>(B.nkeys_max, 1);
  // the key buffers hold what can be written: kept keys of every access (one
  // sort of everything), or kept global keys plus room for candidate shared
  // bins (block-local mode)
  const bool all = o && (o->flags & HGRD_ALL_KEYS);
  const bool split = P.smode && !(o && (o->flags & HGRD_NO_SPLIT)) && !all;
  L.scap = split ? ((o && o->max_shared_keys) ? o->max_shared_keys : P.scap) : 0;
  const uint64_t nsort_all = all ? B.nkeys_max : B.nsort_max_all;  // every live key, or the kept ones
  // (whole rows of 16 keys: the candidate scan reads its keys by rows)
  L.key_words = (std::max<uint64_t>(split ? B.nsort_max_split + L.scap : nsort_all, 1) + 63) & ~63ull;
  // a candidate run holds at least two keys
  L.cand_cap = std::max<uint64_t>(L.key_words / 2, 1);
  // defaults scale with the problem and come back as HGRD_ENOMEM (with the
  // count needed) when a check outgrows them: per-run witnesses rarely exceed
  // the written keys, and the instances on one granule never exceed the keys
  L.raw_cap = (o && o->max_raw_witness)
                  ? o->max_raw_witness
                  : std::min<uint64_t>(1ull << 24, std::max<uint64_t>(1ull << 12, 2 * L.key_words));
  L.pair_cap = (o && o->pair_cap) ? o->pair_cap : std::min<uint64_t>(1ull << 20, nk);
  const uint64_t nunits = std::max<int64_t>(P.nunits, 1);
  const uint32_t lfl = o ? o->flags : 0u;
  L.cfilter = P.cfilter && !(lfl & HGRD_NO_CELL_FILTER) && ((lfl & HGRD_CELL_FILTER) || P.cfilter_auto);
  const uint64_t scan_n = std::max(nunits, L.raw_cap);
  // look-back status of the sort passes: tiles of the larger of the key sort
  // and the witness sort
  const uint64_t ns = std::max<uint64_t>(split ? B.nsort_max_split : nsort_all, 1);
  L.nsort = ns;
  const uint64_t tiles = std::max((ns + RS_MIN_TILE - 1) / RS_MIN_TILE, (L.raw_cap + RS_MIN_TILE - 1) / RS_MIN_TILE);
  L.status_words = tiles * RS_RADIX;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  L.counters = take(C_WORDS * 8);
  L.hist = take(MAX_PASSES * 256 * 8);  // right after the counters: one clear covers both
  L.prog = take(sizeof(DProg));
  L.unit_cnt = take(nunits * 8);
  L.unit_off = take(nunits * 8);
  L.partials = take(((scan_n + SCAN_TILE - 1) / SCAN_TILE + 1) * 8);
  L.status = take(L.status_words * 8);
  L.keysA = take(L.key_words * 8);
  L.keysB = take(L.key_words * 8);
  L.raw = take(L.raw_cap * 8);
  L.raw2 = take(L.raw_cap * 8);
  L.flags = take(L.raw_cap * 8);
  L.excl = take(L.raw_cap * 8);
  L.pairs = take((size_t)L.pair_cap * sizeof(PairRec));
  // block-local mode: bin table (start << 32 | count per candidate bin) and
  // the base of every block's candidate keys
  L.stbl = take(P.smode ? (size_t)P.nblk * (size_t)P.nsbins * 8 : 0);
  L.sbase = take(P.smode ? (size_t)P.nblk * 8 : 0);
  // cell filter: one state word per cell
  L.cells = take(L.cfilter ? (size_t)P.ncells * 4 : 0);
  L.total = off;
  return L;
}

// the cell filter runs inside the first sort pass, when there is one
bool filter_runs(const Layout& W, int passes) { return W.cfilter && passes > 0; }

int nsm_of_current_device() {
  static thread_local int cached_dev = -1, cached_n = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != cached_dev) {
    cudaDeviceGetAttribute(&cached_n, cudaDevAttrMultiProcessorCount, dev);
    cached_dev = dev;
  }
  return cached_n > 0 ? cached_n : 1;
}

// stage timing (HGRD_PROFILE): one event before the first stage and one after each
struct Prof {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<std::string> names;
  void reset(bool enable, cudaStream_t st) {
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear();
    names.clear();
    on = enable;
    s = st;
    if (on) mark("");
  }
  void mark(const char* name) {
    if (!on) return;
    cudaEvent_t e;
    note_created();
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    ev.push_back(e);
    names.push_back(name);
  }
};
thread_local Prof g_prof;

#define CK(x)                                                                               \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess) return fail(HGRD_EDEVICE, std::string("CUDA: ") + cudaGetErrorString(e_)); \
  } while (0)

int prechecks(const hgrd_desc* d, void* d_ws, size_t ws_bytes, const hgrd_check_opts* o, Layout* Lo) {
  if (!d) return fail(HGRD_EINVAL, "null descriptor");
  if (!d->bound) return fail(HGRD_EINVAL, "descriptor is not bound (call hgrd_bind_host_params)");
  *Lo = layout(*d->bound, o);
  if (!d_ws) return fail(HGRD_EINVAL, "null workspace");
  if (((uintptr_t)d_ws & 255) != 0) return fail(HGRD_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < Lo->total)
    return fail(HGRD_ENOMEM, "workspace too small: need " + std::to_string(Lo->total) + " bytes");
  return HGRD_OK;
}

// offset of the buffer holding the merged witnesses after enqueue (the
// device-wide merge sorts raw <-> raw2 in WP passes and merges into the other)
size_t uniq_off(const Layout& W) {
  const int WP = (WIT_SORT_HI - WIT_SORT_LO + 7) / 8;
  return (WP % 2 == 0) ? W.raw2 : W.raw;
}

// the device-wide witness merge: radix sort of the raw words, head flags,
// scan, OR-merge; its kernels read the count from counters[C_NRAWBIG]
cudaError_t enqueue_witness_big(const Launch& L, const Layout& W, char* ws, int P) {
  auto U = [&](size_t off) { return (uint64_t*)(ws + off); };
  uint64_t* cnt = U(W.counters);
  const int WP = (WIT_SORT_HI - WIT_SORT_LO + 7) / 8;
  uint64_t* nraw = cnt + C_NRAWBIG;
  cudaError_t e;
  if ((e = launch_zero_status(L, U(W.status), nraw, W.status_words)) != cudaSuccess) return e;
  uint64_t* whist = U(W.hist) + 8 * 256;
  if ((e = launch_histogram(L, U(W.raw), nraw, W.raw_cap, WIT_SORT_LO, WP, whist)) != cudaSuccess) return e;
  uint64_t* win = U(W.raw);
  uint64_t* wout = U(W.raw2);
  for (int p = 0; p < WP; p++) {
    if ((e = launch_onesweep(L, win, wout, nraw, W.raw_cap, WIT_SORT_LO + 8 * p, whist + p * 256, U(W.status),
                             cnt + C_TICKET0 + P + p, (uint32_t)(P + p + 1), cnt + C_ERR)) != cudaSuccess)
      return e;
    std::swap(win, wout);
  }
  // win: sorted raw witnesses; wout receives the merged set
  if ((e = launch_zero(L, wout, nraw, W.raw_cap)) != cudaSuccess) return e;
  if ((e = launch_heads(L, win, nraw, W.raw_cap, U(W.flags))) != cudaSuccess) return e;
  if ((e = launch_scan(L, U(W.flags), U(W.excl), nraw, W.raw_cap, U(W.partials), cnt + C_NUNIQ)) != cudaSuccess)
    return e;
  if ((e = launch_merge(L, win, U(W.flags), U(W.excl), nraw, W.raw_cap, wout)) != cudaSuccess) return e;
  return launch_kind_counts(L, wout, cnt, nraw);
}

// The witness merge as an instantiated graph per (device, workspace, layout,
// sort passes, onesweep shape): the split kernel, then a conditional IF node
// whose body (captured from enqueue_witness_big) runs only when the split
// kernel opens it.  nullptr when graphs are unavailable; the caller then
// launches the kernels directly.
std::mutex g_wg_mu;
std::map<std::vector<uint64_t>, cudaGraphExec_t> g_wg;
bool g_wg_off = false;

cudaGraphExec_t witness_graph(const Launch& L, const Layout& W, char* ws, int P) {
  int dev = 0;
  cudaGetDevice(&dev);
  const std::vector<uint64_t> key = {(uint64_t)dev, (uint64_t)(uintptr_t)ws, W.counters, W.raw, W.raw2, W.flags,
                                     W.excl, W.partials, W.hist, W.status, W.raw_cap, W.status_words,
                                     (uint64_t)P, sort_variant_key()};
  std::lock_guard<std::mutex> lk(g_wg_mu);
  auto it = g_wg.find(key);
  if (it != g_wg.end()) return it->second;
  if (g_wg_off || g_wg.size() >= 256) return nullptr;
  note_created(2);  // a capture stream and the instantiated graph
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle h{};
  ok = ok && cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNode_t split = nullptr, cond = nullptr;
  uint64_t* cnt = (uint64_t*)(ws + W.counters);
  uint64_t raw_cap = W.raw_cap;
  if (ok) {
    void* args[] = {(void*)&cnt, (void*)&raw_cap, (void*)&h};
    cudaKernelNodeParams kp{};
    kp.func = (void*)witness_split_cond_fn();
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    ok = cudaGraphAddKernelNode(&split, g, nullptr, 0, &kp) == cudaSuccess;
  }
  cudaGraphNodeParams cp{};
  if (ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    ok = cudaGraphAddNode(&cond, g, &split, nullptr, 1, &cp) == cudaSuccess;
  }
  if (ok) ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      uint64_t captured = 0;
      Launch LC{cs, L.nsm, &captured};
      const bool launched = enqueue_witness_big(LC, W, ws, P) == cudaSuccess;
      cudaGraph_t out = nullptr;
      ok = cudaStreamEndCapture(cs, &out) == cudaSuccess && launched;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (cs) cudaStreamDestroy(cs);
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();  // clear a sticky launch-configuration error, if any
    g_wg_off = true;
    return nullptr;
  }
  g_wg[key] = exec;
  return exec;
}

// the buffer holding the merged witnesses after enqueue
uint64_t* uniq_buffer(const hgrd_desc* d, const Layout& W, char* ws) {
  const int WP = (WIT_SORT_HI - WIT_SORT_LO + 7) / 8;
  (void)d;
  return (uint64_t*)(ws + ((WP % 2 == 0) ? W.raw2 : W.raw));
}

// The canonical-pair search for the minimal witness (device side): the
// instances of its two accesses on its granule, gathered into the pair
// records.  Needs only device results (the merged witnesses), so it can
// follow the witness merge in the same stream or graph; with no witness its
// kernels find nothing to do.
cudaError_t enqueue_pair_search(const Launch& L, const hgrd_desc* d, const hgrd_check_opts* o, const Layout& W,
                                char* ws, const uint64_t* duniq, const DProg* dprog) {
  const Bound& B = *d->bound;
  const DProg& HP = B.prog;
  cudaStream_t s = L.s;
  cudaError_t e;
  PairRec* pr = (PairRec*)(ws + W.pairs);
  if ((e = cudaMemsetAsync(ws + W.counters + 8 * C_NPAIR, 0, 8, s)) != cudaSuccess) return e;
  // a global-memory witness: search only the blocks of its run (listed in
  // the unit-offset buffer, free after the write pass); the one-CTA path
  // sorted nothing, so it searches every unit
  uint64_t* blist = (uint64_t*)(ws + W.unit_off);
  if ((e = cudaMemsetAsync(ws + W.counters + 8 * C_NPB, 0, 8, s)) != cudaSuccess) return e;
  // the path enqueue took for these options (the same decisions, made again)
  const uint32_t fl = o ? o->flags : 0u;
  const bool small = !(fl & (HGRD_NO_SMALL | HGRD_JIT)) && small_single_ok(B, o ? o->only_accesses : 0u);
  const bool split = HP.smode && !(fl & HGRD_NO_SPLIT);
  const int passes = split ? B.sort_passes_split : B.sort_passes;
  if (!small) {
    const uint64_t* sorted = (uint64_t*)(ws + ((passes & 1) ? W.keysB : W.keysA));
    const uint64_t* nsorted = (const uint64_t*)(ws + W.counters) + (filter_runs(W, passes) ? C_NGC : C_NG);
    if ((e = launch_pair_blocks(L, sorted, nsorted, dprog, duniq,
                                (uint64_t*)(ws + W.counters), blist)) != cudaSuccess)
      return e;
  }
  // the specialised kernels when this binding has them (either module holds the search)
  const bool jsplit = jit_ready(B, true), jplain = !jsplit && jit_ready(B, false);
  if ((jsplit || jplain) && !(fl & HGRD_NO_JIT))
    return launch_jit_expand(L, B, 2, HP, nullptr, blist, nullptr, nullptr, nullptr, 0, (uint64_t*)(ws + W.counters),
                             nullptr, nullptr, 0xffffffffu, jsplit, duniq, pr, W.pair_cap);
  return launch_expand(L, 2, B.wide, dprog, HP, nullptr, blist, nullptr, nullptr, 0, (uint64_t*)(ws + W.counters),
                       duniq, pr, W.pair_cap);
}

// An enqueue being captured into a check graph (HGRD_GRAPH): the graph, a
// pinned copy of the program, the device copy the graph's kernels read (owned
// by the graph, filled from the pinned copy outside the graph), and a stream
// for capturing the conditional witness-merge body.
struct Capture {
  cudaGraph_t graph;
  DProg* pinned_prog;
  DProg* dev_prog;
  cudaStream_t body_stream;
};

// The device program the last check enqueued on a workspace ran with (its
// slot in the workspace, or a check graph's own copy): a later pair search
// from collect reads the same one.
std::mutex g_wsprog_mu;
std::map<const void*, const DProg*> g_wsprog;
void note_ws_prog(const void* ws, const DProg* p) {
  std::lock_guard<std::mutex> lk(g_wsprog_mu);
  g_wsprog[ws] = p;
}
const DProg* ws_prog(const void* ws, const DProg* dflt) {
  std::lock_guard<std::mutex> lk(g_wsprog_mu);
  auto it = g_wsprog.find(ws);
  return it == g_wsprog.end() ? dflt : it->second;
}

// The conditional witness merge inside a stream capture on s: the split
// kernel, then an IF node (appended to the capture's dependencies) whose body
// is the device-wide merge captured on the capture's body stream.
cudaError_t capture_witness_cond(const Launch& L, const Layout& W, char* ws, int P, const Capture& cc) {
  cudaGraphConditionalHandle h{};
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, cc.graph, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  if ((e = launch_witness_split_cond(L, (uint64_t*)(ws + W.counters), W.raw_cap, h)) != cudaSuccess) return e;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if ((e = cudaStreamGetCaptureInfo(L.s, &st, nullptr, &g, &deps, nullptr, &ndeps)) != cudaSuccess) return e;
  if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t cond = nullptr;
  if ((e = cudaGraphAddNode(&cond, g, deps, nullptr, ndeps, &cp)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(L.s, &cond, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
      cudaSuccess)
    return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(cc.body_stream, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return e;
  uint64_t captured = 0;
  Launch LC{cc.body_stream, L.nsm, &captured};
  const cudaError_t eb = enqueue_witness_big(LC, W, ws, P);
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(cc.body_stream, &out);
  return eb != cudaSuccess ? eb : e;
}

// `noalloc`: create no CUDA object on the way (no profiling events, no
// cached witness-merge graph); hgrd_check_noalloc's promise rests on it
int enqueue(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, cudaStream_t s,
            const DProg* dprog_resident = nullptr, const Capture* cc = nullptr, bool pair = false,
            bool noalloc = false) {
  Layout W;
  int rc = prechecks(d, d_ws, ws_bytes, o, &W);
  if (rc) return rc;
  const Bound& B = *d->bound;
  const DProg& HP = B.prog;
  char* ws = (char*)d_ws;
  auto U = [&](size_t off) { return (uint64_t*)(ws + off); };
  uint64_t* cnt = U(W.counters);
  // the compiled program: uploaded into the workspace, already resident, or
  // (in a check graph) the graph's own device copy
  const DProg* dprog = dprog_resident ? dprog_resident : cc ? cc->dev_prog : (const DProg*)(ws + W.prog);
  // a check restricted to a subset of the accesses runs a copy of the
  // program with the other accesses removed (their keys are never made)
  const uint32_t only = o ? o->only_accesses : 0u;
  const bool restricted = only != 0 && only != 0xffffffffu && !dprog_resident;
  // block-local mode for shared-array keys unless the caller asks for one global sort
  const bool split = HP.smode && !(o && (o->flags & HGRD_NO_SPLIT));
  g_stats = hgrd_stats{};
  g_stats.int64_path = B.wide;
  g_stats.eval_ops = B.eval_ops;
  g_stats.sort_passes = (uint32_t)(split ? B.sort_passes_split : B.sort_passes);
  g_stats.shared_bins = split ? 1u : 0u;
  // specialised expansion kernels: compiled on request (HGRD_JIT, or
  // hgrd_jit_compile ahead of time), then used for every check of this binding
  const uint32_t fl = o ? o->flags : 0u;
  bool jit = false;
  if (!(fl & HGRD_NO_JIT)) {
    if (fl & HGRD_JIT) {
      const int jrc = jit_prepare(B, split, nullptr);
      if (jrc != HGRD_OK) return jrc;
      jit = true;
    } else {
      jit = jit_ready(B, split);
    }
  }
  g_stats.jit = jit ? 1u : 0u;
  if (jit) {  // the specialised walk evaluates loop-invariant and ranged accesses once per thread
    if (!B.eval_ops_jit) B.eval_ops_jit = jit_eval_ops(HP);
    g_stats.eval_ops = B.eval_ops_jit;
  }
  const uint32_t only_mask = (jit && restricted) ? only : 0xffffffffu;
  Launch L{s, nsm_of_current_device(), &g_stats.kernel_launches};
  if (noalloc) g_prof.on = false;  // the events of an earlier profiled check stay readable, none are made
  else g_prof.reset(o && (o->flags & HGRD_PROFILE), s);

  const uint64_t nsort = W.nsort;
  CK(cudaMemsetAsync(cnt, 0, W.hist + MAX_PASSES * 256 * 8 - W.counters, s));  // counters and histograms
  bool any = false;
  for (int a = 0; a < HP.nacc; a++) any |= !HP.acc[a].dead;
  if (!any || B.nkeys_max == 0 || HP.nunits == 0) return HGRD_OK;  // nothing can be live
  // the program this check runs: a copy when it is restricted to a subset of
  // the accesses (the others marked dead) or has its own room for shared keys
  const DProg* hprog = &HP;
  if (!dprog_resident) {
    const bool all_keys = o && (o->flags & HGRD_ALL_KEYS);
    if (restricted || (split && W.scap != HP.scap) || all_keys) {
      static thread_local DProg run_prog;
      run_prog = HP;
      if (all_keys)  // every live access writes its keys
        for (int a = 0; a < run_prog.nacc; a++)
          if (!run_prog.acc[a].dead) run_prog.emask |= 1u << a;
      if (restricted)
        for (int a = 0; a < run_prog.nacc; a++)
          if (!((only >> a) & 1u)) run_prog.acc[a].dead = 1;
      if (split) run_prog.scap = W.scap;
      hprog = &run_prog;
    }
    if (cc) {  // the graph's device copy is filled from this pinned one, outside the graph
      memcpy(cc->pinned_prog, hprog, sizeof(DProg));
    } else {
      CK(cudaMemcpyAsync(ws + W.prog, hprog, sizeof(DProg), cudaMemcpyHostToDevice, s));
      g_stats.h2d_bytes += sizeof(DProg);
    }
  }
  if (!cc && !noalloc) note_ws_prog(ws, dprog);  // (the no-allocation check runs no later pair search)
  g_prof.mark("setup");
  // a small check runs whole in one CTA (the batched form's on-chip kernel),
  // unless specialised kernels were asked for; its verdict lands in the
  // counters and merged-witness buffer as usual
  if (!(fl & (HGRD_NO_SMALL | HGRD_JIT)) && !dprog_resident && small_single_ok(B, restricted ? only : 0u)) {
    CK(launch_small_single(L, dprog, cnt, U(W.raw2), uniq_buffer(d, W, ws)));
    g_prof.mark("small");
    g_stats.small = 1;
    g_stats.shared_bins = 0;
    g_stats.jit = 0;
    g_stats.sort_passes = 0;
    if (pair && !(fl & HGRD_NO_PAIR)) CK(enqueue_pair_search(L, d, o, W, ws, uniq_buffer(d, W, ws), dprog));
    return HGRD_OK;
  }

  const int P = split ? B.sort_passes_split : B.sort_passes;
  uint64_t* keysA = U(W.keysA);
  uint64_t* keysB = U(W.keysB);
  // keys the sort and the candidate scan walk: the written ones (of accesses
  // that may race), only those of global arrays in block-local mode (the
  // candidate bins follow them in the final buffer)
  uint64_t* nkeys = cnt + C_NG;
  // cell filter: the count pass fills the per-cell table (its key pointer);
  // the first sort pass drops the written keys of cells without a writer and
  // two threads, so later passes and the scans see only the kept ones.
  // Candidate-bin keys go behind all written global keys in the final buffer
  // (at C_NG), which no pass writes.
  const bool cf = filter_runs(W, P);
  uint32_t* ctab = cf ? (uint32_t*)(ws + W.cells) : nullptr;
  if (cf) {
    // the cells the count pass can note: those of the accesses whose keys
    // are written (in the block-local mode, of the global arrays only)
    uint64_t lo = ~0ull, hi = 0;
    for (int a = 0; a < hprog->nacc; a++) {
      const DAcc& A = hprog->acc[a];
      if (!((hprog->emask >> a) & 1u) || A.dead || (split && A.shared)) continue;
      const uint64_t end = A.cbase + (A.shared ? (uint64_t)hprog->nblk * A.ngran : A.ngran);
      lo = std::min(lo, A.cbase);
      hi = std::max(hi, end);
    }
    if (hi > lo) CK(cudaMemsetAsync(ctab + lo, 0, (hi - lo) * 4, s));
  }
  uint64_t* fin = (P & 1) ? keysB : keysA;  // where the sorted keys end
  uint64_t* cnt_tab = cf ? (uint64_t*)ctab : nullptr;
  // compact form (cell filter, plain pipeline): the write pass, which runs
  // with the cell table complete, also appends the keys of kept cells to a
  // compact buffer (the raw-witness buffer, free until the exact scan); when
  // they all fit (at most TAIL_KEYS), one CTA sorts them whole by the full
  // key (the scans need a run's keys ordered by interval, block, warp
  // interval and warp; the lanes of a warp in any order) into the final
  // buffer, and the filter's histogram, the sort passes and the tail return
  // at once.  Otherwise the filter and the passes run as below.
  const bool compact = cf && !split;
  uint64_t* cbuf = compact ? U(W.raw) : nullptr;
  const uint64_t ccap = compact ? std::min<uint64_t>(W.raw_cap, TAIL_KEYS) : 0;
  const uint32_t* wtab = compact ? ctab : nullptr;
  if (jit) {
    const int m0 = split ? 3 : 0, m1 = split ? 4 : 1;
    CK(launch_jit_expand(L, B, m0, *hprog, U(W.unit_cnt), nullptr, cnt_tab, nullptr, U(W.hist), 1, cnt, U(W.stbl),
                         U(W.sbase), only_mask, split));
    g_prof.mark("expand_count");
    CK(launch_scan(L, U(W.unit_cnt), U(W.unit_off), nullptr, (uint64_t)HP.nunits, U(W.partials), nkeys));
    // look-back status of the tiles the key sort will use: no stale epoch may
    // survive (with the cell filter, its histogram kernel clears them)
    if (!cf) CK(launch_zero_status(L, U(W.status), nkeys, W.status_words));
    g_prof.mark("unit_scan");
    CK(launch_jit_expand(L, B, m1, *hprog, nullptr, U(W.unit_off), keysA, fin, nullptr, P, cnt, U(W.stbl),
                         U(W.sbase), only_mask, split, nullptr, nullptr, 0, wtab, cbuf, ccap));
    g_prof.mark("expand_write");
  } else if (split) {
    CK(launch_expand_block(L, 3, B.wide, dprog, HP, U(W.unit_cnt), nullptr, cnt_tab, nullptr, U(W.hist), cnt,
                           U(W.stbl), U(W.sbase)));
    g_prof.mark("expand_count");
    CK(launch_scan(L, U(W.unit_cnt), U(W.unit_off), nullptr, (uint64_t)HP.nunits, U(W.partials), nkeys));
    // look-back status of the tiles the key sort will use: no stale epoch may
    // survive (with the cell filter, its histogram kernel clears them)
    if (!cf) CK(launch_zero_status(L, U(W.status), nkeys, W.status_words));
    g_prof.mark("unit_scan");
    CK(launch_expand_block(L, 4, B.wide, dprog, HP, nullptr, U(W.unit_off), keysA, fin, nullptr, cnt, U(W.stbl),
                           U(W.sbase)));
    g_prof.mark("expand_write");
  } else {
    CK(launch_expand(L, 0, B.wide, dprog, HP, U(W.unit_cnt), nullptr, cnt_tab, U(W.hist), 1, cnt, nullptr, nullptr,
                     0));
    g_prof.mark("expand_count");
    CK(launch_scan(L, U(W.unit_cnt), U(W.unit_off), nullptr, (uint64_t)HP.nunits, U(W.partials), nkeys));
    // look-back status of the tiles the key sort will use: no stale epoch may
    // survive (with the cell filter, its histogram kernel clears them)
    if (!cf) CK(launch_zero_status(L, U(W.status), nkeys, W.status_words));
    g_prof.mark("unit_scan");
    CK(launch_expand(L, 1, B.wide, dprog, HP, nullptr, U(W.unit_off), keysA, nullptr, P, cnt, nullptr, nullptr, 0,
                     wtab, cbuf, ccap));
    g_prof.mark("expand_write");
  }
  if (compact) CK(launch_compact_sort(L, cbuf, fin, cnt + C_NCOMPACT, ccap, cnt + C_TAIL, cnt + C_NGC));
  uint64_t* in = keysA;
  uint64_t* out = keysB;
  const uint64_t* nsorted = nkeys;  // keys the first pass reads
  if (cf) {
    // digit histogram of the first pass over the kept keys, and their count
    CK(launch_cell_hist(L, keysA, nkeys, nsort, ctab, HP.ncells, HP.PB + HP.IVB, U(W.hist), HP.SB, cnt + C_NGC,
                        U(W.status), W.status_words, compact ? cnt + C_TAIL : nullptr));
    nkeys = cnt + C_NGC;
    g_prof.mark("cell_filter");
  }
  // the expansion (or the filter) counted digit 0; each pass counts the digit
  // of the next.  After the first pass, at most 4096 keys left are sorted on
  // the remaining digits by one CTA, straight into the final buffer, and the
  // later passes return at once.
  for (int p = 0; p < P; p++) {
    CK(launch_onesweep(L, in, out, p == 0 ? nsorted : nkeys, nsort, HP.SB + 8 * p, U(W.hist) + p * 256,
                       U(W.status), cnt + C_TICKET0 + p, (uint32_t)(p + 1), cnt + C_ERR,
                       p + 1 < P ? U(W.hist) + (p + 1) * 256 : nullptr, HP.SB + 8 * (p + 1),
                       p == 0 ? ctab : nullptr, HP.ncells, HP.PB + HP.IVB,
                       (p > 0 || compact) ? cnt + C_TAIL : nullptr, p));
    if (p == 0 && P > 1) CK(launch_tail_sort(L, out, fin, nkeys, nsort, HP.SB + 8, P - 1, cnt + C_TAIL));
    std::swap(in, out);
    static const char* pn[8] = {"sort_pass0", "sort_pass1", "sort_pass2", "sort_pass3",
                                "sort_pass4", "sort_pass5", "sort_pass6", "sort_pass7"};
    g_prof.mark(pn[p & 7]);
  }
  // `in` holds the sorted keys; `out` is free for the candidate list
  const uint64_t cand_cap = W.cand_cap;
  CK(launch_candidates(L, in, W.key_words, nkeys, dprog, out, cand_cap, cnt, o && (o->flags & HGRD_SCAN_BALLOT)));
  if (split) CK(launch_shared_cand(L, HP, U(W.stbl), U(W.sbase), out, cand_cap, cnt));
  g_prof.mark("candidates");
  CK(launch_exact(L, in, nkeys, dprog, out, cand_cap, U(W.raw), W.raw_cap, cnt, o && (o->flags & HGRD_STOP_FIRST),
                  split));
  g_prof.mark("exact");
  // canonical order of the witnesses: up to WSMALL_MAX merged by one CTA in
  // shared memory, more by the device-wide radix sort and merge.  Outside a
  // stream capture the device-wide kernels run as the body of a conditional
  // graph node that the split kernel opens only when they have work;
  // otherwise they are launched and find nothing to do.
  uint64_t* wout = U(uniq_off(W));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cap));
  cudaGraphExec_t wg =
      (cap == cudaStreamCaptureStatusNone && !dprog_resident && !noalloc) ? witness_graph(L, W, ws, P) : nullptr;
  if (wg) {
    CK(cudaGraphLaunch(wg, s));
    (*L.launches)++;
  } else if (cc) {
    CK(capture_witness_cond(L, W, ws, P, *cc));
  } else {
    CK(launch_witness_split(L, cnt, W.raw_cap));
    CK(enqueue_witness_big(L, W, ws, P));
  }
  CK(launch_witness_small(L, U(W.raw), U(W.raw2), wout, cnt, W.raw_cap));
  g_prof.mark("witness_merge");
  if (pair && !(fl & HGRD_NO_PAIR)) {
    CK(enqueue_pair_search(L, d, o, W, ws, wout, dprog));
    g_prof.mark("pair_search");
  }
  return HGRD_OK;
}

// HGRD_GRAPH: one instantiated graph per (device, binding, workspace,
// options, expansion kernels, sort shape), captured by the first check and
// replayed by the later ones.  The cache holds at most CG_MAX graphs; past
// that, checks run uncaptured.
struct CheckGraph {
  cudaGraphExec_t exec = nullptr;
  DProg* pinned = nullptr;  // the program, pinned host copy
  DProg* dprog = nullptr;   // its device copy, which the graph's kernels read
  hgrd_stats stats{};       // what the captured enqueue reported
};
std::mutex g_cg_mu;
std::map<std::vector<uint64_t>, CheckGraph> g_cg;
constexpr size_t CG_MAX = 64;

int enqueue_graph(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, cudaStream_t s,
                  bool pair) {
  hgrd_check_opts oo = *o;
  oo.flags &= ~(uint32_t)HGRD_GRAPH;
  Layout W;
  int rc = prechecks(d, d_ws, ws_bytes, &oo, &W);
  if (rc) return rc;
  const Bound& B = *d->bound;
  // the decisions that shape the captured work, taken before the capture
  // (compiling and loading kernels is no stream work)
  const bool split = B.prog.smode && !(oo.flags & HGRD_NO_SPLIT);
  if ((oo.flags & HGRD_JIT) && !(oo.flags & HGRD_NO_JIT)) {
    rc = jit_prepare(B, split, nullptr);
    if (rc) return rc;
  }
  const bool jit = !(oo.flags & HGRD_NO_JIT) && jit_ready(B, split);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const std::vector<uint64_t> key = {(uint64_t)dev,         B.gen,           (uint64_t)(uintptr_t)d_ws,
                                     (uint64_t)ws_bytes,    oo.max_raw_witness, oo.pair_cap,
                                     oo.flags,              oo.only_accesses, oo.max_shared_keys,
                                     (uint64_t)jit,         sort_variant_key(), (uint64_t)pair};
  // The graph's kernels read the program from the graph's own device copy,
  // which stays resident between replays.  The synchronous check (`pair`)
  // copies it in from the pinned host copy before every replay, as one
  // self-contained check whose inputs cross the bus each call; the enqueue
  // path copies it once, when the graph is made.
  auto launch = [&](const CheckGraph& e, bool upload) -> int {
    g_stats = e.stats;
    if (upload) {
      CK(cudaMemcpyAsync(e.dprog, e.pinned, sizeof(DProg), cudaMemcpyHostToDevice, s));
      g_stats.h2d_bytes += sizeof(DProg);
    }
    note_ws_prog(d_ws, e.dprog);
    CK(cudaGraphLaunch(e.exec, s));
    return HGRD_OK;
  };
  {
    std::lock_guard<std::mutex> lk(g_cg_mu);
    auto it = g_cg.find(key);
    if (it != g_cg.end()) return launch(it->second, pair);
    if (g_cg.size() >= CG_MAX) return enqueue(d, &oo, d_ws, ws_bytes, s, nullptr, nullptr, pair);
  }
  CheckGraph e;
  cudaStream_t cs = nullptr, bs = nullptr;
  cudaGraph_t g = nullptr;
  note_created(5);  // pinned and device program copies, two capture streams, the instantiated graph
  bool ok = cudaHostAlloc((void**)&e.pinned, sizeof(DProg), cudaHostAllocDefault) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&e.dprog, sizeof(DProg)) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaGraphCreate(&g, 0) == cudaSuccess;
  ok = ok && cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  int erc = HGRD_OK;
  if (ok) {
    const Capture cc{g, e.pinned, e.dprog, bs};
    erc = enqueue(d, &oo, d_ws, ws_bytes, cs, nullptr, &cc, pair);
    cudaGraph_t out = nullptr;
    ok = cudaStreamEndCapture(cs, &out) == cudaSuccess && erc == HGRD_OK;
  }
  if (ok) {
    e.stats = g_stats;
    ok = cudaGraphInstantiate(&e.exec, g, 0) == cudaSuccess;
  }
  if (cs) cudaStreamDestroy(cs);
  if (bs) cudaStreamDestroy(bs);
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.pinned) cudaFreeHost(e.pinned);
    if (e.dprog) cudaFree(e.dprog);
    cudaGetLastError();  // a failed capture leaves no sticky error behind
    if (erc != HGRD_OK && erc != HGRD_EDEVICE) return erc;  // a real refusal of these options
    return enqueue(d, &oo, d_ws, ws_bytes, s, nullptr, nullptr, pair);  // no graph: the same check, launched directly
  }
  std::lock_guard<std::mutex> lk(g_cg_mu);
  auto it = g_cg.emplace(key, e).first;
  return launch(it->second, true);
}

// the public enqueue: captured / replayed as a graph on request; `pair`
// appends the canonical-pair search (the synchronous check wants it)
int enqueue_api(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, cudaStream_t s,
                bool pair = false) {
  if (o && (o->flags & HGRD_GRAPH) && !(o->flags & HGRD_PROFILE) && d && d->bound)
    return enqueue_graph(d, o, d_ws, ws_bytes, s, pair);
  if (o && (o->flags & HGRD_GRAPH)) {
    hgrd_check_opts oo = *o;
    oo.flags &= ~(uint32_t)HGRD_GRAPH;
    return enqueue(d, &oo, d_ws, ws_bytes, s, nullptr, nullptr, pair);
  }
  return enqueue(d, o, d_ws, ws_bytes, s, nullptr, nullptr, pair);
}

struct Inst {
  uint32_t blk, thr;
  uint32_t it[4];
  int acc;
  int64_t iv;
};
bool key_less(const Inst& a, const Inst& b) {
  return std::tie(a.blk, a.thr, a.it[0], a.it[1], a.it[2], a.it[3]) <
         std::tie(b.blk, b.thr, b.it[0], b.it[1], b.it[2], b.it[3]);
}

// Pinned host staging for the readbacks of collect, one per host thread,
// grown on demand (copies into it are DMA transfers; it is never freed: the
// process exit reclaims it, after which the CUDA runtime may be gone).
struct Pinned {
  char* p = nullptr;
  size_t n = 0;
  char* get(size_t need) {
    if (need <= n) return p;
    size_t m = std::max<size_t>(need, 1 << 20);
    void* q = nullptr;
    note_created();
    if (cudaHostAlloc(&q, m, cudaHostAllocDefault) != cudaSuccess) return nullptr;
    if (p) cudaFreeHost(p);
    p = (char*)q;
    n = m;
    return p;
  }
};
thread_local Pinned g_pin;
constexpr uint64_t WIT_PREFIX = 4096;   // witnesses fetched with the counters
constexpr uint64_t PAIR_PREFIX = 1024;  // pair-search records fetched with their count

int collect(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, cudaStream_t s,
            hgrd_witness* host_out, uint64_t cap, hgrd_verdict* v, bool want_pair, bool pair_enqueued = false) {
  Layout W;
  int rc = prechecks(d, d_ws, ws_bytes, o, &W);
  if (rc) return rc;
  if (!v) return fail(HGRD_EINVAL, "null verdict");
  if (cap && !host_out) return fail(HGRD_EINVAL, "null witness buffer with nonzero capacity");
  const Bound& B = *d->bound;
  const DProg& HP = B.prog;
  char* ws = (char*)d_ws;
  // counters and a prefix of the merged witnesses in one round trip
  const uint64_t* duniq = uniq_buffer(d, W, ws);
  const uint64_t wpre = std::min<uint64_t>(std::min<uint64_t>(std::max<uint64_t>(cap, 1), WIT_PREFIX), W.raw_cap);
  // with the pair search already enqueued, a prefix of its records too
  const uint64_t ppre = std::min<uint64_t>(PAIR_PREFIX, W.pair_cap);
  const size_t pair_at = C_WORDS * 8 + wpre * 8;
  char* stage = g_pin.get(pair_at + (pair_enqueued ? ppre * sizeof(PairRec) : 0));
  if (!stage) return fail(HGRD_ENOMEM, "pinned host staging buffer");
  CK(cudaMemcpyAsync(stage, ws + W.counters, C_WORDS * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(stage + C_WORDS * 8, duniq, wpre * 8, cudaMemcpyDeviceToHost, s));
  g_stats.d2h_bytes += C_WORDS * 8 + wpre * 8;
  if (pair_enqueued && want_pair && !(o && (o->flags & HGRD_NO_PAIR))) {
    CK(cudaMemcpyAsync(stage + pair_at, ws + W.pairs, ppre * sizeof(PairRec), cudaMemcpyDeviceToHost, s));
    g_stats.d2h_bytes += ppre * sizeof(PairRec);
  }
  CK(cudaStreamSynchronize(s));
  uint64_t cnt[C_WORDS];
  memcpy(cnt, stage, sizeof(cnt));
  // the pair records fetched with the counters, copied out before any later
  // readback regrows (and so frees) the staging buffer
  std::vector<PairRec> pair_pre;
  if (pair_enqueued && want_pair && !(o && (o->flags & HGRD_NO_PAIR))) {
    pair_pre.resize(std::min<uint64_t>(cnt[C_NPAIR], ppre));
    memcpy(pair_pre.data(), stage + pair_at, pair_pre.size() * sizeof(PairRec));
  }
  // more per-run witnesses than the one-CTA path keeps: run the device-wide
  // pipeline, unless the caller wants the first races only (those kept are
  // real races, and there is at least one)
  if ((cnt[C_ERR] & ERR_SMALL_FULL) && !(o && (o->flags & HGRD_STOP_FIRST))) {
    hgrd_check_opts o2 = o ? *o : hgrd_check_opts{};
    o2.flags |= HGRD_NO_SMALL;
    o2.flags &= ~(uint32_t)HGRD_GRAPH;
    const int r2 = enqueue(d, &o2, d_ws, ws_bytes, s, nullptr, nullptr, pair_enqueued);
    if (r2) return r2;
    return collect(d, &o2, d_ws, ws_bytes, s, host_out, cap, v, want_pair, pair_enqueued);
  }
  if (cnt[C_ERR] & ERR_TIMEOUT) return fail(HGRD_ETIMEOUT, "a bounded device wait (sort look-back) gave up");
  if (cnt[C_ERR] & ERR_LOCK_RUN)
    return fail(HGRD_EUNSUPPORTED, "acquire-release guards with varying elements on a location with more than " +
                                       std::to_string(LOCK_RUN_MAX) + " keys");
  g_stats.n_candidates = cnt[C_NCAND];
  {
    const uint32_t fl = o ? o->flags : 0u;
    const int passes = (d->bound->prog.smode && !(fl & HGRD_NO_SPLIT)) ? d->bound->sort_passes_split
                                                                       : d->bound->sort_passes;
    const bool cf = filter_runs(W, passes) && !g_stats.small;
    g_stats.n_sorted_keys = cf ? cnt[C_NGC] : cnt[C_NG];
    g_stats.n_written_keys = g_stats.small ? 0 : cnt[C_NG];
    g_stats.cell_filter = cf ? 1u : 0u;
  }
  g_stats.n_binned_keys = g_stats.shared_bins ? cnt[C_NSC] : 0;
  g_stats.n_raw_witness = cnt[C_NRAW];
  if (cnt[C_ERR] & ERR_SHARED_FULL)
    return fail(HGRD_ENOMEM, "room for keys of candidate shared-memory bins too small: need " +
                                 std::to_string(cnt[C_NSC]) + " (hgrd_check_opts.max_shared_keys)");
  if (cnt[C_NCAND] > W.cand_cap) return fail(HGRD_EUNSUPPORTED, "candidate list overflow");
  if (cnt[C_NRAW] > W.raw_cap)
    return fail(HGRD_ENOMEM, "raw witness buffer too small: need " + std::to_string(cnt[C_NRAW]) +
                                 " (hgrd_check_opts.max_raw_witness)");
  memset(v, 0, sizeof(*v));
  v->n_instances = B.n_instances;
  v->n_keys = cnt[C_NKEYS];
  v->n_oob = cnt[C_NOOB];
  v->n_witness = cnt[C_NUNIQ];
  v->n_by_kind[0] = cnt[C_KIND0];
  v->n_by_kind[1] = cnt[C_KIND1];
  v->n_by_kind[2] = cnt[C_KIND2];
  v->racy = v->n_witness > 0;
  for (int k = 0; k < 3; k++)
    for (int a = 0; a < 32; a++) v->pair_kind[k][a] = (uint32_t)(cnt[C_PAIRS + k * 16 + a / 2] >> (32 * (a & 1)));
  const uint64_t ncopy = std::min<uint64_t>(std::max<uint64_t>(cap, 1), v->n_witness);
  std::vector<uint64_t> hw(ncopy);
  memcpy(hw.data(), stage + C_WORDS * 8, std::min(ncopy, wpre) * 8);
  if (ncopy > wpre) {  // the rest of the requested witnesses
    char* rest = g_pin.get((ncopy - wpre) * 8);
    if (!rest) return fail(HGRD_ENOMEM, "pinned host staging buffer");
    CK(cudaMemcpyAsync(rest, duniq + wpre, (ncopy - wpre) * 8, cudaMemcpyDeviceToHost, s));
    g_stats.d2h_bytes += (ncopy - wpre) * 8;
    CK(cudaStreamSynchronize(s));
    memcpy(hw.data() + wpre, rest, (ncopy - wpre) * 8);
  }
  auto unpack = [&](uint64_t w) {
    hgrd_witness x{};
    x.space = (uint8_t)((w >> 58) & 1);
    x.array = (uint8_t)((w >> 53) & 31);
    const uint64_t gran = (w >> 13) & ((1ull << 40) - 1);
    x.acc_lo = (uint8_t)((w >> 8) & 31);
    x.acc_hi = (uint8_t)((w >> 3) & 31);
    x.kind_mask = (uint8_t)(w & 7);
    x.byte_addr = gran * (uint64_t)B.array_granule[x.array];
    return x;
  };
  for (uint64_t k = 0; k < std::min<uint64_t>(cap, v->n_witness); k++) host_out[k] = unpack(hw[k]);
  if (v->racy) v->min_w = unpack(hw[0]);

  if (v->racy && want_pair && !(o && (o->flags & HGRD_NO_PAIR))) {
    // canonical instance pair: gather the instances of acc_lo / acc_hi on the
    // minimal witness's granule, then take the smallest racing (x, y)
    PairRec* pr = (PairRec*)(ws + W.pairs);
    if (!pair_enqueued) {
      Launch L{s, nsm_of_current_device(), &g_stats.kernel_launches};
      CK(enqueue_pair_search(L, d, o, W, ws, duniq, ws_prog(ws, (const DProg*)(ws + W.prog))));
    }
    // the record count and a prefix of the records in one round trip (made
    // already, with the counters, when the search ran in the enqueue)
    uint64_t np = 0;
    const char* pre = nullptr;
    if (pair_enqueued) {
      np = cnt[C_NPAIR];
      pre = (const char*)pair_pre.data();
    } else {
      char* pst = g_pin.get(16 + ppre * sizeof(PairRec));
      if (!pst) return fail(HGRD_ENOMEM, "pinned host staging buffer");
      CK(cudaMemcpyAsync(pst, ws + W.counters + 8 * C_NPAIR, 8, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(pst + 16, pr, ppre * sizeof(PairRec), cudaMemcpyDeviceToHost, s));
      g_stats.d2h_bytes += 8 + ppre * sizeof(PairRec);
      CK(cudaStreamSynchronize(s));
      memcpy(&np, pst, 8);
      pre = pst + 16;
    }
    if (np <= W.pair_cap) {
      std::vector<PairRec> recs(np);
      memcpy(recs.data(), pre, std::min(np, ppre) * sizeof(PairRec));
      if (np > ppre) {
        char* rest = g_pin.get((np - ppre) * sizeof(PairRec));
        if (!rest) return fail(HGRD_ENOMEM, "pinned host staging buffer");
        CK(cudaMemcpyAsync(rest, pr + ppre, (np - ppre) * sizeof(PairRec), cudaMemcpyDeviceToHost, s));
        g_stats.d2h_bytes += (np - ppre) * sizeof(PairRec);
        CK(cudaStreamSynchronize(s));
        memcpy(recs.data() + ppre, rest, (np - ppre) * sizeof(PairRec));
      }
      std::vector<Inst> X, Y;
      for (auto& r : recs) {
        Inst in{r.blk, r.thr, {r.it[0], r.it[1], r.it[2], r.it[3]}, r.acc, r.iv};
        if (r.acc == v->min_w.acc_lo) X.push_back(in);
        if (r.acc == v->min_w.acc_hi) Y.push_back(in);
      }
      std::sort(X.begin(), X.end(), key_less);
      std::sort(Y.begin(), Y.end(), key_less);
      const int lo = v->min_w.acc_lo, hi = v->min_w.acc_hi;
      const uint32_t allow = ((HP.einter[lo] >> hi) & 1u) | (((HP.eintra[lo] >> hi) & 1u) ? 6u : 0u);
      const bool shared = v->min_w.space == HGRD_SPACE_SHARED;
      bool found = false;
      for (size_t i = 0; i < X.size() && !found; i++)
        for (size_t j = 0; j < Y.size(); j++) {
          const Inst &x = X[i], &y = Y[j];
          if (lo == hi && !key_less(x, y)) continue;
          // recorded intervals carry the warp interval in their low WVB bits
          const int64_t ivx = (x.iv - HP.ivmin) >> HP.WVB, ivy = (y.iv - HP.ivmin) >> HP.WVB;
          uint32_t kind = 0;
          if (x.blk == y.blk && x.thr == y.thr) kind = 0;
          else if (x.blk != y.blk) kind = shared ? 0 : 1;
          else if (ivx != ivy) kind = 0;
          else if (x.thr / 32 != y.thr / 32) kind = 2;
          else kind = x.iv == y.iv ? 4 : 0;  // same warp: ordered by a warp barrier unless one interval
          if ((kind & allow) && ((HP.lockpair[lo] >> hi) & 1u)) {
            // guards decided per instance: ordered when both hold one element
            // and the narrower scope covers the kind (device across blocks)
            const uint64_t gran = v->min_w.byte_addr / (uint64_t)B.array_granule[v->min_w.array];
            auto elem = [&](int a, const Inst& s2) -> int64_t {
              const DLock& Lk = HP.lock[a];
              if (Lk.form == LOCK_OWN) return (int64_t)(gran / (uint64_t)HP.acc[a].G);
              const int64_t t = s2.thr, b = s2.blk;
              const int64_t tx = t % HP.block[0], ty = (t / HP.block[0]) % HP.block[1], tz = t / (HP.block[0] * HP.block[1]);
              const int64_t bx = b % HP.grid[0], by = (b / HP.grid[0]) % HP.grid[1], bz = b / (HP.grid[0] * HP.grid[1]);
              return Lk.c0 + Lk.c[0] * tx + Lk.c[1] * ty + Lk.c[2] * tz + Lk.c[3] * bx + Lk.c[4] * by + Lk.c[5] * bz;
            };
            if (HP.lock[lo].arr == HP.lock[hi].arr && elem(lo, x) == elem(hi, y) &&
                (kind != 1 || std::min(HP.lock[lo].scope, HP.lock[hi].scope) == 1))
              kind = 0;
          }
          if (kind & allow) {
            auto put = [](hgrd_inst& o2, const Inst& s2) {
              o2.lin_block = s2.blk;
              o2.lin_thread = s2.thr;
              for (int l = 0; l < 4; l++) o2.iter[l] = s2.it[l];
              o2.access = (uint8_t)s2.acc;
            };
            put(v->min_x, x);
            put(v->min_y, y);
            found = true;
            break;
          }
        }
      v->pair_found = found;
    }
  }
  return (host_out && v->n_witness > cap) ? HGRD_ETRUNCATED : HGRD_OK;
}

}  // namespace

// entry points for the batched path (batch.cu)
size_t item_workspace_bytes(const Bound& B, const hgrd_check_opts* o) { return layout(B, o).total; }

int item_enqueue(const hgrd_desc* d, const hgrd_check_opts* o, void* ws, size_t bytes, cudaStream_t s,
                 const DProg* dprog_resident, uint64_t** counters, const uint64_t** uniq, uint64_t* raw_cap,
                 uint64_t* cand_cap) {
  int rc = enqueue(d, o, ws, bytes, s, dprog_resident);
  if (rc) return rc;
  const Layout W = layout(*d->bound, o);
  *counters = (uint64_t*)((char*)ws + W.counters);
  *uniq = uniq_buffer(d, W, (char*)ws);
  *raw_cap = W.raw_cap;
  *cand_cap = W.cand_cap;
  return HGRD_OK;
}

}  // namespace hgrd

using namespace hgrd;

extern "C" {

int hgrd_workspace_size(const hgrd_desc* d, const hgrd_check_opts* o, size_t* bytes) {
  hgrd_check_opts tmp;
  o = norm_opts(o, &tmp);
  if (!d || !bytes) return fail(HGRD_EINVAL, "null argument");
  if (!d->bound) return fail(HGRD_EINVAL, "descriptor is not bound");
  *bytes = layout(*d->bound, o).total;
  return HGRD_OK;
}

int hgrd_last_profile(hgrd_stage_time* out, uint32_t cap, uint32_t* n) {
  if (!n || (cap && !out)) return fail(HGRD_EINVAL, "null argument");
  Prof& p = g_prof;
  const uint32_t stages = p.ev.empty() ? 0 : (uint32_t)p.ev.size() - 1;
  *n = stages;
  if (!stages) return HGRD_OK;
  if (cudaEventSynchronize(p.ev.back()) != cudaSuccess) return fail(HGRD_EDEVICE, "event synchronize failed");
  for (uint32_t k = 0; k < stages && k < cap; k++) {
    memset(out[k].name, 0, sizeof(out[k].name));
    strncpy(out[k].name, p.names[k + 1].c_str(), sizeof(out[k].name) - 1);
    float ms = 0;
    cudaEventElapsedTime(&ms, p.ev[k], p.ev[k + 1]);
    out[k].ms = ms;
  }
  return HGRD_OK;
}

int hgrd_check_enqueue(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, void* stream) {
  hgrd_check_opts tmp;
  o = norm_opts(o, &tmp);
  return enqueue_api(d, o, d_ws, ws_bytes, (cudaStream_t)stream);
}

int hgrd_check_collect(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, void* stream,
                       hgrd_witness* host_out, uint64_t cap, hgrd_verdict* v) {
  hgrd_check_opts tmp;
  o = norm_opts(o, &tmp);
  return collect(d, o, d_ws, ws_bytes, (cudaStream_t)stream, host_out, cap, v, false);
}

int hgrd_check(const hgrd_desc* d, const hgrd_check_opts* o, void* d_ws, size_t ws_bytes, void* stream,
               hgrd_witness* host_out, uint64_t cap, hgrd_verdict* v) {
  hgrd_check_opts tmp;
  o = norm_opts(o, &tmp);
  int rc = enqueue_api(d, o, d_ws, ws_bytes, (cudaStream_t)stream, true);
  if (rc) return rc;
  return collect(d, o, d_ws, ws_bytes, (cudaStream_t)stream, host_out, cap, v, true, true);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// hgrd_check_noalloc: the same check with the workspace taken from a fixed
// device array compiled into this library, for callers that cannot allocate
// device memory themselves: code that runs while another component owns all
// device memory (a caching allocator or a memory pool that must not be
// bypassed), code called from inside such an allocator, or embedders that
// have no access to cudaMalloc.  The array exists once per device that loads
// the library and lives until the process exits.
#include <mutex>

namespace hgrd {
namespace {

constexpr size_t NOALLOC_BYTES = 64ull << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_ws[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;

// Device address of the array for the current device.  In host code the
// symbol is only a stand-in, so the address is looked up once per device,
// with that device current, and kept.
int noalloc_base(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HGRD_EDEVICE, std::string("CUDA: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(HGRD_EUNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess || !p)
      return fail(HGRD_EDEVICE, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return HGRD_OK;
}

}  // namespace
}  // namespace hgrd

extern "C" int hgrd_check_noalloc(const hgrd_desc* d, const hgrd_check_opts* o, void* stream,
                                  hgrd_witness* host_out, uint64_t cap, hgrd_verdict* v) {
  if (!d || !v) return fail(HGRD_EINVAL, "null argument");
  if (cap && !host_out) return fail(HGRD_EINVAL, "null witness buffer with nonzero capacity");
  if (!d->bound) return fail(HGRD_EINVAL, "descriptor is not bound (call hgrd_bind_host_params)");
  {
    // the readbacks below synchronise the stream, which a capture forbids
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess) return fail(HGRD_EDEVICE, std::string("CUDA: ") + cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
      return fail(HGRD_EINVAL, "hgrd_check_noalloc cannot run on a capturing stream (it reads results back)");
  }
  hgrd_check_opts oo{};
  if (o) oo = *o;
  if (oo.flags & HGRD_ALL_KEYS) oo.flags |= HGRD_NO_SPLIT;
  oo.flags &= ~(uint32_t)HGRD_PROFILE;  // stage timing would create CUDA events
  oo.flags &= ~(uint32_t)HGRD_JIT;      // loading a compiled module takes device memory
  oo.flags |= HGRD_NO_JIT | HGRD_NO_SMALL | HGRD_NO_CELL_FILTER;  // smallest workspace
  oo.flags &= ~(uint32_t)HGRD_GRAPH;  // the capture would allocate host and device resources
  const Layout W = layout(*d->bound, &oo);
  if (W.total > NOALLOC_BYTES)
    return fail(HGRD_ENOMEM, "hgrd_check_noalloc: this binding needs " + std::to_string(W.total) +
                                 " bytes of scratch; the built-in array holds " + std::to_string(NOALLOC_BYTES) +
                                 " (use hgrd_check with a caller workspace)");
  void* base = nullptr;
  int rc = noalloc_base(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = enqueue(d, &oo, base, NOALLOC_BYTES, s, nullptr, nullptr, false, true);
  if (rc) return rc;
  char* ws = (char*)base;
  uint64_t cnt[C_WORDS];
  CK(cudaMemcpyAsync(cnt, ws + W.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (cnt[C_ERR] & ERR_TIMEOUT) return fail(HGRD_ETIMEOUT, "a bounded device wait (sort look-back) gave up");
  if (cnt[C_ERR] & ERR_LOCK_RUN)
    return fail(HGRD_EUNSUPPORTED, "acquire-release guards with varying elements on a location with more than " +
                                       std::to_string(LOCK_RUN_MAX) + " keys");
  if (cnt[C_ERR] & ERR_SHARED_FULL)
    return fail(HGRD_ENOMEM, "room for keys of candidate shared-memory bins too small: need " +
                                 std::to_string(cnt[C_NSC]) + " (hgrd_check_opts.max_shared_keys)");
  if (cnt[C_NCAND] > W.cand_cap) return fail(HGRD_EUNSUPPORTED, "candidate list overflow");
  if (cnt[C_NRAW] > W.raw_cap)
    return fail(HGRD_ENOMEM, "raw witness buffer too small: need " + std::to_string(cnt[C_NRAW]) +
                                 " (hgrd_check_opts.max_raw_witness)");
  const Bound& B = *d->bound;
  memset(v, 0, sizeof(*v));
  v->n_instances = B.n_instances;
  v->n_keys = cnt[C_NKEYS];
  v->n_oob = cnt[C_NOOB];
  v->n_witness = cnt[C_NUNIQ];
  v->n_by_kind[0] = cnt[C_KIND0];
  v->n_by_kind[1] = cnt[C_KIND1];
  v->n_by_kind[2] = cnt[C_KIND2];
  v->racy = v->n_witness > 0;
  for (int k = 0; k < 3; k++)
    for (int a = 0; a < 32; a++) v->pair_kind[k][a] = (uint32_t)(cnt[C_PAIRS + k * 16 + a / 2] >> (32 * (a & 1)));
  auto unpack = [&](uint64_t w) {
    hgrd_witness x{};
    x.space = (uint8_t)((w >> 58) & 1);
    x.array = (uint8_t)((w >> 53) & 31);
    x.acc_lo = (uint8_t)((w >> 8) & 31);
    x.acc_hi = (uint8_t)((w >> 3) & 31);
    x.kind_mask = (uint8_t)(w & 7);
    x.byte_addr = ((w >> 13) & ((1ull << 40) - 1)) * (uint64_t)B.array_granule[x.array];
    return x;
  };
  const uint64_t* duniq = uniq_buffer(d, W, ws);
  if (v->racy) {
    uint64_t w0 = 0;
    CK(cudaMemcpyAsync(&w0, duniq, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    v->min_w = unpack(w0);
  }
  // the packed 8-byte words land in the caller's 16-byte records and are
  // widened in place from the back, so no host staging buffer is needed
  const uint64_t n = std::min<uint64_t>(cap, v->n_witness);
  if (n) {
    CK(cudaMemcpyAsync(host_out, duniq, n * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t* packed = (const uint64_t*)host_out;
    for (uint64_t k = n; k-- > 0;) {
      const uint64_t w = packed[k];
      host_out[k] = unpack(w);
    }
  }
  return (host_out && v->n_witness > cap) ? HGRD_ETRUNCATED : HGRD_OK;
}
