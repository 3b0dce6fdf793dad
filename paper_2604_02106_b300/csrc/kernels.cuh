// Launch wrappers of the check pipeline's kernels (all enqueue only).
#pragma once
#include <cuda_runtime.h>

#include "hgrd_internal.h"

namespace hgrd {

// Work shapes
constexpr int RS_MIN_TILE = 1536;  // smallest onesweep tile of the shapes the sort autotuner picks from
constexpr int RS_RADIX = 256;
constexpr int CA_THREADS = 256;    // candidate scan
constexpr int CA_LONG = 1 << 16;   // a run longer than this is handed to the exact scan unmeasured
constexpr int CA_RANGE = 2048;     // keys owned by one warp of the candidate scan
constexpr int CA_AHEAD = 4;        // 32-key steps loaded ahead by each warp
constexpr int SCAN_TILE = 1024;               // values per CTA of the exclusive scans
constexpr int SCAN_PER = SCAN_TILE / 256;     // per thread (256 threads)
constexpr int MAX_PASSES = 16;

// cached per device: raise a kernel's dynamic shared-memory limit to at least
// smem (once), and its resident CTAs per SM for a launch shape
cudaError_t allow_smem(const void* fn, size_t smem);
int resident_ctas(const void* fn, int threads, size_t smem);

struct Launch {
  cudaStream_t s;
  int nsm;
  uint64_t* launches;  // incremented per kernel enqueued
};

// expansion: mode 0 = count keys per unit + digit histograms + out-of-bounds,
// 1 = write keys, 2 = gather the instances of the minimal witness
// (mode 1 with cbuf: keys of the cells the filter table ctab keeps are also
// appended to cbuf[0, ccap), their count in counters[C_NCOMPACT])
cudaError_t launch_expand(const Launch& L, int mode, bool wide, const DProg* d_prog, const DProg& h_prog,
                          uint64_t* unit_cnt, const uint64_t* unit_off, uint64_t* keys, uint64_t* hist, int npass,
                          uint64_t* counters, const uint64_t* uniq, PairRec* pairs, uint64_t pair_cap,
                          const uint32_t* ctab = nullptr, uint64_t* cbuf = nullptr, uint64_t ccap = 0);

// exclusive scan of uint64 values; n = min(*n_dev, n_max) when n_dev is given
cudaError_t launch_scan(const Launch& L, const uint64_t* in, uint64_t* out, const uint64_t* n_dev, uint64_t n_max,
                        uint64_t* partials, uint64_t* total);

// histograms of npass 8-bit digits starting at bit `shift0` of n keys
cudaError_t launch_histogram(const Launch& L, const uint64_t* keys, const uint64_t* n_dev, uint64_t n_max, int shift0,
                             int npass, uint64_t* hist);
// cell filter: the first pass's digit histogram (at `shift`, added to hist)
// of the keys [0, *n_dev) whose cell (key >> rsh) the count pass found
// written and touched by two threads, and their count (added to *n_kept);
// it also clears the look-back status words the first sort pass over those
// keys uses (at most max_words); nothing when *skip is set
cudaError_t launch_cell_hist(const Launch& L, const uint64_t* keys, const uint64_t* n_dev, uint64_t n_max,
                             const uint32_t* tab, uint64_t ncells, int rsh, uint64_t* hist, int shift,
                             uint64_t* n_kept, uint64_t* status, uint64_t max_words, const uint64_t* skip = nullptr);
// one stable onesweep pass on the digit at `shift`, given the pass's 256
// digit counts (each CTA scans them into the digits' starts); when next_hist
// is given, also counts the digit at `next_shift` for the following pass;
// with a cell table, only the keys the cell filter keeps are sorted (to
// out[0, kept))
cudaError_t launch_onesweep(const Launch& L, const uint64_t* in, uint64_t* out, const uint64_t* n_dev, uint64_t n_max,
                            int shift, const uint64_t* dcount, uint64_t* status, uint64_t* ticket, uint32_t epoch,
                            uint64_t* err, uint64_t* next_hist = nullptr, int next_shift = 0,
                            const uint32_t* ctab = nullptr, uint64_t ncells = 0, int rsh = 0,
                            const uint64_t* skip = nullptr, int pass = -1);
// the sort shapes in force on the current device (the device's shape and the
// per-pass choices), as one number for cache keys
uint64_t sort_variant_key();
// the passes after the first over the digits from shift0 (npass of them) in
// one CTA when at most 4096 keys remain; sets *done then (the passes given
// `skip` = done return at once; so does this one when *done is set already)
constexpr int TAIL_KEYS = 4096;
cudaError_t launch_tail_sort(const Launch& L, const uint64_t* in, uint64_t* out, const uint64_t* n_dev, uint64_t n_max,
                             int shift0, int npass, uint64_t* done);
// compact form: the whole sort of the write pass's compact buffer by one CTA,
// when all *n_dev keys it counted are there (at most n_max <= TAIL_KEYS);
// writes their count to *kept_out and sets *done
cudaError_t launch_compact_sort(const Launch& L, const uint64_t* in, uint64_t* out, const uint64_t* n_dev,
                                uint64_t n_max, uint64_t* done, uint64_t* kept_out);

// conflict scan, phase A: runs that may hold a race -> (start, end) list.
// keys holds key_cap words (a multiple of 16 for the row form, which reads
// whole rows of 16 keys); ballot = the 32-key warp-step form
cudaError_t launch_candidates(const Launch& L, const uint64_t* keys, uint64_t key_cap, const uint64_t* n_dev,
                              const DProg* d_prog, uint64_t* cand, uint64_t cand_cap, uint64_t* counters,
                              bool ballot = false);
// conflict scan, phase B: exact per-access summaries -> packed raw witnesses
cudaError_t launch_exact(const Launch& L, const uint64_t* keys, const uint64_t* n_dev, const DProg* d_prog,
                         const uint64_t* cand, uint64_t cand_cap, uint64_t* raw, uint64_t raw_cap,
                         uint64_t* counters, bool stop_first = false, bool bins = false);

// block-local mode (DProg::smode): mode 3 = count global keys per unit and
// summarise the shared bins of every block, 4 = write global keys and the
// keys of candidate bins (behind the *n_global sorted keys, in keys_s)
cudaError_t launch_expand_block(const Launch& L, int mode, bool wide, const DProg* d_prog, const DProg& h_prog,
                                uint64_t* unit_cnt, const uint64_t* unit_off, uint64_t* keys_g, uint64_t* keys_s,
                                uint64_t* hist, uint64_t* counters, uint64_t* stbl, uint64_t* sbase);
// candidate bins -> exact-scan entries appended to the candidate list
cudaError_t launch_shared_cand(const Launch& L, const DProg& h_prog, const uint64_t* stbl, const uint64_t* sbase,
                               uint64_t* cand, uint64_t cand_cap, uint64_t* counters);

// witness merge: head flags, merge by atomic OR into uniq, kind counts
cudaError_t launch_heads(const Launch& L, const uint64_t* w, const uint64_t* n_dev, uint64_t n_max, uint64_t* flags);
cudaError_t launch_merge(const Launch& L, const uint64_t* w, const uint64_t* flags, const uint64_t* excl,
                         const uint64_t* n_dev, uint64_t n_max, uint64_t* uniq);
// (kind counts of a device-wide merge; *gate = 0 means the one-CTA merge ran and counted them)
cudaError_t launch_kind_counts(const Launch& L, const uint64_t* uniq, uint64_t* counters, const uint64_t* gate);
// pair search: the blocks of a global-memory witness's run in the sorted keys
// (counters[C_NPB] = 1 + their count, or left 0 when every unit must be searched)
cudaError_t launch_pair_blocks(const Launch& L, const uint64_t* keys, const uint64_t* n_dev, const DProg* d_prog,
                               const uint64_t* uniq, uint64_t* counters, uint64_t* blocks);
// at most WSMALL_MAX raw witnesses are merged by witness_small: witness_split
// sets counters[C_NRAWBIG] (0 in that case, else the count) for the
// device-wide kernels
constexpr int WSMALL_MAX = 4096;
cudaError_t launch_witness_split(const Launch& L, uint64_t* counters, uint64_t raw_cap);
// the split kernel for a graph: (counters, raw_cap, conditional handle) opens
// the handle's node when the device-wide merge has work
const void* witness_split_cond_fn();
// the split kernel of the conditional witness merge, launched on a stream
// that is being captured into the graph owning h
cudaError_t launch_witness_split_cond(const Launch& L, uint64_t* counters, uint64_t raw_cap,
                                      cudaGraphConditionalHandle h);
// the onesweep CTA shape in use on the current device
int sort_variant_current();
// witness_small: the few raw words sorted by rank across the GPU into
// `sorted` (room for min(n, WSMALL_MAX) words), then merged by one CTA into
// `uniq`, which may be `raw`
cudaError_t launch_witness_small(const Launch& L, const uint64_t* raw, uint64_t* sorted, uint64_t* uniq,
                                 uint64_t* counters, uint64_t raw_cap);
// zero the look-back status words of the tiles a sort of *n_dev keys uses
// (at most max_words)
cudaError_t launch_zero_status(const Launch& L, uint64_t* status, const uint64_t* n_dev, uint64_t max_words);
// zero the first min(*n_dev, n_max) words of p
cudaError_t launch_zero(const Launch& L, uint64_t* p, const uint64_t* n_dev, uint64_t n_max);

}  // namespace hgrd
