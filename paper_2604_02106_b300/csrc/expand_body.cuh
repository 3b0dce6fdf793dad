// Bodies of the expansion kernels.  Two kinds of kernels run them:
//   interpreted  (kernels.cu) the compiled affine program is staged in shared
//                memory and evaluated term by term (expand_unit);
//   specialised  (jit.cpp) source generated from the program's structure and
//                compiled at run time: every guard, index and interval becomes
//                straight-line code over registers, the coefficients are read
//                from the kernel's parameter block.
// Both hand a unit expander X to the same bodies, so the keys, counts and bins
// they produce are the same by construction.  X provides
//   template <int SEL, class Step> uint64_t unit(int lane, int64_t u, uint32_t only, Step&& step)
// with expand_unit's contract (step called per access and loop vector with a
// live in-bounds lane in the warp; returns this lane's out-of-bounds
// instances), over the accesses in `only` and in the set SEL names:
//   SEL_ALL every access; SEL_KEPT accesses whose keys are written (emask);
//   SEL_KEPT_GLOBAL those of them on global arrays.
// step's last argument `mult` (at least 1) says how many identical instances
// the call stands for: the specialised count pass evaluates an access whose
// guards, index and interval do not depend on the loop counters once per unit
// and hands over all the unit's loop vectors at once (the keys, counts and
// bins are those of mult calls with 1); the other callers always pass 1.
// The specialised expander fixes SEL's set at compile time, so work only
// the other accesses need (their ops, guards, indexes) is never emitted.
// X also provides unit_once(lane, u, only, step), the same walk for a count
// pass, where an expander may take loop-invariant accesses once per unit
// with mult > 1, and unit_combine(lane, u, only, step, flush), the same for
// the block-local count pass, where it may also hand the instances of a
// shared-array access with one granule per instance to
//   flush(a, bin, count, lt)
// instead of step: `count` instances of thread lt on (granule, interval) bin
// `bin`, combined while consecutive instances of the access stay in one bin.
// The bin's count, min / max thread and writer bit end up the same.
#pragma once
#include "kcommon.cuh"

namespace hgrd {
namespace dev {

// Cell filter (count pass): note that (block << TB | thread) `gid` touched
// cell c, as a writer or not.  One word per cell: 0 = untouched; otherwise
// bit 31 = a writer touched it and bits 0..30 = gid + 1 of the one id seen so
// far, or CELL_MANY once two different ids were seen.  The word only moves
// forward (untouched -> one id -> many, writer bit 0 -> 1), so the
// compare-and-swap loop ends after at most three changes by other threads;
// the first note of a cell is one CAS.  Idempotent, so multiplicities need
// no care.  gid + 1 < CELL_MANY holds because gid has at most 30 bits.
constexpr uint32_t CELL_MANY = 0x7fffffffu, CELL_W = 0x80000000u;
__device__ __forceinline__ void cell_note(uint32_t* tab, uint64_t c, uint32_t gid, bool w) {
  const uint32_t me = (gid + 1u) | (w ? CELL_W : 0u);
  uint32_t old = atomicCAS(&tab[c], 0u, me);
  while (old != 0u) {
    const uint32_t id = (old & CELL_MANY) == gid + 1u ? gid + 1u : CELL_MANY;
    const uint32_t nv = id | ((old | me) & CELL_W);
    if (nv == old) break;
    const uint32_t prev = atomicCAS(&tab[c], old, nv);
    if (prev == old) break;
    old = prev;
  }
}

// A key is kept for the sort when its cell saw a writer and two different
// (block, thread) ids (only such a cell can hold a race); cells past the
// table (shared memory) are always kept.
__device__ __forceinline__ bool cell_kept(const uint32_t* __restrict__ tab, uint64_t ncells, uint64_t c) {
  return c >= ncells || tab[c] == (CELL_MANY | CELL_W);
}

enum { SEL_ALL = 0, SEL_KEPT = 1, SEL_KEPT_GLOBAL = 2 };

// Modes 0 (count keys per unit + digit histograms of `npass` digits), 1 (write
// keys at the unit offsets; with `cbuf`, keys of the cells the filter table
// `ctab` keeps are also appended to cbuf[0, ccap), their count in
// counters[C_NCOMPACT]) and 2 (gather the instances of the minimal witness's
// granule).  Warp = unit, grid-stride over units; mode 2 visits
// only the units of the blocks unit_off lists when counters[C_NPB] = 1 + their
// count.  shist: npass x 256 words of shared memory (mode 0).
template <typename T, int MODE, class X>
__device__ __forceinline__ void expand_units_body(const DProg* __restrict__ P, X& ex, uint32_t* shist,
                                                  uint64_t* __restrict__ unit_cnt,
                                                  const uint64_t* __restrict__ unit_off, uint64_t* __restrict__ keys,
                                                  uint64_t* __restrict__ hist, int npass, uint64_t* __restrict__ counters,
                                                  const uint64_t* __restrict__ uniq, PairRec* __restrict__ pairs,
                                                  uint64_t pair_cap, uint32_t only_in,
                                                  const uint32_t* __restrict__ ctab = nullptr,
                                                  uint64_t* __restrict__ cbuf = nullptr, uint64_t ccap = 0) {
  constexpr int WPC = EXP_THREADS / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (MODE == 0) {
    for (int i = threadIdx.x; i < npass * 256; i += EXP_THREADS) shist[i] = 0;
    __syncthreads();
  }
  // the minimal witness for the pair search
  uint32_t t_arr = 0, t_lo = 0, t_hi = 0;
  uint64_t t_gran = 0;
  if (MODE == 2) {
    if (counters[C_NUNIQ] == 0) return;
    const uint64_t w0 = uniq[0];
    t_arr = (uint32_t)(w0 >> 53) & 31;
    t_gran = (w0 >> 13) & ((1ull << 40) - 1);
    t_lo = (uint32_t)(w0 >> 8) & 31;
    t_hi = (uint32_t)(w0 >> 3) & 31;
  }
  const int64_t nunits = P->nunits;
  const int SB = P->SB;  // lowest sorted key bit
  const uint32_t emask = ex.emask_of(P);  // a constant in the specialised kernels
  uint64_t oob = 0, drop = 0;
  const uint32_t only = MODE == 2 ? ((1u << t_lo) | (1u << t_hi)) : only_in;
  if (MODE == 1 && blockIdx.x == 0 && threadIdx.x == 0) counters[C_NKEYS] = counters[C_NG] + counters[C_NDROP];
  const uint64_t npb = MODE == 2 ? counters[C_NPB] : 0;
  const int64_t upb = (int64_t)P->wpb * P->nchunk;
  const int64_t nvisit = npb ? (int64_t)(npb - 1) * upb : nunits;
  for (int64_t j = (int64_t)blockIdx.x * WPC + warp; j < nvisit; j += (int64_t)gridDim.x * WPC) {
    const int64_t u = npb ? (int64_t)unit_off[j / upb] * upb + j % upb : j;
    uint64_t cursor = (MODE == 1) ? unit_off[u] : 0;
    // the write pass expands only the accesses whose keys are kept
    auto step = [&](int a, const DAcc& A, bool inb, unsigned bal, int64_t idx, int64_t iv, int64_t b, int lt,
                       const int32_t* ic, uint32_t mult) {
                     const int G = A.G;
                     if (MODE == 2) {
                       if (inb) {
                         const uint64_t g0 = (uint64_t)idx * (uint64_t)G;
                         if ((uint32_t)A.arr == t_arr && t_gran >= g0 && t_gran < g0 + (uint64_t)G) {
                           const uint64_t slot = atomicAdd((unsigned long long*)&counters[C_NPAIR], 1ull);
                           if (slot < pair_cap) {
                             PairRec r;
                             r.blk = (uint32_t)b;
                             r.thr = (uint32_t)lt;
                             for (int l = 0; l < MAXLOOP; ++l) r.it[l] = (uint32_t)ic[l];
                             r.acc = a;
                             r.pad = 0;
                             r.iv = iv;
                             pairs[slot] = r;
                           }
                         }
                       }
                       return;
                     }
                     if (MODE == 0 && !((emask >> a) & 1u)) {  // counted, never written
                       if (inb) drop += (uint64_t)G * mult;
                       return;
                     }
                     if (inb) {
                       const int rank = __popc(bal & lanemask_lt());
                       for (int j = 0; j < G; ++j) {
                         const uint64_t key = make_key(P, A, a, idx, iv, b, lt, j);
                         if (MODE == 1) {
                           keys[cursor + (uint64_t)rank * G + j] = key;
                           // with the cell filter's table complete, a key of a cell that
                           // can race is also appended to the compact buffer (any order)
                           if (cbuf && cell_kept(ctab, P->ncells, shr64(key, P->PB + P->IVB))) {
                             const uint64_t g = atomicAdd((unsigned long long*)&counters[C_NCOMPACT], 1ull);
                             if (g < ccap) cbuf[g] = key;
                           }
                         } else if (keys) {  // count pass with the cell filter: `keys` is its table
                           cell_note(reinterpret_cast<uint32_t*>(keys), shr64(key, P->PB + P->IVB),
                                     (uint32_t)((uint64_t)b << P->TB | (uint64_t)lt), (P->wmask >> a) & 1u);
                         } else {
                           for (int p = 0; p < npass; ++p)
                             atomicAdd(&shist[p * 256 + ((uint32_t)(key >> (SB + 8 * p)) & 255u)], mult);
                         }
                       }
                     }
                     cursor += (uint64_t)__popc(bal) * G * mult;
                   };
    // the count pass may take loop-invariant accesses once per unit, and so
    // may the pair search (an access whose instances ignore the loop vector
    // is recorded at the unit's first loop vector only: a thread's later
    // instances of it have larger keys and race with the same instances, so
    // the smallest racing pair is among the recorded ones); the write pass
    // expands only the accesses whose keys are kept
    if (MODE == 0 || MODE == 2)
      oob += ex.template unit_once<SEL_ALL>(lane, u, only, step);
    else
      oob += ex.template unit<MODE == 1 ? SEL_KEPT : SEL_ALL>(lane, u, only, step);
    if (MODE == 0 && lane == 0) unit_cnt[u] = cursor;
  }
  if (MODE == 0) {
    for (int o = 16; o; o >>= 1) {
      oob += __shfl_down_sync(FULL, oob, o);
      drop += __shfl_down_sync(FULL, drop, o);
    }
    if (lane == 0 && oob) atomicAdd((unsigned long long*)&counters[C_NOOB], (unsigned long long)oob);
    if (lane == 0 && drop) atomicAdd((unsigned long long*)&counters[C_NDROP], (unsigned long long)drop);
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += EXP_THREADS)
      if (shist[i]) atomicAdd((unsigned long long*)&hist[i], (unsigned long long)shist[i]);
  }
}

// Block-local mode: one CTA per simulated block (grid-stride over blocks); its
// warps take the block's units.  A shared-memory race needs a writer and two
// threads of one block in one interval (Table 2), so a (shared granule,
// interval) bin of the block can only race when it has both; such a bin is a
// candidate, the rest never reach the key buffer.
//   MODE 3 (count): global-array keys per unit and their digit-0 histogram,
//     as mode 0; per bin the instance count, min / max thread and a writer
//     bit.  The block's candidate bins get consecutive room in the shared-key
//     region (base from a device counter, so blocks land in any order); table
//     row b keeps (start << 32 | count) per candidate bin, 0 for the others.
//   MODE 4 (write): global keys at their unit offsets (emission order, as
//     mode 1); keys of candidate bins into their bin, in any order, at
//     keys_s[n_global + base(b) + start + slot].  A block without candidate
//     bins expands its global-array accesses only.
// bins: block_body_words(MODE, nsbins) words of shared memory.
template <typename T, int MODE, class X>
__device__ __forceinline__ void expand_block_body(const DProg* __restrict__ P, X& ex, uint32_t* bins,
                                                  uint64_t* __restrict__ unit_cnt,
                                                  const uint64_t* __restrict__ unit_off, uint64_t* __restrict__ keys_g,
                                                  uint64_t* __restrict__ keys_s, uint64_t* __restrict__ hist,
                                                  uint64_t* __restrict__ counters, uint64_t* __restrict__ stbl,
                                                  uint64_t* __restrict__ sbase, uint32_t only_in) {
  constexpr int WPC = EXP_THREADS / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NB = (int)P->nsbins;
  const int niv = P->niv;
  const int64_t ivmin = P->ivmin;
  // MODE 3: count | min thread | max thread | writer bits | digit-0 histogram | scan scratch
  uint32_t* s_cnt = bins;
  uint32_t* s_mn = bins + NB;
  uint32_t* s_mx = bins + 2 * NB;
  uint32_t* s_wb = bins + 3 * NB;
  const int NW = (NB + 31) >> 5;
  uint32_t* shist = s_wb + NW;
  uint64_t* ws = reinterpret_cast<uint64_t*>(bins + ((3 * NB + NW + 256 + 1) & ~1));
  // MODE 4: write cursors (start of the bin's room, or NONE)
  constexpr uint32_t NONE = 0xffffffffu;
  uint32_t* s_cur = bins;
  const int64_t nblk = P->nblk;
  const int64_t upb = (int64_t)P->wpb * P->nchunk;
  const int SB = P->SB;  // lowest sorted key bit
  const uint32_t wmask = P->wmask;
  const uint32_t emask = ex.emask_of(P);  // a constant in the specialised kernels
  uint64_t oob = 0, drop = 0;
  if (MODE == 3) {
    for (int i = threadIdx.x; i < NB; i += EXP_THREADS) {
      s_cnt[i] = 0;
      s_mn[i] = NONE;
      s_mx[i] = 0;
    }
    for (int i = threadIdx.x; i < NW; i += EXP_THREADS) s_wb[i] = 0;
    for (int i = threadIdx.x; i < 256; i += EXP_THREADS) shist[i] = 0;
  } else if (blockIdx.x == 0 && threadIdx.x == 0) {
    counters[C_NKEYS] = counters[C_NG] + counters[C_NS] + counters[C_NDROP];
  }
  const uint64_t n_g = MODE == 4 ? counters[C_NG] : 0;
  __syncthreads();
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    uint64_t sb = 0;
    bool has = true;  // the block has candidate bins
    if (MODE == 4) {
      const uint64_t base = sbase[b];
      has = base != NO_ROW;
      if (has) {  // (uniform over the CTA: every thread read the same base)
        for (int i = threadIdx.x; i < NB; i += EXP_THREADS) {
          const uint64_t e = stbl[(uint64_t)b * NB + i];
          s_cur[i] = (uint32_t)e ? (uint32_t)(e >> 32) : NONE;
        }
        sb = n_g + base;
        __syncthreads();
      }
    }
    for (int64_t u = b * upb + warp; u < (b + 1) * upb; u += WPC) {
      uint64_t cursor = MODE == 4 ? unit_off[u] : 0;
      auto step = [&](int a, const DAcc& A, bool inb, unsigned bal, int64_t idx, int64_t iv, int64_t bb, int lt,
                         const int32_t*, uint32_t mult) {
                       const int G = A.G;
                       if (MODE == 3 && !((emask >> a) & 1u)) {  // counted, never written
                         if (inb) drop += (uint64_t)G * mult;
                         return;
                       }
                       if (A.shared) {
                         if (!inb) return;
                         const uint32_t bin0 =
                             (uint32_t)(((uint64_t)A.sgbase + (uint64_t)idx * G) * niv + (uint64_t)(iv - ivmin));
                         for (int j = 0; j < G; ++j) {
                           const uint32_t bin = bin0 + (uint32_t)(j * niv);
                           if (MODE == 3) {
                             atomicAdd(&s_cnt[bin], mult);
                             atomicMin(&s_mn[bin], (uint32_t)lt);
                             atomicMax(&s_mx[bin], (uint32_t)lt);
                             if ((wmask >> a) & 1u) atomicOr(&s_wb[bin >> 5], 1u << (bin & 31));
                           } else if (s_cur[bin] != NONE) {
                             const uint32_t pos = atomicAdd(&s_cur[bin], 1u);
                             keys_s[sb + pos] = make_key(P, A, a, idx, iv, bb, lt, j);
                           }
                         }
                         return;
                       }
                       if (inb) {
                         const int rank = __popc(bal & lanemask_lt());
                         for (int j = 0; j < G; ++j) {
                           const uint64_t key = make_key(P, A, a, idx, iv, bb, lt, j);
                           if (MODE == 4)
                             keys_g[cursor + (uint64_t)rank * G + j] = key;
                           else if (keys_g)  // count pass with the cell filter: `keys_g` is its table
                             cell_note(reinterpret_cast<uint32_t*>(keys_g), shr64(key, P->PB + P->IVB),
                                       (uint32_t)((uint64_t)bb << P->TB | (uint64_t)lt), (wmask >> a) & 1u);
                           else
                             atomicAdd(&shist[(uint32_t)(key >> SB) & 255u], mult);
                         }
                       }
                       cursor += (uint64_t)__popc(bal) * G * mult;
                     };
      auto flush = [&](int a, uint32_t bin, uint32_t count, int lt) {
        atomicAdd(&s_cnt[bin], count);
        atomicMin(&s_mn[bin], (uint32_t)lt);
        atomicMax(&s_mx[bin], (uint32_t)lt);
        if ((wmask >> a) & 1u) atomicOr(&s_wb[bin >> 5], 1u << (bin & 31));
      };
      // the write pass expands only the accesses whose keys are kept, and of
      // those only the global ones in a block without candidate bins
      if (MODE == 3)
        oob += ex.template unit_combine<SEL_ALL>(lane, u, only_in, step, flush);
      else if (has)
        oob += ex.template unit<SEL_KEPT>(lane, u, only_in, step);
      else
        oob += ex.template unit<SEL_KEPT_GLOBAL>(lane, u, only_in, step);
      if (MODE == 3 && lane == 0) unit_cnt[u] = cursor;
    }
    // the block's shared tables are read and reset below (count pass) or
    // reloaded for the next block (write pass with a bin-table row); a write
    // pass over a block without one touched no shared memory
    if (MODE == 3 || has) __syncthreads();
    if (MODE == 3) {
      // candidate bins of block b: room in the order of a strided walk
      uint64_t csum = 0, asum = 0;
      for (int i = threadIdx.x; i < NB; i += EXP_THREADS) {
        const uint32_t c = s_cnt[i];
        asum += c;
        if (((s_wb[i >> 5] >> (i & 31)) & 1u) && s_mn[i] < s_mx[i]) csum += c;
      }
      for (int o = 16; o; o >>= 1) asum += __shfl_down_sync(FULL, asum, o);
      if (lane == 0 && asum) atomicAdd((unsigned long long*)&counters[C_NS], (unsigned long long)asum);
      uint64_t start = block_excl_scan(csum, ws, ws + 8);
      if (threadIdx.x == 0) {
        const uint64_t tot = ws[8];
        // base of the block's candidate keys, or NO_ROW: no candidate bin, or no
        // room (the check then reports it); a block without a row writes no
        // bin-table row and no shared keys
        uint64_t base = NO_ROW;
        if (tot) {
          base = atomicAdd((unsigned long long*)&counters[C_NSC], (unsigned long long)tot);
          if (base + tot > P->scap) {
            atomicOr((unsigned long long*)&counters[C_ERR], (unsigned long long)ERR_SHARED_FULL);
            base = NO_ROW;
          }
        }
        sbase[b] = base;
        ws[9] = base;
      }
      __syncthreads();
      // the block's bin-table row, and every bin reset for the next block in
      // the same walk (a thread resets the bins it reads; the writer bits,
      // shared by 32 bins, after a barrier)
      const bool row = ws[9] != NO_ROW;
      for (int i = threadIdx.x; i < NB; i += EXP_THREADS) {
        if (row) {
          const uint32_t c = s_cnt[i];
          const bool cand = ((s_wb[i >> 5] >> (i & 31)) & 1u) && s_mn[i] < s_mx[i];
          stbl[(uint64_t)b * NB + i] = cand ? ((start << 32) | c) : 0ull;
          if (cand) start += c;
        }
        s_cnt[i] = 0;
        s_mn[i] = NONE;
        s_mx[i] = 0;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < NW; i += EXP_THREADS) s_wb[i] = 0;
      __syncthreads();
    }
  }
  if (MODE == 3) {
    for (int o = 16; o; o >>= 1) {
      oob += __shfl_down_sync(FULL, oob, o);
      drop += __shfl_down_sync(FULL, drop, o);
    }
    if (lane == 0 && oob) atomicAdd((unsigned long long*)&counters[C_NOOB], (unsigned long long)oob);
    if (lane == 0 && drop) atomicAdd((unsigned long long*)&counters[C_NDROP], (unsigned long long)drop);
    for (int i = threadIdx.x; i < 256; i += EXP_THREADS)
      if (shist[i]) atomicAdd((unsigned long long*)&hist[i], (unsigned long long)shist[i]);
  }
}

}  // namespace dev
}  // namespace hgrd
