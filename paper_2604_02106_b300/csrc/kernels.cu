// Kernels of the exhaustive race check (sm_103a).
//
//  expand     every (block, thread, loop vector, access) instance of the user
//             kernel -> 64-bit keys (Table 1's addr / tb / id made concrete).
//             One CUDA warp evaluates one simulated warp of the user kernel,
//             lane = simulated thread, so each (loop vector, access) step is a
//             warp-uniform instruction stream and live keys compact with a
//             ballot into coalesced stores.
//  onesweep   stable LSD radix sort, 8-bit digits: per-warp shared-memory
//             digit histograms ranked with __match_any_sync, decoupled
//             look-back across tiles with a bounded spin.
//  candidates phase A of the conflict scan: one streaming read of the sorted
//             keys flags the runs of equal (array, granule) that can hold a
//             race (a writer plus two threads in one interval, or a writer plus
//             two blocks in global memory).
//  exact      phase B: per flagged run, lane = access id keeps min/max of
//             block, warp and thread per barrier interval and block; pairs
//             are decided with ballots and __match_any_sync (Table 2).
//  witness    merge per-run witnesses into the canonical set.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "expand_body.cuh"

namespace hgrd {

namespace {

using namespace dev;

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------------------------------ expand
// The interpreted expander: the compiled program staged in shared memory,
// one slot file of 32 lanes per warp.
template <typename T>
struct InterpX {
  const DProg* P;
  T* sl;
  __device__ __forceinline__ uint32_t emask_of(const DProg* Q) const { return Q->emask; }
  template <int SEL, class Step>
  __device__ __forceinline__ uint64_t unit(int lane, int64_t u, uint32_t only, Step&& step) {
    if (SEL != SEL_ALL) only &= P->emask;
    if (SEL == SEL_KEPT_GLOBAL)
      for (int a = 0; a < P->nacc; ++a)
        if (P->acc[a].shared) only &= ~(1u << a);
    return expand_unit<T>(P, sl, lane, u, only,
                          [&](int a, const DAcc& A, bool inb, unsigned bal, int64_t idx, int64_t iv, int64_t b,
                              int lt, const int32_t* ic) { step(a, A, inb, bal, idx, iv, b, lt, ic, 1u); });
  }
  // the interpreter hands every instance to step
  template <int SEL, class Step>
  __device__ __forceinline__ uint64_t unit_once(int lane, int64_t u, uint32_t only, Step&& step) {
    return unit<SEL>(lane, u, only, step);
  }
  template <int SEL, class Step, class Flush>
  __device__ __forceinline__ uint64_t unit_combine(int lane, int64_t u, uint32_t only, Step&& step, Flush&&) {
    return unit<SEL>(lane, u, only, step);
  }
};

// Stages the program into shared memory; returns the byte after the warps' slot files.
template <typename T>
__device__ __forceinline__ unsigned char* stage_program(const DProg* Pg, unsigned char* smem, InterpX<T>* ex) {
  const uint4* src = reinterpret_cast<const uint4*>(Pg);
  uint4* dst = reinterpret_cast<uint4*>(smem);
  for (int i = threadIdx.x; i < (int)(sizeof(DProg) / 16); i += EXP_THREADS) dst[i] = src[i];
  __syncthreads();
  const DProg* P = reinterpret_cast<const DProg*>(smem);
  const int nslot = P->nslot;
  unsigned char* after = smem + sizeof(DProg);
  ex->P = P;
  ex->sl = reinterpret_cast<T*>(after) + (size_t)(threadIdx.x >> 5) * nslot * 32;
  return after + (size_t)(EXP_THREADS / 32) * nslot * 32 * sizeof(T);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(EXP_THREADS) expand_kernel(const DProg* __restrict__ Pg, uint64_t* __restrict__ unit_cnt,
                                                             const uint64_t* __restrict__ unit_off,
                                                             uint64_t* __restrict__ keys, uint64_t* __restrict__ hist,
                                                             int npass, uint64_t* __restrict__ counters,
                                                             const uint64_t* __restrict__ uniq,
                                                             PairRec* __restrict__ pairs, uint64_t pair_cap,
                                                             const uint32_t* __restrict__ ctab,
                                                             uint64_t* __restrict__ cbuf, uint64_t ccap) {
  extern __shared__ __align__(16) unsigned char smem[];
  InterpX<T> ex;
  uint32_t* shist = reinterpret_cast<uint32_t*>(stage_program<T>(Pg, smem, &ex));
  expand_units_body<T, MODE>(ex.P, ex, shist, unit_cnt, unit_off, keys, hist, npass, counters, uniq, pairs, pair_cap,
                             0xffffffffu, ctab, cbuf, ccap);
}

// ------------------------------------------------------------------ scan

__device__ __forceinline__ uint64_t dev_n(const uint64_t* n_dev, uint64_t n_max) {
  if (!n_dev) return n_max;
  uint64_t n = *n_dev;
  return n < n_max ? n : n_max;
}

__global__ void __launch_bounds__(256) scan_reduce(const uint64_t* __restrict__ in, const uint64_t* n_dev, uint64_t n_max,
                                                   uint64_t* __restrict__ partials) {
  const uint64_t n = dev_n(n_dev, n_max);
  __shared__ uint64_t ws[8];
  __shared__ uint64_t tot;
  for (uint64_t tile = blockIdx.x; tile * SCAN_TILE < n; tile += gridDim.x) {
    uint64_t s = 0;
    for (int k = 0; k < SCAN_TILE / 256; ++k) {
      uint64_t i = tile * SCAN_TILE + (uint64_t)k * 256 + threadIdx.x;
      if (i < n) s += in[i];
    }
    block_excl_scan(s, ws, &tot);
    if (threadIdx.x == 0) partials[tile] = tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) scan_partials(uint64_t* partials, const uint64_t* n_dev, uint64_t n_max,
                                                     uint64_t* total) {
  const uint64_t n = dev_n(n_dev, n_max);
  const uint64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  __shared__ uint64_t ws[8];
  __shared__ uint64_t tot;
  uint64_t carry = 0;
  for (uint64_t c = 0; c < nt; c += 256) {
    uint64_t i = c + threadIdx.x;
    uint64_t v = i < nt ? partials[i] : 0;
    uint64_t e = block_excl_scan(v, ws, &tot);
    if (i < nt) partials[i] = carry + e;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(256) scan_apply(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                  const uint64_t* n_dev, uint64_t n_max,
                                                  const uint64_t* __restrict__ partials) {
  const uint64_t n = dev_n(n_dev, n_max);
  __shared__ uint64_t ws[8];
  __shared__ uint64_t tot;
  for (uint64_t tile = blockIdx.x; tile * SCAN_TILE < n; tile += gridDim.x) {
    // each thread owns SCAN_PER consecutive elements of the tile
    const uint64_t b0 = tile * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_PER;
    uint64_t v[SCAN_PER], s = 0;
    for (int k = 0; k < SCAN_PER; ++k) {
      v[k] = (b0 + k < n) ? in[b0 + k] : 0;
      s += v[k];
    }
    uint64_t run = partials[tile] + block_excl_scan(s, ws, &tot);
    for (int k = 0; k < SCAN_PER; ++k) {
      if (b0 + k < n) out[b0 + k] = run;
      run += v[k];
    }
  }
}

// Up to SCAN_FUSE_TILES tiles: scan_apply_fused takes the raw tile sums of
// scan_reduce and adds up the ones before its tile itself (no partials pass);
// the CTA holding the last tile writes the total.
constexpr uint64_t SCAN_FUSE_TILES = 256;
__global__ void __launch_bounds__(256) scan_apply_fused(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                        const uint64_t* n_dev, uint64_t n_max,
                                                        const uint64_t* __restrict__ sums, uint64_t* total) {
  const uint64_t n = dev_n(n_dev, n_max);
  const uint64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  __shared__ uint64_t ws[8];
  __shared__ uint64_t tot;
  for (uint64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    // tiles before this one: thread i holds sums[i] (nt <= 256)
    const uint64_t before = threadIdx.x < tile ? sums[threadIdx.x] : 0;
    block_excl_scan(before, ws, &tot);
    const uint64_t base = tot;
    if (tile == nt - 1 && threadIdx.x == 0 && total) *total = base + sums[tile];
    const uint64_t b0 = tile * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_PER;
    uint64_t v[SCAN_PER], s = 0;
    for (int k = 0; k < SCAN_PER; ++k) {
      v[k] = (b0 + k < n) ? in[b0 + k] : 0;
      s += v[k];
    }
    uint64_t run = base + block_excl_scan(s, ws, &tot);
    for (int k = 0; k < SCAN_PER; ++k) {
      if (b0 + k < n) out[b0 + k] = run;
      run += v[k];
    }
  }
  if (nt == 0 && blockIdx.x == 0 && threadIdx.x == 0 && total) *total = 0;
}

// ------------------------------------------------------------------ expand, block-local shared bins
template <typename T, int MODE>
__global__ void __launch_bounds__(EXP_THREADS) expand_block_kernel(
    const DProg* __restrict__ Pg, uint64_t* __restrict__ unit_cnt, const uint64_t* __restrict__ unit_off,
    uint64_t* __restrict__ keys_g, uint64_t* __restrict__ keys_s, uint64_t* __restrict__ hist,
    uint64_t* __restrict__ counters, uint64_t* __restrict__ stbl, uint64_t* __restrict__ sbase) {
  extern __shared__ __align__(16) unsigned char smem[];
  InterpX<T> ex;
  uint32_t* bins = reinterpret_cast<uint32_t*>(stage_program<T>(Pg, smem, &ex));
  expand_block_body<T, MODE>(ex.P, ex, bins, unit_cnt, unit_off, keys_g, keys_s, hist, counters, stbl, sbase,
                             0xffffffffu);
}

// candidate bins of the block-local mode -> exact-scan entries, after the
// global candidates; an entry's start carries SHARED_ENTRY and both ends are
// relative to the first shared key (the exact scan adds the global key count)
constexpr uint64_t SHARED_ENTRY = 1ull << 63;
// A warp per block; blocks without a bin-table row are skipped.
__global__ void shared_cand_kernel(const uint64_t* __restrict__ stbl, const uint64_t* __restrict__ sbase, int64_t nblk,
                                   int64_t nb, uint64_t* __restrict__ cand, uint64_t cand_cap, uint64_t* counters) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = gw; b < nblk; b += nw) {
    const uint64_t sb = sbase[b];
    if (sb == NO_ROW) continue;
    for (int64_t i0 = 0; i0 < nb; i0 += 32) {
      const int64_t i = i0 + lane;
      const uint64_t e = i < nb ? stbl[(uint64_t)b * (uint64_t)nb + (uint64_t)i] : 0ull;
      const bool has = (uint32_t)e != 0;
      const unsigned m = __ballot_sync(FULL, has);
      if (!m) continue;
      uint64_t base = 0;
      if (lane == __ffs(m) - 1)
        base = atomicAdd((unsigned long long*)&counters[C_NCAND], (unsigned long long)__popc(m));
      base = __shfl_sync(FULL, base, __ffs(m) - 1);
      if (has) {
        const uint64_t g = base + __popc(m & lanemask_lt());
        const uint64_t s = sb + (e >> 32);
        if (g < cand_cap) {
          cand[2 * g] = SHARED_ENTRY | s;
          cand[2 * g + 1] = s + (uint32_t)e;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ cell filter
// Cell filter: the digit histogram of the first sort pass over the keys it
// keeps, and their count
__global__ void __launch_bounds__(256) cell_hist_kernel(const uint64_t* __restrict__ keys, const uint64_t* n_dev,
                                                        uint64_t n_max, const uint32_t* __restrict__ tab,
                                                        uint64_t ncells, int rsh, uint64_t* __restrict__ hist, int shift,
                                                        uint64_t* __restrict__ n_kept, uint64_t* __restrict__ status,
                                                        uint64_t max_words, const uint64_t* skip) {
  if (skip && *skip) return;  // the compact form sorted the kept keys already
  __shared__ uint32_t sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t n = dev_n(n_dev, n_max);
  {  // the look-back status of the tiles the first sort pass will use
    uint64_t words = (n + RS_MIN_TILE - 1) / RS_MIN_TILE * RS_RADIX;
    if (words > max_words) words = max_words;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
      status[i] = 0;
  }
  uint32_t kept = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    if (cell_kept(tab, ncells, shr64(k, rsh))) {
      atomicAdd(&sh[(uint32_t)(k >> shift) & 255u], 1u);
      ++kept;
    }
  }
  for (int o = 16; o; o >>= 1) kept += __shfl_down_sync(FULL, kept, o);
  if ((threadIdx.x & 31) == 0 && kept) atomicAdd((unsigned long long*)n_kept, (unsigned long long)kept);
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd((unsigned long long*)&hist[threadIdx.x], (unsigned long long)sh[threadIdx.x]);
}

// ------------------------------------------------------------------ radix sort
__global__ void __launch_bounds__(256) histogram_kernel(const uint64_t* __restrict__ keys, const uint64_t* n_dev,
                                                        uint64_t n_max, int shift0, int npass,
                                                        uint64_t* __restrict__ hist) {
  __shared__ uint32_t sh[MAX_PASSES * 256];
  const uint64_t n = dev_n(n_dev, n_max);
  for (int i = threadIdx.x; i < npass * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    for (int p = 0; p < npass; ++p) atomicAdd(&sh[p * 256 + (uint32_t)((k >> (shift0 + 8 * p)) & 255)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * 256; i += blockDim.x)
    if (sh[i]) atomicAdd((unsigned long long*)&hist[i], (unsigned long long)sh[i]);
}

constexpr uint64_t ST_AGG = 1ull << 54, ST_PREFIX = 2ull << 54, ST_VAL = (1ull << 54) - 1;

// The pass's global start of each digit, from its digit counts: one warp
// scans the 256 counts (eight per lane) into sgb (shared memory).
__device__ __forceinline__ void digit_bases(const uint64_t* __restrict__ dcount, uint64_t* sgb) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  uint64_t v[8], s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v[j] = dcount[lane * 8 + j];
    s += v[j];
  }
  uint64_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  uint64_t run = x - s;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    sgb[lane * 8 + j] = run;
    run += v[j];
  }
}
constexpr uint32_t SPIN_LIMIT = 1u << 22;

// Onesweep pass, templated on the CTA shape (threads T, keys per thread KPT,
// CTAs per SM the registers are budgeted for) and on the warp ranking (RA:
// the leader of each digit's peers takes the warp's running count with one
// shared atomic add and passes it on by shuffle, so the slots pipeline; else
// a read, a leader write and two warp barriers per slot) and on how a lane
// finds the lanes with its digit (MS: nine ballots, one per digit bit and
// one for "has a key"; else the match instruction); the sort autotuner picks
// the shape.  Each CTA loops over tiles taken from a ticket counter, so tiles are
// handled in increasing order and the look-back only waits on tiles held by
// running CTAs.
template <int T, int KPT, int MINB, bool RA = false, int MS = 0>
__global__ void __launch_bounds__(T, MINB) onesweep_kernel(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                          const uint64_t* n_dev, uint64_t n_max, int shift,
                                                          const uint64_t* __restrict__ dcount, uint64_t* status,
                                                          unsigned long long* ticket, uint32_t epoch, uint64_t* err,
                                                          uint64_t* next_hist, int next_shift,
                                                          const uint32_t* __restrict__ ctab, uint64_t ncells, int rsh,
                                                          const uint64_t* skip) {
  if (skip && *skip) return;  // one CTA already sorted the remaining digits
  constexpr int W = T / 32, TILE = T * KPT;
  extern __shared__ __align__(16) unsigned char osm[];
  uint32_t* whist = reinterpret_cast<uint32_t*>(osm);  // [W][256]
  uint32_t* nhist = whist + W * RS_RADIX;               // digit counts of the next pass
  uint32_t* tstart = nhist + RS_RADIX;                  // tile-local start of each digit
  uint32_t* dsum = tstart + RS_RADIX;                   // tile count of each digit
  uint64_t* gofs = reinterpret_cast<uint64_t*>(dsum + RS_RADIX);
  uint64_t* stage = gofs + RS_RADIX;
  uint64_t* s_tile = stage + TILE;
  uint32_t* s_kept = reinterpret_cast<uint32_t*>(s_tile + 1);  // keys of the tile that stay
  uint64_t* gbase = s_tile + 2;                                 // the pass's start of each digit
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t n = dev_n(n_dev, n_max);
  const uint64_t ntiles = (n + TILE - 1) / TILE;
  // the grid is sized for the most keys the pass can see; CTAs past the
  // tiles there are leave before touching the ticket
  if ((uint64_t)blockIdx.x >= ntiles) return;
  const uint64_t ep = (uint64_t)epoch << 56;
  for (int d = threadIdx.x; d < RS_RADIX; d += T) nhist[d] = 0;
  digit_bases(dcount, gbase);
  for (;;) {
    if (threadIdx.x == 0) *s_tile = atomicAdd(ticket, 1ull);
    for (int i = threadIdx.x; i < W * RS_RADIX; i += T) whist[i] = 0;
    __syncthreads();
    const uint64_t tile = *s_tile;
    if (tile >= ntiles) break;
    const uint64_t base = tile * TILE;
    const uint64_t wbase = base + (uint64_t)warp * (KPT * 32);
    uint64_t k[KPT];
    uint32_t dr[KPT];  // digit in bits 0..8 (256 = no key), warp-local rank above
#pragma unroll
    for (int s = 0; s < KPT; ++s) {
      const uint64_t i = wbase + (uint64_t)s * 32 + lane;
      k[s] = i < n ? in[i] : 0;
    }
    const unsigned lt = lanemask_lt();
    // warp-level stable ranking, slot-major = memory order
#pragma unroll
    for (int s = 0; s < KPT; ++s) {
      const uint64_t i = wbase + (uint64_t)s * 32 + lane;
      const bool live = i < n && (!ctab || cell_kept(ctab, ncells, shr64(k[s], rsh)));
      const uint32_t d = live ? (uint32_t)((k[s] >> shift) & 255) : 256u;
      if (next_hist && d < 256u) atomicAdd(&nhist[(uint32_t)(k[s] >> next_shift) & 255u], 1u);
      unsigned peers;
      // MS 1: ballots in every slot; MS 2: ballots in odd slots, the match
      // instruction in even ones (the ALU and the shared-memory pipe share the work)
      if (MS == 1 || (MS == 2 && (s & 1))) {
        const unsigned has = __ballot_sync(FULL, d < 256u);
        peers = d < 256u ? has : ~has;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const unsigned bb = __ballot_sync(FULL, (d >> b) & 1u);
          peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
      } else {
        peers = __match_any_sync(FULL, d);
      }
      uint32_t old = 0;
      if constexpr (RA) {
        // one warp's atomics reach shared memory in issue order, slot after slot
        const int leader = __ffs(peers) - 1;
        if (d < 256u && lane == leader) old = atomicAdd(&whist[warp * RS_RADIX + d], (uint32_t)__popc(peers));
        old = __shfl_sync(FULL, old, leader);
        dr[s] = d | ((old + __popc(peers & lt)) << 9);
      } else {
        if (d < 256u) old = whist[warp * RS_RADIX + d];
        dr[s] = d | ((old + __popc(peers & lt)) << 9);
        __syncwarp();
        if (d < 256u && lane == __ffs(peers) - 1) whist[warp * RS_RADIX + d] = old + __popc(peers);
        __syncwarp();
      }
    }
    __syncthreads();
    // digits: counts across warps, warp-exclusive prefixes; the tile's
    // aggregate is published before its keys move, the look-back comes after
    for (int t = threadIdx.x; t < RS_RADIX; t += T) {
      uint32_t sum = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const uint32_t c = whist[w * RS_RADIX + t];
        whist[w * RS_RADIX + t] = sum;
        sum += c;
      }
      dsum[t] = sum;
      st_relaxed(status + tile * RS_RADIX + t, ep | (tile == 0 ? ST_PREFIX : ST_AGG) | sum);
    }
    __syncthreads();
    if (warp == 0) {  // tile-local digit starts: lane l scans digits 8l .. 8l+7
      uint32_t v[8], s8 = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        v[j] = dsum[lane * 8 + j];
        s8 += v[j];
      }
      uint32_t x = s8;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
      }
      uint32_t run = x - s8;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        tstart[lane * 8 + j] = run;
        run += v[j];
      }
      if (lane == 31) *s_kept = run;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < KPT; ++s) {
      const uint32_t d = dr[s] & 511u;
      if (d < 256u) stage[tstart[d] + whist[warp * RS_RADIX + d] + (dr[s] >> 9)] = k[s];
    }
    // look-back: the keys of the tile before this one with each digit
    for (int t = threadIdx.x; t < RS_RADIX; t += T) {
      uint64_t excl = 0;
      if (tile != 0) {
        // walk back over the predecessors LBW at a time: the loads of a
        // window are independent, so one memory round trip covers LBW tiles;
        // aggregates add up to the nearest inclusive prefix (tile 0 always
        // publishes one), a tile not yet published is read again
        constexpr int LBW = 4;
        uint64_t p = tile - 1;
        uint32_t spins = 0;
        for (;;) {
          const int m = p >= (uint64_t)(LBW - 1) ? LBW : (int)p + 1;
          uint64_t wv[LBW];
#pragma unroll
          for (int j = 0; j < LBW; ++j)
            if (j < m) wv[j] = ld_relaxed(status + (p - (uint64_t)j) * RS_RADIX + t);
          bool done = false, stall = false;
          uint64_t used = 0;
#pragma unroll
          for (int j = 0; j < LBW; ++j) {
            if (j >= m || done || stall) continue;
            const bool ready = (wv[j] >> 56) == epoch && (wv[j] & (3ull << 54)) != 0;
            if (!ready) {
              stall = true;
              continue;
            }
            excl += wv[j] & ST_VAL;
            if ((wv[j] & ST_PREFIX) || p == (uint64_t)j) done = true;
            else ++used;
          }
          if (done) break;
          p -= used;
          if (stall) {
            if (++spins > SPIN_LIMIT) {
              atomicOr((unsigned long long*)err, (unsigned long long)ERR_TIMEOUT);
              break;
            }
            __nanosleep(32);
          }
        }
        st_relaxed(status + tile * RS_RADIX + t, ep | ST_PREFIX | (excl + dsum[t]));
      }
      gofs[t] = gbase[t] + excl;
    }
    __syncthreads();
    const uint32_t cnt = *s_kept;
    for (uint32_t i = threadIdx.x; i < cnt; i += T) {
      const uint64_t key = stage[i];
      const uint32_t d = (uint32_t)((key >> shift) & 255);
      out[gofs[d] + (i - tstart[d])] = key;
    }
    __syncthreads();
  }
  for (int d = threadIdx.x; d < RS_RADIX; d += T)
    if (next_hist && nhist[d]) atomicAdd((unsigned long long*)&next_hist[d], (unsigned long long)nhist[d]);
}

// The digits after the first pass of a sort that kept at most TAIL_MAX keys:
// one CTA loads them into shared memory and runs the remaining LSD passes
// there (the onesweep ranking, nine ballots and a shared atomic per slot,
// with one tile and so no look-back), writes the result where the last pass
// would have, and sets *done so the device-wide passes after it return at
// once.  With more keys it does nothing.
constexpr int TAIL_T = 1024, TAIL_KPT = 4, TAIL_MAX = TAIL_T * TAIL_KPT;
static_assert(TAIL_MAX == TAIL_KEYS, "the compact form's capacity");
constexpr size_t tail_smem() { return (size_t)2 * TAIL_MAX * 8 + (size_t)(TAIL_T / 32) * RS_RADIX * 4 + RS_RADIX * 4; }
__global__ void __launch_bounds__(TAIL_T) tail_sort_kernel(const uint64_t* in, uint64_t* out, const uint64_t* n_dev,
                                                           uint64_t n_max, int shift0, int npass, uint64_t* done) {
  extern __shared__ __align__(16) unsigned char tsm[];
  uint64_t* A = reinterpret_cast<uint64_t*>(tsm);
  uint64_t* Bk = A + TAIL_MAX;
  uint32_t* whist = reinterpret_cast<uint32_t*>(Bk + TAIL_MAX);  // [32 warps][256]
  uint32_t* dbase = whist + (TAIL_T / 32) * RS_RADIX;             // digit starts
  if (*done) return;  // the compact form sorted the keys already
  const uint64_t n = dev_n(n_dev, n_max);
  if (n > (uint64_t)TAIL_MAX || npass <= 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  for (uint32_t i = threadIdx.x; i < n; i += TAIL_T) A[i] = in[i];
  for (int p = 0; p < npass; ++p) {
    const int shift = shift0 + 8 * p;
    for (int i = threadIdx.x; i < (TAIL_T / 32) * RS_RADIX; i += TAIL_T) whist[i] = 0;
    __syncthreads();
    // warp w ranks keys [128 w, 128 w + 128), slot after slot
    uint64_t k[TAIL_KPT];
    uint32_t dr[TAIL_KPT];
#pragma unroll
    for (int s = 0; s < TAIL_KPT; ++s) {
      const uint32_t i = (uint32_t)warp * (TAIL_KPT * 32) + (uint32_t)s * 32 + lane;
      k[s] = i < n ? A[i] : 0;
      const uint32_t d = i < n ? (uint32_t)((k[s] >> shift) & 255) : 256u;
      const unsigned has = __ballot_sync(FULL, d < 256u);
      unsigned peers = d < 256u ? has : ~has;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const unsigned bb = __ballot_sync(FULL, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bb : ~bb;
      }
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (d < 256u && lane == leader) old = atomicAdd(&whist[warp * RS_RADIX + d], (uint32_t)__popc(peers));
      old = __shfl_sync(FULL, old, leader);
      dr[s] = d | ((old + __popc(peers & lt)) << 9);
    }
    __syncthreads();
    if (threadIdx.x < RS_RADIX) {  // per digit: starts of the warps' shares, digit total
      uint32_t sum = 0;
      for (int w = 0; w < TAIL_T / 32; ++w) {
        const uint32_t c = whist[w * RS_RADIX + threadIdx.x];
        whist[w * RS_RADIX + threadIdx.x] = sum;
        sum += c;
      }
      dbase[threadIdx.x] = sum;
    }
    __syncthreads();
    if (warp == 0) {  // digit starts: lane l scans digits 8l .. 8l+7
      uint32_t v[8], s8 = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        v[j] = dbase[lane * 8 + j];
        s8 += v[j];
      }
      uint32_t x = s8;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
      }
      uint32_t run = x - s8;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        dbase[lane * 8 + j] = run;
        run += v[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < TAIL_KPT; ++s) {
      const uint32_t d = dr[s] & 511u;
      if (d < 256u) Bk[dbase[d] + whist[warp * RS_RADIX + d] + (dr[s] >> 9)] = k[s];
    }
    __syncthreads();
    uint64_t* t = A;
    A = Bk;
    Bk = t;
  }
  for (uint32_t i = threadIdx.x; i < n; i += TAIL_T) out[i] = A[i];
  if (threadIdx.x == 0) *done = 1;
}

// Sort of at most TAIL_MAX keys by rank, across the GPU: key e goes to the
// number of keys below it plus the number of equal keys before it in the
// input (equal keys are the same word, so any order of them is the sorted
// one).  Every CTA that has keys to place stages the whole input in shared
// memory and each warp ranks its keys against it, 32 comparisons a step: a
// few thousand keys take a few microseconds spread over the GPU rather than
// a barrier-bound network in one CTA.
constexpr int CR_T = 512, CR_W = CR_T / 32;
__device__ __forceinline__ void rank_place(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint32_t n,
                                           uint64_t* s) {
  if (blockIdx.x * CR_W >= n) return;  // no key for this CTA
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t i = threadIdx.x; i < n; i += CR_T) s[i] = in[i];
  __syncthreads();
  for (uint32_t e = blockIdx.x * CR_W + (threadIdx.x >> 5); e < n; e += gridDim.x * CR_W) {
    const uint64_t x = s[e];
    uint32_t r = 0;
#pragma unroll 4
    for (uint32_t j = lane; j < n; j += 32) {
      const uint64_t y = s[j];
      r += (uint32_t)(y < x) + (uint32_t)((y == x) & (j < e));
    }
    r = __reduce_add_sync(FULL, r);
    if (lane == 0) out[r] = x;
  }
}

// The compact form's sort: the write pass's compact buffer of kept keys (any
// order), when every key it counted is there (at most n_max), placed by rank
// into the final buffer; their count to *kept_out, and *done set.
__global__ void __launch_bounds__(CR_T) compact_sort_kernel(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                           const uint64_t* n_dev, uint64_t n_max, uint64_t* done,
                                                           uint64_t* kept_out) {
  __shared__ uint64_t s[TAIL_MAX];
  const uint64_t n64 = *n_dev;
  if (n64 > n_max || n64 > (uint64_t)TAIL_MAX) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *kept_out = n64;
    *done = 1;
  }
  rank_place(in, out, (uint32_t)n64, s);
}

// Onesweep pass with early counts (the shapes the tuner prefers on B300).
// Per tile: keys to registers, then each warp's digit histogram with shared
// atomics; the tile's digit counts are published at once (before any key is
// ranked) and the first window of the look-back is loaded, so predecessors
// and successors rarely wait on each other; the tile-local start of every
// (warp, digit) follows from one scan.  The stable ranking then walks the
// warp's keys slot by slot in memory order (RANK 3: each lane sets its bit in
// a per-(warp, digit) mask with a shared atomic OR and reads back its peers;
// RANK 0: the match instruction; RANK 5: per warp, the match instruction when
// the warp's keys hold at most 16 distinct digits, counted from its histogram
// by the digit threads, else the atomic OR) and stores every key straight to
// its place in the shared staging tile.  The look-back finishes, and the keys
// leave in digit runs.  With the cell filter, keys of unkept cells take no
// part.  At the start of a tile the tile one grid ahead (the one this CTA will
// likely take next) is prefetched into L2.
template <int T, int KPT, int MINB, int RANK>
__global__ void __launch_bounds__(T, MINB) onesweep3_kernel(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                           const uint64_t* n_dev, uint64_t n_max, int shift,
                                                           const uint64_t* __restrict__ dcount, uint64_t* status,
                                                           unsigned long long* ticket, uint32_t epoch, uint64_t* err,
                                                           uint64_t* next_hist, int next_shift,
                                                           const uint32_t* __restrict__ ctab, uint64_t ncells, int rsh,
                                                           const uint64_t* skip) {
  static_assert(T >= RS_RADIX && KPT <= 32, "one thread per digit; live keys fit a 32-bit mask");
  if (skip && *skip) return;  // one CTA already sorted the remaining digits
  constexpr int W = T / 32, TILE = T * KPT, LBW = 4;
  extern __shared__ __align__(16) unsigned char osm[];
  uint64_t* stage = reinterpret_cast<uint64_t*>(osm);            // TILE keys in digit order
  int64_t* gdst = reinterpret_cast<int64_t*>(stage + TILE);      // per digit: output index - tile start
  uint32_t* whist = reinterpret_cast<uint32_t*>(gdst + RS_RADIX);  // [W][256] counts, then starts
  uint32_t* wmask = whist + W * RS_RADIX;                         // [W][256] peer masks (RANK 3, 5)
  uint32_t* dstart = wmask + (RANK != 0 ? W * RS_RADIX : 0);      // tile-local start of each digit
  uint32_t* nhist = dstart + RS_RADIX;                            // digit counts of the next pass
  uint32_t* wsum = nhist + RS_RADIX;                              // 8 warp totals + tile total
  uint32_t* s_tile = wsum + 16;
  uint32_t* wdist = s_tile + 2;                                   // [W] distinct digits of each warp
  uint64_t* gbase = reinterpret_cast<uint64_t*>(wdist + 32);      // the pass's start of each digit
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = threadIdx.x;
  const uint64_t n = dev_n(n_dev, n_max);
  const uint64_t ntiles = (n + TILE - 1) / TILE;
  if ((uint64_t)blockIdx.x >= ntiles) return;
  const uint64_t ep = (uint64_t)epoch << 56;
  for (int d = t; d < RS_RADIX; d += T) nhist[d] = 0;
  digit_bases(dcount, gbase);
  if (RANK != 0)
    for (int i = t; i < W * RS_RADIX; i += T) wmask[i] = 0;
  const unsigned lt = lanemask_lt();
  uint32_t* wh = whist + warp * RS_RADIX;
  uint32_t* wm = wmask + warp * RS_RADIX;
  for (;;) {
    if (t == 0) {
      const unsigned long long tk = atomicAdd(ticket, 1ull);
      s_tile[0] = (uint32_t)tk;
      s_tile[1] = (uint32_t)(tk >> 32);
    }
    for (int i = t; i < W * RS_RADIX; i += T) whist[i] = 0;
    if (RANK == 5 && t < W) wdist[t] = 0;
    __syncthreads();
    const uint64_t tile = (uint64_t)s_tile[0] | ((uint64_t)s_tile[1] << 32);
    if (tile >= ntiles) break;
    const uint64_t base = tile * TILE;
    const bool full = base + TILE <= n;
    const uint32_t rem = full ? TILE : (uint32_t)(n - base);
    if (t == 0) {  // the tile one grid ahead, into L2 (a hint: 16-byte multiples inside the input)
      const uint64_t nt = tile + gridDim.x;
      if (nt < ntiles) {
        const uint64_t nb = nt * TILE;
        const uint32_t bytes = (uint32_t)(((nb + TILE <= n ? (uint64_t)TILE : n - nb) * 8) & ~15ull);
        if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(in + nb), "r"(bytes) : "memory");
      }
    }
    const uint64_t* src = in + base + warp * (KPT * 32) + lane;
    uint64_t k[KPT];
    if (full) {
#pragma unroll
      for (int s = 0; s < KPT; ++s) k[s] = __ldcs(src + s * 32);
    } else {
#pragma unroll
      for (int s = 0; s < KPT; ++s) {
        const uint32_t i = warp * (KPT * 32) + s * 32 + lane;
        k[s] = i < rem ? src[s * 32] : 0;
      }
    }
    // live keys (in range, and of a kept cell when the filter runs); the
    // warp's digit histogram
    uint32_t live = 0;
#pragma unroll
    for (int s = 0; s < KPT; ++s) {
      const uint32_t i = warp * (KPT * 32) + s * 32 + lane;
      const bool l = i < rem && (!ctab || cell_kept(ctab, ncells, shr64(k[s], rsh)));
      live |= (uint32_t)l << s;
      if (l) atomicAdd(&wh[(uint32_t)(k[s] >> shift) & 255u], 1u);
    }
    __syncthreads();
    // per digit: the tile's count, published at once, and each warp's
    // exclusive prefix; the first window of predecessors is loaded now and
    // read after the ranking
    uint32_t dsum = 0;
    uint64_t wv[LBW];
    const uint64_t p0 = tile - 1;
    const int m0 = tile == 0 ? 0 : (p0 >= (uint64_t)(LBW - 1) ? LBW : (int)p0 + 1);
    if (t < RS_RADIX) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const uint32_t c = whist[w * RS_RADIX + t];
        whist[w * RS_RADIX + t] = dsum;
        dsum += c;
        if (RANK == 5) {  // the distinct digits of warp w, 32 at a time
          const uint32_t nz = __popc(__ballot_sync(FULL, c != 0));
          if (lane == 0 && nz) atomicAdd(&wdist[w], nz);
        }
      }
      st_relaxed(status + tile * RS_RADIX + t, ep | (tile == 0 ? ST_PREFIX : ST_AGG) | dsum);
#pragma unroll
      for (int j = 0; j < LBW; ++j)
        if (j < m0) wv[j] = ld_relaxed(status + (p0 - (uint64_t)j) * RS_RADIX + t);
      // tile-local digit starts: scan of the counts, warps of 32 digits
      uint32_t x = dsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      dstart[t] = x - dsum;
    }
    __syncthreads();
    if (t < RS_RADIX) {
      uint32_t add = 0;
#pragma unroll
      for (int w = 0; w < RS_RADIX / 32; ++w) add += (w < (t >> 5)) ? wsum[w] : 0u;
      const uint32_t ds = dstart[t] + add;
      dstart[t] = ds;
#pragma unroll
      for (int w = 0; w < W; ++w) whist[w * RS_RADIX + t] += ds;
    }
    __syncthreads();
    const bool use_match = RANK == 0 || (RANK == 5 && wdist[warp] <= 16);
    // stable ranking in memory order (slot after slot, lanes in order);
    // every key goes straight to its place in the staging tile
#pragma unroll
    for (int s = 0; s < KPT; ++s) {
      const bool l = (live >> s) & 1u;
      const uint32_t d = (uint32_t)(k[s] >> shift) & 255u;
      unsigned peers;
      if (!use_match) {
        if (l) atomicOr(&wm[d], 1u << lane);
        __syncwarp();
        peers = l ? wm[d] : 0u;
      } else {
        peers = __match_any_sync(FULL, l ? d : 256u + lane);
      }
      const uint32_t old = l ? wh[d] : 0u;
      if (l) stage[old + __popc(peers & lt)] = k[s];
      __syncwarp();
      if (l && lane == 31 - __clz(peers)) {
        wh[d] = old + __popc(peers);
        if (!use_match) wm[d] = 0u;
      }
      __syncwarp();
    }
    // the look-back: the keys of the tiles before this one with each digit
    if (t < RS_RADIX) {
      uint64_t excl = 0;
      if (tile != 0) {
        uint64_t p = p0;
        int m = m0;
        uint32_t spins = 0;
        for (;;) {
          bool done = false, stall = false;
          uint64_t used = 0;
#pragma unroll
          for (int j = 0; j < LBW; ++j) {
            if (j >= m || done || stall) continue;
            const bool ready = (wv[j] >> 56) == epoch && (wv[j] & (3ull << 54)) != 0;
            if (!ready) {
              stall = true;
              continue;
            }
            excl += wv[j] & ST_VAL;
            if ((wv[j] & ST_PREFIX) || p == (uint64_t)j) done = true;
            else ++used;
          }
          if (done) break;
          p -= used;
          if (stall) {
            if (++spins > SPIN_LIMIT) {
              atomicOr((unsigned long long*)err, (unsigned long long)ERR_TIMEOUT);
              break;
            }
            __nanosleep(32);
          }
          m = p >= (uint64_t)(LBW - 1) ? LBW : (int)p + 1;
#pragma unroll
          for (int j = 0; j < LBW; ++j)
            if (j < m) wv[j] = ld_relaxed(status + (p - (uint64_t)j) * RS_RADIX + t);
        }
        st_relaxed(status + tile * RS_RADIX + t, ep | ST_PREFIX | (excl + dsum));
      }
      gdst[t] = (int64_t)(gbase[t] + excl) - (int64_t)dstart[t];
      if (t == RS_RADIX - 1) wsum[8] = dstart[t] + dsum;  // keys kept in this tile
    }
    __syncthreads();
    // out in digit runs (consecutive keys of a digit go to consecutive places)
    if (full && !ctab) {
#pragma unroll 4
      for (int j = 0; j < KPT; ++j) {
        const uint32_t i = j * T + t;
        const uint64_t key = stage[i];
        __stcs(out + (gdst[(uint32_t)(key >> shift) & 255u] + i), key);
        if (next_hist) atomicAdd(&nhist[(uint32_t)(key >> next_shift) & 255u], 1u);
      }
    } else {
      const uint32_t kept = wsum[8];
      for (uint32_t i = t; i < kept; i += T) {
        const uint64_t key = stage[i];
        out[gdst[(uint32_t)(key >> shift) & 255u] + i] = key;
        if (next_hist) atomicAdd(&nhist[(uint32_t)(key >> next_shift) & 255u], 1u);
      }
    }
    __syncthreads();
  }
  for (int d = t; d < RS_RADIX; d += T)
    if (next_hist && nhist[d]) atomicAdd((unsigned long long*)&next_hist[d], (unsigned long long)nhist[d]);
}

template <int T, int KPT, int RANK>
constexpr size_t onesweep3_smem() {
  return (size_t)T * KPT * 8 + RS_RADIX * 8 + (size_t)(T / 32) * RS_RADIX * 4 * (RANK != 0 ? 2 : 1) +
         2 * RS_RADIX * 4 + 32 * 4 + 16 + 32 * 4 + RS_RADIX * 8;
}

template <int T, int KPT>
constexpr size_t onesweep_smem() {
  return (size_t)(T / 32) * RS_RADIX * 4 + 3 * RS_RADIX * 4 + RS_RADIX * 8 + (size_t)T * KPT * 8 + 16 +
         RS_RADIX * 8;  // + ticket, kept, digit starts
}

// ------------------------------------------------------------------ conflict scan, phase A
// One warp walks a range of CA_RANGE sorted keys, 32 keys per step, lane =
// key.  Each lane compares its key with the previous one; ballots give the
// run starts, sub-run (interval) starts, thread changes, block changes and
// writers of the step, and bit arithmetic on those masks gives every run's
// OR-reductions.  Flags of the run and sub-run still open at the end of a
// step are carried to the next one.  A run belongs to the warp whose range
// holds its first key; the warp reads past its range to finish that run.
//   sub-run (same array, granule, interval) may race inside a block:
//       it has a writer and two different threads;
//   run (same array, granule) in global memory may race across blocks:
//       it has a writer and two different blocks.
__device__ __forceinline__ unsigned m_le(int l) { return l >= 31 ? FULL : ((2u << l) - 1u); }
__device__ __forceinline__ unsigned m_lt(int l) { return l <= 0 ? 0u : (l >= 32 ? FULL : ((1u << l) - 1u)); }
__device__ __forceinline__ int top_bit(unsigned m) { return m ? 31 - __clz(m) : -1; }

struct CandCarry {
  uint64_t prev, start;
  bool owned, runW, runBD, runC, subW, subTD, glob;  // glob: the open run is in global memory
};

struct CandCtx {
  uint64_t n, r0, r1, m_run, m_sub, m_blk, m_wv, m_t, m_w, g_lim;
  uint32_t wmask, amask;
  bool g_all;
  unsigned below;
  int lane;
  uint64_t* cand;
  uint64_t cand_cap;
  uint64_t* counters;
};

// One 32-key step at position p (keys already loaded).  Returns true when the
// warp is past its range and holds no open run of its own.
__device__ __forceinline__ bool cand_step(const CandCtx& X, CandCarry& c, uint64_t k, uint64_t p) {
  const int lane = X.lane;
  const uint64_t i = p + lane;
  const bool valid = i < X.n;
  uint64_t pk = __shfl_up_sync(FULL, k, 1);
  if (lane == 0) pk = c.prev;
  const uint64_t x = k ^ pk;
  const bool rs = valid && (i == 0 || (x & X.m_run) != 0);
  const bool ss = valid && (rs || (x & X.m_sub) != 0);
  // two instances of one sub-run that may race inside a block: another block
  // (a superset), else in one warp interval another thread, else another warp
  // (a warp barrier orders the threads of one warp only)
  const bool td = valid && !ss && ((x & X.m_blk) != 0 || (x & ((x & X.m_wv) ? X.m_w : X.m_t)) != 0);
  const bool bd = valid && !rs && (x & X.m_blk) != 0;
  const bool w = valid && ((X.wmask >> ((uint32_t)k & X.amask)) & 1u);
  const unsigned RS = __ballot_sync(FULL, rs), SS = __ballot_sync(FULL, ss), TD = __ballot_sync(FULL, td);
  const unsigned BD = __ballot_sync(FULL, bd), WM = __ballot_sync(FULL, w);
  const unsigned below = X.below;
  if (WM == 0 && !c.subW && !(c.runW && c.glob) && !c.runC) {
    // no writer in this step and none open that could still race: no run can
    // become a candidate here (in shared memory only the open sub-run's
    // writer matters); only the boundaries and the thread / block flags move on
    const int ql = top_bit(RS);
    if (ql >= 0) {
      c.start = p + ql;
      c.owned = c.start >= X.r0 && c.start < X.r1;
      c.runBD = (BD & ~m_lt(ql)) != 0;
      c.runC = false;
      c.runW = false;
      const uint64_t kq = __shfl_sync(FULL, k, ql);
      c.glob = X.g_all || kq < X.g_lim;
    } else {
      c.runBD |= BD != 0;
    }
    const int tl = top_bit(SS);
    c.subTD = tl >= 0 ? (TD & ~m_lt(tl)) != 0 : (c.subTD || TD != 0);
    const uint64_t rem = X.n - p;
    c.prev = __shfl_sync(FULL, k, rem >= 32 ? 31 : (int)rem - 1);
    if (c.owned && p + 32 - c.start > (uint64_t)CA_LONG) {  // as below: a writer may still follow
      if (lane == 0) {
        const uint64_t g = atomicAdd((unsigned long long*)&X.counters[C_NCAND], 1ull);
        if (g < X.cand_cap) {
          X.cand[2 * g] = c.start;
          X.cand[2 * g + 1] = 0;
        }
      }
      c.owned = false;
    }
    return p + 32 >= X.r1 && !c.owned;
  }
  // candidacy of the sub-run that ends just before this lane's sub-run start
  const int t = top_bit(SS & below);
  const unsigned rs_sub = t >= 0 ? (below & ~m_lt(t)) : below;
  const bool subW = (WM & rs_sub) || (t < 0 && c.subW);
  const bool subTD = (TD & rs_sub) || (t < 0 && c.subTD);
  const unsigned CS = __ballot_sync(FULL, ss && subW && subTD);
  // the run that ends just before this lane's run start
  const int q = top_bit(RS & below);
  const unsigned rw = q >= 0 ? (below & ~m_lt(q)) : below;            // [q, lane-1]
  const unsigned rc = q >= 0 ? (m_le(lane) & ~m_le(q)) : m_le(lane);  // (q, lane]
  const bool rW = (WM & rw) || (q < 0 && c.runW);
  const bool rBD = (BD & rw) || (q < 0 && c.runBD);
  const bool rC = (CS & rc) || (q < 0 && c.runC);
  const uint64_t rstart = q >= 0 ? p + q : c.start;
  const bool owned = q >= 0 ? (rstart >= X.r0 && rstart < X.r1) : c.owned;
  const bool emit = rs && i > 0 && owned && (rC || ((X.g_all || pk < X.g_lim) && rW && rBD));
  const unsigned EM = __ballot_sync(FULL, emit);
  if (EM) {
    uint64_t base = 0;
    if (lane == 0) base = atomicAdd((unsigned long long*)&X.counters[C_NCAND], (unsigned long long)__popc(EM));
    base = __shfl_sync(FULL, base, 0);
    if (emit) {
      const uint64_t g = base + __popc(EM & below);
      if (g < X.cand_cap) {
        X.cand[2 * g] = rstart;
        X.cand[2 * g + 1] = i;
      }
    }
  }
  // carries for the next step
  const int ql = top_bit(RS);
  if (ql >= 0) {
    c.start = p + ql;
    c.owned = c.start >= X.r0 && c.start < X.r1;
    c.runW = (WM & ~m_lt(ql)) != 0;
    c.runBD = (BD & ~m_lt(ql)) != 0;
    c.runC = (CS & ~m_le(ql)) != 0;
    const uint64_t kq = __shfl_sync(FULL, k, ql);
    c.glob = X.g_all || kq < X.g_lim;
  } else {
    c.runW |= WM != 0;
    c.runBD |= BD != 0;
    c.runC |= CS != 0;
  }
  const int tl = top_bit(SS);
  if (tl >= 0) {
    c.subW = (WM & ~m_lt(tl)) != 0;
    c.subTD = (TD & ~m_lt(tl)) != 0;
  } else {
    c.subW |= WM != 0;
    c.subTD |= TD != 0;
  }
  const uint64_t rem = X.n - p;  // keys left from this step on
  c.prev = __shfl_sync(FULL, k, rem >= 32 ? 31 : (int)rem - 1);
  // a run longer than CA_LONG goes to the exact scan with its end unknown
  if (c.owned && p + 32 - c.start > (uint64_t)CA_LONG) {
    if (lane == 0) {
      const uint64_t g = atomicAdd((unsigned long long*)&X.counters[C_NCAND], 1ull);
      if (g < X.cand_cap) {
        X.cand[2 * g] = c.start;
        X.cand[2 * g + 1] = 0;
      }
    }
    c.owned = false;
  }
  return p + 32 >= X.r1 && !c.owned;
}

__global__ void __launch_bounds__(CA_THREADS, 2) candidates_kernel(const uint64_t* __restrict__ keys, const uint64_t* n_dev,
                                                               const DProg* __restrict__ P, uint64_t* __restrict__ cand,
                                                               uint64_t cand_cap, uint64_t* counters) {
  CandCtx X;
  X.lane = threadIdx.x & 31;
  X.n = *n_dev;
  const int PB = P->PB, IVB = P->IVB, AB = P->AB, TB = P->TB, BB = P->BB;
  const int rsh = PB + IVB;
  X.wmask = P->wmask;
  X.amask = AB ? (1u << AB) - 1u : 0u;
  const uint64_t shbase = P->shared_cell_base;
  // field tests on k ^ previous key: run id, run+interval, block+thread, block
  X.m_run = rsh >= 64 ? 0 : ~0ull << rsh;
  X.m_sub = PB >= 64 ? 0 : ~0ull << PB;
  // block, warp-interval, thread and warp fields
  X.m_blk = lowbits(~0ull, BB) << (AB + TB + P->WVB);
  X.m_wv = lowbits(~0ull, P->WVB) << (AB + TB);
  X.m_t = lowbits(~0ull, TB) << AB;
  X.m_w = TB > 5 ? (lowbits(~0ull, TB - 5) << (AB + 5)) : 0ull;
  // keys below g_lim belong to global-memory runs
  X.g_all = rsh >= 64 ? shbase > 0 : (rsh > 0 && shbase >= (1ull << (64 - rsh)));
  X.g_lim = X.g_all ? ~0ull : (rsh >= 64 ? 0ull : shbase << rsh);
  X.below = m_lt(X.lane);
  X.cand = cand;
  X.cand_cap = cand_cap;
  X.counters = counters;
  const uint64_t n = X.n;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  // keys per warp: CA_RANGE, less when there are few keys for the warps (a
  // multiple of the keys one look-ahead step loads)
  constexpr uint64_t STEP = 32 * CA_AHEAD;
  const uint64_t want = (n + nw - 1) / nw;
  const uint64_t range = want >= (uint64_t)CA_RANGE ? (uint64_t)CA_RANGE
                                                    : (want <= 2 * STEP ? 2 * STEP : (want + STEP - 1) / STEP * STEP);
  const uint64_t nranges = (n + range - 1) / range;
  for (uint64_t rg = gw; rg < nranges; rg += nw) {
    X.r0 = rg * range;
    X.r1 = X.r0 + range;
    CandCarry c;
    c.prev = X.r0 > 0 ? keys[X.r0 - 1] : 0;
    c.start = 0;
    c.owned = c.runW = c.runBD = c.runC = c.subW = c.subTD = false;
    c.glob = X.g_all || c.prev < X.g_lim;
    bool done = false;
    // two groups of CA_AHEAD steps in flight: the next group's loads are
    // issued before the current group is scanned
    uint64_t kk[CA_AHEAD], nx[CA_AHEAD];
#pragma unroll
    for (int j = 0; j < CA_AHEAD; ++j) {
      const uint64_t i = X.r0 + 32 * j + X.lane;
      kk[j] = i < n ? __ldcs(keys + i) : 0;
    }
    for (uint64_t p = X.r0; !done && p < n; p += 32 * CA_AHEAD) {
#pragma unroll
      for (int j = 0; j < CA_AHEAD; ++j) {
        const uint64_t i = p + 32 * (CA_AHEAD + j) + X.lane;
        nx[j] = i < n ? __ldcs(keys + i) : 0;
      }
#pragma unroll
      for (int j = 0; j < CA_AHEAD; ++j)
        if (!done && p + 32 * j < n) done = cand_step(X, c, kk[j], p + 32 * j);
#pragma unroll
      for (int j = 0; j < CA_AHEAD; ++j) kk[j] = nx[j];
    }
    if (!done && c.owned) {  // the array ended inside a run of this warp
      const bool last = c.runC || (c.subW && c.subTD) || ((X.g_all || c.prev < X.g_lim) && c.runW && c.runBD);
      if (last && X.lane == 0) {
        const uint64_t g = atomicAdd((unsigned long long*)&counters[C_NCAND], 1ull);
        if (g < cand_cap) {
          cand[2 * g] = c.start;
          cand[2 * g + 1] = n;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ conflict scan, phase A, lane rows
// The same decision as candidates_kernel with each lane walking a row of 32
// consecutive keys, so the field tests run once per key on one lane instead
// of once per key on a warp-wide step.  A warp's step is 1024 keys (64 tile
// rows of 16 keys, 128 bytes each), brought to shared memory by one tensor
// copy (TMA) with the 128-byte swizzle: chunk c (16 bytes) of tile row r
// lands at chunk c ^ (r & 7).  Each warp runs its own pipeline of CB_STAGES
// steps (one mbarrier per stage) across the ranges it owns.  A warp owns the
// runs that start in its range and reads past the range end, with plain
// loads, to finish its last run.
//
// Per lane, the flags of its 32 keys become bit masks (bit j = key j: run
// start, sub-run start, writer, a new thread of the sub-run, a new block of
// the run, as in cand_step); segmented prefix ORs over the masks close the
// runs that start and end inside the row at once, and leave three parts for
// the warp: the part before the row's first sub-run start, the sub-runs
// closed before its first run start, and the part after its last run start.
// Ballots over the lanes give each lane the flags carried into its row (an
// OR over the lanes since the last start, as in candidates_kernel's steps),
// which close the run that was open at the row's start.
constexpr int CB_THREADS = 128, CB_STAGES = 2, CB_ROW = 32, CB_STEP = 32 * CB_ROW, CB_STEP_BYTES = CB_STEP * 8;
constexpr int CB_TILE_ROW = 16;  // keys per 128-byte tile row of the tensor copy
constexpr int CB_RANGE = 8 * CB_STEP;
constexpr uint32_t CB_SPIN_LIMIT = 1u << 22;

struct RowCarry {
  uint64_t prev, start;
  bool owned, runW, runBD, runC, subW, subTD;
};

__device__ __forceinline__ void cb_mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cb_issue(uint32_t bar, uint32_t dst, const CUtensorMap* tm, uint64_t row) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(CB_STEP_BYTES) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"((int32_t)row), "r"(bar)
      : "memory");
}
// bounded wait on a stage's phase (non-blocking tests, a short sleep after
// the first few; at most CB_SPIN_LIMIT tests, well under a second); false
// when the limit ran out
__device__ __forceinline__ bool cb_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t spins = 0; spins < CB_SPIN_LIMIT; ++spins) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (spins >= 8) __nanosleep(64);
  }
  return false;
}

struct RowCtx {
  uint64_t n, r0, r1, m_blk, m_wv, m_w, m_t, g_lim;
  int rsh;                          // run code: key >> rsh
  uint32_t mr_h, mr_l, ms_h, ms_l;  // run and sub-run fields (halves of ~0 << (PB + IVB), ~0 << PB)
  uint32_t m_bt;                    // block and thread fields (low word)
  const uint64_t* keys;
  uint32_t wrep;  // writer bit of each access id, repeated every 2^AB bits over the word
  bool g_all;
  int lane;
  unsigned below;
  uint64_t* cand;
  uint64_t cand_cap;
  uint64_t* counters;
};

__device__ __forceinline__ void cb_put(const RowCtx& X, uint64_t g, uint64_t s, uint64_t e) {
  if (g < X.cand_cap) {
    X.cand[2 * g] = s;
    X.cand[2 * g + 1] = e;
  }
}

// Segmented prefix OR over a row: bit p of the result is the OR of f over
// [the last start at or before p, p], bit 0 always starting a segment
// (Kogge-Stone doubling over the "continues from p - 1" mask).
__device__ __forceinline__ uint32_t seg_or(uint32_t f, uint32_t starts) {
  uint32_t c = ~starts & 0xfffffffeu;
  f |= (f << 1) & c;
  c &= c << 1;
  f |= (f << 2) & c;
  c &= c << 2;
  f |= (f << 4) & c;
  c &= c << 4;
  f |= (f << 8) & c;
  c &= c << 8;
  f |= (f << 16) & c;
  return f;
}

// Flags of 16 keys (k, the key before them pk) into bits sh .. sh + 15 of the
// row masks.  FORM 2: the run code starts in the low word (PB + IVB <= 32) and
// there are no warp intervals; FORM 1: the block, warp-interval and thread
// fields sit in the low word (PB <= 32); FORM 0: any layout.
template <int FORM>
__device__ __forceinline__ void row_flags(const RowCtx& X, const uint64_t (&k)[CB_TILE_ROW], uint64_t& pk, int sh,
                                          uint32_t& RS, uint32_t& SS, uint32_t& TD, uint32_t& BD, uint32_t& W) {
#pragma unroll
  for (int j = 0; j < CB_TILE_ROW; ++j) {
    const uint64_t key = k[j];
    const uint32_t xl = (uint32_t)key ^ (uint32_t)pk, xh = (uint32_t)(key >> 32) ^ (uint32_t)(pk >> 32);
    // writer: bit (key mod 32) of the writer bits repeated every 2^AB places
    const uint32_t wr = __funnelshift_r(X.wrep, X.wrep, (uint32_t)key) & 1u;
    const uint32_t bit = 1u << (sh + j);
    if (FORM == 2) {
      // each flag a predicate that sets its bit by a predicated OR
      const uint32_t rv = xh | (xl & X.mr_l), sv = xh | (xl & X.ms_l);
      asm("{\n\t.reg .pred prs, pss, ptd, pbd, pw;\n\t"
          "setp.ne.u32 prs, %5, 0;\n\t"
          "setp.ne.u32 pss, %6, 0;\n\t"
          "setp.ne.and.u32 ptd, %7, 0, !pss;\n\t"
          "setp.ne.and.u32 pbd, %8, 0, !prs;\n\t"
          "setp.ne.u32 pw, %9, 0;\n\t"
          "@prs or.b32 %0, %0, %10;\n\t"
          "@pss or.b32 %1, %1, %10;\n\t"
          "@ptd or.b32 %2, %2, %10;\n\t"
          "@pbd or.b32 %3, %3, %10;\n\t"
          "@pw or.b32 %4, %4, %10;\n\t}"
          : "+r"(RS), "+r"(SS), "+r"(TD), "+r"(BD), "+r"(W)
          : "r"(rv), "r"(sv), "r"(xl & X.m_bt), "r"(xl & (uint32_t)X.m_blk), "r"(wr), "r"(bit));
    } else {
      bool rs, ss, blk, wv, wp, th;
      rs = ((xh & X.mr_h) | (xl & X.mr_l)) != 0;
      ss = ((xh & X.ms_h) | (xl & X.ms_l)) != 0;
      if (FORM == 1) {
        blk = (xl & (uint32_t)X.m_blk) != 0;
        wv = (xl & (uint32_t)X.m_wv) != 0;
        wp = (xl & (uint32_t)X.m_w) != 0;
        th = (xl & (uint32_t)X.m_t) != 0;
      } else {
        const uint64_t x = ((uint64_t)xh << 32) | xl;
        blk = (x & X.m_blk) != 0;
        wv = (x & X.m_wv) != 0;
        wp = (x & X.m_w) != 0;
        th = (x & X.m_t) != 0;
      }
      const bool td = !ss && (blk || (wv ? wp : th));
      const bool bd = !rs && blk;
      if (rs) RS |= bit;
      if (ss) SS |= bit;
      if (td) TD |= bit;
      if (bd) BD |= bit;
      if (wr) W |= bit;
    }
    pk = key;
  }
}

// One step of the keys [p, p + lim) (lim <= CB_STEP; lane l's row starts at
// p + 32 l): the rows come from the step's shared-memory tile rows at srow,
// or from global memory (srow = ~0), and are flagged, closed and carried.
// own: the step lies inside the warp's range (every run starting in it
// belongs to the warp).
template <int FORM>
__device__ __forceinline__ void row_step(const RowCtx& X, RowCarry& c, uint32_t srow, uint64_t p, bool own,
                                         uint32_t lim) {
  const int lane = X.lane;
  const bool full = lim == (uint32_t)CB_STEP;
  const uint64_t end = p + lim;
  const uint64_t i0 = p + (uint64_t)lane * CB_ROW;
  uint64_t pk;
  uint32_t RS = 0, SS = 0, TD = 0, BD = 0, W = 0;
  uint64_t klast, kfirst;
  {
    // the key before the row: the last one of the lane before (lane 0: the carry)
    uint64_t prevk = 0;
    if (srow != 0xffffffffu) {
      if (lane > 0) {
        const uint32_t r = 2 * lane - 1;
        asm volatile("ld.shared.u64 %0, [%1];" : "=l"(prevk) : "r"(srow + r * 128u + (((7u ^ (r & 7u)) << 4) | 8u)));
      }
    } else if (lane > 0 && i0 < end) {
      prevk = X.keys[i0 - 1];
    }
    pk = lane == 0 ? (i0 == 0 ? ~0ull : c.prev) : prevk;
  }
  const uint64_t pk0 = pk;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint64_t k[CB_TILE_ROW];
    if (srow != 0xffffffffu) {
      const uint32_t r = 2 * (uint32_t)lane + h;
      const uint32_t base = srow + r * 128u;
#pragma unroll
      for (int ch = 0; ch < CB_TILE_ROW / 2; ++ch)
        asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];"
                     : "=l"(k[2 * ch]), "=l"(k[2 * ch + 1])
                     : "r"(base + ((((uint32_t)ch) ^ (r & 7u)) << 4)));
    } else {
      const uint64_t r = i0 + (uint64_t)h * CB_TILE_ROW;
#pragma unroll
      for (int j = 0; j < CB_TILE_ROW; ++j) k[j] = r + j < end ? X.keys[r + j] : 0;
    }
    if (h == 0) {
      kfirst = k[0];
      if (i0 == 0) pk = ~k[0];  // the array's first key starts a run
    }
    row_flags<FORM>(X, k, pk, 16 * h, RS, SS, TD, BD, W);
    if (h == 1) klast = k[CB_TILE_ROW - 1];
  }
  if (!full) {  // positions past the array's end take no part
    const uint64_t rem = i0 < end ? end - i0 : 0;
    const uint32_t VM = rem >= (uint64_t)CB_ROW ? 0xffffffffu : ((1u << rem) - 1u);
    RS &= VM;
    SS &= VM;
    TD &= VM;
    BD &= VM;
    W &= VM;
  }
  // global-memory runs: keys below g_lim (monotone in the sorted order; a
  // row's last key counts only when the whole row lies below the end)
  uint32_t GL;
  if (X.g_all || (full && klast < X.g_lim)) {
    GL = 0xffffffffu;
  } else if (kfirst >= X.g_lim) {
    GL = 0;
  } else {  // the row may cross into the shared arrays: find where
    GL = 0;
    for (int j = 0; j < CB_ROW; ++j) {
      uint64_t kj;
      if (srow != 0xffffffffu) {
        const uint32_t r = 2 * (uint32_t)lane + (j >> 4), ch = (uint32_t)(j & 15) >> 1;
        asm volatile("ld.shared.u64 %0, [%1];"
                     : "=l"(kj)
                     : "r"(srow + r * 128u + (((ch ^ (r & 7u)) << 4) | (uint32_t)((j & 1) << 3))));
      } else {
        kj = i0 + j < end ? X.keys[i0 + j] : ~0ull;
      }
      if (kj < X.g_lim) GL |= 1u << j;
    }
  }
  const bool gprev = X.g_all || pk0 < X.g_lim;
  const bool seenSS = SS != 0, seenRS = RS != 0;
  const uint32_t lt_fSS = seenSS ? (SS & (0u - SS)) - 1u : 0xffffffffu;  // before the first sub-run start
  const uint32_t lt_fRS = seenRS ? (RS & (0u - RS)) - 1u : 0xffffffffu;  // before the first run start
  const int lRS = seenRS ? 31 - __clz(RS) : 0;
  const uint32_t ge_lSS = seenSS ? ~((1u << (31 - __clz(SS))) - 1u) : 0xffffffffu;  // from the last one on
  const uint32_t ge_lRS = seenRS ? ~((1u << lRS) - 1u) : 0xffffffffu;
  // sub-runs: writer and new thread so far, and the ends of the sub-runs that
  // start and end inside the row that may race
  const uint32_t SC = seg_or(W, SS) & seg_or(TD, SS) & (SS >> 1) & ~lt_fSS;
  // runs: writer and new block so far, and any racing sub-run so far; runs
  // that start and end inside the row end at the positions before a run start
  const uint32_t em =
      own ? ((RS >> 1) & ~lt_fRS & (seg_or(SC, RS) | (GL & seg_or(W, RS) & seg_or(BD, RS)))) : 0u;
  const bool preSW = (W & lt_fSS) != 0, preSTD = (TD & lt_fSS) != 0;
  const bool preRW = (W & lt_fRS) != 0, preRBD = (BD & lt_fRS) != 0, preRC = (SC & lt_fRS) != 0;
  const int fRS = seenRS ? __ffs(RS) - 1 : 0;
  const bool preG = fRS == 0 ? gprev : ((GL >> (fRS - 1)) & 1u) != 0;
  // flags carried into each row: OR over the lanes since the last start
  const unsigned below = X.below;
  const unsigned SSL = __ballot_sync(FULL, seenSS), RSL = __ballot_sync(FULL, seenRS);
  const unsigned BSW = __ballot_sync(FULL, (W & ge_lSS) != 0), BSTD = __ballot_sync(FULL, (TD & ge_lSS) != 0);
  const int qs = top_bit(SSL & below);
  const unsigned rg_s = qs >= 0 ? (below & ~m_lt(qs)) : below;
  const bool inSW = (BSW & rg_s) != 0 || (qs < 0 && c.subW);
  const bool inSTD = (BSTD & rg_s) != 0 || (qs < 0 && c.subTD);
  // the sub-run open at the row's start, closed inside the row
  const bool firstSubC = seenSS && (inSW || preSW) && (inSTD || preSTD);
  const bool sufRC = (SC & ge_lRS) != 0 || (!seenRS && firstSubC);
  const unsigned BRW = __ballot_sync(FULL, (W & ge_lRS) != 0), BRBD = __ballot_sync(FULL, (BD & ge_lRS) != 0);
  const unsigned BRC = __ballot_sync(FULL, sufRC);
  const int qr = top_bit(RSL & below);
  const unsigned rg_r = qr >= 0 ? (below & ~m_lt(qr)) : below;
  const bool inRW = (BRW & rg_r) != 0 || (qr < 0 && c.runW);
  const bool inRBD = (BRBD & rg_r) != 0 || (qr < 0 && c.runBD);
  const bool inRC = (BRC & rg_r) != 0 || (qr < 0 && c.runC);
  const uint32_t lastOff = (uint32_t)lane * CB_ROW + (uint32_t)lRS;  // the last run start, from p
  const uint32_t srcOff = __shfl_sync(FULL, lastOff, qr >= 0 ? qr : 0);
  const uint64_t inStart = qr >= 0 ? p + srcOff : c.start;
  const bool inOwned = qr >= 0 ? own : c.owned;
  const bool firstEmit =
      seenRS && inOwned && (inRC || preRC || firstSubC || (preG && (inRW || preRW) && (inRBD || preRBD)));
  // candidate entries: one atomic per lane that has any
  const uint32_t cnt = (uint32_t)__popc(em) + (firstEmit ? 1u : 0u);
  if (cnt) {
    uint64_t base = atomicAdd((unsigned long long*)&X.counters[C_NCAND], (unsigned long long)cnt);
    if (firstEmit) cb_put(X, base++, inStart, i0 + (uint64_t)fRS);
    for (uint32_t m = em; m; m &= m - 1) {
      const int e = __ffs(m) - 1;                       // the run's last key
      const int s = 31 - __clz(RS & ((2u << e) - 1u));  // its first: the last run start at or before e
      cb_put(X, base++, i0 + (uint64_t)s, i0 + (uint64_t)e + 1);
    }
  }
  // carries for the next step: the lanes from the last start on
  const int ql = top_bit(RSL);
  if (ql >= 0) {
    c.start = p + __shfl_sync(FULL, lastOff, ql);
    c.owned = own;
    const unsigned up = ~m_lt(ql);
    c.runW = (BRW & up) != 0;
    c.runBD = (BRBD & up) != 0;
    c.runC = (BRC & up) != 0;
  } else {
    c.runW |= BRW != 0;
    c.runBD |= BRBD != 0;
    c.runC |= BRC != 0;
  }
  const int qsl = top_bit(SSL);
  if (qsl >= 0) {
    const unsigned up = ~m_lt(qsl);
    c.subW = (BSW & up) != 0;
    c.subTD = (BSTD & up) != 0;
  } else {
    c.subW |= BSW != 0;
    c.subTD |= BSTD != 0;
  }
  // the step's last key
  c.prev = full ? __shfl_sync(FULL, klast, 31) : X.keys[end - 1];
  // a run longer than CA_LONG goes to the exact scan with its end unknown
  if (c.owned && end - c.start > (uint64_t)CA_LONG) {
    if (lane == 0) {
      const uint64_t g = atomicAdd((unsigned long long*)&X.counters[C_NCAND], 1ull);
      cb_put(X, g, c.start, 0);
    }
    c.owned = false;
  }
}

template <int FORM>
__device__ __forceinline__ void scan_ranges(const CUtensorMap* tmap, RowCtx& X, uint64_t gw, uint64_t nw,
                                            uint64_t range, uint64_t nr_w, uint32_t buf0, uint32_t bar0,
                                            uint64_t* counters) {
  const int lane = X.lane;
  const uint64_t n = X.n;
  const uint32_t spr = (uint32_t)(range / CB_STEP);
  const uint64_t last_r0 = (gw + (nr_w - 1) * nw) * range;
  const uint64_t last_r1 = last_r0 + range < n ? last_r0 + range : n;
  const uint64_t nq = (nr_w - 1) * spr + (last_r1 - last_r0 + CB_STEP - 1) / CB_STEP;  // steps of this warp
  // the producer walks the same step sequence CB_STAGES steps ahead: first
  // tile row of the next step to load, and its place in its range
  uint64_t nrow = gw * range / CB_TILE_ROW, nrange_row = nrow;
  uint32_t nstep = 0;
  auto advance = [&]() {
    if (++nstep == spr) {
      nstep = 0;
      nrange_row += nw * range / CB_TILE_ROW;
      nrow = nrange_row;
    } else {
      nrow += CB_STEP / CB_TILE_ROW;
    }
  };
  if (lane == 0) {
    for (int s = 0; s < CB_STAGES; ++s) cb_mbar_init(bar0 + 8 * s);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  uint64_t issued = 0;
  for (; issued < CB_STAGES && issued < nq; ++issued) {
    if (lane == 0) cb_issue(bar0 + 8 * (uint32_t)issued, buf0 + (uint32_t)issued * CB_STEP_BYTES, tmap, nrow);
    advance();
  }
  __syncwarp();
  bool failed = false;
  uint64_t q = 0;
  for (uint64_t m = 0; m < nr_w && !failed; ++m) {
    X.r0 = (gw + m * nw) * range;
    X.r1 = X.r0 + range < n ? X.r0 + range : n;
    RowCarry c;
    c.prev = X.r0 > 0 ? X.keys[X.r0 - 1] : 0;
    c.start = 0;
    c.owned = c.runW = c.runBD = c.runC = c.subW = c.subTD = false;
    uint64_t p = X.r0;
    for (; p < X.r1; p += CB_STEP, ++q) {
      const uint32_t st = (uint32_t)q % CB_STAGES;
      if (!cb_wait(bar0 + 8 * st, (uint32_t)(q / CB_STAGES) & 1u)) {
        failed = true;
        break;
      }
      const uint32_t srow = buf0 + st * CB_STEP_BYTES;
      row_step<FORM>(X, c, srow, p, true, p + CB_STEP <= n ? (uint32_t)CB_STEP : (uint32_t)(n - p));
      // the stage is free again (its keys are consumed): the step CB_STAGES ahead
      __syncwarp();
      if (issued < nq) {
        if (lane == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          cb_issue(bar0 + 8 * st, buf0 + st * CB_STEP_BYTES, tmap, nrow);
        }
        ++issued;
        advance();
      }
    }
    if (failed) break;
    if (!c.owned) continue;
    // past the range: the warp's last run ends at e, the first key of another
    // run (found 32 keys at a time), or at the array's end; its keys past the
    // range are flagged with plain loads, then the run is closed
    uint64_t e = p;
    bool found = false;
    const uint64_t rid = shr64(c.prev, X.rsh);
    while (!found && e < n && e - c.start <= (uint64_t)CA_LONG) {
      const uint64_t i = e + (uint64_t)lane;
      const unsigned other = __ballot_sync(FULL, i < n && shr64(X.keys[i], X.rsh) != rid);
      if (other) {
        e += (uint64_t)(__ffs(other) - 1);
        found = true;
      } else {
        e = e + 32 < n ? e + 32 : n;
      }
    }
    for (; c.owned && p < e; p += CB_STEP)
      row_step<FORM>(X, c, 0xffffffffu, p, false, p + CB_STEP <= e ? (uint32_t)CB_STEP : (uint32_t)(e - p));
    if (c.owned && lane == 0) {
      if (!found && e < n) {  // longer than CA_LONG: the exact scan finds the end
        const uint64_t g = atomicAdd((unsigned long long*)&counters[C_NCAND], 1ull);
        cb_put(X, g, c.start, 0);
      } else if (c.runC || (c.subW && c.subTD) || ((X.g_all || c.prev < X.g_lim) && c.runW && c.runBD)) {
        const uint64_t g = atomicAdd((unsigned long long*)&counters[C_NCAND], 1ull);
        cb_put(X, g, c.start, e);
      }
    }
  }
  if (failed) {
    if (lane == 0) atomicOr((unsigned long long*)&counters[C_ERR], (unsigned long long)ERR_TIMEOUT);
    // copies still in flight land before the CTA leaves (each wait bounded)
    for (uint64_t r = q; r < issued; ++r)
      if (!cb_wait(bar0 + 8 * (uint32_t)(r % CB_STAGES), (uint32_t)(r / CB_STAGES) & 1u)) break;
  }
}

__global__ void __launch_bounds__(CB_THREADS) candidates_rows_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                    const uint64_t* __restrict__ keys,
                                                                    const uint64_t* n_dev, const DProg* __restrict__ P,
                                                                    uint64_t* __restrict__ cand, uint64_t cand_cap,
                                                                    uint64_t* counters) {
  extern __shared__ __align__(16) unsigned char cbsm[];
  __shared__ __align__(8) uint64_t bars[CB_THREADS / 32][CB_STAGES];
  RowCtx X;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  X.lane = lane;
  X.below = m_lt(lane);
  X.n = *n_dev;
  const int PB = P->PB, IVB = P->IVB, AB = P->AB, TB = P->TB, BB = P->BB, WVB = P->WVB;
  const int rsh = PB + IVB;
  const uint64_t m_run = rsh >= 64 ? 0 : ~0ull << rsh, m_sub = PB >= 64 ? 0 : ~0ull << PB;
  X.rsh = rsh;
  X.mr_h = (uint32_t)(m_run >> 32);
  X.mr_l = (uint32_t)m_run;
  X.ms_h = (uint32_t)(m_sub >> 32);
  X.ms_l = (uint32_t)m_sub;
  X.keys = keys;
  X.wrep = P->wmask;
  for (int sh = 1 << AB; sh < 32; sh <<= 1) X.wrep |= X.wrep << sh;
  X.m_blk = lowbits(~0ull, BB) << (AB + TB + WVB);
  X.m_wv = lowbits(~0ull, WVB) << (AB + TB);
  X.m_t = lowbits(~0ull, TB) << AB;
  X.m_w = TB > 5 ? (lowbits(~0ull, TB - 5) << (AB + 5)) : 0ull;
  X.m_bt = (uint32_t)(X.m_blk | X.m_t);
  const uint64_t shbase = P->shared_cell_base;
  X.g_all = rsh >= 64 ? shbase > 0 : (rsh > 0 && shbase >= (1ull << (64 - rsh)));
  X.g_lim = X.g_all ? ~0ull : (rsh >= 64 ? 0ull : shbase << rsh);
  X.cand = cand;
  X.cand_cap = cand_cap;
  X.counters = counters;
  const uint64_t n = X.n;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  // keys per range: CB_RANGE, fewer (whole steps) when there are few keys for the warps
  const uint64_t want = (n + nw - 1) / nw;
  const uint64_t range = want >= (uint64_t)CB_RANGE
                             ? (uint64_t)CB_RANGE
                             : ((want + CB_STEP - 1) / CB_STEP > 0 ? (want + CB_STEP - 1) / CB_STEP : 1) * CB_STEP;
  const uint64_t nranges = (n + range - 1) / range;
  if (gw >= nranges) return;
  const uint64_t nr_w = (nranges - 1 - gw) / nw + 1;  // ranges of this warp
  // the warp's stages: 1024-byte aligned in the shared window (the swizzle pattern repeats every 1024 bytes)
  const uint32_t sm0 = (uint32_t)__cvta_generic_to_shared(cbsm);
  const uint32_t buf0 = ((sm0 + 1023u) & ~1023u) + (uint32_t)wib * CB_STAGES * CB_STEP_BYTES;
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[wib][0]);
  if (rsh < 32 && WVB == 0) scan_ranges<2>(&tmap, X, gw, nw, range, nr_w, buf0, bar0, counters);
  else if (PB <= 32) scan_ranges<1>(&tmap, X, gw, nw, range, nr_w, buf0, bar0, counters);
  else scan_ranges<0>(&tmap, X, gw, nw, range, nr_w, buf0, bar0, counters);
}

// ------------------------------------------------------------------ conflict scan, phase B
// Exact kinds of one candidate bin of the block-local mode: keys [s, e) of one
// shared granule, one interval and one block, in any order.  Lane = access a:
// min / max warp of a over the bin and, per warp w, min / max thread of a in
// w, kept in the warp's shared-memory tables (reset to empty after use).
// Diff-warp pairs come from the warp sums, same-warp pairs from the thread
// sums of each warp present (Table 2, intra-block kinds).
struct BinTables {
  uint32_t tlo[32 * 32], thi[32 * 32], wlo[32], whi[32];
};
__device__ __forceinline__ void bin_tables_reset(BinTables* T, int lane) {
  for (int i = lane; i < 32 * 32; i += 32) {
    T->tlo[i] = 0xffffffffu;
    T->thi[i] = 0;
  }
  T->wlo[lane] = 0xffffffffu;
  T->whi[lane] = 0;
  __syncwarp();
}
__device__ __forceinline__ RunMasks exact_bin(const uint64_t* keys, uint64_t s, uint64_t e,
                                              const DProg* __restrict__ P, int lane, uint32_t eintra, BinTables* T) {
  const int PB = P->PB, IVB = P->IVB, AB = P->AB, TB = P->TB;
  RunMasks R;
  R.rid = shr64(keys[s], PB + IVB);
  uint32_t pw = 0;  // warps present
  for (uint64_t pos = s; pos < e; pos += 32) {
    const uint64_t i = pos + lane;
    uint32_t bit = 0;
    if (i < e) {
      const uint64_t key = keys[i];
      const uint32_t t = (uint32_t)lowbits(key >> AB, TB);
      const uint32_t a = (uint32_t)lowbits(key, AB);
      const uint32_t w = t >> 5;
      atomicMin(&T->tlo[a * 32 + w], t);
      atomicMax(&T->thi[a * 32 + w], t);
      atomicMin(&T->wlo[a], w);
      atomicMax(&T->whi[a], w);
      bit = 1u << w;
    }
    pw |= __reduce_or_sync(FULL, bit);
  }
  __syncwarp();
  Sum ws;
  ws.p = T->wlo[lane] <= T->whi[lane];
  ws.lo = T->wlo[lane];
  ws.hi = T->whi[lane];
  R.blk = racy_row(ws, lane) & eintra;
  R.warp = 0;
  for (uint32_t m = pw; m; m &= m - 1) {
    const int w = __ffs(m) - 1;
    Sum ts;
    ts.lo = T->tlo[lane * 32 + w];
    ts.hi = T->thi[lane * 32 + w];
    ts.p = ts.lo <= ts.hi;
    R.warp |= racy_row(ts, lane) & eintra;
    T->tlo[lane * 32 + w] = 0xffffffffu;
    T->thi[lane * 32 + w] = 0;
  }
  T->wlo[lane] = 0xffffffffu;
  T->whi[lane] = 0;
  R.inter = 0;
  __syncwarp();
  return R;
}

// Entries of the block-local mode's candidate bins carry SHARED_ENTRY and
// offsets relative to the first shared key, which sits right after the
// counters[C_NG] written global keys (the *n_dev sorted ones unless the cell
// filter dropped some); their kinds come from exact_bin and the warp's tables
// in dynamic shared memory (launched with `bins` set).
__global__ void __launch_bounds__(256) exact_kernel(const uint64_t* __restrict__ keys, const uint64_t* n_dev,
                                                    const DProg* __restrict__ P, const uint64_t* __restrict__ cand,
                                                    uint64_t cand_cap, uint64_t* __restrict__ raw, uint64_t raw_cap,
                                                    uint64_t* counters, int stop_first, int bins) {
  extern __shared__ __align__(16) unsigned char xsm[];
  const int lane = threadIdx.x & 31;
  const uint64_t n = *n_dev;
  // candidate-bin keys sit behind all written global keys (counters[C_NG]),
  // which is n unless the cell filter dropped some before the sort
  const uint64_t nsb = counters[C_NG];
  uint64_t ncand = counters[C_NCAND];
  if (ncand > cand_cap) ncand = cand_cap;
  const uint32_t einter = lane < P->nacc ? P->einter[lane] : 0u;
  const uint32_t eintra = lane < P->nacc ? P->eintra[lane] : 0u;
  BinTables* T = bins ? reinterpret_cast<BinTables*>(xsm) + (threadIdx.x >> 5) : nullptr;
  if (bins) bin_tables_reset(T, lane);
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t c = gw; c < ncand; c += nw) {
    if (stop_first && *(volatile uint64_t*)&counters[C_NRAW] != 0) break;
    const uint64_t c0 = cand[2 * c], c1 = cand[2 * c + 1];
    const RunMasks R = (c0 & SHARED_ENTRY)
                           ? exact_bin(keys, nsb + (c0 & ~SHARED_ENTRY), nsb + c1, P, lane, eintra, T)
                           : exact_run(keys, c0, c1, n, P, lane, einter, eintra, stop_first != 0);
    if (R.lock_overflow && lane == 0) atomicOr((unsigned long long*)&counters[C_ERR], (unsigned long long)ERR_LOCK_RUN);
    record_pairs(counters + C_PAIRS, R, lane);
    uint32_t row = witness_row(R, lane);
    const uint32_t cntw = (uint32_t)__popc(row);
    uint32_t incl = cntw;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    if (total == 0) continue;
    uint64_t wbase = 0;
    if (lane == 0) wbase = atomicAdd((unsigned long long*)&counters[C_NRAW], (unsigned long long)total);
    wbase = __shfl_sync(FULL, wbase, 0);
    uint32_t space, arr;
    uint64_t gran;
    run_location(P, R.rid, &space, &arr, &gran);
    uint64_t o = wbase + incl - cntw;
    while (row) {
      const int bb = __ffs(row) - 1;
      row &= row - 1;
      if (o < raw_cap) raw[o] = pack_witness(space, arr, gran, (uint32_t)lane, (uint32_t)bb, witness_kind(R, bb));
      ++o;
    }
  }
}

// ------------------------------------------------------------------ pair search: blocks of the witness's run
// The instances on a global-memory witness's granule are the keys of its run
// in the sorted stream, so only their blocks need the pair search.  One CTA
// finds the run (warp 0: 32 probes per step, the count of probes below the
// target narrows the range 33-fold), collects its blocks (runs of at most
// PB_MAX keys; longer runs, and shared-memory witnesses, leave
// counters[C_NPB] at 0: every unit is searched), sorts them, drops repeats,
// and lists them in `blocks`.
constexpr int PB_MAX = 4096;
__device__ __forceinline__ uint64_t first_at_or_above(const uint64_t* keys, uint64_t n, int sh, uint64_t target,
                                                     int lane) {
  uint64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const uint64_t step = (hi - lo) / 33;
    const uint64_t p = lo + (uint64_t)(lane + 1) * step;  // < hi for every lane
    const uint32_t c = (uint32_t)__popc(__ballot_sync(FULL, shr64(keys[p], sh) < target));
    const uint64_t nlo = c ? lo + (uint64_t)c * step + 1 : lo;
    const uint64_t nhi = c < 32 ? lo + (uint64_t)(c + 1) * step : hi;
    lo = nlo;
    hi = nhi;
  }
  const bool below = lo + lane < hi && shr64(keys[lo + lane], sh) < target;
  return lo + (uint64_t)__popc(__ballot_sync(FULL, below));
}

__global__ void __launch_bounds__(256) pair_blocks_kernel(const uint64_t* __restrict__ keys, const uint64_t* n_dev,
                                                          const DProg* __restrict__ P,
                                                          const uint64_t* __restrict__ uniq, uint64_t* counters,
                                                          uint64_t* __restrict__ blocks) {
  __shared__ uint64_t sb[PB_MAX];
  __shared__ uint64_t s_run[2];
  if (counters[C_NUNIQ] == 0) return;
  const uint64_t w0 = uniq[0];
  if ((w0 >> 58) & 1) return;
  const uint32_t arr = (uint32_t)(w0 >> 53) & 31;
  const uint64_t gran = (w0 >> 13) & ((1ull << 40) - 1);
  int li = -1;
  for (int l = 0; l < P->nlay; ++l)
    if (P->lay_arr[l] == (int32_t)arr && !P->lay_shared[l]) li = l;
  if (li < 0) return;
  const uint64_t cell = P->lay_cbase[li] + gran;
  const uint64_t n = *n_dev;  // sorted keys
  const int sh = P->PB + P->IVB;
  if (threadIdx.x < 32) {
    const uint64_t lo = first_at_or_above(keys, n, sh, cell, threadIdx.x);
    const uint64_t hi = first_at_or_above(keys, n, sh, cell + 1, threadIdx.x);
    if (threadIdx.x == 0) {
      s_run[0] = lo;
      s_run[1] = hi;
    }
  }
  __syncthreads();
  const uint64_t lo = s_run[0], hi = s_run[1];
  if (hi <= lo || hi - lo > (uint64_t)PB_MAX) return;
  const uint32_t m = (uint32_t)(hi - lo);
  uint32_t p2 = 1;
  while (p2 < m) p2 <<= 1;
  const int bsh = P->AB + P->TB + P->WVB;  // block field
  for (uint32_t i = threadIdx.x; i < p2; i += 256) sb[i] = i < m ? lowbits(keys[lo + i] >> bsh, P->BB) : ~0ull;
  __syncthreads();
  for (uint32_t k = 2; k <= p2; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < p2; i += 256) {
        const uint32_t x = i ^ j;
        if (x > i) {
          const uint64_t a = sb[i], b = sb[x];
          if ((a > b) == ((i & k) == 0)) {
            sb[i] = b;
            sb[x] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    uint32_t c = 0;
    for (uint32_t i = 0; i < m; ++i)
      if (i == 0 || sb[i] != sb[i - 1]) blocks[c++] = sb[i];
    counters[C_NPB] = (uint64_t)c + 1;
  }
}

// ------------------------------------------------------------------ witness merge
__global__ void heads_kernel(const uint64_t* __restrict__ w, const uint64_t* n_dev, uint64_t n_max,
                             uint64_t* __restrict__ flags) {
  const uint64_t n = dev_n(n_dev, n_max);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || (w[i] >> WIT_SORT_LO) != (w[i - 1] >> WIT_SORT_LO)) ? 1 : 0;
}

__global__ void merge_kernel(const uint64_t* __restrict__ w, const uint64_t* __restrict__ flags,
                             const uint64_t* __restrict__ excl, const uint64_t* n_dev, uint64_t n_max,
                             uint64_t* __restrict__ uniq) {
  const uint64_t n = dev_n(n_dev, n_max);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t u = excl[i] + flags[i] - 1;
    atomicOr((unsigned long long*)&uniq[u], (unsigned long long)w[i]);
  }
}

__global__ void witness_split_kernel(uint64_t* counters, uint64_t raw_cap) {
  uint64_t n = counters[C_NRAW];
  if (n > raw_cap) n = raw_cap;
  counters[C_NRAWBIG] = n > (uint64_t)WSMALL_MAX ? n : 0;
}

// the same decision inside a graph: it also opens (1) or keeps shut (0) the
// conditional node holding the device-wide merge
__global__ void witness_split_cond_kernel(uint64_t* counters, uint64_t raw_cap, cudaGraphConditionalHandle h) {
  uint64_t n = counters[C_NRAW];
  if (n > raw_cap) n = raw_cap;
  const bool big = n > (uint64_t)WSMALL_MAX;
  counters[C_NRAWBIG] = big ? n : 0;
  cudaGraphSetConditional(h, big ? 1u : 0u);
}

__global__ void zero_status_kernel(uint64_t* __restrict__ status, const uint64_t* n_dev, uint64_t max_words) {
  const uint64_t n = *n_dev;
  uint64_t words = (n + RS_MIN_TILE - 1) / RS_MIN_TILE * RS_RADIX;
  if (words > max_words) words = max_words;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
    status[i] = 0;
}

__global__ void zero_kernel(uint64_t* __restrict__ p, const uint64_t* n_dev, uint64_t n_max) {
  const uint64_t n = dev_n(n_dev, n_max);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

// Up to WSMALL_MAX raw witnesses are merged in two steps: the packed words
// are sorted by rank across the GPU into a scratch buffer (the kind mask
// sits in the lowest bits, so the words of one (space, array, granule,
// acc_lo, acc_hi) end up adjacent and in canonical order), then one CTA
// writes one output word per group with the kinds OR-ed.
__global__ void __launch_bounds__(CR_T) witness_rank_kernel(const uint64_t* __restrict__ raw,
                                                           uint64_t* __restrict__ sorted, const uint64_t* counters,
                                                           uint64_t raw_cap) {
  __shared__ uint64_t s[WSMALL_MAX];
  uint64_t n64 = counters[C_NRAW];
  if (n64 > raw_cap) n64 = raw_cap;
  if (n64 == 0 || n64 > (uint64_t)WSMALL_MAX) return;
  rank_place(raw, sorted, (uint32_t)n64, s);
}

__global__ void __launch_bounds__(1024) witness_small_kernel(const uint64_t* __restrict__ sorted,
                                                             uint64_t* __restrict__ uniq, uint64_t* counters,
                                                             uint64_t raw_cap) {
  __shared__ uint64_t s[WSMALL_MAX];
  __shared__ uint32_t wsum[32];
  uint64_t n64 = counters[C_NRAW];
  if (n64 > raw_cap) n64 = raw_cap;
  if (n64 == 0 || n64 > (uint64_t)WSMALL_MAX) return;
  const uint32_t n = (uint32_t)n64;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint32_t i = tid; i < n; i += 1024) s[i] = sorted[i];
  __syncthreads();
  // group heads over contiguous chunks, a CTA-wide exclusive scan of their counts
  const uint32_t chunk = (n + 1023) / 1024;
  const uint32_t c0 = min(n, tid * chunk), c1 = min(n, c0 + chunk);
  uint32_t heads = 0;
  for (uint32_t i = c0; i < c1; ++i) heads += (i == 0 || (s[i] >> WIT_SORT_LO) != (s[i - 1] >> WIT_SORT_LO)) ? 1u : 0u;
  uint32_t x = heads;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = wsum[lane];
    uint32_t t = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, t, o);
      if (lane >= (uint32_t)o) t += y;
    }
    wsum[lane] = t - v;
    if (lane == 31) counters[C_NUNIQ] = t;
  }
  __syncthreads();
  uint32_t u = wsum[warp] + x - heads;
  uint32_t k0 = 0, k1 = 0, k2 = 0;  // witnesses of each race kind
  for (uint32_t i = c0; i < c1; ++i) {
    if (!(i == 0 || (s[i] >> WIT_SORT_LO) != (s[i - 1] >> WIT_SORT_LO))) continue;
    uint64_t w = s[i];
    for (uint32_t j = i + 1; j < n && (s[j] >> WIT_SORT_LO) == (s[i] >> WIT_SORT_LO); ++j) w |= s[j];
    uniq[u++] = w;
    k0 += (uint32_t)w & 1u;
    k1 += (uint32_t)(w >> 1) & 1u;
    k2 += (uint32_t)(w >> 2) & 1u;
  }
  for (int o = 16; o; o >>= 1) {
    k0 += __shfl_down_sync(FULL, k0, o);
    k1 += __shfl_down_sync(FULL, k1, o);
    k2 += __shfl_down_sync(FULL, k2, o);
  }
  if (lane == 0) {
    if (k0) atomicAdd((unsigned long long*)&counters[C_KIND0], (unsigned long long)k0);
    if (k1) atomicAdd((unsigned long long*)&counters[C_KIND1], (unsigned long long)k1);
    if (k2) atomicAdd((unsigned long long*)&counters[C_KIND2], (unsigned long long)k2);
  }
}

__global__ void kind_counts_kernel(const uint64_t* __restrict__ uniq, uint64_t* counters, const uint64_t* gate) {
  if (*gate == 0) return;  // the one-CTA merge counted them
  const uint64_t n = counters[C_NUNIQ];
  uint64_t c0 = 0, c1 = 0, c2 = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = uniq[i] & 7;
    c0 += k & 1;
    c1 += (k >> 1) & 1;
    c2 += (k >> 2) & 1;
  }
  for (int o = 16; o; o >>= 1) {
    c0 += __shfl_down_sync(FULL, c0, o);
    c1 += __shfl_down_sync(FULL, c1, o);
    c2 += __shfl_down_sync(FULL, c2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c0) atomicAdd((unsigned long long*)&counters[C_KIND0], (unsigned long long)c0);
    if (c1) atomicAdd((unsigned long long*)&counters[C_KIND1], (unsigned long long)c1);
    if (c2) atomicAdd((unsigned long long*)&counters[C_KIND2], (unsigned long long)c2);
  }
}

int occupancy_grid(const void* fn, int threads, size_t smem, int nsm) { return resident_ctas(fn, threads, smem) * nsm; }

}  // namespace

// ------------------------------------------------------------------ launch-attribute caches
// The dynamic shared-memory limit set on each kernel and its resident CTAs
// per SM, per device: the runtime queries behind them cost microseconds of
// host time on every launch otherwise.
namespace {
std::mutex g_attr_mu;
std::map<std::tuple<int, const void*>, size_t> g_smem_set;
std::map<std::tuple<int, const void*, int, size_t>, int> g_resident;
int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev;
}
}  // namespace

cudaError_t allow_smem(const void* fn, size_t smem) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_attr_mu);
  size_t& have = g_smem_set[std::make_tuple(dev, fn)];
  if (smem <= have) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) have = smem;
  return e;
}

int resident_ctas(const void* fn, int threads, size_t smem) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto key = std::make_tuple(dev, fn, threads, smem);
  auto it = g_resident.find(key);
  if (it != g_resident.end()) return it->second;
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  if (per < 1) per = 1;
  g_resident[key] = per;
  return per;
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_expand(const Launch& L, int mode, bool wide, const DProg* d_prog, const DProg& h_prog,
                          uint64_t* unit_cnt, const uint64_t* unit_off, uint64_t* keys, uint64_t* hist, int npass,
                          uint64_t* counters, const uint64_t* uniq, PairRec* pairs, uint64_t pair_cap,
                          const uint32_t* ctab, uint64_t* cbuf, uint64_t ccap) {
  const size_t esz = wide ? 8 : 4;
  const size_t smem = sizeof(DProg) + (size_t)(EXP_THREADS / 32) * h_prog.nslot * 32 * esz +
                      (mode == 0 ? (size_t)npass * 256 * 4 : 0);
  const void* fn = nullptr;
  if (!wide) {
    fn = mode == 0   ? (const void*)expand_kernel<int32_t, 0>
         : mode == 1 ? (const void*)expand_kernel<int32_t, 1>
                     : (const void*)expand_kernel<int32_t, 2>;
  } else {
    fn = mode == 0   ? (const void*)expand_kernel<int64_t, 0>
         : mode == 1 ? (const void*)expand_kernel<int64_t, 1>
                     : (const void*)expand_kernel<int64_t, 2>;
  }
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  const int64_t need = (h_prog.nunits + EXP_THREADS / 32 - 1) / (EXP_THREADS / 32);
  int64_t grid = occupancy_grid(fn, EXP_THREADS, smem, L.nsm);
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  void* args[] = {(void*)&d_prog, (void*)&unit_cnt, (void*)&unit_off, (void*)&keys,     (void*)&hist,
                  (void*)&npass,  (void*)&counters, (void*)&uniq,     (void*)&pairs,    (void*)&pair_cap,
                  (void*)&ctab,   (void*)&cbuf,     (void*)&ccap};
  (*L.launches)++;
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(EXP_THREADS), args, smem, L.s);
}

cudaError_t launch_scan(const Launch& L, const uint64_t* in, uint64_t* out, const uint64_t* n_dev, uint64_t n_max,
                        uint64_t* partials, uint64_t* total) {
  uint64_t tiles = (n_max + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 0) tiles = 1;
  unsigned grid = (unsigned)(tiles < (uint64_t)L.nsm * 8 ? tiles : (uint64_t)L.nsm * 8);
  if (tiles <= SCAN_FUSE_TILES) {
    scan_reduce<<<grid, 256, 0, L.s>>>(in, n_dev, n_max, partials);
    scan_apply_fused<<<grid, 256, 0, L.s>>>(in, out, n_dev, n_max, partials, total);
    (*L.launches) += 2;
    return cudaGetLastError();
  }
  scan_reduce<<<grid, 256, 0, L.s>>>(in, n_dev, n_max, partials);
  scan_partials<<<1, 256, 0, L.s>>>(partials, n_dev, n_max, total);
  scan_apply<<<grid, 256, 0, L.s>>>(in, out, n_dev, n_max, partials);
  (*L.launches) += 3;
  return cudaGetLastError();
}

cudaError_t launch_histogram(const Launch& L, const uint64_t* keys, const uint64_t* n_dev, uint64_t n_max, int shift0,
                             int npass, uint64_t* hist) {
  uint64_t blocks = (n_max + 255) / 256;
  unsigned grid = (unsigned)(blocks < (uint64_t)L.nsm * 4 ? (blocks ? blocks : 1) : (uint64_t)L.nsm * 4);
  histogram_kernel<<<grid, 256, 0, L.s>>>(keys, n_dev, n_max, shift0, npass, hist);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_cell_hist(const Launch& L, const uint64_t* keys, const uint64_t* n_dev, uint64_t n_max,
                             const uint32_t* tab, uint64_t ncells, int rsh, uint64_t* hist, int shift,
                             uint64_t* n_kept, uint64_t* status, uint64_t max_words, const uint64_t* skip) {
  uint64_t blocks = (n_max + 255) / 256;
  unsigned grid = (unsigned)(blocks < (uint64_t)L.nsm * 8 ? (blocks ? blocks : 1) : (uint64_t)L.nsm * 8);
  cell_hist_kernel<<<grid, 256, 0, L.s>>>(keys, n_dev, n_max, tab, ncells, rsh, hist, shift, n_kept, status,
                                          max_words, skip);
  (*L.launches)++;
  return cudaGetLastError();
}

struct SortVariant {
  const void* fn;
  int threads, kpt;
  size_t smem;
};
const SortVariant* sort_variants(int* count) {
  static const SortVariant v[] = {
      // early-count shapes first: index 0 is the default before any tuning
      {(const void*)onesweep3_kernel<256, 32, 2, 3>, 256, 32, onesweep3_smem<256, 32, 3>()},
      {(const void*)onesweep3_kernel<256, 28, 2, 3>, 256, 28, onesweep3_smem<256, 28, 3>()},
      {(const void*)onesweep3_kernel<256, 32, 2, 5>, 256, 32, onesweep3_smem<256, 32, 5>()},
      {(const void*)onesweep3_kernel<256, 28, 2, 5>, 256, 28, onesweep3_smem<256, 28, 5>()},
      {(const void*)onesweep3_kernel<256, 32, 2, 0>, 256, 32, onesweep3_smem<256, 32, 0>()},
      {(const void*)onesweep3_kernel<384, 16, 2, 3>, 384, 16, onesweep3_smem<384, 16, 3>()},
      {(const void*)onesweep3_kernel<384, 16, 2, 5>, 384, 16, onesweep3_smem<384, 16, 5>()},
      {(const void*)onesweep_kernel<256, 16, 3>, 256, 16, onesweep_smem<256, 16>()},
      {(const void*)onesweep_kernel<256, 12, 4>, 256, 12, onesweep_smem<256, 12>()},
      {(const void*)onesweep_kernel<512, 8, 2>, 512, 8, onesweep_smem<512, 8>()},
      {(const void*)onesweep_kernel<384, 12, 2>, 384, 12, onesweep_smem<384, 12>()},
      {(const void*)onesweep_kernel<256, 24, 2>, 256, 24, onesweep_smem<256, 24>()},
      {(const void*)onesweep_kernel<128, 16, 8>, 128, 16, onesweep_smem<128, 16>()},
      {(const void*)onesweep_kernel<256, 16, 3, true>, 256, 16, onesweep_smem<256, 16>()},
      {(const void*)onesweep_kernel<256, 12, 4, true>, 256, 12, onesweep_smem<256, 12>()},
      {(const void*)onesweep_kernel<512, 8, 2, true>, 512, 8, onesweep_smem<512, 8>()},
      {(const void*)onesweep_kernel<256, 16, 3, true, 1>, 256, 16, onesweep_smem<256, 16>()},
      {(const void*)onesweep_kernel<512, 8, 2, true, 1>, 512, 8, onesweep_smem<512, 8>()},
      {(const void*)onesweep_kernel<256, 16, 3, true, 2>, 256, 16, onesweep_smem<256, 16>()},
      {(const void*)onesweep_kernel<512, 8, 2, true, 2>, 512, 8, onesweep_smem<512, 8>()},
  };
  *count = (int)(sizeof(v) / sizeof(v[0]));
  return v;
}
int g_sort_variant[64];  // per device; 0 = the default shape (onesweep3 256 x 32, atomic-OR ranking)
// per device and key-sort pass: 1 + the shape chosen for that pass, 0 = the device's shape
int g_sort_pass_variant[64][MAX_PASSES];

int sort_variant_current() {
  int dev = 0;
  cudaGetDevice(&dev);
  return (dev >= 0 && dev < 64) ? g_sort_variant[dev] : 0;
}

uint64_t sort_variant_key() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 0;
  uint64_t h = (uint64_t)g_sort_variant[dev];
  for (int p = 0; p < MAX_PASSES; p++) h = h * 31 + (uint64_t)g_sort_pass_variant[dev][p];
  return h;
}

cudaError_t launch_onesweep(const Launch& L, const uint64_t* in, uint64_t* out, const uint64_t* n_dev, uint64_t n_max,
                            int shift, const uint64_t* dcount, uint64_t* status, uint64_t* ticket, uint32_t epoch,
                            uint64_t* err, uint64_t* next_hist, int next_shift, const uint32_t* ctab,
                            uint64_t ncells, int rsh, const uint64_t* skip, int pass) {
  int nv = 0, dev = 0;
  const SortVariant* V = sort_variants(&nv);
  cudaGetDevice(&dev);
  int v = (dev >= 0 && dev < 64) ? g_sort_variant[dev] : 0;
  if (dev >= 0 && dev < 64 && pass >= 0 && pass < MAX_PASSES && g_sort_pass_variant[dev][pass] > 0)
    v = g_sort_pass_variant[dev][pass] - 1;
  const SortVariant& S = V[v < nv ? v : 0];
  const uint64_t tile = (uint64_t)S.threads * S.kpt;
  const uint64_t tiles = (n_max + tile - 1) / tile;
  cudaError_t e = allow_smem(S.fn, S.smem);
  if (e != cudaSuccess) return e;
  int grid = occupancy_grid(S.fn, S.threads, S.smem, L.nsm);
  if ((uint64_t)grid > tiles) grid = (int)(tiles ? tiles : 1);
  unsigned long long* tk = (unsigned long long*)ticket;
  void* args[] = {(void*)&in, (void*)&out, (void*)&n_dev, (void*)&n_max, (void*)&shift, (void*)&dcount,
                  (void*)&status, (void*)&tk, (void*)&epoch, (void*)&err, (void*)&next_hist, (void*)&next_shift,
                  (void*)&ctab, (void*)&ncells, (void*)&rsh, (void*)&skip};
  (*L.launches)++;
  return cudaLaunchKernel(S.fn, dim3(grid), dim3(S.threads), args, S.smem, L.s);
}

cudaError_t launch_tail_sort(const Launch& L, const uint64_t* in, uint64_t* out, const uint64_t* n_dev, uint64_t n_max,
                             int shift0, int npass, uint64_t* done) {
  cudaError_t e = allow_smem((const void*)tail_sort_kernel, tail_smem());
  if (e != cudaSuccess) return e;
  tail_sort_kernel<<<1, TAIL_T, tail_smem(), L.s>>>(in, out, n_dev, n_max, shift0, npass, done);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_compact_sort(const Launch& L, const uint64_t* in, uint64_t* out, const uint64_t* n_dev,
                                uint64_t n_max, uint64_t* done, uint64_t* kept_out) {
  const uint64_t ctas = (n_max + CR_W - 1) / CR_W;
  const unsigned grid = (unsigned)(ctas < (uint64_t)L.nsm ? (ctas ? ctas : 1) : (uint64_t)L.nsm);
  compact_sort_kernel<<<grid, CR_T, 0, L.s>>>(in, out, n_dev, n_max, done, kept_out);
  (*L.launches)++;
  return cudaGetLastError();
}

namespace {
// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependence on the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}
// the key buffer as rows of 16 keys (128 B), boxes of one scan step's rows, 128-byte swizzle
bool key_rows_map(CUtensorMap* tm, const uint64_t* keys, uint64_t key_cap) {
  EncodeTiledFn enc = encode_tiled();
  const uint64_t rows = key_cap / CB_TILE_ROW;
  if (!enc || rows == 0 || rows > (1ull << 31) || (reinterpret_cast<uintptr_t>(keys) & 127u)) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)CB_TILE_ROW, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)CB_TILE_ROW * 8};
  const cuuint32_t box[2] = {(cuuint32_t)CB_TILE_ROW, (cuuint32_t)(CB_STEP / CB_TILE_ROW)};
  const cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t*>(keys), dim, stride, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

cudaError_t launch_candidates(const Launch& L, const uint64_t* keys, uint64_t key_cap, const uint64_t* n_dev,
                              const DProg* d_prog, uint64_t* cand, uint64_t cand_cap, uint64_t* counters,
                              bool ballot) {
  CUtensorMap tm;
  if (!ballot && key_rows_map(&tm, keys, key_cap)) {
    const size_t smem = (size_t)(CB_THREADS / 32) * CB_STAGES * CB_STEP_BYTES + 1024;
    cudaError_t e = allow_smem((const void*)candidates_rows_kernel, smem);
    if (e != cudaSuccess) return e;
    const int grid = occupancy_grid((const void*)candidates_rows_kernel, CB_THREADS, smem, L.nsm);
    candidates_rows_kernel<<<grid, CB_THREADS, smem, L.s>>>(tm, keys, n_dev, d_prog, cand, cand_cap, counters);
  } else {
    const int grid = occupancy_grid((const void*)candidates_kernel, CA_THREADS, 0, L.nsm);
    candidates_kernel<<<grid, CA_THREADS, 0, L.s>>>(keys, n_dev, d_prog, cand, cand_cap, counters);
  }
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_exact(const Launch& L, const uint64_t* keys, const uint64_t* n_dev, const DProg* d_prog,
                         const uint64_t* cand, uint64_t cand_cap, uint64_t* raw, uint64_t raw_cap,
                         uint64_t* counters, bool stop_first, bool bins) {
  const size_t smem = bins ? 8 * sizeof(BinTables) : 0;
  if (bins) {
    cudaError_t e = allow_smem((const void*)exact_kernel, smem);
    if (e != cudaSuccess) return e;
  }
  int grid = occupancy_grid((const void*)exact_kernel, 256, smem, L.nsm);
  exact_kernel<<<grid, 256, smem, L.s>>>(keys, n_dev, d_prog, cand, cand_cap, raw, raw_cap, counters,
                                         stop_first ? 1 : 0, bins ? 1 : 0);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_expand_block(const Launch& L, int mode, bool wide, const DProg* d_prog, const DProg& h_prog,
                                uint64_t* unit_cnt, const uint64_t* unit_off, uint64_t* keys_g, uint64_t* keys_s,
                                uint64_t* hist, uint64_t* counters, uint64_t* stbl, uint64_t* sbase) {
  const size_t esz = wide ? 8 : 4;
  const size_t tables = block_body_words(mode, (uint64_t)h_prog.nsbins) * 4;
  const size_t smem = sizeof(DProg) + (size_t)EXP_THREADS * h_prog.nslot * esz + tables;
  const void* fn = nullptr;
  if (!wide)
    fn = mode == 3 ? (const void*)expand_block_kernel<int32_t, 3> : (const void*)expand_block_kernel<int32_t, 4>;
  else
    fn = mode == 3 ? (const void*)expand_block_kernel<int64_t, 3> : (const void*)expand_block_kernel<int64_t, 4>;
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  int64_t grid = occupancy_grid(fn, EXP_THREADS, smem, L.nsm);
  if (grid > h_prog.nblk) grid = h_prog.nblk;
  if (grid < 1) grid = 1;
  void* args[] = {(void*)&d_prog, (void*)&unit_cnt, (void*)&unit_off, (void*)&keys_g, (void*)&keys_s,
                  (void*)&hist,   (void*)&counters, (void*)&stbl,     (void*)&sbase};
  (*L.launches)++;
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(EXP_THREADS), args, smem, L.s);
}

cudaError_t launch_shared_cand(const Launch& L, const DProg& h_prog, const uint64_t* stbl, const uint64_t* sbase,
                               uint64_t* cand, uint64_t cand_cap, uint64_t* counters) {
  const uint64_t blocks = ((uint64_t)h_prog.nblk + 7) / 8;  // a warp per block
  const unsigned grid = (unsigned)std::min<uint64_t>(std::max<uint64_t>(blocks, 1), (uint64_t)L.nsm * 8);
  shared_cand_kernel<<<grid, 256, 0, L.s>>>(stbl, sbase, h_prog.nblk, h_prog.nsbins, cand, cand_cap, counters);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_heads(const Launch& L, const uint64_t* w, const uint64_t* n_dev, uint64_t n_max, uint64_t* flags) {
  uint64_t blocks = (n_max + 255) / 256;
  unsigned grid = (unsigned)(blocks < (uint64_t)L.nsm * 8 ? (blocks ? blocks : 1) : (uint64_t)L.nsm * 8);
  heads_kernel<<<grid, 256, 0, L.s>>>(w, n_dev, n_max, flags);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_merge(const Launch& L, const uint64_t* w, const uint64_t* flags, const uint64_t* excl,
                         const uint64_t* n_dev, uint64_t n_max, uint64_t* uniq) {
  uint64_t blocks = (n_max + 255) / 256;
  unsigned grid = (unsigned)(blocks < (uint64_t)L.nsm * 8 ? (blocks ? blocks : 1) : (uint64_t)L.nsm * 8);
  merge_kernel<<<grid, 256, 0, L.s>>>(w, flags, excl, n_dev, n_max, uniq);
  (*L.launches)++;
  return cudaGetLastError();
}

const void* witness_split_cond_fn() { return (const void*)witness_split_cond_kernel; }
cudaError_t launch_witness_split_cond(const Launch& L, uint64_t* counters, uint64_t raw_cap,
                                      cudaGraphConditionalHandle h) {
  witness_split_cond_kernel<<<1, 1, 0, L.s>>>(counters, raw_cap, h);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_witness_split(const Launch& L, uint64_t* counters, uint64_t raw_cap) {
  witness_split_kernel<<<1, 1, 0, L.s>>>(counters, raw_cap);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_witness_small(const Launch& L, const uint64_t* raw, uint64_t* sorted, uint64_t* uniq,
                                 uint64_t* counters, uint64_t raw_cap) {
  const unsigned ctas = (unsigned)((WSMALL_MAX + CR_W - 1) / CR_W);
  witness_rank_kernel<<<ctas < (unsigned)L.nsm ? ctas : (unsigned)L.nsm, CR_T, 0, L.s>>>(raw, sorted, counters,
                                                                                        raw_cap);
  witness_small_kernel<<<1, 1024, 0, L.s>>>(sorted, uniq, counters, raw_cap);
  (*L.launches) += 2;
  return cudaGetLastError();
}

cudaError_t launch_zero_status(const Launch& L, uint64_t* status, const uint64_t* n_dev, uint64_t max_words) {
  uint64_t blocks = (max_words + 255) / 256;
  unsigned grid = (unsigned)(blocks < (uint64_t)L.nsm * 8 ? (blocks ? blocks : 1) : (uint64_t)L.nsm * 8);
  zero_status_kernel<<<grid, 256, 0, L.s>>>(status, n_dev, max_words);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_zero(const Launch& L, uint64_t* p, const uint64_t* n_dev, uint64_t n_max) {
  uint64_t blocks = (n_max + 255) / 256;
  unsigned grid = (unsigned)(blocks < (uint64_t)L.nsm * 8 ? (blocks ? blocks : 1) : (uint64_t)L.nsm * 8);
  zero_kernel<<<grid, 256, 0, L.s>>>(p, n_dev, n_max);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_pair_blocks(const Launch& L, const uint64_t* keys, const uint64_t* n_dev, const DProg* d_prog,
                               const uint64_t* uniq, uint64_t* counters, uint64_t* blocks) {
  pair_blocks_kernel<<<1, 256, 0, L.s>>>(keys, n_dev, d_prog, uniq, counters, blocks);
  (*L.launches)++;
  return cudaGetLastError();
}

cudaError_t launch_kind_counts(const Launch& L, const uint64_t* uniq, uint64_t* counters, const uint64_t* gate) {
  kind_counts_kernel<<<L.nsm, 256, 0, L.s>>>(uniq, counters, gate);
  (*L.launches)++;
  return cudaGetLastError();
}

}  // namespace hgrd

// ------------------------------------------------------------------ sort autotuner
namespace hgrd {
namespace {
__global__ void random_keys_kernel(uint64_t* k, uint64_t n, uint64_t seed) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    k[i] = z ^ (z >> 31);
  }
}
}  // namespace
}  // namespace hgrd

#include "hgrd_host.h"

extern "C" int hgrd_sort_variant(int set, int* current, int* count) {
  using namespace hgrd;
  int nv = 0, dev = 0;
  sort_variants(&nv);
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return fail(HGRD_EUNSUPPORTED, "device index too large");
  if (set >= nv) return fail(HGRD_EINVAL, "no such sort variant");
  if (set >= 0) g_sort_variant[dev] = set;
  if (current) *current = g_sort_variant[dev];
  if (count) *count = nv;
  return HGRD_OK;
}

extern "C" int hgrd_sort_pass_variant(int pass, int set, int* current) {
  using namespace hgrd;
  int nv = 0, dev = 0;
  sort_variants(&nv);
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return fail(HGRD_EUNSUPPORTED, "device index too large");
  if (pass < 0 || pass >= MAX_PASSES) return fail(HGRD_EINVAL, "no such sort pass");
  if (set >= nv) return fail(HGRD_EINVAL, "no such sort variant");
  if (set >= -1) g_sort_pass_variant[dev][pass] = set + 1;
  if (current) *current = g_sort_pass_variant[dev][pass] - 1;
  return HGRD_OK;
}

extern "C" int hgrd_debug_lookback_timeout(void* d_ws, size_t ws_bytes, void* stream) {
  using namespace hgrd;
  constexpr uint64_t n = 12288;
  const uint64_t tiles = (n + RS_MIN_TILE - 1) / RS_MIN_TILE;
  const size_t need = (2 * n + tiles * RS_RADIX + 256 + 16) * 8;
  if (!d_ws) return fail(HGRD_EINVAL, "null workspace");
  if (ws_bytes < need) return fail(HGRD_ENOMEM, "workspace too small: need " + std::to_string(need));
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t* kin = (uint64_t*)d_ws;
  uint64_t* kout = kin + n;
  uint64_t* status = kout + n;
  uint64_t* gb = status + tiles * RS_RADIX;
  uint64_t* cnt = gb + 256;  // n, ticket, err
  int dev = 0;
  cudaGetDevice(&dev);
  uint64_t launches = 0;
  Launch L{s, 1, &launches};
  cudaDeviceGetAttribute(&L.nsm, cudaDevAttrMultiProcessorCount, dev);
  // keys, zero digit counts (every digit starts at 0, every position stays
  // below n), no status yet, and the ticket of the first tile already handed out
  random_keys_kernel<<<L.nsm, 256, 0, s>>>(kin, n, 0x7153);
  const uint64_t host[3] = {n, 1, 0};
  if (cudaMemsetAsync(gb, 0, 256 * 8, s) != cudaSuccess ||
      cudaMemsetAsync(status, 0, tiles * RS_RADIX * 8, s) != cudaSuccess ||
      cudaMemcpyAsync(cnt, host, sizeof(host), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(HGRD_EDEVICE, "set-up copies failed");
  cudaError_t e = launch_onesweep(L, kin, kout, cnt, n, 0, gb, status, cnt + 1, 1, cnt + 2);
  uint64_t errw = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&errw, cnt + 2, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(HGRD_EDEVICE, std::string("CUDA: ") + cudaGetErrorString(e));
  if (errw & ERR_TIMEOUT) return fail(HGRD_ETIMEOUT, "a bounded device wait (sort look-back) gave up");
  return HGRD_OK;
}

extern "C" int hgrd_sort_tune(void* d_ws, size_t ws_bytes, void* stream, int* best, float* ms, int cap) {
  using namespace hgrd;
  if (!d_ws) return fail(HGRD_EINVAL, "null workspace");
  cudaStream_t s = (cudaStream_t)stream;
  int nv = 0, dev = 0;
  const SortVariant* V = sort_variants(&nv);
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return fail(HGRD_EUNSUPPORTED, "device index too large");
  // keys in | keys out | status | hist | counters
  const size_t fixed = 3 * 4096 + 256;
  uint64_t n = ws_bytes > fixed ? (uint64_t)((ws_bytes - fixed) / (16.0 + 256.0 * 8 / RS_MIN_TILE)) : 0;
  n = std::min<uint64_t>(n, 1ull << 25) & ~(uint64_t)4095;
  if (n < 4096) return fail(HGRD_ENOMEM, "sort tuning workspace too small");
  char* w = (char*)d_ws;
  uint64_t* kin = (uint64_t*)w;
  uint64_t* kout = kin + n;
  uint64_t* status = kout + n;
  const size_t sw = ((n + RS_MIN_TILE - 1) / RS_MIN_TILE) * RS_RADIX;
  uint64_t* hist = status + sw;
  uint64_t* cnt = hist + 256;  // n, ticket, err
  uint64_t launches = 0;
  Launch L{s, 1, &launches};
  cudaDeviceGetAttribute(&L.nsm, cudaDevAttrMultiProcessorCount, dev);
  random_keys_kernel<<<L.nsm * 4, 256, 0, s>>>(kin, n, 0x5EED);
  cudaMemcpyAsync(cnt, &n, 8, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(hist, 0, 256 * 8, s);
  launch_histogram(L, kin, cnt, n, 0, 1, hist);
  cudaEvent_t e0, e1;
  note_created(2);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int saved = g_sort_variant[dev];
  float best_ms = 1e30f;
  int best_v = saved;
  uint32_t epoch = 1;
  for (int v = 0; v < nv; v++) {
    g_sort_variant[dev] = v;
    float vbest = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
      cudaMemsetAsync(status, 0, sw * 8, s);
      cudaMemsetAsync(cnt + 1, 0, 16, s);
      cudaEventRecord(e0, s);
      cudaError_t e = launch_onesweep(L, kin, kout, cnt, n, 0, hist, status, cnt + 1, epoch, cnt + 2);
      cudaEventRecord(e1, s);
      if (e != cudaSuccess) {
        g_sort_variant[dev] = saved;
        return fail(HGRD_EDEVICE, std::string("CUDA: ") + cudaGetErrorString(e));
      }
      cudaEventSynchronize(e1);
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) vbest = std::min(vbest, t);
    }
    if (ms && v < cap) ms[v] = vbest;
    if (vbest < best_ms) {
      best_ms = vbest;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  uint64_t errw = 0;
  cudaMemcpy(&errw, cnt + 2, 8, cudaMemcpyDeviceToHost);
  g_sort_variant[dev] = best_v;
  if (best) *best = best_v;
  if (errw) return fail(HGRD_ETIMEOUT, "a bounded device wait gave up during sort tuning");
  return HGRD_OK;
}
