// Batched check of many (kernel, host binding) items in one launch sequence.
//
// The paper checks one kernel under the host facts of one launch site; a
// host loop (Sec. 4, class (4)) or a whole program yields many such items of
// very uneven size.  Items are split by a size class:
//   small  (all keys fit on chip): one persistent, work-queued kernel; a CTA
//          pops the next item (largest first) and runs the whole check for it
//          in shared memory — expansion, a CTA-local stable radix sort, the
//          exact scan of every run, and the witness merge;
//   large: the device-wide pipeline of hgrd_check, items spread over several
//          streams by longest-processing-time-first, each followed by a
//          gather of its verdict.
// The whole sequence can be captured once into a CUDA graph and replayed.  An
// autotuner picks the small-item threshold and the stream count by timing
// the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "hgrd_host.h"
#include "jit.h"
#include "kcommon.cuh"

namespace hgrd {

size_t item_workspace_bytes(const Bound& B, const hgrd_check_opts* o);
int item_enqueue(const hgrd_desc* d, const hgrd_check_opts* o, void* ws, size_t bytes, cudaStream_t s,
                 const DProg* dprog_resident, uint64_t** counters, const uint64_t** uniq, uint64_t* raw_cap,
                 uint64_t* cand_cap);

namespace {

using namespace dev;

constexpr int SB_THREADS = 256;
constexpr int SB_WARPS = SB_THREADS / 32;
constexpr int SB_KEYS = 4096;   // keys of one small item (two on-chip buffers)
constexpr int SB_UNITS = 1024;  // simulated warps of one small item
constexpr int SB_RAW = 1024;    // per-run witnesses of one small item
constexpr int SB_SLOTS = 64;    // slot file entries per simulated lane
constexpr int SB_PASSES = 4;    // radix passes (32 sorted bits)
constexpr int OUT_WORDS = 56;   // n_keys, n_oob, n_witness, kind0..2, flags, n_raw, 48 racy-pair words
enum { F_RAW_OVERFLOW = 1, F_TIMEOUT = 2, F_CAND_OVERFLOW = 4, F_SHARED_OVERFLOW = 8, F_LOCK_RUN = 16 };

struct SmallSmem {
  DProg prog;
  int32_t slots[SB_WARPS][SB_SLOTS * 32];
  uint64_t ka[SB_KEYS], kb[SB_KEYS];
  uint32_t ucnt[SB_UNITS + 1];
  uint32_t whist[SB_WARPS][256];
  uint32_t dstart[256];
  uint64_t raw[SB_RAW];
  uint64_t ws[SB_WARPS + 1];
  uint64_t pairs[48];
  uint64_t oob;
  uint32_t item, nraw, nkeys, nuniq;
  uint32_t kinds[3];
};

// exclusive scan of one value per thread over the CTA (8 warps)
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint64_t* ws, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < SB_WARPS ? (uint32_t)ws[lane] : 0;
    uint32_t si = s;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, si, o);
      if (lane >= o) si += y;
    }
    if (lane < SB_WARPS) ws[lane] = si - s;
    if (lane == SB_WARPS - 1) ws[SB_WARPS] = si;
  }
  __syncthreads();
  const uint32_t r = x - v + (uint32_t)ws[warp];
  if (total) *total = (uint32_t)ws[SB_WARPS];
  __syncthreads();
  return r;
}

// one stable counting-sort pass of n <= SB_KEYS keys on the 8-bit digit at
// `shift`: warps own contiguous ranges and rank in memory order
__device__ void cta_sort_pass(SmallSmem& S, const uint64_t* src, uint64_t* dst, uint32_t n, int shift) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int CH = SB_KEYS / SB_WARPS / 32;  // 32-key chunks per warp
  const uint32_t per = ((n + SB_WARPS * 32 - 1) / (SB_WARPS * 32)) * 32;
  const uint32_t w0 = warp * per;
  for (int i = threadIdx.x; i < SB_WARPS * 256; i += SB_THREADS) (&S.whist[0][0])[i] = 0;
  __syncthreads();
  const unsigned lt = lanemask_lt();
  uint32_t rk[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const uint32_t i = w0 + c * 32 + lane;
    const bool in = (uint32_t)(c * 32) < per && i < n;
    const uint32_t d = in ? (uint32_t)(src[i] >> shift) & 255u : 256u + lane;
    const unsigned peers = __match_any_sync(FULL, d);
    uint32_t old = 0;
    if (in) old = S.whist[warp][d];
    rk[c] = old + __popc(peers & lt);
    __syncwarp();
    if (in && lane == __ffs(peers) - 1) S.whist[warp][d] = old + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const int t = threadIdx.x;  // digit
  uint32_t sum = 0;
  for (int w = 0; w < SB_WARPS; ++w) {
    const uint32_t c = S.whist[w][t];
    S.whist[w][t] = sum;
    sum += c;
  }
  S.dstart[t] = cta_excl_scan(sum, S.ws, nullptr);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const uint32_t i = w0 + c * 32 + lane;
    if ((uint32_t)(c * 32) < per && i < n) {
      const uint64_t k = src[i];
      const uint32_t d = (uint32_t)(k >> shift) & 255u;
      dst[S.dstart[d] + S.whist[warp][d] + rk[c]] = k;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(SB_THREADS) batch_small_kernel(const DProg* __restrict__ progs,
                                                                 const uint32_t* __restrict__ order, uint32_t nsmall,
                                                                 unsigned long long* queue, uint64_t* __restrict__ outs,
                                                                 uint64_t* __restrict__ wits, uint32_t wcap,
                                                                 const uint32_t* __restrict__ masks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) S.item = (uint32_t)atomicAdd(queue, 1ull);
    __syncthreads();
    if (S.item >= nsmall) break;
    const uint32_t item = order[S.item];
    {
      const uint4* src = reinterpret_cast<const uint4*>(progs + item);
      uint4* dst = reinterpret_cast<uint4*>(&S.prog);
      for (int i = threadIdx.x; i < (int)(sizeof(DProg) / 16); i += SB_THREADS) dst[i] = src[i];
    }
    __syncthreads();
    // a restricted check: the accesses outside the item's mask are not run
    if (masks && threadIdx.x < MAXACC && threadIdx.x < S.prog.nacc && !((masks[item] >> threadIdx.x) & 1u))
      S.prog.acc[threadIdx.x].dead = 1;
    if (threadIdx.x == 0) {
      S.oob = 0;
      S.nraw = 0;
      S.kinds[0] = S.kinds[1] = S.kinds[2] = 0;
    }
    if (threadIdx.x < 48) S.pairs[threadIdx.x] = 0;
    __syncthreads();
    const DProg* P = &S.prog;
    const int64_t nunits = P->nunits;
    int32_t* sl = S.slots[warp];
    // count keys per unit
    uint64_t oob = 0;
    for (int64_t u = warp; u < nunits; u += SB_WARPS) {
      uint32_t cursor = 0;
      oob += expand_unit<int32_t>(P, sl, lane, u, 0xffffffffu,
                                  [&](int, const DAcc& A, bool, unsigned bal, int64_t, int64_t, int64_t, int,
                                      const int32_t*) { cursor += (uint32_t)__popc(bal) * A.G; });
      if (lane == 0) S.ucnt[u] = cursor;
    }
    for (int o = 16; o; o >>= 1) oob += __shfl_down_sync(FULL, oob, o);
    if (lane == 0 && oob) atomicAdd((unsigned long long*)&S.oob, (unsigned long long)oob);
    __syncthreads();
    // unit offsets (nunits <= SB_UNITS = 4 per thread)
    {
      uint32_t v[4], s = 0;
      for (int k = 0; k < 4; ++k) {
        const int u = threadIdx.x * 4 + k;
        v[k] = u < nunits ? S.ucnt[u] : 0;
        s += v[k];
      }
      uint32_t total = 0;
      uint32_t run = cta_excl_scan(s, S.ws, &total);
      for (int k = 0; k < 4; ++k) {
        const int u = threadIdx.x * 4 + k;
        if (u < nunits) S.ucnt[u] = run;
        run += v[k];
      }
      if (threadIdx.x == 0) S.nkeys = total;
      __syncthreads();
    }
    // write keys in unit order
    for (int64_t u = warp; u < nunits; u += SB_WARPS) {
      uint32_t cursor = S.ucnt[u];
      expand_unit<int32_t>(P, sl, lane, u, 0xffffffffu,
                           [&](int a, const DAcc& A, bool inb, unsigned bal, int64_t idx, int64_t iv, int64_t b,
                               int lt, const int32_t*) {
                             const int G = A.G;
                             if (inb) {
                               const int rank = __popc(bal & lanemask_lt());
                               for (int j = 0; j < G; ++j) S.ka[cursor + rank * G + j] = make_key(P, A, a, idx, iv, b, lt, j);
                             }
                             cursor += (uint32_t)__popc(bal) * G;
                           });
    }
    __syncthreads();
    const uint32_t n = S.nkeys;
    // stable LSD sort on the (cell, interval) bits
    uint64_t* src = S.ka;
    uint64_t* dst = S.kb;
    const int passes = (P->RB + P->PB - P->SB + 7) / 8;
    for (int p = 0; p < passes; ++p) {
      cta_sort_pass(S, src, dst, n, P->SB + 8 * p);
      uint64_t* t = src;
      src = dst;
      dst = t;
    }
    // exact scan of every run: a warp handles the runs that start in its range
    {
      const int rsh = P->PB + P->IVB;
      const uint32_t einter = lane < P->nacc ? P->einter[lane] : 0u;
      const uint32_t eintra = lane < P->nacc ? P->eintra[lane] : 0u;
      const uint32_t per = ((n + SB_WARPS * 32 - 1) / (SB_WARPS * 32)) * 32;
      const uint32_t r0 = warp * per, r1 = min(n, r0 + per);
      for (uint32_t c = r0; c < r1; c += 32) {
        const uint32_t i = c + lane;
        const bool st = i < r1 && (i == 0 || shr64(src[i], rsh) != shr64(src[i - 1], rsh));
        unsigned m = __ballot_sync(FULL, st);
        while (m) {
          const int l = __ffs(m) - 1;
          m &= m - 1;
          const uint32_t s0 = c + l;
          if (s0 + 1 >= n || shr64(src[s0 + 1], rsh) != shr64(src[s0], rsh)) continue;  // one key: no pair
          const RunMasks R = exact_run(src, s0, 0, n, P, lane, einter, eintra);
          record_pairs(S.pairs, R, lane);
          uint32_t row = witness_row(R, lane);
          const uint32_t cntw = (uint32_t)__popc(row);
          uint32_t incl = cntw;
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
          }
          const uint32_t total = __shfl_sync(FULL, incl, 31);
          if (!total) continue;
          uint32_t base = 0;
          if (lane == 0) base = atomicAdd(&S.nraw, total);
          base = __shfl_sync(FULL, base, 0);
          uint32_t space, arr;
          uint64_t gran;
          run_location(P, R.rid, &space, &arr, &gran);
          uint32_t o = base + incl - cntw;
          while (row) {
            const int bb = __ffs(row) - 1;
            row &= row - 1;
            if (o < SB_RAW) S.raw[o] = pack_witness(space, arr, gran, (uint32_t)lane, (uint32_t)bb, witness_kind(R, bb));
            ++o;
          }
        }
      }
    }
    __syncthreads();
    // canonical order: bitonic sort of the raw words, then merge equal locations
    const uint32_t nraw = S.nraw;
    const uint32_t m = nraw < SB_RAW ? nraw : SB_RAW;
    uint32_t p2 = 1;
    while (p2 < m) p2 <<= 1;
    for (uint32_t i = m + threadIdx.x; i < p2; i += SB_THREADS) S.raw[i] = ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= p2; k <<= 1)
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < p2; i += SB_THREADS) {
          const uint32_t l = i ^ j;
          if (l > i) {
            const uint64_t x = S.raw[i], y = S.raw[l];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              S.raw[i] = y;
              S.raw[l] = x;
            }
          }
        }
        __syncthreads();
      }
    // heads and their ranks (4 per thread, m <= 1024); kb is free now
    {
      uint32_t h[4], s = 0;
      for (int q = 0; q < 4; ++q) {
        const uint32_t i = threadIdx.x * 4 + q;
        h[q] = (i < m && (i == 0 || (S.raw[i] >> WIT_SORT_LO) != (S.raw[i - 1] >> WIT_SORT_LO))) ? 1u : 0u;
        s += h[q];
      }
      uint32_t total = 0;
      uint32_t run = cta_excl_scan(s, S.ws, &total);
      uint64_t* uq = (src == S.ka) ? S.kb : S.ka;
      for (uint32_t i = threadIdx.x; i < m; i += SB_THREADS) uq[i] = 0;
      __syncthreads();
      for (int q = 0; q < 4; ++q) {
        const uint32_t i = threadIdx.x * 4 + q;
        run += h[q];
        if (i < m) atomicOr((unsigned long long*)&uq[run - 1], (unsigned long long)S.raw[i]);
      }
      if (threadIdx.x == 0) S.nuniq = total;
      __syncthreads();
      uint32_t c0 = 0, c1 = 0, c2 = 0;
      for (uint32_t i = threadIdx.x; i < total; i += SB_THREADS) {
        c0 += uq[i] & 1;
        c1 += (uq[i] >> 1) & 1;
        c2 += (uq[i] >> 2) & 1;
      }
      if (c0) atomicAdd(&S.kinds[0], c0);
      if (c1) atomicAdd(&S.kinds[1], c1);
      if (c2) atomicAdd(&S.kinds[2], c2);
      __syncthreads();
      uint64_t* o = outs + (size_t)item * OUT_WORDS;
      if (threadIdx.x == 0) {
        o[0] = S.nkeys;
        o[1] = S.oob;
        o[2] = total;
        o[3] = S.kinds[0];
        o[4] = S.kinds[1];
        o[5] = S.kinds[2];
        o[6] = nraw > SB_RAW ? F_RAW_OVERFLOW : 0;
        o[7] = nraw;
      }
      if (threadIdx.x < 48) o[8 + threadIdx.x] = S.pairs[threadIdx.x];
      const uint32_t nc = total < wcap ? total : wcap;
      for (uint32_t i = threadIdx.x; i < nc; i += SB_THREADS) wits[(size_t)item * wcap + i] = uq[i];
    }
    __syncthreads();
  }
}

// verdict of one large item, copied next to the small items' verdicts
__global__ void gather_kernel(const uint64_t* __restrict__ cnt, const uint64_t* __restrict__ uniq, uint64_t raw_cap,
                              uint64_t cand_cap, uint64_t* __restrict__ out, uint64_t* __restrict__ wits, uint32_t wcap) {
  const uint64_t nu = cnt[C_NUNIQ];
  if (threadIdx.x == 0) {
    out[0] = cnt[C_NKEYS];
    out[1] = cnt[C_NOOB];
    out[2] = nu;
    out[3] = cnt[C_KIND0];
    out[4] = cnt[C_KIND1];
    out[5] = cnt[C_KIND2];
    out[6] = (cnt[C_NRAW] > raw_cap ? F_RAW_OVERFLOW : 0) | ((cnt[C_ERR] & ERR_TIMEOUT) ? F_TIMEOUT : 0) |
             ((cnt[C_ERR] & ERR_LOCK_RUN) ? F_LOCK_RUN : 0) |
             (cnt[C_NCAND] > cand_cap ? F_CAND_OVERFLOW : 0) | ((cnt[C_ERR] & ERR_SHARED_FULL) ? F_SHARED_OVERFLOW : 0);
    out[7] = cnt[C_NRAW];
  }
  if (threadIdx.x < 48) out[8 + threadIdx.x] = cnt[C_PAIRS + threadIdx.x];
  const uint64_t nc = nu < wcap ? nu : wcap;
  if (!(cnt[C_NRAW] > raw_cap))
    for (uint64_t i = threadIdx.x; i < nc; i += blockDim.x) wits[i] = uniq[i];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// nkeys: the most keys the check can make
bool small_ok_keys(const Bound& B, uint32_t limit, uint64_t nkeys) {
  const DProg& P = B.prog;
  return !B.wide && nkeys <= limit && nkeys <= (uint64_t)SB_KEYS && P.nunits <= SB_UNITS &&
         P.RB + P.PB - P.SB <= 8 * SB_PASSES && P.nslot <= SB_SLOTS;
}
bool small_ok(const Bound& B, uint32_t limit) { return small_ok_keys(B, limit, B.nkeys_max); }

// The one-CTA verdict of a single small check, written where the device-wide
// pipeline leaves its results: the counters and the merged-witness buffer.
__global__ void small_finish_kernel(const uint64_t* __restrict__ out, const uint64_t* __restrict__ wits,
                                    uint32_t wcap, uint64_t* __restrict__ counters, uint64_t* __restrict__ uniq) {
  if (threadIdx.x == 0) {
    counters[C_NKEYS] = out[0];
    counters[C_NOOB] = out[1];
    counters[C_NUNIQ] = out[2];
    counters[C_KIND0] = out[3];
    counters[C_KIND1] = out[4];
    counters[C_KIND2] = out[5];
    counters[C_NRAW] = out[7];
    if (out[6] & F_RAW_OVERFLOW) counters[C_ERR] |= ERR_SMALL_FULL;
  }
  if (threadIdx.x < 48) counters[C_PAIRS + threadIdx.x] = out[8 + threadIdx.x];
  const uint64_t n = out[2] < wcap ? out[2] : wcap;
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) uniq[i] = wits[i];
}

// The top-k pairs of every item by the ranker's logits (one warp per item,
// k rounds of a warp arg-max, ties to the lower pair index: the order of a
// stable sort by decreasing score), as the mask of their accesses.  An item
// with at most k eligible pairs checks all of them (its cover); an item
// whose best logit is below min_score, or without pairs, is not ranked (0).
__global__ void topk_mask_kernel(const float* __restrict__ logits, const uint32_t* __restrict__ poff,
                                 const uint32_t* __restrict__ pab, const uint32_t* __restrict__ cover, uint32_t n,
                                 uint32_t topk, float min_score, uint32_t* __restrict__ mask_out) {
  const int lane = threadIdx.x & 31;
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i = w0; i < n; i += nw) {
    const uint32_t lo = poff[i], np = poff[i + 1] - lo;
    uint32_t mask = 0;
    if (np && np <= topk) {
      mask = cover[i];
    } else if (np) {
      // pairs lane, lane + 32, ...: at most 528 per item, 17 per lane
      uint32_t taken = 0;
      for (uint32_t r = 0; r < topk; ++r) {
        float best = -INFINITY;
        uint32_t bi = 0xffffffffu;
        for (uint32_t j = lane, q = 0; j < np; j += 32, ++q) {
          const float z = logits[lo + j];
          if (!((taken >> q) & 1u) && (z > best || (z == best && j < bi))) {
            best = z;
            bi = j;
          }
        }
        for (int o = 16; o; o >>= 1) {
          const float zb = __shfl_xor_sync(FULL, best, o);
          const uint32_t jb = __shfl_xor_sync(FULL, bi, o);
          if (zb > best || (zb == best && jb < bi)) {
            best = zb;
            bi = jb;
          }
        }
        if (r == 0 && !(best >= min_score)) break;  // not ranked
        if (bi == 0xffffffffu) break;
        if ((bi & 31u) == (uint32_t)lane) taken |= 1u << (bi >> 5);
        const uint32_t ab = pab[lo + bi];
        mask |= (1u << (ab & 31u)) | (1u << ((ab >> 8) & 31u));
      }
    }
    if (lane == 0) mask_out[i] = mask;
  }
}

}  // namespace

// a check restricted to the accesses in `only` (0 or all ones: every access)
// can make keys of those accesses alone
bool small_single_ok(const Bound& B, uint32_t only) {
  if (only == 0u || only == 0xffffffffu) return small_ok(B, SB_KEYS);
  const DProg& P = B.prog;
  uint64_t nk = 0;
  for (int a = 0; a < P.nacc; a++)
    if (!P.acc[a].dead && ((only >> a) & 1u))
      nk += (uint64_t)P.nblk * (uint64_t)P.nthr * (uint64_t)P.nit * (uint64_t)P.acc[a].G;
  return small_ok_keys(B, SB_KEYS, nk);
}

cudaError_t launch_small_single(const Launch& L, const DProg* d_prog, uint64_t* counters, uint64_t* scratch,
                                uint64_t* uniq) {
  const size_t smem = sizeof(SmallSmem);
  cudaError_t e = allow_smem((const void*)batch_small_kernel, smem);
  if (e != cudaSuccess) return e;
  uint64_t* out = scratch;
  uint64_t* wits = scratch + 64;
  batch_small_kernel<<<1, SB_THREADS, smem, L.s>>>(d_prog, (const uint32_t*)(counters + C_SMALLQ + 1), 1,
                                                  (unsigned long long*)(counters + C_SMALLQ), out, wits, SB_RAW,
                                                  nullptr);
  small_finish_kernel<<<1, 256, 0, L.s>>>(out, wits, SB_RAW, counters, uniq);
  (*L.launches) += 2;
  return cudaGetLastError();
}

}  // namespace hgrd

using namespace hgrd;

struct hgrd_batch {
  std::vector<const hgrd_desc*> items;
  DProg* h_progs = nullptr;  // pinned copy of every item's program
  hgrd_batch_opts opts{};
  uint32_t small_limit = SB_KEYS, nstreams = 4;
  std::vector<uint32_t> small, large;  // item ids, largest first
  std::vector<int> large_stream;       // stream of each large item
  std::vector<cudaStream_t> streams;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  size_t region_bytes = 0;  // per large-item stream
  size_t off_progs = 0, off_order = 0, off_outs = 0, off_wits = 0, off_queue = 0, off_regions = 0, total = 0;
  uint32_t wcap = 64;
  cudaGraphExec_t exec = nullptr;
  void* exec_ws = nullptr;
  cudaStream_t exec_stream = nullptr;
  uint32_t* h_order = nullptr;
  // ranked form (hgrd_batch_rank_prepare): eligible pairs of every item and
  // their features, pinned staging for selections and restricted programs
  bool rank_ready = false;
  std::vector<uint32_t> pair_off, pair_ab, cover;  // pairs of item i: [pair_off[i], pair_off[i+1])
  std::vector<float> feat;                          // 96 features per pair
  std::vector<uint32_t> sel;    // small items of a selective run
  std::vector<uint32_t> rmask;  // accesses each item checks in a selective run
  std::vector<DProg> lprog;     // restricted programs of large items
  const void* feat_ws = nullptr;  // workspace the features were uploaded to
  size_t off_feat = 0, off_logit = 0, off_poff = 0, off_pab = 0, off_cover = 0, off_dmask = 0, off_rmask = 0,
         off_mlp = 0, rank_total = 0;
};

namespace {

constexpr uint32_t MAX_STREAMS = 16;

void plan(hgrd_batch* b) {
  const size_t n = b->items.size();
  std::vector<uint32_t> ids(n);
  for (size_t i = 0; i < n; i++) ids[i] = (uint32_t)i;
  std::stable_sort(ids.begin(), ids.end(), [&](uint32_t x, uint32_t y) {
    return b->items[x]->bound->nkeys_max > b->items[y]->bound->nkeys_max;
  });
  b->small.clear();
  b->large.clear();
  for (uint32_t id : ids) (small_ok(*b->items[id]->bound, b->small_limit) ? b->small : b->large).push_back(id);
  // longest processing time first over the large-item streams (stream 0 runs the small items)
  const uint32_t nl = std::max<uint32_t>(1, b->nstreams - 1);
  std::vector<double> load(nl, 0.0);
  b->large_stream.assign(b->large.size(), 0);
  for (size_t k = 0; k < b->large.size(); k++) {
    const uint32_t j = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
    b->large_stream[k] = 1 + (int)j;
    load[j] += (double)b->items[b->large[k]]->bound->nkeys_max + 2e5;  // + launch overhead in key units
  }
  for (size_t k = 0; k < b->small.size(); k++) b->h_order[k] = b->small[k];
}

int drop_graph(hgrd_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->exec_ws = nullptr;
  return HGRD_OK;
}

#define BK(x)                                                                                  \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) return fail(HGRD_EDEVICE, std::string("CUDA: ") + cudaGetErrorString(e_)); \
  } while (0)

// Enqueue the batch.  A selective run (run != nullptr) checks only the items
// with run[i] set, each on the accesses of masks[i] (all ones: the whole item;
// fewer: a restricted check, whose races are races of the item): small items
// through the on-chip kernel with the masks applied there, large ones on
// restricted copies of their programs.
int enqueue_batch(hgrd_batch* b, char* ws, cudaStream_t s, const uint8_t* run = nullptr,
                  const uint32_t* masks = nullptr) {
  const size_t n = b->items.size();
  hgrd_check_opts io{};
  io.flags = HGRD_NO_PAIR;
  BK(cudaMemcpyAsync(ws + b->off_progs, b->h_progs, n * sizeof(DProg), cudaMemcpyHostToDevice, s));
  uint32_t nsmall = (uint32_t)b->small.size();
  const uint32_t* d_masks = nullptr;
  if (run) {
    // (pageable host copies: each returns once its source is staged)
    b->sel.clear();
    for (uint32_t id : b->small)
      if (run[id]) b->sel.push_back(id);
    // a large item restricted to few enough keys runs whole on chip too
    for (uint32_t id : b->large)
      if (run[id] && masks[id] != 0xffffffffu && small_single_ok(*b->items[id]->bound, masks[id]))
        b->sel.push_back(id);
    nsmall = (uint32_t)b->sel.size();
    if (nsmall)
      BK(cudaMemcpyAsync(ws + b->off_order, b->sel.data(), (size_t)nsmall * 4, cudaMemcpyHostToDevice, s));
    b->rmask.assign(masks, masks + n);
    BK(cudaMemcpyAsync(ws + b->off_rmask, b->rmask.data(), n * 4, cudaMemcpyHostToDevice, s));
    d_masks = (const uint32_t*)(ws + b->off_rmask);
    // restricted programs of the large items that run on part of their accesses
    b->lprog.resize(b->large.size());
    uint32_t k = 0;
    for (uint32_t id : b->large) {
      if (!run[id] || masks[id] == 0xffffffffu || small_single_ok(*b->items[id]->bound, masks[id])) continue;
      DProg& q = b->lprog[k++];
      q = b->h_progs[id];
      for (int a = 0; a < q.nacc; a++)
        if (!((masks[id] >> a) & 1u)) q.acc[a].dead = 1;
      BK(cudaMemcpyAsync(ws + b->off_progs + (size_t)id * sizeof(DProg), &q, sizeof(DProg), cudaMemcpyHostToDevice, s));
    }
  } else {
    BK(cudaMemcpyAsync(ws + b->off_order, b->h_order, std::max<size_t>(1, b->small.size()) * 4,
                       cudaMemcpyHostToDevice, s));
  }
  BK(cudaMemsetAsync(ws + b->off_queue, 0, 256, s));
  BK(cudaMemsetAsync(ws + b->off_outs, 0, n * OUT_WORDS * 8, s));
  BK(cudaEventRecord(b->fork, s));
  for (uint32_t j = 0; j < b->nstreams; j++) BK(cudaStreamWaitEvent(b->streams[j], b->fork, 0));
  const DProg* dprogs = (const DProg*)(ws + b->off_progs);
  uint64_t* outs = (uint64_t*)(ws + b->off_outs);
  uint64_t* wits = (uint64_t*)(ws + b->off_wits);
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsmall) {
    const size_t smem = sizeof(SmallSmem);
    BK(cudaFuncSetAttribute((const void*)batch_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint32_t grid = (uint32_t)std::min<size_t>(nsmall, (size_t)nsm);
    batch_small_kernel<<<grid, SB_THREADS, smem, b->streams[0]>>>(dprogs, (const uint32_t*)(ws + b->off_order),
                                                                  nsmall, (unsigned long long*)(ws + b->off_queue),
                                                                  outs, wits, b->wcap, d_masks);
    BK(cudaGetLastError());
    g_stats.kernel_launches++;
  }
  for (size_t k = 0; k < b->large.size(); k++) {
    const uint32_t id = b->large[k];
    if (run && (!run[id] || (masks[id] != 0xffffffffu && small_single_ok(*b->items[id]->bound, masks[id]))))
      continue;  // not in this run, or restricted to the on-chip kernel
    const int j = b->large_stream[k];
    char* reg = ws + b->off_regions + (size_t)(j - 1) * b->region_bytes;
    uint64_t* cnt = nullptr;
    const uint64_t* uq = nullptr;
    uint64_t raw_cap = 0, cand_cap = 0;
    const uint64_t launches = g_stats.kernel_launches;
    hgrd_stats keep = g_stats;
    hgrd_check_opts jo = io;
    // a restricted program runs on the interpreted kernels (specialised ones
    // are built for the whole program's structure)
    if (run && masks[id] != 0xffffffffu) jo.flags |= HGRD_NO_JIT;
    int rc = item_enqueue(b->items[id], &jo, reg, b->region_bytes, b->streams[j], dprogs + id, &cnt, &uq, &raw_cap,
                          &cand_cap);
    keep.kernel_launches = launches + g_stats.kernel_launches;
    g_stats = keep;
    if (rc) return rc;
    gather_kernel<<<1, 128, 0, b->streams[j]>>>(cnt, uq, raw_cap, cand_cap, outs + (size_t)id * OUT_WORDS,
                                                wits + (size_t)id * b->wcap, b->wcap);
    BK(cudaGetLastError());
    g_stats.kernel_launches++;
  }
  for (uint32_t j = 0; j < b->nstreams; j++) {
    BK(cudaEventRecord(b->join[j], b->streams[j]));
    BK(cudaStreamWaitEvent(s, b->join[j], 0));
  }
  return HGRD_OK;
}

// every item's verdict words and kept witnesses, read back in one round trip
int read_outs(hgrd_batch* b, char* ws, cudaStream_t s, std::vector<uint64_t>* outs, std::vector<uint64_t>* wits) {
  const size_t n = b->items.size();
  outs->resize(n * OUT_WORDS);
  wits->resize((size_t)n * b->wcap);
  BK(cudaMemcpyAsync(outs->data(), ws + b->off_outs, outs->size() * 8, cudaMemcpyDeviceToHost, s));
  BK(cudaMemcpyAsync(wits->data(), ws + b->off_wits, wits->size() * 8, cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
  return HGRD_OK;
}

// item i's verdict from its words o and witnesses q (into w + i * wcap)
int decode_item(const hgrd_batch* b, size_t i, const uint64_t* o, const uint64_t* q, hgrd_item_verdict* v,
                hgrd_witness* w, uint32_t wcap) {
  const Bound& B = *b->items[i]->bound;
  hgrd_item_verdict& x = *v;
  memset(&x, 0, sizeof(x));
  x.n_instances = B.n_instances;
  x.n_keys = o[0];
  x.n_oob = o[1];
  x.n_witness = o[2];
  x.n_by_kind[0] = o[3];
  x.n_by_kind[1] = o[4];
  x.n_by_kind[2] = o[5];
  x.racy = o[2] > 0;
  for (int k = 0; k < 3; k++)
    for (int a = 0; a < 32; a++) x.pair_kind[k][a] = (uint32_t)(o[8 + k * 16 + a / 2] >> (32 * (a & 1)));
  x.small = std::find(b->small.begin(), b->small.end(), (uint32_t)i) != b->small.end();
  x.status = (o[6] & F_TIMEOUT)                                               ? HGRD_ETIMEOUT
             : (o[6] & F_LOCK_RUN)                                               ? HGRD_EUNSUPPORTED
             : (o[6] & (F_RAW_OVERFLOW | F_CAND_OVERFLOW | F_SHARED_OVERFLOW)) ? HGRD_ENOMEM
                                                                                : HGRD_OK;
  if (x.status) return x.status;
  const uint32_t nc = (uint32_t)std::min<uint64_t>({(uint64_t)wcap, (uint64_t)b->wcap, o[2]});
  x.n_copied = nc;
  for (uint32_t k = 0; k < nc; k++) {
    hgrd_witness& y = w[i * (size_t)wcap + k];
    memset(&y, 0, sizeof(y));
    y.space = (uint8_t)((q[k] >> 58) & 1);
    y.array = (uint8_t)((q[k] >> 53) & 31);
    y.acc_lo = (uint8_t)((q[k] >> 8) & 31);
    y.acc_hi = (uint8_t)((q[k] >> 3) & 31);
    y.kind_mask = (uint8_t)(q[k] & 7);
    y.byte_addr = ((q[k] >> 13) & ((1ull << 40) - 1)) * (uint64_t)B.array_granule[y.array];
  }
  return HGRD_OK;
}


}  // namespace

extern "C" {

int hgrd_batch_create(const hgrd_desc* const* items, uint32_t n, const hgrd_batch_opts* o, hgrd_batch** out) {
  if (!items || !out || n == 0) return fail(HGRD_EINVAL, "empty batch or null argument");
  std::unique_ptr<hgrd_batch> b(new hgrd_batch());
  if (o) b->opts = *o;
  b->wcap = b->opts.witness_cap ? b->opts.witness_cap : 64;
  b->nstreams = b->opts.streams ? std::min(b->opts.streams, MAX_STREAMS) : 4;
  if (b->nstreams < 2) b->nstreams = 2;
  b->small_limit = b->opts.small_keys ? b->opts.small_keys : SB_KEYS;
  for (uint32_t i = 0; i < n; i++) {
    if (!items[i] || !items[i]->bound) return fail(HGRD_EINVAL, "batch item " + std::to_string(i) + " is not bound");
    b->items.push_back(items[i]);
  }
  note_created(2);
  if (cudaMallocHost((void**)&b->h_progs, n * sizeof(DProg)) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_order, n * sizeof(uint32_t)) != cudaSuccess)
    return fail(HGRD_EDEVICE, "pinned host allocation failed");
  for (uint32_t i = 0; i < n; i++) b->h_progs[i] = items[i]->bound->prog;
  // specialised kernels for the items that always run the device-wide pipeline
  if (b->opts.flags & HGRD_BATCH_JIT)
    for (uint32_t i = 0; i < n; i++) {
      const Bound& Bi = *items[i]->bound;
      if (small_ok(Bi, SB_KEYS)) continue;
      const int rc = jit_prepare(Bi, Bi.prog.smode != 0, nullptr);
      if (rc) return rc;
    }
  b->streams.resize(MAX_STREAMS);
  b->join.resize(MAX_STREAMS);
  note_created(2 * MAX_STREAMS + 1);
  for (uint32_t j = 0; j < MAX_STREAMS; j++) {
    if (cudaStreamCreateWithFlags(&b->streams[j], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) != cudaSuccess)
      return fail(HGRD_EDEVICE, "stream creation failed");
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(HGRD_EDEVICE, "event creation failed");
  // workspace: programs, order, verdicts, witnesses, queue, then one region per
  // large-item stream, sized for the largest item that could ever run there
  hgrd_check_opts io{};
  io.flags = HGRD_NO_PAIR;
  size_t region = 256;
  for (uint32_t i = 0; i < n; i++) region = std::max(region, item_workspace_bytes(*items[i]->bound, &io));
  b->region_bytes = align256(region);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  b->off_progs = take(n * sizeof(DProg));
  b->off_order = take(n * 4);
  b->off_outs = take(n * OUT_WORDS * 8);
  b->off_wits = take((size_t)n * b->wcap * 8);
  b->off_queue = take(256);
  b->off_regions = take((MAX_STREAMS - 1) * b->region_bytes);
  b->total = off;
  plan(b.get());
  *out = b.release();
  return HGRD_OK;
}

int hgrd_batch_workspace_size(const hgrd_batch* b, size_t* bytes) {
  if (!b || !bytes) return fail(HGRD_EINVAL, "null argument");
  *bytes = b->total;
  return HGRD_OK;
}

int hgrd_batch_run(hgrd_batch* b, void* d_ws, size_t ws_bytes, void* stream) {
  if (!b || !d_ws) return fail(HGRD_EINVAL, "null argument");
  if (((uintptr_t)d_ws & 255) != 0) return fail(HGRD_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < b->total) return fail(HGRD_ENOMEM, "workspace too small: need " + std::to_string(b->total));
  cudaStream_t s = (cudaStream_t)stream;
  g_stats = hgrd_stats{};
  if (!(b->opts.flags & HGRD_BATCH_GRAPH)) return enqueue_batch(b, (char*)d_ws, s);
  if (!b->exec || b->exec_ws != d_ws || b->exec_stream != s) {
    drop_graph(b);
    cudaStream_t cap = nullptr;
    note_created(2);  // the capture stream and the instantiated graph
    BK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    BK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_batch(b, (char*)d_ws, cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(HGRD_EDEVICE, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(HGRD_EDEVICE, std::string("graph instantiate: ") + cudaGetErrorString(e));
    b->exec_ws = d_ws;
    b->exec_stream = s;
  }
  const uint64_t launches = g_stats.kernel_launches;
  BK(cudaGraphLaunch(b->exec, s));
  g_stats.kernel_launches = launches;
  return HGRD_OK;
}

int hgrd_batch_collect(hgrd_batch* b, void* d_ws, size_t ws_bytes, void* stream, hgrd_item_verdict* v,
                       hgrd_witness* w, uint32_t wcap) {
  if (!b || !d_ws || !v) return fail(HGRD_EINVAL, "null argument");
  if (ws_bytes < b->total) return fail(HGRD_ENOMEM, "workspace too small");
  if (wcap && !w) return fail(HGRD_EINVAL, "null witness buffer");
  std::vector<uint64_t> outs, wits;
  int rc = read_outs(b, (char*)d_ws, (cudaStream_t)stream, &outs, &wits);
  if (rc) return rc;
  int worst = HGRD_OK;
  for (size_t i = 0; i < b->items.size(); i++) {
    const int st = decode_item(b, i, &outs[i * OUT_WORDS], &wits[i * b->wcap], &v[i], w, wcap);
    if (st) worst = st;
  }
  return worst;
}

int hgrd_batch_tune(hgrd_batch* b, void* d_ws, size_t ws_bytes, void* stream, hgrd_batch_opts* chosen) {
  if (!b || !d_ws) return fail(HGRD_EINVAL, "null argument");
  if (ws_bytes < b->total) return fail(HGRD_ENOMEM, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t limits[] = {0, 1024, (uint32_t)SB_KEYS};
  const uint32_t nstreams[] = {2, 4, 8, 16};
  cudaEvent_t e0, e1;
  note_created(2);
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  float best = 1e30f;
  uint32_t best_l = b->small_limit, best_s = b->nstreams;
  const uint32_t save_flags = b->opts.flags;
  b->opts.flags &= ~(uint32_t)HGRD_BATCH_GRAPH;
  for (uint32_t l : limits)
    for (uint32_t ns : nstreams) {
      b->small_limit = l;
      b->nstreams = ns;
      plan(b);
      float ms = 0;
      for (int rep = 0; rep < 2; rep++) {  // the first run warms up
        BK(cudaEventRecord(e0, s));
        int rc = enqueue_batch(b, (char*)d_ws, s);
        if (rc) return rc;
        BK(cudaEventRecord(e1, s));
        BK(cudaEventSynchronize(e1));
        BK(cudaEventElapsedTime(&ms, e0, e1));
      }
      if (ms < best) {
        best = ms;
        best_l = l;
        best_s = ns;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->opts.flags = save_flags;
  b->small_limit = best_l;
  b->nstreams = best_s;
  plan(b);
  drop_graph(b);
  if (chosen) {
    *chosen = b->opts;
    chosen->small_keys = best_l ? best_l : 1;
    chosen->streams = best_s;
  }
  return HGRD_OK;
}

int hgrd_batch_rank_prepare(hgrd_batch* b) {
  if (!b) return fail(HGRD_EINVAL, "null argument");
  constexpr uint32_t MAXP = 32 * 33 / 2;
  const size_t n = b->items.size();
  b->pair_off.assign(n + 1, 0);
  b->pair_ab.clear();
  b->cover.assign(n, 0);
  b->feat.clear();
  std::vector<float> f((size_t)MAXP * HGRD_MLP_IN);
  std::vector<uint8_t> ab(2 * MAXP);
  for (size_t i = 0; i < n; i++) {
    uint32_t np = 0;
    const int rc = hgrd_pair_features(b->items[i], f.data(), ab.data(), MAXP, &np);
    if (rc < 0) return rc;
    b->feat.insert(b->feat.end(), f.begin(), f.begin() + (size_t)np * HGRD_MLP_IN);
    for (uint32_t k = 0; k < np; k++) {
      b->pair_ab.push_back((uint32_t)ab[2 * k] | ((uint32_t)ab[2 * k + 1] << 8));
      b->cover[i] |= (1u << ab[2 * k]) | (1u << ab[2 * k + 1]);
    }
    b->pair_off[i + 1] = b->pair_off[i] + np;
  }
  const size_t np = b->pair_off[n];
  size_t off = align256(b->total);
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  b->off_feat = take(np * HGRD_MLP_IN * 4);
  b->off_logit = take(np * 4);
  b->off_poff = take((n + 1) * 4);
  b->off_pab = take(np * 4);
  b->off_cover = take(n * 4);
  b->off_dmask = take(n * 4);
  b->off_rmask = take(n * 4);
  b->off_mlp = take(hgrd_mlp_workspace_bytes((uint32_t)std::max<size_t>(np, 1)));
  b->rank_total = off;
  b->rank_ready = true;
  b->feat_ws = nullptr;
  return HGRD_OK;
}

int hgrd_batch_ranked_workspace_size(const hgrd_batch* b, size_t* bytes) {
  if (!b || !bytes) return fail(HGRD_EINVAL, "null argument");
  if (!b->rank_ready) return fail(HGRD_EINVAL, "call hgrd_batch_rank_prepare first");
  *bytes = b->rank_total;
  return HGRD_OK;
}

int hgrd_batch_check_ranked(hgrd_batch* b, const void* d_model, uint32_t topk, float min_score, void* d_ws,
                            size_t ws_bytes, void* stream, hgrd_item_verdict* v, hgrd_witness* w, uint32_t wcap,
                            uint8_t* stage, hgrd_batch_rank_info* info) {
  if (!b || !d_ws || !v) return fail(HGRD_EINVAL, "null argument");
  if (!b->rank_ready) return fail(HGRD_EINVAL, "call hgrd_batch_rank_prepare first");
  if (((uintptr_t)d_ws & 255) != 0) return fail(HGRD_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < b->rank_total) return fail(HGRD_ENOMEM, "workspace too small: need " + std::to_string(b->rank_total));
  if (wcap && !w) return fail(HGRD_EINVAL, "null witness buffer");
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  const size_t n = b->items.size();
  const uint32_t np = b->pair_off[n];
  hgrd_batch_rank_info inf{};
  inf.n_pairs = np;
  g_stats = hgrd_stats{};
  auto t0 = std::chrono::steady_clock::now();
  // 1. the features are static per binding: uploaded once per workspace
  if (b->feat_ws != d_ws) {
    BK(cudaMemcpyAsync(ws + b->off_feat, b->feat.data(), b->feat.size() * 4, cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(ws + b->off_poff, b->pair_off.data(), (n + 1) * 4, cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(ws + b->off_pab, b->pair_ab.data(), (size_t)np * 4, cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(ws + b->off_cover, b->cover.data(), n * 4, cudaMemcpyHostToDevice, s));
    b->feat_ws = d_ws;
  }
  // 2. one inference over every eligible pair of every item, then the
  // top-k access masks on the device
  std::vector<uint32_t> dmask(n, 0);
  if (np && d_model && topk) {
    int rc = hgrd_mlp_predict(d_model, (const float*)(ws + b->off_feat), np, (float*)(ws + b->off_logit),
                              ws + b->off_mlp, hgrd_mlp_workspace_bytes(np), s);
    if (rc) return rc;
    const uint32_t grid = (uint32_t)std::min<size_t>((n + 7) / 8, 4096);
    topk_mask_kernel<<<grid, 256, 0, s>>>((const float*)(ws + b->off_logit), (const uint32_t*)(ws + b->off_poff),
                                          (const uint32_t*)(ws + b->off_pab), (const uint32_t*)(ws + b->off_cover),
                                          (uint32_t)n, topk, min_score, (uint32_t*)(ws + b->off_dmask));
    BK(cudaGetLastError());
    g_stats.kernel_launches += 5;
    BK(cudaMemcpyAsync(dmask.data(), ws + b->off_dmask, n * 4, cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
  }
  auto t1 = std::chrono::steady_clock::now();
  // 3. stage one: every item, large ranked items restricted to the accesses of
  // their top pairs (small items are whole checks on chip already)
  std::vector<uint8_t> is_small(n, 0), run(n, 1), done(n, 1);
  for (uint32_t id : b->small) is_small[id] = 1;
  std::vector<uint32_t> masks(n, 0xffffffffu);
  for (size_t i = 0; i < n; i++)
    if (!is_small[i] && dmask[i]) {
      masks[i] = dmask[i];
      inf.ranked++;
    }
  int rc = enqueue_batch(b, ws, s, run.data(), masks.data());
  if (rc) return rc;
  std::vector<uint64_t> outs, wits;
  rc = read_outs(b, ws, s, &outs, &wits);
  if (rc) return rc;
  int worst = HGRD_OK;
  for (size_t i = 0; i < n; i++) {
    const uint64_t* o = &outs[i * OUT_WORDS];
    const bool racy = o[2] > 0;
    if (masks[i] != 0xffffffffu && !racy && masks[i] != b->cover[i]) {
      done[i] = 0;  // clean on part of its accesses: the whole check decides
      continue;
    }
    if (masks[i] != 0xffffffffu) inf.confirmed += racy;
    if (stage) stage[i] = masks[i] == 0xffffffffu ? 0 : (racy ? 1 : 3);
    const int st = decode_item(b, i, o, &wits[i * b->wcap], &v[i], w, wcap);
    if (st) worst = st;
  }
  auto t2 = std::chrono::steady_clock::now();
  // 4. stage two: the whole check of the items stage one left open
  for (size_t i = 0; i < n; i++) {
    run[i] = !done[i];
    masks[i] = 0xffffffffu;
    inf.second += run[i];
  }
  if (inf.second) {
    rc = enqueue_batch(b, ws, s, run.data(), masks.data());
    if (rc) return rc;
    rc = read_outs(b, ws, s, &outs, &wits);
    if (rc) return rc;
    for (size_t i = 0; i < n; i++) {
      if (!run[i]) continue;
      if (stage) stage[i] = 2;
      const int st = decode_item(b, i, &outs[i * OUT_WORDS], &wits[i * b->wcap], &v[i], w, wcap);
      if (st) worst = st;
    }
  }
  auto t3 = std::chrono::steady_clock::now();
  inf.ms_score = std::chrono::duration<float, std::milli>(t1 - t0).count();
  inf.ms_stage1 = std::chrono::duration<float, std::milli>(t2 - t1).count();
  inf.ms_stage2 = std::chrono::duration<float, std::milli>(t3 - t2).count();
  if (info) *info = inf;
  return worst;
}

void hgrd_batch_free(hgrd_batch* b) {
  if (!b) return;
  drop_graph(b);
  for (auto st : b->streams)
    if (st) cudaStreamDestroy(st);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->h_progs) cudaFreeHost(b->h_progs);
  if (b->h_order) cudaFreeHost(b->h_order);
  delete b;
}

}  // extern "C"
