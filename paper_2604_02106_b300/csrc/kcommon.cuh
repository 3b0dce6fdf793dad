// Device code shared by the single-check kernels (kernels.cu), the batched
// kernels (batch.cu) and the specialised expansion kernels compiled at run
// time: evaluation of the compiled affine program, the expansion of one
// simulated warp, and the exact scan of one run.
#pragma once
#if !defined(__CUDACC_RTC__)
#include <cuda_runtime.h>

#include "kernels.cuh"
#else
#include "hgrd_internal.h"
#endif

namespace hgrd {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint64_t shr64(uint64_t x, int s) { return s >= 64 ? 0 : x >> s; }
__device__ __forceinline__ uint64_t lowbits(uint64_t x, int n) { return n >= 64 ? x : (x & ((1ull << n) - 1)); }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T divq(T n, const Magic& g);
template <>
__device__ __forceinline__ int32_t divq<int32_t>(int32_t n, const Magic& g) {
  return magic_div32(n, g);
}
template <>
__device__ __forceinline__ int64_t divq<int64_t>(int64_t n, const Magic& g) {
  return magic_div64(n, g);
}

// c0 + sum(coef * slot) over the lane's column of the warp's slot file
template <typename T>
__device__ __forceinline__ T lin_eval(const DProg* __restrict__ P, const DLin& L, const T* sl, int lane) {
  T v = (T)L.c0;
  for (int t = 0; t < L.n; ++t) {
    const DTerm tm = P->term[L.first + t];
    v += (T)tm.coef * sl[tm.slot * 32 + lane];
  }
  return v;
}

template <typename T>
__device__ __forceinline__ void run_ops(const DProg* __restrict__ P, int first, int count, T* sl, int lane) {
  for (int k = first; k < first + count; ++k) {
    const DOp op = P->ops[k];
    T v = lin_eval<T>(P, op.lin, sl, lane);
    if (op.kind == OP_DIV) {
      v = divq<T>(v, op.mg);
    } else if (op.kind == OP_MOD) {
      v = v - divq<T>(v, op.mg) * (T)op.d;
    }
    sl[op.dst * 32 + lane] = v;
  }
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t x, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// exclusive scan over a CTA of 256 threads' values; `ws` holds 8 words
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* ws, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = warp_incl_scan(v, lane);
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t s = lane < 8 ? ws[lane] : 0;
    uint64_t si = warp_incl_scan(s, lane);
    if (lane < 8) ws[lane] = si - s;
    if (lane == 7 && total) *total = si;
  }
  __syncthreads();
  uint64_t r = x - v + ws[warp];
  __syncthreads();
  return r;
}

// With warp-barrier intervals the interval handed to the key is
// ivmin + ((iv - ivmin) << WVB | wv - wvmin): make_key splits it again.
__device__ __forceinline__ int64_t pack_wv(const DProg* __restrict__ P, int64_t iv, int64_t wv) {
  return P->ivmin + (int64_t)((uint64_t)(iv - P->ivmin) << P->WVB | (uint64_t)(wv - P->wvmin));
}

// Expansion of unit u = (block b, warp w of the block) of the user kernel,
// lane = simulated thread.  For every loop vector and every access in `only`
// (bit per access id), evaluates guards and index and calls
//   step(a, A, inb, bal, idx, iv, b, lt, ic)
// whenever some lane of the warp holds a live in-bounds instance (inb for
// this lane, bal = ballot of inb).  Returns this lane's live instances that
// fell outside their array.
template <typename T, typename Step>
__device__ __forceinline__ uint64_t expand_unit(const DProg* __restrict__ P, T* sl, int lane, int64_t u,
                                                uint32_t only, Step&& step) {
  const int nthr = P->nthr, wpb = P->wpb, nacc = P->nacc, nloop = P->nloop;
  const int bdx = P->block[0], bdy = P->block[1];
  const int64_t gdx = P->grid[0], gdy = P->grid[1];
  const int64_t nit = P->nit;
  const int64_t bw = u / P->nchunk;                // (block, warp)
  const int64_t it0 = (u - bw * P->nchunk) * P->itc;  // first loop vector of the chunk
  const int64_t it1 = min(nit, it0 + P->itc);
  const int64_t b = bw / wpb;
  const int lt = (int)(bw - b * wpb) * 32 + lane;
  const bool act = lt < nthr;
  sl[0 * 32 + lane] = (T)(lt % bdx);
  sl[1 * 32 + lane] = (T)((lt / bdx) % bdy);
  sl[2 * 32 + lane] = (T)(lt / (bdx * bdy));
  sl[3 * 32 + lane] = (T)(b % gdx);
  sl[4 * 32 + lane] = (T)((b / gdx) % gdy);
  sl[5 * 32 + lane] = (T)(b / (gdx * gdy));
  for (int l = 0; l < MAXLOOP; ++l) sl[(6 + l) * 32 + lane] = 0;
  run_ops<T>(P, 0, P->nfix, sl, lane);
  uint64_t oob = 0;
  // loop counters of it0 (mixed radix, innermost loop fastest)
  int32_t ic[MAXLOOP] = {0, 0, 0, 0};
  if (it0 > 0) {  // it0 > 0 implies every loop bound is at least 1
    int64_t r = it0;
    for (int l = nloop - 1; l >= 0; --l) {
      ic[l] = (int32_t)(r % P->ub[l]);
      r /= P->ub[l];
    }
  }
  for (int64_t it = it0; it < it1; ++it) {
    if (it > it0) {
      int l = nloop - 1;
      while (l >= 0) {
        if (++ic[l] < P->ub[l]) break;
        ic[l] = 0;
        --l;
      }
    }
    for (int l = 0; l < nloop; ++l) sl[(6 + l) * 32 + lane] = (T)ic[l];
    run_ops<T>(P, P->nfix, P->niter, sl, lane);
    for (int a = 0; a < nacc; ++a) {
      const DAcc& A = P->acc[a];
      if (A.dead || !((only >> a) & 1u)) continue;
      bool live = act;
      const int ng = A.ng, gf = A.gfirst;
      for (int g = 0; g < ng; ++g) {
        const DLin gl = P->guard[gf + g];
        live = live && lin_eval<T>(P, gl, sl, lane) >= 0;
      }
      const DLin il = A.idx;
      const T idx = lin_eval<T>(P, il, sl, lane);
      const bool inb = live && (A.bounds_free || (idx >= 0 && (int64_t)idx <= A.maxidx));
      oob += (live && !inb) ? 1 : 0;
      const unsigned bal = __ballot_sync(FULL, inb);
      if (bal == 0) continue;
      int64_t iv = 0;
      if (inb) {
        const DLin vl = A.iv;
        iv = (int64_t)lin_eval<T>(P, vl, sl, lane);
        if (P->WVB) iv = pack_wv(P, iv, (int64_t)lin_eval<T>(P, A.wv, sl, lane));
      }
      step(a, A, inb, bal, (int64_t)idx, iv, b, lt, ic);
    }
  }
  return oob;
}

// granule j of a live in-bounds instance as a sort key:
// ((cell << IVB | interval - ivmin) << PB) | block << (WVB+TB+AB) | warp interval << (TB+AB)
//   | thread << AB | access
__device__ __forceinline__ uint64_t make_key(const DProg* __restrict__ P, const DAcc& A, int a, int64_t idx,
                                             int64_t iv, int64_t b, int lt, int j) {
  const uint64_t cell = A.cbase + (A.shared ? (uint64_t)b * A.ngran : 0ull) + (uint64_t)idx * (uint64_t)A.G + j;
  const uint64_t ivw = (uint64_t)(iv - P->ivmin);  // (interval << WVB) | warp interval
  const int WVB = P->WVB, TA = P->TB + P->AB;
  return (((cell << P->IVB) | (ivw >> WVB)) << P->PB) | ((uint64_t)b << (WVB + TA)) |
         (lowbits(ivw, WVB) << TA) | ((uint64_t)lt << P->AB) | (uint64_t)a;
}

// min / max of one id over a group of instances
struct Sum {
  bool p;
  uint32_t lo, hi;
  __device__ __forceinline__ void reset() { p = false; }
  __device__ __forceinline__ void add(uint32_t v) {
    if (!p) {
      p = true;
      lo = hi = v;
    } else {
      lo = v < lo ? v : lo;
      hi = v > hi ? v : hi;
    }
  }
};

// lane = access a: the accesses b present in the group that form a pair with
// two different ids among their instances (every present b, unless a and b
// are both one and the same single id)
__device__ __forceinline__ uint32_t racy_row(const Sum& s, int lane) {
  const unsigned P = __ballot_sync(FULL, s.p);
  if (!P) return 0;
  const bool single = s.p && s.lo == s.hi;
  const unsigned S = __ballot_sync(FULL, single);
  const unsigned eq = __match_any_sync(FULL, single ? s.lo : (0x80000000u | (unsigned)lane));
  const unsigned nonr = single ? (eq & S) : 0u;
  return s.p ? (P & ~nonr) : 0u;
}

// Exact race kinds of the run starting at key s (end e, or 0 = until the run
// id changes) of sorted keys[0, n).  Lane a gets, for each access b, whether
// the pair (a, b) races across blocks (global memory, any interval), inside a
// block between warps, or inside a warp, in the same interval (Table 2) and,
// for the intra-warp kind, the same warp interval (Sec. 5.2: a warp barrier
// orders the threads of one warp only).
struct RunMasks {
  uint64_t rid;
  uint32_t inter, blk, warp;
  bool lock_overflow = false;  // guards decided per instance on a run longer than LOCK_RUN_MAX
};

// (space, array, granule) of run id `rid` in the array layout
__device__ __forceinline__ void run_location(const DProg* __restrict__ P, uint64_t rid, uint32_t* space, uint32_t* arr,
                                             uint64_t* gran) {
  int li = 0;
  while (li + 1 < P->nlay && P->lay_cbase[li + 1] <= rid) ++li;
  const uint64_t cell = rid - P->lay_cbase[li];
  const bool sh = P->lay_shared[li];
  *gran = sh ? cell % P->lay_ngran[li] : cell;
  *arr = (uint32_t)P->lay_arr[li];
  *space = sh ? 1u : 0u;
}

// The element a guarded instance holds (Sec. 6.5's syn() address): affine in
// the ids of its thread and block, or its own element on granule `gran`.
__device__ __forceinline__ int64_t lock_element(const DProg* __restrict__ P, int a, uint32_t blk, uint32_t thr,
                                                uint64_t gran) {
  const DLock& L = P->lock[a];
  if (L.form == LOCK_OWN) return (int64_t)(gran / (uint64_t)P->acc[a].G);
  const int64_t tx = thr % P->block[0], ty = (thr / P->block[0]) % P->block[1], tz = thr / (P->block[0] * P->block[1]);
  const int64_t bx = blk % P->grid[0], by = (blk / P->grid[0]) % P->grid[1], bz = blk / (P->grid[0] * P->grid[1]);
  return L.c0 + L.c[0] * tx + L.c[1] * ty + L.c[2] * tz + L.c[3] * bx + L.c[4] * by + L.c[5] * bz;
}

// Race kinds of the guarded pairs whose elements vary, instance pair by
// instance pair over the run [s, end) (Table 2 with Sec. 6.5's addr(syn)
// test): a pair of different threads races with its kind (inter-block
// across blocks in global memory; else same barrier interval, different
// warps: intra-block; same warp and warp interval: intra-warp) unless both
// are guarded at one element and the guards' narrower scope covers the kind
// (device scope across blocks).  Rows by lane = access, as the summaries.
__device__ __forceinline__ void lock_pairs_run(const uint64_t* keys, uint64_t s, uint64_t end, const DProg* __restrict__ P,
                                               int lane, bool glob, uint64_t gran, RunMasks& R) {
  const int PB = P->PB, AB = P->AB, TB = P->TB, BB = P->BB, WVB = P->WVB;
  uint32_t mi = 0, mb = 0, mw = 0;
  for (uint64_t xi = s; xi < end; ++xi) {
    const uint64_t kx = keys[xi];
    const uint32_t ax = (uint32_t)lowbits(kx, AB);
    const uint32_t rowx = P->lockpair[ax];
    if (!rowx) continue;
    const uint32_t bx = (uint32_t)lowbits(kx >> (AB + TB + WVB), BB), tx = (uint32_t)lowbits(kx >> AB, TB);
    const uint64_t subx = shr64(kx, PB);
    const uint32_t wvx = (uint32_t)lowbits(kx >> (AB + TB), WVB);
    const int64_t lx = lock_element(P, (int)ax, bx, tx, gran);
    const uint32_t allow_inter = P->einter[ax], allow_intra = P->eintra[ax];
    for (uint64_t y0 = xi + 1; y0 < end; y0 += 32) {
      const uint64_t yi = y0 + lane;
      uint32_t k = 0, ay = 0;
      if (yi < end) {
        const uint64_t ky = keys[yi];
        ay = (uint32_t)lowbits(ky, AB);
        if ((rowx >> ay) & 1u) {
          const uint32_t by = (uint32_t)lowbits(ky >> (AB + TB + WVB), BB), ty = (uint32_t)lowbits(ky >> AB, TB);
          if (bx != by) k = glob ? 1u : 0u;
          else if (tx == ty || shr64(ky, PB) != subx) k = 0;
          else if ((tx >> 5) != (ty >> 5)) k = 2;
          else k = (uint32_t)lowbits(ky >> (AB + TB), WVB) == wvx ? 4u : 0u;
          k &= ((allow_inter >> ay) & 1u) | (((allow_intra >> ay) & 1u) ? 6u : 0u);
          if (k && P->lock[ax].arr == P->lock[ay].arr && lx == lock_element(P, (int)ay, by, ty, gran) &&
              (k != 1u || min(P->lock[ax].scope, P->lock[ay].scope) == 1))
            k = 0;  // ordered by the acquire-release both hold
        }
      }
      const uint32_t r1 = __reduce_or_sync(FULL, (k & 1u) ? 1u << ay : 0u);
      const uint32_t r2 = __reduce_or_sync(FULL, (k & 2u) ? 1u << ay : 0u);
      const uint32_t r4 = __reduce_or_sync(FULL, (k & 4u) ? 1u << ay : 0u);
      if ((uint32_t)lane == ax) {
        mi |= r1;
        mb |= r2;
        mw |= r4;
      }
      mi |= ((r1 >> lane) & 1u) << ax;
      mb |= ((r2 >> lane) & 1u) << ax;
      mw |= ((r4 >> lane) & 1u) << ax;
    }
  }
  R.inter |= mi;
  R.blk |= mb;
  R.warp |= mw;
}

__device__ __forceinline__ RunMasks exact_run(const uint64_t* keys, uint64_t s, uint64_t e, uint64_t n,
                                              const DProg* __restrict__ P, int lane, uint32_t einter,
                                              uint32_t eintra, bool stop_first = false) {
  const int PB = P->PB, IVB = P->IVB, AB = P->AB, TB = P->TB, BB = P->BB, WVB = P->WVB;
  const int rsh = PB + IVB;
  RunMasks R;
  R.rid = shr64(keys[s], rsh);
  const bool glob = R.rid < P->shared_cell_base;
  // pairs decided instance pair by instance pair stay out of the summaries
  if (P->lockany && lane < MAXACC) {
    einter &= ~P->lockpair[lane];
    eintra &= ~P->lockpair[lane];
  }
  uint64_t end = s;
  // thread per (iv, block, warp interval, warp); warp per (iv, block); block
  // per run.  Keys of one (iv, block) are contiguous and ordered by warp
  // interval, each warp's keys contiguous inside a warp interval.
  Sum tw, wb, br;
  tw.reset();
  wb.reset();
  br.reset();
  uint32_t m_inter = 0, m_blk = 0, m_warp = 0;
  uint64_t cur_sub = ~0ull;
  uint32_t cur_b = 0xffffffffu, cur_w = 0xffffffffu;
  for (uint64_t pos = s;; pos += 32) {
    const uint64_t i = pos + lane;
    const bool ok = i < n && (e == 0 || i < e);
    const uint64_t kk = ok ? keys[i] : 0;
    const bool inrun = ok && shr64(kk, rsh) == R.rid;
    const unsigned m = __ballot_sync(FULL, inrun);
    const int cnt = __popc(m);
    end = pos + cnt;
    for (int jj = 0; jj < cnt; ++jj) {
      const uint64_t key = __shfl_sync(FULL, kk, jj);
      const uint64_t sub = shr64(key, PB);
      const uint32_t b = (uint32_t)lowbits(key >> (AB + TB + WVB), BB);
      const uint32_t t = (uint32_t)lowbits(key >> AB, TB);
      const uint32_t wpi = t >> 5;
      const uint32_t wgi = (uint32_t)lowbits(key >> (AB + TB), WVB) << 16 | wpi;  // (warp interval, warp)
      const uint32_t a = (uint32_t)lowbits(key, AB);
      if (sub != cur_sub || b != cur_b) {
        m_warp |= racy_row(tw, lane) & eintra;
        m_blk |= racy_row(wb, lane) & eintra;
        tw.reset();
        wb.reset();
        cur_sub = sub;
        cur_b = b;
        cur_w = wgi;
      } else if (wgi != cur_w) {
        m_warp |= racy_row(tw, lane) & eintra;
        tw.reset();
        cur_w = wgi;
      }
      if ((uint32_t)lane == a) {
        tw.add(t);
        wb.add(wpi);
        br.add(b);
      }
    }
    if (cnt < 32) break;
    // stop-at-first: every pair found so far is a real race; quit once one exists
    if (stop_first) {
      const uint32_t mi = glob ? (racy_row(br, lane) & einter) : 0u;
      if (__any_sync(FULL, (m_warp | m_blk | mi) != 0)) break;
    }
  }
  m_warp |= racy_row(tw, lane) & eintra;
  m_blk |= racy_row(wb, lane) & eintra;
  if (glob) m_inter |= racy_row(br, lane) & einter;
  R.inter = m_inter;
  R.blk = m_blk;
  R.warp = m_warp;
  if (P->lockany) {
    // the run's own end (a stop-at-first scan may have left it early)
    while (true) {
      const uint64_t i = end + lane;
      const bool inrun = i < n && (e == 0 || i < e) && shr64(keys[i], rsh) == R.rid;
      const unsigned m = __ballot_sync(FULL, inrun);
      end += __popc(m);
      if (m != FULL) break;
    }
    if (end - s > LOCK_RUN_MAX) {
      R.lock_overflow = true;
    } else {
      uint32_t space, arr;
      uint64_t gran;
      run_location(P, R.rid, &space, &arr, &gran);
      lock_pairs_run(keys, s, end, P, lane, glob, gran, R);
    }
  }
  return R;
}

// OR this lane's rows of the run into the racy-pair matrices (two 32-bit rows per word)
__device__ __forceinline__ void record_pairs(uint64_t* pairs, const RunMasks& R, int lane) {
  const int sh = 32 * (lane & 1);
  if (R.inter) atomicOr((unsigned long long*)&pairs[0 * 16 + (lane >> 1)], (unsigned long long)R.inter << sh);
  if (R.blk) atomicOr((unsigned long long*)&pairs[1 * 16 + (lane >> 1)], (unsigned long long)R.blk << sh);
  if (R.warp) atomicOr((unsigned long long*)&pairs[2 * 16 + (lane >> 1)], (unsigned long long)R.warp << sh);
}

// witness words of lane a for accesses b >= a; `n` counts them
__device__ __forceinline__ uint32_t witness_row(const RunMasks& R, int lane) {
  const uint32_t ge = lane == 0 ? FULL : ~((1u << lane) - 1u);
  return (R.inter | R.blk | R.warp) & ge;
}
__device__ __forceinline__ uint32_t witness_kind(const RunMasks& R, int b) {
  return ((R.inter >> b) & 1u) | (((R.blk >> b) & 1u) << 1) | (((R.warp >> b) & 1u) << 2);
}

}  // namespace dev
}  // namespace hgrd
