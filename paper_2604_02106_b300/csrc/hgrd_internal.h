// Library-internal definitions shared by the host compiler (desc.cpp) and the
// kernels (*.cu).  Nothing here is part of the C ABI.
#pragma once
#include <cstddef>
#include <cstdint>

#if !defined(__CUDACC_RTC__)  // the run-time compiled kernels need none of the C ABI
#include "../../include/hgrd.h"
#endif

#if defined(__CUDACC__)
#define HGRD_HD __host__ __device__ __forceinline__
#else
#define HGRD_HD inline
#endif

namespace hgrd {

constexpr int MAXACC = 32;
constexpr int MAXARR = 32;
constexpr int MAXLOOP = 4;
constexpr int NVAR = 10;  // slots 0..5: tx ty tz bx by bz; 6..9: loop counters
constexpr int MAXTERM = 768;
constexpr int MAXOP = 192;
constexpr int MAXGUARD = 128;
constexpr int MAXSLOT = 128;

// Division by a positive constant d of a numerator whose magnitude is below
// 2^N (N = 31 on the 32-bit path, 62 on the 64-bit path): Granlund &
// Montgomery, "Division by invariant integers using multiplication" (PLDI
// 1994), Theorem 4.2 with l = ceil(log2 d), m = floor(2^(N+l)/d) + 1,
// q = floor(|n| * m / 2^(N+l)); the sign follows C truncation.
struct Magic {
  uint64_t m;
  int32_t shift;  // N + l
  int32_t pad;
};

HGRD_HD uint64_t magic_udiv(uint64_t n, const Magic& g) {
#if defined(__CUDA_ARCH__)
  uint64_t lo = n * g.m, hi = __umul64hi(n, g.m);
#else
  unsigned __int128 p = (unsigned __int128)n * g.m;
  uint64_t lo = (uint64_t)p, hi = (uint64_t)(p >> 64);
#endif
  if (g.shift >= 64) return hi >> (g.shift - 64);
  return (hi << (64 - g.shift)) | (lo >> g.shift);
}

// 32-bit path: |n| < 2^31 and m <= 2^32 + 1, so |n| * m < 2^64 fits a
// single 64-bit product.
HGRD_HD int32_t magic_div32(int32_t n, const Magic& g) {
  uint64_t a = (uint64_t)(n < 0 ? -(int64_t)n : (int64_t)n);
  int32_t q = (int32_t)((a * g.m) >> g.shift);
  return n < 0 ? -q : q;
}
// non-negative numerator below 2^31, N = 31 magic number
HGRD_HD uint32_t magic_udiv31(uint32_t n, const Magic& g) { return (uint32_t)(((uint64_t)n * g.m) >> g.shift); }
HGRD_HD int64_t magic_div64(int64_t n, const Magic& g) {
  uint64_t a = (uint64_t)(n < 0 ? -n : n);
  int64_t q = (int64_t)magic_udiv(a, g);
  return n < 0 ? -q : q;
}

struct DTerm {
  int32_t slot, pad;
  int64_t coef;
};
struct DLin {
  int32_t first, n;  // terms [first, first + n)
  int64_t c0;
};
enum { OP_LIN = 0, OP_DIV = 1, OP_MOD = 2 };
struct DOp {
  int32_t kind, dst;
  DLin lin;
  int64_t d;
  Magic mg;
};
struct DAcc {
  DLin idx, iv, wv;  // index, block-barrier interval, warp-barrier interval
  int32_t gfirst, ng;  // guards: each DLin must be >= 0
  int32_t G;           // granule keys per instance (width / granule)
  int32_t arr;         // descriptor array id
  int64_t maxidx;      // in bounds iff 0 <= idx <= maxidx
  uint64_t cbase;      // first cell code of the array
  uint64_t ngran;      // granules of one copy of the array
  int32_t shared, dead;
  int32_t bounds_free, pad;
  int64_t sgbase;  // shared arrays: first granule of the array among one block's shared granules
};

// The acquire-release guard of an access whose guard element the exact scan
// evaluates per instance (Sec. 6.5): AFFINE, c0 + sum c[v] * id[v] over the
// thread and block ids (tx ty tz bx by bz; constants included), or OWN, the
// access's own element (granule / G of the location).
enum { LOCK_NONE = 0, LOCK_AFFINE = 1, LOCK_OWN = 2 };
struct DLock {
  int32_t form, arr;   // LOCK_*, lock array
  int32_t scope, pad;  // narrower scope of the guard's parts: 0 block, 1 device
  int64_t c0, c[6];
};

// Everything the kernels need about one bound descriptor.  Lives in the
// device workspace; all lanes read it with uniform addresses.
struct alignas(16) DProg {
  int32_t grid[3], block[3];
  int32_t nthr, wpb;  // threads and warps per block
  int64_t nblk, nunits;
  int32_t nloop, nacc;
  int32_t ub[MAXLOOP];
  int64_t nit;     // loop vectors per thread
  int64_t itc;     // loop vectors per unit: a unit is (block, warp, chunk of itc loop vectors)
  int64_t nchunk;  // chunks per (block, warp)
  int32_t wide, nfix, niter, nslot;
  int32_t nterm, nguard, pad0, pad1;
  // key layout: key = ((cell << IVB | iv - ivmin) << PB) | lin_b << (WVB+TB+AB)
  //                   | (wv - wvmin) << (TB+AB) | lin_t << AB | access
  // (WVB = 0 unless warp barriers split some warp's accesses)
  int32_t AB, TB, BB, IVB, PB, RB;
  int64_t ivmin;
  uint64_t shared_cell_base;  // cell codes at or above this belong to shared arrays
  uint32_t wmask;             // accesses that write (W or A)
  int32_t nlay;               // arrays in layout order (global first)
  // accesses with at least one live access they may race with (pair rule E);
  // the others are counted but their keys are never written
  uint32_t emask, pad3;
  // block-local ordering of shared-array keys: their runs never leave a block,
  // so they are written straight into per-block (granule, interval) bins
  // instead of going through the global sort
  int32_t smode, niv;         // smode: shared keys use the bins; niv: intervals
  int64_t nsbins;             // bins of one block: shared granules x intervals
  int32_t RBG, pad2;          // run-code bits of the global-array keys (the sorted ones)
  uint64_t scap;              // room for keys of candidate bins (more: HGRD_ENOMEM)
  // warp-barrier intervals (Sec. 5.2): WVB bits of wv - wvmin sit between the
  // block and the thread, and the sort then orders keys by (run, interval,
  // block, warp interval) from bit SB up; without them SB = PB
  int32_t WVB, SB;
  int64_t wvmin;
  // cell filter: the count pass records per cell (granule of an array copy)
  // the smallest and largest (block << TB | thread) touching it and whether a
  // writer did; only keys of cells with a writer and two threads are sorted.
  // Table at the count pass's key pointer: gmin[ncells], gmax[ncells] (u32),
  // writer bits[(ncells + 31) / 32]
  int32_t cfilter, cfilter_auto;  // table fits; worth it by default
  uint64_t ncells;
  // division by nchunk, wpb, grid x, grid y, block x, block y of numerators
  // below 2^31 (unit, block and thread ids): magic numbers with N = 31
  Magic dv[6];
  uint32_t einter[MAXACC], eintra[MAXACC];
  // access pairs guarded at one lock array whose guard elements can differ
  // between instances: the exact scan decides them pair by pair of
  // instances (lockpair[a] bit b), the other pairs from the summaries
  uint32_t lockpair[MAXACC];
  int32_t lockany, pad5;
  DLock lock[MAXACC];
  uint64_t lay_cbase[MAXARR + 1];
  uint64_t lay_ngran[MAXARR];
  int32_t lay_arr[MAXARR], lay_shared[MAXARR];
  DOp ops[MAXOP];  // [0, nfix): once per (block, warp); [nfix, nfix+niter): per loop vector
  DAcc acc[MAXACC];
  DLin guard[MAXGUARD];
  DTerm term[MAXTERM];
};

// Pair-search record of one instance touching the minimal witness's granule.
struct PairRec {
  uint32_t blk, thr;
  uint32_t it[4];
  int32_t acc, pad;
  int64_t iv;
};

// Raw / canonical witness packed into 64 bits so the same radix sort orders
// them: space(1) array(5) granule(40) acc_lo(5) acc_hi(5) kind(3), low to high
// significance reversed (kind in the low bits).
HGRD_HD uint64_t pack_witness(uint32_t space, uint32_t arr, uint64_t gran, uint32_t lo, uint32_t hi, uint32_t kind) {
  return ((uint64_t)space << 58) | ((uint64_t)arr << 53) | (gran << 13) | ((uint64_t)lo << 8) | ((uint64_t)hi << 3) |
         kind;
}
constexpr int WIT_SORT_LO = 3;   // lowest sorted bit (the kind mask is merged, not sorted)
constexpr int WIT_SORT_HI = 59;  // one past the highest used bit

// Device counters block at the start of the workspace (uint64 words).
enum {
  C_NKEYS = 0,
  C_NOOB,
  C_NCAND,
  C_NRAW,
  C_ERR,
  C_NUNIQ,
  C_KIND0,
  C_KIND1,
  C_KIND2,
  C_NPAIR,
  C_NG,   // keys of global arrays (the sorted stream)
  C_NS,   // keys of shared arrays (smode: counted per block bin, not sorted)
  C_NSC,  // keys of shared arrays in candidate bins (smode: written behind the sorted keys)
  C_NDROP,  // keys of accesses that cannot race with any access (counted, never written)
  C_NRAWBIG,  // raw witnesses left to the device-wide merge (0 when one CTA merges them)
  C_NPB,      // pair search: 1 + blocks listed for it (0: search every unit)
  C_NGC = 33,  // cell filter: global keys kept for the sort (C_NG: all written ones)
  C_TAIL = 34,  // 1 when one CTA sorted the keys on the digits after the first pass
  C_NCOMPACT = 35,  // cell filter: kept keys the write pass also appended to the compact buffer
  C_TICKET0 = 16,  // one tile ticket per sort pass (up to 16 passes)
  C_PAIRS = 64,    // racy access-pair matrices: 3 kinds x 32 rows x 32 bits, two rows per word
  C_SMALLQ = 120,  // one-CTA path of a small check: work queue, then an order word of zero
  C_WORDS = 128
};
enum { ERR_TIMEOUT = 1, ERR_OVERFLOW = 2, ERR_SHARED_FULL = 4, ERR_SMALL_FULL = 8, ERR_LOCK_RUN = 16 };
// most keys of one location the exact scan checks instance pair by instance
// pair for guards whose elements vary (more: ERR_LOCK_RUN)
constexpr uint64_t LOCK_RUN_MAX = 8192;

// the expansion kernels run 8 warps per CTA, one simulated warp per warp
constexpr int EXP_THREADS = 256;
// most (shared granule, interval) bins of one block in the block-local mode
constexpr int SBIN_MAX = 4096;
// block-local mode: base of a block that has no bin-table row (no candidate bin)
constexpr uint64_t NO_ROW = ~0ull;
// 32-bit shared-memory words the block-local expansion needs for nb bins:
// mode 3 = count, min / max thread, writer bits, digit histogram, scan scratch;
// mode 4 = write cursors
HGRD_HD uint64_t block_body_words(int mode, uint64_t nb) {
  return mode == 3 ? ((3 * nb + (nb + 31) / 32 + 256 + 1) & ~1ull) + 2 * 10 : nb;
}

}  // namespace hgrd

static_assert(sizeof(hgrd::DProg) % 16 == 0, "DProg is copied to shared memory in 16-byte words");
