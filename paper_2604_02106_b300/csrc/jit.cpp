// Specialised expansion kernels, compiled at run time.
//
// The interpreted expansion evaluates the bound program term by term from
// shared memory: every instance pays for loads of the program's terms and
// slot values and for the loop over them.  Here the program's STRUCTURE
// (which slots each op, guard, index and interval reads, which ops divide,
// which accesses are live, how many loops) is turned into CUDA source where
// all of that is straight-line code over registers; the VALUES (coefficients,
// divisors' magic numbers, bounds, launch shape) stay in the DProg, passed by
// value as the kernel's parameter block, so every binding with the same
// structure (a parameter sweep, the same kernel at another size) reuses one
// compiled module.  The kernel bodies are the ones the interpreted kernels
// run (expand_body.cuh): only the unit expander differs.
//
// NVRTC compiles the source for sm_103a to a cubin, loaded with the runtime's
// library API.  Modules are cached per process by their source text.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "hgrd_host.h"
#include "jit.h"

namespace hgrd {

namespace {

#include "jit_headers.inc"  // kJitHeaderNames / kJitHeaders: the device headers as text (written by the build)

// Fixed-width integer and size types for the run-time compiler, which has no C library headers.
const char* kStdInt =
    "#pragma once\n"
    "typedef signed char int8_t; typedef short int16_t; typedef int int32_t; typedef long long int64_t;\n"
    "typedef unsigned char uint8_t; typedef unsigned short uint16_t; typedef unsigned int uint32_t;\n"
    "typedef unsigned long long uint64_t; typedef unsigned long long uintptr_t;\n";
const char* kStdDef = "#pragma once\ntypedef unsigned long size_t; typedef long ptrdiff_t;\n";

std::string S(long long v) { return std::to_string(v); }

// c0 + sum coef * slot, all in T, reading the values from the parameter block
std::string lin(const DProg& P, const std::string& at, const DLin& L) {
  std::string e = "((T)" + at + ".c0";
  for (int t = 0; t < L.n; t++)
    e += " + (T)P->term[" + S(L.first + t) + "].coef * s" + S(P.term[L.first + t].slot);
  return e + ")";
}

std::string op_code(const DProg& P, int k, bool declare) {
  const DOp& op = P.ops[k];
  const std::string at = "P->ops[" + S(k) + "]";
  std::string v = lin(P, at + ".lin", op.lin);
  if (op.kind == OP_DIV)
    v = "divq<T>(" + v + ", " + at + ".mg)";
  else if (op.kind == OP_MOD)
    v = "modq<T>(" + v + ", " + at + ".mg, (T)" + at + ".d)";
  return std::string("      ") + (declare ? "const T " : "") + "s" + S(op.dst) + " = " + v + ";\n";
}

// What the generated walk does with each access: which slots depend on the
// loop counters, and which accesses are evaluated once per unit (loop
// invariant; count-only; ranged: one instance repeated over the counters its
// loop guards admit) rather than once per loop vector.
struct Analysis {
  const DProg& P;
  int nl;
  std::vector<char> dep;  // slot depends on the loop counters
  explicit Analysis(const DProg& p) : P(p), nl(p.nloop), dep(MAXSLOT + 16, 0) {
    for (int l = 0; l < nl; l++) dep[6 + l] = 1;
    for (int k = 0; k < P.nfix + P.niter; k++)
      if (lin_dep(P.ops[k].lin)) dep[P.ops[k].dst] = 1;
  }
  // per shared-array access with one granule per instance: bin updates combine
  bool combinable(int a) const {
    const DAcc& A = P.acc[a];
    return !A.dead && A.shared && A.G == 1 && ((P.emask >> a) & 1u);
  }
  bool lin_dep(const DLin& L) const {
    for (int t = 0; t < L.n; t++)
      if (dep[P.term[L.first + t].slot]) return true;
    return false;
  }
  bool guards_invariant(int a) const {
    const DAcc& A = P.acc[a];
    for (int g = 0; g < A.ng; g++)
      if (lin_dep(P.guard[A.gfirst + g])) return false;
    return true;
  }
  // keys dropped, index always in bounds, guards loop-invariant: only counted
  bool count_only(int a) const {
    const DAcc& A = P.acc[a];
    return !((P.emask >> a) & 1u) && A.bounds_free && guards_invariant(a);
  }
  // guards, index and intervals read no loop-dependent slot
  bool invariant(int a) const {
    const DAcc& A = P.acc[a];
    if (count_only(a)) return true;
    return !lin_dep(A.idx) && !lin_dep(A.iv) && !(P.WVB && lin_dep(A.wv)) && guards_invariant(a);
  }
  // with one loop, a guard that reads the loop counter and nothing else
  // (c0 + c * k >= 0) bounds k to an interval known per unit
  bool loop_guard(const DLin& L) const { return nl == 1 && L.n == 1 && P.term[L.first].slot == 6; }
  // index and intervals ignore the loop, every loop-dependent guard is a loop guard
  bool ranged(int a) const {
    const DAcc& A = P.acc[a];
    if (A.dead || invariant(a) || lin_dep(A.idx) || lin_dep(A.iv) || (P.WVB && lin_dep(A.wv))) return false;
    for (int g = 0; g < A.ng; g++) {
      const DLin& L = P.guard[A.gfirst + g];
      if (lin_dep(L) && !loop_guard(L)) return false;
    }
    return true;
  }
};

}  // namespace

std::string jit_source(const DProg& P, bool split) {
  const int nl = P.nloop;
  std::string src;
  src += "#include \"expand_body.cuh\"\n";
  src += "namespace hgrd { namespace dev {\n";
  src += std::string("typedef ") + (P.wide ? "int64_t" : "int32_t") + " T;\n";
  src += "template <typename U> __device__ __forceinline__ U modq(U v, const Magic& g, U d) { return v - divq<U>(v, g) * d; }\n";
  // c0 + c * k >= 0 (c != 0) narrows [lo, hi]: k >= ceil(-c0 / c) for c > 0, k <= floor(c0 / -c) for c < 0
  src += "__device__ __forceinline__ int64_t fdiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }\n";
  // (unit coefficients, the usual case, skip the 64-bit division: it runs per unit)
  src += "__device__ __forceinline__ void loop_guard_range(int64_t c0, int64_t c, int64_t& lo, int64_t& hi) {\n"
         "  if (c == 1) lo = max(lo, -c0);\n"
         "  else if (c == -1) hi = min(hi, c0);\n"
         "  else if (c > 0) lo = max(lo, -fdiv(c0, c));\n"
         "  else hi = min(hi, fdiv(c0, -c));\n}\n";
  src += "struct GenX {\n  const DProg* __restrict__ P;\n";
  // the accesses whose keys are written, as the source was generated for
  src += "  __device__ __forceinline__ uint32_t emask_of(const DProg*) const { return " + S(P.emask) + "u; }\n";
  src += "  template <int SEL, class Step>\n";
  src += "  __device__ __forceinline__ uint64_t unit(int lane, int64_t u, uint32_t only, Step&& step) {\n";
  src += "    return walk<SEL, false, false>(lane, u, only, step, [](int, uint32_t, uint32_t, int) {});\n  }\n";
  src += "  template <int SEL, class Step>\n";
  src += "  __device__ __forceinline__ uint64_t unit_once(int lane, int64_t u, uint32_t only, Step&& step) {\n";
  src += "    return walk<SEL, false, true>(lane, u, only, step, [](int, uint32_t, uint32_t, int) {});\n  }\n";
  src += "  template <int SEL, class Step, class Flush>\n";
  src += "  __device__ __forceinline__ uint64_t unit_combine(int lane, int64_t u, uint32_t only, Step&& step, "
         "Flush&& flush) {\n";
  src += "    return walk<SEL, true, true>(lane, u, only, step, flush);\n  }\n";
  src += "  template <int SEL, bool COMBINE, bool ONCE, class Step, class Flush>\n";
  src += "  __device__ __forceinline__ uint64_t walk(int lane, int64_t u, uint32_t only, Step&& step, Flush&& flush) {\n";
  // unit -> (block, warp, chunk) and the thread / block coordinates: in
  // 32-bit unsigned arithmetic when every unit and block id fits (64-bit
  // division is a long software sequence), skipping divisions by 1
  const bool u32 = (uint64_t)P.nunits < (1ull << 31) && (uint64_t)P.nblk < (1ull << 31);
  if (u32) {
    src += "    const uint32_t uu = (uint32_t)u, nch = (uint32_t)P->nchunk, wpb = (uint32_t)P->wpb;\n";
    src += "    const uint32_t bw = nch == 1u ? uu : magic_udiv31(uu, P->dv[0]);\n";
    src += "    const int64_t it0 = (int64_t)(uu - bw * nch) * P->itc;\n";
    src += "    const uint32_t b32 = magic_udiv31(bw, P->dv[1]);\n";
    src += "    const int64_t b = (int64_t)b32;\n";
    src += "    const int lt = (int)(bw - b32 * wpb) * 32 + lane;\n";
    src += "    const uint32_t gx = (uint32_t)P->grid[0], gy = (uint32_t)P->grid[1];\n";
    src += "    const uint32_t bq = magic_udiv31(b32, P->dv[2]), bq2 = magic_udiv31(bq, P->dv[3]);\n";
    src += "    const T s3 = (T)(b32 - bq * gx), s4 = (T)(bq - bq2 * gy), s5 = (T)bq2;\n";
  } else {
    src += "    const int64_t bw = u / P->nchunk;\n";
    src += "    const int64_t it0 = (u - bw * P->nchunk) * P->itc;\n";
    src += "    const int64_t b = bw / P->wpb;\n";
    src += "    const int lt = (int)(bw - b * P->wpb) * 32 + lane;\n";
    src += "    const int64_t gdx = P->grid[0], gdy = P->grid[1];\n";
    src += "    const T s3 = (T)(b % gdx), s4 = (T)((b / gdx) % gdy), s5 = (T)(b / (gdx * gdy));\n";
  }
  src += "    const int64_t it1 = min(P->nit, it0 + P->itc);\n";
  src += "    const bool act = lt < P->nthr;\n";
  src += "    const uint32_t bdx = (uint32_t)P->block[0], bdy = (uint32_t)P->block[1], ult = (uint32_t)lt;\n";
  src += "    const uint32_t tq = magic_udiv31(ult, P->dv[4]), tq2 = magic_udiv31(tq, P->dv[5]);\n";
  src += "    const T s0 = (T)(ult - tq * bdx), s1 = (T)(tq - tq2 * bdy), s2 = (T)tq2;\n";
  // loop counters: slots 6.. for the live loops, zero for the others
  for (int l = nl; l < MAXLOOP; l++) src += "    const T s" + S(6 + l) + " = 0; (void)s" + S(6 + l) + ";\n";
  src += "    (void)s0; (void)s1; (void)s2; (void)s3; (void)s4; (void)s5;\n";
  // fixed ops: the loop slots are zero while they run; they never read them
  for (int l = 0; l < nl; l++) src += "    T s" + S(6 + l) + " = 0;\n";
  for (int k = 0; k < P.nfix; k++) src += op_code(P, k, true).substr(2);
  src += "    int32_t ic[4] = {0, 0, 0, 0};\n";
  src += "    if (it0 > 0) {\n      int64_t r = it0;\n";
  for (int l = nl - 1; l >= 0; l--)
    src += "      ic[" + S(l) + "] = (int32_t)(r % P->ub[" + S(l) + "]); r /= P->ub[" + S(l) + "];\n";
  src += "    }\n    uint64_t oob = 0;\n";
  const Analysis An(P);
  auto combinable = [&](int a) { return An.combinable(a); };
  auto lin_dep = [&](const DLin& L) { return An.lin_dep(L); };
  auto count_only = [&](int a) { return An.count_only(a); };
  auto invariant = [&](int a) { return An.invariant(a); };
  auto loop_guard = [&](const DLin& L) { return An.loop_guard(L); };
  auto ranged = [&](int a) { return An.ranged(a); };
  // [lo, hi] of the loop counter admitted by access a's loop guards
  auto range_code = [&](int a, const std::string& ind) {
    const DAcc& A = P.acc[a];
    std::string c = ind + "int64_t lo" + S(a) + " = 0, hi" + S(a) + " = (int64_t)P->ub[0] - 1;\n";
    for (int g = 0; g < A.ng; g++) {
      const DLin& L = P.guard[A.gfirst + g];
      if (!loop_guard(L)) continue;
      const std::string gg = "P->guard[" + S(A.gfirst + g) + "]";
      c += ind + "loop_guard_range(" + gg + ".c0, P->term[" + S(L.first) + "].coef, lo" + S(a) + ", hi" + S(a) + ");\n";
    }
    return c;
  };
  // one access: per loop vector (once = false), or once per unit standing for
  // the unit's nrep loop vectors (once = true, count pass only)
  auto access_code = [&](int a, bool once, const std::string& rep = "nrep", const std::string& icv = "ic") {
    const DAcc& A = P.acc[a];
    const std::string at = "P->acc[" + S(a) + "]";
    const std::string ind = once ? "        " : "      ";
    // in the selected set at compile time (SEL_KEPT: keys written; SEL_KEPT_GLOBAL: and a global array)
    const bool kept = (P.emask >> a) & 1u;
    const std::string in_sel = "(SEL == SEL_ALL || (SEL == SEL_KEPT && " + S(kept) + ") || (SEL == SEL_KEPT_GLOBAL && " +
                               S(kept && !A.shared) + "))";
    std::string c;
    c += ind + "if (" + in_sel + " && (only & " + S(1ll << a) + "u)) {  // access " + S(a) +
         (once ? (rep == "nrep" ? ", loop-invariant\n" : ", over its loop guards' range\n") : "\n");
    c += ind + "  bool live = act;\n";
    for (int g = 0; g < A.ng; g++) {
      // taken once over a range: the loop guards hold on the whole range
      if (once && rep != "nrep" && loop_guard(P.guard[A.gfirst + g])) continue;
      c += ind + "  live = live && " + lin(P, "P->guard[" + S(A.gfirst + g) + "]", P.guard[A.gfirst + g]) + " >= 0;\n";
    }
    // a count-only access taken once per unit never reads its index or
    // interval: in bounds everywhere, its live instances are its keys
    const bool no_idx = once && count_only(a);
    c += ind + "  const T idx = " + (no_idx ? std::string("0") : lin(P, at + ".idx", A.idx)) + ";\n";
    if (A.bounds_free)
      c += ind + "  const bool inb = live;\n";
    else
      c += ind + "  const bool inb = live && idx >= 0 && (int64_t)idx <= " + at + ".maxidx;\n";
    c += ind + "  oob += (live && !inb) ? " + std::string(once ? rep : "1") + " : 0;\n";
    // with warp-barrier intervals the key's interval field carries both ids
    const std::string iv = no_idx   ? std::string("(int64_t)0")
                           : P.WVB ? "pack_wv(P, (int64_t)" + lin(P, at + ".iv", A.iv) + ", (int64_t)" +
                                         lin(P, at + ".wv", A.wv) + ")"
                                   : "(int64_t)" + lin(P, at + ".iv", A.iv);
    bool closing = false;
    if (combinable(a) && once) {
      c += ind + "  if constexpr (COMBINE) {\n";
      c += ind + "    if (inb) flush(" + S(a) + ", (uint32_t)(((uint64_t)" + at + ".sgbase + (uint64_t)idx) * P->niv + " +
           "(uint64_t)(" + iv + " - P->ivmin)), " + rep + ", lt);\n";
      c += ind + "  } else {\n";
      closing = true;
    } else if (combinable(a)) {
      c += ind + "  if constexpr (COMBINE) {\n";
      c += ind + "    if (inb) {\n";
      c += ind + "      const uint32_t bin = (uint32_t)(((uint64_t)" + at + ".sgbase + (uint64_t)idx) * P->niv + " +
           "(uint64_t)(" + iv + " - P->ivmin));\n";
      c += ind + "      if (bin != pb" + S(a) + ") {\n";
      c += ind + "        if (pc" + S(a) + ") flush(" + S(a) + ", pb" + S(a) + ", pc" + S(a) + ", lt);\n";
      c += ind + "        pb" + S(a) + " = bin;\n" + ind + "        pc" + S(a) + " = 0;\n" + ind + "      }\n";
      c += ind + "      ++pc" + S(a) + ";\n" + ind + "    }\n";
      c += ind + "  } else {\n";
      closing = true;
    }
    if (no_idx && !closing) {
      // a count-only access taken once: its live instances are counted by
      // the lanes that hold them, no ballot
      c += ind + "  if (inb) {\n";
      c += ind + "    DAcc A = " + at + ";\n";
      c += ind + "    A.G = " + S(A.G) + "; A.shared = " + S(A.shared) + "; A.arr = " + S(A.arr) + ";\n";
      c += ind + "    step(" + S(a) + ", A, true, 0u, (int64_t)0, (int64_t)0, b, lt, " + icv + ", " + rep + ");\n";
      c += ind + "  }\n";
      c += ind + "}\n";
      return c;
    }
    c += ind + "  const unsigned bal = __ballot_sync(0xffffffffu, inb);\n";
    c += ind + "  if (bal) {\n";
    c += ind + "    int64_t iv = 0;\n";
    c += ind + "    if (inb) iv = " + iv + ";\n";
    // the access's structural fields as literals, so the step's granule loop
    // and its shared / global branch fold away
    c += ind + "    DAcc A = " + at + ";\n";
    c += ind + "    A.G = " + S(A.G) + "; A.shared = " + S(A.shared) + "; A.arr = " + S(A.arr) + ";\n";
    c += ind + "    step(" + S(a) + ", A, inb, bal, (int64_t)idx, iv, b, lt, " + icv + ", " + (once ? rep : "1u") +
         ");\n";
    c += ind + "  }\n";
    if (closing) c += ind + "  }\n";
    c += ind + "}\n";
    return c;
  };
  for (int a = 0; a < P.nacc; a++)
    if (combinable(a)) src += "    uint32_t pb" + S(a) + " = 0xffffffffu, pc" + S(a) + " = 0;\n";
  // the count passes take loop-invariant accesses once per unit
  {
    std::string once;
    for (int a = 0; a < P.nacc; a++)
      if (!P.acc[a].dead && invariant(a)) once += access_code(a, true);
    std::string ranges;
    for (int a = 0; a < P.nacc; a++) {
      if (!ranged(a)) continue;
      // the unit's loop counters [it0, it1) inside the guards' range: one
      // instance standing for all of them, recorded at the first
      ranges += range_code(a, "      ");
      ranges += "      {\n        const int64_t f" + S(a) + " = max(lo" + S(a) + ", it0), l" + S(a) + " = min(hi" + S(a) +
                ", it1 - 1);\n";
      ranges += "        const uint32_t m" + S(a) + " = l" + S(a) + " >= f" + S(a) + " ? (uint32_t)(l" + S(a) + " - f" +
                S(a) + " + 1) : 0u;\n";
      ranges += "        if (m" + S(a) + ") {\n          int32_t icr[4] = {(int32_t)f" + S(a) + ", 0, 0, 0};\n";
      std::string body = access_code(a, true, "m" + S(a), "icr");
      std::string ind2;
      for (size_t pos = 0; pos < body.size();) {  // two more spaces of indentation
        size_t e = body.find('\n', pos);
        ranges += "  " + body.substr(pos, e - pos + 1);
        pos = e + 1;
      }
      ranges += "        }\n      }\n";
    }
    if (!once.empty() || !ranges.empty()) {
      src += "    if constexpr (ONCE) {\n      const uint32_t nrep = (uint32_t)(it1 - it0);\n";
      if (!once.empty()) src += "      if (nrep) {\n" + once + "      }\n";
      src += ranges + "    }\n";
    }
  }
  // the loop visits only loop counters where some access its body evaluates
  // can be live: with one loop, the union of the ranged accesses' ranges
  // (any other access evaluated there spans the whole loop)
  std::string it_lo = "it0", it_hi = "it1";
  {
    bool any_ranged = false;
    for (int a = 0; a < P.nacc; a++) any_ranged |= ranged(a);
    if (any_ranged) {
      src += "    int64_t vlo = 0x7fffffffffffffffll, vhi = -1;  // loop counters the body may need\n";
      for (int a = 0; a < P.nacc; a++) {
        const DAcc& A = P.acc[a];
        if (A.dead) continue;
        const bool kept = (P.emask >> a) & 1u;
        const std::string sel = "(SEL == SEL_ALL || (SEL == SEL_KEPT && " + S(kept) + ") || (SEL == SEL_KEPT_GLOBAL && " +
                                S(kept && !A.shared) + ")) && (only & " + S(1ll << a) + "u)";
        // in a ONCE walk the loop skips invariant and ranged accesses
        const std::string in_loop = (invariant(a) || ranged(a)) ? "!ONCE && " + sel : sel;
        if (ranged(a)) {
          src += "    if (" + in_loop + ") {\n" + range_code(a, "      ");
          src += "      vlo = min(vlo, lo" + S(a) + ");\n      vhi = max(vhi, hi" + S(a) + ");\n    }\n";
        } else {
          src += "    if (" + in_loop + ") { vlo = 0; vhi = (int64_t)P->ub[0] - 1; }\n";
        }
      }
      src += "    const int64_t iv0 = max(it0, vlo), iv1 = min(it1, vhi + 1);\n";
      it_lo = "iv0";
      it_hi = "iv1";
    }
  }
  src += "    for (int64_t it = " + it_lo + "; it < " + it_hi + "; ++it) {\n";
  if (it_lo != "it0") src += "      ic[0] = (int32_t)it;\n      s6 = (T)it;\n";
  if (nl > 0 && it_lo == "it0") {
    src += "      if (it > it0) {\n";
    std::string close;
    for (int l = nl - 1; l >= 0; l--) {
      src += std::string(8 + 2 * (nl - 1 - l), ' ') + "if (++ic[" + S(l) + "] >= P->ub[" + S(l) + "]) {\n";
      src += std::string(10 + 2 * (nl - 1 - l), ' ') + "ic[" + S(l) + "] = 0;\n";
      close = std::string(8 + 2 * (nl - 1 - l), ' ') + "}\n" + close;
    }
    src += close + "      }\n";
    for (int l = 0; l < nl; l++) src += "      s" + S(6 + l) + " = (T)ic[" + S(l) + "];\n";
  }
  for (int k = P.nfix; k < P.nfix + P.niter; k++) src += op_code(P, k, true);
  for (int a = 0; a < P.nacc; a++) {
    if (P.acc[a].dead) continue;
    if (invariant(a) || ranged(a)) {
      src += "      if constexpr (!ONCE) {\n" + access_code(a, false) + "      }\n";
    } else {
      src += access_code(a, false);
    }
  }
  src += "    }\n";
  for (int a = 0; a < P.nacc; a++)
    if (combinable(a))
      src += "    if constexpr (COMBINE) { if (pc" + S(a) + ") flush(" + S(a) + ", pb" + S(a) + ", pc" + S(a) + ", lt); }\n";
  src += "    return oob;\n  }\n};\n}}  // namespace hgrd::dev\n";
  src += "using namespace hgrd;\nusing namespace hgrd::dev;\n";
  const char* sig =
      "(const __grid_constant__ DProg Pp, uint64_t* unit_cnt, const uint64_t* unit_off, uint64_t* keys_g, "
      "uint64_t* keys_s, uint64_t* hist, int npass, uint64_t* counters, uint64_t* stbl, uint64_t* sbase, "
      "uint32_t only, const uint64_t* uniq, PairRec* pairs, uint64_t pair_cap, const uint32_t* ctab, uint64_t* cbuf, "
      "uint64_t ccap) {\n"
      "  extern __shared__ __align__(16) unsigned char smem[];\n  GenX ex{&Pp};\n";
  // the pair search (2), and the count and write kernels of one pipeline:
  // block-local (3, 4) or plain (0, 1)
  src += "extern \"C\" __global__ void __launch_bounds__(EXP_THREADS) hgrd_jit_expand2" + std::string(sig);
  src += "  expand_units_body<T, 2>(&Pp, ex, reinterpret_cast<uint32_t*>(smem), unit_cnt, unit_off, keys_g, hist, "
         "npass, counters, uniq, pairs, pair_cap, only);\n}\n";
  // the write kernels (1, 4) are register hungry (key stores of every kept
  // access in flight); three CTAs per SM keep them at 80 registers
  if (!split) {
    for (int m : {0, 1}) {
      src += "extern \"C\" __global__ void __launch_bounds__(EXP_THREADS" + std::string(m == 1 ? ", 3" : "") +
             ") hgrd_jit_expand" + S(m) + sig;
      src += "  expand_units_body<T, " + S(m) +
             ">(&Pp, ex, reinterpret_cast<uint32_t*>(smem), unit_cnt, unit_off, keys_g, hist, npass, counters, "
             "nullptr, nullptr, 0, only" + std::string(m == 1 ? ", ctab, cbuf, ccap" : "") + ");\n}\n";
    }
  }
  for (int m : {3, 4}) {
    if (!split) break;
    src += "extern \"C\" __global__ void __launch_bounds__(EXP_THREADS" + std::string(m == 4 ? ", 3" : "") +
           ") hgrd_jit_expand" + S(m) + sig;
    src += "  expand_block_body<T, " + S(m) +
           ">(&Pp, ex, reinterpret_cast<uint32_t*>(smem), unit_cnt, unit_off, keys_g, keys_s, hist, counters, "
           "stbl, sbase, only);\n}\n";
  }
  return src;
}

namespace {

struct JitModule {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t k[5] = {};
  bool ok = false;
  std::string log;
};

std::mutex g_jit_mu;
std::map<std::string, std::unique_ptr<JitModule>> g_jit_cache;

JitModule* compile(const std::string& src, double* ms) {
  auto t0 = std::chrono::steady_clock::now();
  auto mod = std::make_unique<JitModule>();
  std::vector<const char*> names, texts;
  names.push_back("cstdint");
  texts.push_back(kStdInt);
  names.push_back("stdint.h");
  texts.push_back(kStdInt);
  names.push_back("cstddef");
  texts.push_back(kStdDef);
  names.push_back("stddef.h");
  texts.push_back(kStdDef);
  for (size_t i = 0; i < sizeof(kJitHeaderNames) / sizeof(kJitHeaderNames[0]); i++) {
    names.push_back(kJitHeaderNames[i]);
    texts.push_back(kJitHeaders[i]);
  }
  nvrtcProgram prog = nullptr;
  nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "hgrd_expand_jit.cu", (int)names.size(), texts.data(),
                                     names.data());
  if (r != NVRTC_SUCCESS) {
    mod->log = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r);
  } else {
    const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-lineinfo", "-DNDEBUG"};
    r = nvrtcCompileProgram(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    std::string log(ls, '\0');
    if (ls) nvrtcGetProgramLog(prog, &log[0]);
    if (r != NVRTC_SUCCESS) {
      mod->log = "nvrtcCompileProgram: " + std::string(nvrtcGetErrorString(r)) + "\n" + log;
    } else {
      size_t n = 0;
      nvrtcGetCUBINSize(prog, &n);
      std::vector<char> cubin(n);
      nvrtcGetCUBIN(prog, cubin.data());
      note_created();
      cudaError_t e = cudaLibraryLoadData(&mod->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
      if (e != cudaSuccess) {
        mod->log = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
      } else {
        static const char* kn[5] = {"hgrd_jit_expand0", "hgrd_jit_expand1", "hgrd_jit_expand2", "hgrd_jit_expand3",
                                    "hgrd_jit_expand4"};
        const bool split = src.find("hgrd_jit_expand3") != std::string::npos;
        mod->ok = true;
        for (int m = 0; m < 5 && mod->ok; m++) {
          if (m != 2 && split != (m >= 3)) continue;
          e = cudaLibraryGetKernel(&mod->k[m], mod->lib, kn[m]);
          if (e != cudaSuccess) {
            mod->ok = false;
            mod->log = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
          }
        }
      }
    }
    nvrtcDestroyProgram(&prog);
  }
  *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  JitModule* raw = mod.get();
  g_jit_cache[src] = std::move(mod);
  return raw;
}

}  // namespace

int jit_prepare(const Bound& B, bool split, double* ms) {
  if (ms) *ms = 0;
  std::lock_guard<std::mutex> lk(g_jit_mu);
  const void*& slot = B.jit[split ? 1 : 0];
  if (slot) return ((const JitModule*)slot)->ok ? HGRD_OK : fail(HGRD_EUNSUPPORTED, ((const JitModule*)slot)->log);
  const std::string src = jit_source(B.prog, split);
  auto it = g_jit_cache.find(src);
  JitModule* m = nullptr;
  if (it != g_jit_cache.end()) {
    m = it->second.get();
  } else {
    double t = 0;
    m = compile(src, &t);
    if (ms) *ms = t;
  }
  slot = m;
  return m->ok ? HGRD_OK : fail(HGRD_EUNSUPPORTED, "specialised expansion unavailable: " + m->log);
}

uint64_t jit_eval_ops(const DProg& P) {
  // the integer operations the specialised count pass evaluates: a term is
  // one multiply-add, a guard or bound test one compare, a division by a
  // constant three, a remainder two more; per thread the unit's fixed ops and
  // every access taken once (loop-invariant, count-only, ranged), per thread
  // and loop vector the loop ops and the other accesses
  const Analysis An(P);
  auto op_cost = [&](const DOp& op) {
    return (uint64_t)op.lin.n + (op.kind == OP_DIV ? 3u : op.kind == OP_MOD ? 5u : 0u);
  };
  // (a count-only access: its guards alone)
  auto acc_cost = [&](int a) {
    const DAcc& A = P.acc[a];
    uint64_t c = An.count_only(a) ? 0 : (uint64_t)A.idx.n + 2 + (uint64_t)A.iv.n + (P.WVB ? (uint64_t)A.wv.n + 2 : 0);
    for (int g = 0; g < A.ng; g++) c += (uint64_t)P.guard[A.gfirst + g].n + 1;
    return c;
  };
  // an op counts when an evaluated expression reads it (directly or through
  // later ops); ops only count-only accesses' indexes read are never computed
  std::vector<char> need(MAXSLOT, 0);
  auto mark = [&](const DLin& L) {
    for (int t = 0; t < L.n; t++) need[P.term[L.first + t].slot] = 1;
  };
  for (int a = 0; a < P.nacc; a++) {
    const DAcc& A = P.acc[a];
    if (A.dead) continue;
    if (!An.count_only(a)) {
      mark(A.idx);
      mark(A.iv);
      if (P.WVB) mark(A.wv);
    }
    for (int g = 0; g < A.ng; g++) mark(P.guard[A.gfirst + g]);
  }
  for (int k = P.nfix + P.niter - 1; k >= 0; k--)
    if (need[P.ops[k].dst]) mark(P.ops[k].lin);
  auto op_need = [&](int k) { return need[P.ops[k].dst] ? op_cost(P.ops[k]) : (uint64_t)0; };
  uint64_t once = 0, per_it = 0;
  bool loop_body = false;
  for (int k = 0; k < P.nfix; k++) once += op_need(k);
  for (int a = 0; a < P.nacc; a++) {
    const DAcc& A = P.acc[a];
    if (A.dead) continue;
    if (An.invariant(a) || An.ranged(a)) {
      once += acc_cost(a);
    } else {
      per_it += acc_cost(a);
      loop_body = true;
    }
  }
  if (loop_body)
    for (int k = P.nfix; k < P.nfix + P.niter; k++) per_it += op_need(k);
  return (uint64_t)P.nblk * (uint64_t)P.nthr * (once + (uint64_t)P.nit * per_it);
}

bool jit_ready(const Bound& B, bool split) {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  const void* m = B.jit[split ? 1 : 0];
  return m && ((const JitModule*)m)->ok;
}

cudaError_t launch_jit_expand(const Launch& L, const Bound& B, int mode, const DProg& h_prog, uint64_t* unit_cnt,
                              const uint64_t* unit_off, uint64_t* keys_g, uint64_t* keys_s, uint64_t* hist, int npass,
                              uint64_t* counters, uint64_t* stbl, uint64_t* sbase, uint32_t only, bool split,
                              const uint64_t* uniq, PairRec* pairs, uint64_t pair_cap, const uint32_t* ctab,
                              uint64_t* cbuf, uint64_t ccap) {
  const JitModule* m = (const JitModule*)B.jit[split ? 1 : 0];
  const void* fn = (const void*)m->k[mode];
  size_t smem = 0;
  int64_t need = 0;
  if (mode <= 2) {
    smem = mode == 0 ? (size_t)npass * 256 * 4 : 0;
    need = (h_prog.nunits + EXP_THREADS / 32 - 1) / (EXP_THREADS / 32);
  } else {
    smem = block_body_words(mode, (uint64_t)h_prog.nsbins) * 4;
    need = h_prog.nblk;
  }
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)resident_ctas(fn, EXP_THREADS, smem) * L.nsm;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  void* args[] = {(void*)&h_prog, (void*)&unit_cnt, (void*)&unit_off, (void*)&keys_g, (void*)&keys_s,
                  (void*)&hist,   (void*)&npass,    (void*)&counters, (void*)&stbl,   (void*)&sbase,
                  (void*)&only,   (void*)&uniq,     (void*)&pairs,    (void*)&pair_cap,
                  (void*)&ctab,   (void*)&cbuf,     (void*)&ccap};
  (*L.launches)++;
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(EXP_THREADS), args, smem, L.s);
}

}  // namespace hgrd

extern "C" int hgrd_jit_compile(const hgrd_desc* d, const hgrd_check_opts* o, double* compile_ms) {
  if (!d) return hgrd::fail(HGRD_EINVAL, "null descriptor");
  if (!d->bound) return hgrd::fail(HGRD_EINVAL, "descriptor is not bound (call hgrd_bind_host_params)");
  const bool split = d->bound->prog.smode && !(o && (o->flags & HGRD_NO_SPLIT));
  return hgrd::jit_prepare(*d->bound, split, compile_ms);
}

extern "C" int hgrd_jit_source(const hgrd_desc* d, const hgrd_check_opts* o, char* out, size_t cap,
                               size_t* len) {
  if (!d) return hgrd::fail(HGRD_EINVAL, "null descriptor");
  if (!d->bound) return hgrd::fail(HGRD_EINVAL, "descriptor is not bound (call hgrd_bind_host_params)");
  const bool split = d->bound->prog.smode && !(o && (o->flags & HGRD_NO_SPLIT));
  const std::string s = hgrd::jit_source(d->bound->prog, split);
  if (len) *len = s.size();
  if (out && cap) {
    const size_t n = s.size() < cap - 1 ? s.size() : cap - 1;
    memcpy(out, s.data(), n);
    out[n] = 0;
  }
  return HGRD_OK;
}
