// CPU oracle for the host-guided GPU data-race check.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// definition that the GPU path is compared against.  It shares no code with
// the GPU library: it has its own descriptor parser and its own evaluator,
// and nothing outside tests/, the smoke check and the bench's CPU-baseline
// leg may load it.
//
// What it computes (the paper's race definition, applied to every concrete
// instance of a kernel under one host-supplied binding):
//   * Sec. 2 ("Data races on GPUs"): two accesses from different threads that
//     alias, at least one a write, not ordered by synchronisation, form a race;
//     shared memory is per threadblock, global memory is grid-wide; the race
//     type is inter-threadblock / intra-threadblock (different warps) /
//     intra-warp (same warp, warp = 32 consecutive linear thread ids).
//   * Sec. 6.1 ("Avoiding race checks"): a block barrier between two accesses
//     leaves only the inter-threadblock check (barrier-interval ids: same
//     block and different interval = ordered); a warp barrier (syncwarp)
//     between them rules out the intra-warp race only (warp-interval ids:
//     same warp and different warp interval = ordered; Sec. 5.2, "Intra-warp
//     races"); two loads or two atomics are trivially race free.
//   * Appendix A ("Extending with scoped operations"): two device-scope
//     atomics never race; two atomics of at least block scope never race
//     inside a block; a block-scope atomic does not order threads of another
//     block (race of insufficient scope).
//   * Sec. 6.5 ("Support acquire-release synchronization") and Table 2's
//     highlighted addr(syn(Ai)) != addr(syn(Aj)) constraint: two instances
//     whose accesses are both guarded by acquire-release (a lock, or a
//     producer's release and a consumer's acquire) at the same address do not
//     race; guarded at different addresses, or only one of them guarded, they
//     still may.  Appendix A ("Scoped acquire-release"): an inter-threadblock
//     pair needs device scope on both, an intra-threadblock or intra-warp pair
//     block scope or wider (always the case); the scope of a guard is the
//     narrower of its parts.
//   * Table 1 / Table 2: addr, tb, id, wp constraints per race type.
//   * Sec. 4 / 5.1, host classes (1)-(5): the binding supplies every parameter
//     and launch dimension; `assert` lines must hold for it.
//
// The enumeration: every (block, thread, loop vector, access) tuple in linear
// order; live instances (all guards true) that lie inside their array are
// bucketed in an ordered map keyed by (space, array, block-for-shared,
// granule); each bucket is checked pair by pair.  Nothing is blocked, fused
// or reordered beyond that.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

namespace {

enum { OK = 0, TRUNC = 1, EINVAL_ = -1, EPARSE = -2, EBIND = -3, EHOST = -4, EOVF = -5 };

struct Fail {
  int code;
  std::string msg;
};

// ---------------------------------------------------------------- AST
enum NodeKind { N_NUM, N_NAME, N_BIN, N_NEG };
enum NameClass { C_TID, C_BID, C_BDIM, C_GDIM, C_LOOP, C_PARAM };

struct Node {
  NodeKind k;
  int64_t num = 0;
  NameClass cls = C_PARAM;
  int slot = 0;  // component or loop index or param index
  char op = 0;
  std::shared_ptr<Node> a, b;
};
using P = std::shared_ptr<Node>;

struct Env {
  int64_t tid[3], bid[3], bdim[3], gdim[3];
  int64_t loop[4];
  const int64_t* params;
};

int64_t add_(int64_t x, int64_t y) {
  int64_t r;
  if (__builtin_add_overflow(x, y, &r)) throw Fail{EOVF, "integer overflow while evaluating an expression"};
  return r;
}
int64_t sub_(int64_t x, int64_t y) {
  int64_t r;
  if (__builtin_sub_overflow(x, y, &r)) throw Fail{EOVF, "integer overflow while evaluating an expression"};
  return r;
}
int64_t mul_(int64_t x, int64_t y) {
  int64_t r;
  if (__builtin_mul_overflow(x, y, &r)) throw Fail{EOVF, "integer overflow while evaluating an expression"};
  return r;
}

int64_t eval(const Node* n, const Env& e) {
  switch (n->k) {
    case N_NUM: return n->num;
    case N_NAME:
      switch (n->cls) {
        case C_TID: return e.tid[n->slot];
        case C_BID: return e.bid[n->slot];
        case C_BDIM: return e.bdim[n->slot];
        case C_GDIM: return e.gdim[n->slot];
        case C_LOOP: return e.loop[n->slot];
        case C_PARAM: return e.params[n->slot];
      }
      return 0;
    case N_NEG:
      return sub_(0, eval(n->a.get(), e));
    case N_BIN: {
      int64_t x = eval(n->a.get(), e), y = eval(n->b.get(), e);
      switch (n->op) {
        case '+': return add_(x, y);
        case '-': return sub_(x, y);
        case '*': return mul_(x, y);
        case '/':
          if (y <= 0) throw Fail{EBIND, "divisor is not positive"};
          return x / y;  // C: truncation toward zero
        case '%':
          if (y <= 0) throw Fail{EBIND, "divisor is not positive"};
          return x % y;  // C: sign of the dividend
      }
    }
  }
  return 0;
}

// true when the value can differ between instances (thread, block or loop ids)
bool varies(const Node* n) {
  switch (n->k) {
    case N_NUM: return false;
    case N_NAME: return n->cls == C_TID || n->cls == C_BID || n->cls == C_LOOP;
    case N_NEG: return varies(n->a.get());
    case N_BIN: return varies(n->a.get()) || varies(n->b.get());
  }
  return false;
}
bool uses_thread(const Node* n) {
  switch (n->k) {
    case N_NUM: return false;
    case N_NAME: return n->cls == C_TID || n->cls == C_BID;
    case N_NEG: return uses_thread(n->a.get());
    case N_BIN: return uses_thread(n->a.get()) || uses_thread(n->b.get());
  }
  return false;
}
void collect_divisors(const Node* n, std::vector<const Node*>& out) {
  if (n->k == N_NEG) collect_divisors(n->a.get(), out);
  if (n->k == N_BIN) {
    collect_divisors(n->a.get(), out);
    collect_divisors(n->b.get(), out);
    if (n->op == '/' || n->op == '%') out.push_back(n->b.get());
  }
}

// ---------------------------------------------------------------- descriptor
struct Cond {
  P lhs, rhs;
  std::string op;
};
struct Array {
  std::string name;
  int space = 0;  // 0 global, 1 shared
  P bytes;
  int64_t granule = 0;
};
struct Access {
  int kind = 0;  // 0 R, 1 W, 2 A
  int array = 0;
  int64_t width = 0;
  int scope = 1;  // 0 block, 1 device
  P idx, iv, wv;  // iv: block-barrier interval; wv: warp-barrier interval
  std::vector<Cond> guards;
  int sync_array = -1;  // acquire-release guard (Sec. 6.5): array of its address, -1 none
  P sync;               // element of that array the guard acquires / releases
  int sync_scope = 1;   // 0 block, 1 device (the narrower of the guard's parts)
};
struct Desc {
  std::vector<std::string> params;
  std::vector<std::pair<std::string, P>> loops;
  std::vector<Array> arrays;
  std::vector<Access> acc;
  std::vector<Cond> asserts;
  std::map<std::string, P> lets;
};

struct Lexer {
  const std::string& s;
  size_t i = 0;
  explicit Lexer(const std::string& str) : s(str) {}
  void ws() {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\t')) i++;
  }
  bool done() {
    ws();
    return i >= s.size();
  }
  char peek() {
    ws();
    return i < s.size() ? s[i] : 0;
  }
};

struct Parser {
  Desc& d;
  explicit Parser(Desc& dd) : d(dd) {}

  [[noreturn]] void bad(const std::string& m) { throw Fail{EPARSE, m}; }

  P name_node(const std::string& id) {
    static const char* comp = "xyz";
    auto mk = [](NameClass c, int s) {
      auto n = std::make_shared<Node>();
      n->k = N_NAME;
      n->cls = c;
      n->slot = s;
      return n;
    };
    if (id.size() == 2 && (id[0] == 't' || id[0] == 'b') && strchr(comp, id[1]))
      return mk(id[0] == 't' ? C_TID : C_BID, (int)(strchr(comp, id[1]) - comp));
    if (id.size() == 3 && (id.rfind("bd", 0) == 0 || id.rfind("gd", 0) == 0) && strchr(comp, id[2]))
      return mk(id[0] == 'b' ? C_BDIM : C_GDIM, (int)(strchr(comp, id[2]) - comp));
    for (size_t k = 0; k < d.loops.size(); k++)
      if (d.loops[k].first == id) return mk(C_LOOP, (int)k);
    for (size_t k = 0; k < d.params.size(); k++)
      if (d.params[k] == id) return mk(C_PARAM, (int)k);
    auto it = d.lets.find(id);
    if (it != d.lets.end()) return it->second;
    bad("unknown name '" + id + "'");
  }

  P primary(Lexer& L) {
    char c = L.peek();
    if (c == '(') {
      L.i++;
      P e = expr(L);
      if (L.peek() != ')') bad("missing ')'");
      L.i++;
      return e;
    }
    if (c == '-') {
      L.i++;
      auto n = std::make_shared<Node>();
      n->k = N_NEG;
      n->a = primary(L);
      return n;
    }
    if (c >= '0' && c <= '9') {
      int64_t v = 0;
      while (L.i < L.s.size() && L.s[L.i] >= '0' && L.s[L.i] <= '9') {
        if (__builtin_mul_overflow(v, (int64_t)10, &v) || __builtin_add_overflow(v, (int64_t)(L.s[L.i] - '0'), &v))
          bad("integer literal too large");
        L.i++;
      }
      auto n = std::make_shared<Node>();
      n->k = N_NUM;
      n->num = v;
      return n;
    }
    if (isalpha((unsigned char)c) || c == '_') {
      size_t j = L.i;
      while (j < L.s.size() && (isalnum((unsigned char)L.s[j]) || L.s[j] == '_')) j++;
      std::string id = L.s.substr(L.i, j - L.i);
      L.i = j;
      return name_node(id);
    }
    bad(std::string("unexpected character '") + (c ? c : '?') + "'");
  }
  P term(Lexer& L) {
    P x = primary(L);
    for (;;) {
      char c = L.peek();
      if (c != '*' && c != '/' && c != '%') return x;
      L.i++;
      P y = primary(L);
      auto n = std::make_shared<Node>();
      n->k = N_BIN;
      n->op = c;
      n->a = x;
      n->b = y;
      if (c == '*' && varies(x.get()) && varies(y.get())) bad("product of two instance-dependent terms");
      if ((c == '/' || c == '%') && varies(y.get())) bad("divisor depends on thread, block or loop ids");
      x = n;
    }
  }
  P expr(Lexer& L) {
    P x = term(L);
    for (;;) {
      char c = L.peek();
      if (c != '+' && c != '-') return x;
      L.i++;
      P y = term(L);
      auto n = std::make_shared<Node>();
      n->k = N_BIN;
      n->op = c;
      n->a = x;
      n->b = y;
      x = n;
    }
  }
  P full_expr(const std::string& s) {
    Lexer L(s);
    P e = expr(L);
    if (!L.done()) bad("trailing text in expression '" + s + "'");
    return e;
  }
  Cond cond(const std::string& s, bool allow_ne) {
    static const char* ops[] = {"<=", ">=", "==", "!=", "<", ">"};
    for (const char* op : ops) {
      size_t p = s.find(op);
      if (p == std::string::npos) continue;
      std::string o(op);
      if (o == "!=" && !allow_ne) bad("'!=' is not allowed in a guard");
      Cond c;
      c.op = o;
      c.lhs = full_expr(s.substr(0, p));
      c.rhs = full_expr(s.substr(p + o.size()));
      return c;
    }
    bad("condition without comparison: '" + s + "'");
  }
};

std::string trim(const std::string& s) {
  size_t a = s.find_first_not_of(" \t\r"), b = s.find_last_not_of(" \t\r");
  return a == std::string::npos ? "" : s.substr(a, b - a + 1);
}
std::vector<std::string> split(const std::string& s, char c) {
  std::vector<std::string> out;
  size_t st = 0;
  for (;;) {
    size_t p = s.find(c, st);
    out.push_back(trim(s.substr(st, p == std::string::npos ? std::string::npos : p - st)));
    if (p == std::string::npos) break;
    st = p + 1;
  }
  return out;
}
std::vector<std::string> words(const std::string& s) {
  std::vector<std::string> out;
  size_t i = 0;
  while (i < s.size()) {
    while (i < s.size() && isspace((unsigned char)s[i])) i++;
    size_t j = i;
    while (j < s.size() && !isspace((unsigned char)s[j])) j++;
    if (j > i) out.push_back(s.substr(i, j - i));
    i = j;
  }
  return out;
}
bool is_ident(const std::string& s) {
  if (s.empty() || !(isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
  for (char c : s)
    if (!(isalnum((unsigned char)c) || c == '_')) return false;
  return true;
}

Desc parse(const std::string& text) {
  Desc d;
  Parser ps(d);
  std::vector<std::string> names = {"tx", "ty", "tz", "bx", "by", "bz", "bdx", "bdy", "bdz", "gdx", "gdy", "gdz"};
  auto fresh = [&](const std::string& n) {
    if (!is_ident(n)) ps.bad("bad name '" + n + "'");
    if (std::find(names.begin(), names.end(), n) != names.end()) ps.bad("name '" + n + "' declared twice");
    names.push_back(n);
  };
  bool have_kernel = false;
  for (const std::string& raw : split(text, '\n')) {
    std::string line = raw.substr(0, raw.find('#'));
    line = trim(line);
    if (line.empty()) continue;
    std::vector<std::string> w = words(line);
    const std::string& dir = w[0];
    std::string rest = trim(line.substr(dir.size()));
    if (dir == "kernel") {
      have_kernel = true;
    } else if (dir == "param") {
      for (size_t k = 1; k < w.size(); k++) {
        fresh(w[k]);
        d.params.push_back(w[k]);
      }
    } else if (dir == "loop") {
      if (w.size() < 3) ps.bad("loop needs a variable and a bound");
      if (d.loops.size() >= 4) ps.bad("at most 4 loops");
      fresh(w[1]);
      P bound = ps.full_expr(trim(rest.substr(w[1].size())));
      if (varies(bound.get())) ps.bad("loop bound must be uniform");
      d.loops.push_back({w[1], bound});
    } else if (dir == "array") {
      std::vector<std::string> f = split(rest, ';');
      std::vector<std::string> h = words(f[0]);
      if (h.size() < 3) ps.bad("array needs name, space and size");
      fresh(h[0]);
      Array a;
      a.name = h[0];
      if (h[1] == "global") a.space = 0;
      else if (h[1] == "shared") a.space = 1;
      else ps.bad("array space must be global or shared");
      size_t p = f[0].find(h[1]) + h[1].size();
      a.bytes = ps.full_expr(trim(f[0].substr(p)));
      if (varies(a.bytes.get())) ps.bad("array size must be uniform");
      for (size_t k = 1; k < f.size(); k++) {
        std::vector<std::string> kv = words(f[k]);
        if (kv.size() == 2 && kv[0] == "granule") a.granule = std::stoll(kv[1]);
        else ps.bad("unknown array field '" + f[k] + "'");
        if (a.granule <= 0) ps.bad("granule must be positive");
      }
      if (d.arrays.size() >= 32) ps.bad("at most 32 arrays");
      d.arrays.push_back(a);
    } else if (dir == "let") {
      size_t eq = rest.find('=');
      if (eq == std::string::npos) ps.bad("let needs '='");
      std::string n = trim(rest.substr(0, eq));
      fresh(n);
      d.lets[n] = ps.full_expr(trim(rest.substr(eq + 1)));
    } else if (dir == "assert") {
      Cond c = ps.cond(rest, true);
      if (varies(c.lhs.get()) || varies(c.rhs.get())) ps.bad("assert must be uniform");
      d.asserts.push_back(c);
    } else if (dir == "access") {
      std::vector<std::string> f = split(rest, ';');
      std::vector<std::string> h = words(f[0]);
      if (h.size() != 2) ps.bad("access needs kind and array");
      Access a;
      if (h[0] == "R") a.kind = 0;
      else if (h[0] == "W") a.kind = 1;
      else if (h[0] == "A") a.kind = 2;
      else ps.bad("access kind must be R, W or A");
      int found = -1;
      for (size_t k = 0; k < d.arrays.size(); k++)
        if (d.arrays[k].name == h[1]) found = (int)k;
      if (found < 0) ps.bad("unknown array '" + h[1] + "'");
      a.array = found;
      bool have_idx = false;
      for (size_t k = 1; k < f.size(); k++) {
        const std::string& fld = f[k];
        std::vector<std::string> fw = words(fld);
        if (fw.empty()) continue;
        std::string body = trim(fld.substr(fw[0].size()));
        if (fw[0] == "width") {
          a.width = std::stoll(body);
          if (a.width <= 0) ps.bad("width must be positive");
        } else if (fw[0] == "iv") {
          a.iv = ps.full_expr(body);
          if (uses_thread(a.iv.get())) ps.bad("interval must not depend on thread or block ids");
        } else if (fw[0] == "wv") {
          a.wv = ps.full_expr(body);
          if (uses_thread(a.wv.get())) ps.bad("warp interval must not depend on thread or block ids");
        } else if (fw[0] == "idx") {
          a.idx = ps.full_expr(body);
          have_idx = true;
        } else if (fw[0] == "if") {
          a.guards.push_back(ps.cond(body, false));
        } else if (fw[0] == "scope") {
          if (body == "block") a.scope = 0;
          else if (body == "device") a.scope = 1;
          else ps.bad("scope must be block or device");
        } else if (fw[0] == "sync") {
          // sync <array> <element>: the access is guarded by acquire-release at that address
          if (fw.size() < 3) ps.bad("sync needs an array and an element");
          int sa = -1;
          for (size_t k = 0; k < d.arrays.size(); k++)
            if (d.arrays[k].name == fw[1]) sa = (int)k;
          if (sa < 0) ps.bad("unknown sync array '" + fw[1] + "'");
          if (d.arrays[sa].space != 0) ps.bad("a sync array must be global");
          a.sync_array = sa;
          a.sync = ps.full_expr(trim(body.substr(body.find(fw[1]) + fw[1].size())));
        } else if (fw[0] == "syncscope") {
          if (body == "block") a.sync_scope = 0;
          else if (body == "device") a.sync_scope = 1;
          else ps.bad("syncscope must be block or device");
        } else if (fw[0] == "line") {
          // source line of the access: informational
        } else {
          ps.bad("unknown access field '" + fw[0] + "'");
        }
      }
      if (!have_idx || a.width == 0) ps.bad("access needs width and idx");
      if (!a.iv) {
        a.iv = std::make_shared<Node>();
        a.iv->k = N_NUM;
      }
      if (!a.wv) {
        a.wv = std::make_shared<Node>();
        a.wv->k = N_NUM;
      }
      if (d.acc.size() >= 32) ps.bad("at most 32 accesses");
      d.acc.push_back(a);
    } else {
      ps.bad("unknown directive '" + dir + "'");
    }
  }
  if (!have_kernel) ps.bad("missing 'kernel' line");
  // granule of each array: explicit, else the gcd of the widths used on it
  for (size_t k = 0; k < d.arrays.size(); k++) {
    int64_t g = 0;
    for (auto& a : d.acc)
      if (a.array == (int)k) g = std::gcd(g, a.width);
    if (d.arrays[k].granule == 0) d.arrays[k].granule = g ? g : 4;
    for (auto& a : d.acc)
      if (a.array == (int)k && a.width % d.arrays[k].granule) ps.bad("width is not a multiple of the granule");
  }
  return d;
}

bool holds(const Cond& c, const Env& e) {
  int64_t x = eval(c.lhs.get(), e), y = eval(c.rhs.get(), e);
  if (c.op == "<") return x < y;
  if (c.op == "<=") return x <= y;
  if (c.op == ">") return x > y;
  if (c.op == ">=") return x >= y;
  if (c.op == "==") return x == y;
  return x != y;
}

// ---------------------------------------------------------------- checking
struct Inst {
  int64_t blk, thr;
  int64_t it[4];
  int acc;
  int64_t iv, wv;
  int64_t sync;  // element of the access's acquire-release guard (when it has one)
};

// Kinds a pair of accesses may race with (bit0 inter-block, bit1 intra-block,
// bit2 intra-warp).  Sec. 6.1 trivially-race-free rule and Appendix A scopes.
int allowed_kinds(const Desc& d, int a, int b) {
  const Access &x = d.acc[a], &y = d.acc[b];
  if (x.array != y.array) return 0;
  if (x.kind == 0 && y.kind == 0) return 0;  // two loads
  int m = 7;
  if (x.kind == 2 && y.kind == 2) m = (x.scope == 0 || y.scope == 0) ? 1 : 0;
  if (d.arrays[x.array].space == 1) m &= ~1;  // shared memory: one copy per block
  return m;
}

// Race type of one pair of instances that touch the same location
// (Table 2): 0 when they cannot race.
int pair_kind(const Inst& x, const Inst& y) {
  if (x.blk == y.blk && x.thr == y.thr) return 0;  // same thread: program order
  if (x.blk != y.blk) return 1;                    // barriers never order blocks
  if (x.iv != y.iv) return 0;                      // separated by a block barrier
  if (x.thr / 32 != y.thr / 32) return 2;          // a warp barrier does not order warps
  return x.wv == y.wv ? 4 : 0;                     // same warp: a warp barrier orders them
}

// Race type of one pair of instances once acquire-release is taken into
// account (Sec. 6.5, Table 2, Appendix A): guards at one address order the
// pair if their scope covers its type.
int race_kind(const Desc& d, const Inst& x, const Inst& y) {
  const int k = pair_kind(x, y);
  if (!k) return 0;
  const Access &A = d.acc[x.acc], &B = d.acc[y.acc];
  if (A.sync_array < 0 || B.sync_array < 0) return k;       // syn() is NULL for one of them
  if (A.sync_array != B.sync_array || x.sync != y.sync) return k;  // the guard addresses differ
  const int scope = std::min(A.sync_scope, B.sync_scope);
  if (k == 1 && scope == 0) return k;  // inter-threadblock needs device scope
  return 0;
}

struct Key {
  int space, array;
  int64_t blk, granule;
  bool operator<(const Key& o) const {
    return std::tie(space, array, blk, granule) < std::tie(o.space, o.array, o.blk, o.granule);
  }
};

bool key_less(const Inst& a, const Inst& b) {
  return std::tie(a.blk, a.thr, a.it[0], a.it[1], a.it[2], a.it[3]) <
         std::tie(b.blk, b.thr, b.it[0], b.it[1], b.it[2], b.it[3]);
}

}  // namespace

extern "C" {

typedef struct {
  int32_t grid[3], block[3];
  uint32_t nparams;
  const int64_t* params;
} orc_binding;
typedef struct {
  uint8_t space, array, acc_lo, acc_hi, kind_mask, pad[3];
  uint64_t byte_addr;
} orc_witness;
typedef struct {
  uint32_t lin_block, lin_thread;
  uint32_t iter[4];
  uint8_t access, pad[3];
} orc_inst;
typedef struct {
  int32_t racy, pad;
  uint64_t n_witness, n_by_kind[3], n_instances, n_keys, n_oob;
  orc_witness min_w;
  orc_inst min_x, min_y;
} orc_verdict;

// Check one descriptor under one binding.  filter_array >= 0 keeps only
// buckets of that array whose granule lies in [gran_lo, gran_hi) (a sample of
// the full answer, used on workloads too large to bucket whole); counts of
// instances, keys and out-of-bounds instances are always whole-kernel.
// filter_array == -2 keeps the buckets of every array whose granule g has
// g % gran_hi == gran_lo (band gran_lo of gran_hi): the bands partition the
// buckets, and with them the witnesses, so separate runs can share the work.
// flags bit 0 skips the search for the canonical instance pair (min_x and
// min_y stay zero); everything else is computed as without it.
int orc_check(const char* text, const orc_binding* bind, int filter_array, uint64_t gran_lo, uint64_t gran_hi,
              orc_witness* out, uint64_t cap, orc_verdict* v, char* err, size_t errlen, int flags) {
  try {
    if (!text || !bind || !v) throw Fail{EINVAL_, "null argument"};
    if (filter_array == -2 && (gran_hi == 0 || gran_lo >= gran_hi)) throw Fail{EINVAL_, "bad band"};
    memset(v, 0, sizeof(*v));
    Desc d = parse(std::string(text));
    if (bind->nparams != d.params.size()) throw Fail{EBIND, "parameter count does not match the descriptor"};
    Env e{};
    e.params = bind->params;
    for (int k = 0; k < 3; k++) {
      if (bind->grid[k] < 1 || bind->block[k] < 1) throw Fail{EBIND, "launch dimensions must be >= 1"};
      e.gdim[k] = bind->grid[k];
      e.bdim[k] = bind->block[k];
    }
    if (e.bdim[0] * e.bdim[1] * e.bdim[2] > 1024) throw Fail{EBIND, "more than 1024 threads per block"};
    // divisors, loop bounds, sizes and asserts are all uniform: evaluate now
    std::vector<const Node*> divs;
    for (auto& kv : d.lets) collect_divisors(kv.second.get(), divs);
    for (auto& a : d.acc) {
      collect_divisors(a.idx.get(), divs);
      collect_divisors(a.iv.get(), divs);
      collect_divisors(a.wv.get(), divs);
      if (a.sync_array >= 0) collect_divisors(a.sync.get(), divs);
      for (auto& g : a.guards) {
        collect_divisors(g.lhs.get(), divs);
        collect_divisors(g.rhs.get(), divs);
      }
    }
    for (auto& l : d.loops) collect_divisors(l.second.get(), divs);
    for (auto& a : d.arrays) collect_divisors(a.bytes.get(), divs);
    for (auto& c : d.asserts) {
      collect_divisors(c.lhs.get(), divs);
      collect_divisors(c.rhs.get(), divs);
    }
    for (const Node* dv : divs)
      if (eval(dv, e) <= 0) throw Fail{EBIND, "divisor is not positive"};
    for (auto& c : d.asserts)
      if (!holds(c, e)) throw Fail{EHOST, "host assert does not hold for this binding"};
    std::vector<int64_t> ub;
    for (auto& l : d.loops) ub.push_back(std::max<int64_t>(0, eval(l.second.get(), e)));
    while (ub.size() < 4) ub.push_back(1);
    std::vector<int64_t> bytes;
    for (auto& a : d.arrays) {
      int64_t b = eval(a.bytes.get(), e);
      if (b < 0) throw Fail{EBIND, "array size is negative"};
      bytes.push_back(b);
    }
    const int64_t nthr = e.bdim[0] * e.bdim[1] * e.bdim[2];
    const int64_t nblk = e.gdim[0] * e.gdim[1] * e.gdim[2];
    uint64_t n_inst = (uint64_t)nblk * (uint64_t)nthr * d.acc.size();
    for (int l = 0; l < (int)d.loops.size(); l++) n_inst *= (uint64_t)ub[l];
    v->n_instances = n_inst;

    std::map<Key, std::vector<Inst>> buckets;
    uint64_t n_keys = 0, n_oob = 0;
    // enumerate every (block, thread, loop vector, access) in linear order
    for (e.bid[2] = 0; e.bid[2] < e.gdim[2]; e.bid[2]++)
      for (e.bid[1] = 0; e.bid[1] < e.gdim[1]; e.bid[1]++)
        for (e.bid[0] = 0; e.bid[0] < e.gdim[0]; e.bid[0]++)
          for (e.tid[2] = 0; e.tid[2] < e.bdim[2]; e.tid[2]++)
            for (e.tid[1] = 0; e.tid[1] < e.bdim[1]; e.tid[1]++)
              for (e.tid[0] = 0; e.tid[0] < e.bdim[0]; e.tid[0]++)
                for (e.loop[0] = 0; e.loop[0] < ub[0]; e.loop[0]++)
                  for (e.loop[1] = 0; e.loop[1] < ub[1]; e.loop[1]++)
                    for (e.loop[2] = 0; e.loop[2] < ub[2]; e.loop[2]++)
                      for (e.loop[3] = 0; e.loop[3] < ub[3]; e.loop[3]++)
                        for (int a = 0; a < (int)d.acc.size(); a++) {
                          const Access& A = d.acc[a];
                          bool live = true;
                          for (auto& g : A.guards) live = live && holds(g, e);
                          if (!live) continue;
                          int64_t idx = eval(A.idx.get(), e), off;
                          if (__builtin_mul_overflow(idx, A.width, &off)) throw Fail{EOVF, "byte offset overflows"};
                          const int64_t w = A.width, size = bytes[A.array];
                          if (off < 0 || off > size - w) {
                            n_oob++;
                            continue;
                          }
                          Inst in;
                          in.blk = e.bid[0] + e.bid[1] * e.gdim[0] + e.bid[2] * e.gdim[0] * e.gdim[1];
                          in.thr = e.tid[0] + e.tid[1] * e.bdim[0] + e.tid[2] * e.bdim[0] * e.bdim[1];
                          for (int l = 0; l < 4; l++) in.it[l] = l < (int)d.loops.size() ? e.loop[l] : 0;
                          in.acc = a;
                          in.iv = eval(A.iv.get(), e);
                          in.wv = eval(A.wv.get(), e);
                          in.sync = A.sync_array >= 0 ? eval(A.sync.get(), e) : 0;
                          const int64_t g = d.arrays[A.array].granule;
                          for (int64_t gr = off / g; gr < (off + w) / g; gr++) {
                            n_keys++;
                            if (filter_array >= 0 &&
                                (A.array != filter_array || gr < (int64_t)gran_lo || gr >= (int64_t)gran_hi))
                              continue;
                            if (filter_array == -2 && (uint64_t)gr % gran_hi != gran_lo) continue;
                            const int sp = d.arrays[A.array].space;
                            buckets[Key{sp, A.array, sp == 1 ? in.blk : -1, gr}].push_back(in);
                          }
                        }
    v->n_keys = n_keys;
    v->n_oob = n_oob;

    // per bucket: every pair of accesses, every pair of instances
    const int na = (int)d.acc.size();
    std::map<std::tuple<int, int, int64_t, int, int>, int> wit;  // (space,array,byte,lo,hi) -> mask
    for (auto& kv : buckets) {
      const std::vector<Inst>& B = kv.second;
      std::vector<std::vector<const Inst*>> by(na);
      for (const Inst& in : B) by[in.acc].push_back(&in);
      for (int a = 0; a < na; a++)
        for (int b = a; b < na; b++) {
          const int allow = allowed_kinds(d, a, b);
          if (!allow || by[a].empty() || by[b].empty()) continue;
          int mask = 0;
          for (size_t i = 0; i < by[a].size() && mask != allow; i++)
            for (size_t j = (a == b ? i + 1 : 0); j < by[b].size() && mask != allow; j++)
              mask |= race_kind(d, *by[a][i], *by[b][j]) & allow;
          if (mask) {
            const int64_t byte = kv.first.granule * d.arrays[kv.first.array].granule;
            wit[{kv.first.space, kv.first.array, byte, a, b}] |= mask;
          }
        }
    }
    v->n_witness = wit.size();
    v->racy = !wit.empty();
    uint64_t k = 0;
    for (auto& kv : wit) {
      orc_witness w{};
      w.space = (uint8_t)std::get<0>(kv.first);
      w.array = (uint8_t)std::get<1>(kv.first);
      w.byte_addr = (uint64_t)std::get<2>(kv.first);
      w.acc_lo = (uint8_t)std::get<3>(kv.first);
      w.acc_hi = (uint8_t)std::get<4>(kv.first);
      w.kind_mask = (uint8_t)kv.second;
      for (int t = 0; t < 3; t++)
        if (w.kind_mask >> t & 1) v->n_by_kind[t]++;
      if (k == 0) v->min_w = w;
      if (out && k < cap) out[k] = w;
      k++;
    }
    // canonical instance pair of the minimal witness: the smallest
    // (key(x), key(y)) with x of access acc_lo, y of access acc_hi, both on the
    // witness's granule (any block for shared memory), racing
    if (v->racy && !(flags & 1)) {
      const orc_witness& mw = v->min_w;
      const int64_t g = d.arrays[mw.array].granule;
      const int allow = allowed_kinds(d, mw.acc_lo, mw.acc_hi);
      bool found = false;
      Inst bx{}, byy{};
      for (auto& kv : buckets) {
        if (kv.first.space != mw.space || kv.first.array != mw.array ||
            kv.first.granule * g != (int64_t)mw.byte_addr)
          continue;
        for (const Inst& x : kv.second) {
          if (x.acc != mw.acc_lo) continue;
          for (const Inst& y : kv.second) {
            if (y.acc != mw.acc_hi) continue;
            if (mw.acc_lo == mw.acc_hi && !key_less(x, y)) continue;
            if (!(race_kind(d, x, y) & allow)) continue;
            bool better = !found || key_less(x, bx) || (!key_less(bx, x) && key_less(y, byy));
            if (better) {
              bx = x;
              byy = y;
              found = true;
            }
          }
        }
      }
      auto put = [](orc_inst& o, const Inst& s) {
        o.lin_block = (uint32_t)s.blk;
        o.lin_thread = (uint32_t)s.thr;
        for (int l = 0; l < 4; l++) o.iter[l] = (uint32_t)s.it[l];
        o.access = (uint8_t)s.acc;
      };
      if (found) {
        put(v->min_x, bx);
        put(v->min_y, byy);
      }
    }
    if (err && errlen) err[0] = 0;
    return (out && v->n_witness > cap) ? TRUNC : OK;
  } catch (const Fail& f) {
    if (err && errlen) snprintf(err, errlen, "%s", f.msg.c_str());
    return f.code;
  } catch (const std::exception& ex) {
    if (err && errlen) snprintf(err, errlen, "%s", ex.what());
    return EPARSE;
  }
}

}  // extern "C"
