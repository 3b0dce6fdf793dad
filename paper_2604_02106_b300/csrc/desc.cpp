// Descriptor parsing, host binding and compilation to the device program.
//
// hgrd_load_desc: text -> AST arena + static checks (quasi-affine forms,
//   uniform divisors, loop bounds, sizes and asserts; intervals free of
//   thread/block ids).
// hgrd_bind_host_params: the host-code classes of Sec. 4 / Sec. 5.1 made
//   concrete — every parameter and launch dimension gets its value, asserts
//   are evaluated (class (1)), launch dims bound the ids (class (2)), shared
//   host variables arrive as related values (class (3)), host loop values are
//   swept tuple by tuple (class (4)), allocation sizes arrive as positive
//   values (class (5)).  Expressions are folded into affine forms over the
//   ten instance variables and div/mod nodes, bounded by interval arithmetic
//   over the instance box, and compiled into a DProg for the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "hgrd_host.h"

namespace hgrd {

thread_local std::string g_err;
thread_local hgrd_stats g_stats;
std::atomic<uint64_t> g_created{0};

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

namespace {

struct Err {
  int code;
  std::string msg;
};
[[noreturn]] void raise(int code, const std::string& m) { throw Err{code, m}; }

// ------------------------------------------------------------- tokenizer
struct Tok {
  char t;  // 'n' number, 'i' identifier, else the operator character; 'L','G','E','N' for <= >= == !=
  int64_t v;
  std::string s;
};

std::vector<Tok> tokenize(const std::string& s) {
  std::vector<Tok> out;
  size_t i = 0;
  while (i < s.size()) {
    char c = s[i];
    if (c == ' ' || c == '\t' || c == '\r') {
      i++;
      continue;
    }
    if (isdigit((unsigned char)c)) {
      unsigned __int128 v = 0;
      while (i < s.size() && isdigit((unsigned char)s[i])) {
        v = v * 10 + (s[i] - '0');
        if (v > (unsigned __int128)INT64_MAX) raise(HGRD_EPARSE, "integer literal too large");
        i++;
      }
      out.push_back({'n', (int64_t)v, ""});
      continue;
    }
    if (isalpha((unsigned char)c) || c == '_') {
      size_t j = i;
      while (j < s.size() && (isalnum((unsigned char)s[j]) || s[j] == '_')) j++;
      out.push_back({'i', 0, s.substr(i, j - i)});
      i = j;
      continue;
    }
    if (i + 1 < s.size() && s[i + 1] == '=' && (c == '<' || c == '>' || c == '=' || c == '!')) {
      out.push_back({c == '<' ? 'L' : c == '>' ? 'G' : c == '=' ? 'E' : 'N', 0, ""});
      i += 2;
      continue;
    }
    if (strchr("+-*/%()<>", c)) {
      out.push_back({c, 0, ""});
      i++;
      continue;
    }
    raise(HGRD_EPARSE, std::string("unexpected character '") + c + "'");
  }
  return out;
}

}  // namespace

// ------------------------------------------------------------- parser
struct ExprParser {
  hgrd_desc& d;
  const std::vector<Tok>& t;
  size_t p = 0;

  ExprParser(hgrd_desc& dd, const std::vector<Tok>& tt) : d(dd), t(tt) {}

  int mk(char op, int64_t v, int a, int b) {
    AstNode n;
    n.op = op;
    n.val = v;
    n.a = a;
    n.b = b;
    n.varies = (a >= 0 && d.ast[a].varies) || (b >= 0 && d.ast[b].varies);
    n.thread = (a >= 0 && d.ast[a].thread) || (b >= 0 && d.ast[b].thread);
    d.ast.push_back(n);
    return (int)d.ast.size() - 1;
  }
  int leaf_name(const std::string& s) {
    static const char* vars[6] = {"tx", "ty", "tz", "bx", "by", "bz"};
    static const char* dims[6] = {"bdx", "bdy", "bdz", "gdx", "gdy", "gdz"};
    for (int k = 0; k < 6; k++)
      if (s == vars[k]) {
        int n = mk('v', k, -1, -1);
        d.ast[n].varies = d.ast[n].thread = true;
        return n;
      }
    for (int k = 0; k < 6; k++)
      if (s == dims[k]) return mk('d', k, -1, -1);
    for (size_t k = 0; k < d.loops.size(); k++)
      if (d.loops[k].name == s) {
        int n = mk('v', 6 + (int)k, -1, -1);
        d.ast[n].varies = true;
        return n;
      }
    for (size_t k = 0; k < d.params.size(); k++)
      if (d.params[k] == s) return mk('p', (int64_t)k, -1, -1);
    auto it = d.lets.find(s);
    if (it != d.lets.end()) return it->second;
    raise(HGRD_EPARSE, "unknown name '" + s + "'");
  }
  int atom() {
    if (p >= t.size()) raise(HGRD_EPARSE, "expression ends early");
    const Tok& k = t[p++];
    if (k.t == 'n') return mk('n', k.v, -1, -1);
    if (k.t == 'i') return leaf_name(k.s);
    if (k.t == '-') return mk('~', 0, atom(), -1);
    if (k.t == '(') {
      int e = sum();
      if (p >= t.size() || t[p].t != ')') raise(HGRD_EPARSE, "missing ')'");
      p++;
      return e;
    }
    raise(HGRD_EPARSE, "unexpected token in expression");
  }
  int product() {
    int x = atom();
    while (p < t.size() && (t[p].t == '*' || t[p].t == '/' || t[p].t == '%')) {
      char op = t[p++].t;
      int y = atom();
      if (op == '*' && d.ast[x].varies && d.ast[y].varies)
        raise(HGRD_EPARSE, "not quasi-affine: product of two instance-dependent factors");
      if (op != '*' && d.ast[y].varies) raise(HGRD_EPARSE, "not quasi-affine: divisor depends on thread, block or loop ids");
      x = mk(op, 0, x, y);
    }
    return x;
  }
  int sum() {
    int x = product();
    while (p < t.size() && (t[p].t == '+' || t[p].t == '-')) {
      char op = t[p++].t;
      x = mk(op, 0, x, product());
    }
    return x;
  }
};

static std::string trim(const std::string& s) {
  size_t a = s.find_first_not_of(" \t\r"), b = s.find_last_not_of(" \t\r");
  return a == std::string::npos ? std::string() : s.substr(a, b - a + 1);
}

static int parse_expr(hgrd_desc& d, const std::string& s) {
  std::vector<Tok> t = tokenize(s);
  if (t.empty()) raise(HGRD_EPARSE, "empty expression");
  ExprParser ep(d, t);
  int e = ep.sum();
  if (ep.p != t.size()) raise(HGRD_EPARSE, "trailing text in expression '" + s + "'");
  return e;
}

static CondDecl parse_cond(hgrd_desc& d, const std::string& s, bool allow_ne) {
  std::vector<Tok> t = tokenize(s);
  size_t at = t.size();
  for (size_t k = 0; k < t.size(); k++)
    if (strchr("<>LGEN", t[k].t)) {
      if (at != t.size()) raise(HGRD_EPARSE, "more than one comparison in '" + s + "'");
      at = k;
    }
  if (at == t.size()) raise(HGRD_EPARSE, "condition without comparison: '" + s + "'");
  CondDecl c;
  c.op = t[at].t;
  if (c.op == 'N' && !allow_ne) raise(HGRD_EPARSE, "'!=' is not allowed in a guard");
  std::vector<Tok> l(t.begin(), t.begin() + at), r(t.begin() + at + 1, t.end());
  if (l.empty() || r.empty()) raise(HGRD_EPARSE, "comparison needs two sides");
  ExprParser pl(d, l), pr(d, r);
  c.lhs = pl.sum();
  if (pl.p != l.size()) raise(HGRD_EPARSE, "bad left side in '" + s + "'");
  c.rhs = pr.sum();
  if (pr.p != r.size()) raise(HGRD_EPARSE, "bad right side in '" + s + "'");
  return c;
}

static std::vector<std::string> split_fields(const std::string& s) {
  std::vector<std::string> out;
  size_t st = 0;
  for (;;) {
    size_t q = s.find(';', st);
    out.push_back(trim(s.substr(st, q == std::string::npos ? std::string::npos : q - st)));
    if (q == std::string::npos) break;
    st = q + 1;
  }
  return out;
}

static std::string first_word(const std::string& in, std::string* rest) {
  const std::string s = in;  // `rest` may alias `in`
  size_t a = s.find_first_not_of(" \t");
  if (a == std::string::npos) {
    if (rest) *rest = "";
    return "";
  }
  size_t b = s.find_first_of(" \t", a);
  if (rest) *rest = b == std::string::npos ? "" : trim(s.substr(b));
  return s.substr(a, b == std::string::npos ? std::string::npos : b - a);
}

static bool ident(const std::string& s) {
  if (s.empty() || !(isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
  for (char c : s)
    if (!(isalnum((unsigned char)c) || c == '_')) return false;
  return true;
}

void parse_desc(hgrd_desc& d, const std::string& text) {
  std::vector<std::string> taken = {"tx", "ty", "tz", "bx", "by", "bz", "bdx", "bdy", "bdz", "gdx", "gdy", "gdz"};
  auto declare = [&](const std::string& n) {
    if (!ident(n)) raise(HGRD_EPARSE, "bad name '" + n + "'");
    if (std::find(taken.begin(), taken.end(), n) != taken.end()) raise(HGRD_EPARSE, "name '" + n + "' declared twice");
    taken.push_back(n);
  };
  bool kernel = false;
  size_t pos = 0;
  while (pos <= text.size()) {
    size_t nl = text.find('\n', pos);
    std::string line = text.substr(pos, nl == std::string::npos ? std::string::npos : nl - pos);
    pos = nl == std::string::npos ? text.size() + 1 : nl + 1;
    size_t hash = line.find('#');
    if (hash != std::string::npos) line = line.substr(0, hash);
    line = trim(line);
    if (line.empty()) continue;
    std::string rest;
    std::string dir = first_word(line, &rest);
    if (dir == "kernel") {
      kernel = true;
      d.name = rest;
    } else if (dir == "param") {
      std::string r = rest;
      while (!r.empty()) {
        std::string nm = first_word(r, &r);
        declare(nm);
        d.params.push_back(nm);
      }
    } else if (dir == "loop") {
      std::string bound;
      std::string nm = first_word(rest, &bound);
      if (d.loops.size() >= (size_t)MAXLOOP) raise(HGRD_EUNSUPPORTED, "more than 4 loops");
      declare(nm);
      LoopDecl L;
      L.name = nm;
      L.bound = parse_expr(d, bound);
      if (d.ast[L.bound].varies) raise(HGRD_EPARSE, "loop bound must not depend on thread, block or loop ids");
      d.loops.push_back(L);
    } else if (dir == "array") {
      std::vector<std::string> f = split_fields(rest);
      std::string r1, r2;
      std::string nm = first_word(f[0], &r1);
      std::string sp = first_word(r1, &r2);
      declare(nm);
      ArrayDecl a;
      a.name = nm;
      if (sp == "global") a.space = HGRD_SPACE_GLOBAL;
      else if (sp == "shared") a.space = HGRD_SPACE_SHARED;
      else raise(HGRD_EPARSE, "array space must be global or shared");
      a.bytes = parse_expr(d, r2);
      if (d.ast[a.bytes].varies) raise(HGRD_EPARSE, "array size must not depend on thread, block or loop ids");
      for (size_t k = 1; k < f.size(); k++) {
        std::string v;
        std::string key = first_word(f[k], &v);
        if (key != "granule") raise(HGRD_EPARSE, "unknown array field '" + key + "'");
        a.granule = std::stoll(v);
        if (a.granule <= 0) raise(HGRD_EPARSE, "granule must be positive");
      }
      if (d.arrays.size() >= (size_t)MAXARR) raise(HGRD_EUNSUPPORTED, "more than 32 arrays");
      d.arrays.push_back(a);
    } else if (dir == "let") {
      size_t eq = rest.find('=');
      if (eq == std::string::npos) raise(HGRD_EPARSE, "let needs '='");
      std::string nm = trim(rest.substr(0, eq));
      declare(nm);
      d.lets[nm] = parse_expr(d, rest.substr(eq + 1));
    } else if (dir == "assert") {
      CondDecl c = parse_cond(d, rest, true);
      if (d.ast[c.lhs].varies || d.ast[c.rhs].varies)
        raise(HGRD_EPARSE, "assert must not depend on thread, block or loop ids");
      d.asserts.push_back(c);
    } else if (dir == "access") {
      std::vector<std::string> f = split_fields(rest);
      std::string r1;
      std::string kind = first_word(f[0], &r1);
      AccessDecl a;
      if (kind == "R") a.kind = 0;
      else if (kind == "W") a.kind = 1;
      else if (kind == "A") a.kind = 2;
      else raise(HGRD_EPARSE, "access kind must be R, W or A");
      a.arr = -1;
      for (size_t k = 0; k < d.arrays.size(); k++)
        if (d.arrays[k].name == trim(r1)) a.arr = (int)k;
      if (a.arr < 0) raise(HGRD_EPARSE, "unknown array '" + trim(r1) + "'");
      bool has_idx = false;
      for (size_t k = 1; k < f.size(); k++) {
        std::string body;
        std::string key = first_word(f[k], &body);
        if (key.empty()) continue;
        if (key == "width") {
          a.width = std::stoll(body);
          if (a.width <= 0) raise(HGRD_EPARSE, "width must be positive");
        } else if (key == "iv") {
          a.iv = parse_expr(d, body);
          if (d.ast[a.iv].thread) raise(HGRD_EPARSE, "interval must not depend on thread or block ids");
        } else if (key == "wv") {
          a.wv = parse_expr(d, body);
          if (d.ast[a.wv].thread) raise(HGRD_EPARSE, "warp interval must not depend on thread or block ids");
        } else if (key == "idx") {
          a.idx = parse_expr(d, body);
          has_idx = true;
        } else if (key == "if") {
          a.guards.push_back(parse_cond(d, body, false));
        } else if (key == "scope") {
          if (body == "block") a.scope = 0;
          else if (body == "device") a.scope = 1;
          else raise(HGRD_EPARSE, "scope must be block or device");
        } else if (key == "sync") {
          std::string sexpr;
          const std::string sname = trim(first_word(body, &sexpr));
          for (size_t k = 0; k < d.arrays.size(); k++)
            if (d.arrays[k].name == sname) a.sync_arr = (int)k;
          if (a.sync_arr < 0) raise(HGRD_EPARSE, "unknown sync array '" + sname + "'");
          if (d.arrays[a.sync_arr].space != HGRD_SPACE_GLOBAL) raise(HGRD_EPARSE, "a sync array must be global");
          a.sync = parse_expr(d, sexpr);
        } else if (key == "syncscope") {
          if (body == "block") a.sync_scope = 0;
          else if (body == "device") a.sync_scope = 1;
          else raise(HGRD_EPARSE, "syncscope must be block or device");
        } else if (key == "line") {
          a.line = (int)std::stoll(body);
        } else {
          raise(HGRD_EPARSE, "unknown access field '" + key + "'");
        }
      }
      if (!has_idx || a.width == 0) raise(HGRD_EPARSE, "access needs width and idx");
      if (d.acc.size() >= (size_t)MAXACC) raise(HGRD_EUNSUPPORTED, "more than 32 accesses");
      d.acc.push_back(a);
    } else {
      raise(HGRD_EPARSE, "unknown directive '" + dir + "'");
    }
  }
  if (!kernel) raise(HGRD_EPARSE, "missing 'kernel' line");
  for (size_t k = 0; k < d.arrays.size(); k++) {
    int64_t g = 0;
    for (auto& a : d.acc)
      if (a.arr == (int)k) g = std::gcd(g, a.width);
    if (!d.arrays[k].granule) d.arrays[k].granule = g ? g : 4;
    for (auto& a : d.acc)
      if (a.arr == (int)k && a.width % d.arrays[k].granule)
        raise(HGRD_EPARSE, "access width is not a multiple of the array granule");
  }
}

// ------------------------------------------------------------- folding
namespace {

int64_t add_c(int64_t a, int64_t b) {
  int64_t r;
  if (__builtin_add_overflow(a, b, &r)) raise(HGRD_EOVERFLOW, "constant folding overflows int64");
  return r;
}
int64_t mul_c(int64_t a, int64_t b) {
  int64_t r;
  if (__builtin_mul_overflow(a, b, &r)) raise(HGRD_EOVERFLOW, "constant folding overflows int64");
  return r;
}

struct Lin {
  int64_t c0 = 0;
  int64_t cv[NVAR] = {};
  std::map<int, int64_t> cn;  // node id -> coefficient
  bool is_const() const {
    for (int k = 0; k < NVAR; k++)
      if (cv[k]) return false;
    return cn.empty();
  }
  std::string key() const {
    std::string s = std::to_string(c0);
    for (int k = 0; k < NVAR; k++) s += "," + std::to_string(cv[k]);
    for (auto& kv : cn) s += ";" + std::to_string(kv.first) + ":" + std::to_string(kv.second);
    return s;
  }
};

Lin lin_add(const Lin& a, const Lin& b, int64_t sb) {
  Lin r = a;
  r.c0 = add_c(r.c0, mul_c(sb, b.c0));
  for (int k = 0; k < NVAR; k++) r.cv[k] = add_c(r.cv[k], mul_c(sb, b.cv[k]));
  for (auto& kv : b.cn) {
    int64_t c = add_c(r.cn[kv.first], mul_c(sb, kv.second));
    if (c) r.cn[kv.first] = c;
    else r.cn.erase(kv.first);
  }
  return r;
}
Lin lin_scale(const Lin& a, int64_t s) {
  Lin r;
  if (s == 0) return r;
  r.c0 = mul_c(a.c0, s);
  for (int k = 0; k < NVAR; k++) r.cv[k] = mul_c(a.cv[k], s);
  for (auto& kv : a.cn) r.cn[kv.first] = mul_c(kv.second, s);
  return r;
}

struct Node {
  Lin num;
  int64_t d;
  int op;  // OP_DIV or OP_MOD
  bool loop = false;
  int64_t lo = 0, hi = 0;
};

struct Folder {
  const hgrd_desc& d;
  const int64_t* params;
  int64_t dims[6];
  std::vector<Node> nodes;
  std::map<std::string, int> memo_nodes;
  std::map<int, Lin> memo;

  Folder(const hgrd_desc& dd, const int64_t* p, const int64_t* dm) : d(dd), params(p) {
    for (int k = 0; k < 6; k++) dims[k] = dm[k];
  }

  int64_t cdiv(int64_t a, int64_t b) { return a / b; }

  Lin fold(int i) {
    auto it = memo.find(i);
    if (it != memo.end()) return it->second;
    const AstNode& n = d.ast[i];
    Lin r;
    switch (n.op) {
      case 'n': r.c0 = n.val; break;
      case 'v': r.cv[n.val] = 1; break;
      case 'd': r.c0 = dims[n.val]; break;
      case 'p': r.c0 = params[n.val]; break;
      case '~': r = lin_scale(fold(n.a), -1); break;
      case '+': r = lin_add(fold(n.a), fold(n.b), 1); break;
      case '-': r = lin_add(fold(n.a), fold(n.b), -1); break;
      case '*': {
        Lin x = fold(n.a), y = fold(n.b);
        if (x.is_const()) r = lin_scale(y, x.c0);
        else if (y.is_const()) r = lin_scale(x, y.c0);
        else raise(HGRD_EPARSE, "not quasi-affine product");
        break;
      }
      case '/':
      case '%': {
        Lin x = fold(n.a), y = fold(n.b);
        if (!y.is_const()) raise(HGRD_EPARSE, "divisor depends on instance ids");
        int64_t dv = y.c0;
        if (dv <= 0) raise(HGRD_EBIND, "divisor is not positive for this binding");
        if (x.is_const()) {
          r.c0 = n.op == '/' ? x.c0 / dv : x.c0 % dv;
        } else if (dv == 1) {
          if (n.op == '/') r = x;
        } else {
          Node nd;
          nd.num = x;
          nd.d = dv;
          nd.op = n.op == '/' ? OP_DIV : OP_MOD;
          std::string k = std::string(1, n.op) + std::to_string(dv) + "|" + x.key();
          auto f = memo_nodes.find(k);
          int id;
          if (f != memo_nodes.end()) {
            id = f->second;
          } else {
            id = (int)nodes.size();
            nodes.push_back(nd);
            memo_nodes[k] = id;
          }
          r.cn[id] = 1;
        }
        break;
      }
      default: raise(HGRD_EPARSE, "internal: bad AST node");
    }
    memo[i] = r;
    return r;
  }
  int64_t value(int i) {
    Lin l = fold(i);
    if (!l.is_const()) raise(HGRD_EPARSE, "expression is not uniform");
    return l.c0;
  }
};

bool cond_holds(int64_t x, int64_t y, char op) {
  switch (op) {
    case '<': return x < y;
    case 'L': return x <= y;
    case '>': return x > y;
    case 'G': return x >= y;
    case 'E': return x == y;
    default: return x != y;
  }
}

// guard lins that must be >= 0 for `lhs op rhs`
std::vector<Lin> guard_lins(const Lin& l, const Lin& r, char op) {
  std::vector<Lin> out;
  Lin one;
  one.c0 = 1;
  switch (op) {
    case '<': out.push_back(lin_add(lin_add(r, l, -1), one, -1)); break;
    case 'L': out.push_back(lin_add(r, l, -1)); break;
    case '>': out.push_back(lin_add(lin_add(l, r, -1), one, -1)); break;
    case 'G': out.push_back(lin_add(l, r, -1)); break;
    case 'E':
      out.push_back(lin_add(l, r, -1));
      out.push_back(lin_add(r, l, -1));
      break;
  }
  return out;
}

__int128 iabs(__int128 x) { return x < 0 ? -x : x; }

int ceil_log2(uint64_t x) {
  int b = 0;
  while (b < 64 && ((uint64_t)1 << b) < x) b++;
  return b;
}

Magic make_magic(int64_t d, int N) {
  Magic g{};
  int l = ceil_log2((uint64_t)d);
  unsigned __int128 num = (unsigned __int128)1 << (N + l);
  g.m = (uint64_t)(num / (uint64_t)d) + 1;
  g.shift = N + l;
  return g;
}

}  // namespace

// ------------------------------------------------------------- binding
struct Compiler {
  hgrd_desc& d;
  Folder F;
  Bound& B;
  DProg& P;
  int64_t vlo[NVAR], vhi[NVAR];

  Compiler(hgrd_desc& dd, const int64_t* params, const int64_t* dims, Bound& b)
      : d(dd), F(dd, params, dims), B(b), P(b.prog) {}

  void range(const Lin& l, int64_t& lo, int64_t& hi) {
    __int128 a = l.c0, b = l.c0;
    for (int k = 0; k < NVAR; k++) {
      __int128 x = (__int128)l.cv[k] * vlo[k], y = (__int128)l.cv[k] * vhi[k];
      a += std::min(x, y);
      b += std::max(x, y);
    }
    for (auto& kv : l.cn) {
      const Node& n = F.nodes[kv.first];
      __int128 x = (__int128)kv.second * n.lo, y = (__int128)kv.second * n.hi;
      a += std::min(x, y);
      b += std::max(x, y);
    }
    if (a < INT64_MIN / 2 || b > INT64_MAX / 2) raise(HGRD_EOVERFLOW, "an index expression can leave the int64 range");
    lo = (int64_t)a;
    hi = (int64_t)b;
  }
  // upper bound on |any partial sum| while evaluating the form term by term
  __int128 magnitude(const Lin& l) {
    __int128 m = l.c0 < 0 ? -(__int128)l.c0 : l.c0;
    for (int k = 0; k < NVAR; k++) {
      __int128 c = l.cv[k] < 0 ? -(__int128)l.cv[k] : l.cv[k];
      m += c * std::max(iabs((__int128)vlo[k]), iabs((__int128)vhi[k]));
    }
    for (auto& kv : l.cn) {
      const Node& n = F.nodes[kv.first];
      __int128 c = kv.second < 0 ? -(__int128)kv.second : kv.second;
      m += c * std::max(iabs((__int128)n.lo), iabs((__int128)n.hi));
    }
    return m;
  }
  bool lin_loop(const Lin& l) {
    for (int k = 6; k < NVAR; k++)
      if (l.cv[k]) return true;
    for (auto& kv : l.cn)
      if (F.nodes[kv.first].loop) return true;
    return false;
  }
};

int bind_desc(hgrd_desc& d, const hgrd_binding* bind) {
  try {
    if (!bind) raise(HGRD_EINVAL, "null binding");
    if (bind->nparams != d.params.size()) raise(HGRD_EBIND, "parameter count does not match the descriptor");
    if (bind->nparams && !bind->params) raise(HGRD_EINVAL, "null parameter array");
    std::unique_ptr<Bound> bp(new Bound());
    static std::atomic<uint64_t> next_gen{1};
    bp->gen = next_gen++;
    Bound& B = *bp;
    memset(&B.prog, 0, sizeof(DProg));
    DProg& P = B.prog;
    int64_t dims[6];
    for (int k = 0; k < 3; k++) {
      if (bind->grid[k] < 1 || bind->block[k] < 1) raise(HGRD_EBIND, "launch dimensions must be >= 1");
      dims[k] = bind->block[k];
      dims[3 + k] = bind->grid[k];
      P.grid[k] = bind->grid[k];
      P.block[k] = bind->block[k];
    }
    const int64_t nthr = dims[0] * dims[1] * dims[2];
    if (nthr > 1024) raise(HGRD_EBIND, "more than 1024 threads per block");
    const int64_t nblk = dims[3] * dims[4] * dims[5];
    std::vector<int64_t> params(bind->params, bind->params + bind->nparams);
    Compiler C(d, params.data(), dims, B);
    Folder& F = C.F;
    // divisors anywhere are checked by folding; asserts (host class (1))
    for (auto& c : d.asserts) {
      int64_t x = F.value(c.lhs), y = F.value(c.rhs);
      if (!cond_holds(x, y, c.op)) raise(HGRD_EHOSTCONSTRAINT, "host assert does not hold for this binding");
    }
    int64_t ub[MAXLOOP] = {1, 1, 1, 1};
    for (size_t l = 0; l < d.loops.size(); l++) ub[l] = std::max<int64_t>(0, F.value(d.loops[l].bound));
    std::vector<int64_t> bytes;
    for (auto& a : d.arrays) {
      int64_t b = F.value(a.bytes);
      if (b < 0) raise(HGRD_EBIND, "array size is negative");
      bytes.push_back(b);
    }
    B.array_bytes = bytes;
    for (auto& a : d.arrays) B.array_granule.push_back(a.granule);
    B.n_instances = 0;
    {
      unsigned __int128 n = (unsigned __int128)nblk * nthr * d.acc.size();
      for (size_t l = 0; l < d.loops.size(); l++) n *= (uint64_t)ub[l];
      if (n > (unsigned __int128)UINT64_MAX) raise(HGRD_EOVERFLOW, "instance count exceeds 2^64");
      B.n_instances = (uint64_t)n;
    }
    int64_t nit = 1;
    for (size_t l = 0; l < d.loops.size(); l++) nit *= ub[l];
    // variable ranges over the instance box (class (2): ids below launch dims)
    for (int k = 0; k < 6; k++) C.vlo[k] = 0;
    for (int k = 0; k < 3; k++) {
      C.vhi[k] = dims[k] - 1;          // tx ty tz < bdx bdy bdz
      C.vhi[3 + k] = dims[3 + k] - 1;  // bx by bz < gdx gdy gdz
    }
    for (int l = 0; l < MAXLOOP; l++) {
      C.vlo[6 + l] = 0;
      C.vhi[6 + l] = std::max<int64_t>(0, ub[l] - 1);
    }
    // fold every access expression
    struct AccF {
      Lin idx, iv, wv;
      std::vector<Lin> guards;
      bool dead = false;
    };
    std::vector<AccF> af(d.acc.size());
    for (size_t a = 0; a < d.acc.size(); a++) {
      const AccessDecl& A = d.acc[a];
      af[a].idx = F.fold(A.idx);
      if (A.iv >= 0) af[a].iv = F.fold(A.iv);
      if (A.wv >= 0) af[a].wv = F.fold(A.wv);
      for (auto& g : A.guards) {
        for (Lin& l : guard_lins(F.fold(g.lhs), F.fold(g.rhs), g.op)) af[a].guards.push_back(l);
      }
    }
    // acquire-release guards (Sec. 6.5): the form of each guard's element, a
    // constant, the access's own index, or another; folded on a copy of the
    // folder so that no expression node of theirs joins the program
    std::vector<char> s_const(d.acc.size(), 0), s_own(d.acc.size(), 0);  // (both, when the index is constant)
    std::vector<char> s_ids(d.acc.size(), 0);  // affine in thread and block ids alone
    std::vector<int64_t> sval(d.acc.size(), 0);
    std::vector<Lin> slin(d.acc.size());
    for (size_t a = 0; a < d.acc.size(); a++) {
      if (d.acc[a].sync_arr < 0) continue;
      Folder F2 = F;
      const Lin s = F2.fold(d.acc[a].sync);
      s_const[a] = s.is_const();
      sval[a] = s.c0;
      s_own[a] = s.key() == af[a].idx.key();
      bool ids = s.cn.empty();
      for (int k = 6; k < NVAR; k++) ids = ids && s.cv[k] == 0;
      s_ids[a] = ids;
      slin[a] = s;
    }
    // node ranges and loop dependence, in creation order (operands first)
    for (size_t i = 0; i < F.nodes.size(); i++) {
      Node& n = F.nodes[i];
      int64_t lo, hi;
      C.range(n.num, lo, hi);
      n.loop = C.lin_loop(n.num);
      if (n.op == OP_DIV) {
        n.lo = lo / n.d;
        n.hi = hi / n.d;
      } else if (lo >= 0) {
        n.lo = hi < n.d ? lo : 0;
        n.hi = std::min(hi, n.d - 1);
      } else if (hi <= 0) {
        n.lo = lo > -n.d ? lo : -(n.d - 1);
        n.hi = 0;
      } else {
        n.lo = std::max(lo, -(n.d - 1));
        n.hi = std::min(hi, n.d - 1);
      }
    }
    // guards: drop the always-true, mark never-true accesses dead
    for (auto& A : af) {
      std::vector<Lin> keep;
      for (Lin& g : A.guards) {
        int64_t lo, hi;
        C.range(g, lo, hi);
        if (hi < 0) A.dead = true;
        else if (lo < 0) keep.push_back(g);
      }
      A.guards = keep;
    }
    if (nit == 0) {
      for (auto& A : af) A.dead = true;
    }
    // integer width: every form evaluated on the device must keep all partial
    // sums inside int32 for the 32-bit path, else inside 2^62
    __int128 mag = 0;
    auto see = [&](const Lin& l) { mag = std::max(mag, C.magnitude(l)); };
    for (auto& n : F.nodes) see(n.num);
    for (size_t a = 0; a < af.size(); a++) {
      if (af[a].dead) continue;
      see(af[a].idx);
      see(af[a].iv);
      see(af[a].wv);
      for (auto& g : af[a].guards) see(g);
    }
    for (auto& n : F.nodes) mag = std::max(mag, (__int128)std::max(iabs((__int128)n.lo), iabs((__int128)n.hi)));
    const bool wide = mag >= ((__int128)1 << 31) - 1;
    if (mag >= ((__int128)1 << 62)) raise(HGRD_EOVERFLOW, "index arithmetic can exceed 2^62");
    P.wide = wide;
    const int N = wide ? 62 : 31;

    // ---- compile to the device program
    // slots: 0..9 variables; then one slot per node and per hoisted partial
    int nslot = NVAR;
    std::vector<int> node_slot(F.nodes.size(), -1);
    std::vector<DOp> fix, iter;
    std::vector<DTerm> terms;
    auto emit_terms = [&](const Lin& l, bool want_loop, bool want_fixed, DLin& out) {
      out.first = (int)terms.size();
      out.n = 0;
      for (int k = 0; k < NVAR; k++) {
        if (!l.cv[k]) continue;
        bool isloop = k >= 6;
        if (isloop ? want_loop : want_fixed) {
          terms.push_back(DTerm{k, 0, l.cv[k]});
          out.n++;
        }
      }
      for (auto& kv : l.cn) {
        bool isloop = F.nodes[kv.first].loop;
        if (isloop ? want_loop : want_fixed) {
          terms.push_back(DTerm{node_slot[kv.first], 0, kv.second});
          out.n++;
        }
      }
    };
    auto has_fixed_terms = [&](const Lin& l) {
      for (int k = 0; k < 6; k++)
        if (l.cv[k]) return true;
      for (auto& kv : l.cn)
        if (!F.nodes[kv.first].loop) return true;
      return false;
    };
    // a form evaluated per loop vector: hoist its fixed part into a slot
    auto compile_lin = [&](const Lin& l, DLin& out) {
      if (!C.lin_loop(l)) {
        if (!has_fixed_terms(l)) {  // constant
          out.first = (int)terms.size();
          out.n = 0;
          out.c0 = l.c0;
          return;
        }
        DOp op{};
        op.kind = OP_LIN;
        op.dst = nslot++;
        emit_terms(l, false, true, op.lin);
        op.lin.c0 = l.c0;
        fix.push_back(op);
        out.first = (int)terms.size();
        terms.push_back(DTerm{op.dst, 0, 1});
        out.n = 1;
        out.c0 = 0;
        return;
      }
      if (has_fixed_terms(l)) {
        DOp op{};
        op.kind = OP_LIN;
        op.dst = nslot++;
        emit_terms(l, false, true, op.lin);
        op.lin.c0 = l.c0;
        fix.push_back(op);
        DLin lp;
        emit_terms(l, true, false, lp);
        // lp's terms are contiguous; append the partial slot
        terms.push_back(DTerm{op.dst, 0, 1});
        out.first = lp.first;
        out.n = lp.n + 1;
        out.c0 = 0;
        return;
      }
      emit_terms(l, true, false, out);
      out.c0 = l.c0;
    };
    for (size_t i = 0; i < F.nodes.size(); i++) {
      Node& n = F.nodes[i];
      DOp op{};
      op.kind = n.op;
      op.d = n.d;
      op.mg = make_magic(n.d, N);
      node_slot[i] = -1;
      if (!n.loop) {
        op.dst = nslot++;
        emit_terms(n.num, false, true, op.lin);
        op.lin.c0 = n.num.c0;
        fix.push_back(op);
      } else {
        compile_lin(n.num, op.lin);
        op.dst = nslot++;
        iter.push_back(op);
      }
      node_slot[i] = op.dst;
    }
    // access table
    P.nacc = (int)d.acc.size();
    std::vector<DLin> guards;
    int64_t ivmin = INT64_MAX, ivmax = INT64_MIN;
    int64_t wvmin = INT64_MAX, wvmax = INT64_MIN;
    // block-barrier interval range of each live access (whole range: dead)
    std::vector<int64_t> acc_ivlo(d.acc.size(), INT64_MIN), acc_ivhi(d.acc.size(), INT64_MAX);
    for (size_t a = 0; a < d.acc.size(); a++) {
      DAcc& X = P.acc[a];
      const AccessDecl& A = d.acc[a];
      X.arr = A.arr;
      X.shared = d.arrays[A.arr].space == HGRD_SPACE_SHARED;
      X.G = (int32_t)(A.width / d.arrays[A.arr].granule);
      const int64_t by = bytes[A.arr];
      X.maxidx = by >= A.width ? (by - A.width) / A.width : -1;
      X.ngran = (uint64_t)(by / d.arrays[A.arr].granule);
      X.dead = af[a].dead;
      if (X.dead) continue;
      compile_lin(af[a].idx, X.idx);
      compile_lin(af[a].iv, X.iv);
      compile_lin(af[a].wv, X.wv);
      X.gfirst = (int)guards.size();
      X.ng = (int)af[a].guards.size();
      for (auto& g : af[a].guards) {
        DLin dl;
        compile_lin(g, dl);
        guards.push_back(dl);
      }
      int64_t lo, hi;
      C.range(af[a].idx, lo, hi);
      X.bounds_free = lo >= 0 && hi <= X.maxidx;
      if (__int128(std::max(iabs((__int128)lo), iabs((__int128)hi))) * A.width >= ((__int128)1 << 62))
        raise(HGRD_EOVERFLOW, "byte offsets can exceed 2^62");
      C.range(af[a].iv, lo, hi);
      acc_ivlo[a] = lo;
      acc_ivhi[a] = hi;
      ivmin = std::min(ivmin, lo);
      ivmax = std::max(ivmax, hi);
      C.range(af[a].wv, lo, hi);
      wvmin = std::min(wvmin, lo);
      wvmax = std::max(wvmax, hi);
    }
    // facts kept for the ranker's pair features
    B.acc_info.resize(d.acc.size());
    for (size_t a = 0; a < d.acc.size(); a++) {
      AccInfo& I = B.acc_info[a];
      const AccessDecl& A = d.acc[a];
      I.kind = A.kind;
      I.scope = A.scope;
      I.arr = A.arr;
      I.shared = d.arrays[A.arr].space == HGRD_SPACE_SHARED;
      I.width = A.width;
      I.G = P.acc[a].G;
      I.maxidx = P.acc[a].maxidx;
      I.dead = af[a].dead;
      I.nguards = (int)af[a].guards.size();
      if (I.dead) continue;
      for (int k = 0; k < NVAR; k++) I.cv[k] = af[a].idx.cv[k];
      I.nnodes = (int)af[a].idx.cn.size();
      for (auto& kv : af[a].idx.cn) I.loop_nodes += F.nodes[kv.first].loop ? 1 : 0;
      C.range(af[a].idx, I.idx_lo, I.idx_hi);
      C.range(af[a].iv, I.iv_lo, I.iv_hi);
    }
    if (fix.size() + iter.size() > (size_t)MAXOP || terms.size() > (size_t)MAXTERM ||
        guards.size() > (size_t)MAXGUARD || nslot > MAXSLOT)
      raise(HGRD_EUNSUPPORTED, "descriptor too complex for the device program limits");
    P.nfix = (int)fix.size();
    P.niter = (int)iter.size();
    for (size_t k = 0; k < fix.size(); k++) P.ops[k] = fix[k];
    for (size_t k = 0; k < iter.size(); k++) P.ops[fix.size() + k] = iter[k];
    P.nterm = (int)terms.size();
    for (size_t k = 0; k < terms.size(); k++) P.term[k] = terms[k];
    P.nguard = (int)guards.size();
    for (size_t k = 0; k < guards.size(); k++) P.guard[k] = guards[k];
    P.nslot = nslot;
    P.nthr = (int32_t)nthr;
    P.wpb = (int32_t)((nthr + 31) / 32);
    P.nblk = nblk;
    // long loops over few threads: split each simulated warp's loop vectors
    // into chunks so that the expansion has enough independent units
    {
      const int64_t base_units = nblk * P.wpb;
      int64_t chunks = 1;
      if (nit > 64 && base_units < 32768) chunks = std::min<int64_t>((nit + 63) / 64, (32768 + base_units - 1) / base_units);
      P.itc = std::max<int64_t>(1, (nit + chunks - 1) / chunks);
      P.nchunk = nit > 0 ? (nit + P.itc - 1) / P.itc : 1;
    }
    P.nunits = nblk * P.wpb * P.nchunk;
    {
      const int64_t dvs[6] = {P.nchunk, P.wpb, bind->grid[0], bind->grid[1], bind->block[0], bind->block[1]};
      for (int k = 0; k < 6; k++) P.dv[k] = make_magic(std::max<int64_t>(1, dvs[k]), 31);
    }
    P.nloop = (int32_t)d.loops.size();
    for (int l = 0; l < MAXLOOP; l++) P.ub[l] = (int32_t)(l < P.nloop ? ub[l] : 1);
    for (int l = 0; l < P.nloop; l++)
      if (ub[l] > INT32_MAX) raise(HGRD_EUNSUPPORTED, "loop bound above 2^31");
    P.nit = nit;

    // ---- block-pair pruning: an access of a global array whose index is
    // affine (no division or remainder) covers, in block b, at most the
    // bytes [(lo + s(b)) w, (hi + s(b)) w + w), with [lo, hi] the index range
    // over the threads and loop counters and s(b) its block-id terms.  Two
    // accesses whose hulls of two different blocks never meet cannot race
    // across blocks; their inter-block kind leaves the pair rule.  (A sweep
    // over the blocks' hulls sorted by start; skipped past a work budget.)
    std::vector<char> affine(d.acc.size(), 0);
    std::vector<int64_t> hlo(d.acc.size(), 0), hhi(d.acc.size(), 0);
    for (size_t a = 0; a < d.acc.size(); a++) {
      const Lin& L = af[a].idx;
      if (af[a].dead || d.arrays[d.acc[a].arr].space != HGRD_SPACE_GLOBAL || !L.cn.empty()) continue;
      int64_t lo = L.c0, hi = L.c0;
      bool empty = false;
      auto widen = [&](int64_t c, int64_t r) {
        if (r <= 0) empty = true;
        const int64_t t = c * (r - 1);
        (t < 0 ? lo : hi) += t;
      };
      for (int k = 0; k < 3; k++) widen(L.cv[k], dims[k]);
      for (size_t l = 0; l < d.loops.size(); l++) widen(L.cv[6 + l], ub[l]);
      affine[a] = !empty;
      hlo[a] = lo;
      hhi[a] = hi;
    }
    auto bshift = [&](size_t a, int64_t b) {
      const int64_t bx = b % dims[3], by = (b / dims[3]) % dims[4], bz = b / (dims[3] * dims[4]);
      return af[a].idx.cv[3] * bx + af[a].idx.cv[4] * by + af[a].idx.cv[5] * bz;
    };
    std::vector<std::vector<signed char>> disj(d.acc.size(), std::vector<signed char>(d.acc.size(), -1));
    int64_t sweep_budget = (int64_t)1 << 21;  // block hulls swept in all (32 B each on the host)
    auto blocks_disjoint = [&](int a, int b) -> bool {
      if (disj[a][b] >= 0) return disj[a][b] != 0;
      const int sides = a == b ? 1 : 2;
      if (nblk * sides > sweep_budget) return false;
      sweep_budget -= nblk * sides;
      struct Hull {
        int64_t lo, hi, blk;
        int side;
      };
      std::vector<Hull> v;
      v.reserve((size_t)(nblk * sides));
      const int acc2[2] = {a, b};
      for (int sd = 0; sd < sides; sd++) {
        const int x = acc2[sd];
        const int64_t w = d.acc[x].width;
        for (int64_t blk = 0; blk < nblk; blk++) {
          const int64_t s0 = bshift((size_t)x, blk);
          v.push_back({(hlo[x] + s0) * w, (hhi[x] + s0) * w + w - 1, blk, sd});
        }
      }
      std::sort(v.begin(), v.end(), [](const Hull& p, const Hull& q) { return p.lo < q.lo; });
      // per side: the largest hull ends of two different blocks seen so far
      int64_t hi1[2] = {INT64_MIN, INT64_MIN}, hi2[2] = {INT64_MIN, INT64_MIN};
      int64_t bk1[2] = {-1, -1}, bk2[2] = {-1, -1};
      bool meet = false;
      for (const Hull& h : v) {
        const int o = sides == 1 ? 0 : 1 - h.side;
        if ((bk1[o] != h.blk ? hi1[o] : hi2[o]) >= h.lo) {
          meet = true;
          break;
        }
        const int sd = h.side;
        if (h.blk == bk1[sd]) {
          hi1[sd] = std::max(hi1[sd], h.hi);
        } else if (h.blk == bk2[sd]) {
          hi2[sd] = std::max(hi2[sd], h.hi);
          if (hi2[sd] > hi1[sd]) {
            std::swap(hi1[sd], hi2[sd]);
            std::swap(bk1[sd], bk2[sd]);
          }
        } else if (h.hi > hi1[sd]) {
          hi2[sd] = hi1[sd];
          bk2[sd] = bk1[sd];
          hi1[sd] = h.hi;
          bk1[sd] = h.blk;
        } else if (h.hi > hi2[sd]) {
          hi2[sd] = h.hi;
          bk2[sd] = h.blk;
        }
      }
      disj[a][b] = disj[b][a] = meet ? 0 : 1;
      return !meet;
    };

    // ---- thread-tile pruning: two accesses of one width whose index terms
    // on the thread and block ids are equal reach element c0 + L(v) + l, with
    // L(v) the id terms of thread v and l the loop terms.  When L is
    // injective over the launch with every two values at least S apart (a
    // mixed-radix test: id coefficients sorted by size, each at least S plus
    // the span of the smaller ones), and the two accesses' element ranges
    // around L(v) fit inside a window narrower than S, no two different
    // threads ever touch one element: the pair cannot race in any kind
    // (Table 2 needs two threads).  In shared memory only the thread ids
    // count (the block's own copy).  Exact: a superset of each thread's
    // elements, guards only removing instances.
    auto threads_disjoint = [&](int a, int b) -> bool {
      const Lin &A = af[a].idx, &B = af[b].idx;
      if (!A.cn.empty() || !B.cn.empty() || d.acc[a].width != d.acc[b].width) return false;
      const bool shared = d.arrays[d.acc[a].arr].space == HGRD_SPACE_SHARED;
      const int nid = shared ? 3 : 6;
      for (int k = 0; k < nid; k++)
        if (A.cv[k] != B.cv[k]) return false;
      // loop-term ranges of each access
      auto lrange = [&](const Lin& L, int64_t* lo, int64_t* hi) {
        *lo = L.c0;
        *hi = L.c0;
        for (size_t l = 0; l < d.loops.size(); l++) {
          if (ub[l] <= 0) return false;
          const int64_t t = L.cv[6 + l] * (ub[l] - 1);
          (t < 0 ? *lo : *hi) += t;
        }
        return true;
      };
      int64_t alo, ahi, blo, bhi;
      if (!lrange(A, &alo, &ahi) || !lrange(B, &blo, &bhi)) return false;
      // L(v1) - L(v2) must avoid [blo - ahi, bhi - alo] for v1 != v2
      const int64_t need = std::max(std::abs(blo - ahi), std::abs(bhi - alo)) + 1;
      std::vector<std::pair<int64_t, int64_t>> t;  // (|coefficient|, range) of the ids that vary
      for (int k = 0; k < nid; k++) {
        if (dims[k] <= 1) continue;
        if (A.cv[k] == 0) return false;  // two threads differing in this id alone meet
        t.push_back({std::abs(A.cv[k]), dims[k]});
      }
      std::sort(t.begin(), t.end());
      __int128 below = 0;  // span of the smaller terms
      for (auto& [c, r] : t) {
        if ((__int128)c < below + need) return false;
        below += (__int128)c * (r - 1);
      }
      return true;
    };

    // Accesses whose byte ranges over the whole launch never meet share no
    // location: no pair in any kind.  Exact: each range holds every element
    // its access can reach (interval arithmetic over the ids, the loop
    // counters and the division and remainder nodes; guards only remove
    // instances).
    auto ranges_disjoint = [&](int a, int b) -> bool {
      const AccInfo &X = B.acc_info[a], &Y = B.acc_info[b];
      const __int128 xlo = (__int128)X.idx_lo * X.width, xhi = (__int128)X.idx_hi * X.width + X.width;
      const __int128 ylo = (__int128)Y.idx_lo * Y.width, yhi = (__int128)Y.idx_hi * Y.width + Y.width;
      return xhi <= ylo || yhi <= xlo;
    };

    // ---- pair rule E (Sec. 6.1 trivially race free; Appendix A scopes)
    // Two instances of one block are ordered unless they share a barrier
    // interval (Sec. 6.1, block barrier; Table 2), so accesses whose interval
    // ranges are disjoint can form no intra-block or intra-warp pair; in
    // shared memory, where every pair is of one block, no pair at all.
    for (int a = 0; a < P.nacc; a++) {
      const AccessDecl& x = d.acc[a];
      if (x.kind != 0) P.wmask |= 1u << a;
      for (int b = 0; b < P.nacc; b++) {
        const AccessDecl& y = d.acc[b];
        if (x.arr != y.arr || (x.kind == 0 && y.kind == 0)) continue;
        int m = 7;
        if (x.kind == 2 && y.kind == 2) m = (x.scope == 0 || y.scope == 0) ? 1 : 0;
        if (d.arrays[x.arr].space == HGRD_SPACE_SHARED) m &= ~1;
        if (acc_ivhi[a] < acc_ivlo[b] || acc_ivhi[b] < acc_ivlo[a]) m &= 1;
        if (m && !af[a].dead && !af[b].dead && (ranges_disjoint(a, b) || threads_disjoint(a, b))) m = 0;
        // acquire-release guards at one global address order a pair when
        // their narrower scope covers its type: always inside a block, across
        // blocks with device scope on both (Sec. 6.5, Table 2, Appendix A).
        // Decided here when every racing instance pair of the two accesses
        // has equal guard elements (both constant and equal, or each access
        // guarded at its own index with equal widths: one location, one
        // element) or none has (two different constants).
        if (m && x.sync_arr >= 0 && x.sync_arr == y.sync_arr && !af[a].dead && !af[b].dead) {
          bool same = false, per_instance = false;
          if (s_own[a] && s_own[b] && x.width == y.width)
            same = true;
          else if (s_const[a] && s_const[b])
            same = sval[a] == sval[b];
          else if ((s_own[a] || s_ids[a]) && (s_own[b] || s_ids[b]))
            per_instance = true;  // elements from the ids or the location: compared per instance pair
          else
            raise(HGRD_EUNSUPPORTED,
                  "an acquire-release guard element must be constant, the access's own index, or affine in "
                  "thread and block ids (no loop counter, division or remainder)");
          if (same) m &= std::min(x.sync_scope, y.sync_scope) == 1 ? 0 : 1;
          if (per_instance) {
            P.lockpair[a] |= 1u << b;
            P.lockpair[b] |= 1u << a;
            P.lockany = 1;
          }
        }
        if ((m & 1) && affine[a] && affine[b] && blocks_disjoint(a, b)) m &= ~1;
        if (m & 1) P.einter[a] |= 1u << b;
        if (m & 6) P.eintra[a] |= 1u << b;
      }
    }
    // guard elements of the accesses decided per instance pair: affine in the
    // ids (evaluated from the key's block and thread), else the access's own
    // element (from the location)
    for (int a = 0; a < P.nacc; a++) {
      if (!P.lockpair[a]) continue;
      DLock& L = P.lock[a];
      L.arr = d.acc[a].sync_arr;
      L.scope = d.acc[a].sync_scope;
      if (s_ids[a]) {
        L.form = LOCK_AFFINE;
        L.c0 = slin[a].c0;
        for (int v = 0; v < 6; v++) L.c[v] = slin[a].cv[v];
      } else {
        L.form = LOCK_OWN;
      }
    }

    // an access that may race with no live access (every partner a read when
    // it reads, two device-scope atomics, or never executed) can be in no
    // witness: its instances are still evaluated and counted, its keys dropped
    {
      uint32_t live = 0;
      for (int a = 0; a < P.nacc; a++)
        if (!P.acc[a].dead) live |= 1u << a;
      for (int a = 0; a < P.nacc; a++)
        if (((P.einter[a] | P.eintra[a]) & live) && !P.acc[a].dead) P.emask |= 1u << a;
    }

    // ---- key layout
    uint64_t cells = 0;
    int nl = 0;
    for (int pass = 0; pass < 2; pass++) {
      if (pass == 1) P.shared_cell_base = cells;
      for (size_t k = 0; k < d.arrays.size(); k++) {
        const bool sh = d.arrays[k].space == HGRD_SPACE_SHARED;
        if (sh != (pass == 1)) continue;
        uint64_t ng = (uint64_t)(bytes[k] / d.arrays[k].granule);
        unsigned __int128 c = sh ? (unsigned __int128)ng * (uint64_t)nblk : ng;
        P.lay_cbase[nl] = cells;
        P.lay_ngran[nl] = ng;
        P.lay_arr[nl] = (int32_t)k;
        P.lay_shared[nl] = sh;
        for (int a = 0; a < P.nacc; a++)
          if (d.acc[a].arr == (int)k) P.acc[a].cbase = cells;
        if ((unsigned __int128)cells + c > ((unsigned __int128)1 << 62)) raise(HGRD_EOVERFLOW, "too many granules");
        cells += (uint64_t)c;
        nl++;
      }
    }
    P.lay_cbase[nl] = cells;
    P.nlay = nl;
    if (ivmin > ivmax) ivmin = ivmax = 0;
    P.ivmin = ivmin;
    P.IVB = ceil_log2((uint64_t)(ivmax - ivmin) + 1);
    P.AB = ceil_log2((uint64_t)P.nacc);
    P.TB = ceil_log2((uint64_t)nthr);
    P.BB = ceil_log2((uint64_t)nblk);
    // warp-barrier intervals matter only where accesses of one warp can sit
    // in different ones (one warp with a single thread has no intra-warp pair)
    if (wvmin > wvmax || nthr < 2) wvmin = wvmax = 0;
    P.wvmin = wvmin;
    P.WVB = ceil_log2((uint64_t)(wvmax - wvmin) + 1);
    if (P.WVB > 16) raise(HGRD_EUNSUPPORTED, "more than 2^16 warp-barrier intervals");
    if (P.WVB && P.IVB + P.WVB > 62) raise(HGRD_EOVERFLOW, "interval ids need more than 62 bits");
    P.PB = P.AB + P.TB + P.WVB + P.BB;
    P.SB = P.WVB ? P.AB + P.TB : P.PB;
    P.RB = ceil_log2(std::max<uint64_t>(cells, 1)) + P.IVB;
    if (P.RB + P.PB > 64) raise(HGRD_EOVERFLOW, "sort key needs more than 64 bits for this binding");
    // key count bound: every live instance of every access, all granules
    unsigned __int128 kmax = 0;
    for (int a = 0; a < P.nacc; a++)
      if (!P.acc[a].dead) kmax += (unsigned __int128)nblk * nthr * (uint64_t)nit * (uint64_t)P.acc[a].G;
    if (kmax >= ((unsigned __int128)1 << 40)) raise(HGRD_EUNSUPPORTED, "more than 2^40 keys");
    B.nkeys_max = (uint64_t)kmax;
    uint64_t nshared_kept = 0;
    for (int a = 0; a < P.nacc; a++) {
      if (P.acc[a].dead || !((P.emask >> a) & 1u)) continue;
      const uint64_t k = (uint64_t)nblk * (uint64_t)nthr * (uint64_t)nit * (uint64_t)P.acc[a].G;
      B.nsort_max_all += k;
      if (!P.acc[a].shared) B.nsort_max_split += k;
      else nshared_kept += k;
    }
    // cell filter: worth a per-cell table when many keys would be sorted and
    // the table (4 B per cell) stays small; the (block, thread) id fits 30 bits
    P.ncells = P.lay_cbase[P.nlay];
    P.cfilter = P.ncells <= (1ull << 23) && P.BB + P.TB <= 30;
    P.cfilter_auto = P.cfilter && B.nsort_max_all >= (1ull << 16);
    // default room for keys of candidate shared bins: all kept shared keys up
    // to 2^24, a sixteenth of them beyond (below 2^32); a check that needs
    // more reports HGRD_ENOMEM with the count
    P.scap = std::min<uint64_t>(std::min<uint64_t>(nshared_kept, 0xffffffffull),
                                std::max<uint64_t>(1ull << 24, nshared_kept / 16));
    // Block-local mode: shared-memory runs never leave their block and a
    // shared-memory race needs two threads of one block in one interval
    // (Table 2), so shared keys can be counted per (granule, interval) bin of
    // their block instead of being sorted with the global ones.  Worth it when
    // a block has several simulated warps to keep one CTA busy; the bins of a
    // block must fit shared memory next to the program and the slot files,
    // the bin table of all blocks must stay at most 2^25 entries, and one
    // block's shared keys must be countable in 32 bits.
    {
      uint64_t sgran = 0;
      for (int li = 0; li < P.nlay; li++)
        if (P.lay_shared[li]) {
          for (int a = 0; a < P.nacc; a++)
            if (d.acc[a].arr == P.lay_arr[li]) P.acc[a].sgbase = (int64_t)sgran;
          sgran += P.lay_ngran[li];
        }
      P.niv = (int32_t)((ivmax - ivmin) + 1);
      P.nsbins = (int64_t)(sgran * (uint64_t)P.niv);
      const int64_t upb = (int64_t)P.wpb * P.nchunk;
      // (only when some shared-array key is written: accesses whose keys are
      // counted, never written, need no bins)
      bool any_shared_live = false;
      for (int a = 0; a < P.nacc; a++) any_shared_live |= !P.acc[a].dead && P.acc[a].shared && ((P.emask >> a) & 1u);
      unsigned __int128 per_block = 0;
      for (int a = 0; a < P.nacc; a++)
        if (!P.acc[a].dead && P.acc[a].shared) per_block += (unsigned __int128)nthr * (uint64_t)nit * (uint64_t)P.acc[a].G;
      const uint64_t smem = sizeof(DProg) + (uint64_t)EXP_THREADS * nslot * (wide ? 8 : 4) +
                            (uint64_t)P.nsbins * 13 + 2048;
      // shared locations with guards decided per instance pair go through the
      // global sort and the exact scan's pairwise check
      bool shared_lock = false;
      for (int a = 0; a < P.nacc; a++) shared_lock |= P.lockpair[a] && P.acc[a].shared;
      P.smode = !P.WVB && !shared_lock && any_shared_live && upb >= 4 && P.nsbins > 0 && P.nsbins <= SBIN_MAX &&
                (unsigned __int128)P.nsbins * (uint64_t)nblk <= ((unsigned __int128)1 << 25) &&
                per_block < 0xffffffffu && smem <= 200 * 1024;
      P.RBG = P.smode ? ceil_log2(std::max<uint64_t>(P.shared_cell_base, 1)) + P.IVB : P.RB;
    }
    // radix passes from bit SB: the run code, and with warp-barrier
    // intervals also the block and warp-interval fields below it
    B.sort_passes = (P.RB + P.PB - P.SB + 7) / 8;
    B.sort_passes_split = (P.RBG + P.PB - P.SB + 7) / 8;
    B.wide = wide;
    // integer operations of evaluating every instance once (the count pass's
    // algorithmic work): a term is one multiply-add, a guard or bound test
    // one compare, a division by a constant three (multiply-high, shift,
    // sign), a remainder two more; per thread the ops fixed for the unit, per
    // thread and loop vector the loop ops, then each live access's guards,
    // index with its two bound tests, and interval
    {
      auto op_cost = [&](const DOp& op) {
        return (uint64_t)op.lin.n + (op.kind == OP_DIV ? 3u : op.kind == OP_MOD ? 5u : 0u);
      };
      uint64_t fixed = 0, per_it = 0;
      for (int k = 0; k < P.nfix; k++) fixed += op_cost(P.ops[k]);
      for (int k = P.nfix; k < P.nfix + P.niter; k++) per_it += op_cost(P.ops[k]);
      for (int a = 0; a < P.nacc; a++) {
        const DAcc& A = P.acc[a];
        if (A.dead) continue;
        per_it += (uint64_t)A.idx.n + 2 + (uint64_t)A.iv.n + (P.WVB ? (uint64_t)A.wv.n + 2 : 0);
        for (int g = 0; g < A.ng; g++) per_it += (uint64_t)P.guard[A.gfirst + g].n + 1;
      }
      B.eval_ops = (uint64_t)nblk * (uint64_t)nthr * (fixed + (uint64_t)nit * per_it);
    }
    d.bound = std::move(bp);
    return HGRD_OK;
  } catch (const Err& e) {
    return fail(e.code, e.msg);
  } catch (const std::exception& e) {
    return fail(HGRD_EPARSE, e.what());
  }
}

// 96 features of the access pair (a, b) of a bound descriptor; see
// hgrd_pair_features for the list
static float sgnlog(double x) { return (float)((x < 0 ? -1 : 1) * std::log2(1.0 + std::fabs(x)) / 16.0); }

void pair_features(const hgrd_desc& d, int a, int b, float* f) {
  const Bound& B = *d.bound;
  const DProg& P = B.prog;
  for (int k = 0; k < HGRD_MLP_IN; k++) f[k] = 0.f;
  const AccInfo* X[2] = {&B.acc_info[a], &B.acc_info[b]};
  for (int s = 0; s < 2; s++) {
    const AccInfo& I = *X[s];
    float* g = f + 32 * s;
    g[I.kind] = 1.f;
    g[3] = (I.kind == 2 && I.scope == 0) ? 1.f : 0.f;
    g[4] = (float)std::log2((double)I.width) / 4.f;
    g[5] = (float)I.shared;
    for (int k = 0; k < NVAR; k++) g[6 + k] = sgnlog((double)I.cv[k]);
    g[16] = I.nnodes / 4.f;
    g[17] = I.nguards / 4.f;
    g[18] = (float)(std::log2(1.0 + (double)(I.idx_hi - I.idx_lo)) / 32.0);
    const double cover = (double)(I.idx_hi - I.idx_lo + 1) / (double)std::max<int64_t>(1, I.maxidx + 1);
    g[19] = (float)std::min(1.0, std::max(0.0, cover));
    g[20] = I.idx_lo < 0 ? 1.f : 0.f;
    g[21] = I.idx_hi > I.maxidx ? 1.f : 0.f;
    g[22] = I.iv_lo == I.iv_hi ? 1.f : 0.f;
    g[23] = (float)std::min<int64_t>(8, std::max<int64_t>(-8, I.iv_lo)) / 8.f;
    g[24] = (I.cv[0] | I.cv[1] | I.cv[2]) == 0 ? 1.f : 0.f;
    g[25] = (I.cv[3] | I.cv[4] | I.cv[5]) == 0 ? 1.f : 0.f;
    g[26] = ((I.cv[6] | I.cv[7] | I.cv[8] | I.cv[9]) == 0 && I.loop_nodes == 0) ? 1.f : 0.f;
    bool cst = I.nnodes == 0;
    for (int k = 0; k < NVAR; k++) cst = cst && I.cv[k] == 0;
    g[27] = cst ? 1.f : 0.f;
    for (int l = 0; l < 4; l++) g[28 + l] = I.cv[6 + l] != 0 ? 1.f : 0.f;
  }
  const AccInfo &A = *X[0], &Bb = *X[1];
  float* h = f + 64;
  h[0] = a == b ? 1.f : 0.f;
  h[1] = (A.iv_lo <= Bb.iv_hi && Bb.iv_lo <= A.iv_hi) ? 1.f : 0.f;
  h[2] = (A.iv_lo == A.iv_hi && Bb.iv_lo == Bb.iv_hi && A.iv_lo == Bb.iv_lo) ? 1.f : 0.f;
  h[3] = (float)((P.einter[a] >> b) & 1u);
  h[4] = (float)((P.eintra[a] >> b) & 1u);
  h[5] = (A.kind != 0 && Bb.kind != 0) ? 1.f : 0.f;
  h[6] = (A.kind == 2 && Bb.kind == 2) ? 1.f : 0.f;
  // the two index ranges in bytes overlap
  const double alo = (double)A.idx_lo * A.width, ahi = (double)A.idx_hi * A.width + A.width;
  const double blo = (double)Bb.idx_lo * Bb.width, bhi = (double)Bb.idx_hi * Bb.width + Bb.width;
  h[7] = (alo < bhi && blo < ahi) ? 1.f : 0.f;
  bool same = A.nnodes == Bb.nnodes && A.width == Bb.width;
  for (int k = 0; k < NVAR; k++) same = same && A.cv[k] == Bb.cv[k];
  h[8] = same ? 1.f : 0.f;
  for (int k = 0; k < NVAR; k++) h[9 + k] = sgnlog((double)(A.cv[k] * A.width - Bb.cv[k] * Bb.width));
  h[19] = (float)std::log2((double)P.nthr) / 10.f;
  h[20] = (float)std::log2((double)P.nblk) / 24.f;
  h[21] = (float)std::log2((double)std::max<int64_t>(1, P.nit)) / 24.f;
  h[22] = P.nacc / 32.f;
  h[23] = (float)std::log2(1.0 + (double)B.array_bytes[A.arr]) / 32.f;
  h[24] = A.shared ? 0.f : 1.f;
  h[25] = A.width == Bb.width ? 1.f : 0.f;
  // smallest thread stride in bytes against the access widths: strides below
  // the width make neighbouring threads overlap
  const double sa = std::fabs((double)A.cv[0] * A.width), sb = std::fabs((double)Bb.cv[0] * Bb.width);
  h[26] = (sa > 0 && sa < A.width) ? 1.f : 0.f;
  h[27] = (sb > 0 && sb < Bb.width) ? 1.f : 0.f;
  h[28] = (A.cv[0] == 0 && A.cv[1] == 0 && A.cv[2] == 0 && A.cv[3] == 0 && A.cv[4] == 0 && A.cv[5] == 0) ? 1.f : 0.f;
  h[29] = (Bb.cv[0] == 0 && Bb.cv[1] == 0 && Bb.cv[2] == 0 && Bb.cv[3] == 0 && Bb.cv[4] == 0 && Bb.cv[5] == 0) ? 1.f
                                                                                                                : 0.f;
  h[30] = (float)std::min(1.0, (std::min(ahi, bhi) - std::max(alo, blo)) / std::max(1.0, std::min(ahi - alo, bhi - blo)));
  if (h[30] < 0) h[30] = 0;
  // the two accesses span the same barrier intervals (a read one interval
  // after the write it pairs with differs here)
  h[31] = (A.iv_lo == Bb.iv_lo && A.iv_hi == Bb.iv_hi) ? 1.f : 0.f;
}

int load_desc(const char* text, size_t len, hgrd_desc** out) {
  try {
    if (!text || !out) raise(HGRD_EINVAL, "null argument");
    std::unique_ptr<hgrd_desc> d(new hgrd_desc());
    parse_desc(*d, std::string(text, len));
    *out = d.release();
    return HGRD_OK;
  } catch (const Err& e) {
    return fail(e.code, e.msg);
  } catch (const std::exception& e) {
    return fail(HGRD_EPARSE, e.what());
  }
}

// ---- host-admissible parameter ranges (the symbolic-parameter mode)
// a*P + c of an AST node when it is affine in at most one parameter P and
// reads no launch dimension, id or loop counter; ok = false otherwise
struct Aff1 {
  bool ok;
  int p;  // parameter index, -1 for a constant
  __int128 a, c;
};
static Aff1 affine1(const hgrd_desc& d, int n, int depth = 0) {
  const Aff1 bad{false, -1, 0, 0};
  if (n < 0 || depth > 256) return bad;
  const AstNode& x = d.ast[n];
  const __int128 LIM = (__int128)1 << 100;
  auto fits = [&](const Aff1& r) { return r.ok && r.a < LIM && r.a > -LIM && r.c < LIM && r.c > -LIM; };
  switch (x.op) {
    case 'n': return {true, -1, 0, x.val};
    case 'p': return {true, (int)x.val, 1, 0};
    case '~': {
      Aff1 u = affine1(d, x.a, depth + 1);
      if (!u.ok) return bad;
      return {true, u.p, -u.a, -u.c};
    }
    case '+':
    case '-': {
      Aff1 u = affine1(d, x.a, depth + 1), w = affine1(d, x.b, depth + 1);
      if (!u.ok || !w.ok || (u.p >= 0 && w.p >= 0 && u.p != w.p)) return bad;
      const __int128 sg = x.op == '+' ? 1 : -1;
      Aff1 r{true, u.p >= 0 ? u.p : w.p, u.a + sg * w.a, u.c + sg * w.c};
      return fits(r) ? r : bad;
    }
    case '*': {
      Aff1 u = affine1(d, x.a, depth + 1), w = affine1(d, x.b, depth + 1);
      if (!u.ok || !w.ok) return bad;
      if (u.p >= 0 && w.p >= 0) return bad;
      const Aff1& k = u.p < 0 ? u : w;  // the constant factor
      const Aff1& v = u.p < 0 ? w : u;
      Aff1 r{true, v.p, v.a * k.c, v.c * k.c};
      return fits(r) ? r : bad;
    }
    default:
      return bad;
  }
}
static __int128 floor_div(__int128 a, __int128 b) {
  __int128 q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}
static __int128 ceil_div(__int128 a, __int128 b) { return -floor_div(-a, b); }

// bounds on each parameter from asserts that constrain it alone
void param_bounds(const hgrd_desc& d, std::vector<__int128>& lo, std::vector<__int128>& hi) {
  const __int128 INF = (__int128)1 << 100;
  lo.assign(d.params.size(), -INF);
  hi.assign(d.params.size(), INF);
  for (const CondDecl& c : d.asserts) {
    Aff1 l = affine1(d, c.lhs), r = affine1(d, c.rhs);
    if (!l.ok || !r.ok || (l.p >= 0 && r.p >= 0 && l.p != r.p)) continue;
    const int p = l.p >= 0 ? l.p : r.p;
    if (p < 0) continue;
    const __int128 a = l.a - r.a, k = r.c - l.c;  // a*P op k
    if (a == 0) continue;
    // a*P <= ub and / or a*P >= lb
    bool has_ub = false, has_lb = false;
    __int128 ub = 0, lb = 0;
    switch (c.op) {
      case '<': has_ub = true; ub = k - 1; break;
      case 'L': has_ub = true; ub = k; break;
      case '>': has_lb = true; lb = k + 1; break;
      case 'G': has_lb = true; lb = k; break;
      case 'E': has_ub = has_lb = true; ub = lb = k; break;
      default: break;
    }
    if (a < 0) {  // divide by a negative coefficient: the sides swap
      std::swap(has_ub, has_lb);
      std::swap(ub, lb);
    }
    if (has_ub) hi[p] = std::min(hi[p], floor_div(ub, a));
    if (has_lb) lo[p] = std::max(lo[p], ceil_div(lb, a));
  }
}

}  // namespace hgrd

extern "C" {

int hgrd_load_desc(const char* text, size_t len, hgrd_desc** out) { return hgrd::load_desc(text, len, out); }

int hgrd_bind_host_params(hgrd_desc* d, const hgrd_binding* b) {
  if (!d) return hgrd::fail(HGRD_EINVAL, "null descriptor");
  return hgrd::bind_desc(*d, b);
}

void hgrd_free_desc(hgrd_desc* d) { delete d; }

int hgrd_desc_params(const hgrd_desc* d, hgrd_param_info* out, uint32_t cap, uint32_t* n) {
  if (!d || !n || (cap && !out)) return hgrd::fail(HGRD_EINVAL, "null argument");
  std::vector<__int128> lo, hi;
  hgrd::param_bounds(*d, lo, hi);
  *n = (uint32_t)d->params.size();
  for (uint32_t i = 0; i < *n && i < cap; i++) {
    hgrd_param_info& x = out[i];
    memset(&x, 0, sizeof(x));
    strncpy(x.name, d->params[i].c_str(), sizeof(x.name) - 1);
    x.has_lo = lo[i] > -((__int128)1 << 62);
    x.has_hi = hi[i] < ((__int128)1 << 62);
    x.lo = x.has_lo ? (int64_t)lo[i] : INT64_MIN;
    x.hi = x.has_hi ? (int64_t)hi[i] : INT64_MAX;
  }
  return HGRD_OK;
}

int hgrd_bound_info(const hgrd_desc* d, uint64_t* n_instances, uint64_t* max_keys) {
  if (!d || !n_instances || !max_keys) return hgrd::fail(HGRD_EINVAL, "null argument");
  if (!d->bound) return hgrd::fail(HGRD_EINVAL, "descriptor is not bound (call hgrd_bind_host_params)");
  *n_instances = d->bound->n_instances;
  *max_keys = d->bound->nkeys_max;
  return HGRD_OK;
}

int hgrd_bound_hash(const hgrd_desc* d, uint64_t* h) {
  if (!d || !h) return hgrd::fail(HGRD_EINVAL, "null argument");
  if (!d->bound) return hgrd::fail(HGRD_EINVAL, "descriptor is not bound (call hgrd_bind_host_params)");
  // FNV-1a over the compiled program (every value the check reads) and the
  // array sizes and granules (the witnesses' byte addresses)
  uint64_t x = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t len) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t k = 0; k < len; k++) x = (x ^ c[k]) * 1099511628211ull;
  };
  const hgrd::Bound& B = *d->bound;
  mix(&B.prog, sizeof(B.prog));
  mix(B.array_bytes.data(), B.array_bytes.size() * sizeof(int64_t));
  mix(B.array_granule.data(), B.array_granule.size() * sizeof(int64_t));
  *h = x;
  return HGRD_OK;
}

const char* hgrd_last_error(void) { return hgrd::g_err.c_str(); }

int hgrd_last_stats(hgrd_stats* s) {
  if (!s) return hgrd::fail(HGRD_EINVAL, "null argument");
  *s = hgrd::g_stats;
  s->cuda_objects_created = hgrd::g_created.load(std::memory_order_relaxed);
  return HGRD_OK;
}

int hgrd_pair_features(const hgrd_desc* d, float* out, uint8_t* pairs, uint32_t cap, uint32_t* n) {
  if (!d || !n || (cap && (!out || !pairs))) return hgrd::fail(HGRD_EINVAL, "null argument");
  if (!d->bound) return hgrd::fail(HGRD_EINVAL, "descriptor is not bound");
  const hgrd::DProg& P = d->bound->prog;
  uint32_t k = 0;
  for (int a = 0; a < P.nacc; a++)
    for (int b = a; b < P.nacc; b++) {
      if (!(((P.einter[a] | P.eintra[a]) >> b) & 1u)) continue;  // never races (Sec. 6.1)
      if (P.acc[a].dead || P.acc[b].dead) continue;
      if (k < cap) {
        hgrd::pair_features(*d, a, b, out + (size_t)k * HGRD_MLP_IN);
        pairs[2 * k] = (uint8_t)a;
        pairs[2 * k + 1] = (uint8_t)b;
      }
      k++;
    }
  *n = k;
  return k > cap ? HGRD_ETRUNCATED : HGRD_OK;
}

int hgrd_debug_divmod(int64_t n, int64_t d, int wide, int64_t* q, int64_t* r) {
  if (!q || !r || d <= 0) return hgrd::fail(HGRD_EINVAL, "bad argument");
  const int N = wide ? 62 : 31;
  const int64_t lim = (int64_t)1 << N;
  if (n <= -lim || n >= lim || d >= lim) return hgrd::fail(HGRD_EINVAL, "outside the method's range");
  hgrd::Magic g = hgrd::make_magic(d, N);
  if (wide) {
    *q = hgrd::magic_div64(n, g);
  } else {
    *q = hgrd::magic_div32((int32_t)n, g);
  }
  *r = n - *q * d;
  return HGRD_OK;
}

}  // extern "C"
