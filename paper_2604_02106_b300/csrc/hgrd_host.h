// Host-side library state: parsed descriptors and their bindings.
#pragma once
#include <atomic>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "hgrd_internal.h"

struct AstNode {
  char op;  // n num, v instance var (val = slot), d launch dim (val 0..5), p param (val = index), ~ neg, + - * / %
  int64_t val = 0;
  int a = -1, b = -1;
  bool varies = false;  // depends on thread, block or loop ids
  bool thread = false;  // depends on thread or block ids
};
struct CondDecl {
  int lhs = -1, rhs = -1;
  char op = '<';  // < L(<=) > G(>=) E(==) N(!=)
};
struct LoopDecl {
  std::string name;
  int bound = -1;
};
struct ArrayDecl {
  std::string name;
  int space = HGRD_SPACE_GLOBAL;
  int bytes = -1;
  int64_t granule = 0;
};
struct AccessDecl {
  int kind = 0;  // 0 read, 1 write, 2 atomic
  int arr = -1;
  int64_t width = 0;
  int scope = 1;  // 0 block, 1 device (atomics)
  int idx = -1, iv = -1, wv = -1;  // wv: warp-barrier interval (Sec. 5.2)
  int sync_arr = -1, sync = -1;    // acquire-release guard (Sec. 6.5): global array and element
  int sync_scope = 1;              // 0 block, 1 device (the narrower of the guard's parts)
  int line = 0;
  std::vector<CondDecl> guards;
};

namespace hgrd {
// What the ranker's features need about one bound access.
struct AccInfo {
  int kind = 0, scope = 1, arr = 0, shared = 0;
  int64_t width = 4, G = 1;
  int64_t cv[NVAR] = {};  // folded coefficients on tx ty tz bx by bz and the loop counters
  int nnodes = 0, nguards = 0, loop_nodes = 0, dead = 0;
  int64_t idx_lo = 0, idx_hi = 0, maxidx = 0, iv_lo = 0, iv_hi = 0;
};

// Result of hgrd_bind_host_params: the compiled program and host facts.
struct Bound {
  uint64_t gen = 0;  // process-unique id of this binding (keys the cached check graphs)
  std::vector<AccInfo> acc_info;
  DProg prog;
  std::vector<int64_t> array_bytes, array_granule;
  uint64_t n_instances = 0;
  uint64_t nkeys_max = 0;
  // bounds of the keys the global sort sees: written keys of every access
  // (one sort of everything) or of global-array accesses (block-local mode)
  uint64_t nsort_max_all = 0, nsort_max_split = 0;
  uint64_t eval_ops = 0;  // integer operations of evaluating every instance once
  mutable uint64_t eval_ops_jit = 0;  // the same on the specialised kernels (0: not computed yet)
  int sort_passes = 0;        // radix passes over all keys
  int sort_passes_split = 0;  // radix passes over the global-array keys (block-local mode)
  bool wide = false;
  // specialised expansion modules of the plain [0] and block-local [1]
  // pipelines, once tried (owned by the process cache)
  mutable const void* jit[2] = {nullptr, nullptr};
};
extern thread_local std::string g_err;
extern thread_local hgrd_stats g_stats;
// CUDA objects and buffers the library has created since it was loaded
// (streams, events, instantiated graphs, pinned host buffers, loaded
// modules); reported in hgrd_stats.cuda_objects_created
extern std::atomic<uint64_t> g_created;
inline void note_created(uint64_t n = 1) { g_created.fetch_add(n, std::memory_order_relaxed); }
int fail(int code, const std::string& msg);
}  // namespace hgrd

struct hgrd_desc {
  std::string name;
  std::vector<AstNode> ast;
  std::vector<std::string> params;
  std::vector<LoopDecl> loops;
  std::vector<ArrayDecl> arrays;
  std::vector<AccessDecl> acc;
  std::vector<CondDecl> asserts;
  std::map<std::string, int> lets;
  std::unique_ptr<hgrd::Bound> bound;
};
