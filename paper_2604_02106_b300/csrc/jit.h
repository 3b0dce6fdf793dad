// Specialised expansion kernels compiled at run time (jit.cpp).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "hgrd_host.h"
#include "kernels.cuh"

namespace hgrd {

// CUDA source of the specialised expansion kernels for the program's
// structure: the count and write kernels of the block-local pipeline (split)
// or of the plain one
std::string jit_source(const DProg& P, bool split);
// compile (or find in the process cache) the kernels for B; *ms = compile time
// spent by this call.  HGRD_EUNSUPPORTED with the compiler's log on failure.
int jit_prepare(const Bound& B, bool split, double* ms);
// integer operations of the specialised count pass (loop-invariant and
// ranged accesses taken once per thread, the others per loop vector)
uint64_t jit_eval_ops(const DProg& P);
// whether B already holds loaded kernels for the pipeline
bool jit_ready(const Bound& B, bool split);
// one expansion launch (mode 0..4) on the specialised kernels of B's plain
// or block-local (split) module; mode 2 (pair search) is in both
cudaError_t launch_jit_expand(const Launch& L, const Bound& B, int mode, const DProg& h_prog, uint64_t* unit_cnt,
                              const uint64_t* unit_off, uint64_t* keys_g, uint64_t* keys_s, uint64_t* hist, int npass,
                              uint64_t* counters, uint64_t* stbl, uint64_t* sbase, uint32_t only, bool split,
                              const uint64_t* uniq = nullptr, PairRec* pairs = nullptr, uint64_t pair_cap = 0,
                              const uint32_t* ctab = nullptr, uint64_t* cbuf = nullptr, uint64_t ccap = 0);

}  // namespace hgrd
