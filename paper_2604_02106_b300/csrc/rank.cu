// Ranked check: the learned ranker orders the access pairs of a bound kernel,
// a restricted exact check of the top-ranked pairs' accesses runs first and
// stops at its first confirmed race; only when it finds none does the full
// exhaustive check run.  Races are pairwise, so a race found among a subset
// of the accesses is a race of the kernel; a race-free verdict always comes
// from the full scan.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <string>
#include <vector>

#include "hgrd_host.h"

namespace hgrd {
void pair_features(const hgrd_desc& d, int a, int b, float* f);
bool small_single_ok(const Bound& B, uint32_t only);
}

using namespace hgrd;

namespace {
constexpr uint32_t MAXPAIRS = 32 * 33 / 2;
size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
size_t rank_extra() {
  return a256((size_t)MAXPAIRS * HGRD_MLP_IN * 4) + a256((size_t)MAXPAIRS * 4) + a256(hgrd_mlp_workspace_bytes(MAXPAIRS));
}
}  // namespace

extern "C" {

int hgrd_ranked_workspace_size(const hgrd_desc* d, const hgrd_check_opts* o, size_t* bytes) {
  size_t b = 0;
  int rc = hgrd_workspace_size(d, o, &b);
  if (rc) return rc;
  *bytes = a256(b) + rank_extra();
  return HGRD_OK;
}

int hgrd_check_ranked(const hgrd_desc* d, const hgrd_check_opts* o, const void* d_model, const float* host_scores,
                      uint32_t topk, float min_score, void* d_ws, size_t ws_bytes, void* stream,
                      hgrd_witness* host_out, uint64_t cap, hgrd_verdict* v, hgrd_rank_info* info) {
  if (!d || !v || !d_ws) return fail(HGRD_EINVAL, "null argument");
  if (!d->bound) return fail(HGRD_EINVAL, "descriptor is not bound");
  size_t need = 0, base = 0;
  int rc = hgrd_ranked_workspace_size(d, o, &need);
  if (rc) return rc;
  if (ws_bytes < need) return fail(HGRD_ENOMEM, "workspace too small: need " + std::to_string(need));
  rc = hgrd_workspace_size(d, o, &base);
  if (rc) return rc;
  base = a256(base);
  cudaStream_t s = (cudaStream_t)stream;
  hgrd_rank_info inf{};
  auto t0 = std::chrono::steady_clock::now();
  // a check small enough for one CTA costs about what a restricted check
  // would: no ranking, straight to the full check
  const uint32_t fl = o ? o->flags : 0u;
  const bool one_cta = !(fl & (HGRD_NO_SMALL | HGRD_JIT)) && small_single_ok(*d->bound, 0u);
  // 1. eligible pairs and their scores (features and scores staged in pinned
  // host buffers kept per thread)
  static thread_local float* feat = nullptr;
  static thread_local float* zs = nullptr;
  if (!feat) {
    note_created(2);
    if (cudaMallocHost((void**)&feat, (size_t)MAXPAIRS * HGRD_MLP_IN * 4) != cudaSuccess ||
        cudaMallocHost((void**)&zs, (size_t)MAXPAIRS * 4) != cudaSuccess) {
      if (feat) cudaFreeHost(feat);
      feat = nullptr;
      return fail(HGRD_EDEVICE, "pinned staging buffers");
    }
  }
  std::vector<uint8_t> ab(2 * MAXPAIRS);
  uint32_t np = 0;
  if ((d_model || host_scores) && !one_cta) {
    rc = hgrd_pair_features(d, feat, ab.data(), MAXPAIRS, &np);
    if (rc < 0) return rc;
  }
  inf.n_pairs = np;
  // the accesses of every eligible pair: the only ones that can race
  uint32_t cover = 0;
  for (uint32_t k = 0; k < np; k++) cover |= (1u << ab[2 * k]) | (1u << ab[2 * k + 1]);
  // with at most top-k pairs every pair is checked first: no scores needed
  const bool all_pairs = np && np <= topk;
  std::vector<float> score(np, 0.f);
  if (all_pairs) {
  } else if (np && host_scores) {
    std::copy(host_scores, host_scores + np, score.begin());
  } else if (np && d_model) {
    char* w = (char*)d_ws + base;
    float* dx = (float*)w;
    float* dz = (float*)(w + a256((size_t)MAXPAIRS * HGRD_MLP_IN * 4));
    void* mws = w + a256((size_t)MAXPAIRS * HGRD_MLP_IN * 4) + a256((size_t)MAXPAIRS * 4);
    if (cudaMemcpyAsync(dx, feat, (size_t)np * HGRD_MLP_IN * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(HGRD_EDEVICE, "feature upload failed");
    rc = hgrd_mlp_predict(d_model, dx, np, dz, mws, hgrd_mlp_workspace_bytes(MAXPAIRS), s);
    if (rc) return rc;
    if (cudaMemcpyAsync(zs, dz, (size_t)np * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(HGRD_EDEVICE, "score download failed");
    std::copy(zs, zs + np, score.begin());
  }
  inf.ms_rank = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  hgrd_check_opts oo{};
  if (o) oo = *o;
  oo.flags |= HGRD_NO_PAIR | HGRD_STOP_FIRST;
  // 2. restricted check of the accesses of the top-k pairs
  const float best = np ? *std::max_element(score.begin(), score.end()) : 0.f;
  if (np && (d_model || host_scores) && topk && (all_pairs || best >= min_score)) {
    std::vector<uint32_t> ord(np);
    std::iota(ord.begin(), ord.end(), 0u);
    std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) { return score[x] > score[y]; });
    uint32_t mask = 0;
    for (uint32_t k = 0; k < std::min(topk, np); k++) mask |= (1u << ab[2 * ord[k]]) | (1u << ab[2 * ord[k] + 1]);
    inf.access_mask = mask;
    oo.only_accesses = mask;
    rc = hgrd_check(d, &oo, d_ws, base, stream, host_out, cap, v);
    if (rc < 0) return rc;
    inf.keys_ranked = v->n_keys;
    if (v->racy) {
      inf.stage = 1;
      v->n_instances = d->bound->n_instances;
      if (info) *info = inf;
      return rc;
    }
    // the checked accesses cover every eligible pair: no race anywhere (an
    // access in no eligible pair races with nothing, Sec. 6.1)
    if (mask == cover) {
      inf.stage = 2;
      v->n_instances = d->bound->n_instances;
      if (info) *info = inf;
      return rc;
    }
  }
  // 3. the full exhaustive check (stops at its first race)
  oo.only_accesses = 0;
  rc = hgrd_check(d, &oo, d_ws, base, stream, host_out, cap, v);
  if (rc < 0) return rc;
  inf.keys_full = v->n_keys;
  inf.stage = 2;
  if (info) *info = inf;
  return rc;
}

}  // extern "C"
