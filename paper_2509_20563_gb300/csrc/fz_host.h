// fz_host.h -- host-side pieces shared by the API translation units: the
// context object and small argument helpers.
#pragma once

#include <vector>

#include "fz_internal.cuh"

namespace fz {
// A cached batched call: the key of its batch shape, the autotuned launch
// shape and, when the sequence could be captured, the instantiated graph.
struct BatchPlan {
  bool decompress = false;
  std::vector<uint64_t> key;
  BatchTune tune{};
  uint32_t chunk[2] = {0, 0};  // compress plans: the chunk of each encode class (0 = class absent)
  cudaGraphExec_t exec = nullptr;
};
}  // namespace fz

struct fz_ctx {
  int device = 0;
  int sm_count = 0;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  void *h_pinned = nullptr;  // host mirror of the call's result block
  // stage profiling (CUDA events on the call's stream)
  bool profiling = false;
  cudaEvent_t cev[FZ_MAX_STAGES + 1] = {};
  cudaEvent_t dev_[FZ_MAX_STAGES + 1] = {};
  const char *cname[FZ_MAX_STAGES] = {};
  const char *dname[FZ_MAX_STAGES] = {};
  uint32_t nc = 0, nd = 0;
  uint64_t launches = 0;
  // batched calls: workspace, pinned job tables / results, capture stream and
  // the cached plans (autotuned launch shapes and instantiated graphs)
  // [0] batched compress, [1] batched decompress: separate, so that neither
  // kind's growth invalidates the other kind's graphs
  void *bws[2] = {nullptr, nullptr};
  size_t bws_bytes[2] = {0, 0};
  void *h_batch[2] = {nullptr, nullptr};
  size_t h_batch_bytes[2] = {0, 0};
  cudaStream_t cap_stream = nullptr;
  std::vector<fz::BatchPlan *> plans;
  bool batch_tuning = true;
  bool batch_graphs = true;
  long long spin_cycles = 0;  // bound of every look-back wait, in clock cycles (0: the library default)
};

namespace fz {

constexpr size_t kAlign = 256;
inline size_t up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

inline fz_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return FZ_OK;
  if (e == cudaErrorMemoryAllocation) return FZ_ENOMEM;
  return FZ_ECUDA;
}

// Validate ndim/dims; fills N.
inline bool valid_dims(uint32_t ndim, const uint64_t *dims, uint64_t *n) {
  if (!dims || ndim < 1 || ndim > 3) return false;
  uint64_t v = 1;
  for (uint32_t a = 0; a < ndim; ++a) {
    if (dims[a] == 0 || dims[a] >= (1ull << 32)) return false;
    v *= dims[a];
    if (v >= (1ull << 32)) return false;
  }
  *n = v;
  return true;
}

inline bool overlaps(const void *a, uint64_t na, const void *b, uint64_t nb) {
  uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

// Defined in fz_api.cu.
size_t layout_compress_split(const Geom &g, char *zbase, char *rbase, CompressWs &ws, size_t *rest_bytes);
fz_status check_header(const fz_header &h, uint64_t in_bytes, Geom &g);
void destroy_batch_plans(fz_ctx *ctx, int kind = -1);  // kind 0 compress, 1 decompress, -1 both

}  // namespace fz
