// qs_host.hpp -- host-side helpers shared by the translation units of
// libqscatter: descriptor validation, derived constants, workspace plan.
#pragma once

#include <cstddef>
#include <cstdint>

#include "qscatter.h"
#include "qs_device.cuh"

namespace qs {
namespace detail {

constexpr int kSmemLimit = 227 * 1024;

int32_t validate_laser(const qs_laser* L);
int32_t validate_beam(const qs_beam* B);
int32_t validate_bins(const qs_bins* b);
int32_t validate_samples(const qs_samples* s);
int32_t exec_opts(const qs_exec* e, int* precision, int* wbits, int* block, int* grid);
int32_t exec_tile(const qs_exec* e, int* tile);
// Points p at the cycle-resolved chi tables of the current context, building
// them on first use there (one launch on `st` and a wait; QS_ERR_UNSUPPORTED
// while `st` is being captured).
int32_t cycle_tables(Params& p, cudaStream_t st);
// QS_EXEC_CHECK_FINITE requested?
bool exec_check_finite(const qs_exec* e);
// QS_OK unless `st` is being captured into a graph (QS_ERR_UNSUPPORTED):
// a call that waits for its stream cannot be captured.
int32_t sync_allowed(cudaStream_t st);
// Waits for `st` after copying `count` excluded-sample counts (device
// doubles `stride` bytes apart) to the host: QS_ERR_NONFINITE if any is > 0.
int32_t nonfinite_status(const double* d_nonfinite, int64_t count, size_t stride,
                         cudaStream_t st);
void fill_params(Params& p, const qs_laser* L, const qs_beam* B, const qs_samples* S,
                 const qs_bins* b, int wbits);
int32_t device_sms(int* sms);

// Workspace plan: u64 histogram accumulators (+ under/over/outside slots),
// smoothed-spectrum accumulators, then FP64 partials (kNumMom per CTA) for
// the largest grid that can be resident.
struct Plan {
  int64_t nspec = 0, nmap = 0, naeff = 0, nsmooth = 0;   // accumulator slots
  int gmax = 1;
  size_t ws_bytes = 0;
  size_t off_spec = 0, off_map = 0, off_aeff = 0, off_smooth = 0, off_part = 0;
};
size_t align_up(size_t v, size_t a);
void make_plan(Plan& pl, const qs_bins* b, int block, int grid_req, int sms);

struct Smem {
  size_t bytes = 0;
  bool hist = false;
  bool smooth = false;
};
Smem smem_plan(const Plan& pl, int precision, int cells, int variant, bool weighted, int block);
int pick_grid(int occ_per_sm, int sms, int block, int grid_req, int64_t n, int gmax);

// A failed runtime call: clear the (non-sticky) error state so that it does
// not surface in the caller's next, unrelated CUDA call, and report it.
inline int32_t cuda_fail() {
  (void)cudaGetLastError();
  return QS_ERR_CUDA;
}

// The current device and a key of the current CUDA context, unique for the
// life of the process (the driver's context id, plus one).  What a context
// owns -- the module's __device__ arrays and their contents, kernel
// attributes, streams and events -- is cached under this key, so that after
// a cudaDeviceReset (which destroys the context and reloads the module in
// the next one) the library rebuilds it instead of using stale addresses or
// handles.  Makes the device's primary context current if the calling
// thread has no context yet.
int32_t current_context(int* dev, unsigned long long* key);

// Per-device "done in this context" marks.
struct CtxMark {
  unsigned long long key[64] = {};
  bool done(int dev, unsigned long long k) const { return key[dev] == k; }
  void set(int dev, unsigned long long k) { key[dev] = k; }
};

// Raises kernel f's dynamic shared memory limit to `bytes`, once per
// context (the attribute lives in the context's copy of the module).
template <typename F>
int32_t allow_smem(F f, CtxMark& mark, int bytes) {
  int dev = 0;
  unsigned long long key = 0;
  if (int32_t st = current_context(&dev, &key)) return st;
  if (!mark.done(dev, key)) {
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
        cudaSuccess)
      return cuda_fail();
    mark.set(dev, key);
  }
  return QS_OK;
}

}  // namespace detail
}  // namespace qs
