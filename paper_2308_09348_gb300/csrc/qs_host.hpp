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

}  // namespace detail
}  // namespace qs
