// Batched apply over independent problems (uneven grids, ragged column counts).
#include "common.cuh"

extern "C" pide_status pide_apply(pide_handle h, const double* b_dev, double* u_dev, int32_t B,
                                  int32_t max_sweeps, double tol, const double* g_dev,
                                  void* stream, pide_info* info);

extern "C" pide_status pide_apply_batched_impl(const pide_handle* hs, int32_t nprob,
                                               const double* const* b, double* const* u,
                                               const int32_t* Bs, int32_t sweeps, void* stream) {
  for (int k = 0; k < nprob; ++k) {
    pide_status s = pide_apply(hs[k], b[k], u[k], Bs[k], sweeps, 0.0, nullptr, stream, nullptr);
    if (s != PIDE_OK) return s;
  }
  return PIDE_OK;
}
