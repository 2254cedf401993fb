// dict.cuh -- launch paths of the dictionary statistics (Section 4.2) shared
// by the files that drive them.
#pragma once
#include "common.cuh"

namespace csc {

// phi / psi like dict_stats_impl, without reading the nonzero count back:
// the grids cover the list capacity and the kernels take the count from the
// workspace header.  The caller must check header->scan_total against
// WsLayout::nnz_cap after its next synchronisation (above it, phi and psi are
// not valid).
int dict_stats_deferred(const Geom &g, const float *Z, const float *X, float *phi, float *psi,
                        unsigned char *ws, const WsLayout &L, cudaStream_t st);

}  // namespace csc
