// dict.cuh -- launch paths of the dictionary statistics (Section 4.2) and of
// the nonzero list of Z, shared by the files that drive them.
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

// The nonzeros of Z in (position, atom) order into caller arrays of cap
// entries (the same compaction); *nnz_out = their number (read back: one
// synchronisation).
int sparse_code_impl(const Geom &g, const float *Z, int *k_out, int *s_out, float *val_out, long long cap,
                     long long *nnz_out, unsigned char *ws, const WsLayout &L, cudaStream_t st);

}  // namespace csc
