// Host-side launchers of the reverse-mode kernels (adjoint.cuh).
#pragma once

#include "adjoint.cuh"
#include "launch.h"

namespace mpa {

template <typename T> cudaError_t kca_launch(int mode, int logL, const KCAParams<T>& p, cudaStream_t st);
template <typename T> cudaError_t kra_launch(int logL, const KRAParams<T>& p, cudaStream_t st);
// The forward row pass (KR_MPA) that also writes A(t) to p.keep.
template <typename T> cudaError_t kr_keep_launch(int logL, const KRParams<T>& p, cudaStream_t st);
template <typename T> cudaError_t rscan_launch(const RScanParams<T>& p, cudaStream_t st);
template <typename T>
cudaError_t scan_store_launch(const cx<T>* v, cx<T>* psi, const cx<T>* psi0c, long long N, int M, cudaStream_t st);
template <typename T>
cudaError_t scale_to_state_launch(const cx<T>* in, double2* state, double scale, long long N, cudaStream_t st);
cudaError_t reduce_parts_launch(const double* part, int per, int n, double* acc, cudaStream_t st);

template <typename T> cudaError_t ssc_launch(int mode, int logL, const SSCParams<T>& p, cudaStream_t st);
template <typename T> cudaError_t ssr_launch(int mode, int logL, const SSRParams<T>& p, cudaStream_t st);

// Tile widths of the reverse passes (columns per column tile, rows per row tile).
template <typename T> int kca_tile_cols(int logL);
template <typename T> int kra_tile_rows(int logL);

}  // namespace mpa
