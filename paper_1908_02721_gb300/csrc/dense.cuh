// Dense FP64 linear algebra of the TT-rounding stage (S7-S11).
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"

namespace fasttt {

// C(i,j) = alpha * sum_k A(i,k) B(k,j) + beta * C(i,j) with element strides.
// sym = true: C is known to be symmetric (square, row-major); only tiles on or
// above the diagonal are computed and the lower triangle is mirrored.
// A(i,k) = A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj], C(i,j) = C[i*sci + j*scj].
void gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
              const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
              cudaStream_t s, bool sym = false);

// dst (cols x rows, row-major) = transpose of src (rows x cols, row-major)
void transpose_f64(const double* src, int64_t rows, int64_t cols, double* dst, cudaStream_t s);

// Truncated SVD of a row-major M x N matrix Z.  `choose_rank` receives the
// singular values (descending, min(M,N) of them, on the host) and returns r.
// On return: U (M x r row-major), sigma (r), Vt (r x N row-major), all device.
struct SvdOut {
  int64_t r = 0;
  std::vector<double> sigma_all;  // every computed singular value, descending
  DBuf<double> U, sigma, Vt;
  int64_t sweeps = 0;
};
void svd_truncated(const double* Z, int64_t M, int64_t N, const std::function<int64_t(const std::vector<double>&)>& choose_rank,
                   int64_t max_sweeps, SvdOut& out, cudaStream_t s);

}  // namespace fasttt
