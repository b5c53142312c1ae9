// Block-sparse bond of the first SVD sweep (Alg. 6): G_k = W_{k-1} x_1 P_k kept
// as W and the right quasi-permutation maps of Alg. 4 instead of a dense core.
#pragma once

#include <vector>

#include "common.cuh"

namespace fasttt {

class SparseBond {
 public:
  // W: rp x A row-major (column alpha = W_{k-1}[:, alpha]); ridx[alpha] = i_k
  // (nondecreasing), rchild[alpha] = alpha_k in [0, N); every alpha_k occurs.
  SparseBond(const double* W, int64_t rp, int64_t A, const int32_t* ridx, const int32_t* rchild, int64_t nk,
             int64_t N, cudaStream_t s);
  // Gram = Z Z^T (M x M, M = rp * nk) of Z = unfold_2(G_k), row (a, i) = a * nk + i
  void gram(double* Gram, cudaStream_t s) const;
  // W_out = U^T Z (rr x N row-major) for U (M x rr row-major)
  void project(const double* U, int64_t rr, DBuf<double>& W_out, cudaStream_t s) const;

  int64_t rp, A, nk, N;
  const int32_t* ridx;
  DBuf<double> Wt;               // A x rp: column alpha of W contiguous
  DBuf<uint64_t> sorted_keys;    // beta of alpha, sorted (stable)
  DBuf<uint32_t> sorted_vals;    // alpha in that order
  DBuf<int64_t> boff, ioff;      // first sorted position of each beta; first alpha of each i
  std::vector<int64_t> hioff;    // ioff on the host
};

}  // namespace fasttt
