// Integer grouping stage of FastTT (S1-S5): ingest, Alg. 9 split selection,
// Alg. 4/5 sweeps and the middle unfolding.
#pragma once

#include <vector>

#include "common.cuh"

namespace fasttt {

struct Ingested {
  int d = 0;
  std::vector<int64_t> dims;
  int64_t nnz_in = 0, nnz = 0, dropped = 0;
  DBuf<int32_t> idx;   // (d, nnz) kept entries, SoA
  DBuf<double> vals;   // nnz
  double norm2 = 0.0;
};

// S1: range/finite checks, explicit zeros dropped, values upcast to FP64,
// ||A||^2 by a fixed-order tree.  Throws EINVAL on bad input.
void ingest(int d, const int64_t* dims, int64_t nnz, const int32_t* d_idx, const void* d_vals,
            int val_dtype, Ingested& out, cudaStream_t s);

struct Grouped {
  int p = 0;
  int64_t R = 0;
  std::vector<int64_t> Rs;   // R for p = 1..d (Alg. 9), empty when p was given
  std::vector<int64_t> rt;   // r~_0..r~_d
  // core k < p (index k-1): alpha_{k-1} and i_k of every alpha_k
  std::vector<DBuf<int32_t>> left_parent, left_index;
  // core k > p (index k-p-1): i_k and alpha_k of every alpha_{k-1}
  std::vector<DBuf<int32_t>> right_index, right_child;
  // middle unfolding X (p < d: unfold_2(V), rows (alpha_{p-1}, i_p), cols alpha_p;
  // p = d: unfold_1^T(V), rows i_d, cols alpha_{d-1}), entries sorted by (row, col)
  int64_t mid_rows = 0, mid_cols = 0;
  DBuf<int64_t> mid_row, mid_col;
  DBuf<double> mid_val;
};

// S2-S5.  p_req = 0 runs Alg. 9.  Throws EDUP on a repeated coordinate.
void group(const Ingested& in, int p_req, int64_t max_rank, Grouped& out, cudaStream_t s);

// Alg. 9 on the host: argmin_p of eq. (13) with the bounds of eq. (10).
int select_p_host(const std::vector<int64_t>& dims, const std::vector<int64_t>& Rs, int64_t max_rank);

}  // namespace fasttt
