// Value Depar (S6): Alg. 3 with exact parallelism on the rows, then the
// columns, of the sparse middle unfolding.
#pragma once

#include "common.cuh"

namespace fasttt {

// One Depar pass over the "rows" (major index) of a sparse matrix whose entries
// are sorted by (major, minor).
struct DeparPass {
  int64_t nz = 0;          // nonzero majors
  int64_t beta = 0;        // classes
  DBuf<int64_t> ids;       // nonzero majors, ascending (nz)
  DBuf<int32_t> cls;       // class of each nonzero major (nz)
  DBuf<double> pref;       // prefactor = first nonzero of each major (nz)
  DBuf<double> lam;        // per class: 2-norm of its members' prefactors (beta)
  // class representatives, entries sorted by (class, minor)
  int64_t rep_n = 0;
  DBuf<int32_t> rep_cls;
  DBuf<int64_t> rep_minor;
  DBuf<double> rep_val;    // normalised values (first of each class exactly 1.0)
};

void depar_pass(const int64_t* major, const int64_t* minor, const double* val, int64_t n, DeparPass& out,
                cudaStream_t s);

struct DeparResult {
  DeparPass rows;          // X = S D
  DeparPass cols;          // D = D' T (pass over the columns of D)
  // D' entries (beta_r x beta_c) sorted by (col class, row class):
  // rows.cls-space row index, cols.cls-space column index, value
  int64_t dp_n = 0;
  DBuf<int32_t> dp_row, dp_col;
  DBuf<double> dp_val;
};

// enabled = 0 gives the identity factorisation (every nonzero row / column its
// own class, prefactors 1, Lambda = 1).
void value_depar(const int64_t* row, const int64_t* col, const double* val, int64_t n, int64_t ncols,
                 bool enabled, DeparResult& out, cudaStream_t s);

}  // namespace fasttt
