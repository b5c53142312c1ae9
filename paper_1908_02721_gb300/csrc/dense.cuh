// Dense FP64 linear algebra of the TT-rounding stage (S7-S11).
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"

namespace fasttt {

// C(i,j) = alpha * sum_k A(i,k) B(k,j) + beta * C(i,j) with element strides, to
// FP64 accuracy.  sym = true: C is known to be symmetric (square, row-major, scj = 1,
// leading dimension sci >= N);
// only tiles on or above the diagonal are computed and the lower triangle is
// mirrored.  A(i,k) = A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj],
// C(i,j) = C[i*sci + j*scj].  Large products run on the tensor cores (exact bf16
// slices, gemm_ozaki with 7 slices) unless the engine is set to DFMA; the rest,
// and any product the tensor path declines, on gemm_f64_dfma.
void gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
              const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
              cudaStream_t s, bool sym = false);

// The same product with FP64 DFMA (64 x 64 x 16 shared-memory tiles).
void gemm_f64_dfma(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
                   const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
                   cudaStream_t s, bool sym = false);

// The product on the tcgen05 tensor cores from exact bf16 slices of the operands
// (gemm_ozaki.cu): slices = 7 gives FP64-level products (8 slices of 7 bits), 3
// FP32-level (3 slices of 8 bits).  Returns false (C untouched) when the shape does
// not apply.  A kernel that gives up on a bounded wait sets a sticky device flag;
// ozaki_take_timeout reads and clears it and fails with FASTTT_ETIMEOUT if set.
bool gemm_ozaki(int slices, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai,
                int64_t sak, const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci,
                int64_t scj, cudaStream_t s, bool sym = false);

void ozaki_take_timeout(cudaStream_t s);
// Reads and clears the sticky flag without throwing; true if it was set.
bool ozaki_clear_timeout(cudaStream_t s);

// Products below this many multiply-adds stay on the DFMA / mma.sync kernels.
constexpr double kTensorGemmMin = 4194304.0;   // 2^22

// The same product as gemm_f64 on the tensor cores: split-TF32 operands (3
// products), FP32 accumulation, FP64 in and out.  FP32-level accuracy.
void gemm_tf32x3(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
                 const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
                 cudaStream_t s, bool sym = false);

// gemm_f64 or, with mixed = true, an FP32-level product: the tcgen05 kernel on 3
// exact bf16 slices for large products, split-TF32 mma.sync otherwise.
inline void gemm(bool mixed, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai,
                 int64_t sak, const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci,
                 int64_t scj, cudaStream_t s, bool sym = false) {
  if (!mixed) {
    gemm_f64(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym);
    return;
  }
  if (gemm_engine() == 0 && (double)M * (double)N * (double)K >= kTensorGemmMin &&
      gemm_ozaki(3, M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym))
    return;
  gemm_tf32x3(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym);
}

// One-sided Jacobi SVD (Hestenes) of the column-major m x n A (leading dimension
// lda): on return A V has orthogonal columns (A <- A V) and V (nv x n, column-major,
// ldv; identity on entry) holds the rotations.  Returns the sweeps; ETIMEOUT when
// the sweep bound is reached.
int64_t jacobi_svd_f64(double* A, int64_t m, int64_t lda, int n, double* V, int64_t nv, int64_t ldv,
                       int64_t max_sweeps, cudaStream_t s);

// The same result for a tall A (lg >= 1024, n <= kMaxTsqrCols) through Householder
// TSQR (tsqr.cu): Jacobi on the stacked R factors only (at most 4n x n), then
// A <- Q (R V).  A is lg x n column-major with leading dimension lg.
constexpr int kMaxTsqrCols = 128;
bool tsqr_applies(int64_t lg, int n);
int64_t tsqr_jacobi(double* A, int64_t lg, int n, double* V, int64_t max_sweeps, cudaStream_t s);

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
// mixed = true: the Gram and the projections are FP32-level tensor-core products
// (3 exact bf16 slices, or split TF32 for small products), the Gram's eigenpairs
// from the FP32 start refined with FP32-level products, and the bond is redone with
// FP64-level products when that level cannot decide its rank; the direct route
// stays FP64.
// ortho = 1 (left): U must come out orthonormal; 2 (right): the rows of Vt must.
// In mixed precision the factor that the tall-side product amplifies by
// sigma_1 / sigma_r is re-orthonormalised by CholeskyQR (FP64 Cholesky) and its
// partner recomputed (the re-orthogonalisation that keeps FP32-level products usable).
void svd_truncated(const double* Z, int64_t M, int64_t N, const std::function<int64_t(const std::vector<double>&)>& choose_rank,
                   int64_t max_sweeps, SvdOut& out, cudaStream_t s, bool mixed = false, int ortho = 0);

// Eigendecomposition of the symmetric n x n G (row-major FP64) by Householder
// tridiagonalisation, multisection and inverse iteration (tridiag.cu).  V (n x n)
// receives eigenvector j in V[j*n .. j*n + n), lam_out the eigenvalues.  mixed:
// the back-transformation GEMMs run at FP32 level.  Returns false (V undefined)
// when the route does not apply or its vectors could not be made orthonormal.
// need (optional): called with the eigenvalues (ascending) before any eigenvector is
// formed, returns how many of the largest are wanted; only their vectors are computed
// (the other rows of V are zero).  kmax > 0 (with need): need asks for kmax or fewer
// when the kmax largest eigenvalues are exact, so only those are computed; the others
// are all set to their mean (the trace of T less the computed ones, capped at the
// smallest computed one), which keeps every sum of the smallest eigenvalues from the
// n - kmax smallest up exact.  If need asks for more, the rest are computed.
bool sym_eig_tridiag(const double* G, int n, double* V, std::vector<double>& lam_out, cudaStream_t s, bool mixed,
                     const std::function<int64_t(const std::vector<double>&)>& need = nullptr, int64_t kmax = 0);

// The FP32 start of the fast eigensolver (tridiag.cu): G scaled by a power of
// two and rounded to FP32, FP32 Householder tridiagonalisation, bisection and
// inverse iteration (subspace iteration with Gram-Schmidt on clusters of close
// eigenvalues), back-transformation with FP32-level products.  V (row j = an
// approximate eigenvector, FP64 storage) and approximate eigenvalues; false when
// the route does not apply (a cluster larger than it handles, no cooperative launch).
bool sym_eig_start_f32(const double* G, int n, double* V, std::vector<double>& lam_out, cudaStream_t s);

// Fast eigensolver: sym_eig_start_f32, then the Ogita-Aishima refinement with
// FP64-level tensor-core products (mixed: FP32-level) and a Rayleigh-Ritz step on
// runs of close eigenvalues.  Same layout as sym_eig_tridiag; false when a step
// declines (the caller takes the FP64 tridiagonal route).
bool sym_eig_fast(const double* G, int n, double* V, std::vector<double>& lam_out, int64_t max_sweeps, cudaStream_t s,
                  bool mixed);

// The iterative eigensolver of the Gram route (FP32 Jacobi start, Ogita-Aishima
// refinement, FP64 one-sided Jacobi polish); same layout as sym_eig_tridiag.
void sym_eig_iterative(const double* G, int n, double* V, std::vector<double>& lam_out, int64_t max_sweeps,
                       cudaStream_t s);

// The left singular factor of a matrix Z (M x N) given only its Gram Z Z^T
// (M x M, symmetric): eigenvectors of the Gram as in svd_truncated's Gram route,
// the min(M, N) singular values sqrt(max(lambda, 0)) descending (the other
// eigenvalues are zero), r = choose_rank of those.
// Fills out.r, out.sigma_all, out.sigma and out.U (M x r); out.Vt stays empty.
// kcap > 0: no rank above kcap will be kept (a rank cap); when it is at most a quarter of
// M, the FP64 tridiagonal route with only the kept eigenvectors goes first, and with
// partial = true it computes only the kcap + 16 largest eigenvalues (out.sigma_all then
// holds the mean of the others in their place: exact tail sums, not the values).
void svd_from_gram(const double* Gram, int64_t M, int64_t N,
                   const std::function<int64_t(const std::vector<double>&)>& choose_rank, int64_t max_sweeps,
                   SvdOut& out, cudaStream_t s, bool mixed = false, int64_t kcap = 0, bool partial = false);

// ---------------------------------------------------------------- chol.cu

// Upper Cholesky factor of the symmetric n x n row-major H in place (H = R^T R,
// strict lower triangle zeroed), FP64 with FP64-level GEMM updates.  False when
// a pivot is not above tiny_rel * max_i H_ii (or not finite).
bool cholesky_upper(double* H, int64_t n, double tiny_rel, cudaStream_t s);

// R^T X = B in place for the n x n upper R (row-major) and B (n rows x ncols,
// row stride ldb), by substitution (recursive; the off-diagonal updates are
// GEMMs, FP32-level when mixed).
void trsm_upper_t(const double* R, int64_t n, double* B, int64_t ldb, int64_t ncols, bool mixed, cudaStream_t s);

// V (n x n row-major) <- I.
void identity_f64(double* V, int64_t n, cudaStream_t s);

// Gram-route bonds of the mixed precision that kept their FP32-level result, and
// those redone with FP64-level products, since the library was loaded.
int64_t mixed_bonds_kept();
int64_t mixed_bonds_escalated();

// ||H - I||_F of the n x n row-major H.
double identity_deviation(const double* H, int64_t n, cudaStream_t s);

// CholeskyQR2 of the rows of Z (M x N row-major, M <= N): Z <- Q with orthonormal
// rows and, when R is not null, R (M x M row-major upper) with Z_in = R^T Q.  The
// Grams and the solve updates are FP32-level products when mixed; the Cholesky
// factorisations and R = R2 R1 are FP64.  False (Z undefined) on a Cholesky
// breakdown or when the second Gram is further than 0.5 from I (Z too ill
// conditioned for the Gram's precision); dev_out gets that distance.  Without R
// (a re-orthonormalisation) and with ||Z Z^T - I||_F <= 0.1, one pass suffices:
// Z <- R1^-T Z as one GEMM.
bool cholqr2_rows(double* Z, int64_t M, int64_t N, double* R, bool mixed, cudaStream_t s, double* dev_out = nullptr);

// The columns of the row-major rows x r matrix U made orthonormal by CholeskyQR2
// (through its transpose); false as cholqr2_rows.
bool orthonormalise_cols_cholqr2(double* U, int64_t rows, int64_t r, bool mixed, cudaStream_t s);

// Estimate of ||G~ - G||_F for a Gram G~ of Z (Z^T Z when M >= N, else Z Z^T)
// that was formed with FP32-level products: the mean of ||(G~ - G) x||^2 over
// four +-1 probe vectors x (an unbiased estimate of the squared Frobenius norm),
// G x taken as Z^T (Z x) or Z (Z^T x) in FP64.
double gram_error_probe(const double* Z, int64_t M, int64_t N, const double* G, cudaStream_t s);

}  // namespace fasttt
