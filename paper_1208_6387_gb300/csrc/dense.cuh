// Dense FP64 building blocks of the pattern set-up (once per pattern; not the per-iteration hot path).
#pragma once
#include "common.cuh"

namespace fetirp {

constexpr int TILE = 64;

// Tile-level structure of a lower-triangular factor stored densely (column-major, ld = npad = nt * TILE).
// nz[I * nt + J] (I >= J) says whether tile (I, J) of L can be nonzero after fill-in.  The per-step work lists
// of the right-looking factorisation are kept on the device so that refactorisation needs no host work.
struct TilePlan {
  int nt = 0;
  std::vector<uint8_t> nz;            // nt * nt
  std::vector<int> col_rows;          // for column J: rows I > J with nz(I, J), concatenated
  std::vector<int> col_off;           // nt + 1
  std::vector<int> row_cols;          // for row I: columns J < I with nz(I, J) (backward-solve lists)
  std::vector<int> row_off;           // nt + 1
  std::vector<int2> pairs;            // for step k: (I, J) with I >= J > k, nz(I,k) && nz(J,k)
  std::vector<int> pair_off;          // nt + 1
  DBuf<int> d_col_rows, d_row_cols;
  DBuf<int2> d_pairs;
  void build(int nt_, const std::vector<uint8_t>& nz0);   // symbolic factorisation (fill) + lists
  void upload(cudaStream_t s);
};

// A <- L (lower, in place) with zero-pivot detection: a pivot p_j <= tol * diag0[j] (or not finite) marks
// dof j as a zero pivot: zp[j] = 1 and column j of L is set to 0.  diag0 holds the diagonal before
// factorisation.  Rows of zero-pivot dofs are zeroed at the end, so L is the Cholesky factor of the
// nonsingular block K_rr embedded with zeros (the generalized inverse of Sec. 2).
void chol_tiles(double* A, int npad, const TilePlan& plan, const double* diag0, int* zp, double tol,
                cudaStream_t s);

// X <- L^{-1} X (trans = false) or X <- L^{-T} X (trans = true), X column-major npad x nrhs (ld = ldx),
// zero-pivot rows of the result set to 0.  Right-looking over tile columns, skipping zero tiles.
// Dinv (optional): inverted diagonal tiles from tile_inverses(); each diagonal step is then a parallel product.
// identity_rhs (forward solves only): X holds the identity on entry, so in step J only the first 64 (J + 1)
// columns can be nonzero (L^{-1} is lower triangular) and the others are skipped: a third of the work.
// stop_tile (backward solves only): only the block rows J >= stop_tile of the solution are wanted; each of them
// depends on later block rows only, so the sweep stops there and updates no earlier block row (X above
// stop_tile is left partly updated).
// start_tile (forward solves only): the block rows J < start_tile of X are zero on entry (a right-hand side that
// lives on the trailing block rows), so they stay zero and the sweep starts at start_tile.
void tri_solve(const double* L, int npad, const TilePlan& plan, const int* zp, double* X, int ldx, int nrhs,
               bool trans, cudaStream_t s, const double* Dinv = nullptr, bool identity_rhs = false,
               int stop_tile = 0, int start_tile = 0);
// C (n_out x n_out, ld ldc) = X^T X for a lower-triangular X (column-major, ld, krows rows summed).
void lauum(const double* X, int ld, int krows, int n_out, double* C, int ldc, cudaStream_t s);
// Dinv (npad/64 tiles of 64 x 64, column-major) = inverses of the diagonal tiles of L (zero pivots -> 0).
void tile_inverses(const double* L, int npad, const int* zp, double* Dinv, cudaStream_t s);

// C(m, n) = alpha * sum_k A(m, k) B(k, n) + beta * C(m, n) with arbitrary element strides:
// A(m, k) = A[m * sAm + k * sAk], B(k, n) = B[k * sBk + n * sBn], C(m, n) = C[m * sCm + n * sCn].
// FP64 arithmetic.  Generic (set-up and small coarse products).  A skinny product (fewer 32 x 32 output tiles
// than SMs, a long reduction) splits its reduction dimension over more CTAs when the caller passes scratch of at
// least gemm_f64_scratch(M, N, K) doubles (stream-ordered: reusable by the next call on the same stream), and
// not inside a stream capture; the partials are added in a fixed order.
size_t gemm_f64_scratch(int M, int N, int K);
void gemm_f64(int M, int N, int K, double alpha, const double* A, long long sAm, long long sAk,
              const double* B, long long sBk, long long sBn, double beta, double* C, long long sCm,
              long long sCn, cudaStream_t s, double* scratch = nullptr, size_t scratch_elems = 0);

void copy_diag(const double* A, int npad, double* diag, cudaStream_t s);
void zero_zp_rows(double* A, int npad, const int* zp, cudaStream_t s);

}  // namespace fetirp
