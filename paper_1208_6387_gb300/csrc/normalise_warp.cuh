// One-warp F-normalisation of a k x k block (k <= 32), shared by the stand-alone normalisation kernel and
// the persistent block iteration.
#pragma once
#include "ops.cuh"

namespace fetirp {

// Pivoted factorisation, triangular inverse and outputs of k_normalise for k <= 32 by one warp.  On this GPU a
// dependent FP64 operation costs ~64 cycles and a divide or square root 450-700, so the serial chain is kept
// short: the square-root-free form eta_P = L D L^T (unit lower L) takes one reciprocal per step, the pivot
// argmax compares the FP64 bit patterns as integers (positive doubles order like their bits), and the square
// roots of D are taken once, in parallel, at the end.  M = L D^{1/2} is the pivoted Cholesky factor, so T and
// alpha are those of the block path.  Lane i owns row i of the Schur complement (rows are lane-private; the
// pivot column is broadcast by shuffles); no block-wide barrier is needed.
template <int LD>
__device__ inline void normalise_warp(int k, double (*A)[LD], double (*Lc)[LD], int* piv, double* Dg,
                                      const double* rhs, double trunc, double* __restrict__ T,
                                      double* __restrict__ alpha, int* __restrict__ n_kept) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool own = lane < k;
  double d = own ? A[lane][lane] : 0.0;
  long long mk = (own && d > 0.0) ? __double_as_longlong(d) : -1ll;
  for (int o = 16; o > 0; o >>= 1) mk = max(mk, __shfl_xor_sync(FULL, mk, o));
  const double thresh = mk > 0 ? trunc * __longlong_as_double(mk) : 0.0;
  bool done = !own;
  int r = 0;
  if (mk > 0) {
    for (int step = 0; step < k; ++step) {
      const long long key = (!done && d > 0.0) ? __double_as_longlong(d) : -1ll;
      long long best_k = key;
      for (int o = 16; o > 0; o >>= 1) best_k = max(best_k, __shfl_xor_sync(FULL, best_k, o));
      if (best_k < 0) break;
      const double best = __longlong_as_double(best_k);
      if (!(best > thresh)) break;
      const int p = __ffs(__ballot_sync(FULL, key == best_k)) - 1;   // ties -> lowest index
      const double rp = 1.0 / best;
      const double aip = own ? A[lane][p] : 0.0;
      if (lane == p) {
        piv[step] = p;
        Dg[step] = best;
        Lc[p][step] = 1.0;
        done = true;
      } else if (!done) {
        Lc[lane][step] = aip * rp;
      }
#pragma unroll 8
      for (int j = 0; j < k; ++j) {   // A[i][j] -= A[i][p] A[j][p] / A[p][p] on the free rows
        const double ajp = __shfl_sync(FULL, aip, j);
        if (!done) A[lane][j] -= (aip * ajp) * rp;
      }
      d = own ? A[lane][lane] : 0.0;
      r = step + 1;
    }
  }
  __syncwarp();
  // Dg <- D^{-1/2} (one square root and divide per lane, in parallel)
  if (lane < r) Dg[lane] = 1.0 / sqrt(Dg[lane]);
  // X = L^{-1} (unit lower r x r, L[a][b] = Lc[piv[a]][b]); lane c forms column c of X in A's storage
  for (int l = 0; l < r; ++l) {
    if (lane < k) {
      double v = 0.0;
      if (lane == l) {
        v = 1.0;
      } else if (lane < l) {
        const double* m = Lc[piv[l]];
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = lane;
        for (; j + 3 < l; j += 4) {
          s0 = fma(m[j], A[j][lane], s0);
          s1 = fma(m[j + 1], A[j + 1][lane], s1);
          s2 = fma(m[j + 2], A[j + 2][lane], s2);
          s3 = fma(m[j + 3], A[j + 3][lane], s3);
        }
        for (; j < l; ++j) s0 = fma(m[j], A[j][lane], s0);
        v = -((s0 + s1) + (s2 + s3));
      }
      A[l][lane] = v;
    }
  }
  // M^{-1} = D^{-1/2} X:  T[piv[a]][c] = dsq[c] X[c][a] for a, c < r, zero elsewhere;
  // alpha[c] = dsq[c] sum_a X[c][a] rhs[piv[a]]
  for (int idx = lane; idx < k * k; idx += 32) T[idx] = 0.0;
  __syncwarp();
  if (lane < r) {
#pragma unroll 8
    for (int c = 0; c < r; ++c) T[(size_t)piv[lane] * k + c] = Dg[c] * A[c][lane];
  }
  if (lane < k) {
    double v0 = 0.0, v1 = 0.0;
    if (lane < r) {
      int a = 0;
#pragma unroll 4
      for (; a + 1 < r; a += 2) {
        v0 = fma(A[lane][a], rhs[piv[a]], v0);
        v1 = fma(A[lane][a + 1], rhs[piv[a + 1]], v1);
      }
      if (a < r) v0 = fma(A[lane][a], rhs[piv[a]], v0);
    }
    alpha[lane] = lane < r ? Dg[lane] * (v0 + v1) : 0.0;
  }
  if (lane == 0) *n_kept = r;
}

}  // namespace fetirp
