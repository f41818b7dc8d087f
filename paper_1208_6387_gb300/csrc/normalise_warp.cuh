// One-warp F-normalisation of a k x k block (k <= 32), shared by the stand-alone normalisation kernel and
// the persistent block iteration.
#pragma once
#include "ops.cuh"

namespace fetirp {

// Pivoted factorisation, triangular inverse and outputs of k_normalise for k <= 32 by one warp.  On this GPU a
// dependent FP64 operation costs ~64 cycles and a divide or square root 450-700, so the serial chain is kept
// short: the square-root-free form eta_P = L D L^T (unit lower L) needs one reciprocal per step, which every
// lane forms for its own diagonal while the argmax runs; the argmax and the threshold test compare the FP64
// bit patterns as integers (positive finite doubles order like their bits); the trailing update is one FMA
// per entry with the multiplier l_ip = a_ip / d_p, and the square roots of D are taken once, in parallel,
// at the end.  M = L D^{1/2} is the pivoted Cholesky factor, so T and
// alpha are those of the block path.  Lane i owns row i of the Schur complement (rows are lane-private; the
// pivot column is broadcast by shuffles); no block-wide barrier is needed.
template <int LD>
__device__ inline void normalise_warp(int k, double (*A)[LD], double (*Lc)[LD], int* piv, double* Dg,
                                      const double* rhs, double trunc, double* __restrict__ T,
                                      double* __restrict__ alpha, int* __restrict__ n_kept) {
  const unsigned FULL = 0xffffffffu;
  const long long FINITE = 0x7FF0000000000000ll;   // bit pattern of +inf: positive finite doubles lie in (0, FINITE)
  const int lane = threadIdx.x & 31;
  const bool own = lane < k;
  double d = own ? A[lane][lane] : 0.0;
  auto key_of = [&](double x, bool ok) {   // ordering key of a candidate pivot; -1 when it cannot be one
    const long long b = __double_as_longlong(x);
    return (ok && b > 0 && b < FINITE) ? b : -1ll;
  };
  long long mk = key_of(d, own);
  for (int o = 16; o > 0; o >>= 1) mk = max(mk, __shfl_xor_sync(FULL, mk, o));
  const double thresh = mk > 0 ? trunc * __longlong_as_double(mk) : 0.0;
  const long long thresh_k = __double_as_longlong(thresh);   // thresh >= 0: integer order is numeric order
  bool done = !own;
  int r = 0;
  if (mk > 0) {
    for (int step = 0; step < k; ++step) {
      const long long key = key_of(d, !done);
      const double rd = 1.0 / d;   // every lane's reciprocal, overlapping the argmax below
      long long best_k = key;
      for (int o = 16; o > 0; o >>= 1) best_k = max(best_k, __shfl_xor_sync(FULL, best_k, o));
      if (best_k < 0 || best_k <= thresh_k) break;
      const int p = __ffs(__ballot_sync(FULL, key == best_k)) - 1;   // ties -> lowest index
      const double rp = __shfl_sync(FULL, rd, p);
      const double aip = own ? A[lane][p] : 0.0;
      const double lip = aip * rp;
      if (lane == p) {
        piv[step] = p;
        Dg[step] = d;
        Lc[p][step] = 1.0;
        done = true;
      } else if (!done) {
        Lc[lane][step] = lip;
      }
#pragma unroll 8
      for (int j = 0; j < k; ++j) {   // A[i][j] -= (A[i][p] / A[p][p]) A[j][p] on the free rows
        const double ajp = __shfl_sync(FULL, aip, j);
        if (!done) A[lane][j] = fma(-lip, ajp, A[lane][j]);
      }
      if (!done) d = fma(-lip, aip, d);
      r = step + 1;
    }
  }
  __syncwarp();
  // Dg <- D^{-1/2} (one square root and divide per lane, in parallel)
  if (lane < r) Dg[lane] = 1.0 / sqrt(Dg[lane]);
  // X = L^{-1} (unit lower r x r, L[a][b] = Lc[piv[a]][b]) by columns in A's storage: lane c starts from e_c and
  // eliminates forward; x_j of its column is final at step j, and only the entries below it change
  if (lane < k)
    for (int l = 0; l < r; ++l) A[l][lane] = (l == lane) ? 1.0 : 0.0;
  for (int j = 0; j < r; ++j) {
    if (lane < r && lane <= j) {
      const double xj = A[j][lane];
#pragma unroll 4
      for (int l = j + 1; l < r; ++l) A[l][lane] = fma(-Lc[piv[l]][j], xj, A[l][lane]);
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
