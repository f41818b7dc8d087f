// Block Gram products, F-normalisation and the block update of multivector FETI (Table 1 right column: step
// length, iterate and residual updates, with the F-normalisation and full reorthogonalisation of the
// numerical-issues subsection).
#include <mutex>

#include "ds.cuh"
#include "ops.cuh"
#include "normalise_warp.cuh"

namespace fetirp {

// Partial C_chunk = A[rows of chunk]^T B[rows of chunk]; grid (a tiles, b tiles, chunks); FP64 accumulation.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_gram_partial(int n, int a, int b, const TA* __restrict__ A, int lda,
                                                      const TB* __restrict__ B, int ldb, int rows_per_chunk,
                                                      double* __restrict__ partial) {
  __shared__ double sa[16][65];
  __shared__ double sb[16][65];
  const int a0 = blockIdx.x * 64, b0 = blockIdx.y * 64, ch = blockIdx.z;
  const int r0 = ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  double acc[4][4] = {};
  for (int rr = r0; rr < r1; rr += 16) {
    for (int idx = tid; idx < 16 * 64; idx += 256) {
      const int c = idx % 64, q = idx / 64, r = rr + q;
      sa[q][c] = (r < r1 && a0 + c < a) ? (double)A[(size_t)r * lda + a0 + c] : 0.0;
      sb[q][c] = (r < r1 && b0 + c < b) ? (double)B[(size_t)r * ldb + b0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      double av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { av[u] = sa[q][tx * 4 + u]; bv[u] = sb[q][ty * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* P = partial + (size_t)ch * a * b;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = a0 + tx * 4 + u;
    if (i >= a) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = b0 + ty * 4 + v;
      if (j < b) P[(size_t)i * b + j] = acc[u][v];
    }
  }
}

// eta = W^T Q (k x k) and wr = W^T r (k) in one pass, as a k x (k+1) row-major block: grid = row chunks, each
// thread owns outputs idx = tid, tid + 256, ...; chunk partials are added in chunk order afterwards.
__global__ void __launch_bounds__(256) k_eta_partial(int n, int k, const double* __restrict__ W,
                                                     const double* __restrict__ Q, const double* __restrict__ r,
                                                     int rows_per_chunk, double* __restrict__ partial) {
  __shared__ double sw[16][64];
  __shared__ double sq[16][65];
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  const int nout = k * (k + 1);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // k <= 64: k(k+1) <= 4160 <= 5 * 256 * ... (looped below)
  for (int base = 0; base < nout; base += 5 * 256) {
    for (int q = 0; q < 5; ++q) acc[q] = 0.0;
    for (int rr = r0; rr < r1; rr += 16) {
      const int nrow = min(16, r1 - rr);
      for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
        const int q = idx / 64, c = idx % 64;
        const bool ok = q < nrow && c < k;
        sw[q][c] = ok ? W[(size_t)(rr + q) * k + c] : 0.0;
        sq[q][c] = ok ? Q[(size_t)(rr + q) * k + c] : 0.0;
      }
      if (threadIdx.x < 16) sq[threadIdx.x][64] = threadIdx.x < nrow ? r[rr + threadIdx.x] : 0.0;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int o = base + q * 256 + threadIdx.x;
        if (o < nout) {
          const int i = o / (k + 1), j = o % (k + 1);
          const int jj = (j == k) ? 64 : j;
          double v = acc[q];
          for (int t = 0; t < nrow; ++t) v = fma(sw[t][i], sq[t][jj], v);
          acc[q] = v;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int o = base + q * 256 + threadIdx.x;
      if (o < nout) partial[(size_t)blockIdx.x * nout + o] = acc[q];
    }
  }
}

// The same [eta | wr] partials in double-single arithmetic on the FP32 pipe (the inner solves of the mixed forms;
// this GPU's FP32 pipe issues ~75 times the FP64 one).  Every FP64 element is split once, when it is staged, into
// an unevaluated pair hi + lo of FP32 values (|lo| <= 2^-24 |hi|, 48 bits in all); each product is formed from
// the pairs with Dekker's exact product of the high parts by an FMA plus the two cross terms, and added to a
// (hi, lo) running sum by Knuth's TwoSum (Dekker 1971; Knuth, TAOCP vol. 2).  Relative accuracy of a column sum
// ~2^-46, converted to FP64 at the end.  The _rn intrinsics keep the compiler from contracting the error-free
// transformations into FMAs.
__device__ __forceinline__ void ds_madd(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float ph = __fmul_rn(ah, bh);
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  const float t = __fadd_rn(sh, ph), bb = __fsub_rn(t, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(ph, bb));
  sl = __fadd_rn(sl, __fadd_rn(e, pl));
  sh = t;
}
__device__ __forceinline__ void ds_split(double v, float& h, float& l) { d2ds(v, h, l); }
// Register tiling: every thread sums 4 x 4 outputs (rows i of W, columns j of [Q | r]) over a slice of the chunk's
// rows, so each staged pair is read once per 4 products; the slices are added in slice order at the end.
constexpr int ETA_DS_ROWS = 32;   // rows staged per step
__global__ void __launch_bounds__(256) k_eta_partial_ds(int n, int k, const double* __restrict__ W,
                                                        const double* __restrict__ Q, const double* __restrict__ r,
                                                        int rows_per_chunk, double* __restrict__ partial) {
  __shared__ float swh[ETA_DS_ROWS][68], swl[ETA_DS_ROWS][68];   // W rows, columns 0..k-1 (padded to 68)
  __shared__ float sqh[ETA_DS_ROWS][68], sql[ETA_DS_ROWS][68];   // [Q | r] rows, columns 0..k (padded)
  __shared__ double red[256][4];
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  const int nout = k * (k + 1);
  const int bi = (k + 3) / 4, bj = (k + 4) / 4, nblk = bi * bj;
  const int slices = max(1, 256 / nblk);
  const int tid = threadIdx.x;
  const int sl = tid / nblk;
  const bool active = sl < slices;
  for (int b0 = 0; b0 < nblk; b0 += 256) {   // more than 256 blocks (k > 60): several passes
    const int blk = b0 + (slices > 1 ? tid % nblk : tid);
    const bool act = active && blk < nblk;
    const int i0 = (blk / bj) * 4, j0 = (blk % bj) * 4;
    float h[4][4] = {}, l[4][4] = {};
    for (int rr = r0; rr < r1; rr += ETA_DS_ROWS) {
      const int nrow = min(ETA_DS_ROWS, r1 - rr);
      __syncthreads();
      // only the k (W) and k + 1 ([Q | r]) used columns are converted (an FP64 -> FP32 conversion issues on this
      // GPU's narrow FP64 path); the padding columns the 4 x 4 blocks may touch are zero-filled without one
      const int kq = k + 1;
      for (int idx = tid; idx < ETA_DS_ROWS * kq; idx += 256) {
        const int q = idx / kq, c = idx % kq;
        if (q < nrow) {
          if (c < k) ds_split(W[(size_t)(rr + q) * k + c], swh[q][c], swl[q][c]);
          ds_split(c < k ? Q[(size_t)(rr + q) * k + c] : r[rr + q], sqh[q][c], sql[q][c]);
        } else {
          if (c < k) { swh[q][c] = 0.f; swl[q][c] = 0.f; }
          sqh[q][c] = 0.f; sql[q][c] = 0.f;
        }
      }
      for (int idx = tid; idx < ETA_DS_ROWS * (68 - k); idx += 256) {   // columns >= k of W, >= k + 1 of Q
        const int q = idx / (68 - k), c = k + idx % (68 - k);
        swh[q][c] = 0.f; swl[q][c] = 0.f;
        if (c > k) { sqh[q][c] = 0.f; sql[q][c] = 0.f; }
      }
      __syncthreads();
      if (act)
        for (int t = sl; t < nrow; t += slices) {
          float ah[4], al[4], bh[4], bl[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            ah[u] = swh[t][i0 + u]; al[u] = swl[t][i0 + u];
            bh[u] = sqh[t][j0 + u]; bl[u] = sql[t][j0 + u];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) ds_madd(ah[u], al[u], bh[v], bl[v], h[u][v], l[u][v]);
        }
    }
    // add the slices in slice order, 4 outputs of the block at a time
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      __syncthreads();
#pragma unroll
      for (int v = 0; v < 4; ++v) red[tid][v] = act ? ds2d(h[u][v], l[u][v]) : 0.0;
      __syncthreads();
      if (act && sl == 0) {
        const int i = i0 + u;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double acc = red[tid][v];
          for (int q = 1; q < slices; ++q) acc += red[tid + q * nblk][v];
          const int j = j0 + v;
          if (i < k && j <= k) partial[(size_t)blockIdx.x * nout + (size_t)i * (k + 1) + j] = acc;
        }
      }
    }
  }
}

__global__ void k_reduce_chunks(int count, int chunks, const double* __restrict__ partial, double* __restrict__ C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double acc = 0.0;
  for (int c = 0; c < chunks; ++c) acc += partial[(size_t)c * count + i];
  C[i] = acc;
}

// KMAX = 32 (one-warp factorisation, small shared footprint) or 64 (block-wide factorisation).
template <int KMAX>
__global__ void __launch_bounds__(512) k_normalise(int k, const double* __restrict__ ext_partial, int chunks,
                                                   double trunc, double* __restrict__ T, double* __restrict__ alpha,
                                                   int* __restrict__ n_kept) {
  __shared__ double A[KMAX][KMAX + 1];    // eta, then (after the factorisation) X = M^{-1}
  __shared__ double Lc[KMAX][KMAX + 1];   // Lc[i][step], original row index i
  __shared__ int piv[KMAX];
  __shared__ int ipiv[KMAX];
  __shared__ int done[KMAX];
  __shared__ double rhs[KMAX];
  __shared__ int s_r, s_p;
  __shared__ double s_dmax, s_ipp, s_ilp;   // pivot reciprocal and its square root, computed once per step
  __shared__ double dinv[KMAX];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nout = k * (k + 1);
  double* ext = &Lc[0][0];   // [eta | wr] (k (k+1) <= KMAX (KMAX + 1) entries) lives in Lc's storage until needed
  // Sum of the chunk partials.  Every thread takes one output and a strided subset of the chunks (loads
  // coalesced over the outputs and independent of one another), then the subsets are added in a fixed order.
  const int groups = max(1, (int)blockDim.x / nout);
  // chunks g, g + groups, ...: eight independent loads at a time, summed as a tree (dependent FP64 adds are
  // slow on this GPU, so the chains are kept short)
  auto strided_sum = [&](int o, int g) {
    double acc = 0.0;
    for (int c = g; c < chunks; c += 8 * groups) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int cc = c + u * groups;
        v[u] = cc < chunks ? ext_partial[(size_t)cc * nout + o] : 0.0;
      }
      acc += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    return acc;
  };
  if (groups == 1) {
    for (int o = tid; o < nout; o += blockDim.x) ext[o] = strided_sum(o, 0);
  } else {
    double* red = &A[0][0];   // groups * nout <= blockDim.x entries
    if (tid < groups * nout) red[tid] = strided_sum(tid % nout, tid / nout);
    __syncthreads();
    for (int o = tid; o < nout; o += blockDim.x) {
      double v = 0.0;
      for (int g = 0; g < groups; ++g) v += red[g * nout + o];
      ext[o] = v;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, j = idx % k;
    // both triangles are summed and averaged: the computed W^T Q is not symmetric to working accuracy (W is
    // rebuilt from an FP32 history, in range(P) only to FP32 accuracy), and one triangle alone slows the
    // mixed-precision inner solve by an order of magnitude on the 3D elastic structure
    A[i][j] = 0.5 * (ext[i * (k + 1) + j] + ext[j * (k + 1) + i]);
  }
  if (tid < k) { done[tid] = 0; rhs[tid] = ext[tid * (k + 1) + k]; ipiv[tid] = -1; }
  __syncthreads();
  for (int idx = tid; idx < KMAX * (KMAX + 1); idx += blockDim.x) (&Lc[0][0])[idx] = 0.0;
  __syncthreads();
  if (KMAX <= 32) {
    if (warp == 0) normalise_warp<KMAX + 1>(k, A, Lc, piv, dinv, rhs, trunc, T, alpha, n_kept);
    return;
  }
  if (warp == 0) {
    double m = 0.0;
    for (int i = lane; i < k; i += 32) m = fmax(m, A[i][i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) { s_dmax = m; s_r = 0; }
  }
  __syncthreads();
  // step 0 pivot
  if (warp == 0) {
    double best = -1.0;
    int bi = -1;
    for (int i = lane; i < k; i += 32)
      if (A[i][i] > best) { best = A[i][i]; bi = i; }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) { best = ob; bi = oi; }
    }
    if (lane == 0) {
      s_p = (bi >= 0 && best > trunc * s_dmax && s_dmax > 0.0) ? bi : -1;
      if (s_p >= 0) {
        done[bi] = 1; piv[0] = bi; s_r = 1;
        s_ipp = 1.0 / best;
        s_ilp = sqrt(s_ipp);
      }
    }
  }
  __syncthreads();
  for (int step = 0; step < k; ++step) {
    const int p = s_p;
    if (p < 0) break;
    // column `step` of the factor and the trailing update (A[.][p] is not modified in this phase)
    const double inv_pp = s_ipp, inv_lp = s_ilp;
    for (int i = tid; i < k; i += blockDim.x) {
      if (i == p) Lc[i][step] = A[p][p] * inv_lp;
      else if (!done[i]) Lc[i][step] = A[i][p] * inv_lp;
    }
    for (int idx = tid; idx < k * k; idx += blockDim.x) {   // lower triangle only (A is read as symmetric)
      const int i = idx / k, j = idx % k;
      if (j <= i && !done[i] && !done[j]) {
        const double v = A[i][j] - A[i][p] * A[j][p] * inv_pp;
        A[i][j] = v;
        A[j][i] = v;
      }
    }
    __syncthreads();
    if (warp == 0) {   // next pivot: argmax of the remaining diagonal (ties -> lowest index)
      double best = -1.0;
      int bi = -1;
      for (int i = lane; i < k; i += 32)
        if (!done[i] && A[i][i] > best) { best = A[i][i]; bi = i; }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        s_p = (step + 1 < k && bi >= 0 && best > trunc * s_dmax) ? bi : -1;
        if (s_p >= 0) {
          done[bi] = 1; piv[step + 1] = bi; s_r = step + 2;
          s_ipp = 1.0 / best;
          s_ilp = sqrt(s_ipp);
        }
      }
    }
    __syncthreads();
  }
  const int r = s_r;
  // X = M^{-1} with M[a][b] = Lc[piv[a]][b] (lower triangular r x r): X = I, then for each l the row X[l] is
  // final after dividing by M[l][l], and rows below are updated
  for (int idx = tid; idx < KMAX * KMAX; idx += blockDim.x)
    A[idx / KMAX][idx % KMAX] = (idx / KMAX == idx % KMAX) ? 1.0 : 0.0;
  __syncthreads();
  for (int l = tid; l < r; l += blockDim.x) dinv[l] = 1.0 / Lc[piv[l]][l];
  __syncthreads();
  for (int l = 0; l < r; ++l) {
    const double inv = dinv[l];
    for (int c = tid; c <= l; c += blockDim.x) A[l][c] *= inv;
    __syncthreads();
    for (int idx = tid; idx < (r - 1 - l) * (l + 1); idx += blockDim.x) {
      const int i = l + 1 + idx / (l + 1), c = idx % (l + 1);
      A[i][c] -= Lc[piv[i]][l] * A[l][c];
    }
    __syncthreads();
  }
  // T[piv[a]][c] = X[c][a] for a, c < r; zero elsewhere; alpha[c] = sum_a X[c][a] rhs[piv[a]]
  for (int a = tid; a < r; a += blockDim.x) ipiv[piv[a]] = a;
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += blockDim.x) {
    const int row = idx / k, c = idx % k;
    const int a = ipiv[row];
    T[idx] = (c < r && a >= 0) ? A[c][a] : 0.0;
  }
  for (int c = tid; c < k; c += blockDim.x) {
    double v = 0.0;
    if (c < r)
      for (int a = 0; a < r; ++a) v += A[c][a] * rhs[piv[a]];
    alpha[c] = v;
  }
  if (tid == 0) *n_kept = r;
}

// Wn = W T, Qn = Q T, lambda += W (T alpha), r -= Q (T alpha); per-CTA partial sums of the new r^2.
// History: a warp takes 32 / kp rows at once (kp = k rounded up to a power of two), one lane per column:
// every element of W and Q is converted once and row j of the block is broadcast by shuffles (TH arithmetic;
// for k > 32 a lane holds two columns).  lambda and r: one thread per row, FP64 dot products with T alpha
// (a reduction across lanes would cost several times the FP64 operations, and FP64 is the scarce pipe).
template <typename TH>
__global__ void __launch_bounds__(256) k_update(int n, int k, const double* __restrict__ W,
                                                const double* __restrict__ Q, const double* __restrict__ T,
                                                const double* __restrict__ alpha, TH* __restrict__ Wn,
                                                TH* __restrict__ Qn, const int* __restrict__ d_off,
                                                double* __restrict__ lam,
                                                double* __restrict__ r, double* __restrict__ rr_partial,
                                                AdvanceArgs adv) {
  __shared__ TH sT[64][65];
  __shared__ double beta[64];
  __shared__ double warp_rr[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < k * k; idx += blockDim.x) sT[idx / k][idx % k] = (TH)T[idx];
  if (tid < k) {
    double v = 0.0;
    for (int c = 0; c < k; ++c) v = fma(T[(size_t)tid * k + c], alpha[c], v);
    beta[tid] = v;
  }
  __syncthreads();
  int kp = 1;
  while (kp < k) kp <<= 1;
  const int rows_w = kp >= 32 ? 1 : 32 / kp;          // rows per warp pass
  const int seg = kp >= 32 ? 32 : kp;                  // lanes per row
  const int sub = lane / seg, c0 = lane % seg;
  const bool two = k > 32;                             // second column c0 + 32
  const long long off = d_off ? (long long)*d_off : 0;   // a multiple of k: the new block of the history
  const size_t blk = hist_col(off, n, k);
  const long long stride = (long long)gridDim.x * 8 * rows_w;
  for (long long base = ((long long)blockIdx.x * 8 + warp) * rows_w; base < n; base += stride) {
    const long long row = base + sub;
    const bool ok = row < n;
    const bool v0 = ok && c0 < k, v1 = two && ok && c0 + 32 < k;
    const TH w0h = v0 ? from_f64<TH>(W[row * k + c0]) : TH(0), q0h = v0 ? from_f64<TH>(Q[row * k + c0]) : TH(0);
    const TH w1h = v1 ? from_f64<TH>(W[row * k + c0 + 32]) : TH(0);
    const TH q1h = v1 ? from_f64<TH>(Q[row * k + c0 + 32]) : TH(0);
    TH wn0 = TH(0), qn0 = TH(0), wn1 = TH(0), qn1 = TH(0);
    const int ca = c0 < k ? c0 : 0, cb = c0 + 32 < k ? c0 + 32 : 0;
    for (int j = 0; j < k; ++j) {
      const int src = j < 32 ? j : j - 32;
      const TH wj = __shfl_sync(0xffffffffu, j < 32 ? w0h : w1h, src, seg);
      const TH qj = __shfl_sync(0xffffffffu, j < 32 ? q0h : q1h, src, seg);
      wn0 = fma(wj, sT[j][ca], wn0);
      qn0 = fma(qj, sT[j][ca], qn0);
      if (two) {
        wn1 = fma(wj, sT[j][cb], wn1);
        qn1 = fma(qj, sT[j][cb], qn1);
      }
    }
    if (v0) {
      Wn[blk + row * k + c0] = wn0;
      Qn[blk + row * k + c0] = qn0;
    }
    if (v1) {
      Wn[blk + row * k + c0 + 32] = wn1;
      Qn[blk + row * k + c0 + 32] = qn1;
    }
  }
  double rr = 0.0;
  for (long long row = (long long)blockIdx.x * blockDim.x + tid; row < n; row += (long long)gridDim.x * blockDim.x) {
    const double* w = W + row * k;
    const double* q = Q + row * k;
    double l0 = 0.0, l1 = 0.0, d0 = 0.0, d1 = 0.0;
    int c = 0;
    for (; c + 1 < k; c += 2) {
      l0 = fma(w[c], beta[c], l0);
      l1 = fma(w[c + 1], beta[c + 1], l1);
      d0 = fma(q[c], beta[c], d0);
      d1 = fma(q[c + 1], beta[c + 1], d1);
    }
    if (c < k) {
      l0 = fma(w[c], beta[c], l0);
      d0 = fma(q[c], beta[c], d0);
    }
    lam[row] += l0 + l1;
    const double rn = r[row] - (d0 + d1);
    r[row] = rn;
    rr = fma(rn, rn, rr);
  }
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  if (lane == 0) warp_rr[warp] = rr;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += warp_rr[w];
    rr_partial[blockIdx.x] = s;
    // the last CTA to finish (every CTA has read the history offset by then) advances the history state
    if (adv.cols) {
      __threadfence();
      const unsigned prev = atomicAdd(adv.counter, 1u);
      if (prev == gridDim.x - 1) {
        int c = *adv.cols + adv.k;
        if ((long long)c + adv.k > adv.cap) c = 0;
        *adv.cols = c;
        *adv.dropped += adv.k - *adv.n_kept;
        *adv.iters += 1;
        *adv.counter = 0u;
        __threadfence();
      }
    }
  }
}

__global__ void k_sum_sq(int n, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double red[256];
  double v = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v = fma(x[i], x[i], v);
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

__global__ void k_axpy(int n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], y[i]);
}

// ------------------------------------------------------------------------------------------------ host
template <typename TA, typename TB>
void gram(int n, int a, int b, const TA* A, int lda, const TB* B, int ldb, double* C, DBuf<double>& partial,
          cudaStream_t s) {
  if (a <= 0 || b <= 0) return;
  const int ta = ceil_div(a, 64), tb = ceil_div(b, 64);
  int chunks = std::max(1, std::min(ceil_div(n, 64), 304 / std::max(1, ta * tb)));
  const int rows = std::max(1, ceil_div(n, chunks));
  chunks = std::max(1, ceil_div(n, rows));
  partial.ensure((size_t)chunks * a * b);
  k_gram_partial<TA, TB><<<dim3(ta, tb, chunks), 256, 0, s>>>(n, a, b, A, lda, B, ldb, rows, partial.p);
  FETIRP_LAUNCH_CHECK();
  k_reduce_chunks<<<ceil_div(a * b, 256), 256, 0, s>>>(a * b, chunks, partial.p, C);
  FETIRP_LAUNCH_CHECK();
}

template void gram<float, double>(int, int, int, const float*, int, const double*, int, double*, DBuf<double>&,
                                  cudaStream_t);
template void gram<double, double>(int, int, int, const double*, int, const double*, int, double*,
                                   DBuf<double>&, cudaStream_t);

// up to four chunks per SM (the sums are FP64-pipe bound: more resident warps keep the pipe busy)
int eta_chunks(int n) { return std::max(1, std::min(608, ceil_div(n, 256))); }

// (h, l) += (bh, bl) for unevaluated FP32 pairs: Knuth's TwoSum of the high parts, the low parts and the error
// added, then renormalised (Dekker's Fast2Sum)
__device__ __forceinline__ void ds_add(float& h, float& l, float bh, float bl) {
  const float s = __fadd_rn(h, bh), bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  const float t = __fadd_rn(__fadd_rn(l, bl), e);
  h = __fadd_rn(s, t);
  l = __fsub_rn(t, __fsub_rn(h, s));
}

// eta and W^T r for a narrow block (k = K <= 4): one thread per row, every thread holding all K (K + 1) sums as
// FP32 pairs (the same products and sums as k_eta_partial_ds), added over the warp by shuffles in a fixed tree,
// over the CTA's warps in warp order in FP64; one partial per CTA in the layout of k_eta_partial_ds.
template <int K>
__global__ void __launch_bounds__(256) k_eta_small_ds(int n, const double* __restrict__ W, const double* __restrict__ Q,
                                                      const double* __restrict__ r, int rows_per_chunk,
                                                      double* __restrict__ partial) {
  constexpr int NO = K * (K + 1);
  __shared__ double red[8][NO];
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  float h[NO], l[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) { h[o] = 0.f; l[o] = 0.f; }
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    float wh[K], wl[K], qh[K + 1], ql[K + 1];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      ds_split(W[(size_t)row * K + c], wh[c], wl[c]);
      ds_split(Q[(size_t)row * K + c], qh[c], ql[c]);
    }
    ds_split(r[row], qh[K], ql[K]);
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int j = 0; j <= K; ++j) ds_madd(wh[i], wl[i], qh[j], ql[j], h[i * (K + 1) + j], l[i * (K + 1) + j]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, h[o], off), bl = __shfl_xor_sync(0xffffffffu, l[o], off);
      ds_add(h[o], l[o], bh, bl);
    }
    if (lane == 0) red[warp][o] = ds2d(h[o], l[o]);
  }
  __syncthreads();
  if (threadIdx.x < NO) {
    double acc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[w][threadIdx.x];
    partial[(size_t)blockIdx.x * NO + threadIdx.x] = acc;
  }
}

// out[g][o] = sum of the chunk partials c = g, g + G, g + 2G, ... of output o (G = gridDim.y groups), four
// independent running sums added in a fixed order: the first level of the eta reduction, spread over many SMs
// (the FP64 adds of all chunks on the one normalising SM would take longer than the product itself)
__global__ void k_eta_group_sums(int nout, int chunks, const double* __restrict__ partial, double* __restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y, G = gridDim.y;
  if (o >= nout) return;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int c = g;
  for (; c + 3 * G < chunks; c += 4 * G) {
    a0 += partial[(size_t)c * nout + o];
    a1 += partial[(size_t)(c + G) * nout + o];
    a2 += partial[(size_t)(c + 2 * G) * nout + o];
    a3 += partial[(size_t)(c + 3 * G) * nout + o];
  }
  for (; c < chunks; c += G) a0 += partial[(size_t)c * nout + o];
  out[(size_t)g * nout + o] = (a0 + a1) + (a2 + a3);
}

int eta_partials(int n, int k, const double* W, const double* Q, const double* r, DBuf<double>& partial,
                 cudaStream_t s, bool ds, int* n_read) {
  const bool small = ds && k == 4;
  // narrow blocks: one CTA per SM, a few thousand rows each (every thread sums several rows before the
  // per-CTA reduction); otherwise up to 608 chunks of >= 256 rows
  const int chunks = small ? std::max(1, std::min(152, ceil_div(n, 1024))) : eta_chunks(n);
  const int rows = ceil_div(n, chunks);
  const int nout = k * (k + 1);
  partial.ensure((size_t)(chunks + ETA_GROUPS) * nout);
  if (small) k_eta_small_ds<4><<<chunks, 256, 0, s>>>(n, W, Q, r, rows, partial.p);
  else if (ds) k_eta_partial_ds<<<chunks, 256, 0, s>>>(n, k, W, Q, r, rows, partial.p);
  else k_eta_partial<<<chunks, 256, 0, s>>>(n, k, W, Q, r, rows, partial.p);
  FETIRP_LAUNCH_CHECK();
  *n_read = std::min(chunks, ETA_GROUPS);
  if (chunks <= ETA_GROUPS) return 0;
  k_eta_group_sums<<<dim3(ceil_div(nout, 256), ETA_GROUPS), 256, 0, s>>>(nout, chunks, partial.p,
                                                                         partial.p + (size_t)chunks * nout);
  FETIRP_LAUNCH_CHECK();
  return chunks;   // the normalisation reads ETA_GROUPS group sums from this chunk offset
}

// C (m x k, row-major) = A (m x m, row-major) B (m x k, row-major) in FP64.  One CTA per 4 rows of C, one warp
// per row, lanes over (column, j-slice) pairs: lane = slice * k' + column with k' = k rounded up to a power of
// two <= 32, so that every lane does useful FMAs; the slices of a column are added by a fixed shuffle tree.
__global__ void __launch_bounds__(128) k_small_gemm(int m, int k, const double* __restrict__ A,
                                                    const double* __restrict__ B, double* __restrict__ C) {
  // grid.y > 1: split of the inner dimension; part y sums j in [y m / Y, (y + 1) m / Y) and writes its own
  // m x k slice of C (the slices are added in order by k_sum_slices)
  const int row = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const int j0 = (int)((long long)blockIdx.y * m / gridDim.y), j1 = (int)((long long)(blockIdx.y + 1) * m / gridDim.y);
  C += (size_t)blockIdx.y * m * k;
  const double* a = A + (size_t)row * m;
  for (int g0 = 0; g0 < k; g0 += 32) {
    const int kk = min(32, k - g0);
    int kp = 1;
    while (kp < kk) kp <<= 1;                // columns handled by this pass, power of two
    const int slices = 32 / kp;
    const int g = g0 + (lane % kp), sl = lane / kp;
    double acc = 0.0;
    if (g < k) {   // four independent partial sums: the loads of four terms are in flight together
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = j0 + sl;
      for (; j + 3 * slices < j1; j += 4 * slices) {
        s0 = fma(a[j], B[(size_t)j * k + g], s0);
        s1 = fma(a[j + slices], B[(size_t)(j + slices) * k + g], s1);
        s2 = fma(a[j + 2 * slices], B[(size_t)(j + 2 * slices) * k + g], s2);
        s3 = fma(a[j + 3 * slices], B[(size_t)(j + 3 * slices) * k + g], s3);
      }
      for (; j < j1; j += slices) s0 = fma(a[j], B[(size_t)j * k + g], s0);
      acc = (s0 + s1) + (s2 + s3);
    }
    for (int off = kp; off < 32; off <<= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (sl == 0 && g < k) C[(size_t)row * k + g] = acc;
  }
}

// C[i] = sum of the `parts` slices P[p][i] in slice order
__global__ void k_sum_slices(int count, int parts, const double* __restrict__ P, double* __restrict__ C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double acc = P[i];
  for (int q = 1; q < parts; ++q) acc += P[(size_t)q * count + i];
  C[i] = acc;
}

int small_gemm_parts(int m) {
  // FP64 FMAs bound this product on this GPU: enough CTAs to reach every SM, inner slices of >= 128 terms
  return std::max(1, std::min(SMALL_GEMM_MAX_PARTS, std::min(ceil_div(608, ceil_div(m, 4)), m / 128)));
}

void small_gemm(int m, int k, const double* A, const double* B, double* C, cudaStream_t s, double* part) {
  if (m <= 0 || k <= 0) return;
  if (k > 64) throw Error(1, "k > 64");
  const int parts = part ? small_gemm_parts(m) : 1;
  k_small_gemm<<<dim3(ceil_div(m, 4), parts), 128, 0, s>>>(m, k, A, B, parts > 1 ? part : C);
  FETIRP_LAUNCH_CHECK();
  if (parts > 1) {
    k_sum_slices<<<ceil_div(m * k, 256), 256, 0, s>>>(m * k, parts, part, C);
    FETIRP_LAUNCH_CHECK();
  }
}


// C = A B in double-single arithmetic (A: m x m, B: m x k, both as FP32 pairs), one warp per row of C with the
// same lane layout as k_small_gemm (no inner split: each lane's column sum is a (hi, lo) pair, and the slices
// of a column are added in FP64 by the shuffle tree)
__global__ void __launch_bounds__(128) k_small_gemm_ds(int m, int k, const float* __restrict__ Ah,
                                                       const float* __restrict__ Al, const float* __restrict__ Bh,
                                                       const float* __restrict__ Bl, double* __restrict__ C) {
  // grid.y > 1: split of the inner dimension as in k_small_gemm (slices added in order by k_sum_slices)
  const int row = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const int j0 = (int)((long long)blockIdx.y * m / gridDim.y), j1 = (int)((long long)(blockIdx.y + 1) * m / gridDim.y);
  C += (size_t)blockIdx.y * m * k;
  const float* ah = Ah + (size_t)row * m;
  const float* al = Al + (size_t)row * m;
  for (int g0 = 0; g0 < k; g0 += 32) {
    const int kk = min(32, k - g0);
    int kp = 1;
    while (kp < kk) kp <<= 1;
    const int slices = 32 / kp;
    const int g = g0 + (lane % kp), sl = lane / kp;
    double acc = 0.0;
    if (g < k) {
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      int j = j0 + sl;
      for (; j + slices < j1; j += 2 * slices) {
        ds_madd(ah[j], al[j], Bh[(size_t)j * k + g], Bl[(size_t)j * k + g], h0, l0);
        ds_madd(ah[j + slices], al[j + slices], Bh[(size_t)(j + slices) * k + g], Bl[(size_t)(j + slices) * k + g],
                h1, l1);
      }
      for (; j < j1; j += slices) ds_madd(ah[j], al[j], Bh[(size_t)j * k + g], Bl[(size_t)j * k + g], h0, l0);
      acc = ds2d(h0, l0) + ds2d(h1, l1);
    }
    for (int off = kp; off < 32; off <<= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (sl == 0 && g < k) C[(size_t)row * k + g] = acc;
  }
}

void small_gemm_ds(int m, int k, const float* Ah, const float* Al, const float* Bh, const float* Bl, double* C,
                   cudaStream_t s, double* part) {
  if (m <= 0 || k <= 0) return;
  if (k > 64) throw Error(1, "k > 64");
  const int parts = part ? small_gemm_parts(m) : 1;
  k_small_gemm_ds<<<dim3(ceil_div(m, 4), parts), 128, 0, s>>>(m, k, Ah, Al, Bh, Bl, parts > 1 ? part : C);
  FETIRP_LAUNCH_CHECK();
  if (parts > 1) {
    k_sum_slices<<<ceil_div(m * k, 256), 256, 0, s>>>(m * k, parts, part, C);
    FETIRP_LAUNCH_CHECK();
  }
}

void normalise(int k, const double* ext_partial, int chunks, double trunc, double* T, double* alpha, int* n_kept,
               cudaStream_t s) {
  if (k > 64) throw Error(1, "block width k > 64 is not supported");
  if (k <= 32) k_normalise<32><<<1, 512, 0, s>>>(k, ext_partial, chunks, trunc, T, alpha, n_kept);
  else k_normalise<64><<<1, 512, 0, s>>>(k, ext_partial, chunks, trunc, T, alpha, n_kept);
  FETIRP_LAUNCH_CHECK();
}

template <typename TH>
void update(int n, int k, const double* W, const double* Q, const double* T, const double* alpha, TH* Wn, TH* Qn,
            const int* d_off, double* lam, double* r, double* rr_partial, int rr_blocks,
            cudaStream_t s, const AdvanceArgs& adv) {
  k_update<TH><<<rr_blocks, 256, 0, s>>>(n, k, W, Q, T, alpha, Wn, Qn, d_off, lam, r, rr_partial, adv);
  FETIRP_LAUNCH_CHECK();
}
template void update<double>(int, int, const double*, const double*, const double*, const double*, double*,
                             double*, const int*, double*, double*, double*, int, cudaStream_t, const AdvanceArgs&);
template void update<float>(int, int, const double*, const double*, const double*, const double*, float*, float*,
                            const int*, double*, double*, double*, int, cudaStream_t, const AdvanceArgs&);

// C[c][g] = sum over the rows of group g: w(row) * r[row] * Qh[row][c]  (= Qh^T S(r), the split multivector
// S(r) having at most two nonzero groups per row).  The products w(row) r[row] of the group lists are formed
// once per call (k_group_wr: FP64, and split into an FP32 hi + lo pair for an FP32 history).  Work items
// (64-column tile, group, 256-row chunk) are taken from the live history count a on the device, so a fixed
// grid serves every iteration of a captured graph.  Per item the chunk's rows and weights are staged in shared
// memory with one round of independent loads, the 8 warps take every 8th row (a warp reads 64 consecutive
// history columns of one row; eight rows' loads are issued together before their products), and the warp sums
// are added in warp order; chunk partials are then added in chunk order (deterministic).
constexpr int GS_ROWS = 256;   // rows per chunk
constexpr int GS_COLS = 64;    // history columns per item
constexpr int GS_GRID = 608;   // 4 CTAs per SM (64 registers a thread: the batched loads)
__global__ void k_group_wr(int total, const int* __restrict__ grp_row, const int* __restrict__ grp_src,
                           const double* __restrict__ grp_w, const double* __restrict__ r, double* __restrict__ wd,
                           float* __restrict__ wh, float* __restrict__ wl) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const double v = grp_w[e] * r[grp_src ? grp_src[e] : grp_row[e]];
  wd[e] = v;
  d2ds(v, wh[e], wl[e]);
}
template <typename TH>
__global__ void __launch_bounds__(256, 4) k_gram_split(int a_max, const int* __restrict__ d_a, int k,
                                                    const TH* __restrict__ Qh, int n, int hk,
                                                    const int* __restrict__ grp_ptr, const int* __restrict__ grp_row,
                                                    const double* __restrict__ wd, const float* __restrict__ wh,
                                                    const float* __restrict__ wl, int chunks,
                                                    double* __restrict__ partial) {
  __shared__ int srow[GS_ROWS];
  __shared__ double sw[GS_ROWS];
  __shared__ float swh[GS_ROWS], swl[GS_ROWS];   // w r[row] split into FP32 hi + lo (FP32 history)
  __shared__ double red[8][GS_COLS];
  const int a = d_a ? min(*d_a, a_max) : a_max;
  if (a <= 0) return;
  const int ctiles = (a + GS_COLS - 1) / GS_COLS;
  const int items = ctiles * k * chunks;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int ct = it % ctiles, rest = it / ctiles, g = rest % k, ch = rest / k;
    const int e0 = grp_ptr[g] + ch * GS_ROWS, cnt = min(GS_ROWS, grp_ptr[g + 1] - e0);
    const int c0 = ct * GS_COLS + lane, c1 = c0 + 32;
    const bool ok0 = c0 < a, ok1 = c1 < a;
    const TH* q0p = Qh + hist_col(ok0 ? c0 : 0, n, hk);
    const TH* q1p = Qh + hist_col(ok1 ? c1 : 0, n, hk);
    double a0 = 0.0, a1 = 0.0;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    __syncthreads();   // the previous item's shared-memory reads are done
    if (tid < cnt) {
      srow[tid] = grp_row[e0 + tid];
      if (sizeof(TH) == 4) {
        swh[tid] = wh[e0 + tid];
        swl[tid] = wl[e0 + tid];
      } else {
        sw[tid] = wd[e0 + tid];
      }
    }
    __syncthreads();
    {
      if (sizeof(TH) == 4) {
        // FP32 history: double-single arithmetic on the FP32 pipe (Dekker 1971; Knuth TwoSum).  q * s_hi is
        // split exactly into p + e by an FMA, q * s_lo is rounded (its error is ~2^-48 |q s|), and each column
        // sum is an unevaluated pair (hi, lo) updated by TwoSum; FP64 converts only the pairs at the end.  The
        // _rn intrinsics keep the compiler from contracting the error-free transformations into FMAs.
        for (int i0 = warp; i0 < cnt; i0 += 64) {   // rows i0, i0 + 8, ..., i0 + 56: loads first, then products
          float qa[8], qb[8], sh[8], sl[8];
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const int i = i0 + 8 * v;
            const bool okr = i < cnt;
            const int ic = okr ? i : 0;   // every shared index stays below GS_ROWS
            const size_t ro = (size_t)srow[ic] * hk;
            qa[v] = okr && ok0 ? (float)q0p[ro] : 0.f;
            qb[v] = okr && ok1 ? (float)q1p[ro] : 0.f;
            sh[v] = okr ? swh[ic] : 0.f;
            sl[v] = okr ? swl[ic] : 0.f;
          }
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            if (i0 + 8 * v >= cnt) break;
            {
              const float q0 = qa[v];
              const float p = __fmul_rn(q0, sh[v]), e = fmaf(q0, sh[v], -p), t = fmaf(q0, sl[v], e);
              const float u = __fadd_rn(h0, p), bb = __fsub_rn(u, h0);
              l0 = __fadd_rn(l0, __fadd_rn(__fadd_rn(__fsub_rn(h0, __fsub_rn(u, bb)), __fsub_rn(p, bb)), t));
              h0 = u;
            }
            {
              const float q1 = qb[v];
              const float p = __fmul_rn(q1, sh[v]), e = fmaf(q1, sh[v], -p), t = fmaf(q1, sl[v], e);
              const float u = __fadd_rn(h1, p), bb = __fsub_rn(u, h1);
              l1 = __fadd_rn(l1, __fadd_rn(__fadd_rn(__fsub_rn(h1, __fsub_rn(u, bb)), __fsub_rn(p, bb)), t));
              h1 = u;
            }
          }
        }
      } else {
  #pragma unroll 8
        for (int i = warp; i < cnt; i += 8) {
          const size_t ro = (size_t)srow[i] * hk;
          const double wv = sw[i];
          const double q0 = ok0 ? (double)q0p[ro] : 0.0;
          const double q1 = ok1 ? (double)q1p[ro] : 0.0;
          a0 = fma(wv, q0, a0);
          a1 = fma(wv, q1, a1);
        }
      }
    }
    if (sizeof(TH) == 4) {
      a0 = ds2d(h0, l0);
      a1 = ds2d(h1, l1);
    }
    red[warp][lane] = a0;   // (the previous item's reads of red ended before this item's staging barrier)
    red[warp][lane + 32] = a1;
    __syncthreads();
    if (tid < GS_COLS) {
      const int c = ct * GS_COLS + tid;
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) v += red[w][tid];
      if (c < a) partial[((size_t)ch * a + c) * k + g] = v;
    }
  }
}

// C[c] = sum over all rows of Qh[row][c] * r[row] (history times one vector: the Galerkin start).  Same item
// loop and arithmetic as k_gram_split, with rows_per_chunk-row chunks staged 256 rows at a time; the chunk
// partials (chunk-major, a per chunk) are added in chunk order by k_reduce_chunks.
template <typename TH>
__global__ void __launch_bounds__(256) k_hist_dot(int n, int a, const TH* __restrict__ Qh, int hk,
                                                  const double* __restrict__ r, int rows_per_chunk, int chunks,
                                                  double* __restrict__ partial) {
  __shared__ double sr[256];
  __shared__ float srh[256], srl[256];
  __shared__ double red[8][GS_COLS];
  const int ctiles = (a + GS_COLS - 1) / GS_COLS;
  const int items = ctiles * chunks;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int ct = it % ctiles, ch = it / ctiles;
    const int r0 = ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const int c0 = ct * GS_COLS + lane, c1 = c0 + 32;
    const bool ok0 = c0 < a, ok1 = c1 < a;
    const TH* q0p = Qh + hist_col(ok0 ? c0 : 0, n, hk);
    const TH* q1p = Qh + hist_col(ok1 ? c1 : 0, n, hk);
    double a0 = 0.0, a1 = 0.0;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    for (int sb = r0; sb < r1; sb += 256) {
      const int cnt = min(256, r1 - sb);
      __syncthreads();
      if (tid < cnt) {
        const double v = r[sb + tid];
        sr[tid] = v;
        d2ds(v, srh[tid], srl[tid]);
      }
      __syncthreads();
      if (sizeof(TH) == 4) {
#pragma unroll 8
        for (int i = warp; i < cnt; i += 8) {
          const size_t ro = (size_t)(sb + i) * hk;
          const float sh = srh[i], sl = srl[i];
          const float q0 = ok0 ? (float)q0p[ro] : 0.f;
          const float q1 = ok1 ? (float)q1p[ro] : 0.f;
          {
            const float p = __fmul_rn(q0, sh), e = fmaf(q0, sh, -p), t = fmaf(q0, sl, e);
            const float u = __fadd_rn(h0, p), bb = __fsub_rn(u, h0);
            l0 = __fadd_rn(l0, __fadd_rn(__fadd_rn(__fsub_rn(h0, __fsub_rn(u, bb)), __fsub_rn(p, bb)), t));
            h0 = u;
          }
          {
            const float p = __fmul_rn(q1, sh), e = fmaf(q1, sh, -p), t = fmaf(q1, sl, e);
            const float u = __fadd_rn(h1, p), bb = __fsub_rn(u, h1);
            l1 = __fadd_rn(l1, __fadd_rn(__fadd_rn(__fsub_rn(h1, __fsub_rn(u, bb)), __fsub_rn(p, bb)), t));
            h1 = u;
          }
        }
      } else {
#pragma unroll 8
        for (int i = warp; i < cnt; i += 8) {
          const size_t ro = (size_t)(sb + i) * hk;
          const double wv = sr[i];
          a0 = fma(wv, ok0 ? (double)q0p[ro] : 0.0, a0);
          a1 = fma(wv, ok1 ? (double)q1p[ro] : 0.0, a1);
        }
      }
    }
    if (sizeof(TH) == 4) {
      a0 = ds2d(h0, l0);
      a1 = ds2d(h1, l1);
    }
    __syncthreads();
    red[warp][lane] = a0;
    red[warp][lane + 32] = a1;
    __syncthreads();
    if (tid < GS_COLS) {
      const int c = ct * GS_COLS + tid;
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) v += red[w][tid];
      if (c < a) partial[(size_t)ch * a + c] = v;
    }
  }
}

// C[i] = sum over the chunk partials of output i: one warp per output, lane j adds chunks j, j + 32, ... and the
// lanes are added by a fixed shuffle tree (deterministic; the chunks of one output are read in parallel)
__global__ void k_reduce_chunks_dyn(int a_max, const int* __restrict__ d_a, int k, int chunks,
                                    const double* __restrict__ partial, double* __restrict__ C) {
  const int a = d_a ? min(*d_a, a_max) : a_max;
  const int count = a * k;
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= count) return;   // whole warps leave together (i is the same for the 32 lanes)
  double acc = 0.0;
  for (int c = lane; c < chunks; c += 32) acc += partial[(size_t)c * count + i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) C[i] = acc;
}

template <typename TH>
void gram_split(int a_max, const int* d_a, int k, const TH* Qh, int n, int hk, const double* r, const int* grp_ptr,
                const int* grp_row, const double* grp_w, int n_entries, int max_group_rows, double* C,
                DBuf<double>& partial, DBuf<double>& wr, cudaStream_t s, const int* grp_src) {
  if (a_max <= 0) return;
  const int chunks = std::max(1, ceil_div(max_group_rows, GS_ROWS));
  partial.ensure((size_t)chunks * a_max * k);
  wr.ensure(2 * (size_t)std::max(n_entries, 1));
  double* wd = wr.p;
  float* wh = reinterpret_cast<float*>(wr.p + std::max(n_entries, 1));
  float* wl = wh + std::max(n_entries, 1);
  if (n_entries > 0) {
    k_group_wr<<<ceil_div(n_entries, 256), 256, 0, s>>>(n_entries, grp_row, grp_src, grp_w, r, wd, wh, wl);
    FETIRP_LAUNCH_CHECK();
  }
  const int items = ceil_div(a_max, GS_COLS) * k * chunks;
  k_gram_split<TH><<<std::min(items, GS_GRID), 256, 0, s>>>(a_max, d_a, k, Qh, n, hk, grp_ptr, grp_row, wd, wh, wl,
                                                             chunks, partial.p);
  FETIRP_LAUNCH_CHECK();
  k_reduce_chunks_dyn<<<(unsigned)ceil_div((long long)a_max * k * 32, 256), 256, 0, s>>>(a_max, d_a, k, chunks,
                                                                                    partial.p, C);
  FETIRP_LAUNCH_CHECK();
}
template void gram_split<double>(int, const int*, int, const double*, int, int, const double*, const int*,
                                 const int*, const double*, int, int, double*, DBuf<double>&, DBuf<double>&,
                                 cudaStream_t, const int*);
template void gram_split<float>(int, const int*, int, const float*, int, int, const double*, const int*, const int*,
                                const double*, int, int, double*, DBuf<double>&, DBuf<double>&, cudaStream_t,
                                const int*);

template <typename TH>
void hist_dot(int n, int a, const TH* Qh, int hk, const double* r, double* C, DBuf<double>& partial,
              cudaStream_t s) {
  if (a <= 0 || n <= 0) return;
  const int ctiles = ceil_div(a, GS_COLS);
  int chunks = std::max(1, std::min(ceil_div(4 * GS_GRID, ctiles), ceil_div(n, 256)));
  // the partials live in a buffer that captured graphs also use: never grow it here
  if (partial.n < (size_t)a) throw Error(1, "hist_dot: partial buffer smaller than the history");
  chunks = std::min<long long>(chunks, (long long)(partial.n / a));
  const int rows = ceil_div(n, chunks);
  k_hist_dot<TH><<<std::min(ctiles * chunks, GS_GRID), 256, 0, s>>>(n, a, Qh, hk, r, rows, chunks, partial.p);
  FETIRP_LAUNCH_CHECK();
  k_reduce_chunks<<<ceil_div(a, 256), 256, 0, s>>>(a, chunks, partial.p, C);
  FETIRP_LAUNCH_CHECK();
}
template void hist_dot<double>(int, int, const double*, int, const double*, double*, DBuf<double>&, cudaStream_t);
template void hist_dot<float>(int, int, const float*, int, const double*, double*, DBuf<double>&, cudaStream_t);

// W[row][g] += alpha * sum_c Wh[row][c] C[c][g] over a history of `a` columns; products and sums in TH (FP32
// history: FFMA; FP64 history: DFMA).  Grid (64-row tiles, history splits): each CTA sums its share of the
// history columns for 64 rows x KP columns (KP = k rounded up to a power of two >= 8), with the next 32-column
// tile of the history loaded into registers while the current one is used.  With one split the CTA updates W
// itself; otherwise it stores a partial, and the last CTA of a row tile to finish (atomic ticket, reset by
// that CTA) adds the partials in split order and updates W (deterministic).
constexpr int TU_ROWS = 64, TU_CH = 32;
template <typename TH, int KP>
__global__ void __launch_bounds__(256) k_tall_update(int n, int a_max, const int* __restrict__ d_a, int k,
                                                     const TH* __restrict__ Wh, int hk,
                                                     const TH* __restrict__ C, int splits, TH* __restrict__ part,
                                                     unsigned* __restrict__ tickets, double alpha,
                                                     double* __restrict__ W) {
  constexpr int TXC = KP < 16 ? KP : 16;           // column threads
  constexpr int TY = 256 / TXC;                     // row threads
  constexpr int RPT = TU_ROWS / TY, CPT = KP / TXC;   // rows, columns per thread
  constexpr int LA = TU_CH * TU_ROWS / 256;         // history elements a thread loads per tile
  constexpr int LC = (TU_CH * KP + 255) / 256;      // C elements a thread loads per tile
  __shared__ TH sa[TU_CH][TU_ROWS + 1];   // [c][row]
  __shared__ TH sc[TU_CH][KP];            // [c][g]
  __shared__ bool last;
  const int a = d_a ? min(*d_a, a_max) : a_max;
  if (a <= 0) return;
  const int r0 = blockIdx.x * TU_ROWS;
  const int per = (a + splits - 1) / splits;
  const int c_begin = min(a, (int)blockIdx.y * per), c_end = min(a, c_begin + per);
  const int tid = threadIdx.x;
  const int ty = tid / TXC, tx = tid % TXC;
  TH acc[RPT][CPT] = {};
  TH pa[LA], pc[LC];
  auto load = [&](int c0) {
    const int cc = tid % TU_CH;   // the same history column for all of the thread's loads
    const bool okc = c0 + cc < c_end;
    const TH* col = Wh + hist_col(okc ? c0 + cc : 0, n, hk);
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      const int rr = (tid + 256 * i) / TU_CH;
      pa[i] = (r0 + rr < n && okc) ? col[(size_t)(r0 + rr) * hk] : TH(0);
    }
#pragma unroll
    for (int i = 0; i < LC; ++i) {
      const int idx = tid + 256 * i, cc = idx / KP, gg = idx % KP;
      pc[i] = (idx < TU_CH * KP && c0 + cc < c_end && gg < k) ? C[(size_t)(c0 + cc) * k + gg] : TH(0);
    }
  };
  if (c_begin < c_end) load(c_begin);
  for (int c0 = c_begin; c0 < c_end; c0 += TU_CH) {
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      const int idx = tid + 256 * i;
      sa[idx % TU_CH][idx / TU_CH] = pa[i];
    }
#pragma unroll
    for (int i = 0; i < LC; ++i) {
      const int idx = tid + 256 * i;
      if (idx < TU_CH * KP) sc[idx / KP][idx % KP] = pc[i];
    }
    __syncthreads();
    if (c0 + TU_CH < c_end) load(c0 + TU_CH);   // in flight while this tile is used
#pragma unroll 8
    for (int cc = 0; cc < TU_CH; ++cc) {
      TH w[RPT], b[CPT];
#pragma unroll
      for (int u = 0; u < RPT; ++u) w[u] = sa[cc][ty + TY * u];
#pragma unroll
      for (int v = 0; v < CPT; ++v) b[v] = sc[cc][tx + TXC * v];
#pragma unroll
      for (int u = 0; u < RPT; ++u)
#pragma unroll
        for (int v = 0; v < CPT; ++v) acc[u][v] = fma(w[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  if (splits == 1) {
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int row = r0 + ty + TY * u;
#pragma unroll
      for (int v = 0; v < CPT; ++v) {
        const int g = tx + TXC * v;
        if (row < n && g < k) W[(size_t)row * k + g] = fma(alpha, to_f64(acc[u][v]), W[(size_t)row * k + g]);
      }
    }
    return;
  }
  TH* P = part + (size_t)blockIdx.y * n * k;
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int row = r0 + ty + TY * u;
#pragma unroll
    for (int v = 0; v < CPT; ++v) {
      const int g = tx + TXC * v;
      if (row < n && g < k) P[(size_t)row * k + g] = acc[u][v];
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned prev = atomicAdd(&tickets[blockIdx.x], 1u);
    last = prev == (unsigned)splits - 1;
    if (last) tickets[blockIdx.x] = 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int rows = min(TU_ROWS, n - r0);
  for (int idx = tid; idx < rows * k; idx += 256) {
    const size_t o = (size_t)r0 * k + idx;
    TH v0 = TH(0), v1 = TH(0);
    int sp = 0;
    for (; sp + 1 < splits; sp += 2) {
      v0 += __ldcg(part + (size_t)sp * n * k + o);
      v1 += __ldcg(part + (size_t)(sp + 1) * n * k + o);
    }
    if (sp < splits) v0 += __ldcg(part + (size_t)sp * n * k + o);
    W[o] = fma(alpha, to_f64(v0 + v1), W[o]);
  }
}

// The FP32-history update for k = 4, 8, 16 or 32 on a tall block (one split): 256-row tiles, each thread RPT rows
// (ty + TY u) x 4 columns (4 tx ..), with 16-byte shared loads along the history index (about 1 load per 8 FMAs,
// so the FP32 pipe rather than the shared-memory port bounds it).  A tile of 32 history columns is 32 / K blocks of
// the block layout (width K), 256 rows each; it is copied to shared memory with 16-byte asynchronous copies
// (cp.async) into two stages, the next tile in flight while the current one is used.  Rows >= n and history
// columns >= a are zero-filled by the copy.  Per output the history columns are added in increasing order, one
// FMA each, as in k_tall_update.
constexpr int TW_ROWS = 256, TW_LD = 36;
constexpr int TW_STAGE_FLOATS = TW_ROWS * TW_LD + 32 * 32;
constexpr int TW_SMEM = 2 * TW_STAGE_FLOATS * 4;
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;   // source bytes; the rest of the 16 is zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
template <int K>
__global__ void __launch_bounds__(256, 2) k_tall_update_w(int n, int a_max, const int* __restrict__ d_a,
                                                         const float* __restrict__ Wh,
                                                         const float* __restrict__ Cf, double alpha,
                                                         double* __restrict__ W) {
  static_assert(K == 4 || K == 8 || K == 16 || K == 32, "history block width 4, 8, 16 or 32");
  constexpr int TXN = K / 4;          // column groups of 4
  constexpr int TY = 256 / TXN;       // row threads
  constexpr int RPT = TW_ROWS / TY;   // rows per thread
  extern __shared__ __align__(16) float tw_smem[];
  const int a = d_a ? min(*d_a, a_max) : a_max;
  if (a <= 0) return;
  const int r0 = blockIdx.x * TW_ROWS;
  const int tid = threadIdx.x, tx = tid / TY, ty = tid % TY;
  float acc[RPT][4];
#pragma unroll
  for (int u = 0; u < RPT; ++u)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[u][j] = 0.f;
  auto issue = [&](int c0, int st) {   // tile of history columns c0 .. c0 + 31 into stage st
    float* sa = tw_smem + st * TW_STAGE_FLOATS;
    float* sc = sa + TW_ROWS * TW_LD;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = tid + 256 * i, row = q >> 3, part = q & 7;   // part: 4 history columns
      const int rr = r0 + row, c = c0 + part * 4;
      const bool ok = c + 4 <= a && rr < n;
      const float* blk = Wh + (size_t)(c / K) * n * K + (c % K);
      cp_async16(sa + row * TW_LD + part * 4, blk + (size_t)(ok ? rr : 0) * K, ok);
    }
    if (tid < 8 * K) {   // 32 x K coefficients, 4 per copy
      const int cc = tid / (K / 4), gp = tid % (K / 4);
      const bool okc = c0 + cc < a;
      cp_async16(sc + cc * K + gp * 4, Cf + (size_t)(okc ? c0 + cc : 0) * K + gp * 4, okc);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int ntile = (a + 31) / 32;
  issue(0, 0);
  for (int t = 0; t < ntile; ++t) {
    if (t + 1 < ntile) {
      issue((t + 1) * 32, (t + 1) & 1);   // the stage it overwrites was released by the barrier below
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();   // tile t is in shared memory for every thread
    const float* sa = tw_smem + (t & 1) * TW_STAGE_FLOATS;
    const float* sc = sa + TW_ROWS * TW_LD;
#pragma unroll 1
    for (int cq = 0; cq < 8; ++cq) {
      float4 bv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = *reinterpret_cast<const float4*>(sc + (cq * 4 + j) * K + tx * 4);
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const float4 av = *reinterpret_cast<const float4*>(sa + (ty + TY * u) * TW_LD + cq * 4);
        acc[u][0] = fmaf(av.x, bv[0].x, acc[u][0]);
        acc[u][1] = fmaf(av.x, bv[0].y, acc[u][1]);
        acc[u][2] = fmaf(av.x, bv[0].z, acc[u][2]);
        acc[u][3] = fmaf(av.x, bv[0].w, acc[u][3]);
        acc[u][0] = fmaf(av.y, bv[1].x, acc[u][0]);
        acc[u][1] = fmaf(av.y, bv[1].y, acc[u][1]);
        acc[u][2] = fmaf(av.y, bv[1].z, acc[u][2]);
        acc[u][3] = fmaf(av.y, bv[1].w, acc[u][3]);
        acc[u][0] = fmaf(av.z, bv[2].x, acc[u][0]);
        acc[u][1] = fmaf(av.z, bv[2].y, acc[u][1]);
        acc[u][2] = fmaf(av.z, bv[2].z, acc[u][2]);
        acc[u][3] = fmaf(av.z, bv[2].w, acc[u][3]);
        acc[u][0] = fmaf(av.w, bv[3].x, acc[u][0]);
        acc[u][1] = fmaf(av.w, bv[3].y, acc[u][1]);
        acc[u][2] = fmaf(av.w, bv[3].z, acc[u][2]);
        acc[u][3] = fmaf(av.w, bv[3].w, acc[u][3]);
      }
    }
    __syncthreads();   // every thread is done with stage t & 1 before tile t + 2 is copied into it
  }
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int row = r0 + ty + TY * u;
    if (row >= n) continue;
    double* w = W + (size_t)row * K + tx * 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] += alpha * (double)acc[u][j];
  }
}

// Cf[i] = (float)C[i] for the first a * k coefficients (a read on the device): the FP32 history update then
// loads FP32 coefficients (one conversion per coefficient instead of one per coefficient and row tile)
__global__ void k_coef_to_f32(int a_max, const int* __restrict__ d_a, int k, const double* __restrict__ C,
                              float* __restrict__ Cf) {
  const int a = d_a ? min(*d_a, a_max) : a_max;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a * k; i += gridDim.x * blockDim.x) Cf[i] = d2f_rn(C[i]);
}

void tall_update_init() {
  static std::mutex mu;
  static bool attr_set[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  FETIRP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(1, "device ordinal out of range");
  if (!attr_set[dev]) {
    FETIRP_CUDA(cudaFuncSetAttribute(k_tall_update_w<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TW_SMEM));
    FETIRP_CUDA(cudaFuncSetAttribute(k_tall_update_w<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TW_SMEM));
    FETIRP_CUDA(cudaFuncSetAttribute(k_tall_update_w<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, TW_SMEM));
    FETIRP_CUDA(cudaFuncSetAttribute(k_tall_update_w<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TW_SMEM));
    attr_set[dev] = true;
  }
}

int tall_update_splits(int n, int a_max) {
  const int tiles = ceil_div(n, TU_ROWS);
  return std::max(1, std::min(std::max(1, 1216 / tiles), ceil_div(a_max, TU_CH)));
}

// scratch of tall_update in TH elements: split partials, then (FP32 history) the FP32 coefficients
static size_t tu_cf_off(int n, int a_max, int k) { return ((size_t)tall_update_splits(n, a_max) * n * k + 63) / 64 * 64; }
size_t tall_update_scratch(int n, int a_max, int k, bool fp32) {
  const size_t elems = fp32 ? tu_cf_off(n, a_max, k) + (size_t)a_max * k : (size_t)tall_update_splits(n, a_max) * n * k;
  return (elems * (fp32 ? 4 : 8) + 7) / 8;
}

template <typename TH>
void tall_update(int n, int a_max, const int* d_a, int k, const TH* Wh, int hk, const double* C, double alpha,
                 double* W, DBuf<double>& scratch, DBuf<unsigned>& tickets, cudaStream_t s) {
  if (a_max <= 0 || n <= 0) return;
  if (k > 64) throw Error(1, "k > 64");
  const int splits = tall_update_splits(n, a_max);
  const int tiles = ceil_div(n, TU_ROWS);
  const size_t cf_off = tu_cf_off(n, a_max, k);
  scratch.ensure(tall_update_scratch(n, a_max, k, sizeof(TH) == 4));
  if (tickets.n < (size_t)tiles) {   // tickets start at zero and every use leaves them at zero
    tickets.alloc(tiles);
    FETIRP_CUDA(cudaMemsetAsync(tickets.p, 0, sizeof(unsigned) * tiles, s));
  }
  TH* part = reinterpret_cast<TH*>(scratch.p);
  const TH* Ct = reinterpret_cast<const TH*>(C);
  if (sizeof(TH) == 4) {
    float* Cf = reinterpret_cast<float*>(part + cf_off);
    k_coef_to_f32<<<std::min(ceil_div(a_max * k, 256), 1216), 256, 0, s>>>(a_max, d_a, k, C, Cf);
    FETIRP_LAUNCH_CHECK();
    Ct = reinterpret_cast<const TH*>(Cf);
  }
  if (sizeof(TH) == 4 && splits == 1 && (k == 32 || k == 16 || k == 8 || k == 4) && hk == k) {
    tall_update_init();
    const float* wh = reinterpret_cast<const float*>(Wh);
    const float* cf = reinterpret_cast<const float*>(Ct);
    const int grid = ceil_div(n, TW_ROWS);
    if (k == 32) k_tall_update_w<32><<<grid, 256, TW_SMEM, s>>>(n, a_max, d_a, wh, cf, alpha, W);
    else if (k == 16) k_tall_update_w<16><<<grid, 256, TW_SMEM, s>>>(n, a_max, d_a, wh, cf, alpha, W);
    else if (k == 8) k_tall_update_w<8><<<grid, 256, TW_SMEM, s>>>(n, a_max, d_a, wh, cf, alpha, W);
    else k_tall_update_w<4><<<grid, 256, TW_SMEM, s>>>(n, a_max, d_a, wh, cf, alpha, W);
    FETIRP_LAUNCH_CHECK();
    return;
  }
  const dim3 grid(tiles, splits);
  if (k <= 8)
    k_tall_update<TH, 8><<<grid, 256, 0, s>>>(n, a_max, d_a, k, Wh, hk, Ct, splits, part, tickets.p, alpha, W);
  else if (k <= 16)
    k_tall_update<TH, 16><<<grid, 256, 0, s>>>(n, a_max, d_a, k, Wh, hk, Ct, splits, part, tickets.p, alpha, W);
  else if (k <= 32)
    k_tall_update<TH, 32><<<grid, 256, 0, s>>>(n, a_max, d_a, k, Wh, hk, Ct, splits, part, tickets.p, alpha, W);
  else
    k_tall_update<TH, 64><<<grid, 256, 0, s>>>(n, a_max, d_a, k, Wh, hk, Ct, splits, part, tickets.p, alpha, W);
  FETIRP_LAUNCH_CHECK();
}
template void tall_update<double>(int, int, const int*, int, const double*, int, const double*, double, double*,
                                  DBuf<double>&, DBuf<unsigned>&, cudaStream_t);
template void tall_update<float>(int, int, const int*, int, const float*, int, const double*, double, double*,
                                 DBuf<double>&, DBuf<unsigned>&, cudaStream_t);

void sum_sq(int n, const double* x, double* out_partial, int blocks, cudaStream_t s) {
  k_sum_sq<<<blocks, 256, 0, s>>>(n, x, out_partial);
  FETIRP_LAUNCH_CHECK();
}

void axpy_f64(int n, double a, const double* x, double* y, cudaStream_t s) {
  if (n <= 0) return;
  k_axpy<<<ceil_div(n, 256), 256, 0, s>>>(n, a, x, y);
  FETIRP_LAUNCH_CHECK();
}

}  // namespace fetirp
