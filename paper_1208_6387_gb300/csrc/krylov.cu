// Block Gram products, F-normalisation and the block update of multivector FETI (Table 1 right column,
// lines 5.2-5.4, with the F-normalisation and full reorthogonalisation of the numerical-issues subsection).
#include "ops.cuh"

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

__global__ void k_reduce_chunks(int count, int chunks, const double* __restrict__ partial, double* __restrict__ C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double acc = 0.0;
  for (int c = 0; c < chunks; ++c) acc += partial[(size_t)c * count + i];
  C[i] = acc;
}

// One CTA: pivoted Cholesky of eta with truncation, T = Pi M^{-T}, alpha = T^T (W^T r).
// Pivot search by warp shuffles; the triangular inverse by a right-looking sweep, parallel over (row, column).
// ext_partial: `chunks` row-chunk partials of the k x (k+1) block [eta | W^T r]; they are added here in chunk
// order (one warp per output entry), so no separate reduction launch is needed.
__global__ void __launch_bounds__(512) k_normalise(int k, const double* __restrict__ ext_partial, int chunks,
                                                   double trunc, double* __restrict__ T, double* __restrict__ alpha,
                                                   int* __restrict__ n_kept) {
  __shared__ double A[64][65];    // eta, then (after the factorisation) X = M^{-1}
  __shared__ double Lc[64][65];   // Lc[i][step], original row index i
  __shared__ int piv[64];
  __shared__ int ipiv[64];
  __shared__ int done[64];
  __shared__ double rhs[64];
  __shared__ int s_r, s_p;
  __shared__ double s_dmax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nout = k * (k + 1);
  double* ext = &Lc[0][0];   // [eta | wr] (k (k+1) <= 64 * 65 entries) lives in Lc's storage until Lc is needed
  for (int o = warp; o < nout; o += blockDim.x / 32) {
    double v = 0.0;
    for (int c = lane; c < chunks; c += 32) v += ext_partial[(size_t)c * nout + o];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) ext[o] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, j = idx % k;
    A[i][j] = 0.5 * (ext[i * (k + 1) + j] + ext[j * (k + 1) + i]);
  }
  if (tid < k) { done[tid] = 0; rhs[tid] = ext[tid * (k + 1) + k]; ipiv[tid] = -1; }
  __syncthreads();
  for (int idx = tid; idx < 64 * 65; idx += blockDim.x) (&Lc[0][0])[idx] = 0.0;
  __syncthreads();
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
      if (s_p >= 0) { done[bi] = 1; piv[0] = bi; s_r = 1; }
    }
  }
  __syncthreads();
  for (int step = 0; step < k; ++step) {
    const int p = s_p;
    if (p < 0) break;
    // column `step` of the factor and the trailing update (A[.][p] is not modified in this phase)
    const double inv_pp = 1.0 / A[p][p];
    const double inv_lp = sqrt(inv_pp);
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
        if (s_p >= 0) { done[bi] = 1; piv[step + 1] = bi; s_r = step + 2; }
      }
    }
    __syncthreads();
  }
  const int r = s_r;
  // X = M^{-1} with M[a][b] = Lc[piv[a]][b] (lower triangular r x r): X = I, then for each l the row X[l] is
  // final after dividing by M[l][l], and rows below are updated
  for (int idx = tid; idx < 64 * 64; idx += blockDim.x) A[idx / 64][idx % 64] = (idx / 64 == idx % 64) ? 1.0 : 0.0;
  __syncthreads();
  for (int l = 0; l < r; ++l) {
    const double inv = 1.0 / Lc[piv[l]][l];
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
// One warp per row (grid-stride), k <= 64.  The history (Wn, Qn) is stored in TH.
template <typename TH>
__global__ void __launch_bounds__(256) k_update(int n, int k, const double* __restrict__ W,
                                                const double* __restrict__ Q, const double* __restrict__ T,
                                                const double* __restrict__ alpha, TH* __restrict__ Wn,
                                                TH* __restrict__ Qn, const int* __restrict__ d_off, long long ldn,
                                                double* __restrict__ lam,
                                                double* __restrict__ r, double* __restrict__ rr_partial,
                                                AdvanceArgs adv) {
  __shared__ double sT[64][65];
  __shared__ double beta[64];
  __shared__ double warp_rr[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < k * k; idx += blockDim.x) sT[idx / k][idx % k] = T[idx];
  __syncthreads();
  if (tid < k) {
    double v = 0.0;
    for (int c = 0; c < k; ++c) v += sT[tid][c] * alpha[c];
    beta[tid] = v;
  }
  __syncthreads();
  double rr = 0.0;
  const int warps_total = gridDim.x * 8;
  if (d_off) {
    Wn += *d_off;
    Qn += *d_off;
  }
  for (int row = blockIdx.x * 8 + warp; row < n; row += warps_total) {
    const double* w = W + (size_t)row * k;
    const double* q = Q + (size_t)row * k;
    double dl = 0.0, dr = 0.0;
    for (int c = lane; c < k; c += 32) {
      TH wn = TH(0), qn = TH(0);
      for (int j = 0; j < k; ++j) {
        wn = fma((TH)w[j], (TH)sT[j][c], wn);
        qn = fma((TH)q[j], (TH)sT[j][c], qn);
      }
      Wn[(size_t)row * ldn + c] = wn;
      Qn[(size_t)row * ldn + c] = qn;
      dl = fma(w[c], beta[c], dl);
      dr = fma(q[c], beta[c], dr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dl += __shfl_xor_sync(0xffffffffu, dl, o);
      dr += __shfl_xor_sync(0xffffffffu, dr, o);
    }
    if (lane == 0) {
      lam[row] += dl;
      const double rn = r[row] - dr;
      r[row] = rn;
      rr = fma(rn, rn, rr);
    }
  }
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

void gram_f64(int n, int a, int b, const double* A, int lda, const double* B, int ldb, double* C,
              DBuf<double>& partial, cudaStream_t s) {
  gram<double, double>(n, a, b, A, lda, B, ldb, C, partial, s);
}
template void gram<float, double>(int, int, int, const float*, int, const double*, int, double*, DBuf<double>&,
                                  cudaStream_t);
template void gram<double, double>(int, int, int, const double*, int, const double*, int, double*,
                                   DBuf<double>&, cudaStream_t);

__global__ void k_split_eta(int k, const double* __restrict__ ext, double* __restrict__ eta, double* __restrict__ wr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * (k + 1)) return;
  const int i = idx / (k + 1), j = idx % (k + 1);
  if (j == k) wr[i] = ext[idx];
  else eta[i * k + j] = ext[idx];
}

// Sum of chunk partials, one warp per output: lanes take chunks lane, lane+32, ... and a fixed shuffle tree
// combines them (deterministic).
__global__ void k_reduce_chunks_warp(int count, int chunks, const double* __restrict__ partial,
                                     double* __restrict__ C) {
  const int o = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (o >= count) return;
  double v = 0.0;
  for (int c = lane; c < chunks; c += 32) v += partial[(size_t)c * count + o];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (lane == 0) C[o] = v;
}

int eta_chunks(int n) { return std::max(1, std::min(152, ceil_div(n, 16))); }

void eta_partials(int n, int k, const double* W, const double* Q, const double* r, DBuf<double>& partial,
                  cudaStream_t s) {
  const int chunks = eta_chunks(n);
  const int rows = ceil_div(n, chunks);
  const int nout = k * (k + 1);
  partial.ensure((size_t)chunks * nout + nout);
  k_eta_partial<<<chunks, 256, 0, s>>>(n, k, W, Q, r, rows, partial.p);
  FETIRP_LAUNCH_CHECK();
}

// C (m x k, row-major) = A (m x m, row-major) B (m x k, row-major) in FP64.  One CTA per 4 rows of C, one warp
// per row, lanes over (column, j-slice) pairs: lane = slice * k' + column with k' = k rounded up to a power of
// two <= 32, so that every lane does useful FMAs; the slices of a column are added by a fixed shuffle tree.
__global__ void __launch_bounds__(128) k_small_gemm(int m, int k, const double* __restrict__ A,
                                                    const double* __restrict__ B, double* __restrict__ C) {
  const int row = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const double* a = A + (size_t)row * m;
  for (int g0 = 0; g0 < k; g0 += 32) {
    const int kk = min(32, k - g0);
    int kp = 1;
    while (kp < kk) kp <<= 1;                // columns handled by this pass, power of two
    const int slices = 32 / kp;
    const int g = g0 + (lane % kp), sl = lane / kp;
    double acc = 0.0;
    if (g < k)
      for (int j = sl; j < m; j += slices) acc = fma(a[j], B[(size_t)j * k + g], acc);
    for (int off = kp; off < 32; off <<= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (sl == 0 && g < k) C[(size_t)row * k + g] = acc;
  }
}

void small_gemm(int m, int k, const double* A, const double* B, double* C, cudaStream_t s) {
  if (m <= 0 || k <= 0) return;
  if (k > 64) throw Error(1, "k > 64");
  k_small_gemm<<<ceil_div(m, 4), 128, 0, s>>>(m, k, A, B, C);
  FETIRP_LAUNCH_CHECK();
}

void normalise(int k, const double* ext_partial, int chunks, double trunc, double* T, double* alpha, int* n_kept,
               cudaStream_t s) {
  if (k > 64) throw Error(1, "block width k > 64 is not supported");
  k_normalise<<<1, 512, 0, s>>>(k, ext_partial, chunks, trunc, T, alpha, n_kept);
  FETIRP_LAUNCH_CHECK();
}

template <typename TH>
void update(int n, int k, const double* W, const double* Q, const double* T, const double* alpha, TH* Wn, TH* Qn,
            const int* d_off, long long ldn, double* lam, double* r, double* rr_partial, int rr_blocks,
            cudaStream_t s, const AdvanceArgs& adv) {
  k_update<TH><<<rr_blocks, 256, 0, s>>>(n, k, W, Q, T, alpha, Wn, Qn, d_off, ldn, lam, r, rr_partial, adv);
  FETIRP_LAUNCH_CHECK();
}
template void update<double>(int, int, const double*, const double*, const double*, const double*, double*,
                             double*, const int*, long long, double*, double*, double*, int, cudaStream_t,
                             const AdvanceArgs&);
template void update<float>(int, int, const double*, const double*, const double*, const double*, float*, float*,
                            const int*, long long, double*, double*, double*, int, cudaStream_t, const AdvanceArgs&);

// C[c][g] = sum over the rows of group g: w(row) * r[row] * Qh[row][c]  (= Qh^T S(r), the split multivector
// S(r) having at most two nonzero groups per row).  Grid (128-column tiles, groups, row chunks): each CTA
// stages its chunk of (row, w r[row]) in shared memory, each thread owns one column and sums the chunk's rows
// in order; chunk partials are then added in chunk order (deterministic).
constexpr int GS_ROWS = 128;   // rows per chunk
template <typename TH>
__global__ void __launch_bounds__(128) k_gram_split(int a_max, const int* __restrict__ d_a, int k,
                                                    const TH* __restrict__ Qh, long long ldq,
                                                    const double* __restrict__ r, const int* __restrict__ grp_ptr,
                                                    const int* __restrict__ grp_row, const double* __restrict__ grp_w,
                                                    int chunks, double* __restrict__ partial) {
  __shared__ int srow[GS_ROWS];
  __shared__ double sw[GS_ROWS];
  const int a = d_a ? min(*d_a, a_max) : a_max;
  if ((int)blockIdx.x * 128 >= a) return;
  const int c = blockIdx.x * 128 + threadIdx.x;
  const int g = blockIdx.y, ch = blockIdx.z;
  const int e0 = grp_ptr[g] + ch * GS_ROWS, e1 = min(grp_ptr[g + 1], e0 + GS_ROWS);
  const int cnt = max(0, e1 - e0);
  if (threadIdx.x < cnt) {
    const int row = grp_row[e0 + threadIdx.x];
    srow[threadIdx.x] = row;
    sw[threadIdx.x] = grp_w[e0 + threadIdx.x] * r[row];
  }
  __syncthreads();
  if (c >= a) return;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int i = 0;
  for (; i + 8 <= cnt; i += 8) {
    double q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) q[u] = (double)Qh[(size_t)srow[i + u] * ldq + c];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = fma(sw[i + u], q[u], acc[u]);
  }
  for (; i < cnt; ++i) acc[0] = fma(sw[i], (double)Qh[(size_t)srow[i] * ldq + c], acc[0]);
  partial[((size_t)ch * a + c) * k + g] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

__global__ void k_reduce_chunks_dyn(int a_max, const int* __restrict__ d_a, int k, int chunks,
                                    const double* __restrict__ partial, double* __restrict__ C) {
  const int a = d_a ? min(*d_a, a_max) : a_max;
  const int count = a * k;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double acc = 0.0;
  for (int c = 0; c < chunks; ++c) acc += partial[(size_t)c * count + i];
  C[i] = acc;
}

template <typename TH>
void gram_split(int a_max, const int* d_a, int k, const TH* Qh, long long ldq, const double* r, const int* grp_ptr,
                const int* grp_row, const double* grp_w, int max_group_rows, double* C, DBuf<double>& partial,
                cudaStream_t s) {
  if (a_max <= 0) return;
  const int chunks = std::max(1, ceil_div(max_group_rows, GS_ROWS));
  partial.ensure((size_t)chunks * a_max * k);
  k_gram_split<TH><<<dim3(ceil_div(a_max, 128), k, chunks), 128, 0, s>>>(a_max, d_a, k, Qh, ldq, r, grp_ptr, grp_row,
                                                                           grp_w, chunks, partial.p);
  FETIRP_LAUNCH_CHECK();
  k_reduce_chunks_dyn<<<ceil_div(a_max * k, 256), 256, 0, s>>>(a_max, d_a, k, chunks, partial.p, C);
  FETIRP_LAUNCH_CHECK();
}
template void gram_split<double>(int, const int*, int, const double*, long long, const double*, const int*,
                                 const int*, const double*, int, double*, DBuf<double>&, cudaStream_t);
template void gram_split<float>(int, const int*, int, const float*, long long, const double*, const int*, const int*,
                                const double*, int, double*, DBuf<double>&, cudaStream_t);

// W[row][g] += alpha * sum_c Wh[row][c] C[c][g] over a history of `a` columns; products and sums in TH (FP32
// history: FFMA; FP64 history: DFMA).  Grid (64-row tiles, history splits): each CTA sums its share of the
// history columns for 64 rows x k columns (256 threads, 4 rows x k/16 columns each) into a partial; a second
// pass adds the partials in split order and updates W (deterministic).
constexpr int TU_ROWS = 64, TU_CH = 32;
template <typename TH>
__global__ void __launch_bounds__(256) k_tall_update_partial(int n, int a_max, const int* __restrict__ d_a, int k,
                                                             const TH* __restrict__ Wh, long long ldh,
                                                             const double* __restrict__ C, int splits,
                                                             TH* __restrict__ part) {
  __shared__ TH sa[TU_CH][TU_ROWS + 1];   // [c][row]
  __shared__ TH sc[TU_CH][64];            // [c][g]
  const int a = d_a ? min(*d_a, a_max) : a_max;
  const int r0 = blockIdx.x * TU_ROWS;
  const int per = (a + splits - 1) / splits;
  const int c_begin = blockIdx.y * per, c_end = min(a, c_begin + per);
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;       // rows ty*4 .. +3, columns tx, tx+16, tx+32, tx+48
  TH acc[4][4] = {};
  for (int c0 = c_begin; c0 < c_end; c0 += TU_CH) {
    for (int idx = tid; idx < TU_CH * TU_ROWS; idx += 256) {
      const int cc = idx % TU_CH, rr = idx / TU_CH;
      sa[cc][rr] = (r0 + rr < n && c0 + cc < c_end) ? Wh[(size_t)(r0 + rr) * ldh + c0 + cc] : TH(0);
    }
    for (int idx = tid; idx < TU_CH * 64; idx += 256) {
      const int cc = idx / 64, gg = idx % 64;
      sc[cc][gg] = (c0 + cc < c_end && gg < k) ? (TH)C[(size_t)(c0 + cc) * k + gg] : TH(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int cc = 0; cc < TU_CH; ++cc) {
      TH w[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { w[u] = sa[cc][ty * 4 + u]; b[u] = sc[cc][tx + 16 * u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(w[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  TH* P = part + (size_t)blockIdx.y * n * 64;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int row = r0 + ty * 4 + u;
    if (row >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) P[(size_t)row * 64 + tx + 16 * v] = acc[u][v];
  }
}

template <typename TH>
__global__ void k_tall_update_finish(int n, int k, int splits, const int* __restrict__ d_a, const TH* __restrict__ part,
                                     double alpha, double* __restrict__ W) {
  if (d_a && *d_a <= 0) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  TH acc = TH(0);
  for (int sp = 0; sp < splits; ++sp) acc += part[((size_t)sp * n + row) * 64 + g];
  W[idx] += alpha * (double)acc;
}

template <typename TH>
int tall_update_splits(int n, int a_max) {
  const int tiles = ceil_div(n, TU_ROWS);
  return std::max(1, std::min(std::max(1, 304 / tiles), ceil_div(a_max, TU_CH)));
}

template <typename TH>
void tall_update(int n, int a_max, const int* d_a, int k, const TH* Wh, long long ldh, const double* C, double alpha,
                 double* W, DBuf<double>& scratch, cudaStream_t s) {
  if (a_max <= 0 || n <= 0) return;
  if (k > 64) throw Error(1, "k > 64");
  const int splits = tall_update_splits<TH>(n, a_max);
  const size_t need = ((size_t)splits * n * 64 * sizeof(TH) + sizeof(double) - 1) / sizeof(double);
  scratch.ensure(need);
  TH* part = reinterpret_cast<TH*>(scratch.p);
  k_tall_update_partial<TH><<<dim3(ceil_div(n, TU_ROWS), splits), 256, 0, s>>>(n, a_max, d_a, k, Wh, ldh, C, splits,
                                                                               part);
  FETIRP_LAUNCH_CHECK();
  const long long tot = (long long)n * k;
  k_tall_update_finish<TH><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, k, splits, d_a, part, alpha, W);
  FETIRP_LAUNCH_CHECK();
}
template void tall_update<double>(int, int, const int*, int, const double*, long long, const double*, double,
                                  double*, DBuf<double>&, cudaStream_t);
template void tall_update<float>(int, int, const int*, int, const float*, long long, const double*, double, double*,
                                 DBuf<double>&, cudaStream_t);

// End of a block iteration: history count += k (restart when the next block would not fit), dropped
// directions and iterations counted on the device.
__global__ void k_advance(int* cols, int k, long long cap, const int* n_kept, int* dropped, int* iters) {
  int c = *cols + k;
  if ((long long)c + k > cap) c = 0;
  *cols = c;
  *dropped += k - *n_kept;
  *iters += 1;
}

void advance(int* cols, int k, long long cap, const int* n_kept, int* dropped, int* iters, cudaStream_t s) {
  k_advance<<<1, 1, 0, s>>>(cols, k, cap, n_kept, dropped, iters);
  FETIRP_LAUNCH_CHECK();
}

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
