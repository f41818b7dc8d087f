// Block Gram products, F-normalisation and the block update of multivector FETI (Table 1 right column,
// lines 5.2-5.4, with the F-normalisation and full reorthogonalisation of the numerical-issues subsection).
#include "ops.cuh"

namespace fetirp {

// Partial C_chunk = A[rows of chunk]^T B[rows of chunk]; grid (a tiles, b tiles, chunks).
__global__ void __launch_bounds__(256) k_gram_partial(int n, int a, int b, const double* __restrict__ A, int lda,
                                                      const double* __restrict__ B, int ldb, int rows_per_chunk,
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
      sa[q][c] = (r < r1 && a0 + c < a) ? A[(size_t)r * lda + a0 + c] : 0.0;
      sb[q][c] = (r < r1 && b0 + c < b) ? B[(size_t)r * ldb + b0 + c] : 0.0;
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

__global__ void k_reduce_chunks(int count, int chunks, const double* __restrict__ partial, double* __restrict__ C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double acc = 0.0;
  for (int c = 0; c < chunks; ++c) acc += partial[(size_t)c * count + i];
  C[i] = acc;
}

// One CTA: pivoted Cholesky of eta with truncation, T = Pi M^{-T}, alpha = T^T (W^T r).
__global__ void __launch_bounds__(256) k_normalise(int k, const double* __restrict__ eta,
                                                   const double* __restrict__ wr, double trunc,
                                                   double* __restrict__ T, double* __restrict__ alpha,
                                                   int* __restrict__ n_kept) {
  __shared__ double A[64][65];
  __shared__ double Lc[64][65];   // Lc[i][step], original row index i
  __shared__ double Minv[64][65];
  __shared__ int piv[64];
  __shared__ int done[64];
  __shared__ double rhs[64];
  __shared__ int s_r, s_p;
  __shared__ double s_dmax;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, j = idx % k;
    A[i][j] = 0.5 * (eta[(size_t)i * k + j] + eta[(size_t)j * k + i]);
    Lc[i][j] = 0.0;
  }
  if (tid < k) { done[tid] = 0; rhs[tid] = wr[tid]; }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < k; ++i) m = fmax(m, A[i][i]);
    s_dmax = m;
    s_r = 0;
  }
  __syncthreads();
  for (int step = 0; step < k; ++step) {
    if (tid == 0) {
      int p = -1;
      double best = 0.0;
      for (int i = 0; i < k; ++i)
        if (!done[i] && (p < 0 || A[i][i] > best)) { best = A[i][i]; p = i; }
      s_p = (p >= 0 && best > trunc * s_dmax && s_dmax > 0.0) ? p : -1;
      if (s_p >= 0) { done[p] = 1; piv[step] = p; s_r = step + 1; }
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) break;
    const double lp = sqrt(A[p][p]);
    for (int i = tid; i < k; i += blockDim.x) {
      if (i == p) Lc[i][step] = lp;
      else if (!done[i]) Lc[i][step] = A[i][p] / lp;
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += blockDim.x) {
      const int i = idx / k, j = idx % k;
      if (!done[i] && !done[j]) A[i][j] -= Lc[i][step] * Lc[j][step];
    }
    __syncthreads();
  }
  const int r = s_r;
  // M[a][b] = Lc[piv[a]][b] (lower triangular r x r); Minv = M^{-1}, column c per thread
  for (int c = tid; c < r; c += blockDim.x) {
    for (int i = 0; i < r; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int l = c; l < i; ++l) v -= Lc[piv[i]][l] * Minv[l][c];
      Minv[i][c] = (i < c) ? 0.0 : v / Lc[piv[i]][i];
    }
  }
  __syncthreads();
  // T[piv[a]][c] = Minv[c][a] for a, c < r; zero elsewhere
  for (int idx = tid; idx < k * k; idx += blockDim.x) T[idx] = 0.0;
  __syncthreads();
  for (int idx = tid; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, c = idx % r;
    T[(size_t)piv[a] * k + c] = Minv[c][a];
  }
  __syncthreads();
  for (int c = tid; c < k; c += blockDim.x) {
    double v = 0.0;
    if (c < r)
      for (int a = 0; a < r; ++a) v += Minv[c][a] * rhs[piv[a]];
    alpha[c] = v;
  }
  if (tid == 0) *n_kept = r;
}

// Wn = W T, Qn = Q T, lambda += W (T alpha), r -= Q (T alpha); per-CTA partial sums of the new r^2.
// One warp per row (grid-stride), k <= 64.
__global__ void __launch_bounds__(256) k_update(int n, int k, const double* __restrict__ W,
                                                const double* __restrict__ Q, const double* __restrict__ T,
                                                const double* __restrict__ alpha, double* __restrict__ Wn,
                                                double* __restrict__ Qn, long long ldn, double* __restrict__ lam,
                                                double* __restrict__ r, double* __restrict__ rr_partial) {
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
  for (int row = blockIdx.x * 8 + warp; row < n; row += warps_total) {
    const double* w = W + (size_t)row * k;
    const double* q = Q + (size_t)row * k;
    double dl = 0.0, dr = 0.0;
    for (int c = lane; c < k; c += 32) {
      double wn = 0.0, qn = 0.0;
      for (int j = 0; j < k; ++j) {
        wn = fma(w[j], sT[j][c], wn);
        qn = fma(q[j], sT[j][c], qn);
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
void gram_f64(int n, int a, int b, const double* A, int lda, const double* B, int ldb, double* C,
              DBuf<double>& partial, cudaStream_t s) {
  if (a <= 0 || b <= 0) return;
  const int ta = ceil_div(a, 64), tb = ceil_div(b, 64);
  int chunks = std::max(1, std::min(ceil_div(n, 64), 304 / std::max(1, ta * tb)));
  const int rows = std::max(1, ceil_div(n, chunks));
  chunks = std::max(1, ceil_div(n, rows));
  partial.ensure((size_t)chunks * a * b);
  k_gram_partial<<<dim3(ta, tb, chunks), 256, 0, s>>>(n, a, b, A, lda, B, ldb, rows, partial.p);
  FETIRP_LAUNCH_CHECK();
  k_reduce_chunks<<<ceil_div(a * b, 256), 256, 0, s>>>(a * b, chunks, partial.p, C);
  FETIRP_LAUNCH_CHECK();
}

void normalise(int k, const double* eta, const double* wr, double trunc, double* T, double* alpha, int* n_kept,
               cudaStream_t s) {
  if (k > 64) throw Error(1, "block width k > 64 is not supported");
  k_normalise<<<1, 256, 0, s>>>(k, eta, wr, trunc, T, alpha, n_kept);
  FETIRP_LAUNCH_CHECK();
}

void update(int n, int k, const double* W, const double* Q, const double* T, const double* alpha, double* Wn,
            double* Qn, long long ldn, double* lam, double* r, double* rr_partial, int rr_blocks, cudaStream_t s) {
  k_update<<<rr_blocks, 256, 0, s>>>(n, k, W, Q, T, alpha, Wn, Qn, ldn, lam, r, rr_partial);
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
