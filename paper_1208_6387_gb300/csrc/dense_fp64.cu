// Dense FP64 tile kernels of the pattern set-up: Cholesky with zero-pivot detection (Sec. 2, floating
// subdomains), right-looking multi-right-hand-side triangular solves and a strided generic GEMM.
#include <algorithm>

#include "dense.cuh"

namespace fetirp {

// ------------------------------------------------------------------------------------------------ plan
void TilePlan::build(int nt_, const std::vector<uint8_t>& nz0) {
  nt = nt_;
  nz = nz0;
  col_rows.clear(); col_off.assign(nt + 1, 0);
  pairs.clear(); pair_off.assign(nt + 1, 0);
  for (int k = 0; k < nt; ++k) {
    nz[(size_t)k * nt + k] = 1;
    col_off[k] = (int)col_rows.size();
    std::vector<int> rows;
    for (int I = k + 1; I < nt; ++I)
      if (nz[(size_t)I * nt + k]) rows.push_back(I);
    for (int I : rows) col_rows.push_back(I);
    pair_off[k] = (int)pairs.size();
    // fill-in: (I, J) becomes nonzero when both (I, k) and (J, k) are
    for (size_t a = 0; a < rows.size(); ++a)
      for (size_t b = 0; b <= a; ++b) {
        int I = rows[a], J = rows[b];
        nz[(size_t)I * nt + J] = 1;
        pairs.push_back(make_int2(I, J));
      }
  }
  col_off[nt] = (int)col_rows.size();
  pair_off[nt] = (int)pairs.size();
  row_cols.clear(); row_off.assign(nt + 1, 0);
  for (int I = 0; I < nt; ++I) {
    row_off[I] = (int)row_cols.size();
    for (int J = 0; J < I; ++J)
      if (nz[(size_t)I * nt + J]) row_cols.push_back(J);
  }
  row_off[nt] = (int)row_cols.size();
}

void TilePlan::upload(cudaStream_t s) {
  d_col_rows.upload(col_rows, s);
  d_row_cols.upload(row_cols, s);
  d_pairs.upload(pairs, s);
}

// ------------------------------------------------------------------------------------------------ kernels
__global__ void k_copy_diag(const double* A, int npad, double* diag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npad) diag[i] = A[(size_t)i * npad + i];
}

__global__ void k_zero_zp_rows(double* A, int npad, const int* zp) {
  int j = blockIdx.x;                 // row
  if (!zp[j]) return;
  for (int c = threadIdx.x; c < npad; c += blockDim.x) A[(size_t)c * npad + j] = 0.0;
}

// Factor the diagonal tile k in place (one CTA, 256 threads).  Square-root-free inside the loop (a dependent
// FP64 divide costs ~450 cycles and a square root ~700 on this GPU): step j scales the remaining column by the
// pivot's reciprocal (multipliers l_r = a_rj / d_j), the trailing update is one FMA per entry with the unscaled
// column, a_rc -= l_r a_cj, and every column is scaled by 1 / sqrt(d_j) once at the end, in parallel, giving
// L = L_unit D^{1/2}.  One step of lookahead: thread 0 updates the next diagonal entry first and forms its
// reciprocal while the other threads finish the update.  Zero pivots (d_j <= tol * diag0_j, or not finite) get
// a zero multiplier column (no update) and a zero column of L.
__global__ void __launch_bounds__(256) k_potrf_tile(double* A, int npad, int k, const double* diag0, int* zp,
                                                    double tol) {
  __shared__ double a[TILE][TILE + 1];   // a[row][col]
  __shared__ double thr[TILE];           // tol * diag0 of the tile's dofs
  __shared__ double dd[TILE];            // pivots d_j (0 for zero pivots), then 1 / sqrt(d_j)
  __shared__ double lcol[TILE];          // multipliers of the current step
  __shared__ double s_rinv;
  const int tid = threadIdx.x;
  double* T = A + (size_t)k * TILE * npad + (size_t)k * TILE;
  for (int idx = tid; idx < TILE * TILE; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    a[r][c] = T[(size_t)c * npad + r];
  }
  if (tid < TILE) thr[tid] = tol * diag0[k * TILE + tid];
  __syncthreads();
  if (tid == 0) {
    const double d = a[0][0];
    const bool zero = !(d > thr[0]);   // also catches NaN and negative roundoff
    dd[0] = zero ? 0.0 : d;
    s_rinv = zero ? 0.0 : 1.0 / d;
  }
  __syncthreads();
  const int rr = tid % TILE, cg = tid / TILE;   // update: row rr, columns j+1+cg, j+5+cg, ...
  for (int j = 0; j + 1 < TILE; ++j) {
    const double rinv = s_rinv;
    for (int r = j + 1 + tid; r < TILE; r += 256) lcol[r] = a[r][j] * rinv;
    __syncthreads();
    if (tid == 0) {   // lookahead: the next pivot and its reciprocal
      const double d = fma(-lcol[j + 1], a[j + 1][j], a[j + 1][j + 1]);
      a[j + 1][j + 1] = d;
      const bool zero = !(d > thr[j + 1]);
      dd[j + 1] = zero ? 0.0 : d;
      s_rinv = zero ? 0.0 : 1.0 / d;
    }
    if (rr > j) {
      const double lr = lcol[rr];
      for (int c = j + 1 + cg; c <= rr; c += 4)
        if (c != j + 1 || rr != j + 1) a[rr][c] = fma(-lr, a[c][j], a[rr][c]);
    }
    __syncthreads();
  }
  if (tid < TILE) {
    const int gj = k * TILE + tid;
    const double d = dd[tid];
    zp[gj] = d > 0.0 ? 0 : 1;
    dd[tid] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
  __syncthreads();
  for (int idx = tid; idx < TILE * TILE; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    T[(size_t)c * npad + r] = (r >= c) ? a[r][c] * dd[c] : 0.0;
  }
}

// For step k: tiles (I, k), I in rows[0..cnt): L_Ik = A_Ik L_kk^{-T} (zero-pivot columns -> 0).  The rows of
// a tile are independent, so grid.y splits each tile into four 16-row blocks (more SMs on the FP64 work).
constexpr int TR_ROWS = 16;
__global__ void __launch_bounds__(256) k_trsm_tiles(double* A, int npad, int k, const int* rows, const int* zp) {
  __shared__ double l[TILE][TILE + 1];
  __shared__ double x[TR_ROWS][TILE + 1];
  __shared__ double rinv[TILE];
  const int tid = threadIdx.x;
  const int I = rows[blockIdx.x];
  const int rb = blockIdx.y * TR_ROWS;
  const double* D = A + (size_t)k * TILE * npad + (size_t)k * TILE;
  double* X = A + (size_t)k * TILE * npad + (size_t)I * TILE + rb;
  for (int idx = tid; idx < TILE * TILE; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    l[r][c] = D[(size_t)c * npad + r];
  }
  for (int idx = tid; idx < TR_ROWS * TILE; idx += 256) {
    int r = idx % TR_ROWS, c = idx / TR_ROWS;
    x[r][c] = X[(size_t)c * npad + r];
  }
  __syncthreads();
  if (tid < TILE) rinv[tid] = zp[k * TILE + tid] != 0 ? 0.0 : 1.0 / l[tid][tid];
  __syncthreads();
  for (int j = 0; j < TILE; ++j) {
    if (tid < TR_ROWS) x[tid][j] *= rinv[j];
    __syncthreads();
    const int w = TILE - 1 - j;
    for (int idx = tid; idx < w * TR_ROWS; idx += 256) {
      int c = j + 1 + idx / TR_ROWS, r = idx % TR_ROWS;
      x[r][c] -= x[r][j] * l[c][j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < TR_ROWS * TILE; idx += 256) {
    int r = idx % TR_ROWS, c = idx / TR_ROWS;
    X[(size_t)c * npad + r] = x[r][c];
  }
}

// For step k: A_IJ -= L_Ik L_Jk^T for each pair (I, J).  grid.y: the four 32 x 32 quadrants of the output
// tile (2 x 2 per thread), the strictly upper quadrant of a diagonal tile skipped (never read).
__global__ void __launch_bounds__(256) k_update_pairs(double* A, int npad, int k, const int2* pairs) {
  __shared__ double sa[16][33];   // [kk][row]
  __shared__ double sb[16][33];
  const int tid = threadIdx.x;
  const int2 pr = pairs[blockIdx.x];
  const int I = pr.x, J = pr.y;
  const int qr = (blockIdx.y & 1) * 32, qc = (blockIdx.y >> 1) * 32;
  if (I == J && qr < qc) return;
  const double* LI = A + (size_t)k * TILE * npad + (size_t)I * TILE + qr;
  const double* LJ = A + (size_t)k * TILE * npad + (size_t)J * TILE + qc;
  const int tx = tid % 16, ty = tid / 16;     // rows ty*2.., cols tx*2..
  double acc[2][2] = {};
  for (int kk0 = 0; kk0 < TILE; kk0 += 16) {
    for (int idx = tid; idx < 16 * 32; idx += 256) {
      int r = idx % 32, kk = idx / 32;
      sa[kk][r] = LI[(size_t)(kk0 + kk) * npad + r];
      sb[kk][r] = LJ[(size_t)(kk0 + kk) * npad + r];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const double a0 = sa[kk][ty * 2], a1 = sa[kk][ty * 2 + 1];
      const double b0 = sb[kk][tx * 2], b1 = sb[kk][tx * 2 + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  double* C = A + (size_t)(J * TILE + qc) * npad + (size_t)I * TILE + qr;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) C[(size_t)(tx * 2 + q) * npad + ty * 2 + p] -= acc[p][q];
}

// Inverse of every diagonal tile, all tiles in parallel (one CTA per tile): Dinv_J = L_JJ^{-1} by forward
// substitution on the identity, zero-pivot rows and columns left at 0 (the same linear map as solving with
// the zero pivot skipped).  Stored column-major, 64 x 64 per tile.
__global__ void __launch_bounds__(256) k_tile_inverse(const double* L, int npad, const int* zp, double* Dinv) {
  __shared__ double l[TILE][TILE + 1];
  __shared__ double x[TILE][TILE + 1];
  const int tid = threadIdx.x;
  const int J = blockIdx.x;
  const double* D = L + (size_t)J * TILE * npad + (size_t)J * TILE;
  for (int idx = tid; idx < TILE * TILE; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    l[r][c] = D[(size_t)c * npad + r];
    x[r][c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  __shared__ double rinv[TILE];
  if (tid < TILE) rinv[tid] = zp[J * TILE + tid] != 0 ? 0.0 : 1.0 / l[tid][tid];
  __syncthreads();
  for (int j = 0; j < TILE; ++j) {
    if (tid < TILE) x[j][tid] *= rinv[j];
    __syncthreads();
    for (int idx = tid; idx < (TILE - 1 - j) * TILE; idx += 256) {
      int r = j + 1 + idx / TILE, c = idx % TILE;
      x[r][c] -= l[r][j] * x[j][c];
    }
    __syncthreads();
  }
  double* out = Dinv + (size_t)J * TILE * TILE;
  for (int idx = tid; idx < TILE * TILE; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    out[(size_t)c * TILE + r] = x[r][c];
  }
}

// X_J <- Dinv_J X_J (forward) or Dinv_J^T X_J (backward) for a chunk of RC right-hand sides (64 RC / 256
// outputs per thread).  Narrow solves use RC = 4 so that their FP64 work spreads over many SMs; every CTA owns
// its right-hand sides, so the in-place update is race-free.
template <int RC>
__global__ void __launch_bounds__(256) k_tri_diag_inv(const double* __restrict__ Dinv, int J, double* X, int ldx,
                                                      int nrhs, int trans) {
  constexpr int RPT = TILE * RC / 256, RS = 256 / RC;
  __shared__ double a[TILE][TILE + 1];   // a[r][c] = op(Dinv_J)(r, c)
  __shared__ double x[TILE][RC + 1];     // x[row][rhs]
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * RC;
  const double* D = Dinv + (size_t)J * TILE * TILE;
  for (int idx = tid; idx < TILE * TILE; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    const double v = D[(size_t)c * TILE + r];   // Dinv(r, c)
    if (trans) a[c][r] = v; else a[r][c] = v;
  }
  for (int idx = tid; idx < TILE * RC; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    x[r][c] = (c0 + c < nrhs) ? X[(size_t)(c0 + c) * ldx + (size_t)J * TILE + r] : 0.0;
  }
  __syncthreads();
  const int tx = tid % RC, ty = tid / RC;   // rhs tx, rows ty + RS u
  double acc[RPT] = {};
#pragma unroll 8
  for (int q = 0; q < TILE; ++q) {
    const double b = x[q][tx];
#pragma unroll
    for (int u = 0; u < RPT; ++u) acc[u] = fma(a[ty + RS * u][q], b, acc[u]);
  }
  const int c = c0 + tx;
  if (c < nrhs) {
#pragma unroll
    for (int u = 0; u < RPT; ++u) X[(size_t)c * ldx + (size_t)J * TILE + ty + RS * u] = acc[u];
  }
}

// Triangular solve on one diagonal tile J for a chunk of 64 right-hand sides (blockIdx.x).
__global__ void __launch_bounds__(256) k_tri_diag(const double* L, int npad, int J, const int* zp, double* X,
                                                  int ldx, int nrhs, int trans) {
  __shared__ double l[TILE][TILE + 1];
  __shared__ double x[TILE][TILE + 1];   // x[row][rhs]
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * TILE;
  const double* D = L + (size_t)J * TILE * npad + (size_t)J * TILE;
  for (int idx = tid; idx < TILE * TILE; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    l[r][c] = D[(size_t)c * npad + r];
    x[r][c] = (c0 + c < nrhs) ? X[(size_t)(c0 + c) * ldx + (size_t)J * TILE + r] : 0.0;
  }
  __syncthreads();
  __shared__ double rinv[TILE];
  if (tid < TILE) rinv[tid] = zp[J * TILE + tid] != 0 ? 0.0 : 1.0 / l[tid][tid];
  __syncthreads();
  if (!trans) {
    for (int j = 0; j < TILE; ++j) {
      if (tid < TILE) x[j][tid] *= rinv[j];
      __syncthreads();
      for (int idx = tid; idx < (TILE - 1 - j) * TILE; idx += 256) {
        int r = j + 1 + idx / TILE, c = idx % TILE;
        x[r][c] -= l[r][j] * x[j][c];
      }
      __syncthreads();
    }
  } else {
    for (int j = TILE - 1; j >= 0; --j) {
      if (tid < TILE) x[j][tid] *= rinv[j];
      __syncthreads();
      for (int idx = tid; idx < j * TILE; idx += 256) {
        int r = idx / TILE, c = idx % TILE;   // rows r < j
        x[r][c] -= l[j][r] * x[j][c];
      }
      __syncthreads();
    }
  }
  for (int idx = tid; idx < TILE * TILE; idx += 256) {
    int r = idx % TILE, c = idx / TILE;
    if (c0 + c < nrhs) X[(size_t)(c0 + c) * ldx + (size_t)J * TILE + r] = x[r][c];
  }
}

// After solving tile J: X_I -= L_IJ X_J (forward, I in list) or X_I -= L_JI^T X_J (backward, I in list).
// grid (list count, chunks of 16 right-hand sides, four 16-row blocks): 16 rows x 16 rhs per CTA, one output
// per thread, so that narrow solves (one column per occurrence) spread their FP64 work over many SMs.
constexpr int TU_RHS = 16;
__global__ void __launch_bounds__(256) k_tri_update(const double* L, int npad, int J, const int* list, double* X,
                                                    int ldx, int nrhs, int trans) {
  __shared__ double sa[16][17];        // [kk][row of output]
  __shared__ double sb[16][TU_RHS + 1]; // [kk][rhs]
  const int tid = threadIdx.x;
  const int I = list[blockIdx.x];
  const int c0 = blockIdx.y * TU_RHS;
  const int rb = blockIdx.z * 16;
  const int tx = tid % 16, ty = tid / 16;   // rhs tx, row ty
  double acc = 0.0;
  for (int kk0 = 0; kk0 < TILE; kk0 += 16) {
    if (!trans) {
      const int r = tid % 16, kk = tid / 16;
      sa[kk][r] = L[(size_t)(J * TILE + kk0 + kk) * npad + I * TILE + rb + r];
    } else {
      const int kk = tid % 16, r = tid / 16;
      sa[kk][r] = L[(size_t)(I * TILE + rb + r) * npad + J * TILE + kk0 + kk];
    }
    {
      const int k2 = tid % 16, c = tid / 16;
      sb[k2][c] = (c0 + c < nrhs) ? X[(size_t)(c0 + c) * ldx + (size_t)J * TILE + kk0 + k2] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fma(sa[kk][ty], sb[kk][tx], acc);
    __syncthreads();
  }
  const int c = c0 + tx;
  if (c < nrhs) X[(size_t)c * ldx + (size_t)I * TILE + rb + ty] -= acc;
}

// Generic strided GEMM, 32x32 output tile per CTA, 2x2 per thread (small FP64 products: more CTAs).
// 32 x 32 output tile per CTA.  With part != nullptr the reduction dimension is split: CTA z sums k in
// [z * kc, min(K, (z + 1) * kc)) and stores its raw sum in part[z][m][n] (k_gemm_f64_sum_parts finishes).
__global__ void __launch_bounds__(256) k_gemm_f64_32(int M, int N, int K, double alpha, const double* __restrict__ A,
                                                     long long sAm, long long sAk, const double* __restrict__ B,
                                                     long long sBk, long long sBn, double beta, double* C,
                                                     long long sCm, long long sCn, double* part, int kc) {
  __shared__ double sa[32][33];
  __shared__ double sb[32][33];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  const int tx = tid % 16, ty = tid / 16;
  const int kbeg = part ? (int)blockIdx.z * kc : 0;
  if (part) K = min(K, kbeg + kc);
  double acc[2][2] = {};
  for (int k0 = kbeg; k0 < K; k0 += 32) {
    for (int idx = tid; idx < 32 * 32; idx += 256) {
      int r, kk;
      if (sAk == 1) { kk = idx % 32; r = idx / 32; } else { r = idx % 32; kk = idx / 32; }
      const int m = m0 + r, k = k0 + kk;
      sa[kk][r] = (m < M && k < K) ? A[m * sAm + k * sAk] : 0.0;
      int c, k2;
      if (sBk == 1) { k2 = idx % 32; c = idx / 32; } else { c = idx % 32; k2 = idx / 32; }
      const int n = n0 + c, kb = k0 + k2;
      sb[k2][c] = (n < N && kb < K) ? B[kb * sBk + n * sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double a0 = sa[kk][ty * 2], a1 = sa[kk][ty * 2 + 1];
      const double b0 = sb[kk][tx * 2], b1 = sb[kk][tx * 2 + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int m = m0 + ty * 2 + p;
    if (m >= M) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int n = n0 + tx * 2 + q;
      if (n >= N) continue;
      if (part) {
        part[((size_t)blockIdx.z * M + m) * N + n] = acc[p][q];
        continue;
      }
      double* c = C + m * sCm + n * sCn;
      *c = alpha * acc[p][q] + (beta == 0.0 ? 0.0 : beta * *c);
    }
  }
}

// C = alpha * (sum of the split partials, in split order) + beta * C
__global__ void k_gemm_f64_sum_parts(int M, int N, int splits, const double* __restrict__ part, double alpha,
                                     double beta, double* C, long long sCm, long long sCn) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long mn = (long long)M * N;
  if (i >= mn) return;
  double acc = 0.0;
  for (int z = 0; z < splits; ++z) acc += part[z * mn + i];
  const long long m = i / N, n = i % N;
  double* c = C + m * sCm + n * sCn;
  *c = alpha * acc + (beta == 0.0 ? 0.0 : beta * *c);
}

// Generic strided GEMM, 64x64 output tile per CTA, 4x4 per thread, FP64.
__global__ void __launch_bounds__(256) k_gemm_f64(int M, int N, int K, double alpha, const double* __restrict__ A,
                                                  long long sAm, long long sAk, const double* __restrict__ B,
                                                  long long sBk, long long sBn, double beta, double* C,
                                                  long long sCm, long long sCn) {
  __shared__ double sa[16][TILE + 1];
  __shared__ double sb[16][TILE + 1];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.x * TILE, n0 = blockIdx.y * TILE;
  const int tx = tid % 16, ty = tid / 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int idx = tid; idx < 16 * TILE; idx += 256) {
      int r, kk;
      if (sAk == 1) { kk = idx % 16; r = idx / 16; } else { r = idx % TILE; kk = idx / TILE; }
      int m = m0 + r, k = k0 + kk;
      sa[kk][r] = (m < M && k < K) ? A[m * sAm + k * sAk] : 0.0;
      int c, k2;
      if (sBk == 1) { k2 = idx % 16; c = idx / 16; } else { c = idx % TILE; k2 = idx / TILE; }
      int n = n0 + c, kb = k0 + k2;
      sb[k2][c] = (n < N && kb < K) ? B[kb * sBk + n * sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { av[q] = sa[kk][ty * 4 + q]; bv[q] = sb[kk][tx * 4 + q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(av[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int m = m0 + ty * 4 + p;
    if (m >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int n = n0 + tx * 4 + q;
      if (n >= N) continue;
      double* c = C + m * sCm + n * sCn;
      *c = alpha * acc[p][q] + (beta == 0.0 ? 0.0 : beta * *c);
    }
  }
}

// C = X^T X for a lower-triangular X (column-major, ld), the product S^+ = L_S^{-T} L_S^{-1} of the pattern
// set-up.  One CTA per lower output tile (I >= J) of 64 x 64, 4 x 4 outputs per thread: C_IJ sums
// X(k, i) X(k, j) over rows k >= 64 I only (X(k, i) = 0 for k < i), and the tile is written to C and, mirrored,
// to C_JI.  A third of the flops of the dense product (triangular operand, symmetric result).
__global__ void __launch_bounds__(256) k_lauum(const double* __restrict__ X, int ld, int krows, int n_out,
                                               double* __restrict__ C, int ldc) {
  __shared__ double sa[16][TILE + 1];   // [kk][i]
  __shared__ double sb[16][TILE + 1];   // [kk][j]
  // lower tile index -> (I, J), I >= J: blockIdx.x = I (I + 1) / 2 + J
  const int t = blockIdx.x;
  int I = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  while (I * (I + 1) / 2 > t) --I;
  const int J = t - I * (I + 1) / 2;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const double* XI = X + (size_t)I * TILE * ld;
  const double* XJ = X + (size_t)J * TILE * ld;
  double acc[4][4] = {};
  for (int k0 = I * TILE; k0 < krows; k0 += 16) {
    for (int idx = tid; idx < 16 * TILE; idx += 256) {
      const int kk = idx % 16, c = idx / 16;
      const int k = k0 + kk;
      sa[kk][c] = k < krows ? XI[(size_t)c * ld + k] : 0.0;
      sb[kk][c] = k < krows ? XJ[(size_t)c * ld + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { av[q] = sa[kk][ty * 4 + q]; bv[q] = sb[kk][tx * 4 + q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(av[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = I * TILE + ty * 4 + p;
    if (i >= n_out) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = J * TILE + tx * 4 + q;
      if (j >= n_out) continue;
      C[(size_t)i * ldc + j] = acc[p][q];
      if (I != J) C[(size_t)j * ldc + i] = acc[p][q];
    }
  }
}

// ------------------------------------------------------------------------------------------------ host
void lauum(const double* X, int ld, int krows, int n_out, double* C, int ldc, cudaStream_t s) {
  const int nt = ceil_div(n_out, TILE);
  if (nt <= 0) return;
  k_lauum<<<nt * (nt + 1) / 2, 256, 0, s>>>(X, ld, krows, n_out, C, ldc);
  FETIRP_LAUNCH_CHECK();
}

void copy_diag(const double* A, int npad, double* diag, cudaStream_t s) {
  k_copy_diag<<<ceil_div(npad, 256), 256, 0, s>>>(A, npad, diag);
  FETIRP_LAUNCH_CHECK();
}

void zero_zp_rows(double* A, int npad, const int* zp, cudaStream_t s) {
  k_zero_zp_rows<<<npad, 256, 0, s>>>(A, npad, zp);
  FETIRP_LAUNCH_CHECK();
}

void chol_tiles(double* A, int npad, const TilePlan& plan, const double* diag0, int* zp, double tol,
                cudaStream_t s) {
  for (int k = 0; k < plan.nt; ++k) {
    k_potrf_tile<<<1, 256, 0, s>>>(A, npad, k, diag0, zp, tol);
    FETIRP_LAUNCH_CHECK();
    int nr = plan.col_off[k + 1] - plan.col_off[k];
    if (nr > 0) {
      k_trsm_tiles<<<dim3(nr, TILE / TR_ROWS), 256, 0, s>>>(A, npad, k, plan.d_col_rows.p + plan.col_off[k], zp);
      FETIRP_LAUNCH_CHECK();
    }
    int np = plan.pair_off[k + 1] - plan.pair_off[k];
    if (np > 0) {
      k_update_pairs<<<dim3(np, 4), 256, 0, s>>>(A, npad, k, plan.d_pairs.p + plan.pair_off[k]);
      FETIRP_LAUNCH_CHECK();
    }
  }
  zero_zp_rows(A, npad, zp, s);
}

void tile_inverses(const double* L, int npad, const int* zp, double* Dinv, cudaStream_t s) {
  k_tile_inverse<<<npad / TILE, 256, 0, s>>>(L, npad, zp, Dinv);
  FETIRP_LAUNCH_CHECK();
}

void tri_solve(const double* L, int npad, const TilePlan& plan, const int* zp, double* X, int ldx, int nrhs_all,
               bool trans, cudaStream_t s, const double* Dinv, bool identity_rhs, int stop_tile, int start_tile) {
  if (nrhs_all <= 0) return;
  int nrhs = nrhs_all;
  int chunks = ceil_div(nrhs, TILE);
  auto diag = [&](int J, int tr) {
    if (Dinv && ceil_div(nrhs, 16) < 152) k_tri_diag_inv<4><<<ceil_div(nrhs, 4), 256, 0, s>>>(Dinv, J, X, ldx, nrhs, tr);
    else if (Dinv) k_tri_diag_inv<16><<<ceil_div(nrhs, 16), 256, 0, s>>>(Dinv, J, X, ldx, nrhs, tr);
    else k_tri_diag<<<chunks, 256, 0, s>>>(L, npad, J, zp, X, ldx, nrhs, tr);
  };
  if (!trans) {
    for (int J = std::max(0, start_tile); J < plan.nt; ++J) {
      if (identity_rhs) {   // columns c >= 64 (J + 1) of L^{-1} are still zero in block rows <= J
        nrhs = std::min(nrhs_all, (J + 1) * TILE);
        chunks = ceil_div(nrhs, TILE);
      }
      diag(J, 0);
      FETIRP_LAUNCH_CHECK();
      int nr = plan.col_off[J + 1] - plan.col_off[J];
      if (nr > 0) {
        k_tri_update<<<dim3(nr, ceil_div(nrhs, TU_RHS), TILE / 16), 256, 0, s>>>(L, npad, J, plan.d_col_rows.p + plan.col_off[J],
                                                                      X, ldx, nrhs, 0);
        FETIRP_LAUNCH_CHECK();
      }
    }
  } else {
    const int J0 = std::max(0, stop_tile);
    for (int J = plan.nt - 1; J >= J0; --J) {
      diag(J, 1);
      FETIRP_LAUNCH_CHECK();
      // targets: the block rows I < J of row J (ascending), those >= J0 only
      int b = plan.row_off[J];
      const int e = plan.row_off[J + 1];
      if (J0 > 0)
        b = (int)(std::lower_bound(plan.row_cols.begin() + b, plan.row_cols.begin() + e, J0) - plan.row_cols.begin());
      const int nr = e - b;
      if (nr > 0) {
        k_tri_update<<<dim3(nr, ceil_div(nrhs, TU_RHS), TILE / 16), 256, 0, s>>>(L, npad, J, plan.d_row_cols.p + b,
                                                                      X, ldx, nrhs, 1);
        FETIRP_LAUNCH_CHECK();
      }
    }
  }
}

// Reduction-dimension split of a skinny product: up to eight CTAs per SM (17 KB of shared memory each), >= 256
// terms each; 1 = no split
static int gemm_f64_splits(int M, int N, int K, int* kc_out) {
  const long long t64 = (long long)ceil_div(M, TILE) * ceil_div(N, TILE);
  const long long tiles = (long long)ceil_div(M, 32) * ceil_div(N, 32);
  if (t64 >= 2 * 152 || tiles >= 152 || K < 1024) return 1;
  int splits = (int)std::min<long long>(ceil_div(K, 256), std::max<long long>(1, 8 * 152 / tiles));
  if (splits <= 1) return 1;
  const int kc = ceil_div(ceil_div(K, splits), 32) * 32;
  if (kc_out) *kc_out = kc;
  return ceil_div(K, kc);
}

size_t gemm_f64_scratch(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 0;
  const int splits = gemm_f64_splits(M, N, K, nullptr);
  return splits > 1 ? (size_t)splits * M * N : 0;
}

void gemm_f64(int M, int N, int K, double alpha, const double* A, long long sAm, long long sAk, const double* B,
              long long sBk, long long sBn, double beta, double* C, long long sCm, long long sCn,
              cudaStream_t s, double* scratch, size_t scratch_elems) {
  if (M <= 0 || N <= 0) return;
  dim3 grid(ceil_div(M, TILE), ceil_div(N, TILE));
  if ((long long)grid.x * grid.y < 2 * 152) {   // too few 64x64 tiles to occupy the SMs' FP64 units
    dim3 g32(ceil_div(M, 32), ceil_div(N, 32));
    int kc = 0;
    const int splits = gemm_f64_splits(M, N, K, &kc);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (splits > 1) FETIRP_CUDA(cudaStreamIsCapturing(s, &cap));
    if (splits > 1 && scratch && scratch_elems >= (size_t)splits * M * N && cap == cudaStreamCaptureStatusNone) {
      g32.z = splits;
      k_gemm_f64_32<<<g32, 256, 0, s>>>(M, N, K, alpha, A, sAm, sAk, B, sBk, sBn, beta, C, sCm, sCn, scratch, kc);
      FETIRP_LAUNCH_CHECK();
      const long long mn = (long long)M * N;
      k_gemm_f64_sum_parts<<<(unsigned)((mn + 255) / 256), 256, 0, s>>>(M, N, splits, scratch, alpha, beta, C, sCm,
                                                                         sCn);
      FETIRP_LAUNCH_CHECK();
      return;
    }
    k_gemm_f64_32<<<g32, 256, 0, s>>>(M, N, K, alpha, A, sAm, sAk, B, sBk, sBn, beta, C, sCm, sCn, nullptr, 0);
  } else {
    k_gemm_f64<<<grid, 256, 0, s>>>(M, N, K, alpha, A, sAm, sAk, B, sBk, sBn, beta, C, sCm, sCn);
  }
  FETIRP_LAUNCH_CHECK();
}

}  // namespace fetirp
