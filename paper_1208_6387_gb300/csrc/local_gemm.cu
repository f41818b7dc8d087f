// Local multi-right-hand-side products Z_p = S_p^+ Y_p for every pattern in one launch: every occurrence
// of a pattern (and every multivector column) is one right-hand side of that pattern's one operator
// (the multi-RHS product of the efficient-implementation subsection).  SIMT forms (FP64 DFMA, FP32 FFMA).
#include "ops.cuh"

namespace fetirp {

struct LocalTiles {
  LocalProblem P;
  int tiles_m[MAXP];
  int tile_off[MAXP + 1];
};

template <typename T>
__global__ void __launch_bounds__(256) k_local_gemm(LocalTiles LT) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T sa[BK][BM + 1];   // S(i, j): [j][i]
  __shared__ T sb[BK][BN + 1];   // Y(j, rhs): [j][rhs]
  int p = 0;
  while (p + 1 < LT.P.n_pat && (int)blockIdx.x >= LT.tile_off[p + 1]) ++p;
  const int t = blockIdx.x - LT.tile_off[p];
  const int m0 = (t % LT.tiles_m[p]) * BM, n0 = (t / LT.tiles_m[p]) * BN;
  const int nb = LT.P.n_b[p], nr = LT.P.n_rhs[p];
  const long long ld = LT.P.ld[p];
  const T* S = (const T*)LT.P.S[p];
  const T* Y = (const T*)LT.P.Y[p];
  T* Z = (T*)LT.P.Z[p];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;   // rows tx*4.., rhs ty*4..
  T acc[4][4] = {};
  for (int k0 = 0; k0 < nb; k0 += BK) {
    for (int idx = tid; idx < BK * BM; idx += 256) {
      const int kk = idx % BK, r = idx / BK;
      const int i = m0 + r, j = k0 + kk;
      sa[kk][r] = (i < nb && j < nb) ? S[(size_t)i * nb + j] : T(0);
      const int c = n0 + r;
      sb[kk][r] = (c < nr && j < nb) ? Y[(long long)c * ld + j] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { av[q] = sa[kk][tx * 4 + q]; bv[q] = sb[kk][ty * 4 + q]; }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int c = n0 + ty * 4 + b;
    if (c >= nr) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = m0 + tx * 4 + a;
      if (i < nb) Z[(long long)c * ld + i] = acc[a][b];
    }
  }
}

template <typename T>
static void launch_local(const LocalProblem& P, cudaStream_t s) {
  LocalTiles LT;
  LT.P = P;
  int total = 0;
  for (int p = 0; p < P.n_pat; ++p) {
    LT.tile_off[p] = total;
    LT.tiles_m[p] = ceil_div(P.n_b[p], 64);
    total += LT.tiles_m[p] * ceil_div(P.n_rhs[p], 64);
  }
  LT.tile_off[P.n_pat] = total;
  if (total == 0) return;
  k_local_gemm<T><<<total, 256, 0, s>>>(LT);
  FETIRP_LAUNCH_CHECK();
}

void local_gemm_f64(const LocalProblem& P, cudaStream_t s) { launch_local<double>(P, s); }
void local_gemm_f32(const LocalProblem& P, cudaStream_t s) { launch_local<float>(P, s); }

}  // namespace fetirp
