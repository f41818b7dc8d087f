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

template <typename T, int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_local_gemm(LocalTiles LT) {
  constexpr int TM = BM / 16, TN = BN / 16;   // per thread: TM rows x TN right-hand sides
  constexpr int LA = (BK * BM + 255) / 256, LB = (BK * BN + 255) / 256;
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
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;   // rows tx*TM.., rhs ty*TN..
  T acc[TM][TN] = {};
  for (int k0 = 0; k0 < nb; k0 += BK) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int idx = tid + 256 * u;
      const int kk = idx % BK, r = idx / BK;
      const int i = m0 + r, j = k0 + kk;
      if (idx < BK * BM) sa[kk][r] = (i < nb && j < nb) ? S[(size_t)i * nb + j] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int idx = tid + 256 * u;
      const int kk = idx % BK, r = idx / BK;
      const int c = n0 + r, j = k0 + kk;
      if (idx < BK * BN) sb[kk][r] = (c < nr && j < nb) ? Y[(long long)c * ld + j] : T(0);
    }
    __syncthreads();
#pragma unroll 16
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int q = 0; q < TM; ++q) av[q] = sa[kk][tx * TM + q];
#pragma unroll
      for (int q = 0; q < TN; ++q) bv[q] = sb[kk][ty * TN + q];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < TN; ++b) {
    const int c = n0 + ty * TN + b;
    if (c >= nr) continue;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int i = m0 + tx * TM + a;
      if (i < nb) Z[(long long)c * ld + i] = acc[a][b];
    }
  }
}

template <typename T, int BM, int BN>
static int plan_tiles(const LocalProblem& P, LocalTiles& LT) {
  LT.P = P;
  int total = 0;
  for (int p = 0; p < P.n_pat; ++p) {
    LT.tile_off[p] = total;
    LT.tiles_m[p] = ceil_div(P.n_b[p], BM);
    total += LT.tiles_m[p] * ceil_div(P.n_rhs[p], BN);
  }
  LT.tile_off[P.n_pat] = total;
  return total;
}

// 64 x 64 tiles (K steps of 16), or, when that tiling would not give every SM a CTA (small problems),
// 32 x 32 or 16 x 16 tiles with K steps of 64: fewer dependent load rounds per CTA, more CTAs.
template <typename T>
static void launch_local(const LocalProblem& P, cudaStream_t s) {
  LocalTiles LT;
  int total = plan_tiles<T, 64, 64>(P, LT);
  if (total == 0) return;
  if (total >= 152) {
    k_local_gemm<T, 64, 64, 16><<<total, 256, 0, s>>>(LT);
  } else if ((total = plan_tiles<T, 32, 32>(P, LT)) >= 152) {
    k_local_gemm<T, 32, 32, 64><<<total, 256, 0, s>>>(LT);
  } else {
    total = plan_tiles<T, 16, 16>(P, LT);
    k_local_gemm<T, 16, 16, 64><<<total, 256, 0, s>>>(LT);
  }
  FETIRP_LAUNCH_CHECK();
}

void local_gemm_f64(const LocalProblem& P, cudaStream_t s) { launch_local<double>(P, s); }
void local_gemm_f32(const LocalProblem& P, cudaStream_t s) { launch_local<float>(P, s); }

}  // namespace fetirp
