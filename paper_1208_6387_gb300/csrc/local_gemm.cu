// Local multi-right-hand-side products Z_p = S_p^+ Y_p for every pattern in one launch: every occurrence
// of a pattern (and every multivector column) is one right-hand side of that pattern's one operator
// (the multi-RHS product of the efficient-implementation subsection).  SIMT forms (FP64 DFMA, FP32 FFMA).
#include "ops.cuh"

namespace fetirp {

// One launch over every pattern's tiles.  A(i, j) of pattern p is mode 0: A[i * lda + j] (dense, row-major);
// mode 1: A[j * lda + i] for j <= i, 0 above the diagonal (a lower-triangular factor stored transposed);
// mode 2: A[i * lda + j] for j >= i, 0 below (the transpose of that factor).  The triangular modes skip the
// K steps that lie entirely in the zero triangle.
struct LocalTiles {
  const void* A[MAXP];
  long long lda[MAXP];
  int mode[MAXP];
  const void* Y[MAXP];
  void* Z[MAXP];
  long long ld[MAXP];
  int n_b[MAXP];
  int n_rhs[MAXP];
  int tiles_m[MAXP];
  int tile_off[MAXP + 1];
  int n_pat;
};

template <typename T, int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_local_gemm(LocalTiles LT) {
  constexpr int TM = BM / 16, TN = BN / 16;   // per thread: TM rows x TN right-hand sides
  constexpr int LA = (BK * BM + 255) / 256, LB = (BK * BN + 255) / 256;
  __shared__ T sa[BK][BM + 1];   // A(i, j): [j][i]
  __shared__ T sb[BK][BN + 1];   // Y(j, rhs): [j][rhs]
  int p = 0;
  while (p + 1 < LT.n_pat && (int)blockIdx.x >= LT.tile_off[p + 1]) ++p;
  const int t = blockIdx.x - LT.tile_off[p];
  const int m0 = (t % LT.tiles_m[p]) * BM, n0 = (t / LT.tiles_m[p]) * BN;
  const int nb = LT.n_b[p], nr = LT.n_rhs[p], mode = LT.mode[p];
  const long long ld = LT.ld[p], lda = LT.lda[p];
  const T* A = (const T*)LT.A[p];
  const T* Y = (const T*)LT.Y[p];
  T* Z = (T*)LT.Z[p];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;   // rows tx*TM.., rhs ty*TN..
  // K range holding the tile's nonzeros: mode 1 stops after the tile's last row, mode 2 starts at its first
  const int kbeg = mode == 2 ? m0 / BK * BK : 0;
  const int kend = mode == 1 ? min(nb, m0 + BM) : nb;
  T acc[TM][TN] = {};
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    if (mode == 1) {   // transposed storage: consecutive threads along i
#pragma unroll
      for (int u = 0; u < LA; ++u) {
        const int idx = tid + 256 * u;
        const int r = idx % BM, kk = idx / BM;
        const int i = m0 + r, j = k0 + kk;
        if (idx < BK * BM) sa[kk][r] = (i < nb && j <= i) ? A[(size_t)j * lda + i] : T(0);
      }
    } else {
#pragma unroll
      for (int u = 0; u < LA; ++u) {
        const int idx = tid + 256 * u;
        const int kk = idx % BK, r = idx / BK;
        const int i = m0 + r, j = k0 + kk;
        if (idx < BK * BM) sa[kk][r] = (i < nb && j < nb && (mode == 0 || j >= i)) ? A[(size_t)i * lda + j] : T(0);
      }
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

template <int BM, int BN>
static int plan_tiles(LocalTiles& LT) {
  int total = 0;
  for (int p = 0; p < LT.n_pat; ++p) {
    LT.tile_off[p] = total;
    LT.tiles_m[p] = ceil_div(LT.n_b[p], BM);
    total += LT.tiles_m[p] * ceil_div(LT.n_rhs[p], BN);
  }
  LT.tile_off[LT.n_pat] = total;
  return total;
}

// 64 x 64 tiles (K steps of 16), or, when that tiling would not give every SM a CTA (small problems),
// 32 x 32 or 16 x 16 tiles with K steps of 64: fewer dependent load rounds per CTA, more CTAs.  Triangular
// products ask for four CTAs per SM before taking the large tile: their CTAs' K ranges differ (up to 2x).
template <typename T>
static void launch_tiles(LocalTiles LT, bool triangular, cudaStream_t s) {
  int total = plan_tiles<64, 64>(LT);
  if (total == 0) return;
  if (total >= (triangular ? 4 : 1) * 152) {
    k_local_gemm<T, 64, 64, 16><<<total, 256, 0, s>>>(LT);
  } else if ((total = plan_tiles<32, 32>(LT)) >= 152) {
    k_local_gemm<T, 32, 32, 64><<<total, 256, 0, s>>>(LT);
  } else {
    total = plan_tiles<16, 16>(LT);
    k_local_gemm<T, 16, 16, 64><<<total, 256, 0, s>>>(LT);
  }
  FETIRP_LAUNCH_CHECK();
}

template <typename T>
static void launch_local(const LocalProblem& P, cudaStream_t s) {
  // first launch: Z = S Y for the dense patterns, W = Lam Y for the factored ones; second: Z = Lam^T W
  LocalTiles L1{}, L2{};
  L1.n_pat = L2.n_pat = P.n_pat;
  bool factored = false;
  for (int p = 0; p < P.n_pat; ++p) {
    const bool f = P.X[p] != nullptr;
    if (f && sizeof(T) != 8) throw Error(1, "the factored local product is FP64 only");
    factored = factored || f;
    L1.n_b[p] = L2.n_b[p] = P.n_b[p];
    L1.ld[p] = L2.ld[p] = P.ld[p];
    L1.n_rhs[p] = P.n_rhs[p];
    L1.A[p] = f ? (const void*)P.X[p] : P.S[p];
    L1.lda[p] = f ? P.ldx[p] : P.n_b[p];
    L1.mode[p] = f ? 1 : 0;
    L1.Y[p] = P.Y[p];
    L1.Z[p] = f ? (void*)P.W[p] : P.Z[p];
    L2.n_rhs[p] = f ? P.n_rhs[p] : 0;
    L2.A[p] = P.X[p];
    L2.lda[p] = P.ldx[p];
    L2.mode[p] = 2;
    L2.Y[p] = P.W[p];
    L2.Z[p] = P.Z[p];
  }
  launch_tiles<T>(L1, factored, s);
  if (factored) launch_tiles<T>(L2, true, s);
}

void local_gemm_f64(const LocalProblem& P, cudaStream_t s) { launch_local<double>(P, s); }
void local_gemm_f32(const LocalProblem& P, cudaStream_t s) { launch_local<float>(P, s); }

}  // namespace fetirp
