// Persistent block ORTHODIR iteration for latency-bound structures (small n_lambda, k <= 32, SIMT local
// products).  One cooperative launch runs whole iterations of Table 1 (right) with full reorthogonalisation
// and F-normalisation; the per-kernel launch and ramp cost of the multi-kernel form (about sixteen launches
// per iteration) is replaced by eight grid barriers.  Phases of one iteration (a = stored history columns):
//   P1  Gram items of C = Q_h^T S(r) and X = G^T S(r) per occurrence (one item list), Z = S(r)
//   P2  C = sum of the Gram chunks, A = (G^T G)^{-1} X
//   P3  Z <- Z - G A - W_h C   (projection and reorthogonalisation, split over the history columns)
//   P4  Z_loc = S^+ gather(Z) (local products of all occurrences; the gather is done while staging)
//   P5  X = G^T scatter(Z_loc)            P6  A = (G^T G)^{-1} X
//   P7  Q = scatter(Z_loc) - G A, eta partials [Z^T Q | Z^T r]; a two-level reduction, then the last CTA
//       normalises (T, alpha)
//   P8  W_h[:, a..a+k) = Z T, Q_h[...] = Q T, lambda += Z T alpha, r -= Q T alpha, ||r||^2 partials
// The residual test runs on the device at the start of every iteration.  Data written by other CTAs is read
// after a grid barrier: every CTA's writes happen before its __threadfence() and arrival, and the polling thread
// observes the new generation, then executes a fence.acq_rel.gpu before the CTA-wide __syncthreads() that
// releases the other threads, so their later loads of the other CTAs' data are ordered after those writes in
// the PTX memory model (acquire at GPU scope, made CTA-wide by the barrier).  No loads of mutable data use the
// non-coherent (ld.global.nc / __ldg) path.  The file is also compiled with -Xptxas -dlcm=cg (global loads
// cached in L2 only) as a second guard.  Every barrier wait is bounded by A.timeout_ns (globaltimer); an
// expired wait sets *A.err and the CTA returns, so a failure ends the launch instead of hanging it.
#include <mutex>

#include "ds.cuh"
#include "ops.cuh"
#include "normalise_warp.cuh"

namespace fetirp {
namespace {

constexpr int PT = 256;                      // threads per CTA
constexpr int P_GS_ROWS = 128;
constexpr int P_TU_ROWS = 64, P_TU_CH = 32;
constexpr int P_GTV_COLS = 8, P_MAXKD = 6;
constexpr int P_LT = 16, P_LK = 64;          // local products: 16 x 16 output tiles, K steps of 64
constexpr int P_SMEM = 26 * 1024;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier on A.bar = {count, generation}: thread 0 of every CTA arrives, the last arrival resets the
// count and advances the generation, the others poll the generation with a time limit.
__device__ bool grid_sync(const PersistArgs& A) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = A.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned prev = atomicAdd(A.bar, 1u);
    if (prev == (unsigned)(A.ncta + A.missing) - 1) {
      atomicExch(A.bar, 0u);
      __threadfence();
      atomicAdd(A.bar + 1, 1u);
    } else {
      const unsigned long long t0 = gtimer();
      while (*gen == g) {
        if (gtimer() - t0 > A.timeout_ns) {
          atomicExch(A.err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    asm volatile("fence.acq_rel.gpu;" ::: "memory");   // acquire: the other CTAs' writes before their arrival
    if (*(volatile int*)A.err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// S(r)[row][g]: r[row] / (slots of the row) for each of the row's slots in column g (the split of P1)
__device__ __forceinline__ double split_val(const PersistArgs& A, int row, int g) {
  const int g0 = A.row_grp[2 * row], g1 = A.row_grp[2 * row + 1];
  const double w = A.r[row] * A.row_wt[row];
  double z = 0.0;
  if (g0 == g) z += w;
  if (g1 == g) z += w;
  return z;
}

// scatter(Z_loc)[row][g] = sum over the row's slots: sign * Z_loc(slot, g)
template <typename TL>
__device__ __forceinline__ double qraw(const PersistArgs& A, int row, int g) {
  const TL* Z = (const TL*)A.Zbuf;
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int sg = A.L.row_sign[2 * row + e];
    if (sg == 0) continue;
    const double z = neg_if(to_f64(Z[A.row_z[2 * row + e] + (long long)g * A.row_zld[2 * row + e]]), sg < 0);
    acc = e == 0 ? z : acc + z;
  }
  return acc;
}

// (G A)[row][g] = sum over the row's slots: sign * Nb[j] . A[gofs(s)..][g], from the per-row tables (the
// coefficients and the coarse column are loaded independently, then A)
__device__ __forceinline__ double gapply(const PersistArgs& A, int row, int g) {
  const int k = A.k;
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int g0 = A.rowg_gofs[2 * row + e];
    if (g0 < 0) continue;
    const int kd = A.rowg_kd[2 * row + e];   // only the occurrence's own coarse rows of A are read
    const double* c = A.rowg_coef + (size_t)(2 * row + e) * P_MAXKD;
    const double* a = A.Ac + (size_t)g0 * k + g;
    double t = 0.0;
#pragma unroll
    for (int m = 0; m < P_MAXKD; ++m)
      if (m < kd) t = fma(c[m], a[(size_t)m * k], t);
    acc += t;
  }
  return acc;
}

// X[gofs(s)+m][g] = sum over the slots j of s: Nb[j][m] * y(j, g), y the trace of V on the slot's links, where
// V is S(r) (from_split) or scatter(Z_loc).  Item: (occurrence, 8 columns); the threads split the slots and the
// per-thread sums are added in a fixed order (deterministic).
template <typename TL, bool from_split>
__device__ void gtv_item(const PersistArgs& A, int it, unsigned char* smem) {
  const Layout& L = A.L;
  const int k = A.k;
  double (*red)[P_MAXKD] = reinterpret_cast<double (*)[P_MAXKD]>(smem);
  const int cgroups = (k + P_GTV_COLS - 1) / P_GTV_COLS;
  const int t = threadIdx.x;
  const int s = it / cgroups, gbase = (it % cgroups) * P_GTV_COLS;
  const int p = L.occ_pat[s];
  const int kd = L.kdim[p];
  const double* Nb = L.Nb[p];
  const int b0 = L.occ_obase[s], nb = L.occ_obase[s + 1] - b0;
  const int g0 = L.occ_gofs[s];
  const int kk = min(P_GTV_COLS, k - gbase);
  const int lanes = PT / kk;
  const int g = gbase + t % kk, sub = t / kk;
  double acc[P_MAXKD] = {};
  if (sub < lanes) {
    for (int j = sub; j < nb; j += lanes) {
      const int slot = b0 + j;
      double y = 0.0;
      for (int e = 0; e < L.ell_w; ++e) {
        const int sg = L.ell_sign[(size_t)slot * L.ell_w + e];
        if (sg == 0) continue;
        const int row = L.ell_row[(size_t)slot * L.ell_w + e];
        const double v = from_split ? split_val(A, row, g) : qraw<TL>(A, row, g);
        y += neg_if(v, sg < 0);
      }
#pragma unroll
      for (int m = 0; m < P_MAXKD; ++m)
        if (m < kd) acc[m] = fma(Nb[(size_t)j * kd + m], y, acc[m]);
    }
  }
  __syncthreads();   // the previous item's reads of the shared buffer are done
#pragma unroll
  for (int m = 0; m < P_MAXKD; ++m) red[t][m] = acc[m];
  __syncthreads();
  if (t < kk) {
    for (int m = 0; m < kd; ++m) {
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
      int q = 0;
      for (; q + 3 < lanes; q += 4) {
        v0 += red[q * kk + t][m];
        v1 += red[(q + 1) * kk + t][m];
        v2 += red[(q + 2) * kk + t][m];
        v3 += red[(q + 3) * kk + t][m];
      }
      for (; q < lanes; ++q) v0 += red[q * kk + t][m];
      A.Xc[(size_t)(g0 + m) * k + gbase + t] = (v0 + v1) + (v2 + v3);
    }
  }
}

template <typename TL, bool from_split>
__device__ void phase_gtv(const PersistArgs& A, unsigned char* smem) {
  const int items = A.L.n_occ * ((A.k + P_GTV_COLS - 1) / P_GTV_COLS);
  for (int it = blockIdx.x; it < items; it += A.ncta) gtv_item<TL, from_split>(A, it, smem);
}

// C partials of Q_h^T S(r).  Item: (128 history columns, group, 128-row chunk); the chunk's (row, w r[row]) pairs
// are staged in shared memory, the 8 warps take every 8th row, each lane four columns, the warp sums are added
// in warp order (deterministic); FP32 history: double-single sums on the FP32 pipe (see the split Gram kernel).
constexpr int P_GC = 128;
template <typename TH>
__device__ void gram_item(const PersistArgs& A, int a, int it, unsigned char* smem) {
  int* srow = reinterpret_cast<int*>(smem);
  double* sw = reinterpret_cast<double*>(smem + 512);
  float* swh = reinterpret_cast<float*>(smem + 512 + 1024);
  float* swl = swh + P_GS_ROWS;
  double (*red)[P_GC] = reinterpret_cast<double (*)[P_GC]>(smem + 512 + 1024 + 1024);
  const TH* Qh = (const TH*)A.Qh;
  const int k = A.k;   // also the history block width
  const int ctiles = (a + P_GC - 1) / P_GC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ct = it % ctiles, rest = it / ctiles, g = rest % k, ch = rest / k;
  const int e0 = A.grp_ptr[g] + ch * P_GS_ROWS, e1 = min(A.grp_ptr[g + 1], e0 + P_GS_ROWS);
  const int cnt = max(0, e1 - e0);
  __syncthreads();
  if (tid < cnt) {
    const int row = A.grp_row[e0 + tid];
    const double v = A.grp_w[e0 + tid] * A.r[row];
    srow[tid] = row;
    sw[tid] = v;
    d2ds(v, swh[tid], swl[tid]);
  }
  __syncthreads();
  bool ok[4];
  const TH* qp[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = ct * P_GC + lane + 32 * u;
    ok[u] = c < a;
    qp[u] = Qh + hist_col(ok[u] ? c : 0, A.n, k);
  }
  double res[4];
  if (sizeof(TH) == 4) {
    float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int i = warp; i < cnt; i += 8) {
      const size_t ro = (size_t)srow[i] * k;
      const float sh = swh[i], sl = swl[i];
      float qv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) qv[u] = ok[u] ? (float)qp[u][ro] : 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float pp = __fmul_rn(qv[u], sh), e = fmaf(qv[u], sh, -pp), tt = fmaf(qv[u], sl, e);
        const float uu = __fadd_rn(h[u], pp), bb = __fsub_rn(uu, h[u]);
        l[u] = __fadd_rn(l[u], __fadd_rn(__fadd_rn(__fsub_rn(h[u], __fsub_rn(uu, bb)), __fsub_rn(pp, bb)), tt));
        h[u] = uu;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) res[u] = ds2d(h[u], l[u]);
  } else {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int i = warp; i < cnt; i += 8) {
      const size_t ro = (size_t)srow[i] * k;
      const double wv = sw[i];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(wv, ok[u] ? (double)qp[u][ro] : 0.0, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) res[u] = acc[u];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) red[warp][lane + 32 * u] = res[u];
  __syncthreads();
  if (tid < P_GC) {
    const int cc = ct * P_GC + tid;
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += red[w][tid];
    if (cc < a) A.gram_part[((size_t)ch * a + cc) * k + g] = v;
  }
}

// P1: the Gram items and the G^T S(r) items as one list (balanced over the CTAs), then Z = S(r)
template <typename TH, typename TL>
__device__ void phase_one(const PersistArgs& A, int a, unsigned char* smem) {
  const int n_gtv = A.L.n_G > 0 ? A.L.n_occ * ((A.k + P_GTV_COLS - 1) / P_GTV_COLS) : 0;
  const int n_gram = a > 0 ? ((a + P_GC - 1) / P_GC) * A.k * A.gs_chunks : 0;
  for (int it = blockIdx.x; it < n_gtv + n_gram; it += A.ncta) {
    if (it < n_gtv) gtv_item<TL, true>(A, it, smem);
    else gram_item<TH>(A, a, it - n_gtv, smem);
  }
  for (int row = blockIdx.x * PT + threadIdx.x; row < A.n; row += A.ncta * PT) {
    double* z = A.Zr + (size_t)row * A.k;
    for (int g = 0; g < A.k; ++g) z[g] = 0.0;
    const int g0 = A.row_grp[2 * row], g1 = A.row_grp[2 * row + 1];
    const double w = A.r[row] * A.row_wt[row];
    if (g0 >= 0) z[g0] += w;
    if (g1 >= 0) z[g1] += w;
  }
}

// Ac = Ginv Xc (n_G x n_G times n_G x k, FP64): one warp per row, four independent partial sums per lane
__device__ void phase_small_gemm(const PersistArgs& A) {
  const int m = A.L.n_G, k = A.k;
  const int lane = threadIdx.x & 31;
  int kp = 1;
  while (kp < k) kp <<= 1;
  const int slices = 32 / kp;
  const int g = lane % kp, sl = lane / kp;
  for (int row = blockIdx.x * (PT / 32) + (threadIdx.x >> 5); row < m; row += A.ncta * (PT / 32)) {
    const double* a = A.Ginv + (size_t)row * m;
    double acc = 0.0;
    if (g < k) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = sl;
      for (; j + 3 * slices < m; j += 4 * slices) {
        s0 = fma(a[j], A.Xc[(size_t)j * k + g], s0);
        s1 = fma(a[j + slices], A.Xc[(size_t)(j + slices) * k + g], s1);
        s2 = fma(a[j + 2 * slices], A.Xc[(size_t)(j + 2 * slices) * k + g], s2);
        s3 = fma(a[j + 3 * slices], A.Xc[(size_t)(j + 3 * slices) * k + g], s3);
      }
      for (; j < m; j += slices) s0 = fma(a[j], A.Xc[(size_t)j * k + g], s0);
      acc = (s0 + s1) + (s2 + s3);
    }
    for (int off = kp; off < 32; off <<= 1) acc += __shfl_down_sync(FULL, acc, off);
    if (sl == 0 && g < k) A.Ac[(size_t)row * k + g] = acc;
  }
}

// Z[row][g] -= (G A)[row][g] + sum_c W_h[row][c] C[c][g] over c < a.  Items (64-row tile, history split) with
// the same tiling, prefetch and last-CTA split reduction as the stand-alone history update.
template <typename TH, int KP>
__device__ void phase_tall(const PersistArgs& A, int a, unsigned char* smem) {
  constexpr int TXC = KP < 16 ? KP : 16, TY = PT / TXC;
  constexpr int RPT = P_TU_ROWS / TY, CPT = KP / TXC;
  constexpr int LA = P_TU_CH * P_TU_ROWS / PT, LC = (P_TU_CH * KP + PT - 1) / PT;
  TH (*sa)[P_TU_ROWS + 1] = reinterpret_cast<TH (*)[P_TU_ROWS + 1]>(smem);
  TH (*sc)[KP] = reinterpret_cast<TH (*)[KP]>(smem + sizeof(TH) * P_TU_CH * (P_TU_ROWS + 1));
  int* s_last = reinterpret_cast<int*>(smem + sizeof(TH) * P_TU_CH * (P_TU_ROWS + 1 + KP));
  const int n = A.n, k = A.k;
  const int tid = threadIdx.x;
  const int tiles = (n + P_TU_ROWS - 1) / P_TU_ROWS;
  if (a <= 0) {   // no history yet: the projection alone
    for (int tile = blockIdx.x; tile < tiles; tile += A.ncta) {
      const int r0 = tile * P_TU_ROWS, rows = min(P_TU_ROWS, n - r0);
      for (int idx = tid; idx < rows * k; idx += PT) {
        const int row = r0 + idx / k, g = idx % k;
        A.Zr[(size_t)row * k + g] -= gapply(A, row, g);
      }
    }
    return;
  }
  const TH* Wh = (const TH*)A.Wh;
  TH* part = (TH*)A.tu_part;
  const int splits = A.tu_splits;
  const int per = (a + splits - 1) / splits;
  const int items = tiles * splits;
  const int ty = tid / TXC, tx = tid % TXC;
  for (int it = blockIdx.x; it < items; it += A.ncta) {
    const int tile = it % tiles, sp = it / tiles;
    const int r0 = tile * P_TU_ROWS;
    const int c_begin = min(a, sp * per), c_end = min(a, c_begin + per);
    TH acc[RPT][CPT] = {};
    TH pa[LA], pc[LC];
    auto load = [&](int c0) {
      const int cc = tid % P_TU_CH;   // the same history column for all of the thread's loads
      const bool okc = c0 + cc < c_end;
      const TH* col = Wh + hist_col(okc ? c0 + cc : 0, n, k);
#pragma unroll
      for (int i = 0; i < LA; ++i) {
        const int rr = (tid + PT * i) / P_TU_CH;
        pa[i] = (r0 + rr < n && okc) ? col[(size_t)(r0 + rr) * k] : TH(0);
      }
#pragma unroll
      for (int i = 0; i < LC; ++i) {
        const int idx = tid + PT * i, cc = idx / KP, gg = idx % KP;
        pc[i] = (idx < P_TU_CH * KP && c0 + cc < c_end && gg < k) ? from_f64<TH>(A.C[(size_t)(c0 + cc) * k + gg]) : TH(0);
      }
    };
    if (c_begin < c_end) load(c_begin);
    for (int c0 = c_begin; c0 < c_end; c0 += P_TU_CH) {
      __syncthreads();   // the previous tile (or item) is consumed
#pragma unroll
      for (int i = 0; i < LA; ++i) {
        const int idx = tid + PT * i;
        sa[idx % P_TU_CH][idx / P_TU_CH] = pa[i];
      }
#pragma unroll
      for (int i = 0; i < LC; ++i) {
        const int idx = tid + PT * i;
        if (idx < P_TU_CH * KP) sc[idx / KP][idx % KP] = pc[i];
      }
      __syncthreads();
      if (c0 + P_TU_CH < c_end) load(c0 + P_TU_CH);
#pragma unroll 8
      for (int cc = 0; cc < P_TU_CH; ++cc) {
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
    }
    if (splits == 1) {
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const int row = r0 + ty + TY * u;
#pragma unroll
        for (int v = 0; v < CPT; ++v) {
          const int g = tx + TXC * v;
          if (row < n && g < k) {
            const size_t o = (size_t)row * k + g;
            A.Zr[o] = A.Zr[o] - gapply(A, row, g) - to_f64(acc[u][v]);
          }
        }
      }
      continue;
    }
    TH* P = part + (size_t)sp * n * k;
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
      const unsigned prev = atomicAdd(&A.tu_tickets[tile], 1u);
      *s_last = prev == (unsigned)splits - 1;
      if (*s_last) A.tu_tickets[tile] = 0u;
    }
    __syncthreads();
    if (!*s_last) continue;
    __threadfence();
    const int rows = min(P_TU_ROWS, n - r0);
    for (int idx = tid; idx < rows * k; idx += PT) {
      const size_t o = (size_t)r0 * k + idx;
      TH v0 = TH(0), v1 = TH(0), v2 = TH(0), v3 = TH(0);
      int q = 0;
      for (; q + 3 < splits; q += 4) {
        v0 += part[(size_t)q * n * k + o];
        v1 += part[(size_t)(q + 1) * n * k + o];
        v2 += part[(size_t)(q + 2) * n * k + o];
        v3 += part[(size_t)(q + 3) * n * k + o];
      }
      for (; q < splits; ++q) v0 += part[(size_t)q * n * k + o];
      const int row = r0 + idx / k, g = idx % k;
      A.Zr[o] = A.Zr[o] - gapply(A, row, g) - to_f64((v0 + v1) + (v2 + v3));
    }
  }
}

// Z_loc = S^+ Y for every pattern: 16 x 16 output tiles, K staged 64 at a time.  Y is not stored: the staged
// right-hand-side entries are the gather of Z (Eq. 9) computed on the fly, y(slot, g) = sum over the slot's
// links of sign * Z[row][g] (the same sum, in the same order, as a separate gather).
template <typename TL>
__device__ void phase_local(const PersistArgs& A, unsigned char* smem) {
  TL (*sa)[P_LT + 1] = reinterpret_cast<TL (*)[P_LT + 1]>(smem);
  TL (*sb)[P_LT + 1] = reinterpret_cast<TL (*)[P_LT + 1]>(smem + sizeof(TL) * P_LK * (P_LT + 1));
  int* cslot = reinterpret_cast<int*>(smem + 2 * sizeof(TL) * P_LK * (P_LT + 1));   // [16] first slot, -1 none
  int* ccol = cslot + P_LT;                                                         // [16] multivector column
  const Layout& L = A.L;
  const int n_pat = L.n_pat;
  const int k = A.k;
  const int items = A.tile_off[n_pat];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  TL* Zbuf = (TL*)A.Zbuf;
  for (int it = blockIdx.x; it < items; it += A.ncta) {
    int p = 0;
    while (p + 1 < n_pat && it >= A.tile_off[p + 1]) ++p;
    const int t = it - A.tile_off[p];
    const int m0 = (t % A.tiles_m[p]) * P_LT, n0 = (t / A.tiles_m[p]) * P_LT;
    const int nb = L.n_b[p], nr = A.n_rhs[p];
    const long long ld = A.ld[p];
    const TL* S = (const TL*)A.S[p];
    TL* Z = Zbuf + A.ybase[p];
    __syncthreads();   // the previous item's shared-memory reads are done
    if (tid < P_LT) {
      const int c = n0 + tid;
      cslot[tid] = c < nr ? L.occ_obase[A.pocc[p][c / k]] : -1;
      ccol[tid] = c % k;
    }
    TL acc = TL(0);
    for (int k0 = 0; k0 < nb; k0 += P_LK) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < P_LK * P_LT / PT; ++u) {
        const int idx = tid + PT * u;
        const int kk = idx % P_LK, r = idx / P_LK;
        const int i = m0 + r, j = k0 + kk;
        sa[kk][r] = (i < nb && j < nb) ? S[(size_t)i * nb + j] : TL(0);
        TL yv = TL(0);
        if (cslot[r] >= 0 && j < nb) {
          const int slot = cslot[r] + j, g = ccol[r];
          double y = 0.0;
          for (int e = 0; e < L.ell_w; ++e) {
            const int sg = L.ell_sign[(size_t)slot * L.ell_w + e];
            if (sg == 0) continue;
            y += neg_if(A.Zr[(size_t)L.ell_row[(size_t)slot * L.ell_w + e] * k + g], sg < 0);
          }
          yv = from_f64<TL>(y);
        }
        sb[kk][r] = yv;
      }
      __syncthreads();
#pragma unroll 16
      for (int kk = 0; kk < P_LK; ++kk) acc = fma(sa[kk][tx], sb[kk][ty], acc);
    }
    const int i = m0 + tx, c = n0 + ty;
    if (i < nb && c < nr) Z[(long long)c * ld + i] = acc;
  }
}

// Q = scatter(Z_loc) - G A on the CTA's contiguous rows, with the eta partials [Z^T Q | Z^T r] of those rows;
// the last CTA to finish adds the partials in CTA order and normalises (T, alpha, n_kept).
template <typename TL>
__device__ void phase_q_eta(const PersistArgs& A, unsigned char* smem) {
  const int n = A.n, k = A.k;
  const int nout = k * (k + 1);
  double (*sw)[32] = reinterpret_cast<double (*)[32]>(smem);                     // [16][32]
  double (*sq)[33] = reinterpret_cast<double (*)[33]>(smem + 16 * 32 * 8);       // [16][33]
  int* s_last = reinterpret_cast<int*>(smem + 16 * 32 * 8 + 16 * 33 * 8);
  const int tid = threadIdx.x;
  const int R = (n + A.ncta - 1) / A.ncta;
  const int r0 = min(n, blockIdx.x * R), r1 = min(n, r0 + R);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // outputs tid + 256 q (nout <= 32 * 33 <= 5 * 256)
  for (int rr = r0; rr < r1; rr += 16) {
    const int nrow = min(16, r1 - rr);
    __syncthreads();
    for (int idx = tid; idx < nrow * k; idx += PT) {   // one (row, column) per thread (16 k <= 512)
      const int q = idx / k, c = idx % k;
      const int row = rr + q;
      const double v = qraw<TL>(A, row, c) - gapply(A, row, c);
      A.Q[(size_t)row * k + c] = v;
      sw[q][c] = A.Zr[(size_t)row * k + c];
      sq[q][c] = v;
    }
    if (tid < 16) sq[tid][32] = tid < nrow ? A.r[rr + tid] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int o = q * PT + tid;
      if (o < nout) {
        const int i = o / (k + 1), j = o % (k + 1);
        const int jj = (j == k) ? 32 : j;
        double v0 = acc[q], v1 = 0.0;
        int t = 0;
        for (; t + 1 < nrow; t += 2) {
          v0 = fma(sw[t][i], sq[t][jj], v0);
          v1 = fma(sw[t + 1][i], sq[t + 1][jj], v1);
        }
        if (t < nrow) v0 = fma(sw[t][i], sq[t][jj], v0);
        acc[q] = v0 + v1;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int o = q * PT + tid;
    if (o < nout) A.eta_part[(size_t)blockIdx.x * nout + o] = acc[q];
  }
  // two-level reduction of the CTA partials, in a fixed order whichever CTAs perform it: the last CTA of every
  // group of 16 adds its group's partials, the last group reducer adds the group sums and normalises
  __threadfence();
  __syncthreads();
  constexpr int GSZ = 16;
  const int grp = blockIdx.x / GSZ, ng = (A.ncta + GSZ - 1) / GSZ;
  const int gsize = min(GSZ, A.ncta - grp * GSZ);
  if (tid == 0) {
    const unsigned prev = atomicAdd(&A.eta_gticket[grp], 1u);
    *s_last = prev == (unsigned)gsize - 1;
    if (*s_last) A.eta_gticket[grp] = 0u;
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  double* gpart = A.eta_part + (size_t)A.ncta * nout;
  for (int o = tid; o < nout; o += PT) {
    double u[GSZ];
#pragma unroll
    for (int q = 0; q < GSZ; ++q) u[q] = q < gsize ? A.eta_part[(size_t)(grp * GSZ + q) * nout + o] : 0.0;
#pragma unroll
    for (int w = GSZ / 2; w > 0; w >>= 1)
#pragma unroll
      for (int q = 0; q < w; ++q) u[q] += u[q + w];
    gpart[(size_t)grp * nout + o] = u[0];
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned prev = atomicAdd(A.eta_ticket, 1u);
    *s_last = prev == (unsigned)ng - 1;
    if (*s_last) *A.eta_ticket = 0u;
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  const bool stamp = A.clk && tid == 0;
  const unsigned long long t0 = stamp ? gtimer() : 0ull;
  // the last group reducer: eta and W^T r from the group sums, then the one-warp normalisation
  double (*Am)[33] = reinterpret_cast<double (*)[33]>(smem);                       // [32][33]
  double (*Lc)[33] = reinterpret_cast<double (*)[33]>(smem + 32 * 33 * 8);         // [32][33]
  int* piv = reinterpret_cast<int*>(smem + 2 * 32 * 33 * 8);
  double* Dg = reinterpret_cast<double*>(smem + 2 * 32 * 33 * 8 + 32 * 4);
  double* rhs = Dg + 32;
  double* ext = &Lc[0][0];
  for (int o = tid; o < nout; o += PT) {
    double v = 0.0;
    for (int g = 0; g < ng; g += GSZ) {
      double u[GSZ];
#pragma unroll
      for (int q = 0; q < GSZ; ++q) u[q] = g + q < ng ? gpart[(size_t)(g + q) * nout + o] : 0.0;
#pragma unroll
      for (int w = GSZ / 2; w > 0; w >>= 1)
#pragma unroll
        for (int q = 0; q < w; ++q) u[q] += u[q + w];
      v += u[0];
    }
    ext[o] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += PT) {
    const int i = idx / k, j = idx % k;
    Am[i][j] = 0.5 * (ext[i * (k + 1) + j] + ext[j * (k + 1) + i]);
  }
  if (tid < k) rhs[tid] = ext[tid * (k + 1) + k];
  __syncthreads();
  for (int idx = tid; idx < 32 * 33; idx += PT) (&Lc[0][0])[idx] = 0.0;
  __syncthreads();
  const unsigned long long t1 = stamp ? gtimer() : 0ull;
  if (tid < 32) normalise_warp<33>(k, Am, Lc, piv, Dg, rhs, A.trunc, A.T, A.alpha, A.n_kept);
  if (stamp) {   // timing: the last CTA's reduction and normalisation
    A.clk[9] += t1 - t0;
    A.clk[10] += gtimer() - t1;
  }
}

// history columns [a, a + k) = Z T and Q T, lambda += Z T alpha, r -= Q T alpha, per-CTA ||r||^2 partial;
// CTA 0 then advances the history count (restart rule), the dropped count and the iteration count.
template <typename TH>
__device__ void phase_update(const PersistArgs& A, int a, unsigned char* smem) {
  TH (*sT)[33] = reinterpret_cast<TH (*)[33]>(smem);
  double* beta = reinterpret_cast<double*>(smem + sizeof(TH) * 32 * 33 + 8);
  double* warp_rr = beta + 32;
  const int n = A.n, k = A.k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  TH* Wn = (TH*)A.Wh + hist_col(a, A.n, A.k);   // the new block (a is a multiple of k)
  TH* Qn = (TH*)A.Qh + hist_col(a, A.n, A.k);
  for (int idx = tid; idx < k * k; idx += PT) sT[idx / k][idx % k] = from_f64<TH>(A.T[idx]);
  if (tid < k) {
    double v = 0.0;
    for (int c = 0; c < k; ++c) v = fma(A.T[(size_t)tid * k + c], A.alpha[c], v);
    beta[tid] = v;
  }
  __syncthreads();
  int kp = 1;
  while (kp < k) kp <<= 1;
  const int rows_w = kp >= 32 ? 1 : 32 / kp;
  const int seg = kp >= 32 ? 32 : kp;
  const int sub = lane / seg, c0 = lane % seg;
  double rr = 0.0;
  const long long stride = (long long)A.ncta * (PT / 32) * rows_w;
  for (long long base = ((long long)blockIdx.x * (PT / 32) + warp) * rows_w; base < n; base += stride) {
    const long long row = base + sub;
    const bool ok = row < n && c0 < k;
    const double w0 = ok ? A.Zr[row * k + c0] : 0.0, q0 = ok ? A.Q[row * k + c0] : 0.0;
    const TH w0h = from_f64<TH>(w0), q0h = from_f64<TH>(q0);
    TH wn = TH(0), qn = TH(0);
    const int ca = c0 < k ? c0 : 0;
    for (int j = 0; j < k; ++j) {
      const TH wj = __shfl_sync(FULL, w0h, j, seg);
      const TH qj = __shfl_sync(FULL, q0h, j, seg);
      wn = fma(wj, sT[j][ca], wn);
      qn = fma(qj, sT[j][ca], qn);
    }
    if (ok) {
      Wn[row * k + c0] = wn;
      Qn[row * k + c0] = qn;
    }
    double dl = ok ? w0 * beta[c0] : 0.0, dr = ok ? q0 * beta[c0] : 0.0;
    for (int o = seg >> 1; o > 0; o >>= 1) {
      dl += __shfl_xor_sync(FULL, dl, o);
      dr += __shfl_xor_sync(FULL, dr, o);
    }
    if (row < n && c0 == 0) {
      A.lam[row] += dl;
      const double rn = A.r[row] - dr;
      A.r[row] = rn;
      rr = fma(rn, rn, rr);
    }
  }
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(FULL, rr, o);
  if (lane == 0) warp_rr[warp] = rr;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < PT / 32; ++w) s += warp_rr[w];
    A.rr_part[blockIdx.x] = s;
    if (blockIdx.x == 0) {
      int c = a + k;
      if ((long long)c + k > A.cap) c = 0;
      A.state[0] = c;
      A.state[1] += k - *A.n_kept;
      A.state[2] += 1;
    }
  }
}

template <typename TH, typename TL, int KP>
__global__ void __launch_bounds__(PT) k_persist(PersistArgs A) {
  __shared__ __align__(16) unsigned char smem[P_SMEM];
  __shared__ int s_go;
  const bool stamp = A.clk && blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long t_prev = stamp ? gtimer() : 0ull;
  auto phase_end = [&](int ph) {   // grid barrier, then (timing) CTA 0 books the phase's time
    if (!grid_sync(A)) return false;
    if (stamp) {
      const unsigned long long t = gtimer();
      A.clk[ph] += t - t_prev;
      t_prev = t;
    }
    return true;
  };
  for (int it = 0; it < A.max_iters; ++it) {
    if (it > 0) {   // device residual test: every CTA adds the partials in the same order
      if (threadIdx.x < 32) {
        double v = 0.0;
        for (int c = threadIdx.x; c < A.ncta; c += 32) v += A.rr_part[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (threadIdx.x == 0) s_go = (v > A.target2 && *A.n_kept > 0) ? 1 : 0;
      }
      __syncthreads();
      if (!s_go) return;
    }
    const int a = A.state[0];
    phase_one<TH, TL>(A, a, smem);   // P1
    if (!phase_end(0)) return;
    // P2
    if (a > 0) {
      const int count = a * A.k;
      for (int i = blockIdx.x * PT + threadIdx.x; i < count; i += A.ncta * PT) {
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        int c = 0;
        for (; c + 3 < A.gs_chunks; c += 4) {
          v0 += A.gram_part[(size_t)c * count + i];
          v1 += A.gram_part[(size_t)(c + 1) * count + i];
          v2 += A.gram_part[(size_t)(c + 2) * count + i];
          v3 += A.gram_part[(size_t)(c + 3) * count + i];
        }
        for (; c < A.gs_chunks; ++c) v0 += A.gram_part[(size_t)c * count + i];
        A.C[i] = (v0 + v1) + (v2 + v3);
      }
    }
    if (A.L.n_G > 0) phase_small_gemm(A);
    if (!phase_end(1)) return;
    phase_tall<TH, KP>(A, a, smem);   // P3
    if (!phase_end(2)) return;
    phase_local<TL>(A, smem);         // P4 + P5: gather fused into the local products
    if (!phase_end(4)) return;
    if (A.L.n_G > 0) phase_gtv<TL, false>(A, smem);   // P6
    if (!phase_end(5)) return;
    if (A.L.n_G > 0) phase_small_gemm(A);             // P7
    if (!phase_end(6)) return;
    phase_q_eta<TL>(A, smem);         // P8
    if (!phase_end(7)) return;
    phase_update<TH>(A, a, smem);     // P9
    if (!phase_end(8)) return;
  }
}

// Persistent launches on one device are chained (each waits for the previous one's completion event), so that
// two of them, from different contexts or server workers, are never resident together: each needs all of its
// CTAs co-resident for its grid barriers.
std::mutex g_chain_mutex;
cudaEvent_t g_chain_event[64] = {};

template <typename TH, typename TL>
void launch(const PersistArgs& A, cudaStream_t s) {
  void* args[] = {const_cast<PersistArgs*>(&A)};
  const void* fn;
  if (A.k <= 8) fn = (const void*)k_persist<TH, TL, 8>;
  else if (A.k <= 16) fn = (const void*)k_persist<TH, TL, 16>;
  else fn = (const void*)k_persist<TH, TL, 32>;
  int dev = 0;
  FETIRP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(1, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_chain_mutex);
  if (!g_chain_event[dev]) FETIRP_CUDA(cudaEventCreateWithFlags(&g_chain_event[dev], cudaEventDisableTiming));
  else FETIRP_CUDA(cudaStreamWaitEvent(s, g_chain_event[dev], 0));
  FETIRP_CUDA(cudaLaunchCooperativeKernel(fn, dim3(A.ncta), dim3(PT), args, 0, s));
  ++g_launch_count;
  FETIRP_CUDA(cudaEventRecord(g_chain_event[dev], s));
}

template <typename TH, typename TL>
int ctas(int k) {
  const void* fn;
  if (k <= 8) fn = (const void*)k_persist<TH, TL, 8>;
  else if (k <= 16) fn = (const void*)k_persist<TH, TL, 16>;
  else fn = (const void*)k_persist<TH, TL, 32>;
  int dev = 0, sms = 0, per = 0;
  FETIRP_CUDA(cudaGetDevice(&dev));
  FETIRP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FETIRP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, PT, 0));
  return sms * std::min(per, 2);
}

}  // namespace

void persist_iterations(const PersistArgs& A, bool fp64, cudaStream_t s) {
  if (A.k < 1 || A.k > 32) throw Error(1, "persistent iteration needs 1 <= k <= 32");
  if (fp64) launch<double, double>(A, s);
  else launch<float, float>(A, s);
}

int persist_ctas(bool fp64, int k) { return fp64 ? ctas<double, double>(k) : ctas<float, float>(k); }

}  // namespace fetirp
