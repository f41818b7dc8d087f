// Interface operators of one structure: the signed Boolean gather/scatter (Eq. 2, blocked storage of
// Eq. 9), the coarse space G = [B(s) N(s)] of Eq. 3 and the multivector split.
#include "ops.cuh"

namespace fetirp {

// y(slot, g) = sum over the slot's links: sign * V[row][g]   (ELL links, independent loads)
__device__ __forceinline__ double trace_of(const Layout& L, const double* __restrict__ V, int k, int slot, int g) {
  const int* er = L.ell_row + (size_t)slot * L.ell_w;
  const int8_t* es = L.ell_sign + (size_t)slot * L.ell_w;
  double y = 0.0;
#pragma unroll 4
  for (int e = 0; e < L.ell_w; ++e) y = fma((double)es[e], V[(size_t)er[e] * k + g], y);
  return y;
}

// X[gofs(s)+m][g] = sum_{links of s} sign * Nb[j][m] * V[row][g]        (one CTA per occurrence)
// Thread t takes column g = t % k and every (256/k)-th boundary dof; partial sums per kernel mode m live in
// registers and are reduced over the threads of one column in a fixed order (deterministic).
constexpr int GTV_THREADS = 256;
constexpr int GTV_COLS = 8;     // columns per CTA (grid.y splits the block of k columns)
constexpr int MAX_KDIM = 6;
__global__ void __launch_bounds__(GTV_THREADS) k_gt_v(Layout L, const double* __restrict__ V, int k,
                                                       double* __restrict__ X) {
  __shared__ double red[GTV_THREADS][MAX_KDIM];
  const int s = blockIdx.x;
  const int p = L.occ_pat[s];
  const int kd = L.kdim[p];
  const double* Nb = L.Nb[p];
  const int b0 = L.occ_obase[s], nb = L.occ_obase[s + 1] - b0;
  const int g0 = L.occ_gofs[s];
  const int t = threadIdx.x;
  const int gbase = blockIdx.y * GTV_COLS;
  const int kk = min(GTV_COLS, k - gbase);
  const int lanes = GTV_THREADS / kk;       // threads per column
  const int g = gbase + t % kk, sub = t / kk;
  double acc[MAX_KDIM] = {};
  if (sub < lanes) {
#pragma unroll 2
    for (int j = sub; j < nb; j += lanes) {
      const double y = trace_of(L, V, k, b0 + j, g);
#pragma unroll
      for (int m = 0; m < MAX_KDIM; ++m)
        if (m < kd) acc[m] = fma(Nb[(size_t)j * kd + m], y, acc[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < MAX_KDIM; ++m) red[t][m] = acc[m];
  __syncthreads();
  if (t < kk) {
    for (int m = 0; m < kd; ++m) {
      double v = 0.0;
      for (int q = 0; q < lanes; ++q) v += red[q * kk + t][m];
      X[(size_t)(g0 + m) * k + gbase + t] = v;
    }
  }
}

// out[row][g] = beta*out + alpha * sum_{slots of row} sign * sum_m Nb[j][m] A[gofs+m][g]
__global__ void k_g_apply(Layout L, const double* __restrict__ A, int k, double alpha, double beta,
                          double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_lambda * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int sg = L.row_sign[2 * row + e];
    if (sg == 0) continue;
    const int slot = L.row_slot[2 * row + e];
    const int s = L.slot_occ[slot];
    const int p = L.occ_pat[s];
    const int kd = L.kdim[p];
    const int j = slot - L.occ_obase[s];
    const double* Nb = L.Nb[p] + (size_t)j * kd;
    const double* a = A + (size_t)L.occ_gofs[s] * k + g;
    double t = 0.0;
    for (int m = 0; m < kd; ++m) t = fma(Nb[m], a[(size_t)m * k], t);
    acc = sg > 0 ? acc + t : acc - t;
  }
  double* o = out + idx;
  *o = (beta == 0.0 ? 0.0 : beta * *o) + alpha * acc;
}

// Block (s, t) of G^T G for one neighbour pair: sum over rows linking s and t.  Threads split the boundary
// dofs of s; per-thread partials are reduced in a fixed order.
__global__ void __launch_bounds__(128) k_gtg(Layout L, const int* __restrict__ pair_s, const int* __restrict__ pair_t,
                                             double* __restrict__ GtG) {
  __shared__ double red[128][MAX_KDIM * MAX_KDIM];
  const int s = pair_s[blockIdx.x], t = pair_t[blockIdx.x];
  const int ps = L.occ_pat[s], pt = L.occ_pat[t];
  const int ks = L.kdim[ps], kt = L.kdim[pt];
  const int b0 = L.occ_obase[s], b1 = L.occ_obase[s + 1];
  double acc[MAX_KDIM * MAX_KDIM] = {};
  for (int slot = b0 + threadIdx.x; slot < b1; slot += blockDim.x) {
    const double* ns = L.Nb[ps] + (size_t)(slot - b0) * ks;
    for (int e = L.slot_ptr[slot]; e < L.slot_ptr[slot + 1]; ++e) {
      const int row = L.slot_row[e];
      const int sg = L.slot_sign[e];
      for (int f = 0; f < 2; ++f) {
        const int sg2 = L.row_sign[2 * row + f];
        if (sg2 == 0) continue;
        const int slot2 = L.row_slot[2 * row + f];
        if (L.slot_occ[slot2] != t) continue;
        const double* nt = L.Nb[pt] + (size_t)(slot2 - L.occ_obase[t]) * kt;
        const double w = (double)(sg * sg2);
        for (int m = 0; m < ks; ++m)
          for (int m2 = 0; m2 < kt; ++m2) acc[m * MAX_KDIM + m2] = fma(w * ns[m], nt[m2], acc[m * MAX_KDIM + m2]);
      }
    }
  }
  for (int q = 0; q < MAX_KDIM * MAX_KDIM; ++q) red[threadIdx.x][q] = acc[q];
  __syncthreads();
  for (int idx = threadIdx.x; idx < ks * kt; idx += blockDim.x) {
    const int m = idx / kt, m2 = idx % kt;
    double v = 0.0;
    for (int q = 0; q < (int)blockDim.x; ++q) v += red[q][m * MAX_KDIM + m2];
    GtG[(size_t)(L.occ_gofs[s] + m) * L.n_G + L.occ_gofs[t] + m2] = v;
  }
}

template <typename TO>
__global__ void k_gather(Layout L, const double* __restrict__ V, int k, PatView<TO> Y, double alpha, double beta) {
  const int s = blockIdx.x;
  const int p = L.occ_pat[s];
  const int q = L.occ_q[s];
  const int b0 = L.occ_obase[s], nb = L.occ_obase[s + 1] - b0;
  TO* base = Y.base[p];
  const long long ld = Y.ld[p], off = Y.off[p];
  const int gbase = blockIdx.y * GTV_COLS, kk = min(GTV_COLS, k - gbase);
  for (int idx = threadIdx.x; idx < nb * kk; idx += blockDim.x) {
    const int g = gbase + idx / nb, j = idx % nb;
    const double acc = trace_of(L, V, k, b0 + j, g);
    TO* y = base + ((long long)q * k + g) * ld + off + j;
    *y = (TO)((beta == 0.0 ? 0.0 : beta * (double)*y) + alpha * acc);
  }
}

// Gather with the result split into a tf32 pair: hi = tf32(y) (round to nearest), lo = y - hi (FP32).
__global__ void k_gather_split(Layout L, const double* __restrict__ V, int k, PatView<float> Yh, PatView<float> Yl) {
  const int s = blockIdx.x;
  const int p = L.occ_pat[s];
  const int q = L.occ_q[s];
  const int b0 = L.occ_obase[s], nb = L.occ_obase[s + 1] - b0;
  const int gbase = blockIdx.y * GTV_COLS, kk = min(GTV_COLS, k - gbase);
  for (int idx = threadIdx.x; idx < nb * kk; idx += blockDim.x) {
    const int g = gbase + idx / nb, j = idx % nb;
    const float v = (float)trace_of(L, V, k, b0 + j, g);
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
    const float h = __uint_as_float(t);
    const long long o = ((long long)q * k + g) * Yh.ld[p] + Yh.off[p] + j;
    Yh.base[p][o] = h;
    Yl.base[p][o] = v - h;
  }
}

template <typename TI>
__global__ void k_scatter(Layout L, PatView<TI> Z, int k, double beta, double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_lambda * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int sg = L.row_sign[2 * row + e];
    if (sg == 0) continue;
    const int slot = L.row_slot[2 * row + e];
    const int s = L.slot_occ[slot];
    const int p = L.occ_pat[s];
    const int q = L.occ_q[s];
    const int j = slot - L.occ_obase[s];
    acc += (double)sg * (double)Z.base[p][((long long)q * k + g) * Z.ld[p] + Z.off[p] + j];
  }
  double* o = out + idx;
  *o = (beta == 0.0 ? 0.0 : beta * *o) + acc;
}

__global__ void k_split(Layout L, const double* __restrict__ r, int k, double* __restrict__ Z) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= L.n_lambda) return;
  double* z = Z + (size_t)row * k;
  for (int g = 0; g < k; ++g) z[g] = 0.0;
  int cnt = (L.row_sign[2 * row] != 0) + (L.row_sign[2 * row + 1] != 0);
  if (cnt == 0) return;
  const double w = r[row] / cnt;
  for (int e = 0; e < 2; ++e) {
    if (L.row_sign[2 * row + e] == 0) continue;
    const int s = L.slot_occ[L.row_slot[2 * row + e]];
    z[L.occ_group[s]] += w;
  }
}

// ---- sparse-column form of P^T F P S(r) -------------------------------------------------------------
// Y for the (occurrence, group) pairs only: pair i (pattern p, pattern-local index i - pair_off[p]) gathers
// column pair_g[i] of V on the slots of occurrence pair_occ[i] (the same sum as the dense gather).
template <typename TO>
__global__ void __launch_bounds__(256) k_gather_pairs(Layout L, const double* __restrict__ V, int k,
                                                      const int* __restrict__ pair_occ,
                                                      const int* __restrict__ pair_g, PairView<TO> Y) {
  const int i = blockIdx.x;
  const int s = pair_occ[i], g = pair_g[i];
  const int p = L.occ_pat[s];
  const int b0 = L.occ_obase[s], nb = L.occ_obase[s + 1] - b0;
  TO* y = Y.base[p] + (long long)(i - Y.pair_off[p]) * Y.ld[p];
  for (int j = threadIdx.x; j < nb; j += blockDim.x) y[j] = (TO)trace_of(L, V, k, b0 + j, g);
}

// as k_gather_pairs, the FP32 value split into a tf32 pair (hi = tf32(y), lo = y - hi)
__global__ void __launch_bounds__(256) k_gather_pairs_split(Layout L, const double* __restrict__ V, int k,
                                                            const int* __restrict__ pair_occ,
                                                            const int* __restrict__ pair_g, PairView<float> Yh,
                                                            PairView<float> Yl) {
  const int i = blockIdx.x;
  const int s = pair_occ[i], g = pair_g[i];
  const int p = L.occ_pat[s];
  const int b0 = L.occ_obase[s], nb = L.occ_obase[s + 1] - b0;
  const long long o = (long long)(i - Yh.pair_off[p]) * Yh.ld[p];
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const float v = (float)trace_of(L, V, k, b0 + j, g);
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
    const float h = __uint_as_float(t);
    Yh.base[p][o + j] = h;
    Yl.base[p][o + j] = v - h;
  }
}

// Yc[slot][g] = sum_c M_s[j][c] A[mrow[c]][g]: the local response of occurrence s to the coarse correction
// G X restricted to its own and its neighbours' kernel modes (M_s = S^+ B(s)^T G_nbr(s), precomputed).
// Grid (occurrence, 64-slot chunk); thread = (slot j, quarter of the k columns): each M entry is loaded once
// (coalesced over j) and used for the thread's columns; A's rows of the occurrence are staged in shared memory.
template <typename TM>
__global__ void __launch_bounds__(256) k_coarse_response(Layout L, int k, const TM* __restrict__ M,
                                                         const long long* __restrict__ moff,
                                                         const int* __restrict__ mcol_ptr,
                                                         const int* __restrict__ mcol_row, const long long* mld,
                                                         const double* __restrict__ A, double* __restrict__ Yc) {
  __shared__ TM sa[48][64];   // A rows of the occurrence's columns (<= 7 x 6 modes, k <= 64), in TM
  const int s = blockIdx.x;
  const int p = L.occ_pat[s];
  const int b0 = L.occ_obase[s], nb = L.occ_obase[s + 1] - b0;
  const int c0 = mcol_ptr[s], nc = mcol_ptr[s + 1] - c0;
  for (int idx = threadIdx.x; idx < nc * k; idx += blockDim.x) {
    const int c = idx / k, g = idx % k;
    sa[c][g] = (TM)A[(size_t)mcol_row[c0 + c] * k + g];
  }
  __syncthreads();
  const int j = blockIdx.y * 64 + threadIdx.x % 64;
  if (j >= nb) return;
  const int gq = threadIdx.x / 64;                 // columns g = gq, gq + 4, ...
  const TM* m = M + moff[s] + j;
  const long long ld = mld[p];
  TM acc[16];   // k <= 64: at most 16 columns per thread; TM arithmetic (FP64 form: FP64, else FP32)
#pragma unroll
  for (int u = 0; u < 16; ++u) acc[u] = TM(0);
  for (int c = 0; c < nc; ++c) {
    const TM mv = m[(long long)c * ld];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int g = gq + 4 * u;
      if (g < k) acc[u] = fma(mv, sa[c][g], acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int g = gq + 4 * u;
    if (g < k) Yc[(size_t)(b0 + j) * k + g] = (double)acc[u];
  }
}

// out[row][g] = sum over the row's slots: sign * (Z_loc(pair(s, g), j) - Yc[slot][g]); pairs that do not exist
// (the split column does not touch the occurrence) contribute no local solution.
template <typename TI>
__global__ void k_scatter_pairs(Layout L, PairView<TI> Z, int k, const int* __restrict__ pair_of,
                                const double* __restrict__ Yc, double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_lambda * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int sg = L.row_sign[2 * row + e];
    if (sg == 0) continue;
    const int slot = L.row_slot[2 * row + e];
    const int s = L.slot_occ[slot];
    const int p = L.occ_pat[s];
    const int j = slot - L.occ_obase[s];
    const int lp = pair_of[(size_t)s * k + g];
    const double z = lp >= 0 ? (double)Z.base[p][(long long)lp * Z.ld[p] + j] : 0.0;
    acc += (double)sg * (z - Yc[(size_t)slot * k + g]);
  }
  out[idx] = acc;
}

// ------------------------------------------------------------------------------------------------ host
void gt_v(const Layout& L, const double* V, int k, double* X, cudaStream_t s) {
  if (L.n_occ == 0) return;
  if (k > 64) throw Error(1, "k > 64");
  k_gt_v<<<dim3(L.n_occ, ceil_div(k, GTV_COLS)), GTV_THREADS, 0, s>>>(L, V, k, X);
  FETIRP_LAUNCH_CHECK();
}


void g_apply(const Layout& L, const double* A, int k, double alpha, double beta, double* out, cudaStream_t s) {
  long long n = (long long)L.n_lambda * k;
  if (n == 0) return;
  k_g_apply<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, A, k, alpha, beta, out);
  FETIRP_LAUNCH_CHECK();
}


void gtg_dense(const Layout& L, const int*, const int*, int n_pairs, const int* pair_s, const int* pair_t,
               double* GtG, cudaStream_t s) {
  FETIRP_CUDA(cudaMemsetAsync(GtG, 0, sizeof(double) * (size_t)L.n_G * L.n_G, s));
  if (n_pairs == 0) return;
  k_gtg<<<n_pairs, 128, 0, s>>>(L, pair_s, pair_t, GtG);
  FETIRP_LAUNCH_CHECK();
}

template <typename TO>
void gather(const Layout& L, const double* V, int k, const PatView<TO>& Y, cudaStream_t s, double alpha,
            double beta) {
  if (L.n_occ == 0) return;
  k_gather<TO><<<dim3(L.n_occ, ceil_div(k, GTV_COLS)), 256, 0, s>>>(L, V, k, Y, alpha, beta);
  FETIRP_LAUNCH_CHECK();
}

template <typename TI>
void scatter(const Layout& L, const PatView<TI>& Z, int k, double beta, double* out, cudaStream_t s) {
  long long n = (long long)L.n_lambda * k;
  if (n == 0) return;
  k_scatter<TI><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, Z, k, beta, out);
  FETIRP_LAUNCH_CHECK();
}

void gather_split(const Layout& L, const double* V, int k, const PatView<float>& Yh, const PatView<float>& Yl,
                  cudaStream_t s) {
  if (L.n_occ == 0) return;
  k_gather_split<<<dim3(L.n_occ, ceil_div(k, GTV_COLS)), 256, 0, s>>>(L, V, k, Yh, Yl);
  FETIRP_LAUNCH_CHECK();
}

void split(const Layout& L, const double* r, int k, double* Z, cudaStream_t s) {
  if (L.n_lambda == 0) return;
  k_split<<<ceil_div(L.n_lambda, 256), 256, 0, s>>>(L, r, k, Z);
  FETIRP_LAUNCH_CHECK();
}

template void gather<double>(const Layout&, const double*, int, const PatView<double>&, cudaStream_t, double,
                             double);
template void gather<float>(const Layout&, const double*, int, const PatView<float>&, cudaStream_t, double, double);
template void scatter<double>(const Layout&, const PatView<double>&, int, double, double*, cudaStream_t);
template void scatter<float>(const Layout&, const PatView<float>&, int, double, double*, cudaStream_t);

void gather_pairs_f64(const Layout& L, const double* V, int k, const int* pair_occ, const int* pair_g, int n_pairs,
                      const PairView<double>& Y, cudaStream_t s) {
  if (n_pairs == 0) return;
  k_gather_pairs<double><<<n_pairs, 256, 0, s>>>(L, V, k, pair_occ, pair_g, Y);
  FETIRP_LAUNCH_CHECK();
}
void gather_pairs_f32(const Layout& L, const double* V, int k, const int* pair_occ, const int* pair_g, int n_pairs,
                      const PairView<float>& Y, cudaStream_t s) {
  if (n_pairs == 0) return;
  k_gather_pairs<float><<<n_pairs, 256, 0, s>>>(L, V, k, pair_occ, pair_g, Y);
  FETIRP_LAUNCH_CHECK();
}
void gather_pairs_split(const Layout& L, const double* V, int k, const int* pair_occ, const int* pair_g, int n_pairs,
                        const PairView<float>& Yh, const PairView<float>& Yl, cudaStream_t s) {
  if (n_pairs == 0) return;
  k_gather_pairs_split<<<n_pairs, 256, 0, s>>>(L, V, k, pair_occ, pair_g, Yh, Yl);
  FETIRP_LAUNCH_CHECK();
}
template <typename TM>
void coarse_response(const Layout& L, int k, const TM* M, const long long* moff, const int* mcol_ptr,
                     const int* mcol_row, const long long* mld, const double* A, double* Yc, cudaStream_t s) {
  if (L.n_occ == 0) return;
  if (k > 64) throw Error(1, "k > 64");
  int max_nb = 1;
  for (int p = 0; p < L.n_pat; ++p) max_nb = std::max(max_nb, L.n_b[p]);
  k_coarse_response<TM><<<dim3(L.n_occ, ceil_div(max_nb, 64)), 256, 0, s>>>(L, k, M, moff, mcol_ptr, mcol_row, mld,
                                                                            A, Yc);
  FETIRP_LAUNCH_CHECK();
}
template void coarse_response<double>(const Layout&, int, const double*, const long long*, const int*, const int*,
                                       const long long*, const double*, double*, cudaStream_t);
template void coarse_response<float>(const Layout&, int, const float*, const long long*, const int*, const int*,
                                      const long long*, const double*, double*, cudaStream_t);
template <typename TI>
void scatter_pairs(const Layout& L, const PairView<TI>& Z, int k, const int* pair_of, const double* Yc, double* out,
                   cudaStream_t s) {
  long long n = (long long)L.n_lambda * k;
  if (n == 0) return;
  k_scatter_pairs<TI><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, Z, k, pair_of, Yc, out);
  FETIRP_LAUNCH_CHECK();
}
template void scatter_pairs<double>(const Layout&, const PairView<double>&, int, const int*, const double*, double*,
                                    cudaStream_t);
template void scatter_pairs<float>(const Layout&, const PairView<float>&, int, const int*, const double*, double*,
                                   cudaStream_t);

}  // namespace fetirp
