// Interface operators of one structure: the signed Boolean gather/scatter (Eq. 2, blocked storage of
// Eq. 9), the coarse space G = [B(s) N(s)] of Eq. 3 and the multivector split.
#include <type_traits>

#include "ds.cuh"
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

// X[gofs(s)+m][g] = sum_{links (row, e) of s} (sign Nb[j])[m] * V[row][g], the signed coefficients taken from the
// per-row tables.  Grid (occurrence, chunk of its links); warp w takes every 8th link of the chunk, four links
// at a time (independent loads: link code, then its row of V and its coefficients), lane = column g (and g + 32
// for k <= 64), so every link reads one contiguous row of V.  The warps' sums are added in warp order; with
// several chunks per occurrence the last CTA of the occurrence (ticket) adds the chunks' partial sums in chunk
// order and re-arms the ticket (deterministic, no atomics on values).
constexpr int GTV_THREADS = 256;
constexpr int MAX_KDIM = 6;
template <bool WIDE>   // WIDE: 32 < k <= 64 (two columns per lane)
__global__ void __launch_bounds__(GTV_THREADS, WIDE ? 2 : 3) k_gt_v(Layout L, const double* __restrict__ V, int k,
                                                          double* __restrict__ X, int chunk) {
  __shared__ double red[GTV_THREADS / 32][MAX_KDIM][64];
  __shared__ int s_last;
  const int s = blockIdx.x, c = blockIdx.y, nch = gridDim.y;
  const int kd = L.kdim[L.occ_pat[s]];
  const int l0 = L.slot_ptr[L.occ_obase[s]], nl = L.slot_ptr[L.occ_obase[s + 1]] - l0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool c0 = lane < k, c1 = WIDE && lane + 32 < k;
  const int i_end = min(nl, (c + 1) * chunk);
  double a0[MAX_KDIM] = {}, a1[MAX_KDIM] = {};
  if (kd > 0) {
    for (int i = c * chunk + w; i < i_end; i += 32) {
      int code[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) code[u] = i + 8 * u < i_end ? L.slot_code[l0 + i + 8 * u] : -1;
      double v0[4], v1[4], cf[4][MAX_KDIM];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int cu = max(code[u], 0);
        const double* vr = V + (size_t)(cu >> 1) * k + lane;
        v0[u] = c0 ? vr[0] : 0.0;
        v1[u] = WIDE && c1 ? vr[32] : 0.0;
        const double* cp = L.rowg_coef + (size_t)cu * MAX_KDIM;
#pragma unroll
        for (int m = 0; m < MAX_KDIM; ++m) cf[u][m] = (m < kd && code[u] >= 0) ? cp[m] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int m = 0; m < MAX_KDIM; ++m) {
          a0[m] = fma(cf[u][m], v0[u], a0[m]);
          if (WIDE) a1[m] = fma(cf[u][m], v1[u], a1[m]);
        }
    }
  }
#pragma unroll
  for (int m = 0; m < MAX_KDIM; ++m) {
    red[w][m][lane] = a0[m];
    red[w][m][lane + 32] = a1[m];
  }
  __syncthreads();
  const int t = threadIdx.x;
  double* part = L.gtv_part + (size_t)s * nch * MAX_KDIM * 64;
  for (int i = t; i < kd * k; i += blockDim.x) {
    const int m = i / k, g = i % k;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < GTV_THREADS / 32; ++q) v += red[q][m][g];
    if (nch == 1)
      X[(size_t)(L.occ_gofs[s] + m) * k + g] = v;
    else
      part[((size_t)c * MAX_KDIM + m) * 64 + g] = v;
  }
  if (nch == 1) return;
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&L.gtv_ticket[s], 1u) == (unsigned)(nch - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = t; i < kd * k; i += blockDim.x) {
    const int m = i / k, g = i % k;
    double v = 0.0;
    for (int q = 0; q < nch; ++q) v += __ldcg(part + ((size_t)q * MAX_KDIM + m) * 64 + g);
    X[(size_t)(L.occ_gofs[s] + m) * k + g] = v;
  }
  if (t == 0) L.gtv_ticket[s] = 0u;
}

// out[row][g] = beta*out + alpha * sum over the row's slots: (sign Nb[j]) . A[gofs(s)..][g], from the per-row
// tables (coarse column, kernel dimension and signed coefficients of each slot), so that the only dependent
// load is A's (small, cache-resident)
__global__ void k_g_apply(Layout L, const double* __restrict__ A, int k, double alpha, double beta,
                          double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_lambda * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int g0 = L.rowg_gofs[2 * row + e];
    if (g0 < 0) continue;
    const int kd = L.rowg_kd[2 * row + e];
    const double* c = L.rowg_coef + (size_t)(2 * row + e) * MAX_KDIM;
    const double* a = A + (size_t)g0 * k + g;
    double t = 0.0;
#pragma unroll
    for (int m = 0; m < MAX_KDIM; ++m)
      if (m < kd) t = fma(c[m], a[(size_t)m * k], t);
    acc += t;
  }
  double* o = out + idx;
  *o = (beta == 0.0 ? 0.0 : beta * *o) + alpha * acc;
}

// ---- double-single forms of G^T V and G A (the projections inside the inner solves of the mixed forms) -------
// The same sums on the FP32 pipe: every FP64 operand is an unevaluated pair hi + lo of FP32 values (48 bits; the
// coefficients of G and the coarse vectors are split once per call or per structure, V when it is loaded), each
// product is Dekker's exact product of the high parts plus the cross terms, and each running sum a (hi, lo)
// pair updated by Knuth's TwoSum; ~2^-46 relative, converted to FP64 at the end (Dekker 1971; Knuth, TAOCP
// vol. 2).  On this GPU the FP32 pipe issues ~75 times the FP64 one.
__device__ __forceinline__ void dsm(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float ph = __fmul_rn(ah, bh);
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  const float t = __fadd_rn(sh, ph), bb = __fsub_rn(t, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(ph, bb));
  sl = __fadd_rn(sl, __fadd_rn(e, pl));
  sh = t;
}
__device__ __forceinline__ void dsplit(double v, float& h, float& l) { d2ds(v, h, l); }

__global__ void k_split_pairs(long long n, const double* __restrict__ x, float* __restrict__ h,
                              float* __restrict__ l) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dsplit(x[i], h[i], l[i]);
}

// KL lanes per link (k <= KL <= 32, a power of two; WIDE: k <= 64 with two columns per lane and KL = 32): a warp
// works on 32 / KL links at once, so that small blocks (k = 4, 8, 16) keep every lane busy.  Lane (sub, g):
// column g of links sub, sub + 32 / KL, ...; the lanes of a column are added in FP64 by shuffles at the end.
template <int KL, bool WIDE>
__global__ void __launch_bounds__(GTV_THREADS, WIDE ? 2 : 3) k_gt_v_ds(Layout L, const double* __restrict__ V, int k,
                                                            double* __restrict__ X, int chunk) {
  static_assert(!WIDE || KL == 32, "two columns per lane only with 32 lanes per link");
  constexpr int SUB = 32 / KL;            // links a warp works on at once
  constexpr int WORKERS = (GTV_THREADS / 32) * SUB;
  __shared__ double red[GTV_THREADS / 32][MAX_KDIM][64];
  __shared__ int s_last;
  const int s = blockIdx.x, c = blockIdx.y, nch = gridDim.y;
  const int kd = L.kdim[L.occ_pat[s]];
  const int l0 = L.slot_ptr[L.occ_obase[s]], nl = L.slot_ptr[L.occ_obase[s + 1]] - l0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane % KL, sub = lane / KL, wid = w * SUB + sub;
  const bool c0 = g < k, c1 = WIDE && g + 32 < k;
  const int i_end = min(nl, (c + 1) * chunk);
  float h0[MAX_KDIM] = {}, e0[MAX_KDIM] = {}, h1[MAX_KDIM] = {}, e1[MAX_KDIM] = {};
  if (kd > 0) {
    for (int i = c * chunk + wid; i < i_end; i += 4 * WORKERS) {   // four links per step: loads in flight together
      int code[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) code[u] = i + WORKERS * u < i_end ? L.slot_code[l0 + i + WORKERS * u] : -1;
      double v0[4], v1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double* vr = V + (size_t)(max(code[u], 0) >> 1) * k + g;
        v0[u] = (c0 && code[u] >= 0) ? vr[0] : 0.0;
        v1[u] = (WIDE && c1 && code[u] >= 0) ? vr[32] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (code[u] < 0) continue;
        float vh0, vl0, vh1 = 0.f, vl1 = 0.f;
        dsplit(v0[u], vh0, vl0);
        if (WIDE) dsplit(v1[u], vh1, vl1);
        const float* ch = L.rowg_coef_hi + (size_t)code[u] * MAX_KDIM;
        const float* cl = L.rowg_coef_lo + (size_t)code[u] * MAX_KDIM;
#pragma unroll
        for (int m = 0; m < MAX_KDIM; ++m)
          if (m < kd) {
            const float a = ch[m], b = cl[m];
            dsm(a, b, vh0, vl0, h0[m], e0[m]);
            if (WIDE) dsm(a, b, vh1, vl1, h1[m], e1[m]);
          }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < MAX_KDIM; ++m) {
    double d0 = ds2d(h0[m], e0[m]), d1 = ds2d(h1[m], e1[m]);
#pragma unroll
    for (int off = KL; off < 32; off <<= 1) {   // the warp's links of column g, in a fixed order
      d0 += __shfl_xor_sync(0xffffffffu, d0, off);
      if (WIDE) d1 += __shfl_xor_sync(0xffffffffu, d1, off);
    }
    if (sub == 0) {
      red[w][m][g] = d0;
      if (WIDE) red[w][m][g + 32] = d1;
    }
  }
  __syncthreads();
  const int t = threadIdx.x;
  double* part = L.gtv_part + (size_t)s * nch * MAX_KDIM * 64;
  for (int i = t; i < kd * k; i += blockDim.x) {
    const int m = i / k, gg = i % k;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < GTV_THREADS / 32; ++q) v += red[q][m][gg];
    if (nch == 1)
      X[(size_t)(L.occ_gofs[s] + m) * k + gg] = v;
    else
      part[((size_t)c * MAX_KDIM + m) * 64 + gg] = v;
  }
  if (nch == 1) return;
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&L.gtv_ticket[s], 1u) == (unsigned)(nch - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = t; i < kd * k; i += blockDim.x) {
    const int m = i / k, gg = i % k;
    double v = 0.0;
    for (int q = 0; q < nch; ++q) v += __ldcg(part + ((size_t)q * MAX_KDIM + m) * 64 + gg);
    X[(size_t)(L.occ_gofs[s] + m) * k + gg] = v;
  }
  if (t == 0) L.gtv_ticket[s] = 0u;
}

// out = beta out + alpha G A with A given as FP32 pairs (Ah + Al)
__global__ void k_g_apply_ds(Layout L, const float* __restrict__ Ah, const float* __restrict__ Al, int k,
                             double alpha, double beta, double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_lambda * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  float h = 0.f, l = 0.f;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int g0 = L.rowg_gofs[2 * row + e];
    if (g0 < 0) continue;
    const int kd = L.rowg_kd[2 * row + e];
    const float* ch = L.rowg_coef_hi + (size_t)(2 * row + e) * MAX_KDIM;
    const float* cl = L.rowg_coef_lo + (size_t)(2 * row + e) * MAX_KDIM;
    const size_t a0 = (size_t)g0 * k + g;
#pragma unroll
    for (int m = 0; m < MAX_KDIM; ++m)
      if (m < kd) dsm(ch[m], cl[m], Ah[a0 + (size_t)m * k], Al[a0 + (size_t)m * k], h, l);
  }
  double* o = out + idx;
  const double x = ds2d(h, l);
  // the projection's call (alpha = -1, beta = 1) costs one FP64 add per element
  const bool minus = bits64(alpha) == bits64(-1.0), keep = bits64(beta) == bits64(1.0);
  if (keep && minus) *o = *o - x;
  else *o = is_zero(beta) ? alpha * x : fma(alpha, x, beta * *o);
}

// The same for k = K (4 or 8) with one thread per row: the row's links and coefficients are read once for all K
// columns, the coarse pairs as float4; per element the same products in the same order as k_g_apply_ds.
template <int K>
__global__ void k_g_apply_ds_rows(Layout L, const float* __restrict__ Ah, const float* __restrict__ Al,
                                  double alpha, double beta, double* __restrict__ out) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= L.n_lambda) return;
  float h[K], l[K];
#pragma unroll
  for (int g = 0; g < K; ++g) h[g] = l[g] = 0.f;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int g0 = L.rowg_gofs[2 * row + e];
    if (g0 < 0) continue;
    const int kd = L.rowg_kd[2 * row + e];
    const float* ch = L.rowg_coef_hi + (size_t)(2 * row + e) * MAX_KDIM;
    const float* cl = L.rowg_coef_lo + (size_t)(2 * row + e) * MAX_KDIM;
#pragma unroll
    for (int m = 0; m < MAX_KDIM; ++m)
      if (m < kd) {
        const float a = ch[m], b = cl[m];
        const float4* ph = reinterpret_cast<const float4*>(Ah + (size_t)(g0 + m) * K);
        const float4* pl = reinterpret_cast<const float4*>(Al + (size_t)(g0 + m) * K);
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
          const float4 vh = ph[q], vl = pl[q];
          dsm(a, b, vh.x, vl.x, h[4 * q], l[4 * q]);
          dsm(a, b, vh.y, vl.y, h[4 * q + 1], l[4 * q + 1]);
          dsm(a, b, vh.z, vl.z, h[4 * q + 2], l[4 * q + 2]);
          dsm(a, b, vh.w, vl.w, h[4 * q + 3], l[4 * q + 3]);
        }
      }
  }
  double* o = out + (size_t)row * K;
  const bool minus = bits64(alpha) == bits64(-1.0), keep = bits64(beta) == bits64(1.0);
#pragma unroll
  for (int g = 0; g < K; ++g) {
    const double x = ds2d(h[g], l[g]);
    if (keep && minus) o[g] = o[g] - x;
    else o[g] = is_zero(beta) ? alpha * x : fma(alpha, x, beta * o[g]);
  }
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
    const double* ns = L.slot_nb ? L.slot_nb + (size_t)slot * MAX_KDIM : L.Nb[ps] + (size_t)(slot - b0) * ks;
    for (int e = L.slot_ptr[slot]; e < L.slot_ptr[slot + 1]; ++e) {
      const int row = L.slot_row[e];
      const int sg = L.slot_sign[e];
      for (int f = 0; f < 2; ++f) {
        const int sg2 = L.row_sign[2 * row + f];
        if (sg2 == 0) continue;
        const int slot2 = L.row_slot[2 * row + f];
        if (L.slot_occ[slot2] != t) continue;
        const double* nt =
            L.slot_nb ? L.slot_nb + (size_t)slot2 * MAX_KDIM : L.Nb[pt] + (size_t)(slot2 - L.occ_obase[t]) * kt;
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

// Gather of one tile of GT_SLOTS slots of an occurrence (grid: occurrence x tile).  The tile's slot pointers and
// links (a contiguous range of the slot CSR) are staged in shared memory; warp w takes slots w, w + 8, ...: the
// first link of all its eight slots is loaded at once (most slots have one link), further links after; lane =
// column g (and g + 32), so a link reads one contiguous row of V.  The traces go through a shared tile and are
// written column by column (pattern frame, Eq. 9 blocked storage), coalesced over the slots.  Per slot the
// links are added in CSR order, as the plain definition does.
constexpr int GT_SLOTS = 64, GT_LINKS = 512;
// SPLIT 0: plain; 1: FP32 value split into a tf32 pair (TO = float); 2: split into a bf16 pair (TO = bf16),
// hi -> Y, lo -> Y2.  The links are summed in FP64: the first link's signed value by a sign-bit flip, each further
// one (a minority of the slots have more than one) by an FP64 add; FP32 and narrower outputs are then rounded to
// FP32 by integer operations (d2f_rn), so that the narrow FP64 pipe does no per-element conversion.
// KL lanes per slot (k <= KL for KL < 32; KL = 32 also takes k <= 64 with a second column per lane): a warp
// works on 32 / KL slots at once, so that small blocks keep every lane busy.
template <typename TO, int SPLIT, int KL>
__global__ void __launch_bounds__(256) k_gather_tile(Layout L, const double* __restrict__ V, int k, PatView<TO> Y,
                                                     PatView<TO> Y2, double alpha, double beta) {
  using ACC = std::conditional_t<std::is_same<TO, double>::value, double, float>;
  constexpr int SUB = 32 / KL, UPW = 8 / SUB;   // slots a warp works on at once; slots per lane
  __shared__ int sptr[GT_SLOTS + 1];
  __shared__ int srow[GT_LINKS];
  __shared__ int8_t ssg[GT_LINKS];
  __shared__ ACC tile[GT_SLOTS][65];
  const int s = blockIdx.x;
  const int b0 = L.occ_obase[s], nb = L.occ_obase[s + 1] - b0;
  const int j0 = blockIdx.y * GT_SLOTS;
  if (j0 >= nb) return;   // grid.y covers the largest occurrence
  const int p = L.occ_pat[s], q = L.occ_q[s];
  const int ns = min(GT_SLOTS, nb - j0);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t <= ns) sptr[t] = L.slot_ptr[b0 + j0 + t];
  __syncthreads();
  const int e0 = sptr[0], ne = sptr[ns] - e0;
  const bool fits = ne <= GT_LINKS;
  if (fits)
    for (int i = t; i < ne; i += blockDim.x) {
      srow[i] = L.slot_row[e0 + i];
      ssg[i] = L.slot_sign[e0 + i];
    }
  __syncthreads();
  const int* lr = fits ? srow : L.slot_row + e0;
  const int8_t* ls = fits ? ssg : L.slot_sign + e0;
  const int g = lane % KL, wid = w * SUB + lane / KL;   // column, slot worker (8 SUB workers)
  const bool c0 = g < k, c1 = KL == 32 && g + 32 < k;
  double y0[UPW], y1[UPW];
  int ea[UPW], eb[UPW];
#pragma unroll
  for (int u = 0; u < UPW; ++u) {
    const int jl = wid + 8 * SUB * u;
    ea[u] = jl < ns ? sptr[jl] - e0 : 0;
    eb[u] = jl < ns ? sptr[jl + 1] - e0 : 0;
    y0[u] = 0.0;
    y1[u] = 0.0;
    if (ea[u] < eb[u]) {
      const bool neg = ls[ea[u]] < 0;
      const double* vr = V + (size_t)lr[ea[u]] * k + g;
      if (c0) y0[u] = neg_if(vr[0], neg);
      if (c1) y1[u] = neg_if(vr[32], neg);
    }
  }
#pragma unroll
  for (int u = 0; u < UPW; ++u) {
    for (int e = ea[u] + 1; e < eb[u]; ++e) {
      const bool neg = ls[e] < 0;
      const double* vr = V + (size_t)lr[e] * k + g;
      if (c0) y0[u] += neg_if(vr[0], neg);
      if (c1) y1[u] += neg_if(vr[32], neg);
    }
    const int jl = wid + 8 * SUB * u;
    if (jl < ns) {
      tile[jl][g] = from_f64<ACC>(y0[u]);
      if (KL == 32) tile[jl][g + 32] = from_f64<ACC>(y1[u]);
    }
  }
  __syncthreads();
  const long long ld = Y.ld[p], off = Y.off[p] + j0;
  for (int idx = t; idx < k * GT_SLOTS; idx += blockDim.x) {
    const int g = idx / GT_SLOTS, jl = idx % GT_SLOTS;
    if (jl >= ns) continue;
    const long long o = ((long long)q * k + g) * ld + off + jl;
    if constexpr (SPLIT == 1) {
      const float v = tile[jl][g];
      uint32_t h;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
      Y.base[p][o] = (TO)__uint_as_float(h);
      Y2.base[p][o] = (TO)(v - __uint_as_float(h));
    } else if constexpr (SPLIT == 2) {
      const float v = tile[jl][g];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      Y.base[p][o] = (TO)h;
      Y2.base[p][o] = (TO)__float2bfloat16_rn(v - __bfloat162float(h));
    } else {
      TO* y = Y.base[p] + o;
      const ACC a = (ACC)alpha, b = (ACC)beta;
      *y = (TO)(b == ACC(0) ? a * tile[jl][g] : b * (ACC)*y + a * tile[jl][g]);
    }
  }
}
// Node-by-node rotation of the traces of the occurrences with a general rotation (grid: node-column tiles x
// listed occurrence).  MODE 0: y <- R y (pattern frame -> global frame); 1: y <- R^T y; 2: the trace is the
// tf32 pair y = Y + Y2 (from the splitting gather): y <- R^T y, split again into a tf32 pair (hi -> Y,
// lo -> Y2).  Products in FP64.
template <typename T, int MODE>
__global__ void k_rotate_traces(Layout L, PatView<T> Y, PatView<T> Y2, int k) {
  const int i = blockIdx.y;
  const int s = L.gen_occ[i];
  const int p = L.occ_pat[s], q = L.occ_q[s];
  const int dpn = L.dpn[p];
  const int nbn = L.n_b[p] / dpn;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nbn * k) return;
  const int g = (int)(idx / nbn), b = (int)(idx % nbn);
  const double* R = L.gen_R + 9 * (size_t)i;
  const long long o = ((long long)q * k + g) * Y.ld[p] + Y.off[p] + (long long)b * dpn;
  T* y = Y.base[p] + o;
  double v[3] = {0.0, 0.0, 0.0}, w[3];
  for (int c = 0; c < dpn; ++c) v[c] = MODE == 2 ? (double)y[c] + (double)Y2.base[p][o + c] : (double)y[c];
  for (int c = 0; c < dpn; ++c) {
    double t = 0.0;
    for (int c2 = 0; c2 < dpn; ++c2) t = fma(MODE == 0 ? R[3 * c + c2] : R[3 * c2 + c], v[c2], t);
    w[c] = t;
  }
  for (int c = 0; c < dpn; ++c) {
    if (MODE == 2) {
      const float f = (float)w[c];
      uint32_t h;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
      y[c] = (T)__uint_as_float(h);
      Y2.base[p][o + c] = (T)(f - __uint_as_float(h));
    } else {
      y[c] = (T)w[c];
    }
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
    const TI z = Z.base[p][((long long)q * k + g) * Z.ld[p] + Z.off[p] + j];
    double v;
    if constexpr (std::is_same<TI, float>::value) v = f2d(z);   // exact, integer operations
    else v = (double)z;
    v = neg_if(v, sg < 0);
    acc = e == 0 ? v : acc + v;   // the first slot costs no FP64 add
  }
  double* o = out + idx;
  *o = is_zero(beta) ? acc : beta * *o + acc;
}

// S(r)[row][g] = sum over the row's slots in column g of r[row] / (slots of the row); one thread per element
// (coalesced stores), from the per-row column and weight tables
__global__ void k_split(Layout L, const double* __restrict__ r, int k, double* __restrict__ Z) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_lambda * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  const int g0 = L.row_grp[2 * row], g1 = L.row_grp[2 * row + 1];
  const bool m0 = g0 == g, m1 = g1 == g;
  double z = 0.0;
  if (m0 || m1) {   // at most two of a row's k elements: the FP64 product only there
    const double w = r[row] * L.row_wt[row];
    z = m0 && m1 ? w + w : w;
  }
  Z[idx] = z;
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
  if (k > 32)
    k_gt_v<true><<<dim3(L.n_occ, L.gtv_chunks), GTV_THREADS, 0, s>>>(L, V, k, X, L.gtv_chunk);
  else
    k_gt_v<false><<<dim3(L.n_occ, L.gtv_chunks), GTV_THREADS, 0, s>>>(L, V, k, X, L.gtv_chunk);
  FETIRP_LAUNCH_CHECK();
}


void gt_v_ds(const Layout& L, const double* V, int k, double* X, cudaStream_t s) {
  if (L.n_occ == 0) return;
  if (k > 64) throw Error(1, "k > 64");
  if (!L.rowg_coef_hi) throw Error(1, "double-single coefficients of G not built");
  // Chunk of links per CTA: the layout's (sized for 32 lanes per link), or, when a warp works on several links at
  // once (k <= 16), long enough for about eight rounds of four links per worker, so that the loads in flight
  // rather than the per-CTA reduction and its ticket set the time; never more chunks than the layout's partials.
  const int kl = k > 16 ? 32 : k > 8 ? 16 : k > 4 ? 8 : 4;
  const int workers = (GTV_THREADS / 32) * (32 / kl);
  const int max_links = L.gtv_chunk * L.gtv_chunks;   // >= the links of the largest occurrence
  int nch = L.gtv_chunks;
  if (8 * 4 * workers > L.gtv_chunk) nch = std::max(1, std::min(nch, ceil_div(max_links, 8 * 4 * workers)));
  const int chunk = (int)round_up(ceil_div(max_links, nch), 32);
  const dim3 grid(L.n_occ, ceil_div(max_links, chunk));
  if (k > 32) k_gt_v_ds<32, true><<<grid, GTV_THREADS, 0, s>>>(L, V, k, X, chunk);
  else if (k > 16) k_gt_v_ds<32, false><<<grid, GTV_THREADS, 0, s>>>(L, V, k, X, chunk);
  else if (k > 8) k_gt_v_ds<16, false><<<grid, GTV_THREADS, 0, s>>>(L, V, k, X, chunk);
  else if (k > 4) k_gt_v_ds<8, false><<<grid, GTV_THREADS, 0, s>>>(L, V, k, X, chunk);
  else k_gt_v_ds<4, false><<<grid, GTV_THREADS, 0, s>>>(L, V, k, X, chunk);
  FETIRP_LAUNCH_CHECK();
}

// G restricted to the rows (Layout.rowg_*): entry (row, e) of row r is sign * N_b of the e-th slot's occurrence at
// the slot's dof, in the global frame; for a general rotation R of the occurrence (node b, global component c)
// sum_c2 R[c][c2] N_b[b dpn + c2].  rowg_gofs / rowg_kd (the structure) are given; the values come from the
// patterns' current kernels, so they follow every refactorisation.  Also their FP32 pairs (hi = fl32(v),
// lo = fl32(v - hi)) and, with general rotations, slot_nb.
__device__ __forceinline__ double slot_kernel(const Layout& L, const double* __restrict__ rot,
                                              const int8_t* __restrict__ general, int slot, int m) {
  const int o = L.slot_occ[slot];
  const int p = L.occ_pat[o];
  const int j = slot - L.occ_obase[o], kd = L.kdim[p];
  const double* nb = L.Nb[p];
  if (!general[o]) return nb[(size_t)j * kd + m];
  const int dpn = L.dpn[p], b = j / dpn, c = j % dpn;
  const double* R = rot + (size_t)9 * o;
  double v = 0.0;
  for (int c2 = 0; c2 < dpn; ++c2) v += R[3 * c + c2] * nb[(size_t)(b * dpn + c2) * kd + m];
  return v;
}

__global__ void k_row_coefs(Layout L, const double* __restrict__ rot, const int8_t* __restrict__ general,
                            double* __restrict__ coef, float* __restrict__ hi, float* __restrict__ lo) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // 2 row + e
  if (i >= 2 * (long long)L.n_lambda) return;
  const int kd = L.rowg_kd[i];
  const int slot = L.row_slot[i];
  const double sg = (double)L.row_sign[i];
#pragma unroll
  for (int m = 0; m < MAX_KDIM; ++m) {
    const double v = m < kd ? sg * slot_kernel(L, rot, general, slot, m) : 0.0;
    const float h = __double2float_rn(v);
    coef[i * MAX_KDIM + m] = v;
    hi[i * MAX_KDIM + m] = h;
    lo[i * MAX_KDIM + m] = __double2float_rn(v - (double)h);
  }
}

__global__ void k_slot_kernels(Layout L, const double* __restrict__ rot, const int8_t* __restrict__ general,
                               double* __restrict__ snb) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= L.n_slots) return;
  const int kd = L.kdim[L.occ_pat[L.slot_occ[slot]]];
#pragma unroll
  for (int m = 0; m < MAX_KDIM; ++m) snb[(size_t)slot * MAX_KDIM + m] = m < kd ? slot_kernel(L, rot, general, slot, m) : 0.0;
}

void row_coefs(const Layout& L, const double* rot, const int8_t* general, double* coef, float* hi, float* lo,
               double* slot_nb, cudaStream_t s) {
  const long long n = 2 * (long long)L.n_lambda;
  if (n > 0) {
    k_row_coefs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, rot, general, coef, hi, lo);
    FETIRP_LAUNCH_CHECK();
  }
  if (slot_nb && L.n_slots > 0) {
    k_slot_kernels<<<ceil_div(L.n_slots, 256), 256, 0, s>>>(L, rot, general, slot_nb);
    FETIRP_LAUNCH_CHECK();
  }
}

void split_pairs(long long n, const double* x, float* h, float* l, cudaStream_t s) {
  if (n <= 0) return;
  k_split_pairs<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, x, h, l);
  FETIRP_LAUNCH_CHECK();
}

void g_apply_ds(const Layout& L, const float* Ah, const float* Al, int k, double alpha, double beta, double* out,
                cudaStream_t s) {
  long long n = (long long)L.n_lambda * k;
  if (n == 0) return;
  const bool vec = (reinterpret_cast<uintptr_t>(Ah) | reinterpret_cast<uintptr_t>(Al)) % 16 == 0;
  if (k == 4 && vec)
    k_g_apply_ds_rows<4><<<ceil_div(L.n_lambda, 256), 256, 0, s>>>(L, Ah, Al, alpha, beta, out);
  else if (k == 8 && vec)
    k_g_apply_ds_rows<8><<<ceil_div(L.n_lambda, 256), 256, 0, s>>>(L, Ah, Al, alpha, beta, out);
  else
    k_g_apply_ds<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, Ah, Al, k, alpha, beta, out);
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

static int max_slots(const Layout& L) {
  int m = 1;
  for (int p = 0; p < L.n_pat; ++p) m = std::max(m, L.n_b[p]);
  return m;
}
// launch k_gather_tile with the lanes per slot that fit k
template <typename TO, int SPLIT>
void launch_gather_tile(const Layout& L, const double* V, int k, const PatView<TO>& Y, const PatView<TO>& Y2,
                        double alpha, double beta, cudaStream_t s) {
  const dim3 grid(L.n_occ, ceil_div(max_slots(L), GT_SLOTS));
  if (k > 16) k_gather_tile<TO, SPLIT, 32><<<grid, 256, 0, s>>>(L, V, k, Y, Y2, alpha, beta);
  else if (k > 8) k_gather_tile<TO, SPLIT, 16><<<grid, 256, 0, s>>>(L, V, k, Y, Y2, alpha, beta);
  else if (k > 4) k_gather_tile<TO, SPLIT, 8><<<grid, 256, 0, s>>>(L, V, k, Y, Y2, alpha, beta);
  else k_gather_tile<TO, SPLIT, 4><<<grid, 256, 0, s>>>(L, V, k, Y, Y2, alpha, beta);
  FETIRP_LAUNCH_CHECK();
}

template <typename TO>
void gather(const Layout& L, const double* V, int k, const PatView<TO>& Y, cudaStream_t s, double alpha,
            double beta) {
  if (L.n_occ == 0) return;
  if (k > 64) throw Error(1, "k > 64");
  launch_gather_tile<TO, 0>(L, V, k, Y, Y, alpha, beta, s);
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
  if (k > 64) throw Error(1, "k > 64");
  launch_gather_tile<float, 1>(L, V, k, Yh, Yl, 1.0, 0.0, s);
}

__global__ void k_perm_split(int n, int k, int pw, const int* __restrict__ src, const double* __restrict__ w,
                             const double* __restrict__ r, double* __restrict__ Z, int g_only) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int kk = g_only >= 0 ? 1 : k;
  if (idx >= (long long)n * kk) return;
  const int row = (int)(idx / kk), g = g_only >= 0 ? g_only : (int)(idx % kk);
  const size_t e0 = ((size_t)row * k + g) * pw;
  double z = 0.0;
  for (int e = 0; e < pw; ++e) {
    const double we = w[e0 + e];
    if (we != 0.0) z = fma(we, r[src[e0 + e]], z);
  }
  Z[idx] = z;
}
void perm_split(int n, int k, int pw, const int* src, const double* w, const double* r, double* Z, cudaStream_t s,
                int g_only) {
  const long long tot = (long long)n * (g_only >= 0 ? 1 : k);
  if (tot == 0) return;
  k_perm_split<<<(unsigned)ceil_div(tot, 256), 256, 0, s>>>(n, k, pw, src, w, r, Z, g_only);
  FETIRP_LAUNCH_CHECK();
}

static int max_nodes(const Layout& L) {
  int m = 1;
  for (int p = 0; p < L.n_pat; ++p) m = std::max(m, L.n_b[p] / std::max(L.dpn[p], 1));
  return m;
}
template <typename T>
void rotate_traces(const Layout& L, const PatView<T>& Y, int k, bool to_local, cudaStream_t s) {
  if (L.n_gen == 0) return;
  const dim3 grid((unsigned)ceil_div((long long)max_nodes(L) * k, 256), L.n_gen);
  if (to_local) k_rotate_traces<T, 1><<<grid, 256, 0, s>>>(L, Y, Y, k);
  else k_rotate_traces<T, 0><<<grid, 256, 0, s>>>(L, Y, Y, k);
  FETIRP_LAUNCH_CHECK();
}
template void rotate_traces<double>(const Layout&, const PatView<double>&, int, bool, cudaStream_t);
template void rotate_traces<float>(const Layout&, const PatView<float>&, int, bool, cudaStream_t);
void rotate_split(const Layout& L, const PatView<float>& Yh, const PatView<float>& Yl, int k, cudaStream_t s) {
  if (L.n_gen == 0) return;
  const dim3 grid((unsigned)ceil_div((long long)max_nodes(L) * k, 256), L.n_gen);
  k_rotate_traces<float, 2><<<grid, 256, 0, s>>>(L, Yh, Yl, k);
  FETIRP_LAUNCH_CHECK();
}

void gather_split_bf16(const Layout& L, const double* V, int k, const PatView<__nv_bfloat16>& Yh,
                       const PatView<__nv_bfloat16>& Yl, cudaStream_t s) {
  if (L.n_occ == 0) return;
  if (k > 64) throw Error(1, "k > 64");
  launch_gather_tile<__nv_bfloat16, 2>(L, V, k, Yh, Yl, 1.0, 0.0, s);
}

void split(const Layout& L, const double* r, int k, double* Z, cudaStream_t s) {
  if (L.n_lambda == 0) return;
  k_split<<<(unsigned)ceil_div((long long)L.n_lambda * k, 256), 256, 0, s>>>(L, r, k, Z);
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
