// Kernels of the preconditioned iteration: the weighted gather/scatter of the preconditioners of Eqs. 4-5,
// tilde-F^{-1} V = sum_s Delta(s) B(s) X(s) B(s)^T Delta(s) V, and the scaled occurrence split of the
// preconditioned residual.
#include "ops.cuh"

namespace fetirp {

// Y(slot, g) = sum over the slot's links e: w[e] V[row_e][g] (w = sign x Delta of the link; slot CSR order)
__global__ void k_gather_w(Layout L, const double* __restrict__ V, int k, PatView<double> Y,
                           const double* __restrict__ link_w) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_slots * k) return;
  const int slot = (int)(idx / k), g = (int)(idx % k);
  const int s = L.slot_occ[slot];
  const int p = L.occ_pat[s], q = L.occ_q[s];
  const int j = slot - L.occ_obase[s];
  double y = 0.0;
  for (int e = L.slot_ptr[slot]; e < L.slot_ptr[slot + 1]; ++e) y = fma(link_w[e], V[(size_t)L.slot_row[e] * k + g], y);
  Y.base[p][((long long)q * k + g) * Y.ld[p] + Y.off[p] + j] = y;
}

// out[row][g] = sum over the row's (at most two) slots: row_w[2 row + e] Z(slot_e, g)
__global__ void k_scatter_w(Layout L, PatView<double> Z, int k, const double* __restrict__ row_w,
                            double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_lambda * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (L.row_sign[2 * row + e] == 0) continue;
    const int slot = L.row_slot[2 * row + e];
    const int s = L.slot_occ[slot];
    const int p = L.occ_pat[s], q = L.occ_q[s];
    const int j = slot - L.occ_obase[s];
    acc = fma(row_w[2 * row + e], Z.base[p][((long long)q * k + g) * Z.ld[p] + Z.off[p] + j], acc);
  }
  out[idx] = acc;
}

// Z[row][g] = sum over the row's slots whose occurrence is in column g: row_d[2 row + e] z[row]
__global__ void k_split_w(Layout L, const double* __restrict__ z, int k, const double* __restrict__ row_d,
                          double* __restrict__ Z) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)L.n_lambda * k) return;
  const int row = (int)(idx / k), g = (int)(idx % k);
  double v = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e)
    if (L.row_grp[2 * row + e] == g) v = fma(row_d[2 * row + e], z[row], v);
  Z[idx] = v;
}

void gather_w(const Layout& L, const double* V, int k, const PatView<double>& Y, const double* link_w,
              cudaStream_t s) {
  const long long n = (long long)L.n_slots * k;
  if (n == 0) return;
  k_gather_w<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(L, V, k, Y, link_w);
  FETIRP_LAUNCH_CHECK();
}

void scatter_w(const Layout& L, const PatView<double>& Z, int k, const double* row_w, double* out, cudaStream_t s) {
  const long long n = (long long)L.n_lambda * k;
  if (n == 0) return;
  k_scatter_w<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(L, Z, k, row_w, out);
  FETIRP_LAUNCH_CHECK();
}

void split_w(const Layout& L, const double* z, int k, const double* row_d, double* Z, cudaStream_t s) {
  const long long n = (long long)L.n_lambda * k;
  if (n == 0) return;
  k_split_w<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(L, z, k, row_d, Z);
  FETIRP_LAUNCH_CHECK();
}

}  // namespace fetirp
