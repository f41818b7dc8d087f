// Tensor-core (tcgen05) local products; see tc_gemm.cu.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace fetirp {

constexpr int TC_MAXP = 4;   // patterns per launch (tensor maps travel as kernel parameters)

// Operands are tf32 pairs (FP32 arrays) or bf16 pairs (bf16 arrays); leading dimensions in elements, 16-byte rows.
struct TcProblem {
  int n_pat = 0;
  const void* S_hi[16];    // n_b x n_b, leading dimension lds, rounded high part
  const void* S_lo[16];    // S - S_hi, rounded
  long long lds[16];
  const void* Y_hi[16];    // n_rhs x n_b (K contiguous), leading dimension ldy
  const void* Y_lo[16];
  float* Z[16];            // n_rhs x n_b, leading dimension ldy
  long long ldy[16];
  int n_b[16];
  int n_rhs[16];
  // K-split scratch: when the output tiles alone would leave SMs idle, the reduction dimension is split over
  // tc_ksplits(*this) CTAs per tile whose FP32 partials (layout of Z, one copy per split) are added in split order;
  // part_elems must then be at least tc_ksplits(*this) * sum_p n_rhs[p] * ldy[p] (else no split is made)
  float* part = nullptr;
  long long part_elems = 0;
};

// K-split factor of the tensor-core product of T (1 or 2): 2 when at most half an SM's worth of 256 x 256 output
// tiles exist and the reduction dimension is long enough to share.
int tc_ksplits(const TcProblem& T);

// Z = (S_hi + S_lo)(Y_hi + Y_lo) without the lo*lo term, FP32 accumulation in TMEM.  d_error: device int
// that receives a nonzero code if a bounded wait inside the kernel expired (0 otherwise).
void tc_gemm_tf32x3(const TcProblem& T, int* d_error, cudaStream_t s);
// The same with bf16 pairs (kind::f16: twice the tf32 tensor rate, 16 significant bits per pair).
void tc_gemm_bf16x3(const TcProblem& T, int* d_error, cudaStream_t s);

// One-time kernel attribute set-up (large dynamic shared memory); call before any graph capture.
void tc_init();

// hi = bf16(x), lo = bf16(x - hi) (round to nearest) of x rounded to FP32; x is FP64 or FP32, outputs bf16 with
// leading dimension ld_out (columns cols .. ld_out - 1 zero).  In place (x == hi) is not allowed.
void split_bf16(const double* x, long long rows, long long cols, long long ld_in, __nv_bfloat16* hi,
                __nv_bfloat16* lo, long long ld_out, cudaStream_t s);
void split_bf16(const float* x, long long rows, long long cols, long long ld_in, __nv_bfloat16* hi,
                __nv_bfloat16* lo, long long ld_out, cudaStream_t s);
// hi = tf32(x) (round to nearest), lo = x - hi of x rounded to FP32; x is FP64, outputs FP32 with leading
// dimension ld_out.
void split_tf32(const double* x, long long rows, long long cols, long long ld_in, float* hi, float* lo,
                long long ld_out, cudaStream_t s);
// The nb rows of Y^T = (Lam Pi)^T in tf32 pairs, where Lam = L_S^{-1} is stored transposed (X[i * ldx + j] =
// Lam(j, i)), Pi = I - N_b (N_b^T N_b)^{-1} N_b^T the orthogonal projector off the kernel traces, A = Lam N_b and
// E = N_b (N_b^T N_b)^{-1} (nb x kd, row-major; kd = 0: Pi = I).  Y^T Y = Pi S^+ Pi = S^dag (Moore-Penrose).
void pinv_rows_tf32(const double* X, long long ldx, const double* A, const double* E, int kd, long long nb,
                    float* hi, float* lo, long long ld_out, cudaStream_t s);

}  // namespace fetirp
