// Tensor-core (tcgen05) local products; see tc_gemm.cu.
#pragma once
#include "common.cuh"

namespace fetirp {

constexpr int TC_MAXP = 4;   // patterns per launch (tensor maps travel as kernel parameters)

struct TcProblem {
  int n_pat = 0;
  const float* S_hi[16];   // n_b x n_b, leading dimension lds (multiple of 4), tf32-rounded high part
  const float* S_lo[16];   // S - S_hi
  long long lds[16];
  const float* Y_hi[16];   // n_rhs x n_b (K contiguous), leading dimension ldy (multiple of 4)
  const float* Y_lo[16];
  float* Z[16];            // n_rhs x n_b, leading dimension ldy
  long long ldy[16];
  int n_b[16];
  int n_rhs[16];
};

// Z = (S_hi + S_lo)(Y_hi + Y_lo) without the lo*lo term, FP32 accumulation in TMEM.  d_error: device int
// that receives a nonzero code if a bounded wait inside the kernel expired (0 otherwise).
void tc_gemm_tf32x3(const TcProblem& T, int* d_error, cudaStream_t s);

// One-time kernel attribute set-up (large dynamic shared memory); call before any graph capture.
void tc_init();

// hi = tf32(x) (round to nearest), lo = x - hi; x is FP64, outputs FP32 with leading dimension ld_out.
void split_tf32(const double* x, long long rows, long long cols, long long ld_in, float* hi, float* lo,
                long long ld_out, cudaStream_t s);

}  // namespace fetirp
