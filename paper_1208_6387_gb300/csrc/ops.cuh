// Device layout of one structure and the interface operators of the hot path.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace fetirp {

constexpr int MAXP = 16;   // patterns per structure handled by one launch

// Per-pattern view of a block of local vectors: element (occurrence q of the pattern, column g, boundary
// dof j) lives at base[(q * k + g) * ld + off + j].  Used for Y (gathered traces) and Z (local solutions).
template <typename T>
struct PatView {
  T* base[MAXP];
  long long ld[MAXP];
  long long off[MAXP];
};

// Structure layout on the device (built once per structure).  "Slot" = (occurrence s, boundary dof j),
// slot = obase[s] + j.  Links are folded into the pattern frame (rotation sign included).
struct Layout {
  int n_lambda = 0, n_occ = 0, n_slots = 0, n_G = 0, n_pat = 0, k = 1;
  // gather CSR by slot: entries (row, sign)
  const int* slot_ptr;
  const int* slot_row;
  const int8_t* slot_sign;
  const int* slot_code;   // 2 row + e: the link's entry (row, e-th slot of the row) in the per-row tables
  // the same links in ELL form: ell_w entries per slot (sign 0 = padding, row 0)
  int ell_w = 1;
  const int* ell_row;
  const int8_t* ell_sign;
  // scatter by row: up to two (slot, sign); sign 0 = empty
  const int* row_slot;
  const int8_t* row_sign;
  const int* slot_occ;   // slot -> occurrence
  // occurrence tables
  const int* occ_obase;  // n_occ + 1
  const int* occ_pat;
  const int* occ_q;      // index among the pattern's occurrences
  const int* occ_gofs;   // first coarse column of the occurrence
  const int* occ_group;  // multivector column
  // pattern tables (indexed by pattern)
  const double* Nb[MAXP];   // n_b x kdim row-major: kernel restricted to the boundary (pattern frame)
  int n_b[MAXP];
  int kdim[MAXP];
  // split by row: the multivector column of each of the row's two slots (-1: none) and 1 / (slots of the row)
  const int* row_grp;
  const double* row_wt;
  // G by row: for each of the row's two slots, the occurrence's first coarse column (-1: none), its kernel
  // dimension and sign * Nb[j][m] (m < 6)
  const int* rowg_gofs;
  const int* rowg_kd;
  const double* rowg_coef;
  // G^T V: links per CTA, CTAs per occurrence, per-chunk partial sums (n_occ x gtv_chunks x 6 x 64) and the
  // per-occurrence tickets of the last-CTA reduction (zero between launches)
  int gtv_chunk = 1, gtv_chunks = 1;
  double* gtv_part;
  unsigned* gtv_ticket;
  // occurrences whose rotation is not a signed permutation (vector fields only): their links stay in the global
  // frame (slot = boundary node x dofs per node + GLOBAL component), and the traces are turned into the pattern
  // frame (R^T per node) after the gather and back (R) before the scatter.  gen_R: 9 doubles (row-major R) per
  // listed occurrence.  slot_nb (NULL when n_gen = 0): the global-frame kernel restricted to every slot,
  // MAX_KDIM values per slot (R-hat N_b of the slot's occurrence).
  // the coefficients rowg_coef as FP32 pairs (hi + lo) for the double-single projections (NULL: not built)
  const float* rowg_coef_hi = nullptr;
  const float* rowg_coef_lo = nullptr;
  int n_gen = 0;
  const int* gen_occ = nullptr;
  const double* gen_R = nullptr;
  const double* slot_nb = nullptr;
  int dpn[MAXP];
};

// ---- coarse space G = [ ... B(s) N(s) ... ] (Eq. 3) ------------------------------------------------
// X[gofs(s) + m][g] = sum over links (row, sign) of s: sign * Nb[j][m] * V[row][g]   (X = G^T V)
void gt_v(const Layout& L, const double* V, int k, double* X, cudaStream_t s);
// out[row][g] = beta * out[row][g] + alpha * (G A)[row][g]
void g_apply(const Layout& L, const double* A, int k, double alpha, double beta, double* out, cudaStream_t s);
// Double-single forms (FP32 pairs, ~2^-46 relative; the inner solves of the mixed forms): X = G^T V, and
// out = beta out + alpha G A with A given as pairs Ah + Al (split_pairs); need Layout.rowg_coef_hi/lo.
void gt_v_ds(const Layout& L, const double* V, int k, double* X, cudaStream_t s);
void g_apply_ds(const Layout& L, const float* Ah, const float* Al, int k, double alpha, double beta, double* out,
                cudaStream_t s);
// h[i] + l[i] = x[i] to ~2^-48 (h = fl32(x), l = fl32(x - h))
void split_pairs(long long n, const double* x, float* h, float* l, cudaStream_t s);
// C (m x k) = A B with A given as FP32 pairs (m x m) and B as FP32 pairs (m x k), double-single sums, FP64 out
void small_gemm_ds(int m, int k, const float* Ah, const float* Al, const float* Bh, const float* Bl, double* C,
                   cudaStream_t s, double* part = nullptr);
// dense G^T G (n_G x n_G, row-major), nb_ptr/nb_list: neighbour occurrences of every occurrence
// Layout.rowg_coef and its FP32 pairs (hi, lo; 12 n_lambda entries each) from the patterns' kernels N_b, with
// rot (9 per occurrence) and general (1 = a general rotation); slot_nb (n_slots x 6, may be NULL) likewise.
// Reads Layout's row, slot, occurrence tables, Nb, kdim, dpn and rowg_kd.
void row_coefs(const Layout& L, const double* rot, const int8_t* general, double* coef, float* hi, float* lo,
               double* slot_nb, cudaStream_t s);
void gtg_dense(const Layout& L, const int* nb_ptr, const int* nb_list, int n_pairs, const int* pair_s,
               const int* pair_t, double* GtG, cudaStream_t s);

// ---- gather / scatter (Eq. 9 blocked storage, signed Boolean assembly) -------------------------------
// Y[(q * k + g) * ld + off + j] = beta * Y[...] + alpha * sum over links of slot (s, j): sign * V[row][g]
template <typename TO>
void gather(const Layout& L, const double* V, int k, const PatView<TO>& Y, cudaStream_t s, double alpha = 1.0,
            double beta = 0.0);
// Turn the traces of the occurrences with a general rotation (Layout.gen_occ) between the global frame and the
// pattern frame, node by node, in place: to_local: y <- R^T y (after the gather); else y <- R y (before the
// scatter).  Y as in gather; k columns.
template <typename T>
void rotate_traces(const Layout& L, const PatView<T>& Y, int k, bool to_local, cudaStream_t s);
// to the pattern frame as rotate_traces(to_local) on the tf32 pairs (Yh + Yl) that gather_split wrote for
// every occurrence, then split again into a tf32 pair in place (hi -> Yh, lo -> Yl)
void rotate_split(const Layout& L, const PatView<float>& Yh, const PatView<float>& Yl, int k, cudaStream_t s);
// As gather, FP32 result split into a tf32 pair (hi = tf32(y), lo = y - hi) for the tensor-core product.
// Yh and Yl share leading dimensions and offsets.
void gather_split(const Layout& L, const double* V, int k, const PatView<float>& Yh, const PatView<float>& Yl,
                  cudaStream_t s);
// As gather_split with a bf16 pair (hi = bf16(y), lo = bf16(y - hi)) for the bf16 tensor-core product.
void gather_split_bf16(const Layout& L, const double* V, int k, const PatView<__nv_bfloat16>& Yh,
                       const PatView<__nv_bfloat16>& Yl, cudaStream_t s);
// out[row][g] = beta * out[row][g] + sum over the row's slots: sign * Z(slot, g)
template <typename TI>
void scatter(const Layout& L, const PatView<TI>& Z, int k, double beta, double* out, cudaStream_t s);

// ---- multivector split (occurrence share of the residual) ------------------------------------------
// Z[row][g] = sum over the row's occurrences s with group(s) = g: r[row] / (number of occurrences in row)
void split(const Layout& L, const double* r, int k, double* Z, cudaStream_t s);
// The permutation multivector of Eq. 8: Z[row][g] = sum_e w[(row k + g) pw + e] r[src[...]] over the pw entries of
// row `row` of Pi^g (column g = Pi^g r; padding entries have w = 0).  g_only >= 0: only that column, written
// to Z as a single vector (Z[row]).
void perm_split(int n, int k, int pw, const int* src, const double* w, const double* r, double* Z, cudaStream_t s,
                int g_only = -1);

// ---- preconditioners of Eqs. 4-5 (weighted assembly) ----------------------------------------------
// Y(slot, g) = sum over the slot's links e: link_w[e] V[row_e][g] (link_w: sign x scaling, slot CSR order)
void gather_w(const Layout& L, const double* V, int k, const PatView<double>& Y, const double* link_w,
              cudaStream_t s);
// out[row][g] = sum over the row's slots: row_w[2 row + e] Z(slot_e, g)
void scatter_w(const Layout& L, const PatView<double>& Z, int k, const double* row_w, double* out, cudaStream_t s);
// the scaled occurrence split: Z[row][g] = sum over the row's slots in column g of row_d[2 row + e] z[row]
void split_w(const Layout& L, const double* z, int k, const double* row_d, double* Z, cudaStream_t s);

// ---- local products Z_p = S_p^+ Y_p ----------------------------------------------------------------
// FP64 (DFMA) and FP32 (FFMA) SIMT forms; one launch for every pattern.
struct LocalProblem {
  const void* S[MAXP];    // n_b x n_b row-major (symmetric)
  int n_b[MAXP];
  int n_rhs[MAXP];        // n_occ_p * k
  long long ld[MAXP];     // leading dimension of Y_p / Z_p (>= n_b)
  const void* Y[MAXP];
  void* Z[MAXP];
  int n_pat;
  // Factored form (FP64 only; X[p] non-null): S^+ Y = Lam^T (Lam Y) with Lam = L_S^{-1} the inverse of the
  // Schur-complement factor (lower triangular), stored transposed: X[c * ldx + r] = Lam(r, c).  Two triangular
  // products through the scratch W[p] (n_rhs x ld) instead of one product with a formed S^+; S is then unused.
  const double* X[MAXP];
  long long ldx[MAXP];
  double* W[MAXP];
};
void local_gemm_f64(const LocalProblem& P, cudaStream_t s);
void local_gemm_f32(const LocalProblem& P, cudaStream_t s);

// ---- sparse-column form of P^T F P S(r) (right-hand sides only where the split column touches) ----------
// Pattern p's pair right-hand sides: base[p] + (i - pair_off[p]) * ld[p] for global pair index i.
template <typename T>
struct PairView {
  T* base[MAXP];
  long long ld[MAXP];
  int pair_off[MAXP + 1];
};
void gather_pairs_f64(const Layout& L, const double* V, int k, const int* pair_occ, const int* pair_g, int n_pairs,
                      const PairView<double>& Y, cudaStream_t s);
void gather_pairs_f32(const Layout& L, const double* V, int k, const int* pair_occ, const int* pair_g, int n_pairs,
                      const PairView<float>& Y, cudaStream_t s);
void gather_pairs_split(const Layout& L, const double* V, int k, const int* pair_occ, const int* pair_g, int n_pairs,
                        const PairView<float>& Yh, const PairView<float>& Yl, cudaStream_t s);
// Yc[slot][g] = (M_s A)[j][g]: M_s is n_b x c_s column-major at M + moff[s] with column stride mld[pattern];
// its columns are the coarse rows mcol_row[mcol_ptr[s] .. mcol_ptr[s+1]) of A (n_G x k)
template <typename TM>
void coarse_response(const Layout& L, int k, const TM* M, const long long* moff, const int* mcol_ptr,
                     const int* mcol_row, const long long* mld, const double* A, double* Yc, cudaStream_t s);
// out[row][g] = sum over the row's slots: sign * (Z(pair_of[s][g], j) - Yc[slot][g])
template <typename TI>
void scatter_pairs(const Layout& L, const PairView<TI>& Z, int k, const int* pair_of, const double* Yc, double* out,
                   cudaStream_t s);

// ---- direction history layout ----------------------------------------------------------------------
// The stored directions W_h, Q_h (n rows, `cap` columns) are kept in blocks of hk columns, one block per block
// iteration: each block is n x hk, row-major and contiguous.  Writing a block is one contiguous stream and a
// row tile of a block is one contiguous piece (a row-major n x cap array would put every row of a large
// structure on its own page).  Column c of row `row` is at hist_col(c, n, hk) + row * hk.
__host__ __device__ __forceinline__ size_t hist_col(long long c, long long n, int hk) {
  return (size_t)(c / hk) * (size_t)n * (size_t)hk + (size_t)(c % hk);
}

// ---- persistent block iteration (latency-bound structures) -------------------------------------------
// One cooperative launch runs whole block iterations (split, Gram, projections, reorthogonalisation, F,
// eta, normalisation, update) as nine phases separated by grid barriers, and stops on the device when
// ||r||^2 <= target2 or no direction was kept.  Every wait is bounded (timeout_ns); an expired wait sets *err.
struct PersistArgs {
  Layout L;
  int n = 0, k = 0, ncta = 0;
  long long cap = 0;
  // local products: S_p (n_b x n_b row-major); Y and Z one buffer each, pattern p at ybase[p], column stride ld[p]
  const void* S[MAXP];
  long long ybase[MAXP];
  long long ld[MAXP];
  int n_rhs[MAXP];
  int tiles_m[MAXP];
  int tile_off[MAXP + 1];
  void* Ybuf;
  void* Zbuf;
  const int* pocc[MAXP];      // occurrences of every pattern, in local-product column order
  // per-row tables: multivector columns of the row's slots (-1 none), 1 / slot count, Z offsets of the slots
  const int* row_grp;
  const double* row_wt;
  const long long* row_z;
  const int* row_zld;
  // per row and slot: first coarse column of the slot's occurrence (-1 none), its kernel modes, and
  // sign * Nb[j][0..modes)
  const int* rowg_gofs;
  const int* rowg_kd;
  const double* rowg_coef;
  // iteration vectors and the direction history (element type of the history: TH)
  double* r;
  double* lam;
  double* Zr;
  double* Q;
  void* Wh;
  void* Qh;
  // Gram of the split residual
  const int* grp_ptr;
  const int* grp_row;
  const double* grp_w;
  int gs_chunks;
  double* gram_part;
  double* C;
  // coarse space
  const double* Ginv;
  double* Xc;
  double* Ac;
  // history update
  int tu_splits;
  void* tu_part;
  unsigned* tu_tickets;
  // eta and the normalisation
  double* eta_part;            // CTA partials, then (after ncta * k (k+1) values) group sums
  unsigned* eta_ticket;
  unsigned* eta_gticket;       // per group of 16 CTAs
  double trunc;
  double* T;
  double* alpha;
  int* n_kept;
  // update and control: state = [history columns, dropped, iterations]
  double* rr_part;
  int* state;
  int max_iters;
  double target2;
  unsigned* bar;
  int* err;
  unsigned long long timeout_ns;
  int missing;                 // CTAs a barrier waits for beyond ncta: 0 (a test sets 1 to make the waits expire)
  // optional (timing): nanoseconds spent by CTA 0 in each of the nine phases, barrier wait included, summed
  unsigned long long* clk;
};
void persist_iterations(const PersistArgs& A, bool fp64, cudaStream_t s);
int persist_ctas(bool fp64, int k);   // co-resident CTAs of the launch (0 if the kernel cannot be co-resident)

// ---- block Gram products and the F-normalised update (numerical-issues subsection) -----------------
// C (a x b, row-major) = A^T B, A n x a (ld lda), B n x b (ld ldb), FP64 accumulation over n in a fixed
// order (two passes: per-chunk partials, then an ordered sum).
template <typename TA, typename TB>
void gram(int n, int a, int b, const TA* A, int lda, const TB* B, int ldb, double* C, DBuf<double>& partial,
          cudaStream_t s);
// Reorthogonalisation coefficients C = Qh^T S(r) (a x k, row-major) of the split multivector S(r) without
// forming it: group g's rows (grp_ptr/grp_row) with weights grp_w = 1/(occurrences of the row).  FP64 sums
// (double-single for an FP32 history).  Qh: n rows in the block layout of width hk (hist_col).  The number of
// stored directions a is read from d_a on the device when d_a != NULL (at most a_max), so one captured launch
// serves every iteration.
// n_entries = grp_ptr[k]; wr: scratch of 2 n_entries doubles (the weighted split values, FP64 and FP32 hi + lo).
// grp_src (optional): the entry's value is w r[grp_src[e]] instead of w r[grp_row[e]] (a column of S(r) that
// takes r from other rows, as the permutation multivector [r, Pi r, ...] does).
template <typename TH>
void gram_split(int a_max, const int* d_a, int k, const TH* Qh, int n, int hk, const double* r, const int* grp_ptr,
                const int* grp_row, const double* grp_w, int n_entries, int max_group_rows, double* C,
                DBuf<double>& partial, DBuf<double>& wr, cudaStream_t s,
                const int* grp_src = nullptr);
// C[c] = sum_rows Qh[row][c] r[row] for c < a (history times one vector, FP64-class sums; Qh in the block
// layout of width hk); partial must hold at least a values (it is not grown: captured graphs share it)
template <typename TH>
void hist_dot(int n, int a, const TH* Qh, int hk, const double* r, double* C, DBuf<double>& partial,
              cudaStream_t s);
// W (n x k, FP64) += alpha * Wh (n x a, history type TH, block layout of width hk) * C (a x k, FP64),
// computed in TH arithmetic.
// scratch: split partials, tall_update_splits(n, a_max) * n * k values of TH; tickets: one counter per 64-row
// tile, zero between calls (both grown here; callers that capture graphs size them first).
int tall_update_splits(int n, int a_max);
// device scratch (in doubles) that tall_update needs for n rows, a_max columns, k outputs
size_t tall_update_scratch(int n, int a_max, int k, bool fp32);
// one-time kernel attribute set-up of the history update (large dynamic shared memory); call outside capture
void tall_update_init();
template <typename TH>
void tall_update(int n, int a_max, const int* d_a, int k, const TH* Wh, int hk, const double* C, double alpha,
                 double* W, DBuf<double>& scratch, DBuf<unsigned>& tickets, cudaStream_t s);
// Row-chunk partials of [eta | wr] = W^T [Q | r], a k x (k+1) block, FP64 sums: at most eta_chunks(n) of them
// (k = 4 with ds: one per SM).  With more than ETA_GROUPS chunks they are first added into ETA_GROUPS group sums
// (fixed order) stored after the chunks.  The return value is the offset, in blocks of k (k+1), of what
// normalise() must add, and *n_read their number (the chunks themselves, or the ETA_GROUPS group sums).
constexpr int ETA_GROUPS = 16;
int eta_chunks(int n);
// ds: the products and sums in double-single FP32 arithmetic (~2^-46 relative; the inner solves of the mixed
// forms), else FP64.
int eta_partials(int n, int k, const double* W, const double* Q, const double* r, DBuf<double>& partial,
                 cudaStream_t s, bool ds, int* n_read);
// C (m x k) = A (m x m) B (m x k), row-major, FP64, one warp per row (small coarse products).
// part (optional, small_gemm_parts(m) * m * k doubles): the inner dimension is split over that many CTA rows
// and the slices added in order (deterministic)
constexpr int SMALL_GEMM_MAX_PARTS = 8;
int small_gemm_parts(int m);
void small_gemm(int m, int k, const double* A, const double* B, double* C, cudaStream_t s, double* part = nullptr);
// Normalisation of eta = W^T P~ (k x k) so that T^T eta T = I on the kept directions: pivoted
// Cholesky eta = Pi M M^T Pi^T, stopping when the largest remaining pivot <= trunc * (largest diagonal);
// T = Pi M^{-T} on the kept columns (zero columns for dropped ones); alpha = T^T wr with wr = W^T r.
// Input: the row-chunk partials of [eta | wr] from eta_partials().  One CTA, k <= 64.
void normalise(int k, const double* ext_partial, int chunks, double trunc, double* T, double* alpha, int* n_kept,
               cudaStream_t s);
// Wn = W T, Qn = Q T (n x k each, written to history), lambda += Wn alpha, r -= Qn alpha, and
// rr_partial[block] = partial sums of r^2 after the update.
// History bookkeeping done by the last CTA of update(): stored directions += k (restart when the next block
// would not fit), dropped and iteration counters.  cols = NULL: nothing.
struct AdvanceArgs {
  int* cols = nullptr;
  int k = 0;
  long long cap = 0;
  const int* n_kept = nullptr;
  int* dropped = nullptr;
  int* iters = nullptr;
  unsigned* counter = nullptr;   // zero between launches
};
// Wn, Qn: the history (block layout of width k); d_off (device, may be NULL): the column where the new block
// starts (a multiple of k).
template <typename TH>
void update(int n, int k, const double* W, const double* Q, const double* T, const double* alpha, TH* Wn, TH* Qn,
            const int* d_off, double* lam, double* r, double* rr_partial, int rr_blocks,
            cudaStream_t s, const AdvanceArgs& adv = AdvanceArgs());
void sum_sq(int n, const double* x, double* out_partial, int blocks, cudaStream_t s);
void axpy_f64(int n, double a, const double* x, double* y, cudaStream_t s);

}  // namespace fetirp
