// C ABI of the library (include/fetirp.h): patterns, occurrences, the coarse problem, the block interface
// operator and the multivector FETI solver driver.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>

#include "../../include/fetirp.h"
#include "common.cuh"
#include "dense.cuh"
#include "ops.cuh"
#include "tc.cuh"

using namespace fetirp;

namespace fetirp {
thread_local unsigned long long g_launch_count = 0;
}

namespace {

// ------------------------------------------------------------------------------------------- small kernels
__global__ void k_csr_to_dense(int n, int npad, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                               const double* __restrict__ val, const int* __restrict__ newidx, double* A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  if (i >= n) { A[(size_t)i * npad + i] = 1.0; return; }
  const int ri = newidx[i];
  for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) A[(size_t)newidx[col[e]] * npad + ri] = val[e];
}

__global__ void k_set_diag(double* A, int ld, int from, int to, double v) {
  const int i = from + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < to) A[(size_t)i * ld + i] = v;
}

// N[z_m][m] = 1 for the zero-pivot dofs z_m (identity block of the kernel basis).
__global__ void k_set_entries(double* N, int npad, const int* zpiv, int kd) {
  const int m = threadIdx.x;
  if (m < kd) N[(size_t)m * npad + zpiv[m]] = 1.0;
}

// In-place inverse of a small SPD matrix (dimension <= 6) by Gauss-Jordan, one thread (pattern set-up).
__global__ void k_small_spd_inverse(double* C, int n) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a[6][12];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) a[i][j] = j < n ? C[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    const double inv = 1.0 / a[c][c];
    for (int j = 0; j < 2 * n; ++j) a[c][j] *= inv;
    for (int i = 0; i < n; ++i)
      if (i != c) {
        const double f = a[i][c];
        for (int j = 0; j < 2 * n; ++j) a[i][j] -= f * a[c][j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[i * n + j] = a[i][j + n];
}

__global__ void k_to_f32(size_t n, const double* __restrict__ x, float* __restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

// Boundary rows of K^+ y (pattern frame, new ordering) minus, or the full local solution back to the
// original dof order and the global frame: u_g[node][c] = sum_c' R[c][c'] u_l[node][c'].
__global__ void k_unpermute_rotate(int n_dofs, int dpn, int npad, const double* __restrict__ U,
                                   const int* __restrict__ newidx, const int* __restrict__ occ_list,
                                   const double* __restrict__ rot, const long long* __restrict__ uoff, int n_occ_p,
                                   double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_dofs * n_occ_p) return;
  const int q = (int)(idx / n_dofs), d = (int)(idx % n_dofs);
  const int s = occ_list[q];
  const int node = d / dpn, c = d % dpn;
  const double* R = rot + 9 * s;
  double v = 0.0;
  for (int c2 = 0; c2 < dpn; ++c2) {
    const double r = dpn > 1 ? R[3 * c + c2] : 1.0;
    if (r != 0.0) v = fma(r, U[(size_t)q * npad + newidx[node * dpn + c2]], v);
  }
  out[uoff[s] + d] = v;
}

// ------------------------------------------------------------------------------------------- host data
struct PatternData {
  int n_nodes = 0, dpn = 1, n = 0, n_b = 0, n_i = 0, npad = 0, nbpad = 0, expected = -1, kdim = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<int> bnd_nodes, bpos, newidx, oldidx, zpiv;
  TilePlan plan, planS;
  DBuf<int64_t> d_rowptr;
  DBuf<int> d_col, d_newidx, zp;
  DBuf<double> d_val, L, diag0, S64, N, Nb, Dinv, LS, XS, DinvS, Sdag, Nwork;
  DBuf<int> zpS, d_zpiv;
  std::vector<int> h_zp;
  int* h_zp_pinned = nullptr;
  std::vector<double> h_nrhs;
  const int* d_zpiv_list(int) const { return d_zpiv.p; }
  void upload_zpiv(cudaStream_t s) { if (!zpiv.empty()) d_zpiv.upload(zpiv, s); }
  ~PatternData() {
    if (h_zp_pinned) cudaFreeHost(h_zp_pinned);
  }
  DBuf<float> S32, S_hi, S_lo;   // FP32 S^dag and its tf32 pair (leading dimension lds)
  long long lds = 0;
  // s64_ok: S64, Sdag (kdim > 0), S32 and the tf32 pair hold the current factorisation's FP64 S^+, S^dag and
  // their FP32 roundings.  Large patterns (n_b >= TC_SDAG_MIN_NB) form those only on first use (ensure_splus64)
  // and cut the bf16 pair of S^dag at factorisation from a tensor-core Gram of the rows of (L_S^{-1} Pi)^T
  // (Ypair: tf32 pair, leading dimension lds); until then their FP64 local products go through the factor
  // (LocalProblem::X).
  std::atomic<bool> s64_ok{false};
  std::mutex s64_mu;
  DBuf<float> Ypair;
  DBuf<double> gemm_scratch;   // split partials of the skinny products with N_b (gemm_f64)
  DBuf<__nv_bfloat16> Sb_hi, Sb_lo;   // bf16 pair of S^dag (leading dimension ldsb, a multiple of 8)
  long long ldsb = 0;
  long long ld_y8 = 0;                // Y/Z leading dimension of the bf16 products (round_up(n_b, 8))
  long long ld_y = 0;          // Y/Z leading dimension (round_up(n_b, 4))
};

// How one context uses a pattern: its occurrences in the current structure and their loads and work vectors.
// The factor (PatternData) itself is read-only after set-up and may be shared by several contexts.
struct PatternUse {
  std::vector<int> occs;       // occurrences of this pattern (ids), q = position
  DBuf<int> d_occs;
  DBuf<double> F;              // npad x n_occ loads (pattern frame, new ordering)
  DBuf<double> U;              // npad x n_occ work (local solves)
  DBuf<double> Yf;             // npad x n_occ: L^{-1} F, the forward sweep of the loads (from d, for the recovery)
};

struct OccData {
  int pattern = 0;
  int R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};     // signed permutation folded into the links
  bool general = false;                       // a rotation of a vector field that is not a signed permutation
  double Rd[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}; // the rotation (row-major, global = R local) in both cases
  std::vector<double> f_local;  // pattern frame, original dof order
  std::vector<int> link_j, link_row;
  std::vector<int8_t> link_sign;
};


}  // namespace

// Sparse-column form of P^T F P S(r): right-hand sides (occurrence, group) only where the split column touches
// the occurrence, and the local coarse responses M_s = S^+ B(s)^T G_nbr(s).  Built once per structure and k.
struct SplitPlan {
  int k = -1;
  int n_pairs = 0;
  int pair_off[fetirp::MAXP + 1] = {};
  long long ybase[fetirp::MAXP] = {};
  long long ytotal = 0;
  DBuf<int> d_pair_occ, d_pair_g, d_pair_of;   // per pair; pair_of[s * k + g] = pattern-local index or -1
  DBuf<int> d_mcol_ptr, d_mcol_row;            // per occurrence: coarse rows of its columns of M
  DBuf<long long> d_moff, d_mld;               // offset of M_s; column stride per pattern
  DBuf<double> M64;                            // S^+ E (FP64 form)
  DBuf<float> M32;                             // S^dag E rounded to FP32 (low-precision forms)
  DBuf<double> Vs, Yc;                         // S(r) (n x k) and the coarse responses per slot (n_slots x k)
  DBuf<double> Y64, Z64;
  DBuf<float> Y32, Z32, Ylo32;
};

struct fetirp_ctx_s {
  fetirp_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  std::vector<std::shared_ptr<PatternData>> pats;   // shared with child contexts
  std::vector<PatternUse> use;                       // per pattern, this context's structure
  bool is_child = false;
  std::vector<OccData> occs;
  int k_user = 0;
  std::vector<int> groups_user;
  std::vector<int64_t> row_blocks;   // multiplier-row offsets of independent sub-structures (empty: one)
  // permutation multivector (Eq. 8): column g of the block is Pi^g z; Pi^g in ELL form (pw entries per row and
  // column, weight 0 = padding), built on the host when the permutation is set
  struct Perm {
    bool on = false, shortcut = false;
    int k = 0, pw = 1;
    int64_t n = 0;
    std::vector<int> src;       // [(row k + g) pw + e]
    std::vector<double> w;
    DBuf<int> d_src, d_grp_src;
    DBuf<double> d_w;
  } perm;

  // structure state (prepare)
  bool prepared = false;
  int64_t n_lambda = -1;
  int k = 1, n_G = 0, n_Gpad = 0;
  Layout L{};
  DBuf<int> d_slot_ptr, d_slot_row, d_row_slot, d_slot_occ, d_occ_obase, d_occ_pat, d_occ_q, d_occ_gofs,
      d_occ_group, d_pair_s, d_pair_t, d_grp_ptr, d_grp_row, d_ell_row, d_gen_occ;
  DBuf<double> d_rot, d_gen_R, d_slot_nb;   // rotation of every occurrence; general rotations and their slot kernels
  DBuf<int8_t> d_occ_general;               // per occurrence: 1 = a general rotation
  // the structure tables above are kept between builds while no call changed the structure (topo_valid) and the
  // patterns' sizes and kernel dimensions are those they were built for (topo_sig)
  bool topo_valid = false;
  int topo_nl = 0;
  std::vector<long long> topo_sig;
  DBuf<int8_t> d_ell_sign;
  DBuf<double> d_grp_w;
  // tables of the persistent iteration: multivector columns of the row's slots, 1 / slot count, offsets of the
  // row's slots in the local product buffers (for the current k)
  DBuf<int> d_row_grp, d_row_zld, d_rowg_gofs, d_rowg_kd;
  DBuf<double> d_row_wt, d_rowg_coef;
  // double-single projection of the inner solves: coefficients of G and (G^T G)^{-1} as FP32 pairs, and the
  // split coarse vectors
  DBuf<float> ds_coef, ds_ginv, ds_xa;
  bool ds_project = false;              // set while the inner iterations of a mixed form are enqueued
  DBuf<int> d_slot_code;        // per link: 2 row + e (its entry in the per-row tables)
  int n_grp_entries = 0;        // entries of the per-group row lists
  double n_gcoef = 0;           // coefficients of G by row (sum over rows and their slots of the mode count)
  DBuf<double> grp_wr;          // per entry: w r[row] in FP64 and as an FP32 pair (history Gram scratch)
  DBuf<double> d_gtv_part;      // G^T V per-chunk partial sums
  DBuf<double> sg_part;         // inner-dimension slices of (G^T G)^{-1} X
  DBuf<unsigned> d_gtv_ticket;  // G^T V last-CTA tickets (self-resetting)
  DBuf<long long> d_row_z;
  DBuf<unsigned> d_pbar;     // {barrier count, barrier generation, eta ticket, error flag, 64 group tickets}
  DBuf<double> pers_eta, prr;
  DBuf<unsigned long long> pers_clk;   // timing: per-phase nanoseconds of the persistent iteration
  bool inject_stall = false;           // test hook: the next persistent launch waits for a CTA that never comes
  std::vector<double> h_prr;
  std::vector<int> h_group;            // multivector column of every occurrence (current structure)
  SplitPlan sp;
  DBuf<int8_t> d_slot_sign, d_row_sign;
  DBuf<long long> d_uoff;
  int n_pairs = 0;
  int n_gen = 0;                       // occurrences with a general rotation (turned on the device)
  int max_group_rows = 0;
  std::vector<int> pofs;               // first coarse column of every pattern
  std::vector<long long> uoff;         // offset of every occurrence in u_out
  long long n_u = 0;
  DBuf<double> GtG, Ginv, e, d, lambda0, c;
  TilePlan planG;
  DBuf<int> zpG;
  // preconditioner of Eqs. 4-5 (FETIRP_PRECOND_*): the scaling of every link / row entry, the local operators
  // X_p of the patterns (pattern frame), the coarse matrix G^T tilde-F^{-1} G of the weighted projector and its
  // inverse, scratch blocks
  struct Precond {
    int kind = 0, scaling = 1;
    DBuf<double> link_w, row_w, row_d, grp_wd, GtMG, GtMGinv, T1, T2;
    DBuf<double> X[MAXP];
    TilePlan plan;
    DBuf<int> zp;
  } pc;

  // work
  DBuf<double> lam, r, t1, W, Q, Zr, Whist, Qhist, C, eta, wr, T, alpha, rr_part, Xc, Ac, gram_part, V1, V2;
  DBuf<float> Whist32, Qhist32;   // direction history of the low-precision inner solves
  DBuf<double> tu_part;           // split partials of the history update
  DBuf<unsigned> tu_tickets;      // per row tile: CTAs of the history update that have stored their partial
  DBuf<double> eta_part;          // row-chunk partials of eta and W^T r
  DBuf<int> n_kept;
  DBuf<double> Y64, Z64, W64;     // W64: scratch of the factored FP64 local product (large patterns)
  DBuf<float> Y32, Z32, Ylo32;
  DBuf<float> tc_part;            // K-split partials of the tensor-core product (small blocks only)
  DBuf<int> tc_error;
  DBuf<double> spd_A, spd_X, spd_diag;   // work of the coarse matrix inverse
  DBuf<double> gemm_scratch;             // split partials of the skinny coarse products (gemm_f64)
  long long hist_cap = 0;
  int rr_blocks = 0;
  fetirp_stats last{};

  // per-phase accounting (CUDA events when opt.timing = 1)
  struct PhaseRec { int phase; int e0, e1; };
  std::vector<cudaEvent_t> ev_pool;     // events recorded directly on the stream (reused by every call)
  size_t ev_used = 0;
  std::vector<cudaEvent_t> gev_pool;    // event nodes of the captured iteration graph (live with the graph)
  size_t gev_used = 0;
  std::vector<PhaseRec> recs;
  double phase_flops[FETIRP_NPHASE] = {}, phase_bytes[FETIRP_NPHASE] = {};
  long long phase_launches[FETIRP_NPHASE] = {};
  double graph_phase_ms[FETIRP_NPHASE] = {};
  bool phases_pending = false;          // a fetirp_factorize call's phases belong to the next solve
  int phase_override = -1;              // >= 0: every phase scope books into this phase (outer residual, recovery)
  // device-resident iteration state and the captured iteration graph
  DBuf<int> d_state;                    // [0] stored directions, [1] dropped directions, [2] iterations
  int* h_state = nullptr;               // pinned mirror for read-back
  double* h_rr = nullptr;               // pinned read-back of the residual partials
  bool owns_stream = false;
  bool capturing = false;
  bool in_iteration = false;            // enqueuing block iterations outside a capture (accounted per iteration)
  std::vector<cudaStream_t> fstreams;   // one per concurrently factorised pattern
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int prec = -1, k = 0, G = 0, th = 0, timing = 0;
    long long cap = 0;
    std::vector<PhaseRec> recs;
    long long launches[FETIRP_NPHASE] = {};
    long long total_launches = 0;
  } gc;
  long long pending_launches = 0;
  ~fetirp_ctx_s() {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : gev_pool) cudaEventDestroy(e);
    if (h_state) cudaFreeHost(h_state);
    if (h_rr) cudaFreeHost(h_rr);
    for (cudaStream_t st : fstreams) cudaStreamDestroy(st);
    if (fork_ev) cudaEventDestroy(fork_ev);
    for (cudaEvent_t e : join_ev) cudaEventDestroy(e);
    if (owns_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace {

// Books every phase scope opened while it lives into one phase (work that belongs to a step of its own, such as
// the FP64 residual of the outer refinement, whose F-apply would otherwise count as local product, gather and
// scatter).  The outermost override wins.
struct PhaseOverride {
  fetirp_ctx ctx;
  int saved;
  PhaseOverride(fetirp_ctx c, int ph) : ctx(c), saved(c->phase_override) {
    if (saved < 0) ctx->phase_override = ph;
  }
  ~PhaseOverride() { ctx->phase_override = saved; }
};

void set_err(fetirp_ctx ctx, const std::string& m) {
  if (ctx) ctx->err = m;
}

template <typename F>
fetirp_status guarded(fetirp_ctx ctx, F&& f) {
  if (!ctx) return FETIRP_EINVAL;
  try {
    ctx->err.clear();
    FETIRP_CUDA(cudaSetDevice(ctx->opt.device));
    DevAllocator a;   // the context's device allocator hooks, if any, for this thread while the call runs
    a.alloc = ctx->opt.alloc;
    a.free = ctx->opt.free;
    a.user = ctx->opt.alloc_user;
    a.stream = ctx->stream;
    AllocatorScope scope(a);
    return f();
  } catch (const Error& e) {
    set_err(ctx, e.what());
    return (fetirp_status)e.status;
  } catch (const std::bad_alloc&) {
    set_err(ctx, "host allocation failed");
    return FETIRP_ENOMEM;
  } catch (const std::exception& e) {
    set_err(ctx, e.what());
    return FETIRP_EINVAL;
  }
}

// Brackets one phase of work: counts its launches and algorithmic work, and with opt.timing records a pair
// of CUDA events on the context stream.
struct PhaseScope {
  fetirp_ctx ctx;
  int phase;
  unsigned long long l0;
  int e0 = -1;
  PhaseScope(fetirp_ctx c, int ph_, double flops, double bytes)
      : ctx(c), phase(c->phase_override >= 0 ? c->phase_override : ph_), l0(g_launch_count) {
    const int ph = phase;
    if (!ctx->capturing && !ctx->in_iteration) {   // block iterations are accounted per iteration instead
      ctx->phase_flops[ph] += flops;
      ctx->phase_bytes[ph] += bytes;
    }
    if (ctx->opt.timing && (ctx->opt.timing_mask == 0 || ((ctx->opt.timing_mask >> ph) & 1))) e0 = record();
  }
  int record() {
    std::vector<cudaEvent_t>& pool = ctx->capturing ? ctx->gev_pool : ctx->ev_pool;
    size_t& used = ctx->capturing ? ctx->gev_used : ctx->ev_used;
    if (used == pool.size()) {
      cudaEvent_t e;
      FETIRP_CUDA(cudaEventCreate(&e));
      pool.push_back(e);
    }
    const int id = (int)used++;
    if (ctx->capturing)   // an event node inside the captured graph, re-recorded at every replay
      FETIRP_CUDA(cudaEventRecordWithFlags(pool[id], ctx->stream, cudaEventRecordExternal));
    else
      FETIRP_CUDA(cudaEventRecord(pool[id], ctx->stream));
    return id;
  }
  ~PhaseScope() {
    const long long n = (long long)(g_launch_count - l0);
    if (ctx->capturing) ctx->gc.launches[phase] += n;
    else ctx->phase_launches[phase] += n;
    if (e0 >= 0) {
      try {
        const int e1 = record();
        (ctx->capturing ? ctx->gc.recs : ctx->recs).push_back({phase, e0, e1});
      } catch (...) {
      }
    }
  }
};

void reset_phases(fetirp_ctx ctx) {
  ctx->ev_used = 0;   // the captured graph's events are a pool of their own
  ctx->recs.clear();
  for (int i = 0; i < FETIRP_NPHASE; ++i) {
    ctx->phase_flops[i] = ctx->phase_bytes[i] = ctx->graph_phase_ms[i] = 0.0;
    ctx->phase_launches[i] = 0;
  }
}

// Call after the stream is synchronised.
void collect_phases(fetirp_ctx ctx, fetirp_stats& st) {
  for (int i = 0; i < FETIRP_NPHASE; ++i) {
    st.phase_ms[i] = ctx->graph_phase_ms[i];
    st.phase_flops[i] = ctx->phase_flops[i];
    st.phase_bytes[i] = ctx->phase_bytes[i];
    st.phase_launches[i] = ctx->phase_launches[i];
  }
  for (auto& r : ctx->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_pool[r.e0], ctx->ev_pool[r.e1]) == cudaSuccess) st.phase_ms[r.phase] += ms;
  }
}

// Arithmetic forms of the block operator (the solve's AUTO choice is not one)
bool operator_precision(int p) {
  return p == FETIRP_PREC_FP64 || p == FETIRP_PREC_FP32 || p == FETIRP_PREC_TF32X3 || p == FETIRP_PREC_BF16X3;
}

#define REQUIRE(cond, msg) \
  do {                     \
    if (!(cond)) throw Error(FETIRP_EINVAL, msg); \
  } while (0)

// ----------------------------------------------------------------------------------------- pattern set-up
// FP64 factorisation on the device: dense factor of K in interior-first/boundary-last order with zero-pivot
// detection (Sec. 2), kernel N, Schur complement pseudo-inverse S^+ = L_S^{-T} L_S^{-1} (stated after Eq. 3).
// Several patterns are factorised concurrently, each on its own stream forked from the context stream;
// work buffers stay resident so that a refactorisation allocates nothing.
void factor_stage_a(PatternData& P, double pivot_tol, cudaStream_t s) {
  const int n = P.n, npad = P.npad;
  P.L.ensure((size_t)npad * npad);
  FETIRP_CUDA(cudaMemsetAsync(P.L.p, 0, sizeof(double) * (size_t)npad * npad, s));
  k_csr_to_dense<<<ceil_div(npad, 128), 128, 0, s>>>(n, npad, P.d_rowptr.p, P.d_col.p, P.d_val.p, P.d_newidx.p,
                                                      P.L.p);
  FETIRP_LAUNCH_CHECK();
  P.diag0.ensure(npad);
  P.zp.ensure(npad);
  copy_diag(P.L.p, npad, P.diag0.p, s);
  chol_tiles(P.L.p, npad, P.plan, P.diag0.p, P.zp.p, pivot_tol, s);
  P.Dinv.ensure((size_t)npad * TILE);
  tile_inverses(P.L.p, npad, P.zp.p, P.Dinv.p, s);
  P.h_zp.resize(npad);
  if (!P.h_zp_pinned) FETIRP_CUDA(cudaMallocHost(&P.h_zp_pinned, sizeof(int) * npad));
  FETIRP_CUDA(cudaMemcpyAsync(P.h_zp_pinned, P.zp.p, sizeof(int) * npad, cudaMemcpyDeviceToHost, s));
}

void factor_check(PatternData& P) {
  P.zpiv.clear();
  for (int i = 0; i < P.npad; ++i)
    if (P.h_zp_pinned[i]) P.zpiv.push_back(i);
  for (int z : P.zpiv)
    if (z < P.n_i || z >= P.n)
      throw Error(FETIRP_ESINGULAR, "zero pivot outside the boundary block: interior stiffness is singular");
  P.kdim = (int)P.zpiv.size();
  if (P.kdim > 6)
    throw Error(FETIRP_ESINGULAR, "kernel dimension " + std::to_string(P.kdim) + " > 6 (disconnected pattern?)");
  if (P.expected >= 0 && P.kdim != P.expected)
    throw Error(FETIRP_ESINGULAR, "detected kernel dimension " + std::to_string(P.kdim) + " != expected " +
                                      std::to_string(P.expected));
}

// Patterns with at least this many boundary dofs form S^dag on the tensor cores (factor_stage_b)
constexpr int TC_SDAG_MIN_NB = 1024;
void form_splus64(PatternData& P, cudaStream_t s);
void form_sdag64(PatternData& P, cudaStream_t s);

void factor_stage_b(PatternData& P, int* tc_error, cudaStream_t s) {
  const int npad = P.npad, kd = P.kdim;
  // kernel: N_r = -K_rr^{-1} K_rz, N_z = I (right-hand side built on the host from the CSR)
  P.N.ensure((size_t)npad * std::max(kd, 1));
  if (kd > 0) {
    P.h_nrhs.assign((size_t)npad * kd, 0.0);
    for (int m = 0; m < kd; ++m) {
      const int old = P.oldidx[P.zpiv[m]];
      for (int64_t e = P.rowptr[old]; e < P.rowptr[old + 1]; ++e)
        P.h_nrhs[(size_t)m * npad + P.newidx[P.col[e]]] = -P.val[e];
      for (int z : P.zpiv) P.h_nrhs[(size_t)m * npad + z] = 0.0;
    }
    FETIRP_CUDA(cudaMemcpyAsync(P.N.p, P.h_nrhs.data(), sizeof(double) * P.h_nrhs.size(), cudaMemcpyHostToDevice, s));
    tri_solve(P.L.p, npad, P.plan, P.zp.p, P.N.p, npad, kd, false, s, P.Dinv.p);
    tri_solve(P.L.p, npad, P.plan, P.zp.p, P.N.p, npad, kd, true, s, P.Dinv.p);
    k_set_entries<<<1, 32, 0, s>>>(P.N.p, npad, P.d_zpiv_list(kd), kd);
    FETIRP_LAUNCH_CHECK();
  }
  P.Nb.ensure((size_t)P.n_b * std::max(kd, 1));
  for (int m = 0; m < kd; ++m)
    FETIRP_CUDA(cudaMemcpy2DAsync(P.Nb.p + m, sizeof(double) * kd, P.N.p + (size_t)m * npad + P.n_i,
                                  sizeof(double), sizeof(double), P.n_b, cudaMemcpyDeviceToDevice, s));
  // S^+ from the trailing block L_S
  const int nbp = P.nbpad;
  P.LS.ensure((size_t)nbp * nbp);
  P.XS.ensure((size_t)nbp * nbp);
  P.zpS.ensure(nbp);
  P.DinvS.ensure((size_t)nbp * TILE);
  FETIRP_CUDA(cudaMemsetAsync(P.LS.p, 0, sizeof(double) * (size_t)nbp * nbp, s));
  FETIRP_CUDA(cudaMemsetAsync(P.XS.p, 0, sizeof(double) * (size_t)nbp * nbp, s));
  FETIRP_CUDA(cudaMemsetAsync(P.zpS.p, 0, sizeof(int) * nbp, s));
  FETIRP_CUDA(cudaMemcpy2DAsync(P.LS.p, sizeof(double) * nbp, P.L.p + (size_t)P.n_i * npad + P.n_i,
                                sizeof(double) * npad, sizeof(double) * P.n_b, P.n_b, cudaMemcpyDeviceToDevice, s));
  FETIRP_CUDA(cudaMemcpyAsync(P.zpS.p, P.zp.p + P.n_i, sizeof(int) * P.n_b, cudaMemcpyDeviceToDevice, s));
  if (nbp > P.n_b) {
    k_set_diag<<<ceil_div(nbp - P.n_b, 128), 128, 0, s>>>(P.LS.p, nbp, P.n_b, nbp, 1.0);
    FETIRP_LAUNCH_CHECK();
  }
  k_set_diag<<<ceil_div(nbp, 128), 128, 0, s>>>(P.XS.p, nbp, 0, nbp, 1.0);
  FETIRP_LAUNCH_CHECK();
  tile_inverses(P.LS.p, nbp, P.zpS.p, P.DinvS.p, s);
  tri_solve(P.LS.p, nbp, P.planS, P.zpS.p, P.XS.p, nbp, nbp, false, s, P.DinvS.p, true);   // X = L_S^{-1}
  const int nb = P.n_b;
  P.lds = round_up(nb, 4);
  P.ldsb = round_up(nb, 8);
  P.ld_y8 = P.ldsb;
  // every operator buffer is sized here, so that forming them later (ensure_splus64) allocates nothing
  P.S64.ensure((size_t)nb * nb);
  if (kd > 0) P.Sdag.ensure((size_t)nb * nb);
  P.Nwork.ensure((size_t)nb * std::max(kd, 1) * 2 + 2 * kd * kd);
  P.gemm_scratch.ensure(std::max<size_t>({gemm_f64_scratch(nb, kd, nb), gemm_f64_scratch(kd, kd, nb), 1}));
  P.S32.ensure((size_t)nb * nb);
  P.S_hi.ensure((size_t)nb * P.lds);
  P.S_lo.ensure((size_t)nb * P.lds);
  P.Sb_hi.ensure((size_t)nb * P.ldsb);
  P.Sb_lo.ensure((size_t)nb * P.ldsb);
  if (nb < TC_SDAG_MIN_NB) {
    form_splus64(P, s);
    const double* Sdag = kd > 0 ? P.Sdag.p : P.S64.p;
    split_bf16(Sdag, nb, nb, nb, P.Sb_hi.p, P.Sb_lo.p, P.ldsb, s);
    P.s64_ok = true;
    return;
  }
  // Large patterns: the bf16 pair of S^dag = Pi S^+ Pi = Y^T Y, Y = Lam Pi, Lam = L_S^{-1},
  // Pi = I - N_b C^{-1} N_b^T, C = N_b^T N_b.  Y is formed in FP64 (Lam minus a rank-kd term, so the large kernel
  // components of S^+ never appear), rounded to tf32 pairs, and Y^T Y is one tensor-core product (tf32x3, FP32
  // accumulation), rounded to the bf16 pair: no FP64 S^+ (n_b^3 / 3 FP64 flops) is formed.  That S^dag is
  // accurate to ~1e-6 of sqrt(S^dag_ii S^dag_jj) (tf32 pair products, FP32 sums over n_b terms): the level of
  // the bf16 pair's own rounding (2^-17), not that of an FP32 rounding, so the FP32 and tf32 forms of S^dag
  // come from the FP64 S^+ (ensure_splus64).
  P.s64_ok = false;
  const double* A = nullptr;
  const double* E = nullptr;
  if (kd > 0) {
    double* Aw = P.Nwork.p;                  // Lam N_b      (nb x kd, row-major)
    double* Ew = Aw + (size_t)nb * kd;       // N_b C^{-1}   (nb x kd)
    double* Cm = Ew + (size_t)nb * kd;       // N_b^T N_b, then its inverse (kd x kd)
    gemm_f64(nb, kd, nb, 1.0, P.XS.p, 1, nbp, P.Nb.p, kd, 1, 0.0, Aw, kd, 1, s, P.gemm_scratch.p, P.gemm_scratch.n);
    gemm_f64(kd, kd, nb, 1.0, P.Nb.p, 1, kd, P.Nb.p, kd, 1, 0.0, Cm, kd, 1, s, P.gemm_scratch.p, P.gemm_scratch.n);
    k_small_spd_inverse<<<1, 32, 0, s>>>(Cm, kd);
    FETIRP_LAUNCH_CHECK();
    gemm_f64(nb, kd, kd, 1.0, P.Nb.p, kd, 1, Cm, kd, 1, 0.0, Ew, kd, 1, s);
    A = Aw;
    E = Ew;
  }
  P.Ypair.ensure((size_t)2 * nb * P.lds);
  float* Yh = P.Ypair.p;
  float* Yl = P.Ypair.p + (size_t)nb * P.lds;
  pinv_rows_tf32(P.XS.p, nbp, A, E, kd, nb, Yh, Yl, P.lds, s);
  TcProblem T;
  T.n_pat = 1;
  T.S_hi[0] = Yh; T.S_lo[0] = Yl; T.lds[0] = P.lds;
  T.Y_hi[0] = Yh; T.Y_lo[0] = Yl; T.ldy[0] = P.lds;
  T.Z[0] = P.S_hi.p;   // FP32 S^dag (leading dimension lds) in the tf32 buffer until ensure_splus64 fills it
  T.n_b[0] = nb; T.n_rhs[0] = nb;
  tc_gemm_tf32x3(T, tc_error, s);
  split_bf16(P.S_hi.p, nb, nb, P.lds, P.Sb_hi.p, P.Sb_lo.p, P.ldsb, s);
}

// S^+ = Lam^T Lam in FP64 (k_lauum, n_b^3 / 3 flops), with a kernel the Moore-Penrose inverse
// S^dag = Pi S^+ Pi, Pi = I - N_b (N_b^T N_b)^{-1} N_b^T (form_sdag64), and S^dag rounded to FP32 and to the
// tf32 pair.  S^+ from zero pivots carries large components along the kernel (a body held at a few dofs) that
// the projector P removes again, so rounding them for the low-precision products would survive that
// cancellation; S^dag has none.  P^T F P is the same for every generalized inverse (Sec. 2), so the inner
// operator is unchanged.
void form_splus64(PatternData& P, cudaStream_t s) {
  const int nb = P.n_b, nbp = P.nbpad, kd = P.kdim;
  const size_t nn = (size_t)nb * nb;
  lauum(P.XS.p, nbp, nbp, nb, P.S64.p, nb, s);   // S^+ = X^T X
  const double* Sdag = P.S64.p;
  if (kd > 0) {
    form_sdag64(P, s);
    Sdag = P.Sdag.p;
  }
  k_to_f32<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(nn, Sdag, P.S32.p);
  FETIRP_LAUNCH_CHECK();
  split_tf32(Sdag, nb, nb, nb, P.S_hi.p, P.S_lo.p, P.lds, s);
}

void form_sdag64(PatternData& P, cudaStream_t s) {
  const int nb = P.n_b, kd = P.kdim;
  double* A = P.Nwork.p;                  // S^+ N_b       (nb x kd, row-major)
  double* E = A + (size_t)nb * kd;        // N_b C^{-1}    (nb x kd)
  double* Cm = E + (size_t)nb * kd;       // N_b^T N_b, then its inverse (kd x kd)
  double* D = Cm + kd * kd;               // N_b^T S^+ N_b (kd x kd)
  gemm_f64(nb, kd, nb, 1.0, P.S64.p, nb, 1, P.Nb.p, kd, 1, 0.0, A, kd, 1, s, P.gemm_scratch.p, P.gemm_scratch.n);
  gemm_f64(kd, kd, nb, 1.0, P.Nb.p, 1, kd, P.Nb.p, kd, 1, 0.0, Cm, kd, 1, s, P.gemm_scratch.p, P.gemm_scratch.n);
  gemm_f64(kd, kd, nb, 1.0, P.Nb.p, 1, kd, A, kd, 1, 0.0, D, kd, 1, s, P.gemm_scratch.p, P.gemm_scratch.n);
  k_small_spd_inverse<<<1, 32, 0, s>>>(Cm, kd);
  FETIRP_LAUNCH_CHECK();
  gemm_f64(nb, kd, kd, 1.0, P.Nb.p, kd, 1, Cm, kd, 1, 0.0, E, kd, 1, s);
  FETIRP_CUDA(cudaMemcpyAsync(P.Sdag.p, P.S64.p, sizeof(double) * (size_t)nb * nb, cudaMemcpyDeviceToDevice, s));
  gemm_f64(nb, nb, kd, -1.0, E, kd, 1, A, 1, kd, 1.0, P.Sdag.p, nb, 1, s);    // - E A^T
  gemm_f64(nb, nb, kd, -1.0, A, kd, 1, E, 1, kd, 1.0, P.Sdag.p, nb, 1, s);    // - A E^T
  gemm_f64(nb, kd, kd, 1.0, E, kd, 1, D, kd, 1, 0.0, A, kd, 1, s);            // A <- E D
  gemm_f64(nb, nb, kd, 1.0, A, kd, 1, E, 1, kd, 1.0, P.Sdag.p, nb, 1, s);     // + E D E^T
}

// The FP64 S^+ (S^dag) of a large pattern and the FP32 and tf32 forms of S^dag, formed on first use after a
// factorisation by the callers that need them: products in FP64 as a matrix (FP64 solves, the persistent FP64
// iteration, the sparse-column plan, fetirp_get_pattern) and every FP32 or tf32x3 product.  Allocates nothing
// (factor_stage_b sized the buffers); blocks until formed; patterns are shared by child contexts, hence the
// lock.
void ensure_splus64(PatternData& P, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(P.s64_mu);
  if (P.s64_ok) return;
  form_splus64(P, s);
  FETIRP_CUDA(cudaStreamSynchronize(s));
  P.s64_ok = true;
}

// The operators that products in precision prec read: everything but the bf16 pair needs ensure_splus64.
// Their formation counts as set-up (the factorisation phase).
void ensure_operators(fetirp_ctx ctx, int prec) {
  if (prec == FETIRP_PREC_BF16X3) return;
  const bool by_use = ctx->use.size() == ctx->pats.size();   // the patterns of the current structure only
  std::vector<PatternData*> todo;
  double flops = 0.0;
  for (size_t p = 0; p < ctx->pats.size(); ++p) {
    PatternData& P = *ctx->pats[p];
    if ((by_use && ctx->use[p].occs.empty()) || P.s64_ok) continue;
    todo.push_back(&P);
    flops += 2.0 * ((double)P.n_b * P.n_b * P.n_b / 6.0);
  }
  if (todo.empty()) return;
  PhaseScope ph(ctx, FETIRP_PHASE_FACTOR, flops, 0.0);
  for (PatternData* P : todo) ensure_splus64(*P, ctx->stream);
}

// Per-pattern work on concurrent streams: fork_patterns(ctx, n) makes n streams wait for the work enqueued so far
// on the context stream; join_patterns(ctx, n) makes the context stream wait for all of them.
void fork_patterns(fetirp_ctx ctx, size_t np) {
  while (ctx->fstreams.size() < np) {
    cudaStream_t st;
    FETIRP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ctx->fstreams.push_back(st);
  }
  if (!ctx->fork_ev) FETIRP_CUDA(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
  FETIRP_CUDA(cudaEventRecord(ctx->fork_ev, ctx->stream));
  for (size_t i = 0; i < np; ++i) FETIRP_CUDA(cudaStreamWaitEvent(ctx->fstreams[i], ctx->fork_ev, 0));
}
void join_patterns(fetirp_ctx ctx, size_t np) {
  for (size_t i = 0; i < np; ++i) {
    if (ctx->join_ev.size() <= i) {
      cudaEvent_t e;
      FETIRP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      ctx->join_ev.push_back(e);
    }
    FETIRP_CUDA(cudaEventRecord(ctx->join_ev[i], ctx->fstreams[i]));
    FETIRP_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->join_ev[i], 0));
  }
}

// FP64 flops of one pattern's set-up, counted from its tile plans (64^3 FMAs per tile product): the tile
// Cholesky (diagonal factorisations, panel solves, trailing updates of every tile pair with fill), the kernel
// solves, L_S^{-1} (a forward solve on the identity with the zero upper tiles skipped) and S^+ = L_S^{-T} L_S^{-1}
// (lower triangle).  The Moore-Penrose correction (rank 2 kd) and the splits are not counted.
double factor_flops(const PatternData& P) {
  const double t3 = (double)TILE * TILE * TILE;
  const double nt = P.plan.nt;
  double f = 2.0 * t3 * (double)P.plan.pairs.size()          // trailing updates
             + (2.0 / 3.0) * t3 * nt                          // diagonal tiles
             + t3 * (double)P.plan.col_rows.size();           // panel solves
  f += 2.0 * 2.0 * (double)P.kdim * TILE * TILE * (double)(P.plan.col_rows.size() + P.plan.nt);   // kernel N
  const double nb = P.n_b;
  f += 2.0 * (nb * nb * nb / 6.0);                             // L_S^{-1}
  if (P.n_b < TC_SDAG_MIN_NB) f += 2.0 * (nb * nb * nb / 6.0);   // S^+ = L_S^{-T} L_S^{-1} (large: tensor cores)
  return f;
}

void check_tc_error(fetirp_ctx ctx);

void factorize_patterns(fetirp_ctx ctx, const std::vector<PatternData*>& pats) {
  double flops = 0.0;
  for (const PatternData* P : pats) flops += factor_flops(*P);
  PhaseScope ph(ctx, FETIRP_PHASE_FACTOR, flops, 0.0);
  const size_t np = pats.size();
  fork_patterns(ctx, np);
  for (size_t i = 0; i < np; ++i) factor_stage_a(*pats[i], ctx->opt.pivot_tol, ctx->fstreams[i]);
  for (size_t i = 0; i < np; ++i) FETIRP_CUDA(cudaStreamSynchronize(ctx->fstreams[i]));
  for (size_t i = 0; i < np; ++i) {
    factor_check(*pats[i]);
    pats[i]->upload_zpiv(ctx->fstreams[i]);
  }
  if (!ctx->tc_error.p) {   // zeroed before the pattern streams run (they were forked earlier)
    ctx->tc_error.alloc(1);
    ctx->tc_error.zero(ctx->stream);
    FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  for (size_t i = 0; i < np; ++i) factor_stage_b(*pats[i], ctx->tc_error.p, ctx->fstreams[i]);
  join_patterns(ctx, np);
  FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
  check_tc_error(ctx);   // the tensor-core S^dag of large patterns
}

// Dense SPD inverse in FP64 (coarse matrix G^T G): tile Cholesky, X = L^{-1}, A^{-1} = X^T X.
void spd_inverse(fetirp_ctx ctx, const double* A_rowmajor, int n, int npad, TilePlan& plan, DBuf<int>& zp,
                 double* out_rowmajor) {
  cudaStream_t s = ctx->stream;
  ctx->spd_A.ensure((size_t)npad * npad);
  ctx->spd_X.ensure((size_t)npad * npad);
  ctx->spd_diag.ensure(npad);
  DBuf<double>&A = ctx->spd_A, &X = ctx->spd_X, &diag = ctx->spd_diag;
  FETIRP_CUDA(cudaMemsetAsync(A.p, 0, sizeof(double) * (size_t)npad * npad, s));
  FETIRP_CUDA(cudaMemsetAsync(X.p, 0, sizeof(double) * (size_t)npad * npad, s));
  FETIRP_CUDA(cudaMemcpy2DAsync(A.p, sizeof(double) * npad, A_rowmajor, sizeof(double) * n, sizeof(double) * n, n,
                                cudaMemcpyDeviceToDevice, s));   // symmetric: row-major == column-major
  if (npad > n) {
    k_set_diag<<<ceil_div(npad - n, 128), 128, 0, s>>>(A.p, npad, n, npad, 1.0);
    FETIRP_LAUNCH_CHECK();
  }
  zp.ensure(npad);
  copy_diag(A.p, npad, diag.p, s);
  chol_tiles(A.p, npad, plan, diag.p, zp.p, 1e-13, s);
  std::vector<int> h(npad);
  FETIRP_CUDA(cudaMemcpyAsync(h.data(), zp.p, sizeof(int) * npad, cudaMemcpyDeviceToHost, s));
  FETIRP_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i)
    if (h[i]) throw Error(FETIRP_ESINGULAR, "coarse matrix G^T G is singular (an occurrence is not constrained)");
  k_set_diag<<<ceil_div(npad, 128), 128, 0, s>>>(X.p, npad, 0, npad, 1.0);
  FETIRP_LAUNCH_CHECK();
  tri_solve(A.p, npad, plan, zp.p, X.p, npad, npad, false, s, nullptr, true);   // X = L^{-1}
  lauum(X.p, npad, npad, n, out_rowmajor, n, s);                               // A^{-1} = X^T X
  FETIRP_CUDA(cudaStreamSynchronize(s));
}

TilePlan dense_plan(int nt) {
  TilePlan p;
  std::vector<uint8_t> nz((size_t)nt * nt, 0);
  for (int I = 0; I < nt; ++I)
    for (int J = 0; J <= I; ++J) nz[(size_t)I * nt + J] = 1;
  p.build(nt, nz);
  return p;
}

// ----------------------------------------------------------------------------------------- structure
// A call that changed the structure (occurrences, groups, permutation, preconditioner, row blocks, patterns)
void invalidate(fetirp_ctx ctx) {
  ctx->prepared = false;
  ctx->topo_valid = false;
}
void check_periodic(fetirp_ctx ctx);
void precond_setup(fetirp_ctx ctx);

// Local-product buffers for a block of k columns in every precision (allocated before any graph capture).
// Does some pattern of the context apply S^+ in FP64 through its factor (no formed S^+)?
bool factored_f64(fetirp_ctx ctx) {
  for (auto& P : ctx->pats)
    if (!P->s64_ok) return true;
  return false;
}

// The factored FP64 local product of pattern P, if it has no formed S^+: LocalProblem fields X, ldx, W.
void set_factored(LocalProblem& LP, int p, const PatternData& P, double* W) {
  if (P.s64_ok) return;
  LP.X[p] = P.XS.p;
  LP.ldx[p] = P.nbpad;
  LP.W[p] = W;
}

void ensure_apply_buffers(fetirp_ctx ctx, int k) {
  long long total = 0, total8 = 0;
  for (size_t p = 0; p < ctx->pats.size(); ++p) {
    total += (long long)ctx->use[p].occs.size() * k * ctx->pats[p]->ld_y;
    total8 += (long long)ctx->use[p].occs.size() * k * ctx->pats[p]->ld_y8;
  }
  total = std::max(total, total8);   // the bf16 products use the FP32 buffers with leading dimension ld_y8
  ctx->Y64.ensure(total); ctx->Z64.ensure(total);
  if (factored_f64(ctx)) ctx->W64.ensure(total);
  ctx->Y32.ensure(total); ctx->Z32.ensure(total); ctx->Ylo32.ensure(total);
  TcProblem T;   // would the tensor-core product split its reduction dimension?
  T.n_pat = (int)ctx->pats.size();
  for (int p = 0; p < T.n_pat; ++p) {
    T.n_b[p] = ctx->pats[p]->n_b;
    T.n_rhs[p] = (int)ctx->use[p].occs.size() * k;
  }
  const int sp = tc_ksplits(T);
  if (sp > 1) ctx->tc_part.ensure((size_t)sp * total);
}

void build_structure(fetirp_ctx ctx, int64_t n_lambda, const double* c_host, const double* c_dev) {
  cudaStream_t s = ctx->stream;
  const int n_occ = (int)ctx->occs.size();
  if (n_occ == 0) throw Error(FETIRP_ESTATE, "no occurrence has been added");
  REQUIRE(n_lambda > 0 && n_lambda < (1LL << 31), "n_lambda out of range");
  const int nl = (int)n_lambda;
  REQUIRE(ctx->row_blocks.empty() || ctx->row_blocks.back() == n_lambda, "row blocks do not cover n_lambda rows");
  const int n_pat = (int)ctx->pats.size();
  if (n_pat > MAXP) throw Error(FETIRP_EINVAL, "more than 16 patterns in one structure");
  // structure tables (host work and uploads): rebuilt only when the structure or the patterns' shapes changed
  std::vector<long long> sig;
  for (auto& P : ctx->pats) {
    sig.push_back(P->n); sig.push_back(P->n_b); sig.push_back(P->kdim); sig.push_back(P->npad);
    sig.push_back(P->ld_y); sig.push_back(P->dpn);
  }
  if (!(ctx->topo_valid && ctx->topo_nl == nl && ctx->topo_sig == sig)) {
    ctx->topo_valid = false;
    // occurrence tables
    std::vector<int> obase(n_occ + 1, 0), occ_pat(n_occ), occ_q(n_occ), occ_gofs(n_occ), group(n_occ);
    ctx->use.resize(n_pat);
    for (auto& u : ctx->use) u.occs.clear();
    for (int o = 0; o < n_occ; ++o) {
      PatternData& P = *ctx->pats[ctx->occs[o].pattern];
      PatternUse& Us = ctx->use[ctx->occs[o].pattern];
      occ_pat[o] = ctx->occs[o].pattern;
      occ_q[o] = (int)Us.occs.size();
      Us.occs.push_back(o);
      obase[o + 1] = obase[o] + P.n_b;
    }
    ctx->pofs.assign(n_pat + 1, 0);
    for (int p = 0; p < n_pat; ++p) ctx->pofs[p + 1] = ctx->pofs[p] + ctx->pats[p]->kdim * (int)ctx->use[p].occs.size();
    for (int o = 0; o < n_occ; ++o) occ_gofs[o] = ctx->pofs[occ_pat[o]] + occ_q[o] * ctx->pats[occ_pat[o]]->kdim;
    ctx->n_G = ctx->pofs[n_pat];
    // multivector groups
    int k;
    if (ctx->perm.on) {   // the block is [z, Pi z, ...]; occurrence groups only serve the tables below
      if (ctx->perm.n != n_lambda) throw Error(FETIRP_EINVAL, "the permutation's size differs from n_lambda");
      k = ctx->perm.k;
      for (int o = 0; o < n_occ; ++o) group[o] = (int)((long long)o * std::min(k, n_occ) / n_occ);
    } else if (ctx->k_user > 0) {
      k = ctx->k_user;
      group = ctx->groups_user;
    } else {
      k = std::max(1, std::min(ctx->opt.block_k, n_occ));
      for (int o = 0; o < n_occ; ++o) group[o] = (int)((long long)o * k / n_occ);
    }
    REQUIRE((int)group.size() == n_occ, "groups do not match the number of occurrences");
    if (k > 64) throw Error(FETIRP_EINVAL, "block width k > 64 is not supported");
    ctx->k = k;
    ctx->h_group = group;
    // links -> gather CSR by slot, scatter lists by row
    const int n_slots = obase[n_occ];
    std::vector<int> cnt_slot(n_slots, 0);
    std::vector<int> row_cnt(nl, 0), row_slot(2 * (size_t)nl, 0);
    std::vector<int8_t> row_sign(2 * (size_t)nl, 0);
    for (int o = 0; o < n_occ; ++o) {
      const OccData& O = ctx->occs[o];
      for (size_t i = 0; i < O.link_row.size(); ++i) {
        const int row = O.link_row[i];
        if (row >= nl) throw Error(FETIRP_EINVAL, "lambda_row >= n_lambda");
        const int slot = obase[o] + O.link_j[i];
        cnt_slot[slot]++;
        if (row_cnt[row] >= 2) throw Error(FETIRP_EINVAL, "multiplier row " + std::to_string(row) + " has more than two entries");
        row_slot[2 * (size_t)row + row_cnt[row]] = slot;
        row_sign[2 * (size_t)row + row_cnt[row]] = O.link_sign[i];
        row_cnt[row]++;
      }
    }
    for (int r = 0; r < nl; ++r) {
      if (row_cnt[r] == 0) throw Error(FETIRP_EINVAL, "multiplier row " + std::to_string(r) + " has no entry");
      if (row_cnt[r] == 2 && row_slot[2 * (size_t)r] > row_slot[2 * (size_t)r + 1]) {
        std::swap(row_slot[2 * (size_t)r], row_slot[2 * (size_t)r + 1]);
        std::swap(row_sign[2 * (size_t)r], row_sign[2 * (size_t)r + 1]);
      }
    }
    std::vector<int> slot_ptr(n_slots + 1, 0);
    for (int i = 0; i < n_slots; ++i) slot_ptr[i + 1] = slot_ptr[i] + cnt_slot[i];
    std::vector<int> slot_row(slot_ptr[n_slots]), fill(slot_ptr.begin(), slot_ptr.end() - 1);
    std::vector<int8_t> slot_sign(slot_ptr[n_slots]);
    std::vector<int> slot_code(slot_ptr[n_slots]);   // 2 row + e: the link's entry in the per-row tables
    for (int r = 0; r < nl; ++r)   // rows in increasing order inside every slot
      for (int e = 0; e < row_cnt[r]; ++e) {
        const int slot = row_slot[2 * (size_t)r + e];
        slot_row[fill[slot]] = r;
        slot_sign[fill[slot]] = row_sign[2 * (size_t)r + e];
        slot_code[fill[slot]] = 2 * r + e;
        fill[slot]++;
      }
    int max_links = 1;   // links of the largest occurrence
    for (int o = 0; o < n_occ; ++o) max_links = std::max(max_links, slot_ptr[obase[o + 1]] - slot_ptr[obase[o]]);
    std::vector<int> slot_occ(n_slots);
    for (int o = 0; o < n_occ; ++o)
      for (int j = obase[o]; j < obase[o + 1]; ++j) slot_occ[j] = o;
    int ell_w = 1;
    for (int i = 0; i < n_slots; ++i) ell_w = std::max(ell_w, slot_ptr[i + 1] - slot_ptr[i]);
    std::vector<int> ell_row((size_t)n_slots * ell_w, 0);
    std::vector<int8_t> ell_sign((size_t)n_slots * ell_w, 0);
    for (int i = 0; i < n_slots; ++i)
      for (int e = slot_ptr[i]; e < slot_ptr[i + 1]; ++e) {
        ell_row[(size_t)i * ell_w + (e - slot_ptr[i])] = slot_row[e];
        ell_sign[(size_t)i * ell_w + (e - slot_ptr[i])] = slot_sign[e];
      }
    // rows of every multivector group with the multiplicity weight 1/(occurrences in the row): the split
    // S(r)[row][g] = sum over the row's occurrences in group g of r[row] / count
    std::vector<std::vector<std::pair<int, double>>> grp(k);
    for (int r = 0; r < nl; ++r) {
      const double w = 1.0 / row_cnt[r];
      int g1 = group[slot_occ[row_slot[2 * (size_t)r]]];
      if (row_cnt[r] == 2) {
        int g2 = group[slot_occ[row_slot[2 * (size_t)r + 1]]];
        if (g1 == g2) { grp[g1].push_back({r, 2.0 * w}); continue; }
        grp[g2].push_back({r, w});
      }
      grp[g1].push_back({r, w});
    }
    std::vector<int> grp_ptr(k + 1, 0), grp_row, grp_src;
    std::vector<double> grp_w;
    if (ctx->perm.on) {   // column g of S(r) = Pi^g r: entries (row, source row, weight) of Pi^g, row by row
      const int pw = ctx->perm.pw;
      for (int g = 0; g < k; ++g) {
        for (int r = 0; r < nl; ++r)
          for (int e = 0; e < pw; ++e) {
            const size_t i = ((size_t)r * k + g) * pw + e;
            if (ctx->perm.w[i] == 0.0) continue;
            grp_row.push_back(r);
            grp_src.push_back(ctx->perm.src[i]);
            grp_w.push_back(ctx->perm.w[i]);
          }
        grp_ptr[g + 1] = (int)grp_row.size();
      }
    } else {
      for (int g = 0; g < k; ++g) {
        std::sort(grp[g].begin(), grp[g].end());
        for (auto& e : grp[g]) { grp_row.push_back(e.first); grp_w.push_back(e.second); }
        grp_ptr[g + 1] = (int)grp_row.size();
      }
    }
    // neighbour pairs (s, t) sharing a row, plus (s, s)
    std::vector<std::vector<int>> nbr(n_occ);
    for (int o = 0; o < n_occ; ++o) nbr[o].push_back(o);
    for (int r = 0; r < nl; ++r)
      if (row_cnt[r] == 2) {
        const int a = slot_occ[row_slot[2 * (size_t)r]], b = slot_occ[row_slot[2 * (size_t)r + 1]];
        nbr[a].push_back(b);
        nbr[b].push_back(a);
      }
    std::vector<int> pair_s, pair_t;
    for (int o = 0; o < n_occ; ++o) {
      std::sort(nbr[o].begin(), nbr[o].end());
      nbr[o].erase(std::unique(nbr[o].begin(), nbr[o].end()), nbr[o].end());
      for (int t : nbr[o]) { pair_s.push_back(o); pair_t.push_back(t); }
    }
    // upload
    ctx->d_slot_ptr.upload(slot_ptr, s);
    ctx->d_slot_row.upload(slot_row, s);
    ctx->d_slot_sign.upload(slot_sign, s);
    ctx->d_slot_code.upload(slot_code, s);
    ctx->d_row_slot.upload(row_slot, s);
    ctx->d_row_sign.upload(row_sign, s);
    ctx->d_slot_occ.upload(slot_occ, s);
    ctx->d_occ_obase.upload(obase, s);
    ctx->d_occ_pat.upload(occ_pat, s);
    ctx->d_occ_q.upload(occ_q, s);
    ctx->d_occ_gofs.upload(occ_gofs, s);
    ctx->d_occ_group.upload(group, s);
    ctx->max_group_rows = 0;
    for (int g = 0; g < k; ++g) ctx->max_group_rows = std::max(ctx->max_group_rows, grp_ptr[g + 1] - grp_ptr[g]);
    ctx->n_grp_entries = grp_ptr[k];
    ctx->grp_wr.ensure(2 * (size_t)std::max(ctx->n_grp_entries, 1));
    ctx->d_ell_row.upload(ell_row, s);
    ctx->d_ell_sign.upload(ell_sign, s);
    ctx->d_grp_ptr.upload(grp_ptr, s);
    ctx->d_grp_row.upload(grp_row, s);
    ctx->d_grp_w.upload(grp_w, s);
    if (ctx->pc.kind != 0) {
      // scaling Delta(s) of every row entry (Eqs. 4-5, sum over the row's entries = 1): multiplicity 1 / count, or
      // stiffness: the other side's share of the diagonal stiffness at the link's dof (global frame); 1 on
      // Dirichlet rows
      auto kdiag = [&](int slot) -> double {   // diagonal of R-hat K R-hat^T at the slot's global dof
        const int o = slot_occ[slot];
        const PatternData& P = *ctx->pats[occ_pat[o]];
        const int j = slot - obase[o];
        const int b = j / P.dpn, c = j % P.dpn, node = P.bnd_nodes[b];
        auto entry = [&](int i, int jj) {
          for (int64_t e = P.rowptr[i]; e < P.rowptr[i + 1]; ++e)
            if (P.col[e] == jj) return P.val[e];
          return 0.0;
        };
        if (!ctx->occs[o].general) return entry(node * P.dpn + c, node * P.dpn + c);
        const double* R = ctx->occs[o].Rd;
        double v = 0.0;
        for (int c2 = 0; c2 < P.dpn; ++c2)
          for (int c3 = 0; c3 < P.dpn; ++c3)
            v += R[3 * c + c2] * R[3 * c + c3] * entry(node * P.dpn + c2, node * P.dpn + c3);
        return v;
      };
      std::vector<double> delta(2 * (size_t)nl, 0.0), row_w(2 * (size_t)nl, 0.0);
      for (int r = 0; r < nl; ++r) {
        if (row_cnt[r] == 1) { delta[2 * (size_t)r] = 1.0; continue; }
        if (ctx->pc.scaling == 0) { delta[2 * (size_t)r] = delta[2 * (size_t)r + 1] = 0.5; continue; }
        const double k0 = kdiag(row_slot[2 * (size_t)r]), k1 = kdiag(row_slot[2 * (size_t)r + 1]);
        if (!(k0 > 0.0 && k1 > 0.0)) throw Error(FETIRP_EINVAL, "stiffness scaling needs a positive diagonal");
        delta[2 * (size_t)r] = k1 / (k0 + k1);
        delta[2 * (size_t)r + 1] = k0 / (k0 + k1);
      }
      for (size_t i = 0; i < delta.size(); ++i) row_w[i] = row_sign[i] * delta[i];
      std::vector<double> link_w(slot_row.size());
      for (size_t e = 0; e < slot_row.size(); ++e) link_w[e] = slot_sign[e] * delta[(size_t)slot_code[e]];
      // group lists with the Delta weights (same rows as grp_row): the split of the preconditioned residual
      std::vector<double> grp_wd(grp_row.size(), 0.0);
      if (!ctx->perm.on)
        for (int g = 0; g < k; ++g)
          for (int i = grp_ptr[g]; i < grp_ptr[g + 1]; ++i) {
            const int r = grp_row[i];
            for (int e = 0; e < row_cnt[r]; ++e)
              if (group[slot_occ[row_slot[2 * (size_t)r + e]]] == g) grp_wd[i] += delta[2 * (size_t)r + e];
          }
      else
        grp_wd = grp_w;
      ctx->pc.row_d.upload(delta, s);
      ctx->pc.row_w.upload(row_w, s);
      ctx->pc.link_w.upload(link_w, s);
      ctx->pc.grp_wd.upload(grp_wd, s);
      FETIRP_CUDA(cudaStreamSynchronize(s));
    }
    if (ctx->perm.on) {
      ctx->perm.d_grp_src.upload(grp_src, s);
      ctx->perm.d_src.upload(ctx->perm.src, s);
      ctx->perm.d_w.upload(ctx->perm.w, s);
    }
    {
      std::vector<long long> pbase(n_pat + 1, 0);
      for (int p = 0; p < n_pat; ++p)
        pbase[p + 1] = pbase[p] + (long long)ctx->use[p].occs.size() * k * ctx->pats[p]->ld_y;
      std::vector<int> row_grp(2 * (size_t)nl, -1), row_zld(2 * (size_t)nl, 0);
      std::vector<double> row_wt(nl);
      std::vector<long long> row_z(2 * (size_t)nl, 0);
      for (int r = 0; r < nl; ++r) {
        row_wt[r] = 1.0 / row_cnt[r];
        for (int e = 0; e < row_cnt[r]; ++e) {
          const int slot = row_slot[2 * (size_t)r + e];
          const int o = slot_occ[slot];
          const int p = occ_pat[o];
          const long long ld = ctx->pats[p]->ld_y;
          row_grp[2 * (size_t)r + e] = group[o];
          row_z[2 * (size_t)r + e] = pbase[p] + (long long)occ_q[o] * k * ld + (slot - obase[o]);
          row_zld[2 * (size_t)r + e] = (int)ld;
        }
      }
      ctx->d_row_grp.upload(row_grp, s);
      ctx->d_row_zld.upload(row_zld, s);
      ctx->d_row_wt.upload(row_wt, s);
      ctx->d_row_z.upload(row_z, s);
      // G restricted to the row: coarse column of each slot's occurrence and its kernel dimension; the values
      // sign * N_b[j][m] follow every factorisation and are formed on the device (row_coefs, below)
      std::vector<int> rowg_gofs(2 * (size_t)nl, -1), rowg_kd(2 * (size_t)nl, 0);
      for (int r = 0; r < nl; ++r)
        for (int e = 0; e < row_cnt[r]; ++e) {
          const int o = slot_occ[row_slot[2 * (size_t)r + e]];
          const PatternData& P = *ctx->pats[occ_pat[o]];
          if (P.kdim > 6 || P.kdim == 0) continue;   // such structures do not use the persistent iteration
          rowg_gofs[2 * (size_t)r + e] = occ_gofs[o];
          rowg_kd[2 * (size_t)r + e] = P.kdim;
        }
      std::vector<int> gen_occ;
      std::vector<double> gen_R;
      std::vector<int8_t> occ_general(n_occ, 0);
      for (int o = 0; o < n_occ; ++o)
        if (ctx->occs[o].general) {
          gen_occ.push_back(o);
          gen_R.insert(gen_R.end(), ctx->occs[o].Rd, ctx->occs[o].Rd + 9);
          occ_general[o] = 1;
        }
      ctx->n_gen = (int)gen_occ.size();
      if (ctx->n_gen > 0) {
        for (int p = 0; p < n_pat; ++p)
          if (ctx->pats[p]->kdim > 6) throw Error(FETIRP_EINVAL, "general rotations need kernel dimensions <= 6");
        ctx->d_gen_occ.upload(gen_occ, s);
        ctx->d_gen_R.upload(gen_R, s);
        ctx->d_slot_nb.ensure((size_t)n_slots * 6);
      }
      ctx->d_occ_general.upload(occ_general, s);
      ctx->n_gcoef = 0;
      for (int kd : rowg_kd) ctx->n_gcoef += kd;
      ctx->d_rowg_gofs.upload(rowg_gofs, s);
      ctx->d_rowg_kd.upload(rowg_kd, s);
      ctx->d_rowg_coef.ensure(12 * (size_t)nl);
      ctx->ds_coef.ensure(2 * 12 * (size_t)nl);
    }
    ctx->d_pair_s.upload(pair_s, s);
    ctx->d_pair_t.upload(pair_t, s);
    ctx->n_pairs = (int)pair_s.size();
    std::vector<double> rot(9 * (size_t)n_occ);
    for (int o = 0; o < n_occ; ++o) std::memcpy(&rot[9 * (size_t)o], ctx->occs[o].Rd, sizeof(double) * 9);
    ctx->d_rot.upload(rot, s);
    ctx->uoff.assign(n_occ + 1, 0);
    for (int o = 0; o < n_occ; ++o) ctx->uoff[o + 1] = ctx->uoff[o] + ctx->pats[occ_pat[o]]->n;
    ctx->n_u = ctx->uoff[n_occ];
    ctx->d_uoff.upload(ctx->uoff, s);

    Layout& L = ctx->L;
    L = Layout{};
    L.n_lambda = nl; L.n_occ = n_occ; L.n_slots = n_slots; L.n_G = ctx->n_G; L.n_pat = n_pat; L.k = k;
    L.slot_ptr = ctx->d_slot_ptr.p; L.slot_row = ctx->d_slot_row.p; L.slot_sign = ctx->d_slot_sign.p;
    L.row_slot = ctx->d_row_slot.p; L.row_sign = ctx->d_row_sign.p; L.slot_occ = ctx->d_slot_occ.p;
    L.ell_w = ell_w; L.ell_row = ctx->d_ell_row.p; L.ell_sign = ctx->d_ell_sign.p;
    L.occ_obase = ctx->d_occ_obase.p; L.occ_pat = ctx->d_occ_pat.p; L.occ_q = ctx->d_occ_q.p;
    L.occ_gofs = ctx->d_occ_gofs.p; L.occ_group = ctx->d_occ_group.p;
    int max_nb = 1;
    for (int p = 0; p < n_pat; ++p) {
      L.Nb[p] = ctx->pats[p]->Nb.p;
      L.n_b[p] = ctx->pats[p]->n_b;
      L.kdim[p] = ctx->pats[p]->kdim;
      max_nb = std::max(max_nb, ctx->pats[p]->n_b);
    }
    L.row_grp = ctx->d_row_grp.p; L.row_wt = ctx->d_row_wt.p;
    L.rowg_gofs = ctx->d_rowg_gofs.p; L.rowg_kd = ctx->d_rowg_kd.p; L.rowg_coef = ctx->d_rowg_coef.p;
    L.rowg_coef_hi = ctx->ds_coef.p;
    L.rowg_coef_lo = ctx->ds_coef.p + 12 * (size_t)nl;
    L.slot_code = ctx->d_slot_code.p;
    for (int p = 0; p < n_pat; ++p) L.dpn[p] = ctx->pats[p]->dpn;
    L.n_gen = ctx->n_gen;
    L.gen_occ = ctx->n_gen ? ctx->d_gen_occ.p : nullptr;
    L.gen_R = ctx->n_gen ? ctx->d_gen_R.p : nullptr;
    L.slot_nb = ctx->n_gen ? ctx->d_slot_nb.p : nullptr;
    {  // G^T V chunks: at most 512 links per CTA, and at least two CTAs per SM while chunks keep >= 64 links
      int chunks =
          std::max(ceil_div(max_links, 512), std::min(ceil_div(max_links, 64), ceil_div(2 * 152, std::max(n_occ, 1))));
      L.gtv_chunk = (int)round_up(ceil_div(max_links, chunks), 32);
      L.gtv_chunks = ceil_div(max_links, L.gtv_chunk);
      ctx->d_gtv_part.ensure((size_t)std::max(n_occ, 1) * L.gtv_chunks * 6 * 64);
      ctx->d_gtv_ticket.ensure((size_t)std::max(n_occ, 1));
      ctx->d_gtv_ticket.zero(s);
      L.gtv_part = ctx->d_gtv_part.p; L.gtv_ticket = ctx->d_gtv_ticket.p;
    }
    // per-pattern loads (pattern frame, new ordering) and work
    for (int p = 0; p < n_pat; ++p) {
      PatternData& P = *ctx->pats[p];
      PatternUse& Us = ctx->use[p];
      const int no = (int)Us.occs.size();
      std::vector<double> F((size_t)P.npad * std::max(no, 1), 0.0);
      for (int q = 0; q < no; ++q) {
        const OccData& O = ctx->occs[Us.occs[q]];
        for (int d = 0; d < P.n; ++d) F[(size_t)q * P.npad + P.newidx[d]] = O.f_local[d];
      }
      Us.F.upload(F, s);
      Us.U.ensure((size_t)P.npad * std::max(no, 1));
      Us.d_occs.upload(Us.occs, s);
    }
    ctx->topo_valid = true;
    ctx->topo_nl = nl;
    ctx->topo_sig = sig;
  }
  const int k = ctx->k;
  Layout& L = ctx->L;
  for (int p = 0; p < n_pat; ++p) L.Nb[p] = ctx->pats[p]->Nb.p;
  ctx->sp.k = -1;   // the sparse-column plan belongs to the previous structure or factorisation
  // G by row from the current kernels
  row_coefs(L, ctx->d_rot.p, ctx->d_occ_general.p, ctx->d_rowg_coef.p, ctx->ds_coef.p, ctx->ds_coef.p + 12 * (size_t)nl,
            ctx->n_gen ? ctx->d_slot_nb.p : nullptr, s);
  // coarse problem: G^T G (FP64), its inverse, e, lambda_0 (projector paragraph)
  PhaseScope ph(ctx, FETIRP_PHASE_COARSE, 0.0, 0.0);
  ctx->n_Gpad = (int)round_up(std::max(ctx->n_G, 1), TILE);
  ctx->GtG.ensure((size_t)std::max(ctx->n_G, 1) * std::max(ctx->n_G, 1));
  ctx->Ginv.ensure((size_t)std::max(ctx->n_G, 1) * std::max(ctx->n_G, 1));
  ctx->e.ensure(std::max(ctx->n_G, 1));
  ctx->d.ensure(nl);
  ctx->lambda0.ensure(nl);
  ctx->c.ensure(nl);
  if (c_host) ctx->c.upload(c_host, nl, s);
  else if (c_dev) FETIRP_CUDA(cudaMemcpyAsync(ctx->c.p, c_dev, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
  else ctx->c.zero(s);
  ctx->Xc.ensure((size_t)std::max(ctx->n_G, 1) * 64);
  ctx->Ac.ensure((size_t)std::max(ctx->n_G, 1) * 64);
  ctx->sg_part.ensure((size_t)small_gemm_parts(std::max(ctx->n_G, 1)) * std::max(ctx->n_G, 1) * 64);
  if (ctx->n_G > 0) {
    gtg_dense(L, nullptr, nullptr, ctx->n_pairs, ctx->d_pair_s.p, ctx->d_pair_t.p, ctx->GtG.p, s);
    ctx->planG = dense_plan(ctx->n_Gpad / TILE);
    ctx->planG.upload(s);
    spd_inverse(ctx, ctx->GtG.p, ctx->n_G, ctx->n_Gpad, ctx->planG, ctx->zpG, ctx->Ginv.p);
    const long long ng2 = (long long)ctx->n_G * ctx->n_G;
    ctx->ds_ginv.ensure(2 * (size_t)ng2);
    split_pairs(ng2, ctx->Ginv.p, ctx->ds_ginv.p, ctx->ds_ginv.p + ng2, s);
    ctx->ds_xa.ensure(4 * (size_t)ctx->n_G * 64);
    // e_s = N^T f_s
    size_t scr = gemm_f64_scratch(ctx->n_G, 1, ctx->n_G);
    for (int p = 0; p < n_pat; ++p)
      scr = std::max(scr, gemm_f64_scratch(ctx->pats[p]->kdim, (int)ctx->use[p].occs.size(), ctx->pats[p]->npad));
    ctx->gemm_scratch.ensure(std::max<size_t>(scr, 1));
    for (int p = 0; p < n_pat; ++p) {
      PatternData& P = *ctx->pats[p];
      PatternUse& Us = ctx->use[p];
      const int no = (int)Us.occs.size();
      if (no == 0 || P.kdim == 0) continue;
      gemm_f64(P.kdim, no, P.npad, 1.0, P.N.p, P.npad, 1, Us.F.p, 1, P.npad, 0.0, ctx->e.p + ctx->pofs[p], 1, P.kdim,
               s, ctx->gemm_scratch.p, ctx->gemm_scratch.n);
    }
    gemm_f64(ctx->n_G, 1, ctx->n_G, 1.0, ctx->Ginv.p, ctx->n_G, 1, ctx->e.p, 1, 1, 0.0, ctx->Ac.p, 1, 1, s,
             ctx->gemm_scratch.p, ctx->gemm_scratch.n);
    g_apply(L, ctx->Ac.p, 1, 1.0, 0.0, ctx->lambda0.p, s);
  } else {
    ctx->lambda0.zero(s);
  }
  // d = sum_s B(s) K(s)^+ f(s) - c (Eq. 3).  Only the boundary rows of K^+ f enter d: the backward sweep stops at
  // the first boundary block row (the boundary is ordered last).  Patterns on concurrent streams.
  PatView<double> V{};
  fork_patterns(ctx, n_pat);
  for (int p = 0; p < n_pat; ++p) {
    PatternData& P = *ctx->pats[p];
    PatternUse& Us = ctx->use[p];
    const int no = (int)Us.occs.size();
    cudaStream_t ps = ctx->fstreams[p];
    if (no > 0) {
      const size_t bytes = sizeof(double) * (size_t)P.npad * no;
      FETIRP_CUDA(cudaMemcpyAsync(Us.U.p, Us.F.p, bytes, cudaMemcpyDeviceToDevice, ps));
      tri_solve(P.L.p, P.npad, P.plan, P.zp.p, Us.U.p, P.npad, no, false, ps, P.Dinv.p);
      Us.Yf.ensure((size_t)P.npad * no);
      FETIRP_CUDA(cudaMemcpyAsync(Us.Yf.p, Us.U.p, bytes, cudaMemcpyDeviceToDevice, ps));
      tri_solve(P.L.p, P.npad, P.plan, P.zp.p, Us.U.p, P.npad, no, true, ps, P.Dinv.p, false, P.n_i / TILE);
    }
    V.base[p] = Us.U.p; V.ld[p] = P.npad; V.off[p] = P.n_i;
  }
  join_patterns(ctx, n_pat);
  rotate_traces<double>(L, V, 1, false, s);
  scatter<double>(L, V, 1, 0.0, ctx->d.p, s);
  axpy_f64(nl, -1.0, ctx->c.p, ctx->d.p, s);
  // work buffers
  ctx->rr_blocks = std::max(1, std::min(1024, ceil_div(nl, 32)));   // <= the pinned read-back size
  ctx->rr_part.ensure(ctx->rr_blocks);
  ctx->lam.ensure(nl); ctx->r.ensure(nl); ctx->t1.ensure(nl);
  ctx->W.ensure((size_t)nl * k); ctx->Q.ensure((size_t)nl * k); ctx->Zr.ensure((size_t)nl * k);
  ctx->V1.ensure((size_t)nl * 64); ctx->V2.ensure((size_t)nl * 64);
  ctx->eta.ensure((size_t)k * k); ctx->wr.ensure(k);
  ctx->eta_part.ensure((size_t)(eta_chunks(nl) + ETA_GROUPS) * k * (k + 1)); ctx->T.ensure((size_t)k * k); ctx->alpha.ensure(k);
  ctx->n_kept.ensure(1);
  ctx->d_state.ensure(4);
  if (!ctx->tc_error.p) { ctx->tc_error.alloc(1); ctx->tc_error.zero(s); }
  tc_init();
  ensure_apply_buffers(ctx, k);
  if (ctx->gc.exec) { cudaGraphExecDestroy(ctx->gc.exec); ctx->gc.exec = nullptr; }   // buffers may have moved
  ctx->n_lambda = n_lambda;
  ctx->prepared = true;
  FETIRP_CUDA(cudaStreamSynchronize(s));
  if (ctx->pc.kind != 0) precond_setup(ctx);
  if (ctx->perm.on && ctx->perm.shortcut && k > 1 && ctx->pc.kind == 0) check_periodic(ctx);
}

// ----------------------------------------------------------------------------------------- operators
// V <- P V = V - G (G^T G)^{-1} G^T V (Eq. 6), FP64 throughout: with the rigid modes of elasticity G^T G is
// ill-conditioned enough that FP32 products leave G-components that make the inner operator nonsymmetric.
void project(fetirp_ctx ctx, double* V, int k) {
  if (ctx->n_G == 0) return;
  cudaStream_t s = ctx->stream;
  const double nl = ctx->L.n_lambda, nG = ctx->n_G;
  // G^T V and G A: 2 flops per coefficient of G (sign N_b[j][m] per link) and column, each; (G^T G)^{-1} X
  PhaseScope ph(ctx, FETIRP_PHASE_PROJECT, 2.0 * nG * nG * k + 4.0 * ctx->n_gcoef * k, 16.0 * nl * k + 8.0 * nG * nG);
  ctx->Xc.ensure((size_t)ctx->n_G * k);
  ctx->Ac.ensure((size_t)ctx->n_G * k);
  if (ctx->ds_project) {   // inner solves of the mixed forms: double-single sums on the FP32 pipe (~2^-46)
    const long long ngk = (long long)ctx->n_G * k;
    float* xh = ctx->ds_xa.p;
    float* xl = xh + (size_t)ctx->n_G * 64;
    float* ah = xl + (size_t)ctx->n_G * 64;
    float* al = ah + (size_t)ctx->n_G * 64;
    const long long ng2 = (long long)ctx->n_G * ctx->n_G;
    gt_v_ds(ctx->L, V, k, ctx->Xc.p, s);
    split_pairs(ngk, ctx->Xc.p, xh, xl, s);
    small_gemm_ds(ctx->n_G, k, ctx->ds_ginv.p, ctx->ds_ginv.p + ng2, xh, xl, ctx->Ac.p, s, ctx->sg_part.p);
    split_pairs(ngk, ctx->Ac.p, ah, al, s);
    g_apply_ds(ctx->L, ah, al, k, -1.0, 1.0, V, s);
    return;
  }
  gt_v(ctx->L, V, k, ctx->Xc.p, s);
  small_gemm(ctx->n_G, k, ctx->Ginv.p, ctx->Xc.p, ctx->Ac.p, s, ctx->sg_part.p);
  g_apply(ctx->L, ctx->Ac.p, k, -1.0, 1.0, V, s);
}

// gather -> local products -> scatter, each bracketed as its own phase
template <typename T>
void run_local(fetirp_ctx ctx, const Layout& L, const double* src, double* out, int k, const PatView<T>& Yv,
               const PatView<T>& Zv, const LocalProblem& LP, double es) {
  cudaStream_t s = ctx->stream;
  double flops = 0, sbytes = 0, rhs_elems = 0;
  for (int p = 0; p < LP.n_pat; ++p) {
    flops += 2.0 * LP.n_b[p] * (double)LP.n_b[p] * LP.n_rhs[p];
    sbytes += (double)LP.n_b[p] * LP.n_b[p] * es;
    rhs_elems += (double)LP.n_b[p] * LP.n_rhs[p];
  }
  const double vbytes = 8.0 * L.n_lambda * k;
  {
    PhaseScope ph(ctx, FETIRP_PHASE_GATHER, 0.0, vbytes + rhs_elems * es);
    gather<T>(L, src, k, Yv, s);
    rotate_traces<T>(L, Yv, k, true, s);
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_LOCAL, flops, sbytes + 2.0 * rhs_elems * es);
    if (es == 8.0) local_gemm_f64(LP, s);
    else local_gemm_f32(LP, s);
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_SCATTER, 0.0, vbytes + rhs_elems * es);
    rotate_traces<T>(L, Zv, k, false, s);
    scatter<T>(L, Zv, k, 0.0, out, s);
  }
}

// out = F in (F = sum_s B K^+ B^T through S^+), block of k columns; optional projections around it.
void apply_F(fetirp_ctx ctx, const double* in, double* out, int k, int prec, bool project_in, bool project_out) {
  cudaStream_t s = ctx->stream;
  const Layout& L = ctx->L;
  const double* src = in;
  if (project_in && ctx->n_G > 0) {
    ctx->V2.ensure((size_t)L.n_lambda * k);
    FETIRP_CUDA(cudaMemcpyAsync(ctx->V2.p, in, sizeof(double) * (size_t)L.n_lambda * k, cudaMemcpyDeviceToDevice, s));
    project(ctx, ctx->V2.p, k);
    src = ctx->V2.p;
  }
  const int n_pat = (int)ctx->pats.size();
  long long total = 0;
  std::vector<long long> base(n_pat);
  for (int p = 0; p < n_pat; ++p) {
    base[p] = total;
    total += (long long)ctx->use[p].occs.size() * k * ctx->pats[p]->ld_y;
  }
  LocalProblem LP{};
  LP.n_pat = n_pat;
  if (prec == FETIRP_PREC_FP64) {
    ctx->Y64.ensure(total); ctx->Z64.ensure(total);
    if (factored_f64(ctx)) ctx->W64.ensure(total);
    PatView<double> Yv{}, Zv{};
    for (int p = 0; p < n_pat; ++p) {
      PatternData& P = *ctx->pats[p];
      Yv.base[p] = ctx->Y64.p + base[p]; Yv.ld[p] = P.ld_y; Yv.off[p] = 0;
      Zv.base[p] = ctx->Z64.p + base[p]; Zv.ld[p] = P.ld_y; Zv.off[p] = 0;
      LP.S[p] = P.S64.p; LP.n_b[p] = P.n_b; LP.n_rhs[p] = (int)ctx->use[p].occs.size() * k; LP.ld[p] = P.ld_y;
      LP.Y[p] = Yv.base[p]; LP.Z[p] = Zv.base[p];
      set_factored(LP, p, P, P.s64_ok ? nullptr : ctx->W64.p + base[p]);
    }
    run_local<double>(ctx, L, src, out, k, Yv, Zv, LP, 8.0);
  } else if (prec == FETIRP_PREC_FP32) {
    ctx->Y32.ensure(total); ctx->Z32.ensure(total);
    PatView<float> Yv{}, Zv{};
    for (int p = 0; p < n_pat; ++p) {
      PatternData& P = *ctx->pats[p];
      Yv.base[p] = ctx->Y32.p + base[p]; Yv.ld[p] = P.ld_y; Yv.off[p] = 0;
      Zv.base[p] = ctx->Z32.p + base[p]; Zv.ld[p] = P.ld_y; Zv.off[p] = 0;
      LP.S[p] = P.S32.p; LP.n_b[p] = P.n_b; LP.n_rhs[p] = (int)ctx->use[p].occs.size() * k; LP.ld[p] = P.ld_y;
      LP.Y[p] = Yv.base[p]; LP.Z[p] = Zv.base[p];
    }
    run_local<float>(ctx, L, src, out, k, Yv, Zv, LP, 4.0);
  } else if (prec == FETIRP_PREC_TF32X3) {
    ctx->Y32.ensure(total); ctx->Ylo32.ensure(total); ctx->Z32.ensure(total);
    if (!ctx->tc_error.p) { ctx->tc_error.alloc(1); ctx->tc_error.zero(s); }
    PatView<float> Yh{}, Yl{}, Zv{};
    TcProblem T;
    T.n_pat = n_pat;
    T.part = ctx->tc_part.p;
    T.part_elems = (long long)ctx->tc_part.n;
    double flops = 0, bytes = 0, rhs_elems = 0;
    for (int p = 0; p < n_pat; ++p) {
      PatternData& P = *ctx->pats[p];
      Yh.base[p] = ctx->Y32.p + base[p]; Yh.ld[p] = P.ld_y; Yh.off[p] = 0;
      Yl.base[p] = ctx->Ylo32.p + base[p]; Yl.ld[p] = P.ld_y; Yl.off[p] = 0;
      Zv.base[p] = ctx->Z32.p + base[p]; Zv.ld[p] = P.ld_y; Zv.off[p] = 0;
      T.S_hi[p] = P.S_hi.p; T.S_lo[p] = P.S_lo.p; T.lds[p] = P.lds;
      T.Y_hi[p] = Yh.base[p]; T.Y_lo[p] = Yl.base[p]; T.Z[p] = Zv.base[p]; T.ldy[p] = P.ld_y;
      T.n_b[p] = P.n_b; T.n_rhs[p] = (int)ctx->use[p].occs.size() * k;
      flops += 2.0 * P.n_b * (double)P.n_b * T.n_rhs[p];
      bytes += 2.0 * P.n_b * (double)P.n_b * 4 + 3.0 * P.n_b * (double)T.n_rhs[p] * 4;
      rhs_elems += (double)P.n_b * T.n_rhs[p];
    }
    const double vbytes = 8.0 * L.n_lambda * k;
    {
      PhaseScope ph(ctx, FETIRP_PHASE_GATHER, 0.0, vbytes + 2.0 * rhs_elems * 4);
      gather_split(L, src, k, Yh, Yl, s);
      rotate_split(L, Yh, Yl, k, s);   // general rotations: turned to the pattern frame and split again
    }
    {
      PhaseScope ph(ctx, FETIRP_PHASE_LOCAL, flops, bytes);
      tc_gemm_tf32x3(T, ctx->tc_error.p, s);
    }
    {
      PhaseScope ph(ctx, FETIRP_PHASE_SCATTER, 0.0, vbytes + rhs_elems * 4);
      rotate_traces<float>(L, Zv, k, false, s);
      scatter<float>(L, Zv, k, 0.0, out, s);
    }
  } else if (prec == FETIRP_PREC_BF16X3) {
    if (L.n_gen > 0)
      throw Error(FETIRP_EINVAL, "bf16x3 takes rotations of vector fields in 90-degree steps only");
    long long total8 = 0;
    std::vector<long long> base8(n_pat);
    for (int p = 0; p < n_pat; ++p) {
      base8[p] = total8;
      total8 += (long long)ctx->use[p].occs.size() * k * ctx->pats[p]->ld_y8;
    }
    ctx->Y32.ensure(total8); ctx->Ylo32.ensure(total8); ctx->Z32.ensure(total8);
    if (!ctx->tc_error.p) { ctx->tc_error.alloc(1); ctx->tc_error.zero(s); }
    PatView<__nv_bfloat16> Yh{}, Yl{};
    PatView<float> Zv{};
    TcProblem T;
    T.n_pat = n_pat;
    T.part = ctx->tc_part.p;
    T.part_elems = (long long)ctx->tc_part.n;
    double flops = 0, bytes = 0, rhs_elems = 0;
    for (int p = 0; p < n_pat; ++p) {
      PatternData& P = *ctx->pats[p];
      Yh.base[p] = reinterpret_cast<__nv_bfloat16*>(ctx->Y32.p) + base8[p]; Yh.ld[p] = P.ld_y8; Yh.off[p] = 0;
      Yl.base[p] = reinterpret_cast<__nv_bfloat16*>(ctx->Ylo32.p) + base8[p]; Yl.ld[p] = P.ld_y8; Yl.off[p] = 0;
      Zv.base[p] = ctx->Z32.p + base8[p]; Zv.ld[p] = P.ld_y8; Zv.off[p] = 0;
      T.S_hi[p] = P.Sb_hi.p; T.S_lo[p] = P.Sb_lo.p; T.lds[p] = P.ldsb;
      T.Y_hi[p] = Yh.base[p]; T.Y_lo[p] = Yl.base[p]; T.Z[p] = Zv.base[p]; T.ldy[p] = P.ld_y8;
      T.n_b[p] = P.n_b; T.n_rhs[p] = (int)ctx->use[p].occs.size() * k;
      flops += 2.0 * P.n_b * (double)P.n_b * T.n_rhs[p];
      bytes += 2.0 * P.n_b * (double)P.n_b * 2 + 2.0 * P.n_b * (double)T.n_rhs[p] * 2 + 4.0 * P.n_b * T.n_rhs[p];
      rhs_elems += (double)P.n_b * T.n_rhs[p];
    }
    const double vbytes = 8.0 * L.n_lambda * k;
    {
      PhaseScope ph(ctx, FETIRP_PHASE_GATHER, 0.0, vbytes + 2.0 * rhs_elems * 2);
      gather_split_bf16(L, src, k, Yh, Yl, s);
    }
    {
      PhaseScope ph(ctx, FETIRP_PHASE_LOCAL, flops, bytes);
      tc_gemm_bf16x3(T, ctx->tc_error.p, s);
    }
    {
      PhaseScope ph(ctx, FETIRP_PHASE_SCATTER, 0.0, vbytes + rhs_elems * 4);
      scatter<float>(L, Zv, k, 0.0, out, s);
    }
  } else {
    throw Error(FETIRP_EINVAL, "unsupported precision");
  }
  if (project_out) project(ctx, out, k);
}

// ---------------------------------------------------------------------------------------- preconditioners
// tilde-F^{-1} V = sum_s Delta(s) B(s) X(s) B(s)^T Delta(s) V (Eqs. 4-5) on a block of k columns, FP64: the
// scaled gather, the local operator of the occurrence's pattern (pattern frame), the scaled scatter.
void apply_M(fetirp_ctx ctx, const double* in, double* out, int k) {
  cudaStream_t s = ctx->stream;
  const Layout& L = ctx->L;
  const int n_pat = (int)ctx->pats.size();
  long long total = 0;
  std::vector<long long> base(n_pat);
  for (int p = 0; p < n_pat; ++p) {
    base[p] = total;
    total += (long long)ctx->use[p].occs.size() * k * ctx->pats[p]->ld_y;
  }
  ctx->Y64.ensure(total);
  ctx->Z64.ensure(total);
  PatView<double> Yv{}, Zv{};
  LocalProblem LP{};
  LP.n_pat = n_pat;
  for (int p = 0; p < n_pat; ++p) {
    PatternData& P = *ctx->pats[p];
    Yv.base[p] = ctx->Y64.p + base[p]; Yv.ld[p] = P.ld_y; Yv.off[p] = 0;
    Zv.base[p] = ctx->Z64.p + base[p]; Zv.ld[p] = P.ld_y; Zv.off[p] = 0;
    LP.S[p] = ctx->pc.X[p].p; LP.n_b[p] = P.n_b; LP.n_rhs[p] = (int)ctx->use[p].occs.size() * k; LP.ld[p] = P.ld_y;
    LP.Y[p] = Yv.base[p]; LP.Z[p] = Zv.base[p];
  }
  gather_w(L, in, k, Yv, ctx->pc.link_w.p, s);
  rotate_traces<double>(L, Yv, k, true, s);
  local_gemm_f64(LP, s);
  rotate_traces<double>(L, Zv, k, false, s);
  scatter_w(L, Zv, k, ctx->pc.row_w.p, out, s);
}

// The projector of Eqs. 6-7 in the preconditioner's metric, on a block of k columns in place:
//   Q V  = V - tilde-F^{-1} G (G^T tilde-F^{-1} G)^{-1} G^T V        (transpose = false)
//   Q^T V = V - G (G^T tilde-F^{-1} G)^{-1} G^T tilde-F^{-1} V        (transpose = true)
// Without a preconditioner both are P = I - G (G^T G)^{-1} G^T.
void project_q(fetirp_ctx ctx, double* V, int k, bool transpose) {
  if (ctx->pc.kind == 0) { project(ctx, V, k); return; }
  if (ctx->n_G == 0) return;
  cudaStream_t s = ctx->stream;
  const Layout& L = ctx->L;
  const int nl = L.n_lambda;
  PhaseScope ph(ctx, FETIRP_PHASE_PROJECT, 0.0, 0.0);
  double* T1 = ctx->pc.T1.p;
  double* T2 = ctx->pc.T2.p;
  if (transpose) {
    apply_M(ctx, V, T1, k);
    gt_v(L, T1, k, ctx->Xc.p, s);
    small_gemm(ctx->n_G, k, ctx->pc.GtMGinv.p, ctx->Xc.p, ctx->Ac.p, s, ctx->sg_part.p);
    g_apply(L, ctx->Ac.p, k, -1.0, 1.0, V, s);
  } else {
    gt_v(L, V, k, ctx->Xc.p, s);
    small_gemm(ctx->n_G, k, ctx->pc.GtMGinv.p, ctx->Xc.p, ctx->Ac.p, s, ctx->sg_part.p);
    g_apply(L, ctx->Ac.p, k, 1.0, 0.0, T1, s);
    apply_M(ctx, T1, T2, k);
    axpy_f64(nl * k, -1.0, T2, V, s);
  }
}

// Local operators X_p of the chosen preconditioner, G^T tilde-F^{-1} G and its inverse, and lambda_0 in the
// preconditioner's metric (Table 1's initialisation with the projector of Eqs. 6-7).
void precond_setup(fetirp_ctx ctx) {
  cudaStream_t s = ctx->stream;
  const Layout& L = ctx->L;
  const int nl = L.n_lambda, n_pat = (int)ctx->pats.size();
  auto& pc = ctx->pc;
  for (int p = 0; p < n_pat; ++p) {
    const PatternData& P = *ctx->pats[p];
    const int nb = P.n_b;
    // K_bb in the pattern frame, boundary dofs in slot order (bpos * dpn + c)
    std::vector<double> Kbb((size_t)nb * nb, 0.0);
    std::vector<int> slot_of(P.n, -1);
    for (int b = 0; b < (int)P.bnd_nodes.size(); ++b)
      for (int c = 0; c < P.dpn; ++c) slot_of[P.bnd_nodes[b] * P.dpn + c] = b * P.dpn + c;
    for (int i = 0; i < P.n; ++i) {
      if (slot_of[i] < 0) continue;
      for (int64_t e = P.rowptr[i]; e < P.rowptr[i + 1]; ++e) {
        const int j = slot_of[P.col[e]];
        if (j < 0) continue;
        if (pc.kind == FETIRP_PRECOND_SUPERLUMPED && j != slot_of[i]) continue;
        Kbb[(size_t)slot_of[i] * nb + j] += P.val[e];
      }
    }
    pc.X[p].upload(Kbb, s);
    if (pc.kind == FETIRP_PRECOND_DIRICHLET) {
      // S = K_bb - K_bi K_ii^{-1} K_ib with W = L_ii^{-1} K_ib from the interior block of the factor (the forward
      // solve of the interior rows involves only L_ii), S -= W^T W
      const int npad = P.npad, ni = P.n_i;
      std::vector<double> rhs((size_t)npad * nb, 0.0);   // column-major, new (interior-first) ordering
      for (int i = 0; i < P.n; ++i) {
        const int nr = P.newidx[i];
        if (nr >= ni) continue;
        for (int64_t e = P.rowptr[i]; e < P.rowptr[i + 1]; ++e) {
          const int j = slot_of[P.col[e]];
          if (j >= 0) rhs[(size_t)j * npad + nr] += P.val[e];
        }
      }
      DBuf<double> Wd;
      Wd.upload(rhs, s);
      tri_solve(P.L.p, npad, P.plan, P.zp.p, Wd.p, npad, nb, false, s, P.Dinv.p);
      gemm_f64(nb, nb, ni, -1.0, Wd.p, npad, 1, Wd.p, 1, npad, 1.0, pc.X[p].p, nb, 1, s);
      FETIRP_CUDA(cudaStreamSynchronize(s));
    }
  }
  pc.T1.ensure((size_t)nl * 64);
  pc.T2.ensure((size_t)nl * 64);
  if (ctx->n_G == 0) return;
  const int nG = ctx->n_G;
  // G^T tilde-F^{-1} G, 64 columns of G at a time
  pc.GtMG.ensure((size_t)nG * nG);
  pc.GtMGinv.ensure((size_t)nG * nG);
  std::vector<double> unit;
  DBuf<double> dunit;
  for (int c0 = 0; c0 < nG; c0 += 64) {
    const int kb = std::min(64, nG - c0);
    unit.assign((size_t)nG * kb, 0.0);
    for (int i = 0; i < kb; ++i) unit[(size_t)(c0 + i) * kb + i] = 1.0;
    dunit.upload(unit, s);
    g_apply(L, dunit.p, kb, 1.0, 0.0, pc.T1.p, s);
    apply_M(ctx, pc.T1.p, pc.T2.p, kb);
    gt_v(L, pc.T2.p, kb, ctx->Xc.p, s);
    FETIRP_CUDA(cudaMemcpy2DAsync(pc.GtMG.p + c0, sizeof(double) * nG, ctx->Xc.p, sizeof(double) * kb,
                                  sizeof(double) * kb, nG, cudaMemcpyDeviceToDevice, s));
    FETIRP_CUDA(cudaStreamSynchronize(s));   // unit and dunit are reused by the next block
  }
  pc.plan = dense_plan(ctx->n_Gpad / TILE);
  pc.plan.upload(s);
  spd_inverse(ctx, pc.GtMG.p, nG, ctx->n_Gpad, pc.plan, pc.zp, pc.GtMGinv.p);
  // lambda_0 = tilde-F^{-1} G (G^T tilde-F^{-1} G)^{-1} e
  gemm_f64(nG, 1, nG, 1.0, pc.GtMGinv.p, nG, 1, ctx->e.p, 1, 1, 0.0, ctx->Ac.p, 1, 1, s);
  g_apply(L, ctx->Ac.p, 1, 1.0, 0.0, pc.T1.p, s);
  apply_M(ctx, pc.T1.p, ctx->lambda0.p, 1);
  FETIRP_CUDA(cudaStreamSynchronize(s));
}

// The periodic shortcut computes the F-image of [z, Pi z, ...] from the one of z, which is exact only when Pi
// commutes with P^T F P (a structure made of rotated copies, Pi the map of multiplier rows under the rotation).
// Checked once per structure in FP64 on a seeded vector: P^T F P (Pi v) against Pi (P^T F P v).
void check_periodic(fetirp_ctx ctx) {
  cudaStream_t s = ctx->stream;
  const int nl = ctx->L.n_lambda, k = ctx->perm.k, pw = ctx->perm.pw;
  std::vector<double> v(nl);
  uint64_t x = 0x9E3779B97F4A7C15ull;
  for (int i = 0; i < nl; ++i) {   // splitmix64 values in [-1, 1)
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
  }
  ctx->V1.upload(v.data(), nl, s);
  perm_split(nl, k, pw, ctx->perm.d_src.p, ctx->perm.d_w.p, ctx->V1.p, ctx->t1.p, s, 1);   // Pi v
  apply_F(ctx, ctx->t1.p, ctx->W.p, 1, FETIRP_PREC_FP64, true, true);                       // P^T F P Pi v
  apply_F(ctx, ctx->V1.p, ctx->Q.p, 1, FETIRP_PREC_FP64, true, true);                       // P^T F P v
  perm_split(nl, k, pw, ctx->perm.d_src.p, ctx->perm.d_w.p, ctx->Q.p, ctx->t1.p, s, 1);     // Pi P^T F P v
  std::vector<double> a(nl), b(nl);
  FETIRP_CUDA(cudaMemcpyAsync(a.data(), ctx->W.p, sizeof(double) * nl, cudaMemcpyDeviceToHost, s));
  FETIRP_CUDA(cudaMemcpyAsync(b.data(), ctx->t1.p, sizeof(double) * nl, cudaMemcpyDeviceToHost, s));
  FETIRP_CUDA(cudaStreamSynchronize(s));
  double dn = 0.0, bn = 0.0;
  for (int i = 0; i < nl; ++i) { dn += (a[i] - b[i]) * (a[i] - b[i]); bn += b[i] * b[i]; }
  if (!(std::sqrt(dn) <= 1e-9 * std::sqrt(bn)))
    throw Error(FETIRP_EINVAL, "the periodic shortcut needs P^T F P Pi = Pi P^T F P; relative mismatch " +
                                   std::to_string(std::sqrt(dn / std::max(bn, 1e-300))));
}

double norm2(fetirp_ctx ctx, const double* x, int n) {
  {
    PhaseScope ph(ctx, FETIRP_PHASE_UPDATE, 2.0 * n, 8.0 * n);
    sum_sq(n, x, ctx->rr_part.p, ctx->rr_blocks, ctx->stream);
  }
  std::vector<double> h(ctx->rr_blocks);
  FETIRP_CUDA(cudaMemcpyAsync(h.data(), ctx->rr_part.p, sizeof(double) * ctx->rr_blocks, cudaMemcpyDeviceToHost,
                              ctx->stream));
  FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
  double acc = 0.0;
  for (double v : h) acc += v;
  return std::sqrt(acc);
}

// Residual r = P^T (d - F lambda) in FP64 (the projected residual of Table 1).
void residual(fetirp_ctx ctx) {
  PhaseOverride ov(ctx, FETIRP_PHASE_OUTER);
  const int nl = ctx->L.n_lambda;
  apply_F(ctx, ctx->lam.p, ctx->r.p, 1, FETIRP_PREC_FP64, false, false);
  // r = d - F lambda
  cudaStream_t s = ctx->stream;
  ctx->t1.ensure(nl);
  FETIRP_CUDA(cudaMemcpyAsync(ctx->t1.p, ctx->d.p, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
  axpy_f64(nl, -1.0, ctx->r.p, ctx->t1.p, s);
  FETIRP_CUDA(cudaMemcpyAsync(ctx->r.p, ctx->t1.p, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
  project_q(ctx, ctx->r.p, 1, true);
}

// lambda <- lambda_0 + P (lambda - lambda_0) in FP64: keeps G^T lambda = e exactly after corrections built
// from directions that were stored in FP32 (their rounding leaves range(P) at the 1e-7 level).
void reproject_lambda(fetirp_ctx ctx) {
  if (ctx->n_G == 0) return;
  PhaseOverride ov(ctx, FETIRP_PHASE_OUTER);
  const int nl = ctx->L.n_lambda;
  cudaStream_t s = ctx->stream;
  axpy_f64(nl, -1.0, ctx->lambda0.p, ctx->lam.p, s);
  project_q(ctx, ctx->lam.p, 1, false);
  axpy_f64(nl, 1.0, ctx->lambda0.p, ctx->lam.p, s);
}

struct Hist {
  long long cols = 0;    // columns stored
  bool stalled = false;  // the last inner solve stopped making progress (see block_orthodir)
};

template <typename TH> TH* hist_w(fetirp_ctx ctx);
template <typename TH> TH* hist_q(fetirp_ctx ctx);
template <> double* hist_w<double>(fetirp_ctx ctx) { return ctx->Whist.p; }
template <> double* hist_q<double>(fetirp_ctx ctx) { return ctx->Qhist.p; }
template <> float* hist_w<float>(fetirp_ctx ctx) { return ctx->Whist32.p; }
template <> float* hist_q<float>(fetirp_ctx ctx) { return ctx->Qhist32.p; }

// One block iteration, enqueued only (no host read-back), so that it can be captured in a CUDA graph.  The
// number of stored directions lives on the device (d_state[0]); every kernel that depends on it reads it there.
// Reorthogonalisation coefficients C = Q_h^T W are FP64 sums; since Q_h lies in range(P) and W = P S(r),
// C = Q_h^T S(r) is taken from the split structure of S(r) (at most two nonzero columns per row).
// One block iteration with a preconditioner of Eqs. 4-5 (Table 1, right column, preconditioned): the directions
// are the split of z = Q tilde-F^{-1} r (scaled by Delta, or the permutation images of z), made admissible by Q,
// reorthogonalised against the history and made admissible again (the extra Q keeps the rounding of the
// subtraction out of range(G)); their F-image is Q^T F W.  The reorthogonalisation coefficients Q_h^T Q S(z) =
// Q_h^T S(z) come from the split structure as in the unpreconditioned iteration.
template <typename TH>
void enqueue_iteration_pc(fetirp_ctx ctx, int prec, TH* Wh, TH* Qh) {
  cudaStream_t s = ctx->stream;
  const int nl = ctx->L.n_lambda, k = ctx->k;
  const long long cap = ctx->hist_cap;
  int* d_cols = ctx->d_state.p;
  double* z = ctx->t1.p;
  const bool permuted = ctx->perm.on;
  {
    PhaseScope ph(ctx, FETIRP_PHASE_PROJECT, 0.0, 0.0);
    apply_M(ctx, ctx->r.p, z, 1);
  }
  project_q(ctx, z, 1, false);
  {
    PhaseScope ph(ctx, FETIRP_PHASE_UPDATE, 0.0, 0.0);
    if (permuted) perm_split(nl, k, ctx->perm.pw, ctx->perm.d_src.p, ctx->perm.d_w.p, z, ctx->Zr.p, s);
    else split_w(ctx->L, z, k, ctx->pc.row_d.p, ctx->Zr.p, s);
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_GRAM, 0.0, 0.0);
    gram_split<TH>((int)cap, d_cols, k, Qh, nl, k, z, ctx->d_grp_ptr.p, ctx->d_grp_row.p, ctx->pc.grp_wd.p,
                   ctx->n_grp_entries, ctx->max_group_rows, ctx->C.p, ctx->gram_part, ctx->grp_wr, s,
                   permuted ? ctx->perm.d_grp_src.p : nullptr);
  }
  project_q(ctx, ctx->Zr.p, k, false);
  {
    PhaseScope ph(ctx, FETIRP_PHASE_REORTH, 0.0, 0.0);
    tall_update<TH>(nl, (int)cap, d_cols, k, Wh, k, ctx->C.p, -1.0, ctx->Zr.p, ctx->tu_part, ctx->tu_tickets, s);
  }
  project_q(ctx, ctx->Zr.p, k, false);
  apply_F(ctx, ctx->Zr.p, ctx->Q.p, k, prec, false, false);
  project_q(ctx, ctx->Q.p, k, true);   // P~ = Q^T F W
  int eta_off = 0, eta_n = 1;
  {
    PhaseScope ph(ctx, FETIRP_PHASE_GRAM, 0.0, 0.0);
    eta_off = eta_partials(nl, k, ctx->Zr.p, ctx->Q.p, ctx->r.p, ctx->eta_part, s, prec != FETIRP_PREC_FP64,
                           &eta_n);
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_NORMALISE, 0.0, 0.0);
    normalise(k, ctx->eta_part.p + (size_t)eta_off * k * (k + 1), eta_n,
              prec == FETIRP_PREC_FP64 ? ctx->opt.eig_trunc : ctx->opt.eig_trunc_inner, ctx->T.p, ctx->alpha.p,
              ctx->n_kept.p, s);
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_UPDATE, 0.0, 0.0);
    AdvanceArgs adv;
    adv.cols = d_cols; adv.k = k; adv.cap = cap; adv.n_kept = ctx->n_kept.p;
    adv.dropped = ctx->d_state.p + 1; adv.iters = ctx->d_state.p + 2;
    adv.counter = reinterpret_cast<unsigned*>(ctx->d_state.p + 3);
    update<TH>(nl, k, ctx->Zr.p, ctx->Q.p, ctx->T.p, ctx->alpha.p, Wh, Qh, d_cols, ctx->lam.p, ctx->r.p,
               ctx->rr_part.p, ctx->rr_blocks, s, adv);
  }
}

template <typename TH>
void enqueue_iteration(fetirp_ctx ctx, int prec, TH* Wh, TH* Qh) {
  if (ctx->pc.kind != 0) { enqueue_iteration_pc<TH>(ctx, prec, Wh, Qh); return; }
  int eta_off = 0, eta_n = 1;
  cudaStream_t s = ctx->stream;
  const int nl = ctx->L.n_lambda, k = ctx->k;
  struct DsScope {   // double-single projections while the inner iteration of a mixed form is enqueued
    fetirp_ctx c;
    bool saved;
    DsScope(fetirp_ctx c_, bool on) : c(c_), saved(c_->ds_project) { c->ds_project = on; }
    ~DsScope() { c->ds_project = saved; }
  } ds_scope(ctx, prec != FETIRP_PREC_FP64);
  const long long cap = ctx->hist_cap;
  int* d_cols = ctx->d_state.p;
  const bool permuted = ctx->perm.on;
  {
    PhaseScope ph(ctx, FETIRP_PHASE_UPDATE, 0.0, 0.0);
    if (permuted)   // Eq. 8: [r, Pi r, ..., Pi^(k-1) r]
      perm_split(nl, k, ctx->perm.pw, ctx->perm.d_src.p, ctx->perm.d_w.p, ctx->r.p, ctx->Zr.p, s);
    else
      split(ctx->L, ctx->r.p, k, ctx->Zr.p, s);
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_GRAM, 0.0, 0.0);
    gram_split<TH>((int)cap, d_cols, k, Qh, nl, k, ctx->r.p, ctx->d_grp_ptr.p, ctx->d_grp_row.p, ctx->d_grp_w.p,
                   ctx->n_grp_entries, ctx->max_group_rows, ctx->C.p, ctx->gram_part, ctx->grp_wr, s,
                   permuted ? ctx->perm.d_grp_src.p : nullptr);
  }
  project(ctx, ctx->Zr.p, k);
  {
    PhaseScope ph(ctx, FETIRP_PHASE_REORTH, 0.0, 0.0);
    tall_update<TH>(nl, (int)cap, d_cols, k, Wh, k, ctx->C.p, -1.0, ctx->Zr.p, ctx->tu_part, ctx->tu_tickets, s);
  }
  if (permuted && ctx->perm.shortcut) {
    // periodic shortcut (Table 1, right, for a periodic structure): F commutes with Pi, so the F-image of
    // [r, Pi r, ...] is [p, Pi p, ...] with the one column p = P^T F P r; the reorthogonalised block's image
    // follows by the same linear combination, P~ = [p, Pi p, ...] - Q_h C, with no further F-apply
    apply_F(ctx, ctx->r.p, ctx->t1.p, 1, prec, true, true);
    {
      PhaseScope ph(ctx, FETIRP_PHASE_UPDATE, 0.0, 0.0);
      perm_split(nl, k, ctx->perm.pw, ctx->perm.d_src.p, ctx->perm.d_w.p, ctx->t1.p, ctx->Q.p, s);
    }
    {
      PhaseScope ph(ctx, FETIRP_PHASE_REORTH, 0.0, 0.0);
      tall_update<TH>(nl, (int)cap, d_cols, k, Qh, k, ctx->C.p, -1.0, ctx->Q.p, ctx->tu_part, ctx->tu_tickets, s);
    }
  } else {
    apply_F(ctx, ctx->Zr.p, ctx->Q.p, k, prec, false, true);   // P~ = P^T F W (the F-image of the directions, Table 1)
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_GRAM, 0.0, 0.0);
    eta_off = eta_partials(nl, k, ctx->Zr.p, ctx->Q.p, ctx->r.p, ctx->eta_part, s, prec != FETIRP_PREC_FP64,
                           &eta_n);
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_NORMALISE, 0.0, 0.0);
    normalise(k, ctx->eta_part.p + (size_t)eta_off * k * (k + 1), eta_n,
              prec == FETIRP_PREC_FP64 ? ctx->opt.eig_trunc : ctx->opt.eig_trunc_inner, ctx->T.p, ctx->alpha.p,
              ctx->n_kept.p, s);
  }
  {
    PhaseScope ph(ctx, FETIRP_PHASE_UPDATE, 0.0, 0.0);
    AdvanceArgs adv;
    adv.cols = d_cols; adv.k = k; adv.cap = cap; adv.n_kept = ctx->n_kept.p;
    adv.dropped = ctx->d_state.p + 1; adv.iters = ctx->d_state.p + 2;
    adv.counter = reinterpret_cast<unsigned*>(ctx->d_state.p + 3);
    update<TH>(nl, k, ctx->Zr.p, ctx->Q.p, ctx->T.p, ctx->alpha.p, Wh, Qh, d_cols, ctx->lam.p, ctx->r.p,
               ctx->rr_part.p, ctx->rr_blocks, s, adv);
  }
}

// Algorithmic work of one iteration with `a` stored directions (the per-phase flops and compulsory bytes).
void account_iteration(fetirp_ctx ctx, int prec, long long a, double es, bool persistent = false) {
  const double nl = ctx->L.n_lambda, k = ctx->k, nG = ctx->n_G;
  double* F = ctx->phase_flops;
  double* B = ctx->phase_bytes;
  double f0 = 0.0, b0 = 0.0;
  for (int i = 0; i < FETIRP_NPHASE; ++i) { f0 += F[i]; b0 += B[i]; }
  F[FETIRP_PHASE_GRAM] += 4.0 * nl * a + 2.0 * nl * k * (k + 1.0);
  B[FETIRP_PHASE_GRAM] += es * nl * a + 24.0 * nl + 8.0 * nl * (2.0 * k + 1.0);
  F[FETIRP_PHASE_REORTH] += 2.0 * nl * a * k;
  B[FETIRP_PHASE_REORTH] += es * nl * a + 16.0 * nl * k;
  F[FETIRP_PHASE_UPDATE] += 4.0 * nl * k * k + 4.0 * nl * k;
  F[FETIRP_PHASE_NORMALISE] += (2.0 / 3.0) * k * k * k;   // pivoted Cholesky + triangular inverse, O(k^3)
  B[FETIRP_PHASE_NORMALISE] += 8.0 * (2.0 * k * k + 2.0 * k);
  B[FETIRP_PHASE_UPDATE] += 8.0 * nl * (3.0 * k + 4.0) + 2.0 * es * nl * k;
  F[FETIRP_PHASE_PROJECT] += 2.0 * (2.0 * nG * nG * k + 4.0 * ctx->n_gcoef * k);
  B[FETIRP_PHASE_PROJECT] += 2.0 * (16.0 * nl * k + 8.0 * nG * nG);
  const double e_loc = prec == FETIRP_PREC_FP64 ? 8.0 : prec == FETIRP_PREC_BF16X3 ? 2.0 : 4.0;
  const bool pair = prec == FETIRP_PREC_TF32X3 || prec == FETIRP_PREC_BF16X3;   // operands as hi/lo pairs
  const double kf = ctx->perm.on && ctx->perm.shortcut ? 1.0 : k;   // columns of the iteration's F-apply
  if (kf != k) {   // periodic shortcut: one more history pass (Q -= Q_h C) and one more permuted copy
    F[FETIRP_PHASE_REORTH] += 2.0 * nl * a * k;
    B[FETIRP_PHASE_REORTH] += es * nl * a + 16.0 * nl * k;
  }
  double rhs = 0;
  for (size_t pi = 0; pi < ctx->pats.size(); ++pi) {
    const PatternData* P = ctx->pats[pi].get();
    const double R = (double)ctx->use[pi].occs.size() * kf;
    F[FETIRP_PHASE_LOCAL] += 2.0 * P->n_b * (double)P->n_b * R;
    B[FETIRP_PHASE_LOCAL] += (pair ? 2.0 : 1.0) * e_loc * P->n_b * (double)P->n_b +
                             (prec == FETIRP_PREC_TF32X3 ? 3.0 : 2.0) * e_loc * P->n_b * R;
    rhs += P->n_b * R;
  }
  B[FETIRP_PHASE_GATHER] += 8.0 * nl * kf + (pair ? 2.0 : 1.0) * e_loc * rhs;
  B[FETIRP_PHASE_SCATTER] += 8.0 * nl * kf + e_loc * rhs;
  if (persistent) {   // the whole iteration ran in one launch: its work is also that of the iterate phase
    double f1 = 0.0, b1 = 0.0;
    for (int i = 0; i < FETIRP_NPHASE; ++i) { f1 += F[i]; b1 += B[i]; }
    F[FETIRP_PHASE_ITERATE] += f1 - f0;
    B[FETIRP_PHASE_ITERATE] += b1 - b0;
  }
}

// Replay (or run) G iterations; returns the residual norm after the last one and the kept count.
template <typename TH>
void run_iterations(fetirp_ctx ctx, int prec, int G, bool use_graph, TH* Wh, TH* Qh) {
  cudaStream_t s = ctx->stream;
  auto& gc = ctx->gc;
  const int th = (int)sizeof(TH);
  if (use_graph) {
    const int tkey = ctx->opt.timing ? (1 + (ctx->opt.timing_mask & 0xFFFF) * 2) : 0;
    const bool valid = gc.exec && gc.prec == prec && gc.k == ctx->k && gc.G == G && gc.th == th &&
                       gc.cap == ctx->hist_cap && gc.timing == tkey;
    if (!valid) {
      if (gc.exec) { cudaGraphExecDestroy(gc.exec); gc.exec = nullptr; }
      gc.recs.clear();
      for (auto& v : gc.launches) v = 0;
      ctx->gev_used = 0;
      const unsigned long long l0 = g_launch_count;
      cudaGraph_t graph = nullptr;
      FETIRP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      ctx->capturing = true;
      try {
        for (int i = 0; i < G; ++i) enqueue_iteration<TH>(ctx, prec, Wh, Qh);
      } catch (...) {
        ctx->capturing = false;
        cudaStreamEndCapture(s, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      ctx->capturing = false;
      FETIRP_CUDA(cudaStreamEndCapture(s, &graph));
      cudaError_t e = cudaGraphInstantiate(&gc.exec, graph, 0);
      cudaGraphDestroy(graph);
      FETIRP_CUDA(e);
      gc.total_launches = (long long)(g_launch_count - l0);
      g_launch_count = l0;   // captured, not launched
      gc.prec = prec; gc.k = ctx->k; gc.G = G; gc.th = th; gc.cap = ctx->hist_cap; gc.timing = tkey;

    }
    FETIRP_CUDA(cudaGraphLaunch(gc.exec, s));
    g_launch_count += gc.total_launches;
    for (int p = 0; p < FETIRP_NPHASE; ++p) ctx->phase_launches[p] += gc.launches[p];
  } else {
    ctx->in_iteration = true;
    try {
      for (int i = 0; i < G; ++i) enqueue_iteration<TH>(ctx, prec, Wh, Qh);
    } catch (...) {
      ctx->in_iteration = false;
      throw;
    }
    ctx->in_iteration = false;
  }
}

// The persistent iteration serves latency-bound structures: FP64 or FP32 local products (SIMT), k <= 32, at
// most six kernel modes per occurrence, n_lambda up to 262144.
bool persist_eligible(fetirp_ctx ctx, int prec) {
  if (!ctx->opt.persistent) return false;
  if (prec != FETIRP_PREC_FP64 && prec != FETIRP_PREC_FP32) return false;
  if (ctx->k > 32 || ctx->L.n_lambda > 262144) return false;
  if (ctx->L.n_gen > 0) return false;   // general rotations turn the traces in separate passes
  if (ctx->perm.on) return false;       // the persistent phases build the occurrence split
  if (ctx->pc.kind != 0) return false;  // the persistent phases use the unweighted projector
  for (auto& P : ctx->pats)
    if (P->kdim > 6) return false;
  return persist_ctas(prec == FETIRP_PREC_FP64, ctx->k) > 0;
}

// Arguments of the persistent launch; sizes the buffers it needs (outside any capture).
template <typename TH>
PersistArgs persist_args(fetirp_ctx ctx, bool fp64, TH* Wh, TH* Qh) {
  cudaStream_t s = ctx->stream;
  const Layout& L = ctx->L;
  const int nl = L.n_lambda, k = ctx->k, n_pat = (int)ctx->pats.size();
  PersistArgs A{};
  A.L = L;
  A.n = nl;
  A.k = k;
  A.ncta = persist_ctas(fp64, k);
  A.cap = ctx->hist_cap;
  long long total = 0;
  for (int p = 0; p < n_pat; ++p) {
    PatternData& P = *ctx->pats[p];
    A.ybase[p] = total;
    A.ld[p] = P.ld_y;
    A.n_rhs[p] = (int)ctx->use[p].occs.size() * k;
    ensure_splus64(P, s);   // the persistent product reads S^+ or the FP32 S^dag as a matrix
    A.S[p] = fp64 ? (const void*)P.S64.p : (const void*)P.S32.p;
    A.pocc[p] = ctx->use[p].d_occs.p;
    total += (long long)ctx->use[p].occs.size() * k * P.ld_y;
  }
  int tiles = 0;
  for (int p = 0; p < n_pat; ++p) {
    A.tile_off[p] = tiles;
    A.tiles_m[p] = ceil_div(L.n_b[p], 16);
    tiles += A.tiles_m[p] * ceil_div(A.n_rhs[p], 16);
  }
  A.tile_off[n_pat] = tiles;
  if (fp64) {
    ctx->Y64.ensure(total); ctx->Z64.ensure(total);
    A.Ybuf = ctx->Y64.p; A.Zbuf = ctx->Z64.p;
  } else {
    ctx->Y32.ensure(total); ctx->Z32.ensure(total);
    A.Ybuf = ctx->Y32.p; A.Zbuf = ctx->Z32.p;
  }
  A.row_grp = ctx->d_row_grp.p; A.row_wt = ctx->d_row_wt.p; A.row_z = ctx->d_row_z.p; A.row_zld = ctx->d_row_zld.p;
  A.rowg_gofs = ctx->d_rowg_gofs.p; A.rowg_kd = ctx->d_rowg_kd.p; A.rowg_coef = ctx->d_rowg_coef.p;
  A.r = ctx->r.p; A.lam = ctx->lam.p; A.Zr = ctx->Zr.p; A.Q = ctx->Q.p;
  A.Wh = Wh; A.Qh = Qh;
  A.grp_ptr = ctx->d_grp_ptr.p; A.grp_row = ctx->d_grp_row.p; A.grp_w = ctx->d_grp_w.p;
  A.gs_chunks = std::max(1, ceil_div(ctx->max_group_rows, 128));
  A.gram_part = ctx->gram_part.p; A.C = ctx->C.p;
  A.Ginv = ctx->Ginv.p; A.Xc = ctx->Xc.p; A.Ac = ctx->Ac.p;
  // history splits sized for the persistent grid (about one item per CTA; never more than tu_part holds)
  A.tu_splits = std::max(1, std::min(tall_update_splits(nl, (int)ctx->hist_cap), A.ncta / ceil_div(nl, 64)));
  A.tu_part = ctx->tu_part.p; A.tu_tickets = ctx->tu_tickets.p;
  const int nout = k * (k + 1);
  ctx->pers_eta.ensure((size_t)(A.ncta + 64) * nout);
  ctx->prr.ensure(A.ncta);
  ctx->h_prr.assign(A.ncta, 0.0);
  if (!ctx->d_pbar.p) ctx->d_pbar.alloc(4 + 64);
  A.eta_part = ctx->pers_eta.p; A.eta_ticket = ctx->d_pbar.p + 2; A.eta_gticket = ctx->d_pbar.p + 4;
  A.trunc = fp64 ? ctx->opt.eig_trunc : ctx->opt.eig_trunc_inner;
  A.T = ctx->T.p; A.alpha = ctx->alpha.p; A.n_kept = ctx->n_kept.p;
  A.rr_part = ctx->prr.p; A.state = ctx->d_state.p;
  A.bar = ctx->d_pbar.p; A.err = reinterpret_cast<int*>(ctx->d_pbar.p + 3);
  A.timeout_ns = 2000000000ull;
  A.missing = 0;
  if (ctx->inject_stall) {   // one launch only, with a short limit
    A.missing = 1;
    A.timeout_ns = 200000000ull;
    ctx->inject_stall = false;
  }
  A.clk = nullptr;
  if (ctx->opt.timing) {
    if (!ctx->pers_clk.p) ctx->pers_clk.alloc(11);
    FETIRP_CUDA(cudaMemsetAsync(ctx->pers_clk.p, 0, 11 * sizeof(unsigned long long), s));
    A.clk = ctx->pers_clk.p;
  }
  return A;
}

// Block ORTHODIR iterations on P^T F_prec P (Table 1 right with full reorthogonalisation and
// F-normalisation).  Updates lam and r in place until ||r|| <= target or the caps are hit.  Directions kept in
// the history stay F_prec-orthonormal, so a later call with the same precision reuses them (Galerkin start).
// TH is the storage type of the direction history: FP64 for the plain form, FP32 inside the mixed forms.
// Iterations run in groups of check_every, captured once as a CUDA graph and replayed; the residual is read
// back after every group.
template <typename TH>
double block_orthodir(fetirp_ctx ctx, int prec, double target, double rnorm, Hist& H, fetirp_stats& st,
                      int& it_budget) {
  cudaStream_t s = ctx->stream;
  const int nl = ctx->L.n_lambda, k = ctx->k;
  const long long cap = ctx->hist_cap;
  TH* Wh = hist_w<TH>(ctx);
  TH* Qh = hist_q<TH>(ctx);
  const double es = sizeof(TH);
  // Galerkin start on the stored directions: lam += W_h (W_h^T r), r -= Q_h (W_h^T r)
  if (H.cols > 0) {
    const int a = (int)H.cols;
    {
      PhaseScope ph(ctx, FETIRP_PHASE_GRAM, 2.0 * nl * a, nl * (es * a + 8.0));
      hist_dot<TH>(nl, a, Wh, k, ctx->r.p, ctx->C.p, ctx->gram_part, s);
    }
    {
      PhaseScope ph(ctx, FETIRP_PHASE_REORTH, 4.0 * nl * a, 2.0 * es * nl * a + 32.0 * nl);
      tall_update<TH>(nl, a, nullptr, 1, Wh, k, ctx->C.p, 1.0, ctx->lam.p, ctx->tu_part, ctx->tu_tickets, s);
      tall_update<TH>(nl, a, nullptr, 1, Qh, k, ctx->C.p, -1.0, ctx->r.p, ctx->tu_part, ctx->tu_tickets, s);
    }
    rnorm = norm2(ctx, ctx->r.p, nl);
  }
  ctx->h_state[0] = (int)H.cols;
  ctx->h_state[1] = 0;
  ctx->h_state[2] = 0;
  ctx->h_state[3] = 0;   // last-CTA counter of update()
  FETIRP_CUDA(cudaMemcpyAsync(ctx->d_state.p, ctx->h_state, 4 * sizeof(int), cudaMemcpyHostToDevice, s));
  const int G = std::max(1, ctx->opt.check_every);
  int kept = k;
  if (persist_eligible(ctx, prec)) {
    // whole block iterations in one cooperative launch; the device stops at ||r||^2 <= target^2
    const bool fp64 = prec == FETIRP_PREC_FP64;
    PersistArgs A = persist_args(ctx, fp64, Wh, Qh);
    A.target2 = target * target;
    while (rnorm > target && it_budget > 0 && kept > 0) {
      FETIRP_CUDA(cudaMemsetAsync(ctx->d_pbar.p, 0, (4 + 64) * sizeof(unsigned), s));
      FETIRP_CUDA(cudaMemsetAsync(ctx->tu_tickets.p, 0, sizeof(unsigned) * ctx->tu_tickets.n, s));
      FETIRP_CUDA(cudaMemcpyAsync(ctx->h_state + 5, ctx->d_state.p + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
      A.max_iters = it_budget;
      {
        PhaseScope ph(ctx, FETIRP_PHASE_ITERATE, 0.0, 0.0);
        persist_iterations(A, fp64, s);
      }
      FETIRP_CUDA(cudaMemcpyAsync(ctx->h_state, ctx->d_state.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
      FETIRP_CUDA(cudaMemcpyAsync(ctx->h_state + 4, ctx->n_kept.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      FETIRP_CUDA(cudaMemcpyAsync(ctx->h_state + 6, ctx->d_pbar.p + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
      FETIRP_CUDA(cudaMemcpyAsync(ctx->h_prr.data(), ctx->prr.p, sizeof(double) * A.ncta, cudaMemcpyDeviceToHost, s));
      FETIRP_CUDA(cudaStreamSynchronize(s));
      if (ctx->h_state[6] != 0)
        throw Error(FETIRP_ETIMEOUT, "a grid barrier of the persistent iteration did not complete in time");
      if (A.clk) {   // phases inside the launch (CTA 0, barrier waits included); their sum is the iterate phase
        unsigned long long ns[11];
        FETIRP_CUDA(cudaMemcpy(ns, A.clk, sizeof(ns), cudaMemcpyDeviceToHost));
        FETIRP_CUDA(cudaMemsetAsync(A.clk, 0, sizeof(ns), s));
        // P8 (scatter, eta) contains the last CTA's eta reduction and normalisation, also booked as normalise
        const int map[11] = {FETIRP_PHASE_GRAM, FETIRP_PHASE_GRAM, FETIRP_PHASE_REORTH, FETIRP_PHASE_GATHER,
                             FETIRP_PHASE_LOCAL, FETIRP_PHASE_PROJECT, FETIRP_PHASE_PROJECT, FETIRP_PHASE_SCATTER,
                             FETIRP_PHASE_UPDATE, FETIRP_PHASE_NORMALISE, FETIRP_PHASE_NORMALISE};
        for (int i = 0; i < 11; ++i) ctx->graph_phase_ms[map[i]] += 1e-6 * (double)ns[i];
      }
      const int done = ctx->h_state[2] - ctx->h_state[5];
      for (int i = 0; i < done; ++i) {   // host mirror of the device history count (same restart rule)
        account_iteration(ctx, prec, H.cols, es, true);
        H.cols += k;
        if (H.cols + k > cap) H.cols = 0;
      }
      double acc = 0.0;
      for (int i = 0; i < A.ncta; ++i) acc += ctx->h_prr[i];
      rnorm = std::sqrt(acc);
      kept = ctx->h_state[4];
      st.iterations += done;
      it_budget -= done;
      if (done < A.max_iters) break;   // the device found ||r|| <= target (or no direction kept)
    }
  } else {
  // An inner solve of a mixed form whose residual has not dropped below 0.99 of its best for STALL iterations has
  // reached what its low-precision operator (or, with the periodic shortcut, the rounded commutation of F with
  // Pi) allows: it stops, and the outer FP64 step continues from the true residual with a fresh history.
  const bool watch = prec != FETIRP_PREC_FP64;
  const int STALL = std::max(200, 8 * G);
  double best = rnorm;
  int it_here = 0, best_it = 0;
  while (rnorm > target && it_budget > 0 && kept > 0) {
    const int g = std::min(G, it_budget);
    run_iterations<TH>(ctx, prec, g, g == G && ctx->opt.use_graphs, Wh, Qh);
    for (int i = 0; i < g; ++i) {   // host mirror of the device history count (same restart rule)
      account_iteration(ctx, prec, H.cols, es);
      H.cols += k;
      if (H.cols + k > cap) H.cols = 0;
    }
    FETIRP_CUDA(cudaMemcpyAsync(ctx->h_rr, ctx->rr_part.p, sizeof(double) * ctx->rr_blocks,
                                cudaMemcpyDeviceToHost, s));
    FETIRP_CUDA(cudaMemcpyAsync(ctx->h_state + 4, ctx->n_kept.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FETIRP_CUDA(cudaStreamSynchronize(s));
    if (ctx->opt.timing && g == G && ctx->opt.use_graphs)
      for (auto& r : ctx->gc.recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->gev_pool[r.e0], ctx->gev_pool[r.e1]) == cudaSuccess)
          ctx->graph_phase_ms[r.phase] += ms;
      }
    double acc = 0.0;
    for (int i = 0; i < ctx->rr_blocks; ++i) acc += ctx->h_rr[i];
    rnorm = std::sqrt(acc);
    kept = ctx->h_state[4];
    st.iterations += g;
    it_budget -= g;
    it_here += g;
    if (rnorm < 0.99 * best) {
      best = rnorm;
      best_it = it_here;
    } else if (watch && it_here - best_it >= STALL) {
      H.stalled = true;
      break;
    }
  }
  }
  FETIRP_CUDA(cudaMemcpyAsync(ctx->h_state, ctx->d_state.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
  FETIRP_CUDA(cudaStreamSynchronize(s));
  st.dropped_directions += ctx->h_state[1];
  return rnorm;
}

// res: d - F lambda for the current lambda when the caller has it (the solve's last FP64 residual), else null.
void recover(fetirp_ctx ctx, double* d_u_out, const double* res) {
  cudaStream_t s = ctx->stream;
  PhaseOverride ov(ctx, FETIRP_PHASE_RECOVER);
  PhaseScope ph(ctx, FETIRP_PHASE_RECOVER, 0.0, 0.0);
  const Layout& L = ctx->L;
  const int nl = L.n_lambda;
  const int n_pat = (int)ctx->pats.size();
  // alpha = (G^T G)^{-1} G^T (d - F lambda)   (first row of Eq. 3)
  if (ctx->n_G > 0) {
    if (!res) {
      apply_F(ctx, ctx->lam.p, ctx->t1.p, 1, FETIRP_PREC_FP64, false, false);
      ctx->V1.ensure(nl);
      FETIRP_CUDA(cudaMemcpyAsync(ctx->V1.p, ctx->d.p, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
      axpy_f64(nl, -1.0, ctx->t1.p, ctx->V1.p, s);
      res = ctx->V1.p;
    }
    gt_v(L, res, 1, ctx->Xc.p, s);
    gemm_f64(ctx->n_G, 1, ctx->n_G, 1.0, ctx->Ginv.p, ctx->n_G, 1, ctx->Xc.p, 1, 1, 0.0, ctx->Ac.p, 1, 1, s,
             ctx->gemm_scratch.p, ctx->gemm_scratch.n);
  }
  // u(s) = K^+ (f(s) - B(s)^T lambda) - N(s) alpha(s), with K^+ = L^{-T} L^{-1} and, by linearity,
  // L^{-1} (f - B^T lambda) = L^{-1} f - L^{-1} B^T lambda: the first term is the forward sweep kept from d, the
  // second lives on the boundary block rows only (the boundary is ordered last), so its sweep starts there.
  PatView<double> V{};
  for (int p = 0; p < n_pat; ++p) {
    PatternData& P = *ctx->pats[p];
    PatternUse& Us = ctx->use[p];
    const int no = (int)Us.occs.size();
    if (no > 0) FETIRP_CUDA(cudaMemsetAsync(Us.U.p, 0, sizeof(double) * (size_t)P.npad * no, s));
    V.base[p] = Us.U.p; V.ld[p] = P.npad; V.off[p] = P.n_i;
  }
  rotate_traces<double>(L, V, 1, false, s);   // general rotations: to the global frame, add -B^T lambda,
  gather<double>(L, ctx->lam.p, 1, V, s, -1.0, 1.0);
  rotate_traces<double>(L, V, 1, true, s);    // and back to the pattern frame
  fork_patterns(ctx, n_pat);   // patterns on concurrent streams
  for (int p = 0; p < n_pat; ++p) {
    PatternData& P = *ctx->pats[p];
    PatternUse& Us = ctx->use[p];
    const int no = (int)Us.occs.size();
    if (no == 0) continue;
    cudaStream_t ps = ctx->fstreams[p];
    double* Usol = Us.U.p;
    tri_solve(P.L.p, P.npad, P.plan, P.zp.p, Us.U.p, P.npad, no, false, ps, P.Dinv.p, false, 0, P.n_i / TILE);
    axpy_f64((int)((long long)P.npad * no), 1.0, Us.Yf.p, Us.U.p, ps);
    tri_solve(P.L.p, P.npad, P.plan, P.zp.p, Us.U.p, P.npad, no, true, ps, P.Dinv.p);
    if (P.kdim > 0 && ctx->n_G > 0)
      gemm_f64(P.npad, no, P.kdim, -1.0, P.N.p, 1, P.npad, ctx->Ac.p + ctx->pofs[p], 1, P.kdim, 1.0, Usol, 1,
               P.npad, ps);
    const long long tot = (long long)P.n * no;
    k_unpermute_rotate<<<(unsigned)((tot + 255) / 256), 256, 0, ps>>>(P.n, P.dpn, P.npad, Usol, P.d_newidx.p,
                                                                      Us.d_occs.p, ctx->d_rot.p, ctx->d_uoff.p, no,
                                                                      d_u_out);
    FETIRP_LAUNCH_CHECK();
  }
  join_patterns(ctx, n_pat);
}

bool hist_fp64(fetirp_ctx ctx) { return ctx->opt.precision == FETIRP_PREC_FP64 || ctx->pc.kind != 0; }

void ensure_history(fetirp_ctx ctx) {
  const int nl = ctx->L.n_lambda, k = ctx->k;
  // History: at most n_lambda directions can be F-orthogonal, and at most max_iter blocks are made; the two
  // arrays are also kept under 8 GB.  A full history restarts the recurrence.
  long long want = std::min<long long>((long long)std::max(1, ctx->opt.max_iter) * k, round_up(nl, k));
  // the two history arrays may take half of the device memory that is free (HBM is the limit, not a constant)
  size_t free_b = 0, total_b = 0;
  FETIRP_CUDA(cudaMemGetInfo(&free_b, &total_b));
  // FP64 history for the plain form, and for every preconditioned solve: the split of the weighted projection
  // (Q_h^T Q S(z) = Q_h^T S(z)) holds only for images exactly in range(Q^T), and rounding them to FP32 leaves
  // components that the preconditioner's contrast amplifies (measured: no convergence on the 1 / 1000 checkerboard)
  const bool h64 = hist_fp64(ctx);
  const double es_h = h64 ? 8.0 : 4.0;
  const double held = h64 ? 8.0 * (ctx->Whist.n + ctx->Qhist.n)
                                                             : 4.0 * (ctx->Whist32.n + ctx->Qhist32.n);
  const double avail = ctx->opt.history_bytes > 0 ? (double)ctx->opt.history_bytes : 0.5 * ((double)free_b + held);
  long long limit = (long long)(avail / (2.0 * es_h * std::max(nl, 1)));
  long long cap = std::max<long long>(k, std::min(want, limit));
  cap = cap / k * k;
  if (h64) {
    if (cap != ctx->hist_cap || (long long)ctx->Whist.n < (long long)nl * cap) {
      ctx->Whist.alloc((size_t)nl * cap);
      ctx->Qhist.alloc((size_t)nl * cap);
    }
  } else if (cap != ctx->hist_cap || (long long)ctx->Whist32.n < (long long)nl * cap) {
    ctx->Whist32.alloc((size_t)nl * cap);
    ctx->Qhist32.alloc((size_t)nl * cap);
  }
  if (cap != ctx->hist_cap && ctx->gc.exec) { cudaGraphExecDestroy(ctx->gc.exec); ctx->gc.exec = nullptr; }
  ctx->hist_cap = cap;
  const void* before[5] = {ctx->C.p, ctx->gram_part.p, ctx->Whist32.p, ctx->tu_part.p, ctx->tu_tickets.p};
  ctx->C.ensure((size_t)cap * k);
  // gram partials: the largest product is (cap x k) over nl rows
  const int ta = ceil_div(cap, 64), tb = ceil_div(k, 64);
  const int chunks = std::max(1, std::min(ceil_div(nl, 64), 304 / std::max(1, ta * tb)));
  // any product a x b with a <= cap, b <= k uses at most max(chunks * cap * k, 304 * 64 * 64) partials
  const int gs_chunks = std::max(1, ceil_div(ctx->max_group_rows, 128));
  ctx->gram_part.ensure(std::max<size_t>(std::max<size_t>((size_t)(chunks + 1) * cap * k, (size_t)304 * 64 * 64),
                                         (size_t)gs_chunks * cap * k));
  ctx->tu_part.ensure(std::max(tall_update_scratch(nl, (int)cap, k, true), tall_update_scratch(nl, (int)cap, k, false)));
  tall_update_init();
  {
    const int tiles = ceil_div(nl, 64);
    if (ctx->tu_tickets.n < (size_t)tiles) {
      ctx->tu_tickets.alloc(tiles);
      FETIRP_CUDA(cudaMemsetAsync(ctx->tu_tickets.p, 0, sizeof(unsigned) * tiles, ctx->stream));
    }
  }
  const void* after[5] = {ctx->C.p, ctx->gram_part.p, ctx->Whist32.p, ctx->tu_part.p, ctx->tu_tickets.p};
  if (ctx->gc.exec && std::memcmp(before, after, sizeof(before)) != 0) {
    cudaGraphExecDestroy(ctx->gc.exec);
    ctx->gc.exec = nullptr;
  }
}

// A bounded wait inside the tensor-core kernel that expired leaves a nonzero code in tc_error.
void check_tc_error(fetirp_ctx ctx) {
  if (!ctx->tc_error.p) return;
  int code = 0;
  FETIRP_CUDA(cudaMemcpyAsync(&code, ctx->tc_error.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
  if (code != 0) {
    ctx->tc_error.zero(ctx->stream);
    throw Error(FETIRP_ETIMEOUT, "tensor-core pipeline wait expired (code " + std::to_string(code) + ")");
  }
}

fetirp_status run_solve(fetirp_ctx ctx, double* d_lambda, double* d_u, fetirp_stats* stats) {
  cudaStream_t s = ctx->stream;
  const int nl = ctx->L.n_lambda;
  fetirp_stats st{};
  st.kernel_dim_total = ctx->n_G;
  const unsigned long long l0 = g_launch_count;
  int prec = ctx->opt.precision;
  if (prec == FETIRP_PREC_AUTO) {   // latency-bound structures: FP32 SIMT products (persistent); else tf32x3
    int max_nb = 0;
    for (size_t p = 0; p < ctx->pats.size(); ++p)
      if (!ctx->use[p].occs.empty()) max_nb = std::max(max_nb, ctx->pats[p]->n_b);
    prec = (max_nb <= 512 && nl <= 262144) ? FETIRP_PREC_FP32 : FETIRP_PREC_TF32X3;
  }
  // operators formed on first use count as set-up (factorisation phase), not as solve time
  ensure_operators(ctx, prec);
  cudaEvent_t e0, e1;
  FETIRP_CUDA(cudaEventCreate(&e0));
  FETIRP_CUDA(cudaEventCreate(&e1));
  FETIRP_CUDA(cudaEventRecord(e0, s));
  ensure_history(ctx);
  FETIRP_CUDA(cudaMemcpyAsync(ctx->lam.p, ctx->lambda0.p, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
  residual(ctx);
  const double r0 = norm2(ctx, ctx->r.p, nl);
  double rn = r0;
  // independent sub-structures (fetirp_set_row_blocks): stop when ||r|| <= tol * min_b ||r0_b||, so that every
  // block meets the relative tolerance on its own (||r_b|| <= ||r||); the reported residual is the worst block's
  double r0_ref = r0;
  std::vector<double> r0_blk;
  if (ctx->row_blocks.size() > 2) {
    std::vector<double> h(nl);
    FETIRP_CUDA(cudaMemcpyAsync(h.data(), ctx->r.p, sizeof(double) * nl, cudaMemcpyDeviceToHost, s));
    FETIRP_CUDA(cudaStreamSynchronize(s));
    for (size_t b = 0; b + 1 < ctx->row_blocks.size(); ++b) {
      double acc = 0.0;
      for (int64_t i = ctx->row_blocks[b]; i < ctx->row_blocks[b + 1]; ++i) acc += h[i] * h[i];
      r0_blk.push_back(std::sqrt(acc));
      if (r0_blk.back() > 0.0) r0_ref = std::min(r0_ref, r0_blk.back());
    }
  }
  const double target = ctx->opt.tol * r0_ref;
  int budget = ctx->opt.max_iter;
  Hist H;
  // relative tolerance of every inner solve: the user's, or (0) one above the operator's rounding level
  const double inner_tol = ctx->opt.inner_tol > 0.0   ? ctx->opt.inner_tol
                           : prec == FETIRP_PREC_BF16X3 ? 1e-4
                           : prec == FETIRP_PREC_TF32X3 ? 1e-5
                                                        : 1e-6;
  if (r0 > 0.0) {
    if (prec == FETIRP_PREC_FP64) {
      rn = block_orthodir<double>(ctx, FETIRP_PREC_FP64, target, rn, H, st, budget);
      residual(ctx);   // report the FP64 residual of the final iterate
      rn = norm2(ctx, ctx->r.p, nl);
    } else {
      // outer FP64 defect correction: inner solves on the low-precision operator reuse their directions
      for (int outer = 0; outer < ctx->opt.max_outer && rn > target && budget > 0; ++outer) {
        const double inner_target = std::max(inner_tol * rn, 0.5 * target);
        if (hist_fp64(ctx)) block_orthodir<double>(ctx, prec, inner_target, rn, H, st, budget);
        else block_orthodir<float>(ctx, prec, inner_target, rn, H, st, budget);
        if (H.stalled) {   // the stored directions no longer serve the next inner solve
          H.cols = 0;
          H.stalled = false;
        }
        reproject_lambda(ctx);
        residual(ctx);
        rn = norm2(ctx, ctx->r.p, nl);
        st.outer_steps++;
      }
    }
  }
  st.rel_residual = r0 > 0.0 ? rn / r0 : 0.0;
  if (!r0_blk.empty() && r0 > 0.0) {   // the worst block's own relative residual
    std::vector<double> h(nl);
    FETIRP_CUDA(cudaMemcpyAsync(h.data(), ctx->r.p, sizeof(double) * nl, cudaMemcpyDeviceToHost, s));
    FETIRP_CUDA(cudaStreamSynchronize(s));
    double worst = 0.0;
    for (size_t b = 0; b < r0_blk.size(); ++b) {
      double acc = 0.0;
      for (int64_t i = ctx->row_blocks[b]; i < ctx->row_blocks[b + 1]; ++i) acc += h[i] * h[i];
      if (r0_blk[b] > 0.0) worst = std::max(worst, std::sqrt(acc) / r0_blk[b]);
    }
    st.rel_residual = worst;
  }
  st.f_applies = st.iterations;   // one block F-apply per block iteration
  check_tc_error(ctx);
  if (d_lambda)
    FETIRP_CUDA(cudaMemcpyAsync(d_lambda, ctx->lam.p, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
  if (d_u) recover(ctx, d_u, ctx->t1.p);   // t1 = d - F lambda from the last residual() above
  FETIRP_CUDA(cudaEventRecord(e1, s));
  FETIRP_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  FETIRP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  st.solve_ms = ms;
  st.setup_ms = ctx->last.setup_ms;
  st.launches = (int64_t)(g_launch_count - l0) + ctx->last.launches;
  collect_phases(ctx, st);
  ctx->last = st;
  if (stats) *stats = st;
  if (!(st.rel_residual <= ctx->opt.tol)) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "tolerance not reached: relative residual %.3e after %d iterations, %d outer steps",
                  st.rel_residual, st.iterations, st.outer_steps);
    set_err(ctx, buf);
    return FETIRP_ENOCONV;
  }
  return FETIRP_OK;
}

// Resets the per-phase accounting (unless keep_phases: a factorisation just ran and belongs to the call).
void prepare_timed(fetirp_ctx ctx, int64_t n_lambda, const double* c_host, const double* c_dev,
                   bool keep_phases = false) {
  if (!keep_phases && !ctx->phases_pending) reset_phases(ctx);
  ctx->phases_pending = false;
  const unsigned long long l0 = g_launch_count;
  auto t0 = std::chrono::steady_clock::now();
  build_structure(ctx, n_lambda, c_host, c_dev);
  ctx->last.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  ctx->last.launches = (int64_t)(g_launch_count - l0) + ctx->pending_launches;
  ctx->pending_launches = 0;
}

}  // namespace

// ------------------------------------------------------------------------------ allocation-free apply
// Scratch of fetirp_apply_block_device_noalloc: a fixed array in the library's device image.  Host code only
// ever uses the device address returned by cudaGetSymbolAddress (the name itself is a host-side stand-in).
static __device__ __align__(256) unsigned char g_noalloc_scratch[FETIRP_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_addr[64] = {};

// Device address of the scratch array on the current device (looked up once per device).
unsigned char* noalloc_scratch(int device) {
  if (device < 0 || device >= 64) throw Error(FETIRP_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    FETIRP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[device] = static_cast<unsigned char*>(p);
  }
  return g_noalloc_addr[device];
}

// P V with caller-provided coarse vectors (the context's structure scratch of G^T V and of the coarse product,
// allocated when the structure was built, is used; nothing is allocated here).
void project_with(fetirp_ctx ctx, double* V, int k, double* Xc, double* Ac) {
  if (ctx->n_G == 0) return;
  gt_v(ctx->L, V, k, Xc, ctx->stream);
  small_gemm(ctx->n_G, k, ctx->Ginv.p, Xc, Ac, ctx->stream, ctx->sg_part.p);
  g_apply(ctx->L, Ac, k, -1.0, 1.0, V, ctx->stream);
}

// Q = P^T F P V with every scratch buffer carved from `base` (size `cap` bytes); throws FETIRP_EINVAL when
// the call needs more.
void apply_noalloc(fetirp_ctx ctx, const double* V, double* Q, int k, int prec, unsigned char* base, size_t cap) {
  cudaStream_t s = ctx->stream;
  const Layout& L = ctx->L;
  const int n_pat = (int)ctx->pats.size();
  const size_t es = prec == FETIRP_PREC_FP64 ? sizeof(double) : sizeof(float);
  long long pbase[MAXP] = {};
  long long total = 0;
  for (int p = 0; p < n_pat; ++p) {
    pbase[p] = total;
    total += (long long)ctx->use[p].occs.size() * k * ctx->pats[p]->ld_y;
  }
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t nv = up(sizeof(double) * (size_t)L.n_lambda * k);
  const size_t nc = up(sizeof(double) * (size_t)std::max(ctx->n_G, 1) * k);
  const size_t ny = up(es * (size_t)total);
  const size_t need = nv + 2 * nc + (prec == FETIRP_PREC_TF32X3 ? 3 : 2) * ny;
  if (need > cap)
    throw Error(FETIRP_EINVAL, "fetirp_apply_block_device_noalloc needs " + std::to_string(need) +
                                   " bytes of scratch, more than its fixed " + std::to_string(cap) + " bytes");
  unsigned char* q = base;
  double* V2 = reinterpret_cast<double*>(q); q += nv;
  double* Xc = reinterpret_cast<double*>(q); q += nc;
  double* Ac = reinterpret_cast<double*>(q); q += nc;
  unsigned char* Yb = q; q += ny;
  unsigned char* Zb = q; q += ny;
  unsigned char* Ylb = q;
  FETIRP_CUDA(cudaMemcpyAsync(V2, V, sizeof(double) * (size_t)L.n_lambda * k, cudaMemcpyDeviceToDevice, s));
  project_with(ctx, V2, k, Xc, Ac);
  LocalProblem LP{};
  LP.n_pat = n_pat;
  if (prec == FETIRP_PREC_FP64 || prec == FETIRP_PREC_FP32) {
    PatView<double> Yd{}, Zd{};
    PatView<float> Yf{}, Zf{};
    for (int p = 0; p < n_pat; ++p) {
      PatternData& P = *ctx->pats[p];
      void* y = Yb + pbase[p] * es;
      void* z = Zb + pbase[p] * es;
      Yd.base[p] = (double*)y; Zd.base[p] = (double*)z;
      Yf.base[p] = (float*)y; Zf.base[p] = (float*)z;
      Yd.ld[p] = Zd.ld[p] = Yf.ld[p] = Zf.ld[p] = P.ld_y;
      LP.S[p] = prec == FETIRP_PREC_FP64 ? (const void*)P.S64.p : (const void*)P.S32.p;
      LP.n_b[p] = P.n_b; LP.n_rhs[p] = (int)ctx->use[p].occs.size() * k; LP.ld[p] = P.ld_y;
      LP.Y[p] = y; LP.Z[p] = z;
    }
    if (prec == FETIRP_PREC_FP64) {
      gather<double>(L, V2, k, Yd, s);
      rotate_traces<double>(L, Yd, k, true, s);
      local_gemm_f64(LP, s);
      rotate_traces<double>(L, Zd, k, false, s);
      scatter<double>(L, Zd, k, 0.0, Q, s);
    } else {
      gather<float>(L, V2, k, Yf, s);
      rotate_traces<float>(L, Yf, k, true, s);
      local_gemm_f32(LP, s);
      rotate_traces<float>(L, Zf, k, false, s);
      scatter<float>(L, Zf, k, 0.0, Q, s);
    }
  } else {
    PatView<float> Yh{}, Yl{}, Zv{};
    TcProblem T;
    T.n_pat = n_pat;
    T.part = ctx->tc_part.p;
    T.part_elems = (long long)ctx->tc_part.n;
    for (int p = 0; p < n_pat; ++p) {
      PatternData& P = *ctx->pats[p];
      Yh.base[p] = (float*)(Yb + pbase[p] * es);
      Yl.base[p] = (float*)(Ylb + pbase[p] * es);
      Zv.base[p] = (float*)(Zb + pbase[p] * es);
      Yh.ld[p] = Yl.ld[p] = Zv.ld[p] = P.ld_y;
      T.S_hi[p] = P.S_hi.p; T.S_lo[p] = P.S_lo.p; T.lds[p] = P.lds;
      T.Y_hi[p] = Yh.base[p]; T.Y_lo[p] = Yl.base[p]; T.Z[p] = Zv.base[p]; T.ldy[p] = P.ld_y;
      T.n_b[p] = P.n_b; T.n_rhs[p] = (int)ctx->use[p].occs.size() * k;
    }
    gather_split(L, V2, k, Yh, Yl, s);
    rotate_split(L, Yh, Yl, k, s);
    tc_gemm_tf32x3(T, ctx->tc_error.p, s);
    rotate_traces<float>(L, Zv, k, false, s);
    scatter<float>(L, Zv, k, 0.0, Q, s);
  }
  project_with(ctx, Q, k, Xc, Ac);
}

}  // namespace

// =========================================================================================== C ABI
extern "C" {

fetirp_status fetirp_apply_block_device_noalloc(fetirp_ctx ctx, int32_t k, const double* d_V, double* d_Q,
                                                int32_t precision) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (!ctx->prepared) throw Error(FETIRP_ESTATE, "call fetirp_prepare or fetirp_solve first");
    REQUIRE(k >= 1 && k <= 64, "k must be in 1..64");
    REQUIRE(d_V && d_Q, "NULL buffer");
    REQUIRE(precision >= FETIRP_PREC_FP64 && precision <= FETIRP_PREC_TF32X3, "unsupported precision");
    ensure_operators(ctx, precision);
    apply_noalloc(ctx, d_V, d_Q, k, precision, noalloc_scratch(ctx->opt.device), FETIRP_NOALLOC_SCRATCH_BYTES);
    return FETIRP_OK;
  });
}


void fetirp_default_options(fetirp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = FETIRP_PREC_FP64;
  o->tol = 1e-8;
  o->max_iter = 2000;
  o->block_k = 32;
  o->max_outer = 30;
  o->inner_tol = 0.0;
  o->pivot_tol = 1e-9;
  o->eig_trunc = 1e-12;
  o->cuda_stream = nullptr;
  o->device = 0;
  o->check_every = 4;
  o->timing = 0;
  o->eig_trunc_inner = 1e-6;
  o->use_graphs = 1;
  o->timing_mask = 0;
  o->history_bytes = 0;
  o->persistent = 1;
}

const char* fetirp_status_string(fetirp_status s) {
  switch (s) {
    case FETIRP_OK: return "FETIRP_OK";
    case FETIRP_EINVAL: return "FETIRP_EINVAL";
    case FETIRP_ENOMEM: return "FETIRP_ENOMEM";
    case FETIRP_ESINGULAR: return "FETIRP_ESINGULAR";
    case FETIRP_ENOCONV: return "FETIRP_ENOCONV";
    case FETIRP_ECUDA: return "FETIRP_ECUDA";
    case FETIRP_ESTATE: return "FETIRP_ESTATE";
    case FETIRP_ETIMEOUT: return "FETIRP_ETIMEOUT";
  }
  return "unknown status";
}

fetirp_status fetirp_create(const fetirp_options* opt, fetirp_ctx* out) {
  if (!out) return FETIRP_EINVAL;
  *out = nullptr;
  std::unique_ptr<fetirp_ctx_s> ctx(new (std::nothrow) fetirp_ctx_s());
  if (!ctx) return FETIRP_ENOMEM;
  if (opt) ctx->opt = *opt;
  else fetirp_default_options(&ctx->opt);
  const fetirp_options& o = ctx->opt;
  if (!(o.tol > 0) || o.max_iter < 1 || o.block_k < 1 || o.max_outer < 1 || !(o.inner_tol >= 0) ||
      !(o.pivot_tol > 0) || !(o.eig_trunc > 0) || !(o.eig_trunc_inner > 0) || o.check_every < 0 ||
      !(operator_precision(o.precision) || o.precision == FETIRP_PREC_AUTO) ||
      ((o.alloc == nullptr) != (o.free == nullptr)))
    return FETIRP_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) return FETIRP_ECUDA;
  if (cudaSetDevice(o.device) != cudaSuccess) return FETIRP_ECUDA;
  ctx->stream = (cudaStream_t)o.cuda_stream;
  if (!ctx->stream) {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return FETIRP_ECUDA;
    ctx->owns_stream = true;
  }
  if (cudaMallocHost(&ctx->h_state, 8 * sizeof(int)) != cudaSuccess) return FETIRP_ENOMEM;
  if (cudaMallocHost(&ctx->h_rr, 1024 * sizeof(double)) != cudaSuccess) return FETIRP_ENOMEM;
  *out = ctx.release();
  return FETIRP_OK;
}

fetirp_status fetirp_create_child(fetirp_ctx parent, const fetirp_options* opt, fetirp_ctx* out) {
  if (!parent || !out) return FETIRP_EINVAL;
  fetirp_options o = opt ? *opt : parent->opt;
  o.device = parent->opt.device;
  fetirp_status st = fetirp_create(&o, out);
  if (st != FETIRP_OK) return st;
  (*out)->pats = parent->pats;   // shared, read-only factors
  (*out)->is_child = true;
  return FETIRP_OK;
}

const char* fetirp_last_error(fetirp_ctx ctx) { return ctx ? ctx->err.c_str() : "invalid context"; }

void fetirp_destroy(fetirp_ctx ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->opt.device);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

fetirp_status fetirp_create_pattern(fetirp_ctx ctx, int32_t n_nodes, int32_t dpn, const int64_t* rowptr,
                                    const int32_t* col, const double* val, int32_t n_bnd, const int32_t* bnd_nodes,
                                    int32_t expected_kernel_dim, int32_t* pattern_id) {
  return guarded(ctx, [&]() -> fetirp_status {
    REQUIRE(n_nodes > 0 && dpn >= 1 && dpn <= 3, "n_nodes must be > 0 and dofs_per_node in 1..3");
    REQUIRE(rowptr && col && val && bnd_nodes && pattern_id, "NULL argument");
    REQUIRE((long long)n_nodes * dpn < (1LL << 30), "pattern too large");
    REQUIRE(n_bnd > 0 && n_bnd <= n_nodes, "n_bnd out of range");
    REQUIRE(expected_kernel_dim >= -1, "expected_kernel_dim must be >= -1");
    if ((int)ctx->pats.size() >= MAXP) throw Error(FETIRP_EINVAL, "at most 16 patterns per context");
    if (ctx->is_child) throw Error(FETIRP_ESTATE, "patterns are added to the library context, not to a child");
    auto P = std::make_shared<PatternData>();
    P->n_nodes = n_nodes; P->dpn = dpn; P->n = n_nodes * dpn; P->expected = expected_kernel_dim;
    const int n = P->n;
    REQUIRE(rowptr[0] == 0, "rowptr[0] must be 0");
    for (int i = 0; i < n; ++i) REQUIRE(rowptr[i + 1] >= rowptr[i], "rowptr must be non-decreasing");
    const int64_t nnz = rowptr[n];
    P->rowptr.assign(rowptr, rowptr + n + 1);
    P->col.assign(col, col + nnz);
    P->val.assign(val, val + nnz);
    for (int64_t e = 0; e < nnz; ++e) {
      REQUIRE(col[e] >= 0 && col[e] < n, "column index out of range");
      REQUIRE(std::isfinite(val[e]), "non-finite stiffness value");
    }
    P->bpos.assign(n_nodes, -1);
    for (int b = 0; b < n_bnd; ++b) {
      REQUIRE(bnd_nodes[b] >= 0 && bnd_nodes[b] < n_nodes, "boundary node out of range");
      REQUIRE(P->bpos[bnd_nodes[b]] < 0, "duplicate boundary node");
      P->bpos[bnd_nodes[b]] = b;
    }
    P->bnd_nodes.assign(bnd_nodes, bnd_nodes + n_bnd);
    P->n_b = n_bnd * dpn;
    P->n_i = n - P->n_b;
    P->newidx.assign(n, -1);
    P->oldidx.assign(n, -1);
    int next = 0;
    for (int node = 0; node < n_nodes; ++node)
      if (P->bpos[node] < 0)
        for (int c = 0; c < dpn; ++c) { P->newidx[node * dpn + c] = next; P->oldidx[next] = node * dpn + c; ++next; }
    for (int b = 0; b < n_bnd; ++b)
      for (int c = 0; c < dpn; ++c) {
        const int old = bnd_nodes[b] * dpn + c;
        P->newidx[old] = next; P->oldidx[next] = old; ++next;
      }
    P->npad = (int)round_up(n, TILE);
    P->ld_y = round_up(P->n_b, 4);
    P->nbpad = (int)round_up(P->n_b, TILE);
    const int nt = P->npad / TILE;
    std::vector<uint8_t> nz((size_t)nt * nt, 0);
    for (int i = 0; i < n; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        int a = P->newidx[i] / TILE, b = P->newidx[col[e]] / TILE;
        nz[(size_t)std::max(a, b) * nt + std::min(a, b)] = 1;
      }
    P->plan.build(nt, nz);
    P->plan.upload(ctx->stream);
    P->planS = dense_plan(P->nbpad / TILE);
    P->planS.upload(ctx->stream);
    P->d_rowptr.upload(P->rowptr, ctx->stream);
    P->d_col.upload(P->col, ctx->stream);
    P->d_val.upload(P->val, ctx->stream);
    P->d_newidx.upload(P->newidx, ctx->stream);
    factorize_patterns(ctx, {P.get()});
    *pattern_id = (int)ctx->pats.size();
    ctx->pats.push_back(P);
    invalidate(ctx);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_add_occurrence(fetirp_ctx ctx, int32_t pattern_id, const double* rot, int32_t n_links,
                                    const int32_t* local_node, const int8_t* global_comp, const int32_t* lambda_row,
                                    const int8_t* sign, const double* f_global, int32_t* occ_id) {
  return guarded(ctx, [&]() -> fetirp_status {
    REQUIRE(pattern_id >= 0 && pattern_id < (int)ctx->pats.size(), "unknown pattern id");
    REQUIRE(n_links >= 0, "n_links < 0");
    REQUIRE(occ_id && f_global, "NULL argument");
    REQUIRE(n_links == 0 || (local_node && global_comp && lambda_row && sign), "NULL link array");
    const PatternData& P = *ctx->pats[pattern_id];
    OccData O;
    O.pattern = pattern_id;
    if (rot) {   // a proper rotation: finite, R R^T = I and det R = +1 (to 1e-12)
      for (int i = 0; i < 9; ++i) REQUIRE(std::isfinite(rot[i]), "non-finite rotation entry");
      double dev = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double d = a == b ? -1.0 : 0.0;
          for (int c = 0; c < 3; ++c) d += rot[3 * a + c] * rot[3 * b + c];
          dev = std::max(dev, std::fabs(d));
        }
      const double detr = rot[0] * (rot[4] * rot[8] - rot[5] * rot[7]) - rot[1] * (rot[3] * rot[8] - rot[5] * rot[6]) +
                          rot[2] * (rot[3] * rot[7] - rot[4] * rot[6]);
      REQUIRE(dev <= 1e-12 && std::fabs(detr - 1.0) <= 1e-12,
              "rot must be a proper rotation (R R^T = I and det R = +1 to 1e-12)");
    }
    if (rot && P.dpn > 1) {   // one dof per node: the rotation only places the pattern, no component turns
      for (int c = 0; c < P.dpn; ++c)
        for (int c2 = P.dpn; c2 < 3; ++c2)
          REQUIRE(std::fabs(rot[3 * c + c2]) <= 1e-12 && std::fabs(rot[3 * c2 + c]) <= 1e-12,
                  "rotation mixes a modelled component with an absent one");
      bool perm = true;   // a signed permutation (the rotations of the cube): folded into the links
      for (int r = 0; r < P.dpn; ++r) {
        int nzc = 0;
        for (int c = 0; c < P.dpn; ++c) {
          const double v = rot[3 * r + c];
          if (v != 0.0 && v != 1.0 && v != -1.0) perm = false;
          if (v != 0.0) ++nzc;
        }
        if (nzc != 1) perm = false;
      }
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          const bool modelled = r < P.dpn && c < P.dpn;
          O.Rd[3 * r + c] = modelled ? rot[3 * r + c] : (r == c ? 1.0 : 0.0);
          O.R[3 * r + c] = perm ? (int)O.Rd[3 * r + c] : (r == c ? 1 : 0);
        }
      O.general = !perm;
    }
    O.link_j.resize(n_links);
    O.link_row.resize(n_links);
    O.link_sign.resize(n_links);
    for (int i = 0; i < n_links; ++i) {
      REQUIRE(local_node[i] >= 0 && local_node[i] < P.n_nodes, "link node out of range");
      REQUIRE(P.bpos[local_node[i]] >= 0, "link on a node that is not a boundary node of the pattern");
      REQUIRE(global_comp[i] >= 0 && global_comp[i] < P.dpn, "link component out of range");
      REQUIRE(sign[i] == 1 || sign[i] == -1, "link sign must be +1 or -1");
      REQUIRE(lambda_row[i] >= 0, "negative lambda_row");
      const int c = global_comp[i];
      int c2 = c, rs = 1;   // general rotation: the slot holds the global component, turned on the device
      if (P.dpn > 1 && !O.general)
        for (int cc = 0; cc < P.dpn; ++cc)
          if (O.R[3 * c + cc] != 0) { c2 = cc; rs = O.R[3 * c + cc]; }
      O.link_j[i] = P.bpos[local_node[i]] * P.dpn + c2;
      O.link_row[i] = lambda_row[i];
      O.link_sign[i] = (int8_t)(sign[i] * rs);
    }
    // f in the pattern frame: f_l = R^T f_g per node
    O.f_local.assign(P.n, 0.0);
    for (int node = 0; node < P.n_nodes; ++node)
      for (int c2 = 0; c2 < P.dpn; ++c2) {
        double v = 0.0;
        for (int c = 0; c < P.dpn; ++c) {
          const double fg = f_global[node * P.dpn + c];
          REQUIRE(std::isfinite(fg), "non-finite load");
          v += (P.dpn > 1 ? O.Rd[3 * c + c2] : (c == c2 ? 1.0 : 0.0)) * fg;
        }
        O.f_local[node * P.dpn + c2] = v;
      }
    *occ_id = (int)ctx->occs.size();
    ctx->occs.push_back(std::move(O));
    invalidate(ctx);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_clear_occurrences(fetirp_ctx ctx) {
  return guarded(ctx, [&]() -> fetirp_status {
    ctx->occs.clear();
    ctx->row_blocks.clear();
    ctx->k_user = 0;
    ctx->groups_user.clear();
    ctx->perm.on = false;
    invalidate(ctx);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_set_groups(fetirp_ctx ctx, int32_t k, const int32_t* group_of_occ) {
  return guarded(ctx, [&]() -> fetirp_status {
    REQUIRE(k >= 1 && k <= 64, "k must be in 1..64");
    REQUIRE(group_of_occ, "NULL groups");
    const int n = (int)ctx->occs.size();
    for (int o = 0; o < n; ++o) REQUIRE(group_of_occ[o] >= 0 && group_of_occ[o] < k, "group id out of range");
    ctx->k_user = k;
    ctx->groups_user.assign(group_of_occ, group_of_occ + n);
    ctx->perm.on = false;
    invalidate(ctx);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_prepare(fetirp_ctx ctx, int64_t n_lambda, const double* c) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (c)
      for (int64_t i = 0; i < n_lambda; ++i) REQUIRE(std::isfinite(c[i]), "non-finite c");
    prepare_timed(ctx, n_lambda, c, nullptr);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_solve(fetirp_ctx ctx, int64_t n_lambda, const double* c, double* lambda_out, double* u_out,
                           fetirp_stats* stats) {
  return guarded(ctx, [&]() -> fetirp_status {
    REQUIRE(lambda_out && u_out, "NULL output");
    if (c)
      for (int64_t i = 0; i < n_lambda; ++i) REQUIRE(std::isfinite(c[i]), "non-finite c");
    prepare_timed(ctx, n_lambda, c, nullptr);
    DBuf<double> dl(n_lambda), du(ctx->n_u);
    fetirp_status st = run_solve(ctx, dl.p, du.p, stats);
    FETIRP_CUDA(cudaMemcpyAsync(lambda_out, dl.p, sizeof(double) * n_lambda, cudaMemcpyDeviceToHost, ctx->stream));
    FETIRP_CUDA(cudaMemcpyAsync(u_out, du.p, sizeof(double) * ctx->n_u, cudaMemcpyDeviceToHost, ctx->stream));
    FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
    return st;
  });
}

fetirp_status fetirp_autotune_k(fetirp_ctx ctx, int64_t n_lambda, const double* c, int32_t n_cand,
                                const int32_t* candidates, int32_t* best_k, double* times_ms) {
  return guarded(ctx, [&]() -> fetirp_status {
    REQUIRE(n_cand >= 1 && candidates && best_k, "bad candidate list");
    const int n_occ = (int)ctx->occs.size();
    if (n_occ == 0) throw Error(FETIRP_ESTATE, "no occurrence has been added");
    double best = 1e300;
    int bk = -1;
    std::vector<int> g(n_occ);
    for (int i = 0; i < n_cand; ++i) {
      const int k = std::max(1, std::min(candidates[i], std::min(64, n_occ)));
      REQUIRE(candidates[i] >= 1 && candidates[i] <= 64, "candidate k out of 1..64");
      for (int o = 0; o < n_occ; ++o) g[o] = (int)((long long)o * k / n_occ);
      ctx->k_user = k;
      ctx->groups_user = g;
      invalidate(ctx);
      prepare_timed(ctx, n_lambda, c, nullptr);
      DBuf<double> dl(n_lambda), du(ctx->n_u);
      fetirp_stats st{};
      const fetirp_status rs = run_solve(ctx, dl.p, du.p, &st);
      const double t = rs == FETIRP_OK ? st.solve_ms : 1e300;
      if (times_ms) times_ms[i] = rs == FETIRP_OK ? t : INFINITY;
      if (t < best) { best = t; bk = k; }
    }
    if (bk < 0) throw Error(FETIRP_ENOCONV, "no candidate k reached the tolerance");
    for (int o = 0; o < n_occ; ++o) g[o] = (int)((long long)o * bk / n_occ);
    ctx->k_user = bk;
    ctx->groups_user = g;
    invalidate(ctx);
    *best_k = bk;
    return FETIRP_OK;
  });
}

fetirp_status fetirp_solve_device(fetirp_ctx ctx, int64_t n_lambda, const double* d_c, double* d_lambda,
                                  double* d_u, fetirp_stats* stats) {
  return guarded(ctx, [&]() -> fetirp_status {
    REQUIRE(d_lambda && d_u, "NULL output");
    prepare_timed(ctx, n_lambda, nullptr, d_c);
    return run_solve(ctx, d_lambda, d_u, stats);
  });
}

fetirp_status fetirp_apply_block_device(fetirp_ctx ctx, int32_t k, const double* d_V, double* d_Q, int32_t precision) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (!ctx->prepared) throw Error(FETIRP_ESTATE, "call fetirp_prepare or fetirp_solve first");
    REQUIRE(k >= 1 && k <= 64, "k must be in 1..64");
    REQUIRE(d_V && d_Q, "NULL buffer");
    REQUIRE(operator_precision(precision), "unsupported precision");
    ensure_operators(ctx, precision);
    apply_F(ctx, d_V, d_Q, k, precision, true, true);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_apply_block(fetirp_ctx ctx, int32_t k, const double* V, double* Q, int32_t precision) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (!ctx->prepared) throw Error(FETIRP_ESTATE, "call fetirp_prepare or fetirp_solve first");
    REQUIRE(k >= 1 && k <= 64, "k must be in 1..64");
    REQUIRE(V && Q, "NULL buffer");
    REQUIRE(operator_precision(precision), "unsupported precision");
    const size_t n = (size_t)ctx->L.n_lambda * k;
    DBuf<double> dv(n), dq(n);
    ensure_operators(ctx, precision);
    dv.upload(V, n, ctx->stream);
    apply_F(ctx, dv.p, dq.p, k, precision, true, true);
    check_tc_error(ctx);
    FETIRP_CUDA(cudaMemcpyAsync(Q, dq.p, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
    return FETIRP_OK;
  });
}

}  // extern "C" (reopened below)

namespace {

// Pairs, local coarse responses and buffers of the sparse-column form (host tables from the links).
void split_plan_build(fetirp_ctx ctx) {
  cudaStream_t s = ctx->stream;
  SplitPlan& SP = ctx->sp;
  const Layout& L = ctx->L;
  if (L.n_gen > 0)
    throw Error(FETIRP_EINVAL, "the sparse-column form takes rotations of vector fields in 90-degree steps only");
  if (ctx->perm.on) throw Error(FETIRP_EINVAL, "the sparse-column form needs the occurrence split, not a permutation");
  const int n_occ = L.n_occ, k = ctx->k, n_pat = (int)ctx->pats.size(), nl = L.n_lambda;
  std::vector<int> obase(n_occ + 1, 0), occ_pat(n_occ), occ_gofs(n_occ);
  for (int p = 0; p < n_pat; ++p)
    for (size_t q = 0; q < ctx->use[p].occs.size(); ++q) occ_pat[ctx->use[p].occs[q]] = p;
  for (int o = 0; o < n_occ; ++o) {
    obase[o + 1] = obase[o] + ctx->pats[occ_pat[o]]->n_b;
    occ_gofs[o] = ctx->pofs[occ_pat[o]] + 0;
  }
  for (int p = 0; p < n_pat; ++p)
    for (size_t q = 0; q < ctx->use[p].occs.size(); ++q)
      occ_gofs[ctx->use[p].occs[q]] = ctx->pofs[p] + (int)q * ctx->pats[p]->kdim;
  // owners of every row: (occurrence, boundary dof, sign)
  struct Own { int o, j, sg; };
  std::vector<std::array<Own, 2>> own(nl);
  std::vector<int> nown(nl, 0);
  for (int o = 0; o < n_occ; ++o) {
    const OccData& O = ctx->occs[o];
    for (size_t i = 0; i < O.link_row.size(); ++i) {
      const int r = O.link_row[i];
      own[r][nown[r]++] = Own{o, O.link_j[i], O.link_sign[i]};
    }
  }
  std::vector<std::vector<int>> nbr(n_occ);
  for (int r = 0; r < nl; ++r)
    if (nown[r] == 2) {
      nbr[own[r][0].o].push_back(own[r][1].o);
      nbr[own[r][1].o].push_back(own[r][0].o);
    }
  for (auto& v : nbr) { std::sort(v.begin(), v.end()); v.erase(std::unique(v.begin(), v.end()), v.end()); }
  // pairs, pattern by pattern in local-product column order
  std::vector<int> pair_occ, pair_g, pair_of((size_t)n_occ * k, -1);
  for (int p = 0; p < n_pat; ++p) {
    SP.pair_off[p] = (int)pair_occ.size();
    for (int o : ctx->use[p].occs) {
      std::vector<int> gs{ctx->h_group[o]};
      for (int t : nbr[o]) gs.push_back(ctx->h_group[t]);
      std::sort(gs.begin(), gs.end());
      gs.erase(std::unique(gs.begin(), gs.end()), gs.end());
      for (int g : gs) {
        pair_of[(size_t)o * k + g] = (int)pair_occ.size() - SP.pair_off[p];
        pair_occ.push_back(o);
        pair_g.push_back(g);
      }
    }
  }
  SP.pair_off[n_pat] = (int)pair_occ.size();
  SP.n_pairs = (int)pair_occ.size();
  SP.ytotal = 0;
  for (int p = 0; p < n_pat; ++p) {
    SP.ybase[p] = SP.ytotal;
    SP.ytotal += (long long)(SP.pair_off[p + 1] - SP.pair_off[p]) * ctx->pats[p]->ld_y;
  }
  // E_s = B(s)^T G over the kernel modes of s and its neighbours; M = S E per pattern (FP64 products)
  std::vector<std::vector<double>> hNb(n_pat);
  for (int p = 0; p < n_pat; ++p) {
    const PatternData& P = *ctx->pats[p];
    hNb[p].resize((size_t)P.n_b * P.kdim);
    if (P.kdim > 0)
      FETIRP_CUDA(cudaMemcpyAsync(hNb[p].data(), P.Nb.p, sizeof(double) * hNb[p].size(), cudaMemcpyDeviceToHost, s));
  }
  FETIRP_CUDA(cudaStreamSynchronize(s));
  std::vector<int> mcol_ptr(n_occ + 1, 0), mcol_row;
  std::vector<long long> moff(n_occ, 0), mld(fetirp::MAXP, 1), mbase(n_pat + 1, 0);
  std::vector<std::vector<double>> E(n_pat);
  std::vector<int> mcols(n_pat, 0);
  for (int p = 0; p < n_pat; ++p) {
    const long long ld = ctx->pats[p]->ld_y;
    mld[p] = ld;
    for (int o : ctx->use[p].occs) {
      std::vector<int> us{o};
      for (int t : nbr[o]) us.push_back(t);
      std::sort(us.begin(), us.end());
      std::vector<int> col0(us.size());
      int nc = 0;
      for (size_t i = 0; i < us.size(); ++i) { col0[i] = nc; nc += ctx->pats[occ_pat[us[i]]]->kdim; }
      if (nc > 48) throw Error(FETIRP_EINVAL, "sparse-column form: more than 48 coarse columns touch one occurrence");
      moff[o] = (long long)mcols[p];   // columns before o within pattern p (made absolute below)
      mcols[p] += nc;
      const size_t base = E[p].size();
      E[p].resize(base + (size_t)nc * ld, 0.0);
      const OccData& O = ctx->occs[o];
      for (size_t i = 0; i < O.link_row.size(); ++i) {
        const int r = O.link_row[i], j = O.link_j[i], sgo = O.link_sign[i];
        for (int e = 0; e < nown[r]; ++e) {
          const Own& w = own[r][e];
          const size_t ui = std::lower_bound(us.begin(), us.end(), w.o) - us.begin();
          const int kd = ctx->pats[occ_pat[w.o]]->kdim;
          for (int m = 0; m < kd; ++m)
            E[p][base + (size_t)(col0[ui] + m) * ld + j] += (double)(sgo * w.sg) * hNb[occ_pat[w.o]][(size_t)w.j * kd + m];
        }
      }
      for (size_t i = 0; i < us.size(); ++i)
        for (int m = 0; m < ctx->pats[occ_pat[us[i]]]->kdim; ++m) mcol_row.push_back(occ_gofs[us[i]] + m);
      mcol_ptr[o + 1] = nc;
    }
  }
  for (int o = 0; o < n_occ; ++o) mcol_ptr[o + 1] += mcol_ptr[o];
  // mcol_row was filled pattern by pattern: reorder to occurrence order
  {
    std::vector<int> rows(mcol_row.size());
    size_t pos = 0;
    std::vector<size_t> start(n_occ);
    for (int p = 0; p < n_pat; ++p)
      for (int o : ctx->use[p].occs) { start[o] = pos; pos += mcol_ptr[o + 1] - mcol_ptr[o]; }
    for (int o = 0; o < n_occ; ++o)
      for (int c = 0; c < mcol_ptr[o + 1] - mcol_ptr[o]; ++c) rows[mcol_ptr[o] + c] = mcol_row[start[o] + c];
    mcol_row.swap(rows);
  }
  long long mtotal = 0;
  for (int p = 0; p < n_pat; ++p) { mbase[p] = mtotal; mtotal += (long long)mcols[p] * mld[p]; }
  for (int p = 0; p < n_pat; ++p)
    for (int o : ctx->use[p].occs) moff[o] = mbase[p] + moff[o] * mld[p];
  DBuf<double> dE(std::max<long long>(mtotal, 1)), dMd(std::max<long long>(mtotal, 1));
  for (int p = 0; p < n_pat; ++p)
    if (!E[p].empty())
      FETIRP_CUDA(cudaMemcpyAsync(dE.p + mbase[p], E[p].data(), sizeof(double) * E[p].size(), cudaMemcpyHostToDevice, s));
  SP.M64.ensure(std::max<long long>(mtotal, 1));
  SP.M32.ensure(std::max<long long>(mtotal, 1));
  for (int p = 0; p < n_pat; ++p) ensure_splus64(*ctx->pats[p], s);
  for (int pass = 0; pass < 2; ++pass) {   // S^+ E, then S^dag E
    LocalProblem LP{};
    LP.n_pat = n_pat;
    for (int p = 0; p < n_pat; ++p) {
      const PatternData& P = *ctx->pats[p];
      LP.S[p] = pass == 0 ? (const void*)P.S64.p : (const void*)(P.kdim > 0 ? P.Sdag.p : P.S64.p);
      LP.n_b[p] = P.n_b;
      LP.n_rhs[p] = mcols[p];
      LP.ld[p] = mld[p];
      LP.Y[p] = dE.p + mbase[p];
      LP.Z[p] = (pass == 0 ? SP.M64.p : dMd.p) + mbase[p];
    }
    local_gemm_f64(LP, s);
  }
  k_to_f32<<<(unsigned)((mtotal + 255) / 256), 256, 0, s>>>((size_t)mtotal, dMd.p, SP.M32.p);
  FETIRP_LAUNCH_CHECK();
  SP.d_pair_occ.upload(pair_occ, s);
  SP.d_pair_g.upload(pair_g, s);
  SP.d_pair_of.upload(pair_of, s);
  SP.d_mcol_ptr.upload(mcol_ptr, s);
  SP.d_mcol_row.upload(mcol_row, s);
  SP.d_moff.upload(moff, s);
  SP.d_mld.upload(mld, s);
  SP.Vs.ensure((size_t)nl * k);
  SP.Yc.ensure((size_t)std::max(L.n_slots, 1) * k);
  FETIRP_CUDA(cudaStreamSynchronize(s));   // the temporaries dE, dMd are released on return
  SP.k = k;
}

// Q = P^T F P S(r) by the sparse-column form (equal to apply_F on the dense S(r))
void apply_split(fetirp_ctx ctx, const double* d_r, double* d_Q, int prec) {
  SplitPlan& SP = ctx->sp;
  if (SP.k != ctx->k) split_plan_build(ctx);
  ensure_operators(ctx, prec);   // formed by the plan; again after a refactorisation
  cudaStream_t s = ctx->stream;
  const Layout& L = ctx->L;
  const int k = ctx->k, n_pat = (int)ctx->pats.size();
  split(L, d_r, k, SP.Vs.p, s);
  if (ctx->n_G > 0) {   // X = (G^T G)^{-1} G^T S(r) and its local responses M_s X
    gt_v(L, SP.Vs.p, k, ctx->Xc.p, s);
    small_gemm(ctx->n_G, k, ctx->Ginv.p, ctx->Xc.p, ctx->Ac.p, s, ctx->sg_part.p);
    if (prec == FETIRP_PREC_FP64)
      coarse_response<double>(L, k, SP.M64.p, SP.d_moff.p, SP.d_mcol_ptr.p, SP.d_mcol_row.p, SP.d_mld.p, ctx->Ac.p,
                              SP.Yc.p, s);
    else
      coarse_response<float>(L, k, SP.M32.p, SP.d_moff.p, SP.d_mcol_ptr.p, SP.d_mcol_row.p, SP.d_mld.p, ctx->Ac.p,
                             SP.Yc.p, s);
  } else {
    SP.Yc.zero(s);
  }
  auto view = [&](auto* base, auto& V) {
    for (int p = 0; p < n_pat; ++p) { V.base[p] = base + SP.ybase[p]; V.ld[p] = ctx->pats[p]->ld_y; }
    for (int p = 0; p <= n_pat; ++p) V.pair_off[p] = SP.pair_off[p];
  };
  const long long tot = std::max<long long>(SP.ytotal, 1);
  if (prec == FETIRP_PREC_FP64) {
    SP.Y64.ensure(tot); SP.Z64.ensure(tot);
    PairView<double> Y{}, Z{};
    view(SP.Y64.p, Y); view(SP.Z64.p, Z);
    gather_pairs_f64(L, SP.Vs.p, k, SP.d_pair_occ.p, SP.d_pair_g.p, SP.n_pairs, Y, s);
    LocalProblem LP{};
    LP.n_pat = n_pat;
    for (int p = 0; p < n_pat; ++p) {
      LP.S[p] = ctx->pats[p]->S64.p; LP.n_b[p] = ctx->pats[p]->n_b; LP.ld[p] = Y.ld[p];
      LP.n_rhs[p] = SP.pair_off[p + 1] - SP.pair_off[p]; LP.Y[p] = Y.base[p]; LP.Z[p] = Z.base[p];
    }
    local_gemm_f64(LP, s);
    scatter_pairs<double>(L, Z, k, SP.d_pair_of.p, SP.Yc.p, d_Q, s);
  } else {
    SP.Y32.ensure(tot); SP.Z32.ensure(tot);
    PairView<float> Y{}, Z{};
    view(SP.Y32.p, Y); view(SP.Z32.p, Z);
    if (prec == FETIRP_PREC_FP32) {
      gather_pairs_f32(L, SP.Vs.p, k, SP.d_pair_occ.p, SP.d_pair_g.p, SP.n_pairs, Y, s);
      LocalProblem LP{};
      LP.n_pat = n_pat;
      for (int p = 0; p < n_pat; ++p) {
        LP.S[p] = ctx->pats[p]->S32.p; LP.n_b[p] = ctx->pats[p]->n_b; LP.ld[p] = Y.ld[p];
        LP.n_rhs[p] = SP.pair_off[p + 1] - SP.pair_off[p]; LP.Y[p] = Y.base[p]; LP.Z[p] = Z.base[p];
      }
      local_gemm_f32(LP, s);
    } else {
      SP.Ylo32.ensure(tot);
      PairView<float> Yl{};
      view(SP.Ylo32.p, Yl);
      gather_pairs_split(L, SP.Vs.p, k, SP.d_pair_occ.p, SP.d_pair_g.p, SP.n_pairs, Y, Yl, s);
      if (!ctx->tc_error.p) { ctx->tc_error.alloc(1); ctx->tc_error.zero(s); }
      TcProblem T;
      T.n_pat = n_pat;
      for (int p = 0; p < n_pat; ++p) {
        const PatternData& P = *ctx->pats[p];
        T.S_hi[p] = P.S_hi.p; T.S_lo[p] = P.S_lo.p; T.lds[p] = P.lds;
        T.Y_hi[p] = Y.base[p]; T.Y_lo[p] = Yl.base[p]; T.Z[p] = Z.base[p]; T.ldy[p] = Y.ld[p];
        T.n_b[p] = P.n_b; T.n_rhs[p] = SP.pair_off[p + 1] - SP.pair_off[p];
      }
      tc_gemm_tf32x3(T, ctx->tc_error.p, s);
    }
    scatter_pairs<float>(L, Z, k, SP.d_pair_of.p, SP.Yc.p, d_Q, s);
  }
  project(ctx, d_Q, k);   // P^T
}

}  // namespace

extern "C" {

fetirp_status fetirp_apply_split_device(fetirp_ctx ctx, const double* d_r, double* d_Q, int32_t precision) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (!ctx->prepared) throw Error(FETIRP_ESTATE, "call fetirp_prepare or fetirp_solve first");
    REQUIRE(d_r && d_Q, "NULL buffer");
    REQUIRE(precision >= FETIRP_PREC_FP64 && precision <= FETIRP_PREC_TF32X3, "unsupported precision");
    apply_split(ctx, d_r, d_Q, precision);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_apply_split(fetirp_ctx ctx, const double* r, double* Q, int32_t precision) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (!ctx->prepared) throw Error(FETIRP_ESTATE, "call fetirp_prepare or fetirp_solve first");
    REQUIRE(r && Q, "NULL buffer");
    REQUIRE(precision >= FETIRP_PREC_FP64 && precision <= FETIRP_PREC_TF32X3, "unsupported precision");
    const size_t nl = (size_t)ctx->L.n_lambda, n = nl * ctx->k;
    DBuf<double> dr(nl), dq(n);
    dr.upload(r, nl, ctx->stream);
    apply_split(ctx, dr.p, dq.p, precision);
    check_tc_error(ctx);
    FETIRP_CUDA(cudaMemcpyAsync(Q, dq.p, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
    return FETIRP_OK;
  });
}

fetirp_status fetirp_set_permutation(fetirp_ctx ctx, int64_t n_lambda, const int64_t* rowptr, const int32_t* col,
                                     const double* val, int32_t n_images, int32_t shortcut) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (!rowptr) {   // back to the occurrence split
      ctx->perm.on = false;
      invalidate(ctx);
      return FETIRP_OK;
    }
    REQUIRE(n_lambda > 0 && n_lambda < (1LL << 31), "n_lambda out of range");
    REQUIRE(col && val, "NULL permutation array");
    REQUIRE(n_images >= 1 && n_images <= 64, "n_images must be in 1..64");
    REQUIRE(shortcut == 0 || shortcut == 1, "shortcut must be 0 or 1");
    const int n = (int)n_lambda;
    REQUIRE(rowptr[0] == 0, "rowptr[0] must be 0");
    for (int i = 0; i < n; ++i) REQUIRE(rowptr[i + 1] >= rowptr[i], "rowptr must be non-decreasing");
    for (int64_t e = 0; e < rowptr[n]; ++e) {
      REQUIRE(col[e] >= 0 && col[e] < n, "permutation column out of range");
      REQUIRE(std::isfinite(val[e]), "non-finite permutation entry");
    }
    // powers Pi^g, g < n_images, row by row: (Pi^g)[row] = sum_e Pi[row][c_e] (Pi^(g-1))[c_e]
    constexpr int PW_MAX = 8;
    using Row = std::vector<std::pair<int, double>>;
    std::vector<Row> cur(n), next(n);
    for (int i = 0; i < n; ++i) cur[i] = {{i, 1.0}};
    std::vector<std::vector<Row>> pows;
    pows.push_back(cur);
    int pw = 1;
    for (int g = 1; g < n_images; ++g) {
      for (int i = 0; i < n; ++i) {
        Row acc;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
          for (const auto& t : cur[col[e]]) acc.push_back({t.first, val[e] * t.second});
        std::sort(acc.begin(), acc.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        Row merged;
        for (const auto& t : acc) {
          if (!merged.empty() && merged.back().first == t.first) merged.back().second += t.second;
          else merged.push_back(t);
        }
        Row kept;
        for (const auto& t : merged)
          if (t.second != 0.0) kept.push_back(t);
        if ((int)kept.size() > PW_MAX)
          throw Error(FETIRP_EINVAL, "a row of a power of the permutation has more than 8 entries");
        pw = std::max(pw, (int)kept.size());
        next[i] = std::move(kept);
      }
      cur.swap(next);
      pows.push_back(cur);
    }
    auto& P = ctx->perm;
    P.k = n_images;
    P.pw = pw;
    P.n = n_lambda;
    P.src.assign((size_t)n * n_images * pw, 0);
    P.w.assign((size_t)n * n_images * pw, 0.0);
    for (int g = 0; g < n_images; ++g)
      for (int i = 0; i < n; ++i)
        for (size_t e = 0; e < pows[g][i].size(); ++e) {
          const size_t at = ((size_t)i * n_images + g) * pw + e;
          P.src[at] = pows[g][i][e].first;
          P.w[at] = pows[g][i][e].second;
        }
    P.shortcut = shortcut == 1;
    P.on = true;
    invalidate(ctx);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_set_preconditioner(fetirp_ctx ctx, int32_t kind, int32_t scaling) {
  return guarded(ctx, [&]() -> fetirp_status {
    REQUIRE(kind >= FETIRP_PRECOND_NONE && kind <= FETIRP_PRECOND_SUPERLUMPED, "unknown preconditioner");
    REQUIRE(scaling == FETIRP_SCALING_MULTIPLICITY || scaling == FETIRP_SCALING_STIFFNESS, "unknown scaling");
    ctx->pc.kind = kind;
    ctx->pc.scaling = scaling;
    invalidate(ctx);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_set_row_blocks(fetirp_ctx ctx, int32_t n_blocks, const int64_t* row_offset) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (n_blocks == 0 || !row_offset) {
      ctx->row_blocks.clear();
      return FETIRP_OK;
    }
    REQUIRE(n_blocks >= 1, "n_blocks < 0");
    REQUIRE(row_offset[0] == 0, "row_offset[0] must be 0");
    for (int b = 0; b < n_blocks; ++b) REQUIRE(row_offset[b + 1] > row_offset[b], "row blocks must be non-empty");
    ctx->row_blocks.assign(row_offset, row_offset + n_blocks + 1);
    return FETIRP_OK;
  });
}

fetirp_status fetirp_device_status(fetirp_ctx ctx) {
  return guarded(ctx, [&]() -> fetirp_status {
    check_tc_error(ctx);   // synchronises the context stream, reads the flag and clears it
    return FETIRP_OK;
  });
}

fetirp_status fetirp_inject_barrier_stall(fetirp_ctx ctx) {
  return guarded(ctx, [&]() -> fetirp_status {
    ctx->inject_stall = true;
    return FETIRP_OK;
  });
}

fetirp_status fetirp_factorize(fetirp_ctx ctx) {
  return guarded(ctx, [&]() -> fetirp_status {
    if (ctx->is_child) throw Error(FETIRP_ESTATE, "a child context shares its parent's factors; factorise the parent");
    reset_phases(ctx);
    const unsigned long long l0 = g_launch_count;
    std::vector<PatternData*> all;
    for (auto& P : ctx->pats) all.push_back(P.get());
    factorize_patterns(ctx, all);
    ctx->phases_pending = true;
    ctx->pending_launches = (long long)(g_launch_count - l0);
    ctx->prepared = false;   // d, the coarse problem and G's values follow the new factors; the structure stands
    return FETIRP_OK;
  });
}

fetirp_status fetirp_get_pattern(fetirp_ctx ctx, int32_t pid, int32_t* n_b_out, int32_t* kdim_out, double* splus,
                                 double* kernel) {
  return guarded(ctx, [&]() -> fetirp_status {
    REQUIRE(pid >= 0 && pid < (int)ctx->pats.size(), "unknown pattern id");
    PatternData& P = *ctx->pats[pid];
    if (n_b_out) *n_b_out = P.n_b;
    if (kdim_out) *kdim_out = P.kdim;
    if (splus) ensure_splus64(P, ctx->stream);
    if (splus)
      FETIRP_CUDA(cudaMemcpyAsync(splus, P.S64.p, sizeof(double) * (size_t)P.n_b * P.n_b, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    if (kernel && P.kdim > 0) {
      std::vector<double> N((size_t)P.npad * P.kdim);
      FETIRP_CUDA(cudaMemcpyAsync(N.data(), P.N.p, sizeof(double) * N.size(), cudaMemcpyDeviceToHost, ctx->stream));
      FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
      for (int d = 0; d < P.n; ++d)
        for (int m = 0; m < P.kdim; ++m) kernel[(size_t)d * P.kdim + m] = N[(size_t)m * P.npad + P.newidx[d]];
    }
    FETIRP_CUDA(cudaStreamSynchronize(ctx->stream));
    return FETIRP_OK;
  });
}

}  // extern "C"
