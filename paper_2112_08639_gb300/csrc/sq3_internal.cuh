// Internal declarations shared by the translation units of libsq3.
#pragma once
#include <cuda.h>

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <vector>

#include "../../include/sq3.h"

#define SQ3_MAX_FD_RADIUS 6
#define SQ3_MAX_NPL 1000
#define SQ3_DEV_SCAL 3072
// dev_scal slots: 0..63 bounds/outputs/norms, 64..2065 Fermi-operator
// moments and coefficients, from SQ3_SCAL_MISC: the potential's range
// (2 values + 2 x 304 partials) and the SCF driver's scalars
#define SQ3_SCAL_MISC 2304
// bf16 pieces per FP32 operand in the mixed path (3 pieces, 6 products)
#define MIXED_PIECES 3
// largest Ns accepted by sq3_lanczos_bounds_noalloc (static scratch size)
#define SQ3_NOALLOC_MAX_NS 8192
// chunks of vectors a host block is uploaded in (sq3_cheb_filter_from_host)
#define SQ3_UPLOAD_CHUNKS 2
// nonlocal pass: points per CTA (an 8 x 8 x NL_BZ brick)
#define NL_BZ 4
#define NL_BRICK_PTS (64 * NL_BZ)

namespace sq3 {

// Device-side status word values (first error wins).
enum DevStatus : int {
  DEV_OK = 0,
  DEV_NOTPD = 1,
  DEV_NOCONV = 2,
  DEV_NONFINITE = 3,
  DEV_TIMEOUT = 4,
};

// Grid and stencil description passed by value to kernels.
struct Grid {
  int nx, ny, nz;
  long long N;
  double hx, hy, hz;
  int radius;                        // fd_order / 2
  double w[SQ3_MAX_FD_RADIUS + 1];   // second-derivative weights (unscaled)
};

// Projectors on the device: their energies and the brick tables of the
// nonlocal pass.  On the host the projectors that share one index list (the
// <= 4 of an atom) are grouped into balls first; the tables are per ball.
struct Projectors {
  int n_proj = 0;
  int n_ball = 0;
  double* gamma = nullptr;      // n_proj
  // Nonlocal-pass tables per 8 x 8 x NL_BZ brick b of the grid (bricks x
  // fastest; local point t = tx + 8 ty + 64 tz), grouped by ball:
  //   local balls of brick b: slots nb_ball_ptr[b] .. nb_ball_ptr[b+1]-1;
  //     slot s carries projector ids nb_slot_pid[4s .. 4s+3] (-1 = none)
  //   point-major entries of point t: nb_pt_ptr[NL_BRICK_PTS b + t] ..
  //     nb_pt_ptr[NL_BRICK_PTS b + t + 1] - 1, each the local ball
  //     (nb_pt_lb, relative to the brick's first slot) and the ball's four
  //     c_p values at the point (nb_pt_val, zero padded)
  //   ball-major entries of slot s: nb_bl_ptr[s] .. nb_bl_ptr[s+1]-1, each
  //     the point (nb_bl_pt) and the four values (nb_bl_val)
  int* nb_ball_ptr = nullptr;
  int* nb_slot_pid = nullptr;
  int* nb_pt_ptr = nullptr;
  short* nb_pt_lb = nullptr;
  double* nb_pt_val = nullptr;
  float* nb_pt_valf = nullptr;
  int* nb_bl_ptr = nullptr;
  short* nb_bl_pt = nullptr;
  double* nb_bl_val = nullptr;
  float* nb_bl_valf = nullptr;
  int max_brick_balls = 0;     // most balls touching one brick
  int max_brick_entries = 0;   // most (point, ball) entries in one brick
  // Gershgorin bounds on the spectrum of V_nl = sum_p gamma_p c_p c_p^T
  // (from the projectors' overlap matrix): vnl_lo <= lambda <= vnl_hi
  double vnl_lo = 0.0, vnl_hi = 0.0;
  // host copy of the balls (for the force tables): ball B covers grid
  // indices h_bidx[h_bptr[B] .. h_bptr[B+1]-1]; its h_bnp[B] projectors are
  // h_bp0[B] + q with values h_bval[h_boff[B] + q * len + e] (c = chi sqrt(dV))
  std::vector<int> h_bptr, h_bidx, h_bp0, h_bnp, h_boff;
  std::vector<double> h_bval;
  std::vector<double> h_gamma;
  // force tables (forces.cu), built on the first force call: per ball the
  // rows fq_ptr[B] .. fq_ptr[B+1]-1, each a grid index fq_idx and 16 values
  // (4 projectors x {c, d/dx c, d/dy c, d/dz c}, FD first derivative)
  bool fq_ok = false;
  int* fq_ptr = nullptr;
  int* fq_idx = nullptr;
  double* fq_val = nullptr;
  float* fq_valf = nullptr;
  int fq_max_rows = 0;
};

}  // namespace sq3

namespace sq3 {
// Stage classes for the optional per-stage CUDA-event timing.
enum Stage {
  ST_STENCIL = 0, ST_NL_PROJECT, ST_GRAM, ST_CHOL, ST_TRINV, ST_XRINV,
  ST_HS_GEMM, ST_LANCZOS, ST_CHEB_GEMM, ST_FERMI, ST_D_ACCUM, ST_RHO,
  ST_SPLIT, ST_COPY, ST_NL_PASS, ST_COUNT
};
struct ProfRec { int stage; int launches; cudaEvent_t a, b; };
}  // namespace sq3

struct sq3_ctx {
  int device = 0;
  bool prof = false;
  // BF16 pieces of an orthonormalised block X, written by the last X R^-1
  // product of the mixed Cholesky QR: cols in the split workspace's colX,
  // rows at pieces_rows.  Used (instead of splitting X again) by the mixed
  // projection and density only while reuse_pieces is set, i.e. inside the
  // SCF driver, which alone knows that X has not changed in between; any
  // library call that writes X clears pieces_X.
  bool reuse_pieces = false;
  const void* pieces_X = nullptr;
  int pieces_Ns = 0;
  void* pieces_rows = nullptr;
  // H X of the mixed projection, kept in the work block wsX with the FP32
  // potential it was applied with (Vf_hx), for the next filter of the same
  // X inside the SCF driver: its first step is then (s1/e)(H X + (V - V_hx) X
  // - c X), elementwise, instead of a stencil and a nonlocal pass
  const void* hx_X = nullptr;
  int hx_Ns = 0;
  float* Vf_hx = nullptr;
  std::vector<sq3::ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  cudaStream_t stream = nullptr;
  bool grid_ok = false, pot_ok = false;
  sq3::Grid grid{};
  double Lx = 0, Ly = 0, Lz = 0, dV = 0;
  double* V = nullptr;      // N doubles
  float* Vf = nullptr;      // N floats
  double v_min = 0, v_max = 0;
  sq3::Projectors proj;
  int* dev_status = nullptr;      // device status word
  double* dev_scal = nullptr;     // SQ3_DEV_SCAL device scalars: bounds,
                                  // outputs, moments, coefficients
  double* host_scal = nullptr;    // pinned mirror
  // workspace
  void* wsX = nullptr; size_t wsX_bytes = 0;        // one N x Ns block
  void* wsX2 = nullptr; size_t wsX2_bytes = 0;      // second block (mixed)
  double* wsMat = nullptr; size_t wsMat_bytes = 0;  // Ns x Ns matrices
  double* wsT = nullptr; size_t wsT_bytes = 0;      // stored T_j
  double* wsProj = nullptr; size_t wsProj_bytes = 0;  // projection coeffs
  void* wsSplit = nullptr; size_t wsSplit_bytes = 0;  // bf16 split operands
  double* wsFoe = nullptr; size_t wsFoe_bytes = 0;    // quadrature node values
  float* wsLin32 = nullptr; size_t wsLin32_bytes = 0;  // FP32 factor, inverse, temporaries
  // self-consistent-field pieces (scf.cu): real Fourier basis tables of the
  // grid (rebuilt after sq3_setup_grid) and two N-point buffers + partials
  double* scfTab = nullptr; size_t scfTab_bytes = 0;
  bool scf_tab_ok = false;
  double* wsScf = nullptr; size_t wsScf_bytes = 0;
  // density mixer (sq3_mixer_setup / sq3_mixer_step): settings, step count
  // and the ring of history differences in wsMix
  struct MixState {
    bool ready = false, have_prev = false;
    int h = 0, period = 1, m = 0, head = 0;
    long long k = 0;
    double beta = 0.0, k0 = 0.0;
  } mix;
  double* wsMix = nullptr; size_t wsMix_bytes = 0;
  // SCF driver (sq3_scf_solve): output density, V_eff, Hs, Ds, Lanczos work
  double* wsDrv = nullptr; size_t wsDrv_bytes = 0;
  // atom-centred Gaussians and forces (atoms.cu, forces.cu): 1-D tables,
  // charges, partial sums
  double* wsAtoms = nullptr; size_t wsAtoms_bytes = 0;
  // uploads of a host block (sq3_cheb_filter_from_host): a stream of their
  // own and one event per chunk, created on first use
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t upload_ev[SQ3_UPLOAD_CHUNKS] = {};
};

namespace sq3 {

int ensure(void** p, size_t* have, size_t need);

// Records CUDA events around the launches issued during its lifetime on the
// context's stream when profiling is enabled; `launches` is how many kernels
// those are.
struct Prof {
  sq3_ctx* ctx; int stage; int launches; cudaEvent_t a = nullptr, b = nullptr;
  Prof(sq3_ctx* c, int st, int n = 1);
  ~Prof();
};
int cuda_err(cudaError_t e);
int check_device_status(sq3_ctx* ctx);
// Sets DEV_NONFINITE in *status when one of the n device values is not finite.
void check_finite(const double* a, long long n, int* status, cudaStream_t st);
// out[0], out[1] = smallest and largest of the n device values (fixed-order
// reduction; part: 608 doubles of device scratch); non-finite values set
// DEV_NONFINITE.
void minmax(const double* a, long long n, double* part, double* out, int* status,
            cudaStream_t st);
// Tiled TMA tensor map over a dense array (FP32 or FP64 elements), no
// swizzle, zero fill; dims and box innermost first, strides in bytes for
// dims 1..rank-1.  Returns SQ3_OK, SQ3_EINVAL (alignment) or SQ3_ECUDA.
int encode_tensor_map(CUtensorMap* map, bool fp64, int rank, void* base,
                      const unsigned long long* dims, const unsigned long long* strides,
                      const unsigned* box);

// ---- stencil / Hamiltonian (stencil.cu) ----
// out = s1 * (H_loc y - c y) + s2 * yprev, per vector, for Ns vectors, with
// H_loc = -1/2 Lap + V.
// The nonlocal term is added by
// launch_nl_pass.  yprev may alias out (each element reads only its own
// yprev before writing it); y must not alias out.
template <typename T>
void launch_cheb_step(const sq3_ctx* ctx, const T* y, const T* yprev, T* out, int Ns,
                      double s1, double c, double s2, cudaStream_t st);
// In-place nonlocal pass on a local step's output (see stencil.cu):
// out += s1 * sum_p c_p gC[p]; gC_next (zeroed, may be null) += gamma c^T out.
// Dynamic shared memory of the nonlocal pass for element size es, VB vectors
// per box, NBUF boxes, and the largest brick (balls, entries).
size_t nl_pass_smem_bytes(int es, int VB, int NBUF, int max_balls, int max_entries);
// Host tables of a projector set (projector_tables.cu): the balls (the
// Projectors host copies), the brick tables (the nb_* arrays: sptr, spid,
// qptr, qlb, qval, zptr, zpt, zval) and the Gershgorin bounds of V_nl.  The
// CSR input must already be validated; repeated indices are merged.
struct ProjectorHostTables {
  std::vector<int> bptr, bidx, bp0, bnp, boff;
  std::vector<double> bval;
  std::vector<int> sptr, spid, qptr, zptr;
  std::vector<short> qlb, zpt;
  std::vector<double> qval, zval;
  int max_brick_balls = 0, max_brick_entries = 0;
  double vnl_lo = 0.0, vnl_hi = 0.0;
};
void projector_host_tables(int nx, int ny, int nz, double dV, int n_proj, const int* ptr,
                           const int* idx, const double* val, const double* gamma,
                           ProjectorHostTables& T);
// With gC == nullptr the pass only projects (gC_next += gamma c^T out) and
// leaves out untouched.  Returns an SQ3_* status (EINVAL when a brick's
// tables exceed shared memory or out is not 16-byte aligned).
template <typename T>
int launch_nl_pass(const sq3_ctx* ctx, T* out, const T* gC, T* gC_next, int Ns,
                   double s1, cudaStream_t st);

// ---- atom-centred Gaussians (atoms.cu) ----
// Host tables of the 1-D periodic image sums of exp(-(x - R)^2 / w^2) (or
// their x-derivatives) for every atom: gx | gy | gz, natoms x n each.
void atom_tables(const sq3_ctx* c, int natoms, const double* pos, double w, bool deriv,
                 std::vector<double>& tab);

// ---- FP64 GEMM (gemm_f64.cu) ----
enum Epi { EPI_STORE = 0, EPI_ATOMIC = 1, EPI_CHEB = 2, EPI_RHO = 3 };
struct GemmArgs {
  int M, N, K;
  const double* A; long long lda; bool a_kcontig;   // A(m,k)
  const double* B; long long ldb; bool b_kcontig;   // B(k,n)
  double* C; long long ldc;
  double alpha, beta;
  int splits;                 // split-K factor (EPI_ATOMIC)
  // 1: only tiles on or above the diagonal are computed (C symmetric);
  // 2: B is upper triangular (B(k,n) = 0 for k > n), so K stops at the
  //    tile's last column;
  // 3: only tiles on or below the diagonal are computed.
  int tri;
  // EPI_CHEB: C = 2*acc - P, P(m,n) = P[m + n*ldp]; trace of C -> *trace.
  const double* P; long long ldp; double* trace;
  // EPI_RHO: rho[m] += alpha * sum_n X(m,n) acc(m,n), X(m,n)=X[m+n*ldx]
  const double* X; long long ldx; double* rho;
};
void gemm_f64(const GemmArgs& g, Epi epi, cudaStream_t st);

// ---- dense linear algebra (linalg.cu) ----
int cholesky_lower_f64(sq3_ctx* ctx, double* S, int n, double* diag_ws,
                       cudaStream_t st);
void tri_inverse_transpose_f64(const double* L, double* Rinv, int n,
                               double* diag_ws, cudaStream_t st);
void symmetrize_f64(double* A, int n, cudaStream_t st);
// ---- FP32 linear algebra for the mixed Cholesky QR (linalg32.cu) ----
// F = deviation Cholesky factor of S = I + E (S FP64 column-major n x n):
// S = (I + F)(I + F)^T with F lower (diagonal included), FP32.  Sets
// DEV_NOTPD when a pivot 1 + t is not above 1e-3.
int deviation_cholesky_f32(sq3_ctx* ctx, const double* S, float* F, int n, cudaStream_t st);
// The same on the unit-diagonal scaling D^{-1} S D^{-1} = (I + F)(I + F)^T,
// D = diag(S)^{1/2}; dinv (n floats) receives 1 / sqrt(S_ii).  Then
// S = R^T R with R = (I + F)^T D.
int scaled_deviation_cholesky_f32(sq3_ctx* ctx, const double* S, float* F, float* dinv, int n,
                                  cudaStream_t st);
// *out = |S - I|_F^2 (S FP64 column-major n x n)
// |S - I|_F^2 into *out; part: 32 doubles of device scratch (block sums)
void deviation_norm_f64(const double* S, int n, double* out, double* part, cudaStream_t st);
// R(i, :) *= dinv[i] (column-major n x n)
void scale_rows_f32(float* R, int n, const float* dinv, cudaStream_t st);
// Rinv = L^{-T} (upper, column-major FP32) of the lower-triangular L, or of
// I + L when dev (then without its identity part, Rinv - I, when
// !add_identity).  W: n*n floats, tmp: n*n/2 floats of workspace.  Returns
// the number of kernel launches.
int rinv_from_lower_f32(const float* L, int n, bool dev, float* W, float* tmp, float* Rinv,
                        cudaStream_t st, bool add_identity = true);
void convert_f64_to_f32(const double* A, long long tot, float* B, cudaStream_t st);
void mirror_upper_f64(double* A, int n, cudaStream_t st);
// Words of Lanczos scratch for vectors of length n and `steps` (<= 64)
// steps: the basis (steps + 1 vectors), w, alpha, beta, the step counter and
// the per-block partial sums of one step (alpha over the n / 8 mat-vec
// blocks; two passes of 64 projections and beta^2 over the n / 256 blocks).
constexpr size_t lanczos_work_words(size_t n, size_t steps) {
  return (steps + 2) * n + 2 * steps + 8 + (n * 32 + 255) / 256 +
         ((n + 255) / 256) * (2 * 64 + 1);
}
void lanczos_bounds_f64(sq3_ctx* ctx, const double* Hs, int n, int steps,
                        double* d_bounds, double* work, cudaStream_t st);

// ---- Chebyshev Fermi-operator expansion (foe.cu) ----
// npl < 1: degree from sq3_fermi_degree(sigma, xi, fermi_tol); eval_mode 1:
// Paterson-Stockmeyer (FP64 path); *npl_used (may be null) = the degree.
int density_kernel_from_hs(sq3_ctx* ctx, const double* Hs, int Ns, int npl,
                           double sigma, double Ne, const double* bounds_in,
                           double* D, double* out_host, bool mixed, double fermi_tol = 0.0,
                           int eval_mode = 0, int* npl_used = nullptr);

// ---- mixed-precision path (mixed.cu) ----
int hamiltonian_apply_f32(sq3_ctx* ctx, const float* X, float* Y, int Ns);
int orthonormalise_mixed(sq3_ctx* ctx, float* X, int Ns);
int project_mixed(sq3_ctx* ctx, const float* X, int Ns, double* Hs);
int cheb_recurrence_mixed(sq3_ctx* ctx, const double* Hs, int Ns, int h,
                          const double* bounds, double* mom, float* T);
// part: moments_tail_part_words(npl, h) doubles of device scratch
size_t moments_tail_part_words(int npl, int h);
int moments_tail_mixed(sq3_ctx* ctx, const float* T, int Ns, int npl, int h, double* mom,
                       double* part);
int accumulate_d_mixed(sq3_ctx* ctx, const float* T, int Ns, int npl, int h,
                       const double* coef, double* D, float* A2);
int density_mixed(sq3_ctx* ctx, const float* X, const double* D, int Ns,
                  double* rho);

// ---- Paterson-Stockmeyer evaluation of the expansion (foe.cu, mixed.cu) ----
// s baby steps T_0..T_s, giant steps G_q = T_{qs} (q <= Q), Q = npl / s.
constexpr int PS_FROB_BLOCKS = 16;   // blocks per Frobenius product <G_q, T_r>
int ps_layout(int npl, int* s_out, int* Q_out);
// mom[qs + r] = 2 <G_q, T_r> - mom[qs - r] from the block sums
// part[((q - 1)(s - 1) + r - 1) PS_FROB_BLOCKS + b], in increasing q
void ps_moments_finish(const double* part, int s, int Q, int npl, double* mom, cudaStream_t st);
// alpha[q s + r]: Ds = sum_q (sum_{r<s} alpha[q s + r] T_r) T_q(T_s); work:
// (Q + 1) s doubles
void ps_alpha(const double* coef, int npl, int s, int Q, double* work, double* alpha,
              cudaStream_t st);
// The mixed path's form: FP32 matrices, tensor-core products with BF16
// pieces.  W: ps_mixed_bytes(Ns, s, Q) bytes of device workspace, shared by
// the two calls (the moments call leaves the baby and giant steps in it).
size_t ps_mixed_bytes(int Ns, int s, int Q);
int ps_moments_mixed(sq3_ctx* ctx, const double* Hs, int Ns, int npl, int s, int Q,
                     const double* bounds, double* mom, void* W);
int ps_kernel_mixed(sq3_ctx* ctx, int Ns, int npl, int s, int Q, const double* coef, void* W,
                    double* D);

}  // namespace sq3
