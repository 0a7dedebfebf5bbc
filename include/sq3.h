/*
 * sq3.h -- C ABI of the GB300 (sm_103a) SQ3 hot path.
 *
 * SQ3 is the real-space density-kernel method for Kohn-Sham DFT at high
 * temperature of arXiv 2112.08639.  One fixed-potential iteration (Sec. 4 of
 * the paper) is:
 *
 *   X  <- p_m(H) X                 Chebyshev filter      sq3_cheb_filter
 *   X  <- X R^{-1}, X^T X = R^T R  orthonormalisation    sq3_orthonormalise
 *   Hs  = X^T H X                  projection            sq3_project
 *   Ds  = g(Hs) ~ sum'_j c_j T_j(Hhat), mu, E_band, E_ent
 *                                  density kernel        sq3_kernel_from_hs
 *   rho = 2 sum_i (X Ds)_i X_i / dV                       sq3_density
 *
 * with H = -1/2 Lap_12 + V + sum_p gamma_p c_p c_p^T on a periodic grid.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grid index k = i + nx*j + nx*ny*l (x fastest).  N = nx*ny*nz.
 * - A block X of Ns vectors is N x Ns column-major: vector i occupies
 *   X[i*N .. i*N+N-1].  Vectors are Euclidean-normalised (u = psi sqrt(dV)).
 * - Element type of X follows the precision argument: SQ3_FP64 -> double,
 *   SQ3_MIXED -> float.  Ns x Ns matrices (Hs, Ds) and rho are always double.
 * - Unless stated otherwise, array pointers are DEVICE pointers to
 *   caller-owned memory on the context's device; the library never frees or
 *   retains them after the call returns.
 * - Work is ordered on the context's CUDA stream.  Every entry point returns
 *   only after that stream has reached the end of its work, so outputs are
 *   ready and device-side errors have been checked.
 * - The context owns its workspace (device memory sized on first use and
 *   grown when a larger Ns or N is seen); it is released by sq3_destroy.
 * - Return value: SQ3_OK (0) or a negative SQ3_E* code.  No C++ exception
 *   crosses the ABI and no kernel traps; device-side failures are reported
 *   through these codes.  sq3_status_string() names a code.
 */
#ifndef SQ3_H
#define SQ3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sq3_ctx sq3_ctx;

typedef enum {
  SQ3_FP64 = 0,   /* X double; every step in FP64                           */
  SQ3_MIXED = 1   /* X float; stencil FP32; Gram/projection/recurrence/XD on
                     tcgen05 BF16 split products with FP32 accumulation;
                     Cholesky, Fermi level, energies and reductions in FP64  */
} sq3_prec;

enum {
  SQ3_OK = 0,
  SQ3_EINVAL = -1,      /* bad argument (null pointer, size, precision)      */
  SQ3_ENOTSETUP = -2,   /* grid or potential not set                          */
  SQ3_ECUDA = -3,       /* a CUDA runtime/driver call failed                  */
  SQ3_ENOTPD = -4,      /* Cholesky pivot <= 0: X^T X not positive definite   */
  SQ3_ENOCONV = -5,     /* Fermi-level bracket or spectral-bound check failed */
  SQ3_ETIMEOUT = -6,    /* a bounded device-side wait ran out                 */
  SQ3_ENONFINITE = -7,  /* NaN/Inf detected in an output                      */
  SQ3_ENOMEM = -8       /* workspace allocation failed                        */
};

/* Create a context on CUDA device `device` whose work is ordered on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * *out receives the context.  Errors: SQ3_EINVAL, SQ3_ECUDA. */
int sq3_create(sq3_ctx** out, int device, void* cuda_stream);

/* Release the context and its workspace.  NULL is accepted. */
void sq3_destroy(sq3_ctx* ctx);

/* Periodic orthorhombic grid nx x ny x nz over a cell Lx x Ly x Lz (bohr)
 * with a central finite-difference Laplacian of order fd_order (even, 2..12;
 * the paper uses 12, Sec. 5).  Weights: Fornberg closed form
 * w_p = 2(-1)^(p+1)(n!)^2/(p^2 (n-p)!(n+p)!), w_0 = -2 sum 1/p^2, n = order/2.
 * Requires fd_order/2 <= nx, ny, nz and nx <= 512.  Resets the potential and
 * projectors.  Errors: SQ3_EINVAL. */
int sq3_setup_grid(sq3_ctx* ctx, int nx, int ny, int nz,
                   double Lx, double Ly, double Lz, int fd_order);

/* Effective local potential V_eff = V_xc + phi (Sec. 2, Eq. (KSeqn)) on the
 * grid: device array of N doubles.  Copied into the context, with its range
 * (the filter's spectral bounds use it).
 * Errors: SQ3_ENOTSETUP (no grid), SQ3_EINVAL, SQ3_ENONFINITE (a value is
 * NaN or infinite; the context then has no potential until the next
 * successful call). */
int sq3_set_potential(sq3_ctx* ctx, const double* V);

/* Kleinman-Bylander projectors (Sec. 2, Eq. (nonlocaloperator)) as a CSR
 * table in HOST memory: projector p covers grid indices
 * idx[ptr[p] .. ptr[p+1]-1] with continuum values val (chi_p at those points,
 * NOT multiplied by sqrt(dV)) and energy gamma[p] (Ha).  The library forms
 * c_p = chi_p sqrt(dV) and applies V_nl = sum_p gamma_p c_p c_p^T.
 * Projectors that share an index list (the lm components of one atom) are
 * grouped internally.  n_proj = 0 removes the projectors.  Copied into the
 * context.  Errors: SQ3_ENOTSETUP, SQ3_EINVAL (index out of range, ptr not
 * monotone, a value or energy not finite — checked before the context's
 * current projectors are replaced, so a rejected table changes nothing — or
 * projectors so dense that one 8 x 8 x 4 brick of the grid holds
 * more (point, projector) entries than the nonlocal pass can stage in shared
 * memory, about 7,700).  A grid index may repeat within a projector; its
 * values add. */
int sq3_set_projectors(sq3_ctx* ctx, int n_proj, const int* ptr,
                       const int* idx, const double* val, const double* gamma);

/* Host-only: the tables sq3_set_projectors would build from the same CSR
 * arguments on an nx x ny x nz grid of cell volume element dV, without a
 * context or a device.  info (HOST, 6 ints): {balls (runs of <= 4
 * projectors sharing an index list), (point, ball) entries after repeated
 * indices are merged, 8 x 8 x 4 bricks, most balls in one brick, most
 * entries in one brick, shared-memory bytes of the FP32 nonlocal pass};
 * bounds (HOST, 2 doubles): Gershgorin bounds lo <= lambda <= hi of the
 * spectrum of V_nl = sum_p gamma_p c_p c_p^T, c_p = chi_p sqrt(dV) (from the
 * projectors' overlap matrix; 0 is always inside).  Errors: SQ3_EINVAL as
 * sq3_set_projectors' table checks (and for a bad grid, dV <= 0 or a NULL
 * output). */
int sq3_projector_table_info(int nx, int ny, int nz, double dV, int n_proj, const int* ptr,
                             const int* idx, const double* val, const double* gamma, int* info,
                             double* bounds);

/* Y = H X for a block of Ns vectors (Sec. 2, Eq. (KSeqn)); X and Y are N x Ns
 * column-major of the precision's element type and must not overlap.
 * Errors: SQ3_ENOTSETUP, SQ3_EINVAL. */
int sq3_hamiltonian_apply(sq3_ctx* ctx, const void* X, void* Y, int Ns,
                          sq3_prec prec);

/* Chebyshev filter X <- p_m(H) X in place (Sec. 4, first paragraph: the
 * CheFSI filter of Zhou et al. 2006), p_m(t) = T_m((t-c)/e)/T_m((a0-c)/e)
 * with c = (b+a)/2, e = (b-a)/2, evaluated by the scaled three-term
 * recurrence.  a: lower end of the damped interval (cutoff), b: upper bound
 * of the spectrum of H, a0: lower-bound estimate (p_m(a0) = 1).
 * Requires a0 < a < b and degree >= 1.  Errors: SQ3_ENOTSETUP, SQ3_EINVAL. */
int sq3_cheb_filter(sq3_ctx* ctx, void* X, int Ns, int degree,
                    double a, double b, double a0, sq3_prec prec);

/* The Chebyshev filter of sq3_cheb_filter for a block held in host memory:
 * X_host (N x Ns column-major, element type of prec, read only) is copied to
 * the device block X (same layout, overwritten) in two chunks of whole
 * vectors (the first ceil(Ns/8), then the rest) on a stream of the context's
 * own, and each chunk is filtered on the context's stream as soon as its
 * copy has landed, so the copy of the second chunk overlaps the filtering
 * of the first (the filter
 * acts on every vector separately; the paper has no counterpart, it
 * concerns only where the block lives).  On return X holds p_m(H) X_host
 * and no copy is in flight.  X_host should be page-locked for the copies to
 * overlap; pageable memory gives the same result without the overlap.
 * Parameters and errors as sq3_cheb_filter (SQ3_ECUDA if a copy fails). */
int sq3_cheb_filter_from_host(sq3_ctx* ctx, const void* X_host, void* X, int Ns,
                              int degree, double a, double b, double a0, sq3_prec prec);

/* Orthonormalise X in place by Cholesky QR: S = X^T X = R^T R (R upper
 * triangular, FP64 Cholesky on the device), X <- X R^{-1} (Sec. 4: "followed
 * by orthonormalization"; the method is this library's reading).  In
 * SQ3_MIXED the step is applied twice (CholQR2).  Errors: SQ3_ENOTPD. */
int sq3_orthonormalise(sq3_ctx* ctx, void* X, int Ns, sq3_prec prec);

/* Hs = X^T H X, symmetrised, written to the device Ns x Ns double array Hs
 * (Sec. 3, Eq. (DsHsRelation): H_ij = <phi_i|H|phi_j>). */
int sq3_project(sq3_ctx* ctx, const void* X, int Ns, sq3_prec prec,
                double* Hs);

/* Density kernel from a subspace Hamiltonian (Sec. 4):
 *   Hhat = (Hs - chi I)/xi; T_0 = I, T_1 = Hhat, T_{j+1} = 2 Hhat T_j - T_{j-1}
 *   (Eq. (ThreeTermRecurrenceRelation)); moments m_j = tr T_j;
 *   c_j(mu), d_j, e_j by Chebyshev-Gauss quadrature of Eq. (ChebyshevCoeff)
 *   with M = max(1024, 8(npl+1)) nodes; mu by multisection (the bracket
 *   shrinks 64-fold per round, to double precision) on
 *   2 sum'_j c_j(mu) m_j = Ne (Eq. (FermiLevelCalc));
 *   Ds = sum'_j c_j T_j (Eq. (ChebyshevExpansion));
 *   E_band = 2 sum'_j d_j m_j; E_ent = 2 sigma sum'_j e_j m_j.
 * prec: SQ3_FP64 runs the recurrence in FP64; SQ3_MIXED keeps T_j in FP32
 * with BF16-split tensor-core products (the Fermi level in FP64; traces and
 * Ds summed in FP64).
 * Hs: device Ns x Ns double (symmetric).  kT: sigma in Ha.  bounds_in: HOST
 * pointer to {chi, xi} to use as given, or NULL to estimate them with a
 * 40-step Lanczos on Hs (extremal Ritz values widened by their residual
 * bounds, then xi *= 1.001).  D: device Ns x Ns double output (may be NULL).
 * out: HOST array of 6 doubles receiving {mu, E_band, E_ent, chi, xi,
 * 2 tr Ds}.  Requires npl >= 1 and 0 < Ne < 2 Ns.
 * Errors: SQ3_EINVAL, SQ3_ENOCONV (the initial bracket holds no root, or the
 * moments exceed the bound |m_j| <= Ns by more than 1e-6 relative, which
 * means the spectrum left [-1, 1]). */
int sq3_kernel_from_hs(sq3_ctx* ctx, const double* Hs, int Ns, int npl,
                       double kT, double Ne, sq3_prec prec,
                       const double* bounds_in, double* D, double* out);

/* The density kernel of sq3_kernel_from_hs with two options (Sec. 4 picks
 * n_pl by hand; Sec. 5 notes that the degree needed falls as T rises):
 * - npl < 1: the degree is chosen after the spectral bounds are known, as
 *   sq3_fermi_degree(kT, xi, fermi_tol) (capped at 1000); *npl_used (HOST,
 *   may be NULL) receives the degree used.
 * - eval_mode SQ3_EVAL_PATERSON_STOCKMEYER: the same polynomial
 *   sum'_j c_j T_j(Hhat) evaluated with O(sqrt(npl)) matrix products: s =
 *   ceil(sqrt(2 npl)) baby steps T_0..T_s, giant steps T_{qs} = T_q(T_s)
 *   (the Chebyshev composition identity) for the moments m_{qs+r} =
 *   2 tr(T_{qs} T_r) - m_{qs-r}, and Ds = sum_q A_q T_q(T_s) by Clenshaw's
 *   recurrence in T_s with A_q = sum_{r<s} alpha_{qr} T_r
 *   ((s - 1) + 2 floor(npl/s) - 1 products instead of npl - 1 in FP64, or
 *   ceil(npl/2) + 1 for SQ3_MIXED's recurrence with the product identity);
 *   equal to the recurrence up to rounding.  With SQ3_MIXED the matrices are
 *   FP32 and the products tcgen05 GEMMs of BF16 pieces, as the mixed
 *   recurrence.
 * Other arguments and errors as sq3_kernel_from_hs. */
#define SQ3_EVAL_RECURRENCE 0
#define SQ3_EVAL_PATERSON_STOCKMEYER 1
int sq3_kernel_from_hs_ex(sq3_ctx* ctx, const double* Hs, int Ns, int npl, double fermi_tol,
                          int eval_mode, double kT, double Ne, sq3_prec prec,
                          const double* bounds_in, double* D, double* out, int* npl_used);

/* sq3_project followed by sq3_kernel_from_hs: the density-kernel step of one
 * SQ3 iteration.  Hs_out (device, may be NULL) receives Hs. */
int sq3_density_kernel(sq3_ctx* ctx, const void* X, int Ns, int npl,
                       double kT, double Ne, sq3_prec prec,
                       const double* bounds_in, double* Hs_out, double* D,
                       double* out);

/* rho_k = (2/dV) sum_i X_ki (X Ds)_ki (Sec. 3, Eq. (phi_tilde) and
 * Eq. (density:NewForm)); X Ds is formed tile by tile and never stored.
 * D: device Ns x Ns double, symmetric (the density kernel is); the mixed
 * path reads its upper triangle only (x D x^T = x B x^T with the triangular
 * B = 2 triu(D, 1) + diag(D)), the FP64 path all of it.  rho: device N
 * doubles (overwritten). */
int sq3_density(sq3_ctx* ctx, const void* X, const double* D, int Ns,
                sq3_prec prec, double* rho);
/* (sq3_density returns SQ3_ENONFINITE when rho holds a NaN or infinity,
 * i.e. when X or D did; sq3_kernel_from_hs likewise when D or one of its
 * scalar outputs is not finite.) */

/* ---- Self-consistent-field pieces (no Hamiltonian or potential needed;
 * the grid must be set).  All arrays are device arrays of N doubles in grid
 * order (x fastest), owned by the caller.  Each call returns after its work
 * on the context's stream is done.  Every sum runs in a fixed order, so
 * repeated calls agree bit for bit. ---- */

/* Electrostatic potential (Sec. 2, Eq. (poisson)): phi with
 * -L_h phi = 4 pi (rho + b - mean(rho + b)), L_h the grid's finite-difference
 * Laplacian (the one of the Hamiltonian), solved exactly in the real Fourier
 * basis of the grid (in which L_h is diagonal); phi has zero mean (the
 * constant mode is dropped: a neutral total charge fixes phi up to a
 * constant).  b may be NULL (phi of rho alone).  phi may alias rho or b.
 * Errors: SQ3_EINVAL (null rho or phi), SQ3_ENOTSETUP, SQ3_ENOMEM,
 * SQ3_ECUDA. */
int sq3_poisson(sq3_ctx* ctx, const double* rho, const double* b, double* phi);

/* Effective potential V_eff = phi[rho + b] + V_xc[rho] (Sec. 2,
 * Eq. (KSeqn) and Eq. (poisson)) with the LDA: Slater exchange and the
 * Perdew-Wang 1992 correlation of the spin-unpolarised electron gas, rho
 * clamped below at 1e-14.  veff: output (may alias rho).  phi: optional
 * output of the electrostatic potential (NULL = not returned; must not
 * alias rho, b or veff).  b may be NULL.  terms: optional HOST array of 3
 * doubles receiving E_xc = int eps_xc rho, int V_xc rho and
 * 1/2 int (b - rho) phi (the terms of the free energy that depend on rho;
 * integrals are sums times the grid's volume element).  Feed veff to
 * sq3_set_potential for the next iteration.
 * Errors: SQ3_EINVAL, SQ3_ENOTSETUP, SQ3_ENOMEM, SQ3_ECUDA,
 * SQ3_ENONFINITE (a term is not finite). */
int sq3_effective_potential(sq3_ctx* ctx, const double* rho, const double* b,
                            double* veff, double* phi, double* terms);

/* Free energy (Sec. 3, Eq. (FreeEnergy:NewForm); Sec. 2,
 * Eq. (ON:FreeEnergy)):
 *   F = E_band + E_xc[rho] - int V_xc[rho] rho + 1/2 int (b - rho) phi[rho + b]
 *       - E_self + E_ent,
 * with the overlap correction E_c = 0 (the pseudocharges b are the nuclei's
 * charges themselves).  rho: the electron density of the iteration that gave
 * E_band and E_ent (sq3_density, sq3_density_kernel); b: the pseudocharge
 * density (sum b dV = -N_e); e_self: the pseudocharges' self energy, which
 * the caller knows in closed form (Z^2 / (sqrt(2 pi) r_c) per Gaussian).
 * out: HOST array of 4 doubles: F, E_xc, int V_xc rho, 1/2 int (b - rho) phi.
 * Errors: as sq3_effective_potential. */
int sq3_free_energy(sq3_ctx* ctx, const double* rho, const double* b,
                    double e_band, double e_ent, double e_self, double* out);

/* Density mixer (Sec. 5 cites periodic Pulay mixing with a Kerker
 * preconditioner).  sq3_mixer_setup (re)starts it: history = number of
 * past differences kept (1..8), period = a Pulay extrapolation every
 * period-th step (1 = every step), beta = mixing parameter (> 0), k0 =
 * Kerker wave number in 1/bohr (<= 0: no preconditioner).  Its device
 * state is (3 + 2 history) N doubles, held by the context until it is
 * destroyed; sq3_setup_grid stops the mixer.
 * sq3_mixer_step takes one step from the input x_in of an iteration and its
 * output x_out (device, N doubles each) and writes the next input x_next
 * (may alias x_in or x_out).  With f = x_out - x_in and the differences
 * DX, DF of the previous inputs and residuals: every period-th step that
 * has a history, x_next = x_bar + beta K f_bar with x_bar = x_in - DX c,
 * f_bar = f - DF c and c the least-squares solution of DF c ~ f (normal
 * equations by Cholesky; a difference that depends linearly on the earlier
 * ones, pivot below 1e-12 of its diagonal, is dropped); otherwise
 * x_next = x_in + beta K f.  K: the Kerker preconditioner below, or the
 * identity.  Errors: SQ3_EINVAL, SQ3_ENOTSETUP (no grid, or no
 * sq3_mixer_setup since the last grid), SQ3_ENOMEM, SQ3_ECUDA. */
int sq3_mixer_setup(sq3_ctx* ctx, int history, int period, double beta, double k0);
int sq3_mixer_step(sq3_ctx* ctx, const double* x_in, const double* x_out,
                   double* x_next);

/* Kerker preconditioner of the density mixing (Sec. 5 cites the real-space
 * Kerker preconditioner): out = K r with K(G) = G^2 / (G^2 + k0^2) on the
 * periodic cell's reciprocal vectors (K(0) = 0: the result has zero mean),
 * applied in the real Fourier basis of the grid.  k0 > 0 in 1/bohr.  out
 * may alias r.  Errors: SQ3_EINVAL, SQ3_ENOTSETUP, SQ3_ENOMEM, SQ3_ECUDA. */
int sq3_kerker(sq3_ctx* ctx, const double* r, double* out, double k0);

/* Rigorous bounds of the spectrum of the context's H (grid and potential
 * set): out[0] = min V + (lower Gershgorin bound of V_nl), out[1] = the
 * largest eigenvalue of the FD kinetic operator -1/2 L_h over the grid's
 * frequencies + max V + (upper Gershgorin bound of V_nl, from the overlaps
 * of the projectors).  out: HOST array of 2 doubles.  Host arithmetic on
 * values the set-up calls keep; no GPU work.  The upper bound is the b of
 * the Chebyshev filter (Sec. 4: the CheFSI filter needs an upper bound of
 * the spectrum).  Errors: SQ3_EINVAL, SQ3_ENOTSETUP. */
int sq3_hamiltonian_bounds(sq3_ctx* ctx, double* out);

/* Atom-centred Gaussians on the grid (device output, N doubles):
 *   out(x) = sum_J q_J sum_images exp(-|x - R_J - images|^2 / width^2)
 *            [/ (pi^{3/2} width^3) when normalised != 0],
 * then, when total != 0, rescaled so that sum out dV = total.  With
 * q_J = -Z, width = r_c, normalised and total = -Ne this is the Gaussian
 * pseudocharge density b of the nuclei (Sec. 2, Eq. (poisson); its
 * potential is the local pseudopotential -Z erf(r/r_c)/r per atom); with
 * q = NULL (all 1) and total = Ne the atomic-superposition starting
 * density; with q = NULL, total = 0 and normalised = 0 one radial
 * descriptor of the learned starting density.  pos: HOST natoms x 3
 * positions (bohr; any real values, the cell is periodic).  q: HOST natoms
 * weights or NULL.  sum_out: HOST, receives sum out dV before rescaling
 * (may be NULL).  Images are summed while the Gaussian exceeds exp(-784).
 * Errors: SQ3_EINVAL, SQ3_ENOTSETUP, SQ3_ENOMEM, SQ3_ECUDA, SQ3_ENONFINITE. */
int sq3_atom_gaussians(sq3_ctx* ctx, int natoms, const double* pos, const double* q,
                       double width, int normalised, double total, double* out,
                       double* sum_out);

/* Hellmann-Feynman forces on the nuclei (Sec. 3, Eq. (force:NewForm); Sec. 2,
 * Eq. (ON:forces)) for the Gaussian pseudocharges of sq3_atom_gaussians
 * (charge -Z, width rc, rescaled to sum b dV = -Ne) and the context's
 * projectors:
 *   f_I = sum_x grad b_I(x) phi(x) dV
 *         + 4 sum_{p of I} gamma_p (X^T c_p)^T D (X^T grad_h c_p),
 * the second line being the nonlocal term -4 sum gamma (c . u_i)
 * (c . grad_h u~_i) of Eq. (force:NewForm) with u~ = X D, rewritten by the
 * antisymmetry of the periodic FD first derivative grad_h (of the
 * Laplacian's order); f_sc = 0 (E_self is constant, E_c = 0).
 * phi: device N doubles, the electrostatic potential of rho + b
 * (sq3_effective_potential's phi).  X: device N x Ns block (precision's
 * type), D: device Ns x Ns density kernel (both ignored, may be NULL,
 * without projectors).  atom_of: HOST array of n_proj atom indices (NULL
 * without projectors).  forces: HOST natoms x 3 (Ha/bohr).  parts: HOST
 * natoms x 3 x 2 {local, nonlocal} or NULL.  The first call after
 * sq3_set_projectors tabulates grad_h c on the host.
 * Errors: SQ3_EINVAL, SQ3_ENOTSETUP, SQ3_ENOMEM, SQ3_ECUDA, SQ3_ENONFINITE. */
int sq3_forces(sq3_ctx* ctx, int natoms, const double* pos, double Z, double rc, double Ne,
               const double* phi, const void* X, const double* D, int Ns, sq3_prec prec,
               const int* atom_of, double* forces, double* parts);

/* Velocity Verlet for the QMD of the nuclei (Sec. 5 runs QMD on the forces
 * of Eq. (force:NewForm)); host arithmetic on HOST arrays, no GPU work.
 * A step from (R, V, F(R)) is: phase 0, V += dt F / (2 m), R += dt V; the
 * caller then computes F at the new R (SCF and sq3_forces); phase 1,
 * V += dt F / (2 m), and when ke_target > 0 the velocities are rescaled
 * to that kinetic energy (the isokinetic ensemble the paper's QMD uses,
 * held by rescaling after every step).  R, V, F: natoms x 3 (bohr,
 * bohr per atomic time unit, Ha/bohr); masses: natoms electron masses;
 * dt in atomic time units.  Errors: SQ3_EINVAL. */
int sq3_verlet(int natoms, const double* masses, double dt, double* R, double* V,
               const double* F, int phase, double ke_target);

/* ---- Batched filtering of many independent cells (the paper has no
 * counterpart: throughput for many uneven cells on one GPU).  Each cell has
 * its own periodic grid (12th-order FD Laplacian), local potential and FP32
 * block; one Chebyshev filter (as sq3_cheb_filter with SQ3_MIXED and no
 * projectors, equal up to FP32 rounding) of every cell runs as ONE
 * persistent launch: CTAs claim (cell, vector) items from a device counter,
 * largest cells first, and take the vector through all of its filter
 * steps, so its iterates stay in L2 between steps (no CTA waits on
 * another); the launch is captured once into a CUDA graph and replayed;
 * the tile height and the resident CTAs per SM are chosen by
 * sq3_batch_autotune. ---- */
typedef struct sq3_batch sq3_batch;
int sq3_batch_create(int device, void* cuda_stream, sq3_batch** out);
/* Releases the batch's work blocks and FP32 potentials (not the cells'
 * blocks, which stay the caller's). */
void sq3_batch_destroy(sq3_batch* batch);
/* Adds a cell: grid nx x ny x nz over Lx x Ly x Lz (nx a multiple of 4,
 * 16 <= nx <= 512, ny, nz >= 6), V device N doubles (converted to FP32 and
 * kept), X device N x Ns floats (16-byte aligned; filtered in place by
 * sq3_batch_filter, stays the caller's), filter degree 1..256.  Returns
 * the cell's index (>= 0) or SQ3_EINVAL / SQ3_ENOMEM / SQ3_ECUDA. */
int sq3_batch_add_cell(sq3_batch* batch, int nx, int ny, int nz, double Lx, double Ly,
                       double Lz, const double* V, float* X, int Ns, int degree);
/* Filter bounds of a cell (a0 < a < b), as sq3_cheb_filter. */
int sq3_batch_set_bounds(sq3_batch* batch, int cell, double a, double b, double a0);
/* X_c <- p_{m_c}(H_c) X_c for every cell; returns after the work is done.
 * The first call after cells were added captures the graph. */
int sq3_batch_filter(sq3_batch* batch);
/* Times each candidate launch shape (1 or 2 CTAs per SM; every cell's
 * tile height as chosen or halved) with one graph replay each, on copies
 * of the cells' blocks (which are put back), and keeps the fastest;
 * *ctas_per_sm and *ty_divisor (HOST, may be NULL) receive the choice. */
int sq3_batch_autotune(sq3_batch* batch, int* ctas_per_sm, int* ty_divisor);

/* ---- Learned starting density (the paper has no counterpart: it does
 * not say how each SCF starts).  A multilayer perceptron over atom-centred
 * Gaussian descriptors predicts the density of a cell from its atom
 * positions; it is trained on self-consistent densities the method itself
 * produced.  Per grid point x of the context's grid:
 *   d_k(x) = log(1 + sum_J sum_images exp(-|x - R_J|^2 / w_k^2) / m_k),
 *            m_k = natoms pi^{3/2} w_k^3 / Omega (the sum's mean over the
 *            cell; the logarithm keeps the narrow widths, a hundred times
 *            their mean near an atom, from saturating the first layer)
 *   h1 = tanh(W1 d + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3)
 *        (128 units each), y = softplus(w4 . h3 + b4),
 *   rho(x) = Ne y(x) / (sum_x y dV);
 * loss L = sum_x (rho(x) - rho_ref(x))^2 dV.  The three matrix products of
 * each pass and the weight gradients run on the tensor cores with BF16
 * operands and FP32 accumulation; activations, the output layer and the
 * reductions in FP32/FP64; Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32
 * master weights.  Parameters, as one FP32 array: W1 [128][F] row-major,
 * b1 [128], W2 [128][128], b2, W3 [128][128], b3, w4 [128], b4 [1]. ---- */
typedef struct sq3_mlp sq3_mlp;

/* A model for the context's grid with n_features (1..16) descriptor widths
 * (HOST array, bohr), weights initialised from `seed` (N(0, 1/fan_in),
 * biases 0).  Errors: SQ3_EINVAL, SQ3_ENOTSETUP (no grid), SQ3_ENOMEM. */
int sq3_mlp_create(sq3_ctx* ctx, int n_features, const double* widths, int seed,
                   sq3_mlp** out);
/* Release a model; it may be released after its context (it does not
 * touch the context), but no other call may use it once the context is
 * destroyed. */
void sq3_mlp_destroy(sq3_mlp* mlp);
/* Number of parameters (128 F + 33,281). */
int sq3_mlp_num_params(const sq3_mlp* mlp);
/* HOST arrays of sq3_mlp_num_params floats.  Setting resets Adam. */
int sq3_mlp_set_params(sq3_mlp* mlp, const float* params);
int sq3_mlp_get_params(sq3_mlp* mlp, float* params);
/* Descriptors of the grid for natoms positions (HOST natoms x 3, bohr);
 * the features every later predict/gradient/train call uses. */
int sq3_mlp_features(sq3_mlp* mlp, int natoms, const double* pos);
/* rho (device, N doubles) = the model's density with Ne electrons. */
int sq3_mlp_predict(sq3_mlp* mlp, double Ne, double* rho);
/* Loss against rho_ref (device, N doubles) and its gradient (HOST array of
 * num_params doubles, or NULL); rho_scratch: device N doubles receiving
 * the prediction.  Errors: SQ3_EINVAL, SQ3_ENOTSETUP (no features),
 * SQ3_ENONFINITE. */
int sq3_mlp_gradient(sq3_mlp* mlp, const double* rho_ref, double Ne, double* rho_scratch,
                     double* loss, double* grad);
/* One Adam step of size lr on the gradient of sq3_mlp_gradient; loss:
 * HOST, the loss before the step. */
int sq3_mlp_train_step(sq3_mlp* mlp, const double* rho_ref, double Ne, double lr,
                       double* rho_scratch, double* loss);

/* Starting density of a QMD step by extrapolation (the paper leaves the
 * SCF's start open): out = max(prev + a - b, 0) rescaled to Ne electrons,
 * with prev the previous step's converged density and a, b a model density
 * (the learned one, or the atomic superposition) at the new and the
 * previous positions, so that the model's systematic error cancels and its
 * response to the atoms' motion remains.  All device arrays of N doubles;
 * out may alias prev.  Errors: SQ3_EINVAL, SQ3_ENOTSETUP, SQ3_ENONFINITE. */
int sq3_extrapolate_density(sq3_ctx* ctx, const double* prev, const double* a,
                            const double* b, double Ne, double* out);

/* ---- Self-consistent-field driver (Sec. 2: the SCF loop; Sec. 4: the SQ3
 * iteration inside each SCF iteration; Sec. 5: periodic Pulay mixing with a
 * Kerker preconditioner). ---- */
typedef struct sq3_scf_params {
  int Ns;            /* auxiliary vectors (columns of X)                    */
  int degree;        /* Chebyshev filter degree m                          */
  int npl;           /* Fermi-operator degree; <= 0: chosen per iteration
                        by sq3_fermi_degree(kT, xi, fermi_tol)            */
  int first_passes;  /* filter + Cholesky QR passes in the first iteration */
  int passes;        /* ... in every later iteration                       */
  int max_iter;      /* SCF iterations before SQ3_ENOCONV                  */
  int mix_history;   /* mixer history (1..8)                               */
  int mix_period;    /* Pulay extrapolation every mix_period-th step       */
  double kT;         /* sigma (Ha)                                         */
  double Ne;         /* electrons, 0 < Ne < 2 Ns                           */
  double tol;        /* stop when sum |rho_out - rho_in| dV / Ne < tol     */
  double e_self;     /* self energy of the pseudocharges (Ha)              */
  double mix_beta;   /* mixing parameter                                   */
  double kerker_k0;  /* Kerker wave number (1/bohr); <= 0: none            */
  double fermi_tol;  /* occupation tolerance of the adaptive degree        */
  double filter_cut; /* first iteration without chi0/xi0: damped interval
                        starts this fraction of the spectral width above its
                        lower bound (<= 0: 0.05)                           */
  double chi0, xi0;  /* xi0 > 0: spectral centre/half-width of the starting
                        block's Hs (e.g. the previous solve's), which sets
                        the first iteration's damped interval              */
  double cut_shift;  /* the damped interval starts this far (Ha) above the
                        largest Ritz value (0: at it)                      */
  int kernel_eval;   /* SQ3_EVAL_RECURRENCE or SQ3_EVAL_PATERSON_STOCKMEYER,
                        as sq3_kernel_from_hs_ex                          */
  int reserved;
} sq3_scf_params;

typedef struct sq3_scf_result {
  int iterations;    /* SCF iterations run                                 */
  int converged;     /* 1 when err < tol                                   */
  int npl_last;      /* Fermi-operator degree of the last iteration        */
  int reserved;
  double F;          /* free energy of the last output density (Ha)        */
  double e_band, e_ent, mu;
  double e_xc, vxc_rho, e_es;   /* the density terms of F                 */
  double err;        /* last sum |rho_out - rho_in| dV / Ne               */
  double chi, xi;    /* Lanczos bounds of the last Hs                      */
  double b_up;       /* the filter's upper spectral bound, last iteration  */
} sq3_scf_result;

/* Values per iteration in the history array of sq3_scf_solve:
 * err, mu, E_band, E_ent, F, npl, wall ms, chi, xi. */
#define SQ3_SCF_HIST 9

/* Converged SCF solve of one cell from a starting density and block.
 * Each iteration: V_eff = phi[rho_in + b] + V_xc[rho_in] (as
 * sq3_effective_potential) becomes the context's potential; the filter's
 * upper bound is sq3_hamiltonian_bounds' out[1]; `passes` (first_passes in
 * the first iteration) times X <- p_m(H) X and Cholesky QR, the damped
 * interval [a, b] with a = lambda_max(Hs) + cut_shift, a0 = lambda_min(Hs)
 * of the latest block's Lanczos bounds (the first pass of the first iteration uses
 * chi0/xi0, or filter_cut); Hs = X^T H X, its 40-step Lanczos bounds, the
 * density kernel Ds (sq3_kernel_from_hs with those bounds), rho_out
 * (sq3_density), err = sum |rho_out - rho_in| dV / Ne, F of rho_out
 * (sq3_free_energy with e_self); then, unless err < tol, rho_in is mixed
 * (sq3_mixer_setup(mix_history, mix_period, mix_beta, kerker_k0) at the
 * start, sq3_mixer_step each iteration).  Projectors, if any, are the
 * context's (sq3_set_projectors) and stay fixed.
 * b: device N doubles, the pseudocharge density (sum b dV = -Ne).
 * rho: device N doubles; in: starting density; out: the converged output
 * density (the last mixed input when not converged).  X: device block
 * N x Ns of the precision's element type; in: starting block (random, or
 * the previous solve's); out: the last orthonormal block.  D: device Ns x Ns
 * doubles receiving the last Ds, or NULL.  res: HOST result.  history: HOST
 * array of max_iter x SQ3_SCF_HIST doubles (row per iteration), or NULL.
 * Errors: SQ3_EINVAL, SQ3_ENOTSETUP, SQ3_ENOCONV (max_iter reached; res
 * holds the last iteration), and every error of the calls above. */
int sq3_scf_solve(sq3_ctx* ctx, const sq3_scf_params* params, const double* b,
                  double* rho, void* X, sq3_prec prec, double* D,
                  sq3_scf_result* res, double* history);

/* Self-test of the device-side failure path (no counterpart in the paper):
 * one CTA waits on an mbarrier that nothing completes, through the bounded
 * wait (about one second of wall time) that every TMA and tensor-core wait
 * of the library uses; the wait runs out, the kernel records a timeout in
 * the context's status word and returns, and the host reads it.  Returns
 * SQ3_ETIMEOUT when the path works (the status word is cleared, so the
 * context stays usable), SQ3_OK if the wait did not run out, SQ3_EINVAL for
 * a NULL context, SQ3_ECUDA on a CUDA error.  No fault, trap or hang. */
int sq3_selftest_timeout(sq3_ctx* ctx);

/* Per-stage timing (tracing).  When enabled, the library records a CUDA
 * event pair on the context's stream around the launches of each stage of
 * the path; sq3_profile_read synchronises the stream, writes for each stage
 * s < n_stages the summed device time ms[s] (milliseconds) and the number of
 * kernel launches launches[s], clears the records, and returns the number of
 * stages the library knows (SQ3_N_STAGES).  Stage order:
 *   0 stencil/filter step, 1 nonlocal projection, 2 Gram X^T X,
 *   3 Cholesky, 4 triangular inverse, 5 X R^{-1}, 6 X^T (H X),
 *   7 Lanczos, 8 Chebyshev recurrence GEMM, 9 Fermi level/coefficients,
 *   10 Ds accumulation, 11 density X Ds row-dot, 12 BF16 split,
 *   13 device copies, 14 nonlocal pass (apply and next-step projection).
 * Host pointers; either may be NULL. */
#define SQ3_N_STAGES 15
int sq3_profile_enable(sq3_ctx* ctx, int enable);
int sq3_profile_read(sq3_ctx* ctx, double* ms, long long* launches,
                     int n_stages);

/* Allocation-free spectral bounds of a subspace Hamiltonian.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot let a library allocate device memory: processes that reserve
 * all of HBM up front for their own arena and forbid allocations by
 * libraries, and loops where a device allocation, which may synchronise the
 * whole device, would stall work on other streams.  It computes the same
 * bounds as the Lanczos step of sq3_kernel_from_hs with bounds_in == NULL:
 * 40 Lanczos steps with full reorthogonalisation on the symmetric Hs,
 * extremal Ritz values widened by their residual bounds, then xi *= 1.001,
 * and writes {chi, xi} to `bounds`.
 *
 * Hs: device Ns x Ns double, symmetric (caller-owned).  bounds: DEVICE
 * array of 2 doubles (caller-owned).  cuda_stream: the cudaStream_t the work
 * is ordered on (NULL = legacy default stream); the call returns after that
 * stream has finished the work.  It needs no context, and calls no
 * cudaMalloc, cudaFree or allocating routine: its scratch is a fixed
 * device array inside the library, sized for Ns <= 8192 and 40 steps
 * (349,304 doubles: 2.79 MB, 2.66 MiB), which every GPU that loads the
 * library holds until the process exits.  The first call on a device looks
 * up that array's device address (with the device current), and so does the
 * first call after the device's context was reset or created anew (the
 * address is cached per context); make that first call before any stream
 * capture.  An error left pending by earlier, unrelated asynchronous work
 * is cleared on entry and not reported by this call.  All
 * calls share the array and it keeps the previous call's contents, so two
 * calls whose GPU work overlaps (other streams, other host threads) race
 * and give wrong bounds: serialise them.
 * Errors: SQ3_EINVAL (null pointer, Ns < 1, or Ns > 8192), SQ3_ECUDA. */
int sq3_lanczos_bounds_noalloc(const double* Hs, int Ns, double* bounds,
                               void* cuda_stream);

/* Degree of the Chebyshev expansion of the Fermi function (Sec. 4,
 * Eq. (ChebyshevExpansion); Sec. 5 notes that the degree needed falls as the
 * temperature rises).  Host-only arithmetic, no GPU work: the Fermi function
 * of width sigma (Ha) is analytic except at its poles mu +- i pi sigma (2k + 1),
 * so on [chi - xi, chi + xi] its Chebyshev coefficients decay at least like
 * rho^-j, rho = a + sqrt(1 + a^2), a = pi sigma / xi (the Bernstein ellipse
 * through the nearest pole, for mu anywhere in the interval).  Returns
 * ceil(ln(1 / tol) / ln rho), at least 1: the degree at which the expansion
 * error of the occupations is below tol for every mu in the interval.
 * xi: half-width of the spectrum of Hs (the xi sq3_kernel_from_hs reports);
 * tol in (0, 1).  Degrees above 1000 exceed what sq3_kernel_from_hs accepts.
 * Errors: SQ3_EINVAL (sigma <= 0, xi <= 0, tol outside (0, 1), or a degree
 * beyond 2^31). */
int sq3_fermi_degree(double sigma, double xi, double tol);

/* Human-readable name of a status code (static string). */
const char* sq3_status_string(int status);

/* Library build string: version and target architecture (static string). */
const char* sq3_version(void);

/* Name of the last CUDA runtime error behind an SQ3_ECUDA returned on the
 * calling host thread ("none" if there was none; static string). */
const char* sq3_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SQ3_H */
