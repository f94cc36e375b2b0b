/*
 * pwh.h — C ABI of libpwh: the plane-wave pseudopotential Kohn–Sham Hamiltonian
 * applied to a block of bands, H|psi>, and a block Davidson eigensolver built on
 * it, on one NVIDIA GB300 (sm_103a).
 *
 * The operator is the norm-conserving form (overlap S = 1) of Eq. pauli_ks
 * (Sec. "Fully relativistic projector augmented-wave method"): the kinetic term
 * p^2/2m acting on the FFT mesh, the local potential V_LOC(r), and the separable
 * nonlocal term sum_{ij} D_ij |beta_i><beta_j|.  In the plane-wave basis
 * c_{k,n}(G) (Sec. "New parallelization levels"), Hartree atomic units:
 *
 *   (H psi)_G = 1/2|k+G|^2 psi_G + sum_{G'} Vt(G-G') psi_{G'}
 *             + sum_{ij} beta_i(G) D_ij <beta_j|psi>
 *
 * where Vt is the discrete Fourier transform of V sampled on the FFT grid.
 *
 * Conventions for every entry point:
 *  - Every call validates its arguments and returns a pwh_status; no C++
 *    exception crosses the ABI.  On failure pwh_last_error() gives a message
 *    (thread-local, valid until the next call on the same thread).
 *  - Complex numbers are interleaved (re, im) pairs of doubles (complex128).
 *  - Band blocks are column-major: band b occupies elements [b*ld, b*ld + npw).
 *  - Plane waves are in the public order of pwh_get_miller(): ascending |k+G|^2,
 *    plane waves whose |k+G|^2 agree to a relative 1e-10 ordered
 *    lexicographically by signed Miller indices (the reproducible ordering of
 *    Sec. "Large-record data file format").
 *  - The caller owns psi / hpsi / eigenvalue buffers; the library owns its
 *    copies of V, beta, D, index maps and workspaces (freed by
 *    pwh_destroy_system).
 *  - All device work is ordered on the stream given at creation.  Calls on one
 *    system are not thread-safe; different systems are independent.
 */
#ifndef PWH_H
#define PWH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pwh_system pwh_system; /* opaque, library-owned */

typedef enum {
  PWH_OK = 0,
  PWH_ERR_ARG = 1,           /* invalid argument (null pointer, size, layout) */
  PWH_ERR_CUDA = 2,          /* a CUDA runtime call or kernel failed */
  PWH_ERR_OOM = 3,           /* device allocation failed */
  PWH_ERR_NOT_CONVERGED = 4, /* eigensolver stopped at max_iter; results written */
  PWH_ERR_NONFINITE = 5,     /* a NaN/Inf appeared in a residual */
  PWH_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
  PWH_ERR_STATE = 7          /* call out of order (e.g. apply before set_potential) */
} pwh_status;

typedef enum {
  PWH_FP64 = 0,       /* every step to FP64 accuracy: FP64 arithmetic, except
                         the FFT passes of the compiled cubic boxes (edges 30,
                         36, 40, 48, 50, 60, 72, 80, 90, 96, 120, 144), which
                         compute in double-float (pairs of FP32 numbers, 48
                         significant bits, about 2^-46 relative rounding per
                         operation), and the large GEMMs (exact integer-slice
                         products on the tensor cores) */
  PWH_MIXED = 1,      /* FFT + potential in FP32; projector GEMMs on the BF16
                         tensor cores with FP32 accumulation, each operand split
                         into two BF16 terms (hi*hi + hi*lo + lo*hi, about 16
                         significant bits); inputs and outputs stay complex128 */
  PWH_MIXED_FAST = 2  /* as PWH_MIXED with one BF16 term per operand (8 bits) */
} pwh_precision;

typedef struct {
  double lattice[9];  /* rows a1, a2, a3 in bohr (row-major 3x3) */
  double kpoint[3];   /* k in fractional units of the reciprocal vectors b_i */
  double ecut_ha;     /* wavefunction cutoff, Hartree: 1/2|k+G|^2 <= ecut_ha */
  int32_t fft[3];     /* FFT grid; 0 => smallest even 2,3,5-smooth N_i >= 4*mmax_i+1,
                         the alias-free box for G_max = 2 G_c (Sec. "Advanced
                         implementation of exact (Fock) exchange") */
  int32_t precision;  /* pwh_precision used by pwh_apply_h */
  void* stream;       /* cudaStream_t; NULL = legacy default stream */
} pwh_system_desc;

/* Build the plane-wave sphere {G : 1/2|k+G|^2 <= ecut_ha} (membership decided in
 * FP64 from integer Miller indices), its public ordering, the FFT box, the
 * z-stick decomposition used by the FFT passes and the kinetic diagonal.  Host
 * work plus device uploads on desc->stream.  *out receives a new system.
 * Errors: PWH_ERR_ARG (null, non-positive cutoff, singular lattice, an explicit
 * FFT size that is odd, not 2,3,5-smooth, above 512 or below 4*mmax+1),
 * PWH_ERR_OOM, PWH_ERR_CUDA. */
pwh_status pwh_create_system(const pwh_system_desc* desc, pwh_system** out);

/* Synchronize the system's stream and free everything it owns.  NULL is a no-op. */
pwh_status pwh_destroy_system(pwh_system* sys);

/* npw = number of plane waves; fft_out = (N1, N2, N3); nsticks = number of
 * nonzero z-columns of the sphere.  Any output pointer may be NULL. */
pwh_status pwh_get_dims(const pwh_system* sys, int64_t* npw, int32_t fft_out[3],
                        int64_t* nsticks);

/* Copy the Miller indices (m1, m2, m3) of every plane wave, in public order, into
 * the host array miller[npw*3] (row-major, caller-owned). */
pwh_status pwh_get_miller(const pwh_system* sys, int32_t* miller);

/* Copy the kinetic diagonal 1/2|k+G|^2 (public order) into host kin[npw]. */
pwh_status pwh_get_kinetic(const pwh_system* sys, double* kin);

/* Set V_LOC(r): N1*N2*N3 doubles in C order (i3 fastest); grid point
 * (i1,i2,i3) is r = sum_d (i_d/N_d) a_d.  Copied in (host pointer if
 * on_device == 0, device pointer otherwise); the caller keeps ownership. */
pwh_status pwh_set_potential(pwh_system* sys, const double* v_r, int32_t on_device);

/* Set the nonlocal part: nproj projectors beta (complex128, nproj columns of
 * length npw, column-major ld = npw, public order) and D, either nproj real
 * diagonal entries (d_is_diag = 1) or an nproj x nproj complex128 Hermitian
 * matrix (column-major).  nproj = 0 removes the nonlocal term.  Copied in. */
pwh_status pwh_set_projectors(pwh_system* sys, int32_t nproj, const void* beta,
                              const void* D, int32_t d_is_diag, int32_t on_device);

/* Select the compute precision of pwh_apply_h (pwh_precision). */
pwh_status pwh_set_precision(pwh_system* sys, int32_t precision);

/* hpsi = H psi for nb bands (plus the ACE exchange term -zeta zeta^H psi when
 * pwh_set_ace has set one).  psi, hpsi: DEVICE complex128, column-major with
 * leading dimensions ld_psi, ld_hpsi >= npw; they must not overlap.
 * Asynchronous on the system's stream.  Requires pwh_set_potential first
 * (PWH_ERR_STATE otherwise).  nb = 0 is a no-op. */
pwh_status pwh_apply_h(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi,
                       void* hpsi, int64_t ld_hpsi);

/* Same as pwh_apply_h on HOST buffers (ld = npw): copies psi to the device,
 * applies H, copies hpsi back and synchronizes the stream before returning. */
pwh_status pwh_apply_h_host(pwh_system* sys, int32_t nb, const void* psi_host,
                            void* hpsi_host);

/* Internal-order entry used by the eigensolver and by tests of the passes:
 * band data already permuted to the library's stick order (see
 * pwh_get_internal_order).  Same layout rules as pwh_apply_h. */
pwh_status pwh_apply_h_internal(pwh_system* sys, int32_t nb, const void* psi,
                                int64_t ld_psi, void* hpsi, int64_t ld_hpsi);

/* Allocation-free variant of the kinetic + local-potential part of H, for
 * callers that cannot let a library allocate device memory: host codes that
 * hand all device memory to their own pool at start-up, or that call from a
 * point where the device-wide synchronisation cudaMalloc/cudaFree may cause is
 * not acceptable.  The paper has no counterpart; it is an interface addition.
 *
 * hpsi = (1/2|k+G|^2 + V_LOC) psi in FP64, bands in the library's internal
 * plane-wave order (as pwh_apply_h_internal, nonlocal term left out).  psi,
 * hpsi: device complex128, column-major, ld >= npw, caller-owned.  No cudaMalloc,
 * cudaFree or other allocating routine is called: the FFT stick buffer is a
 * fixed 32 MiB device array inside the library, held on every GPU that loads
 * the library until the process exits.  Bands are processed in batches that
 * fit it; a system whose single band needs more than 32 MiB (N3 x nsticks x 16
 * bytes) is rejected with PWH_ERR_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (every entry a call reads it first writes, so nothing
 * needs clearing); calls whose work overlaps on the GPU (different streams or
 * systems, no ordering between them) race on it.  Asynchronous on the
 * system's stream; requires pwh_set_potential (PWH_ERR_STATE otherwise). */
pwh_status pwh_apply_local_noalloc(pwh_system* sys, int32_t nb, const void* psi,
                                   int64_t ld_psi, void* hpsi, int64_t ld_hpsi);

/* Copy the permutation from internal (stick-major) to public order into host
 * int_to_pub[npw]: internal plane wave i is public plane wave int_to_pub[i]. */
pwh_status pwh_get_internal_order(const pwh_system* sys, int32_t* int_to_pub);

/* ----------------------------------------------------- real bands at k = 0 --
 * At the Gamma point a real band psi(r) has c(-G) = conj c(G), so half of the
 * sphere holds it (the Gamma-only real-wavefunction codes named in Sec.
 * "Advanced implementation of exact (Fock) exchange" and Sec. "Many-body
 * perturbation theory").  The half sphere: G = 0 and every plane wave whose
 * first nonzero Miller index (m1, then m2, then m3) is positive, in public
 * order; npw_half = (npw + 1) / 2.  The coefficient at G = 0 of a real band is
 * real; the imaginary part a caller stores there is ignored.
 *
 * *npw_half receives the size of the half sphere and, when pub_index is not
 * NULL, the host array pub_index[npw_half] the public index of each of its
 * plane waves.  The first call builds the map (host work and a small device
 * upload).  Errors: PWH_ERR_ARG when k != 0. */
pwh_status pwh_get_gamma_half(pwh_system* sys, int64_t* npw_half, int32_t* pub_index);

/* hpsi = H psi for nb real bands on the half sphere, in the system's
 * precision (pwh_set_precision).  Two real bands share one complex band
 * Psi = psi_a + i psi_b of the full sphere, so the FFTs and projector GEMMs run
 * on ceil(nb/2) bands; H psi_a and H psi_b are the conjugate-symmetric and
 * antisymmetric parts of H Psi.  psi, hpsi: DEVICE complex128, column-major,
 * ld_psi, ld_hpsi >= npw_half, not overlapping.  Asynchronous on the system's
 * stream, except that the first call after pwh_set_projectors checks (on the
 * device, then synchronizes) that the projectors keep real functions real:
 * beta_p(-G) = conj beta_p(G) to 1e-10 of max|beta| and a real D.  Errors:
 * PWH_ERR_ARG (k != 0, projectors that fail that check, ld too small),
 * PWH_ERR_STATE (no potential), PWH_ERR_OOM, PWH_ERR_CUDA.  nb = 0 is a no-op. */
pwh_status pwh_apply_h_gamma(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi,
                             void* hpsi, int64_t ld_hpsi);

/* ------------------------------------------------------------ eigensolver --
 * Block Davidson for the lowest nb eigenpairs of H: the iterative
 * diagonalisation with subspace diagonalisation of O_ij = <psi_i|O|psi_j>
 * (Sec. "New parallelization levels"), a Davidson-like algorithm [Davidson
 * 1975] (Sec. "Dynamic perturbations", optical absorption).  Each iteration:
 * Rayleigh-Ritz on span(V) (FP64 device Jacobi), Ritz vectors X and residuals
 * R = HX - X diag(theta), convergence when every ||r_n||_2 <= tol, new
 * directions t_n = K (.) r_n for the unconverged bands (K: Teter-Payne-Allan,
 * Phys. Rev. B 40, 12255 (1989), with x = (1/2|k+G|^2) / E_ref and
 * E_ref = <x_n|T|x_n> the kinetic energy of the Ritz vector), projected out of
 * V twice and orthonormalised by two Cholesky-QR passes (columns whose norm
 * fell below 1e-10 of their norm before the projection, or whose unit-diagonal
 * Cholesky pivot is below 1e-12, are dropped), restart to V = X when the subspace would exceed m_max. */
typedef enum {
  PWH_PRECOND_TPA = 0,   /* Teter-Payne-Allan diagonal preconditioner */
  PWH_PRECOND_MLP = 1,   /* TPA times exp(learned correction), see pwh_set_mlp */
  PWH_PRECOND_NONE = 2   /* t_n = r_n */
} pwh_precond;

typedef struct {
  int32_t nb;                /* eigenpairs wanted, 1..1024, <= npw */
  int32_t max_iter;          /* iteration cap (>= 1) */
  int32_t max_subspace_mult; /* m_max = max_subspace_mult * nb (>= 2, m_max <= 4096) */
  int32_t precond;           /* pwh_precond */
  int32_t mixed;             /* 0: FP64 throughout.  1: first iterate with the
                                reduced-precision H of the system's precision
                                (PWH_MIXED if the system is PWH_FP64) until
                                max ||r|| <= switch_tol, then restart from the
                                Ritz vectors with the FP64 H */
  int32_t jd_inner;          /* mixed solves only: >0 turns the FP64 phase into
                                Jacobi-Davidson steps, each band's correction
                                equation (I-XX^H)(H-theta)(I-XX^H) t = -r solved
                                by jd_inner preconditioned CG steps with the
                                reduced-precision H, then V = [X, T] and an
                                FP64 Rayleigh-Ritz; 0 = plain Davidson */
  double tol;                /* FP64 residual target (Hartree), > 0 */
  double switch_tol;         /* mixed phase target, >= tol */
} pwh_davidson_opts;

typedef struct {
  int32_t iters;             /* Rayleigh-Ritz steps taken */
  int32_t n_apply;           /* band applications of H (all precisions) */
  int32_t n_apply_fp64;      /* of which in FP64 */
  int32_t switch_iter;       /* iteration of the hand-over to FP64, -1 if none */
  double t_total_s, t_mixed_s, t_fp64_s;  /* wall time, seconds */
  double max_resid;          /* final max ||r_n||_2 */
} pwh_davidson_stats;

/* psi_io: DEVICE complex128, nb columns of length npw (ld_psi >= npw, public
 * order): starting bands in (linearly independent), eigenvectors out.
 * eig: HOST double[nb], ascending.  stats may be NULL.  Synchronous; runs on
 * the system's stream.  Returns PWH_ERR_NOT_CONVERGED at max_iter (results
 * still written), PWH_ERR_NONFINITE if a residual norm is not finite,
 * PWH_ERR_TIMEOUT if a bounded device wait gave up. */
pwh_status pwh_davidson_solve(pwh_system* sys, const pwh_davidson_opts* opts, void* psi_io,
                              int64_t ld_psi, double* eig, pwh_davidson_stats* stats);

/* Per-iteration record of the last pwh_davidson_solve on this system (a
 * diagnostic; the solver keeps it on the host, no device work). */
typedef struct {
  int32_t iter;        /* Rayleigh-Ritz step, from 1 */
  int32_t fp64;        /* 1 if the step ran in the FP64 phase */
  int32_t m;           /* subspace size of the step */
  int32_t n_above;     /* bands whose residual is above the phase's target */
  double max_resid;    /* max ||r_n||_2 after the step */
  double t_s;          /* seconds since the solve started (host clock) */
} pwh_davidson_trace_entry;

/* Copies up to cap entries of that record to out (host) and stores the number
 * of iterations recorded in *count (which may exceed cap). */
pwh_status pwh_get_davidson_trace(const pwh_system* sys, int32_t cap,
                                  pwh_davidson_trace_entry* out, int32_t* count);

/* pwh_davidson_solve with the bands in HOST memory: psi_host holds nb
 * contiguous columns of length npw (ld = npw, public order, complex128),
 * starting bands in, eigenvectors out.  The library copies them to a device
 * buffer it owns (allocated on first use, kept with the system), solves on the
 * system's stream and copies the eigenvectors back before returning.  Pinned
 * host memory gives the fastest copies; pageable memory works.  Same status
 * codes as pwh_davidson_solve; on PWH_ERR_NOT_CONVERGED the results are still
 * copied back. */
pwh_status pwh_davidson_solve_host(pwh_system* sys, const pwh_davidson_opts* opts, void* psi_host,
                                   double* eig, pwh_davidson_stats* stats);

/* pwh_davidson_solve for real bands at k = 0 (the real-wavefunction form of
 * the Gamma-only codes, Sec. "Advanced implementation of exact (Fock)
 * exchange"): psi_io holds nb real bands on the half sphere
 * (pwh_get_gamma_half: npw_half rows, public order, ld_psi >= npw_half,
 * DEVICE complex128), starting bands in, eigenvectors out (c(0) real).  Every
 * step of the complex solver runs on the half sphere: inner products are the
 * real ones, 2 Re of the complex products over the half sphere with c(0)
 * counted once (the solver stores c(0) / sqrt 2 internally); H is applied two
 * bands per complex band (pwh_apply_h_gamma).  The eigenvalues are those of
 * the complex solver at k = 0.  Same options, statistics, synchronous
 * behaviour and status codes as pwh_davidson_solve, plus the errors of
 * pwh_apply_h_gamma (k != 0, projectors that do not keep real functions
 * real). */
pwh_status pwh_davidson_solve_gamma(pwh_system* sys, const pwh_davidson_opts* opts, void* psi_io,
                                    int64_t ld_psi, double* eig, pwh_davidson_stats* stats);

/* ---------------------------------------------------- overlap operator S --
 * Ultrasoft / PAW projectors make the Kohn-Sham problem generalised,
 * H x = e S x (the S of Eq. pauli_ks, Sec. "Fully relativistic projector
 * augmented-wave method").  The separable form over the projectors of
 * pwh_set_projectors is used:
 *   S = 1 + sum_ij |beta_i> q_ij <beta_j|,   q Hermitian, S positive definite. */

/* Set q: nproj real diagonal values (q_is_diag = 1) or an nproj x nproj
 * complex128 Hermitian matrix (column-major; its Hermitian part is used), on the
 * host or the device (on_device).  Builds, once, the separable inverse square
 * root S^-1/2 = 1 + beta K beta^H (FP64: beta^H beta and two device Jacobi
 * eigendecompositions of nproj x nproj matrices, GEMMs).  From then on
 * pwh_davidson_solve and pwh_batch_davidson_solve solve H x = e S x through the
 * Loewdin form S^-1/2 H S^-1/2 (same eigenvalues; the eigenvectors returned are
 * S-orthonormal; the reported residual max ||H' phi - e phi|| is that of the
 * transformed problem, and ||H x - e S x|| <= ||S^1/2|| times it).  pwh_apply_h
 * keeps applying H.  q = NULL removes the overlap; pwh_set_projectors removes
 * it too.  Synchronous.  Errors: PWH_ERR_STATE (no projectors), PWH_ERR_ARG
 * (S not positive definite), PWH_ERR_OOM, PWH_ERR_CUDA.  The real-band solver
 * (pwh_davidson_solve_gamma) refuses a system with an overlap (PWH_ERR_ARG). */
pwh_status pwh_set_overlap(pwh_system* sys, const void* q, int32_t q_is_diag, int32_t on_device);

/* spsi = S psi for nb bands (the identity when no overlap is set), FP64.
 * psi, spsi: DEVICE complex128, public order, column-major, ld >= npw, not
 * overlapping.  Asynchronous on the system's stream. */
pwh_status pwh_apply_s(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi, void* spsi,
                       int64_t ld_spsi);

/* ------------------------------------------------ exact exchange and ACE --
 * The Fock exchange operator of Eq. Vx (Sec. "Advanced implementation of exact
 * (Fock) exchange and hybrid functionals"), Hartree units:
 *   (V_x phi)(r) = - sum_j occ_j psi_j(r) v_j(r),  v_j(G) = 4 pi rho_j(G) / |G|^2,
 *   rho_j(r) = conj(psi_j(r)) phi(r),
 * with the pair-density potentials of Eq. Poisson solved on the full FFT box
 * (the divergent G = 0 term is left out); psi_j and phi at the system's k.
 * On the default box (N_d >= 4 mmax_d + 1) the FFT route is exact. */

/* out = V_x phi for nb bands.  psi_occ: nocc occupied bands, occ: host weights
 * (finite); phi, out: nb bands; all DEVICE complex128, public order,
 * column-major, ld >= npw.  FP64.  Device scratch of (nocc + 64 MB / box + 2)
 * full boxes is allocated for the call and freed before it returns;
 * synchronous.  Cost: nb * nocc pair densities, two 3D FFTs each.  Errors:
 * PWH_ERR_ARG, PWH_ERR_OOM, PWH_ERR_CUDA. */
pwh_status pwh_exx_apply(pwh_system* sys, int32_t nocc, const void* psi_occ, int64_t ld_occ,
                         const double* occ, int32_t nb, const void* phi, int64_t ld_phi,
                         void* out, int64_t ld_out);

/* Adaptively compressed exchange (ACE, Eq. Vxace): from nocc occupied bands
 * psi_occ (DEVICE, public order, ld >= npw) with host weights occ (> 0),
 * xi_i = V_x psi_i, M = <psi_j|xi_m>, and the operator
 * alpha * sum_jm |xi_j> (M^-1)_jm <xi_m| = -zeta zeta^H (zeta = sqrt(alpha)
 * xi L^-H, -M = L L^H).  The system keeps zeta; from then on pwh_apply_h, the
 * eigensolvers and the real-band routes add -zeta zeta^H psi to H psi (two
 * GEMMs in the system's precision: FP64-equivalent or FP32-equivalent on the
 * tensor cores).  alpha: the exchange fraction (e.g. 0.25).  The operator
 * equals alpha V_x on the span of psi_occ.  *rank (optional) receives the
 * number of kept directions (columns of M that are numerically dependent are
 * dropped).  nocc = 0 removes the term.  Synchronous.  Errors: PWH_ERR_ARG
 * (sizes, weights, alpha, an exchange matrix without a positive direction),
 * PWH_ERR_OOM, PWH_ERR_CUDA.  The real-band routes (pwh_apply_h_gamma,
 * pwh_davidson_solve_gamma) accept the term only when zeta are real
 * functions (psi_occ real at k = 0), else PWH_ERR_ARG. */
pwh_status pwh_set_ace(pwh_system* sys, int32_t nocc, const void* psi_occ, int64_t ld_occ,
                       const double* occ, double alpha, int32_t* rank);

/* ------------------------------------------------------------- SCF steps --
 * The steps either side of H|psi> in a self-consistent Kohn-Sham calculation
 * (Sec. "Introduction"): the density of the occupied bands, then the new local
 * potential.  Hartree atomic units, FP64, grids in the layout of
 * pwh_set_potential (N1*N2*N3 doubles, C order, i3 fastest, point (i1,i2,i3) at
 * r = sum_d (i_d/N_d) a_d), all DEVICE pointers on the system's stream. */

/* rho(r) = sum_n occ[n] |psi_n(r)|^2 with psi_n(r) = Omega^{-1/2} sum_G
 * c_n(G) e^{i(k+G).r}, on the system's FFT grid.  psi: nb bands, public order,
 * ld_psi >= npw; occ: HOST double[nb]; rho: output grid.  The integral of rho
 * (grid sum times Omega/N) is sum_n occ[n] ||c_n||^2.  Synchronous. */
pwh_status pwh_density(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi,
                       const double* occ, double* rho);

/* v_out = v_ion + V_H + v_xc from the density rho (v_ion may be NULL):
 * V_H(G) = 4 pi rho(G)/|G|^2, the Fourier-space solution of the Poisson
 * equation on the FFT box (the Hartree kernel of the exact-exchange pair
 * densities, Sec. "Advanced implementation of exact (Fock) exchange"), with
 * G = 0 (neutralising background) and the Nyquist planes of even N_d set to
 * zero; v_xc: local-density exchange (Slater) and correlation
 * (Perdew-Zunger, Phys. Rev. B 23, 5048 (1981)); points with rho <= 1e-20
 * get none.  energies (HOST double[3], may be NULL): E_H = 1/2 int V_H rho,
 * E_xc = int rho eps_xc, int v_xc rho.  v_out may alias v_ion.  Synchronous. */
pwh_status pwh_hartree_xc(pwh_system* sys, const double* rho, const double* v_ion, double* v_out,
                          double* energies);

/* ----------------------------------------------------- learned preconditioner --
 * Not in the paper.  A 4 -> 64 -> 64 -> 1 SiLU network corrects the TPA
 * diagonal per (shell of equal |k+G|, band): K = K_TPA * exp(clip(s, -3, 3)),
 * s = MLP(f1..f4) with, for shell g and band n (Ritz value theta, residual
 * norm |r|, kinetic energy E = <x|T|x>, mean potential vbar, x = T_g / E):
 *   f1 = log(x + 0.05), f2 = (theta - vbar)/E, f3 = clip(log10|r|, -12, 2),
 *   f4 = (T_g + vbar - theta)/(T_g + E).
 * Parameter blob (FP32, pwh_mlp_num_params floats): W1 (64x4 row-major), b1,
 * W2 (64x64), b2, W3 (64), b3, then min f1..f4 and max f1..f4 of the training
 * data; outside that box the preconditioner uses plain TPA (s = 0).
 * All array arguments below are DEVICE pointers unless stated. */
pwh_status pwh_mlp_num_params(int32_t* n);

/* s[r] = MLP(feats[4r .. 4r+3]) for r < rows (FP32). */
pwh_status pwh_mlp_forward(pwh_system* sys, const float* params, const float* feats, int64_t rows,
                           float* s_out);

/* loss = sum_r w_r (s_r - y_r)^2 / wsum and grad_out = d loss / d params (the
 * first 4545 entries of the blob), by reverse-mode differentiation. */
pwh_status pwh_mlp_loss_grad(pwh_system* sys, const float* params, const float* feats,
                             const float* y, const float* w, int64_t rows, double wsum,
                             float* grad_out, float* loss_out);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step counts
 * from 1) on the 4545 network parameters; m, v: moment buffers. */
pwh_status pwh_mlp_adam(pwh_system* sys, float* params, const float* grad, float* m, float* v,
                        int32_t step, float lr);

/* Training rows from one point of a Davidson trajectory: X (nb Ritz vectors),
 * HX = H X (FP64), theta (HOST double[nb]) and the converged bands Xstar, all
 * complex128 npw x nb in public order.  Row n*nshell + g: feats (4 floats),
 * target y = log d - log K_TPA minus the band's weighted mean and weight w,
 * where d = -<r,e>_g/<r,r>_g maps the residual r = HX - X theta onto the
 * exact correction e = Xstar Xstar^H x - x on shell g (w = <r,r>_g/<r,r>;
 * rows with d <= 0 get w = 0).  Synchronous. */
pwh_status pwh_mlp_training_rows(pwh_system* sys, int32_t nb, const void* X, const void* HX,
                                 const double* theta, const void* Xstar, float* feats, float* y,
                                 float* w);

/* Install the parameter blob (HOST pointer, n = pwh_mlp_num_params) used by
 * PWH_PRECOND_MLP. */
pwh_status pwh_set_mlp(pwh_system* sys, const float* blob, int32_t n);

/* Shell decomposition (HOST outputs, any may be NULL except nshell): shell
 * index of every public plane wave and 1/2|k+G|^2 of every shell. */
pwh_status pwh_get_shells(const pwh_system* sys, int32_t* nshell, int32_t* shell_of_pw,
                          double* shell_kinetic);

/* -------------------------------------------------------------- measurement --
 * Per-family kernel timing: with timing on, the library brackets the launches
 * of each kernel family with CUDA events on the system's stream and
 * accumulates their durations (adds an event pair per launch).  Turning it on
 * or off synchronizes the stream and clears the totals. */
typedef struct {
  char name[32];     /* family: fft_z_inverse_fp64|fp32, fft_plane_fp64|fp32,
                        fft_z_forward_fp64|fp32, tc_gemm_becp, tc_gemm_backproj,
                        cgemm_fp64, cgemm_fp32, jacobi_fp64, cholqr_fp64,
                        jacobi_fp32, zgemm_fp64_tc (sliced FP64-equivalent
                        GEMM), zgemm_fp32_tc (three-slice FP32-equivalent
                        GEMM) */
  int64_t launches;  /* timed launches (bracketed groups) */
  double total_ms;   /* summed device time */
  double flops;      /* algorithmic floating-point operations of those launches
                        (nominal 5 N log2 N per length-N complex FFT, 8 MNK per
                        complex GEMM, 2 MNK per real tensor-core GEMM, 40 m^2
                        per Jacobi round); 0 where not counted (cholqr) */
  double bytes;      /* algorithmic device-memory bytes of those launches */
} pwh_kernel_time;

pwh_status pwh_set_kernel_timing(pwh_system* sys, int32_t on);

/* Synchronize and copy up to max_out family totals into out; *count receives
 * the number of families. */
pwh_status pwh_get_kernel_times(pwh_system* sys, pwh_kernel_time* out, int32_t max_out,
                                int32_t* count);

/* Number of kernels this library has launched in the process so far (host
 * counter, all systems). */
pwh_status pwh_launch_count(int64_t* count);

/* Batched eigensolves of n independent systems (cells x k-points: the pool and
 * image levels of Sec. "New parallelization levels"): a pool of nthreads host
 * threads runs pwh_davidson_solve on every system, each on its own stream, so
 * their kernels overlap on the GPU.  Arrays of length n: systems (distinct,
 * each created with its own stream for overlap), opts, psi_io (DEVICE),
 * ld_psi, eig (HOST double[nb_i]), stats (may be NULL), status_out (HOST).
 * Returns PWH_OK when every solve did, else the first failing status (its
 * message names the system). */
pwh_status pwh_batch_davidson_solve(int32_t n, pwh_system* const* systems,
                                    const pwh_davidson_opts* opts, void* const* psi_io,
                                    const int64_t* ld_psi, double* const* eig,
                                    pwh_davidson_stats* stats, pwh_status* status_out,
                                    int32_t nthreads);

/* Subspace diagonalisation (the dense eigensolve of the O_ij matrices, Sec.
 * "New parallelization levels"), as used by pwh_davidson_solve: the lowest nk
 * eigenpairs of the n x n Hermitian H (DEVICE complex128, column-major, ld >=
 * n, only read).  theta: DEVICE double[nk] ascending; C: DEVICE complex128
 * n x nk (ld = n), orthonormal eigenvectors.  Q (optional, DEVICE, ld = ldq >= n)
 * receives all n eigenvectors sorted by eigenvalue; with warm > 0, Q must hold
 * on entry the eigenvectors of the leading warm x warm block of H (a previous
 * call's output) and the iteration starts in that basis.  Parallel cyclic
 * Jacobi: sweeps in FP32 to FP32 convergence (in one 16-CTA cluster with the
 * matrix in distributed shared memory when it fits there, n up to about 440),
 * then, for precision = PWH_FP64, the accumulated basis made unitary in FP64
 * (Newton-Schulz), Q^H H Q in FP64 and FP64 sweeps until
 * max|A_ij| <= 1e-13 max|A_ii|; for PWH_MIXED the FP32 result (one FP32
 * Newton-Schulz step; eigenvalues to about 1e-7 ||H||), as the reduced-precision
 * phase of pwh_davidson_solve uses.  Asynchronous on the system's stream;
 * n <= 4096; another precision gives PWH_ERR_ARG. */
pwh_status pwh_subspace_eigh(pwh_system* sys, int32_t n, const void* H, int64_t ldh, int32_t nk,
                             double* theta, void* C, void* Q, int64_t ldq, int32_t warm,
                             int32_t precision);

/* Cholesky-QR factor of the eigensolver's orthonormalisation (the iterative
 * orthonormalisation of Sec. "New parallelization levels"): from the Gram
 * matrix S = T^H T (k x k, DEVICE complex128, column-major, ld = k) of k
 * columns, Tr (DEVICE k x k, ld = k) such that the first *kept columns of
 * T Tr are orthonormal (the others zero).  Column j is dropped when S_jj <= 0,
 * when t0 (optional DEVICE double[k], the column norms before a projection)
 * is given and sqrt(S_jj) < drop_rel t0[j], or when the pivot of the
 * unit-diagonal matrix falls to the rounding level of the arithmetic (1e-12
 * in FP64, 1e-6 for PWH_MIXED: FP32).  Up to 156 (FP64) / 221 (FP32) columns on
 * one block with the triangle in shared memory, above that a blocked
 * factorisation and inverse over the whole GPU.  k <= 1024.  kept: HOST int;
 * the call synchronises the stream to read it. */
pwh_status pwh_subspace_cholqr(pwh_system* sys, int32_t precision, int32_t k, const void* S,
                               const double* t0, double drop_rel, void* Tr, int32_t* kept);

/* Complex GEMM of the subspace algebra (the O_ij = <psi_i|O|psi_j> products and
 * basis rotations of Sec. "New parallelization levels"), as the eigensolver
 * uses it: C = alpha op(A) B + beta C, op(A) = A^H when conj_a else A; op(A)
 * is M x K, B is K x N, C is M x N; all DEVICE complex128, column-major with
 * the given leading dimensions (lda >= rows of A as stored).  alpha, beta:
 * HOST double[2] (re, im).  precision PWH_FP64: FP64 arithmetic (products of
 * at least 2e8 flops as exact integer-slice products on the tensor cores);
 * PWH_MIXED: operands rounded to FP32, FP32 accumulation (relative error about
 * sqrt(K) 1e-7), result widened (products of at least 4e8 flops and 48
 * columns of A^H B or 96 of A B, or 1 and 16 columns when K (A^H B) or M (A B)
 * is at least 65,536, as three BF16 slices of each FP32 operand, six slice
 * products on the tensor cores).
 * Asynchronous on the system's stream; uses the system's workspaces (one GEMM
 * at a time per system). */
pwh_status pwh_subspace_gemm(pwh_system* sys, int32_t precision, int32_t conj_a, int32_t M,
                             int32_t N, int32_t K, const double* alpha, const void* A, int64_t lda,
                             const void* B, int64_t ldb, const double* beta, void* C, int64_t ldc);

/* Synchronize the system's stream and report device-side failures: returns
 * PWH_ERR_TIMEOUT (and clears the flag) if a bounded wait inside a kernel gave
 * up since the last call, so that its results must be discarded. */
pwh_status pwh_sync(pwh_system* sys);

const char* pwh_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PWH_H */
