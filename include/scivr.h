/*
 * scivr.h -- C ABI of libscivr: GB300 (sm_103a) time-averaged semiclassical
 * initial-value-representation (TA-SC-IVR) power spectra.
 *
 * Method: Tamascelli, Dambrosio, Conte, Ceotto, arXiv:1312.4698.  The
 * library evaluates the Monte Carlo estimate of the separable-approximation
 * spectral density (Eq. sep_approx) in the discrete form of Eq. I(E)_discreto:
 *
 *   I(E_k) = dt^2 / (2 pi T n_good) * sum_{j good} w_j
 *            | sum_{c=0}^{n_steps} <chi|p_j(c dt), q_j(c dt)> e^{i (S_j(c dt) + E_k c dt + phi_j(c dt))} |^2
 *
 * with T = n_steps dt, Husimi-sampled initial conditions (Sec. III.A), a
 * fourth-order symplectic integrator, the Herman-Kluk prefactor phase phi_t
 * (Eq. prefactor) and the stability filter |det(M^T M) - 1| > tol (Sec. II).
 *
 * Conventions for every entry point:
 *   - atomic units, hbar = 1, mass-weighted normal coordinates (masses 1);
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device, allocated and owned by the caller; "host" pointers are ordinary
 *     memory, read during the call and not retained;
 *   - `stream` is a cudaStream_t (NULL = legacy default stream); all work is
 *     enqueued asynchronously on it; no call synchronises the device unless
 *     stated;
 *   - every call returns a scivr_status; on failure nothing (or nothing
 *     further) is enqueued and scivr_last_error() describes the cause.
 *     Argument checks happen before any launch and return SCIVR_EINVAL.
 *     Launch or runtime failures return SCIVR_ECUDA.
 */
#ifndef SCIVR_H
#define SCIVR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SCIVR_OK = 0,
    SCIVR_EINVAL = -1,        /* invalid argument (shape, range, null pointer) */
    SCIVR_ENOMEM = -2,        /* device allocation failed */
    SCIVR_ECUDA = -3,         /* CUDA launch or runtime error */
    SCIVR_ETIMEOUT = -4,      /* a bounded device-side wait expired */
    SCIVR_EUNSUPPORTED = -5   /* valid request this build does not implement */
} scivr_status;

/* Diagonal part of the potential. */
enum { SCIVR_DIAG_HARMONIC = 0,   /* omega_i^2 q_i^2 / 2 */
       SCIVR_DIAG_MORSE = 1 };    /* D_i (1 - exp(-a_i q_i))^2 */

/* Potential kinds. */
enum { SCIVR_PES_POLY = 0,        /* diagonal + cubic + quartic coupling monomials */
       SCIVR_PES_CART3 = 1 };     /* Cartesian triatomic surface in its normal modes (F = 3) */

/* Arithmetic of the propagation. */
enum { SCIVR_FP64 = 0,            /* everything in IEEE double */
       SCIVR_MIXED = 1 };         /* monodromy, potential, det M and the det A
                                     elimination in FP32; p, q, S and the
                                     continuous prefactor phase in FP64 */

/* Kernel schedule of scivr_propagate. */
enum { SCIVR_KERNEL_AUTO = 0,     /* library choice (tuned per F, precision, n_traj) */
       SCIVR_KERNEL_THREAD = 1,   /* one thread per trajectory */
       SCIVR_KERNEL_GROUP = 2 };  /* a lane group per trajectory, batched determinants */

/* Arithmetic of the time -> energy Fourier step. */
enum { SCIVR_FT_FP64 = 0,         /* FP64 fused-multiply-add contraction (CUDA cores) */
       SCIVR_FT_TC_BF16 = 1,      /* tensor cores: one BF16 digit per operand, FP32 accumulation */
       SCIVR_FT_TC_BF16X3 = 2,    /* tensor cores: two BF16 digits, three digit products */
       SCIVR_FT_TC_BF16X6 = 3,    /* tensor cores: three BF16 digits, six products (FP32-level) */
       SCIVR_FT_CZT64 = 4 };      /* FP64 chirp-z transform (Bluestein convolution by FFTs) */

/* What scivr_propagate records per step. */
enum { SCIVR_AMP_TA = 0,          /* time-averaged SC-IVR summand (Eq. I(E)_discreto) */
       SCIVR_AMP_HK = 1 };        /* Herman-Kluk SC-IVR summand with its sampling weight (Eq. I(E)_SCIVR) */

#define SCIVR_MAX_F 24            /* largest number of modes */
#define SCIVR_MAX_CHI 8           /* largest number of reference states per call */

typedef struct scivr_pes_s *scivr_pes;   /* opaque, library-owned */

/* Potential energy surface, V(q) = sum_i diag_i(q_i)
 *                                 + sum_m c3[m] q_i q_j q_k      (i <= j <= k = idx3[3m..3m+2])
 *                                 + sum_m c4[m] q_i q_j q_k q_l  (i <= j <= k <= l = idx4[4m..4m+3]).
 * The paper's molecules use analytic fitted surfaces (Sec. IV); the
 * Morse-diagonal form is its H2 potential and uncoupled-oscillator study.
 * All arrays are host memory, copied by scivr_create_pes. */
typedef struct {
    int32_t F;              /* number of modes, 1..SCIVR_MAX_F */
    int32_t kind;           /* SCIVR_PES_POLY */
    int32_t diag_kind;      /* SCIVR_DIAG_HARMONIC or SCIVR_DIAG_MORSE */
    const double *omega;    /* [F] harmonic frequencies (> 0) */
    const double *D;        /* [F] Morse depths (> 0; ignored for harmonic) */
    const double *a;        /* [F] Morse range parameters (> 0; ignored for harmonic) */
    int32_t n3;             /* number of cubic monomials (>= 0) */
    const int32_t *idx3;    /* [n3 * 3], each triple sorted, entries in [0, F) */
    const double *c3;       /* [n3] */
    int32_t n4;             /* number of quartic monomials (>= 0) */
    const int32_t *idx4;    /* [n4 * 4], each quadruple sorted, entries in [0, F) */
    const double *c4;       /* [n4] */
} scivr_pes_desc;

/* Propagation parameters (host memory, read during the call). */
typedef struct {
    double dt;              /* time step (> 0) */
    int32_t n_steps;        /* steps to T = n_steps dt (>= 1); K = n_steps + 1 samples */
    int32_t precision;      /* SCIVR_FP64 or SCIVR_MIXED */
    double stab_tol;        /* trajectory is bad once |det(M)^2 - 1| > stab_tol (paper: 1e-6) */
    const double *gamma;    /* [F] coherent-state widths (> 0) */
    const double *p_eq;     /* [n_chi * F] reference-state momenta */
    const double *q_eq;     /* [n_chi * F] reference-state positions */
    int32_t n_chi;          /* number of reference states, 1..SCIVR_MAX_CHI */
    int32_t kernel;         /* SCIVR_KERNEL_AUTO / _THREAD / _GROUP */
    int32_t amplitude;      /* SCIVR_AMP_TA (0) or SCIVR_AMP_HK */
    int32_t amp_prec;       /* amplitude storage: SCIVR_FP64 (0, complex double) or SCIVR_MIXED
                               (complex float, 8 bytes a sample; precision SCIVR_MIXED and
                               amplitude SCIVR_AMP_TA only) */
} scivr_prop_params;

/* Optional final-state outputs of scivr_propagate (device pointers, each may be NULL). */
typedef struct {
    double *p;              /* [F][n_traj] momenta at T */
    double *q;              /* [F][n_traj] positions at T */
    double *S;              /* [n_traj] classical action at T */
    double *theta;          /* [n_traj] continuous arg det A at T (phi_T = theta / 2) */
    double *detM;           /* [n_traj] det M at T */
    double *detA;           /* [n_traj][2] det A at T (re, im) */
    double *M;              /* [n_traj][2F][2F] monodromy at T, rows (p, q), columns (p0, q0) */
    double *stab;           /* [n_traj] max over steps of |det(M)^2 - 1| (+inf once not finite);
                               the stability measure the good flag thresholds */
} scivr_final_state;

/* Create a potential from a descriptor (Sec. IV potentials; see scivr_pes_desc).
 * Allocates device memory on the current device.  *out receives the handle.
 * Errors: SCIVR_EINVAL (F out of range, non-positive omega/D/a, unsorted or
 * out-of-range monomial indices, NULL arrays with nonzero counts),
 * SCIVR_ENOMEM, SCIVR_ECUDA. */
int scivr_create_pes(const scivr_pes_desc *d, scivr_pes *out);

/* ------------------------------------------------------------------------ */
/* Cartesian surfaces and normal modes                                        */
/* ------------------------------------------------------------------------ */

/* Cartesian surface of a bent triatomic, atoms 0 and 2 bonded to the central atom 1
 * (Sec. III.A: the molecular surfaces are functions of the Cartesian coordinates and
 * the host converts them to mass-weighted normal modes before propagation):
 *   V(x) = sum_b D[b] (1 - exp(-a[b] (r_b - re[b])))^2 + (k_bend / 2) (cos theta - cos theta_e)^2,
 * r_0 = |x0 - x1|, r_1 = |x2 - x1|, theta the angle 0-1-2.  x: [9] bohr, atom-major.
 * Units: hartree, bohr, electron masses. */
typedef struct {
    double mass[3];         /* atom masses (> 0) */
    double D[2];            /* Morse depths of bonds 0-1 and 2-1 (> 0) */
    double a[2];            /* Morse range parameters (> 0) */
    double re[2];           /* equilibrium bond lengths (> 0) */
    double k_bend;          /* bend force constant (> 0) */
    double theta_e;         /* equilibrium angle, radians, in (0, pi) */
} scivr_cart_triatomic;

/* Normal modes of a triatomic surface (Sec. III.A, the conversion matrix of the host
 * driver): the equilibrium geometry x_eq (atom 1 at the origin, the molecule in the
 * xy plane, the bisector along +y), the Hessian there, its mass-weighted form
 * M^{-1/2} H M^{-1/2} diagonalised by Jacobi rotations, and the three vibrations (the
 * largest eigenvalues; translations and rotations have eigenvalue zero) in increasing
 * frequency.  Outputs (host memory, caller-owned; any may be NULL):
 *   omega [3]: harmonic frequencies sqrt(eigenvalue), hartree;
 *   x_eq [9];
 *   Lm [9][3]: x = x_eq + Lm q, Lm[i][m] = L[i][m] / sqrt(mass of the atom of coordinate i)
 *              with L the orthonormal mass-weighted eigenvectors, each signed so that its
 *              first component of magnitude above 1e-3 is positive.
 * Host only (no device work).  Errors: SCIVR_EINVAL (NULL c, non-positive or non-finite
 * parameters, theta_e outside (0, pi)). */
int scivr_normal_modes(const scivr_cart_triatomic *c, double *omega, double *x_eq, double *Lm);

/* Conversions between n Cartesian geometries x [n][9] and normal coordinates q [n][3]
 * of the triatomic: x = x_eq + Lm q and q = Lm^T M (x - x_eq), M the diagonal of atom
 * masses (the projection onto the vibrations: Lm^T M Lm = I; translations and
 * rotations of x are dropped).  Host arrays, caller-owned.  Errors: as
 * scivr_normal_modes, SCIVR_EINVAL for n < 0 or NULL arrays with n > 0. */
int scivr_normal_to_cartesian(const scivr_cart_triatomic *c, int64_t n, const double *q, double *x);
int scivr_cartesian_to_normal(const scivr_cart_triatomic *c, int64_t n, const double *x, double *q);

/* Potential whose V(q), gradient and Hessian are those of the Cartesian surface at
 * x = x_eq + Lm q (the normal modes of scivr_normal_modes; F = 3): the propagation
 * kernels evaluate the surface through the bond and angle coordinates and the chain
 * rule at every force stage.  Propagation: SCIVR_FP64 with the thread-per-trajectory
 * schedule (SCIVR_KERNEL_AUTO chooses it); other precisions or schedules return
 * SCIVR_EUNSUPPORTED.  Allocates device memory on the current device.
 * Errors: as scivr_normal_modes, SCIVR_ENOMEM, SCIVR_ECUDA. */
int scivr_create_pes_cartesian(const scivr_cart_triatomic *c, scivr_pes *out);

/* Release a potential created by scivr_create_pes or scivr_create_pes_cartesian
 * (synchronises the device so that no launch still reads it).  NULL is accepted. */
int scivr_destroy_pes(scivr_pes pes);

/* Number of modes of a potential (0 for NULL). */
int32_t scivr_pes_modes(scivr_pes pes);

/* Husimi sampling of initial conditions (Sec. III.A, after Eq. I(E)_discreto):
 * q0_i = q_eq_i + z_i / sqrt(gamma_i), p0_i = p_eq_i + z_{F+i} sqrt(gamma_i),
 * with z standard normal, i.e. the density |<p0 q0|chi>|^2 / (2 pi)^F around
 * chi = |p_eq, q_eq>, and weights w = 1 / |<p0 q0|chi>|^2 (this carries the
 * paper's (2 pi)^-F).  Normal z_d of trajectory j comes from Philox4x32-10
 * (counter (j mod 2^32, j / 2^32, d / 4, 0), key (seed mod 2^32, seed / 2^32))
 * and Box-Muller on words (0,1) and (2,3) with uniforms (u + 1/2) 2^-32.
 * gamma, p_eq, q_eq: host [F].  p0, q0: device [F][n_traj]; w: device [n_traj].
 * Errors: SCIVR_EINVAL (NULL pointers, n_traj < 1, gamma <= 0). */
int scivr_sample_initial(scivr_pes pes, const double *gamma, const double *p_eq,
                         const double *q_eq, int64_t n_traj, uint64_t seed,
                         double *p0, double *q0, double *w, void *stream);

/* Propagate n_traj trajectories from (p0, q0) to T = n_steps dt and record, for
 * every reference state x and step c = 0..n_steps, the amplitude
 *   amp[x][j][c] = <chi_x|p_j(c dt), q_j(c dt)> exp(i (S_j(c dt) + phi_j(c dt)))
 * (the summand of Eq. I(E)_discreto without the energy factor).  With
 * prm->amplitude = SCIVR_AMP_HK it records instead the Herman-Kluk summand of
 * Eq. I(E)_SCIVR times the importance weight of the Husimi density of the first
 * reference state, w_j = 1/|<p_j(0) q_j(0)|chi_0>|^2 (the density scivr_sample_initial
 * draws from when given chi_0; every reference state shares the trajectories),
 *   amp[x][j][c] = C_j(c dt) e^{i S_j(c dt)} <chi_x|p_j(c dt), q_j(c dt)> <p_j(0), q_j(0)|chi_x> w_j,
 * C = |det A|^{1/2} e^{i theta/2} (Eq. prefactor on the branch theta follows),
 * whose mean over trajectories drawn from that density is <chi_x|e^{-iHt}|chi_x>
 * (scivr_spectrum_hk).  For x = 0 the summand is C e^{iS} <chi_0|p q> / <chi_0|p0 q0>,
 * exactly 1 at c = 0.  Integrator:
 * Yoshida's fourth-order triple jump of exact drift/kick sub-flows for (p, q),
 * the action S and the monodromy M (Sec. III.A).  phi = theta/2 with theta the
 * continuous arg det A of the Herman-Kluk matrix (Eq. prefactor), unwrapped
 * per step relative to the reference rotation exp(-i sum_i gamma_i t).  A
 * trajectory is marked bad (good[j] = 0) once |det(M)^2 - 1| > stab_tol or any
 * state value is not finite (Sec. II, Sec. III.B); bad trajectories are still
 * propagated to T and their amplitudes are unspecified.
 * A reference state that combines the recorded coherent states, chi = sum_x c_x chi_x
 * (the symmetry-adapted states of Sec. IV), has the time-averaged amplitude
 * sum_x conj(c_x) amp[x][j][c]: the overlap is linear in <chi| and e^{i (S + phi)} is
 * common to all x, so its spectrum is scivr_spectrum of those combined rows with the same
 * weights.  The Herman-Kluk summand is bilinear in chi and has no such form.
 * p0, q0: device [F][n_traj].  amp: device complex double (re, im interleaved)
 * [n_chi][n_traj][amp_ld], amp_ld >= n_steps + 1, 16-byte aligned; with
 * prm->amp_prec = SCIVR_MIXED complex float (re, im) of the same shape, 8-byte
 * aligned (the mixed path forms each amplitude sample in FP32, so nothing is lost
 * but the sample at c = 0, rounded from FP64).  good:
 * device [n_traj].  fin: host struct of optional device outputs (NULL = none).
 * Precision SCIVR_MIXED keeps the monodromy, the potential and det M in FP32;
 * positions, momenta, the action, the elimination that gives det A and the
 * product of its pivots in double-FP32 pairs (FP64-class, about 2^-46 relative
 * per operation, on the FP32 pipe); the argument of det A and the phase in FP64.
 * Its det M deviation is FP32 rounding: give it a stab_tol scaled accordingly.  The mixed
 * path tests det M every 16 steps and at the last step (FP64: every step).
 * Built: SCIVR_FP64 for F <= 9 (both schedules), SCIVR_MIXED for F <= 24
 * (lane-group schedule; one trajectory per warp above F = 9, two column
 * groups per trajectory and tensors read from L2 above F = 16).  A surface of
 * kind SCIVR_PES_CART3 (scivr_create_pes_cartesian) runs on SCIVR_FP64 with the
 * thread schedule only.
 * Errors: SCIVR_EINVAL (NULL pointers, n_traj < 1, n_steps < 1, dt <= 0,
 * gamma <= 0, amp_ld too small, F mismatch, n_chi out of range, amp_prec
 * not SCIVR_FP64 or SCIVR_MIXED, or SCIVR_MIXED with FP64 precision or HK amplitudes),
 * SCIVR_EUNSUPPORTED (precision or kernel not built for this F). */
int scivr_propagate(scivr_pes pes, const scivr_prop_params *prm, int64_t n_traj,
                    const double *p0, const double *q0, void *amp, int64_t amp_ld,
                    uint8_t *good, const scivr_final_state *fin, void *stream);

/* Time-averaged spectrum of one reference state, Eq. I(E)_discreto:
 *   I(E_k) = dt^2 / (2 pi T n_good) sum_{j: good[j] != 0} w_j | sum_{c=0}^{n_steps} amp[j][c] e^{i E_k c dt} |^2
 * with E_k = E_min + k (E_max - E_min) / (n_E - 1), k = 0..n_E-1 (endpoints
 * included, Sec. III.A) and T = n_steps dt.  Bad trajectories contribute
 * nothing, whatever their amplitudes hold.  If n_good = 0, I is all zeros.
 * amp: device complex double [n_traj][amp_ld] (amp_prec = SCIVR_FP64, 16-byte
 * aligned) or complex float (amp_prec = SCIVR_MIXED, 8-byte aligned; every
 * Fourier mode reads it, widening to FP64 where the mode computes in FP64).  w:
 * device [n_traj].  good: device [n_traj].  I_out: device [n_E].  n_good_out:
 * device int64 (may be NULL).  ft_mode SCIVR_FT_FP64 contracts in FP64 on
 * the CUDA cores; the SCIVR_FT_TC_* modes split both operands into BF16
 * digits and contract on the tensor cores (tcgen05) with FP32 accumulation,
 * then sum tiles in FP64: their error is that of the digit count (about
 * 2^-8, 2^-16, 2^-24 relative to the largest terms).  SCIVR_FT_CZT64 evaluates the
 * same sums in FP64 through Bluestein's identity E_k c dt = E_min c dt + w (k^2 + c^2
 * - (k - c)^2)/2 (w = dE dt): a convolution by length-8192 FP64 FFTs per trajectory,
 * about 10 L log2 L flops instead of 8 K n_E, with FP64 rounding; it takes
 * n_steps + 1 <= 7169 and n_E <= 12288 (SCIVR_EUNSUPPORTED otherwise; energies beyond
 * 8193 - (n_steps + 1) are transformed in blocks) and allocates about 200 KB plus
 * 8 n_E bytes per SM.  Allocates
 * stream-ordered scratch (cudaMallocAsync): FP64 mode about
 * 16 (n_steps+1) n_E + 8 n_E ceil(n_traj/64) bytes; tensor-core modes about
 * 4 d (n_steps+1) (n_traj + 2 n_E) + 8 n_E ceil(n_traj/128) bytes, d digits.
 * Errors: SCIVR_EINVAL (NULL pointers, n_traj < 1, n_steps < 1, n_E < 2,
 * E_max <= E_min, dt <= 0, amp_ld < n_steps + 1), SCIVR_EUNSUPPORTED
 * (amp_prec or ft_mode not built), SCIVR_ENOMEM.  A tensor-core wait that
 * expires is reported by scivr_check_status. */
int scivr_spectrum(const void *amp, int64_t amp_ld, int32_t amp_prec, const double *w,
                   const uint8_t *good, int64_t n_traj, int32_t n_steps, double dt,
                   double E_min, double E_max, int32_t n_E, int32_t ft_mode,
                   double *I_out, int64_t *n_good_out, void *stream);

/* Plain Herman-Kluk SC-IVR spectrum of one reference state, Eq. I(E)_SCIVR,
 * from amplitudes recorded with SCIVR_AMP_HK:
 *   C(c dt) = (1/n_good) sum_{j: good[j] != 0} amp[j][c]   (the survival amplitude),
 *   I(E_k) = (dt/pi) Re[ C(0)/2 + sum_{c=1}^{n_steps} C(c dt) e^{i E_k c dt} ]
 * (Eq. I(E)_timedependent by the rectangle rule on the symmetric grid
 * c = -n_steps..n_steps, folded onto c >= 0 with C(-t) = conj C(t)), E_k as
 * for scivr_spectrum.  amp: device complex double [n_traj][amp_ld].  good:
 * device [n_traj].  I_out: device [n_E].  C_out: device complex double
 * [n_steps+1] (may be NULL).  n_good_out: device int64 (may be NULL).  The
 * column sums over trajectories run in a fixed order (bitwise reproducible).
 * Allocates stream-ordered scratch of about 16 (n_steps+1) ceil(n_traj/4096)
 * bytes.  Errors: as scivr_spectrum. */
int scivr_spectrum_hk(const void *amp, int64_t amp_ld, const uint8_t *good, int64_t n_traj, int32_t n_steps,
                      double dt, double E_min, double E_max, int32_t n_E, double *I_out, void *C_out,
                      int64_t *n_good_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched runs: many molecules (different F, n_traj, n_steps) in one call    */
/* ------------------------------------------------------------------------ */

/* One molecule of a batch.  Device pointers as for scivr_propagate and
 * scivr_spectrum; the host arrays inside prm are copied by scivr_batch_create. */
typedef struct {
    scivr_pes pes;
    scivr_prop_params prm;
    int64_t n_traj;
    const double *p0, *q0;        /* device [F][n_traj] */
    const double *w;              /* device [n_traj] */
    void *amp;                    /* device complex double [n_chi][n_traj][amp_ld] (complex float if prm.amp_prec = SCIVR_MIXED) */
    int64_t amp_ld;
    uint8_t *good;                /* device [n_traj] */
    double E_min, E_max;
    int32_t n_E;
    double *I_out;                /* device [n_chi][n_E] */
    int64_t *n_good_out;          /* device [1], may be NULL */
} scivr_batch_item;

typedef struct scivr_batch_s *scivr_batch;   /* opaque plan, library-owned */

/* Build a plan for a batch (Sec. III.B: trajectories of all molecules are
 * independent).  Molecules are grouped by (F, precision); each group runs as
 * one persistent lane-group launch whose CTAs pull (molecule, trajectory
 * tile) work items, largest cost first, so molecules of different sizes
 * share the GPU.  The CTA shape of each group is chosen by the library's
 * autotuner (timed once per (F, precision, device) and cached, in-process
 * and in the file named by SCIVR_TUNE_CACHE if set).  All device memory
 * the launches need (work lists, per-molecule launch records, Fourier
 * scratch for the largest molecule) is allocated here; the caller's
 * buffers are not touched until scivr_batch_launch.  ft_mode as for
 * scivr_spectrum.  Synchronises the device.  Errors: SCIVR_EINVAL (any item
 * invalid; the message names it), SCIVR_EUNSUPPORTED (precision not built
 * for the item's F: mixed above F = 24, FP64 above F = 9), SCIVR_ENOMEM, SCIVR_ECUDA. */
int scivr_batch_create(const scivr_batch_item *items, int32_t n_items, int32_t ft_mode,
                       scivr_batch *out);

/* Enqueue the whole batch on `stream`: per group a counter reset and one
 * persistent propagation launch, then every molecule's spectra.  Performs
 * no allocation and no synchronisation, so a stream capture of this call
 * yields a CUDA graph that can be replayed while the plan lives. */
int scivr_batch_launch(scivr_batch b, void *stream);

/* Number of propagation groups of a plan and, for group g, its F, precision
 * and the CTA warps the autotuner chose (any pointer may be NULL). */
int scivr_batch_info(scivr_batch b, int32_t g, int32_t *n_groups, int32_t *F, int32_t *precision,
                     int32_t *warps);

/* The plan's propagation schedule: *one_launch = 1 when every mixed-precision
 * molecule runs in one persistent launch (the multi-F kernel: CTAs of four warps pull
 * (molecule, trajectory tile) items of all classes from one list, costliest first, and
 * run the body specialised for each item's F; built when every class is one of 3, 6, 9,
 * 12, 15, 24 and there are at least two), 0 when each F-class has its own persistent
 * launch.  scivr_batch_create picks by timing both on a probe of the plan (32 steps,
 * up to 2048 trajectories per molecule); the environment variable SCIVR_BATCH_SCHEDULE
 * = "one" or "per-class" forces the choice.  Above F = 9 the one launch reads the
 * coupling tensors from L2, so those molecules' results may differ in rounding from
 * their per-class runs.  Errors: SCIVR_EINVAL (NULL arguments). */
int scivr_batch_schedule(scivr_batch b, int32_t *one_launch);

/* Free a plan (synchronises the device).  NULL is accepted. */
int scivr_batch_destroy(scivr_batch b);

/* Same result as scivr_spectrum (same arguments, same checks) without allocating
 * any device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc or cudaMallocAsync -- processes whose
 * device memory is owned by another component's fixed pool or caching
 * allocator, and latency-critical callers for which an allocation could block
 * or fail under memory pressure.
 *
 * Its scratch (the good count and per-slice column sums) lives in one
 * library-owned device array of 4 MiB (2^19 doubles) that every GPU which loads
 * libscivr holds until the process exits.  Limit: n_E <= 524256; larger grids
 * return SCIVR_EINVAL and launch nothing.  Each call looks up the array's
 * device address (cudaGetSymbolAddress) with the calling device current, so a
 * device reset between calls is harmless; a call made while `stream` is being
 * captured reuses the address of the last call on that device instead, so make
 * the first call on each device before any stream capture begins.  All calls
 * share the one array and overwrite what the previous call left there (nothing
 * in it needs to start at zero), so calls that overlap on the GPU -- on
 * different streams, or on different host threads -- race and must be
 * serialised by the caller.  The caller still provides amp, w, good, I_out and
 * n_good_out exactly as for scivr_spectrum. */
int scivr_spectrum_noalloc(const void *amp, int64_t amp_ld, int32_t amp_prec, const double *w,
                           const uint8_t *good, int64_t n_traj, int32_t n_steps, double dt,
                           double E_min, double E_max, int32_t n_E, int32_t ft_mode,
                           double *I_out, int64_t *n_good_out, void *stream);

/* Synchronise `stream`, then read and clear this device's status word:
 * SCIVR_ETIMEOUT if a bounded device-side wait (mbarrier) expired in a kernel
 * since the last check, SCIVR_OK otherwise (SCIVR_ECUDA on a CUDA error). */
int scivr_check_status(void *stream);

/* Launch a one-CTA kernel that waits, with a limit of `seconds`, on an
 * mbarrier that nothing completes, exercising the bounded-wait path that the
 * tensor-core kernels use.  A following scivr_check_status must return
 * SCIVR_ETIMEOUT.  seconds must lie in (0, 10]. */
int scivr_selftest_wait_timeout(double seconds, void *stream);

/* Arithmetic-rate probe (measurement, no counterpart in the paper): launches
 * independent fused multiply-add chains on every SM, in FP32 (precision SCIVR_MIXED)
 * or FP64 (SCIVR_FP64), each thread iters x 16 FMAs; *flops_per_launch (host)
 * receives 2 x the FMAs of the launch.  The caller times the launch on `stream`;
 * flops / time is the pipe's attainable rate, the denominator of the propagation
 * kernels' roofline.  Errors: SCIVR_EINVAL (precision, iters < 1, NULL output),
 * SCIVR_ECUDA. */
int scivr_fma_probe(int32_t precision, int64_t iters, double *flops_per_launch, void *stream);

/* Message describing the last failure on the calling thread ("" if none). */
const char *scivr_last_error(void);

/* Number of kernel launches this library has enqueued on the calling thread
 * since the counter was last reset (for launch accounting in benchmarks). */
int64_t scivr_launch_count(int reset);

#ifdef __cplusplus
}
#endif

#endif /* SCIVR_H */
