/*
 * tddft.h -- C ABI of the GB300 (sm_103a) spinor real-time TDDFT propagation library.
 *
 * One handle holds one periodic system: a cubic FFT grid in an orthorhombic cell,
 * atoms with an erf-screened local potential and separable Kleinman-Bylander
 * projectors with spin-orbit coupling, a set of k-points and the occupied
 * two-component spinors psi_{k,i}.  Each call of tddft_step advances the spinors
 * by the time-dependent non-collinear Kohn-Sham equation (arXiv 2506.21908,
 * Eq. TDSDFT) with the Hamiltonian of Eq. HNC-SDFT:
 *
 *     H = [-1/2 nabla^2 + v_loc + v_H + vbar_xc] I_2 + (b_xc + mu_B B(t)) . sigma + V_NL,
 *
 * vbar_xc and b_xc from the adiabatic locally collinear LSDA (Eqs. LC+ALDA2, LC+ALDA),
 * the spin Zeeman term of Eq. zeeman_potential (mu_B = 1/2), and
 * V_NL = sum_a |beta~> (D_l + lambda_l L.S) <beta~| (Eq. Vps, Eq. Vps-soc and the L.S
 * form of Sec. 4.4).  Laser fields enter in velocity gauge: kinetic 1/2|G+k+A(t)|^2 and
 * projector phases exp(-i (k+A).d).  The paper does not state its propagator; this
 * library uses enforced time-reversal symmetry (ETRS) with a predictor and n_sc
 * corrector passes, the exponential as a Chebyshev series (or a Taylor series).
 * Each step ends with the density n(r) and magnetisation m(r) (Eqs. rho1-rho3) and
 * the potential recomputed from them.
 *
 * Conventions for every entry point
 *   - Every function returns a tddft_status (0 = success) and never aborts.  On failure
 *     tddft_last_error(h) returns a message; the state is unchanged except after
 *     TDDFT_ERR_DIVERGED.
 *   - The caller owns every array it passes; the library copies inputs during the call
 *     and owns all device memory it allocates (released by tddft_destroy).
 *   - Grid arrays are indexed [z][y][x] with x fastest; r = (x hx, y hy, z hz).
 *   - Spinor arrays are interleaved complex128 (re, im) laid out
 *     [nk][nstates][2][nz][ny][nx], normalised with <a|b> = sum_r conj(a) b dV.
 *   - Pointers flagged on_device = 1 are device pointers on the handle's device,
 *     accessed on the handle's stream (tddft_set_stream); otherwise host pointers.
 *   - Atomic units throughout (bohr, hartree, a.u. of time and field).
 *   - tddft_step is asynchronous on the handle's stream; calls that return host data
 *     synchronise that stream.
 */
#ifndef TDDFT_H
#define TDDFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tddft_ctx* tddft_handle;

typedef enum {
  TDDFT_OK = 0,
  TDDFT_ERR_ARG = -1,         /* invalid argument (null pointer, size, unsupported grid) */
  TDDFT_ERR_CUDA = -2,        /* a CUDA runtime call or kernel launch failed */
  TDDFT_ERR_OOM = -3,         /* device allocation failed */
  TDDFT_ERR_STATE = -4,       /* call out of order (e.g. step before set_states) */
  TDDFT_ERR_DIVERGED = -5,    /* non-finite density or norm detected */
  TDDFT_ERR_BOUND = -6,       /* the potential left the Chebyshev spectral window */
  TDDFT_ERR_UNSUPPORTED = -7  /* valid request outside what this build implements */
} tddft_status;

enum { TDDFT_FP64 = 0, TDDFT_FP32_MIXED = 1 };
enum { TDDFT_EXP_CHEBYSHEV = 0, TDDFT_EXP_TAYLOR = 1, TDDFT_EXP_CRANK_NICOLSON = 2 };
enum { TDDFT_SPIN_NONCOLLINEAR = 0, TDDFT_SPIN_COLLINEAR = 1, TDDFT_SPIN_UNPOLARISED = 2 };
/* Projector contraction (Eq. Vps with the L.S blocks): FP64 / FP32 on the CUDA cores, or on the
 * tensor cores (tcgen05, FP32-mixed precision, grid size divisible by 16) as one TF32 product or as
 * a split product hi*hi + hi*lo + lo*hi of TF32, BF16 or FP16 parts (each value = hi + lo; TF32 x3
 * and FP16 x3 close to FP32 accuracy, BF16 x3 about 16 bits); FP32 accumulation in every case.  The
 * tensor-core forms contract brick by brick (bricks of 32 or 16 x 8 x 8 grid points against every
 * projector sphere reaching into them) for both the projection <beta~|psi> and V_NL psi; the
 * projection restarts its tensor-core accumulation every few chunks of a brick and adds the groups
 * on the CUDA cores, so that the accumulation's rounding does not bias it. */
enum { TDDFT_PROJ_FP64 = 0, TDDFT_PROJ_FP32 = 1, TDDFT_PROJ_TF32 = 2, TDDFT_PROJ_TF32X3 = 3,
       TDDFT_PROJ_BF16X3 = 4, TDDFT_PROJ_F16X3 = 5 };

/* Energies returned by tddft_observables, indices into E[TDDFT_NE]. */
enum {
  TDDFT_E_KIN = 0,    /* sum w f <psi| 1/2|G+k+A|^2 |psi>                                   */
  TDDFT_E_NL = 1,     /* sum w f <psi|V_NL|psi>                                            */
  TDDFT_E_LOC = 2,    /* int v_loc n                                                       */
  TDDFT_E_H = 3,      /* 1/2 int v_H n                                                     */
  TDDFT_E_XC = 4,     /* int n eps_xc (the functional value)                               */
  TDDFT_E_Z = 5,      /* int mu_B B . m  (Sec. 3.4)                                        */
  TDDFT_E_TOTAL = 6,  /* sum of the six terms above (ion-ion constant excluded)            */
  TDDFT_E_TIME = 7,   /* current time t                                                    */
  TDDFT_E_XC_POT = 8, /* int <rho_v, V_v^xc>, the potential-weighted form of Eq. xc_energy4 */
  TDDFT_E_NELEC = 9,  /* int n                                                             */
  TDDFT_NE = 10
};

/* Orthorhombic cell: rows are lattice vectors (bohr).  Off-diagonal entries must be 0. */
typedef struct { double a[3][3]; } tddft_cell;

/* FFT grid: n[0] = n[1] = n[2] = n with n in {8, 12, 16, 24, 32, 48, 64, 96}. */
typedef struct { int n[3]; } tddft_grid;

/* Atoms: pos[natoms][3] (bohr, cartesian), species[natoms] in [0, nspecies). natoms may be 0. */
typedef struct {
  int natoms;
  const double* pos;
  const int* species;
} tddft_atoms;

/* Species data (Eq. KSpot, Eq. Vps, Eq. Vps-soc).  Per species s:
 *   local potential -Z[s] erf(r / rc_loc[s]) / r, periodic, G = 0 keeps pi Z rc^2 / Omega;
 *   projectors beta_{l,m}(d) = N_l |d|^l exp(-|d|^2 / (2 width[s]^2)) Y^real_lm(d/|d|),
 *   |d| < r_cut (minimum image), continuum-normalised, l = 0..lmax (lmax <= 2);
 *   coupling on (l, m, sigma): D[s][l] I + lambda_so[s][l] L.S  (Ha).
 * D and lambda_so are [nspecies][lmax+1].  r_cut must be at most half the shortest cell side
 * (points are kept for |d| < r_cut, so each has a single minimum image). */
typedef struct {
  int nspecies;
  const double* Z;
  const double* rc_loc;
  const double* width;
  int lmax;
  const double* D;
  const double* lambda_so;
  double r_cut;
} tddft_projectors;

/* Run parameters.
 *   precision : TDDFT_FP64, or TDDFT_FP32_MIXED (spinors, FFTs, potential apply and projectors
 *               in FP32, the series constants as float pairs and the series accumulators updated
 *               in float-float arithmetic; density, XC, Hartree, energies and norms in FP64)
 *   proj_mode : TDDFT_PROJ_FP64 / TDDFT_PROJ_FP32 (CUDA cores; they follow the precision) or one of
 *               the tensor-core modes TDDFT_PROJ_TF32 / _TF32X3 / _BF16X3 / _F16X3 (FP32-mixed
 *               precision and a grid size divisible by 16, else TDDFT_ERR_UNSUPPORTED; the discrete
 *               adjoint uses the CUDA-core contraction in every mode)
 *   nk, kpts[nk][3] (1/bohr, cartesian), kw[nk] (weights)
 *   nstates   : propagated spinors per k-point; occ[nk][nstates] occupations f
 *   dt        : time step (may be negative to run backwards)
 *   exp_kind  : TDDFT_EXP_CHEBYSHEV, TDDFT_EXP_TAYLOR, or TDDFT_EXP_CRANK_NICOLSON: the
 *               Cayley transform (1 + i tau H/2)^{-1} (1 - i tau H/2) in place of exp(-i tau H),
 *               applied through its own Chebyshev expansion on the spectral window (coefficients
 *               by Gauss-Chebyshev quadrature of the rational function, truncated like the
 *               exponential's; equivalent to solving the linear system to that tolerance)
 *   exp_order : 0 = automatic (Chebyshev and Crank-Nicolson: smallest K with |a_k| < cheb_tol
 *               for all k > K, separately for dt and dt/2); > 0 = this order for every
 *               exponential (Taylor default 4)
 *   cheb_tol  : truncation tolerance for automatic orders (0 = 1e-16 FP64, 1e-9 FP32-mixed)
 *   n_sc      : corrector passes per step; sc_tol > 0 stops them early when
 *               max |delta rho_v| < sc_tol (that check synchronises the stream)
 *   e_min, e_max : Chebyshev spectral window; both 0 = automatic at tddft_set_states
 *   xc        : 1 = locally collinear LSDA (Slater + PW92), 0 = no exchange-correlation
 *   spin_mode : TDDFT_SPIN_NONCOLLINEAR (default, Eq. HNC-SDFT); TDDFT_SPIN_COLLINEAR, the
 *               sigma_z-only potential of Eq. HSDFT (LSDA on the channel densities rho_uu, rho_dd,
 *               field along z, only B_z couples); TDDFT_SPIN_UNPOLARISED (LDA at n/2 per channel,
 *               no spin field, B ignored).  The last two need lambda_so = 0 (L.S couples the
 *               channels; TDDFT_ERR_ARG otherwise) and have no tddft_backward
 *               (TDDFT_ERR_UNSUPPORTED). */
typedef struct {
  int precision;
  int proj_mode;
  int nk;
  const double* kpts;
  const double* kw;
  int nstates;
  const double* occ;
  double dt;
  int exp_kind;
  int exp_order;
  double cheb_tol;
  int n_sc;
  double sc_tol;
  double e_min;
  double e_max;
  int xc;
  int spin_mode;
} tddft_params;

/* Create a handle on the current CUDA device: validates the inputs, builds the G mesh,
 * the local potential, projector tables and L.S blocks, and allocates device memory.
 * *out receives the handle (NULL on failure). */
tddft_status tddft_create(const tddft_cell* cell, const tddft_grid* grid, const tddft_atoms* atoms,
                          const tddft_projectors* proj, const tddft_params* params,
                          tddft_handle* out);

/* Tabulated external fields (velocity-gauge vector potential A and magnetic field B) at nt
 * increasing times t[nt]; A[nt][3], B[nt][3].  Values between nodes are linearly
 * interpolated; outside the table the end values are used.  Without a table A = B = 0. */
tddft_status tddft_set_fields(tddft_handle h, int nt, const double* t, const double* A,
                              const double* B);

/* Load spinors (complex128, layout above) at time t0; computes rho_v, the potential and,
 * when e_min = e_max = 0, the Chebyshev spectral window. */
tddft_status tddft_set_states(tddft_handle h, const void* psi, int on_device, double t0);

/* Copy the current spinors out as complex128 (layout above). */
tddft_status tddft_get_states(tddft_handle h, void* psi, int on_device);

/* The same two calls with complex64 spinors (interleaved float pairs, same layout).  An
 * FP32-mixed handle stores its spinors in this form, so loading moves half the bytes of the
 * complex128 call and converts nothing; an FP64 handle widens them exactly.  Host buffers may be
 * pageable or page-locked. */
tddft_status tddft_set_states_c64(tddft_handle h, const void* psi, int on_device, double t0);
tddft_status tddft_get_states_c64(tddft_handle h, void* psi, int on_device);

/* Advance nsteps ETRS steps (asynchronous on the handle's stream). */
tddft_status tddft_step(tddft_handle h, int nsteps);

/* Observables of the current state (synchronises).  Any output may be NULL.
 *   n[N_g], m[3][N_g] : density and magnetisation (1/bohr^3)
 *   E[TDDFT_NE]       : energy terms (indices above)
 *   M[3]              : int m dV
 *   norms[nk*nstates] : <psi_i|psi_i>
 * Returns TDDFT_ERR_BOUND if any potential since set_states left the spectral window and
 * TDDFT_ERR_DIVERGED on non-finite values (outputs are still written). */
tddft_status tddft_observables(tddft_handle h, double* n, double* m, double* E, double* M,
                               double* norms);

/* Current spin-matrix potential as the 4-vector V_v = [v+b_z, v-b_z, 2 b_x, -2 b_y]
 * (Eq. potential4), host array [4][N_g]. */
tddft_status tddft_get_potential(tddft_handle h, double* V);

/* out = H psi for nk*nstates spinors (complex128 layout above) with the current potential
 * and A(t) at the current time; in and out may not alias.  A diagnostic of the operator
 * that tddft_step exponentiates. */
tddft_status tddft_apply_hamiltonian(tddft_handle h, const void* in, void* out, int on_device);

/* Discrete adjoint of the propagation (reverse mode).  Starting from the current state, runs
 * nsteps forward steps (leaving the handle at the end state, as tddft_step would), evaluates
 * L = sum_r dL_drho[c][r] rho_v[c](r) on the final spin density 4-vector rho_v =
 * {rho_uu, rho_dd, Re rho_ud, Im rho_ud} (host array [4][N_g]; L = M_z = int m_z dV is
 * dL_drho = dV {1, -1, 0, 0}), and returns loss = L and the exact derivatives of L with respect
 * to every entry of the field table set by tddft_set_fields: dL_dA[nt][3], dL_dB[nt][3] (host;
 * either may be NULL).  The derivative follows every operation of the forward step: both
 * Chebyshev series (Clenshaw-type reverse recurrence reusing the Hamiltonian kernels), the
 * potential's dependence on the density through Hartree and the locally collinear LSDA
 * (analytic Jacobian), the velocity-gauge kinetic term and projector phases, and the Zeeman term.
 * Memory: spinor copies at every ckpt_every-th step (checkpoints), ckpt_every copies for the
 * recomputed segment, and one copy per Chebyshev term of a step, allocated for the call only.
 * Requires Chebyshev or Crank-Nicolson exponentials, sc_tol = 0, and two z-slabs of the grid in shared memory
 * (n <= 64 in FP64, n <= 96 in FP32-mixed); otherwise TDDFT_ERR_UNSUPPORTED.  The paper has no
 * adjoint; the loss and parameterisation follow the differentiation workload of this library. */
tddft_status tddft_backward(tddft_handle h, int nsteps, int ckpt_every, const double* dL_drho, double* loss,
                            double* dL_dA, double* dL_dB);

/* Per-atom magnetic moments and electron counts of the current state: m and n integrated over
 * each atom's Voronoi cell (every grid point belongs to its nearest atom, minimum image, ties to
 * the lowest index -- the NearestAtom rule of Algorithm 1).  M[natoms][3], N[natoms] host arrays
 * (either may be NULL); the cells partition the cell, so the sums equal the totals of
 * tddft_observables.  No-op without atoms. */
tddft_status tddft_atom_moments(tddft_handle h, double* M, double* N);

/* Global spin torques at the current state and time t, the terms of dM/dt = i <[H, sigma]>
 * summed over the occupied spinors with weights w_k f_i (M = int m dV, m = psi^dagger sigma psi):
 *   soc[3]    spin-orbit torque of the L.S projector blocks (Eq. SOtorque):
 *             sum_k w_k sum_i f_i sum_a c^dagger 2 i [D_a, S] c, with c = <beta~_a|psi_ki> at
 *             k + A(t) and S = sigma / 2 on the spin index of c;
 *   xc[3]     2 int b_xc x m dV (part of Eq. GMT; zero at every point in the locally collinear
 *             approximation, where b_xc is parallel to m);
 *   zeeman[3] 2 mu_B B(t) x M (Eq. magrot).
 * The kinetic term and D_l I commute with the spin and give nothing, so the three add up to
 * dM/dt.  Host arrays of 3 doubles, any may be NULL.  Computed in FP64 from the projections
 * (FP32 in FP32-mixed mode) and the FP64 density and XC field; synchronises the stream. */
tddft_status tddft_torques(tddft_handle h, double* soc, double* xc, double* zeeman);

/* Testing hook of the failure-detection path (the paper has no counterpart).  Every bounded wait
 * of the bulk-copy FFT pass and the first wait of the tensor-core projector gather try first with
 * `first_polls` polls of their mbarrier (0 restores the default, 2^26); when that first try gives
 * up, the kernel sets its error bit and waits again with the default limit, so the copies and
 * matrix products in flight still complete and no index leaves its buffer.  The next
 * tddft_observables of a handle whose kernels set the bit returns TDDFT_ERR_CUDA (the results of
 * that handle are then invalid: the tensor-core kernels launched after the bit was set skip their
 * work).  Applies to every handle on the current device until called again. */
tddft_status tddft_set_wait_test_limit(unsigned first_polls);

/* Measured peak rates of the current GPU, the denominators of the roofline fractions that the
 * copy bandwidth and the library GEMM do not give (the paper has no counterpart): out[0] FP64 and
 * out[1] FP32 fused multiply-adds on the CUDA cores, out[2] TF32, out[3] FP16 and out[4] BF16 dense
 * tcgen05 products with FP32 accumulation, in TFLOP/s (2 FLOPs per multiply-add), from kernels that
 * touch no global memory, timed with CUDA events (about 0.3 s in all).  Writes min(nout, 5)
 * values; synchronises the device; allocates and frees a few bytes of device memory.  Errors:
 * TDDFT_ERR_ARG (null out or nout < 1), TDDFT_ERR_CUDA. */
tddft_status tddft_measure_peaks(double* out, int nout);

/* Use this CUDA stream (a cudaStream_t; NULL = legacy default stream) for all work. */
tddft_status tddft_set_stream(tddft_handle h, void* stream);

/* Introspection: Chebyshev orders for dt and dt/2, the spectral window, and the number of
 * kernel launches issued since creation.  Any pointer may be NULL. */
tddft_status tddft_info(tddft_handle h, int* K_full, int* K_half, double* e_min, double* e_max,
                        long long* launches);

/* Per-kernel-class timing with CUDA events on the handle's stream.  enable = 1 starts
 * (and clears) recording; tddft_profile_read synchronises and returns, for class c,
 * ms[c] total milliseconds, count[c] launches and bytes[c] the algorithmic DRAM bytes of
 * those launches (each spinor array a launch must read or write counted once; tables
 * shared by all spinors not counted).  Classes: 0 FFT xy-plane pass, 1 FFT z pass with
 * kinetic multiply, 2 Hamiltonian/Chebyshev epilogue, 3 projector gather, 4 density,
 * 5 potential (XC, Hartree, assembly), 6 other, 7 projector scatter on the tensor cores.
 * ncls <= 8; any output may be NULL. */
tddft_status tddft_profile(tddft_handle h, int enable);
tddft_status tddft_profile_read(tddft_handle h, int ncls, double* ms, long long* count, double* bytes);

/* Allocation-free Hartree (Poisson) solve; the paper has no counterpart to this entry
 * point.  For callers that cannot allocate device memory -- frameworks that reserve all
 * device memory up front and forbid further allocations, or loops that cannot afford an
 * allocation's implicit synchronisation.
 *
 * Computes v_H(r) = sum_{G != 0} 4 pi n(G) / |G|^2 exp(i G.r) / N^3 (G = 0 term dropped), the
 * same Hartree potential the library adds to V_v, for a real density n[N^3] on an n x n x n
 * grid of the orthorhombic cell with side lengths L[3] (bohr).  n_dev and vH_dev are device
 * pointers (FP64, [z][y][x]) on the current device; the caller owns both; work is queued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) and the call returns without
 * synchronising.
 *
 * It allocates nothing: no cudaMalloc, cudaFree or allocating library routine.  Its scratch
 * is one file-scope static device array of 64^3 + 64 complex FP64 values (4 MiB + 1 KiB),
 * present on every GPU that loads the library until the process exits.  Hence n must be one
 * of 8, 12, 16, 24, 32, 48, 64; larger grids return TDDFT_ERR_ARG.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not call the entry point
 * again in a process that has reset the device (cudaDeviceReset), whose cached address is gone.  Every call on a device shares the array, so calls that overlap on the
 * GPU (different streams, or host threads) race with each other; each call overwrites the
 * part it uses before reading it, so nothing carries over from earlier calls.
 * Errors: TDDFT_ERR_ARG (null pointer, unsupported n, non-positive L), TDDFT_ERR_CUDA;
 * tddft_last_error(NULL) describes the failure. */
tddft_status tddft_hartree_noalloc(const double* n_dev, double* vH_dev, int n, const double* L, void* stream);

/* Message describing the last failure on this handle (or, when h is NULL, the last failed
 * tddft_create or tddft_hartree_noalloc).  The string stays valid until the next call on
 * the handle. */
const char* tddft_last_error(tddft_handle h);

/* Release the handle and all its device memory.  NULL is accepted. */
void tddft_destroy(tddft_handle h);

#ifdef __cplusplus
}
#endif
#endif /* TDDFT_H */
