/*
 * mala.h -- C ABI of the GB300 (sm_103a) MALA inference hot path.
 *
 * The library computes, for every point of a real-space grid, the SNAP-style
 * bispectrum descriptors of the atoms within a cutoff (paper Sec. "Bispectrum
 * descriptors", Eqs. ionicdensity, SNAPExpansion, snap_dim), feeds them through
 * a per-point feed-forward network (Sec. "Machine learning with neural
 * networks", Eq. ffnn) to the local density of states (LDOS) on N_E energies,
 * and integrates the LDOS into the density of states D(e) (Eq. DOS.from.ldos),
 * the Fermi level (root of the electron-count equation, Sec. "Observable
 * calculation"), the band energy (Eq. band.energy) and the electronic density
 * n(r) (Eq. density.from.ldos), with the energy integrals evaluated as weighted
 * sums (Eqs. ldosintegralgeneral, ldosintegralsummation, fermidiracspecial).
 *
 * Conventions shared by every entry point
 *   - Status: every call returns MALA_OK (0), MALA_PENDING (1) or a negative
 *     MALA_ERR_* code and never aborts; mala_last_error() gives a message for
 *     the calling thread's last non-OK status.  Nothing throws across the ABI.
 *   - Units: Angstrom for lengths, eV for energies.
 *   - Grid: point (ix, iy, iz) of an orthorhombic cell with side lengths
 *     L = diag(cell) sits at ((ix/Nx) Lx, (iy/Ny) Ly, (iz/Nz) Lz); its flat
 *     index is p = ix + Nx (iy + Ny iz); P = Nx Ny Nz.  Only orthorhombic
 *     cells are accepted (MALA_ERR_UNSUPPORTED otherwise).
 *   - Host vs device: pointers documented as "host" are read during the call
 *     and may be freed on return; "device" pointers must be device memory of
 *     the context's GPU, written in stream order on `stream`.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that return host results (fermi, band energy, D(e)) synchronise
 *     that stream before returning.
 *   - Precision: MALA_MIXED computes descriptors in FP32 (compensated sum over
 *     neighbours), the network in BF16 on the tensor cores with FP32
 *     accumulation, and the Fermi level, weights and energy reductions in FP64;
 *     MALA_FP64_PLAIN computes every step in FP64 on the GPU.
 */
#ifndef MALA_H
#define MALA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MALA_OK 0
#define MALA_PENDING 1
#define MALA_ERR_INVALID_ARG (-1)
#define MALA_ERR_OOM (-2)          /* allocation failed or the context's HBM budget is exceeded */
#define MALA_ERR_UNSUPPORTED (-3)  /* valid input outside what this build handles */
#define MALA_ERR_FERMI_BRACKET (-4)/* N(mu) - N_e has no sign change on the bracket */
#define MALA_ERR_TIMEOUT (-5)      /* a bounded device or host wait ran out */
#define MALA_ERR_CUDA (-6)         /* a CUDA runtime/driver call failed */
#define MALA_ERR_NOT_FOUND (-7)    /* unknown ticket */

typedef enum { MALA_FP64_PLAIN = 0, MALA_MIXED = 1 } mala_precision;

typedef struct mala_ctx mala_ctx;
typedef struct mala_model mala_model;

/* One atomic configuration (host memory).  species may be NULL (all 0). */
typedef struct {
    int32_t n_atoms;
    const double* pos;       /* host [n_atoms][3], Cartesian */
    const int32_t* species;  /* host [n_atoms], values 0..n_species-1, or NULL */
    double cell[3][3];       /* rows are the lattice vectors; must be diagonal */
    int32_t grid[3];         /* Nx, Ny, Nz >= 1 */
    int32_t periodic[3];     /* 1 = periodic along that axis, 0 = open */
} mala_snapshot;

/* Descriptor hyperparameters.  f_c(r) = (cos(pi (r-rmin0)/(rcut-rmin0)) + 1)/2,
 * omega = rfac0 pi (r-rmin0)/(rcut-rmin0); wself is the weight of the delta(0)
 * self term of Eq. (ionicdensity); weights[s] is the element weight w_eta of
 * species s (NULL: 1 for every species).  twojmax must be even and <= 10. */
typedef struct {
    int32_t twojmax;
    double rcut, rfac0, rmin0, wself;
    int32_t n_species;
    const double* weights;   /* host [n_species] or NULL */
} mala_bispectrum_params;

/* Feed-forward network x_{l+1} = act(W_l x_l + b_l), Eq. (ffnn); act is
 * LeakyReLU(leaky_slope) on hidden layers and the identity on the output layer
 * (activate_output = 1 applies it there too).  Optional input standardisation
 * x0 = (B - in_shift) * in_scale.  All arrays are host FP64. */
typedef struct {
    int32_t n_layers;             /* >= 1 */
    const int32_t* dims;          /* host [n_layers + 1]; dims[0] = n_B, dims[n_layers] = N_E */
    const double* const* W;       /* host, W[l] is [dims[l+1]][dims[l]] row-major */
    const double* const* b;       /* host, b[l] is [dims[l+1]] */
    double leaky_slope;
    int32_t activate_output;
    const double* in_shift;       /* host [dims[0]] or NULL */
    const double* in_scale;       /* host [dims[0]] or NULL */
} mala_mlp_desc;

/* Energy grid e_xi = e0 + xi de (xi = 0..n_E-1), electronic temperature kT and
 * electron count N_e for the Fermi level. */
typedef struct {
    int32_t n_E;
    double e0_eV, de_eV, kT_eV, n_electrons;
} mala_energy_grid;

/* Results of a whole prediction (mala_predict, mala_poll). */
typedef struct {
    int32_t status;              /* MALA_OK or an error of that request */
    int32_t n_B, n_E;
    int64_t n_points;
    double fermi_eV;             /* Fermi level */
    double band_energy_eV;       /* E_b = sum_xi w1_xi(eF) D_xi */
    double electron_count;       /* dV sum_r n(r), FP64 */
    const double* dos;           /* host [n_E]: D(e_xi), owned by the library */
    const void* B_dev;           /* device [P][n_B] (float for MIXED, double for FP64_PLAIN) */
    const void* ldos_dev;        /* device [P][n_E] (bf16 for MIXED, double for FP64_PLAIN) */
    const void* density_dev;     /* device [P] (float for MIXED, double for FP64_PLAIN) */
    double submit_to_done_s;     /* serving latency (mala_poll only) */
    double entropy_term_eV;      /* -tau S_s, Eqs. (electronicentropyDOS), (KSfreeenergy) */
    double gpu_start_ms;         /* served requests: device-clock interval of the batch that carried it, */
    double gpu_end_ms;           /* ms since the server started (CUDA events on the slot's stream); else 0 */
} mala_result;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context allocates for its own workspaces (0 = no cap); requests
 * that would exceed it fail with MALA_ERR_OOM.  The context owns its streams,
 * the Clebsch-Gordan tables and its workspaces. */
int mala_create(mala_ctx** out, int device, size_t hbm_budget_bytes);
void mala_destroy(mala_ctx* ctx);
const char* mala_last_error(void);
int mala_version(void);
/* Bytes of device memory the context currently holds. */
size_t mala_device_bytes(const mala_ctx* ctx);

/* Per-kernel timing.  mala_profile(ctx, 1) clears the totals and makes the
 * library bracket each of its kernel launches with CUDA events recorded on the
 * stream the kernel is launched on; mala_profile(ctx, 0) stops recording.
 * mala_profile_get waits for the recorded events and returns the summed
 * duration (ms) and the number of launches of the named kernel ("k_neighbors",
 * "k_ui", "k_zb", "k_mlp", "k_dos_reduce", "k_fermi", "k_density", ...), or
 * of every kernel of the library for the name "all". */
int mala_profile(mala_ctx* ctx, int enable);
int mala_profile_get(mala_ctx* ctx, const char* kernel, double* total_ms, int64_t* launches);

/* Tile-shape tuning (no counterpart in the paper, whose descriptor code runs
 * with fixed shapes).  mode 1, the default: the first MALA_MIXED descriptor
 * pass for a new key (twojmax, neighbour capacity in bands of 8, grid points
 * in powers of two) times every compiled variant of compute_ui (segment length
 * x warps per CTA) and of compute_zi/bi (warps per CTA) on that pass's own
 * data and keeps the fastest for the context and its serving slots; later
 * passes with the key use it.  mode 0: the default variants.  mode 2: the
 * variants ui_variant and zb_variant for every pass (testing).  Every variant
 * adds the same terms in the same order, so all give the same bits.  Modes 0
 * and 2 forget earlier choices. */
int mala_set_tuning(mala_ctx* ctx, int mode, int ui_variant, int zb_variant);
/* Numbers of compiled compute_ui and compute_zi/bi variants (host only). */
int mala_tuning_variants(int32_t* n_ui, int32_t* n_zb);
/* The choices made so far, one line per key with every variant's time, as
 * NUL-terminated text in buf (truncated to len bytes). */
int mala_tuning_report(mala_ctx* ctx, char* buf, size_t len);

/* The CUDA-core peaks of the context's device, measured (no counterpart in
 * the paper: they are the denominators of the descriptor kernels' roofline
 * fractions).  Independent fused multiply-add chains on every SM, timed by
 * CUDA events on the context's stream, best of three after a warm-up run, an
 * FMA counted as two FLOP: FP32 with scalar FMAs, FP32 with packed FP32x2
 * FMAs, FP64 (any output may be NULL).  Synchronous; about 20 ms. */
int mala_measure_peaks(mala_ctx* ctx, double* fp32_scalar_tflops, double* fp32_packed_tflops,
                       double* fp64_tflops);

/* ---- network ---------------------------------------------------------- */

/* Upload a network once (BF16 copies for MALA_MIXED, FP64 for MALA_FP64_PLAIN);
 * the descriptor arrays may be freed on return.  mala_destroy frees the device
 * memory of the context's remaining networks; mala_model_destroy is still
 * needed afterwards to free the handle itself. */
int mala_model_create(mala_ctx* ctx, const mala_mlp_desc* desc, mala_model** out);
void mala_model_destroy(mala_model* model);

/* ---- the hot path, one step at a time ----------------------------------- */

/* Neighbour lists of every grid point (Eq. ionicdensity: |R_a + s L - r| < rcut,
 * strict, over all periodic images s).  Membership is decided in FP64 exactly
 * as (x_a + s L) - r rounded without fused multiply-add where FP32 cannot
 * decide it.  Outputs (device, point-major): counts[P]; atoms[P][cap] and
 * shifts[P][cap][3] (image shift s) for the first min(count, cap) neighbours in
 * an unspecified order.  *max_count (host) receives the largest count. */
int mala_neighbor_lists(mala_ctx* ctx, const mala_snapshot* snap, double rcut, int32_t cap,
                        int32_t* counts_dev, int32_t* atoms_dev, int32_t* shifts_dev,
                        int32_t* max_count, void* stream);

/* Bispectrum descriptors B[P][n_B] (device; float for MALA_MIXED, double for
 * MALA_FP64_PLAIN) with n_B = (twojmax+2)(twojmax+3)(twojmax+4)/24, component
 * order lexicographic in (J1, J2, J) over 0 <= J2 <= J1 <= J <= twojmax,
 * J1+J2+J even, |J1-J2| <= J <= J1+J2 (Eq. snap_dim). */
int mala_descriptors(mala_ctx* ctx, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                     void* B_dev, mala_precision precision, void* stream);

/* Descriptors of n snapshots (snaps[0..n), any mix of atom counts, cells and
 * grids, one bispectrum setting) in one sequence of launches: the snapshots'
 * grid tiles are numbered one after another and every kernel launch walks
 * tiles of several snapshots.  B_dev holds the snapshots' rows in order,
 * [sum_i P_i][n_B] (P_i = the product of snaps[i].grid); each snapshot's rows
 * are bit for bit those mala_descriptors gives for it alone. */
int mala_descriptors_batch(mala_ctx* ctx, int32_t n, const mala_snapshot* snaps, const mala_bispectrum_params* bp,
                           void* B_dev, mala_precision precision, void* stream);

/* Gaussian descriptors (Sec. "Total energy calculation", Eq. structfact_function
 * with a Gaussian f, the "Gaussian representation" of the atomic positions):
 * for every grid point r, G(r) = sum over atoms alpha and periodic images s
 * with |R_alpha + s L - r| < rcut (the membership rule of mala_neighbor_lists)
 * of exp(-|R_alpha + s L - r|^2 / (2 sigma^2)).  G_dev: device [P], float for
 * MALA_MIXED (offsets as float pairs, FP32 sum), double for MALA_FP64_PLAIN. */
int mala_gaussian_descriptors(mala_ctx* ctx, const mala_snapshot* snap, double rcut, double sigma, void* G_dev,
                              mala_precision precision, void* stream);

/* Expansion coefficients u^J of Eq. (SNAPExpansion) for every grid point,
 * J = 0..twojmax, device complex output u_dev[P][sum_J (J+1)^2][2] (row-major
 * [ma][mb] blocks in increasing J; float for MIXED, double for FP64_PLAIN). */
int mala_expansion_coefficients(mala_ctx* ctx, const mala_snapshot* snap,
                                const mala_bispectrum_params* bp, void* u_dev,
                                mala_precision precision, void* stream);

/* LDOS[P][N_E] = network(B) (device; bf16 for MALA_MIXED, double for
 * MALA_FP64_PLAIN).  B_dev as written by mala_descriptors with the same
 * precision.  dos_sum_dev (device double [N_E], may be NULL) receives the
 * column sums sum_r LDOS(r, xi) of the values written to ldos_dev. */
int mala_ldos_forward(mala_ctx* ctx, const mala_model* model, const void* B_dev, int64_t P,
                      void* ldos_dev, double* dos_sum_dev, mala_precision precision, void* stream);

/* Energy integrals of an LDOS[P][N_E] (device, bf16 for MIXED, double for
 * FP64_PLAIN) on a cell of volume cell_volume: D_xi = dV sum_r LDOS(r, xi)
 * with dV = cell_volume / P; the Fermi level by FP64 bisection of
 * N(mu) = sum_xi w0_xi(mu) D_xi - N_e on [e_0 - 20 kT, e_max + 20 kT] down to a
 * width of 1e-12 eV (at most 200 halvings); the band energy sum_xi w1_xi D_xi;
 * the density n(r) = sum_xi w0_xi(eF) LDOS(r, xi) into density_dev (device
 * [P], float for MIXED, double for FP64_PLAIN).  w0/w1 are the exact integrals
 * of the piecewise-linear interpolant times e^0 / e^1 times the Fermi function,
 * in closed form through Li2/Li3.  dos_sum_dev (device [N_E], may be NULL)
 * supplies precomputed column sums (mala_ldos_forward's); otherwise they are
 * computed from ldos_dev.  Host outputs (any may be NULL): dos_host[N_E],
 * fermi_eV, band_energy_eV, electron_count (dV sum_r n(r) in FP64) and
 * entropy_term_eV = -tau S_s = -kT sum_xi wS_xi D_xi, the entropy contribution
 * to the free energy (Eqs. electronicentropyDOS, KSfreeenergy), wS the exact
 * integrals of the interpolant times -[f ln f + (1-f) ln(1-f)], also in closed
 * form through Li2/Li3. */
int mala_integrate(mala_ctx* ctx, const void* ldos_dev, int64_t P, double cell_volume,
                   const mala_energy_grid* eg, const double* dos_sum_dev, void* density_dev,
                   double* dos_host, double* fermi_eV, double* band_energy_eV,
                   double* electron_count, double* entropy_term_eV, mala_precision precision, void* stream);

/* mala_integrate without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (their
 * process's device memory belongs to another framework's allocator, they run
 * under a hard memory cap, or they cannot afford the device-wide
 * synchronisation an allocation may imply).  Arguments, outputs and results
 * are those of mala_integrate; every scratch buffer comes from one fixed
 * static device array of MALA_NOALLOC_SCRATCH_BYTES that each GPU loading the
 * library holds until the process exits.  Limit: 9.5 n_E + 296 + max(
 * ceil(P/128) n_E [only when dos_sum_dev is NULL], the CTAs of the density
 * pass [at most six per SM]) doubles must fit in the array; larger sizes
 * return MALA_ERR_UNSUPPORTED with the numbers in the message.  Every call
 * looks up the array's device address in the current context (a host-side
 * query, no allocation); make the first call on a device before any stream
 * capture.  All calls share the array and leave their contents in it: calls
 * that overlap on the GPU (other streams or threads) race, so issue them one
 * at a time.  Host copies go through the context's pinned buffer and
 * directly into dos_host. */
#define MALA_NOALLOC_SCRATCH_BYTES (8u << 20)
int mala_integrate_noalloc(mala_ctx* ctx, const void* ldos_dev, int64_t P, double cell_volume,
                           const mala_energy_grid* eg, const double* dos_sum_dev, void* density_dev,
                           double* dos_host, double* fermi_eV, double* band_energy_eV,
                           double* electron_count, double* entropy_term_eV, mala_precision precision,
                           void* stream);

/* Electron count N(mu) = sum_xi w0_xi(mu) D_xi of a density of states D (host
 * [n_E], the values mala_integrate returns in dos_host) at chemical potential
 * mu, with the same FP64 closed-form weights the Fermi-level search uses.
 * eg->n_electrons is ignored.  Synchronous. */
int mala_electron_count(mala_ctx* ctx, const double* dos_host, const mala_energy_grid* eg, double mu,
                        double* count);

/* ---- band-energy forces (Sec. "Total energy calculation", Eqs. forces and
 * forcesmala with E = E_b of Eq. band.energy) ------------------------------
 *
 * f_alpha = -dE_b/dR_alpha = -(dE_b/d LDOS)(d LDOS/dB)(dB/dR_alpha), evaluated
 * right to left as the paper prescribes: a vector per grid point, the
 * network's backward pass, then the descriptor adjoint.  Each factor has its
 * own entry point.  MALA_MIXED: FP32 descriptors and u, FP32 backward pass
 * (the library's own register-tiled GEMM for the dense products), FP32
 * adjoint, forces summed per atom
 * in 2^-40 fixed point (order-independent).  MALA_FP64_PLAIN: the same in
 * FP64.  Synchronous; forces_host is [n_atoms][3] doubles in eV/Angstrom. */

/* dE_b/dD_xi at fixed electron number (the first factor divided by dV):
 * E_b = sum w1_xi(mu) D_xi with mu(D) fixed by N(mu) = eg->n_electrons, so
 * dE_b/dD_xi = w1_xi - mu~ w0_xi with mu~ = (dE_b/dmu)/(dN/dmu) at fixed D
 * (closed forms for the piecewise-linear D, FP64).  dos_host: D (host, [n_E]);
 * grad_host (host, [n_E]); *fermi the Fermi level, *mu_tilde = mu~ (either may
 * be NULL).  Errors: MALA_ERR_FERMI_BRACKET as in mala_integrate,
 * MALA_ERR_UNSUPPORTED when dN/dmu = 0. */
int mala_band_energy_gradient(mala_ctx* ctx, const double* dos_host, const mala_energy_grid* eg,
                              double* grad_host, double* fermi, double* mu_tilde, void* stream);

/* The network's vector-Jacobian product: beta[p][j] = sum_e v[e] dLDOS[p][e]/dB[p][j]
 * for every row of B (device, [P][n_B], float for MALA_MIXED, double for
 * MALA_FP64_PLAIN) into beta_dev (device, same type and shape); v_host: host
 * [n_E] doubles.  LeakyReLU derivatives use sigma'(0) = slope. */
int mala_ldos_backward(mala_ctx* ctx, const mala_model* model, const void* B_dev, int64_t P,
                       const double* v_host, void* beta_dev, mala_precision precision, void* stream);

/* The descriptor adjoint: forces_host[a][k] = -sum_r sum_j beta[r][j] dB(r, j)/dR_{a,k}
 * over every grid point r of the snapshot (beta_dev: device [P][n_B], float for
 * MALA_MIXED, double for MALA_FP64_PLAIN, rows in grid order).  The neighbour
 * sets are those of mala_neighbor_lists; positions enter through every
 * periodic image. */
int mala_descriptor_forces(mala_ctx* ctx, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                           const void* beta_dev, double* forces_host, mala_precision precision, void* stream);

/* The whole chain: the forward path of mala_predict (result in *res, device
 * pointers into the context's workspace as there) followed by the three
 * factors; forces_host: [n_atoms][3].  On MALA_ERR_FERMI_BRACKET no forces are
 * written. */
int mala_band_forces(mala_ctx* ctx, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                     const mala_model* model, const mala_energy_grid* eg, mala_precision precision,
                     double* forces_host, mala_result* res, void* stream);

/* ---- the whole path ----------------------------------------------------- */

/* Descriptors -> LDOS -> integrals for one snapshot.  Intermediate B and LDOS
 * live in the context's workspace; result->B_dev / ldos_dev / density_dev point
 * into it and stay valid until the next call on this context.
 * density_host (host [P], float for MIXED, double for FP64_PLAIN; may be NULL)
 * receives a copy of n(r).  Synchronises `stream`. */
int mala_predict(mala_ctx* ctx, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                 const mala_model* model, const mala_energy_grid* eg, mala_precision precision,
                 void* density_host, mala_result* result, void* stream);

/* The whole path for n snapshots at once (Sec. "Observable calculation" per
 * snapshot): descriptors of all snapshots as in mala_descriptors_batch, the
 * network over all their points in one launch, then the integrals of each
 * snapshot with its own energy grid / electron count egs[i].  results[i]
 * describes snapshot i: its B, LDOS and density pointers are its rows inside
 * the context's workspace (valid until the next call on the context), its
 * dos points to library-owned host memory.  density_host (host [sum_i P_i],
 * float for MIXED, double for FP64_PLAIN; may be NULL) receives n(r) of all
 * snapshots in order.  A snapshot whose electron count has no bracket gets
 * status MALA_ERR_FERMI_BRACKET in its result; the call returns the first
 * failure (MALA_OK when all succeeded).  Synchronises `stream`. */
int mala_predict_batch(mala_ctx* ctx, int32_t n, const mala_snapshot* snaps, const mala_bispectrum_params* bp,
                       const mala_model* model, const mala_energy_grid* egs, mala_precision precision,
                       void* density_host, mala_result* results, void* stream);

/* ---- grid-centred ACE descriptors (Sec. "Atomic cluster expansion
 * descriptors", Eqs. unweighted_ionicdensity .. ace_grid) ------------------
 *
 * Grid basis A_{mu n l m}(r) = sum over the neighbours of r of species mu (all
 * periodic images within rcut, the membership rule of mala_neighbor_lists) of
 * R_n(|d|) Y_l^m(d/|d|), d = R_alpha - r, with
 * R_n(r) = T_n(1 - 2r/rcut) (1 + cos(pi r/rcut))/2 (Chebyshev polynomials of the
 * first kind) and complex orthonormal spherical harmonics (Condon-Shortley
 * phase); no element weights, no self term; an atom on the grid point adds to
 * l = 0 only.  Invariants, column order:
 *   N = 1: A_{mu n 0 0}, for (mu, n), n < nmax1;
 *   N = 2: sum_m <l m l -m|0 0> A_{c1 l m} A_{c2 l -m}, for channel pairs c1 <= c2
 *          of (mu, n), n < nmax2 (lexicographic), then l = 0..lmax2;
 *   N = 3: sum <l1 m1 l2 m2|l3 M><l3 M l3 -M|0 0> A_{c1 l1 m1} A_{c2 l2 m2} A_{c3 l3 -M}
 *          for sorted triples c1 <= c2 <= c3 of channels (mu, n, l), n < nmax3,
 *          l <= lmax3 (lexicographic), |l1 - l2| <= l3 <= l1 + l2, l1 + l2 + l3 even.
 * Limits: n_species <= 8, max(nmax) <= 16, max(lmax) <= 8,
 * n_species x max(nmax) x (lmax+1)(lmax+2)/2 <= 1024 (MALA_ERR_UNSUPPORTED beyond). */
typedef struct {
    double rcut;        /* Angstrom */
    int32_t n_species;  /* snapshot species indices must lie in 0..n_species-1 */
    int32_t nmax1;      /* radial functions of the N = 1 columns */
    int32_t nmax2, lmax2;
    int32_t nmax3, lmax3;
} mala_ace_params;

/* Number of ACE columns for the parameters (host only, no context). */
int mala_ace_count(const mala_ace_params* params, int32_t* n_desc);

/* ACE descriptors D[P][n_desc] (device; float for MALA_MIXED, double for
 * MALA_FP64_PLAIN) of one snapshot.  Synchronous. */
int mala_ace_descriptors(mala_ctx* ctx, const mala_snapshot* snap, const mala_ace_params* params, void* D_dev,
                         mala_precision precision, void* stream);

/* ---- serving ------------------------------------------------------------ */

/* Queue a prediction.  The library copies every input (the caller may free
 * them on return), admits the request when its device memory fits in the
 * budget, and runs it on the GPU concurrently with other admitted requests.
 * A free serving slot takes the oldest queued request that fits together with
 * the later queued ones of the same network, precision, bispectrum setting and
 * n_E (up to 16 requests, 8e6 grid points, within the budget) and runs them as
 * one batch (mala_predict_batch's path): LDOS rows are those of a lone run bit
 * for bit; the DOS sums, hence the integrals, may differ from a lone run in the
 * last bits.  Non-blocking; *ticket identifies the request. */
int mala_submit(mala_ctx* ctx, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                const mala_model* model, const mala_energy_grid* eg, mala_precision precision,
                uint64_t* ticket);
/* MALA_PENDING while the request runs, MALA_OK when *out is filled (device
 * pointers stay valid until mala_release), or the request's error. */
int mala_poll(mala_ctx* ctx, uint64_t ticket, mala_result* out);
/* Block until the ticket completes or timeout_s passes (MALA_ERR_TIMEOUT). */
int mala_wait(mala_ctx* ctx, uint64_t ticket, double timeout_s, mala_result* out);
/* Free the device outputs of a completed request (a batch's shared outputs
 * are freed when its last request is released). */
int mala_release(mala_ctx* ctx, uint64_t ticket);

#ifdef __cplusplus
}
#endif
#endif /* MALA_H */
