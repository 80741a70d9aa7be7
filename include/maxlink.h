/*
 * maxlink.h - C ABI of the GB300-native coupled Yee FDTD / molecular-ensemble step.
 *
 * Method: arXiv 2512.06173 (MaxwellLink), Sec. II.A.1 and II.B.1.  One time step
 * advances a 3D Yee grid (Eq. Maxwell with the constitutive relation Eq. Dromega)
 * with CPML absorbing layers, lets every molecule gather its regularised field
 * (Eq. E_regu_Emi), advance its density matrix (Eq. von-Neumann-tls, optional
 * Lindblad terms) and scatter its current gamma * d<mu>/dt * kappa (Eq. J_mol,
 * Eq. Polarization_mol) into the E update.  All of the step runs in CUDA kernels
 * for sm_103a; there is no CPU fallback.
 *
 * Conventions (all entry points):
 *   - Units c = eps0 = mu0 = hbar = 1, cell edge 1 (Appendix A), dt = Courant number.
 *   - Staggering: Ex(i,j,k) at (i+1/2,j,k), Ey at (i,j+1/2,k), Ez at (i,j,k+1/2),
 *     Hx at (i,j+1/2,k+1/2), Hy at (i+1/2,j,k+1/2), Hz at (i+1/2,j+1/2,k);
 *     E lives at integer steps, H at half steps.
 *   - Host arrays over the grid are (nz, ny, nx) row-major, x fastest.
 *   - Non-periodic axes end in PEC walls at index 0 and n (behind the CPML, if any).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that only enqueue work return before it finishes; device-side
 *     failures are latched in a status word read by ml_sync_status.
 *   - Every call returns an ml_status; ml_last_error() gives a message for the
 *     last failure on the calling thread.  No exception crosses the ABI.
 *   - The library copies every input; the caller keeps ownership of its buffers.
 *     Device memory of a grid is owned by the library until ml_grid_destroy; it comes
 *     from the allocator of ml_set_allocator.
 */
#ifndef MAXLINK_H
#define MAXLINK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ML_OK = 0,
    ML_ERR_INVALID_ARG = 1, /* bad size, index, pointer or combination of options */
    ML_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    ML_ERR_OOM = 3,         /* device allocation failed */
    ML_ERR_STATE = 4,       /* call not valid in the object's current state */
    ML_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    ML_ERR_NUMERIC = 6      /* a NaN or Inf reached a molecule's field or current */
} ml_status;

typedef enum { ML_F32 = 0, ML_F64 = 1 } ml_precision;

typedef struct ml_grid ml_grid;

/* Dispersive pole (Sec. II.A.1 mentions Drude/Lorentz dielectric functions):
 * dJ/dt + gamma J + omega0^2 P = wp^2 E with dP/dt = J.  omega0 = 0: a Drude term;
 * omega0 > 0: a Lorentz oscillator of strength wp^2 = delta_eps omega0^2.  Advanced by
 * the centred ADE J^{n+1/2} = [(1 - gamma dt/2) J^{n-1/2} + dt (wp^2 E^n - omega0^2 P^n)]
 * / (1 + gamma dt/2), P^{n+1} = P^n + dt J^{n+1/2}. */
typedef struct {
    double wp, gamma, omega0;
} ml_pole;

#define ML_MAX_POLES 4  /* dispersive poles per material */

/* Material of a cell: eps_inf and up to ML_MAX_POLES poles whose currents add up in
 * the E update.  The first pole is (wp, gamma, omega0), the others extra[0..n_extra);
 * a pole with wp = 0 is absent.  n_extra outside 0..ML_MAX_POLES-1, eps_inf <= 0, or a
 * negative omega0 or gamma is ML_ERR_INVALID_ARG.  A zero-initialised tail (n_extra =
 * 0) gives the single-pole material. */
typedef struct {
    double eps_inf, wp, gamma, omega0;
    int n_extra;
    ml_pole extra[ML_MAX_POLES - 1];
} ml_material;

/* Soft current-sheet source on the plane `index` normal to `axis`, polarised along
 * `comp` (comp != axis): J_comp(t) = amp exp(-((t-t0)/width)^2/2) cos(omega (t-t0)),
 * evaluated at t = (n+1/2) dt (the Gaussian-pulse plane wave of Appendix B). */
typedef struct {
    int axis, index, comp;
    double amp, omega, width, t0;
} ml_source;

#define ML_MAX_SOURCES 4
#define ML_MAX_MATERIALS 64
#define ML_MAX_LEVELS 8
#define ML_MAX_FREQS 64

typedef struct {
    int nx, ny, nz;             /* cells, each >= 1 */
    double courant;             /* dt; stable for courant <= 1/sqrt(3) in 3D */
    int precision;              /* ML_F32 or ML_F64: field and molecule arithmetic */
    int periodic[3];            /* 1 = periodic axis (no CPML allowed on it) */
    int pml[6];                 /* CPML cells on faces x-,x+,y-,y+,z-,z+ */
    double pml_m;               /* grading exponent (3) */
    double pml_sigma_max;       /* sigma at the outer wall (0.8 (m+1) = 3.2) */
    double pml_kappa_max;       /* kappa at the outer wall (>= 1) */
    double pml_alpha_max;       /* alpha at the inner edge, decreasing linearly (0.05) */
    const uint8_t *mat;         /* host (nz,ny,nx) material index, or NULL = material 0 */
    int n_materials;            /* 1..ML_MAX_MATERIALS */
    const ml_material *materials;
    int design_box[6];          /* x0,y0,z0,sx,sy,sz of a continuous-eps region (sx=0: none) */
    const double *design_eps;   /* host (sz,sy,sx) relative permittivity, no Drude inside */
    int n_sources;              /* 0..ML_MAX_SOURCES */
    const ml_source *sources;
    int zchunk;                 /* planes per z chunk of the field pass: 0 = automatic
                                   (about 8 blocks per SM for this grid alone), >= 2 = that
                                   length (longer chunks suit grids stepped in a batch,
                                   where other grids fill the GPU); 1 or < 0 is
                                   ML_ERR_INVALID_ARG.  The results do not depend on it
                                   except the summation order of ml_absorbed. */
} ml_grid_desc;

/* Molecule table (Sec. II.B.1).  Matrices are n x n row-major complex numbers
 * stored as interleaved (re, im) doubles in shared pools; molecule m's matrices
 * start at complex element off[m].  H0 and the three dipole operators must be
 * Hermitian; rho a density matrix. */
typedef struct {
    int count;
    const int32_t *nlev;        /* 2..ML_MAX_LEVELS */
    const int64_t *off;         /* offset into the pools, complex elements */
    const double *pos;          /* (count,3) centre in grid units */
    const double *sigma;        /* Gaussian width in cells; ceil(3 sigma) <= 7 */
    const double *gamma;        /* coupling rescale of Eq. Polarization_mol */
    const double *decay;        /* ladder decay rate: L_k = sqrt(decay)|k-1><k| */
    const double *dephase;      /* pure dephasing:    L_k = sqrt(dephase)|k><k|  */
    const int32_t *kind;        /* 0: exact 2x2 unitary (n=2, no Lindblad); 1: RK4 */
    const int32_t *nsub;        /* RK4 substeps per field step (>= 1) */
    const double *H0;           /* pool, interleaved complex */
    const double *mu;           /* 3 pools back to back (x, y, z), each `pool` complex */
    const double *rho;          /* pool, initial density matrices */
    int64_t pool;               /* complex elements in each pool */
} ml_molecule_desc;

/* what to read with ml_get_molecules (all as double) */
enum {
    ML_MOL_RHO = 0,     /* pool of interleaved complex rho (2*pool doubles) */
    ML_MOL_EFIELD = 1,  /* (count,3) regularised field of the last step (Eq. E_regu_Em); a
                           component along which all of the molecule's dipole operators
                           vanish does not enter its Hamiltonian, is not gathered and reads 0 */
    ML_MOL_MUDOT = 2,   /* (count,3) d<mu>/dt of the last step (Eq. dipole_derivative) */
    ML_MOL_ENERGY = 3,  /* (count) sum over steps of Tr(rho H0) (time average = / steps) */
    ML_MOL_POP = 4      /* (count, ML_MAX_LEVELS) diagonal of rho, zero-padded */
};

/* component mask bits for ml_get_fields / ml_set_fields (order of the copies) */
enum { ML_EX = 1, ML_EY = 2, ML_EZ = 4, ML_HX = 8, ML_HY = 16, ML_HZ = 32, ML_ALL = 63 };

/* ---- Device memory ---------------------------------------------------------------
 * The paper's problem statement (Sec. III) keeps the EM solver and the molecular drivers
 * in separate programs with their own memory; here both live in one process next to the
 * caller's framework, so every device buffer the library allocates (grids, molecule
 * tables, flux planes, batches, the adjoint's work memory, cavities, drives) comes from
 * one process-wide allocator that the caller may supply:
 *   alloc(&ptr, bytes, stream, ctx): return 0 and set *ptr to at least `bytes` bytes of
 *       device memory of the current device, 256-byte aligned; nonzero (or a NULL *ptr)
 *       when it cannot, and the library call then fails with ML_ERR_OOM;
 *   free(ptr, bytes, stream, ctx): give a buffer back.
 * `stream` is NULL (the legacy default stream): the library zeroes new memory on that
 * stream, waits for it, and frees only after the work that used the memory has finished.
 * The default allocator is cudaMallocAsync / cudaFreeAsync on that stream.  The Python
 * binding installs one backed by PyTorch's caching allocator when it loads the library.
 * Every buffer is returned to the allocator it came from, so the allocator may be
 * replaced at any time; `ctx` must stay valid while buffers from it are alive.
 * ml_set_allocator(NULL, NULL, NULL) restores the default.  ml_gather_static allocates
 * nothing and does not use the allocator.  Error: ML_ERR_INVALID_ARG when exactly one
 * of the two functions is NULL. */
typedef int (*ml_alloc_fn)(void **ptr, size_t bytes, void *stream, void *ctx);
typedef void (*ml_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
ml_status ml_set_allocator(ml_alloc_fn alloc, ml_free_fn free_fn, void *ctx);

/* Message of the last failure on this thread ("" if none).  Never NULL. */
const char *ml_last_error(void);

/* Version string of the library build.  0.2: ml_material carries up to ML_MAX_POLES
 * dispersive poles (omega0, n_extra, extra[]) and ml_grid_desc ends with zchunk; a
 * caller built against 0.1 descriptors must be rebuilt.  0.3 adds entry points only
 * (ml_set_allocator, ml_set_wait_limit, ml_batch_set_timing / ml_batch_timing,
 * ml_gather_static); 0.2 callers need no change. */
const char *ml_version(void);

/* Create a grid (Eq. Maxwell on a Yee lattice, Eq. Dromega per cell), zero fields.
 * Copies the descriptor's arrays.  *out receives the handle. */
ml_status ml_grid_create(const ml_grid_desc *desc, void *stream, ml_grid **out);

/* Free all device memory of the grid.  Synchronises the device. */
ml_status ml_grid_destroy(ml_grid *g);

/* Append molecules (Eq. Polarization_mol: centre, Gaussian width, coupling, and the
 * Sec. II.B.1 model: H0, dipole operators, Lindblad rates, initial rho).  Their
 * kernel windows must lie inside the grid on non-periodic axes.  Builds the kernel
 * weights and the cell-binned molecule lists.  *first_id (may be NULL) receives the
 * index of the first appended molecule. */
ml_status ml_add_molecules(ml_grid *g, const ml_molecule_desc *m, void *stream, int *first_id);

/* Add a DFT flux plane: E-plane `index` normal to `axis`, nfreq frequencies.  The
 * accumulators integrate E(t=(n+1)dt) and H(t=(n+1/2)dt) with weight e^{i w t} dt
 * from the next step on.  *id receives the plane index. */
ml_status ml_add_flux_plane(ml_grid *g, int axis, int index, int nfreq, const double *omega, int *id);

/* Enqueue nsteps coupled time steps on `stream`. */
ml_status ml_step(ml_grid *g, int64_t nsteps, void *stream);

/* Copy the selected components (mask of ML_EX..ML_HZ, in that order) to dst:
 * each nz*ny*nx elements of the grid's precision.  dst is device memory if
 * dst_on_device, else host memory (the call then synchronises `stream`). */
ml_status ml_get_fields(ml_grid *g, unsigned mask, void *dst, int dst_on_device, void *stream);

/* Overwrite the selected components from src (same layout as ml_get_fields).
 * Tangential E on PEC walls is kept at zero by every later step. */
ml_status ml_set_fields(ml_grid *g, unsigned mask, const void *src, int src_on_device, void *stream);

/* Read molecular state `what` (ML_MOL_*) as doubles into dst.  dst_on_device: 1 = dst is
 * device memory; 0 = host memory, the call synchronises `stream`; 2 = page-locked host
 * memory, the copy is enqueued on `stream` and the call returns at once (dst holds the
 * values once the stream reaches the copy; the caller synchronises before reading).  Modes 0
 * and 2 stage through one device buffer of the grid: calls on different streams are ordered
 * by the caller.  Error: ML_ERR_INVALID_ARG for another dst_on_device. */
ml_status ml_get_molecules(ml_grid *g, int what, double *dst, int dst_on_device, void *stream);

/* Population sink: every later ml_step writes the level populations of the new state
 * (the diagonal of rho^{n+1}, Eq. population_decay_superradiance's P_e for two levels) of
 * molecule m, as doubles, into
 *     host[((s mod ring_steps) * count + m) * ML_MAX_LEVELS + l],  l < nlev(m),
 * where s is the index of the step being taken (ml_step_count before it); the other
 * entries are never written.  The molecule kernel stores them directly into `host`, which
 * must be page-locked host memory the device can address (cudaHostAlloc, cudaMallocHost
 * or cudaHostRegister), so no copy or extra kernel enters the stream; the values of a
 * step are in place once the stream has passed that step.  `host` stays owned by the
 * caller and must outlive the sink.  NULL removes the sink.  Batches (ml_batch_step) and
 * the sweeps of ml_adjoint_run do not write it.  Errors: ML_ERR_INVALID_ARG for
 * ring_steps < 1 or a pointer the device cannot address. */
ml_status ml_set_population_sink(ml_grid *g, double *host, int64_t ring_steps);

/* Net flux through plane `id` per frequency: Re sum over the plane of
 * (E~ x H~*) . n (Sec. IV.C, IV.D spectra), H~ averaged over the two half cells
 * around the plane.  out: host, nfreq doubles.  Synchronises `stream`. */
ml_status ml_flux(ml_grid *g, int id, double *out, void *stream);

/* Raw DFT accumulators of plane `id` (E_b, E_c, H_b, H_c with (a,b,c) cyclic, each
 * (nfreq, n_c, n_b) complex) as interleaved doubles into host `out`. */
ml_status ml_flux_data(ml_grid *g, int id, double *out, void *stream);

/* Work done on the dispersive poles so far: sum over pole cells and poles of
 * J_p . (E^n + E^{n+1})/2 dt (for a Drude pole the absorbed energy; a Lorentz pole's
 * share includes the energy it stores).  Host out. */
ml_status ml_absorbed(ml_grid *g, double *out, void *stream);

/* Synchronise `stream` and return the latched device status (then clear it):
 * ML_ERR_NUMERIC when a NaN or Inf reached a molecule's regularised field or current,
 * ML_ERR_TIMEOUT when a field-pass block gave up waiting for a plane of its copy ring
 * (the block then waits, bounded, for its own copies in flight and exits without
 * writing the rest of its tile, so the step's fields are not valid; later steps run
 * normally).  The paper's hub detects failed or silent drivers with a barrier and
 * timeouts (Sec. III); here the failure is reported by the device. */
ml_status ml_sync_status(ml_grid *g, void *stream);

/* Bound of the field pass's waits for a plane of its copy ring: `probes` suspended
 * probes of up to 1 ms each (default 2000).  0 makes every wait give up at once, so
 * the next ml_step reports ML_ERR_TIMEOUT through ml_sync_status (a host-side way to
 * exercise the timeout path; nothing is left waiting).  Taken by the next ml_step or
 * ml_batch_step.  Error: ML_ERR_INVALID_ARG outside 0 .. 2^31 - 1. */
ml_status ml_set_wait_limit(ml_grid *g, int64_t probes);

/* Steps taken so far. */
int64_t ml_step_count(const ml_grid *g);

/* Number of molecules. */
int ml_molecule_count(const ml_grid *g);

/* Per-kernel timing (tracing).  With ml_set_timing(g, 1) every kernel that
 * ml_step enqueues is bracketed by CUDA events recorded on the launching stream.
 * ml_timing synchronises those events and writes, for the kernel classes
 * {molecules, field pass, plane sampling, plane fold, molecular current, gather},
 * the summed milliseconds into ms[0..5] and the launch counts into counts[0..5],
 * then clears the record.
 * Either output pointer may be NULL. */
ml_status ml_set_timing(ml_grid *g, int enable);
ml_status ml_timing(ml_grid *g, double *ms, int64_t *counts);

/* Number of kernels this grid has launched since creation (all classes). */
int64_t ml_launch_count(const ml_grid *g);

/* Checkpoint the full state (fields, CPML memory, pole currents and polarisations,
 * molecules, DFT accumulators, step count) into host_buf.  With host_buf == NULL only *bytes is
 * set to the size needed.  ml_restore takes a buffer written by ml_checkpoint of a
 * grid created with the same descriptor, molecules and planes. */
ml_status ml_checkpoint(ml_grid *g, void *host_buf, size_t *bytes, void *stream);
ml_status ml_restore(ml_grid *g, const void *host_buf, size_t bytes, void *stream);

/* Discrete adjoint of nsteps coupled steps, for gradients of a transmitted flux
 * (the Sec. IV spectra as objective; the paper does not differentiate its solver).
 * From the grid's present state the call runs nsteps steps (the grid ends exactly
 * as after ml_step(g, nsteps)), with the DFT sums of plane `plane_id` restarted at
 * the first of them, and returns
 *   *objective  = that plane's net flux (as ml_flux) at frequency index `freq`,
 *   grad_eps    = d objective / d eps for each design-box cell, (sz, sy, sx) doubles
 *                 (NULL to skip; requires a design box),
 *   grad_gamma  = d objective / d gamma_m for each molecule, nmol doubles (NULL to skip).
 * Gradient buffers are device memory if on_device, else host memory.  The reverse
 * sweep is the exact transpose of the discrete step (CPML, Drude, PEC walls,
 * periodic axes, molecule gather/step/scatter); the field history is rebuilt from
 * full-state device checkpoints taken every ckpt_every steps, each segment
 * recomputed once (device memory ~ nsteps/ckpt_every checkpoints plus ckpt_every
 * design-box E records).  Molecules of both kinds (the exact two-level step, and the
 * RK4 GKSL step of up to ML_MAX_LEVELS levels with decay, dephasing and substeps, whose
 * stages are walked back) with gamma != 0; every dispersive pole slot, Drude and
 * Lorentz (the polarisation's adjoint is carried beside the current's).  Allocates its work memory for the call and frees it;
 * synchronises `stream`.  With both gradient pointers NULL the call runs only the
 * forward steps and returns the objective (no checkpoints, no reverse sweep). */
ml_status ml_adjoint_run(ml_grid *g, int64_t nsteps, int ckpt_every, int plane_id, int freq, double *objective,
                         double *grad_eps, double *grad_gamma, int on_device, void *stream);

/* Replace the design-box permittivities ((sz, sy, sx) doubles, each > 0) or the
 * couplings gamma_m (nmol doubles) of the molecules; device memory if on_device.
 * Synchronise `stream`; later steps use the new values. */
ml_status ml_set_design_eps(ml_grid *g, const double *eps, int on_device, void *stream);
ml_status ml_set_couplings(ml_grid *g, const double *gamma, int on_device, void *stream);

/* ---- Single-mode cavity (Sec. II, classical photonic dynamics in normal modes) -----
 * The field is one cavity mode per polarisation lambda = x, y (Eq. H_F_normalmode in the
 * single-mode limit, mode function e_lambda / sqrt(V)); molecules couple to it through
 * their mean dipoles.  Per step of length dt (the grid coupling's reading):
 *   E~_m = -gamma_m sum_lambda [eps q_lambda + (eps^2 / omega_c^2) d_lambda] e_lambda
 *          (Eq. E_normalmode, held over the step, built from q^n and d^n),
 *   rho_m advanced as in ml_step (exact 2x2 or RK4 GKSL),
 *   d_lambda^{n+1} = sum_m gamma_m <mu_lambda>(rho^{n+1})       (Eq. dklambda_def),
 *   q, p by velocity Verlet on q'' = -omega_c^2 q - eps d       (Eq. eom_cavmd_a),
 *   half kicks with d^n and d^{n+1}.
 * eps = omega_c / sqrt(V eps0) (Eq. varepsilon_cavmd) is given directly.  The molecule
 * descriptor is that of ml_add_molecules; positions and widths are ignored.  The sums
 * over molecules run in a fixed order (deterministic), in FP64. */
typedef struct {
    double omega_c;   /* mode frequency (> 0) */
    double coupling;  /* eps of Eq. varepsilon_cavmd */
    double dt;        /* time step (> 0) */
    double q0[2];     /* initial mode coordinates, polarisations x and y */
    double p0[2];     /* initial mode momenta */
    int precision;    /* ML_F32 or ML_F64: the molecules' arithmetic (mode state is FP64) */
} ml_cavity_desc;

typedef struct ml_cavity ml_cavity;

/* Create a cavity with `m` (copied; count >= 1).  d^0 is computed from the initial
 * density matrices in FP64.  Errors: ML_ERR_INVALID_ARG (descriptor, molecule table as
 * for ml_add_molecules), ML_ERR_OOM, ML_ERR_CUDA. */
ml_status ml_cavity_create(const ml_cavity_desc *d, const ml_molecule_desc *m, ml_cavity **out);
ml_status ml_cavity_destroy(ml_cavity *c);

/* Enqueue nsteps steps on `stream` (one launch per step for two-level ensembles, whose
 * last block adds the dipole sum and updates the mode; two for others: the molecules,
 * then the dipole sum and the mode update; runs of 64 steps replay a CUDA graph
 * captured on first use). */
ml_status ml_cavity_step(ml_cavity *c, int64_t nsteps, void *stream);

/* Mode state after the enqueued steps into host `out`:
 * q_x, q_y, p_x, p_y, d_x, d_y.  Synchronises `stream`; ML_ERR_NUMERIC if a molecule's
 * field or dipole rate became non-finite. */
ml_status ml_cavity_mode(ml_cavity *c, double *out, void *stream);

/* Molecular state `what` (ML_MOL_*, layouts as for ml_get_molecules) into host `dst`;
 * synchronises `stream`. */
ml_status ml_cavity_get_molecules(ml_cavity *c, int what, double *dst, void *stream);

/* Steps taken. */
int64_t ml_cavity_step_count(const ml_cavity *c);

/* ---- Laser-driven molecules (Sec. II, analytical solutions: classical path) --------
 * No back-action: every molecule sees the prescribed wave of Eq. E_analytical, a
 * function of z - c t (c = 1) travelling along z:
 *   E~_m(t) = gamma_m E0 pol env(u) cos(omega u + phase),  u = z_m - center - t,
 *   env(u) = cos^2(pi u / (2 half_width)) for |u| < half_width, else 0
 * (a carrier under a pulse envelope of compact support; the paper leaves the waveform
 * open), held over each step from t = n dt as in ml_step; molecules advance as in
 * ml_step.  z_m is the molecule descriptor's z position; widths are ignored. */
typedef struct {
    double amplitude;        /* E0 */
    double omega;            /* carrier frequency (wave number omega / c) */
    double phase;
    double center;           /* the pulse centre's z at t = 0 */
    double half_width;       /* > 0 */
    double polarization[3];  /* pol (not normalised by the library) */
    double dt;               /* > 0 */
    int precision;           /* ML_F32 or ML_F64 */
} ml_drive_desc;

typedef struct ml_drive ml_drive;

/* Create with `m` (copied; count >= 1, positions required).  Errors as for
 * ml_cavity_create. */
ml_status ml_drive_create(const ml_drive_desc *d, const ml_molecule_desc *m, ml_drive **out);
ml_status ml_drive_destroy(ml_drive *d);
/* Enqueue nsteps steps (one launch each; runs of 64 replay a captured graph). */
ml_status ml_drive_step(ml_drive *d, int64_t nsteps, void *stream);
/* Molecular state `what` (ML_MOL_*) into host `dst`; synchronises `stream`;
 * ML_ERR_NUMERIC if a molecule's field or dipole rate became non-finite. */
ml_status ml_drive_get_molecules(ml_drive *d, int what, double *dst, void *stream);
int64_t ml_drive_step_count(const ml_drive *d);

/* ---- Batches of independent grids (many realisations of uneven sizes) ----------
 * A batch advances several grids of the same precision and time step together:
 * each step is one launch per kernel class over every instance's blocks (gather,
 * molecules, current, one persistent field pass, and a DFT fold every 64 steps),
 * and runs of 64 steps are replayed from a CUDA graph captured on first use.
 * Results are identical to stepping each grid with ml_step.  The grids keep their
 * own state and API (fields, flux, absorbed energy, checkpoints); while a batch
 * exists, structural changes to a member (molecules, planes) are picked up at the
 * next ml_batch_step.  Destroying a batch leaves the grids intact. */
typedef struct ml_batch ml_batch;

/* n grids (distinct, same precision and Courant number); *out receives the handle. */
ml_status ml_batch_create(ml_grid *const *grids, int n, ml_batch **out);

/* Enqueue nsteps steps of every grid in the batch on `stream`. */
ml_status ml_batch_step(ml_batch *b, int64_t nsteps, void *stream);

/* Field-pass grid: blocks_per_sm blocks per SM looping over the tiles (1..occupancy),
 * or 0 for one block per tile; use_graph = 0 launches every step directly. */
ml_status ml_batch_set_tuning(ml_batch *b, int blocks_per_sm, int use_graph);

/* Time trial_steps steps for each field-pass grid shape, restore every grid after
 * each trial, keep the fastest.  *blocks_per_sm and *ms (either may be NULL) receive
 * the choice and its time.  Synchronises `stream`. */
ml_status ml_batch_autotune(ml_batch *b, int trial_steps, void *stream, int *blocks_per_sm, double *ms);

/* Kernels (and graph launches) this batch has enqueued. */
int64_t ml_batch_launch_count(const ml_batch *b);

/* Per-kernel timing of a batch (tracing): while enabled, steps run without the graph
 * and every launch is bracketed by CUDA events on the stream; ml_batch_timing writes the
 * summed milliseconds and launch counts per kernel class {molecules, field pass, -, fold,
 * molecular current, -} into ms[0..5] / counts[0..5] (either may be NULL) and clears the
 * record.  The events separate the launches, so traced steps do not overlap kernels as
 * untraced ones do. */
ml_status ml_batch_set_timing(ml_batch *b, int enable);
ml_status ml_batch_timing(ml_batch *b, double *ms, int64_t *counts);

/* Free the batch's own device memory and graph (not the grids).  Synchronises. */
ml_status ml_batch_destroy(ml_batch *b);

/* ---- Allocation-free gather (the paper has no counterpart) --------------------
 *
 * ml_gather_static computes the regularised field of Eq. E_regu_Emi,
 *     out[m][c] = gamma_m * sum over cells of E_c * kappa_m^c,
 * for nmol molecules from an FP32 field that the caller owns, with the same
 * separable, normalised Gaussian weights as a grid's step.  It exists for callers
 * that cannot let a library allocate device memory: programs whose GPU memory is
 * reserved up front by their own allocator or a fixed budget, and loops where a
 * cudaMalloc, which may synchronise the device, is not acceptable.  It needs no
 * grid handle and allocates nothing; its only scratch is a fixed device array in
 * the library, ML_STATIC_GATHER_MAX_MOLECULES x 16 planes x 3 floats (3 MiB),
 * present on every GPU the library is loaded on, and nothing in it has to start
 * at zero (each call writes every scratch element it reads).
 *
 * Arguments (all device memory unless said otherwise):
 *   E          3 components Ex, Ey, Ez, each nz*ny*nx floats, (nz, ny, nx) row-major:
 *              the layout ml_get_fields writes for mask ML_EX|ML_EY|ML_EZ.
 *   nx,ny,nz   grid dimensions (>= 1).
 *   periodic   HOST int[3]; nonzero = periodic axis (indices wrap), else cells
 *              outside the grid are left out of the sum.
 *   nmol       0..ML_STATIC_GATHER_MAX_MOLECULES; larger counts are rejected with
 *              ML_ERR_INVALID_ARG before anything is enqueued.
 *   pos        (nmol, 3) doubles, centre in cell units; sigma, gamma: nmol doubles.
 *              A molecule with sigma outside (0, 7/3] or |pos| >= 1e9 gets NaN.
 *   out        (nmol, 3) floats, written by the call.
 *   stream     cudaStream_t as void*; the call enqueues two kernels and returns.
 * The caller keeps ownership of every buffer and must keep them alive until the
 * stream reaches the call.
 *
 * The first call on each device does a one-time set-up (it looks up the device
 * address of the scratch array with the device current); make that first call
 * before any stream capture.  The looked-up address is kept for the life of the
 * process, so do not call the entry point after cudaDeviceReset on that device.  The
 * stream must belong to the current device (else ML_ERR_INVALID_ARG).  All calls on a device share the one scratch array,
 * so calls that overlap on the GPU (on different streams, or from several host
 * threads) race and give wrong results: order them on one stream or synchronise
 * between them. */
#define ML_STATIC_GATHER_MAX_MOLECULES 16384
ml_status ml_gather_static(const float *E, int nx, int ny, int nz, const int *periodic, int nmol,
                           const double *pos, const double *sigma, const double *gamma, float *out,
                           void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MAXLINK_H */
