/*
 * libmm -- stray field between two magnets at a continuous relative
 * displacement, their own demagnetising fields, and the LLG / slider step that
 * consumes them, on one NVIDIA GB300 (sm_103a).
 *
 * Method: I. Rissanen and L. Laurson, "Moving magnets in a micromagnetic
 * finite difference framework", arXiv:1801.04181.
 *
 * Conventions for every call
 *  - Units are SI.  Magnetisation arrays are unit vectors m = M / Ms, float32,
 *    structure of arrays [3][nz][ny][nx] (x fastest), N = nx ny nz cells.
 *  - Magnet 0 is the base, magnet 1 the slider (Sec. III).  The slider is
 *    displaced from its lattice place by the vector u (metres); cell i of
 *    magnet g has its centre at (offset_g + i) * cell (+ u for the slider).
 *  - Pointers named *_dev are CUDA device pointers, *_host host pointers.  The
 *    caller owns every pointer it passes; the library copies in and writes
 *    out and never keeps or frees caller memory.  The library owns its own
 *    buffers, allocated when the geometry is planned (first compute after
 *    mm_set_grid / mm_set_displacement), never per call.
 *  - Work is enqueued on the stream given in mm_options (NULL = legacy default
 *    stream).  Calls returning host values (forces, step results, state)
 *    synchronise that stream.
 *  - Errors are returned as mm_status, never by aborting; mm_last_error()
 *    gives a message.  Device-side range errors (displacement beyond the
 *    planned box during a step) surface as MM_ERANGE from the call that
 *    synchronises.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_ctx mm_ctx;

typedef enum {
  MM_OK = 0,
  MM_EINVAL = -1,   /* bad argument or call order */
  MM_ENOMEM = -2,   /* device allocation failed */
  MM_ECUDA = -3,    /* CUDA runtime error (message in mm_last_error) */
  MM_ERANGE = -4,   /* displacement left the planned potential box */
  MM_ETIMEOUT = -5, /* an iteration did not converge, or a wait on the tensor core ran out, within its bound */
  MM_ESTATE = -6,   /* state buffer of the wrong size or version */
  MM_ENOTSUP = -7,  /* geometry or option the library does not support */
  MM_ETOOBIG = -8   /* larger than the fixed scratch of mm_spline_field_noalloc */
} mm_status;

/*
 * Precision of the field passes.  MM_FP32: every pass in FP32.  MM_MIXED: the
 * reduced-precision form -- the y transforms of the convolutions (Sec. III.A)
 * become complex DFT-matrix products on the tensor cores, with BF16 operands
 * split into hi + lo parts (hi.hi + hi.lo + lo.hi, FP32 accumulation; about
 * 2^-16 relative per dot product) and the y prefilter of the B-spline folded
 * into the inverse DFT matrix; the x transforms, the z plane mixing, the
 * gather and the LLG stage stay FP32.  Every source then takes the separate
 * y-forward / plane-mixing / y-inverse passes; sources of more than 8 layers
 * (z by FFT) return MM_ENOTSUP.  Fields agree with FP32 to ~1e-5 relative L2.
 */
enum { MM_FP32 = 0, MM_MIXED = 1 };

enum { MM_PERIODIC_X = 1, MM_PERIODIC_Y = 2 };

enum { MM_RK45 = 0, MM_EULER = 1 };

typedef struct {
  int precision;     /* MM_FP32 or MM_MIXED */
  int margin;        /* potential box margin in cells beyond the spline support (Sec. III.A: 4) */
  int adaptive;      /* 1: Dormand-Prince 5(4) step-size control; 0: fixed dt */
  double rtol;       /* adaptive: accepted max-norm error of m per step */
  double dt_min, dt_max;
  void* stream;      /* cudaStream_t */
  /*
   * Periodic in-plane boundaries (Sec. III: the extension supports periodic
   * boundary conditions; Sec. IV.B runs the friction films periodic in the
   * film plane): MM_PERIODIC_X | MM_PERIODIC_Y, 0 = open.  Along a periodic
   * axis both magnets must span one period (equal nx, resp. ny; even, and of
   * the form 2^a 3^b 5^c); the kernels are summed over (2 pbc_images + 1)
   * periodic images per periodic axis (the Nyquist offset of the period
   * averaged over its two truncations), the convolutions are circular over
   * the period, the potential covers the whole period with a periodic cubic
   * B-spline (Sec. III.A: its margin values are the other side's), the
   * interpolation and the exchange field wrap around.  z stays open.  Not with
   * sources of more than 8 layers, the energy gradients or the comparison
   * variants (MM_ENOTSUP).
   */
  int periodic;
  int pbc_images;    /* images on each side of the period, 0 .. 64 */
  /*
   * Time integrator of the LLG and the slider's Newton equation (Sec. III:
   * the equations of motion are solved in the Euler solver and in the
   * adaptive Dormand-Prince RK45 solver).  MM_RK45 (default): Dormand-Prince
   * 5(4) with first-same-as-last reuse, adaptive or fixed dt.  MM_EULER:
   * explicit Euler, y + dt f(t, y) with one field evaluation per step and m
   * renormalised, fixed dt only (adaptive = 1 gives MM_EINVAL); no eddy
   * coupling (mm_set_conductivity with sigma > 0 gives MM_ENOTSUP).
   */
  int integrator;
} mm_options;

/* Defaults: FP32, margin 4, adaptive, rtol 1e-5, dt in [1e-16, 1e-11] s, default stream,
 * open boundaries (periodic 0, pbc_images 2). */
void mm_default_options(mm_options* opt);

/* Context.  Does not allocate device memory until a grid is planned. */
mm_status mm_create(mm_ctx** out, const mm_options* opt);
void mm_destroy(mm_ctx* ctx);
const char* mm_last_error(const mm_ctx* ctx);
const char* mm_status_string(mm_status s);

/*
 * Grid of magnet `mag` (0 base, 1 slider): nx x ny x nz cuboid cells of size
 * dx x dy x dz metres (Sec. II: uniform M per cell at its centre) with lattice
 * offset `offset_cells` (x, y, z).  Both magnets must use the same cell size.
 * Every source of up to 8 layers takes z by a direct sum over planes: inside
 * the fused y pass when both magnets have at most 4 layers (thin films), else
 * in a pass of its own between a y-forward and a y-inverse pass.  Sources of
 * more than 8 layers take z by FFT (Sec. III.A on a three-dimensional grid).  Grids whose FFT lines do
 * not fit one shared-memory pass return MM_ENOTSUP when planned, and so do
 * magnets of more than 2^30 cells (here).
 */
mm_status mm_set_grid(mm_ctx* ctx, int mag, int nx, int ny, int nz, double dx, double dy, double dz,
                      const long long offset_cells[3]);

/* Material of magnet `mag` (Sec. II): saturation magnetisation Ms (A/m),
 * exchange constant Aex (J/m), uniaxial anisotropy Ku (J/m^3) along ku_axis,
 * Gilbert damping alpha. */
mm_status mm_set_material(mm_ctx* ctx, int mag, double Ms, double Aex, double Ku,
                          const double ku_axis[3], double alpha);

/* Uniform Zeeman field (A/m) acting on both magnets. */
mm_status mm_set_external_field(mm_ctx* ctx, const double H[3]);

/*
 * Spring drive of the slider (Sec. IV.B):  m x'' = k (v_d t + x0 - x) - gamma_v m x' + F_m . e,
 * F_m the Eq. (EQForce) force of the base on the slider, x the slider position
 * along the unit direction e (drive_dir, normalised here).  mass <= 0 keeps
 * the slider fixed.
 */
mm_status mm_set_mechanics(mm_ctx* ctx, double mass, double k_spring, double v_drive,
                           double gamma_visc, const double drive_dir[3], double x0_spring);

/* Copy m of magnet `mag` in / out (3 N floats).  _dev: device pointer;
 * _host: host pointer (pinned memory recommended; the copy is asynchronous on
 * the context stream for upload, synchronous for download). */
mm_status mm_set_magnetization(mm_ctx* ctx, int mag, const float* m_dev);
mm_status mm_get_magnetization(mm_ctx* ctx, int mag, float* m_dev);
mm_status mm_upload_magnetization(mm_ctx* ctx, int mag, const float* m_host);
mm_status mm_download_magnetization(mm_ctx* ctx, int mag, float* m_host);

/*
 * Slider displacement u (metres, 3-vector) relative to its lattice place
 * (Fig. 3: the partial movement x_p is its sub-cell part).  Resets the slider
 * coordinate x along the drive direction to 0 and re-plans the potential boxes
 * when the whole-cell part of u changes.
 */
mm_status mm_set_displacement(mm_ctx* ctx, const double u_m[3]);

/* Slider mechanical state: position x (m) along the drive direction (added to
 * the displacement), velocity v (m/s) and time t (s). */
mm_status mm_set_slider_state(mm_ctx* ctx, double x, double v, double t);
mm_status mm_get_slider_state(mm_ctx* ctx, double* x, double* v, double* t);

/*
 * Scalar potential phi = sum_j S(r_i - r_j) . M_j of source `src` on the box
 * around the other magnet (Sec. III.A, cell-centred S, four-cell margin).
 * prefiltered = 0: phi (A); 1: its cubic B-spline coefficients (mirror ends).
 * out_dev receives dims[0]*dims[1]*dims[2] floats, x fastest; `capacity` is its
 * size in floats (MM_EINVAL if too small; call with out_dev = NULL to query
 * dims and lo).  lo: box origin in source lattice nodes.
 */
mm_status mm_compute_potential(mm_ctx* ctx, int src, int prefiltered, float* out_dev,
                               size_t capacity, int dims[3], long long lo[3]);

/*
 * Stray field H = -grad phi_src (A/m) at the displaced cell centres of the
 * other magnet (Sec. II.A, tricubic B-spline, 64 coefficients per centre), and
 * the Eq. (EQForce) force / interaction energy on that magnet (mm_get_force).
 * H_dev: 3 N_target floats, may be NULL.
 */
mm_status mm_compute_stray_field(mm_ctx* ctx, int src, float* H_dev);

/* Own demagnetising field of `mag`, H = -sum_j N(r_i - r_j) M_j (A/m), 3 N floats. */
mm_status mm_compute_demag(mm_ctx* ctx, int mag, float* H_dev);

/* Whole field evaluation at the current m and u: both demag fields, both
 * stray fields, both forces. */
mm_status mm_compute_fields(mm_ctx* ctx);

/* Force (N) on magnet `on_mag` from the other one's stray field, Eq. (EQForce),
 * and the interaction energy (J) of that magnet in it, from the latest field
 * evaluation.  FP64.  Synchronises. */
mm_status mm_get_force(mm_ctx* ctx, int on_mag, double F_out[3], double* E_int_out);

/*
 * Gradients of the interaction energy E of magnet 1 - src in the stray field
 * of `src` (the E that mm_get_force(1 - src) returns; Sec. II.A with
 * Eq. (EQForce): E = mu0 V Ms_t sum_i m_t(i) . grad phi_src(x_i)) at the
 * current m and displacement, computed by the transposed path:
 *   dE_du:          3 doubles, dE/du (J/m) of the slider displacement u
 *                   (exact for the spline interpolant: -F along the slider's
 *                   motion when the target is the slider, +F otherwise);
 *   dE_dm_src_dev:  3 N_src floats (J), dE/dm of the source's unit
 *                   magnetisation, SoA like m: the transposed gradient
 *                   evaluation, B-spline prefilter and potential sum;
 *   dE_dm_tgt_dev:  3 N_tgt floats (J), dE/dm of the target's unit
 *                   magnetisation (mu0 V Ms_t grad phi at its cells).
 * Any output may be NULL.  Device pointers, caller-owned.  Also refreshes the
 * target's stray field and force.  Synchronises.
 */
mm_status mm_backward_energy(mm_ctx* ctx, int src, double dE_du[3], float* dE_dm_src_dev,
                             float* dE_dm_tgt_dev);

/* dm/dt (1/s) of the LLG equation (Sec. II eq. 1, Landau-Lifshitz form) at the
 * current state, and the effective field (A/m); either pointer may be NULL. */
mm_status mm_compute_torque(mm_ctx* ctx, int mag, float* dmdt_dev, float* Heff_dev);

/*
 * Advance magnetisation and slider by `nsteps` accepted Dormand-Prince 5(4)
 * steps (Sec. III).  *dt_inout: step size to try (s), returns the next one.
 * t_out: simulated time after the steps (may be NULL).  Synchronises once per
 * step attempt to read the error norm.
 */
mm_status mm_step(mm_ctx* ctx, int nsteps, double* t_out, double* dt_inout);

/*
 * Many independent pairs (one context each) advanced together: every context
 * takes `nsteps` accepted Dormand-Prince steps exactly as mm_step would take
 * them on its own (the same launches in the same order on its own stream, so
 * each pair's result is bit-identical to mm_step's), with its own adaptive dt.
 * Every pair's first attempt is queued before the first wait, and a pair's next
 * attempt is queued as soon as its previous one is concluded, so while the host
 * waits on one pair the streams of the others keep the GPU busy; contexts
 * created on different streams run concurrently.  The paper steps one pair;
 * batching many pairs is this library's addition.
 *   ctxs: npairs distinct contexts; dt_inout: npairs step sizes (s) to try,
 *   returning the next ones; t_out: npairs simulated times after the steps
 *   (may be NULL); failed_pair: index of the pair whose error is returned
 *   (-1 on success; may be NULL), its text in mm_last_error of that context.
 * On an error the other pairs may hold an unconcluded attempt, which the next
 * mm_step / mm_step_batch discards like a rejected one.  MM_EINVAL for a NULL
 * or repeated context or a non-positive dt.
 */
mm_status mm_step_batch(mm_ctx* const* ctxs, int npairs, int nsteps, double* t_out, double* dt_inout,
                        int* failed_pair);

/*
 * Host-only helper for batches: spread npairs pairs of the given costs (any
 * non-negative unit, e.g. modelled bytes per field evaluation) over nlanes
 * streams, longest processing time first (pairs by decreasing cost, ties by
 * index, each to the least loaded lane, ties by lane index).  lane_out: npairs
 * lane indices in [0, nlanes).  MM_EINVAL for nlanes < 1 or a negative or
 * non-finite cost.  Needs no GPU.
 */
mm_status mm_assign_lanes(const double* cost, int npairs, int nlanes, int* lane_out);

/*
 * Host-only query of the shared-memory FFT planner's model choice: the radix
 * of each stage (first stage first; at most 8) for transforms of length L
 * (mm_get_tuned_plan gives the autotuned one, which takes precedence).  Fewest
 * stages of radices up to 16; among their orderings, the near-fewest modelled
 * shared-memory bank conflicts, then the radix set {4, 9, 15, 16} the pass
 * kernels are also compiled for, then the largest last and first radix.
 * MM_EINVAL unless L = 2^a 3^b 5^c >= 1; MM_ENOTSUP for plans with too many
 * stages.  Needs no GPU.
 */
mm_status mm_fft_plan(int L, int radices[8], int* nstages);

/*
 * Autotuner of the FFT plans (the batched form's schedule choice; the paper
 * has no counterpart).  For every transform length this context's pass
 * kernels use, times up to `candidates` radix orderings (the planner's model
 * choice first, then the next orderings by modelled shared-memory
 * wavefronts) on the context's own data, `reps` field evaluations each with
 * CUDA events around the passes that use the length, and keeps the fastest
 * for the whole process: contexts created later, and this one, build their
 * tables of that length from it; a length tuned before is reused, not timed
 * again.  Leaves m, the slider and the timing record as they were (the
 * fields of the last evaluation stay in the buffers).  *n_tuned (may be NULL):
 * lengths timed.  Synchronises.  MM_EINVAL for candidates outside 1..16 or
 * reps < 1.
 */
mm_status mm_autotune(mm_ctx* ctx, int candidates, int reps, int* n_tuned);

/* The radix order mm_autotune chose for length L (first stage first), host
 * only; MM_ESTATE if L has not been tuned in this process. */
mm_status mm_get_tuned_plan(int L, int radices[8], int* nstages);

/*
 * Power bookkeeping at the current state (Sec. III, after Eq. (EQForce)), W:
 *   P_in      = -F_m^s . v_s, the power the moving slider pumps into the
 *               magnets (F_m^s the force of the base on the slider, v_s = v e
 *               its velocity along the drive direction; 0 for a fixed slider);
 *   P_diss[g] = gamma0 alpha mu0 V / ((1 + alpha^2) Ms) sum_i |M_i x H_eff,i|^2,
 *               the Gilbert relaxation of magnet g (gamma0 = mu0 1.7595e11, the
 *               LLG prefactor of Sec. II eq. 1, whose H is in A/m);
 *   P_visc    = gamma_v mass v^2, the viscous damping of the drive.
 * In the steady state P_in balances P_diss[0] + P_diss[1] + the drive's share,
 * and <P_diss / v> estimates the friction force.  Evaluates the fields at the
 * current m and displacement (like mm_compute_torque, so the next mm_step
 * recomputes its first stage).  Any output pointer may be NULL.  Synchronises.
 */
mm_status mm_get_power(mm_ctx* ctx, double* P_in, double P_diss[2], double* P_visc);

/*
 * Comparison variant (Sec. III.A mentions a four-point central difference for
 * the gradient): the stray field of `src` at the other magnet's displaced cell
 * centres as H_a = -(-phi(+2) + 8 phi(+1) - 8 phi(-1) + phi(-2)) / (12 d_a),
 * phi the same B-spline interpolant of the potential evaluated at the centres
 * one and two cells away along each axis, instead of its analytic gradient.
 * H_dev: 3 N_target floats (A/m).  Needs a margin of at least 2 (MM_ENOTSUP
 * otherwise).  No force or energy.
 */
mm_status mm_compute_stray_field_fd4(mm_ctx* ctx, int src, float* H_dev);

/*
 * Comparison variant (Sec. II.A: the demagnetising field "can be interpolated
 * in two ways"; this is the direct one, which Sec. IV.A compares with the
 * potential method): the stray field of `src` at the other magnet's displaced
 * cell centres by cubic B-spline interpolation of each component of the field
 * of the tensor method, H_a(n) = -sum_j sum_b N_ab(n - j) M_b(j) (N the
 * cell-averaged demagnetising tensor of the self-demag field), computed on the
 * nodes of the same box as the potential and prefiltered with mirror ends,
 * 64 taps per component.  H_dev: 3 N_target floats (A/m).  No force or
 * energy.  Sources of more than 8 layers (z by FFT): MM_ENOTSUP.
 */
mm_status mm_compute_stray_field_componentwise(mm_ctx* ctx, int src, float* H_dev);

/*
 * Eddy currents of conducting magnet `mag` (Sec. III.B, the method of Torres
 * et al.), from the rate of change of the flux density in its cells,
 * dBdt_dev (3 N floats, T/s, SoA like m; for B = mu0 (H_d + H_ext + M) the
 * caller forms it, e.g. from dm/dt and the demag of dM/dt), and a uniform
 * conductivity sigma (S/m):
 *   1. E_sol(r_i) = -sum_j dB/dt(r_j) x S(r_i - r_j), S the cell-integrated
 *      kernel of the scalar potential (Sec. III.A); the sign of the section's
 *      first formula (Faraday's law), which its second form drops;
 *   2. phi_E: Laplace's equation in the magnet with d phi_E / dn = E_sol . n
 *      on its surface, cell-centred (flux (phi_nb - phi) / d between cells,
 *      E_sol . n of the cell at surface faces, the source's mean removed),
 *      solved by red-black successive over-relaxation in FP64 to a max-norm
 *      residual of 1e-9 of the source (at most 40000 sweeps; MM_ETIMEOUT
 *      otherwise), zero mean;
 *   3. J = sigma (E_sol - grad phi_E), the gradient taking the boundary
 *      condition's ghost values at surface faces;
 *   4. H_eddy(r_i) = sum_j J(r_j) x S(r_i - r_j) (Biot-Savart), A/m.
 * H_dev, J_dev: 3 N floats each (A/m, A/m^2), either may be NULL; sweeps_out:
 * the SOR sweeps taken (may be NULL).  Device pointers, caller-owned.
 * Synchronises.  MM_ENOTSUP under periodic boundaries.
 */
mm_status mm_eddy_field(mm_ctx* ctx, int mag, const float* dBdt_dev, double sigma, float* H_dev, float* J_dev,
                        int* sweeps_out);

/*
 * Conductivity sigma (S/m) of magnet `mag`; sigma > 0 couples its eddy field
 * into the time step (Sec. III.B: the eddy field joins the effective field).
 * Reading of the coupling (the paper gives the field computation, not its
 * place in the step): explicit and lagged by one accepted step.  After each
 * accepted step, B = mu0 (H_demag + H_stray + H_ext + Ms y5) of the step's
 * last field evaluation (the first-same-as-last stage at the 5th-order
 * solution y5); with the B of the previous step, dB/dt = (B - B_prev) / dt,
 * and the eddy field of mm_eddy_field's steps 1-4 is added to H_eff in every
 * stage of the next step.  Setting m, the displacement, the slider state, the
 * external field, a material or the checkpoint state restarts the lag (no
 * eddy field until two steps have passed).  The currents of a conducting
 * magnet also act on the other magnet: their field there
 * (mm_eddy_field_on_other, at the accepted displacement) is added to that
 * magnet's H_eff in the same way, whether or not it conducts.  sigma = 0
 * (default) turns it off.  Each accepted step then runs the SOR of step 2
 * (synchronising).  Not under periodic boundaries (MM_ENOTSUP).
 */
mm_status mm_set_conductivity(mm_ctx* ctx, int mag, double sigma);

/* The eddy field the next step's stages add for magnet `mag` (3 N floats,
 * A/m, device pointer): its own and that of the other magnet's currents;
 * zeros while there is none. */
mm_status mm_get_eddy_field(mm_ctx* ctx, int mag, float* H_dev);

/*
 * The field of currents J of magnet `mag` inside the other magnet, at its
 * displaced cell centres (Sec. III.B's H_eddy = sum_j J(r_j) x S(r - r_j);
 * Sec. II: not being the gradient of a potential, the eddy field is
 * interpolated inside the moving magnet as field vectors).  On the nodes of
 * the potential box around the other magnet (Sec. III.A's box, margin from
 * mm_options) each component is a potential sum with the rearranged input
 * (0, -J_z, J_y), (J_z, 0, -J_x), (-J_y, J_x, 0), then prefiltered and
 * evaluated by the cubic B-spline at the displaced centres.  J_dev: 3 N
 * floats of magnet `mag` (A/m^2, [3][nz][ny][nx]); H_dev: 3 N_t floats of
 * the other magnet (A/m).  Device pointers, caller-owned; runs on the
 * context's stream.  MM_ENOTSUP under periodic boundaries.
 */
mm_status mm_eddy_field_on_other(mm_ctx* ctx, int mag, const float* J_dev, float* H_dev);

/*
 * Divergence and curl diagnostics of a field (Sec. IV.A): for H_dev (3 N
 * floats, [3][nz][ny][nx], A/m, device) on cells dx x dy x dz,
 *   D = (1/N') sum |div H|,  C = (1/N') sum ||curl H||   (A/m^2)
 * with two-point central differences (H(i+1) - H(i-1)) / (2 d) over the N'
 * cells that have both neighbours along every axis of at least three cells;
 * an axis of fewer than three cells contributes no derivative.  FP32
 * differences, FP64 sums in a fixed order.  Runs on the context's stream with
 * its scratch; synchronises.
 */
mm_status mm_field_div_curl(mm_ctx* ctx, const float* H_dev, int nx, int ny, int nz, double dx, double dy,
                            double dz, double* D, double* C);

/* Accepted / rejected step counters since creation. */
mm_status mm_get_step_stats(mm_ctx* ctx, long long* accepted, long long* rejected);

/*
 * Record of the most recent step attempts of mm_step / mm_step_batch (the
 * context keeps the last 4096), oldest first: for each attempt its start time
 * t (s), its size dt (s), its error norm err (the max over both magnets' cells
 * and components of |dt sum_j (b5_j - b4_j) k_j|, the Dormand-Prince local
 * error estimate of Sec. III's modified RK45, computed in fixed-dt mode
 * too) and whether it was accepted
 * (err <= rtol, or dt <= dt_min, or fixed-dt mode).  Writes the last
 * min(capacity, kept) attempts to the arrays that are not NULL (host
 * pointers, capacity entries each) and their number to *n_out.  Host only.
 * mm_clear_attempt_log forgets the record.
 */
mm_status mm_get_attempt_log(mm_ctx* ctx, int capacity, double* t_out, double* dt_out, double* err_out,
                             int* accepted_out, int* n_out);
mm_status mm_clear_attempt_log(mm_ctx* ctx);

/* Checkpoint: m of both magnets, slider state, displacement and time.
 * mm_get_state with buf = NULL returns the size in *bytes. */
mm_status mm_get_state(mm_ctx* ctx, void* buf, size_t* bytes);
mm_status mm_set_state(mm_ctx* ctx, const void* buf, size_t bytes);

/*
 * Kernel values for tests: kind 0 -> S (3 values per offset, metres), kind 1
 * -> N (6 values: xx yy zz xy xz yz), at n target-minus-source offsets
 * (offsets_dev: 3n doubles, metres), evaluated in FP64 on the device by the
 * same code that builds the spectra.  out_dev: 3n or 6n doubles.
 */
mm_status mm_eval_kernel_fp64(int kind, int n, const double* offsets_dev, double dx, double dy,
                              double dz, double* out_dev);

/* FFT grid and potential box of the path from `src` (for reporting).
 * fft_dims: Qx, Qy and Qz (0 when z is summed directly: sources of up to 8 layers). */
mm_status mm_get_plan_info(mm_ctx* ctx, int src, int fft_dims[3], int box_dims[3],
                           long long box_lo[3], int coef_dims[3]);

/* Per-kernel timing with CUDA events on the context stream (off by default).
 * Classes: 0 x-forward FFT, 1 y pass, 2 x-inverse FFT, 3 gather, 4 LLG stage,
 * 5 slider/reduction, 6 combine/normalise; sources of more than 4 layers:
 * 7 y forward, 8 z pass (z FFT or direct z sum), 9 y inverse. */
mm_status mm_set_timing(mm_ctx* ctx, int on);
mm_status mm_get_timing(mm_ctx* ctx, int kernel_class, double* total_ms, long long* launches);
mm_status mm_reset_timing(mm_ctx* ctx);

/* Number of kernel launches this context has issued (all classes). */
long long mm_launch_count(const mm_ctx* ctx);

/*
 * Stray field, force and interaction energy from a caller-held coefficient
 * box, with no device memory allocated by the call.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate while
 * they drive the library -- an application whose device memory is owned by its
 * own pool allocator and forbids raw cudaMalloc, or a stepping loop that
 * cannot afford the device synchronisation of cudaMalloc / cudaFree.
 *
 * Inputs (all caller-owned): coef_dev, B-spline coefficients of a source
 * potential on a box, dims (x, y, z) floats x fastest, whose node [0][0][0]
 * is source lattice node coef_lo (e.g. mm_compute_potential with
 * prefiltered = 1); pos0_nodes, position of target cell (0,0,0) in source
 * lattice nodes (target offset - source offset +- slider displacement, in
 * cells); m_dev, unit magnetisation of the nx x ny x nz target (nz <= 4); cell
 * size dx, dy, dz (m); Ms of the target (A/m).
 * Outputs (caller-owned device memory): H_dev, 3 N floats of H = -grad phi
 * (A/m), may be NULL; FE_dev, 4 doubles: Eq. (EQForce) force F (N) on the
 * target and its interaction energy E (J).  Asynchronous on `stream`
 * (cudaStream_t, NULL = default stream).
 *
 * Scratch: a fixed 2 MiB array inside the library (resident on every GPU that
 * loads it until exit), good for targets of up to 65536 tiles of 32 x 8 cell
 * columns; larger targets return MM_ETOOBIG.  A target whose spline support
 * leaves the box returns MM_ERANGE.  The first call on each device looks up the
 * array's address; make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race and must be serialised.
 */
mm_status mm_spline_field_noalloc(const float* coef_dev, const int coef_dims[3],
                                  const long long coef_lo[3], const double pos0_nodes[3],
                                  const float* m_dev, int nx, int ny, int nz, double dx, double dy,
                                  double dz, double Ms, float* H_dev, double* FE_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
