/*
 * airebo.h -- C ABI of the GB300 AIREBO energy/force library (libairebo.so).
 *
 * The library evaluates the AIREBO potential of Hoehnerbach & Bientinesi,
 * "Optimizing AIREBO" (Sec. 2.1): the REBO term E = f_R + b_ij f_A with the
 * bond order b_ij (Alg. 1, Sec. 2.1.3), the torsion term (Alg. 2) and the
 * bond-order- and connectivity-switched Lennard-Jones term (Alg. 3,
 * Sec. 2.1.2), on one GPU.  The problem statement follows Sec. 2: positions
 * in, forces F_i = -grad_i V out; a long neighbour list with a skin, rebuilt
 * only when an atom has moved more than half the skin; a short REBO list
 * rebuilt every step from an intermediate list (Sec. 4.1).
 *
 * Conventions shared by every call:
 *  - Units: Angstrom, eV, eV/Angstrom, fs, amu ("metal" units).
 *  - Atom arrays are structure-of-arrays: x[3][n] (all x, then all y, then
 *    all z), double.  Types are int8: 0 = carbon, 1 = hydrogen.
 *  - The box is orthorhombic and periodic in all three directions; each edge
 *    must exceed 4 x the largest REBO cut-off (8 A with the usual values), so
 *    that a path of three bonds never meets two images of one atom.
 *    Positions may lie outside the box; at a neighbour build they must lie
 *    within 127 box lengths of it.
 *  - Forces are -dE/dx.  The virial is W_ab = -sum_terms sum_atoms
 *    x_a * dE/dx_b with positions unwrapped within each term, i.e.
 *    W = -dE/d(strain); order xx, yy, zz, xy, xz, yz.
 *  - Energies are reported as four doubles: total, REBO, LJ, torsion.
 *  - Device pointers ("d_") are owned by the caller, must stay valid for the
 *    duration of the call, and are used on the handle's stream.  Host
 *    pointers ("h_") are plain host memory.  The library owns its lists and
 *    scratch buffers and frees them in airebo_destroy.
 *  - Every call returns an airebo_status and never aborts the process;
 *    airebo_last_error() gives a text for the last failure on a handle.
 *  - Calls that return results to the host synchronise the handle's stream.
 */
#ifndef AIREBO_H
#define AIREBO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct airebo_ctx* airebo_handle;

typedef enum {
    AIREBO_OK = 0,
    AIREBO_ERR_ARG = 1,        /* bad argument: null pointer, size, box too small, bad parameter text */
    AIREBO_ERR_CUDA = 2,       /* a CUDA runtime call failed (text in airebo_last_error) */
    AIREBO_ERR_CAPACITY = 3,   /* more than 16 REBO neighbours on an atom (twice the bound of Sec. 4.3) */
    AIREBO_ERR_TIMEOUT = 4,    /* reserved: a bounded device-side wait gave up */
    AIREBO_ERR_NONFINITE = 5,  /* a position is NaN or infinite, or two atoms closer than 1e-6 A */
    AIREBO_ERR_STATE = 6       /* call out of order, e.g. compute before neighbor */
} airebo_status;

/*
 * Precisions.  AIREBO_FP64: every term in FP64.  AIREBO_MIXED: FP32 geometry,
 * splines and bond order; FP64 positions, displacements, accumulation and
 * integrator -- except that the Lennard-Jones pairs with C_ij = 1 and no b*
 * take their displacement from the split positions below (exact to about
 * 1e-11 A before its one rounding to FP32) and sum their pair forces in 64-bit
 * fixed point and their energy in double-float, so that they need no FP64
 * instruction.  AIREBO_DF64: as AIREBO_FP64, except that the pair arithmetic
 * of the Lennard-Jones pairs with C_ij = 1 and no b* runs in double-float
 * (pairs of FP32 numbers, about 48 significant bits) on the FP32 pipe, from
 * positions split on a 2^-12 A grid, with the pair forces summed in 64-bit
 * fixed point (2^-40 eV/A), and the torsion term runs in double-float on the
 * FP64 short list -- FP64-class results at FP32-pipe rates.  It
 * needs every |coordinate| below 2000 A and pair forces below 1e6 eV/A
 * (AIREBO_ERR_ARG / AIREBO_ERR_NONFINITE otherwise), as does AIREBO_MIXED;
 * with the Morse form both run their LJ pairs as before the split (FP64
 * displacements and FP64 sums).
 */
enum { AIREBO_FP64 = 0, AIREBO_MIXED = 1, AIREBO_DF64 = 2 };

typedef struct {
    double skin;          /* neighbour-list skin, Angstrom (default 1.0) */
    int precision;        /* AIREBO_FP64, AIREBO_MIXED or AIREBO_DF64 (see above) */
    int enable_rebo;      /* 1: REBO term (Alg. 1) */
    int enable_lj;        /* 1: LJ term (Alg. 3) */
    int enable_torsion;   /* 1: torsion term (Alg. 2) */
    int max_lj_nbrs;      /* initial long-list capacity per atom; 0 = from the density */
    int bstar_screen;     /* AIREBO_FP64 and AIREBO_DF64 (default 1): b* enters the LJ term only
                             through S_b, which is exactly 1 below b_min and 0 above b_max; the
                             first b* pass evaluates b* in FP32 together with a rigorous bound on
                             its distance from the exact value of the same formula (each operation's
                             rounding error and the FP32 roundings of the inputs and parameters,
                             bounded upward), and decides S_b when the whole interval lies outside
                             [b_min, b_max] by more than 1e-9 (room for the FP64 evaluation's own
                             rounding); every other pair is evaluated in FP64.  The decided S_b are
                             the FP64 ones.  0: every b* evaluated in FP64.  Ignored by
                             AIREBO_MIXED. */
} airebo_options;

/* Fill opts with the defaults: skin 1.0 A, FP64, all three terms on, auto capacity, b* screen on. */
void airebo_default_options(airebo_options* opts);

/*
 * Create a handle.  params: the parameter set as text, one entry per line
 * "name count v1 ... vcount" (scalars of f_R, f_A, the switches, LJ and
 * torsion, and the knot data of the g, P, pi^rc and T splines); the handle
 * keeps its own copy.  stream: a cudaStream_t (NULL = default stream) on which
 * every later call enqueues its work.  The current CUDA device at creation is
 * the handle's device.  Returns AIREBO_ERR_ARG for unparsable or incomplete
 * text.
 */
airebo_status airebo_create(const char* params, const airebo_options* opts, void* stream, airebo_handle* out);

/* Free every buffer of the handle.  NULL is accepted. */
void airebo_destroy(airebo_handle h);

/* Text of the last error on the handle ("" if none). */
const char* airebo_last_error(airebo_handle h);

/*
 * Build the neighbour lists (Sec. 2, Sec. 4.1): bin atoms into cells, then a
 * half list of pairs with r < 3 sigma_ij + skin for the LJ term and a full
 * intermediate list with r < Dmax_ij + skin for the REBO term, with explicit
 * periodic images.  d_pos: device double[3][n]; d_types: device int8[n]
 * (copied); box: host double[3].  Grows its capacities as needed (one stream
 * synchronisation).  n may be 0 and must stay below 2^28 (268,435,456).
 */
airebo_status airebo_neighbor(airebo_handle h, const double* d_pos, const int8_t* d_types, int64_t n,
                              const double* box);

/*
 * Energy and forces at d_pos (Sec. 2: positions in, F_i = -grad_i V out, with
 * the energy of Sec. 2.1; same atoms as the last airebo_neighbor; the lists
 * stay valid while no atom has moved more than skin/2 since it).
 * d_force: device double[3][n], overwritten.  d_energy4 (device double[4]),
 * d_virial6 (device double[6]) and d_energy_per_atom (device double[n]) may
 * be NULL; the virial is only computed when d_virial6 is given.  Per-atom
 * energies split every term evenly between the two atoms that define it: a
 * REBO bond i-j (Alg. 1) and a torsion term around the bond i-j (Alg. 2)
 * give half to i and half to j, an LJ pair i-j (Alg. 3, b* included) half to
 * each, so they do not depend on the atom numbering and sum to the total.
 * Synchronises the stream once to check capacity flags, and regrows and
 * recomputes when a scratch capacity was exceeded.
 */
airebo_status airebo_compute(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                             double* d_virial6, double* d_energy_per_atom);

/*
 * Same as airebo_compute with host buffers: copies h_pos to the device, runs
 * the neighbour build when needed (first call, new n or box, or an atom moved
 * more than skin/2), computes, and copies forces, energies, virial and
 * per-atom energies (h_energy_per_atom, host double[n], nullable) back.
 * h_types/box are read on the first call and whenever n changes.
 */
airebo_status airebo_compute_host(airebo_handle h, const double* h_pos, const int8_t* h_types, int64_t n,
                                  const double* box, double* h_force, double* h_energy4, double* h_virial6,
                                  double* h_energy_per_atom);

/* *out_flag = 1 if some atom moved more than skin/2 since the last neighbour build. */
airebo_status airebo_needs_rebuild(airebo_handle h, const double* d_pos, int* out_flag);

/*
 * Velocity-Verlet NVE (the MD step of Sec. 2): nsteps steps of dt fs on
 * d_pos/d_vel (device double[3][n], Angstrom, Angstrom/fs, updated in place),
 * d_force holds the forces on return.  Rebuilds the lists when an atom moved
 * more than skin/2 (checked every step).  Masses are 12.011 (C) and 1.008 (H)
 * amu.  On entry d_force must hold the forces at d_pos (from airebo_compute
 * or the previous airebo_nve call).  d_energy4 (nullable, device double[4])
 * receives potential energy total, kinetic energy, their sum, and the number
 * of list builds of the handle so far, after the last step.  The lists must
 * have been built for these atoms.
 */
airebo_status airebo_nve(airebo_handle h, double* d_pos, double* d_vel, double* d_force, double dt, int nsteps,
                         double* d_energy4);

/*
 * The NVE step of airebo_nve with no host synchronisation: every step is
 * enqueued on the handle's stream, and the rebuild decision is taken on the
 * device -- a kernel compares the largest displacement since the last build
 * with skin/2 and gates the kernels of the list build, which then run or
 * return at once.  The cell grid and every capacity are those of the last
 * synchronous airebo_neighbor / airebo_compute (a build may not grow them):
 * an overflow, a non-finite position or a range error is recorded on the
 * device and reported by airebo_check, which the caller must call after the
 * steps (the results of steps after an overflow are not valid).  d_energy4
 * (nullable) as in airebo_nve; its fourth value counts the builds run by the
 * host and by the device.  Errors: AIREBO_ERR_STATE before airebo_neighbor,
 * AIREBO_ERR_ARG for a bad dt or step count.
 */
airebo_status airebo_nve_async(airebo_handle h, double* d_pos, double* d_vel, double* d_force, double dt, int nsteps,
                               double* d_energy4);

/*
 * Capture nsteps steps of airebo_nve_async into the handle's CUDA graph
 * (replacing any graph captured before), after a synchronous evaluation at
 * d_pos that grows every scratch capacity, with headroom for the steps ahead
 * (lists rebuilt at d_pos with a quarter more room per atom, 16 REBO slots
 * per atom, a quarter more connectivity-map entries and b* queue), and writes
 * the forces at d_pos to d_force.  Each airebo_graph_launch then runs nsteps MD steps, rebuilds
 * included, in one launch; call airebo_check after launches.  The handle must
 * have been created on a non-default stream; a synchronous airebo_neighbor
 * (new atoms, box or capacities) needs a new capture.
 */
airebo_status airebo_graph_capture_nve(airebo_handle h, double* d_pos, double* d_vel, double* d_force, double dt,
                                       int nsteps, double* d_energy4);

/* The NVE step with host buffers: copy in, nsteps steps, copy positions,
 * velocities, forces and d_energy4's four values back. */
airebo_status airebo_nve_host(airebo_handle h, double* h_pos, double* h_vel, double* h_force, double dt,
                              int nsteps, double* h_energy4);

/*
 * Counters of the last compute (int64[8]): bonds, b* pairs, b* pairs with a
 * nonzero S_b derivative, LJ pairs within the cut-off evaluated in the pair
 * kernel, connectivity-map capacity, list rebuilds, LJ list capacity, b*
 * pairs evaluated in the full-precision pass (the others were decided by the
 * first pass: exactly in MIXED or with the screen off, by the FP32 screen in
 * FP64).  Synchronises.
 */
airebo_status airebo_counters(airebo_handle h, int64_t* out8);


/*
 * Copy a neighbour list to the host (for checks).  which: 0 = LJ half list
 * (each pair once, in the row of the atom that sorts first by cell at the
 * last build; i==j with a positive image; r < 3 sigma + skin), 1 = REBO
 * intermediate list (r < Dmax + skin, full), 2 = exact REBO list of the last
 * compute (r < Dmax, full, at most 8 per atom).  h_cnt: int32[n];
 * h_j: int32[n * cap]; h_img: int8[n * cap * 3] (image S, x_j + S L - x_i).
 * Entries beyond cap per atom are dropped (*h_cnt still counts them).
 */
airebo_status airebo_export_lists(airebo_handle h, int which, int32_t* h_cnt, int32_t* h_j, int8_t* h_img, int64_t cap);

/*
 * Per-kernel timing with CUDA events recorded on the handle's stream around
 * each launch.  airebo_set_timing(h, 1) starts (and zeroes) the record;
 * airebo_kernel_times fills ms[k] (total milliseconds) and launches[k] for
 * k = 0 FP32 positions and short list, 1 REBO bonds, 2 torsion, 3
 * connectivity map, 4 LJ pairs (the pair kernel, the kernel of the pairs
 * along a path, and the merge of the fixed-point LJ sums in the mixed and DF64
 * paths), 5 b* pairs (first pass), 6 neighbour build, 7 NVE
 * half steps, 8 b* pairs (second pass).  out arrays: 9 entries.
 */
airebo_status airebo_set_timing(airebo_handle h, int on);
airebo_status airebo_kernel_times(airebo_handle h, double* ms, int64_t* launches);

/*
 * Measure the FMA throughput of the current device with a register-resident
 * loop (precision AIREBO_FP64 or AIREBO_MIXED for FP32); *tflops receives
 * the achieved TFLOP/s (an FMA counts 2).  A roofline denominator for the
 * ALU-bound kernels; it runs for a few tens of milliseconds.
 */
airebo_status airebo_alu_peak(int precision, double* tflops);

/*
 * Accuracy check of the FP64 reciprocal and reciprocal square root the
 * kernels use (a hardware approximation refined by one third-order Newton
 * step): h_ulp4 (host int64[4]) receives the largest difference, in units in
 * the last place, from CUDA's correctly rounded 1/x and from 1/sqrt(x) over
 * 4M values of x spread over [2^-30, 2^30) on the current device, then the
 * same for the hardware approximations without the Newton step.  A
 * diagnostic; the paper has no counterpart.
 */
airebo_status airebo_math_check(int64_t* h_ulp4);

/*
 * Accuracy check of the double-float operations of the AIREBO_DF64 torsion
 * kernel on the current device, against FP64 on the same (exactly
 * representable) inputs over 4M seeded operands +-m 2^t (m in [1, 2), t in
 * [-20, 20)): h_err8 (host double[8]) receives the largest error of a + b
 * relative to |a| + |b|; of a * b, a / b, 1/a and 1/sqrt(|a|) relative; of
 * sin(pi t) and cos(pi t) for t in [0, 2) absolute (against CUDA's FP64
 * sincospi); and of the conversion from double, relative.  A diagnostic.
 */
airebo_status airebo_dd_check(double* h_err8);

/*
 * Energy and forces as airebo_compute, plus the gradient of the energy with
 * respect to the parameters of the inter-molecular term (Sec. 2.1.2, the
 * E^LJ of Alg. 3; the spline knot data of the bond order, Sec. 2.1.3, have
 * their own call, airebo_knot_grad):
 * h_grad6 (host double[6]) = dE/d epsilon[CC, CH, HH] (lj.epsilon, or
 * morse.epsilon for the Morse form), dE/d sigma[CC, CH, HH] (lj.sigma, which
 * also sets the switch and cut-off radii).  Slower than airebo_compute: every
 * LJ pair takes the general path.  Synchronises.
 */
airebo_status airebo_param_grad(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                                double* h_grad6);

/*
 * Parameter derivatives of the forces, for force matching: with a direction
 * d_v (device double[3][n]), h_out6 (host double[6]) receives
 * v . dF/d epsilon[CC, CH, HH] and v . dF/d sigma[CC, CH, HH] of the
 * inter-molecular term (Sec. 2.1.2, the E^LJ of Alg. 3; epsilon is lj.epsilon
 * or morse.epsilon), F the forces of airebo_compute -- e.g. v = 2 (F - F_ref)
 * gives the gradient of sum |F - F_ref|^2.  The forces of the pair term are
 * linear in epsilon, and dE/dsigma has the pair term's own form with the
 * sigma-derivatives of its radial factors, so both come from one pass over
 * the pairs (radial part, C_ij path, and the reverse b* in the S_b
 * transition).  Also evaluates forces and energy like airebo_compute
 * (d_energy4 nullable); every LJ pair takes the general path.  Synchronises.
 */
airebo_status airebo_force_param_grad(airebo_handle h, const double* d_pos, const double* d_v, double* d_force,
                                      double* d_energy4, double* h_out6);

/*
 * Replace epsilon[3] (lj.epsilon or morse.epsilon) and/or sigma[3] (lj.sigma)
 * of the inter-molecular term; either pointer may be NULL.  Changing sigma
 * moves the LJ cut-off, so the next call must be airebo_neighbor (compute
 * returns AIREBO_ERR_STATE until then).  Synchronises.
 */
airebo_status airebo_set_lj_params(airebo_handle h, const double* eps3, const double* sigma3);

/*
 * Batched independent systems: nsys periodic boxes evaluated as one set of
 * launches.  d_pos/d_types hold all atoms, system s owning atoms
 * [h_offsets[s], h_offsets[s+1]) (host int64[nsys+1], from 0 to n);
 * h_boxes: host double[3 * nsys], each edge > 4 x the largest REBO cut-off.
 * Builds one cell grid per system; no pair crosses systems.  After it,
 * airebo_compute, airebo_nve and the other calls act on all systems at once.
 */
airebo_status airebo_neighbor_batch(airebo_handle h, const double* d_pos, const int8_t* d_types, int64_t n,
                                    int nsys, const int64_t* h_offsets, const double* h_boxes);

/* Forces (d_force, device double[3][n]) and the potential energy of each
 * system (d_energy_sys, device double[nsys]; one system after
 * airebo_neighbor).  Synchronises like airebo_compute. */
airebo_status airebo_compute_batch(airebo_handle h, const double* d_pos, double* d_force, double* d_energy_sys);

/*
 * Enqueue one evaluation without any host synchronisation or capacity growth
 * (d_energy4, d_energy_sys nullable; per-system energies need one earlier
 * synchronous evaluation that wanted them).  Capacity and error flags are
 * read by airebo_check, which synchronises and returns what airebo_compute
 * would have returned for the same evaluation: AIREBO_ERR_NONFINITE for a
 * non-finite position, overlapping atoms or an LJ pair force beyond the
 * fixed-point range, AIREBO_ERR_ARG for a coordinate beyond 2000 A in
 * AIREBO_MIXED / AIREBO_DF64 (each found condition is named in
 * airebo_last_error), else AIREBO_ERR_CAPACITY if a scratch capacity was
 * exceeded (run airebo_compute once, then retry).
 */
airebo_status airebo_compute_async(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                                   double* d_energy_sys);
airebo_status airebo_check(airebo_handle h);

/*
 * Capture one evaluation (as airebo_compute_async, with these pointers) into
 * a CUDA graph on the handle's stream, after a synchronous evaluation that
 * grows every capacity; airebo_graph_launch replays it.  The handle must have
 * been created on a non-default stream.  A neighbour rebuild or a new atom
 * count needs a new capture.
 */
airebo_status airebo_graph_capture(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                                   double* d_energy_sys);
airebo_status airebo_graph_launch(airebo_handle h);

/*
 * Pick the launch shapes for this handle's system by timing them with CUDA
 * events on the handle's stream: the number of atoms an LJ warp claims at a
 * time (2..16), and the grids of the grid-stride REBO/torsion kernels and of
 * the b* kernels, in waves of resident blocks (2, 4, 8, 16 or 32 times the
 * blocks that fit on all SMs at once); each candidate is the median of 5
 * evaluations.  Runs about 50 evaluations at d_pos (d_force is overwritten).
 * Untuned handles start at (2, 16, 16), the shapes tuned on a 1M-atom
 * polyethylene in FP64.
 * out3 (nullable, host int[3]) receives (lj_chunk, bond_waves, bstar_waves).  A
 * graph captured earlier keeps the shapes it was captured with.  Errors:
 * those of airebo_compute; AIREBO_ERR_STATE before airebo_neighbor.
 */
airebo_status airebo_autotune(airebo_handle h, const double* d_pos, double* d_force, int* out3);

/*
 * Set the launch shapes directly (for example to copy a tuned choice to
 * another handle of the same system): lj_chunk in 1..64 atoms per warp claim,
 * bond_waves and bstar_waves in 1..32 waves (defaults 4, 8, 8).
 * AIREBO_ERR_ARG outside those ranges.  Results do not depend on the shapes
 * beyond the order of floating-point atomic additions.
 */
airebo_status airebo_set_launch_shape(airebo_handle h, int lj_chunk, int bond_waves, int bstar_waves);

/*
 * Gradient of the total energy with respect to every spline knot datum of the
 * parameter set (the tabulated data of the angular functions g_C, gamma_C and
 * g_H, of the P_ij bicubic correction and of the pi^rc and T_ij tricubic
 * splines, Sec. 2 (REBO bond order)), for fitting.  Each spline is built from
 * its knot data linearly, so the energy depends on a datum only through the
 * bond orders (b_ij and the b* of the LJ switch) that read it.
 *
 * Also evaluates forces and energy like airebo_compute (d_energy4 nullable).
 * h_grad: host double[AIREBO_KNOT_COUNT] in the parameter file's order and
 * layout: gC1.data (18), gC2.data (18), gH.data (12), P.CC, P.CH, P.HC (100
 * each: 5 x 5 knots x (f, f_NC, f_NH, f_NC_NH)), piRC.CC, piRC.CH, piRC.HH
 * and Tij.CC (1800 each: 5 x 5 x 9 knots x (f, fx, fy, fz, fxy, fxz, fyz,
 * fxyz)).  count must equal AIREBO_KNOT_COUNT.  The gradient is in the
 * handle's precision; the first call allocates a device buffer of about
 * 270 KB that the handle keeps.  Errors: those of airebo_compute;
 * AIREBO_ERR_ARG for a wrong count.
 */
#define AIREBO_KNOT_COUNT 7548
airebo_status airebo_knot_grad(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                               double* h_grad, int64_t count);

/*
 * Check of the b* screen's error bound (handles with bstar_screen = 1, FP64
 * or DF64): one evaluation at d_pos (d_force receives the forces), then, for
 * every pair queued for b* (Alg. 3, Sec. 2.1.3), the FP64 b* against the
 * FP32 b* with its rigorous error bound.  h_out6 (host double[6]): pairs with
 * a finite bound, pairs with an infinite one (sent to the FP64 pass), the
 * largest |b*_32 - b*_64| / bound (at most 1 if the bound holds), the largest
 * bound, the pairs whose difference exceeds their bound, and the largest
 * difference.  A diagnostic.  AIREBO_ERR_STATE when the screen is off.
 */
airebo_status airebo_bstar_bound_check(airebo_handle h, const double* d_pos, double* d_force, double* h_out6);

/*
 * Replace every spline knot datum of the handle's parameter set (the data
 * whose gradient airebo_knot_grad returns, Sec. 2.1.3), in the same order and
 * layout; the knot abscissae and all scalars stay.  The spline coefficients
 * are rebuilt and uploaded; the lists stay valid.  count must equal
 * AIREBO_KNOT_COUNT; AIREBO_ERR_ARG for a wrong count or a non-finite value
 * (the handle then keeps its old data).  Synchronises.
 */
airebo_status airebo_set_knots(airebo_handle h, const double* h_knots, int64_t count);

/*
 * Rebuild check that allocates no device memory (the paper has no
 * counterpart: it is a service for callers that cannot call cudaMalloc, such
 * as code running inside a framework that owns all device memory, or code
 * that must not allocate after its set-up).  Same test as
 * airebo_needs_rebuild -- *h_flag = 1 if max_i |x_i - x_ref,i| > skin/2 --
 * but it needs no handle: d_pos and d_ref are device double[3][n] given by
 * the caller, stream is a cudaStream_t (NULL = default stream); *h_max_disp
 * (nullable) receives max |x - x_ref| in Angstrom.  Synchronises the stream.
 * Its scratch is a fixed 64 KB array inside the library image, held by every
 * GPU that loads the library until exit, so n is limited to 2,097,152 atoms
 * (larger n returns AIREBO_ERR_ARG).  The first call on a device looks up the
 * array's device address (set-up), and looks it up again after the device's
 * context was replaced (cudaDeviceReset); make that first call before any
 * stream capture.  All calls share the array: calls whose kernels overlap on
 * the GPU race and must be serialised by the caller.
 */
airebo_status airebo_needs_rebuild_noalloc(const double* d_pos, const double* d_ref, int64_t n, double skin,
                                           void* stream, int* h_flag, double* h_max_disp);

#ifdef __cplusplus
}
#endif

#endif /* AIREBO_H */
