/*
 * lfe.h -- C-ABI of the B300 alchemical nonbonded engine.
 *
 * The library evaluates, on one GPU, the lambda-dependent potential of the
 * linear-basis-function lambda-dynamics method (Correa, Abreu, Nair,
 * Tuckerman, Section 2.2, Eq. 4):
 *
 *   U(r, lambda) = U_vv + U_uu + h_A(lambda) U_uv + h_B(lambda) U_soft (+ bonded)
 *
 *   U_vv, U_uu  solvent-solvent and solute-solute nonbonded energy (LJ +
 *               Ewald/PME Coulomb), unchanged along lambda;
 *   U_uv        the full solute-solvent LJ + Coulomb interaction, including its
 *               reciprocal-space cross term and neutralising-background share;
 *   U_soft      the capped soft-LJ basis, sum over solute-solvent pairs of
 *               eps_ij u_cap(r_ij / sigma_ij) (Eq. 5-6);
 *   h_A, h_B    the smoothstep switches of Eq. 7-10,
 *
 * together with the forces -grad U and the generalized force
 *   dU/dlambda = h_A'(lambda) U_uv + h_B'(lambda) U_soft       (Section 2.1)
 * that drives the alchemical coordinate.  lfe_step advances atoms with a
 * Langevin middle-scheme integrator (Section 2.6), rigid waters and X-H
 * constraints, and the mirror-periodic coordinate theta (Eq. 3) under the
 * dual OPES bias (Eq. 11-14).
 *
 * Conventions for every call:
 *   - Units: nm, ps, amu, kJ/mol, e, K.  Coulomb constant 138.935458.
 *   - Arrays are row-major doubles: positions and forces are [3 N] (x, y, z of
 *     atom 0, then atom 1, ...), in the caller's atom order.
 *   - The caller owns every array it passes; inputs are copied before the call
 *     returns (or before the stream reaches the copy, for device inputs);
 *     outputs are written into caller memory.  The library never frees caller
 *     memory and keeps no caller pointer.
 *   - `on_device` / `out_on_device` = 1 means the pointer is device memory
 *     usable on `stream` (for example a torch tensor's data_ptr()); 0 means
 *     host memory.  `stream` is a cudaStream_t or NULL for the legacy stream.
 *     Device outputs are complete when `stream` reaches the end of the call's
 *     work; host outputs are complete when the call returns.
 *   - Every call returns LFE_OK (0) or a negative LFE_ERR_* code and records
 *     a message readable with lfe_last_error.  No call aborts the process or
 *     traps the GPU; bounded device waits report LFE_ERR_TIMEOUT.
 */
#ifndef LFE_H
#define LFE_H

#ifdef __cplusplus
extern "C" {
#endif

#define LFE_OK             0
#define LFE_ERR_ARG       -1   /* bad size, r_cut > box/2, non-finite input, sigma < 0 ... */
#define LFE_ERR_CUDA      -2   /* a CUDA runtime call failed */
#define LFE_ERR_OVERFLOW  -3   /* neighbour-list capacity exceeded (after one internal regrowth) */
#define LFE_ERR_NONFINITE -4   /* a force, energy or position became NaN/Inf */
#define LFE_ERR_TIMEOUT   -5   /* a bounded device wait expired */
#define LFE_ERR_STATE     -6   /* call out of order (e.g. step without neighbour list) */

#define LFE_FP32_MIXED 0       /* FP32 pair/PME arithmetic, 64-bit fixed-point accumulation */
#define LFE_FP64       1       /* the same kernels instantiated in double precision */

/* Number of doubles written by lfe_eval into energy_terms. */
#define LFE_NTERMS 10
/* energy_terms layout */
#define LFE_T_U        0   /* U(lambda), kJ/mol (nonbonded + bonded) */
#define LFE_T_DUDL     1   /* dU/dlambda */
#define LFE_T_UVV      2
#define LFE_T_UUU      3
#define LFE_T_UUV      4
#define LFE_T_USOFT    5
#define LFE_T_UBONDED  6
#define LFE_T_NPAIRS   7   /* unordered non-excluded pairs with r < r_cut (counted) */
#define LFE_T_HA       8   /* h_A(lambda) */
#define LFE_T_HB       9   /* h_B(lambda) */

typedef struct lfe_system lfe_system;   /* opaque; owns all of its device memory */
typedef struct lfe_batch lfe_batch;     /* opaque; a set of systems run together */

/* Run parameters.  Fields marked "step" matter only for lfe_step. */
typedef struct {
    double box[3];            /* orthorhombic box, nm; r_cut <= min(box)/2 required */
    double r_cut;             /* nonbonded cutoff, nm */
    double r_switch;          /* LJ switch start, nm; < 0: plain truncation */
    double ewald_alpha;       /* Ewald splitting parameter, nm^-1 */
    int pme_grid[3];          /* PME grid; each a product of 2, 3 and 5, 8..128 */
    int pme_order;            /* B-spline order; must be 4 */
    double skin;              /* neighbour-list buffer, nm: > 0 fixed; <= 0 0.1 until
                                 lfe_autotune chooses it */
    int precision;            /* LFE_FP32_MIXED or LFE_FP64 */
    double temperature;       /* step: K */
    double friction;          /* step: atoms' Langevin friction, 1/ps */
    double dt;                /* step: time step, ps */
    double lambda_mass;       /* step: theta mass, amu nm^2 (<= 0: theta frozen) */
    double lambda_friction;   /* step: theta Langevin friction, 1/ps */
    double theta0;            /* step: initial theta in [0, 2) */
    int opes_stride;          /* step: steps between kernel deposits (0: no OPES) */
    double opes_dE_std;       /* step: OPES-Standard barrier, kJ/mol (0 disables) */
    double opes_dE_exp;       /* step: OPES-Explore barrier, kJ/mol (0 disables) */
    double opes_sigma;        /* step: kernel width on theta */
    int opes_max_kernels;     /* step: kernel capacity per bias (default 1024 if <= 0) */
    unsigned long long seed;  /* step: Philox4x32-10 key */
    double lambda_temperature; /* step: theta's thermostat temperature, K (<= 0: `temperature`).  A hot
                                * theta is the lambda-d-AFED protocol (Section 3.2: 5000-10000 K with
                                * masses 1e4-1e6 amu nm^2); the OPES biases keep the physical beta */
    double sc_alpha;          /* > 0: soft-core coupling instead of the linear-basis soft term: the
                               * solute-solvent LJ is the Beutler et al. (1994) form at lambda,
                               * 4 eps l^p [1/D^2 - 1/D] S(r), D = sc_alpha (1 - l) + (r/sigma)^6
                               * (the paper contrasts its Eq. 4-6 coupling with soft-core and gives
                               * no formula); the solute-solvent Coulomb terms keep h_A.  Then
                               * U = U_vv + U_uu + h_A U_uv + U_soft with U_soft the soft-core term
                               * at lambda, dU/dl = h_A' U_uv + dU_soft/dl.  Parameter gradients and
                               * lambda exchange (which rely on the linear basis) are refused.
                               * 0: linear-basis coupling (default) */
    double sc_power;          /* p of the soft-core form (>= 1 when sc_alpha > 0) */
} lfe_params;

/* System description (host arrays, copied by lfe_create).
 *   excl      [2 n_excl]  pairs left out of the ordinary pair sum.  They get
 *                         the Ewald exclusion correction -k_e q_i q_j erf(a r)/r.
 *   pairs14   [2 n_14]    subset of excl that also gets scaled 1-4 terms
 *   scale14   [2 n_14]    (s_LJ, s_Coulomb) per 1-4 pair
 *   water_OHH [3 n_waters] rigid waters (O, H, H) held at water_rOH /
 *                         water_rHH by an exact Newton solve of the three
 *                         distance constraints (the result SETTLE gives)
 *   constraints [2 n_cons], constraint_len [n_cons]: X-H distance constraints;
 *                         every constraint must share its first atom with the
 *                         other constraints of its group (star groups of <= 4)
 *   bonds [2 nb] + bond_par [2 nb] (k, r0): 1/2 k (r - r0)^2
 *   angles [3 na] + angle_par [2 na] (k, theta0), vertex in the middle
 *   torsions [4 nt] + torsion_par [3 nt] (k, n, phi0): k (1 + cos(n phi - phi0))
 *   mass [n]  amu; 0 freezes the atom (it never moves).
 *   solute [n] 1 = solute atom, 0 = solvent.  Solute-solvent pairs are
 *             exactly the lambda-coupled ones (coupling route, Section 2.2).
 */
typedef struct {
    int n_atoms;
    const double* pos;
    const double* charge;
    const double* sigma;
    const double* epsilon;
    const unsigned char* solute;
    const double* mass;
    int n_excl;        const int* excl;
    int n_14;          const int* pairs14;      const double* scale14;
    int n_waters;      const int* water_OHH;    double water_rOH, water_rHH;
    int n_constraints; const int* constraints;  const double* constraint_len;
    int n_bonds;       const int* bonds;        const double* bond_par;
    int n_angles;      const int* angles;       const double* angle_par;
    int n_torsions;    const int* torsions;     const double* torsion_par;
} lfe_topology;

/* Create a system: validates and copies the description, allocates device
 * memory on the current device, builds the neighbour list.  *out is NULL on
 * failure (the message is then available from lfe_last_error(NULL)). */
int lfe_create(const lfe_params* params, const lfe_topology* topo, lfe_system** out);

/* Replace positions ([3N] doubles, host or device, caller order).  Host
 * positions are checked (non-finite: LFE_ERR_ARG, nothing changed).  The
 * neighbour list is rebuilt on the device when an atom lies more than skin/2
 * from where the list was built; otherwise it is kept (it stays valid).  The
 * call returns after queueing the work on `stream` (host input is copied
 * before it returns); a capacity overflow in that rebuild is settled by the
 * next call that synchronises (lfe_eval, lfe_param_grad, lfe_get_state). */
int lfe_set_positions(lfe_system* sys, const double* pos, int on_device, void* stream);

/* Replace velocities ([3N], host). */
int lfe_set_velocities(lfe_system* sys, const double* vel);

/* Change the atoms' integration parameters (time step ps, Langevin friction
 * 1/ps, temperature K) for the following lfe_step calls, e.g. for a short
 * small-step, high-friction equilibration from a packed start (the paper
 * equilibrates before production, Section 2.6).  theta keeps its own
 * friction; its time step follows dt.  The step graph is recaptured. */
int lfe_set_integrator(lfe_system* sys, double dt, double friction, double temperature);

/* Rebuild the cluster-pair list from the current positions (cell sort,
 * clustering, bounding boxes, tile list, exclusion masks). */
int lfe_build_neighbors(lfe_system* sys, void* stream);

/* Evaluate U(lambda), its forces and dU/dlambda (Eq. 4) at the current
 * positions.  forces: [3N] or NULL; energy_terms: [LFE_NTERMS] or NULL. */
int lfe_eval(lfe_system* sys, double lambda, double* forces, double* energy_terms,
             int out_on_device, void* stream);

/* Gradients of U(lambda) and dU/dlambda (Eq. 4, with the capped soft basis of
 * Eq. 5-6 and the switching functions of Eq. 7-10) with respect to each solute
 * atom's charge q_i, LJ sigma_i and LJ epsilon_i, at the current positions.
 * Solute atoms are in caller order (ascending atom index); per atom the
 * entries are (q, sigma, epsilon):
 *   dU_dp      [3 n_u]  dU/dp_i = dU_uu/dp_i + h_A dU_uv/dp_i + h_B dU_soft/dp_i
 *   d2U_dl_dp  [3 n_u]  d2U/(dlambda dp_i) = h_A' dU_uv/dp_i + h_B' dU_soft/dp_i
 *   basis      [9 n_u]  the class derivatives: basis[9 i + 3 p + c] with c = 0
 *                       dU_uu/dp, 1 dU_uv/dp, 2 dU_soft/dp
 * Any output may be NULL.  Lorentz-Berthelot mixing: d sigma_ij / d sigma_i =
 * 1/2 and d eps_ij / d eps_i = eps_ij / (2 eps_i); where eps_i = 0 the epsilon
 * derivative is singular and is reported as 0.  The reciprocal part uses the
 * smooth-PME grid of the system; bonded terms do not depend on these
 * parameters.  Everything is computed in FP64 on the device, in either
 * precision mode.  out_on_device != 0: outputs are device pointers, written
 * in stream order; otherwise host pointers, and the call returns after
 * synchronising.  lambda outside [0, 1] or a system without solute atoms:
 * LFE_ERR_ARG.  The dynamics' lambda state is left unchanged. */
int lfe_param_grad(lfe_system* sys, double lambda, double* dU_dp, double* d2U_dl_dp, double* basis,
                   int out_on_device, void* stream);

/* Replace the solute atoms' charges, LJ sigma and LJ epsilon (each [n_u] in
 * solute caller order; NULL leaves that parameter unchanged; on_device != 0
 * means device pointers).  Values are checked (finite; sigma, epsilon >= 0:
 * LFE_ERR_ARG otherwise, nothing changed).  The self and neutralising-
 * background energies follow the new charges and captured step graphs are
 * rebuilt on the next lfe_step.  Returns after synchronising.  The packed-
 * transform scale of the solute PME grid keeps the value chosen at creation. */
int lfe_set_solute_params(lfe_system* sys, const double* charge, const double* sigma, const double* epsilon,
                          int on_device, void* stream);

/* Advance n_steps of atoms + theta (replays one captured CUDA graph per step
 * on `stream`, rebuilding the neighbour list on the device when an atom has
 * moved more than skin/2).  Returns after the work is queued; errors raised
 * on the device are reported by the next call that synchronises. */
int lfe_step(lfe_system* sys, int n_steps, void* stream);

/* Copy state to host: pos [3N], vel [3N] (either may be NULL); ext (may be
 * NULL) receives LFE_NEXT doubles: [theta, p_theta, lambda, dU/dlambda, U,
 * n_kernels_std, n_kernels_exp, step, neighbour rebuilds done by lfe_step
 * (and by evaluations that found a rebuild left pending by the last step),
 * tiles of the current neighbour list (8 i atoms x 32 j atoms each), pairs
 * within r_cut counted by the last step's pair kernel, tiles of the pruned
 * list (lfe_set_list_prune; 0 before the first pruning), prunings done by
 * lfe_step].
 * Synchronises the device and reports errors raised by queued steps. */
#define LFE_NEXT 13
int lfe_get_state(lfe_system* sys, double* pos, double* vel, double* ext);

/* Monte Carlo volume move (Section 2.6: the runs are isothermal-isobaric
 * with a Monte Carlo barostat, Aqvist et al. 2004; the paper gives no
 * equations): at the current lambda, V' = V + dv_max (2 u0 - 1) (nm^3);
 * every box edge scales by s = (V'/V)^(1/3) and every molecule's centre of
 * mass by s with its atoms moved rigidly (molecules = connected components
 * of the exclusion list; a molecule of massless atoms scales about its
 * geometric centre); accepted with probability min(1, exp(-(U' - U +
 * P (V' - V)) / k_B T + N_mol ln(V'/V))), U the evaluation's potential energy
 * at the current lambda, T the atoms' temperature, P in bar.  u0 and the
 * acceptance uniform u1 are the first two words of Philox4x32-10 at counter
 * (attempt_lo, attempt_hi, 0, 4) with key seed, as (x + 0.5) / 2^32.  A move
 * whose box would break r_cut <= L/2, or V' <= 0, is rejected.  A rejected
 * move restores positions and box exactly; an accepted one recomputes the
 * box-dependent tables and constants, rebuilds the neighbour list and
 * recaptures the step graph.  Velocities are unchanged.  Outputs (host, any
 * may be NULL): accepted (0/1), box_out [3] (the box after the move),
 * energies [2] (U before, U at the proposed state; equal when rejected before
 * evaluation).  Synchronises the device.  Checkpoints store the box.
 * Errors: LFE_ERR_ARG (non-finite pressure, dv_max <= 0), LFE_ERR_STATE
 * (temperature <= 0). */
int lfe_mc_volume_move(lfe_system* sys, double pressure_bar, double dv_max, unsigned long long seed,
                       unsigned long long attempt, int* accepted, double* box_out, double* energies);

/* One step with host input and output: the stepping of Section 2.6 with
 * the configuration read back every step (the paper saves configurations
 * every 200 fs; this serves callers that read or replace them every step),
 * the equivalent of
 * lfe_set_positions(pos_in, host) + lfe_step(1) + lfe_get_state(pos_out,
 * vel_out, ext_out), replayed as one captured CUDA graph that holds the
 * host-to-device copy, the step and the device-to-host copies, followed by
 * one stream synchronisation.  pos_in [3N] (NULL: keep the device
 * positions), pos_out [3N] and vel_out [3N] (either may be NULL) are host
 * arrays in page-locked memory (cudaHostAlloc or cudaHostRegister;
 * otherwise LFE_ERR_ARG), caller order; ext_out (ordinary host memory, may
 * be NULL) receives the LFE_NEXT values of lfe_get_state.  pos_in is checked
 * on the device, inside the graph (a coordinate that is not finite: the
 * step leaves the state as it was, the outputs receive that state, and the
 * call returns LFE_ERR_ARG).  The
 * graph is captured on the first call and again whenever the host pointers
 * change.  A neighbour-list overflow inside the step is recovered (grow,
 * rebuild, replay) before the call returns.  Returns after synchronising
 * `stream`. */
int lfe_step_io(lfe_system* sys, const double* pos_in, double* pos_out, double* vel_out, double* ext_out,
                void* stream);

/* Dynamic pruning of the neighbour list (a buffered pair list pruned
 * between rebuilds): with an inner buffer 0 < b < the list buffer (skin),
 * the pair kernel of lfe_step works on a list cut from the built one, which
 * keeps a j entry of a tile when it lies within r_cut + b of one of the
 * tile's i atoms whose pair with it is computed; the cut is made in the
 * step graph (a conditional node after the conditional rebuild) after every
 * rebuild and whenever an atom has moved more than b/2 since the last cut,
 * so every pair within r_cut is still evaluated and the results equal those
 * of the full list up to the order of FP32 partial sums.  The list buffer
 * then only sets how often the list is rebuilt.  b = 0 (the default), or b
 * not below the list buffer, switches it off.  A system in a batch
 * (lfe_batch_*) prunes in the batch's steps the same way; lfe_eval and
 * eager stepping always use the built list.  Recaptures the step graphs.
 * Errors: LFE_ERR_ARG (b < 0 or not finite). */
int lfe_set_list_prune(lfe_system* sys, double inner_buffer);

/* lfe_step_io with the positions and velocities as floats: pos_in, pos_out
 * and vel_out are float arrays [3N] in page-locked host memory (same
 * ownership, checks, NULL meanings and errors as lfe_step_io); ext_out stays
 * double [LFE_NEXT].  The input is widened exactly to the device coordinate
 * type, so an FP32 system steps from the same bits as through lfe_step_io
 * with the same floats widened to double; the outputs are the device state
 * rounded to float (the device positions and velocities of an FP32 system
 * are floats already).  Halves the bytes crossing the host link. */
int lfe_step_io_f32(lfe_system* sys, const float* pos_in, float* pos_out, float* vel_out, double* ext_out,
                    void* stream);

/* d-AFED (Eq. 15): n_cv torsions xi_k (atoms[4k .. 4k+3], the IUPAC sign:
 * atan2(|b2| b1 . (b2 x b3), (b1 x b2) . (b2 x b3)) with b1 = r_j - r_i,
 * b2 = r_k - r_j, b3 = r_l - r_k, minimum images) are coupled to auxiliary
 * angles s_k by kappa_k / 2 (xi_k - s_k)^2, the difference wrapped into
 * [-pi, pi).  Each s_k has mass mass[k] (amu nm^2 rad^-2) and is advanced by
 * the same middle scheme as the atoms at its own temperature (K) with
 * friction (ps^-1), with the atoms' time step; s0 (rad, may be NULL: the
 * current torsions) are the initial angles, momenta start at 0.  The
 * coupling forces join the atomic forces and the coupling energy joins U.
 * n_cv = 0 removes the coupling.  Indices out of range, a repeated atom in a
 * torsion, kappa < 0, mass <= 0 or non-finite input: LFE_ERR_ARG.  The
 * auxiliary angles, momenta and thermostat velocities are part of
 * checkpoints (a checkpoint restores
 * only into a system with the same number of coupled torsions).
 * Paper values: 1000 K, 50 amu nm^2 rad^-2, kappa 1000 kJ mol^-1 rad^-2. */
int lfe_set_dafed(lfe_system* sys, int n_cv, const int* atoms, const double* kappa, const double* mass,
                  double temperature, double friction, const double* s0);

/* Current auxiliary angles s [n_cv], momenta p_s [n_cv] and the torsions xi
 * [n_cv] at the current positions (host arrays, any may be NULL).
 * Synchronises. */
int lfe_dafed_state(lfe_system* sys, double* s, double* p_s, double* xi);

/* Thermostat of the extended variables: theta (when lambda_mass > 0) and
 * the d-AFED auxiliary angles (Section 2.6 couples them to a regulated
 * Nose-Hoover-Langevin thermostat with time constant 40 fs, friction
 * 25 ps^-1 and regulation parameter 1, citing Abreu and Tuckerman; the
 * paper gives no equations, and these are that method's).
 * kind LFE_EXT_LANGEVIN (the default): each variable takes the atoms' middle
 * scheme, Langevin with its own friction (lambda_friction for theta, the
 * d-AFED friction for the auxiliary angles).  kind LFE_EXT_RNHL: each variable
 * x of mass m, momentum p and temperature T (kT = k_B T) moves with the
 * regulated velocity dx/dt = sqrt(n kT / m) tanh(p / sqrt(n m kT)), n =
 * n_reg, has dp/dt = f - v_eta p, and its thermostat velocity follows
 * dv_eta = (p dx/dt - kT) / Q dt - gamma v_eta dt + sqrt(2 gamma kT / Q) dW
 * with Q = kT tau^2 (tau in ps) and gamma the same friction as above; the
 * position marginal stays Boltzmann.  One step: p += dt f; x += dt/2 dx/dt;
 * NH(dt/2), the exact Ornstein-Uhlenbeck step of v_eta over dt (the
 * variable's standard normal), NH(dt/2), where NH(h) is v_eta += h/2 G,
 * p *= exp(-v_eta h), v_eta += h/2 G with G = (p dx/dt - kT) / Q; x += dt/2
 * dx/dt.  Every thermostat velocity is set to 0; the velocities are part of
 * checkpoints.  Synchronises.  Errors: LFE_ERR_ARG (unknown kind; for RNHL,
 * tau or n_reg not finite and > 0). */
#define LFE_EXT_LANGEVIN 0
#define LFE_EXT_RNHL 1
int lfe_set_ext_thermostat(lfe_system* sys, int kind, double tau, double n_reg);

/* Thermostat velocities v_eta of theta (one value) and of the d-AFED
 * auxiliary angles (n_cv values), host arrays, either may be NULL; zero
 * under the Langevin thermostat.  Synchronises. */
int lfe_ext_thermostat_state(lfe_system* sys, double* v_eta_theta, double* v_eta_aux);

/* Eq. 16 at the current positions: mass_out[k] = c [sum_i |d xi_k / d r_i|^2
 * / m_i]^-1 over the four atoms of torsion k (atoms of mass 0 are fixed and
 * do not contribute; a torsion with none movable: LFE_ERR_ARG). */
int lfe_dafed_masses(lfe_system* sys, int n_cv, const int* atoms, double c, double* mass_out);

/* Thermodynamic integration (Eq. 2): every step adds dU/dlambda, evaluated
 * at that step's lambda, to one of LFE_TI_BINS equal lambda bins (bin b holds
 * lambda in [b/n, (b+1)/n); lambda = 1 is in the last bin).  lfe_ti returns,
 * into host arrays of LFE_TI_BINS (either may be NULL), the bin means (NaN
 * for an empty bin) and sample counts, and in *delta_g (may be NULL) the
 * integral over lambda in [0, 1] of the mean-force profile: trapezoid rule
 * over the centres of the occupied bins, with the line through the two
 * nearest occupied centres extended to lambda = 0 and lambda = 1 (a
 * constant if one bin is occupied, NaN if none).  reset != 0 clears the
 * accumulators afterwards.  Synchronises.  The accumulators are part of
 * checkpoints. */
#define LFE_TI_BINS 100
int lfe_ti(lfe_system* sys, double* mean, double* count, double* delta_g, int reset);

/* Write / read a versioned binary checkpoint (positions, velocities, theta,
 * p_theta, OPES kernels, step counter, TI accumulators; checksum verified on
 * restore). */
int lfe_checkpoint(lfe_system* sys, const char* path);
int lfe_restore(lfe_system* sys, const char* path);

/* Mean device time (ms) of each kernel stage over `reps` eager evaluations at
 * lambda, timed with CUDA events on `stream`: list build, pair kernel (the
 * step's launch shape), PME stages, exclusions, bonded terms, output, FP64
 * solute-solvent energies and, for FP32 systems, "pairs_full" (the pair
 * kernel once more with a grid that fills every multiprocessor); with
 * pruning on (lfe_set_list_prune), "prune" (cutting the pruned list from
 * the built one) and "pairs_pruned" (the pair kernel on it).  names/ms
 * arrays of length max_n; returns the number of stages written (>= 0) or an
 * error code. */
int lfe_time_stages(lfe_system* sys, double lambda, int reps, void* stream,
                    const char** names, double* ms, int max_n);

/* Set theta (wrapped into [0, 2)) and its momentum; lambda follows Eq. 3.
 * For replicas held at a fixed lambda (lambda_mass <= 0) this sets lambda.
 * Synchronises the device.  Errors: LFE_ERR_ARG (non-finite input). */
int lfe_set_theta(lfe_system* sys, double theta, double p_theta);

/* Neighbour-list capacity (Section 2.6 states the cutoff and switch the list
 * serves; the list itself is this library's data structure).  Replaces the
 * tile list by one holding exactly `tiles` tiles of 8 i atoms x 32 j atoms
 * (and, with a solute, the solute-solvent pair list by one of `tiles` solute
 * tiles and 32 x `tiles` pairs) and flags a rebuild, so that the next step
 * or evaluation builds the lists again within them.  When a later build
 * needs more room the library grows the lists by itself: a build inside a
 * captured step marks the step and the
 * ones after it as skipped, and the next synchronising call (or every 64
 * steps) grows the list, rebuilds it and replays the skipped steps; results
 * are those of an uncapped list.  Meant for memory-constrained callers and
 * for exercising that recovery.  Synchronises the device.  Errors:
 * LFE_ERR_ARG (tiles < 1), LFE_ERR_CUDA. */
int lfe_set_list_capacity(lfe_system* sys, int tiles);

/* Autotuner: choose the evaluation's launch shapes for this system by
 * timing it on the device: when the system steps (dt > 0), the mean time
 * of `reps` captured steps from a saved state (a temporary checkpoint file
 * in /tmp, restored before every candidate and at the end); otherwise, or
 * when the trial steps fail, its captured evaluation graph (the five
 * concurrent branches of the step, timed with and without a preceding list
 * rebuild, weighted 1:3).  Knobs: blocks of the pair kernel per multiprocessor (1 up to
 * the resident maximum), blocks of the FP64 solute-solvent energy kernel
 * (0.5 to 4 per multiprocessor) and lines per block of the df64 transform
 * passes (4 or 16) and, when lfe_params.skin <= 0 and the objective is the
 * stepped one, the neighbour-list buffer (0.10, 0.14, 0.18, 0.22 or 0.26 nm,
 * each with every pair-kernel block count: a wider buffer means fewer
 * rebuilds and longer tile lists), one knob at a time otherwise, `reps`
 * (1..10000) steps or graph
 * replays per candidate (mean step time, or the median replay), a candidate
 * replacing the current choice only when 2 % faster.  The replays leave the state
 * (positions, velocities, theta, counters, accumulators) as it was; the next
 * lfe_step recaptures its graph with the chosen shapes.  Call it on an
 * equilibrated system (the stepped objective needs stable dynamics).  Launch shapes change
 * only how work is split over blocks and warps, and the buffer only which
 * tiles hold the pairs within the cutoff, so results stay within the
 * precision mode's tolerance (summation order).  cache_path (or NULL): a JSON
 * file of tuned entries keyed on the device, atom counts, density, cutoff,
 * grid and precision; a matching entry is applied without timing, a new one
 * is added.  Outputs (each may be NULL): best_ms = the objective (ms) of
 * the choice; params[5] = (pair blocks per SM, uv energy blocks, df64 lines,
 * 1 if taken from the cache else 0, list buffer in 1e-3 nm).  Errors: LFE_ERR_ARG (reps out of range,
 * cache not writable), LFE_ERR_CUDA.  Not part of the paper's method: it
 * serves the batched-replica workload's "sizes chosen by an autotuner". */
int lfe_autotune(lfe_system* sys, int reps, const char* cache_path, double* best_ms, int* params);

/* Measured arithmetic throughput of the current device in TFLOP/s (FMA =
 * 2 flops): 8 independent FMA chains per thread over 8 blocks of 256 threads
 * per multiprocessor, best of three timed launches (CUDA events), for FP32
 * and FP64 (either pointer may be NULL to skip).  A measured denominator
 * beside the unit-count peak (SMs x 128 FP32 lanes x 2 x clock) that the pair
 * kernel's ALU roofline is quoted against; allocates 2 KB of device memory
 * for the result sink.  Errors: LFE_ERR_CUDA.  The paper has no counterpart. */
int lfe_alu_peak(double* fp32_tflops, double* fp64_tflops);

/* Batched replicas (lambda windows, solvents, solutes; sizes may differ):
 * lfe_batch_create groups existing systems (not copied; they must outlive
 * the batch and must not be destroyed while it exists).  lfe_batch_step
 * advances every replica n_steps with one graph launch per step: each
 * replica's rebuild decision and device-side neighbour-list rebuild, PME,
 * exclusion, bonded and integrator kernels form its own chain, and the pair
 * kernels of all FP32 replicas run as ONE launch over their concatenated
 * tile lists once every list is ready (FP64 replicas keep their own);
 * results are identical to stepping each system alone (the pair kernel's
 * partial sums cover fixed chunks of each system's tiles, whichever warp
 * takes them).  lfe_batch_time_pairs (ms, host) is the mean device time of
 * that shared launch over `reps` launches at the current lists (the forces
 * and energies it adds are cleared afterwards; call it between steps).
 * lfe_batch_eval evaluates replica i at lambdas[i] and writes
 * energy_terms[i][LFE_NTERMS] (host); positions and velocities are read with
 * lfe_get_state on each system.  Errors of a batch call are described by
 * lfe_batch_last_error. */
int lfe_batch_create(lfe_system* const* systems, int n, lfe_batch** out);
int lfe_batch_eval(lfe_batch* b, const double* lambdas, double* energy_terms, void* stream);
int lfe_batch_step(lfe_batch* b, int n_steps, void* stream);
int lfe_batch_time_pairs(lfe_batch* b, int reps, double* ms, void* stream);

/* Lambda replica exchange (the paper's HREX reference protocol, Section 2.6,
 * on the linear-basis potential of Eq. 4).  `ladder` lists n >= 2 replicas
 * of the batch (indices) in increasing lambda; each must have a frozen theta
 * (lambda_mass <= 0).  Every replica of the ladder is evaluated at its own
 * lambda (positions as they stand), and the pairs (k, k+1) with k of the
 * parity of `attempt` are tried: the swap changes the total energy by
 * Delta = (h_A(l_k+1) - h_A(l_k)) (U_uv,k - U_uv,k+1)
 *       + (h_B(l_k+1) - h_B(l_k)) (U_soft,k - U_soft,k+1)
 * and is accepted when Delta <= 0 or u < exp(-Delta / k_B T), u = (x + 0.5)/2^32
 * with x the first word of Philox4x32-10 at counter (k, attempt_lo,
 * attempt_hi, 3) under key (seed_lo, seed_hi).  An accepted pair exchanges
 * the two replicas' lambdas (theta set to the new lambda, p_theta 0) and
 * its two ladder entries, so that `ladder` stays in lambda order.
 * accepted[n-1] (may be NULL): 1 for each accepted pair.  Errors:
 * LFE_ERR_ARG (ladder, temperature, dynamical theta), others from the
 * evaluations. */
int lfe_batch_exchange(lfe_batch* b, int n, int* ladder, double temperature, unsigned long long seed,
                       unsigned long long attempt, int* accepted, void* stream);
/* The same exchange on the device, inside lfe_batch_step: after every
 * `stride` batch steps (stride <= 0 switches it off) a captured exchange
 * graph is enqueued on the step's stream -- an evaluation of every replica
 * of the ladder at its own lambda and current configuration (with its own
 * conditional list rebuild), then one device kernel that takes the
 * attempt's Metropolis decisions exactly as lfe_batch_exchange does (same
 * Delta, same Philox counter (k, attempt_lo, attempt_hi, 3), attempts
 * numbered from 0 when the exchange is set) and swaps the lambdas and the
 * ladder entries on the device.  The host takes no decision and reads no
 * energy; before each attempt it checks each replica's list-overflow flag
 * (regrowing a list that overflowed, so that no energy comes from a
 * truncated list).  lfe_batch_set_exchange validates the ladder as
 * lfe_batch_exchange does and resets the counters; lfe_batch_exchange_state
 * (synchronises) reads back the ladder [n], the number of attempts and the
 * accepted swaps per ladder position [n-1] (any pointer may be NULL; the
 * replicas' lambdas are read with lfe_get_state).  Errors: LFE_ERR_ARG,
 * LFE_ERR_STATE (soft-core coupling; no exchange set). */
int lfe_batch_set_exchange(lfe_batch* b, int n, const int* ladder, double temperature, unsigned long long seed,
                           int stride);
int lfe_batch_exchange_state(lfe_batch* b, int* ladder, unsigned long long* attempts, unsigned long long* accepted);
const char* lfe_batch_last_error(const lfe_batch* b);
void lfe_batch_destroy(lfe_batch* b);

/* Smooth-PME reciprocal-space class energies and forces of one
 * configuration, computed without any device allocation.  The paper has no
 * counterpart: this entry exists for callers that cannot let a library call
 * cudaMalloc -- processes whose device memory belongs to a pool or allocator
 * that forbids hidden allocations, services that must not grow their memory
 * after start-up, and code running where allocation calls are not
 * permitted.  A call issues only kernel launches and memsets on `stream`.
 *
 * The grids and tables live in one fixed file-scope device array sized for
 * LFE_NOALLOC_MAX_GRID grid points (about 4.4 MB), which every GPU that loads
 * the library holds until the process exits; larger grids are rejected with
 * LFE_ERR_ARG.  All pointers are device memory on the current device:
 *   pos [3n], charge [n], solute [n] (1 = solute), forces [3n] (written),
 *   energies [3] (written): the class energies (reciprocal + self +
 *   neutralising background) E_vv, E_uu, E_uv.
 * box [3] and grid [3] are host arrays; lambda selects h_A(lambda) for the
 * forces (solvent atoms feel phi_v + h_A phi_u, solute atoms phi_u + h_A
 * phi_v).  Outputs are complete when the stream reaches the end of the call.
 * The first call on a device (with that device current) looks up the
 * array's device address with cudaGetSymbolAddress.  Every call shares the
 * array and overwrites what the last call left there: calls that overlap on
 * the GPU (different streams, or threads without ordering) race and give
 * wrong results.  Errors: LFE_ERR_ARG (sizes, grid too large), LFE_ERR_CUDA;
 * the message is available from lfe_last_error(NULL). */
#define LFE_NOALLOC_MAX_GRID 110592   /* 48 x 48 x 48 */
int lfe_pme_noalloc(int n, const double* pos, const double* charge, const unsigned char* solute,
                    const double* box, double alpha, const int* grid, double lambda,
                    double* forces, double* energies, void* stream);

/* Message of the last error recorded for sys (or of the last failed
 * lfe_create or lfe_pme_noalloc when sys is NULL).  Valid until the next call
 * on sys. */
const char* lfe_last_error(const lfe_system* sys);

void lfe_destroy(lfe_system* sys);

#ifdef __cplusplus
}
#endif
#endif
