// lfe_views.cuh -- plain-pointer views of a system's device buffers, passed
// by value to kernels, and the host-side launcher declarations.
#pragma once
#include <string>

#include "lfe.h"
#include "lfe_dev.cuh"
#include "df64.cuh"

namespace lfe {

template <typename real>
struct SysView {
    int n;          // atoms
    int n_pad;      // cluster slots (n_cl * 32)
    int n_cl;       // clusters
    int n_ucl;      // solute clusters (they come first)
    int n_u;        // solute atoms
    int n_solv;     // solvent atoms
    real L[3], invL[3];
    real rc2;       // r_cut^2
    real rsw;       // LJ switch start (r_cut when there is no switch)
    real sw_inv_w;  // 1 / (r_cut - r_switch)
    real alpha;     // Ewald alpha
    real two_a_sqrtpi;
    double sc_alpha;   // > 0: soft-core coupling of the solute-solvent LJ (see lfe_params)
    double sc_power;
    // master state, caller order
    R4<real>* x;
    R4<real>* v;
    R4<real>* xref;     // positions at the last neighbour-list build
    R4<real>* xpr;      // positions at the last pruning of the pair list
    real* invm;
    const real* q;      // charges (e)
    const real* sig;
    const real* eps;
    const unsigned char* sol;
    const int* solute_list;   // solute atoms, caller order
    const int* solv_list;     // solvent atoms, caller order
    // cluster-sorted arrays
    R4<real>* xq;       // wrapped x, y, z and sqrt(k_e) q
    R2<real>* lj;       // sigma/2, 2 sqrt(eps)
    int* perm;          // slot -> atom (-1 = padding)
    int* iperm;         // atom -> slot
    long long* F;       // fixed-point forces [3][n_pad] of the neighbour-list terms (slot order)
    long long* Fa;      // fixed-point forces [3][n] of the other terms (atom order): PME, exclusion
                        // and 1-4 corrections, bonded, d-AFED -- independent of the list build
    long long* E;       // energy accumulators [E_N]
    int* flags;         // [FL_N]
    LamState* lam;
};

template <typename real>
struct NblView {
    // column sort of the solvent: ncx x ncy columns in xy, each sorted by z
    // and cut into clusters of 32 consecutive atoms (near-cubic clusters)
    int ncx, ncy, ncols;
    real cinvx, cinvy;    // columns per nm
    int* col_of;          // [n_solv] column of each solvent atom (solv_list order)
    int* col_cnt;         // [ncols] histogram (zeroed after the scan)
    int* col_start;       // [ncols + 1]
    int* col_fill;        // [ncols] scatter counters (zeroed after use)
    int* col_cl;          // [ncols + 1] first solvent cluster of each column
    int* tmp;             // [n_solv] solvent atoms grouped by column
    int* tmp2;            // [n_solv] ... and sorted by z inside each column
    int* n_cl_solv;       // [1] solvent clusters of the current build
    int n_cl_max;         // capacity in clusters
    R4<float>* bbc;       // cluster bounding-box centres [n_cl_max]
    R4<float>* bbh;       // half extents [n_cl_max]
    R4<float>* bbc8;      // 8-slot sub-cluster boxes [4 n_cl_max] (the i side of the tiles)
    R4<float>* bbh8;      // their half extents (w < 0: no atoms)
    int* tile_cnt;        // [27 x 4 n_cl_max] tiles per (i sub-cluster, shift), then offsets inside it
    int* tile_tot;        // [4 n_cl_max] tiles per i sub-cluster (zeroed by the scan)
    int* tile_off;        // [4 n_cl_max + 1] first tile of each i sub-cluster
    int4* stage_hdr;      // [stage_cap] tiles as found: (I8, shift, class, ordinal in (I8, shift); -1 = unused)
    int* stage_j;         // [stage_cap * 32] their j slots
    int stage_cap;
    int4* tiles;          // [cap]  (I8, shift code, class, -)
    int* jidx;            // [cap * 32] j slots of each tile (-1 = empty)
    unsigned char* masks; // [cap * 32] one byte per j entry: bit r = pair (i atom r, j entry) computed
    int cap;
    float cut2;           // (r_cut + skin)^2
    float skin_half2;     // (skin / 2)^2
    const int* ex_start;  // exclusion CSR, caller order [n + 1]
    const int* ex_list;
    const int* mol;       // [n] molecule id (connected component of the exclusions: its lowest atom)
    const unsigned long long* exm;   // [n] exclusion partners as bits of (partner - molecule id), bit 63 set:
                                     // the molecule spans more than 63 atom indices (search the list)
    // dense solute-solvent pair list (pairs within r_cut + skin at build time)
    int* uv_cnt;          // [n_ucl_tiles_max] per-tile counts
    int* uv_off;          // [n_ucl_tiles_max + 1]
    int4* uvp;            // [uv_cap] (slot_i, slot_j, shift code, -)
    int uv_cap;
    int uv_tiles_max;     // capacity of uv_cnt / uv_off
    int n_sm;             // multiprocessors of the device (grid-stride kernels)
    int ntiles_flag;      // flags slot holding the tile count (FL_NTILES; FL_PTILES for the pruned list)
};

// Dynamic pruning of the tile list: between rebuilds, a shorter list is cut
// from the built one, keeping the j entries within r_cut + inner buffer of
// one of their tile's i atoms at the positions of the pruning; it is pruned
// again once an atom has moved more than half the inner buffer since.
struct PruneView {
    float cut2;           // (r_cut + inner buffer)^2
    unsigned* kb;         // [cap] per tile of the built list: j entries kept
    int* base;            // [cap] place of the tile's first kept entry in its sub-cluster's output
                          // (bit 30: the tile ends a run of one shift and class)
    int* cnt;             // [4 n_cl_max] pruned tiles per i sub-cluster (zeroed by the scan)
    int* off;             // [4 n_cl_max + 1] first pruned tile of each i sub-cluster
};

template <typename real>
struct ExclView {
    int n_excl, n14;
    const int2* excl;       // caller-order pairs
    const int2* p14;
    const R2<real>* s14;    // (s_LJ, s_C)
    const R2<double>* s14d; // the same scales in FP64 (parameter gradients)
    // per-atom partner lists (caller order, both directions)
    const int* ex_start;      // [n + 1] exclusion partners
    const int* ex_list;
    const int* p14_start;     // [n + 1] 1-4 partners
    const int* p14_list;
    const R2<real>* p14_s;    // (s_LJ, s_C) of each 1-4 partner entry
};

template <typename real>
struct PmeView {
    int K[3];
    int KK;                   // K0 K1 K2
    real kscale[3];           // K_d / L_d
    double kscale64[3];       // K_d / L_d in double (fractional coordinates)
    long long* Qfix;          // [2][KK]  (solvent, solute) fixed point
    R2<real>* Z;              // [KK] complex work grid
    const real* gfac[3];      // per-axis exp(-pi^2 m^2 / (L^2 alpha^2)) * |b(m)|^2
    const real* msq[3];       // per-axis (m_d / L_d)^2
    real conv_pre;            // k_e / (pi V)
    real qu_scale;            // power of two applied to the solute grid in the packed transform
    const R2<real>* tw[3];    // twiddles exp(+2 pi i t / K_d)
    int nrad[3];
    int rad[3][8];
    real* phi_u;              // [n_u] reciprocal potential of the other class at solute atoms
    R2<double>* Zraw64;       // optional: FP64 copy of the packed charge grid written by the first pass
    const R2<double>* Zin64;  // optional: FP64 input grid of the axis-2 (first) per-axis pass, read instead of Z
    int lines;                // df64 per-axis passes: lines per block (4 or 16; 0 = the largest that fits)
    // plane / column transform (used when a K1 x K2 plane fits in shared memory)
    int planes;               // 1: plane kernels in use, 0: one kernel per axis
    int ngroups, cg_max;      // column groups of the axis-0 pass and the largest group
    const int* cg_start;      // [ngroups + 1]
    const int* cg_col;        // [K1 K2] flat column index k1 K2 + k2, grouped, ascending in a group
    const int* cg_part;       // [K1 K2] position in the group of each column's partner (-k1, -k2)
};

template <typename real>
struct BondView {
    int nb, na, nt;
    const int2* b;  const R2<real>* bp;
    const int4* a;  const R2<real>* ap;     // a.w unused
    const int4* t;  const R4<real>* tp;     // (k, n, phi0, -)
};

// constraint groups: a rigid water (3 atoms, 3 constraints), a star of
// X-H constraints around a centre atom, or a single unconstrained atom
enum { GROUP_SINGLE = 0, GROUP_WATER = 1, GROUP_STAR = 2 };
struct Group {
    int atom[4];
    int natom;
    int ncons;
    int ci[3], cj[3];     // constraint k joins atom[ci[k]] and atom[cj[k]]
    float len[3];
    int kind;             // GROUP_*: water (0-1, 0-2, 1-2) or star (0-k) shapes
};

template <typename real>
struct StepView {
    const Group* groups;
    int n_groups;
    real dt, a_fric, kT;       // a = exp(-gamma dt)
    uint2 key;
    real skin_half2;
    real prune_half2;          // (inner buffer / 2)^2 of the pruned list (0: no pruning)
    real* noise;               // [3 n] Ornstein-Uhlenbeck kicks of the step, formed ahead by k_noise
};

// Thermostat of the extended variables (theta and the d-AFED auxiliary
// angles, Section 2.6): kind 0 Langevin on the variable (friction gamma),
// kind 1 regulated Nose-Hoover-Langevin with time constant tau (Q = kT
// tau^2), regulation parameter n_reg and friction gamma on its velocity
struct ExtThermo {
    int kind;
    int pad;
    double tau, n_reg;
};

// constants of one extended variable's step (mass m, k_B T, a = exp(-gamma
// dt)), formed once per setting so that the step itself divides by nothing:
// im = 1 / m, amp = sqrt(kT (1 - a^2) / m) (Langevin); iQ = 1 / (kT tau^2),
// ipc = 1 / sqrt(n m kT), c = n kT ipc = sqrt(n kT / m), amp_eta = sqrt(kT
// (1 - a^2) iQ) (regulated Nose-Hoover-Langevin)
struct ExtConst {
    double im, amp, iQ, ipc, c, amp_eta;
};

__host__ __device__ inline ExtConst ext_const(const ExtThermo& th, double m, double kT, double a_fric)
{
    ExtConst k{};
    k.im = m > 0.0 ? 1.0 / m : 0.0;
    k.amp = m > 0.0 ? sqrt(kT * (1.0 - a_fric * a_fric) / m) : 0.0;
    if (th.kind == 1 && m > 0.0 && kT > 0.0) {
        k.iQ = 1.0 / (kT * th.tau * th.tau);
        k.ipc = 1.0 / sqrt(th.n_reg * m * kT);
        k.c = th.n_reg * kT * k.ipc;
        k.amp_eta = sqrt(kT * (1.0 - a_fric * a_fric) * k.iQ);
    }
    return k;
}

struct ThetaPre;

// d-AFED (Eq. 15): torsions coupled harmonically to auxiliary angles that
// have their own mass and temperature
struct DafedView {
    int n;                    // coupled torsions (0: off)
    const int4* atoms;        // [n] (i, j, k, l)
    const double* kappa;      // [n] kJ mol^-1 rad^-2
    const double* mass;       // [n] amu nm^2 rad^-2
    double* s;                // [n] auxiliary angles, [-pi, pi)
    double* p;                // [n] their momenta
    double* fs;               // [n] force on s of the last evaluation, kappa (xi - s)
    double* xi;               // [n] torsion values of the last evaluation
    double dt, a_fric, kT;    // time step, exp(-gamma dt), k_B T of the auxiliary variables
    uint2 key;
    ExtThermo th;             // thermostat of the auxiliary variables
    double* veta;             // [n] their thermostat velocities (regulated Nose-Hoover-Langevin)
    const ThetaPre* pre;      // the step's counter (formed at its start)
    const ExtConst* ec;       // [n] constants of each variable's step
};

// values of the theta step that depend only on the state at its start,
// formed while the forces are evaluated
struct ThetaPre {
    double V[2], dV[2];        // both OPES biases and their theta-derivatives at theta
    double noise;              // the theta integrator's standard normal
    unsigned long long step;   // the step counter at the start of the step
    // formed by k_theta_step once dU/dlambda is known, taken over by
    // k_theta_commit at the end of the step
    double dUdl, theta, p_theta, v_eta;
};

template <typename real>
struct ThetaView {
    double m, dt, a_fric, kT;
    int stride;
    int max_k;
    int on[2];              // biases enabled
    double beta, nu[2], epsr[2], sigma;
    double* centre;         // [2][max_k]
    double* weight;         // [2][max_k]
    double* S;              // [2][max_k]  unnormalised KDE at each centre
    OpesState* st;
    uint2 key;
    double const_uv;        // background share of U_uv (constant)
    double const_vv, const_uu;
    ThetaPre* pre;
    double* ti_sum;                 // [LFE_TI_BINS] sum of dU/dlambda per lambda bin (Eq. 2)
    unsigned long long* ti_cnt;     // [LFE_TI_BINS] samples per bin
    ExtThermo th;                   // theta's thermostat
    ExtConst tc;                    // its constants at m, kT, a_fric
};

// FP64 geometry and Ewald constants of the parameter-gradient kernel
struct AdjConst {
    double L[3], invL[3];
    double alpha, two_a_sqrtpi;   // Ewald alpha and 2 alpha / sqrt(pi)
    double rc2;                   // r_cut^2
    double rsw, swi;              // LJ switch start and 1 / (r_cut - r_sw) (0: no switch)
    double bg_pre;                // -k_e pi / (2 V alpha^2)
};

// ------------------------------------------------------------- launchers
// Launches kernel k on st; with pdl the launch carries the programmatic
// stream-serialisation attribute (only for a kernel that begins with
// pdl_wait() and whose predecessor in the stream is a kernel).  Launch errors
// surface through cudaGetLastError like those of <<< >>> launches.
template <typename... KArgs, typename... Args>
inline void launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

template <typename real> void launch_build_nbl(const SysView<real>& s, const NblView<real>& nb, cudaStream_t st);
// one FP32 system's share of a pair-kernel launch over many systems
struct PairJob {
    SysView<float> s;
    NblView<float> nb;
};
// the systems of one batched pair launch, passed by value (kernel parameter
// space holds up to 32,764 bytes: 60 systems of 536 bytes)
constexpr int PAIR_BATCH_MAX = 60;
struct PairJobs {
    PairJob j[PAIR_BATCH_MAX];
};
static_assert(sizeof(PairJobs) <= 32764, "the batched pair launch's systems must fit the kernel parameter space");
// jobs: a host array (captured by value into the launches)
void launch_pairs_batch(const PairJob* jobs, int njobs, int nblocks, cudaStream_t st);
int pairs_batch_blocks();   // one resident wave of the launch over many systems
void launch_hrex(LamState* const* lams, const double* terms, int* ladder, int n, double beta, unsigned long long seed,
                 unsigned long long* attempt, unsigned long long* accepted, cudaStream_t st);
template <typename real> void launch_pairs(const SysView<real>& s, const NblView<real>& nb, int nwarps, cudaStream_t st);
template <typename real> int pairs_blocks_per_sm();
template <typename real> void launch_uv_energy(const SysView<real>& s, const NblView<real>& nb, int nblocks, cudaStream_t st);
template <typename real> void launch_excl(const SysView<real>& s, const ExclView<real>& ex, cudaStream_t st);
template <typename real> void launch_pme(const SysView<real>& s, const PmeView<real>& p,
                                         const PmeView<df64>* energy64, cudaStream_t st);
template <typename real> void launch_spread(const SysView<real>& s, const PmeView<real>& p, cudaStream_t st);
template <typename real> void launch_fft(const PmeView<real>& p, int axis, int sign, int from_fixed, cudaStream_t st);
// shared memory of one per-axis pass of length K (at most 48 KB without opt-in)
template <typename real> size_t fft_smem(int K);
// mode: CONV_BOTH energies + potentials, CONV_ENERGY energies only, CONV_POTENTIAL potentials only
enum { CONV_BOTH = 0, CONV_ENERGY = 1, CONV_POTENTIAL = 2 };
template <typename real> void launch_conv(const PmeView<real>& p, long long* E, const LamState* lam, int mode,
                                          cudaStream_t st);
template <typename real> void launch_gather(const SysView<real>& s, const PmeView<real>& p, cudaStream_t st);
// plane / column transform: PLANE_FWD_FIX reads the fixed-point grids,
// clears them and writes the FP64 copy when Zraw64 is set; PLANE_FWD_KEEP
// reads them and leaves them (another pass reads them too; the grids are
// cleared once both have); PLANE_FWD transforms Z in place, PLANE_INV is the
// inverse transform of axes 1 and 2
enum { PLANE_FWD_FIX = 0, PLANE_FWD = 1, PLANE_INV = 2, PLANE_FWD_KEEP = 3 };
// axis-2 input of a per-axis pass (launch_fft from_fixed): FFT_FROM_Z the
// transform grid (or the FP64 copy), FFT_FROM_FIX the fixed-point grids
// (cleared, FP64 copy written), FFT_FROM_FIX_KEEP the fixed-point grids left
// as they are
enum { FFT_FROM_Z = 0, FFT_FROM_FIX = 1, FFT_FROM_FIX_KEEP = 2 };
template <typename real> void launch_planes(const PmeView<real>& p, int mode, cudaStream_t st);
// axis-0 transform of every column group with the convolution (mode as for
// launch_conv); CONV_POTENTIAL and CONV_BOTH end with the inverse axis-0 transform
template <typename real> void launch_columns(const PmeView<real>& p, long long* E, const LamState* lam, int mode,
                                             cudaStream_t st);
// shared-memory sizes of the plane and column kernels, and their attribute setup
template <typename real> size_t planes_smem(const PmeView<real>& p);
template <typename real> size_t columns_smem(const PmeView<real>& p);
template <typename real> void planes_setup(const PmeView<real>& p);
template <typename real> void energy_columns_setup(const PmeView<real>& p);
template <typename real> void launch_bonded(const SysView<real>& s, const BondView<real>& b, cudaStream_t st);
// pdl: launched as a programmatic dependent of the kernel before it in the
// stream (the kernels wait for their prerequisites before reading anything)
template <typename real> void launch_integrate(const SysView<real>& s, const StepView<real>& g, cudaStream_t st,
                                               bool pdl = false);
// theta's step: k_theta_step (dU/dlambda and the new theta, momentum and
// thermostat velocity, kept in ThetaPre) then k_theta_commit (U, the TI bin,
// the lambda state, OPES deposits, the step counter, clearing the energy
// accumulators); launch_theta runs both as one launch
template <typename real> void launch_theta(const SysView<real>& s, const ThetaView<real>& t, cudaStream_t st);
template <typename real> void launch_theta_step(const SysView<real>& s, const ThetaView<real>& t, cudaStream_t st,
                                                bool pdl = false);
template <typename real> void launch_theta_commit(const SysView<real>& s, const ThetaView<real>& t,
                                                  cudaStream_t st, bool pdl = false);
// d-AFED: forces of Eq. 15 on the atoms and the auxiliary variables (with
// the coupling energy), and the auxiliary variables' step
template <typename real> void launch_dafed_force(const SysView<real>& s, const DafedView& d, cudaStream_t st);
template <typename real> void launch_dafed_step(const SysView<real>& s, const DafedView& d, cudaStream_t st);
// torsion values of d's atoms at the current positions into out[n]; with
// c > 0, the masses of Eq. 16 (c [sum_i |d xi / d r_i|^2 / m_i]^-1) instead
template <typename real> void launch_dafed_probe(const SysView<real>& s, const DafedView& d, double c, double* out,
                                                 cudaStream_t st);
// the parts of the integrators that do not depend on the step's forces (the
// atoms' random kicks, the OPES bias at the current theta): launched
// alongside the force evaluation
template <typename real> void launch_prestep(const SysView<real>& s, const StepView<real>& g,
                                             const ThetaView<real>& t, cudaStream_t st);
template <typename real> void launch_rebuild_cond(const SysView<real>& s, cudaGraphConditionalHandle h, cudaStream_t st);
template <typename real> void launch_set_lambda(const SysView<real>& s, double lam, cudaStream_t st);
template <typename real> void launch_eval_out(const SysView<real>& s, double* forces, double* terms,
                                              double const_vv, double const_uu, double const_uv,
                                              cudaStream_t st);
// new positions from caller doubles: master and sorted copies, and the
// rebuild flag raised when an atom has moved more than skin/2 since the last
// build (the rebuild itself follows launch_rebuild_cond's conditional node);
// the pruning flag likewise for half the inner buffer (prune_half2 > 0)
template <typename real, typename TIO> void launch_assign_moved(const SysView<real>& s, const TIO* pos,
                                                                real skin_half2, real prune_half2, cudaStream_t st);
// the conditional pruning of the step graph: its decision kernel and, for
// the node's body, the pruning itself (built list nb -> pruned list np)
template <typename real> void launch_prune_cond(const SysView<real>& s, cudaGraphConditionalHandle h, cudaStream_t st);
template <typename real> void launch_prune(const SysView<real>& s, const NblView<real>& nb, const NblView<real>& np,
                                           const PruneView& pv, cudaStream_t st);
template <typename real, typename TIO> void launch_check_positions(const SysView<real>& s, const TIO* pos,
                                                                   cudaStream_t st);
template <typename real> void launch_refresh_sorted(const SysView<real>& s, cudaStream_t st);
template <typename real> void launch_scale_molecules(const SysView<real>& s, const int* mstart, const int* matoms,
                                                     const double* mass, int n_mol, double sc, const double* L,
                                                     cudaStream_t st);
template <typename real> void launch_pack_state(const SysView<real>& s, const OpesState* o, double* out,
                                                cudaStream_t st);
template <typename real> void launch_pack_state_f32(const SysView<real>& s, const OpesState* o, float* xv,
                                                    double* tail, cudaStream_t st);
// phi: FP64 grid of the class potentials (phi_v real, phi_u imaginary)
template <typename real> void launch_param_grad(const SysView<real>& s, const NblView<real>& nb,
                                                const ExclView<real>& ex, const PmeView<real>& pm,
                                                const R2<double>* phi, const AdjConst& c, double* dU,
                                                double* d2U, double* basis, cudaStream_t st);
template <typename real> void launch_set_solute_params(const SysView<real>& s, real* q, real* sig, real* eps,
                                                       const double* stage, cudaStream_t st);

// message returned by lfe_last_error(NULL)
void record_global_error(const std::string& m);

}  // namespace lfe
