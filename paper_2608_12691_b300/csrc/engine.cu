// engine.cu -- host side of the library: validation, device buffers, the
// neighbour-list capacity policy, eager evaluation, the captured per-step
// CUDA graph (with a device-side conditional node for list rebuilds),
// checkpoints and the C-ABI entry points declared in include/lfe.h.
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <unistd.h>
#include <memory>
#include <string>
#include <vector>
#include <algorithm>
#include <functional>
#include <fstream>
#include <sstream>
#include <type_traits>

#include "lfe.h"
#include "lfe_views.cuh"

using namespace lfe;

namespace {

thread_local std::string g_create_error;

struct Failure {
    int code;
    std::string msg;
};

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            throw Failure{LFE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};      \
    } while (0)

[[noreturn]] void fail(int code, const std::string& m) { throw Failure{code, m}; }

// Philox4x32-10 (Salmon et al. 2011) on the host, for the uniforms of the
// lambda exchange and the Monte Carlo volume move
void philox_host(unsigned c[4], unsigned k0, unsigned k1)
{
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * c[0], p1 = 0xCD9E8D57ull * c[2];
        const unsigned n0 = (unsigned)(p1 >> 32) ^ c[1] ^ k0, n1 = (unsigned)p1;
        const unsigned n2 = (unsigned)(p0 >> 32) ^ c[3] ^ k1, n3 = (unsigned)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// x * 0 is 0 for every finite x and NaN for an infinity or a NaN, so one
// branch-free (vectorisable) sum answers for the whole array
// every value finite: an IEEE double is infinite or NaN exactly when its 11
// exponent bits are all ones, and then adding 1 to the exponent field carries
// into the sign bit; integer AND/ADD/OR only, so the loop vectorises and runs
// at memory speed (positions just written by a device copy are read from DRAM)
bool finite_all(const float* a, size_t n)
{
    const uint32_t E = 0x7f800000u, ONE = 0x00800000u;
    uint32_t acc = 0;
    for (size_t i = 0; i < n; ++i) {
        uint32_t b;
        std::memcpy(&b, a + i, sizeof b);
        acc |= (b & E) + ONE;
    }
    return (acc >> 31) == 0;
}

bool finite_all(const double* a, size_t n)
{
    const uint64_t E = 0x7ff0000000000000ull, ONE = 0x0010000000000000ull;
    uint64_t acc = 0;
    for (size_t i = 0; i < n; ++i) {
        uint64_t b;
        std::memcpy(&b, a + i, sizeof b);
        acc |= (b & E) + ONE;
    }
    return (acc >> 63) == 0;
}

bool radix_plan(int K, int* rad, int* nrad)
{
    int n = 0, k = K;
    while (k % 4 == 0 && n < 8) { rad[n++] = 4; k /= 4; }
    while (k % 2 == 0 && n < 8) { rad[n++] = 2; k /= 2; }
    while (k % 3 == 0 && n < 8) { rad[n++] = 3; k /= 3; }
    while (k % 5 == 0 && n < 8) { rad[n++] = 5; k /= 5; }
    *nrad = n;
    return k == 1;
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}

}  // namespace

namespace lfe {
void record_global_error(const std::string& m) { g_create_error = m; }
}  // namespace lfe

struct SystemBase {
    virtual ~SystemBase() {}
    int precision = 0;
    virtual void set_positions(const double* pos, int on_device, cudaStream_t st) = 0;
    virtual void set_velocities(const double* vel) = 0;
    virtual void set_integrator(double dt, double friction, double temperature) = 0;
    virtual void build_neighbors(cudaStream_t st) = 0;
    virtual void eval(double lam, double* forces, double* terms, int out_on_device, cudaStream_t st) = 0;
    virtual void step(int n, cudaStream_t st) = 0;
    virtual void get_state(double* pos, double* vel, double* ext) = 0;
    virtual void checkpoint(const char* path) = 0;
    virtual void restore(const char* path) = 0;
    virtual int time_stages(double lam, int reps, cudaStream_t st, const char** names, double* ms, int max_n) = 0;
    virtual void param_grad(double lam, double* dU, double* d2U, double* basis, int on_device, cudaStream_t st) = 0;
    virtual void ti(double* mean, double* count, double* delta_g, int reset) = 0;
    virtual void set_dafed(int n, const int* atoms, const double* kappa, const double* mass, double temperature,
                           double friction, const double* s0) = 0;
    virtual void dafed_state(double* s, double* p, double* xi) = 0;
    virtual void set_ext_thermostat(int kind, double tau, double n_reg) = 0;
    virtual void ext_thermostat_state(double* v_theta, double* v_aux) = 0;
    virtual void dafed_masses(int n, const int* atoms, double c, double* out) = 0;
    virtual void set_solute_params(const double* q, const double* sig, const double* eps, int on_device,
                                   cudaStream_t st) = 0;
    // batched replicas: record this system's whole step (evaluation, both
    // integrators, step end and its own conditional rebuild node) on stream
    // s, which is being captured into a larger graph
    virtual void record_step(cudaStream_t s) = 0;
    // the same step in three parts, so that a batch can run the pair kernels
    // of its FP32 systems as one launch between the rebuilds and the
    // integrators: rebuild decision and conditional rebuild | evaluation
    // (with or without this system's own pair kernel) | integrators and step end
    virtual void record_pre(cudaStream_t s) = 0;
    virtual void record_eval(cudaStream_t s, bool with_pairs) = 0;
    virtual void record_post(cudaStream_t s) = 0;
    virtual bool pair_job(PairJob* out) = 0;   // false for FP64 systems
    // the evaluation of the device-side lambda exchange: rebuild decision and
    // conditional rebuild, every evaluation kernel, and the output kernel
    // writing the energy terms to `terms` (device) and consuming the forces
    virtual void record_exchange_eval(cudaStream_t s, double* terms) = 0;
    virtual LamState* lam_state_device() = 0;
    virtual void note_batch_steps(int n) = 0;
    virtual bool overflow_pending(cudaStream_t st) = 0;
    virtual void recover(cudaStream_t st) = 0;
    virtual cudaStream_t side_stream() = 0;
    virtual void autotune(int reps, const char* cache_path, double* best_ms, int* params) = 0;
    virtual void set_theta(double theta, double p_theta) = 0;
    virtual void set_list_capacity(int tiles) = 0;
    virtual void set_list_prune(double inner) = 0;
    virtual void step_io(const double* pos_in, double* pos_out, double* vel_out, double* ext_out,
                         cudaStream_t st) = 0;
    virtual void step_io_f32(const float* pos_in, float* pos_out, float* vel_out, double* ext_out,
                             cudaStream_t st) = 0;
    virtual void lambda_state(double* lam, double* mass) = 0;
    virtual bool soft_core() const = 0;
    virtual void mc_volume_move(double pressure_bar, double dv_max, unsigned long long seed,
                                unsigned long long attempt, int* accepted, double* box_out, double* energies) = 0;
    unsigned generation = 0;   // bumped whenever device buffers are reallocated
};

struct lfe_system {
    std::unique_ptr<SystemBase> impl;
    std::string err;
};

template <typename real>
struct System final : SystemBase {
    lfe_params P{};
    int n = 0, n_u = 0, n_solv = 0, n_ucl = 0, n_cl = 0, n_pad = 0;
    std::vector<void*> allocs;
    SysView<real> S{};
    NblView<real> N{};
    // the pruned list (dynamic pruning between rebuilds, off unless an inner
    // buffer below the list buffer is set): its arrays, sized like the built
    // list's, and the pruning's work arrays
    int4* pt_tiles = nullptr;
    int* pt_jidx = nullptr;
    unsigned char* pt_masks = nullptr;
    PruneView PV{};
    double prune_skin = 0.0;      // inner buffer (nm); 0 = no pruning
    bool prune_on() const { return prune_skin > 0.0 && prune_skin < P.skin; }
    NblView<real> pruned_view() const
    {
        NblView<real> v = N;
        v.tiles = pt_tiles;
        v.jidx = pt_jidx;
        v.masks = pt_masks;
        v.ntiles_flag = FL_PTILES;
        return v;
    }
    ExclView<real> X{};
    PmeView<real> M{};
    PmeView<double> M64{};      // FP32 systems: FP64 copy of the packed charge grid (and the adjoint's FP64 pass)
    PmeView<df64> M2{};         // FP32 systems: the energy branch in df64
    bool dual = false;
    BondView<real> B{};
    DafedView D{};
    StepView<real> G{};
    ThetaView<real> T{};
    int pair_warps = 0;
    int uv_blocks = 0;
    int nsm = 148;              // multiprocessors of the device
    double const_vv = 0, const_uu = 0, const_uv = 0;
    cudaStream_t cs = nullptr, cs2 = nullptr;
    static constexpr int NBR = 5;
    cudaStream_t br[NBR] = {};   // capture branches
    cudaEvent_t ev_fork = nullptr, ev_z = nullptr, ev_q = nullptr, ev_ex = nullptr, ev_rec = nullptr, ev_built = nullptr,
                ev_uv = nullptr, ev_join[NBR] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int* h_flags = nullptr;        // pinned
    double* d_terms = nullptr;     // [LFE_NTERMS]
    double* d_fbuf = nullptr;      // [3n] staging for host force output
    double* d_pos = nullptr;       // [3n] staging for host positions
    LamState* lam_save = nullptr;
    LamState* lam0 = nullptr;      // all-zero lambda state (h_A = 0: unmixed class potentials)
    real* d_q = nullptr;           // writable views of S.q, S.sig, S.eps
    real* d_sig = nullptr;
    real* d_eps = nullptr;
    double* d_pg = nullptr;        // [15 n_u] parameter-gradient outputs (dU, d2U, basis)
    double* d_pstage = nullptr;    // [3 n_u] staged solute parameters
    std::vector<double> h_q, h_sig, h_eps;   // parameters as given (caller order)
    std::vector<int> h_solute;               // solute atoms, caller order
    std::vector<double> h_mass;
    int device = 0;

    template <class T2>
    T2* dalloc(size_t count)
    {
        void* p = nullptr;
        if (count == 0) count = 1;
        CK(cudaMalloc(&p, count * sizeof(T2)));
        CK(cudaMemset(p, 0, count * sizeof(T2)));
        allocs.push_back(p);
        return static_cast<T2*>(p);
    }
    template <class T2>
    T2* upload(const std::vector<T2>& v)
    {
        T2* d = dalloc<T2>(v.size());
        if (!v.empty()) CK(cudaMemcpy(d, v.data(), v.size() * sizeof(T2), cudaMemcpyHostToDevice));
        return d;
    }
    void dfree(void* p)
    {
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) { cudaFree(p); allocs.erase(it); }
    }

    ~System() override
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (pos_exec) cudaGraphExecDestroy(pos_exec);
        if (pos_graph) cudaGraphDestroy(pos_graph);
        if (io_exec) cudaGraphExecDestroy(io_exec);
        if (io_graph) cudaGraphDestroy(io_graph);
        if (h_io_tail) cudaFreeHost(h_io_tail);
        for (void* p : allocs) cudaFree(p);
        if (h_flags) cudaFreeHost(h_flags);
        if (h_state) cudaFreeHost(h_state);
        if (cs) cudaStreamDestroy(cs);
        if (cs2) cudaStreamDestroy(cs2);
        for (int k = 0; k < NBR; ++k) {
            if (br[k]) cudaStreamDestroy(br[k]);
            if (ev_join[k]) cudaEventDestroy(ev_join[k]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_z) cudaEventDestroy(ev_z);
        if (ev_q) cudaEventDestroy(ev_q);
        if (ev_ex) cudaEventDestroy(ev_ex);
        if (ev_rec) cudaEventDestroy(ev_rec);
        if (ev_built) cudaEventDestroy(ev_built);
        if (ev_uv) cudaEventDestroy(ev_uv);
    }

    void create(const lfe_params& p, const lfe_topology& t)
    {
        P = p;
        precision = p.precision;
        CK(cudaGetDevice(&device));
        n = t.n_atoms;
        // ---------------------------------------------------- validation
        if (n <= 0) fail(LFE_ERR_ARG, "n_atoms must be positive");
        if (!t.pos || !t.charge || !t.sigma || !t.epsilon || !t.solute || !t.mass)
            fail(LFE_ERR_ARG, "per-atom arrays must not be NULL");
        for (int d = 0; d < 3; ++d) {
            if (!(p.box[d] > 0) || !std::isfinite(p.box[d])) fail(LFE_ERR_ARG, "box lengths must be positive");
            if (!(p.r_cut <= 0.5 * p.box[d])) fail(LFE_ERR_ARG, "r_cut must not exceed half of every box length");
            if (p.pme_grid[d] < 8 || p.pme_grid[d] > 128) fail(LFE_ERR_ARG, "pme_grid entries must be in [8, 128]");
            int rr[8], nr;
            if (!radix_plan(p.pme_grid[d], rr, &nr)) fail(LFE_ERR_ARG, "pme_grid entries must factor into 2, 3, 5");
        }
        if (!(p.r_cut > 0)) fail(LFE_ERR_ARG, "r_cut must be positive");
        if (p.r_switch >= p.r_cut) fail(LFE_ERR_ARG, "r_switch must be below r_cut (or negative for none)");
        if (!(p.ewald_alpha > 0)) fail(LFE_ERR_ARG, "ewald_alpha must be positive");
        if (!std::isfinite(p.lambda_temperature)) fail(LFE_ERR_ARG, "lambda_temperature must be finite");
        if (!(p.sc_alpha >= 0.0) || !std::isfinite(p.sc_alpha)) fail(LFE_ERR_ARG, "sc_alpha must be >= 0");
        if (p.sc_alpha > 0.0 && !(p.sc_power >= 1.0 && std::isfinite(p.sc_power)))
            fail(LFE_ERR_ARG, "sc_power must be >= 1 with soft-core coupling");
        if (p.pme_order != 4) fail(LFE_ERR_ARG, "pme_order must be 4");
        if (p.precision != LFE_FP32_MIXED && p.precision != LFE_FP64) fail(LFE_ERR_ARG, "unknown precision");
        if (!finite_all(t.pos, 3 * (size_t)n) || !finite_all(t.charge, n) || !finite_all(t.sigma, n) ||
            !finite_all(t.epsilon, n) || !finite_all(t.mass, n))
            fail(LFE_ERR_ARG, "non-finite per-atom input");
        for (int i = 0; i < n; ++i) {
            if (t.sigma[i] < 0 || t.epsilon[i] < 0) fail(LFE_ERR_ARG, "sigma and epsilon must be >= 0");
            if (t.mass[i] < 0) fail(LFE_ERR_ARG, "mass must be >= 0");
        }
        auto chk_idx = [&](const int* a, long cnt, const char* what) {
            if (cnt > 0 && !a) fail(LFE_ERR_ARG, std::string(what) + " is NULL");
            for (long k = 0; k < cnt; ++k)
                if (a[k] < 0 || a[k] >= n) fail(LFE_ERR_ARG, std::string(what) + " index out of range");
        };
        chk_idx(t.excl, 2L * t.n_excl, "excl");
        chk_idx(t.pairs14, 2L * t.n_14, "pairs14");
        chk_idx(t.water_OHH, 3L * t.n_waters, "water_OHH");
        chk_idx(t.constraints, 2L * t.n_constraints, "constraints");
        chk_idx(t.bonds, 2L * t.n_bonds, "bonds");
        chk_idx(t.angles, 3L * t.n_angles, "angles");
        chk_idx(t.torsions, 4L * t.n_torsions, "torsions");
        if (t.n_excl < 0 || t.n_14 < 0 || t.n_waters < 0 || t.n_constraints < 0 || t.n_bonds < 0 ||
            t.n_angles < 0 || t.n_torsions < 0)
            fail(LFE_ERR_ARG, "negative list length");
        for (int e = 0; e < t.n_excl; ++e)
            if (t.excl[2 * e] == t.excl[2 * e + 1]) fail(LFE_ERR_ARG, "an exclusion pairs an atom with itself");

        // --------------------------------------------------- atom lists
        std::vector<int> sl, vl;
        for (int i = 0; i < n; ++i) (t.solute[i] ? sl : vl).push_back(i);
        n_u = (int)sl.size();
        n_solv = (int)vl.size();
        n_ucl = (n_u + 31) / 32;
        // column sort: edge near (32 / rho)^(1/3) so that 32-atom clusters are
        // close to cubic; every column may end with one padded cluster
        const double Vbox = p.box[0] * p.box[1] * p.box[2];
        const double rho_s = std::max(1.0, n_solv / Vbox);
        const double col_edge = std::cbrt(32.0 / rho_s);
        N.ncx = std::max(1, std::min(1024, (int)std::lround(p.box[0] / col_edge)));
        N.ncy = std::max(1, std::min(1024, (int)std::lround(p.box[1] / col_edge)));
        N.ncols = N.ncx * N.ncy;
        N.cinvx = (real)(N.ncx / p.box[0]);
        N.cinvy = (real)(N.ncy / p.box[1]);
        n_cl = n_ucl + (n_solv + 31) / 32 + (n_solv > 0 ? N.ncols : 0);
        n_pad = 32 * n_cl;
        N.n_cl_max = n_cl;

        // ---------------------------------------------- per-atom buffers
        std::vector<R4<real>> hx(n), hv(n);
        std::vector<real> hq(n), hs(n), he(n), hw(n);
        std::vector<unsigned char> hsol(n);
        h_mass.assign(t.mass, t.mass + n);
        for (int i = 0; i < n; ++i) {
            hx[i] = R4<real>{(real)t.pos[3 * i], (real)t.pos[3 * i + 1], (real)t.pos[3 * i + 2], (real)0};
            hv[i] = R4<real>{0, 0, 0, 0};
            hq[i] = (real)t.charge[i];
            hs[i] = (real)t.sigma[i];
            he[i] = (real)t.epsilon[i];
            hw[i] = t.mass[i] > 0 ? (real)(1.0 / t.mass[i]) : (real)0;
            hsol[i] = t.solute[i] ? 1 : 0;
        }
        S.n = n; S.n_pad = n_pad; S.n_cl = n_cl; S.n_ucl = n_ucl; S.n_u = n_u; S.n_solv = n_solv;
        for (int d = 0; d < 3; ++d) {
            S.L[d] = (real)p.box[d];
            S.invL[d] = (real)(1.0 / p.box[d]);
        }
        S.rc2 = (real)(p.r_cut * p.r_cut);
        if (p.r_switch >= 0) {
            S.rsw = (real)p.r_switch;
            S.sw_inv_w = (real)(1.0 / (p.r_cut - p.r_switch));
        } else {
            S.rsw = (real)p.r_cut;
            S.sw_inv_w = (real)0;
        }
        S.alpha = (real)p.ewald_alpha;
        S.two_a_sqrtpi = (real)(2.0 * p.ewald_alpha / std::sqrt(PI));
        S.sc_alpha = p.sc_alpha;
        S.sc_power = p.sc_alpha > 0.0 ? p.sc_power : 1.0;
        S.x = upload(hx);
        S.v = upload(hv);
        S.xref = dalloc<R4<real>>(n);
        S.xpr = dalloc<R4<real>>(n);
        CK(cudaMemset(S.xpr, 0, sizeof(R4<real>) * n));
        S.invm = upload(hw);
        d_q = upload(hq);
        d_sig = upload(hs);
        d_eps = upload(he);
        S.q = d_q;
        S.sig = d_sig;
        S.eps = d_eps;
        h_q.assign(t.charge, t.charge + n);
        h_sig.assign(t.sigma, t.sigma + n);
        h_eps.assign(t.epsilon, t.epsilon + n);
        h_solute = sl;
        d_pg = dalloc<double>(15 * (size_t)std::max(1, n_u));
        d_pstage = dalloc<double>(3 * (size_t)std::max(1, n_u));
        S.sol = upload(hsol);
        S.solute_list = upload(sl);
        S.solv_list = upload(vl);
        S.xq = dalloc<R4<real>>(n_pad);
        S.lj = dalloc<R2<real>>(n_pad);
        S.perm = dalloc<int>(n_pad);
        S.iperm = dalloc<int>(n);
        S.F = dalloc<long long>(3 * (size_t)n_pad);
        S.Fa = dalloc<long long>(3 * (size_t)n);
        S.E = dalloc<long long>(E_N);
        S.flags = dalloc<int>(FL_N);
        S.lam = dalloc<LamState>(1);
        CK(cudaMallocHost(&h_flags, sizeof(int) * FL_N));
        d_terms = dalloc<double>(LFE_NTERMS);
        d_fbuf = dalloc<double>(3 * (size_t)n);
        d_pos = dalloc<double>(3 * (size_t)n);

        // ---------------------------------------------------- neighbours
        double skin = p.skin > 0 ? p.skin : 0.1;
        skin_auto = !(p.skin > 0);
        P.skin = skin;
        const double V = p.box[0] * p.box[1] * p.box[2];
        N.col_of = dalloc<int>(n_solv);
        N.col_cnt = dalloc<int>(N.ncols);
        N.col_start = dalloc<int>(N.ncols + 1);
        N.col_fill = dalloc<int>(N.ncols);
        N.col_cl = dalloc<int>(N.ncols + 1);
        N.tmp = dalloc<int>(n_solv);
        N.tmp2 = dalloc<int>(n_solv);
        N.n_cl_solv = dalloc<int>(1);
        N.bbc = dalloc<R4<float>>(n_cl);
        N.bbh = dalloc<R4<float>>(n_cl);
        N.bbc8 = dalloc<R4<float>>(4 * (size_t)n_cl);
        N.bbh8 = dalloc<R4<float>>(4 * (size_t)n_cl);
        N.tile_cnt = dalloc<int>(27 * 4 * (size_t)n_cl);
        N.tile_tot = dalloc<int>(4 * (size_t)n_cl);
        N.tile_off = dalloc<int>(4 * (size_t)n_cl + 1);
        N.ntiles_flag = FL_NTILES;
        PV.cnt = dalloc<int>(4 * (size_t)n_cl);
        PV.off = dalloc<int>(4 * (size_t)n_cl + 1);
        CK(cudaMemset(PV.cnt, 0, sizeof(int) * 4 * (size_t)n_cl));
        N.cap = 1024;
        N.tiles = dalloc<int4>(N.cap);
        N.jidx = dalloc<int>((size_t)N.cap * 32);
        N.masks = dalloc<unsigned char>((size_t)N.cap * 32);
        pt_tiles = dalloc<int4>(N.cap);
        pt_jidx = dalloc<int>((size_t)N.cap * 32);
        pt_masks = dalloc<unsigned char>((size_t)N.cap * 32);
        PV.kb = dalloc<unsigned>(N.cap);
        PV.base = dalloc<int>(N.cap);
        N.stage_cap = N.cap;
        N.stage_hdr = dalloc<int4>(N.stage_cap);
        N.stage_j = dalloc<int>((size_t)N.stage_cap * 32);
        grow_uv(std::max(1, n_ucl * 512), std::max(1024, n_u * 2048));
        N.cut2 = (float)((p.r_cut + skin) * (p.r_cut + skin));
        N.skin_half2 = (float)(0.25 * skin * skin);
        {
            std::vector<int> cnt(n + 1, 0), lst(2 * (size_t)t.n_excl);
            for (int e = 0; e < t.n_excl; ++e) { cnt[t.excl[2 * e] + 1]++; cnt[t.excl[2 * e + 1] + 1]++; }
            for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
            std::vector<int> fillv(n, 0);
            for (int e = 0; e < t.n_excl; ++e) {
                int a = t.excl[2 * e], b = t.excl[2 * e + 1];
                lst[cnt[a] + fillv[a]++] = b;
                lst[cnt[b] + fillv[b]++] = a;
            }
            N.ex_start = upload(cnt);
            N.ex_list = upload(lst);
            // molecule id = connected component of the exclusion graph
            std::vector<int> parent(n);
            for (int i = 0; i < n; ++i) parent[i] = i;
            std::function<int(int)> find = [&](int i) {
                while (parent[i] != i) { parent[i] = parent[parent[i]]; i = parent[i]; }
                return i;
            };
            for (int e = 0; e < t.n_excl; ++e) {
                const int ra = find(t.excl[2 * e]), rb = find(t.excl[2 * e + 1]);
                if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
            }
            std::vector<int> mol(n);
            for (int i = 0; i < n; ++i) mol[i] = find(i);
            N.mol = upload(mol);
            h_mol = mol;
            // each atom's exclusion partners as a bitmask over its molecule's
            // atom indices, for molecules within 63 consecutive indices of
            // their lowest atom (the mask build tests a partner with one bit)
            std::vector<int> span(n, 0);
            for (int i = 0; i < n; ++i) span[mol[i]] = std::max(span[mol[i]], i - mol[i]);
            std::vector<unsigned long long> exm(n, 0ull);
            for (int i = 0; i < n; ++i) {
                if (span[mol[i]] > 62) {
                    exm[i] = 1ull << 63;
                    continue;
                }
                for (int k = cnt[i]; k < cnt[i + 1]; ++k) exm[i] |= 1ull << (lst[k] - mol[i]);
            }
            N.exm = upload(exm);
        }

        // ---------------------------------------------------- exclusions
        {
            std::vector<int2> ex(t.n_excl), e14(t.n_14);
            std::vector<R2<real>> s14(t.n_14);
            std::vector<R2<double>> s14d(t.n_14);
            for (int e = 0; e < t.n_excl; ++e) ex[e] = make_int2(t.excl[2 * e], t.excl[2 * e + 1]);
            for (int e = 0; e < t.n_14; ++e) {
                e14[e] = make_int2(t.pairs14[2 * e], t.pairs14[2 * e + 1]);
                s14[e] = R2<real>{(real)t.scale14[2 * e], (real)t.scale14[2 * e + 1]};
                s14d[e] = R2<double>{t.scale14[2 * e], t.scale14[2 * e + 1]};
            }
            X.n_excl = t.n_excl;
            X.n14 = t.n_14;
            X.excl = upload(ex);
            X.p14 = upload(e14);
            X.s14 = upload(s14);
            X.s14d = upload(s14d);
            X.ex_start = N.ex_start;
            X.ex_list = N.ex_list;
            std::vector<int> cnt(n + 1, 0), lst(2 * (size_t)t.n_14), fillv(n, 0);
            std::vector<R2<real>> ls(2 * (size_t)t.n_14);
            for (int e = 0; e < t.n_14; ++e) { cnt[t.pairs14[2 * e] + 1]++; cnt[t.pairs14[2 * e + 1] + 1]++; }
            for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
            for (int e = 0; e < t.n_14; ++e) {
                const int a = t.pairs14[2 * e], b = t.pairs14[2 * e + 1];
                const int pa = cnt[a] + fillv[a]++, pb = cnt[b] + fillv[b]++;
                lst[pa] = b;
                lst[pb] = a;
                ls[pa] = s14[e];
                ls[pb] = s14[e];
            }
            X.p14_start = upload(cnt);
            X.p14_list = upload(lst);
            X.p14_s = upload(ls);
        }

        // ----------------------------------------------------------- PME
        {
            dual = (p.precision == LFE_FP32_MIXED);
            M.KK = 1;
            double sv = 0, su = 0;
            for (int i = 0; i < n; ++i) (t.solute[i] ? su : sv) += t.charge[i] * t.charge[i];
            const double sc = (su > 0 && sv > 0) ? std::sqrt(sv / su) : 1.0;
            const double qu_scale = std::exp2(std::round(std::log2(std::max(1.0, sc))));
            for (int d = 0; d < 3; ++d) {
                const int K = p.pme_grid[d];
                M.K[d] = K;
                M.KK *= K;
                M.kscale[d] = (real)(K / p.box[d]);
                M.kscale64[d] = K / p.box[d];
                radix_plan(K, M.rad[d], &M.nrad[d]);
                // |b(m)|^2 with the order-4 spline values M4(1) = 1/6, M4(2) = 2/3, M4(3) = 1/6
                std::vector<double> gf(K), ms(K);
                std::vector<R2<double>> tw(K);
                pme_axis_tables(K, p.box[d], gf, ms);
                for (int m = 0; m < K; ++m) tw[m] = R2<double>{std::cos(2.0 * PI * m / K), std::sin(2.0 * PI * m / K)};
                std::vector<real> gfr(K), msr(K);
                std::vector<R2<real>> twr(K);
                for (int m = 0; m < K; ++m) {
                    gfr[m] = (real)gf[m];
                    msr[m] = (real)ms[m];
                    twr[m] = R2<real>{(real)tw[m].x, (real)tw[m].y};
                }
                M.gfac[d] = upload(gfr);
                M.msq[d] = upload(msr);
                M.tw[d] = upload(twr);
                if (dual) {
                    M64.K[d] = K;
                    M64.kscale[d] = K / p.box[d];
                    M64.kscale64[d] = K / p.box[d];
                    M64.nrad[d] = M.nrad[d];
                    for (int r = 0; r < 8; ++r) M64.rad[d][r] = M.rad[d][r];
                    M64.gfac[d] = upload(gf);
                    M64.msq[d] = upload(ms);
                    M64.tw[d] = upload(tw);
                    std::vector<df64> gf2(K), ms2(K);
                    std::vector<R2<df64>> tw2(K);
                    for (int m = 0; m < K; ++m) {
                        gf2[m] = df64(gf[m]);
                        ms2[m] = df64(ms[m]);
                        tw2[m] = R2<df64>{df64(tw[m].x), df64(tw[m].y)};
                    }
                    M2.K[d] = K;
                    M2.kscale[d] = df64(K / p.box[d]);
                    M2.kscale64[d] = K / p.box[d];
                    M2.nrad[d] = M.nrad[d];
                    for (int r = 0; r < 8; ++r) M2.rad[d][r] = M.rad[d][r];
                    M2.gfac[d] = upload(gf2);
                    M2.msq[d] = upload(ms2);
                    M2.tw[d] = upload(tw2);
                }
            }
            M.conv_pre = (real)(KE / (PI * V));
            M.qu_scale = (real)qu_scale;
            M.Qfix = dalloc<long long>(2 * (size_t)M.KK);
            M.Z = dalloc<R2<real>>(M.KK);
            M.phi_u = dalloc<real>(std::max(1, n_u));
            M.Zraw64 = nullptr;
            if (dual) {
                M64.KK = M.KK;
                M64.conv_pre = KE / (PI * V);
                M64.qu_scale = qu_scale;
                M64.Qfix = nullptr;
                M64.Z = dalloc<R2<double>>(M.KK);
                M64.phi_u = nullptr;
                M64.Zraw64 = nullptr;
                M.Zraw64 = M64.Z;
                M2.KK = M.KK;
                M2.conv_pre = df64(KE / (PI * V));
                M2.qu_scale = df64(qu_scale);
                M2.Qfix = nullptr;
                M2.Z = dalloc<R2<df64>>(M.KK);
                M2.phi_u = nullptr;
                M2.Zraw64 = nullptr;
                M2.Zin64 = M64.Z;
                M2.Qfix = M.Qfix;   // read directly by the captured step (FFT_FROM_FIX_KEEP)
            }
            const int Kmax = std::max(M.K[0], std::max(M.K[1], M.K[2]));
            if (fft_smem<real>(Kmax) > 48 * 1024 || (dual && fft_smem<double>(Kmax) > 48 * 1024))
                fail(LFE_ERR_ARG, "PME grid too large for the FFT tile");
            column_groups();
        }

        // ----------------------------------------------- constant energies
        constant_energies();

        // --------------------------------------------------------- bonded
        {
            std::vector<int2> bi(t.n_bonds);
            std::vector<R2<real>> bp(t.n_bonds);
            for (int e = 0; e < t.n_bonds; ++e) {
                bi[e] = make_int2(t.bonds[2 * e], t.bonds[2 * e + 1]);
                bp[e] = R2<real>{(real)t.bond_par[2 * e], (real)t.bond_par[2 * e + 1]};
            }
            std::vector<int4> ai(t.n_angles);
            std::vector<R2<real>> ap(t.n_angles);
            for (int e = 0; e < t.n_angles; ++e) {
                ai[e] = make_int4(t.angles[3 * e], t.angles[3 * e + 1], t.angles[3 * e + 2], 0);
                ap[e] = R2<real>{(real)t.angle_par[2 * e], (real)t.angle_par[2 * e + 1]};
            }
            std::vector<int4> ti(t.n_torsions);
            std::vector<R4<real>> tp(t.n_torsions);
            for (int e = 0; e < t.n_torsions; ++e) {
                ti[e] = make_int4(t.torsions[4 * e], t.torsions[4 * e + 1], t.torsions[4 * e + 2], t.torsions[4 * e + 3]);
                tp[e] = R4<real>{(real)t.torsion_par[3 * e], (real)t.torsion_par[3 * e + 1],
                                 (real)t.torsion_par[3 * e + 2], (real)0};
            }
            B.nb = t.n_bonds; B.na = t.n_angles; B.nt = t.n_torsions;
            B.b = upload(bi); B.bp = upload(bp);
            B.a = upload(ai); B.ap = upload(ap);
            B.t = upload(ti); B.tp = upload(tp);
        }

        // ---------------------------------------------- constraint groups
        {
            std::vector<int> owner(n, -1);
            std::vector<Group> groups;
            for (int w = 0; w < t.n_waters; ++w) {
                Group g{};
                for (int k = 0; k < 3; ++k) g.atom[k] = t.water_OHH[3 * w + k];
                g.natom = 3;
                g.ncons = 3;
                g.ci[0] = 0; g.cj[0] = 1; g.len[0] = (float)t.water_rOH;
                g.ci[1] = 0; g.cj[1] = 2; g.len[1] = (float)t.water_rOH;
                g.ci[2] = 1; g.cj[2] = 2; g.len[2] = (float)t.water_rHH;
                g.kind = GROUP_WATER;
                for (int k = 0; k < 3; ++k) {
                    if (owner[g.atom[k]] >= 0) fail(LFE_ERR_ARG, "an atom belongs to two rigid waters");
                    owner[g.atom[k]] = (int)groups.size();
                }
                groups.push_back(g);
            }
            // star groups: every constraint's first atom is the centre
            std::vector<int> centre_group(n, -1);
            for (int c = 0; c < t.n_constraints; ++c) {
                const int a = t.constraints[2 * c], b = t.constraints[2 * c + 1];
                if (!(t.constraint_len[c] > 0)) fail(LFE_ERR_ARG, "constraint lengths must be positive");
                int gi = centre_group[a];
                if (gi < 0) {
                    if (owner[a] >= 0) fail(LFE_ERR_ARG, "constraint centre already in another group");
                    Group g{};
                    g.atom[0] = a;
                    g.natom = 1;
                    g.ncons = 0;
                    g.kind = GROUP_STAR;
                    gi = (int)groups.size();
                    groups.push_back(g);
                    centre_group[a] = gi;
                    owner[a] = gi;
                }
                Group& g = groups[gi];
                if (g.natom >= 4 || g.ncons >= 3) fail(LFE_ERR_ARG, "more than 3 constraints share one centre");
                if (owner[b] >= 0) fail(LFE_ERR_ARG, "a constrained atom belongs to two groups");
                owner[b] = gi;
                g.atom[g.natom] = b;
                g.ci[g.ncons] = 0;
                g.cj[g.ncons] = g.natom;
                g.len[g.ncons] = (float)t.constraint_len[c];
                g.natom++;
                g.ncons++;
            }
            for (int i = 0; i < n; ++i)
                if (owner[i] < 0) {
                    Group g{};
                    g.atom[0] = i;
                    g.natom = 1;
                    g.kind = GROUP_SINGLE;
                    owner[i] = (int)groups.size();
                    groups.push_back(g);
                }
            // same-shape groups next to each other keep warps on one code path
            std::stable_sort(groups.begin(), groups.end(), [](const Group& x, const Group& y) {
                return x.kind != y.kind ? x.kind < y.kind : x.natom < y.natom;
            });
            G.groups = upload(groups);
            G.n_groups = (int)groups.size();
        }
        G.noise = dalloc<real>(3 * (size_t)n);
        T.pre = dalloc<ThetaPre>(1);
        T.ti_sum = dalloc<double>(LFE_TI_BINS);
        T.ti_cnt = dalloc<unsigned long long>(LFE_TI_BINS);
        G.dt = (real)p.dt;
        G.a_fric = (real)std::exp(-p.friction * p.dt);
        G.kT = (real)(KB * p.temperature);
        G.key = make_uint2((unsigned)(p.seed & 0xffffffffull), (unsigned)(p.seed >> 32));
        G.skin_half2 = (real)(0.25 * skin * skin);

        // ---------------------------------------------------- theta/OPES
        T.m = p.lambda_mass;
        T.dt = p.dt;
        T.a_fric = std::exp(-p.lambda_friction * p.dt);
        T.kT = KB * (p.lambda_temperature > 0 ? p.lambda_temperature : p.temperature);
        T.th = ext_th;
        T.tc = ext_const(T.th, T.m, T.kT, T.a_fric);
        T.stride = p.opes_stride;
        T.max_k = p.opes_max_kernels > 0 ? p.opes_max_kernels : 1024;
        T.sigma = p.opes_sigma > 0 ? p.opes_sigma : 0.1;
        T.beta = 1.0 / (KB * (p.temperature > 0 ? p.temperature : 298.0));
        const double dE[2] = {p.opes_dE_std, p.opes_dE_exp};
        for (int b = 0; b < 2; ++b) {
            T.on[b] = dE[b] > 0 && p.opes_stride > 0;
            if (T.on[b]) {
                const double gam = T.beta * dE[b];
                if (gam <= 1.0) fail(LFE_ERR_ARG, "OPES barrier must exceed k_B T");
                T.nu[b] = b == 0 ? 1.0 - 1.0 / gam : gam - 1.0;
                T.epsr[b] = std::exp(-T.beta * dE[b] / T.nu[b]);
            } else {
                T.nu[b] = 1.0;
                T.epsr[b] = 1.0;
            }
        }
        T.centre = dalloc<double>(2 * (size_t)T.max_k);
        T.weight = dalloc<double>(2 * (size_t)T.max_k);
        T.S = dalloc<double>(2 * (size_t)T.max_k);
        T.st = dalloc<OpesState>(1);
        T.key = G.key;
        T.const_vv = const_vv;
        T.const_uu = const_uu;
        T.const_uv = const_uv;

        // initial lambda state from theta0
        {
            LamState L{};
            double th = p.theta0 - 2.0 * std::floor(p.theta0 / 2.0);
            L.theta = th;
            L.dlam_dtheta = th <= 1.0 ? 1.0 : -1.0;
            L.lambda = th <= 1.0 ? th : 2.0 - th;
            CK(cudaMemcpy(S.lam, &L, sizeof(L), cudaMemcpyHostToDevice));
            launch_set_lambda(S, L.lambda, nullptr);
            lam_save = dalloc<LamState>(1);
            lam0 = dalloc<LamState>(1);
        }
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
        pair_warps = nsm * 4 * pairs_blocks_per_sm<real>();   // one resident wave of 4-warp blocks
        // half a block per multiprocessor for the FP64 solute-solvent energies
        // (a few thousand pairs): 32 batched replicas step 3 % faster than with
        // two per multiprocessor, a single system alike (the autotuner checks)
        uv_blocks = std::max(1, nsm / 2);
        N.n_sm = nsm;
        {
            const char* ev = std::getenv("LFE_EAGER_STEPS");
            eager = ev && ev[0] == '1';
        }
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking));
        // the pair branch (the step's critical path: rebuild, pair kernel,
        // then the integrator) gets the higher priority: its blocks are
        // scheduled ahead of the other branches', which end with slack (the
        // captured step graph is instantiated with per-node priorities;
        // octanol box, 4 pair blocks per SM: 118.6 us per step against 122.2
        // with the PME branches first and 118.2 with equal priorities)
        int prio_lo = 0, prio_hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        for (int k = 0; k < NBR; ++k) {
            CK(cudaStreamCreateWithPriority(&br[k], cudaStreamNonBlocking, k == 0 ? prio_hi : prio_lo));
            CK(cudaEventCreateWithFlags(&ev_join[k], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_z, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_q, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_ex, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_rec, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_built, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_uv, cudaEventDisableTiming));
        build_neighbors(nullptr);
        CK(cudaStreamSynchronize(nullptr));
        {
            // mass-weighted zero velocities; theta at rest
        }
    }

    // Column groups of the axis-0 pass of the plane/column transform: chunks
    // of consecutive k2 at one k1, each with the partner columns (-k1, -k2)
    // of its columns, so that the convolution's (m, -m) pairs stay inside
    // one block.  The plane kernels are used when a plane and a group fit in
    // shared memory.
    void column_groups()
    {
        const int K1 = M.K[1], K2 = M.K[2], K12 = K1 * K2;
        auto partner = [&](int c) { const int k1 = c / K2, k2 = c % K2; return ((K1 - k1) % K1) * K2 + (K2 - k2) % K2; };
        int optin = 0;
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
        // CW consecutive columns per chunk: 8 in FP32; 4 in FP64, whose
        // scarce units want more, smaller blocks
        auto build = [&](auto& V, int CW) {
            std::vector<char> seen(K12, 0);
            std::vector<int> start(1, 0), cols, part;
            int gmax = 0;
            for (int k1 = 0; k1 < K1; ++k1)
                for (int c0 = 0; c0 < K2; c0 += CW) {
                    std::vector<int> g;
                    for (int k2 = c0; k2 < std::min(c0 + CW, K2); ++k2) {
                        const int c = k1 * K2 + k2;
                        if (seen[c]) continue;
                        seen[c] = 1;
                        g.push_back(c);
                        const int pc = partner(c);
                        if (!seen[pc]) { seen[pc] = 1; g.push_back(pc); }
                    }
                    if (g.empty()) continue;
                    std::sort(g.begin(), g.end());
                    for (int c : g) {
                        cols.push_back(c);
                        part.push_back((int)(std::lower_bound(g.begin(), g.end(), partner(c)) - g.begin()));
                    }
                    start.push_back((int)cols.size());
                    gmax = std::max(gmax, (int)g.size());
                }
            V.ngroups = (int)start.size() - 1;
            V.cg_max = gmax;
            V.cg_start = upload(start);
            V.cg_col = upload(cols);
            V.cg_part = upload(part);
            V.planes = (planes_smem(V) + 1024 <= (size_t)optin && columns_smem(V) + 1024 <= (size_t)optin) ? 1 : 0;
        };
        build(M, sizeof(real) == 8 ? 4 : 8);
        if (dual) build(M64, 4);
        if (dual) build(M2, 4);
        if (dual && !(M64.planes && M2.planes)) M.planes = M64.planes = M2.planes = 0;   // one transform layout
        if (M.planes) {
            planes_setup(M);
            if (dual) planes_setup(M64);
            if (dual) energy_columns_setup(M2);
            CK(cudaGetLastError());
        }
    }

    // self and neutralising-background energies of each class (they depend
    // on the charges only)
    // influence-function factor exp(-pi^2 m^2 / alpha^2) |b(m)|^2 and m^2 of
    // one axis (m = k / L for k <= K/2, (k - K) / L above) with the order-4
    // B-spline moduli |b(m)|^-2 = |sum_{k=0..2} M4(k+1) e^{2 pi i m k / K}|^2
    void pme_axis_tables(int K, double L, std::vector<double>& gf, std::vector<double>& ms) const
    {
        for (int m = 0; m < K; ++m) {
            double re = 0, im = 0;
            const double mk[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
            for (int k = 0; k < 3; ++k) {
                re += mk[k] * std::cos(2.0 * PI * m * k / K);
                im += mk[k] * std::sin(2.0 * PI * m * k / K);
            }
            const double b2 = 1.0 / (re * re + im * im);
            const int mm = (m <= K / 2) ? m : m - K;
            const double mr = mm / L;
            gf[m] = std::exp(-PI * PI * mr * mr / (P.ewald_alpha * P.ewald_alpha)) * b2;
            ms[m] = mr * mr;
        }
    }

    void constant_energies()
    {
        std::vector<unsigned char> is_u(n, 0);
        for (int a : h_solute) is_u[a] = 1;
        double s2[2] = {0, 0}, Q[2] = {0, 0};
        for (int i = 0; i < n; ++i) {
            const int c = is_u[i];
            s2[c] += h_q[i] * h_q[i];
            Q[c] += h_q[i];
        }
        const double a = P.ewald_alpha, V = P.box[0] * P.box[1] * P.box[2];
        const double self_v = -KE * a / std::sqrt(PI) * s2[0], self_u = -KE * a / std::sqrt(PI) * s2[1];
        const double pre = -KE * PI / (2.0 * V * a * a);
        const_vv = self_v + pre * Q[0] * Q[0];
        const_uu = self_u + pre * Q[1] * Q[1];
        const_uv = pre * 2.0 * Q[0] * Q[1];
        T.const_vv = const_vv;
        T.const_uu = const_uu;
        T.const_uv = const_uv;
    }

    void check_flags(cudaStream_t st)
    {
        CK(cudaMemcpyAsync(h_flags, S.flags, sizeof(int) * FL_N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const int e = h_flags[FL_ERROR];
        if (e) {
            int zero = 0;
            CK(cudaMemcpy(S.flags + FL_ERROR, &zero, sizeof(int), cudaMemcpyHostToDevice));
            if (e & ERRB_OVERFLOW) fail(LFE_ERR_OVERFLOW, "neighbour-list capacity exceeded");
            if (e & ERRB_NONFINITE) fail(LFE_ERR_NONFINITE, "non-finite force, energy or position");
            if (e & ERRB_CONSTRAINT) fail(LFE_ERR_NONFINITE, "constraint iteration did not converge");
        }
    }

    void invalidate_graph()
    {
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
    }

    // tile list of `need` tiles and a staging list of at least `need_stage`
    // (the staging list holds the same tiles before they are placed)
    void grow_tiles(int need, int need_stage = 0)
    {
        ++generation;
        dfree(N.tiles);
        dfree(N.jidx);
        dfree(N.masks);
        dfree(N.stage_hdr);
        dfree(N.stage_j);
        dfree(pt_tiles);
        dfree(pt_jidx);
        dfree(pt_masks);
        dfree(PV.kb);
        dfree(PV.base);
        N.cap = need + 256;
        N.tiles = dalloc<int4>(N.cap);
        N.jidx = dalloc<int>((size_t)N.cap * 32);
        N.masks = dalloc<unsigned char>((size_t)N.cap * 32);
        pt_tiles = dalloc<int4>(N.cap);
        pt_jidx = dalloc<int>((size_t)N.cap * 32);
        pt_masks = dalloc<unsigned char>((size_t)N.cap * 32);
        PV.kb = dalloc<unsigned>(N.cap);
        PV.base = dalloc<int>(N.cap);
        N.stage_cap = std::max(N.cap, need_stage + 256);
        N.stage_hdr = dalloc<int4>(N.stage_cap);
        N.stage_j = dalloc<int>((size_t)N.stage_cap * 32);
        invalidate_graph();
    }

    // the solute-solvent pair list: tiles of solute sub-clusters it can take
    // (counts and offsets) and pairs it can hold
    void grow_uv(int tiles, int pairs)
    {
        ++generation;
        dfree(N.uv_cnt);
        dfree(N.uv_off);
        dfree(N.uvp);
        N.uv_tiles_max = tiles;
        N.uv_cnt = dalloc<int>(N.uv_tiles_max);
        N.uv_off = dalloc<int>(N.uv_tiles_max + 1);
        N.uv_cap = pairs;
        N.uvp = dalloc<int4>(N.uv_cap);
        invalidate_graph();
    }

    // a build that wanted more room than some list has (flags as last read)
    bool list_short() const
    {
        return h_flags[FL_NTILES] > N.cap || h_flags[FL_NSTAGE] > N.stage_cap || h_flags[FL_NUVT] > N.uv_tiles_max ||
               h_flags[FL_NUV] > N.uv_cap;
    }

    // growth after an overflow seen in the flags: every list that ran short
    // is doubled past what the build asked for (the tile list at least
    // doubles).  A build whose solute-solvent tiles did not all fit counted
    // the pairs of the first ones only, so the pair list is then sized for
    // the bound of 256 pairs per tile.
    void grow_for_flags()
    {
        const int uvt = h_flags[FL_NUVT], uvp = h_flags[FL_NUV];
        if (uvt > N.uv_tiles_max || uvp > N.uv_cap) {
            const long long pairs = std::max<long long>(2LL * uvp, uvt > N.uv_tiles_max ? 256LL * uvt : 0LL);
            grow_uv(std::max(N.uv_tiles_max, 2 * uvt), (int)std::max<long long>(N.uv_cap, pairs));
        }
        grow_tiles(std::max(h_flags[FL_NTILES], N.cap) * 2, 2 * h_flags[FL_NSTAGE]);
    }

    // a rebuild left pending by the last step (steps rebuild at their start)
    // is done before anything outside the step graph reads the list
    void settle_rebuild(cudaStream_t st)
    {
        CK(cudaMemcpyAsync(h_flags, S.flags, sizeof(int) * FL_N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (!h_flags[FL_REBUILD] || (h_flags[FL_ERROR] & ERRB_OVERFLOW)) return;
        const int v[2] = {0, h_flags[FL_NREBUILD] + 1};
        CK(cudaMemcpy(S.flags + FL_REBUILD, &v[0], sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(S.flags + FL_NREBUILD, &v[1], sizeof(int), cudaMemcpyHostToDevice));
        build_neighbors(st);
    }

    void build_neighbors(cudaStream_t st) override
    {
        launch_build_nbl(S, N, st);
        CK(cudaMemcpyAsync(h_flags, S.flags, sizeof(int) * FL_N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (list_short()) {
            grow_for_flags();
            int zero = 0;
            CK(cudaMemcpy(S.flags + FL_ERROR, &zero, sizeof(int), cudaMemcpyHostToDevice));
            launch_build_nbl(S, N, st);
            check_flags(st);
        }
        CK(cudaGetLastError());
    }

    // New positions go through a small captured graph: assign, refresh the
    // sorted copy, and rebuild the neighbour list only when an atom lies more
    // than skin/2 from where the list was built (a device-side decision, so
    // the call does not wait for the device).  A capacity overflow in that
    // rebuild is settled by the next call that synchronises.
    cudaGraph_t pos_graph = nullptr;
    cudaGraphExec_t pos_exec = nullptr;
    unsigned pos_gen = ~0u;
    bool pos_pending = false;

    void capture_pos_graph()
    {
        if (pos_exec) { cudaGraphExecDestroy(pos_exec); pos_exec = nullptr; }
        if (pos_graph) { cudaGraphDestroy(pos_graph); pos_graph = nullptr; }
        cudaStream_t s0 = cs;
        CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
        cudaStreamCaptureStatus status;
        cudaGraph_t g = nullptr;
        CK(cudaStreamGetCaptureInfo(s0, &status, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        launch_assign_moved(S, d_pos, G.skin_half2, G.prune_half2, s0);
        launch_rebuild_cond(S, h, s0);
        add_cond_build(s0, h);
        CK(cudaStreamEndCapture(s0, &pos_graph));
        CK(cudaGraphInstantiate(&pos_exec, pos_graph, 0));
        pos_gen = generation;
    }

    // after set_positions: a rebuild that ran out of tile capacity is redone
    // with more capacity (synchronises)
    void settle_positions(cudaStream_t st)
    {
        if (!pos_pending) return;
        pos_pending = false;
        CK(cudaMemcpyAsync(h_flags, S.flags, sizeof(int) * FL_N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (h_flags[FL_ERROR] & ERRB_OVERFLOW) {
            int clr[2] = {0, 0};
            CK(cudaMemcpy(S.flags, clr, sizeof(clr), cudaMemcpyHostToDevice));
            grow_for_flags();
            build_neighbors(st);
        }
    }

    void set_positions(const double* pos, int on_device, cudaStream_t st) override
    {
        if (!pos) fail(LFE_ERR_ARG, "pos is NULL");
        if (!on_device && !finite_all(pos, 3 * (size_t)n)) fail(LFE_ERR_ARG, "non-finite position");
        CK(cudaMemcpyAsync(d_pos, pos, sizeof(double) * 3 * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           st));
        if (!pos_exec || pos_gen != generation) capture_pos_graph();
        CK(cudaGraphLaunch(pos_exec, st));
        pos_pending = true;
    }

    void set_integrator(double dt, double friction, double temperature) override
    {
        if (!(dt > 0) || !(friction >= 0) || !(temperature >= 0) || !std::isfinite(dt) || !std::isfinite(friction) ||
            !std::isfinite(temperature))
            fail(LFE_ERR_ARG, "dt must be > 0, friction and temperature >= 0");
        CK(cudaDeviceSynchronize());
        if (exec) recover_overflow(nullptr);
        P.dt = dt;
        P.friction = friction;
        P.temperature = temperature;
        G.dt = (real)dt;
        G.a_fric = (real)std::exp(-friction * dt);
        G.kT = (real)(KB * temperature);
        T.dt = dt;
        T.a_fric = std::exp(-P.lambda_friction * dt);
        T.kT = KB * (P.lambda_temperature > 0 ? P.lambda_temperature : temperature);
        D.dt = dt;
        D.a_fric = std::exp(-dafed_friction * dt);
        T.tc = ext_const(T.th, T.m, T.kT, T.a_fric);
        dafed_consts();
        invalidate_graph();
        ++generation;
    }

    void set_velocities(const double* vel) override
    {
        if (!vel) fail(LFE_ERR_ARG, "vel is NULL");
        std::vector<R4<real>> hv(n);
        for (int i = 0; i < n; ++i)
            hv[i] = R4<real>{(real)vel[3 * i], (real)vel[3 * i + 1], (real)vel[3 * i + 2], (real)0};
        CK(cudaMemcpy(S.v, hv.data(), sizeof(R4<real>) * n, cudaMemcpyHostToDevice));
    }

    // evaluations outside the step graphs run on the built list (a pruned
    // list is only cut inside recorded steps)
    void eval_kernels(cudaStream_t st) { record_eval_on(st, true, N); }

    void eval(double lam, double* forces, double* terms, int out_on_device, cudaStream_t st) override
    {
        if (!(lam >= 0.0 && lam <= 1.0)) fail(LFE_ERR_ARG, "lambda must be in [0, 1]");
        settle_positions(st);
        if (exec) recover_overflow(st);
        settle_rebuild(st);
        // the dynamics' lambda state is saved and put back: an evaluation at
        // an arbitrary lambda does not move theta
        CK(cudaMemcpyAsync(lam_save, S.lam, sizeof(LamState), cudaMemcpyDeviceToDevice, st));
        launch_set_lambda(S, lam, st);
        eval_kernels(st);
        double* fdst = forces ? (out_on_device ? forces : d_fbuf) : nullptr;
        double* tdst = terms ? (out_on_device ? terms : d_terms) : nullptr;
        launch_eval_out(S, fdst, tdst, const_vv, const_uu, const_uv, st);
        CK(cudaMemcpyAsync(S.lam, lam_save, sizeof(LamState), cudaMemcpyDeviceToDevice, st));
        CK(cudaGetLastError());
        if (!out_on_device) {
            if (forces) CK(cudaMemcpyAsync(forces, d_fbuf, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
            if (terms) CK(cudaMemcpyAsync(terms, d_terms, sizeof(double) * LFE_NTERMS, cudaMemcpyDeviceToHost, st));
        }
        check_flags(st);
    }

    // Appends to the graph being captured on st a conditional node (handle h)
    // whose body rebuilds the neighbour list; st continues after it.
    void add_cond_build(cudaStream_t st, cudaGraphConditionalHandle h)
    {
        add_cond_node(st, h, [&](cudaStream_t c) { launch_build_nbl(S, N, c); });
    }

    // a conditional node (handle h) whose body `body` records on the stream it
    // is given; st continues after it
    template <class Body>
    void add_cond_node(cudaStream_t st, cudaGraphConditionalHandle h, Body body)
    {
        cudaStreamCaptureStatus status;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        CK(cudaStreamGetCaptureInfo(st, &status, nullptr, &g, &deps, nullptr, &ndeps));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
        cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
        CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        CK(cudaStreamBeginCaptureToGraph(cs2, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        body(cs2);
        cudaGraph_t body_out = nullptr;
        CK(cudaStreamEndCapture(cs2, &body_out));
    }

    // Appends to the graph being captured on st a conditional node (handle h)
    // whose body cuts the pruned list from the built one; st continues after it.
    void add_cond_prune(cudaStream_t st, cudaGraphConditionalHandle h)
    {
        add_cond_node(st, h, [&](cudaStream_t c) { launch_prune(S, N, pruned_view(), PV, c); });
    }

    // The evaluation as five concurrent branches (used inside the captured
    // step graph and timed by the autotuner): pair kernel | FP32 PME chain |
    // df64 energy branch of the reciprocal sum (it starts once the first FP32
    // pass has left the FP64 copy of the charge grid) | exclusions, bonded
    // terms (and, with a theta view, the step's force-independent integrator
    // parts) | FP64 solute-solvent energies.  The branches only meet in
    // atomic fixed-point accumulators, so their order does not change any
    // result.  With a conditional handle the first branch starts with the
    // step's conditional rebuild of the neighbour list: only the pair kernel
    // and the solute-solvent energies read the list and the cluster-sorted
    // copy, so the PME, exclusion and bonded work runs beside the rebuild.
    // join = false (the step graphs): the branches are left open, each with
    // its end recorded in ev_join[k] and the end of the solute-solvent energy
    // kernel (the last reader of the positions outside branches 0, 1 and 3)
    // in ev_uv; record_ext_steps continues them
    void eval_kernels_branched(cudaStream_t s0, const ThetaView<real>* pre = nullptr,
                               const cudaGraphConditionalHandle* rebuild = nullptr, bool build_first = false,
                               bool join = true)
    {
        CK(cudaEventRecord(ev_fork, s0));
        for (int k = 0; k < NBR; ++k) CK(cudaStreamWaitEvent(br[k], ev_fork, 0));
        if (rebuild) {
            launch_rebuild_cond(S, *rebuild, br[0]);
            add_cond_build(br[0], *rebuild);
        } else if (build_first) {
            launch_build_nbl(S, N, br[0]);   // an unconditional rebuild (autotuner)
        }
        CK(cudaEventRecord(ev_built, br[0]));
        if (pre) launch_prestep(S, G, *pre, br[3]);
        // with pruning, the step's pair kernel runs on the pruned list, cut
        // again (conditional node) when it is due
        const bool pruned = rebuild && prune_on();
        if (pruned) {
            cudaStreamCaptureStatus status;
            cudaGraph_t g = nullptr;
            CK(cudaStreamGetCaptureInfo(br[0], &status, nullptr, &g, nullptr, nullptr, nullptr));
            cudaGraphConditionalHandle hp;
            CK(cudaGraphConditionalHandleCreate(&hp, g, 0, cudaGraphCondAssignDefault));
            launch_prune_cond(S, hp, br[0]);
            add_cond_prune(br[0], hp);
        }
        launch_pairs(S, pruned ? pruned_view() : N, pair_warps, br[0]);
        // with both layouts in planes, the energy branch reads the
        // fixed-point charge grids itself as soon as the spread is done,
        // beside the FP32 plane pass (no FP64 copy); the grids are cleared
        // once both passes have read them
        const bool early = dual && M.planes && M2.planes;
        launch_spread(S, M, br[1]);
        if (M.planes) {
            if (early) CK(cudaEventRecord(ev_q, br[1]));
            launch_planes(M, early ? PLANE_FWD_KEEP : PLANE_FWD_FIX, br[1]);
            CK(cudaEventRecord(ev_z, br[1]));
            launch_columns(M, S.E, S.lam, dual ? CONV_POTENTIAL : CONV_BOTH, br[1]);
            launch_planes(M, PLANE_INV, br[1]);
        } else {
            launch_fft(M, 2, +1, 1, br[1]);
            CK(cudaEventRecord(ev_z, br[1]));
            launch_fft(M, 1, +1, 0, br[1]);
            launch_fft(M, 0, +1, 0, br[1]);
            launch_conv(M, S.E, S.lam, dual ? CONV_POTENTIAL : CONV_BOTH, br[1]);
            launch_fft(M, 0, -1, 0, br[1]);
            launch_fft(M, 1, -1, 0, br[1]);
            launch_fft(M, 2, -1, 0, br[1]);
        }
        launch_gather(S, M, br[1]);
        if (dual) {
            if (early) {
                // per-axis passes for the axes 2 and 1 (many small blocks
                // beside the other branches), then the column pass
                CK(cudaStreamWaitEvent(br[2], ev_q, 0));
                launch_fft(M2, 2, +1, FFT_FROM_FIX_KEEP, br[2]);
                CK(cudaStreamWaitEvent(br[2], ev_z, 0));
                CK(cudaMemsetAsync(M.Qfix, 0, sizeof(long long) * 2 * (size_t)M.KK, br[2]));
                launch_fft(M2, 1, +1, 0, br[2]);
                launch_columns(M2, S.E, S.lam, CONV_ENERGY, br[2]);
            } else if (M2.planes) {
                CK(cudaStreamWaitEvent(br[2], ev_z, 0));
                launch_fft(M2, 2, +1, 0, br[2]);
                launch_fft(M2, 1, +1, 0, br[2]);
                launch_columns(M2, S.E, S.lam, CONV_ENERGY, br[2]);
            } else {
                CK(cudaStreamWaitEvent(br[2], ev_z, 0));
                launch_fft(M2, 2, +1, 0, br[2]);
                launch_fft(M2, 1, +1, 0, br[2]);
                launch_fft(M2, 0, +1, 0, br[2]);
                launch_conv(M2, S.E, S.lam, CONV_ENERGY, br[2]);
            }
        }
        // with the regulated thermostat, theta's step (a chain of FP64
        // transcendentals) is taken as soon as dU/dlambda is known
        const bool theta_early = pre && pre->th.kind == 1;
        launch_excl(S, X, br[3]);
        if (theta_early) CK(cudaEventRecord(ev_ex, br[3]));
        launch_bonded(S, B, br[3]);
        launch_dafed_force(S, D, br[3]);
        CK(cudaStreamWaitEvent(br[4], ev_built, 0));
        launch_uv_energy(S, N, uv_blocks, br[4]);
        CK(cudaEventRecord(ev_uv, br[4]));
        if (theta_early) {
            // theta's step needs dU/dlambda only: the solute-solvent, the
            // exclusion and 1-4 and the reciprocal class energies; it runs as
            // soon as they are in (the step's end commits it), on the branch
            // of the reciprocal energies as a programmatic dependent of their
            // last kernel
            cudaStream_t tb = theta_branch();
            CK(cudaStreamWaitEvent(tb, ev_ex, 0));
            CK(cudaStreamWaitEvent(tb, ev_uv, 0));
            launch_theta_step(S, *pre, tb, true);
        }
        for (int k = 0; k < NBR; ++k) {
            CK(cudaEventRecord(ev_join[k], br[k]));
            if (join) CK(cudaStreamWaitEvent(s0, ev_join[k], 0));
        }
    }

    // ------------------------------------------------------- autotuner
    // Launch shapes of the evaluation, chosen by timing the captured
    // evaluation graph (its five concurrent branches, as in the step; with
    // and without a preceding list rebuild, weighted 1:3) for each
    // candidate: blocks of the pair kernel per multiprocessor, blocks
    // of the FP64 solute-solvent energy kernel, lines per block of the df64
    // transform passes.  One knob at a time (coordinate descent), each
    // candidate replayed `reps` times after three untimed replays; the
    // median decides, and a candidate replaces the current choice only when
    // it is at least 2 % faster (the evaluation graph is timed, not the
    // step, and differences below that are within run-to-run noise).  The replays only add into the force and energy
    // accumulators, which are cleared afterwards: positions, velocities,
    // theta and every counter are untouched.  A JSON cache (one entry per
    // line) keyed on the device, atom counts, density, cutoff, grid and
    // precision skips the timing when the same kind of system is tuned again.
    std::string tune_key()
    {
        cudaDeviceProp prop{};
        CK(cudaGetDeviceProperties(&prop, device));
        const double rho = n / (P.box[0] * P.box[1] * P.box[2]);
        char buf[512];
        std::snprintf(buf, sizeof(buf), "%s|sm%d|n%d|nu%d|rho%.1f|rc%.3f|K%dx%dx%d|p%d", prop.name, nsm, n, n_u, rho,
                      P.r_cut, M.K[0], M.K[1], M.K[2], P.precision);
        return std::string(buf);
    }

    static bool cache_find(const std::string& path, const std::string& key, int* v, double* ms)
    {
        std::ifstream f(path);
        if (!f) return false;
        std::string line;
        const std::string kq = "\"key\": \"" + key + "\"";
        while (std::getline(f, line)) {
            if (line.find(kq) == std::string::npos) continue;
            auto num = [&](const char* name, double& out) {
                const std::string t = std::string("\"") + name + "\": ";
                const size_t at = line.find(t);
                if (at == std::string::npos) return false;
                out = std::strtod(line.c_str() + at + t.size(), nullptr);
                return true;
            };
            double a, b, c, d, e;
            if (num("pair_blocks_per_sm", a) && num("uv_blocks", b) && num("df64_lines", c) && num("eval_ms", d)) {
                v[0] = (int)a; v[1] = (int)b; v[2] = (int)c; *ms = d;
                if (num("skin_pm", e)) v[3] = (int)e;
                return true;
            }
        }
        return false;
    }

    static void cache_store(const std::string& path, const std::string& key, const int* v, double ms)
    {
        std::vector<std::string> keep;
        {
            std::ifstream f(path);
            std::string line;
            const std::string kq = "\"key\": \"" + key + "\"";
            while (f && std::getline(f, line))
                if (line.rfind("{\"key\": ", 0) == 0 && line.find(kq) == std::string::npos) {
                    if (!line.empty() && line.back() == ',') line.pop_back();
                    keep.push_back(line);
                }
        }
        char buf[768];
        std::snprintf(buf, sizeof(buf),
                      "{\"key\": \"%s\", \"pair_blocks_per_sm\": %d, \"uv_blocks\": %d, \"df64_lines\": %d, "
                      "\"skin_pm\": %d, \"eval_ms\": %.6f}",
                      key.c_str(), v[0], v[1], v[2], v[3], ms);
        keep.push_back(buf);
        std::ofstream f(path, std::ios::trunc);
        if (!f) fail(LFE_ERR_ARG, "cannot write the tuning cache " + path);
        f << "{\"lfe_autotune\": 1, \"entries\": [\n";
        for (size_t i = 0; i < keep.size(); ++i) f << keep[i] << (i + 1 < keep.size() ? ",\n" : "\n");
        f << "]}\n";
    }

    void apply_tuning(const int* v)
    {
        const int bmax = pairs_blocks_per_sm<real>();
        pair_warps = nsm * 4 * std::min(std::max(v[0], 1), bmax);
        uv_blocks = std::max(v[1], 1);
        M2.lines = v[2] == 4 ? 4 : 0;
        if (skin_auto && v[3] > 0 && v[3] != skin_pm()) set_skin(v[3] * 1e-3);
        invalidate_graph();
        ++generation;   // batches that hold this system's step recapture it
    }

    // List buffer (nm): the list holds pairs within r_cut + skin and is
    // rebuilt once an atom has moved more than skin/2 since the last build.
    // A new buffer takes effect with a rebuild at the current positions
    // before the next evaluation.
    bool skin_auto = false;   // the caller left the buffer to lfe_autotune
    static constexpr int SKIN_CANDIDATES_PM[5] = {100, 140, 180, 220, 260};
    int skin_pm() const { return (int)std::lround(P.skin * 1e3); }

    void set_skin(double skin)
    {
        P.skin = skin;
        N.cut2 = (float)((P.r_cut + skin) * (P.r_cut + skin));
        N.skin_half2 = (float)(0.25 * skin * skin);
        G.skin_half2 = (real)(0.25 * skin * skin);
        prune_consts();
        force_rebuild();
        invalidate_graph();
        ++generation;
    }

    // inner buffer b (nm) of the pruned list: pairs within r_cut + b of the
    // pruning positions, pruned again once an atom has moved b/2; active only
    // while b is below the list buffer
    void prune_consts()
    {
        const double b = prune_on() ? prune_skin : 0.0;
        PV.cut2 = (float)((P.r_cut + b) * (P.r_cut + b));
        G.prune_half2 = (real)(0.25 * b * b);
    }

    void set_list_prune(double inner) override
    {
        if (!std::isfinite(inner) || inner < 0.0) fail(LFE_ERR_ARG, "the inner buffer must be finite and >= 0");
        CK(cudaDeviceSynchronize());
        if (exec) recover_overflow(nullptr);
        prune_skin = inner;
        prune_consts();
        const int one = 1;
        CK(cudaMemcpy(S.flags + FL_PRUNE, &one, sizeof(int), cudaMemcpyHostToDevice));
        invalidate_graph();
        ++generation;
    }

    void force_rebuild()
    {
        const int one = 1;
        CK(cudaMemcpy(S.flags + FL_REBUILD, &one, sizeof(int), cudaMemcpyHostToDevice));
    }

    double time_eval_graph(int reps, bool with_build)
    {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        eval_kernels_branched(cs, nullptr, nullptr, with_build);
        CK(cudaStreamEndCapture(cs, &g));
        CK(cudaGraphInstantiate(&e, g, 0));
        for (int r = 0; r < 3; ++r) CK(cudaGraphLaunch(e, cs));
        std::vector<cudaEvent_t> ev(2 * reps);
        for (auto& x : ev) CK(cudaEventCreate(&x));
        for (int r = 0; r < reps; ++r) {
            CK(cudaEventRecord(ev[2 * r], cs));
            CK(cudaGraphLaunch(e, cs));
            CK(cudaEventRecord(ev[2 * r + 1], cs));
        }
        CK(cudaStreamSynchronize(cs));
        std::vector<float> t(reps);
        for (int r = 0; r < reps; ++r) CK(cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]));
        for (auto& x : ev) cudaEventDestroy(x);
        cudaGraphExecDestroy(e);
        cudaGraphDestroy(g);
        std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
        return t[reps / 2];
    }

    void autotune(int reps, const char* cache_path, double* best_ms, int* params) override
    {
        if (reps < 1 || reps > 10000) fail(LFE_ERR_ARG, "reps must be in [1, 10000]");
        const std::string key = tune_key();
        int v[4] = {pairs_blocks_per_sm<real>(), std::max(1, nsm / 2), 16, skin_pm()};
        double best = 0.0;
        if (cache_path && cache_find(cache_path, key, v, &best)) {
            apply_tuning(v);
            if (best_ms) *best_ms = best;
            if (params) { params[0] = v[0]; params[1] = v[1]; params[2] = v[2]; params[3] = 1; params[4] = v[3]; }
            return;
        }
        // a valid list for the current positions, nothing pending
        settle_positions(cs);
        if (exec) recover_overflow(cs);
        settle_rebuild(cs);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpyAsync(lam_save, S.lam, sizeof(LamState), cudaMemcpyDeviceToDevice, cs));
        const int bmax = pairs_blocks_per_sm<real>();
        // Step-based objective when the system steps: the mean time of `reps`
        // captured steps (with the rebuilds the dynamics needs) from a saved
        // state that is restored before every candidate and at the end.  It
        // falls back to the evaluation graph when the state cannot be saved
        // or the trial steps fail (e.g. a packed start that needs its
        // equilibration first).
        std::string ck;
        int nreb0 = 0;
        bool by_steps = P.dt > 0;
        if (by_steps) {
            char tmpl[] = "/tmp/lfe_tune_XXXXXX";
            const int fd = mkstemp(tmpl);
            if (fd < 0) {
                by_steps = false;
            } else {
                close(fd);
                ck = tmpl;
            }
        }
        auto time_steps_from_saved = [&]() -> double {
            restore(ck.c_str());
            step(3, cs);
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventRecord(e0, cs));
            step(reps, cs);
            CK(cudaEventRecord(e1, cs));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            recover_overflow(cs);
            check_flags(cs);
            return ms / reps;
        };
        if (by_steps) {
            CK(cudaMemcpy(&nreb0, S.flags + FL_NREBUILD, sizeof(int), cudaMemcpyDeviceToHost));
            checkpoint(ck.c_str());
            try {
                apply_tuning(v);
                time_steps_from_saved();
            } catch (const Failure&) {
                by_steps = false;
                restore(ck.c_str());
            }
        }
        // the expected evaluation time of a step: a quarter of the steps start
        // with a list rebuild (the pair kernel then waits for it), the rest
        // do not
        constexpr double REBUILD_FRACTION = 0.25;
        auto measure = [&](const int* c) {
            apply_tuning(c);
            if (by_steps) return time_steps_from_saved();
            return (1.0 - REBUILD_FRACTION) * time_eval_graph(reps, false) +
                   REBUILD_FRACTION * time_eval_graph(reps, true);
        };
        best = measure(v);
        auto pair_blocks = [&]() {
            for (int b = 1; b <= bmax; ++b) {
                if (b == v[0]) continue;
                int c[4] = {b, v[1], v[2], v[3]};
                const double t = measure(c);
                if (t < 0.98 * best) { best = t; v[0] = b; }
            }
        };
        pair_blocks();
        if (n_ucl > 0) {
            for (int ub : {nsm / 2, nsm, nsm * 2, nsm * 4}) {
                if (ub < 1 || ub == v[1]) continue;
                int c[4] = {v[0], ub, v[2], v[3]};
                const double t = measure(c);
                if (t < 0.98 * best) { best = t; v[1] = ub; }
            }
        }
        if (dual) {
            int c[4] = {v[0], v[1], v[2] == 16 ? 4 : 16, v[3]};
            const double t = measure(c);
            if (t < 0.98 * best) { best = t; v[2] = c[2]; }
        }
        // the list buffer, when the caller left it to the tuner (stepped
        // objective only: its cost is the rebuild rate against longer tile
        // lists), then the pair kernel's blocks again for the chosen lists
        if (skin_auto && by_steps) {
            // every buffer with every pair-kernel block count: the two trade
            // against each other (a longer list wants the kernel to keep more
            // of the GPU), so one knob at a time can stop at a worse pair
            const int sk0 = v[3];
            for (int sk : SKIN_CANDIDATES_PM) {
                if (sk == sk0) continue;
                for (int b = 1; b <= bmax; ++b) {
                    int c[4] = {b, v[1], v[2], sk};
                    const double t = measure(c);
                    if (t < 0.98 * best) { best = t; v[0] = b; v[3] = sk; }
                }
            }
        }
        apply_tuning(v);
        if (by_steps) {
            // back to the saved state (the counters of rebuilds as before)
            restore(ck.c_str());
            CK(cudaMemcpy(S.flags + FL_NREBUILD, &nreb0, sizeof(int), cudaMemcpyHostToDevice));
        }
        if (!ck.empty()) unlink(ck.c_str());
        // the replays only accumulated forces and energies: clear them
        CK(cudaMemcpyAsync(S.lam, lam_save, sizeof(LamState), cudaMemcpyDeviceToDevice, cs));
        CK(cudaMemsetAsync(S.F, 0, sizeof(long long) * 3 * (size_t)n_pad, cs));
        CK(cudaMemsetAsync(S.Fa, 0, sizeof(long long) * 3 * (size_t)n, cs));
        CK(cudaMemsetAsync(S.E, 0, sizeof(long long) * E_N, cs));
        CK(cudaStreamSynchronize(cs));
        check_flags(cs);
        if (cache_path) cache_store(cache_path, key, v, best);
        if (best_ms) *best_ms = best;
        if (params) { params[0] = v[0]; params[1] = v[1]; params[2] = v[2]; params[3] = 0; params[4] = v[3]; }
    }

    // Replace the tile list by one of exactly `tiles` tiles (the build kernels
    // never write past it) and flag a rebuild: the next step or evaluation
    // builds the list again, and when it needs more tiles the overflow path
    // (skipped steps, growth, rebuild, replay) takes over.
    void set_list_capacity(int tiles) override
    {
        if (tiles < 1) fail(LFE_ERR_ARG, "list capacity must be at least one tile");
        CK(cudaDeviceSynchronize());
        grow_tiles(tiles, tiles);
        N.cap = tiles;
        N.stage_cap = tiles;
        if (S.n_ucl > 0) grow_uv(tiles, 32 * tiles);
        const int one = 1;
        CK(cudaMemcpy(S.flags + FL_REBUILD, &one, sizeof(int), cudaMemcpyHostToDevice));
    }

    // theta (wrapped into [0, 2)), its momentum, and the lambda of Eq. 3 with
    // its switching functions
    void set_theta(double theta, double p_theta) override
    {
        if (!std::isfinite(theta) || !std::isfinite(p_theta)) fail(LFE_ERR_ARG, "theta and p_theta must be finite");
        CK(cudaDeviceSynchronize());
        LamState L;
        CK(cudaMemcpy(&L, S.lam, sizeof(L), cudaMemcpyDeviceToHost));
        double th = theta - 2.0 * std::floor(theta / 2.0);
        if (!(th >= 0.0 && th < 2.0)) th = 0.0;
        L.theta = th;
        L.p_theta = p_theta;
        L.dlam_dtheta = th <= 1.0 ? 1.0 : -1.0;
        L.lambda = th <= 1.0 ? th : 2.0 - th;
        switching_fns(L.lambda, L.hA, L.hB, L.dhA, L.dhB);
        CK(cudaMemcpy(S.lam, &L, sizeof(L), cudaMemcpyHostToDevice));
    }

    // ---------------------------------------------------- barostat
    // Molecules (connected components of the exclusion graph, numbered in
    // order of their lowest atom) as CSR over caller-order atoms, and the
    // masses in FP64, set up on the first volume move.
    std::vector<int> h_mol;
    int n_mol = 0;
    int* d_mstart = nullptr;
    int* d_matoms = nullptr;
    double* d_mass = nullptr;
    R4<real>* d_xsave = nullptr;

    void setup_molecules()
    {
        if (d_mstart) return;
        std::vector<int> id(n, -1), order;
        std::vector<int> root_id(n, -1);
        for (int i = 0; i < n; ++i) {
            const int r = h_mol[i];
            if (root_id[r] < 0) root_id[r] = n_mol++;
            id[i] = root_id[r];
        }
        std::vector<int> start(n_mol + 1, 0), atoms(n);
        for (int i = 0; i < n; ++i) start[id[i] + 1]++;
        for (int m = 0; m < n_mol; ++m) start[m + 1] += start[m];
        std::vector<int> fill(n_mol, 0);
        for (int i = 0; i < n; ++i) atoms[start[id[i]] + fill[id[i]]++] = i;
        d_mstart = upload(start);
        d_matoms = upload(atoms);
        d_mass = upload(h_mass);
        d_xsave = dalloc<R4<real>>(n);
    }

    // New box lengths: every box-dependent table and constant follows (the
    // column geometry keeps its column counts, the reciprocal-space tables,
    // grid scales, convolution prefactor and the self / background energies
    // are recomputed), graphs are recaptured and the neighbour list is
    // rebuilt by the next step or evaluation.
    void set_box(const double* box)
    {
        for (int d = 0; d < 3; ++d) {
            if (!(box[d] > 0) || !std::isfinite(box[d])) fail(LFE_ERR_ARG, "box lengths must be positive");
            if (!(P.r_cut <= 0.5 * box[d])) fail(LFE_ERR_ARG, "r_cut must not exceed half of every box length");
        }
        CK(cudaDeviceSynchronize());
        for (int d = 0; d < 3; ++d) {
            P.box[d] = box[d];
            S.L[d] = (real)box[d];
            S.invL[d] = (real)(1.0 / box[d]);
        }
        N.cinvx = (real)(N.ncx / box[0]);
        N.cinvy = (real)(N.ncy / box[1]);
        const double V = box[0] * box[1] * box[2];
        for (int d = 0; d < 3; ++d) {
            const int K = M.K[d];
            std::vector<double> gf(K), ms(K);
            pme_axis_tables(K, box[d], gf, ms);
            std::vector<real> gfr(K), msr(K);
            for (int m = 0; m < K; ++m) {
                gfr[m] = (real)gf[m];
                msr[m] = (real)ms[m];
            }
            CK(cudaMemcpy(const_cast<real*>(M.gfac[d]), gfr.data(), sizeof(real) * K, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(const_cast<real*>(M.msq[d]), msr.data(), sizeof(real) * K, cudaMemcpyHostToDevice));
            M.kscale[d] = (real)(K / box[d]);
            M.kscale64[d] = K / box[d];
            if (dual) {
                CK(cudaMemcpy(const_cast<double*>(M64.gfac[d]), gf.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
                CK(cudaMemcpy(const_cast<double*>(M64.msq[d]), ms.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
                std::vector<df64> gf2(K), ms2(K);
                for (int m = 0; m < K; ++m) {
                    gf2[m] = df64(gf[m]);
                    ms2[m] = df64(ms[m]);
                }
                CK(cudaMemcpy(const_cast<df64*>(M2.gfac[d]), gf2.data(), sizeof(df64) * K, cudaMemcpyHostToDevice));
                CK(cudaMemcpy(const_cast<df64*>(M2.msq[d]), ms2.data(), sizeof(df64) * K, cudaMemcpyHostToDevice));
                M64.kscale[d] = K / box[d];
                M64.kscale64[d] = K / box[d];
                M2.kscale[d] = df64(K / box[d]);
                M2.kscale64[d] = K / box[d];
            }
        }
        M.conv_pre = (real)(KE / (PI * V));
        if (dual) {
            M64.conv_pre = KE / (PI * V);
            M2.conv_pre = df64(KE / (PI * V));
        }
        constant_energies();
        const int one = 1;
        CK(cudaMemcpy(S.flags + FL_REBUILD, &one, sizeof(int), cudaMemcpyHostToDevice));
        invalidate_graph();
        ++generation;
    }

    // One Monte Carlo volume move at the current lambda (Section 2.6's NPT
    // runs; Aqvist et al. 2004): V' = V + dv_max (2 u0 - 1), every molecule
    // scaled about its centre of mass, accepted with probability
    // min(1, exp(-(U' - U + P (V' - V)) / kT + N_mol ln(V'/V))), with u0 and
    // the acceptance uniform u1 the first two words of Philox4x32-10 at
    // counter (attempt_lo, attempt_hi, 0, 4) and key seed, as (x + 0.5) / 2^32.
    // A rejected move restores the positions and the box exactly.
    void mc_volume_move(double pressure_bar, double dv_max, unsigned long long seed, unsigned long long attempt,
                        int* accepted, double* box_out, double* energies) override
    {
        if (!std::isfinite(pressure_bar) || !(dv_max > 0) || !std::isfinite(dv_max))
            fail(LFE_ERR_ARG, "pressure must be finite and dv_max positive");
        if (!(P.temperature > 0)) fail(LFE_ERR_STATE, "the barostat needs a positive temperature");
        setup_molecules();
        double lam = 0.0;
        lambda_state(&lam, nullptr);
        double t0[LFE_NTERMS], t1[LFE_NTERMS];
        eval(lam, nullptr, t0, 0, nullptr);
        unsigned c[4] = {(unsigned)attempt, (unsigned)(attempt >> 32), 0u, 4u};
        philox_host(c, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
        const double u0 = (c[0] + 0.5) / 4294967296.0, u1 = (c[1] + 0.5) / 4294967296.0;
        const double box0[3] = {P.box[0], P.box[1], P.box[2]};
        const double V = box0[0] * box0[1] * box0[2];
        const double Vn = V + dv_max * (2.0 * u0 - 1.0);
        bool acc = false;
        double U1 = t0[0];
        if (Vn > 0.0) {
            const double sc = std::cbrt(Vn / V);
            const double box1[3] = {sc * box0[0], sc * box0[1], sc * box0[2]};
            bool fits = true;
            for (int d = 0; d < 3; ++d) fits = fits && P.r_cut <= 0.5 * box1[d];
            if (fits) {
                CK(cudaMemcpy(d_xsave, S.x, sizeof(R4<real>) * n, cudaMemcpyDeviceToDevice));
                launch_scale_molecules(S, d_mstart, d_matoms, d_mass, n_mol, sc, box0, nullptr);
                CK(cudaGetLastError());
                set_box(box1);
                eval(lam, nullptr, t1, 0, nullptr);
                U1 = t1[0];
                const double kT = 0.0083144626 * P.temperature;
                const double Pk = pressure_bar * 0.0602214076;
                const double x = -(U1 - t0[0] + Pk * (Vn - V)) / kT + n_mol * std::log(Vn / V);
                acc = u1 < (x >= 0.0 ? 1.0 : std::exp(x));
                if (!acc) {
                    CK(cudaMemcpy(S.x, d_xsave, sizeof(R4<real>) * n, cudaMemcpyDeviceToDevice));
                    set_box(box0);
                }
            }
        }
        if (accepted) *accepted = acc ? 1 : 0;
        if (box_out)
            for (int d = 0; d < 3; ++d) box_out[d] = P.box[d];
        if (energies) {
            energies[0] = t0[0];
            energies[1] = U1;
        }
    }

    bool soft_core() const override { return P.sc_alpha > 0.0; }

    void lambda_state(double* lam, double* mass) override
    {
        CK(cudaDeviceSynchronize());
        LamState L;
        CK(cudaMemcpy(&L, S.lam, sizeof(L), cudaMemcpyDeviceToHost));
        if (lam) *lam = L.lambda;
        if (mass) *mass = T.m;
    }

    cudaStream_t side_stream() override { return cs2; }

    void record_pre(cudaStream_t s0) override
    {
        cudaStreamCaptureStatus status;
        cudaGraph_t g = nullptr;
        CK(cudaStreamGetCaptureInfo(s0, &status, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        launch_rebuild_cond(S, h, s0);
        add_cond_build(s0, h);
        if (prune_on()) {
            cudaGraphConditionalHandle hp;
            CK(cudaGraphConditionalHandleCreate(&hp, g, 0, cudaGraphCondAssignDefault));
            launch_prune_cond(S, hp, s0);
            add_cond_prune(s0, hp);
        }
    }

    // the pair list of the recorded steps: the pruned one when pruning is on
    // (record_pre then cuts it when due)
    NblView<real> step_list() const { return prune_on() ? pruned_view() : N; }

    void record_eval(cudaStream_t s0, bool with_pairs) override { record_eval_on(s0, with_pairs, step_list()); }

    void record_eval_on(cudaStream_t s0, bool with_pairs, const NblView<real>& list)
    {
        if (with_pairs) launch_pairs(S, list, pair_warps, s0);
        launch_uv_energy(S, N, uv_blocks, s0);
        launch_pme(S, M, dual ? &M2 : nullptr, s0);
        launch_excl(S, X, s0);
        launch_bonded(S, B, s0);
        launch_dafed_force(S, D, s0);
    }

    void record_post(cudaStream_t s0) override
    {
        launch_prestep(S, G, T, s0);
        launch_integrate(S, G, s0);
        launch_theta(S, T, s0);
        launch_dafed_step(S, D, s0);
    }

    void record_step(cudaStream_t s0) override
    {
        record_pre(s0);
        record_eval(s0, true);
        record_post(s0);
    }

    void record_exchange_eval(cudaStream_t s0, double* terms) override
    {
        record_pre(s0);
        record_eval(s0, true);
        launch_eval_out(S, nullptr, terms, const_vv, const_uu, const_uv, s0);
    }

    LamState* lam_state_device() override { return S.lam; }

    bool pair_job(PairJob* out) override
    {
        if constexpr (std::is_same<real, float>::value) {
            out->s = S;
            out->nb = step_list();
            return true;
        }
        return false;
    }

    void note_batch_steps(int n) override
    {
        steps_requested += (unsigned long long)n;
    }

    bool overflow_pending(cudaStream_t st) override
    {
        CK(cudaMemcpyAsync(h_flags, S.flags, sizeof(int) * FL_N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return (h_flags[FL_ERROR] & ERRB_OVERFLOW) != 0;
    }

    void recover(cudaStream_t st) override
    {
        if (!exec) capture_step_graph();
        recover_overflow(st);
    }

    // theta's branch: the reciprocal energies' (the df64 branch 2 of FP32
    // systems, the PME branch 1 of FP64 systems)
    cudaStream_t theta_branch() const { return dual ? br[2] : br[1]; }

    // the end of a captured step, continuing the open branches of
    // eval_kernels_branched (theta's view given; under the regulated
    // thermostat theta's step has been taken on theta's branch):
    //  - the atoms' integrator on branch 3 once the forces are complete
    //    (pairs on branch 0, reciprocal gather on 1, exclusions, bonded and
    //    d-AFED forces on 3) and the last other reader of the positions (the
    //    solute-solvent energies on 4) is done;
    //  - theta's commit (or its whole step) on theta's branch once every
    //    reader of the lambda state is done;
    //  - the auxiliary angles' step on branch 1 once their forces (branch 3)
    //    and the pair branch (whose rebuild can raise a list overflow, which
    //    skips the step's state updates) are in.
    // The integrator and the commit are programmatic dependents of the pair
    // kernel and of theta's step (both let their dependents be scheduled
    // early): they are in place when their last prerequisite ends.
    void record_ext_steps(cudaStream_t s0)
    {
        const bool early = T.th.kind == 1;
        cudaStream_t tb = early ? theta_branch() : br[4];
        // the waits below read the branch ends recorded by the evaluation
        for (int k = 0; k < NBR; ++k)
            if (br[k] != tb) CK(cudaStreamWaitEvent(tb, ev_join[k], 0));
        if (early) launch_theta_commit(S, T, tb, true);
        else launch_theta(S, T, tb);
        CK(cudaEventRecord(ev_rec, tb));
        CK(cudaStreamWaitEvent(br[3], ev_join[0], 0));
        CK(cudaStreamWaitEvent(br[3], ev_join[1], 0));
        CK(cudaStreamWaitEvent(br[3], ev_uv, 0));
        launch_integrate(S, G, br[3], true);
        if (D.n) {
            CK(cudaStreamWaitEvent(br[1], ev_join[3], 0));
            CK(cudaStreamWaitEvent(br[1], ev_join[0], 0));
            launch_dafed_step(S, D, br[1]);
        }
        CK(cudaEventRecord(ev_join[1], br[1]));
        CK(cudaEventRecord(ev_join[3], br[3]));
        CK(cudaStreamWaitEvent(s0, ev_rec, 0));
        for (int k = 0; k < NBR; ++k) CK(cudaStreamWaitEvent(s0, ev_join[k], 0));
    }

    void capture_step_graph()
    {
        cudaStream_t s0 = cs;
        CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
        cudaStreamCaptureStatus status;
        cudaGraph_t g = nullptr;
        CK(cudaStreamGetCaptureInfo(s0, &status, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        eval_kernels_branched(s0, &T, &h, false, false);
        record_ext_steps(s0);
        CK(cudaStreamEndCapture(s0, &graph));
        CK(cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority));
    }

    // One step with host input and output as one captured graph: the copy of
    // the new positions from page-locked host memory, their assignment and
    // rebuild decision (as lfe_set_positions), the step (as lfe_step), the
    // state packing and the copies into the caller's page-locked buffers (as
    // lfe_get_state).  The graph is specific to the host pointers and is
    // recaptured when they or the device buffers change.
    cudaGraph_t io_graph = nullptr;
    cudaGraphExec_t io_exec = nullptr;
    const void* io_key[4] = {nullptr, nullptr, nullptr, nullptr};
    unsigned io_gen = ~0u;
    double* h_io_tail = nullptr;   // pinned copy of the scalar state of the last io step

    static bool host_pinned(const void* p)
    {
        if (!p) return true;
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeHost;
    }

    // the host element type of the graph (8: double, 4: float) is part of its key
    template <typename TIO>
    void capture_io_graph(const TIO* pos_in, TIO* pos_out, TIO* vel_out)
    {
        if (io_exec) { cudaGraphExecDestroy(io_exec); io_exec = nullptr; }
        if (io_graph) { cudaGraphDestroy(io_graph); io_graph = nullptr; }
        const size_t nv = 3 * (size_t)n;
        constexpr bool F32 = sizeof(TIO) == 4;
        // device staging: the input positions, then the packed positions and
        // velocities (the doubles' staging is the state-packing buffer)
        TIO* d_in;
        TIO* d_xv;
        if constexpr (F32) {
            d_in = d_io32;
            d_xv = d_io32 + nv;
        } else {
            d_in = d_pos;
            d_xv = d_state;
        }
        double* d_tail = d_state + 6 * (size_t)n;
        cudaStream_t s0 = cs;
        CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
        cudaStreamCaptureStatus status;
        cudaGraph_t g = nullptr;
        CK(cudaStreamGetCaptureInfo(s0, &status, nullptr, &g, nullptr, nullptr, nullptr));
        if (pos_in) {
            // the step's own conditional rebuild (first branch below) acts
            // on the flag that the new positions raise
            CK(cudaMemcpyAsync(d_in, pos_in, sizeof(TIO) * nv, cudaMemcpyHostToDevice, s0));
            launch_check_positions(S, (const TIO*)d_in, s0);
            launch_assign_moved(S, (const TIO*)d_in, G.skin_half2, G.prune_half2, s0);
        }
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        eval_kernels_branched(s0, &T, &h, false, false);
        record_ext_steps(s0);
        if constexpr (F32)
            launch_pack_state_f32(S, T.st, d_xv, d_tail, s0);
        else
            launch_pack_state(S, T.st, d_state, s0);
        CK(cudaMemcpyAsync(h_io_tail, d_tail, sizeof(double) * 16, cudaMemcpyDeviceToHost, s0));
        if (pos_out) CK(cudaMemcpyAsync(pos_out, d_xv, sizeof(TIO) * nv, cudaMemcpyDeviceToHost, s0));
        if (vel_out) CK(cudaMemcpyAsync(vel_out, d_xv + nv, sizeof(TIO) * nv, cudaMemcpyDeviceToHost, s0));
        CK(cudaStreamEndCapture(s0, &io_graph));
        CK(cudaGraphInstantiate(&io_exec, io_graph, cudaGraphInstantiateFlagUseNodePriority));
        io_key[0] = pos_in;
        io_key[1] = pos_out;
        io_key[2] = vel_out;
        io_key[3] = (const void*)sizeof(TIO);
        io_gen = generation;
    }

    float* d_io32 = nullptr;   // [9n] float staging of lfe_step_io_f32

    // the state as floats (positions and velocities) for the float variant's
    // rare general paths
    void get_state_f32(float* pos, float* vel, double* ext)
    {
        const size_t nv = 3 * (size_t)n;
        std::vector<double> p(pos ? nv : 0), v(vel ? nv : 0);
        get_state(pos ? p.data() : nullptr, vel ? v.data() : nullptr, ext);
        for (size_t i = 0; i < p.size(); ++i) pos[i] = (float)p[i];
        for (size_t i = 0; i < v.size(); ++i) vel[i] = (float)v[i];
    }

    template <typename TIO>
    void step_io_t(const TIO* pos_in, TIO* pos_out, TIO* vel_out, double* ext_out, cudaStream_t st)
    {
        constexpr bool F32 = sizeof(TIO) == 4;
        const char* who = F32 ? "lfe_step_io_f32" : "lfe_step_io";
        if (!(P.dt > 0)) fail(LFE_ERR_STATE, "dt must be positive to step");
        if (!host_pinned(pos_in) || !host_pinned(pos_out) || !host_pinned(vel_out))
            fail(LFE_ERR_ARG, std::string("host buffers of ") + who + " must be page-locked");
        if (eager || pos_pending || since_check > 0) {
            // a queued overflow or pending position update is settled first
            CK(cudaStreamSynchronize(st));
            if (exec) recover_overflow(st);
            if (pos_pending) settle_positions(st);
            pos_pending = false;
        }
        auto state_out = [&] {
            if constexpr (F32)
                get_state_f32(pos_out, vel_out, ext_out);
            else
                get_state(pos_out, vel_out, ext_out);
        };
        if (eager) {
            if (pos_in && !finite_all(pos_in, 3 * (size_t)n)) fail(LFE_ERR_ARG, "non-finite position");
            if (pos_in) {
                if constexpr (F32) {
                    const std::vector<double> p(pos_in, pos_in + 3 * (size_t)n);
                    set_positions(p.data(), 0, st);
                } else {
                    set_positions(pos_in, 0, st);
                }
            }
            step(1, st);
            state_out();
            return;
        }
        if (!d_state) {
            d_state = dalloc<double>(6 * (size_t)n + 16);
            CK(cudaMallocHost(&h_state, sizeof(double) * (6 * (size_t)n + 16)));
        }
        if (F32 && !d_io32) d_io32 = dalloc<float>(9 * (size_t)n);
        if (!h_io_tail) CK(cudaMallocHost(&h_io_tail, sizeof(double) * 16));
        if (!io_exec || io_gen != generation || io_key[0] != pos_in || io_key[1] != pos_out ||
            io_key[2] != vel_out || io_key[3] != (const void*)sizeof(TIO))
            capture_io_graph(pos_in, pos_out, vel_out);
        CK(cudaGraphLaunch(io_exec, st));
        ++steps_requested;
        CK(cudaStreamSynchronize(st));
        const int err = (int)h_io_tail[13];
        if (err & ERRB_BADPOS) {
            // the positions were checked on the device and refused: the step
            // left the state as it was (the outputs hold that state)
            const int rest = err & ~ERRB_BADPOS;
            CK(cudaMemcpy(S.flags + FL_ERROR, &rest, sizeof(int), cudaMemcpyHostToDevice));
            --steps_requested;
            fail(LFE_ERR_ARG, "non-finite position");
        }
        if (err) {
            // the step was skipped (list overflow) or failed: the general path
            // settles it and reads the state again
            if (err & ERRB_OVERFLOW) {
                if (!exec) capture_step_graph();
                recover_overflow(st);
            }
            state_out();
            return;
        }
        if (ext_out)
            for (int k = 0; k < LFE_NEXT; ++k) ext_out[k] = h_io_tail[k];
    }

    void step_io(const double* pos_in, double* pos_out, double* vel_out, double* ext_out, cudaStream_t st) override
    {
        step_io_t(pos_in, pos_out, vel_out, ext_out, st);
    }

    void step_io_f32(const float* pos_in, float* pos_out, float* vel_out, double* ext_out,
                     cudaStream_t st) override
    {
        step_io_t(pos_in, pos_out, vel_out, ext_out, st);
    }

    // steps requested through lfe_step since creation, and launches since
    // the last overflow check
    unsigned long long steps_requested = 0;
    int since_check = 0;
    unsigned long long step_base = 0;     // LamState step counter at creation / restore

    // eager stepping (environment LFE_EAGER_STEPS=1): the same kernels as the
    // captured graph, launched one by one, with the rebuild decided on the
    // host after every step.  Used for per-kernel profiling (profilers do not
    // attribute kernels inside graphs that hold conditional nodes).
    bool eager = false;

    void step_eager(cudaStream_t st)
    {
        eval_kernels(st);
        launch_prestep(S, G, T, st);
        launch_integrate(S, G, st);
        launch_theta(S, T, st);
        launch_dafed_step(S, D, st);
        CK(cudaMemcpyAsync(h_flags, S.flags, sizeof(int) * FL_N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (h_flags[FL_REBUILD]) {
            int v[2] = {0, h_flags[FL_NREBUILD] + 1};
            CK(cudaMemcpy(S.flags + FL_REBUILD, &v[0], sizeof(int), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(S.flags + FL_NREBUILD, &v[1], sizeof(int), cudaMemcpyHostToDevice));
            build_neighbors(st);
        }
    }

    void step(int nsteps, cudaStream_t st) override
    {
        if (nsteps < 0) fail(LFE_ERR_ARG, "n_steps must be >= 0");
        if (!(P.dt > 0)) fail(LFE_ERR_STATE, "dt must be positive to step");
        if (eager) {
            for (int i = 0; i < nsteps; ++i) step_eager(st);
            return;
        }
        if (!exec) capture_step_graph();
        for (int i = 0; i < nsteps; ++i) {
            CK(cudaGraphLaunch(exec, st));
            ++steps_requested;
            if (++since_check >= 64) recover_overflow(st);
        }
    }

    // A rebuild inside the graph that overflowed the tile capacity sets the
    // overflow bit; every later step is a no-op.  Here (every 64 steps and at
    // every synchronising call) the host grows the capacity, rebuilds the
    // list, recaptures the graph and replays the skipped steps.
    void recover_overflow(cudaStream_t st)
    {
        since_check = 0;
        for (int attempt = 0; attempt < 4; ++attempt) {
            CK(cudaMemcpyAsync(h_flags, S.flags, sizeof(int) * FL_N, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (!(h_flags[FL_ERROR] & ERRB_OVERFLOW)) return;
            LamState L;
            CK(cudaMemcpy(&L, S.lam, sizeof(L), cudaMemcpyDeviceToHost));
            const unsigned long long done = L.step - step_base;
            const long long missing = (long long)steps_requested - (long long)done;
            grow_for_flags();
            int clr[2] = {0, 0};
            CK(cudaMemcpy(S.flags, clr, sizeof(clr), cudaMemcpyHostToDevice));
            build_neighbors(st);
            capture_step_graph();
            for (long long i = 0; i < missing; ++i) CK(cudaGraphLaunch(exec, st));
        }
        fail(LFE_ERR_OVERFLOW, "neighbour-list capacity kept overflowing");
    }

    // one packing kernel and one copy into pinned memory; the rare overflow
    // and error cases are handled after it (and the state packed again)
    double* d_state = nullptr;     // [6n + 16]
    double* h_state = nullptr;     // pinned copy

    void get_state(double* pos, double* vel, double* ext) override
    {
        if (!d_state) {
            d_state = dalloc<double>(6 * (size_t)n + 16);
            CK(cudaMallocHost(&h_state, sizeof(double) * (6 * (size_t)n + 16)));
        }
        CK(cudaDeviceSynchronize());
        // positions and velocities go straight into the caller's arrays, the
        // scalar state into the pinned buffer
        const size_t nv = 3 * (size_t)n;
        for (int pass = 0; pass < 2; ++pass) {
            launch_pack_state(S, T.st, d_state, nullptr);
            CK(cudaMemcpyAsync(h_state + 2 * nv, d_state + 2 * nv, sizeof(double) * 16, cudaMemcpyDeviceToHost,
                               nullptr));
            if (pos) CK(cudaMemcpyAsync(pos, d_state, sizeof(double) * nv, cudaMemcpyDeviceToHost, nullptr));
            if (vel) CK(cudaMemcpyAsync(vel, d_state + nv, sizeof(double) * nv, cudaMemcpyDeviceToHost, nullptr));
            CK(cudaStreamSynchronize(nullptr));
            const int err = (int)h_state[6 * (size_t)n + 13];
            if (!err) break;
            if (pass == 1 || !(err & ERRB_OVERFLOW)) {
                check_flags(nullptr);   // reports the error (clears the bit)
                break;
            }
            // a neighbour list that ran out of capacity: queued steps replay
            if (exec) recover_overflow(nullptr);
            if (pos_pending) settle_positions(nullptr);
        }
        pos_pending = false;
        const double* e = h_state + 6 * (size_t)n;
        if (ext)
            for (int k = 0; k < LFE_NEXT; ++k) ext[k] = e[k];
    }

    // Eq. 2: bin means and the trapezoid integral of the mean-force profile
    // over the occupied bin centres, extended linearly to lambda = 0 and 1
    void ti(double* mean, double* count, double* delta_g, int reset) override
    {
        CK(cudaDeviceSynchronize());
        std::vector<double> sum(LFE_TI_BINS);
        std::vector<unsigned long long> cnt(LFE_TI_BINS);
        CK(cudaMemcpy(sum.data(), T.ti_sum, sizeof(double) * LFE_TI_BINS, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cnt.data(), T.ti_cnt, sizeof(unsigned long long) * LFE_TI_BINS, cudaMemcpyDeviceToHost));
        std::vector<double> xs, ys;
        for (int b = 0; b < LFE_TI_BINS; ++b) {
            const double m = cnt[b] ? sum[b] / (double)cnt[b] : std::nan("");
            if (mean) mean[b] = m;
            if (count) count[b] = (double)cnt[b];
            if (cnt[b]) {
                xs.push_back((b + 0.5) / LFE_TI_BINS);
                ys.push_back(m);
            }
        }
        if (delta_g) {
            const size_t k = xs.size();
            double g = std::nan("");
            if (k == 1) {
                g = ys[0];
            } else if (k > 1) {
                g = 0.0;
                for (size_t i = 0; i + 1 < k; ++i) g += 0.5 * (ys[i] + ys[i + 1]) * (xs[i + 1] - xs[i]);
                const double lo = ys[0] - (ys[1] - ys[0]) / (xs[1] - xs[0]) * xs[0];
                const double hi = ys[k - 1] + (ys[k - 1] - ys[k - 2]) / (xs[k - 1] - xs[k - 2]) * (1.0 - xs[k - 1]);
                g += 0.5 * (lo + ys[0]) * xs[0] + 0.5 * (ys[k - 1] + hi) * (1.0 - xs[k - 1]);
            }
            *delta_g = g;
        }
        if (reset) {
            CK(cudaMemset(T.ti_sum, 0, sizeof(double) * LFE_TI_BINS));
            CK(cudaMemset(T.ti_cnt, 0, sizeof(unsigned long long) * LFE_TI_BINS));
        }
    }

    // ------------------------------------------------------------- d-AFED
    double dafed_friction = 0.0;
    double* d_probe = nullptr;     // [n_cv] probe output

    void dafed_view_from(int n_cv, const int* atoms, DafedView& V, std::vector<int4>& at)
    {
        if (n_cv < 0) fail(LFE_ERR_ARG, "negative number of coupled torsions");
        if (n_cv > 0 && !atoms) fail(LFE_ERR_ARG, "atoms is NULL");
        at.resize(n_cv);
        for (int k = 0; k < n_cv; ++k) {
            const int* a = atoms + 4 * k;
            for (int j = 0; j < 4; ++j)
                if (a[j] < 0 || a[j] >= n) fail(LFE_ERR_ARG, "torsion atom index out of range");
            if (a[0] == a[1] || a[0] == a[2] || a[0] == a[3] || a[1] == a[2] || a[1] == a[3] || a[2] == a[3])
                fail(LFE_ERR_ARG, "a torsion repeats an atom");
            at[k] = make_int4(a[0], a[1], a[2], a[3]);
        }
        V.n = n_cv;
    }

    // couple n torsions to auxiliary angles (Eq. 15); n = 0 switches it off
    void set_dafed(int n_cv, const int* atoms, const double* kappa, const double* mass, double temperature,
                   double friction, const double* s0) override
    {
        std::vector<int4> at;
        DafedView V{};
        dafed_view_from(n_cv, atoms, V, at);
        if (n_cv > 0) {
            if (!kappa || !mass) fail(LFE_ERR_ARG, "kappa and mass must not be NULL");
            for (int k = 0; k < n_cv; ++k) {
                if (!(kappa[k] >= 0) || !std::isfinite(kappa[k])) fail(LFE_ERR_ARG, "kappa must be finite and >= 0");
                if (!(mass[k] > 0) || !std::isfinite(mass[k])) fail(LFE_ERR_ARG, "auxiliary masses must be > 0");
                if (s0 && !std::isfinite(s0[k])) fail(LFE_ERR_ARG, "non-finite initial auxiliary angle");
            }
            if (!(temperature >= 0) || !(friction >= 0) || !std::isfinite(temperature) || !std::isfinite(friction))
                fail(LFE_ERR_ARG, "auxiliary temperature and friction must be >= 0");
        }
        CK(cudaDeviceSynchronize());
        if (exec) recover_overflow(nullptr);
        for (void* ptr : {(void*)D.atoms, (void*)D.kappa, (void*)D.mass, (void*)D.s, (void*)D.p, (void*)D.fs,
                          (void*)D.xi, (void*)D.veta, (void*)d_dafed_ec, (void*)d_probe})
            if (ptr) dfree(ptr);
        D = DafedView{};
        d_probe = nullptr;
        d_dafed_ec = nullptr;
        if (n_cv > 0) {
            D.n = n_cv;
            D.atoms = upload(at);
            D.kappa = upload(std::vector<double>(kappa, kappa + n_cv));
            D.mass = upload(std::vector<double>(mass, mass + n_cv));
            D.s = dalloc<double>(n_cv);
            D.p = dalloc<double>(n_cv);
            D.fs = dalloc<double>(n_cv);
            D.xi = dalloc<double>(n_cv);
            D.veta = dalloc<double>(n_cv);
            D.th = ext_th;
            D.pre = T.pre;
            d_dafed_ec = dalloc<ExtConst>(n_cv);
            D.ec = d_dafed_ec;
            d_probe = dalloc<double>(n_cv);
            D.dt = P.dt;
            dafed_friction = friction;
            D.a_fric = std::exp(-friction * P.dt);
            D.kT = KB * temperature;
            D.key = G.key;
            dafed_consts();
            if (s0) {
                std::vector<double> w(n_cv);
                for (int k = 0; k < n_cv; ++k) w[k] = s0[k] - 2.0 * PI * std::floor((s0[k] + PI) / (2.0 * PI));
                CK(cudaMemcpy(D.s, w.data(), sizeof(double) * n_cv, cudaMemcpyHostToDevice));
            } else {
                launch_dafed_probe(S, D, 0.0, D.s, nullptr);   // start on the torsions
            }
            CK(cudaDeviceSynchronize());
            CK(cudaGetLastError());
        }
        invalidate_graph();
        ++generation;
    }

    // Thermostat of theta and the auxiliary angles (Section 2.6): kind 0
    // Langevin, kind 1 regulated Nose-Hoover-Langevin (see ext_step); every
    // thermostat velocity starts from zero
    ExtThermo ext_th{0, 0, 0.04, 1.0};
    ExtConst* d_dafed_ec = nullptr;   // D.ec

    // the auxiliary variables' step constants at their masses, kT and friction
    void dafed_consts()
    {
        if (!D.n) return;
        std::vector<double> m(D.n);
        CK(cudaMemcpy(m.data(), D.mass, sizeof(double) * D.n, cudaMemcpyDeviceToHost));
        std::vector<ExtConst> k(D.n);
        for (int i = 0; i < D.n; ++i) k[i] = ext_const(D.th, m[i], D.kT, D.a_fric);
        CK(cudaMemcpy(d_dafed_ec, k.data(), sizeof(ExtConst) * D.n, cudaMemcpyHostToDevice));
    }

    void set_ext_thermostat(int kind, double tau, double n_reg) override
    {
        if (kind != 0 && kind != 1) fail(LFE_ERR_ARG, "thermostat kind must be 0 (Langevin) or 1 (RNHL)");
        if (kind == 1 && (!(tau > 0) || !std::isfinite(tau) || !(n_reg > 0) || !std::isfinite(n_reg)))
            fail(LFE_ERR_ARG, "RNHL needs tau > 0 and a regulation parameter > 0");
        CK(cudaDeviceSynchronize());
        if (exec) recover_overflow(nullptr);
        ext_th = ExtThermo{kind, 0, kind == 1 ? tau : 0.04, kind == 1 ? n_reg : 1.0};
        T.th = ext_th;
        T.tc = ext_const(T.th, T.m, T.kT, T.a_fric);
        D.th = ext_th;
        const double zero = 0.0;
        CK(cudaMemcpy(reinterpret_cast<char*>(S.lam) + offsetof(LamState, v_eta), &zero, sizeof(double),
                      cudaMemcpyHostToDevice));
        if (D.n) CK(cudaMemset(D.veta, 0, sizeof(double) * D.n));
        dafed_consts();
        invalidate_graph();
        ++generation;
    }

    void ext_thermostat_state(double* v_theta, double* v_aux) override
    {
        CK(cudaDeviceSynchronize());
        if (v_theta) {
            LamState L;
            CK(cudaMemcpy(&L, S.lam, sizeof(L), cudaMemcpyDeviceToHost));
            *v_theta = L.v_eta;
        }
        if (v_aux && D.n) CK(cudaMemcpy(v_aux, D.veta, sizeof(double) * D.n, cudaMemcpyDeviceToHost));
    }

    void dafed_state(double* s_out, double* p_out, double* xi_out) override
    {
        CK(cudaDeviceSynchronize());
        if (D.n == 0) return;
        if (s_out) CK(cudaMemcpy(s_out, D.s, sizeof(double) * D.n, cudaMemcpyDeviceToHost));
        if (p_out) CK(cudaMemcpy(p_out, D.p, sizeof(double) * D.n, cudaMemcpyDeviceToHost));
        if (xi_out) {
            launch_dafed_probe(S, D, 0.0, d_probe, nullptr);
            CK(cudaMemcpy(xi_out, d_probe, sizeof(double) * D.n, cudaMemcpyDeviceToHost));
        }
    }

    // Eq. 16 at the current positions (atoms of mass 0 do not contribute)
    void dafed_masses(int n_cv, const int* atoms, double c, double* out) override
    {
        if (!(c > 0) || !out) fail(LFE_ERR_ARG, "c must be > 0 and out not NULL");
        std::vector<int4> at;
        DafedView V{};
        dafed_view_from(n_cv, atoms, V, at);
        if (n_cv == 0) return;
        int4* d_at = upload(at);
        double* d_out = dalloc<double>(n_cv);
        V.atoms = d_at;
        CK(cudaDeviceSynchronize());
        launch_dafed_probe(S, V, c, d_out, nullptr);
        CK(cudaMemcpy(out, d_out, sizeof(double) * n_cv, cudaMemcpyDeviceToHost));
        dfree(d_at);
        dfree(d_out);
        for (int k = 0; k < n_cv; ++k)
            if (!std::isfinite(out[k])) fail(LFE_ERR_ARG, "no movable atom in a torsion");
    }

    // checkpoint layout: header | x | v | xref | LamState | OpesState | centre | weight | S | TI sums |
    // TI counts | d-AFED s | d-AFED p | d-AFED thermostat velocities | checksum
    struct CkHeader {
        char magic[8];
        int version, precision, n, max_k, n_cv, pad;
        double box[3];
        double skin;      // list buffer of the run that wrote it
    };

    void checkpoint(const char* path) override
    {
        CK(cudaDeviceSynchronize());
        check_flags(nullptr);
        CkHeader h{};
        std::memcpy(h.magic, "LFECKPT1", 8);
        h.version = 5;
        h.skin = P.skin;
        h.precision = precision;
        for (int d = 0; d < 3; ++d) h.box[d] = P.box[d];
        h.n = n;
        h.max_k = T.max_k;
        h.n_cv = D.n;
        std::vector<unsigned char> buf;
        auto put = [&](const void* p, size_t sz) {
            const unsigned char* c = static_cast<const unsigned char*>(p);
            buf.insert(buf.end(), c, c + sz);
        };
        auto put_dev = [&](const void* d, size_t sz) {
            std::vector<unsigned char> tmp(sz);
            CK(cudaMemcpy(tmp.data(), d, sz, cudaMemcpyDeviceToHost));
            put(tmp.data(), sz);
        };
        put(&h, sizeof(h));
        put_dev(S.x, sizeof(R4<real>) * n);
        put_dev(S.v, sizeof(R4<real>) * n);
        put_dev(S.xref, sizeof(R4<real>) * n);
        put_dev(S.lam, sizeof(LamState));
        put_dev(T.st, sizeof(OpesState));
        put_dev(T.centre, sizeof(double) * 2 * T.max_k);
        put_dev(T.weight, sizeof(double) * 2 * T.max_k);
        put_dev(T.S, sizeof(double) * 2 * T.max_k);
        put_dev(T.ti_sum, sizeof(double) * LFE_TI_BINS);
        put_dev(T.ti_cnt, sizeof(unsigned long long) * LFE_TI_BINS);
        if (D.n) {
            put_dev(D.s, sizeof(double) * D.n);
            put_dev(D.p, sizeof(double) * D.n);
            put_dev(D.veta, sizeof(double) * D.n);
        }
        uint64_t cs_ = fnv1a(buf.data(), buf.size());
        put(&cs_, sizeof(cs_));
        FILE* f = std::fopen(path, "wb");
        if (!f) fail(LFE_ERR_ARG, std::string("cannot open ") + path);
        size_t w = std::fwrite(buf.data(), 1, buf.size(), f);
        std::fclose(f);
        if (w != buf.size()) fail(LFE_ERR_ARG, "short write");
    }

    void restore(const char* path) override
    {
        FILE* f = std::fopen(path, "rb");
        if (!f) fail(LFE_ERR_ARG, std::string("cannot open ") + path);
        std::vector<unsigned char> buf;
        unsigned char tmp[65536];
        size_t r;
        while ((r = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + r);
        std::fclose(f);
        const size_t body = sizeof(CkHeader) + 3 * sizeof(R4<real>) * n + sizeof(LamState) + sizeof(OpesState) +
                            3 * sizeof(double) * 2 * T.max_k + (sizeof(double) + sizeof(unsigned long long)) * LFE_TI_BINS +
                            3 * sizeof(double) * D.n;
        if (buf.size() != body + sizeof(uint64_t)) fail(LFE_ERR_ARG, "checkpoint size does not match this system");
        uint64_t stored;
        std::memcpy(&stored, buf.data() + body, sizeof(stored));
        if (stored != fnv1a(buf.data(), body)) fail(LFE_ERR_ARG, "checkpoint checksum mismatch");
        CkHeader h;
        std::memcpy(&h, buf.data(), sizeof(h));
        if (std::memcmp(h.magic, "LFECKPT1", 8) != 0 || h.version != 5 || h.precision != precision || h.n != n ||
            h.max_k != T.max_k || h.n_cv != D.n)
            fail(LFE_ERR_ARG, "checkpoint header does not match this system");
        if (h.box[0] != P.box[0] || h.box[1] != P.box[1] || h.box[2] != P.box[2]) set_box(h.box);
        size_t off = sizeof(CkHeader);
        auto get_dev = [&](void* d, size_t sz) {
            CK(cudaMemcpy(d, buf.data() + off, sz, cudaMemcpyHostToDevice));
            off += sz;
        };
        const unsigned char* px = buf.data() + off;
        (void)px;
        // rebuild the list from the saved reference positions so that the
        // tile list (and every rounding downstream of it) is the same as in
        // the run that wrote the checkpoint; then install the current x
        std::vector<unsigned char> xcur(buf.begin() + off, buf.begin() + off + sizeof(R4<real>) * n);
        off += sizeof(R4<real>) * n;
        get_dev(S.v, sizeof(R4<real>) * n);
        get_dev(S.x, sizeof(R4<real>) * n);   // xref -> x for the build
        get_dev(S.lam, sizeof(LamState));
        get_dev(T.st, sizeof(OpesState));
        get_dev(T.centre, sizeof(double) * 2 * T.max_k);
        get_dev(T.weight, sizeof(double) * 2 * T.max_k);
        get_dev(T.S, sizeof(double) * 2 * T.max_k);
        get_dev(T.ti_sum, sizeof(double) * LFE_TI_BINS);
        get_dev(T.ti_cnt, sizeof(unsigned long long) * LFE_TI_BINS);
        if (D.n) {
            get_dev(D.s, sizeof(double) * D.n);
            get_dev(D.p, sizeof(double) * D.n);
            get_dev(D.veta, sizeof(double) * D.n);
        }
        int zero[FL_N] = {0, 0, 0, 0};
        CK(cudaMemcpy(S.flags, zero, sizeof(int) * 2, cudaMemcpyHostToDevice));
        build_neighbors(nullptr);
        CK(cudaMemcpy(S.x, xcur.data(), xcur.size(), cudaMemcpyHostToDevice));
        refresh_sorted(nullptr);
        // a list built at the saved reference positions with a smaller
        // buffer than the writer's may miss pairs at the current positions
        if (h.skin > P.skin) force_rebuild();
        CK(cudaDeviceSynchronize());
        LamState L;
        CK(cudaMemcpy(&L, S.lam, sizeof(L), cudaMemcpyDeviceToHost));
        step_base = L.step;
        steps_requested = 0;
    }

    // recompute the sorted coordinates from x in the current slot order
    void refresh_sorted(cudaStream_t st)
    {
        launch_refresh_sorted(S, st);
        CK(cudaStreamSynchronize(st));
    }

    int time_stages(double lam, int reps, cudaStream_t st, const char** names, double* ms, int max_n) override
    {
        static const char* stage_names[] = {"nbl_build", "pairs", "pme_spread", "pme_fft_fwd", "pme_conv",
                                            "pme_fft_inv", "pme_gather", "excl_14", "bonded", "eval_out",
                                            "uv_energy_fp64", "pairs_full"};
        const int ns = 12;
        std::vector<cudaEvent_t> ev(ns + 5);
        double acc_prune = 0.0, acc_pruned_pairs = 0.0;
        for (auto& e : ev) CK(cudaEventCreate(&e));
        std::vector<double> acc(ns, 0.0);
        CK(cudaMemcpyAsync(lam_save, S.lam, sizeof(LamState), cudaMemcpyDeviceToDevice, st));
        launch_set_lambda(S, lam, st);
        for (int r = 0; r < reps; ++r) {
            CK(cudaEventRecord(ev[0], st));
            launch_build_nbl(S, N, st);
            CK(cudaEventRecord(ev[1], st));
            launch_pairs(S, N, pair_warps, st);
            CK(cudaEventRecord(ev[2], st));
            launch_uv_energy(S, N, uv_blocks, st);
            CK(cudaEventRecord(ev[11], st));
            launch_spread(S, M, st);
            CK(cudaEventRecord(ev[3], st));
            if (M.planes) {
                // fwd: planes (+ the df64 energy branch); conv: the column
                // pass with its axis-0 transforms; inv: planes
                launch_planes(M, PLANE_FWD_FIX, st);
                if (dual) {
                    launch_fft(M2, 2, +1, 0, st);
                    launch_fft(M2, 1, +1, 0, st);
                    launch_columns(M2, S.E, S.lam, CONV_ENERGY, st);
                }
                CK(cudaEventRecord(ev[4], st));
                launch_columns(M, S.E, S.lam, dual ? CONV_POTENTIAL : CONV_BOTH, st);
                CK(cudaEventRecord(ev[5], st));
                launch_planes(M, PLANE_INV, st);
            } else {
                launch_fft(M, 2, +1, 1, st);
                if (dual) {
                    launch_fft(M2, 2, +1, 0, st);
                    launch_fft(M2, 1, +1, 0, st);
                    launch_fft(M2, 0, +1, 0, st);
                    launch_conv(M2, S.E, S.lam, CONV_ENERGY, st);
                }
                launch_fft(M, 1, +1, 0, st);
                launch_fft(M, 0, +1, 0, st);
                CK(cudaEventRecord(ev[4], st));
                launch_conv(M, S.E, S.lam, dual ? CONV_POTENTIAL : CONV_BOTH, st);
                CK(cudaEventRecord(ev[5], st));
                launch_fft(M, 0, -1, 0, st);
                launch_fft(M, 1, -1, 0, st);
                launch_fft(M, 2, -1, 0, st);
            }
            CK(cudaEventRecord(ev[6], st));
            launch_gather(S, M, st);
            CK(cudaEventRecord(ev[7], st));
            launch_excl(S, X, st);
            CK(cudaEventRecord(ev[8], st));
            launch_bonded(S, B, st);
            CK(cudaEventRecord(ev[9], st));
            launch_eval_out(S, nullptr, nullptr, const_vv, const_uu, const_uv, st);
            CK(cudaEventRecord(ev[10], st));
            CK(cudaEventSynchronize(ev[10]));
            // stage k runs from ev[k] to ev[k+1], except that the FP64
            // solute-solvent energy kernel (stage 10) sits between ev[2] and
            // ev[11], and the spread stage starts at ev[11]
            for (int k = 0; k < 10; ++k) {
                float t = 0;
                CK(cudaEventElapsedTime(&t, k == 2 ? ev[11] : ev[k], ev[k + 1]));
                acc[k] += t;
            }
            float tu = 0;
            CK(cudaEventElapsedTime(&tu, ev[2], ev[11]));
            acc[10] += tu;
            // the pair kernel once more with the grid that fills every
            // multiprocessor (the step's tuned shape may leave room for the
            // concurrent branches); its forces are cleared again
            if constexpr (std::is_same<real, float>::value) {
                CK(cudaEventRecord(ev[12], st));
                launch_pairs(S, N, nsm * 4 * pairs_blocks_per_sm<real>(), st);
                CK(cudaEventRecord(ev[13], st));
                launch_eval_out(S, nullptr, nullptr, const_vv, const_uu, const_uv, st);
                CK(cudaEventSynchronize(ev[13]));
                float tf = 0;
                CK(cudaEventElapsedTime(&tf, ev[12], ev[13]));
                acc[11] += tf;
            }
            // with pruning: the pruning of the built list, and the pair kernel
            // on the pruned list in the step's shape
            if (prune_on()) {
                CK(cudaEventRecord(ev[14], st));
                launch_prune(S, N, pruned_view(), PV, st);
                CK(cudaEventRecord(ev[15], st));
                launch_pairs(S, pruned_view(), pair_warps, st);
                CK(cudaEventRecord(ev[16], st));
                launch_eval_out(S, nullptr, nullptr, const_vv, const_uu, const_uv, st);
                CK(cudaEventSynchronize(ev[16]));
                float a = 0, b = 0;
                CK(cudaEventElapsedTime(&a, ev[14], ev[15]));
                CK(cudaEventElapsedTime(&b, ev[15], ev[16]));
                acc_prune += a;
                acc_pruned_pairs += b;
            }
        }
        CK(cudaMemcpyAsync(S.lam, lam_save, sizeof(LamState), cudaMemcpyDeviceToDevice, st));
        for (auto& e : ev) cudaEventDestroy(e);
        check_flags(st);
        std::vector<std::pair<const char*, double>> out;
        for (int k = 0; k < (std::is_same<real, float>::value ? ns : ns - 1); ++k) out.emplace_back(stage_names[k], acc[k]);
        if (prune_on()) {
            out.emplace_back("prune", acc_prune);
            out.emplace_back("pairs_pruned", acc_pruned_pairs);
        }
        const int m = std::min((int)out.size(), max_n);
        for (int k = 0; k < m; ++k) {
            if (names) names[k] = out[k].first;
            if (ms) ms[k] = reps > 0 ? out[k].second / reps : 0.0;
        }
        return m;
    }

    // Parameter gradients of the solute atoms at lambda.  The class
    // potentials come from one more FP64 reciprocal pass with h_A = 0 (the
    // FP64 copy of the charge grid for FP32 systems, the FP64 grid itself
    // for FP64 systems); the kernel recomputes every real-space interaction
    // of each solute atom.
    void param_grad(double lam, double* dU, double* d2U, double* basis, int on_device, cudaStream_t st) override
    {
        if (P.sc_alpha > 0.0) fail(LFE_ERR_STATE, "parameter gradients need the linear-basis coupling (sc_alpha = 0)");
        if (!(lam >= 0.0 && lam <= 1.0)) fail(LFE_ERR_ARG, "lambda must be in [0, 1]");
        if (n_u == 0) fail(LFE_ERR_ARG, "the system has no solute atoms");
        settle_positions(st);
        if (exec) recover_overflow(st);
        settle_rebuild(st);
        CK(cudaMemcpyAsync(lam_save, S.lam, sizeof(LamState), cudaMemcpyDeviceToDevice, st));
        launch_set_lambda(S, lam, st);
        const PmeView<double>* P64;
        if constexpr (std::is_same<real, double>::value) P64 = &M;
        else P64 = &M64;
        launch_spread(S, M, st);
        if (M.planes) {
            launch_planes(M, PLANE_FWD_FIX, st);
            if (dual) {
                launch_fft(M64, 2, +1, 0, st);
                launch_fft(M64, 1, +1, 0, st);
            }
            launch_columns(*P64, S.E, lam0, CONV_POTENTIAL, st);
            launch_planes(*P64, PLANE_INV, st);
        } else {
            launch_fft(M, 2, +1, 1, st);
            if (dual) launch_fft(M64, 2, +1, 0, st);
            launch_fft(*P64, 1, +1, 0, st);
            launch_fft(*P64, 0, +1, 0, st);
            launch_conv(*P64, S.E, lam0, CONV_POTENTIAL, st);
            launch_fft(*P64, 0, -1, 0, st);
            launch_fft(*P64, 1, -1, 0, st);
            launch_fft(*P64, 2, -1, 0, st);
        }
        AdjConst c{};
        for (int d = 0; d < 3; ++d) {
            c.L[d] = P.box[d];
            c.invL[d] = 1.0 / P.box[d];
        }
        c.alpha = P.ewald_alpha;
        c.two_a_sqrtpi = 2.0 * P.ewald_alpha / std::sqrt(PI);
        c.rc2 = P.r_cut * P.r_cut;
        c.rsw = P.r_switch >= 0 ? P.r_switch : P.r_cut;
        c.swi = P.r_switch >= 0 ? 1.0 / (P.r_cut - P.r_switch) : 0.0;
        c.bg_pre = -KE * PI / (2.0 * P.box[0] * P.box[1] * P.box[2] * P.ewald_alpha * P.ewald_alpha);
        double* g_dU = d_pg;
        double* g_d2 = d_pg + 3 * (size_t)n_u;
        double* g_b = d_pg + 6 * (size_t)n_u;
        launch_param_grad(S, N, X, M, P64->Z, c, g_dU, g_d2, g_b, st);
        CK(cudaMemcpyAsync(S.lam, lam_save, sizeof(LamState), cudaMemcpyDeviceToDevice, st));
        CK(cudaGetLastError());
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (dU) CK(cudaMemcpyAsync(dU, g_dU, sizeof(double) * 3 * n_u, kind, st));
        if (d2U) CK(cudaMemcpyAsync(d2U, g_d2, sizeof(double) * 3 * n_u, kind, st));
        if (basis) CK(cudaMemcpyAsync(basis, g_b, sizeof(double) * 9 * n_u, kind, st));
        if (!on_device) CK(cudaStreamSynchronize(st));
    }

    // Replace the solute atoms' charges, sigma and epsilon (each [n_u] in
    // solute caller order, NULL = unchanged).  The constant self and
    // background energies follow the new charges; captured step graphs are
    // rebuilt because those constants are kernel arguments.
    void set_solute_params(const double* q, const double* sig, const double* eps, int on_device,
                           cudaStream_t st) override
    {
        if (n_u == 0) fail(LFE_ERR_ARG, "the system has no solute atoms");
        const double* src[3] = {q, sig, eps};
        std::vector<double> v[3];
        for (int k = 0; k < 3; ++k) {
            v[k].resize(n_u);
            std::vector<double>& cur = k == 0 ? h_q : (k == 1 ? h_sig : h_eps);
            if (!src[k]) {
                for (int b = 0; b < n_u; ++b) v[k][b] = cur[h_solute[b]];
            } else if (on_device) {
                CK(cudaMemcpyAsync(v[k].data(), src[k], sizeof(double) * n_u, cudaMemcpyDeviceToHost, st));
            } else {
                std::copy(src[k], src[k] + n_u, v[k].begin());
            }
        }
        if (on_device) CK(cudaStreamSynchronize(st));
        for (int k = 0; k < 3; ++k)
            for (int b = 0; b < n_u; ++b) {
                if (!std::isfinite(v[k][b])) fail(LFE_ERR_ARG, "non-finite solute parameter");
                if (k > 0 && v[k][b] < 0) fail(LFE_ERR_ARG, "sigma and epsilon must be >= 0");
            }
        CK(cudaDeviceSynchronize());
        if (exec) recover_overflow(nullptr);
        for (int b = 0; b < n_u; ++b) {
            h_q[h_solute[b]] = v[0][b];
            h_sig[h_solute[b]] = v[1][b];
            h_eps[h_solute[b]] = v[2][b];
        }
        for (int k = 0; k < 3; ++k)
            CK(cudaMemcpyAsync(d_pstage + (size_t)k * n_u, v[k].data(), sizeof(double) * n_u,
                               cudaMemcpyHostToDevice, st));
        launch_set_solute_params(S, d_q, d_sig, d_eps, d_pstage, st);
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        constant_energies();
        invalidate_graph();
        ++generation;
    }
};

// ------------------------------------------------------- batched replicas
// Replicas (lambda windows, solvents, solutes; uneven sizes) advance together:
// one captured CUDA graph holds every replica's step as its own chain of
// kernels (each with its own device-side conditional rebuild), forked from
// and joined to one stream, so one graph launch moves all replicas and the
// GPU runs the chains concurrently.
struct lfe_batch {
    std::vector<lfe_system*> sys;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> join, built;
    cudaStream_t s0 = nullptr, s_pair = nullptr;
    cudaEvent_t fork = nullptr, pairs_done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int since_check = 0;
    std::vector<unsigned> gens;
    std::string err;
    // device-side lambda exchange every `ex_stride` batch steps: its own
    // captured graph (the replicas' evaluations, then k_hrex), enqueued by
    // lfe_batch_step after the step graph without synchronising; the ladder,
    // the attempt counter and the accepted counts stay on the device
    int ex_stride = 0, ex_n = 0;
    unsigned long long ex_seed = 0;
    double ex_beta = 0.0;
    unsigned long long ex_steps = 0;          // batch steps since the exchange was set
    int* d_ladder = nullptr;
    unsigned long long* d_ex_ctr = nullptr;   // [0] attempts, [1 .. n-1] accepted per ladder position
    double* d_ex_terms = nullptr;             // [replicas][LFE_NTERMS]
    LamState** d_ex_lams = nullptr;
    cudaGraph_t ex_graph = nullptr;
    cudaGraphExec_t ex_exec = nullptr;
    std::vector<int> ex_members;

    void capture_exchange()
    {
        if (ex_exec) { cudaGraphExecDestroy(ex_exec); ex_exec = nullptr; }
        if (ex_graph) { cudaGraphDestroy(ex_graph); ex_graph = nullptr; }
        std::vector<LamState*> lams(sys.size());
        for (size_t i = 0; i < sys.size(); ++i) lams[i] = sys[i]->impl->lam_state_device();
        CK(cudaMemcpy(d_ex_lams, lams.data(), sizeof(LamState*) * sys.size(), cudaMemcpyHostToDevice));
        CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
        CK(cudaEventRecord(fork, s0));
        for (int i : ex_members) {
            CK(cudaStreamWaitEvent(lanes[i], fork, 0));
            sys[i]->impl->record_exchange_eval(lanes[i], d_ex_terms + (size_t)i * LFE_NTERMS);
            CK(cudaEventRecord(join[i], lanes[i]));
            CK(cudaStreamWaitEvent(s0, join[i], 0));
        }
        launch_hrex(d_ex_lams, d_ex_terms, d_ladder, ex_n, ex_beta, ex_seed, d_ex_ctr, d_ex_ctr + 1, s0);
        CK(cudaStreamEndCapture(s0, &ex_graph));
        CK(cudaGraphInstantiate(&ex_exec, ex_graph, 0));
    }

    // the FP32 replicas' pair kernels run as one launch (k_pairs2, one row of its grid per replica)
    std::vector<PairJob> h_jobs;
    int n_jobs = 0;
    std::vector<int> shared;     // replica i takes part in the shared launch
    int pair_blocks = 0;

    ~lfe_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto s : lanes) if (s) cudaStreamDestroy(s);
        for (auto e : join) if (e) cudaEventDestroy(e);
        for (auto e : built) if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (pairs_done) cudaEventDestroy(pairs_done);
        if (s0) cudaStreamDestroy(s0);
        if (s_pair) cudaStreamDestroy(s_pair);
        if (ex_exec) cudaGraphExecDestroy(ex_exec);
        if (ex_graph) cudaGraphDestroy(ex_graph);
        if (d_ladder) cudaFree(d_ladder);
        if (d_ex_ctr) cudaFree(d_ex_ctr);
        if (d_ex_terms) cudaFree(d_ex_terms);
        if (d_ex_lams) cudaFree(d_ex_lams);
    }

    // the descriptors of the FP32 replicas (views of their device buffers,
    // refreshed whenever the graph is recaptured)
    void upload_jobs()
    {
        h_jobs.clear();
        shared.assign(sys.size(), 0);
        for (size_t i = 0; i < sys.size(); ++i) {
            PairJob j;
            if (sys[i]->impl->pair_job(&j)) {
                h_jobs.push_back(j);
                shared[i] = 1;
            }
        }
        n_jobs = (int)h_jobs.size();
        // one resident wave: measured on 16 water + 16 octanol replicas, the
        // batch step takes 2.58 ms with it, 2.78 / 3.19 / 3.92 / 5.88 ms with
        // 4 / 3 / 2 / 1 blocks per multiprocessor (the shared launch is the
        // step's critical path)
        if (!pair_blocks) pair_blocks = pairs_batch_blocks();
    }

    // mean device time (ms) of the shared pair launch over reps launches, at
    // the replicas' current lists; the forces and energies it adds are cleared
    // afterwards (between steps they are zero: the integrators and the step
    // ends consume them)
    double time_pairs(int reps, cudaStream_t st)
    {
        CK(cudaDeviceSynchronize());
        upload_jobs();
        if (!n_jobs || reps <= 0) return 0.0;
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        launch_pairs_batch(h_jobs.data(), n_jobs, pair_blocks, st);
        CK(cudaEventRecord(a, st));
        for (int r = 0; r < reps; ++r) launch_pairs_batch(h_jobs.data(), n_jobs, pair_blocks, st);
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        for (auto& j : h_jobs) {
            CK(cudaMemsetAsync(j.s.F, 0, sizeof(long long) * 3 * (size_t)j.s.n_pad, st));
            CK(cudaMemsetAsync(j.s.E, 0, sizeof(long long) * E_N, st));
        }
        CK(cudaStreamSynchronize(st));
        return ms / reps;
    }

    void invalidate()
    {
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
        if (ex_exec) { cudaGraphExecDestroy(ex_exec); ex_exec = nullptr; }
        if (ex_graph) { cudaGraphDestroy(ex_graph); ex_graph = nullptr; }
    }

    // one step of every replica: each replica's rebuild decision and
    // conditional rebuild on its own lane; the FP32 replicas' pair kernels as
    // one launch once all their lists are ready; each replica's other
    // evaluation kernels on its lane meanwhile; its integrators once its
    // forces are complete
    void capture()
    {
        upload_jobs();
        CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
        CK(cudaEventRecord(fork, s0));
        for (size_t i = 0; i < sys.size(); ++i) {
            CK(cudaStreamWaitEvent(lanes[i], fork, 0));
            sys[i]->impl->record_pre(lanes[i]);
            CK(cudaEventRecord(built[i], lanes[i]));
        }
        if (n_jobs) {
            CK(cudaStreamWaitEvent(s_pair, fork, 0));
            for (size_t i = 0; i < sys.size(); ++i)
                if (shared[i]) CK(cudaStreamWaitEvent(s_pair, built[i], 0));
            launch_pairs_batch(h_jobs.data(), n_jobs, pair_blocks, s_pair);
            CK(cudaEventRecord(pairs_done, s_pair));
        }
        for (size_t i = 0; i < sys.size(); ++i) {
            sys[i]->impl->record_eval(lanes[i], !shared[i]);
            if (shared[i]) CK(cudaStreamWaitEvent(lanes[i], pairs_done, 0));
            sys[i]->impl->record_post(lanes[i]);
            CK(cudaEventRecord(join[i], lanes[i]));
            CK(cudaStreamWaitEvent(s0, join[i], 0));
        }
        CK(cudaStreamEndCapture(s0, &graph));
        CK(cudaGraphInstantiate(&exec, graph, 0));
        gens.clear();
        for (auto* s : sys) gens.push_back(s->impl->generation);
    }

    bool stale() const
    {
        for (size_t i = 0; i < sys.size(); ++i)
            if (sys[i]->impl->generation != gens[i]) return true;
        return false;
    }

    // every 64 steps: replicas whose list overflowed are regrown and replay
    // their skipped steps alone; the batch graph is then recaptured
    void check(cudaStream_t st)
    {
        since_check = 0;
        bool any = false;
        for (auto* s : sys)
            if (s->impl->overflow_pending(st)) {
                s->impl->recover(st);
                any = true;
            }
        if (any) invalidate();
    }

    void step(int n, cudaStream_t st)
    {
        if (exec && stale()) invalidate();
        if (!exec) capture();
        if (ex_stride > 0 && !ex_exec) capture_exchange();
        for (int k = 0; k < n; ++k) {
            CK(cudaGraphLaunch(exec, st));
            for (auto* s : sys) s->impl->note_batch_steps(1);
            if (ex_stride > 0 && (++ex_steps % (unsigned long long)ex_stride) == 0ull) {
                // an overflowed list must be regrown before the exchange reads energies
                if (since_check > 0) {
                    check(st);
                    if (!exec) capture();
                }
                if (!ex_exec) capture_exchange();
                CK(cudaGraphLaunch(ex_exec, st));
            }
            if (++since_check >= 64) {
                check(st);
                if (!exec) capture();
                if (ex_stride > 0 && !ex_exec) capture_exchange();
            }
        }
    }
};

const char* lfe_batch_last_error_impl(const lfe_batch* b) { return b ? b->err.c_str() : ""; }

// ---------------------------------------------------------------- C-ABI
namespace {
int guard(lfe_system* sys, const std::function<void()>& f)
{
    if (!sys) return LFE_ERR_ARG;
    try {
        f();
        sys->err.clear();
        return LFE_OK;
    } catch (const Failure& e) {
        sys->err = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        sys->err = e.what();
        return LFE_ERR_ARG;
    }
}
}  // namespace

extern "C" {

int lfe_create(const lfe_params* params, const lfe_topology* topo, lfe_system** out)
{
    if (out) *out = nullptr;
    if (!params || !topo || !out) {
        g_create_error = "NULL argument";
        return LFE_ERR_ARG;
    }
    auto sys = new lfe_system();
    try {
        if (params->precision == LFE_FP64) {
            auto s = new System<double>();
            sys->impl.reset(s);
            s->create(*params, *topo);
        } else {
            auto s = new System<float>();
            sys->impl.reset(s);
            s->create(*params, *topo);
        }
    } catch (const Failure& e) {
        g_create_error = e.msg;
        delete sys;
        return e.code;
    } catch (const std::exception& e) {
        g_create_error = e.what();
        delete sys;
        return LFE_ERR_ARG;
    }
    g_create_error.clear();
    *out = sys;
    return LFE_OK;
}

int lfe_set_positions(lfe_system* sys, const double* pos, int on_device, void* stream)
{
    return guard(sys, [&] { sys->impl->set_positions(pos, on_device, (cudaStream_t)stream); });
}

int lfe_set_velocities(lfe_system* sys, const double* vel)
{
    return guard(sys, [&] { sys->impl->set_velocities(vel); });
}

int lfe_set_integrator(lfe_system* sys, double dt, double friction, double temperature)
{
    return guard(sys, [&] { sys->impl->set_integrator(dt, friction, temperature); });
}

int lfe_build_neighbors(lfe_system* sys, void* stream)
{
    return guard(sys, [&] { sys->impl->build_neighbors((cudaStream_t)stream); });
}

int lfe_eval(lfe_system* sys, double lambda, double* forces, double* energy_terms, int out_on_device, void* stream)
{
    return guard(sys, [&] { sys->impl->eval(lambda, forces, energy_terms, out_on_device, (cudaStream_t)stream); });
}

int lfe_param_grad(lfe_system* sys, double lambda, double* dU_dp, double* d2U_dl_dp, double* basis,
                   int out_on_device, void* stream)
{
    return guard(sys, [&] {
        sys->impl->param_grad(lambda, dU_dp, d2U_dl_dp, basis, out_on_device, (cudaStream_t)stream);
    });
}

int lfe_set_solute_params(lfe_system* sys, const double* charge, const double* sigma, const double* epsilon,
                          int on_device, void* stream)
{
    return guard(sys, [&] {
        sys->impl->set_solute_params(charge, sigma, epsilon, on_device, (cudaStream_t)stream);
    });
}

int lfe_set_dafed(lfe_system* sys, int n_cv, const int* atoms, const double* kappa, const double* mass,
                  double temperature, double friction, const double* s0)
{
    return guard(sys, [&] { sys->impl->set_dafed(n_cv, atoms, kappa, mass, temperature, friction, s0); });
}

int lfe_dafed_state(lfe_system* sys, double* s, double* p_s, double* xi)
{
    return guard(sys, [&] { sys->impl->dafed_state(s, p_s, xi); });
}

int lfe_set_ext_thermostat(lfe_system* sys, int kind, double tau, double n_reg)
{
    return guard(sys, [&] { sys->impl->set_ext_thermostat(kind, tau, n_reg); });
}

int lfe_ext_thermostat_state(lfe_system* sys, double* v_eta_theta, double* v_eta_aux)
{
    return guard(sys, [&] { sys->impl->ext_thermostat_state(v_eta_theta, v_eta_aux); });
}

int lfe_dafed_masses(lfe_system* sys, int n_cv, const int* atoms, double c, double* mass_out)
{
    return guard(sys, [&] { sys->impl->dafed_masses(n_cv, atoms, c, mass_out); });
}

int lfe_ti(lfe_system* sys, double* mean, double* count, double* delta_g, int reset)
{
    return guard(sys, [&] { sys->impl->ti(mean, count, delta_g, reset); });
}

int lfe_step(lfe_system* sys, int n_steps, void* stream)
{
    return guard(sys, [&] { sys->impl->step(n_steps, (cudaStream_t)stream); });
}

int lfe_get_state(lfe_system* sys, double* pos, double* vel, double* ext)
{
    return guard(sys, [&] { sys->impl->get_state(pos, vel, ext); });
}

int lfe_checkpoint(lfe_system* sys, const char* path)
{
    return guard(sys, [&] {
        if (!path) fail(LFE_ERR_ARG, "path is NULL");
        sys->impl->checkpoint(path);
    });
}

int lfe_restore(lfe_system* sys, const char* path)
{
    return guard(sys, [&] {
        if (!path) fail(LFE_ERR_ARG, "path is NULL");
        sys->impl->restore(path);
    });
}

int lfe_time_stages(lfe_system* sys, double lambda, int reps, void* stream, const char** names, double* ms,
                    int max_n)
{
    int r = 0;
    int rc = guard(sys, [&] { r = sys->impl->time_stages(lambda, reps, (cudaStream_t)stream, names, ms, max_n); });
    return rc == LFE_OK ? r : rc;
}

int lfe_autotune(lfe_system* sys, int reps, const char* cache_path, double* best_ms, int* params)
{
    return guard(sys, [&] { sys->impl->autotune(reps, cache_path, best_ms, params); });
}

int lfe_set_theta(lfe_system* sys, double theta, double p_theta)
{
    return guard(sys, [&] { sys->impl->set_theta(theta, p_theta); });
}

int lfe_set_list_capacity(lfe_system* sys, int tiles)
{
    return guard(sys, [&] { sys->impl->set_list_capacity(tiles); });
}

int lfe_mc_volume_move(lfe_system* sys, double pressure_bar, double dv_max, unsigned long long seed,
                       unsigned long long attempt, int* accepted, double* box_out, double* energies)
{
    return guard(sys, [&] { sys->impl->mc_volume_move(pressure_bar, dv_max, seed, attempt, accepted, box_out,
                                                       energies); });
}

int lfe_set_list_prune(lfe_system* sys, double inner_buffer)
{
    return guard(sys, [&] { sys->impl->set_list_prune(inner_buffer); });
}

int lfe_step_io_f32(lfe_system* sys, const float* pos_in, float* pos_out, float* vel_out, double* ext_out,
                    void* stream)
{
    return guard(sys, [&] { sys->impl->step_io_f32(pos_in, pos_out, vel_out, ext_out, (cudaStream_t)stream); });
}

int lfe_step_io(lfe_system* sys, const double* pos_in, double* pos_out, double* vel_out, double* ext_out,
                void* stream)
{
    return guard(sys, [&] { sys->impl->step_io(pos_in, pos_out, vel_out, ext_out, (cudaStream_t)stream); });
}



int lfe_batch_create(lfe_system* const* systems, int n, lfe_batch** out)
{
    if (out) *out = nullptr;
    if (!systems || n <= 0 || !out) {
        g_create_error = "lfe_batch_create: need a non-empty array of systems";
        return LFE_ERR_ARG;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j)
            if (!systems[i] || systems[i] == systems[j]) {
                g_create_error = "lfe_batch_create: systems must be distinct and non-NULL";
                return LFE_ERR_ARG;
            }
    auto b = new lfe_batch();
    b->sys.assign(systems, systems + n);
    try {
        CK(cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&b->s_pair, cudaStreamNonBlocking));
        b->lanes.resize(n);
        for (int i = 0; i < n; ++i) CK(cudaStreamCreateWithFlags(&b->lanes[i], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&b->pairs_done, cudaEventDisableTiming));
        b->join.resize(n);
        b->built.resize(n);
        for (int i = 0; i < n; ++i) {
            CK(cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&b->built[i], cudaEventDisableTiming));
        }
    } catch (const Failure& e) {
        g_create_error = e.msg;
        delete b;
        return e.code;
    }
    g_create_error.clear();
    *out = b;
    return LFE_OK;
}

int lfe_batch_eval(lfe_batch* b, const double* lambdas, double* energy_terms, void* stream)
{
    if (!b || !lambdas) return LFE_ERR_ARG;
    for (size_t i = 0; i < b->sys.size(); ++i) {
        const int rc = lfe_eval(b->sys[i], lambdas[i], nullptr, energy_terms ? energy_terms + LFE_NTERMS * i : nullptr,
                                0, stream);
        if (rc != LFE_OK) {
            b->err = "replica " + std::to_string(i) + ": " + b->sys[i]->err;
            return rc;
        }
    }
    return LFE_OK;
}

int lfe_batch_exchange(lfe_batch* b, int n, int* ladder, double temperature, unsigned long long seed,
                       unsigned long long attempt, int* accepted, void* stream)
{
    if (!b || !ladder || n < 2 || !(temperature > 0) || !std::isfinite(temperature)) {
        if (b) b->err = "lfe_batch_exchange: bad arguments (ladder of >= 2 replicas, temperature > 0)";
        return LFE_ERR_ARG;
    }
    try {
        std::vector<char> seen(b->sys.size(), 0);
        std::vector<double> lam(n), uuv(n), us(n);
        for (int k = 0; k < n; ++k) {
            const int r = ladder[k];
            if (r < 0 || r >= (int)b->sys.size() || seen[r]) fail(LFE_ERR_ARG, "ladder entries must be distinct replica indices");
            seen[r] = 1;
            if (b->sys[r]->impl->soft_core())
                fail(LFE_ERR_STATE, "lambda exchange needs the linear-basis coupling (sc_alpha = 0)");
            double m = 0;
            b->sys[r]->impl->lambda_state(&lam[k], &m);
            if (m > 0) fail(LFE_ERR_ARG, "replica " + std::to_string(r) + " has a dynamical theta (lambda_mass > 0)");
            if (k > 0 && !(lam[k] >= lam[k - 1])) fail(LFE_ERR_ARG, "ladder must list the replicas in lambda order");
        }
        // the basis energies of every configuration at its own lambda
        for (int k = 0; k < n; ++k) {
            double t[LFE_NTERMS];
            b->sys[ladder[k]]->impl->eval(lam[k], nullptr, t, 0, (cudaStream_t)stream);
            uuv[k] = t[4];
            us[k] = t[5];
        }
        const double beta = 1.0 / (lfe::KB * temperature);
        for (int k = 0; k + 1 < n; ++k)
            if (accepted) accepted[k] = 0;
        for (int k = (int)(attempt & 1ull); k + 1 < n; k += 2) {
            double ha, hb, hA2, hB2, d0, d1;
            lfe::switching_fns(lam[k], ha, hb, d0, d1);
            lfe::switching_fns(lam[k + 1], hA2, hB2, d0, d1);
            // Eq. 4 is linear in the basis energies: the swap changes the
            // total energy by (dh_A)(U_uv,i - U_uv,j) + (dh_B)(U_soft,i - U_soft,j)
            const double delta = (hA2 - ha) * (uuv[k] - uuv[k + 1]) + (hB2 - hb) * (us[k] - us[k + 1]);
            unsigned c[4] = {(unsigned)k, (unsigned)(attempt & 0xffffffffull), (unsigned)(attempt >> 32), 3u};
            philox_host(c, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
            const double u = (c[0] + 0.5) / 4294967296.0;
            if (delta <= 0.0 || u < std::exp(-beta * delta)) {
                b->sys[ladder[k]]->impl->set_theta(lam[k + 1], 0.0);
                b->sys[ladder[k + 1]]->impl->set_theta(lam[k], 0.0);
                std::swap(ladder[k], ladder[k + 1]);
                if (accepted) accepted[k] = 1;
            }
        }
    } catch (const Failure& e) {
        b->err = e.msg;
        return e.code;
    }
    return LFE_OK;
}

int lfe_batch_step(lfe_batch* b, int n_steps, void* stream)
{
    if (!b || n_steps < 0) return LFE_ERR_ARG;
    try {
        b->step(n_steps, (cudaStream_t)stream);
    } catch (const Failure& e) {
        b->err = e.msg;
        return e.code;
    }
    return LFE_OK;
}

int lfe_batch_set_exchange(lfe_batch* b, int n, const int* ladder, double temperature, unsigned long long seed,
                           int stride)
{
    if (!b) return LFE_ERR_ARG;
    try {
        CK(cudaDeviceSynchronize());
        if (stride <= 0) {
            b->ex_stride = 0;
            return LFE_OK;
        }
        if (!ladder || n < 2 || !(temperature > 0) || !std::isfinite(temperature))
            fail(LFE_ERR_ARG, "lfe_batch_set_exchange: ladder of >= 2 replicas and temperature > 0 required");
        std::vector<char> seen(b->sys.size(), 0);
        double prev = -1.0;
        for (int k = 0; k < n; ++k) {
            const int r = ladder[k];
            if (r < 0 || r >= (int)b->sys.size() || seen[r]) fail(LFE_ERR_ARG, "ladder entries must be distinct replica indices");
            seen[r] = 1;
            if (b->sys[r]->impl->soft_core())
                fail(LFE_ERR_STATE, "lambda exchange needs the linear-basis coupling (sc_alpha = 0)");
            double lam = 0, m = 0;
            b->sys[r]->impl->lambda_state(&lam, &m);
            if (m > 0) fail(LFE_ERR_ARG, "replica " + std::to_string(r) + " has a dynamical theta (lambda_mass > 0)");
            if (!(lam >= prev)) fail(LFE_ERR_ARG, "ladder must list the replicas in lambda order");
            prev = lam;
        }
        const size_t R = b->sys.size();
        if (!b->d_ladder) {
            CK(cudaMalloc(&b->d_ladder, sizeof(int) * R));
            CK(cudaMalloc(&b->d_ex_ctr, sizeof(unsigned long long) * R));
            CK(cudaMalloc(&b->d_ex_terms, sizeof(double) * LFE_NTERMS * R));
            CK(cudaMalloc(&b->d_ex_lams, sizeof(LamState*) * R));
        }
        CK(cudaMemcpy(b->d_ladder, ladder, sizeof(int) * n, cudaMemcpyHostToDevice));
        CK(cudaMemset(b->d_ex_ctr, 0, sizeof(unsigned long long) * R));
        CK(cudaMemset(b->d_ex_terms, 0, sizeof(double) * LFE_NTERMS * R));
        b->ex_members.assign(ladder, ladder + n);
        b->ex_n = n;
        b->ex_seed = seed;
        b->ex_beta = 1.0 / (lfe::KB * temperature);
        b->ex_stride = stride;
        b->ex_steps = 0;
        if (b->ex_exec) { cudaGraphExecDestroy(b->ex_exec); b->ex_exec = nullptr; }
        if (b->ex_graph) { cudaGraphDestroy(b->ex_graph); b->ex_graph = nullptr; }
    } catch (const Failure& e) {
        b->err = e.msg;
        return e.code;
    }
    return LFE_OK;
}

int lfe_batch_exchange_state(lfe_batch* b, int* ladder, unsigned long long* attempts, unsigned long long* accepted)
{
    if (!b) return LFE_ERR_ARG;
    try {
        if (!b->d_ladder) fail(LFE_ERR_STATE, "no device exchange has been set");
        CK(cudaDeviceSynchronize());
        if (ladder) CK(cudaMemcpy(ladder, b->d_ladder, sizeof(int) * b->ex_n, cudaMemcpyDeviceToHost));
        std::vector<unsigned long long> c(b->sys.size());
        CK(cudaMemcpy(c.data(), b->d_ex_ctr, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost));
        if (attempts) *attempts = c[0];
        if (accepted)
            for (int k = 0; k + 1 < b->ex_n; ++k) accepted[k] = c[1 + k];
    } catch (const Failure& e) {
        b->err = e.msg;
        return e.code;
    }
    return LFE_OK;
}

int lfe_batch_time_pairs(lfe_batch* b, int reps, double* ms, void* stream)
{
    if (!b || reps <= 0 || !ms) return LFE_ERR_ARG;
    try {
        *ms = b->time_pairs(reps, (cudaStream_t)stream);
    } catch (const Failure& e) {
        b->err = e.msg;
        return e.code;
    }
    return LFE_OK;
}

void lfe_batch_destroy(lfe_batch* b) { delete b; }

const char* lfe_batch_last_error(const lfe_batch* b) { return lfe_batch_last_error_impl(b); }

const char* lfe_last_error(const lfe_system* sys)
{
    if (!sys) return g_create_error.c_str();
    return sys->err.c_str();
}

void lfe_destroy(lfe_system* sys) { delete sys; }

}  // extern "C"

template struct System<float>;
template struct System<double>;
