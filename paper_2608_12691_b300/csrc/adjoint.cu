// adjoint.cu -- derivatives of U(lambda) and dU/dlambda with respect to the
// solute atoms' charges and Lennard-Jones sigma and epsilon (the gradients
// force-field fitting to solvation free energies needs), and the device side
// of replacing those parameters.
//
// U(lambda) = U_vv + U_uu + h_A U_uv + h_B U_soft (Eq. 4) is linear in the
// bases, so for a solute parameter p_i
//   dU/dp_i            = dU_uu/dp_i + h_A dU_uv/dp_i + h_B dU_soft/dp_i
//   d2U/(dlambda dp_i) = h_A' dU_uv/dp_i + h_B' dU_soft/dp_i,
// and every basis derivative is a sum over the atom's interactions:
//   charge:  k_e q_j erfc(alpha r)/r over non-excluded pairs within r_c,
//            -k_e q_j erf(alpha r)/r over excluded partners, s_C k_e q_j / r
//            over 1-4 partners, the self term -2 k_e alpha q_i / sqrt(pi),
//            the background share -k_e pi Q_c / (V alpha^2), and the smooth-PME
//            reciprocal potential of each class at the atom's site;
//   sigma:   sigma_ij = (sigma_i + sigma_j)/2 enters the switched LJ, the 1-4
//            LJ and the capped soft basis (Eq. 5-6) with weight 1/2;
//   epsilon: eps_ij = sqrt(eps_i eps_j), so dE/deps_i = E/(2 eps_i)
//            (0 where eps_i = 0, where the derivative is singular).
// One block per solute atom recomputes its interactions from the current
// positions (no per-pair state is kept between the forward evaluation and
// this pass): it scans every cluster slot for partners within r_c, its own
// exclusion and 1-4 lists, and the 4x4x4 B-spline stencil of an FP64
// potential grid.  Everything is FP64 and every sum is a fixed-order block
// reduction, so the result is reproducible bit for bit.
#include "lfe_views.cuh"
#include "pme_dev.cuh"

namespace lfe {

namespace {

constexpr int PG_THREADS = 256;
constexpr int PG_EX_SMEM = 256;    // exclusion partners staged in shared memory
constexpr int PG_NACC = 10;

// accumulator slots
enum { A_Q_OWN = 0, A_Q_UV, A_S_OWN, A_S_UV, A_S_SOFT, A_E_OWN, A_E_UV, A_E_SOFT, A_QV, A_QU };

__device__ __forceinline__ void min_image(double d[3], const AdjConst& c)
{
    for (int k = 0; k < 3; ++k) d[k] -= c.L[k] * rint(d[k] * c.invL[k]);
}

// quintic LJ switch S(r) (1 below r_sw; swi = 0 means no switch)
__device__ __forceinline__ double lj_switch(double r, const AdjConst& c)
{
    const double t = fmax(0.0, (r - c.rsw) * c.swi);
    return 1.0 - t * t * t * (10.0 - 15.0 * t + 6.0 * t * t);
}

// capped soft-LJ reduced potential u_cap(x) and du/dx (Eq. 6): a degree-6
// polynomial below x = 1, the plain 4 x^-12 - 4 x^-6 above
__device__ __forceinline__ double ucap(double x, double& du)
{
    if (x < 1.0) {
        const double x2 = x * x, x3 = x2 * x, x4 = x2 * x2;
        du = ((-5208.0 * x2 + 10944.0 * x) - 5760.0) * x3;
        return ((-868.0 * x2 + 2188.8 * x) - 1440.0) * x4 + 119.2;
    }
    const double i2 = 1.0 / (x * x), i6 = i2 * i2 * i2;
    du = (-48.0 * i6 * i6 + 24.0 * i6) / x;
    return 4.0 * (i6 * i6 - i6);
}

}  // namespace

template <typename real>
__global__ void __launch_bounds__(PG_THREADS) k_param_grad(SysView<real> s, NblView<real> nb, ExclView<real> ex,
                                                           PmeView<real> pm, const R2<double>* phi, AdjConst c,
                                                           double* dU, double* d2U, double* basis)
{
    __shared__ int ex_sh[PG_EX_SMEM];
    __shared__ double red[PG_NACC][PG_THREADS / 32];
    const int b = blockIdx.x;
    const int tid = threadIdx.x;
    const int a = s.solute_list[b];
    const R4<real> pa = s.xq[s.iperm[a]];
    const double xa[3] = {(double)pa.x, (double)pa.y, (double)pa.z};
    const double sa = (double)s.sig[a], ea = (double)s.eps[a];
    const int mol_a = nb.mol[a];
    const int e0 = nb.ex_start[a], ne = nb.ex_start[a + 1] - e0;
    const bool ex_in_smem = ne <= PG_EX_SMEM;
    for (int e = tid; e < min(ne, PG_EX_SMEM); e += PG_THREADS) ex_sh[e] = nb.ex_list[e0 + e];
    __syncthreads();

    double acc[PG_NACC];
    for (int k = 0; k < PG_NACC; ++k) acc[k] = 0.0;

    // ---------------------------------------------- non-excluded pairs
    for (int j = tid; j < s.n_pad; j += PG_THREADS) {
        const int aj = s.perm[j];
        if (aj < 0) continue;
        const double qj = (double)s.q[aj];
        const bool uj = s.sol[aj] != 0;
        acc[uj ? A_QU : A_QV] += qj;
        if (aj == a) continue;
        const R4<real> pj = s.xq[j];
        double d[3] = {(double)pj.x - xa[0], (double)pj.y - xa[1], (double)pj.z - xa[2]};
        min_image(d, c);
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(r2 < c.rc2)) continue;
        if (nb.mol[aj] == mol_a) {
            bool excluded = false;
            if (ex_in_smem) {
                for (int e = 0; e < ne; ++e) excluded |= (ex_sh[e] == aj);
            } else {
                for (int e = 0; e < ne; ++e) excluded |= (nb.ex_list[e0 + e] == aj);
            }
            if (excluded) continue;
        }
        const double r = sqrt(r2);
        const int cls = uj ? 0 : 1;    // 0: the solute's own class (uu), 1: uv
        acc[A_Q_OWN + cls] += KE * qj * erfc(c.alpha * r) / r;
        const double sg = 0.5 * (sa + (double)s.sig[aj]);
        const double ep = sqrt(ea * (double)s.eps[aj]);
        if (ep > 0.0) {
            const double S = lj_switch(r, c);
            const double s2 = sg * sg / r2, s6 = s2 * s2 * s2;
            acc[A_S_OWN + cls] += 12.0 * ep / sg * (2.0 * s6 * s6 - s6) * S;
            if (ea > 0.0) acc[A_E_OWN + cls] += 4.0 * ep * (s6 * s6 - s6) * S / (2.0 * ea);
            if (cls == 1 && sg > 0.0) {
                const double x = r / sg;
                double du;
                const double u = ucap(x, du);
                acc[A_S_SOFT] += -ep * du * x / (2.0 * sg) * S;
                if (ea > 0.0) acc[A_E_SOFT] += ep * u * S / (2.0 * ea);
            }
        }
    }

    // ------------------------------------------- excluded partners: -erf
    for (int e = tid; e < ne; e += PG_THREADS) {
        const int aj = nb.ex_list[e0 + e];
        const R4<real> pj = s.xq[s.iperm[aj]];
        double d[3] = {(double)pj.x - xa[0], (double)pj.y - xa[1], (double)pj.z - xa[2]};
        min_image(d, c);
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double f = r < 1e-12 ? c.two_a_sqrtpi : erf(c.alpha * r) / r;
        acc[A_Q_OWN + (s.sol[aj] ? 0 : 1)] -= KE * (double)s.q[aj] * f;
    }

    // ----------------------------------------------------- 1-4 partners
    for (int e = tid; e < ex.n14; e += PG_THREADS) {
        const int2 pr = ex.p14[e];
        int aj;
        if (pr.x == a) aj = pr.y;
        else if (pr.y == a) aj = pr.x;
        else continue;
        const R2<double> sc = ex.s14d[e];
        const R4<real> pj = s.xq[s.iperm[aj]];
        double d[3] = {(double)pj.x - xa[0], (double)pj.y - xa[1], (double)pj.z - xa[2]};
        min_image(d, c);
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double r = sqrt(r2);
        const int cls = s.sol[aj] ? 0 : 1;
        acc[A_Q_OWN + cls] += sc.y * KE * (double)s.q[aj] / r;
        const double sg = 0.5 * (sa + (double)s.sig[aj]);
        const double ep = sqrt(ea * (double)s.eps[aj]);
        if (ep > 0.0) {
            const double s2 = sg * sg / r2, s6 = s2 * s2 * s2;
            acc[A_S_OWN + cls] += sc.x * 12.0 * ep / sg * (2.0 * s6 * s6 - s6);
            if (ea > 0.0) acc[A_E_OWN + cls] += sc.x * 4.0 * ep * (s6 * s6 - s6) / (2.0 * ea);
        }
    }

    // ---------------- reciprocal: class potentials at the atom's site
    // phi holds phi_v (real part) and phi_u (imaginary part) on the grid;
    // dU_uu/dq_i gets phi_u(r_i), dU_uv/dq_i gets phi_v(r_i)
    if (tid < 64) {
        const int j0 = tid >> 4, j1 = (tid >> 2) & 3, j2 = tid & 3;
        const real xs[3] = {pa.x, pa.y, pa.z};
        double th[3][4], dth[4];
        int f[3];
        for (int dd = 0; dd < 3; ++dd) {
            double w;
            grid_coord(xs[dd], pm.kscale64[dd], pm.K[dd], f[dd], w);
            bspline4(w, th[dd], dth);
        }
        const int k0 = wrapk(f[0] - j0, pm.K[0]), k1 = wrapk(f[1] - j1, pm.K[1]), k2 = wrapk(f[2] - j2, pm.K[2]);
        const double w = th[0][j0] * th[1][j1] * th[2][j2];
        const R2<double> z = phi[(k0 * pm.K[1] + k1) * pm.K[2] + k2];
        acc[A_Q_OWN] += w * z.y;
        acc[A_Q_UV] += w * z.x;
    }

    // --------------------------------------------- fixed-order reduction
    const int lane = tid & 31, warp = tid >> 5;
    for (int k = 0; k < PG_NACC; ++k) {
        const double v = warp_sum_d(acc[k]);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double g[PG_NACC];
        for (int k = 0; k < PG_NACC; ++k) {
            double v = 0.0;
            for (int w = 0; w < PG_THREADS / 32; ++w) v += red[k][w];
            g[k] = v;
        }
        // self term and the solute's shares of the neutralising background
        g[A_Q_OWN] += -c.two_a_sqrtpi * KE * (double)s.q[a] + 2.0 * c.bg_pre * g[A_QU];
        g[A_Q_UV] += 2.0 * c.bg_pre * g[A_QV];
        const double G[3][3] = {{g[A_Q_OWN], g[A_Q_UV], 0.0},
                                {g[A_S_OWN], g[A_S_UV], g[A_S_SOFT]},
                                {g[A_E_OWN], g[A_E_UV], g[A_E_SOFT]}};
        const LamState L = *s.lam;
        for (int p = 0; p < 3; ++p) {
            if (basis)
                for (int k = 0; k < 3; ++k) basis[9 * b + 3 * p + k] = G[p][k];
            dU[3 * b + p] = G[p][0] + L.hA * G[p][1] + L.hB * G[p][2];
            d2U[3 * b + p] = L.dhA * G[p][1] + L.dhB * G[p][2];
        }
    }
}

template <typename real>
void launch_param_grad(const SysView<real>& s, const NblView<real>& nb, const ExclView<real>& ex,
                       const PmeView<real>& pm, const R2<double>* phi, const AdjConst& c, double* dU,
                       double* d2U, double* basis, cudaStream_t st)
{
    if (s.n_u == 0) return;
    k_param_grad<real><<<s.n_u, PG_THREADS, 0, st>>>(s, nb, ex, pm, phi, c, dU, d2U, basis);
}

// Replace the solute atoms' charges, sigma and epsilon (stage: [3][n_u] in
// solute caller order) and refresh their cluster-sorted copies in place with
// the same expressions the neighbour build uses.
template <typename real>
__global__ void k_set_solute_params(SysView<real> s, real* q, real* sig, real* eps, const double* stage)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= s.n_u) return;
    const int a = s.solute_list[b];
    q[a] = (real)stage[b];
    sig[a] = (real)stage[s.n_u + b];
    eps[a] = (real)stage[2 * s.n_u + b];
    const int slot = s.iperm[a];
    R4<real> o = s.xq[slot];
    o.w = q[a] * (real)sqrt(KE);
    s.xq[slot] = o;
    R2<real> l;
    l.x = (real)0.5 * sig[a];
    l.y = (real)2 * sqrt(eps[a]);
    s.lj[slot] = l;
}

template <typename real>
void launch_set_solute_params(const SysView<real>& s, real* q, real* sig, real* eps, const double* stage,
                              cudaStream_t st)
{
    if (s.n_u == 0) return;
    k_set_solute_params<real><<<(s.n_u + 127) / 128, 128, 0, st>>>(s, q, sig, eps, stage);
}

#define LFE_INST(real)                                                                                        \
    template void launch_param_grad<real>(const SysView<real>&, const NblView<real>&, const ExclView<real>&,  \
                                          const PmeView<real>&, const R2<double>*, const AdjConst&, double*, \
                                          double*, double*, cudaStream_t);                                   \
    template void launch_set_solute_params<real>(const SysView<real>&, real*, real*, real*, const double*,    \
                                                 cudaStream_t);
LFE_INST(float)
LFE_INST(double)
#undef LFE_INST

}  // namespace lfe
