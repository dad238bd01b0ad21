// dyn.cu -- bonded terms, outputs, the Langevin middle-scheme integrator with
// constraint groups, and the theta / dual-OPES update (all per-step kernels
// that are not pair or PME work).
#include "lfe_views.cuh"

namespace lfe {

template <typename real>
__device__ __forceinline__ real minimg(real d, real L, real invL)
{
    return d - L * rint(d * invL);
}
__device__ __forceinline__ float minimg(float d, float L, float invL) { return d - L * rintf(d * invL); }

// One coordinate of the cluster-sorted copy used by the pair and PME
// kernels: the wrapped position at the last list build plus the (minimum-
// image) displacement since.  It is not re-wrapped between builds: the
// periodic shift stored with each tile refers to the images of the build, so
// an atom that crosses a box face must keep a continuous coordinate (it may
// leave [0, L) by at most skin/2 before the next build).
template <typename real>
__device__ __forceinline__ real sorted_coord(real x, real xref, real L, real invL)
{
    return wrap_box(xref, L, invL) + minimg(x - xref, L, invL);
}

template <typename real>
__device__ __forceinline__ void add_force(const SysView<real>& s, int atom, real fx, real fy, real fz)
{
    atomic_add_ll(&s.Fa[atom], to_fixed(fx, FSCALE));
    atomic_add_ll(&s.Fa[s.n + atom], to_fixed(fy, FSCALE));
    atomic_add_ll(&s.Fa[2 * s.n + atom], to_fixed(fz, FSCALE));
}

// ------------------------------------------------------------ set lambda
template <typename real>
__global__ void k_set_lambda(SysView<real> s, double lam)
{
    LamState* L = s.lam;
    double hA, hB, dA, dB;
    switching_fns(lam, hA, hB, dA, dB);
    L->lambda = lam; L->hA = hA; L->hB = hB; L->dhA = dA; L->dhB = dB;
}

template <typename real>
void launch_set_lambda(const SysView<real>& s, double lam, cudaStream_t st)
{
    k_set_lambda<real><<<1, 1, 0, st>>>(s, lam);
}

// --------------------------------------------------------------- outputs
__device__ __forceinline__ double efix(const long long* E, int k) { return (double)E[k] * (1.0 / ESCALE); }

template <typename real>
__global__ void k_eval_out(SysView<real> s, double* forces, double* terms, double cvv, double cuu, double cuv)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < s.n) {
        const int slot = s.iperm[a];
        const long long fx = s.F[slot] + s.Fa[a], fy = s.F[s.n_pad + slot] + s.Fa[s.n + a],
                        fz = s.F[2 * s.n_pad + slot] + s.Fa[2 * s.n + a];
        s.F[slot] = 0; s.F[s.n_pad + slot] = 0; s.F[2 * s.n_pad + slot] = 0;
        s.Fa[a] = 0; s.Fa[s.n + a] = 0; s.Fa[2 * s.n + a] = 0;
        if (forces) {
            forces[3 * a] = (double)fx * (1.0 / FSCALE);
            forces[3 * a + 1] = (double)fy * (1.0 / FSCALE);
            forces[3 * a + 2] = (double)fz * (1.0 / FSCALE);
            if (!isfinite(forces[3 * a]) || !isfinite(forces[3 * a + 1]) || !isfinite(forces[3 * a + 2]))
                atomicOr(&s.flags[FL_ERROR], ERRB_NONFINITE);
        }
    }
    // one thread of the last block finalises the energies after all blocks
    // have read their forces (energies are independent of the force slots)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long* E = s.E;
        LamState* L = s.lam;
        const double Uvv = efix(E, E_PAIR_VV) + efix(E, E_EXCL_VV) + efix(E, E_14_VV) + efix(E, E_REC_VV) + cvv;
        const double Uuu = efix(E, E_PAIR_UU) + efix(E, E_EXCL_UU) + efix(E, E_14_UU) + efix(E, E_REC_UU) + cuu;
        const double Uuv = efix(E, E_PAIR_UV) + efix(E, E_EXCL_UV) + efix(E, E_14_UV) + efix(E, E_REC_UV) + cuv;
        const double Us = efix(E, E_PAIR_SOFT);
        const double Ub = efix(E, E_BONDED);
        // soft-core coupling: U_soft is already the soft-core term at lambda
        const bool sc = s.sc_alpha > 0.0;
        const double U = Uvv + Uuu + L->hA * Uuv + (sc ? Us : L->hB * Us) + Ub + efix(E, E_DAFED);
        const double dU = L->dhA * Uuv + (sc ? efix(E, E_DSC) : L->dhB * Us);
        if (terms) {
            terms[0] = U; terms[1] = dU; terms[2] = Uvv; terms[3] = Uuu; terms[4] = Uuv;
            terms[5] = Us; terms[6] = Ub; terms[7] = (double)E[E_NPAIRS]; terms[8] = L->hA; terms[9] = L->hB;
        }
        L->U = U;
        L->dUdl = dU;
        if (!isfinite(U) || !isfinite(dU)) atomicOr(&s.flags[FL_ERROR], ERRB_NONFINITE);
        for (int k = 0; k < E_N; ++k) E[k] = 0;
    }
}

template <typename real>
void launch_eval_out(const SysView<real>& s, double* forces, double* terms, double cvv, double cuu, double cuv,
                     cudaStream_t st)
{
    k_eval_out<real><<<(s.n + 255) / 256, 256, 0, st>>>(s, forces, terms, cvv, cuu, cuv);
}

template <typename real>
__global__ void k_refresh_sorted(SysView<real> s)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const int slot = s.iperm[a];
    const R4<real> x = s.x[a], xr = s.xref[a];
    R4<real> o = s.xq[slot];
    o.x = sorted_coord(x.x, xr.x, s.L[0], s.invL[0]);
    o.y = sorted_coord(x.y, xr.y, s.L[1], s.invL[1]);
    o.z = sorted_coord(x.z, xr.z, s.L[2], s.invL[2]);
    s.xq[slot] = o;
}

template <typename real>
void launch_refresh_sorted(const SysView<real>& s, cudaStream_t st)
{
    k_refresh_sorted<real><<<(s.n + 255) / 256, 256, 0, st>>>(s);
}

// new positions from caller doubles (caller order): assign the master copy,
// refresh the cluster-sorted copy in the current slot order, and raise the
// rebuild flag when an atom lies more than skin/2 from where the list was
// built (a non-finite position raises it too)
template <typename real, typename TIO>
__global__ void k_assign_moved(SysView<real> s, const TIO* pos, real skin_half2, real prune_half2)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (s.flags[FL_ERROR] & ERRB_BADPOS) return;   // refused by k_check_positions: nothing changes
    bool far = false, pfar = false;
    if (a < s.n) {
        const int slot = s.iperm[a];
        const R4<real> x{(real)pos[3 * a], (real)pos[3 * a + 1], (real)pos[3 * a + 2], (real)0};
        s.x[a] = x;
        const R4<real> xr = s.xref[a];
        R4<real> o = s.xq[slot];
        o.x = sorted_coord(x.x, xr.x, s.L[0], s.invL[0]);
        o.y = sorted_coord(x.y, xr.y, s.L[1], s.invL[1]);
        o.z = sorted_coord(x.z, xr.z, s.L[2], s.invL[2]);
        s.xq[slot] = o;
        const real dx = minimg(x.x - xr.x, s.L[0], s.invL[0]);
        const real dy = minimg(x.y - xr.y, s.L[1], s.invL[1]);
        const real dz = minimg(x.z - xr.z, s.L[2], s.invL[2]);
        far = !(dx * dx + dy * dy + dz * dz <= skin_half2);
        if (prune_half2 > (real)0) {
            const R4<real> xp = s.xpr[a];
            const real ex = minimg(x.x - xp.x, s.L[0], s.invL[0]);
            const real ey = minimg(x.y - xp.y, s.L[1], s.invL[1]);
            const real ez = minimg(x.z - xp.z, s.L[2], s.invL[2]);
            pfar = !(ex * ex + ey * ey + ez * ez <= prune_half2);
        }
    }
    const bool any_far = __any_sync(0xffffffffu, far), any_pfar = __any_sync(0xffffffffu, pfar);
    if ((threadIdx.x & 31) == 0) {
        if (any_far) atomicOr(&s.flags[FL_REBUILD], 1);
        if (any_pfar) atomicOr(&s.flags[FL_PRUNE], 1);
    }
}

template <typename real, typename TIO>
void launch_assign_moved(const SysView<real>& s, const TIO* pos, real skin_half2, real prune_half2, cudaStream_t st)
{
    k_assign_moved<real, TIO><<<(s.n + 255) / 256, 256, 0, st>>>(s, pos, skin_half2, prune_half2);
}

// new positions (caller doubles or floats) checked on the device before
// they are assigned: any coordinate that is not finite raises ERRB_BADPOS,
// and the step that follows leaves the state as it was
template <typename real, typename TIO>
__global__ void k_check_positions(SysView<real> s, const TIO* pos)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = i < 3 * s.n && !isfinite(pos[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&s.flags[FL_ERROR], ERRB_BADPOS);
}

template <typename real, typename TIO>
void launch_check_positions(const SysView<real>& s, const TIO* pos, cudaStream_t st)
{
    k_check_positions<real, TIO><<<(3 * s.n + 255) / 256, 256, 0, st>>>(s, pos);
}

// Monte Carlo volume move (the NPT runs of Section 2.6): every molecule's
// centre of mass (its geometric centre when all its atoms are massless) is
// scaled by sc, its atoms moved rigidly with it; offsets from the molecule's
// first atom are taken under the minimum image of the old box, in FP64.
// One thread per molecule (molecules as CSR over caller-order atoms).
template <typename real>
__global__ void k_scale_molecules(SysView<real> s, const int* mstart, const int* matoms, const double* mass,
                                  int n_mol, double sc, double L0, double L1, double L2)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_mol) return;
    const int b = mstart[m], e = mstart[m + 1];
    const double L[3] = {L0, L1, L2};
    const R4<real> p0r = s.x[matoms[b]];
    const double p0[3] = {(double)p0r.x, (double)p0r.y, (double)p0r.z};
    double c[3] = {0, 0, 0}, cu[3] = {0, 0, 0}, wsum = 0;
    for (int k = b; k < e; ++k) {
        const R4<real> p = s.x[matoms[k]];
        const double w = mass[matoms[k]];
        const double pv[3] = {(double)p.x, (double)p.y, (double)p.z};
        for (int d = 0; d < 3; ++d) {
            double dd = pv[d] - p0[d];
            dd -= L[d] * rint(dd / L[d]);
            c[d] += w * dd;
            cu[d] += dd;
        }
        wsum += w;
    }
    const int na = e - b;
    for (int d = 0; d < 3; ++d) c[d] = wsum > 0.0 ? c[d] / wsum : cu[d] / na;
    for (int k = b; k < e; ++k) {
        const int a = matoms[k];
        const R4<real> p = s.x[a];
        const double pv[3] = {(double)p.x, (double)p.y, (double)p.z};
        double q[3];
        for (int d = 0; d < 3; ++d) {
            double dd = pv[d] - p0[d];
            dd -= L[d] * rint(dd / L[d]);
            q[d] = sc * (p0[d] + c[d]) + (dd - c[d]);
        }
        s.x[a] = R4<real>{(real)q[0], (real)q[1], (real)q[2], p.w};
    }
}

template <typename real>
void launch_scale_molecules(const SysView<real>& s, const int* mstart, const int* matoms, const double* mass,
                            int n_mol, double sc, const double* L, cudaStream_t st)
{
    if (n_mol == 0) return;
    k_scale_molecules<real><<<(n_mol + 127) / 128, 128, 0, st>>>(s, mstart, matoms, mass, n_mol, sc, L[0], L[1],
                                                                    L[2]);
}

// positions, velocities (caller order, doubles) and the scalar state in one
// buffer, so that lfe_get_state needs one copy: out[0, 3n) x, [3n, 6n) v,
// then theta, p_theta, lambda, dU/dlambda, U, kernels of both biases, step,
// rebuilds, the error bits, the tile count
template <typename real, typename TIO>
__global__ void k_pack_state(SysView<real> s, const OpesState* o, TIO* out, double* e)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < s.n) {
        const R4<real> x = s.x[a], v = s.v[a];
        out[3 * a] = (TIO)x.x; out[3 * a + 1] = (TIO)x.y; out[3 * a + 2] = (TIO)x.z;
        TIO* ov = out + 3 * (size_t)s.n;
        ov[3 * a] = (TIO)v.x; ov[3 * a + 1] = (TIO)v.y; ov[3 * a + 2] = (TIO)v.z;
    }
    if (a == 0) {
        const LamState* L = s.lam;
        e[0] = L->theta; e[1] = L->p_theta; e[2] = L->lambda; e[3] = L->dUdl; e[4] = L->U;
        e[5] = o->n[0]; e[6] = o->n[1]; e[7] = (double)L->step;
        e[8] = s.flags[FL_NREBUILD]; e[9] = s.flags[FL_NTILES]; e[10] = L->npairs; e[11] = s.flags[FL_PTILES];
        e[12] = s.flags[FL_NPRUNE]; e[13] = s.flags[FL_ERROR];
    }
}

template <typename real>
void launch_pack_state(const SysView<real>& s, const OpesState* o, double* out, cudaStream_t st)
{
    k_pack_state<real, double><<<(s.n + 255) / 256, 256, 0, st>>>(s, o, out, out + 6 * (size_t)s.n);
}

// the same with positions and velocities as floats (xv [6n]) and the scalar
// state (tail [16]) in FP64
template <typename real>
void launch_pack_state_f32(const SysView<real>& s, const OpesState* o, float* xv, double* tail, cudaStream_t st)
{
    k_pack_state<real, float><<<(s.n + 255) / 256, 256, 0, st>>>(s, o, xv, tail);
}

// Dihedral of atoms (i, j, k, l) from r_ij = x_i - x_j, r_kj = x_k - x_j,
// r_kl = x_k - x_l (minimum images): phi = atan2(|r_kj| r_ij . n, m . n) with
// m = r_ij x r_kj, n = r_kj x r_kl (the IUPAC sign), and the forces
// -dU/dphi grad phi on the four atoms for a given dU/dphi.
template <typename T>
struct Torsion {
    T m[3], n[3], m2, n2, rkj2, lkj, p, q;
    __device__ __forceinline__ T angle(const T* rij, const T* rkj, const T* rkl)
    {
        m[0] = rij[1] * rkj[2] - rij[2] * rkj[1];
        m[1] = rij[2] * rkj[0] - rij[0] * rkj[2];
        m[2] = rij[0] * rkj[1] - rij[1] * rkj[0];
        n[0] = rkj[1] * rkl[2] - rkj[2] * rkl[1];
        n[1] = rkj[2] * rkl[0] - rkj[0] * rkl[2];
        n[2] = rkj[0] * rkl[1] - rkj[1] * rkl[0];
        m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
        n2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        rkj2 = rkj[0] * rkj[0] + rkj[1] * rkj[1] + rkj[2] * rkj[2];
        lkj = sqrt(rkj2);
        p = (rij[0] * rkj[0] + rij[1] * rkj[1] + rij[2] * rkj[2]) / rkj2;
        q = (rkl[0] * rkj[0] + rkl[1] * rkj[1] + rkl[2] * rkj[2]) / rkj2;
        const T yv = lkj * (rij[0] * n[0] + rij[1] * n[1] + rij[2] * n[2]);
        const T xv = m[0] * n[0] + m[1] * n[1] + m[2] * n[2];
        return atan2(yv, xv);
    }
    __device__ __forceinline__ void forces(T dUdphi, T* fi, T* fj, T* fk, T* fl) const
    {
        for (int k = 0; k < 3; ++k) {
            fi[k] = -dUdphi * lkj / m2 * m[k];
            fl[k] = dUdphi * lkj / n2 * n[k];
        }
        for (int k = 0; k < 3; ++k) {
            fj[k] = -fi[k] + p * fi[k] - q * fl[k];
            fk[k] = -fl[k] - p * fi[k] + q * fl[k];
        }
    }
};

// ---------------------------------------------------------------- bonded
// harmonic bonds 1/2 k (r - r0)^2, harmonic angles 1/2 k (theta - theta0)^2,
// periodic torsions k (1 + cos(n phi - phi0)); minimum-image vectors
template <typename real>
__global__ void k_bonded(SysView<real> s, BondView<real> b)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double en = 0.0;
    const real* L = s.L;
    const real* iL = s.invL;
    auto vec = [&](int i, int j, real* d) {
        R4<real> pi = s.x[i], pj = s.x[j];
        d[0] = minimg(pj.x - pi.x, L[0], iL[0]);
        d[1] = minimg(pj.y - pi.y, L[1], iL[1]);
        d[2] = minimg(pj.z - pi.z, L[2], iL[2]);
    };
    if (e < b.nb) {
        const int2 ij = b.b[e];
        const R2<real> par = b.bp[e];
        real d[3];
        vec(ij.x, ij.y, d);
        const real r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const real dr = r - par.y;
        en = 0.5 * (double)par.x * (double)dr * (double)dr;
        const real g = par.x * dr / r;   // dU/dr / r; force on i = +g d
        add_force(s, ij.x, g * d[0], g * d[1], g * d[2]);
        add_force(s, ij.y, -g * d[0], -g * d[1], -g * d[2]);
    } else if (e < b.nb + b.na) {
        const int4 t = b.a[e - b.nb];
        const R2<real> par = b.ap[e - b.nb];
        real u[3], v[3];
        vec(t.y, t.x, u);   // vertex -> i
        vec(t.y, t.z, v);   // vertex -> k
        const real lu2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const real lv2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const real luv = sqrt(lu2 * lv2);
        real c = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / luv;
        c = fmin((real)1, fmax((real)-1, c));
        const real th = acos(c);
        const real dth = th - par.y;
        en = 0.5 * (double)par.x * (double)dth * (double)dth;
        real sn = sqrt(fmax((real)1e-24, (real)1 - c * c));
        const real pre = par.x * dth / sn;   // F = pre * dc/dx
        real fi[3], fk[3];
        for (int k = 0; k < 3; ++k) {
            fi[k] = pre * (v[k] / luv - c * u[k] / lu2);
            fk[k] = pre * (u[k] / luv - c * v[k] / lv2);
        }
        add_force(s, t.x, fi[0], fi[1], fi[2]);
        add_force(s, t.z, fk[0], fk[1], fk[2]);
        add_force(s, t.y, -fi[0] - fk[0], -fi[1] - fk[1], -fi[2] - fk[2]);
    } else if (e < b.nb + b.na + b.nt) {
        const int4 t = b.t[e - b.nb - b.na];
        const R4<real> par = b.tp[e - b.nb - b.na];
        // r_ij = x_i - x_j, r_kj = x_k - x_j, r_kl = x_k - x_l
        real rij[3], rkj[3], rkl[3];
        vec(t.y, t.x, rij);
        vec(t.y, t.z, rkj);
        vec(t.w, t.z, rkl);
        Torsion<real> tor;
        const real phi = tor.angle(rij, rkj, rkl);
        const real arg = par.y * phi - par.z;
        en = (double)par.x * (1.0 + cos((double)arg));
        const real dUdphi = -par.x * par.y * sin(arg);
        real fi[3], fl[3], fj[3], fk[3];
        tor.forces(dUdphi, fi, fj, fk, fl);
        add_force(s, t.x, fi[0], fi[1], fi[2]);
        add_force(s, t.y, fj[0], fj[1], fj[2]);
        add_force(s, t.z, fk[0], fk[1], fk[2]);
        add_force(s, t.w, fl[0], fl[1], fl[2]);
    }
    long long v = __double2ll_rn(warp_sum_d(en) * ESCALE);
    if ((threadIdx.x & 31) == 0 && v) atomic_add_ll(&s.E[E_BONDED], v);
}

template <typename real>
void launch_bonded(const SysView<real>& s, const BondView<real>& b, cudaStream_t st)
{
    const int n = b.nb + b.na + b.nt;
    if (n == 0) return;
    k_bonded<real><<<(n + 255) / 256, 256, 0, st>>>(s, b);
}

// ------------------------------------------------------------------ d-AFED
// Eq. 15: U = sum_k kappa_k / 2 wrap(xi_k - s_k)^2 with wrap into [-pi, pi).
// One thread per coupled torsion, FP64 geometry from the master positions.
__device__ __forceinline__ double wrap_pi(double x)
{
    return x - 2.0 * PI * floor((x + PI) / (2.0 * PI));
}

template <typename real>
__device__ __forceinline__ double dafed_geom(const SysView<real>& s, int4 t, Torsion<double>& tor)
{
    auto vec = [&](int i, int j, double* d) {
        const R4<real> pi = s.x[i], pj = s.x[j];
        const double dd[3] = {(double)pj.x - (double)pi.x, (double)pj.y - (double)pi.y, (double)pj.z - (double)pi.z};
        for (int k = 0; k < 3; ++k) d[k] = dd[k] - (double)s.L[k] * rint(dd[k] / (double)s.L[k]);
    };
    double rij[3], rkj[3], rkl[3];
    vec(t.y, t.x, rij);
    vec(t.y, t.z, rkj);
    vec(t.w, t.z, rkl);
    return tor.angle(rij, rkj, rkl);
}

template <typename real>
__global__ void k_dafed_force(SysView<real> s, DafedView d)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double en = 0.0;
    if (k < d.n) {
        const int4 t = d.atoms[k];
        Torsion<double> tor;
        const double xi = dafed_geom(s, t, tor);
        const double dl = wrap_pi(xi - d.s[k]);
        en = 0.5 * d.kappa[k] * dl * dl;
        double fi[3], fj[3], fk[3], fl[3];
        tor.forces(d.kappa[k] * dl, fi, fj, fk, fl);
        add_force(s, t.x, (real)fi[0], (real)fi[1], (real)fi[2]);
        add_force(s, t.y, (real)fj[0], (real)fj[1], (real)fj[2]);
        add_force(s, t.z, (real)fk[0], (real)fk[1], (real)fk[2]);
        add_force(s, t.w, (real)fl[0], (real)fl[1], (real)fl[2]);
        d.fs[k] = d.kappa[k] * dl;
        d.xi[k] = xi;
    }
    const long long v = __double2ll_rn(warp_sum_d(en) * ESCALE);
    if ((threadIdx.x & 31) == 0 && v) atomic_add_ll(&s.E[E_DAFED], v);
}

// One step of an extended variable (x, p) of mass m under force f at
// temperature kT, with the variable's standard normal n0: the leapfrog
// middle layout (full kick, half drift, thermostat, half drift).  Langevin
// (kind 0): the thermostat is the exact Ornstein-Uhlenbeck step of the
// velocity, a = exp(-gamma dt).  Regulated Nose-Hoover-Langevin (kind 1,
// Section 2.6's thermostat of the extended variables): the drift is the
// regulated velocity K'(p) = sqrt(n kT / m) tanh(p / sqrt(n m kT)) of the
// kinetic function K(p) = n kT ln cosh(p / sqrt(n m kT)), and the
// thermostat is NH(dt/2) OU(dt) NH(dt/2) on (p, v_eta): NH(h) is v_eta +=
// h/2 G; p *= exp(-v_eta h); v_eta += h/2 G with G = (p K'(p) - kT) / Q,
// Q = kT tau^2, and OU the exact Ornstein-Uhlenbeck step of v_eta.  Its
// invariant density is exp(-(U + K(p) + Q v_eta^2 / 2) / kT).
__device__ __forceinline__ void ext_step(const ExtThermo& th, const ExtConst& k, double m, double kT, double dt,
                                         double a_fric, double f, double n0, double& x, double& p, double& v_eta)
{
    if (th.kind == 1) {
        // K'(p) is taken three times (after the kick, after each friction
        // scaling of p): G and the drifts reuse it while p is unchanged
        const double q = 0.25 * dt;
        p += dt * f;
        double u = k.c * tanh(p * k.ipc);
        x += 0.5 * dt * u;
        double ve = v_eta;
        ve += q * (p * u - kT) * k.iQ;
        p *= exp(-ve * 0.5 * dt);
        u = k.c * tanh(p * k.ipc);
        ve += q * (p * u - kT) * k.iQ;
        ve = a_fric * ve + k.amp_eta * n0;
        ve += q * (p * u - kT) * k.iQ;
        p *= exp(-ve * 0.5 * dt);
        u = k.c * tanh(p * k.ipc);
        ve += q * (p * u - kT) * k.iQ;
        x += 0.5 * dt * u;
        v_eta = ve;
    } else {
        double v = (p + dt * f) * k.im;
        x += 0.5 * dt * v;
        v = a_fric * v + k.amp * n0;
        x += 0.5 * dt * v;
        p = m * v;
    }
}

// the auxiliary variables' step at their own temperature (normal from
// Philox at counter (k, step_lo, step_hi, 2))
template <typename real>
__global__ void k_dafed_step(SysView<real> s, DafedView d)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    if (s.flags[FL_ERROR] & ERRB_SKIP) return;   // step skipped (see k_integrate)
    const unsigned long long step = d.pre->step;   // runs beside k_theta, which advances the counter
    double n0, n1, n2;
    normals3<double>(make_uint4((unsigned)k, (unsigned)step, (unsigned)(step >> 32), 2u), d.key, n0, n1, n2);
    double x = d.s[k], p = d.p[k], ve = d.veta ? d.veta[k] : 0.0;
    ext_step(d.th, d.ec[k], d.mass[k], d.kT, d.dt, d.a_fric, d.fs[k], n0, x, p, ve);
    d.s[k] = wrap_pi(x);
    d.p[k] = p;
    if (d.veta) d.veta[k] = ve;
}

template <typename real>
__global__ void k_dafed_probe(SysView<real> s, DafedView d, double c, double* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const int4 t = d.atoms[k];
    Torsion<double> tor;
    const double xi = dafed_geom(s, t, tor);
    if (!(c > 0.0)) {
        out[k] = xi;
        return;
    }
    double g[4][3];
    tor.forces(-1.0, g[0], g[1], g[2], g[3]);   // -dU/dphi grad phi with dU/dphi = -1: grad phi
    const int at[4] = {t.x, t.y, t.z, t.w};
    double tot = 0.0;
    for (int a = 0; a < 4; ++a) {
        const double w = (double)s.invm[at[a]];
        tot += w * (g[a][0] * g[a][0] + g[a][1] * g[a][1] + g[a][2] * g[a][2]);
    }
    out[k] = c / tot;
}

template <typename real>
void launch_dafed_force(const SysView<real>& s, const DafedView& d, cudaStream_t st)
{
    if (d.n == 0) return;
    k_dafed_force<real><<<(d.n + 31) / 32, 32, 0, st>>>(s, d);
}
template <typename real>
void launch_dafed_step(const SysView<real>& s, const DafedView& d, cudaStream_t st)
{
    if (d.n == 0) return;
    k_dafed_step<real><<<(d.n + 31) / 32, 32, 0, st>>>(s, d);
}
template <typename real>
void launch_dafed_probe(const SysView<real>& s, const DafedView& d, double c, double* out, cudaStream_t st)
{
    if (d.n == 0) return;
    k_dafed_probe<real><<<(d.n + 31) / 32, 32, 0, st>>>(s, d, c, out);
}

// ------------------------------------------------------------ integrator
// Langevin middle scheme per constraint group: kick v += dt F/m, half drift,
// Ornstein-Uhlenbeck v = a v + sqrt(kT (1 - a^2)/m) R, half drift, constrain
// the new positions along the old bond vectors (Newton iteration on the
// group's Lagrange multipliers); the velocity carried to the next step is the
// post-noise velocity plus the constraint displacement over dt (for an
// unconstrained atom the post-noise velocity itself).  All of it is done in
// coordinates relative to the group's first atom (small numbers, so FP32
// keeps full relative precision and the velocity comes from the displacement
// itself, not from a difference of two absolute positions).  The group shape
// (single atom, rigid water, X-Hn star) is a template parameter so that every
// array index is a compile-time constant and the state stays in registers.
// Consumes (zeroes) the fixed-point forces, refreshes the sorted coordinates
// and flags a neighbour rebuild when an atom has moved more than skin/2 since
// the last build.
template <int KIND, int NA>
struct Shape {
    static constexpr int NC = KIND == GROUP_WATER ? 3 : NA - 1;
    static __device__ __forceinline__ constexpr int ci(int k) { return KIND == GROUP_WATER ? (k == 2 ? 1 : 0) : 0; }
    static __device__ __forceinline__ constexpr int cj(int k) { return KIND == GROUP_WATER ? (k == 0 ? 1 : 2) : k + 1; }
};

template <typename real, int KIND, int NA>
__device__ __forceinline__ void integrate_group(const SysView<real>& s, const StepView<real>& g, const Group& G,
                                                unsigned long long step)
{
    using Sh = Shape<KIND, NA>;
    constexpr int NC = Sh::NC;
    (void)step;
    real o0[3];
    real rel0[NA][3];
    real p[NA][3];
    real vou[NA][3];   // post-noise velocity
    real pu[NA][3];    // position before the constraints
    real w[NA];
    int slot[NA];
    // every load of the group is issued before any store (the stores that
    // clear the forces would otherwise order the next atom's loads after
    // them), in two dependent rounds: indices and per-atom records, then the
    // slot-indexed forces and sorted records
    R4<real> xa4[NA], va4[NA], xr4[NA], xq4[NA], xp4[NA];
    real kick[NA][3];
    long long fl[NA][3], fla[NA][3];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int atom = G.atom[a];
        slot[a] = s.iperm[atom];
        xa4[a] = s.x[atom];
        va4[a] = s.v[atom];
        xr4[a] = s.xref[atom];
        xp4[a] = g.prune_half2 > (real)0 ? s.xpr[atom] : R4<real>{0, 0, 0, 0};
        w[a] = s.invm[atom];
#pragma unroll
        for (int d = 0; d < 3; ++d) kick[a][d] = g.noise[3 * atom + d];
    }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
#pragma unroll
        for (int d = 0; d < 3; ++d) fl[a][d] = s.F[(size_t)d * s.n_pad + slot[a]];
#pragma unroll
        for (int d = 0; d < 3; ++d) fla[a][d] = s.Fa[(size_t)d * s.n + G.atom[a]];
        xq4[a] = s.xq[slot[a]];
    }
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s.F[(size_t)d * s.n_pad + slot[a]] = 0;
            s.Fa[(size_t)d * s.n + G.atom[a]] = 0;
            fl[a][d] += fla[a][d];
        }
    o0[0] = xa4[0].x; o0[1] = xa4[0].y; o0[2] = xa4[0].z;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const real xa[3] = {xa4[a].x, xa4[a].y, xa4[a].z};
#pragma unroll
        for (int d = 0; d < 3; ++d) rel0[a][d] = a == 0 ? (real)0 : minimg(xa[d] - o0[d], s.L[d], s.invL[d]);
        if (w[a] == (real)0) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                p[a][d] = pu[a][d] = rel0[a][d];
                vou[a][d] = (real)0;
            }
            continue;
        }
        const real vv[3] = {va4[a].x, va4[a].y, va4[a].z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const real f = (real)((double)fl[a][d] * (1.0 / FSCALE));
            real vd = vv[d] + g.dt * w[a] * f;
            real disp = (real)0.5 * g.dt * vd;
            vd = g.a_fric * vd + kick[a][d];
            disp += (real)0.5 * g.dt * vd;
            p[a][d] = pu[a][d] = rel0[a][d] + disp;
            vou[a][d] = vd;
        }
    }
    if (NC > 0) {
        real sref[NC > 0 ? NC : 1][3];
#pragma unroll
        for (int k = 0; k < NC; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) sref[k][d] = rel0[Sh::cj(k)][d] - rel0[Sh::ci(k)][d];
        const real tol = sizeof(real) == 4 ? (real)2e-6 : (real)1e-12;
        bool conv = false;
        for (int it = 0; it < 32; ++it) {
            real r[NC > 0 ? NC : 1][3], sig[NC > 0 ? NC : 1];
            conv = true;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                real r2 = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    r[k][d] = p[Sh::cj(k)][d] - p[Sh::ci(k)][d];
                    r2 += r[k][d] * r[k][d];
                }
                const real l2 = (real)G.len[k] * (real)G.len[k];
                sig[k] = r2 - l2;
                if (fabs(sig[k]) > tol * l2) conv = false;
            }
            if (conv) break;
            // J_kl = 2 r_k . (M_kl s_l), M_kl = w_cj(k) c(cj_k, l) - w_ci(k) c(ci_k, l),
            // c(a, l) = +1 if a is the second atom of constraint l, -1 if the first
            real J[NC > 0 ? NC : 1][NC > 0 ? NC : 1];
#pragma unroll
            for (int k = 0; k < NC; ++k)
#pragma unroll
                for (int l = 0; l < NC; ++l) {
                    const real cjj = Sh::cj(k) == Sh::cj(l) ? (real)1 : (Sh::cj(k) == Sh::ci(l) ? (real)-1 : (real)0);
                    const real cii = Sh::ci(k) == Sh::cj(l) ? (real)1 : (Sh::ci(k) == Sh::ci(l) ? (real)-1 : (real)0);
                    const real M = w[Sh::cj(k)] * cjj - w[Sh::ci(k)] * cii;
                    J[k][l] = (real)2 * M * (r[k][0] * sref[l][0] + r[k][1] * sref[l][1] + r[k][2] * sref[l][2]);
                }
            real dl[NC > 0 ? NC : 1];
            if (NC == 1) {
                dl[0] = -sig[0] / J[0][0];
            } else if (NC == 2) {
                const real det = J[0][0] * J[1][NC - 1] - J[0][NC - 1] * J[NC - 1][0];
                dl[0] = (-sig[0] * J[NC - 1][NC - 1] + sig[NC - 1] * J[0][NC - 1]) / det;
                dl[NC - 1] = (-sig[NC - 1] * J[0][0] + sig[0] * J[NC - 1][0]) / det;
            } else {
                constexpr int A = NC > 2 ? 1 : 0, Bq = NC > 2 ? 2 : 0;
                const real c00 = J[A][A] * J[Bq][Bq] - J[A][Bq] * J[Bq][A];
                const real c01 = J[A][Bq] * J[Bq][0] - J[A][0] * J[Bq][Bq];
                const real c02 = J[A][0] * J[Bq][A] - J[A][A] * J[Bq][0];
                const real det = J[0][0] * c00 + J[0][A] * c01 + J[0][Bq] * c02;
                const real b0 = -sig[0], b1 = -sig[A], b2 = -sig[Bq];
                // Cramer's rule
                dl[0] = (b0 * c00 + J[0][A] * (J[A][Bq] * b2 - b1 * J[Bq][Bq]) + J[0][Bq] * (b1 * J[Bq][A] - J[A][A] * b2)) / det;
                dl[A] = (J[0][0] * (b1 * J[Bq][Bq] - J[A][Bq] * b2) + b0 * c01 + J[0][Bq] * (J[A][0] * b2 - b1 * J[Bq][0])) / det;
                dl[Bq] = (J[0][0] * (J[A][A] * b2 - b1 * J[Bq][A]) + J[0][A] * (b1 * J[Bq][0] - J[A][0] * b2) + b0 * c02) / det;
            }
#pragma unroll
            for (int l = 0; l < NC; ++l)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    p[Sh::cj(l)][d] += dl[l] * w[Sh::cj(l)] * sref[l][d];
                    p[Sh::ci(l)][d] -= dl[l] * w[Sh::ci(l)] * sref[l][d];
                }
        }
        if (!conv) atomicOr(&s.flags[FL_ERROR], ERRB_CONSTRAINT);
    }
    // keep each group near the box: shift it by whole periods when its first
    // atom leaves [0, L)
    real shift[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) shift[d] = -s.L[d] * floor((o0[d] + p[0][d]) * s.invL[d]);
    const real inv_dt = (real)1 / g.dt;
    bool rebuild = false, bad = false, prune = false;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int atom = G.atom[a];
        R4<real> xnew, vnew;
        if (w[a] == (real)0) {
            vnew.x = vnew.y = vnew.z = (real)0;
        } else if (NC == 0) {
            vnew.x = vou[a][0];
            vnew.y = vou[a][1];
            vnew.z = vou[a][2];
        } else {
            vnew.x = vou[a][0] + (p[a][0] - pu[a][0]) * inv_dt;
            vnew.y = vou[a][1] + (p[a][1] - pu[a][1]) * inv_dt;
            vnew.z = vou[a][2] + (p[a][2] - pu[a][2]) * inv_dt;
        }
        vnew.w = (real)0;
        xnew.x = (o0[0] + shift[0]) + p[a][0];
        xnew.y = (o0[1] + shift[1]) + p[a][1];
        xnew.z = (o0[2] + shift[2]) + p[a][2];
        xnew.w = (real)0;
        if (!isfinite(xnew.x) || !isfinite(xnew.y) || !isfinite(xnew.z)) bad = true;
        s.x[atom] = xnew;
        s.v[atom] = vnew;
        const R4<real> xr = xr4[a];
        R4<real> o = xq4[a];
        o.x = sorted_coord(xnew.x, xr.x, s.L[0], s.invL[0]);
        o.y = sorted_coord(xnew.y, xr.y, s.L[1], s.invL[1]);
        o.z = sorted_coord(xnew.z, xr.z, s.L[2], s.invL[2]);
        s.xq[slot[a]] = o;
        const real dx = minimg(xnew.x - xr.x, s.L[0], s.invL[0]);
        const real dy = minimg(xnew.y - xr.y, s.L[1], s.invL[1]);
        const real dz = minimg(xnew.z - xr.z, s.L[2], s.invL[2]);
        if (dx * dx + dy * dy + dz * dz > g.skin_half2) rebuild = true;
        if (g.prune_half2 > (real)0) {
            const R4<real> xp = xp4[a];
            const real ex = minimg(xnew.x - xp.x, s.L[0], s.invL[0]);
            const real ey = minimg(xnew.y - xp.y, s.L[1], s.invL[1]);
            const real ez = minimg(xnew.z - xp.z, s.L[2], s.invL[2]);
            if (ex * ex + ey * ey + ez * ez > g.prune_half2) prune = true;
        }
    }
    // one atomic per warp (thousands of groups cross the skin at once)
    const unsigned act = __activemask();
    const bool any_rebuild = __any_sync(act, rebuild), any_bad = __any_sync(act, bad);
    const bool any_prune = __any_sync(act, prune);
    if ((threadIdx.x & 31) == __ffs(act) - 1) {
        if (any_rebuild && !s.flags[FL_REBUILD]) atomicOr(&s.flags[FL_REBUILD], 1);
        if (any_prune && !s.flags[FL_PRUNE]) atomicOr(&s.flags[FL_PRUNE], 1);
        if (any_bad) atomicOr(&s.flags[FL_ERROR], ERRB_NONFINITE);
    }
}

template <typename real>
__global__ void __launch_bounds__(64) k_integrate(SysView<real> s, StepView<real> g)
{
    pdl_wait();   // launched as a programmatic dependent in the step graph: every input complete from here
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.n_groups) return;
    const Group G = g.groups[gi];
    if (s.flags[FL_ERROR] & ERRB_SKIP) {
        // the neighbour list was truncated (the host regrows it and replays
        // the step) or the new positions were refused: consume the forces,
        // leave the state untouched
        for (int a = 0; a < G.natom; ++a) {
            const int atom = G.atom[a], slot = s.iperm[atom];
            s.F[slot] = 0; s.F[s.n_pad + slot] = 0; s.F[2 * s.n_pad + slot] = 0;
            s.Fa[atom] = 0; s.Fa[s.n + atom] = 0; s.Fa[2 * s.n + atom] = 0;
        }
        return;
    }
    // the kicks were drawn by k_prestep; the counter is not read here (k_theta
    // advances it concurrently)
    const unsigned long long step = 0ull;
    if (G.kind == GROUP_WATER) integrate_group<real, GROUP_WATER, 3>(s, g, G, step);
    else if (G.kind == GROUP_STAR && G.natom == 4) integrate_group<real, GROUP_STAR, 4>(s, g, G, step);
    else if (G.kind == GROUP_STAR && G.natom == 3) integrate_group<real, GROUP_STAR, 3>(s, g, G, step);
    else if (G.kind == GROUP_STAR && G.natom == 2) integrate_group<real, GROUP_STAR, 2>(s, g, G, step);
    else integrate_group<real, GROUP_SINGLE, 1>(s, g, G, step);
}

template <typename real>
void launch_integrate(const SysView<real>& s, const StepView<real>& g, cudaStream_t st, bool pdl)
{
    launch_k(pdl, k_integrate<real>, (g.n_groups + 63) / 64, 64, 0, st, s, g);
}

// Ornstein-Uhlenbeck kick of every atom for the current step:
// sqrt(k_B T (1 - a^2) / m) R with R from Philox4x32-10 at counter
// (atom, step) and Box-Muller; 0 for frozen atoms
template <typename real>
__device__ __forceinline__ void noise_body(const SysView<real>& s, const StepView<real>& g)
{
    const int atom = blockIdx.x * blockDim.x + threadIdx.x;
    if (atom >= s.n) return;
    const real w = s.invm[atom];
    real nr[3] = {(real)0, (real)0, (real)0};
    if (w != (real)0) {
        const unsigned long long step = s.lam->step;
        normals3<real>(make_uint4((unsigned)atom, (unsigned)step, (unsigned)(step >> 32), 0u), g.key, nr[0], nr[1],
                       nr[2]);
        const real sd = sqrt(g.kT * ((real)1 - g.a_fric * g.a_fric) * w);
        for (int d = 0; d < 3; ++d) nr[d] *= sd;
    }
    g.noise[3 * atom] = nr[0];
    g.noise[3 * atom + 1] = nr[1];
    g.noise[3 * atom + 2] = nr[2];
}

// --------------------------------------------------------- theta and OPES
__device__ __forceinline__ double pdiff2(double a, double b)
{
    double d = a - b;
    return d - 2.0 * floor((d + 1.0) / 2.0);
}

// (V, dV/dtheta) of bias b at theta, warp-cooperative (Eq. 11-13)
template <typename real>
__device__ void opes_bias(const ThetaView<real>& t, int b, double th, double& V, double& dV)
{
    const int lane = threadIdx.x & 31;
    const int n = t.st->n[b];
    V = 0.0; dV = 0.0;
    if (!t.on[b] || n == 0) return;
    const double* c = t.centre + b * t.max_k;
    const double* w = t.weight + b * t.max_k;
    const double is2 = 1.0 / (t.sigma * t.sigma);
    double sum = 0.0, dsum = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double d = pdiff2(th, c[k]);
        const double gk = w[k] * exp(-0.5 * d * d * is2);
        sum += gk;
        dsum += -gk * d * is2;
    }
    sum = warp_sum_d(sum);
    dsum = warp_sum_d(dsum);
    sum = __shfl_sync(0xffffffffu, sum, 0);
    dsum = __shfl_sync(0xffffffffu, dsum, 0);
    const double rho = sum / t.st->wsum[b], drho = dsum / t.st->wsum[b];
    const double rb = t.st->rho_bar[b];
    const double arg = rho / rb + t.epsr[b];
    V = t.nu[b] / t.beta * log(arg);
    dV = t.nu[b] / t.beta * (drho / rb) / arg;
}

// deposit a kernel at th into bias b; S_j (unnormalised KDE at each centre)
// is updated incrementally so rho_bar costs O(n) per deposit
template <typename real>
__device__ void opes_deposit(const ThetaView<real>& t, int b, double th, double wnew)
{
    const int lane = threadIdx.x & 31;
    const int n = t.st->n[b];
    if (n >= t.max_k) {
        if (lane == 0) atomicOr(&t.st->pad[0], 1);   // capacity reached: stop depositing
        return;
    }
    double* c = t.centre + b * t.max_k;
    double* w = t.weight + b * t.max_k;
    double* S = t.S + b * t.max_k;
    const double is2 = 1.0 / (t.sigma * t.sigma);
    double snew = 0.0, ssum = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double d = pdiff2(th, c[k]);
        const double gk = exp(-0.5 * d * d * is2);
        snew += w[k] * gk;
        S[k] += wnew * gk;
        ssum += S[k];
    }
    snew = warp_sum_d(snew);
    ssum = warp_sum_d(ssum);
    __syncwarp();
    if (lane == 0) {
        snew += wnew;
        c[n] = th;
        w[n] = wnew;
        S[n] = snew;
        ssum += snew;
        t.st->n[b] = n + 1;
        t.st->wsum[b] += wnew;
        t.st->rho_bar[b] = ssum / ((double)(n + 1) * t.st->wsum[b]);
    }
    __syncwarp();
}

// OPES biases at the current theta and the theta integrator's normal (one
// warp); they depend only on the state at the start of the step
template <typename real>
__device__ __forceinline__ void theta_pre_body(const SysView<real>& s, const ThetaView<real>& t)
{
    const LamState* L = s.lam;
    const double th = L->theta;
    double V0, dV0, V1, dV1;
    opes_bias(t, 0, th, V0, dV0);
    opes_bias(t, 1, th, V1, dV1);
    if (threadIdx.x == 0) {
        const unsigned long long step = L->step;
        double n0 = 0.0, n1, n2;
        if (t.m > 0.0) normals3<double>(make_uint4(0u, (unsigned)step, (unsigned)(step >> 32), 1u), t.key, n0, n1, n2);
        t.pre->V[0] = V0; t.pre->V[1] = V1;
        t.pre->dV[0] = dV0; t.pre->dV[1] = dV1;
        t.pre->noise = n0;
        t.pre->step = step;
    }
}

// the step's force-independent parts in one launch: blocks 0 .. nb-1 draw
// the atoms' kicks, the last block's first warp forms both OPES biases and
// theta's normal
template <typename real>
__global__ void k_prestep(SysView<real> s, StepView<real> g, ThetaView<real> t)
{
    if (blockIdx.x == gridDim.x - 1) {
        if (threadIdx.x < 32) theta_pre_body(s, t);
        return;
    }
    noise_body(s, g);
}

template <typename real>
void launch_prestep(const SysView<real>& s, const StepView<real>& g, const ThetaView<real>& t, cudaStream_t st)
{
    k_prestep<real><<<(s.n + 127) / 128 + 1, 128, 0, st>>>(s, g, t);
}

// theta's step once dU/dlambda is known: it needs only the coupling
// energies (solute-solvent pair, exclusion and 1-4, and reciprocal class
// energies, and the soft basis), so in the captured step it runs as soon as
// those are in, beside the force kernels that finish later.  One lane: FP64
// on a pipe with a small fraction of the FP32 rate, one dependent chain.
// The lambda state is not touched here (the force kernels still read it).
template <typename real>
__device__ __forceinline__ void theta_step_body(const SysView<real>& s, const ThetaView<real>& t)
{
    if (s.flags[FL_ERROR] & ERRB_SKIP) return;   // step skipped (see k_integrate)
    const LamState* L = s.lam;
    const long long* E = s.E;
    const double Uuv = efix(E, E_PAIR_UV) + efix(E, E_EXCL_UV) + efix(E, E_14_UV) + efix(E, E_REC_UV) + t.const_uv;
    const double Us = efix(E, E_PAIR_SOFT);
    const bool sc = s.sc_alpha > 0.0;   // soft-core coupling: U_soft is the term at lambda
    const double dUdl = L->dhA * Uuv + (sc ? efix(E, E_DSC) : L->dhB * Us);
    double thn = L->theta, pn = L->p_theta, ven = L->v_eta;
    if (t.m > 0.0) {
        const double f = -L->dlam_dtheta * dUdl - t.pre->dV[0] - t.pre->dV[1];
        ext_step(t.th, t.tc, t.m, t.kT, t.dt, t.a_fric, f, t.pre->noise, thn, pn, ven);
        thn -= 2.0 * floor(thn / 2.0);
    }
    t.pre->dUdl = dUdl;
    t.pre->theta = thn;
    t.pre->p_theta = pn;
    t.pre->v_eta = ven;
}

template <typename real>
__global__ void k_theta_step(SysView<real> s, ThetaView<real> t)
{
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) theta_step_body(s, t);
}

// the end of the step, once every kernel of it has run: U, the TI bin of
// Eq. 2, the new lambda state (Eq. 3) from k_theta_step's theta, OPES
// deposits, the step counter, and the energy accumulators cleared
template <typename real>
__device__ __forceinline__ void theta_commit_body(const SysView<real>& s, const ThetaView<real>& t)
{
    const int lane = threadIdx.x;
    LamState* L = s.lam;
    long long* E = s.E;
    if (s.flags[FL_ERROR] & ERRB_SKIP) {   // step skipped (see k_integrate): no advance
        if (lane < E_N) E[lane] = 0;
        return;
    }
    double thn = 0.0;
    unsigned long long stepn = 0;
    if (lane == 0) {
        const double Uvv = efix(E, E_PAIR_VV) + efix(E, E_EXCL_VV) + efix(E, E_14_VV) + efix(E, E_REC_VV) + t.const_vv;
        const double Uuu = efix(E, E_PAIR_UU) + efix(E, E_EXCL_UU) + efix(E, E_14_UU) + efix(E, E_REC_UU) + t.const_uu;
        const double Uuv = efix(E, E_PAIR_UV) + efix(E, E_EXCL_UV) + efix(E, E_14_UV) + efix(E, E_REC_UV) + t.const_uv;
        const double Us = efix(E, E_PAIR_SOFT);
        const double Ub = efix(E, E_BONDED);
        const bool sc = s.sc_alpha > 0.0;
        const double U = Uvv + Uuu + L->hA * Uuv + (sc ? Us : L->hB * Us) + Ub + efix(E, E_DAFED);
        const double dUdl = t.pre->dUdl;
        thn = t.pre->theta;
        stepn = L->step + 1;
        // Eq. 2: the mean force is accumulated in lambda bins (at the lambda
        // of this step's evaluation)
        const int bin = min(LFE_TI_BINS - 1, max(0, (int)floor(L->lambda * LFE_TI_BINS)));
        t.ti_sum[bin] += dUdl;
        t.ti_cnt[bin] += 1ull;
        const double lam = thn <= 1.0 ? thn : 2.0 - thn;
        double hA, hB, dA, dB;
        switching_fns(lam, hA, hB, dA, dB);
        L->theta = thn; L->p_theta = t.pre->p_theta; L->v_eta = t.pre->v_eta; L->lambda = lam;
        L->dlam_dtheta = thn <= 1.0 ? 1.0 : -1.0;
        L->hA = hA; L->hB = hB; L->dhA = dA; L->dhB = dB;
        L->dUdl = dUdl; L->U = U; L->V_std = t.pre->V[0]; L->V_exp = t.pre->V[1];
        L->npairs = (double)E[E_NPAIRS];
        if (!isfinite(U) || !isfinite(thn)) atomicOr(&s.flags[FL_ERROR], ERRB_NONFINITE);
        // the step ends here: its counter (the Philox counter of the atoms,
        // theta and the auxiliary angles) advances
        L->step = stepn;
    }
    stepn = __shfl_sync(0xffffffffu, stepn, 0);
    if (t.stride > 0 && (stepn % (unsigned long long)t.stride) == 0ull) {
        // a Standard kernel is reweighted by the total bias at its centre,
        // exp(beta (V_std + V_exp)), so that its density estimate converges
        // to the unbiased distribution while the trajectory runs under the
        // sum of both biases (Eq. 14); both are taken before either deposit
        thn = __shfl_sync(0xffffffffu, thn, 0);
        double Vs, dVs, Ve, dVe;
        opes_bias(t, 0, thn, Vs, dVs);
        opes_bias(t, 1, thn, Ve, dVe);
        if (t.on[0]) opes_deposit(t, 0, thn, exp(t.beta * (Vs + Ve)));
        if (t.on[1]) opes_deposit(t, 1, thn, 1.0);
    }
    // every energy accumulator has been read: clear them for the next step
    __syncwarp();
    if (lane < E_N) E[lane] = 0;
}

template <typename real>
__global__ void k_theta_commit(SysView<real> s, ThetaView<real> t)
{
    pdl_wait();
    theta_commit_body(s, t);
}

// both in one launch (one warp), where nothing runs beside them
template <typename real>
__global__ void k_theta(SysView<real> s, ThetaView<real> t)
{
    if (threadIdx.x == 0) theta_step_body(s, t);
    __syncwarp();
    theta_commit_body(s, t);
}

// Lambda replica exchange on the device (the paper's HREX protocol, Section
// 2.6, on the linear-basis potential of Eq. 4): one attempt over the ladder
// (replica indices in increasing lambda), from the basis energies U_uv and
// U_soft that the exchange evaluation has just written for every replica at
// its current configuration (terms[r][4], terms[r][5]).  The pairs (k, k+1)
// of the attempt's parity are tried; Delta = (h_A(l_k+1) - h_A(l_k))
// (U_uv,k - U_uv,k+1) + (h_B(l_k+1) - h_B(l_k)) (U_soft,k - U_soft,k+1); the
// pair is accepted when Delta <= 0 or u < exp(-beta Delta), u = (x + 0.5) /
// 2^32 with x the first word of Philox4x32-10 at counter (k, attempt_lo,
// attempt_hi, 3).  An accepted pair exchanges the two replicas' lambdas
// (theta = lambda, p_theta = 0) and their ladder entries.  One thread.
__device__ void set_lambda_state(LamState* L, double lam)
{
    double hA, hB, dA, dB;
    switching_fns(lam, hA, hB, dA, dB);
    L->theta = lam;
    L->p_theta = 0.0;
    L->dlam_dtheta = 1.0;
    L->lambda = lam;
    L->hA = hA; L->hB = hB; L->dhA = dA; L->dhB = dB;
}

__global__ void k_hrex(LamState* const* lams, const double* terms, int* ladder, int n, double beta, uint2 key,
                       unsigned long long* attempt, unsigned long long* accepted)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long a = *attempt;
    for (int k = (int)(a & 1ull); k + 1 < n; k += 2) {
        const int ri = ladder[k], rj = ladder[k + 1];
        LamState* Li = lams[ri];
        LamState* Lj = lams[rj];
        const double li = Li->lambda, lj = Lj->lambda;
        double hAi, hBi, hAj, hBj, d0, d1;
        switching_fns(li, hAi, hBi, d0, d1);
        switching_fns(lj, hAj, hBj, d0, d1);
        const double* ti = terms + (size_t)ri * LFE_NTERMS;
        const double* tj = terms + (size_t)rj * LFE_NTERMS;
        const double delta = (hAj - hAi) * (ti[4] - tj[4]) + (hBj - hBi) * (ti[5] - tj[5]);
        const uint4 r = philox4x32_10(make_uint4((unsigned)k, (unsigned)a, (unsigned)(a >> 32), 3u), key);
        const double u = (r.x + 0.5) / 4294967296.0;
        if (delta <= 0.0 || u < exp(-beta * delta)) {
            set_lambda_state(Li, lj);
            set_lambda_state(Lj, li);
            ladder[k] = rj;
            ladder[k + 1] = ri;
            accepted[k] += 1ull;
        }
    }
    *attempt = a + 1ull;
}

void launch_hrex(LamState* const* lams, const double* terms, int* ladder, int n, double beta, unsigned long long seed,
                 unsigned long long* attempt, unsigned long long* accepted, cudaStream_t st)
{
    k_hrex<<<1, 32, 0, st>>>(lams, terms, ladder, n, beta,
                             make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32)), attempt, accepted);
}

// first node of a captured step: the neighbour list is rebuilt (by the
// conditional node that follows) when the previous step left an atom more
// than skin/2 from where the list was built; no rebuild once a rebuild has
// overflowed (the steps after it are no-ops until the host regrows the list)
template <typename real>
__global__ void k_rebuild_cond(SysView<real> s, cudaGraphConditionalHandle h)
{
    const int err = s.flags[FL_ERROR];
    const int rb = s.flags[FL_REBUILD] && !(err & ERRB_SKIP);
    cudaGraphSetConditional(h, rb ? 1u : 0u);
    if (rb) s.flags[FL_NREBUILD] += 1;
    // a step skipped for refused positions keeps a pending rebuild for the next one
    if (!(err & ERRB_BADPOS)) s.flags[FL_REBUILD] = 0;
}

template <typename real>
void launch_rebuild_cond(const SysView<real>& s, cudaGraphConditionalHandle h, cudaStream_t st)
{
    k_rebuild_cond<real><<<1, 1, 0, st>>>(s, h);
}

// after the conditional rebuild: the pruned list is cut again when an atom
// has moved more than half the inner buffer since the last pruning, or the
// list was just built (the build raises FL_PRUNE); not after a skipped step
template <typename real>
__global__ void k_prune_cond(SysView<real> s, cudaGraphConditionalHandle h)
{
    const int err = s.flags[FL_ERROR];
    const int pr = s.flags[FL_PRUNE] && !(err & ERRB_SKIP);
    cudaGraphSetConditional(h, pr ? 1u : 0u);
    if (pr) s.flags[FL_NPRUNE] += 1;
    if (!(err & ERRB_SKIP)) s.flags[FL_PRUNE] = 0;
}

template <typename real>
void launch_prune_cond(const SysView<real>& s, cudaGraphConditionalHandle h, cudaStream_t st)
{
    k_prune_cond<real><<<1, 1, 0, st>>>(s, h);
}

template <typename real>
void launch_theta_step(const SysView<real>& s, const ThetaView<real>& t, cudaStream_t st, bool pdl)
{
    launch_k(pdl, k_theta_step<real>, 1, 32, 0, st, s, t);
}

template <typename real>
void launch_theta_commit(const SysView<real>& s, const ThetaView<real>& t, cudaStream_t st, bool pdl)
{
    launch_k(pdl, k_theta_commit<real>, 1, 32, 0, st, s, t);
}

template <typename real>
void launch_theta(const SysView<real>& s, const ThetaView<real>& t, cudaStream_t st)
{
    k_theta<real><<<1, 32, 0, st>>>(s, t);
}

#define LFE_INST_DYN(real)                                                                               \
    template void launch_set_lambda<real>(const SysView<real>&, double, cudaStream_t);                    \
    template void launch_eval_out<real>(const SysView<real>&, double*, double*, double, double, double,   \
                                        cudaStream_t);                                                    \
    template void launch_assign_moved<real, double>(const SysView<real>&, const double*, real, real,       \
                                                     cudaStream_t);                                        \
    template void launch_assign_moved<real, float>(const SysView<real>&, const float*, real, real,         \
                                                    cudaStream_t);                                         \
    template void launch_prune_cond<real>(const SysView<real>&, cudaGraphConditionalHandle, cudaStream_t);  \
    template void launch_check_positions<real, double>(const SysView<real>&, const double*, cudaStream_t);   \
    template void launch_check_positions<real, float>(const SysView<real>&, const float*, cudaStream_t);     \
    template void launch_pack_state_f32<real>(const SysView<real>&, const OpesState*, float*, double*,      \
                                              cudaStream_t);                                                 \
    template void launch_refresh_sorted<real>(const SysView<real>&, cudaStream_t);                         \
    template void launch_pack_state<real>(const SysView<real>&, const OpesState*, double*, cudaStream_t);   \
    template void launch_scale_molecules<real>(const SysView<real>&, const int*, const int*, const double*, int, \
                                               double, const double*, cudaStream_t);                         \
    template void launch_bonded<real>(const SysView<real>&, const BondView<real>&, cudaStream_t);          \
    template void launch_integrate<real>(const SysView<real>&, const StepView<real>&, cudaStream_t, bool); \
    template void launch_theta<real>(const SysView<real>&, const ThetaView<real>&, cudaStream_t);         \
    template void launch_theta_step<real>(const SysView<real>&, const ThetaView<real>&, cudaStream_t, bool); \
    template void launch_theta_commit<real>(const SysView<real>&, const ThetaView<real>&, cudaStream_t, bool); \
    template void launch_prestep<real>(const SysView<real>&, const StepView<real>&, const ThetaView<real>&,  \
                                       cudaStream_t);                                                       \
    template void launch_dafed_force<real>(const SysView<real>&, const DafedView&, cudaStream_t);            \
    template void launch_dafed_step<real>(const SysView<real>&, const DafedView&, cudaStream_t);             \
    template void launch_dafed_probe<real>(const SysView<real>&, const DafedView&, double, double*, cudaStream_t); \
    template void launch_rebuild_cond<real>(const SysView<real>&, cudaGraphConditionalHandle, cudaStream_t);

LFE_INST_DYN(float)
LFE_INST_DYN(double)

}  // namespace lfe
