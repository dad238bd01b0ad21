// nonbonded.cu -- neighbour search (cell sort, clusters, cluster-pair tiles,
// exclusion masks), the alchemical pair kernel and the exclusion / 1-4 kernel.
//
// Real-space part of Eq. 4-10: for every non-excluded pair with r < r_c
//   Coulomb   k_e q_i q_j erfc(alpha r) / r
//   LJ        4 eps_ij [(sigma_ij/r)^12 - (sigma_ij/r)^6] S(r)
//   soft LJ   eps_ij u_cap(r / sigma_ij) S(r)          (solute-solvent pairs only)
// with S the quintic switch on [r_sw, r_c], Lorentz-Berthelot mixing, class
// weights 1 (vv, uu), h_A (uv Coulomb + LJ) and h_B (soft).
#include "lfe_views.cuh"

namespace lfe {

// ------------------------------------------------------------ math helpers
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float erfc_(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_(double x) { return erfc(x); }
__device__ __forceinline__ float erf_(float x) { return erff(x); }
__device__ __forceinline__ double erf_(double x) { return erf(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float floor_(float x) { return floorf(x); }
__device__ __forceinline__ double floor_(double x) { return floor(x); }
__device__ __forceinline__ float rint_(float x) { return rintf(x); }
__device__ __forceinline__ double rint_(double x) { return rint(x); }

template <typename real>
__device__ __forceinline__ real wrap_coord(real x, real L, real invL)
{
    real w = x - L * floor_(x * invL);
    if (w >= L) w -= L;
    if (w < (real)0) w += L;
    if (w >= L) w = (real)0;
    return w;
}

__device__ __forceinline__ unsigned spread_bits(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// ------------------------------------------------------------- cell sort
template <typename real>
__global__ void k_cell_keys(SysView<real> s, NblView<real> nb)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n_solv) return;
    int a = s.solv_list[i];
    R4<real> p = s.x[a];
    int c[3];
    real pc[3] = {p.x, p.y, p.z};
    for (int d = 0; d < 3; ++d) {
        real w = wrap_coord(pc[d], s.L[d], s.invL[d]);
        int k = (int)(w * nb.cinv[d]);
        c[d] = k < 0 ? 0 : (k >= nb.nc[d] ? nb.nc[d] - 1 : k);
    }
    int key = (int)(spread_bits(c[0]) | (spread_bits(c[1]) << 1) | (spread_bits(c[2]) << 2));
    nb.keys[i] = key;
    atomicAdd(&nb.cnt[key], 1);
}

// exclusive scan of n ints (single block of 1024 threads); zeroes `in` and
// writes the total to *total when total != nullptr
__global__ void k_scan_block(int* in, int* out, int n, int* total, int cap, int* errflag)
{
    __shared__ int part[1024];
    const int tid = threadIdx.x;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = tid * per, e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += in[i];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < blockDim.x; off <<= 1) {
        int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = part[tid] - s;
    for (int i = b; i < e; ++i) {
        int v = in[i];
        out[i] = run;
        run += v;
        in[i] = 0;
    }
    if (tid == blockDim.x - 1) {
        out[n] = part[tid];
        if (total) {
            *total = part[tid];
            if (part[tid] > cap) atomicOr(errflag, ERRB_OVERFLOW);
        }
    }
}

template <typename real>
__global__ void k_cell_scatter(SysView<real> s, NblView<real> nb)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n_solv) return;
    int key = nb.keys[i];
    int pos = nb.start[key] + atomicAdd(&nb.fill[key], 1);
    nb.tmp[pos] = s.solv_list[i];
}

// deterministic order inside each cell: ascending atom index
template <typename real>
__global__ void k_cell_sort(NblView<real> nb)
{
    int key = blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= nb.nkeys) return;
    int b = nb.start[key], e = nb.start[key + 1];
    for (int i = b + 1; i < e; ++i) {
        int v = nb.tmp[i];
        int j = i - 1;
        while (j >= b && nb.tmp[j] > v) { nb.tmp[j + 1] = nb.tmp[j]; --j; }
        nb.tmp[j + 1] = v;
    }
    nb.fill[key] = 0;
}

// slot assignment: solute clusters first (caller order), then solvent atoms in
// cell order; fills the sorted coordinate/parameter arrays and xref
template <typename real>
__global__ void k_assign(SysView<real> s, NblView<real> nb)
{
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= s.n_pad) return;
    int a;
    int us = s.n_ucl * 32;
    if (slot < us) a = slot < s.n_u ? s.solute_list[slot] : -1;
    else {
        int k = slot - us;
        a = k < s.n_solv ? nb.tmp[k] : -1;
    }
    s.perm[slot] = a;
    R4<real> o;
    R2<real> l;
    if (a >= 0) {
        s.iperm[a] = slot;
        R4<real> p = s.x[a];
        s.xref[a] = p;
        o.x = wrap_coord(p.x, s.L[0], s.invL[0]);
        o.y = wrap_coord(p.y, s.L[1], s.invL[1]);
        o.z = wrap_coord(p.z, s.L[2], s.invL[2]);
        o.w = s.q[a] * (real)sqrt(KE);
        l.x = (real)0.5 * s.sig[a];
        l.y = (real)2 * sqrt(s.eps[a]);
    } else {
        o.x = o.y = o.z = o.w = (real)0;
        l.x = l.y = (real)0;
    }
    s.xq[slot] = o;
    s.lj[slot] = l;
}

template <typename real>
__global__ void k_bbox(SysView<real> s, NblView<real> nb)
{
    int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= s.n_cl) return;
    int slot = c * 32 + lane;
    bool ok = s.perm[slot] >= 0;
    R4<real> p = s.xq[slot];
    float lo[3], hi[3];
    float pv[3] = {(float)p.x, (float)p.y, (float)p.z};
    for (int d = 0; d < 3; ++d) {
        lo[d] = ok ? pv[d] : 3.0e38f;
        hi[d] = ok ? pv[d] : -3.0e38f;
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    }
    if (lane == 0) {
        R4<float> cc, hh;
        cc.x = 0.5f * (lo[0] + hi[0]); cc.y = 0.5f * (lo[1] + hi[1]); cc.z = 0.5f * (lo[2] + hi[2]); cc.w = 0.f;
        // a tiny outward margin keeps the float box conservative
        hh.x = 0.5f * (hi[0] - lo[0]) + 1e-5f; hh.y = 0.5f * (hi[1] - lo[1]) + 1e-5f;
        hh.z = 0.5f * (hi[2] - lo[2]) + 1e-5f; hh.w = 0.f;
        nb.bbc[c] = cc;
        nb.bbh[c] = hh;
    }
}

// shift code sh = (sx+1) + 3 (sy+1) + 9 (sz+1); cluster J is taken at
// x_J + s L.  For I == J only sh = 13 (s = 0, j > i) and the upper half
// sh > 13 are used, so each pair image is visited once.
template <typename real>
__device__ __forceinline__ bool tile_pass(const SysView<real>& s, const NblView<real>& nb,
                                          const R4<float>& ci, const R4<float>& hi, int J, int sh)
{
    R4<float> cj = nb.bbc[J], hj = nb.bbh[J];
    int sv[3] = {sh % 3 - 1, (sh / 3) % 3 - 1, sh / 9 - 1};
    float c1[3] = {cj.x, cj.y, cj.z}, c0[3] = {ci.x, ci.y, ci.z};
    float h1[3] = {hj.x, hj.y, hj.z}, h0[3] = {hi.x, hi.y, hi.z};
    float d2 = 0.f;
    for (int d = 0; d < 3; ++d) {
        float g = fabsf(c1[d] + sv[d] * (float)s.L[d] - c0[d]) - h0[d] - h1[d];
        g = fmaxf(g, 0.f);
        d2 += g * g;
    }
    return d2 < nb.cut2;
}

// pass 0: count tiles per i-cluster; pass 1: write them at the scanned offsets
template <typename real, int WRITE>
__global__ void k_tiles(SysView<real> s, NblView<real> nb)
{
    int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (I >= s.n_cl) return;
    R4<float> ci = nb.bbc[I], hi = nb.bbh[I];
    int base = WRITE ? nb.tile_off[I] : 0;
    int count = 0;
    bool iu = I < s.n_ucl;
    for (int J0 = I; J0 < s.n_cl; J0 += 32) {
        int J = J0 + lane;
        bool valid = J < s.n_cl;
        for (int sh = 0; sh < 27; ++sh) {
            bool pass = valid && (J != I || sh >= 13) && tile_pass(s, nb, ci, hi, valid ? J : I, sh);
            unsigned bal = __ballot_sync(0xffffffffu, pass);
            if (WRITE && pass) {
                int pos = base + count + __popc(bal & ((1u << lane) - 1u));
                if (pos < nb.cap) {
                    bool ju = J < s.n_ucl;
                    int cls = (iu && ju) ? 1 : ((iu || ju) ? 2 : 0);
                    nb.tiles[pos] = make_int4(I, J, sh, cls);
                }
            }
            count += __popc(bal);
        }
    }
    if (!WRITE && lane == 0) nb.tile_cnt[I] = count;
}

// interaction masks: bit j of lane i set = pair (I*32+i, J*32+j) is computed
template <typename real>
__global__ void k_masks(SysView<real> s, NblView<real> nb)
{
    int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int nt = min(s.flags[FL_NTILES], nb.cap);
    if (t >= nt) return;
    int4 tl = nb.tiles[t];
    int I = tl.x, J = tl.y, sh = tl.z;
    unsigned jvalid = __ballot_sync(0xffffffffu, s.perm[J * 32 + lane] >= 0);
    int a = s.perm[I * 32 + lane];
    unsigned m = 0u;
    if (a >= 0) {
        m = jvalid;
        if (I == J) {
            if (sh == 13) m &= (lane == 31) ? 0u : (0xffffffffu << (lane + 1));
            else m &= ~(1u << lane);
        }
        for (int e = nb.ex_start[a]; e < nb.ex_start[a + 1]; ++e) {
            int sb = s.iperm[nb.ex_list[e]];
            if ((sb >> 5) == J) m &= ~(1u << (sb & 31));
        }
    }
    nb.masks[(size_t)t * 32 + lane] = m;
}

template <typename real>
void launch_build_nbl(const SysView<real>& s, const NblView<real>& nb, cudaStream_t st)
{
    const int B = 256;
    if (s.n_solv > 0) {
        k_cell_keys<real><<<(s.n_solv + B - 1) / B, B, 0, st>>>(s, nb);
        k_scan_block<<<1, 1024, 0, st>>>(nb.cnt, nb.start, nb.nkeys, nullptr, 0, nullptr);
        k_cell_scatter<real><<<(s.n_solv + B - 1) / B, B, 0, st>>>(s, nb);
        k_cell_sort<real><<<(nb.nkeys + B - 1) / B, B, 0, st>>>(nb);
    }
    k_assign<real><<<(s.n_pad + B - 1) / B, B, 0, st>>>(s, nb);
    int wb = (s.n_cl * 32 + B - 1) / B;
    k_bbox<real><<<wb, B, 0, st>>>(s, nb);
    k_tiles<real, 0><<<wb, B, 0, st>>>(s, nb);
    k_scan_block<<<1, 1024, 0, st>>>(nb.tile_cnt, nb.tile_off, s.n_cl, s.flags + FL_NTILES, nb.cap,
                                     s.flags + FL_ERROR);
    k_tiles<real, 1><<<wb, B, 0, st>>>(s, nb);
    int mb = (int)(((long long)nb.cap * 32 + B - 1) / B);
    k_masks<real><<<mb, B, 0, st>>>(s, nb);
}

// ------------------------------------------------------------ pair kernel
template <typename real>
__device__ __forceinline__ void flush_force(const SysView<real>& s, int slot, long long fx, long long fy,
                                            long long fz)
{
    if (fx | fy | fz) {
        atomic_add_ll(&s.F[slot], fx);
        atomic_add_ll(&s.F[s.n_pad + slot], fy);
        atomic_add_ll(&s.F[2 * s.n_pad + slot], fz);
    }
}

// One warp walks a contiguous chunk of the (I-sorted) tile list.  Lane i
// holds atom I*32+i; the 32 atoms of J rotate through the lanes by shuffles
// together with their force accumulators (Newton's third law inside the
// tile).  The tile's class (vv, uu or uv) is uniform, so the branch on it is
// warp-uniform.  i-forces stay in registers while consecutive tiles share I.
template <typename real>
__global__ void __launch_bounds__(128) k_pairs(SysView<real> s, NblView<real> nb)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    int ntiles = s.flags[FL_NTILES];
    if (ntiles > nb.cap) ntiles = nb.cap;
    const int t0 = (int)(((long long)ntiles * warp) / nwarp);
    const int t1 = (int)(((long long)ntiles * (warp + 1)) / nwarp);
    if (t0 >= t1) return;
    const real hA = (real)s.lam->hA, hB = (real)s.lam->hB;
    const real rc2 = s.rc2, rsw = s.rsw, swi = s.sw_inv_w, alpha = s.alpha, tas = s.two_a_sqrtpi;
    const int src = (lane + 1) & 31;

    int curI = -1;
    real xi = 0, yi = 0, zi = 0, qi = 0, si = 0, ei = 0;
    long long fix = 0, fiy = 0, fiz = 0;
    double evv = 0, euu = 0, euv = 0, esoft = 0;
    int npairs = 0;

    for (int t = t0; t < t1; ++t) {
        const int4 tl = nb.tiles[t];
        if (tl.x != curI) {
            if (curI >= 0) flush_force(s, curI * 32 + lane, fix, fiy, fiz);
            curI = tl.x;
            R4<real> p = s.xq[curI * 32 + lane];
            R2<real> l = s.lj[curI * 32 + lane];
            xi = p.x; yi = p.y; zi = p.z; qi = p.w; si = l.x; ei = l.y;
            fix = fiy = fiz = 0;
        }
        const unsigned m = nb.masks[(size_t)t * 32 + lane];
        const int slot_j = tl.y * 32 + lane;
        R4<real> pj = s.xq[slot_j];
        R2<real> lj = s.lj[slot_j];
        const int sh = tl.z;
        const int sx = sh % 3 - 1, sy = (sh / 3) % 3 - 1, sz = sh / 9 - 1;
        // shift the far-side atom down by L so that the subtraction below is
        // the only rounding in the pair vector
        const real xit = sx == 1 ? xi - s.L[0] : xi;
        const real yit = sy == 1 ? yi - s.L[1] : yi;
        const real zit = sz == 1 ? zi - s.L[2] : zi;
        real xj = sx == -1 ? pj.x - s.L[0] : pj.x;
        real yj = sy == -1 ? pj.y - s.L[1] : pj.y;
        real zj = sz == -1 ? pj.z - s.L[2] : pj.z;
        real qj = pj.w, sj = lj.x, ej = lj.y;
        real fjx = 0, fjy = 0, fjz = 0, fx = 0, fy = 0, fz = 0, e0 = 0, e1 = 0;

        if (tl.w != 2) {
#pragma unroll 2
            for (int k = 0; k < 32; ++k) {
                const int jj = (lane + k) & 31;
                const real dx = xj - xit, dy = yj - yit, dz = zj - zit;
                const real r2 = dx * dx + dy * dy + dz * dz;
                if (((m >> jj) & 1u) && r2 < rc2) {
                    const real rinv = rsqrt_(r2);
                    const real r = r2 * rinv;
                    const real rinv2 = rinv * rinv;
                    const real qq = qi * qj;
                    const real ar = alpha * r;
                    const real ec = qq * erfc_(ar) * rinv;
                    const real fc = (ec + qq * tas * exp_(-ar * ar)) * rinv2;
                    const real sg = si + sj, e4 = ei * ej;
                    const real s2 = sg * sg * rinv2;
                    const real s6 = s2 * s2 * s2;
                    real v = e4 * (s6 * s6 - s6);
                    real fl = e4 * ((real)12 * s6 * s6 - (real)6 * s6) * rinv2;
                    const real tt = fmax((real)0, (r - rsw) * swi);
                    const real tt2 = tt * tt;
                    const real S = (real)1 - tt2 * tt * ((real)10 - (real)15 * tt + (real)6 * tt2);
                    const real dS = (real)-30 * tt2 * ((real)1 - tt) * ((real)1 - tt) * swi;
                    fl = fl * S - v * dS * rinv;
                    v *= S;
                    const real g = fc + fl;
                    fx -= g * dx; fy -= g * dy; fz -= g * dz;
                    fjx += g * dx; fjy += g * dy; fjz += g * dz;
                    e0 += ec + v;
                    ++npairs;
                }
                xj = __shfl_sync(FULL, xj, src); yj = __shfl_sync(FULL, yj, src);
                zj = __shfl_sync(FULL, zj, src); qj = __shfl_sync(FULL, qj, src);
                sj = __shfl_sync(FULL, sj, src); ej = __shfl_sync(FULL, ej, src);
                fjx = __shfl_sync(FULL, fjx, src); fjy = __shfl_sync(FULL, fjy, src);
                fjz = __shfl_sync(FULL, fjz, src);
            }
            if (tl.w == 0) evv += (double)e0;
            else euu += (double)e0;
        } else {
            for (int k = 0; k < 32; ++k) {
                const int jj = (lane + k) & 31;
                const real dx = xj - xit, dy = yj - yit, dz = zj - zit;
                const real r2 = dx * dx + dy * dy + dz * dz;
                if (((m >> jj) & 1u) && r2 < rc2) {
                    const real rinv = rsqrt_(r2);
                    const real r = r2 * rinv;
                    const real rinv2 = rinv * rinv;
                    const real qq = qi * qj;
                    const real ar = alpha * r;
                    const real ec = qq * erfc_(ar) * rinv;
                    const real fc = (ec + qq * tas * exp_(-ar * ar)) * rinv2;
                    const real sg = si + sj, e4 = ei * ej;
                    const real s2 = sg * sg * rinv2;
                    const real s6 = s2 * s2 * s2;
                    real v = e4 * (s6 * s6 - s6);
                    real fl = e4 * ((real)12 * s6 * s6 - (real)6 * s6) * rinv2;
                    const real tt = fmax((real)0, (r - rsw) * swi);
                    const real tt2 = tt * tt;
                    const real S = (real)1 - tt2 * tt * ((real)10 - (real)15 * tt + (real)6 * tt2);
                    const real dS = (real)-30 * tt2 * ((real)1 - tt) * ((real)1 - tt) * swi;
                    fl = fl * S - v * dS * rinv;
                    v *= S;
                    // capped soft basis (Eq. 5-6): identical to LJ for r >= sigma_ij
                    real vs = v, fs = fl;
                    if (e4 == (real)0) { vs = 0; fs = 0; }
                    else if (r < sg) {
                        const real sgi = (real)1 / sg;
                        const real x = r * sgi, x2 = x * x, x3 = x2 * x;
                        const real u = ((real)-868 * x2 + (real)2188.8 * x - (real)1440) * x3 * x + (real)119.2;
                        const real du = ((real)-5208 * x2 + (real)10944 * x - (real)5760) * x3;
                        const real ep = (real)0.25 * e4;
                        vs = ep * u * S;
                        fs = -ep * (du * sgi * S + u * dS) * rinv;
                    }
                    const real g = hA * (fc + fl) + hB * fs;
                    fx -= g * dx; fy -= g * dy; fz -= g * dz;
                    fjx += g * dx; fjy += g * dy; fjz += g * dz;
                    e0 += ec + v;
                    e1 += vs;
                    ++npairs;
                }
                xj = __shfl_sync(FULL, xj, src); yj = __shfl_sync(FULL, yj, src);
                zj = __shfl_sync(FULL, zj, src); qj = __shfl_sync(FULL, qj, src);
                sj = __shfl_sync(FULL, sj, src); ej = __shfl_sync(FULL, ej, src);
                fjx = __shfl_sync(FULL, fjx, src); fjy = __shfl_sync(FULL, fjy, src);
                fjz = __shfl_sync(FULL, fjz, src);
            }
            // solute-solvent energies come from the FP64 kernel k_uv_energy
            (void)e0;
            (void)e1;
        }
        fix += to_fixed(fx, FSCALE);
        fiy += to_fixed(fy, FSCALE);
        fiz += to_fixed(fz, FSCALE);
        flush_force(s, slot_j, to_fixed(fjx, FSCALE), to_fixed(fjy, FSCALE), to_fixed(fjz, FSCALE));
    }
    flush_force(s, curI * 32 + lane, fix, fiy, fiz);
    long long a0 = __double2ll_rn(warp_sum_d(evv) * ESCALE);
    long long a1 = __double2ll_rn(warp_sum_d(euu) * ESCALE);
    long long a2 = __double2ll_rn(warp_sum_d(euv) * ESCALE);
    long long a3 = __double2ll_rn(warp_sum_d(esoft) * ESCALE);
    long long a4 = warp_sum_ll((long long)npairs);
    if (lane == 0) {
        if (a0) atomic_add_ll(&s.E[E_PAIR_VV], a0);
        if (a1) atomic_add_ll(&s.E[E_PAIR_UU], a1);
        if (a2) atomic_add_ll(&s.E[E_PAIR_UV], a2);
        if (a3) atomic_add_ll(&s.E[E_PAIR_SOFT], a3);
        atomic_add_ll(&s.E[E_NPAIRS], a4);
    }
}

// Solute-solvent basis energies U_uv (real-space part) and U_soft in FP64.
// They set dU/dlambda = h_A' U_uv + h_B' U_soft, whose tolerance (1e-6
// relative) is below what FP32 pair arithmetic delivers, so they are recomputed
// here from the same tiles and masks: one thread per (uv tile, i, j) slot in a
// grid-stride loop over the whole GPU, so the few thousand pairs use the FP64
// pipes of every SM while the FP32 pair kernel computes forces.  The pair
// vector is formed exactly: coordinates are floats, their sums are exact in
// double.
template <typename real>
__global__ void __launch_bounds__(256) k_uv_energy(SysView<real> s, NblView<real> nb)
{
    const int n_uv_tiles = s.n_ucl > 0 ? min(nb.tile_off[s.n_ucl], nb.cap) : 0;
    const long long total = (long long)n_uv_tiles * 1024;
    const double rc2 = (double)s.rc2, rsw = (double)s.rsw, swi = (double)s.sw_inv_w;
    const double alpha = (double)s.alpha;
    double euv = 0.0, esoft = 0.0;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(w >> 10), i = (int)((w >> 5) & 31), j = (int)(w & 31);
        const int4 tl = nb.tiles[t];
        if (tl.w != 2) continue;
        if (!((nb.masks[(size_t)t * 32 + i] >> j) & 1u)) continue;
        const int si = tl.x * 32 + i, sj = tl.y * 32 + j;
        const R4<real> pi = s.xq[si], pj = s.xq[sj];
        const int sh = tl.z;
        const int sv[3] = {sh % 3 - 1, (sh / 3) % 3 - 1, sh / 9 - 1};
        const double xi[3] = {(double)pi.x, (double)pi.y, (double)pi.z};
        const double xj[3] = {(double)pj.x, (double)pj.y, (double)pj.z};
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double dd = xj[d] + sv[d] * (double)s.L[d] - xi[d];
            r2 += dd * dd;
        }
        if (!(r2 < rc2)) continue;
        const int a = s.perm[si], b = s.perm[sj];
        const double r = sqrt(r2);
        const double qq = KE * (double)s.q[a] * (double)s.q[b];
        double e = qq * erfc(alpha * r) / r;
        const double sg = 0.5 * ((double)s.sig[a] + (double)s.sig[b]);
        const double ep = sqrt((double)s.eps[a] * (double)s.eps[b]);
        if (ep > 0.0) {
            const double tt = fmax(0.0, (r - rsw) * swi);
            const double S = 1.0 - tt * tt * tt * (10.0 - 15.0 * tt + 6.0 * tt * tt);
            const double s2 = sg * sg / r2, s6 = s2 * s2 * s2;
            const double v = 4.0 * ep * (s6 * s6 - s6) * S;
            e += v;
            if (r < sg) {
                const double x = r / sg, x2 = x * x, x4 = x2 * x2;
                esoft += ep * ((-868.0 * x2 + 2188.8 * x - 1440.0) * x4 + 119.2) * S;
            } else {
                esoft += v;
            }
        }
        euv += e;
    }
    long long a0 = __double2ll_rn(warp_sum_d(euv) * ESCALE);
    long long a1 = __double2ll_rn(warp_sum_d(esoft) * ESCALE);
    if ((threadIdx.x & 31) == 0) {
        if (a0) atomic_add_ll(&s.E[E_PAIR_UV], a0);
        if (a1) atomic_add_ll(&s.E[E_PAIR_SOFT], a1);
    }
}

template <typename real>
void launch_uv_energy(const SysView<real>& s, const NblView<real>& nb, int nblocks, cudaStream_t st)
{
    if (s.n_ucl == 0) return;
    k_uv_energy<real><<<nblocks, 256, 0, st>>>(s, nb);
}

template <typename real>
void launch_pairs(const SysView<real>& s, const NblView<real>& nb, int nwarps, cudaStream_t st)
{
    const int B = 128;
    int blocks = (nwarps * 32 + B - 1) / B;
    k_pairs<real><<<blocks, B, 0, st>>>(s, nb);
}

// ------------------------------------------------- exclusions and 1-4 pairs
// excluded pair (any distance, minimum image): -k_e q_i q_j erf(alpha r)/r;
// 1-4 pair: s_C k_e q_i q_j / r + s_LJ 4 eps_ij [(s/r)^12 - (s/r)^6]
template <typename real>
__global__ void k_excl(SysView<real> s, ExclView<real> ex)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[6] = {0, 0, 0, 0, 0, 0};   // excl vv, uu, uv, 14 vv, uu, uv
    if (e < ex.n_excl + ex.n14) {
        const bool is14 = e >= ex.n_excl;
        const int2 pr = is14 ? ex.p14[e - ex.n_excl] : ex.excl[e];
        const int sa = s.iperm[pr.x], sb = s.iperm[pr.y];
        const R4<real> pa = s.xq[sa], pb = s.xq[sb];
        real d[3] = {pb.x - pa.x, pb.y - pa.y, pb.z - pa.z};
        for (int k = 0; k < 3; ++k) d[k] -= s.L[k] * rint_(d[k] * s.invL[k]);
        const real r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        real en = 0, g = 0;   // g = -(dE/dr)/r
        if (r2 > (real)0) {
            const real rinv = rsqrt_(r2);
            const real rinv2 = rinv * rinv;
            const real qq = pa.w * pb.w;
            if (!is14) {
                const real ar = s.alpha * r2 * rinv;
                const real ev = erf_(ar);
                en = -qq * ev * rinv;
                // dE/dr = qq erf/r^2 - qq (2a/sqrt(pi)) exp(-a^2 r^2)/r
                g = -(qq * ev * rinv2 - qq * s.two_a_sqrtpi * exp_(-ar * ar) * rinv) * rinv;
            } else {
                const R2<real> sc = ex.s14[e - ex.n_excl];
                const R2<real> la = s.lj[sa], lb = s.lj[sb];
                en = sc.y * qq * rinv;
                g = sc.y * qq * rinv2 * rinv;
                const real sg = la.x + lb.x, e4 = la.y * lb.y;
                if (e4 != (real)0) {
                    const real s2 = sg * sg * rinv2, s6 = s2 * s2 * s2;
                    en += sc.x * e4 * (s6 * s6 - s6);
                    g += sc.x * e4 * ((real)12 * s6 * s6 - (real)6 * s6) * rinv2;
                }
            }
            for (int k = 0; k < 3; ++k) {
                long long f = to_fixed(g * d[k], FSCALE);
                atomic_add_ll(&s.F[k * s.n_pad + sa], -f);
                atomic_add_ll(&s.F[k * s.n_pad + sb], f);
            }
        }
        const int ua = s.sol[pr.x], ub = s.sol[pr.y];
        const int cls = (ua && ub) ? 1 : ((ua || ub) ? 2 : 0);
        acc[(is14 ? 3 : 0) + cls] = (double)en;
    }
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < 6; ++c) {
        long long v = __double2ll_rn(warp_sum_d(acc[c]) * ESCALE);
        if (lane == 0 && v) atomic_add_ll(&s.E[(c < 3 ? E_EXCL_VV : E_14_VV) + (c % 3)], v);
    }
}

template <typename real>
void launch_excl(const SysView<real>& s, const ExclView<real>& ex, cudaStream_t st)
{
    int n = ex.n_excl + ex.n14;
    if (n == 0) return;
    const int B = 256;
    k_excl<real><<<(n + B - 1) / B, B, 0, st>>>(s, ex);
}

#define LFE_INST(real)                                                                             \
    template void launch_build_nbl<real>(const SysView<real>&, const NblView<real>&, cudaStream_t); \
    template void launch_pairs<real>(const SysView<real>&, const NblView<real>&, int, cudaStream_t); \
    template void launch_uv_energy<real>(const SysView<real>&, const NblView<real>&, int, cudaStream_t); \
    template void launch_excl<real>(const SysView<real>&, const ExclView<real>&, cudaStream_t);
LFE_INST(float)
LFE_INST(double)

}  // namespace lfe
