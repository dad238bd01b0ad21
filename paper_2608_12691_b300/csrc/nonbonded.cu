// nonbonded.cu -- neighbour search (cell sort, clusters, cluster-pair tiles,
// exclusion masks), the alchemical pair kernel and the exclusion / 1-4 kernel.
//
// Real-space part of Eq. 4-10: for every non-excluded pair with r < r_c
//   Coulomb   k_e q_i q_j erfc(alpha r) / r
//   LJ        4 eps_ij [(sigma_ij/r)^12 - (sigma_ij/r)^6] S(r)
//   soft LJ   eps_ij u_cap(r / sigma_ij) S(r)          (solute-solvent pairs only)
// with S the quintic switch on [r_sw, r_c], Lorentz-Berthelot mixing, class
// weights 1 (vv, uu), h_A (uv Coulomb + LJ) and h_B (soft).
#include <type_traits>

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


__device__ __forceinline__ unsigned spread_bits(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// ------------------------------------------------------------ clustering
// Solvent atoms are binned into ncx x ncy columns in xy, sorted by z inside
// each column and cut into clusters of 32 consecutive atoms; a column's last
// cluster is padded.  With a column edge near (32/rho)^(1/3) the clusters are
// close to cubic.  Solute atoms occupy the first clusters, in caller order.
template <typename real>
__global__ void k_col_keys(SysView<real> s, NblView<real> nb)
{
    pdl_trigger();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n_solv) return;
    const R4<real> p = s.x[s.solv_list[i]];
    const real wx = wrap_box(p.x, s.L[0], s.invL[0]);
    const real wy = wrap_box(p.y, s.L[1], s.invL[1]);
    int cx = (int)(wx * nb.cinvx), cy = (int)(wy * nb.cinvy);
    cx = cx < 0 ? 0 : (cx >= nb.ncx ? nb.ncx - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= nb.ncy ? nb.ncy - 1 : cy);
    const int c = cx * nb.ncy + cy;
    nb.col_of[i] = c;
    atomicAdd(&nb.col_cnt[c], 1);
}

// exclusive prefix of one value per thread over the block (warp shuffles and
// one shared-memory pass over the warp sums); *grand = block total
__device__ __forceinline__ int block_exscan(int v, int* wsum, int* grand)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();   // wsum may still be read by a previous scan
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int x = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane < nw) wsum[lane] = x;
    }
    __syncthreads();
    *grand = wsum[nw - 1];
    return incl - v + (warp > 0 ? wsum[warp - 1] : 0);
}

// exclusive scan of n ints (single block of 1024 threads); zeroes `in`;
// writes the total to *total (when given) and raises the overflow bit when it
// exceeds cap.  CL = 1 also scans the 32-atom clusters of each entry,
// ceil(in / 32), into out2 with their total in *total2 (the column sort).
template <int CL>
__global__ void __launch_bounds__(1024) k_scan_block(int* in, int* out, int n, int* total, int cap, int* errflag,
                                                     int* out2, int* total2)
{
    pdl_wait();
    pdl_trigger();
    constexpr int PER_MAX = 32;
    __shared__ int wsum[32];
    const int tid = threadIdx.x;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = tid * per, e = min(n, b + per);
    int v[PER_MAX];
    int s = 0, s2 = 0;
    if (per <= PER_MAX) {
        // all of this thread's loads in flight at once
#pragma unroll
        for (int k = 0; k < PER_MAX; ++k) {
            v[k] = (k < per && b + k < e) ? in[b + k] : 0;
            s += v[k];
            if (CL) s2 += (v[k] + 31) >> 5;
        }
    } else {
        for (int i = b; i < e; ++i) {
            s += in[i];
            if (CL) s2 += (in[i] + 31) >> 5;
        }
    }
    int grand = 0, grand2 = 0;
    int run = block_exscan(s, wsum, &grand);
    int run2 = CL ? block_exscan(s2, wsum, &grand2) : 0;
    if (per <= PER_MAX) {
#pragma unroll
        for (int k = 0; k < PER_MAX; ++k) {
            if (k < per && b + k < e) {
                out[b + k] = run;
                run += v[k];
                if (CL) {
                    out2[b + k] = run2;
                    run2 += (v[k] + 31) >> 5;
                }
                in[b + k] = 0;
            }
        }
    } else {
        for (int i = b; i < e; ++i) {
            const int x = in[i];
            out[i] = run;
            run += x;
            if (CL) {
                out2[i] = run2;
                run2 += (x + 31) >> 5;
            }
            in[i] = 0;
        }
    }
    if (tid == blockDim.x - 1) {
        out[n] = grand;
        if (total) {
            *total = grand;
            if (grand > cap) atomicOr(errflag, ERRB_OVERFLOW);
        }
        if (CL) {
            out2[n] = grand2;
            *total2 = grand2;
        }
    }
}

template <typename real>
__global__ void k_col_scatter(SysView<real> s, NblView<real> nb)
{
    pdl_wait();
    pdl_trigger();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n_solv) return;
    const int c = nb.col_of[i];
    const int pos = nb.col_start[c] + atomicAdd(&nb.col_fill[c], 1);
    nb.tmp[pos] = s.solv_list[i];
}

constexpr int COL_MAX = 2048;   // atoms per column handled by one block

// one block per column: rank sort by (wrapped z, atom index); four threads
// share the count of each atom's rank
constexpr int COL_THREADS = 1024;

template <typename real>
__global__ void __launch_bounds__(COL_THREADS) k_col_sort(SysView<real> s, NblView<real> nb)
{
    pdl_wait();
    pdl_trigger();
    __shared__ float zs[COL_MAX];
    __shared__ int ids[COL_MAX];
    const int c = blockIdx.x;
    const int b = nb.col_start[c];
    int cnt = nb.col_start[c + 1] - b;
    if (cnt > COL_MAX) {
        if (threadIdx.x == 0) atomicOr(&s.flags[FL_ERROR], ERRB_OVERFLOW);
        cnt = COL_MAX;
    }
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int a = nb.tmp[b + k];
        ids[k] = a;
        zs[k] = (float)wrap_box(s.x[a].z, s.L[2], s.invL[2]);
    }
    __syncthreads();
    const int sub = threadIdx.x & 3;
    for (int k0 = 0; k0 < cnt; k0 += blockDim.x >> 2) {
        const int k = k0 + (threadIdx.x >> 2);
        const bool ok = k < cnt;
        const float z = ok ? zs[k] : 0.f;
        const int a = ok ? ids[k] : 0;
        int rank = 0;
        if (ok)
            for (int m = sub; m < cnt; m += 4) {
                const float zm = zs[m];
                rank += (zm < z) || (zm == z && ids[m] < a);
            }
        rank += __shfl_xor_sync(0xffffffffu, rank, 1);
        rank += __shfl_xor_sync(0xffffffffu, rank, 2);
        if (ok && sub == 0) nb.tmp2[b + rank] = a;
    }
    if (threadIdx.x == 0) nb.col_fill[c] = 0;
}

// slot -> atom: solute clusters first, then the solvent clusters column by
// column; also the sorted coordinates / parameters, xref and the clusters'
// bounding boxes (one warp per cluster)
template <typename real>
__global__ void k_assign(SysView<real> s, NblView<real> nb)
{
    pdl_wait();
    pdl_trigger();
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= s.n_pad) return;
    int a = -1;
    const int us = s.n_ucl * 32;
    if (slot < us) {
        a = slot < s.n_u ? s.solute_list[slot] : -1;
    } else {
        const int c = slot / 32 - s.n_ucl;   // solvent cluster
        if (c < *nb.n_cl_solv) {
            // column of cluster c: last k with col_cl[k] <= c
            int lo = 0, hi = nb.ncols - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (nb.col_cl[mid] <= c) lo = mid;
                else hi = mid - 1;
            }
            const int rank = (c - nb.col_cl[lo]) * 32 + (slot & 31);
            const int cnt = min(nb.col_start[lo + 1] - nb.col_start[lo], COL_MAX);
            if (rank < cnt) a = nb.tmp2[nb.col_start[lo] + rank];
        }
    }
    s.perm[slot] = a;
    R4<real> o;
    R2<real> l;
    if (a >= 0) {
        s.iperm[a] = slot;
        const R4<real> p = s.x[a];
        s.xref[a] = p;
        o.x = wrap_box(p.x, s.L[0], s.invL[0]);
        o.y = wrap_box(p.y, s.L[1], s.invL[1]);
        o.z = wrap_box(p.z, s.L[2], s.invL[2]);
        o.w = s.q[a] * (real)sqrt(KE);
        l.x = (real)0.5 * s.sig[a];
        l.y = (real)2 * sqrt(s.eps[a]);
    } else {
        o.x = o.y = o.z = o.w = (real)0;
        l.x = l.y = (real)0;
    }
    s.xq[slot] = o;
    s.lj[slot] = l;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.flags[FL_NSTAGE] = 0;   // the tile staging list starts empty
        s.flags[FL_PRUNE] = 1;    // a pruned list, where one is used, is cut from the new list
    }
    // the warp holds one cluster: bounding boxes of the cluster (the partner
    // side of the tile search) and of its four 8-slot sub-clusters (the i
    // side); a sub-cluster without atoms gets a negative half extent
    const int c = slot >> 5, lane = slot & 31;
    if (c >= s.n_ucl + *nb.n_cl_solv) return;
    float lo[3], hi[3];
    const float pv[3] = {(float)o.x, (float)o.y, (float)o.z};
    for (int d = 0; d < 3; ++d) {
        lo[d] = a >= 0 ? pv[d] : 3.0e38f;
        hi[d] = a >= 0 ? pv[d] : -3.0e38f;
    }
    auto emit = [&](R4<float>* cen, R4<float>* half, int idx) {
        R4<float> cc, hh;
        const bool any = lo[0] <= hi[0];
        cc.x = 0.5f * (lo[0] + hi[0]); cc.y = 0.5f * (lo[1] + hi[1]); cc.z = 0.5f * (lo[2] + hi[2]); cc.w = 0.f;
        // a tiny outward margin keeps the float box conservative
        hh.x = 0.5f * (hi[0] - lo[0]) + 1e-5f; hh.y = 0.5f * (hi[1] - lo[1]) + 1e-5f;
        hh.z = 0.5f * (hi[2] - lo[2]) + 1e-5f; hh.w = any ? 0.f : -1.f;
        if (!any) cc.x = cc.y = cc.z = hh.x = hh.y = hh.z = 0.f;
        cen[idx] = cc;
        half[idx] = hh;
    };
    for (int o8 = 4; o8 > 0; o8 >>= 1)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o8));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o8));
        }
    if ((lane & 7) == 0) emit(nb.bbc8, nb.bbh8, c * 4 + (lane >> 3));
    for (int o32 = 16; o32 > 4; o32 >>= 1)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o32));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o32));
        }
    if (lane == 0) emit(nb.bbc, nb.bbh, c);
}

template <typename real>
__device__ __forceinline__ int num_clusters(const SysView<real>& s, const NblView<real>& nb)
{
    return s.n_ucl + *nb.n_cl_solv;
}

// shift code sh = (sx+1) + 3 (sy+1) + 9 (sz+1): cluster J is taken at x_J + s L
__device__ __forceinline__ void shift_vec(int sh, int sv[3])
{
    sv[0] = sh % 3 - 1;
    sv[1] = (sh / 3) % 3 - 1;
    sv[2] = sh / 9 - 1;
}

template <typename real>
__device__ __forceinline__ float box_gap2(const SysView<real>& s, const R4<float>& ci, const R4<float>& hi,
                                          const R4<float>& cj, const R4<float>& hj, int sh)
{
    int sv[3];
    shift_vec(sh, sv);
    const float c1[3] = {cj.x, cj.y, cj.z}, c0[3] = {ci.x, ci.y, ci.z};
    const float h1[3] = {hj.x, hj.y, hj.z}, h0[3] = {hi.x, hi.y, hi.z};
    float d2 = 0.f;
    for (int d = 0; d < 3; ++d) {
        float g = fabsf(c1[d] + sv[d] * (float)s.L[d] - c0[d]) - h0[d] - h1[d];
        g = fmaxf(g, 0.f);
        d2 += g * g;
    }
    return d2;
}

// Tile list.  A tile pairs the 8 atoms of one i sub-cluster I8 (slots
// 8 I8 .. 8 I8 + 7 of the cluster-sorted order) with 32 j atoms under one
// periodic shift and one class (vv, uu or uv).  For each (I8, shift) and
// each class of partner cluster (solute, solvent) every atom of every 32-atom
// partner cluster J whose box is within r_cut + skin of I8's box is appended
// to a j list when the atom itself is within r_cut + skin of that box and
// lies in a sub-cluster J8 > I8, or in I8 itself under a shift past the
// middle one (13), or in I8 under no shift (pairs j > i, left to the masks)
// -- so every pair image is listed once.  One block per I8: its threads list
// the partner clusters whose boxes are in range (one box per thread), its
// warps filter those clusters' atoms (TILE_BATCH clusters per warp per batch
// of loads), and a block scan of the kept counts places every kept atom.
//
// One pass: each round (up to TILE_CAND partner clusters) reserves exactly
// the tiles it starts in a staging list -- in the order blocks happen to get
// there -- and writes them with their (I8, shift, class, ordinal).  k_place
// then moves every tile to its final, deterministic place (the tiles of one
// I8 contiguous and shift-major) from the per-(I8, shift) counts written
// here.
constexpr int TILE_WARPS = 4;      // warps of one block (one i sub-cluster)
constexpr int TILE_CAND = 256;     // partner clusters listed per round
constexpr int TILE_BATCH = 8;      // partner clusters whose atoms one warp loads together

struct TileShared {
    int cand[TILE_CAND];           // partner clusters of the round, ascending
    unsigned kb[TILE_CAND];        // their kept lanes
    int kpre[TILE_CAND];           // exclusive prefix of the kept atoms over the round
    int wcnt[TILE_WARPS];
    int wsum[32];
    int r0;                        // staging slots reserved by the round
    int cnt[27];                   // tiles per shift
    float4 ia[8];                  // the sub-cluster's atoms at the build (padding: far away)
};

// one (I8, shift) search by the whole block; returns the number of tiles
// started (the same value in every thread)
template <typename real>
__device__ int tile_search(const SysView<real>& s, const NblView<real>& nb, int I8, int sh, TileShared& sm)
{
    const int tid = threadIdx.x, wl = tid >> 5, lane = tid & 31;
    constexpr int NT = TILE_WARPS * 32;
    const int I = I8 >> 2;
    const int ncl = num_clusters(s, nb);
    const R4<float> ci = nb.bbc8[I8], hi = nb.bbh8[I8];
    const bool iu = I < s.n_ucl;
    int count = 0;        // tiles started (the next tile's ordinal)
    bool dead = false;    // the staging list ran out: nothing more is written
    int svs[3];
    shift_vec(sh, svs);
    const unsigned lt = (1u << lane) - 1u;
    const float shx = svs[0] * (float)s.L[0], shy = svs[1] * (float)s.L[1], shz = svs[2] * (float)s.L[2];
    const float c0[3] = {ci.x, ci.y, ci.z}, h0[3] = {hi.x, hi.y, hi.z};
    // sub-clusters of partner atoms that may pair with I8 under this shift
    const int j8min = sh >= 13 ? I8 : I8 + 1;
    for (int jc = 0; jc < 2; ++jc) {
        const int jb = jc == 0 ? 0 : s.n_ucl, je = jc == 0 ? s.n_ucl : ncl;
        const int cls = (iu && jc == 0) ? 1 : ((iu || jc == 0) ? 2 : 0);
        int nbuf = 0;   // atoms already placed in the open tile (staging slot cur)
        int cur = -1;
        int J0 = max(I, jb);
        while (J0 < je) {
            // list the partner clusters in range, in ascending order
            int nc = 0;
            while (J0 < je && nc + NT <= TILE_CAND) {
                const int J = J0 + tid;
                bool pc = J < je && 4 * J + 3 >= j8min;
                if (pc) pc = box_gap2(s, ci, hi, nb.bbc[J], nb.bbh[J], sh) < nb.cut2;
                const unsigned bal = __ballot_sync(0xffffffffu, pc);
                if (lane == 0) sm.wcnt[wl] = __popc(bal);
                __syncthreads();
                int off = nc, tot = 0;
#pragma unroll
                for (int w = 0; w < TILE_WARPS; ++w) {
                    off += w < wl ? sm.wcnt[w] : 0;
                    tot += sm.wcnt[w];
                }
                if (pc) sm.cand[off + __popc(bal & lt)] = J;
                nc += tot;
                J0 += NT;
                __syncthreads();
            }
            if (nc == 0) continue;
            // filter the candidates' atoms: warp wl takes candidates wl, wl + 4, ...
            for (int cb = wl; cb < nc; cb += TILE_WARPS * TILE_BATCH) {
                R4<real> pbuf[TILE_BATCH];
                bool live[TILE_BATCH];
#pragma unroll
                for (int u = 0; u < TILE_BATCH; ++u) {
                    const int c = cb + TILE_WARPS * u;
                    const int slot = c < nc ? sm.cand[c] * 32 + lane : -1;
                    live[u] = slot >= 0 && (slot >> 3) >= j8min && s.perm[slot] >= 0;
                    if (slot >= 0) pbuf[u] = s.xq[slot];
                }
#pragma unroll
                for (int u = 0; u < TILE_BATCH; ++u) {
                    const int c = cb + TILE_WARPS * u;
                    if (c >= nc) break;
                    bool keep = live[u];
                    if (keep) {
                        const float pv[3] = {(float)pbuf[u].x + shx, (float)pbuf[u].y + shy,
                                             (float)pbuf[u].z + shz};
                        float d2 = 0.f;
                        for (int d = 0; d < 3; ++d) {
                            const float g = fmaxf(fabsf(pv[d] - c0[d]) - h0[d], 0.f);
                            d2 += g * g;
                        }
                        keep = d2 < nb.cut2;
                        // within the list cut of the box: kept only when within
                        // it of one of the sub-cluster's atoms (a pair in range
                        // before the next rebuild is within the cut now)
                        if (keep) {
                            float m = 3.0e38f;
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float4 q = sm.ia[k];
                                const float dx = pv[0] - q.x, dy = pv[1] - q.y, dz = pv[2] - q.z;
                                m = fminf(m, dx * dx + dy * dy + dz * dz);
                            }
                            keep = m < nb.cut2;
                        }
                    }
                    const unsigned kbu = __ballot_sync(0xffffffffu, keep);
                    if (lane == 0) sm.kb[c] = kbu;
                }
            }
            __syncthreads();
            // exclusive prefix of the kept atoms over the candidates (two per thread)
            const int k0 = 2 * tid < nc ? __popc(sm.kb[2 * tid]) : 0;
            const int k1 = 2 * tid + 1 < nc ? __popc(sm.kb[2 * tid + 1]) : 0;
            int K = 0;
            const int ex = block_exscan(k0 + k1, sm.wsum, &K);
            if (2 * tid < nc) sm.kpre[2 * tid] = ex;
            if (2 * tid + 1 < nc) sm.kpre[2 * tid + 1] = ex + k0;
            // reserve exactly the tiles this round starts (none when the kept
            // atoms all fit in the open tile)
            if (K == 0) {
                __syncthreads();
                continue;
            }
            const int nnew = (nbuf + K + 31) / 32 - (nbuf > 0 ? 1 : 0);
            if (tid == 0) sm.r0 = nnew > 0 ? atomicAdd(s.flags + FL_NSTAGE, nnew) : 0;
            __syncthreads();
            const int r0 = sm.r0;
            if (!dead && r0 + nnew > nb.stage_cap) {
                dead = true;
                if (tid == 0) atomicOr(s.flags + FL_ERROR, ERRB_OVERFLOW);
                // the open tile keeps what it has
                if (nbuf > 0 && tid >= nbuf && tid < 32) nb.stage_j[(size_t)cur * 32 + tid] = -1;
            }
            const int total = nbuf + K;
            if (dead) {
                // the reserved slots inside the list are marked unused
                for (int k = r0 + tid; k < min(r0 + nnew, nb.stage_cap); k += NT)
                    nb.stage_hdr[k] = make_int4(0, 0, 0, -1);
            } else {
                for (int k = tid; k < nnew; k += NT) nb.stage_hdr[r0 + k] = make_int4(I8, sh, cls, count + k);
                // every kept atom knows its place: position nbuf + prefix in
                // the run of tiles that starts with the open one
                for (int c = wl; c < nc; c += TILE_WARPS) {
                    const unsigned kbu = sm.kb[c];
                    if (!((kbu >> lane) & 1u)) continue;
                    const int pos = nbuf + sm.kpre[c] + __popc(kbu & lt);
                    const int t = pos >> 5;
                    const int slot = nbuf > 0 ? (t == 0 ? cur : r0 + t - 1) : r0 + t;
                    nb.stage_j[(size_t)slot * 32 + (pos & 31)] = sm.cand[c] * 32 + lane;
                }
                const int tl = (total - 1) >> 5;
                cur = nbuf > 0 ? (tl == 0 ? cur : r0 + tl - 1) : r0 + tl;
            }
            count += nnew;
            nbuf = total & 31;
            if (nbuf == 0) cur = -1;
            __syncthreads();
        }
        if (nbuf > 0 && !dead && tid >= nbuf && tid < 32) nb.stage_j[(size_t)cur * 32 + tid] = -1;
    }
    return count;
}

// One block per i sub-cluster I8; its warps search the shifts that can bring
// partners within the cutoff one after another: every atom lies in [0, L),
// so a shift -1 (+1) along an axis is needed only if I8's box reaches within
// r_cut + skin of the lower (upper) face.  The block then turns the 27
// counts into offsets inside I8 (tile_cnt) and I8's total (tile_tot).
template <typename real>
__global__ void __launch_bounds__(TILE_WARPS * 32) k_tiles(SysView<real> s, NblView<real> nb)
{
    pdl_wait();
    pdl_trigger();
    __shared__ TileShared sm;
    const int I8 = blockIdx.x;
    const int tid = threadIdx.x, wl = tid >> 5, lane = tid & 31;
    const int I = I8 >> 2;
    const R4<float> ci = nb.bbc8[I8], hi = nb.bbh8[I8];
    const bool live = I < num_clusters(s, nb) && hi.w >= 0.f;
    bool ok = live && lane < 27;
    if (ok) {
        const float cut = sqrtf(nb.cut2);
        const float c0[3] = {ci.x, ci.y, ci.z}, h0[3] = {hi.x, hi.y, hi.z};
        int sv[3];
        shift_vec(lane, sv);
        for (int d = 0; d < 3; ++d) {
            if (sv[d] < 0 && !(c0[d] - h0[d] < cut)) ok = false;
            if (sv[d] > 0 && !(c0[d] + h0[d] > (float)s.L[d] - cut)) ok = false;
        }
    }
    const unsigned allow = __ballot_sync(0xffffffffu, ok);   // the same in every warp
    if (tid < 27) sm.cnt[tid] = 0;
    if (tid < 8) {
        const int slot = I8 * 8 + tid;
        const bool real_atom = live && slot < s.n_pad && s.perm[slot] >= 0;
        const R4<real> q = real_atom ? s.xq[slot] : R4<real>{0, 0, 0, 0};
        sm.ia[tid] = real_atom ? make_float4((float)q.x, (float)q.y, (float)q.z, 1.f)
                               : make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f);
    }
    __syncthreads();
    for (unsigned m = allow; m; m &= m - 1u) {
        const int sh = __ffs(m) - 1;
        const int count = tile_search(s, nb, I8, sh, sm);
        if (tid == 0) sm.cnt[sh] = count;
    }
    __syncthreads();
    // offsets of the shifts inside I8, and I8's total for the scan
    if (wl == 0) {
        const int c = lane < 27 ? sm.cnt[lane] : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane < 27) nb.tile_cnt[I8 * 27 + lane] = incl - c;
        if (lane == 26) nb.tile_tot[I8] = incl;
    }
}

// Placement and interaction masks.  Every staged tile goes to its place
// tile_off[I8] + (tiles of I8 under lower shifts) + ordinal.  Mask: one byte
// per j entry k, bit r set = pair (8 I8 + r, jidx[k]) is computed: both
// slots hold atoms, the pair is not excluded, and for a j atom of I8 itself
// under no shift, j > i.  The rows are formed first (one 32-bit row per i
// atom) and transposed by shuffles.  A warp takes four staged tiles at a
// time (lane = 8 tile + row), grid-striding over the staging list.
// Exclusions are searched only for rows whose molecule appears among the j
// atoms: for a molecule within 63 consecutive atom indices, each such j
// entry is tested against the row atom's exclusion bitmask (one bit per
// molecule-local index); otherwise each excluded partner's slot is looked up
// in the tile's ascending j slots by bisection.
constexpr int PLACE_BLOCKS_PER_SM = 16;
constexpr int PLACE_EX_BATCH = 8;     // exclusions looked up per batch of loads

template <typename real>
__global__ void __launch_bounds__(128) k_place(SysView<real> s, NblView<real> nb)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int jsl[4][4][33];   // [warp][tile][k]: j slot (INT_MAX if empty)
    __shared__ unsigned char jloc[4][4][32];   // [warp][tile][k]: j atom - its molecule id (255: none or > 62)
    const int lane = threadIdx.x & 31, wl = (threadIdx.x >> 5) & 3;
    const int g = lane >> 3, r = lane & 7;
    const int nst = min(s.flags[FL_NSTAGE], nb.stage_cap);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; 4 * q < nst; q += nwarps) {
        // the four tiles' loads are issued phase by phase
        int4 h[4];
        int dest[4], js[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) h[u] = 4 * q + u < nst ? nb.stage_hdr[4 * q + u] : make_int4(0, 0, 0, -1);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            dest[u] = h[u].w >= 0 ? nb.tile_off[h[u].x] + nb.tile_cnt[h[u].x * 27 + h[u].y] + h[u].w : -1;
            if (dest[u] >= nb.cap) dest[u] = -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            js[u] = dest[u] >= 0 ? nb.stage_j[(size_t)(4 * q + u) * 32 + lane] : -1;
            if (js[u] >= s.n_pad) js[u] = -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = js[u] >= 0 ? s.perm[js[u]] : -1;
        int jm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) jm[u] = b[u] >= 0 ? nb.mol[b[u]] : -2;
        // the i row of this lane: tile g, atom 8 I8 + r
        const int gI8 = g == 0 ? h[0].x : (g == 1 ? h[1].x : (g == 2 ? h[2].x : h[3].x));
        const int islot = gI8 * 8 + r;
        const int a = s.perm[islot];
        const int ma = a >= 0 ? nb.mol[a] : -3;
        unsigned valid = 0u, same = 0u, before = 0u;
        int mydest = -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            jsl[wl][u][lane] = js[u] >= 0 ? js[u] : 0x7fffffff;
            jloc[wl][u][lane] = (b[u] >= 0 && b[u] - jm[u] <= 62) ? (unsigned char)(b[u] - jm[u]) : (unsigned char)255;
            const unsigned bal = __ballot_sync(0xffffffffu, b[u] >= 0);
            if (dest[u] >= 0) {
                nb.jidx[(size_t)dest[u] * 32 + lane] = js[u];
                if (lane == 0) nb.tiles[dest[u]] = make_int4(h[u].x, h[u].y, h[u].z, 0);
            }
            if (u == g) {
                valid = bal;
                mydest = dest[u];
            }
            // rows of tile u: j atoms of the row's molecule, and (no shift) the
            // j slots of I8 itself at or before the row's slot (not computed)
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                const int mr = __shfl_sync(0xffffffffu, ma, 8 * u + rr);
                const unsigned bs = __ballot_sync(0xffffffffu, jm[u] == mr);
                unsigned bb = 0u;
                if (h[u].y == 13)
                    bb = __ballot_sync(0xffffffffu, js[u] >= h[u].x * 8 && js[u] <= h[u].x * 8 + rr);
                if (lane == 8 * u + rr) {
                    same = bs;
                    before = bb;
                }
            }
        }
        __syncwarp();
        unsigned m = 0u;
        if (mydest >= 0) {
            const int* sl = jsl[wl][g];
            if (a >= 0) m = valid & ~before;
            const unsigned long long xm = (m & same) ? nb.exm[a] : 0ull;
            if ((m & same) && !(xm >> 63)) {
                // the row's molecule within 63 indices: entry k of the same
                // molecule is excluded when its bit in the row atom's mask is set
                for (unsigned t = m & same; t; t &= t - 1u) {
                    const int k = __ffs(t) - 1;
                    const int bl = jloc[wl][g][k];
                    if (bl < 63 && ((xm >> bl) & 1ull)) m &= ~(1u << k);
                }
            } else if (m & same) {
                // excluded partners' slots, PLACE_EX_BATCH loads in flight
                const int e0 = nb.ex_start[a], e1 = nb.ex_start[a + 1];
                for (int eb = e0; eb < e1; eb += PLACE_EX_BATCH) {
                    int sbv[PLACE_EX_BATCH];
#pragma unroll
                    for (int u = 0; u < PLACE_EX_BATCH; ++u) sbv[u] = eb + u < e1 ? nb.ex_list[eb + u] : -1;
#pragma unroll
                    for (int u = 0; u < PLACE_EX_BATCH; ++u) sbv[u] = sbv[u] >= 0 ? s.iperm[sbv[u]] : -1;
#pragma unroll
                    for (int u = 0; u < PLACE_EX_BATCH; ++u) {
                        const int sb = sbv[u];
                        if (sb < 0) continue;
                        int lo = 0, hi = 31;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (sl[mid] < sb) lo = mid + 1;
                            else hi = mid;
                        }
                        if (sl[lo] == sb) m &= ~(1u << lo);
                    }
                }
            }
        } else {
            m = 0u;
        }
        __syncwarp();
        // stored by j entry: lane k of tile u gathers bit k of the tile's 8 rows
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            unsigned col = 0u;
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) col |= ((__shfl_sync(0xffffffffu, m, 8 * u + rr) >> lane) & 1u) << rr;
            if (dest[u] >= 0) nb.masks[(size_t)dest[u] * 32 + lane] = (unsigned char)col;
        }
    }
}

// dense solute-solvent pair list: the computed pairs of the class-2 tiles
// (solute sub-cluster x solvent atoms) that lie within r_cut + skin at build
// time, in (tile, i, k) order.  Lanes hold the tile's j atoms; the 8 i atoms
// are broadcast one by one, so each row costs one ballot.
template <typename real, int WRITE>
__global__ void __launch_bounds__(128) k_uv_pairs(SysView<real> s, NblView<real> nb)
{
    pdl_wait();
    pdl_trigger();
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= nb.uv_tiles_max) return;
    const int nuvt = s.n_ucl > 0 ? min(nb.tile_off[4 * s.n_ucl], nb.cap) : 0;
    if (t == 0 && lane == 0 && !WRITE) {
        s.flags[FL_NUVT] = nuvt;
        if (nuvt > nb.uv_tiles_max) atomicOr(&s.flags[FL_ERROR], ERRB_OVERFLOW);
    }
    unsigned keep = 0u;   // row of lane i < 8: bits k of kept pairs (i, k)
    int4 tl = make_int4(0, 13, 0, 0);
    int js = -1;
    if (t < nuvt) {
        tl = nb.tiles[t];
        if (tl.z == 2) {
            js = nb.jidx[(size_t)t * 32 + lane];
            const unsigned mc = nb.masks[(size_t)t * 32 + lane];
            const R4<real> pi = s.xq[tl.x * 8 + (lane & 7)];
            const R4<real> pj = s.xq[js >= 0 ? js : 0];
            int sv[3];
            shift_vec(tl.y, sv);
            const float xj = (float)pj.x + sv[0] * (float)s.L[0];
            const float yj = (float)pj.y + sv[1] * (float)s.L[1];
            const float zj = (float)pj.z + sv[2] * (float)s.L[2];
            for (int i = 0; i < 8; ++i) {
                const float xi = __shfl_sync(0xffffffffu, (float)pi.x, i);
                const float yi = __shfl_sync(0xffffffffu, (float)pi.y, i);
                const float zi = __shfl_sync(0xffffffffu, (float)pi.z, i);
                const float dx = xj - xi, dy = yj - yi, dz = zj - zi;
                const bool in = js >= 0 && ((mc >> i) & 1u) && dx * dx + dy * dy + dz * dz < nb.cut2;
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (lane == i) keep = bal;
            }
        }
    }
    const int cnt = __popc(keep);
    if (!WRITE) {
        const int c = (int)warp_sum_ll(cnt);
        if (lane == 0) nb.uv_cnt[t] = c;
        return;
    }
    // exclusive prefix of the lanes' counts inside the tile
    int pre = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    int pos = nb.uv_off[t] + pre - cnt;
    const int si = tl.x * 8 + (lane & 7);
    for (int k = 0; k < 32; ++k) {
        const int jk = __shfl_sync(0xffffffffu, js, k);
        if ((keep >> k) & 1u) {
            if (pos < nb.uv_cap) nb.uvp[pos] = make_int4(si, jk, tl.y, 0);
            ++pos;
        }
    }
}

// The build is a chain of kernels on one stream: every kernel after the
// first is launched as a programmatic dependent of the one before it.
template <typename real>
void launch_build_nbl(const SysView<real>& s, const NblView<real>& nb, cudaStream_t st)
{
    const int B = 256;
    bool pdl = false;   // the first kernel follows whatever preceded the build
    if (s.n_solv > 0) {
        k_col_keys<real><<<(s.n_solv + B - 1) / B, B, 0, st>>>(s, nb);
        launch_k(true, k_scan_block<1>, 1, 1024, 0, st, nb.col_cnt, nb.col_start, nb.ncols, (int*)nullptr, 0,
                 (int*)nullptr, nb.col_cl, nb.n_cl_solv);
        launch_k(true, k_col_scatter<real>, (s.n_solv + B - 1) / B, B, 0, st, s, nb);
        launch_k(true, k_col_sort<real>, nb.ncols, COL_THREADS, 0, st, s, nb);
        pdl = true;
    }
    launch_k(pdl, k_assign<real>, (s.n_pad + B - 1) / B, B, 0, st, s, nb);
    launch_k(true, k_tiles<real>, nb.n_cl_max * 4, TILE_WARPS * 32, 0, st, s, nb);
    launch_k(true, k_scan_block<0>, 1, 1024, 0, st, nb.tile_tot, nb.tile_off, nb.n_cl_max * 4, s.flags + FL_NTILES,
             nb.cap, s.flags + FL_ERROR, (int*)nullptr, (int*)nullptr);
    const long long pq = ((long long)nb.stage_cap + 15) / 16;   // blocks of four warps x four tiles
    const long long pmax = (long long)nb.n_sm * PLACE_BLOCKS_PER_SM;
    launch_k(true, k_place<real>, (int)(pq < pmax ? pq : pmax), 128, 0, st, s, nb);
    if (s.n_ucl > 0) {
        const int ub = (nb.uv_tiles_max * 32 + 127) / 128;
        launch_k(true, k_uv_pairs<real, 0>, ub, 128, 0, st, s, nb);
        launch_k(true, k_scan_block<0>, 1, 1024, 0, st, nb.uv_cnt, nb.uv_off, nb.uv_tiles_max, s.flags + FL_NUV,
                 nb.uv_cap, s.flags + FL_ERROR, (int*)nullptr, (int*)nullptr);
        launch_k(true, k_uv_pairs<real, 1>, ub, 128, 0, st, s, nb);
    }
}

// ---------------------------------------------------- dynamic list pruning
// Between rebuilds the pair kernel can run on a shorter list cut from the
// built one (dynamic pruning of a buffered pair list): a j entry is kept when
// it lies within r_cut + b_in of one of the tile's i atoms whose pair with it
// is computed, at the positions of the pruning; every pair that comes within
// r_cut before the next pruning is kept as long as no atom moves more than
// b_in / 2 meanwhile (the integrator raises FL_PRUNE when one does).  Kept
// entries keep their order and their mask bytes; each run of tiles of one i
// sub-cluster, shift and class is packed into as few tiles as its kept
// entries need.  Three kernels: the keep masks and output places of each
// sub-cluster's tiles (one warp per sub-cluster), a scan of the sub-clusters'
// output counts, and the copy (one warp per tile).

// one warp per i sub-cluster, its 8 atoms held by every lane: for each of
// its built tiles (PRUNE_BATCH at a time, loads first) the kept j entries
// (bit l = entry l), the place of the tile's first kept entry in the
// sub-cluster's output (runs of one shift and class start on a whole tile)
// and whether the tile ends its run; then the output tile count
constexpr int PRUNE_BATCH = 8;

template <typename real>
__global__ void __launch_bounds__(128) k_prune_count(SysView<real> s, NblView<real> nb, PruneView pv)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int I8 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (I8 >= 4 * nb.n_cl_max) return;
    const int ntot = min(s.flags[FL_NTILES], nb.cap);
    const int t0 = min(nb.tile_off[I8], ntot), t1 = min(nb.tile_off[I8 + 1], ntot);
    real ix[8], iy[8], iz[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const R4<real> q = t0 < t1 ? s.xq[I8 * 8 + r] : R4<real>{0, 0, 0, 0};
        ix[r] = q.x;
        iy[r] = q.y;
        iz[r] = q.z;
    }
    int pos = 0;     // entries placed (the same value in every lane)
    int prev = -1;   // run key of the previous tile
    for (int c = t0; c < t1; c += PRUNE_BATCH) {
        int4 h[PRUNE_BATCH];
        int sj[PRUNE_BATCH];
        unsigned mk[PRUNE_BATCH];
        R4<real> pj[PRUNE_BATCH];
#pragma unroll
        for (int u = 0; u < PRUNE_BATCH; ++u) {
            const int t = c + u;
            const bool in = t < t1;
            h[u] = in ? nb.tiles[t] : make_int4(0, 13, 0, 0);
            sj[u] = in ? nb.jidx[(size_t)t * 32 + lane] : -1;
            mk[u] = in ? nb.masks[(size_t)t * 32 + lane] : 0u;
        }
        const int4 hn = c + PRUNE_BATCH < t1 ? nb.tiles[c + PRUNE_BATCH] : make_int4(0, -1, 0, 0);
#pragma unroll
        for (int u = 0; u < PRUNE_BATCH; ++u) pj[u] = sj[u] >= 0 ? s.xq[sj[u]] : R4<real>{0, 0, 0, 0};
#pragma unroll
        for (int u = 0; u < PRUNE_BATCH; ++u) {
            const int t = c + u;
            if (t >= t1) break;
            int sv[3];
            shift_vec(h[u].y, sv);
            const real px = pj[u].x + (real)sv[0] * s.L[0];
            const real py = pj[u].y + (real)sv[1] * s.L[1];
            const real pz = pj[u].z + (real)sv[2] * s.L[2];
            real m2 = (real)3.0e38f;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const real dx = px - ix[r], dy = py - iy[r], dz = pz - iz[r];
                const real d2 = dx * dx + dy * dy + dz * dz;
                if ((mk[u] >> r) & 1u) m2 = fmin(m2, d2);
            }
            const unsigned kb = __ballot_sync(0xffffffffu, sj[u] >= 0 && mk[u] && m2 < (real)pv.cut2);
            const int key = h[u].y * 4 + h[u].z;
            if (key != prev) {
                pos = (pos + 31) & ~31;
                prev = key;
            }
            const int4 hx = u + 1 < PRUNE_BATCH ? h[u + 1] : hn;
            const bool close = t + 1 >= t1 || hx.y * 4 + hx.z != key;
            if (lane == 0) {
                pv.kb[t] = kb;
                pv.base[t] = pos | (close ? (1 << 30) : 0);
            }
            pos += __popc(kb);
        }
    }
    pos = (pos + 31) & ~31;
    if (lane == 0) pv.cnt[I8] = pos >> 5;
}

// one warp per built tile (PRUNE_WBATCH at a time, loads first): its kept
// entries (and, for a run's last tile, the padding of the run's last output
// tile) to their places; then the positions of this pruning become the
// reference of the next decision
constexpr int PRUNE_WBATCH = 4;

template <typename real>
__global__ void __launch_bounds__(128) k_prune_write(SysView<real> s, NblView<real> nb, NblView<real> np,
                                                     PruneView pv)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int ntot = min(s.flags[FL_NTILES], nb.cap);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (int t0 = w; t0 < ntot; t0 += PRUNE_WBATCH * nwarps) {
        int4 h[PRUNE_WBATCH];
        unsigned kb[PRUNE_WBATCH];
        int bw[PRUNE_WBATCH], o[PRUNE_WBATCH], sj[PRUNE_WBATCH];
        unsigned char mk[PRUNE_WBATCH];
#pragma unroll
        for (int u = 0; u < PRUNE_WBATCH; ++u) {
            const int t = t0 + u * nwarps;
            const bool in = t < ntot;
            h[u] = in ? nb.tiles[t] : make_int4(0, 0, 0, 0);
            kb[u] = in ? pv.kb[t] : 0u;
            bw[u] = in ? pv.base[t] : 0;
            sj[u] = in ? nb.jidx[(size_t)t * 32 + lane] : -1;
            mk[u] = in ? nb.masks[(size_t)t * 32 + lane] : (unsigned char)0;
        }
#pragma unroll
        for (int u = 0; u < PRUNE_WBATCH; ++u) o[u] = pv.off[h[u].x];
#pragma unroll
        for (int u = 0; u < PRUNE_WBATCH; ++u) {
            if (t0 + u * nwarps >= ntot) break;
            const int base = bw[u] & ((1 << 30) - 1);
            if ((kb[u] >> lane) & 1u) {
                const int p = base + __popc(kb[u] & lt);
                const int dt = o[u] + (p >> 5);
                if (dt < np.cap) {
                    np.jidx[(size_t)dt * 32 + (p & 31)] = sj[u];
                    np.masks[(size_t)dt * 32 + (p & 31)] = mk[u];
                    if ((p & 31) == 0) np.tiles[dt] = make_int4(h[u].x, h[u].y, h[u].z, 0);
                }
            }
            if ((bw[u] >> 30) & 1) {
                const int pend = base + __popc(kb[u]);
                const int dt = o[u] + (pend >> 5);
                if ((pend & 31) != 0 && lane >= (pend & 31) && dt < np.cap) {
                    np.jidx[(size_t)dt * 32 + lane] = -1;
                    np.masks[(size_t)dt * 32 + lane] = 0;
                }
            }
        }
    }
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < s.n; a += gridDim.x * blockDim.x) s.xpr[a] = s.x[a];
}

template <typename real>
void launch_prune(const SysView<real>& s, const NblView<real>& nb, const NblView<real>& np, const PruneView& pv,
                  cudaStream_t st)
{
    const int B = 128;
    const int grid_t = nb.n_sm * 8;
    launch_k(false, k_prune_count<real>, (4 * nb.n_cl_max * 32 + B - 1) / B, B, 0, st, s, nb, pv);
    launch_k(true, k_scan_block<0>, 1, 1024, 0, st, pv.cnt, pv.off, 4 * nb.n_cl_max, s.flags + FL_PTILES, np.cap,
             s.flags + FL_ERROR, (int*)nullptr, (int*)nullptr);
    launch_k(true, k_prune_write<real>, grid_t, B, 0, st, s, nb, np, pv);
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

// erfc(x) and exp(-x^2).  FP32: exp(-x^2) P(t), t = 1/(1 + p x), with a
// degree-7 least-squares fit of erfc(x) exp(x^2) on [0, 4.2] (relative
// error below 5e-8 in exact arithmetic; the fit is reproduced by
// tests/fit_erfc.py).  FP64: the library functions.
__device__ __forceinline__ void erfc_exp(float x, float& erfcv, float& ex)
{
    const float t = __fdividef(1.0f, fmaf(0.345f, x, 1.0f));
    float p = -0.23825677533960984f;
    p = fmaf(p, t, 1.0079999846654213f);
    p = fmaf(p, t, -1.1369167351186891f);
    p = fmaf(p, t, 1.1592655395537621f);
    p = fmaf(p, t, -0.30407340842765385f);
    p = fmaf(p, t, 0.33999728300708898f);
    p = fmaf(p, t, 0.17020566942397877f);
    p = fmaf(p, t, 0.0017784231330017291f);
    ex = __expf(-x * x);
    erfcv = p * ex;
}
__device__ __forceinline__ void erfc_exp(double x, double& erfcv, double& ex)
{
    erfcv = erfc(x);
    ex = exp(-x * x);
}

// Force and energy of one pair within the cutoff (dx, dy, dz = r_j - r_i):
// returns g with force on i = -g (dx, dy, dz) and on j = +g (dx, dy, dz);
// energy = ec + v (Coulomb erfc and switched LJ; uv energies are formed in
// FP64 elsewhere).  For solute-solvent pairs g mixes the bases with h_A and
// the capped soft basis (Eq. 5-6) with h_B.
template <typename real>
struct PairConst {
    real rc2, swi, rsw_swi, alpha, tas, hA, hB;
    bool sc;                 // soft-core coupling of the solute-solvent LJ
    real sc_a1l, sc_lp;      // sc_alpha (1 - lambda), lambda^p
};

template <typename real>
__device__ __forceinline__ real pair_force(real r2, real qq, real sg, real e4, bool uv, const PairConst<real>& c,
                                           real& ec, real& v)
{
    const real rinv = rsqrt_(r2);
    const real r = r2 * rinv;
    const real rinv2 = rinv * rinv;
    real erfcv, ex;
    erfc_exp(c.alpha * r, erfcv, ex);
    ec = qq * erfcv * rinv;
    const real fc = (ec + qq * c.tas * ex) * rinv2;
    const real s2 = sg * sg * rinv2;
    const real s6 = s2 * s2 * s2;
    v = e4 * (s6 * s6 - s6);
    real fl = e4 * ((real)12 * s6 * s6 - (real)6 * s6) * rinv2;
    const real tt = fmax((real)0, r * c.swi - c.rsw_swi);
    const real tt2 = tt * tt;
    const real S = (real)1 - tt2 * tt * ((real)10 - (real)15 * tt + (real)6 * tt2);
    const real omt = (real)1 - tt;
    const real dS = (real)-30 * tt2 * omt * omt * c.swi;
    fl = fl * S - v * dS * rinv;
    v *= S;
    real g = fc + fl;
    if (uv && c.sc) {
        // soft-core coupling: the solute-solvent LJ is the Beutler form at
        // lambda, e4 l^p (1/D^2 - 1/D) S(r) with D = alpha (1 - l) + (r/sigma)^6;
        // Coulomb keeps the h_A weight
        real gs = 0;
        if (e4 != (real)0) {
            const real x6 = (real)1 / s6;     // (r / sigma_ij)^6
            const real D = c.sc_a1l + x6, iD = (real)1 / D;
            const real u = iD * iD - iD;
            const real du = (iD - (real)2 * iD * iD) * iD;   // d(1/D^2 - 1/D)/dD
            const real e = e4 * c.sc_lp;
            gs = -e * (du * (real)6 * x6 * rinv * S + u * dS) * rinv;
        }
        return c.hA * fc + gs;
    }
    if (uv) {
        // capped soft basis (Eq. 5-6): identical to LJ for r >= sigma_ij
        real fs = fl;
        if (e4 == (real)0) {
            fs = 0;
        } else if (r < sg) {
            const real sgi = (real)1 / sg;
            const real x = r * sgi, x2 = x * x, x3 = x2 * x;
            const real u = ((real)-868 * x2 + (real)2188.8 * x - (real)1440) * x3 * x + (real)119.2;
            const real du = ((real)-5208 * x2 + (real)10944 * x - (real)5760) * x3;
            fs = -(real)0.25 * e4 * (du * sgi * S + u * dS) * rinv;
        }
        g = c.hA * g + c.hB * fs;
    }
    return g;
}

template <typename real>
__device__ __forceinline__ PairConst<real> pair_const(const SysView<real>& s)
{
    PairConst<real> c;
    c.rc2 = s.rc2;
    c.swi = s.sw_inv_w;
    c.rsw_swi = s.rsw * s.sw_inv_w;
    c.alpha = s.alpha;
    c.tas = s.two_a_sqrtpi;
    c.hA = (real)s.lam->hA;
    c.hB = (real)s.lam->hB;
    c.sc = s.sc_alpha > 0.0;
    c.sc_a1l = c.sc_lp = 0;
    if (c.sc) {
        const double l = s.lam->lambda;
        c.sc_a1l = (real)(s.sc_alpha * (1.0 - l));
        c.sc_lp = (real)pow(l, s.sc_power);
    }
    return c;
}

// The 24 i-force sums of an 8-atom sub-cluster (x, y, z of each atom), held
// per lane, are added over the warp by halving exchanges (each lane keeps
// the half its partner does not: 12, 6, 3 values) and two final butterfly
// steps; lane 4 k then holds atom k's totals and writes them.
template <typename real>
__device__ __forceinline__ void flush_i8_v(const SysView<real>& s, int I8, real (&v)[24])
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 12, o = 16; h >= 3; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int m = 0; m < h; ++m) {
            const real a = v[m], b = v[m + h];
            v[m] = (up ? b : a) + __shfl_xor_sync(FULL, up ? a : b, o);
        }
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        v[m] += __shfl_xor_sync(FULL, v[m], 2);
        v[m] += __shfl_xor_sync(FULL, v[m], 1);
    }
    if ((lane & 3) == 0) {
        const int k = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        flush_force(s, I8 * 8 + k, to_fixed(v[0], FSCALE), to_fixed(v[1], FSCALE), to_fixed(v[2], FSCALE));
    }
}

template <typename real>
__device__ __forceinline__ void flush_i8(const SysView<real>& s, int I8, real (&fx)[8], real (&fy)[8],
                                         real (&fz)[8])
{
    real v[24];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[3 * k] = fx[k];
        v[3 * k + 1] = fy[k];
        v[3 * k + 2] = fz[k];
    }
    flush_i8_v(s, I8, v);
}

// ---------------------------------------------------- packed FP32 pair kernel
// Blackwell issues two FP32 fused multiply-adds, multiplies or adds as one
// packed instruction (f32x2).  k_pairs2 evaluates the pairs of a lane's j
// atom with i atoms k and k + 4 of the tile as the two halves of float2
// values, so one step covers two pairs: half the steps and about half the
// instructions of the scalar kernel.  Each half rounds exactly like the
// scalar code (the packed operations are per component fmaf/fmul/fadd in
// round-to-nearest); the special-function operations (rsqrt, reciprocal,
// exp2) run once per half.
// The special-function unit's approximations (PTX rsqrt/rcp/ex2 .approx)
// in their flush-to-zero form: no subnormal handling around them.  For any
// pair within the cutoff the arguments and results are far from the
// subnormal range (r^2 of two atoms, 1 + 0.345 x >= 1, 2^y with y > -126
// while alpha r_c < 9), so the results are those of the non-flushing forms,
// with fewer instructions per pair.
__device__ __forceinline__ float rsq_ftz(float a)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float rcp_ftz(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float ex2_ftz(float a)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// pair_force for two pairs: (r2, qq, sigma_ij, 4 eps_ij) per half; returns g
// per half (force on i = -g d, on j = +g d) and the energy ec + v per half.
// Solvent-solvent and solute-solute classes only (the solute-solvent tiles
// take the scalar routine with the soft basis).  exp(-x^2) is 2^(-x^2 log2 e).
// The switching variable is clamped to [0, 1] (a saturating fma; for a pair
// within the cutoff it lies in [0, 1) already), so a half evaluated at
// r^2 = 1e30 (a pair out of range) gives exactly zero force and energy:
// erfc and the Gaussian underflow to 0, (sigma/r)^6 to 0, and S(1) = 0.
__device__ __forceinline__ float2 pair_force2(float2 r2, float2 qq, float2 sg, float2 e4, const PairConst<float>& c,
                                              float2& e)
{
    const float2 rinv = make_float2(rsq_ftz(r2.x), rsq_ftz(r2.y));
    const float2 r = mul2(r2, rinv);
    const float2 ri2 = mul2(rinv, rinv);
    const float2 x = mul2(p2(c.alpha), r);
    const float2 den = fma2(p2(0.345f), x, p2(1.0f));
    const float2 t = make_float2(rcp_ftz(den.x), rcp_ftz(den.y));
    float2 pp = p2(-0.23825677533960984f);
    pp = fma2(pp, t, p2(1.0079999846654213f));
    pp = fma2(pp, t, p2(-1.1369167351186891f));
    pp = fma2(pp, t, p2(1.1592655395537621f));
    pp = fma2(pp, t, p2(-0.30407340842765385f));
    pp = fma2(pp, t, p2(0.33999728300708898f));
    pp = fma2(pp, t, p2(0.17020566942397877f));
    pp = fma2(pp, t, p2(0.0017784231330017291f));
    const float2 xx = mul2(mul2(x, x), p2(-1.4426950408889634f));
    const float2 ex = make_float2(ex2_ftz(xx.x), ex2_ftz(xx.y));
    const float2 erfcv = mul2(pp, ex);
    const float2 ec = mul2(mul2(qq, erfcv), rinv);
    const float2 fc = mul2(fma2(mul2(qq, p2(c.tas)), ex, ec), ri2);
    const float2 s2 = mul2(mul2(sg, sg), ri2);
    const float2 s6 = mul2(mul2(s2, s2), s2);
    float2 v = mul2(e4, fma2(s6, s6, neg2(s6)));
    float2 fl = mul2(mul2(e4, mul2(s6, fma2(s6, p2(12.0f), p2(-6.0f)))), ri2);
    const float2 tt = make_float2(__saturatef(fmaf(r.x, c.swi, -c.rsw_swi)), __saturatef(fmaf(r.y, c.swi, -c.rsw_swi)));
    const float2 tt2 = mul2(tt, tt);
    const float2 inner = fma2(fma2(tt, p2(6.0f), p2(-15.0f)), tt, p2(10.0f));
    const float2 S = fma2(neg2(mul2(tt2, tt)), inner, p2(1.0f));
    const float2 omt = add2(p2(1.0f), neg2(tt));
    const float2 dS = mul2(mul2(tt2, mul2(omt, omt)), p2(-30.0f * c.swi));
    fl = fma2(fl, S, neg2(mul2(mul2(v, dS), rinv)));
    v = mul2(v, S);
    e = add2(ec, v);
    return add2(fc, fl);
}

// The tile list is cut into chunks of PAIR_CHUNK consecutive tiles; a warp
// takes whole chunks.  Lane l holds j entry l of a tile; step kk = 0..3
// pairs the j atom with i atoms kk and kk + 4 (read as float2 halves from a
// per-warp shared record, shifted for the tile) and is skipped by the whole
// warp when none of its 64 pairs lies within the cutoff.  A lane's share of
// the 8 i-forces is kept as float2 in its own column of a per-warp shared
// array and added over the warp when the sub-cluster changes or the chunk
// ends; the lane's FP32 energy sums are turned into fixed point at the same
// points.  So every partial sum covers a set of tiles fixed by the list
// alone (a chunk, or its part of one sub-cluster): the results do not depend
// on which warp takes which chunk, and a launch over many systems gives each
// system the bits of its own launch.  The j-force stays in registers and is
// flushed at the end of every tile.  The tile's class and shift are uniform,
// so the branches on them are warp-uniform; solute-solvent tiles take the
// scalar routine with the soft basis (their energies are formed in FP64 by
// k_uv_energy).
// Launch shape, measured on the octanol box (13,520 atoms, one wave, CUDA
// events): 8 resident blocks of 4 warps (i-forces in shared memory) 41.5 us;
// the same with the i-forces in registers (4 blocks) 41.4 us but a slower
// step (0.149 against 0.142 ms: the kernel shares the GPU with the PME and
// integrator branches); software prefetch of the next tile 42.5 us; the
// scalar kernel 45.8 us.
// resident blocks the register budget is cut for: 8 (64 registers) runs the
// kernel in 43 us against 52 us at 6 (80 registers) and 54 us at 7 (72) on
// the octanol box; inside the step, with the grid at 4 blocks per SM, budgets
// of 79, 91 and 107 registers gave 114.8-115.6, 122.1-122.6 and 125.1-125.5
// us per step against 115.2-117.4 at 64
constexpr int PAIR2_MIN_BLOCKS = 8;
constexpr int PAIR_CHUNK = 8;

struct Pair2Shared {
    // [warp][kk] (x_kk, x_kk+4, y_kk, y_kk+4), (z.., z.., q.., q..), (sigma/2.., .., 2 sqrt(eps).., ..)
    float4 sA[4][4], sB[4][4], sC[4][4];
    float2 sfi[4][12][32];   // [warp][3 kk + component][lane]: i atoms kk (x) and kk + 4 (y)
};

struct Pair2Acc {
    long long evv = 0, euu = 0;   // fixed-point energies (ESCALE)
    int npairs = 0;
};

// chunks [c0, c1) of one system, by one warp
__device__ __forceinline__ void pairs2_chunks(const SysView<float>& s, const NblView<float>& nb, int ntiles, int c0,
                                              int c1, Pair2Shared& sh, Pair2Acc& acc)
{
    const int lane = threadIdx.x & 31, wl = (threadIdx.x >> 5) & 3;
    const PairConst<float> c = pair_const(s);
    float* fA = reinterpret_cast<float*>(sh.sA[wl]);
    float* fB = reinterpret_cast<float*>(sh.sB[wl]);
    float* fC = reinterpret_cast<float*>(sh.sC[wl]);
    float2(&fi)[12][32] = sh.sfi[wl];
    const int hk = (lane & 3) * 4 + ((lane >> 2) & 1);   // lanes 0-7: place of atom `lane` in the records
    float evv = 0, euu = 0;
    auto flush = [&](int I8) {
        float v[24];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 ax = fi[3 * k][lane], ay = fi[3 * k + 1][lane], az = fi[3 * k + 2][lane];
            v[3 * k] = ax.x; v[3 * k + 1] = ay.x; v[3 * k + 2] = az.x;
            v[3 * k + 12] = ax.y; v[3 * k + 13] = ay.y; v[3 * k + 14] = az.y;
        }
        flush_i8_v(s, I8, v);
        acc.evv += to_fixed(evv, ESCALE);
        acc.euu += to_fixed(euu, ESCALE);
        evv = euu = 0;
    };
    for (int ch = c0; ch < c1; ++ch) {
        const int ta = ch * PAIR_CHUNK, tb = min(ta + PAIR_CHUNK, ntiles);
        int curI = -1, curSh = -1;
        float offx = 0.0f, offy = 0.0f, offz = 0.0f;   // the j side's shift (-L where the code says -1)
        for (int t = ta; t < tb; ++t) {
            const int4 tl = nb.tiles[t];
            const unsigned mc = nb.masks[(size_t)t * 32 + lane];
            const int slot_j = nb.jidx[(size_t)t * 32 + lane];
            R4<float> pj = s.xq[slot_j >= 0 ? slot_j : 0];
            const R2<float> ljv = s.lj[slot_j >= 0 ? slot_j : 0];
            if (tl.x != curI) {
                if (curI >= 0) flush(curI);
                curI = tl.x;
                curSh = -1;
                if (lane < 8) {
                    const R2<float> l = s.lj[curI * 8 + lane];
                    fC[hk] = l.x;
                    fC[hk + 2] = l.y;
                }
#pragma unroll
                for (int m = 0; m < 12; ++m) fi[m][lane] = p2(0.0f);
            }
            const int sh3 = tl.y;
            // shift the far-side atom down by L so that the subtraction below is
            // the only rounding in the pair vector; the i record and the j
            // side's offsets change only with the sub-cluster or the shift
            // (tiles come in runs of one sub-cluster and shift)
            if (sh3 != curSh) {
                curSh = sh3;
                const int sx = sh3 % 3 - 1, sy = (sh3 / 3) % 3 - 1, sz = sh3 / 9 - 1;
                offx = sx == -1 ? -s.L[0] : 0.0f;
                offy = sy == -1 ? -s.L[1] : 0.0f;
                offz = sz == -1 ? -s.L[2] : 0.0f;
                if (lane < 8) {
                    // i atom 8 curI + lane, read again (an L1 hit) rather than
                    // held in registers across the sub-cluster's tiles
                    const R4<float> pown = s.xq[curI * 8 + lane];
                    fA[hk] = sx == 1 ? pown.x - s.L[0] : pown.x;
                    fA[hk + 2] = sy == 1 ? pown.y - s.L[1] : pown.y;
                    fB[hk] = sz == 1 ? pown.z - s.L[2] : pown.z;
                    fB[hk + 2] = pown.w;
                }
            }
            pj.x += offx;
            pj.y += offy;
            pj.z += offz;
            __syncwarp();
            const float2 jx = p2(pj.x), jy = p2(pj.y), jz = p2(pj.z);
            float fjx, fjy, fjz, e0;
            if (tl.z != 2) {
                const float2 qj = p2(pj.w), sgj = p2(ljv.x), ej = p2(ljv.y);
                float2 fj2x = p2(0.0f), fj2y = p2(0.0f), fj2z = p2(0.0f), e2 = p2(0.0f);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4 A = sh.sA[wl][kk], B = sh.sB[wl][kk];
                    const float2 dx = add2(jx, neg2(make_float2(A.x, A.y)));
                    const float2 dy = add2(jy, neg2(make_float2(A.z, A.w)));
                    const float2 dz = add2(jz, neg2(make_float2(B.x, B.y)));
                    const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                    const bool in0 = ((mc >> kk) & 1u) && r2.x < c.rc2;
                    const bool in1 = ((mc >> (kk + 4)) & 1u) && r2.y < c.rc2;
                    if (__any_sync(0xffffffffu, in0 || in1)) {
                        // a half out of range is evaluated at r^2 = 1e30, where
                        // pair_force2 returns exact zeros (a warp-uniform branch:
                        // lanes with no pair in range take part with zeros)
                        const float4 C = sh.sC[wl][kk];
                        const float2 rs = make_float2(in0 ? r2.x : 1e30f, in1 ? r2.y : 1e30f);
                        float2 e;
                        float2 g = pair_force2(rs, mul2(make_float2(B.z, B.w), qj), add2(make_float2(C.x, C.y), sgj),
                                               mul2(make_float2(C.z, C.w), ej), c, e);
                        const float2 gx = mul2(g, dx), gy = mul2(g, dy), gz = mul2(g, dz);
                        fi[3 * kk][lane] = add2(fi[3 * kk][lane], neg2(gx));
                        fi[3 * kk + 1][lane] = add2(fi[3 * kk + 1][lane], neg2(gy));
                        fi[3 * kk + 2][lane] = add2(fi[3 * kk + 2][lane], neg2(gz));
                        fj2x = add2(fj2x, gx);
                        fj2y = add2(fj2y, gy);
                        fj2z = add2(fj2z, gz);
                        e2 = add2(e, e2);
                        acc.npairs += (in0 ? 1 : 0) + (in1 ? 1 : 0);
                    }
                }
                fjx = fj2x.x + fj2x.y;
                fjy = fj2y.x + fj2y.y;
                fjz = fj2z.x + fj2z.y;
                e0 = e2.x + e2.y;
            } else {
                // solute-solvent tile: the scalar routine with the soft basis, both halves
                fjx = fjy = fjz = e0 = 0.0f;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4 A = sh.sA[wl][kk], B = sh.sB[wl][kk], C = sh.sC[wl][kk];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float ix = h ? A.y : A.x, iy = h ? A.w : A.z, iz = h ? B.y : B.x, iq = h ? B.w : B.z;
                        const float isg = h ? C.y : C.x, ie = h ? C.w : C.z;
                        const float dx = pj.x - ix, dy = pj.y - iy, dz = pj.z - iz;
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        if (((mc >> (kk + 4 * h)) & 1u) && r2 < c.rc2) {
                            float ec, v;
                            const float g = pair_force(r2, iq * pj.w, isg + ljv.x, ie * ljv.y, true, c, ec, v);
                            const float gx = g * dx, gy = g * dy, gz = g * dz;
                            float2 f0 = fi[3 * kk][lane], f1 = fi[3 * kk + 1][lane], f2 = fi[3 * kk + 2][lane];
                            if (h) {
                                f0.y -= gx; f1.y -= gy; f2.y -= gz;
                            } else {
                                f0.x -= gx; f1.x -= gy; f2.x -= gz;
                            }
                            fi[3 * kk][lane] = f0;
                            fi[3 * kk + 1][lane] = f1;
                            fi[3 * kk + 2][lane] = f2;
                            fjx += gx; fjy += gy; fjz += gz;
                            ++acc.npairs;
                        }
                    }
                }
            }
            __syncwarp();
            if (slot_j >= 0)
                flush_force(s, slot_j, to_fixed(fjx, FSCALE), to_fixed(fjy, FSCALE), to_fixed(fjz, FSCALE));
            if (tl.z == 0) evv += e0;
            else if (tl.z == 1) euu += e0;
        }
        if (curI >= 0) flush(curI);
    }
}

// the warp's energy and pair-count sums into the system's accumulators
__device__ __forceinline__ void pairs2_store(const SysView<float>& s, Pair2Acc& acc)
{
    const long long a0 = warp_sum_ll(acc.evv), a1 = warp_sum_ll(acc.euu), a4 = warp_sum_ll((long long)acc.npairs);
    if ((threadIdx.x & 31) == 0) {
        if (a0) atomic_add_ll(&s.E[E_PAIR_VV], a0);
        if (a1) atomic_add_ll(&s.E[E_PAIR_UU], a1);
        if (a4) atomic_add_ll(&s.E[E_NPAIRS], a4);
    }
    acc = Pair2Acc{};
}

// One system's chunks, handed out in order from the system's chunk counter
// to the warps of the blocks along x as they become free, so that warps that
// drew light chunks take more and the grid ends together.  A chunk's result
// does not depend on the warp that evaluates it (its FP32 sums are formed
// within the chunk, then added as fixed point), so the outcome is the same
// for any assignment.  The last warp to finish sets both counters back to
// zero for the next launch: every warp fences its last counter update before
// it counts itself finished.
__device__ __forceinline__ void pairs2_system(const SysView<float>& s, const NblView<float>& nb, Pair2Shared& sh)
{
    const int lane = threadIdx.x & 31;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    const int ntiles = min(s.flags[nb.ntiles_flag], nb.cap);
    const int nch = (ntiles + PAIR_CHUNK - 1) / PAIR_CHUNK;
    Pair2Acc acc;
    for (;;) {
        int ch = 0;
        if (lane == 0) ch = atomicAdd(&s.flags[FL_PCHUNK], 1);
        ch = __shfl_sync(0xffffffffu, ch, 0);
        if (ch >= nch) break;
        pairs2_chunks(s, nb, ntiles, ch, ch + 1, sh, acc);
    }
    pairs2_store(s, acc);
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(&s.flags[FL_PDONE], 1) == nwarp - 1) {
            atomicExch(&s.flags[FL_PCHUNK], 0);
            atomicExch(&s.flags[FL_PDONE], 0);
        }
    }
}

// One launch for one or many systems: blockIdx.y picks the system, whose
// views are read from the launch's parameter space (a uniform index); its
// blocks along x share out its chunks.  A single system is a launch with one
// row, so a system stepped alone and the same system in a batched launch run
// the same compiled code over the same chunks: their results are identical
// bit for bit.
__global__ void __launch_bounds__(128, PAIR2_MIN_BLOCKS) k_pairs2(const __grid_constant__ PairJobs P)
{
    // the step's end kernels, programmatic dependents, may be scheduled from
    // here on; each waits for this grid to complete before it reads anything
    pdl_trigger();
    __shared__ Pair2Shared sh;
    pairs2_system(P.j[blockIdx.y].s, P.j[blockIdx.y].nb, sh);
}

// The FP64 pair kernel.  One warp walks a contiguous chunk of the
// (I8-sorted) tile list, one 8 x 32 tile at a time, in three phases per tile.  Lane l holds j entry l of the
// tile; the 8 i atoms are broadcast from a per-warp shared-memory record.
// (1) Every lane tests its j atom against the 8 i atoms (mask bit and
// r < r_cut); the pairs in range are listed in shared memory, i atom by i
// atom (ballot and prefix count), one byte (i, j) per pair.  (2) The list is
// evaluated 32 pairs at a time, one pair per lane, so nearly every lane of
// every round computes a pair in range (about 36 % of a tile's 256 slots are
// in range); the j record comes from its owner lane by shuffles, and each
// pair's force g (r_j - r_i) goes to a per-warp [3][8][32] shared matrix at
// (i, j).  (3) Lane j adds its column: the j atom's force, and its share of
// each i atom's force, which stays in registers over consecutive tiles of
// the same I8 and is added over the warp when I8 changes.  No atomics except
// the final fixed-point force and energy sums.  The tile's class (vv, uu or
// uv) and shift are uniform, so the branches on them are warp-uniform.
// Solute-solvent energies are not accumulated here (k_uv_energy forms them).
// With B300's few FP64 units the pair arithmetic dominates, and listing the
// pairs cuts it to the pairs in range (octanol box: 1.47 ms against 2.17 ms
// for the lane-per-j-entry kernel); in FP32, where latency dominates, the
// lane-per-j-entry kernel is faster (45.8 against 54.8 us) and is used.
template <typename real>
__global__ void __launch_bounds__(128, sizeof(real) == 4 ? 4 : 3) k_pairs_listed(SysView<real> s, NblView<real> nb)
{
    __shared__ R4<real> sxq[4][8];        // [warp][i atom] x, y, z (shifted for the tile), sqrt(k_e) q
    __shared__ R2<real> slj[4][8];        // [warp][i atom] sigma/2, 2 sqrt(eps)
    __shared__ unsigned char slist[4][256];   // [warp][pair] (i << 5) | j of the pairs in range
    __shared__ real sw[4][3][8][32];      // [warp][component][i][j] g (r_j - r_i) of each pair in range
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wl = (threadIdx.x >> 5) & 3;
    const unsigned lt = (1u << lane) - 1u;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    int ntiles = s.flags[nb.ntiles_flag];
    if (ntiles > nb.cap) ntiles = nb.cap;
    const int t0 = (int)(((long long)ntiles * warp) / nwarp);
    const int t1 = (int)(((long long)ntiles * (warp + 1)) / nwarp);
    if (t0 >= t1) return;
    const PairConst<real> c = pair_const(s);
    int curI = -1;
    R4<real> pown = {0, 0, 0, 0};   // lanes 0-7: i atom 8 curI + lane, unshifted
    real fx[8], fy[8], fz[8];
    real evv = 0, euu = 0;
    int npairs = 0;
    // the next tile's records are loaded while the current one is computed
    int4 tl_n = nb.tiles[t0];
    unsigned mk_n = nb.masks[(size_t)t0 * 32 + lane];
    int sj_n = nb.jidx[(size_t)t0 * 32 + lane];
    R4<real> pj_n = s.xq[sj_n >= 0 ? sj_n : 0];
    R2<real> lj_n = s.lj[sj_n >= 0 ? sj_n : 0];
    for (int t = t0; t < t1; ++t) {
        const int4 tl = tl_n;
        const unsigned mc = mk_n;
        const int slot_j = sj_n;
        R4<real> pj = pj_n;
        const R2<real> ljv = lj_n;
        if (t + 1 < t1) {
            tl_n = nb.tiles[t + 1];
            mk_n = nb.masks[(size_t)(t + 1) * 32 + lane];
            sj_n = nb.jidx[(size_t)(t + 1) * 32 + lane];
            pj_n = s.xq[sj_n >= 0 ? sj_n : 0];
            lj_n = s.lj[sj_n >= 0 ? sj_n : 0];
        }
        if (tl.x != curI) {
            if (curI >= 0) flush_i8(s, curI, fx, fy, fz);
            curI = tl.x;
            if (lane < 8) {
                pown = s.xq[curI * 8 + lane];
                slj[wl][lane] = s.lj[curI * 8 + lane];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) fx[k] = fy[k] = fz[k] = 0;
        }
        const int sh = tl.y;
        const int sx = sh % 3 - 1, sy = (sh / 3) % 3 - 1, sz = sh / 9 - 1;
        // shift the far-side atom down by L so that the subtraction below is
        // the only rounding in the pair vector
        if (lane < 8)
            sxq[wl][lane] = R4<real>{sx == 1 ? pown.x - s.L[0] : pown.x, sy == 1 ? pown.y - s.L[1] : pown.y,
                                     sz == 1 ? pown.z - s.L[2] : pown.z, pown.w};
        if (sx == -1) pj.x -= s.L[0];
        if (sy == -1) pj.y -= s.L[1];
        if (sz == -1) pj.z -= s.L[2];
        __syncwarp();
        // (1) list the pairs in range
        unsigned vb = 0u;
        int np = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const R4<real> pi = sxq[wl][k];
            const real dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const real r2 = dx * dx + dy * dy + dz * dz;
            const bool in = ((mc >> k) & 1u) && r2 < c.rc2;
            const unsigned bal = __ballot_sync(FULL, in);
            if (in) slist[wl][np + __popc(bal & lt)] = (unsigned char)((k << 5) | lane);
            vb |= (in ? 1u : 0u) << k;
            np += __popc(bal);
        }
        __syncwarp();
        // (2) one pair per lane
        const bool uv = tl.z == 2;
        real e0 = 0;
        for (int r0 = 0; r0 < np; r0 += 32) {
            const int idx = r0 + lane;
            const bool act = idx < np;
            const int code = act ? (int)slist[wl][idx] : 0;
            const int k = code >> 5, j = code & 31;
            const real xj = __shfl_sync(FULL, pj.x, j), yj = __shfl_sync(FULL, pj.y, j);
            const real zj = __shfl_sync(FULL, pj.z, j), qj = __shfl_sync(FULL, pj.w, j);
            const real sj = __shfl_sync(FULL, ljv.x, j), ej = __shfl_sync(FULL, ljv.y, j);
            if (act) {
                const R4<real> pi = sxq[wl][k];
                const R2<real> li = slj[wl][k];
                const real dx = xj - pi.x, dy = yj - pi.y, dz = zj - pi.z;
                const real r2 = dx * dx + dy * dy + dz * dz;
                real ec, v;
                const real g = pair_force(r2, pi.w * qj, li.x + sj, li.y * ej, uv, c, ec, v);
                sw[wl][0][k][j] = g * dx;
                sw[wl][1][k][j] = g * dy;
                sw[wl][2][k][j] = g * dz;
                e0 += ec + v;
                ++npairs;
            }
        }
        __syncwarp();
        // (3) the column of lane j: its j force and its shares of the i forces
        real fjx = 0, fjy = 0, fjz = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if ((vb >> k) & 1u) {
                const real wx = sw[wl][0][k][lane], wy = sw[wl][1][k][lane], wz = sw[wl][2][k][lane];
                fjx += wx; fjy += wy; fjz += wz;
                fx[k] -= wx; fy[k] -= wy; fz[k] -= wz;
            }
        }
        __syncwarp();
        if (slot_j >= 0)
            flush_force(s, slot_j, to_fixed(fjx, FSCALE), to_fixed(fjy, FSCALE), to_fixed(fjz, FSCALE));
        if (tl.z == 0) evv += e0;
        else if (tl.z == 1) euu += e0;
    }
    flush_i8(s, curI, fx, fy, fz);
    const long long a0 = __double2ll_rn(warp_sum_d((double)evv) * ESCALE);
    const long long a1 = __double2ll_rn(warp_sum_d((double)euu) * ESCALE);
    const long long a4 = warp_sum_ll((long long)npairs);
    if (lane == 0) {
        if (a0) atomic_add_ll(&s.E[E_PAIR_VV], a0);
        if (a1) atomic_add_ll(&s.E[E_PAIR_UU], a1);
        atomic_add_ll(&s.E[E_NPAIRS], a4);
    }
}

// Solute-solvent basis energies U_uv (real-space part) and U_soft in FP64
// over the dense solute-solvent pair list.  They set dU/dlambda = h_A' U_uv +
// h_B' U_soft, whose tolerance (1e-6 relative) is below what FP32 pair
// arithmetic delivers; one thread per listed pair spreads the few thousand
// pairs over the FP64 pipes of every SM while the FP32 pair kernel computes
// the forces.  The pair vector is exact: coordinates are floats, their sums
// are exact in double.
template <typename real>
__global__ void __launch_bounds__(256) k_uv_energy(SysView<real> s, NblView<real> nb)
{
    const int n = min(s.flags[FL_NUV], nb.uv_cap);
    const double rc2 = (double)s.rc2, rsw = (double)s.rsw, swi = (double)s.sw_inv_w;
    const double alpha = (double)s.alpha;
    const bool sc = s.sc_alpha > 0.0;
    const double lam = s.lam->lambda;
    const double a1l = sc ? s.sc_alpha * (1.0 - lam) : 0.0, lp = sc ? pow(lam, s.sc_power) : 0.0;
    const double dlp = sc ? (s.sc_power == 1.0 ? 1.0 : s.sc_power * pow(lam, s.sc_power - 1.0)) : 0.0;
    double euv = 0.0, esoft = 0.0, edsc = 0.0;
    // consecutive pairs go to consecutive blocks, so that a list shorter than
    // the grid still spreads over every SM's FP64 units
    for (int w = threadIdx.x * gridDim.x + blockIdx.x; w < n; w += gridDim.x * blockDim.x) {
        const int4 pr = nb.uvp[w];
        const R4<real> pi = s.xq[pr.x], pj = s.xq[pr.y];
        int sv[3];
        shift_vec(pr.z, sv);
        const double dx = (double)pj.x + sv[0] * (double)s.L[0] - (double)pi.x;
        const double dy = (double)pj.y + sv[1] * (double)s.L[1] - (double)pi.y;
        const double dz = (double)pj.z + sv[2] * (double)s.L[2] - (double)pi.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < rc2)) continue;
        const int a = s.perm[pr.x], b = s.perm[pr.y];
        // one reciprocal square root serves r, 1/r and 1/r^2 (every FP64
        // division on this per-pair chain is a long dependent sequence)
        const double rinv = rsqrt(r2);
        const double r = r2 * rinv, rinv2 = rinv * rinv;
        const double qq = KE * (double)s.q[a] * (double)s.q[b];
        double e = qq * erfc(alpha * r) * rinv;
        const double sg = 0.5 * ((double)s.sig[a] + (double)s.sig[b]);
        const double ep = sqrt((double)s.eps[a] * (double)s.eps[b]);
        if (ep > 0.0 && sc) {
            // soft-core coupling at lambda: the energy and its lambda derivative
            const double tt = fmax(0.0, (r - rsw) * swi);
            const double S = 1.0 - tt * tt * tt * (10.0 - 15.0 * tt + 6.0 * tt * tt);
            const double x2 = r2 / (sg * sg), x6 = x2 * x2 * x2;
            const double D = a1l + x6, iD = 1.0 / D, u = iD * iD - iD;
            esoft += 4.0 * ep * lp * u * S;
            edsc += 4.0 * ep * S * (dlp * u + s.sc_alpha * lp * (2.0 * iD - 1.0) * iD * iD);
        } else if (ep > 0.0) {
            const double tt = fmax(0.0, (r - rsw) * swi);
            const double S = 1.0 - tt * tt * tt * (10.0 - 15.0 * tt + 6.0 * tt * tt);
            const double s2 = sg * sg * rinv2, s6 = s2 * s2 * s2;
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
    // a warp without a pair in range (most of a grid spread over every SM)
    // skips the FP64 reductions
    if (!__any_sync(0xffffffffu, euv != 0.0 || esoft != 0.0 || edsc != 0.0)) return;
    const long long a0 = __double2ll_rn(warp_sum_d(euv) * ESCALE);
    const long long a1 = __double2ll_rn(warp_sum_d(esoft) * ESCALE);
    const long long a2 = sc ? __double2ll_rn(warp_sum_d(edsc) * ESCALE) : 0ll;
    if ((threadIdx.x & 31) == 0) {
        if (a0) atomic_add_ll(&s.E[E_PAIR_UV], a0);
        if (a1) atomic_add_ll(&s.E[E_PAIR_SOFT], a1);
        if (a2) atomic_add_ll(&s.E[E_DSC], a2);
    }
}

template <typename real>
void launch_uv_energy(const SysView<real>& s, const NblView<real>& nb, int nblocks, cudaStream_t st)
{
    if (s.n_ucl == 0) return;
    k_uv_energy<real><<<nblocks, 256, 0, st>>>(s, nb);
}

// blocks of the pair kernel resident on one multiprocessor (its grid is one wave)
template <typename real>
int pairs_blocks_per_sm()
{
    int nb = 0;
    cudaError_t e;
    if constexpr (sizeof(real) == 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pairs_listed<real>, 128, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pairs2, 128, 0);
    if (e != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

int pairs_batch_blocks()
{
    int dev = 0, nsm = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || nsm < 1)
        nsm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pairs2, 128, 0) != cudaSuccess || nb < 1) nb = 1;
    return nsm * nb;
}

// jobs: host array; up to PAIR_BATCH_MAX systems per launch, each with
// nblocks / (systems in the launch) blocks (at least one)
void launch_pairs_batch(const PairJob* jobs, int njobs, int nblocks, cudaStream_t st)
{
    for (int j0 = 0; j0 < njobs; j0 += PAIR_BATCH_MAX) {
        const int cnt = min(PAIR_BATCH_MAX, njobs - j0);
        PairJobs P;
        for (int k = 0; k < cnt; ++k) P.j[k] = jobs[j0 + k];
        const int gx = max(1, nblocks / cnt);
        k_pairs2<<<dim3(gx, cnt), 128, 0, st>>>(P);
    }
}

template <typename real>
void launch_pairs(const SysView<real>& s, const NblView<real>& nb, int nwarps, cudaStream_t st)
{
    const int B = 128;
    const int blocks = (nwarps * 32 + B - 1) / B;
    if constexpr (sizeof(real) == 8) {
        k_pairs_listed<real><<<blocks, B, 0, st>>>(s, nb);
    } else {
        PairJob j{s, nb};
        launch_pairs_batch(&j, 1, blocks, st);
    }
}

// ------------------------------------------------- exclusions and 1-4 pairs
// excluded pair (any distance, minimum image): -k_e q_i q_j erf(alpha r)/r;
// 1-4 pair: s_C k_e q_i q_j / r + s_LJ 4 eps_ij [(s/r)^12 - (s/r)^6].
// Gathered per atom (four threads per atom over its exclusion and 1-4
// partner lists): each pair is evaluated from both ends, so every atom's
// force is one sum written with one set of atomics instead of one set per
// pair, and the energy is counted at the end with the lower index.
constexpr int EXCL_BATCH = 4;   // partners per lane whose records are loaded together

template <typename real>
__global__ void k_excl(SysView<real> s, ExclView<real> ex)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = tid >> 2, sub = tid & 3;
    // per-thread energy sums in the working precision (a few terms each),
    // added over the warp in FP64: the FP64 pipe, which several kernels of
    // the step share, does only the warp sums
    real acc[6] = {0, 0, 0, 0, 0, 0};   // excl vv, uu, uv, 14 vv, uu, uv
    real fx = 0, fy = 0, fz = 0;
    if (a < s.n) {
        // master positions, charges sqrt(k_e) q and (sigma / 2, 2 sqrt(eps)),
        // formed as for the cluster-sorted copy
        R4<real> pa = s.x[a];
        pa.w = s.q[a] * (real)sqrt(KE);
        const R2<real> la = {(real)0.5 * s.sig[a], (real)2 * sqrt(s.eps[a])};
        const int ua = s.sol[a];
        for (int pass = 0; pass < 2; ++pass) {
            const bool is14 = pass == 1;
            const int e0 = is14 ? ex.p14_start[a] : ex.ex_start[a];
            const int e1 = is14 ? ex.p14_start[a + 1] : ex.ex_start[a + 1];
          for (int eb = e0 + sub; eb < e1; eb += 4 * EXCL_BATCH) {
            // the partner records of a batch are loaded together (two
            // dependent rounds: partner, its coordinates and charge)
            int bb[EXCL_BATCH];
            R4<real> pbb[EXCL_BATCH];
#pragma unroll
            for (int u = 0; u < EXCL_BATCH; ++u) {
                const int e = eb + 4 * u;
                bb[u] = e < e1 ? (is14 ? ex.p14_list[e] : ex.ex_list[e]) : -1;
            }
#pragma unroll
            for (int u = 0; u < EXCL_BATCH; ++u)
                if (bb[u] >= 0) {
                    pbb[u] = s.x[bb[u]];
                    pbb[u].w = s.q[bb[u]] * (real)sqrt(KE);
                }
#pragma unroll
            for (int u = 0; u < EXCL_BATCH; ++u) {
                const int e = eb + 4 * u;
                if (e >= e1) break;
                const int b = bb[u];
                const R4<real> pb = pbb[u];
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
                        const R2<real> sc = ex.p14_s[e];
                        const R2<real> lb = {(real)0.5 * s.sig[b], (real)2 * sqrt(s.eps[b])};
                        en = sc.y * qq * rinv;
                        g = sc.y * qq * rinv2 * rinv;
                        const real sg = la.x + lb.x, e4 = la.y * lb.y;
                        if (e4 != (real)0) {
                            const real s2 = sg * sg * rinv2, s6 = s2 * s2 * s2;
                            en += sc.x * e4 * (s6 * s6 - s6);
                            g += sc.x * e4 * ((real)12 * s6 * s6 - (real)6 * s6) * rinv2;
                        }
                    }
                }
                // force on a: -g d (d = r_b - r_a)
                fx -= g * d[0];
                fy -= g * d[1];
                fz -= g * d[2];
                if (a < b) {
                    const int ub = s.sol[b];
                    const int cls = (ua && ub) ? 1 : ((ua || ub) ? 2 : 0);
                    const int slotk = (is14 ? 3 : 0) + cls;
#pragma unroll
                    for (int c = 0; c < 6; ++c)
                        if (c == slotk) acc[c] += en;   // constant indices: acc stays in registers
                }
            }
          }
        }
    }
    for (int o = 1; o < 4; o <<= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (a < s.n && sub == 0 && (fx != (real)0 || fy != (real)0 || fz != (real)0)) {
        atomic_add_ll(&s.Fa[a], to_fixed(fx, FSCALE));
        atomic_add_ll(&s.Fa[s.n + a], to_fixed(fy, FSCALE));
        atomic_add_ll(&s.Fa[2 * s.n + a], to_fixed(fz, FSCALE));
    }
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < 6; ++c) {
        long long v = __double2ll_rn(warp_sum_d((double)acc[c]) * ESCALE);
        if (lane == 0 && v) atomic_add_ll(&s.E[(c < 3 ? E_EXCL_VV : E_14_VV) + (c % 3)], v);
    }
}

template <typename real>
void launch_excl(const SysView<real>& s, const ExclView<real>& ex, cudaStream_t st)
{
    if (ex.n_excl + ex.n14 == 0) return;
    const int B = 256;
    k_excl<real><<<(4 * s.n + B - 1) / B, B, 0, st>>>(s, ex);
}

#define LFE_INST(real)                                                                             \
    template void launch_build_nbl<real>(const SysView<real>&, const NblView<real>&, cudaStream_t); \
    template void launch_prune<real>(const SysView<real>&, const NblView<real>&, const NblView<real>&,  \
                                     const PruneView&, cudaStream_t);                                    \
    template void launch_pairs<real>(const SysView<real>&, const NblView<real>&, int, cudaStream_t); \
    template int pairs_blocks_per_sm<real>();                                                          \
    template void launch_uv_energy<real>(const SysView<real>&, const NblView<real>&, int, cudaStream_t); \
    template void launch_excl<real>(const SysView<real>&, const ExclView<real>&, cudaStream_t);
LFE_INST(float)
LFE_INST(double)

}  // namespace lfe
