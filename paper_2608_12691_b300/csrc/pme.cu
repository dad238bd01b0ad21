// pme.cu -- smooth particle-mesh Ewald with the solute/solvent class split.
//
// Essmann et al. (1995), cited for PME in Section 2.6: order-4 cardinal
// B-spline charge spreading, a 3-D transform, multiplication by the influence
// function G(m) = k_e exp(-pi^2 m^2/alpha^2) B(m) / (pi V m^2), and force
// interpolation with the B-spline derivatives.  The solvent grid Q_v and the
// solute grid Q_u are packed into one complex grid Z = Q_v + i Q_u, so one
// complex transform serves both classes; the convolution separates them
// again, forms E_vv, E_uu and E_uv (Eq. 4 basis split of the reciprocal
// energy), and packs the two class potentials the forces need,
//   solvent atoms: phi_v + h_A phi_u,   solute atoms: phi_u + h_A phi_v,
// into one complex grid for the single inverse transform.
#include "lfe_views.cuh"
#include "pme_dev.cuh"
#include <type_traits>

namespace lfe {

// Four lanes per atom: lanes 0-2 of the group form the FP64 B-spline
// weights of one dimension each and share them by shuffles; lane j0 then
// spreads the 16 points of plane j0 of the atom's 4 x 4 x 4 stencil.  The
// products are formed in the same order as by one lane per atom.  Weights
// and products in FP64: the fixed-point grid is shared by the force branch
// and the df64 energy branch, whose class energies set dU/dlambda to 1e-6
// relative.
// round-to-nearest-even of x to int64 (saturating beyond 2^63, NaN to 0),
// the result of __double2ll_rn, with integer operations only: x = m 2^sh
// with the 53-bit significand m, shifted into place and rounded on the bits
// shifted out.  The spread's conversions then stay off the FP64 pipe, which
// its products keep busy.
__device__ __forceinline__ long long d2ll_rn_int(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffull);
    const unsigned long long frac = b & 0xfffffffffffffull;
    const unsigned long long m = frac | 0x10000000000000ull;
    const int sh = e - 1075;
    unsigned long long mag;
    if (sh >= 0) {
        mag = sh > 10 ? 0x7fffffffffffffffull : (m << sh);
    } else if (sh < -53 || e == 0) {
        mag = 0ull;
    } else {
        const int r = -sh;
        const unsigned long long q = m >> r, rem = m & ((1ull << r) - 1ull), half = 1ull << (r - 1);
        mag = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
    }
    if (e == 2047 && frac) mag = 0ull;
    return (b >> 63) ? -(long long)mag : (long long)mag;
}

template <typename real>
__global__ void k_spread(SysView<real> s, PmeView<real> p)
{
    const unsigned FULL = 0xffffffffu;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int atom = tid >> 2, sub = tid & 3;
    const int lb = (threadIdx.x & 31) & ~3;
    int a = -1;
    real q = 0;
    R4<real> xq;
    xq.x = xq.y = xq.z = xq.w = (real)0;
    if (atom < s.n) {
        a = atom;
        xq = s.x[a];
        q = s.q[a];
    }
    double th[4], dth[4];
    int f;
    {
        const int d = sub < 3 ? sub : 2;
        const real x = d == 0 ? xq.x : (d == 1 ? xq.y : xq.z);
        double w;
        grid_coord(x, p.kscale64[d], p.K[d], f, w);
        bspline4(w, th, dth);
    }
    double t0[4], t1[4], t2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        t0[k] = __shfl_sync(FULL, th[k], lb);
        t1[k] = __shfl_sync(FULL, th[k], lb + 1);
        t2[k] = __shfl_sync(FULL, th[k], lb + 2);
    }
    const int f0 = __shfl_sync(FULL, f, lb), f1 = __shfl_sync(FULL, f, lb + 1), f2 = __shfl_sync(FULL, f, lb + 2);
    if (a < 0 || q == (real)0) return;
    long long* grid = p.Qfix + (s.sol[a] ? p.KK : 0);
    const double th0 = sub == 0 ? t0[0] : (sub == 1 ? t0[1] : (sub == 2 ? t0[2] : t0[3]));
    const int k0 = wrapk(f0 - sub, p.K[0]);
    // the grid scale is a power of two: applied first, it changes no bit
    // of the products
    const double a0 = (double)q * th0 * QSCALE;
#pragma unroll
    for (int j1 = 0; j1 < 4; ++j1) {
        const int k1 = wrapk(f1 - j1, p.K[1]);
        const double a1 = a0 * t1[j1];
        const int row = (k0 * p.K[1] + k1) * p.K[2];
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
            const int k2 = wrapk(f2 - j2, p.K[2]);
            atomic_add_ll(&grid[row + k2], d2ll_rn_int(a1 * t2[j2]));
        }
    }
}

// ------------------------------------------------------------------- FFT
template <typename real>
__device__ __forceinline__ R2<real> cmul(R2<real> a, R2<real> b)
{
    R2<real> r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename real>
__device__ __forceinline__ R2<real> cadd(R2<real> a, R2<real> b) { R2<real> r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename real>
__device__ __forceinline__ R2<real> csub(R2<real> a, R2<real> b) { R2<real> r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// multiply by sign * i
template <typename real>
__device__ __forceinline__ R2<real> cmuli(R2<real> a, int sign)
{
    R2<real> r;
    r.x = -(real)sign * a.y;
    r.y = (real)sign * a.x;
    return r;
}

// df64: the sign flip without a df64 product
template <>
__device__ __forceinline__ R2<df64> cmuli<df64>(R2<df64> a, int sign)
{
    R2<df64> r;
    r.x = sign > 0 ? -a.y : a.y;
    r.y = sign > 0 ? a.x : -a.x;
    return r;
}

// in-register R-point DFT y_k = sum_n a_n exp(sign 2 pi i n k / R)
template <typename real>
__device__ __forceinline__ void dft_small(R2<real>* v, int R, int sign)
{
    if (R == 2) {
        R2<real> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        R2<real> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        R2<real> s13 = cadd(v[1], v[3]), d13 = cmuli(csub(v[1], v[3]), sign);
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    } else if (R == 3) {
        const real h = (real)0.86602540378443864676;   // sqrt(3)/2
        R2<real> t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
        R2<real> m1;
        m1.x = v[0].x - (real)0.5 * t1.x;
        m1.y = v[0].y - (real)0.5 * t1.y;
        R2<real> m2 = cmuli(t2, sign);
        m2.x *= h; m2.y *= h;
        v[0] = cadd(v[0], t1);
        v[1] = cadd(m1, m2);
        v[2] = csub(m1, m2);
    } else {  // R == 5
        const real c1 = (real)0.30901699437494742410, c2 = (real)-0.80901699437494742410;
        const real s1 = (real)0.95105651629515357212, s2 = (real)0.58778525229247312917;
        R2<real> a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        R2<real> a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        R2<real> y0 = cadd(v[0], cadd(a1, a2));
        R2<real> p1, p2, q1, q2;
        p1.x = v[0].x + c1 * a1.x + c2 * a2.x; p1.y = v[0].y + c1 * a1.y + c2 * a2.y;
        p2.x = v[0].x + c2 * a1.x + c1 * a2.x; p2.y = v[0].y + c2 * a1.y + c1 * a2.y;
        q1.x = s1 * b1.x + s2 * b2.x; q1.y = s1 * b1.y + s2 * b2.y;
        q2.x = s2 * b1.x - s1 * b2.x; q2.y = s2 * b1.y - s1 * b2.y;
        q1 = cmuli(q1, sign);
        q2 = cmuli(q2, sign);
        v[0] = y0;
        v[1] = cadd(p1, q1);
        v[4] = csub(p1, q1);
        v[2] = cadd(p2, q2);
        v[3] = csub(p2, q2);
    }
}

// One Stockham stage of radix R (compile time, so the R values stay in
// registers) over nl lines of length K held in shared memory: point t of
// line l at buf[l * ls + t * es].  LF: consecutive threads take consecutive
// lines (strided lines), otherwise consecutive points of one line.  tw holds
// exp(sign 2 pi i t / K).
template <typename real, bool LF, int R>
__device__ __forceinline__ void smem_stage(const R2<real>* a, R2<real>* b, int nl, int K, int ls, int es, int Ns,
                                           const R2<real>* tw, int sign)
{
    const int nbf = K / R;
    const int tstep = K / (Ns * R);
    const int total = nl * nbf;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int l, j;
        if (LF) { l = idx % nl; j = idx / nl; }
        else { l = idx / nbf; j = idx - l * nbf; }
        const int k = j % Ns;
        const R2<real>* in = a + l * ls;
        R2<real>* out = b + l * ls;
        R2<real> v[R];
        v[0] = in[j * es];
        // r k tstep < K: no reduction of the twiddle index is needed
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(in[(j + r * nbf) * es], tw[r * k * tstep]);
        dft_small(v, R, sign);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[(base + r * Ns) * es] = v[r];
    }
}

// All stages of the radix plan; returns the buffer that holds the result.
template <typename real, bool LF>
__device__ R2<real>* smem_fft(R2<real>* a, R2<real>* b, int nl, int K, int ls, int es, const int* rad, int nrad,
                              const R2<real>* tw, int sign)
{
    int Ns = 1;
    for (int st = 0; st < nrad; ++st) {
        const int R = rad[st];
        if (R == 4) smem_stage<real, LF, 4>(a, b, nl, K, ls, es, Ns, tw, sign);
        else if (R == 2) smem_stage<real, LF, 2>(a, b, nl, K, ls, es, Ns, tw, sign);
        else if (R == 3) smem_stage<real, LF, 3>(a, b, nl, K, ls, es, Ns, tw, sign);
        else smem_stage<real, LF, 5>(a, b, nl, K, ls, es, Ns, tw, sign);
        __syncthreads();
        R2<real>* t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}


// One pass of 1-D transforms of length K along AXIS for a block of FFT_NL
// (16 in FP32, 4 in FP64, whose scarce units want more blocks in flight)
// lines, in shared memory, by the Stockham autosort formulation (radix 2, 3,
// 4, 5 stages).  AXIS 2 lines are contiguous; AXIS 1 and 0 lines are loaded
// as FFT_NL contiguous columns.  FROMFIX (FFT_FROM_FIX or
// FFT_FROM_FIX_KEEP): the input is the pair of fixed-point charge grids,
// consumed and zeroed here or left for another reader.
template <typename real, int AXIS, int FROMFIX, int FFT_NL>
__global__ void __launch_bounds__(256) k_fft(PmeView<real> p, int sign)
{
    extern __shared__ unsigned char smem_raw[];
    const int K = p.K[AXIS];
    const int LD = K + 1;   // padded line stride: the column loads of axes 0 and 1 hit distinct banks
    R2<real>* tw = reinterpret_cast<R2<real>*>(smem_raw);
    R2<real>* b0 = tw + K;
    R2<real>* b1 = b0 + FFT_NL * LD;
    const int K0 = p.K[0], K1 = p.K[1], K2 = p.K[2];
    const int tid = threadIdx.x, nt = blockDim.x;

    int line0 = 0, fixed_k = 0, c0 = 0, nl = FFT_NL;
    if (AXIS == 2) {
        line0 = blockIdx.x * FFT_NL;
        nl = min(FFT_NL, K0 * K1 - line0);
    } else {
        const int ncb = (K2 + FFT_NL - 1) / FFT_NL;
        fixed_k = blockIdx.x / ncb;
        c0 = (blockIdx.x % ncb) * FFT_NL;
        nl = min(FFT_NL, K2 - c0);
    }
    for (int t = tid; t < K; t += nt) {
        R2<real> w = p.tw[AXIS][t];
        if (sign < 0) w.y = -w.y;
        tw[t] = w;
    }
    auto gidx = [&](int l, int t) -> int {
        if (AXIS == 2) return (line0 + l) * K2 + t;
        if (AXIS == 1) return (fixed_k * K1 + t) * K2 + c0 + l;
        return (t * K1 + fixed_k) * K2 + c0 + l;
    };
    for (int e = tid; e < FFT_NL * K; e += nt) {
        int l, t;
        if (AXIS == 2) { l = e / K; t = e % K; }
        else { t = e / FFT_NL; l = e % FFT_NL; }
        if (l < nl) {
            const int g = gidx(l, t);
            R2<real> v;
            if (FROMFIX != FFT_FROM_Z) {
                const double qv = (double)p.Qfix[g] * (1.0 / QSCALE);
                const double qu = (double)p.Qfix[p.KK + g] * ((double)p.qu_scale / QSCALE);
                v.x = (real)qv;
                v.y = (real)qu;
                if (FROMFIX == FFT_FROM_FIX) {
                    p.Qfix[g] = 0;
                    p.Qfix[p.KK + g] = 0;
                }
                if (FROMFIX == FFT_FROM_FIX && p.Zraw64) {
                    R2<double> w;
                    w.x = qv;
                    w.y = qu;
                    p.Zraw64[g] = w;
                }
            } else if (AXIS == 2 && p.Zin64) {
                const R2<double> w = p.Zin64[g];
                v.x = (real)w.x;
                v.y = (real)w.y;
            } else {
                v = p.Z[g];
            }
            b0[l * LD + t] = v;
        }
    }
    __syncthreads();
    const R2<real>* src = smem_fft<real, false>(b0, b1, nl, K, LD, 1, p.rad[AXIS], p.nrad[AXIS], tw, sign);
    for (int e = tid; e < FFT_NL * K; e += nt) {
        int l, t;
        if (AXIS == 2) { l = e / K; t = e % K; }
        else { t = e / FFT_NL; l = e % FFT_NL; }
        if (l < nl) p.Z[gidx(l, t)] = src[l * LD + t];
    }
}

// Lines per block of a per-axis pass: 16 in FP32; 4 in FP64, whose scarce
// units want more blocks in flight; 16 in df64 (FP32 pipes; measured: step
// 0.149 ms against 0.152 with 8 and 0.155 with 4 lines on the octanol box)
// when the block fits in 48 KB of shared memory, else 4.
template <typename real, int NL>
size_t fft_smem_nl(int K)
{
    return sizeof(R2<real>) * (size_t)(K + 2 * NL * (K + 1));
}

template <typename real>
int fft_lines(int K)
{
    if (sizeof(real) == 4) return 16;
    if (std::is_same<real, df64>::value && fft_smem_nl<real, 16>(K) <= 48 * 1024) return 16;
    return 4;
}

template <typename real>
size_t fft_smem(int K)
{
    return fft_lines<real>(K) == 16 ? fft_smem_nl<real, 16>(K) : fft_smem_nl<real, 4>(K);
}

template <typename real, int NL>
void launch_fft_nl(const PmeView<real>& p, int axis, int sign, int from_fixed, cudaStream_t st)
{
    const int threads = 16 * NL;
    const int K = p.K[axis];
    const size_t smem = fft_smem_nl<real, NL>(K);
    int blocks;
    if (axis == 2) blocks = (p.K[0] * p.K[1] + NL - 1) / NL;
    else blocks = p.K[axis == 1 ? 0 : 1] * ((p.K[2] + NL - 1) / NL);
    if (axis == 2) {
        if (from_fixed == FFT_FROM_FIX) k_fft<real, 2, FFT_FROM_FIX, NL><<<blocks, threads, smem, st>>>(p, sign);
        else if (from_fixed == FFT_FROM_FIX_KEEP)
            k_fft<real, 2, FFT_FROM_FIX_KEEP, NL><<<blocks, threads, smem, st>>>(p, sign);
        else k_fft<real, 2, FFT_FROM_Z, NL><<<blocks, threads, smem, st>>>(p, sign);
    } else if (axis == 1) {
        k_fft<real, 1, FFT_FROM_Z, NL><<<blocks, threads, smem, st>>>(p, sign);
    } else {
        k_fft<real, 0, FFT_FROM_Z, NL><<<blocks, threads, smem, st>>>(p, sign);
    }
}

template <typename real>
void launch_fft(const PmeView<real>& p, int axis, int sign, int from_fixed, cudaStream_t st)
{
    if constexpr (sizeof(real) == 4) {
        launch_fft_nl<real, 16>(p, axis, sign, from_fixed, st);
    } else if constexpr (std::is_same<real, df64>::value) {
        if (p.lines != 4 && fft_lines<real>(p.K[axis]) == 16) launch_fft_nl<real, 16>(p, axis, sign, from_fixed, st);
        else launch_fft_nl<real, 4>(p, axis, sign, from_fixed, st);
    } else {
        launch_fft_nl<real, 4>(p, axis, sign, from_fixed, st);
    }
}

// ------------------------------------------ plane / column transform
// The 3-D transform as two kinds of kernels instead of one launch per axis:
// a plane kernel transforms the K1 x K2 plane of one k0 along axes 2 and 1
// in shared memory, and a column kernel transforms groups of axis-0 columns,
// applies the convolution to every (m, -m) pair (each column group holds the
// partner column (-k1, -k2) of each of its columns) and, for the potentials,
// transforms back along axis 0.  Forward: planes then columns; inverse:
// (columns) then planes.

template <typename real>
__device__ __forceinline__ void load_twiddles(R2<real>* dst, const R2<real>* src, int K, int sign)
{
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
        R2<real> w = src[t];
        if (sign < 0) w.y = -w.y;
        dst[t] = w;
    }
}

constexpr int PLANE_THREADS = 512;
constexpr int LOAD_BATCH = 8;     // global loads per thread issued together
constexpr int COL_THREADS = 256;

template <typename real, int MODE>
__global__ void __launch_bounds__(PLANE_THREADS) k_plane(PmeView<real> p)
{
    extern __shared__ unsigned char smem_raw[];
    const int K1 = p.K[1], K2 = p.K[2];
    const int LD = K2 + 1;
    const int sign = MODE == PLANE_INV ? -1 : +1;
    R2<real>* tw2 = reinterpret_cast<R2<real>*>(smem_raw);
    R2<real>* tw1 = tw2 + K2;
    R2<real>* a = tw1 + K1;
    R2<real>* b = a + K1 * LD;
    const int k0 = blockIdx.x;
    load_twiddles(tw2, p.tw[2], K2, sign);
    load_twiddles(tw1, p.tw[1], K1, sign);
    const int base = k0 * K1 * K2;
    const int KP = K1 * K2;
    // all of a thread's loads of a chunk are issued before any store, so
    // they are in flight together
    for (int e0 = 0; e0 < KP; e0 += LOAD_BATCH * PLANE_THREADS) {
        long long qa[LOAD_BATCH], qb[LOAD_BATCH];
        R2<real> zv[LOAD_BATCH];
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u) {
            const int e = e0 + u * PLANE_THREADS + threadIdx.x;
            if (e < KP) {
                if (MODE == PLANE_FWD_FIX || MODE == PLANE_FWD_KEEP) {
                    qa[u] = p.Qfix[base + e];
                    qb[u] = p.Qfix[p.KK + base + e];
                } else {
                    zv[u] = p.Z[base + e];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u) {
            const int e = e0 + u * PLANE_THREADS + threadIdx.x;
            if (e >= KP) continue;
            const int k1 = e / K2, k2 = e - k1 * K2;
            const int g = base + e;
            R2<real> v;
            if (MODE == PLANE_FWD_FIX || MODE == PLANE_FWD_KEEP) {
                const double qv = (double)qa[u] * (1.0 / QSCALE);
                const double qu = (double)qb[u] * ((double)p.qu_scale / QSCALE);
                v.x = (real)qv;
                v.y = (real)qu;
                if (MODE == PLANE_FWD_FIX) {
                    p.Qfix[g] = 0;
                    p.Qfix[p.KK + g] = 0;
                }
                if (MODE == PLANE_FWD_FIX && p.Zraw64) {
                    R2<double> w;
                    w.x = qv;
                    w.y = qu;
                    p.Zraw64[g] = w;
                }
            } else {
                v = zv[u];
            }
            a[k1 * LD + k2] = v;
        }
    }
    __syncthreads();
    R2<real>* r;
    if (MODE == PLANE_INV) {
        r = smem_fft<real, true>(a, b, K2, K1, 1, LD, p.rad[1], p.nrad[1], tw1, sign);
        r = smem_fft<real, false>(r, r == a ? b : a, K1, K2, LD, 1, p.rad[2], p.nrad[2], tw2, sign);
    } else {
        r = smem_fft<real, false>(a, b, K1, K2, LD, 1, p.rad[2], p.nrad[2], tw2, sign);
        r = smem_fft<real, true>(r, r == a ? b : a, K2, K1, 1, LD, p.rad[1], p.nrad[1], tw1, sign);
    }
    for (int e = threadIdx.x; e < K1 * K2; e += blockDim.x) {
        const int k1 = e / K2, k2 = e - k1 * K2;
        p.Z[base + e] = r[k1 * LD + k2];
    }
}

template <typename real, int MODE>
__global__ void __launch_bounds__(COL_THREADS) k_columns(PmeView<real> p, long long* E, const LamState* lam)
{
    pdl_trigger();   // (theta's step, a programmatic dependent in the step graph, waits for completion)
    extern __shared__ unsigned char smem_raw[];
    __shared__ double red[3][COL_THREADS / 32];
    const int K0 = p.K[0], K1 = p.K[1], K2 = p.K[2];
    const int K12 = K1 * K2;
    const int LD = K0 + 1;
    const int g0 = p.cg_start[blockIdx.x];
    const int nc = p.cg_start[blockIdx.x + 1] - g0;
    R2<real>* twf = reinterpret_cast<R2<real>*>(smem_raw);
    R2<real>* twi = twf + K0;
    R2<real>* a = twi + K0;
    R2<real>* b = a + p.cg_max * LD;
    int* cols = reinterpret_cast<int*>(b + p.cg_max * LD);
    int* part = cols + p.cg_max;
    load_twiddles(twf, p.tw[0], K0, +1);
    load_twiddles(twi, p.tw[0], K0, -1);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        cols[c] = p.cg_col[g0 + c];
        part[c] = p.cg_part[g0 + c];
    }
    __syncthreads();
    for (int e0 = 0; e0 < nc * K0; e0 += LOAD_BATCH * COL_THREADS) {
        R2<real> zv[LOAD_BATCH];
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u) {
            const int e = e0 + u * COL_THREADS + threadIdx.x;
            if (e < nc * K0) {
                const int k0 = e / nc, c = e - k0 * nc;
                zv[u] = p.Z[k0 * K12 + cols[c]];
            }
        }
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u) {
            const int e = e0 + u * COL_THREADS + threadIdx.x;
            if (e < nc * K0) {
                const int k0 = e / nc, c = e - k0 * nc;
                a[c * LD + k0] = zv[u];
            }
        }
    }
    __syncthreads();
    R2<real>* r = smem_fft<real, false>(a, b, nc, K0, LD, 1, p.rad[0], p.nrad[0], twf, +1);
    double evv = 0, euu = 0, euv = 0;
    // df64: the energy products and their per-thread sums stay in df64 (FP32
    // pipes); one conversion to double per thread at the end
    real evv2 = (real)0, euu2 = (real)0, euv2 = (real)0;
    constexpr bool DF = std::is_same<real, df64>::value;
    const real hA = MODE != CONV_ENERGY ? (real)lam->hA : (real)0;
    for (int e = threadIdx.x; e < nc * K0; e += blockDim.x) {
        const int c = e / K0, k0 = e - c * K0;
        const int pc = part[c];
        const int n0 = k0 == 0 ? 0 : K0 - k0;
        if (!(c < pc || (c == pc && k0 <= n0))) continue;   // each (m, -m) pair once
        const int col = cols[c];
        if (k0 == 0 && col == 0) {
            if (MODE != CONV_ENERGY) {
                R2<real> zero;
                zero.x = zero.y = (real)0;
                r[c * LD] = zero;
            }
            continue;
        }
        const int k1 = col / K2, k2 = col - k1 * K2;
        const R2<real> zm = r[c * LD + k0], zn = r[pc * LD + n0];
        // Z = Q_v + i s Q_u:  Q_v(m) = (Z(m) + conj Z(-m)) / 2,  Q_u(m) = (Z(m) - conj Z(-m)) / (2 i s)
        R2<real> qv, qu;
        const real hs = (real)0.5 / p.qu_scale;
        qv.x = (real)0.5 * (zm.x + zn.x);
        qv.y = (real)0.5 * (zm.y - zn.y);
        qu.x = hs * (zm.y + zn.y);
        qu.y = -hs * (zm.x - zn.x);
        const real msq = p.msq[0][k0] + p.msq[1][k1] + p.msq[2][k2];
        const real G = p.conv_pre * p.gfac[0][k0] * p.gfac[1][k1] * p.gfac[2][k2] / msq;
        const bool self = (c == pc && k0 == n0);
        if (MODE != CONV_POTENTIAL) {
            if constexpr (DF) {
                const real g = self ? G * (real)0.5 : G;   // halving or doubling by 2 is exact
                evv2 += g * (qv.x * qv.x + qv.y * qv.y);
                euu2 += g * (qu.x * qu.x + qu.y * qu.y);
                euv2 += (g + g) * (qu.x * qv.x + qu.y * qv.y);
            } else {
                const double mult = self ? 1.0 : 2.0;
                evv += mult * 0.5 * (double)G * ((double)qv.x * (double)qv.x + (double)qv.y * (double)qv.y);
                euu += mult * 0.5 * (double)G * ((double)qu.x * (double)qu.x + (double)qu.y * (double)qu.y);
                euv += mult * (double)G * ((double)qu.x * (double)qv.x + (double)qu.y * (double)qv.y);
            }
        }
        if (MODE != CONV_ENERGY) {
            // W = G [(Q_v + h_A Q_u) + i (Q_u + h_A Q_v)]; at -m the class
            // spectra are the complex conjugates
            R2<real> P, Rr, wm, wn;
            P.x = qv.x + hA * qu.x; P.y = qv.y + hA * qu.y;
            Rr.x = qu.x + hA * qv.x; Rr.y = qu.y + hA * qv.y;
            wm.x = G * (P.x - Rr.y); wm.y = G * (P.y + Rr.x);
            wn.x = G * (P.x + Rr.y); wn.y = G * (-P.y + Rr.x);
            r[c * LD + k0] = wm;
            if (!self) r[pc * LD + n0] = wn;
        }
    }
    if (MODE != CONV_POTENTIAL) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if constexpr (DF) {
            evv = (double)evv2;
            euu = (double)euu2;
            euv = (double)euv2;
        }
        const double v0 = warp_sum_d(evv), v1 = warp_sum_d(euu), v2 = warp_sum_d(euv);
        if (lane == 0) { red[0][warp] = v0; red[1][warp] = v1; red[2][warp] = v2; }
        __syncthreads();
        if (threadIdx.x < 3) {
            double v = 0;
            for (int w = 0; w < COL_THREADS / 32; ++w) v += red[threadIdx.x][w];
            const long long f = __double2ll_rn(v * ESCALE);
            if (f) atomic_add_ll(&E[E_REC_VV + threadIdx.x], f);
        }
    }
    if (MODE == CONV_ENERGY) return;
    __syncthreads();
    R2<real>* o = smem_fft<real, false>(r, r == a ? b : a, nc, K0, LD, 1, p.rad[0], p.nrad[0], twi, -1);
    for (int e = threadIdx.x; e < nc * K0; e += blockDim.x) {
        const int k0 = e / nc, c = e - k0 * nc;
        p.Z[k0 * K12 + cols[c]] = o[c * LD + k0];
    }
}

template <typename real>
size_t planes_smem(const PmeView<real>& p)
{
    return sizeof(R2<real>) * (size_t)(p.K[2] + p.K[1] + 2 * p.K[1] * (p.K[2] + 1));
}

template <typename real>
size_t columns_smem(const PmeView<real>& p)
{
    return sizeof(R2<real>) * (size_t)(2 * p.K[0] + 2 * p.cg_max * (p.K[0] + 1)) + 2 * sizeof(int) * (size_t)p.cg_max;
}

// The attribute is per kernel and process-wide, while systems with
// different grids share the kernels: allow the device's whole opt-in
// shared memory (less the kernel's static shared memory) rather than this
// grid's need.
template <typename K>
static void allow_max_smem(K kernel, int optin)
{
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <typename real>
void planes_setup(const PmeView<real>& p)
{
    (void)p;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    allow_max_smem(k_plane<real, PLANE_FWD_FIX>, optin);
    allow_max_smem(k_plane<real, PLANE_FWD_KEEP>, optin);
    allow_max_smem(k_plane<real, PLANE_FWD>, optin);
    allow_max_smem(k_plane<real, PLANE_INV>, optin);
    allow_max_smem(k_columns<real, CONV_ENERGY>, optin);
    allow_max_smem(k_columns<real, CONV_POTENTIAL>, optin);
    allow_max_smem(k_columns<real, CONV_BOTH>, optin);
}

// the column pass of an energy-only branch (no plane kernels)
template <typename real>
void energy_columns_setup(const PmeView<real>& p)
{
    (void)p;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    allow_max_smem(k_columns<real, CONV_ENERGY>, optin);
}

template <typename real>
void launch_planes(const PmeView<real>& p, int mode, cudaStream_t st)
{
    const size_t sm = planes_smem(p);
    if (mode == PLANE_FWD_FIX) k_plane<real, PLANE_FWD_FIX><<<p.K[0], PLANE_THREADS, sm, st>>>(p);
    else if (mode == PLANE_FWD_KEEP) k_plane<real, PLANE_FWD_KEEP><<<p.K[0], PLANE_THREADS, sm, st>>>(p);
    else if (mode == PLANE_FWD) k_plane<real, PLANE_FWD><<<p.K[0], PLANE_THREADS, sm, st>>>(p);
    else k_plane<real, PLANE_INV><<<p.K[0], PLANE_THREADS, sm, st>>>(p);
}

template <typename real>
void launch_columns(const PmeView<real>& p, long long* E, const LamState* lam, int mode, cudaStream_t st)
{
    const size_t sm = columns_smem(p);
    if (mode == CONV_ENERGY) k_columns<real, CONV_ENERGY><<<p.ngroups, COL_THREADS, sm, st>>>(p, E, lam);
    else if (mode == CONV_POTENTIAL) k_columns<real, CONV_POTENTIAL><<<p.ngroups, COL_THREADS, sm, st>>>(p, E, lam);
    else k_columns<real, CONV_BOTH><<<p.ngroups, COL_THREADS, sm, st>>>(p, E, lam);
}

// ------------------------------------------------------------ convolution
// CONV_ENERGY: E_vv, E_uu, E_uv only; CONV_POTENTIAL: the packed class
// potentials only; CONV_BOTH: both.
template <typename real, int MODE>
__global__ void k_conv(PmeView<real> p, long long* E, const LamState* lam)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int K0 = p.K[0], K1 = p.K[1], K2 = p.K[2];
    double evv = 0, euu = 0, euv = 0;
    if (idx < p.KK) {
        const int k0 = idx / (K1 * K2), k1 = (idx / K2) % K1, k2 = idx % K2;
        const int n0 = (K0 - k0) % K0, n1 = (K1 - k1) % K1, n2 = (K2 - k2) % K2;
        const int nidx = (n0 * K1 + n1) * K2 + n2;
        if (idx == 0) {
            if (MODE != CONV_ENERGY) {
                R2<real> zero;
                zero.x = zero.y = (real)0;
                p.Z[0] = zero;
            }
        } else if (idx <= nidx) {
            const R2<real> zm = p.Z[idx], zn = p.Z[nidx];
            // Z = Q_v + i s Q_u (s = qu_scale, a power of two that brings the
            // solute spectrum to the solvent's magnitude so that the transform's
            // rounding is relative to each class):
            // Q_v(m) = (Z(m) + conj Z(-m)) / 2,  Q_u(m) = (Z(m) - conj Z(-m)) / (2 i s)
            R2<real> qv, qu;
            const real hs = (real)0.5 / p.qu_scale;
            qv.x = (real)0.5 * (zm.x + zn.x);
            qv.y = (real)0.5 * (zm.y - zn.y);
            qu.x = hs * (zm.y + zn.y);
            qu.y = -hs * (zm.x - zn.x);
            const real msq = p.msq[0][k0] + p.msq[1][k1] + p.msq[2][k2];
            const real G = p.conv_pre * p.gfac[0][k0] * p.gfac[1][k1] * p.gfac[2][k2] / msq;
            if (MODE != CONV_POTENTIAL) {
                const double mult = (idx == nidx) ? 1.0 : 2.0;
                evv = mult * 0.5 * (double)G * ((double)qv.x * (double)qv.x + (double)qv.y * (double)qv.y);
                euu = mult * 0.5 * (double)G * ((double)qu.x * (double)qu.x + (double)qu.y * (double)qu.y);
                euv = mult * (double)G * ((double)qu.x * (double)qv.x + (double)qu.y * (double)qv.y);
            }
            if (MODE != CONV_ENERGY) {
                // W = G [(Q_v + h_A Q_u) + i (Q_u + h_A Q_v)]; at -m the class
                // spectra are the complex conjugates
                const real hA = (real)lam->hA;
                R2<real> P, Rr, wm, wn;
                P.x = qv.x + hA * qu.x; P.y = qv.y + hA * qu.y;
                Rr.x = qu.x + hA * qv.x; Rr.y = qu.y + hA * qv.y;
                wm.x = G * (P.x - Rr.y); wm.y = G * (P.y + Rr.x);
                wn.x = G * (P.x + Rr.y); wn.y = G * (-P.y + Rr.x);
                p.Z[idx] = wm;
                if (nidx != idx) p.Z[nidx] = wn;
            }
        }
    }
    if (MODE != CONV_POTENTIAL) {
        long long a0 = __double2ll_rn(warp_sum_d(evv) * ESCALE);
        long long a1 = __double2ll_rn(warp_sum_d(euu) * ESCALE);
        long long a2 = __double2ll_rn(warp_sum_d(euv) * ESCALE);
        if ((threadIdx.x & 31) == 0) {
            if (a0) atomic_add_ll(&E[E_REC_VV], a0);
            if (a1) atomic_add_ll(&E[E_REC_UU], a1);
            if (a2) atomic_add_ll(&E[E_REC_UV], a2);
        }
    }
}

// ----------------------------------------------------------------- gather
// Forces from the potential grid: four lanes per atom, as in the spread.
// Lane d < 3 forms the B-spline weights and derivatives of dimension d
// (lane 3 repeats dimension 2) and shares them by shuffles; lane j0 then
// reads the 16 points of plane j0 of the atom's 4 x 4 x 4 stencil, and the
// four partial gradients are added by two butterfly steps.  Four times the
// warps of one lane per atom, each with a quarter of the dependent grid
// reads.
template <typename real>
__global__ void k_gather(SysView<real> s, PmeView<real> p)
{
    const unsigned FULL = 0xffffffffu;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = tid >> 2, sub = tid & 3;
    const int lb = (threadIdx.x & 31) & ~3;
    const bool live = a < s.n;
    real q = 0;
    bool u = false;
    R4<real> xq;
    xq.x = xq.y = xq.z = xq.w = (real)0;
    if (live) {
        q = s.q[a];
        xq = s.x[a];
        u = s.sol[a] != 0;
    }
    real th[4], dth[4];
    int f;
    {
        const int d = sub < 3 ? sub : 2;
        const real x = d == 0 ? xq.x : (d == 1 ? xq.y : xq.z);
        real w;
        grid_coord(x, p.kscale64[d], p.K[d], f, w);
        bspline4(w, th, dth);
    }
    real t0[4], d0[4], t1[4], d1[4], t2[4], d2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        t0[k] = __shfl_sync(FULL, th[k], lb);
        d0[k] = __shfl_sync(FULL, dth[k], lb);
        t1[k] = __shfl_sync(FULL, th[k], lb + 1);
        d1[k] = __shfl_sync(FULL, dth[k], lb + 1);
        t2[k] = __shfl_sync(FULL, th[k], lb + 2);
        d2[k] = __shfl_sync(FULL, dth[k], lb + 2);
    }
    const int f0 = __shfl_sync(FULL, f, lb), f1 = __shfl_sync(FULL, f, lb + 1), f2 = __shfl_sync(FULL, f, lb + 2);
    real gx = 0, gy = 0, gz = 0;
    if (live && q != (real)0) {
        const real t0j = sub == 0 ? t0[0] : (sub == 1 ? t0[1] : (sub == 2 ? t0[2] : t0[3]));
        const real d0j = sub == 0 ? d0[0] : (sub == 1 ? d0[1] : (sub == 2 ? d0[2] : d0[3]));
        const int k0 = wrapk(f0 - sub, p.K[0]);
#pragma unroll
        for (int j1 = 0; j1 < 4; ++j1) {
            const int k1 = wrapk(f1 - j1, p.K[1]);
            const int row = (k0 * p.K[1] + k1) * p.K[2];
            real sx = 0, sz = 0;
#pragma unroll
            for (int j2 = 0; j2 < 4; ++j2) {
                const int k2 = wrapk(f2 - j2, p.K[2]);
                const R2<real> w = p.Z[row + k2];
                const real phi = u ? w.y : w.x;
                sx += t2[j2] * phi;
                sz += d2[j2] * phi;
            }
            gx += d0j * t1[j1] * sx;
            gy += t0j * d1[j1] * sx;
            gz += t0j * t1[j1] * sz;
        }
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        gx += __shfl_xor_sync(FULL, gx, o);
        gy += __shfl_xor_sync(FULL, gy, o);
        gz += __shfl_xor_sync(FULL, gz, o);
    }
    if (sub == 0 && live && q != (real)0) {
        const real fx = -q * p.kscale[0] * gx, fy = -q * p.kscale[1] * gy, fz = -q * p.kscale[2] * gz;
        atomic_add_ll(&s.Fa[a], to_fixed(fx, FSCALE));
        atomic_add_ll(&s.Fa[s.n + a], to_fixed(fy, FSCALE));
        atomic_add_ll(&s.Fa[2 * s.n + a], to_fixed(fz, FSCALE));
    }
}

template <typename real>
void launch_spread(const SysView<real>& s, const PmeView<real>& p, cudaStream_t st)
{
    k_spread<real><<<(4 * s.n + 127) / 128, 128, 0, st>>>(s, p);
}
template <typename real>
void launch_conv(const PmeView<real>& p, long long* E, const LamState* lam, int mode, cudaStream_t st)
{
    const int b = (p.KK + 255) / 256;
    if (mode == CONV_ENERGY) k_conv<real, CONV_ENERGY><<<b, 256, 0, st>>>(p, E, lam);
    else if (mode == CONV_POTENTIAL) k_conv<real, CONV_POTENTIAL><<<b, 256, 0, st>>>(p, E, lam);
    else k_conv<real, CONV_BOTH><<<b, 256, 0, st>>>(p, E, lam);
}
template <typename real>
void launch_gather(const SysView<real>& s, const PmeView<real>& p, cudaStream_t st)
{
    k_gather<real><<<(4 * s.n + 127) / 128, 128, 0, st>>>(s, p);
}

// energy64 (FP32 systems): the energy branch in df64 (about 48 bits).  The
// first FP32 pass leaves an FP64 copy of the packed charge grid, which
// energy64's first pass reads (Zin64); the branch transforms it and forms the
// three class energies, while the FP32 branch only forms the force
// potentials.
template <typename real>
void launch_pme(const SysView<real>& s, const PmeView<real>& p, const PmeView<df64>* energy64, cudaStream_t st)
{
    if (p.planes) {
        launch_spread(s, p, st);
        launch_planes(p, PLANE_FWD_FIX, st);
        if (energy64) {
            launch_fft(*energy64, 2, +1, 0, st);
            launch_fft(*energy64, 1, +1, 0, st);
            launch_columns(*energy64, s.E, s.lam, CONV_ENERGY, st);
        }
        launch_columns(p, s.E, s.lam, energy64 ? CONV_POTENTIAL : CONV_BOTH, st);
        launch_planes(p, PLANE_INV, st);
        launch_gather(s, p, st);
        return;
    }
    launch_spread(s, p, st);
    launch_fft(p, 2, +1, 1, st);
    if (energy64) {
        launch_fft(*energy64, 2, +1, 0, st);
        launch_fft(*energy64, 1, +1, 0, st);
        launch_fft(*energy64, 0, +1, 0, st);
        launch_conv(*energy64, s.E, s.lam, CONV_ENERGY, st);
    }
    launch_fft(p, 1, +1, 0, st);
    launch_fft(p, 0, +1, 0, st);
    launch_conv(p, s.E, s.lam, energy64 ? CONV_POTENTIAL : CONV_BOTH, st);
    launch_fft(p, 0, -1, 0, st);
    launch_fft(p, 1, -1, 0, st);
    launch_fft(p, 2, -1, 0, st);
    launch_gather(s, p, st);
}

#define LFE_INST_PME(real)                                                                        \
    template void launch_pme<real>(const SysView<real>&, const PmeView<real>&, const PmeView<df64>*, cudaStream_t); \
    template void launch_spread<real>(const SysView<real>&, const PmeView<real>&, cudaStream_t);   \
    template void launch_conv<real>(const PmeView<real>&, long long*, const LamState*, int, cudaStream_t); \
    template void launch_gather<real>(const SysView<real>&, const PmeView<real>&, cudaStream_t);   \
    template void launch_fft<real>(const PmeView<real>&, int, int, int, cudaStream_t);                       \
    template size_t fft_smem<real>(int);                                                                    \
    template void launch_planes<real>(const PmeView<real>&, int, cudaStream_t);                             \
    template void launch_columns<real>(const PmeView<real>&, long long*, const LamState*, int, cudaStream_t); \
    template size_t planes_smem<real>(const PmeView<real>&);                                                \
    template size_t columns_smem<real>(const PmeView<real>&);                                               \
    template void planes_setup<real>(const PmeView<real>&);
LFE_INST_PME(float)
LFE_INST_PME(double)
// the df64 energy branch: transforms, column / convolution energy passes
template void launch_fft<df64>(const PmeView<df64>&, int, int, int, cudaStream_t);
template size_t fft_smem<df64>(int);
template void launch_columns<df64>(const PmeView<df64>&, long long*, const LamState*, int, cudaStream_t);
template size_t columns_smem<df64>(const PmeView<df64>&);
template size_t planes_smem<df64>(const PmeView<df64>&);
template void launch_conv<df64>(const PmeView<df64>&, long long*, const LamState*, int, cudaStream_t);
template void energy_columns_setup<df64>(const PmeView<df64>&);

}  // namespace lfe
