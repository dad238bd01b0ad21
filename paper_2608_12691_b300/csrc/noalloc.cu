// noalloc.cu -- reciprocal-space (smooth PME) evaluation that allocates no
// device memory.
//
// Some callers cannot let a library call cudaMalloc: processes whose device
// memory is owned by a pool or an allocator that forbids hidden allocations,
// long-running services that must not grow their memory after start-up, and
// code running where allocation calls are not permitted.  For them,
// lfe_pme_noalloc keeps every intermediate grid and table in one file-scope
// __device__ array of fixed size, which every GPU that loads this library
// holds until the process exits.  The caller still provides the inputs and
// the outputs in device memory; a call issues only kernel launches and
// memsets on the caller's stream.
//
// The arithmetic is the one of the system path: order-4 B-spline spreading
// into fixed-point class grids, the packed FP32 transform for the forces and
// the FP64 transform for the class energies, the same influence function and
// class split (U_vv, U_uu, U_uv and the h_A-weighted class potentials).
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "lfe.h"
#include "lfe_views.cuh"
#include "pme_dev.cuh"

namespace lfe {

namespace {

constexpr int NA_MAX_K = 128;

struct NaScratch {
    long long Qfix[2 * LFE_NOALLOC_MAX_GRID];   // solvent / solute fixed-point charge grids
    R2<float> Z[LFE_NOALLOC_MAX_GRID];          // packed FP32 transform
    R2<double> Z64[LFE_NOALLOC_MAX_GRID];       // packed FP64 transform (energies)
    long long E[E_N];                           // fixed-point energy accumulators
    double qsum[4];                             // sum q^2 (v, u), sum q (v, u)
    LamState lam;
    float gfac[3][NA_MAX_K], msq[3][NA_MAX_K];
    R2<float> tw[3][NA_MAX_K];
    double gfac64[3][NA_MAX_K], msq64[3][NA_MAX_K];
    R2<double> tw64[3][NA_MAX_K];
};

// the scratch array: shared by every call on a device, it keeps the last
// call's contents; every call clears what must start at zero
__device__ __align__(256) NaScratch g_na_scratch;

std::mutex g_na_mutex;
NaScratch* g_na_addr[256] = {};   // device address of g_na_scratch, per device


bool radix_plan_na(int K, int* rad, int* nrad)
{
    int n = 0, k = K;
    while (k % 4 == 0 && n < 8) { rad[n++] = 4; k /= 4; }
    while (k % 2 == 0 && n < 8) { rad[n++] = 2; k /= 2; }
    while (k % 3 == 0 && n < 8) { rad[n++] = 3; k /= 3; }
    while (k % 5 == 0 && n < 8) { rad[n++] = 5; k /= 5; }
    *nrad = n;
    return k == 1;
}

// charge sums per class (solvent 0, solute 1) for the self and background terms
__global__ void k_na_sums(int n, const double* q, const unsigned char* sol, NaScratch* sc)
{
    double s2[2] = {0, 0}, s1[2] = {0, 0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int c = sol[i] ? 1 : 0;
        s2[c] += q[i] * q[i];
        s1[c] += q[i];
    }
    __shared__ double red[4][32];
    double v[4] = {s2[0], s2[1], s1[0], s1[1]};
    for (int k = 0; k < 4; ++k) {
        double x = warp_sum_d(v[k]);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        sc->qsum[threadIdx.x] = t;
    }
}

// influence-function factors exp(-pi^2 m^2 / alpha^2) |b(m)|^2 with the
// order-4 B-spline moduli, squared reciprocal vectors m^2 (m = k / L for
// k <= K/2, (k - K) / L above) and twiddles exp(2 pi i k / K) of every axis,
// in FP64 and (rounded) FP32: one thread per (axis, k)
struct NaBox {
    double L[3];
    int K[3];
    double alpha;
};

__global__ void k_na_tables(NaBox b, NaScratch* sc)
{
    const int d = blockIdx.x;
    const int K = b.K[d];
    for (int m = threadIdx.x; m < K; m += blockDim.x) {
        // |b(m)|^-2 = |sum_{k=0..2} M4(k+1) e^{2 pi i m k / K}|^2, M4(1..3) = 1/6, 2/3, 1/6
        const double c1 = cospi(2.0 * m / K), s1 = sinpi(2.0 * m / K);
        const double c2 = cospi(4.0 * m / K), s2 = sinpi(4.0 * m / K);
        const double re = 1.0 / 6.0 + (2.0 / 3.0) * c1 + (1.0 / 6.0) * c2;
        const double im = (2.0 / 3.0) * s1 + (1.0 / 6.0) * s2;
        const double b2 = 1.0 / (re * re + im * im);
        const int mm = (m <= K / 2) ? m : m - K;
        const double mr = mm / b.L[d];
        const double gf = exp(-PI * PI * mr * mr / (b.alpha * b.alpha)) * b2;
        sc->gfac64[d][m] = gf;
        sc->msq64[d][m] = mr * mr;
        sc->tw64[d][m] = R2<double>{c1, s1};
        sc->gfac[d][m] = (float)gf;
        sc->msq[d][m] = (float)(mr * mr);
        sc->tw[d][m] = R2<float>{(float)c1, (float)s1};
    }
}

struct NaGeom {
    int n;
    int KK;
    int K[3];
    double L[3];
};

__global__ void k_na_spread(NaGeom g, const double* pos, const double* q, const unsigned char* sol, NaScratch* sc)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= g.n) return;
    const double qa = q[a];
    if (qa == 0.0) return;
    long long* grid = sc->Qfix + (sol[a] ? g.KK : 0);   // the transform reads the solute grid at KK
    int f[3];
    double th[3][4], dth[4];
    for (int d = 0; d < 3; ++d) {
        double w;
        grid_coord<double, double>(pos[3 * a + d], g.K[d] / g.L[d], g.K[d], f[d], w);
        bspline4<double>(w, th[d], dth);
    }
    for (int j0 = 0; j0 < 4; ++j0) {
        const int k0 = wrapk(f[0] - j0, g.K[0]);
        for (int j1 = 0; j1 < 4; ++j1) {
            const int k1 = wrapk(f[1] - j1, g.K[1]);
            const double a1 = qa * th[0][j0] * th[1][j1];
            const int row = (k0 * g.K[1] + k1) * g.K[2];
            for (int j2 = 0; j2 < 4; ++j2) {
                const int k2 = wrapk(f[2] - j2, g.K[2]);
                atomic_add_ll(&grid[row + k2], __double2ll_rn(a1 * th[2][j2] * QSCALE));
            }
        }
    }
}

// force of each atom from the packed potential grid (solvent: real part,
// solute: imaginary part); one thread owns one atom, so it writes directly
__global__ void k_na_gather(NaGeom g, const double* pos, const double* q, const unsigned char* sol,
                            const NaScratch* sc, double* forces)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= g.n) return;
    const double qa = q[a];
    const bool u = sol[a] != 0;
    int f[3];
    double th[3][4], dth[3][4];
    for (int d = 0; d < 3; ++d) {
        double w;
        grid_coord<double, double>(pos[3 * a + d], g.K[d] / g.L[d], g.K[d], f[d], w);
        bspline4<double>(w, th[d], dth[d]);
    }
    double gx = 0, gy = 0, gz = 0;
    for (int j0 = 0; j0 < 4; ++j0) {
        const int k0 = wrapk(f[0] - j0, g.K[0]);
        for (int j1 = 0; j1 < 4; ++j1) {
            const int k1 = wrapk(f[1] - j1, g.K[1]);
            const int row = (k0 * g.K[1] + k1) * g.K[2];
            double sx = 0, sz = 0;
            for (int j2 = 0; j2 < 4; ++j2) {
                const int k2 = wrapk(f[2] - j2, g.K[2]);
                const R2<float> w = sc->Z[row + k2];
                const double phi = u ? (double)w.y : (double)w.x;
                sx += th[2][j2] * phi;
                sz += dth[2][j2] * phi;
            }
            gx += dth[0][j0] * th[1][j1] * sx;
            gy += th[0][j0] * dth[1][j1] * sx;
            gz += th[0][j0] * th[1][j1] * sz;
        }
    }
    forces[3 * a] = -qa * (g.K[0] / g.L[0]) * gx;
    forces[3 * a + 1] = -qa * (g.K[1] / g.L[1]) * gy;
    forces[3 * a + 2] = -qa * (g.K[2] / g.L[2]) * gz;
}

// class energies = reciprocal (FP64 transform) + self + neutralising background
__global__ void k_na_finalize(NaScratch* sc, double alpha, double V, double* energies)
{
    const double self_c = -KE * alpha / sqrt(PI);
    const double pre = -KE * PI / (2.0 * V * alpha * alpha);
    const double qv = sc->qsum[2], qu = sc->qsum[3];
    energies[0] = (double)sc->E[E_REC_VV] * (1.0 / ESCALE) + self_c * sc->qsum[0] + pre * qv * qv;
    energies[1] = (double)sc->E[E_REC_UU] * (1.0 / ESCALE) + self_c * sc->qsum[1] + pre * qu * qu;
    energies[2] = (double)sc->E[E_REC_UV] * (1.0 / ESCALE) + pre * 2.0 * qv * qu;
}

int na_fail(int code, const std::string& m)
{
    record_global_error(m);
    return code;
}

}  // namespace

}  // namespace lfe

using namespace lfe;

extern "C" int lfe_pme_noalloc(int n, const double* pos, const double* charge, const unsigned char* solute,
                               const double* box, double alpha, const int* grid, double lambda, double* forces,
                               double* energies, void* stream)
{
    if (n <= 0 || !pos || !charge || !solute || !box || !grid || !forces || !energies)
        return na_fail(LFE_ERR_ARG, "lfe_pme_noalloc: n must be positive and no pointer may be NULL");
    if (!(alpha > 0) || !std::isfinite(alpha)) return na_fail(LFE_ERR_ARG, "lfe_pme_noalloc: alpha must be > 0");
    if (!(lambda >= 0.0 && lambda <= 1.0)) return na_fail(LFE_ERR_ARG, "lfe_pme_noalloc: lambda must be in [0, 1]");
    long long KK = 1;
    int rad[3][8], nrad[3];
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0) || !std::isfinite(box[d]))
            return na_fail(LFE_ERR_ARG, "lfe_pme_noalloc: box lengths must be positive");
        if (grid[d] < 8 || grid[d] > NA_MAX_K || !radix_plan_na(grid[d], rad[d], &nrad[d]))
            return na_fail(LFE_ERR_ARG, "lfe_pme_noalloc: grid entries must be in [8, 128] and factor into 2, 3, 5");
        KK *= grid[d];
    }
    if (KK > LFE_NOALLOC_MAX_GRID)
        return na_fail(LFE_ERR_ARG, "lfe_pme_noalloc: grid has " + std::to_string(KK) +
                                        " points, more than the fixed scratch holds (LFE_NOALLOC_MAX_GRID = " +
                                        std::to_string(LFE_NOALLOC_MAX_GRID) + ")");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
        return na_fail(LFE_ERR_CUDA, "lfe_pme_noalloc: no usable current device");
    NaScratch* sc = nullptr;
    {
        // first call on a device: look up the device address of the scratch
        // array (host code may not take the address of a __device__ variable)
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(LFE_ERR_CUDA, std::string("lfe_pme_noalloc: cudaGetSymbolAddress failed: ") +
                                                 cudaGetErrorString(e));
            g_na_addr[dev] = static_cast<NaScratch*>(p);
        }
        sc = g_na_addr[dev];
    }
    // influence-function factors and twiddles for this box and grid, formed
    // on the device from arguments passed by value
    NaScratch* dsc = sc;
    const double V = box[0] * box[1] * box[2];
    NaBox nb{};
    for (int d = 0; d < 3; ++d) {
        nb.L[d] = box[d];
        nb.K[d] = grid[d];
    }
    nb.alpha = alpha;
    k_na_tables<<<3, NA_MAX_K, 0, st>>>(nb, dsc);
    cudaError_t e = cudaMemsetAsync(dsc->Qfix, 0, sizeof(long long) * 2 * LFE_NOALLOC_MAX_GRID, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsc->E, 0, sizeof(long long) * E_N, st);
    if (e != cudaSuccess) return na_fail(LFE_ERR_CUDA, std::string("lfe_pme_noalloc: ") + cudaGetErrorString(e));

    // h_A(lambda) through the same device routine as the system path
    SysView<float> sv{};
    sv.lam = &dsc->lam;
    launch_set_lambda(sv, lambda, st);

    PmeView<float> M{};
    PmeView<double> M64{};
    M.KK = (int)KK;
    M64.KK = (int)KK;
    for (int d = 0; d < 3; ++d) {
        M.K[d] = M64.K[d] = grid[d];
        M.kscale[d] = (float)(grid[d] / box[d]);
        M64.kscale[d] = grid[d] / box[d];
        M.kscale64[d] = M64.kscale64[d] = grid[d] / box[d];
        M.nrad[d] = M64.nrad[d] = nrad[d];
        for (int r = 0; r < 8; ++r) M.rad[d][r] = M64.rad[d][r] = rad[d][r];
        M.gfac[d] = dsc->gfac[d];
        M.msq[d] = dsc->msq[d];
        M.tw[d] = dsc->tw[d];
        M64.gfac[d] = dsc->gfac64[d];
        M64.msq[d] = dsc->msq64[d];
        M64.tw[d] = dsc->tw64[d];
    }
    M.conv_pre = (float)(KE / (PI * V));
    M64.conv_pre = KE / (PI * V);
    M.qu_scale = 1.0f;
    M64.qu_scale = 1.0;
    M.Qfix = dsc->Qfix;
    M.Z = dsc->Z;
    M.Zraw64 = dsc->Z64;
    M64.Z = dsc->Z64;
    NaGeom g{};
    g.n = n;
    g.KK = (int)KK;
    for (int d = 0; d < 3; ++d) {
        g.K[d] = grid[d];
        g.L[d] = box[d];
    }
    const int B = 128;
    k_na_sums<<<1, 256, 0, st>>>(n, charge, solute, dsc);
    k_na_spread<<<(n + B - 1) / B, B, 0, st>>>(g, pos, charge, solute, dsc);
    launch_fft(M, 2, +1, 1, st);
    launch_fft(M64, 2, +1, 0, st);
    launch_fft(M64, 1, +1, 0, st);
    launch_fft(M64, 0, +1, 0, st);
    launch_conv(M64, dsc->E, &dsc->lam, CONV_ENERGY, st);
    launch_fft(M, 1, +1, 0, st);
    launch_fft(M, 0, +1, 0, st);
    launch_conv(M, dsc->E, &dsc->lam, CONV_POTENTIAL, st);
    launch_fft(M, 0, -1, 0, st);
    launch_fft(M, 1, -1, 0, st);
    launch_fft(M, 2, -1, 0, st);
    k_na_gather<<<(n + B - 1) / B, B, 0, st>>>(g, pos, charge, solute, dsc, forces);
    k_na_finalize<<<1, 1, 0, st>>>(dsc, alpha, V, energies);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(LFE_ERR_CUDA, std::string("lfe_pme_noalloc: ") + cudaGetErrorString(e));
    return LFE_OK;
}
