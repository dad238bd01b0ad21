// lfe_dev.cuh -- device-side types and helpers shared by the CUDA kernels.
//
// Every kernel is a template over `real` (float for LFE_FP32_MIXED, double
// for LFE_FP64).  Forces, energies and PME charge grids are accumulated in
// 64-bit fixed point so that sums are exact and independent of the order in
// which atomics land (results are bit-reproducible run to run).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lfe {

constexpr double KE = 138.935458;              // kJ mol^-1 nm e^-2
constexpr double KB = 0.0083144626;            // kJ mol^-1 K^-1
constexpr double FSCALE = 4294967296.0;        // forces: 2^32 units per kJ/mol/nm
constexpr double ESCALE = 68719476736.0;       // energies: 2^36 units per kJ/mol (range +-1.3e8)
constexpr double QSCALE = 68719476736.0;       // PME charge grid: 2^36 units per e
constexpr double PI = 3.14159265358979323846;

template <typename T>
struct alignas(4 * sizeof(T)) R4 { T x, y, z, w; };
template <typename T>
struct alignas(2 * sizeof(T)) R2 { T x, y; };

// energy accumulator slots (int64 fixed point, ESCALE), E_NPAIRS is a count
enum {
    E_PAIR_VV = 0, E_PAIR_UU, E_PAIR_UV, E_PAIR_SOFT,
    E_EXCL_VV, E_EXCL_UU, E_EXCL_UV,
    E_14_VV, E_14_UU, E_14_UV,
    E_REC_VV, E_REC_UU, E_REC_UV,
    E_BONDED, E_NPAIRS, E_DAFED,
    E_DSC,          // dU_soft/dlambda of the soft-core coupling
    E_N = 17
};

// error / control flags (FL_PRUNE: the pruned pair list is due; FL_PTILES:
// its tile count; FL_NPRUNE: prunings done by steps; FL_PCHUNK, FL_PDONE: the
// FP32 pair kernel's next chunk and finished warps, zero between launches)
enum { FL_REBUILD = 0, FL_ERROR = 1, FL_NTILES = 2, FL_NREBUILD = 3, FL_NUV = 4, FL_NSTAGE = 5, FL_NUVT = 6,
       FL_PRUNE = 7, FL_PTILES = 8, FL_NPRUNE = 9, FL_PCHUNK = 10, FL_PDONE = 11, FL_N = 12 };
// ERRB_BADPOS: the positions handed to a host-I/O step were not all finite;
// the step is skipped like one after a list overflow (ERRB_SKIP)
enum { ERRB_OVERFLOW = 1, ERRB_NONFINITE = 2, ERRB_CONSTRAINT = 4, ERRB_BADPOS = 8 };
enum { ERRB_SKIP = ERRB_OVERFLOW | ERRB_BADPOS };

// one coordinate wrapped into [0, L) (the positions the neighbour list is
// built from)
__device__ __forceinline__ float floor_w(float x) { return floorf(x); }
__device__ __forceinline__ double floor_w(double x) { return floor(x); }
// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may be scheduled while its predecessor in
// the stream is still running; pdl_wait() returns once the predecessor has
// completed and its memory is visible, so every such kernel calls it before
// touching memory.  pdl_trigger() lets the dependent kernel be scheduled
// early.  Both are no-ops for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <typename real>
__device__ __forceinline__ real wrap_box(real x, real L, real invL)
{
    real w = x - L * floor_w(x * invL);
    if (w >= L) w -= L;
    if (w < (real)0) w += L;
    if (w >= L) w = (real)0;
    return w;
}

// lambda state, written on the device (by lfe_eval's setter or by the theta
// integrator) and read by every kernel that depends on lambda.
struct LamState {
    double lambda, hA, hB, dhA, dhB;
    double theta, p_theta, dlam_dtheta;
    double dUdl, U;                 // last evaluated values
    double V_std, V_exp;            // last OPES bias values
    unsigned long long step;
    double v_eta;                   // theta's thermostat velocity (regulated Nose-Hoover-Langevin)
    double npairs;                  // pairs within r_cut counted by the last step's pair kernel
    double pad;
};

// OPES state for the two biases (std = 0, exp = 1).
struct OpesState {
    int n[2];
    int pad[2];
    double wsum[2];
    double rho_bar[2];
};

template <typename real>
__device__ __forceinline__ long long to_fixed(real v, double scale)
{
    return __double2ll_rn((double)v * scale);
}
template <>
__device__ __forceinline__ long long to_fixed<float>(float v, double scale)
{
    return __float2ll_rn(v * (float)scale);
}

__device__ __forceinline__ void atomic_add_ll(long long* p, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// h_A, h_B and their lambda-derivatives (Eq. 7-10), FP64.
__host__ __device__ __forceinline__ void switching_fns(double lam, double& hA, double& hB, double& dA, double& dB)
{
    constexpr double INV_W = 1.0 / 0.65;   // S32 runs over lambda in [0.35, 1]: no division at run time
    double x = (lam - 0.35) * INV_W;
    double s32 = 0.0, d32 = 0.0;
    if (x >= 1.0) { s32 = 1.0; }
    else if (x > 0.0) {
        double x2 = x * x, x3 = x2 * x, x4 = x2 * x2;
        s32 = x4 * (15.0 - 24.0 * x + 10.0 * x2);
        d32 = 60.0 * x3 * (1.0 - x) * (1.0 - x);
    }
    double s22 = 0.0, d22 = 0.0;
    if (lam >= 1.0) { s22 = 1.0; }
    else if (lam > 0.0) {
        double l2 = lam * lam, l3 = l2 * lam;
        s22 = l3 * (10.0 - 15.0 * lam + 6.0 * l2);
        d22 = 30.0 * l2 * (1.0 - lam) * (1.0 - lam);
    }
    hA = s32;
    hB = s22 - s32;
    dA = d32 * INV_W;
    dB = d22 - d32 * INV_W;
}

// ---------------------------------------------------------- Philox4x32-10
// Counter-based RNG of Salmon et al. (SC 2011).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned int hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned int hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// three standard normals from one Philox call: Box-Muller on (u0,u1), (u2,u3)
template <typename real>
__device__ __forceinline__ void normals3(uint4 c, uint2 k, real& n0, real& n1, real& n2)
{
    uint4 r = philox4x32_10(c, k);
    const double s = 1.0 / 4294967296.0;
    double u0 = (r.x + 0.5) * s, u1 = (r.y + 0.5) * s, u2 = (r.z + 0.5) * s, u3 = (r.w + 0.5) * s;
    double a = sqrt(-2.0 * log(u0)), b = sqrt(-2.0 * log(u2));
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    n0 = (real)(a * cs);
    n1 = (real)(a * sn);
    n2 = (real)(b * cospi(2.0 * u3));
}
// FP32 variant for the mixed-precision path (B300 FP64 throughput is low)
template <>
__device__ __forceinline__ void normals3<float>(uint4 c, uint2 k, float& n0, float& n1, float& n2)
{
    uint4 r = philox4x32_10(c, k);
    const float s = 2.3283064365386963e-10f;  // 2^-32
    float u0 = (r.x + 0.5f) * s, u1 = (r.y + 0.5f) * s, u2 = (r.z + 0.5f) * s, u3 = (r.w + 0.5f) * s;
    // (x + 0.5) rounds to 2^32 for x near 2^32 - 1: keep u strictly below 1
    u0 = fminf(u0, 0.99999994f);
    u2 = fminf(u2, 0.99999994f);
    float a = sqrtf(-2.0f * logf(u0)), b = sqrtf(-2.0f * logf(u2));
    float sn, cs;
    sincospif(2.0f * u1, &sn, &cs);
    n0 = a * cs;
    n1 = a * sn;
    n2 = b * cospif(2.0f * u3);
}

}  // namespace lfe
