// pme_dev.cuh -- B-spline and grid-coordinate helpers shared by the PME
// kernels and the parameter-gradient kernel (Essmann et al. 1995, order 4).
#pragma once
#include "lfe_dev.cuh"

namespace lfe {

__device__ __forceinline__ float floor_p(float x) { return floorf(x); }
__device__ __forceinline__ double floor_p(double x) { return floor(x); }

// order-4 B-spline weights M4(w + j), j = 0..3, for the grid points f - j
// (closed form of the cardinal B-spline on its four unit intervals), and
// their derivatives with respect to w
template <typename real>
__device__ __forceinline__ void bspline4(real w, real th[4], real dth[4])
{
    const real w2 = w * w, w3 = w2 * w, o = (real)1 - w;
    const real s = (real)1 / (real)6;
    th[0] = s * w3;
    th[1] = s * ((real)-3 * w3 + (real)3 * w2 + (real)3 * w + (real)1);
    th[2] = s * ((real)3 * w3 - (real)6 * w2 + (real)4);
    th[3] = s * o * o * o;
    dth[0] = (real)0.5 * w2;
    dth[1] = (real)0.5 * ((real)-3 * w2 + (real)2 * w + (real)1);
    dth[2] = (real)0.5 * ((real)3 * w2 - (real)4 * w);
    dth[3] = (real)-0.5 * o * o;
}

// fractional grid coordinate: integer base f in [0, K) and offset w in
// [0, 1); the product x K/L is formed in double.  Any input (also a
// coordinate far outside the box, or NaN) yields an in-range base, so a
// diverging trajectory can never index outside the grid.
template <typename real, typename wreal>
__device__ __forceinline__ void grid_coord(real x, double ks, int K, int& f, wreal& w)
{
    double u = (double)x * ks;
    // wrapped into [0, K) by whole periods; the division is skipped for the
    // usual coordinate already inside (the result is the same)
    if (!(u >= 0.0 && u < (double)K)) u -= (double)K * floor(u / (double)K);
    if (!(u >= 0.0 && u < (double)K)) u = 0.0;
    const double fl = floor(u);
    f = min(max((int)fl, 0), K - 1);
    w = (wreal)(u - fl);
}

__device__ __forceinline__ int wrapk(int k, int K) { return k < 0 ? k + K : (k >= K ? k - K : k); }

}  // namespace lfe
