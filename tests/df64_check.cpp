// Host build of the df64 (float-pair) arithmetic of the CUDA path, for
// tests/test_df64_host.py: the same algorithms with correctly rounded host
// float operations.
#include "df64.cuh"

extern "C" void df64_ops(double a, double b, double* out)
{
    const lfe::df64 x(a), y(b);
    const lfe::df64 r[4] = {x + y, x - y, x * y, x / y};
    for (int k = 0; k < 4; ++k) {
        out[2 * k] = r[k].hi;
        out[2 * k + 1] = r[k].lo;
    }
    out[8] = x.hi;
    out[9] = x.lo;
    out[10] = y.hi;
    out[11] = y.lo;
}
