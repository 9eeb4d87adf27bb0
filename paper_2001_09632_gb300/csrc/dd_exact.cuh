// Exact DD decisions (Alg. 2: a coefficient counts when |c| exceeds T,
// strictly), shared by the DD pilot kernels.  Include after the
// translation unit's DCT tables (Dc<B>, Dd<B>).
#pragma once
#include "abcs_common.cuh"

namespace abcs {

template <int B>
ABCS_D int rational_sign(int u, int n) {
    if (u == 0) return 1;
    return (((n + 1) >> 1) & 1) ? -1 : 1;    // sign of cos(pi (2n+1) / 4)
}

// Exact decision |c(u,v)| > T for one block, re-reading its pixels.
template <int B>
ABCS_D bool dd_exceeds_exact(const uint8_t* blk, int64_t pitch, int u, int v, int T,
                             uint32_t* status) {
    constexpr int H2 = B / 2;
    if ((u == 0 || u == H2) && (v == 0 || v == H2)) {
        long long S = 0;
        for (int n = 0; n < B; ++n)
            for (int m = 0; m < B; ++m)
                S += rational_sign<B>(u, n) * rational_sign<B>(v, m) * (int)__ldg(blk + n * pitch + m);
        return llabs(S) > (long long)T * B;
    }
    double c = 0.0;
    for (int n = 0; n < B; ++n) {
        double row = 0.0;
        for (int m = 0; m < B; ++m) row = fma((double)__ldg(blk + n * pitch + m), Dd<B>(v, m), row);
        c = fma(Dd<B>(u, n), row, c);
    }
    const double d = fabs(c) - (double)T;
    if (fabs(d) <= 1e-9) {
        set_status(status, ABCS_DEV_AMBIGUOUS);
        return false;
    }
    return d > 0.0;
}

}  // namespace abcs
