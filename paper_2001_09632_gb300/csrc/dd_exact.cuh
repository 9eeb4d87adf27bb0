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

// Exact decision |c(u,v)| > T for one block, by the whole warp (every lane
// returns it): lane l takes pixels l, l + 32, ... of the block, re-read from
// global memory.  At (u, v) in {0, B/2}^2 the coefficient is S / B with an
// integer S, summed exactly; elsewhere in FP64 (error < 1e-11 here), and an
// irrational coefficient within 1e-9 of T is flagged ABCS_DEV_AMBIGUOUS and
// counted as not exceeding.
template <int B>
ABCS_D bool dd_exact_warp(const uint8_t* blk, int64_t pitch, int u, int v, int T, uint32_t* status) {
    constexpr int H2 = B / 2;
    const int lane = threadIdx.x & 31;
    if ((u == 0 || u == H2) && (v == 0 || v == H2)) {
        long long S = 0;
        for (int i = lane; i < B * B; i += 32) {
            const int n = i / B, m = i % B;
            S += rational_sign<B>(u, n) * rational_sign<B>(v, m) * (int)__ldg(blk + n * pitch + m);
        }
        S = warp_sum(S);
        return llabs(S) > (long long)T * B;
    }
    double c = 0.0;
    for (int i = lane; i < B * B; i += 32) {
        const int n = i / B, m = i % B;
        c = fma(Dd<B>(u, n) * Dd<B>(v, m), (double)__ldg(blk + n * pitch + m), c);
    }
    c = __shfl_sync(0xffffffffu, warp_sum(c), 0);
    const double d = fabs(c) - (double)T;
    if (fabs(d) <= 1e-9) {
        if (lane == 0) set_status(status, ABCS_DEV_AMBIGUOUS);
        return false;
    }
    return d > 0.0;
}

}  // namespace abcs
