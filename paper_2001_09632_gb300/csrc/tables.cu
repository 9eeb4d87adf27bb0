// Host-side DCT and zigzag tables, computed once in double precision.
#include <algorithm>
#include <cmath>
#include <vector>

#include "abcs_common.cuh"

namespace abcs {
namespace {

// Orthonormal DCT-II basis: D[k][n] = a_k cos(pi (2n+1) k / (2B)),
// a_0 = sqrt(1/B), a_k = sqrt(2/B) (the 2D-DCT dictionary of Sec. IV).
template <int B>
void fill_dct(float* f, double* d) {
    const double pi = std::acos(-1.0);
    for (int k = 0; k < B; ++k)
        for (int n = 0; n < B; ++n) {
            const double a = std::sqrt((k == 0 ? 1.0 : 2.0) / B);
            const double v = a * std::cos(pi * (2 * n + 1) * k / (2.0 * B));
            d[k * B + n] = v;
            f[k * B + n] = (float)v;
        }
}

// JPEG zigzag scan (ref. [26] of the paper) for a B x B block: positions
// sorted by anti-diagonal s = u + v, then along the diagonal by u ascending
// on odd s and u descending on even s.
template <int B>
void fill_zz(uint16_t* pos) {
    std::vector<int> idx(B * B);
    for (int i = 0; i < B * B; ++i) idx[i] = i;
    auto key = [](int p) {
        const int u = p / B, v = p % B, s = u + v;
        return std::make_pair(s, (s & 1) ? u : -u);
    };
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return key(a) < key(b); });
    for (int r = 0; r < B * B; ++r) pos[r] = (uint16_t)idx[r];
}

HostTables make() {
    HostTables t;
    fill_dct<4>(t.Df4, t.Dd4);
    fill_dct<8>(t.Df8, t.Dd8);
    fill_dct<16>(t.Df16, t.Dd16);
    fill_dct<32>(t.Df32, t.Dd32);
    fill_zz<4>(t.zzpos4);
    fill_zz<8>(t.zzpos8);
    fill_zz<16>(t.zzpos16);
    fill_zz<32>(t.zzpos32);
    return t;
}

}  // namespace

const HostTables& host_tables() {
    static const HostTables t = make();
    return t;
}

}  // namespace abcs
