// BM3D, hard-thresholding step (ref. [22]): the plain denoiser the paper
// pairs with IDA besides DnCNN (Sec. VII).  One CTA per reference patch
// (8 x 8, every third position plus the last row / column):
//   - the 46 x 46 neighbourhood (reference +- 19 positions) in shared memory;
//   - distances d = ||P_ref - P||^2 / 64 of every candidate position;
//   - the group: the reference, then the candidates with d <= tau ordered by
//     (d, row, column), n = the largest power of two <= min(16, count),
//     chosen by repeated block-wide minimum of 64-bit keys (d's bits, index)
//     held in registers (a thread owns a strip of 8 candidates of one row,
//     whose distances share each loaded row segment);
//   - 2D DCT of each patch, orthonormal Haar along the group, hard threshold
//     at lambda sigma (the group's 3D DC kept), count, inverses;
//   - aggregation of w K P (w = 1 / kept, K the 8 x 8 Kaiser window) and of
//     w K into numerator / denominator planes (atomic adds).
// A second kernel divides.  tau = 2500 for sigma <= 40, else 5000.
#include <cmath>

#include "abcs_common.cuh"

namespace abcs {

namespace {

constexpr int kN1 = 8, kN2 = 16, kHalf = 19, kStep = 3, kStrip = 8;
constexpr int kWin = 2 * kHalf + kN1;          // 46: neighbourhood side
constexpr int kWinLd = kWin + 1;
constexpr int kBm3dThreads = 256;

__constant__ float c_bm_dct[8][8];      // D[k][n], orthonormal DCT-II
__constant__ float c_bm_kaiser[8];

ABCS_D unsigned long long bm_min(unsigned long long a, unsigned long long b) { return a < b ? a : b; }

// Orthonormal Haar of length N by butterflies, H_2n = [H_n (x) (1, 1); I_n (x) (1, -1)] / sqrt 2:
// the pairwise sums recurse, the pairwise differences are the last n outputs.
template <int N>
ABCS_D void haar_fwd(float (&x)[16]) {
    if constexpr (N > 1) {
        float s[N / 2], d[N / 2];
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            s[i] = (x[2 * i] + x[2 * i + 1]) * 0.70710678118654752f;
            d[i] = (x[2 * i] - x[2 * i + 1]) * 0.70710678118654752f;
        }
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            x[i] = s[i];
            x[N / 2 + i] = d[i];
        }
        haar_fwd<N / 2>(x);
    }
}

template <int N>
ABCS_D void haar_inv(float (&x)[16]) {
    if constexpr (N > 1) {
        haar_inv<N / 2>(x);
        float y[N];
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            y[2 * i] = (x[i] + x[N / 2 + i]) * 0.70710678118654752f;
            y[2 * i + 1] = (x[i] - x[N / 2 + i]) * 0.70710678118654752f;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = y[i];
    }
}

// coefficient (u, v) of the group's N patches: Haar, zero |c| <= thr (the
// 3D DC kept when dc), inverse into T; returns the coefficients kept
template <int N>
ABCS_D int haar_threshold(const float (&P)[kN2][kN1][kN1 + 1], float (&T)[kN2][kN1][kN1 + 1], int u, int v,
                          float thr, bool dc) {
    float z[16];
#pragma unroll
    for (int g = 0; g < N; ++g) z[g] = P[g][u][v];
    haar_fwd<N>(z);
    int kept = 0;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        const bool keep = fabsf(z[q]) > thr || (q == 0 && dc);
        z[q] = keep ? z[q] : 0.f;
        kept += keep;
    }
    haar_inv<N>(z);
#pragma unroll
    for (int g = 0; g < N; ++g) T[g][u][v] = z[g];
    return kept;
}

// reference position j of a dimension of n pixels: 3 j, the last one n - 8
ABCS_D int bm_ref_pos(int j, int n) { return min(kStep * j, n - kN1); }

__global__ void __launch_bounds__(kBm3dThreads, 4) bm3d_ht_kernel(const float* __restrict__ in, int H, int W,
                                                               const float* __restrict__ sigma, float lam,
                                                               float* __restrict__ num, float* __restrict__ den) {
    __shared__ float nb[kWin * kWinLd];
    __shared__ unsigned long long red[2][kBm3dThreads / 32];
    __shared__ unsigned long long wtop[kBm3dThreads / 32 * kN2];
    __shared__ int sel[kN2];
    __shared__ float P[kN2][kN1][kN1 + 1];
    __shared__ float T[kN2][kN1][kN1 + 1];
    __shared__ int s_cnt;
    griddep_wait();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, k = blockIdx.z;
    const int y = bm_ref_pos(blockIdx.y, H), x = bm_ref_pos(blockIdx.x, W);
    const float* img = in + (int64_t)k * H * W;
    const float s = __ldg(sigma + k);
    const float tau = s <= 40.f ? 2500.f : 5000.f, thr = lam * s;
    // candidate top-left corners [cy0, cy1] x [cx0, cx1]; neighbourhood rows cy0 .. cy1 + 7
    const int cy0 = max(0, y - kHalf), cy1 = min(H - kN1, y + kHalf);
    const int cx0 = max(0, x - kHalf), cx1 = min(W - kN1, x + kHalf);
    const int ncy = cy1 - cy0 + 1, ncx = cx1 - cx0 + 1, nh = ncy + kN1 - 1, nw = ncx + kN1 - 1;
    for (int i = t; i < nh * 64; i += kBm3dThreads) {          // nw <= 46 < 64
        const int r = i >> 6, c = i & 63;
        if (c < nw) nb[r * kWinLd + c] = __ldg(img + (int64_t)(cy0 + r) * W + cx0 + c);
    }
    __syncthreads();
    const int ry = y - cy0, rx = x - cx0, ref = ry * ncx + rx;
    // thread t takes the strip of up to 8 consecutive candidates (oy, 8 sx .. 8 sx + 7):
    // one row segment of 15 pixels per patch row serves all 8 distances.
    // keys: the reference 0, others (bits of d) << 32 | (index + 1); beyond tau: max
    const int spr = (ncx + kStrip - 1) / kStrip, oy = t / spr, ox0 = (t - oy * spr) * kStrip;
    const bool mine = oy < ncy;
    unsigned long long kr[kStrip];
    {
        float acc[kStrip];
#pragma unroll
        for (int q = 0; q < kStrip; ++q) acc[q] = 0.f;
        if (mine) {
#pragma unroll
            for (int i = 0; i < kN1; ++i) {
                float row[kStrip + kN1 - 1], rf[kN1];
#pragma unroll
                for (int j = 0; j < kStrip + kN1 - 1; ++j)
                    row[j] = ox0 + j < nw ? nb[(oy + i) * kWinLd + ox0 + j] : 0.f;
#pragma unroll
                for (int j = 0; j < kN1; ++j) rf[j] = nb[(ry + i) * kWinLd + rx + j];
#pragma unroll
                for (int q = 0; q < kStrip; ++q)
#pragma unroll
                    for (int j = 0; j < kN1; ++j) {
                        const float d = rf[j] - row[q + j];
                        acc[q] = fmaf(d, d, acc[q]);
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < kStrip; ++q) {
            const int ox = ox0 + q, c = oy * ncx + ox;
            const float d = acc[q] * (1.f / 64.f);
            unsigned long long kk = ~0ull;
            if (mine && ox < ncx) {
                if (c == ref) kk = 0ull;
                else if (d <= tau) kk = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(c + 1);
            }
            kr[q] = kk;
        }
    }
    // group size: the largest power of two <= min(16, candidates within tau)
    {
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < kStrip; ++q) cnt += kr[q] != ~0ull;
        cnt = warp_sum(cnt);
        if (lane == 0) red[0][warp] = (unsigned long long)cnt;
        __syncthreads();
        if (t == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < kBm3dThreads / 32; ++w) tot += red[0][w];
            const int lim = tot < (unsigned long long)kN2 ? (int)tot : kN2;
            int n = 1;
            while (2 * n <= lim) n *= 2;
            s_cnt = n;
        }
        __syncthreads();
    }
    const int n = s_cnt;
    // the n smallest keys in order, in two levels: every warp takes the n
    // smallest of its own keys (registers, shuffles), then warp 0 the n
    // smallest of those 8 n.  Keys are distinct; the lane that owned the
    // chosen key drops it and recomputes its minimum.
    {
        unsigned long long lmin = ~0ull;
#pragma unroll
        for (int q = 0; q < kStrip; ++q) lmin = bm_min(lmin, kr[q]);
        for (int g = 0; g < n; ++g) {
            unsigned long long b = lmin;
#pragma unroll
            for (int o = 16; o; o >>= 1) b = bm_min(b, __shfl_xor_sync(0xffffffffu, b, o));
            if (b == lmin && b != ~0ull) {
                lmin = ~0ull;
#pragma unroll
                for (int q = 0; q < kStrip; ++q) {
                    if (kr[q] == b) kr[q] = ~0ull;
                    lmin = bm_min(lmin, kr[q]);
                }
            }
            if (lane == 0) wtop[warp * kN2 + g] = b;
        }
    }
    __syncthreads();
    if (warp == 0) {
        constexpr int PER = kBm3dThreads / 32 * kN2 / 32;          // 4 per lane
        unsigned long long v[PER], lmin = ~0ull;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int i = lane * PER + q, w = i / kN2, g = i % kN2;
            v[q] = g < n ? wtop[w * kN2 + g] : ~0ull;
            lmin = bm_min(lmin, v[q]);
        }
        for (int g = 0; g < n; ++g) {
            unsigned long long b = lmin;
#pragma unroll
            for (int o = 16; o; o >>= 1) b = bm_min(b, __shfl_xor_sync(0xffffffffu, b, o));
            if (b == lmin) {
                lmin = ~0ull;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    if (v[q] == b) v[q] = ~0ull;
                    lmin = bm_min(lmin, v[q]);
                }
            }
            if (lane == 0) sel[g] = b == 0ull ? ref : (int)(b & 0xFFFFFFFFull) - 1;
        }
    }
    __syncthreads();
    // patches of the group
    for (int i = t; i < n * 64; i += kBm3dThreads) {
        const int g = i >> 6, py = (i >> 3) & 7, px = i & 7, c = sel[g];
        const int oy = c / ncx, ox = c - oy * ncx;
        P[g][py][px] = nb[(oy + py) * kWinLd + ox + px];
    }
    __syncthreads();
    // 2D DCT: T = P D^T (rows), then P = D T (columns)
    for (int i = t; i < n * 64; i += kBm3dThreads) {
        const int g = i >> 6, r = (i >> 3) & 7, v = i & 7;
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) a = fmaf(P[g][r][j], c_bm_dct[v][j], a);
        T[g][r][v] = a;
    }
    __syncthreads();
    for (int i = t; i < n * 64; i += kBm3dThreads) {
        const int g = i >> 6, u = (i >> 3) & 7, v = i & 7;
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) a = fmaf(c_bm_dct[u][j], T[g][j][v], a);
        P[g][u][v] = a;
    }
    __syncthreads();
    // Haar along the group per coefficient (u, v) (butterflies in registers),
    // threshold, count, inverse Haar
    int kept = 0;
    if (t < 64) {
        const int u = t >> 3, v = t & 7;
        switch (n) {
            case 1: kept = haar_threshold<1>(P, T, u, v, thr, t == 0); break;
            case 2: kept = haar_threshold<2>(P, T, u, v, thr, t == 0); break;
            case 4: kept = haar_threshold<4>(P, T, u, v, thr, t == 0); break;
            case 8: kept = haar_threshold<8>(P, T, u, v, thr, t == 0); break;
            default: kept = haar_threshold<16>(P, T, u, v, thr, t == 0); break;
        }
    }
    kept = warp_sum(kept);
    if (lane == 0) red[0][warp] = (unsigned long long)kept;
    __syncthreads();
    const float wgt = 1.f / (float)(red[0][0] + red[0][1]);    // threads 0..63 are warps 0 and 1
    // inverse 2D DCT: P = T D (rows of D^T C), then D^T P
    for (int i = t; i < n * 64; i += kBm3dThreads) {
        const int g = i >> 6, u = (i >> 3) & 7, j = i & 7;
        float a = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) a = fmaf(T[g][u][v], c_bm_dct[v][j], a);
        P[g][u][j] = a;
    }
    __syncthreads();
    for (int i = t; i < n * 64; i += kBm3dThreads) {
        const int g = i >> 6, py = (i >> 3) & 7, px = i & 7, c = sel[g];
        float a = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) a = fmaf(c_bm_dct[u][py], P[g][u][px], a);
        const int oy = c / ncx, ox = c - oy * ncx;
        const int64_t o = (int64_t)k * H * W + (int64_t)(cy0 + oy + py) * W + cx0 + ox + px;
        const float kw = wgt * c_bm_kaiser[py] * c_bm_kaiser[px];
        atomicAdd(num + o, kw * a);
        atomicAdd(den + o, kw);
    }
}

__global__ void bm3d_div_kernel(const float* __restrict__ num, const float* __restrict__ den, int64_t n,
                                float* __restrict__ out) {
    griddep_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = num[i] / den[i];
}

}  // namespace

cudaError_t setup_bm3d_tables() {
    float d[8][8], kai[8];
    for (int kk = 0; kk < 8; ++kk)
        for (int nn = 0; nn < 8; ++nn)
            d[kk][nn] = (float)((kk == 0 ? std::sqrt(1.0 / 8) : std::sqrt(2.0 / 8)) *
                                std::cos(3.14159265358979323846 * (2 * nn + 1) * kk / 16.0));
    // Kaiser window, beta = 2: I0(beta sqrt(1 - (2i / 7 - 1)^2)) / I0(beta), I0 by its power series
    auto i0 = [](double z) {
        double sum = 1.0, term = 1.0;
        for (int q = 1; q < 40; ++q) {
            term *= (z / (2.0 * q)) * (z / (2.0 * q));
            sum += term;
        }
        return sum;
    };
    for (int i = 0; i < 8; ++i) {
        const double a = 2.0 * i / 7.0 - 1.0;
        kai[i] = (float)(i0(2.0 * std::sqrt(1.0 - a * a)) / i0(2.0));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_bm_dct, d, sizeof d);
    if (!e) e = cudaMemcpyToSymbol(c_bm_kaiser, kai, sizeof kai);
    return e;
}

int bm3d_refs(int n) { return (n - kN1) / kStep + 1 + ((n - kN1) % kStep ? 1 : 0); }

cudaError_t launch_bm3d(const float* in, float* out, int n_img, int H, int W, const float* sigma, float lambda,
                        float* num, float* den, cudaStream_t s) {
    const int64_t npx = (int64_t)n_img * H * W;
    cudaError_t e = cudaMemsetAsync(num, 0, npx * sizeof(float), s);
    if (!e) e = cudaMemsetAsync(den, 0, npx * sizeof(float), s);
    if (e) return e;
    const dim3 grid((unsigned)bm3d_refs(W), (unsigned)bm3d_refs(H), (unsigned)n_img);
    e = launch_pdl(bm3d_ht_kernel, grid, dim3(kBm3dThreads), 0, s, in, H, W, sigma, lambda, num, den);
    if (!e) {
        const int64_t want = (npx + 255) / 256;
        e = launch_pdl(bm3d_div_kernel, dim3((unsigned)(want < 152 * 16 ? want : 152 * 16)), dim3(256), 0, s,
                       (const float*)num, (const float*)den, npx, out);
    }
    return e;
}

}  // namespace abcs
