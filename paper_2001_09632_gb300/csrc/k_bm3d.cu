// BM3D, hard-thresholding step (ref. [22]): the plain denoiser the paper
// pairs with IDA besides DnCNN (Sec. VII).  One CTA per reference patch
// (8 x 8, every third position plus the last row / column):
//   - the 46 x 46 neighbourhood (reference +- 19 positions) in shared memory;
//   - distances d = ||P_ref - P||^2 / 64 of every candidate position;
//   - the group: the reference, then the candidates with d <= tau ordered by
//     (d, row, column), n = the largest power of two <= min(16, count),
//     chosen by repeated block-wide minimum of 64-bit keys (d's bits, index);
//   - 2D DCT of each patch, orthonormal Haar along the group, hard threshold
//     at lambda sigma (the group's 3D DC kept), count, inverses;
//   - aggregation of w K P (w = 1 / kept, K the 8 x 8 Kaiser window) and of
//     w K into numerator / denominator planes (atomic adds).
// A second kernel divides.  tau = 2500 for sigma <= 40, else 5000.
#include <cmath>

#include "abcs_common.cuh"

namespace abcs {

namespace {

constexpr int kN1 = 8, kN2 = 16, kHalf = 19, kStep = 3;
constexpr int kWin = 2 * kHalf + kN1;          // 46: neighbourhood side
constexpr int kWinLd = kWin + 1;
constexpr int kMaxCand = (2 * kHalf + 1) * (2 * kHalf + 1);   // 1521
constexpr int kBm3dThreads = 256;

__constant__ float c_bm_dct[8][8];      // D[k][n], orthonormal DCT-II
__constant__ float c_bm_haar[5][16][16];  // orthonormal Haar of length 1, 2, 4, 8, 16
__constant__ float c_bm_kaiser[8];

ABCS_D unsigned long long bm_min(unsigned long long a, unsigned long long b) { return a < b ? a : b; }

// reference position j of a dimension of n pixels: 3 j, the last one n - 8
ABCS_D int bm_ref_pos(int j, int n) { return min(kStep * j, n - kN1); }

__global__ void __launch_bounds__(kBm3dThreads) bm3d_ht_kernel(const float* __restrict__ in, int H, int W,
                                                               const float* __restrict__ sigma, float lam,
                                                               float* __restrict__ num, float* __restrict__ den) {
    __shared__ float nb[kWin * kWinLd];
    __shared__ unsigned long long key[kMaxCand];
    __shared__ unsigned long long red[kBm3dThreads / 32];
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
    for (int i = t; i < nh * nw; i += kBm3dThreads) {
        const int r = i / nw, c = i - r * nw;
        nb[r * kWinLd + c] = __ldg(img + (int64_t)(cy0 + r) * W + cx0 + c);
    }
    __syncthreads();
    const int ry = y - cy0, rx = x - cx0, ncand = ncy * ncx, ref = ry * ncx + rx;
    // keys: the reference 0, others (bits of d) << 32 | (index + 1); beyond tau: max
    for (int c = t; c < ncand; c += kBm3dThreads) {
        const int oy = c / ncx, ox = c - oy * ncx;
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < kN1; ++i)
#pragma unroll
            for (int j = 0; j < kN1; ++j) {
                const float d = nb[(ry + i) * kWinLd + rx + j] - nb[(oy + i) * kWinLd + ox + j];
                acc = fmaf(d, d, acc);
            }
        const float d = acc * (1.f / 64.f);
        unsigned long long kk = ~0ull;
        if (c == ref) kk = 0ull;
        else if (d <= tau) kk = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)(c + 1);
        key[c] = kk;
    }
    __syncthreads();
    // group size: the largest power of two <= min(16, candidates within tau)
    {
        int cnt = 0;
        for (int c = t; c < ncand; c += kBm3dThreads) cnt += key[c] != ~0ull;
        cnt = warp_sum(cnt);
        if (lane == 0) red[warp] = (unsigned long long)cnt;
        __syncthreads();
        if (t == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < kBm3dThreads / 32; ++w) tot += red[w];
            const int lim = tot < (unsigned long long)kN2 ? (int)tot : kN2;
            int n = 1;
            while (2 * n <= lim) n *= 2;
            s_cnt = n;
        }
        __syncthreads();
    }
    const int n = s_cnt;
    for (int g = 0; g < n; ++g) {                 // repeated minimum: the n smallest keys in order
        unsigned long long m = ~0ull;
        for (int c = t; c < ncand; c += kBm3dThreads) m = bm_min(m, key[c]);
#pragma unroll
        for (int o = 16; o; o >>= 1) m = bm_min(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red[warp] = m;
        __syncthreads();
        if (t == 0) {
            unsigned long long b = red[0];
            for (int w = 1; w < kBm3dThreads / 32; ++w) b = bm_min(b, red[w]);
            const int c = b == 0ull ? ref : (int)(b & 0xFFFFFFFFull) - 1;
            sel[g] = c;
            key[c] = ~0ull;
        }
        __syncthreads();
    }
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
    // Haar along the group per coefficient (u, v), threshold, count, inverse Haar
    const int ln = 31 - __clz(n);
    int kept = 0;
    if (t < 64) {
        const int u = t >> 3, v = t & 7;
        float z[kN2], w3[kN2];
        for (int g = 0; g < n; ++g) z[g] = P[g][u][v];
        for (int q = 0; q < n; ++q) {
            float a = 0.f;
            for (int g = 0; g < n; ++g) a = fmaf(c_bm_haar[ln][q][g], z[g], a);
            const bool keep = fabsf(a) > thr || (q == 0 && t == 0);
            w3[q] = keep ? a : 0.f;
            kept += keep;
        }
        for (int g = 0; g < n; ++g) {
            float a = 0.f;
            for (int q = 0; q < n; ++q) a = fmaf(c_bm_haar[ln][q][g], w3[q], a);
            T[g][u][v] = a;
        }
    }
    kept = warp_sum(kept);
    if (lane == 0) red[warp] = (unsigned long long)kept;
    __syncthreads();
    const float wgt = 1.f / (float)(red[0] + red[1]);          // threads 0..63 are warps 0 and 1
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
    float d[8][8], haar[5][16][16] = {}, kai[8];
    for (int kk = 0; kk < 8; ++kk)
        for (int nn = 0; nn < 8; ++nn)
            d[kk][nn] = (float)((kk == 0 ? std::sqrt(1.0 / 8) : std::sqrt(2.0 / 8)) *
                                std::cos(3.14159265358979323846 * (2 * nn + 1) * kk / 16.0));
    // orthonormal Haar by doubling: H_2n = [H_n (x) (1, 1); I_n (x) (1, -1)] / sqrt 2
    double Hm[16][16] = {{1.0}};
    int m = 1;
    haar[0][0][0] = 1.f;
    for (int l = 1; l < 5; ++l) {
        double Hn[16][16] = {};
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                Hn[i][2 * j] = Hm[i][j] / std::sqrt(2.0);
                Hn[i][2 * j + 1] = Hm[i][j] / std::sqrt(2.0);
            }
        for (int i = 0; i < m; ++i) {
            Hn[m + i][2 * i] = 1.0 / std::sqrt(2.0);
            Hn[m + i][2 * i + 1] = -1.0 / std::sqrt(2.0);
        }
        m *= 2;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                Hm[i][j] = Hn[i][j];
                haar[l][i][j] = (float)Hn[i][j];
            }
    }
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
    if (!e) e = cudaMemcpyToSymbol(c_bm_haar, haar, sizeof haar);
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
