// Quality of reconstructions against the clean images, the two measures the
// paper reports (PSNR and SSIM, Tables 3, 6, 7): per image, with x clipped to
// [0, 255] (no clipping happens anywhere else in the library),
//   PSNR = 10 log10(255^2 / MSE),
//   SSIM = mean over the valid region of the map of Wang et al. (ref. [18]):
//          11 x 11 Gaussian window (sigma 1.5), C1 = (0.01 L)^2,
//          C2 = (0.03 L)^2, L = 255.
// The local moments are formed from values centred at 128 (the window's
// second moments minus the products of its centred means), which keeps FP32
// cancellation small; sums over an image are per-CTA FP32 partials added in
// FP64 in a fixed order.
#include <cmath>

#include "abcs_common.cuh"

namespace abcs {

namespace {

constexpr int kQK = 11;                          // window size
constexpr int kQT = 32;                          // output tile (valid-region positions) per CTA side
constexpr int kQI = kQT + kQK - 1;               // input tile side
__constant__ float c_gauss[kQK];                 // normalised 1D Gaussian, sigma 1.5

// MSE partials: grid (chunks, images)
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ x, const uint8_t* __restrict__ ref,
                                                  int H, int W, int64_t pitch, int64_t stride,
                                                  double* __restrict__ part) {
    __shared__ double sh[32];
    griddep_wait();
    const int k = blockIdx.y;
    const int64_t npx = (int64_t)H * W;
    const float* xk = x + (int64_t)k * npx;
    const uint8_t* rk = ref + (int64_t)k * stride;
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), xx = (int)(i - (int64_t)y * W);
        const float d = fminf(fmaxf(__ldg(xk + i), 0.f), 255.f) - (float)__ldg(rk + (int64_t)y * pitch + xx);
        s = fmaf(d, d, s);
    }
    const double t = block_sum((double)s, sh);
    if (threadIdx.x == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = t;
}

// SSIM partials: grid (tiles x, tiles y, images); the CTA's 32 x 32 map
// positions need a 42 x 42 input tile
__global__ void __launch_bounds__(256) ssim_kernel(const float* __restrict__ x, const uint8_t* __restrict__ ref,
                                                   int H, int W, int64_t pitch, int64_t stride,
                                                   double* __restrict__ part) {
    __shared__ float ta[kQI][kQI + 1], tb[kQI][kQI + 1];
    __shared__ float hs[5][kQI][kQT + 1];        // horizontal pass: mu_a, mu_b, a'a', b'b', a'b' (centred)
    __shared__ double sh[32];
    griddep_wait();
    const int k = blockIdx.z;
    const int oh = H - kQK + 1, ow = W - kQK + 1;
    const int y0 = blockIdx.y * kQT, x0 = blockIdx.x * kQT;
    const float* xk = x + (int64_t)k * H * W;
    const uint8_t* rk = ref + (int64_t)k * stride;
    for (int i = threadIdx.x; i < kQI * kQI; i += blockDim.x) {
        const int r = i / kQI, c = i % kQI;
        const int yy = min(y0 + r, H - 1), xx = min(x0 + c, W - 1);   // past the edge: clamped, never used
        ta[r][c] = fminf(fmaxf(__ldg(xk + (int64_t)yy * W + xx), 0.f), 255.f);
        tb[r][c] = (float)__ldg(rk + (int64_t)yy * pitch + xx);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kQI * kQT; i += blockDim.x) {
        const int r = i / kQT, c = i % kQT;
        float ma = 0.f, mb = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int d = 0; d < kQK; ++d) {
            const float w = c_gauss[d], a = ta[r][c + d], b = tb[r][c + d];
            const float ac = a - 128.f, bc = b - 128.f;
            ma = fmaf(w, a, ma);
            mb = fmaf(w, b, mb);
            aa = fmaf(w, ac * ac, aa);
            bb = fmaf(w, bc * bc, bb);
            ab = fmaf(w, ac * bc, ab);
        }
        hs[0][r][c] = ma; hs[1][r][c] = mb; hs[2][r][c] = aa; hs[3][r][c] = bb; hs[4][r][c] = ab;
    }
    __syncthreads();
    const float C1 = 6.5025f, C2 = 58.5225f;     // (0.01 * 255)^2, (0.03 * 255)^2
    float s = 0.f;
    for (int i = threadIdx.x; i < kQT * kQT; i += blockDim.x) {
        const int r = i / kQT, c = i % kQT;
        if (y0 + r >= oh || x0 + c >= ow) continue;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int d = 0; d < kQK; ++d) {
            const float w = c_gauss[d];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = fmaf(w, hs[q][r + d][c], m[q]);
        }
        const float mac = m[0] - 128.f, mbc = m[1] - 128.f;
        const float saa = m[2] - mac * mac, sbb = m[3] - mbc * mbc, sab = m[4] - mac * mbc;
        const float num = (2.f * m[0] * m[1] + C1) * (2.f * sab + C2);
        const float den = (m[0] * m[0] + m[1] * m[1] + C1) * (saa + sbb + C2);
        s += num / den;
    }
    const double t = block_sum((double)s, sh);
    if (threadIdx.x == 0) part[((int64_t)k * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

// one warp per image: partials in a fixed order
__global__ void quality_finish_kernel(const double* __restrict__ mse_part, int n_mse,
                                      const double* __restrict__ ssim_part, int n_ssim, int64_t npx,
                                      int64_t nvalid, double* __restrict__ psnr, double* __restrict__ ssim) {
    griddep_wait();
    const int k = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < n_mse; j += 32) a += mse_part[(int64_t)k * n_mse + j];
    for (int j = threadIdx.x; j < n_ssim; j += 32) b += ssim_part[(int64_t)k * n_ssim + j];
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
        const double mse = a / (double)npx;
        psnr[k] = mse > 0.0 ? 10.0 * log10(255.0 * 255.0 / mse) : INFINITY;
        ssim[k] = b / (double)nvalid;
    }
}

}  // namespace

cudaError_t setup_quality_tables() {
    float g[kQK];
    double s = 0.0, v[kQK];
    for (int i = 0; i < kQK; ++i) {
        const double t = i - (kQK - 1) / 2.0;
        v[i] = std::exp(-t * t / (2.0 * 1.5 * 1.5));
        s += v[i];
    }
    for (int i = 0; i < kQK; ++i) g[i] = (float)(v[i] / s);
    return cudaMemcpyToSymbol(c_gauss, g, sizeof g);
}

size_t quality_ws_bytes(int n_img, int H, int W) {
    const int tx = (W - kQK + 1 + kQT - 1) / kQT, ty = (H - kQK + 1 + kQT - 1) / kQT;
    return ((size_t)n_img * (64 + (size_t)tx * ty)) * sizeof(double);
}

cudaError_t launch_psnr_ssim(const float* x, const uint8_t* ref, int n_img, int H, int W, int64_t pitch,
                             int64_t stride, double* psnr, double* ssim, void* ws, cudaStream_t s) {
    const int oh = H - kQK + 1, ow = W - kQK + 1;
    const int tx = (ow + kQT - 1) / kQT, ty = (oh + kQT - 1) / kQT;
    double* mse_part = static_cast<double*>(ws);
    double* ssim_part = mse_part + (size_t)n_img * 64;
    cudaError_t e = launch_pdl(mse_kernel, dim3(64, n_img), dim3(256), 0, s, x, ref, H, W, pitch, stride, mse_part);
    if (!e)
        e = launch_pdl(ssim_kernel, dim3(tx, ty, n_img), dim3(256), 0, s, x, ref, H, W, pitch, stride, ssim_part);
    if (!e)
        e = launch_pdl(quality_finish_kernel, dim3(n_img), dim3(32), 0, s, (const double*)mse_part, 64,
                       (const double*)ssim_part, tx * ty, (int64_t)H * W, (int64_t)oh * ow, psnr, ssim);
    return e;
}

}  // namespace abcs
